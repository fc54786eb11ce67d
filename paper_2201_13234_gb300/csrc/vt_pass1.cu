// vt_pass1.cu -- first labelling pass.
//
// The paper's two-step method (Algorithms 2 and 3) settles a voxel from the
// sites whose investigation ball contains it, because the winner must be
// among the sites whose score there is at most a score some site already
// achieves.  Here one CTA takes a brick of voxels and turns that around:
//  1. it stages into shared memory the sites of every bin within a margin M
//     of the brick (all threads load cooperatively);
//  2. UB = the smallest upper bound, over the brick, of a staged site's score:
//     every voxel's best score is at most UB.  A site farther than M_UB from
//     the brick along some axis scores more than UB everywhere on it
//     (M_UB = ceil(sqrt(UB)) + 1 in f-units for Voronoi and Laguerre; the
//     fastest growth over UB plus the earliest birth for Johnson-Mehl).  If
//     M_UB > M the region is restaged with margin M_UB, so that in the end
//     the staged sites hold every possible winner and every voxel is
//     certified by construction;
//  3. each warp takes one tile (warp box) of the brick: the images of staged
//     sites whose lower bound over the tile is at most U0 = the tile's
//     smallest upper bound form its list; if one site's upper bound is below
//     every other site's lower bound the tile is that site (uniform tile);
//  4. otherwise the warp scores the entry with the smallest upper bound, then
//     the others, skipping an entry whose lower bound exceeds the running
//     bound U (the largest best score of the tile so far).  FP32 mode keeps
//     each voxel's two smallest packed (score, index) keys and rescores
//     exactly every voxel whose two keys lie within the error bound; exact
//     mode compares (int64 / IEEE double score, id) directly.
// A brick whose staging or lists do not fit (dense clusters) is left to the
// second pass.
#include "vt_device.cuh"

namespace vt {

constexpr int kP1Warps = 4;       // one warp per tile of the brick (WX x WY x WZ)
constexpr int kP1Threads = 32 * kP1Warps;
constexpr int kP1MinBlocks = 5;   // register budget: 5 CTAs (20 warps) per SM
constexpr int kP1Cap = 512;       // staged sites per brick
constexpr int kP1Cl = 256;        // staged sites kept after culling
constexpr int kP1MaxRows = 256;   // bin rows of a staged region
constexpr int kL1 = 128;          // list entries per warp
constexpr unsigned kK1 = 0x7Fu;   // 7 index bits in a key: truncation < 2^-16 relative

struct P1Count {
  unsigned long long cand, resc, unif, rest;
  int overflow;
};

// Put a brick on the second-pass list (each brick once), with the margin M
// (fixed point) of a region that holds every possible winner of the brick
// when UB (an upper bound, f-units, of every voxel's best score) is finite.
__device__ __forceinline__ void defer_brick(const Work& wk, int64_t b, int64_t M, float UB) {
  if (atomicExch(&wk.p2_flag[b], 1) == 0) {
    const unsigned long long slot = atomicAdd(&wk.cnt[C_P2], 1ull);
    wk.p2_list[3 * slot] = (int32_t)b;
    wk.p2_list[3 * slot + 1] = (int32_t)(M < 0x7FFFFFFF ? M : 0x7FFFFFFF);
    wk.p2_list[3 * slot + 2] = __float_as_int(UB);
    atomicAdd(&wk.cnt[C_DEFER], 1ull);
  }
}

// Region margin (fixed point) beyond which every site scores more than UB
// over the brick: V/L F_out >= D_out >= (M + 1)^2 > UB needs M >= sqrt(UB);
// JM F_out >= (M + 1) / (512 vmax) (1 - 2^-51) - absf > UB.
template <int KIND>
__device__ __forceinline__ int64_t margin_for(float UB, const FUnits& U) {
  if (!(UB < kInf)) return (int64_t)1 << 40;
  const float x = KIND == KJ ? __fmul_ru(__fmul_ru(__fadd_ru(UB, U.absf), 512.0f),
                                         __fmul_ru(U.vmax_ru, 1.0f + 0x1p-18f))
                             : __fsqrt_ru(UB);
  return x < 1e12f ? __float2ll_ru(x) + 1 : ((int64_t)1 << 40);
}

// Upper bound (f-units) of the largest best score of the tile so far, from
// the best keys (the key order is the value order; the index bits are
// cleared after the maximum).
template <class C, unsigned IDXMASK>
__device__ __forceinline__ float u_f32(const Lane<C>& G, const unsigned (&k1)[C::NV], float absf) {
  constexpr unsigned kAll = C::NV >= 32 ? 0xFFFFFFFFu : ((1u << C::NV) - 1);
  unsigned m = 0;
  if (G.vmask == kAll) {
#pragma unroll
    for (int v = 0; v < C::NV; v++) m = max(m, k1[v]);
  } else {
#pragma unroll
    for (int v = 0; v < C::NV; v++)
      if (G.vmask & (1u << v)) m = max(m, k1[v]);
  }
  m = __reduce_max_sync(0xffffffffu, m) & ~IDXMASK;
  if (m >= 0x7f800000u) return kInf;
  return __fmaf_ru(__uint_as_float(m), 1.0f + 0x1p-14f, 2.0f * absf);
}

template <int KIND, class C>
__device__ __forceinline__ float u_exact(const Lane<C>& G, const long long (&bs)[C::NV],
                                         const double (&ba)[C::NV], const FUnits& U) {
  float m = -kInf;
#pragma unroll
  for (int v = 0; v < C::NV; v++)
    if (G.vmask & (1u << v)) m = fmaxf(m, exact_to_f_ru<KIND>(bs[v], ba[v], U));
  return warp_max(m);
}

// Voronoi and Laguerre: F_r(v) - F_s(v) = 2 v.(q_s - q_r) + (c_r - c_s) with
// c = |q|^2 + a (kept in Entry::b) is linear in v, so its minimum over the
// tile [0, h] is at a corner.  True when list entry r scores more than entry
// s at every voxel of the tile: r can then never win there.  The terms are
// FP32 roundings of exact integers; the 2^-18 relative allowance covers them.
__device__ __forceinline__ bool dominated(const Entry& r, const Entry& s, float hx, float hy,
                                          float hz) {
  const float tx = 2.0f * (s.qx - r.qx) * hx;
  const float ty = 2.0f * (s.qy - r.qy) * hy;
  const float tz = 2.0f * (s.qz - r.qz) * hz;
  const float m = (r.b - s.b) + fminf(0.f, tx) + fminf(0.f, ty) + fminf(0.f, tz);
  const float mag = r.b + s.b + fabsf(tx) + fabsf(ty) + fabsf(tz);
  return m > __fmaf_ru(mag, 0x1p-18f, 64.0f);
}

// Relative width of the rescoring band: the packed key truncates F by less
// than 2^-16 (7 index bits) and the FP32 evaluation errs by at most 2^-19
// relative (plus 2 absf), so (1 + 2^-16)(1 + 2^-19)/(1 - 2^-19) < 1 + 2^-15:
// if a voxel's second key is above f1 (1 + 2^-15) + 4 absf, its first key's
// site is the exact winner.
constexpr float kBand = 0x1p-15f;

// FP32 score of a list entry at one voxel (centre c relative to the warp origin).
template <int KIND>
__device__ __forceinline__ float f32_at(const Entry& e, float cx, float cy, float cz) {
  const float dx = cx - e.qx, dy = cy - e.qy, dz = cz - e.qz;
  if (KIND == KJ) return fmaf(sqrt_approx(fmaf(dx, dx, fmaf(dz, dz, dy * dy))), e.b, e.a);
  return fmaf(dx, dx, fmaf(dz, dz, fmaf(dy, dy, e.a)));
}

// Exact winner at one voxel, found by the whole warp: lanes split the list
// entries that could still win (lower bound <= Ub), screen them in FP32 at the
// voxel, score exactly (int64 / IEEE double) those within the band of the
// smallest FP32 score, and reduce (score, id) lexicographically.
template <int KIND>
__device__ __forceinline__ int rescore_warp(const Work& wk, const Entry* list, int len, float Ub,
                                         float cx, float cy, float cz, float absf) {
  const int lane = threadIdx.x & 31;
  float fmin = kInf;
  for (int e = lane; e < len; e += 32) {
    const Entry x = list[e];
    if (x.lo <= Ub) fmin = fminf(fmin, f32_at<KIND>(x, cx, cy, cz));
  }
  fmin = warp_min(fmin);
  const float thr = __fmaf_ru(fmin, 1.0f + 2.0f * kBand, 4.0f * absf);
  long long bs = 0x7FFFFFFFFFFFFFFFll;
  double ba = kInf;
  int bid = 0x7FFFFFFF;
  const int icx = (int)cx, icy = (int)cy, icz = (int)cz;
  for (int e = lane; e < len; e += 32) {
    const Entry x = list[e];
    if (x.lo > Ub || f32_at<KIND>(x, cx, cy, cz) > thr) continue;
    const int dx = icx - __float2int_rn(x.qx);
    const int dy = icy - __float2int_rn(x.qy);
    const int dz = icz - __float2int_rn(x.qz);
    const long long D = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
    const ExactSite xs = exact_site<KIND>(wk, x.src);
    if (KIND == KJ) {
      const double a = __dadd_rn(xs.t, __ddiv_rn(__dsqrt_rn((double)D), xs.den));
      if (a < ba || (a == ba && x.id < bid)) { ba = a; bid = x.id; }
    } else {
      const long long sc = KIND == KL ? D - xs.w : D;
      if (sc < bs || (sc == bs && x.id < bid)) { bs = sc; bid = x.id; }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const int oid = __shfl_xor_sync(0xffffffffu, bid, o);
    if (KIND == KJ) {
      const double oa = __shfl_xor_sync(0xffffffffu, ba, o);
      if (oa < ba || (oa == ba && oid < bid)) { ba = oa; bid = oid; }
    } else {
      const long long os = __shfl_xor_sync(0xffffffffu, bs, o);
      if (os < bs || (os == bs && oid < bid)) { bs = os; bid = oid; }
    }
  }
  return bid;
}

// A staged candidate: one periodic image of a site, at exact float
// coordinates relative to the first voxel centre of the brick, with the
// site's FP32 data, its ids and the lower bound of its F over the brick.
struct Staged {
  float qx, qy, qz, a;
  float b;
  int id, src;
  float lob;
};

// Shared memory of a first-pass CTA.  The staged images are needed only until
// they are culled into cl[], so the warps' candidate lists reuse their space.
struct P1Smem {
  union {
    Staged st[kP1Cap];
    Entry list[kP1Warps][kL1];
  } u;
  Staged cl[kP1Cl];
  int seg_src[2 * kP1MaxRows];  // per bin row: start of its one or two site runs
  int seg_off[kP1MaxRows];      // per bin row: length of its first run
  int roff[kP1MaxRows + 1];     // per bin row: offset of its sites in the staged list
  unsigned long long tkey[kP1Warps];  // per tile: smallest (upper bound bits << 32 | slot)
  unsigned long long tkw[kP1Warps][kP1Warps];  // the same, per staging warp
  int bpos[kP1Warps];                 // per tile: position of that image in cl[]
  int ccount[kP1Cap / 32];            // kept images per chunk of 32 staged ones
  int wtot[kP1Warps];
  Region R;
  int nstaged, ncull, overflow, next;
};
static_assert(sizeof(Staged) * kP1Cap == sizeof(Entry) * kP1Warps * kL1, "list overlay");

// Exclusive scan of a[0..n) in shared memory (n <= 8 * kP1Threads); returns
// the total.  Every thread of the CTA calls it.
__device__ int p1_block_scan(int* a, int n, int* wtot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + kP1Threads - 1) / kP1Threads;
  const int beg = min(tid * per, n), end = min(beg + per, n);
  int s = 0;
  for (int i = beg; i < end; i++) s += a[i];
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[warp] = x;
  __syncthreads();
  int wp = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kP1Warps; w++) {
    if (w < warp) wp += wtot[w];
    total += wtot[w];
  }
  int run = wp + x - s;
  for (int i = beg; i < end; i++) {
    int v = a[i];
    a[i] = run;
    run += v;
  }
  __syncthreads();
  return total;
}

// Tile t of the brick whose first voxel is (x0, y0, z0): offset of its first
// centre from the brick's first centre and its extent clipped to the grid
// (fixed point, exact floats).  False when the tile lies outside the grid.
// The warp that labels tile t derives the same numbers from its lane setup.
template <class C>
__device__ __forceinline__ bool tile_geom(const Inst& I, int t, int x0, int y0, int z0, float& ox,
                                          float& oy, float& oz, float& hx, float& hy,
                                          float& hz) {
  const int tx = t % C::WX, ty = (t / C::WX) % C::WY, tz = t / (C::WX * C::WY);
  const int ax = x0 + tx * C::BXW, ay = y0 + ty * C::BYW, az = z0 + tz * C::BZW;
  ox = (float)(kQ * tx * C::BXW);
  oy = (float)(kQ * ty * C::BYW);
  oz = (float)(kQ * tz * C::BZW);
  hx = (float)(kQ * (min(C::BXW, I.n[0] - ax) - 1));
  hy = (float)(kQ * (min(C::BYW, I.n[1] - ay) - 1));
  hz = (float)(kQ * (min(C::BZW, I.n[2] - az) - 1));
  return ax < I.n[0] && ay < I.n[1] && az < I.n[2];
}

// Stage the sites of region R (every bin once) into shared memory, each as
// the periodic image(s) that are nearest for some voxel of the brick box
// [ob, ob + hb] (usually one; more only when the brick reaches past half a
// period from a site).  Each image carries its lower bound over the brick;
// per tile, S.tkey keeps the smallest upper bound over the tile among the
// staged images, with that image's slot.  Thread t copies a contiguous run of
// the flattened site list (one search for its first bin row, then a forward
// walk), so its loads are independent.  On return S.nstaged holds the count
// (at most kP1Cap: when the region holds more, S.overflow is set and a prefix
// is staged, still enough for upper bounds).  Every thread calls it.
template <int KIND, class C>
__device__ void p1_stage(const Work& wk, const Inst& I, const Region& R, const int* ob,
                         const int* hb, int x0, int y0, int z0, const FUnits& U, P1Smem& S) {
  const int tid = threadIdx.x;
  const int rows = (R.bhi[1] - R.blo[1] + 1) * (R.bhi[2] - R.blo[2] + 1);
  if (rows > kP1MaxRows) {
    if (tid == 0) S.overflow = 1;
    __syncthreads();
    return;
  }
  for (int r = tid; r < rows; r += kP1Threads) {
    int s0, l0, s1, l1;
    row_runs(wk, I, R, r, s0, l0, s1, l1);
    S.seg_src[2 * r] = s0;
    S.seg_src[2 * r + 1] = s1;
    S.seg_off[r] = l0;
    S.roff[r] = l0 + l1;
  }
  __syncthreads();
  const int grand = p1_block_scan(S.roff, rows, S.wtot);
  const int total = grand < kP1Cap ? grand : kP1Cap;
  if (tid == 0) {
    S.roff[rows] = grand;
    S.next = total;
    if (grand > kP1Cap) S.overflow = 1;
  }
  __syncthreads();
  unsigned long long tk[kP1Warps];
#pragma unroll
  for (int t = 0; t < kP1Warps; t++) tk[t] = ~0ull;
  const float hbx = (float)hb[0], hby = (float)hb[1], hbz = (float)hb[2];
  const int per_t = (total + kP1Threads - 1) / kP1Threads;
  const int beg = tid * per_t, end = min(beg + per_t, total);
  if (beg < end) {
    int lo = 0, hi = rows - 1;  // last row starting at or before beg
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (S.roff[mid] <= beg) lo = mid; else hi = mid - 1;
    }
    int r = lo;
    for (int i = beg; i < end; i++) {
      while (i >= S.roff[r + 1]) r++;
      const int k = i - S.roff[r], l0 = S.seg_off[r];
      const int src = k < l0 ? S.seg_src[2 * r] + k : S.seg_src[2 * r + 1] + (k - l0);
      const int4 p = wk.spos[src];
      const float2 fa = KIND == KV ? make_float2(0.f, 0.f) : wk.sfa[src];
      const int pq[3] = {p.x, p.y, p.z};
      int q[3], ilo[3], cnt[3], n = 1;
#pragma unroll
      for (int a = 0; a < 3; a++) {
        int x = pq[a] - ob[a];
        ilo[a] = 0;
        cnt[a] = 1;
        if (a < I.nd && I.per[a]) {
          const int L = I.L[a], hL = L >> 1;
          const int d = (hb[a] >> 1) - x;
          if (d >= hL) x += L; else if (d < -hL) x -= L;
          const bool minus = -x < -hL, plus = hb[a] - x >= hL;
          ilo[a] = minus ? -1 : 0;
          cnt[a] = 1 + (int)minus + (int)plus;
        }
        q[a] = x;
        n *= cnt[a];
      }
      for (int j = 0; j < n; j++) {
        int slot = i;
        int c[3] = {q[0], q[1], q[2]};
        if (j > 0) {
          slot = atomicAdd(&S.next, 1);
          if (slot >= kP1Cap) break;
          int jj = j;
#pragma unroll
          for (int a = 0; a < 3; a++) {
            c[a] = q[a] + (ilo[a] + jj % cnt[a]) * I.L[a];
            jj /= cnt[a];
          }
        } else {
#pragma unroll
          for (int a = 0; a < 3; a++) c[a] = q[a] + ilo[a] * I.L[a];
        }
        Staged e;
        e.qx = (float)c[0]; e.qy = (float)c[1]; e.qz = (float)c[2];
        e.a = fa.x;
        e.b = fa.y;
        e.id = p.w;
        e.src = src;
        float blo, bhi;
        f_bounds_f<KIND>(e.qx, e.qy, e.qz, hbx, hby, hbz, e.a, e.b, U.absf, blo, bhi);
        e.lob = blo;
        S.u.st[slot] = e;
#pragma unroll
        for (int t = 0; t < kP1Warps; t++) {
          float ox, oy, oz, hx, hy, hz, tlo, thi;
          if (!tile_geom<C>(I, t, x0, y0, z0, ox, oy, oz, hx, hy, hz)) continue;
          f_bounds_f<KIND>(e.qx - ox, e.qy - oy, e.qz - oz, hx, hy, hz, e.a, e.b, U.absf, tlo,
                           thi);
          const unsigned long long key =
              ((unsigned long long)__float_as_uint(thi) << 32) | (unsigned)slot;
          tk[t] = tk[t] < key ? tk[t] : key;
        }
      }
    }
  }
  // per tile: warp minimum of the keys (upper bounds are non-negative floats,
  // whose bit patterns order like their values); thread t then takes the
  // minimum over the warps for tile t
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int t = 0; t < kP1Warps; t++) {
    const unsigned hk = (unsigned)(tk[t] >> 32);
    const unsigned h = __reduce_min_sync(0xffffffffu, hk);
    const unsigned slot = __reduce_min_sync(0xffffffffu, hk == h ? (unsigned)tk[t] : ~0u);
    if (lane == 0) S.tkw[warp][t] = ((unsigned long long)h << 32) | slot;
  }
  __syncthreads();
  if (tid < kP1Warps) {
    unsigned long long m = S.tkw[0][tid];
#pragma unroll
    for (int w = 1; w < kP1Warps; w++) m = S.tkw[w][tid] < m ? S.tkw[w][tid] : m;
    S.tkey[tid] = m;
  }
  if (tid == 0) {
    if (S.next > kP1Cap) S.overflow = 1;
    S.nstaged = S.next < kP1Cap ? S.next : kP1Cap;
  }
  __syncthreads();
}

// Keep, in staging order, the staged images whose lower bound over the brick
// is at most UB (the others score more than some staged image everywhere on
// the brick), in S.cl; S.bpos[t] receives the new position of each tile's
// smallest-upper-bound image (which is always kept).  Returns the count kept
// (more than kP1Cl means that cl[] overflowed).  Every thread calls it.
__device__ int p1_cull(P1Smem& S, int ns, float UB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nchunks = (ns + 31) >> 5;
  for (int c = warp; c < nchunks; c += kP1Warps) {
    const int i = (c << 5) + lane;
    const bool keep = i < ns && S.u.st[i].lob <= UB;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) S.ccount[c] = __popc(bal);
  }
  __syncthreads();
  for (int c = warp; c < nchunks; c += kP1Warps) {
    int base = 0;
    for (int k = 0; k < c; k++) base += S.ccount[k];
    const int i = (c << 5) + lane;
    const bool keep = i < ns && S.u.st[i].lob <= UB;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int pos = base + __popc(bal & ((1u << lane) - 1));
    if (keep && pos < kP1Cl) {
      S.cl[pos] = S.u.st[i];
#pragma unroll
      for (int t = 0; t < kP1Warps; t++)
        if ((unsigned)i == (unsigned)S.tkey[t]) S.bpos[t] = pos;
    }
    if (c == nchunks - 1 && lane == 0) S.ncull = base + __popc(bal);
  }
  __syncthreads();
  return S.ncull;
}

// The list entry of culled image s for a tile whose first centre lies at
// (wx, wy, wz) from the brick's, with its lower and upper bound over the tile
// [0, h].  V/L keep c = |q|^2 + a in b (for the dominance test).
template <int KIND>
__device__ __forceinline__ Entry tile_entry(const Staged& s, float wx, float wy, float wz,
                                            float hx, float hy, float hz, float absf, float& hi) {
  Entry x;
  x.qx = s.qx - wx;
  x.qy = s.qy - wy;
  x.qz = s.qz - wz;
  x.a = s.a;
  x.b = KIND == KJ ? s.b : fmaf(x.qx, x.qx, fmaf(x.qy, x.qy, fmaf(x.qz, x.qz, s.a)));
  x.id = s.id;
  x.src = s.src;
  f_bounds_f<KIND>(x.qx, x.qy, x.qz, hx, hy, hz, s.a, s.b, absf, x.lo, hi);
  return x;
}

// One warp labels tile `warp` of the brick (first voxel (x0, y0, z0)) from the
// culled images; ob is the brick's first voxel centre.
//  - list: entry 0 is the image with the smallest upper bound U0 over the
//    tile; then, in one parallel pass, every image whose lower bound is at
//    most U0 and (V/L) that entry 0 does not dominate on the tile.  No other
//    image can win anywhere on the tile;
//  - if every listed image belongs to entry 0's site the tile is uniform;
//  - else entry 0 is scored, then the others in order, skipping an entry whose
//    lower bound exceeds the running bound U (the largest best score of the
//    tile so far).
template <int KIND, class C, int PREC>
__device__ void p1_warp(const Work& wk, const Inst& I, const FUnits& U, P1Smem& S, int x0, int y0,
                        int z0, const int* ob, P1Count& n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Lane<C> G;
  lane_setup_box<C>(I, x0, y0, z0, G);
  if (!G.active) return;
  Entry* list = S.u.list[warp];
  const int ncl = S.ncull;
  // tile origin relative to the brick origin, tile extent (exact floats)
  const float wx = (float)(G.ox - ob[0]), wy = (float)(G.oy - ob[1]), wz = (float)(G.oz - ob[2]);
  const float hx = (float)G.hx, hy = (float)G.hy, hz = (float)G.hz;
  const float U0 = __uint_as_float((unsigned)(S.tkey[warp] >> 32));
  const int bp = S.bpos[warp];
  float bhi;
  const Entry bx = tile_entry<KIND>(S.cl[bp], wx, wy, wz, hx, hy, hz, U.absf, bhi);
  if (lane == 0) list[0] = bx;
  int len = 1;
  bool other = false;
  for (int base = 0; base < ncl; base += 32) {
    const int i = base + lane;
    bool keep = false;
    Entry x;
    if (i < ncl && i != bp) {
      float hi;
      x = tile_entry<KIND>(S.cl[i], wx, wy, wz, hx, hy, hz, U.absf, hi);
      keep = x.lo <= U0;
      if (KIND != KJ && keep) keep = !dominated(x, bx, hx, hy, hz);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    other = other || __any_sync(0xffffffffu, keep && x.id != bx.id);
    const int pos = len + __popc(bal & ((1u << lane) - 1));
    if (keep && pos < kL1) list[pos] = x;
    len += __popc(bal);
  }
  __syncwarp();
  if (len > kL1) {
    n.overflow = 1;
    return;
  }
  if (!other) {
    store_uniform<C>(I, G, bx.id);
    n.unif++;
    return;
  }

  // scoring: entry 0 first
  int evals = 1;
  int lab[C::NV];
  if (PREC == P_F32) {
    unsigned k1[C::NV], k2[C::NV];
#pragma unroll
    for (int v = 0; v < C::NV; v++) k1[v] = k2[v] = 0xFFFFFFFFu;
    eval_f32<KIND, C, kK1>(bx, 0u, G, k1, k2);
    float Uc = fminf(U0, u_f32<C, kK1>(G, k1, U.absf));
#pragma unroll 1
    for (int e = 1; e < len; e++) {
      const Entry x = list[e];
      if (x.lo > Uc) continue;
      eval_f32<KIND, C, kK1>(x, (unsigned)e, G, k1, k2);
      ++evals;
      if (evals <= 3 || evals % 3 == 0) Uc = fminf(Uc, u_f32<C, kK1>(G, k1, U.absf));
    }
    unsigned near = 0;  // voxels of this lane whose two keys lie within the band
#pragma unroll
    for (int v = 0; v < C::NV; v++) {
      const float f1 = __uint_as_float(k1[v] & ~kK1);
      const float f2 = __uint_as_float(k2[v] & ~kK1);
      lab[v] = list[k1[v] & kK1].id;
      if (f2 <= __fmaf_ru(f1, 1.0f + kBand, 4.0f * U.absf)) near |= 1u << v;
    }
    near &= G.vmask;
    store_labels<C>(I, G, lab);
    // the warp rescores each flagged voxel in turn and its lane overwrites
    // that voxel's label (same thread as the tile store: program order holds)
    int nresc = 0;
    for (unsigned any = __ballot_sync(0xffffffffu, near != 0); any;
         any = __ballot_sync(0xffffffffu, near != 0)) {
      const int src = __ffs(any) - 1;
      const int v = __ffs(__shfl_sync(0xffffffffu, near, src)) - 1;
      if (lane == src) near &= near - 1;
      const int i = v & 3, j = (v >> 2) % C::MY, k = (v >> 2) / C::MY;
      const int sx = src % C::LX, sy = (src / C::LX) % C::LY, sz = src / (C::LX * C::LY);
      const float cx = (float)(kQ * (sx * C::MX + i));
      const float cy = (float)(kQ * (sy * C::MY + j));
      const float cz = (float)(kQ * (sz * C::MZ + k));
      const int id = rescore_warp<KIND>(wk, list, len, Uc, cx, cy, cz, U.absf);
      if (lane == src) I.labels[label_index(I, G.vx + i, G.vy + j, G.vz + k)] = id;
      nresc++;
    }
    if (lane == 0) n.resc += nresc;
  } else {
    long long bs[C::NV];
    double ba[C::NV];
#pragma unroll
    for (int v = 0; v < C::NV; v++) {
      bs[v] = 0x7FFFFFFFFFFFFFFFll;
      ba[v] = kInf;
      lab[v] = 0x7FFFFFFF;
    }
    eval_exact<KIND, C>(bx, exact_site<KIND>(wk, bx.src), G, bs, ba, lab);
    float Uc = fminf(U0, u_exact<KIND, C>(G, bs, ba, U));
#pragma unroll 1
    for (int e = 1; e < len; e++) {
      const Entry x = list[e];
      if (x.lo > Uc) continue;
      eval_exact<KIND, C>(x, exact_site<KIND>(wk, x.src), G, bs, ba, lab);
      ++evals;
      if (evals <= 3 || evals % 3 == 0) Uc = fminf(Uc, u_exact<KIND, C>(G, bs, ba, U));
    }
  }
  n.cand += (unsigned long long)evals * 32ull * C::NV;
  if (PREC != P_F32) store_labels<C>(I, G, lab);
}

// One CTA labels one brick (WX x WY x WZ tiles):
//  - stage the region of margin M: at first the plan's margin (in mean cell
//    radii) plus a tile's half-diagonal (and, for Laguerre, the largest
//    weight);
//  - U0(t) = smallest upper bound over tile t of a staged image's F, and
//    UB = max over the tiles of U0(t): every voxel's best is at most UB, and a
//    site farther than M_UB (from UB, as below) from the brick along some
//    axis has F > UB everywhere on it;
//  - if M_UB > M (or nothing was staged), restage with the larger margin;
//  - cull the images whose lower bound over the brick exceeds UB;
//  - each warp then labels its tile from the culled images.
template <int KIND, class C, int PREC>
__device__ void p1_brick(const Work& wk, const Inst& I, const FUnits& U, int64_t lb, P1Smem& S,
                         P1Count& n) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int bxi = (int)(lb % I.bricks[0]);
  const int64_t rr = lb / I.bricks[0];
  const int byi = (int)(rr % I.bricks[1]), bzi = (int)(rr / I.bricks[1]);
  const int x0 = bxi * C::BX, y0 = byi * C::BY, z0 = bzi * C::BZ;
  const int x1 = min(x0 + C::BX, I.n[0]) - 1, y1 = min(y0 + C::BY, I.n[1]) - 1,
            z1 = min(z0 + C::BZ, I.n[2]) - 1;
  const int ob[3] = {kQ * x0 + kQ / 2, kQ * y0 + kQ / 2, kQ * z0 + kQ / 2};
  const int hb[3] = {kQ * (x1 - x0), kQ * (y1 - y0), kQ * (z1 - z0)};
  const float hd = 0.5f * sqrtf((float)(C::BXW * C::BXW + C::BYW * C::BYW + C::BZW * C::BZW));
  float m0 = (float)kQ * ((float)I.margin + hd);
  if (KIND == KL) m0 = sqrtf(m0 * m0 + (float)U.wglob);
  int64_t M = (int64_t)m0 + 1;
  const int bwmax = max(I.bw[0], max(I.bw[1], I.bw[2]));
  float UB = kInf;
#pragma unroll 1
  for (int round = 0;; round++) {
    if (tid < 3) {  // one axis per thread
      const int c = tid == 0 ? ob[0] : tid == 1 ? ob[1] : ob[2];
      const int h = tid == 0 ? hb[0] : tid == 1 ? hb[1] : hb[2];
      make_region_axis(I, tid, c, c + h, M, S.R);
    }
    if (tid < kP1Warps) S.tkey[tid] = ~0ull;
    if (tid == 0) {
      S.nstaged = 0;
      S.overflow = 0;
    }
    __syncthreads();
    const Region& R = S.R;
    p1_stage<KIND, C>(wk, I, R, ob, hb, x0, y0, z0, U, S);
    const int ns = S.nstaged;
    const bool full = R.full[0] && R.full[1] && R.full[2];
    if (round == 1 && tid == 0) n.rest++;
    if (ns == 0) {
      if (S.overflow) {  // too many bin rows to stage: the second pass grows rings
        if (tid == 0) defer_brick(wk, I.brick_base + lb, M, kInf);
        return;
      }
      if (full) return;  // no valid site at all (the error word is set)
      M = 2 * M + (int64_t)kQ * bwmax;
      __syncthreads();
      continue;
    }
    UB = 0.f;
#pragma unroll
    for (int t = 0; t < kP1Warps; t++) {
      const unsigned long long k = S.tkey[t];
      if (k != ~0ull) UB = fmaxf(UB, __uint_as_float((unsigned)(k >> 32)));
    }
    const int64_t need = margin_for<KIND>(UB, U);
    if (S.overflow) {  // the second pass labels it from the certified margin
      if (tid == 0) defer_brick(wk, I.brick_base + lb, need, UB);
      return;
    }
    if (need <= M || full) break;
    M = need;
    __syncthreads();
  }
  // every possible winner of every voxel of the brick is staged
  if (p1_cull(S, S.nstaged, UB) > kP1Cl) {
    if (tid == 0) defer_brick(wk, I.brick_base + lb, M, UB);
    return;
  }
  const int wx = warp % C::WX, wy = (warp / C::WX) % C::WY, wz = warp / (C::WX * C::WY);
  p1_warp<KIND, C, PREC>(wk, I, U, S, x0 + wx * C::BXW, y0 + wy * C::BYW, z0 + wz * C::BZW, ob,
                         n);
  if (__syncthreads_or(n.overflow)) {
    if (tid == 0) defer_brick(wk, I.brick_base + lb, M, UB);
  }
  n.overflow = 0;
}

__device__ __forceinline__ void flush_counts(const Work& wk, const P1Count& n) {
  unsigned long long c = n.cand, r = n.resc, u = n.unif;
#pragma unroll
  for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicAdd(&wk.cnt[C_CAND], c);
    if (r) atomicAdd(&wk.cnt[C_RESCORED], r);
    if (u) atomicAdd(&wk.cnt[C_UNIFORM], u);
  }
  if (threadIdx.x == 0 && n.rest) atomicAdd(&wk.cnt[C_RESTAGE], n.rest);
}

template <int KIND, class C, int PREC>
__global__ void __launch_bounds__(kP1Threads, kP1MinBlocks)
    k_pass1(const Work wk, const __grid_constant__ Inst I) {
  __shared__ P1Smem S;
  if (wk.err[E_CODE]) return;
  P1Count n{0, 0, 0, 0, 0};
  const FUnits U = load_funits<KIND>(wk, 0);
  for (int64_t b = blockIdx.x; b < I.n_bricks; b += gridDim.x) {
    p1_brick<KIND, C, PREC>(wk, I, U, b, S, n);
    __syncthreads();
  }
  flush_counts(wk, n);
}

// One brick of a batch instance.  Not inlined: each of the six variants keeps
// its own register allocation instead of the union of all six.
template <int KIND, class C, int PREC>
__device__ __noinline__ void p1_brick_call(const Work& wk, const Inst& I, int ii, int64_t lb,
                                           P1Smem& S, P1Count& n) {
  p1_brick<KIND, C, PREC>(wk, I, load_funits<KIND>(wk, ii), lb, S, n);
}

template <int PREC>
__global__ void __launch_bounds__(kP1Threads, kP1MinBlocks) k_pass1_batch(const Work wk) {
  __shared__ P1Smem S;
  if (wk.err[E_CODE]) return;
  P1Count n{0, 0, 0, 0, 0};
  for (int64_t t = blockIdx.x; t < wk.total_bricks; t += gridDim.x) {
    const int ii = find_inst(wk.insts, wk.n_inst, t, [](const Inst& x) { return x.brick_base; });
    const Inst& I = wk.insts[ii];
    const int64_t lb = t - I.brick_base;
    if (I.nd == 3) {
      if (I.kind == KV) p1_brick_call<KV, Cfg3, PREC>(wk, I, ii, lb, S, n);
      else if (I.kind == KL) p1_brick_call<KL, Cfg3, PREC>(wk, I, ii, lb, S, n);
      else p1_brick_call<KJ, Cfg3, PREC>(wk, I, ii, lb, S, n);
    } else {
      if (I.kind == KV) p1_brick_call<KV, Cfg2, PREC>(wk, I, ii, lb, S, n);
      else if (I.kind == KL) p1_brick_call<KL, Cfg2, PREC>(wk, I, ii, lb, S, n);
      else p1_brick_call<KJ, Cfg2, PREC>(wk, I, ii, lb, S, n);
    }
    __syncthreads();
  }
  flush_counts(wk, n);
}

// ------------------------------------------------------------ host side

static int g_p1_blocks_per_sm[3][2][2];  // [kind][3D?][prec]
static int g_p1_batch_blocks_per_sm[2];

template <int KIND, class C, int PREC>
static cudaError_t occ_one(int& out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out, k_pass1<KIND, C, PREC>, kP1Threads,
                                                       0);
}

cudaError_t init_pass1() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  cudaError_t e;
#define VT_OCC(K, C3, C, P) \
  if ((e = occ_one<K, C, P>(g_p1_blocks_per_sm[K][C3][P])) != cudaSuccess) return e;
  VT_OCC(KV, 1, Cfg3, P_F32) VT_OCC(KV, 1, Cfg3, P_EXACT) VT_OCC(KV, 0, Cfg2, P_F32)
  VT_OCC(KV, 0, Cfg2, P_EXACT) VT_OCC(KL, 1, Cfg3, P_F32) VT_OCC(KL, 1, Cfg3, P_EXACT)
  VT_OCC(KL, 0, Cfg2, P_F32) VT_OCC(KL, 0, Cfg2, P_EXACT) VT_OCC(KJ, 1, Cfg3, P_F32)
  VT_OCC(KJ, 1, Cfg3, P_EXACT) VT_OCC(KJ, 0, Cfg2, P_F32) VT_OCC(KJ, 0, Cfg2, P_EXACT)
#undef VT_OCC
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_p1_batch_blocks_per_sm[0],
                                                         k_pass1_batch<P_F32>, kP1Threads, 0)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_p1_batch_blocks_per_sm[1],
                                                         k_pass1_batch<P_EXACT>, kP1Threads, 0)) !=
      cudaSuccess)
    return e;
  done = cudaSuccess;
  return done;
}

static unsigned p1_grid(int bps, int sms, int64_t bricks) {
  int64_t g = (int64_t)(bps > 0 ? bps : 1) * sms * 8;
  return (unsigned)(bricks < g ? (bricks > 0 ? bricks : 1) : g);
}

template <int KIND, class C>
static void launch_p1(const Work& wk, const Inst& I, int sms, cudaStream_t st) {
  const int c3 = C::MZ > 1 ? 1 : 0;
  if (I.precision == P_F32)
    k_pass1<KIND, C, P_F32><<<p1_grid(g_p1_blocks_per_sm[KIND][c3][P_F32], sms, I.n_bricks),
                              kP1Threads, 0, st>>>(wk, I);
  else
    k_pass1<KIND, C, P_EXACT><<<p1_grid(g_p1_blocks_per_sm[KIND][c3][P_EXACT], sms, I.n_bricks),
                                kP1Threads, 0, st>>>(wk, I);
}

cudaError_t launch_pass1(const Work& wk, const Inst& I, int sms, cudaStream_t st) {
  if (I.nd == 3) {
    if (I.kind == KV) launch_p1<KV, Cfg3>(wk, I, sms, st);
    else if (I.kind == KL) launch_p1<KL, Cfg3>(wk, I, sms, st);
    else launch_p1<KJ, Cfg3>(wk, I, sms, st);
  } else {
    if (I.kind == KV) launch_p1<KV, Cfg2>(wk, I, sms, st);
    else if (I.kind == KL) launch_p1<KL, Cfg2>(wk, I, sms, st);
    else launch_p1<KJ, Cfg2>(wk, I, sms, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_pass1_batch(const Work& wk, int prec, int sms, cudaStream_t st) {
  if (prec == P_F32)
    k_pass1_batch<P_F32><<<p1_grid(g_p1_batch_blocks_per_sm[0], sms, wk.total_bricks), kP1Threads,
                           0, st>>>(wk);
  else
    k_pass1_batch<P_EXACT><<<p1_grid(g_p1_batch_blocks_per_sm[1], sms, wk.total_bricks),
                             kP1Threads, 0, st>>>(wk);
  return cudaGetLastError();
}

}  // namespace vt
