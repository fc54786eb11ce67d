// vt_pass1.cu -- first labelling pass.
//
// The paper's two-step method (Algorithms 2 and 3) settles a voxel from the
// sites whose investigation ball contains it, because the winner must be
// among the sites whose score there is at most a score some site already
// achieves.  Here each brick of voxels gathers the sites that may win on it:
//  1. the sites of every bin within a margin M of the brick are staged into
//     shared memory, each as the periodic image(s) nearest to the brick;
//  2. U0(t) = the smallest upper bound over tile t of a staged image's score,
//     and UB = max over the tiles of U0(t): every voxel's best score is at
//     most UB.  A site farther than M_UB from the brick along some axis scores
//     more than UB everywhere on it (M_UB = ceil(sqrt(UB)) + 1 in f-units for
//     Voronoi and Laguerre; the fastest growth over UB plus the earliest birth
//     for Johnson-Mehl).  If M_UB > M the region is restaged with margin M_UB,
//     so that in the end the staged sites hold every possible winner and every
//     voxel is certified by construction; images whose lower bound over the
//     brick exceeds UB are culled;
//  3. each tile (warp box) builds its list: the image with the smallest upper
//     bound, then every image whose lower bound is at most U0 and (Voronoi,
//     Laguerre) that the first one does not dominate on the tile.  If every
//     listed image belongs to one site the tile is uniform;
//  4. otherwise the tile scores the first entry, then the others, skipping an
//     entry whose lower bound exceeds the running bound U (the largest best
//     score of the tile so far).  FP32 mode keeps each voxel's two smallest
//     packed (score, index) keys and rescores exactly every voxel whose two
//     keys lie within the error bound; exact mode compares (int64 / IEEE
//     double score, id) directly.
// Steps 1-2 (staging) and 3-4 (scoring) run as two kernels over chunks of
// bricks (k_stage, k_tiles: see the kernels' section below).  A brick whose
// staged images do not fit, or whose tiles its first region does not
// certify, is retried by a third kernel that culls while it stages and grows
// the region until the brick is certified (k_recull_warp, one warp per brick,
// staging then scoring); one whose lists still do not fit (dense clusters)
// is left to the second pass.
#include <cstring>

#include "vt_device.cuh"

namespace vt {

constexpr int kP1Cons = 4;        // tiles of a brick (WX x WY x WZ), one scoring warp each
constexpr int kP1St = 448;        // staged images per round
constexpr int kP1MaxRows = 256;   // bin rows of a staged region
constexpr int kL1 = 128;          // list entries per scoring warp
constexpr int kL1R = 256;         // lists of 256 entries: one more index bit per key
constexpr int kRL = 128;          // culling re-run: list entries per warp (longer lists in chunks)
static_assert(Cfg3::WX * Cfg3::WY * Cfg3::WZ == kP1Cons, "3D tiles per brick");
static_assert(Cfg3c::WX * Cfg3c::WY * Cfg3c::WZ == kP1Cons, "3D tiles per brick");
static_assert(Cfg2::WX * Cfg2::WY * Cfg2::WZ == kP1Cons, "2D tiles per brick");
static_assert(Cfg2c::WX * Cfg2c::WY * Cfg2c::WZ == kP1Cons, "2D tiles per brick");
static_assert(cfg_index<Cfg3>() == 0 && cfg_index<Cfg3c>() == 1 && cfg_index<Cfg2>() == 2 &&
                  cfg_index<Cfg2c>() == 3,
              "tile configuration indices");
static_assert(kDeferDone == kDeferStage + kP1Cons, "a listed brick is done when all its tiles are");

struct P1Count {
  unsigned long long cand, resc, unif, rest;
};

// Put a brick on the second-pass list (each brick once), with the margin M
// (fixed point) of a region that holds every possible winner of the brick
// when UB (an upper bound, f-units, of every voxel's best score) is finite.
// Its flag records why (kDeferStage: the staged images did not fit, which
// the culling re-run retries; kDeferList: anything else).
__device__ __forceinline__ bool defer_brick(const Work& wk, int64_t b, int64_t M, float UB,
                                            int why) {
  if (atomicCAS(&wk.p2_flag[b], 0, why) == 0) {
    const unsigned long long slot = atomicAdd(&wk.cnt[C_P2], 1ull);
    wk.p2_list[3 * slot] = (int32_t)b;
    wk.p2_list[3 * slot + 1] = (int32_t)(M < 0x7FFFFFFF ? M : 0x7FFFFFFF);
    wk.p2_list[3 * slot + 2] = __float_as_int(UB);
    atomicAdd(&wk.cnt[C_DEFER], 1ull);
    return true;
  }
  return false;
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

// The same for absolute-scale keys: the largest first key's value F + S,
// less S, plus the evaluation's error bound (2^-20 (F + S) + 2 absf).
template <class C>
__device__ __forceinline__ float u_f32q(const Lane<C>& G, const unsigned (&k1)[C::NV], float S,
                                        unsigned sb, float absf) {
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
  m = __reduce_max_sync(0xffffffffu, m);
  if (m == 0xFFFFFFFFu) return kInf;
  const float f = qkey_value(m, sb);
  return __fadd_ru(__fsub_ru(f, S), __fmaf_ru(f, 0x1p-20f, 2.0f * absf));
}

template <int KIND, class C>
__device__ __forceinline__ float u_exact(const Lane<C>& G, const long long (&bs)[C::NV],
                                         const double (&ba)[C::NV], const FUnits& U) {
  return warp_max(lane_max_exact_f_ru<KIND, C::NV>(G.vmask, bs, ba, U));
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

// Relative keys (the culling re-run's lists of 256; the scoring kernel's
// lists of 128 use the absolute-scale keys of eval_f32q): the packed key
// truncates F by less than 2^-16 (7 index bits) or 2^-15 (8 bits) and the
// FP32 evaluation errs by at most 2^-19 relative (plus 2 absf), so
// (1 + 2^-15)(1 + 2^-19)/(1 - 2^-19) < 1 + 2^-14: if a voxel's second key is
// above f1 (1 + band) + 4 absf, its first key's site is the exact winner.
// kBand: rescore_warp's screen keeps the entries within 1 + 2 kBand of the
// smallest plain FP32 score at the voxel (each errs by at most 2^-19).
constexpr float kBand = 0x1p-15f;
template <int LCAP>
struct ListKeys {
  static_assert(LCAP == 128 || LCAP == 256, "7 or 8 index bits per key");
  static constexpr unsigned mask = LCAP - 1;  // index bits of a packed key
  static constexpr float band = LCAP == 128 ? 0x1p-15f : 0x1p-14f;
};

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
template <int KIND, class GET>
__device__ __forceinline__ int rescore_core(const Work& wk, GET&& get, int len, float Ub, float cx,
                                            float cy, float cz, float absf) {
  const int lane = threadIdx.x & 31;
  float fmin = kInf;
  for (int e = lane; e < len; e += 32) {
    const Entry x = get(e);
    if (x.lo <= Ub) fmin = fminf(fmin, f32_at<KIND>(x, cx, cy, cz));
  }
  fmin = warp_min(fmin);
  const float thr = __fmaf_ru(fmin, 1.0f + 2.0f * kBand, 4.0f * absf);
  long long bs = 0x7FFFFFFFFFFFFFFFll;
  double ba = kInf;
  int bid = 0x7FFFFFFF;
  const int icx = (int)cx, icy = (int)cy, icz = (int)cz;
  for (int e = lane; e < len; e += 32) {
    const Entry x = get(e);
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

template <int KIND>
__device__ __forceinline__ int rescore_warp(const Work& wk, const Entry* list, int len, float Ub,
                                           float cx, float cy, float cz, float absf) {
  return rescore_core<KIND>(wk, [&](int e) { return list[e]; }, len, Ub, cx, cy, cz, absf);
}

// The same over every culled image of the brick (area st[0, n), the tile's
// first centre at (wx, wy, wz) from the brick's): a superset of any of the
// tile's lists, for tiles scored in chunks.
template <int KIND>
__device__ __noinline__ int rescore_area(const Work& wk, const Staged* st, int n, float wx,
                                         float wy, float wz, float cx, float cy, float cz,
                                         float absf) {
  return rescore_core<KIND>(
      wk,
      [&](int e) {
        const Staged& q = st[e];
        Entry x;
        x.qx = q.qx - wx;
        x.qy = q.qy - wy;
        x.qz = q.qz - wz;
        x.a = q.a;
        x.b = q.b;
        x.lo = 0.f;
        x.id = q.id;
        x.src = q.src;
        return x;
      },
      n, kInf, cx, cy, cz, absf);
}

// The same, out of line: Voronoi and Laguerre rescore rarely, and keeping
// the body out of the scoring loop shortens the code the SM fetches
// (1-2% on uniform sites); Johnson-Mehl rescores often enough that the call
// costs more (3%), so it keeps the inline form.
template <int KIND>
__device__ __noinline__ int rescore_warp_ool(const Work& wk, const Entry* list, int len, float Ub,
                                             float cx, float cy, float cz, float absf) {
  return rescore_warp<KIND>(wk, list, len, Ub, cx, cy, cz, absf);
}

// The staging area of one staging warp (the kept images fill st[0, ncull)
// once the brick is staged and culled).
template <int CAP>
struct P1AreaT {
  static constexpr int cap = CAP;
  Staged st[CAP];                    // staged images, then (culled in place) the kept ones
  unsigned long long tkey[kP1Cons];  // per tile: smallest (upper bound bits << 32 | slot)
  int bpos[kP1Cons];                 // per tile: position of that image after culling
  int ncull;
  int inst;                          // instance of the brick (batches)
  int skip;                          // the brick went to the second pass
  long long brick;                   // brick index within the instance; -1: no more
  long long M;                       // staging margin (fixed point)
  float UB;                          // upper bound of every voxel's best score (f-units)
  int org[3];                        // first voxel of the brick
  long long slot;                    // culling re-run: the brick's second-pass list entry
  Region R;                          // region of the current staging round
};
using P1Area = P1AreaT<kP1St>;


// First centre (ob) and centre extent (hb) of the brick whose first voxel is
// (x0, y0, z0).
template <class C>
__device__ __forceinline__ void brick_box(const Inst& I, int x0, int y0, int z0, int* ob,
                                          int* hb) {
  ob[0] = kQ * x0 + kQ / 2;
  ob[1] = kQ * y0 + kQ / 2;
  ob[2] = kQ * z0 + kQ / 2;
  hb[0] = kQ * (min(x0 + C::BX, I.n[0]) - 1 - x0);
  hb[1] = kQ * (min(y0 + C::BY, I.n[1]) - 1 - y0);
  hb[2] = kQ * (min(z0 + C::BZ, I.n[2]) - 1 - z0);
}

// First voxel, first centre and centre extent of brick lb.  The staging
// warp divides; the scoring warps read the first voxel it records.
template <class C>
__device__ __forceinline__ void brick_geom(const Inst& I, long long lb, int& x0, int& y0, int& z0,
                                           int* ob, int* hb) {
  // brick indices fit 32 bits (at most 2^31 bricks per instance): 32-bit
  // unsigned division, far cheaper than the 64-bit routine
  const unsigned ul = (unsigned)lb, b0 = (unsigned)I.bricks[0], b1 = (unsigned)I.bricks[1];
  const unsigned rr = ul / b0;
  const int bxi = (int)(ul - rr * b0);
  const int bzi = (int)(rr / b1), byi = (int)(rr - (unsigned)bzi * b1);
  x0 = bxi * C::BX;
  y0 = byi * C::BY;
  z0 = bzi * C::BZ;
  brick_box<C>(I, x0, y0, z0, ob, hb);
}

__device__ __forceinline__ int warp_incl_scan(int x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Upper bound of F over a tile whose squared farthest extents per axis are
// d2 = sx + sy + sz (each rounded up), with the same allowances as f_bounds_f.
template <int KIND>
__device__ __forceinline__ float tile_hi(float sx, float sy, float sz, float a, float b,
                                         float absf) {
  const float d = __fadd_ru(__fadd_ru(sx, sy), sz);
  if (KIND == KV) return d;
  if (KIND == KL) return __fadd_ru(d, __fmul_ru(a, 1.0f + 0x1p-22f));
  const float h0 = __fmaf_ru(__fsqrt_ru(d), __fmul_ru(b, 1.0f + 0x1p-22f),
                             __fmul_ru(a, 1.0f + 0x1p-22f));
  return __fadd_ru(__fmul_ru(h0, 1.0f + 0x1p-20f), absf);
}

// Position k of a centre-out walk over [0, n) from c: c, c + 1, c - 1,
// c + 2, c - 2, ..., then the longer side alone.
__device__ __forceinline__ int centre_out(int k, int n, int c) {
  const int m = min(c, n - 1 - c);
  if (k <= 2 * m) return (k & 1) ? c + ((k + 1) >> 1) : c - (k >> 1);
  const int r = k - 2 * m;
  return c - m == 0 ? c + m + r : c - m - r;
}

// The four tiles of a brick relative to its first centre: tile t spans
// x [ox(t & 1), + hx[t & 1]], y [oy(t >> 1), + hy[t >> 1]], z [0, hz]
// (ox(0) = oy(0) = 0); a tile outside the grid is off.
struct TileBoxes {
  float ox1, oy1, hx[2], hy[2], hz;
  bool on[kP1Cons];
};

template <class C>
__device__ __forceinline__ TileBoxes tile_boxes(const Inst& I, int x0, int y0, const int* hb) {
  TileBoxes T;
  T.ox1 = (float)(kQ * C::BXW);
  T.oy1 = (float)(kQ * C::BYW);
  T.hx[0] = (float)(kQ * (min(C::BXW, I.n[0] - x0) - 1));
  T.hx[1] = (float)(kQ * (min(C::BXW, I.n[0] - x0 - C::BXW) - 1));
  T.hy[0] = (float)(kQ * (min(C::BYW, I.n[1] - y0) - 1));
  T.hy[1] = (float)(kQ * (min(C::BYW, I.n[1] - y0 - C::BYW) - 1));
  T.hz = (float)hb[2];
  const bool ax1 = x0 + C::BXW < I.n[0], ay1 = y0 + C::BYW < I.n[1];
  T.on[0] = true;
  T.on[1] = ax1;
  T.on[2] = ay1;
  T.on[3] = ax1 && ay1;
  return T;
}

// Whether staged image e can win a voxel of some tile: its lower bound over
// tile t is at most U0(t), the tile's smallest upper bound of a staged image
// (every best score on the tile is at most U0(t)); tk[t] holds U0(t) in its
// high word once reduced over the warp.
template <int KIND>
__device__ __forceinline__ bool wins_some_tile(const Staged& e, const TileBoxes& T,
                                               const unsigned long long (&tk)[kP1Cons],
                                               float absf) {
  bool any = false;
#pragma unroll
  for (int t = 0; t < kP1Cons; t++) {
    if (!T.on[t] || tk[t] == ~0ull) continue;
    float lo, hi;
    f_bounds_f<KIND>(e.qx - ((t & 1) ? T.ox1 : 0.f), e.qy - ((t >> 1) ? T.oy1 : 0.f), e.qz,
                     T.hx[t & 1], T.hy[t >> 1], T.hz, e.a, e.b, absf, lo, hi);
    any = any || lo <= __uint_as_float((unsigned)(tk[t] >> 32));
  }
  return any;
}

// Drop the staged images [0, ns) whose lower bound over the brick exceeds
// the brick bound of the images staged so far (the largest, over the tiles,
// of the tile's smallest upper bound).  That bound only decreases as images
// are added, so no image dropped here would pass the final cull.  The tiles'
// keys are reduced over the warp and their slots follow the images (a key's
// image is always kept: its lower bound is below its upper bound); the kept
// images keep their order.  Returns how many are kept (kP1St + 1, which
// stops staging as an overflow, should a key's image have been dropped).
// An image that passes the brick test is also dropped unless it can win a
// voxel of some tile (wins_some_tile): a void tile next to a dense cluster
// no longer keeps the cluster's far side for the cluster's own tiles.
template <int KIND, class AR>
__device__ __forceinline__ int p1_midcull(AR& A, int ns, unsigned long long (&tk)[kP1Cons],
                                          const TileBoxes& T, float absf) {
  const int lane = threadIdx.x & 31;
  float UB = 0.f;
#pragma unroll
  for (int t = 0; t < kP1Cons; t++) {
    const unsigned hk = (unsigned)(tk[t] >> 32);
    const unsigned h = __reduce_min_sync(0xffffffffu, hk);
    const unsigned slot = __reduce_min_sync(0xffffffffu, hk == h ? (unsigned)tk[t] : ~0u);
    tk[t] = ((unsigned long long)h << 32) | slot;
    if (tk[t] != ~0ull) UB = fmaxf(UB, __uint_as_float(h));
  }
  if (lane < kP1Cons) A.bpos[lane] = -1;
  __syncwarp();
  int cnt = 0;
  for (int c0 = 0; c0 < ns; c0 += 32) {
    const int i = c0 + lane;
    Staged e;
    bool keep = false;
    if (i < ns) {
      e = A.st[i];
      keep = e.lob <= UB && wins_some_tile<KIND>(e, T, tk, absf);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int pos = cnt + __popc(bal & ((1u << lane) - 1));
    __syncwarp();
    if (keep) {
      A.st[pos] = e;
#pragma unroll
      for (int t = 0; t < kP1Cons; t++)
        if ((unsigned)i == (unsigned)tk[t]) A.bpos[t] = pos;
    }
    cnt += __popc(bal);
    __syncwarp();
  }
  __syncwarp();
  bool lost = false;
#pragma unroll
  for (int t = 0; t < kP1Cons; t++) {
    if (tk[t] == ~0ull) continue;
    const int p = A.bpos[t];
    lost = lost || p < 0;
    tk[t] = (tk[t] & 0xFFFFFFFF00000000ull) | (unsigned)(p < 0 ? 0 : p);
  }
  __syncwarp();
  return lost ? AR::cap + 1 : cnt;
}

// Producer, one round: stage the sites of region A.R into A.st, each as the
// periodic image(s) that are nearest for some voxel of the brick box
// [ob, ob + hb] (usually one; more only when the brick reaches past half a
// period from a site), with its lower bound over the brick; tk[t] receives,
// per tile, the smallest (upper bound bits, slot) key over the staged images.
// Lane j takes bin row j (+32k); a warp scan of the row lengths places the
// sites, and each lane then takes one site per chunk of 32, found by a
// binary search over the lanes' scanned lengths.  The loads of the next chunk
// are issued before the current chunk is processed.  The four tiles of a
// brick (2 x 2 x 1) share their extents per axis, so one image's upper bounds
// over them come from five squares.  Returns the number of images staged (at
// most kP1St); *overflow when the region held more.
// CULL (the re-run for bricks whose region overflowed): rows are walked from
// the brick's own row outwards (y within z), so that near images come first
// and tighten the bound early, and when the next chunk would not fit, the
// images already staged are culled against the bound so far (p1_midcull);
// staging stops at the first chunk that still does not fit.
template <int KIND, class C, bool CULL, class AR>
__device__ int p1_stage(const Work& wk, const Inst& I, const FUnits& U, AR& A, const int* ob,
                        const int* hb, int x0, int y0, int z0, unsigned long long (&tk)[kP1Cons],
                        bool& overflow) {
  static_assert(C::WX == 2 && C::WY == 2 && C::WZ == 1, "2 x 2 x 1 tiles per brick");
  const int lane = threadIdx.x & 31;
  const Region& R = A.R;
#pragma unroll
  for (int t = 0; t < kP1Cons; t++) tk[t] = ~0ull;
  overflow = false;
  const int rows = (R.bhi[1] - R.blo[1] + 1) * (R.bhi[2] - R.blo[2] + 1);
  if (rows > kP1MaxRows) {
    overflow = true;
    return 0;
  }
  const float hbx = (float)hb[0], hby = (float)hb[1], hbz = (float)hb[2];
  // tile boxes (relative to the brick's first centre): x [ox_i, ox_i + hx_i],
  // y [oy_j, oy_j + hy_j], z [0, hbz]; a tile outside the grid is skipped
  const float ox1 = (float)(kQ * C::BXW), oy1 = (float)(kQ * C::BYW);
  const float hx0 = (float)(kQ * (min(C::BXW, I.n[0] - x0) - 1));
  const float hx1 = (float)(kQ * (min(C::BXW, I.n[0] - x0 - C::BXW) - 1));
  const float hy0 = (float)(kQ * (min(C::BYW, I.n[1] - y0) - 1));
  const float hy1 = (float)(kQ * (min(C::BYW, I.n[1] - y0 - C::BYW) - 1));
  const bool ax1 = x0 + C::BXW < I.n[0], ay1 = y0 + C::BYW < I.n[1];
  // the farthest extent from q to [a, a + h] is |q - (a + h/2)| + h/2 (exact:
  // every h is a multiple of 512), two FMA-pipe operations instead of a max
  const float hx0h = 0.5f * hx0, hx1h = 0.5f * hx1, hy0h = 0.5f * hy0, hy1h = 0.5f * hy1;
  const float mx1 = ox1 + hx1h, my1 = oy1 + hy1h, hbzh = 0.5f * hbz;
  int ry = 1, rz = 1, cy = 0, cz = 0;  // CULL: region rows, and the brick's own row in it
  if constexpr (CULL) {
    ry = R.bhi[1] - R.blo[1] + 1;
    rz = R.bhi[2] - R.blo[2] + 1;
    cy = min(max(floordiv_pos(ob[1] + (hb[1] >> 1), kQ * I.bw[1]) - R.blo[1], 0), ry - 1);
    cz = min(max(floordiv_pos(ob[2] + (hb[2] >> 1), kQ * I.bw[2]) - R.blo[2], 0), rz - 1);
  }
  int base = 0;     // images placed so far
  float UBr = kInf;  // CULL: running bound (f-units), see below
  for (int rg = 0; rg < rows && !(CULL && overflow); rg += 32) {
    int s0 = 0, l0 = 0, s1 = 0, l1 = 0;
    if (rg + lane < rows) {
      int r = rg + lane;
      if constexpr (CULL) {
        const int rq = floordiv_pos(r, ry);
        r = centre_out(r - rq * ry, ry, cy) + ry * centre_out(rq, rz, cz);
      }
      row_runs(wk, I, R, r, s0, l0, s1, l1);
    }
    const int cnt = l0 + l1;
    const int incl = warp_incl_scan(cnt);
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    // sorted-array index of site i of this row group, or -1
    auto src_of = [&](int i) -> int {
      int j = 0;
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, j + step - 1);
        if (v <= i) j += step;
      }
      const int ej = __shfl_sync(0xffffffffu, incl - cnt, j);
      const int a0 = __shfl_sync(0xffffffffu, s0, j), n0 = __shfl_sync(0xffffffffu, l0, j);
      const int a1 = __shfl_sync(0xffffffffu, s1, j);
      const int k = i - ej;
      return i < tot ? (k < n0 ? a0 + k : a1 + (k - n0)) : -1;
    };
    int srcN = src_of(lane);
    int4 pN = make_int4(0, 0, 0, 0);
    float2 fN = make_float2(0.f, 0.f);
    if (srcN >= 0) {
      pN = wk.spos[srcN];
      if (KIND != KV) fN = wk.sfa[srcN];
    }
    for (int c0 = 0; c0 < tot; c0 += 32) {
      const int src = srcN;
      const int4 p = pN;
      const float2 fa = fN;
      if (c0 + 32 < tot) {  // next chunk's loads, in flight while this one is processed
        srcN = src_of(c0 + 32 + lane);
        if (srcN >= 0) {
          pN = wk.spos[srcN];
          if (KIND != KV) fN = wk.sfa[srcN];
        }
      }
      // images of this lane's site
      const int pq[3] = {p.x, p.y, p.z};
      int q[3], ilo[3], icnt[3], n = src >= 0 ? 1 : 0;
#pragma unroll
      for (int a = 0; a < 3; a++) {
        int x = pq[a] - ob[a];
        ilo[a] = 0;
        icnt[a] = 1;
        if (a < I.nd && I.per[a]) {
          const int L = I.L[a], hL = L >> 1;
          const int d = (hb[a] >> 1) - x;
          if (d >= hL) x += L; else if (d < -hL) x -= L;
          const bool minus = -x < -hL, plus = hb[a] - x >= hL;
          ilo[a] = minus ? -1 : 0;
          icnt[a] = 1 + (int)minus + (int)plus;
        }
        q[a] = x;
        n *= icnt[a];
      }
      // CULL, one image per site (the common case): an image whose lower bound
      // over the brick exceeds the running bound UBr can never win a voxel nor
      // set a tile's key, and would fail the cull: it is not staged
      if (CULL && __all_sync(0xffffffffu, n <= 1) && n == 1) {
        float blo, bhi;
        f_bounds_f<KIND>((float)q[0], (float)q[1], (float)q[2], hbx, hby, hbz, fa.x, fa.y, U.absf,
                         blo, bhi);
        if (!(blo <= UBr)) n = 0;
      }
      // slots: lane order when no site has extra images, else a warp scan
      int slot0;
      if constexpr (CULL) {
        int excl, ctot;
        if (__all_sync(0xffffffffu, n <= 1)) {
          const unsigned bal = __ballot_sync(0xffffffffu, n == 1);
          excl = __popc(bal & ((1u << lane) - 1));
          ctot = __popc(bal);
        } else {
          const int nincl = warp_incl_scan(n);
          excl = nincl - n;
          ctot = __shfl_sync(0xffffffffu, nincl, 31);
        }
        if (base + ctot > AR::cap) {
          const TileBoxes T = tile_boxes<C>(I, x0, y0, hb);
          base = p1_midcull<KIND>(A, base, tk, T, U.absf);
        }
        if (base + ctot > AR::cap) {  // uniform: staging stops with base <= cap + 1
          overflow = true;
          break;
        }
        slot0 = base + excl;
        base += ctot;
      } else if (__all_sync(0xffffffffu, n <= 1)) {
        const unsigned bal = __ballot_sync(0xffffffffu, n == 1);
        slot0 = base + __popc(bal & ((1u << lane) - 1));
        base += __popc(bal);
      } else {
        const int nincl = warp_incl_scan(n);
        slot0 = base + nincl - n;
        base += __shfl_sync(0xffffffffu, nincl, 31);
      }
      for (int j = 0; j < n; j++) {
        const int slot = slot0 + j;
        if (slot >= AR::cap) {
          overflow = true;
          break;
        }
        // image j = k0 + icnt0 (k1 + icnt1 k2), every icnt in {1, 2, 3} and
        // j < 27: a multiply-shift divides exactly (no integer division)
        int c[3];
        int jj = j;
#pragma unroll
        for (int a = 0; a < 3; a++) {
          const int cn = icnt[a];
          const int d = cn == 1 ? jj : cn == 2 ? (jj >> 1) : ((jj * 43691) >> 17);
          c[a] = q[a] + (ilo[a] + (jj - d * cn)) * I.L[a];
          jj = d;
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
        A.st[slot] = e;
        // farthest extents to the tiles, per axis (exact), squared rounded up
        const float ex0 = fabsf(e.qx - hx0h) + hx0h, ex1 = fabsf(e.qx - mx1) + hx1h;
        const float ey0 = fabsf(e.qy - hy0h) + hy0h, ey1 = fabsf(e.qy - my1) + hy1h;
        const float ez = fabsf(e.qz - hbzh) + hbzh;
        const float sx0 = __fmul_ru(ex0, ex0), sx1 = __fmul_ru(ex1, ex1);
        const float sy0 = __fmul_ru(ey0, ey0), sy1 = __fmul_ru(ey1, ey1);
        const float sz = __fmul_ru(ez, ez);
        const unsigned long long sl = (unsigned)slot;
// a lane stages its images in increasing slot order, so comparing the bound
// bits alone keeps the smallest (bound, slot) key
#define VT_TILE_KEY(T, SX, SY, ON)                                                          \
  if (ON) {                                                                                 \
    const unsigned hb_ = __float_as_uint(tile_hi<KIND>(SX, SY, sz, e.a, e.b, U.absf));      \
    if (hb_ < (unsigned)(tk[T] >> 32)) tk[T] = ((unsigned long long)hb_ << 32) | sl;        \
  }
        VT_TILE_KEY(0, sx0, sy0, true)
        VT_TILE_KEY(1, sx1, sy0, ax1)
        VT_TILE_KEY(2, sx0, sy1, ay1)
        VT_TILE_KEY(3, sx1, sy1, ax1 && ay1)
#undef VT_TILE_KEY
      }
      // CULL: the running bound, the largest, over the tiles of the brick, of
      // the smallest upper bound staged so far (a bound on every voxel's best
      // score; infinite until every tile has one)
      if constexpr (CULL) {
        unsigned m = 0;
#pragma unroll
        for (int t = 0; t < kP1Cons; t++) {
          const bool on = t == 0 || (t == 1 && ax1) || (t == 2 && ay1) || (t == 3 && ax1 && ay1);
          const unsigned h = __reduce_min_sync(0xffffffffu, (unsigned)(tk[t] >> 32));
          if (on) m = m > h ? m : h;
        }
        UBr = m == 0xFFFFFFFFu ? kInf : __uint_as_float(m);
      }
    }
  }
  // per tile: warp minimum of the keys (upper bounds are non-negative floats,
  // whose bit patterns order like their values)
#pragma unroll
  for (int t = 0; t < kP1Cons; t++) {
    const unsigned hk = (unsigned)(tk[t] >> 32);
    const unsigned h = __reduce_min_sync(0xffffffffu, hk);
    const unsigned slot = __reduce_min_sync(0xffffffffu, hk == h ? (unsigned)tk[t] : ~0u);
    tk[t] = ((unsigned long long)h << 32) | slot;
  }
  overflow = __any_sync(0xffffffffu, overflow);
  return base < AR::cap ? base : AR::cap;
}

// Producer: steps 1-2 for brick lb of instance I into area A (the whole
// warp together; the caller sets A.brick and A.inst).
//  - the first region has the plan's margin (in mean cell radii) plus a
//    tile's half-diagonal (and, for Laguerre, the largest weight);
//  - UB = max over the tiles of U0(t); if the margin M_UB that UB needs
//    exceeds M (or nothing was staged), the region is restaged;
//  - the images whose lower bound over the brick exceeds UB are culled.
template <int KIND, class C, bool CULL = false, bool ONE_ROUND = false, class AR>
__device__ void p1_produce(const Work& wk, const Inst& I, const FUnits& U, long long lb, AR& A,
                           P1Count& n) {
  const int lane = threadIdx.x & 31;
  int x0, y0, z0, ob[3], hb[3];
  brick_geom<C>(I, lb, x0, y0, z0, ob, hb);
  if (lane == 0) {
    A.org[0] = x0;
    A.org[1] = y0;
    A.org[2] = z0;
  }
  const float hd = 0.5f * sqrtf((float)(C::BXW * C::BXW + C::BYW * C::BYW + C::BZW * C::BZW));
  float m0 = (float)kQ * ((float)I.margin + hd);
  if (KIND == KL) m0 = sqrtf(m0 * m0 + (float)U.wglob);
  long long M = (long long)m0 + 1;
  const int bwmax = max(I.bw[0], max(I.bw[1], I.bw[2]));
  const long long gb = I.brick_base + lb;
  float UB = kInf;
  unsigned long long tk[kP1Cons];
  int ns = 0;
#pragma unroll 1
  for (int round = 0;; round++) {
    if (lane < 3) {  // one axis per lane
      const int c = lane == 0 ? ob[0] : lane == 1 ? ob[1] : ob[2];
      const int h = lane == 0 ? hb[0] : lane == 1 ? hb[1] : hb[2];
      make_region_axis(I, lane, c, c + h, M, A.R);
    }
    __syncwarp();
    bool overflow;
    ns = p1_stage<KIND, C, CULL>(wk, I, U, A, ob, hb, x0, y0, z0, tk, overflow);
    __syncwarp();
    const bool full = A.R.full[0] && A.R.full[1] && A.R.full[2];
    if (round == 1 && lane == 0) n.rest++;
    if (ns == 0) {
      if (overflow || full) {  // too many bin rows (the second pass grows rings), or no valid site
        if (lane == 0) {
          if (overflow) defer_brick(wk, gb, M, kInf, kDeferList);
          A.skip = 1;
        }
        return;
      }
      M = 2 * M + (long long)kQ * bwmax;
      __syncwarp();
      continue;
    }
    UB = 0.f;
#pragma unroll
    for (int t = 0; t < kP1Cons; t++)
      if (tk[t] != ~0ull) UB = fmaxf(UB, __uint_as_float((unsigned)(tk[t] >> 32)));
    const long long need = margin_for<KIND>(UB, U);
    if (overflow) {  // the second pass labels it from the certified margin
      if (lane == 0) {
        if constexpr (CULL) {  // listed already: tighten its entry
          wk.p2_list[3 * A.slot + 1] = (int32_t)(need < 0x7FFFFFFF ? need : 0x7FFFFFFF);
          wk.p2_list[3 * A.slot + 2] = __float_as_int(UB);
        } else {
          defer_brick(wk, gb, need, UB, kDeferStage);
        }
        A.skip = 1;
      }
      return;
    }
    // ONE_ROUND (the staging kernel) with I.late: keep the first region; each
    // tile is certified after scoring against its own best scores (p1_consume)
    if ((ONE_ROUND && I.late) || need <= M || full) break;
    M = need;
    __syncwarp();
  }
  // every staged image that can win a voxel of the brick (its lower bound is
  // at most UB; CULL: and at most some tile's own bound) is kept, the others
  // culled in place (a chunk is read whole before it is written, at positions
  // that never pass the ones still to be read); unless ONE_ROUND, every
  // possible winner of every voxel was staged
  TileBoxes T;
  if constexpr (CULL) T = tile_boxes<C>(I, x0, y0, hb);
  int cnt = 0;
  for (int c0 = 0; c0 < ns; c0 += 32) {
    const int i = c0 + lane;
    Staged e;
    bool keep = false;
    if (i < ns) {
      e = A.st[i];
      keep = e.lob <= UB;
      if constexpr (CULL) keep = keep && wins_some_tile<KIND>(e, T, tk, U.absf);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int pos = cnt + __popc(bal & ((1u << lane) - 1));
    __syncwarp();
    if (keep) {
      A.st[pos] = e;
#pragma unroll
      for (int t = 0; t < kP1Cons; t++)
        if ((unsigned)i == (unsigned)tk[t]) A.bpos[t] = pos;
    }
    cnt += __popc(bal);
    __syncwarp();
  }
  if (lane == 0) {
    A.skip = 0;
    A.ncull = cnt;
    A.M = M;
    A.UB = UB;
  }
#pragma unroll
  for (int t = 0; t < kP1Cons; t++)
    if (lane == t) A.tkey[t] = tk[t];
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

// The brick as a scoring warp sees it: the culled images (in a staging area
// in shared memory, or in the pool of global memory), this tile's key, and the
// margin and bound of the region that certified the brick.
struct BrickView {
  const Staged* st;         // culled images [0, ncull)
  int ncull;
  int skip;                 // the brick went to the second pass: nothing to score
  int org[3];               // first voxel of the brick
  unsigned long long tkey;  // this tile: (smallest upper bound bits << 32) | ...
  int bpos;                 // ... and the position of that image in st
  long long M;
  float UB;
  long long slot;           // culling re-run: the brick's second-pass list entry
  bool check;               // certify each tile after scoring (the region was not grown
                            // until certified): every site not staged lies at least dlo[a]
                            // below / dhi[a] above the brick's voxel centres on axis a
  int dlo[3], dhi[3];
};

// Distance (fixed point) from the voxel centres of the tile at offset toff
// (centre extent th) in its brick (centre extent hb) to the nearest site that
// was not staged: at least this far along one axis.
__device__ __forceinline__ long long unstaged_distance(const BrickView& B, const int* toff,
                                                       const int* th, const int* hb) {
  long long d = 0x7FFFFFFFll;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (B.dlo[a] != 0x7FFFFFFF) d = min(d, (long long)B.dlo[a] + toff[a]);
    if (B.dhi[a] != 0x7FFFFFFF) d = min(d, (long long)B.dhi[a] + (hb[a] - toff[a] - th[a]));
  }
  return d;
}

// The warp rescores each voxel flagged in `near` in turn, and the voxel's
// lane overwrites its label (the same thread stored the tile's labels, so
// program order holds).  Returns the count (lane 0; 0 on the other lanes).
template <int KIND, class C, class RES>
__device__ __forceinline__ unsigned long long rescore_near(const Inst& I, const Lane<C>& G,
                                                           unsigned near, RES&& rescore) {
  const int lane = threadIdx.x & 31;
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
    const int id = rescore(cx, cy, cz);
    if (lane == src) I.labels[label_index(I, G.vx + i, G.vy + j, G.vz + k)] = id;
    nresc++;
  }
  return lane == 0 ? (unsigned long long)nresc : 0ull;
}

// The scoring kernel refreshes a tile's running bound every kRefresh
// evaluations (the first after kRefresh - 1 besides entry 0).
constexpr int kRefresh = 4;

// A tile whose list exceeds LCAP entries (a dense cluster, in the culling
// re-run, whose brick is certified by construction): the brick's images are
// listed again and scored in chunks of LCAP - 1 entries.  After each chunk
// every voxel's two keys keep their scores and take the reserved index
// LCAP - 1, and the site of a first key from the chunk is stored as the
// voxel's label (the last one stored is the winner's); a later entry with an
// equal score wins the key and leaves the carried key second, which the band
// flags.  Near voxels are rescored over all the brick's images
// (rescore_area).  The exact mode carries its (score, id) state across
// chunks as it is.
template <int KIND, class C, int PREC, int LCAP>
__device__ bool p1_long(const Work& wk, const Inst& I, const FUnits& U, Entry* list,
                        const BrickView& B, const Lane<C>& G, const Entry& bx, float U0, float wx,
                        float wy, float wz, float hx, float hy, float hz, P1Count& n) {
  const int lane = threadIdx.x & 31;
  constexpr unsigned K1 = ListKeys<LCAP>::mask;
  constexpr unsigned kRes = K1;     // index of a carried key
  constexpr int kChunk = LCAP - 1;  // list positions of a chunk
  const int ncl = B.ncull, bp = B.bpos;
  int evals = 0;
  float Uc = U0;
  unsigned k1[C::NV], k2[C::NV];
  long long bs[C::NV];
  double ba[C::NV];
  int lab[C::NV];
#pragma unroll
  for (int v = 0; v < C::NV; v++) {
    k1[v] = k2[v] = 0xFFFFFFFFu;
    bs[v] = 0x7FFFFFFFFFFFFFFFll;
    ba[v] = kInf;
    lab[v] = 0x7FFFFFFF;
  }
  auto score = [&](int len) {
    __syncwarp();
#pragma unroll 1
    for (int e = 0; e < len; e++) {
      const Entry x = list[e];
      if (x.lo > Uc) continue;
      ++evals;
      if (PREC == P_F32) {
        eval_f32<KIND, C, K1>(x, (unsigned)e, G, k1, k2);
        if (evals % kRefresh == 0) Uc = fminf(Uc, u_f32<C, K1>(G, k1, U.absf));
      } else {
        eval_exact<KIND, C>(x, exact_site<KIND>(wk, x.src), G, bs, ba, lab);
        if (evals % kRefresh == 0) Uc = fminf(Uc, u_exact<KIND, C>(G, bs, ba, U));
      }
    }
    if (PREC == P_F32) {
#pragma unroll
      for (int v = 0; v < C::NV; v++) {
        const unsigned ix = k1[v] & K1;
        if (ix != kRes && k1[v] != 0xFFFFFFFFu && ((G.vmask >> v) & 1u)) {
          const int i = v & 3, j = (v >> 2) % C::MY, k = (v >> 2) / C::MY;
          I.labels[label_index(I, G.vx + i, G.vy + j, G.vz + k)] = list[ix].id;
        }
        if (k1[v] != 0xFFFFFFFFu) k1[v] |= kRes;
        if (k2[v] != 0xFFFFFFFFu) k2[v] |= kRes;
      }
    }
    __syncwarp();
  };
  if (lane == 0) {
    list[0] = bx;
    atomicAdd(&wk.cnt[C_LONG], 1ull);
  }
  int len = 1;
  for (int base = 0; base < ncl; base += 32) {
    const int i = base + lane;
    bool keep = false;
    Entry x;
    if (i < ncl && i != bp) {
      float hi;
      x = tile_entry<KIND>(B.st[i], wx, wy, wz, hx, hy, hz, U.absf, hi);
      keep = x.lo <= U0;
      if (KIND != KJ && keep) keep = !dominated(x, bx, hx, hy, hz);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (len + __popc(bal) > kChunk) {
      score(len);
      len = 0;
    }
    const int pos = len + __popc(bal & ((1u << lane) - 1));
    if (keep) list[pos] = x;
    len += __popc(bal);
  }
  score(len);
  n.cand += (unsigned long long)evals * 32ull * C::NV;
  if (PREC == P_F32) {
    unsigned near = 0;  // the labels are stored; near voxels are overwritten
#pragma unroll
    for (int v = 0; v < C::NV; v++) {
      const float f1 = __uint_as_float(k1[v] & ~K1);
      const float f2 = __uint_as_float(k2[v] & ~K1);
      if (f2 <= __fmaf_ru(f1, 1.0f + ListKeys<LCAP>::band, 4.0f * U.absf)) near |= 1u << v;
    }
    near &= G.vmask;
    n.resc += rescore_near<KIND, C>(I, G, near, [&](float cx, float cy, float cz) {
      return rescore_area<KIND>(wk, B.st, ncl, wx, wy, wz, cx, cy, cz, U.absf);
    });
  } else {
    store_labels<C>(I, G, lab);
  }
  return true;
}

// Scoring: steps 3-4 for tile `warp` (0 .. kP1Cons-1) of brick lb.  B.st is
// read only while the list is built; release() is called once, as soon as it
// is no longer read.
//  - list: entry 0 is the image with the smallest upper bound U0 over the
//    tile; then, in one parallel pass, every image whose lower bound is at
//    most U0 and (V/L) that entry 0 does not dominate on the tile.  No other
//    image can win anywhere on the tile;
//  - if every listed image belongs to entry 0's site the tile is uniform;
//  - else entry 0 is scored, then the others in order, skipping an entry whose
//    lower bound exceeds the running bound U (the largest best score of the
//    tile so far).
// Returns whether the tile is settled (its labels stored, or no voxel of it in
// the grid); false for a skipped brick or a list that did not fit (RELIST:
// the culling re-run, whose brick keeps its list entry, updated here).
template <int KIND, class C, int PREC, int LCAP, bool RELIST = false, class REL>
__device__ bool p1_consume(const Work& wk, const Inst& I, const FUnits& U, Entry* list,
                           const BrickView& B, long long lb, int warp, REL&& release,
                           P1Count& n) {
  const int lane = threadIdx.x & 31;
  if (B.skip) {
    release();
    return false;
  }
  const int x0 = B.org[0], y0 = B.org[1], z0 = B.org[2];
  int ob[3], hb[3];
  brick_box<C>(I, x0, y0, z0, ob, hb);
  Lane<C> G;
  lane_setup_box<C>(I, x0 + (warp % C::WX) * C::BXW, y0 + ((warp / C::WX) % C::WY) * C::BYW,
                    z0 + (warp / (C::WX * C::WY)) * C::BZW, G);
  if (!G.active) {  // a tile outside the grid has nothing to label
    release();
    return true;
  }
  constexpr unsigned K1 = ListKeys<LCAP>::mask;
  const int ncl = B.ncull;
  // tile origin relative to the brick origin, tile extent (exact floats)
  const float wx = (float)(G.ox - ob[0]), wy = (float)(G.oy - ob[1]), wz = (float)(G.oz - ob[2]);
  const float hx = (float)G.hx, hy = (float)G.hy, hz = (float)G.hz;
  const float U0 = __uint_as_float((unsigned)(B.tkey >> 32));
  const int bp = B.bpos;
  float bhi;
  const Entry bx = tile_entry<KIND>(B.st[bp], wx, wy, wz, hx, hy, hz, U.absf, bhi);
  if (lane == 0) list[0] = bx;
  int len = 1;
  bool other = false;
  float hmax = bhi;  // largest upper bound over the tile of a listed image
  for (int base = 0; base < ncl; base += 32) {
    const int i = base + lane;
    bool keep = false;
    Entry x;
    if (i < ncl && i != bp) {
      float hi;
      x = tile_entry<KIND>(B.st[i], wx, wy, wz, hx, hy, hz, U.absf, hi);
      keep = x.lo <= U0;
      if (KIND != KJ && keep) keep = !dominated(x, bx, hx, hy, hz);
      if (keep) hmax = fmaxf(hmax, hi);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    other = other || __any_sync(0xffffffffu, keep && x.id != bx.id);
    const int pos = len + __popc(bal & ((1u << lane) - 1));
    if (keep && pos < LCAP) list[pos] = x;
    len += __popc(bal);
  }
  const long long Mb = B.M;
  const float UBb = B.UB;
  const long long slot = RELIST ? B.slot : -1;
  if constexpr (RELIST) {
    // the re-run's warp still holds its area: score the long list in chunks
    if (len > LCAP) {
      const bool settled =
          p1_long<KIND, C, PREC, LCAP>(wk, I, U, list, B, G, bx, U0, wx, wy, wz, hx, hy, hz, n);
      release();
      return settled;
    }
  }
  release();  // B.st is no longer read
  if (len > LCAP) {
    if (lane == 0) {
      if (RELIST) {  // culling re-run: the brick stays listed, with this region's bounds
        wk.p2_list[3 * slot + 1] = (int32_t)(Mb < 0x7FFFFFFF ? Mb : 0x7FFFFFFF);
        wk.p2_list[3 * slot + 2] = __float_as_int(UBb);
      } else {
        defer_brick(wk, I.brick_base + lb, Mb, UBb, kDeferList);
      }
    }
    return false;
  }
  // distance to the nearest unstaged site; a tile is certified when every such
  // site scores more than the tile's largest best score (margin_for gives the
  // distance beyond which a site does)
  long long dout = 0x7FFFFFFFll;
  if (B.check) {
    const int toff[3] = {G.ox - ob[0], G.oy - ob[1], G.oz - ob[2]};
    const int th[3] = {G.hx, G.hy, G.hz};
    dout = unstaged_distance(B, toff, th, hb);
  }
  if (!other && (!B.check || margin_for<KIND>(U0, U) < dout)) {
    store_uniform<C>(I, G, bx.id);
    n.unif++;
    return true;
  }
  // not certified after scoring: the brick is staged again, grown until
  // certified, by the culling re-run (kDeferStage)
  auto uncertified = [&]() {
    if (lane == 0 && defer_brick(wk, I.brick_base + lb, Mb, UBb, kDeferStage)) n.rest++;
    return false;
  };

  // scoring: entry 0 first
  int evals = 1;
  int lab[C::NV];
  if (PREC == P_F32 && LCAP == 128 && KIND != KJ) {
    // absolute-scale keys (eval_f32q; Voronoi and Laguerre: Johnson-Mehl's
    // loop is bound by its square root, so it keeps the relative keys below):
    // S >= 2 U0 (every voxel's best score is at most U0) and S >= hmax / 12
    // (every listed score stays below 13 S)
    const float S = pow2_ceil(fmaxf(2.0f * U0, warp_max(hmax) * (1.0f / 12.0f)));
    const unsigned sb = __float_as_uint(S), sq = sb * kQMul;
    // near-tie distance in keys: every best score lies below 2 S, where the
    // quantum is q = ulp(S) and an evaluation errs by at most 2.5 q (four
    // roundings below 2 S and that of a); two scores whose quanta differ by
    // more than T = 6 are in the order of their keys
    constexpr unsigned nearK = kQMul * 7u;
    unsigned k1[C::NV], k2[C::NV];
#pragma unroll
    for (int v = 0; v < C::NV; v++) k1[v] = k2[v] = 0xFFFFFFFFu;
    eval_f32q<KIND, C>(bx, 0u - sq, S, G, k1, k2);
    float Uc = fminf(U0, u_f32q<C>(G, k1, S, sb, U.absf));
    int until = kRefresh - 1;  // evaluations until the running bound is refreshed
#pragma unroll 1
    for (int e = 1; e < len; e++) {
      const Entry x = list[e];
      if (x.lo > Uc) continue;
      eval_f32q<KIND, C>(x, (unsigned)e - sq, S, G, k1, k2);
      ++evals;
      if (--until == 0) {
        until = kRefresh;
        Uc = fminf(Uc, u_f32q<C>(G, k1, S, sb, U.absf));
      }
    }
    if (B.check && !(margin_for<KIND>(u_f32q<C>(G, k1, S, sb, U.absf), U) < dout))
      return uncertified();
    // a voxel is settled by its first key unless its second key lies within
    // nearK of it: k2 - k1 >= 129 (T + 1) means quanta at least T + 1 apart
    // (the indices differ by less than 129), so the first key's entry scores
    // strictly less than every other
    unsigned near = 0;
#pragma unroll
    for (int v = 0; v < C::NV; v++) {
      lab[v] = list[k1[v] % kQMul].id;
      if (k2[v] - k1[v] < nearK) near |= 1u << v;
    }
    near &= G.vmask;
    store_labels<C>(I, G, lab);
    n.resc += rescore_near<KIND, C>(I, G, near, [&](float cx, float cy, float cz) {
      return KIND == KJ ? rescore_warp<KIND>(wk, list, len, Uc, cx, cy, cz, U.absf)
                        : rescore_warp_ool<KIND>(wk, list, len, Uc, cx, cy, cz, U.absf);
    });
  } else if (PREC == P_F32) {
    unsigned k1[C::NV], k2[C::NV];
#pragma unroll
    for (int v = 0; v < C::NV; v++) k1[v] = k2[v] = 0xFFFFFFFFu;
    eval_f32<KIND, C, K1>(bx, 0u, G, k1, k2);
    float Uc = fminf(U0, u_f32<C, K1>(G, k1, U.absf));
#pragma unroll 1
    for (int e = 1; e < len; e++) {
      const Entry x = list[e];
      if (x.lo > Uc) continue;
      eval_f32<KIND, C, K1>(x, (unsigned)e, G, k1, k2);
      ++evals;
      if (evals % 3 == 0) Uc = fminf(Uc, u_f32<C, K1>(G, k1, U.absf));
    }
    if (B.check && !(margin_for<KIND>(u_f32<C, K1>(G, k1, U.absf), U) < dout)) return uncertified();
    unsigned near = 0;  // voxels of this lane whose two keys lie within the band
#pragma unroll
    for (int v = 0; v < C::NV; v++) {
      const float f1 = __uint_as_float(k1[v] & ~K1);
      const float f2 = __uint_as_float(k2[v] & ~K1);
      lab[v] = list[k1[v] & K1].id;
      if (f2 <= __fmaf_ru(f1, 1.0f + ListKeys<LCAP>::band, 4.0f * U.absf)) near |= 1u << v;
    }
    near &= G.vmask;
    store_labels<C>(I, G, lab);
    n.resc += rescore_near<KIND, C>(I, G, near, [&](float cx, float cy, float cz) {
      return KIND == KJ ? rescore_warp<KIND>(wk, list, len, Uc, cx, cy, cz, U.absf)
                        : rescore_warp_ool<KIND>(wk, list, len, Uc, cx, cy, cz, U.absf);
    });
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
    n.cand += (unsigned long long)evals * 32ull * C::NV;
    if (B.check && !(margin_for<KIND>(u_exact<KIND, C>(G, bs, ba, U), U) < dout))
      return uncertified();
    store_labels<C>(I, G, lab);
    return true;
  }
  n.cand += (unsigned long long)evals * 32ull * C::NV;
  return true;
}

__device__ __forceinline__ void flush_counts(const Work& wk, const P1Count& n) {
  unsigned long long c = n.cand, r = n.resc, u = n.unif;
#pragma unroll
  for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicAdd(&wk.cnt[C_CAND], c);
    if (r) atomicAdd(&wk.cnt[C_RESCORED], r);
    if (u) atomicAdd(&wk.cnt[C_UNIFORM], u);
    if (n.rest) atomicAdd(&wk.cnt[C_RESTAGE], n.rest);
  }
}

// The areas and lists live in dynamic shared memory (more than the 48 KB of
// static shared memory once there are more than two areas).
extern __shared__ __align__(16) unsigned char vt_p1_smem[];

// ------------------------------------------------------------ staging and scoring kernels
//
// The common path runs the first pass as two kernels over a chunk of bricks,
// so that neither waits on the other inside an SM:
//  - k_stage: one warp per brick (steps 1-2) in its own staging area of
//    shared memory; it copies the culled images into the chunk's pool in
//    global memory (one atomic per brick reserves the run) and writes the
//    brick's record (tile keys, margin, bound);
//  - k_tiles: one warp per tile (steps 3-4), the four tiles of a brick in the
//    four warps of a CTA; it reads the brick's record and run (from L2: the
//    chunk's pool is sized to stay there) and scores as above.
// A brick whose staged images do not fit its area goes to the culling re-run
// (k_recull_warp); one whose run does not fit the pool goes to the second
// pass with its certified margin and bound.

constexpr int kAst = 256;      // staging area of the staging kernel (images per warp)
constexpr long long kChunkBricks = 65536;  // bricks per staging/scoring chunk
constexpr int kAWarps = 4;     // staging kernel: warps (bricks in flight) per CTA
constexpr int kAMinBlocks = 6; // staging kernel: register budget for 24 warps per SM
constexpr int kBWarps = 4;     // scoring kernel: warps (tiles) per CTA
constexpr int kBMinBlocks = 6; // scoring kernel: register budget for 24 warps per SM
using AreaA = P1AreaT<kAst>;
static_assert(kBWarps == kP1Cons, "the four tiles of a brick share a CTA");

template <class AR>
__device__ __forceinline__ BrickView view_of(const AR& A, int warp) {
  BrickView B;
  B.st = A.st;
  B.ncull = A.ncull;
  B.skip = A.skip;
  B.org[0] = A.org[0];
  B.org[1] = A.org[1];
  B.org[2] = A.org[2];
  B.tkey = A.tkey[warp];
  B.bpos = A.bpos[warp];
  B.M = A.M;
  B.UB = A.UB;
  B.slot = A.slot;
  B.check = false;  // the re-run grows each region until it certifies the brick
#pragma unroll
  for (int a = 0; a < 3; a++) B.dlo[a] = B.dhi[a] = 0x7FFFFFFF;
  return B;
}

template <bool BATCH>
__device__ __forceinline__ int inst_of_brick(const Work& wk, long long g) {
  if (!BATCH) return 0;
  return find_inst(wk.insts, wk.n_inst, g, [](const Inst& x) { return x.brick_base; });
}

// Stage the global bricks [b0, b1) (one instance, or the batch table) into
// the pool of chunk `chunk`.
template <int KIND, class C, bool BATCH>
__global__ void __launch_bounds__(32 * kAWarps, kAMinBlocks)
    k_stage(const Work wk, const __grid_constant__ Inst one, long long b0, long long b1,
            int chunk) {
  AreaA& A = reinterpret_cast<AreaA*>(vt_p1_smem)[threadIdx.x >> 5];
  if (wk.err[E_CODE]) return;
  const int lane = threadIdx.x & 31;
  P1Count n{0, 0, 0, 0};
  const long long nw = (long long)gridDim.x * kAWarps;
#pragma unroll 1
  for (long long g = b0 + (long long)blockIdx.x * kAWarps + (threadIdx.x >> 5); g < b1; g += nw) {
    const int ii = inst_of_brick<BATCH>(wk, g);
    const Inst& I = BATCH ? wk.insts[ii] : one;
    p1_produce<KIND, C, false, true>(wk, I, load_funits<KIND>(wk, ii), g - I.brick_base, A, n);
    __syncwarp();
    int off = -1;
    const int ncull = A.ncull;
    if (!A.skip) {
      if (lane == 0) {
        off = atomicAdd(&wk.pcur[chunk], ncull);
        if ((long long)off + ncull > wk.pool_cap) {  // the pool is full: second pass
          defer_brick(wk, g, A.M, A.UB, kDeferList);
          off = -1;
        }
      }
      off = __shfl_sync(0xffffffffu, off, 0);
    }
    if (off >= 0)
      for (int i = lane; i < ncull; i += 32) wk.pool[off + i] = A.st[i];
    BrickRec& R = wk.brec[g];
    if (lane < kP1Cons) R.tkey[lane] = (A.tkey[lane] & 0xFFFFFFFF00000000ull) | (unsigned)A.bpos[lane];
    if (lane == 0) {
      R.off = off;
      R.ncull = ncull;
      R.org[0] = A.org[0];
      R.org[1] = A.org[1];
      R.org[2] = A.org[2];
      R.M = (int)(A.M < 0x7FFFFFFF ? A.M : 0x7FFFFFFF);
      R.UB = A.UB;
      R.inst = ii;
    }
    if (lane < 3) {  // how far the unstaged sites lie from the brick, per axis and side
      int ob[3], hb[3];
      brick_box<C>(I, A.org[0], A.org[1], A.org[2], ob, hb);
      const int a = lane;
      const bool bounded = a < I.nd && !A.R.full[a];
      R.dlo[a] = bounded && A.R.bl[a] ? ob[a] - A.R.Rlo[a] : 0x7FFFFFFF;
      R.dhi[a] = bounded && A.R.bh[a] ? A.R.Rhi[a] - (ob[a] + hb[a]) : 0x7FFFFFFF;
    }
    __syncwarp();
  }
  flush_counts(wk, n);
}

// Score the tiles of the global bricks [b0, b1) that k_stage staged.
template <int KIND, class C, int PREC, bool BATCH>
__global__ void __launch_bounds__(32 * kBWarps, kBMinBlocks)
    k_tiles(const Work wk, const __grid_constant__ Inst one, long long b0, long long b1) {
  __shared__ Entry lists[kBWarps][kL1];
  if (wk.err[E_CODE]) return;
  const int w = threadIdx.x >> 5;
  P1Count n{0, 0, 0, 0};
  const long long ntiles = (b1 - b0) * kP1Cons;
  const long long nw = (long long)gridDim.x * kBWarps;
#pragma unroll 1
  for (long long t = (long long)blockIdx.x * kBWarps + w; t < ntiles; t += nw) {
    const long long g = b0 + t / kP1Cons;
    const int tw = (int)(t - (g - b0) * kP1Cons);
    const BrickRec& R = wk.brec[g];
    const int ii = BATCH ? R.inst : 0;
    const Inst& I = BATCH ? wk.insts[ii] : one;
    BrickView B;
    const int off = R.off;
    B.skip = off < 0;
    B.st = wk.pool + (off < 0 ? 0 : off);
    B.ncull = R.ncull;
    B.org[0] = R.org[0];
    B.org[1] = R.org[1];
    B.org[2] = R.org[2];
    B.tkey = R.tkey[tw];
    B.bpos = (int)(unsigned)B.tkey;
    B.M = R.M;
    B.UB = R.UB;
    B.slot = -1;
    B.check = I.late != 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      B.dlo[a] = R.dlo[a];
      B.dhi[a] = R.dhi[a];
    }
    p1_consume<KIND, C, PREC, kL1>(wk, I, load_funits<KIND>(wk, ii), lists[w], B,
                                   g - I.brick_base, tw, [] {}, n);
  }
  flush_counts(wk, n);
}

// The culling re-run, one warp per brick: each warp stages a listed brick
// with the running cull (p1_stage<CULL>, growing the region until the brick
// is certified) into its own area, then scores the brick's four tiles in turn
// from that area.  No warp waits for another, so a brick whose staging is long
// (a void far from every site) holds up no other warp.  The brick's flag
// gains one per settled tile, so that a brick all of whose tiles were settled
// reads kDeferDone and the second pass skips it; a brick that fails again
// keeps its list entry, with this run's (tighter) margin and bound.
// A second wave with a larger area (kRBigCap images, one warp per CTA)
// retries the bricks whose culled images still overflowed the first wave's
// area (their flag is still kDeferStage): a void tile next to a dense cluster
// keeps the brick's bound large, so the whole cluster stays staged.
constexpr int kRWarps = 2;        // first wave: warps (bricks in flight) per CTA
constexpr int kRBigCap = 1024;    // second wave: staged images per warp
template <int CAP>
struct RecullWarpT {
  P1AreaT<CAP> area;
  Entry list[kRL];
};
template <int CAP, int NW>
constexpr size_t recull_smem() { return sizeof(RecullWarpT<CAP>) * NW; }

template <int KIND, class C, int PREC, int CAP, int NW>
__global__ void __launch_bounds__(32 * NW)
    k_recull_warp(const Work wk, const __grid_constant__ Inst I) {
  RecullWarpT<CAP>& S = reinterpret_cast<RecullWarpT<CAP>*>(vt_p1_smem)[threadIdx.x >> 5];
  if (wk.err[E_CODE]) return;
  P1Count n{0, 0, 0, 0};
  const FUnits U = load_funits<KIND>(wk, 0);
  const int lane = threadIdx.x & 31;
  const long long total = (long long)*(volatile unsigned long long*)&wk.cnt[C_P2];
  const long long nw = (long long)gridDim.x * NW;
#pragma unroll 1
  for (long long t = (long long)blockIdx.x * NW + (threadIdx.x >> 5); t < total; t += nw) {
    const long long gb = wk.p2_list[3 * t];
    if (wk.p2_flag[gb] != kDeferStage) continue;  // left for the second pass
    const long long lb = gb - I.brick_base;
    P1AreaT<CAP>& A = S.area;
    if (lane == 0) {
      A.brick = lb;
      A.inst = 0;
      A.skip = 1;
      A.slot = t;
    }
    __syncwarp();
    p1_produce<KIND, C, true>(wk, I, U, lb, A, n);
    __syncwarp();
    if (A.skip) continue;
    int settled = 0;
#pragma unroll 1
    for (int tw = 0; tw < kP1Cons; tw++) {
      const BrickView B = view_of(A, tw);
      settled += p1_consume<KIND, C, PREC, kRL, true>(wk, I, U, S.list, B, lb, tw, [] {}, n);
      __syncwarp();
    }
    if (settled && lane == 0)
      if (atomicAdd(&wk.p2_flag[gb], settled) + settled == kDeferDone)
        atomicAdd(&wk.cnt[C_RECULL], 1ull);
  }
  flush_counts(wk, n);
}

// Every brick of the grid listed for the culling re-run (a plan whose bricks
// skip the staging and scoring kernels: clustered sites, whose bricks those
// kernels mostly cannot settle).  Entry b is brick b with margin 0 (a second
// pass would start from the plan's margin) and no bound.
__global__ void k_list_all(const Work wk, const __grid_constant__ Inst I) {
  const long long nb = I.n_bricks;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    const long long g = I.brick_base + b;
    wk.p2_list[3 * b] = (int32_t)g;
    wk.p2_list[3 * b + 1] = 0;
    wk.p2_list[3 * b + 2] = __float_as_int(kInf);
    wk.p2_flag[g] = kDeferStage;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    wk.cnt[C_P2] = (unsigned long long)nb;
    wk.cnt[C_DEFER] = (unsigned long long)nb;
  }
}

// ------------------------------------------------------------ host side

static int g_stage_blocks_per_sm[3][4];        // [kind][tile configuration]
static int g_tiles_blocks_per_sm[3][4][2];     // [kind][tile configuration][prec]
static int g_recull_blocks_per_sm[3][4][2];     // the culling re-run
static int g_recull_big_blocks_per_sm[3][4];    // ... its second wave (FP32)

constexpr size_t kStageSmem = sizeof(AreaA) * kAWarps;

template <typename K>
static cudaError_t p1_prep(K kernel, int threads, size_t smem, int* blocks_per_sm) {
  if (smem > 0) {
    cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, threads, smem);
}

template <int KIND, class C, int PREC>
static cudaError_t occ_one() {
  const int c3 = cfg_index<C>();
  cudaError_t e;
  if ((e = p1_prep(k_tiles<KIND, C, PREC, false>, 32 * kBWarps, 0,
                   &g_tiles_blocks_per_sm[KIND][c3][PREC])) != cudaSuccess ||
      (e = p1_prep(k_tiles<KIND, C, PREC, true>, 32 * kBWarps, 0,
                   &g_tiles_blocks_per_sm[KIND][c3][PREC])) != cudaSuccess ||
      (e = p1_prep(k_recull_warp<KIND, C, PREC, kP1St, kRWarps>, 32 * kRWarps,
                   recull_smem<kP1St, kRWarps>(), &g_recull_blocks_per_sm[KIND][c3][PREC])) !=
          cudaSuccess)
    return e;
  if (PREC == P_F32 &&
      (e = p1_prep(k_recull_warp<KIND, C, P_F32, kRBigCap, 1>, 32, recull_smem<kRBigCap, 1>(),
                   &g_recull_big_blocks_per_sm[KIND][c3])) != cudaSuccess)
    return e;
  if (PREC == P_F32) {
    int b2 = 0;
    if ((e = p1_prep(k_stage<KIND, C, true>, 32 * kAWarps, kStageSmem, &b2)) != cudaSuccess)
      return e;
    return p1_prep(k_stage<KIND, C, false>, 32 * kAWarps, kStageSmem,
                   &g_stage_blocks_per_sm[KIND][c3]);
  }
  return cudaSuccess;
}

cudaError_t init_pass1() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  cudaError_t e;
#define VT_OCC(K, C, P) \
  if ((e = occ_one<K, C, P>()) != cudaSuccess) return e;
#define VT_OCC_K(K)                                                                   \
  VT_OCC(K, Cfg3, P_F32) VT_OCC(K, Cfg3, P_EXACT) VT_OCC(K, Cfg3c, P_F32)            \
  VT_OCC(K, Cfg3c, P_EXACT) VT_OCC(K, Cfg2, P_F32) VT_OCC(K, Cfg2, P_EXACT)          \
  VT_OCC(K, Cfg2c, P_F32) VT_OCC(K, Cfg2c, P_EXACT)
  VT_OCC_K(KV) VT_OCC_K(KL) VT_OCC_K(KJ)
#undef VT_OCC_K
#undef VT_OCC
  done = cudaSuccess;
  return done;
}

// Bricks of one staging/scoring chunk (the pool holds the culled images of
// one chunk).
int64_t pass1_chunk_bricks() { return kChunkBricks; }

// Staging then scoring, chunk by chunk, of the global bricks [t0, t1);
// *chunk numbers the chunks of the call (each has its pool cursor).
template <int KIND, class C, bool BATCH>
static void launch_chunks(const Work& wk, const Inst& one, int prec, long long t0, long long t1,
                          int sms, int* chunk, cudaStream_t st) {
  const int c3 = cfg_index<C>();
  const int bsa = g_stage_blocks_per_sm[KIND][c3] > 0 ? g_stage_blocks_per_sm[KIND][c3] : 1;
  const int bsb = g_tiles_blocks_per_sm[KIND][c3][prec] > 0 ? g_tiles_blocks_per_sm[KIND][c3][prec]
                                                            : 1;
  for (long long b0 = t0; b0 < t1; b0 += kChunkBricks) {
    const long long b1 = b0 + kChunkBricks < t1 ? b0 + kChunkBricks : t1;
    const long long nb = b1 - b0;
    const long long ga = (nb + kAWarps - 1) / kAWarps;
    const unsigned grid_a = (unsigned)(ga < (long long)bsa * sms ? ga : (long long)bsa * sms);
    k_stage<KIND, C, BATCH><<<grid_a, 32 * kAWarps, kStageSmem, st>>>(wk, one, b0, b1, *chunk);
    const long long gb = nb * kP1Cons / kBWarps;
    const long long gbmax = (long long)bsb * sms * 4;
    const unsigned grid_b = (unsigned)(gb < gbmax ? gb : gbmax);
    if (prec == P_F32)
      k_tiles<KIND, C, P_F32, BATCH><<<grid_b, 32 * kBWarps, 0, st>>>(wk, one, b0, b1);
    else
      k_tiles<KIND, C, P_EXACT, BATCH><<<grid_b, 32 * kBWarps, 0, st>>>(wk, one, b0, b1);
    ++*chunk;
  }
}

template <class C, bool BATCH>
static void launch_chunks_kind(const Work& wk, const Inst& one, int kind, int prec, long long t0,
                               long long t1, int sms, int* chunk, cudaStream_t st) {
  if (kind == KV) launch_chunks<KV, C, BATCH>(wk, one, prec, t0, t1, sms, chunk, st);
  else if (kind == KL) launch_chunks<KL, C, BATCH>(wk, one, prec, t0, t1, sms, chunk, st);
  else launch_chunks<KJ, C, BATCH>(wk, one, prec, t0, t1, sms, chunk, st);
}

template <bool BATCH>
static void launch_chunks_cfg(const Work& wk, const Inst& one, int ci, int kind, int prec,
                              long long t0, long long t1, int sms, int* chunk, cudaStream_t st) {
  if (ci == 0) launch_chunks_kind<Cfg3, BATCH>(wk, one, kind, prec, t0, t1, sms, chunk, st);
  else if (ci == 1) launch_chunks_kind<Cfg3c, BATCH>(wk, one, kind, prec, t0, t1, sms, chunk, st);
  else if (ci == 2) launch_chunks_kind<Cfg2, BATCH>(wk, one, kind, prec, t0, t1, sms, chunk, st);
  else launch_chunks_kind<Cfg2c, BATCH>(wk, one, kind, prec, t0, t1, sms, chunk, st);
}

cudaError_t launch_pass1(const Work& wk, const Inst& I, int sms, cudaStream_t st) {
  int chunk = 0;
  const int prec = I.precision == P_F32 ? P_F32 : P_EXACT;
  const long long t0 = I.brick_base, t1 = I.brick_base + I.n_bricks;
  launch_chunks_cfg<false>(wk, I, cfg_index(I.nd, I.cfg), I.kind, prec, t0, t1, sms, &chunk, st);
  return cudaGetLastError();
}

// One wave of the culling re-run (the list's length is read on the device;
// its warps take the list's entries in grid stride).
template <int KIND, class C>
static void launch_recull(const Work& wk, const Inst& I, int sms, cudaStream_t st) {
  const int c3 = cfg_index<C>();
  const int pr = I.precision == P_F32 ? P_F32 : P_EXACT;
  const int bps = g_recull_blocks_per_sm[KIND][c3][pr];
  const unsigned grid = (unsigned)((bps > 0 ? bps : 1) * sms);
  constexpr size_t sm1 = recull_smem<kP1St, kRWarps>();
  if (pr == P_F32) {
    k_recull_warp<KIND, C, P_F32, kP1St, kRWarps><<<grid, 32 * kRWarps, sm1, st>>>(wk, I);
    const int bb = g_recull_big_blocks_per_sm[KIND][c3];
    const unsigned grid2 = (unsigned)((bb > 0 ? bb : 1) * sms);
    k_recull_warp<KIND, C, P_F32, kRBigCap, 1><<<grid2, 32, recull_smem<kRBigCap, 1>(), st>>>(
        wk, I);
  } else {
    k_recull_warp<KIND, C, P_EXACT, kP1St, kRWarps><<<grid, 32 * kRWarps, sm1, st>>>(wk, I);
  }
}

template <class C>
static void launch_recull_kind(const Work& wk, const Inst& I, int sms, cudaStream_t st) {
  if (I.kind == KV) launch_recull<KV, C>(wk, I, sms, st);
  else if (I.kind == KL) launch_recull<KL, C>(wk, I, sms, st);
  else launch_recull<KJ, C>(wk, I, sms, st);
}

cudaError_t launch_list_all(const Work& wk, const Inst& I, cudaStream_t st) {
  const long long blocks = (I.n_bricks + 255) / 256;
  k_list_all<<<(unsigned)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, st>>>(wk, I);
  return cudaGetLastError();
}

cudaError_t launch_pass1_recull(const Work& wk, const Inst& I, int sms, cudaStream_t st) {
  const int ci = cfg_index(I.nd, I.cfg);
  if (ci == 0) launch_recull_kind<Cfg3>(wk, I, sms, st);
  else if (ci == 1) launch_recull_kind<Cfg3c>(wk, I, sms, st);
  else if (ci == 2) launch_recull_kind<Cfg2>(wk, I, sms, st);
  else launch_recull_kind<Cfg2c>(wk, I, sms, st);
  return cudaGetLastError();
}

// The instances of one class (kind and dimension) occupy the global bricks
// [t0, t1): staged and scored chunk by chunk, each brick's instance looked up
// from the batch table.
cudaError_t launch_pass1_group(const Work& wk, int nd, int compact, int kind, int prec,
                               long long t0, long long t1, int sms, int* chunk, cudaStream_t st) {
  if (t1 <= t0) return cudaSuccess;
  Inst none;
  memset(&none, 0, sizeof(none));
  launch_chunks_cfg<true>(wk, none, cfg_index(nd, compact), kind, prec, t0, t1, sms, chunk, st);
  return cudaGetLastError();
}

}  // namespace vt
