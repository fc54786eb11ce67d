// vt_label.cu -- the labelling kernels.
//
// The paper's two-step method (Algorithms 2 and 3, Section 3) first settles
// every voxel that lies in some site's investigation ball, then brute-forces
// the rest.  Its correctness rests on one fact: a voxel's winner is among the
// sites whose score at that voxel is below a threshold that some site already
// achieves there.  The GPU path keeps that fact and turns the loops around
// (voxel-centric instead of site-centric):
//
//  pass 1 (k_pass1): one CTA per brick of voxels.  The CTA stages into shared
//    memory the sites of every bin within a margin of the brick (the "region").
//    Each warp owns a box of the brick; for each staged site it takes the
//    periodic image(s) nearest the box (Appendix A) and exact lower/upper bounds
//    of the site's score over the box, keeps only the sites whose lower bound is
//    at most the smallest upper bound, and scores them per voxel in ascending
//    bands of the lower bound, dropping any site whose bound exceeds the best
//    score already certain for every voxel of the box.
//    In FP32 mode each voxel keeps its best and second-best packed key (the
//    FP32 score with its low mantissa bits replaced by the list index); a voxel
//    whose two keys are within the error bound is rescored exactly (int64 /
//    IEEE double), so labels equal the exact definition.
//    A voxel is certified when its best score is below a lower bound of the
//    score of every site outside the region (distance to the region's faces,
//    minus the largest weight / plus the earliest birth); a brick with any
//    uncertified voxel, or whose staging overflowed, goes on the pass-2 list.
//  pass 2 (k_pass2): for each listed brick, grow the region ring by ring
//    (doubling the margin), stage only the bins of the new ring whose lower
//    bound can still beat the brick's current worst best score, score exactly,
//    and stop when every voxel is certified (at the latest when the region
//    covers the whole box, which is the brute force of the paper's step 2).
#include "vt_internal.cuh"

namespace vt {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kCap = 384;     // staged sites per CTA
constexpr int kLcap = 256;    // list entries per warp (8 index bits in a key)
constexpr int kMaxSeg = 512;  // staging segments (two per bin row)
constexpr unsigned kIdxMask = 0xFFu;
constexpr int kBinGroup = kThreads;  // pass 2: bins tested per round

// Warp tile geometry.  A lane owns a micro-tile of 4 x MY x MZ voxels (x runs
// of 4 for 16-byte stores); the lanes of a warp form LX x LY x LZ micro-tiles
// and the warps of a CTA WX x WY x WZ warp boxes.
template <int MY_, int MZ_, int LX_, int LY_, int LZ_, int WX_, int WY_, int WZ_>
struct Cfg {
  static constexpr int MX = 4, MY = MY_, MZ = MZ_;
  static constexpr int LX = LX_, LY = LY_, LZ = LZ_;
  static constexpr int WX = WX_, WY = WY_, WZ = WZ_;
  static constexpr int NV = MX * MY * MZ;
  static constexpr int BXW = MX * LX, BYW = MY * LY, BZW = MZ * LZ;
  static constexpr int BX = BXW * WX, BY = BYW * WY, BZ = BZW * WZ;
  static_assert(LX * LY * LZ == 32, "32 lanes");
  static_assert(WX * WY * WZ == kWarps, "warps per CTA");
};
using Cfg3 = Cfg<1, 4, 2, 8, 2, 2, 2, 1>;  // warp box 8x8x8, brick 16x16x8
using Cfg2 = Cfg<4, 1, 4, 8, 1, 2, 2, 1>;  // warp box 16x32, brick 32x64

// One candidate (a site image) of a warp's list.  FP32 mode stores the image
// position relative to the warp origin as exact floats; exact mode stores the
// same integers bit-cast.
struct Entry {
  float qx, qy, qz;
  float a, b;   // FP32 data: L (W - w); JM (t - tmin, 1/(512 v))
  float lo;     // lower bound of the score over the warp box
  int id;       // site id
  int sidx;     // staging slot (exact data)
};

struct Region {
  int blo[3], bhi[3];  // bin index range, unwrapped on periodic axes
  int full[3];         // the range holds every bin of the axis exactly once
  int bl[3], bh[3];    // a face of the region is a real boundary (sites beyond it)
  int Rlo[3], Rhi[3];  // region extent [Rlo, Rhi) in fixed point (unwrapped)
};

struct Smem {
  Inst inst;
  Region R, P;
  int4 spos[kCap];
  longlong2 saux[kCap];
  float2 sfa[kCap];
  Entry list[kWarps][kLcap];
  int seg_src[kMaxSeg + 1];
  int seg_off[kMaxSeg + 1];
  int wtot[kWarps];
  int nstaged, overflow, any_unc, has_prev, tile;
  long long wglob;
  double tmin, vmax;
  float absf, inv_vmax_rd;
  unsigned int ukey;  // pass 2: brick-wide upper bound (ordered float key)
  unsigned long long cand, resc;
};

// ------------------------------------------------------------ small helpers

__device__ __forceinline__ unsigned fkey(float f) {  // order-preserving float -> uint
  unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Exclusive scan of a[0..n) in shared memory (n <= 8 * kThreads); returns the
// total.  Every thread of the CTA must call it.
__device__ int block_scan(int* a, int n, int* wtot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + kThreads - 1) / kThreads;
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
  for (int w = 0; w < kWarps; w++) {
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

// Unwrapped bin of fixed-point coordinate x on a periodic axis (bins need not
// divide the period: the last bin may be short).
__device__ __forceinline__ int64_t ubin_per(const Inst& I, int a, int64_t x) {
  const int64_t L = I.L[a], Bw = (int64_t)kQ * I.bw[a];
  int64_t k = floordiv(x, L);
  return k * I.nb[a] + (x - k * L) / Bw;
}
__device__ __forceinline__ int64_t ubin_lo_coord(const Inst& I, int a, int64_t u) {
  int64_t k = floordiv(u, I.nb[a]);
  return k * I.L[a] + (u - k * I.nb[a]) * (int64_t)kQ * I.bw[a];
}
__device__ __forceinline__ int64_t ubin_hi_coord(const Inst& I, int a, int64_t u) {  // exclusive
  int64_t k = floordiv(u, I.nb[a]);
  int64_t e = (u - k * I.nb[a] + 1) * (int64_t)kQ * I.bw[a];
  return k * I.L[a] + (e < I.L[a] ? e : I.L[a]);
}
__device__ __forceinline__ int wrap_bin(const Inst& I, int a, int u) {
  if (!I.per[a]) return u;
  int nb = I.nb[a];
  int r = u % nb;
  return r < 0 ? r + nb : r;
}

// Region of the bins whose sites lie within M (fixed point) of the centre box
// [clo, chi] (clipped to the box on open axes, each bin once on periodic axes).
__device__ void make_region(const Inst& I, const int64_t* clo, const int64_t* chi, int64_t M,
                            Region& R) {
  for (int a = 0; a < 3; a++) {
    const int nb = I.nb[a];
    const int64_t Bw = (int64_t)kQ * I.bw[a];
    if (a >= I.nd) {
      R.blo[a] = R.bhi[a] = 0;
      R.full[a] = 1;
      R.bl[a] = R.bh[a] = 0;
      R.Rlo[a] = 0;
      R.Rhi[a] = I.L[a];
      continue;
    }
    const int64_t xlo = clo[a] - M, xhi = chi[a] + M;
    if (I.per[a]) {
      int64_t ulo = ubin_per(I, a, xlo), uhi = ubin_per(I, a, xhi);
      if (uhi - ulo + 1 >= nb) {
        R.blo[a] = 0; R.bhi[a] = nb - 1; R.full[a] = 1; R.bl[a] = R.bh[a] = 0;
        R.Rlo[a] = 0; R.Rhi[a] = I.L[a];
      } else {
        R.blo[a] = (int)ulo; R.bhi[a] = (int)uhi; R.full[a] = 0; R.bl[a] = R.bh[a] = 1;
        R.Rlo[a] = (int)ubin_lo_coord(I, a, ulo);
        R.Rhi[a] = (int)ubin_hi_coord(I, a, uhi);
      }
    } else {
      int64_t ulo = floordiv(xlo, Bw), uhi = floordiv(xhi, Bw);
      if (ulo < 0) ulo = 0;
      if (uhi > nb - 1) uhi = nb - 1;
      R.blo[a] = (int)ulo; R.bhi[a] = (int)uhi;
      R.full[a] = (ulo == 0 && uhi == nb - 1);
      R.bl[a] = ulo > 0; R.bh[a] = uhi < nb - 1;
      R.Rlo[a] = (int)(ulo * Bw);
      R.Rhi[a] = (int)((uhi + 1) * Bw < I.L[a] ? (uhi + 1) * Bw : I.L[a]);
    }
  }
}

// Smallest distance (fixed point) from centre coordinate c to a real face of
// the region along axis a; INT_MAX if the axis has none.
__device__ __forceinline__ int face_gap(const Region& R, int a, int c) {
  int g = 0x7FFFFFFF;
  if (R.bl[a]) g = min(g, c - R.Rlo[a] + 1);
  if (R.bh[a]) g = min(g, R.Rhi[a] - c);
  return g;
}

// ------------------------------------------------------------ lane geometry

template <class C>
struct Lane {
  int ox, oy, oz;        // warp origin: centre of the warp box's first voxel (fixed point)
  int vx, vy, vz;        // first voxel of the lane's micro-tile
  int hx, hy, hz;        // last centre of the (clipped) warp box, relative to the origin
  bool active;           // the warp box has voxels in the grid
  float cx[4], cy[C::MY], cz[C::MZ];  // micro-tile centres relative to the origin
  unsigned vmask;        // micro-tile voxels inside the grid
};

template <class C>
__device__ __forceinline__ void lane_setup(const Inst& I, int bx0, int by0, int bz0, Lane<C>& G) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wx = warp % C::WX, wy = (warp / C::WX) % C::WY, wz = warp / (C::WX * C::WY);
  const int x0 = bx0 + wx * C::BXW, y0 = by0 + wy * C::BYW, z0 = bz0 + wz * C::BZW;
  G.active = x0 < I.n[0] && y0 < I.n[1] && z0 < I.n[2];
  G.ox = kQ * x0 + kQ / 2;
  G.oy = kQ * y0 + kQ / 2;
  G.oz = kQ * z0 + kQ / 2;
  G.hx = kQ * (min(C::BXW, I.n[0] - x0) - 1);
  G.hy = kQ * (min(C::BYW, I.n[1] - y0) - 1);
  G.hz = kQ * (min(C::BZW, I.n[2] - z0) - 1);
  const int lx = lane % C::LX, ly = (lane / C::LX) % C::LY, lz = lane / (C::LX * C::LY);
  G.vx = x0 + lx * C::MX;
  G.vy = y0 + ly * C::MY;
  G.vz = z0 + lz * C::MZ;
#pragma unroll
  for (int j = 0; j < 4; j++) G.cx[j] = (float)(kQ * (lx * C::MX + j));
#pragma unroll
  for (int j = 0; j < C::MY; j++) G.cy[j] = (float)(kQ * (ly * C::MY + j));
#pragma unroll
  for (int j = 0; j < C::MZ; j++) G.cz[j] = (float)(kQ * (lz * C::MZ + j));
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < C::MZ; k++)
#pragma unroll
    for (int j = 0; j < C::MY; j++)
#pragma unroll
      for (int i = 0; i < 4; i++) {
        bool in = G.active && G.vx + i < I.n[0] && G.vy + j < I.n[1] && G.vz + k < I.n[2];
        if (in) m |= 1u << ((k * C::MY + j) * 4 + i);
      }
  G.vmask = m;
}

// ------------------------------------------------------------ candidate bounds

// Periodic images of staged site i that are the nearest image for some voxel
// of the warp box: per axis the image closest to the box centre plus, when the
// box reaches past half a period from it, the neighbouring image(s).
struct Img {
  int q[3];      // central image relative to the warp origin
  int lo[3];     // lowest image offset (in periods): -1 or 0
  int cnt[3];    // images per axis
  int n;         // total images
};

template <class C>
__device__ __forceinline__ void images(const Inst& I, const Lane<C>& G, int4 p, Img& m) {
  const int o[3] = {G.ox, G.oy, G.oz};
  const int h[3] = {G.hx, G.hy, G.hz};
  const int pq[3] = {p.x, p.y, p.z};
  m.n = 1;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    int q = pq[a] - o[a];
    m.lo[a] = 0;
    m.cnt[a] = 1;
    if (a < I.nd && I.per[a]) {
      const int L = I.L[a], hL = L >> 1;
      int d = (h[a] >> 1) - q;
      if (d >= hL) q += L; else if (d < -hL) q -= L;
      bool minus = -q < -hL;          // low end of the box prefers q - L
      bool plus = h[a] - q >= hL;     // high end prefers q + L
      m.lo[a] = minus ? -1 : 0;
      m.cnt[a] = 1 + (int)minus + (int)plus;
    }
    m.q[a] = q;
    m.n *= m.cnt[a];
  }
}

__device__ __forceinline__ void image_pos(const Inst& I, const Img& m, int j, int* q) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    int k = j % m.cnt[a];
    j /= m.cnt[a];
    q[a] = m.q[a] + (m.lo[a] + k) * I.L[a];
  }
}

// Squared distance bounds from image q (relative) to the box [0, h].
__device__ __forceinline__ void dist_bounds(const int* q, const int* h, long long& lo,
                                            long long& hi) {
  lo = 0;
  hi = 0;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    int g = max(0, max(-q[a], q[a] - h[a]));
    int e = max(q[a], h[a] - q[a]);
    lo += (long long)g * g;
    hi += (long long)e * e;
  }
}

// Lower/upper bounds of the score of an image over the box, in the units the
// list is evaluated in (FP32: shifted score; exact: the score itself).
template <int KIND, int PREC>
__device__ __forceinline__ void score_bounds(const Smem& S, int sidx, long long dlo, long long dhi,
                                             float& lo, float& hi) {
  if (KIND == KV) {
    lo = __ll2float_rd(dlo);
    hi = __ll2float_ru(dhi);
  } else if (KIND == KL) {
    long long w = S.saux[sidx].x;
    long long off = PREC == P_F32 ? S.wglob - w : -w;
    lo = __ll2float_rd(dlo + off);
    hi = __ll2float_ru(dhi + off);
  } else {
    if (PREC == P_F32) {
      const float2 fa = S.sfa[sidx];
      float tl = fa.x * (1.0f - 0x1p-22f), th = fa.x * (1.0f + 0x1p-22f);
      float il = fa.y * (1.0f - 0x1p-22f), ih = fa.y * (1.0f + 0x1p-22f);
      float l = __fmaf_rd(__fsqrt_rd(__ll2float_rd(dlo)), il, tl);
      float u = __fmaf_ru(__fsqrt_ru(__ll2float_ru(dhi)), ih, th);
      lo = __fmaf_rd(l, -0x1p-20f, l) - S.absf;
      hi = __fmaf_ru(u, 0x1p-20f, u) + S.absf;
    } else {
      const longlong2 ax = S.saux[sidx];
      double t = __longlong_as_double(ax.x), den = __longlong_as_double(ax.y);
      double al = __dadd_rn(t, __ddiv_rn(__dsqrt_rn((double)dlo), den));
      double ah = __dadd_rn(t, __ddiv_rn(__dsqrt_rn((double)dhi), den));
      lo = __double2float_rd(al);
      hi = __double2float_ru(ah);
    }
  }
}

// ------------------------------------------------------------ evaluation

// FP32 screening of one list entry over the lane's micro-tile: the score is
// a sum of non-negative terms (exact deltas, fma chain), so it is never
// negative and its bit pattern orders like the value.  The key replaces the
// low 8 mantissa bits by the entry index; each voxel keeps the two smallest.
template <int KIND, class C>
__device__ __forceinline__ void eval_f32(const Entry& e, unsigned idx, const Lane<C>& G,
                                         unsigned (&k1)[C::NV], unsigned (&k2)[C::NV]) {
  float dx[4];
#pragma unroll
  for (int i = 0; i < 4; i++) dx[i] = G.cx[i] - e.qx;
#pragma unroll
  for (int k = 0; k < C::MZ; k++) {
    const float dz = G.cz[k] - e.qz;
#pragma unroll
    for (int j = 0; j < C::MY; j++) {
      const float dy = G.cy[j] - e.qy;
      const float base = (KIND == KJ) ? fmaf(dz, dz, dy * dy) : fmaf(dz, dz, fmaf(dy, dy, e.a));
#pragma unroll
      for (int i = 0; i < 4; i++) {
        float f = fmaf(dx[i], dx[i], base);
        if (KIND == KJ) f = fmaf(sqrt_approx(f), e.b, e.a);
        const unsigned key = (__float_as_uint(f) & ~kIdxMask) | idx;
        const int v = (k * C::MY + j) * 4 + i;
        const unsigned hi = max(k1[v], key);
        k1[v] = min(k1[v], key);
        k2[v] = min(k2[v], hi);
      }
    }
  }
}

// Exact score of an entry at one voxel (micro-tile offsets i, j, k).
// V/L: int64; JM: IEEE double in the order t + sqrt(D) / (512 v).
struct Exact {
  long long s;  // V/L score
  double a;     // JM arrival
};

template <int KIND, class C>
__device__ __forceinline__ long long exact_d2(const Lane<C>& G, int qx, int qy, int qz, int i,
                                              int j, int k) {
  const int dx = (int)G.cx[i] - qx, dy = (int)G.cy[j] - qy, dz = (int)G.cz[k] - qz;
  return (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
}

// Exact evaluation of one list entry over the micro-tile (exact mode and the
// second pass): lexicographic minimum of (score, id).
template <int KIND, class C>
__device__ __forceinline__ void eval_exact(const Smem& S, const Entry& e, const Lane<C>& G,
                                           long long (&bs)[C::NV], double (&ba)[C::NV],
                                           int (&bid)[C::NV]) {
  const int qx = __float_as_int(e.qx), qy = __float_as_int(e.qy), qz = __float_as_int(e.qz);
  long long w = 0;
  double t = 0.0, den = 1.0;
  if (KIND == KL) w = S.saux[e.sidx].x;
  if (KIND == KJ) {
    t = __longlong_as_double(S.saux[e.sidx].x);
    den = __longlong_as_double(S.saux[e.sidx].y);
  }
#pragma unroll
  for (int k = 0; k < C::MZ; k++)
#pragma unroll
    for (int j = 0; j < C::MY; j++) {
      const int dy = (int)G.cy[j] - qy, dz = (int)G.cz[k] - qz;
      const long long yz = (long long)dy * dy + (long long)dz * dz;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int v = (k * C::MY + j) * 4 + i;
        const int dx = (int)G.cx[i] - qx;
        const long long D = (long long)dx * dx + yz;
        if (KIND == KJ) {
          const double a = __dadd_rn(t, __ddiv_rn(__dsqrt_rn((double)D), den));
          if (a < ba[v] || (a == ba[v] && e.id < bid[v])) { ba[v] = a; bid[v] = e.id; }
        } else {
          const long long s = KIND == KL ? D - w : D;
          if (s < bs[v] || (s == bs[v] && e.id < bid[v])) { bs[v] = s; bid[v] = e.id; }
        }
      }
    }
}

// ------------------------------------------------------------ warp list

// Build the warp's candidate list from staged slots [0, n): every image whose
// lower bound over the box is at most U0 = min over all images of the upper
// bound.  Returns the list length, or -1 if it overflows.
template <int KIND, class C, int PREC>
__device__ int build_list(Smem& S, const Lane<C>& G, int n, float& U0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Inst& I = S.inst;
  const int h[3] = {G.hx, G.hy, G.hz};
  // pass A: smallest upper bound
  float umin = __int_as_float(0x7f800000);
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    Img m;
    int cnt = 0;
    if (i < n) {
      images<C>(I, G, S.spos[i], m);
      cnt = m.n;
    }
    const int cmax = __reduce_max_sync(0xffffffffu, cnt);
    for (int j = 0; j < cmax; j++) {
      if (j < cnt) {
        int q[3];
        image_pos(I, m, j, q);
        long long dlo, dhi;
        dist_bounds(q, h, dlo, dhi);
        float lo, hi;
        score_bounds<KIND, PREC>(S, i, dlo, dhi, lo, hi);
        umin = fminf(umin, hi);
      }
    }
  }
  U0 = warp_min(umin);
  // pass B: keep images with lo <= U0
  int len = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    Img m;
    int cnt = 0;
    int4 p = make_int4(0, 0, 0, 0);
    if (i < n) {
      p = S.spos[i];
      images<C>(I, G, p, m);
      cnt = m.n;
    }
    const int cmax = __reduce_max_sync(0xffffffffu, cnt);
    for (int j = 0; j < cmax; j++) {
      bool keep = false;
      int q[3] = {0, 0, 0};
      float lo = 0.f;
      if (j < cnt) {
        image_pos(I, m, j, q);
        long long dlo, dhi;
        dist_bounds(q, h, dlo, dhi);
        float hi;
        score_bounds<KIND, PREC>(S, i, dlo, dhi, lo, hi);
        keep = lo <= U0;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      const int pos = len + __popc(bal & ((1u << lane) - 1));
      if (keep && pos < kLcap) {
        Entry e;
        if (PREC == P_F32) {
          e.qx = (float)q[0]; e.qy = (float)q[1]; e.qz = (float)q[2];
          const float2 fa = (KIND == KV) ? make_float2(0.f, 0.f) : S.sfa[i];
          e.a = fa.x; e.b = fa.y;
        } else {
          e.qx = __int_as_float(q[0]); e.qy = __int_as_float(q[1]); e.qz = __int_as_float(q[2]);
          e.a = e.b = 0.f;
        }
        e.lo = lo;
        e.id = p.w;
        e.sidx = i;
        S.list[warp][pos] = e;
      }
      len += __popc(bal);
    }
  }
  __syncwarp();
  return len <= kLcap ? len : -1;
}

// ------------------------------------------------------------ pass 1

template <class C>
struct BrickGeo {
  int x0, y0, z0, x1, y1, z1;  // voxel box (inclusive, clipped)
};

template <class C>
__device__ __forceinline__ BrickGeo<C> brick_geo(const Inst& I, int64_t lb) {
  BrickGeo<C> b;
  const int bxi = (int)(lb % I.bricks[0]);
  const int64_t r = lb / I.bricks[0];
  const int byi = (int)(r % I.bricks[1]);
  const int bzi = (int)(r / I.bricks[1]);
  b.x0 = bxi * C::BX; b.y0 = byi * C::BY; b.z0 = bzi * C::BZ;
  b.x1 = min(b.x0 + C::BX, I.n[0]) - 1;
  b.y1 = min(b.y0 + C::BY, I.n[1]) - 1;
  b.z1 = min(b.z0 + C::BZ, I.n[2]) - 1;
  return b;
}

// Per-tile constants from the instance statistics (thread 0).
template <int KIND>
__device__ __forceinline__ void load_stats(const Work& wk, Smem& S, int ii) {
  const IStat st = wk.istat[ii];
  S.wglob = KIND == KL ? st.wmax : 0;
  if (KIND == KJ) {
    S.tmin = dkey_inv(~st.tmin);
    S.vmax = dkey_inv(st.vmax);
    const double tabs = dkey_inv(st.tabs);
    S.absf = __double2float_ru(tabs * 0x1p-48) + 0x1p-100f;
    S.inv_vmax_rd = __double2float_rd(__ddiv_rd(1.0, __dmul_ru(512.0, S.vmax)));
  } else {
    S.tmin = 0.0; S.vmax = 1.0; S.absf = 0.f; S.inv_vmax_rd = 0.f;
  }
}

// First-pass margin (fixed point): the instance's margin, widened for Laguerre
// so that it also covers the largest weight (power distance g^2 - w_max).
template <int KIND>
__device__ __forceinline__ int64_t p1_margin(const Smem& S) {
  int64_t M = (int64_t)kQ * S.inst.margin;
  if (KIND == KL) M = (int64_t)ceil(sqrt((double)M * (double)M + (double)S.wglob));
  return M;
}

// Stage the sites of region S.R into shared memory; sets S.nstaged or
// S.overflow.  Every thread calls it.
__device__ void stage_region(const Work& wk, Smem& S) {
  const Inst& I = S.inst;
  const Region& R = S.R;
  const int tid = threadIdx.x;
  const int ry = R.bhi[1] - R.blo[1] + 1, rz = R.bhi[2] - R.blo[2] + 1;
  const int rows = ry * rz, nseg = 2 * rows;
  if (nseg > kMaxSeg) {
    if (tid == 0) S.overflow = 1;
    __syncthreads();
    return;
  }
  for (int r = tid; r < rows; r += kThreads) {
    const int by = wrap_bin(I, 1, R.blo[1] + r % ry), bz = wrap_bin(I, 2, R.blo[2] + r / ry);
    const int64_t row = I.bin_base + ((int64_t)bz * I.nb[1] + by) * I.nb[0];
    int a0 = R.blo[0], a1 = R.bhi[0], c0 = 0, c1 = -1;
    if (I.per[0] && !R.full[0]) {
      const int nb = I.nb[0];
      const int k0 = wrap_bin(I, 0, R.blo[0]), len = R.bhi[0] - R.blo[0] + 1;
      a0 = k0;
      a1 = k0 + len - 1;
      if (a1 >= nb) { c0 = 0; c1 = a1 - nb; a1 = nb - 1; }
    }
    const int s0 = wk.bin_start[row + a0], e0 = wk.bin_start[row + a1 + 1];
    S.seg_src[2 * r] = s0;
    S.seg_off[2 * r] = e0 - s0;
    if (c1 >= c0) {
      const int s1 = wk.bin_start[row + c0], e1 = wk.bin_start[row + c1 + 1];
      S.seg_src[2 * r + 1] = s1;
      S.seg_off[2 * r + 1] = e1 - s1;
    } else {
      S.seg_src[2 * r + 1] = 0;
      S.seg_off[2 * r + 1] = 0;
    }
  }
  __syncthreads();
  const int total = block_scan(S.seg_off, nseg, S.wtot);
  if (total > kCap) {
    if (tid == 0) S.overflow = 1;
    __syncthreads();
    return;
  }
  if (tid == 0) S.seg_off[nseg] = total;
  __syncthreads();
  for (int i = tid; i < total; i += kThreads) {
    int lo = 0, hi = nseg - 1;  // last segment with off <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (S.seg_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int src = S.seg_src[lo] + (i - S.seg_off[lo]);
    S.spos[i] = wk.spos[src];
    if (I.kind != KV) {
      S.saux[i] = wk.saux[src];
      S.sfa[i] = wk.sfa[src];
    }
  }
  if (tid == 0) S.nstaged = total;
  __syncthreads();
}

__device__ __forceinline__ long long label_index(const Inst& I, int x, int y, int z) {
  return ((long long)z * I.n[1] + y) * I.n[0] + x;
}

template <class C>
__device__ __forceinline__ void store_labels(const Inst& I, const Lane<C>& G,
                                             const int (&lab)[C::NV]) {
#pragma unroll
  for (int k = 0; k < C::MZ; k++)
#pragma unroll
    for (int j = 0; j < C::MY; j++) {
      const int v0 = (k * C::MY + j) * 4;
      const unsigned row = (G.vmask >> v0) & 0xFu;
      if (!row) continue;
      const long long base = label_index(I, G.vx, G.vy + j, G.vz + k);
      if (row == 0xFu && I.vec_ok) {
        __stcs(reinterpret_cast<int4*>(I.labels + base),
               make_int4(lab[v0], lab[v0 + 1], lab[v0 + 2], lab[v0 + 3]));
      } else {
#pragma unroll
        for (int i = 0; i < 4; i++)
          if (row & (1u << i)) I.labels[base + i] = lab[v0 + i];
      }
    }
}

// Certification gap per voxel: min over axes of the distance to a real face.
template <class C>
__device__ __forceinline__ int voxel_gap(const Region& R, const Lane<C>& G, int i, int j, int k) {
  const int cx = G.ox + (int)G.cx[i], cy = G.oy + (int)G.cy[j], cz = G.oz + (int)G.cz[k];
  return min(face_gap(R, 0, cx), min(face_gap(R, 1, cy), face_gap(R, 2, cz)));
}

__device__ __forceinline__ int box_gap(const Region& R, int ox, int oy, int oz, int hx, int hy,
                                       int hz) {
  int g = 0x7FFFFFFF;
  const int lo[3] = {ox, oy, oz}, hi[3] = {ox + hx, oy + hy, oz + hz};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (R.bl[a]) g = min(g, lo[a] - R.Rlo[a] + 1);
    if (R.bh[a]) g = min(g, R.Rhi[a] - hi[a]);
  }
  return g;
}

// Lower bound (FP32 units) of the score of any site outside the region at
// gap g: V/L g^2 (the shift W_glob cancels the largest weight); JM the
// earliest birth plus g at the fastest speed.
template <int KIND>
__device__ __forceinline__ float lb_f32(const Smem& S, int g) {
  if (g == 0x7FFFFFFF) return __int_as_float(0x7f800000);
  if (KIND == KJ) {
    const float x = __fmul_rd((float)g, S.inv_vmax_rd);
    return __fmaf_rd(x, -0x1p-20f, x) - S.absf;
  }
  return __ll2float_rd((long long)g * g);
}

// Exact-units lower bound: V g^2; L g^2 - W_glob; JM tmin + g / (512 vmax)
// in the same rounded operations as the score (monotone, hence a bound).
template <int KIND>
__device__ __forceinline__ bool certified_exact(const Smem& S, int g, long long bs, double ba) {
  if (g == 0x7FFFFFFF) return true;
  if (KIND == KJ) {
    const double lb = __dadd_rn(S.tmin, __ddiv_rn((double)g, __dmul_rn(512.0, S.vmax)));
    return ba < lb;
  }
  const long long lb = (long long)g * g - S.wglob;
  return bs < lb;
}

template <int KIND, class C>
__device__ __forceinline__ float u_f32(const Lane<C>& G, const unsigned (&k1)[C::NV], float absf) {
  unsigned m = 0;
#pragma unroll
  for (int v = 0; v < C::NV; v++)
    if (G.vmask & (1u << v)) m = max(m, k1[v] & ~kIdxMask);
  m = __reduce_max_sync(0xffffffffu, m);
  if (m >= 0x7f800000u) return __int_as_float(0x7f800000);
  return __fmaf_ru(__uint_as_float(m), 1.0f + 0x1p-14f, 2.0f * absf);
}

template <int KIND, class C>
__device__ __forceinline__ float u_exact(const Lane<C>& G, const long long (&bs)[C::NV],
                                         const double (&ba)[C::NV]) {
  float m = -__int_as_float(0x7f800000);
#pragma unroll
  for (int v = 0; v < C::NV; v++)
    if (G.vmask & (1u << v))
      m = fmaxf(m, KIND == KJ ? __double2float_ru(ba[v]) : __ll2float_ru(bs[v]));
  return warp_max(m);
}

// Exact rescoring of one voxel over every list entry that could still win.
template <int KIND, class C>
__device__ __noinline__ int rescore_voxel(const Smem& S, const Entry* list, int len, float U,
                                          const Lane<C>& G, int i, int j, int k) {
  long long bs = 0x7FFFFFFFFFFFFFFFll;
  double ba = __longlong_as_double(0x7ff0000000000000ll);
  int bid = 0x7FFFFFFF;
  for (int e = 0; e < len; e++) {
    const Entry en = list[e];
    if (en.lo > U) continue;
    const int qx = (int)en.qx, qy = (int)en.qy, qz = (int)en.qz;
    const long long D = exact_d2<KIND, C>(G, qx, qy, qz, i, j, k);
    if (KIND == KJ) {
      const longlong2 ax = S.saux[en.sidx];
      const double a = __dadd_rn(__longlong_as_double(ax.x),
                                 __ddiv_rn(__dsqrt_rn((double)D), __longlong_as_double(ax.y)));
      if (a < ba || (a == ba && en.id < bid)) { ba = a; bid = en.id; }
    } else {
      const long long s = KIND == KL ? D - S.saux[en.sidx].x : D;
      if (s < bs || (s == bs && en.id < bid)) { bs = s; bid = en.id; }
    }
  }
  return bid;
}

// Score the warp's list in three bands of its lower bounds, tightening the
// prune bound U as voxels settle.  FP32 mode.
template <int KIND, class C>
__device__ __forceinline__ int run_list_f32(const Smem& S, const Entry* list, int len, float U0,
                                            const Lane<C>& G, unsigned (&k1)[C::NV],
                                            unsigned (&k2)[C::NV], float& U) {
  const int lane = threadIdx.x & 31;
  float lmin = __int_as_float(0x7f800000);
  for (int e = lane; e < len; e += 32) lmin = fminf(lmin, list[e].lo);
  lmin = warp_min(lmin);
  U = U0;
  const float span = U0 - lmin;
  const float t1 = lmin + 0.125f * span, t2 = lmin + 0.5f * span;
  int evals = 0;
#pragma unroll 1
  for (int band = 0; band < 3; band++) {
#pragma unroll 1
    for (int e = 0; e < len; e++) {
      const float lo = list[e].lo;
      if (!(band == 0 ? lo <= t1 : (band == 1 ? (lo > t1 && lo <= t2) : lo > t2))) continue;
      if (lo > U) continue;
      eval_f32<KIND, C>(list[e], (unsigned)e, G, k1, k2);
      if ((++evals & 3) == 0) U = fminf(U, u_f32<KIND, C>(G, k1, S.absf));
    }
    U = fminf(U, u_f32<KIND, C>(G, k1, S.absf));
  }
  return evals;
}

template <int KIND, class C>
__device__ __forceinline__ int run_list_exact(const Smem& S, const Entry* list, int len, float U0,
                                              const Lane<C>& G, long long (&bs)[C::NV],
                                              double (&ba)[C::NV], int (&bid)[C::NV], float& U) {
  const int lane = threadIdx.x & 31;
  float lmin = __int_as_float(0x7f800000);
  for (int e = lane; e < len; e += 32) lmin = fminf(lmin, list[e].lo);
  lmin = warp_min(lmin);
  U = U0;
  const float span = U0 - lmin;
  const float t1 = lmin + 0.125f * span, t2 = lmin + 0.5f * span;
  int evals = 0;
#pragma unroll 1
  for (int band = 0; band < 3; band++) {
#pragma unroll 1
    for (int e = 0; e < len; e++) {
      const float lo = list[e].lo;
      if (!(band == 0 ? lo <= t1 : (band == 1 ? (lo > t1 && lo <= t2) : lo > t2))) continue;
      if (lo > U) continue;
      eval_exact<KIND, C>(S, list[e], G, bs, ba, bid);
      if ((++evals & 3) == 0) U = fminf(U, u_exact<KIND, C>(G, bs, ba));
    }
    U = fminf(U, u_exact<KIND, C>(G, bs, ba));
  }
  return evals;
}

template <int KIND, class C, int PREC>
__device__ void p1_brick(const Work& wk, Smem& S, int ii, int64_t gbrick) {
  const Inst& I = S.inst;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const BrickGeo<C> B = brick_geo<C>(I, gbrick - I.brick_base);
  if (tid == 0) {
    load_stats<KIND>(wk, S, ii);
    const int64_t clo[3] = {(int64_t)kQ * B.x0 + kQ / 2, (int64_t)kQ * B.y0 + kQ / 2,
                            (int64_t)kQ * B.z0 + kQ / 2};
    const int64_t chi[3] = {(int64_t)kQ * B.x1 + kQ / 2, (int64_t)kQ * B.y1 + kQ / 2,
                            (int64_t)kQ * B.z1 + kQ / 2};
    S.nstaged = 0;
    S.overflow = 0;
    S.any_unc = 0;
    S.cand = 0;
    S.resc = 0;
    make_region(I, clo, chi, p1_margin<KIND>(S), S.R);
  }
  __syncthreads();
  stage_region(wk, S);
  if (S.overflow) {
    if (tid == 0) {
      const unsigned long long slot = atomicAdd(&wk.cnt[C_P2], 1ull);
      wk.p2_list[slot] = (int32_t)gbrick;
      atomicAdd(&wk.cnt[C_DEFER], 1ull);
    }
    return;
  }
  Lane<C> G;
  lane_setup<C>(I, B.x0, B.y0, B.z0, G);
  bool unc = false;
  if (G.active) {
    float U0;
    const int len = build_list<KIND, C, PREC>(S, G, S.nstaged, U0);
    const Entry* list = S.list[warp];
    int lab[C::NV];
    if (len < 0) {
      unc = true;  // list overflow: the whole brick goes to pass 2
#pragma unroll
      for (int v = 0; v < C::NV; v++) lab[v] = 0;
    } else if (PREC == P_F32) {
      unsigned k1[C::NV], k2[C::NV];
#pragma unroll
      for (int v = 0; v < C::NV; v++) k1[v] = k2[v] = 0xFFFFFFFFu;
      float U;
      const int evals = run_list_f32<KIND, C>(S, list, len, U0, G, k1, k2, U);
      if (lane == 0) atomicAdd(&S.cand, (unsigned long long)evals * 32ull * C::NV);
      // near ties -> exact rescoring; labels; certification
      const float lbox = lb_f32<KIND>(S, box_gap(S.R, G.ox, G.oy, G.oz, G.hx, G.hy, G.hz));
      const bool box_ok = U < lbox;
      int nresc = 0;
#pragma unroll
      for (int k = 0; k < C::MZ; k++)
#pragma unroll
        for (int j = 0; j < C::MY; j++)
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const int v = (k * C::MY + j) * 4 + i;
            const float f1 = __uint_as_float(k1[v] & ~kIdxMask);
            const float f2 = __uint_as_float(k2[v] & ~kIdxMask);
            const bool valid = (G.vmask >> v) & 1u;
            int id = list[k1[v] & kIdxMask].id;
            if (valid && k1[v] != 0xFFFFFFFFu &&
                f2 <= __fmaf_ru(f1, 1.0f + 0x1p-13f, 4.0f * S.absf)) {
              id = rescore_voxel<KIND, C>(S, list, len, U, G, i, j, k);
              nresc++;
            }
            lab[v] = id;
            if (valid && !box_ok) {
              const float b = (k1[v] == 0xFFFFFFFFu)
                                  ? __int_as_float(0x7f800000)
                                  : __fmaf_ru(f1, 1.0f + 0x1p-14f, 2.0f * S.absf);
              if (!(b < lb_f32<KIND>(S, voxel_gap<C>(S.R, G, i, j, k)))) unc = true;
            }
          }
      if (nresc) atomicAdd(&S.resc, (unsigned long long)nresc);
    } else {
      long long bs[C::NV];
      double ba[C::NV];
#pragma unroll
      for (int v = 0; v < C::NV; v++) {
        bs[v] = 0x7FFFFFFFFFFFFFFFll;
        ba[v] = __longlong_as_double(0x7ff0000000000000ll);
        lab[v] = 0x7FFFFFFF;
      }
      float U;
      const int evals = run_list_exact<KIND, C>(S, list, len, U0, G, bs, ba, lab, U);
      if (lane == 0) atomicAdd(&S.cand, (unsigned long long)evals * 32ull * C::NV);
#pragma unroll
      for (int k = 0; k < C::MZ; k++)
#pragma unroll
        for (int j = 0; j < C::MY; j++)
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const int v = (k * C::MY + j) * 4 + i;
            if (((G.vmask >> v) & 1u) &&
                !certified_exact<KIND>(S, voxel_gap<C>(S.R, G, i, j, k), bs[v], ba[v]))
              unc = true;
          }
    }
    if (len >= 0) store_labels<C>(I, G, lab);
  }
  const int any = __syncthreads_or(unc);
  if (tid == 0) {
    if (any) {
      const unsigned long long slot = atomicAdd(&wk.cnt[C_P2], 1ull);
      wk.p2_list[slot] = (int32_t)gbrick;
    }
    atomicAdd(&wk.cnt[C_CAND], S.cand);
    if (S.resc) atomicAdd(&wk.cnt[C_RESCORED], S.resc);
  }
}

// ------------------------------------------------------------ pass 2

// Distance between intervals [a0, a1] and [b0, b1] (0 if they meet).
__device__ __forceinline__ int64_t gap1(int64_t a0, int64_t a1, int64_t b0, int64_t b1) {
  const int64_t d = b0 - a1 > a0 - b1 ? b0 - a1 : a0 - b1;
  return d > 0 ? d : 0;
}

// Lower bound, over centres c in [clo, chi] and sites p of wrapped bin wb, of
// the per-axis distance |c - p| (nearest image on a periodic axis: both lie in
// [0, L), so the images -L, 0, +L cover the minimum).
__device__ __forceinline__ int64_t bin_gap(const Inst& I, int a, int wb, int64_t clo, int64_t chi) {
  const int64_t Bw = (int64_t)kQ * I.bw[a];
  const int64_t lo = (int64_t)wb * Bw;
  const int64_t hi = (lo + Bw < (int64_t)I.L[a] ? lo + Bw : (int64_t)I.L[a]) - 1;
  int64_t g = gap1(clo, chi, lo, hi);
  if (I.per[a]) {
    const int64_t L = I.L[a];
    const int64_t g1 = gap1(clo, chi, lo - L, hi - L), g2 = gap1(clo, chi, lo + L, hi + L);
    g = g < g1 ? g : g1;
    g = g < g2 ? g : g2;
  }
  return g;
}

// Is wrapped bin wb of axis a inside region P?
__device__ __forceinline__ bool in_region_axis(const Inst& I, const Region& P, int a, int wb) {
  if (P.full[a]) return true;
  if (I.per[a]) {
    const int nb = I.nb[a];
    int d = (wb - P.blo[a]) % nb;
    if (d < 0) d += nb;
    return d <= P.bhi[a] - P.blo[a];
  }
  return wb >= P.blo[a] && wb <= P.bhi[a];
}

// Evaluate staged slots [0, n) against the warp's exact state, building the
// list in chunks; U is the warp's current bound.
template <int KIND, class C>
__device__ void p2_consume(Smem& S, const Lane<C>& G, int n, long long (&bs)[C::NV],
                           double (&ba)[C::NV], int (&bid)[C::NV], float& U) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Inst& I = S.inst;
  const int h[3] = {G.hx, G.hy, G.hz};
  Entry* list = S.list[warp];
  int len = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    Img m;
    int cnt = 0;
    int4 p = make_int4(0, 0, 0, 0);
    if (i < n) {
      p = S.spos[i];
      images<C>(I, G, p, m);
      cnt = m.n;
    }
    const int cmax = __reduce_max_sync(0xffffffffu, cnt);
    for (int j = 0; j < cmax; j++) {
      bool keep = false;
      int q[3] = {0, 0, 0};
      float lo = 0.f;
      if (j < cnt) {
        image_pos(I, m, j, q);
        long long dlo, dhi;
        dist_bounds(q, h, dlo, dhi);
        float hi;
        score_bounds<KIND, P_EXACT>(S, i, dlo, dhi, lo, hi);
        keep = lo <= U;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (len + __popc(bal) > kLcap) {  // flush the list first
        __syncwarp();
        for (int e = 0; e < len; e++)
          if (list[e].lo <= U) eval_exact<KIND, C>(S, list[e], G, bs, ba, bid);
        U = fminf(U, u_exact<KIND, C>(G, bs, ba));
        len = 0;
        __syncwarp();
      }
      const int pos = len + __popc(bal & ((1u << lane) - 1));
      if (keep) {
        Entry e;
        e.qx = __int_as_float(q[0]); e.qy = __int_as_float(q[1]); e.qz = __int_as_float(q[2]);
        e.a = e.b = 0.f;
        e.lo = lo;
        e.id = p.w;
        e.sidx = i;
        list[pos] = e;
      }
      len += __popc(bal);
    }
  }
  __syncwarp();
  float Ul = U;
  run_list_exact<KIND, C>(S, list, len, U, G, bs, ba, bid, Ul);
  U = fminf(U, Ul);
  __syncwarp();
}

template <int KIND, class C>
__device__ void p2_brick(const Work& wk, Smem& S, int ii, int64_t gbrick) {
  const Inst& I = S.inst;
  const int tid = threadIdx.x, warp = tid >> 5;
  const BrickGeo<C> B = brick_geo<C>(I, gbrick - I.brick_base);
  const int64_t clo[3] = {(int64_t)kQ * B.x0 + kQ / 2, (int64_t)kQ * B.y0 + kQ / 2,
                          (int64_t)kQ * B.z0 + kQ / 2};
  const int64_t chi[3] = {(int64_t)kQ * B.x1 + kQ / 2, (int64_t)kQ * B.y1 + kQ / 2,
                          (int64_t)kQ * B.z1 + kQ / 2};
  if (tid == 0) {
    load_stats<KIND>(wk, S, ii);
    S.has_prev = 0;
    S.ukey = fkey(__int_as_float(0x7f800000));
  }
  __syncthreads();
  Lane<C> G;
  lane_setup<C>(I, B.x0, B.y0, B.z0, G);
  long long bs[C::NV];
  double ba[C::NV];
  int bid[C::NV];
#pragma unroll
  for (int v = 0; v < C::NV; v++) {
    bs[v] = 0x7FFFFFFFFFFFFFFFll;
    ba[v] = __longlong_as_double(0x7ff0000000000000ll);
    bid[v] = 0x7FFFFFFF;
  }
  float U = __int_as_float(0x7f800000);
  int64_t M = p1_margin<KIND>(S);
  int bwmax = I.bw[0];
  if (I.bw[1] > bwmax) bwmax = I.bw[1];
  if (I.nd > 2 && I.bw[2] > bwmax) bwmax = I.bw[2];
#pragma unroll 1
  for (int round = 0;; round++) {
    if (tid == 0) {
      make_region(I, clo, chi, M, S.R);
      S.nstaged = 0;
    }
    __syncthreads();
    const Region R = S.R;
    const int ex = R.bhi[0] - R.blo[0] + 1, ey = R.bhi[1] - R.blo[1] + 1,
              ez = R.bhi[2] - R.blo[2] + 1;
    const long long nbins = (long long)ex * ey * ez;
    const float Ub = fkey_inv(S.ukey);
    // walk the region's bins in groups; stage those of the new ring that can win
#pragma unroll 1
    for (long long g0 = 0; g0 < nbins; g0 += kBinGroup) {
      const long long f = g0 + tid;
      int cnt = 0, src = 0;
      if (f < nbins) {
        const int ix = (int)(f % ex), iy = (int)((f / ex) % ey), iz = (int)(f / ((long long)ex * ey));
        const int ub[3] = {R.blo[0] + ix, R.blo[1] + iy, R.blo[2] + iz};
        int wb[3];
        bool inprev = S.has_prev != 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
          wb[a] = wrap_bin(I, a, ub[a]);
          if (inprev) inprev = in_region_axis(I, S.P, a, wb[a]);
        }
        if (!inprev) {
          const int64_t gb = I.bin_base + ((int64_t)wb[2] * I.nb[1] + wb[1]) * I.nb[0] + wb[0];
          src = wk.bin_start[gb];
          cnt = wk.bin_start[gb + 1] - src;
          if (cnt > 0 && Ub != __int_as_float(0x7f800000)) {
            // lower bound of any site of the bin over the brick
            long long dlo = 0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
              if (a >= I.nd) continue;
              const int64_t g = bin_gap(I, a, wb[a], clo[a], chi[a]);
              dlo += (long long)(g * g);
            }
            bool skip;
            if (KIND == KV) {
              skip = __ll2float_rd(dlo) > Ub;
            } else if (KIND == KL) {
              skip = __ll2float_rd(dlo - (long long)wk.bstat[2 * gb]) > Ub;
            } else {
              const double tm = dkey_inv(~wk.bstat[2 * gb]), vm = dkey_inv(wk.bstat[2 * gb + 1]);
              const double a = __dadd_rn(tm, __ddiv_rn(__dsqrt_rn((double)dlo), __dmul_rn(512.0, vm)));
              skip = __double2float_rd(a) > Ub;
            }
            if (skip) cnt = 0;
          }
        }
      }
      // compact this group's bins behind the already staged sites
      S.seg_src[tid] = src;
      S.seg_off[tid] = cnt;
      __syncthreads();
      const int gtot = block_scan(S.seg_off, kBinGroup, S.wtot);
      if (tid == 0) S.seg_off[kBinGroup] = gtot;
      __syncthreads();
      // copy in pieces of at most kCap sites, flushing whenever staging is full
      for (int done = 0; done < gtot;) {
        const int room = kCap - S.nstaged;
        const int take = min(room, gtot - done);
        for (int i = tid; i < take; i += kThreads) {
          const int gi = done + i;
          int lo = 0, hi = kBinGroup - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.seg_off[mid] <= gi) lo = mid; else hi = mid - 1;
          }
          const int s = S.seg_src[lo] + (gi - S.seg_off[lo]);
          const int d = S.nstaged + i;
          S.spos[d] = wk.spos[s];
          if (KIND != KV) {
            S.saux[d] = wk.saux[s];
            S.sfa[d] = wk.sfa[s];
          }
        }
        __syncthreads();
        done += take;
        const int now = S.nstaged + take;
        if (now == kCap) {
          if (G.active) p2_consume<KIND, C>(S, G, now, bs, ba, bid, U);
          __syncthreads();
          if (tid == 0) S.nstaged = 0;
        } else if (tid == 0) {
          S.nstaged = now;
        }
        __syncthreads();
      }
    }
    if (S.nstaged > 0 && G.active) p2_consume<KIND, C>(S, G, S.nstaged, bs, ba, bid, U);
    __syncthreads();
    // brick-wide bound (max over warps) and certification against this region
    if (tid == 0) S.ukey = fkey(-__int_as_float(0x7f800000));
    __syncthreads();
    if ((tid & 31) == 0 && G.active) atomicMax(&S.ukey, fkey(U));
    bool cert = true;
    if (G.active) {
#pragma unroll
      for (int k = 0; k < C::MZ; k++)
#pragma unroll
        for (int j = 0; j < C::MY; j++)
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const int v = (k * C::MY + j) * 4 + i;
            if (((G.vmask >> v) & 1u) &&
                !certified_exact<KIND>(S, voxel_gap<C>(R, G, i, j, k), bs[v], ba[v]))
              cert = false;
          }
    }
    const int all = __syncthreads_and(cert);
    const bool full = R.full[0] && R.full[1] && R.full[2];
    if (all || full) break;
    if (tid == 0) {
      S.P = R;
      S.has_prev = 1;
    }
    M = 2 * M + (int64_t)kQ * bwmax;
    __syncthreads();
  }
  (void)warp;
  if (G.active) store_labels<C>(I, G, bid);
}

// ------------------------------------------------------------ kernels

__device__ __forceinline__ void load_inst(Smem& S, const Inst& src) {
  const int words = sizeof(Inst) / 4;
  const int* s = reinterpret_cast<const int*>(&src);
  int* d = reinterpret_cast<int*>(&S.inst);
  for (int i = threadIdx.x; i < words; i += kThreads) d[i] = s[i];
}

extern __shared__ __align__(16) unsigned char vt_smem[];

template <int KIND, class C, int PREC>
__global__ void __launch_bounds__(kThreads) k_pass1(const Work wk, const __grid_constant__ Inst one) {
  Smem& S = *reinterpret_cast<Smem*>(vt_smem);
  if (wk.err[E_CODE]) return;
  load_inst(S, one);
  __syncthreads();
  p1_brick<KIND, C, PREC>(wk, S, 0, one.brick_base + blockIdx.x);
}

template <int KIND, class C>
__global__ void __launch_bounds__(kThreads) k_pass2(const Work wk, const __grid_constant__ Inst one) {
  Smem& S = *reinterpret_cast<Smem*>(vt_smem);
  if (wk.err[E_CODE]) return;
  load_inst(S, one);
  const unsigned long long n = *(volatile unsigned long long*)&wk.cnt[C_P2];
  for (unsigned long long t = blockIdx.x; t < n; t += gridDim.x) {
    __syncthreads();
    p2_brick<KIND, C>(wk, S, 0, wk.p2_list[t]);
  }
}

// Batch kernels: one persistent first pass over every brick of every
// instance (work taken from an atomic cursor), then the second pass.
__device__ __forceinline__ int batch_inst(const Work& wk, int64_t gbrick) {
  return find_inst(wk.insts, wk.n_inst, gbrick, [](const Inst& I) { return I.brick_base; });
}

template <int PREC>
__device__ void p1_dispatch(const Work& wk, Smem& S, int ii, int64_t gb) {
  const Inst& I = S.inst;
  if (I.nd == 3) {
    if (I.kind == KV) p1_brick<KV, Cfg3, PREC>(wk, S, ii, gb);
    else if (I.kind == KL) p1_brick<KL, Cfg3, PREC>(wk, S, ii, gb);
    else p1_brick<KJ, Cfg3, PREC>(wk, S, ii, gb);
  } else {
    if (I.kind == KV) p1_brick<KV, Cfg2, PREC>(wk, S, ii, gb);
    else if (I.kind == KL) p1_brick<KL, Cfg2, PREC>(wk, S, ii, gb);
    else p1_brick<KJ, Cfg2, PREC>(wk, S, ii, gb);
  }
}

template <int PREC>
__global__ void __launch_bounds__(kThreads) k_pass1_batch(const Work wk, unsigned long long* cursor) {
  Smem& S = *reinterpret_cast<Smem*>(vt_smem);
  if (wk.err[E_CODE]) return;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) S.tile = (int)atomicAdd(cursor, 1ull);
    __syncthreads();
    const int64_t gb = S.tile;
    if (gb >= wk.total_bricks) break;
    const int ii = batch_inst(wk, gb);
    load_inst(S, wk.insts[ii]);
    __syncthreads();
    p1_dispatch<PREC>(wk, S, ii, gb);
  }
}

__global__ void __launch_bounds__(kThreads) k_pass2_batch(const Work wk) {
  Smem& S = *reinterpret_cast<Smem*>(vt_smem);
  if (wk.err[E_CODE]) return;
  const unsigned long long n = *(volatile unsigned long long*)&wk.cnt[C_P2];
  for (unsigned long long t = blockIdx.x; t < n; t += gridDim.x) {
    __syncthreads();
    const int64_t gb = wk.p2_list[t];
    const int ii = batch_inst(wk, gb);
    load_inst(S, wk.insts[ii]);
    __syncthreads();
    const Inst& I = S.inst;
    if (I.nd == 3) {
      if (I.kind == KV) p2_brick<KV, Cfg3>(wk, S, ii, gb);
      else if (I.kind == KL) p2_brick<KL, Cfg3>(wk, S, ii, gb);
      else p2_brick<KJ, Cfg3>(wk, S, ii, gb);
    } else {
      if (I.kind == KV) p2_brick<KV, Cfg2>(wk, S, ii, gb);
      else if (I.kind == KL) p2_brick<KL, Cfg2>(wk, S, ii, gb);
      else p2_brick<KJ, Cfg2>(wk, S, ii, gb);
    }
  }
}

// ------------------------------------------------------------ host launch

size_t label_smem_bytes() { return sizeof(Smem); }

void brick_dims(int nd, int cfg, int* b) {
  (void)cfg;
  if (nd == 3) { b[0] = Cfg3::BX; b[1] = Cfg3::BY; b[2] = Cfg3::BZ; }
  else { b[0] = Cfg2::BX; b[1] = Cfg2::BY; b[2] = 1; }
}

template <typename K>
static cudaError_t prep(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(Smem));
}

template <int KIND, class C>
static cudaError_t prep_kind() {
  cudaError_t e;
  if ((e = prep(k_pass1<KIND, C, P_F32>)) != cudaSuccess) return e;
  if ((e = prep(k_pass1<KIND, C, P_EXACT>)) != cudaSuccess) return e;
  return prep(k_pass2<KIND, C>);
}

// Opt every kernel into the shared memory it needs (once per process; the
// attribute is per function, not per stream, so it is set outside any capture).
cudaError_t init_label_kernels() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  cudaError_t e;
  if ((e = prep_kind<KV, Cfg3>()) != cudaSuccess || (e = prep_kind<KL, Cfg3>()) != cudaSuccess ||
      (e = prep_kind<KJ, Cfg3>()) != cudaSuccess || (e = prep_kind<KV, Cfg2>()) != cudaSuccess ||
      (e = prep_kind<KL, Cfg2>()) != cudaSuccess || (e = prep_kind<KJ, Cfg2>()) != cudaSuccess ||
      (e = prep(k_pass1_batch<P_F32>)) != cudaSuccess ||
      (e = prep(k_pass1_batch<P_EXACT>)) != cudaSuccess || (e = prep(k_pass2_batch)) != cudaSuccess)
    return e;
  done = cudaSuccess;
  return done;
}

template <int KIND, class C>
static cudaError_t launch_single(const Work& wk, const Inst& I, int prec, int p2_grid,
                                 cudaStream_t st, cudaEvent_t mid) {
  if (prec == P_F32)
    k_pass1<KIND, C, P_F32><<<(unsigned)I.n_bricks, kThreads, sizeof(Smem), st>>>(wk, I);
  else
    k_pass1<KIND, C, P_EXACT><<<(unsigned)I.n_bricks, kThreads, sizeof(Smem), st>>>(wk, I);
  if (mid) cudaEventRecord(mid, st);
  k_pass2<KIND, C><<<p2_grid, kThreads, sizeof(Smem), st>>>(wk, I);
  return cudaGetLastError();
}

// First pass, then (after the optional event `mid`) the second pass.
cudaError_t launch_label(const Work& wk, const Inst& I, int p2_grid, cudaStream_t st,
                         cudaEvent_t mid) {
  if (I.nd == 3) {
    if (I.kind == KV) return launch_single<KV, Cfg3>(wk, I, I.precision, p2_grid, st, mid);
    if (I.kind == KL) return launch_single<KL, Cfg3>(wk, I, I.precision, p2_grid, st, mid);
    return launch_single<KJ, Cfg3>(wk, I, I.precision, p2_grid, st, mid);
  }
  if (I.kind == KV) return launch_single<KV, Cfg2>(wk, I, I.precision, p2_grid, st, mid);
  if (I.kind == KL) return launch_single<KL, Cfg2>(wk, I, I.precision, p2_grid, st, mid);
  return launch_single<KJ, Cfg2>(wk, I, I.precision, p2_grid, st, mid);
}

cudaError_t launch_label_batch(const Work& wk, int prec, unsigned long long* cursor, int grid,
                               cudaStream_t st) {
  if (prec == P_F32)
    k_pass1_batch<P_F32><<<grid, kThreads, sizeof(Smem), st>>>(wk, cursor);
  else
    k_pass1_batch<P_EXACT><<<grid, kThreads, sizeof(Smem), st>>>(wk, cursor);
  k_pass2_batch<<<grid, kThreads, sizeof(Smem), st>>>(wk);
  return cudaGetLastError();
}

}  // namespace vt
