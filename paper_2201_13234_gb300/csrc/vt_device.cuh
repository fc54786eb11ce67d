// vt_device.cuh -- device-side building blocks shared by the two labelling
// passes (vt_pass1.cu, vt_pass2.cu): warp-tile geometry, bin regions, the
// periodic images of a site near a box, score bounds, the FP32 screening and
// the exact evaluation of one candidate over a lane's micro-tile.
//
// Scores are compared in "f-units", a shifted form of each score that is
// never negative, so that FP32 values order like their bit patterns:
//   Voronoi       F = D                          (D = squared distance, 1/512^2 voxel^2)
//   Laguerre      F = D - w + W                  (W = the instance's largest weight)
//   Johnson-Mehl  F = a - t_min                  (a = t + sqrt(D)/(512 v) in IEEE double,
//                                                 t_min = the instance's earliest birth)
// Each shift is common to all sites, so the argmin is unchanged.
#pragma once
#include "vt_internal.cuh"

namespace vt {

constexpr float kInf = __builtin_huge_valf();

// Warp tile geometry.  A lane owns a micro-tile of 4 x MY x MZ voxels (x runs
// of 4 for 16-byte label stores); the 32 lanes form LX x LY x LZ micro-tiles
// (the warp box); a second-pass brick is WX x WY x WZ warp boxes.
template <int MY_, int MZ_, int LX_, int LY_, int LZ_, int WX_, int WY_, int WZ_>
struct Cfg {
  static constexpr int MX = 4, MY = MY_, MZ = MZ_;
  static constexpr int LX = LX_, LY = LY_, LZ = LZ_;
  static constexpr int WX = WX_, WY = WY_, WZ = WZ_;
  static constexpr int NV = MX * MY * MZ;
  static constexpr int BXW = MX * LX, BYW = MY * LY, BZW = MZ * LZ;
  static constexpr int BX = BXW * WX, BY = BYW * WY, BZ = BZW * WZ;
  static_assert(LX * LY * LZ == 32, "32 lanes");
};
using Cfg3 = Cfg<1, 4, 2, 8, 2, 2, 2, 1>;   // warp box 8x8x8, brick 16x16x8
using Cfg3c = Cfg<1, 2, 2, 8, 2, 2, 2, 1>;  // compact: warp box 8x8x4, brick 16x16x4
using Cfg2 = Cfg<4, 1, 4, 8, 1, 2, 2, 1>;   // warp box 16x32, brick 32x64
using Cfg2c = Cfg<2, 1, 4, 8, 1, 2, 2, 1>;  // compact: warp box 16x16, brick 32x32

// Index of a tile configuration: 3D default, 3D compact, 2D default, 2D
// compact (vt_options.brick_cfg selects default or compact).
template <class C>
__host__ __device__ constexpr int cfg_index() {
  return (C::MZ > 1 ? 0 : 2) + ((C::MZ > 1 ? C::MZ : C::MY) == 4 ? 0 : 1);
}
__host__ __device__ constexpr int cfg_index(int nd, int compact) {
  return (nd == 3 ? 0 : 2) + (compact ? 1 : 0);
}

// One candidate (a site image) of a warp's list.  The image position is kept
// relative to the warp origin as exact floats (|q| < 2^24).
struct Entry {
  float qx, qy, qz;
  float a, b;   // FP32 per-site data: L (W - w); JM (t - t_min, 1/(512 v))
  float lo;     // lower bound of F over the warp box
  int id;       // site id
  int src;      // index of the site in the sorted arrays (exact data)
};

struct Region {
  int blo[3], bhi[3];  // bin index range, unwrapped on periodic axes
  int full[3];         // the range holds every bin of the axis exactly once
  int bl[3], bh[3];    // a face of the region is a real boundary (sites beyond it)
  int Rlo[3], Rhi[3];  // region extent [Rlo, Rhi) in fixed point (unwrapped)
};

// Per-instance constants of the f-units.
struct FUnits {
  long long wglob;    // L: W
  double tmin, vmax;  // JM
  float absf;         // JM: absolute error allowance (2^-48 max |t|)
  float inv_vmax_rd;  // JM: 1 / (512 vmax), rounded down
  float vmax_ru;      // JM: vmax rounded up
};

template <int KIND>
__device__ __forceinline__ FUnits load_funits(const Work& wk, int ii) {
  const IStat st = wk.istat[ii];
  FUnits u;
  u.wglob = KIND == KL ? st.wmax : 0;
  if (KIND == KJ) {
    u.tmin = dkey_inv(~st.tmin);
    u.vmax = dkey_inv(st.vmax);
    u.absf = __double2float_ru(dkey_inv(st.tabs) * 0x1p-48) + 0x1p-100f;
    u.inv_vmax_rd = __double2float_rd(__ddiv_rd(1.0, __dmul_ru(512.0, u.vmax)));
    u.vmax_ru = __double2float_ru(u.vmax);
  } else {
    u.tmin = 0.0;
    u.vmax = 1.0;
    u.absf = 0.f;
    u.inv_vmax_rd = 0.f;
    u.vmax_ru = 1.f;
  }
  return u;
}

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

// Square root by the hardware approximation (sqrt.approx.f32: at most 1 ulp
// of error per the CUDA math documentation of sqrtf without -prec-sqrt); the
// screening error budget allows 2^-20 relative.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ int wrap_bin(const Inst& I, int a, int u) {
  if (!I.per[a]) return u;
  const int nb = I.nb[a];
  // a region that is not a whole period lies within one period of [0, nb)
  int r = u < 0 ? u + nb : u >= nb ? u - nb : u;
  if ((unsigned)r >= (unsigned)nb) {
    r = u % nb;
    if (r < 0) r += nb;
  }
  return r;
}

// Axis a of the region of the bins whose sites lie within M (fixed point) of
// the centre interval [clo, chi]: clipped to the box on an open axis, each bin
// once on a periodic axis.  A site outside the region is more than M away
// from every centre of the box along that axis.  32-bit arithmetic: M is
// clamped to 2^26, beyond every period (any M >= L gives the same region).
__device__ __forceinline__ void make_region_axis(const Inst& I, int a, int clo, int chi,
                                                 int64_t M64, Region& R) {
  if (a >= I.nd) {
    R.blo[a] = R.bhi[a] = 0;
    R.full[a] = 1;
    R.bl[a] = R.bh[a] = 0;
    R.Rlo[a] = 0;
    R.Rhi[a] = I.L[a];
    return;
  }
  const int M = (int)(M64 < ((int64_t)1 << 26) ? M64 : ((int64_t)1 << 26));
  const int nb = I.nb[a], L = I.L[a], Bw = kQ * I.bw[a];
  const int xlo = clo - M, xhi = chi + M;
  if (I.per[a]) {
    const int k0 = floordiv_pos(xlo, L), k1 = floordiv_pos(xhi, L);
    const int ulo = k0 * nb + floordiv_pos(xlo - k0 * L, Bw),
              uhi = k1 * nb + floordiv_pos(xhi - k1 * L, Bw);
    if (uhi - ulo + 1 >= nb) {
      R.blo[a] = 0; R.bhi[a] = nb - 1; R.full[a] = 1; R.bl[a] = R.bh[a] = 0;
      R.Rlo[a] = 0; R.Rhi[a] = L;
    } else {
      R.blo[a] = ulo; R.bhi[a] = uhi; R.full[a] = 0; R.bl[a] = R.bh[a] = 1;
      const int kl = floordiv_pos(ulo, nb), kh = floordiv_pos(uhi, nb);
      R.Rlo[a] = kl * L + (ulo - kl * nb) * Bw;
      const int e = (uhi - kh * nb + 1) * Bw;
      R.Rhi[a] = kh * L + (e < L ? e : L);
    }
  } else {
    int ulo = floordiv_pos(xlo, Bw), uhi = floordiv_pos(xhi, Bw);
    if (ulo < 0) ulo = 0;
    if (uhi > nb - 1) uhi = nb - 1;
    R.blo[a] = ulo; R.bhi[a] = uhi;
    R.full[a] = (ulo == 0 && uhi == nb - 1);
    R.bl[a] = ulo > 0; R.bh[a] = uhi < nb - 1;
    R.Rlo[a] = ulo * Bw;
    R.Rhi[a] = (uhi + 1) * Bw < L ? (uhi + 1) * Bw : L;
  }
}

// The whole region of the centre box [clo, chi] (see make_region_axis).
__device__ __forceinline__ void make_region(const Inst& I, const int64_t* clo,
                                            const int64_t* chi, int64_t M, Region& R) {
#pragma unroll
  for (int a = 0; a < 3; a++) make_region_axis(I, a, (int)clo[a], (int)chi[a], M, R);
}

// The one or two contiguous runs of sorted sites of a bin row (by, bz) of
// region R: [s0, s0 + l0) and [s1, s1 + l1).
__device__ __forceinline__ void row_runs(const Work& wk, const Inst& I, const Region& R, int r,
                                         int& s0, int& l0, int& s1, int& l1) {
  const int ry = R.bhi[1] - R.blo[1] + 1;
  const int rz = floordiv_pos(r, ry);  // r >= 0: the quotient, without an integer division
  const int by = wrap_bin(I, 1, R.blo[1] + (r - rz * ry)), bz = wrap_bin(I, 2, R.blo[2] + rz);
  const int64_t row = I.bin_base + ((int64_t)bz * I.nb[1] + by) * I.nb[0];
  int a0 = R.blo[0], a1 = R.bhi[0], c0 = 0, c1 = -1;
  if (I.per[0] && !R.full[0]) {
    const int nb = I.nb[0];
    const int k0 = wrap_bin(I, 0, R.blo[0]), len = R.bhi[0] - R.blo[0] + 1;
    a0 = k0;
    a1 = k0 + len - 1;
    if (a1 >= nb) { c0 = 0; c1 = a1 - nb; a1 = nb - 1; }
  }
  s0 = wk.bin_start[row + a0];
  l0 = wk.bin_start[row + a1 + 1] - s0;
  s1 = 0;
  l1 = 0;
  if (c1 >= c0) {
    s1 = wk.bin_start[row + c0];
    l1 = wk.bin_start[row + c1 + 1] - s1;
  }
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

// Geometry of the warp box whose first voxel is (x0, y0, z0).
template <class C>
__device__ __forceinline__ void lane_setup_box(const Inst& I, int x0, int y0, int z0,
                                               Lane<C>& G) {
  const int lane = threadIdx.x & 31;
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

// ------------------------------------------------------------ images and bounds

// Periodic images of a site that are the nearest image for some voxel of the
// warp box: per axis the image closest to the box centre plus, when the box
// reaches past half a period from it, the neighbouring image(s).
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
  // j = k0 + cnt0 (k1 + cnt1 k2), every cnt in {1, 2, 3} and j < 27: a
  // multiply-shift divides exactly there (no integer division)
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const int c = m.cnt[a];
    const int d = c == 1 ? j : c == 2 ? (j >> 1) : ((j * 43691) >> 17);
    q[a] = m.q[a] + (m.lo[a] + (j - d * c)) * I.L[a];
    j = d;
  }
}

// Bounds of F over the box [0, h] for the image at q (relative, exact
// integers), computed in FP32 with directed rounding (and, for
// Johnson-Mehl, a relative and an absolute allowance for the double-precision
// rounding of the arrival time itself).  lo <= F(v) <= hi for every voxel v.
template <int KIND>
__device__ __forceinline__ void f_bounds(const int* q, const int* h, float2 fa, const FUnits& U,
                                         float& lo, float& hi) {
  float g[3], e[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    g[a] = (float)max(0, max(-q[a], q[a] - h[a]));
    e[a] = (float)max(q[a], h[a] - q[a]);
  }
  const float dlo = __fmaf_rd(g[0], g[0], __fmaf_rd(g[1], g[1], __fmul_rd(g[2], g[2])));
  const float dhi = __fmaf_ru(e[0], e[0], __fmaf_ru(e[1], e[1], __fmul_ru(e[2], e[2])));
  if (KIND == KV) {
    lo = dlo;
    hi = dhi;
  } else if (KIND == KL) {
    lo = __fadd_rd(dlo, __fmul_rd(fa.x, 1.0f - 0x1p-22f));
    hi = __fadd_ru(dhi, __fmul_ru(fa.x, 1.0f + 0x1p-22f));
  } else {
    const float l0 = __fmaf_rd(__fsqrt_rd(dlo), __fmul_rd(fa.y, 1.0f - 0x1p-22f),
                               __fmul_rd(fa.x, 1.0f - 0x1p-22f));
    const float h0 = __fmaf_ru(__fsqrt_ru(dhi), __fmul_ru(fa.y, 1.0f + 0x1p-22f),
                               __fmul_ru(fa.x, 1.0f + 0x1p-22f));
    lo = __fsub_rd(__fmul_rd(l0, 1.0f - 0x1p-20f), U.absf);
    hi = __fadd_ru(__fmul_ru(h0, 1.0f + 0x1p-20f), U.absf);
  }
}

// The same bounds for an image given as exact floats q relative to the box's
// first centre, box extent h (floats), FP32 site data (a, b).
template <int KIND>
__device__ __forceinline__ void f_bounds_f(float qx, float qy, float qz, float hx, float hy,
                                           float hz, float a, float b, float absf, float& lo,
                                           float& hi) {
  const float gx = fmaxf(0.f, fmaxf(-qx, qx - hx)), ex = fmaxf(qx, hx - qx);
  const float gy = fmaxf(0.f, fmaxf(-qy, qy - hy)), ey = fmaxf(qy, hy - qy);
  const float gz = fmaxf(0.f, fmaxf(-qz, qz - hz)), ez = fmaxf(qz, hz - qz);
  const float dlo = __fmaf_rd(gx, gx, __fmaf_rd(gy, gy, __fmul_rd(gz, gz)));
  const float dhi = __fmaf_ru(ex, ex, __fmaf_ru(ey, ey, __fmul_ru(ez, ez)));
  if (KIND == KV) {
    lo = dlo;
    hi = dhi;
  } else if (KIND == KL) {
    lo = __fadd_rd(dlo, __fmul_rd(a, 1.0f - 0x1p-22f));
    hi = __fadd_ru(dhi, __fmul_ru(a, 1.0f + 0x1p-22f));
  } else {
    const float l0 = __fmaf_rd(__fsqrt_rd(dlo), __fmul_rd(b, 1.0f - 0x1p-22f),
                               __fmul_rd(a, 1.0f - 0x1p-22f));
    const float h0 = __fmaf_ru(__fsqrt_ru(dhi), __fmul_ru(b, 1.0f + 0x1p-22f),
                               __fmul_ru(a, 1.0f + 0x1p-22f));
    lo = __fsub_rd(__fmul_rd(l0, 1.0f - 0x1p-20f), absf);
    hi = __fadd_ru(__fmul_ru(h0, 1.0f + 0x1p-20f), absf);
  }
}

// ------------------------------------------------------------ evaluation

// FP32 screening of one list entry over the lane's micro-tile.  F is a sum of
// non-negative terms (exact deltas, fma chain), so it is never negative and
// its bit pattern orders like its value; the key replaces the low mantissa
// bits by the entry index and each voxel keeps its two smallest keys.
template <int KIND, class C, unsigned IDXMASK>
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
        const unsigned key = (__float_as_uint(f) & ~IDXMASK) | idx;
        const int v = (k * C::MY + j) * 4 + i;
        const unsigned hi = max(k1[v], key);
        k1[v] = min(k1[v], key);
        k2[v] = min(k2[v], hi);
      }
    }
  }
}

// Absolute-scale keys (lists of at most 128 entries).  The tile's scores are
// computed as F + S, S a power of two at least twice every voxel's best score
// and at least 1/12 of every listed score: rounding then quantizes F to
// multiples of q = ulp(S), and bits(F + S) grows with F.  The key is
// bits(F + S) * 129 + index, reduced modulo 2^32 (the caller passes
// index - 129 bits(S)): (bits(F + S) - bits(S)) * 129 + index, below 2^32 while
// F + S < 16 S.  An integer multiply-add packs the index (the FMA pipe), so the
// top-2 update takes three ALU operations instead of four.
constexpr unsigned kQMul = 129;  // > the largest list index (127)

// Smallest power of two >= max(x, 1) (x finite and non-negative).
__device__ __forceinline__ float pow2_ceil(float x) {
  unsigned b = __float_as_uint(fmaxf(x, 1.0f));
  if (b & 0x7FFFFFu) b = (b & 0x7F800000u) + 0x800000u;
  return __uint_as_float(b);
}

template <int KIND, class C>
__device__ __forceinline__ void eval_f32q(const Entry& e, unsigned idxq, float S, const Lane<C>& G,
                                          unsigned (&k1)[C::NV], unsigned (&k2)[C::NV]) {
  const float a = e.a + S;
  float dx[4];
#pragma unroll
  for (int i = 0; i < 4; i++) dx[i] = G.cx[i] - e.qx;
#pragma unroll
  for (int k = 0; k < C::MZ; k++) {
    const float dz = G.cz[k] - e.qz;
#pragma unroll
    for (int j = 0; j < C::MY; j++) {
      const float dy = G.cy[j] - e.qy;
      const float base = (KIND == KJ) ? fmaf(dz, dz, dy * dy) : fmaf(dz, dz, fmaf(dy, dy, a));
#pragma unroll
      for (int i = 0; i < 4; i++) {
        float f = fmaf(dx[i], dx[i], base);
        if (KIND == KJ) f = fmaf(sqrt_approx(f), e.b, a);
        const unsigned key = __float_as_uint(f) * kQMul + idxq;
        const int v = (k * C::MY + j) * 4 + i;
        const unsigned hi = max(k1[v], key);
        k1[v] = min(k1[v], key);
        k2[v] = min(k2[v], hi);
      }
    }
  }
}

// The FP32 value F + S of an absolute-scale key.
__device__ __forceinline__ float qkey_value(unsigned key, unsigned sbits) {
  return __uint_as_float(key / kQMul + sbits);
}

// Exact data of a site: L weight; JM birth time and 512 v.
struct ExactSite {
  long long w;
  double t, den;
};

template <int KIND>
__device__ __forceinline__ ExactSite exact_site(const Work& wk, int src) {
  ExactSite x;
  x.w = 0;
  x.t = 0.0;
  x.den = 1.0;
  if (KIND != KV) {
    const longlong2 a = wk.saux[src];
    if (KIND == KL) x.w = a.x;
    else { x.t = __longlong_as_double(a.x); x.den = __longlong_as_double(a.y); }
  }
  return x;
}

// Exact evaluation of one list entry over the micro-tile: lexicographic
// minimum of (score, id).  V/L: int64 D - w; JM: IEEE double
// t + sqrt(D) / (512 v) in that order, each operation rounded to nearest.
template <int KIND, class C>
__device__ __forceinline__ void eval_exact(const Entry& e, const ExactSite& x, const Lane<C>& G,
                                           long long (&bs)[C::NV], double (&ba)[C::NV],
                                           int (&bid)[C::NV]) {
  const int qx = __float2int_rn(e.qx), qy = __float2int_rn(e.qy), qz = __float2int_rn(e.qz);
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
          const double a = __dadd_rn(x.t, __ddiv_rn(__dsqrt_rn((double)D), x.den));
          if (a < ba[v] || (a == ba[v] && e.id < bid[v])) { ba[v] = a; bid[v] = e.id; }
        } else {
          const long long s = KIND == KL ? D - x.w : D;
          if (s < bs[v] || (s == bs[v] && e.id < bid[v])) { bs[v] = s; bid[v] = e.id; }
        }
      }
    }
}

// f-units upper bound of an exact best score.
template <int KIND>
__device__ __forceinline__ float exact_to_f_ru(long long s, double a, const FUnits& U) {
  if (KIND == KJ) return __double2float_ru(__dsub_ru(a, U.tmin));
  if (KIND == KL) return __ll2float_ru(s + U.wglob);
  return __ll2float_ru(s);
}

// Largest exact best score over the lane's voxels inside the grid, as a float
// rounded up (-inf for a lane without one).  exact_to_f_ru is monotone in the
// score, so the lane's largest score is found first (64-bit integer compares;
// Johnson-Mehl times through their order-preserving keys) and converted once:
// 64-bit conversions and compares run on the FP64 pipe, which is narrow here.
template <int KIND, int NV>
__device__ __forceinline__ float lane_max_exact_f_ru(unsigned vmask, const long long (&bs)[NV],
                                                     const double (&ba)[NV], const FUnits& U) {
  if (!(vmask & ((NV < 32 ? (1u << NV) : 0u) - 1u))) return -kInf;
  if (KIND == KJ) {
    unsigned long long mk = 0;
#pragma unroll
    for (int v = 0; v < NV; v++)
      if (vmask & (1u << v)) mk = mk > dkey(ba[v]) ? mk : dkey(ba[v]);
    return exact_to_f_ru<KIND>(0, dkey_inv(mk), U);
  }
  long long mx = bs[0];
  bool any = false;
#pragma unroll
  for (int v = 0; v < NV; v++)
    if (vmask & (1u << v)) {
      mx = any && mx > bs[v] ? mx : bs[v];
      any = true;
    }
  return exact_to_f_ru<KIND>(mx, 0.0, U);
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

// Same label for every voxel of the micro-tile.
template <class C>
__device__ __forceinline__ void store_uniform(const Inst& I, const Lane<C>& G, int id) {
  int lab[C::NV];
#pragma unroll
  for (int v = 0; v < C::NV; v++) lab[v] = id;
  store_labels<C>(I, G, lab);
}

}  // namespace vt
