// vt_pass2.cu -- second labelling pass: bricks the first pass left (their
// candidate lists did not fit, even in its culling re-run) are labelled by
// growing rings of bins.
//
// This is the GPU form of the paper's step 2 (Algorithms 2 and 3): voxels not
// settled by the first step are settled from a larger candidate set, at worst
// from every site.  One CTA takes a brick (2 x 2 x 1 warp tiles).  Round k
// stages, in chunks that fit in shared memory, the sites of the bins in the
// ring between the region of margin M_{k-1} and M_k = 2 M_{k-1} + one bin
// (M_0 and an upper bound of the brick's best scores come from the first
// pass, so that one round usually certifies the brick),
// skipping every bin whose lower bound already exceeds the brick's largest
// best score; each warp scores the staged sites of its tile exactly
// (int64 / IEEE double, lexicographic (score, id)).  A voxel is certified once
// its best score is below the bound every site outside the region must
// exceed; the rings stop when every voxel is certified or the region covers
// the whole grid.
#include "vt_device.cuh"

namespace vt {

constexpr int kP2Warps = 4;
constexpr int kP2Threads = 32 * kP2Warps;
constexpr int kP2Cap = 384;    // staged sites per chunk
constexpr int kP2Lcap = 256;   // list entries per warp
constexpr int kP2Group = kP2Threads;  // bins tested per round of the ring walk

struct P2Smem {
  Inst inst;
  Region R, P;
  int4 spos[kP2Cap];
  float2 sfa[kP2Cap];
  int ssrc[kP2Cap];
  Entry list[kP2Warps][kP2Lcap];
  short order[kP2Warps][kP2Lcap];  // evaluation order of a warp's list
  short elig[kP2Warps][kP2Lcap];   // list entries not yet excluded by the bound
  float elo[kP2Warps][kP2Lcap];    // and their lower bounds
  int seg_src[kP2Group + 1];
  int seg_off[kP2Group + 1];
  int wtot[kP2Warps];
  int nstaged, has_prev;
  unsigned int ukey;  // brick-wide upper bound of the best scores (ordered float key)
};

// Exclusive scan of a[0..n) in shared memory (n <= 8 * kP2Threads); returns
// the total.  Every thread of the CTA calls it.
__device__ int block_scan(int* a, int n, int* wtot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + kP2Threads - 1) / kP2Threads;
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
  for (int w = 0; w < kP2Warps; w++) {
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

// Smallest distance (fixed point) from centre coordinate c to a real face of
// the region along axis a; INT_MAX if the axis has none.
__device__ __forceinline__ int face_gap(const Region& R, int a, int c) {
  int g = 0x7FFFFFFF;
  if (R.bl[a]) g = min(g, c - R.Rlo[a] + 1);
  if (R.bh[a]) g = min(g, R.Rhi[a] - c);
  return g;
}

template <class C>
__device__ __forceinline__ int voxel_gap(const Region& R, const Lane<C>& G, int i, int j, int k) {
  const int cx = G.ox + (int)G.cx[i], cy = G.oy + (int)G.cy[j], cz = G.oz + (int)G.cz[k];
  return min(face_gap(R, 0, cx), min(face_gap(R, 1, cy), face_gap(R, 2, cz)));
}

// Certified: the best exact score is below the lower bound of the score of any
// site outside the region at gap g (V: g^2; L: g^2 - W; JM: t_min + g/(512 v_max)
// in the score's own rounded operations, which are monotone).
template <int KIND>
__device__ __forceinline__ bool certified_exact(const FUnits& U, int g, long long bs, double ba) {
  if (g == 0x7FFFFFFF) return true;
  if (KIND == KJ) {
    const double lb = __dadd_rn(U.tmin, __ddiv_rn((double)g, __dmul_rn(512.0, U.vmax)));
    return ba < lb;
  }
  return bs < (long long)g * g - U.wglob;
}

template <int KIND, class C>
__device__ __forceinline__ float u_exact2(const Lane<C>& G, const long long (&bs)[C::NV],
                                          const double (&ba)[C::NV], const FUnits& U) {
  return warp_max(lane_max_exact_f_ru<KIND, C::NV>(G.vmask, bs, ba, U));
}

// Score the staged slots [0, n) into the warp's exact state; U is the warp's
// running bound (f-units).
template <int KIND, class C>
__device__ void p2_consume(const Work& wk, P2Smem& S, const Lane<C>& G, const FUnits& U, int n,
                           long long (&bs)[C::NV], double (&ba)[C::NV], int (&bid)[C::NV],
                           float& Uw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Inst& I = S.inst;
  const int h[3] = {G.hx, G.hy, G.hz};
  Entry* list = S.list[warp];
  short* order = S.order[warp];
  // The list is scored in increasing order of its lower bounds (a rank sort,
  // ties by position), so that the running bound tightens early; the first
  // entry whose lower bound exceeds it ends the list.  The running bound costs
  // a conversion per voxel and a warp reduction: it is refreshed after the
  // first evaluations, then every fourth (a stale bound is still an upper
  // bound, it only prunes less).
  int evals = 0;
  float hmin = kInf;  // smallest upper bound over the tile of an image seen so far
  short* elig = S.elig[warp];
  float* elo = S.elo[warp];
  auto run = [&](int len) {
    Uw = fminf(Uw, warp_min(hmin));
    __syncwarp();
    // the entries still within the bound, compacted; then their ranks
    int ne = 0;
    for (int e0 = 0; e0 < len; e0 += 32) {
      const int e = e0 + lane;
      const float le = e < len ? list[e].lo : 0.f;
      const bool ok = e < len && le <= Uw;
      const unsigned bal = __ballot_sync(0xffffffffu, ok);
      const int pos = ne + __popc(bal & ((1u << lane) - 1));
      if (ok) {
        elig[pos] = (short)e;
        elo[pos] = le;
      }
      ne += __popc(bal);
    }
    __syncwarp();
    for (int i0 = 0; i0 < ne; i0 += 32) {
      const int i = i0 + lane;
      const float li = i < ne ? elo[i] : 0.f;
      int r = 0;
      for (int f = 0; f < ne; f++) {
        const float lf = elo[f];
        r += (lf < li) || (lf == li && f < i);
      }
      if (i < ne) order[r] = elig[i];
    }
    __syncwarp();
    for (int r = 0; r < ne; r++) {
      const Entry x = list[order[r]];
      if (x.lo > Uw) break;
      eval_exact<KIND, C>(x, exact_site<KIND>(wk, x.src), G, bs, ba, bid);
      if (++evals <= 3 || (evals & 3) == 0) Uw = fminf(Uw, u_exact2<KIND, C>(G, bs, ba, U));
    }
    __syncwarp();
  };
  int len = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    Img m;
    int cnt = 0;
    int4 p = make_int4(0, 0, 0, 0);
    float2 fa = make_float2(0.f, 0.f);
    if (i < n) {
      p = S.spos[i];
      fa = S.sfa[i];
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
        float hi;
        f_bounds<KIND>(q, h, fa, U, lo, hi);
        hmin = fminf(hmin, hi);
        keep = lo <= Uw;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (len + __popc(bal) > kP2Lcap) {
        run(len);
        len = 0;
      }
      const int pos = len + __popc(bal & ((1u << lane) - 1));
      if (keep) {
        Entry e;
        e.qx = (float)q[0]; e.qy = (float)q[1]; e.qz = (float)q[2];
        e.a = fa.x; e.b = fa.y;
        e.lo = lo;
        e.id = p.w;
        e.src = S.ssrc[i];
        list[pos] = e;
      }
      len += __popc(bal);
    }
  }
  run(len);
}

// Label brick gbrick.  M0 (fixed point) and UB (f-units) come from the first
// pass: when UB is finite, every voxel's best score is at most UB and the
// region of margin M0 holds every possible winner.
template <int KIND, class C>
__device__ void p2_brick(const Work& wk, P2Smem& S, int ii, int64_t gbrick, int64_t M0,
                         float UB) {
  const Inst& I = S.inst;
  const int tid = threadIdx.x, warp = tid >> 5;
  const FUnits U = load_funits<KIND>(wk, ii);
  const int64_t lb = gbrick - I.brick_base;
  const unsigned ul = (unsigned)lb, b0 = (unsigned)I.bricks[0], b1 = (unsigned)I.bricks[1];
  const unsigned rr = ul / b0;  // brick indices fit 32 bits
  const int bxi = (int)(ul - rr * b0);
  const int bzi = (int)(rr / b1), byi = (int)(rr - (unsigned)bzi * b1);
  const int x0 = bxi * C::BX, y0 = byi * C::BY, z0 = bzi * C::BZ;
  const int x1 = min(x0 + C::BX, I.n[0]) - 1, y1 = min(y0 + C::BY, I.n[1]) - 1,
            z1 = min(z0 + C::BZ, I.n[2]) - 1;
  const int64_t clo[3] = {(int64_t)kQ * x0 + kQ / 2, (int64_t)kQ * y0 + kQ / 2,
                          (int64_t)kQ * z0 + kQ / 2};
  const int64_t chi[3] = {(int64_t)kQ * x1 + kQ / 2, (int64_t)kQ * y1 + kQ / 2,
                          (int64_t)kQ * z1 + kQ / 2};
  if (tid == 0) {
    S.has_prev = 0;
    S.ukey = fkey(UB < kInf ? UB : kInf);
  }
  __syncthreads();
  Lane<C> G;
  {
    const int wx = warp % C::WX, wy = (warp / C::WX) % C::WY, wz = warp / (C::WX * C::WY);
    lane_setup_box<C>(I, x0 + wx * C::BXW, y0 + wy * C::BYW, z0 + wz * C::BZW, G);
  }
  long long bs[C::NV];
  double ba[C::NV];
  int bid[C::NV];
#pragma unroll
  for (int v = 0; v < C::NV; v++) {
    bs[v] = 0x7FFFFFFFFFFFFFFFll;
    ba[v] = kInf;
    bid[v] = 0x7FFFFFFF;
  }
  float Uw = UB < kInf ? UB : kInf;
  int64_t M = M0 > 0 ? M0 : (int64_t)kQ * I.margin;
  const int bwmax = max(I.bw[0], max(I.bw[1], I.bw[2]));
#pragma unroll 1
  for (;;) {
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
#pragma unroll 1
    for (long long g0 = 0; g0 < nbins; g0 += kP2Group) {
      const long long f = g0 + tid;
      int cnt = 0, src = 0;
      if (f < nbins) {
        const int ub[3] = {R.blo[0] + (int)(f % ex), R.blo[1] + (int)((f / ex) % ey),
                           R.blo[2] + (int)(f / ((long long)ex * ey))};
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
          if (cnt > 0 && Ub < kInf) {
            // lower bound (f-units) of any site of the bin over the brick
            long long dlo = 0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
              if (a >= I.nd) continue;
              const int64_t g = bin_gap(I, a, wb[a], clo[a], chi[a]);
              dlo += (long long)(g * g);
            }
            float lbf;
            if (KIND == KV) {
              lbf = __ll2float_rd(dlo);
            } else if (KIND == KL) {
              lbf = __ll2float_rd(dlo - (long long)wk.bstat[2 * gb] + U.wglob);
            } else {
              const double tm = dkey_inv(~wk.bstat[2 * gb]), vm = dkey_inv(wk.bstat[2 * gb + 1]);
              const double x = __ddiv_rd(__dsqrt_rd((double)dlo), __dmul_ru(512.0, vm));
              lbf = __fsub_rd(__double2float_rd(__dadd_rd(__dsub_rd(tm, U.tmin), x) *
                                                (1.0 - 0x1p-40)),
                              U.absf);
            }
            if (lbf > Ub) cnt = 0;
          }
        }
      }
      S.seg_src[tid] = src;
      S.seg_off[tid] = cnt;
      __syncthreads();
      const int gtot = block_scan(S.seg_off, kP2Group, S.wtot);
      if (tid == 0) S.seg_off[kP2Group] = gtot;
      __syncthreads();
      for (int done = 0; done < gtot;) {
        const int room = kP2Cap - S.nstaged;
        const int take = min(room, gtot - done);
        for (int i = tid; i < take; i += kP2Threads) {
          const int gi = done + i;
          int lo = 0, hi = kP2Group - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.seg_off[mid] <= gi) lo = mid; else hi = mid - 1;
          }
          const int s = S.seg_src[lo] + (gi - S.seg_off[lo]);
          const int d = S.nstaged + i;
          S.spos[d] = wk.spos[s];
          S.sfa[d] = KIND == KV ? make_float2(0.f, 0.f) : wk.sfa[s];
          S.ssrc[d] = s;
        }
        __syncthreads();
        done += take;
        const int now = S.nstaged + take;
        if (now == kP2Cap) {
          if (G.active) p2_consume<KIND, C>(wk, S, G, U, now, bs, ba, bid, Uw);
          __syncthreads();
          if (tid == 0) S.nstaged = 0;
        } else if (tid == 0) {
          S.nstaged = now;
        }
        __syncthreads();
      }
    }
    if (S.nstaged > 0 && G.active) p2_consume<KIND, C>(wk, S, G, U, S.nstaged, bs, ba, bid, Uw);
    __syncthreads();
    if (tid == 0) S.ukey = fkey(-kInf);
    __syncthreads();
    if ((tid & 31) == 0 && G.active) atomicMax(&S.ukey, fkey(Uw));
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
                !certified_exact<KIND>(U, voxel_gap<C>(R, G, i, j, k), bs[v], ba[v]))
              cert = false;
          }
    }
    const int all = __syncthreads_and(cert);
    if (all || (R.full[0] && R.full[1] && R.full[2])) break;
    if (tid == 0) {
      S.P = R;
      S.has_prev = 1;
    }
    M = 2 * M + (int64_t)kQ * bwmax;
    __syncthreads();
  }
  if (G.active) store_labels<C>(I, G, bid);
}

__device__ __forceinline__ void load_inst(P2Smem& S, const Inst& src) {
  const int words = sizeof(Inst) / 4;
  const int* s = reinterpret_cast<const int*>(&src);
  int* d = reinterpret_cast<int*>(&S.inst);
  for (int i = threadIdx.x; i < words; i += kP2Threads) d[i] = s[i];
}

extern __shared__ __align__(16) unsigned char vt_p2_smem[];

template <int KIND, class C>
__global__ void __launch_bounds__(kP2Threads) k_pass2(const Work wk, const __grid_constant__ Inst one) {
  P2Smem& S = *reinterpret_cast<P2Smem*>(vt_p2_smem);
  if (wk.err[E_CODE]) return;
  const unsigned long long n = *(volatile unsigned long long*)&wk.cnt[C_P2];
  if (blockIdx.x >= n) return;
  load_inst(S, one);
  for (unsigned long long t = blockIdx.x; t < n; t += gridDim.x) {
    const int64_t gb = wk.p2_list[3 * t];
    if (wk.p2_flag[gb] == kDeferDone) continue;  // settled by the first pass's re-run
    __syncthreads();
    p2_brick<KIND, C>(wk, S, 0, gb, wk.p2_list[3 * t + 1], __int_as_float(wk.p2_list[3 * t + 2]));
  }
}

template <class C>
__device__ __forceinline__ void p2_brick_kind(const Work& wk, P2Smem& S, int ii, int64_t gb,
                                              int64_t M0, float UB) {
  if (S.inst.kind == KV) p2_brick<KV, C>(wk, S, ii, gb, M0, UB);
  else if (S.inst.kind == KL) p2_brick<KL, C>(wk, S, ii, gb, M0, UB);
  else p2_brick<KJ, C>(wk, S, ii, gb, M0, UB);
}

__global__ void __launch_bounds__(kP2Threads) k_pass2_batch(const Work wk) {
  P2Smem& S = *reinterpret_cast<P2Smem*>(vt_p2_smem);
  if (wk.err[E_CODE]) return;
  const unsigned long long n = *(volatile unsigned long long*)&wk.cnt[C_P2];
  for (unsigned long long t = blockIdx.x; t < n; t += gridDim.x) {
    const int64_t gb = wk.p2_list[3 * t];
    if (wk.p2_flag[gb] == kDeferDone) continue;
    __syncthreads();
    const int64_t M0 = wk.p2_list[3 * t + 1];
    const float UB = __int_as_float(wk.p2_list[3 * t + 2]);
    const int ii = find_inst(wk.insts, wk.n_inst, gb, [](const Inst& x) { return x.brick_base; });
    load_inst(S, wk.insts[ii]);
    __syncthreads();
    const Inst& I = S.inst;
    const int ci = cfg_index(I.nd, I.cfg);
    if (ci == 0) p2_brick_kind<Cfg3>(wk, S, ii, gb, M0, UB);
    else if (ci == 1) p2_brick_kind<Cfg3c>(wk, S, ii, gb, M0, UB);
    else if (ci == 2) p2_brick_kind<Cfg2>(wk, S, ii, gb, M0, UB);
    else p2_brick_kind<Cfg2c>(wk, S, ii, gb, M0, UB);
  }
}

// ------------------------------------------------------------ host side

template <typename K>
static cudaError_t prep(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(P2Smem));
}

cudaError_t init_pass2() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  cudaError_t e;
#define VT_PREP(C)                                                                         \
  if ((e = prep(k_pass2<KV, C>)) != cudaSuccess || (e = prep(k_pass2<KL, C>)) != cudaSuccess || \
      (e = prep(k_pass2<KJ, C>)) != cudaSuccess)                                              \
    return e;
  VT_PREP(Cfg3) VT_PREP(Cfg3c) VT_PREP(Cfg2) VT_PREP(Cfg2c)
#undef VT_PREP
  if ((e = prep(k_pass2_batch)) != cudaSuccess) return e;
  done = cudaSuccess;
  return done;
}

template <class C>
static void launch_p2(const Work& wk, const Inst& I, int grid, cudaStream_t st) {
  const size_t sm = sizeof(P2Smem);
  if (I.kind == KV) k_pass2<KV, C><<<grid, kP2Threads, sm, st>>>(wk, I);
  else if (I.kind == KL) k_pass2<KL, C><<<grid, kP2Threads, sm, st>>>(wk, I);
  else k_pass2<KJ, C><<<grid, kP2Threads, sm, st>>>(wk, I);
}

cudaError_t launch_pass2(const Work& wk, const Inst& I, int grid, cudaStream_t st) {
  const int ci = cfg_index(I.nd, I.cfg);
  if (ci == 0) launch_p2<Cfg3>(wk, I, grid, st);
  else if (ci == 1) launch_p2<Cfg3c>(wk, I, grid, st);
  else if (ci == 2) launch_p2<Cfg2>(wk, I, grid, st);
  else launch_p2<Cfg2c>(wk, I, grid, st);
  return cudaGetLastError();
}

cudaError_t launch_pass2_batch(const Work& wk, int grid, cudaStream_t st) {
  k_pass2_batch<<<grid, kP2Threads, sizeof(P2Smem), st>>>(wk);
  return cudaGetLastError();
}

}  // namespace vt
