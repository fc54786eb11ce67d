// vt_bin.cu -- validation and deterministic counting-sort binning of sites.
//
// The paper keeps no spatial index (its step 1 loops over the sites, Section
// 3.2.2); the GPU path needs one to find, for a block of voxels, the sites
// that can win there.  Sites are sorted into a uniform grid of bins (bin
// width bw voxels per axis, x fastest) by a counting sort:
//   k_count     validate each site, histogram of bins, per-bin and
//               per-instance statistics (Laguerre max w; JM min t, max |t|,
//               max v) with integer atomics;
//   k_scan_*    exclusive scan of the histogram (three small kernels);
//   k_scatter   record each site's index at bin_start + atomic cursor
//               (unordered within the bin);
//   k_rank      place each site at bin_start + (number of sites of its bin
//               with a smaller index): the result is sorted by (bin, id) and
//               does not depend on the order in which atomics were served.
// All instances of a batch are binned by the same launches (concatenated
// arrays, instance found by binary search).
#include "vt_internal.cuh"

namespace vt {

constexpr int kScanTile = 2048;  // bins per scan block (256 threads x 8)

struct SiteCtx {
  const Inst* I;
  int ii;
  int64_t s;
};

__device__ __forceinline__ SiteCtx site_ctx(const Work& wk, const Inst& one, int64_t g) {
  SiteCtx c;
  if (wk.insts) {
    c.ii = find_inst(wk.insts, wk.n_inst, g, [](const Inst& I) { return I.site_base; });
    c.I = &wk.insts[c.ii];
  } else {
    c.ii = 0;
    c.I = &one;
  }
  c.s = g - c.I->site_base;
  return c;
}

// atomicMax of x into a per-instance word: the lanes of the warp that reach it
// for the same instance reduce first (two 32-bit reductions give the 64-bit
// maximum), so that one atomic per warp and instance is issued.
__device__ __forceinline__ void inst_max(unsigned long long* addr, unsigned long long x, int ii) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, ii);
  const unsigned hi = __reduce_max_sync(peers, (unsigned)(x >> 32));
  const unsigned lo = __reduce_max_sync(peers, (unsigned)(x >> 32) == hi ? (unsigned)x : 0u);
  if ((threadIdx.x & 31) == __ffs(peers) - 1)
    atomicMax(addr, ((unsigned long long)hi << 32) | lo);
}
__device__ __forceinline__ void inst_max(long long* addr, unsigned long long x, int ii) {
  inst_max(reinterpret_cast<unsigned long long*>(addr), x, ii);
}

__global__ void k_count(const Work wk, const __grid_constant__ Inst one, int skip_pruned) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= wk.total_sites) return;
  if (skip_pruned && wk.pruned[g]) {  // binning again without the discarded sites
    wk.site_bin[g] = -1;
    return;
  }
  SiteCtx c = site_ctx(wk, one, g);
  const Inst& I = *c.I;
  const int nd = I.nd;
  int q[3] = {0, 0, kQ / 2};
  bool ok = true;
  for (int a = 0; a < nd; a++) {
    q[a] = I.sites[c.s * nd + a];
    ok = ok && q[a] >= 0 && q[a] < I.L[a];
  }
  long long w = 0;
  double t = 0.0, v = 0.0;
  if (I.kind == KL) {
    w = I.w[c.s];
    ok = ok && w >= 0 && w < (1ll << 52);
  } else if (I.kind == KJ) {
    t = I.t[c.s];
    v = I.v[c.s];
    ok = ok && isfinite(t) && fabs(t) < 1099511627776.0 /* 2^40 */ && isfinite(v) &&
         v >= 1e-12 && v <= 1e12;
  }
  if (!ok) {
    set_error(wk.err, 2 /* VT_ERR_RANGE */, c.ii, c.s);
    wk.site_bin[g] = -1;
    return;
  }
  int64_t b = 0;
  for (int a = 2; a >= 0; a--) b = b * I.nb[a] + q[a] / (kQ * I.bw[a]);
  int64_t gb = I.bin_base + b;
  wk.site_bin[g] = (int32_t)gb;
  atomicAdd(&wk.bin_count[gb], 1);
  IStat* st = &wk.istat[c.ii];
  if (I.kind == KL) {
    atomicMax(&wk.bstat[2 * gb], (unsigned long long)w);
    inst_max(&st->wmax, (unsigned long long)w, c.ii);
  } else if (I.kind == KJ) {
    // min t stored as max of the complemented key; the block is zero-initialised
    atomicMax(&wk.bstat[2 * gb], ~dkey(t));
    atomicMax(&wk.bstat[2 * gb + 1], dkey(v));
    inst_max(&st->tmin, ~dkey(t), c.ii);
    inst_max(&st->tabs, dkey(fabs(t)), c.ii);
    inst_max(&st->vmax, dkey(v), c.ii);
  }
}

// Local exclusive scan of kScanTile bins per block; zeroes the counts so that
// they can serve as scatter cursors.
__global__ void k_scan_local(const Work wk) {
  __shared__ int warp_sum[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + tid * 8;
  int v[8], s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    int64_t b = base + i;
    v[i] = b < wk.total_bins ? wk.bin_count[b] : 0;
    s += v[i];
  }
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[warp] = x;
  __syncthreads();
  int wp = 0, tot = 0;
  for (int w = 0; w < 8; w++) {
    if (w < warp) wp += warp_sum[w];
    tot += warp_sum[w];
  }
  int run = wp + x - s;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    int64_t b = base + i;
    if (b < wk.total_bins) {
      wk.bin_start[b] = run;
      wk.bin_count[b] = 0;
    }
    run += v[i];
  }
  if (tid == 0) wk.scan_blk[blockIdx.x] = tot;
}

// Exclusive scan of the block totals (one block); the grand total goes to
// scan_blk[n_scan_blocks].
__global__ void k_scan_top(const Work wk) {
  __shared__ int part[1024];
  const int n = wk.n_scan_blocks, tid = threadIdx.x, T = blockDim.x;
  const int per = (n + T - 1) / T;
  const int beg = min(tid * per, n), end = min(beg + per, n);
  int s = 0;
  for (int i = beg; i < end; i++) s += wk.scan_blk[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < T; i++) {
      int v = part[i];
      part[i] = run;
      run += v;
    }
    wk.scan_blk[n] = run;
  }
  __syncthreads();
  int run = part[tid];
  for (int i = beg; i < end; i++) {
    int v = wk.scan_blk[i];
    wk.scan_blk[i] = run;
    run += v;
  }
}

__global__ void k_scan_add(const Work wk) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < wk.total_bins) wk.bin_start[b] += wk.scan_blk[b / kScanTile];
  if (b == 0) wk.bin_start[wk.total_bins] = wk.scan_blk[wk.n_scan_blocks];
}

// Scatter the site ids into their bins (unordered within a bin).
__global__ void k_scatter(const Work wk, int32_t* tid_of) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= wk.total_sites) return;
  int32_t gb = wk.site_bin[g];
  if (gb < 0) return;
  int pos = wk.bin_start[gb] + atomicAdd(&wk.bin_count[gb], 1);
  tid_of[pos] = (int32_t)g;
}

// Final placement sorted by (bin, id): a site goes to bin_start + the number
// of sites of its bin with a smaller global index; it also writes the exact
// and the FP32 per-site data that the labelling kernels stage.
__global__ void k_rank(const Work wk, const __grid_constant__ Inst one, const int32_t* tid_of) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= wk.total_sites) return;
  int32_t gb = wk.site_bin[g];
  if (gb < 0) return;
  SiteCtx c = site_ctx(wk, one, g);
  const Inst& I = *c.I;
  int q[3] = {0, 0, kQ / 2};
  for (int a = 0; a < I.nd; a++) q[a] = I.sites[c.s * I.nd + a];
  int beg = wk.bin_start[gb], end = beg + wk.bin_count[gb];
  int rank = 0;
  for (int k = beg; k < end; k++) rank += tid_of[k] < (int32_t)g;
  int dst = beg + rank;
  wk.spos[dst] = make_int4(q[0], q[1], q[2], (int)c.s);
  const IStat st = wk.istat[c.ii];
  if (I.kind == KL) {
    long long w = I.w[c.s];
    wk.saux[dst] = make_longlong2(w, 0);
    wk.sfa[dst] = make_float2(__ll2float_rn((long long)st.wmax - w), 0.f);
  } else if (I.kind == KJ) {
    double t = I.t[c.s], v = I.v[c.s];
    double den = __dmul_rn(512.0, v);
    wk.saux[dst] = make_longlong2(__double_as_longlong(t), __double_as_longlong(den));
    double tmin = dkey_inv(~st.tmin);
    wk.sfa[dst] = make_float2(__double2float_rn(__dsub_rn(t, tmin)),
                              __double2float_rn(__ddiv_rn(1.0, den)));
  }
}

// Johnson-Mehl: discard the sites that another site reaches before they are
// born (Section 3.3, remark after the choice of t0: such sites create no
// cell).  Site s is discarded when a site j with v_j >= v_s satisfies
// t_j + |q_s - q_j| / (512 v_j) < t_s by more than a rounding margin, the
// arrival bounded from above by directed rounding.  Then for every voxel x
//   t_j + |x - q_j| / (512 v_j) <= t_j + |q_s - q_j| / (512 v_j) + |x - q_s| / (512 v_s)
//                               <  t_s + |x - q_s| / (512 v_s)
// (triangle inequality, which also holds for the periodic minimum-image
// distance), so s arrives later everywhere; the margin, 2^-40 of the scores'
// magnitudes, exceeds the rounding of both scores, so s also loses in the
// scores' own arithmetic and can never win or tie.  Only the bins within s's
// reach (t_s - t_min) 512 v_max are searched, at most kPruneBins per side: a
// site that is not found dominated is kept.
constexpr int kPruneBins = 3;

__device__ __forceinline__ int wrap_axis(const Inst& I, int a, int u) {
  if (!I.per[a]) return u;
  const int r = u % I.nb[a];
  return r < 0 ? r + I.nb[a] : r;
}

// One warp per site: the lanes share out the bins of the search box, 32 at a
// time, and the warp stops at the first round in which a lane found a
// dominating site.  Each candidate is first screened in single precision on
// the binned copies (t_j - t_min, 1 / (512 v_j)): the single-precision
// estimate of t_s - a_j(q_s) has a relative error below 2^-21 of
// (t_s - t_min) + (a_j - t_min), so an estimate below -2^-16 of that sum
// proves that j arrives after s's birth and the exact test is skipped.
__global__ void __launch_bounds__(128) k_jm_prune(const Work wk, const __grid_constant__ Inst one) {
  const int lane = threadIdx.x & 31;
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= wk.total_sites) return;  // uniform across the warp
  const SiteCtx c = site_ctx(wk, one, g);
  const Inst& I = *c.I;
  bool out = false;
  if (I.kind == KJ && wk.site_bin[g] >= 0) {
    int q[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1}, hp[3] = {0, 0, 0};
    for (int a = 0; a < I.nd; a++) q[a] = I.sites[c.s * I.nd + a];
    const double ts = I.t[c.s], dens = __dmul_rn(512.0, I.v[c.s]);
    const IStat st = wk.istat[c.ii];
    const double tmin = dkey_inv(~st.tmin), vmax = dkey_inv(st.vmax);
    const double reach = __dmul_ru(__dmul_ru(__dsub_ru(ts, tmin), 512.0), vmax);
    // longest arrival delay of s (time units), rounded up in single precision:
    // only its size matters (it scales the margin), and a larger one is safe
    long long diag = 0;
    for (int a = 0; a < I.nd; a++) diag += (long long)I.n[a] * I.n[a];
    const double span = (double)__fmul_ru(
        __fdiv_ru(__fmul_ru(__fsqrt_ru(__ll2float_ru(diag)), 512.0f), __double2float_rd(dens)),
        1.0f + 0x1p-20f);
    const float tsr = __double2float_rn(__dsub_rn(ts, tmin));
    for (int a = 0; a < I.nd; a++) {
      // the bins within reach of q (fixed point, rounded up; capped past the
      // kPruneBins bins searched), in integer arithmetic
      const int Bw = kQ * I.bw[a];
      const int b0 = q[a] / Bw;
      const int ri = __double2int_ru(fmin(reach, (double)((kPruneBins + 1) * Bw)));
      int l = max(floordiv_pos(q[a] - ri, Bw), b0 - kPruneBins);
      int h = min(floordiv_pos(q[a] + ri, Bw), b0 + kPruneBins);
      if (I.per[a]) {
        if (h - l + 1 >= I.nb[a]) { l = 0; h = I.nb[a] - 1; }
      } else {
        l = max(l, 0);
        h = min(h, I.nb[a] - 1);
      }
      lo[a] = l;
      ext[a] = h - l + 1;
      hp[a] = b0 - l;  // the site's own bin, as a position in the box
    }
    // the 27 bins around the site's own first (a dominating site is usually
    // there, and the warp stops after one round), then the rest of the box
    const int nbt = reach > 0.0 ? ext[0] * ext[1] * ext[2] : 0;
    const int ntot = nbt > 0 ? 27 + nbt : 0;
    for (int i0 = 0; i0 < ntot; i0 += 32) {
      const int s = i0 + lane;
      bool hit = false;
      int pos[3];
      bool visit;
      if (s < 27) {
        pos[0] = hp[0] + s % 3 - 1;
        pos[1] = hp[1] + (s / 3) % 3 - 1;
        pos[2] = hp[2] + s / 9 - 1;
        visit = true;
        for (int a = 0; a < 3; a++) visit = visit && pos[a] >= 0 && pos[a] < ext[a];
      } else {
        const int i = s - 27;
        pos[0] = i % ext[0];
        pos[1] = (i / ext[0]) % ext[1];
        pos[2] = i / (ext[0] * ext[1]);
        bool inner = true;
        for (int a = 0; a < 3; a++) inner = inner && abs(pos[a] - hp[a]) <= 1;
        visit = s < ntot && !inner;
      }
      if (visit) {
        const int bx = wrap_axis(I, 0, lo[0] + pos[0]);
        const int by = wrap_axis(I, 1, lo[1] + pos[1]);
        const int bz = wrap_axis(I, 2, lo[2] + pos[2]);
        const int64_t b = I.bin_base + ((int64_t)bz * I.nb[1] + by) * I.nb[0] + bx;
        for (int k = wk.bin_start[b]; k < wk.bin_start[b + 1] && !hit; k++) {
          const int4 p = wk.spos[k];
          if (p.w == (int)c.s) continue;
          const float2 fa = wk.sfa[k];
          const int pj[3] = {p.x, p.y, p.z};
          long long D = 0;
          for (int a = 0; a < I.nd; a++) {
            int d = q[a] - pj[a];
            if (I.per[a]) {
              const int L = I.L[a];
              if (d > L / 2) d -= L; else if (d < -(L / 2)) d += L;
            }
            D += (long long)d * d;
          }
          const float ajr = __fadd_rn(fa.x, __fmul_rn(__fsqrt_rn(__ll2float_rn(D)), fa.y));
          if (__fsub_rn(tsr, ajr) < -0x1p-16f * __fadd_rn(tsr, ajr)) continue;
          const longlong2 aj = wk.saux[k];
          const double tj = __longlong_as_double(aj.x), denj = __longlong_as_double(aj.y);
          if (!(denj >= dens)) continue;
          const double aup = __dadd_ru(tj, __ddiv_ru(__dsqrt_ru((double)D), denj));
          const double margin = 0x1p-40 * (1.0 + fabs(ts) + fabs(tj) + span);
          hit = __dsub_rd(ts, aup) > margin;
        }
      }
      if (__any_sync(0xffffffffu, hit)) {
        out = true;
        break;
      }
    }
  }
  if (lane == 0) {
    wk.pruned[g] = out;
    if (out) atomicAdd(&wk.cnt[C_PRUNED], 1ull);
  }
}

// ------------------------------------------------------------------ launch

cudaError_t launch_jm_prune(const Work& wk, const Inst& one, cudaStream_t st) {
  const int T = 128;  // four sites per block, one per warp
  k_jm_prune<<<(unsigned)((wk.total_sites * 32 + T - 1) / T), T, 0, st>>>(wk, one);
  return cudaGetLastError();
}

cudaError_t launch_binning(const Work& wk, const Inst& one, int32_t* tid_of, cudaStream_t st,
                           bool skip_pruned) {
  const int T = 256;
  const unsigned gs = (unsigned)((wk.total_sites + T - 1) / T);
  const unsigned gbins = (unsigned)((wk.total_bins + T - 1) / T);
  k_count<<<gs, T, 0, st>>>(wk, one, skip_pruned ? 1 : 0);
  k_scan_local<<<wk.n_scan_blocks, 256, 0, st>>>(wk);
  k_scan_top<<<1, 1024, 0, st>>>(wk);
  k_scan_add<<<gbins, T, 0, st>>>(wk);
  k_scatter<<<gs, T, 0, st>>>(wk, tid_of);
  k_rank<<<gs, T, 0, st>>>(wk, one, tid_of);
  return cudaGetLastError();
}

}  // namespace vt
