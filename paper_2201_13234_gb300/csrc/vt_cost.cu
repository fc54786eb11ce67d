// vt_cost.cu -- the paper's cost model of its two-step algorithm, evaluated on
// the GPU over the sites (Section 3.2.3 for Voronoi diagrams, Section 3.3.2 for
// Johnson-Mehl and, with the ball of Eq. rs Laguerre, Laguerre diagrams).
//
// Step 1 of the two-step algorithm scores every voxel of each site's
// investigation ball, step 2 scores every voxel no ball reached against every
// site.  With v'_s = min(V, v_s) (Eq. v', v_s the volume of site s's ball) the
// expected number of scores per voxel is (Eq. nstep12_jmak divided by N_v)
//     C(x) = sum_s v'_s / V + N_s prod_s (1 - v'_s / V),
// where the ball of site s at threshold x has radius v_s (x - t_s)^+ for
// Johnson-Mehl (Eq. rs JM; x = t0) and sqrt((x + w_s)^+) for Laguerre
// (Eq. rs Laguerre with G = 1 and G t_s = -w_s; x in voxel^2).  For Voronoi
// diagrams every ball has the same radius and C is the closed form of
// Eq. nstep12_3d, minimised by the ball fraction of Eq. v0_3d.
//
// The threshold that minimises C is searched between the bounds the paper
// gives (end of Sections 3.3.2 and 3.4): a scan of 129 points, then a
// golden-section refinement of the best bracket.  The sums over the sites run
// on the GPU in a fixed order (per block, then block by block on the host),
// so repeated calls give the same result.
#include <cmath>
#include <cstring>
#include <vector>

#include "vt.h"
#include "vt_internal.cuh"

namespace vt {

constexpr int kCostThreads = 256;
constexpr int kCostBlocks = 240;  // site slices (one per block and threshold)
constexpr int kCostMaxK = 129;    // thresholds per launch

struct CostIn {
  int nd, kind;
  double V, coeff;  // domain volume (voxels^d), volume of a ball of radius 1
  long long ns;
  const int64_t* w;
  const double* t;
  const double* v;
};

// Ball volume fraction v_s / V of site s at threshold x (uncapped).
__device__ __forceinline__ double ball_fraction(const CostIn& c, long long s, double x) {
  double r;
  if (c.kind == KJ) {
    r = c.v[s] * (x - c.t[s]);
    if (r <= 0.0) return 0.0;
  } else {
    const double r2 = x + (double)c.w[s] / (512.0 * 512.0);
    if (r2 <= 0.0) return 0.0;
    r = sqrt(r2);
  }
  const double vol = c.nd == 2 ? c.coeff * r * r : c.coeff * r * r * r;
  return vol / c.V;
}

// Block (bx, k): the sites s = bx, bx + kCostBlocks, ... (strided over the
// threads of the block) at threshold x[k]: sum of min(1, f_s), sum of
// log(1 - f_s) over the sites with f_s < 1, and whether any f_s >= 1.
__global__ void __launch_bounds__(kCostThreads) k_cost(const CostIn c, const double* x,
                                                       double* part) {
  __shared__ double s1[kCostThreads], s2[kCostThreads];
  __shared__ int sz[kCostThreads];
  const int k = blockIdx.y;
  const double xk = x[k];
  double a = 0.0, b = 0.0;
  int z = 0;
  for (long long s = (long long)blockIdx.x * kCostThreads + threadIdx.x; s < c.ns;
       s += (long long)gridDim.x * kCostThreads) {
    double f = ball_fraction(c, s, xk);
    if (f >= 1.0) {
      f = 1.0;
      z = 1;
    } else {
      b += log1p(-f);
    }
    a += f;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  sz[threadIdx.x] = z;
  __syncthreads();
  for (int o = kCostThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
      sz[threadIdx.x] |= sz[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* p = part + 3 * ((size_t)k * gridDim.x + blockIdx.x);
    p[0] = s1[0];
    p[1] = s2[0];
    p[2] = (double)sz[0];
  }
}

// Per block: min t, min v and max v (Johnson-Mehl), max w (Laguerre), for
// the bounds of the threshold search and the reach of the largest ball.
__global__ void __launch_bounds__(kCostThreads) k_cost_range(const CostIn c, double* part) {
  __shared__ double s0[kCostThreads], s1[kCostThreads], s2[kCostThreads];
  double a = INFINITY, b = c.kind == KJ ? INFINITY : -INFINITY, d = -INFINITY;
  for (long long s = (long long)blockIdx.x * kCostThreads + threadIdx.x; s < c.ns;
       s += (long long)gridDim.x * kCostThreads) {
    if (c.kind == KJ) {
      a = fmin(a, c.t[s]);
      b = fmin(b, c.v[s]);
      d = fmax(d, c.v[s]);
    } else {
      b = fmax(b, (double)c.w[s]);
    }
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  s2[threadIdx.x] = d;
  __syncthreads();
  for (int o = kCostThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] = fmin(s0[threadIdx.x], s0[threadIdx.x + o]);
      s1[threadIdx.x] = c.kind == KJ ? fmin(s1[threadIdx.x], s1[threadIdx.x + o])
                                     : fmax(s1[threadIdx.x], s1[threadIdx.x + o]);
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = s0[0];
    part[3 * blockIdx.x + 1] = s1[0];
    part[3 * blockIdx.x + 2] = s2[0];
  }
}

// Host side: the evaluator keeps its device buffers in the caller's
// workspace (thresholds, then the per-block partial sums).
struct CostEval {
  CostIn in;
  double* d_x;
  double* d_part;
  cudaStream_t st;
  std::vector<double> h_part;

  // C(x_k) for n <= kCostMaxK thresholds.
  cudaError_t eval(const double* xs, int n, double* out) {
    cudaError_t e = cudaMemcpyAsync(d_x, xs, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_cost<<<dim3(kCostBlocks, n), kCostThreads, 0, st>>>(in, d_x, d_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    h_part.resize((size_t)3 * kCostBlocks * n);
    e = cudaMemcpyAsync(h_part.data(), d_part, sizeof(double) * h_part.size(),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    for (int k = 0; k < n; k++) {
      double a = 0.0, b = 0.0;
      bool z = false;
      for (int bx = 0; bx < kCostBlocks; bx++) {  // block order: deterministic
        const double* p = &h_part[3 * ((size_t)k * kCostBlocks + bx)];
        a += p[0];
        b += p[1];
        z = z || p[2] != 0.0;
      }
      out[k] = a + (z ? 0.0 : (double)in.ns * std::exp(b));
    }
    return cudaSuccess;
  }
};

size_t cost_workspace_bytes() {
  return sizeof(double) * ((size_t)kCostMaxK + (size_t)3 * kCostBlocks * kCostMaxK);
}

static double ball_coeff(int nd) { return nd == 2 ? M_PI : 4.0 * M_PI / 3.0; }

static CostEval make_eval(int nd, const int64_t* n, int kind, int64_t ns, const int64_t* w,
                          const double* t, const double* v, void* ws, cudaStream_t st) {
  CostEval E;
  E.in.nd = nd;
  E.in.kind = kind;
  E.in.V = 1.0;
  for (int a = 0; a < nd; a++) E.in.V *= (double)n[a];
  E.in.coeff = ball_coeff(nd);
  E.in.ns = ns;
  E.in.w = w;
  E.in.t = t;
  E.in.v = v;
  E.d_x = static_cast<double*>(ws);
  E.d_part = E.d_x + kCostMaxK;
  E.st = st;
  return E;
}

cudaError_t cost_model_eval(int nd, const int64_t* n, int kind, int64_t ns, const int64_t* w,
                            const double* t, const double* v, const double* xs, int count,
                            double* out, void* ws, cudaStream_t st) {
  CostEval E = make_eval(nd, n, kind, ns, w, t, v, ws, st);
  for (int i = 0; i < count; i += kCostMaxK) {
    const int m = count - i < kCostMaxK ? count - i : kCostMaxK;
    cudaError_t e = E.eval(xs + i, m, out + i);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The threshold minimising C, C there, and the radius (voxels) of the largest
// investigation ball at that threshold.  Voronoi: x = r0^2 (voxel^2) from
// Eq. v0_3d and C from Eq. nstep12_3d; Laguerre: x in voxel^2; Johnson-Mehl:
// x = t0.
cudaError_t cost_model_threshold(int nd, const int64_t* n, uint32_t per_mask, int kind,
                                 int64_t ns, const int64_t* w, const double* t, const double* v,
                                 double* x_out, double* c_out, double* reach, void* ws,
                                 cudaStream_t st) {
  double V = 1.0, sum_l2 = 0.0;
  for (int a = 0; a < nd; a++) {
    V *= (double)n[a];
    sum_l2 += (double)n[a] * (double)n[a];
  }
  if (kind == KV) {
    const double f = ns < 2 ? 1.0 : -std::expm1(-std::log((double)ns) / (double)(ns - 1));
    const double r0 = std::pow(f * V / ball_coeff(nd), 1.0 / nd);
    *x_out = r0 * r0;
    *c_out = (double)ns * (f + std::pow(1.0 - f, (double)ns));
    *reach = r0;
    return cudaSuccess;
  }
  // search interval
  std::vector<double> hp(3 * kCostBlocks);
  CostEval E = make_eval(nd, n, kind, ns, w, t, v, ws, st);
  k_cost_range<<<kCostBlocks, kCostThreads, 0, st>>>(E.in, E.d_part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(hp.data(), E.d_part, sizeof(double) * hp.size(),
                           cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return e;
  double r0 = INFINITY, r1 = kind == KJ ? INFINITY : -INFINITY, r2 = -INFINITY;
  for (int b = 0; b < kCostBlocks; b++) {
    r0 = std::fmin(r0, hp[3 * b]);
    r1 = kind == KJ ? std::fmin(r1, hp[3 * b + 1]) : std::fmax(r1, hp[3 * b + 1]);
    r2 = std::fmax(r2, hp[3 * b + 2]);
  }
  const bool periodic = (per_mask & ((1u << nd) - 1)) != 0;
  double lo, hi;
  if (kind == KJ) {
    lo = r0;
    hi = r0 + (periodic ? 0.5 : 1.0) * std::sqrt(sum_l2) / r1;
  } else {
    lo = -r1 / (512.0 * 512.0);
    hi = lo + (periodic ? 0.25 : 1.0) * sum_l2;
  }
  // scan
  const int G = kCostMaxK - 1;
  std::vector<double> xs(G + 1), cs(G + 1);
  for (int i = 0; i <= G; i++) xs[i] = lo + (hi - lo) * i / G;
  if ((e = E.eval(xs.data(), G + 1, cs.data())) != cudaSuccess) return e;
  int best = 0;
  for (int i = 1; i <= G; i++)
    if (cs[i] < cs[best]) best = i;
  // golden section on the bracket around the best scan point
  double a = lo + (hi - lo) * (best > 0 ? best - 1 : 0) / G;
  double b = lo + (hi - lo) * (best < G ? best + 1 : G) / G;
  const double gr = 0.6180339887498949;
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a), f1, f2;
  if ((e = E.eval(&x1, 1, &f1)) != cudaSuccess || (e = E.eval(&x2, 1, &f2)) != cudaSuccess)
    return e;
  for (int it = 0; it < 40; it++) {
    if (f1 < f2) {
      b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a);
      if ((e = E.eval(&x1, 1, &f1)) != cudaSuccess) return e;
    } else {
      a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a);
      if ((e = E.eval(&x2, 1, &f2)) != cudaSuccess) return e;
    }
  }
  double xm = 0.5 * (a + b), fm;
  if ((e = E.eval(&xm, 1, &fm)) != cudaSuccess) return e;
  if (fm <= cs[best]) {
    *x_out = xm;
    *c_out = fm;
  } else {
    *x_out = xs[best];
    *c_out = cs[best];
  }
  *reach = kind == KJ ? r2 * std::fmax(0.0, *x_out - r0)
                      : std::sqrt(std::fmax(0.0, *x_out + r1 / (512.0 * 512.0)));
  return cudaSuccess;
}

}  // namespace vt
