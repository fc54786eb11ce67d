// vt_scores.cu -- the score image D of the paper's algorithms.
//
// Algorithm 1 keeps, next to the label image I, the image D of each voxel's
// best score (the distance to the nearest site for Voronoi diagrams), and
// Algorithms 2 and 3 initialise and update the same D (Sections 3.1-3.3).
// Once a voxel's label is exact (the lowest-id minimiser of the score), its
// entry of D is that site's exact score at the voxel, with the nearest
// periodic image on every periodic axis (Appendix A, Eq. dL: each axis term
// of the squared distance is smallest at the wrapped difference, and every
// score is increasing in the squared distance).  This kernel writes it after
// the labelling, from the labels and the caller's site arrays:
//   Voronoi       int64   D = sum of squared differences  (1/512 voxel units)
//   Laguerre      int64   D - w
//   Johnson-Mehl  double  t + sqrt(D) / (512 v), IEEE round-to-nearest in that
//                         order with no fused operation (Eq. JMAK2)
// It streams the labels in (4 bytes per voxel) and the scores out (8 bytes per
// voxel); the sites it gathers stay in L2.
#include "vt_internal.cuh"

namespace vt {

constexpr int kScoreThreads = 256;
constexpr int kScoreRun = 128;  // voxels of a row per warp and work item (4 per lane)

template <int KIND>
__device__ __forceinline__ void score_of(const Inst& I, int id, int cx, int cy, int cz,
                                         long long& is, double& ds) {
  if ((unsigned)id >= (unsigned)I.n_sites) {  // not a label of this problem
    is = 0x7FFFFFFFFFFFFFFFll;
    ds = __longlong_as_double(0x7FF8000000000000ll);
    return;
  }
  const int c[3] = {cx, cy, cz};
  long long D = 0;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a >= I.nd) break;
    int d = c[a] - I.sites[(long long)id * I.nd + a];
    if (I.per[a]) {  // |d| < L: one shift reaches [-L/2, L/2)
      const int hL = I.L[a] >> 1;
      if (d >= hL) d -= I.L[a];
      else if (d < -hL) d += I.L[a];
    }
    D += (long long)d * d;
  }
  if (KIND == KV) {
    is = D;
  } else if (KIND == KL) {
    is = D - I.w[id];
  } else {
    ds = __dadd_rn(I.t[id], __ddiv_rn(__dsqrt_rn((double)D), __dmul_rn(512.0, I.v[id])));
  }
}

// One warp per run of kScoreRun voxels of a row (y, z); lane l takes voxels
// 4 l .. 4 l + 3 of the run.  vec: labels and scores of a row start on 16-byte
// boundaries (n_x a multiple of 4, aligned buffers).
template <int KIND>
__global__ void __launch_bounds__(kScoreThreads) k_scores(const __grid_constant__ Inst I,
                                                          const int32_t* err, void* scores,
                                                          int vec) {
  if (err[E_CODE]) return;  // the labels are unspecified after a data error
  const int lane = threadIdx.x & 31;
  const unsigned runs = (unsigned)((I.n[0] + kScoreRun - 1) / kScoreRun);
  const long long items = (long long)runs * I.n[1] * I.n[2];
  const long long wstride = (long long)gridDim.x * (kScoreThreads / 32);
  for (long long it = (long long)blockIdx.x * (kScoreThreads / 32) + (threadIdx.x >> 5);
       it < items; it += wstride) {
    const long long row = it / runs;  // (z n_y + y)
    const int x0 = (int)(it - row * runs) * kScoreRun + 4 * lane;
    if (x0 >= I.n[0]) continue;
    const int y = (int)(row % I.n[1]), z = (int)(row / I.n[1]);
    const long long base = row * I.n[0] + x0;
    int lab[4];
    const int nx = min(4, I.n[0] - x0);
    if (vec && nx == 4) {
      const int4 l4 = __ldcs(reinterpret_cast<const int4*>(I.labels + base));
      lab[0] = l4.x; lab[1] = l4.y; lab[2] = l4.z; lab[3] = l4.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; j++) lab[j] = j < nx ? I.labels[base + j] : 0;
    }
    const int cy = kQ * y + kQ / 2, cz = kQ * z + kQ / 2;
    long long is[4];
    double ds[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      is[j] = 0;
      ds[j] = 0.0;
      if (j < nx) score_of<KIND>(I, lab[j], kQ * (x0 + j) + kQ / 2, cy, cz, is[j], ds[j]);
    }
    long long* out = reinterpret_cast<long long*>(scores) + base;
    long long o[4];
#pragma unroll
    for (int j = 0; j < 4; j++) o[j] = KIND == KJ ? __double_as_longlong(ds[j]) : is[j];
    if (vec && nx == 4) {
      __stcs(reinterpret_cast<longlong2*>(out), make_longlong2(o[0], o[1]));
      __stcs(reinterpret_cast<longlong2*>(out) + 1, make_longlong2(o[2], o[3]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; j++)
        if (j < nx) out[j] = o[j];
    }
  }
}

cudaError_t launch_scores(const Inst& I, const int32_t* err, void* scores, int sms,
                          cudaStream_t st) {
  const int vec = (I.n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(I.labels) % 16 == 0) &&
                  (reinterpret_cast<uintptr_t>(scores) % 16 == 0);
  const unsigned grid = (unsigned)(sms * 8);
  if (I.kind == KV) k_scores<KV><<<grid, kScoreThreads, 0, st>>>(I, err, scores, vec);
  else if (I.kind == KL) k_scores<KL><<<grid, kScoreThreads, 0, st>>>(I, err, scores, vec);
  else k_scores<KJ><<<grid, kScoreThreads, 0, st>>>(I, err, scores, vec);
  return cudaGetLastError();
}

}  // namespace vt
