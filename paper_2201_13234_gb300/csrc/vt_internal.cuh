// vt_internal.cuh -- data structures and small device helpers shared by the
// binning kernels (vt_bin.cu), the labelling kernels (vt_label.cu) and the
// host planner (vt_api.cu).
//
// Fixed point: 512 units per voxel; voxel k of an axis has its centre at
// 512 k + 256; a site coordinate lies in [0, L) with L = 512 n.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vt {

constexpr int kQ = 512;
constexpr int kMaxN = 16384;  // voxels per axis: every FP32 coordinate delta (images included) stays below 2^24, hence exact

enum Kind : int32_t { KV = 0, KL = 1, KJ = 2 };
enum Prec : int32_t { P_F32 = 0, P_EXACT = 1 };

// Device counters (unsigned long long each), see vt_stats.
enum Counter : int {
  C_CAND = 0,       // voxel x candidate evaluations (first pass)
  C_RESCORED = 1,   // voxels rescored exactly
  C_P2 = 2,         // bricks appended to the second-pass list
  C_DEFER = 3,      // of which: staging overflow
  C_P2_CURSOR = 4,  // second-pass work cursor
  C_RESTAGE = 5,    // first-pass bricks whose region was staged more than once
  C_P1_CURSOR = 6,  // batch first-pass work cursor
  C_UNIFORM = 7,    // first-pass tiles settled by the uniform test (one site wins everywhere)
  C_PRUNED = 8,     // Johnson-Mehl sites discarded before labelling (reached before their birth)
  C_RECULL = 9,     // listed bricks settled by the first pass's culling re-run
  C_LONG = 10,      // re-run tiles whose lists were scored in chunks
  C_N = 11
};

// Second-pass list flags (per brick): why it was listed, and, after the
// culling re-run, kDeferStage plus the number of its tiles that run settled
// (four tiles per brick): kDeferDone means the second pass has nothing to do.
constexpr int kDeferList = 1;   // candidate list or bin rows too long, no staging retry
constexpr int kDeferStage = 2;  // staged images did not fit: retried with a running cull
constexpr int kDeferDone = kDeferStage + 4;

// Error word layout (int32[4]): code, instance, site (low), site (high).
enum ErrSlot : int { E_CODE = 0, E_INST = 1, E_SITE_LO = 2, E_SITE_HI = 3 };

// One labelling problem.  Plain old data: copied by value into kernel
// parameters (single grid) or into the workspace (batch), then into shared
// memory per tile.
struct Inst {
  int32_t nd, kind;
  int32_t n[3];       // voxels per axis (n[2] = 1 in 2D)
  int32_t L[3];       // 512 n
  int32_t per[3];     // periodic flags
  int32_t bw[3];      // bin width (voxels)
  int32_t nb[3];      // bins per axis
  int32_t bricks[3];  // second-pass bricks per axis (2 x 2 x 1 tiles)
  int32_t tiles[3];   // first-pass tiles (warp boxes) per axis
  int32_t cfg;        // brick configuration id
  int32_t margin;     // first-pass staging margin (voxels), before the Laguerre widening
  int32_t precision;  // Prec
  int32_t vec_ok;     // labels row-aligned for 16-byte stores
  int32_t late;       // first pass: certify each tile after scoring (one staging round), else
                      // grow each brick's region until it is certified before scoring
  int64_t n_sites;
  int64_t site_base;  // offset of this instance in the concatenated per-site arrays
  int64_t bin_base;   // offset in the concatenated per-bin arrays
  int64_t brick_base; // first global brick id
  int64_t n_bricks;
  int64_t tile_base;  // first global tile id
  int64_t n_tiles;
  const int32_t* sites;  // [n_sites][nd] caller input
  const int64_t* w;
  const double* t;
  const double* v;
  int32_t* labels;
};

// A staged candidate of the first pass: one periodic image of a site, at
// exact float coordinates relative to the first voxel centre of its brick,
// with the site's FP32 data, its ids and the lower bound of its score (f-units)
// over the brick.
struct Staged {
  float qx, qy, qz, a;
  float b;
  int id, src;
  float lob;
};

// What the staging kernel leaves for the scoring kernel about one brick: its
// culled images (a run of the chunk's pool), per tile the smallest upper bound
// of an image and that image's position in the run, and the margin and bound
// of the region that certified it.  off < 0: the brick was left to the second
// pass (or had no site), nothing to score.
struct BrickRec {
  unsigned long long tkey[4];  // per tile: (upper bound bits << 32) | position in the run
  int off;                     // first image in the pool, or -1
  int ncull;                   // images in the run
  int org[3];                  // first voxel of the brick
  int M;                       // staging margin (fixed point, clamped to int32)
  float UB;                    // upper bound of every voxel's best score (f-units)
  int inst;                    // instance (batches)
  int dlo[3], dhi[3];          // per axis: every site that was not staged lies at least this
                               // far (fixed point) below the brick's first voxel centre /
                               // above its last; 0x7FFFFFFF: no such site on that side
  int pad[2];
};
static_assert(sizeof(BrickRec) == 96, "brick record");

// Per-instance statistics gathered while binning (ordered-integer encodings
// so that they can be reduced with integer atomics).
struct IStat {
  long long wmax;            // Laguerre: max w
  unsigned long long tmin;   // JM: dkey(min t)
  unsigned long long tabs;   // JM: dkey(max |t|)
  unsigned long long vmax;   // JM: dkey(max v)
};

// Device workspace, sliced by the host planner out of the caller's buffer.
struct Work {
  int32_t* err;                  // [4]
  uint8_t* pruned;               // [total_sites] Johnson-Mehl: 1 if the site was discarded
  unsigned long long* cnt;       // [C_N]
  IStat* istat;                  // [n_inst]
  int32_t* bin_count;            // [total_bins]   counts, then scatter cursors
  int32_t* bin_start;            // [total_bins+1] exclusive scan (global site offsets)
  int32_t* scan_blk;             // [n_scan_blocks]
  int32_t* site_bin;             // [total_sites]  global bin of each site (-1 = invalid)
  int4* spos;                    // [total_sites]  sorted: x, y, z (256 in 2D), id
  longlong2* saux;               // [total_sites]  sorted exact data: L (w, 0); JM (t, 512 v) bits
  float2* sfa;                   // [total_sites]  sorted FP32 data: L (W-w, 0); JM (t-tmin, 1/(512v))
  unsigned long long* bstat;     // [total_bins][2] L: wmax; JM: dkey(tmin), dkey(vmax)
  int32_t* p2_list;              // [3 * total_bricks]: brick, margin (fixed point), UB (float bits)
  int32_t* p2_flag;              // [total_bricks] brick already listed for pass 2
  BrickRec* brec;                // [total_bricks] first pass: staging -> scoring
  Staged* pool;                  // [pool_cap] culled images of the bricks of one chunk
  int32_t* pcur;                 // [n_chunks] pool cursor of each chunk (zeroed)
  int64_t pool_cap;
  const Inst* insts;             // batch table (nullptr: single instance in the kernel parameter)
  int32_t n_inst;
  int32_t n_scan_blocks;
  int64_t total_sites;
  int64_t total_bins;
  int64_t total_bricks;
  int64_t total_tiles;
};

// ---------------------------------------------------------------- helpers

// floor(a / b) for b > 0 and |a| < 2^28, without an integer division: a
// single-precision quotient (within 1/4 of a / b over that range: the float
// of a errs by at most 16, relevant only when b >= 512, and the quotient by a
// few ulp) is floored, then corrected once either way.
__device__ __forceinline__ int floordiv_pos(int a, int b) {
  int q = __float2int_rd(__fdividef((float)a, (float)b));
  int r = a - q * b;
  if (r < 0) {
    --q;
    r += b;
  }
  if (r >= b) ++q;
  return q;
}

// Order-preserving map of a double onto an unsigned 64-bit key.
__device__ __forceinline__ unsigned long long dkey(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

// Index of the instance whose [base, base+count) range holds g (batch only).
template <typename F>
__device__ __forceinline__ int find_inst(const Inst* insts, int n, int64_t g, F base_of) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base_of(insts[mid]) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void set_error(int32_t* err, int code, int inst, int64_t site) {
  if (atomicCAS(&err[E_CODE], 0, code) == 0) {
    err[E_INST] = inst;
    err[E_SITE_LO] = (int32_t)(site & 0xFFFFFFFF);
    err[E_SITE_HI] = (int32_t)(site >> 32);
  }
}

}  // namespace vt
