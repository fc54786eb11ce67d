/*
 * vt.h -- GB300 (sm_103a) library for digital images of Voronoi, Laguerre and
 * Johnson-Mehl tessellations (Moulinec, "A simple and fast algorithm for
 * computing discrete Voronoi, Johnson-Mehl or Laguerre diagrams of points",
 * arxiv 2201.13234).
 *
 * Problem (Section 3, opening list): label every voxel of a regular 2D or 3D
 * grid on the box [0,L_1) x ... x [0,L_d), periodic or not per axis, with the
 * site that minimises a score:
 *   Voronoi       |x - x_s|^2                       (Eq. Voronoi_Cell, squared)
 *   Laguerre      |x - x_s|^2 - w_s                 (power distance, Section 2.3,
 *                                                   w_s = r_s^2)
 *   Johnson-Mehl  t_s + |x - x_s| / v_s             (Eq. JMAK2; v_s is the growth
 *                                                   speed G, per site here)
 * with the L-periodic distance of Appendix A (Eq. dL) on periodic axes.
 *
 * Conventions shared by every entry point:
 *   - Fixed point: 512 units per voxel.  Axis i has n_i voxels and length
 *     L_i = 512 n_i units; voxel k has its centre at 512 k + 256.
 *   - Sites: int32 coordinates in [0, L_i), array [n_sites][ndim], x first.
 *   - Laguerre weights: int64 w_s in [0, 2^52), in units of (1/512 voxel)^2, so
 *     the score D - w_s is exact in int64.
 *   - Johnson-Mehl: double t_s (finite, |t_s| < 2^40) and double v_s (finite,
 *     1e-12 <= v_s <= 1e12), speed in voxels per time unit.  The arrival time
 *     is evaluated in IEEE double as t_s + (sqrt((double)D) / (512 v_s)), each
 *     operation rounded to nearest, no fused multiply-add, in that order.
 *   - Labels: int32 0-based site ids, array [n_z][n_y][n_x] (x fastest).  Among
 *     equal scores the lowest id wins, as the strict "<" over increasing s of
 *     Algorithms 1-3 does.  Results are bit-identical to that definition.
 *   - Sizes: 1 <= n_i <= 16384, n_x n_y n_z < 2^40, 1 <= n_sites < 2^31 - 1.
 *
 * Memory: every device buffer (sites, weights, times, speeds, labels and the
 * workspace) is owned by the caller and must stay alive until the stream work
 * that uses it has finished.  The library owns only its small host-side
 * contexts and allocates no device memory.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls are asynchronous on it.  Errors that the host can see
 * (arguments, sizes, a short workspace) are returned at once; errors in the
 * data (a coordinate outside the box, a weight, time or speed out of range)
 * are found on the GPU and returned by vt_sync, and the labels are then
 * unspecified.
 */
#ifndef VT_H
#define VT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VT_OK = 0,
  VT_ERR_ARG = 1,       /* bad argument (null pointer, ndim, dims, n_sites ...) */
  VT_ERR_RANGE = 2,     /* a site, weight, time or speed outside its range (device) */
  VT_ERR_CUDA = 3,      /* a CUDA runtime call failed; see vt_last_error */
  VT_ERR_NOMEM = 4,     /* host allocation failed */
  VT_ERR_TIMEOUT = 5,   /* reserved: a bounded device wait gave up */
  VT_ERR_WORKSPACE = 6  /* the workspace is smaller than vt_*_workspace_size says */
} vt_status;

typedef enum { VT_VORONOI = 0, VT_LAGUERRE = 1, VT_JOHNSON_MEHL = 2 } vt_kind;

typedef enum {
  VT_FP32_RESCORE = 0,  /* FP32 screening, exact rescoring of near ties (default) */
  VT_EXACT = 1          /* every score in exact int64 / IEEE double arithmetic */
} vt_precision;

/* Tuning knobs.  Zero fields take the library's defaults. */
typedef struct {
  int32_t precision;    /* vt_precision */
  int32_t brick_cfg;    /* tiles scored by one warp: 0 = 8x8x8 voxels (2D 16x32), 1 = compact
                           8x8x4 (2D 16x16; fewer candidates per voxel, more tiles); vt_autotune
                           times both and keeps the faster; VT_ERR_ARG for other values */
  double bin_scale;     /* mean sites per bin (default 1.0) */
  double margin_scale;  /* first-pass staging margin beyond the brick, in mean cell radii */
  int32_t timing;       /* 1: record CUDA events around each stage (reported by vt_sync) */
  int32_t certify;      /* first pass: 1 = stage each brick's sites once and certify each tile
                           after scoring (tiles that fail are staged again), 2 = grow each
                           brick's region until it is certified before scoring, 3 = send every
                           brick straight to the re-run that culls as it stages and grows each
                           region until certified (clustered sites), 0 = the library's default
                           (1; Johnson-Mehl 2) and vt_autotune times all three.  Labels are the
                           same either way.  Batches take 0, 1 or 2. */
} vt_options;

/* Counters of the last call, filled by vt_sync. */
typedef struct {
  int64_t voxels;          /* voxels labelled */
  int64_t candidates;      /* voxel x candidate score evaluations in the first pass */
  int64_t rescored;        /* voxels whose FP32 margin was within the error bound */
  int64_t pass2_bricks;    /* bricks the second pass labelled (the first pass could not
                              certify them) */
  int64_t deferred_bricks; /* bricks listed for the first pass's culling re-run: their staged
                              candidates overflowed shared memory or a tile was not certified
                              (every brick under vt_options.certify = 3) */
  int32_t dev_error;       /* vt_status found on the device (VT_OK if none) */
  int32_t error_instance;  /* batch instance of dev_error (-1 if none) */
  int64_t error_site;      /* offending site index (-1 if none) */
  float stage_ms[3];       /* with vt_options.timing: binning, first pass, second pass (ms) */
  float scores_ms;         /* with vt_options.timing: the score image of vt_label_scores (ms) */
  int64_t uniform_tiles;   /* first-pass tiles won by one site everywhere (no per-voxel scoring) */
  int64_t restaged_bricks; /* first-pass bricks whose first staging margin was too small */
  int64_t pruned_sites;    /* Johnson-Mehl sites discarded beforehand: another site reaches
                              them before their birth, so they have no cell (Section 3.3) */
  int64_t recull_bricks;   /* of those, the bricks the culling re-run (which culls as it stages
                              and grows each region until certified) settled; the rest go to
                              the second pass */
  int64_t long_tiles;      /* tiles of that re-run whose candidate lists exceeded 256 entries
                              (dense clusters), scored in chunks */
} vt_stats;

/* ------------------------------------------------------------------------
 * Single grids.
 * ---------------------------------------------------------------------- */
typedef struct vt_ctx vt_ctx;

/* Create a context for one grid.  dims[0..ndim-1] = (n_x, n_y[, n_z]);
 * bit i of periodic_mask makes axis i periodic (Appendix A).  opt may be NULL.
 * Returns VT_ERR_ARG for ndim not in {2,3} or a dimension out of range. */
vt_status vt_create(vt_ctx** out, int32_t ndim, const int64_t* dims, uint32_t periodic_mask,
                    const vt_options* opt);

/* Bytes of device workspace that a call with n_sites sites of the given kind
 * needs (256-byte alignment is enough). */
vt_status vt_workspace_size(const vt_ctx* ctx, int64_t n_sites, int32_t kind, size_t* bytes);

/* Voronoi labels (Eq. Voronoi_Cell; Algorithm 2 computes the same image).
 * d_sites: device int32 [n_sites][ndim]; d_labels: device int32 [N_v];
 * d_workspace: device buffer of at least vt_workspace_size bytes. */
vt_status vt_voronoi(vt_ctx* ctx, int64_t n_sites, const int32_t* d_sites, int32_t* d_labels,
                     void* d_workspace, size_t workspace_bytes, void* stream);

/* Laguerre labels (power distance, Section 2.3 and Appendix B).
 * d_w: device int64 [n_sites], w_s = r_s^2 in (1/512 voxel)^2. */
vt_status vt_laguerre(vt_ctx* ctx, int64_t n_sites, const int32_t* d_sites, const int64_t* d_w,
                      int32_t* d_labels, void* d_workspace, size_t workspace_bytes, void* stream);

/* Johnson-Mehl labels (Eqs. JMAK2 and JM1).  d_t, d_v: device double [n_sites]. */
vt_status vt_johnson_mehl(vt_ctx* ctx, int64_t n_sites, const int32_t* d_sites, const double* d_t,
                          const double* d_v, int32_t* d_labels, void* d_workspace,
                          size_t workspace_bytes, void* stream);

/* Labels and the score image D (Algorithm 1 computes D beside I; Algorithms 2
 * and 3 initialise and update it, Sections 3.1-3.3): each voxel's best score,
 * i.e. the exact score of its label's site at the voxel, nearest periodic
 * image on periodic axes.  Same operation and arguments as vt_voronoi /
 * vt_laguerre / vt_johnson_mehl for kind VT_VORONOI / VT_LAGUERRE /
 * VT_JOHNSON_MEHL (d_w, d_t, d_v as there, NULL where the kind has none), plus
 *   d_scores  device buffer of N_v 8-byte values, x fastest, 8-byte aligned:
 *             Voronoi int64 D (squared distance, units of (1/512 voxel)^2),
 *             Laguerre int64 D - w_s, Johnson-Mehl double arrival time
 *             t_s + sqrt(D) / (512 v_s) (IEEE, in that order, no fused op).
 * The scores are written after the labels, by a kernel that reads them back
 * (12 more bytes per voxel of memory traffic); after a device error (vt_sync
 * returns VT_ERR_RANGE) both images are unspecified.  VT_ERR_ARG for a null or
 * misaligned d_scores. */
vt_status vt_label_scores(vt_ctx* ctx, int32_t kind, int64_t n_sites, const int32_t* d_sites,
                          const int64_t* d_w, const double* d_t, const double* d_v,
                          int32_t* d_labels, void* d_scores, void* d_workspace,
                          size_t workspace_bytes, void* stream);

/* Labels from host buffers, with the labels stored straight into host memory
 * (the end-to-end path: on a GPU coherently attached to its CPU the kernels'
 * label stores travel over that link, overlapped with the labelling, instead
 * of a copy after it).  Same operation and arguments as vt_voronoi /
 * vt_laguerre / vt_johnson_mehl for kind VT_VORONOI / VT_LAGUERRE /
 * VT_JOHNSON_MEHL, except:
 *   h_sites, h_w, h_t, h_v  host memory (any; page-locked copies faster), read
 *                           by copies enqueued on `stream`: keep them intact
 *                           until the call's work has finished;
 *   h_labels                page-locked host memory mapped into the device
 *                           address space (cudaHostAlloc, or cudaHostRegister
 *                           with the mapped flag; on systems with unified
 *                           addressing every page-locked allocation is);
 *                           VT_ERR_ARG, with nothing launched, otherwise;
 *   d_workspace             at least vt_workspace_size_host bytes (the inputs
 *                           are staged in its tail).
 * Asynchronous on `stream`: read h_labels after vt_sync. */
vt_status vt_workspace_size_host(const vt_ctx* ctx, int64_t n_sites, int32_t kind,
                                 size_t* bytes);
vt_status vt_label_host(vt_ctx* ctx, int32_t kind, int64_t n_sites, const int32_t* h_sites,
                        const int64_t* h_w, const double* h_t, const double* h_v,
                        int32_t* h_labels, void* d_workspace, size_t workspace_bytes,
                        void* stream);

/* Voronoi labels without any device allocation, for callers that cannot
 * allocate GPU memory: a plugin whose host application owns every device
 * allocation and passes in only input and output buffers, or a latency-bound
 * loop that cannot afford the device-wide synchronisation of cudaMalloc and
 * cudaFree.  The paper has no counterpart: this is vt_voronoi run on a 64 MiB
 * scratch buffer that the library holds as a static device array (every GPU
 * that loads it keeps the 64 MiB until the process exits).  Returns
 * VT_ERR_WORKSPACE, with a message, when the grid and n_sites need more
 * scratch than that (the plan this context would run for them: grids up to
 * about 390^3 voxels fit, the first pass reserving about one byte per voxel).  The first call on each device looks up
 * the buffer's device address with that device current and caches it: make
 * that first call before any stream capture, and make no call after a
 * cudaDeviceReset in the same process.  All calls share the one buffer, which
 * keeps the last call's contents (the call clears what must start at zero):
 * calls that overlap on the GPU, from any thread, stream or context, race and
 * must be serialised by the caller.  The counters and the device error word
 * live in that buffer too: call vt_sync for this call before any other
 * vt_voronoi_static call is enqueued, or the counters and error it reports
 * belong to the later call. */
vt_status vt_voronoi_static(vt_ctx* ctx, int64_t n_sites, const int32_t* d_sites,
                            int32_t* d_labels, void* stream);

/* The paper's cost model of its two-step algorithm (Section 3.2.3, Eqs.
 * nstep12_3d and v0_3d; Section 3.3.2, Eqs. v' and nstep12_jmak; the ball of
 * Eq. rs Laguerre for Laguerre diagrams): the expected number of score
 * evaluations per voxel,
 *   C(x) = sum_s min(1, v_s / V) + N_s prod_s (1 - min(1, v_s / V)),
 * with V the grid's volume in voxels and v_s the volume of site s's
 * investigation ball at threshold x:
 *   Voronoi       x = r0^2 (voxel^2), every ball of radius r0 (closed form)
 *   Laguerre      x in voxel^2, radius sqrt((x + w_s / 512^2)^+)
 *   Johnson-Mehl  x = t0, radius v_s (x - t_s)^+.
 * The sums over the sites run on the GPU (device arrays d_w, d_t, d_v as for
 * labelling; NULL where the kind has none) in a fixed order, so a call is
 * repeatable.  thresholds[n_thresholds] and evals_per_voxel[n_thresholds] are
 * host arrays.  Synchronous; d_workspace as for labelling (vt_workspace_size
 * bytes are enough).  Call it outside any stream capture. */
vt_status vt_cost_model(vt_ctx* ctx, int32_t kind, int64_t n_sites, const int64_t* d_w,
                        const double* d_t, const double* d_v, const double* thresholds,
                        int32_t n_thresholds, double* evals_per_voxel, void* d_workspace,
                        size_t workspace_bytes, void* stream);

/* The threshold x that minimises the cost model above, searched between the
 * bounds of Sections 3.3.2 and 3.4 (Voronoi: Eq. v0_3d in closed form), and
 * C(x) there (*threshold, *evals_per_voxel: host).  Synchronous. */
vt_status vt_cost_threshold(vt_ctx* ctx, int32_t kind, int64_t n_sites, const int64_t* d_w,
                            const double* d_t, const double* d_v, double* threshold,
                            double* evals_per_voxel, void* d_workspace, size_t workspace_bytes,
                            void* stream);

/* Time a few staging margins and bin sizes on these very inputs and keep the
 * fastest for later calls of this context with the same kind and site count.
 * The staging margins tried include the radius of the largest investigation
 * ball at the cost model's optimal threshold (vt_cost_threshold).
 * Synchronous; call it outside any stream capture.  The labels buffer is
 * overwritten. */
vt_status vt_autotune(vt_ctx* ctx, int32_t kind, int64_t n_sites, const int32_t* d_sites,
                      const int64_t* d_w, const double* d_t, const double* d_v,
                      int32_t* d_labels, void* d_workspace, size_t workspace_bytes,
                      void* stream);

/* Wait for the context's last call on `stream`, read its device error word and
 * counters, and return the device error (VT_OK if none).  stats may be NULL. */
vt_status vt_sync(vt_ctx* ctx, void* stream, vt_stats* stats);

/* Message of the context's last error ("" if none).  ctx may be NULL for
 * errors of vt_create. */
const char* vt_last_error(const vt_ctx* ctx);

void vt_destroy(vt_ctx* ctx);

/* ------------------------------------------------------------------------
 * Batches: many independent grids of uneven size, site count and kind,
 * labelled by one persistent launch that a CUDA graph replays.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t ndim;
  int32_t kind;            /* vt_kind */
  int64_t dims[3];
  uint32_t periodic_mask;
  int64_t n_sites;
  const int32_t* d_sites;  /* device [n_sites][ndim] */
  const int64_t* d_w;      /* Laguerre only */
  const double* d_t;       /* Johnson-Mehl only */
  const double* d_v;       /* Johnson-Mehl only */
  int32_t* d_labels;       /* device [N_v], or page-locked host memory mapped into the
                              device address space: the kernels then store the labels
                              straight into host memory */
} vt_instance;

typedef struct vt_batch vt_batch;

/* Copy the instance table and plan every instance.  The device pointers are
 * fixed for the batch's lifetime (the captured graph refers to them). */
vt_status vt_batch_create(vt_batch** out, int32_t n, const vt_instance* instances,
                          const vt_options* opt);

vt_status vt_batch_workspace_size(const vt_batch* b, size_t* bytes);

/* Pick each instance's bin size and staging margin by timing it alone, then
 * drop any captured graph.  Synchronous; labels are overwritten. */
vt_status vt_batch_autotune(vt_batch* b, void* d_workspace, size_t workspace_bytes, void* stream);

/* Label every instance.  The first call with a given workspace captures the
 * whole pipeline (binning of all instances, one persistent first-pass kernel
 * over all their bricks, the second pass) into a CUDA graph; later calls
 * replay it.  use_graph = 0 launches the same kernels without a graph. */
vt_status vt_batch_run(vt_batch* b, void* d_workspace, size_t workspace_bytes, void* stream,
                       int32_t use_graph);

vt_status vt_batch_sync(vt_batch* b, void* stream, vt_stats* stats);
const char* vt_batch_last_error(const vt_batch* b);
void vt_batch_destroy(vt_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* VT_H */
