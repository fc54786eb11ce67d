// vt_api.cu -- the C ABI: contexts, the planner (bin size, staging margin,
// brick grid), the workspace layout, launches, the autotuner, and the batch
// path that captures the whole pipeline in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "vt.h"
#include "vt_device.cuh"

namespace vt {
cudaError_t launch_binning(const Work& wk, const Inst& one, int32_t* tid_of, cudaStream_t st,
                           bool skip_pruned = false);
cudaError_t launch_jm_prune(const Work& wk, const Inst& one, cudaStream_t st);
cudaError_t init_pass1();
cudaError_t init_pass2();
cudaError_t launch_pass1(const Work& wk, const Inst& I, int sms, cudaStream_t st);
cudaError_t launch_pass1_recull(const Work& wk, const Inst& I, int sms, cudaStream_t st);
cudaError_t launch_list_all(const Work& wk, const Inst& I, cudaStream_t st);
cudaError_t launch_pass2(const Work& wk, const Inst& I, int grid, cudaStream_t st);
cudaError_t launch_pass1_group(const Work& wk, int nd, int compact, int kind, int prec,
                               long long t0, long long t1, int sms, int* chunk, cudaStream_t st);
int64_t pass1_chunk_bricks();
size_t cost_workspace_bytes();
cudaError_t cost_model_eval(int nd, const int64_t* n, int kind, int64_t ns, const int64_t* w,
                            const double* t, const double* v, const double* xs, int count,
                            double* out, void* ws, cudaStream_t st);
cudaError_t cost_model_threshold(int nd, const int64_t* n, uint32_t per_mask, int kind,
                                 int64_t ns, const int64_t* w, const double* t, const double* v,
                                 double* x_out, double* c_out, double* reach, void* ws,
                                 cudaStream_t st);
cudaError_t launch_pass2_batch(const Work& wk, int grid, cudaStream_t st);
cudaError_t launch_scores(const Inst& I, const int32_t* err, void* scores, int sms,
                          cudaStream_t st);

// Opt every kernel into its resources (once per process, outside any capture).
static cudaError_t init_label_kernels() {
  cudaError_t e = init_pass1();
  return e == cudaSuccess ? init_pass2() : e;
}

// Tile (warp box) and brick extents, in voxels, of a tile configuration
// (compact: vt_options.brick_cfg = 1).
template <class C>
static void dims_of(int* t, int* b) {
  t[0] = C::BXW; t[1] = C::BYW; t[2] = C::BZW;
  b[0] = C::BX; b[1] = C::BY; b[2] = C::BZ;
}
static void cfg_dims(int nd, int compact, int* t, int* b) {
  const int ci = cfg_index(nd, compact);
  if (ci == 0) dims_of<Cfg3>(t, b);
  else if (ci == 1) dims_of<Cfg3c>(t, b);
  else if (ci == 2) dims_of<Cfg2>(t, b);
  else dims_of<Cfg2c>(t, b);
  if (nd == 2) t[2] = b[2] = 1;
}
}  // namespace vt

using namespace vt;

namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kPoolPerBrick = 64;  // culled images reserved per brick of a first-pass chunk
constexpr int kScanTile = 2048;
constexpr int64_t kMaxBins = int64_t(1) << 28;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
  }
  return n;
}

// First-pass staging margin beyond the tile's half-diagonal, in mean cell
// radii (a tile the region does not certify, or a brick whose bound needs
// more under the other certification rule, is staged again with a larger one).
double default_margin_scale(int kind) { return kind == KJ ? 1.5 : kind == KL ? 0.5 : 0.75; }

// Geometry and parameters of one instance (everything but the device pointers
// and the offsets into the concatenated arrays).
struct Plan {
  int nd = 3, kind = 0, prec = 0, cfg = 0, late = 1;
  int direct = 0;  // 1: every brick goes straight to the culling re-run
  int64_t n[3] = {1, 1, 1};
  uint32_t per = 0;
  int64_t n_sites = 0;
  double bin_scale = 1.0, margin_scale = 2.0;
  int bw[3] = {1, 1, 1}, nb[3] = {1, 1, 1}, bricks[3] = {1, 1, 1}, tiles[3] = {1, 1, 1};
  int margin = 1;
  int64_t nbins = 1, nbricks = 1, ntiles = 1;
};

void finish_plan(Plan& p) {
  const int64_t nv = p.n[0] * p.n[1] * p.n[2];
  const double per_site = (double)nv / (double)std::max<int64_t>(p.n_sites, 1);
  // bin width: about bin_scale sites per bin
  double edge = std::pow(per_site * p.bin_scale, 1.0 / p.nd);
  int bw = (int)std::max(1.0, std::floor(edge + 0.5));
  for (;;) {
    int64_t nb = 1;
    for (int a = 0; a < p.nd; a++) nb *= (p.n[a] + bw - 1) / bw;
    if (nb <= kMaxBins) break;
    bw++;
  }
  for (int a = 0; a < 3; a++) {
    p.bw[a] = a < p.nd ? (int)std::min<int64_t>(bw, p.n[a]) : 1;
    p.nb[a] = (int)((p.n[a] + p.bw[a] - 1) / p.bw[a]);
  }
  p.nbins = (int64_t)p.nb[0] * p.nb[1] * p.nb[2];
  // staging margin: margin_scale mean cell radii
  const double rc = p.nd == 3 ? std::cbrt(per_site * 3.0 / (4.0 * M_PI))
                              : std::sqrt(per_site / M_PI);
  int64_t nmax = std::max(p.n[0], std::max(p.n[1], p.n[2]));
  p.margin = (int)std::min<int64_t>(nmax, (int64_t)std::ceil(p.margin_scale * rc) + 1);
  int b[3], t[3];
  cfg_dims(p.nd, p.cfg, t, b);
  p.nbricks = 1;
  p.ntiles = 1;
  for (int a = 0; a < 3; a++) {
    p.bricks[a] = (int)((p.n[a] + b[a] - 1) / b[a]);
    p.tiles[a] = (int)((p.n[a] + t[a] - 1) / t[a]);
    p.nbricks *= p.bricks[a];
    p.ntiles *= p.tiles[a];
  }
}

Inst make_inst(const Plan& p) {
  Inst I;
  std::memset(&I, 0, sizeof(I));
  I.nd = p.nd;
  I.kind = p.kind;
  for (int a = 0; a < 3; a++) {
    I.n[a] = (int32_t)p.n[a];
    I.L[a] = (int32_t)(kQ * p.n[a]);
    I.per[a] = a < p.nd ? (int32_t)((p.per >> a) & 1u) : 0;
    I.bw[a] = p.bw[a];
    I.nb[a] = p.nb[a];
    I.bricks[a] = p.bricks[a];
    I.tiles[a] = p.tiles[a];
  }
  I.cfg = p.cfg;
  I.late = p.late;
  I.margin = p.margin;
  I.precision = p.prec;
  I.n_sites = p.n_sites;
  I.n_bricks = p.nbricks;
  I.n_tiles = p.ntiles;
  return I;
}

// Workspace layout for a set of instances (offsets in bytes).
struct Layout {
  size_t err, cnt, istat, bin_count, bstat, p2_flag, pcur, zero_end;
  size_t bin_start, scan_blk, site_bin, tid_of, spos, saux, sfa, pruned, p2_list, brec, pool, insts,
      total;
  int64_t total_sites, total_bins, total_bricks, total_tiles, pool_cap;
  int n_inst, n_scan_blocks, n_chunks;
};

Layout make_layout(int64_t sites, int64_t bins, int64_t bricks, int64_t tiles, int n_inst,
                   bool aux) {
  Layout L;
  L.total_sites = sites;
  L.total_bins = bins;
  L.total_bricks = bricks;
  L.total_tiles = tiles;
  L.n_inst = n_inst;
  L.n_scan_blocks = (int)((bins + kScanTile - 1) / kScanTile);
  size_t o = 0;
  L.err = o; o = align_up(o + 16);
  L.cnt = o; o = align_up(o + 8 * C_N);
  L.istat = o; o = align_up(o + sizeof(IStat) * n_inst);
  L.bin_count = o; o = align_up(o + 4 * (size_t)bins);
  L.bstat = o; o = align_up(o + (aux ? 16 * (size_t)bins : 0));
  L.p2_flag = o; o = align_up(o + 4 * (size_t)bricks);
  // first pass: one pool cursor per chunk (a batch may split one more chunk
  // at each of its twelve class boundaries)
  const int64_t chunk = vt::pass1_chunk_bricks();
  L.n_chunks = (int)((bricks + chunk - 1) / chunk) + 12;
  L.pcur = o; o = align_up(o + 4 * (size_t)L.n_chunks);
  L.zero_end = o;
  L.bin_start = o; o = align_up(o + 4 * (size_t)(bins + 1));
  L.scan_blk = o; o = align_up(o + 4 * (size_t)(L.n_scan_blocks + 1));
  L.site_bin = o; o = align_up(o + 4 * (size_t)sites);
  L.tid_of = o; o = align_up(o + 4 * (size_t)sites);
  L.spos = o; o = align_up(o + 16 * (size_t)sites);
  L.saux = o; o = align_up(o + (aux ? 16 * (size_t)sites : 0));
  L.sfa = o; o = align_up(o + (aux ? 8 * (size_t)sites : 0));
  L.pruned = o; o = align_up(o + (aux ? (size_t)sites : 0));
  L.p2_list = o; o = align_up(o + 12 * (size_t)bricks);
  L.brec = o; o = align_up(o + sizeof(BrickRec) * (size_t)bricks);
  L.pool_cap = std::min<int64_t>(bricks, chunk) * kPoolPerBrick;
  L.pool = o; o = align_up(o + sizeof(Staged) * (size_t)L.pool_cap);
  L.insts = o; o = align_up(o + sizeof(Inst) * (size_t)n_inst);
  L.total = o;
  return L;
}

Work make_work(const Layout& L, void* ws, bool batch) {
  char* b = static_cast<char*>(ws);
  Work w;
  std::memset(&w, 0, sizeof(w));
  w.err = reinterpret_cast<int32_t*>(b + L.err);
  w.cnt = reinterpret_cast<unsigned long long*>(b + L.cnt);
  w.istat = reinterpret_cast<IStat*>(b + L.istat);
  w.bin_count = reinterpret_cast<int32_t*>(b + L.bin_count);
  w.bstat = reinterpret_cast<unsigned long long*>(b + L.bstat);
  w.bin_start = reinterpret_cast<int32_t*>(b + L.bin_start);
  w.scan_blk = reinterpret_cast<int32_t*>(b + L.scan_blk);
  w.site_bin = reinterpret_cast<int32_t*>(b + L.site_bin);
  w.spos = reinterpret_cast<int4*>(b + L.spos);
  w.saux = reinterpret_cast<longlong2*>(b + L.saux);
  w.sfa = reinterpret_cast<float2*>(b + L.sfa);
  w.pruned = reinterpret_cast<uint8_t*>(b + L.pruned);
  w.p2_list = reinterpret_cast<int32_t*>(b + L.p2_list);
  w.p2_flag = reinterpret_cast<int32_t*>(b + L.p2_flag);
  w.brec = reinterpret_cast<BrickRec*>(b + L.brec);
  w.pool = reinterpret_cast<Staged*>(b + L.pool);
  w.pcur = reinterpret_cast<int32_t*>(b + L.pcur);
  w.pool_cap = L.pool_cap;
  w.insts = batch ? reinterpret_cast<const Inst*>(b + L.insts) : nullptr;
  w.n_inst = L.n_inst;
  w.n_scan_blocks = L.n_scan_blocks;
  w.total_sites = L.total_sites;
  w.total_bins = L.total_bins;
  w.total_bricks = L.total_bricks;
  w.total_tiles = L.total_tiles;
  return w;
}

bool valid_kind(int k) { return k == KV || k == KL || k == KJ; }

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

}  // namespace

struct vt_ctx {
  int nd = 3;
  int64_t n[3] = {1, 1, 1};
  uint32_t per = 0;
  vt_options opt{};
  std::string err;
  void* last_ws = nullptr;
  Layout last_layout{};
  struct Tuned { double bin_scale, margin_scale; int cfg, late, direct; };
  std::map<std::pair<int, int64_t>, Tuned> tuned;  // (kind, n) -> plan parameters
  unsigned long long* host = nullptr;  // pinned readback: err (2 words) + counters
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // stage timing
  bool timed = false;                                                 // last call recorded ev
  bool scored = false;                                                // ... and ev[4]
};

struct vt_batch {
  std::vector<Plan> plans;
  std::vector<vt_instance> inst;
  vt_options opt{};
  std::string err;
  Inst* host_table = nullptr;  // pinned
  Layout layout{};
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  void* graph_ws = nullptr;
  unsigned long long* host = nullptr;
  void* last_ws = nullptr;
  std::vector<int> order;  // device table position -> the caller's instance index
};

namespace {

vt_status cuda_fail(std::string& err, cudaError_t e, const char* what) {
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return VT_ERR_CUDA;
}

// Certification of the first pass: vt_options.certify 1 (after scoring) or 2
// (before scoring), else a default by kind (Johnson-Mehl: before; its cells
// vary most in size) until the autotuner has timed both.
int default_late(const vt_options& o, int kind) {
  return o.certify == 1 ? 1 : o.certify == 2 ? 0 : (kind == KJ ? 0 : 1);
}

Plan ctx_plan(const vt_ctx* c, int kind, int64_t n_sites, double bin_scale, double margin_scale,
              int cfg, int late) {
  Plan p;
  p.nd = c->nd;
  p.kind = kind;
  p.prec = c->opt.precision == VT_EXACT ? P_EXACT : P_F32;
  p.cfg = cfg;
  p.late = late;
  p.direct = c->opt.certify == 3 ? 1 : 0;
  for (int a = 0; a < 3; a++) p.n[a] = c->n[a];
  p.per = c->per;
  p.n_sites = n_sites;
  p.bin_scale = bin_scale;
  p.margin_scale = margin_scale;
  finish_plan(p);
  return p;
}

void ctx_scales(const vt_ctx* c, int kind, int64_t n_sites, double& bs, double& ms, int& cfg,
                int& late) {
  auto it = c->tuned.find({kind, n_sites});
  bs = c->opt.bin_scale > 0 ? c->opt.bin_scale : 1.0;
  ms = c->opt.margin_scale > 0 ? c->opt.margin_scale : default_margin_scale(kind);
  cfg = c->opt.brick_cfg;
  late = default_late(c->opt, kind);
  if (it != c->tuned.end()) {
    bs = it->second.bin_scale;
    ms = it->second.margin_scale;
    cfg = it->second.cfg;
    late = it->second.late;
  }
}

// Whether the tuned plan sends every brick straight to the culling re-run.
int ctx_direct(const vt_ctx* c, int kind, int64_t n_sites) {
  auto it = c->tuned.find({kind, n_sites});
  return it != c->tuned.end() ? it->second.direct : 0;
}

const double kTuneBin[] = {0.5, 1.0, 2.0};
const double kTuneMargin[] = {0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0};

size_t plan_ws_bytes(const Plan& p);

// Time one plan: a warm-up run, then the median of up to three timed runs;
// a plan already slower than 1.5x the best so far is not timed again.
template <class RunF>
vt_status time_plan(std::string& err, const Plan& p, RunF run, cudaStream_t st, double best,
                    double* out_ms) {
  Timer tm;
  float ms[3] = {0.f, 0.f, 0.f};
  int n = 0;
  for (int rep = 0; rep < 4; rep++) {
    cudaEventRecord(tm.a, st);
    vt_status s = run(p);
    if (s != VT_OK) return s;
    cudaEventRecord(tm.b, st);
    cudaError_t e = cudaEventSynchronize(tm.b);
    if (e != cudaSuccess) return cuda_fail(err, e, "autotune");
    float t = 0.f;
    cudaEventElapsedTime(&t, tm.a, tm.b);
    if (rep == 0) continue;  // warm-up
    ms[n++] = t;
    if (t > 1.5 * best) break;
  }
  // median of n <= 3 values
  if (n == 3) {
    const float lo = std::min(ms[0], std::min(ms[1], ms[2]));
    const float hi = std::max(ms[0], std::max(ms[1], ms[2]));
    *out_ms = ms[0] + ms[1] + ms[2] - lo - hi;
  } else {
    *out_ms = n == 2 ? std::max(ms[0], ms[1]) : ms[0];
  }
  return VT_OK;
}

// Search the bin scale and the staging margin: the margin first (at the
// current bin scale), then the bin scale at the best margin.
template <class PlanF, class RunF>
vt_status tune_scales(std::string& err, PlanF plan_of, RunF run, size_t ws_bytes, cudaStream_t st,
                      double& bb, double& bm, double seed = 0.0, double* best_ms = nullptr) {
  double best = 1e300;
  double b0 = bb;
  std::vector<double> margins(std::begin(kTuneMargin), std::end(kTuneMargin));
  bool near = false;
  for (double m : margins) near = near || std::fabs(m - seed) <= 0.1 * m;
  if (seed > 0.0 && !near) margins.push_back(seed);
  for (double m : margins) {
    Plan p = plan_of(b0, m);
    if (plan_ws_bytes(p) > ws_bytes) continue;
    double t;
    vt_status s = time_plan(err, p, run, st, best, &t);
    if (s != VT_OK) return s;
    if (t < best) { best = t; bm = m; bb = b0; }
  }
  for (double b : kTuneBin) {
    if (b == b0) continue;
    Plan p = plan_of(b, bm);
    if (plan_ws_bytes(p) > ws_bytes) continue;
    double t;
    vt_status s = time_plan(err, p, run, st, best, &t);
    if (s != VT_OK) return s;
    if (t < best) { best = t; bb = b; }
  }
  if (best_ms) *best_ms = best;
  return VT_OK;
}

// Time plan p (one alternative setting); take the setting (field(p)) if it is
// faster than best_ms.
template <class RunF, class FieldF>
vt_status tune_cfg(std::string& err, const Plan& p, RunF run, size_t ws_bytes, cudaStream_t st,
                   double& best_ms, int& value, FieldF field) {
  if (plan_ws_bytes(p) > ws_bytes) return VT_OK;
  double t;
  vt_status s = time_plan(err, p, run, st, best_ms, &t);
  if (s != VT_OK) return s;
  if (t < best_ms) {
    value = field(p);
    best_ms = t;
  }
  return VT_OK;
}

size_t plan_ws_bytes(const Plan& p) {
  return make_layout(p.n_sites, p.nbins, p.nbricks, p.ntiles, 1, p.kind != KV).total;
}

vt_status check_ptrs(std::string& err, int kind, const void* sites, const void* w, const void* t,
                     const void* v, const void* labels, const void* ws) {
  if (!sites || !labels || !ws) {
    err = "null device pointer";
    return VT_ERR_ARG;
  }
  if (kind == KL && !w) {
    err = "Laguerre needs weights";
    return VT_ERR_ARG;
  }
  if (kind == KJ && (!t || !v)) {
    err = "Johnson-Mehl needs birth times and speeds";
    return VT_ERR_ARG;
  }
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) {
    err = "workspace must be 256-byte aligned";
    return VT_ERR_ARG;
  }
  return VT_OK;
}

// Enqueue the whole single-grid pipeline.
vt_status run_plan(std::string& err, const Plan& p, const int32_t* sites, const int64_t* w,
                   const double* t, const double* v, int32_t* labels, void* ws, size_t ws_bytes,
                   cudaStream_t st, Layout* out_layout, cudaEvent_t* ev = nullptr,
                   void* scores = nullptr, bool recull = true) {
  const Layout L = make_layout(p.n_sites, p.nbins, p.nbricks, p.ntiles, 1, p.kind != KV);
  if (ws_bytes < L.total) {
    err = "workspace too small: need " + std::to_string(L.total) + " bytes";
    return VT_ERR_WORKSPACE;
  }
  cudaError_t e = init_label_kernels();
  if (e != cudaSuccess) return cuda_fail(err, e, "kernel attributes");
  Work wk = make_work(L, ws, false);
  Inst I = make_inst(p);
  I.sites = sites;
  I.w = w;
  I.t = t;
  I.v = v;
  I.labels = labels;
  I.vec_ok = (I.n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(labels) % 16 == 0);
  char* b = static_cast<char*>(ws);
  if (ev) cudaEventRecord(ev[0], st);
  if ((e = cudaMemsetAsync(b, 0, L.zero_end, st)) != cudaSuccess)
    return cuda_fail(err, e, "memset");
  if ((e = launch_binning(wk, I, reinterpret_cast<int32_t*>(b + L.tid_of), st)) != cudaSuccess)
    return cuda_fail(err, e, "binning launch");
  if (p.kind == KJ) {  // discard the sites reached before their birth, then bin again
    if ((e = launch_jm_prune(wk, I, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(b + L.istat, 0, L.zero_end - L.istat, st)) != cudaSuccess ||
        (e = launch_binning(wk, I, reinterpret_cast<int32_t*>(b + L.tid_of), st, true)) !=
            cudaSuccess)
      return cuda_fail(err, e, "binning launch");
  }
  if (ev) cudaEventRecord(ev[1], st);
  if ((e = p.direct ? launch_list_all(wk, I, st) : launch_pass1(wk, I, sm_count(), st)) !=
          cudaSuccess ||
      (recull && (e = launch_pass1_recull(wk, I, sm_count(), st)) != cudaSuccess))
    return cuda_fail(err, e, "first pass launch");
  if (ev) cudaEventRecord(ev[2], st);
  if ((e = launch_pass2(wk, I, sm_count() * 3, st)) != cudaSuccess)
    return cuda_fail(err, e, "second pass launch");
  if (ev) cudaEventRecord(ev[3], st);
  if (scores) {  // the score image D, from the finished labels
    if ((e = launch_scores(I, wk.err, scores, sm_count(), st)) != cudaSuccess)
      return cuda_fail(err, e, "score image launch");
    if (ev) cudaEventRecord(ev[4], st);
  }
  if (out_layout) *out_layout = L;
  return VT_OK;
}

vt_status read_stats(std::string& err, unsigned long long*& host, void* ws, const Layout& L,
                     cudaStream_t st, vt_stats* stats, int64_t voxels,
                     const std::vector<int>* inst_of = nullptr) {
  if (!ws) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    return VT_OK;
  }
  cudaError_t e;
  if (!host) {
    if ((e = cudaHostAlloc(&host, 16 + 8 * C_N, cudaHostAllocDefault)) != cudaSuccess)
      return cuda_fail(err, e, "cudaHostAlloc");
  }
  char* b = static_cast<char*>(ws);
  if ((e = cudaMemcpyAsync(host, b + L.err, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(host + 2, b + L.cnt, 8 * C_N, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(err, e, "sync");
  int32_t ew[4];
  std::memcpy(ew, host, sizeof(ew));
  if (ew[E_CODE] && inst_of && ew[E_INST] >= 0 && ew[E_INST] < (int)inst_of->size())
    ew[E_INST] = (*inst_of)[ew[E_INST]];  // device table order -> the caller's order
  const unsigned long long* c = host + 2;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->voxels = voxels;
    stats->candidates = (int64_t)c[C_CAND];
    stats->rescored = (int64_t)c[C_RESCORED];
    stats->pass2_bricks = (int64_t)(c[C_P2] - c[C_RECULL]);
    stats->recull_bricks = (int64_t)c[C_RECULL];
    stats->deferred_bricks = (int64_t)c[C_DEFER];
    stats->uniform_tiles = (int64_t)c[C_UNIFORM];
    stats->restaged_bricks = (int64_t)c[C_RESTAGE];
    stats->pruned_sites = (int64_t)c[C_PRUNED];
    stats->long_tiles = (int64_t)c[C_LONG];
    stats->dev_error = ew[E_CODE];
    stats->error_instance = ew[E_CODE] ? ew[E_INST] : -1;
    stats->error_site =
        ew[E_CODE] ? (int64_t)(((uint64_t)(uint32_t)ew[E_SITE_HI] << 32) | (uint32_t)ew[E_SITE_LO])
                   : -1;
  }
  if (ew[E_CODE]) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "input out of range: instance %d, site %lld", ew[E_INST],
                  (long long)(((uint64_t)(uint32_t)ew[E_SITE_HI] << 32) | (uint32_t)ew[E_SITE_LO]));
    err = buf;
    return (vt_status)ew[E_CODE];
  }
  return VT_OK;
}

vt_status ctx_run(vt_ctx* c, int kind, int64_t n_sites, const int32_t* sites, const int64_t* w,
                  const double* t, const double* v, int32_t* labels, void* ws, size_t ws_bytes,
                  void* stream, void* scores = nullptr) {
  if (!c) return VT_ERR_ARG;
  c->err.clear();
  if (n_sites < 1 || n_sites >= 0x7FFFFFFF) {
    c->err = "n_sites out of range";
    return VT_ERR_ARG;
  }
  vt_status s = check_ptrs(c->err, kind, sites, w, t, v, labels, ws);
  if (s != VT_OK) return s;
  double bs, ms;
  int cfg, late;
  ctx_scales(c, kind, n_sites, bs, ms, cfg, late);
  Plan p = ctx_plan(c, kind, n_sites, bs, ms, cfg, late);
  if (c->opt.certify == 0) p.direct = ctx_direct(c, kind, n_sites);
  Layout L;
  cudaEvent_t* ev = nullptr;
  if (c->opt.timing) {
    for (int i = 0; i < 5; i++)
      if (!c->ev[i] && cudaEventCreate(&c->ev[i]) != cudaSuccess) {
        c->err = "cudaEventCreate failed";
        return VT_ERR_CUDA;
      }
    ev = c->ev;
  }
  s = run_plan(c->err, p, sites, w, t, v, labels, ws, ws_bytes,
               static_cast<cudaStream_t>(stream), &L, ev, scores);
  if (s == VT_OK) {
    c->last_ws = ws;
    c->last_layout = L;
    c->timed = ev != nullptr;
    c->scored = scores != nullptr;
  }
  return s;
}

}  // namespace

namespace vt {
// Set the message vt_last_error returns (used by the static-scratch entry point).
void ctx_set_error(vt_ctx* ctx, const std::string& msg) {
  if (ctx) ctx->err = msg;
}

// Scratch bytes of the plan that a call of this context with n_sites sites
// of this kind runs now (its tuned or default bin size and margin).
vt_status ctx_plan_bytes(const vt_ctx* c, int kind, int64_t n_sites, size_t* bytes) {
  if (!c || !bytes || !valid_kind(kind) || n_sites < 1 || n_sites >= 0x7FFFFFFF) return VT_ERR_ARG;
  double bs, ms;
  int cfg, late;
  ctx_scales(c, kind, n_sites, bs, ms, cfg, late);
  *bytes = plan_ws_bytes(ctx_plan(c, kind, n_sites, bs, ms, cfg, late));
  return VT_OK;
}
}  // namespace vt

// ====================================================================== C ABI

extern "C" {

static std::string g_create_err;

vt_status vt_create(vt_ctx** out, int32_t ndim, const int64_t* dims, uint32_t periodic_mask,
                    const vt_options* opt) {
  if (!out || !dims || (ndim != 2 && ndim != 3)) {
    g_create_err = "vt_create: ndim must be 2 or 3 and pointers non-null";
    return VT_ERR_ARG;
  }
  int64_t nv = 1;
  for (int a = 0; a < ndim; a++) {
    if (dims[a] < 1 || dims[a] > kMaxN) {
      g_create_err = "vt_create: each dimension must be in [1, 16384]";
      return VT_ERR_ARG;
    }
    nv *= dims[a];
  }
  if (nv >= (int64_t(1) << 40)) {
    g_create_err = "vt_create: too many voxels";
    return VT_ERR_ARG;
  }
  if (opt && (opt->precision != VT_FP32_RESCORE && opt->precision != VT_EXACT)) {
    g_create_err = "vt_create: unknown precision";
    return VT_ERR_ARG;
  }
  if (opt && (opt->brick_cfg != 0 && opt->brick_cfg != 1)) {
    g_create_err = "vt_create: brick_cfg must be 0 (default tiles) or 1 (compact tiles)";
    return VT_ERR_ARG;
  }
  if (opt && (opt->certify < 0 || opt->certify > 3)) {
    g_create_err = "vt_create: certify must be 0, 1, 2 or 3";
    return VT_ERR_ARG;
  }
  vt_ctx* c = new (std::nothrow) vt_ctx();
  if (!c) return VT_ERR_NOMEM;
  c->nd = ndim;
  for (int a = 0; a < 3; a++) c->n[a] = a < ndim ? dims[a] : 1;
  c->per = periodic_mask & ((1u << ndim) - 1);
  if (opt) c->opt = *opt;
  *out = c;
  return VT_OK;
}

vt_status vt_workspace_size(const vt_ctx* c, int64_t n_sites, int32_t kind, size_t* bytes) {
  if (!c || !bytes || !valid_kind(kind) || n_sites < 1 || n_sites >= 0x7FFFFFFF) return VT_ERR_ARG;
  double bs, ms;
  int cfg, late;
  ctx_scales(c, kind, n_sites, bs, ms, cfg, late);
  size_t need = plan_ws_bytes(ctx_plan(c, kind, n_sites, bs, ms, cfg, late));
  // room for every plan the autotuner may try (bin sizes and tile configurations)
  for (double b : kTuneBin)
    for (int k = 0; k < 2; k++)
      need = std::max(need, plan_ws_bytes(ctx_plan(c, kind, n_sites, b, ms, k, late)));
  *bytes = std::max(need, vt::cost_workspace_bytes());  // the cost model uses it too
  return VT_OK;
}

vt_status vt_voronoi(vt_ctx* c, int64_t n_sites, const int32_t* d_sites, int32_t* d_labels,
                     void* ws, size_t ws_bytes, void* stream) {
  return ctx_run(c, KV, n_sites, d_sites, nullptr, nullptr, nullptr, d_labels, ws, ws_bytes,
                 stream);
}

vt_status vt_laguerre(vt_ctx* c, int64_t n_sites, const int32_t* d_sites, const int64_t* d_w,
                      int32_t* d_labels, void* ws, size_t ws_bytes, void* stream) {
  return ctx_run(c, KL, n_sites, d_sites, d_w, nullptr, nullptr, d_labels, ws, ws_bytes, stream);
}

vt_status vt_johnson_mehl(vt_ctx* c, int64_t n_sites, const int32_t* d_sites, const double* d_t,
                          const double* d_v, int32_t* d_labels, void* ws, size_t ws_bytes,
                          void* stream) {
  return ctx_run(c, KJ, n_sites, d_sites, nullptr, d_t, d_v, d_labels, ws, ws_bytes, stream);
}

// Inputs from host memory, labels stored straight into page-locked host
// memory (over the coherent CPU-GPU link): the inputs are copied into the tail
// of the workspace, then the pipeline runs with the device view of h_labels.
static size_t host_inputs_bytes(const vt_ctx* c, int32_t kind, int64_t n) {
  size_t b = align_up(sizeof(int32_t) * (size_t)c->nd * (size_t)n);
  if (kind == KL) b += align_up(sizeof(int64_t) * (size_t)n);
  if (kind == KJ) b += 2 * align_up(sizeof(double) * (size_t)n);
  return b;
}

vt_status vt_workspace_size_host(const vt_ctx* c, int64_t n_sites, int32_t kind, size_t* bytes) {
  vt_status s = vt_workspace_size(c, n_sites, kind, bytes);
  if (s == VT_OK) *bytes = align_up(*bytes) + host_inputs_bytes(c, kind, n_sites);
  return s;
}

vt_status vt_label_host(vt_ctx* c, int32_t kind, int64_t n_sites, const int32_t* h_sites,
                        const int64_t* h_w, const double* h_t, const double* h_v,
                        int32_t* h_labels, void* ws, size_t ws_bytes, void* stream) {
  if (!c) return VT_ERR_ARG;
  c->err.clear();
  if (!valid_kind(kind) || n_sites < 1 || n_sites >= 0x7FFFFFFF) {
    c->err = "invalid kind or n_sites";
    return VT_ERR_ARG;
  }
  vt_status s = check_ptrs(c->err, kind, h_sites, h_w, h_t, h_v, h_labels, ws);
  if (s != VT_OK) return s;
  size_t base = 0;
  if ((s = vt_workspace_size(c, n_sites, kind, &base)) != VT_OK) return s;
  base = align_up(base);
  if (ws_bytes < base + host_inputs_bytes(c, kind, n_sites)) {
    c->err = "workspace too small (see vt_workspace_size_host)";
    return VT_ERR_WORKSPACE;
  }
  void* dlab = nullptr;
  if (cudaHostGetDevicePointer(&dlab, h_labels, 0) != cudaSuccess || !dlab) {
    cudaGetLastError();
    c->err = "labels must be page-locked host memory mapped into the device address space";
    return VT_ERR_ARG;
  }
  char* tail = static_cast<char*>(ws) + base;
  int32_t* d_sites = reinterpret_cast<int32_t*>(tail);
  tail += align_up(sizeof(int32_t) * (size_t)c->nd * (size_t)n_sites);
  int64_t* d_w = nullptr;
  double *d_t = nullptr, *d_v = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(d_sites, h_sites, sizeof(int32_t) * c->nd * n_sites,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && kind == KL) {
    d_w = reinterpret_cast<int64_t*>(tail);
    e = cudaMemcpyAsync(d_w, h_w, sizeof(int64_t) * n_sites, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess && kind == KJ) {
    d_t = reinterpret_cast<double*>(tail);
    d_v = reinterpret_cast<double*>(tail + align_up(sizeof(double) * n_sites));
    e = cudaMemcpyAsync(d_t, h_t, sizeof(double) * n_sites, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_v, h_v, sizeof(double) * n_sites, cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return cuda_fail(c->err, e, "input copy");
  return ctx_run(c, kind, n_sites, d_sites, d_w, d_t, d_v, static_cast<int32_t*>(dlab), ws, base,
                 stream);
}

vt_status vt_label_scores(vt_ctx* c, int32_t kind, int64_t n_sites, const int32_t* d_sites,
                          const int64_t* d_w, const double* d_t, const double* d_v,
                          int32_t* d_labels, void* d_scores, void* ws, size_t ws_bytes,
                          void* stream) {
  if (!c) return VT_ERR_ARG;
  c->err.clear();
  if (!valid_kind(kind)) {
    c->err = "invalid kind";
    return VT_ERR_ARG;
  }
  if (!d_scores || reinterpret_cast<uintptr_t>(d_scores) % 8) {
    c->err = "scores must be a non-null, 8-byte aligned device buffer";
    return VT_ERR_ARG;
  }
  return ctx_run(c, kind, n_sites, d_sites, d_w, d_t, d_v, d_labels, ws, ws_bytes, stream,
                 d_scores);
}

static vt_status cost_args(vt_ctx* c, int32_t kind, int64_t n_sites, const int64_t* d_w,
                           const double* d_t, const double* d_v, void* ws, size_t ws_bytes) {
  if (!c) return VT_ERR_ARG;
  c->err.clear();
  if (!valid_kind(kind) || n_sites < 1 || n_sites >= 0x7FFFFFFF) {
    c->err = "invalid kind or n_sites";
    return VT_ERR_ARG;
  }
  if ((kind == KL && !d_w) || (kind == KJ && (!d_t || !d_v))) {
    c->err = "missing weights, birth times or speeds";
    return VT_ERR_ARG;
  }
  if (kind != KV && (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign)) {
    c->err = "the cost model needs a 256-byte aligned workspace";
    return VT_ERR_ARG;
  }
  if (kind != KV && ws_bytes < vt::cost_workspace_bytes()) {
    c->err = "workspace too small for the cost model";
    return VT_ERR_WORKSPACE;
  }
  return VT_OK;
}

vt_status vt_cost_model(vt_ctx* c, int32_t kind, int64_t n_sites, const int64_t* d_w,
                        const double* d_t, const double* d_v, const double* thresholds,
                        int32_t n_thresholds, double* evals_per_voxel, void* ws, size_t ws_bytes,
                        void* stream) {
  vt_status s = cost_args(c, kind, n_sites, d_w, d_t, d_v, ws, ws_bytes);
  if (s != VT_OK) return s;
  if (n_thresholds < 0 || (n_thresholds > 0 && (!thresholds || !evals_per_voxel))) {
    c->err = "thresholds and results must be host arrays of n_thresholds values";
    return VT_ERR_ARG;
  }
  if (kind == KV) {  // Eq. nstep12_3d: one ball radius for all sites
    double V = 1.0;
    for (int a = 0; a < c->nd; a++) V *= (double)c->n[a];
    const double coeff = c->nd == 2 ? M_PI : 4.0 * M_PI / 3.0;
    for (int i = 0; i < n_thresholds; i++) {
      const double r2 = std::max(0.0, thresholds[i]);
      const double f = std::min(1.0, coeff * std::pow(r2, 0.5 * c->nd) / V);
      evals_per_voxel[i] = (double)n_sites * (f + std::pow(1.0 - f, (double)n_sites));
    }
    return VT_OK;
  }
  cudaError_t e = cost_model_eval(c->nd, c->n, kind, n_sites, d_w, d_t, d_v, thresholds,
                                  n_thresholds, evals_per_voxel, ws,
                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? VT_OK : cuda_fail(c->err, e, "cost model");
}

vt_status vt_cost_threshold(vt_ctx* c, int32_t kind, int64_t n_sites, const int64_t* d_w,
                            const double* d_t, const double* d_v, double* threshold,
                            double* evals_per_voxel, void* ws, size_t ws_bytes, void* stream) {
  vt_status s = cost_args(c, kind, n_sites, d_w, d_t, d_v, ws, ws_bytes);
  if (s != VT_OK) return s;
  if (!threshold || !evals_per_voxel) {
    c->err = "null result pointer";
    return VT_ERR_ARG;
  }
  double reach = 0.0;
  cudaError_t e = cost_model_threshold(c->nd, c->n, c->per, kind, n_sites, d_w, d_t, d_v,
                                       threshold, evals_per_voxel, &reach, ws,
                                       static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? VT_OK : cuda_fail(c->err, e, "cost model");
}

vt_status vt_autotune(vt_ctx* c, int32_t kind, int64_t n_sites, const int32_t* d_sites,
                      const int64_t* d_w, const double* d_t, const double* d_v,
                      int32_t* d_labels, void* ws, size_t ws_bytes, void* stream) {
  if (!c || !valid_kind(kind)) return VT_ERR_ARG;
  c->err.clear();
  vt_status s = check_ptrs(c->err, kind, d_sites, d_w, d_t, d_v, d_labels, ws);
  if (s != VT_OK) return s;
  double bb = 1.0, bm = default_margin_scale(kind);
  int bc = 0, bl = 1;
  ctx_scales(c, kind, n_sites, bb, bm, bc, bl);
  // seed: the radius of the largest investigation ball of the paper's cost
  // model at its optimal threshold, in mean cell radii, is tried too
  double seed = 0.0;
  if (kind == KV || ws_bytes >= vt::cost_workspace_bytes()) {
    double x = 0.0, cst = 0.0, reach = 0.0;
    cudaError_t e = cost_model_threshold(c->nd, c->n, c->per, kind, n_sites, d_w, d_t, d_v, &x,
                                         &cst, &reach, ws, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c->err, e, "cost model");
    const double nv = (double)(c->n[0] * c->n[1] * c->n[2]);
    const double per_site = nv / (double)n_sites;
    const double rc = c->nd == 3 ? std::cbrt(per_site * 3.0 / (4.0 * M_PI))
                                 : std::sqrt(per_site / M_PI);
    seed = std::min(4.0, std::max(0.25, reach / rc));
  }
  auto run_of = [&](const Plan& p) {
    return run_plan(c->err, p, d_sites, d_w, d_t, d_v, d_labels, ws, ws_bytes,
                    static_cast<cudaStream_t>(stream), nullptr);
  };
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  double best = 0.0;
  // scales first, at the default certification rule and tile shape
  auto plan_of = [&](double b, double m) { return ctx_plan(c, kind, n_sites, b, m, bc, bl); };
  s = tune_scales(c->err, plan_of, run_of, ws_bytes, st, bb, bm, seed, &best);
  if (s != VT_OK) return s;
  // then the other certification rule (unless the options fix it) and the
  // other tile shape, each at the settings chosen so far
  if (c->opt.certify == 0) {
    s = tune_cfg(c->err, ctx_plan(c, kind, n_sites, bb, bm, bc, 1 - bl), run_of, ws_bytes, st, best,
                 bl, [](const Plan& p) { return p.late; });
    if (s != VT_OK) return s;
  }
  s = tune_cfg(c->err, ctx_plan(c, kind, n_sites, bb, bm, 1 - bc, bl), run_of, ws_bytes, st, best,
               bc, [](const Plan& p) { return p.cfg; });
  if (s != VT_OK) return s;
  // last, every brick straight to the culling re-run (pays on clustered
  // sites, whose bricks the staging kernel mostly cannot settle)
  int direct = 0;
  if (c->opt.certify == 0) {
    Plan pd = ctx_plan(c, kind, n_sites, bb, bm, bc, bl);
    pd.direct = 1;
    s = tune_cfg(c->err, pd, run_of, ws_bytes, st, best, direct,
                 [](const Plan& p) { return p.direct; });
    if (s != VT_OK) return s;
  }
  c->tuned[{kind, n_sites}] = {bb, bm, bc, bl, direct};
  return VT_OK;
}

vt_status vt_sync(vt_ctx* c, void* stream, vt_stats* stats) {
  if (!c) return VT_ERR_ARG;
  vt_status s = read_stats(c->err, c->host, c->last_ws, c->last_layout,
                           static_cast<cudaStream_t>(stream), stats, c->n[0] * c->n[1] * c->n[2]);
  if (stats && c->timed) {
    for (int i = 0; i < 3; i++) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]) == cudaSuccess) stats->stage_ms[i] = ms;
    }
    float ms = 0.f;
    if (c->scored && cudaEventElapsedTime(&ms, c->ev[3], c->ev[4]) == cudaSuccess)
      stats->scores_ms = ms;
  }
  return s;
}

const char* vt_last_error(const vt_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

void vt_destroy(vt_ctx* c) {
  if (!c) return;
  if (c->host) cudaFreeHost(c->host);
  for (auto e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

// ------------------------------------------------------------------ batches

vt_status vt_batch_create(vt_batch** out, int32_t n, const vt_instance* in, const vt_options* opt) {
  if (!out || !in || n < 1) return VT_ERR_ARG;
  if (opt && (opt->brick_cfg < 0 || opt->brick_cfg > 1 || opt->certify < 0 || opt->certify > 2)) {
    g_create_err = "vt_batch_create: brick_cfg must be 0 or 1 and certify 0, 1 or 2";
    return VT_ERR_ARG;
  }
  vt_batch* b = new (std::nothrow) vt_batch();
  if (!b) return VT_ERR_NOMEM;
  if (opt) b->opt = *opt;
  int64_t sites = 0, bins = 0, bricks = 0, tiles = 0;
  bool aux = false;
  for (int i = 0; i < n; i++) {
    const vt_instance& x = in[i];
    bool ok = (x.ndim == 2 || x.ndim == 3) && valid_kind(x.kind) && x.n_sites >= 1 &&
              x.d_sites && x.d_labels && (x.kind != KL || x.d_w) &&
              (x.kind != KJ || (x.d_t && x.d_v));
    int64_t nv = 1;
    for (int a = 0; ok && a < x.ndim; a++) {
      ok = x.dims[a] >= 1 && x.dims[a] <= kMaxN;
      nv *= x.dims[a];
    }
    if (!ok || nv >= (int64_t(1) << 40)) {
      delete b;
      g_create_err = "vt_batch_create: instance " + std::to_string(i) + " is invalid";
      return VT_ERR_ARG;
    }
    vt_instance xi = x;
    // page-locked host labels: the kernels store through the device view
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, x.d_labels) == cudaSuccess && pa.type == cudaMemoryTypeHost) {
      void* dl = nullptr;
      if (cudaHostGetDevicePointer(&dl, x.d_labels, 0) != cudaSuccess || !dl) {
        cudaGetLastError();
        delete b;
        g_create_err = "vt_batch_create: labels of instance " + std::to_string(i) +
                       " are host memory not mapped into the device address space";
        return VT_ERR_ARG;
      }
      xi.d_labels = static_cast<int32_t*>(dl);
    }
    cudaGetLastError();  // no device here, or an address unknown to CUDA: taken as given
    Plan p;
    p.nd = x.ndim;
    p.kind = x.kind;
    p.prec = b->opt.precision == VT_EXACT ? P_EXACT : P_F32;
    for (int a = 0; a < 3; a++) p.n[a] = a < x.ndim ? x.dims[a] : 1;
    p.per = x.periodic_mask & ((1u << x.ndim) - 1);
    p.n_sites = x.n_sites;
    p.bin_scale = b->opt.bin_scale > 0 ? b->opt.bin_scale : 1.0;
    p.margin_scale = b->opt.margin_scale > 0 ? b->opt.margin_scale : default_margin_scale(x.kind);
    p.cfg = b->opt.brick_cfg == 1 ? 1 : 0;
    p.late = default_late(b->opt, x.kind);
    finish_plan(p);
    b->plans.push_back(p);
    b->inst.push_back(xi);
    sites += p.n_sites;
    bins += p.nbins;
    bricks += p.nbricks;
    tiles += p.ntiles;
    aux = aux || x.kind != KV;
  }
  if (sites >= 0x7FFFFFFF || bins >= 0x7FFFFFFF || bricks >= 0x7FFFFFFF) {
    delete b;
    g_create_err = "vt_batch_create: batch too large";
    return VT_ERR_ARG;
  }
  b->layout = make_layout(sites, bins, bricks, tiles, n, aux);
  *out = b;
  return VT_OK;
}

static void batch_relayout(vt_batch* b) {
  int64_t sites = 0, bins = 0, bricks = 0, tiles = 0;
  bool aux = false;
  for (auto& p : b->plans) {
    finish_plan(p);
    sites += p.n_sites;
    bins += p.nbins;
    bricks += p.nbricks;
    tiles += p.ntiles;
    aux = aux || p.kind != KV;
  }
  b->layout = make_layout(sites, bins, bricks, tiles, (int)b->plans.size(), aux);
}

vt_status vt_batch_workspace_size(const vt_batch* b, size_t* bytes) {
  if (!b || !bytes) return VT_ERR_ARG;
  // the autotuner may pick smaller bins and compact tiles: reserve for its
  // densest choice
  vt_batch tmp;
  tmp.plans = b->plans;
  for (auto& p : tmp.plans) {
    p.bin_scale = std::min(p.bin_scale, kTuneBin[0]);
    p.cfg = 1;
  }
  batch_relayout(&tmp);
  *bytes = std::max(b->layout.total, tmp.layout.total);
  return VT_OK;
}

// The pinned instance table is allocated outside any stream capture.
static vt_status ensure_host_table(vt_batch* b) {
  if (b->host_table) return VT_OK;
  cudaError_t e = cudaHostAlloc(&b->host_table, sizeof(Inst) * b->plans.size(), cudaHostAllocDefault);
  return e == cudaSuccess ? VT_OK : cuda_fail(b->err, e, "cudaHostAlloc");
}

// Class of an instance: its first-pass kernels (dimension, tile configuration
// and kind), 12 in all.
constexpr int kClasses = 12;
static int batch_class(const Plan& p) { return cfg_index(p.nd, p.cfg) * 3 + p.kind; }

// The device table lists the instances sorted by class (stable), so that each
// class covers a contiguous range of global bricks and one specialized kernel
// per class labels it; every offset follows the table order.
static vt_status batch_enqueue(vt_batch* b, void* ws, cudaStream_t st) {
  const Layout& L = b->layout;
  const int n = (int)b->plans.size();
  cudaError_t e;
  if (!b->host_table) return VT_ERR_ARG;
  b->order.resize(n);
  for (int i = 0; i < n; i++) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    return batch_class(b->plans[x]) < batch_class(b->plans[y]);
  });
  int64_t sb = 0, bb = 0, kb = 0, tb = 0;
  int64_t range[kClasses][2];
  for (int c = 0; c < kClasses; c++) range[c][0] = range[c][1] = 0;
  for (int j = 0; j < n; j++) {
    const int i = b->order[j];
    Inst I = make_inst(b->plans[i]);
    const vt_instance& x = b->inst[i];
    I.sites = x.d_sites;
    I.w = x.d_w;
    I.t = x.d_t;
    I.v = x.d_v;
    I.labels = x.d_labels;
    I.vec_ok = (I.n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(x.d_labels) % 16 == 0);
    I.site_base = sb;
    I.bin_base = bb;
    I.brick_base = kb;
    I.tile_base = tb;
    const int c = batch_class(b->plans[i]);
    if (range[c][1] == range[c][0]) range[c][0] = kb;
    sb += b->plans[i].n_sites;
    bb += b->plans[i].nbins;
    kb += b->plans[i].nbricks;
    tb += b->plans[i].ntiles;
    range[c][1] = kb;
    b->host_table[j] = I;
  }
  if ((e = init_label_kernels()) != cudaSuccess) return cuda_fail(b->err, e, "kernel attributes");
  char* base = static_cast<char*>(ws);
  Work wk = make_work(L, ws, true);
  Inst none;
  std::memset(&none, 0, sizeof(none));
  if ((e = cudaMemsetAsync(base, 0, L.zero_end, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + L.insts, b->host_table, sizeof(Inst) * n, cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return cuda_fail(b->err, e, "batch setup");
  if ((e = launch_binning(wk, none, reinterpret_cast<int32_t*>(base + L.tid_of), st)) !=
      cudaSuccess)
    return cuda_fail(b->err, e, "batch binning");
  bool any_jm = false;
  for (const Plan& p : b->plans) any_jm = any_jm || p.kind == KJ;
  if (any_jm) {  // discard the Johnson-Mehl sites reached before their birth, then bin again
    if ((e = launch_jm_prune(wk, none, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + L.istat, 0, L.zero_end - L.istat, st)) != cudaSuccess ||
        (e = launch_binning(wk, none, reinterpret_cast<int32_t*>(base + L.tid_of), st, true)) !=
            cudaSuccess)
      return cuda_fail(b->err, e, "batch binning");
  }
  const int prec = b->opt.precision == VT_EXACT ? P_EXACT : P_F32;
  int chunk = 0;
  for (int c = 0; c < kClasses; c++) {
    const int ci = c / 3;
    if ((e = launch_pass1_group(wk, ci < 2 ? 3 : 2, ci & 1, c % 3, prec, range[c][0],
                                range[c][1], sm_count(), &chunk, st)) != cudaSuccess)
      return cuda_fail(b->err, e, "batch label");
  }
  if ((e = launch_pass2_batch(wk, sm_count() * 3, st)) != cudaSuccess)
    return cuda_fail(b->err, e, "batch label");
  return VT_OK;
}

vt_status vt_batch_run(vt_batch* b, void* ws, size_t ws_bytes, void* stream, int32_t use_graph) {
  if (!b || !ws) return VT_ERR_ARG;
  b->err.clear();
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) {
    b->err = "workspace must be 256-byte aligned";
    return VT_ERR_ARG;
  }
  if (ws_bytes < b->layout.total) {
    b->err = "workspace too small";
    return VT_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  b->last_ws = ws;
  vt_status hs = ensure_host_table(b);
  if (hs != VT_OK) return hs;
  if (!use_graph) return batch_enqueue(b, ws, st);
  if (!b->exec || b->graph_ws != ws) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
    }
    if ((e = init_label_kernels()) != cudaSuccess) return cuda_fail(b->err, e, "kernel attributes");
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(b->err, e, "stream");
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(b->err, e, "begin capture");
    }
    vt_status s = batch_enqueue(b, ws, cap);
    e = cudaStreamEndCapture(cap, &b->graph);
    cudaStreamDestroy(cap);
    if (s != VT_OK) return s;
    if (e != cudaSuccess) return cuda_fail(b->err, e, "end capture");
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
      return cuda_fail(b->err, e, "instantiate");
    b->graph_ws = ws;
  }
  if ((e = cudaGraphLaunch(b->exec, st)) != cudaSuccess) return cuda_fail(b->err, e, "graph launch");
  return VT_OK;
}

vt_status vt_batch_autotune(vt_batch* b, void* ws, size_t ws_bytes, void* stream) {
  if (!b || !ws) return VT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (size_t i = 0; i < b->plans.size(); i++) {
    const vt_instance& x = b->inst[i];
    const Plan base = b->plans[i];
    auto plan_of = [&](double bs, double m) {
      Plan p = base;
      p.bin_scale = bs;
      p.margin_scale = m;
      finish_plan(p);
      return p;
    };
    // the batch path has no culling re-run (its staging overflows go to the
    // second pass), so its plans are timed without one
    auto run_of = [&](const Plan& p) {
      return run_plan(b->err, p, x.d_sites, x.d_w, x.d_t, x.d_v, x.d_labels, ws, ws_bytes, st,
                      nullptr, nullptr, nullptr, false);
    };
    double bb = base.bin_scale, bm = base.margin_scale, best = 0.0;
    vt_status s = tune_scales(b->err, plan_of, run_of, ws_bytes, st, bb, bm, 0.0, &best);
    if (s != VT_OK) return s;
    Plan pc = plan_of(bb, bm);
    int cfg = pc.cfg, late = pc.late;
    pc.cfg = 1 - pc.cfg;
    finish_plan(pc);
    if ((s = tune_cfg(b->err, pc, run_of, ws_bytes, st, best, cfg,
                      [](const Plan& q) { return q.cfg; })) != VT_OK)
      return s;
    if (b->opt.certify == 0) {  // the other certification rule, at the chosen setting
      Plan pl = plan_of(bb, bm);
      pl.cfg = cfg;
      pl.late = 1 - late;
      finish_plan(pl);
      double tb = 0.0;
      Plan pb = pl;
      pb.late = late;
      if ((s = time_plan(b->err, pb, run_of, st, 1e300, &tb)) != VT_OK ||
          (s = tune_cfg(b->err, pl, run_of, ws_bytes, st, tb, late,
                        [](const Plan& q) { return q.late; })) != VT_OK)
        return s;
    }
    b->plans[i] = plan_of(bb, bm);
    b->plans[i].cfg = cfg;
    b->plans[i].late = late;
    finish_plan(b->plans[i]);
  }
  batch_relayout(b);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  return VT_OK;
}

vt_status vt_batch_sync(vt_batch* b, void* stream, vt_stats* stats) {
  if (!b) return VT_ERR_ARG;
  int64_t nv = 0;
  for (auto& p : b->plans) nv += p.n[0] * p.n[1] * p.n[2];
  return read_stats(b->err, b->host, b->last_ws, b->layout, static_cast<cudaStream_t>(stream),
                    stats, nv, &b->order);
}

const char* vt_batch_last_error(const vt_batch* b) {
  return b ? b->err.c_str() : g_create_err.c_str();
}

void vt_batch_destroy(vt_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->host_table) cudaFreeHost(b->host_table);
  if (b->host) cudaFreeHost(b->host);
  delete b;
}

}  // extern "C"
