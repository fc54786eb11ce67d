"""Python binding of the vt C ABI (``include/vt.h``): argument marshalling only.

Every step of the labelling runs in the CUDA library ``_build/libvt.so``;
PyTorch only provides device memory and streams.  There is no CPU fallback:
if the library is missing or fails to load, every call raises.

The functions named ``vt_*`` mirror the C entry points one to one (pointers
are passed as integers, ``stream`` as a raw ``cudaStream_t`` integer).
``Grid`` and ``Batch`` wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

KIND = {"voronoi": 0, "laguerre": 1, "jm": 2}
VT_FP32_RESCORE = 0
VT_EXACT = 1
STATUS = {0: "VT_OK", 1: "VT_ERR_ARG", 2: "VT_ERR_RANGE", 3: "VT_ERR_CUDA", 4: "VT_ERR_NOMEM",
          5: "VT_ERR_TIMEOUT", 6: "VT_ERR_WORKSPACE"}

EXPORTED = ["vt_create", "vt_workspace_size", "vt_voronoi", "vt_laguerre", "vt_johnson_mehl",
            "vt_label_scores", "vt_workspace_size_host", "vt_label_host",
            "vt_voronoi_static", "vt_cost_model", "vt_cost_threshold", "vt_autotune", "vt_sync", "vt_last_error", "vt_destroy", "vt_batch_create",
            "vt_batch_workspace_size", "vt_batch_autotune", "vt_batch_run", "vt_batch_sync",
            "vt_batch_last_error", "vt_batch_destroy"]


class VtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.stats = None  # vt_sync / vt_batch_sync: the counters of the failed call


class vt_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("brick_cfg", C.c_int32), ("bin_scale", C.c_double),
                ("margin_scale", C.c_double), ("timing", C.c_int32), ("certify", C.c_int32)]


class vt_stats(C.Structure):
    _fields_ = [("voxels", C.c_int64), ("candidates", C.c_int64), ("rescored", C.c_int64),
                ("pass2_bricks", C.c_int64), ("deferred_bricks", C.c_int64),
                ("dev_error", C.c_int32), ("error_instance", C.c_int32),
                ("error_site", C.c_int64), ("stage_ms", C.c_float * 3), ("scores_ms", C.c_float),
                ("uniform_tiles", C.c_int64), ("restaged_bricks", C.c_int64),
                ("pruned_sites", C.c_int64), ("recull_bricks", C.c_int64),
                ("long_tiles", C.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}
        d["stage_ms"] = list(self.stage_ms)
        return d


class vt_instance(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("kind", C.c_int32), ("dims", C.c_int64 * 3),
                ("periodic_mask", C.c_uint32), ("n_sites", C.c_int64), ("d_sites", C.c_void_p),
                ("d_w", C.c_void_p), ("d_t", C.c_void_p), ("d_v", C.c_void_p),
                ("d_labels", C.c_void_p)]


_lib = None


def library_path() -> str:
    """The CUDA library to load: ``VT_LIBRARY`` if set (an alternate build of
    the same sources), else the in-tree build."""
    return os.environ.get("VT_LIBRARY") or _build.LIB


def load(build_if_missing: bool = False):
    """Load ``libvt.so`` (building it first if asked).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and path == _build.LIB:
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P, i32, i64, u32, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_size_t
    sig = {
        "vt_create": ([C.POINTER(P), i32, C.POINTER(C.c_int64), u32, C.POINTER(vt_options)], i32),
        "vt_workspace_size": ([P, i64, i32, C.POINTER(sz)], i32),
        "vt_voronoi": ([P, i64, P, P, P, sz, P], i32),
        "vt_laguerre": ([P, i64, P, P, P, P, sz, P], i32),
        "vt_johnson_mehl": ([P, i64, P, P, P, P, P, sz, P], i32),
        "vt_label_scores": ([P, i32, i64, P, P, P, P, P, P, P, sz, P], i32),
        "vt_workspace_size_host": ([P, i64, i32, C.POINTER(sz)], i32),
        "vt_label_host": ([P, i32, i64, P, P, P, P, P, P, sz, P], i32),
        "vt_voronoi_static": ([P, i64, P, P, P], i32),
        "vt_cost_model": ([P, i32, i64, P, P, P, P, i32, P, P, sz, P], i32),
        "vt_cost_threshold": ([P, i32, i64, P, P, P, P, P, P, sz, P], i32),
        "vt_autotune": ([P, i32, i64, P, P, P, P, P, P, sz, P], i32),
        "vt_sync": ([P, P, C.POINTER(vt_stats)], i32),
        "vt_last_error": ([P], C.c_char_p),
        "vt_destroy": ([P], None),
        "vt_batch_create": ([C.POINTER(P), i32, C.POINTER(vt_instance), C.POINTER(vt_options)],
                            i32),
        "vt_batch_workspace_size": ([P, C.POINTER(sz)], i32),
        "vt_batch_autotune": ([P, P, sz, P], i32),
        "vt_batch_run": ([P, P, sz, P, i32], i32),
        "vt_batch_sync": ([P, P, C.POINTER(vt_stats)], i32),
        "vt_batch_last_error": ([P], C.c_char_p),
        "vt_batch_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


# ---------------------------------------------------------------- raw ABI


def _check(status: int, ctx=None, batch=False):
    if status != 0:
        lib = load()
        msg = (lib.vt_batch_last_error if batch else lib.vt_last_error)(ctx)
        raise VtError(status, (msg or b"").decode())


def vt_create(dims, periodic_mask: int, options: vt_options | None = None) -> int:
    lib = load()
    out = C.c_void_p()
    d = (C.c_int64 * len(dims))(*[int(x) for x in dims])
    _check(lib.vt_create(C.byref(out), len(dims), d, periodic_mask,
                         C.byref(options) if options is not None else None))
    return out.value


def vt_workspace_size(ctx: int, n_sites: int, kind: int) -> int:
    n = C.c_size_t()
    _check(load().vt_workspace_size(ctx, n_sites, kind, C.byref(n)), ctx)
    return n.value


def vt_voronoi(ctx, n_sites, d_sites, d_labels, d_ws, ws_bytes, stream):
    _check(load().vt_voronoi(ctx, n_sites, d_sites, d_labels, d_ws, ws_bytes, stream), ctx)


def vt_laguerre(ctx, n_sites, d_sites, d_w, d_labels, d_ws, ws_bytes, stream):
    _check(load().vt_laguerre(ctx, n_sites, d_sites, d_w, d_labels, d_ws, ws_bytes, stream), ctx)


def vt_johnson_mehl(ctx, n_sites, d_sites, d_t, d_v, d_labels, d_ws, ws_bytes, stream):
    _check(load().vt_johnson_mehl(ctx, n_sites, d_sites, d_t, d_v, d_labels, d_ws, ws_bytes,
                                  stream), ctx)


def vt_label_scores(ctx, kind, n_sites, d_sites, d_w, d_t, d_v, d_labels, d_scores, d_ws,
                    ws_bytes, stream):
    _check(load().vt_label_scores(ctx, kind, n_sites, d_sites, d_w, d_t, d_v, d_labels,
                                  d_scores, d_ws, ws_bytes, stream), ctx)


def vt_workspace_size_host(ctx, n_sites, kind) -> int:
    out = C.c_size_t(0)
    _check(load().vt_workspace_size_host(ctx, n_sites, kind, C.byref(out)), ctx)
    return out.value


def vt_label_host(ctx, kind, n_sites, h_sites, h_w, h_t, h_v, h_labels, d_ws, ws_bytes, stream):
    _check(load().vt_label_host(ctx, kind, n_sites, h_sites, h_w, h_t, h_v, h_labels, d_ws,
                                ws_bytes, stream), ctx)


def vt_voronoi_static(ctx, n_sites, d_sites, d_labels, stream):
    """Voronoi labels on the library's static 64 MiB device scratch (no
    allocation); calls share that buffer, so overlapping calls race."""
    _check(load().vt_voronoi_static(ctx, n_sites, d_sites, d_labels, stream), ctx)


def vt_cost_model(ctx, kind, n_sites, d_w, d_t, d_v, thresholds, d_ws, ws_bytes, stream):
    """The paper's cost model (expected score evaluations per voxel) at each of
    the host ``thresholds``; returns a list of floats."""
    n = len(thresholds)
    xs = (C.c_double * max(n, 1))(*[float(x) for x in thresholds])
    out = (C.c_double * max(n, 1))()
    _check(load().vt_cost_model(ctx, kind, n_sites, d_w, d_t, d_v, xs, n, out, d_ws, ws_bytes,
                                stream), ctx)
    return [out[i] for i in range(n)]


def vt_cost_threshold(ctx, kind, n_sites, d_w, d_t, d_v, d_ws, ws_bytes, stream):
    """(threshold, evals_per_voxel) minimising the paper's cost model."""
    x = C.c_double()
    c = C.c_double()
    _check(load().vt_cost_threshold(ctx, kind, n_sites, d_w, d_t, d_v, C.byref(x), C.byref(c),
                                    d_ws, ws_bytes, stream), ctx)
    return x.value, c.value


def vt_autotune(ctx, kind, n_sites, d_sites, d_w, d_t, d_v, d_labels, d_ws, ws_bytes, stream):
    _check(load().vt_autotune(ctx, kind, n_sites, d_sites, d_w, d_t, d_v, d_labels, d_ws,
                              ws_bytes, stream), ctx)


def _sync_result(status, st, ctx, batch):
    """The counters as a dict; on a device error, VtError with the counters
    (instance and site of the error included) in its ``stats``."""
    if status != 0:
        lib = load()
        msg = (lib.vt_batch_last_error if batch else lib.vt_last_error)(ctx)
        err = VtError(status, (msg or b"").decode())
        err.stats = st.as_dict()
        raise err
    return st.as_dict()


def vt_sync(ctx, stream) -> dict:
    st = vt_stats()
    return _sync_result(load().vt_sync(ctx, stream, C.byref(st)), st, ctx, False)


def vt_last_error(ctx) -> str:
    return (load().vt_last_error(ctx) or b"").decode()


def vt_destroy(ctx):
    load().vt_destroy(ctx)


def vt_batch_create(instances, options: vt_options | None = None) -> int:
    arr = (vt_instance * len(instances))(*instances)
    out = C.c_void_p()
    _check(load().vt_batch_create(C.byref(out), len(instances), arr,
                                  C.byref(options) if options is not None else None),
           None, batch=True)
    return out.value


def vt_batch_workspace_size(b) -> int:
    n = C.c_size_t()
    _check(load().vt_batch_workspace_size(b, C.byref(n)), b, batch=True)
    return n.value


def vt_batch_autotune(b, d_ws, ws_bytes, stream):
    _check(load().vt_batch_autotune(b, d_ws, ws_bytes, stream), b, batch=True)


def vt_batch_run(b, d_ws, ws_bytes, stream, use_graph=1):
    _check(load().vt_batch_run(b, d_ws, ws_bytes, stream, use_graph), b, batch=True)


def vt_batch_sync(b, stream) -> dict:
    st = vt_stats()
    return _sync_result(load().vt_batch_sync(b, stream, C.byref(st)), st, b, True)


def vt_batch_last_error(b) -> str:
    return (load().vt_batch_last_error(b) or b"").decode()


def vt_batch_destroy(b):
    load().vt_batch_destroy(b)


# ---------------------------------------------------------------- torch wrappers


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


def _ws_tensor(nbytes: int, device):
    import torch
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


class Grid:
    """A labelling context for one grid (owns a ``vt_ctx``)."""

    def __init__(self, dims, periodic: bool | int = False, precision: int = VT_FP32_RESCORE,
                 bin_scale: float = 0.0, margin_scale: float = 0.0, brick_cfg: int = 0,
                 timing: bool = False, certify: int = 0):
        self.dims = tuple(int(d) for d in dims)
        mask = periodic if isinstance(periodic, int) and not isinstance(periodic, bool) else \
            ((1 << len(self.dims)) - 1 if periodic else 0)
        self.opt = vt_options(precision, brick_cfg, bin_scale, margin_scale, int(timing), certify)
        self.ctx = vt_create(self.dims, mask, self.opt)
        self._ws = None
        self._ws_host = None

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            try:
                vt_destroy(ctx)
            except Exception:
                pass

    @property
    def n_voxels(self) -> int:
        n = 1
        for d in self.dims:
            n *= d
        return n

    def workspace_size(self, n_sites: int, kind: str) -> int:
        return vt_workspace_size(self.ctx, n_sites, KIND[kind])

    def workspace(self, n_sites: int, kind: str, device="cuda"):
        need = self.workspace_size(n_sites, kind)
        if self._ws is None or self._ws.numel() < need:
            self._ws = _ws_tensor(need, device)
        return self._ws

    def label(self, kind: str, sites, w=None, t=None, v=None, labels=None, workspace=None,
              stream=None):
        """Label every voxel; ``sites`` int32 [N_s, ndim] on the GPU.  Returns the
        int32 label tensor shaped ``dims[::-1]``.  Asynchronous on ``stream``."""
        import torch
        n = int(sites.shape[0])
        dev = sites.device
        if labels is None:
            labels = torch.empty(self.dims[::-1], dtype=torch.int32, device=dev)
        ws = workspace if workspace is not None else self.workspace(n, kind, dev)
        h = _stream_handle(stream)
        nb = ws.numel() * ws.element_size()
        if kind == "voronoi":
            vt_voronoi(self.ctx, n, _ptr(sites), _ptr(labels), _ptr(ws), nb, h)
        elif kind == "laguerre":
            vt_laguerre(self.ctx, n, _ptr(sites), _ptr(w), _ptr(labels), _ptr(ws), nb, h)
        elif kind == "jm":
            vt_johnson_mehl(self.ctx, n, _ptr(sites), _ptr(t), _ptr(v), _ptr(labels), _ptr(ws),
                            nb, h)
        else:
            raise ValueError(kind)
        return labels

    def label_scores(self, kind: str, sites, w=None, t=None, v=None, labels=None, scores=None,
                     workspace=None, stream=None):
        """Labels and the score image D (int64 for Voronoi and Laguerre, float64
        arrival times for Johnson-Mehl), both shaped ``dims[::-1]``.
        Asynchronous on ``stream``; returns (labels, scores)."""
        import torch
        n = int(sites.shape[0])
        dev = sites.device
        if labels is None:
            labels = torch.empty(self.dims[::-1], dtype=torch.int32, device=dev)
        if scores is None:
            scores = torch.empty(self.dims[::-1], device=dev,
                                 dtype=torch.float64 if kind == "jm" else torch.int64)
        ws = workspace if workspace is not None else self.workspace(n, kind, dev)
        vt_label_scores(self.ctx, KIND[kind], n, _ptr(sites), _ptr(w), _ptr(t), _ptr(v),
                        _ptr(labels), _ptr(scores), _ptr(ws), ws.numel() * ws.element_size(),
                        _stream_handle(stream))
        return labels, scores

    def label_host(self, kind: str, sites, w=None, t=None, v=None, labels=None, stream=None,
                   device=None):
        """Label from host tensors (CPU), storing the labels straight into
        ``labels``, a page-locked CPU int32 tensor shaped ``dims[::-1]``
        (allocated pinned when omitted).  Asynchronous on ``stream``: read the
        labels after ``sync``."""
        import torch
        n = int(sites.shape[0])
        if labels is None:
            labels = torch.empty(self.dims[::-1], dtype=torch.int32).pin_memory()
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        need = vt_workspace_size_host(self.ctx, n, KIND[kind])
        key = ("host", n, kind, str(dev))
        if self._ws_host is None or self._ws_host[0] != key:
            self._ws_host = (key, _ws_tensor(need, dev))
        ws = self._ws_host[1]
        vt_label_host(self.ctx, KIND[kind], n, _ptr(sites), _ptr(w), _ptr(t), _ptr(v),
                      _ptr(labels), _ptr(ws), ws.numel(), _stream_handle(stream))
        return labels

    def autotune(self, kind: str, sites, w=None, t=None, v=None, labels=None, stream=None):
        import torch
        n = int(sites.shape[0])
        if labels is None:
            labels = torch.empty(self.dims[::-1], dtype=torch.int32, device=sites.device)
        ws = self.workspace(n, kind, sites.device)
        vt_autotune(self.ctx, KIND[kind], n, _ptr(sites), _ptr(w), _ptr(t), _ptr(v),
                    _ptr(labels), _ptr(ws), ws.numel(), _stream_handle(stream))

    def sync(self, stream=None) -> dict:
        return vt_sync(self.ctx, _stream_handle(stream))

    def cost_model(self, kind: str, n_sites: int, thresholds, w=None, t=None, v=None,
                   stream=None):
        """Expected score evaluations per voxel of the paper's two-step algorithm
        at each threshold (Voronoi r0^2 in voxel^2, Laguerre x in voxel^2,
        Johnson-Mehl t0)."""
        dev = next((a.device for a in (w, t, v) if a is not None), None)
        ws = self.workspace(n_sites, kind, dev if dev is not None else "cuda")
        return vt_cost_model(self.ctx, KIND[kind], n_sites, _ptr(w), _ptr(t), _ptr(v),
                             list(thresholds), _ptr(ws), ws.numel(), _stream_handle(stream))

    def cost_threshold(self, kind: str, n_sites: int, w=None, t=None, v=None, stream=None):
        """(threshold, evals_per_voxel) minimising the paper's cost model."""
        dev = next((a.device for a in (w, t, v) if a is not None), None)
        ws = self.workspace(n_sites, kind, dev if dev is not None else "cuda")
        return vt_cost_threshold(self.ctx, KIND[kind], n_sites, _ptr(w), _ptr(t), _ptr(v),
                                 _ptr(ws), ws.numel(), _stream_handle(stream))


class Batch:
    """Many grids labelled by one persistent launch (CUDA graph replay)."""

    def __init__(self, items, precision: int = VT_FP32_RESCORE, brick_cfg: int = 0):
        """items: list of dicts with keys kind, dims, periodic, sites, w, t, v,
        labels (torch CUDA tensors); the tensors must outlive the batch."""
        self.items = items
        insts = []
        for it in items:
            dims = tuple(int(d) for d in it["dims"])
            d3 = (C.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
            mask = ((1 << len(dims)) - 1) if it["periodic"] else 0
            insts.append(vt_instance(len(dims), KIND[it["kind"]], d3, mask,
                                     int(it["sites"].shape[0]), _ptr(it["sites"]),
                                     _ptr(it.get("w")), _ptr(it.get("t")), _ptr(it.get("v")),
                                     _ptr(it["labels"])))
        self.opt = vt_options(precision, brick_cfg, 0.0, 0.0, 0, 0)
        self.b = vt_batch_create(insts, self.opt)
        self._ws = None

    def __del__(self):
        b = getattr(self, "b", None)
        if b:
            try:
                vt_batch_destroy(b)
            except Exception:
                pass

    def workspace(self, device="cuda"):
        need = vt_batch_workspace_size(self.b)
        if self._ws is None or self._ws.numel() < need:
            self._ws = _ws_tensor(need, device)
        return self._ws

    def autotune(self, stream=None):
        ws = self.workspace()
        vt_batch_autotune(self.b, _ptr(ws), ws.numel(), _stream_handle(stream))

    def run(self, stream=None, use_graph: bool = True):
        ws = self.workspace()
        vt_batch_run(self.b, _ptr(ws), ws.numel(), _stream_handle(stream), int(use_graph))

    def sync(self, stream=None) -> dict:
        return vt_batch_sync(self.b, _stream_handle(stream))
