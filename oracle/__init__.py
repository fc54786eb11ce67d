"""CPU oracle for discrete Voronoi / Laguerre / Johnson-Mehl labelling.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it to check and time the CUDA library.  The library never
imports it, and the two share no code; only the seeded generators in
``synthetic`` feed both.

The arithmetic lives in ``vt_oracle.c`` (plain C, OpenMP, no fused
multiply-add); this module compiles it with gcc and calls it through ctypes.

* ``brute``       -- Algorithm 1 of the paper (every voxel x every site).
* ``twostep``     -- Algorithms 2 and 3 and the Laguerre variant (Section 3):
                     investigation balls, then brute force on the voxels left.
* ``*_threshold`` -- the cost model that picks the ball size (Eqs. v0_3d and
                     nstep12_jmak); labels do not depend on it.

Labels come back as int32 arrays shaped ``dims[::-1]`` (x fastest), holding
0-based site ids; ties go to the lowest id.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libvt_oracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"voronoi": 0, "laguerre": 1, "jm": 2}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libvt_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int, C.c_double
            lib.vto_brute.argtypes = [i32, P, i32, i32, i64, P, P, P, P, i64, i64, P, i32]
            lib.vto_brute.restype = i32
            lib.vto_brute_scores.argtypes = [i32, P, i32, i32, i64, P, P, P, P, i64, i64, P, P,
                                             P, i32]
            lib.vto_brute_scores.restype = i32
            lib.vto_brute_points.argtypes = [i32, P, i32, i32, i64, P, P, P, P, i64, P, P, i32]
            lib.vto_brute_points.restype = i32
            lib.vto_twostep.argtypes = [i32, P, i32, i32, i64, P, P, P, P, i64, dbl, i64, i64,
                                        P, P, i32]
            lib.vto_twostep.restype = i32
            lib.vto_v0_fraction.argtypes = [i64]
            lib.vto_v0_fraction.restype = dbl
            lib.vto_voronoi_cost.argtypes = [i64, dbl]
            lib.vto_voronoi_cost.restype = dbl
            lib.vto_voronoi_r0.argtypes = [i32, P, i64]
            lib.vto_voronoi_r0.restype = dbl
            lib.vto_growth_cost.argtypes = [i32, P, i32, i64, P, P, P, dbl]
            lib.vto_growth_cost.restype = dbl
            lib.vto_growth_threshold.argtypes = [i32, P, i32, i32, i64, P, P, P]
            lib.vto_growth_threshold.restype = dbl
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Args:
    """Contiguous copies of an instance's arrays, kept alive for a call."""

    def __init__(self, inst):
        self.nd = len(inst.dims)
        self.dims = np.ascontiguousarray(np.asarray(inst.dims, dtype=np.int64))
        # periodic: True / False for every axis, or an int whose bit i makes axis i periodic
        if isinstance(inst.periodic, (bool, np.bool_)):
            self.mask = (1 << self.nd) - 1 if inst.periodic else 0
        else:
            self.mask = int(inst.periodic) & ((1 << self.nd) - 1)
        self.kind = KIND[inst.kind]
        self.q = np.ascontiguousarray(inst.sites, dtype=np.int32)
        self.ns = int(self.q.shape[0])
        self.w = None if inst.w is None else np.ascontiguousarray(inst.w, dtype=np.int64)
        self.t = None if inst.t is None else np.ascontiguousarray(inst.t, dtype=np.float64)
        self.v = None if inst.v is None else np.ascontiguousarray(inst.v, dtype=np.float64)

    def head(self):
        return (self.nd, _ptr(self.dims), self.mask, self.kind, self.ns, _ptr(self.q),
                _ptr(self.w), _ptr(self.t), _ptr(self.v))


def _slab_shape(inst, z0, z1):
    d = list(inst.dims)
    d[-1] = z1 - z0
    return tuple(d[::-1])


def brute(inst, z0: int = 0, z1: int | None = None, threads: int = 0) -> np.ndarray:
    """Algorithm 1 on the slab z0 <= (last index) < z1."""
    lib = _load()
    a = _Args(inst)
    z1 = inst.dims[-1] if z1 is None else z1
    out = np.empty(_slab_shape(inst, z0, z1), dtype=np.int32)
    rc = lib.vto_brute(*a.head(), z0, z1, _ptr(out), threads)
    if rc:
        raise RuntimeError(f"vto_brute failed ({rc})")
    return out


def brute_scores(inst, z0: int = 0, z1: int | None = None, threads: int = 0):
    """Algorithm 1 on the slab, returning (labels, scores): each voxel's best
    score, int64 (Voronoi D, Laguerre D - w, fixed point) or float64
    (Johnson-Mehl arrival time)."""
    lib = _load()
    a = _Args(inst)
    z1 = inst.dims[-1] if z1 is None else z1
    shape = _slab_shape(inst, z0, z1)
    lab = np.empty(shape, dtype=np.int32)
    if inst.kind == "jm":
        isc, dsc = None, np.empty(shape, dtype=np.float64)
    else:
        isc, dsc = np.empty(shape, dtype=np.int64), None
    rc = lib.vto_brute_scores(*a.head(), z0, z1, _ptr(lab), _ptr(isc), _ptr(dsc), threads)
    if rc:
        raise RuntimeError(f"vto_brute_scores failed ({rc})")
    return lab, (dsc if inst.kind == "jm" else isc)


def brute_points(inst, flat: np.ndarray, threads: int = 0) -> np.ndarray:
    """Algorithm 1 at the voxels with the given flat (x-fastest) indices."""
    lib = _load()
    a = _Args(inst)
    flat = np.ascontiguousarray(flat, dtype=np.int64)
    out = np.empty(flat.shape[0], dtype=np.int32)
    rc = lib.vto_brute_points(*a.head(), flat.shape[0], _ptr(flat), _ptr(out), threads)
    if rc:
        raise RuntimeError(f"vto_brute_points failed ({rc})")
    return out


def v0_fraction(ns: int) -> float:
    return _load().vto_v0_fraction(ns)


def voronoi_cost(ns: int, f: float) -> float:
    return _load().vto_voronoi_cost(ns, f)


def voronoi_r0(dims, ns: int) -> float:
    d = np.asarray(dims, dtype=np.int64)
    return _load().vto_voronoi_r0(len(dims), _ptr(d), ns)


def growth_cost(inst, x: float) -> float:
    a = _Args(inst)
    return _load().vto_growth_cost(a.nd, _ptr(a.dims), a.kind, a.ns, _ptr(a.w), _ptr(a.t),
                                   _ptr(a.v), x)


def growth_threshold(inst) -> float:
    a = _Args(inst)
    return _load().vto_growth_threshold(a.nd, _ptr(a.dims), a.mask, a.kind, a.ns, _ptr(a.w),
                                        _ptr(a.t), _ptr(a.v))


def default_threshold(inst):
    """(thr_i, thr_d) from the paper's cost model: r0^2 for Voronoi (Eq. v0_3d),
    the minimiser of Eq. nstep12_jmak for Laguerre (in 1/512^2 voxel^2) and JM."""
    if inst.kind == "voronoi":
        r0 = voronoi_r0(inst.dims, inst.n_sites)
        return int(np.floor((512.0 * r0) ** 2)), 0.0
    x = growth_threshold(inst)
    if inst.kind == "laguerre":
        return int(np.floor(x * 512.0 * 512.0)), 0.0
    return 0, float(x)


def ball_threshold(inst, radius_vox: float):
    """(thr_i, thr_d) for investigation balls of at least ``radius_vox`` voxels
    (Voronoi and Laguerre: score threshold r^2 in fixed point)."""
    if inst.kind == "jm":
        raise ValueError("use growth_threshold for Johnson-Mehl")
    return int((512.0 * radius_vox) ** 2), 0.0


def twostep(inst, z0: int = 0, z1: int | None = None, threads: int = 0,
            threshold=None, return_counts: bool = False):
    """Algorithms 2/3 on the slab z0 <= (last index) < z1.  ``threshold`` is
    ``(thr_i, thr_d)``; by default the cost model's choice."""
    lib = _load()
    a = _Args(inst)
    z1 = inst.dims[-1] if z1 is None else z1
    thr_i, thr_d = default_threshold(inst) if threshold is None else threshold
    out = np.empty(_slab_shape(inst, z0, z1), dtype=np.int32)
    counts = np.zeros(4, dtype=np.int64)
    rc = lib.vto_twostep(*a.head(), int(thr_i), float(thr_d), z0, z1, _ptr(out), _ptr(counts),
                         threads)
    if rc:
        raise RuntimeError(f"vto_twostep failed ({rc})")
    if return_counts:
        return out, {"step1": int(counts[0]), "step2": int(counts[1]),
                     "left": int(counts[2]), "tested": int(counts[3])}
    return out


def labels(inst, threads: int = 0) -> np.ndarray:
    """Full label image: brute force for small problems, two-step otherwise."""
    if inst.n_voxels * inst.n_sites <= 2_000_000:
        return brute(inst, threads=threads)
    return twostep(inst, threads=threads)
