"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
entry point that include/vt.h declares, and validates host-side arguments
(no GPU call is made here)."""
import ctypes as C
import os
import re

import pytest

import paper_2201_13234_gb300 as vt
from paper_2201_13234_gb300 import build as vtbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    vtbuild.build()
    return vt.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "vt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert _declared() == sorted(vt.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    # and nothing of the oracle
    assert not hasattr(lib, "vto_brute")


def test_create_validates_arguments(lib):
    with pytest.raises(vt.VtError) as e:
        vt.vt_create((16, 16, 16, 16), 0)
    assert e.value.status == 1
    with pytest.raises(vt.VtError):
        vt.vt_create((0, 16), 0)
    with pytest.raises(vt.VtError):
        vt.vt_create((16385, 16), 0)
    with pytest.raises(vt.VtError):
        vt.vt_create((16, 16), 0, vt.vt_options(7, 0, 0.0, 0.0, 0, 0))
    ctx = vt.vt_create((64, 64, 64), 7)
    assert ctx
    vt.vt_destroy(ctx)


def test_options_validated_host_side(lib):
    """Tile shape 0/1 and certification rules 0-3 are accepted by vt_create;
    anything else is VT_ERR_ARG with a message (no GPU call is made)."""
    for cfg in (0, 1):
        for certify in (0, 1, 2, 3):
            ctx = vt.vt_create((32, 32, 32), 7, vt.vt_options(0, cfg, 0.0, 0.0, 0, certify))
            assert ctx
            vt.vt_destroy(ctx)
    for cfg, certify in ((2, 0), (-1, 0), (0, 4), (0, -1)):
        with pytest.raises(vt.VtError) as e:
            vt.vt_create((32, 32, 32), 7, vt.vt_options(0, cfg, 0.0, 0.0, 0, certify))
        assert e.value.status == 1
        msg = vt.vt_last_error(None)
        assert ("certify" in msg) if certify not in (0,) else ("brick_cfg" in msg)


def test_stats_struct_matches_header(lib):
    """The binding's vt_stats and vt_options mirror include/vt.h field by
    field (names in order), so counters such as long_tiles land where the
    library writes them."""
    text = open(os.path.join(ROOT, "include", "vt.h")).read()
    for struct, cls in (("vt_stats", vt.vt_stats), ("vt_options", vt.vt_options)):
        body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\} " + struct + ";", text,
                         re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"\b([a-z_0-9]+)(?:\[\d+\])?\s*;", body)
        assert names == [f for f, _ in cls._fields_], struct


def test_workspace_size_host_side(lib):
    ctx = vt.vt_create((128, 96, 64), 7)
    try:
        a = vt.vt_workspace_size(ctx, 100, 0)
        b = vt.vt_workspace_size(ctx, 10000, 0)
        c = vt.vt_workspace_size(ctx, 10000, 2)
        assert 0 < a < b < c  # more sites, more bins; JM stores extra per-site data
        assert a % 256 == 0
        with pytest.raises(vt.VtError):
            vt.vt_workspace_size(ctx, 0, 0)
        with pytest.raises(vt.VtError):
            vt.vt_workspace_size(ctx, 10, 5)
    finally:
        vt.vt_destroy(ctx)


def test_calls_reject_null_pointers_before_any_gpu_work(lib):
    ctx = vt.vt_create((32, 32), 3)
    try:
        with pytest.raises(vt.VtError) as e:
            vt.vt_voronoi(ctx, 10, None, None, None, 0, None)
        assert e.value.status == 1
        with pytest.raises(vt.VtError):
            vt.vt_laguerre(ctx, 10, 256, None, 256, 256, 1 << 20, None)  # no weights
        with pytest.raises(vt.VtError):
            vt.vt_voronoi(ctx, 0, 256, 256, 256, 1 << 20, None)  # no sites
        assert "n_sites" in vt.vt_last_error(ctx)
    finally:
        vt.vt_destroy(ctx)


def test_batch_create_validates(lib):
    bad = vt.vt_instance(4, 0, (C.c_int64 * 3)(8, 8, 8), 0, 10, 256, None, None, None, 256)
    with pytest.raises(vt.VtError):
        vt.vt_batch_create([bad])
    good = vt.vt_instance(3, 0, (C.c_int64 * 3)(8, 8, 8), 7, 10, 256, None, None, None, 256)
    b = vt.vt_batch_create([good, good])
    assert vt.vt_batch_workspace_size(b) > 0
    vt.vt_batch_destroy(b)


def test_oracle_is_not_reachable_from_the_package():
    import sys
    import subprocess
    code = ("import sys, paper_2201_13234_gb300 as vt; vt.load(); "
            "assert 'oracle' not in sys.modules; print('ok')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr


def test_absolute_scale_key_arithmetic():
    """The scoring kernel's absolute-scale keys, emulated bit for bit in
    float32 / uint32: with S a power of two, every score F + S below 13 S
    (1 + 2^-20) packs as (bits(F + S) - bits(S)) * 129 + index below 2^32,
    the key order is the (value, index) order, and value and index unpack."""
    import numpy as np
    rng = np.random.default_rng(7)
    for e in (0, 10, 40, 100):
        S = np.float32(2.0 ** e)
        sb = int(np.float32(S).view(np.uint32))
        f = (S + rng.uniform(0, 12.0, 4000).astype(np.float32) * S).astype(np.float32)
        f = np.concatenate([f, np.float32([S, np.float32(13 * S) * np.float32(1 + 2 ** -20)])])
        idx = rng.integers(0, 128, f.size).astype(np.uint64)
        bits = f.view(np.uint32).astype(np.uint64)
        # the kernel computes bits * 129 + (index - 129 bits(S)) modulo 2^32
        key = (bits * 129 + ((idx - 129 * sb) % 2 ** 32)) % 2 ** 32
        exact = (bits - sb) * 129 + idx
        assert (exact < 2 ** 32).all() and (key == exact).all()
        assert (key // 129 + sb == bits).all() and (key % 129 == idx).all()
        order = np.lexsort((idx, f))
        assert (np.diff(key[order].astype(np.int64)) >= 0).all()


def test_batch_rejects_the_every_brick_rule(lib):
    """Batches have no culling re-run, so certify = 3 is refused by
    vt_batch_create before any instance is looked at (no GPU call)."""
    inst = vt.vt_instance(3, 0, (C.c_int64 * 3)(16, 16, 16), 7, 10, 8, None, None, None, 8)
    with pytest.raises(vt.VtError) as e:
        vt.vt_batch_create([inst], vt.vt_options(0, 0, 0.0, 0.0, 0, 3))
    assert e.value.status == 1
    assert "certify" in vt.vt_batch_last_error(None)
