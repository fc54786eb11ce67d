"""vt_voronoi_static: Voronoi labels with no device allocation.

Some callers cannot allocate GPU memory at all: plugins whose host application
owns every device allocation and passes in only input and output buffers, or
loops that cannot pay the synchronisation of cudaMalloc and cudaFree.  For
them the library keeps a 64 MiB static device scratch buffer.  This test calls
that entry point through the C ABI twice in a row, on two different inputs so
that the second call starts from the first call's leftovers, and checks each
result against the ordinary workspace entry point (labels are integer ids:
the match must be exact).  It also checks that a problem too large for the
buffer is refused before any GPU work.

The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_13234_gb300 as vt  # noqa: E402

DEV = torch.device("cuda:0")


def _labels_with_workspace(ctx, n, sites, shape, stream):
    ws_bytes = vt.vt_workspace_size(ctx, n, vt.KIND["voronoi"])
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=DEV)
    out = torch.full(shape, -1, dtype=torch.int32, device=DEV)
    vt.vt_voronoi(ctx, n, sites.data_ptr(), out.data_ptr(), ws.data_ptr(), ws_bytes, stream)
    vt.vt_sync(ctx, stream)
    return out


def test_static_scratch_entry_matches_workspace_entry():
    stream = torch.cuda.current_stream().cuda_stream
    cases = [synthetic.make_instance("voronoi", (96, 80, 72), 700, seed=21, periodic=True),
             synthetic.make_instance("voronoi", (300, 257), 1500, seed=22, periodic=False)]
    for inst in cases:  # two calls in a row on the one shared buffer
        mask = (1 << len(inst.dims)) - 1 if inst.periodic else 0
        ctx = vt.vt_create(inst.dims, mask)
        try:
            sites = torch.from_numpy(np.ascontiguousarray(inst.sites)).to(DEV)
            want = _labels_with_workspace(ctx, inst.n_sites, sites, inst.dims[::-1], stream)
            got = torch.full(inst.dims[::-1], -1, dtype=torch.int32, device=DEV)
            vt.vt_voronoi_static(ctx, inst.n_sites, sites.data_ptr(), got.data_ptr(), stream)
            st = vt.vt_sync(ctx, stream)
            assert st["dev_error"] == 0
            assert torch.equal(got, want), f"{inst.name}: {(got != want).sum().item()} labels differ"
        finally:
            vt.vt_destroy(ctx)


def test_static_scratch_refuses_oversized_problems():
    ctx = vt.vt_create((1024, 1024, 1024), 7)
    try:
        n = 5_000_000
        assert vt.vt_workspace_size(ctx, n, vt.KIND["voronoi"]) > 64 << 20
        with pytest.raises(vt.VtError) as e:
            vt.vt_voronoi_static(ctx, n, 256, 256, torch.cuda.current_stream().cuda_stream)
        assert e.value.status == 6
        assert "static" in vt.vt_last_error(ctx)
    finally:
        vt.vt_destroy(ctx)
