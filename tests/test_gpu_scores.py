"""GPU parity of the score image D (vt_label_scores): each voxel's best score
next to its label, as Algorithm 1 keeps them, against the oracle's brute
force (oracle.brute_scores) bit for bit -- int64 squared distances and power
distances, IEEE double Johnson-Mehl arrival times."""
import numpy as np
import pytest

import oracle
import synthetic
from test_gpu_parity import KINDS, PRECS, Q, _t, rand_inst

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_13234_gb300 as vt  # noqa: E402


def gpu_scores(inst, precision=vt.VT_FP32_RESCORE):
    g = vt.Grid(inst.dims, periodic=inst.periodic, precision=precision)
    lab, sc = g.label_scores(inst.kind, _t(inst.sites), w=_t(inst.w), t=_t(inst.t), v=_t(inst.v))
    st = g.sync()
    assert st["dev_error"] == 0
    return lab.cpu().numpy(), sc.cpu().numpy()


def check(inst, what=""):
    want_lab, want_sc = oracle.brute_scores(inst)
    for prec in PRECS:
        lab, sc = gpu_scores(inst, prec)
        assert (lab == want_lab).all(), f"{what} prec={prec}: labels differ"
        assert sc.dtype == want_sc.dtype
        bad = np.argwhere(sc.view(np.int64) != want_sc.view(np.int64))  # bit for bit
        assert bad.size == 0, (f"{what} prec={prec}: {bad.shape[0]} scores differ, first at "
                               f"{tuple(bad[0])}: gpu {sc[tuple(bad[0])]} oracle "
                               f"{want_sc[tuple(bad[0])]}")


@pytest.mark.parametrize("periodic", [False, True, 0b101], ids=["open", "periodic", "mask101"])
@pytest.mark.parametrize("kind", KINDS)
def test_scores_3d(kind, periodic):
    rng = np.random.default_rng(4000 + 10 * KINDS.index(kind) + int(periodic))
    check(rand_inst(rng, kind, (45, 38, 29), periodic, 150), f"{kind} 3d")


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("kind", KINDS)
def test_scores_2d_ragged(kind, periodic):
    rng = np.random.default_rng(5000 + 10 * KINDS.index(kind) + int(periodic))
    check(rand_inst(rng, kind, (203, 131), periodic, 300), f"{kind} 2d")


@pytest.mark.parametrize("kind", KINDS)
def test_scores_ties_and_near_ties(kind):
    rng = np.random.default_rng(6000 + KINDS.index(kind))
    check(rand_inst(rng, kind, (33, 29, 18), True, 60, ties=True), f"{kind} ties")
    base = np.array([[12 * Q, 20 * Q, 16 * Q], [36 * Q, 20 * Q, 16 * Q],
                     [24 * Q, 8 * Q, 16 * Q], [24 * Q, 32 * Q, 16 * Q]], dtype=np.int32)
    inst = synthetic.make_instance(kind, (48, 40, 32), 4, seed=1, periodic=False, sites=base)
    if kind == "laguerre":
        inst.w = np.full(4, 5 * Q * Q, dtype=np.int64)
    if kind == "jm":
        inst.t = np.zeros(4)
        inst.v = np.ones(4)
    check(inst, f"{kind} mirrored sites")


def test_scores_voronoi_sites_at_centres_are_the_squared_edt():
    """Sites at voxel centres: D is 512^2 times the exact squared Euclidean
    distance transform of the site voxels (scipy, no periodicity)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(61)
    dims = (40, 36, 28)
    vox = np.stack([rng.integers(0, n, size=80) for n in dims], axis=1)
    sites = (Q * vox + Q // 2).astype(np.int32)
    inst = synthetic.make_instance("voronoi", dims, 80, seed=1, periodic=False, sites=sites)
    _, sc = gpu_scores(inst)
    mask = np.ones(dims[::-1], dtype=bool)
    mask[tuple(vox[:, ::-1].T)] = False
    edt2 = ndimage.distance_transform_edt(mask) ** 2
    assert (sc == np.rint(edt2 * Q * Q).astype(np.int64)).all()


def test_scores_fullsize_slab():
    """1024^3 periodic Laguerre with 10^6 sites: one z-slab of the score image
    against the brute force (restricted to that slab)."""
    inst = synthetic.precision_1024_1e6("laguerre", False)
    g = vt.Grid(inst.dims, periodic=True)
    lab, sc = g.label_scores(inst.kind, _t(inst.sites), w=_t(inst.w))
    assert g.sync()["dev_error"] == 0
    z = 517
    flat = (z * 1024 * 1024 + np.random.default_rng(3).integers(0, 1024 * 1024, size=300))
    want = oracle.brute_points(inst, flat)
    assert (lab.view(-1)[torch.from_numpy(flat).to(lab.device)].cpu().numpy() == want).all()
    # the scores of those voxels: exact power distances of their labels' sites
    got = sc.view(-1)[torch.from_numpy(flat).to(sc.device)].cpu().numpy()
    c = np.stack([(flat % 1024), (flat // 1024) % 1024, flat // (1024 * 1024)], axis=1)
    c = Q * c + Q // 2
    q = inst.sites[want].astype(np.int64)
    d = c - q
    L = Q * 1024
    d = np.where(d >= L // 2, d - L, np.where(d < -L // 2, d + L, d))
    assert (got == (d * d).sum(axis=1) - inst.w[want]).all()
