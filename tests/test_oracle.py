"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: labels
worked out by hand, closed forms of two-site bisectors, the image-sum form of
the periodic distance (Eq. d' of Appendix A), invariances stated in the paper,
brute force against the two-step algorithm, and the numbers the paper prints
for its cost model.  None of these needs a GPU.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic
from synthetic import Instance

HERE = os.path.dirname(os.path.abspath(__file__))
Q = 512


def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


def _inst(kind, dims, periodic, sites, w=None, t=None, v=None):
    return Instance(kind=kind, dims=tuple(dims), periodic=periodic,
                    sites=np.asarray(sites, dtype=np.int32),
                    w=None if w is None else np.asarray(w, dtype=np.int64),
                    t=None if t is None else np.asarray(t, dtype=np.float64),
                    v=None if v is None else np.asarray(v, dtype=np.float64))


def _centres(dims):
    """Voxel centres [N_v, nd] (x fastest), fixed point."""
    grids = np.meshgrid(*[Q * np.arange(n, dtype=np.int64) + Q // 2 for n in dims[::-1]],
                        indexing="ij")
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)


def _image_sum_d2(inst):
    """Squared distance [N_v, N_s] by the image form of Appendix A (Eq. d'):
    the minimum over the shifts k in {-1,0,1}^d of the Euclidean distance,
    which is exact here because every site and voxel lies in the unit cell."""
    c = _centres(inst.dims)
    q = inst.sites.astype(np.int64)
    L = np.array([Q * n for n in inst.dims], dtype=np.int64)
    nd = len(inst.dims)
    if isinstance(inst.periodic, (bool, np.bool_)):
        per = [bool(inst.periodic)] * nd
    else:  # bit i of the mask: axis i is periodic (Appendix A, per-axis periods)
        per = [bool((int(inst.periodic) >> a) & 1) for a in range(nd)]
    shifts = list(itertools.product(*[(-1, 0, 1) if p else (0,) for p in per]))
    best = None
    for k in shifts:
        img = q + np.asarray(k, dtype=np.int64) * L
        d = c[:, None, :] - img[None, :, :]
        d2 = (d * d).sum(axis=2)
        best = d2 if best is None else np.minimum(best, d2)
    return best


def _numpy_labels(inst):
    """Independent brute force in numpy: argmin returns the first (lowest-id)
    minimum, the tie rule of Algorithm 1."""
    D = _image_sum_d2(inst)
    if inst.kind == "voronoi":
        s = D
    elif inst.kind == "laguerre":
        s = D - inst.w[None, :]
    else:
        s = inst.t[None, :] + np.sqrt(D.astype(np.float64)) / (512.0 * inst.v[None, :])
    return np.argmin(s, axis=1).astype(np.int32).reshape(inst.dims[::-1])


def _random_inst(rng, kind, nd, periodic, ns, dims=None, ties=False):
    if dims is None:
        dims = tuple(int(x) for x in rng.integers(3, 13 if nd == 3 else 40, size=nd))
    L = np.array([Q * n for n in dims])
    if ties:
        # sites on a coarse lattice (half voxels) with duplicates: many exact ties
        sites = np.stack([rng.integers(0, 2 * n, size=ns) * (Q // 2) for n in dims], axis=1)
        sites[ns // 2:] = sites[: ns - ns // 2]
    else:
        sites = np.stack([rng.integers(0, l, size=ns) for l in L], axis=1)
    w = t = v = None
    if kind == "laguerre":
        r = rng.integers(0, 4 * Q, size=ns)
        if ties:
            r = (r // Q) * Q
        w = r.astype(np.int64) ** 2
    if kind == "jm":
        t = rng.uniform(0, 5.0, size=ns)
        if ties:
            t = np.floor(t)
        v = rng.choice([0.5, 1.0, 2.0], size=ns)
    return _inst(kind, dims, periodic, sites, w, t, v)


# ---------------------------------------------------------------- hand-worked


@pytest.mark.parametrize("case", _golden("hand_cases.json")["cases"], ids=lambda c: c["name"])
def test_hand_worked_cases(case):
    sites = np.rint(np.asarray(case["sites"]) * Q).astype(np.int32)
    w = t = v = None
    if case["kind"] == "laguerre":
        rq = np.rint(np.asarray(case["radii"]) * Q).astype(np.int64)
        w = rq * rq
    if case["kind"] == "jm":
        t, v = case["t"], case["v"]
    inst = _inst(case["kind"], case["dims"], case["periodic"], sites, w, t, v)
    want = np.asarray(case["labels"], dtype=np.int32)
    assert oracle.brute(inst).ravel().tolist() == want.tolist()
    assert oracle.twostep(inst).ravel().tolist() == want.tolist()


def test_single_site_labels_everything_zero():
    inst = _inst("voronoi", (7, 5, 3), True, [[100, 2000, 900]])
    assert (oracle.brute(inst) == 0).all()
    assert (oracle.twostep(inst) == 0).all()


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("seed", range(6))
def test_two_site_bisector_voronoi_laguerre(seed):
    """Two sites, open box: label 0 iff 2 c.(q1-q0) <= |q1|^2-|q0|^2 + w0 - w1
    (the half-space form of the power bisector; ties go to site 0)."""
    rng = np.random.default_rng(seed)
    for kind in ("voronoi", "laguerre"):
        inst = _random_inst(rng, kind, 3 if seed % 2 else 2, False, 2)
        c = _centres(inst.dims)
        q0, q1 = inst.sites.astype(np.int64)
        w0, w1 = (inst.w if kind == "laguerre" else np.zeros(2, dtype=np.int64))
        lhs = 2 * (c @ (q1 - q0))
        rhs = q1 @ q1 - q0 @ q0 + w0 - w1
        want = np.where(lhs <= rhs, 0, 1).reshape(inst.dims[::-1])
        assert (oracle.brute(inst) == want).all()


@pytest.mark.parametrize("seed", range(4))
def test_two_site_hyperbola_jm(seed):
    """Two sites: label 0 iff d0/(v0) - d1/(v1) <= t1 - t0 (Eq. JM1), checked
    with hypot-based distances wherever the two arrivals differ by > 1e-9."""
    rng = np.random.default_rng(100 + seed)
    inst = _random_inst(rng, "jm", 3 if seed % 2 else 2, False, 2)
    c = _centres(inst.dims).astype(np.float64) / Q
    q = inst.sites.astype(np.float64) / Q
    d0 = np.array([math.hypot(*row) for row in (c - q[0])])
    d1 = np.array([math.hypot(*row) for row in (c - q[1])])
    gap = (inst.t[1] + d1 / inst.v[1]) - (inst.t[0] + d0 / inst.v[0])
    lab = oracle.brute(inst).ravel()
    clear = np.abs(gap) > 1e-9
    assert clear.mean() > 0.9
    assert (lab[clear] == np.where(gap[clear] > 0, 0, 1)).all()


def test_axis_aligned_bisector_counts():
    """Sites mirrored about the plane x = 6 (a voxel face) on a 12 x 5 x 4 box:
    each cell holds exactly half of the voxels."""
    inst = _inst("voronoi", (12, 5, 4), False, [[3 * Q, 2 * Q, Q], [9 * Q, 2 * Q, Q]])
    lab = oracle.brute(inst)
    assert np.bincount(lab.ravel()).tolist() == [120, 120]
    assert (lab[:, :, :6] == 0).all() and (lab[:, :, 6:] == 1).all()


# ------------------------------------------------- periodic distance (App. A)


@pytest.mark.parametrize("kind", ["voronoi", "laguerre", "jm"])
@pytest.mark.parametrize("nd", [2, 3])
def test_brute_matches_image_sum_form(kind, nd):
    rng = np.random.default_rng(7 * nd + len(kind))
    for periodic in (False, True):
        for ties in (False, True):
            inst = _random_inst(rng, kind, nd, periodic, 9, ties=ties)
            assert (oracle.brute(inst) == _numpy_labels(inst)).all()


@pytest.mark.parametrize("kind", ["voronoi", "laguerre", "jm"])
@pytest.mark.parametrize("nd,mask", [(3, 0b001), (3, 0b010), (3, 0b100), (3, 0b101),
                                     (3, 0b011), (2, 0b01), (2, 0b10)])
def test_brute_matches_image_sum_form_mixed_periodicity(kind, nd, mask):
    """Appendix A's periods are per axis: with only some axes periodic, the
    distance is the minimum over the shifts along those axes alone."""
    rng = np.random.default_rng(100 * nd + mask + 7 * len(kind))
    for ties in (False, True):
        inst = _random_inst(rng, kind, nd, mask, 9, ties=ties)
        assert (oracle.brute(inst) == _numpy_labels(inst)).all()
        assert (oracle.twostep(inst) == oracle.brute(inst)).all()


def test_mixed_periodicity_differs_from_both_extremes():
    """A site near the low face of a periodic axis reaches voxels near the
    high face of that axis only: the mixed mask's labels differ from the
    all-open and the all-periodic ones."""
    dims = (12, 10, 8)
    sites = np.array([[Q * 1 + 10, Q * 5, Q * 4], [Q * 6, Q * 5, Q * 4],
                      [Q * 6, Q * 1 + 7, Q * 4]], dtype=np.int32)
    lab = {m: oracle.brute(_inst("voronoi", dims, m, sites)) for m in (0b000, 0b001, 0b111)}
    assert (lab[0b001] != lab[0b000]).any() and (lab[0b001] != lab[0b111]).any()
    # along x the last voxel column is nearer to site 0 through the wrap
    assert lab[0b001][4, 5, 11] == 0 and lab[0b000][4, 5, 11] == 1
    # along y (open in 0b001) the wrap does not apply
    assert lab[0b001][4, 9, 6] == lab[0b000][4, 9, 6]


@pytest.mark.parametrize("kind", ["voronoi", "laguerre", "jm"])
def test_periodic_shift_equivariance(kind):
    """Shifting every site by whole voxels (mod L) rolls the label image."""
    rng = np.random.default_rng(11)
    inst = _random_inst(rng, kind, 3, True, 12, dims=(10, 8, 6))
    lab = oracle.brute(inst)
    shift = np.array([3, -2, 5])
    L = np.array([Q * n for n in inst.dims])
    moved = Instance(**{**inst.__dict__, "sites": np.mod(inst.sites + Q * shift, L).astype(np.int32)})
    lab2 = oracle.brute(moved)
    assert (lab2 == np.roll(lab, shift=tuple(shift[::-1]), axis=(0, 1, 2))).all()


# --------------------------------------------------------------- invariants


def test_laguerre_equal_weights_is_voronoi_and_shift_invariant():
    """Remark of Section 2.3 and Appendix B: equal weights give the Voronoi
    diagram, and a common shift of the weights (time reference) changes nothing."""
    rng = np.random.default_rng(3)
    for periodic in (False, True):
        base = _random_inst(rng, "voronoi", 3, periodic, 15, dims=(11, 9, 7))
        vor = oracle.brute(base)
        lag = Instance(**{**base.__dict__, "kind": "laguerre",
                          "w": np.full(15, 12345, dtype=np.int64)})
        assert (oracle.brute(lag) == vor).all()
        lag2 = _random_inst(rng, "laguerre", 3, periodic, 15, dims=(11, 9, 7))
        shifted = Instance(**{**lag2.__dict__, "w": lag2.w + 987654321})
        assert (oracle.brute(shifted) == oracle.brute(lag2)).all()


def test_jm_equal_times_is_voronoi():
    """Remark of Section 2.3: equal birth times (and speeds) give the Voronoi
    diagram.  Exact in IEEE double here because D < 2^40 and |t| <= 10^3 keep
    distinct square roots distinct after the add."""
    rng = np.random.default_rng(5)
    for periodic in (False, True):
        base = _random_inst(rng, "voronoi", 3, periodic, 20, dims=(12, 10, 8))
        jm = Instance(**{**base.__dict__, "kind": "jm", "t": np.full(20, 37.25),
                         "v": np.full(20, 2.0)})
        assert (oracle.brute(jm) == oracle.brute(base)).all()


@pytest.mark.parametrize("periodic", [False, True])
def test_jm_sites_reached_before_birth_own_no_voxel(periodic):
    """Remark of Section 3.3: a site that a faster-or-equal site reaches before
    its own birth creates no cell.  Dominance is found here in numpy (hypot
    distances, nearest image on a periodic axis) with a 1e-9 gap, and none of
    the dominated sites may appear in the oracle's labels."""
    rng = np.random.default_rng(31 if periodic else 32)
    dims = (14, 12, 10)
    ns = 60
    L = np.array([Q * n for n in dims], dtype=np.float64)
    sites = np.stack([rng.integers(0, int(l), size=ns) for l in L], axis=1)
    t = rng.uniform(0.0, 20.0, size=ns)
    v = rng.choice([0.5, 1.0, 2.0], size=ns)
    inst = _inst("jm", dims, periodic, sites, t=t, v=v)
    q = sites.astype(np.float64)
    dominated = []
    for s_ in range(ns):
        d = q - q[s_]
        if periodic:
            d = d - L * np.round(d / L)
        dist = np.sqrt((d * d).sum(axis=1)) / Q  # voxels
        arrive = t + dist / v                    # each site's arrival at q_s
        ok = (v >= v[s_]) & (np.arange(ns) != s_) & (arrive < t[s_] - 1e-9)
        if ok.any():
            dominated.append(s_)
    assert len(dominated) >= 5  # the case is not vacuous
    lab = oracle.brute(inst)
    assert not np.isin(lab, dominated).any()


@pytest.mark.parametrize("kind", ["voronoi", "laguerre", "jm"])
@pytest.mark.parametrize("periodic", [False, True])
def test_brute_scores_are_the_image_sum_minimum(kind, periodic):
    """The score image: each voxel's best score equals the minimum over the
    sites of the image-sum form (Eq. d'), exactly (int64, or the same IEEE
    double operations in numpy for Johnson-Mehl), and the labels are those of
    the plain brute force."""
    rng = np.random.default_rng(41 + (kind == "jm") + 2 * periodic)
    inst = _random_inst(rng, kind, 3, periodic, 25, dims=(11, 9, 7))
    lab, sc = oracle.brute_scores(inst)
    D = _image_sum_d2(inst)
    if kind == "voronoi":
        want = D.min(axis=1)
    elif kind == "laguerre":
        want = (D - inst.w[None, :]).min(axis=1)
    else:
        arrive = inst.t[None, :] + np.sqrt(D.astype(np.float64)) / (512.0 * inst.v[None, :])
        want = arrive.min(axis=1)
    assert (sc.ravel() == want).all()
    assert (lab == oracle.brute(inst)).all()


def test_voronoi_scores_are_the_squared_distance_transform():
    """With every site at a voxel centre (open box), the Voronoi score image is
    the squared Euclidean distance transform of the site voxels, here taken
    from scipy's exact EDT (times 512^2 for the fixed point)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(43)
    for dims in ((23, 17, 11), (40, 31)):
        ns = 12
        vox = np.stack([rng.integers(0, n, size=ns) for n in dims], axis=1)
        inst = _inst("voronoi", dims, False, vox * Q + Q // 2)
        _, sc = oracle.brute_scores(inst)
        mask = np.ones(dims[::-1], dtype=bool)
        mask[tuple(vox[:, ::-1].T)] = False
        edt = ndimage.distance_transform_edt(mask)
        assert (sc == np.rint(edt * edt).astype(np.int64) * Q * Q).all()


def test_global_invariants_and_duplicates():
    rng = np.random.default_rng(9)
    for kind in ("voronoi", "laguerre", "jm"):
        inst = _random_inst(rng, kind, 3, True, 30, dims=(9, 8, 7))
        inst.sites[20:] = inst.sites[:10]  # ids 20..29 duplicate ids 0..9
        if inst.w is not None:
            inst.w[20:] = inst.w[:10]
        if inst.t is not None:
            inst.t[20:] = inst.t[:10]
            inst.v[20:] = inst.v[:10]
        lab = oracle.brute(inst)
        counts = np.bincount(lab.ravel(), minlength=30)
        assert counts.sum() == inst.n_voxels
        assert lab.min() >= 0 and lab.max() < 30
        assert counts[20:].sum() == 0  # an exact duplicate never beats the lower id


def test_permutation_of_tie_free_sites():
    rng = np.random.default_rng(21)
    inst = _random_inst(rng, "voronoi", 3, False, 25, dims=(10, 9, 8))
    lab = oracle.brute(inst)
    perm = rng.permutation(25)
    moved = Instance(**{**inst.__dict__, "sites": inst.sites[perm]})
    inv = np.argsort(perm)
    assert (oracle.brute(moved) == inv[lab]).all()


# ------------------------------------------------- two-step == brute force


@pytest.mark.parametrize("kind", ["voronoi", "laguerre", "jm"])
def test_twostep_equals_brute_any_threshold(kind):
    """Algorithms 2/3 reach the brute-force labels for every ball size,
    including no balls at all (pure step 2) and balls covering everything."""
    rng = np.random.default_rng(31 + len(kind))
    for trial in range(12):
        nd = 2 + trial % 2
        inst = _random_inst(rng, kind, nd, bool(trial & 2), int(rng.integers(1, 25)),
                            ties=bool(trial & 4))
        want = oracle.brute(inst)
        thr_opt = oracle.default_threshold(inst) if inst.n_sites > 1 else (0, 0.0)
        for thr in (thr_opt, (-1, -1e9), (0, 0.0), (1 << 50, 1e12)):
            got = oracle.twostep(inst, threshold=thr)
            assert (got == want).all(), (trial, thr)


def test_twostep_slabs_tile_the_grid():
    inst = synthetic.make_instance("laguerre", (24, 20, 18), 40, seed=4, periodic=True)
    full = oracle.twostep(inst)
    parts = [oracle.twostep(inst, z0=a, z1=b) for a, b in ((0, 5), (5, 6), (6, 18))]
    assert (np.concatenate(parts, axis=0) == full).all()
    flat = np.arange(0, inst.n_voxels, 97)
    assert (oracle.brute_points(inst, flat) == full.ravel()[flat]).all()


# --------------------------------------------------------- cost model pins


def test_r0_matches_paper():
    g = _golden("paper_values.json")["voronoi_r0_unit_cube_1000_sites"]
    r0 = oracle.voronoi_r0((1, 1, 1), 1000)
    assert abs(r0 - g["value"]) < g["abs_tol"]
    # Eq. v0_3d minimises Eq. nstep12_3d
    f = oracle.v0_fraction(1000)
    for eps in (0.97, 0.99, 1.01, 1.03):
        assert oracle.voronoi_cost(1000, f) < oracle.voronoi_cost(1000, f * eps)


def test_asymptotic_cost():
    g = _golden("paper_values.json")["asymptotic_evaluations_per_voxel"]
    ns = g["n_sites"]
    per_voxel = ns * oracle.voronoi_cost(ns, oracle.v0_fraction(ns))
    assert abs(per_voxel / (math.log(ns) + 1.0) - 1.0) < g["rel_tol"]


def test_count_model_matches_measured_evaluations():
    """Fig. voro4: distance evaluations of Algorithm 2 per voxel and per site
    follow Eq. nstep12_3d, at the optimal r0 and off it."""
    g = _golden("paper_values.json")["voronoi_count_model_200cube_1000_sites"]
    dims, ns = tuple(g["grid"]), g["n_sites"]
    inst = synthetic.make_instance("voronoi", dims, ns, seed=12, periodic=True)
    nv = inst.n_voxels
    r_opt = oracle.voronoi_r0(dims, ns)
    for r in (r_opt, 0.8 * r_opt, 1.2 * r_opt):
        f = (4.0 / 3.0) * math.pi * r ** 3 / nv
        thr = int((Q * r) ** 2)
        _, cnt = oracle.twostep(inst, threshold=(thr, 0.0), return_counts=True)
        measured = (cnt["step1"] + cnt["step2"]) / (nv * ns)
        model = oracle.voronoi_cost(ns, f)
        assert abs(measured / model - 1.0) < g["rel_tol"] * (1 if r == r_opt else 2), (r, measured, model)


def test_growth_search_reduces_to_voronoi_optimum():
    """With equal birth times and speeds, Eq. nstep12_jmak is Eq. nstep12_3d,
    so the searched t0 must give the ball volume of Eq. v0_3d."""
    dims, ns = (100, 100, 100), 2000
    sites = synthetic.uniform_sites(dims, ns, seed=1)
    inst = _inst("jm", dims, True, sites, t=np.zeros(ns), v=np.ones(ns))
    t0 = oracle.growth_threshold(inst)
    f = (4.0 / 3.0) * math.pi * t0 ** 3 / inst.n_voxels
    assert abs(f / oracle.v0_fraction(ns) - 1.0) < 2e-3
    lag = _inst("laguerre", dims, True, sites, w=np.zeros(ns, dtype=np.int64))
    x = oracle.growth_threshold(lag)
    f2 = (4.0 / 3.0) * math.pi * x ** 1.5 / inst.n_voxels
    assert abs(f2 / oracle.v0_fraction(ns) - 1.0) < 2e-3
