"""GPU port of the paper's cost model (vt_cost_model, vt_cost_threshold):
the expected score evaluations per voxel of the two-step algorithm, Eq.
nstep12_jmak with Eq. v' (Johnson-Mehl, Laguerre) and Eqs. nstep12_3d /
v0_3d (Voronoi), against the oracle's CPU evaluation of the same equations,
and the threshold search against the oracle's (same bounds, same scan and
refinement; only the order of the sums over the sites differs)."""
import math

import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_13234_gb300 as vt  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


CASES = [("jm", (96, 80, 64), True, 3000), ("jm", (700, 500), False, 4000),
         ("laguerre", (96, 80, 64), False, 2500), ("laguerre", (600, 600), True, 3000)]


@pytest.mark.parametrize("kind,dims,periodic,ns", CASES)
def test_cost_model_matches_oracle(kind, dims, periodic, ns):
    inst = synthetic.make_instance(kind, dims, ns, seed=17, periodic=periodic)
    g = vt.Grid(dims, periodic=periodic)
    xo = oracle.growth_threshold(inst)
    xs = [xo * f for f in (0.25, 0.5, 0.9, 1.0, 1.1, 2.0, 4.0)] + [-1.0, 0.0]
    got = g.cost_model(kind, ns, xs, w=_t(inst.w), t=_t(inst.t), v=_t(inst.v))
    want = [oracle.growth_cost(inst, x) for x in xs]
    for x, a, b in zip(xs, got, want):
        assert a == pytest.approx(b, rel=1e-9, abs=1e-12), f"x={x}"
    # the search: the GPU's threshold is as good as the oracle's, by the oracle's own measure
    xg, cg = g.cost_threshold(kind, ns, w=_t(inst.w), t=_t(inst.t), v=_t(inst.v))
    co = oracle.growth_cost(inst, xo)
    assert oracle.growth_cost(inst, xg) <= co * (1 + 1e-6)
    assert cg == pytest.approx(oracle.growth_cost(inst, xg), rel=1e-9)
    assert xg == pytest.approx(xo, rel=2e-3, abs=1e-6)


def test_cost_model_repeatable():
    inst = synthetic.make_instance("jm", (64, 64, 64), 5000, seed=3, periodic=True)
    g = vt.Grid(inst.dims, periodic=True)
    a = g.cost_model("jm", inst.n_sites, [5.0, 12.5, 20.0], t=_t(inst.t), v=_t(inst.v))
    b = g.cost_model("jm", inst.n_sites, [5.0, 12.5, 20.0], t=_t(inst.t), v=_t(inst.v))
    assert a == b


@pytest.mark.parametrize("ns", [2, 100, 1000, 10 ** 6])
def test_voronoi_closed_form(ns):
    """Eq. v0_3d: the optimal ball fraction, r0 from it, and Eq. nstep12_3d at
    that ball, per voxel (N_s times the oracle's per-site form)."""
    dims = (200, 200, 200)
    g = vt.Grid(dims, periodic=True)
    x, c = g.cost_threshold("voronoi", ns)
    r0 = oracle.voronoi_r0(dims, ns)
    assert x == pytest.approx(r0 * r0, rel=1e-12)
    f = oracle.v0_fraction(ns)
    assert c == pytest.approx(ns * oracle.voronoi_cost(ns, f), rel=1e-12)
    # the model at other radii is larger (f is its minimiser)
    for s in (0.8, 1.25):
        assert g.cost_model("voronoi", ns, [x * s * s])[0] >= c * (1 - 1e-12)


def test_equal_births_reduce_to_voronoi_ball():
    """With equal births and speeds the Johnson-Mehl balls are all alike, and
    the searched t0 gives the ball volume of Eq. v0_3d (within the search's
    resolution), as for Voronoi diagrams (Section 2.3 remark)."""
    dims, ns = (128, 128, 128), 1000
    inst = synthetic.make_instance("jm", dims, ns, seed=5, periodic=True)
    inst.t = np.zeros(ns)
    inst.v = np.ones(ns)
    g = vt.Grid(dims, periodic=True)
    t0, _ = g.cost_threshold("jm", ns, t=_t(inst.t), v=_t(inst.v))
    v0 = 4.0 / 3.0 * math.pi * t0 ** 3
    assert v0 / (128.0 ** 3) == pytest.approx(oracle.v0_fraction(ns), rel=2e-3)


def test_fullsize_jm_threshold():
    inst = synthetic.jm_1024_1e5()
    g = vt.Grid(inst.dims, periodic=True)
    xg, cg = g.cost_threshold("jm", inst.n_sites, t=_t(inst.t), v=_t(inst.v))
    xo = oracle.growth_threshold(inst)
    assert oracle.growth_cost(inst, xg) <= oracle.growth_cost(inst, xo) * (1 + 1e-6)
    assert cg == pytest.approx(oracle.growth_cost(inst, xg), rel=1e-9)
