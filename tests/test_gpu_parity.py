"""GPU parity: labels from the CUDA library (through the C ABI) against the CPU
oracle, element by element, on seeded synthetic inputs.  Labels are integer
site ids, so the bar is bit-exact equality everywhere."""
import math

import numpy as np
import pytest

import oracle
import synthetic
from synthetic import Instance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, never run there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_13234_gb300 as vt  # noqa: E402

Q = 512
DEV = torch.device("cuda:0")


def _t(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_gpu(inst, precision=vt.VT_FP32_RESCORE, **kw):
    g = vt.Grid(inst.dims, periodic=inst.periodic, precision=precision, **kw)
    lab = g.label(inst.kind, _t(inst.sites), w=_t(inst.w), t=_t(inst.t), v=_t(inst.v))
    stats = g.sync()
    return lab.cpu().numpy(), stats


def assert_same(got, want, inst, what=""):
    bad = np.argwhere(got != want)
    if bad.size:
        k = tuple(bad[0])
        raise AssertionError(f"{what} {inst.kind} {inst.dims} periodic={inst.periodic}: "
                             f"{bad.shape[0]} mismatches, first at {k}: gpu {got[k]} oracle {want[k]}")


def rand_inst(rng, kind, dims, periodic, ns, ties=False):
    L = [Q * n for n in dims]
    if ties:
        sites = np.stack([rng.integers(0, 2 * n, size=ns) * (Q // 2) for n in dims], axis=1)
        sites[ns // 2:] = sites[: ns - ns // 2]
    else:
        sites = np.stack([rng.integers(0, l, size=ns) for l in L], axis=1)
    inst = Instance(kind=kind, dims=tuple(dims), periodic=periodic, sites=sites.astype(np.int32))
    if kind == "laguerre":
        r = rng.lognormal(math.log(2.0), 0.5, size=ns)
        rq = np.floor(Q * r + 0.5).astype(np.int64)
        if ties:
            rq = (rq // Q) * Q
        inst.w = rq * rq
    if kind == "jm":
        inst.t = rng.uniform(0, 10.0, size=ns)
        if ties:
            inst.t = np.floor(inst.t)
        inst.v = rng.choice([0.5, 1.0, 1.5], size=ns)
    return inst


KINDS = ["voronoi", "laguerre", "jm"]
PRECS = [vt.VT_FP32_RESCORE, vt.VT_EXACT]


@pytest.mark.parametrize("prec", PRECS, ids=["fp32", "exact"])
@pytest.mark.parametrize("periodic", [False, True], ids=["open", "periodic"])
@pytest.mark.parametrize("kind", KINDS)
def test_parity_3d_ragged(kind, periodic, prec):
    rng = np.random.default_rng(1000 + 10 * KINDS.index(kind) + 2 * int(periodic) + prec)
    inst = rand_inst(rng, kind, (70, 45, 37), periodic, 180)
    got, st = run_gpu(inst, prec)
    assert st["dev_error"] == 0
    assert_same(got, oracle.brute(inst), inst)


@pytest.mark.parametrize("prec", PRECS, ids=["fp32", "exact"])
@pytest.mark.parametrize("periodic", [False, True], ids=["open", "periodic"])
@pytest.mark.parametrize("kind", KINDS)
def test_parity_2d_ragged(kind, periodic, prec):
    rng = np.random.default_rng(2000 + 10 * KINDS.index(kind) + 2 * int(periodic) + prec)
    inst = rand_inst(rng, kind, (301, 211), periodic, 400)
    got, _ = run_gpu(inst, prec)
    assert_same(got, oracle.brute(inst), inst)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("nd,mask", [(3, 0b001), (3, 0b010), (3, 0b100), (3, 0b101),
                                     (3, 0b110), (2, 0b01), (2, 0b10)])
def test_parity_mixed_periodicity(kind, nd, mask):
    """Per-axis periods (Appendix A): only the axes whose bit is set wrap.
    Ragged sizes, both precisions, against the brute force."""
    rng = np.random.default_rng(3000 + 10 * KINDS.index(kind) + mask + 100 * nd)
    dims = (70, 45, 37) if nd == 3 else (301, 211)
    inst = rand_inst(rng, kind, dims, mask, 180 if nd == 3 else 400)
    want = oracle.brute(inst)
    for prec in PRECS:
        got, st = run_gpu(inst, prec)
        assert st["dev_error"] == 0
        assert_same(got, want, inst, f"mask={mask:b} prec={prec}")
    # sites near the faces: the wrap matters on the periodic axes only
    near = inst.sites.copy()
    L = np.array([Q * n for n in dims])
    near[: len(near) // 2] = np.where(near[: len(near) // 2] < L // 2,
                                      near[: len(near) // 2] % (2 * Q),
                                      L - 1 - near[: len(near) // 2] % (2 * Q))
    inst.sites = near.astype(np.int32)
    got, _ = run_gpu(inst)
    assert_same(got, oracle.brute(inst), inst, f"faces, mask={mask:b}")


@pytest.mark.parametrize("prec", PRECS, ids=["fp32", "exact"])
@pytest.mark.parametrize("nd", [3, 2])
@pytest.mark.parametrize("kind", KINDS)
def test_parity_compact_tiles(kind, nd, prec):
    """brick_cfg = 1: compact warp tiles (8x8x4 voxels, 2D 16x16) in both
    passes, ragged sizes, open and periodic, with ties."""
    rng = np.random.default_rng(7000 + 10 * KINDS.index(kind) + nd + prec)
    dims = (70, 45, 37) if nd == 3 else (301, 211)
    for periodic in (False, True):
        for ties in (False, True):
            inst = rand_inst(rng, kind, dims, periodic, 180 if nd == 3 else 400, ties=ties)
            got, st = run_gpu(inst, prec, brick_cfg=1)
            assert st["dev_error"] == 0
            assert_same(got, oracle.brute(inst), inst, f"compact ties={ties}")


@pytest.mark.parametrize("kind", KINDS)
def test_compact_tiles_clustered_and_second_pass(kind):
    """Compact tiles with dense clusters: list overflows reach the second pass
    and its bricks (16x16x4) are labelled exactly."""
    dims = (96, 80, 64)
    dense = synthetic.matern_sites(dims, 6, 400.0, 3.0, seed=10, periodic=True)
    inst = synthetic.make_instance(kind, dims, dense.shape[0], seed=10, periodic=True, sites=dense)
    if kind == "jm":
        inst.t = np.zeros_like(inst.t)
    want = oracle.brute(inst)
    for prec in PRECS:
        got, st = run_gpu(inst, prec, brick_cfg=1, margin_scale=0.05)
        assert_same(got, want, inst, "compact, dense clusters")
    sites = synthetic.matern_sites((128, 128, 128), 20, 100.0, 8.0, seed=21, periodic=True)
    inst = synthetic.make_instance(kind, (128, 128, 128), sites.shape[0], seed=21, periodic=True,
                                   sites=sites)
    got, st = run_gpu(inst, brick_cfg=1)
    assert_same(got, oracle.twostep(inst), inst, "compact, voids")


@pytest.mark.parametrize("certify", [1, 2, 3])
@pytest.mark.parametrize("kind", KINDS)
def test_both_certification_rules_exact(kind, certify):
    """vt_options.certify: tiles certified after scoring (1; a tile whose
    unstaged sites could still win sends its brick to the re-run), bricks
    grown until certified before scoring (2), or every brick straight to the
    re-run, which culls as it stages (3).  Small margins make the first rule
    fail often; labels are exact either way."""
    rng = np.random.default_rng(8000 + 10 * KINDS.index(kind) + certify)
    cases = [((70, 45, 37), False), ((70, 45, 37), True)]
    if certify == 3:  # 2D bricks (32 x 64, ragged) through the re-run too
        cases += [((150, 210), False), ((150, 210), 0b01)]
    for dims, periodic in cases:
        inst = rand_inst(rng, kind, dims, periodic, 250)
        for ms in (0.05, 0.5, 2.0):
            for prec in PRECS:
                got, st = run_gpu(inst, prec, certify=certify, margin_scale=ms)
                assert st["dev_error"] == 0
                assert_same(got, oracle.brute(inst), inst, f"certify={certify} ms={ms}")
                if certify == 3:
                    assert st["deferred_bricks"] > 0
    with pytest.raises(vt.VtError):
        vt.Grid((16, 16, 16), certify=4)


def test_brick_cfg_validated_and_autotuned():
    with pytest.raises(vt.VtError):
        vt.Grid((16, 16, 16), brick_cfg=2)
    inst = synthetic.make_instance("laguerre", (96, 64, 48), 400, seed=12, periodic=True)
    for cfg in (0, 1):
        g = vt.Grid(inst.dims, periodic=True, brick_cfg=cfg)
        g.autotune("laguerre", _t(inst.sites), w=_t(inst.w))
        lab = g.label("laguerre", _t(inst.sites), w=_t(inst.w))
        g.sync()
        assert_same(lab.cpu().numpy(), oracle.brute(inst), inst, f"autotuned from cfg {cfg}")


@pytest.mark.parametrize("kind", KINDS)
def test_parity_ties_and_duplicates(kind):
    rng = np.random.default_rng(7)
    for periodic in (False, True):
        for dims in ((33, 29, 18), (90, 77)):
            inst = rand_inst(rng, kind, dims, periodic, 60, ties=True)
            want = oracle.brute(inst)
            for prec in PRECS:
                got, _ = run_gpu(inst, prec)
                assert_same(got, want, inst, f"prec={prec}")


@pytest.mark.parametrize("kind", KINDS)
def test_edge_cases(kind):
    rng = np.random.default_rng(3)
    cases = [
        rand_inst(rng, kind, (24, 20, 12), True, 1),      # one site: all labels 0
        rand_inst(rng, kind, (24, 20, 12), False, 2),
        rand_inst(rng, kind, (5, 3, 7), True, 3),         # warp box wider than half a period
        rand_inst(rng, kind, (3, 2), True, 4),
        rand_inst(rng, kind, (1, 1, 1), True, 5),
        rand_inst(rng, kind, (1, 97), False, 9),          # 1-voxel-thick grids
        rand_inst(rng, kind, (64, 1, 40), True, 30),
        rand_inst(rng, kind, (130, 1), True, 7),
    ]
    for inst in cases:
        want = oracle.brute(inst)
        for prec in PRECS:
            got, _ = run_gpu(inst, prec)
            assert_same(got, want, inst, f"prec={prec}")


@pytest.mark.parametrize("kind", KINDS)
def test_clustered_sites_and_second_pass(kind):
    """Matern clusters leave large voids (the first pass grows its seed rings
    far); clusters too dense for even the culling re-run's larger staging
    area (1 500 sites within 4 voxels) go to the second pass, which grows
    rings from a margin."""
    dims = (96, 80, 64)
    sites = synthetic.matern_sites(dims, 12, 25.0, 4.0, seed=9, periodic=True)
    inst = synthetic.make_instance(kind, dims, sites.shape[0], seed=9, periodic=True, sites=sites)
    want = oracle.twostep(inst)
    for ms in (0.0, 0.05, 6.0):
        got, st = run_gpu(inst, margin_scale=ms)
        assert_same(got, want, inst, f"margin_scale={ms}")
    dense = synthetic.matern_sites(dims, 6, 1500.0, 4.0, seed=10, periodic=True)
    inst = synthetic.make_instance(kind, dims, dense.shape[0], seed=10, periodic=True, sites=dense)
    if kind == "jm":
        # equal births: no site is reached by another before its own birth, so
        # none is pruned and the dense clusters still overflow the first pass
        inst.t = np.zeros_like(inst.t)
    want = oracle.brute(inst)
    for prec in PRECS:
        for ms in (0.05, 2.0):
            got, st = run_gpu(inst, prec, margin_scale=ms)
            assert_same(got, want, inst, f"dense clusters, margin_scale={ms}")
            assert st["pass2_bricks"] > 0
            assert st.get("pruned_sites", 0) == 0


@pytest.mark.parametrize("kind", ["voronoi", "laguerre"])
def test_matern_voids_settled_by_culling_rerun(kind):
    """Matern clusters at the density of the 1024^3 / 10^6-site workload
    (10^4 parents per 1024^3, 100 children within 8 voxels), on 128^3: the
    regions of bricks in the voids between clusters hold more sites than the
    staging area, so the first pass lists them; its culling re-run stages
    them again, dropping far sites as it goes, and settles most of them."""
    dims = (128, 128, 128)
    sites = synthetic.matern_sites(dims, 20, 100.0, 8.0, seed=21, periodic=True)
    inst = synthetic.make_instance(kind, dims, sites.shape[0], seed=21, periodic=True, sites=sites)
    want = oracle.twostep(inst)
    for prec in PRECS:
        got, st = run_gpu(inst, prec)
        assert_same(got, want, inst, f"precision={prec}")
        assert st["deferred_bricks"] > 0
        assert st["recull_bricks"] > 0
        assert st["pass2_bricks"] < st["deferred_bricks"]


def test_matern_voids_with_duplicate_sites_lowest_id_wins():
    """The clustered workload with every site doubled (the copy has the higher
    id): each voxel's best score is an exact tie, which the culling re-run's
    8-bit keys and the second pass must both resolve to the lower id."""
    dims = (128, 128, 128)
    base = synthetic.matern_sites(dims, 20, 50.0, 8.0, seed=22, periodic=True)
    sites = np.concatenate([base, base])
    inst = synthetic.make_instance("voronoi", dims, sites.shape[0], seed=22, periodic=True,
                                   sites=sites)
    want = oracle.twostep(inst)
    assert want.max() < base.shape[0]  # the copies never win
    for prec in PRECS:
        got, st = run_gpu(inst, prec)
        assert_same(got, want, inst, f"duplicates, precision={prec}")
        assert st["recull_bricks"] > 0


@pytest.mark.parametrize("kind", KINDS)
def test_bin_scales(kind):
    rng = np.random.default_rng(12)
    inst = rand_inst(rng, kind, (60, 52, 44), True, 250)
    want = oracle.brute(inst)
    for bs in (0.05, 0.5, 4.0, 64.0):
        got, _ = run_gpu(inst, bin_scale=bs)
        assert_same(got, want, inst, f"bin_scale={bs}")


def test_heavy_weights_and_late_births():
    rng = np.random.default_rng(5)
    inst = rand_inst(rng, "laguerre", (72, 64, 40), False, 120)
    inst.w[::17] = (Q * 40) ** 2  # a few huge cells
    assert_same(run_gpu(inst)[0], oracle.twostep(inst), inst)
    jm = rand_inst(rng, "jm", (72, 64, 40), True, 300)
    jm.t = rng.uniform(0, 1000.0, size=300)  # most sites are swallowed before birth
    jm.v = np.full(300, 0.25)
    assert_same(run_gpu(jm)[0], oracle.twostep(jm), jm)


def test_near_ties_rescored_exactly():
    """Sites mirrored about voxel planes put many voxel centres exactly on a
    bisector; +-1 fixed-point offsets put others within one unit of it."""
    dims = (48, 40, 32)
    base = np.array([[12 * Q, 20 * Q, 16 * Q], [36 * Q, 20 * Q, 16 * Q],
                     [24 * Q, 8 * Q, 16 * Q], [24 * Q, 32 * Q, 16 * Q]], dtype=np.int64)
    pert = base.copy()
    pert[1, 0] += 1
    pert[3, 1] -= 1
    for sites in (base, pert):
        for kind in KINDS:
            inst = synthetic.make_instance(kind, dims, 4, seed=1, periodic=False,
                                           sites=sites.astype(np.int32))
            if kind == "laguerre":
                inst.w = np.full(4, 5 * Q * Q, dtype=np.int64)
            if kind == "jm":
                inst.t = np.zeros(4)
                inst.v = np.ones(4)
            want = oracle.brute(inst)
            got, st = run_gpu(inst)
            assert_same(got, want, inst)
            if sites is base:
                assert st["rescored"] > 0


def test_fp32_and_exact_agree_and_deterministic():
    inst = synthetic.make_instance("laguerre", (128, 128, 128), 2000, seed=8, periodic=True)
    a, sa = run_gpu(inst)
    b, sb = run_gpu(inst)
    c, _ = run_gpu(inst, vt.VT_EXACT)
    assert (a == b).all() and (a == c).all()
    assert sa == sb
    flat = np.random.default_rng(0).integers(0, inst.n_voxels, size=3000)
    assert (a.ravel()[flat] == oracle.brute_points(inst, flat)).all()


def test_out_of_range_site_reported_not_faulted():
    inst = synthetic.make_instance("voronoi", (32, 32, 32), 50, seed=1, periodic=True)
    inst.sites[17, 1] = Q * 32  # == L: outside [0, L)
    g = vt.Grid(inst.dims, periodic=True)
    g.label("voronoi", _t(inst.sites))
    with pytest.raises(vt.VtError) as e:
        g.sync()
    assert e.value.status == 2
    bad = rand_inst(np.random.default_rng(0), "jm", (16, 16), False, 10)
    bad.v[3] = 0.0
    g2 = vt.Grid(bad.dims)
    g2.label("jm", _t(bad.sites), t=_t(bad.t), v=_t(bad.v))
    with pytest.raises(vt.VtError):
        g2.sync()
    # the context stays usable afterwards
    ok, _ = run_gpu(synthetic.make_instance("voronoi", (32, 32, 32), 50, seed=1, periodic=True))
    assert ok.min() >= 0


INVALID = [
    ("voronoi", "site", -1),
    ("voronoi", "site", None),             # == L: outside [0, L)
    ("laguerre", "w", -1),
    ("laguerre", "w", 2 ** 52),
    ("jm", "t", float("nan")),
    ("jm", "t", float("inf")),
    ("jm", "t", -float("inf")),
    ("jm", "t", 2.0 ** 40),
    ("jm", "t", -(2.0 ** 40)),
    ("jm", "v", 0.0),
    ("jm", "v", -1.0),
    ("jm", "v", 1e-13),
    ("jm", "v", 1.5e12),
    ("jm", "v", float("nan")),
    ("jm", "v", float("inf")),
]


@pytest.mark.parametrize("kind,field,value", INVALID,
                         ids=[f"{k}-{f}-{v}" for k, f, v in INVALID])
def test_invalid_input_reported_with_site_and_context_usable(kind, field, value):
    """Each out-of-range site coordinate, weight, birth time or speed is found
    on the device (no trap): vt_sync returns VT_ERR_RANGE naming the site, and
    the context labels the next, valid input correctly."""
    inst = synthetic.make_instance(kind, (32, 24, 20), 60, seed=2, periodic=True)
    good = synthetic.make_instance(kind, (32, 24, 20), 60, seed=2, periodic=True)
    bad_site = 41
    if field == "site":
        inst.sites[bad_site, 1] = Q * 24 if value is None else value
    else:
        arr = getattr(inst, field).copy()
        arr[bad_site] = value
        setattr(inst, field, arr)
    g = vt.Grid(inst.dims, periodic=True)
    g.label(kind, _t(inst.sites), w=_t(inst.w), t=_t(inst.t), v=_t(inst.v))
    with pytest.raises(vt.VtError) as e:
        g.sync()
    assert e.value.status == 2
    assert e.value.stats["dev_error"] == 2
    assert e.value.stats["error_instance"] == 0 and e.value.stats["error_site"] == bad_site
    lab = g.label(kind, _t(good.sites), w=_t(good.w), t=_t(good.t), v=_t(good.v))
    assert g.sync()["dev_error"] == 0
    assert_same(lab.cpu().numpy(), oracle.brute(good), good, "after an error")


def test_invalid_input_in_batch_names_the_instance():
    insts = _batch_items(6, seed=9)
    j = next(i for i, x in enumerate(insts) if x.kind == "jm" and i > 0)
    insts[j].t = insts[j].t.copy()
    insts[j].t[insts[j].n_sites - 1] = float("nan")
    items = [dict(kind=i.kind, dims=i.dims, periodic=i.periodic, sites=_t(i.sites), w=_t(i.w),
                  t=_t(i.t), v=_t(i.v),
                  labels=torch.empty(i.dims[::-1], dtype=torch.int32, device=DEV)) for i in insts]
    b = vt.Batch(items)
    b.run()
    with pytest.raises(vt.VtError) as e:
        b.sync()
    assert e.value.stats["error_instance"] == j
    assert e.value.stats["error_site"] == insts[j].n_sites - 1


def test_autotune_keeps_labels_exact():
    inst = synthetic.make_instance("jm", (96, 96, 64), 500, seed=4, periodic=True)
    g = vt.Grid(inst.dims, periodic=True)
    args = dict(w=None, t=_t(inst.t), v=_t(inst.v))
    g.autotune("jm", _t(inst.sites), **args)
    lab = g.label("jm", _t(inst.sites), **args)
    g.sync()
    assert_same(lab.cpu().numpy(), oracle.twostep(inst), inst)


def _batch_items(n, seed):
    insts = []
    rng = np.random.default_rng(seed)
    for j in range(n):
        kind = KINDS[j % 3]
        nd = 2 + (j // 3) % 2
        dims = tuple(int(x) for x in (rng.integers(20, 70, size=3) if nd == 3 else
                                      rng.integers(60, 300, size=2)))
        insts.append(rand_inst(rng, kind, dims, bool(j % 2), int(rng.integers(1, 200))))
    return insts


@pytest.mark.parametrize("prec", PRECS, ids=["fp32", "exact"])
def test_batch_graph_matches_oracle(prec):
    insts = _batch_items(13, seed=3)
    items = []
    for inst in insts:
        items.append(dict(kind=inst.kind, dims=inst.dims, periodic=inst.periodic,
                          sites=_t(inst.sites), w=_t(inst.w), t=_t(inst.t), v=_t(inst.v),
                          labels=torch.full(inst.dims[::-1], -1, dtype=torch.int32, device=DEV)))
    b = vt.Batch(items, precision=prec)
    for use_graph in (True, True, False):
        for it in items:
            it["labels"].fill_(-1)
        b.run(use_graph=use_graph)
        st = b.sync()
        assert st["dev_error"] == 0
        for inst, it in zip(insts, items):
            assert_same(it["labels"].cpu().numpy(), oracle.brute(inst), inst, "batch")


def test_batch_with_host_labels_matches_oracle():
    """Batch instances whose labels are page-locked host buffers: the batch
    maps them and the kernels store the labels straight into host memory,
    with and without the graph."""
    insts = _batch_items(7, seed=5)
    items = [dict(kind=i.kind, dims=i.dims, periodic=i.periodic, sites=_t(i.sites), w=_t(i.w),
                  t=_t(i.t), v=_t(i.v),
                  labels=torch.full(i.dims[::-1], -1, dtype=torch.int32).pin_memory())
             for i in insts]
    b = vt.Batch(items)
    for use_graph in (True, False):
        for it in items:
            it["labels"].fill_(-1)
        b.run(use_graph=use_graph)
        assert b.sync()["dev_error"] == 0
        for inst, it in zip(insts, items):
            assert not it["labels"].is_cuda
            assert_same(it["labels"].numpy(), oracle.brute(inst), inst, "batch, host labels")


def test_batch_compact_tiles_and_mixed_configurations():
    """A batch built with compact tiles, then autotuned (each instance may keep
    either tile configuration): twelve kernel classes, labels exact."""
    insts = _batch_items(9, seed=8)
    items = [dict(kind=i.kind, dims=i.dims, periodic=i.periodic, sites=_t(i.sites), w=_t(i.w),
                  t=_t(i.t), v=_t(i.v),
                  labels=torch.full(i.dims[::-1], -1, dtype=torch.int32, device=DEV)) for i in insts]
    b = vt.Batch(items, brick_cfg=1)
    for tune in (False, True):
        if tune:
            b.autotune()
        for it in items:
            it["labels"].fill_(-1)
        b.run()
        assert b.sync()["dev_error"] == 0
        for inst, it in zip(insts, items):
            assert_same(it["labels"].cpu().numpy(), oracle.brute(inst), inst, "compact batch")


def test_batch_autotune():
    insts = _batch_items(6, seed=4)
    items = [dict(kind=i.kind, dims=i.dims, periodic=i.periodic, sites=_t(i.sites), w=_t(i.w),
                  t=_t(i.t), v=_t(i.v),
                  labels=torch.empty(i.dims[::-1], dtype=torch.int32, device=DEV)) for i in insts]
    b = vt.Batch(items)
    b.autotune()
    b.run()
    b.sync()
    for inst, it in zip(insts, items):
        assert_same(it["labels"].cpu().numpy(), oracle.brute(inst), inst, "tuned batch")


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["voronoi", "laguerre", "jm"])
def test_host_buffers_match_device_path(kind):
    """vt_label_host: inputs from CPU memory, labels stored straight into
    page-locked CPU memory; identical to the device path and to the oracle."""
    import torch
    inst = synthetic.make_instance(kind, (72, 64, 40), 1500, seed=23, periodic=True)
    g = vt.Grid(inst.dims, periodic=True)
    args = dict(w=_t(inst.w), t=_t(inst.t), v=_t(inst.v))
    dev = g.label(kind, _t(inst.sites), **args).cpu().numpy()
    g.sync()
    cpu = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a))
    host = g.label_host(kind, cpu(inst.sites), w=cpu(inst.w), t=cpu(inst.t), v=cpu(inst.v))
    g.sync()
    assert host.is_pinned() and not host.is_cuda
    assert (host.numpy() == dev).all()
    flat = np.random.default_rng(5).integers(0, inst.n_voxels, size=2000)
    assert (host.numpy().ravel()[flat] == oracle.brute_points(inst, flat)).all()


@pytest.mark.gpu
@pytest.mark.parametrize("periodic", [False, True])
def test_jm_sites_reached_before_birth_are_pruned_labels_exact(periodic):
    """Late births and mixed speeds: many sites are reached by another site's
    growth before they are born (no cell, Section 3.3 remark); they are
    discarded beforehand and the labels still equal the brute force."""
    rng = np.random.default_rng(41 + int(periodic))
    inst = rand_inst(rng, "jm", (40, 36, 30), periodic, 1500)
    inst.t = rng.uniform(0.0, 60.0, 1500)
    inst.v = np.where(rng.random(1500) < 0.7, 1.0, rng.uniform(0.25, 3.0, 1500))
    inst.sites[1499] = inst.sites[3]          # a duplicate position, born later or earlier
    got, st = run_gpu(inst)
    assert st["pruned_sites"] > 100
    assert_same(got, oracle.brute(inst), inst, "pruned")
    exact, st2 = run_gpu(inst, vt.VT_EXACT)
    assert st2["pruned_sites"] == st["pruned_sites"]
    assert_same(exact, got, inst, "exact")


@pytest.mark.parametrize("kind", ["voronoi", "laguerre"])
def test_dense_clusters_long_lists_scored_in_chunks(kind):
    """Clusters of 400 sites within 5 voxels: tiles inside them list more than
    256 images even after the culling re-run's cull, so the re-run scores
    their lists in chunks (long_tiles > 0 on Voronoi; Laguerre's weights let
    the dominance test prune its lists below 256 here), carrying each voxel's
    two best keys and its label across chunks; the labels are the brute
    force's in both precisions, and duplicated sites (exact ties across
    chunks) go to the lower id."""
    dims = (96, 96, 64)
    for dup in (False, True):
        # 400 sites per cluster either way (200 doubled), so that a brick's
        # culled images still fit the re-run's staging area
        base = synthetic.matern_sites(dims, 8, 200.0 if dup else 400.0, 5.0, seed=31,
                                      periodic=True)
        sites = np.concatenate([base, base]) if dup else base
        inst = synthetic.make_instance(kind, dims, sites.shape[0], seed=31, periodic=True,
                                       sites=sites)
        want = oracle.brute(inst)
        for prec in PRECS:
            got, st = run_gpu(inst, prec)
            assert_same(got, want, inst, f"dense clusters, duplicates={dup}, precision={prec}")
            if kind == "voronoi":
                assert st["long_tiles"] > 0
