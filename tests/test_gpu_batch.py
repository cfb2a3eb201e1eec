"""Batched and served boxes (include/lbdp_batch.h) against the same boxes run
alone.

Every box of a batch runs the arithmetic of the single-box path node by node,
with the same per-particle block split of the link and cover sums, so its
result must be bit-identical to the box run alone with lb_step -- in every
precision mode, whatever else shares the batch, however many steps each box
has left, whatever launch shape the autotuner picked, and through CUDA-graph
and plain launches alike.  The single-box path itself is held to the CPU
oracle by test_gpu_parity.py; one batched FP64 box is also compared with the
oracle directly here.
"""
import numpy as np
import pytest

from paper_2202_01631_gb300 import workloads as W
from tests.pair_util import compare, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbdp():
    from paper_2202_01631_gb300 import build
    build.build()
    import torch
    torch.cuda.init()
    from paper_2202_01631_gb300 import lbdp as mod
    return mod


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = np.arange(nz)[:, None, None]
    return dict(rho=1.0 + 0.005 * rng.uniform(-1, 1, shape), u=0.005 * rng.uniform(-1, 1, (3,) + shape),
                psi=np.tanh((z - nz / 2 + 0.3) / 2.0) + 0.1 * rng.uniform(-1, 1, shape),
                phi=0.2 + 0.05 * rng.uniform(-1, 1, shape))


def _specs():
    """Uneven boxes: walls and periodic axes, 0 to 2 spheres, some driven
    through nodes (covering and uncovering), one across a periodic wrap."""
    return [
        dict(params=dict(W.BASE_PARAMS, nx=24, ny=20, nz=28, periodic=(1, 1, 0), E=0.3, phi_b=1.0, k_d=2e-3),
             particles=[dict(pos=(11.3, 9.7, 13.6), R=4.5, m_hat=(0.2, 0.4, -1.0), alpha=1e-2, mu_plus=0.1,
                             mu_minus=-0.1, theta_c_deg=60.0, vel=(0.05, 0.0, 0.01), fixed=1)]),
        dict(params=dict(W.BASE_PARAMS, nx=33, ny=17, nz=21, periodic=(1, 1, 1), E=-0.2, k_d=1e-3,
                         body_force=(1e-5, 0.0, -1e-5)),
             particles=[]),
        dict(params=dict(W.BASE_PARAMS, nx=40, ny=36, nz=30, periodic=(1, 1, 0), k_d=1e-3),
             particles=[dict(pos=(10.2, 12.6, 14.9), R=4.1, m_hat=(1.0, 0.0, 0.3), alpha=1e-2, mu_plus=0.2,
                             mu_minus=0.2, theta_c_deg=120.0),
                        dict(pos=(27.4, 22.3, 15.3), R=3.6, m_hat=(0.0, 1.0, -0.5), alpha=5e-3, mu_plus=-0.1,
                             mu_minus=0.3, theta_c_deg=80.0, ext_force=(0.0, 0.0, 0.02))]),
        dict(params=dict(W.BASE_PARAMS, nx=21, ny=23, nz=26, periodic=(1, 1, 1), E=0.1, phi_b=0.5),
             particles=[dict(pos=(0.4, 11.2, 12.7), R=3.9, m_hat=(-1.0, 0.2, 0.1), alpha=1e-2, mu_plus=0.3,
                             mu_minus=0.0, theta_c_deg=100.0, vel=(-0.07, 0.02, 0.0), fixed=1)]),
    ]


def _setup(box, spec, k):
    p = spec["params"]
    box.set_fields(**_fields((p["nz"], p["ny"], p["nx"]), 100 + k))
    for d in spec["particles"]:
        box.add_particle(**d)


def _alone(lbdp, spec, k, precision, steps):
    box = lbdp.Box(precision=precision, **spec["params"])
    _setup(box, spec, k)
    box.step(steps)
    return box


def _assert_same(a, b):
    fa, fb = a.fields(), b.fields()
    for key in ("rho", "u", "psi", "phi"):
        assert np.array_equal(fa[key], fb[key]), key
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.mask(), b.mask())
    for pa, pb in zip(a.particles(), b.particles()):
        for key in pa:
            assert np.array_equal(pa[key], pb[key]), key
    assert np.array_equal(a.conservation(), b.conservation())


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_batch_matches_alone(lbdp, precision):
    specs = _specs()
    steps = [10, 7, 10, 3]
    batch = lbdp.Batch(precision=precision, arena_bytes=1 << 30, graph_steps=4)
    try:
        members = []
        for k, spec in enumerate(specs):
            b = batch.add_box(**spec["params"])
            _setup(b, spec, k)
            batch.set_steps(b, steps[k])
            members.append(b)
        launches = batch.run(100)          # stops when every box is done: 2 graphs + 2 plain steps
        assert launches == 10 * 10         # 9 per launch plan + the count-down, per step
        batch.sync()
        for k, b in enumerate(members):
            assert batch.steps_left(b) == 0
            _assert_same(b, _alone(lbdp, specs[k], k, precision, steps[k]))
    finally:
        batch.close()


def test_batch_autotuned_launch_shapes(lbdp):
    """Every candidate shape (z chunk of the fused and transport kernels), and
    the tuner's pick, give the same bits; the tuning runs leave the state
    unchanged."""
    specs = _specs()
    ref = [_alone(lbdp, s, k, "fp32", 6) for k, s in enumerate(specs)]
    assert lbdp.lbb_num_configs() == 3
    assert [lbdp.lbb_config_shape(k) for k in range(3)] == [(256, 8), (256, 16), (256, 32)]
    for cfg in [[0, 0], [2, 1], [1, 2], None]:
        batch = lbdp.Batch(precision="fp32", arena_bytes=1 << 30, graph_steps=3)
        try:
            members = []
            for k, spec in enumerate(specs):
                b = batch.add_box(**spec["params"])
                _setup(b, spec, k)
                batch.set_steps(b, 6)
                members.append(b)
            with pytest.raises(lbdp.LbError):
                batch.set_config([3, 0])   # no such candidate
            if cfg is None:
                got, ms = batch.tune(reps=3)
                assert all(0 <= c < lbdp.lbb_num_configs() for c in got) and all(m > 0 for m in ms)
            else:
                batch.set_config(cfg)
            batch.run(6)
            for k, b in enumerate(members):
                _assert_same(b, ref[k])
        finally:
            batch.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_single_box_chunk_lengths_and_tuner(lbdp, precision):
    """A single box gives the same bits with every z chunk length of its two
    bulk kernels (one plane up to the whole box, ragged last chunks included)
    and after lb_tune in mid-run; the tuner's timing launches leave the state
    unchanged."""
    spec = _specs()[2]
    ref = _alone(lbdp, spec, 2, precision, 8)
    nz = spec["params"]["nz"]
    for planes in [(1, 1), (7, 4), (4, 7), (16, 30), (nz, 9), (0, 0)]:
        box = lbdp.Box(precision=precision, **spec["params"])
        _setup(box, spec, 2)
        box.set_planes(*planes)
        got = box.planes()
        for want, k in zip(planes, ("k_fused", "k_scalars")):
            if want:
                assert got[k] * -(-nz // got[k]) >= nz and got[k] <= want
        box.step(8)
        _assert_same(box, ref)
    box = lbdp.Box(precision=precision, **spec["params"])
    _setup(box, spec, 2)
    with pytest.raises(lbdp.LbError):
        box.set_planes(-1, 0)
    box.step(3)
    planes, ms = box.tune(reps=2)
    assert box.planes() == planes and all(1 <= v <= nz for v in planes.values())
    assert all(m > 0 for m in ms.values())
    box.step(5)
    _assert_same(box, ref)


@pytest.mark.parametrize("shape", [(1, 1, 40), (33, 17, 3), (40, 5, 2)])
def test_tuner_on_thin_boxes(lbdp, shape):
    """The chunk tuner and explicit chunk lengths on boxes thinner than a
    column tile or a chunk (one node wide, three planes, two planes): every
    choice stays within the box and gives the bits of the heuristic."""
    nx, ny, nz = shape
    params = dict(W.BASE_PARAMS, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), E=0.2, k_d=1e-3,
                  body_force=(1e-5, 0.0, 0.0))

    def run(planes):
        box = lbdp.Box(precision="fp32", **params)
        box.set_fields(**_fields((nz, ny, nx), 7))
        if planes == "tune":
            got, ms = box.tune(reps=2)
            assert all(1 <= v <= nz for v in got.values()) and all(m > 0 for m in ms.values())
        elif planes is not None:
            box.set_planes(*planes)
            assert all(1 <= v <= nz for v in box.planes().values())
        box.step(12)
        return box

    ref = run(None)
    for planes in ("tune", (1, 1), (64, 64), (2, 5)):
        _assert_same(run(planes), ref)


def test_single_box_graph_runs_match_plain_steps(lbdp):
    """lb_step runs whole groups of steps of a box without particles as
    captured CUDA graphs and the rest as plain launches: one step at a time, in
    graph-sized runs, and across a change of the launch grids (which makes it
    capture again) or an added particle between runs (after which it launches
    plainly), the bits are the same."""
    spec = _specs()[1]
    extra = dict(pos=(16.2, 8.1, 10.3), R=2.6, m_hat=(0.0, 0.0, 1.0), alpha=0.0, mu_plus=0.0, mu_minus=0.0,
                 theta_c_deg=90.0)

    def run(chunks):
        box = lbdp.Box(precision="fp32", **spec["params"])
        _setup(box, spec, 1)
        for c in chunks:
            if c == "planes":
                box.set_planes(5, 3)
            elif c == "particle":
                box.add_particle(**extra)
            else:
                box.step(c)
        return box

    one = run([1] * 9 + ["planes"] + [1] * 16 + ["particle"] + [1] * 17)
    graphs = run([9, "planes", 16, "particle", 17])
    _assert_same(graphs, one)


def test_batch_members_leave_and_join(lbdp):
    """A box removed mid-run returns its memory; a new box joins the running
    batch; the others continue undisturbed."""
    specs = _specs()
    batch = lbdp.Batch(precision="fp32", arena_bytes=1 << 30, graph_steps=2)
    try:
        m0 = batch.add_box(**specs[0]["params"])
        _setup(m0, specs[0], 0)
        m1 = batch.add_box(**specs[1]["params"])
        _setup(m1, specs[1], 1)
        batch.set_steps(m0, 9)
        batch.set_steps(m1, 9)
        batch.run(4)
        used_before = batch.memory()[1]
        m1.close()
        assert batch.memory()[1] < used_before
        m2 = batch.add_box(**specs[2]["params"])
        _setup(m2, specs[2], 2)
        batch.set_steps(m2, 5)
        batch.run(5)
        _assert_same(m0, _alone(lbdp, specs[0], 0, "fp32", 9))
        _assert_same(m2, _alone(lbdp, specs[2], 2, "fp32", 5))
    finally:
        batch.close()


def test_batch_fp64_box_vs_oracle(lbdp):
    """The batched path against the CPU oracle directly (FP64, <= 1e-10)."""
    wl = W.plain_fp64(seed=2, edge=24)
    _, ref = make_pair(wl.params, wl.fields, wl.particles)
    batch = lbdp.Batch(precision="fp64", arena_bytes=1 << 30, graph_steps=8)
    try:
        b = batch.add_box(**wl.params)
        b.set_fields(**wl.fields)
        for d in wl.particles:
            b.add_particle(**d)
        other = batch.add_box(**_specs()[1]["params"])   # a neighbour in the batch
        _setup(other, _specs()[1], 1)
        batch.set_steps(b, 60)
        batch.set_steps(other, 60)
        batch.run(60)
        ref.step(60)
        d = compare(b, ref)
        assert d["mask_mismatch"] == 0, d
        assert max(v for k, v in d.items() if k != "mask_mismatch") <= 1e-10, d
    finally:
        batch.close()


def test_server_results_same_alone_and_in_the_mix(lbdp):
    """Continuous batching: requests of different sizes and lengths arrive
    while others run; the arena holds only some of them at once, so later
    ones wait and are admitted as memory frees up.  Each result (final psi,
    phi, particle state, totals) equals the same request run alone."""
    specs = _specs()
    steps = [12, 30, 9, 17, 5]
    order = [0, 2, 1, 3, 0]
    probe = lbdp.Batch(precision="fp32", arena_bytes=1 << 28)
    sizes = [probe.box_bytes(**specs[i]["params"]) for i in order]
    probe.close()
    arena = sizes[1] + sizes[2] + 4096         # room for about two of the larger boxes
    srv = lbdp.Server(precision="fp32", arena_bytes=arena, chunk_steps=8)
    try:
        outs = {}
        ids = []
        for j, i in enumerate(order):
            p = specs[i]["params"]
            shape = (p["nz"], p["ny"], p["nx"])
            f = _fields(shape, 100 + i)
            outs[j] = (np.empty(shape), np.empty(shape))
            ids.append(srv.submit(p, specs[i]["particles"], psi=f["psi"], phi=f["phi"], steps=steps[j],
                                  arrival=0.01 * j, out_psi=outs[j][0], out_phi=outs[j][1]))
        results, rounds, max_queued = {}, 0, 0
        while len(results) < len(order):
            active, queued = srv.pump(now=1.0 + rounds)
            max_queued = max(max_queued, queued)
            for r in srv.poll():
                results[r["id"]] = r
            rounds += 1
            assert rounds < 200
        assert max_queued > 0                   # the arena really limited admission
        for j, i in enumerate(order):
            r = results[ids[j]]
            assert r["status"] == 0
            assert r["arrival"] <= r["admitted"] <= r["done"]
            p = specs[i]["params"]
            alone = lbdp.Box(precision="fp32", **p)
            f = _fields((p["nz"], p["ny"], p["nx"]), 100 + i)
            alone.set_fields(psi=f["psi"], phi=f["phi"])
            for d in specs[i]["particles"]:
                alone.add_particle(**d)
            alone.step(steps[j])
            fa = alone.fields()
            assert np.array_equal(outs[j][0], fa["psi"])
            assert np.array_equal(outs[j][1], fa["phi"])
            assert np.array_equal(r["sums"], alone.conservation())
            for pa, pb in zip(r["particles"], alone.particles()):
                for key in pa:
                    assert np.array_equal(pa[key], pb[key]), key
            alone.close()
    finally:
        srv.close()
