"""The lattice-Boltzmann transport of psi and phi (scalar_scheme = 1: D3Q7,
relaxation time 1, moving-wall bounce-back at particles) against the FP64 CPU
oracle, which stores and streams the D3Q7 distributions themselves; the CUDA
path evaluates the same update from the node fields without storing them.

Same bars as the finite-difference scheme: FP64 <= 1e-10 max-abs on every
field and the particle state, FP32 <= 1e-4 norm-relative; a box of the batch
gives the same bits as the box alone.
"""
import numpy as np
import pytest

from paper_2202_01631_gb300 import workloads as W
from tests.pair_util import compare, make_pair, norm_rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4
LB = dict(scalar_scheme=1)


@pytest.fixture(scope="module")
def lbdp():
    from paper_2202_01631_gb300 import build
    build.build()
    import torch
    torch.cuda.init()
    from paper_2202_01631_gb300 import lbdp as mod
    return mod


def _assert64(d, tol=TOL64):
    assert d["mask_mismatch"] == 0, d
    bad = {k: v for k, v in d.items() if k != "mask_mismatch" and v > tol}
    assert not bad, d


def _noisy_fields(shape, seed, psi_amp=0.3, phi_amp=0.1, u_amp=0.01):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = np.arange(nz)[:, None, None]
    return dict(rho=1.0 + 0.01 * rng.uniform(-1, 1, shape),
                u=u_amp * rng.uniform(-1, 1, (3,) + shape),
                psi=np.tanh((z - nz / 2 + 0.3) / 2.0) + psi_amp * rng.uniform(-1, 1, shape),
                phi=0.2 + phi_amp * rng.uniform(-1, 1, shape))


def test_rejects_unknown_scheme(lbdp):
    with pytest.raises(lbdp.LbError):
        lbdp.Box(precision="fp64", **dict(W.BASE_PARAMS, nx=8, ny=8, nz=8, scalar_scheme=2))


def test_lb_fluid_walls_ragged_fp64(lbdp):
    """Walls on two axes (bounce-back of the D3Q7 distributions), a ragged
    box, body force, solubility and sink."""
    params = dict(W.BASE_PARAMS, nx=37, ny=11, nz=14, periodic=(0, 1, 0), E=-0.2, k_d=1e-3,
                  body_force=(0.0, 3e-5, 1e-5), **LB)
    box, ref = make_pair(params, _noisy_fields((14, 11, 37), 2), [])
    box.step(60)
    ref.step(60)
    _assert64(compare(box, ref))


def test_lb_single_column_fp64(lbdp):
    """Degenerate 1x1xN box: every lateral neighbour is the node itself."""
    params = dict(W.BASE_PARAMS, nx=1, ny=1, nz=40, periodic=(1, 1, 0), M_psi=0.5, E=0.4, k_d=0.01, **LB)
    z = np.arange(40.0)
    box, ref = make_pair(params, dict(psi=np.tanh((z - 19.5) / 2.0)[:, None, None]), [])
    box.step(300)
    ref.step(300)
    _assert64(compare(box, ref))


def test_lb_plain_config_fp64_1000_steps(lbdp):
    """The FP64 bar on the plain 32^3 configuration with the LB transport."""
    wl = W.plain_fp64(seed=3)
    box, ref = make_pair(dict(wl.params, **LB), wl.fields, wl.particles)
    box.step(1000)
    ref.step(1000)
    _assert64(compare(box, ref, check_pops=False))
    assert ref.error() == 0


def test_lb_driven_sphere_covering_fp64(lbdp):
    """A sphere driven through a two-phase, solute-carrying fluid: moving-wall
    bounce-back of the distributions on every D3Q7 link into the surface,
    covering and uncovering every few steps; totals stay exact."""
    n = 24
    params = dict(W.BASE_PARAMS, nx=n, ny=n, nz=n, periodic=(1, 1, 1), E=0.3, M_psi=0.2, k_d=0.0, **LB)
    fields = _noisy_fields((n, n, n), 5, psi_amp=0.1)
    part = dict(pos=(6.31, 11.77, 12.13), R=4.2, vel=(0.09, 0.02, -0.03), omega=(0.0, 0.0, 0.01),
                fixed=1, m_hat=(0.3, 0.1, 1.0), mu_plus=0.1, mu_minus=0.2, theta_c_deg=70.0, alpha=0.0)
    box, ref = make_pair(params, fields, [part])
    m0 = ref.mask().copy()
    s0 = ref.conservation()
    box.step(60)
    ref.step(60)
    assert np.sum(ref.mask() != m0) > 20
    _assert64(compare(box, ref))
    sg = box.conservation()
    assert abs(sg[1] - s0[1]) < 1e-9 and abs(sg[2] - s0[2]) < 1e-9


def test_lb_free_spheres_across_periodic_wrap_fp64(lbdp):
    """Two free Janus spheres (activity, slip, wetting, external loads), one
    crossing the periodic x boundary, walls in z."""
    n = 28
    params = dict(W.BASE_PARAMS, nx=n, ny=n - 4, nz=n, periodic=(1, 1, 0), k_d=1e-3, **LB)
    fields = W.flat_interface_fields(n, n - 4, n, z0=14.0)
    parts = [dict(pos=(0.6, 10.3, 14.2), R=3.7, m_hat=(1.0, 0.5, -0.2), alpha=1e-2, mu_plus=0.3,
                  mu_minus=0.5, theta_c_deg=110.0, ext_force=(-0.06, 0.0, 0.0), ext_torque=(0, 0, 0.1)),
             dict(pos=(14.4, 11.9, 13.6), R=3.3, m_hat=(0.0, -1.0, 0.3), alpha=1e-2, mu_plus=-0.2,
                  mu_minus=0.1, theta_c_deg=60.0, vel=(0.0, 0.01, 0.0))]
    box, ref = make_pair(params, fields, parts)
    box.step(120)
    ref.step(120)
    _assert64(compare(box, ref))
    assert ref.error() == 0


def test_lb_plain_config_fp32(lbdp):
    wl = W.plain_fp64(seed=0)
    box, ref = make_pair(dict(wl.params, **LB), wl.fields, wl.particles, precision="fp32")
    box.step(wl.steps)
    ref.step(wl.steps)
    mg = ref.mask()
    assert np.array_equal(box.mask(), mg)
    fg, fr = box.fields(), ref.fields()
    for k in ("u", "psi", "phi", "rho"):
        assert norm_rel(fg[k], fr[k], mg) < TOL32, k
    pg, pr = box.particles()[0], ref.particles()[0]
    assert np.max(np.abs(pg["pos"] - pr["pos"])) / 4.0 < TOL32


def test_lb_full_size_interface_fp32_100_steps(lbdp):
    """The 128^3 interface workload with the LB transport, 100 steps: every
    field, velocity included, within 1e-4 of its maximum over the whole box."""
    wl = W.interface(theta_c_deg=60.0, solubility_ratio=2.0, mobility=0.1)
    box, ref = make_pair(dict(wl.params, **LB), wl.fields, wl.particles, precision="fp32")
    box.step(100)
    ref.step(100)
    mg = ref.mask()
    assert np.array_equal(box.mask(), mg)
    fg, fr = box.fields(), ref.fields()
    for k in ("u", "psi", "phi", "rho"):
        assert norm_rel(fg[k], fr[k], mg) < TOL32, k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lb_box_in_batch_same_bits(lbdp, precision):
    """An LB box and a finite-difference box share a batch; each gives the
    bits it gives alone."""
    specs = [dict(W.BASE_PARAMS, nx=24, ny=20, nz=28, periodic=(1, 1, 0), E=0.3, phi_b=1.0, k_d=2e-3, **LB),
             dict(W.BASE_PARAMS, nx=33, ny=17, nz=21, periodic=(1, 1, 1), E=-0.2, k_d=1e-3)]
    part = dict(pos=(11.3, 9.7, 13.6), R=4.5, m_hat=(0.2, 0.4, -1.0), alpha=1e-2, mu_plus=0.1,
                mu_minus=-0.1, theta_c_deg=60.0, vel=(0.05, 0.0, 0.01), fixed=1)

    def setup(b, k):
        p = specs[k]
        b.set_fields(**_noisy_fields((p["nz"], p["ny"], p["nx"]), 40 + k))
        if k == 0:
            b.add_particle(**part)

    batch = lbdp.Batch(precision=precision, arena_bytes=1 << 30, graph_steps=4)
    try:
        members = []
        for k, p in enumerate(specs):
            b = batch.add_box(**p)
            setup(b, k)
            batch.set_steps(b, 9)
            members.append(b)
        batch.run(9)
        batch.sync()
        for k, b in enumerate(members):
            alone = lbdp.Box(precision=precision, **specs[k])
            setup(alone, k)
            alone.step(9)
            fa, fb = alone.fields(), b.fields()
            for key in ("rho", "u", "psi", "phi"):
                assert np.array_equal(fa[key], fb[key]), key
            assert np.array_equal(alone.conservation(), b.conservation())
            for pa, pb in zip(alone.particles(), b.particles()):
                for key in pa:
                    assert np.array_equal(pa[key], pb[key]), key
            alone.close()
    finally:
        batch.close()
