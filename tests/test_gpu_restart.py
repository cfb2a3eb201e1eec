"""Checkpoint and restart, non-finite input, and cancelled served requests.

* lb_save_state / lb_load_state: a box saved after some steps and restored
  into a fresh box continues bit for bit as the saved box does (fields,
  populations, masks, particle state), with spheres that cover and uncover
  nodes and carry covering impulses across the checkpoint.
* lb_set_fields refuses NaN or Inf host input (LB_ERR_NONFINITE) and leaves
  the box as it was; a box whose own arithmetic overflows reports
  LB_ERR_NONFINITE from lb_conservation.  Both failures are made on the host
  side: the device only ever sees finite inputs, or runs to NaN in plain
  arithmetic, which faults nothing.
* lbs_cancel: a queued and a resident request cancelled between pumps end
  with LB_ERR_CANCELLED, their memory is reused, and every other request's
  result is the same as without the cancellations.
"""
import numpy as np
import pytest

from paper_2202_01631_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LB_ERR_PARAM, LB_ERR_NONFINITE, LB_ERR_CANCELLED = -1, -3, -8


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
    nz = shape[0]
    z = np.arange(nz)[:, None, None]
    return dict(rho=1.0 + 0.005 * rng.uniform(-1, 1, shape), u=0.005 * rng.uniform(-1, 1, (3,) + shape),
                psi=np.tanh((z - nz / 2 + 0.3) / 2.0) + 0.1 * rng.uniform(-1, 1, shape),
                phi=0.2 + 0.05 * rng.uniform(-1, 1, shape))


PARAMS = dict(W.BASE_PARAMS, nx=30, ny=26, nz=34, periodic=(1, 1, 0), E=0.3, phi_b=1.0, k_d=2e-3)
SPHERES = [dict(pos=(9.3, 12.7, 16.6), R=4.2, m_hat=(0.2, 0.4, -1.0), alpha=1e-2, mu_plus=0.1, mu_minus=-0.1,
                theta_c_deg=60.0, vel=(0.06, 0.02, 0.01), fixed=1),
           dict(pos=(22.4, 5.1, 17.9), R=3.6, m_hat=(1.0, 0.0, 0.3), alpha=5e-3, mu_plus=0.2, mu_minus=0.2,
                theta_c_deg=110.0, ext_force=(0.0, 0.01, 0.0))]


def _box(lbdp, precision):
    box = lbdp.Box(precision=precision, **PARAMS)
    box.set_fields(**_fields((34, 26, 30), 3))
    for d in SPHERES:
        box.add_particle(**d)
    return box


def _state(box):
    f = box.fields()
    return [f[k] for k in ("rho", "u", "psi", "phi")] + [box.populations(), box.mask()] + \
        [p[k] for p in box.particles() for k in sorted(p)] + [box.conservation()]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_restart_continues_bit_for_bit(lbdp, precision):
    a = _box(lbdp, precision)
    a.step(25)
    blob = a.save_state()
    a.step(20)
    b = lbdp.Box(precision=precision, **PARAMS)   # fresh, no particles
    b.load_state(blob)
    assert len(b.particles()) == 2
    b.step(20)
    changed = int(np.count_nonzero(b.mask() != _box(lbdp, precision).mask()))
    assert changed > 0                             # the driven sphere covered nodes
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_load_state_rejects_another_box(lbdp):
    a = _box(lbdp, "fp32")
    a.step(3)
    blob = a.save_state()
    for other in (dict(PARAMS, nx=31), dict(PARAMS, kappa=0.05)):
        b = lbdp.Box(precision="fp32", **other)
        with pytest.raises(lbdp.LbError) as e:
            b.load_state(blob)
        assert e.value.status == LB_ERR_PARAM
        b.close()
    c = lbdp.Box(precision="fp64", **PARAMS)
    with pytest.raises(lbdp.LbError):
        c.load_state(blob)
    c.close()
    a.close()


def test_nonfinite_host_field_is_refused(lbdp):
    box = _box(lbdp, "fp32")
    box.step(5)
    before = box.fields()
    bad = before["psi"].copy()
    bad[3, 4, 5] = np.nan
    with pytest.raises(lbdp.LbError) as e:
        box.set_fields(psi=bad)
    assert e.value.status == LB_ERR_NONFINITE
    bad = before["u"].copy()
    bad[1, 0, 0, 0] = np.inf
    with pytest.raises(lbdp.LbError) as e:
        box.set_fields(u=bad)
    assert e.value.status == LB_ERR_NONFINITE
    after = box.fields()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    box.close()


def test_overflowing_box_reports_nonfinite(lbdp):
    """Relaxation time at the stability limit, a strong body force and a
    perturbed start: the populations overflow within a few hundred steps (the
    FP64 oracle reaches 1e254 at step 350 on the same input)."""
    rng = np.random.default_rng(1)
    box = lbdp.Box(precision="fp32", **dict(W.BASE_PARAMS, nx=16, ny=16, nz=16, periodic=(1, 1, 1), tau=0.5001,
                                               body_force=(0.05, 0.0, 0.0), thermo_force=0))
    box.set_fields(rho=1 + 0.05 * rng.uniform(-1, 1, (16, 16, 16)), u=0.1 * rng.uniform(-1, 1, (3, 16, 16, 16)))
    box.step(400)
    with pytest.raises(lbdp.LbError) as e:
        box.conservation()
    assert e.value.status == LB_ERR_NONFINITE
    box.close()


def test_server_cancel_queued_and_resident(lbdp):
    specs = [dict(PARAMS, nx=24, ny=20, nz=28), dict(PARAMS, nx=20, ny=20, nz=20),
             dict(PARAMS, nx=26, ny=22, nz=24), dict(PARAMS, nx=22, ny=18, nz=30)]
    sphere = [dict(SPHERES[1], pos=(8.2, 9.1, 10.3), R=3.1)]
    probe = lbdp.Batch(precision="fp32", arena_bytes=1 << 28)
    sizes = [probe.box_bytes(**p) for p in specs]
    probe.close()
    arena = sizes[0] + sizes[1] + 4096            # two resident at a time

    def run(keep, cancel_plan):
        srv = lbdp.Server(precision="fp32", arena_bytes=arena, chunk_steps=4)
        try:
            ids, outs = {}, {}
            for j in keep:
                p = specs[j]
                shape = (p["nz"], p["ny"], p["nx"])
                f = _fields(shape, 40 + j)
                outs[j] = np.full(shape, -7.0)
                ids[j] = srv.submit(p, sphere, psi=f["psi"], phi=f["phi"], steps=24, arrival=0.0,
                                    out_psi=outs[j])
            res, rounds = {}, 0
            while len(res) < len(keep):
                srv.pump(now=float(rounds))
                if rounds == 0:
                    for j in cancel_plan:
                        srv.cancel(ids[j], now=0.5)
                    with pytest.raises(lbdp.LbError):
                        srv.cancel(10 ** 9)
                for r in srv.poll():
                    res[r["id"]] = r
                rounds += 1
                assert rounds < 100
            return {j: res[ids[j]] for j in keep}, outs
        finally:
            srv.close()

    # after the first pump requests 0 and 1 are resident, 2 and 3 queued
    got, outs = run([0, 1, 2, 3], cancel_plan=[1, 2])
    ref, ref_outs = run([0, 3], cancel_plan=[])
    for j in (1, 2):
        assert got[j]["status"] == LB_ERR_CANCELLED
        assert np.all(outs[j] == -7.0)             # nothing written for a cancelled request
    for j in (0, 3):
        assert got[j]["status"] == 0
        assert np.array_equal(outs[j], ref_outs[j])
        assert np.array_equal(got[j]["sums"], ref[j]["sums"])
