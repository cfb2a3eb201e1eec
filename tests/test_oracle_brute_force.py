"""Brute force on 8^3 boxes: the oracle against an independent NumPy
transcription of the whole step (tests/brute_step.py, which imports nothing
from the oracle), 10 steps, every field, the populations, the solid mask and
the particle state to 1e-13.

Two boxes with walls in z: a sphere of radius 2 driven through the lattice at
a fixed velocity (covering and uncovering every few steps, Janus production,
wetting, slip, solubility coupling), and a free wetting Janus sphere pushed
by an external force (the implicit velocity solve and the rotation).  A
dropped term, a wrong sign or a transposed index anywhere in the oracle's
step shows up as an O(1e-3) difference after a few steps.
"""
import math

import numpy as np
import pytest

from oracle.lbref import Oracle
from tests.brute_step import BruteBox, Sphere, wetting_h_from_angle

TOL = 1e-13


def _initial(shape, seed):
    rng = np.random.default_rng(seed)
    nz = shape[0]
    z = np.arange(nz)[:, None, None]
    return dict(rho=1.0 + 0.01 * rng.uniform(-1, 1, shape),
                u=0.01 * rng.uniform(-1, 1, (3,) + shape),
                psi=np.tanh((z - 3.7) / 1.6) + 0.05 * rng.uniform(-1, 1, shape),
                phi=0.3 + 0.1 * rng.uniform(-1, 1, shape))


PRM = dict(tau=0.9, rho0=1.0, body_force=(1e-5, -2e-5, 0.0), A=0.0625, kappa=0.04, M_psi=0.1, C=0.0625,
           M_phi=0.8, E=0.35, phi_b=0.8, k_d=3e-3)

CASES = {
    "driven": dict(pos=(3.3, 3.6, 3.9), R=2.0, m_hat=(0.3, -0.5, 0.8), alpha=2e-2, mu_plus=0.15,
                   mu_minus=-0.1, theta_c_deg=65.0, vel=(0.11, 0.07, 0.02), omega=(0.0, 0.03, 0.01), fixed=1),
    "free": dict(pos=(4.2, 3.1, 4.1), R=2.0, m_hat=(-0.6, 0.2, 0.5), alpha=1e-2, mu_plus=0.3, mu_minus=0.05,
                 theta_c_deg=120.0, ext_force=(0.04, -0.03, 0.01), ext_torque=(0.0, 0.02, -0.01), rho_p=0.6),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_ten_steps_match_independent_transcription(case):
    nx = ny = 8
    nz = 8
    shape = (nz, ny, nx)
    periodic = (1, 1, 0)
    init = _initial(shape, 7 if case == "driven" else 8)
    d = CASES[case]
    H = wetting_h_from_angle(d["theta_c_deg"]) * math.sqrt(PRM["kappa"] * PRM["A"])

    o = Oracle(dict(PRM, nx=nx, ny=ny, nz=nz, periodic=periodic))
    o.set_fields(**init)
    o.add_particle(**{k: v for k, v in d.items() if k != "theta_c_deg"}, H=H)

    b = BruteBox(nx, ny, nz, periodic, **PRM)
    b.set_fields(**init)
    b.add_sphere(Sphere(d["pos"], d["R"], d["m_hat"], rho_p=d.get("rho_p", 1.0), alpha=d["alpha"],
                        mu_plus=d["mu_plus"], mu_minus=d["mu_minus"], H=H, vel=d.get("vel", (0, 0, 0)),
                        omega=d.get("omega", (0, 0, 0)), ext_force=d.get("ext_force", (0, 0, 0)),
                        ext_torque=d.get("ext_torque", (0, 0, 0)), fixed=d.get("fixed", 0)))
    changes = 0
    for _ in range(10):
        before = b.mask.copy()
        o.step(1)
        b.step()
        changes += int(np.count_nonzero(before != b.mask))
        assert np.array_equal(o.mask().reshape(-1), b.mask)
        f = o.fields()
        assert np.max(np.abs(f["rho"].reshape(-1) - b.f.sum(axis=0))) < TOL
        assert np.max(np.abs(f["u"].reshape(3, -1) - b.u)) < TOL
        assert np.max(np.abs(f["psi"].reshape(-1) - b.psi)) < TOL
        assert np.max(np.abs(f["phi"].reshape(-1) - b.phi)) < TOL
        assert np.max(np.abs(o.populations().reshape(19, -1) - b.f)) < TOL
        p = o.particles()[0]
        sp = b.spheres[0]
        for got, want in ((p["pos"], sp.X), (p["vel"], sp.V[:3]), (p["omega"], sp.V[3:]), (p["m_hat"], sp.m),
                          (p["force"], sp.force), (p["torque"], sp.torque)):
            assert np.max(np.abs(got - want)) < TOL, (got, want)
    if case == "driven":
        assert changes >= 6
    else:
        assert np.linalg.norm(b.spheres[0].V[:3]) > 1e-3
