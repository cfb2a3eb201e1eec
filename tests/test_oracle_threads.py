"""The oracle's node loops run on several host cores (OpenMP) with results
bit-identical to one thread: every sum over nodes is taken in node order by
one thread.  Checked on a box with walls, two spheres (one driven through the
lattice, so nodes are covered and uncovered) and both transport schemes."""
import numpy as np
import pytest

from oracle import lbref
from paper_2202_01631_gb300 import workloads as W


def _run(threads, scheme, steps=12):
    lbref.set_threads(threads)
    rng = np.random.default_rng(5)
    nx, ny, nz = 22, 20, 26
    shape = (nz, ny, nx)
    o = lbref.Oracle(dict(W.BASE_PARAMS, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), E=0.3, phi_b=1.0,
                          k_d=2e-3, scalar_scheme=scheme))
    z = np.arange(nz)[:, None, None]
    o.set_fields(rho=1 + 0.005 * rng.uniform(-1, 1, shape), u=0.005 * rng.uniform(-1, 1, (3,) + shape),
                 psi=np.tanh((z - 12.3) / 2) + 0.1 * rng.uniform(-1, 1, shape),
                 phi=0.2 + 0.05 * rng.uniform(-1, 1, shape))
    o.add_particle(pos=(10.3, 9.7, 12.6), R=4.2, m_hat=(0.2, 0.4, -1.0), alpha=1e-2, mu_plus=0.1,
                   mu_minus=-0.1, theta_c_deg=60.0, vel=(0.09, 0.0, 0.03), fixed=1)
    o.add_particle(pos=(2.3, 17.1, 13.9), R=3.2, m_hat=(1, 0, 0), alpha=1e-2, mu_plus=0.2, theta_c_deg=110.0)
    o.step(steps)
    f = o.fields()
    parts = np.concatenate([np.concatenate(list(q.values())) for q in o.particles()])
    return [f[k] for k in ("rho", "u", "psi", "phi")] + [o.populations(), parts, o.mask()]


@pytest.mark.parametrize("scheme", [0, 1])
def test_thread_count_gives_identical_bits(scheme):
    try:
        one = _run(1, scheme)
        many = _run(4, scheme)
    finally:
        lbref.set_threads(0)
    for a, b in zip(one, many):
        assert np.array_equal(a, b)
