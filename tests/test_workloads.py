"""The seeded synthetic workloads keep the geometric promises the runs rely
on: spheres inside their boxes, clear of the walls by a quarter of the box
(an active sphere can leave the interface and swim a few radii within a run),
and apart from each other; mobility within the paper's range."""
import numpy as np

from paper_2202_01631_gb300 import workloads as W


def _check_box(wl):
    p = wl.params
    L = p["nz"]
    assert p["periodic"] == (1, 1, 0)
    for d in wl.particles:
        z, R = d["pos"][2], d["R"]
        assert z - R >= L / 4.0 - 1e-12 and z + R <= L - L / 4.0 + 1e-12
        assert abs(d["mu_plus"]) <= 0.1 and abs(d["mu_minus"]) <= 0.1
        assert abs(np.linalg.norm(d["m_hat"]) - 1.0) < 1e-12
    for i, a in enumerate(wl.particles):
        for b in wl.particles[i + 1:]:
            dv = np.array(a["pos"]) - np.array(b["pos"])
            dv[:2] -= L * np.round(dv[:2] / L)
            assert np.linalg.norm(dv) >= a["R"] + b["R"] + 4.0 - 1e-12


def test_batched_boxes():
    """Periodic boxes (no wall to swim into) with the drawn ranges of the
    batched form; the psi slab has its two interfaces where stated."""
    wls = W.batched(seed=0, n_boxes=64)
    assert len(wls) == 64
    for wl in wls:
        L = wl.params["nx"]
        assert 32 <= L <= 96 and len(wl.particles) == 1
        assert wl.params["periodic"] == (1, 1, 1)
        d = wl.particles[0]
        assert 4.0 <= d["R"] <= 8.0 and abs(d["mu_plus"]) <= 0.2 and 45.0 <= d["theta_c_deg"] <= 135.0
        assert 2.0 * d["R"] + 4.0 <= L   # the sphere and its periodic image stay apart
        psi = wl.fields["psi"][:, 0, 0]
        assert abs(psi[0] + 1) < 1e-2 and abs(psi[L // 2] - 1) < 1e-2
        crossings = np.nonzero(np.diff((psi > 0).astype(int)))[0]
        assert len(crossings) == 2
        assert abs(crossings[0] + 0.5 - L / 4.0) <= 1.0 and abs(crossings[1] + 0.5 - 3 * L / 4.0) <= 1.0


def test_serving_requests():
    reqs = W.serving_requests(seed=0, n=32)
    times = [t for t, _ in reqs]
    assert times == sorted(times) and len(reqs) == 32
    for _, wl in reqs:
        L = wl.params["nx"]
        assert 24 <= L <= 128 and 1 <= len(wl.particles) <= 4
        assert 500 <= wl.steps <= 20000
        for d in wl.particles:
            assert d["R"] <= min(8.0, L / 8.0) + 1e-12
        _check_box(wl)
