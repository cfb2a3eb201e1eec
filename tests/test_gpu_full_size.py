"""The benchmark's own workload at full size against the oracle.

The default benchmark times the 256^3 box with eight spheres of R = 6 below a
flat interface at z = 128 (the precision configuration), FP32, with the z
chunk lengths its autotuner picks.  Here the same box, tuned the same way,
runs 20 steps on the GPU and the FP64 oracle runs the same 20 steps on every
host core (about half a minute): every fluid node and every particle is
compared, not a sample.  FP32 holds the 1e-4 norm-relative bar on u, psi,
phi and rho and on the trajectory; the FP16-storage arm of the benchmark is
held to the band its 16-bit deviation storage reaches (its error is reported
in the assertion message).
"""
import numpy as np
import pytest

from paper_2202_01631_gb300 import workloads as W
from tests.pair_util import norm_rel

pytestmark = pytest.mark.gpu

STEPS = 20
TOL32 = 1e-4


@pytest.fixture(scope="module")
def lbdp():
    from paper_2202_01631_gb300 import build
    build.build()
    import torch
    torch.cuda.init()
    from paper_2202_01631_gb300 import lbdp as mod
    return mod


@pytest.fixture(scope="module")
def reference():
    """The oracle's state after STEPS steps of the 256^3 workload."""
    from oracle import lbref
    wl = W.precision(seed=0, edge=256)
    lbref.set_threads(0)
    ref = lbref.Oracle(dict(wl.params))
    ref.set_fields(**wl.fields)
    for p in wl.particles:
        ref.add_particle(**p)
    ref.step(STEPS)
    out = dict(fields=ref.fields(), mask=ref.mask(), particles=ref.particles())
    del ref
    return wl, out


def _run(lbdp, wl, precision):
    box = lbdp.Box(precision=precision, **wl.params)
    box.set_fields(**wl.fields)
    for p in wl.particles:
        box.add_particle(**p)
    planes, _ = box.tune(reps=2)   # the launch configuration the benchmark times
    box.step(STEPS)
    out = dict(fields=box.fields(), mask=box.mask(), particles=box.particles(), planes=planes)
    box.close()
    return out


def test_benchmark_workload_fp32_matches_oracle(lbdp, reference):
    wl, ref = reference
    got = _run(lbdp, wl, "fp32")
    mr = ref["mask"]
    assert np.array_equal(got["mask"], mr)
    errs = {k: norm_rel(got["fields"][k], ref["fields"][k], mr) for k in ("u", "psi", "phi", "rho")}
    # the flow is well above FP32 rounding: the tanh profile relaxes towards
    # its equilibrium width and drives it
    assert float(np.max(np.abs(ref["fields"]["u"]))) > 1e-5
    for k, e in errs.items():
        assert e < TOL32, (k, errs, got["planes"])
    R = wl.particles[0]["R"]
    for pg, pr in zip(got["particles"], ref["particles"]):
        assert np.max(np.abs(pg["pos"] - pr["pos"])) / R < TOL32
        assert np.max(np.abs(pg["m_hat"] - pr["m_hat"])) < TOL32


def test_benchmark_workload_fp16_storage_band(lbdp, reference):
    wl, ref = reference
    got = _run(lbdp, wl, "fp16")
    mr = ref["mask"]
    assert np.array_equal(got["mask"], mr)
    errs = {k: norm_rel(got["fields"][k], ref["fields"][k], mr) for k in ("u", "psi", "phi", "rho")}
    assert errs["u"] < 1e-2, errs
    for k in ("psi", "phi", "rho"):
        assert errs[k] < 5e-3, (k, errs)
