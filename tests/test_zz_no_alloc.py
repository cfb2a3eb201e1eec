"""lb_totals_noalloc: the conservation totals without any device allocation.

Callers whose device memory is owned by their own allocator (or that cannot
afford the synchronisation of cudaMalloc) get the FP64 totals of their own
device arrays from this entry point; its partial sums live in a fixed array
inside the library.  The test feeds it the state of a box and checks it
against lb_conservation on that same state, for two different states in a
row (so nothing left in the shared array from the first call can leak into
the second).  This file is collected last so that a stop-at-first-failure
run has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-12   # FP64 sums of ~3e4 node values in a different order


def _device_state(box, torch, dtype):
    f = box.populations()
    fl = box.fields()
    m = box.mask()
    dev = torch.device("cuda")
    return (torch.from_numpy(np.ascontiguousarray(f)).to(dev, dtype),
            torch.from_numpy(np.ascontiguousarray(fl["psi"])).to(dev, dtype),
            torch.from_numpy(np.ascontiguousarray(fl["phi"])).to(dev, dtype),
            torch.from_numpy(np.ascontiguousarray(m)).to(dev))


def _totals(lbdp, torch, box, prec, dtype):
    f, psi, phi, mask = _device_state(box, torch, dtype)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    p = box.params
    lbdp.lb_totals_noalloc(prec, p.nx, p.ny, p.nz, f.data_ptr(), psi.data_ptr(), phi.data_ptr(),
                           mask.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_totals_noalloc_match_lb_conservation():
    import torch
    from paper_2202_01631_gb300 import build, workloads as W
    build.build()
    from paper_2202_01631_gb300 import lbdp

    wl = W.plain_fp64(seed=2)
    box = lbdp.Box(precision="fp64", **wl.params)
    box.set_fields(**wl.fields)
    for p in wl.particles:
        box.add_particle(**p)
    box.step(30)
    ref1 = box.conservation()
    got1 = _totals(lbdp, torch, box, "fp64", torch.float64)

    # a second, different state right after: the shared array must not leak
    box.step(17)
    ref2 = box.conservation()
    got2 = _totals(lbdp, torch, box, "fp64", torch.float64)

    for got, ref in ((got1, ref1), (got2, ref2)):
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= REL * np.maximum(np.abs(ref), 1.0)), (got, ref)
    assert not np.allclose(ref1, ref2, rtol=0, atol=0)

    # FP32 inputs: the same totals within FP32 rounding of the inputs
    got32 = _totals(lbdp, torch, box, "fp32", torch.float32)
    assert np.all(np.abs(got32 - ref2) <= 1e-6 * np.maximum(np.abs(ref2), 1.0))


def test_totals_noalloc_rejects_oversized_box():
    import torch
    from paper_2202_01631_gb300 import lbdp
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbdp.LbError) as e:
        lbdp.lb_totals_noalloc("fp64", 300, 300, 300, t.data_ptr(), t.data_ptr(), t.data_ptr(), None,
                               t.data_ptr(), None)
    assert e.value.status == -1
