"""Device memory of one box (lb_device_bytes, host-only): the region holds,
per node, the double-buffered populations, psi and phi and masks, the
chemical potentials, the velocity, the force and the four stress fields near
particles, the boundary flag and the FP64 staging used for host transfers,
plus a per-box constant (particle records and per-block partials).  The
per-node figure is what the design notes quote for the 128^3 and 256^3
boxes."""
import pytest

from paper_2202_01631_gb300 import lbdp
from paper_2202_01631_gb300 import workloads as W

# bytes per node: pops 2 x 19 x s, psi/phi 2 x 2 x f, masks 2, mu 2 f, u 3 f,
# force 3 f, stress 4 f, flag 1, staging 6 x 8
PER_NODE = {"fp64": 2 * 19 * 8 + 4 * 8 + 2 + 2 * 8 + 3 * 8 + 3 * 8 + 4 * 8 + 1 + 48,
            "fp32": 2 * 19 * 4 + 4 * 4 + 2 + 2 * 4 + 3 * 4 + 3 * 4 + 4 * 4 + 1 + 48,
            "fp16": 2 * 19 * 2 + 4 * 4 + 2 + 2 * 4 + 3 * 4 + 3 * 4 + 4 * 4 + 1 + 48,
            "bf16": 2 * 19 * 2 + 4 * 4 + 2 + 2 * 4 + 3 * 4 + 3 * 4 + 4 * 4 + 1 + 48}


@pytest.mark.parametrize("precision", sorted(PER_NODE))
def test_device_bytes_per_node(precision):
    sizes = {}
    for n in (64, 128, 256):
        p = lbdp.box_params(precision, None, **dict(W.BASE_PARAMS, nx=n, ny=n, nz=n))
        sizes[n] = lbdp.lb_device_bytes(p)
    # the slope between two sizes is the per-node figure (256-byte padding of
    # each array aside), the intercept the per-box constant
    slope = (sizes[256] - sizes[128]) / (256 ** 3 - 128 ** 3)
    assert abs(slope - PER_NODE[precision]) < 1e-3
    const = sizes[64] - PER_NODE[precision] * 64 ** 3
    assert 0 < const < 4 << 20
    # the per-box part grows only with the number of reduction blocks
    assert abs(sizes[256] - (PER_NODE[precision] * 256 ** 3 + const)) < 1 << 16
