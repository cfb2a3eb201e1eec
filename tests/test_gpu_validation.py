"""The validation studies as tests (FP32, all runs of a study in one batch).

* Phoretic speed against mobility (Sec. "Results", the mobility dependence,
  Fig. 3B): a free Janus sphere in bulk fluid producing solute on its cap
  swims along its axis with a steady speed that is a straight line in the
  mobility mu = mu_+ = mu_- (R^2 > 0.99) and changes sign with it.  A small
  offset at mu = 0 is the solute's free-energy coupling; the line's slope is
  positive (v_s = mu (1 - n n).grad phi drives the fluid towards high solute,
  so the sphere moves away from its producing cap for mu > 0).
* Rest height of a neutral sphere at a flat interface against Young's
  construction z_c - z_int = -R cos(theta) (contact-angle relation of Sec.
  "Particles", theta through the oil): the sign follows cos(theta), 60 and
  120 degrees are mirror images, 90 degrees stays at the interface, and the
  magnitude lies within a band of Young's value (the diffuse interface of
  width 1.1 against a six-node sphere)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2202_01631_gb300 import build
    build.build()
    import torch
    torch.cuda.init()
    from paper_2202_01631_gb300 import lbdp, validation, workloads
    return lbdp, validation, workloads


def test_phoretic_speed_linear_in_mobility(mods):
    lbdp, V, W = mods
    args = V.parse(["phoretic", "--steps", "8000", "--every", "500"])
    s = V.phoretic(args, lbdp, W, verbose=False)
    speed = s["speed_along_m"]
    mus = sorted(speed)
    assert s["r2"] > 0.99
    assert s["line_slope"] > 0
    # sign change across mu = 0, and the ends of opposite sign
    assert speed[mus[0]] < 0 < speed[mus[-1]]
    # the offset at mu = 0 is small against the response at |mu| = 0.2
    assert abs(s["line_intercept"]) < 0.2 * abs(speed[mus[-1]] - speed[mus[0]])


def test_contact_angle_rest_height(mods):
    lbdp, V, W = mods
    args = V.parse(["contact", "--steps", "20000", "--every", "1000", "--edge", "64", "--R", "6"])
    s = V.contact(args, lbdp, W, verbose=False)
    h = s["rest_height"]
    R = 6.0
    assert abs(h[90.0]) < 0.1 * R
    assert h[60.0] < 0 < h[120.0]                      # -R cos(theta)
    assert abs(h[60.0] + h[120.0]) < 0.05 * R          # mirror images
    for th in (60.0, 120.0):
        young = -R * math.cos(math.radians(th))
        assert 0.7 < h[th] / young < 1.5, (th, h[th], young)
