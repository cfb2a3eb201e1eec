"""Run the same seeded input through the CUDA library and the CPU oracle."""
import numpy as np

from oracle.lbref import Oracle

FIELDS = ("rho", "u", "psi", "phi")
PSTATE = ("pos", "vel", "omega", "m_hat", "force", "torque")


def oracle_params(params):
    """The oracle maps solubility_ratio to E itself."""
    return dict(params)


def make_pair(params, fields, particles, precision="fp64"):
    from paper_2202_01631_gb300.lbdp import Box
    box = Box(precision=precision, **params)
    ref = Oracle(oracle_params(params))
    if fields:
        box.set_fields(**fields)
        ref.set_fields(**fields)
    for p in particles:
        box.add_particle(**p)
        ref.add_particle(**p)
    return box, ref


def _nanmax(d):
    """max |d| with any NaN or Inf counted as an infinite difference."""
    d = np.abs(d)
    if not np.all(np.isfinite(d)):
        return float("inf")
    return float(np.max(d)) if d.size else 0.0


def max_abs(a, b, mask=None):
    if mask is not None:
        sel = mask == 0
        if a.ndim == 4:
            return _nanmax(a[:, sel] - b[:, sel])
        return _nanmax(a[sel] - b[sel])
    return _nanmax(a - b)


def norm_rel(a, b, mask=None):
    """max|a - b| / max|b| over fluid nodes."""
    sel = (mask == 0) if mask is not None else np.ones(b.shape[-3:], bool)
    bb = b[..., sel] if b.ndim == 4 else b[sel]
    aa = a[..., sel] if a.ndim == 4 else a[sel]
    den = float(np.max(np.abs(bb)))
    return _nanmax(aa - bb) / (den if den > 0 else 1.0)


def compare(box, ref, check_pops=True):
    """Dict of max-abs differences per field over fluid nodes (masks must match)."""
    mg, mr = box.mask(), ref.mask()
    out = {"mask_mismatch": int(np.sum(mg != mr))}
    fg, fr = box.fields(), ref.fields()
    for k in FIELDS:
        out[k] = max_abs(fg[k], fr[k], mr)
    if check_pops:
        out["f"] = max_abs(box.populations(), ref.populations(), mr)
    pg, pr = box.particles(), ref.particles()
    for k in PSTATE:
        out["p_" + k] = max([_nanmax(a[k] - b[k]) for a, b in zip(pg, pr)] or [0.0])
    return out
