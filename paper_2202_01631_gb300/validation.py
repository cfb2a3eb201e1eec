"""Long-run validation studies of the model on the GPU (all runs of a study
advance together in one batch).

* ``phoretic`` -- a free Janus sphere in bulk fluid produces solute on its cap
  (Eq. activity) and moves by the phoretic slip of Eq. MuJ.  Its steady speed
  along the cap axis must be linear in the mobility and change sign with it
  (Sec. "Results", the mobility dependence); the solute's free-energy
  coupling adds a small offset at zero mobility.
* ``contact`` -- a neutral sphere released at a flat interface relaxes to the
  height set by its contact angle (Eq. fe_wetting and the contact-angle
  relation).  With theta measured through the oil phase (psi = -1, below the
  interface) Young's construction gives z_c - z_int = -R cos(theta).

    python -m paper_2202_01631_gb300.validation phoretic --steps 8000
    python -m paper_2202_01631_gb300.validation contact --steps 20000

Each study prints one JSON line per sample and a summary line; called from
Python, each returns its summary (tests/test_gpu_validation.py asserts them).
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np


def _batch(lbdp, precision):
    return lbdp.Batch(precision=precision, arena_bytes=8 << 30, graph_steps=16)


def _emit(row, verbose):
    if verbose:
        print(json.dumps(row), flush=True)


def phoretic(args, lbdp, W, verbose=True):
    mobilities = [float(m) for m in args.mobilities.split(",")]
    L = args.edge
    batch = _batch(lbdp, args.precision)
    boxes = []
    m_hat = (0.0, 0.0, 1.0)
    for mu in mobilities:
        p = dict(W.BASE_PARAMS, nx=L, ny=L, nz=L, periodic=(1, 1, 1), k_d=args.k_d, E=0.0, phi_b=0.0)
        b = batch.add_box(**p)
        b.set_fields(psi=np.full((L, L, L), 1.0))   # bulk water
        b.add_particle(pos=(L / 2 + 0.25, L / 2 + 0.25, L / 2 + 0.3), R=args.R, m_hat=m_hat, alpha=args.alpha,
                       mu_plus=mu, mu_minus=mu, theta_c_deg=90.0)
        batch.set_steps(b, args.steps)
        boxes.append(b)
    samples = {mu: [] for mu in mobilities}
    done = 0
    while done < args.steps:
        k = min(args.every, args.steps - done)
        batch.run(k)
        batch.sync()
        done += k
        row = {"step": done}
        for mu, b in zip(mobilities, boxes):
            q = b.particles()[0]
            v = float(np.dot(q["vel"], q["m_hat"]))
            samples[mu].append(v)
            row["mu=%g" % mu] = v
        _emit(row, verbose)
    # steady speed: mean over the last quarter of the samples
    tail = max(1, len(samples[mobilities[0]]) // 4)
    speed = {mu: float(np.mean(samples[mu][-tail:])) for mu in mobilities}
    x = np.array(mobilities)
    y = np.array([speed[mu] for mu in mobilities])
    slope = float(np.dot(x, y) / np.dot(x, x))
    resid = float(np.max(np.abs(y - slope * x)) / max(np.max(np.abs(y)), 1e-300))
    # least-squares line with an intercept (the solute's free-energy coupling
    # moves the sphere a little even at zero mobility) and its R^2
    A = np.vstack([x, np.ones_like(x)]).T
    (b1, b0), *_ = np.linalg.lstsq(A, y, rcond=None)
    r2 = float(1.0 - np.sum((y - (b1 * x + b0)) ** 2) / np.sum((y - np.mean(y)) ** 2))
    summary = {"study": "phoretic", "edge": L, "R": args.R, "alpha": args.alpha, "k_d": args.k_d,
               "steps": args.steps, "speed_along_m": speed, "fit_speed_per_mobility": slope,
               "max_rel_deviation_from_linear": resid, "line_slope": float(b1), "line_intercept": float(b0),
               "r2": r2}
    _emit({"summary": summary}, verbose)
    batch.close()
    return summary


def contact(args, lbdp, W, verbose=True):
    thetas = [float(t) for t in args.thetas.split(",")]
    L = args.edge
    z0 = L / 2.0
    batch = _batch(lbdp, args.precision)
    boxes = []
    for th in thetas:
        p = dict(W.BASE_PARAMS, nx=L, ny=L, nz=L, periodic=(1, 1, 0), k_d=0.0, E=0.0, phi_b=0.0)
        b = batch.add_box(**p)
        b.set_fields(**W.flat_interface_fields(L, L, L, z0=z0))
        b.add_particle(pos=(L / 2 + 0.25, L / 2 + 0.25, z0 + 0.3), R=args.R, m_hat=(0.0, 0.0, 1.0), alpha=0.0,
                       mu_plus=0.0, mu_minus=0.0, theta_c_deg=th)
        batch.set_steps(b, args.steps)
        boxes.append(b)
    track = {th: [] for th in thetas}
    done = 0
    while done < args.steps:
        k = min(args.every, args.steps - done)
        batch.run(k)
        batch.sync()
        done += k
        row = {"step": done}
        for th, b in zip(thetas, boxes):
            h = float(b.particles()[0]["pos"][2] - z0)
            track[th].append(h)
            row["theta=%g" % th] = h
        _emit(row, verbose)
    tail = max(1, len(track[thetas[0]]) // 4)
    rest = {th: float(np.mean(track[th][-tail:])) for th in thetas}
    young = {th: -args.R * math.cos(math.radians(th)) for th in thetas}
    summary = {"study": "contact", "edge": L, "R": args.R, "steps": args.steps, "rest_height": rest,
               "young_minus_R_cos_theta": young}
    _emit({"summary": summary}, verbose)
    batch.close()
    return summary


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["phoretic", "contact"])
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--edge", type=int, default=48)
    ap.add_argument("--R", type=float, default=4.0)
    ap.add_argument("--alpha", type=float, default=1e-2)
    ap.add_argument("--k_d", type=float, default=1e-3)
    ap.add_argument("--mobilities", default="-0.2,-0.1,0,0.1,0.2")
    ap.add_argument("--thetas", default="60,90,120")
    return ap.parse_args(argv)


def main(argv=None):
    args = parse(argv)
    from paper_2202_01631_gb300 import build
    build.build()
    import torch  # noqa: F401  (initialises the CUDA context the library shares)
    from paper_2202_01631_gb300 import lbdp
    from paper_2202_01631_gb300 import workloads as W
    if args.study == "phoretic":
        phoretic(args, lbdp, W)
    else:
        contact(args, lbdp, W)
    return 0


if __name__ == "__main__":
    sys.exit(main())
