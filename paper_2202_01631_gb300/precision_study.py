"""Error of FP32 arithmetic and reduced-precision storage against FP64.

The same seeded input -- by default the 256^3 box with eight Janus spheres
R=6 in the slab 20 < z < 60 below a flat interface at z = 128, or with
``--workload interface`` the 128^3 box with one sphere R=8 at the interface
(contact angle, solubility ratio and mobility as given) -- is advanced in every
precision mode of the library side by side; every ``--every`` steps the
fields and particles of each mode are read back and compared with the FP64
mode (which the parity tests hold to the CPU oracle within 1e-10 on smaller
boxes).  Reported per field: max-abs difference and max|a - b| / max|b| over
nodes that are fluid in both runs; per particle: |dX| / R.

    python -m paper_2202_01631_gb300.precision_study --steps 5000 --every 1000
    python -m paper_2202_01631_gb300.precision_study --workload interface --theta 120 \
        --ratio 0.5 --mobility -0.1 --steps 20000 --every 5000 --modes fp32,fp16

prints one JSON line per checkpoint and a final summary line.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def _far_mask(wl, pos, margin):
    """Nodes farther than R + margin from every sphere centre (periodic x, y)."""
    p = wl.params
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    far = np.ones((nz, ny, nx), dtype=bool)
    for q, X in zip(wl.particles, pos):
        d = [x - X[0], y - X[1], z - X[2]]
        for a, L in ((0, nx), (1, ny)):
            d[a] = d[a] - L * np.round(d[a] / L)
        far &= (d[0] ** 2 + d[1] ** 2 + d[2] ** 2) > (q["R"] + margin) ** 2
    return far


def _errors(ref, got, mref, mgot, far):
    """Per field: max-abs, max|a-b|/max|b| and RMS-relative over nodes fluid
    in both runs, and max|a-b|/max|b| over fluid nodes away from the spheres."""
    fluid = (mref == 0) & (mgot == 0)
    sel_far = fluid & far
    out = {}
    for k in ("rho", "u", "psi", "phi"):
        a, b = got[k], ref[k]
        if a.ndim == 3:
            a, b = a[None], b[None]
        d = a[:, fluid] - b[:, fluid]
        bb = b[:, fluid]
        den = float(np.max(np.abs(bb)))
        mx = float(np.max(np.abs(d))) if d.size else 0.0
        if not np.all(np.isfinite(d)):
            mx = float("inf")
        rms = float(np.sqrt(np.mean(d * d)) / max(np.sqrt(np.mean(bb * bb)), 1e-300))
        dfar = np.abs(a[:, sel_far] - b[:, sel_far])
        out[k] = {"max_abs": mx, "norm_rel": mx / den if den > 0 else mx, "rms_rel": rms,
                  "norm_rel_far": (float(np.max(dfar)) / den if den > 0 else 0.0) if dfar.size else 0.0}
    out["mask_mismatch"] = int(np.sum(mref != mgot))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="precision", choices=["precision", "interface"],
                    help="precision: 256^3 with eight spheres; interface: one sphere at a flat interface")
    ap.add_argument("--edge", type=int, default=0, help="box edge (default 256 / 128 by workload)")
    ap.add_argument("--theta", type=float, default=60.0, help="interface workload: contact angle (deg)")
    ap.add_argument("--ratio", type=float, default=2.0, help="interface workload: solubility ratio")
    ap.add_argument("--mobility", type=float, default=0.1, help="interface workload: phoretic mobility")
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--modes", default="fp32,fp16,bf16")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-particles", action="store_true", help="the same box without spheres")
    ap.add_argument("--far", type=float, default=4.0, help="margin (nodes) beyond R of the far-field error")
    args = ap.parse_args(argv)

    import torch
    from paper_2202_01631_gb300 import build
    build.build()
    from paper_2202_01631_gb300 import lbdp
    from paper_2202_01631_gb300 import workloads as W

    if args.workload == "precision":
        wl = W.precision(seed=args.seed, edge=args.edge or 256)
    else:
        wl = W.interface(theta_c_deg=args.theta, solubility_ratio=args.ratio, mobility=args.mobility,
                         seed=args.seed, edge=args.edge or 128)
    if args.no_particles:
        wl.particles = []
    modes = ["fp64"] + [m for m in args.modes.split(",") if m and m != "fp64"]
    boxes = {}
    for m in modes:
        b = lbdp.Box(precision=m, **wl.params)
        b.set_fields(**wl.fields)
        for p in wl.particles:
            b.add_particle(**p)
        boxes[m] = b
    R = np.array([p["R"] for p in wl.particles])
    timing = {m: 0.0 for m in modes}
    done = 0
    history = []
    while done < args.steps:
        k = min(args.every, args.steps - done)
        for m in modes:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            boxes[m].step(k)
            boxes[m].sync()
            timing[m] += time.perf_counter() - t0
        done += k
        ref = boxes["fp64"]
        fr, mr = ref.fields(), ref.mask()
        pr = ref.particles()
        far = _far_mask(wl, [q["pos"] for q in pr], args.far)
        row = {"step": done}
        for m in modes[1:]:
            b = boxes[m]
            e = _errors(fr, b.fields(), mr, b.mask(), far)
            pg = b.particles()
            e["particle_dX_over_R"] = float(max([np.linalg.norm(a["pos"] - c["pos"]) / r
                                                 for a, c, r in zip(pg, pr, R)] or [0.0]))
            # totals per node: conservation drift against FP64
            e["totals_diff_per_node"] = [float(abs(x - y) / wl.nodes)
                                         for x, y in zip(b.conservation(), ref.conservation())]
            row[m] = e
        history.append(row)
        print(json.dumps(row), flush=True)
    nodes = wl.nodes
    summary = {"workload": wl.name, "nodes": nodes, "spheres": len(wl.particles), "steps": args.steps,
               "theta_c_deg": wl.particles[0]["theta_c_deg"] if wl.particles else None,
               "solubility_ratio": wl.params.get("solubility_ratio"),
               "mobility": wl.particles[0]["mu_plus"] if wl.particles else None,
               "mlups": {m: nodes * args.steps / timing[m] / 1e6 for m in modes},
               "final": history[-1] if history else None}
    print(json.dumps({"summary": summary}), flush=True)
    for b in boxes.values():
        b.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
