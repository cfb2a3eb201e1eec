"""Seeded synthetic inputs for the lattice step.

This module only builds inputs: box sizes, parameters, initial fields and
particle descriptors, all drawn from ``numpy.random.default_rng(seed)``.  It
holds none of the model's arithmetic, so both the CUDA library and the CPU
oracle can be driven from the same inputs.  Conversions that belong to the
model (contact angle to surface field, solubility ratio to ``E``) are left to
each side; a workload carries ``theta_c_deg`` and ``solubility_ratio``.

Workloads (parameters follow Sec. "Numerical details" unless stated):

* ``plain_fp64``  -- 32^3 box, periodic in x and y, walls in z; binary fluid
  psi = tanh((z-16)/2); solute 0; one Janus sphere R=4 at (16,16,10) with a
  seeded orientation, cap production 1e-3, contact angle 90 degrees.
* ``interface``   -- 128^3 box with one sphere R=8 straddling the flat
  interface z=64; contact angle, solubility ratio and phoretic mobility given.
* ``precision``   -- 256^3 box, 8 spheres R=6 at seeded positions in the slab
  20 < z < 60 below the interface z=128.
* ``batched``     -- 64 cubic boxes, edge uniform in 32..96, each with one
  sphere R in [4, 8] straddling a flat interface at mid-height; contact
  angle, solubility ratio and mobility uniform in [45, 135] deg, [0.25, 4],
  [-0.2, 0.2].
* ``serving_requests`` -- a Poisson stream (mean 20 requests/s) of boxes with
  edge uniform in 24..128, step counts log-uniform in 500..20000 and 1 to 4
  spheres, parameters drawn as for ``batched``.
* ``scaled``      -- any of the above shrunk to a smaller edge for tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

# Free-energy and transport parameters shared by the workloads: A = C,
# kappa (Sec. "Numerical details"); psi mobility 0.1 and solute diffusivity
# D = C * M_phi = 0.1 as the plain-method configuration states them.
BASE_PARAMS = dict(tau=1.0, rho0=1.0, body_force=(0.0, 0.0, 0.0),
                   A=0.0625, kappa=0.04, M_psi=0.1, C=0.0625, M_phi=1.6,
                   phi_b=0.0, k_d=1e-3, thermo_force=1)


@dataclasses.dataclass
class Workload:
    name: str
    params: Dict                      # nx, ny, nz, periodic, ... , solubility_ratio
    fields: Dict[str, np.ndarray]     # rho [nz,ny,nx], u [3,nz,ny,nx], psi, phi
    particles: List[Dict]             # descriptors with theta_c_deg
    steps: int

    @property
    def nodes(self) -> int:
        p = self.params
        return int(p["nx"]) * int(p["ny"]) * int(p["nz"])


def random_unit_vector(rng: np.random.Generator) -> np.ndarray:
    """Orientation uniform on the sphere: a normalised 3-D Gaussian draw."""
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def flat_interface_fields(nx: int, ny: int, nz: int, z0: float, width: float = 2.0,
                          phi_init: float = 0.0, rho: float = 1.0) -> Dict[str, np.ndarray]:
    """psi = tanh((z - z0) / width) (water above z0), solute uniform, fluid at rest."""
    z = np.arange(nz, dtype=np.float64)
    prof = np.tanh((z - z0) / width)
    psi = np.ascontiguousarray(np.broadcast_to(prof[:, None, None], (nz, ny, nx)))
    return dict(rho=np.full((nz, ny, nx), rho), u=np.zeros((3, nz, ny, nx)),
                psi=psi, phi=np.full((nz, ny, nx), phi_init))


def plain_fp64(seed: int = 0, edge: int = 32) -> Workload:
    s = edge / 32.0
    rng = np.random.default_rng(seed)
    params = dict(BASE_PARAMS, nx=edge, ny=edge, nz=edge, periodic=(1, 1, 0),
                  solubility_ratio=1.0)
    fields = flat_interface_fields(edge, edge, edge, z0=16.0 * s)
    part = dict(pos=(16.0 * s, 16.0 * s, 10.0 * s), R=4.0 * s, m_hat=tuple(random_unit_vector(rng)),
                alpha=1e-3, mu_plus=0.0, mu_minus=0.0, theta_c_deg=90.0, rho_p=1.0)
    return Workload("plain_fp64_%d" % edge, params, fields, [part], 200)


def interface(theta_c_deg: float = 90.0, solubility_ratio: float = 1.0, mobility: float = 0.1,
              seed: int = 0, edge: int = 128, steps: int = 20000) -> Workload:
    s = edge / 128.0
    rng = np.random.default_rng(seed)
    phi_b = 0.0 if solubility_ratio == 1.0 else 1.0
    params = dict(BASE_PARAMS, nx=edge, ny=edge, nz=edge, periodic=(1, 1, 0),
                  solubility_ratio=solubility_ratio, phi_b=phi_b)
    fields = flat_interface_fields(edge, edge, edge, z0=64.0 * s)
    # the centre sits a quarter node off the lattice planes so that no node
    # lies exactly on the sphere surface
    c = 64.0 * s + 0.25
    part = dict(pos=(c, c, 64.0 * s + 0.3), R=8.0 * s, m_hat=tuple(random_unit_vector(rng)),
                alpha=1e-3, mu_plus=mobility, mu_minus=mobility, theta_c_deg=theta_c_deg,
                rho_p=1.0)
    return Workload("interface_%d" % edge, params, fields, [part], steps)


def precision(seed: int = 0, edge: int = 256, n_spheres: int = 8, R: float = 6.0,
              steps: int = 1000) -> Workload:
    s = edge / 256.0
    rng = np.random.default_rng(seed)
    params = dict(BASE_PARAMS, nx=edge, ny=edge, nz=edge, periodic=(1, 1, 0),
                  solubility_ratio=1.0)
    fields = flat_interface_fields(edge, edge, edge, z0=128.0 * s)
    Rs = R * s
    parts: List[Dict] = []
    tries = 0
    while len(parts) < n_spheres:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place the spheres")
        pos = np.array([rng.uniform(0, edge), rng.uniform(0, edge),
                        rng.uniform(20.0 * s, 60.0 * s)])
        if pos[2] - Rs < 3.0:
            continue
        ok = True
        for q in parts:
            d = pos - np.array(q["pos"])
            d[:2] -= edge * np.round(d[:2] / edge)
            if np.linalg.norm(d) < 2 * Rs + 4.0:
                ok = False
                break
        if ok:
            parts.append(dict(pos=tuple(pos), R=Rs, m_hat=tuple(random_unit_vector(rng)),
                              alpha=1e-3, mu_plus=0.1, mu_minus=0.1, theta_c_deg=90.0,
                              rho_p=1.0))
    return Workload("precision_%d" % edge, params, fields, parts, steps)


def _sweep_box(rng: np.random.Generator, edge: int, n_spheres: int, r_range, name: str,
               steps: int) -> Workload:
    """A cubic box (periodic x/y, walls in z) with a flat interface at
    mid-height and n_spheres spheres straddling it, kept 4 nodes apart and
    at least edge/4 from the walls (an active sphere can leave the interface
    and swim a few radii in a run); contact angle, solubility ratio and
    mobility (within the paper's +-0.1) drawn uniformly."""
    theta = float(rng.uniform(45.0, 135.0))
    ratio = float(rng.uniform(0.25, 4.0))
    mob = float(rng.uniform(-0.1, 0.1))
    params = dict(BASE_PARAMS, nx=edge, ny=edge, nz=edge, periodic=(1, 1, 0),
                  solubility_ratio=ratio, phi_b=1.0)
    z0 = edge / 2.0
    fields = flat_interface_fields(edge, edge, edge, z0=z0)
    parts: List[Dict] = []
    tries = 0
    while len(parts) < n_spheres:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place the spheres")
        R = float(rng.uniform(*r_range))
        pos = np.array([rng.uniform(0, edge), rng.uniform(0, edge), z0 + 0.3 + rng.uniform(-0.5, 0.5) * R])
        ok = pos[2] - R >= edge / 4.0 and pos[2] + R <= edge - edge / 4.0
        for q in parts:
            d = pos - np.array(q["pos"])
            d[:2] -= edge * np.round(d[:2] / edge)
            ok = ok and np.linalg.norm(d) >= R + q["R"] + 4.0
        if ok:
            parts.append(dict(pos=tuple(pos), R=R, m_hat=tuple(random_unit_vector(rng)), alpha=1e-3,
                              mu_plus=mob, mu_minus=mob, theta_c_deg=theta, rho_p=1.0))
    return Workload(name, params, fields, parts, steps)


def _slab_box(rng: np.random.Generator, edge: int, r_range, name: str, steps: int) -> Workload:
    """A cubic box periodic on every axis holding a slab of water between two
    flat interfaces (z = edge/4 and 3 edge/4), one sphere straddling the lower
    one; radius, contact angle, solubility ratio and mobility drawn uniformly.
    With no wall an active sphere may swim anywhere during the run."""
    R = float(rng.uniform(*r_range))
    theta = float(rng.uniform(45.0, 135.0))
    ratio = float(rng.uniform(0.25, 4.0))
    mob = float(rng.uniform(-0.2, 0.2))
    params = dict(BASE_PARAMS, nx=edge, ny=edge, nz=edge, periodic=(1, 1, 1),
                  solubility_ratio=ratio, phi_b=1.0)
    z = np.arange(edge, dtype=np.float64)
    z1, z2 = edge / 4.0, 3.0 * edge / 4.0
    prof = np.tanh((z - z1) / 2.0) - np.tanh((z - z2) / 2.0) - 1.0
    fields = dict(rho=np.ones((edge, edge, edge)), u=np.zeros((3, edge, edge, edge)),
                  psi=np.ascontiguousarray(np.broadcast_to(prof[:, None, None], (edge, edge, edge))),
                  phi=np.zeros((edge, edge, edge)))
    pos = (float(rng.uniform(0, edge)), float(rng.uniform(0, edge)), z1 + 0.3 + float(rng.uniform(-0.5, 0.5)) * R)
    parts = [dict(pos=pos, R=R, m_hat=tuple(random_unit_vector(rng)), alpha=1e-3, mu_plus=mob, mu_minus=mob,
                  theta_c_deg=theta, rho_p=1.0)]
    return Workload(name, params, fields, parts, steps)


def batched(seed: int = 0, n_boxes: int = 64, edge_range=(32, 96), steps: int = 5000) -> List[Workload]:
    """Independent boxes for the batched form, one sphere each with R in
    [4, 8], contact angle in [45, 135] degrees, solubility ratio in [0.25, 4]
    and mobility in [-0.2, 0.2]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_boxes):
        edge = int(rng.integers(edge_range[0], edge_range[1] + 1))
        out.append(_slab_box(rng, edge, (4.0, 8.0), "batched_%d_%d" % (k, edge), steps))
    return out


def serving_requests(seed: int = 0, n: int = 32, rate: float = 20.0, edge_range=(24, 128),
                     steps_range=(500, 20000), spheres=(1, 4)):
    """[(arrival time in s, Workload)] of a seeded Poisson request stream."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += float(rng.exponential(1.0 / rate))
        edge = int(rng.integers(edge_range[0], edge_range[1] + 1))
        steps = int(round(math.exp(rng.uniform(math.log(steps_range[0]), math.log(steps_range[1])))))
        ns = int(rng.integers(spheres[0], spheres[1] + 1))
        rmax = min(8.0, edge / 8.0)
        out.append((t, _sweep_box(rng, edge, ns, (min(3.0, rmax), rmax), "request_%d_%d" % (k, edge), steps)))
    return out


def uniform_fields(nx: int, ny: int, nz: int, rng: Optional[np.random.Generator] = None,
                   psi_amp: float = 0.0, phi_amp: float = 0.0, u_amp: float = 0.0,
                   rho_amp: float = 0.0) -> Dict[str, np.ndarray]:
    """Rest state plus optional seeded uniform noise of the given amplitudes."""
    shape = (nz, ny, nx)
    rng = rng or np.random.default_rng(0)
    return dict(rho=1.0 + rho_amp * rng.uniform(-1, 1, shape),
                u=u_amp * rng.uniform(-1, 1, (3,) + shape),
                psi=psi_amp * rng.uniform(-1, 1, shape),
                phi=phi_amp * rng.uniform(-1, 1, shape))


def min_node_surface_gap(wl: Workload) -> float:
    """Smallest | |x - X| - R | over nodes and spheres (a geometric near-tie
    detector: a node closer than ~1e-9 to a surface could be classified
    differently after rounding)."""
    p = wl.params
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    per = p["periodic"]
    best = math.inf
    for q in wl.particles:
        X = np.array(q["pos"], dtype=np.float64)
        R = float(q["R"])
        lo = np.floor(X - R - 2).astype(int)
        hi = np.ceil(X + R + 2).astype(int)
        axes = []
        for a, L in enumerate((nx, ny, nz)):
            c = np.arange(lo[a], hi[a] + 1)
            if per[a]:
                c = c % L
            else:
                c = c[(c >= 0) & (c < L)]
            d = c - X[a]
            if per[a]:
                d = np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d))
            axes.append(d)
        dx, dy, dz = np.meshgrid(axes[0], axes[1], axes[2], indexing="ij")
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        best = min(best, float(np.min(np.abs(r - R))))
    return best
