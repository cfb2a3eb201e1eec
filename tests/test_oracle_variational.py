"""Variational and symmetry pins of the oracle's chemical potentials and of
the Janus mobility rule.

* The chemical potentials are the derivatives of the free energy: mu_psi =
  dF/dpsi and mu_phi = dF/dphi (Sec. "Computational model", Eqs.
  free_energy and chem_potentials), with the wetting term added to F over
  the solid surface (Sec. "Particles", Eq. fe_wetting).  The test writes the
  lattice free energy in NumPy -- bulk density f = A psi^4/4 - A psi^2/2 +
  C (phi - phi_b - E tanh psi)^2/2 at every fluid node, the gradient energy
  as a sum over fluid-fluid links, and H psi integrated over each sphere's
  surface with the lattice surface element of a boundary link -- and
  differentiates it node by node with the complex step (exact to rounding).
  The oracle's mu at every fluid node must agree to ~1e-12.  A wrong sign or
  a dropped 1/cosh^2 in the solubility term, a wrong Laplacian weight or a
  wrong factor in the wetting ghost fails it.
* Swapping mu_+ and mu_- of a fixed sphere in a uniform solute gradient
  mirrors the slip field: the torque about m x grad phi flips sign exactly,
  vanishes when mu_+ = mu_-, and turns m (the mu_+ side, Eq. MuJ) towards
  low solute when mu_+ > mu_- > 0 -- the more repulsive face turns towards
  the phase with less product (Sec. "Conclusions").
"""
import math

import numpy as np
import pytest

from oracle.lbref import Oracle, wetting_h
from tests.oracle_util import C19

W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _geometry(shape, periodic, spheres):
    """Solid owner per node (0 fluid, k+1 sphere k, first match) and, per
    sphere, its boundary links (node, direction, unit normal at the link
    midpoint)."""
    nz, ny, nx = shape
    L = (nx, ny, nz)
    owner = np.zeros(shape, dtype=np.int64)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = (x, y, z)

    def offset(X, extra=(0.0, 0.0, 0.0)):
        d = []
        for a in range(3):
            v = coords[a] - X[a]
            if periodic[a]:
                v = np.where(v > 0.5 * L[a], v - L[a], np.where(v < -0.5 * L[a], v + L[a], v))
            d.append(v + extra[a])
        return d

    for k, (X, R) in enumerate(spheres):
        d = offset(X)
        inside = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 < R * R
        owner = np.where((owner == 0) & inside, k + 1, owner)
    links = []
    for k, (X, R) in enumerate(spheres):
        for i in range(1, 19):
            c = C19[i]
            nbr_owner, valid = _shifted(owner, c, periodic, fill=-1)
            sel = (owner == 0) & valid & (nbr_owner == k + 1)
            d = offset(X, 0.5 * c)
            r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
            for idx in zip(*np.nonzero(sel)):
                nh = np.array([d[0][idx], d[1][idx], d[2][idx]]) / r[idx]
                links.append((k, idx, i, nh))
    return owner, links


def _shifted(a, c, periodic, fill):
    """b[x] = a[x + c] (periodic wrap or `fill` beyond a wall) and the
    validity of each entry."""
    b = a
    valid = np.ones(a.shape, dtype=bool)
    for ax_field, comp, per in ((2, int(c[0]), periodic[0]), (1, int(c[1]), periodic[1]),
                                (0, int(c[2]), periodic[2])):
        if comp == 0:
            continue
        b = np.roll(b, -comp, axis=ax_field)
        if not per:
            v = np.ones(a.shape, dtype=bool)
            sl = [slice(None)] * 3
            sl[ax_field] = slice(-1, None) if comp > 0 else slice(0, 1)
            v[tuple(sl)] = False
            valid &= v
    b = np.where(valid, b, fill)
    return b, valid


def lattice_free_energy(psi, phi, owner, links, H, prm, periodic):
    """F = sum_fluid f(psi, phi) + (3 kappa / 2) sum_x sum_i w_i (psi(x+c_i) -
    psi(x))^2 over ordered fluid-fluid pairs + sum_links H 6 w_i |c_i.n| psi(x).

    The gradient term equals kappa |grad psi|^2 / 2 in the continuum limit
    (sum_i w_i c_i c_i = I/3); 6 w_i |c_i.n| is the surface element one
    boundary link carries (1 per node on a flat lattice plane, checked
    below)."""
    A, kappa, C, E, phib = prm["A"], prm["kappa"], prm["C"], prm["E"], prm["phi_b"]
    fluid = owner == 0
    d = phi - (phib + E * np.tanh(psi))
    bulk = 0.25 * A * psi ** 4 - 0.5 * A * psi ** 2 + 0.5 * C * d * d
    F = np.sum(np.where(fluid, bulk, 0.0))
    for i in range(1, 19):
        nb, valid = _shifted(psi, C19[i], periodic, fill=0.0)
        nbf, _ = _shifted(fluid, C19[i], periodic, fill=False)
        pair = fluid & valid & nbf
        F = F + 1.5 * kappa * W19[i] * np.sum(np.where(pair, (nb - psi) ** 2, 0.0))
    for k, idx, i, nh in links:
        F = F + H[k] * 6.0 * W19[i] * abs(float(np.dot(C19[i], nh))) * psi[idx]
    return F


def test_surface_element_of_a_flat_plane():
    """sum over the links crossing a lattice plane, per node, of 6 w_i |c_i.n|
    is 1 (the plane's area per node) for each axis normal."""
    for a in range(3):
        n = np.zeros(3)
        n[a] = 1.0
        s = sum(6 * W19[i] * abs(C19[i] @ n) for i in range(1, 19) if C19[i] @ n < 0)
        assert abs(s - 1.0) < 1e-15


@pytest.mark.parametrize("E", [0.0, 0.45, -0.6])
def test_mu_is_the_variational_derivative_of_the_free_energy(E):
    shape = (9, 8, 8)
    periodic = (1, 1, 0)
    rng = np.random.default_rng(11)
    nz = shape[0]
    z = np.arange(nz)[:, None, None]
    psi = np.tanh((z - 4.3) / 1.5) + 0.3 * rng.uniform(-1, 1, shape)
    phi = 0.4 + 0.3 * rng.uniform(-1, 1, shape)
    prm = dict(A=0.0625, kappa=0.04, C=0.09, E=E, phi_b=0.7)
    spheres = [((3.3, 3.6, 4.2), 2.1, 60.0), ((6.9, 0.4, 5.1), 1.6, 125.0)]
    o = Oracle(dict(nx=8, ny=8, nz=9, periodic=periodic, M_psi=0.1, M_phi=1.0, k_d=0.0, **prm))
    o.set_fields(psi=psi, phi=phi)
    for X, R, th in spheres:
        o.add_particle(pos=X, R=R, theta_c_deg=th, fixed=1)
    mps, mph = o.mu()
    owner, links = _geometry(shape, periodic, [(X, R) for X, R, _ in spheres])
    assert np.array_equal(owner, o.mask().astype(np.int64))
    H = [wetting_h(th) * math.sqrt(prm["kappa"] * prm["A"]) for _, _, th in spheres]
    assert len(links) > 40 and all(abs(h) > 1e-3 for h in H)
    step = 1e-20
    worst = 0.0
    for idx in zip(*np.nonzero(owner == 0)):
        p = psi.astype(complex)
        p[idx] += 1j * step
        d_psi = lattice_free_energy(p, phi.astype(complex), owner, links, H, prm, periodic).imag / step
        q = phi.astype(complex)
        q[idx] += 1j * step
        d_phi = lattice_free_energy(psi.astype(complex), q, owner, links, H, prm, periodic).imag / step
        worst = max(worst, abs(d_psi - mps[idx]), abs(d_phi - mph[idx]))
    assert worst < 1e-12, worst


def _torque(mu_plus, mu_minus):
    n = 16
    o = Oracle(dict(nx=n, ny=n, nz=n, periodic=(1, 1, 0), thermo_force=0, A=0.0, kappa=0.0, E=0.0,
                    M_phi=0.5, k_d=0.0))
    G = 2e-3
    z = np.arange(n, dtype=float)
    o.set_fields(phi=np.ascontiguousarray(np.broadcast_to((0.5 + G * z)[:, None, None], (n, n, n))))
    # centre on a mirror plane of the lattice (x -> 16 - x, y -> 16 - y)
    o.add_particle(pos=(8.0, 8.0, 7.6), R=3.7, m_hat=(1.0, 0.0, 0.0), mu_plus=mu_plus, mu_minus=mu_minus,
                   fixed=1)
    o.step(1)
    t = o.particles()[0]["torque"]
    m_x_grad = np.cross([1.0, 0.0, 0.0], [0.0, 0.0, G])
    return t, float(np.dot(t, m_x_grad / np.linalg.norm(m_x_grad)))


def test_janus_mobility_sides():
    t0, a0 = _torque(0.2, 0.2)
    t1, a1 = _torque(0.3, 0.1)
    t2, a2 = _torque(0.1, 0.3)
    # uniform mobility: no torque (mirror symmetry)
    assert np.max(np.abs(t0)) < 1e-15
    # mu_+ (the m side) more repulsive: m turns towards -grad phi, i.e. the
    # torque points along -(m x grad phi)
    assert a1 < -1e-6
    # swapped sides: the mirror image
    assert abs(a1 + a2) <= 1e-12 * abs(a1)
    assert abs(t1[0]) < 1e-15 and abs(t1[2]) < 1e-15
