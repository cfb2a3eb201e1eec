"""Pins of the oracle's lattice-Boltzmann variant of the psi/phi transport
(scalar_scheme = 1: D3Q7 distributions whose equilibrium carries the chemical
potential, relaxation time 1, moving-wall bounce-back at particles).

As for the finite-difference scheme, nothing here retypes an oracle formula:
the variant is checked against exact discrete Fourier solutions (diffusion
and advection, amplitude and phase), exact invariants, the exact source/sink
balance and the closed-form flat interface of Eq. free_energy.
"""
import math

import numpy as np

from oracle.lbref import Oracle
from tests.oracle_util import neighbours_inside

PASSIVE = dict(A=0.0, kappa=0.0, E=0.0, thermo_force=0, scalar_scheme=1)


def _lap7_symbol(n):
    k = 2 * np.pi * np.fft.fftfreq(n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    return kx, ky, kz, 2 * (np.cos(kx) - 1) + 2 * (np.cos(ky) - 1) + 2 * (np.cos(kz) - 1)


def _blob(n):
    x = np.arange(n) - n // 2
    zz, yy, xx = np.meshgrid(x, x, x, indexing="ij")
    return np.exp(-((xx - 1.3) ** 2 + yy ** 2 + (zz + 0.7) ** 2) / 6.0)


def test_lb_diffusion_matches_spectral_solution():
    """Fluid at rest: the D3Q7 scheme with relaxation time 1 and the
    equilibrium of mobility M is linear, so each Fourier mode k is multiplied
    per step by 1 + D lambda7(k) - k_d with D = C M_phi and lambda7 the symbol
    of the 7-point Laplacian (Eq. diffusion_reaction with mu_phi = C phi)."""
    n, steps, Cc, Mphi, kd = 16, 40, 0.0625, 1.6, 2e-3
    o = Oracle(dict(nx=n, ny=n, nz=n, C=Cc, M_phi=Mphi, k_d=kd, **PASSIVE))
    phi0 = _blob(n)
    o.set_fields(phi=phi0)
    o.step(steps)
    _, _, _, lam = _lap7_symbol(n)
    G = 1.0 + Cc * Mphi * lam - kd
    want = np.real(np.fft.ifftn(np.fft.fftn(phi0) * G ** steps))
    assert np.max(np.abs(o.fields()["phi"] - want)) < 1e-12


def test_lb_advection_matches_spectral_solution():
    """Uniform flow u (no force, so it stays uniform): the first moment of the
    equilibrium is g u, and streaming makes each mode gain the factor
    -i sum_a u_a sin k_a per step on top of the diffusive one -- amplitude and
    phase, so a wrong sign or a transposed component fails."""
    n, steps, Cc, Mphi = 16, 30, 0.0625, 0.8
    u0 = np.array([0.04, -0.02, 0.03])
    o = Oracle(dict(nx=n, ny=n, nz=n, C=Cc, M_phi=Mphi, k_d=0.0, **PASSIVE))
    phi0 = _blob(n)
    u = np.broadcast_to(u0[:, None, None, None], (3, n, n, n)).copy()
    o.set_fields(u=u, phi=phi0)
    o.step(steps)
    kx, ky, kz, lam = _lap7_symbol(n)
    G = 1.0 + Cc * Mphi * lam - 1j * (u0[0] * np.sin(kx) + u0[1] * np.sin(ky) + u0[2] * np.sin(kz))
    want = np.real(np.fft.ifftn(np.fft.fftn(phi0) * G ** steps))
    got = o.fields()
    assert np.max(np.abs(got["u"] - u)) < 1e-14
    assert np.max(np.abs(got["phi"] - want)) < 1e-12


def test_lb_totals_conserved_with_moving_sphere():
    """Without sources the totals of psi and phi are invariants of collision
    and streaming; the moving-wall bounce-back carries g c.u_b into the
    surface, and covering/uncovering plus the uniform correction restore the
    totals exactly (reading C12)."""
    n = 16
    rng = np.random.default_rng(4)
    o = Oracle(dict(nx=n, ny=n, nz=n, E=0.3, M_psi=0.1, M_phi=0.8, scalar_scheme=1))
    o.set_fields(psi=0.3 * rng.uniform(-1, 1, (n, n, n)), phi=0.2 * rng.uniform(0, 1, (n, n, n)),
                 u=0.01 * rng.uniform(-1, 1, (3, n, n, n)))
    o.add_particle(pos=(6.3, 8.2, 7.9), R=3.2, vel=(0.06, 0.01, -0.03), fixed=1,
                   mu_plus=0.1, mu_minus=0.2, theta_c_deg=60.0, m_hat=(0, 1, 1))
    s0 = o.conservation()
    m0 = o.mask().copy()
    o.step(50)
    s1 = o.conservation()
    assert np.sum(o.mask() != m0) > 0
    assert abs(s1[1] - s0[1]) < 1e-12 * n ** 3
    assert abs(s1[2] - s0[2]) < 1e-12 * n ** 3
    assert o.error() == 0


def test_lb_source_sink_balance():
    """Per step the total solute changes by alpha N_active - k_d sum(phi - phi0)
    (Eq. diffusion_reaction, Eq. activity): the sources enter the rest
    population, which streaming does not move; N_active by brute force."""
    n = 16
    alpha, kd, E = 1e-3, 2e-3, 0.2
    rng = np.random.default_rng(5)
    X, R, m = np.array([8.3, 7.7, 8.1]), 3.4, np.array([1.0, 2.0, -0.5])
    m = m / np.linalg.norm(m)
    o = Oracle(dict(nx=n, ny=n, nz=n, k_d=kd, E=E, scalar_scheme=1))
    o.set_fields(psi=0.2 * rng.uniform(-1, 1, (n, n, n)), phi=0.1 * rng.uniform(0, 1, (n, n, n)))
    o.add_particle(pos=tuple(X), R=R, m_hat=tuple(m), alpha=alpha, fixed=1)
    adj, solid = neighbours_inside((n, n, n), (1, 1, 1), X, R)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    d = [np.where(c - Xa > n / 2, c - Xa - n, np.where(c - Xa < -n / 2, c - Xa + n, c - Xa))
         for c, Xa in ((x, X[0]), (y, X[1]), (z, X[2]))]
    n_act = int((adj & (m[0] * d[0] + m[1] * d[1] + m[2] * d[2] <= 0)).sum())
    assert n_act > 10
    for _ in range(3):
        fl = o.fields()
        sink = kd * np.sum((fl["phi"] - E * np.tanh(fl["psi"]))[~solid])
        before = o.conservation()[2]
        o.step(1)
        after = o.conservation()[2]
        assert abs((after - before) - (alpha * n_act - sink)) < 1e-11


def test_lb_flat_interface_profile():
    """The stationary state requires uniform mu whatever the transport scheme,
    so the variant relaxes to the same tanh profile, width sqrt(2 kappa/A), as
    the finite-difference scheme (Eq. free_energy, Sec. "Numerical details").
    Stable for M kappa |lambda7| |lambda19| < 2; M = 0.5 at kappa = 0.04."""
    A, kappa, M, nz = 0.0625, 0.04, 0.5, 48
    o = Oracle(dict(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), A=A, kappa=kappa, M_psi=M, scalar_scheme=1))
    z = np.arange(nz, dtype=float)
    o.set_fields(psi=np.ascontiguousarray(np.tanh((z - (nz - 1) / 2) / 2.0)[:, None, None]))
    o.step(40000)
    psi = o.fields()["psi"][:, 0, 0]
    mu = o.mu()[0][:, 0, 0]
    assert np.max(np.abs(mu - mu.mean())) < 1e-6
    assert abs(psi[0] + 1) < 1e-5 and abs(psi[-1] - 1) < 1e-5
    core = np.abs(psi) < 0.9
    xi_fit = 1.0 / np.polyfit(z[core], np.arctanh(psi[core]), 1)[0]
    assert abs(xi_fit - math.sqrt(2 * kappa / A)) < 0.08 * math.sqrt(2 * kappa / A)


def test_unknown_scheme_rejected():
    import pytest
    with pytest.raises(ValueError):
        Oracle(dict(nx=4, ny=4, nz=4, scalar_scheme=2))


def test_lb_wall_bounce_back_is_zero_flux():
    """At rest, halfway bounce-back of the D3Q7 distributions at a wall
    returns what left: the update is the 7-point Laplacian with zero-flux
    walls, whose modes cos(pi k (z + 1/2) / L) decay by exactly
    1 + D 2 (cos(pi k / L) - 1) per step (D = C M_phi); the total stays."""
    L, steps, Cc, Mphi = 16, 60, 0.0625, 1.6
    o = Oracle(dict(nx=4, ny=3, nz=L, periodic=(1, 1, 0), C=Cc, M_phi=Mphi, k_d=0.0, **PASSIVE))
    z = np.arange(L, dtype=float)
    mode = np.cos(np.pi * 3 * (z + 0.5) / L)
    phi0 = 1.0 + 0.5 * np.cos(np.pi * (z + 0.5) / L) + 0.25 * mode
    o.set_fields(phi=np.ascontiguousarray(np.broadcast_to(phi0[:, None, None], (L, 3, 4))))
    tot0 = o.conservation()[2]
    o.step(steps)
    g1 = 1.0 + Cc * Mphi * 2 * (np.cos(np.pi / L) - 1)
    g3 = 1.0 + Cc * Mphi * 2 * (np.cos(3 * np.pi / L) - 1)
    want = 1.0 + 0.5 * g1 ** steps * np.cos(np.pi * (z + 0.5) / L) + 0.25 * g3 ** steps * mode
    got = o.fields()["phi"]
    assert np.max(np.abs(got - want[:, None, None])) < 1e-12
    assert abs(o.conservation()[2] - tot0) < 1e-11


def test_lb_moving_wall_matches_comoving_fluid():
    """A uniform solute in a fluid moving at U, with a sphere moving at the
    same U: the moving-wall bounce-back hands back h*(x) - g c.U, which is
    exactly what a fluid neighbour at velocity U would send, so phi stays
    uniform over the fluid (covering shifts it as a whole, keeping the total);
    a wrong sign or factor in the surface term leaves a ring around the
    sphere."""
    n = 16
    U = np.array([0.02, -0.01, 0.015])
    o = Oracle(dict(nx=n, ny=n, nz=n, A=0.0, kappa=0.0, E=0.0, phi_b=1.0, k_d=0.0, thermo_force=0,
                    scalar_scheme=1))
    u = np.broadcast_to(U[:, None, None, None], (3, n, n, n)).copy()
    o.set_fields(u=u, phi=np.ones((n, n, n)))
    o.add_particle(pos=(8.3, 7.9, 8.1), R=3.3, vel=tuple(U), fixed=1, alpha=0.0, mu_plus=0.0, mu_minus=0.0,
                   theta_c_deg=90.0, m_hat=(0, 0, 1))
    tot0 = o.conservation()[2]
    for _ in range(4):
        o.step(1)
        fluid = o.mask() == 0
        phi = o.fields()["phi"][fluid]
        assert np.max(phi) - np.min(phi) < 1e-13
        assert abs(o.conservation()[2] - tot0) < 1e-12 * n ** 3
