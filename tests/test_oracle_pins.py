"""Pins of the FP64 CPU oracle against what the model and mathematics fix.

None of these tests retypes an oracle formula: each checks a closed form, an
exact invariant, a spectral solution or a sign law, chosen so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails one
of them.  Paper passages are cited by section and equation.
"""
import math

import numpy as np
import pytest

from oracle.lbref import Oracle, solubility_E, wetting_h
from tests.oracle_util import C19, momentum, neighbours_inside

PASSIVE = dict(A=0.0, kappa=0.0, E=0.0, thermo_force=0)


# --------------------------------------------------------------------------
# lattice and collision
# --------------------------------------------------------------------------

def test_equilibrium_moments():
    """Equilibrium populations carry density, momentum and the ideal-gas
    momentum flux rho u u + rho/3 I (the solvent of Sec. "Computational model"
    is an ideal LB fluid with c_s^2 = 1/3)."""
    rng = np.random.default_rng(1)
    o = Oracle(dict(nx=4, ny=3, nz=5))
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, (5, 3, 4))
    u = 0.05 * rng.uniform(-1, 1, (3, 5, 3, 4))
    o.set_fields(rho=rho, u=u)
    f = o.populations()
    assert np.allclose(f.sum(0), rho, atol=1e-14)
    for a in range(3):
        assert np.allclose(np.tensordot(C19[:, a], f, axes=(0, 0)), rho * u[a], atol=1e-14)
        for b in range(3):
            pab = np.tensordot(C19[:, a] * C19[:, b], f, axes=(0, 0))
            want = rho * u[a] * u[b] + (rho / 3.0 if a == b else 0.0)
            assert np.allclose(pab, want, atol=1e-14)


def test_rest_state_isotropy():
    """Rest populations w_i rho: sum w = 1, sum w c c = I/3 and the fourth
    moment (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9 -- the isotropy the 19-point
    stencils rely on."""
    o = Oracle(dict(nx=1, ny=1, nz=1))
    w = o.populations()[:, 0, 0, 0]
    assert abs(w.sum() - 1.0) < 1e-15
    d = np.eye(3)
    for a in range(3):
        for b in range(3):
            assert abs(np.sum(w * C19[:, a] * C19[:, b]) - d[a, b] / 3.0) < 1e-15
            for c in range(3):
                for e in range(3):
                    m4 = np.sum(w * C19[:, a] * C19[:, b] * C19[:, c] * C19[:, e])
                    want = (d[a, b] * d[c, e] + d[a, c] * d[b, e] + d[a, e] * d[b, c]) / 9.0
                    assert abs(m4 - want) < 1e-15


def test_mass_and_momentum_under_body_force():
    """Periodic box: mass is exact and the total momentum rises by N g per
    step (Guo forcing with the half-force velocity)."""
    rng = np.random.default_rng(2)
    n = 6
    g = (1e-5, -2e-5, 3e-5)
    o = Oracle(dict(nx=n, ny=n, nz=n, body_force=g, **PASSIVE))
    o.set_fields(rho=1 + 0.01 * rng.uniform(-1, 1, (n, n, n)),
                 u=0.01 * rng.uniform(-1, 1, (3, n, n, n)))
    m0 = o.populations().sum()
    p0 = momentum(o.populations())
    for t in range(1, 6):
        o.step(1)
        f = o.populations()
        assert abs(f.sum() - m0) < 1e-12
        assert np.allclose(momentum(f) - p0, t * n ** 3 * np.array(g), atol=1e-13)


def test_poiseuille_profile():
    """Channel between halfway bounce-back walls at z=-1/2 and z=nz-1/2 driven
    by a body force: u_x(z) = g/(2 nu) (z+1/2)(nz-1/2-z), nu = (tau-1/2)/3
    (nu = 1/6 in Sec. "Numerical details")."""
    nz, g = 32, 1e-6
    o = Oracle(dict(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), body_force=(g, 0, 0), **PASSIVE))
    o.step(8000)
    ux = o.fields()["u"][0, :, 0, 0]
    z = np.arange(nz)
    nu = (1.0 - 0.5) / 3.0
    want = g / (2 * nu) * (z + 0.5) * (nz - 0.5 - z)
    assert np.max(np.abs(ux - want)) < 0.01 * want.max()


# --------------------------------------------------------------------------
# scalar transport (Eq. diffusion_reaction)
# --------------------------------------------------------------------------

def _gaussian(n, s2):
    x = np.arange(n) - n // 2
    zz, yy, xx = np.meshgrid(x, x, x, indexing="ij")
    return np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / (2 * s2))


def test_diffusion_matches_spectral_solution():
    """Fluid at rest, solute with mobility M_phi and stiffness C: the explicit
    update is linear and translation invariant, so each Fourier mode k is
    multiplied per step by 1 + D lambda(k) - k_d, with D = C M_phi and
    lambda(k) the symbol of the isotropic 19-point Laplacian.  The spectral
    solution must hold to round-off."""
    n, steps, Cc, Mphi, kd = 16, 40, 0.0625, 1.6, 2e-3
    o = Oracle(dict(nx=n, ny=n, nz=n, C=Cc, M_phi=Mphi, k_d=kd, **PASSIVE))
    phi0 = _gaussian(n, 3.0)
    o.set_fields(phi=phi0)
    o.step(steps)
    k = 2 * np.pi * np.fft.fftfreq(n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    lam = np.zeros_like(kx)
    for wi, c in zip(w[1:], C19[1:]):
        lam += 6 * wi * (np.cos(kx * c[0] + ky * c[1] + kz * c[2]) - 1.0)
    G = 1.0 + Cc * Mphi * lam - kd
    want = np.real(np.fft.ifftn(np.fft.fftn(phi0) * G ** steps))
    got = o.fields()["phi"]
    assert np.max(np.abs(got - want)) < 1e-12


def test_gaussian_spreads_with_diffusivity():
    """Continuum check of the same update: a Gaussian of variance s0 has
    variance s0 + 2 D t per axis and peak (s0/(s0+2Dt))^{3/2}, isotropically,
    with D = C M_phi."""
    n, steps = 32, 50
    Cc, Mphi = 0.0625, 1.6
    D = Cc * Mphi
    o = Oracle(dict(nx=n, ny=n, nz=n, C=Cc, M_phi=Mphi, **PASSIVE))
    s0 = 4.0
    o.set_fields(phi=_gaussian(n, s0))
    o.step(steps)
    phi = o.fields()["phi"]
    x = np.arange(n) - n // 2
    zz, yy, xx = np.meshgrid(x, x, x, indexing="ij")
    mass = phi.sum()
    var = [np.sum(phi * c ** 2) / mass for c in (xx, yy, zz)]
    s_t = s0 + 2 * D * steps
    for v in var:
        assert abs(v - s_t) < 2e-3 * s_t
    peak = phi[n // 2, n // 2, n // 2]
    # the peak also feels the stencil's fourth cumulant: O(1/s_t) relative
    assert abs(peak - (s0 / s_t) ** 1.5) < 2e-2 * (s0 / s_t) ** 1.5
    # axis and diagonal decay agree (isotropy of the 19-point stencil)
    r = 3
    ax = phi[n // 2, n // 2, n // 2 + r]
    di = phi[n // 2, n // 2 + 2, n // 2 + 2]   # |r| = sqrt(8) ~ 2.83
    ref = lambda rr: math.exp(-rr ** 2 / (2 * s_t))
    assert abs(ax / peak - ref(r)) < 0.01
    assert abs(di / peak - ref(math.sqrt(8))) < 0.01


def _flat_interface(kappa, M, steps, nz=48, A=0.0625):
    o = Oracle(dict(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), A=A, kappa=kappa, M_psi=M))
    z = np.arange(nz, dtype=float)
    o.set_fields(psi=np.ascontiguousarray(np.tanh((z - (nz - 1) / 2) / 2.0)[:, None, None]))
    o.step(steps)
    psi = o.fields()["psi"][:, 0, 0]
    mu = o.mu()[0][:, 0, 0]
    core = np.abs(psi) < 0.9
    slope = np.polyfit(z[core], np.arctanh(psi[core]), 1)[0]
    f = A / 4 * psi ** 4 - A / 2 * psi ** 2
    sigma = np.sum(f + A / 4) + 0.5 * kappa * np.sum(np.diff(psi) ** 2)
    return psi, mu, 1.0 / slope, sigma


def test_flat_interface_profile_and_uniform_mu():
    """Binary fluid (Eq. free_energy with B=-A): a flat interface relaxes to
    psi = tanh(z/xi), xi = sqrt(2 kappa/A), bulk psi = +-1, uniform chemical
    potential, and tension (excess free energy per area) (2/3) sqrt(2 kappa A)
    (Sec. "Numerical details").  At the paper's kappa the interface is ~1 node
    wide; doubling xi must cut the lattice error about fourfold (second order)."""
    A = 0.0625
    errs = []
    for kappa, M, steps, tol in ((0.04, 1.0, 16000, 0.08), (0.16, 0.3, 40000, 0.03)):
        psi, mu, xi_fit, sigma = _flat_interface(kappa, M, steps)
        assert np.max(np.abs(mu - mu.mean())) < 1e-6
        assert abs(psi[0] + 1) < 1e-5 and abs(psi[-1] - 1) < 1e-5
        xi = math.sqrt(2 * kappa / A)
        s_th = (2.0 / 3.0) * math.sqrt(2 * kappa * A)
        assert abs(xi_fit - xi) < tol * xi
        assert abs(sigma - s_th) < tol * s_th
        errs.append((abs(xi_fit / xi - 1), abs(sigma / s_th - 1)))
    assert errs[1][0] < errs[0][0] / 3 and errs[1][1] < errs[0][1] / 3


def test_laplace_pressure_of_a_cylinder():
    """Laplace law for the free energy of Eq. free_energy: across a curved
    interface the bulk thermodynamic pressure psi mu - f jumps by sigma/R
    (cylinder), with sigma the tension the same lattice model gives a flat
    interface (excess free energy; (2/3) sqrt(2 kappa A) in the continuum,
    Sec. "Numerical details").  Curvature corrections O(xi/R) set the band."""
    n, R0 = 40, 10.0
    A, kappa = 0.0625, 0.04
    o = Oracle(dict(nx=1, ny=n, nz=n, A=A, kappa=kappa, M_psi=1.0))
    y = np.arange(n) - n / 2 + 0.5
    zz, yy = np.meshgrid(y, y, indexing="ij")
    r = np.sqrt(zz ** 2 + yy ** 2)
    psi0 = np.tanh((R0 - r) / 1.2)[:, :, None]
    o.set_fields(psi=np.ascontiguousarray(psi0))
    o.step(6000)
    psi = o.fields()["psi"][:, :, 0]
    mu = o.mu()[0][:, :, 0]
    f = A / 4 * psi ** 4 - A / 2 * psi ** 2
    p = psi * mu - f
    inside = r < R0 - 4
    outside = r > R0 + 5
    dp = p[inside].mean() - p[outside].mean()
    Rm = math.sqrt(np.sum((1 + psi) / 2) / math.pi)
    # flat-interface tension of the same model
    nz = 32
    fo = Oracle(dict(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), A=A, kappa=kappa, M_psi=1.0))
    z = np.arange(nz, dtype=float)
    fo.set_fields(psi=np.ascontiguousarray(np.tanh((z - 15.5) / 2.0)[:, None, None]))
    fo.step(12000)
    pf = fo.fields()["psi"][:, 0, 0]
    sigma = np.sum(A / 4 * pf ** 4 - A / 2 * pf ** 2 + A / 4) + 0.5 * kappa * np.sum(np.diff(pf) ** 2)
    assert abs(dp - sigma / Rm) < 0.07 * sigma / Rm
    assert dp > 0


def test_laplace_pressure_of_a_droplet():
    """Laplace law in three dimensions: across the surface of a droplet of
    psi = +1 in psi = -1 the bulk pressure psi mu - f jumps by 2 sigma / R,
    twice the cylinder's sigma / R, with sigma the flat-interface tension of
    the same lattice model (the cylinder pin computes it).  At equilibrium the
    chemical potential is uniform.  R = 9 with an interface of width 1.13
    leaves curvature corrections of O(xi / R) ~ 12%, which set the band; a
    wrong curvature factor, or a Laplacian that is not isotropic in all three
    directions, falls far outside it."""
    n, R0 = 32, 9.0
    A, kappa = 0.0625, 0.04
    o = Oracle(dict(nx=n, ny=n, nz=n, A=A, kappa=kappa, M_psi=1.0))
    c = np.arange(n) - n / 2 + 0.5
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
    o.set_fields(psi=np.ascontiguousarray(np.tanh((R0 - r) / math.sqrt(2 * kappa / A))))
    o.step(5000)
    psi = o.fields()["psi"]
    mu = o.mu()[0]
    p = psi * mu - (A / 4 * psi ** 4 - A / 2 * psi ** 2)
    inside, outside = r < R0 - 4, r > R0 + 5
    dp = p[inside].mean() - p[outside].mean()
    Rm = (3 * np.sum((1 + psi) / 2) / (4 * math.pi)) ** (1 / 3)
    # the flat-interface tension of the same model, as in the cylinder pin
    nz = 32
    fo = Oracle(dict(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), A=A, kappa=kappa, M_psi=1.0))
    z = np.arange(nz, dtype=float)
    fo.set_fields(psi=np.ascontiguousarray(np.tanh((z - 15.5) / 2.0)[:, None, None]))
    fo.step(12000)
    pf = fo.fields()["psi"][:, 0, 0]
    sigma = np.sum(A / 4 * pf ** 4 - A / 2 * pf ** 2 + A / 4) + 0.5 * kappa * np.sum(np.diff(pf) ** 2)
    assert dp > 0
    assert abs(dp - 2 * sigma / Rm) < 0.15 * 2 * sigma / Rm
    assert abs(mu[inside].mean() - mu[outside].mean()) < 0.05 * abs(mu[inside].mean())


def test_solubility_equilibrium():
    """Solute at equilibrium follows the shifted minimum phi0 = phi_b + E tanh psi
    (Eq. free_energy); averages in the bulk phases are phi_b +- E tanh(1)
    (Fig. 1: +E tanh 1 where psi = +1)."""
    nz, E = 32, 0.4
    o = Oracle(dict(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), E=E, k_d=0.05, M_psi=1.0))
    z = np.arange(nz, dtype=float)
    o.set_fields(psi=np.ascontiguousarray(np.tanh((z - 15.5) / 2.0)[:, None, None]))
    o.step(16000)
    fl = o.fields()
    psi, phi = fl["psi"][:, 0, 0], fl["phi"][:, 0, 0]
    assert np.max(np.abs(phi - E * np.tanh(psi))) < 1e-8
    assert abs(phi[-4:].mean() - E * math.tanh(1.0)) < 1e-6
    assert abs(phi[:4].mean() + E * math.tanh(1.0)) < 1e-6


def test_solubility_ratio_mapping():
    """phi0(+1)/phi0(-1) = r for E = (r-1)/((r+1) tanh 1) with phi_b = 1."""
    for r in (0.25, 0.5, 1.0, 2.0, 4.0):
        E = solubility_E(r, 1.0)
        assert abs((1 + E * math.tanh(1)) / (1 - E * math.tanh(1)) - r) < 1e-12
    assert abs(solubility_E(2.0) - 0.43768) < 1e-5


# --------------------------------------------------------------------------
# particles (Sec. "Particles")
# --------------------------------------------------------------------------

def test_wetting_map_round_trip():
    """cos(theta_c) = [(1+h)^{3/2} - (1-h)^{3/2}]/2 inverted by bisection:
    h(90) = 0, h(180-theta) = -h(theta), and the forward relation returns
    cos(theta)."""
    assert abs(wetting_h(90.0)) < 1e-15
    for th in (0.0, 30.0, 45.0, 60.0, 75.0, 110.0, 150.0):
        h = wetting_h(th)
        assert abs(h + wetting_h(180.0 - th)) < 1e-14
        fwd = 0.5 * ((1 + h) ** 1.5 - (1 - h) ** 1.5)
        assert abs(fwd - math.cos(math.radians(th))) < 1e-13
    assert abs(wetting_h(60.0) - 0.334933) < 1e-6


def test_rotation_about_spin_axis():
    """The unit vector m turns by |Omega| per step about Omega (right hand)."""
    o = Oracle(dict(nx=12, ny=12, nz=12, **PASSIVE))
    w = 0.01
    o.add_particle(pos=(6.1, 6.2, 6.3), R=2.5, m_hat=(1, 0, 0), omega=(0, 0, w), fixed=1)
    o.step(25)
    m = o.particles()[0]["m_hat"]
    assert np.allclose(m, [math.cos(25 * w), math.sin(25 * w), 0.0], atol=1e-13)


def test_comoving_sphere_keeps_uniform_flow():
    """Galilean check of moving bounce-back: a free sphere carried by a
    uniform flow at the flow's velocity reflects equilibrium into equilibrium,
    feels no net force, and keeps its velocity (steps with no covering)."""
    n = 16
    u0 = np.array([0.004, -0.003, 0.002])
    o = Oracle(dict(nx=n, ny=n, nz=n, **PASSIVE))
    fl = dict(u=np.broadcast_to(u0[:, None, None, None], (3, n, n, n)).copy())
    o.set_fields(**fl)
    # placed so that no node lies within 0.04 of the surface during the run
    o.add_particle(pos=(8.4888702, 7.51895608, 7.89738988), R=3.4162875, vel=tuple(u0))
    m0 = o.mask().copy()
    checked = 0
    for _ in range(8):
        o.step(1)
        if not np.array_equal(m0, o.mask()):
            break
        checked += 1
        u = o.fields()["u"]
        fluid = o.mask() == 0
        for a in range(3):
            assert np.max(np.abs(u[a][fluid] - u0[a])) < 1e-15
        P = o.particles()[0]
        assert np.max(np.abs(P["vel"] - u0)) < 1e-15
        assert np.max(np.abs(P["force"])) < 1e-13
    assert checked == 8


def test_fixed_sphere_momentum_exchange():
    """Momentum bookkeeping of bounce-back on links: per step the fluid gains
    N_fluid g and loses exactly the force the particle receives."""
    n = 14
    g = np.array([2e-5, 0, -1e-5])
    rng = np.random.default_rng(3)
    o = Oracle(dict(nx=n, ny=n, nz=n, body_force=tuple(g), **PASSIVE))
    o.set_fields(u=0.01 * rng.uniform(-1, 1, (3, n, n, n)))
    o.add_particle(pos=(7.2, 6.9, 7.4), R=3.6, fixed=1)
    nf = o.fluid_count()
    p_prev = momentum(o.populations(), o.mask())
    for _ in range(6):
        o.step(1)
        p = momentum(o.populations(), o.mask())
        F = o.particles()[0]["force"]
        assert np.allclose(p - p_prev, nf * g - F, atol=1e-12)
        p_prev = p


def test_moving_sphere_momentum_with_covering():
    """A sphere driven at constant velocity covers and uncovers nodes.  The
    fluid momentum plus the total momentum handed to the particle (link
    exchange and covering impulses, which reach the particle one step later)
    is constant."""
    n = 16
    o = Oracle(dict(nx=n, ny=n, nz=n, **PASSIVE))
    o.add_particle(pos=(5.3, 8.2, 7.9), R=3.2, vel=(0.07, 0.0, 0.02), fixed=1)
    p0 = momentum(o.populations(), o.mask())
    given = np.zeros(3)
    changes = 0
    m_prev = o.mask().copy()
    for t in range(60):
        o.step(1)
        given += o.particles()[0]["force"]
        m = o.mask()
        ch = int(np.sum(m != m_prev))
        changes += ch
        m_prev = m.copy()
        if t > 10 and ch == 0:
            p = momentum(o.populations(), m)
            # pending impulses are zero after a step without covering
            assert np.allclose(p - p0, -given, atol=1e-12)
    assert changes > 20


def test_psi_phi_totals_conserved_with_moving_sphere():
    """Without sources (alpha = k_d = 0) the totals of psi and phi are exact
    invariants of the conservative link update; covering/uncovering restores
    them by spreading the difference over the fluid."""
    n = 16
    rng = np.random.default_rng(4)
    o = Oracle(dict(nx=n, ny=n, nz=n, E=0.3, M_psi=0.2, M_phi=0.8))
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


def test_source_sink_balance():
    """Per step the total solute changes by alpha N_active - k_d sum(phi - phi0)
    (Eq. diffusion_reaction with the Janus production of Eq. activity):
    N_active counts fluid nodes next to the surface on the m.(x-X) <= 0 side,
    found here by brute force over the geometry."""
    n = 16
    alpha, kd, E = 1e-3, 2e-3, 0.2
    rng = np.random.default_rng(5)
    X, R, m = np.array([8.3, 7.7, 8.1]), 3.4, np.array([1.0, 2.0, -0.5])
    m = m / np.linalg.norm(m)
    o = Oracle(dict(nx=n, ny=n, nz=n, k_d=kd, E=E))
    o.set_fields(psi=0.2 * rng.uniform(-1, 1, (n, n, n)), phi=0.1 * rng.uniform(0, 1, (n, n, n)))
    o.add_particle(pos=tuple(X), R=R, m_hat=tuple(m), alpha=alpha, fixed=1)
    adj, solid = neighbours_inside((n, n, n), (1, 1, 1), X, R)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    d = [np.where(c - Xa > n / 2, c - Xa - n, np.where(c - Xa < -n / 2, c - Xa + n, c - Xa))
         for c, Xa in ((x, X[0]), (y, X[1]), (z, X[2]))]
    active = adj & (m[0] * d[0] + m[1] * d[1] + m[2] * d[2] <= 0)
    n_act = int(active.sum())
    assert n_act > 10
    for _ in range(3):
        fl = o.fields()
        fluid = ~solid
        sink = kd * np.sum((fl["phi"] - E * np.tanh(fl["psi"]))[fluid])
        before = o.conservation()[2]
        o.step(1)
        after = o.conservation()[2]
        # naive FP64 sums of ~4000 terms: round-off ~1e-12 of the total
        assert abs((after - before) - (alpha * n_act - sink)) < 1e-11


def test_screening_length():
    """Steady solute around a producing sphere decays as exp(-r/l)/r with
    l = sqrt(D/k_d) (Sec. "Results", single phase fluid)."""
    n, R = 24, 3.0
    Cc, Mphi, kd = 0.0625, 0.8, 0.01
    D = Cc * Mphi
    ell = math.sqrt(D / kd)
    X = np.array([12.2, 11.9, 12.1])
    o = Oracle(dict(nx=n, ny=n, nz=n, C=Cc, M_phi=Mphi, k_d=kd, **PASSIVE))
    o.add_particle(pos=tuple(X), R=R, alpha=1e-3, m_hat=(0, 0, 1), fixed=1)
    o.step(900)
    phi = o.fields()["phi"]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - X[0]) ** 2 + (y - X[1]) ** 2 + (z - X[2]) ** 2)
    rs, prof = [], []
    for r0 in np.arange(R + 2.5, R + 7.5, 1.0):
        sel = (r >= r0 - 0.5) & (r < r0 + 0.5)
        rs.append(r[sel].mean())
        prof.append(phi[sel].mean())
    rs, prof = np.array(rs), np.array(prof)
    slope = np.polyfit(rs, np.log(prof * rs), 1)[0]
    assert abs(-1.0 / slope - ell) < 0.1 * ell


@pytest.mark.parametrize("theta,sign", [(60.0, -1), (120.0, +1)])
def test_wetting_sign(theta, sign):
    """theta_c < 90 makes the surface oil-wet (psi < 0 next to it), theta_c > 90
    water-wet (Fig. 2B: theta < 90 stays in oil, theta > 90 in water)."""
    n = 18
    o = Oracle(dict(nx=n, ny=n, nz=n, periodic=(1, 1, 0), M_psi=0.5))
    z = np.arange(n, dtype=float)
    o.set_fields(psi=np.ascontiguousarray(np.broadcast_to(np.tanh((z - 8.6) / 2.0)[:, None, None],
                                                          (n, n, n))))
    X = (9.1, 8.8, 8.6)
    o.add_particle(pos=X, R=4.2, theta_c_deg=theta, fixed=1)
    o.step(400)
    adj, _ = neighbours_inside((n, n, n), (1, 1, 0), X, 4.2)
    surf = o.fields()["psi"][adj].mean()
    assert sign * surf > 0.05


def test_stokes_drag_terminal_velocity():
    """A sphere pulled by a constant force through a periodic array reaches
    U = F K / (6 pi eta R) with Hasimoto's factor
    K = 1 - 2.8373 (R/L) + 4.19 (R/L)^3 (Ladd's bounce-back on links, cited in
    Sec. "Particles").  The hydrodynamic radius of a lattice sphere differs from
    R by a fraction of a node, hence the 15% band."""
    n, R = 24, 3.0
    F = 6e-3
    o = Oracle(dict(nx=n, ny=n, nz=n, **PASSIVE))
    o.add_particle(pos=(12.1, 11.8, 12.3), R=R, ext_force=(F, 0, 0))
    nf = o.fluid_count()
    # an opposite uniform force on the fluid keeps the total momentum at zero
    o2 = Oracle(dict(nx=n, ny=n, nz=n, body_force=(-F / nf, 0, 0), **PASSIVE))
    o2.add_particle(pos=(12.1, 11.8, 12.3), R=R, ext_force=(F, 0, 0))
    o2.step(700)
    fl = o2.fields()
    fluid = o2.mask() == 0
    U = o2.particles()[0]["vel"][0] - fl["u"][0][fluid].mean()
    eta = 1.0 / 6.0
    K = 1 - 2.8373 * (R / n) + 4.19 * (R / n) ** 3
    U_th = F * K / (6 * math.pi * eta * R)
    assert o2.error() == 0
    assert abs(U - U_th) < 0.15 * U_th
    # an off-lattice sphere drifts sideways only slightly
    assert abs(o2.particles()[0]["vel"][1]) < 0.01 * U


@pytest.mark.parametrize("mu", [-0.2, 0.2])
def test_phoretic_propulsion_sign(mu, request):
    """A Janus sphere producing solute on its m.n <= 0 cap moves along +m when
    its mobility is positive (solute-repelled) and along -m when negative
    (V_p ~ -mu grad phi, Sec. "Particles")."""
    U = _phoretic_speed(mu)
    assert np.sign(U) == np.sign(mu) and abs(U) > 1e-6


def _phoretic_speed(mu, steps=250):
    n, R = 20, 3.0
    m = np.array([0.0, 0.6, 0.8])
    o = Oracle(dict(nx=n, ny=n, nz=n, C=0.0625, M_phi=0.8, k_d=1e-3, **PASSIVE))
    o.add_particle(pos=(10.2, 9.8, 10.1), R=R, m_hat=tuple(m), alpha=1e-2,
                   mu_plus=mu, mu_minus=mu)
    o.step(steps)
    P = o.particles()[0]
    return float(np.dot(P["vel"], P["m_hat"]))


def test_phoretic_speed_linear_in_mobility():
    """At low Peclet number the propulsion speed is linear in mu_+ + mu_-
    (Eq. Vp; Fig. 3B)."""
    mus = np.array([0.05, 0.1, 0.15, 0.2])
    v = np.array([_phoretic_speed(m, steps=150) for m in mus])
    slope, icpt = np.polyfit(mus, v, 1)
    pred = slope * mus + icpt
    r2 = 1 - np.sum((v - pred) ** 2) / np.sum((v - v.mean()) ** 2)
    assert r2 > 0.99 and slope > 0
    assert abs(icpt) < 0.05 * abs(v).max()


def test_total_momentum_with_free_sphere_and_chemical_force():
    """Fluid plus particle momentum is an exact invariant of the step in a
    periodic box: bounce-back uses the velocity the implicit update solves
    for, and the chemical stress flux through each boundary link reaches the
    particle (covering impulses reach it one step later, so the check runs
    after steps without covering)."""
    n, R = 20, 3.6
    z = np.arange(n, dtype=float)
    o = Oracle(dict(nx=n, ny=n, nz=n, E=0.3, M_psi=0.2, k_d=0.0))
    psi = np.ascontiguousarray(np.broadcast_to(np.tanh((z - 10.3) / 1.5)[:, None, None], (n, n, n)))
    o.set_fields(psi=psi, phi=0.1 + 0.05 * np.cos(2 * np.pi * z / n)[:, None, None] * np.ones((n, n, n)))
    o.add_particle(pos=(9.7, 10.2, 9.1), R=R, vel=(0.004, -0.002, 0.006), omega=(0.0, 0.001, 0.0),
                   theta_c_deg=70.0, mu_plus=0.1, mu_minus=0.2, alpha=1e-3, m_hat=(0, 0, 1))
    M = (4.0 / 3.0) * math.pi * R ** 3
    P0 = momentum(o.populations(), o.mask()) + M * o.particles()[0]["vel"]
    m_prev = o.mask().copy()
    checked = changed = 0
    for _ in range(80):
        o.step(1)
        m = o.mask()
        if np.array_equal(m, m_prev):
            P = momentum(o.populations(), m) + M * o.particles()[0]["vel"]
            assert np.max(np.abs(P - P0)) < 1e-12
            checked += 1
        else:
            changed += 1
        m_prev = m.copy()
    assert checked > 10 and changed > 3


def _capillary_force(dz, n=20, nz=32, R=5.0):
    o = Oracle(dict(nx=n, ny=n, nz=nz, periodic=(1, 1, 0), M_psi=0.5))
    z = np.arange(nz, dtype=float)
    o.set_fields(psi=np.ascontiguousarray(np.broadcast_to(np.tanh((z - 15.5) / 1.13)[:, None, None],
                                                          (nz, n, n))))
    o.add_particle(pos=(10.2, 9.9, 15.5 + dz), R=R, theta_c_deg=90.0, fixed=1)
    o.step(500)
    return o.particles()[0]["force"][2]


def test_capillary_restoring_force():
    """A neutrally wetting sphere (theta_c = 90) displaced by dz from a flat
    interface is pulled back (trapping, Fig. 2B; Sec. "Inactive Janus
    particles").  For an undeformed interface the force is -2 pi sigma dz;
    the meniscus of a held sphere lowers it, so the pin is the sign, the exact
    antisymmetry of the mirror-symmetric box, and a band of 0.35-1 of that
    value (sigma = 0.0454, the lattice tension at kappa = 0.04)."""
    up, down = _capillary_force(1.5), _capillary_force(-1.5)
    assert up < 0 < down
    assert abs(up + down) < 1e-9 * abs(up)
    rigid = 2 * math.pi * 0.0454 * 1.5
    assert 0.35 * rigid < abs(up) < 1.0 * rigid


def test_surface_flux_matches_comoving_fluid():
    """A uniform solute in a fluid moving at U past a sphere moving at U: the
    advective flux into the surface, c.u_b g(x) (reading C7b), equals what
    the donor-cell flux to a fluid neighbour moving at U would be, so phi
    stays uniform over the fluid and its total stays; a dropped or
    mis-signed surface flux leaves a ring around the sphere."""
    n = 16
    U = np.array([0.02, -0.01, 0.015])
    o = Oracle(dict(nx=n, ny=n, nz=n, A=0.0, kappa=0.0, E=0.0, phi_b=1.0, k_d=0.0, thermo_force=0))
    u = np.broadcast_to(U[:, None, None, None], (3, n, n, n)).copy()
    o.set_fields(u=u, phi=np.ones((n, n, n)))
    o.add_particle(pos=(8.3, 7.9, 8.1), R=3.3, vel=tuple(U), fixed=1, alpha=0.0, mu_plus=0.0, mu_minus=0.0,
                   theta_c_deg=90.0, m_hat=(0, 0, 1))
    tot0 = o.conservation()[2]
    for _ in range(4):
        o.step(1)
        phi = o.fields()["phi"][o.mask() == 0]
        assert np.max(phi) - np.min(phi) < 1e-13
        assert abs(o.conservation()[2] - tot0) < 1e-12 * n ** 3
