"""An independent NumPy transcription of one lattice step, for the 8^3
brute-force pin of the oracle.

Written from the model and its stated readings only (D3Q19 BGK tau with Guo
forcing; the chemical potentials of Eq. chem_potentials and the pressure
tensor of Eq. free_energy with wetting ghosts; the force g - div P in link
form; Ladd's moving bounce-back with the phoretic slip of Eq. MuJ; the
Nguyen-Ladd implicit particle update; conservative finite-difference
transport with donor-cell advection, the flux into moving surfaces, Janus
production of Eq. activity and the sink; covering and uncovering with the
uniform correction of the psi and phi totals).  It imports nothing from the
oracle and shares no code with it: whole-lattice array operations through a
neighbour table, with Python loops only over the links that touch a sphere.
Slow, small boxes only.
"""
from __future__ import annotations

import math

import numpy as np

# D3Q19 in the documented order
CV = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.int64)
CF = CV.astype(np.float64)
WQ = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
OPP = np.array([int(np.nonzero((CV == -CV[i]).all(axis=1))[0][0]) for i in range(19)])


def wetting_h_from_angle(theta_deg: float) -> float:
    """h with cos(theta) = [(1+h)^{3/2} - (1-h)^{3/2}]/2 (Sec. "Particles"),
    by Newton's method from h = 0 (the relation is monotonic on [-1, 1])."""
    target = math.cos(math.radians(theta_deg))
    h = 0.0
    for _ in range(200):
        g = 0.5 * ((1 + h) ** 1.5 - (1 - h) ** 1.5) - target
        dg = 0.75 * ((1 + h) ** 0.5 + (1 - h) ** 0.5)
        step = g / dg
        h = min(1.0, max(-1.0, h - step))
        if abs(step) < 1e-17:
            break
    return h


class Sphere:
    def __init__(self, pos, R, m_hat, rho_p=1.0, alpha=0.0, mu_plus=0.0, mu_minus=0.0, H=0.0,
                 vel=(0, 0, 0), omega=(0, 0, 0), ext_force=(0, 0, 0), ext_torque=(0, 0, 0), fixed=0):
        self.X = np.array(pos, dtype=np.float64)
        m = np.array(m_hat, dtype=np.float64)
        self.m = m / math.sqrt(float(m @ m))
        self.R = float(R)
        self.M = rho_p * 4.0 / 3.0 * math.pi * R ** 3
        self.I = 0.4 * self.M * R * R
        self.alpha, self.mu_p, self.mu_m, self.H = alpha, mu_plus, mu_minus, H
        self.V = np.array(list(vel) + list(omega), dtype=np.float64)
        self.ext = np.array(list(ext_force) + list(ext_torque), dtype=np.float64)
        self.imp = np.zeros(6)
        self.fixed = bool(fixed)
        self.force = np.zeros(3)
        self.torque = np.zeros(3)


class BruteBox:
    def __init__(self, nx, ny, nz, periodic, tau=1.0, rho0=1.0, body_force=(0, 0, 0), A=0.0625, kappa=0.04,
                 M_psi=0.1, C=0.0625, M_phi=1.6, E=0.0, phi_b=0.0, k_d=0.0):
        self.L = np.array([nx, ny, nz])
        self.per = tuple(bool(p) for p in periodic)
        self.N = nx * ny * nz
        self.tau, self.rho0 = tau, rho0
        self.g = np.array(body_force, dtype=np.float64)
        self.A, self.kappa, self.Mpsi, self.C, self.Mphi = A, kappa, M_psi, C, M_phi
        self.E, self.phib, self.kd = E, phi_b, k_d
        n = np.arange(self.N)
        self.xyz = np.stack([n % nx, (n // nx) % ny, n // (nx * ny)])   # [3][N]
        # neighbour table: nb[i][n] = index of x + c_i, -1 beyond a wall
        self.nb = np.empty((19, self.N), dtype=np.int64)
        for i in range(19):
            c = self.xyz + CV[i][:, None]
            ok = np.ones(self.N, dtype=bool)
            for a in range(3):
                if self.per[a]:
                    c[a] %= self.L[a]
                else:
                    ok &= (c[a] >= 0) & (c[a] < self.L[a])
            self.nb[i] = np.where(ok, c[0] + nx * (c[1] + ny * c[2]), -1)
        self.spheres: list[Sphere] = []
        self.mask = np.zeros(self.N, dtype=np.int64)
        self.f = np.zeros((19, self.N))
        self.u = np.zeros((3, self.N))
        self.psi = np.zeros(self.N)
        self.phi = np.zeros(self.N)

    # ---- set-up --------------------------------------------------------
    def set_fields(self, rho, u, psi, phi):
        rho = np.asarray(rho, dtype=np.float64).reshape(-1)
        u = np.asarray(u, dtype=np.float64).reshape(3, -1)
        self.psi = np.asarray(psi, dtype=np.float64).reshape(-1).copy()
        self.phi = np.asarray(phi, dtype=np.float64).reshape(-1).copy()
        self.u = u.copy()
        self.f = self._feq(rho, u)

    def add_sphere(self, sp: Sphere):
        self.spheres.append(sp)
        k = len(self.spheres)
        inside = (self.mask == 0) & self._inside(sp, self.xyz)
        self.mask[inside] = k
        self.f[:, inside] = 0.0
        self.u[:, inside] = 0.0
        self.psi[inside] = 0.0
        self.phi[inside] = 0.0

    # ---- pieces of the model -------------------------------------------
    @staticmethod
    def _feq(rho, u):
        cu = CF @ u                                   # [19][N]
        uu = (u * u).sum(axis=0)
        return WQ[:, None] * rho[None, :] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu[None, :])

    def _offset(self, sp, pts):
        """x - X with the periodic minimum image, pts [3][...]."""
        d = np.empty(pts.shape)
        for a in range(3):
            v = pts[a] - sp.X[a]
            if self.per[a]:
                Lh = 0.5 * self.L[a]
                v = np.where(v > Lh, v - self.L[a], np.where(v < -Lh, v + self.L[a], v))
            d[a] = v
        return d

    def _inside(self, sp, pts):
        d = self._offset(sp, pts.astype(np.float64))
        return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < sp.R * sp.R

    def _owner(self):
        own = np.zeros(self.N, dtype=np.int64)
        for k, sp in enumerate(self.spheres):
            own = np.where((own == 0) & self._inside(sp, self.xyz), k + 1, own)
        return own

    def _links(self):
        """Boundary links (n, i, k): fluid node n whose neighbour n + c_i is
        inside sphere k (0-based), in node order, then direction order."""
        out = []
        for n in np.nonzero(self.mask == 0)[0]:
            for i in range(1, 19):
                m = self.nb[i, n]
                if m >= 0 and self.mask[m]:
                    out.append((int(n), i, int(self.mask[m]) - 1))
        return out

    def _grad_phi(self, n):
        own = self.phi[n]
        g = np.zeros(3)
        for i in range(1, 19):
            m = self.nb[i, n]
            v = own if (m < 0 or self.mask[m]) else self.phi[m]
            g += WQ[i] * CF[i] * v
        return 3.0 * g

    def _link_geometry(self, n, i, sp):
        r = self._offset(sp, self.xyz[:, n].astype(np.float64)) + 0.5 * CF[i]
        return r, r / math.sqrt(float(r @ r))

    def _boundary_velocity(self, n, i, sp):
        """u_b = U + Omega x r_b + v_s, v_s = mu (1 - n n).grad phi (Eq. MuJ)."""
        r, nh = self._link_geometry(n, i, sp)
        mu = sp.mu_m if float(sp.m @ r) <= 0.0 else sp.mu_p
        gp = self._grad_phi(n)
        vs = mu * (gp - nh * float(nh @ gp))
        ub = sp.V[:3] + np.cross(sp.V[3:], r) + vs
        return r, ub, vs

    # ---- one step ------------------------------------------------------
    def step(self):
        N = self.N
        fluid = self.mask == 0
        links = self._links()
        # S1: chemical potentials and pressure tensor, neighbour values with
        # ghosts (wall: own value; sphere: own + (H/kappa) c.n)
        vals = np.empty((19, N))
        vals[0] = self.psi
        for i in range(1, 19):
            m = self.nb[i]
            vals[i] = np.where(m >= 0, self.psi[np.maximum(m, 0)], self.psi)
            solid = (m >= 0) & (self.mask[np.maximum(m, 0)] != 0)
            vals[i] = np.where(solid, self.psi, vals[i])
        for n, i, k in links:
            sp = self.spheres[k]
            _, nh = self._link_geometry(n, i, sp)
            vals[i, n] = self.psi[n] + (sp.H / self.kappa) * float(CF[i] @ nh)
        lap = 6.0 * (WQ[1:, None] * (vals[1:] - self.psi[None, :])).sum(axis=0)
        gpsi = 3.0 * (CF[1:].T @ (WQ[1:, None] * vals[1:]))            # [3][N]
        phi0 = self.phib + self.E * np.tanh(self.psi)
        dph = self.phi - phi0
        mu_psi = self.A * (self.psi ** 3 - self.psi) - self.kappa * lap - self.C * self.E * dph / np.cosh(self.psi) ** 2
        mu_phi = self.C * dph
        fden = 0.25 * self.A * self.psi ** 4 - 0.5 * self.A * self.psi ** 2 + 0.5 * self.C * dph * dph
        iso = self.psi * mu_psi + self.phi * mu_phi - fden - 0.5 * self.kappa * (gpsi * gpsi).sum(axis=0)
        P = np.einsum("an,bn->abn", gpsi, gpsi) * self.kappa + np.eye(3)[:, :, None] * iso[None, None, :]
        mu_psi = np.where(fluid, mu_psi, 0.0)
        mu_phi = np.where(fluid, mu_phi, 0.0)
        P = np.where(fluid[None, None, :], P, 0.0)

        # S5 + S6a: link sums and the implicit velocity update
        F0 = [np.zeros(6) for _ in self.spheres]
        Z = [np.zeros((6, 6)) for _ in self.spheres]
        for n, i, k in links:
            sp = self.spheres[k]
            r, nh = self._link_geometry(n, i, sp)
            mu = sp.mu_m if float(sp.m @ r) <= 0.0 else sp.mu_p
            gp = self._grad_phi(n)
            vs = mu * (gp - nh * float(nh @ gp))
            dP = CF[i] * (2.0 * self.f[i, n] - 6.0 * WQ[i] * self.rho0 * float(CF[i] @ vs))
            dP = dP + 6.0 * WQ[i] * (P[:, :, n] @ CF[i])
            F0[k][:3] += dP
            F0[k][3:] += np.cross(r, dP)
            g6 = np.concatenate([CF[i], np.cross(r, CF[i])])
            Z[k] += 6.0 * WQ[i] * self.rho0 * np.outer(g6, g6)
        for k, sp in enumerate(self.spheres):
            rhs = F0[k] + sp.imp + sp.ext
            if not sp.fixed:
                Md = np.array([sp.M] * 3 + [sp.I] * 3)
                sp.V = np.linalg.solve(np.diag(Md) + Z[k], Md * sp.V + rhs)
            res = rhs - Z[k] @ sp.V
            sp.force, sp.torque = res[:3].copy(), res[3:].copy()
            sp.imp = np.zeros(6)

        # S2: force g - 6 sum_i w_i [(P(x) + P~_i)/2] . c_i
        Fq = np.repeat(self.g[:, None], N, axis=1)
        div = np.zeros((3, N))
        for i in range(1, 19):
            m = self.nb[i]
            other_ok = (m >= 0) & (self.mask[np.maximum(m, 0)] == 0)
            Pn = np.where(other_ok[None, None, :], P[:, :, np.maximum(m, 0)], P)
            div += WQ[i] * np.einsum("abn,b->an", 0.5 * (P + Pn), CF[i])
        Fq = Fq - 6.0 * div

        # S3: pull streaming with bounce-back, BGK + Guo
        fl = np.empty((19, N))
        fl[0] = self.f[0]
        for j in range(1, 19):
            i = OPP[j]
            src = self.nb[i]                    # x - c_j = x + c_i
            fl[j] = np.where(src >= 0, self.f[j, np.maximum(src, 0)], self.f[i])
        for n, i, k in links:                   # particle link x -> x + c_i
            j = OPP[i]
            _, ub, _ = self._boundary_velocity(n, i, self.spheres[k])
            fl[j, n] = self.f[i, n] - 6.0 * WQ[i] * self.rho0 * float(CF[i] @ ub)
        rho = fl.sum(axis=0)
        u = (CF.T @ fl + 0.5 * Fq) / np.where(fluid, rho, 1.0)
        feq = self._feq(rho, u)
        cu = CF @ u
        guo = WQ[:, None] * (3.0 * (CF @ Fq - (u * Fq).sum(axis=0)[None, :]) + 9.0 * cu * (CF @ Fq))
        fnew = fl - (fl - feq) / self.tau + (1.0 - 0.5 / self.tau) * guo
        self.f = np.where(fluid[None, :], fnew, 0.0)
        self.u = np.where(fluid[None, :], u, 0.0)

        # S4: transport of psi and phi
        dps = np.zeros(N)
        dphs = np.zeros(N)
        for i in range(1, 19):
            m = self.nb[i]
            mm = np.maximum(m, 0)
            ff = (m >= 0) & (self.mask[mm] == 0)
            ubar = 0.5 * (CF[i] @ self.u + CF[i] @ self.u[:, mm])
            ap = np.where(ubar > 0, ubar * self.psi, ubar * self.psi[mm])
            ah = np.where(ubar > 0, ubar * self.phi, ubar * self.phi[mm])
            dps += np.where(ff, WQ[i] * (self.Mpsi * (mu_psi[mm] - mu_psi) - ap), 0.0)
            dphs += np.where(ff, WQ[i] * (self.Mphi * (mu_phi[mm] - mu_phi) - ah), 0.0)
        carried = np.zeros(2)
        adjacent = [set() for _ in range(N)]
        for n, i, k in links:
            _, ub, _ = self._boundary_velocity(n, i, self.spheres[k])
            cub = float(CF[i] @ ub)
            dps[n] -= WQ[i] * cub * self.psi[n]
            dphs[n] -= WQ[i] * cub * self.phi[n]
            carried += 6.0 * WQ[i] * cub * np.array([self.psi[n], self.phi[n]])
            adjacent[n].add(k)
        psi_new = self.psi + 6.0 * dps
        phi_new = self.phi + 6.0 * dphs - self.kd * (self.phi - phi0)
        for n in range(N):
            for k in sorted(adjacent[n]):
                sp = self.spheres[k]
                if float(sp.m @ self._offset(sp, self.xyz[:, n].astype(np.float64))) <= 0.0:
                    phi_new[n] += sp.alpha
        self.psi = np.where(fluid, psi_new, 0.0)
        self.phi = np.where(fluid, phi_new, 0.0)

        # S6b: move and rotate
        for sp in self.spheres:
            X = sp.X + sp.V[:3]
            for a in range(3):
                if self.per[a]:
                    if X[a] >= self.L[a]:
                        X[a] -= self.L[a]
                    elif X[a] < 0:
                        X[a] += self.L[a]
            sp.X = X
            w = sp.V[3:]
            ang = math.sqrt(float(w @ w))
            if ang > 0:
                kax = w / ang
                m = sp.m
                mn = m * math.cos(ang) + np.cross(kax, m) * math.sin(ang) + kax * float(kax @ m) * (1 - math.cos(ang))
                sp.m = mn / math.sqrt(float(mn @ mn))

        # S7: covering and uncovering, then the uniform correction
        new = self._owner()
        deficit = carried.copy()
        old = self.mask
        changed = 0
        for n in np.nonzero(old != new)[0]:
            o, q = old[n], new[n]
            p = self.xyz[:, n].astype(np.float64)
            if o == 0:
                sp = self.spheres[q - 1]
                j = CF.T @ self.f[:, n]
                r = self._offset(sp, p)
                sp.imp += np.concatenate([j, np.cross(r, j)])
                deficit += np.array([self.psi[n], self.phi[n]])
                self.psi[n] = self.phi[n] = 0.0
                self.f[:, n] = 0.0
                self.u[:, n] = 0.0
                changed -= 1
            elif q == 0:
                sp = self.spheres[o - 1]
                nbrs = [m for m in self.nb[1:, n] if m >= 0 and old[m] == 0 and new[m] == 0]
                rb = np.mean([self.f[:, m].sum() for m in nbrs])
                pb = np.mean([self.psi[m] for m in nbrs])
                hb = np.mean([self.phi[m] for m in nbrs])
                r = self._offset(sp, p)
                ub = sp.V[:3] + np.cross(sp.V[3:], r)
                self.f[:, n] = self._feq(np.array([rb]), ub[:, None])[:, 0]
                self.u[:, n] = ub
                sp.imp -= np.concatenate([rb * ub, np.cross(r, rb * ub)])
                self.psi[n], self.phi[n] = pb, hb
                deficit -= np.array([pb, hb])
                changed += 1
            else:
                raise RuntimeError("node passed directly between two spheres")
        self.mask = new
        nfl = int(np.count_nonzero(new == 0))
        fl_new = new == 0
        self.psi = np.where(fl_new, self.psi + deficit[0] / nfl, 0.0)
        self.phi = np.where(fl_new, self.phi + deficit[1] / nfl, 0.0)
