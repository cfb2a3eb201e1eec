/*
 * lbref.c -- plain FP64 CPU oracle of the self-diffusiophoretic lattice
 * Boltzmann time step.  TEST INFRASTRUCTURE ONLY (see lbref.h): it is the
 * slow definition the CUDA path is compared with, written node by node in the
 * order the model states it, with no blocking or fusion.
 *
 * One step, in order (the paper gives the model as PDEs; the discrete reading
 * of each step is stated where it is used):
 *   S1  chemical potentials mu_psi, mu_phi (Eq. chem_potentials) and the
 *       chemical pressure tensor P of the free energy (Eq. free_energy)
 *   S5  momentum exchange sums per particle (bounce-back and chemical stress)
 *   S6a implicit particle velocity update
 *   S2  force on the fluid, g - div P (reading of the coupling, whose
 *       continuum value is -psi grad mu_psi - phi grad mu_phi + g)
 *   S3  D3Q19 pull streaming, halfway bounce-back on walls, moving bounce-back
 *       on particle links with phoretic slip          (Sec. Particles, Eq. for v_s)
 *       then BGK collision with Guo forcing
 *   S4  explicit conservative update of psi and phi   (Eq. diffusion_reaction)
 *       with Janus production (Eq. activity) and the sink k_d (phi - phi0);
 *       or, with scalar_scheme = 1, the same equations by lattice Boltzmann:
 *       D3Q7 distributions collide to an equilibrium built on the chemical
 *       potential and stream with bounce-back at walls and moving surfaces
 *   S6b particle translation and rotation
 *   S7  covering / uncovering of nodes swept by moving particles, and the
 *       uniform correction that keeps the psi and phi totals exact
 *
 * Built with -ffp-contract=off so that no multiply-add is fused; the
 * geometric decisions (solid or fluid, active or inactive) are then taken with
 * exactly the products and sums written here.
 *
 * Threads (OpenMP, when the compiler has it): the node loops whose nodes are
 * independent run in parallel over z.  Every sum over nodes (particle link
 * sums, the flux into the moving surfaces, covering) is taken by one thread in
 * the node order x fastest, then y, then z, so the result is bit-identical for
 * any thread count.
 *
 * Pins (tests/test_oracle_*.py): every function below is checked against a
 * closed form, an invariant, a special case or an independent per-node
 * transcription of the step on 8^3 boxes.  Parity unpinned: the magnitude of
 * the phoretic speed (the continuum relation of Sec. Particles ties the slip
 * to a surface flux, not to the lattice production rate, so only its sign and
 * linearity in the mobility are pinned), and the refill rule of an uncovered
 * node in step_cover (means of the neighbours), a reading held only by the
 * exact totals and momentum it keeps.
 */
#include "lbref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REF_MAXP 255

/* D3Q19 velocity set and weights (order documented in lbref.h). */
static const int CX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W[19] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

typedef struct {
    double X[3], U[3], Om[3], m[3];
    double R, R2, M, I, alpha, mu_p, mu_m, H;
    double ext_f[3], ext_t[3];
    int fixed;
    /* link sums of the current step */
    double F0[3], T0[3], zeta[6][6];
    /* impulses of covering/uncovering, applied in the next step */
    double imp_f[3], imp_t[3];
    double force[3], torque[3];
} ref_part;

struct ref_sim {
    ref_params p;
    long N;
    double* f;    /* [19][N] post-collision populations */
    double* fn;   /* work buffer */
    double *psi, *phi, *mupsi, *muphi, *u, *psin, *phin;
    double* pt;   /* [6][N] chemical pressure tensor xx yy zz xy xz yz */
    unsigned char *mask, *maskn;
    unsigned char* lk;   /* [N] 1: fluid node with a particle neighbour (work flags) */
    int np;
    ref_part part[REF_MAXP];
    long nfluid;
    int err;
    double wall_psi, wall_phi; /* psi, phi carried into the particles this step */
    double* h;  /* [14][N] scheme 1: D3Q7 distributions of psi (0..6), phi (7..13) */
    double* hs; /* [14][N] their post-collision values */
};

/* D3Q7 (directions 0..6 of the D3Q19 table), weights 1/4 and 1/8, c_s^2 = 1/4. */
static const double W7[7] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

static long nidx(const ref_sim* s, int x, int y, int z)
{
    return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * (long)z);
}

/* Neighbour of node (x,y,z) along (dx,dy,dz), wrapped on periodic axes;
 * -1 when it lies beyond a wall. */
static long nbr(const ref_sim* s, int x, int y, int z, int dx, int dy, int dz)
{
    int n[3] = {s->p.nx, s->p.ny, s->p.nz};
    int c[3] = {x + dx, y + dy, z + dz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0) {
            if (!s->p.periodic[a]) return -1;
            c[a] += n[a];
        } else if (c[a] >= n[a]) {
            if (!s->p.periodic[a]) return -1;
            c[a] -= n[a];
        }
    }
    return nidx(s, c[0], c[1], c[2]);
}

/* Minimum-image component of d on an axis of length L. */
static double mimg(double d, int L, int periodic)
{
    if (periodic) {
        if (d > 0.5 * L)
            d -= L;
        else if (d < -0.5 * L)
            d += L;
    }
    return d;
}

/* Node-to-centre offset r = x - X (minimum image). */
static void node_offset(const ref_sim* s, const ref_part* P, int x, int y, int z, double r[3])
{
    r[0] = mimg((double)x - P->X[0], s->p.nx, s->p.periodic[0]);
    r[1] = mimg((double)y - P->X[1], s->p.ny, s->p.periodic[1]);
    r[2] = mimg((double)z - P->X[2], s->p.nz, s->p.periodic[2]);
}

/* A node is inside a sphere when |x - X|^2 < R^2 (strict). */
static int inside(const ref_sim* s, const ref_part* P, int x, int y, int z)
{
    double r[3];
    node_offset(s, P, x, y, z, r);
    double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    return d2 < P->R2;
}

/* Mask value of a node: 0 = fluid, k+1 = inside particle k (first match). */
static unsigned char owner(const ref_sim* s, int x, int y, int z)
{
    for (int k = 0; k < s->np; ++k)
        if (inside(s, &s->part[k], x, y, z)) return (unsigned char)(k + 1);
    return 0;
}

/* ------------------------------------------------------------------ */
/* lattice Boltzmann pieces                                            */
/* ------------------------------------------------------------------ */

/* Second-order equilibrium, f_i^eq = w_i rho [1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u^2]. */
static double feq(int i, double rho, const double u[3])
{
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

static double phi0_of(const ref_sim* s, double psi) { return s->p.phi_b + s->p.E * tanh(psi); }

/* Offset of the link midpoint from the centre: r_b = (x - X) + c_i / 2. */
static void link_offset(const ref_sim* s, const ref_part* P, int x, int y, int z, int i, double r[3])
{
    node_offset(s, P, x, y, z, r);
    r[0] += 0.5 * CX[i];
    r[1] += 0.5 * CY[i];
    r[2] += 0.5 * CZ[i];
}

/* Isotropic gradient of phi at a fluid node, 3 sum_i w_i c_i phi(x+c_i), with
 * the value at x standing in for solid and wall neighbours (no flux). */
static void grad_phi(const ref_sim* s, int x, int y, int z, double g[3])
{
    long n = nidx(s, x, y, z);
    double own = s->phi[n];
    g[0] = g[1] = g[2] = 0.0;
    for (int i = 1; i < 19; ++i) {
        long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
        double v = (m < 0 || s->mask[m]) ? own : s->phi[m];
        g[0] += W[i] * CX[i] * v;
        g[1] += W[i] * CY[i] * v;
        g[2] += W[i] * CZ[i] * v;
    }
    g[0] *= 3.0;
    g[1] *= 3.0;
    g[2] *= 3.0;
}

/* Velocity of the boundary at the midpoint of link x -> x+c_i on particle P:
 * rigid motion plus phoretic slip v_s = mu (1 - n n) . grad phi, with the
 * Janus mobility mu_- where m.n <= 0 and mu_+ elsewhere (Sec. Particles). */
static void link_velocity(const ref_sim* s, const ref_part* P, int x, int y, int z, int i,
                          double r[3], double ub[3], double vs[3])
{
    link_offset(s, P, x, y, z, i, r);
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double nh[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    double side = P->m[0] * r[0] + P->m[1] * r[1] + P->m[2] * r[2];
    double mu = (side <= 0.0) ? P->mu_m : P->mu_p;
    double g[3];
    grad_phi(s, x, y, z, g);
    double ng = nh[0] * g[0] + nh[1] * g[1] + nh[2] * g[2];
    for (int a = 0; a < 3; ++a) vs[a] = mu * (g[a] - nh[a] * ng);
    ub[0] = P->U[0] + (P->Om[1] * r[2] - P->Om[2] * r[1]) + vs[0];
    ub[1] = P->U[1] + (P->Om[2] * r[0] - P->Om[0] * r[2]) + vs[1];
    ub[2] = P->U[2] + (P->Om[0] * r[1] - P->Om[1] * r[0]) + vs[2];
}

/* ------------------------------------------------------------------ */
/* S1: chemical potentials (Eq. chem_potentials) and the chemical      */
/* pressure tensor of the free energy (Eq. free_energy)                */
/* ------------------------------------------------------------------ */

static void step_mu(ref_sim* s)
{
    const ref_params* p = &s->p;
    const long N = s->N;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                if (s->mask[n]) {
                    s->mupsi[n] = 0.0;
                    s->muphi[n] = 0.0;
                    for (int k = 0; k < 6; ++k) s->pt[k * N + n] = 0.0;
                    continue;
                }
                double ps = s->psi[n], ph = s->phi[n];
                /* isotropic Laplacian 6 sum_i w_i (psi(x+c_i) - psi(x)) and
                 * gradient 3 sum_i w_i c_i psi(x+c_i); a solid neighbour
                 * carries the wetting ghost psi(x) + (H/kappa) c_i.n_hat, a
                 * wall neighbour psi(x). */
                double lap = 0.0, g[3] = {0.0, 0.0, 0.0};
                for (int i = 1; i < 19; ++i) {
                    long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                    double v;
                    if (m < 0) {
                        v = ps;
                    } else if (s->mask[m]) {
                        const ref_part* P = &s->part[s->mask[m] - 1];
                        if (P->H != 0.0) {
                            double r[3];
                            link_offset(s, P, x, y, z, i, r);
                            double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                            double cn = (CX[i] * r[0] + CY[i] * r[1] + CZ[i] * r[2]) / rn;
                            v = ps + (P->H / p->kappa) * cn;
                        } else {
                            v = ps;
                        }
                    } else {
                        v = s->psi[m];
                    }
                    lap += W[i] * (v - ps);
                    g[0] += W[i] * CX[i] * v;
                    g[1] += W[i] * CY[i] * v;
                    g[2] += W[i] * CZ[i] * v;
                }
                lap *= 6.0;
                g[0] *= 3.0;
                g[1] *= 3.0;
                g[2] *= 3.0;
                double dphi = ph - phi0_of(s, ps);
                double ch = cosh(ps);
                double mph = p->C * dphi;
                double mps = p->A * (ps * ps * ps - ps) - p->kappa * lap - p->C * p->E * dphi / (ch * ch);
                s->muphi[n] = mph;
                s->mupsi[n] = mps;
                /* P = [psi mu_psi + phi mu_phi - f - kappa |grad psi|^2 / 2] I
                 *     + kappa grad psi grad psi,
                 * f = A psi^4/4 - A psi^2/2 + C (phi - phi0)^2 / 2; its
                 * divergence is psi grad mu_psi + phi grad mu_phi. */
                double f = 0.25 * p->A * ps * ps * ps * ps - 0.5 * p->A * ps * ps + 0.5 * p->C * dphi * dphi;
                double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
                double piso = ps * mps + ph * mph - f - 0.5 * p->kappa * g2;
                s->pt[0 * N + n] = piso + p->kappa * g[0] * g[0];
                s->pt[1 * N + n] = piso + p->kappa * g[1] * g[1];
                s->pt[2 * N + n] = piso + p->kappa * g[2] * g[2];
                s->pt[3 * N + n] = p->kappa * g[0] * g[1];
                s->pt[4 * N + n] = p->kappa * g[0] * g[2];
                s->pt[5 * N + n] = p->kappa * g[1] * g[2];
            }
}

/* P(x) . c for the tensor stored at node n (components xx yy zz xy xz yz). */
static void pt_dot(const ref_sim* s, long n, const double c[3], double out[3])
{
    const long N = s->N;
    double xx = s->pt[n], yy = s->pt[N + n], zz = s->pt[2 * N + n];
    double xy = s->pt[3 * N + n], xz = s->pt[4 * N + n], yz = s->pt[5 * N + n];
    out[0] = xx * c[0] + xy * c[1] + xz * c[2];
    out[1] = xy * c[0] + yy * c[1] + yz * c[2];
    out[2] = xz * c[0] + yz * c[1] + zz * c[2];
}

/* ------------------------------------------------------------------ */
/* S5 + S6a: momentum exchange sums and the implicit velocity update   */
/* ------------------------------------------------------------------ */

/* lk[n] = 1 for the fluid nodes with a neighbour inside a particle (the nodes
 * whose links the sums below visit, in node order). */
static void mark_particle_neighbours(ref_sim* s)
{
    const ref_params* p = &s->p;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                unsigned char f = 0;
                if (!s->mask[n])
                    for (int i = 1; i < 19 && !f; ++i) {
                        long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                        f = (unsigned char)(m >= 0 && s->mask[m]);
                    }
                s->lk[n] = f;
            }
}

/* Gaussian elimination with partial pivoting on a 6x6 system. */
static int solve6(double A[6][6], double b[6], double x[6])
{
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < 6; ++k) {
                double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < 6; ++r) {
            double l = A[r][c] / A[c][c];
            for (int k = c; k < 6; ++k) A[r][k] -= l * A[c][k];
            b[r] -= l * b[c];
        }
    }
    for (int r = 5; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < 6; ++k) acc -= A[r][k] * x[k];
        x[r] = acc / A[r][r];
    }
    return 0;
}

/* Each boundary link x -> x+c_i (x fluid, x+c_i inside particle P) hands the
 * particle the bounce-back momentum c_i (f*_i + f_ibar) with
 * f_ibar = f*_i - 6 w_i rho0 c_i.u_b (Ladd), u_b = U + Omega x r_b + v_s, and
 * the chemical stress flux 6 w_i P(x).c_i.  The part linear in (U, Omega) is
 * collected in the 6x6 drag matrix zeta, the rest in (F0, T0), and
 *   (Mdiag + zeta) V(t+1) = Mdiag V(t) + [F0; T0]
 * is solved for the new velocity (Nguyen and Ladd's implicit update, cited in
 * Sec. "Particles").  The fluid's bounce-back then uses V(t+1), so the
 * momentum the fluid loses is exactly what the particle gains. */
static void step_links(ref_sim* s)
{
    const ref_params* p = &s->p;
    const long N = s->N;
    for (int k = 0; k < s->np; ++k) {
        ref_part* P = &s->part[k];
        for (int a = 0; a < 3; ++a) P->F0[a] = P->T0[a] = 0.0;
        memset(P->zeta, 0, sizeof(P->zeta));
    }
    if (s->np == 0) return;
    mark_particle_neighbours(s);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                if (!s->lk[n]) continue;
                for (int i = 1; i < 19; ++i) {
                    long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                    if (m < 0 || !s->mask[m]) continue;
                    ref_part* P = &s->part[s->mask[m] - 1];
                    double r[3], ub[3], vs[3];
                    link_velocity(s, P, x, y, z, i, r, ub, vs);
                    double cvs = CX[i] * vs[0] + CY[i] * vs[1] + CZ[i] * vs[2];
                    double mag = 2.0 * s->f[i * N + n] - 6.0 * W[i] * p->rho0 * cvs;
                    double dP[3] = {CX[i] * mag, CY[i] * mag, CZ[i] * mag};
                    if (p->thermo_force) {
                        double c[3] = {(double)CX[i], (double)CY[i], (double)CZ[i]}, pc[3];
                        pt_dot(s, n, c, pc);
                        for (int a = 0; a < 3; ++a) dP[a] += 6.0 * W[i] * pc[a];
                    }
                    P->F0[0] += dP[0];
                    P->F0[1] += dP[1];
                    P->F0[2] += dP[2];
                    P->T0[0] += r[1] * dP[2] - r[2] * dP[1];
                    P->T0[1] += r[2] * dP[0] - r[0] * dP[2];
                    P->T0[2] += r[0] * dP[1] - r[1] * dP[0];
                    double g6[6] = {(double)CX[i], (double)CY[i], (double)CZ[i],
                                    r[1] * CZ[i] - r[2] * CY[i],
                                    r[2] * CX[i] - r[0] * CZ[i],
                                    r[0] * CY[i] - r[1] * CX[i]};
                    double zc = 6.0 * W[i] * p->rho0;
                    for (int a = 0; a < 6; ++a)
                        for (int b = 0; b < 6; ++b) P->zeta[a][b] += zc * g6[a] * g6[b];
                }
            }
    for (int k = 0; k < s->np; ++k) {
        ref_part* P = &s->part[k];
        double F0[6];
        for (int a = 0; a < 3; ++a) {
            F0[a] = P->F0[a] + P->imp_f[a] + P->ext_f[a];
            F0[3 + a] = P->T0[a] + P->imp_t[a] + P->ext_t[a];
        }
        double V[6] = {P->U[0], P->U[1], P->U[2], P->Om[0], P->Om[1], P->Om[2]};
        if (!P->fixed) {
            double Mm[6] = {P->M, P->M, P->M, P->I, P->I, P->I};
            double A[6][6], b[6], Vn[6];
            for (int a = 0; a < 6; ++a) {
                for (int c = 0; c < 6; ++c) A[a][c] = P->zeta[a][c];
                A[a][a] += Mm[a];
                b[a] = Mm[a] * V[a] + F0[a];
            }
            if (solve6(A, b, Vn) != 0) s->err = -3;
            for (int a = 0; a < 6; ++a) V[a] = Vn[a];
        }
        for (int a = 0; a < 6; ++a) {
            double zv = 0.0;
            for (int c = 0; c < 6; ++c) zv += P->zeta[a][c] * V[c];
            if (a < 3)
                P->force[a] = F0[a] - zv;
            else
                P->torque[a - 3] = F0[a] - zv;
        }
        for (int a = 0; a < 3; ++a) {
            P->U[a] = V[a];
            P->Om[a] = V[3 + a];
            P->imp_f[a] = P->imp_t[a] = 0.0;
        }
    }
}

/* ------------------------------------------------------------------ */
/* S2 + S3: force, streaming with bounce-back, BGK + Guo collision     */
/* ------------------------------------------------------------------ */

static void step_collide(ref_sim* s)
{
    const ref_params* p = &s->p;
    const long N = s->N;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                if (s->mask[n]) {
                    for (int i = 0; i < 19; ++i) s->fn[i * N + n] = 0.0;
                    s->u[n] = s->u[N + n] = s->u[2 * N + n] = 0.0;
                    continue;
                }
                /* S2: F = g - div P, in the link form
                 * -6 sum_i w_i [(P(x) + P(x+c_i))/2] . c_i, with P(x) standing
                 * in for solid and wall neighbours (their share is the flux
                 * the particle or the wall receives). */
                double F[3] = {p->body_force[0], p->body_force[1], p->body_force[2]};
                if (p->thermo_force) {
                    double div[3] = {0.0, 0.0, 0.0};
                    for (int i = 1; i < 19; ++i) {
                        long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                        double c[3] = {(double)CX[i], (double)CY[i], (double)CZ[i]};
                        double a[3], b[3];
                        pt_dot(s, n, c, a);
                        if (m < 0 || s->mask[m]) {
                            b[0] = a[0];
                            b[1] = a[1];
                            b[2] = a[2];
                        } else {
                            pt_dot(s, m, c, b);
                        }
                        for (int k = 0; k < 3; ++k) div[k] += W[i] * (0.5 * (a[k] + b[k]));
                    }
                    for (int k = 0; k < 3; ++k) F[k] -= 6.0 * div[k];
                }
                /* S3: pull f_j(x) = f*_j(x - c_j); a wall source reflects
                 * f*_{jbar}(x); a particle source reflects with the moving
                 * boundary term (Ladd): f_j = f*_i(x) - 6 w_i rho0 c_i.u_b,
                 * i = jbar, with the particle velocity of this step. */
                double fl[19];
                for (int j = 0; j < 19; ++j) {
                    if (j == 0) {
                        fl[0] = s->f[n];
                        continue;
                    }
                    long m = nbr(s, x, y, z, -CX[j], -CY[j], -CZ[j]);
                    int i = opp(j);
                    if (m < 0) {
                        fl[j] = s->f[i * N + n];
                    } else if (s->mask[m]) {
                        const ref_part* P = &s->part[s->mask[m] - 1];
                        double r[3], ub[3], vs[3];
                        link_velocity(s, P, x, y, z, i, r, ub, vs);
                        double cub = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
                        fl[j] = s->f[i * N + n] - 6.0 * W[i] * p->rho0 * cub;
                    } else {
                        fl[j] = s->f[j * N + m];
                    }
                }
                double rho = 0.0, jm[3] = {0, 0, 0};
                for (int j = 0; j < 19; ++j) {
                    rho += fl[j];
                    jm[0] += CX[j] * fl[j];
                    jm[1] += CY[j] * fl[j];
                    jm[2] += CZ[j] * fl[j];
                }
                double u[3];
                for (int a = 0; a < 3; ++a) u[a] = (jm[a] + 0.5 * F[a]) / rho;
                double omf = 1.0 - 0.5 / p->tau;
                for (int j = 0; j < 19; ++j) {
                    double c[3] = {(double)CX[j], (double)CY[j], (double)CZ[j]};
                    double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
                    /* Guo source w_j [3 (c - u) + 9 (c.u) c] . F */
                    double S = 0.0;
                    for (int a = 0; a < 3; ++a) S += (3.0 * (c[a] - u[a]) + 9.0 * cu * c[a]) * F[a];
                    S *= W[j];
                    double fe = feq(j, rho, u);
                    s->fn[j * N + n] = fl[j] - (fl[j] - fe) / p->tau + omf * S;
                }
                s->u[n] = u[0];
                s->u[N + n] = u[1];
                s->u[2 * N + n] = u[2];
            }
    double* t = s->f;
    s->f = s->fn;
    s->fn = t;
}

/* ------------------------------------------------------------------ */
/* S4: scalar transport (Eq. diffusion_reaction) with source and sink  */
/* ------------------------------------------------------------------ */

static void step_scalars(ref_sim* s)
{
    const ref_params* p = &s->p;
    const long N = s->N;
    s->wall_psi = 0.0;
    s->wall_phi = 0.0;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                if (s->mask[n]) {
                    s->psin[n] = 0.0;
                    s->phin[n] = 0.0;
                    continue;
                }
                double ps = s->psi[n], ph = s->phi[n];
                double u0[3] = {s->u[n], s->u[N + n], s->u[2 * N + n]};
                double dps = 0.0, dph = 0.0;
                unsigned char adj[REF_MAXP];
                memset(adj, 0, (size_t)s->np);
                /* flux on each fluid-fluid link: diffusion M (mu(y) - mu(x))
                 * minus the advective flux, taken upwind (donor cell) with
                 * the link-mean velocity ub = c.(u(x) + u(y))/2.  Links to a
                 * wall carry no flux; a link to a particle carries no
                 * diffusive flux and the advective flux c.u_b g(x), u_b the
                 * boundary velocity of the bounce-back rule (the scalar moves
                 * with the fluid mass that rule exchanges with the wall). */
                for (int i = 1; i < 19; ++i) {
                    long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                    if (m < 0) continue;
                    if (s->mask[m]) {
                        adj[s->mask[m] - 1] = 1;
                        const ref_part* P = &s->part[s->mask[m] - 1];
                        double r[3], ub[3], vs[3];
                        link_velocity(s, P, x, y, z, i, r, ub, vs);
                        double cub = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
                        double aps = cub * ps, aph = cub * ph;
                        dps += W[i] * (0.0 - aps);
                        dph += W[i] * (0.0 - aph);
                        continue;
                    }
                    double cu0 = CX[i] * u0[0] + CY[i] * u0[1] + CZ[i] * u0[2];
                    double cu1 = CX[i] * s->u[m] + CY[i] * s->u[N + m] + CZ[i] * s->u[2 * N + m];
                    double ub = 0.5 * (cu0 + cu1);
                    double aps = ub > 0.0 ? ub * ps : ub * s->psi[m];
                    double aph = ub > 0.0 ? ub * ph : ub * s->phi[m];
                    dps += W[i] * (p->M_psi * (s->mupsi[m] - s->mupsi[n]) - aps);
                    dph += W[i] * (p->M_phi * (s->muphi[m] - s->muphi[n]) - aph);
                }
                s->psin[n] = ps + 6.0 * dps;
                double pn = ph + 6.0 * dph - p->k_d * (ph - phi0_of(s, ps));
                /* Janus production (Eq. activity) at fluid nodes next to the
                 * surface whose offset from the centre has m.(x - X) <= 0 */
                for (int k = 0; k < s->np; ++k) {
                    if (!adj[k]) continue;
                    const ref_part* P = &s->part[k];
                    double r[3];
                    node_offset(s, P, x, y, z, r);
                    double side = P->m[0] * r[0] + P->m[1] * r[1] + P->m[2] * r[2];
                    if (side <= 0.0) pn += P->alpha;
                }
                s->phin[n] = pn;
            }
    /* what the moving surfaces carried out of the fluid, summed in node and
     * link order (the same advective fluxes as above) */
    if (s->np > 0) {
        mark_particle_neighbours(s);
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long n = nidx(s, x, y, z);
                    if (!s->lk[n]) continue;
                    double ps = s->psi[n], ph = s->phi[n];
                    for (int i = 1; i < 19; ++i) {
                        long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                        if (m < 0 || !s->mask[m]) continue;
                        const ref_part* P = &s->part[s->mask[m] - 1];
                        double r[3], ub[3], vs[3];
                        link_velocity(s, P, x, y, z, i, r, ub, vs);
                        double cub = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
                        double aps = cub * ps, aph = cub * ph;
                        s->wall_psi += 6.0 * W[i] * aps;
                        s->wall_phi += 6.0 * W[i] * aph;
                    }
                }
    }
    double* t = s->psi;
    s->psi = s->psin;
    s->psin = t;
    t = s->phi;
    s->phi = s->phin;
    s->phin = t;
}

/* ------------------------------------------------------------------ */
/* S4 by lattice Boltzmann (scalar_scheme = 1)                         */
/* ------------------------------------------------------------------ */

/* Equilibrium of a scalar g with chemical potential mu and mobility M at
 * velocity u, relaxation time 1 (so Gamma = M / (1 - 1/2) = 2M):
 *   h_i = w_i (Gamma mu + g c_i.u) / c_s^2   (i = 1..6),
 *   h_0 = g - sum_{i>0} h_i = g - 3 Gamma mu.
 * Its moments are g, g u and Gamma mu I, which gives
 * dg/dt + div(g u) = M lap mu (Eq. diffusion_reaction). */
static double heq7(int i, double g, double mu, double M, const double u[3])
{
    const double G = 2.0 * M;
    if (i == 0) return g - 3.0 * G * mu;
    const double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    return W7[i] * (G * mu + g * cu) / 0.25;
}

static void step_scalars_lb(ref_sim* s)
{
    const ref_params* p = &s->p;
    const long N = s->N;
    s->wall_psi = 0.0;
    s->wall_phi = 0.0;
    /* collision (relaxation time 1: the post-collision populations are the
     * equilibrium), with the sink and the Janus production added to the rest
     * population of phi */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                if (s->mask[n]) {
                    for (int k = 0; k < 14; ++k) s->hs[k * N + n] = 0.0;
                    continue;
                }
                double u0[3] = {s->u[n], s->u[N + n], s->u[2 * N + n]};
                double ps = s->psi[n], ph = s->phi[n];
                for (int i = 0; i < 7; ++i) {
                    s->hs[i * N + n] = heq7(i, ps, s->mupsi[n], p->M_psi, u0);
                    s->hs[(7 + i) * N + n] = heq7(i, ph, s->muphi[n], p->M_phi, u0);
                }
                double src = -p->k_d * (ph - phi0_of(s, ps));
                unsigned char adj[REF_MAXP];
                memset(adj, 0, (size_t)s->np);
                for (int i = 1; i < 19; ++i) {
                    long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                    if (m >= 0 && s->mask[m]) adj[s->mask[m] - 1] = 1;
                }
                for (int k = 0; k < s->np; ++k) {
                    if (!adj[k]) continue;
                    const ref_part* P = &s->part[k];
                    double r[3];
                    node_offset(s, P, x, y, z, r);
                    double side = P->m[0] * r[0] + P->m[1] * r[1] + P->m[2] * r[2];
                    if (side <= 0.0) src += P->alpha;
                }
                s->hs[7 * N + n] += src;
            }
    /* pull streaming: from the fluid node x - c_i; halfway bounce-back from a
     * wall; from a particle, moving-wall bounce-back that carries g c.u_b into
     * the surface (c the direction from x into the particle) */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                if (s->mask[n]) {
                    for (int k = 0; k < 14; ++k) s->h[k * N + n] = 0.0;
                    s->psin[n] = s->phin[n] = 0.0;
                    continue;
                }
                double sp = 0.0, sh = 0.0;
                for (int i = 0; i < 7; ++i) {
                    double a, b;
                    if (i == 0) {
                        a = s->hs[n];
                        b = s->hs[7 * N + n];
                    } else {
                        const int j = opp(i);   /* direction from x to the source */
                        long m = nbr(s, x, y, z, CX[j], CY[j], CZ[j]);
                        if (m >= 0 && !s->mask[m]) {
                            a = s->hs[i * N + m];
                            b = s->hs[(7 + i) * N + m];
                        } else if (m < 0) {
                            a = s->hs[j * N + n];
                            b = s->hs[(7 + j) * N + n];
                        } else {
                            const ref_part* P = &s->part[s->mask[m] - 1];
                            double r[3], ub[3], vs[3];
                            link_velocity(s, P, x, y, z, j, r, ub, vs);
                            double cub = CX[j] * ub[0] + CY[j] * ub[1] + CZ[j] * ub[2];
                            /* 2 w_j g c_j.u_b / c_s^2 = g c_j.u_b */
                            a = s->hs[j * N + n] - s->psi[n] * cub;
                            b = s->hs[(7 + j) * N + n] - s->phi[n] * cub;
                        }
                    }
                    s->h[i * N + n] = a;
                    s->h[(7 + i) * N + n] = b;
                    sp += a;
                    sh += b;
                }
                s->psin[n] = sp;
                s->phin[n] = sh;
            }
    /* what the moving surfaces carried out of the fluid, in node and link
     * order (the same terms as the particle links above) */
    if (s->np > 0) {
        mark_particle_neighbours(s);
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long n = nidx(s, x, y, z);
                    if (!s->lk[n]) continue;
                    for (int i = 1; i < 7; ++i) {
                        const int j = opp(i);
                        long m = nbr(s, x, y, z, CX[j], CY[j], CZ[j]);
                        if (m < 0 || !s->mask[m]) continue;
                        const ref_part* P = &s->part[s->mask[m] - 1];
                        double r[3], ub[3], vs[3];
                        link_velocity(s, P, x, y, z, j, r, ub, vs);
                        double cub = CX[j] * ub[0] + CY[j] * ub[1] + CZ[j] * ub[2];
                        s->wall_psi += s->psi[n] * cub;
                        s->wall_phi += s->phi[n] * cub;
                    }
                }
    }
    double* t = s->psi;
    s->psi = s->psin;
    s->psin = t;
    t = s->phi;
    s->phi = s->phin;
    s->phin = t;
}

/* Distributions of scheme 1 at equilibrium with mu = 0 (fields set from
 * outside, refilled nodes). */
static void lb_fill_node(ref_sim* s, long n, const double u[3])
{
    const long N = s->N;
    for (int i = 0; i < 7; ++i) {
        s->h[i * N + n] = heq7(i, s->psi[n], 0.0, s->p.M_psi, u);
        s->h[(7 + i) * N + n] = heq7(i, s->phi[n], 0.0, s->p.M_phi, u);
    }
}

/* ------------------------------------------------------------------ */
/* S6b: particle motion with the velocity of this step                 */
/* ------------------------------------------------------------------ */

static void step_move(ref_sim* s)
{
    const int L[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int k = 0; k < s->np; ++k) {
        ref_part* P = &s->part[k];
        /* translate, wrapping periodic axes into [0, L) */
        for (int a = 0; a < 3; ++a) {
            double X = P->X[a] + P->U[a];
            if (s->p.periodic[a]) {
                if (X >= L[a])
                    X -= L[a];
                else if (X < 0.0)
                    X += L[a];
            } else if (X - P->R < 1.0 || X + P->R > L[a] - 2.0) {
                s->err = -4;
            }
            P->X[a] = X;
        }
        /* rotate m by the angle |Omega| about Omega (Rodrigues), renormalise */
        double w = sqrt(P->Om[0] * P->Om[0] + P->Om[1] * P->Om[1] + P->Om[2] * P->Om[2]);
        if (w > 0.0) {
            double k3[3] = {P->Om[0] / w, P->Om[1] / w, P->Om[2] / w};
            double c = cos(w), sn = sin(w);
            double* m = P->m;
            double kxm[3] = {k3[1] * m[2] - k3[2] * m[1], k3[2] * m[0] - k3[0] * m[2],
                             k3[0] * m[1] - k3[1] * m[0]};
            double km = k3[0] * m[0] + k3[1] * m[1] + k3[2] * m[2];
            double mn[3];
            for (int a = 0; a < 3; ++a) mn[a] = m[a] * c + kxm[a] * sn + k3[a] * km * (1.0 - c);
            double nn = sqrt(mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]);
            for (int a = 0; a < 3; ++a) m[a] = mn[a] / nn;
        }
    }
}

/* ------------------------------------------------------------------ */
/* S7: covering and uncovering                                          */
/* ------------------------------------------------------------------ */

static void step_cover(ref_sim* s)
{
    const ref_params* p = &s->p;
    const long N = s->N;
    if (s->np == 0) return;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) s->maskn[nidx(s, x, y, z)] = owner(s, x, y, z);
    /* what the moving surfaces carried out of the fluid this step */
    double dpsi = s->wall_psi, dphi = s->wall_phi;
    long dfl = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nidx(s, x, y, z);
                unsigned char o = s->mask[n], q = s->maskn[n];
                if (o == q) continue;
                if (o == 0) {
                    /* newly covered: the particle takes the momentum its
                     * populations carry, sum_i f_i c_i; the node's psi and phi
                     * are removed */
                    ref_part* P = &s->part[q - 1];
                    double j[3] = {0.0, 0.0, 0.0};
                    for (int i = 0; i < 19; ++i) {
                        j[0] += CX[i] * s->f[i * N + n];
                        j[1] += CY[i] * s->f[i * N + n];
                        j[2] += CZ[i] * s->f[i * N + n];
                    }
                    double r[3];
                    node_offset(s, P, x, y, z, r);
                    for (int a = 0; a < 3; ++a) P->imp_f[a] += j[a];
                    P->imp_t[0] += r[1] * j[2] - r[2] * j[1];
                    P->imp_t[1] += r[2] * j[0] - r[0] * j[2];
                    P->imp_t[2] += r[0] * j[1] - r[1] * j[0];
                    dpsi += s->psi[n];
                    dphi += s->phi[n];
                    s->psi[n] = s->phi[n] = 0.0;
                    if (s->h)
                        for (int k = 0; k < 14; ++k) s->h[k * N + n] = 0.0;
                    for (int i = 0; i < 19; ++i) s->f[i * N + n] = 0.0;
                    s->u[n] = s->u[N + n] = s->u[2 * N + n] = 0.0;
                    --dfl;
                } else if (q == 0) {
                    /* newly uncovered: equilibrium at the boundary velocity with
                     * the mean density of the neighbours that are fluid before
                     * and after; psi, phi = neighbour means */
                    ref_part* P = &s->part[o - 1];
                    double rb = 0.0, pb = 0.0, hb = 0.0;
                    int cnt = 0;
                    for (int i = 1; i < 19; ++i) {
                        long m = nbr(s, x, y, z, CX[i], CY[i], CZ[i]);
                        if (m < 0 || s->mask[m] || s->maskn[m]) continue;
                        double rm = 0.0;
                        for (int k = 0; k < 19; ++k) rm += s->f[k * N + m];
                        rb += rm;
                        pb += s->psi[m];
                        hb += s->phi[m];
                        ++cnt;
                    }
                    if (cnt == 0) {
                        s->err = -4;
                        rb = p->rho0;
                        pb = hb = 0.0;
                    } else {
                        rb /= cnt;
                        pb /= cnt;
                        hb /= cnt;
                    }
                    double r[3], ub[3];
                    node_offset(s, P, x, y, z, r);
                    ub[0] = P->U[0] + (P->Om[1] * r[2] - P->Om[2] * r[1]);
                    ub[1] = P->U[1] + (P->Om[2] * r[0] - P->Om[0] * r[2]);
                    ub[2] = P->U[2] + (P->Om[0] * r[1] - P->Om[1] * r[0]);
                    for (int i = 0; i < 19; ++i) s->f[i * N + n] = feq(i, rb, ub);
                    for (int a = 0; a < 3; ++a) s->u[a * N + n] = ub[a];
                    double j[3] = {rb * ub[0], rb * ub[1], rb * ub[2]};
                    for (int a = 0; a < 3; ++a) P->imp_f[a] -= j[a];
                    P->imp_t[0] -= r[1] * j[2] - r[2] * j[1];
                    P->imp_t[1] -= r[2] * j[0] - r[0] * j[2];
                    P->imp_t[2] -= r[0] * j[1] - r[1] * j[0];
                    s->psi[n] = pb;
                    s->phi[n] = hb;
                    if (s->h) lb_fill_node(s, n, ub);
                    dpsi -= pb;
                    dphi -= hb;
                    ++dfl;
                } else {
                    s->err = -4; /* node passed directly between two particles */
                }
            }
    memcpy(s->mask, s->maskn, (size_t)N);
    s->nfluid += dfl;
    if (dfl == 0 && dpsi == 0.0 && dphi == 0.0) return;
    /* restore the totals of psi and phi: spread the removed minus the added
     * amount (covering, uncovering and the flux into the moving surfaces)
     * uniformly over every fluid node */
    double cps = dpsi / (double)s->nfluid, cph = dphi / (double)s->nfluid;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->mask[n]) continue;
        s->psi[n] += cps;
        s->phi[n] += cph;
        if (s->h) {   /* the rest populations carry the correction */
            s->h[n] += cps;
            s->h[7 * N + n] += cph;
        }
    }
}

/* ------------------------------------------------------------------ */
/* public entry points                                                 */
/* ------------------------------------------------------------------ */

ref_sim* ref_create(const ref_params* p)
{
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || p->tau <= 0.5 || p->rho0 <= 0.0) return NULL;
    if (p->scalar_scheme != 0 && p->scalar_scheme != 1) return NULL;
    ref_sim* s = (ref_sim*)calloc(1, sizeof(ref_sim));
    if (!s) return NULL;
    s->p = *p;
    s->N = (long)p->nx * p->ny * p->nz;
    long N = s->N;
    s->f = (double*)calloc((size_t)(19 * N), sizeof(double));
    s->fn = (double*)calloc((size_t)(19 * N), sizeof(double));
    s->psi = (double*)calloc((size_t)N, sizeof(double));
    s->phi = (double*)calloc((size_t)N, sizeof(double));
    s->psin = (double*)calloc((size_t)N, sizeof(double));
    s->phin = (double*)calloc((size_t)N, sizeof(double));
    s->mupsi = (double*)calloc((size_t)N, sizeof(double));
    s->muphi = (double*)calloc((size_t)N, sizeof(double));
    s->pt = (double*)calloc((size_t)(6 * N), sizeof(double));
    s->u = (double*)calloc((size_t)(3 * N), sizeof(double));
    s->mask = (unsigned char*)calloc((size_t)N, 1);
    s->maskn = (unsigned char*)calloc((size_t)N, 1);
    s->lk = (unsigned char*)calloc((size_t)N, 1);
    if (!s->f || !s->fn || !s->psi || !s->phi || !s->psin || !s->phin || !s->mupsi || !s->muphi ||
        !s->u || !s->mask || !s->maskn || !s->lk || !s->pt) {
        ref_destroy(s);
        return NULL;
    }
    if (p->scalar_scheme == 1) {
        s->h = (double*)calloc((size_t)(14 * N), sizeof(double));
        s->hs = (double*)calloc((size_t)(14 * N), sizeof(double));
        if (!s->h || !s->hs) {
            ref_destroy(s);
            return NULL;
        }
    }
    s->nfluid = N;
    double u0[3] = {0, 0, 0};
    for (int i = 0; i < 19; ++i)
        for (long n = 0; n < N; ++n) s->f[i * N + n] = feq(i, p->rho0, u0);
    if (s->h)
        for (long n = 0; n < N; ++n) lb_fill_node(s, n, u0);
    return s;
}

void ref_destroy(ref_sim* s)
{
    if (!s) return;
    free(s->f);
    free(s->fn);
    free(s->psi);
    free(s->phi);
    free(s->psin);
    free(s->phin);
    free(s->mupsi);
    free(s->muphi);
    free(s->pt);
    free(s->u);
    free(s->mask);
    free(s->maskn);
    free(s->lk);
    free(s->h);
    free(s->hs);
    free(s);
}

int ref_set_fields(ref_sim* s, const double* rho, const double* u, const double* psi, const double* phi)
{
    const long N = s->N;
    for (long n = 0; n < N; ++n) {
        if (psi) s->psi[n] = s->mask[n] ? 0.0 : psi[n];
        if (phi) s->phi[n] = s->mask[n] ? 0.0 : phi[n];
        if (u)
            for (int a = 0; a < 3; ++a) s->u[a * N + n] = s->mask[n] ? 0.0 : u[a * N + n];
    }
    for (long n = 0; n < N; ++n) {
        double r = 0.0;
        for (int i = 0; i < 19; ++i) r += s->f[i * N + n];
        double rr = rho ? rho[n] : r;
        double uu[3] = {s->u[n], s->u[N + n], s->u[2 * N + n]};
        for (int i = 0; i < 19; ++i) s->f[i * N + n] = s->mask[n] ? 0.0 : feq(i, rr, uu);
        if (s->h && !s->mask[n]) lb_fill_node(s, n, uu);
    }
    return 0;
}

int ref_add_particle(ref_sim* s, const ref_particle_desc* d)
{
    if (s->np >= REF_MAXP || d->R <= 0.0) return -1;
    if (d->H != 0.0 && s->p.kappa <= 0.0) return -1;
    ref_part* P = &s->part[s->np];
    memset(P, 0, sizeof(*P));
    double mn = sqrt(d->m_hat[0] * d->m_hat[0] + d->m_hat[1] * d->m_hat[1] + d->m_hat[2] * d->m_hat[2]);
    if (!(mn > 0.0)) return -1;
    for (int a = 0; a < 3; ++a) {
        P->X[a] = d->pos[a];
        P->m[a] = d->m_hat[a] / mn;
        P->U[a] = d->vel[a];
        P->Om[a] = d->omega[a];
        P->ext_f[a] = d->ext_force[a];
        P->ext_t[a] = d->ext_torque[a];
    }
    P->R = d->R;
    P->R2 = d->R * d->R;
    double rp = d->rho_p > 0.0 ? d->rho_p : 1.0;
    P->M = rp * (4.0 / 3.0) * M_PI * d->R * d->R * d->R;
    P->I = 0.4 * P->M * d->R * d->R;
    P->alpha = d->alpha;
    P->mu_p = d->mu_plus;
    P->mu_m = d->mu_minus;
    P->H = d->H;
    P->fixed = d->fixed;
    s->np++;
    const long N = s->N;
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long n = nidx(s, x, y, z);
                if (s->mask[n]) continue;
                if (inside(s, P, x, y, z)) {
                    s->mask[n] = (unsigned char)s->np;
                    s->psi[n] = s->phi[n] = 0.0;
                    for (int i = 0; i < 19; ++i) s->f[i * N + n] = 0.0;
                    if (s->h)
                        for (int k = 0; k < 14; ++k) s->h[k * N + n] = 0.0;
                    s->u[n] = s->u[N + n] = s->u[2 * N + n] = 0.0;
                    s->nfluid--;
                }
            }
    return s->np - 1;
}

int ref_step(ref_sim* s, int nsteps)
{
    for (int t = 0; t < nsteps; ++t) {
        step_mu(s);
        step_links(s);
        step_collide(s);
        if (s->h)
            step_scalars_lb(s);
        else
            step_scalars(s);
        step_move(s);
        step_cover(s);
    }
    return s->err;
}

int ref_read_fields(const ref_sim* s, double* rho, double* u, double* psi, double* phi)
{
    const long N = s->N;
    for (long n = 0; n < N; ++n) {
        if (rho) {
            double r = 0.0;
            for (int i = 0; i < 19; ++i) r += s->f[i * N + n];
            rho[n] = r;
        }
        if (psi) psi[n] = s->psi[n];
        if (phi) phi[n] = s->phi[n];
    }
    if (u) memcpy(u, s->u, (size_t)(3 * N) * sizeof(double));
    return 0;
}

int ref_read_mu(ref_sim* s, double* mu_psi, double* mu_phi)
{
    step_mu(s); /* chemical potentials of the current fields */
    if (mu_psi) memcpy(mu_psi, s->mupsi, (size_t)s->N * sizeof(double));
    if (mu_phi) memcpy(mu_phi, s->muphi, (size_t)s->N * sizeof(double));
    return 0;
}

int ref_read_populations(const ref_sim* s, double* f)
{
    memcpy(f, s->f, (size_t)(19 * s->N) * sizeof(double));
    return 0;
}

int ref_read_mask(const ref_sim* s, unsigned char* mask)
{
    memcpy(mask, s->mask, (size_t)s->N);
    return 0;
}

int ref_read_particles(const ref_sim* s, ref_particle_state* out, int cap)
{
    int n = s->np < cap ? s->np : cap;
    for (int k = 0; k < n; ++k) {
        const ref_part* P = &s->part[k];
        for (int a = 0; a < 3; ++a) {
            out[k].pos[a] = P->X[a];
            out[k].vel[a] = P->U[a];
            out[k].omega[a] = P->Om[a];
            out[k].m_hat[a] = P->m[a];
            out[k].force[a] = P->force[a];
            out[k].torque[a] = P->torque[a];
        }
    }
    return s->np;
}

int ref_conservation(const ref_sim* s, double sums[3])
{
    const long N = s->N;
    double r = 0.0, a = 0.0, b = 0.0;
    for (long n = 0; n < N; ++n) {
        if (s->mask[n]) continue;
        for (int i = 0; i < 19; ++i) r += s->f[i * N + n];
        a += s->psi[n];
        b += s->phi[n];
    }
    sums[0] = r;
    sums[1] = a;
    sums[2] = b;
    return 0;
}

int ref_error(const ref_sim* s) { return s->err; }

int ref_set_threads(int n)
{
#ifdef _OPENMP
    if (n < 1) n = omp_get_num_procs();
    omp_set_num_threads(n);
    return n;
#else
    (void)n;
    return 1;
#endif
}
long ref_fluid_count(const ref_sim* s) { return s->nfluid; }

/* cos(theta_c) = [(1+h)^{3/2} - (1-h)^{3/2}] / 2 (Sec. Particles, wetting);
 * the right side increases monotonically on [-1, 1], so bisection finds h. */
double ref_wetting_h(double theta_deg)
{
    double target = cos(theta_deg * M_PI / 180.0);
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double v = 0.5 * (pow(1.0 + mid, 1.5) - pow(1.0 - mid, 1.5));
        if (v < target)
            lo = mid;
        else
            hi = mid;
        if (hi - lo < 1e-16) break;
    }
    return 0.5 * (lo + hi);
}
