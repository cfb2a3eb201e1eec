// lbdp_kernels.cuh -- the per-step kernels of the lattice update, templated on
// the precision configuration.  One step is
//   k_mu           chemical potentials (Eq. chem_potentials) with wetting
//                  ghosts, and the chemical pressure tensor P of Eq. free_energy
//   k_links        per particle: bounce-back and chemical-stress momentum sums
//                  over its boundary links, implicit velocity update, new
//                  position and orientation (Sec. "Particles")
//   k_collide      force g - div P, D3Q19 pull streaming with halfway
//                  bounce-back on walls and moving bounce-back plus phoretic
//                  slip on particle links, BGK + Guo
//   k_scalars      conservative psi/phi transport (Eq. diffusion_reaction),
//                  Janus production (Eq. activity) and the k_d sink
//   k_cover_mark   per particle: solid mask at the new positions
//   k_cover_apply  per particle: covering/uncovering; the last block folds
//                  the psi/phi deficits into the uniform correction and moves
//                  the particles
// Every kernel is HBM-bound stencil or streaming work: no tensor cores.
#pragma once

#include "lbdp_lattice.cuh"

namespace lbdp {

template <class Pop, class Fld, class Real>
struct Cfg {
    using pop_t = Pop;
    using fld_t = Fld;
    using real = Real;
};
using CfgF64 = Cfg<double, double, double>;
using CfgF32 = Cfg<float, float, float>;
using CfgF16 = Cfg<__half, float, float>;
using CfgBF16 = Cfg<__nv_bfloat16, float, float>;

constexpr int kRowThreads = 128;
constexpr int kPartThreads = 256;

// ---------------------------------------------------------------------------
// shared device helpers
// ---------------------------------------------------------------------------

// Isotropic gradient of phi at a fluid node, 3 sum_i w_i c_i phi(x+c_i), with
// the node's own value standing in for solid and wall neighbours.
template <class Fld>
__device__ __forceinline__ void grad_phi_at(const int nb[19], const Fld* phi, const uint8_t* mask, double own,
                                            double dphi, double g[3])
{
    g[0] = g[1] = g[2] = 0.0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        int m = nb[i];
        double v = (m < 0 || mask[m]) ? own : (double)phi[m] + dphi;
        g[0] += wgt(i) * cx(i) * v;
        g[1] += wgt(i) * cy(i) * v;
        g[2] += wgt(i) * cz(i) * v;
    }
    g[0] *= 3.0;
    g[1] *= 3.0;
    g[2] *= 3.0;
}

// Boundary velocity at the midpoint of link x -> x + c_i of particle q:
// u_b = U + Omega x r + v_s, v_s = mu (1 - n n) . grad phi, mu = mu_- where
// m.r <= 0 else mu_+ (Eq. MuJ).  Returns r (midpoint offset), u_b and v_s.
__device__ __forceinline__ void link_velocity(const DevParams& P, const DevPart& q, int x, int y, int z, int i,
                                              const double gphi[3], double r[3], double ub[3], double vs[3])
{
    node_offset(P, q, x, y, z, r);
    r[0] = __dadd_rn(r[0], 0.5 * cx(i));
    r[1] = __dadd_rn(r[1], 0.5 * cy(i));
    r[2] = __dadd_rn(r[2], 0.5 * cz(i));
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double nh[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    double side = dot3_rn(q.m, r);
    double mu = (side <= 0.0) ? q.mu_m : q.mu_p;
    double ng = nh[0] * gphi[0] + nh[1] * gphi[1] + nh[2] * gphi[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) vs[a] = mu * (gphi[a] - nh[a] * ng);
    ub[0] = q.U[0] + (q.W[1] * r[2] - q.W[2] * r[1]) + vs[0];
    ub[1] = q.U[1] + (q.W[2] * r[0] - q.W[0] * r[2]) + vs[1];
    ub[2] = q.U[2] + (q.W[0] * r[1] - q.W[1] * r[0]) + vs[2];
}

template <class Real>
__device__ __forceinline__ Real feq_i(int i, Real rho, Real ux, Real uy, Real uz)
{
    Real cu = (Real)cx(i) * ux + (Real)cy(i) * uy + (Real)cz(i) * uz;
    Real uu = ux * ux + uy * uy + uz * uz;
    return (Real)wgt(i) * rho * ((Real)1 + (Real)3 * cu + (Real)4.5 * cu * cu - (Real)1.5 * uu);
}

__device__ __forceinline__ float tanh_r(float v) { return tanhf(v); }
__device__ __forceinline__ double tanh_r(double v) { return tanh(v); }
__device__ __forceinline__ float cosh_r(float v) { return coshf(v); }
__device__ __forceinline__ double cosh_r(double v) { return cosh(v); }

// P(n) . c_i from the six stored components (xx yy zz xy xz yz).
template <class F, class R>
__device__ __forceinline__ void pt_dot(const F* pt, size_t N, int n, int i, R out[3])
{
    const R xx = (R)pt[n], yy = (R)pt[N + n], zz = (R)pt[2 * N + n];
    const R xy = (R)pt[3 * N + n], xz = (R)pt[4 * N + n], yz = (R)pt[5 * N + n];
    const R c0 = (R)cx(i), c1 = (R)cy(i), c2 = (R)cz(i);
    out[0] = xx * c0 + xy * c1 + xz * c2;
    out[1] = xy * c0 + yy * c1 + yz * c2;
    out[2] = xz * c0 + yz * c1 + zz * c2;
}

// FP64 block reduction: sums K values per thread over the block in a fixed
// order (warp shuffles, then warps in index order); the result is valid in
// thread 0.
template <int K>
__device__ void block_sum(double (&v)[K], double* smem /* [32*K] */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0)
        for (int k = 0; k < K; ++k) smem[warp * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += smem[w * K + k];
            v[k] = s;
        }
    }
    __syncthreads();
}

// Gaussian elimination with partial pivoting, 6x6 (single thread).
__device__ inline int solve6(double A[6][6], double b[6], double x[6])
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

// Lattice node of slot t in a box of edges s[3] starting at o[3]; false when
// the node falls beyond a wall.
__device__ __forceinline__ bool box_node(const DevParams& P, const int o[3], const int s[3], int t, int& x, int& y,
                                         int& z)
{
    x = wrap_coord(o[0] + t % s[0], P.nx, P.per[0]);
    y = wrap_coord(o[1] + (t / s[0]) % s[1], P.ny, P.per[1]);
    z = wrap_coord(o[2] + t / (s[0] * s[1]), P.nz, P.per[2]);
    return x >= 0 && y >= 0 && z >= 0;
}

// ---------------------------------------------------------------------------
// S1: chemical potentials and pressure tensor
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kRowThreads) k_mu(DevParams P, DevPtrs D)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int n = x + P.nx * (y + P.ny * z);
    if (D.mask[n]) return;
    const size_t N = (size_t)P.N;
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    const R dps = (R)D.corr[0], dph = (R)D.corr[1];
    const R ps = (R)psi[n] + dps, ph = (R)phi[n] + dph;
    int nb[19];
    neighbours(P, x, y, z, nb);
    R lap = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int m = nb[i];
        R v;
        if (m < 0) {
            v = ps;
        } else {
            const uint8_t q = D.mask[m];
            if (q) {
                // wetting ghost psi(x) + (H/kappa) c_i . n_hat at the link midpoint
                const DevPart& pq = D.parts[q - 1];
                if (pq.H != 0.0) {
                    double r[3];
                    node_offset(P, pq, x, y, z, r);
                    r[0] = __dadd_rn(r[0], 0.5 * cx(i));
                    r[1] = __dadd_rn(r[1], 0.5 * cy(i));
                    r[2] = __dadd_rn(r[2], 0.5 * cz(i));
                    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                    double cn = (cx(i) * r[0] + cy(i) * r[1] + cz(i) * r[2]) / rn;
                    v = ps + (R)((pq.H / P.kappa) * cn);
                } else {
                    v = ps;
                }
            } else {
                v = (R)psi[m] + dps;
            }
        }
        const R w = (R)wgt(i);
        lap += w * (v - ps);
        g0 += w * (R)cx(i) * v;
        g1 += w * (R)cy(i) * v;
        g2 += w * (R)cz(i) * v;
    }
    lap *= (R)6;
    g0 *= (R)3;
    g1 *= (R)3;
    g2 *= (R)3;
    const R A = (R)P.A, Cc = (R)P.C, kap = (R)P.kappa;
    const R dphi = ph - ((R)P.phib + (R)P.E * tanh_r(ps));
    const R ch = cosh_r(ps);
    const R mph = Cc * dphi;
    const R mps = A * (ps * ps * ps - ps) - kap * lap - Cc * (R)P.E * dphi / (ch * ch);
    ((F*)D.muphi)[n] = (F)mph;
    ((F*)D.mupsi)[n] = (F)mps;
    // P = [psi mu_psi + phi mu_phi - f - kappa |grad psi|^2/2] I + kappa grad psi grad psi
    const R f = (R)0.25 * A * ps * ps * ps * ps - (R)0.5 * A * ps * ps + (R)0.5 * Cc * dphi * dphi;
    const R gg = g0 * g0 + g1 * g1 + g2 * g2;
    const R piso = ps * mps + ph * mph - f - (R)0.5 * kap * gg;
    F* pt = (F*)D.pt;
    pt[n] = (F)(piso + kap * g0 * g0);
    pt[N + n] = (F)(piso + kap * g1 * g1);
    pt[2 * N + n] = (F)(piso + kap * g2 * g2);
    pt[3 * N + n] = (F)(kap * g0 * g1);
    pt[4 * N + n] = (F)(kap * g0 * g2);
    pt[5 * N + n] = (F)(kap * g1 * g2);
}

// ---------------------------------------------------------------------------
// S5 + S6a: link sums and the implicit velocity update.  Grid (nb1, np): the
// blocks of a particle split its link box; the last block of the particle (a
// ticket counter) sums the partials in block order and solves
//   (Mdiag + zeta) V(t+1) = Mdiag V(t) + [F0; T0]
// then stores the new velocity and the position/orientation after the step.
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kPartThreads) k_links(DevParams P, DevPtrs D)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    constexpr int K = kLinkK;
    __shared__ double smem[32 * K];
    __shared__ DevPart sp;
    __shared__ bool last;
    const int p = blockIdx.y;
    if (threadIdx.x == 0) sp = D.parts[p];
    __syncthreads();
    const DevPart& q = sp;
    const size_t N = (size_t)P.N;
    const S* fs = (const S*)D.f_src;
    const F* phi = (const F*)D.phi_src;
    const F* pt = (const F*)D.pt;
    const int o[3] = {(int)floor(q.X[0] - q.R) - 2, (int)floor(q.X[1] - q.R) - 2, (int)floor(q.X[2] - q.R) - 2};
    const int tot = P.side1[0] * P.side1[1] * P.side1[2];
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const double zc0 = 6.0 * P.rho0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side1, t, x, y, z)) continue;
        const int n = x + P.nx * (y + P.ny * z);
        if (D.mask[n]) continue;
        int nb[19];
        neighbours(P, x, y, z, nb);
        bool have_g = false;
        double gphi[3] = {0.0, 0.0, 0.0};
        for (int i = 1; i < 19; ++i) {
            const int m = nb[i];
            if (m < 0 || D.mask[m] != p + 1) continue;
            if (!have_g) {
                grad_phi_at(nb, phi, D.mask, (double)phi[n] + D.corr[1], D.corr[1], gphi);
                have_g = true;
            }
            double r[3], ub[3], vs[3];
            link_velocity(P, q, x, y, z, i, gphi, r, ub, vs);
            const double fi = (double)PopStore<S>::load(fs, (size_t)i * N + n, i, (R)P.rho0);
            const double w = wgt(i);
            const double c[3] = {(double)cx(i), (double)cy(i), (double)cz(i)};
            const double cvs = c[0] * vs[0] + c[1] * vs[1] + c[2] * vs[2];
            const double mag = 2.0 * fi - 6.0 * w * P.rho0 * cvs;
            double dP[3] = {c[0] * mag, c[1] * mag, c[2] * mag};
            if (P.thermo) {
                // chemical stress flux through the link, 6 w_i P(x) . c_i
                double pc[3];
                pt_dot<F, double>(pt, N, n, i, pc);
                for (int a = 0; a < 3; ++a) dP[a] += 6.0 * w * pc[a];
            }
            acc[0] += dP[0];
            acc[1] += dP[1];
            acc[2] += dP[2];
            acc[3] += r[1] * dP[2] - r[2] * dP[1];
            acc[4] += r[2] * dP[0] - r[0] * dP[2];
            acc[5] += r[0] * dP[1] - r[1] * dP[0];
            const double g6[6] = {c[0], c[1], c[2], r[1] * c[2] - r[2] * c[1], r[2] * c[0] - r[0] * c[2],
                                  r[0] * c[1] - r[1] * c[0]};
            const double zc = zc0 * w;
            int k = 6;
#pragma unroll
            for (int a = 0; a < 6; ++a)
#pragma unroll
                for (int b = a; b < 6; ++b) acc[k++] += zc * g6[a] * g6[b];
        }
    }
    block_sum<K>(acc, smem);
    double* part = D.link_part + ((size_t)p * kMaxPartBlocks + blockIdx.x) * K;
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) part[k] = acc[k];
        __threadfence();
        last = (atomicAdd(D.link_ticket + p, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double sum[K];
    for (int k = 0; k < K; ++k) sum[k] = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        volatile const double* pb = D.link_part + ((size_t)p * kMaxPartBlocks + b) * K;
        for (int k = 0; k < K; ++k) sum[k] += pb[k];
    }
    D.link_ticket[p] = 0u;

    DevPart& dp = D.parts[p];
    double zeta[6][6];
    {
        int k = 6;
        for (int a = 0; a < 6; ++a)
            for (int b = a; b < 6; ++b) {
                zeta[a][b] = sum[k];
                zeta[b][a] = sum[k];
                ++k;
            }
    }
    double F0[6];
    for (int a = 0; a < 3; ++a) {
        F0[a] = sum[a] + q.imp_f[a] + q.ext_f[a];
        F0[3 + a] = sum[3 + a] + q.imp_t[a] + q.ext_t[a];
    }
    double V[6] = {q.U[0], q.U[1], q.U[2], q.W[0], q.W[1], q.W[2]};
    if (!q.fixed) {
        const double Mm[6] = {q.M, q.M, q.M, q.I, q.I, q.I};
        double A[6][6], b[6], Vn[6];
        for (int a = 0; a < 6; ++a) {
            for (int c = 0; c < 6; ++c) A[a][c] = zeta[a][c];
            A[a][a] += Mm[a];
            b[a] = Mm[a] * V[a] + F0[a];
        }
        if (solve6(A, b, Vn) != 0) atomicOr(D.err, kErrSolve);
        for (int a = 0; a < 6; ++a) V[a] = Vn[a];
    }
    for (int a = 0; a < 6; ++a) {
        double zv = 0.0;
        for (int c = 0; c < 6; ++c) zv += zeta[a][c] * V[c];
        if (a < 3)
            dp.force[a] = F0[a] - zv;
        else
            dp.torque[a - 3] = F0[a] - zv;
    }
    const int L[3] = {P.nx, P.ny, P.nz};
    for (int a = 0; a < 3; ++a) {
        dp.U[a] = V[a];
        dp.W[a] = V[3 + a];
        dp.imp_f[a] = 0.0;
        dp.imp_t[a] = 0.0;
        double X = q.X[a] + V[a];
        if (P.per[a]) {
            if (X >= L[a])
                X -= L[a];
            else if (X < 0.0)
                X += L[a];
        } else if (X - q.R < 1.0 || X + q.R > L[a] - 2.0) {
            atomicOr(D.err, kErrWall);
        }
        dp.Xn[a] = X;
        dp.mn[a] = q.m[a];
    }
    // rotate m by the angle |Omega| about Omega (Rodrigues), renormalise
    const double w = sqrt(V[3] * V[3] + V[4] * V[4] + V[5] * V[5]);
    if (w > 0.0) {
        const double k3[3] = {V[3] / w, V[4] / w, V[5] / w};
        const double c = cos(w), sn = sin(w);
        const double* m = q.m;
        const double kxm[3] = {k3[1] * m[2] - k3[2] * m[1], k3[2] * m[0] - k3[0] * m[2],
                               k3[0] * m[1] - k3[1] * m[0]};
        const double km = k3[0] * m[0] + k3[1] * m[1] + k3[2] * m[2];
        double mn[3];
        for (int a = 0; a < 3; ++a) mn[a] = m[a] * c + kxm[a] * sn + k3[a] * km * (1.0 - c);
        const double nn = sqrt(mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]);
        for (int a = 0; a < 3; ++a) dp.mn[a] = mn[a] / nn;
    }
}

// ---------------------------------------------------------------------------
// S2 + S3: force, streaming with bounce-back, BGK collision with Guo forcing
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kRowThreads) k_collide(DevParams P, DevPtrs D)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int n = x + P.nx * (y + P.ny * z);
    if (D.mask[n]) return;
    const size_t N = (size_t)P.N;
    const S* fs = (const S*)D.f_src;
    S* fd = (S*)D.f_dst;
    const F* phi = (const F*)D.phi_src;
    const F* pt = (const F*)D.pt;
    const R rho0 = (R)P.rho0;
    int nb[19];
    neighbours(P, x, y, z, nb);

    // F = g - div P in the link form -6 sum_i w_i [(P(x) + P(x+c_i))/2] . c_i,
    // P(x) standing in for solid and wall neighbours
    R Fx = (R)P.g[0], Fy = (R)P.g[1], Fz = (R)P.g[2];
    if (P.thermo) {
        R d0 = 0, d1 = 0, d2 = 0;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int m = nb[i];
            R a[3], b[3];
            pt_dot<F, R>(pt, N, n, i, a);
            if (m < 0 || D.mask[m]) {
                b[0] = a[0];
                b[1] = a[1];
                b[2] = a[2];
            } else {
                pt_dot<F, R>(pt, N, m, i, b);
            }
            const R w = (R)wgt(i);
            d0 += w * ((R)0.5 * (a[0] + b[0]));
            d1 += w * ((R)0.5 * (a[1] + b[1]));
            d2 += w * ((R)0.5 * (a[2] + b[2]));
        }
        Fx -= (R)6 * d0;
        Fy -= (R)6 * d1;
        Fz -= (R)6 * d2;
    }

    R fl[19];
    bool have_g = false;
    double gphi[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        if (j == 0) {
            fl[0] = (R)PopStore<S>::load(fs, n, 0, rho0);
            continue;
        }
        const int i = opp(j);
        const int m = nb[i];   // source x - c_j = x + c_i
        if (m < 0) {
            fl[j] = (R)PopStore<S>::load(fs, (size_t)i * N + n, i, rho0);
        } else {
            const uint8_t q = D.mask[m];
            if (q) {
                if (!have_g) {
                    grad_phi_at(nb, phi, D.mask, (double)phi[n] + D.corr[1], D.corr[1], gphi);
                    have_g = true;
                }
                double r[3], ub[3], vs[3];
                link_velocity(P, D.parts[q - 1], x, y, z, i, gphi, r, ub, vs);
                const double cub = cx(i) * ub[0] + cy(i) * ub[1] + cz(i) * ub[2];
                const R fi = (R)PopStore<S>::load(fs, (size_t)i * N + n, i, rho0);
                fl[j] = fi - (R)(6.0 * wgt(i) * P.rho0 * cub);
            } else {
                fl[j] = (R)PopStore<S>::load(fs, (size_t)j * N + m, j, rho0);
            }
        }
    }
    R rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        rho += fl[j];
        jx += (R)cx(j) * fl[j];
        jy += (R)cy(j) * fl[j];
        jz += (R)cz(j) * fl[j];
    }
    const R ux = (jx + (R)0.5 * Fx) / rho;
    const R uy = (jy + (R)0.5 * Fy) / rho;
    const R uz = (jz + (R)0.5 * Fz) / rho;
    const R itau = (R)(1.0 / P.tau);
    const R omf = (R)(1.0 - 0.5 / P.tau);
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        const R c0 = (R)cx(j), c1 = (R)cy(j), c2 = (R)cz(j);
        const R cu = c0 * ux + c1 * uy + c2 * uz;
        R Sg = ((R)3 * (c0 - ux) + (R)9 * cu * c0) * Fx + ((R)3 * (c1 - uy) + (R)9 * cu * c1) * Fy +
               ((R)3 * (c2 - uz) + (R)9 * cu * c2) * Fz;
        Sg *= (R)wgt(j);
        const R fe = feq_i<R>(j, rho, ux, uy, uz);
        const R out = fl[j] - (fl[j] - fe) * itau + omf * Sg;
        PopStore<S>::store(fd, (size_t)j * N + n, j, rho0, out);
    }
    F* u = (F*)D.u;
    u[n] = (F)ux;
    u[N + n] = (F)uy;
    u[2 * N + n] = (F)uz;
}

// ---------------------------------------------------------------------------
// S4: psi and phi transport, production and sink
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kRowThreads) k_scalars(DevParams P, DevPtrs D)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int n = x + P.nx * (y + P.ny * z);
    if (D.mask[n]) return;
    const size_t N = (size_t)P.N;
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    const F* mps = (const F*)D.mupsi;
    const F* mph = (const F*)D.muphi;
    const F* u = (const F*)D.u;
    const R dps = (R)D.corr[0], dph = (R)D.corr[1];
    const R ps = (R)psi[n] + dps, ph = (R)phi[n] + dph;
    const R a0 = (R)mps[n], b0 = (R)mph[n];
    const R ux = (R)u[n], uy = (R)u[N + n], uz = (R)u[2 * N + n];
    const R Mps = (R)P.Mpsi, Mph = (R)P.Mphi;
    int nb[19];
    neighbours(P, x, y, z, nb);
    R sps = 0, sph = 0;
    unsigned long long adj = 0ull;
    bool have_g = false;
    double gphi[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int m = nb[i];
        if (m < 0) continue;
        const uint8_t q = D.mask[m];
        if (q) {
            // link into a particle: no diffusive flux; the scalar leaves with
            // the boundary velocity of the bounce-back rule, c.u_b g(x)
            adj |= 1ull << (q - 1);
            if (!have_g) {
                grad_phi_at(nb, phi, D.mask, (double)phi[n] + D.corr[1], D.corr[1], gphi);
                have_g = true;
            }
            double r[3], ub[3], vs[3];
            link_velocity(P, D.parts[q - 1], x, y, z, i, gphi, r, ub, vs);
            const double cub = cx(i) * ub[0] + cy(i) * ub[1] + cz(i) * ub[2];
            const R w = (R)wgt(i);
            sps += w * ((R)0 - (R)(cub * (double)ps));
            sph += w * ((R)0 - (R)(cub * (double)ph));
            continue;
        }
        const R c0 = (R)cx(i), c1 = (R)cy(i), c2 = (R)cz(i);
        const R cu0 = c0 * ux + c1 * uy + c2 * uz;
        const R cu1 = c0 * (R)u[m] + c1 * (R)u[N + m] + c2 * (R)u[2 * N + m];
        const R ub = (R)0.5 * (cu0 + cu1);
        const R psm = (R)psi[m] + dps, phm = (R)phi[m] + dph;
        const R aps = ub > (R)0 ? ub * ps : ub * psm;
        const R aph = ub > (R)0 ? ub * ph : ub * phm;
        const R w = (R)wgt(i);
        sps += w * (Mps * ((R)mps[m] - a0) - aps);
        sph += w * (Mph * ((R)mph[m] - b0) - aph);
    }
    const R pn = ps + (R)6 * sps;
    R hn = ph + (R)6 * sph - (R)P.kd * (ph - ((R)P.phib + (R)P.E * tanh_r(ps)));
    while (adj) {
        const int k = __ffsll((long long)adj) - 1;
        adj &= adj - 1;
        const DevPart& q = D.parts[k];
        double r[3];
        node_offset(P, q, x, y, z, r);
        if (dot3_rn(q.m, r) <= 0.0) hn += (R)q.alpha;
    }
    ((F*)D.psi_dst)[n] = (F)pn;
    ((F*)D.phi_dst)[n] = (F)hn;
}

// ---------------------------------------------------------------------------
// S7: covering / uncovering.  The cover box of particle p holds its old and
// new position with a margin that contains every neighbour of a node that can
// change.  k_cover_mark writes the new mask of the box (ownership over all
// particles at their new positions, first match); k_cover_apply moves the
// fields of the changed nodes and sums what the moving surfaces carried out
// of the fluid.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cover_origin(const DevParams& P, const DevPart& q, int o[3])
{
    for (int a = 0; a < 3; ++a) {
        const int L = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
        double lo = fmin(q.X[a], q.Xn[a]);
        // on a periodic axis the two centres may sit on opposite sides of the
        // wrap; take the lower end of the shorter arc
        if (P.per[a] && fabs(q.X[a] - q.Xn[a]) > 0.5 * L) lo = fmax(q.X[a], q.Xn[a]);
        o[a] = (int)floor(lo - q.R) - 3;
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_cover_mark(DevParams P, DevPtrs D)
{
    const int p = blockIdx.y;
    const DevPart& q = D.parts[p];
    int o[3];
    cover_origin(P, q, o);
    const int tot = P.side2[0] * P.side2[1] * P.side2[2];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side2, t, x, y, z)) continue;
        uint8_t own = 0;
        for (int k = 0; k < P.np; ++k)
            if (inside_at(P, D.parts[k].Xn, D.parts[k].R2, x, y, z)) {
                own = (uint8_t)(k + 1);
                break;
            }
        D.mask_next[x + P.nx * (y + P.ny * z)] = own;
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_cover_apply(DevParams P, DevPtrs D)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    constexpr int K = kCoverK;
    __shared__ double smem[32 * K];
    __shared__ bool last;
    const int p = blockIdx.y;
    const DevPart& q = D.parts[p];
    const size_t N = (size_t)P.N;
    int o[3];
    cover_origin(P, q, o);
    const int tot = P.side2[0] * P.side2[1] * P.side2[2];
    S* f = (S*)D.f_dst;
    F* psi = (F*)D.psi_dst;
    F* phi = (F*)D.phi_dst;
    const F* psi0 = (const F*)D.psi_src;
    const F* phi0 = (const F*)D.phi_src;
    F* u = (F*)D.u;
    const R rho0 = (R)P.rho0;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side2, t, x, y, z)) continue;
        const int n = x + P.nx * (y + P.ny * z);
        const uint8_t ob = D.mask[n], nw = D.mask_next[n];
        int nb[19];
        neighbours(P, x, y, z, nb);
        if (ob == 0) {
            // psi, phi carried into the surface this step through the links of
            // this node into particle p: 6 w_i c_i.u_b g(x), as in k_scalars
            bool have_g = false;
            double gphi[3] = {0.0, 0.0, 0.0};
            for (int i = 1; i < 19; ++i) {
                const int m = nb[i];
                if (m < 0 || D.mask[m] != p + 1) continue;
                if (!have_g) {
                    grad_phi_at(nb, phi0, D.mask, (double)phi0[n] + D.corr[1], D.corr[1], gphi);
                    have_g = true;
                }
                double r[3], ub[3], vs[3];
                link_velocity(P, q, x, y, z, i, gphi, r, ub, vs);
                const double cub = cx(i) * ub[0] + cy(i) * ub[1] + cz(i) * ub[2];
                acc[9] += 6.0 * wgt(i) * (cub * ((double)psi0[n] + D.corr[0]));
                acc[10] += 6.0 * wgt(i) * (cub * ((double)phi0[n] + D.corr[1]));
            }
        }
        if (ob == nw) continue;
        if (ob == 0 && nw == p + 1) {
            // covered: the particle takes the momentum the node's populations
            // carry; psi, phi are removed
            double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                const double fi = (double)PopStore<S>::load(f, (size_t)i * N + n, i, rho0);
                j[0] += cx(i) * fi;
                j[1] += cy(i) * fi;
                j[2] += cz(i) * fi;
            }
            double r[3];
            offset_from(P, q.Xn, x, y, z, r);
            acc[0] += j[0];
            acc[1] += j[1];
            acc[2] += j[2];
            acc[3] += r[1] * j[2] - r[2] * j[1];
            acc[4] += r[2] * j[0] - r[0] * j[2];
            acc[5] += r[0] * j[1] - r[1] * j[0];
            acc[6] += (double)psi[n];
            acc[7] += (double)phi[n];
            acc[8] -= 1.0;
        } else if (ob == p + 1 && nw == 0) {
            // uncovered: equilibrium at the boundary velocity with the mean
            // density of neighbours fluid before and after; psi, phi = means
            double rb = 0.0, pb = 0.0, hb = 0.0;
            int cnt = 0;
            for (int i = 1; i < 19; ++i) {
                const int m = nb[i];
                if (m < 0 || D.mask[m] || D.mask_next[m]) continue;
                R rm = 0;
#pragma unroll
                for (int k = 0; k < 19; ++k) rm += (R)PopStore<S>::load(f, (size_t)k * N + m, k, rho0);
                rb += (double)rm;
                pb += (double)psi[m];
                hb += (double)phi[m];
                ++cnt;
            }
            if (cnt == 0) {
                atomicOr(D.err, kErrOverlap);
                rb = P.rho0;
                pb = hb = 0.0;
            } else {
                rb /= cnt;
                pb /= cnt;
                hb /= cnt;
            }
            double r[3];
            offset_from(P, q.Xn, x, y, z, r);
            const double ub[3] = {q.U[0] + (q.W[1] * r[2] - q.W[2] * r[1]), q.U[1] + (q.W[2] * r[0] - q.W[0] * r[2]),
                                  q.U[2] + (q.W[0] * r[1] - q.W[1] * r[0])};
#pragma unroll
            for (int i = 0; i < 19; ++i)
                PopStore<S>::store(f, (size_t)i * N + n, i, rho0, (R)feq_i<double>(i, rb, ub[0], ub[1], ub[2]));
            u[n] = (F)ub[0];
            u[N + n] = (F)ub[1];
            u[2 * N + n] = (F)ub[2];
            psi[n] = (F)pb;
            phi[n] = (F)hb;
            const double j[3] = {rb * ub[0], rb * ub[1], rb * ub[2]};
            acc[0] -= j[0];
            acc[1] -= j[1];
            acc[2] -= j[2];
            acc[3] -= r[1] * j[2] - r[2] * j[1];
            acc[4] -= r[2] * j[0] - r[0] * j[2];
            acc[5] -= r[0] * j[1] - r[1] * j[0];
            acc[6] -= pb;
            acc[7] -= hb;
            acc[8] += 1.0;
        } else if (ob == p + 1) {
            atomicOr(D.err, kErrOverlap);   // passed straight into another sphere
        }
    }
    block_sum<K>(acc, smem);
    double* part = D.cover_part + ((size_t)p * kMaxPartBlocks + blockIdx.x) * K;
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) part[k] = acc[k];
        __threadfence();
        last = (atomicAdd(D.cover_ticket, 1u) == gridDim.x * gridDim.y - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    // last block of the grid: impulses to their particles, deficits into the
    // uniform correction, particles moved to their new positions
    __threadfence();
    double dps = 0.0, dph = 0.0, dcnt = 0.0;
    for (int k = 0; k < (int)gridDim.y; ++k) {
        double s[K];
        for (int c = 0; c < K; ++c) s[c] = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            volatile const double* cp = D.cover_part + ((size_t)k * kMaxPartBlocks + b) * K;
            for (int c = 0; c < K; ++c) s[c] += cp[c];
        }
        DevPart& dk = D.parts[k];
        for (int a = 0; a < 3; ++a) {
            dk.imp_f[a] = s[a];
            dk.imp_t[a] = s[3 + a];
            dk.X[a] = dk.Xn[a];
            dk.m[a] = dk.mn[a];
        }
        dps += s[6] + s[9];
        dph += s[7] + s[10];
        dcnt += s[8];
    }
    const long long nf = *D.nfluid + (long long)dcnt;
    *D.nfluid = nf;
    D.corr[0] = dps / (double)nf;
    D.corr[1] = dph / (double)nf;
    *D.cover_ticket = 0u;
}

// ---------------------------------------------------------------------------
// host <-> device field conversion and diagnostics
// ---------------------------------------------------------------------------

// Populations to equilibrium of (rho, u) from FP64 staging; fields from
// staging where given, else the current value plus any pending uniform
// correction.  Solid nodes are left untouched.
template <class C>
__global__ void k_set_fields(DevParams P, DevPtrs D, const double* rho_in, const double* u_in, const double* psi_in,
                             const double* phi_in)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    const size_t N = (size_t)P.N;
    const R rho0 = (R)P.rho0;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        if (D.mask[n]) continue;
        F* psi = (F*)D.psi_dst;
        F* phi = (F*)D.phi_dst;
        F* u = (F*)D.u;
        S* f = (S*)D.f_dst;
        psi[n] = psi_in ? (F)psi_in[n] : (F)((double)psi[n] + D.corr[0]);
        phi[n] = phi_in ? (F)phi_in[n] : (F)((double)phi[n] + D.corr[1]);
        if (u_in) {
            u[n] = (F)u_in[n];
            u[N + n] = (F)u_in[N + n];
            u[2 * N + n] = (F)u_in[2 * N + n];
        }
        double rho;
        if (rho_in) {
            rho = rho_in[n];
        } else {
            R s = 0;
#pragma unroll
            for (int i = 0; i < 19; ++i) s += (R)PopStore<S>::load(f, (size_t)i * N + n, i, rho0);
            rho = (double)s;
        }
        const double ux = (double)u[n], uy = (double)u[N + n], uz = (double)u[2 * N + n];
#pragma unroll
        for (int i = 0; i < 19; ++i)
            PopStore<S>::store(f, (size_t)i * N + n, i, rho0, (R)feq_i<double>(i, rho, ux, uy, uz));
    }
}

// Fields to FP64 staging (zeros at solid nodes).  which: bit0 rho, bit1 u,
// bit2 psi, bit3 phi, bit4 mu (mu_psi to out_rho, mu_phi to out_psi).
template <class C>
__global__ void k_get_fields(DevParams P, DevPtrs D, int which, double* out_rho, double* out_u, double* out_psi,
                             double* out_phi)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    const size_t N = (size_t)P.N;
    const R rho0 = (R)P.rho0;
    const S* f = (const S*)D.f_src;
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    const F* u = (const F*)D.u;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const bool solid = D.mask[n] != 0;
        if (which & 1) {
            R s = 0;
            if (!solid)
#pragma unroll
                for (int i = 0; i < 19; ++i) s += (R)PopStore<S>::load(f, (size_t)i * N + n, i, rho0);
            out_rho[n] = solid ? 0.0 : (double)s;
        }
        if (which & 2)
            for (int a = 0; a < 3; ++a) out_u[a * N + n] = solid ? 0.0 : (double)u[a * N + n];
        if (which & 4) out_psi[n] = solid ? 0.0 : (double)psi[n] + D.corr[0];
        if (which & 8) out_phi[n] = solid ? 0.0 : (double)phi[n] + D.corr[1];
        if (which & 16) {
            out_rho[n] = solid ? 0.0 : (double)((const F*)D.mupsi)[n];
            out_psi[n] = solid ? 0.0 : (double)((const F*)D.muphi)[n];
        }
    }
}

template <class C>
__global__ void k_get_pops(DevParams P, DevPtrs D, double* out, int i)
{
    using R = typename C::real;
    using S = typename C::pop_t;
    const size_t N = (size_t)P.N;
    const S* f = (const S*)D.f_src;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (!D.mask[n]) v = (double)PopStore<S>::load(f, (size_t)i * N + n, i, (R)P.rho0);
        out[n] = v;
    }
}

// Conservation sums, pass 1: per-block FP64 partials of rho, psi, phi over
// fluid nodes.
template <class C>
__global__ void __launch_bounds__(256) k_sums(DevParams P, DevPtrs D, double* part)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    __shared__ double smem[32 * 3];
    const size_t N = (size_t)P.N;
    const R rho0 = (R)P.rho0;
    const S* f = (const S*)D.f_src;
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    double v[3] = {0.0, 0.0, 0.0};
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        if (D.mask[n]) continue;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) s += (double)PopStore<S>::load(f, (size_t)i * N + n, i, rho0);
        v[0] += s;
        v[1] += (double)psi[n] + D.corr[0];
        v[2] += (double)phi[n] + D.corr[1];
    }
    block_sum<3>(v, smem);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = v[k];
}

// pass 2: one thread sums the partials in block order
static __global__ void k_sums_final(const double* part, int nblocks, double* out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < 3; ++k) s[k] += part[b * 3 + k];
    for (int k = 0; k < 3; ++k) out[k] = s[k];
}

// New sphere: claim the fluid nodes strictly inside it (both mask buffers)
// and count them.
static __global__ void k_claim(DevParams P, uint8_t* m0, uint8_t* m1, const DevPart* parts, int p,
                               unsigned long long* count)
{
    const size_t N = (size_t)P.N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        if (m0[n]) continue;
        const int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((size_t)P.nx * P.ny));
        if (inside_sphere(P, parts[p], x, y, z)) {
            m0[n] = (uint8_t)(p + 1);
            m1[n] = (uint8_t)(p + 1);
            atomicAdd(count, 1ull);
        }
    }
}

}  // namespace lbdp
