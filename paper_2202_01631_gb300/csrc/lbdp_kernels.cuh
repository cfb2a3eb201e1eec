// lbdp_kernels.cuh -- the node and particle bodies of the lattice update and
// the particle kernels, templated on the precision configuration.  One step
// of a single box is
//   k_pt_part, k_f_part   per particle: chemical stress and force at the fluid
//                  nodes next to the particle (Eqs. chem_potentials,
//                  free_energy; the link-form divergence)
//   k_links        per particle: bounce-back and chemical-stress momentum sums
//                  over its boundary links, implicit velocity update, new
//                  position and orientation (Sec. "Particles")
//   k_collide_particles  collide-stream of the nodes next to particles: moving
//                  bounce-back plus phoretic slip on their particle links
//   kz_fused       (lbdp_zmarch.cuh) chemical potentials, stress, force and
//                  D3Q19 pull collide-stream of every other fluid node
//   k_scalars_particles  psi/phi transport next to particles, with Janus
//                  production (Eq. activity) and the flux into the moving
//                  surfaces
//   kz_scalars     (lbdp_zmarch.cuh) psi/phi transport (Eq.
//                  diffusion_reaction) and the k_d sink of every other node
//   k_cover_mark   per particle: solid mask at the new positions
//   k_cover_apply  per particle: covering/uncovering and boundary flags; the
//                  last block folds the psi/phi deficits into the uniform
//                  correction and moves the particles
// Every kernel is stencil or streaming work: no tensor cores.  Each body is a
// __device__ function of (parameters, pointers, node), so the single-box
// kernels and the batched kernels (lbdp_batch_kernels.cuh) run the same
// arithmetic.
//
// Precision: node and link arithmetic runs in the mode's real type R.  FP64
// is kept where the method needs it in every mode -- the solid/fluid and
// active-cap decisions (exact, unfused products and sums, as in the CPU
// oracle), the force/torque/conservation sums and the particle solve -- and
// nowhere else, because GB300 executes FP64 (and FP64 conversions) on a narrow
// pipe.
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

constexpr uint8_t kWallSlot = 0xFF;    // slot beyond a non-periodic wall

// ---------------------------------------------------------------------------
// precision accessors
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R corr_r(const DevPtrs& D, int k);
template <>
__device__ __forceinline__ float corr_r<float>(const DevPtrs& D, int k) { return D.corr_f[k]; }
template <>
__device__ __forceinline__ double corr_r<double>(const DevPtrs& D, int k) { return D.corr[k]; }

template <class R>
struct PartR;
template <>
struct PartR<float> {
    template <class Q>
    static __device__ __forceinline__ float U(const Q& q, int a) { return q.Uf[a]; }
    template <class Q>
    static __device__ __forceinline__ float W(const Q& q, int a) { return q.Wf[a]; }
    template <class Q>
    static __device__ __forceinline__ float mu_m(const Q& q) { return q.mu_mf; }
    template <class Q>
    static __device__ __forceinline__ float mu_p(const Q& q) { return q.mu_pf; }
    template <class Q>
    static __device__ __forceinline__ float Hk(const Q& q) { return q.Hk_f; }
    template <class Q>
    static __device__ __forceinline__ float alpha(const Q& q) { return q.alpha_f; }
};
template <>
struct PartR<double> {
    template <class Q>
    static __device__ __forceinline__ double U(const Q& q, int a) { return q.U[a]; }
    template <class Q>
    static __device__ __forceinline__ double W(const Q& q, int a) { return q.W[a]; }
    template <class Q>
    static __device__ __forceinline__ double mu_m(const Q& q) { return q.mu_m; }
    template <class Q>
    static __device__ __forceinline__ double mu_p(const Q& q) { return q.mu_p; }
    template <class Q>
    static __device__ __forceinline__ double Hk(const Q& q) { return q.Hk; }
    template <class Q>
    static __device__ __forceinline__ double alpha(const Q& q) { return q.alpha; }
};

// The fields of one particle that its boundary links use, copied from the
// device record into registers with independent loads (one memory round
// trip), for a kernel that reads them for many links of one node.
struct LinkPart {
    Geo g;
    float mf[3], smarg;
    float Uf[3], Wf[3], mu_pf, mu_mf;
    double m[3], U[3], W[3], mu_p, mu_m;
};

__device__ __forceinline__ LinkPart link_part(const DevPart& q)
{
    LinkPart l;
    l.g = q.g;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        l.mf[a] = q.mf[a];
        l.Uf[a] = q.Uf[a];
        l.Wf[a] = q.Wf[a];
        l.m[a] = q.m[a];
        l.U[a] = q.U[a];
        l.W[a] = q.W[a];
    }
    l.smarg = q.smarg;
    l.mu_pf = q.mu_pf;
    l.mu_mf = q.mu_mf;
    l.mu_p = q.mu_p;
    l.mu_m = q.mu_m;
    return l;
}

// ---------------------------------------------------------------------------
// shared device helpers
// ---------------------------------------------------------------------------

// c_i . (a, b, c) with the zero components of c_i dropped at compile time
// once the direction loop is unrolled (x + (-0) folds to x; a product with 0
// could not be removed because of NaN and signed-zero rules).
template <class R>
__device__ __forceinline__ R cdot(int i, R a, R b, R c)
{
    const R ta = cx(i) == 0 ? (R)-0.0 : (cx(i) > 0 ? a : -a);
    const R tb = cy(i) == 0 ? (R)-0.0 : (cy(i) > 0 ? b : -b);
    const R tc = cz(i) == 0 ? (R)-0.0 : (cz(i) > 0 ? c : -c);
    return ta + tb + tc;
}

// Isotropic gradient of phi at a fluid node, 3 sum_i w_i c_i phi(x+c_i), with
// the node's own value standing in for solid and wall neighbours.
template <class R, class Fld>
__device__ __forceinline__ void grad_phi_at(const int nb[19], const Fld* phi, const uint8_t* mask, R own, R dphi,
                                            R g[3])
{
    g[0] = g[1] = g[2] = (R)0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        int m = nb[i];
        // differences from the node's own value (sum_i w_i c_i = 0)
        const R v = (m < 0 || mask[m]) ? (R)0 : add_x((R)phi[m] + dphi, -own);
        const R w = wgt_r<R>(i);
        if (cx(i) != 0) g[0] = fma_x(cx(i) > 0 ? w : -w, v, g[0]);
        if (cy(i) != 0) g[1] = fma_x(cy(i) > 0 ? w : -w, v, g[1]);
        if (cz(i) != 0) g[2] = fma_x(cz(i) > 0 ? w : -w, v, g[2]);
    }
    g[0] = mul_x(g[0], (R)3);
    g[1] = mul_x(g[1], (R)3);
    g[2] = mul_x(g[2], (R)3);
}

// ---------------------------------------------------------------------------
// geometric decisions.  The oracle takes them in FP64 from exact offsets
// (|x - X|^2 < R^2 for solid nodes, m . r <= 0 for the cap side).  Here they
// are taken in FP32 from the integer/fraction split of the centre (Geo) and
// fall back to the oracle's FP64 arithmetic only when the FP32 value lies
// within its error bound of the threshold, so every decision is the oracle's
// while FP64 (a narrow pipe on GB300) is almost never executed.
// ---------------------------------------------------------------------------

// Integer offsets D of node (x, y, z) from centre g: x - X = D - fr.
__device__ __forceinline__ void int_offset(const DevParams& P, const Geo& g, int x, int y, int z, int D[3])
{
    D[0] = min_image_int(x, g.Xi[0], g.fl[0], P.nx, P.per[0]);
    D[1] = min_image_int(y, g.Xi[1], g.fl[1], P.ny, P.per[1]);
    D[2] = min_image_int(z, g.Xi[2], g.fl[2], P.nz, P.per[2]);
}

// FP32 error margins (host and device): the offset d = D - fr in FP32 is off
// by at most 2^-24 (1 + |d|), so |d|^2 near R^2 is off by less than
// 2^-24 (6 R^2 + 4 R + 1) including the rounding of R^2; m . r is off by less
// than 2^-24 (7 |r| + 2) for |r| <= R + 3.  The margins carry 8x of slack.
__host__ __device__ inline float solid_margin(double R) { return (float)(ldexp(1.0, -21) * (R * R + R + 1.0)); }
__host__ __device__ inline float side_margin(double R) { return (float)(ldexp(1.0, -21) * (R + 4.0)); }

// |x - X|^2 < R^2, the oracle's decision.
__device__ __forceinline__ bool solid_test(const Geo& g, const int D[3], float R2f, float marg, double R2)
{
    const float d0 = (float)D[0] - g.fr[0], d1 = (float)D[1] - g.fr[1], d2 = (float)D[2] - g.fr[2];
    const float q = dot_x(d0, d1, d2, d0, d1, d2);
    if (q < R2f - marg) return true;
    if (q > R2f + marg) return false;
    const double e[3] = {__dsub_rn((double)D[0], g.frd[0]), __dsub_rn((double)D[1], g.frd[1]),
                         __dsub_rn((double)D[2], g.frd[2])};
    return dot3_rn(e, e) < R2;
}

// m . r <= 0 for r = (x - X) + c_i/2 (i = 0: the node itself), the oracle's
// decision (Eq. MuJ, Eq. activity: the cap side takes mu_- and produces).
template <class Q>
__device__ __forceinline__ bool cap_minus(const Q& q, const Geo& g, const int D[3], int i)
{
    const float r0 = ((float)D[0] + 0.5f * (float)cx(i)) - g.fr[0];
    const float r1 = ((float)D[1] + 0.5f * (float)cy(i)) - g.fr[1];
    const float r2 = ((float)D[2] + 0.5f * (float)cz(i)) - g.fr[2];
    const float sd = dot_x(q.mf[0], q.mf[1], q.mf[2], r0, r1, r2);
    if (sd < -q.smarg) return true;
    if (sd > q.smarg) return false;
    const double e[3] = {__dsub_rn(__dadd_rn((double)D[0], 0.5 * cx(i)), g.frd[0]),
                         __dsub_rn(__dadd_rn((double)D[1], 0.5 * cy(i)), g.frd[1]),
                         __dsub_rn(__dadd_rn((double)D[2], 0.5 * cz(i)), g.frd[2])};
    return dot3_rn(q.m, e) <= 0.0;
}

// Link midpoint offset r_b = (x - X) + c_i/2 in the arithmetic precision:
// exact in FP64, within 2^-24 (1 + |r|) in FP32.
template <class R>
__device__ __forceinline__ void link_offset_r(const Geo& g, const int D[3], int i, R r[3]);
template <>
__device__ __forceinline__ void link_offset_r<float>(const Geo& g, const int D[3], int i, float r[3])
{
    r[0] = ((float)D[0] + 0.5f * (float)cx(i)) - g.fr[0];
    r[1] = ((float)D[1] + 0.5f * (float)cy(i)) - g.fr[1];
    r[2] = ((float)D[2] + 0.5f * (float)cz(i)) - g.fr[2];
}
template <>
__device__ __forceinline__ void link_offset_r<double>(const Geo& g, const int D[3], int i, double r[3])
{
    r[0] = __dsub_rn(__dadd_rn((double)D[0], 0.5 * cx(i)), g.frd[0]);
    r[1] = __dsub_rn(__dadd_rn((double)D[1], 0.5 * cy(i)), g.frd[1]);
    r[2] = __dsub_rn(__dadd_rn((double)D[2], 0.5 * cz(i)), g.frd[2]);
}

// Boundary velocity at the midpoint of link x -> x + c_i of particle q:
// u_b = U + Omega x r + v_s, v_s = mu (1 - n n) . grad phi, mu = mu_- where
// m.r <= 0 else mu_+ (Eq. MuJ).  Returns r (midpoint offset), u_b and v_s.
template <class R, class Q>
__device__ __forceinline__ void link_velocity(const DevParams& P, const Q& q, int x, int y, int z, int i,
                                              const R gphi[3], R r[3], R ub[3], R vs[3])
{
    int D[3];
    int_offset(P, q.g, x, y, z, D);
    const R mu = cap_minus(q, q.g, D, i) ? PartR<R>::mu_m(q) : PartR<R>::mu_p(q);
    link_offset_r<R>(q.g, D, i, r);
    const R rn = sqrt(dot_x(r[0], r[1], r[2], r[0], r[1], r[2]));
    const R nh[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    const R ng = dot_x(nh[0], nh[1], nh[2], gphi[0], gphi[1], gphi[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) vs[a] = mul_x(mu, fma_x(-nh[a], ng, gphi[a]));
    const R U0 = PartR<R>::U(q, 0), U1 = PartR<R>::U(q, 1), U2 = PartR<R>::U(q, 2);
    const R W0 = PartR<R>::W(q, 0), W1 = PartR<R>::W(q, 1), W2 = PartR<R>::W(q, 2);
    ub[0] = add_x(add_x(U0, cross_x(W1, r[2], W2, r[1])), vs[0]);
    ub[1] = add_x(add_x(U1, cross_x(W2, r[0], W0, r[2])), vs[1]);
    ub[2] = add_x(add_x(U2, cross_x(W0, r[1], W1, r[0])), vs[2]);
}

// Wetting ghost of psi at the solid neighbour x + c_i of fluid node x,
// psi(x) + (H/kappa) c_i . n_hat at the link midpoint, as its difference
// from psi(x).
template <class R>
__device__ __forceinline__ R psi_ghost_diff(const DevParams& P, const DevPart& q, int x, int y, int z, int i)
{
    if (PartR<R>::Hk(q) == (R)0) return (R)0;
    int D[3];
    int_offset(P, q.g, x, y, z, D);
    R r[3];
    link_offset_r<R>(q.g, D, i, r);
    const R rn = sqrt(dot_x(r[0], r[1], r[2], r[0], r[1], r[2]));
    const R cn = cdot<R>(i, r[0], r[1], r[2]) / rn;
    return mul_x(PartR<R>::Hk(q), cn);
}

// Equilibrium population i of (rho, u) as its deviation from the rest
// equilibrium, f_eq - w_i rho0 =
// w_i [(rho - rho0) + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)], rounding written out.
template <class Real>
__device__ __forceinline__ Real geq_i(int i, Real rho, Real rho0, Real ux, Real uy, Real uz)
{
    const Real cu = cdot<Real>(i, ux, uy, uz);
    const Real uu = dot_x(ux, uy, uz, ux, uy, uz);
    const Real t = fma_x((Real)-1.5, uu, fma_x(mul_x((Real)4.5, cu), cu, mul_x((Real)3, cu)));
    return mul_x(wgt_r<Real>(i), fma_x(rho, t, add_x(rho, -rho0)));
}

__device__ __forceinline__ float tanh_r(float v) { return tanhf(v); }
__device__ __forceinline__ double tanh_r(double v) { return tanh(v); }
__device__ __forceinline__ float rcp_rn(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double rcp_rn(double v) { return __drcp_rn(v); }

// phi0 = phi_b + E tanh psi (Eq. free_energy); with E = 0 it is phi_b and tanh
// is not evaluated.
template <class R>
__device__ __forceinline__ R phi0_of(const PrmR<R>& Q, R ps)
{
    return Q.E != (R)0 ? Q.phib + Q.E * tanh_r(ps) : Q.phib;
}

// Chemical potentials and (optionally) the chemical stress at one fluid node
// from ps = psi(x), d[i] = psi(x + c_i) - psi(x) (ghost-resolved; d[0] is not
// read) and ph = phi(x):
//   mu_psi = A(psi^3 - psi) - kappa lap psi - C E (phi - phi0)/cosh^2 psi,
//   mu_phi = C (phi - phi0),  phi0 = phi_b + E tanh psi          (Eq. chem_potentials)
//   P = p_iso I + kappa grad psi grad psi,
//   p_iso = psi mu_psi + phi mu_phi - f - kappa |grad psi|^2/2,
//   f = A psi^4/4 - A psi^2/2 + C (phi - phi0)^2/2.               (Eq. free_energy)
// P is returned by its four independent numbers: pt = (p_iso, grad psi).
// 1/cosh^2 is taken as 1 - tanh^2; with E = 0, phi0 = phi_b and the
// coupling term vanish, and tanh is not evaluated.  The 19-point Laplacian
// 6 sum_i w_i (psi(x+c_i) - psi(x)) sums the differences per weight class;
// the gradient 3 sum_i w_i c_i psi(x+c_i) sums the differences of opposite
// neighbours.
// Written for FP32: A psi (psi^2 - 1) and f + A/4 = A (psi^2 - 1)^2 / 4 + ...
// do not cancel in the bulk phases, the stencils act on differences, and
// p_iso is returned less the bulk pressure A/4.  A constant part of P exerts
// no force: the link-form divergence sums w_i c_i over all 18 directions of a
// node, and the particle stress sums w_i c_i and w_i r_b x c_i over the
// boundary links of a sphere, which vanish for the same reason.
template <class R>
__device__ __forceinline__ void mu_pressure(const PrmR<R>& Q, R ps, const R d[19], R ph, bool want_p, R& mps,
                                            R& mph, R pt[kPtFields])
{
    // the two weight classes summed in two halves each (shorter chains)
    const R sa = (d[1] + d[2] + d[3]) + (d[4] + d[5] + d[6]);
    const R sd = ((d[7] + d[8]) + (d[9] + d[10]) + (d[11] + d[12])) +
                 ((d[13] + d[14]) + (d[15] + d[16]) + (d[17] + d[18]));
    const R lap = fma_x(sa, (R)(1.0 / 3.0), sd * (R)(1.0 / 6.0));
    // opposite pairs (j, j + 1), j odd: c_j = -c_{j+1}
    R ga[3] = {0, 0, 0}, gd[3] = {0, 0, 0};
#pragma unroll
    for (int j = 1; j < 19; j += 2) {
        const R df = d[j] - d[j + 1];
        R* acc = j < 7 ? ga : gd;
        if (cx(j) != 0) acc[0] += cx(j) > 0 ? df : -df;
        if (cy(j) != 0) acc[1] += cy(j) > 0 ? df : -df;
        if (cz(j) != 0) acc[2] += cz(j) > 0 ? df : -df;
    }
    const R g0 = fma_x(ga[0], (R)(1.0 / 6.0), gd[0] * (R)(1.0 / 12.0));
    const R g1 = fma_x(ga[1], (R)(1.0 / 6.0), gd[1] * (R)(1.0 / 12.0));
    const R g2 = fma_x(ga[2], (R)(1.0 / 6.0), gd[2] * (R)(1.0 / 12.0));
    const R t = fma_x(ps, ps, (R)-1);   // psi^2 - 1
    R dphi;
    if (Q.E != (R)0) {
        const R th = tanh_r(ps);
        dphi = ph - (Q.phib + Q.E * th);
        mps = Q.A * ps * t - Q.kappa * lap - Q.C * Q.E * dphi * ((R)1 - th * th);
    } else {
        dphi = ph - Q.phib;
        mps = Q.A * ps * t - Q.kappa * lap;
    }
    mph = Q.C * dphi;
    if (!want_p) return;
    const R fs = (R)0.25 * Q.A * t * t + (R)0.5 * Q.C * dphi * dphi;   // f + A/4
    const R gg = g0 * g0 + g1 * g1 + g2 * g2;
    pt[0] = ps * mps + ph * mph - fs - (R)0.5 * Q.kappa * gg;   // less A/4
    pt[1] = g0;
    pt[2] = g1;
    pt[3] = g2;
}

// P . c_i of the stress pt = (p_iso, grad psi): p_iso c_i + kappa g (g . c_i).
template <class R>
__device__ __forceinline__ void pt_dot_c(int i, R kappa, const R pt[kPtFields], R out[3])
{
    const R ks = kappa * cdot<R>(i, pt[1], pt[2], pt[3]);
    out[0] = fma_x(ks, pt[1], cx(i) == 0 ? (R)0 : (cx(i) > 0 ? pt[0] : -pt[0]));
    out[1] = fma_x(ks, pt[2], cy(i) == 0 ? (R)0 : (cy(i) > 0 ? pt[0] : -pt[0]));
    out[2] = fma_x(ks, pt[3], cz(i) == 0 ? (R)0 : (cz(i) > 0 ? pt[0] : -pt[0]));
}

// psi(x) (with the correction) and the 18 ghost-resolved differences
// psi(x + c_i) - psi(x) of fluid node n, from global memory.
template <class R, class F>
__device__ __forceinline__ R gather_psi(const DevParams& P, const DevPtrs& D, const F* psi, int x, int y, int z,
                                        const int nb[19], R d[19])
{
    const R p0 = (R)psi[nb[0]];
    d[0] = (R)0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int m = nb[i];
        if (m < 0) {
            d[i] = (R)0;
        } else {
            const uint8_t q = D.mask[m];
            d[i] = q ? psi_ghost_diff<R>(P, D.parts[q - 1], x, y, z, i) : (R)psi[m] - p0;
        }
    }
    return p0 + corr_r<R>(D, 0);
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
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += smem[w * K + threadIdx.x];
        smem[32 * K - K + threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) v[k] = smem[32 * K - K + k];
    __syncthreads();
}

// FP64 block reduction over the threads whose values are not all zero (in the
// particle kernels most threads of a box hold none): those threads write
// their K values as rows, in thread order, into shared memory; G threads per
// value add rows g, g + G, ..., and thread k adds its G partials in order.
// The order depends only on which threads contribute, so the result is
// deterministic.  It is valid in thread 0's v and stays in sm[0..K-1]; sm
// holds block_rows_bytes<K>(blockDim.x) bytes (results, 32 warp counts and
// the G x K partials below sm[256], rows from there).  blockDim.x >= G K.
template <int K>
__host__ __device__ constexpr int block_rows_groups()
{
    return K > 16 ? 4 : 16;
}
template <int K>
__host__ __device__ constexpr size_t block_rows_bytes(int threads)
{
    return (size_t)(256 + threads * K) * sizeof(double);
}

template <int K>
__device__ void block_sum_rows(double (&v)[K], double* sm)
{
    constexpr int G = block_rows_groups<K>();
    static_assert(K <= 64 && G * K <= 176, "reduction layout");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int* wcount = (int*)(sm + 64);
    double* part = sm + 80;
    double* rows = sm + 256;
    bool nz = false;
#pragma unroll
    for (int k = 0; k < K; ++k) nz = nz || (v[k] != 0.0);
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int base = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
        const int c = wcount[w];
        base += w < warp ? c : 0;
        total += c;
    }
    if (nz) {
        double* row = rows + (size_t)(base + __popc(bal & ((1u << lane) - 1u))) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) row[k] = v[k];
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < G * K) {
        const int k = t % K, g = t / K;
        double s = 0.0;
        for (int r = g; r < total; r += G) s += rows[(size_t)r * K + k];
        part[g * K + k] = s;
    }
    __syncthreads();
    if (t < K) {
        double s = 0.0;
#pragma unroll
        for (int g = 0; g < G; ++g) s += part[g * K + t];
        sm[t] = s;
    }
    __syncthreads();
    if (t == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = sm[k];
    __syncthreads();
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
// neighbour access of the stencil bodies.  A body sees node x through an
// accessor: mask(i) is the mask of neighbour x + c_i (kWallSlot beyond a
// wall) and get<k>(i) the value of field k there (own(k) = get<k>(0)).  Where
// mask(i) is not 0 the bodies do not use get<k>(i) except multiplied by 0.
// GAcc reads global memory through the D3Q19 neighbour indices; the
// accessors of lbdp_zmarch.cuh read planes staged in shared memory.  All hand
// the same values to the same arithmetic.
// ---------------------------------------------------------------------------
template <class F, int NF>
struct GAcc {
    int nb[19];
    int n;
    const uint8_t* mk;
    const F* f[NF];
    __device__ __forceinline__ int at(int i) const { return nb[i] >= 0 ? nb[i] : n; }
    __device__ __forceinline__ uint8_t mask(int i) const { return nb[i] >= 0 ? mk[at(i)] : kWallSlot; }
    template <int K>
    __device__ __forceinline__ F get(int i) const
    {
        return f[K][at(i)];
    }
};

// Whether node (x, y, z) lies next to a wall (a non-periodic box face).
__device__ __forceinline__ bool near_wall(const DevParams& P, int x, int y, int z)
{
    return (!P.per[0] && (x == 0 || x == P.nx - 1)) || (!P.per[1] && (y == 0 || y == P.ny - 1)) ||
           (!P.per[2] && (z == 0 || z == P.nz - 1));
}

// ---------------------------------------------------------------------------
// S1: chemical potentials and pressure tensor, one thread per node.  Every
// neighbour load is issued before any decision (walls clamp to the node
// itself), so the loads overlap instead of waiting behind mask branches.
// ---------------------------------------------------------------------------
// Fields of the chemical-potential body: 0 psi, 1 phi.  mup_values returns
// mu_psi, mu_phi and (when P.thermo) the pressure tensor of fluid node
// (x, y, z).
// dps, dph: the uniform psi/phi correction still to be added (corr_r); a
// kernel that loops over many nodes reads them once.
template <class C, class A>
__device__ __forceinline__ void mup_values(const DevParams& P, const DevPtrs& D, int x, int y, int z, const A& a,
                                           typename C::real dps, typename C::real dph, typename C::real& mps,
                                           typename C::real& mph, typename C::real (&pt)[kPtFields])
{
    using R = typename C::real;
    const PrmR<R>& Q = prm<R>(P);
    // differences from psi(x): the uniform correction cancels in them
    R d[19];
    uint8_t mk[19];
    const R p0 = (R)a.template get<0>(0);
    d[0] = (R)0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        mk[i] = a.mask(i);
        d[i] = (R)a.template get<0>(i) - p0;
    }
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (mk[i] == kWallSlot)
            d[i] = (R)0;
        else if (mk[i])
            d[i] = psi_ghost_diff<R>(P, D.parts[mk[i] - 1], x, y, z, i);
    }
    mu_pressure<R>(Q, p0 + dps, d, (R)a.template get<1>(0) + dph, P.thermo != 0, mps, mph, pt);
}

// ---------------------------------------------------------------------------
// S2: force on the fluid, F = g - div P in the link form
//   -6 sum_i w_i [(P(x) + P~_i)/2] . c_i = -3 sum_i w_i P~_i . c_i
// (sum_i w_i c_i = 0), with P~_i = P(x) at solid and wall neighbours, and
// P~_i . c_i = p_iso c_i + kappa g (g . c_i) from the stress (p_iso, g) of
// mu_pressure.
// ---------------------------------------------------------------------------
// fdiv_values returns the force of a fluid node (rounded to the field type, as
// stored); fdiv_compute stores it.  Fields of the accessor: the stress
// (p_iso, g_x, g_y, g_z).
template <class C, class A>
__device__ __forceinline__ void fdiv_values(const DevParams& P, const A& a, typename C::real& Fxo,
                                            typename C::real& Fyo, typename C::real& Fzo)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const PrmR<R>& Q = prm<R>(P);
    R Fx = Q.g[0], Fy = Q.g[1], Fz = Q.g[2];
    if (P.thermo) {
        const R o0 = (R)a.template get<0>(0), o1 = (R)a.template get<1>(0), o2 = (R)a.template get<2>(0);
        const R o3 = (R)a.template get<3>(0);
        R d0 = 0, d1 = 0, d2 = 0;   // sum_i w_i (g . c_i) g
        R e0 = 0, e1 = 0, e2 = 0;   // sum_i w_i c_i p_iso
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const bool own = a.mask(i) != 0;
            const R pi = own ? o0 : (R)a.template get<0>(i);
            const R gx = own ? o1 : (R)a.template get<1>(i);
            const R gy = own ? o2 : (R)a.template get<2>(i);
            const R gz = own ? o3 : (R)a.template get<3>(i);
            const R w = wgt_r<R>(i);
            const R ws = w * cdot<R>(i, gx, gy, gz);
            d0 = fma_x(ws, gx, d0);
            d1 = fma_x(ws, gy, d1);
            d2 = fma_x(ws, gz, d2);
            if (cx(i) != 0) e0 = fma_x(cx(i) > 0 ? w : -w, pi, e0);
            if (cy(i) != 0) e1 = fma_x(cy(i) > 0 ? w : -w, pi, e1);
            if (cz(i) != 0) e2 = fma_x(cz(i) > 0 ? w : -w, pi, e2);
        }
        Fx -= (R)3 * fma_x(Q.kappa, d0, e0);
        Fy -= (R)3 * fma_x(Q.kappa, d1, e1);
        Fz -= (R)3 * fma_x(Q.kappa, d2, e2);
    }
    Fxo = (R)(F)Fx;
    Fyo = (R)(F)Fy;
    Fzo = (R)(F)Fz;
}

template <class C, class A>
__device__ __forceinline__ void fdiv_compute(const DevParams& P, const DevPtrs& D, int n, const A& a)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const size_t N = (size_t)P.N;
    R Fx, Fy, Fz;
    fdiv_values<C>(P, a, Fx, Fy, Fz);
    F* force = (F*)D.force;
    force[n] = (F)Fx;
    force[N + n] = (F)Fy;
    force[2 * N + n] = (F)Fz;
}

template <class C>
__device__ __forceinline__ void fdiv_node(const DevParams& P, const DevPtrs& D, int x, int y, int z)
{
    using F = typename C::fld_t;
    const int n = x + P.nx * (y + P.ny * z);
    if (D.mask[n]) return;
    const size_t N = (size_t)P.N;
    const F* pt = (const F*)D.pt;
    GAcc<F, kPtFields> a;
    neighbours(P, x, y, z, a.nb);
    a.n = n;
    a.mk = D.mask;
#pragma unroll
    for (int k = 0; k < kPtFields; ++k) a.f[k] = pt + k * N;
    fdiv_compute<C>(P, D, n, a);
}

// Rotate the unit vector m by the angle |w| about w (Rodrigues):
//   m' = m cos|w| + (w x m) sin|w|/|w| + w (w . m)(1 - cos|w|)/|w|^2,
// then renormalise.  For |w| < 0.1 both ratios are their Taylor series in
// |w|^2, exact to double precision with six terms; the renormalisation is one
// Newton step of 1/sqrt around 1 (|m'| = 1 up to rounding).
__device__ __forceinline__ void rotate_unit(const double m[3], const double w[3], double out[3])
{
    const double w2 = dot_x(w[0], w[1], w[2], w[0], w[1], w[2]);
    double s1, c1, cw;
    if (w2 < 0.01) {
        s1 = fma_x(-w2 / 6.0, fma_x(-w2 / 20.0, fma_x(-w2 / 42.0, fma_x(-w2 / 72.0, fma_x(-w2 / 110.0, 1.0, 1.0),
                                                                       1.0), 1.0), 1.0), 1.0);
        c1 = 0.5 * fma_x(-w2 / 12.0, fma_x(-w2 / 30.0, fma_x(-w2 / 56.0, fma_x(-w2 / 90.0, fma_x(-w2 / 132.0, 1.0,
                                                                                                  1.0), 1.0), 1.0),
                                        1.0), 1.0);
        cw = fma_x(-w2, c1, 1.0);
    } else {
        const double wn = sqrt(w2);
        s1 = sin(wn) / wn;
        cw = cos(wn);
        c1 = (1.0 - cw) / w2;
    }
    const double wxm[3] = {cross_x(w[1], m[2], w[2], m[1]), cross_x(w[2], m[0], w[0], m[2]),
                           cross_x(w[0], m[1], w[1], m[0])};
    const double wm = mul_x(dot_x(w[0], w[1], w[2], m[0], m[1], m[2]), c1);
    double r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) r[a] = fma_x(w[a], wm, fma_x(wxm[a], s1, mul_x(m[a], cw)));
    const double nn2 = dot_x(r[0], r[1], r[2], r[0], r[1], r[2]);
    const double sc = fma_x(-0.5, nn2, 1.5);
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = mul_x(r[a], sc);
}

// Implicit particle update of particle p by warp 0 of the last block, from
// the link totals tot[0..26] (F0[3], T0[3], zeta upper triangle):
//   (Mdiag + zeta) V(t+1) = Mdiag V(t) + [F0 + impulses + loads; T0 + ...]
// (symmetric positive definite: Cholesky with lane a holding row a), force
// and torque F0 - zeta V, then the position and orientation after the step.
// FP64 throughout; the work is spread over lanes because GB300 issues FP64
// at a low rate.  Ls is scratch for 36 doubles.
static __device__ __noinline__ void particle_update(int3 L3, int3 per3, DevPart* parts, unsigned* ticket, int* err, int p,
                                             const DevPart& q, const double* tot, double* Ls)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    if (lane == 0) ticket[p] = 0u;
    const int a = lane < 6 ? lane : 5;   // lanes >= 6 shadow row 5
    double zrow[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int lo = min(a, c), hi = max(a, c);
        zrow[c] = tot[6 + lo * 6 - (lo * (lo - 1)) / 2 + (hi - lo)];
    }
    const double Ma = a < 3 ? q.M : q.I;
    const double F0a = a < 3 ? add_x(add_x(tot[a], q.imp_f[a]), q.ext_f[a])
                             : add_x(add_x(tot[a], q.imp_t[a - 3]), q.ext_t[a - 3]);
    double xv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) xv[c] = c < 3 ? q.U[c] : q.W[c - 3];
    if (!q.fixed) {
        double Arow[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) Arow[c] = c == a ? add_x(zrow[c], Ma) : zrow[c];
        const double ba = fma_x(Ma, a < 3 ? q.U[a] : q.W[a - 3], F0a);
        // right-looking Cholesky A = L L^T: at step j lane j holds the pivot
        double rs[6];
        bool ok = true;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const double piv = __shfl_sync(full, Arow[j], j);
            ok = ok && (piv > 0.0);
            rs[j] = rsqrt(fmax(piv, 1e-300));
            const double laj = mul_x(Arow[j], rs[j]);   // L[a][j] for a >= j
            if (lane < 6) Ls[a * 6 + j] = laj;
#pragma unroll
            for (int c = j + 1; c < 6; ++c) Arow[c] = fma_x(-laj, __shfl_sync(full, laj, c), Arow[c]);
        }
        __syncwarp();
        // L y = b, then L^T x = y (uniform in the warp; L from shared memory)
        double yv[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            double t = __shfl_sync(full, ba, j);
#pragma unroll
            for (int k = 0; k < j; ++k) t = fma_x(-Ls[j * 6 + k], yv[k], t);
            yv[j] = mul_x(t, rs[j]);
        }
#pragma unroll
        for (int j = 5; j >= 0; --j) {
            double t = yv[j];
#pragma unroll
            for (int k = j + 1; k < 6; ++k) t = fma_x(-Ls[k * 6 + j], xv[k], t);
            xv[j] = mul_x(t, rs[j]);
        }
        if (!ok && lane == 0) atomicOr(err, kErrSolve);
    }
    DevPart& dp = parts[p];
    if (lane == 0) {
        // psi, phi carried into the surface: sum 6 w g c.u_b with u_b at V(t+1)
        double wps = tot[kLinkGpsi + 6], wph = tot[kLinkGphi + 6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            wps = fma_x(tot[kLinkGpsi + c], xv[c], wps);
            wph = fma_x(tot[kLinkGphi + c], xv[c], wph);
        }
        dp.wall_psi = wps;
        dp.wall_phi = wph;
    }
    if (lane < 6) {
        double zv = 0.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) zv = fma_x(zrow[c], xv[c], zv);
        if (a < 3)
            dp.force[a] = add_x(F0a, -zv);
        else
            dp.torque[a - 3] = add_x(F0a, -zv);
    }
    if (lane < 3) {
        const int L = a == 0 ? L3.x : (a == 1 ? L3.y : L3.z);
        const int per = a == 0 ? per3.x : (a == 1 ? per3.y : per3.z);
        const double v = a == 0 ? xv[0] : (a == 1 ? xv[1] : xv[2]);
        const double w = a == 0 ? xv[3] : (a == 1 ? xv[4] : xv[5]);
        dp.U[a] = v;
        dp.W[a] = w;
        dp.Uf[a] = (float)v;
        dp.Wf[a] = (float)w;
        dp.imp_f[a] = 0.0;
        dp.imp_t[a] = 0.0;
        double X = add_x(q.X[a], v);
        if (per) {
            if (X >= L)
                X -= L;
            else if (X < 0.0)
                X += L;
        } else if (X - q.R < 1.0 || X + q.R > L - 2.0) {
            atomicOr(err, kErrWall);
        }
        dp.Xn[a] = X;
        const double f = floor(X);
        const double fr = X - f;
        dp.gn.Xi[a] = (int)f;
        dp.gn.frd[a] = fr;
        dp.gn.fr[a] = (float)fr;
        dp.gn.fl[a] = (fr > 0.0 ? kFrPos : 0) | (fr < 0.5 ? kFrBelowHalf : 0) | (fr > 0.5 ? kFrAboveHalf : 0);
    }
    if (lane == 0) {
        const double w3[3] = {xv[3], xv[4], xv[5]};
        double mn[3] = {q.m[0], q.m[1], q.m[2]};
        if (w3[0] != 0.0 || w3[1] != 0.0 || w3[2] != 0.0) rotate_unit(q.m, w3, mn);
#pragma unroll
        for (int c = 0; c < 3; ++c) dp.mn[c] = mn[c];
    }
}

// ---------------------------------------------------------------------------
// S5 + S6a: link sums and the implicit velocity update.  Grid (nb1, np): the
// blocks of a particle split its link box; the last block of the particle (a
// ticket counter) sums the partials in block order and solves
//   (Mdiag + zeta) V(t+1) = Mdiag V(t) + [F0; T0]
// (symmetric positive definite: Cholesky), then stores the new velocity and
// the position/orientation after the step.
// ---------------------------------------------------------------------------
//
// links_block runs block bi of the nbi blocks of particle p; the block split
// (and with it the summation order) is the same in the single-box and the
// batched kernels, so both give identical bits.  smem holds
// block_rows_bytes<kLinkK>(blockDim.x) bytes; sp and last are block-shared.
template <class C>
__device__ __forceinline__ void links_block(const DevParams& P, const DevPtrs& D, int p, int bi, int nbi,
                                            double* smem, DevPart& sp, bool& last)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    constexpr int K = kLinkK;
    if (threadIdx.x == 0) sp = D.parts[p];
    __syncthreads();
    const DevPart& q = sp;
    const PrmR<R>& Q = prm<R>(P);
    const size_t N = (size_t)P.N;
    const S* fs = (const S*)D.f_src;
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    const R dps = corr_r<R>(D, 0), dph = corr_r<R>(D, 1);
    // floor(X) - ceil(R) <= floor(X - R): the box holds every fluid node within
    // R + 2 of the centre
    const int o[3] = {q.g.Xi[0] - q.Rc - 2, q.g.Xi[1] - q.Rc - 2, q.g.Xi[2] - q.Rc - 2};
    const int tot = P.side1[0] * P.side1[1] * P.side1[2];
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const R zc0 = (R)6 * Q.rho0;
    for (int t = bi * blockDim.x + threadIdx.x; t < tot; t += nbi * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side1, t, x, y, z)) continue;
        const int n = x + P.nx * (y + P.ny * z);
        if (D.mask[n]) continue;
        int nb[19];
        neighbours(P, x, y, z, nb);
        // issue every mask load before deciding anything
        bool lk[19];
        bool have = false;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            lk[i] = nb[i] >= 0 && D.mask[nb[i] >= 0 ? nb[i] : n] == p + 1;
            have = have || lk[i];
        }
        if (!have) continue;
        // this node has links into particle p: load everything it needs at once
        // (the populations as deviations g_i = f_i - w_i rho0: their constant
        // part is added exactly below, so the link terms carry small numbers)
        R fv[19];
#pragma unroll
        for (int i = 1; i < 19; ++i) fv[i] = (R)PopStore<S>::load_dev(fs, (size_t)i * N + n, i, Q.rho0);
        const R ps = (R)psi[n] + dps, ph = (R)phi[n] + dph;
        R gphi[3];
        grad_phi_at<R, F>(nb, phi, D.mask, ph, dph, gphi);
        R pt[kPtFields] = {0, 0, 0, 0};
        if (P.thermo) {
            // the stress the fluid's force used this step
            const F* ptg = (const F*)D.pt;
#pragma unroll
            for (int k = 0; k < kPtFields; ++k) pt[k] = (R)ptg[k * N + n];
        }
        R nacc[K];   // this node's links, added to the FP64 sums once
#pragma unroll
        for (int k = 0; k < K; ++k) nacc[k] = (R)0;
        // sum over this node's links of 36 w_i c_i (integers: 2 c_i on an
        // axis link, c_i on a diagonal one)
        int wc36[3] = {0, 0, 0};
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (!lk[i]) continue;
            wc36[0] += (i < 7 ? 2 : 1) * cx(i);
            wc36[1] += (i < 7 ? 2 : 1) * cy(i);
            wc36[2] += (i < 7 ? 2 : 1) * cz(i);
            R r[3], ub[3], vs[3];
            link_velocity<R>(P, q, x, y, z, i, gphi, r, ub, vs);
            const R fi = fv[i];
            const R w6 = (R)6 * wgt_r<R>(i);
            const R c[3] = {(R)cx(i), (R)cy(i), (R)cz(i)};
            const R cvs = cdot<R>(i, vs[0], vs[1], vs[2]);
            const R mag = fma_x(-mul_x(w6, Q.rho0), cvs, mul_x((R)2, fi));
            R dP[3] = {mul_x(c[0], mag), mul_x(c[1], mag), mul_x(c[2], mag)};
            if (P.thermo) {
                // chemical stress flux through the link, 6 w_i P(x) . c_i
                R pc[3];
                pt_dot_c<R>(i, Q.kappa, pt, pc);
                dP[0] = fma_x(w6, pc[0], dP[0]);
                dP[1] = fma_x(w6, pc[1], dP[1]);
                dP[2] = fma_x(w6, pc[2], dP[2]);
            }
            nacc[0] = add_x(nacc[0], dP[0]);
            nacc[1] = add_x(nacc[1], dP[1]);
            nacc[2] = add_x(nacc[2], dP[2]);
            nacc[3] = add_x(nacc[3], cross_x(r[1], dP[2], r[2], dP[1]));
            nacc[4] = add_x(nacc[4], cross_x(r[2], dP[0], r[0], dP[2]));
            nacc[5] = add_x(nacc[5], cross_x(r[0], dP[1], r[1], dP[0]));
            const R g6[6] = {c[0], c[1], c[2], cross_x(r[1], c[2], r[2], c[1]), cross_x(r[2], c[0], r[0], c[2]),
                             cross_x(r[0], c[1], r[1], c[0])};
            const R zc = mul_x(zc0, wgt_r<R>(i));
            int k = 6;
#pragma unroll
            for (int a = 0; a < 6; ++a)
#pragma unroll
                for (int b = a; b < 6; ++b, ++k) nacc[k] = fma_x(mul_x(zc, g6[a]), g6[b], nacc[k]);
            // scalar flux into the surface, 6 w g(x) c.u_b (finite
            // differences) or g(x) c.u_b on the six D3Q7 links (lattice
            // Boltzmann), with c.u_b = (c, r x c) . V(t+1) + c.v_s
            const R ws = P.scheme ? (i < 7 ? (R)1 : (R)0) : w6;
            const R wps = mul_x(ws, ps), wph = mul_x(ws, ph);
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                nacc[kLinkGpsi + a] = fma_x(wps, g6[a], nacc[kLinkGpsi + a]);
                nacc[kLinkGphi + a] = fma_x(wph, g6[a], nacc[kLinkGphi + a]);
            }
            nacc[kLinkGpsi + 6] = fma_x(wps, cvs, nacc[kLinkGpsi + 6]);
            nacc[kLinkGphi + 6] = fma_x(wph, cvs, nacc[kLinkGphi + 6]);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += (double)nacc[k];
        // The constant parts of the link momentum -- 2 w_i rho0 c_i of the
        // bounced populations and 6 w_i (A/4) c_i of the chemical stress, whose
        // stored isotropic part leaves out the bulk pressure A/4 -- in FP64
        // from the exact counts: the force (2 rho0 + 1.5 A) sum_i w_i c_i and
        // its torque about the centre, (x - X) x that force (the c_i / 2 of
        // each link point is parallel to c_i).  Over the closed surface of a
        // sphere they cancel; they are kept so that every link counts as in
        // the definition, next to other spheres too.
        {
            const PrmR<double>& Qd = prm<double>(P);
            const double kc = (2.0 * Qd.rho0 + (P.thermo ? 1.5 * Qd.A : 0.0)) / 36.0;
            const double fc[3] = {kc * (double)wc36[0], kc * (double)wc36[1], kc * (double)wc36[2]};
            int Dn[3];
            int_offset(P, q.g, x, y, z, Dn);
            const double r0[3] = {__dsub_rn((double)Dn[0], q.g.frd[0]), __dsub_rn((double)Dn[1], q.g.frd[1]),
                                  __dsub_rn((double)Dn[2], q.g.frd[2])};
            acc[0] += fc[0];
            acc[1] += fc[1];
            acc[2] += fc[2];
            acc[3] += cross_x(r0[1], fc[2], r0[2], fc[1]);
            acc[4] += cross_x(r0[2], fc[0], r0[0], fc[2]);
            acc[5] += cross_x(r0[0], fc[1], r0[1], fc[0]);
        }
    }
    block_sum_rows<K>(acc, smem);
    double* part = D.link_part + ((size_t)p * kMaxPartBlocks + bi) * K;
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) part[k] = acc[k];
        __threadfence();
        last = (atomicAdd(D.link_ticket + p, 1u) == (unsigned)nbi - 1u);
    }
    __syncthreads();
    if (!last) return;
    // last block of this particle: thread b loads block b's partials; the
    // row reduction adds them in block order
    __threadfence();
    double sum[K];
#pragma unroll
    for (int k = 0; k < K; ++k) sum[k] = 0.0;
    if ((int)threadIdx.x < nbi) {
        const double* pb = D.link_part + ((size_t)p * kMaxPartBlocks + threadIdx.x) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) sum[k] = __ldcg(pb + k);
    }
    block_sum_rows<K>(sum, smem);   // the totals stay in smem[0..K-1]
    if (threadIdx.x >= 32) return;
    particle_update(make_int3(P.nx, P.ny, P.nz), make_int3(P.per[0], P.per[1], P.per[2]), D.parts, D.link_ticket,
                    D.err, p, q, smem, smem + 64);   // totals in smem[0..K-1], K <= 64
}

// ---------------------------------------------------------------------------
// S3: streaming with bounce-back, BGK collision with Guo forcing
// ---------------------------------------------------------------------------

// BGK collision with Guo forcing of node n from its streamed populations,
// given as deviations g_i = f_i - w_i rho0 (FP32 cancellation in the moments
// would otherwise cost the small velocity its low digits):
//   rho = rho0 + sum g,  j = sum c g  (sum_i w_i c_i = 0),  u = (j + F/2)/rho,
//   g_eq = w [(rho - rho0) + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)],
//   S    = w [3 c.F + 9 (c.u)(c.F) - 3 u.F],
//   g* = (1 - 1/tau) g + g_eq / tau + (1 - 1/(2 tau)) S.
// Opposite directions (j, j+1) share c.u and c.F up to sign, so
//   g_eq/tau + (1 - 1/(2tau)) S = P +- Q  with
//   P = cu (a cu + b cF) + e,  Q = c cu + d cF,
// a = 4.5 w rho / tau, b = 9 w (1 - 1/(2 tau)), c = 3 w rho / tau,
// d = 3 w (1 - 1/(2 tau)), e = w (rho - rho0 - 1.5 rho u^2) / tau
// - 3 w (1 - 1/(2 tau)) u.F, per weight class.  Writes f_dst (as deviations
// through the storage) and u.
template <class C>
__device__ __forceinline__ void collide_store(const PrmR<typename C::real>& Q, const DevPtrs& D, size_t N, int n,
                                              const typename C::real (&gl)[19], typename C::real Fx,
                                              typename C::real Fy, typename C::real Fz)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    S* fd = (S*)D.f_dst + n;
    const int NN = (int)N;   // 19 N < 2^31
    const R rho0 = Q.rho0;
    R dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        dr += gl[j];
        if (cx(j) != 0) jx += cx(j) > 0 ? gl[j] : -gl[j];
        if (cy(j) != 0) jy += cy(j) > 0 ? gl[j] : -gl[j];
        if (cz(j) != 0) jz += cz(j) > 0 ? gl[j] : -gl[j];
    }
    const R rho = rho0 + dr;
    const R ir = rcp_rn(rho);   // IEEE 1 / rho
    const R ux = fma_x((R)0.5, Fx, jx) * ir;
    const R uy = fma_x((R)0.5, Fy, jy) * ir;
    const R uz = fma_x((R)0.5, Fz, jz) * ir;
    const R itau = Q.itau, omf = Q.omf, keep = (R)1 - itau;
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R base = (dr - (R)1.5 * rho * uu) * itau;   // (rho - rho0 - 1.5 rho u^2) / tau
    const R tuF = (R)3 * omf * uF;                    // 3 (1 - 1/(2 tau)) u.F
    // rest direction: w0 (base - 3 (1 - 1/(2 tau)) u.F)
    PopStore<S>::store_dev(fd, 0, 0, rho0, fma_x(gl[0], keep, wgt_r<R>(0) * (base - tuF)));
    const R ri = rho * itau;
    R ka[2], kc[2], ke[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const R w = c == 0 ? wgt_r<R>(1) : wgt_r<R>(7);
        ka[c] = (R)4.5 * w * ri;
        kc[c] = (R)3 * w * ri;
        ke[c] = w * (base - tuF);
    }
    const R kb0 = (R)9 * wgt_r<R>(1) * omf, kb1 = (R)9 * wgt_r<R>(7) * omf;
    const R kd0 = (R)3 * wgt_r<R>(1) * omf, kd1 = (R)3 * wgt_r<R>(7) * omf;
#pragma unroll
    for (int j = 1; j < 19; j += 2) {
        const int c = j < 7 ? 0 : 1;
        const R cu = cdot<R>(j, ux, uy, uz);
        const R cF = cdot<R>(j, Fx, Fy, Fz);
        const R Pp = fma_x(cu, fma_x(ka[c], cu, (c ? kb1 : kb0) * cF), ke[c]);
        const R Qq = fma_x(kc[c], cu, (c ? kd1 : kd0) * cF);
        PopStore<S>::store_dev(fd, j * NN, j, rho0, fma_x(gl[j], keep, Pp + Qq));
        PopStore<S>::store_dev(fd, (j + 1) * NN, j + 1, rho0, fma_x(gl[j + 1], keep, Pp - Qq));
    }
    F* u = (F*)D.u + n;
    u[0] = (F)ux;
    u[NN] = (F)uy;
    u[2 * NN] = (F)uz;
}

// Collide-stream of a fluid node next to a particle (and possibly a wall):
// halfway bounce-back on wall links, moving bounce-back with
// u_b = U + Omega x r + v_s on particle links.  Every load of the node is
// issued before any is used (masks, both candidate sources of each
// population, phi around the node, the force; then the record of the node's
// lowest adjacent particle).  nb and q (the masks of the neighbours) come
// from the caller.
template <class C>
__device__ __forceinline__ void collide_boundary_wide(const DevParams& P, const DevPtrs& D, int x, int y, int z,
                                                      const int (&nb)[19], const uint8_t (&q)[19], int lo)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    const int n = x + P.nx * (y + P.ny * z);
    const PrmR<R>& Q = prm<R>(P);
    const size_t N = (size_t)P.N;
    const int NN = (int)N;
    const S* fs = (const S*)D.f_src;
    const F* force = (const F*)D.force;
    const F* phi = (const F*)D.phi_src;
    const R rho0 = Q.rho0;
    const R dph = corr_r<R>(D, 1);
    const LinkPart lp = link_part(D.parts[lo - 1]);
    const R Fx = (R)force[n], Fy = (R)force[NN + n], Fz = (R)force[2 * NN + n];
    const R phn = (R)phi[n];
    R fl[19], fo[19], pv[19];
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        const int i = opp(j);
        const int m = nb[i] >= 0 ? nb[i] : n;
        fl[j] = (R)PopStore<S>::load_dev(fs, j * NN + (j == 0 ? n : m), j, rho0);
        fo[j] = j == 0 ? (R)0 : (R)PopStore<S>::load_dev(fs, i * NN + n, i, rho0);
        pv[j] = j == 0 ? (R)0 : (R)phi[nb[j] >= 0 ? nb[j] : n];
    }
    // population j arrives from x - c_j = x + c_i (i = opp(j)); from a wall
    // or a particle it is the node's own population i, reflected
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int i = opp(j);
        if (nb[i] < 0 || q[i] != 0) fl[j] = fo[j];
    }
    // grad phi as grad_phi_at, from the values loaded above
    R gphi[3] = {0, 0, 0};
    {
        const R own = phn + dph;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const R v = (nb[i] < 0 || q[i]) ? (R)0 : add_x(pv[i] + dph, -own);
            const R w = wgt_r<R>(i);
            if (cx(i) != 0) gphi[0] = fma_x(cx(i) > 0 ? w : -w, v, gphi[0]);
            if (cy(i) != 0) gphi[1] = fma_x(cy(i) > 0 ? w : -w, v, gphi[1]);
            if (cz(i) != 0) gphi[2] = fma_x(cz(i) > 0 ? w : -w, v, gphi[2]);
        }
        gphi[0] = mul_x(gphi[0], (R)3);
        gphi[1] = mul_x(gphi[1], (R)3);
        gphi[2] = mul_x(gphi[2], (R)3);
    }
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int i = opp(j);
        if (nb[i] < 0 || q[i] == 0) continue;
        R r[3], ub[3], vs[3];
        if (q[i] == lo)
            link_velocity<R>(P, lp, x, y, z, i, gphi, r, ub, vs);
        else
            link_velocity<R>(P, D.parts[q[i] - 1], x, y, z, i, gphi, r, ub, vs);
        const R cub = cdot<R>(i, ub[0], ub[1], ub[2]);
        fl[j] = fma_x(-((R)6 * wgt_r<R>(i) * rho0), cub, fl[j]);
    }
    collide_store<C>(Q, D, N, n, fl, Fx, Fy, Fz);
}

// Pull sources of every population of node (x, y, z) loaded as deviations
// into fl (wrapped on periodic axes, clamped to the node itself beyond a wall,
// where bulk_wall_links replaces them): one memory round trip.
template <class C>
__device__ __forceinline__ void pull_loads(const DevParams& P, const DevPtrs& D, int x, int y, int z,
                                           typename C::real (&fl)[19])
{
    using R = typename C::real;
    using S = typename C::pop_t;
    const int nx = P.nx, ny = P.ny, sxy = nx * ny;
    const int NN = (int)P.N;
    const S* fs = (const S*)D.f_src;
    const R rho0 = prm<R>(P).rho0;
    // source x - c_j of population j as xi[1 - c_jx] + yo[1 - c_jy] + zo[1 - c_jz]
    const int xi[3] = {x > 0 ? x - 1 : (P.per[0] ? nx - 1 : 0), x, x < nx - 1 ? x + 1 : (P.per[0] ? 0 : x)};
    const int yo[3] = {(y > 0 ? y - 1 : (P.per[1] ? ny - 1 : 0)) * nx, y * nx,
                       (y < ny - 1 ? y + 1 : (P.per[1] ? 0 : y)) * nx};
    const int zo[3] = {(z > 0 ? z - 1 : (P.per[2] ? P.nz - 1 : 0)) * sxy, z * sxy,
                       (z < P.nz - 1 ? z + 1 : (P.per[2] ? 0 : z)) * sxy};
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        const int m = xi[1 - cx(j)] + yo[1 - cy(j)] + zo[1 - cz(j)];
        fl[j] = (R)PopStore<S>::load_dev(fs, j * NN + m, j, rho0);
    }
}

// Halfway bounce-back of a bulk node next to a wall: a link whose source lies
// beyond a wall brings back the node's own population of the opposite
// direction.
template <class C>
__device__ __forceinline__ void bulk_wall_links(const DevParams& P, const DevPtrs& D, int x, int y, int z,
                                                typename C::real (&fl)[19])
{
    using R = typename C::real;
    using S = typename C::pop_t;
    const int n = x + P.nx * (y + P.ny * z);
    const int NN = (int)P.N;
    const S* fs = (const S*)D.f_src;
    const bool wx[3] = {!P.per[0] && x == 0, false, !P.per[0] && x == P.nx - 1};
    const bool wy[3] = {!P.per[1] && y == 0, false, !P.per[1] && y == P.ny - 1};
    const bool wz[3] = {!P.per[2] && z == 0, false, !P.per[2] && z == P.nz - 1};
#pragma unroll
    for (int j = 1; j < 19; ++j)
        if (wx[1 - cx(j)] || wy[1 - cy(j)] || wz[1 - cz(j)])
            fl[j] = (R)PopStore<S>::load_dev(fs, opp(j) * NN + n, opp(j), prm<R>(P).rho0);
}

// ---------------------------------------------------------------------------
// S4: psi and phi transport, production and sink, one thread per node
// ---------------------------------------------------------------------------
// Links of fluid node x into particles (transport): no diffusive flux; the
// scalars leave with the boundary velocity of the bounce-back rule,
// c.u_b g(x) -- weighted w_i on the D3Q19 links of the finite-difference
// scheme, 1 on the six D3Q7 links of the lattice-Boltzmann one; Janus
// production on the m.(x - X) <= 0 side of each adjacent particle (any of
// the 18 neighbours).  Out of line (few nodes); adds to the running sums in
// order.
template <class R>
struct LinkSums {
    R sps, sph, src;
};

template <class C>
static __device__ __noinline__ LinkSums<typename C::real> scalars_particle_links(
    const DevParams& P, const DevPtrs& D, int x, int y, int z, typename C::real ps, typename C::real ph,
    typename C::real sps, typename C::real sph)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const F* phi = (const F*)D.phi_src;
    const R dph = corr_r<R>(D, 1);
    int nb[19];
    neighbours(P, x, y, z, nb);
    unsigned long long adj = 0ull;
    R gphi[3];
    grad_phi_at<R, F>(nb, phi, D.mask, ph, dph, gphi);
    for (int i = 1; i < 19; ++i) {
        const int m = nb[i];
        if (m < 0) continue;
        const uint8_t mk = D.mask[m];
        if (!mk) continue;
        adj |= 1ull << (mk - 1);
        if (P.scheme && i >= 7) continue;
        R r[3], ubv[3], vs[3];
        link_velocity<R>(P, D.parts[mk - 1], x, y, z, i, gphi, r, ubv, vs);
        const R cub = cdot<R>(i, ubv[0], ubv[1], ubv[2]);
        const R w = P.scheme ? (R)1 : wgt_r<R>(i);
        sps = fma_x(w, -mul_x(cub, ps), sps);
        sph = fma_x(w, -mul_x(cub, ph), sph);
    }
    R src = 0;
    while (adj) {
        const int k = __ffsll((long long)adj) - 1;
        adj &= adj - 1;
        const DevPart& q = D.parts[k];
        int Di[3];
        int_offset(P, q.g, x, y, z, Di);
        if (cap_minus(q, q.g, Di, 0)) src += PartR<R>::alpha(q);
    }
    return {sps, sph, src};
}

// psi and phi side by side: on sm_100-class GPUs two FP32 values go through
// one packed instruction (each lane rounds as the scalar operation does);
// FP64 keeps two scalar operations.
template <class R>
struct Two {
    R a, b;
};
__device__ __forceinline__ Two<float> fma2(Two<float> x, Two<float> y, Two<float> z)
{
    const float2 r = __ffma2_rn(make_float2(x.a, x.b), make_float2(y.a, y.b), make_float2(z.a, z.b));
    return {r.x, r.y};
}
__device__ __forceinline__ Two<double> fma2(Two<double> x, Two<double> y, Two<double> z)
{
    return {fma_x(x.a, y.a, z.a), fma_x(x.b, y.b, z.b)};
}
__device__ __forceinline__ Two<float> add2(Two<float> x, Two<float> y)
{
    const float2 r = __fadd2_rn(make_float2(x.a, x.b), make_float2(y.a, y.b));
    return {r.x, r.y};
}
__device__ __forceinline__ Two<double> add2(Two<double> x, Two<double> y) { return {add_x(x.a, y.a), add_x(x.b, y.b)}; }

// Lattice-Boltzmann transport (scalar_scheme 1): D3Q7, weights 1/4 (rest)
// and 1/8, c_s^2 = 1/4, relaxation time 1, Gamma = 2M.  The post-collision
// distributions are then the equilibrium of the node's own fields,
//   h_i* = M mu + g c_i.u / 2   (i = 1..6),   h_0* = g - 6 M mu (+ sources),
// so the pull stream needs no stored distributions: the node's new total is
//   g'(x) = h_0*(x) + sum_i  h_i*(x - c_i)          (fluid source)
//                          | h_ibar*(x)              (wall: bounce-back)
//                          | h_ibar*(x) - g(x) c_ibar.u_b   (moving surface)
// with ibar the direction from x to the source.  Written per link from x
// towards y = x + c_j (j = ibar), after taking M mu(x) from each of the six
// terms of h_0*:
//   fluid y: M (mu(y) - mu(x)) - g(y) c_j.u(y) / 2,   otherwise g(x) c_j.u(x) / 2
// and -g(x) c_j.u_b more on a particle link (scalars_particle_links).
template <class C, bool kBoundary, class A>
__device__ __forceinline__ void scalars_compute_lb(const DevParams& P, const DevPtrs& D, int x, int y, int z,
                                                   int n, const A& a, typename C::real dps, typename C::real dph)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const PrmR<R>& Q = prm<R>(P);
    const R ps = (R)a.template get<0>(0) + dps, ph = (R)a.template get<1>(0) + dph;
    const R a0 = (R)a.template get<2>(0), b0 = (R)a.template get<3>(0);
    const R ux = (R)a.template get<4>(0), uy = (R)a.template get<5>(0), uz = (R)a.template get<6>(0);
    const R ma0 = Q.Mpsi * a0, mb0 = Q.Mphi * b0;
    const R hps = (R)0.5 * ps, hph = (R)0.5 * ph;
    R sps = 0, sph = 0;
    bool solid_nb = false;
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const uint8_t mk = a.mask(i);
        const R cu0 = cdot<R>(i, ux, uy, uz);
        const R cu1 = cdot<R>(i, (R)a.template get<4>(i), (R)a.template get<5>(i), (R)a.template get<6>(i));
        const R psm = (R)a.template get<0>(i) + dps, phm = (R)a.template get<1>(i) + dph;
        const R tps = mk ? mul_x(hps, cu0) : fma_x(Q.Mpsi, (R)a.template get<2>(i), -ma0) - (R)0.5 * mul_x(psm, cu1);
        const R tph = mk ? mul_x(hph, cu0) : fma_x(Q.Mphi, (R)a.template get<3>(i), -mb0) - (R)0.5 * mul_x(phm, cu1);
        sps += tps;
        sph += tph;
        solid_nb = solid_nb || (mk != 0 && mk != kWallSlot);
    }
#pragma unroll
    for (int i = 7; i < 19; ++i) {
        const uint8_t mk = a.mask(i);
        solid_nb = solid_nb || (mk != 0 && mk != kWallSlot);
    }
    R hn_src = 0;
    if (solid_nb) {
        if (!kBoundary) return;   // left to k_scalars_particles
        const LinkSums<R> l = scalars_particle_links<C>(P, D, x, y, z, ps, ph, sps, sph);
        sps = l.sps;
        sph = l.sph;
        hn_src = l.src;
    }
    // the stored value plus every increment of the step (correction, fluxes,
    // sink, source) summed first: one rounding of the O(1) field per step
    const R ps0 = (R)a.template get<0>(0), ph0 = (R)a.template get<1>(0);
    const R pn = ps0 + (dps + sps);
    const R hn = ph0 + (((dph + sph) - Q.kd * (ph - phi0_of(Q, ps))) + hn_src);
    ((F*)D.psi_dst)[n] = (F)pn;
    ((F*)D.phi_dst)[n] = (F)hn;
}

// Fields of the transport body: 0 psi, 1 phi, 2 mu_psi, 3 mu_phi, 4..6 u.
// kBoundary: nodes next to a particle are transported here; otherwise they
// are left to k_scalars_particles.
// dps, dph as for mup_values.
template <class C, bool kBoundary, class A>
__device__ __forceinline__ void scalars_compute_c(const DevParams& P, const DevPtrs& D, int x, int y, int z, int n,
                                                  const A& a, typename C::real dps, typename C::real dph)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    if (P.scheme) {
        scalars_compute_lb<C, kBoundary>(P, D, x, y, z, n, a, dps, dph);
        return;
    }
    const PrmR<R>& Q = prm<R>(P);
    const R ps = (R)a.template get<0>(0) + dps, ph = (R)a.template get<1>(0) + dph;
    const R a0 = (R)a.template get<2>(0), b0 = (R)a.template get<3>(0);
    const R ux = (R)a.template get<4>(0), uy = (R)a.template get<5>(0), uz = (R)a.template get<6>(0);
    const R ma0 = Q.Mpsi * a0, mb0 = Q.Mphi * b0;
    const Two<R> g0{ps, ph}, corr{dps, dph}, mob{Q.Mpsi, Q.Mphi}, nmu0{-ma0, -mb0};
    Two<R> sg{0, 0};
    bool solid_nb = false;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const uint8_t mk = a.mask(i);
        const R cu0 = cdot<R>(i, ux, uy, uz);
        const R cu1 = cdot<R>(i, (R)a.template get<4>(i), (R)a.template get<5>(i), (R)a.template get<6>(i));
        const R ub = (R)0.5 * (cu0 + cu1);
        const Two<R> gm = add2(Two<R>{(R)a.template get<0>(i), (R)a.template get<1>(i)}, corr);
        // donor-cell upwind advection, diffusion M (mu(x + c) - mu(x)), for
        // psi and phi together
        // -ub g_upwind = -ua g(x) - ud g(x + c) with ua = max(ub, 0), ud = ub - ua:
        // one of the two products is zero, so this is the single rounding of
        // the upwind term, with a max instead of a compare and two selects
        const R ua = ub > (R)0 ? ub : (R)0, ud = ub - ua;
        Two<R> t = fma2(mob, Two<R>{(R)a.template get<2>(i), (R)a.template get<3>(i)}, nmu0);
        t = fma2(Two<R>{-ud, -ud}, gm, t);
        t = fma2(Two<R>{-ua, -ua}, g0, t);
        // links to walls and particles carry no flux here (particle links are
        // handled below)
        const R w = wgt_r<R>(i);
        sg = fma2(Two<R>{w, w}, mk ? Two<R>{0, 0} : t, sg);
        solid_nb = solid_nb || (mk != 0 && mk != kWallSlot);
    }
    R sps = sg.a, sph = sg.b;
    R hn_src = 0;
    if (solid_nb) {
        if (!kBoundary) return;   // left to k_scalars_particles
        const LinkSums<R> l = scalars_particle_links<C>(P, D, x, y, z, ps, ph, sps, sph);
        sps = l.sps;
        sph = l.sph;
        hn_src = l.src;
    }
    // the stored value plus every increment of the step (correction, fluxes,
    // sink, source) summed first: one rounding of the O(1) field per step
    const R ps0 = (R)a.template get<0>(0), ph0 = (R)a.template get<1>(0);
    const R pn = ps0 + fma_x((R)6, sps, dps);
    const R hn = ph0 + ((fma_x((R)6, sph, dph) - Q.kd * (ph - phi0_of(Q, ps))) + hn_src);
    ((F*)D.psi_dst)[n] = (F)pn;
    ((F*)D.phi_dst)[n] = (F)hn;
}

template <class C, bool kBoundary = true, class A>
__device__ __forceinline__ void scalars_compute(const DevParams& P, const DevPtrs& D, int x, int y, int z, int n,
                                                const A& a)
{
    using R = typename C::real;
    scalars_compute_c<C, kBoundary>(P, D, x, y, z, n, a, corr_r<R>(D, 0), corr_r<R>(D, 1));
}

template <class C>
__device__ __forceinline__ void scalars_node(const DevParams& P, const DevPtrs& D, int x, int y, int z)
{
    using F = typename C::fld_t;
    const int n = x + P.nx * (y + P.ny * z);
    if (D.mask[n]) return;
    const size_t N = (size_t)P.N;
    GAcc<F, 7> a;
    neighbours(P, x, y, z, a.nb);
    a.n = n;
    a.mk = D.mask;
    a.f[0] = (const F*)D.psi_src;
    a.f[1] = (const F*)D.phi_src;
    a.f[2] = (const F*)D.mupsi;
    a.f[3] = (const F*)D.muphi;
    a.f[4] = (const F*)D.u;
    a.f[5] = (const F*)D.u + N;
    a.f[6] = (const F*)D.u + 2 * N;
    scalars_compute<C>(P, D, x, y, z, n, a);
}

// ---------------------------------------------------------------------------
// S7: covering / uncovering.  The cover box of particle p holds its old and
// new position with a margin that contains every neighbour of a node that can
// change.  k_cover_mark writes the new mask of the box (ownership over all
// particles at their new positions, first match); k_cover_apply moves the
// fields of the changed nodes, refreshes the boundary flags of the box and
// sums what the moving surfaces carried out of the fluid.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cover_origin(const DevParams& P, const DevPart& q, int o[3])
{
    for (int a = 0; a < 3; ++a) {
        const int L = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
        const int i0 = q.g.Xi[a], i1 = q.gn.Xi[a];
        int lo = min(i0, i1);
        // on a periodic axis the two centres may sit on opposite sides of the
        // wrap; take the lower end of the shorter arc
        if (P.per[a] && abs(i0 - i1) > L / 2) lo = max(i0, i1);
        // floor(lo) - ceil(R) <= floor(lo - R): the box starts at or below the
        // lowest node that can change or neighbour a change
        o[a] = lo - q.Rc - 3;
    }
}

template <class C>
__device__ __forceinline__ void cover_mark_block(const DevParams& P, const DevPtrs& D, int p, int bi, int nbi)
{
    const DevPart& q = D.parts[p];
    int o[3];
    cover_origin(P, q, o);
    const int tot = P.side2[0] * P.side2[1] * P.side2[2];
    for (int t = bi * blockDim.x + threadIdx.x; t < tot; t += nbi * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side2, t, x, y, z)) continue;
        uint8_t own = 0;
        for (int k = 0; k < P.np; ++k) {
            const DevPart& qk = D.parts[k];
            int Dk[3];
            int_offset(P, qk.gn, x, y, z, Dk);
            if (solid_test(qk.gn, Dk, qk.R2f, qk.rmarg, qk.R2)) {
                own = (uint8_t)(k + 1);
                break;
            }
        }
        D.mask_next[x + P.nx * (y + P.ny * z)] = own;
    }
}

//
// cover_apply_block runs block bi of the nbi blocks of particle p; the last of
// the np * nbi blocks of the box (a ticket) finishes the step for all
// particles of the box.  smem holds block_rows_bytes<kCoverK>(blockDim.x)
// bytes.
template <class C>
__device__ __forceinline__ void cover_apply_block(const DevParams& P, const DevPtrs& D, int p, int bi, int nbi,
                                                  double* smem, bool& last)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    using S = typename C::pop_t;
    constexpr int K = kCoverK;
    const DevPart& q = D.parts[p];
    const size_t N = (size_t)P.N;
    int o[3];
    cover_origin(P, q, o);
    const int tot = P.side2[0] * P.side2[1] * P.side2[2];
    S* f = (S*)D.f_dst;
    F* psi = (F*)D.psi_dst;
    F* phi = (F*)D.phi_dst;
    F* u = (F*)D.u;
    const R rho0 = prm<R>(P).rho0;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int t = bi * blockDim.x + threadIdx.x; t < tot; t += nbi * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side2, t, x, y, z)) continue;
        const int n = x + P.nx * (y + P.ny * z);
        const uint8_t ob = D.mask[n], nw = D.mask_next[n];
        int nb[19];
        neighbours(P, x, y, z, nb);
        // boundary flag for the next step (fluid node with a solid neighbour);
        // all mask loads first
        bool adj = false;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int m = nb[i] >= 0 ? nb[i] : n;
            adj = adj || (nb[i] >= 0 && D.mask_next[m]);
        }
        D.bflag[n] = (!nw && adj) ? 1 : 0;
        if (ob == nw) continue;
        if (ob == 0 && nw == p + 1) {
            // covered: the particle takes the momentum the node's populations
            // carry; psi, phi are removed
            R jr[3] = {0, 0, 0};
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                const R fi = (R)PopStore<S>::load_dev(f, (size_t)i * N + n, i, rho0);   // sum c f = sum c g
                if (cx(i) != 0) jr[0] = cx(i) > 0 ? add_x(jr[0], fi) : add_x(jr[0], -fi);
                if (cy(i) != 0) jr[1] = cy(i) > 0 ? add_x(jr[1], fi) : add_x(jr[1], -fi);
                if (cz(i) != 0) jr[2] = cz(i) > 0 ? add_x(jr[2], fi) : add_x(jr[2], -fi);
            }
            const double j[3] = {(double)jr[0], (double)jr[1], (double)jr[2]};
            int Dn[3];
            int_offset(P, q.gn, x, y, z, Dn);
            const double r[3] = {__dsub_rn((double)Dn[0], q.gn.frd[0]), __dsub_rn((double)Dn[1], q.gn.frd[1]),
                                 __dsub_rn((double)Dn[2], q.gn.frd[2])};
            acc[0] += j[0];
            acc[1] += j[1];
            acc[2] += j[2];
            acc[3] += cross_x(r[1], j[2], r[2], j[1]);
            acc[4] += cross_x(r[2], j[0], r[0], j[2]);
            acc[5] += cross_x(r[0], j[1], r[1], j[0]);
            acc[6] += (double)psi[n];
            acc[7] += (double)phi[n];
            acc[8] -= 1.0;
        } else if (ob == p + 1 && nw == 0) {
            // uncovered: equilibrium at the boundary velocity with the mean
            // density of neighbours fluid before and after; psi, phi = means
            R rb = 0, pb = 0, hb = 0;
            int cnt = 0;
            for (int i = 1; i < 19; ++i) {
                const int m = nb[i];
                if (m < 0 || D.mask[m] || D.mask_next[m]) continue;
                R rm = 0;   // rho - rho0 = sum g
#pragma unroll
                for (int k = 0; k < 19; ++k) rm = add_x(rm, (R)PopStore<S>::load_dev(f, (size_t)k * N + m, k, rho0));
                rb = add_x(rb, add_x(rho0, rm));
                pb = add_x(pb, (R)psi[m]);
                hb = add_x(hb, (R)phi[m]);
                ++cnt;
            }
            if (cnt == 0) {
                atomicOr(D.err, kErrOverlap);
                rb = rho0;
                pb = hb = 0;
            } else {
                rb = rb / (R)cnt;
                pb = pb / (R)cnt;
                hb = hb / (R)cnt;
            }
            int Dn[3];
            int_offset(P, q.gn, x, y, z, Dn);
            R r[3];
            link_offset_r<R>(q.gn, Dn, 0, r);
            const R U0 = PartR<R>::U(q, 0), U1 = PartR<R>::U(q, 1), U2 = PartR<R>::U(q, 2);
            const R W0 = PartR<R>::W(q, 0), W1 = PartR<R>::W(q, 1), W2 = PartR<R>::W(q, 2);
            const R ub[3] = {add_x(U0, cross_x(W1, r[2], W2, r[1])), add_x(U1, cross_x(W2, r[0], W0, r[2])),
                             add_x(U2, cross_x(W0, r[1], W1, r[0]))};
#pragma unroll
            for (int i = 0; i < 19; ++i)
                PopStore<S>::store_dev(f, (size_t)i * N + n, i, rho0, geq_i<R>(i, rb, rho0, ub[0], ub[1], ub[2]));
            u[n] = (F)ub[0];
            u[N + n] = (F)ub[1];
            u[2 * N + n] = (F)ub[2];
            psi[n] = (F)pb;
            phi[n] = (F)hb;
            const double j[3] = {(double)mul_x(rb, ub[0]), (double)mul_x(rb, ub[1]), (double)mul_x(rb, ub[2])};
            const double rd[3] = {(double)r[0], (double)r[1], (double)r[2]};
            acc[0] -= j[0];
            acc[1] -= j[1];
            acc[2] -= j[2];
            acc[3] -= cross_x(rd[1], j[2], rd[2], j[1]);
            acc[4] -= cross_x(rd[2], j[0], rd[0], j[2]);
            acc[5] -= cross_x(rd[0], j[1], rd[1], j[0]);
            acc[6] -= (double)psi[n];
            acc[7] -= (double)phi[n];
            acc[8] += 1.0;
        } else if (ob == p + 1) {
            atomicOr(D.err, kErrOverlap);   // passed straight into another sphere
        }
    }
    block_sum_rows<K>(acc, smem);
    double* part = D.cover_part + ((size_t)p * kMaxPartBlocks + bi) * K;
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) part[k] = acc[k];
        __threadfence();
        last = (atomicAdd(D.cover_ticket, 1u) == (unsigned)(nbi * P.np) - 1u);
    }
    __syncthreads();
    if (!last) return;
    // last block of the grid: per particle, thread b loads block b's partials
    // and the block reduction adds them in a fixed order; impulses go to their
    // particles, deficits into the uniform correction, particles move
    __threadfence();
    double dsum_psi = 0.0, dsum_phi = 0.0, dcnt = 0.0;
    for (int k = 0; k < P.np; ++k) {
        double s[K];
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = 0.0;
        if ((int)threadIdx.x < nbi) {
            const double* cp = D.cover_part + ((size_t)k * kMaxPartBlocks + threadIdx.x) * K;
#pragma unroll
            for (int c = 0; c < K; ++c) s[c] = __ldcg(cp + c);
        }
        block_sum_rows<K>(s, smem);
        if (threadIdx.x == 0) {
            DevPart& dk = D.parts[k];
            for (int a = 0; a < 3; ++a) {
                dk.imp_f[a] = s[a];
                dk.imp_t[a] = s[3 + a];
                dk.X[a] = dk.Xn[a];
                dk.m[a] = dk.mn[a];
                dk.mf[a] = (float)dk.mn[a];
            }
            dk.g = dk.gn;
            dsum_psi += s[6] + dk.wall_psi;
            dsum_phi += s[7] + dk.wall_phi;
            dcnt += s[8];
        }
    }
    if (threadIdx.x != 0) return;
    const long long nf = *D.nfluid + (long long)dcnt;
    *D.nfluid = nf;
    D.corr_next[0] = dsum_psi / (double)nf;
    D.corr_next[1] = dsum_phi / (double)nf;
    D.corr_f_next[0] = (float)D.corr_next[0];
    D.corr_f_next[1] = (float)D.corr_next[1];
    *D.cover_ticket = 0u;
}

// ---------------------------------------------------------------------------
// particle kernels of the single box: grid (blocks per particle, particles)
// (the bulk kernels of the single box are in lbdp_zmarch.cuh)
// ---------------------------------------------------------------------------
// Collide-stream of the fluid nodes next to particles, beside the bulk kernel
// (which leaves them out).  These nodes read the particle records and their
// neighbours' masks in chains of dependent loads; inside the bulk kernel,
// under its full memory load and register budget, each such chain would hold
// its block long after the others finish.  Block (b, p) walks the link box of particle
// p; a node next to several particles is collided by the lowest of them.
template <class C>
__device__ __forceinline__ void collide_particles_block(const DevParams& P, const DevPtrs& D, int p, int bi, int nbi)
{
    const DevPart& q = D.parts[p];
    const int o[3] = {q.g.Xi[0] - q.Rc - 2, q.g.Xi[1] - q.Rc - 2, q.g.Xi[2] - q.Rc - 2};
    const int tot = P.side1[0] * P.side1[1] * P.side1[2];
    for (int t = bi * blockDim.x + threadIdx.x; t < tot; t += nbi * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side1, t, x, y, z)) continue;
        const int n = x + P.nx * (y + P.ny * z);
        if (D.mask[n] || !D.bflag[n]) continue;
        int nb[19];
        neighbours(P, x, y, z, nb);
        uint8_t qm[19];
        qm[0] = 0;
        int lo = 256;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            qm[i] = nb[i] >= 0 ? D.mask[nb[i]] : (uint8_t)0;
            if (qm[i] != 0 && qm[i] < lo) lo = qm[i];
        }
        if (lo != p + 1) continue;
        collide_boundary_wide<C>(P, D, x, y, z, nb, qm, lo);
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_collide_particles(const __grid_constant__ DevParams P,
                                                                     const __grid_constant__ DevPtrs D)
{
    collide_particles_block<C>(P, D, blockIdx.y, blockIdx.x, gridDim.x);
}

// Transport of the fluid nodes next to particles, beside kz_scalars (which
// leaves them out), for the same reason and with the same split as
// k_collide_particles.
template <class C>
__device__ __forceinline__ void scalars_particles_block(const DevParams& P, const DevPtrs& D, int p, int bi, int nbi)
{
    const DevPart& q = D.parts[p];
    const int o[3] = {q.g.Xi[0] - q.Rc - 2, q.g.Xi[1] - q.Rc - 2, q.g.Xi[2] - q.Rc - 2};
    const int tot = P.side1[0] * P.side1[1] * P.side1[2];
    for (int t = bi * blockDim.x + threadIdx.x; t < tot; t += nbi * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, P.side1, t, x, y, z)) continue;
        const int n = x + P.nx * (y + P.ny * z);
        if (D.mask[n] || !D.bflag[n]) continue;
        int nb[19];
        neighbours(P, x, y, z, nb);
        int lo = 256;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int m = nb[i] >= 0 ? D.mask[nb[i]] : 0;
            if (m != 0 && m < lo) lo = m;
        }
        if (lo != p + 1) continue;
        scalars_node<C>(P, D, x, y, z);
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_scalars_particles(const __grid_constant__ DevParams P,
                                                                     const __grid_constant__ DevPtrs D)
{
    scalars_particles_block<C>(P, D, blockIdx.y, blockIdx.x, gridDim.x);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads, 1) k_links(DevParams P, DevPtrs D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];   // block_rows_bytes<kLinkK>(kPartThreads)
    __shared__ DevPart sp;
    __shared__ bool last;
    links_block<C>(P, D, blockIdx.y, blockIdx.x, gridDim.x, (double*)smem_raw, sp, last);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_cover_mark(DevParams P, DevPtrs D)
{
    cover_mark_block<C>(P, D, blockIdx.y, blockIdx.x, gridDim.x);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_cover_apply(DevParams P, DevPtrs D)
{
    __shared__ double smem[block_rows_bytes<kCoverK>(kPartThreads) / sizeof(double)];
    __shared__ bool last;
    cover_apply_block<C>(P, D, blockIdx.y, blockIdx.x, gridDim.x, smem, last);
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
    const R rho0 = prm<R>(P).rho0;
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
            R s = 0;   // rho - rho0
#pragma unroll
            for (int i = 0; i < 19; ++i) s += (R)PopStore<S>::load_dev(f, (size_t)i * N + n, i, rho0);
            rho = P.rho0 + (double)s;
        }
        const double ux = (double)u[n], uy = (double)u[N + n], uz = (double)u[2 * N + n];
#pragma unroll
        for (int i = 0; i < 19; ++i)
            PopStore<S>::store_dev(f, (size_t)i * N + n, i, rho0, (R)geq_i<double>(i, rho, P.rho0, ux, uy, uz));
    }
}

// Chemical potentials of the current fields (for the readout only).
template <class C>
__global__ void k_mu_now(DevParams P, DevPtrs D)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const size_t N = (size_t)P.N;
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    const R dph = corr_r<R>(D, 1);
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        R mps = 0, mph = 0;
        if (!D.mask[n]) {
            const int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((size_t)P.nx * P.ny));
            int nb[19];
            neighbours(P, x, y, z, nb);
            R d[19], pt[kPtFields];
            const R ps = gather_psi<R, F>(P, D, psi, x, y, z, nb, d);
            mu_pressure<R>(prm<R>(P), ps, d, (R)phi[n] + dph, false, mps, mph, pt);
        }
        ((F*)D.mupsi)[n] = (F)mps;
        ((F*)D.muphi)[n] = (F)mph;
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
    const R rho0 = prm<R>(P).rho0;
    const S* f = (const S*)D.f_src;
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    const F* u = (const F*)D.u;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const bool solid = D.mask[n] != 0;
        if (which & 1) {
            R s = 0;   // rho - rho0
            if (!solid)
#pragma unroll
                for (int i = 0; i < 19; ++i) s += (R)PopStore<S>::load_dev(f, (size_t)i * N + n, i, rho0);
            out_rho[n] = solid ? 0.0 : P.rho0 + (double)s;
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
        if (!D.mask[n]) v = (double)PopStore<S>::load(f, (size_t)i * N + n, i, prm<R>(P).rho0);
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
    const R rho0 = prm<R>(P).rho0;
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

// Boundary flags of every node from a mask: fluid node with a solid neighbour.
static __global__ void k_bflag_all(DevParams P, const uint8_t* mask, uint8_t* bflag)
{
    const size_t N = (size_t)P.N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((size_t)P.nx * P.ny));
        bool adj = false;
        if (!mask[n]) {
            int nb[19];
            neighbours(P, x, y, z, nb);
            for (int i = 1; i < 19; ++i) adj = adj || (nb[i] >= 0 && mask[nb[i]]);
        }
        bflag[n] = adj ? 1 : 0;
    }
}

}  // namespace lbdp
