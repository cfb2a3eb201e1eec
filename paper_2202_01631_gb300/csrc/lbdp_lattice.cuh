// lbdp_lattice.cuh -- D3Q19 lattice, device-side state layout and geometric
// helpers of the GB300 lattice Boltzmann library.
//
// Layout in HBM (one box):
//   populations  f[2][19][N]   storage type of the precision mode, pull scheme,
//                              double buffered (read f[cur], write f[cur^1]);
//   psi, phi     [2][N]        field type, double buffered;
//   mu_psi, mu_phi, u[3]       [N] each, field type;
//   mask         [2][N] u8     0 fluid, k+1 inside particle k, double buffered;
//   particles    DevPart[np]   FP64 state.
// Node index n = x + nx*(y + ny*z): x is the fastest axis, so a warp reads
// 32 consecutive nodes of one population row (coalesced 128/256-byte lines).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbdp {

constexpr int kMaxParticles = 64;
// The chemical pressure tensor P = p_iso I + kappa grad psi grad psi of a node
// is kept as its four independent numbers (p_iso, grad psi).
constexpr int kPtFields = 4;

// Arithmetic with its rounding written out.  The particle sums and solve,
// the boundary velocities and the refill of uncovered nodes are inlined into
// the single-box and the batched kernels; with every multiply-add fused or
// not fused in the source the compiler has no choice left, and both give the
// same bits.
__device__ __forceinline__ double fma_x(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_x(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_x(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_x(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_x(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_x(float a, float b) { return __fadd_rn(a, b); }
// a b - c d
template <class R>
__device__ __forceinline__ R cross_x(R a, R b, R c, R d)
{
    return fma_x(a, b, -mul_x(c, d));
}
// a . b of 3-vectors
template <class R>
__device__ __forceinline__ R dot_x(R a0, R a1, R a2, R b0, R b1, R b2)
{
    return fma_x(a0, b0, fma_x(a1, b1, mul_x(a2, b2)));
}

// ---------------------------------------------------------------------------
// D3Q19 (order given in include/lbdp.h)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i)
{
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cy(int i)
{
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int cz(int i)
{
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// Weights and their reciprocals in a given precision: selecting among
// constants of that type keeps FP64 out of FP32 code even where a loop over
// the directions is not unrolled.
template <class R>
__host__ __device__ constexpr R wgt_r(int i)
{
    return i == 0 ? (R)(1.0 / 3.0) : (i < 7 ? (R)(1.0 / 18.0) : (R)(1.0 / 36.0));
}
template <class R>
__host__ __device__ constexpr R inv_wgt_r(int i)
{
    return i == 0 ? (R)3 : (i < 7 ? (R)18 : (R)36);
}

// ---------------------------------------------------------------------------
// parameters and particles
// ---------------------------------------------------------------------------
// Model parameters in the arithmetic precision of a kernel.  Both copies are
// filled on the host, so an FP32 kernel never converts from FP64 (GB300 runs
// FP64, conversions included, on a narrow pipe).
template <class R>
struct PrmR {
    R itau, omf;          // 1/tau, 1 - 1/(2 tau)
    R rho0, g[3];
    R A, kappa, Mpsi, C, Mphi, E, phib, kd, inv_kappa;
};

struct DevParams {
    int nx, ny, nz;
    int per[3];
    long long N;
    int np;
    int thermo;
    int scheme;     // psi/phi transport: 0 finite differences, 1 D3Q7 lattice Boltzmann
    double tau, rho0;
    double g[3];
    double A, kappa, Mpsi, C, Mphi, E, phib, kd;
    PrmR<float> pf;
    PrmR<double> pd;
    int side1[3];   // link box edge per axis (clamped to the box on periodic axes)
    int side2[3];   // cover box edge per axis
    int nb1, nb2;   // blocks per particle of the link and cover kernels
};

template <class R>
__host__ __device__ __forceinline__ const PrmR<R>& prm(const DevParams& P);
template <>
__host__ __device__ __forceinline__ const PrmR<float>& prm<float>(const DevParams& P) { return P.pf; }
template <>
__host__ __device__ __forceinline__ const PrmR<double>& prm<double>(const DevParams& P) { return P.pd; }

template <class R>
inline void fill_prm(PrmR<R>& q, const DevParams& P)
{
    q.itau = (R)(1.0 / P.tau);
    q.omf = (R)(1.0 - 0.5 / P.tau);
    q.rho0 = (R)P.rho0;
    for (int a = 0; a < 3; ++a) q.g[a] = (R)P.g[a];
    q.A = (R)P.A;
    q.kappa = (R)P.kappa;
    q.Mpsi = (R)P.Mpsi;
    q.C = (R)P.C;
    q.Mphi = (R)P.Mphi;
    q.E = (R)P.E;
    q.phib = (R)P.phib;
    q.kd = (R)P.kd;
    q.inv_kappa = P.kappa > 0.0 ? (R)(1.0 / P.kappa) : (R)0;
}

// A sphere centre X split for the geometric decisions: X = Xi + fr with
// Xi = floor(X) and fr in [0, 1) exact in FP64 (frd) and rounded to FP32
// (fr).  Offsets x - X of lattice nodes are then D - fr with an integer D, and
// the periodic minimum image of the oracle (a shift by L when |x - X| > L/2)
// is an integer decision once fr is compared with 0 and 1/2 (fl).
enum : int { kFrPos = 1, kFrBelowHalf = 2, kFrAboveHalf = 4 };
struct Geo {
    int Xi[3];
    int fl[3];
    double frd[3];
    float fr[3];
    float pad;
};

__host__ __device__ inline void fill_geo(const double X[3], Geo& g)
{
    for (int a = 0; a < 3; ++a) {
        const double f = floor(X[a]);
        const double fr = X[a] - f;   // exact
        g.Xi[a] = (int)f;
        g.frd[a] = fr;
        g.fr[a] = (float)fr;
        g.fl[a] = (fr > 0.0 ? kFrPos : 0) | (fr < 0.5 ? kFrBelowHalf : 0) | (fr > 0.5 ? kFrAboveHalf : 0);
    }
    g.pad = 0.f;
}

struct DevPart {
    double X[3], U[3], W[3], m[3];   // position, velocity, spin, unit vector
    double Xn[3], mn[3];             // position and unit vector after this step
    Geo g, gn;                       // X and Xn split for the geometric decisions
    float Uf[3], Wf[3];              // U, W in FP32 for the FP32 link arithmetic
    float mf[3];                     // m in FP32
    float R2f, rmarg, smarg;         // R^2 in FP32; FP32 error margins of the
                                     // solid test and of the cap-side test
    float alpha_f, mu_pf, mu_mf, Hk_f;
    double R, R2, M, I, alpha, mu_p, mu_m, H;
    int Rc;                          // ceil(R)
    int pad0;
    double Hk;                       // H / kappa of the wetting ghost
    double ext_f[3], ext_t[3];
    double imp_f[3], imp_t[3];       // covering impulses, applied in the next step
    double force[3], torque[3];
    double wall_psi, wall_phi;       // psi, phi carried into the surface this step
    int fixed;
    int pad;
};

// Device error word bits (reported by lb_sync and the reads).
enum : int {
    kErrOverlap = 1,   // a node passed between particles / no fluid neighbour
    kErrWall = 2,      // a particle came within one node of a wall
    kErrSolve = 4,     // singular particle velocity system
};

// per-block link partials: F0[3], T0[3], zeta upper triangle [21], then the
// coefficients of the scalar flux into the surface, linear in V(t+1):
// sum 6 w psi (c, r x c) [6], sum 6 w psi c.v_s, and the same for phi
constexpr int kLinkK = 41;
constexpr int kLinkGpsi = 27, kLinkGphi = 34;
static_assert(kLinkK <= 64, "the particle update keeps its scratch at smem + 64");
constexpr int kCoverK = 9;    // per-block cover partials: impulse F[3], T[3], dpsi, dphi,
                              // dcount
constexpr int kMaxPartBlocks = 128;

// Raw device pointers of one step (type-erased storage).
struct DevPtrs {
    const void* f_src;
    void* f_dst;
    const void* psi_src;
    void* psi_dst;
    const void* phi_src;
    void* phi_dst;
    void* mupsi;
    void* muphi;
    void* pt;             // [kPtFields][N] chemical stress: p_iso (less A/4), grad psi
    void* force;          // [3][N] force on the fluid, g - div P
    void* u;
    const uint8_t* mask;
    uint8_t* mask_next;
    uint8_t* bflag;       // [N] 1 = fluid node with a solid neighbour
    DevPart* parts;
    double* corr;         // [2]: uniform psi/phi correction still to be added
    float* corr_f;        // [2]: the same in FP32
    double* corr_next;    // [2]: the correction the covering of this step leaves
    float* corr_f_next;   //      for the next one (a second buffer, so that the
                          //      covering can run beside the transport)
    int* err;
    double* link_part;    // [np][kMaxPartBlocks][kLinkK]
    unsigned* link_ticket;   // [np]
    double* cover_part;   // [np][kMaxPartBlocks][kCoverK]
    unsigned* cover_ticket;  // [1]
    long long* nfluid;
};

// ---------------------------------------------------------------------------
// population storage: plain FP64, or shifted by the rest equilibrium
// ---------------------------------------------------------------------------
template <class S>
struct PopStore;

// load/store move f_i; load_dev/store_dev move the deviation from the rest
// equilibrium, g_i = f_i - w_i rho0, in which collide-stream works.
template <>
struct PopStore<double> {
    static __device__ __forceinline__ double load(const double* p, size_t k, int, double) { return p[k]; }
    static __device__ __forceinline__ void store(double* p, size_t k, int, double, double f) { p[k] = f; }
    static __device__ __forceinline__ double load_dev(const double* p, size_t k, int i, double rho0)
    {
        return fma_x(-wgt_r<double>(i), rho0, p[k]);
    }
    static __device__ __forceinline__ void store_dev(double* p, size_t k, int i, double rho0, double g)
    {
        p[k] = fma_x(wgt_r<double>(i), rho0, g);
    }
};

// FP32: f_i - w_i rho0 keeps the O(1e-2) deviations at full FP32 precision.
template <>
struct PopStore<float> {
    static __device__ __forceinline__ float load(const float* p, size_t k, int i, float rho0)
    {
        return fma_x(wgt_r<float>(i), rho0, p[k]);
    }
    static __device__ __forceinline__ void store(float* p, size_t k, int i, float rho0, float f)
    {
        p[k] = fma_x(-wgt_r<float>(i), rho0, f);
    }
    static __device__ __forceinline__ float load_dev(const float* p, size_t k, int, float) { return p[k]; }
    static __device__ __forceinline__ void store_dev(float* p, size_t k, int, float, float g) { p[k] = g; }
};

// FP16/BF16: (f_i - w_i rho0)/w_i, a deviation of the same scale in every
// direction.
template <>
struct PopStore<__half> {
    static __device__ __forceinline__ float load(const __half* p, size_t k, int i, float rho0)
    {
        return (__half2float(p[k]) + rho0) * wgt_r<float>(i);
    }
    static __device__ __forceinline__ void store(__half* p, size_t k, int i, float rho0, float f)
    {
        p[k] = __float2half_rn(fma_x(f, inv_wgt_r<float>(i), -rho0));
    }
    static __device__ __forceinline__ float load_dev(const __half* p, size_t k, int i, float)
    {
        return __half2float(p[k]) * wgt_r<float>(i);
    }
    static __device__ __forceinline__ void store_dev(__half* p, size_t k, int i, float, float g)
    {
        p[k] = __float2half_rn(g * inv_wgt_r<float>(i));
    }
};

template <>
struct PopStore<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, size_t k, int i, float rho0)
    {
        return (__bfloat162float(p[k]) + rho0) * wgt_r<float>(i);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, size_t k, int i, float rho0, float f)
    {
        p[k] = __float2bfloat16_rn(fma_x(f, inv_wgt_r<float>(i), -rho0));
    }
    static __device__ __forceinline__ float load_dev(const __nv_bfloat16* p, size_t k, int i, float)
    {
        return __bfloat162float(p[k]) * wgt_r<float>(i);
    }
    static __device__ __forceinline__ void store_dev(__nv_bfloat16* p, size_t k, int i, float, float g)
    {
        p[k] = __float2bfloat16_rn(g * inv_wgt_r<float>(i));
    }
};

// ---------------------------------------------------------------------------
// geometry (FP64, no fused multiply-add: the solid/fluid and active/inactive
// decisions must be taken with exactly these roundings)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double min_image(double d, int L, int periodic)
{
    if (periodic) {
        double h = 0.5 * (double)L;
        if (d > h)
            d = __dsub_rn(d, (double)L);
        else if (d < -h)
            d = __dadd_rn(d, (double)L);
    }
    return d;
}

__device__ __forceinline__ void offset_from(const DevParams& P, const double Xc[3], int x, int y, int z,
                                            double r[3])
{
    r[0] = min_image(__dsub_rn((double)x, Xc[0]), P.nx, P.per[0]);
    r[1] = min_image(__dsub_rn((double)y, Xc[1]), P.ny, P.per[1]);
    r[2] = min_image(__dsub_rn((double)z, Xc[2]), P.nz, P.per[2]);
}

__device__ __forceinline__ double dot3_rn(const double a[3], const double b[3])
{
    return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

__device__ __forceinline__ bool inside_at(const DevParams& P, const double Xc[3], double R2, int x, int y, int z)
{
    double r[3];
    offset_from(P, Xc, x, y, z, r);
    return dot3_rn(r, r) < R2;
}

__device__ __forceinline__ bool inside_sphere(const DevParams& P, const DevPart& q, int x, int y, int z)
{
    return inside_at(P, q.X, q.R2, x, y, z);
}

// Neighbour node indices of (x,y,z) for the 19 directions; -1 beyond a wall.
__device__ __forceinline__ void neighbours(const DevParams& P, int x, int y, int z, int nb[19])
{
    int xs[3], ys[3], zs[3];
    xs[1] = x;
    ys[1] = y;
    zs[1] = z;
    xs[0] = x > 0 ? x - 1 : (P.per[0] ? P.nx - 1 : -1);
    xs[2] = x < P.nx - 1 ? x + 1 : (P.per[0] ? 0 : -1);
    ys[0] = y > 0 ? y - 1 : (P.per[1] ? P.ny - 1 : -1);
    ys[2] = y < P.ny - 1 ? y + 1 : (P.per[1] ? 0 : -1);
    zs[0] = z > 0 ? z - 1 : (P.per[2] ? P.nz - 1 : -1);
    zs[2] = z < P.nz - 1 ? z + 1 : (P.per[2] ? 0 : -1);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        int a = xs[1 + cx(i)], b = ys[1 + cy(i)], c = zs[1 + cz(i)];
        nb[i] = (a < 0 || b < 0 || c < 0) ? -1 : a + P.nx * (b + P.ny * c);
    }
}

// Integer part of the offset x - X on one axis after the oracle's periodic
// minimum image (d > L/2: d - L; d < -L/2: d + L, with d = x - X exact):
// the offset is exactly D - fr.  With h = L/2 and fr in [0, 1):
//   L even: d > h iff D >= h + 1;        d < -h iff D < -h, or D = -h and fr > 0
//   L odd (h = k + 1/2): d > h iff D >= k + 2, or D = k + 1 and fr < 1/2;
//                        d < -h iff D <= -k - 1, or D = -k and fr > 1/2
__host__ __device__ __forceinline__ int min_image_int(int x, int Xi, int fl, int L, int periodic)
{
    int D = x - Xi;
    if (!periodic) return D;
    if ((L & 1) == 0) {
        const int h = L >> 1;
        if (D >= h + 1)
            D -= L;
        else if (D < -h || (D == -h && (fl & kFrPos)))
            D += L;
    } else {
        const int k = L >> 1;
        if (D >= k + 2 || (D == k + 1 && (fl & kFrBelowHalf)))
            D -= L;
        else if (D <= -k - 1 || (D == -k && (fl & kFrAboveHalf)))
            D += L;
    }
    return D;
}

// Wrap a box coordinate onto the lattice; -1 when it falls beyond a wall.
__device__ __forceinline__ int wrap_coord(int c, int L, int periodic)
{
    if (c < 0 || c >= L) {
        if (!periodic) return -1;
        c %= L;
        if (c < 0) c += L;
    }
    return c;
}

}  // namespace lbdp
