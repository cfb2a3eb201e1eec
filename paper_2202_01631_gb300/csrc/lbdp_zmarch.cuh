// lbdp_zmarch.cuh -- the two bulk kernels of the single-box step, marching
// along z through a tile of 32 x 8 lattice columns.
//
//   kz_fused    chemical potentials, pressure tensor, force and
//               collide-stream in one pass: per plane, the block stages psi,
//               phi and the mask of the 36 x 12 columns around its tile
//               (two-node halo), computes mu and P for the 34 x 10 columns
//               of the plane (one-node halo) into a ring of shared-memory
//               planes, and then the force and the collide-stream of its own
//               tile one plane behind.  mu is written for the transport; P
//               and F never leave the chip.  Nodes next to a particle are
//               left to the side-stream kernels (k_pt_part, k_f_part,
//               k_collide_particles).
//   kz_scalars  the psi/phi transport (Eq. diffusion_reaction) from a ring of
//               three 34 x 10 planes of psi, phi, mu and u.
//
// A tile column is one thread; a block walks ZC planes (its z chunk) with
// one barrier per plane.  Halo planes of a chunk are staged (and, for the
// pressure tensor, computed) by both neighbouring chunks.  Each body is the
// one the unfused kernels run (mup_values, fdiv_values, collide_store,
// scalars_compute) on the same values, so the results are bit-identical to
// those kernels, and hence to the batched kernels.
#pragma once

#include "lbdp_kernels.cuh"

namespace lbdp {

constexpr int kZX = 32, kZY = 8, kZThreads = kZX * kZY;
constexpr int kZ1X = kZX + 2, kZ1Y = kZY + 2, kZ1 = kZ1X * kZ1Y;   // 34 x 10: one-node halo
constexpr int kZ2X = kZX + 4, kZ2Y = kZY + 4, kZ2 = kZ2X * kZ2Y;   // 36 x 12: two-node halo
// ring depths: with these, one barrier per plane separates every write of a
// ring slot from the last read of the plane it held (see kz_fused)
constexpr int kPsiRing = 6, kPhiRing = 4, kPtRing = 4, kScalRing = 5;

// in-plane slot offset of direction i in planes of row width W
template <int W>
__host__ __device__ constexpr int poff(int i)
{
    return cx(i) + W * cy(i);
}

// shape of a one-halo plane for the paired field layout (tile_index_last)
struct ZPlane1 {
    static constexpr int slots = kZ1;
};

// Shared-memory place of field k of slot s in a plane of T::slots slots:
// fields 2j and 2j+1 interleave ([j][slot][2]), so a body that reads both
// gets them in one 64-bit load; an odd last field stands alone.
template <class T>
__host__ __device__ constexpr int tile_index(int k, int s)
{
    return (k & ~1) * T::slots + 2 * s + (k & 1);
}
template <int NF, class T>
__host__ __device__ constexpr int tile_index_last(int k, int s)
{
    return ((NF & 1) && k == NF - 1) ? (NF - 1) * T::slots + s : tile_index<T>(k, s);
}

// The stress of one node (p_iso, grad psi) as one aligned vector, so that a
// neighbour's four numbers come in one shared-memory load.
template <class F>
struct alignas(4 * sizeof(F)) Pt4 {
    F v[4];
};

template <class F>
struct FusedSmem {
    Pt4<F> pt[kPtRing][kZ1];
    F psi[kPsiRing][kZ2];
    F phi[kPhiRing][kZ1];
    uint8_t mk[kPsiRing][kZ2];
};

template <class F>
struct ScalSmem {
    F f[kScalRing][7 * kZ1];
    uint8_t mk[kScalRing][kZ1];
};

// Column coordinate of halo offset l (may be negative) from tile origin o on
// an axis: wrapped on a periodic axis, -1 beyond a wall.
__device__ __forceinline__ int zm_coord(int o, int l, int L, int per) { return wrap_coord(o + l, L, per); }

// ---------------------------------------------------------------------------
// accessors over the shared-memory planes (same interface as GAcc)
// ---------------------------------------------------------------------------
// chemical-potential body: field 0 psi (two-halo planes), field 1 phi (own)
template <class F, bool kClear>
struct ZAccMu {
    const F* ps[3];
    const uint8_t* mk[3];
    int s2;
    F phi_own;
    __device__ __forceinline__ uint8_t mask(int i) const
    {
        return kClear ? (uint8_t)0 : mk[1 + cz(i)][s2 + poff<kZ2X>(i)];
    }
    template <int K>
    __device__ __forceinline__ F get(int i) const
    {
        if (K == 0) return ps[1 + cz(i)][s2 + poff<kZ2X>(i)];
        return phi_own;   // field 1 is read at the node itself only
    }
};

// force body: the stress (p_iso, grad psi) of the one-halo planes
template <class F, bool kClear>
struct ZAccP {
    const Pt4<F>* pt[3];
    const uint8_t* mk[3];
    int s1, s2;
    __device__ __forceinline__ uint8_t mask(int i) const
    {
        return kClear ? (uint8_t)0 : mk[1 + cz(i)][s2 + poff<kZ2X>(i)];
    }
    template <int K>
    __device__ __forceinline__ F get(int i) const
    {
        const Pt4<F> q = pt[1 + cz(i)][s1 + poff<kZ1X>(i)];
        return q.v[K];
    }
};

// transport body: psi, phi, mu_psi, mu_phi, u (one-halo planes, paired)
template <class F, bool kClear>
struct ZAccS {
    const F* f[3];
    const uint8_t* mk[3];
    int s1;
    __device__ __forceinline__ uint8_t mask(int i) const
    {
        return kClear ? (uint8_t)0 : mk[1 + cz(i)][s1 + poff<kZ1X>(i)];
    }
    template <int K>
    __device__ __forceinline__ F get(int i) const
    {
        return f[1 + cz(i)][tile_index_last<7, ZPlane1>(K, s1 + poff<kZ1X>(i))];
    }
};

// ---------------------------------------------------------------------------
// plane staging: each thread fetches up to two slots into registers (the
// loads stay in flight while the block works on earlier planes) and stores
// them into a ring slot later
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async): the copy engine writes the
// shared-memory ring directly, so a staged plane costs no registers and its
// latency is hidden behind the planes computed meanwhile
// ---------------------------------------------------------------------------
template <int B>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, bool valid)
{
    static_assert(B == 4 || B == 8, "4- or 8-byte copies");
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    // src-size 0 writes zeros and reads nothing (a slot beyond a wall)
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gsrc), "n"(B),
                 "r"(valid ? B : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Columns (x + nx y) of this thread's staging slots, fixed for the whole
// march: cps for the two-halo psi/mask slots, cph for the one-halo phi slots;
// -1 for a column beyond a wall or a slot this thread does not have.  The
// flag bit h of wall is set for a psi slot beyond a wall.
struct MuCols {
    int cps[2], cph[2];
};

__device__ __forceinline__ void mu_cols(const DevParams& P, int x0, int y0, MuCols& c)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = threadIdx.x + h * kZThreads;
        c.cps[h] = -1;
        c.cph[h] = -1;
        if (s < kZ2) {
            const int gx = zm_coord(x0, s % kZ2X - 2, P.nx, P.per[0]);
            const int gy = zm_coord(y0, s / kZ2X - 2, P.ny, P.per[1]);
            if (gx >= 0 && gy >= 0) c.cps[h] = gx + P.nx * gy;
        }
        if (s < kZ1) {
            const int gx = zm_coord(x0, s % kZ1X - 1, P.nx, P.per[0]);
            const int gy = zm_coord(y0, s / kZ1X - 1, P.ny, P.per[1]);
            if (gx >= 0 && gy >= 0) c.cph[h] = gx + P.nx * gy;
        }
    }
}

// Issue the copies of psi (two-halo slots) and phi (one-halo slots) of plane
// p into ring slots rpsi, rphi.
template <class F>
__device__ __forceinline__ void mu_plane_async(const DevParams& P, const DevPtrs& D, const MuCols& c, int p,
                                               FusedSmem<F>& sm, int rpsi, int rphi)
{
    const F* psi = (const F*)D.psi_src;
    const F* phi = (const F*)D.phi_src;
    const int gz = wrap_coord(p, P.nz, P.per[2]);
    const int base = gz * P.nx * P.ny;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = threadIdx.x + h * kZThreads;
        if (s < kZ2) {
            const bool ok = c.cps[h] >= 0 && gz >= 0;
            cp_async<(int)sizeof(F)>(&sm.psi[rpsi][s], psi + (ok ? base + c.cps[h] : 0), ok);
        }
        if (s < kZ1) {
            const bool ok = c.cph[h] >= 0 && gz >= 0;
            cp_async<(int)sizeof(F)>(&sm.phi[rphi][s], phi + (ok ? base + c.cph[h] : 0), ok);
        }
    }
}

// The masks of a plane's two-halo slots go through registers (their OR
// decides the mask-free bodies): kWallSlot beyond a wall.
struct MuMask {
    uint8_t m[2];
};

__device__ __forceinline__ void mu_mask_fetch(const DevParams& P, const DevPtrs& D, const MuCols& c, int p,
                                              MuMask& M)
{
    const int gz = wrap_coord(p, P.nz, P.per[2]);
    const int base = gz * P.nx * P.ny;
#pragma unroll
    for (int h = 0; h < 2; ++h) M.m[h] = (c.cps[h] >= 0 && gz >= 0) ? D.mask[base + c.cps[h]] : kWallSlot;
}

// Store the masks into ring slot r; returns whether any is not fluid.
template <class F>
__device__ __forceinline__ bool mu_mask_store(FusedSmem<F>& sm, int r, const MuMask& M)
{
    bool any = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = threadIdx.x + h * kZThreads;
        if (s < kZ2) {
            sm.mk[r][s] = M.m[h];
            any = any || M.m[h] != 0;
        }
    }
    return any;
}

// Transport planes: columns (x + nx y) of this thread's one-halo slots,
// fixed for the march (-1: beyond a wall, or no slot).
struct ScalCols {
    int c[2];
};

__device__ __forceinline__ void scal_cols(const DevParams& P, int x0, int y0, ScalCols& c)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = threadIdx.x + h * kZThreads;
        c.c[h] = -1;
        if (s < kZ1) {
            const int gx = zm_coord(x0, s % kZ1X - 1, P.nx, P.per[0]);
            const int gy = zm_coord(y0, s / kZ1X - 1, P.ny, P.per[1]);
            if (gx >= 0 && gy >= 0) c.c[h] = gx + P.nx * gy;
        }
    }
}

// Issue the copies of the seven transport fields of plane p into ring slot r.
template <class F>
__device__ __forceinline__ void scal_plane_async(const DevParams& P, const DevPtrs& D, const ScalCols& c, int p,
                                                 ScalSmem<F>& sm, int r)
{
    const size_t N = (size_t)P.N;
    const F* u = (const F*)D.u;
    const F* const src[7] = {(const F*)D.psi_src, (const F*)D.phi_src, (const F*)D.mupsi, (const F*)D.muphi,
                             u, u + N, u + 2 * N};
    const int gz = wrap_coord(p, P.nz, P.per[2]);
    const int base = gz * P.nx * P.ny;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = threadIdx.x + h * kZThreads;
        if (s < kZ1) {
            const bool ok = c.c[h] >= 0 && gz >= 0;
            const int g = ok ? base + c.c[h] : 0;
#pragma unroll
            for (int k = 0; k < 7; ++k)
                cp_async<(int)sizeof(F)>(&sm.f[r][tile_index_last<7, ZPlane1>(k, s)], src[k] + g, ok);
        }
    }
}

// The masks of a plane go through registers (their OR decides the mask-free
// body): m[h] for this thread's slots, kWallSlot beyond a wall.
struct ScalMask {
    uint8_t m[2];
};

__device__ __forceinline__ void scal_mask_fetch(const DevParams& P, const DevPtrs& D, const ScalCols& c, int p,
                                                ScalMask& M)
{
    const int gz = wrap_coord(p, P.nz, P.per[2]);
    const int base = gz * P.nx * P.ny;
#pragma unroll
    for (int h = 0; h < 2; ++h) M.m[h] = (c.c[h] >= 0 && gz >= 0) ? D.mask[base + c.c[h]] : kWallSlot;
}

// Store the masks into ring slot r; returns whether any is not fluid.
template <class F>
__device__ __forceinline__ bool scal_mask_store(ScalSmem<F>& sm, int r, const ScalMask& M)
{
    bool any = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = threadIdx.x + h * kZThreads;
        if (s < kZ1) {
            sm.mk[r][s] = M.m[h];
            any = any || M.m[h] != 0;
        }
    }
    return any;
}

// Planes per z chunk of a launch with gridDim.z chunks.
__host__ __device__ __forceinline__ int zm_chunk(int nz, int chunks) { return (nz + chunks - 1) / chunks; }

// ---------------------------------------------------------------------------
// kz_fused
// ---------------------------------------------------------------------------
// This thread's stage-1 slots (mu and the stress of the 34 x 10 columns of a
// plane), fixed for the whole march: the slot in the two-halo plane, and the
// column x + nx y where mu is written (-1: a halo column, another block's).
struct MuSlots {
    int s2[2], wcol[2];
};

__device__ __forceinline__ void mu_slots(const DevParams& P, int x0, int y0, MuSlots& m)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = threadIdx.x + h * kZThreads;
        const int lx = q % kZ1X - 1, ly = q / kZ1X - 1;
        m.s2[h] = (lx + 2) + kZ2X * (ly + 2);
        m.wcol[h] = (q < kZ1 && lx >= 0 && lx < kZX && ly >= 0 && ly < kZY && x0 + lx < P.nx && y0 + ly < P.ny)
                        ? (x0 + lx) + P.nx * (y0 + ly)
                        : -1;
    }
}

// Stage 1 of plane zs: mu and the stress of the 34 x 10 columns, two slots per
// thread; mu is written for the tile's own columns when own_plane.
template <class C, bool kClear>
__device__ __forceinline__ void fused_stage1(const DevParams& P, const DevPtrs& D, FusedSmem<typename C::fld_t>& sm,
                                             const MuSlots& ms, int x0, int y0, int zs, bool own_plane,
                                             const int (&rp)[3], int rf, int rt, typename C::real dps,
                                             typename C::real dph)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const int gz = wrap_coord(zs, P.nz, P.per[2]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = threadIdx.x + h * kZThreads;
        if (q >= kZ1) break;
        const int s2 = ms.s2[h];
        if (sm.mk[rp[1]][s2] != 0) continue;   // solid, or beyond a wall
        // lattice coordinates: needed by the wetting ghosts only
        int x = 0, y = 0;
        if (!kClear) {
            x = zm_coord(x0, q % kZ1X - 1, P.nx, P.per[0]);
            y = zm_coord(y0, q / kZ1X - 1, P.ny, P.per[1]);
        }
        ZAccMu<F, kClear> a;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.ps[k] = sm.psi[rp[k]];
            a.mk[k] = sm.mk[rp[k]];
        }
        a.s2 = s2;
        a.phi_own = sm.phi[rf][q];
        R mps, mph, pt[kPtFields];
        mup_values<C>(P, D, x, y, gz, a, dps, dph, mps, mph, pt);
        if (P.thermo) {
            Pt4<F> v;
#pragma unroll
            for (int k = 0; k < 4; ++k) v.v[k] = (F)pt[k];
            sm.pt[rt][q] = v;
        }
        if (own_plane && ms.wcol[h] >= 0) {
            const int n = ms.wcol[h] + P.nx * P.ny * gz;
            ((F*)D.mupsi)[n] = (F)mps;
            ((F*)D.muphi)[n] = (F)mph;
        }
    }
}

// Stage 2 of plane zs (this thread's column): every global load of the node
// first (its boundary flag and the pull sources of its populations, one round
// trip), then the force from the stress planes while they are in flight, then
// the collide-stream of a bulk node.
template <class C, bool kClear>
__device__ __forceinline__ void fused_stage2(const DevParams& P, const DevPtrs& D,
                                             const FusedSmem<typename C::fld_t>& sm, int x0, int y0, int zs,
                                             const int (&rp)[3], const int (&rt)[3])
{
    using R = typename C::real;
    using F = typename C::fld_t;
    const int tx = threadIdx.x & (kZX - 1), ty = threadIdx.x / kZX;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= P.nx || y >= P.ny) return;
    const int s2 = (tx + 2) + kZ2X * (ty + 2), s1 = (tx + 1) + kZ1X * (ty + 1);
    if (sm.mk[rp[1]][s2] != 0) return;   // inside a particle
    const int n = x + P.nx * (y + P.ny * zs);
    const uint8_t bf = D.bflag[n];
    R fl[19];
    pull_loads<C>(P, D, x, y, zs, fl);
    ZAccP<F, kClear> a;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.pt[k] = sm.pt[rt[k]];
        a.mk[k] = sm.mk[rp[k]];
    }
    a.s1 = s1;
    a.s2 = s2;
    R Fx, Fy, Fz;
    fdiv_values<C>(P, a, Fx, Fy, Fz);
    if (bf) return;   // next to a particle: k_collide_particles
    if (near_wall(P, x, y, zs)) bulk_wall_links<C>(P, D, x, y, zs, fl);
    collide_store<C>(prm<R>(P), D, (size_t)P.N, n, fl, Fx, Fy, Fz);
}

// ring position advanced by one
template <int N>
__device__ __forceinline__ int ring_next(int r)
{
    return r + 1 == N ? 0 : r + 1;
}

// Resident blocks per SM the fused kernel is compiled for: four in FP32
// arithmetic (64 registers; more resident warps hide the population loads
// better than the registers the compiler would otherwise keep), two in FP64
// (its shared-memory ring allows no more).
template <class C>
constexpr int fused_blocks_per_sm()
{
    return sizeof(typename C::real) == 8 ? 2 : 4;
}

// The march of one block: columns x0 .. x0 + 31, y0 .. y0 + 7, planes
// z0 .. z0 + nt - 1 (nt >= 1), smem of sizeof(FusedSmem<F>) bytes.
template <class C>
__device__ __forceinline__ void kz_fused_run(const DevParams& P, const DevPtrs& D, int x0, int y0, int z0, int nt,
                                             unsigned char* smem_raw)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    FusedSmem<F>& sm = *reinterpret_cast<FusedSmem<F>*>(smem_raw);
    MuCols cols;
    mu_cols(P, x0, y0, cols);
    MuSlots ms;
    mu_slots(P, x0, y0, ms);
    const R dps = corr_r<R>(D, 0), dph = corr_r<R>(D, 1);
    // Ring slots: psi and the mask of plane p at (p - z0 + 2) mod 6, phi at
    // (p - z0 + 2) mod 4, the stress at (p - z0 + 1) mod 4.  Bit k of hist:
    // the staged plane k planes behind the newest has a slot that is solid or
    // beyond a wall (block-uniform).  Iteration t computes the stress of
    // plane z0 + t - 1 (stage 1), stores the masks of z0 + t + 1, issues the
    // copies of psi/phi of z0 + t + 2, waits for those of z0 + t + 1, and
    // collides plane z0 + t - 2 (stage 2).  With these ring depths the one
    // barrier per iteration orders every write of a slot after the last read
    // of the plane it held.
    unsigned hist = 0;
    MuMask M;
    for (int k = 0; k < 3; ++k) mu_plane_async<F>(P, D, cols, z0 - 2 + k, sm, k, k);   // z0 - 2 .. z0
    cp_async_commit();
    mu_plane_async<F>(P, D, cols, z0 + 1, sm, 3, 3);
    cp_async_commit();
    cp_async_wait<1>();
    for (int k = 0; k < 3; ++k) {
        mu_mask_fetch(P, D, cols, z0 - 2 + k, M);
        hist = (hist << 1) | (unsigned)__syncthreads_or(mu_mask_store<F>(sm, k, M));
    }
    mu_mask_fetch(P, D, cols, z0 + 1, M);
    // rp0: psi/mask slot of plane z0 + t - 2; rf: phi slot of z0 + t - 1; rt0:
    // stress slot of z0 + t - 1
    int rp0 = 0, rf = 1, rt0 = 0;
    for (int t = 0; t <= nt + 1; ++t) {
        const int rpa = ring_next<kPsiRing>(rp0), rpb = ring_next<kPsiRing>(rpa), rpc = ring_next<kPsiRing>(rpb);
        const int rpd = ring_next<kPsiRing>(rpc);
        {
            const int rp1[3] = {rp0, rpa, rpb};   // planes z0 + t - 2 .. z0 + t
            const bool own = t >= 1 && t <= nt;
            if ((hist & 7u) == 0u)
                fused_stage1<C, true>(P, D, sm, ms, x0, y0, z0 + t - 1, own, rp1, rf, rt0, dps, dph);
            else
                fused_stage1<C, false>(P, D, sm, ms, x0, y0, z0 + t - 1, own, rp1, rf, rt0, dps, dph);
        }
        bool any = false;
        if (t <= nt) any = mu_mask_store<F>(sm, rpc, M);   // masks of z0 + t + 1
        if (t + 2 <= nt + 1) {                               // z0 + t + 2
            mu_mask_fetch(P, D, cols, z0 + t + 2, M);
            const int rfd = rf < 1 ? rf + 3 : rf - 1;         // phi slot of z0 + t + 2
            mu_plane_async<F>(P, D, cols, z0 + t + 2, sm, rpd, rfd);
        }
        cp_async_commit();
        cp_async_wait<1>();   // this thread's copies of plane z0 + t + 1 have landed
        hist = (hist << 1) | (unsigned)__syncthreads_or(any);
        if (t >= 2) {   // plane z0 + t - 2: stress of z0 + t - 3 .. z0 + t - 1
            const int rpm = rp0 == 0 ? kPsiRing - 1 : rp0 - 1;
            const int rp2[3] = {rpm, rp0, rpa};
            const int rt2[3] = {rt0 < 2 ? rt0 + 2 : rt0 - 2, rt0 == 0 ? kPtRing - 1 : rt0 - 1, rt0};
            if ((hist & 0x1Cu) == 0u)
                fused_stage2<C, true>(P, D, sm, x0, y0, z0 + t - 2, rp2, rt2);
            else
                fused_stage2<C, false>(P, D, sm, x0, y0, z0 + t - 2, rp2, rt2);
        }
        rp0 = rpa;
        rf = ring_next<kPhiRing>(rf);
        rt0 = ring_next<kPtRing>(rt0);
    }
    cp_async_wait<0>();
}

// Single box: grid (column tiles in x, in y, z chunks).
template <class C>
__global__ void __launch_bounds__(kZThreads, fused_blocks_per_sm<C>()) kz_fused(const __grid_constant__ DevParams P,
                                                                               const __grid_constant__ DevPtrs D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];   // sizeof(FusedSmem<F>)
    const int zc = zm_chunk(P.nz, gridDim.z);
    const int z0 = blockIdx.z * zc;
    const int nt = min(z0 + zc, P.nz) - z0;   // planes of this chunk
    if (nt <= 0) return;                      // block-uniform
    kz_fused_run<C>(P, D, blockIdx.x * kZX, blockIdx.y * kZY, z0, nt, smem_raw);
}

// ---------------------------------------------------------------------------
// kz_scalars
// ---------------------------------------------------------------------------
template <class C, bool kClear>
__device__ __forceinline__ void scal_stage(const DevParams& P, const DevPtrs& D,
                                           const ScalSmem<typename C::fld_t>& sm, int x0, int y0, int zs,
                                           const int (&r)[3], typename C::real dps, typename C::real dph)
{
    using F = typename C::fld_t;
    const int tx = threadIdx.x & (kZX - 1), ty = threadIdx.x / kZX;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= P.nx || y >= P.ny) return;
    const int s1 = (tx + 1) + kZ1X * (ty + 1);
    if (sm.mk[r[1]][s1] != 0) return;   // inside a particle
    ZAccS<F, kClear> a;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.f[k] = sm.f[r[k]];
        a.mk[k] = sm.mk[r[k]];
    }
    a.s1 = s1;
    scalars_compute_c<C, false>(P, D, x, y, zs, x + P.nx * (y + P.ny * zs), a, dps, dph);
}

// The march of one block, as kz_fused_run (smem of sizeof(ScalSmem<F>) bytes).
template <class C>
__device__ __forceinline__ void kz_scalars_run(const DevParams& P, const DevPtrs& D, int x0, int y0, int z0, int nt,
                                               unsigned char* smem_raw)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    ScalSmem<F>& sm = *reinterpret_cast<ScalSmem<F>*>(smem_raw);
    ScalCols cols;
    scal_cols(P, x0, y0, cols);
    const R dps = corr_r<R>(D, 0), dph = corr_r<R>(D, 1);
    // Plane p in ring slot (p - z0 + 1) mod 5.  Iteration t computes plane
    // z0 + t from planes z0 + t - 1 .. z0 + t + 1 and issues the copies of
    // plane z0 + t + 2 (into the slot of z0 + t - 3, last read at t - 2); the
    // masks of a plane are loaded one iteration before they are stored.
    unsigned hist = 0;
    ScalMask M;
    for (int k = 0; k < 2; ++k) {   // planes z0 - 1, z0
        scal_plane_async<F>(P, D, cols, z0 - 1 + k, sm, k);
        scal_mask_fetch(P, D, cols, z0 - 1 + k, M);
        hist = (hist << 1) | (unsigned)__syncthreads_or(scal_mask_store<F>(sm, k, M));
    }
    cp_async_commit();
    scal_plane_async<F>(P, D, cols, z0 + 1, sm, 2);
    cp_async_commit();
    scal_mask_fetch(P, D, cols, z0 + 1, M);
    int r0 = 0;   // slot of plane z0 + t - 1
    for (int t = 0; t < nt; ++t) {
        const int r1 = r0 + 1 == kScalRing ? 0 : r0 + 1;
        const int r2 = r1 + 1 == kScalRing ? 0 : r1 + 1;
        const int r3 = r2 + 1 == kScalRing ? 0 : r2 + 1;
        const bool any = scal_mask_store<F>(sm, r2, M);   // plane z0 + t + 1
        if (t + 2 <= nt) {
            scal_mask_fetch(P, D, cols, z0 + t + 2, M);
            scal_plane_async<F>(P, D, cols, z0 + t + 2, sm, r3);
        }
        cp_async_commit();
        cp_async_wait<1>();   // this thread's copies of plane z0 + t + 1 have landed
        hist = (hist << 1) | (unsigned)__syncthreads_or(any);
        const int r[3] = {r0, r1, r2};
        if ((hist & 7u) == 0u)
            scal_stage<C, true>(P, D, sm, x0, y0, z0 + t, r, dps, dph);
        else
            scal_stage<C, false>(P, D, sm, x0, y0, z0 + t, r, dps, dph);
        r0 = r1;
    }
    cp_async_wait<0>();
}

// Resident blocks per SM of the transport: three (80 registers) measured
// faster than four (64) on the 256^3 workload.
constexpr int kScalBlocksPerSM = 3;

template <class C>
__global__ void __launch_bounds__(kZThreads, kScalBlocksPerSM) kz_scalars(const __grid_constant__ DevParams P,
                                                                          const __grid_constant__ DevPtrs D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];   // sizeof(ScalSmem<F>)
    const int zc = zm_chunk(P.nz, gridDim.z);
    const int z0 = blockIdx.z * zc;
    const int nt = min(z0 + zc, P.nz) - z0;
    if (nt <= 0) return;   // block-uniform
    kz_scalars_run<C>(P, D, blockIdx.x * kZX, blockIdx.y * kZY, z0, nt, smem_raw);
}

// ---------------------------------------------------------------------------
// the pressure tensor and force next to particles, for the side stream
// ---------------------------------------------------------------------------
// P at every fluid node of the link box of particle p grown by one node (the
// boundary nodes and all their neighbours), into the pressure-tensor array.
// Nodes in two such boxes are written twice with the same values.
__device__ __forceinline__ void pt_box(const DevParams& P, const DevPart& q, int o[3], int s[3])
{
    const int L[3] = {P.nx, P.ny, P.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = q.g.Xi[a] - q.Rc - 3;
        s[a] = P.side1[a] + 2;
        if (P.per[a] && s[a] > L[a]) s[a] = L[a];
    }
}

// Blocks per particle of k_pt_part (about one node of the box per thread).
__host__ __device__ inline int pt_part_blocks(const DevParams& P)
{
    long long t = 1;
    const int L[3] = {P.nx, P.ny, P.nz};
    for (int a = 0; a < 3; ++a) {
        int s = P.side1[a] + 2;
        if (P.per[a] && s > L[a]) s = L[a];
        t *= s;
    }
    const long long b = (t + kPartThreads - 1) / kPartThreads;
    return (int)(b < 1 ? 1 : (b > kMaxPartBlocks ? kMaxPartBlocks : b));
}

// Block bi of the nbi blocks of particle p.
template <class C>
__device__ __forceinline__ void pt_part_block(const DevParams& P, const DevPtrs& D, int p, int bi, int nbi)
{
    using R = typename C::real;
    using F = typename C::fld_t;
    if (!P.thermo) return;
    int o[3], sd[3];
    pt_box(P, D.parts[p], o, sd);
    const int tot = sd[0] * sd[1] * sd[2];
    const size_t N = (size_t)P.N;
    for (int t = bi * blockDim.x + threadIdx.x; t < tot; t += nbi * blockDim.x) {
        int x, y, z;
        if (!box_node(P, o, sd, t, x, y, z)) continue;
        const int n = x + P.nx * (y + P.ny * z);
        if (D.mask[n]) continue;
        GAcc<F, 2> a;
        neighbours(P, x, y, z, a.nb);
        a.n = n;
        a.mk = D.mask;
        a.f[0] = (const F*)D.psi_src;
        a.f[1] = (const F*)D.phi_src;
        R mps, mph, pt[kPtFields];
        mup_values<C>(P, D, x, y, z, a, corr_r<R>(D, 0), corr_r<R>(D, 1), mps, mph, pt);
        F* ptg = (F*)D.pt;
#pragma unroll
        for (int k = 0; k < kPtFields; ++k) ptg[k * N + n] = (F)pt[k];
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_pt_part(const __grid_constant__ DevParams P,
                                                           const __grid_constant__ DevPtrs D)
{
    pt_part_block<C>(P, D, blockIdx.y, blockIdx.x, gridDim.x);
}

// F at the fluid nodes next to particle p (those whose lowest adjacent
// particle is p, as in k_collide_particles), into the force array.
template <class C>
__device__ __forceinline__ void f_part_block(const DevParams& P, const DevPtrs& D, int p, int bi, int nbi)
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
        fdiv_node<C>(P, D, x, y, z);
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) k_f_part(const __grid_constant__ DevParams P,
                                                          const __grid_constant__ DevPtrs D)
{
    f_part_block<C>(P, D, blockIdx.y, blockIdx.x, gridDim.x);
}

}  // namespace lbdp
