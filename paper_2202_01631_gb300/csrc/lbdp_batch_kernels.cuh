// lbdp_batch_kernels.cuh -- kernels that advance many independent boxes of
// one precision mode in one launch per kernel class.
//
// A launch covers up to kLaunchBoxes boxes: grid (blocks, boxes), box =
// blockIdx.y.  The boxes' parameters and pointer sets travel in the launch's
// own parameter block (BoxLaunch, __grid_constant__), so a block reads them
// as uniform constant-bank values -- as the single-box kernels read theirs --
// instead of holding them in registers.  The bulk kernels run the single-box
// z-marching bodies (kz_fused_run, kz_scalars_run) on the 32 x 8 column tiles
// of box b, each block one z chunk of ZC planes (the grid is as wide as the
// widest box; other blocks leave at once).  The particle kernels run the
// single-box particle bodies with exactly the single-box (particle, block)
// split, so a box gives identical bits alone and inside a batch.  A captured
// CUDA graph of these launches holds its parameters, so the host captures
// again when the set of boxes or their buffers change.
#pragma once

#include "lbdp_internal.h"
#include "lbdp_kernels.cuh"
#include "lbdp_zmarch.cuh"

namespace lbdp {

constexpr int kBatchMaxEdgeXY = 255;          // nx, ny of a batched box
constexpr long long kBatchMaxNodes = 1 << 24;  // N of a batched box (exclusive)
constexpr int kBatchMaxBoxes = 4096;
constexpr int kLaunchBoxes = 40;               // boxes per launch (parameter block < 32 KB)

struct BoxDev {
    DevParams P;
    DevPtrs D[2];   // D[s]: pointers for step parity s of the run
};

// Parameter block of one launch: boxes [base, base + nbox) of the batch.
struct BoxLaunch {
    long long* left;   // [batch box] steps still to run
    int base, nbox;
    int par;           // step parity: D[par] is current
    BoxDev box[kLaunchBoxes];
};
static_assert(sizeof(BoxLaunch) <= 32000, "kernel parameter block");

// Planes per block (z chunk) of the bulk kernels: the autotuner's
// candidates, one template instance each.
constexpr int kZChunks[kNumBatchCfgs] = {8, 16, 32};

// Blocks of box P for z chunks of zc planes.
__host__ __device__ inline int zm_blocks(const DevParams& P, int zc)
{
    return ((P.nx + kZX - 1) / kZX) * ((P.ny + kZY - 1) / kZY) * ((P.nz + zc - 1) / zc);
}

// A launch of the batched kernels: parameter block and grids (x = widest
// box, y = boxes).
struct LaunchPlan {
    BoxLaunch L;
    dim3 zgrid[kNumBatchCfgs];
    dim3 link, cover, ptg;
};

// Column tile and z chunk of block bx of box P; false for a block past the
// box's last tile.
__device__ __forceinline__ bool zm_decode(const DevParams& P, int zc, int bx, int& x0, int& y0, int& z0, int& nt)
{
    const int ntx = (P.nx + kZX - 1) / kZX, nty = (P.ny + kZY - 1) / kZY;
    const int nch = (P.nz + zc - 1) / zc;
    if (bx >= ntx * nty * nch) return false;
    x0 = (bx % ntx) * kZX;
    y0 = ((bx / ntx) % nty) * kZY;
    z0 = (bx / (ntx * nty)) * zc;
    nt = min(z0 + zc, P.nz) - z0;
    return true;
}

template <class C, int ZC>
__global__ void __launch_bounds__(kZThreads, fused_blocks_per_sm<C>()) kbz_fused(const __grid_constant__ BoxLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];   // sizeof(FusedSmem<F>)
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    int x0, y0, z0, nt;
    if (!zm_decode(P, ZC, blockIdx.x, x0, y0, z0, nt)) return;   // block-uniform
    kz_fused_run<C>(P, L.box[b].D[L.par], x0, y0, z0, nt, smem_raw);
}

template <class C, int ZC>
__global__ void __launch_bounds__(kZThreads, kScalBlocksPerSM) kbz_scalars(const __grid_constant__ BoxLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];   // sizeof(ScalSmem<F>)
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    int x0, y0, z0, nt;
    if (!zm_decode(P, ZC, blockIdx.x, x0, y0, z0, nt)) return;   // block-uniform
    kz_scalars_run<C>(P, L.box[b].D[L.par], x0, y0, z0, nt, smem_raw);
}

// Particle kernels: blockIdx.x = particle * blocks per particle + block.
template <class C>
__global__ void __launch_bounds__(kPartThreads, 1) kb_links(const __grid_constant__ BoxLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];   // block_rows_bytes<kLinkK>(kPartThreads)
    __shared__ DevPart sp;
    __shared__ bool last;
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const int p = blockIdx.x / P.nb1, bi = blockIdx.x % P.nb1;
    if (p >= P.np) return;
    links_block<C>(P, L.box[b].D[L.par], p, bi, P.nb1, (double*)smem_raw, sp, last);
}

// Stress and force next to the particles, boundary collide-stream and
// boundary transport: the single-box split over (particle, block).
template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_pt_part(const __grid_constant__ BoxLaunch L)
{
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const int nb = pt_part_blocks(P);
    const int p = blockIdx.x / nb, bi = blockIdx.x % nb;
    if (p >= P.np) return;
    pt_part_block<C>(P, L.box[b].D[L.par], p, bi, nb);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_f_part(const __grid_constant__ BoxLaunch L)
{
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const int p = blockIdx.x / P.nb1, bi = blockIdx.x % P.nb1;
    if (p >= P.np) return;
    f_part_block<C>(P, L.box[b].D[L.par], p, bi, P.nb1);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_collide_particles(const __grid_constant__ BoxLaunch L)
{
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const int p = blockIdx.x / P.nb1, bi = blockIdx.x % P.nb1;
    if (p >= P.np) return;
    collide_particles_block<C>(P, L.box[b].D[L.par], p, bi, P.nb1);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_scalars_particles(const __grid_constant__ BoxLaunch L)
{
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const int p = blockIdx.x / P.nb1, bi = blockIdx.x % P.nb1;
    if (p >= P.np) return;
    scalars_particles_block<C>(P, L.box[b].D[L.par], p, bi, P.nb1);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_cover_mark(const __grid_constant__ BoxLaunch L)
{
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const int p = blockIdx.x / P.nb2, bi = blockIdx.x % P.nb2;
    if (p >= P.np) return;
    cover_mark_block<C>(P, L.box[b].D[L.par], p, bi, P.nb2);
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_cover_apply(const __grid_constant__ BoxLaunch L)
{
    __shared__ double smem[block_rows_bytes<kCoverK>(kPartThreads) / sizeof(double)];
    __shared__ bool last;
    const int b = blockIdx.y;
    if (b >= L.nbox || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const int p = blockIdx.x / P.nb2, bi = blockIdx.x % P.nb2;
    if (p >= P.np) return;
    cover_apply_block<C>(P, L.box[b].D[L.par], p, bi, P.nb2, smem, last);
}

// End of a step: every box that ran it counts it.
static __global__ void kb_advance(long long* left, int nbox)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x)
        if (left[b] > 0) left[b] -= 1;
}

}  // namespace lbdp
