// lbdp_batch_kernels.cuh -- kernels that advance many independent boxes of
// one precision mode in one launch per kernel class.
//
// A launch covers up to kLaunchBoxes boxes: grid (blocks, boxes), box =
// blockIdx.y.  The boxes' parameters and pointer sets travel in the launch's
// own parameter block (BoxLaunch, __grid_constant__), so a block reads them
// as uniform constant-bank values -- as the single-box kernels read theirs --
// instead of holding them in registers.  Box b gets gx[b] blocks in
// proportion to its size (the grid is as wide as the widest box; other
// blocks leave at once); each block loops over its box's tiles.  A captured
// CUDA graph of these launches holds its parameters, so the host captures
// again when the set of boxes or their buffers change.
//
// Node tiles are T*CPT consecutive nodes of a box (x fastest).  Particle
// blocks follow exactly the single-box split (particle, block), so a box
// gives identical bits alone and inside a batch.
#pragma once

#include "lbdp_kernels.cuh"

namespace lbdp {

// Floor division of n < 2^24 by d < 2^8 as a multiply-high with
// m = ceil(2^32 / d): with n = q d + r and m d = 2^32 + e (0 <= e < d),
// n m / 2^32 = q + r/d + n e/(d 2^32) and n e < 2^32, so the floor is q.
__host__ __device__ inline unsigned div_magic(unsigned d) { return (unsigned)((0x100000000ull + d - 1) / d); }
__device__ __forceinline__ int div_by(int n, unsigned m) { return (int)__umulhi((unsigned)n, m); }

constexpr int kBatchMaxEdgeXY = 255;          // nx, ny of a batched box
constexpr long long kBatchMaxNodes = 1 << 24;  // N of a batched box (exclusive)
constexpr int kBatchMaxBoxes = 4096;
constexpr int kLaunchBoxes = 40;               // boxes per launch (parameter block < 32 KB)
constexpr int kNodeTileSizes = 2;              // node tiles of 128 << k nodes

struct BoxDev {
    DevParams P;
    DevPtrs D[2];     // D[s]: pointers for step parity s of the run
    unsigned mx, my;  // div_magic(nx), div_magic(ny)
};

// Parameter block of one launch: boxes [base, base + nbox) of the batch.
struct BoxLaunch {
    long long* left;                       // [batch box] steps still to run
    int base, nbox;
    int par;                               // step parity: D[par] is current
    int gx[kNodeTileSizes][kLaunchBoxes];  // node blocks of each box per tile size
    int gt[kLaunchBoxes];                  // blocks of each box for the 32x4x4 tiles
    BoxDev box[kLaunchBoxes];
};
static_assert(sizeof(BoxLaunch) <= 32000, "kernel parameter block");

// A launch of the batched kernels: parameter block and grids (x = widest
// box, y = boxes).
struct LaunchPlan {
    BoxLaunch L;
    dim3 node[kNodeTileSizes];
    dim3 tiles;
    dim3 link, cover;
};

enum NodeClass : int { kNcMup = 0, kNcFdiv = 1, kNcCollide = 2, kNcScalars = 3, kNumNodeClasses = 4 };

template <class C, int NC>
__device__ __forceinline__ void node_body(const DevParams& P, const DevPtrs& D, int x, int y, int z)
{
    if (NC == kNcMup) mup_node<C>(P, D, x, y, z);
    if (NC == kNcFdiv) fdiv_node<C>(P, D, x, y, z);
    if (NC == kNcCollide) collide_node<C>(P, D, x, y, z);
    if (NC == kNcScalars) scalars_node<C>(P, D, x, y, z);
}

// Minimum resident blocks per SM asked of the compiler, which sets the
// register budget: 64 per thread ("tight", the single-box budget) or 80
// ("loose"); the autotuner picks.
template <int NC, int T, int RB>
struct NodeBounds {
    static constexpr int min_blocks = RB == 0 ? 1024 / T : 768 / T;   // 64 or 80 registers
};

template <class C, int NC, int T, int CPT, int TSI, int RB>
__global__ void __launch_bounds__(T, (NodeBounds<NC, T, RB>::min_blocks))
    kb_node(const __grid_constant__ BoxLaunch L)
{
    static_assert((128 << TSI) == T * CPT, "tile size");
    const int b = blockIdx.y;
    if (b >= L.nbox) return;
    const int g = L.gx[TSI][b];
    if ((int)blockIdx.x >= g || L.left[L.base + b] <= 0) return;
    const BoxDev& X = L.box[b];
    const DevParams& P = X.P;
    const DevPtrs& D = X.D[L.par];
    const int N = (int)P.N;
    for (int t = blockIdx.x; t * (128 << TSI) < N; t += g) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int n = t * (128 << TSI) + c * T + (int)threadIdx.x;
            if (n < N) {
                const int r = div_by(n, X.mx);   // y + ny z
                const int z = div_by(r, X.my);
                const int x = n - r * P.nx, y = r - z * P.ny;
                node_body<C, NC>(P, D, x, y, z);
            }
        }
    }
}

// Force and transport with the single-box shared-memory tiles: the blocks of
// box b loop over its 32 x 4 x 4 tiles.
template <class C, int NC>
__global__ void __launch_bounds__(kTileThreads) kb_tiled(const __grid_constant__ BoxLaunch L)
{
    using F = typename C::fld_t;
    constexpr int NF = NC == kNcFdiv ? kPtFields : 7;
    extern __shared__ __align__(16) unsigned char smem_raw[];   // tile_smem<F, NF>()
    F* sf = (F*)smem_raw;
    uint8_t* sm = (uint8_t*)(sf + NF * Tile::slots);
    const int b = blockIdx.y;
    if (b >= L.nbox) return;
    const int g = L.gt[b];
    if ((int)blockIdx.x >= g || L.left[L.base + b] <= 0) return;
    const DevParams& P = L.box[b].P;
    const DevPtrs& D = L.box[b].D[L.par];
    const size_t N = (size_t)P.N;
    const int ntx = (P.nx + 31) >> 5, nty = (P.ny + 3) >> 2, ntz = (P.nz + 3) >> 2;
    const F* pt = (const F*)D.pt;
    const F* u = (const F*)D.u;
    const F* src[NF];
    if (NC == kNcFdiv) {
#pragma unroll
        for (int k = 0; k < NF; ++k) src[k] = pt + k * N;
    } else {
        src[0] = (const F*)D.psi_src;
        src[1] = (const F*)D.phi_src;
        src[2] = (const F*)D.mupsi;
        src[3] = (const F*)D.muphi;
#pragma unroll
        for (int k = 4; k < NF; ++k) src[k] = u + (k - 4) * N;
    }
    for (int t = blockIdx.x; t < ntx * nty * ntz; t += g) {
        const int x0 = (t % ntx) * 32, y0 = ((t / ntx) % nty) * 4, z0 = (t / (ntx * nty)) * 4;
        __syncthreads();   // every node of the previous tile is done with sf, sm
        const bool any = stage_tile<F, NF, Tile>(P, D.mask, src, x0, y0, z0, sf, sm);
        const bool clear = !__syncthreads_or(any);
        tile_nodes(P, sm, x0, y0, z0, [&](int x, int y, int z, int n, int slot) {
            if (clear) {
                const TAccClear<F, NF, Tile> a{{sf, sm, slot}};
                if (NC == kNcFdiv)
                    fdiv_compute<C>(P, D, n, a);
                else
                    scalars_compute<C>(P, D, x, y, z, n, a);
            } else {
                const TAcc<F, NF, Tile> a{sf, sm, slot};
                if (NC == kNcFdiv)
                    fdiv_compute<C>(P, D, n, a);
                else
                    scalars_compute<C>(P, D, x, y, z, n, a);
            }
        });
    }
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
