// lbdp_batch_kernels.cuh -- persistent kernels that advance many independent
// boxes of one precision mode in one launch per kernel class.
//
// The host keeps a device-resident description of the batch (BatchDev): one
// BoxDev per box (its parameters and both pointer sets of its double
// buffers), the buffer that holds each box's current state, the steps each
// box still has to run, and lists of work tiles.  Every kernel runs a fixed
// grid that loops over its tile list, so a captured CUDA graph of these
// launches stays valid while boxes join and leave: only the tables change.
//
// Node tiles cover T*CPT consecutive nodes of one box (x fastest).  Particle
// tiles are the same (particle, block) split the single-box kernels use, so a
// box gives identical bits alone and inside a batch.
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

struct BoxDev {
    DevParams P;
    DevPtrs D[2];     // D[c]: pointers when buffer c holds the current state
    unsigned mx, my;  // div_magic(nx), div_magic(ny)
};

struct NodeTile {
    int box;
    int start;   // first node of the tile
};

struct PartTile {
    int box;
    int p;     // particle of the box
    int bi;    // block of the particle
    int nbi;   // blocks of the particle (the single-box split)
};

// Node tile sizes the batched node kernels use: 128 << k nodes.
constexpr int kNodeTileSizes = 2;

struct BatchDev {
    const BoxDev* boxes;
    int* cur;           // [box] buffer holding the current state
    long long* left;    // [box] steps still to run (0: the box sits out)
    int nbox;
    int n_node[kNodeTileSizes];
    const NodeTile* node[kNodeTileSizes];
    int n_link, n_cover;
    const PartTile* link;
    const PartTile* cover;
};

// Stage box b (with the pointer set of its current buffer) in shared memory.
// Called by the whole block; the leading barrier lets every thread finish
// with the previous box first.
struct BoxShared {
    DevParams P;
    DevPtrs D;
    unsigned mx, my;
};

__device__ __forceinline__ void stage_box(const BatchDev& B, int b, BoxShared& sb)
{
    __syncthreads();
    const BoxDev& src = B.boxes[b];
    const int c = B.cur[b];
    constexpr int nP = sizeof(DevParams) / 4, nD = sizeof(DevPtrs) / 4;
    static_assert(sizeof(DevParams) % 4 == 0 && sizeof(DevPtrs) % 4 == 0, "word copy");
    const unsigned* sp = (const unsigned*)&src.P;
    const unsigned* sd = (const unsigned*)&src.D[c];
    unsigned* dp = (unsigned*)&sb.P;
    unsigned* dd = (unsigned*)&sb.D;
    for (int k = threadIdx.x; k < nP; k += blockDim.x) dp[k] = sp[k];
    for (int k = threadIdx.x; k < nD; k += blockDim.x) dd[k] = sd[k];
    if (threadIdx.x == 0) {
        sb.mx = src.mx;
        sb.my = src.my;
    }
    __syncthreads();
}

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
// ("loose").  Box parameters staged in shared memory occupy registers where
// the single-box kernels read them as constant-bank operands, so the tight
// budget spills a few words; the autotuner picks.
template <int NC, int T, int RB>
struct NodeBounds {
    static constexpr int min_blocks =
        RB == 0 ? 1024 / T : 768 / T;   // 64 or 80 registers
};

template <class C, int NC, int T, int CPT, int TSI, int RB>
__global__ void __launch_bounds__(T, (NodeBounds<NC, T, RB>::min_blocks)) kb_node(const BatchDev* __restrict__ Bp)
{
    static_assert((128 << TSI) == T * CPT, "tile size");
    __shared__ BoxShared sb;
    const BatchDev& B = *Bp;
    const int nt = B.n_node[TSI];
    const NodeTile* tiles = B.node[TSI];
    int have = -1;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const NodeTile tl = tiles[t];
        if (B.left[tl.box] <= 0) continue;
        if (tl.box != have) {
            stage_box(B, tl.box, sb);
            have = tl.box;
        }
        const int N = (int)sb.P.N;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int n = tl.start + c * T + (int)threadIdx.x;
            if (n < N) {
                const int r = div_by(n, sb.mx);   // y + ny z
                const int z = div_by(r, sb.my);
                const int x = n - r * sb.P.nx, y = r - z * sb.P.ny;
                node_body<C, NC>(sb.P, sb.D, x, y, z);
            }
        }
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads, 1) kb_links(const BatchDev* __restrict__ Bp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];   // block_sum_t_bytes<kLinkK>(kPartThreads)
    __shared__ BoxShared sb;
    __shared__ DevPart sp;
    __shared__ bool last;
    const BatchDev& B = *Bp;
    for (int t = blockIdx.x; t < B.n_link; t += gridDim.x) {
        const PartTile tl = B.link[t];
        if (B.left[tl.box] <= 0) continue;
        // restage on every tile: the block's thread 0 may still be finishing
        // the previous particle's solve out of sb and sp
        stage_box(B, tl.box, sb);
        links_block<C>(sb.P, sb.D, tl.p, tl.bi, tl.nbi, (double*)smem_raw, sp, last);
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_cover_mark(const BatchDev* __restrict__ Bp)
{
    __shared__ BoxShared sb;
    const BatchDev& B = *Bp;
    int have = -1;
    for (int t = blockIdx.x; t < B.n_cover; t += gridDim.x) {
        const PartTile tl = B.cover[t];
        if (B.left[tl.box] <= 0) continue;
        if (tl.box != have) {
            stage_box(B, tl.box, sb);
            have = tl.box;
        }
        cover_mark_block<C>(sb.P, sb.D, tl.p, tl.bi, tl.nbi);
    }
}

template <class C>
__global__ void __launch_bounds__(kPartThreads) kb_cover_apply(const BatchDev* __restrict__ Bp)
{
    __shared__ double smem[block_sum_t_bytes<kCoverK>(kPartThreads) / sizeof(double)];
    __shared__ BoxShared sb;
    __shared__ bool last;
    const BatchDev& B = *Bp;
    for (int t = blockIdx.x; t < B.n_cover; t += gridDim.x) {
        const PartTile tl = B.cover[t];
        if (B.left[tl.box] <= 0) continue;
        stage_box(B, tl.box, sb);
        cover_apply_block<C>(sb.P, sb.D, tl.p, tl.bi, tl.nbi, smem, last);
    }
}

// End of a step: every box that ran it flips its buffers and counts it.
static __global__ void kb_advance(const BatchDev* __restrict__ Bp)
{
    const BatchDev& B = *Bp;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B.nbox; b += gridDim.x * blockDim.x) {
        if (B.left[b] > 0) {
            B.left[b] -= 1;
            B.cur[b] ^= 1;
        }
    }
}

}  // namespace lbdp
