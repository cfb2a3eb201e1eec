// lbdp_noalloc.cu -- lb_totals_noalloc: the FP64 conservation totals of a
// caller-owned field set, computed without allocating any device memory.
//
// Some callers cannot allocate: a serving process whose device memory is
// planned and owned by its own arena allocator must not have a library call
// cudaMalloc behind its back, and a latency-critical loop cannot pay for the
// device-wide synchronisation that cudaMalloc and cudaFree may imply.  For
// them this entry point keeps its per-block partial sums in a fixed array in
// the library's own device memory (the file-scope array below, present on
// every device that loads the library until the process exits).  The caller
// passes the inputs and the output buffer; nothing else is allocated.
#include <mutex>

#include "lbdp.h"
#include "lbdp_lattice.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 8;
constexpr int kNodesPerBlock = kThreads * kNodesPerThread;   // 2048
// One partial triple per block: 8192 blocks cover 8192 * 2048 = 16,777,216
// nodes (a 256^3 box).  3 * 8192 doubles = 192 KiB.
constexpr int kMaxBlocks = 8192;
constexpr long long kMaxNodes = (long long)kMaxBlocks * kNodesPerBlock;

// Per-block partial sums (rho, psi, phi).  In host code this name is only a
// stand-in for the device symbol; the kernels get its device address from
// cudaGetSymbolAddress.
static __device__ __align__(256) double g_totals_scratch[3 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Pass 1: block b sums its 2048 nodes (fluid only when a mask is given) and
// writes its triple to part[3b..3b+2]; every used slot is overwritten, so no
// slot has to start at zero.
template <class T>
__global__ void __launch_bounds__(kThreads) k_totals_partial(long long N, const T* f, const T* psi, const T* phi,
                                                             const unsigned char* mask, double* part)
{
    __shared__ double smem[32 * 3];
    double v[3] = {0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * kNodesPerBlock;
    for (int k = 0; k < kNodesPerThread; ++k) {
        const long long n = base + (long long)k * kThreads + threadIdx.x;
        if (n >= N) break;
        if (mask && mask[n]) continue;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) s += (double)f[(size_t)i * N + n];
        v[0] += s;
        v[1] += (double)psi[n];
        v[2] += (double)phi[n];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    if (lane == 0)
        for (int c = 0; c < 3; ++c) smem[warp * 3 + c] = v[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += smem[w * 3 + c];
            part[3 * blockIdx.x + c] = s;
        }
    }
}

// Pass 2: one 256-thread block adds the partials in a fixed order: thread t
// sums blocks t, t + 256, t + 512, ... in turn, then a tree over the threads
// (pairs at distance 128, 64, ..., 1) gives out[3].  The order depends only
// on the block count, so every call gives the same bits for the same inputs.
constexpr int kFinalThreads = 256;
__global__ void __launch_bounds__(kFinalThreads) k_totals_final(const double* part, int nblocks, double* out)
{
    __shared__ double sm[3][kFinalThreads];
    const int t = threadIdx.x;
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = t; b < nblocks; b += kFinalThreads)
        for (int c = 0; c < 3; ++c) s[c] += part[3 * b + c];
    for (int c = 0; c < 3; ++c) sm[c][t] = s[c];
    __syncthreads();
    for (int h = kFinalThreads / 2; h > 0; h >>= 1) {
        if (t < h)
            for (int c = 0; c < 3; ++c) sm[c][t] += sm[c][t + h];
        __syncthreads();
    }
    if (t < 3) out[t] = sm[t][0];
}

// Device address of the scratch array on the current device, looked up once
// per device.
int scratch_on_current_device(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LB_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LB_ERR_PARAM;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        double* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_totals_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LB_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LB_OK;
}

}  // namespace

extern "C" int lb_totals_noalloc(int precision, int nx, int ny, int nz, const void* f, const void* psi,
                                 const void* phi, const unsigned char* mask, double* sums, void* stream)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || !f || !psi || !phi || !sums) return LB_ERR_PARAM;
    if (precision != LB_FP64 && precision != LB_FP32) return LB_ERR_PARAM;
    const long long N = (long long)nx * ny * nz;
    if (N > kMaxNodes) return LB_ERR_PARAM;   // more blocks than scratch slots
    double* part = nullptr;
    const int st = scratch_on_current_device(&part);
    if (st != LB_OK) return st;
    const int nblocks = (int)((N + kNodesPerBlock - 1) / kNodesPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    // cudaLaunchKernel reports the status of this launch itself, not an error
    // some earlier, unrelated call left behind on the thread
    void* pargs[] = {(void*)&N, (void*)&f, (void*)&psi, (void*)&phi, (void*)&mask, (void*)&part};
    const void* fn = precision == LB_FP64 ? (const void*)k_totals_partial<double>
                                          : (const void*)k_totals_partial<float>;
    if (cudaLaunchKernel(fn, dim3(nblocks), dim3(kThreads), pargs, 0, s) != cudaSuccess) return LB_ERR_CUDA;
    const double* cpart = part;
    void* fargs[] = {(void*)&cpart, (void*)&nblocks, (void*)&sums};
    if (cudaLaunchKernel((const void*)k_totals_final, dim3(1), dim3(kFinalThreads), fargs, 0, s) != cudaSuccess)
        return LB_ERR_CUDA;
    return LB_OK;
}
