// lbdp_internal.h -- interface between the C ABI (lbdp_api.cu) and the
// per-precision kernel launchers (lbdp_prec_*.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbdp_lattice.cuh"

namespace lbdp {

// Launch geometry of the row kernels: one thread per node, blocks along x.
struct RowGrid {
    dim3 grid, block;
};

// Kernel classes of one step, in launch order.
enum KernelClass { kKMu = 0, kKLinks, kKCollide, kKScalars, kKCover, kNumKernelClasses };

struct PrecOps {
    int pop_bytes;   // bytes per stored population value
    int fld_bytes;   // bytes per stored field value
    // one full time step (fluid kernels, then particle kernels when np > 0)
    cudaError_t (*step)(const DevParams&, const DevPtrs&, const RowGrid&, cudaStream_t);
    // the same step with an event recorded before the first kernel and after
    // each kernel class: ev[0..5] around mu, links, collide, scalars, cover
    cudaError_t (*step_events)(const DevParams&, const DevPtrs&, const RowGrid&, cudaStream_t, cudaEvent_t* ev);
    // staging (FP64, device) -> state; NULL entries keep the field
    cudaError_t (*set_fields)(const DevParams&, const DevPtrs&, cudaStream_t, const double* rho,
                              const double* u, const double* psi, const double* phi);
    // state -> staging (FP64, device); which: 1 rho, 2 u, 4 psi, 8 phi, 16 mu
    cudaError_t (*get_fields)(const DevParams&, const DevPtrs&, cudaStream_t, int which, double* a,
                              double* u, double* b, double* c);
    cudaError_t (*get_pop)(const DevParams&, const DevPtrs&, cudaStream_t, double* out, int i);
    // FP64 totals over fluid nodes into out[3] (device)
    cudaError_t (*sums)(const DevParams&, const DevPtrs&, cudaStream_t, double* part, int nblocks,
                        double* out);
};

extern const PrecOps kOpsF64;
extern const PrecOps kOpsF32;
extern const PrecOps kOpsF16;
extern const PrecOps kOpsBF16;

cudaError_t launch_bflag(const DevParams& P, const uint8_t* mask, uint8_t* bflag, cudaStream_t s);
cudaError_t launch_claim(const DevParams& P, uint8_t* m0, uint8_t* m1, const DevPart* parts, int p,
                         unsigned long long* count, cudaStream_t s);

}  // namespace lbdp
