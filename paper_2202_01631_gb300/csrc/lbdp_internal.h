// lbdp_internal.h -- interface between the C ABI (lbdp_api.cu,
// lbdp_batch.cu) and the per-precision kernel launchers (lbdp_prec_*.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lbdp.h"
#include "lbdp_lattice.cuh"

struct lbb_batch;

namespace lbdp {

// Launch geometry of the bulk kernels of one box.
struct RowGrid {
    dim3 zgrid;     // grid of kz_fused: 32 x 8 column tiles x z chunks
    dim3 zgrid_s;   // grid of kz_scalars, the same tiles with its own z chunks
};

// Kernel classes of one step, in the order of the sequential profile: the
// particle kernels before the bulk (pressure tensor and force next to the
// particles, link sums and particle update, boundary collide-stream), the
// fused bulk kernel, the bulk transport, the boundary transport, covering.
enum KernelClass { kKParticles = 0, kKFused, kKScalars, kKScalarsParticles, kKCover, kNumKernelClasses };

// Two more streams for the particle kernels of a step, at the device's highest
// priority.  On s: k_pt_part, k_f_part, then (after k_links) k_collide_particles
// (the nodes next to particles, which bounce back with the new particle
// velocities; then bnd_done).  On s2, after k_pt_part: k_links and
// k_cover_mark (the new mask needs only the new positions).  All of it runs
// beside kz_fused, which touches no node next to a particle.  After kz_fused
// (collide_done) k_scalars_particles and then, once the new mask is there,
// k_cover_apply run on s beside kz_scalars, which waits for bnd_done (it
// reads the velocity of the boundary nodes); the main stream ends the step
// by waiting for scal_done, which follows everything on s2 as well.
struct SideStream {
    cudaStream_t s;
    cudaEvent_t fork, bnd_done, collide_done, scal_done;
    cudaStream_t s2;   // the link sums and the new mask
    cudaEvent_t pt_done, links_done, mark_done;
    int prio;   // the stream's priority, also given to each of its launches as an attribute
};

struct PrecOps {
    int pop_bytes;   // bytes per stored population value
    int fld_bytes;   // bytes per stored field value
    // per-device kernel attributes (before the first launch or capture)
    cudaError_t (*prepare)();
    // one full time step (fluid kernels, then particle kernels when np > 0)
    cudaError_t (*step)(const DevParams&, const DevPtrs&, const RowGrid&, cudaStream_t, const SideStream*);
    // the same step with an event recorded before the first kernel and after
    // each kernel class: ev[0..5] around mu, links, collide, scalars, cover
    cudaError_t (*step_events)(const DevParams&, const DevPtrs&, const RowGrid&, cudaStream_t, cudaEvent_t* ev);
    // one bulk kernel alone over grid: which 0 kz_fused, 1 kz_scalars
    cudaError_t (*bulk)(int which, const DevParams&, const DevPtrs&, dim3 grid, cudaStream_t);
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

// One batched step over the boxes of a batch (see lbdp_batch_kernels.cuh):
// the bulk kernels with the z chunk length each one's configuration names,
// the particle kernels with the single-box split and stream order, then the
// step count of every box that ran.
struct BoxLaunch;
constexpr int kNumBatchClasses = 2;   // bulk kernels the autotuner times: fused, transport
constexpr int kNumBatchCfgs = 3;      // z chunks of 8, 16 or 32 planes per block

// A launch of up to kLaunchBoxes boxes: its parameter block and its grids.
struct LaunchPlan;

struct BatchOps {
    // per-device kernel attributes (call once before the first launch or capture)
    cudaError_t (*prepare)();
    // bulk kernel of class nc (0 fused, 1 transport) in configuration cfg over
    // one launch's boxes
    cudaError_t (*node)(int nc, int cfg, const LaunchPlan* L, cudaStream_t s);
    // the whole step at parity par over launches L[0..nl-1], then the count-down
    // of left[0..nbox-1]
    cudaError_t (*step)(const int cfg[kNumBatchClasses], LaunchPlan* L, int nl, int par, long long* left, int nbox,
                        cudaStream_t s, const SideStream* side);
};

extern const PrecOps kOpsF64;
extern const PrecOps kOpsF32;
extern const PrecOps kOpsF16;
extern const PrecOps kOpsBF16;

extern const BatchOps kBatchF64;
extern const BatchOps kBatchF32;
extern const BatchOps kBatchF16;
extern const BatchOps kBatchBF16;

cudaError_t launch_bflag(const DevParams& P, const uint8_t* mask, uint8_t* bflag, cudaStream_t s);
cudaError_t launch_claim(const DevParams& P, uint8_t* m0, uint8_t* m1, const DevPart* parts, int p,
                         unsigned long long* count, cudaStream_t s);

// Placement of a handle's device state: one region from cudaMalloc, or from
// the arena of the batch that owns the handle.
size_t handle_region_bytes(const lb_params* p);
DevPtrs handle_ptrs(const lb_handle* h, int src);
int lb_create_in(const lb_params* p, lbb_batch* batch, void* region, lb_handle** out);
// Return a member box's region to its batch and drop it from the batch.
void batch_release(lb_handle* h);

}  // namespace lbdp

// The state of one box (the lb_handle of the C ABI).
struct lb_handle {
    lb_params prm;
    lbdp::DevParams dp;
    const lbdp::PrecOps* ops;
    cudaStream_t stream;
    bool own_stream;
    int device;
    int cur;   // which buffer of each pair holds the current state
    lbb_batch* batch;   // owning batch, or NULL for a standalone box
    lbdp::SideStream side;   // particle kernels' stream (side.s NULL until created)
    void* region;       // the single device allocation holding every array below
    size_t region_bytes;
    void* f[2];
    void* psi[2];
    void* phi[2];
    void* mupsi;
    void* muphi;
    void* u;
    uint8_t* mask[2];
    lbdp::DevPart* parts;
    double* corr;   // [2] FP64 followed by [2] FP32 copies (corr_f)
    int* err;
    void* pt;
    void* force;
    uint8_t* bflag;
    double* link_part;
    unsigned* link_ticket;
    double* cover_part;
    unsigned* cover_ticket;
    long long* nfluid;
    double* staging;   // 6N FP64 for host transfers: rho, u[3], psi, phi
    double* red_part;
    double* red_out;
    unsigned long long* count;
    int red_blocks;
    int zplanes[2];   // z chunk length of kz_fused, kz_scalars (0 = size heuristic)
    // lb_step's CUDA graphs of kGraphSteps steps from parity 0 / 1, and the
    // parameters and grids they were captured with (recaptured on a change)
    cudaGraphExec_t gexec[2];
    lbdp::DevParams g_dp;
    lbdp::RowGrid g_grid;
    std::vector<lbdp::DevPart> host_parts;
    double rmax;
};
