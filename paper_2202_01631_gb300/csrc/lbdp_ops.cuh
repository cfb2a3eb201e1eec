// lbdp_ops.cuh -- launch wrappers of one precision configuration; included by
// exactly one lbdp_prec_*.cu translation unit each, so the four precision
// modes compile in parallel.
#pragma once

#include "lbdp_batch_kernels.cuh"
#include "lbdp_internal.h"
#include "lbdp_kernels.cuh"
#include "lbdp_zmarch.cuh"

namespace lbdp {

// Shared-memory carve-out hint (percent of the SM's maximum) that leaves room
// for `blocks` resident blocks of `smem` bytes each and gives the rest of the
// SM's on-chip memory to L1, which serves the halo reloads of the tiled
// stencils.  Without it the driver takes the largest carve-out the block count
// allows and leaves L1 a few tens of KB.
inline cudaError_t set_carveout(const void* fn, int blocks, size_t smem)
{
    int dev = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess || per_sm <= 0) return e;
    const size_t need = (size_t)blocks * (smem + 1024);   // 1 KB per block is reserved
    long long pct = (long long)((100 * need + per_sm - 1) / per_sm);
    if (pct > 100) pct = 100;
    return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)pct);
}

// Launch of a side-stream kernel with the side stream's priority as a launch
// attribute, so that it keeps the priority inside captured graphs too.
// The same on another stream of the side group.
template <class... A>
inline void side_launch_on(cudaStream_t st, void (*k)(A...), dim3 grid, size_t smem, const SideStream* side,
                           A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kPartThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = side->prio;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

template <class... A>
inline void side_launch(void (*k)(A...), dim3 grid, size_t smem, const SideStream* side, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kPartThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = side->s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = side->prio;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

// Resident blocks per SM the tiled force and transport kernels are given
// (measured on the 128^3 workload: 5 and 4 beat the 7 and 6 their register
// counts allow by 5 and 10 us).
constexpr int kFdivBlocks = 5, kScalBlocks = 4;

template <class C>
struct Ops {
    using R = typename C::real;
    using F = typename C::fld_t;

    static constexpr size_t kLinkSmem = block_rows_bytes<kLinkK>(kPartThreads);
    static constexpr size_t kFusedSmem = sizeof(FusedSmem<F>);
    static constexpr size_t kZScalSmem = sizeof(ScalSmem<F>);

    // Opt the kernels that use more than 48 KiB of shared memory in, once per
    // device.
    static cudaError_t prepare()
    {
        static bool done[64] = {false};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
        e = cudaFuncSetAttribute(k_links<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinkSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kz_fused<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kz_scalars<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kZScalSmem);
        if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
        return e;
    }

    static dim3 pt_grid(const DevParams& P) { return dim3(pt_part_blocks(P), P.np); }

    // One time step.  With particles and side streams: the particle kernels
    // (pressure tensor and force next to the particles, link sums and the
    // particle update with the new mask on a stream of their own, then the
    // collide-stream of the nodes next to particles) run beside kz_fused; the
    // transport of the bulk waits for the boundary collide-stream (it reads u
    // there), and the boundary transport and covering wait for kz_fused and
    // run beside it.
    // ev (optional, 6 events): the same kernels in sequence, an event before
    // the first and after each kernel class.
    static cudaError_t launch_step(const DevParams& P, const DevPtrs& D, const RowGrid& g, cudaStream_t s,
                                   cudaEvent_t* ev, const SideStream* side)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        const dim3 pg1(P.nb1, P.np), pg2(P.nb2, P.np), pgt = pt_grid(P);
        if (P.np > 0 && side && !ev) {
            cudaEventRecord(side->fork, s);
            cudaStreamWaitEvent(side->s, side->fork, 0);
            side_launch(k_pt_part<C>, pgt, 0, side, P, D);
            cudaEventRecord(side->pt_done, side->s);
            cudaStreamWaitEvent(side->s2, side->pt_done, 0);
            side_launch_on(side->s2, k_links<C>, pg1, kLinkSmem, side, P, D);
            cudaEventRecord(side->links_done, side->s2);
            side_launch_on(side->s2, k_cover_mark<C>, pg2, 0, side, P, D);
            cudaEventRecord(side->mark_done, side->s2);
            side_launch(k_f_part<C>, pg1, 0, side, P, D);
            cudaStreamWaitEvent(side->s, side->links_done, 0);
            side_launch(k_collide_particles<C>, pg1, 0, side, P, D);
            cudaEventRecord(side->bnd_done, side->s);
            kz_fused<C><<<g.zgrid, kZThreads, kFusedSmem, s>>>(P, D);
            cudaEventRecord(side->collide_done, s);
            cudaStreamWaitEvent(side->s, side->collide_done, 0);
            side_launch(k_scalars_particles<C>, pg1, 0, side, P, D);
            cudaStreamWaitEvent(side->s, side->mark_done, 0);
            // covering touches only nodes next to particles, whose fields the
            // side-stream kernels wrote, and leaves the next step's uniform
            // correction in the other buffer: it runs beside the transport
            side_launch(k_cover_apply<C>, pg2, 0, side, P, D);
            cudaEventRecord(side->scal_done, side->s);
            cudaStreamWaitEvent(s, side->bnd_done, 0);
            kz_scalars<C><<<g.zgrid_s, kZThreads, kZScalSmem, s>>>(P, D);
            cudaStreamWaitEvent(s, side->scal_done, 0);   // the step ends with the side stream
            return cudaGetLastError();
        }
        if (ev) cudaEventRecord(ev[0], s);
        if (P.np > 0) {
            k_pt_part<C><<<pgt, kPartThreads, 0, s>>>(P, D);
            k_f_part<C><<<pg1, kPartThreads, 0, s>>>(P, D);
            k_links<C><<<pg1, kPartThreads, kLinkSmem, s>>>(P, D);
            k_collide_particles<C><<<pg1, kPartThreads, 0, s>>>(P, D);
        }
        if (ev) cudaEventRecord(ev[1], s);
        kz_fused<C><<<g.zgrid, kZThreads, kFusedSmem, s>>>(P, D);
        if (ev) cudaEventRecord(ev[2], s);
        kz_scalars<C><<<g.zgrid_s, kZThreads, kZScalSmem, s>>>(P, D);
        if (ev) cudaEventRecord(ev[3], s);
        if (P.np > 0) k_scalars_particles<C><<<pg1, kPartThreads, 0, s>>>(P, D);
        if (ev) cudaEventRecord(ev[4], s);
        if (P.np > 0) {
            k_cover_mark<C><<<pg2, kPartThreads, 0, s>>>(P, D);
            k_cover_apply<C><<<pg2, kPartThreads, 0, s>>>(P, D);
        }
        if (ev) cudaEventRecord(ev[5], s);
        return cudaGetLastError();
    }

    static cudaError_t step(const DevParams& P, const DevPtrs& D, const RowGrid& g, cudaStream_t s,
                            const SideStream* side)
    {
        return launch_step(P, D, g, s, nullptr, side);
    }

    // sequential order with events around the kernel classes (the per-kernel
    // split; no overlap, so each class is timed alone)
    static cudaError_t step_events(const DevParams& P, const DevPtrs& D, const RowGrid& g, cudaStream_t s,
                                   cudaEvent_t* ev)
    {
        return launch_step(P, D, g, s, ev, nullptr);
    }

    static cudaError_t bulk(int which, const DevParams& P, const DevPtrs& D, dim3 grid, cudaStream_t s)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        if (which == 0)
            kz_fused<C><<<grid, kZThreads, kFusedSmem, s>>>(P, D);
        else
            kz_scalars<C><<<grid, kZThreads, kZScalSmem, s>>>(P, D);
        return cudaGetLastError();
    }

    static int grid1d(const DevParams& P)
    {
        long long b = (P.N + 255) / 256;
        return (int)(b < 152 * 16 ? b : 152 * 16);
    }

    static cudaError_t set_fields(const DevParams& P, const DevPtrs& D, cudaStream_t s, const double* rho,
                                  const double* u, const double* psi, const double* phi)
    {
        k_set_fields<C><<<grid1d(P), 256, 0, s>>>(P, D, rho, u, psi, phi);
        return cudaGetLastError();
    }

    static cudaError_t get_fields(const DevParams& P, const DevPtrs& D, cudaStream_t s, int which, double* a,
                                  double* u, double* b, double* c)
    {
        if (which & 16) k_mu_now<C><<<grid1d(P), 256, 0, s>>>(P, D);
        k_get_fields<C><<<grid1d(P), 256, 0, s>>>(P, D, which, a, u, b, c);
        return cudaGetLastError();
    }

    static cudaError_t get_pop(const DevParams& P, const DevPtrs& D, cudaStream_t s, double* out, int i)
    {
        k_get_pops<C><<<grid1d(P), 256, 0, s>>>(P, D, out, i);
        return cudaGetLastError();
    }

    static cudaError_t sums(const DevParams& P, const DevPtrs& D, cudaStream_t s, double* part, int nblocks,
                            double* out)
    {
        k_sums<C><<<nblocks, 256, 0, s>>>(P, D, part);
        k_sums_final<<<1, 32, 0, s>>>(part, nblocks, out);
        return cudaGetLastError();
    }

    static PrecOps table()
    {
        PrecOps t;
        t.pop_bytes = (int)sizeof(typename C::pop_t);
        t.fld_bytes = (int)sizeof(typename C::fld_t);
        t.prepare = &prepare;
        t.step = &step;
        t.step_events = &step_events;
        t.bulk = &bulk;
        t.set_fields = &set_fields;
        t.get_fields = &get_fields;
        t.get_pop = &get_pop;
        t.sums = &sums;
        return t;
    }
};

// Launchers of the batched kernels of one precision configuration.
template <class C>
struct BOps {
    using F = typename C::fld_t;
    using KFn = void (*)(BoxLaunch);

    static KFn fn(int nc, int cfg)
    {
        static_assert(kNumBatchCfgs == 3, "configuration table");
        if (nc == 0) {
            switch (cfg) {
                case 0: return kbz_fused<C, kZChunks[0]>;
                case 1: return kbz_fused<C, kZChunks[1]>;
                default: return kbz_fused<C, kZChunks[2]>;
            }
        }
        switch (cfg) {
            case 0: return kbz_scalars<C, kZChunks[0]>;
            case 1: return kbz_scalars<C, kZChunks[1]>;
            default: return kbz_scalars<C, kZChunks[2]>;
        }
    }

    static size_t smem(int nc) { return nc == 0 ? sizeof(FusedSmem<F>) : sizeof(ScalSmem<F>); }

    static cudaError_t prepare()
    {
        static bool done[64] = {false};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
        e = cudaFuncSetAttribute(kb_links<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)block_rows_bytes<kLinkK>(kPartThreads));
        for (int nc = 0; nc < kNumBatchClasses && e == cudaSuccess; ++nc)
            for (int k = 0; k < kNumBatchCfgs && e == cudaSuccess; ++k)
                e = cudaFuncSetAttribute((const void*)fn(nc, k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem(nc));
        if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
        return e;
    }

    static cudaError_t node(int nc, int cfg, const LaunchPlan* L, cudaStream_t s)
    {
        if (nc < 0 || nc >= kNumBatchClasses || cfg < 0 || cfg >= kNumBatchCfgs) return cudaErrorInvalidValue;
        void* args[] = {(void*)&L->L};
        return cudaLaunchKernel((const void*)fn(nc, cfg), L->zgrid[cfg], dim3(kZThreads), args, smem(nc), s);
    }

    // The single-box step over each launch's boxes, in the single-box order:
    // the particle kernels on the side stream beside the fused bulk kernel,
    // the bulk transport after the boundary collide-stream, the boundary
    // transport and covering beside it.
    static cudaError_t step(const int cfg[kNumBatchClasses], LaunchPlan* Ls, int nl, int par, long long* left,
                            int nbox, cudaStream_t s, const SideStream* side)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        const size_t lsm = block_rows_bytes<kLinkK>(kPartThreads);
        for (int l = 0; l < nl; ++l) {
            LaunchPlan* L = Ls + l;
            L->L.par = par;   // copied into each launch's parameters at the call
            if (side) {
                // the single-box stream order: link sums and the new mask on
                // s2 beside the force and boundary collide on s
                cudaEventRecord(side->fork, s);
                cudaStreamWaitEvent(side->s, side->fork, 0);
                side_launch(kb_pt_part<C>, L->ptg, 0, side, L->L);
                cudaEventRecord(side->pt_done, side->s);
                cudaStreamWaitEvent(side->s2, side->pt_done, 0);
                side_launch_on(side->s2, kb_links<C>, L->link, lsm, side, L->L);
                cudaEventRecord(side->links_done, side->s2);
                side_launch_on(side->s2, kb_cover_mark<C>, L->cover, 0, side, L->L);
                cudaEventRecord(side->mark_done, side->s2);
                side_launch(kb_f_part<C>, L->link, 0, side, L->L);
                cudaStreamWaitEvent(side->s, side->links_done, 0);
                side_launch(kb_collide_particles<C>, L->link, 0, side, L->L);
                cudaEventRecord(side->bnd_done, side->s);
                if ((e = node(0, cfg[0], L, s)) != cudaSuccess) return e;
                cudaEventRecord(side->collide_done, s);
                cudaStreamWaitEvent(side->s, side->collide_done, 0);
                side_launch(kb_scalars_particles<C>, L->link, 0, side, L->L);
                cudaStreamWaitEvent(side->s, side->mark_done, 0);
                side_launch(kb_cover_apply<C>, L->cover, 0, side, L->L);
                cudaEventRecord(side->scal_done, side->s);
                cudaStreamWaitEvent(s, side->bnd_done, 0);
                if ((e = node(1, cfg[1], L, s)) != cudaSuccess) return e;
                cudaStreamWaitEvent(s, side->scal_done, 0);
            } else {
                kb_pt_part<C><<<L->ptg, kPartThreads, 0, s>>>(L->L);
                kb_f_part<C><<<L->link, kPartThreads, 0, s>>>(L->L);
                kb_links<C><<<L->link, kPartThreads, lsm, s>>>(L->L);
                kb_collide_particles<C><<<L->link, kPartThreads, 0, s>>>(L->L);
                if ((e = node(0, cfg[0], L, s)) != cudaSuccess) return e;
                if ((e = node(1, cfg[1], L, s)) != cudaSuccess) return e;
                kb_scalars_particles<C><<<L->link, kPartThreads, 0, s>>>(L->L);
                kb_cover_mark<C><<<L->cover, kPartThreads, 0, s>>>(L->L);
                kb_cover_apply<C><<<L->cover, kPartThreads, 0, s>>>(L->L);
            }
        }
        kb_advance<<<(nbox + 255) / 256, 256, 0, s>>>(left, nbox);
        return cudaGetLastError();
    }

    static BatchOps table()
    {
        BatchOps t;
        t.prepare = &prepare;
        t.node = &node;
        t.prepare = &prepare;
        t.step = &step;
        return t;
    }
};

}  // namespace lbdp
