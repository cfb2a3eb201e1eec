// lbdp_api.cu -- the extern "C" entry points declared in include/lbdp.h:
// parameter validation, device allocation, host<->device staging and the
// per-step launch sequence.
#include <math.h>
#include <string.h>

#include <new>
#include <cmath>
#include <algorithm>
#include <vector>

#include "lbdp.h"
#include "lbdp_internal.h"
#include "lbdp_kernels.cuh"

using namespace lbdp;

namespace {

const PrecOps* ops_for(int prec)
{
    switch (prec) {
        case LB_FP64: return &kOpsF64;
        case LB_FP32: return &kOpsF32;
        case LB_FP16_SHIFT: return &kOpsF16;
        case LB_BF16_SHIFT: return &kOpsBF16;
        default: return nullptr;
    }
}

int validate(const lb_params* p)
{
    if (!p) return LB_ERR_PARAM;
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return LB_ERR_PARAM;
    long long N = (long long)p->nx * p->ny * p->nz;
    if (N * 19 >= (1ll << 31)) return LB_ERR_PARAM;   // 32-bit node indices
    if (!ops_for(p->precision)) return LB_ERR_PARAM;
    if (!(p->tau > 0.5) || !(p->rho0 > 0.0)) return LB_ERR_PARAM;
    if (p->kappa < 0.0 || p->M_psi < 0.0 || p->M_phi < 0.0 || p->k_d < 0.0) return LB_ERR_PARAM;
    for (int a = 0; a < 3; ++a)
        if (p->periodic[a] != 0 && p->periodic[a] != 1) return LB_ERR_PARAM;
    if (p->scalar_scheme != 0 && p->scalar_scheme != 1) return LB_ERR_PARAM;
    return LB_OK;
}

int reduction_blocks(const lb_params* p)
{
    long long N = (long long)p->nx * p->ny * p->nz;
    long long b = (N + 255) / 256;
    return (int)(b < 152 * 8 ? b : 152 * 8);
}

// Every array of a box in one region, each start aligned to 256 bytes.  With
// base == nullptr only the total is computed.
size_t layout(const lb_params* p, const PrecOps* ops, int red_blocks, lb_handle* h, char* base)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    const size_t pb = (size_t)ops->pop_bytes, fb = (size_t)ops->fld_bytes;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* r = base ? (void*)(base + off) : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return r;
    };
    lb_handle tmp;
    lb_handle* t = h ? h : &tmp;
    for (int k = 0; k < 2; ++k) t->f[k] = take(19 * N * pb);
    for (int k = 0; k < 2; ++k) {
        t->psi[k] = take(N * fb);
        t->phi[k] = take(N * fb);
        t->mask[k] = (uint8_t*)take(N);
    }
    t->mupsi = take(N * fb);
    t->muphi = take(N * fb);
    t->u = take(3 * N * fb);
    t->force = take(3 * N * fb);
    t->pt = take(kPtFields * N * fb);
    t->bflag = (uint8_t*)take(N);
    t->parts = (DevPart*)take(kMaxParticles * sizeof(DevPart));
    t->corr = (double*)take(8 * sizeof(double));   // [step parity][psi, phi FP64; psi, phi FP32]
    t->err = (int*)take(sizeof(int));
    t->link_part = (double*)take((size_t)kMaxParticles * kMaxPartBlocks * kLinkK * sizeof(double));
    t->link_ticket = (unsigned*)take(kMaxParticles * sizeof(unsigned));
    t->cover_part = (double*)take((size_t)kMaxParticles * kMaxPartBlocks * kCoverK * sizeof(double));
    t->cover_ticket = (unsigned*)take(sizeof(unsigned));
    t->nfluid = (long long*)take(sizeof(long long));
    t->staging = (double*)take(6 * N * sizeof(double));
    t->red_part = (double*)take((size_t)red_blocks * 3 * sizeof(double));
    t->red_out = (double*)take(3 * sizeof(double));
    t->count = (unsigned long long*)take(sizeof(unsigned long long));
    return off;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LB_OK : (e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA); }

#define LB_TRY(expr)                                   \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

DevPtrs ptrs(const lb_handle* h, int src)
{
    DevPtrs d;
    const int dst = src ^ 1;
    d.f_src = h->f[src];
    d.f_dst = h->f[dst];
    d.psi_src = h->psi[src];
    d.psi_dst = h->psi[dst];
    d.phi_src = h->phi[src];
    d.phi_dst = h->phi[dst];
    d.mupsi = h->mupsi;
    d.muphi = h->muphi;
    d.u = h->u;
    d.mask = h->mask[src];
    d.mask_next = h->mask[dst];
    d.parts = h->parts;
    d.corr = h->corr + 4 * src;
    d.corr_f = (float*)(h->corr + 4 * src + 2);
    d.corr_next = h->corr + 4 * dst;
    d.corr_f_next = (float*)(h->corr + 4 * dst + 2);
    d.err = h->err;
    d.pt = h->pt;
    d.force = h->force;
    d.bflag = h->bflag;
    d.link_part = h->link_part;
    d.link_ticket = h->link_ticket;
    d.cover_part = h->cover_part;
    d.cover_ticket = h->cover_ticket;
    d.nfluid = h->nfluid;
    return d;
}

// Pointers for set/get of the current state: both src and dst name the
// current buffers.
DevPtrs cur_ptrs(const lb_handle* h)
{
    DevPtrs d = ptrs(h, h->cur);
    d.f_dst = h->f[h->cur];
    d.psi_dst = h->psi[h->cur];
    d.phi_dst = h->phi[h->cur];
    d.mask_next = h->mask[h->cur];
    return d;
}

// z chunk length the size heuristic picks: enough chunks for about six waves
// of four blocks per SM on 152 SMs, each chunk at least 6 planes long
// (measured on GB300: 256^3 is fastest with chunks of 12 to 24 planes, 128^3
// with 6 to 8; shorter chunks repeat more halo planes, fewer blocks leave SMs
// idle).  lb_tune replaces it with a measured choice.
int default_planes(const DevParams& P)
{
    const long long cols = (long long)((P.nx + 31) / 32) * ((P.ny + 7) / 8);
    const long long target = 152LL * 4 * 6;
    long long chunks = (target + cols - 1) / cols;
    const long long max_chunks = P.nz / 6 > 1 ? P.nz / 6 : 1;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    return (int)((P.nz + chunks - 1) / chunks);
}

// Grid of a z-marching kernel with chunks of `planes` planes (no empty chunk).
dim3 zm_grid(const DevParams& P, int planes)
{
    if (planes < 1) planes = 1;
    if (planes > P.nz) planes = P.nz;
    const int chunks = (P.nz + planes - 1) / planes;
    return dim3((P.nx + 31) / 32, (P.ny + 7) / 8, (unsigned)chunks);
}

RowGrid row_grid(const lb_handle* h)
{
    RowGrid g;
    const int d = default_planes(h->dp);
    g.zgrid = zm_grid(h->dp, h->zplanes[0] > 0 ? h->zplanes[0] : d);
    g.zgrid_s = zm_grid(h->dp, h->zplanes[1] > 0 ? h->zplanes[1] : d);
    return g;
}

void update_sides(lb_handle* h)
{
    const int L[3] = {h->dp.nx, h->dp.ny, h->dp.nz};
    const int rc = (int)ceil(h->rmax);
    for (int a = 0; a < 3; ++a) {
        int s1 = 2 * rc + 6, s2 = 2 * rc + 9;
        if (h->dp.per[a]) {
            if (s1 > L[a]) s1 = L[a];
            if (s2 > L[a]) s2 = L[a];
        }
        h->dp.side1[a] = s1;
        h->dp.side2[a] = s2;
    }
    // blocks per particle: about one box node per thread, at most kMaxPartBlocks
    const long long t1 = (long long)h->dp.side1[0] * h->dp.side1[1] * h->dp.side1[2];
    const long long t2 = (long long)h->dp.side2[0] * h->dp.side2[1] * h->dp.side2[2];
    const long long b1 = (t1 + 255) / 256, b2 = (t2 + 255) / 256;
    h->dp.nb1 = (int)(b1 < kMaxPartBlocks ? (b1 > 0 ? b1 : 1) : kMaxPartBlocks);
    h->dp.nb2 = (int)(b2 < kMaxPartBlocks ? (b2 > 0 ? b2 : 1) : kMaxPartBlocks);
}

void drop_step_graphs(lb_handle* h)
{
    for (cudaGraphExec_t& g : h->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

void free_all(lb_handle* h)
{
    if (h->device >= 0) cudaSetDevice(h->device);
    drop_step_graphs(h);
    if (h->side.s) {
        cudaStreamSynchronize(h->side.s);
        cudaStreamDestroy(h->side.s);
        cudaEventDestroy(h->side.fork);
        cudaEventDestroy(h->side.bnd_done);
        cudaEventDestroy(h->side.collide_done);
        cudaEventDestroy(h->side.scal_done);
        if (h->side.s2) {
            cudaStreamSynchronize(h->side.s2);
            cudaStreamDestroy(h->side.s2);
            cudaEventDestroy(h->side.pt_done);
            cudaEventDestroy(h->side.links_done);
            cudaEventDestroy(h->side.mark_done);
            h->side.s2 = nullptr;
        }
        h->side.s = nullptr;
    }
    if (h->batch)
        batch_release(h);
    else if (h->region)
        cudaFree(h->region);
    h->region = nullptr;
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

double mimg(double d, int L, int per)
{
    if (per) {
        if (d > 0.5 * L)
            d -= L;
        else if (d < -0.5 * L)
            d += L;
    }
    return d;
}

int read_err(lb_handle* h)
{
    int e = 0;
    LB_TRY(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LB_TRY(cudaStreamSynchronize(h->stream));
    if (e & (kErrOverlap | kErrWall)) return LB_ERR_OVERLAP;
    if (e & kErrSolve) return LB_ERR_NONFINITE;
    return LB_OK;
}


// Steps per captured graph of lb_step (even: a launch leaves the parity).
constexpr int kGraphSteps = 8;

bool same_grid(const dim3& a, const dim3& b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

// kGraphSteps steps from parity p0 captured on the handle's stream.
int capture_steps(lb_handle* h, const RowGrid& g, int p0)
{
    LB_TRY(h->ops->prepare());
    cudaGraph_t graph = nullptr;
    LB_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int st = LB_OK;
    for (int t = 0; t < kGraphSteps && st == LB_OK; ++t)
        st = cuda_status(h->ops->step(h->dp, ptrs(h, (p0 + t) & 1), g, h->stream, h->side.s ? &h->side : nullptr));
    const cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (st == LB_OK) st = cuda_status(e);
    if (st == LB_OK) st = cuda_status(cudaGraphInstantiate(&h->gexec[p0], graph, 0));
    if (graph) cudaGraphDestroy(graph);
    if (st != LB_OK) {
        h->gexec[p0] = nullptr;
        cudaGetLastError();
    }
    return st;
}

// Whether lb_step may capture on the handle's stream: not the legacy default
// stream, and not while the caller is capturing it into a graph of its own
// (then the plain launches become part of the caller's graph).
bool can_capture(lb_handle* h)
{
    if (!h->stream) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

}  // namespace

extern "C" {

int lb_device_bytes(const lb_params* p, size_t* bytes)
{
    int st = validate(p);
    if (st != LB_OK || !bytes) return LB_ERR_PARAM;
    *bytes = handle_region_bytes(p);
    return LB_OK;
}

int lb_create(const lb_params* p, lb_handle** out) { return lbdp::lb_create_in(p, nullptr, nullptr, out); }

void lb_destroy(lb_handle* h)
{
    if (!h) return;
    if (h->device >= 0) cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int lb_set_fields(lb_handle* h, const double* rho, const double* u, const double* psi, const double* phi)
{
    if (!h) return LB_ERR_PARAM;
    const size_t N = (size_t)h->dp.N;
    // a non-finite input would spread through the whole box in a few steps:
    // refuse it before anything is copied
    const struct {
        const double* a;
        size_t n;
    } in[4] = {{rho, N}, {u, 3 * N}, {psi, N}, {phi, N}};
    for (const auto& v : in)
        if (v.a)
            for (size_t k = 0; k < v.n; ++k)
                if (!std::isfinite(v.a[k])) return LB_ERR_NONFINITE;
    cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    double* st_rho = h->staging;
    double* st_u = h->staging + N;
    double* st_psi = h->staging + 4 * N;
    double* st_phi = h->staging + 5 * N;
    if (rho) LB_TRY(cudaMemcpyAsync(st_rho, rho, N * sizeof(double), cudaMemcpyHostToDevice, s));
    if (u) LB_TRY(cudaMemcpyAsync(st_u, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s));
    if (psi) LB_TRY(cudaMemcpyAsync(st_psi, psi, N * sizeof(double), cudaMemcpyHostToDevice, s));
    if (phi) LB_TRY(cudaMemcpyAsync(st_phi, phi, N * sizeof(double), cudaMemcpyHostToDevice, s));
    // one pass: fields from staging (or current value plus the pending uniform
    // correction), populations to equilibrium; then the correction is spent
    LB_TRY(h->ops->set_fields(h->dp, cur_ptrs(h), s, rho ? st_rho : nullptr, u ? st_u : nullptr,
                              psi ? st_psi : nullptr, phi ? st_phi : nullptr));
    LB_TRY(cudaMemsetAsync(h->corr, 0, 8 * sizeof(double), s));
    return LB_OK;
}

double lb_wetting_h(double theta_deg)
{
    const double target = cos(theta_deg * M_PI / 180.0);
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double v = 0.5 * (pow(1.0 + mid, 1.5) - pow(1.0 - mid, 1.5));
        if (v < target)
            lo = mid;
        else
            hi = mid;
        if (hi - lo < 1e-16) break;
    }
    return 0.5 * (lo + hi);
}

double lb_solubility_E(double ratio, double phi_b) { return phi_b * (ratio - 1.0) / ((ratio + 1.0) * tanh(1.0)); }

int lb_add_particle(lb_handle* h, const lb_particle_desc* d, int* id_out)
{
    if (!h || !d) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const DevParams& P = h->dp;
    if ((int)h->host_parts.size() >= kMaxParticles) return LB_ERR_PARAM;
    if (!(d->R > 0.0)) return LB_ERR_PARAM;
    const double mn = sqrt(d->m_hat[0] * d->m_hat[0] + d->m_hat[1] * d->m_hat[1] + d->m_hat[2] * d->m_hat[2]);
    if (!(mn > 0.0)) return LB_ERR_PARAM;
    double H = d->H;
    if (!isnan(d->theta_c_deg)) {
        if (d->theta_c_deg < 0.0 || d->theta_c_deg > 180.0) return LB_ERR_PARAM;
        H = lb_wetting_h(d->theta_c_deg) * sqrt(P.kappa * P.A);
    }
    if (H != 0.0 && !(P.kappa > 0.0)) return LB_ERR_PARAM;
    const int L[3] = {P.nx, P.ny, P.nz};
    DevPart q;
    memset(&q, 0, sizeof(q));
    for (int a = 0; a < 3; ++a) {
        double X = d->pos[a];
        if (P.per[a]) {
            if (X < 0.0 || X >= L[a]) return LB_ERR_PARAM;
        } else if (X - d->R < 1.0 || X + d->R > L[a] - 2.0) {
            return LB_ERR_OVERLAP;
        }
        q.X[a] = X;
        q.Xn[a] = X;
        q.U[a] = d->vel[a];
        q.W[a] = d->omega[a];
        q.m[a] = d->m_hat[a] / mn;
        q.mn[a] = q.m[a];
        q.ext_f[a] = d->ext_force[a];
        q.ext_t[a] = d->ext_torque[a];
    }
    // the covering box must not wrap onto itself on a periodic axis
    for (const DevPart& o : h->host_parts) {
        double r[3];
        for (int a = 0; a < 3; ++a) r[a] = mimg(q.X[a] - o.X[a], L[a], P.per[a]);
        if (sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) < d->R + o.R + 1.0) return LB_ERR_OVERLAP;
    }
    q.R = d->R;
    q.R2 = d->R * d->R;
    q.Rc = (int)ceil(d->R);
    q.R2f = (float)q.R2;
    q.rmarg = solid_margin(d->R);
    q.smarg = side_margin(d->R);
    fill_geo(q.X, q.g);
    q.gn = q.g;
    for (int a = 0; a < 3; ++a) q.mf[a] = (float)q.m[a];
    const double rp = d->rho_p > 0.0 ? d->rho_p : 1.0;
    q.M = rp * (4.0 / 3.0) * M_PI * d->R * d->R * d->R;
    q.I = 0.4 * q.M * d->R * d->R;
    q.alpha = d->alpha;
    q.mu_p = d->mu_plus;
    q.mu_m = d->mu_minus;
    q.H = H;
    q.Hk = H != 0.0 ? H / P.kappa : 0.0;
    q.Hk_f = (float)q.Hk;
    q.alpha_f = (float)q.alpha;
    q.mu_pf = (float)q.mu_p;
    q.mu_mf = (float)q.mu_m;
    for (int a = 0; a < 3; ++a) {
        q.Uf[a] = (float)q.U[a];
        q.Wf[a] = (float)q.W[a];
    }
    q.fixed = d->fixed ? 1 : 0;
    const int k = (int)h->host_parts.size();
    // fetch the device copies first: earlier particles have moved
    if (k > 0) {
        h->host_parts.resize(k);
        LB_TRY(cudaMemcpyAsync(h->host_parts.data(), h->parts, k * sizeof(DevPart), cudaMemcpyDeviceToHost,
                               h->stream));
        LB_TRY(cudaStreamSynchronize(h->stream));
    }
    h->host_parts.push_back(q);
    LB_TRY(cudaMemcpyAsync(h->parts + k, &h->host_parts[k], sizeof(DevPart), cudaMemcpyHostToDevice, h->stream));
    unsigned long long zero = 0, cnt = 0;
    LB_TRY(cudaMemcpyAsync(h->count, &zero, sizeof(zero), cudaMemcpyHostToDevice, h->stream));
    LB_TRY(launch_claim(P, h->mask[h->cur], h->mask[h->cur ^ 1], h->parts, k, h->count, h->stream));
    LB_TRY(launch_bflag(P, h->mask[h->cur], h->bflag, h->stream));
    long long nf = 0;
    LB_TRY(cudaMemcpyAsync(&cnt, h->count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    LB_TRY(cudaMemcpyAsync(&nf, h->nfluid, sizeof(nf), cudaMemcpyDeviceToHost, h->stream));
    LB_TRY(cudaStreamSynchronize(h->stream));
    nf -= (long long)cnt;
    LB_TRY(cudaMemcpyAsync(h->nfluid, &nf, sizeof(nf), cudaMemcpyHostToDevice, h->stream));
    LB_TRY(cudaStreamSynchronize(h->stream));
    h->dp.np = k + 1;
    if (d->R > h->rmax) h->rmax = d->R;
    update_sides(h);
    if (id_out) *id_out = k;
    return LB_OK;
}

int lb_step(lb_handle* h, int nsteps)
{
    if (!h || nsteps < 0) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const RowGrid g = row_grid(h);
    int t = 0;
    // A box without particles runs whole groups of kGraphSteps steps as one
    // graph launch each (measured on GB300: 170 instead of 174 us per step at
    // 128^3); the graphs are captured again when the parameters or the launch
    // grids have changed since.  With particles the step forks onto the side
    // stream, and the captured form measured slower than the plain launches
    // (283 instead of 245 us at 128^3 with one sphere, the side kernels'
    // priority attribute notwithstanding), so those steps stay plain.
    if (h->dp.np == 0 && nsteps >= kGraphSteps && can_capture(h)) {
        if (memcmp(&h->g_dp, &h->dp, sizeof(DevParams)) != 0 || !same_grid(h->g_grid.zgrid, g.zgrid) ||
            !same_grid(h->g_grid.zgrid_s, g.zgrid_s)) {
            drop_step_graphs(h);
            memcpy(&h->g_dp, &h->dp, sizeof(DevParams));
            h->g_grid = g;
        }
        for (; nsteps - t >= kGraphSteps; t += kGraphSteps) {
            if (!h->gexec[h->cur]) {
                const int st = capture_steps(h, g, h->cur);
                if (st != LB_OK) return st;
            }
            LB_TRY(cudaGraphLaunch(h->gexec[h->cur], h->stream));
        }
    }
    for (; t < nsteps; ++t) {
        LB_TRY(h->ops->step(h->dp, ptrs(h, h->cur), g, h->stream, h->side.s ? &h->side : nullptr));
        h->cur ^= 1;
    }
    return LB_OK;
}

int lb_profile_step(lb_handle* h, int nsteps, double* ms, int* launches)
{
    if (!h || nsteps < 0 || !ms) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const RowGrid g = row_grid(h);
    std::vector<cudaEvent_t> ev((size_t)nsteps * 6);
    for (auto& e : ev) LB_TRY(cudaEventCreate(&e));
    int st = LB_OK;
    for (int t = 0; t < nsteps && st == LB_OK; ++t) {
        cudaError_t e = h->ops->step_events(h->dp, ptrs(h, h->cur), g, h->stream, &ev[(size_t)t * 6]);
        if (e != cudaSuccess) st = cuda_status(e);
        h->cur ^= 1;
    }
    for (int k = 0; k < kNumKernelClasses; ++k) ms[k] = 0.0;
    if (st == LB_OK) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_status(e);
    }
    for (int t = 0; t < nsteps && st == LB_OK; ++t)
        for (int k = 0; k < kNumKernelClasses; ++k) {
            float v = 0.f;
            cudaEventElapsedTime(&v, ev[(size_t)t * 6 + k], ev[(size_t)t * 6 + k + 1]);
            ms[k] += v;
        }
    for (auto& e : ev) cudaEventDestroy(e);
    if (launches) *launches = nsteps * (h->dp.np > 0 ? 9 : 2);
    return st;
}

int lb_tune(lb_handle* h, int reps, int planes_out[2], double ms_out[2])
{
    if (!h || reps < 1) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    const DevParams& P = h->dp;
    const DevPtrs D = ptrs(h, h->cur);
    // kz_fused rewrites the stored velocity of the bulk nodes: keep a copy
    const size_t ub = 3 * (size_t)P.N * h->ops->fld_bytes;
    LB_TRY(cudaMemcpyAsync(h->staging, h->u, ub, cudaMemcpyDeviceToDevice, s));
    // candidate chunk lengths, each kept once after rounding to equal chunks
    static const int kCand[] = {4, 6, 8, 12, 16, 24, 32, 48, 64};
    std::vector<int> cand;
    for (int c : kCand) {
        if (c > P.nz && !cand.empty()) break;
        const int p = (int)zm_grid(P, c).z;
        const int planes = (P.nz + p - 1) / p;
        if (std::find(cand.begin(), cand.end(), planes) == cand.end()) cand.push_back(planes);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = cuda_status(cudaEventCreate(&e0));
    if (st == LB_OK) st = cuda_status(cudaEventCreate(&e1));
    int best[2] = {0, 0};
    double best_ms[2] = {1e300, 1e300};
    // kz_scalars reads the chemical potentials and velocity kz_fused leaves:
    // one kz_fused launch first gives it the inputs of a step
    for (int which = 0; which < 2 && st == LB_OK; ++which) {
        for (int planes : cand) {
            const dim3 grid = zm_grid(P, planes);
            for (int w = 0; w < 2 && st == LB_OK; ++w) st = cuda_status(h->ops->bulk(which, P, D, grid, s));
            if (st == LB_OK) st = cuda_status(cudaEventRecord(e0, s));
            for (int r = 0; r < reps && st == LB_OK; ++r) st = cuda_status(h->ops->bulk(which, P, D, grid, s));
            if (st == LB_OK) st = cuda_status(cudaEventRecord(e1, s));
            if (st == LB_OK) st = cuda_status(cudaEventSynchronize(e1));
            float ms = 0.f;
            if (st == LB_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
            if (st != LB_OK) break;
            if (ms / reps < best_ms[which]) {
                best_ms[which] = ms / reps;
                best[which] = planes;
            }
        }
    }
    {
        const cudaError_t e = cudaMemcpyAsync(h->u, h->staging, ub, cudaMemcpyDeviceToDevice, s);
        if (st == LB_OK) st = cuda_status(e);
    }
    if (st == LB_OK) st = cuda_status(cudaStreamSynchronize(s));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != LB_OK) return st;
    for (int k = 0; k < 2; ++k) {
        h->zplanes[k] = best[k];
        if (planes_out) planes_out[k] = best[k];
        if (ms_out) ms_out[k] = best_ms[k];
    }
    return LB_OK;
}

int lb_set_planes(lb_handle* h, const int planes[2])
{
    if (!h || !planes) return LB_ERR_PARAM;
    for (int k = 0; k < 2; ++k)
        if (planes[k] < 0) return LB_ERR_PARAM;
    for (int k = 0; k < 2; ++k) h->zplanes[k] = planes[k] > h->dp.nz ? h->dp.nz : planes[k];
    return LB_OK;
}

int lb_get_planes(const lb_handle* h, int planes[2])
{
    if (!h || !planes) return LB_ERR_PARAM;
    const RowGrid g = row_grid(h);
    planes[0] = (h->dp.nz + (int)g.zgrid.z - 1) / (int)g.zgrid.z;
    planes[1] = (h->dp.nz + (int)g.zgrid_s.z - 1) / (int)g.zgrid_s.z;
    return LB_OK;
}

int lb_step_launches(const lb_handle* h, int nsteps)
{
    if (!h || nsteps < 0) return LB_ERR_PARAM;
    return nsteps * (h->dp.np > 0 ? 9 : 2);
}

int lb_sync(lb_handle* h)
{
    if (!h) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    LB_TRY(cudaStreamSynchronize(h->stream));
    return read_err(h);
}

int lb_read_fields(lb_handle* h, double* rho, double* u, double* psi, double* phi)
{
    if (!h) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const size_t N = (size_t)h->dp.N;
    cudaStream_t s = h->stream;
    const DevPtrs D = cur_ptrs(h);
    struct {
        double* host;
        int bit;
        size_t n;
    } items[4] = {{rho, 1, N}, {u, 2, 3 * N}, {psi, 4, N}, {phi, 8, N}};
    for (auto& it : items) {
        if (!it.host) continue;
        double* st = h->staging;
        LB_TRY(h->ops->get_fields(h->dp, D, s, it.bit, st, st, st, st));
        LB_TRY(cudaMemcpyAsync(it.host, st, it.n * sizeof(double), cudaMemcpyDeviceToHost, s));
        LB_TRY(cudaStreamSynchronize(s));
    }
    return read_err(h);
}

int lb_read_mu(lb_handle* h, double* mu_psi, double* mu_phi)
{
    if (!h || !mu_psi || !mu_phi) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const size_t N = (size_t)h->dp.N;
    cudaStream_t s = h->stream;
    LB_TRY(h->ops->get_fields(h->dp, cur_ptrs(h), s, 16, h->staging, nullptr, h->staging + N, nullptr));
    LB_TRY(cudaMemcpyAsync(mu_psi, h->staging, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(mu_phi, h->staging + N, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaStreamSynchronize(s));
    return LB_OK;
}

int lb_read_populations(lb_handle* h, double* f)
{
    if (!h || !f) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const size_t N = (size_t)h->dp.N;
    cudaStream_t s = h->stream;
    for (int i = 0; i < 19; ++i) {
        LB_TRY(h->ops->get_pop(h->dp, cur_ptrs(h), s, h->staging, i));
        LB_TRY(cudaMemcpyAsync(f + (size_t)i * N, h->staging, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        LB_TRY(cudaStreamSynchronize(s));
    }
    return LB_OK;
}

int lb_read_mask(lb_handle* h, unsigned char* mask)
{
    if (!h || !mask) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    LB_TRY(cudaMemcpyAsync(mask, h->mask[h->cur], (size_t)h->dp.N, cudaMemcpyDeviceToHost, h->stream));
    LB_TRY(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

// Checkpoint blob: header, then the arrays of the current state in a fixed
// order (current-parity buffers; the correction pair of the current parity
// first).
namespace {
constexpr unsigned long long kStateMagic = 0x4C42445053544154ull;   // "LBDPSTAT"
struct StateHeader {
    unsigned long long magic;
    int version, nx, ny, nz, precision, scheme, thermo, np;
    int periodic[3];
    double tau, rho0, g[3], A, kappa, Mpsi, C, Mphi, E, phib, kd;
};

size_t state_layout(const lb_handle* h, int np, size_t* off)
{
    const size_t N = (size_t)h->dp.N;
    const size_t pb = (size_t)h->ops->pop_bytes, fb = (size_t)h->ops->fld_bytes;
    const size_t sz[] = {sizeof(StateHeader), 19 * N * pb, N * fb, N * fb, 3 * N * fb, N, N,
                         (size_t)np * sizeof(DevPart), 8 * sizeof(double), sizeof(long long), sizeof(int)};
    size_t o = 0;
    for (int k = 0; k < 11; ++k) {
        if (off) off[k] = o;
        o += (sz[k] + 15) & ~(size_t)15;
    }
    return o;
}

void fill_header(const lb_handle* h, int np, StateHeader& H)
{
    memset(&H, 0, sizeof(H));
    H.magic = kStateMagic;
    H.version = 1;
    H.nx = h->dp.nx;
    H.ny = h->dp.ny;
    H.nz = h->dp.nz;
    H.precision = h->prm.precision;
    H.scheme = h->dp.scheme;
    H.thermo = h->dp.thermo;
    H.np = np;
    for (int a = 0; a < 3; ++a) {
        H.periodic[a] = h->dp.per[a];
        H.g[a] = h->dp.g[a];
    }
    H.tau = h->dp.tau;
    H.rho0 = h->dp.rho0;
    H.A = h->dp.A;
    H.kappa = h->dp.kappa;
    H.Mpsi = h->dp.Mpsi;
    H.C = h->dp.C;
    H.Mphi = h->dp.Mphi;
    H.E = h->dp.E;
    H.phib = h->dp.phib;
    H.kd = h->dp.kd;
}
}  // namespace

int lb_state_bytes(const lb_handle* h, size_t* bytes)
{
    if (!h || !bytes) return LB_ERR_PARAM;
    *bytes = state_layout(h, h->dp.np, nullptr);
    return LB_OK;
}

int lb_save_state(lb_handle* h, void* buf, size_t bytes)
{
    if (!h || !buf) return LB_ERR_PARAM;
    size_t off[11];
    if (bytes < state_layout(h, h->dp.np, off)) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    unsigned char* b = (unsigned char*)buf;
    const size_t N = (size_t)h->dp.N;
    const size_t pb = (size_t)h->ops->pop_bytes, fb = (size_t)h->ops->fld_bytes;
    const int c = h->cur;
    StateHeader H;
    fill_header(h, h->dp.np, H);
    memcpy(b + off[0], &H, sizeof(H));
    cudaStream_t s = h->stream;
    LB_TRY(cudaMemcpyAsync(b + off[1], h->f[c], 19 * N * pb, cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[2], h->psi[c], N * fb, cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[3], h->phi[c], N * fb, cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[4], h->u, 3 * N * fb, cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[5], h->mask[c], N, cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[6], h->bflag, N, cudaMemcpyDeviceToHost, s));
    if (h->dp.np > 0)
        LB_TRY(cudaMemcpyAsync(b + off[7], h->parts, (size_t)h->dp.np * sizeof(DevPart), cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[8], h->corr + 4 * c, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[8] + 4 * sizeof(double), h->corr + 4 * (c ^ 1), 4 * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[9], h->nfluid, sizeof(long long), cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaMemcpyAsync(b + off[10], h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LB_TRY(cudaStreamSynchronize(s));
    return LB_OK;
}

int lb_load_state(lb_handle* h, const void* buf, size_t bytes)
{
    if (!h || !buf || bytes < sizeof(StateHeader)) return LB_ERR_PARAM;
    if (h->batch) return LB_ERR_STATE;   // a batch member's launch plans hold its particle boxes
    const unsigned char* b = (const unsigned char*)buf;
    StateHeader H, mine;
    memcpy(&H, b, sizeof(H));
    if (H.magic != kStateMagic || H.version != 1 || H.np < 0 || H.np > kMaxParticles) return LB_ERR_PARAM;
    fill_header(h, H.np, mine);
    if (memcmp(&H, &mine, sizeof(H)) != 0) return LB_ERR_PARAM;   // another box or model
    size_t off[11];
    if (bytes < state_layout(h, H.np, off)) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const size_t N = (size_t)h->dp.N;
    const size_t pb = (size_t)h->ops->pop_bytes, fb = (size_t)h->ops->fld_bytes;
    const int c = h->cur;
    cudaStream_t s = h->stream;
    LB_TRY(cudaStreamSynchronize(s));
    std::vector<DevPart> parts((size_t)H.np);
    if (H.np > 0) memcpy(parts.data(), b + off[7], (size_t)H.np * sizeof(DevPart));
    LB_TRY(cudaMemcpyAsync(h->f[c], b + off[1], 19 * N * pb, cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->psi[c], b + off[2], N * fb, cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->phi[c], b + off[3], N * fb, cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->u, b + off[4], 3 * N * fb, cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->mask[c], b + off[5], N, cudaMemcpyHostToDevice, s));
    // the other mask buffer holds the same mask: covering writes only the
    // cover box of each sphere into it
    LB_TRY(cudaMemcpyAsync(h->mask[c ^ 1], b + off[5], N, cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->bflag, b + off[6], N, cudaMemcpyHostToDevice, s));
    if (H.np > 0)
        LB_TRY(cudaMemcpyAsync(h->parts, parts.data(), (size_t)H.np * sizeof(DevPart), cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->corr + 4 * c, b + off[8], 4 * sizeof(double), cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->corr + 4 * (c ^ 1), b + off[8] + 4 * sizeof(double), 4 * sizeof(double),
                           cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->nfluid, b + off[9], sizeof(long long), cudaMemcpyHostToDevice, s));
    LB_TRY(cudaMemcpyAsync(h->err, b + off[10], sizeof(int), cudaMemcpyHostToDevice, s));
    LB_TRY(cudaStreamSynchronize(s));
    h->host_parts = parts;
    h->dp.np = H.np;
    h->rmax = 0.0;
    for (const DevPart& q : parts)
        if (q.R > h->rmax) h->rmax = q.R;
    update_sides(h);
    return LB_OK;
}

int lb_read_particles(lb_handle* h, lb_particle_state* out, int cap, int* n_out)
{
    if (!h || cap < 0 || (cap > 0 && !out)) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    const int np = h->dp.np;
    if (n_out) *n_out = np;
    const int n = np < cap ? np : cap;
    if (n == 0) return read_err(h);
    std::vector<DevPart> tmp(n);
    LB_TRY(cudaMemcpyAsync(tmp.data(), h->parts, n * sizeof(DevPart), cudaMemcpyDeviceToHost, h->stream));
    LB_TRY(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) {
            out[k].pos[a] = tmp[k].X[a];
            out[k].vel[a] = tmp[k].U[a];
            out[k].omega[a] = tmp[k].W[a];
            out[k].m_hat[a] = tmp[k].m[a];
            out[k].force[a] = tmp[k].force[a];
            out[k].torque[a] = tmp[k].torque[a];
        }
    return read_err(h);
}

int lb_conservation(lb_handle* h, double sums[3])
{
    if (!h || !sums) return LB_ERR_PARAM;
    cudaSetDevice(h->device);
    LB_TRY(h->ops->sums(h->dp, cur_ptrs(h), h->stream, h->red_part, h->red_blocks, h->red_out));
    LB_TRY(cudaMemcpyAsync(sums, h->red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB_TRY(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 3; ++k)
        if (!isfinite(sums[k])) return LB_ERR_NONFINITE;
    return read_err(h);
}

const char* lb_error_string(int status)
{
    switch (status) {
        case LB_OK: return "ok";
        case LB_ERR_PARAM: return "invalid argument or parameter";
        case LB_ERR_NOMEM: return "device allocation failed";
        case LB_ERR_NONFINITE: return "non-finite state (NaN/Inf or singular particle system)";
        case LB_ERR_OVERLAP: return "particles met or a particle reached a wall";
        case LB_ERR_CUDA: return "CUDA call failed";
        case LB_ERR_TIMEOUT: return "device wait expired";
        case LB_ERR_STATE: return "call not valid in this state";
        case LB_ERR_CANCELLED: return "request cancelled";
        default: return "unknown status";
    }
}

}  // extern "C"

namespace lbdp {
cudaError_t launch_bflag(const DevParams& P, const uint8_t* mask, uint8_t* bflag, cudaStream_t s)
{
    long long b = (P.N + 255) / 256;
    int blocks = (int)(b < 152 * 16 ? b : 152 * 16);
    k_bflag_all<<<blocks, 256, 0, s>>>(P, mask, bflag);
    return cudaGetLastError();
}

cudaError_t launch_claim(const DevParams& P, uint8_t* m0, uint8_t* m1, const DevPart* parts, int p,
                         unsigned long long* count, cudaStream_t s)
{
    long long b = (P.N + 255) / 256;
    int blocks = (int)(b < 152 * 16 ? b : 152 * 16);
    k_claim<<<blocks, 256, 0, s>>>(P, m0, m1, parts, p, count);
    return cudaGetLastError();
}
}  // namespace lbdp

namespace lbdp {

size_t handle_region_bytes(const lb_params* p)
{
    return layout(p, ops_for(p->precision), reduction_blocks(p), nullptr, nullptr);
}

DevPtrs handle_ptrs(const lb_handle* h, int src) { return ptrs(h, src); }

// Create a box.  region == nullptr: the box allocates its own region;
// otherwise region (handle_region_bytes(p) bytes, 256-byte aligned) belongs to
// batch, which takes it back through batch_release.
int lb_create_in(const lb_params* p, lbb_batch* batch, void* region, lb_handle** out)
{
    if (!out) return LB_ERR_PARAM;
    *out = nullptr;
    int st = validate(p);
    if (st != LB_OK) return st;
    lb_handle* h = new (std::nothrow) lb_handle();
    if (!h) return LB_ERR_NOMEM;
    h->prm = *p;
    h->ops = ops_for(p->precision);
    h->device = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        delete h;
        return LB_ERR_CUDA;
    }
    h->device = dev;
    DevParams& P = h->dp;
    memset(&P, 0, sizeof(P));
    P.nx = p->nx;
    P.ny = p->ny;
    P.nz = p->nz;
    for (int a = 0; a < 3; ++a) {
        P.per[a] = p->periodic[a];
        P.g[a] = p->body_force[a];
    }
    P.N = (long long)p->nx * p->ny * p->nz;
    P.np = 0;
    P.thermo = p->thermo_force;
    P.scheme = p->scalar_scheme;
    P.tau = p->tau;
    P.rho0 = p->rho0;
    P.A = p->A;
    P.kappa = p->kappa;
    P.Mpsi = p->M_psi;
    P.C = p->C;
    P.Mphi = p->M_phi;
    P.E = p->E;
    P.phib = p->phi_b;
    P.kd = p->k_d;
    fill_prm(P.pf, P);
    fill_prm(P.pd, P);
    h->rmax = 0.0;
    update_sides(h);
    h->red_blocks = reduction_blocks(p);

    const size_t N = (size_t)P.N;
    const size_t fb = (size_t)h->ops->fld_bytes;
    cudaError_t e = cudaSuccess;
    if (p->cuda_stream) {
        h->stream = (cudaStream_t)p->cuda_stream;
        h->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = true;
    }
    // the particle kernels' stream, at the highest priority so that its few
    // blocks are placed as soon as the fluid kernels leave room
    if (e == cudaSuccess) {
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        h->side.prio = hi;
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side.s, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.bnd_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.collide_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.scal_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side.s2, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.pt_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.links_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.mark_done, cudaEventDisableTiming);
    }
    h->region_bytes = layout(p, h->ops, h->red_blocks, nullptr, nullptr);
    if (e == cudaSuccess) {
        if (region) {
            h->region = region;
            h->batch = batch;
        } else {
            e = cudaMalloc(&h->region, h->region_bytes);
        }
    }
    if (e != cudaSuccess) {
        h->region = nullptr;
        free_all(h);
        delete h;
        cudaGetLastError();
        return cuda_status(e);
    }
    layout(p, h->ops, h->red_blocks, h, (char*)h->region);
    // rest state: rho = rho0, u = 0, psi = phi = 0, all fluid
    cudaStream_t s = h->stream;
    long long nf = P.N;
    e = cudaMemsetAsync(h->mask[0], 0, N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->mask[1], 0, N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->corr, 0, 8 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->link_ticket, 0, kMaxParticles * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->cover_ticket, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->force, 0, 3 * N * fb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->pt, 0, kPtFields * N * fb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->bflag, 0, N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->u, 0, 3 * N * fb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->mupsi, 0, N * fb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->muphi, 0, N * fb, s);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(h->psi[k], 0, N * fb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->phi[k], 0, N * fb, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->nfluid, &nf, sizeof(long long), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        // populations from rho = rho0 everywhere (staging holds rho0)
        std::vector<double> ones(N, p->rho0);
        e = cudaMemcpyAsync(h->staging, ones.data(), N * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = h->ops->set_fields(P, cur_ptrs(h), s, h->staging, nullptr, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        cudaGetLastError();
        return cuda_status(e);
    }
    *out = h;
    return LB_OK;
}

}  // namespace lbdp
