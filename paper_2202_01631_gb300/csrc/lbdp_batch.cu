// lbdp_batch.cu -- the extern "C" entry points of include/lbdp_batch.h: the
// arena that places boxes in one device allocation, batches of boxes that
// advance together through the persistent kernels of lbdp_batch_kernels.cuh
// (captured in CUDA graphs, launch shapes picked by an autotuner), and the
// continuous-batching request loop.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <vector>

#include "lbdp.h"
#include "lbdp_batch.h"
#include "lbdp_batch_kernels.cuh"
#include "lbdp_internal.h"

using namespace lbdp;

// ---------------------------------------------------------------------------
// arena: first fit over offsets, 256-byte granules, coalescing frees
// ---------------------------------------------------------------------------
struct lb_arena {
    size_t cap = 0;
    size_t used = 0;
    std::map<size_t, size_t> free_ranges;   // offset -> bytes
    std::map<size_t, size_t> held;          // offset -> bytes
};

namespace {

constexpr size_t kGranule = 256;

size_t round_up(size_t b) { return (b + kGranule - 1) / kGranule * kGranule; }

int cuda_status(cudaError_t e)
{
    return e == cudaSuccess ? LB_OK : (e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA);
}

#define LB_TRY(expr)                                   \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

const BatchOps* batch_ops_for(int prec)
{
    switch (prec) {
        case LB_FP64: return &kBatchF64;
        case LB_FP32: return &kBatchF32;
        case LB_FP16_SHIFT: return &kBatchF16;
        case LB_BF16_SHIFT: return &kBatchBF16;
        default: return nullptr;
    }
}

}  // namespace

extern "C" {

int lb_arena_create(size_t capacity, lb_arena** out)
{
    if (!out) return LB_ERR_PARAM;
    *out = nullptr;
    const size_t cap = capacity / kGranule * kGranule;
    if (cap == 0) return LB_ERR_PARAM;
    lb_arena* a = new (std::nothrow) lb_arena();
    if (!a) return LB_ERR_NOMEM;
    a->cap = cap;
    a->free_ranges[0] = cap;
    *out = a;
    return LB_OK;
}

int lb_arena_alloc(lb_arena* a, size_t bytes, size_t* offset)
{
    if (!a || !offset || bytes == 0) return LB_ERR_PARAM;
    const size_t need = round_up(bytes);
    for (auto it = a->free_ranges.begin(); it != a->free_ranges.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, have = it->second;
        a->free_ranges.erase(it);
        if (have > need) a->free_ranges[off + need] = have - need;
        a->held[off] = need;
        a->used += need;
        *offset = off;
        return LB_OK;
    }
    return LB_ERR_NOMEM;
}

int lb_arena_free(lb_arena* a, size_t offset)
{
    if (!a) return LB_ERR_PARAM;
    auto h = a->held.find(offset);
    if (h == a->held.end()) return LB_ERR_PARAM;
    size_t off = h->first, len = h->second;
    a->held.erase(h);
    a->used -= len;
    auto next = a->free_ranges.lower_bound(off);
    if (next != a->free_ranges.end() && next->first == off + len) {
        len += next->second;
        next = a->free_ranges.erase(next);
    }
    if (next != a->free_ranges.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += len;
            return LB_OK;
        }
    }
    a->free_ranges[off] = len;
    return LB_OK;
}

int lb_arena_stats(const lb_arena* a, size_t* used, size_t* largest_free, int* free_ranges)
{
    if (!a) return LB_ERR_PARAM;
    size_t big = 0;
    for (const auto& r : a->free_ranges) big = std::max(big, r.second);
    if (used) *used = a->used;
    if (largest_free) *largest_free = big;
    if (free_ranges) *free_ranges = (int)a->free_ranges.size();
    return LB_OK;
}

void lb_arena_destroy(lb_arena* a) { delete a; }

}  // extern "C"

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
namespace {

struct Member {
    lb_handle* h;
    size_t off;        // arena offset of the box's region
    long long left;    // steps still to run (host mirror of the device count)
    int cur0;          // buffer the launch plans take as current at parity 0
    int np_seen;       // particles when the plans were built
};

}  // namespace

struct lbb_batch {
    int precision = 0;
    const BatchOps* bops = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = -1;
    int sms = 0;
    char* base = nullptr;
    lb_arena* arena = nullptr;
    int graph_steps = 16;   // even
    std::vector<Member> mem;
    bool dirty = true;
    long long* d_left = nullptr;
    std::vector<LaunchPlan> plans;
    int par = 0;            // parity of the steps run since the plans were built
    int cfg[kNumBatchClasses] = {1, 1};   // z chunks of 16 planes until tuned
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // graphs starting at parity 0 / 1
    SideStream side{};   // particle kernels, overlapping the fluid kernels
};

namespace {

constexpr int kStepLaunches = 9;   // per launch plan: 2 bulk kernels, 7 particle kernels

bool cfg_valid(int cfg) { return cfg >= 0 && cfg < kNumBatchCfgs; }

int find_member(const lbb_batch* b, const lb_handle* h)
{
    for (size_t i = 0; i < b->mem.size(); ++i)
        if (b->mem[i].h == h) return (int)i;
    return -1;
}

void drop_graph(lbb_batch* b)
{
    for (auto& g : b->exec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Build the launch plans from the member list: up to kLaunchBoxes boxes per
// launch, each box's pointer sets taken from its current buffer.
void rebuild(lbb_batch* b)
{
    const int nb = (int)b->mem.size();
    b->plans.assign((nb + kLaunchBoxes - 1) / kLaunchBoxes, LaunchPlan());
    for (size_t l = 0; l < b->plans.size(); ++l) {
        LaunchPlan& pl = b->plans[l];
        memset(&pl.L, 0, sizeof(pl.L));
        pl.L.left = b->d_left;
        pl.L.base = (int)l * kLaunchBoxes;
        pl.L.nbox = std::min(kLaunchBoxes, nb - pl.L.base);
        int zmax[kNumBatchCfgs] = {1, 1, 1};
        int lmax = 1, cmax = 1, pmax = 1;
        for (int j = 0; j < pl.L.nbox; ++j) {
            Member& m = b->mem[pl.L.base + j];
            lb_handle* h = m.h;
            BoxDev& bd = pl.L.box[j];
            m.cur0 = h->cur;
            m.np_seen = h->dp.np;
            bd.P = h->dp;
            bd.D[0] = handle_ptrs(h, m.cur0);
            bd.D[1] = handle_ptrs(h, m.cur0 ^ 1);
            for (int k = 0; k < kNumBatchCfgs; ++k) zmax[k] = std::max(zmax[k], zm_blocks(h->dp, kZChunks[k]));
            lmax = std::max(lmax, h->dp.np * h->dp.nb1);
            cmax = std::max(cmax, h->dp.np * h->dp.nb2);
            pmax = std::max(pmax, h->dp.np * pt_part_blocks(h->dp));
        }
        for (int k = 0; k < kNumBatchCfgs; ++k) pl.zgrid[k] = dim3(zmax[k], pl.L.nbox);
        pl.link = dim3(lmax, pl.L.nbox);
        pl.cover = dim3(cmax, pl.L.nbox);
        pl.ptg = dim3(pmax, pl.L.nbox);
    }
    b->par = 0;
    b->dirty = false;
    drop_graph(b);
}

// The plans still describe the batch: same boxes and particles, and every box
// with steps left has run the same steps since they were built.
bool plans_stale(const lbb_batch* b)
{
    if (b->dirty) return true;
    for (const Member& m : b->mem) {
        if (m.np_seen != m.h->dp.np) return true;
        if (m.left > 0 && m.h->cur != (m.cur0 ^ b->par)) return true;
    }
    return false;
}

// Upload the steps each box still has to run (all_one: 1 for every box, used
// while tuning).
int upload_counts(lbb_batch* b, bool all_one)
{
    const int nb = (int)b->mem.size();
    if (nb == 0) return LB_OK;
    std::vector<long long> left(nb);
    for (int i = 0; i < nb; ++i) left[i] = all_one ? 1 : b->mem[i].left;
    LB_TRY(cudaMemcpyAsync(b->d_left, left.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, b->stream));
    return LB_OK;
}

int step(lbb_batch* b, int par)
{
    return cuda_status(b->bops->step(b->cfg, b->plans.data(), (int)b->plans.size(), par, b->d_left,
                                     (int)b->mem.size(), b->stream, &b->side));
}

// graph_steps steps starting at parity p0 (graph_steps is even, so a launch
// of it leaves the parity unchanged)
int capture_graph(lbb_batch* b, int p0)
{
    if (b->exec[p0]) return LB_OK;
    cudaGraph_t g = nullptr;
    LB_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int st = LB_OK;
    for (int t = 0; t < b->graph_steps && st == LB_OK; ++t) st = step(b, (p0 + t) & 1);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (st == LB_OK) st = cuda_status(e2);
    if (st == LB_OK) st = cuda_status(cudaGraphInstantiate(&b->exec[p0], g, 0));
    if (g) cudaGraphDestroy(g);
    if (st != LB_OK) {
        b->exec[p0] = nullptr;
        cudaGetLastError();
    }
    return st;
}

}  // namespace

namespace lbdp {
void batch_release(lb_handle* h)
{
    lbb_batch* b = h->batch;
    const int i = find_member(b, h);
    if (i >= 0) {
        lb_arena_free(b->arena, b->mem[i].off);
        b->mem.erase(b->mem.begin() + i);
    }
    b->dirty = true;
}
}  // namespace lbdp

extern "C" {

int lbb_create(const lbb_params* p, lbb_batch** out)
{
    if (!out) return LB_ERR_PARAM;
    *out = nullptr;
    if (!p || !batch_ops_for(p->precision) || p->graph_steps < 0) return LB_ERR_PARAM;
    lbb_batch* b = new (std::nothrow) lbb_batch();
    if (!b) return LB_ERR_NOMEM;
    b->precision = p->precision;
    b->bops = batch_ops_for(p->precision);
    b->graph_steps = p->graph_steps > 0 ? p->graph_steps : 16;
    b->graph_steps += b->graph_steps & 1;   // even: parity returns after a graph
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) {
        if (p->cuda_stream) {
            b->stream = (cudaStream_t)p->cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) {
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        b->side.prio = hi;
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side.s, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.bnd_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.collide_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.scal_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side.s2, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.pt_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.links_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.mark_done, cudaEventDisableTiming);
    }
    size_t cap = p->arena_bytes;
    if (e == cudaSuccess && cap == 0) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        cap = fr / 4 * 3;
    }
    cap = cap / kGranule * kGranule;
    if (e == cudaSuccess && lb_arena_create(cap, &b->arena) != LB_OK) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->base, cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_left, kBatchMaxBoxes * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_left, 0, kBatchMaxBoxes * sizeof(long long), b->stream);
    if (e == cudaSuccess) e = b->bops->prepare();
    int st = cuda_status(e);
    if (st == LB_OK) st = cuda_status(cudaStreamSynchronize(b->stream));
    if (st != LB_OK) {
        cudaGetLastError();
        lbb_destroy(b);
        return st;
    }
    *out = b;
    return LB_OK;
}

void lbb_destroy(lbb_batch* b)
{
    if (!b) return;
    if (b->device >= 0) cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    std::vector<Member> ms = b->mem;
    for (const Member& m : ms) lb_destroy(m.h);
    drop_graph(b);
    if (b->d_left) cudaFree(b->d_left);
    if (b->base) cudaFree(b->base);
    if (b->arena) lb_arena_destroy(b->arena);
    if (b->side.s) {
        cudaStreamSynchronize(b->side.s);
        cudaStreamDestroy(b->side.s);
    }
    if (b->side.fork) cudaEventDestroy(b->side.fork);
    if (b->side.bnd_done) cudaEventDestroy(b->side.bnd_done);
    if (b->side.collide_done) cudaEventDestroy(b->side.collide_done);
    if (b->side.scal_done) cudaEventDestroy(b->side.scal_done);
    if (b->side.s2) {
        cudaStreamSynchronize(b->side.s2);
        cudaStreamDestroy(b->side.s2);
    }
    if (b->side.pt_done) cudaEventDestroy(b->side.pt_done);
    if (b->side.links_done) cudaEventDestroy(b->side.links_done);
    if (b->side.mark_done) cudaEventDestroy(b->side.mark_done);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

static int check_box(const lbb_batch* b, const lb_params* p)
{
    if (!b || !p) return LB_ERR_PARAM;
    size_t bytes = 0;
    if (lb_device_bytes(p, &bytes) != LB_OK) return LB_ERR_PARAM;
    if (p->precision != b->precision) return LB_ERR_PARAM;
    if (p->nx > kBatchMaxEdgeXY || p->ny > kBatchMaxEdgeXY) return LB_ERR_PARAM;
    if ((long long)p->nx * p->ny * p->nz >= kBatchMaxNodes) return LB_ERR_PARAM;
    return LB_OK;
}

int lbb_box_bytes(const lbb_batch* b, const lb_params* p, size_t* bytes)
{
    if (!bytes) return LB_ERR_PARAM;
    const int st = check_box(b, p);
    if (st != LB_OK) return st;
    *bytes = round_up(handle_region_bytes(p));
    return LB_OK;
}

int lbb_memory(const lbb_batch* b, size_t* capacity, size_t* used, size_t* largest_free)
{
    if (!b) return LB_ERR_PARAM;
    if (capacity) *capacity = b->arena->cap;
    return lb_arena_stats(b->arena, used, largest_free, nullptr);
}

int lbb_add_box(lbb_batch* b, const lb_params* p, lb_handle** out)
{
    if (!out) return LB_ERR_PARAM;
    *out = nullptr;
    int st = check_box(b, p);
    if (st != LB_OK) return st;
    if ((int)b->mem.size() >= kBatchMaxBoxes) return LB_ERR_NOMEM;
    cudaSetDevice(b->device);
    size_t off = 0;
    st = lb_arena_alloc(b->arena, handle_region_bytes(p), &off);
    if (st != LB_OK) return st;
    lb_params q = *p;
    q.cuda_stream = (void*)b->stream;
    lb_handle* h = nullptr;
    st = lb_create_in(&q, b, b->base + off, &h);
    if (st != LB_OK) {
        lb_arena_free(b->arena, off);
        return st;
    }
    b->mem.push_back({h, off, 0, 0, 0});
    b->dirty = true;
    *out = h;
    return LB_OK;
}

int lbb_num_boxes(const lbb_batch* b) { return b ? (int)b->mem.size() : 0; }

int lbb_set_steps(lbb_batch* b, lb_handle* h, long long nsteps)
{
    if (!b || !h || nsteps < 0) return LB_ERR_PARAM;
    const int i = find_member(b, h);
    if (i < 0) return LB_ERR_PARAM;
    b->mem[i].left = nsteps;
    return LB_OK;
}

int lbb_get_steps(const lbb_batch* b, const lb_handle* h, long long* left)
{
    if (!b || !h || !left) return LB_ERR_PARAM;
    const int i = find_member(b, h);
    if (i < 0) return LB_ERR_PARAM;
    *left = b->mem[i].left;
    return LB_OK;
}

int lbb_run(lbb_batch* b, int nsteps, long long* launches)
{
    if (launches) *launches = 0;
    if (!b || nsteps < 0) return LB_ERR_PARAM;
    cudaSetDevice(b->device);
    long long most = 0;
    for (const Member& m : b->mem) most = std::max(most, m.left);
    const int n = (int)std::min<long long>(nsteps, most);
    if (n == 0) return LB_OK;
    if (plans_stale(b)) rebuild(b);
    int st = upload_counts(b, false);
    if (st != LB_OK) return st;
    const int full = n / b->graph_steps, rest = n % b->graph_steps;
    if (full > 0) {
        st = capture_graph(b, b->par);
        if (st != LB_OK) return st;
        for (int k = 0; k < full; ++k) LB_TRY(cudaGraphLaunch(b->exec[b->par], b->stream));
    }
    for (int k = 0; k < rest && st == LB_OK; ++k) st = step(b, (b->par + k) & 1);
    if (st != LB_OK) return st;
    b->par = (b->par + n) & 1;
    for (Member& m : b->mem) {
        const long long ran = std::min<long long>(m.left, n);
        m.left -= ran;
        m.h->cur ^= (int)(ran & 1);
    }
    if (launches) *launches = (long long)n * ((long long)b->plans.size() * kStepLaunches + 1);
    return LB_OK;
}

int lbb_num_configs(void) { return kNumBatchCfgs; }

int lbb_config_shape(int k, int* threads, int* planes)
{
    if (k < 0 || k >= kNumBatchCfgs) return LB_ERR_PARAM;
    if (threads) *threads = kZThreads;
    if (planes) *planes = kZChunks[k];
    return LB_OK;
}

int lbb_set_config(lbb_batch* b, const int cfg[LBB_KERNEL_CLASSES])
{
    if (!b || !cfg) return LB_ERR_PARAM;
    for (int k = 0; k < kNumBatchClasses; ++k)
        if (!cfg_valid(cfg[k])) return LB_ERR_PARAM;
    cudaSetDevice(b->device);
    for (int k = 0; k < kNumBatchClasses; ++k) b->cfg[k] = cfg[k];
    drop_graph(b);
    return LB_OK;
}

int lbb_tune(lbb_batch* b, int reps, int cfg_out[LBB_KERNEL_CLASSES], double ms_out[LBB_KERNEL_CLASSES])
{
    if (!b || reps < 1) return LB_ERR_PARAM;
    if (b->mem.empty()) return LB_ERR_STATE;
    cudaSetDevice(b->device);
    cudaStream_t s = b->stream;
    if (plans_stale(b)) rebuild(b);
    // the fused kernel rewrites the stored velocity: keep a copy in staging
    for (const Member& m : b->mem) {
        const size_t ub = 3 * (size_t)m.h->dp.N * m.h->ops->fld_bytes;
        LB_TRY(cudaMemcpyAsync(m.h->staging, m.h->u, ub, cudaMemcpyDeviceToDevice, s));
    }
    int st = upload_counts(b, true);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == LB_OK) st = cuda_status(cudaEventCreate(&e0));
    if (st == LB_OK) st = cuda_status(cudaEventCreate(&e1));
    int best[kNumBatchClasses] = {0, 0};
    double best_ms[kNumBatchClasses] = {0, 0};
    for (int nc = 0; nc < kNumBatchClasses && st == LB_OK; ++nc) {
        best_ms[nc] = 1e300;
        for (int k = 0; k < kNumBatchCfgs && st == LB_OK; ++k) {
            auto all = [&]() {
                for (LaunchPlan& pl : b->plans) {
                    pl.L.par = b->par;
                    const int e = cuda_status(b->bops->node(nc, k, &pl, s));
                    if (e != LB_OK) return e;
                }
                return (int)LB_OK;
            };
            for (int w = 0; w < 2 && st == LB_OK; ++w) st = all();
            if (st == LB_OK) st = cuda_status(cudaEventRecord(e0, s));
            for (int r = 0; r < reps && st == LB_OK; ++r) st = all();
            if (st == LB_OK) st = cuda_status(cudaEventRecord(e1, s));
            if (st == LB_OK) st = cuda_status(cudaEventSynchronize(e1));
            float ms = 0.f;
            if (st == LB_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
            if (st == LB_OK && ms / reps < best_ms[nc]) {
                best_ms[nc] = ms / reps;
                best[nc] = k;
            }
        }
    }
    for (const Member& m : b->mem) {
        const size_t ub = 3 * (size_t)m.h->dp.N * m.h->ops->fld_bytes;
        cudaError_t e = cudaMemcpyAsync(m.h->u, m.h->staging, ub, cudaMemcpyDeviceToDevice, s);
        if (st == LB_OK) st = cuda_status(e);
    }
    if (st == LB_OK) st = upload_counts(b, false);
    if (st == LB_OK) st = cuda_status(cudaStreamSynchronize(s));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != LB_OK) return st;
    for (int k = 0; k < kNumBatchClasses; ++k) {
        b->cfg[k] = best[k];
        if (cfg_out) cfg_out[k] = best[k];
        if (ms_out) ms_out[k] = best_ms[k];
    }
    drop_graph(b);
    return LB_OK;
}

int lbb_sync(lbb_batch* b)
{
    if (!b) return LB_ERR_PARAM;
    cudaSetDevice(b->device);
    LB_TRY(cudaStreamSynchronize(b->stream));
    int worst = LB_OK;
    for (const Member& m : b->mem) {
        const int st = lb_sync(m.h);
        if (st != LB_OK && worst == LB_OK) worst = st;
    }
    return worst;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// continuous batching
// ---------------------------------------------------------------------------
namespace {

struct Pending {
    long long id;
    lbs_request r;
    std::vector<double> psi, phi;
};

struct Live {
    Pending q;
    lb_handle* h;
    double admitted;
};

}  // namespace

struct lbs_server {
    lbb_batch* batch = nullptr;
    int precision = 0;
    int chunk = 64;
    int max_boxes = 0;
    long long next_id = 0;
    std::deque<Pending> queue;
    std::vector<Live> live;
    std::deque<lbs_result> done;
};

namespace {

void finish(lbs_server* s, Live& L, int status, double t_done)
{
    lbs_result res;
    memset(&res, 0, sizeof(res));
    res.id = L.q.id;
    res.arrival = L.q.r.arrival;
    res.admitted = L.admitted;
    res.status = status;
    if (L.h && status == LB_ERR_CANCELLED) {
        lb_destroy(L.h);   // results of a cancelled request are not read
        L.h = nullptr;
    }
    if (L.h) {
        int n = 0;
        int st = lb_read_particles(L.h, res.particles, 4, &n);
        res.n_particles = n < 4 ? n : 4;
        if (st == LB_OK) st = lb_conservation(L.h, res.sums);
        if (st == LB_OK && (L.q.r.out_psi || L.q.r.out_phi))
            st = lb_read_fields(L.h, nullptr, nullptr, L.q.r.out_psi, L.q.r.out_phi);
        if (res.status == LB_OK) res.status = st;
        lb_destroy(L.h);
        L.h = nullptr;
    }
    res.done = t_done;
    s->done.push_back(res);
}

}  // namespace

extern "C" {

int lbs_create(const lbs_params* p, lbs_server** out)
{
    if (!out) return LB_ERR_PARAM;
    *out = nullptr;
    if (!p || p->chunk_steps < 0 || p->max_boxes < 0) return LB_ERR_PARAM;
    lbs_server* s = new (std::nothrow) lbs_server();
    if (!s) return LB_ERR_NOMEM;
    lbb_params bp;
    memset(&bp, 0, sizeof(bp));
    bp.precision = p->precision;
    bp.arena_bytes = p->arena_bytes;
    bp.cuda_stream = p->cuda_stream;
    const int st = lbb_create(&bp, &s->batch);
    if (st != LB_OK) {
        delete s;
        return st;
    }
    s->precision = p->precision;
    s->chunk = p->chunk_steps > 0 ? p->chunk_steps : 64;
    s->max_boxes = p->max_boxes;
    *out = s;
    return LB_OK;
}

void lbs_destroy(lbs_server* s)
{
    if (!s) return;
    lbb_destroy(s->batch);   // destroys the live boxes
    delete s;
}

lbb_batch* lbs_batch(lbs_server* s) { return s ? s->batch : nullptr; }

int lbs_submit(lbs_server* s, const lbs_request* r, long long* id)
{
    if (!s || !r || r->steps <= 0 || r->n_particles < 0 || r->n_particles > 4) return LB_ERR_PARAM;
    size_t bytes = 0, cap = 0;
    int st = lbb_box_bytes(s->batch, &r->box, &bytes);
    if (st != LB_OK) return st;
    lbb_memory(s->batch, &cap, nullptr, nullptr);
    if (bytes > cap) return LB_ERR_PARAM;   // can never be admitted
    Pending q;
    q.id = s->next_id++;
    q.r = *r;
    const size_t N = (size_t)r->box.nx * r->box.ny * r->box.nz;
    if (r->psi) q.psi.assign(r->psi, r->psi + N);
    if (r->phi) q.phi.assign(r->phi, r->phi + N);
    q.r.psi = nullptr;
    q.r.phi = nullptr;
    s->queue.push_back(std::move(q));
    if (id) *id = s->queue.back().id;
    return LB_OK;
}

int lbs_pump(lbs_server* s, double now, int* active, int* queued)
{
    if (!s) return LB_ERR_PARAM;
    const auto t0 = std::chrono::steady_clock::now();
    auto clock = [&]() {
        return now + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    // admission, in arrival order; a request that does not fit is passed over
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        if (s->max_boxes > 0 && (int)s->live.size() >= s->max_boxes) break;
        size_t bytes = 0, largest = 0;
        lbb_box_bytes(s->batch, &it->r.box, &bytes);
        lbb_memory(s->batch, nullptr, nullptr, &largest);
        if (bytes > largest) {
            ++it;
            continue;
        }
        Live L;
        L.h = nullptr;
        int st = lbb_add_box(s->batch, &it->r.box, &L.h);
        if (st == LB_ERR_NOMEM) {
            ++it;
            continue;
        }
        L.q = std::move(*it);
        it = s->queue.erase(it);
        L.admitted = clock();
        if (st == LB_OK && (!L.q.psi.empty() || !L.q.phi.empty()))
            st = lb_set_fields(L.h, nullptr, nullptr, L.q.psi.empty() ? nullptr : L.q.psi.data(),
                               L.q.phi.empty() ? nullptr : L.q.phi.data());
        for (int k = 0; k < L.q.r.n_particles && st == LB_OK; ++k)
            st = lb_add_particle(L.h, &L.q.r.particles[k], nullptr);
        if (st == LB_OK) st = lbb_set_steps(s->batch, L.h, L.q.r.steps);
        L.q.psi.clear();
        L.q.psi.shrink_to_fit();
        L.q.phi.clear();
        L.q.phi.shrink_to_fit();
        if (st != LB_OK) {
            finish(s, L, st, clock());
            continue;
        }
        s->live.push_back(std::move(L));
    }
    // run until the first resident box finishes, at most one chunk
    long long n = s->chunk;
    for (const Live& L : s->live) {
        long long left = 0;
        lbb_get_steps(s->batch, L.h, &left);
        if (left > 0) n = std::min(n, left);
    }
    int st = LB_OK;
    if (!s->live.empty()) {
        st = lbb_run(s->batch, (int)n, nullptr);
        if (st == LB_OK) {
            cudaError_t e = cudaStreamSynchronize(s->live.front().h->stream);
            if (e != cudaSuccess) st = LB_ERR_CUDA;
        }
    }
    // retire the boxes that have run all their steps
    for (size_t i = 0; i < s->live.size();) {
        long long left = 0;
        lbb_get_steps(s->batch, s->live[i].h, &left);
        if (left > 0 && st == LB_OK) {
            ++i;
            continue;
        }
        finish(s, s->live[i], st, clock());
        s->live.erase(s->live.begin() + i);
    }
    if (active) *active = (int)s->live.size();
    if (queued) *queued = (int)s->queue.size();
    return st;
}

int lbs_cancel(lbs_server* s, long long id, double now)
{
    if (!s) return LB_ERR_PARAM;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if (it->id != id) continue;
        Live L;
        L.q = std::move(*it);
        L.h = nullptr;
        L.admitted = -1.0;   // never admitted
        s->queue.erase(it);
        finish(s, L, LB_ERR_CANCELLED, now);
        return LB_OK;
    }
    for (size_t i = 0; i < s->live.size(); ++i) {
        if (s->live[i].q.id != id) continue;
        // between pumps nothing of the batch is in flight (lbs_pump ends with
        // a stream synchronisation), so the box can leave at once
        finish(s, s->live[i], LB_ERR_CANCELLED, now);
        s->live.erase(s->live.begin() + i);
        return LB_OK;
    }
    return LB_ERR_PARAM;
}

int lbs_poll(lbs_server* s, lbs_result* out, int cap, int* n)
{
    if (!s || cap < 0 || (cap > 0 && !out)) return LB_ERR_PARAM;
    int k = 0;
    while (k < cap && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    if (n) *n = k;
    return LB_OK;
}

}  // extern "C"
