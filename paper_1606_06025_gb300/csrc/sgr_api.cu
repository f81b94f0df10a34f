// sgr_api.cu -- the C ABI of libsgrcolor (declared in include/sgrcolor.h).
//
// Host side of the coloring call: argument checks, the per-device scratch
// arena, the cooperative launch of the persistent coloring kernel, and the
// single read-back of counters and statistics.  The CPU only controls
// progress here, as in the paper's design (Sect. 3.1); all coloring work runs
// in the kernels of sgr_kernels.cu.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "sgr_internal.cuh"
#include "sgrcolor.h"

namespace {

using sgr::Counters;
using sgr::Params;

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Limit of the bounded device-side waits (0: kWaitTimeoutNs) and the host-side
// fault injection of sgr_debug_inject.
std::atomic<unsigned long long> g_wait_ns{0};
std::atomic<long long> g_inject_alloc{0};  // the k-th next device allocation fails (0: none)
std::atomic<int> g_inject_barrier{0};      // coloring launches whose barriers wait for one CTA more

// A device buffer that only grows (freed by sgr_release_scratch).
struct Arena {
    char *ptr = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (ptr) {
            cudaError_t e = cudaFree(ptr);
            ptr = nullptr;
            cap = 0;
            if (e != cudaSuccess) return e;
        }
        if (sgr::inject_alloc_failure()) return cudaErrorMemoryAllocation;
        size_t want = std::max(bytes, cap + cap / 4);
        cudaError_t e = cudaMalloc(&ptr, want);
        if (e != cudaSuccess) {
            ptr = nullptr;
            e = cudaMalloc(&ptr, bytes);
            if (e != cudaSuccess) {
                ptr = nullptr;
                return e;
            }
            want = bytes;
        }
        cap = want;
        return cudaSuccess;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
    }
};

struct DevCtx {
    int device = -1;
    int sms = 0;
    int occ[2][2] = {{0, 0}, {0, 0}};  // [fast][batched]
    int occ_front[2] = {0, 0};          // activation-list kernel, [batched]
    Arena scratch;                      // worklists, counters, bitmaps
    Arena io;                           // device copies for the host-buffer entry
    Counters *host_ctr = nullptr;       // pinned read-back
    int64_t *host_small = nullptr;      // pinned staging (offsets, flags)
    size_t host_small_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const long long *last_trace = nullptr;  // device timeline of the last launch
    long long last_rounds = 0;
    long long last_t_init = 0;
    std::mutex mu;
    bool ready = false;
};

std::mutex g_ctx_mu;
std::vector<DevCtx *> g_ctx;

std::mutex g_tune_mu;
sgr_tuning g_tune = {32, 1024, 0, 0, 0};

thread_local sgr_stats t_stats;

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return SGR_OK;
    if (e == cudaErrorMemoryAllocation) return SGR_ERR_OUT_OF_MEMORY;
    return SGR_ERR_CUDA;
}

int get_ctx(DevCtx **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return SGR_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    if ((int)g_ctx.size() <= dev) g_ctx.resize(dev + 1, nullptr);
    if (!g_ctx[dev]) g_ctx[dev] = new DevCtx();
    DevCtx *c = g_ctx[dev];
    if (!c->ready) {
        c->device = dev;
        if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SGR_ERR_CUDA;
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (!coop) return SGR_ERR_CUDA;
        for (int f = 0; f < 2; ++f)
            for (int b = 0; b < 2; ++b)
                if (sgr::occupancy_blocks_per_sm(f != 0, b != 0, &c->occ[f][b]) != 0)
                    return SGR_ERR_CUDA;
        for (int b = 0; b < 2; ++b)
            if (sgr::occupancy_blocks_per_sm_front(b != 0, &c->occ_front[b]) != 0) return SGR_ERR_CUDA;
        if (cudaMallocHost(&c->host_ctr, sizeof(Counters)) != cudaSuccess) return SGR_ERR_OUT_OF_MEMORY;
        if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)
            return SGR_ERR_CUDA;
        c->ready = true;
    }
    *out = c;
    return SGR_OK;
}

// The context record of a device, without the CUDA set-up get_ctx does.
DevCtx *ctx_struct(int device) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    if ((int)g_ctx.size() <= device) g_ctx.resize(device + 1, nullptr);
    if (!g_ctx[device]) g_ctx[device] = new DevCtx();
    return g_ctx[device];
}

int ensure_host_small(DevCtx *c, size_t count) {
    if (count <= c->host_small_cap) return SGR_OK;
    if (c->host_small) cudaFreeHost(c->host_small);
    c->host_small = nullptr;
    c->host_small_cap = 0;
    size_t want = std::max<size_t>(count, 1024);
    if (cudaMallocHost(&c->host_small, want * sizeof(int64_t)) != cudaSuccess) return SGR_ERR_OUT_OF_MEMORY;
    c->host_small_cap = want;
    return SGR_OK;
}

// topo: the entry point also takes SGR_MODE_TOPO (single graphs only).
bool valid_mode(int mode, bool topo = false) {
    if (mode & ~(SGR_MODE_MASK | SGR_RULE_MASK)) return false;
    const int md = mode & SGR_MODE_MASK, rule = (mode & SGR_RULE_MASK) >> 4;
    return (md == SGR_MODE_DETERMINISTIC || md == SGR_MODE_FAST || (topo && md == SGR_MODE_TOPO)) && rule <= 2;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

sgr_tuning current_tuning() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

// Everything a coloring launch needs beyond the CSR itself.
struct Job {
    bool fast;
    int32_t n;
    long long m;
    const int32_t *ro;
    const int32_t *ci;
    int32_t *colors;
    bool batched;
    int G;
    const long long *vbase_dev;
    const long long *ebase_dev;
    const long long *robase_dev;
    int32_t *gid_dev;  // filled by the caller for batched jobs
    bool front;        // det: allocate the activation lists (rounds may run on them)
    bool tail;         // det: allocate the tail arrays (the last rounds may run in one CTA)
};

// |W_r| at or below which the rounds move to the tail CTA (0: never).
int tail_vertices(const sgr_tuning &t) {
    if (t.tail_vertices < 0) return 0;
    return t.tail_vertices == 0 ? sgr::kTailDefault : std::min(t.tail_vertices, sgr::kTailMax);
}

// Carve the scratch arena for a job.  Returns the byte size; fills p when
// base != nullptr.
size_t layout(const Job &j, const sgr_tuning &t, char *base, Params *p, size_t *zero_bytes) {
    const sgr::ScratchPlan sp = sgr::plan_scratch(j.n, j.m, t.chunk);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return base ? (void *)(base + o) : nullptr;
    };
    // zeroed region first: counters, hub completion counters / flags, hub bitmaps
    Counters *ctr = (Counters *)take(sizeof(Counters));
    unsigned long long *hdone = (unsigned long long *)take(sp.hub_max * 8);
    unsigned *hconf = (unsigned *)take(sp.hub_max * 4);
    unsigned *hbits = (unsigned *)take(sp.hub_words * 4);
    const size_t zero_fast = off;
    const long long np = ((long long)j.n + 63) / 64 * 64;
    unsigned *bm = (unsigned *)take((size_t)np * 8 * 4);
    const bool front = !j.fast && j.front;
    int32_t *astamp = front ? (int32_t *)take((size_t)j.n * 4) : nullptr;
    if (zero_bytes) *zero_bytes = j.fast ? zero_fast : off;
    int32_t *lowdeg = (int32_t *)take((size_t)j.n * 4);
    int32_t *witness = (int32_t *)take((size_t)j.n * 4);
    int32_t *wold = (int32_t *)take(j.fast ? 16 : (size_t)j.n * 16);
    int32_t *sw = (int32_t *)take(sp.hub_max * 4);
    unsigned *scb = (unsigned *)take(sp.hub_max * 4);
    long long *trace = (long long *)take(sizeof(long long) * sgr::kTraceCap * sgr::kTraceFields);
    int32_t *lw0 = (int32_t *)take((size_t)j.n * 4), *lw1 = (int32_t *)take((size_t)j.n * 4);
    int32_t *mw0 = (int32_t *)take((size_t)j.n * 4), *mw1 = (int32_t *)take((size_t)j.n * 4);
    int32_t *hw0 = (int32_t *)take(sp.hub_max * 4), *hw1 = (int32_t *)take(sp.hub_max * 4);
    unsigned *hcb0 = (unsigned *)take(sp.hub_max * 4), *hcb1 = (unsigned *)take(sp.hub_max * 4);
    int32_t *hvert = (int32_t *)take(sp.hub_max * 4);
    unsigned *hbase = (unsigned *)take(sp.hub_max * 4);
    const size_t un = j.fast ? 1 : (size_t)j.n, uhub = j.fast ? 1 : sp.hub_max;
    int32_t *ul0 = (int32_t *)take(un * 4), *ul1 = (int32_t *)take(un * 4);
    int32_t *um0 = (int32_t *)take(un * 4), *um1 = (int32_t *)take(un * 4);
    int32_t *uh0 = (int32_t *)take(uhub * 4), *uh1 = (int32_t *)take(uhub * 4);
    // item -> hub entry map of the unsettled hubs' lower-part work items
    const size_t uitems = j.fast ? 1 : (size_t)(j.m / t.chunk) + sp.hub_max + 1;
    unsigned *ui0 = (unsigned *)take(uitems * 4), *ui1 = (unsigned *)take(uitems * 4);
    unsigned *ur0 = (unsigned *)take(uitems * 32), *ur1 = (unsigned *)take(uitems * 32);
    int32_t *uv0 = (int32_t *)take(uhub * 4), *uv1 = (int32_t *)take(uhub * 4);
    unsigned *ucb0 = (unsigned *)take(uhub * 4), *ucb1 = (unsigned *)take(uhub * 4);
    const size_t an = front ? (size_t)j.n : 1, ahub = front ? sp.hub_max : 1;
    int32_t *vslot = (int32_t *)take(j.fast ? 4 : (size_t)j.n * 4);
    int32_t *al0 = (int32_t *)take(an * 4), *al1 = (int32_t *)take(an * 4);
    int32_t *am0 = (int32_t *)take(an * 4), *am1 = (int32_t *)take(an * 4);
    int32_t *ah0 = (int32_t *)take(ahub * 4), *ah1 = (int32_t *)take(ahub * 4);
    unsigned *acb0 = (unsigned *)take(ahub * 4), *acb1 = (unsigned *)take(ahub * 4);
    const int tmax = (!j.fast && j.tail) ? tail_vertices(t) : 0;
    const long long tcap = tmax ? std::min<long long>(j.m + 8ll * tmax, sgr::kTailCapEntries) : 0;
    int32_t *tlist = tmax ? (int32_t *)take((size_t)tmax * 4) : nullptr;
    unsigned *toff = tmax ? (unsigned *)take((size_t)(tmax + 1) * 4) : nullptr;
    unsigned *tcnt = tmax ? (unsigned *)take((size_t)tmax * 4) : nullptr;
    unsigned *tlow = tmax ? (unsigned *)take((size_t)tmax * 4) : nullptr;
    unsigned *tdeg = tmax ? (unsigned *)take((size_t)tmax * 4) : nullptr;
    unsigned *tcp = tmax ? (unsigned *)take((size_t)(tmax + 1) * 4) : nullptr;
    const long long tch = tmax ? tcap / sgr::kTailChunk + tmax + 1 : 0;  // chunks of the row passes
    unsigned *tcc = tmax ? (unsigned *)take((size_t)tch * 4) : nullptr;
    unsigned *tcm = tmax ? (unsigned *)take((size_t)tch * 4) : nullptr;
    unsigned short *tstage = tmax ? (unsigned short *)take((size_t)tch * sgr::kTailChunk * 2) : nullptr;
    int32_t *tloc = tmax ? (int32_t *)take((size_t)j.n * 4) : nullptr;
    unsigned short *tadj = tmax ? (unsigned short *)take((size_t)tcap * 2 + 16) : nullptr;
    const int tmw = sgr::tail_mask_words(tmax);
    unsigned *twin = (tmax && tmax <= sgr::kTailMaskMax) ? (unsigned *)take((size_t)tmax * tmw * 4) : nullptr;
    if (p && base) {
        std::memset(p, 0, sizeof(*p));
        p->ro = j.ro;
        p->ci = j.ci;
        p->gid = j.gid_dev;
        p->vbase = j.vbase_dev;
        p->ebase = j.ebase_dev;
        p->robase = j.robase_dev;
        p->m = j.m;
        p->n = j.n;
        p->colors = j.colors;
        p->lw[0] = lw0; p->lw[1] = lw1;
        p->mw[0] = mw0; p->mw[1] = mw1;
        p->hw[0] = hw0; p->hw[1] = hw1;
        p->hcb[0] = hcb0; p->hcb[1] = hcb1;
        p->ul[0] = ul0; p->ul[1] = ul1;
        p->um[0] = um0; p->um[1] = um1;
        p->uh[0] = uh0; p->uh[1] = uh1;
        if (!j.fast) {
            p->uitem[0] = ui0; p->uitem[1] = ui1;
            p->uvert[0] = uv0; p->uvert[1] = uv1;
            p->urec[0] = ur0; p->urec[1] = ur1;
        }
        p->ucb[0] = ucb0; p->ucb[1] = ucb1;
        p->al[0] = al0; p->al[1] = al1;
        p->am[0] = am0; p->am[1] = am1;
        p->ah[0] = ah0; p->ah[1] = ah1;
        p->acb[0] = acb0; p->acb[1] = acb1;
        p->astamp = astamp;
        p->vslot = vslot;
        p->front_ok = front ? 1 : 0;
        p->front_policy = t.active_lists;
        p->hvert = hvert;
        p->hbase = hbase;
        p->hbits = hbits;
        p->hdone = hdone;
        p->hconf = hconf;
        p->bm = bm;
        p->np = np;
        p->lowdeg = lowdeg;
        p->witness = witness;
        p->wold = wold;
        p->sw = sw;
        p->scb = scb;
        p->ctr = ctr;
        p->trace = trace;
        p->light_max = t.light_max;
        p->chunk = t.chunk;
        p->tail_max = tmax;
        p->tail_cap = tcap;
        p->tlist = tlist;
        p->toff = toff;
        p->tcnt = tcnt;
        p->tlow = tlow;
        p->tdeg = tdeg;
        p->tcp = tcp;
        p->tcc = tcc;
        p->tcm = tcm;
        p->tail_chunks = (int)tch;
        p->tstage = tstage;
        p->tloc = tloc;
        p->tadj = tadj;
        p->twin = twin;
        p->tail_mw = twin ? tmw : 0;
    }
    return off;
}

void fill_stats(const Counters &h, float ms, int grid, int colors) {
    sgr_stats s;
    std::memset(&s, 0, sizeof(s));
    s.rounds = h.rounds;
    s.sum_w = (int64_t)h.sum_w;
    s.sum_d = (int64_t)h.sum_d;
    s.sum_dscan = (int64_t)h.sum_dscan;
    s.sum_next = (int64_t)h.sum_next;
    s.sum_scatter = (int64_t)h.sum_scatter;
    s.sum_rescan = (int64_t)h.sum_rescan;
    s.num_colors = colors;
    s.rows_sorted = h.unsorted_pairs == h.boundary_pairs ? 1 : 0;
    s.grid_blocks = grid;
    s.block_threads = sgr::kBlock;
    s.device_ms = ms;
    s.tail_rounds = h.tail_rounds;
    s.sum_touch = (int64_t)h.sum_touch;
    s.sum_dep = (int64_t)h.sum_dep;
    s.tail_entries = (int64_t)h.tail_entries;
    s.tail_build = (int64_t)h.tail_build;
    t_stats = s;
}

// The coloring launches of a job: the round loop over whole worklists, which
// also runs init; in deterministic mode with activation lists it may hand the
// rounds over after init (Counters::handoff) to the activation-list kernel,
// which is therefore always launched behind it (and returns at once if not
// needed).  Each launch gets its own grid and a fresh barrier counter.  Either
// grid kernel may hand the last rounds to the one-CTA tail kernel
// (Counters::tail), launched behind them when the job has the tail arrays.
cudaError_t launch_rounds(Params p, bool fast, bool batched, int per_sm_full, int per_sm_front,
                          int sms, const sgr_tuning &t, cudaStream_t st, int *grid_out) {
    int per_sm = per_sm_full;
    if (t.blocks_per_sm > 0) per_sm = std::min(per_sm, t.blocks_per_sm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * sms;
    p.nblocks = (unsigned)grid + sgr::inject_barrier_extra();  // > grid only under fault injection
    p.wait_ns = sgr::wait_limit_ns();
    *grid_out = grid;
    cudaError_t e = sgr::launch_color(p, fast, batched, grid, st);
    if (e != cudaSuccess || fast) return e;
    if (p.front_ok && p.front_policy != 1) {
        int per_sm_f = per_sm_front;
        if (t.blocks_per_sm > 0) per_sm_f = std::min(per_sm_f, t.blocks_per_sm);
        if (per_sm_f < 1) return cudaErrorInvalidConfiguration;
        p.nblocks = (unsigned)(per_sm_f * sms);
        if ((e = cudaMemsetAsync(&p.ctr->bar, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        // (a barrier that timed out in the first launch raised the error flag,
        // which this reset clears: the kernel returns at once, since init did
        // not hand the rounds over)
        if ((e = sgr::launch_color_front(p, batched, (int)p.nblocks, st)) != cudaSuccess) return e;
    }
    if (p.tail_max > 0) return sgr::launch_color_tail(p, batched, st);
    return cudaSuccess;
}

// The topology-driven schedule (Algorithm 6) for a single graph: a FirstFit
// pass and a ConflictResolve pass over all vertices per iteration, relaunched
// by this host loop while an iteration found a vertex to color (one flag read
// back per iteration, as in the paper's baseline).  Caller holds the device
// mutex.
int run_topo(DevCtx *c, const Job &j, int rule, cudaStream_t st, int32_t *k_out) {
    static_assert(sizeof(sgr::TopoCounters) <= 4 * sizeof(int64_t), "read back through host_small");
    int rc = ensure_host_small(c, 4);
    if (rc != SGR_OK) return rc;
    cudaError_t e = c->scratch.ensure(align_up(sizeof(sgr::TopoCounters)));
    if (e != cudaSuccess) return map_cuda(e);
    sgr::TopoCounters *tc = (sgr::TopoCounters *)c->scratch.ptr;
    int grid = 0;
    if (sgr::topo_grid(&grid) != 0) return SGR_ERR_CUDA;
    unsigned *flag = (unsigned *)c->host_small;  // pinned
    if ((e = cudaMemsetAsync(tc, 0, sizeof(*tc), st)) != cudaSuccess) return map_cuda(e);
    if ((e = cudaMemsetAsync(j.colors, 0, (size_t)j.n * 4, st)) != cudaSuccess) return map_cuda(e);
    if ((e = cudaEventRecord(c->ev0, st)) != cudaSuccess) return map_cuda(e);
    long long rounds = 0;
    for (;;) {
        if ((e = cudaMemsetAsync(&tc->changed, 0, sizeof(unsigned), st)) != cudaSuccess) return map_cuda(e);
        if ((e = sgr::launch_topo_iteration(j.ro, j.ci, j.colors, j.n, rule, tc, grid, st)) != cudaSuccess)
            return map_cuda(e);
        if ((e = cudaMemcpyAsync(flag, &tc->changed, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return map_cuda(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
        if (*flag == 0) break;
        if (++rounds > (long long)j.n + 1) return SGR_ERR_NO_CONVERGENCE;
    }
    if ((e = cudaEventRecord(c->ev1, st)) != cudaSuccess) return map_cuda(e);
    sgr::TopoCounters h;
    if ((e = cudaMemcpyAsync(c->host_small, tc, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
    std::memcpy(&h, c->host_small, sizeof(h));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    sgr_stats s;
    std::memset(&s, 0, sizeof(s));
    s.rounds = rounds;
    s.sum_w = (int64_t)h.nw;
    s.sum_d = (int64_t)h.dsum;
    s.sum_next = (int64_t)h.nw - (int64_t)j.n;  // every vertex but the first-round ones came back
    s.num_colors = h.kmax;
    s.grid_blocks = grid;
    s.block_threads = 256;
    s.device_ms = ms;
    t_stats = s;
    c->last_trace = nullptr;  // no per-round timeline on this schedule
    c->last_rounds = 0;
    if (k_out) *k_out = h.kmax;
    return SGR_OK;
}

// Run the coloring launches for a job (single graph or batch) and read back
// the counters.  Caller holds the device mutex.
int run_job(DevCtx *c, Job &j, int mode, cudaStream_t st, int32_t *k_out) {
    if ((mode & SGR_MODE_MASK) == SGR_MODE_TOPO) return run_topo(c, j, (mode & SGR_RULE_MASK) >> 4, st, k_out);
    const sgr_tuning t = current_tuning();
    const bool fast = (mode & SGR_MODE_MASK) == SGR_MODE_FAST;
    const int rule = (mode & SGR_RULE_MASK) >> 4;
    j.fast = fast;
    size_t zero_bytes = 0;
    size_t need = layout(j, t, nullptr, nullptr, &zero_bytes);
    const size_t gid_off = need;
    if (j.batched) need = align_up(need + (size_t)j.n * 4) + align_up((size_t)(j.G + 1) * 8) * 3 +
                          align_up((size_t)j.G * 4);
    cudaError_t e = c->scratch.ensure(need);
    if (e != cudaSuccess) return map_cuda(e);
    if (j.batched) {
        j.gid_dev = (int32_t *)(c->scratch.ptr + gid_off);
    }
    Params p;
    layout(j, t, c->scratch.ptr, &p, nullptr);
    p.rule = rule;
    p.max_rounds = (long long)j.n + 1;
    if ((e = cudaMemsetAsync(c->scratch.ptr, 0, zero_bytes, st)) != cudaSuccess) return map_cuda(e);
    if (j.batched) {
        if ((e = sgr::launch_fill_gid(j.gid_dev, j.vbase_dev, j.G, j.n, st)) != cudaSuccess)
            return map_cuda(e);
    }
    if ((e = cudaEventRecord(c->ev0, st)) != cudaSuccess) return map_cuda(e);
    int grid = 0;
    if ((e = launch_rounds(p, fast, j.batched, c->occ[fast][j.batched], c->occ_front[j.batched], c->sms,
                           t, st, &grid)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaEventRecord(c->ev1, st)) != cudaSuccess) return map_cuda(e);
    if ((e = cudaMemcpyAsync(c->host_ctr, p.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    const Counters h = *c->host_ctr;
    fill_stats(h, ms, grid, h.kmax);
    c->last_trace = p.trace;
    c->last_rounds = h.rounds;
    c->last_t_init = h.t_init_ns;
    if (h.err != 0) return h.err;
    if (k_out) *k_out = h.kmax;
    return SGR_OK;
}

}  // namespace

namespace sgr {

sgr_tuning tuning_snapshot() { return current_tuning(); }

// Scratch bytes color_single_in needs for a graph (deterministic mode, with
// the activation lists and the tail arrays of sgr_color).
size_t single_scratch_bytes(int32_t n, long long m) {
    Job j;
    std::memset(&j, 0, sizeof(j));
    j.n = n;
    j.m = m;
    j.front = true;
    j.tail = true;
    size_t zero_bytes = 0;
    return layout(j, current_tuning(), nullptr, nullptr, &zero_bytes);
}

// The launches of sgr_color (deterministic or fast mode) for one graph in
// device memory, with the scratch at `base` (cap bytes, 256-byte aligned,
// owned by the caller).  The caller holds the device's launch mutex.  Writes
// k to *k_out and the rounds to *rounds_out on success; SGR_ERR_INVALID_ARG
// if the scratch does not fit.  Used by the server for requests it colors
// alone between its batched launches.
int color_single_in(char *base, size_t cap, int32_t n, long long m, const int32_t *ro, const int32_t *ci,
                    int32_t *colors, int mode, cudaStream_t st, int32_t *k_out, long long *rounds_out) {
    if (n <= 0) {
        *k_out = 0;
        return SGR_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SGR_ERR_CUDA;
    const sgr_tuning t = current_tuning();
    const bool fast = (mode & SGR_MODE_MASK) == SGR_MODE_FAST;
    Job j;
    std::memset(&j, 0, sizeof(j));
    j.fast = fast;
    j.n = n;
    j.m = m;
    j.ro = ro;
    j.ci = ci;
    j.colors = colors;
    j.front = true;
    j.tail = true;
    size_t zero_bytes = 0;
    if (layout(j, t, nullptr, nullptr, &zero_bytes) > cap) return SGR_ERR_INVALID_ARG;
    Params p;
    layout(j, t, base, &p, nullptr);
    p.rule = (mode & SGR_RULE_MASK) >> 4;
    p.max_rounds = (long long)n + 1;
    int per_sm = 0, per_sm_f = 0, sms = 0;
    if (occupancy_blocks_per_sm(fast, false, &per_sm) != 0) return SGR_ERR_CUDA;
    if (occupancy_blocks_per_sm_front(false, &per_sm_f) != 0) return SGR_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SGR_ERR_CUDA;
    cudaError_t e = cudaMemsetAsync(base, 0, zero_bytes, st);
    if (e != cudaSuccess) return map_cuda(e);
    int grid = 0;
    if ((e = launch_rounds(p, fast, false, per_sm, per_sm_f, sms, t, st, &grid)) != cudaSuccess)
        return map_cuda(e);
    Counters h;  // pageable: the copy completes before the synchronisation returns
    if ((e = cudaMemcpyAsync(&h, p.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
    if (h.err != 0) return h.err;
    *k_out = h.kmax;
    *rounds_out = h.rounds;
    return SGR_OK;
}

unsigned long long wait_limit_ns() {
    const unsigned long long w = g_wait_ns.load();
    return w ? w : kWaitTimeoutNs;
}

bool inject_alloc_failure() {
    long long k = g_inject_alloc.load();
    while (k > 0) {
        if (g_inject_alloc.compare_exchange_weak(k, k - 1)) return k == 1;
    }
    return false;
}

unsigned inject_barrier_extra() {
    int k = g_inject_barrier.load();
    while (k > 0) {
        if (g_inject_barrier.compare_exchange_weak(k, k - 1)) return 1u;
    }
    return 0u;
}

// Cooperative persistent launches of this process on one device are
// serialised: two of them in flight could each wait in a grid barrier for
// CTAs that cannot become resident.
std::mutex &device_launch_mutex(int device) { return ctx_struct(device)->mu; }

}  // namespace sgr

extern "C" {

int sgr_version(void) { return 10000; }

const char *sgr_status_string(int s) {
    switch (s) {
        case SGR_OK: return "SGR_OK";
        case SGR_PENDING: return "SGR_PENDING";
        case SGR_ERR_INVALID_ARG: return "SGR_ERR_INVALID_ARG";
        case SGR_ERR_INVALID_GRAPH: return "SGR_ERR_INVALID_GRAPH";
        case SGR_ERR_OUT_OF_MEMORY: return "SGR_ERR_OUT_OF_MEMORY";
        case SGR_ERR_CUDA: return "SGR_ERR_CUDA";
        case SGR_ERR_NO_CONVERGENCE: return "SGR_ERR_NO_CONVERGENCE";
        case SGR_ERR_TIMEOUT: return "SGR_ERR_TIMEOUT";
        case SGR_ERR_NOT_FOUND: return "SGR_ERR_NOT_FOUND";
        case SGR_ERR_BUSY: return "SGR_ERR_BUSY";
        default: return "SGR_UNKNOWN_STATUS";
    }
}

int sgr_get_tuning(sgr_tuning *out) {
    if (!out) return SGR_ERR_INVALID_ARG;
    *out = current_tuning();
    return SGR_OK;
}

int sgr_set_tuning(const sgr_tuning *in) {
    if (!in) return SGR_ERR_INVALID_ARG;
    sgr_tuning t = current_tuning();
    if (in->active_lists < 0 || in->active_lists > 2) return SGR_ERR_INVALID_ARG;
    t.active_lists = in->active_lists;
    if (in->tail_vertices < -1 || in->tail_vertices > sgr::kTailMax) return SGR_ERR_INVALID_ARG;
    t.tail_vertices = in->tail_vertices;
    if (in->light_max) {
        if (in->light_max < 1 || in->light_max > sgr::kLightMaxStage) return SGR_ERR_INVALID_ARG;
        t.light_max = in->light_max;
    }
    if (in->chunk) {
        if (in->chunk < 64 || in->chunk > (1 << 24)) return SGR_ERR_INVALID_ARG;
        t.chunk = in->chunk;
    }
    if (in->blocks_per_sm < 0 || in->blocks_per_sm > 64) return SGR_ERR_INVALID_ARG;
    t.blocks_per_sm = in->blocks_per_sm;
    if (t.light_max >= t.chunk) return SGR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = t;
    return SGR_OK;
}

int sgr_set_wait_limit(int64_t ns) {
    if (ns != 0 && (ns < 100000 || ns > 600000000000ll)) return SGR_ERR_INVALID_ARG;
    g_wait_ns.store((unsigned long long)ns);
    return SGR_OK;
}

int sgr_debug_inject(int what, int64_t value) {
    if (value < 0 || value > (1ll << 30)) return SGR_ERR_INVALID_ARG;
    switch (what) {
        case SGR_INJECT_NONE:
            g_inject_alloc.store(0);
            g_inject_barrier.store(0);
            return SGR_OK;
        case SGR_INJECT_FAIL_ALLOC:
            g_inject_alloc.store(value);
            return SGR_OK;
        case SGR_INJECT_BARRIER:
            g_inject_barrier.store((int)value);
            return SGR_OK;
        default:
            return SGR_ERR_INVALID_ARG;
    }
}

int sgr_last_stats(sgr_stats *out) {
    if (!out) return SGR_ERR_INVALID_ARG;
    *out = t_stats;
    return SGR_OK;
}

int sgr_last_trace(int64_t *out, int64_t cap_rounds, int64_t *init_ns) {
    if (!out || cap_rounds < 0) return SGR_ERR_INVALID_ARG;
    DevCtx *c = nullptr;
    int rc = get_ctx(&c);
    if (rc != SGR_OK) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->last_trace) return 0;
    long long r = std::min<long long>(std::min<long long>(c->last_rounds, sgr::kTraceCap), cap_rounds);
    if (r > 0) {
        cudaError_t e = cudaMemcpy(out, c->last_trace, (size_t)r * sgr::kTraceFields * 8,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return map_cuda(e);
    }
    if (init_ns) *init_ns = c->last_t_init;
    return (int)r;
}

int sgr_release_scratch(void) {
    DevCtx *c = nullptr;
    int rc = get_ctx(&c);
    if (rc != SGR_OK) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    c->scratch.release();
    c->io.release();
    c->last_trace = nullptr;
    return SGR_OK;
}

int sgr_color(int32_t n, const int32_t *row_offsets, const int32_t *col_idx, int32_t *colors_out,
              int32_t *num_colors, int mode, sgr_stream_t stream) {
    std::memset(&t_stats, 0, sizeof(t_stats));
    if (n < 0 || !num_colors || !valid_mode(mode, true)) return SGR_ERR_INVALID_ARG;
    if (n == 0) {
        *num_colors = 0;
        return SGR_OK;
    }
    if (!row_offsets || !col_idx || !colors_out) return SGR_ERR_INVALID_ARG;
    if (!is_device_ptr(row_offsets) || !is_device_ptr(colors_out)) return SGR_ERR_INVALID_ARG;
    DevCtx *c = nullptr;
    int rc = get_ctx(&c);
    if (rc != SGR_OK) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *hs = (int32_t *)c->host_ctr;  // reuse pinned memory for two ints
    cudaError_t e = cudaMemcpyAsync(hs, row_offsets, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs + 1, row_offsets + n, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return map_cuda(e);
    const int32_t r0 = hs[0], m = hs[1];
    if (r0 != 0 || m < 0) return SGR_ERR_INVALID_GRAPH;
    if (m > 0 && (((uintptr_t)col_idx & 15) != 0 || !is_device_ptr(col_idx))) return SGR_ERR_INVALID_ARG;
    Job j;
    std::memset(&j, 0, sizeof(j));
    j.n = n;
    j.m = m;
    j.ro = row_offsets;
    j.ci = col_idx;
    j.colors = colors_out;
    j.front = true;
    j.tail = true;
    return run_job(c, j, mode, st, num_colors);
}

int sgr_color_host(int32_t n, const int32_t *ro_h, const int32_t *ci_h, int32_t *colors_h,
                   int32_t *num_colors, int mode, sgr_stream_t stream) {
    std::memset(&t_stats, 0, sizeof(t_stats));
    if (n < 0 || !num_colors || !valid_mode(mode, true)) return SGR_ERR_INVALID_ARG;
    if (n == 0) {
        *num_colors = 0;
        return SGR_OK;
    }
    if (!ro_h || !colors_h) return SGR_ERR_INVALID_ARG;
    const long long m = ro_h[n];
    if (ro_h[0] != 0 || m < 0) return SGR_ERR_INVALID_GRAPH;
    if (m > 0 && !ci_h) return SGR_ERR_INVALID_ARG;
    DevCtx *c = nullptr;
    int rc = get_ctx(&c);
    if (rc != SGR_OK) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t b_ro = align_up((size_t)(n + 1) * 4), b_ci = align_up((size_t)m * 4 + 16);
    const size_t b_co = align_up((size_t)n * 4);
    cudaError_t e = c->io.ensure(b_ro + b_ci + b_co);
    if (e != cudaSuccess) return map_cuda(e);
    int32_t *ro_d = (int32_t *)c->io.ptr;
    int32_t *ci_d = (int32_t *)(c->io.ptr + b_ro);
    int32_t *co_d = (int32_t *)(c->io.ptr + b_ro + b_ci);
    if ((e = cudaMemcpyAsync(ro_d, ro_h, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return map_cuda(e);
    if (m > 0 && (e = cudaMemcpyAsync(ci_d, ci_h, (size_t)m * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return map_cuda(e);
    Job j;
    std::memset(&j, 0, sizeof(j));
    j.n = n;
    j.m = m;
    j.ro = ro_d;
    j.ci = ci_d;
    j.colors = co_d;
    j.front = true;
    j.tail = true;
    int32_t k = 0;
    rc = run_job(c, j, mode, st, &k);
    if (rc != SGR_OK) return rc;
    if ((e = cudaMemcpyAsync(colors_h, co_d, (size_t)n * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
    *num_colors = k;
    return SGR_OK;
}

int sgr_color_batch(int32_t G, const int64_t *vtx_off, const int64_t *edge_off,
                    const int32_t *row_offsets, const int32_t *col_idx, int32_t *colors_out,
                    int32_t *num_colors, int mode, sgr_stream_t stream) {
    std::memset(&t_stats, 0, sizeof(t_stats));
    if (G < 0 || !valid_mode(mode)) return SGR_ERR_INVALID_ARG;
    if (G == 0) return SGR_OK;
    if (!vtx_off || !edge_off || !num_colors || !row_offsets) return SGR_ERR_INVALID_ARG;
    if (vtx_off[0] != 0 || edge_off[0] != 0) return SGR_ERR_INVALID_GRAPH;
    for (int g = 0; g < G; ++g)
        if (vtx_off[g + 1] < vtx_off[g] || edge_off[g + 1] < edge_off[g]) return SGR_ERR_INVALID_GRAPH;
    const long long n = vtx_off[G], m = edge_off[G];
    if (n + G >= (1ll << 31)) return SGR_ERR_INVALID_ARG;
    if (n == 0) {
        for (int g = 0; g < G; ++g) num_colors[g] = 0;
        return SGR_OK;
    }
    if (!colors_out || !is_device_ptr(row_offsets) || !is_device_ptr(colors_out)) return SGR_ERR_INVALID_ARG;
    if (m > 0 && (!col_idx || ((uintptr_t)col_idx & 15) != 0 || !is_device_ptr(col_idx)))
        return SGR_ERR_INVALID_ARG;
    DevCtx *c = nullptr;
    int rc = get_ctx(&c);
    if (rc != SGR_OK) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_host_small(c, 3 * (size_t)(G + 1) + (size_t)G)) != SGR_OK) return rc;
    Job j;
    std::memset(&j, 0, sizeof(j));
    j.n = (int32_t)n;
    j.m = m;
    j.ro = row_offsets;
    j.ci = col_idx;
    j.colors = colors_out;
    j.batched = true;
    j.G = G;
    j.fast = (mode & SGR_MODE_MASK) == SGR_MODE_FAST;
    j.front = true;
    j.tail = true;
    // the batch tail of the arena: gid, vbase, ebase, per-graph k (see run_job)
    const sgr_tuning t = current_tuning();
    size_t zero_bytes = 0;
    const size_t base_need = layout(j, t, nullptr, nullptr, &zero_bytes);
    const size_t need = align_up(base_need + (size_t)n * 4) + align_up((size_t)(G + 1) * 8) * 3 +
                        align_up((size_t)G * 4);
    cudaError_t e = c->scratch.ensure(need);
    if (e != cudaSuccess) return map_cuda(e);
    char *tail = c->scratch.ptr + align_up(base_need + (size_t)n * 4);
    long long *vb_d = (long long *)tail;
    long long *eb_d = (long long *)(tail + align_up((size_t)(G + 1) * 8));
    long long *rb_d = (long long *)(tail + 2 * align_up((size_t)(G + 1) * 8));
    int32_t *k_d = (int32_t *)(tail + 3 * align_up((size_t)(G + 1) * 8));
    std::memcpy(c->host_small, vtx_off, (size_t)(G + 1) * 8);
    std::memcpy(c->host_small + (G + 1), edge_off, (size_t)(G + 1) * 8);
    for (int g = 0; g <= G; ++g) c->host_small[2 * (G + 1) + g] = vtx_off[g] + g;
    if ((e = cudaMemcpyAsync(vb_d, c->host_small, (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaMemcpyAsync(eb_d, c->host_small + (G + 1), (size_t)(G + 1) * 8, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaMemcpyAsync(rb_d, c->host_small + 2 * (G + 1), (size_t)(G + 1) * 8,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return map_cuda(e);
    j.vbase_dev = vb_d;
    j.ebase_dev = eb_d;
    j.robase_dev = rb_d;
    int32_t kall = 0;
    rc = run_job(c, j, mode, st, &kall);
    if (rc != SGR_OK) return rc;
    if ((e = sgr::launch_segmented_max(colors_out, vb_d, G, k_d, st)) != cudaSuccess) return map_cuda(e);
    int32_t *kh = (int32_t *)(c->host_small + 3 * (G + 1));
    if ((e = cudaMemcpyAsync(kh, k_d, (size_t)G * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
    std::memcpy(num_colors, kh, (size_t)G * 4);
    return SGR_OK;
}

}  // extern "C"

namespace {

// The autotuner's candidate grid, measured in this order until the budget is
// spent (the library default first): degree bound of the lane-per-vertex bin,
// hub chunk size (also the warp-per-vertex bound), CTAs per SM (0 = as many
// as fit) and, in deterministic mode, the hand-over size of the one-CTA tail.
// run(t) makes one coloring call under tuning t and returns its status; the
// call's device time is read from the thread's statistics.
template <class Run>
int autotune_grid(int mode, int32_t budget_ms, sgr_tuning *best, double *best_ms, Run run) {
    const sgr_tuning start = current_tuning();
    const bool det = (mode & SGR_MODE_MASK) == SGR_MODE_DETERMINISTIC;
    const int32_t chunks[] = {1024, 512, 256, 2048};
    const int32_t lights[] = {32, 16};
    const int32_t ctas[] = {0, 2};
    const int32_t tails[] = {0, 1024, 2880};
    const int ntails = det ? 3 : 1;
    const double budget = budget_ms > 0 ? budget_ms : 2000.0;
    double spent = 0, best_t = 1e300;
    sgr_tuning bt = start;
    int tried = 0;
    for (int ti = 0; ti < ntails; ++ti)
        for (int32_t b : ctas)
            for (int32_t c : chunks)
                for (int32_t l : lights) {
                    if (tried > 0 && spent > budget) continue;
                    sgr_tuning t = {l, c, b, start.active_lists, det ? tails[ti] : start.tail_vertices};
                    if (sgr_set_tuning(&t) != SGR_OK) continue;
                    double tmin = 1e300;
                    for (int rep = 0; rep < 2; ++rep) {  // the first run also warms caches
                        const int rc = run();
                        if (rc != SGR_OK) {
                            sgr_set_tuning(&start);
                            return rc;
                        }
                        tmin = std::min(tmin, t_stats.device_ms);
                        spent += t_stats.device_ms;
                    }
                    ++tried;
                    if (tmin < best_t) {
                        best_t = tmin;
                        bt = t;
                    }
                }
    sgr_set_tuning(&bt);
    *best = bt;
    if (best_ms) *best_ms = best_t;
    return SGR_OK;
}

}  // namespace

extern "C" {

int sgr_autotune(int32_t n, const int32_t *row_offsets, const int32_t *col_idx,
                 int32_t *colors_out, int mode, int32_t budget_ms, sgr_tuning *best,
                 double *best_ms, sgr_stream_t stream) {
    if (!best || !valid_mode(mode) || n < 0) return SGR_ERR_INVALID_ARG;
    if (n == 0) {
        *best = current_tuning();
        if (best_ms) *best_ms = 0;
        return SGR_OK;
    }
    int32_t k = 0;
    return autotune_grid(mode, budget_ms, best, best_ms, [&] {
        return sgr_color(n, row_offsets, col_idx, colors_out, &k, mode, stream);
    });
}

int sgr_autotune_batch(int32_t G, const int64_t *vtx_off, const int64_t *edge_off,
                       const int32_t *row_offsets, const int32_t *col_idx, int32_t *colors_out,
                       int32_t *num_colors, int mode, int32_t budget_ms, sgr_tuning *best,
                       double *best_ms, sgr_stream_t stream) {
    if (!best || !valid_mode(mode) || G < 0 || (G > 0 && (!vtx_off || !num_colors))) return SGR_ERR_INVALID_ARG;
    if (G == 0 || vtx_off[G] == 0) {
        *best = current_tuning();
        if (best_ms) *best_ms = 0;
        return sgr_color_batch(G, vtx_off, edge_off, row_offsets, col_idx, colors_out, num_colors, mode,
                               stream);
    }
    return autotune_grid(mode, budget_ms, best, best_ms, [&] {
        return sgr_color_batch(G, vtx_off, edge_off, row_offsets, col_idx, colors_out, num_colors, mode,
                               stream);
    });
}

int sgr_validate_csr(int32_t n, const int32_t *row_offsets, const int32_t *col_idx,
                     int32_t *rows_sorted, sgr_stream_t stream) {
    if (n < 0) return SGR_ERR_INVALID_ARG;
    if (n == 0) {
        if (rows_sorted) *rows_sorted = 1;
        return SGR_OK;
    }
    if (!row_offsets || !is_device_ptr(row_offsets)) return SGR_ERR_INVALID_ARG;
    DevCtx *c = nullptr;
    int rc = get_ctx(&c);
    if (rc != SGR_OK) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *hs = (int32_t *)c->host_ctr;
    cudaError_t e = cudaMemcpyAsync(hs, row_offsets, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs + 1, row_offsets + n, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return map_cuda(e);
    if (hs[0] != 0 || hs[1] < 0) return SGR_ERR_INVALID_GRAPH;
    const long long m_v = hs[1];
    if (m_v > 0 && (!col_idx || !is_device_ptr(col_idx))) return SGR_ERR_INVALID_ARG;
    if ((e = c->scratch.ensure(256)) != cudaSuccess) return map_cuda(e);
    unsigned long long *flags = (unsigned long long *)c->scratch.ptr;
    unsigned long long *fh = (unsigned long long *)c->host_ctr;
    if ((e = cudaMemsetAsync(flags, 0, 24, st)) != cudaSuccess) return map_cuda(e);
    if ((e = sgr::launch_validate(n, m_v, row_offsets, col_idx, flags, st)) != cudaSuccess) return map_cuda(e);
    if ((e = cudaMemcpyAsync(fh, flags, 24, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return map_cuda(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
    const unsigned long long f = fh[0], h1 = fh[1], h2 = fh[2];
    const int sorted = (f & 8) ? 0 : 1;
    if (rows_sorted) *rows_sorted = sorted;
    if (f & (1 | 2 | 4 | 16)) return SGR_ERR_INVALID_GRAPH;
    if (h1 != h2) return SGR_ERR_INVALID_GRAPH;
    if (sorted) {
        if ((e = cudaMemsetAsync(flags, 0, 24, st)) != cudaSuccess) return map_cuda(e);
        if ((e = sgr::launch_validate_exact(n, m_v, row_offsets, col_idx, flags, st)) != cudaSuccess)
            return map_cuda(e);
        if ((e = cudaMemcpyAsync(fh, flags, 24, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return map_cuda(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
        if (fh[0] & (1 | 2 | 4 | 16 | 32)) return SGR_ERR_INVALID_GRAPH;
    }
    return SGR_OK;
}

}  // extern "C"


// ---------------------------------------------------------------------------
// Coloring without any allocation by the library (no counterpart in the
// paper).
//
// Some callers must not let a library allocate device memory: an application
// that gives a plugin a fixed share of the GPU and routes every allocation
// through its own pool, or a latency-sensitive loop in which a cudaMalloc or
// cudaFree would synchronise the device and stall work on other streams.  For
// them sgr_color_noalloc runs the same coloring kernel with its scratch in
// g_noalloc_scratch, a fixed-size array that is part of this library's device
// image: every GPU that loads the library holds it until the process exits.
// The caller still owns and passes the graph and the colors buffer.
//
// In host code the name g_noalloc_scratch only stands for the array; its
// device address comes from cudaGetSymbolAddress, taken once per device (with
// that device current) by the first sgr_color_noalloc call on the device.
// Every call shares the one array and leaves the last call's contents in it;
// the call clears what must start at zero.  Two calls whose GPU work
// overlapped would race on it; within one process the calls on a device are
// serialised and each returns only after its work is done.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu[kNoAllocMaxDevices];
char *g_noalloc_ptr[kNoAllocMaxDevices];

}  // namespace

extern "C" int sgr_color_noalloc(int32_t n, const int32_t *row_offsets, const int32_t *col_idx,
                                 int32_t *colors_out, int32_t *num_colors, int mode,
                                 sgr_stream_t stream) {
    std::memset(&t_stats, 0, sizeof(t_stats));
    if (n < 0 || !num_colors || !valid_mode(mode)) return SGR_ERR_INVALID_ARG;
    if (n == 0) {
        *num_colors = 0;
        return SGR_OK;
    }
    if (!row_offsets || !col_idx || !colors_out) return SGR_ERR_INVALID_ARG;
    if (!is_device_ptr(row_offsets) || !is_device_ptr(colors_out)) return SGR_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return SGR_ERR_CUDA;
    // Lock order: the array's mutex, then the device's launch mutex, which
    // every other coloring entry point holds around its cooperative launches
    // (two persistent grids in flight on one device could each wait in a grid
    // barrier for CTAs that cannot become resident).  Nothing takes them in
    // the other order.
    std::lock_guard<std::mutex> lk(g_noalloc_mu[dev]);
    std::lock_guard<std::mutex> dev_lk(sgr::device_launch_mutex(dev));
    if (!g_noalloc_ptr[dev]) {  // set-up, once per device, with that device current
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SGR_ERR_CUDA;
        g_noalloc_ptr[dev] = (char *)ptr;
    }
    char *base = g_noalloc_ptr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    int32_t ends[2] = {0, 0};  // pageable: the copies complete before the synchronisation returns
    cudaError_t e = cudaMemcpyAsync(&ends[0], row_offsets, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], row_offsets + n, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return map_cuda(e);
    const int32_t m = ends[1];
    if (ends[0] != 0 || m < 0) return SGR_ERR_INVALID_GRAPH;
    if (m > 0 && (((uintptr_t)col_idx & 15) != 0 || !is_device_ptr(col_idx))) return SGR_ERR_INVALID_ARG;
    const sgr_tuning t = current_tuning();
    const bool fast = (mode & SGR_MODE_MASK) == SGR_MODE_FAST;
    Job j;
    std::memset(&j, 0, sizeof(j));
    j.fast = fast;
    j.n = n;
    j.m = m;
    j.ro = row_offsets;
    j.ci = col_idx;
    j.colors = colors_out;
    size_t zero_bytes = 0;
    j.front = true;  // the activation lists only if they fit beside the rest
    if (layout(j, t, nullptr, nullptr, &zero_bytes) > kNoAllocScratchBytes) j.front = false;
    if (layout(j, t, nullptr, nullptr, &zero_bytes) > kNoAllocScratchBytes)
        return SGR_ERR_INVALID_ARG;  // the graph needs more scratch than the fixed array holds
    Params p;
    layout(j, t, base, &p, nullptr);
    p.rule = (mode & SGR_RULE_MASK) >> 4;
    p.max_rounds = (long long)n + 1;
    int per_sm = 0, per_sm_f = 0, sms = 0;
    if (sgr::occupancy_blocks_per_sm(fast, false, &per_sm) != 0) return SGR_ERR_CUDA;
    if (sgr::occupancy_blocks_per_sm_front(false, &per_sm_f) != 0) return SGR_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SGR_ERR_CUDA;
    if ((e = cudaMemsetAsync(base, 0, zero_bytes, st)) != cudaSuccess) return map_cuda(e);
    int grid = 0;
    if ((e = launch_rounds(p, fast, false, per_sm, per_sm_f, sms, t, st, &grid)) != cudaSuccess)
        return map_cuda(e);
    Counters h;
    if ((e = cudaMemcpyAsync(&h, p.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return map_cuda(e);
    fill_stats(h, 0.f, grid, h.kmax);
    {  // sgr_last_trace now reads this call's timeline (in the fixed array)
        DevCtx *c = ctx_struct(dev);
        c->last_trace = p.trace;
        c->last_rounds = h.rounds;
        c->last_t_init = h.t_init_ns;
    }
    if (h.err != 0) return h.err;
    *num_colors = h.kmax;
    return SGR_OK;
}
