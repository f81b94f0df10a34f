// sgr_server.cu -- a continuous-batching coloring server (deterministic mode).
//
// Requests (host CSR graphs) arrive at any time through sgr_server_submit.
// A scheduler thread keeps every admitted graph resident on the device: its
// CSR in two arenas (row offsets, column ids), its per-vertex state (colors,
// forbidden-color bitmaps, worklist entries) in a global vertex space where
// it owns a contiguous range.  The rounds of all resident graphs advance
// together: each launch of the resumable persistent kernel runs R rounds of
// Algorithm 7 over the union of their worklists (graphs are disjoint, so each
// still gets exactly its own coloring), then returns.  Between launches the
// scheduler retires graphs whose vertices are all final (device-side status
// pass, then a copy of their colors to the host) and admits queued requests
// whose vertex and entry ranges fit in the free space of the arenas, which are
// sized from the HBM budget at creation.  A new graph joins the running rounds
// at its own round 1 while the others are further along.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sgr_internal.cuh"
#include "sgrcolor.h"

namespace {

using Clock = std::chrono::steady_clock;

int map_err(cudaError_t e) {
    if (e == cudaSuccess) return SGR_OK;
    if (e == cudaErrorMemoryAllocation) return SGR_ERR_OUT_OF_MEMORY;
    return SGR_ERR_CUDA;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator of ranges in [0, cap).
struct RangeAlloc {
    std::map<long long, long long> free_;  // start -> length
    long long cap = 0, used = 0;
    void init(long long c) {
        cap = c;
        used = 0;
        free_.clear();
        if (c > 0) free_[0] = c;
    }
    long long alloc(long long len) {
        if (len <= 0) return 0;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < len) continue;
            const long long off = it->first, rest = it->second - len;
            free_.erase(it);
            if (rest) free_[off + len] = rest;
            used += len;
            return off;
        }
        return -1;
    }
    void release(long long off, long long len) {
        if (len <= 0) return;
        used -= len;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// Host copy of a request's CSR ([row offsets | col_idx]) and later of its
// colors: in the server's pinned staging pool when there is room (the copies
// to and from the device are then asynchronous), in ordinary memory otherwise.
struct HostBuf {
    int32_t *ptr = nullptr;
    long long off = -1, len = 0;  // range in the pinned pool, off < 0: in vec
    std::vector<int32_t> vec;
};

struct Request {
    uint64_t id = 0;
    int32_t n = 0;
    long long m = 0;
    HostBuf csr, out;
    Clock::time_point t_submit, t_done;
    int status = SGR_PENDING;
    int32_t k = 0;
    int slot = -1;
    long long vb = 0, eb = 0, rb = 0;
    long long r_admit = 0;  // server round at which the graph's round 1 runs
    long long ealen = 0;    // entries of its col_idx range (m rounded up to 16 bytes)
    bool direct = false;    // colored alone on the single-graph kernels
};

}  // namespace

struct sgr_server {
    sgr_server_config cfg{};
    int device = 0, sms = 0, per_sm = 0, grid = 0;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    int fatal = SGR_OK;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> reqs;
    std::vector<Request *> slot_req;
    std::vector<int> free_slots;
    uint64_t next_id = 1;
    RangeAlloc va, ea, ra;
    long long Vcap = 0, Ecap = 0, Rcap = 0;
    int G = 0;
    char *dmem = nullptr;
    size_t dbytes = 0;
    sgr::Params P{};
    long long *vbase_d = nullptr, *ebase_d = nullptr, *robase_d = nullptr;
    int32_t *nv_d = nullptr, *rem_d = nullptr, *kmax_d = nullptr;
    int32_t *pinned = nullptr;    // staging pool (int32 words)
    RangeAlloc pa;                // ranges of the staging pool
    long long *tab_h = nullptr;   // pinned mirrors: vbase, ebase, robase (G each)
    int32_t *nv_h = nullptr, *rem_h = nullptr, *kmax_h = nullptr;
    sgr::Counters *ctr_h = nullptr;
    long long round = 1;
    char *direct_mem = nullptr;   // scratch of requests colored alone (part of the budget)
    size_t direct_cap = 0;
    long long direct_min = 0;     // vertices from which a request is colored alone
    long long direct_count = 0;
    cudaStream_t copy_stream = nullptr;  // host<->device copies of requests colored alone
    static constexpr int kDirectPass = 4;  // requests colored alone per pass, at most
    cudaEvent_t ev_in[kDirectPass] = {}, ev_done[kDirectPass] = {};
    // statistics
    std::vector<double> lat_ms;
    long long submitted = 0, completed = 0, failed = 0, launches = 0, rounds_run = 0;
    bool any_submit = false;
    Clock::time_point t_first_submit, t_last_done;
};

namespace {

// Per-vertex device bytes: colors, 8 bitmap words, lower count, five witness
// slots, graph id, two parities of three worklists and hub chunk bases, the
// same for the unsettled lists, six hub arrays, one row offset.
constexpr long long kVertexBytes = 4 + 32 + 4 + 4 + 16 + 4 + 2 * 4 * 4 + 2 * 4 * 4 + 6 * 4 + 4;

int carve(sgr_server *S) {
    // a quarter of the budget for the scratch of requests colored alone
    S->direct_cap = S->direct_min > 0 ? align_up((size_t)(S->cfg.hbm_budget_bytes / 4)) : 0;
    const long long budget = S->cfg.hbm_budget_bytes - (long long)S->direct_cap;
    const int G = S->G;
    const size_t fixed = align_up(sizeof(sgr::Counters)) +
                         align_up(sizeof(long long) * sgr::kTraceCap * sgr::kTraceFields) +
                         3 * align_up((size_t)G * 8) + 3 * align_up((size_t)G * 4) + 64 * 256;
    if (budget < (long long)fixed + (1 << 20)) return SGR_ERR_INVALID_ARG;
    long long Vcap = (long long)((budget - (long long)fixed) * 0.3) / kVertexBytes;
    Vcap = std::min<long long>(Vcap, (1ll << 31) - 2 * G - 64);
    Vcap = Vcap / 64 * 64;
    long long Ecap = (budget - (long long)fixed - Vcap * kVertexBytes) / 4 - 64;
    if (Vcap < 64 || Ecap < 64) return SGR_ERR_INVALID_ARG;
    S->Vcap = Vcap;
    S->Ecap = Ecap;
    S->Rcap = Vcap + G;
    size_t off = 0;
    std::vector<std::pair<void **, size_t>> parts;
    sgr::Params &P = S->P;
    std::memset(&P, 0, sizeof(P));
    auto take = [&](void **dst, size_t bytes) { parts.push_back({dst, bytes}); };
    int32_t *lw0, *lw1, *mw0, *mw1, *hw0, *hw1, *gid, *ro, *ci;
    unsigned *hcb0, *hcb1;
    int32_t *ul0, *ul1, *um0, *um1, *uh0, *uh1;
    unsigned *ucb0, *ucb1;
    take((void **)&P.ctr, sizeof(sgr::Counters));
    take((void **)&P.hdone, (size_t)Vcap * 8);
    take((void **)&P.hconf, (size_t)Vcap * 4);
    take((void **)&P.trace, sizeof(long long) * sgr::kTraceCap * sgr::kTraceFields);
    take((void **)&P.colors, (size_t)Vcap * 4);
    take((void **)&P.bm, (size_t)Vcap * 8 * 4);
    take((void **)&P.lowdeg, (size_t)Vcap * 4);
    take((void **)&P.witness, (size_t)Vcap * 4);
    take((void **)&P.wold, (size_t)Vcap * 16);
    take((void **)&gid, (size_t)Vcap * 4);
    take((void **)&lw0, (size_t)Vcap * 4);
    take((void **)&lw1, (size_t)Vcap * 4);
    take((void **)&mw0, (size_t)Vcap * 4);
    take((void **)&mw1, (size_t)Vcap * 4);
    take((void **)&hw0, (size_t)Vcap * 4);
    take((void **)&hw1, (size_t)Vcap * 4);
    take((void **)&hcb0, (size_t)Vcap * 4);
    take((void **)&hcb1, (size_t)Vcap * 4);
    take((void **)&ul0, (size_t)Vcap * 4);
    take((void **)&ul1, (size_t)Vcap * 4);
    take((void **)&um0, (size_t)Vcap * 4);
    take((void **)&um1, (size_t)Vcap * 4);
    take((void **)&uh0, (size_t)Vcap * 4);
    take((void **)&uh1, (size_t)Vcap * 4);
    take((void **)&ucb0, (size_t)Vcap * 4);
    take((void **)&ucb1, (size_t)Vcap * 4);
    take((void **)&P.hvert, (size_t)Vcap * 4);
    take((void **)&P.hbase, (size_t)Vcap * 4);
    take((void **)&P.sw, (size_t)Vcap * 4);
    take((void **)&P.scb, (size_t)Vcap * 4);
    take((void **)&P.hbits, 256);
    take((void **)&S->vbase_d, (size_t)G * 8);
    take((void **)&S->ebase_d, (size_t)G * 8);
    take((void **)&S->robase_d, (size_t)G * 8);
    take((void **)&S->nv_d, (size_t)G * 4);
    take((void **)&S->rem_d, (size_t)G * 4);
    take((void **)&S->kmax_d, (size_t)G * 4);
    take((void **)&ro, (size_t)S->Rcap * 4);
    take((void **)&ci, (size_t)Ecap * 4 + 64);
    if (S->direct_cap) take((void **)&S->direct_mem, S->direct_cap);
    for (auto &pr : parts) off += align_up(pr.second);
    if (sgr::inject_alloc_failure()) return SGR_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaMalloc(&S->dmem, off);
    if (e != cudaSuccess) {
        S->dmem = nullptr;
        return map_err(e);
    }
    S->dbytes = off;
    off = 0;
    for (auto &pr : parts) {
        *pr.first = S->dmem + off;
        off += align_up(pr.second);
    }
    if ((e = cudaMemset(S->dmem, 0, S->dbytes)) != cudaSuccess) return map_err(e);
    P.ro = ro;
    P.ci = ci;
    P.gid = gid;
    P.vbase = S->vbase_d;
    P.ebase = S->ebase_d;
    P.robase = S->robase_d;
    P.m = Ecap;
    P.n = (int32_t)Vcap;
    P.np = Vcap;
    P.lw[0] = lw0; P.lw[1] = lw1;
    P.mw[0] = mw0; P.mw[1] = mw1;
    P.hw[0] = hw0; P.hw[1] = hw1;
    P.hcb[0] = hcb0; P.hcb[1] = hcb1;
    P.ul[0] = ul0; P.ul[1] = ul1;
    P.um[0] = um0; P.um[1] = um1;
    P.uh[0] = uh0; P.uh[1] = uh1;
    P.ucb[0] = ucb0; P.ucb[1] = ucb1;
    const sgr_tuning t = sgr::tuning_snapshot();
    P.light_max = t.light_max;
    P.chunk = t.chunk;
    P.rule = (S->cfg.mode & SGR_RULE_MASK) >> 4;
    P.max_rounds = LLONG_MAX / 4;  // per-graph caps are kept by the scheduler
    P.resume = 1;
    P.resume_sorted = 1;
    S->va.init(Vcap);
    S->ea.init(Ecap);
    S->ra.init(S->Rcap);
    // the first round number must be visible to the first resumable launch
    sgr::Counters c0;
    std::memset(&c0, 0, sizeof(c0));
    c0.round = 1;
    if ((e = cudaMemcpy(P.ctr, &c0, sizeof(c0), cudaMemcpyHostToDevice)) != cudaSuccess) return map_err(e);
    return SGR_OK;
}

void finish(sgr_server *S, Request *q, int status) {
    // caller holds S->mu
    q->status = status;
    q->t_done = Clock::now();
    if (status == SGR_OK) {
        S->completed++;
        S->lat_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
        S->t_last_done = q->t_done;
    } else {
        S->failed++;
    }
    S->cv_done.notify_all();
}

// caller holds S->mu
void host_alloc(sgr_server *S, HostBuf &b, long long words) {
    b.len = words;
    b.off = words > 0 ? S->pa.alloc(words) : -1;
    if (b.off >= 0) {
        b.ptr = S->pinned + b.off;
    } else {
        b.vec.resize((size_t)std::max<long long>(words, 1));
        b.ptr = b.vec.data();
    }
}

// caller holds S->mu
void host_free(sgr_server *S, HostBuf &b) {
    if (b.off >= 0) S->pa.release(b.off, b.len);
    b.off = -1;
    b.len = 0;
    b.ptr = nullptr;
    std::vector<int32_t>().swap(b.vec);
}

void release_ranges(sgr_server *S, Request *q) {
    // caller holds S->mu
    S->va.release(q->vb, q->n);
    S->ea.release(q->eb, q->ealen);
    S->ra.release(q->rb, (long long)q->n + 1);
}

void release_slot(sgr_server *S, Request *q) {
    // caller holds S->mu
    release_ranges(S, q);
    S->slot_req[q->slot] = nullptr;
    S->free_slots.push_back(q->slot);
    q->slot = -1;
}

void fail_all_resident(sgr_server *S, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    for (int g = 0; g < S->G; ++g) {
        Request *q = S->slot_req[g];
        if (!q) continue;
        release_slot(S, q);
        finish(S, q, status);
    }
}

void worker_loop(sgr_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request *> admitted, direct;
        int resident = 0;
        bool have_pending = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            for (auto it = S->pending.begin(); it != S->pending.end();) {
                Request *q = *it;
                // large graphs are colored alone (one per pass, so that the
                // resident graphs keep advancing); the others join the rounds
                const bool alone = S->direct_cap > 0 && q->n >= S->direct_min &&
                                   sgr::single_scratch_bytes(q->n, q->m) <= S->direct_cap;
                if (alone && (int)direct.size() >= sgr_server::kDirectPass) { ++it; continue; }  // next pass
                if (!alone && S->free_slots.empty()) { ++it; continue; }
                q->ealen = (q->m + 3) & ~3ll;  // every col_idx range starts on 16 bytes
                const long long vb = S->va.alloc(q->n);
                if (vb < 0) { ++it; continue; }
                const long long eb = S->ea.alloc(q->ealen);
                if (eb < 0) { S->va.release(vb, q->n); ++it; continue; }
                const long long rb = S->ra.alloc((long long)q->n + 1);
                if (rb < 0) { S->va.release(vb, q->n); S->ea.release(eb, q->ealen); ++it; continue; }
                q->vb = vb;
                q->eb = eb;
                q->rb = rb;
                if (alone) {
                    q->direct = true;
                    direct.push_back(q);
                } else {
                    q->slot = S->free_slots.back();
                    S->free_slots.pop_back();
                    q->r_admit = S->round;
                    S->slot_req[q->slot] = q;
                    admitted.push_back(q);
                }
                it = S->pending.erase(it);
            }
            resident = S->G - (int)S->free_slots.size();
            have_pending = !S->pending.empty();
            if (resident == 0 && direct.empty()) {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        std::lock_guard<std::mutex> dev_lk(sgr::device_launch_mutex(S->device));
        cudaStream_t st = S->stream;
        cudaError_t e = cudaSuccess;
        // Requests colored alone, one after another with the launches of
        // sgr_color, in the scratch region.  Their CSR copies all go out at
        // once on the copy stream, and each one's colors come back on it while
        // the next one is colored, so that the copies overlap the coloring.
        std::vector<int> status(direct.size(), SGR_OK);
        for (size_t i = 0; i < direct.size(); ++i) {
            Request *q = direct[i];
            cudaError_t ce = cudaMemcpyAsync((int32_t *)S->P.ro + q->rb, q->csr.ptr, ((size_t)q->n + 1) * 4,
                                             cudaMemcpyHostToDevice, S->copy_stream);
            if (ce == cudaSuccess && q->m > 0)
                ce = cudaMemcpyAsync((int32_t *)S->P.ci + q->eb, q->csr.ptr + q->n + 1, (size_t)q->m * 4,
                                     cudaMemcpyHostToDevice, S->copy_stream);
            if (ce == cudaSuccess) ce = cudaEventRecord(S->ev_in[i], S->copy_stream);
            if (ce != cudaSuccess) status[i] = map_err(ce);
        }
        for (size_t i = 0; i < direct.size(); ++i) {
            Request *q = direct[i];
            int32_t k = 0;
            long long rr = 0;
            if (status[i] == SGR_OK) {
                cudaError_t ce = cudaStreamWaitEvent(st, S->ev_in[i], 0);
                status[i] = ce == cudaSuccess
                                ? sgr::color_single_in(S->direct_mem, S->direct_cap, q->n, q->m, S->P.ro + q->rb,
                                                       S->P.ci + q->eb, S->P.colors + q->vb, S->cfg.mode, st, &k,
                                                       &rr)
                                : map_err(ce);
            }
            q->k = k;
            if (status[i] == SGR_OK) {  // (the coloring has finished: color_single_in synchronised st)
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    host_alloc(S, q->out, q->n);
                }
                cudaError_t ce = cudaMemcpyAsync(q->out.ptr, S->P.colors + q->vb, (size_t)q->n * 4,
                                                 cudaMemcpyDeviceToHost, S->copy_stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(S->ev_done[i], S->copy_stream);
                if (ce != cudaSuccess) status[i] = map_err(ce);
            }
        }
        for (size_t i = 0; i < direct.size(); ++i) {  // finish in order as the copies land
            Request *q = direct[i];
            if (status[i] == SGR_OK) {
                const cudaError_t ce = cudaEventSynchronize(S->ev_done[i]);
                if (ce != cudaSuccess) status[i] = map_err(ce);
            }
            std::lock_guard<std::mutex> lk(S->mu);
            host_free(S, q->csr);
            release_ranges(S, q);
            S->direct_count++;
            S->launches++;
            finish(S, q, status[i]);
        }
        if (!direct.empty()) {  // every copy of the pass has landed before its ranges are reused
            const cudaError_t ce = cudaStreamSynchronize(S->copy_stream);
            if (ce != cudaSuccess) {
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->fatal = map_err(ce);
                }
                fail_all_resident(S, map_err(ce));
                std::lock_guard<std::mutex> lk(S->mu);
                S->stop = true;
                break;
            }
        }
        e = cudaSuccess;
        if (resident == 0) continue;
        const int par = (int)(S->round & 1);
        const int G = S->G;
        for (Request *q : admitted) {  // copy the CSR into the arenas (async from pinned staging)
            const int g = q->slot;
            S->tab_h[g] = q->vb;
            S->tab_h[G + g] = q->eb;
            S->tab_h[2 * G + g] = q->rb;
            S->nv_h[g] = q->n;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((int32_t *)S->P.ro + q->rb, q->csr.ptr, ((size_t)q->n + 1) * 4,
                                    cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && q->m > 0)
                e = cudaMemcpyAsync((int32_t *)S->P.ci + q->eb, q->csr.ptr + q->n + 1,
                                    (size_t)q->m * 4, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->vbase_d, S->tab_h, (size_t)G * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->ebase_d, S->tab_h + G, (size_t)G * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->robase_d, S->tab_h + 2 * G, (size_t)G * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->nv_d, S->nv_h, (size_t)G * 4, cudaMemcpyHostToDevice, st);
        for (Request *q : admitted)
            if (e == cudaSuccess) e = sgr::launch_admit(S->P, q->slot, q->vb, q->n, par, S->sms * 4, st);
        const int R = S->cfg.rounds_per_launch > 0 ? S->cfg.rounds_per_launch : (have_pending ? 8 : 64);
        sgr::Params P = S->P;
        P.rounds_per_launch = R;
        P.nblocks = (unsigned)S->grid;
        P.wait_ns = sgr::wait_limit_ns();
        // fresh barrier and error state for this launch
        if (e == cudaSuccess) e = cudaMemsetAsync(&P.ctr->bar, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(&P.ctr->err, 0, sizeof(int), st);
        if (e == cudaSuccess) e = sgr::launch_color(P, false, true, S->grid, st);
        if (e == cudaSuccess)
            e = sgr::launch_slot_status(P.colors, S->vbase_d, S->nv_d, G, S->rem_d, S->kmax_d, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->ctr_h, P.ctr, sizeof(sgr::Counters), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->rem_h, S->rem_d, (size_t)G * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->kmax_h, S->kmax_d, (size_t)G * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (!admitted.empty()) {  // their CSR is on the device now
            std::lock_guard<std::mutex> lk(S->mu);
            for (Request *q : admitted) host_free(S, q->csr);
        }
        const sgr::Counters h = *S->ctr_h;
        if (e != cudaSuccess || h.err != 0) {
            const int status = e != cudaSuccess ? map_err(e) : h.err;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->fatal = status;
            }
            fail_all_resident(S, status);
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
            break;
        }
        S->launches++;
        S->rounds_run += h.round - S->round;
        S->round = h.round;
        // Retire finished graphs, unless a hub's color still waits to be
        // scattered into neighbour bitmaps (its range must not be reused yet).
        // A graph with a symmetric CSR finishes within n of its rounds: in
        // every round the worklist vertex that wins against all its
        // neighbours under the rule keeps its color.  One that is still
        // unfinished after n + 1 of its rounds (a non-symmetric CSR, which
        // the submit checks do not catch) is taken off the worklists and
        // fails with SGR_ERR_NO_CONVERGENCE, as sgr_color would.
        if (h.sc64 != 0) continue;
        std::vector<Request *> stuck;
        for (int g = 0; g < G; ++g) {
            Request *q = S->slot_req[g];
            if (q && S->rem_h[g] != 0 && S->round - q->r_admit > (long long)q->n) stuck.push_back(q);
        }
        for (Request *q : stuck) {
            S->nv_h[q->slot] = 0;
            if (e == cudaSuccess) e = sgr::launch_purge(P, q->vb, q->vb + q->n, (int)(S->round & 1), st);
        }
        if (!stuck.empty()) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(S->nv_d, S->nv_h, (size_t)G * 4, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                const int status = map_err(e);
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->fatal = status;
                }
                fail_all_resident(S, status);
                std::lock_guard<std::mutex> lk(S->mu);
                S->stop = true;
                break;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            for (Request *q : stuck) {
                release_slot(S, q);
                finish(S, q, SGR_ERR_NO_CONVERGENCE);
            }
        }
        std::vector<Request *> retiring;
        for (int g = 0; g < G; ++g) {
            Request *q = S->slot_req[g];
            if (!q || S->rem_h[g] != 0) continue;
            retiring.push_back(q);
            q->k = S->kmax_h[g];
            S->nv_h[g] = 0;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                host_alloc(S, q->out, q->n);
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(q->out.ptr, P.colors + q->vb, (size_t)q->n * 4, cudaMemcpyDeviceToHost, st);
        }
        if (retiring.empty()) continue;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request *q : retiring) {
            release_slot(S, q);
            finish(S, q, e != cudaSuccess ? map_err(e) : SGR_OK);
        }
    }
}

}  // namespace

extern "C" {

int sgr_server_create(const sgr_server_config *cfg, sgr_server **out) {
    if (!cfg || !out) return SGR_ERR_INVALID_ARG;
    if ((cfg->mode & SGR_MODE_MASK) != SGR_MODE_DETERMINISTIC) return SGR_ERR_INVALID_ARG;
    if (cfg->mode & ~(SGR_MODE_MASK | SGR_RULE_MASK) || ((cfg->mode & SGR_RULE_MASK) >> 4) > 2)
        return SGR_ERR_INVALID_ARG;
    if (cfg->max_inflight < 0 || cfg->rounds_per_launch < 0 || cfg->hbm_budget_bytes < 0)
        return SGR_ERR_INVALID_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return SGR_ERR_CUDA;
    sgr_server *S = new sgr_server();
    S->cfg = *cfg;
    if (S->cfg.hbm_budget_bytes == 0) S->cfg.hbm_budget_bytes = 1ll << 30;
    if (S->cfg.staging_bytes == 0) S->cfg.staging_bytes = 1ll << 30;
    if (S->cfg.staging_bytes < 0) S->cfg.staging_bytes = 0;
    S->G = S->cfg.max_inflight > 0 ? S->cfg.max_inflight : 1024;
    S->direct_min = S->cfg.direct_min_vertices == 0 ? 262144 : S->cfg.direct_min_vertices;
    S->device = cfg->device;
    int rc = SGR_OK;
    if (cudaSetDevice(S->device) != cudaSuccess) rc = SGR_ERR_INVALID_ARG;
    if (rc == SGR_OK && cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess)
        rc = SGR_ERR_CUDA;
    if (rc == SGR_OK && sgr::occupancy_blocks_per_sm(false, true, &S->per_sm) != 0) rc = SGR_ERR_CUDA;
    if (rc == SGR_OK) {
        const sgr_tuning t = sgr::tuning_snapshot();
        if (t.blocks_per_sm > 0) S->per_sm = std::min(S->per_sm, t.blocks_per_sm);
        S->grid = S->per_sm * S->sms;
        if (S->grid < 1) rc = SGR_ERR_CUDA;
    }
    if (rc == SGR_OK && cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = SGR_ERR_CUDA;
    if (rc == SGR_OK && cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = SGR_ERR_CUDA;
    for (int i = 0; rc == SGR_OK && i < sgr_server::kDirectPass; ++i)
        if (cudaEventCreateWithFlags(&S->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->ev_done[i], cudaEventDisableTiming) != cudaSuccess)
            rc = SGR_ERR_CUDA;
    if (rc == SGR_OK) rc = carve(S);
    if (rc == SGR_OK) {
        const long long words = S->cfg.staging_bytes / 4;
        const size_t mirror = (size_t)S->G * (3 * 8 + 3 * 4) + sizeof(sgr::Counters) + 256;
        char *m = nullptr;
        if (cudaMallocHost(&m, mirror) != cudaSuccess) rc = SGR_ERR_OUT_OF_MEMORY;
        else {
            std::memset(m, 0, mirror);
            S->tab_h = (long long *)m;
            S->nv_h = (int32_t *)(m + (size_t)S->G * 24);
            S->rem_h = S->nv_h + S->G;
            S->kmax_h = S->rem_h + S->G;
            S->ctr_h = (sgr::Counters *)(((uintptr_t)(S->kmax_h + S->G) + 255) & ~(uintptr_t)255);
        }
        if (rc == SGR_OK && words > 0) {
            if (cudaMallocHost(&S->pinned, (size_t)words * 4) != cudaSuccess) rc = SGR_ERR_OUT_OF_MEMORY;
            else S->pa.init(words);
        }
    }
    if (rc == SGR_OK) {
        S->slot_req.assign(S->G, nullptr);
        for (int g = S->G - 1; g >= 0; --g) S->free_slots.push_back(g);
        S->worker = std::thread(worker_loop, S);
    }
    cudaSetDevice(prev);
    if (rc != SGR_OK) {
        if (S->dmem) cudaFree(S->dmem);
        if (S->pinned) cudaFreeHost(S->pinned);
        if (S->tab_h) cudaFreeHost(S->tab_h);
        if (S->stream) cudaStreamDestroy(S->stream);
        if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
        for (int i = 0; i < sgr_server::kDirectPass; ++i) {
            if (S->ev_in[i]) cudaEventDestroy(S->ev_in[i]);
            if (S->ev_done[i]) cudaEventDestroy(S->ev_done[i]);
        }
        delete S;
        return rc;
    }
    *out = S;
    return SGR_OK;
}

int sgr_server_submit(sgr_server *S, int32_t n, const int32_t *ro, const int32_t *ci,
                      uint64_t *req_id) {
    if (!S || !req_id || n < 0 || (n > 0 && !ro)) return SGR_ERR_INVALID_ARG;
    const long long m = n > 0 ? ro[n] : 0;
    if (n > 0 && (ro[0] != 0 || m < 0)) return SGR_ERR_INVALID_GRAPH;
    if (m > 0 && !ci) return SGR_ERR_INVALID_ARG;
    for (int32_t v = 0; v < n; ++v)
        if (ro[v + 1] < ro[v] || ro[v + 1] > m) return SGR_ERR_INVALID_GRAPH;
    if (n > S->Vcap || m > S->Ecap) return SGR_ERR_OUT_OF_MEMORY;
    Request *q = new Request();
    q->n = n;
    q->m = m;
    auto reject = [&](int status) {
        std::lock_guard<std::mutex> lk(S->mu);
        host_free(S, q->csr);
        delete q;
        return status;
    };
    if (n > 0) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            host_alloc(S, q->csr, (long long)n + 1 + m);
        }
        int32_t *hro = q->csr.ptr, *hci = q->csr.ptr + n + 1;
        std::memcpy(hro, ro, ((size_t)n + 1) * 4);
        // Copy col_idx, counting ids outside [0, n) and adjacent descending
        // pairs on the way; rows are ascending iff every descending pair sits
        // on a row boundary.  Large requests are copied and checked by a few
        // host threads at once, each over its own stretch of entries (a pair
        // across two stretches is read from the caller's array).
        long long bad = 0, desc = 0, bnd = 0;
        const uint32_t un = (uint32_t)n;
        auto copy_check = [&](long long i0, long long i1, long long *b_out, long long *d_out) {
            if (i1 > i0) std::memcpy(hci + i0, ci + i0, (size_t)(i1 - i0) * 4);
            long long b = 0, d = 0;
            for (long long i = i0; i < i1; ++i) {
                b += (uint32_t)ci[i] >= un;
                if (i + 1 < m) d += ci[i] >= ci[i + 1];
            }
            *b_out = b;
            *d_out = d;
        };
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nth = m >= (1ll << 20) ? (int)std::min(8u, std::max(1u, hw / 2)) : 1;
        if (nth == 1) {
            copy_check(0, m, &bad, &desc);
        } else {
            std::vector<long long> bs(nth, 0), ds(nth, 0);
            std::vector<std::thread> th;
            const long long per = (m + nth - 1) / nth;
            for (int t = 1; t < nth; ++t)
                th.emplace_back(copy_check, std::min(m, t * per), std::min(m, (t + 1) * per), &bs[t], &ds[t]);
            copy_check(0, std::min(m, per), &bs[0], &ds[0]);
            for (auto &x : th) x.join();
            for (int t = 0; t < nth; ++t) {
                bad += bs[t];
                desc += ds[t];
            }
        }
        if (bad) return reject(SGR_ERR_INVALID_GRAPH);
        for (int32_t v = 0; v < n; ++v) {
            const int32_t a = hro[v], b = hro[v + 1];
            if (b > a && b < m) bnd += hci[b - 1] >= hci[b];
        }
        if (desc != bnd)  // some row is not ascending: sort rows (the order within a row is free)
            for (int32_t v = 0; v < n; ++v) std::sort(hci + hro[v], hci + hro[v + 1]);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal != SGR_OK) {
        host_free(S, q->csr);
        delete q;
        return S->fatal;
    }
    q->id = S->next_id++;
    q->t_submit = Clock::now();
    if (!S->any_submit) {
        S->any_submit = true;
        S->t_first_submit = q->t_submit;
    }
    S->submitted++;
    S->reqs[q->id] = q;
    *req_id = q->id;
    if (n == 0) {
        finish(S, q, SGR_OK);
        return SGR_OK;
    }
    S->pending.push_back(q);
    S->cv_work.notify_one();
    return SGR_OK;
}

int sgr_server_poll(sgr_server *S, uint64_t req_id, int32_t *colors_host, int32_t *num_colors,
                    int timeout_ms) {
    if (!S) return SGR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return SGR_ERR_NOT_FOUND;
    Request *q = it->second;
    auto ready = [&] { return q->status != SGR_PENDING; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (timeout_ms > 0) S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (q->status == SGR_PENDING) return SGR_PENDING;
    const int status = q->status;
    if (status == SGR_OK) {
        if (colors_host && q->n) std::memcpy(colors_host, q->out.ptr, (size_t)q->n * 4);
        if (num_colors) *num_colors = q->k;
    }
    host_free(S, q->out);
    host_free(S, q->csr);
    S->reqs.erase(it);
    delete q;
    return status;
}

int sgr_server_stats(sgr_server *S, sgr_server_counters *out) {
    if (!S || !out) return SGR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->pending = (int64_t)S->pending.size();
    out->resident = S->G - (int64_t)S->free_slots.size();
    out->launches = S->launches;
    out->rounds = S->rounds_run;
    out->hbm_bytes = (int64_t)S->dbytes;
    out->vertex_capacity = S->Vcap;
    out->entry_capacity = S->Ecap;
    out->direct = S->direct_count;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * (v.size() - 1)));
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double x : v) s += x;
        out->mean_ms = s / v.size();
        const double span =
            std::chrono::duration<double>(S->t_last_done - S->t_first_submit).count();
        out->graphs_per_s = span > 0 ? S->completed / span : 0;
    }
    return S->fatal;
}

int sgr_server_destroy(sgr_server *S) {
    if (!S) return SGR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    if (S->stream) cudaStreamSynchronize(S->stream);
    if (S->copy_stream) cudaStreamSynchronize(S->copy_stream);
    if (S->dmem) cudaFree(S->dmem);
    if (S->pinned) cudaFreeHost(S->pinned);
    if (S->tab_h) cudaFreeHost(S->tab_h);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    for (int i = 0; i < sgr_server::kDirectPass; ++i) {
        if (S->ev_in[i]) cudaEventDestroy(S->ev_in[i]);
        if (S->ev_done[i]) cudaEventDestroy(S->ev_done[i]);
    }
    cudaSetDevice(prev);
    for (auto &kv : S->reqs) delete kv.second;  // their pinned ranges go with the pool
    delete S;
    return SGR_OK;
}

}  // extern "C"
