// sgr_kernels.cu -- the speculative-greedy coloring loop as one persistent
// kernel for sm_103a.
//
// One cooperative launch runs Algorithm 7 (Sect. 3.1) to completion:
//
//   init:    W_1 = V, binned by degree; colors = 0 (fast) or -1 (det: the
//            round-1 FirstFit answer is 1 for every vertex, since all frozen
//            colors are 0); strictly ascending rows are detected.
//   round r: phase A = FirstFit (Algorithm 4) over W_r,
//            grid barrier,
//            phase B = ConflictResolve (Algorithm 5) over W_r: keepers commit,
//            losers are compacted into W_{r+1} (Sect. 3.1 "Atomic Operation
//            Reduction": one atomic per CTA tile, positions from a block scan
//            that keeps the order of the tile),
//            grid barrier, swap W_in / W_out by parity (Algorithm 7's swap).
//
// The phases share one kernel with a software grid barrier: the paper's
// kernel fusion (Sect. 3.3) and its forced thread coarsening (Sect. 3.2), a
// fixed grid of co-resident CTAs looping over the worklist.  Every wait is
// bounded by %globaltimer; on expiry the kernel records SGR_ERR_TIMEOUT and
// returns.
//
// Deterministic mode (frozen reads, judge before clear):
//   * A worklist vertex holds its tentative color as a negative value in
//     `colors`; losers keep -c until their next FirstFit overwrites it.
//   * FirstFit reads a per-vertex bitmap of the final colors of its
//     neighbours (colors 1..256 in 8 bit planes of n words).  A vertex adds
//     its color to every neighbour's bitmap once, when it commits; so at the
//     start of round r the bitmap of v is exactly { F[w] : w in adj(v) } of
//     Algorithm 4 restricted to 1..256, and the first zero bit is its
//     first-fit color (Sect. 3.2 "Bitset Operation").  If bits 1..256 are all
//     set, the vertex falls back to scanning its row.
//   * ConflictResolve compares magnitudes, so a neighbour's commit (-c -> +c)
//     during the phase does not change what it sees.  With ascending rows
//     and the low-keeps rule it scans only the neighbours below v, nearest
//     first, and stops at the first conflict.
// Fast mode reads and writes colors in place while the round runs, as the
// paper's GPU code does: FirstFit gathers the live colors of all neighbours,
// ConflictResolve clears losers to 0 (Sect. 3.1 "Color Clearing").
//
// Load balance (Sect. 3.3, Merrill's thread / warp / CTA mapping): a vertex
// of degree <= light_max is handled by one lane, a vertex of degree <= chunk
// by one warp, a hub by ceil(deg / chunk) warp work items; the item that
// finishes last for a hub (completion counter) resolves it.
//
// Reads of col_idx and row_offsets use the read-only path (__ldg, Sect. 3.3
// "Read-only Data Caching") with 16-byte vector loads; everything the launch
// itself writes (colors, bitmaps, worklists, counters) is read through L2
// (__ldcg).

#include <climits>
#include <cstdint>

#include "sgr_internal.cuh"

namespace sgr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long atom_add_release64(unsigned long long *p,
                                                                 unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;"
                 : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel64(unsigned long long *p,
                                                                 unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;"
                 : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kBarErr = 1ull << 63;

// Record an error status and raise the barrier's error flag, so that every
// CTA leaves at its next barrier.
__device__ __forceinline__ void raise_error(const Params &p, int code) {
    atomicCAS(&p.ctr->err, 0, code);
    atomicOr(&p.ctr->bar, kBarErr);
}

// The CTA's copy of the hot block of Counters (see kHotBytes), taken at the
// last grid barrier or by load_hot_counters.
__device__ __forceinline__ unsigned long long *hot_words() {
    __shared__ __align__(16) unsigned long long s_hot[kHotBytes / 8];
    return s_hot;
}

__device__ __forceinline__ const Counters &hot_counters() {
    return *reinterpret_cast<const Counters *>(hot_words());
}

// Warp 0 copies the hot block (one 8-byte word per lane).
__device__ __forceinline__ void copy_hot_block(const Params &p) {
    static_assert(kHotBytes / 8 == 32, "one word per lane");
    if (threadIdx.x < 32)
        hot_words()[threadIdx.x] = __ldcg(reinterpret_cast<const unsigned long long *>(p.ctr) + threadIdx.x);
}

// Snapshot of the hot block for a launch that enters its round loop without
// a barrier (all threads call it).
__device__ __forceinline__ void load_hot_counters(const Params &p) {
    __syncthreads();
    copy_hot_block(p);
    __syncthreads();
}

// Bounded grid barrier on a monotone arrival counter: barrier number `gen`
// (per CTA, counted from 1) is passed once gen * nblocks CTAs have arrived.
// The arrival is a release and the poll an acquire, so every write the CTA
// made before the barrier is visible to every CTA after it.  On the way out
// warp 0 refreshes the CTA's snapshot of the hot counters.  Returns false
// if this CTA must stop (timeout, or an error flagged by any CTA).
__device__ bool grid_barrier(const Params &p, unsigned &gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        gen += 1;
        const unsigned long long target = (unsigned long long)gen * p.nblocks;
        unsigned long long seen = atom_add_release64(&p.ctr->bar, 1ull) + 1ull;
        int ok = 1;
        if ((seen & ~kBarErr) < target && !(seen & kBarErr)) {
            const unsigned long long t0 = globaltimer();
            for (;;) {
                seen = ld_acquire64(&p.ctr->bar);
                if ((seen & ~kBarErr) >= target || (seen & kBarErr)) break;
                __nanosleep(32);
                if (globaltimer() - t0 > p.wait_ns) {
                    raise_error(p, kErrTimeout);
                    seen |= kBarErr;
                    break;
                }
            }
        }
        if (seen & kBarErr) ok = 0;
        s_ok = ok;
    }
    if (threadIdx.x < 32) {
        __syncwarp();  // lane 0's acquire orders the other lanes' loads
        copy_hot_block(p);
    }
    __syncthreads();
    return s_ok != 0;
}

template <bool kBatched>
__device__ __forceinline__ void row_of(const Params &p, int32_t v, long long &s, long long &e,
                                       int32_t &vb) {
    if (kBatched) {
        const int g = __ldcg(p.gid + v);
        const long long eb = __ldg(p.ebase + g), vbase = __ldg(p.vbase + g);
        const long long rb = __ldg(p.robase + g) + (v - vbase);
        s = eb + __ldg(p.ro + rb);
        e = eb + __ldg(p.ro + rb + 1);
        vb = (int32_t)vbase;
    } else {
        s = __ldg(p.ro + v);
        e = __ldg(p.ro + v + 1);
        vb = 0;
    }
}

// 16-byte load of col_idx entries [4q, 4q+4); entries past m read as 0.
__device__ __forceinline__ int4 load4(const int32_t *__restrict__ ci, long long q, long long m) {
    const long long i = q << 2;
    if (i + 4 <= m) return __ldg(reinterpret_cast<const int4 *>(ci) + q);
    int4 r = make_int4(0, 0, 0, 0);
    if (i < m) r.x = __ldg(ci + i);
    if (i + 1 < m) r.y = __ldg(ci + i + 1);
    if (i + 2 < m) r.z = __ldg(ci + i + 2);
    return r;
}

__device__ __forceinline__ int elem(const int4 &x, int k) {
    return k == 0 ? x.x : (k == 1 ? x.y : (k == 2 ? x.z : x.w));
}

// Does v lose its color to neighbour w that holds the same color?
template <bool kBatched>
__device__ __forceinline__ bool loses_to(const Params &p, int32_t v, int32_t w, int32_t dv) {
    if (p.rule == 0) return w < v;
    if (p.rule == 1) return w > v;
    long long s, e;
    int32_t vb;
    row_of<kBatched>(p, w, s, e, vb);
    const int32_t dw = (int32_t)(e - s);
    return dw != dv ? dw > dv : w < v;
}

struct Acc {
    unsigned long long w = 0, d = 0, dscan = 0, next = 0, scatter = 0;
    unsigned long long kdeg = 0;  // det: degree sum of this phase's keepers
    unsigned long long slow = 0;  // det: vertices that rescanned their row
    unsigned long long keep = 0;  // det: vertices committed in this phase
    int kmax = 0;
};

__device__ __forceinline__ unsigned global_warp() {
    return (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

__device__ __forceinline__ unsigned total_warps() { return (gridDim.x * blockDim.x) >> 5; }

// The hub, medium and light lists of a phase start on different CTAs (a third
// of the grid apart), so that on short lists no warp works through items of
// all three one after the other.
__device__ __forceinline__ unsigned rot_block(int part) {
    return (blockIdx.x + (unsigned)part * (gridDim.x / 3)) % gridDim.x;
}

__device__ __forceinline__ unsigned rot_warp(int part) {
    return (rot_block(part) * blockDim.x + threadIdx.x) >> 5;
}

// A warp's slot in a CTA-major order of all warps (warp 0 of every CTA, then
// warp 1 of every CTA, ...), rotated like rot_block: consecutive batches of a
// short list land on different SMs.
__device__ __forceinline__ unsigned spread_warp(int part) {
    return (threadIdx.x >> 5) * gridDim.x + rot_block(part);
}

// Batch of worklist entries a warp takes at a time: spread a short list over
// all warps, up to 32 entries (one per lane) for long lists.
__device__ __forceinline__ unsigned warp_batch(unsigned cnt) {
    const unsigned NW = total_warps();
    const unsigned b = (cnt + NW - 1) / NW;
    return b < 1 ? 1 : (b > 32 ? 32 : b);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

// ------------------------------------------------------------ forbidden masks

// Colors wb+1 .. wb+256 of entries [a, b) (lanes lane0, lane0+stride, ...)
// into eight 32-bit words; only positive colors count.
__device__ __forceinline__ void mask256_lane(const int32_t *__restrict__ ci, long long m,
                                             const int32_t *colors, long long a, long long b,
                                             int32_t vb, int lane0, int stride, int wb,
                                             int32_t nv, unsigned (&mw)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) mw[j] = 0;
    for (long long q = (a >> 2) + lane0; (q << 2) < b; q += stride) {
        const int4 x = load4(ci, q, m);
        const long long i0 = q << 2;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = i0 + k;
            const int32_t w = vb + elem(x, k);
            if (i >= a && i < b && (unsigned)w < (unsigned)nv) {
                const int c = __ldcg(colors + w);
                const unsigned off = (unsigned)(c - wb - 1);
                if (c > 0 && off < 256u) {
                    const unsigned bit = 1u << (off & 31);
                    const unsigned wd = off >> 5;
#pragma unroll
                    for (int j = 0; j < 8; ++j) mw[j] |= (wd == (unsigned)j) ? bit : 0u;
                }
            }
        }
    }
}

__device__ __forceinline__ void warp_or8(unsigned (&mw)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) mw[j] = __reduce_or_sync(kFull, mw[j]);
}

// first zero bit of the 256-bit window, 256 if none
__device__ __forceinline__ int first_zero8(const unsigned (&mw)[8]) {
    int z = 256;
#pragma unroll
    for (int j = 7; j >= 0; --j)
        if (~mw[j]) z = j * 32 + __ffs(~mw[j]) - 1;
    return z;
}

__device__ __forceinline__ unsigned pick8(const unsigned (&mw)[8], int j) {
    unsigned r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r = (k == j) ? mw[k] : r;
    return r;
}

// Whole-row first fit by one warp over positive colors, windows of 256.
__device__ __forceinline__ int warp_first_fit(const int32_t *__restrict__ ci, long long m,
                                              const int32_t *colors, long long s, long long e,
                                              int32_t vb, int lane, int32_t nv) {
    for (int wb = 0;; wb += 256) {
        unsigned mw[8];
        mask256_lane(ci, m, colors, s, e, vb, lane, 32, wb, nv, mw);
        warp_or8(mw);
        const int z = first_zero8(mw);
        if (z < 256) return wb + z + 1;
    }
}

// ------------------------------------------------------------ compaction

// Order-preserving block compaction of kLightUnroll flags per thread: item u
// of thread (warp w, lane l) sits at tile position (w * kLightUnroll + u) * 32
// + l.  The 32 sub-tile counts are scanned by warp 0; one atomicAdd per CTA
// tile.  out == nullptr only counts the flags.
static_assert(kWarps * kLightUnroll == 32, "one scan lane per sub-tile");

// Exclusive scan of one count per lane of warp 0; lane 0 reserves the total
// at *counter (when out != nullptr) and every lane gets its absolute start.
__device__ __forceinline__ unsigned warp_reserve(unsigned c, unsigned *counter, bool take,
                                                 unsigned &total) {
    const int lane = threadIdx.x & 31;
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    total = __shfl_sync(kFull, incl, 31);
    unsigned base = 0;
    if (lane == 0 && take && total) base = atomicAdd(counter, total);
    return __shfl_sync(kFull, base, 0) + incl - c;
}

__device__ __forceinline__ void block_push(const bool (&flag)[kLightUnroll],
                                           const int32_t (&item)[kLightUnroll],
                                           unsigned *counter, int32_t *out,
                                           unsigned long long &pushed) {
    __shared__ unsigned s_pos[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned bal[kLightUnroll];
#pragma unroll
    for (int u = 0; u < kLightUnroll; ++u) {
        bal[u] = __ballot_sync(kFull, flag[u]);
        if (lane == 0) s_pos[warp * kLightUnroll + u] = __popc(bal[u]);
    }
    __syncthreads();
    if (warp == 0) {
        unsigned tot;
        const unsigned pos = warp_reserve(s_pos[lane], counter, out != nullptr, tot);
        s_pos[lane] = pos;
        if (lane == 0) pushed += tot;
    }
    __syncthreads();
    if (out) {
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u)
            if (flag[u]) out[s_pos[warp * kLightUnroll + u] + __popc(bal[u] & lanemask_lt())] = item[u];
    }
    __syncthreads();
}

// Two order-preserving block compactions in one pass (flags a go to outa,
// flags b to outb): two scans in warp 0, the two atomics issued back to back.
__device__ __forceinline__ void block_push2(const bool (&fa)[kLightUnroll], const bool (&fb)[kLightUnroll],
                                            const int32_t (&item)[kLightUnroll], unsigned *ca,
                                            int32_t *outa, unsigned *cb, int32_t *outb,
                                            unsigned long long &pushed_a) {
    __shared__ unsigned s_a[32], s_b[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned ba[kLightUnroll], bb[kLightUnroll];
#pragma unroll
    for (int u = 0; u < kLightUnroll; ++u) {
        ba[u] = __ballot_sync(kFull, fa[u]);
        bb[u] = __ballot_sync(kFull, fb[u]);
        if (lane == 0) {
            s_a[warp * kLightUnroll + u] = __popc(ba[u]);
            s_b[warp * kLightUnroll + u] = __popc(bb[u]);
        }
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned ca_l = s_a[lane], cb_l = s_b[lane];
        unsigned ia = ca_l, ib = cb_l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned x = __shfl_up_sync(kFull, ia, o), y = __shfl_up_sync(kFull, ib, o);
            if (lane >= o) {
                ia += x;
                ib += y;
            }
        }
        const unsigned ta = __shfl_sync(kFull, ia, 31), tb = __shfl_sync(kFull, ib, 31);
        unsigned oa = 0, ob = 0;
        if (lane == 0) {
            if (ta) oa = atomicAdd(ca, ta);
            if (tb) ob = atomicAdd(cb, tb);
            pushed_a += ta;
        }
        s_a[lane] = __shfl_sync(kFull, oa, 0) + ia - ca_l;
        s_b[lane] = __shfl_sync(kFull, ob, 0) + ib - cb_l;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kLightUnroll; ++u) {
        const unsigned below = lanemask_lt();
        if (fa[u]) outa[s_a[warp * kLightUnroll + u] + __popc(ba[u] & below)] = item[u];
        if (fb[u]) outb[s_b[warp * kLightUnroll + u] + __popc(bb[u] & below)] = item[u];
    }
    __syncthreads();
}

// Warp-level order-preserving push of one flag per lane (out == nullptr: count
// only).
__device__ __forceinline__ void warp_push(bool flag, int32_t item, unsigned *counter,
                                          int32_t *out, unsigned long long &pushed) {
    const unsigned bal = __ballot_sync(kFull, flag);
    if (!bal) return;
    if ((threadIdx.x & 31) == 0) pushed += (unsigned long long)__popc(bal);
    if (!out) return;
    unsigned pos = 0;
    if ((threadIdx.x & 31) == 0) pos = atomicAdd(counter, (unsigned)__popc(bal));
    pos = __shfl_sync(kFull, pos, 0);
    if (flag) out[pos + __popc(bal & lanemask_lt())] = item;
}

// Warp-level order-preserving pushes of U flags per lane into two lists at
// once: one atomic per list for all U (both issued before either result is
// used), entries in (u, lane) order.
template <int U>
__device__ __forceinline__ void warp_push2(const bool (&fa)[U], const bool (&fb)[U],
                                           const int32_t (&item)[U], unsigned *ca, int32_t *outa,
                                           unsigned *cb, int32_t *outb, unsigned long long &pushed_a) {
    const int lane = threadIdx.x & 31;
    unsigned ba[U], bb[U], ta = 0, tb = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        ba[u] = __ballot_sync(kFull, fa[u]);
        bb[u] = __ballot_sync(kFull, fb[u]);
        ta += (unsigned)__popc(ba[u]);
        tb += (unsigned)__popc(bb[u]);
    }
    unsigned oa = 0, ob = 0;
    if (lane == 0) {
        if (ta) oa = atomicAdd(ca, ta);
        if (tb) ob = atomicAdd(cb, tb);
        pushed_a += ta;
    }
    oa = __shfl_sync(kFull, oa, 0);
    ob = __shfl_sync(kFull, ob, 0);
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (fa[u]) outa[oa + __popc(ba[u] & lt)] = item[u];
        if (fb[u]) outb[ob + __popc(bb[u] & lt)] = item[u];
        oa += (unsigned)__popc(ba[u]);
        ob += (unsigned)__popc(bb[u]);
    }
}

// Position of (tile t, warp w, sub-tile u, lane l) in a light list.
__device__ __forceinline__ unsigned tile_index(unsigned t, int u) {
    return t * kLightTile + ((threadIdx.x >> 5) * kLightUnroll + u) * 32 + (threadIdx.x & 31);
}

// index of the hub entry owning chunk q: largest i with cb[i] <= q (32-ary
// search by the whole warp; cb is ascending and cb[0] == 0).
__device__ __forceinline__ unsigned hub_entry(const unsigned *cb, unsigned cnt, unsigned q) {
    const int lane = threadIdx.x & 31;
    unsigned lo = 0, hi = cnt;
    while (hi - lo > 1) {
        const unsigned step = (hi - lo + 31) / 32;
        const unsigned idx = lo + lane * step;
        const bool ok = idx < hi && __ldcg(cb + idx) <= q;
        const unsigned bal = __ballot_sync(kFull, ok);
        const int last = 31 - __clz(bal);
        lo = lo + (unsigned)last * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Work items of a hub's ConflictResolve when only the entries below it are
// read: one per chunk of them, at least one (the item that decides).
__device__ __forceinline__ unsigned lower_chunks(int lowdeg, int chunk) {
    return lowdeg > 0 ? (unsigned)((lowdeg + chunk - 1) / chunk) : 1u;
}

// Warp-aggregated reservations in two hub lists: the lanes that want in
// (each with its number of work items) get their entry k and their first
// item cb from one atomic on each list's counter (entries << 32 | items),
// both atomics issued before either result is used.  Call with the whole
// warp.
__device__ __forceinline__ void hub_list_reserve2(bool wa, unsigned ia, unsigned long long *ca,
                                                  unsigned &ka, unsigned &cba, bool wb, unsigned ib,
                                                  unsigned long long *cb, unsigned &kb, unsigned &cbb) {
    const int lane = threadIdx.x & 31;
    const unsigned ma = __ballot_sync(kFull, wa), mb = __ballot_sync(kFull, wb);
    const unsigned xa = wa ? ia : 0u, xb = wb ? ib : 0u;
    unsigned sa = xa, sb = xb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned ya = __shfl_up_sync(kFull, sa, o), yb = __shfl_up_sync(kFull, sb, o);
        if (lane >= o) {
            sa += ya;
            sb += yb;
        }
    }
    const unsigned ta = __shfl_sync(kFull, sa, 31), tb = __shfl_sync(kFull, sb, 31);
    unsigned long long oa = 0, ob = 0;
    if (lane == 0) {
        if (ma) oa = atomicAdd(ca, ((unsigned long long)__popc(ma) << 32) | ta);
        if (mb) ob = atomicAdd(cb, ((unsigned long long)__popc(mb) << 32) | tb);
    }
    oa = __shfl_sync(kFull, oa, 0);
    ob = __shfl_sync(kFull, ob, 0);
    const unsigned lt = lanemask_lt();
    ka = (unsigned)(oa >> 32) + __popc(ma & lt);
    cba = (unsigned)oa + sa - xa;
    kb = (unsigned)(ob >> 32) + __popc(mb & lt);
    cbb = (unsigned)ob + sb - xb;
}

// Append a hub slot with its chunk count to a (count << 32 | chunks) list.
__device__ __forceinline__ void hub_list_push(unsigned long long *ctr64, int32_t *slots,
                                              unsigned *cb, int32_t slot, unsigned nchunks) {
    const unsigned long long old = atomicAdd(ctr64, (1ull << 32) | (unsigned long long)nchunks);
    const unsigned k = (unsigned)(old >> 32);
    slots[k] = slot;
    cb[k] = (unsigned)old;
}

// ------------------------------------------------------------ det: list sets and the CTA push buffer

// A light / medium / hub list triple with its counters, as pushes see it:
// the unsettled lists U (kind 0) or the activation lists A (kind 1) of one
// parity.  The pointers are taken from the launch parameters where they are
// used, so that no register holds them across the round loop.
struct ListSet {
    int kind;
    int par;
};

__device__ __forceinline__ int32_t *ls_l(const Params &p, ListSet L) { return L.kind ? p.al[L.par] : p.ul[L.par]; }
__device__ __forceinline__ int32_t *ls_m(const Params &p, ListSet L) { return L.kind ? p.am[L.par] : p.um[L.par]; }
__device__ __forceinline__ int32_t *ls_h(const Params &p, ListSet L) { return L.kind ? p.ah[L.par] : p.uh[L.par]; }
__device__ __forceinline__ unsigned *ls_hcb(const Params &p, ListSet L) { return L.kind ? p.acb[L.par] : p.ucb[L.par]; }
__device__ __forceinline__ unsigned *ls_nl(const Params &p, ListSet L) {
    return L.kind ? &p.ctr->nal[L.par] : &p.ctr->nul[L.par];
}
__device__ __forceinline__ unsigned *ls_nm(const Params &p, ListSet L) {
    return L.kind ? &p.ctr->nam[L.par] : &p.ctr->num[L.par];
}
__device__ __forceinline__ unsigned long long *ls_h64(const Params &p, ListSet L) {
    return L.kind ? &p.ctr->ah64[L.par] : &p.ctr->uh64[L.par];
}
// degree sum of the pushed vertices: kept for the activation lists only
__device__ __forceinline__ unsigned long long *ls_deg(const Params &p, ListSet L) {
    return L.kind ? &p.ctr->adeg[L.par] : nullptr;
}

template <bool kBatched>
__device__ __forceinline__ long long vertex_degree(const Params &p, int32_t v) {
    long long s, e;
    int32_t vb;
    row_of<kBatched>(p, v, s, e, vb);
    return e - s;
}

// Append one vertex to its bin of L (global atomics).  The lanes of a warp
// that get here together and push to the same light or medium list share one
// atomic; hubs take one each.
template <bool kBatched>
__device__ void list_push_one(const Params &p, ListSet L, int32_t v) {
    const int32_t bin = __ldcg(p.vslot + v);
    const long long d = (L.kind || bin >= 0) ? vertex_degree<kBatched>(p, v) : 0;
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, bin < 0 ? bin : 0);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    if (bin < 0) {
        unsigned *cnt = bin == -1 ? ls_nl(p, L) : ls_nm(p, L);
        int32_t *list = bin == -1 ? ls_l(p, L) : ls_m(p, L);
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        list[base + __popc(peers & lanemask_lt())] = v;
    } else {
        hub_list_push(ls_h64(p, L), ls_h(p, L), ls_hcb(p, L), bin,
                      (unsigned)((d + p.chunk - 1) / p.chunk));
    }
    if (L.kind) {  // the first active lane adds up the others' degrees
        unsigned long long dsum = 0;
        for (unsigned m = act; m; m &= m - 1)
            dsum += __shfl_sync(act, (unsigned long long)d, __ffs(m) - 1);
        if (lane == __ffs(act) - 1) atomicAdd(ls_deg(p, L), dsum);
    }
}

// Vertices pushed by lanes on divergent paths are staged in shared memory and
// appended to their lists by the whole CTA at the end of the phase
// (flush_push): one atomic per bin and tile instead of one per vertex.  A
// full buffer falls back to list_push_one.
struct PushBuf {
    int32_t *v;
    unsigned *n;
};

__device__ __forceinline__ PushBuf push_buf() {
    __shared__ int32_t s_pv[kPushCap];
    __shared__ unsigned s_pn;
    return PushBuf{s_pv, &s_pn};
}

template <bool kBatched>
__device__ __forceinline__ void stage_push(const Params &p, ListSet L, int32_t v) {
    const PushBuf b = push_buf();
    const unsigned pos = atomicAdd(b.n, 1u);
    if (pos < (unsigned)kPushCap) b.v[pos] = v;
    else list_push_one<kBatched>(p, L, v);
}

// Bin the staged vertices by vslot and append them to L (all threads of the
// CTA; ends with the buffer empty).
template <bool kBatched>
__device__ void flush_push(const Params &p, ListSet L) {
    const PushBuf b = push_buf();
    __syncthreads();
    const unsigned cnt = min(*b.n, (unsigned)kPushCap);
    unsigned long long dsum = 0, dummy = 0;
    for (unsigned base = 0; base < cnt; base += kLightTile) {
        bool fl[kLightUnroll], fm[kLightUnroll];
        int32_t it[kLightUnroll];
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u) {
            const unsigned idx = base + tile_index(0, u);
            const bool act = idx < cnt;
            it[u] = act ? b.v[idx] : 0;
            const int32_t bin = act ? __ldcg(p.vslot + it[u]) : -3;
            fl[u] = bin == -1;
            fm[u] = bin == -2;
            if (act && (L.kind || bin >= 0)) {
                const long long d = vertex_degree<kBatched>(p, it[u]);
                dsum += (unsigned long long)d;
                if (bin >= 0)
                    hub_list_push(ls_h64(p, L), ls_h(p, L), ls_hcb(p, L), bin,
                                  (unsigned)((d + p.chunk - 1) / p.chunk));
            }
        }
        block_push2(fl, fm, it, ls_nl(p, L), ls_l(p, L), ls_nm(p, L), ls_m(p, L), dummy);
    }
    if (L.kind) {
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
        if ((threadIdx.x & 31) == 0 && dsum) atomicAdd(ls_deg(p, L), dsum);
    }
    __syncthreads();
    if (threadIdx.x == 0) *b.n = 0;
    __syncthreads();
}

// ------------------------------------------------------------ det: witness slots
//
// Five witness slots per vertex: witness[v] (slot 0) holds the neighbour that
// beat v last time, wold[v] (16 bytes) the four before it, most recent first,
// -1 where there is none.  Every slot holds -1 or a neighbour that wins
// against v under the rule, so whichever slot's vertex holds v's tentative
// color magnitude in the same round settles v's loss.  Medium vertices and
// hubs on whole worklists check and keep all five (kMulti); light vertices,
// whose rescans are short, and the rounds on the activation lists, which
// track slot 0 as the witness whose change activates a dependent, use slot 0
// only.

__device__ __forceinline__ int mag(int x) { return x < 0 ? -x : x; }

struct Wit {
    int32_t w0;  // slot 0
    int4 o;      // slots 1-4
};

__device__ __forceinline__ Wit wit_none() { return Wit{-1, make_int4(-1, -1, -1, -1)}; }

__device__ __forceinline__ Wit wit_load(const Params &p, int32_t v) {
    return Wit{__ldcg(p.witness + v), __ldcg(reinterpret_cast<const int4 *>(p.wold) + v)};
}

__device__ __forceinline__ int32_t wit_first(const Params &p, int32_t v) { return __ldcg(p.witness + v); }

__device__ __forceinline__ void wit_reset(const Params &p, int32_t v) {
    p.witness[v] = -1;
    reinterpret_cast<int4 *>(p.wold)[v] = make_int4(-1, -1, -1, -1);
}

// Make f v's latest witness.  all: keep the older ones too (w: v's slots;
// f's old slot, or else the oldest, is dropped); otherwise only slot 0.
__device__ __forceinline__ void wit_record(const Params &p, int32_t v, int32_t f, const Wit &w, bool all) {
    if (!all) {
        __stcg(p.witness + v, f);
        return;
    }
    if (f == w.w0) return;
    const int4 o = w.o;
    int4 n;
    if (f == o.x)
        n = make_int4(w.w0, o.y, o.z, o.w);
    else if (f == o.y)
        n = make_int4(w.w0, o.x, o.z, o.w);
    else if (f == o.z)
        n = make_int4(w.w0, o.x, o.y, o.w);
    else
        n = make_int4(w.w0, o.x, o.y, o.z);
    __stcg(p.witness + v, f);
    __stcg(reinterpret_cast<int4 *>(p.wold) + v, n);
}

// The first slot (0-4) of w whose vertex holds magnitude c (c >= 1), or -1;
// the five colors are loaded together.
__device__ __forceinline__ int wit_match(const Params &p, const Wit &w, int c) {
    const int c0 = w.w0 >= 0 ? __ldcg(p.colors + w.w0) : 0;
    const int c1 = w.o.x >= 0 ? __ldcg(p.colors + w.o.x) : 0;
    const int c2 = w.o.y >= 0 ? __ldcg(p.colors + w.o.y) : 0;
    const int c3 = w.o.z >= 0 ? __ldcg(p.colors + w.o.z) : 0;
    const int c4 = w.o.w >= 0 ? __ldcg(p.colors + w.o.w) : 0;
    return mag(c0) == c ? 0 : mag(c1) == c ? 1 : mag(c2) == c ? 2 : mag(c3) == c ? 3 : mag(c4) == c ? 4 : -1;
}

__device__ __forceinline__ int32_t wit_slot(const Wit &w, int q) {
    return q == 0 ? w.w0 : q == 1 ? w.o.x : q == 2 ? w.o.y : q == 3 ? w.o.z : w.o.w;
}

// During FirstFit (bitmaps fixed): does worklist vertex w pick color c
// (1..256)?  Yes iff colors 1..c-1 are all forbidden for w and c is not; the
// bitmap words up to c's are loaded together.
__device__ __forceinline__ bool picks_color(const Params &p, int32_t w, int c) {
    const int P = (c - 1) >> 5, b = (c - 1) & 31;
    unsigned pl[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) pl[j] = j <= P ? __ldcg(p.bm + (size_t)j * p.np + w) : 0u;
    bool full = true;
    unsigned x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < P) full = full && pl[j] == 0xffffffffu;
        if (j == P) x = pl[j];
    }
    const unsigned low = b ? (0xffffffffu >> (32 - b)) : 0u;  // colors below c in its word
    return full && (x & low) == low && !((x >> b) & 1u);
}

// ------------------------------------------------------------ det: FirstFit with witness split
//
// During FirstFit every bitmap is fixed, so a vertex can compute the
// tentative color of any other worklist vertex from that vertex's bitmap.  A
// vertex whose witness (the neighbour that beat it last time) is still on the
// worklist (color < 0) and gets the same tentative color has lost again: it
// goes straight onto W_{r+1}.  The others go onto the unsettled lists U_r for
// ConflictResolve.

// First-fit color from the bitmap of v given its first word; 0 if colors
// 1..256 are all forbidden.
__device__ __forceinline__ int bitmap_color(const Params &p, int32_t v, unsigned w0);

// First color whose bit is clear in the eight words of a bitmap, or 0.
__device__ __forceinline__ int first_zero_bit(const unsigned (&pl)[8]) {
    int c = 0;
#pragma unroll
    for (int j = 7; j >= 0; --j)
        if (~pl[j]) c = j * 32 + __ffs(~pl[j]);
    return c;
}

// First-fit color from planes j0.. of v's bitmap (the planes below j0 full),
// one plane a trip; 0 if colors 1..256 are all forbidden.
__device__ __forceinline__ int bitmap_color_from(const Params &p, int32_t v, int j0) {
    for (int j = j0; j < 8; ++j) {
        const unsigned wv = __ldcg(p.bm + (size_t)j * p.np + v);
        if (~wv) return j * 32 + __ffs(~wv);
    }
    return 0;
}

// During FirstFit: does worklist vertex w, whose tentative color last round
// was tw (so that colors 1 .. tw-1 are all forbidden for it) and whose first
// bitmap word is x0, pick color c (1..256)?  Planes from tw's to c's are
// loaded together, and only when c > 32.
__device__ __forceinline__ bool picks_color_after(const Params &p, int32_t w, int c, int tw, unsigned x0) {
    if (tw > c) return false;  // its color is at least tw
    const int P = (c - 1) >> 5, b = (c - 1) & 31;
    const unsigned low = b ? (0xffffffffu >> (32 - b)) : 0u;  // colors below c in its word
    if (P == 0) return (x0 & low) == low && !((x0 >> b) & 1u);
    if (~x0) return false;  // its color is at most 32
    const int P0 = max(1, (tw - 1) >> 5);
    unsigned pl[8];
#pragma unroll
    for (int j = 1; j < 8; ++j) pl[j] = (j >= P0 && j <= P) ? __ldcg(p.bm + (size_t)j * p.np + w) : 0xffffffffu;
    bool full = true;
    unsigned x = 0;
#pragma unroll
    for (int j = 1; j < 8; ++j) {
        if (j < P) full = full && pl[j] == 0xffffffffu;
        if (j == P) x = pl[j];
    }
    return full && (x & low) == low && !((x >> b) & 1u);
}

__device__ __forceinline__ int bitmap_color(const Params &p, int32_t v, unsigned w0) {
    if (~w0) return __ffs(~w0);
    for (int j = 1; j < 8; ++j) {
        const unsigned wv = __ldcg(p.bm + (size_t)j * p.np + v);
        if (~wv) return j * 32 + __ffs(~wv);
    }
    return 0;
}

// First-fit colors of U vertices per lane (v[u] active if act[u], w0[u] the
// first word of its bitmap).  A vertex whose bitmap is full (colors 1..256
// all forbidden) is resolved by a scan of its row by the whole warp.
template <bool kBatched, int U>
__device__ __forceinline__ void full_first_fit(const Params &p, const bool (&act)[U], const int32_t (&v)[U],
                                               int (&c)[U]);

template <bool kBatched, int U>
__device__ __forceinline__ void first_fit_lane(const Params &p, const bool (&act)[U],
                                               const int32_t (&v)[U], const unsigned (&w0)[U],
                                               int (&c)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) c[u] = act[u] ? bitmap_color(p, v[u], w0[u]) : 0;
    full_first_fit<kBatched, U>(p, act, v, c);
}

// Lanes whose bitmap is full (c == 0: colors 1..256 all forbidden) get their
// first-fit color from a scan of their row by the whole warp.
template <bool kBatched, int U>
__device__ __forceinline__ void full_first_fit(const Params &p, const bool (&act)[U], const int32_t (&v)[U],
                                               int (&c)[U]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        unsigned need = __ballot_sync(kFull, act[u] && c[u] == 0);
        while (need) {  // bitmap full: scan the row (colors above 256 are in use)
            const int src = __ffs(need) - 1;
            need &= need - 1;
            const int32_t x = __shfl_sync(kFull, v[u], src);
            long long s, e;
            int32_t vb;
            row_of<kBatched>(p, x, s, e, vb);
            const int cx = warp_first_fit(p.ci, p.m, p.colors, s, e, vb, lane, p.n);
            if (lane == src) c[u] = cx;
        }
    }
}

// FirstFit and witness check for U vertices per lane; returns tentative
// colors in c[] and whether each is settled.
template <bool kBatched, int U>
__device__ __forceinline__ void det_assign_lane(const Params &p, const bool (&act)[U],
                                                const int32_t (&v)[U], int (&c)[U],
                                                bool (&settled)[U]) {
    // A worklist vertex's color word holds -(its tentative color of the last
    // round), t: bitmaps only gain bits, so colors 1 .. t-1 are still all
    // forbidden, and the search starts at t's plane.  Three trips: (bitmap
    // plane 0, witness, t), then (two planes from t's, the witness's color
    // and plane 0), then the witness's planes up to c's only when c > 32.
    unsigned w0[U], ww0[U], wa[U], wb[U];
    int32_t wit[U];
    int cw[U], t[U], P[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        w0[u] = act[u] ? __ldcg(p.bm + v[u]) : 0u;
        wit[u] = act[u] ? wit_first(p, v[u]) : -1;
        t[u] = act[u] ? -__ldcg(p.colors + v[u]) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        cw[u] = wit[u] >= 0 ? __ldcg(p.colors + wit[u]) : 0;
        ww0[u] = wit[u] >= 0 ? __ldcg(p.bm + wit[u]) : 0u;
        const bool more = act[u] && !~w0[u];
        P[u] = min(6, max(1, (t[u] - 1) >> 5));
        wa[u] = more ? __ldcg(p.bm + (size_t)P[u] * p.np + v[u]) : 0xffffffffu;
        wb[u] = more ? __ldcg(p.bm + (size_t)(P[u] + 1) * p.np + v[u]) : 0xffffffffu;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (!act[u])
            c[u] = 0;
        else if (~w0[u])
            c[u] = __ffs(~w0[u]);
        else if (~wa[u])
            c[u] = P[u] * 32 + __ffs(~wa[u]);
        else if (~wb[u])
            c[u] = (P[u] + 1) * 32 + __ffs(~wb[u]);
        else
            c[u] = bitmap_color_from(p, v[u], P[u] + 2);
    }
    full_first_fit<kBatched, U>(p, act, v, c);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        settled[u] = act[u] && wit[u] >= 0 && cw[u] < 0 && c[u] >= 1 && c[u] <= 256 &&
                     picks_color_after(p, wit[u], c[u], -cw[u], ww0[u]);
        if (act[u]) __stcg(p.colors + v[u], -c[u]);
    }
}

// Light list: CTA tiles, order-preserving pushes of the settled to W_{r+1}
// and of the rest to U_r.
template <bool kBatched>
__device__ void det_assign_light(const Params &p, int par, unsigned cnt, Acc &acc) {
    const int pn = par ^ 1;
    const int32_t *list = p.lw[par];
    const unsigned tiles = (cnt + kLightTile - 1) / kLightTile;
    for (unsigned t = rot_block(2); t < tiles; t += gridDim.x) {
        bool act[kLightUnroll], settled[kLightUnroll], open[kLightUnroll];
        int32_t v[kLightUnroll];
        int c[kLightUnroll];
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u) {
            const unsigned idx = tile_index(t, u);
            act[u] = idx < cnt;
            v[u] = act[u] ? __ldcg(list + idx) : 0;
        }
        det_assign_lane<kBatched, kLightUnroll>(p, act, v, c, settled);
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u) open[u] = act[u] && !settled[u];
        block_push2(settled, open, v, &p.ctr->nl[pn], p.lw[pn], &p.ctr->nul[par], p.ul[par],
                    acc.next);
    }
}

// Medium list: warp chunks of 128 entries, warp-level pushes.
template <bool kBatched>
__device__ void det_assign_medium(const Params &p, int par, unsigned cnt, Acc &acc) {
    constexpr int U = 4;
    const int pn = par ^ 1;
    const int32_t *list = p.mw[par];
    const unsigned NW = total_warps();
    for (unsigned base = spread_warp(1) * 32 * U; base < cnt; base += NW * 32 * U) {
        bool act[U], settled[U];
        int32_t v[U];
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned idx = base + u * 32 + (threadIdx.x & 31);
            act[u] = idx < cnt;
            v[u] = act[u] ? __ldcg(list + idx) : 0;
        }
        det_assign_lane<kBatched, U>(p, act, v, c, settled);
        bool open[U];
#pragma unroll
        for (int u = 0; u < U; ++u) open[u] = act[u] && !settled[u];
        warp_push2<U>(settled, open, v, &p.ctr->nm[pn], p.mw[pn], &p.ctr->num[par], p.um[par], acc.next);
    }
}

// Hub list: one lane per entry (entries are slots; chunk counts come from
// the chunk bases).  With ascending rows and lower ids keeping, an unsettled
// hub's ConflictResolve reads only the entries below it, one work item per
// chunk of them, nearest chunk first; when the launch has room for them
// (p.urec), each item gets a 32-byte record {v, slot, c, vb | start, length,
// items of the hub}, so that ConflictResolve starts scanning after one load.
template <bool kBatched>
__device__ void det_assign_hubs(const Params &p, int par, unsigned long long h64, bool prefix, int kmax,
                                Acc &acc) {
    const int pn = par ^ 1;
    const unsigned cnt = (unsigned)(h64 >> 32), nch = (unsigned)h64;
    const unsigned NW = total_warps();
    const bool records = prefix && p.urec[par] != nullptr;
    // at least four hubs a warp (fewer list atomics), more on long lists, in
    // CTA-major warp order (the hubs' scattered loads spread over the SMs)
    const unsigned B = max(4u, warp_batch(cnt));
    for (unsigned base = spread_warp(0) * B; base < cnt; base += NW * B) {
        const unsigned idx = base + (threadIdx.x & 31);
        bool act[1] = {(threadIdx.x & 31) < B && idx < cnt}, settled[1];
        int32_t slot = act[0] ? __ldcg(p.hw[par] + idx) : 0;
        // the entry's chunk range, loaded with the slot (not after the stores below)
        const unsigned cb0 = act[0] ? __ldcg(p.hcb[par] + idx) : 0u;
        const unsigned cb1 = act[0] ? (idx + 1 < cnt ? __ldcg(p.hcb[par] + idx + 1) : nch) : 0u;
        int32_t v[1] = {act[0] ? __ldcg(p.hvert + slot) : 0};
        long long rs = 0, re = 0;
        int32_t vb = 0;
        int ld = 0;
        if (act[0] && prefix) {  // issued before the bitmap chain
            row_of<kBatched>(p, v[0], rs, re, vb);
            ld = __ldcg(p.lowdeg + v[0]);
        }
        const Wit wv = act[0] ? wit_load(p, v[0]) : wit_none();
        // FirstFit from the hub's whole bitmap (its words in one trip; words
        // above the largest committed color are clear and not read)
        unsigned pv[8];
        const int pmax = p.resume ? 7 : min(7, kmax >> 5);
#pragma unroll
        for (int j = 0; j < 8; ++j) pv[j] = (act[0] && j <= pmax) ? __ldcg(p.bm + (size_t)j * p.np + v[0]) : 0u;
        int c[1] = {act[0] ? first_zero_bit(pv) : 0};
        full_first_fit<kBatched, 1>(p, act, v, c);
        if (act[0]) __stcg(p.colors + v[0], -c[0]);
        // the witness slots, latest first: does one of them, still on the
        // worklist, pick c too?  Their colors and their words of c's plane in
        // one trip; a slot's color word holds -(its last tentative color) t,
        // and colors below t are all forbidden for it, so the word decides
        // when t is in c's plane (else its planes up to c's, one more trip).
        // A hub a slot settles needs no work items.
        settled[0] = false;
        if (act[0] && c[0] >= 1 && c[0] <= 256) {
            const int P = (c[0] - 1) >> 5, b = (c[0] - 1) & 31;
            const unsigned low = b ? (0xffffffffu >> (32 - b)) : 0u;  // colors below c in its word
            const int32_t q[5] = {wv.w0, wv.o.x, wv.o.y, wv.o.z, wv.o.w};
            int cq[5];
            unsigned xq[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                cq[k] = q[k] >= 0 ? __ldcg(p.colors + q[k]) : 0;
                xq[k] = q[k] >= 0 ? __ldcg(p.bm + (size_t)P * p.np + q[k]) : 0xffffffffu;
            }
            int hit = -1;
#pragma unroll
            for (int k = 4; k >= 0; --k) {
                const int t = -cq[k];
                bool pk = false;
                if (cq[k] < 0 && t <= c[0]) {
                    pk = ((t - 1) >> 5) == P ? ((xq[k] & low) == low && !((xq[k] >> b) & 1u))
                                             : picks_color(p, q[k], c[0]);
                }
                if (pk) hit = k;
            }
            if (hit >= 0) {
                settled[0] = true;
                if (hit > 0) wit_record(p, v[0], q[hit], wv, true);
            }
        }
        unsigned nchunks = 0, nu = 0;
        if (act[0]) {
            nchunks = cb1 - cb0;
            nu = prefix ? lower_chunks(ld, p.chunk) : nchunks;
        }
        // settled hubs onto W_{r+1}'s hub list, the others onto U_r's, one
        // atomic per warp and list
        const bool ps = act[0] && settled[0], pu = act[0] && !settled[0];
        unsigned ks, cbs, k, cbu;
        hub_list_reserve2(ps, nchunks, &p.ctr->h64[pn], ks, cbs, pu, nu, &p.ctr->uh64[par], k, cbu);
        if (ps) {
            p.hw[pn][ks] = slot;
            p.hcb[pn][ks] = cbs;
            acc.next += 1;
        }
        if (pu) {
            p.uh[par][k] = slot;
            p.ucb[par][k] = cbu;
            if (records) {
                const long long split = rs + ld;
                uint4 *rec = reinterpret_cast<uint4 *>(p.urec[par]) + 2 * (size_t)cbu;
                for (unsigned t = 0; t < nu; ++t) {  // item t: the t-th chunk below the split
                    const long long hi = split - (long long)t * p.chunk;
                    const long long lo = max(rs, hi - (long long)p.chunk);
                    __stcg(rec + 2 * t, make_uint4((unsigned)v[0], (unsigned)slot, (unsigned)c[0], (unsigned)vb));
                    __stcg(rec + 2 * t + 1, make_uint4((unsigned)(unsigned long long)lo,
                                                       (unsigned)((unsigned long long)lo >> 32),
                                                       (unsigned)max(0ll, hi - lo), nu));
                }
            }
        }
    }
}

// ------------------------------------------------------------ det: rounds on the activation lists
//
// A worklist vertex keeps its tentative color and its loss from round to
// round unless a commit touches it: its first-fit color changes only when a
// neighbour commits that very color (the commit then puts it on an
// activation list A_{r+1}), and its loss only when its witness changes color
// or commits.  Once few vertices are touched per round, phase A FirstFits
// only A_r and hands ConflictResolve A_r plus the vertices whose witness is
// in A_r (its dependents); every other worklist vertex is left as it is,
// since it would compute the same color and lose to the same witness again.
// Results are those of the full round.

// Dependents of y among entries [a, b) of its row (one lane; 16 entries per
// step with every load of the step in flight): worklist vertices whose
// witness is y and that are not on A_r themselves.
template <bool kBatched>
__device__ __forceinline__ void push_dependents_lane(const Params &p, int32_t y, long long a,
                                                     long long b, int32_t vb, int r,
                                                     ListSet L) {
    for (long long q0 = a >> 2; (q0 << 2) < b; q0 += 4) {
        int4 x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            x[k] = ((q0 + k) << 2) < b ? load4(p.ci, q0 + k, p.m) : make_int4(0, 0, 0, 0);
        int32_t z[4][4], wz[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long i = ((q0 + k) << 2) + j;
                z[k][j] = vb + elem(x[k], j);
                const bool ok = i >= a && i < b && (unsigned)z[k][j] < (unsigned)p.n;
                wz[k][j] = ok ? wit_first(p, z[k][j]) : -1;
            }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (wz[k][j] == y && __ldcg(p.colors + z[k][j]) < 0 &&
                    __ldcg(p.astamp + z[k][j]) != r)
                    stage_push<kBatched>(p, L, z[k][j]);
    }
}

// The same over entries [a, b) by the whole warp (one 16-byte block per lane
// and step).
template <bool kBatched>
__device__ __forceinline__ void push_dependents_warp(const Params &p, int32_t y, long long a,
                                                     long long b, int32_t vb, int r,
                                                     ListSet L) {
    for (long long q = (a >> 2) + (threadIdx.x & 31); (q << 2) < b; q += 32) {
        const int4 x = load4(p.ci, q, p.m);
        int32_t z[4], wz[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = (q << 2) + k;
            z[k] = vb + elem(x, k);
            const bool ok = i >= a && i < b && (unsigned)z[k] < (unsigned)p.n;
            wz[k] = ok ? wit_first(p, z[k]) : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (wz[k] == y && __ldcg(p.colors + z[k]) < 0 && __ldcg(p.astamp + z[k]) != r)
                stage_push<kBatched>(p, L, z[k]);
    }
}

// A_r light vertices, one per lane: FirstFit, then the vertex and its
// dependents go to ConflictResolve (staged for L = U_r).  With ascending rows
// and the low-keeps rule a dependent of y is above y, so only the entries
// above y are read.
template <bool kBatched>
__device__ void front_assign_light(const Params &p, int par, unsigned cnt, int r, bool prefix,
                                   ListSet L) {
    const int32_t *list = p.al[par];
    const unsigned NW = total_warps();
    for (unsigned base = rot_warp(2) * 32; base < cnt; base += NW * 32) {
        const unsigned idx = base + (threadIdx.x & 31);
        const bool act[1] = {idx < cnt};
        const int32_t v[1] = {act[0] ? __ldcg(list + idx) : 0};
        const unsigned w0[1] = {act[0] ? __ldcg(p.bm + v[0]) : 0u};
        long long s = 0, e = 0;
        int32_t vb = 0;
        int ld = 0;
        if (act[0]) {
            row_of<kBatched>(p, v[0], s, e, vb);
            if (prefix) ld = __ldcg(p.lowdeg + v[0]);
        }
        int c[1];
        first_fit_lane<kBatched, 1>(p, act, v, w0, c);
        if (act[0]) {
            __stcg(p.colors + v[0], -c[0]);
            stage_push<kBatched>(p, L, v[0]);
            push_dependents_lane<kBatched>(p, v[0], s + ld, e, vb, r, L);
        }
    }
}

// A_r medium vertices: FirstFit one per lane, dependents by the whole warp.
template <bool kBatched>
__device__ void front_assign_medium(const Params &p, int par, unsigned cnt, int r, bool prefix,
                                    ListSet L) {
    const int lane = threadIdx.x & 31;
    const int32_t *list = p.am[par];
    const unsigned NW = total_warps(), B = warp_batch(cnt);
    for (unsigned b0 = rot_warp(1) * B; b0 < cnt; b0 += NW * B) {
        const int nb = (int)min(B, cnt - b0);
        const bool act[1] = {lane < nb};
        const int32_t v[1] = {act[0] ? __ldcg(list + b0 + lane) : 0};
        const unsigned w0[1] = {act[0] ? __ldcg(p.bm + v[0]) : 0u};
        long long sl = 0, el = 0;
        int32_t vbl = 0;
        int ld = 0;
        if (act[0]) {
            row_of<kBatched>(p, v[0], sl, el, vbl);
            if (prefix) ld = __ldcg(p.lowdeg + v[0]);
        }
        int c[1];
        first_fit_lane<kBatched, 1>(p, act, v, w0, c);
        if (act[0]) {
            __stcg(p.colors + v[0], -c[0]);
            stage_push<kBatched>(p, L, v[0]);
        }
        for (int j = 0; j < nb; ++j) {
            const int32_t y = __shfl_sync(kFull, v[0], j), vb = __shfl_sync(kFull, vbl, j);
            const long long a = __shfl_sync(kFull, sl, j) + __shfl_sync(kFull, ld, j);
            const long long e = __shfl_sync(kFull, el, j);
            push_dependents_warp<kBatched>(p, y, a, e, vb, r, L);
        }
    }
}

// A_r hubs: warp items of `chunk` row entries; item 0 also FirstFits the hub.
template <bool kBatched>
__device__ void front_assign_hubs(const Params &p, int par, unsigned long long h64, int r,
                                  bool prefix, ListSet L) {
    const int lane = threadIdx.x & 31;
    const unsigned cnt = (unsigned)(h64 >> 32), nch = (unsigned)h64;
    const long long CH = p.chunk;
    const unsigned NW = total_warps();
    for (unsigned q = global_warp(); q < nch; q += NW) {
        const unsigned i = hub_entry(p.acb[par], cnt, q);
        const int32_t slot = __ldcg(p.ah[par] + i);
        const unsigned j = q - __ldcg(p.acb[par] + i);
        const int32_t v = __ldcg(p.hvert + slot);
        long long s, e;
        int32_t vb;
        row_of<kBatched>(p, v, s, e, vb);
        if (j == 0) {
            const bool act[1] = {lane == 0};
            const int32_t vv[1] = {v};
            const unsigned w0[1] = {lane == 0 ? __ldcg(p.bm + v) : 0u};
            int c[1];
            first_fit_lane<kBatched, 1>(p, act, vv, w0, c);
            if (lane == 0) {
                __stcg(p.colors + v, -c[0]);
                stage_push<kBatched>(p, L, v);
            }
        }
        const long long lo = prefix ? s + __ldcg(p.lowdeg + v) : s;
        const long long a = max(lo, s + (long long)j * CH), b = min(e, s + (long long)(j + 1) * CH);
        if (a < b) push_dependents_warp<kBatched>(p, v, a, b, vb, r, L);
    }
}

// ------------------------------------------------------------ det: ConflictResolve
//
// v (tentative color c) loses iff a neighbour w that wins against it under
// the rule holds the same color magnitude.  A matching magnitude can only be
// a same-round worklist vertex: every final color of a neighbour was avoided
// by v's FirstFit.  So the neighbour that beat v in an earlier round (its
// witness) settles a repeat loss with one read; otherwise v scans its row.

// Lane-level scan of v's row for a conflict; returns the conflicting
// neighbour or -1.  hi >= 0: entries [s, hi) are all below v (ascending row,
// low-keeps rule) and are scanned from the top down; hi < 0: entries [s, e)
// are scanned in order under the loser rule.
template <bool kBatched>
__device__ __forceinline__ int32_t det_scan_lane(const Params &p, int32_t v, int c, int32_t dv,
                                                 long long s, long long e, int32_t vb,
                                                 long long hi, unsigned long long &scanned) {
    if (hi >= 0) {
        for (long long q = (hi - 1) >> 2; hi > s && q >= (s >> 2); --q) {
            const int4 x = load4(p.ci, q, p.m);
            const long long i0 = q << 2;
            int cw[4];
            int32_t ww[4];
            bool ok[4];
#pragma unroll
            for (int k = 3; k >= 0; --k) {
                const long long i = i0 + k;
                ww[k] = vb + elem(x, k);
                ok[k] = i >= s && i < hi && (unsigned)ww[k] < (unsigned)p.n;
                cw[k] = ok[k] ? __ldcg(p.colors + ww[k]) : 0;
            }
#pragma unroll
            for (int k = 3; k >= 0; --k) {
                if (!ok[k]) continue;
                scanned++;
                if (mag(cw[k]) == c) return ww[k];
            }
        }
        return -1;
    }
    for (long long q = s >> 2; (q << 2) < e; ++q) {
        const int4 x = load4(p.ci, q, p.m);
        const long long i0 = q << 2;
        int cw[4];
        int32_t ww[4];
        bool ok[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = i0 + k;
            ww[k] = vb + elem(x, k);
            ok[k] = i >= s && i < e && (unsigned)ww[k] < (unsigned)p.n && ww[k] != v;
            if (p.rule == 0 && ww[k] > v) ok[k] = false;
            if (p.rule == 1 && ww[k] < v) ok[k] = false;
            cw[k] = ok[k] ? __ldcg(p.colors + ww[k]) : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!ok[k]) continue;
            scanned++;
            if (mag(cw[k]) == c && loses_to<kBatched>(p, v, ww[k], dv)) return ww[k];
        }
    }
    return -1;
}

// A commit of color c reaches worklist neighbour w: if w holds tentative
// color c its first-fit color changes, so w goes onto the activation list of
// round act_r (once, whichever commit gets there first).
template <bool kBatched>
__device__ __forceinline__ void activate(const Params &p, int32_t w, int cw, int c, int act_r,
                                         ListSet A) {
    if (cw == -c && atomicMax(p.astamp + w, act_r) < act_r) stage_push<kBatched>(p, A, w);
}

// Record final color c in the bitmaps of the neighbours [a, b) (lanes lane0,
// lane0 + stride, ... over 16-byte blocks; kDeep: four blocks a lane with all
// their loads in flight before any atomic, for the whole-list rounds, whose
// kernel has the registers for it).  Colors above 256 are not recorded;
// FirstFit then falls back to a scan.  act_r > 0: also activate the
// neighbours that hold tentative color c.
template <bool kBatched, bool kDeep = false>
__device__ __forceinline__ void scatter_color(const Params &p, int c, long long a, long long b,
                                              int32_t vb, int lane0, int stride, int act_r,
                                              ListSet A) {
    const bool bits = c <= 256;
    if (!bits && !act_r) return;
    unsigned *plane = p.bm + (size_t)((c - 1) >> 5) * p.np;
    const unsigned bit = 1u << ((c - 1) & 31);
    if constexpr (kDeep) {
        for (long long q0 = (a >> 2) + lane0; (q0 << 2) < b; q0 += 4 * (long long)stride) {
            int4 x[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const long long q = q0 + (long long)t * stride;
                x[t] = (q << 2) < b ? load4(p.ci, q, p.m) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const long long i0 = (q0 + (long long)t * stride) << 2;
                int32_t w[4];
                bool ok[4];
                int cw[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long i = i0 + k;
                    w[k] = vb + elem(x[t], k);
                    ok[k] = i >= a && i < b && (unsigned)w[k] < (unsigned)p.n;
                    cw[k] = (act_r && ok[k]) ? __ldcg(p.colors + w[k]) : 0;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (!ok[k]) continue;
                    if (bits) atomicOr(plane + w[k], bit);
                    if (act_r) activate<kBatched>(p, w[k], cw[k], c, act_r, A);
                }
            }
        }
    } else {
        for (long long q = (a >> 2) + lane0; (q << 2) < b; q += stride) {
            const int4 x = load4(p.ci, q, p.m);
            const long long i0 = q << 2;
            int32_t w[4];
            bool ok[4];
            int cw[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long i = i0 + k;
                w[k] = vb + elem(x, k);
                ok[k] = i >= a && i < b && (unsigned)w[k] < (unsigned)p.n;
                cw[k] = (act_r && ok[k]) ? __ldcg(p.colors + w[k]) : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!ok[k]) continue;
                if (bits) atomicOr(plane + w[k], bit);
                if (act_r) activate<kBatched>(p, w[k], cw[k], c, act_r, A);
            }
        }
    }
}

// Backward scan of entries [s, hi) of v's ascending row (all below v), three
// 16-byte blocks at a time with every load of a batch in flight before the
// checks; returns the nearest neighbour holding magnitude c, or -1.
__device__ __forceinline__ int32_t scan_below(const Params &p, int c, long long s, long long hi,
                                              int32_t vb, unsigned long long &scanned) {
    for (long long qt = (hi - 1) >> 2; hi > s && qt >= (s >> 2); qt -= 3) {
        int4 x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            x[k] = qt - k >= (s >> 2) ? load4(p.ci, qt - k, p.m) : make_int4(0, 0, 0, 0);
        int cw[3][4];
        bool ok[3][4];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long i = ((qt - k) << 2) + j;
                const int32_t w = vb + elem(x[k], j);
                ok[k][j] = qt - k >= (s >> 2) && i >= s && i < hi && (unsigned)w < (unsigned)p.n;
                cw[k][j] = ok[k][j] ? __ldcg(p.colors + w) : 0;
            }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 3; j >= 0; --j) {
                if (!ok[k][j]) continue;
                scanned++;
                if (mag(cw[k][j]) == c) return vb + elem(x[k], j);
            }
    }
    return -1;
}

// Record color c in the bitmaps of the neighbours [s, e) (one lane; three
// 16-byte blocks loaded per batch); act_r > 0 also activates (see activate).
template <bool kBatched>
__device__ __forceinline__ void scatter_lane(const Params &p, int c, long long s, long long e,
                                             int32_t vb, int act_r, ListSet A) {
    const bool bits = c <= 256;
    if ((!bits && !act_r) || e <= s) return;
    unsigned *plane = p.bm + (size_t)((c - 1) >> 5) * p.np;
    const unsigned bit = 1u << ((c - 1) & 31);
    const long long q1 = (e + 3) >> 2;
    for (long long q0 = s >> 2; q0 < q1; q0 += 3) {
        int4 x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = q0 + k < q1 ? load4(p.ci, q0 + k, p.m) : make_int4(0, 0, 0, 0);
        int32_t w[3][4];
        bool ok[3][4];
        int cw[3][4];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long i = ((q0 + k) << 2) + j;
                w[k][j] = vb + elem(x[k], j);
                ok[k][j] = i >= s && i < e && (unsigned)w[k][j] < (unsigned)p.n;
                cw[k][j] = (act_r && ok[k][j]) ? __ldcg(p.colors + w[k][j]) : 0;
            }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!ok[k][j]) continue;
                if (bits) atomicOr(plane + w[k][j], bit);
                if (act_r) activate<kBatched>(p, w[k][j], cw[k][j], c, act_r, A);
            }
    }
}

// Resolve a vertex the witness did not settle (one lane): scan its row,
// record a new witness or commit and scatter.  Returns true for a loser.
template <bool kBatched>
__device__ __forceinline__ bool det_resolve_slow(const Params &p, bool slow, int32_t v, int c,
                                                 bool prefix, int act_r, ListSet A,
                                                 Acc &acc) {
    if (!slow) return false;
    acc.slow++;
    long long s, e;
    int32_t vb;
    row_of<kBatched>(p, v, s, e, vb);
    const int32_t found =
        prefix ? scan_below(p, c, s, s + __ldcg(p.lowdeg + v), vb, acc.dscan)
               : det_scan_lane<kBatched>(p, v, c, (int32_t)(e - s), s, e, vb, -1, acc.dscan);
    if (found >= 0) {
        __stcg(p.witness + v, found);  // light rows keep slot 0 only
        return true;
    }
    __stcg(p.colors + v, c);
    acc.kmax = max(acc.kmax, c);
    acc.keep++;
    acc.kdeg += (unsigned long long)(e - s);
    acc.scatter += (unsigned long long)(e - s);
    scatter_lane<kBatched>(p, c, s, e, vb, act_r, A);
    return false;
}

// Fast path for U light worklist vertices per lane (list positions idx[u]),
// stage by stage for all U: entry, then witness and own color, then the
// witness's color.  In round 1 with ascending rows and the low-keeps rule
// every tentative color is 1, so v loses iff it has a lower neighbour, and
// its nearest lower neighbour becomes its witness.  flag: settled loser;
// slow: not settled here (v and c returned for the slow path).
template <bool kBatched, int U>
__device__ __forceinline__ void det_light_fast(const Params &p, const int32_t *list, unsigned cnt,
                                               const unsigned (&idx)[U], bool prefix, bool round1,
                                               bool (&flag)[U], bool (&slow)[U],
                                               int32_t (&v)[U], int32_t (&c)[U]) {
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        act[u] = idx[u] < cnt;
        v[u] = act[u] ? __ldcg(list + idx[u]) : 0;
    }
    if (round1 && prefix) {
        int ld[U];
        long long s[U];
        int32_t vb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ld[u] = 0;
            s[u] = 0;
            vb[u] = 0;
            c[u] = 1;
            if (act[u]) {
                long long e;
                row_of<kBatched>(p, v[u], s[u], e, vb[u]);
                ld[u] = __ldcg(p.lowdeg + v[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            flag[u] = act[u] && ld[u] > 0;
            slow[u] = act[u] && ld[u] == 0;
            if (flag[u]) __stcg(p.witness + v[u], vb[u] + __ldg(p.ci + s[u] + ld[u] - 1));
        }
        return;
    }
    int32_t wit[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        wit[u] = act[u] ? wit_first(p, v[u]) : -1;
        c[u] = act[u] ? -__ldcg(p.colors + v[u]) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int cw = wit[u] >= 0 ? __ldcg(p.colors + wit[u]) : 0;
        flag[u] = act[u] && wit[u] >= 0 && mag(cw) == c[u];
        slow[u] = act[u] && !flag[u];
    }
}

template <bool kBatched>
__device__ void det_light_detect(const Params &p, const int32_t *list, unsigned cnt, int32_t *out,
                                 unsigned *out_cnt, bool prefix, bool round1, int act_r,
                                 ListSet A, Acc &acc) {
    if (cnt < 2u * gridDim.x * kLightTile) {
        // short worklist: 32 entries per warp, spread over every warp of the grid
        const unsigned NW = total_warps();
        for (unsigned base = rot_warp(2) * 32; base < cnt; base += NW * 32) {
            const unsigned idx[1] = {base + (threadIdx.x & 31)};
            bool flag[1], slow[1];
            int32_t v[1], c[1];
            det_light_fast<kBatched, 1>(p, list, cnt, idx, prefix, round1, flag, slow, v, c);
            bool lost = flag[0];
            if (__any_sync(kFull, slow[0]))
                lost = det_resolve_slow<kBatched>(p, slow[0], v[0], c[0], prefix, act_r, A, acc) ||
                       lost;
            warp_push(lost, v[0], out_cnt, out, acc.next);
        }
        return;
    }
    // long worklist: CTA tiles; the vertices the witness does not settle are
    // queued in shared memory and resolved by all warps of the CTA together.
    __shared__ int32_t s_sv[kSlowCap], s_sc[kSlowCap];
    __shared__ unsigned s_sn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_sn = 0;
    __syncthreads();
    const unsigned tiles = (cnt + kLightTile - 1) / kLightTile;
    for (unsigned t = rot_block(2);; t += gridDim.x) {
        const bool more = t < tiles;
        if (more) {
            bool flag[kLightUnroll], slow[kLightUnroll];
            int32_t v[kLightUnroll], c[kLightUnroll];
            unsigned idx[kLightUnroll];
#pragma unroll
            for (int u = 0; u < kLightUnroll; ++u) idx[u] = tile_index(t, u);
            det_light_fast<kBatched, kLightUnroll>(p, list, cnt, idx, prefix, round1, flag, slow, v, c);
#pragma unroll
            for (int u = 0; u < kLightUnroll; ++u) {
                const unsigned bal = __ballot_sync(kFull, slow[u]);
                if (!bal) continue;
                unsigned pos = 0;
                if (lane == 0) pos = atomicAdd(&s_sn, (unsigned)__popc(bal));
                pos = __shfl_sync(kFull, pos, 0) + __popc(bal & lanemask_lt());
                if (slow[u]) {
                    s_sv[pos] = v[u];
                    s_sc[pos] = c[u];
                }
            }
            block_push(flag, v, out_cnt, out, acc.next);
        }
        __syncthreads();
        const unsigned nslow = s_sn;
        if (nslow > kSlowCap - kLightTile || (!more && nslow > 0)) {  // drain the queue
            for (unsigned g = warp * 32; g < nslow; g += kWarps * 32) {
                const bool sl = g + lane < nslow;
                const int32_t v = sl ? s_sv[g + lane] : 0;
                const int c = sl ? s_sc[g + lane] : 0;
                const bool lost = det_resolve_slow<kBatched>(p, sl, v, c, prefix, act_r, A, acc);
                warp_push(lost, v, out_cnt, out, acc.next);
            }
            __syncthreads();
            if (threadIdx.x == 0) s_sn = 0;
            __syncthreads();
        }
        if (!more) break;
    }
}

// Warp-wide det scan of entries [a, b) of v's row (s = row start); returns
// the conflicting neighbour or -1.  prefix: entries below v, [a, min(b,
// split)), 128 per step from the top down (kPipe: each step's blocks loaded
// during the step before, for the whole-list rounds); `stop` (may be null) is
// polled between steps.
template <bool kBatched, bool kPipe = false>
__device__ __forceinline__ int32_t det_scan_warp(const Params &p, int32_t v, int c, int32_t dv,
                                                 long long s, long long a, long long b, int32_t vb,
                                                 bool prefix, const unsigned *stop,
                                                 unsigned long long &scanned) {
    const int lane = threadIdx.x & 31;
    if (prefix) {
        const long long split = s + __ldcg(p.lowdeg + v);
        const long long hi = min(b, split);
        if (hi <= a) return -1;
        if constexpr (kPipe) {
            const long long qa = a >> 2;
            long long top = (hi - 1) >> 2, q = top - lane;
            int4 x = q >= qa ? load4(p.ci, q, p.m) : make_int4(0, 0, 0, 0);
            for (;;) {  // the next step's blocks are loaded before this step's gathers
                const bool more = top - 32 >= qa;
                const long long nq = q - 32;
                const int4 nx = (more && nq >= qa) ? load4(p.ci, nq, p.m) : make_int4(0, 0, 0, 0);
                int32_t my = -1;
                if (q >= qa) {
                    const long long i0 = q << 2;
                    int cw[4];
                    bool ok[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const long long i = i0 + k;
                        const int32_t w = vb + elem(x, k);
                        ok[k] = i >= a && i < hi && (unsigned)w < (unsigned)p.n;
                        cw[k] = ok[k] ? __ldcg(p.colors + w) : 0;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (!ok[k]) continue;
                        scanned++;
                        if (mag(cw[k]) == c) my = vb + elem(x, k);
                    }
                }
                const unsigned bal = __ballot_sync(kFull, my >= 0);
                if (bal) return __shfl_sync(kFull, my, __ffs(bal) - 1);
                if ((stop && __ldcg(stop)) || !more) return -1;
                top -= 32;
                q = nq;
                x = nx;
            }
        } else {
            for (long long top = (hi - 1) >> 2; top >= (a >> 2); top -= 32) {
                const long long q = top - lane;
                int32_t my = -1;
                if (q >= (a >> 2)) {
                    const int4 x = load4(p.ci, q, p.m);
                    const long long i0 = q << 2;
                    int cw[4];
                    bool ok[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const long long i = i0 + k;
                        const int32_t w = vb + elem(x, k);
                        ok[k] = i >= a && i < hi && (unsigned)w < (unsigned)p.n;
                        cw[k] = ok[k] ? __ldcg(p.colors + w) : 0;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (!ok[k]) continue;
                        scanned++;
                        if (mag(cw[k]) == c) my = vb + elem(x, k);
                    }
                }
                const unsigned bal = __ballot_sync(kFull, my >= 0);
                if (bal) return __shfl_sync(kFull, my, __ffs(bal) - 1);
                if (stop && __ldcg(stop)) return -1;
            }
            return -1;
        }
    }
    for (long long q0 = a >> 2; (q0 << 2) < b; q0 += 32) {
        const long long q = q0 + lane;
        int32_t my = -1;
        if ((q << 2) < b) {
            const int4 x = load4(p.ci, q, p.m);
            const long long i0 = q << 2;
            int cw[4];
            int32_t ww[4];
            bool ok[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long i = i0 + k;
                ww[k] = vb + elem(x, k);
                ok[k] = i >= a && i < b && (unsigned)ww[k] < (unsigned)p.n && ww[k] != v;
                if (p.rule == 0 && ww[k] > v) ok[k] = false;
                if (p.rule == 1 && ww[k] < v) ok[k] = false;
                cw[k] = ok[k] ? __ldcg(p.colors + ww[k]) : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!ok[k]) continue;
                scanned++;
                if (mag(cw[k]) == c && loses_to<kBatched>(p, v, ww[k], dv)) my = ww[k];
            }
        }
        const unsigned bal = __ballot_sync(kFull, my >= 0);
        if (bal) return __shfl_sync(kFull, my, __ffs(bal) - 1);
        if (stop && __ldcg(stop)) return -1;
    }
    return -1;
}

// Warp scan of entries [a, hi) of an ascending row, all below the vertex,
// from the top down (128 entries a step); returns the nearest neighbour
// holding magnitude c, or -1.  The stop flag is read with each step's loads
// and ends the scan after that step.  kPipe: each step's blocks are loaded
// during the step before (whole-list rounds).
template <bool kPipe>
__device__ __forceinline__ int32_t scan_range_down_warp(const Params &p, int c, long long a, long long hi,
                                                        int32_t vb, const unsigned *stop,
                                                        unsigned long long &scanned) {
    if constexpr (kPipe) {
        const int lane = threadIdx.x & 31;
        if (hi <= a) return -1;
        const long long qa = a >> 2;
        long long top = (hi - 1) >> 2, q = top - lane;
        int4 x = q >= qa ? load4(p.ci, q, p.m) : make_int4(0, 0, 0, 0);
        for (;;) {
            // the next step's blocks are loaded before this step's gathers, so
            // that a step waits for one dependent trip, not two
            const bool more = top - 32 >= qa;
            const long long nq = q - 32;
            const int4 nx = (more && nq >= qa) ? load4(p.ci, nq, p.m) : make_int4(0, 0, 0, 0);
            const unsigned halt = __ldcg(stop);
            int32_t my = -1;
            if (q >= qa) {
                const long long i0 = q << 2;
                int cw[4];
                bool ok[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long i = i0 + k;
                    const int32_t w = vb + elem(x, k);
                    ok[k] = i >= a && i < hi && (unsigned)w < (unsigned)p.n;
                    cw[k] = ok[k] ? __ldcg(p.colors + w) : 0;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (!ok[k]) continue;
                    scanned++;
                    if (mag(cw[k]) == c) my = vb + elem(x, k);
                }
            }
            const unsigned bal = __ballot_sync(kFull, my >= 0);
            if (bal) return __shfl_sync(kFull, my, __ffs(bal) - 1);
            if (halt || !more) return -1;
            top -= 32;
            q = nq;
            x = nx;
        }
    } else {
        const int lane = threadIdx.x & 31;
        for (long long top = (hi - 1) >> 2; hi > a && top >= (a >> 2); top -= 32) {
            const long long q = top - lane;
            const bool in = q >= (a >> 2);
            const int4 x = in ? load4(p.ci, q, p.m) : make_int4(0, 0, 0, 0);
            const unsigned halt = __ldcg(stop);
            int32_t my = -1;
            if (in) {
                const long long i0 = q << 2;
                int cw[4];
                bool ok[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long i = i0 + k;
                    const int32_t w = vb + elem(x, k);
                    ok[k] = i >= a && i < hi && (unsigned)w < (unsigned)p.n;
                    cw[k] = ok[k] ? __ldcg(p.colors + w) : 0;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (!ok[k]) continue;
                    scanned++;
                    if (mag(cw[k]) == c) my = vb + elem(x, k);
                }
            }
            const unsigned bal = __ballot_sync(kFull, my >= 0);
            if (bal) return __shfl_sync(kFull, my, __ffs(bal) - 1);
            if (halt) return -1;
        }
        return -1;
    }
}

// Lane scan of the (at most) 16 entries of [s, hi) nearest below hi, all
// loads in flight (ascending row, lower ids win): the nearest one holding
// magnitude c, or -1; *rest = the part still unscanned ([s, *rest)).
__device__ __forceinline__ int32_t scan_below_16(const Params &p, int c, long long s, long long hi, int32_t vb,
                                                 long long *rest, unsigned long long &scanned) {
    const long long qt = (hi - 1) >> 2, qs = s >> 2;
    int4 x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = qt - k >= qs ? load4(p.ci, qt - k, p.m) : make_int4(0, 0, 0, 0);
    int cw[4][4];
    bool ok[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long i = ((qt - k) << 2) + j;
            const int32_t w = vb + elem(x[k], j);
            ok[k][j] = qt - k >= qs && i >= s && i < hi && (unsigned)w < (unsigned)p.n;
            cw[k][j] = ok[k][j] ? __ldcg(p.colors + w) : 0;
        }
    *rest = max(s, (qt - 3) << 2);
    for (int k = 0; k < 4; ++k)
        for (int j = 3; j >= 0; --j) {
            if (!ok[k][j]) continue;
            scanned++;
            if (mag(cw[k][j]) == c) return vb + elem(x[k], j);
        }
    return -1;
}

// Medium vertices (light_max < degree <= chunk), a batch of up to 32 per warp.
// The witness first; then, with ascending rows and lower ids keeping, each
// lane scans the entries nearest below its vertex (in round 1, when every
// tentative color is 1, a vertex loses iff it has a lower neighbour, the
// nearest of which becomes its witness); the rest are scanned by the whole
// warp one vertex at a time, and keepers record their color in their
// neighbours' bitmaps with the whole warp.
template <bool kBatched, bool kMulti>
__device__ void det_medium_detect(const Params &p, const int32_t *list, unsigned cnt, int32_t *out,
                                  unsigned *out_cnt, bool prefix, bool round1, int act_r, ListSet A,
                                  Acc &acc) {
    const int lane = threadIdx.x & 31;
    const unsigned NW = total_warps(), B = warp_batch(cnt);
    for (unsigned b = rot_warp(1) * B; b < cnt; b += NW * B) {
        const unsigned i = b + lane;
        const int nb = (int)min(B, cnt - b);
        int32_t vl = 0, vbl = 0;
        Wit wl = wit_none();
        long long sl = 0, el = 0, restl = 0;
        int cl = 0;
        bool settled = false, found = false, resolved = false;
        if (lane < nb) {
            vl = __ldcg(list + i);
            if (!round1) {
                if (kMulti)
                    wl = wit_load(p, vl);
                else
                    wl.w0 = wit_first(p, vl);
            }
            cl = round1 ? 1 : -__ldcg(p.colors + vl);
            row_of<kBatched>(p, vl, sl, el, vbl);
            const int ld = prefix ? __ldcg(p.lowdeg + vl) : 0;
            if (kMulti) {  // every witness slot
                const int q = round1 ? -1 : wit_match(p, wl, cl);
                settled = q >= 0;
                if (q > 0) wit_record(p, vl, wit_slot(wl, q), wl, true);
            } else if (wl.w0 >= 0) {
                settled = mag(__ldcg(p.colors + wl.w0)) == cl;
            }
            restl = el;
            if (prefix && !settled) {
                const long long split = sl + ld;
                if (round1) {  // every tentative color is 1: any lower neighbour wins
                    found = ld > 0;
                    if (found) __stcg(p.witness + vl, vbl + __ldg(p.ci + split - 1));
                    resolved = true;
                } else if (ld == 0) {
                    resolved = true;  // nothing below: keeps its color
                } else {
                    const int32_t f = scan_below_16(p, cl, sl, split, vbl, &restl, acc.dscan);
                    found = f >= 0;
                    if (found) wit_record(p, vl, f, wl, kMulti);
                    resolved = found || restl <= sl;
                }
            }
        }
        unsigned lost = __ballot_sync(kFull, settled || found);
        const unsigned keep = __ballot_sync(kFull, lane < nb && resolved && !found && !settled);
        const unsigned open = __ballot_sync(kFull, lane < nb && !settled && !resolved);
        for (unsigned m = keep | open; m; m &= m - 1) {
            const int j = __ffs(m) - 1;
            const int32_t v = __shfl_sync(kFull, vl, j), vb = __shfl_sync(kFull, vbl, j);
            const long long s = __shfl_sync(kFull, sl, j), e = __shfl_sync(kFull, el, j);
            const long long rest = __shfl_sync(kFull, restl, j);
            const int c = __shfl_sync(kFull, cl, j);
            if ((open >> j) & 1u) {
                // prefix: the part below the lane's entries; otherwise the whole row
                const int32_t f = det_scan_warp<kBatched, kMulti>(p, v, c, (int32_t)(e - s), s, s,
                                                          prefix ? rest : e, vb, prefix, nullptr, acc.dscan);
                if (f >= 0) {
                    lost |= 1u << j;
                    if (lane == j) wit_record(p, v, f, wl, kMulti);
                    continue;
                }
            }
            if (lane == 0) {
                __stcg(p.colors + v, c);
                acc.kmax = max(acc.kmax, c);
                acc.keep++;
                acc.kdeg += (unsigned long long)(e - s);
                acc.scatter += (unsigned long long)(e - s);
            }
            scatter_color<kBatched, kMulti>(p, c, s, e, vb, lane, 32, act_r, A);
        }
        if (lost) {
            if (lane == 0) acc.next += (unsigned long long)__popc(lost);
            if (out) {
                unsigned pos = 0;
                if (lane == 0) pos = atomicAdd(out_cnt, (unsigned)__popc(lost));
                pos = __shfl_sync(kFull, pos, 0);
                if ((lost >> lane) & 1u) out[pos + __popc(lost & lanemask_lt())] = vl;
            }
        }
    }
}

// lower_only: the list's items cover only the entries below each hub
// (lower_chunks); otherwise its whole row.  round1 with prefix: every
// tentative color is 1, so a hub loses iff it has an entry below it (the
// nearest of which becomes its witness) and no item scans.
//   items / verts (lower_only lists, may be null): the entry of each work item
// and the vertex of each entry, written when the list was built.
template <bool kBatched, bool kMulti>
__device__ void det_hub_detect(const Params &p, const int32_t *slots, const unsigned *cbs,
                               const unsigned *items, const int32_t *verts, const unsigned *recs,
                               unsigned long long h64, int pn, bool prefix, bool push_losers,
                               bool lower_only, bool round1, Acc &acc) {
    const int lane = threadIdx.x & 31;
    const unsigned cnt = (unsigned)(h64 >> 32), nch = (unsigned)h64;
    const long long CH = p.chunk;
    const unsigned NW = total_warps();
    if (recs) {  // lower-part items with records: one load, then the scan
        for (unsigned q = global_warp(); q < nch; q += NW) {
            const uint4 *rp = reinterpret_cast<const uint4 *>(recs) + 2 * (size_t)q;
            const uint4 r0 = __ldcg(rp), r1 = __ldcg(rp + 1);
            const int32_t v = (int32_t)r0.x, slot = (int32_t)r0.y, vb = (int32_t)r0.w;
            const int c = (int)r0.z;
            const long long a = (long long)(((unsigned long long)r1.y << 32) | r1.x);
            const unsigned nchunks = r1.w;
            const Wit wo = (kMulti && lane == 0) ? wit_load(p, v) : wit_none();
            const int32_t found = scan_range_down_warp<kMulti>(p, c, a, a + (long long)r1.z, vb, p.hconf + slot, acc.dscan);
            const bool conf = found >= 0;
            if (lane == 0) {
                if (conf) {
                    wit_record(p, v, found, wo, kMulti);
                    atomicOr(p.hconf + slot, 1u);  // stops the hub's other items early
                }
                // the decision travels in the completion counter (conflicts in
                // the high word); release orders this item's writes before its
                // count, acquire orders the last item's resets after all counts
                const unsigned long long old =
                    atom_add_acq_rel64(p.hdone + slot, conf ? (1ull << 32) + 1ull : 1ull);
                if ((unsigned)old == nchunks - 1) {
                    const bool lost = conf || (old >> 32) != 0;
                    __stcg(p.hconf + slot, 0u);
                    __stcg(p.hdone + slot, 0ull);
                    long long s, e;
                    int32_t vb2;
                    row_of<kBatched>(p, v, s, e, vb2);
                    const long long deg = e - s;
                    if (lost) {
                        if (push_losers)
                            hub_list_push(&p.ctr->h64[pn], p.hw[pn], p.hcb[pn], slot,
                                          (unsigned)((deg + CH - 1) / CH));
                        acc.next += 1;
                    } else {
                        __stcg(p.colors + v, c);
                        acc.kmax = max(acc.kmax, c);
                        acc.keep++;
                        acc.kdeg += (unsigned long long)deg;
                        acc.scatter += (unsigned long long)deg;
                        hub_list_push(&p.ctr->sc64, p.sw, p.scb, slot,
                                      (unsigned)((deg + kScatterChunk - 1) / kScatterChunk));
                    }
                }
            }
        }
        return;
    }
    for (unsigned q = global_warp(); q < nch; q += NW) {
        const bool direct = items != nullptr;
        const unsigned i = direct ? __ldcg(items + q) : hub_entry(cbs, cnt, q);
        const int32_t slot = __ldcg(slots + i);
        const unsigned j = q - __ldcg(cbs + i);
        const int32_t v = direct ? __ldcg(verts + i) : __ldcg(p.hvert + slot);
        long long s, e;
        int32_t vb;
        row_of<kBatched>(p, v, s, e, vb);
        const long long deg = e - s;
        const long long a = s + (long long)j * CH, b = min(e, a + CH);
        const int c = -__ldcg(p.colors + v);
        bool conf = false;
        Wit wo = wit_none();
        if (!(round1 && prefix)) {
            if (kMulti)
                wo = wit_load(p, v);
            else
                wo.w0 = wit_first(p, v);
        }
        if (round1 && prefix) {
            const int ld = __ldcg(p.lowdeg + v);
            conf = ld > 0;
            if (conf && j == 0 && lane == 0) __stcg(p.witness + v, vb + __ldg(p.ci + s + ld - 1));
        } else if (j == 0) {  // the first item tries the witness (every slot, except on the activation lists)
            if (kMulti) {
                const int q = wit_match(p, wo, c);
                conf = q >= 0;
                if (q > 0 && lane == 0) wit_record(p, v, wit_slot(wo, q), wo, true);
            } else {
                conf = wo.w0 >= 0 && mag(__ldcg(p.colors + wo.w0)) == c;
            }
        }
        if (!conf && !(round1 && prefix) && !__ldcg(p.hconf + slot)) {
            const int32_t found = det_scan_warp<kBatched, kMulti>(p, v, c, (int32_t)deg, s, a, b, vb, prefix,
                                                          p.hconf + slot, acc.dscan);
            if (found >= 0) {
                conf = true;
                if (lane == 0) wit_record(p, v, found, wo, kMulti);
            }
        }
        const unsigned nchunks =
            lower_only ? lower_chunks(__ldcg(p.lowdeg + v), p.chunk) : (unsigned)((deg + CH - 1) / CH);
        if (lane == 0) {
            // hconf stops the other items early; the decision travels in the
            // completion counter itself (conflicts in the high word).  The
            // fences order a conflict's hconf write before its count and the
            // last item's reset of hconf after every count.
            if (conf) {
                atomicOr(p.hconf + slot, 1u);
                __threadfence();
            }
            const unsigned long long old =
                atomicAdd(p.hdone + slot, conf ? (1ull << 32) + 1ull : 1ull);
            if ((unsigned)old == nchunks - 1) {
                __threadfence();
                const bool lost = conf || (old >> 32) != 0;
                __stcg(p.hconf + slot, 0u);
                __stcg(p.hdone + slot, 0ull);
                if (lost) {
                    if (push_losers)
                        hub_list_push(&p.ctr->h64[pn], p.hw[pn], p.hcb[pn], slot,
                                      (unsigned)((deg + CH - 1) / CH));
                    acc.next += 1;
                } else {
                    __stcg(p.colors + v, c);
                    acc.kmax = max(acc.kmax, c);
                    acc.keep++;
                    acc.kdeg += (unsigned long long)deg;
                    acc.scatter += (unsigned long long)deg;
                    hub_list_push(&p.ctr->sc64, p.sw, p.scb, slot,
                                  (unsigned)((deg + kScatterChunk - 1) / kScatterChunk));
                }
            }
        }
    }
}

// Scatter the colors of the hubs committed in the last round (chunked).
template <bool kBatched>
__device__ void det_hub_scatter(const Params &p, unsigned long long sc64, int act_r,
                                ListSet A) {
    const int lane = threadIdx.x & 31;
    const unsigned cnt = (unsigned)(sc64 >> 32), nch = (unsigned)sc64;
    const long long CH = kScatterChunk;
    const unsigned NW = total_warps();
    for (unsigned q = global_warp(); q < nch; q += NW) {
        const unsigned i = hub_entry(p.scb, cnt, q);
        const int32_t slot = __ldcg(p.sw + i);
        const unsigned j = q - __ldcg(p.scb + i);
        const int32_t v = __ldcg(p.hvert + slot);
        long long s, e;
        int32_t vb;
        row_of<kBatched>(p, v, s, e, vb);
        const long long a = s + (long long)j * CH, b = min(e, a + CH);
        scatter_color<kBatched>(p, __ldcg(p.colors + v), a, b, vb, lane, 32, act_r, A);
    }
}

// ------------------------------------------------------------ fast mode
//
// FirstFit gathers the live colors of all neighbours; a warp takes 32
// consecutive worklist entries of low degree, stages their rows in shared
// memory with coalesced loads (one streaming copy when the rows are
// contiguous), then each lane works on its own row.

__device__ __forceinline__ int stage_rows(const int32_t *__restrict__ ci, long long m, long long s,
                                          int deg, bool act, int32_t *sbuf) {
    const int lane = threadIdx.x & 31;
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int pre = incl - deg;
    const int total = __shfl_sync(kFull, incl, 31);
    const long long e = s + deg;
    const long long s_next = __shfl_down_sync(kFull, s, 1);
    const bool act_next = __shfl_down_sync(kFull, act ? 1 : 0, 1) != 0;
    const bool contig = __all_sync(kFull, !act || lane == 31 || !act_next || e == s_next);
    if (contig) {
        const long long s0 = __shfl_sync(kFull, s, 0);
        const long long end = s0 + total;
        for (long long q = (s0 >> 2) + lane; (q << 2) < end; q += 32) {
            const int4 x = load4(ci, q, m);
            const long long i0 = q << 2;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long i = i0 + k;
                if (i >= s0 && i < end) sbuf[i - s0] = elem(x, k);
            }
        }
    } else {
        for (int p0 = 0; p0 < total; p0 += 32) {
            const int pos = p0 + lane;
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = lo + step;
                if (__shfl_sync(kFull, pre, cand) <= pos) lo = cand;
            }
            const long long src = __shfl_sync(kFull, s, lo) + (pos - __shfl_sync(kFull, pre, lo));
            if (pos < total) sbuf[pos] = __ldg(ci + src);
        }
    }
    __syncwarp();
    return pre;
}

template <bool kBatched>
__device__ void fast_light_assign(const Params &p, const int32_t *list, unsigned cnt,
                                  int32_t *sbuf, Acc &acc) {
    const unsigned tiles = (cnt + kLightTile - 1) / kLightTile;
    for (unsigned t = blockIdx.x; t < tiles; t += gridDim.x) {
        for (int u = 0; u < kLightUnroll; ++u) {
            const unsigned idx = tile_index(t, u);
            const bool act = idx < cnt;
            int32_t v = 0, vb = 0;
            long long s = 0, e = 0;
            if (act) {
                v = __ldcg(list + idx);
                row_of<kBatched>(p, v, s, e, vb);
            }
            const int deg = (int)(e - s);
            const int pre = stage_rows(p.ci, p.m, s, deg, act, sbuf);
            if (act) {
                unsigned long long mask = 0;
#pragma unroll 8
                for (int j = 0; j < deg; ++j) {
                    const int32_t w = vb + sbuf[pre + j];
                    if ((unsigned)w < (unsigned)p.n) {
                        const int c = __ldcg(p.colors + w);
                        if (c > 0 && c <= 64) mask |= 1ull << (c - 1);
                    }
                }
                const int c = __ffsll((long long)~mask);
                __stcg(p.colors + v, c);
                acc.w += 1;
                acc.d += (unsigned long long)deg;
            }
            __syncwarp();
        }
    }
}

// Lane-level fast-mode conflict test against a staged row.
template <bool kBatched>
__device__ __forceinline__ bool fast_conflict_staged(const Params &p, const int32_t *row, int deg,
                                                     int32_t v, int32_t vb, int c, bool prefix,
                                                     unsigned long long &scanned) {
    bool conf = false;
    for (int j0 = 0; j0 < deg && !conf; j0 += 8) {
        int cw[8];
        int32_t ww[8];
        bool ok[8];
        bool past = false;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = j0 + k;
            ww[k] = j < deg ? vb + row[j] : -1;
            ok[k] = j < deg && (unsigned)ww[k] < (unsigned)p.n && ww[k] != v;
            if (prefix && ok[k] && ww[k] >= v) {
                ok[k] = false;
                past = true;
            }
            if (p.rule == 0 && ww[k] > v) ok[k] = false;
            if (p.rule == 1 && ww[k] < v) ok[k] = false;
            cw[k] = ok[k] ? __ldcg(p.colors + ww[k]) : 0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (!ok[k]) continue;
            scanned++;
            if (cw[k] == c && loses_to<kBatched>(p, v, ww[k], deg)) conf = true;
        }
        if (past) break;
    }
    return conf;
}

template <bool kBatched>
__device__ void fast_light_detect(const Params &p, const int32_t *list, unsigned cnt,
                                  int32_t *out, unsigned *out_cnt, bool prefix, int32_t *sbuf,
                                  Acc &acc) {
    const unsigned tiles = (cnt + kLightTile - 1) / kLightTile;
    for (unsigned t = blockIdx.x; t < tiles; t += gridDim.x) {
        bool flag[kLightUnroll];
        int32_t item[kLightUnroll];
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u) {
            flag[u] = false;
            item[u] = 0;
            const unsigned idx = tile_index(t, u);
            const bool act = idx < cnt;
            int32_t v = 0, vb = 0;
            long long s = 0, e = 0;
            if (act) {
                v = __ldcg(list + idx);
                row_of<kBatched>(p, v, s, e, vb);
            }
            const int deg = (int)(e - s);
            const int pre = stage_rows(p.ci, p.m, s, deg, act, sbuf);
            if (act) {
                const int c = __ldcg(p.colors + v);
                if (fast_conflict_staged<kBatched>(p, sbuf + pre, deg, v, vb, c, prefix, acc.dscan)) {
                    __stcg(p.colors + v, 0);
                    flag[u] = true;
                    item[u] = v;
                } else {
                    acc.kmax = max(acc.kmax, c);
                }
            }
            __syncwarp();
        }
        block_push(flag, item, out_cnt, out, acc.next);
    }
}

// Warp-wide fast-mode conflict test over [a, b): live colors, stop at the
// first conflict (or, with ascending rows and low-keeps, at the first
// neighbour above v).
template <bool kBatched>
__device__ __forceinline__ bool fast_conflict_warp(const Params &p, int32_t v, int c, int32_t dv,
                                                   long long a, long long b, int32_t vb,
                                                   bool prefix, unsigned long long &scanned) {
    const int lane = threadIdx.x & 31;
    for (long long q0 = (a >> 2); (q0 << 2) < b; q0 += 32) {
        const long long q = q0 + lane;
        bool my = false, past = false;
        if ((q << 2) < b) {
            const int4 x = load4(p.ci, q, p.m);
            const long long i0 = q << 2;
            int cw[4];
            int32_t ww[4];
            bool ok[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long i = i0 + k;
                ww[k] = vb + elem(x, k);
                ok[k] = i >= a && i < b && (unsigned)ww[k] < (unsigned)p.n && ww[k] != v;
                if (prefix && ok[k] && ww[k] >= v) {
                    ok[k] = false;
                    past = true;
                }
                if (p.rule == 0 && ww[k] > v) ok[k] = false;
                if (p.rule == 1 && ww[k] < v) ok[k] = false;
                cw[k] = ok[k] ? __ldcg(p.colors + ww[k]) : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!ok[k]) continue;
                scanned++;
                if (cw[k] == c && loses_to<kBatched>(p, v, ww[k], dv)) my = true;
            }
        } else {
            past = true;
        }
        if (__any_sync(kFull, my)) return true;
        if (prefix && __any_sync(kFull, past)) return false;
    }
    return false;
}

template <bool kBatched>
__device__ void fast_medium_assign(const Params &p, const int32_t *list, unsigned cnt, Acc &acc) {
    const int lane = threadIdx.x & 31;
    const unsigned NW = total_warps(), B = warp_batch(cnt);
    for (unsigned b = global_warp() * B; b < cnt; b += NW * B) {
        const unsigned i = b + lane;
        const int nb = (int)min(B, cnt - b);
        int32_t vl = 0, vbl = 0;
        long long sl = 0, el = 0;
        if (lane < nb) {
            vl = __ldcg(list + i);
            row_of<kBatched>(p, vl, sl, el, vbl);
        }
        for (int j = 0; j < nb; ++j) {
            const int32_t v = __shfl_sync(kFull, vl, j), vb = __shfl_sync(kFull, vbl, j);
            const long long s = __shfl_sync(kFull, sl, j), e = __shfl_sync(kFull, el, j);
            const int c = warp_first_fit(p.ci, p.m, p.colors, s, e, vb, lane, p.n);
            if (lane == 0) {
                __stcg(p.colors + v, c);
                acc.w += 1;
                acc.d += (unsigned long long)(e - s);
            }
        }
    }
}

template <bool kBatched>
__device__ void fast_medium_detect(const Params &p, const int32_t *list, unsigned cnt,
                                   int32_t *out, unsigned *out_cnt, bool prefix, Acc &acc) {
    const int lane = threadIdx.x & 31;
    const unsigned NW = total_warps(), B = warp_batch(cnt);
    for (unsigned b = global_warp() * B; b < cnt; b += NW * B) {
        const unsigned i = b + lane;
        const int nb = (int)min(B, cnt - b);
        int32_t vl = 0, vbl = 0;
        long long sl = 0, el = 0;
        if (lane < nb) {
            vl = __ldcg(list + i);
            row_of<kBatched>(p, vl, sl, el, vbl);
        }
        unsigned lost = 0;
        for (int j = 0; j < nb; ++j) {
            const int32_t v = __shfl_sync(kFull, vl, j), vb = __shfl_sync(kFull, vbl, j);
            const long long s = __shfl_sync(kFull, sl, j), e = __shfl_sync(kFull, el, j);
            const int c = __ldcg(p.colors + v);
            if (fast_conflict_warp<kBatched>(p, v, c, (int32_t)(e - s), s, e, vb, prefix, acc.dscan)) {
                lost |= 1u << j;
                if (lane == 0) __stcg(p.colors + v, 0);
            } else if (lane == 0) {
                acc.kmax = max(acc.kmax, c);
            }
        }
        if (lost) {
            unsigned pos = 0;
            if (lane == 0) pos = atomicAdd(out_cnt, (unsigned)__popc(lost));
            pos = __shfl_sync(kFull, pos, 0);
            if ((lost >> lane) & 1u) out[pos + __popc(lost & lanemask_lt())] = vl;
            if (lane == 0) acc.next += (unsigned long long)__popc(lost);
        }
    }
}

template <bool kBatched>
__device__ void fast_hub_assign(const Params &p, int par, unsigned long long h64, int kmax,
                                Acc &acc) {
    const int lane = threadIdx.x & 31;
    const unsigned cnt = (unsigned)(h64 >> 32), nch = (unsigned)h64;
    const long long CH = p.chunk;
    const unsigned NW = total_warps();
    for (unsigned q = global_warp(); q < nch; q += NW) {
        const unsigned i = hub_entry(p.hcb[par], cnt, q);
        const int32_t slot = __ldcg(p.hw[par] + i);
        const unsigned j = q - __ldcg(p.hcb[par] + i);
        const int32_t v = __ldcg(p.hvert + slot);
        long long s, e;
        int32_t vb;
        row_of<kBatched>(p, v, s, e, vb);
        const long long deg = e - s;
        const long long a = s + (long long)j * CH, b = min(e, a + CH);
        long long nb = (long long)kmax + 64;  // a guess; the last item falls back if full
        if (nb > deg) nb = deg;
        const int nbits = (int)nb + 1;
        const int words = (nbits + 31) >> 5;
        const unsigned base = __ldcg(p.hbase + slot);
        for (int wb = 0; wb < words; wb += 8) {
            unsigned mw[8];
            mask256_lane(p.ci, p.m, p.colors, a, b, vb, lane, 32, wb * 32, p.n, mw);
            warp_or8(mw);
            if (lane < 8 && wb + lane < words) {
                const unsigned x = pick8(mw, lane);
                if (x) atomicOr(p.hbits + base + wb + lane, x);
            }
        }
        const unsigned nchunks = (unsigned)((deg + CH - 1) / CH);
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
            __threadfence();
            last = ((unsigned)atomicAdd(p.hdone + slot, 1ull) == nchunks - 1) ? 1u : 0u;
            if (last) __threadfence();
        }
        last = __shfl_sync(kFull, last, 0);
        if (last) {
            unsigned best = UINT_MAX;
            for (int k = lane; k < words; k += 32) {
                const unsigned wv = __ldcg(p.hbits + base + k);
                if (~wv) best = min(best, (unsigned)(k * 32 + __ffs(~wv) - 1));
                __stcg(p.hbits + base + k, 0u);
            }
            best = __reduce_min_sync(kFull, best);
            int c;
            if (best < (unsigned)nbits) c = (int)best + 1;
            else c = warp_first_fit(p.ci, p.m, p.colors, s, e, vb, lane, p.n);
            if (lane == 0) {
                __stcg(p.colors + v, c);
                __stcg(p.hdone + slot, 0ull);
                acc.w += 1;
                acc.d += (unsigned long long)deg;
            }
        }
    }
}

template <bool kBatched>
__device__ void fast_hub_detect(const Params &p, int par, unsigned long long h64, bool prefix,
                                Acc &acc) {
    const int lane = threadIdx.x & 31;
    const int pn = par ^ 1;
    const unsigned cnt = (unsigned)(h64 >> 32), nch = (unsigned)h64;
    const long long CH = p.chunk;
    const unsigned NW = total_warps();
    for (unsigned q = global_warp(); q < nch; q += NW) {
        const unsigned i = hub_entry(p.hcb[par], cnt, q);
        const int32_t slot = __ldcg(p.hw[par] + i);
        const unsigned j = q - __ldcg(p.hcb[par] + i);
        const int32_t v = __ldcg(p.hvert + slot);
        long long s, e;
        int32_t vb;
        row_of<kBatched>(p, v, s, e, vb);
        const long long deg = e - s;
        const long long a = s + (long long)j * CH, b = min(e, a + CH);
        const int c = __ldcg(p.colors + v);
        const bool skip = prefix && (vb + __ldg(p.ci + a)) >= v;
        const bool conf =
            !skip && fast_conflict_warp<kBatched>(p, v, c, (int32_t)deg, a, b, vb, prefix, acc.dscan);
        const unsigned nchunks = (unsigned)((deg + CH - 1) / CH);
        if (lane == 0) {
            if (conf) atomicOr(p.hconf + slot, 1u);
            __threadfence();
            if ((unsigned)atomicAdd(p.hdone + slot, 1ull) == nchunks - 1) {
                __threadfence();
                const unsigned lost = __ldcg(p.hconf + slot);
                __stcg(p.hconf + slot, 0u);
                __stcg(p.hdone + slot, 0ull);
                if (lost) {
                    __stcg(p.colors + v, 0);
                    hub_list_push(&p.ctr->h64[pn], p.hw[pn], p.hcb[pn], slot, nchunks);
                    acc.next += 1;
                } else {
                    acc.kmax = max(acc.kmax, c);
                }
            }
        }
    }
}

// ------------------------------------------------------------ init

template <bool kFast, bool kBatched>
__device__ void init_phase(const Params &p) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    // (1) adjacent col_idx pairs out of strict ascending order
    unsigned long long bad = 0;
    const long long nq = (p.m + 3) >> 2;
    for (long long q = tid; q < nq; q += nthreads) {
        const int4 x = load4(p.ci, q, p.m);
        const long long i0 = q << 2;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (i0 + k + 1 < p.m && elem(x, k) >= elem(x, k + 1)) bad++;
        if (i0 + 4 < p.m && x.w >= __ldg(p.ci + i0 + 4)) bad++;
    }
    // (2) binning of all vertices into W_1 (parity 1), in vertex order
    unsigned long long boundary = 0, dummy = 0, roots = 0;
    const unsigned nt = ((unsigned)p.n + kLightTile - 1) / kLightTile;
    for (unsigned t = blockIdx.x; t < nt; t += gridDim.x) {
        bool is_light[kLightUnroll], is_med[kLightUnroll];
        int32_t vv[kLightUnroll];
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u) {
            is_light[u] = false;
            is_med[u] = false;
            const long long v64 = (long long)tile_index(t, u);
            vv[u] = (int32_t)v64;
            if (v64 >= p.n) continue;
            const int32_t v = (int32_t)v64;
            long long s, e;
            int32_t vb;
            row_of<kBatched>(p, v, s, e, vb);
            if (e > s && e < p.m && __ldg(p.ci + e - 1) >= __ldg(p.ci + e)) boundary++;
            __stcg(p.colors + v, kFast ? 0 : -1);
            if (!kFast) wit_reset(p, v);
            const long long deg = e - s;
            if (!kFast) {  // entries below v, assuming an ascending row (used only if it is)
                long long lo = s, hi = e;
                while (lo < hi) {
                    const long long mid = (lo + hi) >> 1;
                    if (vb + __ldg(p.ci + mid) < v) lo = mid + 1;
                    else hi = mid;
                }
                p.lowdeg[v] = (int32_t)(lo - s);
                roots += lo == s;
            }
            if (deg <= p.light_max) {
                is_light[u] = true;
                if (!kFast && p.front_ok) p.vslot[v] = -1;
            } else if (deg <= p.chunk) {
                is_med[u] = true;
                if (!kFast && p.front_ok) p.vslot[v] = -2;
            } else {
                const unsigned slot = atomicAdd(&p.ctr->nslots, 1u);
                const unsigned words = (unsigned)((deg + 2 + 31) / 32);
                if (!kFast && p.front_ok) p.vslot[v] = (int32_t)slot;
                p.hvert[slot] = v;
                p.hbase[slot] = atomicAdd(&p.ctr->hwords, words);
                hub_list_push(&p.ctr->h64[1], p.hw[1], p.hcb[1], (int32_t)slot,
                              (unsigned)((deg + p.chunk - 1) / p.chunk));
            }
        }
        block_push(is_light, vv, &p.ctr->nl[1], p.lw[1], dummy);
        block_push(is_med, vv, &p.ctr->nm[1], p.mw[1], dummy);
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(kFull, bad, o);
        boundary += __shfl_xor_sync(kFull, boundary, o);
        roots += __shfl_xor_sync(kFull, roots, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(&p.ctr->unsorted_pairs, bad);
        if (boundary) atomicAdd(&p.ctr->boundary_pairs, boundary);
        if (roots) atomicAdd(&p.ctr->nroots, roots);
    }
}

// End of phase B: the CTA's largest committed color and (det) the number and
// degree sum of its keepers, which leave the worklist.
__device__ void flush_phase(const Params &p, int kloc, unsigned long long kdeg,
                            unsigned long long nslow, unsigned long long nkeep) {
    __shared__ int s_k[kWarps];
    __shared__ unsigned long long s_d[kWarps], s_s[kWarps], s_n[kWarps];
    int k = kloc;
    for (int o = 16; o > 0; o >>= 1) {
        k = max(k, __shfl_xor_sync(kFull, k, o));
        kdeg += __shfl_xor_sync(kFull, kdeg, o);
        nslow += __shfl_xor_sync(kFull, nslow, o);
        nkeep += __shfl_xor_sync(kFull, nkeep, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_k[threadIdx.x >> 5] = k;
        s_d[threadIdx.x >> 5] = kdeg;
        s_s[threadIdx.x >> 5] = nslow;
        s_n[threadIdx.x >> 5] = nkeep;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = 0;
        unsigned long long d = 0, sl = 0, nk = 0;
        for (int w = 0; w < kWarps; ++w) {
            b = max(b, s_k[w]);
            d += s_d[w];
            sl += s_s[w];
            nk += s_n[w];
        }
        // no return values below: nothing waits on these atomics
        if (b > 0) atomicMax(&p.ctr->kmax, b);
        if (d) atomicAdd(&p.ctr->dcur, 0ull - d);
        if (nk) atomicAdd(&p.ctr->wcount, 0ull - nk);
        if (sl) {
            atomicAdd(&p.ctr->nslow, sl);
            atomicAdd(&p.ctr->sum_rescan, sl);
        }
    }
}

__device__ void flush_stats(const Params &p, Acc &acc) {
    unsigned long long v[5] = {acc.w, acc.d, acc.dscan, acc.next, acc.scatter};
#pragma unroll
    for (int j = 0; j < 5; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(kFull, v[j], o);
    if ((threadIdx.x & 31) == 0) {
        if (v[0]) atomicAdd(&p.ctr->sum_w, v[0]);
        if (v[1]) atomicAdd(&p.ctr->sum_d, v[1]);
        if (v[2]) atomicAdd(&p.ctr->sum_dscan, v[2]);
        if (v[3]) atomicAdd(&p.ctr->sum_next, v[3]);
        if (v[4]) atomicAdd(&p.ctr->sum_scatter, v[4]);
    }
}

#include "sgr_tail.cuh"

// The round loop.  kFront (det only): rounds 2.. run on the activation lists;
// the launch continues after an init launch of the kFront = false kernel that
// handed the rounds over (Counters::handoff), and returns at once otherwise.
// The two kinds of rounds are separate kernels so that neither pays for the
// registers of the other.
template <bool kFast, bool kBatched, bool kFront>
__global__ void __launch_bounds__(kBlock, kMinBlocks) sgr_color_kernel(const Params p) {
    static_assert(!(kFast && kFront), "activation lists are a deterministic-mode path");
    __shared__ int32_t s_stage[kFast ? kWarps : 1][kFast ? 32 * kLightMaxStage : 1];
    int32_t *sbuf = s_stage[kFast ? (threadIdx.x >> 5) : 0];
    Acc acc;
    unsigned gen = 0;
    Counters *ctr = p.ctr;
    const bool recorder = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t0 = globaltimer();
    if (kFront && threadIdx.x == 0) *push_buf().n = 0;  // first used after a barrier
    bool sorted;
    long long r;
    if (kFront) {
        if (__ldcg(&ctr->handoff) == 0) return;  // the init launch colored everything
        t0 = __ldcg(&ctr->t_start);
        sorted = __ldcg(&ctr->unsorted_pairs) == __ldcg(&ctr->boundary_pairs);
        r = 1;
    } else if (!p.resume) {
        if (recorder) {
            ctr->t_start = t0;
            if (!kFast) {
                ctr->dcur = (unsigned long long)p.m;
                ctr->wcount = (unsigned long long)p.n;
            }
        }
        init_phase<kFast, kBatched>(p);
        if (!grid_barrier(p, gen)) { flush_stats(p, acc); return; }
        if (recorder) ctr->t_init_ns = (long long)(globaltimer() - t0);
        sorted = __ldcg(&ctr->unsorted_pairs) == __ldcg(&ctr->boundary_pairs);
        r = 1;
        if (!kFast && p.front_ok && p.front_policy != 1) {
            // hand the rounds to the activation-list kernel when the commits of
            // round 1 can only stale few vertices: at most (round-1 keepers) x
            // (average degree) activations, under n / 16 (a mesh in natural
            // order; on random graphs most of W_2 would be activated and the
            // whole-list rounds are faster).  Every CTA decides alike.
            const unsigned long long roots = __ldcg(&ctr->nroots);
            const bool few = sorted && p.rule == 0 && p.n > 0 &&
                             16.0 * (double)roots * ((double)p.m / (double)p.n) < (double)p.n;
            if (p.front_policy == 2 || few) {
                if (recorder) ctr->handoff = 1;
                return;
            }
        }
    } else {  // continue the rounds of an earlier launch (graphs admitted in between)
        sorted = p.resume_sorted != 0;
        r = __ldcg(&ctr->round);
    }
    const bool prefix = sorted && p.rule == 0;
    const long long r_end = p.resume ? r + p.rounds_per_launch : LLONG_MAX;
    if (kFront || p.resume) load_hot_counters(p);  // no barrier since the last writes
    const Counters &hc = hot_counters();
    bool ok = true;
    bool tail_try = !kFast && p.tail_max > 0 && !p.resume;
    for (;; ++r) {
        if (r == r_end) break;
        const int par = (int)(r & 1), pn = par ^ 1;
        const unsigned nl = hc.nl[par];
        const unsigned nm = hc.nm[par];
        const unsigned long long h64 = hc.h64[par];
        // |W_r|: the list sizes, or (activation lists: not every loser is
        // pushed) the count of uncommitted vertices
        const unsigned long long wsize =
            kFront ? hc.wcount
                   : (unsigned long long)nl + nm + (unsigned long long)(h64 >> 32);
        if (wsize == 0) {
            if (recorder && !kFast) ctr->sc64 = 0;  // nobody is left to read those bitmaps
            break;
        }
        if (r > p.max_rounds) {
            if (recorder) raise_error(p, kErrNoConvergence);
            break;
        }
        const bool front = kFront && r >= 2;  // this round runs on A_r
        if (!kFast) {  // colors of hubs committed last round go to their neighbours' bitmaps
            const unsigned long long sc64 = hc.sc64;
            if (sc64 >> 32) {
                det_hub_scatter<kBatched>(p, sc64, kFront ? (int)r : 0, ListSet{1, par});
                if (kFront) flush_push<kBatched>(p, ListSet{1, par});
                if (!(ok = grid_barrier(p, gen))) break;
            }
        }
        // few vertices left: the tail CTA takes the remaining rounds (the
        // bitmaps are complete here, deferred hub scatters included)
        if (!kFast && tail_try && wsize <= (unsigned long long)p.tail_max &&
            hc.dcur <= (unsigned long long)p.tail_cap) {
            const int rc = tail_build<kBatched>(p, gen, (unsigned)wsize);
            if (rc < 0) {
                ok = false;
                break;
            }
            if (rc > 0) {
                if (recorder) {
                    if (kFront && r >= 2) ctr->sum_next += wsize;  // |W_r|, losers of round r-1
                    ctr->tail_build += hc.dcur;
                }
                break;
            }
            tail_try = false;  // the W-adjacency does not fit: the grid goes on
        }
        unsigned anl = 0, anm = 0;
        unsigned long long ah = 0;
        if (front) {  // A_r is complete now
            anl = hc.nal[par];
            anm = hc.nam[par];
            ah = hc.ah64[par];
            if ((unsigned long long)anl + anm + (ah >> 32) == 0) {
                // nothing can change: only a non-symmetric input gets here
                if (recorder) raise_error(p, kErrNoConvergence);
                break;
            }
        }
        if (recorder) {
            if (kFast) {
                ctr->nl[pn] = 0;
                ctr->nm[pn] = 0;
                ctr->h64[pn] = 0;
            } else {  // det: W_{r+1}'s counters were cleared during the last phase B
                ctr->sc64 = 0;
                ctr->sum_w += wsize;                       // |W_r|
                ctr->sum_d += hc.dcur;                     // D_r: degrees of W_r
                if (kFront && r >= 2) ctr->sum_next += wsize;  // |W_r| = losers of round r-1
            }
            if (r <= kTraceCap) p.trace[kTraceFields * (r - 1)] = (long long)wsize;
        }
        const bool shortcut = !kFast && r == 1 && !p.resume;  // det round 1: all colors are 1
        if (!kFast && recorder) {  // worklist entries phase A visits
            if (front) {
                ctr->sum_touch += (unsigned long long)anl + anm + (ah >> 32);
                ctr->sum_dep += hc.adeg[par];
            } else if (!shortcut) {
                ctr->sum_touch += wsize;
            }
        }
        // ---- phase A: FirstFit over W_r (det round 1: every tentative color is 1)
        if (kFast) {
            const int kmax = hc.kmax;
            fast_hub_assign<kBatched>(p, par, h64, kmax, acc);
            fast_medium_assign<kBatched>(p, p.mw[par], nm, acc);
            fast_light_assign<kBatched>(p, p.lw[par], nl, sbuf, acc);
        } else if (front) {  // FirstFit over A_r; A_r and its dependents go to ConflictResolve
            front_assign_hubs<kBatched>(p, par, ah, (int)r, prefix, ListSet{0, par});
            front_assign_medium<kBatched>(p, par, anm, (int)r, prefix, ListSet{0, par});
            front_assign_light<kBatched>(p, par, anl, (int)r, prefix, ListSet{0, par});
            flush_push<kBatched>(p, ListSet{0, par});
        } else if (!shortcut) {
            det_assign_hubs<kBatched>(p, par, h64, prefix, hc.kmax, acc);
            det_assign_medium<kBatched>(p, par, nm, acc);
            det_assign_light<kBatched>(p, par, nl, acc);
        }
        if (!(ok = grid_barrier(p, gen))) break;
        if (recorder && r <= kTraceCap)
            p.trace[kTraceFields * (r - 1) + 1] = (long long)(globaltimer() - t0);
        // ---- phase B: ConflictResolve over W_r, commit keepers, compact losers
        Acc b;
        if (kFast) {
            fast_hub_detect<kBatched>(p, par, h64, prefix, b);
            fast_medium_detect<kBatched>(p, p.mw[par], nm, p.mw[pn], &ctr->nm[pn], prefix, b);
            fast_light_detect<kBatched>(p, p.lw[par], nl, p.lw[pn], &ctr->nl[pn], prefix, sbuf, b);
        } else {
            // round 1 reads W_1 itself; later rounds only the vertices the
            // witness did not settle in phase A (or, on the activation lists,
            // A_r and its dependents).  On the activation lists every commit
            // activates its stale neighbours for round r+1 and no loser is
            // pushed: the ones not activated stay as they are.
            const unsigned bnl = shortcut ? nl : hc.nul[par];
            const unsigned bnm = shortcut ? nm : hc.num[par];
            const unsigned long long bh = shortcut ? h64 : hc.uh64[par];
            const int act_r = kFront ? (int)(r + 1) : 0;
            if (recorder) {  // W_r's counters are in registers; U_{r+1} must start empty
                ctr->sum_touch += (unsigned long long)bnl + bnm + (bh >> 32);
                ctr->nl[par] = 0;
                ctr->nm[par] = 0;
                ctr->h64[par] = 0;
                ctr->nul[pn] = 0;
                ctr->num[pn] = 0;
                ctr->uh64[pn] = 0;
                if (kFront) {  // A_r's too
                    ctr->nal[par] = 0;
                    ctr->nam[par] = 0;
                    ctr->ah64[par] = 0;
                    ctr->adeg[par] = 0;
                }
            }
            const bool lower_only = prefix && !shortcut && !kFront;
            det_hub_detect<kBatched, !kFront>(p, shortcut ? p.hw[par] : p.uh[par],
                                     shortcut ? p.hcb[par] : p.ucb[par],
                                     lower_only ? p.uitem[par] : nullptr,
                                     lower_only ? p.uvert[par] : nullptr,
                                     lower_only ? p.urec[par] : nullptr, bh, pn, prefix, !kFront,
                                     lower_only, shortcut, b);
            det_medium_detect<kBatched, !kFront>(p, shortcut ? p.mw[par] : p.um[par], bnm,
                                        kFront ? nullptr : p.mw[pn], &ctr->nm[pn], prefix, shortcut,
                                        act_r, ListSet{1, pn}, b);
            det_light_detect<kBatched>(p, shortcut ? p.lw[par] : p.ul[par], bnl,
                                       kFront ? nullptr : p.lw[pn], &ctr->nl[pn], prefix, shortcut,
                                       act_r, ListSet{1, pn}, b);
            if (kFront) flush_push<kBatched>(p, ListSet{1, pn});
        }
        acc.w += b.w;
        acc.d += b.d;
        acc.dscan += b.dscan;
        acc.next += b.next;
        acc.scatter += b.scatter;
        flush_phase(p, b.kmax, b.kdeg, b.slow, b.keep);
        if (!(ok = grid_barrier(p, gen))) break;
        if (recorder && r <= kTraceCap) {
            p.trace[kTraceFields * (r - 1) + 2] = (long long)(globaltimer() - t0);
            p.trace[kTraceFields * (r - 1) + 3] = (long long)__ldcg(&ctr->nslow);
            ctr->nslow = 0;
        }
    }
    if (recorder && ok) {
        ctr->rounds = r - 1;
        ctr->round = r;
    }
    if (kFront) acc.next = 0;  // counted from |W_r| above
    flush_stats(p, acc);
}

// ------------------------------------------------------------ batch helpers

__global__ void fill_gid_kernel(int32_t *gid, const long long *vbase, int G) {
    const int g = blockIdx.x;
    if (g >= G) return;
    const long long a = vbase[g], b = vbase[g + 1];
    for (long long v = a + threadIdx.x; v < b; v += blockDim.x) gid[v] = g;
}

__global__ void segmented_max_kernel(const int32_t *colors, const long long *vbase, int G,
                                     int32_t *out) {
    const int g = blockIdx.x;
    if (g >= G) return;
    const long long a = vbase[g], b = vbase[g + 1];
    int k = 0;
    for (long long v = a + threadIdx.x; v < b; v += blockDim.x) k = max(k, colors[v]);
    for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(kFull, k, o));
    __shared__ int s_k[kWarps];
    if ((threadIdx.x & 31) == 0) s_k[threadIdx.x >> 5] = k;
    __syncthreads();
    if (threadIdx.x == 0) {
        int b2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b2 = max(b2, s_k[w]);
        out[g] = b2;
    }
}

// ------------------------------------------------------------ server helpers

// Admit graph slot g (global vertices [vb, vb + n), det mode) into the
// resident state between two resumable launches: reset its per-vertex state,
// compute lower-neighbour counts, and append its vertices, binned by degree,
// to the worklists of parity `par` (the next round's W_in).  Hubs use their
// vertex id as slot.
__global__ void __launch_bounds__(kBlock) admit_kernel(const Params p, int g, long long vb,
                                                       int32_t n, int par) {
    unsigned long long dsum = 0, dummy = 0;
    const unsigned nt = ((unsigned)n + kLightTile - 1) / kLightTile;
    for (unsigned t = blockIdx.x; t < nt; t += gridDim.x) {
        bool is_light[kLightUnroll], is_med[kLightUnroll];
        int32_t vv[kLightUnroll];
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u) {
            is_light[u] = false;
            is_med[u] = false;
            const long long i = (long long)tile_index(t, u);
            vv[u] = (int32_t)(vb + i);
            if (i >= n) continue;
            const int32_t v = (int32_t)(vb + i);
            const_cast<int32_t *>(p.gid)[v] = g;
            __stcg(p.colors + v, -1);
            wit_reset(p, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) p.bm[(size_t)j * p.np + v] = 0u;
            const long long eb = p.ebase[g];
            const long long s = eb + __ldg(p.ro + p.robase[g] + i);
            const long long e = eb + __ldg(p.ro + p.robase[g] + i + 1);
            long long lo = s, hi = e;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (vb + __ldg(p.ci + mid) < v) lo = mid + 1;
                else hi = mid;
            }
            p.lowdeg[v] = (int32_t)(lo - s);
            const long long deg = e - s;
            dsum += (unsigned long long)deg;
            if (deg <= p.light_max) {
                is_light[u] = true;
            } else if (deg <= p.chunk) {
                is_med[u] = true;
            } else {
                p.hvert[v] = v;
                hub_list_push(&p.ctr->h64[par], p.hw[par], p.hcb[par], v,
                              (unsigned)((deg + p.chunk - 1) / p.chunk));
            }
        }
        block_push(is_light, vv, &p.ctr->nl[par], p.lw[par], dummy);
        block_push(is_med, vv, &p.ctr->nm[par], p.mw[par], dummy);
    }
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
    if ((threadIdx.x & 31) == 0 && dsum) atomicAdd(&p.ctr->dcur, dsum);
}

// Exclusive scan of one value per thread over the whole CTA (blockDim.x a
// multiple of 32, at most 1024); *total receives the sum.  Begins and ends
// with a __syncthreads().
__device__ unsigned cta_excl_scan(unsigned x, unsigned *total) {
    __shared__ unsigned s_w[32], s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    unsigned incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned v = lane < nw ? s_w[lane] : 0u;
        unsigned vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(kFull, vi, o);
            if (lane >= o) vi += t;
        }
        if (lane < nw) s_w[lane] = vi - v;
        if (lane == 31) s_tot = vi;
    }
    __syncthreads();
    *total = s_tot;
    return s_w[warp] + incl - x;
}

// Server: take the vertices of one resident graph (global ids [lo, hi)) off
// the worklists of parity `par` (the next round's W_in), in place and in
// order, with their degrees off the worklist's degree sum.  One CTA; runs
// between two resumable launches, when the graph is retired before it
// finished (its round cap passed).  Writes land at or below every entry still
// to be read (kept entries only move down), and each tile's reads precede its
// writes (the scans' barriers).
__global__ void __launch_bounds__(1024) purge_kernel(const Params p, long long lo, long long hi, int par) {
    unsigned long long dsum = 0;
    for (int which = 0; which < 2; ++which) {  // light, then medium list
        int32_t *list = which ? p.mw[par] : p.lw[par];
        unsigned *cnt = which ? &p.ctr->nm[par] : &p.ctr->nl[par];
        const unsigned n = *cnt;
        unsigned put = 0;
        for (unsigned base = 0; base < n; base += blockDim.x) {
            const unsigned i = base + threadIdx.x;
            int32_t v = 0;
            bool keep = false;
            if (i < n) {
                v = list[i];
                keep = v < lo || v >= hi;
                if (!keep) dsum += (unsigned long long)vertex_degree<true>(p, v);
            }
            unsigned tot;
            const unsigned pos = cta_excl_scan(keep ? 1u : 0u, &tot);
            if (keep) list[put + pos] = v;
            put += tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) *cnt = put;
    }
    {  // hub list: entries (slot, chunk base); kept entries get new chunk bases
        const unsigned long long h = p.ctr->h64[par];
        const unsigned n = (unsigned)(h >> 32), nch = (unsigned)h;
        int32_t *slots = p.hw[par];
        unsigned *cbs = p.hcb[par];
        unsigned put = 0, cput = 0;
        for (unsigned base = 0; base < n; base += blockDim.x) {
            const unsigned i = base + threadIdx.x;
            int32_t slot = 0;
            unsigned nc = 0;
            bool keep = false;
            if (i < n) {
                slot = slots[i];
                nc = (i + 1 < n ? cbs[i + 1] : nch) - cbs[i];
                const int32_t v = p.hvert[slot];
                keep = v < lo || v >= hi;
                if (!keep) dsum += (unsigned long long)vertex_degree<true>(p, v);
            }
            unsigned tot, ctot;
            const unsigned pos = cta_excl_scan(keep ? 1u : 0u, &tot);
            const unsigned cpos = cta_excl_scan(keep ? nc : 0u, &ctot);
            if (keep) {
                slots[put + pos] = slot;
                cbs[put + pos] = cput + cpos;
            }
            put += tot;
            cput += ctot;
        }
        __syncthreads();
        if (threadIdx.x == 0) p.ctr->h64[par] = ((unsigned long long)put << 32) | cput;
    }
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
    if ((threadIdx.x & 31) == 0 && dsum) atomicAdd(&p.ctr->dcur, 0ull - dsum);
}

// Per resident graph slot: vertices not yet final and the largest color.
__global__ void slot_status_kernel(const int32_t *colors, const long long *vbase,
                                   const int32_t *nv, int G, int32_t *rem, int32_t *kmax) {
    const int g = blockIdx.x;
    if (g >= G) return;
    const long long a = vbase[g], b = a + nv[g];
    int open = 0, k = 0;
    for (long long v = a + threadIdx.x; v < b; v += blockDim.x) {
        const int c = __ldcg(colors + v);
        open += c <= 0;
        k = max(k, c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        open += __shfl_xor_sync(kFull, open, o);
        k = max(k, __shfl_xor_sync(kFull, k, o));
    }
    __shared__ int s_o[kWarps], s_k[kWarps];
    if ((threadIdx.x & 31) == 0) {
        s_o[threadIdx.x >> 5] = open;
        s_k[threadIdx.x >> 5] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int o2 = 0, k2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            o2 += s_o[w];
            k2 = max(k2, s_k[w]);
        }
        rem[g] = o2;
        kmax[g] = k2;
    }
}

// ------------------------------------------------------------ validation

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// flags[0]: bit0 offsets broken, bit1 id out of range, bit2 self-loop,
// bit3 some row not strictly ascending, bit4 duplicate (ascending rows only),
// bit5 asymmetric (exact search, ascending rows only);
// flags[1] / flags[2]: sums of hash(v,w) / hash(w,v) over all entries.
__global__ void validate_kernel(int32_t n, long long m, const int32_t *ro, const int32_t *ci,
                                unsigned long long *flags, int exact_pass) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long f = 0, h1 = 0, h2 = 0;
    for (long long v = warp; v < n; v += nwarps) {
        const int s = ro[v], e = ro[v + 1];
        if (e < s || s < 0 || e > m || (v == 0 && s != 0)) { f |= 1; continue; }
        for (int i = s + lane; i < e; i += 32) {
            const int w = ci[i];
            if (w < 0 || w >= n) { f |= 2; continue; }
            if (w == (int)v) f |= 4;
            if (i > s) {
                const int u = ci[i - 1];
                if (u >= w) f |= 8;
                if (u == w) f |= 16;
            }
            if (!exact_pass) {
                h1 += mix64(((unsigned long long)(unsigned)v << 32) | (unsigned)w);
                h2 += mix64(((unsigned long long)(unsigned)w << 32) | (unsigned)v);
            } else {
                int lo = ro[w], hi = ro[w + 1];
                if (lo < 0 || hi > m || hi < lo) { f |= 1; continue; }
                bool found = false;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    const int x = ci[mid];
                    if (x == (int)v) { found = true; break; }
                    if (x < (int)v) lo = mid + 1;
                    else hi = mid;
                }
                if (!found) f |= 32;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        f |= __shfl_xor_sync(kFull, f, o);
        h1 += __shfl_xor_sync(kFull, h1, o);
        h2 += __shfl_xor_sync(kFull, h2, o);
    }
    if (lane == 0) {
        if (f) atomicOr(flags, f);
        if (h1) atomicAdd(flags + 1, h1);
        if (h2) atomicAdd(flags + 2, h2);
    }
}

}  // namespace

int occupancy_blocks_per_sm(bool fast, bool batched, int *out) {
    cudaError_t e;
    if (fast) {
        e = batched ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          out, sgr_color_kernel<true, true, false>, kBlock, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          out, sgr_color_kernel<true, false, false>, kBlock, 0);
    } else {
        e = batched ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          out, sgr_color_kernel<false, true, false>, kBlock, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          out, sgr_color_kernel<false, false, false>, kBlock, 0);
    }
    return (int)e;
}

int occupancy_blocks_per_sm_front(bool batched, int *out) {
    return (int)(batched ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               out, sgr_color_kernel<false, true, true>, kBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               out, sgr_color_kernel<false, false, true>, kBlock, 0));
}

cudaError_t launch_color(const Params &p, bool fast, bool batched, int grid, cudaStream_t s) {
    void *args[] = {(void *)&p};
    const void *fn;
    if (fast) fn = batched ? (const void *)sgr_color_kernel<true, true, false>
                           : (const void *)sgr_color_kernel<true, false, false>;
    else fn = batched ? (const void *)sgr_color_kernel<false, true, false>
                      : (const void *)sgr_color_kernel<false, false, false>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, 0, s);
}

cudaError_t launch_color_front(const Params &p, bool batched, int grid, cudaStream_t s) {
    void *args[] = {(void *)&p};
    const void *fn = batched ? (const void *)sgr_color_kernel<false, true, true>
                             : (const void *)sgr_color_kernel<false, false, true>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, 0, s);
}

cudaError_t launch_color_tail(const Params &p, bool batched, cudaStream_t s) {
    const void *fn = batched ? (const void *)sgr_tail_kernel<true> : (const void *)sgr_tail_kernel<false>;
    const size_t smem = tail_launch_smem(p.tail_max);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&p};
    return cudaLaunchKernel(fn, dim3(1), dim3(kTailThreads), args, smem, s);
}

cudaError_t launch_admit(const Params &p, int g, long long vb, int32_t n, int par, int grid,
                         cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    admit_kernel<<<grid, kBlock, 0, s>>>(p, g, vb, n, par);
    return cudaGetLastError();
}

cudaError_t launch_purge(const Params &p, long long lo, long long hi, int par, cudaStream_t s) {
    purge_kernel<<<1, 1024, 0, s>>>(p, lo, hi, par);
    return cudaGetLastError();
}

cudaError_t launch_slot_status(const int32_t *colors, const long long *vbase, const int32_t *nv,
                               int G, int32_t *rem, int32_t *kmax, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    slot_status_kernel<<<G, kBlock, 0, s>>>(colors, vbase, nv, G, rem, kmax);
    return cudaGetLastError();
}

cudaError_t launch_fill_gid(int32_t *gid, const long long *vbase_dev, int G, int32_t n,
                            cudaStream_t s) {
    (void)n;
    if (G <= 0) return cudaSuccess;
    fill_gid_kernel<<<G, 256, 0, s>>>(gid, vbase_dev, G);
    return cudaGetLastError();
}

cudaError_t launch_segmented_max(const int32_t *colors, const long long *vbase_dev, int G,
                                 int32_t *out_dev, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    segmented_max_kernel<<<G, 256, 0, s>>>(colors, vbase_dev, G, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_validate(int32_t n, long long m, const int32_t *ro, const int32_t *ci,
                            unsigned long long *flags_dev, cudaStream_t s) {
    int blocks = (int)((((long long)n * 32) + 255) / 256);
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    validate_kernel<<<blocks, 256, 0, s>>>(n, m, ro, ci, flags_dev, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_validate_exact(int32_t n, long long m, const int32_t *ro, const int32_t *ci,
                                  unsigned long long *flags_dev, cudaStream_t s) {
    int blocks = (int)((((long long)n * 32) + 255) / 256);
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    validate_kernel<<<blocks, 256, 0, s>>>(n, m, ro, ci, flags_dev, 1);
    return cudaGetLastError();
}

}  // namespace sgr
