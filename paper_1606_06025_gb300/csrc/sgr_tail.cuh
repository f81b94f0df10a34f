// sgr_tail.cuh -- the last deterministic rounds in one CTA.
//
// Included by sgr_kernels.cu inside its anonymous namespace, after the
// helpers it uses (row_of, load4, grid_barrier, warp_first_fit).
//
// Once few vertices are left on the worklist, a round of Algorithm 7 is a
// short chain of dependent steps (FirstFit, ConflictResolve, commit), and the
// persistent grid pays two or three grid-wide barriers and a few L2 round
// trips for the list bookkeeping per round, whatever the amount of work.  At
// |W_r| <= tail_max the grid therefore builds, once, the subgraph induced by
// W_r with 16-bit local ids and hands the remaining rounds to one CTA of 1024
// threads that keeps every per-vertex state (forbidden-color bitmap,
// tentative color, witness) in shared memory and uses __syncthreads() as the
// round barrier.
//
// Why the result is that of the full rounds (Algorithm 7 with Algorithms 4
// and 5 under frozen reads, judge before clear): from round r on only the
// vertices of W_r change.  FirstFit of v reads the final colors of all of
// v's neighbours; those outside W_r are final already and recorded in v's
// bitmap (all commits of earlier rounds, the deferred hub scatters included,
// are in the bitmaps when the grid hands over), and those inside W_r commit
// in the CTA, which adds each commit to the bitmaps of the committer's
// W-neighbours.  ConflictResolve compares tentative colors, which only
// vertices of W_r hold, so only the W-neighbours matter there too.  Colors
// above 256 are not in the bitmaps; a vertex whose 256 bits are all set
// falls back to a scan of its full row over the final colors, which the CTA
// writes to `colors` at every commit.

// ------------------------------------------------------------ build (whole grid)

// Order-preserving block compaction (as block_push) of item pairs (item to
// out, item2 to out2) that writes no position at or beyond cap; the counter
// still counts every flag.
__device__ __forceinline__ void block_push_capped(const bool (&flag)[kLightUnroll],
                                                  const int32_t (&item)[kLightUnroll],
                                                  const unsigned (&item2)[kLightUnroll],
                                                  unsigned *counter, int32_t *out, unsigned *out2,
                                                  unsigned cap) {
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
        s_pos[lane] = warp_reserve(s_pos[lane], counter, true, tot);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kLightUnroll; ++u) {
        const unsigned pos = s_pos[warp * kLightUnroll + u] + __popc(bal[u] & lanemask_lt());
        if (flag[u] && pos < cap) {
            out[pos] = item[u];
            out2[pos] = item2[u];
        }
    }
    __syncthreads();
}

// Exclusive scan in place of a[0..n) and b[0..n) (b may be null) by the
// whole CTA (a[n], b[n] receive the totals); tiles of 16 consecutive entries
// per thread, all loads of a tile in flight.  Ends with a __syncthreads().
constexpr int kScanPer = 16;

__device__ void cta_scan2(unsigned *a, unsigned *b, unsigned n) {
    __shared__ unsigned s_wa[kWarps], s_wb[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned ca = 0, cb = 0;  // carries from earlier tiles
    for (unsigned base = 0; base < n; base += kScanPer * kBlock) {
        const unsigned i0 = base + kScanPer * threadIdx.x;
        unsigned va[kScanPer], vb[kScanPer], sa = 0, sb = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            va[k] = i0 + k < n ? __ldcg(a + i0 + k) : 0u;
            vb[k] = (b && i0 + k < n) ? __ldcg(b + i0 + k) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            sa += va[k];
            sb += vb[k];
        }
        unsigned ia = sa, ib = sb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned x = __shfl_up_sync(kFull, ia, o), y = __shfl_up_sync(kFull, ib, o);
            if (lane >= o) {
                ia += x;
                ib += y;
            }
        }
        if (lane == 31) {
            s_wa[warp] = ia;
            s_wb[warp] = ib;
        }
        __syncthreads();
        unsigned pa = ca, pb = cb, ta = 0, tb = 0;
        for (int w = 0; w < kWarps; ++w) {
            if (w < warp) {
                pa += s_wa[w];
                pb += s_wb[w];
            }
            ta += s_wa[w];
            tb += s_wb[w];
        }
        pa += ia - sa;
        pb += ib - sb;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            if (i0 + k < n) {
                a[i0 + k] = pa;
                if (b) b[i0 + k] = pb;
            }
            pa += va[k];
            pb += vb[k];
        }
        ca += ta;
        cb += tb;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a[n] = ca;
        if (b) b[n] = cb;
    }
    __syncthreads();
}

// CTA 0, after the compaction: the chunk prefix of the pass over the rows
// (ceil(degree / kTailChunk) warp items per local vertex) and the map from a
// chunk to its local vertex.
__device__ __noinline__ void tail_chunk_prefix(const Params &p, unsigned nT) {
    for (unsigned i = threadIdx.x; i < nT; i += blockDim.x)
        p.tcp[i] = (__ldcg(p.tdeg + i) + kTailChunk - 1) / kTailChunk;
    __syncthreads();
    cta_scan2(p.tcp, nullptr, nT);
    const bool fits = __ldcg(p.tcp + nT) <= (unsigned)p.tail_chunks;
    if (threadIdx.x == 0 && !fits) p.ctr->tail_fail = 1;
    if (fits)
        for (unsigned i = threadIdx.x; i < nT; i += blockDim.x) {
            const unsigned q1 = __ldcg(p.tcp + i + 1);
            for (unsigned q = __ldcg(p.tcp + i); q < q1; ++q) p.tcm[q] = i;
        }
    __syncthreads();
}

// CTA 0, after the row pass (which added every chunk's counts into tcnt and
// tlow): the start of every run, its count rounded up to 8 so that every run
// starts on 16 bytes.  Sets tail_fail if the runs exceed tail_cap.
__device__ __noinline__ void tail_run_prefix(const Params &p, unsigned nT) {
    for (unsigned i = threadIdx.x; i < nT; i += blockDim.x) p.toff[i] = (__ldcg(p.tcnt + i) + 7u) & ~7u;
    __syncthreads();
    cta_scan2(p.toff, nullptr, nT);
    if (threadIdx.x == 0 && (long long)__ldcg(p.toff + nT) > p.tail_cap) p.ctr->tail_fail = 1;
    __syncthreads();
}

// One warp item of the pass over the rows: entries [a, b) of local vertex
// i's row.  Lane l takes four consecutive 16-byte blocks of each 128-block
// step (all loads in flight), so lane order is row order.  The neighbours
// still on the worklist (color <= 0) go, as local ids and in row order, to
// the chunk's slot of kTailChunk entries in tstage; their number goes to
// tcc[q] and is added, with the number of them below the vertex, into the
// vertex's tcnt / tlow.
template <bool kBatched>
__device__ __noinline__ void tail_chunk_pass(const Params &p, unsigned nT, unsigned q) {
    const int lane = threadIdx.x & 31;
    const unsigned i = __ldcg(p.tcm + q);
    const int32_t v = __ldcg(p.tlist + i);
    const unsigned j = q - __ldcg(p.tcp + i);
    long long s, e;
    int32_t vb;
    row_of<kBatched>(p, v, s, e, vb);
    const long long a = s + (long long)j * kTailChunk, b = min(e, a + kTailChunk);
    unsigned short *out = p.tstage + (size_t)q * kTailChunk;
    unsigned put = 0, below = 0;
    for (long long q0 = a >> 2; (q0 << 2) < b; q0 += 128) {
        int4 x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const long long qq = q0 + 4 * lane + t;
            x[t] = (qq << 2) < b ? load4(p.ci, qq, p.m) : make_int4(0, 0, 0, 0);
        }
        bool in[4][4];
        int cw[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long idx = ((q0 + 4 * lane + t) << 2) + k;
                const int32_t u = vb + elem(x[t], k);
                in[t][k] = idx >= a && idx < b && (unsigned)u < (unsigned)p.n && u != v;
                cw[t][k] = in[t][k] ? __ldcg(p.colors + u) : 1;
            }
        int32_t lu[4][4];
        unsigned c = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                in[t][k] = in[t][k] && cw[t][k] <= 0;
                c += in[t][k] ? 1u : 0u;
                below += (in[t][k] && vb + elem(x[t], k) < v) ? 1u : 0u;
                lu[t][k] = in[t][k] ? __ldcg(p.tloc + vb + elem(x[t], k)) : 0;
            }
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned tt = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += tt;
        }
        unsigned pos = put + incl - c;
        put += __shfl_sync(kFull, incl, 31);
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (in[t][k]) out[pos++] = (unsigned short)lu[t][k];
    }
    for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(kFull, below, o);
    if (lane == 0) {
        p.tcc[q] = put;
        if (put) atomicAdd(p.tcnt + i, put);
        if (below) atomicAdd(p.tlow + i, below);
    }
}

// Copy of chunk q's staged entries to its place in the run of its vertex:
// after the entries of the vertex's earlier chunks (their counts summed by
// the warp).  With winner bit sets, the entries that win against the vertex
// under the rule get their bit in its row of twin.
__device__ __noinline__ void tail_chunk_copy(const Params &p, unsigned q) {
    const int lane = threadIdx.x & 31;
    const unsigned i = __ldcg(p.tcm + q);
    const unsigned n = __ldcg(p.tcc + q);
    unsigned before = 0;
    for (unsigned k = __ldcg(p.tcp + i) + lane; k < q; k += 32) before += __ldcg(p.tcc + k);
    before = __reduce_add_sync(kFull, before);
    const unsigned short *src = p.tstage + (size_t)q * kTailChunk;
    unsigned short *dst = p.tadj + __ldcg(p.toff + i) + before;
    for (unsigned k = lane; k < n; k += 32) dst[k] = src[k];
    if (!p.twin) return;
    unsigned *wrow = p.twin + (size_t)i * p.tail_mw;
    const int32_t v = __ldcg(p.tlist + i);
    const unsigned dv = p.rule == 2 ? __ldcg(p.tdeg + i) : 0u;
    for (unsigned k = lane; k < n; k += 32) {
        const unsigned lu = src[k];
        const int32_t u = __ldcg(p.tlist + lu);
        bool win;
        if (p.rule == 0) {
            win = u < v;
        } else if (p.rule == 1) {
            win = u > v;
        } else {  // higher degree, then lower id
            const unsigned du = __ldcg(p.tdeg + lu);
            win = du != dv ? du > dv : u < v;
        }
        if (win) atomicOr(wrow + (lu >> 5), 1u << (lu & 31));
    }
}

// The grid's part of the hand-over at the top of round r (all CTAs call it
// alike).  Returns 1 when the tail CTA takes over (the caller leaves its
// round loop), 0 when the W-adjacency does not fit (the caller goes on with
// the round on the grid and does not try again), -1 when a barrier failed.
template <bool kBatched>
__device__ __noinline__ int tail_build(const Params &p, unsigned &gen, unsigned wsize) {
    Counters *ctr = p.ctr;
    // (1) W_r = the vertices not yet final, into tlist, with their degrees
    const unsigned nt = ((unsigned)p.n + kLightTile - 1) / kLightTile;
    for (unsigned t = blockIdx.x; t < nt; t += gridDim.x) {
        bool f[kLightUnroll];
        int32_t vv[kLightUnroll];
        unsigned dv[kLightUnroll];
#pragma unroll
        for (int u = 0; u < kLightUnroll; ++u) {
            const unsigned idx = tile_index(t, u);
            vv[u] = (int32_t)idx;
            f[u] = idx < (unsigned)p.n && __ldcg(p.colors + idx) <= 0;
            dv[u] = 0;
            if (f[u]) {
                long long rs, re;
                int32_t vb;
                row_of<kBatched>(p, (int32_t)idx, rs, re, vb);
                dv[u] = (unsigned)(re - rs);
            }
        }
        block_push_capped(f, vv, dv, &ctr->tail_n, p.tlist, p.tdeg, (unsigned)p.tail_max);
    }
    if (!grid_barrier(p, gen)) return -1;
    const unsigned nT = __ldcg(&ctr->tail_n);
    if (nT > (unsigned)p.tail_max || nT != wsize) {  // only a broken input gets here
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr->tail_fail = 1;
        return 0;  // every CTA sees the same nT and returns alike
    }
    // (2) local ids, counts and winner bit sets cleared; CTA 0: chunk prefix
    // and chunk map
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nT; i += gridDim.x * blockDim.x) {
        p.tloc[__ldcg(p.tlist + i)] = (int32_t)i;
        p.tcnt[i] = 0;
        p.tlow[i] = 0;
    }
    if (p.twin) {
        const size_t words = (size_t)nT * p.tail_mw;
        for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
             w += (size_t)gridDim.x * blockDim.x)
            p.twin[w] = 0u;
    }
    if (blockIdx.x == 0) tail_chunk_prefix(p, nT);
    if (!grid_barrier(p, gen)) return -1;
    if (__ldcg(&ctr->tail_fail)) return 0;
    // (3) the W-neighbours of every chunk, staged in row order
    const unsigned nch = __ldcg(p.tcp + nT);
    for (unsigned q = global_warp(); q < nch; q += total_warps()) tail_chunk_pass<kBatched>(p, nT, q);
    if (!grid_barrier(p, gen)) return -1;
    // (4) CTA 0: run starts
    if (blockIdx.x == 0) tail_run_prefix(p, nT);
    if (!grid_barrier(p, gen)) return -1;
    if (__ldcg(&ctr->tail_fail)) return 0;
    // (5) the runs, each in row order
    for (unsigned q = global_warp(); q < nch; q += total_warps()) tail_chunk_copy(p, q);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->tail = 1;
    return 1;  // the end of the launch orders these writes before the tail CTA
}

// ------------------------------------------------------------ the tail CTA
//
// Per local vertex the CTA keeps one 64-bit word tk: the tentative color of
// the round in the high half (0 once the vertex is final) and its rank under
// the loser rule in the low half (u wins against v iff rank(u) > rank(v)).
// A vertex the witness does not settle scans its run for a winning
// W-neighbour with the same tentative color and stops at the first one, which
// becomes its witness.  On ascending rows under the id rules the run is in
// row order and split at the vertex itself, so the scan visits only winners,
// nearest first (downward from the split when lower ids win, upward when
// higher ids win): the nearest winner is the likeliest to lose again itself,
// to stay on the worklist and settle the next round with one read, and a
// conflict is usually within a few entries.  Otherwise the whole run is
// scanned with the rank test.  Each unsettled vertex is first scanned by a
// group of eight lanes over its eight nearest 16-byte blocks, one block a lane,
// all in flight at once; the few that go on past them are finished by whole
// warps.  Keepers record their color at their W-neighbours in a separate
// warp-parallel pass.

struct TailSmem {
    unsigned long long *tk;  // [T] tentative color << 32 | rank
    unsigned *bits;          // [8][T] forbidden colors 1..256, plane-major
    int32_t *vid;            // [T] vertex id
    int32_t *deg;            // [T] degree
    unsigned *off;           // [T] start of the W-neighbour run in tadj
    unsigned *lbest;         // [T] per long-queue entry: nearest conflict (distance << 16 | local id)
    unsigned short *cnt;     // [T] W-neighbours
    unsigned short *low;     // [T] W-neighbours below the vertex (row-ordered runs)
    short *wit;              // [T] local id of the neighbour that beat it last, or -1
    short *wo;               // [3][T] the ones that beat it before, most recent first, or -1
    unsigned short *res;     // [T] run position where a warp resumes the scan
    unsigned short *q;       // [T] unsettled vertices of the round (also: full bitmaps)
    unsigned short *lq;      // [T] unsettled vertices whose scan continues past the lane's blocks
    unsigned short *kq;      // [T] keepers of the round
    unsigned short *al;      // [2][T]: the vertices still on the worklist, by round parity
};

// The arrays' stride: T rounded up to a multiple of 8, so that every array
// starts on a 16-byte boundary whatever the hand-over size.
__device__ __forceinline__ int tail_stride(int tail_max) { return (tail_max + 7) & ~7; }

__device__ __forceinline__ TailSmem tail_smem(unsigned char *raw, int T) {
    TailSmem s;
    s.tk = (unsigned long long *)raw;
    s.bits = (unsigned *)(s.tk + T);
    s.vid = (int32_t *)(s.bits + 8 * T);
    s.deg = s.vid + T;
    s.off = (unsigned *)(s.deg + T);
    s.lbest = s.off + T;
    s.cnt = (unsigned short *)(s.lbest + T);
    s.low = s.cnt + T;
    s.wit = (short *)(s.low + T);
    s.wo = s.wit + T;
    s.res = (unsigned short *)(s.wo + 3 * T);
    s.q = s.res + T;
    s.lq = s.q + T;
    s.kq = s.lq + T;
    s.al = s.kq + T;
    return s;
}

// Make f (a winning W-neighbour that conflicts) i's latest witness; the
// earlier ones follow, f's old slot or else the oldest dropped.
__device__ __forceinline__ void tail_wit_record(const TailSmem &s, int T, int i, int f) {
    const int w0 = s.wit[i];
    if (f == w0) return;
    const short a = s.wo[i], b = s.wo[T + i];
    if (f != a) {
        if (f != b) s.wo[2 * T + i] = b;
        s.wo[T + i] = a;
    }
    s.wo[i] = (short)w0;
    s.wit[i] = (short)f;
}

// s.wit of a vertex that kept its color this round: it leaves the worklist in
// the next round's FirstFit pass.
constexpr short kTailKept = -2;

__device__ __forceinline__ unsigned tk_color(unsigned long long x) { return (unsigned)(x >> 32); }
__device__ __forceinline__ unsigned tk_rank(unsigned long long x) { return (unsigned)x; }

// A block of a run.  The tail CTA compacts the runs in place, so they are
// read through the coherent path (plain global loads, cached in L1, which
// sees the CTA's own writes after a __syncthreads), not the read-only one.
__device__ __forceinline__ uint4 ld_run(const uint4 *q) { return *q; }

// Entry k of a 16-byte block of eight 16-bit local ids.
__device__ __forceinline__ int tail_elem(const uint4 &x, int k) {
    const unsigned w = k < 2 ? x.x : (k < 4 ? x.y : (k < 6 ? x.z : x.w));
    return (int)((k & 1) ? (w >> 16) : (w & 0xffffu));
}

// The part of i's run its scan covers: positions [lo, hi), downward (mode 0:
// lower ids win, row-ordered run), upward over the winners (mode 1: higher
// ids win, row-ordered run) or upward over the whole run with the rank test
// (mode 2).
struct TailRange {
    int lo, hi;
};

__device__ __forceinline__ TailRange tail_range(const TailSmem &s, int mode, int i) {
    if (mode == 0) return {0, (int)s.low[i]};
    if (mode == 1) return {(int)s.low[i], (int)s.cnt[i]};
    return {0, (int)s.cnt[i]};
}

// Is local vertex u (entry at run position pos) a conflicting winner?
__device__ __forceinline__ bool tail_conflict(const TailSmem &s, int mode, int u, unsigned c, unsigned mine) {
    const unsigned long long t = s.tk[u];
    return tk_color(t) == c && (mode != 2 || tk_rank(t) > mine);
}

// First scan of an unsettled vertex: a group of kTailGroup lanes, one
// 16-byte block (8 entries) per lane and step, blocks in scan order by lane,
// kTailGroupSteps steps at most; a warp scans 32 / kTailGroup vertices at a
// time.  Vertices whose range goes on past these blocks without a conflict
// are finished by whole warps, segment by segment (tail_scan_segments).
constexpr int kTailGroup = 8;
constexpr int kTailGroupSteps = 1;
constexpr int kTailGroupBlocks = kTailGroup * kTailGroupSteps;

// First conflicting winner of one block in scan order (down: from its top
// entry), positions restricted to [lo, hi); -1 if none.
__device__ __forceinline__ int tail_block_hit(const TailSmem &s, int mode, const uint4 &x, int b, int lo, int hi,
                                              unsigned c, unsigned mine) {
    int hit = -1;
    const bool down = mode == 0;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const int k = down ? kk : 7 - kk;  // visited last wins: the first in scan order
        const int pos = 8 * b + k;
        if (pos < lo || pos >= hi) continue;
        const int u = tail_elem(x, k);
        if (tail_conflict(s, mode, u, c, mine)) hit = u;
    }
    return hit;
}

// Warp scan of four segments of 32 blocks (one block a lane, all four loads
// in flight) of the rest of i's range, from s.res[i] on in scan order: the
// segments j0, j0 + step, j0 + 2 step and j0 + 3 step.  Returns the nearest
// conflicting winner among them as (distance from the start of the rest << 16
// | local id), the same on all lanes, or 0xffffffff.
__device__ __forceinline__ unsigned tail_scan_segments(const Params &p, const TailSmem &s, int mode, int i,
                                                       int j0, int step, unsigned &scanned) {
    const int lane = threadIdx.x & 31;
    const TailRange rg0 = tail_range(s, mode, i);
    const bool down = mode == 0;
    const int lo = down ? rg0.lo : (int)s.res[i], hi = down ? (int)s.res[i] : rg0.hi;
    const uint4 *run = reinterpret_cast<const uint4 *>(p.tadj + s.off[i]);
    const unsigned long long me = s.tk[i];
    const int bl = lo >> 3, bh = (hi - 1) >> 3;
    uint4 x[4];
    int bb[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int d = (j0 + t * step) * 32 + lane;  // distance in blocks from the start
        bb[t] = down ? bh - d : bl + d;
        x[t] = (hi > lo && bb[t] >= bl && bb[t] <= bh) ? ld_run(run + bb[t]) : make_uint4(0, 0, 0, 0);
    }
    unsigned best = 0xffffffffu, n = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (hi <= lo || bb[t] < bl || bb[t] > bh) continue;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int pos = 8 * bb[t] + k;
            if (pos < lo || pos >= hi) continue;
            ++n;
            const int u = tail_elem(x[t], k);
            if (tail_conflict(s, mode, u, tk_color(me), tk_rank(me))) {
                const unsigned dist = (unsigned)(down ? hi - 1 - pos : pos - lo);
                best = min(best, (dist << 16) | (unsigned)u);
            }
        }
    }
    scanned += n;
    return __reduce_min_sync(kFull, best);
}

// Blocks of the rest of i's range (from s.res[i] on).
__device__ __forceinline__ int tail_rest_blocks(const TailSmem &s, int mode, int i) {
    const TailRange rg0 = tail_range(s, mode, i);
    const int lo = mode == 0 ? rg0.lo : (int)s.res[i], hi = mode == 0 ? (int)s.res[i] : rg0.hi;
    return hi > lo ? ((hi - 1) >> 3) - (lo >> 3) + 1 : 0;
}

// Drop the final vertices from i's run, in place and in order, and recount
// the entries below the vertex.  One warp, 128 blocks a step with all their
// loads in flight: a step writes only below its own first block + 128, and
// the next step reads from there on.
__device__ __forceinline__ void tail_compact_run(const Params &p, const TailSmem &s, int i) {
    const int lane = threadIdx.x & 31;
    unsigned short *run = p.tadj + s.off[i];
    const int n = s.cnt[i], lo_old = s.low[i], nb = (n + 7) >> 3;
    unsigned put = 0, low = 0;
    for (int b0 = 0; b0 < nb; b0 += 128) {
        uint4 x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int b = b0 + 32 * t + lane;
            x[t] = b < nb ? ld_run(reinterpret_cast<const uint4 *>(run) + b) : make_uint4(0, 0, 0, 0);
        }
        unsigned keep[4], kl = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int b = b0 + 32 * t + lane;
            keep[t] = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int pos = 8 * b + k;
                if (b < nb && pos < n && tk_color(s.tk[tail_elem(x[t], k)]) != 0) {
                    keep[t] |= 1u << k;
                    kl += pos < lo_old ? 1u : 0u;
                }
            }
        }
        __syncwarp();  // every lane has read its blocks before any write
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const unsigned c = __popc(keep[t]);
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            unsigned at = put + incl - c;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if ((keep[t] >> k) & 1u) run[at++] = (unsigned short)tail_elem(x[t], k);
            put += __shfl_sync(kFull, incl, 31);
        }
        low += __reduce_add_sync(kFull, kl);
        __syncwarp();
    }
    if (lane == 0) {
        s.cnt[i] = (unsigned short)put;
        s.low[i] = (unsigned short)low;
    }
}

// ------------------------------------------------------------ bit-matrix rounds
//
// Once at most kEngMax vertices are left, a round of the general loop above
// still costs five CTA barriers and a few trips to the runs and the winner
// sets in global memory, for little work.  The CTA then switches to a form
// of the same rounds that reads nothing from global memory:
// * the subgraph the survivors induce becomes a bit matrix in shared memory,
//   rows and columns ordered by rank, so that the bits of row v below column
//   v are v's winners under the loser rule and the bits above it the
//   neighbours v wins against.  It is built once: the winners from each
//   survivor's run (only the part that holds winners when the run is in row
//   order), then the rest by transposing 32 x 32 bit blocks;
// * thread v owns survivor v and is the only one to read or write its
//   forbidden-color bitmap (colors 1..256);
// * a round is three passes between CTA barriers:
//   1. FirstFit from the bitmap (a full bitmap: the whole row over the final
//      colors, one warp); v's bit goes into the class set of its tentative
//      color, for the kEngWin colors from the last round's least one up
//      (tentative colors never decrease: bitmaps only gain bits);
//   2. ConflictResolve: v loses iff the part of its row below v and the class
//      set of its color meet, over the words of the class set that are not
//      zero (for a color outside the window, a loop over the winners'
//      tentative colors); keepers commit and join the keeper set;
//   3. the others add the colors of their neighbours in the keeper set to
//      their bitmaps, over the words of the keeper set that are not zero.
// These are the rounds of the general loop (the same bitmaps, tentative
// colors and winners), with the conflict test done on sets.

struct TailStats {
    unsigned long long kdeg, kdegr, nres, sum_w, sum_next;
    unsigned work;
    int kmax;
    long long trounds;
};

// Color cu + 1 (cu < 256) into an 8-word bitmap held in registers.
__device__ __forceinline__ void eng_add_color(unsigned (&add)[8], unsigned cu) {
    if (cu < 256u) {
        const unsigned bit = 1u << (cu & 31), wd = cu >> 5;
#pragma unroll
        for (int j = 0; j < 8; ++j) add[j] |= (wd == (unsigned)j) ? bit : 0u;
    }
}

template <bool kBatched>
__device__ __forceinline__ bool tail_engine(const Params &p, const TailSmem &s, int T, int mode,
                                            unsigned char *raw, const unsigned short *list, unsigned len,
                                            unsigned cbase0, unsigned long long t0, long long &r,
                                            TailStats &st) {
    __shared__ unsigned e_n, e_alive, e_nkeep, e_nfb, e_cmin, e_cbase, e_kz;
    constexpr int S = kEngStride;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kTailThreads / 32;
    const unsigned lt = lanemask_lt();
    unsigned *M = reinterpret_cast<unsigned *>(raw);  // [kEngMax][S]
    unsigned *cls = M + kEngMax * S;                  // [kEngWin][S] class sets
    unsigned *cz = cls + kEngWin * S;                 // [kEngWin] their words that are not zero
    unsigned *K = cz + kEngWin;                       // [32] the round's keepers
    unsigned *tc = K + 32;                            // [kEngMax] tentative color, 0 once final
    int32_t *ev = reinterpret_cast<int32_t *>(tc + kEngMax);
    int32_t *ed = ev + kEngMax;
    unsigned *rk = reinterpret_cast<unsigned *>(ed + kEngMax);  // build: ranks; rounds: full bitmaps
    unsigned *eold = rk + kEngMax;  // the general rounds' local id
    unsigned *eoff = eold + kEngMax;
    unsigned *elo = eoff + kEngMax;
    unsigned *ehi = elo + kEngMax;
    unsigned *ebm = ehi + kEngMax;  // [8][kEngMax] forbidden colors 1..256, plane-major
    unsigned short *map = reinterpret_cast<unsigned short *>(ebm + 8 * kEngMax);  // [kTailMax]
    // ---- the survivors: the list's vertices that did not keep last round
    if (tid == 0) e_n = 0;
    __syncthreads();
    for (unsigned k0 = (unsigned)warp * 32; k0 < len; k0 += kTailThreads) {
        const unsigned k = k0 + lane;
        const int i = k < len ? (int)list[k] : -1;
        const bool sv = i >= 0 && s.wit[i] != kTailKept;
        const unsigned m = __ballot_sync(kFull, sv);
        unsigned at = 0;
        if (lane == 0 && m) at = atomicAdd(&e_n, (unsigned)__popc(m));
        at = __shfl_sync(kFull, at, 0);
        if (sv) s.q[at + __popc(m & lt)] = (unsigned short)i;
    }
    __syncthreads();
    const unsigned E = e_n;
    int i0 = -1;
    unsigned b[8], rank = 0;
    int32_t vid = 0, deg = 0;
    unsigned off = 0;
    TailRange rg{0, 0};
#pragma unroll
    for (int j = 0; j < 8; ++j) b[j] = 0u;
    if ((unsigned)tid < E) {
        i0 = s.q[tid];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = s.bits[j * T + i0];
        vid = s.vid[i0];
        deg = s.deg[i0];
        off = s.off[i0];
        rg = tail_range(s, mode, i0);  // the part of the run that holds the winners
        rank = tk_rank(s.tk[i0]);
    }
    __syncthreads();  // the general loop's arrays are dead from here on
    for (int k = tid; k < kEngMax * S + kEngWin * S + kEngWin + 32 + kEngMax; k += kTailThreads) M[k] = 0u;
    for (int k = tid; k < kTailMax; k += kTailThreads) map[k] = 0xffffu;
    if ((unsigned)tid < E) rk[tid] = rank;
    __syncthreads();
    if ((unsigned)tid < E) {  // index = the number of survivors with a higher rank
        unsigned idx = 0;
        const uint4 *r4 = reinterpret_cast<const uint4 *>(rk);
        const unsigned n4 = E >> 2;
        for (unsigned u = 0; u < n4; ++u) {
            const uint4 x = r4[u];
            idx += (x.x > rank ? 1u : 0u) + (x.y > rank ? 1u : 0u) + (x.z > rank ? 1u : 0u) +
                   (x.w > rank ? 1u : 0u);
        }
        for (unsigned u = n4 << 2; u < E; ++u) idx += rk[u] > rank ? 1u : 0u;
        map[i0] = (unsigned short)idx;
        eold[idx] = (unsigned)i0;
        ev[idx] = vid;
        ed[idx] = deg;
        eoff[idx] = off;
        elo[idx] = (unsigned)rg.lo;
        ehi[idx] = (unsigned)rg.hi;
#pragma unroll
        for (int j = 0; j < 8; ++j) ebm[j * kEngMax + idx] = b[j];
    }
    __syncthreads();
    // ---- the winners of each row, one warp a row: from the winner bit sets
    // written at the hand-over (the row's words gathered through the map of
    // new to old local ids, one ballot a word), else from the run (entries no
    // longer on the worklist map to nothing; a lane takes one 16-byte block
    // and ORs the bits of one word at a time into the row)
    unsigned work = 0;
    if (p.twin) {
        const int MW = p.tail_mw;  // at most 64
        unsigned n0 = 0u, n1 = 0u;  // the next row's bit set, loaded one row ahead
        if ((unsigned)warp < E) {
            const unsigned *tw = p.twin + (size_t)eold[warp] * MW;
            n0 = lane < MW ? __ldg(tw + lane) : 0u;
            n1 = lane + 32 < MW ? __ldg(tw + 32 + lane) : 0u;
        }
        for (unsigned v = (unsigned)warp; v < E; v += nwarps) {
            const unsigned t0 = n0, t1 = n1;
            if (v + nwarps < E) {
                const unsigned *tw = p.twin + (size_t)eold[v + nwarps] * MW;
                n0 = lane < MW ? __ldg(tw + lane) : 0u;
                n1 = lane + 32 < MW ? __ldg(tw + 32 + lane) : 0u;
            }
            for (unsigned w = 0; w <= (v >> 5); ++w) {
                const unsigned u = 32 * w + (unsigned)lane;
                const unsigned o = u < v ? eold[u] : 0u;
                const unsigned a0 = __shfl_sync(kFull, t0, (int)((o >> 5) & 31u));
                const unsigned a1 = __shfl_sync(kFull, t1, (int)((o >> 5) & 31u));
                const unsigned word = (o >> 10) ? a1 : a0;
                const unsigned m = __ballot_sync(kFull, u < v && ((word >> (o & 31)) & 1u));
                if (lane == 0) M[v * S + w] = m;
            }
            if (lane == 0) work += (unsigned)MW * 2u;  // a bit set, in 16-bit entries
        }
    } else for (unsigned v = (unsigned)warp; v < E; v += nwarps) {
        const uint4 *run = reinterpret_cast<const uint4 *>(p.tadj + eoff[v]);
        const int lo = (int)elo[v], hi = (int)ehi[v];
        unsigned *row = M + v * S;
        if (hi > lo) {
            for (int bb = (lo >> 3) + lane; bb <= ((hi - 1) >> 3); bb += 32) {
                const uint4 x = ld_run(run + bb);
                unsigned cw = 0xffffffffu, cbits = 0u;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int pos = 8 * bb + k;
                    if (pos < lo || pos >= hi) continue;
                    const unsigned u = map[tail_elem(x, k)];
                    if (u >= v) continue;  // gone from the worklist, or not a winner
                    if ((u >> 5) != cw) {
                        if (cbits) atomicOr(row + cw, cbits);
                        cw = u >> 5;
                        cbits = 0u;
                    }
                    cbits |= 1u << (u & 31);
                }
                if (cbits) atomicOr(row + cw, cbits);
            }
        }
        if (lane == 0) work += (unsigned)(hi > lo ? hi - lo : 0);
    }
    __syncthreads();
    // ---- the neighbours each row wins against: 32 x 32 blocks of the part
    // below the diagonal, transposed (lane l holds row 32 bi + l of block
    // (bi, bj); column j of the block is row 32 bj + j's word bi)
    {
        const unsigned EB = (E + 31) >> 5;
        for (unsigned q = (unsigned)warp; q < EB * (EB + 1) / 2; q += nwarps) {
            unsigned bi = 0;
            while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
            const unsigned bj = q - bi * (bi + 1) / 2;  // bj <= bi
            const unsigned a = M[(32 * bi + lane) * S + bj];
            __syncwarp();
            unsigned mine = 0u;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const unsigned t = __ballot_sync(kFull, (a >> j) & 1u);
                if (lane == j) mine = t;
            }
            if (mine) M[(32 * bj + lane) * S + bi] |= mine;  // above the diagonal: no winners there
        }
    }
    bool live = (unsigned)tid < E, kept = false;
    if (live) {
        vid = ev[tid];
        deg = ed[tid];
    }
    if (tid == 0) {
        e_alive = E;
        e_nkeep = 0;
        e_nfb = 0;
        e_kz = 0;
        e_cmin = 0xffffffffu;
        e_cbase = cbase0;
    }
    __syncthreads();
    // ---- the rounds
    const unsigned vw = (unsigned)tid >> 5, vbit = 1u << (tid & 31), lowm = vbit - 1u;
    const unsigned wmask = vw >= 31u ? 0xffffffffu : (2u << vw) - 1u;  // words 0 .. vw
    const unsigned *row = M + (live ? tid : 0) * S;
    unsigned long long kdeg = 0, kdegr = 0, nres = 0;
    int kmax = 0;
    bool ok = true;
    for (;; ++r) {
        const unsigned alive = e_alive;
        if (alive == 0) break;
        if (r > p.max_rounds) {
            if (tid == 0) raise_error(p, kErrNoConvergence);
            ok = false;
            break;
        }
        const unsigned cb = e_cbase;
        if (tid == 0) {  // the last round read these before its last barrier
            e_nkeep = 0;
            e_kz = 0;
            st.sum_w += alive;
            if (r <= kTraceCap) p.trace[kTraceFields * (r - 1)] = (long long)alive;
        }
        // 1. FirstFit; class sets written a warp word at a time
        if (kept) {
            tc[tid] = 0u;
            kept = false;
        }
        unsigned c = 0;
        if (live) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const unsigned wv = ebm[j * kEngMax + tid];
                if (c == 0 && ~wv) c = (unsigned)(j * 32 + __ffs(~wv));
            }
            if (c == 0)
                rk[atomicAdd(&e_nfb, 1u)] = (unsigned)tid;  // 256 colors in use
            else
                tc[tid] = c;
        }
        {
            const unsigned sl = (live && c && c - cb < (unsigned)kEngWin) ? c - cb : 0xffffffffu;
            const unsigned grp = __match_any_sync(kFull, sl);
            if (sl != 0xffffffffu && (grp & lt) == 0u) {
                cls[sl * S + vw] = grp;
                atomicOr(cz + sl, 1u << vw);
            }
        }
        const unsigned cm = __reduce_min_sync(kFull, live && c ? c : 0xffffffffu);
        if (lane == 0 && cm != 0xffffffffu) atomicMin(&e_cmin, cm);
        __syncthreads();
        if (e_nfb) {  // full bitmaps: first fit over the final colors of the whole row
            const unsigned nfb = e_nfb;
            for (unsigned k = (unsigned)warp; k < nfb; k += nwarps) {
                const unsigned v = rk[k];
                long long rs, re;
                int32_t vb;
                row_of<kBatched>(p, ev[v], rs, re, vb);
                const unsigned cc = (unsigned)warp_first_fit(p.ci, p.m, p.colors, rs, re, vb, lane, p.n);
                if (lane == 0) {
                    tc[v] = cc;
                    if (cc - cb < (unsigned)kEngWin) {
                        atomicOr(cls + (cc - cb) * S + (v >> 5), 1u << (v & 31));
                        atomicOr(cz + (cc - cb), 1u << (v >> 5));
                    }
                    atomicMin(&e_cmin, cc);
                }
            }
            __syncthreads();
            if (live && c == 0) c = tc[tid];
        }
        if (tid == 0 && r <= kTraceCap) p.trace[kTraceFields * (r - 1) + 1] = (long long)(globaltimer() - t0);
        // 2. ConflictResolve on the winners (the row below v)
        bool keep = false;
        if (live) {
            bool lose = false;
            const unsigned sl = c - cb;
            if (sl < (unsigned)kEngWin) {
                const unsigned *cs = cls + sl * S;
                for (unsigned z = cz[sl] & wmask; z && !lose; z &= z - 1u) {
                    const unsigned w = (unsigned)__ffs(z) - 1u;
                    lose = (row[w] & cs[w] & (w == vw ? lowm : 0xffffffffu)) != 0u;
                }
            } else {
                for (unsigned w = 0; w <= vw && !lose; ++w) {
                    unsigned x = row[w] & (w == vw ? lowm : 0xffffffffu);
                    while (x && !lose) {
                        const unsigned u = (w << 5) + (unsigned)__ffs(x) - 1u;
                        x &= x - 1u;
                        lose = tc[u] == c;
                    }
                }
            }
            if (!lose) {
                keep = true;
                __stcg(p.colors + vid, (int)c);
                kmax = max(kmax, (int)c);
                kdeg += (unsigned long long)deg;
                kdegr += (unsigned long long)deg * (unsigned long long)st.trounds;
            }
        }
        {
            const unsigned km = __ballot_sync(kFull, keep), lm = __ballot_sync(kFull, live);
            if (lane == 0) {
                K[warp] = km;
                if (km) {
                    atomicAdd(&e_nkeep, (unsigned)__popc(km));
                    atomicOr(&e_kz, 1u << warp);
                }
                nres += (unsigned)__popc(lm);
            }
        }
        __syncthreads();
        // 3. the keepers' colors into the others' bitmaps; class sets cleared
        for (int k = tid; k < kEngWin * S; k += kTailThreads) cls[k] = 0u;
        if (tid < kEngWin) cz[tid] = 0u;
        if (keep) {
            live = false;
            kept = true;
        }
        if (live) {
            unsigned add[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) add[j] = 0u;
            for (unsigned z = e_kz; z; z &= z - 1u) {
                const unsigned w = (unsigned)__ffs(z) - 1u;
                for (unsigned x = row[w] & K[w]; x; x &= x - 1u)
                    eng_add_color(add, tc[(w << 5) + (unsigned)__ffs(x) - 1u] - 1u);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (add[j]) ebm[j * kEngMax + tid] |= add[j];
        }
        if (tid == 0) {
            const unsigned left = alive - e_nkeep;
            st.sum_next += left;
            e_alive = left;
            e_nfb = 0;
            if (e_cmin != 0xffffffffu) e_cbase = e_cmin;
            e_cmin = 0xffffffffu;
            if (r <= kTraceCap) {
                p.trace[kTraceFields * (r - 1) + 2] = (long long)(globaltimer() - t0);
                p.trace[kTraceFields * (r - 1) + 3] = (long long)alive;
            }
        }
        ++st.trounds;
        __syncthreads();
    }
    st.work += work;
    st.kdeg += kdeg;
    st.kdegr += kdegr;
    st.nres += nres;
    st.kmax = max(st.kmax, kmax);
    return ok;
}

template <bool kBatched>
__global__ void __launch_bounds__(kTailThreads, 1) sgr_tail_kernel(const Params p) {
    Counters *ctr = p.ctr;
    if (__ldcg(&ctr->tail) == 0) return;
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int T = tail_stride(p.tail_max);
    const TailSmem s = tail_smem(s_raw, T);
    __shared__ unsigned s_nq, s_nlq, s_nfb, s_alive, s_nkeep, s_nnext, s_compact_at, s_cbase, s_cmin;
    // winner bit sets (hand-overs up to kTailMaskMax): class masks, per
    // tentative color cbase .. cbase + kTailClasses - 1, of the vertices that
    // hold it this round, after the per-vertex arrays
    const bool masks = p.twin != nullptr;
    const int MW = p.tail_mw;
    unsigned *cls = reinterpret_cast<unsigned *>(s_raw + (size_t)T * 80);
    __shared__ unsigned long long s_D, s_kdeg, s_kdegr, s_work, s_nres;
    __shared__ int s_kmax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kTailThreads / 32;
    const int nT = (int)__ldcg(&ctr->tail_n);
    const int rule = p.rule;
    const bool sorted = __ldcg(&ctr->unsorted_pairs) == __ldcg(&ctr->boundary_pairs);
    const int mode = (sorted && rule <= 1) ? rule : 2;
    const unsigned long long t0 = __ldcg(&ctr->t_start);
    long long r = __ldcg(&ctr->round);
    // ---- load the worklist's state
    if (tid == 0) {
        s_D = 0;
        s_alive = (unsigned)nT;
        s_kmax = 0;
        s_nq = s_nlq = s_nfb = s_nkeep = s_nnext = 0;
        s_compact_at = (unsigned)nT / 8;
        s_kdeg = s_work = 0;
        s_cbase = 1;  // no color is lower
        s_cmin = 0xffffffffu;
    }
    if (masks)
        for (int k = tid; k < kTailClasses * MW; k += kTailThreads) cls[k] = 0u;
    __syncthreads();
    // every thread's vertices (kLoadPer at most) load together, one step of
    // the chain vertex -> bitmaps, witness -> its color -> its local id at a
    // time, so that each step has all of its loads in flight
    constexpr int kLoadPer = (kTailMax + kTailThreads - 1) / kTailThreads;
    unsigned long long dsum = 0;
    int32_t lv[kLoadPer], lw[kLoadPer];
#pragma unroll
    for (int k = 0; k < kLoadPer; ++k) {
        const int i = tid + k * kTailThreads;
        lv[k] = i < nT ? __ldcg(p.tlist + i) : -1;
    }
#pragma unroll
    for (int k = 0; k < kLoadPer; ++k) {
        const int i = tid + k * kTailThreads;
        lw[k] = -1;
        if (i < nT) {
            const int32_t v = lv[k];
            const unsigned d = __ldcg(p.tdeg + i);
            s.vid[i] = v;
            s.deg[i] = (int32_t)d;
            s.off[i] = __ldcg(p.toff + i);
            s.cnt[i] = (unsigned short)__ldcg(p.tcnt + i);
            s.low[i] = (unsigned short)__ldcg(p.tlow + i);
#pragma unroll
            for (int j = 0; j < 8; ++j) s.bits[j * T + i] = __ldcg(p.bm + (size_t)j * p.np + v);
            lw[k] = wit_first(p, v);  // the latest witness
            s.al[i] = (unsigned short)i;
            dsum += d;
        }
    }
    // the witnesses, if they are still on the worklist (each is a neighbour
    // that wins against v: the grid only records those); the grid's slots 1-3
    // become the earlier ones
#pragma unroll
    for (int k = 0; k < kLoadPer; ++k) {
        const int i = tid + k * kTailThreads;
        if (i >= nT) continue;
        const int4 o = __ldcg(reinterpret_cast<const int4 *>(p.wold) + lv[k]);
        const int32_t w[4] = {lw[k], o.x, o.y, o.z};
        bool on[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) on[j] = w[j] >= 0 && w[j] < p.n && __ldcg(p.colors + w[j]) <= 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const short l = (short)(on[j] ? __ldcg(p.tloc + w[j]) : -1);
            if (j == 0)
                s.wit[i] = l;
            else
                s.wo[(j - 1) * T + i] = l;
        }
    }
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
    if (lane == 0 && dsum) atomicAdd(&s_D, dsum);
    __syncthreads();
    // ranks: lower id wins (rule 0), higher id wins (rule 1), or higher
    // degree, then lower id (rule 2: the rank is the position among W_r)
    for (int i = tid; i < nT; i += kTailThreads) {
        unsigned rank;
        if (rule == 0) {
            rank = 0x7fffffffu - (unsigned)s.vid[i];
        } else if (rule == 1) {
            rank = (unsigned)s.vid[i];
        } else {
            rank = 0;
            const int di = s.deg[i], vi = s.vid[i];
            for (int j = 0; j < nT; ++j) {
                const int dj = s.deg[j], vj = s.vid[j];
                rank += (di != dj ? di > dj : vi < vj) ? 1u : 0u;
            }
        }
        s.tk[i] = (1ull << 32) | rank;  // on the worklist (any nonzero color)
    }
    __syncthreads();
    // Per-thread statistics, reduced once after the last round: keepers'
    // degrees (K) and the same weighted by the local round they kept in (J),
    // so that sum over rounds of D_r = R D_0 - ((R - 1) K - J); unsettled
    // vertices (rescans); largest color; W-adjacency entries read.
    unsigned long long kdeg = 0, kdegr = 0, nres = 0;
    int kmax = 0;
    unsigned work = 0;
    unsigned long long sum_w = 0, sum_next = 0;  // thread 0
    long long trounds = 0;
    int par = 0;
    unsigned lprev = (unsigned)nT;  // length of the list this round's FirstFit pass reads
    bool ok = true;
    const unsigned lt = lanemask_lt();
    const int mw4 = (nT + 127) / 128;  // 16-byte words of a bit set that hold local ids
    bool engine = false;
    for (;; ++r) {
        const unsigned alive = s_alive;
        if (alive == 0) break;
        if (alive <= (unsigned)kEngMax) {  // the bit-matrix rounds take the rest
            engine = true;
            break;
        }
        // every tentative color from a bitmap is at least the last round's
        // least one (bitmaps only gain bits, the worklist only shrinks)
        const unsigned cbase = s_cbase;
        unsigned cmin = 0xffffffffu;
        if (r > p.max_rounds) {
            if (tid == 0) raise_error(p, kErrNoConvergence);
            ok = false;
            break;
        }
        if (tid == 0) {
            // the previous round's counters have been read by every thread
            // (before the round barrier), and nothing adds to them before
            // this round's first barrier
            s_nkeep = 0;
            s_nlq = 0;
            s_nq = 0;
            sum_w += alive;
            if (r <= kTraceCap) p.trace[kTraceFields * (r - 1)] = (long long)alive;
        }
        // ---- FirstFit from the bitmaps.  The previous round's keepers leave
        // the worklist here (their tentative color becomes 0), and the others
        // form this round's list, appended a warp at a time.
        const unsigned short *al_prev = s.al + par * T;
        unsigned short *al = s.al + (par ^ 1) * T;
        par ^= 1;
        for (unsigned k0 = (unsigned)warp * 32; k0 < lprev; k0 += kTailThreads) {
            const unsigned k = k0 + lane;
            const int i = k < lprev ? (int)al_prev[k] : -1;
            bool stay = false;
            if (i >= 0) {
                const unsigned long long t = s.tk[i];
                if (s.wit[i] == kTailKept) {
                    s.tk[i] = (unsigned long long)tk_rank(t);
                } else {
                    stay = true;
                    unsigned c = 0;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const unsigned wv = s.bits[j * T + i];
                        if (c == 0 && ~wv) c = (unsigned)(j * 32 + __ffs(~wv));
                    }
                    if (c == 0) s.q[atomicAdd(&s_nfb, 1u)] = (unsigned short)i;  // 256 colors in use
                    s.tk[i] = ((unsigned long long)(c ? c : 1u) << 32) | tk_rank(t);
                    if (c) {
                        cmin = min(cmin, c);
                        if (masks && c - cbase < (unsigned)kTailClasses)
                            atomicOr(cls + (c - cbase) * MW + (i >> 5), 1u << (i & 31));
                    }
                }
            }
            const unsigned m = __ballot_sync(kFull, stay);
            unsigned at = 0;
            if (lane == 0 && m) at = atomicAdd(&s_nnext, (unsigned)__popc(m));
            at = __shfl_sync(kFull, at, 0);
            if (stay) al[at + __popc(m & lt)] = (unsigned short)i;
        }
        cmin = __reduce_min_sync(kFull, cmin);
        if (lane == 0 && cmin != 0xffffffffu) atomicMin(&s_cmin, cmin);
        __syncthreads();
        if (s_nfb) {  // full bitmaps: first fit over the final colors of the whole row
            const unsigned nfb = s_nfb;
            for (unsigned k = warp; k < nfb; k += nwarps) {
                const int i = s.q[k];
                long long rs, re;
                int32_t vb;
                row_of<kBatched>(p, s.vid[i], rs, re, vb);
                const int c = warp_first_fit(p.ci, p.m, p.colors, rs, re, vb, lane, p.n);
                if (lane == 0) s.tk[i] = ((unsigned long long)c << 32) | tk_rank(s.tk[i]);
            }
            __syncthreads();
            if (tid == 0) s_nfb = 0;
        }
        if (alive <= s_compact_at) {  // most of the worklist has gone: drop it from the runs
            for (unsigned k = warp; k < alive; k += nwarps) tail_compact_run(p, s, al[k]);
            __syncthreads();
            if (tid == 0) s_compact_at = alive / 2;
        }
        if (tid == 0 && r <= kTraceCap)
            p.trace[kTraceFields * (r - 1) + 1] = (long long)(globaltimer() - t0);
        // ---- ConflictResolve: the witness first (a vertex that loses again
        // to the same neighbour is settled by one read), then a scan of the
        // run for the others, kTailGroup lanes a vertex
        for (unsigned k0 = (unsigned)warp * 32; k0 < alive; k0 += kTailThreads) {
            const unsigned k = k0 + lane;
            const int i = k < alive ? (int)al[k] : -1;
            bool uns = false;
            if (i >= 0) {
                const unsigned c = tk_color(s.tk[i]);
                const int w = s.wit[i];
                uns = !(w >= 0 && tk_color(s.tk[w]) == c);
                if (uns) {  // the earlier witnesses; one that settles it moves to slot 0
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int wj = s.wo[j * T + i];
                        if (uns && wj >= 0 && tk_color(s.tk[wj]) == c) {
                            uns = false;
                            s.wo[j * T + i] = (short)w;
                            s.wit[i] = (short)wj;
                        }
                    }
                }
            }
            const unsigned um = __ballot_sync(kFull, uns);
            unsigned at = 0;
            if (lane == 0 && um) {
                at = atomicAdd(&s_nq, (unsigned)__popc(um));
                nres += (unsigned)__popc(um);
            }
            at = __shfl_sync(kFull, at, 0);
            if (uns) s.q[at + __popc(um & lt)] = (unsigned short)i;
        }
        __syncthreads();
        const unsigned nq = s_nq;
        {  // first blocks of every unsettled vertex: kTailGroup lanes each
            constexpr int kPerWarp = 32 / kTailGroup;
            const int g = lane / kTailGroup, gl = lane % kTailGroup;
            const unsigned gmask = ((1u << kTailGroup) - 1u) << (g * kTailGroup);
            const bool down = mode == 0;
            for (unsigned base = (unsigned)warp * kPerWarp; base < nq; base += (unsigned)nwarps * kPerWarp) {
                const unsigned idx = base + g;
                const bool act = idx < nq;
                const int i = act ? (int)s.q[idx] : 0;
                const TailRange rg = act ? tail_range(s, mode, i) : TailRange{0, 0};
                const unsigned long long me = s.tk[i];
                const uint4 *run = reinterpret_cast<const uint4 *>(p.tadj + s.off[i]);
                const int bl = rg.lo >> 3, bh = rg.hi > rg.lo ? (rg.hi - 1) >> 3 : bl - 1;
                const int nblk = bh - bl + 1;
                // its color has a class mask: the winners that hold it are the
                // bits of (its winner set) & (the class), 16 bytes a lane and step
                const unsigned cme = tk_color(me);
                const bool mk = act && masks && cme <= 256 && cme - cbase < (unsigned)kTailClasses;
                int mhit = -1;
                if (mk) {
                    const uint4 *wr = reinterpret_cast<const uint4 *>(p.twin + (size_t)i * MW);
                    const uint4 *cr = reinterpret_cast<const uint4 *>(cls + (cme - cbase) * MW);
                    for (int k4 = gl; k4 < mw4; k4 += kTailGroup) {
                        const uint4 a = __ldg(wr + k4), b = cr[k4];
                        const unsigned x[4] = {a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w};
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            if (x[w]) mhit = max(mhit, 32 * (4 * k4 + w) + 31 - __clz(x[w]));
                        work += 8;
                    }
                }
#pragma unroll
                for (int o = kTailGroup / 2; o > 0; o >>= 1) mhit = max(mhit, __shfl_xor_sync(kFull, mhit, o));
                int found = -1;
                for (int step = 0; step < kTailGroupSteps; ++step) {
                    const int d = step * kTailGroup + gl;
                    const bool have = act && !mk && found < 0 && d < nblk;
                    int hit = -1;
                    if (have) {
                        const int b = down ? bh - d : bl + d;
                        hit = tail_block_hit(s, mode, ld_run(run + b), b, rg.lo, rg.hi, tk_color(me), tk_rank(me));
                        work += 8;
                    }
                    const unsigned gb = __ballot_sync(kFull, hit >= 0) & gmask;
                    const int src = gb ? __ffs(gb) - 1 : lane;
                    const int h = __shfl_sync(kFull, hit, src);
                    if (gb && found < 0) found = h;
                    if (!__any_sync(kFull, act && !mk && found < 0 && (step + 1) * kTailGroup < nblk)) break;
                }
                if (mk) found = mhit;
                if (act && gl == 0) {
                    if (found >= 0) {
                        tail_wit_record(s, T, i, found);
                    } else if (mk || nblk <= kTailGroupBlocks) {  // no winner with its color: keeps it
                        const unsigned c = tk_color(me);
                        s.kq[atomicAdd(&s_nkeep, 1u)] = (unsigned short)i;
                        s.wit[i] = kTailKept;
                        __stcg(p.colors + s.vid[i], (int)c);
                        kmax = max(kmax, (int)c);
                        kdeg += (unsigned long long)s.deg[i];
                        kdegr += (unsigned long long)s.deg[i] * (unsigned long long)trounds;
                    } else {  // the range goes on: a warp finishes it
                        s.res[i] = (unsigned short)(down ? 8 * (bh - kTailGroupBlocks + 1) : 8 * (bl + kTailGroupBlocks));
                        const unsigned q = atomicAdd(&s_nlq, 1u);
                        s.lq[q] = (unsigned short)i;
                        s.lbest[q] = 0xffffffffu;
                    }
                }
            }
        }
        __syncthreads();
        const unsigned nlq = s_nlq;
        if (nlq) {  // the rest of long scans: 32-block segments over 32 / nlq warps per vertex
            const unsigned wpe = max(1u, (unsigned)nwarps / nlq), stride = (unsigned)nwarps / wpe;
            for (unsigned k = warp / wpe; k < nlq && warp / wpe < stride; k += stride) {
                const int i = s.lq[k];
                const int nseg = (tail_rest_blocks(s, mode, i) + 31) >> 5;
                for (int j0 = (int)(warp % wpe); j0 < nseg; j0 += 4 * (int)wpe) {
                    const unsigned b = tail_scan_segments(p, s, mode, i, j0, (int)wpe, work);
                    if (b != 0xffffffffu) {  // the nearer segments are other warps' or scanned already
                        if (lane == 0) atomicMin(s.lbest + k, b);
                        break;
                    }
                }
            }
            __syncthreads();
            for (unsigned k = tid; k < nlq; k += kTailThreads) {
                const int i = s.lq[k];
                const unsigned b = s.lbest[k];
                if (b != 0xffffffffu) {
                    tail_wit_record(s, T, i, (int)(b & 0xffffu));
                } else {
                    const unsigned c = tk_color(s.tk[i]);
                    s.kq[atomicAdd(&s_nkeep, 1u)] = (unsigned short)i;
                    s.wit[i] = kTailKept;
                    __stcg(p.colors + s.vid[i], (int)c);
                    kmax = max(kmax, (int)c);
                    kdeg += (unsigned long long)s.deg[i];
                    kdegr += (unsigned long long)s.deg[i] * (unsigned long long)trounds;
                }
            }
        }
        __syncthreads();
        if (masks)  // every class mask has been read
            for (int k = tid; k < kTailClasses * MW; k += kTailThreads) cls[k] = 0u;
        // ---- keepers record their colors at their W-neighbours: 32-block
        // segments over 32 / nk warps per keeper, four segments a warp with all
        // loads in flight.  Their tentative colors stay until the next FirstFit
        // pass.
        const unsigned nk = s_nkeep;
        if (nk) {
            const unsigned wpk = max(1u, (unsigned)nwarps / nk), stride = (unsigned)nwarps / wpk;
            for (unsigned k = warp / wpk; k < nk && warp / wpk < stride; k += stride) {
                const int i = s.kq[k];
                const unsigned c = tk_color(s.tk[i]);
                if (c > 256) continue;
                unsigned *plane = s.bits + (size_t)((c - 1) >> 5) * T;
                const unsigned bit = 1u << ((c - 1) & 31);
                const uint4 *run = reinterpret_cast<const uint4 *>(p.tadj + s.off[i]);
                const int n = s.cnt[i], nb = (n + 7) >> 3, nseg = (nb + 31) >> 5;
                for (int j0 = (int)(warp % wpk); j0 < nseg; j0 += 4 * (int)wpk) {
                    uint4 x[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int b = (j0 + t * (int)wpk) * 32 + lane;
                        x[t] = b < nb ? ld_run(run + b) : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int b = (j0 + t * (int)wpk) * 32 + lane;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk)
                            if (b < nb && 8 * b + kk < n) atomicOr(plane + tail_elem(x[t], kk), bit);
                    }
                }
                if (lane == 0 && warp % wpk == 0) work += (unsigned)n;
            }
        }
        if (tid == 0) {
            const unsigned left = alive - nk;
            sum_next += left;
            s_alive = left;
            s_nnext = 0;  // every append of this round came before its first barrier
            if (s_cmin != 0xffffffffu) s_cbase = s_cmin;
            s_cmin = 0xffffffffu;
            if (r <= kTraceCap) {
                p.trace[kTraceFields * (r - 1) + 2] = (long long)(globaltimer() - t0);
                p.trace[kTraceFields * (r - 1) + 3] = (long long)nq;
            }
        }
        lprev = alive;
        ++trounds;
        __syncthreads();  // bitmaps and the counters of the next round are complete
    }
    if (engine) {
        TailStats st{kdeg, kdegr, nres, sum_w, sum_next, work, kmax, trounds};
        ok = tail_engine<kBatched>(p, s, T, mode, s_raw, s.al + par * T, lprev, s_cbase, t0, r, st);
        kdeg = st.kdeg;
        kdegr = st.kdegr;
        nres = st.nres;
        sum_w = st.sum_w;
        sum_next = st.sum_next;
        work = st.work;
        kmax = st.kmax;
        trounds = st.trounds;
    }
    // ---- statistics of all rounds: one reduction
    unsigned long long wsum = work;
    for (int o = 16; o > 0; o >>= 1) {
        wsum += __shfl_xor_sync(kFull, wsum, o);
        kdeg += __shfl_xor_sync(kFull, kdeg, o);
        kdegr += __shfl_xor_sync(kFull, kdegr, o);
        nres += __shfl_xor_sync(kFull, nres, o);
        kmax = max(kmax, __shfl_xor_sync(kFull, kmax, o));
    }
    if (tid == 0) s_kdeg = s_kdegr = s_work = s_nres = 0;
    __syncthreads();
    if (lane == 0) {
        if (wsum) atomicAdd(&s_work, wsum);
        if (kdeg) atomicAdd(&s_kdeg, kdeg);
        if (kdegr) atomicAdd(&s_kdegr, kdegr);
        if (nres) atomicAdd(&s_nres, nres);
        if (kmax) atomicMax(&s_kmax, kmax);
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned long long R = (unsigned long long)trounds;
        const unsigned long long sum_d = R ? R * s_D - ((R - 1) * s_kdeg - s_kdegr) : 0;
        if (s_work) atomicAdd(&ctr->tail_entries, s_work);
        if (s_kmax) atomicMax(&ctr->kmax, s_kmax);
        atomicAdd(&ctr->sum_w, sum_w);
        atomicAdd(&ctr->sum_d, sum_d);
        atomicAdd(&ctr->sum_next, sum_next);
        atomicAdd(&ctr->sum_rescan, s_nres);
        ctr->tail_rounds = trounds;
        if (ok) {
            ctr->rounds = r - 1;
            ctr->round = r;
        }
    }
}
