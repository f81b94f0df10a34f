// sgr_internal.cuh -- device-side state shared by the kernels and the C ABI.
//
// Data layout in device memory (one coloring call):
//   colors[n]            int32; > 0 final (or, in fast mode, live) color,
//                        < 0 tentative color of the current round (det mode),
//                        0 uncolored.
//   light lists lw[2]    vertex ids of degree <= light_max, double buffered by
//                        round parity (Algorithm 7's W_in / W_out swap).
//   medium lists mw[2]   vertex ids of degree in (light_max, chunk].
//   hub lists hw[2]      hub slot ids (degree > chunk) + chunk base hcb[2].
//   det unsettled lists  ul/um/uh(+ucb), by parity: the part of W_r whose
//                        witness did not settle it in FirstFit, for ConflictResolve.
//   hub slots            hvert (slot -> vertex), hbase (offset of the slot's
//                        forbidden-color bitmap in hbits, fast mode), hdone /
//                        hconf (per-round completion counter and conflict flag).
//   bm[8][np]            det mode: bit c-1 of plane (c-1)/32 at vertex v is set
//                        once a neighbour of v has committed color c (c <= 256).
//   lowdeg[n]            det mode: entries below v in its (ascending) row.
//   witness[n]           det mode: the neighbour that beat v last time, or -1.
//   wold[4n]             det mode: the four before it (16 bytes a vertex),
//                        most recent first, -1 where there is none.
//   hub scatter list     det mode: hubs committed this round (slot + chunk
//                        base), whose colors are scattered at the next round.
//   activation lists     det mode al/am/ah(+acb), by parity: the worklist
//                        vertices whose tentative color a commit of the last
//                        round made stale (a neighbour committed that color).
//   astamp[n]            det mode: the round v was last put on an activation list.
//   vslot[n]             det mode: hub slot of v, or -1 (light) / -2 (medium).
//   tail arrays          det mode: the last rounds in one CTA (sgr_tail.cuh):
//                        tlist (local id -> vertex), tloc[n] (vertex -> local
//                        id), per local vertex the start / count of its
//                        W-neighbours in tadj (16-bit local ids) and the
//                        chunk prefix of the build.
//   Counters             list sizes, grid barrier, max
//                        color so far, error code, statistics.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "sgrcolor.h"

namespace sgr {

constexpr int kBlock = 256;                      // threads per CTA
constexpr int kWarps = kBlock / 32;
constexpr int kLightUnroll = 4;                  // 32-vertex sub-tiles per warp and light tile
constexpr int kLightTile = kBlock * kLightUnroll;
constexpr int kSlowCap = 2 * kLightTile;          // det: queued slow vertices per CTA
constexpr int kPushCap = 4096;                   // det: vertices staged per CTA before a list append
constexpr int kScatterChunk = 128;               // det: entries per hub-scatter work item (one step)
constexpr int kMinBlocks = 3;                    // CTAs per SM the register budget targets
constexpr int kLightMaxStage = 32;               // largest light degree (staged rows per lane)
constexpr int kTraceCap = 1 << 16;               // rounds recorded in the timeline
constexpr int kTraceFields = 4;                  // |W_r|, ns at end of phase A / phase B, rescans
constexpr unsigned long long kWaitTimeoutNs = 4000000000ull;  // default limit of a bounded device wait
constexpr int kTailThreads = 1024;               // threads of the tail CTA
constexpr int kTailMax = 2880;                   // largest |W_r| the tail CTA takes (shared memory)
constexpr int kTailDefault = 2048;               // default hand-over size
constexpr int kTailChunk = 1024;                 // row entries per warp item of the tail build
constexpr long long kTailCapEntries = 24ll << 20;  // largest W-adjacency (16-bit entries)
// Shared memory of the tail CTA for hand-over size t (per local vertex: 64-bit
// state, 8 bitmap words, four 32-bit and twelve 16-bit fields; arrays strided
// by t rounded up to 8).
constexpr int kTailMaskMax = 2048;               // largest hand-over with winner bit sets
constexpr int kTailClasses = 32;                 // tentative colors with a class bit set per round
// 32-bit words of one bit set over the local ids of a hand-over of size t
// (a multiple of four: rows start on 16 bytes).
constexpr int tail_mask_words(int t) { return ((t + 31) / 32 + 3) & ~3; }
constexpr size_t tail_smem_bytes(int t) {
    return (size_t)((t + 7) & ~7) * (8 + 8 * 4 + 4 * 4 + 12 * 2) + 64 +
           (t <= kTailMaskMax ? (size_t)kTailClasses * tail_mask_words(t) * 4 : 0);
}
// The tail CTA's bit-matrix rounds (at most kEngMax vertices left, one a
// thread): the induced subgraph as kEngMax rows of kEngStride words (one
// word of padding, so that the threads of a warp read a column without bank
// conflicts), kEngWin class sets and their nonzero-word masks, the keeper
// set, tentative colors, vertex ids and degrees; and, only while the matrix
// is built, ranks, the general rounds' local ids, run offsets and ranges,
// bitmaps and the map from those local ids.
constexpr int kEngMax = 512;
constexpr int kEngStride = kEngMax / 32 + 1;
constexpr int kEngWin = 32;
constexpr size_t kEngBytes =
    4 * ((size_t)kEngMax * kEngStride + (size_t)kEngWin * kEngStride + kEngWin + 32 +
         (1 + 2 + 1 + 4 + 8) * (size_t)kEngMax) +
    2 * (size_t)kTailMax;
constexpr size_t tail_launch_smem(int t) {
    return tail_smem_bytes(t) > kEngBytes ? tail_smem_bytes(t) : kEngBytes;
}

constexpr int kErrNoConvergence = SGR_ERR_NO_CONVERGENCE;
constexpr int kErrTimeout = SGR_ERR_TIMEOUT;

// The first kHotBytes of Counters are the fields every CTA reads after a
// grid barrier; one warp per CTA copies them into shared memory at each
// barrier (hot_counters() in sgr_kernels.cu), so that the grid's reads do
// not all go to the same L2 line.  The barrier's arrival counter has a line
// of its own.
constexpr int kHotBytes = 256;

struct Counters {
    // ---- hot block (read through the per-CTA snapshot)
    unsigned int nl[2];             // light list sizes by round parity
    unsigned int nm[2];             // medium list sizes
    unsigned long long h64[2];      // hub lists: (entries << 32) | total chunks
    unsigned int nul[2], num[2];    // det: unsettled light / medium vertices of the round
    unsigned long long uh64[2];     // det: unsettled hubs (entries << 32 | chunks)
    unsigned int nal[2], nam[2];    // det: activated light / medium vertices
    unsigned long long ah64[2];     // det: activated hubs (entries << 32 | chunks)
    unsigned long long adeg[2];     // det: degree sum of the activated vertices
    unsigned long long wcount;      // det: |W_r|, vertices not yet committed
    unsigned long long sc64;        // hub scatter list: (entries << 32) | total chunks
    unsigned long long dcur;        // det: degree sum of the current worklist
    int kmax;                       // largest committed color
    int err;                        // 0 or a negative status
    unsigned long long hot_pad[14];
    // ---- grid barrier: arrivals (bits 0..62), error flag (bit 63)
    unsigned long long bar;
    unsigned long long bar_pad[15];
    // ---- the rest
    unsigned long long nroots;      // det: vertices with no entry below them (round-1 keepers on ascending rows)
    unsigned long long t_start;     // globaltimer at the start of the launch that ran init
    int handoff;                    // det: init handed the rounds to the activation-list kernel
    int tail;                       // det: the rounds continue in the tail CTA
    int tail_fail;                  // det: the W-adjacency would not fit; rounds stay on the grid
    unsigned tail_n;                // det: |W_r| at the hand-over (local ids 0 .. tail_n-1)
    long long tail_rounds;          // det: rounds the tail CTA ran
    unsigned long long sum_touch;   // det: worklist entries the grid phases visited
    unsigned long long sum_dep;     // det: row entries read to find witness dependents
    unsigned long long tail_entries;  // det: W-adjacency entries the tail CTA read
    unsigned long long tail_build;  // det: row entries the tail hand-over scanned
    unsigned int nslots;            // hub slots handed out
    unsigned int hwords;            // hub bitmap words handed out
    unsigned long long unsorted_pairs;   // adjacent col_idx pairs with a[i] >= a[i+1]
    unsigned long long boundary_pairs;   // ... of them across row boundaries
    unsigned long long sum_w, sum_d, sum_dscan, sum_next, sum_scatter, sum_rescan;
    unsigned long long nslow;       // det: worklist vertices that rescanned their row this round
    long long rounds;
    long long round;                // resumable launches: the next round to run
    long long t_init_ns;            // globaltimer: end of the init pass (after its barrier)
};
static_assert(offsetof(Counters, err) + sizeof(int) <= kHotBytes, "hot fields fit the snapshot");
static_assert(offsetof(Counters, bar) == kHotBytes, "the barrier counter starts its own line");

struct Params {
    const int32_t *ro;
    const int32_t *ci;
    const int32_t *gid;        // batched: vertex -> graph id
    const long long *vbase;    // batched: graph -> first global vertex
    const long long *ebase;    // batched: graph -> first global entry
    const long long *robase;   // batched: graph -> index of its first row offset in ro
    long long m;               // total col_idx entries
    int32_t n;                 // total vertices
    int32_t *colors;
    int32_t *lw[2];
    int32_t *mw[2];
    int32_t *hw[2];
    unsigned int *hcb[2];
    int32_t *ul[2];            // det: light vertices the witness did not settle (parity of r)
    int32_t *um[2];            // det: medium vertices the witness did not settle
    int32_t *uh[2];            // det: hub slots the witness did not settle
    unsigned *uitem[2];        // det (optional): ConflictResolve work item -> entry of uh (lower-part items)
    int32_t *uvert[2];         // det (optional): entry of uh -> vertex
    unsigned *urec[2];         // det (optional): per lower-part work item of uh, a 32-byte record
                               //   {v, slot, tentative color, vb | start (64-bit), length, items}
    unsigned int *ucb[2];      // det: their chunk bases
    int32_t *hvert;
    unsigned int *hbase;
    unsigned int *hbits;
    unsigned long long *hdone; // per hub slot: finished items (low word), conflicts (high word, det)
    unsigned int *hconf;
    unsigned int *bm;          // det: 8 planes of np words
    long long np;              // plane stride (>= n, multiple of 64)
    int32_t *lowdeg;           // det
    int32_t *witness;          // det: the neighbour that last beat v, or -1
    int32_t *wold;             // det: [4n] the four neighbours that beat v before it, or -1
    int32_t *al[2];            // det: activation lists (light, medium, hub slots + chunk bases)
    int32_t *am[2];
    int32_t *ah[2];
    unsigned int *acb[2];
    int32_t *astamp;           // det: round v was last activated for (zero-initialised)
    int32_t *vslot;            // det: hub slot, -1 light, -2 medium
    int front_ok;              // det: the activation lists are allocated
    int front_policy;          // det: 0 when few round-1 keepers, 1 never, 2 always
    int tail_max;              // det: |W_r| at or below which the rounds go to the tail CTA (0: never)
    long long tail_cap;        // det: capacity of tadj in entries
    int32_t *tlist;            // det tail: local id -> vertex (tail_max)
    int32_t *tloc;             // det tail: vertex -> local id (n; valid on W_r)
    unsigned *toff;            // det tail: start of each local vertex's W-neighbours in tadj (tail_max + 1)
    unsigned *tcnt;            // det tail: number of W-neighbours (tail_max)
    unsigned *tlow;            // det tail: W-neighbours below the vertex (tail_max)
    unsigned *tdeg;            // det tail: degree (tail_max)
    unsigned *tcp;             // det tail: chunk prefix of the build (tail_max + 1)
    unsigned *tcc;             // det tail: per chunk, its W-neighbours (tail_chunks)
    unsigned *tcm;             // det tail: per chunk, its local vertex (tail_chunks)
    int tail_chunks;           // det tail: capacity of tcc / tcm
    unsigned short *tadj;      // det tail: W-neighbours as local ids, 16-byte aligned runs
    unsigned short *tstage;    // det tail: the same per chunk, kTailChunk entries a chunk
    unsigned *twin;            // det tail: per local vertex, the bit set of the W-neighbours that
                               // win against it (tail_mw words a row), or null
    int tail_mw;               // det tail: words per row of twin
    int32_t *sw;               // det: hub scatter list slots
    unsigned int *scb;         // det: hub scatter list chunk bases
    Counters *ctr;
    long long *trace;
    int light_max;             // <= kLightMaxStage
    int chunk;                 // hub chunk edges; medium degree bound
    int rule;                  // 0 low keeps, 1 low loses, 2 degree
    long long max_rounds;
    unsigned long long wait_ns;  // limit of every bounded device-side wait (grid barriers)
    unsigned int nblocks;
    int resume;                // 1: skip init and continue from Counters::round
    int resume_sorted;         // resume: every resident graph has ascending rows
    long long rounds_per_launch;  // resume: rounds to advance before returning
};

// Scratch sizes for a graph of n vertices / m entries under a chunk size.
struct ScratchPlan {
    size_t hub_max;     // upper bound on hub vertices
    size_t hub_words;   // upper bound on hub bitmap words
};

inline ScratchPlan plan_scratch(long long n, long long m, int chunk) {
    ScratchPlan p;
    long long h = m / (chunk + 1) + 1;
    if (h > n) h = n;
    if (h < 1) h = 1;
    p.hub_max = (size_t)h;
    p.hub_words = (size_t)((m + 2 * h) / 32 + 2 * h + 8);
    return p;
}

// Host-side shared state (implemented in sgr_api.cu).
sgr_tuning tuning_snapshot();
std::mutex &device_launch_mutex(int device);
unsigned long long wait_limit_ns();  // sgr_set_wait_limit, or kWaitTimeoutNs
// The single-graph launches with caller-owned scratch (caller holds the
// device launch mutex); used by the server for requests it colors alone.
size_t single_scratch_bytes(int32_t n, long long m);
int color_single_in(char *base, size_t cap, int32_t n, long long m, const int32_t *ro, const int32_t *ci,
                    int32_t *colors, int mode, cudaStream_t st, int32_t *k_out, long long *rounds_out);
// Host-side fault injection (sgr_debug_inject): true when this device
// allocation must fail as out of memory; the extra CTAs the next coloring
// launch's grid barriers wait for (0 normally; consumed by the call).
bool inject_alloc_failure();
unsigned inject_barrier_extra();

// Launches (implemented in sgr_kernels.cu).
int occupancy_blocks_per_sm(bool fast, bool batched, int *out);
cudaError_t launch_color(const Params &p, bool fast, bool batched, int grid, cudaStream_t s);
// Deterministic rounds on the activation lists (after an init launch that set
// Counters::handoff; returns at once if it did not).
int occupancy_blocks_per_sm_front(bool batched, int *out);
cudaError_t launch_color_front(const Params &p, bool batched, int grid, cudaStream_t s);
// The last deterministic rounds in one CTA (after a launch that set
// Counters::tail; returns at once if none did).
cudaError_t launch_color_tail(const Params &p, bool batched, cudaStream_t s);
cudaError_t launch_admit(const Params &p, int g, long long vb, int32_t n, int par, int grid,
                         cudaStream_t s);
// Server: take graph [lo, hi)'s vertices off the worklists of parity par.
cudaError_t launch_purge(const Params &p, long long lo, long long hi, int par, cudaStream_t s);
cudaError_t launch_slot_status(const int32_t *colors, const long long *vbase, const int32_t *nv,
                               int G, int32_t *rem, int32_t *kmax, cudaStream_t s);
cudaError_t launch_fill_gid(int32_t *gid, const long long *vbase_dev, int G, int32_t n,
                            cudaStream_t s);
cudaError_t launch_segmented_max(const int32_t *colors, const long long *vbase_dev, int G,
                                 int32_t *out_dev, cudaStream_t s);
cudaError_t launch_validate(int32_t n, long long m, const int32_t *ro, const int32_t *ci,
                            unsigned long long *flags_dev, cudaStream_t s);
cudaError_t launch_validate_exact(int32_t n, long long m, const int32_t *ro, const int32_t *ci,
                                  unsigned long long *flags_dev, cudaStream_t s);

// The topology-driven schedule (Algorithm 6, sgr_topo.cu): per iteration, a
// FirstFit pass and a ConflictResolve pass over all n vertices.
struct TopoCounters {
    unsigned changed;         // the iteration found a vertex to color (cleared by the host)
    int kmax;                 // largest final color
    unsigned long long nw;    // sum over iterations of the vertices colored tentatively (sum |W_r|)
    unsigned long long dsum;  // ... and of their degrees (sum D_r)
};
int topo_grid(int *out);
cudaError_t launch_topo_iteration(const int32_t *ro, const int32_t *ci, int32_t *colors, int32_t n, int rule,
                                  TopoCounters *tc, int grid, cudaStream_t s);

}  // namespace sgr
