/*
 * sgrcolor.h -- C ABI of libsgrcolor: data-driven speculative-greedy (SGR)
 * graph coloring on one GB300 GPU.
 *
 * The method (X. Chen et al., "Efficient and High-quality Sparse Graph
 * Coloring on GPUs", Sect. 3, Algorithms 4, 5 and 7): keep a worklist W of
 * uncolored vertices; each round gives every vertex of W the smallest color
 * c >= 1 that none of its neighbours holds (FirstFit, Algorithm 4), then finds
 * adjacent pairs of W that picked the same color (ConflictResolve,
 * Algorithm 5); one vertex of each such pair is cleared and pushed onto the
 * next worklist (Algorithm 7).  The loop ends when the worklist is empty.
 *
 * Graphs are undirected, given as symmetric CSR: row_offsets[n+1] (int32,
 * row_offsets[0] == 0, non-decreasing) and col_idx[m] (int32, m =
 * row_offsets[n] directed entries, each in [0, n)).  No self-loops, no
 * duplicate entries in a row (Sect. 3: R and C arrays).  Rows need not be
 * sorted; sorted rows are detected on the device and let ConflictResolve
 * stop at the first neighbour above the vertex.
 * Colors come back as int32 values 1..k, k = number of colors (Sect. 2.1:
 * 0 means uncolored and never appears in a result).
 *
 * Modes (the `mode` argument is an OR of one SGR_MODE_* and one SGR_RULE_*):
 *   SGR_MODE_DETERMINISTIC: every FirstFit of a round reads the colors fixed
 *     at the start of the round, and conflicts are judged on all tentative
 *     colors of the round before any is cleared.  The result depends only on
 *     the graph and the rule, and equals the CPU oracle bit for bit.
 *   SGR_MODE_FAST: FirstFit and ConflictResolve read and write colors in
 *     place while other vertices of the round do the same, as the paper's GPU
 *     code does (Sect. 3.1, "Color Clearing").  Always a valid coloring; the
 *     exact colors may change from run to run.
 *   SGR_MODE_TOPO: the deterministic rounds on the topology-driven schedule of
 *     Algorithm 6 (Sect. 3.1, the paper's baseline design): every iteration
 *     visits all n vertices, FirstFit for those not final and
 *     ConflictResolve for those holding a tentative color, and the host
 *     relaunches the two passes while an iteration found a vertex to color.
 *     Same colors, k and rounds as SGR_MODE_DETERMINISTIC; it is there to
 *     compare the schedules.  sgr_color and sgr_color_host only; the other
 *     entry points refuse it (SGR_ERR_INVALID_ARG).
 *   SGR_RULE_LOW_KEEPS (default): of two neighbours with the same color, the
 *     lower vertex id keeps it.
 *   SGR_RULE_LOW_LOSES: the lower id is recolored, as printed in Algorithm 2
 *     and Algorithm 5.
 *   SGR_RULE_DEGREE: the heuristic of Sect. 3.2: the larger degree keeps the
 *     color; on equal degree the smaller id keeps it.
 *
 * Ownership and memory: the caller owns every input and output buffer.  The
 * library keeps a per-device scratch arena (worklists, counters, bitmaps),
 * grown on demand and never shrunk, released by sgr_release_scratch().
 * Errors: every entry point returns an sgr_status; on error, HOST output
 * parameters (num_colors, req_id, ...) are left untouched and DEVICE output
 * buffers hold unspecified values.
 * Threads: calls on different host threads may run concurrently; the
 * coloring launches of all entry points on one device (sgr_color,
 * sgr_color_noalloc, sgr_color_host, sgr_color_batch, sgr_autotune and the
 * servers' scheduler threads) are serialised by the library, since two
 * cooperative persistent grids in flight on one device could each wait for
 * CTAs the other holds.
 */
#ifndef SGRCOLOR_H
#define SGRCOLOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (cudaStream_t / CUstream); NULL is the legacy default
 * stream of the calling thread. */
typedef struct CUstream_st *sgr_stream_t;

typedef enum {
    SGR_OK = 0,
    SGR_PENDING = 1,               /* server: request not finished yet */
    SGR_ERR_INVALID_ARG = -1,      /* bad pointer, size, mode or alignment */
    SGR_ERR_INVALID_GRAPH = -2,    /* CSR breaks the input contract */
    SGR_ERR_OUT_OF_MEMORY = -3,    /* device or host allocation failed */
    SGR_ERR_CUDA = -4,             /* a CUDA call failed */
    SGR_ERR_NO_CONVERGENCE = -5,   /* round cap reached (only on broken input) */
    SGR_ERR_TIMEOUT = -6,          /* a bounded device-side wait ran out */
    SGR_ERR_NOT_FOUND = -7,        /* server: unknown request id */
    SGR_ERR_BUSY = -8              /* server: over budget or queue full */
} sgr_status;

#define SGR_MODE_DETERMINISTIC 0
#define SGR_MODE_FAST 1
#define SGR_MODE_TOPO 2
#define SGR_MODE_MASK 0x3
#define SGR_RULE_LOW_KEEPS (0 << 4)
#define SGR_RULE_LOW_LOSES (1 << 4)
#define SGR_RULE_DEGREE (2 << 4)
#define SGR_RULE_MASK (0x3 << 4)

/* Statistics of the last coloring call made on this host thread. */
typedef struct {
    int64_t rounds;        /* iterations of Algorithm 7's loop */
    int64_t sum_w;         /* sum over rounds of |W_r| */
    int64_t sum_d;         /* sum over rounds of the degrees of W_r (FirstFit scan) */
    int64_t sum_dscan;     /* col_idx entries ConflictResolve had to inspect */
    int64_t sum_next;      /* sum over rounds of |W_{r+1}| (pushed losers) */
    int64_t sum_scatter;   /* det mode: neighbour bitmap updates by committed vertices */
    int64_t sum_rescan;    /* det mode: worklist vertices ConflictResolve rescanned */
    int32_t num_colors;    /* k (max color); per-graph values are returned separately */
    int32_t rows_sorted;   /* 1 if every row was strictly ascending */
    int32_t grid_blocks;   /* CTAs of the persistent kernel */
    int32_t block_threads; /* threads per CTA */
    double device_ms;      /* device time of the coloring kernel(s), CUDA events */
    int64_t tail_rounds;   /* deterministic mode: rounds run by the one-CTA tail */
    int64_t sum_touch;     /* deterministic mode: worklist entries the grid phases visited */
    int64_t sum_dep;       /* deterministic mode: row entries read to find witness dependents */
    int64_t tail_entries;  /* deterministic mode: W-adjacency entries the tail read */
    int64_t tail_build;    /* deterministic mode: row entries the tail hand-over scanned */
} sgr_stats;

/* Load-balance and launch parameters (Sect. 3.2 thread coarsening, Sect. 3.3
 * load balancing).  Zero fields mean "library default". */
typedef struct {
    int32_t light_max;     /* degree bound of the lane-per-vertex bin, 1..32 */
    int32_t chunk;         /* edges per warp work item of the hub bin; also the
                              degree bound of the warp-per-vertex bin (>= 64) */
    int32_t blocks_per_sm; /* persistent CTAs per SM (capped by occupancy) */
    int32_t active_lists;  /* deterministic mode: 0 = a round runs on the
                              activation lists (the vertices a commit made
                              stale, plus those whose witness they are) once
                              that is cheaper than the whole worklist;
                              1 = never; 2 = from round 2 on.  The colors are
                              the same in every case. */
    int32_t tail_vertices; /* deterministic mode: once at most this many
                              vertices are left on the worklist, the remaining
                              rounds run in one CTA on the subgraph they
                              induce; 0 = library default (2048), -1 = never,
                              else 1..2880.  The colors are the same. */
} sgr_tuning;

/*
 * Color one graph.  Algorithm 7 with Algorithms 4 and 5 (Sect. 3.1-3.3).
 *   n            number of vertices, 0 <= n < 2^31.
 *   row_offsets  DEVICE pointer, n+1 int32.
 *   col_idx      DEVICE pointer, m = row_offsets[n] int32, 16-byte aligned
 *                (any cudaMalloc / torch allocation is).
 *   colors_out   DEVICE pointer, n int32; receives colors 1..k.
 *   num_colors   HOST pointer; receives k (0 when n == 0).
 *   mode         SGR_MODE_* | SGR_RULE_*.
 *   stream       stream the work is ordered on.  The call blocks until the
 *                coloring is done (one stream synchronisation to read m before
 *                launch and one to read k and the statistics after).
 * Returns SGR_OK, SGR_ERR_INVALID_ARG (null pointer with n > 0, unknown mode,
 * unaligned col_idx), SGR_ERR_INVALID_GRAPH (row_offsets[0] != 0 or m < 0),
 * SGR_ERR_OUT_OF_MEMORY, SGR_ERR_CUDA, SGR_ERR_TIMEOUT or
 * SGR_ERR_NO_CONVERGENCE.  On a CSR that breaks the contract (not symmetric,
 * ids outside [0, n)) the coloring is unspecified, but the call ends (round
 * cap n + 1) and never reads outside the given arrays: out-of-range ids are
 * skipped.  sgr_validate_csr checks a graph first.
 */
int sgr_color(int32_t n, const int32_t *row_offsets, const int32_t *col_idx,
              int32_t *colors_out, int32_t *num_colors, int mode, sgr_stream_t stream);

/*
 * sgr_color without any allocation by the library.  The paper has no
 * counterpart: this entry point exists for callers that must not let a
 * library allocate device memory -- an application that gives this code a
 * fixed share of the GPU and routes every allocation through its own pool, or
 * a latency-sensitive loop in which cudaMalloc / cudaFree would synchronise
 * the device and stall other streams.
 *   Arguments, layout and results are those of sgr_color (device buffers
 *   owned by the caller, colors 1..k, k on the host).  Modes: those of
 *   sgr_color except SGR_MODE_TOPO, which is refused with
 *   SGR_ERR_INVALID_ARG.
 *   Scratch: a fixed 16 MiB array inside the library's device image, held by
 *   every GPU that loads the library until the process exits (enough for
 *   graphs of about 200,000 vertices and a few million entries).  A graph
 *   whose scratch does not fit is refused with SGR_ERR_INVALID_ARG before any
 *   device work.
 *   The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents; each call
 *   clears what must start at zero.  Calls whose GPU work overlaps would race
 *   on the array; within one process the calls on a device are serialised
 *   with each other and with every other coloring entry point (see Threads
 *   above), and each returns after its work is complete.
 *   The call makes no cudaMalloc, cudaFree or other allocating call.
 *   sgr_last_stats reports device_ms = 0 for it; sgr_last_trace then reads
 *   its timeline from the array (until the next call on the device).
 */
int sgr_color_noalloc(int32_t n, const int32_t *row_offsets, const int32_t *col_idx,
                      int32_t *colors_out, int32_t *num_colors, int mode, sgr_stream_t stream);

/*
 * Same as sgr_color with HOST buffers: copies the CSR to library-owned device
 * memory on `stream`, colors it and copies the colors back.  Pinned host
 * memory makes the copies faster but is not required.
 */
int sgr_color_host(int32_t n, const int32_t *row_offsets_host, const int32_t *col_idx_host,
                   int32_t *colors_host, int32_t *num_colors, int mode, sgr_stream_t stream);

/*
 * Color G independent graphs packed into one concatenated CSR, all in one
 * persistent kernel (rounds of all graphs advance together).  Coloring a
 * disjoint union with per-graph id offsets gives each graph exactly the
 * coloring it gets alone: the rules compare ids only within a graph.
 *   vtx_off   HOST, G+1 int64: graph g owns global vertices [vtx_off[g], vtx_off[g+1]).
 *   edge_off  HOST, G+1 int64: graph g's entries are col_idx[edge_off[g] .. edge_off[g+1]).
 *   row_offsets DEVICE, vtx_off[G] + G int32: graph g's n_g+1 LOCAL offsets
 *             start at row_offsets[vtx_off[g] + g] (first one 0).
 *   col_idx   DEVICE, edge_off[G] int32 LOCAL ids, 16-byte aligned base.
 *   colors_out DEVICE, vtx_off[G] int32; graph g's colors at vtx_off[g].
 *   num_colors HOST, G int32: per-graph k.
 * Requires vtx_off[G] < 2^31.  Errors as sgr_color.
 */
int sgr_color_batch(int32_t G, const int64_t *vtx_off, const int64_t *edge_off,
                    const int32_t *row_offsets, const int32_t *col_idx, int32_t *colors_out,
                    int32_t *num_colors, int mode, sgr_stream_t stream);

/*
 * Coloring server (continuous batching).  Deterministic mode only; the rule
 * bits of `mode` apply.  Requests of any size arrive at any time; a scheduler
 * thread keeps each admitted graph (its CSR, colors and worklist entries)
 * resident on the device, advances the rounds of all resident graphs together
 * in one persistent launch, retires finished graphs and admits waiting ones
 * as room frees up under the HBM budget.  Every result equals sgr_color on
 * the same graph in the same mode (the graphs are disjoint, the loser rules
 * only compare ids within a graph).  The paper has no server; this is a
 * systems addition around its Algorithm 7.
 */
typedef struct sgr_server sgr_server;

typedef struct {
    int64_t hbm_budget_bytes;  /* device memory the server allocates at creation (0: 1 GiB):
                                  a quarter for the scratch of requests colored alone (when
                                  direct_min_vertices >= 0), of the rest about 30% for
                                  per-vertex state and the remainder for col_idx */
    int32_t max_inflight;      /* graphs resident at once (0: 1024) */
    int32_t mode;              /* SGR_MODE_DETERMINISTIC | SGR_RULE_* */
    int32_t device;            /* CUDA device ordinal */
    int32_t rounds_per_launch; /* rounds advanced per launch (0: 8 while requests wait, else 64) */
    int64_t staging_bytes;     /* pinned host memory for request copies (0: 1 GiB, < 0: none);
                                  requests that do not fit use ordinary memory */
    int32_t direct_min_vertices; /* requests with at least this many vertices are colored
                                  alone on the single-graph kernels of sgr_color (with its
                                  activation lists and one-CTA tail), between two batched
                                  launches, in a scratch region of the budget (0: 262144,
                                  < 0: never); smaller ones share the batched rounds */
} sgr_server_config;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t pending;           /* waiting for admission */
    int64_t resident;          /* admitted, not yet finished */
    int64_t launches;          /* persistent launches so far */
    int64_t rounds;            /* rounds advanced so far */
    int64_t hbm_bytes;         /* device memory held */
    int64_t vertex_capacity;   /* vertices that can be resident at once */
    int64_t entry_capacity;    /* col_idx entries that can be resident at once */
    double p50_ms, p99_ms, mean_ms;  /* submit-to-finish latency of completed requests */
    double graphs_per_s;       /* completed / (last completion - first submission) */
    int64_t direct;            /* requests colored alone on the single-graph kernels */
} sgr_server_counters;

/* Create a server on cfg->device; allocates its whole budget up front.
 * SGR_ERR_INVALID_ARG for fast mode, unknown bits or a budget under ~2 MiB;
 * SGR_ERR_OUT_OF_MEMORY if the budget cannot be allocated. */
int sgr_server_create(const sgr_server_config *cfg, sgr_server **out);

/* Queue one graph (HOST CSR, same contract as sgr_color; rows need not be
 * sorted, self-loop entries are ignored).  The CSR is copied (into the pinned
 * staging pool when it has room); the caller may free it on return.  Checks
 * offsets and the id range (SGR_ERR_INVALID_GRAPH); a graph larger than the
 * server's capacity gives SGR_ERR_OUT_OF_MEMORY.  *req_id receives a fresh
 * id.  Thread-safe. */
int sgr_server_submit(sgr_server *s, int32_t n, const int32_t *row_offsets_host,
                      const int32_t *col_idx_host, uint64_t *req_id);

/* Wait up to timeout_ms (0: do not wait, < 0: wait indefinitely) for a request.
 * SGR_PENDING if not finished yet; SGR_OK with colors_host (HOST, n int32,
 * may be NULL) and *num_colors filled, after which the id is forgotten;
 * SGR_ERR_NOT_FOUND for an unknown or already collected id; or the request's
 * error, after which the id is forgotten too.  Every request ends: a graph
 * still unfinished after n + 1 of its own rounds (only a CSR that is not
 * symmetric gets there; the submit checks do not test symmetry) is taken off
 * the device, its slot and memory are freed, and it fails with
 * SGR_ERR_NO_CONVERGENCE, as sgr_color would.  Thread-safe. */
int sgr_server_poll(sgr_server *s, uint64_t req_id, int32_t *colors_host, int32_t *num_colors,
                    int timeout_ms);

/* Counters and latency percentiles so far.  Returns SGR_OK or the error that
 * stopped the server. */
int sgr_server_stats(sgr_server *s, sgr_server_counters *out);

/* Stop the scheduler, free device memory and drop uncollected requests. */
int sgr_server_destroy(sgr_server *s);

/*
 * Check the input contract on the device: row_offsets[0] == 0,
 * non-decreasing offsets, ids in [0, n), no self-loops, no duplicate entry in
 * a row, and symmetry (w in adj(v) iff v in adj(w)).  Returns SGR_OK or
 * SGR_ERR_INVALID_GRAPH; *rows_sorted (HOST, may be NULL) receives 1 when
 * every row is strictly ascending.  Pointers as in sgr_color.
 */
int sgr_validate_csr(int32_t n, const int32_t *row_offsets, const int32_t *col_idx,
                     int32_t *rows_sorted, sgr_stream_t stream);

/*
 * Pick the tuning for a graph by measurement: color it (sgr_color, device
 * buffers) under a grid of candidates -- hub chunk size {1024, 512, 256, 2048}
 * x degree bound of the lane-per-vertex bin {32, 16} x CTAs per SM {all, 2},
 * and in deterministic mode x tail hand-over size {2048, 1024, 2880} -- best of
 * two runs each by the kernels' event time, in that order (the library default
 * first), until budget_ms of device time is spent (0: 2000 ms; at least one
 * candidate always runs).  The fastest candidate becomes the process-wide
 * tuning and is returned in *best (HOST) with its time in *best_ms (HOST, may
 * be NULL).  colors_out receives the coloring of the last candidate run (a
 * valid coloring; in deterministic mode the same for every candidate).  The
 * paper leaves autotuning out of its scope (Sect. 3.2, thread coarsening).
 * The threads per CTA are fixed at 256: the tile layout of the kernels is
 * built for it.  Errors as sgr_color; the tuning is restored on error.
 */
int sgr_autotune(int32_t n, const int32_t *row_offsets, const int32_t *col_idx,
                 int32_t *colors_out, int mode, int32_t budget_ms, sgr_tuning *best,
                 double *best_ms, sgr_stream_t stream);

/*
 * The same for a batch: measures sgr_color_batch on the given packed graphs
 * (arguments as in sgr_color_batch) under the candidate grid of sgr_autotune
 * and installs the fastest tuning; colors_out and num_colors receive the last
 * run's results.  Errors as sgr_color_batch.
 */
int sgr_autotune_batch(int32_t G, const int64_t *vtx_off, const int64_t *edge_off,
                       const int32_t *row_offsets, const int32_t *col_idx, int32_t *colors_out,
                       int32_t *num_colors, int mode, int32_t budget_ms, sgr_tuning *best,
                       double *best_ms, sgr_stream_t stream);

/* Statistics of the last sgr_color / sgr_color_host / sgr_color_batch call
 * on this host thread. */
int sgr_last_stats(sgr_stats *out);

/*
 * Device timeline of the last coloring launch on the current device: for
 * round r (0-based, at most cap_rounds and 65536 rounds) out[4r] = |W_r|,
 * out[4r+1] / out[4r+2] = nanoseconds from kernel start to the end of the
 * FirstFit / ConflictResolve phase (read from %globaltimer by CTA 0 after each
 * grid barrier), out[4r+3] = worklist vertices whose ConflictResolve had to
 * scan their row in that round (deterministic mode; 0 in fast mode).  *init_ns (HOST, may be NULL) receives the end of the
 * initial binning pass.  Returns the number of rounds written (>= 0) or a
 * negative status.  Valid until the next call on the device.  out is HOST.
 */
int sgr_last_trace(int64_t *out, int64_t cap_rounds, int64_t *init_ns);

/*
 * Limit of every bounded device-side wait (the grid barriers of the
 * persistent coloring kernels), process-wide, in nanoseconds: 0 restores the
 * default of 4 s; otherwise 100 us .. 600 s.  A wait that runs out makes
 * every CTA of the launch leave at its next barrier, and the call returns
 * SGR_ERR_TIMEOUT; the device stays usable.  A watchdog for callers that
 * would rather fail fast; the paper has no counterpart.  Returns SGR_OK or
 * SGR_ERR_INVALID_ARG.
 */
int sgr_set_wait_limit(int64_t ns);

/*
 * Host-side fault injection for tests of the error paths (no counterpart in
 * the paper).  No GPU fault is ever caused: the failures are made on the host.
 *   SGR_INJECT_NONE          disarm everything (value ignored).
 *   SGR_INJECT_FAIL_ALLOC    the value-th next device allocation of the
 *                            library (scratch arena, host-buffer arena,
 *                            server budget) fails as out of memory without
 *                            calling cudaMalloc (value >= 1; 0 disarms).
 *   SGR_INJECT_BARRIER       the next `value` coloring calls launch their
 *                            round kernel with a barrier count one CTA larger
 *                            than the grid, so that its first grid barrier's
 *                            bounded wait runs out (see sgr_set_wait_limit)
 *                            and the call returns SGR_ERR_TIMEOUT.
 * Returns SGR_OK or SGR_ERR_INVALID_ARG (unknown kind, value < 0).
 */
#define SGR_INJECT_NONE 0
#define SGR_INJECT_FAIL_ALLOC 1
#define SGR_INJECT_BARRIER 2
int sgr_debug_inject(int what, int64_t value);

/* Get / set the process-wide tuning used by later calls. */
int sgr_get_tuning(sgr_tuning *out);
int sgr_set_tuning(const sgr_tuning *in);

/* Free the scratch arena of the current device. */
int sgr_release_scratch(void);

/* Human-readable name of a status code (static storage). */
const char *sgr_status_string(int status);

/* Library version, major * 10000 + minor * 100 + patch. */
int sgr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SGRCOLOR_H */
