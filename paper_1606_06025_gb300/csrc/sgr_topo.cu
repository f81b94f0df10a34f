// sgr_topo.cu -- the deterministic rounds on the topology-driven schedule of
// Algorithm 6 (Sect. 3.1, "The Baseline Design"): every iteration visits
// every vertex; FirstFit runs for the vertices not final yet and
// ConflictResolve for the ones that took a tentative color, and the host
// relaunches the pair while an iteration found a vertex to color.
//
// The colors follow the deterministic readings of the worklist path: each
// FirstFit sees only the colors final at the start of the iteration
// (tentative colors are stored negated and count as uncolored), and a
// conflict is judged on the tentative colors of the whole iteration, keepers
// included (a same-iteration keeper holds the same magnitude, a color final
// earlier cannot: FirstFit avoided it).  The set of vertices an iteration
// colors is therefore W_r, and the result equals the worklist path's (and the
// oracle's) bit for bit.  This schedule is the paper's baseline for the
// data-driven design: it pays a pass over all n vertices per iteration.
//
// Mapping: a warp takes 32 consecutive vertices, one per lane; rows longer
// than 32 entries are then done one at a time by the whole warp.
#include "sgr_internal.cuh"

namespace sgr {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kTopoBlock = 256;
constexpr int kTopoLaneMax = 32;  // rows up to this long are done by one lane

__device__ __forceinline__ int magnitude(int x) { return x < 0 ? -x : x; }

// First color >= 1 that no final neighbour (color > 0) holds, over entries
// [s, e) taken by lanes lane0, lane0 + step, ...; `lanes` is the mask of the
// lanes that share the row (one lane, or the whole warp).  One pass marks
// colors 1..256 in eight words; only a row whose 256 lowest colors are all
// taken is read again, 32 colors a pass.
__device__ __forceinline__ int topo_first_fit(const int32_t *ci, const int32_t *colors, int32_t n, long long s,
                                              long long e, int lane0, int step, unsigned lanes) {
    unsigned m[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (long long i = s + lane0; i < e; i += step) {
        const int32_t w = __ldg(ci + i);
        if ((unsigned)w >= (unsigned)n) continue;
        const int c = __ldcg(colors + w);
        if (c <= 0 || c > 256) continue;
        const unsigned word = (unsigned)(c - 1) >> 5, bit = 1u << ((c - 1) & 31);
#pragma unroll
        for (int j = 0; j < 8; ++j) m[j] |= word == (unsigned)j ? bit : 0u;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const unsigned x = lanes != 1u ? __reduce_or_sync(lanes, m[j]) : m[j];
        if (~x) return j * 32 + __ffs(~x);
    }
    for (int base = 256;; base += 32) {
        unsigned mask = 0;
        for (long long i = s + lane0; i < e; i += step) {
            const int32_t w = __ldg(ci + i);
            if ((unsigned)w >= (unsigned)n) continue;
            const int c = __ldcg(colors + w);
            if (c > base && c <= base + 32) mask |= 1u << (c - base - 1);
        }
        if (lanes != 1u) mask = __reduce_or_sync(lanes, mask);
        if (~mask) return base + __ffs(~mask);
    }
}

// Does neighbour w win against v under the rule (0: lower id keeps, 1: higher
// id keeps, 2: larger degree keeps, then the lower id)?
__device__ __forceinline__ bool topo_beats(const int32_t *ro, int rule, int32_t w, int32_t v, int dv) {
    if (rule == 0) return w < v;
    if (rule == 1) return w > v;
    const int dw = __ldg(ro + w + 1) - __ldg(ro + w);
    return dw != dv ? dw > dv : w < v;
}

// Some neighbour in [s, e) (lanes as above) that wins against v holds the
// magnitude c.
__device__ __forceinline__ bool topo_conflict(const int32_t *ro, const int32_t *ci, const int32_t *colors, int32_t n,
                                              int rule, int32_t v, int c, long long s, long long e, int lane0, int step,
                                              unsigned lanes) {
    const int dv = (int)(e - s);
    bool hit = false;
    for (long long i = s + lane0; i < e && !hit; i += step) {
        const int32_t w = __ldg(ci + i);
        if ((unsigned)w >= (unsigned)n || w == v) continue;
        hit = magnitude(__ldcg(colors + w)) == c && topo_beats(ro, rule, w, v, dv);
    }
    if (lanes != 1u) hit = __any_sync(lanes, hit);
    return hit;
}

// FirstFit over every vertex not final yet: colors[v] = -(first free color).
__global__ void __launch_bounds__(kTopoBlock) topo_assign_kernel(const int32_t *ro, const int32_t *ci,
                                                                   int32_t *colors, int32_t n, TopoCounters *tc) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (kTopoBlock / 32);
    unsigned long long nw = 0, dsum = 0;
    for (long long base = ((long long)blockIdx.x * (kTopoBlock / 32) + (threadIdx.x >> 5)) * 32; base < n;
         base += warps * 32) {
        const int32_t v = (int32_t)(base + lane);
        const bool open = v < n && __ldcg(colors + v) <= 0;
        long long s = 0, e = 0;
        if (open) {
            s = __ldg(ro + v);
            e = __ldg(ro + v + 1);
            nw += 1;
            dsum += (unsigned long long)(e - s);
        }
        const bool heavy = open && e - s > kTopoLaneMax;
        if (open && !heavy) __stcg(colors + v, -topo_first_fit(ci, colors, n, s, e, 0, 1, 1u));
        for (unsigned hb = __ballot_sync(kFullMask, heavy); hb; hb &= hb - 1) {
            const int src = __ffs(hb) - 1;
            const int32_t hv = (int32_t)(base + src);
            const long long hs = __shfl_sync(kFullMask, s, src), he = __shfl_sync(kFullMask, e, src);
            const int c = topo_first_fit(ci, colors, n, hs, he, lane, 32, kFullMask);
            if (lane == 0) __stcg(colors + hv, -c);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nw += __shfl_xor_sync(kFullMask, nw, o);
        dsum += __shfl_xor_sync(kFullMask, dsum, o);
    }
    if (lane == 0 && nw) {
        atomicAdd(&tc->nw, nw);
        atomicAdd(&tc->dsum, dsum);
        tc->changed = 1u;
    }
}

// ConflictResolve over every vertex holding a tentative color: keepers make
// it final (colors[v] = c), losers keep -c and stay uncolored.
__global__ void __launch_bounds__(kTopoBlock) topo_resolve_kernel(const int32_t *ro, const int32_t *ci,
                                                                    int32_t *colors, int32_t n, int rule,
                                                                    TopoCounters *tc) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (kTopoBlock / 32);
    int kmax = 0;
    for (long long base = ((long long)blockIdx.x * (kTopoBlock / 32) + (threadIdx.x >> 5)) * 32; base < n;
         base += warps * 32) {
        const int32_t v = (int32_t)(base + lane);
        const int cv = v < n ? __ldcg(colors + v) : 0;
        const bool tent = cv < 0;
        long long s = 0, e = 0;
        if (tent) {
            s = __ldg(ro + v);
            e = __ldg(ro + v + 1);
        }
        const bool heavy = tent && e - s > kTopoLaneMax;
        if (tent && !heavy && !topo_conflict(ro, ci, colors, n, rule, v, -cv, s, e, 0, 1, 1u)) {
            __stcg(colors + v, -cv);
            kmax = max(kmax, -cv);
        }
        for (unsigned hb = __ballot_sync(kFullMask, heavy); hb; hb &= hb - 1) {
            const int src = __ffs(hb) - 1;
            const int32_t hv = (int32_t)(base + src);
            const int hc = -__shfl_sync(kFullMask, cv, src);
            const long long hs = __shfl_sync(kFullMask, s, src), he = __shfl_sync(kFullMask, e, src);
            if (!topo_conflict(ro, ci, colors, n, rule, hv, hc, hs, he, lane, 32, kFullMask) && lane == 0) {
                __stcg(colors + hv, hc);
                kmax = max(kmax, hc);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(kFullMask, kmax, o));
    if (lane == 0 && kmax) atomicMax(&tc->kmax, kmax);
}

}  // namespace

int topo_grid(int *out) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topo_assign_kernel, kTopoBlock, 0) != cudaSuccess)
        return -1;
    *out = sms * (per_sm > 0 ? per_sm : 1);
    return 0;
}

cudaError_t launch_topo_iteration(const int32_t *ro, const int32_t *ci, int32_t *colors, int32_t n, int rule,
                                  TopoCounters *tc, int grid, cudaStream_t s) {
    topo_assign_kernel<<<grid, kTopoBlock, 0, s>>>(ro, ci, colors, n, tc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    topo_resolve_kernel<<<grid, kTopoBlock, 0, s>>>(ro, ci, colors, n, rule, tc);
    return cudaGetLastError();
}

}  // namespace sgr
