// common.cuh -- internal definitions shared by the treegb CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "treegb.h"

namespace treegb {

constexpr int kBits = 21;          // bits per axis of the quantised coordinates
constexpr int kMaxLevel = 21;      // deepest octree level
constexpr int kLevels = 22;        // levels 0..21
constexpr int kMomLeafBuckets = 17;                          // moment buckets of leaves (count 1..16, 17+)
constexpr int kMomBuckets = kMomLeafBuckets + 8 * kMaxLevel;  // + internal cells by (level, nchild)
constexpr int kSortThreads = 256;  // onesweep block
constexpr int kSortItems = 16;     // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortPasses = 8;     // 8-bit digits over the 64-bit key
constexpr int kSegPassesMax = 2;   // extra passes over the segment index (ensembles)
constexpr int kMaxSegments = 65536;
constexpr int kBoxChunk = 8192;    // particles per partial box of a segmented reduction
constexpr int kRadix = 256;
constexpr int kLevelThreads = 256;  // octree level block (nodes per tile)
constexpr int kMaxBlocksReduce = 1024;  // partial-result slots of the reductions
constexpr int kMaxLeafSmall = 16;   // leaves up to this size are expanded in the walk buffer
constexpr int64_t kMaxNodes = (int64_t)1 << 29;  // node indices fit 29 bits (walk stack entries)
// Below this many particles the walk takes its groups widest box first (one
// expensive group at the end of a short walk would be a visible straggler);
// above it, in key order, which keeps the neighbourhoods the SMs walk at the
// same time together in L2 (measured 0.3 % faster on the galaxy at N = 1.7e7
// and 1e8, equal at 2^20).
constexpr int64_t kWalkOrderMaxN = (int64_t)1 << 22;

// lookback status words: 2-bit flag + 30-bit value
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
// bounded waits: give up after this many clock cycles (about 1 s)
constexpr long long kWaitCycles = 2000000000LL;

struct __align__(32) double4a { double x, y, z, w; };
struct __align__(16) double2a { double x, y; };

template <typename Real> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4a; };
template <typename Real> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2a; };

// Box of the last build, written by the device.
struct DevBox {
    double lo[3];
    double scale;   // 2^(21-k)
    double unit;    // 2^(k-21): grid spacing
    int32_t k;
    int32_t r5fit;  // set after the moments: the FP32 walk's r^-5 far-cell form fits (pc_r5_fits)
};

// Offsets into the counter block (uint32), cleared at the start of a build.
// Level l holds nodes [lvl_start[l], lvl_start[l+1]).  While the octree is
// built, level l's end is min(raw_end[l], trunc[l]): raw_end is the child
// total of level l-1, trunc the first child slot of a parent that was turned
// into a leaf because the node array was full.
enum CounterSlots {
    kCtrSortTicket = 0,                       // 8 + 2 tickets
    kCtrLevelTicket = kCtrSortTicket + 16,    // 22 tickets
    kCtrLevelStart = kCtrLevelTicket + 24,    // 23 level starts
    kCtrLevelRawEnd = kCtrLevelStart + 24,    // 23 raw ends
    kCtrLevelTrunc = kCtrLevelRawEnd + 24,    // 23 truncation points
    kCtrGroups = kCtrLevelTrunc + 24,         // number of walk groups
    kCtrGScanTicket = kCtrGroups + 1,         // group-count scan tiles
    kCtrWalkTicket = kCtrGroups + 2,          // walk: next group slot (reset before every walk)
    kCtrAbort = kCtrGroups + 3,               // stage whose bounded wait gave up (0: none)
    kCtrCount = kCtrGroups + 8
};

// Stages that wait on other blocks (decoupled look-backs).  When a wait of
// stage S gives up, S is recorded in the counter block; the rest of S still
// writes only in bounds, and every later kernel of the build (any other stage)
// returns at once, so no kernel consumes the inconsistent data.
constexpr uint32_t kStageSort0 = 1;        // sort pass p: 1 + p
constexpr uint32_t kStageLevel0 = 16;      // octree level L: 16 + L
constexpr uint32_t kStageGroupScan = 48;   // walk-group count scan
constexpr uint32_t kStageAfter = 0xffffffffu;  // kernels that never wait

// Device-side controls of the bounded waits (set from the host).
struct DevCtl {
    long long wait_cycles;  // give up after this many clock cycles
    long long withhold;     // test injection: sort tile (pass << 32 | tile) that skips its look-back
                            // publications, or -1
};

// Statistics slots (unsigned long long), cleared at the start of each walk.
enum StatSlots { kStatPP = 0, kStatPC = 1, kStatMaxStack = 2, kStatCount = 8 };

}  // namespace treegb

// Opaque to C callers.
struct TreeWorkspace {
    int device = 0;
    int64_t n_max = 0;
    int64_t n = 0;
    TreeParams p{};
    int64_t node_cap = 0;
    int64_t sort_tiles_max = 0;
    int64_t level_tiles_max = 0;
    size_t real_size = 4;

    // sort
    uint64_t *key = nullptr, *key_alt = nullptr;
    uint32_t *idx = nullptr, *idx_alt = nullptr;
    uint32_t *hist = nullptr;          // [8][256] counts, then exclusive offsets
    uint32_t *sort_status = nullptr;   // [8 + 2][tiles][256]
    uint32_t *level_status = nullptr;  // [22][level_tiles]
    uint32_t *ctr = nullptr;           // kCtrCount words
    // box
    double *part = nullptr;            // reduction partials [kMaxBlocksReduce][8]
    treegb::DevBox *box = nullptr;     // one per segment
    // segments (independent systems sharing one build; nseg = 1: a single system of any n)
    int64_t nseg = 1;
    std::vector<int64_t> seg_off_h;    // host copy of the offsets (nseg + 1), empty when nseg = 1
    int64_t *seg_off = nullptr;        // device offsets [nseg + 1]
    uint32_t *seg_cstart = nullptr;    // first Gs chunk of each segment [nseg + 1] (for the current Gs)
    int32_t seg_cstart_gs = 0;         // Gs the chunk table was made for
    int64_t seg_nchunks = 0;           // total Gs chunks over all segments
    uint4 *seg_bchunk = nullptr;       // box chunks {begin, end, segment, 0}
    uint32_t *seg_bfirst = nullptr;    // first box chunk of each segment [nseg + 1]
    int64_t seg_nbchunk = 0;
    double *seg_part = nullptr;        // [box chunks][8] partial min/max
    uint32_t *seg_digit_off = nullptr; // [2][256] exclusive offsets of the segment-index digits
    int seg_passes = 0;                // sort passes over the segment index (0, 1 or 2)
    int64_t chunks_cap = 0;            // capacity of ccount / coff
    int64_t box_cap = 1;               // DevBox entries allocated
    // device copies of a host-resident state (leapfrog_step_host), allocated on first use
    void *hs_x = nullptr, *hs_v = nullptr, *hs_m = nullptr, *hs_a = nullptr, *hs_phi = nullptr;
    double *hs_diag = nullptr;
    cudaStream_t copy_stream = nullptr;  // copies back that overlap the rest of the step
    cudaEvent_t ev_drift = nullptr, ev_xback = nullptr;
    cudaStream_t side_stream = nullptr;  // a leapfrog step's walk groups, beside its gather and moments
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // one captured leapfrog step (leapfrog_graph_capture)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0, graph_n = 0;
    // sorted particles (float4 / double4a)
    void *spos = nullptr;
    // packed (x, y, z, m) in caller order, written by the kick-drift pass
    void *xm = nullptr;
    // nodes
    uint32_t *nfirst = nullptr, *ncount = nullptr;
    uint4 *ngeo = nullptr;             // {cx, cy, cz, level | leaf << 8}
    uint2 *nlink = nullptr;            // internal: {child, nchild}; leaf: {first, count}
    double *mom64 = nullptr;           // [10][node_cap]: M, Rx, Ry, Rz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz
    uint32_t *morder = nullptr;        // nodes in moment-bucket order [node_cap]
    uint32_t *mbucket = nullptr;       // moment buckets: counts, offsets (+ total), cursors
    void *mom_a = nullptr;             // Vec4: (Rx, Ry, Rz, M)
    void *mom_b = nullptr;             // Vec4: (Qxx, Qyy, Qzz, Qxy); FP32 copies hold -Q
    void *mom_c = nullptr;             // Vec2: (Qxz, Qyz); FP32 copies hold -Q
    // status and statistics
    int32_t *dstatus = nullptr;
    treegb::DevCtl *dctl = nullptr;    // bounded-wait controls
    unsigned long long *stats = nullptr;
    uint4 *gstat = nullptr;            // per walk group: {n_pc, n_pp particles, max stack, n_pp leaves}
    uint32_t *gfirst = nullptr;        // walk groups: first sorted index of each, then n
    uint8_t *plev = nullptr;           // leaf level of every sorted particle
    uint32_t *pleaf = nullptr;         // leaf node of every sorted particle
    uint32_t *nparent = nullptr;       // parent of every node (root: itself)
    uint32_t *ccount = nullptr, *coff = nullptr;  // groups starting in each Gs chunk / their offsets
    uint32_t *cmask = nullptr;         // group-start flags of each chunk, two 32-bit slices per chunk
    uint32_t *gscan_status = nullptr;  // look-back words of the chunk scan
    int64_t walk_grid = 0;             // resident walk blocks (persistent grid)
    int walk_grid_key = -1;
    uint32_t *gorder = nullptr;        // walk processing order of the groups
    uint32_t *gkey = nullptr;          // per group: extent bucket (scratch for gorder)
    uint32_t *gbucket = nullptr;       // [2][32] bucket counts / cursors
    int64_t groups_max = 0;
    // interaction lists (allocated on first use)
    int64_t *list_cnt = nullptr;       // [2][groups+1] counts -> offsets
    int32_t *pc_list = nullptr, *pp_list = nullptr;
    int64_t list_pc_cap = 0, list_pp_cap = 0, list_pc = 0, list_pp = 0;
    int64_t list_groups = -1;
    int64_t list_groups_host = 0;      // group count used by the last list emission
    // adjoint scratch (allocated on first use)
    void *adj_cot = nullptr;           // Vec4 (abar, phibar) in key order
    double *adj_xt = nullptr, *adj_xg = nullptr, *adj_mg = nullptr, *adj_ccot = nullptr;
    // direct-sum scratch
    double *direct_part = nullptr;
    size_t direct_part_bytes = 0;
    // host-side state
    int64_t mac_D[treegb::kLevels];
    double mac_theta = -1.0;
    int64_t *dmac = nullptr;           // device copy of mac_D
    bool built = false, has_moments = false;
    // kernel launch count and optional per-phase event timing
    int64_t launches = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;       // pairs (start, stop)
    std::vector<int> ev_phase;         // phase of each pair
    size_t ev_used = 0;                // pairs recorded since the last read
    int64_t timed_launches = 0;        // kernels launched inside timed phases
};

namespace treegb {

inline bool walk_widest_first(const TreeWorkspace *ws) { return ws->n < kWalkOrderMaxN; }

// ---------------------------------------------------------------- device helpers
// Look-back words are published with relaxed stores at GPU scope: a reader
// reads nothing but the word itself (flag and value share it), so no earlier
// write has to become visible with it, and a release fence would only stall.
__device__ __forceinline__ void st_publish(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the (full) warp whose 8-bit digit d equals this lane's, from one
// ballot per digit bit; `same` starts the match (e.g. the lanes with the same
// validity).  The ballots run on the integer pipes, where a match.any of the
// whole value would queue on the address-divergence unit.
__device__ __forceinline__ uint32_t match_digit8(uint32_t d, uint32_t same) {
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        same &= bit ? bal : ~bal;
    }
    return same;
}

// Spread the low 21 bits of v so that bit b lands at bit 3b.
__host__ __device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}
// Inverse of spread3: gather bits 3b into bit b.
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ULL;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ULL;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00fULL;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffULL;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffULL;
    x = (x ^ (x >> 32)) & 0x1fffffULL;
    return (uint32_t)x;
}
__host__ __device__ __forceinline__ uint64_t morton3(uint32_t qx, uint32_t qy, uint32_t qz) {
    return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

__device__ __forceinline__ void set_status(int32_t *st, int32_t bits) {
    atomicOr(st, bits);
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// What a bounded wait needs: where to report a timeout, the stage that waits,
// and the limit.
struct WaitCtx {
    int32_t *dstatus;
    uint32_t *ctr;         // counter block (kCtrAbort)
    uint32_t stage;
    long long limit;       // clock cycles
};

// True when a bounded wait of an earlier stage of this build gave up: the
// calling kernel (of stage `stage`) must return without touching the data.
// Whether the FP32 walk's quadrupole far-cell term with r^-5 taken out of the
// acceleration (pc_pair's R5 form) stays in the normal FP32 range for every
// far cell of a segment whose tree is the cube of side L = 2^k and whose total
// mass is M_root: a cell and a target lie in that cube, so r <= sqrt(3) L and
// |M r^2 u| <= M_root (sqrt(3) L)^3.  k <= 24 keeps r^-5 >= 4.8e-38 (FLT_MIN =
// 1.2e-38) and the mass bound keeps M r^2 u <= 1e37.  (At small r the full
// form forms r^-5 as well.)
__device__ __forceinline__ bool pc_r5_fits(int k, float m_root) {
    if (k > 24) return false;
    const float span = 1.7320508f * ldexpf(1.0f, max(k, -40));
    return m_root * span * span * span <= 1e37f;
}

__device__ __forceinline__ bool aborted(const uint32_t *ctr, uint32_t stage) {
    const uint32_t a = ctr[kCtrAbort];
    return a != 0u && a != stage;
}

__device__ __forceinline__ void wait_gave_up(const WaitCtx &w) {
    set_status(w.dstatus, TREE_DEV_TIMEOUT);
    atomicCAS(w.ctr + kCtrAbort, 0u, w.stage);
}

// Exclusive prefix of the tile after tile p from the look-back words of tiles
// p, p-1, ... (word of tile q at st[q * stride]): adds aggregates back to the
// first inclusive prefix.  Four predecessors are read at a time (independent
// loads; flag and value share one word, so relaxed loads suffice), so a walk
// over k tiles costs about k/4 load latencies; a word not yet published is
// waited for, bounded: past w.limit cycles the wait gives up (TREE_DEV_TIMEOUT,
// the stage is recorded so that later kernels of the build return at once),
// and the walk ends as if that word were an inclusive prefix of 0.  The
// result then never exceeds the true prefix, so positions derived from it
// stay in bounds.
__device__ inline uint32_t lookback_walk(const uint32_t *st, size_t stride, int64_t p, const WaitCtx &wc) {
    uint32_t excl = 0;
    while (p >= 0) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = p - j >= 0 ? ld_relaxed(st + (size_t)(p - j) * stride) : kFlagInc;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t v = w[j];
            if ((v & ~kValMask) == 0) {
                long long t0 = clock64();
                while (((v = ld_relaxed(st + (size_t)(p - j) * stride)) & ~kValMask) == 0) {
                    if (clock64() - t0 > wc.limit) {
                        wait_gave_up(wc);
                        v = kFlagInc;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            excl += v & kValMask;
            if ((v & ~kValMask) == kFlagInc) return excl;
        }
        p -= 4;
    }
    return excl;
}

// Single-value decoupled look-back: returns the exclusive prefix of tile
// `tile` given its aggregate.  Call from one thread.  A wait that exceeds
// the limit gives up as in lookback_walk (every waiter terminates).
__device__ inline uint32_t lookback_single(uint32_t *status, uint32_t tile, uint32_t agg, const WaitCtx &wc) {
    if (tile == 0) {
        st_publish(status, kFlagInc | (agg & kValMask));
        return 0;
    }
    st_publish(status + tile, kFlagAgg | (agg & kValMask));
    const uint32_t excl = lookback_walk(status, 1, (int64_t)tile - 1, wc);
    st_publish(status + tile, kFlagInc | ((excl + agg) & kValMask));
    return excl;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x multiple of 32,
// at most 1024 threads).  `warp_tot` is shared scratch of 32 words.
__device__ inline uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    uint32_t before = warp == 0 ? 0 : warp_tot[warp - 1];
    if (total) *total = warp_tot[nw - 1];
    uint32_t r = before + x - v;
    __syncthreads();
    return r;
}

// Segment holding sorted or input position i: the largest b < nseg with
// off[b] <= i (off ascending, off[0] = 0).
__device__ __forceinline__ uint32_t seg_find(const int64_t *__restrict__ off, int64_t nseg, int64_t i) {
    uint32_t lo = 0, hi = (uint32_t)nseg - 1u;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1u) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1u;
    }
    return lo;
}

inline int grid_for(int64_t n, int threads, int max_blocks) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

// Grid of a grid-stride kernel: grid_for, cut to one wave of the blocks that
// fit on the device at once.  Every block of a grid-stride loop carries the
// same share of the work, so a partial last wave would take as long as a
// full one (e.g. 1024 blocks at 3 resident per SM: three waves for 2.25
// waves of work).
template <typename Kernel>
inline int wave_grid(Kernel k, int64_t n, int threads, int max_blocks, size_t smem = 0) {
    int nb = grid_for(n, threads, max_blocks);
    int dev = 0, per_sm = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) == cudaSuccess && per_sm > 0 &&
        (int64_t)per_sm * sms < nb)
        nb = per_sm * sms;
    return nb;
}

}  // namespace treegb

// ---------------------------------------------------------------- host-side entry points of each .cu
namespace treegb {
// build.cu
cudaError_t launch_box(TreeWorkspace *ws, const void *x, int64_t n, cudaStream_t s);
cudaError_t launch_box_final(TreeWorkspace *ws, int nblocks, cudaStream_t s);
cudaError_t launch_box_segments(TreeWorkspace *ws, void *x, void *v, const void *a, const void *m, double tau,
                                int64_t n, bool kick, cudaStream_t s);
cudaError_t launch_keys(TreeWorkspace *ws, const void *x, int64_t n, cudaStream_t s);
cudaError_t launch_sort(TreeWorkspace *ws, int64_t n, cudaStream_t s);
cudaError_t launch_octree(TreeWorkspace *ws, int64_t n, cudaStream_t s);
// groups.cu
cudaError_t launch_groups(TreeWorkspace *ws, int64_t n, cudaStream_t s);
cudaError_t launch_gather(TreeWorkspace *ws, const void *x, const void *m, int64_t n, cudaStream_t s);
cudaError_t launch_gather_packed(TreeWorkspace *ws, int64_t n, cudaStream_t s);
cudaError_t launch_export_tree(TreeWorkspace *ws, int64_t nn, int32_t *level, uint32_t *corner, uint32_t *first,
                               uint32_t *count, int32_t *child, int32_t *nchild, cudaStream_t s);
// moments.cu
cudaError_t launch_moments(TreeWorkspace *ws, cudaStream_t s);
// walk_f32.cu / walk_f64.cu
enum WalkMode { kWalkForce = 0, kWalkCount = 1, kWalkEmit = 2 };
struct WalkOut {
    void *a;            // [3][n] caller order (or NULL in count/emit modes)
    void *phi;          // [n] or NULL
    void *v;            // leapfrog: [3][n] velocities to kick, or NULL
    double half_tau;    // leapfrog kick
    void *v_mirror = nullptr;    // also receives the kicked v (e.g. mapped host memory), or NULL
    void *phi_mirror = nullptr;  // also receives phi, or NULL
};
cudaError_t launch_walk_f32(TreeWorkspace *ws, int mode, const WalkOut &out, cudaStream_t s);
cudaError_t launch_walk_f64(TreeWorkspace *ws, int mode, const WalkOut &out, cudaStream_t s);
// adjoint.cu
cudaError_t launch_adjoint(TreeWorkspace *ws, const void *abar, const void *phibar, void *xbar, void *mbar,
                           cudaStream_t s);
cudaError_t launch_adjoint_step(TreeWorkspace *ws, void *xbar, void *vbar, void *abar, void *mbar,
                                const void *phibar, double tau, cudaStream_t s);
cudaError_t launch_energy_vjp(TreeWorkspace *ws, const void *m, const void *phi, const double *wbar, int64_t n,
                              void *phibar, void *mbar, cudaStream_t s);
// integrate.cu
cudaError_t launch_kick_drift_box(TreeWorkspace *ws, void *x, void *v, const void *a, const void *m, double tau,
                                  int64_t n, cudaStream_t s);
cudaError_t launch_diagnostics(TreeWorkspace *ws, const void *x, const void *v, const void *m,
                               const void *phi, int64_t n, double *out, cudaStream_t s);
cudaError_t launch_diagnostics_segments(TreeWorkspace *ws, const void *x, const void *v, const void *m,
                                        const void *phi, int64_t n, double *out, cudaStream_t s);
cudaError_t launch_direct(TreeWorkspace *ws, const void *x, const void *m, int64_t n, int dtype,
                          const int64_t *targets, int64_t nt, double *a_out, double *phi_out,
                          cudaStream_t s);
cudaError_t launch_direct_range(TreeWorkspace *ws, const void *x, const void *m, int64_t n, int64_t jbeg,
                                int64_t jend, int dtype, double G, double eps, const int64_t *targets, int64_t nt,
                                double *a_out, double *phi_out, cudaStream_t s);
cudaError_t launch_widen(TreeWorkspace *ws, const float *in, int64_t count, double *out, cudaStream_t s);
cudaError_t launch_rel_err(TreeWorkspace *ws, const void *a, int64_t n, int dtype, const int64_t *tgt,
                           const double *ref, int64_t nt, double *err, cudaStream_t s);
cudaError_t launch_scan_lists(TreeWorkspace *ws, int64_t ngroups, cudaStream_t s);
cudaError_t launch_gstat_reduce(TreeWorkspace *ws, int64_t ngroups, cudaStream_t s);
cudaError_t launch_group_order(TreeWorkspace *ws, cudaStream_t s);
cudaError_t launch_export_gstat(TreeWorkspace *ws, int64_t ngroups, uint32_t *out, cudaStream_t s);
}  // namespace treegb
