// groups.cu -- walk groups from the sorted keys and the octree.
//
// Particles are taken in key order in chunks of Gs; a chunk is cut between
// consecutive particles i-1, i that do not share the cell `delta` levels
// above the finer of their two leaves:
//   P(i-1, i) < max(leaf_level(i-1), leaf_level(i)) - delta,
// P = number of leading octal digits the two keys share (21 if equal), and
// where their smallest common cell (level P) holds more than cmax = 128 Gs
// particles.  Neighbours in a group are then close on the scale of their own
// leaves, every group fits in the cell delta levels above its coarsest leaf,
// and in a cell of at most cmax particles.  This keeps a chunk that jumps
// between distant parts of the Morton curve, or a sparse group whose box
// would enclose a dense region, from turning its walk into a near-direct
// sum.  delta = 0 keeps plain chunks (no cuts at all).
// Output: gfirst[0..ng] (group g = sorted particles [gfirst[g], gfirst[g+1]))
// and the group count in the counter block.
#include "common.cuh"

namespace treegb {

constexpr int kGScanThreads = 256;
constexpr int kGScanItems = 8;
constexpr int kGScanTile = kGScanThreads * kGScanItems;

// Leaf level and leaf node of every sorted particle.  A warp takes 32
// consecutive nodes and fills the particle ranges of their leaves one leaf at
// a time, lanes over the particles (coalesced writes).
__global__ void __launch_bounds__(256) k_leaf_levels(const uint32_t *__restrict__ ctr, const uint4 *__restrict__ ngeo,
                                                     const uint2 *__restrict__ nlink, uint8_t *__restrict__ plev,
                                                     uint32_t *__restrict__ pleaf) {
    if (aborted(ctr, kStageAfter)) return;
    const uint32_t nn = ctr[kCtrLevelStart + kLevels];
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < nn; base += stride) {
        const uint32_t c = base + lane;
        uint32_t lv = 0, first = 0, count = 0;
        bool leaf = false;
        if (c < nn) {
            const uint4 g = ngeo[c];
            leaf = (g.w >> 8) & 1u;
            if (leaf) {
                const uint2 l = nlink[c];
                lv = g.w & 0xffu;
                first = l.x;
                count = l.y;
            }
        }
        uint32_t todo = __ballot_sync(0xffffffffu, leaf);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t f = __shfl_sync(0xffffffffu, first, src), k = __shfl_sync(0xffffffffu, count, src);
            const uint32_t l = __shfl_sync(0xffffffffu, lv, src);
            for (uint32_t j = lane; j < k; j += 32) {
                plev[f + j] = (uint8_t)l;
                pleaf[f + j] = base + (uint32_t)src;
            }
        }
    }
}

__device__ __forceinline__ bool group_starts(const uint64_t *__restrict__ skey, const uint8_t *__restrict__ plev,
                                             const uint32_t *__restrict__ pleaf, const uint32_t *__restrict__ nparent,
                                             const uint32_t *__restrict__ ncount, int64_t i, int64_t s0, int delta,
                                             uint32_t cmax) {
    if (i == s0) return true;
    if (delta <= 0) return false;
    const uint64_t d = skey[i - 1] ^ skey[i];
    const int shared = d ? (62 - (63 - __clzll((long long)d))) / 3 : kMaxLevel;
    const int lmax = max((int)plev[i - 1], (int)plev[i]);
    if (shared < lmax - delta) return true;
    // smallest common cell: the ancestor of i's leaf at level `shared` (at most
    // delta steps up here); when i's leaf is already no finer than that level,
    // both particles share the leaf and it bounds the population from above
    uint32_t node = pleaf[i];
    for (int lv = plev[i]; lv > shared; --lv) node = nparent[node];
    return ncount[node] > cmax;
}

// Chunks restart at every segment: segment b owns chunks [cstart[b],
// cstart[b+1]), chunk c of it covering [off[b] + (c - cstart[b]) Gs, ...).
__device__ __forceinline__ uint32_t chunk_seg(const uint32_t *__restrict__ cstart, int64_t nseg, int64_t c) {
    uint32_t lo = 0, hi = (uint32_t)nseg - 1u;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1u) >> 1;
        if ((int64_t)cstart[mid] <= c) lo = mid;
        else hi = mid - 1u;
    }
    return lo;
}

// One warp per chunk: number of groups that start inside it (count pass,
// which also keeps the start flags of every 32-particle slice in cmask), then
// the group starts themselves (write pass, from cmask).
template <bool WRITE>
__global__ void __launch_bounds__(256) k_group_chunks(const uint64_t *__restrict__ skey, const uint8_t *__restrict__ plev,
                                                      const uint32_t *__restrict__ pleaf,
                                                      const uint32_t *__restrict__ nparent,
                                                      const uint32_t *__restrict__ ncount, uint32_t cmax,
                                                      int64_t n, int gs, int delta, int64_t nchunks,
                                                      const int64_t *__restrict__ seg_off,
                                                      const uint32_t *__restrict__ cstart, int64_t nseg,
                                                      uint32_t *__restrict__ ccount, const uint32_t *__restrict__ coff,
                                                      uint32_t *__restrict__ cmask, uint32_t *__restrict__ gfirst,
                                                      const uint32_t *__restrict__ ctr) {
    if (aborted(ctr, kStageAfter)) return;
    const int lane = threadIdx.x & 31;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= nchunks) return;
    int64_t s0 = c * gs, s1 = min(n, s0 + gs);
    if (nseg > 1) {
        const uint32_t b = chunk_seg(cstart, nseg, c);
        s0 = seg_off[b] + (c - (int64_t)cstart[b]) * gs;
        s1 = min(seg_off[b + 1], s0 + gs);
    }
    uint32_t base = WRITE ? coff[c] : 0u;
    uint32_t total = 0;
    for (int64_t off = 0; off < gs; off += 32) {
        const int64_t i = s0 + off + lane;
        uint32_t b;
        bool st;
        if (WRITE) {
            b = cmask[2 * c + (off >> 5)];
            st = (b >> lane) & 1u;
        } else {
            st = off + lane < gs && i < s1 && group_starts(skey, plev, pleaf, nparent, ncount, i, s0, delta, cmax);
            b = __ballot_sync(0xffffffffu, st);
            if (lane == 0) cmask[2 * c + (off >> 5)] = b;
        }
        if (WRITE && st) gfirst[base + total + __popc(b & lanemask_lt())] = (uint32_t)i;
        total += __popc(b);
    }
    if (!WRITE && lane == 0) ccount[c] = total;
    if (WRITE && lane == 0 && c == nchunks - 1) gfirst[ctr[kCtrGroups]] = (uint32_t)n;
}

// Exclusive scan of ccount into coff (single pass, decoupled look-back);
// the total is the group count.
__global__ void __launch_bounds__(kGScanThreads) k_group_scan(const uint32_t *__restrict__ ccount,
                                                              uint32_t *__restrict__ coff, int64_t nchunks,
                                                              uint32_t *status, uint32_t *ctr, int32_t *dstatus,
                                                              const DevCtl *__restrict__ ctl) {
    __shared__ uint32_t s_tile, s_excl, wt[32];
    if (aborted(ctr, kStageGroupScan)) return;
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr + kCtrGScanTicket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kGScanTile + (int64_t)threadIdx.x * kGScanItems;
    uint32_t v[kGScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kGScanItems; ++k) {
        v[k] = base + k < nchunks ? ccount[base + k] : 0u;
        sum += v[k];
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(sum, wt, &tot);
    if (threadIdx.x == 0)
        s_excl = lookback_single(status, tile, tot, WaitCtx{dstatus, ctr, kStageGroupScan, ctl->wait_cycles});
    __syncthreads();
    uint32_t run = s_excl + ex;
#pragma unroll
    for (int k = 0; k < kGScanItems; ++k) {
        if (base + k < nchunks) coff[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == kGScanThreads - 1 && (int64_t)(tile + 1) * kGScanTile >= nchunks) ctr[kCtrGroups] = run;
}

cudaError_t launch_groups(TreeWorkspace *ws, int64_t n, cudaStream_t s) {
    const int gs = ws->p.group_size;
    const int64_t nchunks = ws->nseg > 1 ? ws->seg_nchunks : (n + gs - 1) / gs;
    const int64_t tiles = (nchunks + kGScanTile - 1) / kGScanTile;
    cudaError_t e = cudaMemsetAsync(ws->gscan_status, 0, (size_t)tiles * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_leaf_levels<<<grid_for(ws->node_cap, 256, 152 * 8), 256, 0, s>>>(ws->ctr, ws->ngeo, ws->nlink, ws->plev,
                                                                        ws->pleaf);
    const unsigned wb = (unsigned)((nchunks * 32 + 255) / 256);
    const uint32_t cmax = 128u * (uint32_t)gs;
    k_group_chunks<false><<<wb, 256, 0, s>>>(ws->key, ws->plev, ws->pleaf, ws->nparent, ws->ncount, cmax, n, gs,
                                            ws->p.group_split, nchunks, ws->seg_off, ws->seg_cstart, ws->nseg, ws->ccount,
                                            nullptr, ws->cmask, nullptr, ws->ctr);
    k_group_scan<<<(unsigned)tiles, kGScanThreads, 0, s>>>(ws->ccount, ws->coff, nchunks, ws->gscan_status, ws->ctr,
                                                          ws->dstatus, ws->dctl);
    k_group_chunks<true><<<wb, 256, 0, s>>>(ws->key, ws->plev, ws->pleaf, ws->nparent, ws->ncount, cmax, n, gs,
                                           ws->p.group_split, nchunks, ws->seg_off, ws->seg_cstart, ws->nseg, nullptr,
                                           ws->coff, ws->cmask, ws->gfirst, ws->ctr);
    ws->launches += 4;
    return cudaGetLastError();
}

}  // namespace treegb
