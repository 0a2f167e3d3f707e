// api.cu -- the C ABI (include/treegb.h): workspace management, argument
// checks, call sequencing and the host-side opening-criterion table.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

using namespace treegb;

namespace {

#define TRY_CUDA(expr)                              \
    do {                                            \
        cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) return TREE_ERR_CUDA; \
    } while (0)

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

tree_status_t check_params(const TreeParams *p) {
    if (!p) return TREE_ERR_ARG;
    if (!(p->eps >= 0.0) || !isfinite(p->eps)) return TREE_ERR_ARG;
    if (!(p->theta >= 0.0) || !isfinite(p->theta)) return TREE_ERR_ARG;
    if (!isfinite(p->G)) return TREE_ERR_ARG;
    if (p->order != 0 && p->order != 2) return TREE_ERR_ARG;
    if (p->leaf_cap < 1 || p->leaf_cap > 16) return TREE_ERR_ARG;
    if (p->group_size != 16 && p->group_size != 32 && p->group_size != 64) return TREE_ERR_ARG;
    if (p->stack_depth < 256 || p->stack_depth > 8192 || p->stack_depth % 32) return TREE_ERR_ARG;
    if (p->precision != TREE_F32 && p->precision != TREE_F64) return TREE_ERR_ARG;
    if (p->kahan != 0 && p->kahan != 1) return TREE_ERR_ARG;
    if (p->group_split < 0 || p->group_split > kMaxLevel) return TREE_ERR_ARG;
    if (p->node_cap < 0 || p->node_cap >= kMaxNodes) return TREE_ERR_ARG;
    return TREE_OK;
}

// D_l = min{ d >= 0 : s_l^2 < fl(theta^2 * d) }, s_l = 2^(21-l); fl(theta^2 d) is
// non-decreasing in d, so a binary search over the exact predicate finds it.
// Group-cell distances satisfy d2 <= 3 (2^21)^2 < 2^44, so thresholds above
// that never accept.
void mac_table(double theta, int64_t *D) {
    const double th2 = theta * theta;
    const int64_t never = INT64_MAX;
    for (int l = 0; l < kLevels; ++l) {
        const int64_t s = (int64_t)1 << (kBits - l);
        const double s2 = (double)(s * s);
        if (!(th2 > 0.0)) { D[l] = never; continue; }
        int64_t lo = 0, hi = (int64_t)1 << 50;  // predicate false at lo=0 (s2 > 0), test hi
        if (!(s2 < th2 * (double)hi)) { D[l] = never; continue; }
        while (hi - lo > 1) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (s2 < th2 * (double)mid) hi = mid;
            else lo = mid;
        }
        D[l] = hi;
    }
}

int64_t default_node_cap(int64_t n_max, int leaf_cap) {
    // About 1.2 nodes per leaf-capacity worth of particles, with generous slack;
    // the build degrades gracefully (TREE_DEV_NODES) if a distribution needs more.
    double c = (double)n_max * (8.0 / (leaf_cap + 1.0) + 0.25) + 4096.0;
    if (c > (double)(kMaxNodes - 1)) c = (double)(kMaxNodes - 1);
    return (int64_t)c;
}

void free_all(TreeWorkspace *ws) {
    void *ptrs[] = {ws->key, ws->key_alt, ws->idx, ws->idx_alt, ws->hist, ws->sort_status, ws->level_status,
                    ws->ctr, ws->part, ws->box, ws->spos, ws->nfirst, ws->ncount, ws->ngeo, ws->nlink,
                    ws->mom64, ws->mom_a, ws->mom_b, ws->mom_c, ws->dstatus, ws->stats, ws->gstat,
                    ws->list_cnt, ws->pc_list, ws->pp_list, ws->direct_part, ws->dmac, ws->gorder,
                    ws->gkey, ws->gbucket, ws->gfirst, ws->plev, ws->ccount, ws->coff, ws->gscan_status,
                    ws->adj_cot, ws->adj_xt, ws->adj_xg, ws->adj_mg, ws->adj_ccot, ws->pleaf, ws->nparent,
                    ws->seg_off, ws->seg_cstart, ws->seg_bchunk, ws->seg_bfirst, ws->seg_part,
                    ws->seg_digit_off, ws->cmask, ws->morder, ws->mbucket, ws->xm, ws->hs_x, ws->hs_v,
                    ws->hs_m, ws->hs_a, ws->hs_phi, ws->hs_diag, ws->dctl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (ws->graph_exec) cudaGraphExecDestroy(ws->graph_exec);
    if (ws->graph) cudaGraphDestroy(ws->graph);
    if (ws->cap_stream) cudaStreamDestroy(ws->cap_stream);
    if (ws->copy_stream) cudaStreamDestroy(ws->copy_stream);
    if (ws->ev_drift) cudaEventDestroy(ws->ev_drift);
    if (ws->ev_xback) cudaEventDestroy(ws->ev_xback);
    ws->copy_stream = nullptr;
    ws->ev_drift = ws->ev_xback = nullptr;
    if (ws->side_stream) cudaStreamDestroy(ws->side_stream);
    if (ws->ev_fork) cudaEventDestroy(ws->ev_fork);
    if (ws->ev_join) cudaEventDestroy(ws->ev_join);
    ws->side_stream = nullptr;
    ws->ev_fork = ws->ev_join = nullptr;
    ws->graph_exec = nullptr;
    ws->graph = nullptr;
    ws->cap_stream = nullptr;
    for (cudaEvent_t e : ws->ev) cudaEventDestroy(e);
    ws->ev.clear();
    ws->ev_phase.clear();
}

template <typename T>
bool dalloc(T **p, size_t count) {
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T)) == cudaSuccess;
}

// Records a (start, stop) event pair around one phase when timing is on.
struct PhaseScope {
    TreeWorkspace *ws;
    cudaStream_t s;
    size_t pair = SIZE_MAX;
    int64_t l0 = 0;
    PhaseScope(TreeWorkspace *w, int phase, cudaStream_t st) : ws(w), s(st) {
        if (!ws->timing) return;
        l0 = ws->launches;
        if (ws->ev_used == ws->ev_phase.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
            ws->ev.push_back(a);
            ws->ev.push_back(b);
            ws->ev_phase.push_back(phase);
        }
        pair = ws->ev_used++;
        ws->ev_phase[pair] = phase;
        cudaEventRecord(ws->ev[2 * pair], s);
    }
    ~PhaseScope() {
        if (pair == SIZE_MAX) return;
        cudaEventRecord(ws->ev[2 * pair + 1], s);
        ws->timed_launches += ws->launches - l0;
    }
};

// Release the segment tables (back to a single system of any n).
void free_segments(TreeWorkspace *ws) {
    void *ptrs[] = {ws->seg_off, ws->seg_cstart, ws->seg_bchunk, ws->seg_bfirst, ws->seg_part, ws->seg_digit_off};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    ws->seg_off = nullptr;
    ws->seg_cstart = nullptr;
    ws->seg_bchunk = nullptr;
    ws->seg_bfirst = nullptr;
    ws->seg_part = nullptr;
    ws->seg_digit_off = nullptr;
    ws->seg_off_h.clear();
    ws->nseg = 1;
    ws->seg_passes = 0;
    ws->seg_nbchunk = 0;
    ws->seg_nchunks = 0;
    ws->seg_cstart_gs = 0;
}

void drop_graph(TreeWorkspace *ws) {
    if (ws->graph_exec) cudaGraphExecDestroy(ws->graph_exec);
    if (ws->graph) cudaGraphDestroy(ws->graph);
    ws->graph_exec = nullptr;
    ws->graph = nullptr;
    ws->graph_launches = 0;
}

// First Gs chunk of every segment for the current group size (synchronous
// upload; called when the segments or the group size change, never inside
// a step, so that a step stays free of host synchronisation).
tree_status_t upload_seg_chunks(TreeWorkspace *ws) {
    if (ws->nseg <= 1 || ws->seg_cstart_gs == ws->p.group_size) return TREE_OK;
    const int64_t gs = ws->p.group_size;
    std::vector<uint32_t> cs((size_t)ws->nseg + 1);
    int64_t c = 0;
    for (int64_t b = 0; b < ws->nseg; ++b) {
        cs[b] = (uint32_t)c;
        c += (ws->seg_off_h[b + 1] - ws->seg_off_h[b] + gs - 1) / gs;
    }
    cs[ws->nseg] = (uint32_t)c;
    TRY_CUDA(cudaMemcpy(ws->seg_cstart, cs.data(), cs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    ws->seg_nchunks = c;
    ws->seg_cstart_gs = ws->p.group_size;
    return TREE_OK;
}

// Step and build calls: n must match the segments when they are set.
tree_status_t check_n(const TreeWorkspace *ws, int64_t n) {
    if (n < 0) return TREE_ERR_ARG;
    if (n > ws->n_max) return TREE_ERR_CAPACITY;
    if (ws->nseg > 1 && n != ws->seg_off_h[ws->nseg]) return TREE_ERR_ARG;
    return TREE_OK;
}

tree_status_t upload_mac(TreeWorkspace *ws, cudaStream_t s) {
    if (ws->mac_theta != ws->p.theta) {
        mac_table(ws->p.theta, ws->mac_D);
        ws->mac_theta = ws->p.theta;
        // synchronous copy from pageable host memory: the table is 176 bytes
        TRY_CUDA(cudaMemcpyAsync(ws->dmac, ws->mac_D, sizeof(ws->mac_D), cudaMemcpyHostToDevice, s));
        TRY_CUDA(cudaStreamSynchronize(s));
    }
    return TREE_OK;
}

}  // namespace

extern "C" {

const char *tree_version(void) { return "treegb 0.1"; }

const char *tree_status_string(tree_status_t s) {
    switch (s) {
        case TREE_OK: return "ok";
        case TREE_ERR_ARG: return "invalid argument";
        case TREE_ERR_CUDA: return "CUDA runtime error";
        case TREE_ERR_ALLOC: return "device allocation failed";
        case TREE_ERR_CAPACITY: return "size exceeds a fixed capacity (workspace n_max, or the no-allocation target limit)";
        case TREE_ERR_STATE: return "call order violated";
        case TREE_ERR_DEVICE: return "device status word is set";
    }
    return "unknown status";
}

tree_status_t tree_params_default(TreeParams *p) {
    if (!p) return TREE_ERR_ARG;
    p->G = 1.0;
    p->eps = 0.01;
    p->theta = 0.7;
    p->order = 2;
    p->leaf_cap = 16;
    p->group_size = 32;
    p->stack_depth = 1024;
    p->precision = TREE_F32;
    p->kahan = 1;
    p->group_split = 3;
    p->node_cap = 0;
    return TREE_OK;
}

tree_status_t tree_mac_table(double theta, int64_t *D) {
    if (!D || !(theta >= 0.0) || !isfinite(theta)) return TREE_ERR_ARG;
    mac_table(theta, D);
    return TREE_OK;
}

tree_status_t tree_workspace_create(int64_t n_max, const TreeParams *p, TreeWorkspace **out) {
    if (!out) return TREE_ERR_ARG;
    *out = nullptr;
    tree_status_t st = check_params(p);
    if (st != TREE_OK) return st;
    if (n_max < 0 || n_max >= (int64_t)kValMask) return TREE_ERR_ARG;
    TreeWorkspace *ws = new (std::nothrow) TreeWorkspace();
    if (!ws) return TREE_ERR_ALLOC;
    ws->p = *p;
    if (cudaGetDevice(&ws->device) != cudaSuccess) { delete ws; return TREE_ERR_CUDA; }
    ws->n_max = n_max;
    ws->node_cap = p->node_cap > 0 ? p->node_cap : default_node_cap(n_max, p->leaf_cap);
    ws->real_size = p->precision == TREE_F64 ? 8 : 4;
    const size_t N = (size_t)(n_max > 0 ? n_max : 1);
    const size_t NC = (size_t)ws->node_cap;
    ws->sort_tiles_max = (n_max + kSortTile - 1) / kSortTile + 1;
    ws->level_tiles_max = (ws->node_cap + kLevelThreads - 1) / kLevelThreads + 1;
    ws->groups_max = n_max + 1;  // a group holds at least one particle
    const int64_t chunks_max = (n_max + 15) / 16 + 1;
    const size_t v4 = p->precision == TREE_F64 ? sizeof(double4a) : sizeof(float4);
    const size_t v2 = p->precision == TREE_F64 ? sizeof(double2a) : sizeof(float2);
    bool ok = dalloc(&ws->key, N) && dalloc(&ws->key_alt, N) && dalloc(&ws->idx, N) && dalloc(&ws->idx_alt, N) &&
              dalloc(&ws->hist, 2 * kSortPasses * kRadix) &&
              dalloc(&ws->sort_status, (size_t)(kSortPasses + kSegPassesMax) * ws->sort_tiles_max * kRadix) &&
              dalloc(&ws->level_status, (size_t)kLevels * ws->level_tiles_max) && dalloc(&ws->ctr, kCtrCount) &&
              dalloc(&ws->part, (size_t)kMaxBlocksReduce * 8) && dalloc(&ws->box, 1) &&
              dalloc((unsigned char **)&ws->spos, N * v4) && dalloc((unsigned char **)&ws->xm, N * v4) &&
              dalloc(&ws->nfirst, NC) && dalloc(&ws->ncount, NC) &&
              dalloc(&ws->ngeo, NC) && dalloc(&ws->nlink, NC) && dalloc(&ws->mom64, 10 * NC) &&
              dalloc(&ws->morder, NC) && dalloc(&ws->mbucket, 3 * kMomBuckets + 1) &&
              dalloc((unsigned char **)&ws->mom_a, NC * v4) && dalloc((unsigned char **)&ws->mom_b, NC * v4) &&
              dalloc((unsigned char **)&ws->mom_c, NC * v2) && dalloc(&ws->dstatus, 1) &&
              dalloc(&ws->stats, kStatCount) && dalloc(&ws->gstat, (size_t)ws->groups_max) &&
              dalloc(&ws->gorder, (size_t)ws->groups_max) && dalloc(&ws->gkey, (size_t)ws->groups_max) &&
              dalloc(&ws->gbucket, 64) && dalloc(&ws->gfirst, (size_t)ws->groups_max + 1) &&
              dalloc(&ws->plev, N) && dalloc(&ws->pleaf, N) && dalloc(&ws->nparent, NC) &&
              dalloc(&ws->ccount, (size_t)chunks_max) && dalloc(&ws->coff, (size_t)chunks_max) &&
              dalloc(&ws->cmask, 2 * (size_t)chunks_max) &&
              dalloc(&ws->gscan_status, (size_t)(chunks_max / 2048 + 2)) &&
              dalloc(&ws->dmac, kLevels) && dalloc(&ws->dctl, 1);
    ws->chunks_cap = chunks_max;
    ws->box_cap = 1;
    if (!ok) {
        free_all(ws);
        delete ws;
        cudaGetLastError();
        return TREE_ERR_ALLOC;
    }
    const DevCtl ctl{kWaitCycles, -1};
    if (cudaMemset(ws->dstatus, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(ws->stats, 0, kStatCount * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemcpy(ws->dctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_all(ws);
        delete ws;
        return TREE_ERR_CUDA;
    }
    *out = ws;
    return TREE_OK;
}

tree_status_t tree_workspace_destroy(TreeWorkspace *ws) {
    if (!ws) return TREE_ERR_ARG;
    cudaDeviceSynchronize();
    free_all(ws);
    delete ws;
    return TREE_OK;
}

tree_status_t tree_set_params(TreeWorkspace *ws, const TreeParams *p) {
    if (!ws) return TREE_ERR_ARG;
    tree_status_t st = check_params(p);
    if (st != TREE_OK) return st;
    if (p->leaf_cap != ws->p.leaf_cap || p->precision != ws->p.precision) return TREE_ERR_ARG;
    const bool regroup = p->group_size != ws->p.group_size || p->group_split != ws->p.group_split;
    const int64_t keep_cap = ws->p.node_cap;
    ws->p = *p;
    ws->p.node_cap = keep_cap;
    // a captured step holds the old parameters
    drop_graph(ws);
    if (regroup) {
        // the walk groups come from the tree build: a new grouping needs a new build
        ws->list_groups = -1;
        ws->built = false;
        ws->has_moments = false;
        TRY_CUDA(cudaDeviceSynchronize());
        tree_status_t st2 = upload_seg_chunks(ws);
        if (st2 != TREE_OK) return st2;
    }
    return TREE_OK;
}

tree_status_t tree_set_segments(TreeWorkspace *ws, int64_t nseg, const int64_t *offsets) {
    if (!ws) return TREE_ERR_ARG;
    if (nseg < 0 || nseg > kMaxSegments) return TREE_ERR_ARG;
    if (nseg > 1) {
        if (!offsets || offsets[0] != 0) return TREE_ERR_ARG;
        for (int64_t b = 0; b < nseg; ++b)
            if (offsets[b + 1] <= offsets[b]) return TREE_ERR_ARG;
        if (offsets[nseg] > ws->n_max) return TREE_ERR_CAPACITY;
        if (nseg >= ws->node_cap) return TREE_ERR_CAPACITY;
    }
    // the tables below may be in use by queued work
    TRY_CUDA(cudaDeviceSynchronize());
    drop_graph(ws);
    free_segments(ws);
    ws->built = false;
    ws->has_moments = false;
    ws->list_groups = -1;
    if (nseg <= 1) return TREE_OK;
    const int64_t n = offsets[nseg];
    // box chunks of at most kBoxChunk particles, never straddling segments
    std::vector<uint4> bch;
    std::vector<uint32_t> bfirst((size_t)nseg + 1);
    for (int64_t b = 0; b < nseg; ++b) {
        bfirst[b] = (uint32_t)bch.size();
        for (int64_t i = offsets[b]; i < offsets[b + 1]; i += kBoxChunk) {
            const int64_t e = i + kBoxChunk < offsets[b + 1] ? i + kBoxChunk : offsets[b + 1];
            bch.push_back(make_uint4((uint32_t)i, (uint32_t)e, (uint32_t)b, 0u));
        }
    }
    bfirst[nseg] = (uint32_t)bch.size();
    // exclusive offsets of the segment-index digits (low byte, high byte)
    std::vector<uint32_t> doff(2 * kRadix, 0u);
    {
        std::vector<int64_t> cnt(2 * kRadix, 0);
        for (int64_t b = 0; b < nseg; ++b) {
            const int64_t sz = offsets[b + 1] - offsets[b];
            cnt[b & 0xff] += sz;
            cnt[kRadix + ((b >> 8) & 0xff)] += sz;
        }
        for (int q = 0; q < 2; ++q) {
            int64_t run = 0;
            for (int d = 0; d < kRadix; ++d) {
                doff[q * kRadix + d] = (uint32_t)run;
                run += cnt[q * kRadix + d];
            }
        }
    }
    const int64_t chunks_need = (n + 15) / 16 + nseg + 1;
    bool ok = dalloc(&ws->seg_off, (size_t)nseg + 1) && dalloc(&ws->seg_cstart, (size_t)nseg + 1) &&
              dalloc(&ws->seg_bchunk, bch.size()) && dalloc(&ws->seg_bfirst, (size_t)nseg + 1) &&
              dalloc(&ws->seg_part, bch.size() * 8) && dalloc(&ws->seg_digit_off, 2 * kRadix);
    if (ok && nseg > ws->box_cap) {
        cudaFree(ws->box);
        ws->box = nullptr;
        ok = dalloc(&ws->box, (size_t)nseg);
        ws->box_cap = ok ? nseg : 0;
    }
    if (ok && chunks_need > ws->chunks_cap) {
        cudaFree(ws->ccount);
        cudaFree(ws->coff);
        cudaFree(ws->cmask);
        cudaFree(ws->gscan_status);
        ws->ccount = ws->coff = ws->cmask = ws->gscan_status = nullptr;
        ok = dalloc(&ws->ccount, (size_t)chunks_need) && dalloc(&ws->coff, (size_t)chunks_need) &&
             dalloc(&ws->cmask, 2 * (size_t)chunks_need) &&
             dalloc(&ws->gscan_status, (size_t)(chunks_need / 2048 + 2));
        ws->chunks_cap = ok ? chunks_need : 0;
    }
    if (!ok) {
        cudaGetLastError();
        free_segments(ws);
        return TREE_ERR_ALLOC;
    }
    TRY_CUDA(cudaMemcpy(ws->seg_off, offsets, ((size_t)nseg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemcpy(ws->seg_bchunk, bch.data(), bch.size() * sizeof(uint4), cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemcpy(ws->seg_bfirst, bfirst.data(), bfirst.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    TRY_CUDA(cudaMemcpy(ws->seg_digit_off, doff.data(), doff.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    ws->seg_off_h.assign(offsets, offsets + nseg + 1);
    ws->nseg = nseg;
    ws->seg_passes = nseg <= 256 ? 1 : 2;
    ws->seg_nbchunk = (int64_t)bch.size();
    return upload_seg_chunks(ws);
}

tree_status_t tree_get_segments(const TreeWorkspace *ws, int64_t *nseg) {
    if (!ws || !nseg) return TREE_ERR_ARG;
    *nseg = ws->nseg;
    return TREE_OK;
}

tree_status_t tree_get_params(const TreeWorkspace *ws, TreeParams *p) {
    if (!ws || !p) return TREE_ERR_ARG;
    *p = ws->p;
    return TREE_OK;
}

tree_status_t tree_build(TreeWorkspace *ws, const void *x, int64_t n, int32_t dtype, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    tree_status_t stn = check_n(ws, n);
    if (stn != TREE_OK) return stn;
    if (dtype != ws->p.precision) return TREE_ERR_ARG;
    if (n > 0 && !x) return TREE_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    ws->n = n;
    ws->built = false;
    ws->has_moments = false;
    ws->list_groups = -1;
    if (n == 0) { ws->built = true; return TREE_OK; }
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, kCtrCount * sizeof(uint32_t), s));
    TRY_CUDA(cudaMemsetAsync(ws->hist, 0, kSortPasses * kRadix * sizeof(uint32_t), s));
    for (int p = 0; p < kSortPasses + ws->seg_passes; ++p)
        TRY_CUDA(cudaMemsetAsync(ws->sort_status + (size_t)p * ws->sort_tiles_max * kRadix, 0,
                                 (size_t)tiles * kRadix * sizeof(uint32_t), s));
    TRY_CUDA(cudaMemsetAsync(ws->level_status, 0, (size_t)kLevels * ws->level_tiles_max * sizeof(uint32_t), s));
    {
        PhaseScope ph(ws, TREE_PHASE_BOX, s);
        TRY_CUDA(launch_box(ws, x, n, s));
    }
    {
        PhaseScope ph(ws, TREE_PHASE_KEYS, s);
        TRY_CUDA(launch_keys(ws, x, n, s));
    }
    {
        PhaseScope ph(ws, TREE_PHASE_SORT, s);
        TRY_CUDA(launch_sort(ws, n, s));
    }
    {
        PhaseScope ph(ws, TREE_PHASE_OCTREE, s);
        TRY_CUDA(launch_octree(ws, n, s));
        TRY_CUDA(launch_groups(ws, n, s));
    }
    ws->built = true;
    return TREE_OK;
}

tree_status_t tree_moments(TreeWorkspace *ws, const void *x, const void *m, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (!ws->built) return TREE_ERR_STATE;
    if (ws->n == 0) { ws->has_moments = true; return TREE_OK; }
    if (!x || !m) return TREE_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    {
        PhaseScope ph(ws, TREE_PHASE_GATHER, s);
        TRY_CUDA(launch_gather(ws, x, m, ws->n, s));
    }
    {
        PhaseScope ph(ws, TREE_PHASE_MOMENTS, s);
        TRY_CUDA(launch_moments(ws, s));
    }
    ws->has_moments = true;
    return TREE_OK;
}

static tree_status_t walk(TreeWorkspace *ws, int mode, const WalkOut &out, cudaStream_t s) {
    tree_status_t st = upload_mac(ws, s);
    if (st != TREE_OK) return st;
    PhaseScope ph(ws, mode == kWalkForce ? TREE_PHASE_WALK : TREE_PHASE_LISTS, s);
    if (walk_widest_first(ws)) TRY_CUDA(launch_group_order(ws, s));
    if (ws->p.precision == TREE_F64) TRY_CUDA(launch_walk_f64(ws, mode, out, s));
    else TRY_CUDA(launch_walk_f32(ws, mode, out, s));
    return TREE_OK;
}

static tree_status_t build_lists(TreeWorkspace *ws, cudaStream_t s) {
    uint32_t ngd = 0;
    TRY_CUDA(cudaMemcpyAsync(&ngd, ws->ctr + kCtrGroups, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t ng = ngd;
    ws->list_groups_host = ng;
    WalkOut none{nullptr, nullptr, nullptr, 0.0};
    tree_status_t st = walk(ws, kWalkCount, none, s);
    if (st != TREE_OK) return st;
    if (!ws->list_cnt && !dalloc(&ws->list_cnt, (size_t)(2 * (ws->groups_max + 1)))) return TREE_ERR_ALLOC;
    {
        PhaseScope ph(ws, TREE_PHASE_LISTS, s);
        TRY_CUDA(launch_scan_lists(ws, ng, s));
    }
    int64_t tot[2];
    TRY_CUDA(cudaMemcpyAsync(&tot[0], ws->list_cnt + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaMemcpyAsync(&tot[1], ws->list_cnt + (ng + 1) + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    if (tot[0] > ws->list_pc_cap) {
        if (ws->pc_list) cudaFree(ws->pc_list);
        ws->pc_list = nullptr;
        ws->list_pc_cap = 0;
        if (!dalloc(&ws->pc_list, (size_t)tot[0])) return TREE_ERR_ALLOC;
        ws->list_pc_cap = tot[0];
    }
    if (tot[1] > ws->list_pp_cap) {
        if (ws->pp_list) cudaFree(ws->pp_list);
        ws->pp_list = nullptr;
        ws->list_pp_cap = 0;
        if (!dalloc(&ws->pp_list, (size_t)tot[1])) return TREE_ERR_ALLOC;
        ws->list_pp_cap = tot[1];
    }
    st = walk(ws, kWalkEmit, none, s);
    if (st != TREE_OK) return st;
    ws->list_pc = tot[0];
    ws->list_pp = tot[1];
    ws->list_groups = ng;
    return TREE_OK;
}

tree_status_t tree_forces(TreeWorkspace *ws, void *a, void *phi, int32_t flags, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (!ws->has_moments) return TREE_ERR_STATE;
    if (ws->n == 0) return TREE_OK;
    const bool lists_only = (flags & TREE_FLAG_EMIT_LISTS) && (flags & TREE_FLAG_LISTS_ONLY);
    if (!a && !lists_only) return TREE_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (flags & TREE_FLAG_EMIT_LISTS) {
        tree_status_t st = build_lists(ws, s);
        if (st != TREE_OK) return st;
        if (lists_only) return TREE_OK;
    }
    WalkOut out{a, phi, nullptr, 0.0};
    return walk(ws, kWalkForce, out, s);
}

static tree_status_t adjoint_ready(TreeWorkspace *ws) {
    if (!ws->has_moments || ws->list_groups < 0) return TREE_ERR_STATE;
    if (!ws->adj_xt) {
        const size_t N = (size_t)ws->n_max, NC = (size_t)ws->node_cap;
        const size_t v4 = ws->p.precision == TREE_F64 ? sizeof(double4a) : sizeof(float4);
        if (!(dalloc((unsigned char **)&ws->adj_cot, N * v4) && dalloc(&ws->adj_xt, 3 * N) &&
              dalloc(&ws->adj_xg, 3 * N) && dalloc(&ws->adj_mg, N) && dalloc(&ws->adj_ccot, 10 * NC))) {
            return TREE_ERR_ALLOC;
        }
    }
    return TREE_OK;
}

tree_status_t tree_forces_adjoint(TreeWorkspace *ws, const void *a_bar, const void *phi_bar, void *x_bar, void *m_bar,
                                  void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (ws->n > 0 && (!a_bar || (!x_bar && !m_bar))) return TREE_ERR_ARG;
    tree_status_t st = adjoint_ready(ws);
    if (st != TREE_OK) return st;
    if (ws->n == 0) return TREE_OK;
    cudaStream_t s = as_stream(stream);
    PhaseScope ph(ws, TREE_PHASE_ADJOINT, s);
    TRY_CUDA(launch_adjoint(ws, a_bar, phi_bar, x_bar, m_bar, s));
    return TREE_OK;
}

tree_status_t leapfrog_adjoint_step(TreeWorkspace *ws, void *x_bar, void *v_bar, void *a_bar, void *m_bar,
                                    const void *phi_bar, double tau, void *stream) {
    if (!ws || !isfinite(tau)) return TREE_ERR_ARG;
    if (ws->n > 0 && (!x_bar || !v_bar || !a_bar || !m_bar)) return TREE_ERR_ARG;
    tree_status_t st = adjoint_ready(ws);
    if (st != TREE_OK) return st;
    if (ws->n == 0) return TREE_OK;
    cudaStream_t s = as_stream(stream);
    PhaseScope ph(ws, TREE_PHASE_ADJOINT, s);
    TRY_CUDA(launch_adjoint_step(ws, x_bar, v_bar, a_bar, m_bar, phi_bar, tau, s));
    return TREE_OK;
}

tree_status_t tree_energy_vjp(TreeWorkspace *ws, const void *m, const void *phi, const double *w_bar, int64_t n,
                              void *phi_bar, void *m_bar, void *stream) {
    if (!ws || n < 0) return TREE_ERR_ARG;
    if (n == 0) return TREE_OK;
    if (!m || !phi || !w_bar || (!phi_bar && !m_bar)) return TREE_ERR_ARG;
    TRY_CUDA(launch_energy_vjp(ws, m, phi, w_bar, n, phi_bar, m_bar, as_stream(stream)));
    return TREE_OK;
}

tree_status_t tree_accel(TreeWorkspace *ws, const void *x, const void *m, int64_t n, void *a, void *phi,
                         void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (n > 0 && (!x || !m || !a)) return TREE_ERR_ARG;
    tree_status_t st = tree_build(ws, x, n, ws->p.precision, stream);
    if (st != TREE_OK) return st;
    st = tree_moments(ws, x, m, stream);
    if (st != TREE_OK) return st;
    return tree_forces(ws, a, phi, 0, stream);
}

// The side stream and events a leapfrog step forks its walk groups onto
// (created outside any stream capture).
static tree_status_t ensure_side_stream(TreeWorkspace *ws) {
    if (!ws->side_stream) TRY_CUDA(cudaStreamCreateWithFlags(&ws->side_stream, cudaStreamNonBlocking));
    if (!ws->ev_fork) TRY_CUDA(cudaEventCreateWithFlags(&ws->ev_fork, cudaEventDisableTiming));
    if (!ws->ev_join) TRY_CUDA(cudaEventCreateWithFlags(&ws->ev_join, cudaEventDisableTiming));
    return TREE_OK;
}

// First part of a step: the first kick and the drift (Eqs. 2-3), fused with
// the box of the new positions.  After it, x holds r^{n+1} and is only read.
static tree_status_t leapfrog_begin(TreeWorkspace *ws, void *x, void *v, const void *m, void *a, double tau,
                                    int64_t n, cudaStream_t s) {
    ws->n = n;
    ws->built = false;
    ws->has_moments = false;
    ws->list_groups = -1;
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, kCtrCount * sizeof(uint32_t), s));
    TRY_CUDA(cudaMemsetAsync(ws->hist, 0, kSortPasses * kRadix * sizeof(uint32_t), s));
    for (int p = 0; p < kSortPasses + ws->seg_passes; ++p)
        TRY_CUDA(cudaMemsetAsync(ws->sort_status + (size_t)p * ws->sort_tiles_max * kRadix, 0,
                                 (size_t)tiles * kRadix * sizeof(uint32_t), s));
    TRY_CUDA(cudaMemsetAsync(ws->level_status, 0, (size_t)kLevels * ws->level_tiles_max * sizeof(uint32_t), s));
    // Eqs. 2-3 fused with the box of the new positions
    PhaseScope ph(ws, TREE_PHASE_BOX, s);
    TRY_CUDA(launch_kick_drift_box(ws, x, v, a, m, tau, n, s));
    return TREE_OK;
}

// Rest of a step: the tree at r^{n+1} (Eq. 4) and the forces, written back
// with the second kick (Eq. 5) fused in.
static tree_status_t leapfrog_finish(TreeWorkspace *ws, const void *x, void *v, void *a, void *phi, double tau,
                                     int64_t n, cudaStream_t s, void *v_mirror = nullptr,
                                     void *phi_mirror = nullptr) {
    {
        PhaseScope ph(ws, TREE_PHASE_KEYS, s);
        TRY_CUDA(launch_keys(ws, x, n, s));
    }
    {
        PhaseScope ph(ws, TREE_PHASE_SORT, s);
        TRY_CUDA(launch_sort(ws, n, s));
    }
    {
        // The walk groups need the octree only, and the gather and the moments
        // do not need the groups: the groups run on the side stream meanwhile
        // (their kernels wait on dependent loads, the moments on the FP64 pipe)
        // and are joined before the walk.  The phase's events, on s, time the
        // octree; its launch count includes the groups.
        PhaseScope ph(ws, TREE_PHASE_OCTREE, s);
        TRY_CUDA(launch_octree(ws, n, s));
        TRY_CUDA(cudaEventRecord(ws->ev_fork, s));
        TRY_CUDA(cudaStreamWaitEvent(ws->side_stream, ws->ev_fork, 0));
        TRY_CUDA(launch_groups(ws, n, ws->side_stream));
        TRY_CUDA(cudaEventRecord(ws->ev_join, ws->side_stream));
    }
    ws->built = true;
    {
        PhaseScope ph(ws, TREE_PHASE_GATHER, s);
        TRY_CUDA(launch_gather_packed(ws, n, s));
    }
    {
        PhaseScope ph(ws, TREE_PHASE_MOMENTS, s);
        TRY_CUDA(launch_moments(ws, s));
    }
    ws->has_moments = true;
    TRY_CUDA(cudaStreamWaitEvent(s, ws->ev_join, 0));
    WalkOut out{a, phi, v, 0.5 * tau};
    out.v_mirror = v_mirror;
    out.phi_mirror = phi_mirror;
    return walk(ws, kWalkForce, out, s);
}

tree_status_t leapfrog_step(TreeWorkspace *ws, void *x, void *v, const void *m, void *a, void *phi, double tau,
                            int64_t n, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (!isfinite(tau)) return TREE_ERR_ARG;
    tree_status_t stn = check_n(ws, n);
    if (stn != TREE_OK) return stn;
    if (n == 0) return TREE_OK;
    if (!x || !v || !m || !a) return TREE_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    tree_status_t st = ensure_side_stream(ws);
    if (st != TREE_OK) return st;
    st = leapfrog_begin(ws, x, v, m, a, tau, n, s);
    if (st != TREE_OK) return st;
    return leapfrog_finish(ws, x, v, a, phi, tau, n, s);
}

tree_status_t leapfrog_step_host(TreeWorkspace *ws, void *x, void *v, const void *m, void *a, void *phi, double tau,
                                 int64_t n, double *diag, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (!isfinite(tau)) return TREE_ERR_ARG;
    tree_status_t st = check_n(ws, n);
    if (st != TREE_OK) return st;
    if (n == 0) return TREE_OK;
    if (!x || !v || !m || !a) return TREE_ERR_ARG;
    const size_t rs = ws->real_size, N = (size_t)ws->n_max;
    if (!ws->hs_x) {
        if (!(dalloc((unsigned char **)&ws->hs_x, 3 * N * rs) && dalloc((unsigned char **)&ws->hs_v, 3 * N * rs) &&
              dalloc((unsigned char **)&ws->hs_m, N * rs) && dalloc((unsigned char **)&ws->hs_a, 3 * N * rs) &&
              dalloc((unsigned char **)&ws->hs_phi, N * rs) && dalloc(&ws->hs_diag, 8))) {
            cudaGetLastError();
            return TREE_ERR_ALLOC;
        }
    }
    if (!ws->copy_stream) TRY_CUDA(cudaStreamCreateWithFlags(&ws->copy_stream, cudaStreamNonBlocking));
    if (!ws->ev_drift) TRY_CUDA(cudaEventCreateWithFlags(&ws->ev_drift, cudaEventDisableTiming));
    if (!ws->ev_xback) TRY_CUDA(cudaEventCreateWithFlags(&ws->ev_xback, cudaEventDisableTiming));
    st = ensure_side_stream(ws);
    if (st != TREE_OK) return st;
    cudaStream_t s = as_stream(stream);
    const size_t b3 = 3 * (size_t)n * rs, b1 = (size_t)n * rs;
    {
        PhaseScope ph(ws, TREE_PHASE_H2D, s);
        TRY_CUDA(cudaMemcpyAsync(ws->hs_x, x, b3, cudaMemcpyHostToDevice, s));
        TRY_CUDA(cudaMemcpyAsync(ws->hs_v, v, b3, cudaMemcpyHostToDevice, s));
        TRY_CUDA(cudaMemcpyAsync(ws->hs_m, m, b1, cudaMemcpyHostToDevice, s));
        TRY_CUDA(cudaMemcpyAsync(ws->hs_a, a, b3, cudaMemcpyHostToDevice, s));
    }
    st = leapfrog_begin(ws, ws->hs_x, ws->hs_v, ws->hs_m, ws->hs_a, tau, n, s);
    if (st != TREE_OK) return st;
    // r^{n+1} is final once the drift has run: copy it back on a second
    // stream while the tree is built and walked
    TRY_CUDA(cudaEventRecord(ws->ev_drift, s));
    TRY_CUDA(cudaStreamWaitEvent(ws->copy_stream, ws->ev_drift, 0));
    TRY_CUDA(cudaMemcpyAsync(x, ws->hs_x, b3, cudaMemcpyDeviceToHost, ws->copy_stream));
    TRY_CUDA(cudaEventRecord(ws->ev_xback, ws->copy_stream));
    // Where the caller's v, a (and phi) are mapped page-locked memory, the walk
    // writes the new a, the kicked v and phi into them as it goes (besides the
    // device copies that the diagnostics read), so nothing is left to copy
    // back after it; otherwise they are copied back after the walk.
    void *va = nullptr, *aa = nullptr, *pa = nullptr;
    const bool mapped = cudaHostGetDevicePointer(&va, v, 0) == cudaSuccess &&
                        cudaHostGetDevicePointer(&aa, a, 0) == cudaSuccess &&
                        (!phi || cudaHostGetDevicePointer(&pa, phi, 0) == cudaSuccess);
    if (!mapped) cudaGetLastError();  // not mapped: the copies back below
    st = mapped ? leapfrog_finish(ws, ws->hs_x, ws->hs_v, aa, ws->hs_phi, tau, n, s, va, pa)
                : leapfrog_finish(ws, ws->hs_x, ws->hs_v, ws->hs_a, ws->hs_phi, tau, n, s);
    if (st != TREE_OK) return st;
    if (diag) {
        PhaseScope ph(ws, TREE_PHASE_DIAG, s);
        TRY_CUDA(launch_diagnostics(ws, ws->hs_x, ws->hs_v, ws->hs_m, ws->hs_phi, n, ws->hs_diag, s));
    }
    {
        PhaseScope ph(ws, TREE_PHASE_D2H, s);
        if (!mapped) {
            TRY_CUDA(cudaMemcpyAsync(v, ws->hs_v, b3, cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaMemcpyAsync(a, ws->hs_a, b3, cudaMemcpyDeviceToHost, s));
            if (phi) TRY_CUDA(cudaMemcpyAsync(phi, ws->hs_phi, b1, cudaMemcpyDeviceToHost, s));
        }
        if (diag) TRY_CUDA(cudaMemcpyAsync(diag, ws->hs_diag, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    // the caller's stream completes only after x's copy has landed too
    TRY_CUDA(cudaStreamWaitEvent(s, ws->ev_xback, 0));
    return TREE_OK;
}

tree_status_t tree_diagnostics(TreeWorkspace *ws, const void *x, const void *v, const void *m, const void *phi,
                               int64_t n, double *out, void *stream) {
    if (!ws || !out || n < 0) return TREE_ERR_ARG;
    if (n > 0 && (!x || !v || !m)) return TREE_ERR_ARG;
    PhaseScope ph(ws, TREE_PHASE_DIAG, as_stream(stream));
    TRY_CUDA(launch_diagnostics(ws, x, v, m, phi, n, out, as_stream(stream)));
    return TREE_OK;
}

tree_status_t tree_diagnostics_segments(TreeWorkspace *ws, const void *x, const void *v, const void *m,
                                        const void *phi, int64_t n, double *out, void *stream) {
    if (!ws || !out) return TREE_ERR_ARG;
    tree_status_t stn = check_n(ws, n);
    if (stn != TREE_OK) return stn;
    if (ws->nseg <= 1) return tree_diagnostics(ws, x, v, m, phi, n, out, stream);
    if (!x || !v || !m) return TREE_ERR_ARG;
    PhaseScope ph(ws, TREE_PHASE_DIAG, as_stream(stream));
    TRY_CUDA(launch_diagnostics_segments(ws, x, v, m, phi, n, out, as_stream(stream)));
    return TREE_OK;
}

tree_status_t leapfrog_graph_capture(TreeWorkspace *ws, void *x, void *v, const void *m, void *a, void *phi,
                                     double tau, int64_t n, double *diag) {
    if (!ws) return TREE_ERR_ARG;
    if (!isfinite(tau)) return TREE_ERR_ARG;
    tree_status_t st = check_n(ws, n);
    if (st != TREE_OK) return st;
    if (n == 0 || !x || !v || !m || !a) return TREE_ERR_ARG;
    TRY_CUDA(cudaDeviceSynchronize());
    drop_graph(ws);
    if (!ws->cap_stream) TRY_CUDA(cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking));
    st = ensure_side_stream(ws);
    if (st != TREE_OK) return st;
    cudaStream_t cs = ws->cap_stream;
    // everything a step may do on the host first (the opening-criterion table)
    st = upload_mac(ws, cs);
    if (st != TREE_OK) return st;
    const bool timing = ws->timing;
    ws->timing = false;
    const int64_t l0 = ws->launches;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        ws->timing = timing;
        return TREE_ERR_CUDA;
    }
    st = leapfrog_step(ws, x, v, m, a, phi, tau, n, cs);
    if (st == TREE_OK && diag) st = tree_diagnostics(ws, x, v, m, phi, n, diag, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    ws->timing = timing;
    const int64_t captured = ws->launches - l0;
    ws->launches = l0;
    // nothing ran: the workspace holds no tree of these positions yet
    ws->built = false;
    ws->has_moments = false;
    ws->list_groups = -1;
    if (st != TREE_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != TREE_OK ? st : TREE_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return TREE_ERR_CUDA;
    }
    ws->graph = g;
    ws->graph_exec = ex;
    ws->graph_launches = captured;
    ws->graph_n = n;
    return TREE_OK;
}

tree_status_t leapfrog_graph_launch(TreeWorkspace *ws, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (!ws->graph_exec) return TREE_ERR_STATE;
    TRY_CUDA(cudaGraphLaunch(ws->graph_exec, as_stream(stream)));
    ws->launches += ws->graph_launches;
    ws->n = ws->graph_n;
    ws->built = true;
    ws->has_moments = true;
    ws->list_groups = -1;
    return TREE_OK;
}

namespace {
// Force-error reference of the autotuner: the FP64 direct sum of Eq. 1 for a
// fixed sample of targets, each against the sources of its own system.
struct TuneRef {
    int64_t nt = 0;
    std::vector<int64_t> blk_first, blk_count, blk_src0, blk_src1;  // per system block
    int64_t *tgt = nullptr;      // device [nt]
    double *ref = nullptr;       // device, block b at 3 * blk_first[b]: [3][blk_count[b]]
    double *err = nullptr;       // device [nt]
    double *x64 = nullptr, *m64 = nullptr;  // FP64 copies of FP32 inputs
    TreeWorkspace *ws = nullptr;  // scratch of the direct sums
    ~TuneRef() {
        if (tgt) cudaFree(tgt);
        if (ref) cudaFree(ref);
        if (err) cudaFree(err);
        if (x64) cudaFree(x64);
        if (m64) cudaFree(m64);
        if (ws) tree_workspace_destroy(ws);
    }
};

tree_status_t tune_reference(TuneRef &R, const TreeParams *base, int64_t nseg, const int64_t *offsets, const void *x,
                             const void *m, int64_t n, cudaStream_t s) {
    // up to 16 systems, evenly spaced, up to 512 targets in all, evenly spaced inside each system
    const int64_t ns = nseg > 1 ? nseg : 1;
    const int64_t nsys = ns < 16 ? ns : 16;
    const int64_t per = nseg > 1 ? 32 : 512;
    std::vector<int64_t> h;
    for (int64_t j = 0; j < nsys; ++j) {
        const int64_t b = j * ns / nsys;
        const int64_t a0 = nseg > 1 ? offsets[b] : 0, a1 = nseg > 1 ? offsets[b + 1] : n;
        const int64_t cnt = a1 - a0 < per ? a1 - a0 : per;
        R.blk_first.push_back((int64_t)h.size());
        R.blk_count.push_back(cnt);
        R.blk_src0.push_back(a0);
        R.blk_src1.push_back(a1);
        for (int64_t k = 0; k < cnt; ++k) h.push_back(a0 + k * (a1 - a0) / cnt);
    }
    R.nt = (int64_t)h.size();
    TreeParams p = *base;
    p.node_cap = 0;
    tree_status_t st = tree_workspace_create(1, &p, &R.ws);
    if (st != TREE_OK) return st;
    if (!dalloc(&R.tgt, (size_t)R.nt) || !dalloc(&R.ref, 3 * (size_t)R.nt) || !dalloc(&R.err, (size_t)R.nt))
        return TREE_ERR_ALLOC;
    TRY_CUDA(cudaMemcpyAsync(R.tgt, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const void *xr = x, *mr = m;
    if (base->precision == TREE_F32) {
        if (!dalloc(&R.x64, 3 * (size_t)n) || !dalloc(&R.m64, (size_t)n)) return TREE_ERR_ALLOC;
        TRY_CUDA(launch_widen(R.ws, (const float *)x, 3 * n, R.x64, s));
        TRY_CUDA(launch_widen(R.ws, (const float *)m, n, R.m64, s));
        xr = R.x64;
        mr = R.m64;
    }
    for (size_t b = 0; b < R.blk_first.size(); ++b)
        TRY_CUDA(launch_direct_range(R.ws, xr, mr, n, R.blk_src0[b], R.blk_src1[b], TREE_F64, base->G, base->eps,
                                     R.tgt + R.blk_first[b], R.blk_count[b], R.ref + 3 * R.blk_first[b], nullptr, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    return TREE_OK;
}

// Median relative error of the accelerations a ([3][n], base precision) over the sample.
tree_status_t tune_error(TuneRef &R, const void *a, int64_t n, int dtype, cudaStream_t s, double *med) {
    for (size_t b = 0; b < R.blk_first.size(); ++b)
        TRY_CUDA(launch_rel_err(R.ws, a, n, dtype, R.tgt + R.blk_first[b], R.ref + 3 * R.blk_first[b],
                                R.blk_count[b], R.err + R.blk_first[b], s));
    std::vector<double> e((size_t)R.nt);
    TRY_CUDA(cudaMemcpyAsync(e.data(), R.err, e.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    if (e.empty()) { *med = 0.0; return TREE_OK; }
    // lower median: deterministic and a member of the sample
    const size_t k = (e.size() - 1) / 2;
    std::nth_element(e.begin(), e.begin() + k, e.end());
    *med = e[k];
    return TREE_OK;
}
}  // namespace

tree_status_t tree_autotune(const TreeParams *base, int64_t nseg, const int64_t *offsets, const void *x,
                            const void *m, int64_t n, int32_t reps, double max_err, TreeParams *best, double *table,
                            int32_t *ncand, void *stream) {
    if (!base || !best || !x || !m || n <= 0 || reps < 1 || isnan(max_err)) return TREE_ERR_ARG;
    if (table && !ncand) return TREE_ERR_ARG;
    if (nseg > 1) {
        if (!offsets || offsets[0] != 0 || offsets[nseg] != n) return TREE_ERR_ARG;
        for (int64_t b = 0; b < nseg; ++b)
            if (offsets[b + 1] <= offsets[b]) return TREE_ERR_ARG;
    }
    tree_status_t st = check_params(base);
    if (st != TREE_OK) return st;
    cudaStream_t s = as_stream(stream);
    const int lcaps[3] = {4, 8, 16}, gss[3] = {16, 32, 64}, stacks[2] = {512, 1024};
    const int32_t rows = table ? *ncand : 0;
    int32_t used = 0;
    double best_ms = INFINITY;
    TuneRef R;
    st = tune_reference(R, base, nseg, offsets, x, m, n, s);
    if (st != TREE_OK) return st;
    void *a = nullptr;
    const size_t rs = base->precision == TREE_F64 ? 8 : 4;
    TRY_CUDA(cudaMalloc(&a, 3 * (size_t)n * rs));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(a);
        return TREE_ERR_CUDA;
    }
    tree_status_t ret = TREE_OK;
    for (int li = 0; li < 3 && ret == TREE_OK; ++li) {
        TreeParams p = *base;
        p.leaf_cap = lcaps[li];
        p.node_cap = 0;
        TreeWorkspace *ws = nullptr;
        st = tree_workspace_create(n, &p, &ws);
        if (st != TREE_OK) { ret = st; break; }
        if (nseg > 1) st = tree_set_segments(ws, nseg, offsets);
        for (int gi = 0; gi < 3 && st == TREE_OK; ++gi) {
            for (int si = 0; si < 2 && st == TREE_OK; ++si) {
                p.group_size = gss[gi];
                p.stack_depth = stacks[si];
                st = tree_set_params(ws, &p);
                if (st != TREE_OK) break;
                double ms = INFINITY, err = INFINITY;
                int32_t dev = 0;
                // one untimed evaluation, then reps timed ones
                for (int r = 0; r <= reps && st == TREE_OK; ++r) {
                    if (r == 1) cudaEventRecord(e0, s);
                    st = tree_build(ws, x, n, p.precision, s);
                    if (st == TREE_OK) st = tree_moments(ws, x, m, s);
                    if (st == TREE_OK) st = tree_forces(ws, a, nullptr, 0, s);
                }
                if (st != TREE_OK) break;
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) { st = TREE_ERR_CUDA; break; }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                st = tree_get_status(ws, &dev, 1);
                if (st == TREE_ERR_DEVICE) st = TREE_OK;  // the status bits decide below
                if (st != TREE_OK) break;
                st = tune_error(R, a, n, p.precision, s, &err);
                if (st != TREE_OK) break;
                // a candidate that overflowed its stack, or whose forces miss the error bound, does not count
                const bool ok = dev == 0 && (!(max_err > 0.0) || err <= max_err);
                if (ok) ms = (double)t / reps;
                if (table && used < rows) {
                    table[5 * used + 0] = p.leaf_cap;
                    table[5 * used + 1] = p.group_size;
                    table[5 * used + 2] = p.stack_depth;
                    table[5 * used + 3] = ok ? ms : INFINITY;
                    table[5 * used + 4] = dev == 0 ? err : INFINITY;
                }
                ++used;
                if (ms < best_ms) {
                    best_ms = ms;
                    *best = p;
                }
            }
        }
        if (st != TREE_OK) ret = st;
        tree_workspace_destroy(ws);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    if (ncand) *ncand = used;
    if (ret == TREE_OK && !isfinite(best_ms)) ret = TREE_ERR_DEVICE;
    return ret;
}

tree_status_t tree_export_boxes(TreeWorkspace *ws, double *lo, int32_t *k) {
    if (!ws || (!lo && !k)) return TREE_ERR_ARG;
    if (!ws->built || ws->n == 0) return TREE_ERR_STATE;
    TRY_CUDA(cudaDeviceSynchronize());
    std::vector<DevBox> b((size_t)ws->nseg);
    TRY_CUDA(cudaMemcpy(b.data(), ws->box, b.size() * sizeof(DevBox), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < b.size(); ++i) {
        if (lo) for (int d = 0; d < 3; ++d) lo[3 * i + d] = b[i].lo[d];
        if (k) k[i] = b[i].k;
    }
    return TREE_OK;
}

tree_status_t tree_direct_forces(TreeWorkspace *ws, const void *x, const void *m, int64_t n, int32_t dtype,
                                 const int64_t *targets, int64_t nt, double *a_out, double *phi_out, void *stream) {
    if (!ws || n < 0 || nt < 0) return TREE_ERR_ARG;
    if (dtype != TREE_F32 && dtype != TREE_F64) return TREE_ERR_ARG;
    if (nt == 0) return TREE_OK;
    if (!x || !m || !targets || !a_out || n < 1) return TREE_ERR_ARG;
    PhaseScope ph(ws, TREE_PHASE_DIRECT, as_stream(stream));
    TRY_CUDA(launch_direct(ws, x, m, n, dtype, targets, nt, a_out, phi_out, as_stream(stream)));
    return TREE_OK;
}

tree_status_t tree_timing_enable(TreeWorkspace *ws, int32_t enable) {
    if (!ws) return TREE_ERR_ARG;
    ws->timing = enable != 0;
    if (ws->timing) {
        ws->ev_used = 0;
        ws->timed_launches = 0;
    }
    return TREE_OK;
}

tree_status_t tree_timing_read(TreeWorkspace *ws, double *ms, int64_t *calls, int64_t *launches) {
    if (!ws || !ms) return TREE_ERR_ARG;
    TRY_CUDA(cudaDeviceSynchronize());
    for (int i = 0; i < TREE_NPHASES; ++i) {
        ms[i] = 0.0;
        if (calls) calls[i] = 0;
    }
    for (size_t k = 0; k < ws->ev_used; ++k) {
        float t = 0.f;
        TRY_CUDA(cudaEventElapsedTime(&t, ws->ev[2 * k], ws->ev[2 * k + 1]));
        const int ph = ws->ev_phase[k];
        ms[ph] += t;
        if (calls) calls[ph] += 1;
    }
    if (launches) *launches = ws->timed_launches;
    return TREE_OK;
}

tree_status_t tree_set_waits(TreeWorkspace *ws, int64_t wait_cycles, int32_t withhold_pass, int64_t withhold_tile) {
    if (!ws || wait_cycles < 0) return TREE_ERR_ARG;
    if ((withhold_pass < 0) != (withhold_tile < 0)) return TREE_ERR_ARG;
    if (withhold_pass >= kSortPasses + kSegPassesMax || withhold_tile > 0xffffffffLL) return TREE_ERR_ARG;
    TRY_CUDA(cudaDeviceSynchronize());
    DevCtl ctl;
    TRY_CUDA(cudaMemcpy(&ctl, ws->dctl, sizeof(ctl), cudaMemcpyDeviceToHost));
    if (wait_cycles > 0) ctl.wait_cycles = wait_cycles;
    ctl.withhold = withhold_pass < 0 ? -1 : (((long long)withhold_pass << 32) | (long long)withhold_tile);
    TRY_CUDA(cudaMemcpy(ws->dctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice));
    return TREE_OK;
}

tree_status_t tree_get_status(TreeWorkspace *ws, int32_t *status, int32_t clear) {
    if (!ws || !status) return TREE_ERR_ARG;
    TRY_CUDA(cudaDeviceSynchronize());
    TRY_CUDA(cudaMemcpy(status, ws->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (clear) TRY_CUDA(cudaMemset(ws->dstatus, 0, sizeof(int32_t)));
    return *status ? TREE_ERR_DEVICE : TREE_OK;
}

tree_status_t tree_get_info(TreeWorkspace *ws, TreeInfo *info) {
    if (!ws || !info) return TREE_ERR_ARG;
    memset(info, 0, sizeof(*info));
    TRY_CUDA(cudaDeviceSynchronize());
    info->n = ws->n;
    info->n_groups = 0;
    info->list_pc = ws->list_groups >= 0 ? ws->list_pc : 0;
    info->list_pp = ws->list_groups >= 0 ? ws->list_pp : 0;
    info->launches = ws->launches;
    info->n_segments = ws->nseg;
    if (!ws->built || ws->n == 0) return TREE_OK;
    uint32_t ctr[kCtrCount];
    DevBox box;
    TRY_CUDA(cudaMemcpy(ctr, ws->ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
    TRY_CUDA(cudaMemcpy(&box, ws->box, sizeof(box), cudaMemcpyDeviceToHost));
    for (int l = 0; l <= kLevels; ++l) info->level_offset[l] = ctr[kCtrLevelStart + l];
    info->n_nodes = info->level_offset[kLevels];
    info->depth = 0;
    for (int l = 0; l < kLevels; ++l)
        if (info->level_offset[l + 1] > info->level_offset[l]) info->depth = l;
    info->n_groups = ctr[kCtrGroups];
    info->box_k = box.k;
    for (int d = 0; d < 3; ++d) info->box_lo[d] = box.lo[d];
    if (ws->has_moments) {
        TRY_CUDA(launch_gstat_reduce(ws, info->n_groups, 0));
        unsigned long long st[kStatCount];
        TRY_CUDA(cudaMemcpy(st, ws->stats, sizeof(st), cudaMemcpyDeviceToHost));
        info->pp_pairs = (int64_t)st[kStatPP];
        info->pc_pairs = (int64_t)st[kStatPC];
        info->max_stack = (int64_t)st[kStatMaxStack];
    }
    info->launches = ws->launches;  // including the statistics reduction above
    return TREE_OK;
}

tree_status_t tree_export_tree(TreeWorkspace *ws, uint64_t *keys, uint32_t *perm, int32_t *level, uint32_t *corner,
                               uint32_t *first, uint32_t *count, int32_t *child, int32_t *nchild, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (!ws->built) return TREE_ERR_STATE;
    TreeInfo info;
    tree_status_t st = tree_get_info(ws, &info);
    if (st != TREE_OK) return st;
    cudaStream_t s = as_stream(stream);
    const size_t n = (size_t)ws->n;
    if (keys && n) TRY_CUDA(cudaMemcpyAsync(keys, ws->key, n * 8, cudaMemcpyDeviceToDevice, s));
    if (perm && n) TRY_CUDA(cudaMemcpyAsync(perm, ws->idx, n * 4, cudaMemcpyDeviceToDevice, s));
    TRY_CUDA(launch_export_tree(ws, info.n_nodes, level, corner, first, count, child, nchild, s));
    return TREE_OK;
}

tree_status_t tree_export_moments(TreeWorkspace *ws, double *M, double *R, double *Q, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (!ws->has_moments) return TREE_ERR_STATE;
    TreeInfo info;
    tree_status_t st = tree_get_info(ws, &info);
    if (st != TREE_OK) return st;
    const size_t nn = (size_t)info.n_nodes, cap = (size_t)ws->node_cap;
    cudaStream_t s = as_stream(stream);
    if (nn == 0) return TREE_OK;
    if (M) TRY_CUDA(cudaMemcpyAsync(M, ws->mom64, nn * 8, cudaMemcpyDeviceToDevice, s));
    for (int d = 0; d < 3; ++d)
        if (R) TRY_CUDA(cudaMemcpyAsync(R + d * nn, ws->mom64 + (1 + d) * cap, nn * 8, cudaMemcpyDeviceToDevice, s));
    for (int c = 0; c < 6; ++c)
        if (Q) TRY_CUDA(cudaMemcpyAsync(Q + c * nn, ws->mom64 + (4 + c) * cap, nn * 8, cudaMemcpyDeviceToDevice, s));
    return TREE_OK;
}

tree_status_t tree_export_group_stats(TreeWorkspace *ws, uint32_t *out, void *stream) {
    if (!ws || !out) return TREE_ERR_ARG;
    if (!ws->has_moments) return TREE_ERR_STATE;
    uint32_t ng = 0;
    TRY_CUDA(cudaDeviceSynchronize());
    TRY_CUDA(cudaMemcpy(&ng, ws->ctr + kCtrGroups, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    TRY_CUDA(launch_export_gstat(ws, ng, out, as_stream(stream)));
    return TREE_OK;
}

tree_status_t tree_export_groups(TreeWorkspace *ws, uint32_t *gfirst, void *stream) {
    if (!ws || !gfirst) return TREE_ERR_ARG;
    if (!ws->built) return TREE_ERR_STATE;
    if (ws->n == 0) return TREE_OK;
    uint32_t ng = 0;
    TRY_CUDA(cudaDeviceSynchronize());
    TRY_CUDA(cudaMemcpy(&ng, ws->ctr + kCtrGroups, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    TRY_CUDA(cudaMemcpyAsync(gfirst, ws->gfirst, ((size_t)ng + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                             as_stream(stream)));
    return TREE_OK;
}

tree_status_t tree_export_lists_groups(TreeWorkspace *ws, int64_t nsel, const int64_t *gsel, int64_t *pc_off,
                                       int32_t *pc_list, int64_t *pp_off, int32_t *pp_list, void *stream) {
    if (!ws || nsel < 0 || (nsel > 0 && !gsel) || !pc_off || !pp_off) return TREE_ERR_ARG;
    if (ws->list_groups < 0) return TREE_ERR_STATE;
    const int64_t ng = ws->list_groups;
    for (int64_t k = 0; k < nsel; ++k)
        if (gsel[k] < 0 || gsel[k] >= ng) return TREE_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    // both offset tables, [2][ng + 1]
    std::vector<int64_t> off((size_t)(2 * (ng + 1)));
    TRY_CUDA(cudaMemcpyAsync(off.data(), ws->list_cnt, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t *pco = off.data(), *ppo = off.data() + ng + 1;
    pc_off[0] = 0;
    pp_off[0] = 0;
    for (int64_t k = 0; k < nsel; ++k) {
        const int64_t g = gsel[k];
        pc_off[k + 1] = pc_off[k] + (pco[g + 1] - pco[g]);
        pp_off[k + 1] = pp_off[k] + (ppo[g + 1] - ppo[g]);
    }
    for (int64_t k = 0; k < nsel; ++k) {
        const int64_t g = gsel[k];
        const int64_t npc = pco[g + 1] - pco[g], npp = ppo[g + 1] - ppo[g];
        if (pc_list && npc > 0)
            TRY_CUDA(cudaMemcpyAsync(pc_list + pc_off[k], ws->pc_list + pco[g], (size_t)npc * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, s));
        if (pp_list && npp > 0)
            TRY_CUDA(cudaMemcpyAsync(pp_list + pp_off[k], ws->pp_list + ppo[g], (size_t)npp * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, s));
    }
    TRY_CUDA(cudaStreamSynchronize(s));
    return TREE_OK;
}

tree_status_t tree_export_lists(TreeWorkspace *ws, int64_t *pc_off, int32_t *pc_list, int64_t *pp_off,
                                int32_t *pp_list, void *stream) {
    if (!ws) return TREE_ERR_ARG;
    if (ws->list_groups < 0) return TREE_ERR_STATE;
    cudaStream_t s = as_stream(stream);
    const size_t ng = (size_t)ws->list_groups;
    if (pc_off) TRY_CUDA(cudaMemcpyAsync(pc_off, ws->list_cnt, (ng + 1) * 8, cudaMemcpyDeviceToDevice, s));
    if (pp_off) TRY_CUDA(cudaMemcpyAsync(pp_off, ws->list_cnt + ng + 1, (ng + 1) * 8, cudaMemcpyDeviceToDevice, s));
    if (pc_list && ws->list_pc)
        TRY_CUDA(cudaMemcpyAsync(pc_list, ws->pc_list, (size_t)ws->list_pc * 4, cudaMemcpyDeviceToDevice, s));
    if (pp_list && ws->list_pp)
        TRY_CUDA(cudaMemcpyAsync(pp_list, ws->pp_list, (size_t)ws->list_pp * 4, cudaMemcpyDeviceToDevice, s));
    return TREE_OK;
}

}  // extern "C"
