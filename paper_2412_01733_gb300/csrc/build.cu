// build.cu -- canonical tree construction on the GPU (Sec. 2 octree):
//   box reduction (FP64), 63-bit Morton keys with the radix histograms of all
//   eight sort passes fused in, stable onesweep LSD radix sort of
//   (key, index), breadth-first octree built level by level with a
//   decoupled look-back scan, and the gather of positions/masses into key
//   order.
#include <float.h>
#include <math.h>

#include "common.cuh"

namespace treegb {

// ============================================================== box reduction
// Per-block FP64 min/max of the three coordinates; non-finite values set
// TREE_DEV_NONFINITE and are left out of the box.
template <typename Real>
__global__ void __launch_bounds__(256) k_box_partial(const Real *__restrict__ x, int64_t n,
                                                     double *__restrict__ part, int32_t *dstatus) {
    // min/max are exact in the input precision; widen to FP64 once per warp
    __shared__ double sh[6][8];
    const Real big = sizeof(Real) == 4 ? (Real)FLT_MAX : (Real)DBL_MAX;
    Real mn[3] = {big, big, big}, mx[3] = {-big, -big, -big};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const Real v = x[d * n + i];
            if (!isfinite(v)) { bad = true; continue; }
            mn[d] = min(mn[d], v);
            mx[d] = max(mx[d], v);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(dstatus, TREE_DEV_NONFINITE);
    double dmn[3], dmx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        dmn[d] = mn[d] == big ? DBL_MAX : (double)mn[d];
        dmx[d] = mx[d] == -big ? -DBL_MAX : (double)mx[d];
        for (int o = 16; o > 0; o >>= 1) {
            dmn[d] = fmin(dmn[d], __shfl_xor_sync(0xffffffffu, dmn[d], o));
            dmx[d] = fmax(dmx[d], __shfl_xor_sync(0xffffffffu, dmx[d], o));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) { sh[d][warp] = dmn[d]; sh[3 + d][warp] = dmx[d]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int c = threadIdx.x;
        double r = sh[c][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = c < 3 ? fmin(r, sh[c][w]) : fmax(r, sh[c][w]);
        part[blockIdx.x * 8 + c] = r;
    }
}

// lo = min, ext = max_d (hi_d - lo_d) in FP64, L = 2^k the smallest power of
// two strictly greater than ext (k = 0 when ext = 0): with ext = f 2^e,
// f in [0.5, 1), that power is 2^e.
__device__ void box_from_minmax(double (&lo)[3], double (&hi)[3], DevBox *box) {
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (!(lo[d] <= hi[d])) { lo[d] = 0.0; hi[d] = 0.0; }  // no finite value on this axis
        double e = __dsub_rn(hi[d], lo[d]);
        if (e > ext) ext = e;
    }
    int k = 0;
    if (ext > 0.0) frexp(ext, &k);
    for (int d = 0; d < 3; ++d) box->lo[d] = lo[d];
    box->k = k;
    box->r5fit = 0;  // decided after the moments
    box->scale = ldexp(1.0, kBits - k);
    box->unit = ldexp(1.0, k - kBits);
}

// One block: each thread folds a strided share of the partials, then the
// block folds the threads (min and max are exact in any order).
__global__ void __launch_bounds__(256) k_box_final(const double *__restrict__ part, int nblocks, DevBox *box) {
    __shared__ double sh[6][8];
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], part[b * 8 + d]);
            hi[d] = fmax(hi[d], part[b * 8 + 3 + d]);
        }
    }
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) { sh[d][warp] = lo[d]; sh[3 + d][warp] = hi[d]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            for (int d = 0; d < 3; ++d) {
                lo[d] = fmin(lo[d], sh[d][w]);
                hi[d] = fmax(hi[d], sh[3 + d][w]);
            }
        box_from_minmax(lo, hi, box);
    }
}

cudaError_t launch_box_final(TreeWorkspace *ws, int nblocks, cudaStream_t s) {
    k_box_final<<<1, 256, 0, s>>>(ws->part, nblocks, ws->box);
    ws->launches += 1;
    return cudaGetLastError();
}

// Segmented box: one block per chunk {begin, end, segment} (chunks never
// straddle segments), optionally fused with the kick + drift of Eqs. 2-3
// (the same arithmetic as the unsegmented kick-drift pass); then one thread
// per segment folds its chunks.
template <typename Real, bool KICK>
__global__ void __launch_bounds__(256) k_box_chunks(Real *__restrict__ x, Real *__restrict__ v,
                                                    const Real *__restrict__ a, const Real *__restrict__ m,
                                                    typename Vec4<Real>::T *__restrict__ xm, Real half_tau, Real tau,
                                                    int64_t n, const uint4 *__restrict__ chunks, int64_t nchunks,
                                                    double *__restrict__ part, int32_t *dstatus) {
    __shared__ double sh[6][8];
    const Real big = sizeof(Real) == 4 ? (Real)FLT_MAX : (Real)DBL_MAX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const uint4 ch = chunks[c];
        Real mn[3] = {big, big, big}, mx[3] = {-big, -big, -big};
        bool bad = false;
        for (int64_t i = ch.x + threadIdx.x; i < (int64_t)ch.y; i += blockDim.x) {
            Real xn[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Real xx;
                if (KICK) {
                    const Real vv = fma(half_tau, a[d * n + i], v[d * n + i]);
                    xx = fma(tau, vv, x[d * n + i]);
                    v[d * n + i] = vv;
                    x[d * n + i] = xx;
                } else {
                    xx = x[d * n + i];
                }
                xn[d] = xx;
                if (!isfinite(xx)) { bad = true; continue; }
                mn[d] = min(mn[d], xx);
                mx[d] = max(mx[d], xx);
            }
            if (KICK) {
                typename Vec4<Real>::T p;
                p.x = xn[0]; p.y = xn[1]; p.z = xn[2]; p.w = m[i];
                xm[i] = p;
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(dstatus, TREE_DEV_NONFINITE);
        double dmn[3], dmx[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            dmn[d] = mn[d] == big ? DBL_MAX : (double)mn[d];
            dmx[d] = mx[d] == -big ? -DBL_MAX : (double)mx[d];
            for (int o = 16; o > 0; o >>= 1) {
                dmn[d] = fmin(dmn[d], __shfl_xor_sync(0xffffffffu, dmn[d], o));
                dmx[d] = fmax(dmx[d], __shfl_xor_sync(0xffffffffu, dmx[d], o));
            }
        }
        if (lane == 0) {
            for (int d = 0; d < 3; ++d) { sh[d][warp] = dmn[d]; sh[3 + d][warp] = dmx[d]; }
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            const int q = threadIdx.x;
            double r = sh[q][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = q < 3 ? fmin(r, sh[q][w]) : fmax(r, sh[q][w]);
            part[c * 8 + q] = r;
        }
        __syncthreads();
    }
}

__global__ void k_box_seg_final(const double *__restrict__ part, const uint32_t *__restrict__ bfirst, int64_t nseg,
                                DevBox *box) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nseg) return;
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (uint32_t c = bfirst[b]; c < bfirst[b + 1]; ++c) {
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], part[c * 8 + d]);
            hi[d] = fmax(hi[d], part[c * 8 + 3 + d]);
        }
    }
    box_from_minmax(lo, hi, box + b);
}

template <typename Real>
static cudaError_t box_seg_impl(TreeWorkspace *ws, Real *x, Real *v, const Real *a, const Real *m, double tau,
                                int64_t n, bool kick, cudaStream_t s) {
    using V4 = typename Vec4<Real>::T;
    const int nb = grid_for(ws->seg_nbchunk * 256, 256, 152 * 16);
    if (kick)
        k_box_chunks<Real, true><<<nb, 256, 0, s>>>(x, v, a, m, (V4 *)ws->xm, (Real)(0.5 * tau), (Real)tau, n,
                                                   ws->seg_bchunk, ws->seg_nbchunk, ws->seg_part, ws->dstatus);
    else
        k_box_chunks<Real, false><<<nb, 256, 0, s>>>(x, nullptr, nullptr, nullptr, nullptr, Real(0), Real(0), n,
                                                    ws->seg_bchunk, ws->seg_nbchunk, ws->seg_part, ws->dstatus);
    k_box_seg_final<<<grid_for(ws->nseg, 128, 1 << 20), 128, 0, s>>>(ws->seg_part, ws->seg_bfirst, ws->nseg,
                                                                     ws->box);
    ws->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_box_segments(TreeWorkspace *ws, void *x, void *v, const void *a, const void *m, double tau,
                                int64_t n, bool kick, cudaStream_t s) {
    if (ws->p.precision == TREE_F64)
        return box_seg_impl<double>(ws, (double *)x, (double *)v, (const double *)a, (const double *)m, tau, n,
                                    kick, s);
    return box_seg_impl<float>(ws, (float *)x, (float *)v, (const float *)a, (const float *)m, tau, n, kick, s);
}

template <typename Real>
static cudaError_t box_impl(TreeWorkspace *ws, const Real *x, int64_t n, cudaStream_t s) {
    const int nb = wave_grid(k_box_partial<Real>, n, 256, kMaxBlocksReduce);
    k_box_partial<Real><<<nb, 256, 0, s>>>(x, n, ws->part, ws->dstatus);
    ws->launches += 1;
    return launch_box_final(ws, nb, s);
}

cudaError_t launch_box(TreeWorkspace *ws, const void *x, int64_t n, cudaStream_t s) {
    if (ws->nseg > 1)
        return launch_box_segments(ws, const_cast<void *>(x), nullptr, nullptr, nullptr, 0.0, n, false, s);
    if (ws->p.precision == TREE_F64) return box_impl(ws, (const double *)x, n, s);
    return box_impl(ws, (const float *)x, n, s);
}

// ============================================================== keys + histograms
// q_d = min(2^21-1, floor(fl(x_d - lo_d) * 2^(21-k))), negatives to 0: the
// FP64 subtraction is the only rounding (the scaling is by a power of two).
// The key interleaves q_x, q_y, q_z (x highest).  The same pass counts the
// eight 8-bit digits of every key for the radix sort (warp-aggregated
// shared-memory atomics).
// SEG: every particle is quantised in the box of its own segment.

// The floor and both clamps are one saturating round-down conversion
// (cvt.rmi.u32.f64 clamps out-of-range values, negatives to 0) and an integer
// min; a NaN lands in some in-range cell (the box pass has already raised
// TREE_DEV_NONFINITE for it).
__device__ __forceinline__ uint32_t quantize(double x, double lo, double sc) {
    return min(__double2uint_rd(__dmul_rn(__dsub_rn(x, lo), sc)), (1u << kBits) - 1u);
}
// FP32 coordinates: x sc and lo sc are exact in FP64 (a float, or the box
// corner, times a power of two stays far inside the FP64 range), so one fused
// multiply-add, x sc - lo sc, rounds (x - lo) sc exactly as the FP64
// subtraction followed by the exact scaling does: the same q_d with a third
// of the FP64 instructions (the FP64 pipe runs at 1/64 of the FP32 rate here).
__device__ __forceinline__ uint32_t quantize(float x, double lo, double sc) {
    return min(__double2uint_rd(fma((double)x, sc, -(lo * sc))), (1u << kBits) - 1u);
}

template <typename Real, bool SEG>
__global__ void __launch_bounds__(256) k_keys(const Real *__restrict__ x, int64_t n,
                                              const DevBox *__restrict__ box, const int64_t *__restrict__ seg_off,
                                              int64_t nseg, uint64_t *__restrict__ key,
                                              uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[kSortPasses][kRadix];
    for (int i = threadIdx.x; i < kSortPasses * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const double lo0 = box->lo[0], lo1 = box->lo[1], lo2 = box->lo[2], scale = box->scale;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < n;
        uint64_t k = 0;
        if (valid) {
            double lo[3] = {lo0, lo1, lo2};
            double sc = scale;
            if (SEG) {
                const DevBox *bx = box + seg_find(seg_off, nseg, i);
                lo[0] = bx->lo[0]; lo[1] = bx->lo[1]; lo[2] = bx->lo[2];
                sc = bx->scale;
            }
            uint32_t q[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) q[d] = quantize(x[d * n + i], lo[d], sc);
            k = morton3(q[0], q[1], q[2]);
            key[i] = k;
        }
        // The low five digits (the finest 13 levels) of 32 keys rarely repeat,
        // so each lane counts its own with a shared atomic; the top three
        // digits are aggregated over the lanes that share them first.
        const uint32_t vm = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int p = 0; p < kSortPasses; ++p) {
            const uint32_t dg = (uint32_t)((k >> (8 * p)) & 0xffu);
            if (p < kSortPasses - 3) {
                if (valid) atomicAdd(&sh[p][dg], 1u);
            } else {
                const uint32_t peers = match_digit8(dg, valid ? vm : ~vm);
                if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&sh[p][dg], (uint32_t)__popc(peers));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSortPasses * kRadix; i += blockDim.x) {
        uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

// Exclusive scan of each pass's 256 digit counts -> hist[2048 + p*256 + d].
__global__ void __launch_bounds__(256) k_hist_scan(uint32_t *hist) {
    __shared__ uint32_t wt[32];
    const int p = blockIdx.x, d = threadIdx.x;
    uint32_t c = hist[p * kRadix + d];
    uint32_t e = block_exclusive_scan(c, wt, nullptr);
    hist[kSortPasses * kRadix + p * kRadix + d] = e;
}

// ============================================================== onesweep pass
// One block sorts one tile of kSortTile keys by the 8-bit digit at `shift`:
// warp-level ranking with digit-matching ballots (stable: a warp owns a contiguous
// segment and walks it item by item, lanes in order), per-digit decoupled
// look-back across tiles for the global position, then a scatter through
// shared memory so that global writes are runs of equal digits.
struct SortSmem {
    uint64_t keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t whist[kSortThreads / 32][kRadix];
    uint32_t start[kRadix];
    uint32_t gbase[kRadix];
    uint32_t wt[32];
    uint32_t tile;
};

// MODE: kPassFirst (values = input positions), kPassKey, kPassSeg (digit of
// the segment index of the value's input position: segments are the most
// significant sort digits, so each ends up in its own contiguous range).
enum SortPass { kPassFirst = 0, kPassKey = 1, kPassSeg = 2 };

template <int MODE>
__device__ __forceinline__ uint32_t sort_digit(uint64_t k, uint32_t v, int shift, const int64_t *seg_off,
                                               int64_t nseg) {
    if (MODE == kPassSeg) return (seg_find(seg_off, nseg, v) >> shift) & 0xffu;
    return (uint32_t)((k >> shift) & 0xffu);
}

template <int MODE>
__global__ void __launch_bounds__(kSortThreads, MODE == kPassSeg ? 2 : 3) k_onesweep(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t n, int shift, const uint32_t *__restrict__ digit_off,
    uint32_t *status, uint32_t *ticket, int32_t *dstatus, const int64_t *__restrict__ seg_off, int64_t nseg,
    uint32_t *ctr, uint32_t pass, const DevCtl *__restrict__ ctl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t stage = kStageSort0 + pass;
    if (aborted(ctr, stage)) return;  // an earlier pass gave up a wait: its output is not a permutation
    for (int i = tid; i < (kSortThreads / 32) * kRadix; i += kSortThreads) (&S.whist[0][0])[i] = 0;
    if (tid == 0) S.tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = S.tile;
    const int64_t base = (int64_t)tile * kSortTile;

    // the digit of item i (0x100 past the end): kept for segment passes (a
    // binary search), recomputed from the key otherwise (fewer live registers)
    constexpr int kDg = MODE == kPassSeg ? kSortItems : 1;
    uint64_t k[kSortItems];
    uint32_t v[kSortItems], dgs[kDg], rk[kSortItems];
    const int64_t wbase = base + warp * (kSortItems * 32);
    auto digit = [&](int i) -> uint32_t {
        if (MODE == kPassSeg) return dgs[i % kDg];
        return wbase + i * 32 + lane < n ? (uint32_t)((k[i] >> shift) & 0xffu) : 0x100u;
    };
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t pos = wbase + i * 32 + lane;
        if (pos < n) {
            k[i] = kin[pos];
            v[i] = MODE == kPassFirst ? (uint32_t)pos : vin[pos];
            if (MODE == kPassSeg) dgs[i % kDg] = sort_digit<MODE>(k[i], v[i], shift, seg_off, nseg);
        } else {
            k[i] = 0; v[i] = 0;
            if (MODE == kPassSeg) dgs[i % kDg] = 0x100u;
        }
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t d = digit(i);
        const bool ok = d < 0x100u;
        const uint32_t vm = __ballot_sync(0xffffffffu, ok);
        const uint32_t peers = match_digit8(d, ok ? vm : ~vm);
        uint32_t cnt = 0;
        if (d < 0x100u) cnt = S.whist[warp][d];
        __syncwarp();
        const uint32_t pr = __popc(peers & lt);
        if (d < 0x100u && pr == 0) S.whist[warp][d] = cnt + __popc(peers);
        __syncwarp();
        rk[i] = cnt + pr;
    }
    __syncthreads();
    // thread t owns digit t: exclusive offsets over warps, tile count
    uint32_t tcount = 0;
    {
        const int d = tid;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            uint32_t c = S.whist[w][d];
            S.whist[w][d] = tcount;
            tcount += c;
        }
    }
    // per-digit look-back: status[tile * 256 + d]
    {
        const int d = tid;
        uint32_t *st = status + d;  // word of digit d in tile t is st[t * 256]
        uint32_t excl = 0;
        const WaitCtx wc{dstatus, ctr, stage, ctl->wait_cycles};
        // test injection: this tile keeps its words unpublished, so the tiles
        // after it run into their wait limit
        const bool publish = ctl->withhold != (((long long)pass << 32) | (long long)tile);
        if (tile == 0) {
            if (publish) st_publish(st, kFlagInc | tcount);
        } else {
            if (publish) st_publish(st + (size_t)tile * kRadix, kFlagAgg | tcount);
            excl = lookback_walk(st, kRadix, (int64_t)tile - 1, wc);
            if (publish) st_publish(st + (size_t)tile * kRadix, kFlagInc | ((excl + tcount) & kValMask));
        }
        S.gbase[d] = digit_off[d] + excl;
    }
    uint32_t st0 = block_exclusive_scan(tcount, S.wt, nullptr);
    S.start[tid] = st0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t d = digit(i);
        if (d < 0x100u) {
            const uint32_t p = S.start[d] + S.whist[warp][d] + rk[i];
            S.keys[p] = k[i];
            S.vals[p] = v[i];
        }
    }
    __syncthreads();
    const int64_t rem = n - base;
    const int valid = rem < kSortTile ? (int)rem : kSortTile;
    for (int j = tid; j < valid; j += kSortThreads) {
        const uint64_t kk = S.keys[j];
        const uint32_t vv = S.vals[j];
        const uint32_t d = sort_digit<MODE>(kk, vv, shift, seg_off, nseg);
        const uint32_t o = S.gbase[d] + (uint32_t)j - S.start[d];
        kout[o] = kk;
        vout[o] = vv;
    }
}

// The passes alternate between the two key/value buffers and must end in
// ws->key / ws->idx: with an odd number of passes the keys start in key_alt.
static bool sort_starts_alt(const TreeWorkspace *ws) { return ((kSortPasses + ws->seg_passes) & 1) != 0; }

template <typename Real>
static cudaError_t keys_impl(TreeWorkspace *ws, const Real *x, int64_t n, cudaStream_t s) {
    uint64_t *dst = sort_starts_alt(ws) ? ws->key_alt : ws->key;
    if (ws->nseg > 1)
        k_keys<Real, true><<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(
            x, n, ws->box, ws->seg_off, ws->nseg, dst, ws->hist);
    else
        k_keys<Real, false><<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(
            x, n, ws->box, nullptr, 1, dst, ws->hist);
    k_hist_scan<<<kSortPasses, kRadix, 0, s>>>(ws->hist);
    ws->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_keys(TreeWorkspace *ws, const void *x, int64_t n, cudaStream_t s) {
    if (ws->p.precision == TREE_F64) return keys_impl(ws, (const double *)x, n, s);
    return keys_impl(ws, (const float *)x, n, s);
}

cudaError_t launch_sort(TreeWorkspace *ws, int64_t n, cudaStream_t s) {
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    const size_t smem = sizeof(SortSmem);
    static bool attr_done[64] = {};
    if (ws->device < 64 && !attr_done[ws->device]) {
        // the key passes fit three blocks per SM (registers and shared memory)
        // when the carveout gives shared memory all it can
        const void *fn[3] = {(const void *)k_onesweep<kPassFirst>, (const void *)k_onesweep<kPassKey>,
                             (const void *)k_onesweep<kPassSeg>};
        cudaError_t e = cudaSuccess;
        for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
            e = cudaFuncSetAttribute(fn[f], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(fn[f], cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
        }
        if (e != cudaSuccess) return e;
        attr_done[ws->device] = true;
    }
    const bool alt = sort_starts_alt(ws);
    uint64_t *kin = alt ? ws->key_alt : ws->key, *kout = alt ? ws->key : ws->key_alt;
    uint32_t *vin = alt ? ws->idx_alt : ws->idx, *vout = alt ? ws->idx : ws->idx_alt;
    const int npass = kSortPasses + ws->seg_passes;
    for (int p = 0; p < npass; ++p) {
        uint32_t *st = ws->sort_status + (size_t)p * ws->sort_tiles_max * kRadix;
        uint32_t *tk = ws->ctr + kCtrSortTicket + p;
        const unsigned g = (unsigned)tiles;
        const uint32_t pu = (uint32_t)p;
        if (p == 0) {
            k_onesweep<kPassFirst><<<g, kSortThreads, smem, s>>>(kin, vin, kout, vout, n, 0,
                                                                 ws->hist + kSortPasses * kRadix, st, tk,
                                                                 ws->dstatus, nullptr, 1, ws->ctr, pu, ws->dctl);
        } else if (p < kSortPasses) {
            k_onesweep<kPassKey><<<g, kSortThreads, smem, s>>>(kin, vin, kout, vout, n, 8 * p,
                                                               ws->hist + kSortPasses * kRadix + p * kRadix, st, tk,
                                                               ws->dstatus, nullptr, 1, ws->ctr, pu, ws->dctl);
        } else {
            const int q = p - kSortPasses;
            k_onesweep<kPassSeg><<<g, kSortThreads, smem, s>>>(kin, vin, kout, vout, n, 8 * q,
                                                               ws->seg_digit_off + q * kRadix, st, tk, ws->dstatus,
                                                               ws->seg_off, ws->nseg, ws->ctr, pu, ws->dctl);
        }
        uint64_t *tk_ = kin; kin = kout; kout = tk_;
        uint32_t *tv_ = vin; vin = vout; vout = tv_;
    }
    ws->launches += npass;
    // the sorted data is now in ws->key / ws->idx
    return cudaGetLastError();
}

// ============================================================== octree
// Level 0 holds one root per segment (segment b = node b, the sorted range
// [off[b], off[b+1])), or the single root of all n particles.
__global__ void k_tree_init(uint32_t *ctr, uint32_t *nfirst, uint32_t *ncount, uint32_t *nparent, int64_t n,
                            const int64_t *__restrict__ seg_off, int64_t nseg) {
    if (aborted(ctr, kStageAfter)) return;
    const int t = threadIdx.x;
    if (blockIdx.x == 0) {
        if (t < kLevels + 1) {
            ctr[kCtrLevelTrunc + t] = 0xffffffffu;
            ctr[kCtrLevelRawEnd + t] = 0;
            ctr[kCtrLevelStart + t] = 0;
        }
        __syncthreads();
        if (t == 0) ctr[kCtrLevelRawEnd + 0] = n > 0 ? (uint32_t)nseg : 0u;
    }
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + t;
    if (b < nseg) {
        nfirst[b] = nseg > 1 ? (uint32_t)seg_off[b] : 0u;
        ncount[b] = nseg > 1 ? (uint32_t)(seg_off[b + 1] - seg_off[b]) : (uint32_t)n;
        nparent[b] = (uint32_t)b;
    }
}

// Octant boundaries of a node's sorted range [first, first + count), count
// >= 1: b[o] = first index whose octant digit at `shift` is >= o, o = 1..7
// (keys in the range share their higher digits, so the digit is
// non-decreasing).  Seven branchless lower-bound searches advance in lock
// step, so each step issues seven independent loads: a large node costs
// log2(count) load latencies, not seven times that.
__device__ __forceinline__ void octant_bounds(const uint64_t *__restrict__ skey, uint32_t first, uint32_t count,
                                              int shift, uint32_t (&b)[9]) {
    uint32_t base[7];
#pragma unroll
    for (int o = 0; o < 7; ++o) base[o] = first;
    uint32_t len = count;
    while (len > 1) {
        const uint32_t half = len >> 1;
#pragma unroll
        for (int o = 0; o < 7; ++o)
            if ((uint32_t)((skey[base[o] + half] >> shift) & 7u) < (uint32_t)(o + 1)) base[o] += half;
        len -= half;
    }
#pragma unroll
    for (int o = 0; o < 7; ++o) b[o + 1] = base[o] + ((uint32_t)((skey[base[o]] >> shift) & 7u) < (uint32_t)(o + 1));
    b[0] = first;
    b[8] = first + count;
}

// Level L: every node decides leaf/internal; internal nodes find their
// octant boundaries by binary search, a block scan plus a decoupled
// look-back across tiles numbers the children breadth-first, and the
// children's ranges are written for level L+1.
__global__ void __launch_bounds__(kLevelThreads) k_level(
    int L, const uint64_t *__restrict__ skey, uint32_t *__restrict__ nfirst, uint32_t *__restrict__ ncount,
    uint4 *__restrict__ ngeo, uint2 *__restrict__ nlink, uint32_t *__restrict__ nparent, uint32_t *ctr,
    uint32_t *lstatus, uint32_t lcap, uint32_t node_cap, int32_t *dstatus, const DevCtl *__restrict__ ctl) {
    __shared__ uint32_t s_tile, s_excl, s_total;
    __shared__ uint32_t wt[32];
    const uint32_t stage = kStageLevel0 + (uint32_t)L;
    if (aborted(ctr, stage)) return;
    const uint32_t start = ctr[kCtrLevelStart + L];
    const uint32_t raw = ctr[kCtrLevelRawEnd + L], tr = ctr[kCtrLevelTrunc + L];
    const uint32_t end = raw < tr ? raw : tr;
    const uint32_t nl = end > start ? end - start : 0;
    const uint32_t ntiles = (nl + kLevelThreads - 1) / kLevelThreads;
    const int tid = threadIdx.x;
    if (blockIdx.x == 0 && tid == 0) {
        ctr[kCtrLevelStart + L + 1] = end;
        if (ntiles == 0) ctr[kCtrLevelRawEnd + L + 1] = end;
    }
    const int shift = 3 * (kMaxLevel - 1 - L);
    const uint32_t cmask = ~((1u << (kBits - L)) - 1u);
    while (true) {
        if (tid == 0) s_tile = atomicAdd(ctr + kCtrLevelTicket + L, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        __syncthreads();
        if (tile >= ntiles) break;
        const uint32_t node = start + tile * kLevelThreads + tid;
        const bool valid = node < end;
        uint32_t first = 0, count = 0;
        uint64_t k0 = 0;
        if (valid) {
            first = nfirst[node];
            count = ncount[node];
            k0 = skey[first];
        }
        bool internal = valid && count > lcap && L < kMaxLevel;
        uint32_t b[9];
        uint32_t nch = 0;
        if (internal) {
            octant_bounds(skey, first, count, shift, b);
#pragma unroll
            for (int o = 0; o < 8; ++o) nch += b[o + 1] > b[o] ? 1u : 0u;
        }
        uint32_t tot;
        const uint32_t loc = block_exclusive_scan(nch, wt, &tot);
        if (tid == 0) {
            s_excl = lookback_single(lstatus, tile, tot, WaitCtx{dstatus, ctr, stage, ctl->wait_cycles});
            s_total = tot;
        }
        __syncthreads();
        const uint32_t cf = end + s_excl + loc;
        if (internal && (uint64_t)cf + nch > node_cap) {
            internal = false;
            atomicMin(ctr + kCtrLevelTrunc + L + 1, cf);
            set_status(dstatus, TREE_DEV_NODES);
        }
        if (valid) {
            const uint32_t cx = compact3(k0 >> 2) & cmask, cy = compact3(k0 >> 1) & cmask,
                           cz = compact3(k0) & cmask;
            ngeo[node] = make_uint4(cx, cy, cz, (uint32_t)L | (internal ? 0u : 0x100u));
            nlink[node] = internal ? make_uint2(cf, nch) : make_uint2(first, count);
        }
        if (internal) {
            uint32_t c = cf;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                if (b[o + 1] > b[o]) {
                    nfirst[c] = b[o];
                    ncount[c] = b[o + 1] - b[o];
                    nparent[c] = node;
                    ++c;
                }
            }
        }
        if (tile == ntiles - 1 && tid == 0) ctr[kCtrLevelRawEnd + L + 1] = end + s_excl + s_total;
        __syncthreads();
    }
}

cudaError_t launch_octree(TreeWorkspace *ws, int64_t n, cudaStream_t s) {
    k_tree_init<<<grid_for(ws->nseg, 128, 1 << 20), 128, 0, s>>>(ws->ctr, ws->nfirst, ws->ncount, ws->nparent, n,
                                                                 ws->seg_off, ws->nseg);
    double maxl = (double)ws->nseg;
    for (int L = 0; L < kLevels; ++L) {
        double bound = fmin(fmin(maxl, (double)n), (double)ws->node_cap);
        int nb = grid_for((int64_t)bound, kLevelThreads, 152 * 8);
        uint32_t *lst = ws->level_status + (size_t)L * ws->level_tiles_max;
        k_level<<<nb, kLevelThreads, 0, s>>>(L, ws->key, ws->nfirst, ws->ncount, ws->ngeo, ws->nlink,
                                             ws->nparent, ws->ctr, lst, (uint32_t)ws->p.leaf_cap,
                                             (uint32_t)ws->node_cap, ws->dstatus, ws->dctl);
        maxl *= 8.0;
    }
    ws->launches += 1 + kLevels;
    return cudaGetLastError();
}

// ============================================================== gather
template <typename Real>
__global__ void __launch_bounds__(256) k_gather(const Real *__restrict__ x, const Real *__restrict__ m,
                                                const uint32_t *__restrict__ idx, int64_t n,
                                                typename Vec4<Real>::T *__restrict__ spos,
                                                const uint32_t *__restrict__ ctr) {
    if (aborted(ctr, kStageAfter)) return;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = idx[s];
        typename Vec4<Real>::T p;
        p.x = x[i];
        p.y = x[n + i];
        p.z = x[2 * n + i];
        p.w = m[i];
        spos[s] = p;
    }
}

// From the packed (x, y, z, m) copy the kick-drift pass wrote: one aligned
// vector load per particle.
template <typename V4>
__global__ void __launch_bounds__(256) k_gather_packed(const V4 *__restrict__ xm, const uint32_t *__restrict__ idx,
                                                       int64_t n, V4 *__restrict__ spos,
                                                       const uint32_t *__restrict__ ctr) {
    if (aborted(ctr, kStageAfter)) return;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        spos[s] = xm[idx[s]];
}

cudaError_t launch_gather_packed(TreeWorkspace *ws, int64_t n, cudaStream_t s) {
    int nb = grid_for(n, 256, 152 * 16);
    if (ws->p.precision == TREE_F64)
        k_gather_packed<double4a><<<nb, 256, 0, s>>>((const double4a *)ws->xm, ws->idx, n, (double4a *)ws->spos,
                                                     ws->ctr);
    else
        k_gather_packed<float4><<<nb, 256, 0, s>>>((const float4 *)ws->xm, ws->idx, n, (float4 *)ws->spos, ws->ctr);
    ws->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather(TreeWorkspace *ws, const void *x, const void *m, int64_t n, cudaStream_t s) {
    int nb = grid_for(n, 256, 152 * 16);
    if (ws->p.precision == TREE_F64)
        k_gather<double><<<nb, 256, 0, s>>>((const double *)x, (const double *)m, ws->idx, n,
                                            (double4a *)ws->spos, ws->ctr);
    else
        k_gather<float><<<nb, 256, 0, s>>>((const float *)x, (const float *)m, ws->idx, n,
                                           (float4 *)ws->spos, ws->ctr);
    ws->launches += 1;
    return cudaGetLastError();
}

// ============================================================== export (tests)
__global__ void k_export_tree(const uint4 *__restrict__ ngeo, const uint2 *__restrict__ nlink,
                              const uint32_t *__restrict__ nfirst, const uint32_t *__restrict__ ncount,
                              int64_t nn, int32_t *level, uint32_t *corner, uint32_t *first, uint32_t *count,
                              int32_t *child, int32_t *nchild) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nn; c += (int64_t)gridDim.x * blockDim.x) {
        const uint4 g = ngeo[c];
        const uint2 l = nlink[c];
        const bool leaf = (g.w >> 8) & 1u;
        if (level) level[c] = (int32_t)(g.w & 0xffu);
        if (corner) { corner[c] = g.x; corner[nn + c] = g.y; corner[2 * nn + c] = g.z; }
        if (first) first[c] = nfirst[c];
        if (count) count[c] = ncount[c];
        if (child) child[c] = leaf ? -1 : (int32_t)l.x;
        if (nchild) nchild[c] = leaf ? 0 : (int32_t)l.y;
    }
}

cudaError_t launch_export_tree(TreeWorkspace *ws, int64_t nn, int32_t *level, uint32_t *corner, uint32_t *first,
                               uint32_t *count, int32_t *child, int32_t *nchild, cudaStream_t s) {
    if (nn <= 0) return cudaSuccess;
    k_export_tree<<<grid_for(nn, 256, 152 * 8), 256, 0, s>>>(ws->ngeo, ws->nlink, ws->nfirst, ws->ncount, nn,
                                                              level, corner, first, count, child, nchild);
    ws->launches += 1;
    return cudaGetLastError();
}

}  // namespace treegb
