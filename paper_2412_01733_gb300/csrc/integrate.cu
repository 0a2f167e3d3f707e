// integrate.cu -- leapfrog kick+drift fused with the box reduction (Eqs. 2-3),
// FP64 diagnostics, the direct-summation reference of Eq. 1, and the small
// scans/reductions over per-group walk records.
#include <float.h>
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace treegb {

// ============================================================== kick + drift + box
// v += tau/2 a (Eq. 2); x += tau v (Eq. 3); per-block FP64 min/max of the new
// positions for the next tree (the same partial layout as the box kernel).
// The new positions also go, with the masses, into a packed (x, y, z, m) copy
// in caller order, from which the tree's gather reads one aligned vector per
// particle instead of four scattered scalars.
template <typename Real>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 6 : 3) k_kick_drift_box(Real *__restrict__ x, Real *__restrict__ v,
                                                        const Real *__restrict__ a, const Real *__restrict__ m,
                                                        typename Vec4<Real>::T *__restrict__ xm, Real half_tau,
                                                        Real tau, int64_t n, double *__restrict__ part,
                                                        int32_t *dstatus) {
    __shared__ double sh[6][8];
    const Real big = sizeof(Real) == 4 ? (Real)FLT_MAX : (Real)DBL_MAX;
    Real mn[3] = {big, big, big}, mx[3] = {-big, -big, -big};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Real xn[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const Real vv = fma(half_tau, a[d * n + i], v[d * n + i]);
            const Real xx = fma(tau, vv, x[d * n + i]);
            v[d * n + i] = vv;
            x[d * n + i] = xx;
            xn[d] = xx;
            if (!isfinite(xx)) { bad = true; continue; }
            mn[d] = min(mn[d], xx);
            mx[d] = max(mx[d], xx);
        }
        typename Vec4<Real>::T p;
        p.x = xn[0]; p.y = xn[1]; p.z = xn[2]; p.w = m[i];
        xm[i] = p;
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

cudaError_t launch_kick_drift_box(TreeWorkspace *ws, void *x, void *v, const void *a, const void *m, double tau,
                                  int64_t n, cudaStream_t s) {
    if (ws->nseg > 1) return launch_box_segments(ws, x, v, a, m, tau, n, true, s);
    int nb;
    if (ws->p.precision == TREE_F64) {
        nb = wave_grid(k_kick_drift_box<double>, n, 256, kMaxBlocksReduce);
        k_kick_drift_box<double><<<nb, 256, 0, s>>>((double *)x, (double *)v, (const double *)a, (const double *)m,
                                                    (double4a *)ws->xm, 0.5 * tau, tau, n, ws->part, ws->dstatus);
    } else {
        nb = wave_grid(k_kick_drift_box<float>, n, 256, kMaxBlocksReduce);
        k_kick_drift_box<float><<<nb, 256, 0, s>>>((float *)x, (float *)v, (const float *)a, (const float *)m,
                                                   (float4 *)ws->xm, (float)(0.5 * tau), (float)tau, n, ws->part,
                                                   ws->dstatus);
    }
    ws->launches += 1;
    return launch_box_final(ws, nb, s);
}

// ============================================================== diagnostics (FP64)
// E_kin = 1/2 sum m v^2, W = 1/2 sum m phi, P = sum m v, L = sum m x cross v.
// Fixed grid and fixed reduction order: deterministic.
// Per-particle products in the input precision, summed in that precision
// over runs of 32 particles per thread, then accumulated in FP64.  A run is
// its own loop, so the FP64 flush issues once per run (folded into the
// particle loop as a predicated branch, it issued for every particle).
template <typename Real>
__device__ __forceinline__ void diag_accumulate(const Real *__restrict__ x, const Real *__restrict__ v,
                                                const Real *__restrict__ m, const Real *__restrict__ phi, int64_t n,
                                                int64_t i, int64_t end, int64_t step, double (&q)[8]) {
    while (i < end) {
        Real r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < 32 && i < end; ++k, i += step) {
            const Real mi = m[i];
            const Real x0 = x[i], x1 = x[n + i], x2 = x[2 * n + i];
            const Real v0 = v[i], v1 = v[n + i], v2 = v[2 * n + i];
            r[0] += mi * (v0 * v0 + v1 * v1 + v2 * v2);
            if (phi) r[1] += mi * phi[i];
            r[2] += mi * v0; r[3] += mi * v1; r[4] += mi * v2;
            r[5] += mi * (x1 * v2 - x2 * v1);
            r[6] += mi * (x2 * v0 - x0 * v2);
            r[7] += mi * (x0 * v1 - x1 * v0);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) q[c] += (double)r[c];
    }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_diag_partial(const Real *__restrict__ x, const Real *__restrict__ v,
                                                      const Real *__restrict__ m, const Real *__restrict__ phi,
                                                      int64_t n, double *__restrict__ part) {
    __shared__ double sh[8][8];
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    diag_accumulate(x, v, m, phi, n, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, n,
                    (int64_t)gridDim.x * blockDim.x, q);
    q[0] *= 0.5;
    q[1] *= 0.5;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        for (int o = 16; o > 0; o >>= 1) q[c] += __shfl_xor_sync(0xffffffffu, q[c], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int c = 0; c < 8; ++c) sh[c][warp] = q[c];
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        part[blockIdx.x * 8 + threadIdx.x] = t;
    }
}

// One block of 256 threads: 32 threads per component each add every 32nd
// partial, then one thread per component adds their 32 sums (fixed order).
__global__ void __launch_bounds__(256) k_diag_final(const double *__restrict__ part, int nb, double *out) {
    const int c = threadIdx.x & 7, j = threadIdx.x >> 3;  // 32 lanes per component
    double r = 0;
    for (int b = j; b < nb; b += 32) r += part[b * 8 + c];
    __shared__ double sh[8][33];
    sh[c][j] = r;
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0;
        for (int k = 0; k < 32; ++k) t += sh[threadIdx.x][k];
        out[threadIdx.x] = t;
    }
}

cudaError_t launch_diagnostics(TreeWorkspace *ws, const void *x, const void *v, const void *m,
                               const void *phi, int64_t n, double *out, cudaStream_t s) {
    const int nb = ws->p.precision == TREE_F64 ? wave_grid(k_diag_partial<double>, n, 256, kMaxBlocksReduce)
                                               : wave_grid(k_diag_partial<float>, n, 256, kMaxBlocksReduce);
    if (ws->p.precision == TREE_F64)
        k_diag_partial<double><<<nb, 256, 0, s>>>((const double *)x, (const double *)v, (const double *)m,
                                                  (const double *)phi, n, ws->part);
    else
        k_diag_partial<float><<<nb, 256, 0, s>>>((const float *)x, (const float *)v, (const float *)m,
                                                 (const float *)phi, n, ws->part);
    k_diag_final<<<1, 256, 0, s>>>(ws->part, nb, out);
    ws->launches += 2;
    return cudaGetLastError();
}

// Per-segment diagnostics: the same sums over each segment's own particles,
// one block per box chunk (chunks never straddle segments), then one thread
// per segment adds its chunks in order.  out: [nseg][8].
template <typename Real>
__global__ void __launch_bounds__(256) k_diag_chunks(const Real *__restrict__ x, const Real *__restrict__ v,
                                                     const Real *__restrict__ m, const Real *__restrict__ phi,
                                                     int64_t n, const uint4 *__restrict__ chunks, int64_t nchunks,
                                                     double *__restrict__ part) {
    __shared__ double sh[8][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const uint4 c = chunks[ch];
        double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        diag_accumulate(x, v, m, phi, n, (int64_t)c.x + threadIdx.x, (int64_t)c.y, (int64_t)blockDim.x, q);
        q[0] *= 0.5;
        q[1] *= 0.5;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            for (int o = 16; o > 0; o >>= 1) q[k] += __shfl_xor_sync(0xffffffffu, q[k], o);
        if (lane == 0)
            for (int k = 0; k < 8; ++k) sh[k][warp] = q[k];
        __syncthreads();
        if (threadIdx.x < 8) {
            double t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
            part[ch * 8 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

__global__ void k_diag_seg_final(const double *__restrict__ part, const uint32_t *__restrict__ bfirst, int64_t nseg,
                                 double *__restrict__ out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nseg) return;
    double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t c = bfirst[b]; c < bfirst[b + 1]; ++c)
        for (int k = 0; k < 8; ++k) r[k] += part[c * 8 + k];
    for (int k = 0; k < 8; ++k) out[b * 8 + k] = r[k];
}

cudaError_t launch_diagnostics_segments(TreeWorkspace *ws, const void *x, const void *v, const void *m,
                                        const void *phi, int64_t n, double *out, cudaStream_t s) {
    const int nb = grid_for(ws->seg_nbchunk * 256, 256, 152 * 16);
    if (ws->p.precision == TREE_F64)
        k_diag_chunks<double><<<nb, 256, 0, s>>>((const double *)x, (const double *)v, (const double *)m,
                                                 (const double *)phi, n, ws->seg_bchunk, ws->seg_nbchunk,
                                                 ws->seg_part);
    else
        k_diag_chunks<float><<<nb, 256, 0, s>>>((const float *)x, (const float *)v, (const float *)m,
                                                (const float *)phi, n, ws->seg_bchunk, ws->seg_nbchunk,
                                                ws->seg_part);
    k_diag_seg_final<<<grid_for(ws->nseg, 128, 1 << 20), 128, 0, s>>>(ws->seg_part, ws->seg_bfirst, ws->nseg, out);
    ws->launches += 2;
    return cudaGetLastError();
}

// ============================================================== direct sum (Eq. 1)
// blockIdx.x: 128 targets; blockIdx.y: one chunk of the sources [jbeg, jend).
// Pair terms in the working precision through the reciprocal square root;
// per-128-source partial sums folded with Kahan compensation; the chunk totals
// are written in FP64 and summed over chunks in a fixed order.  A target index
// outside [0, n) reads nothing and gets NaN results.
constexpr int kDirThreads = 128;

template <typename Real>
__global__ void __launch_bounds__(kDirThreads) k_direct(const Real *__restrict__ x, const Real *__restrict__ m,
                                                        int64_t n, int64_t jbeg, int64_t jend,
                                                        const int64_t *__restrict__ tgt, int64_t nt, int64_t chunk,
                                                        double eps2d, double *__restrict__ part) {
    using V4 = typename Vec4<Real>::T;
    __shared__ V4 src[kDirThreads];
    const int64_t t = blockIdx.x * (int64_t)kDirThreads + threadIdx.x;
    const int64_t ti = t < nt ? tgt[t] : -1;
    const bool valid = ti >= 0 && ti < n;
    Real px = 0, py = 0, pz = 0;
    if (valid) { px = x[ti]; py = x[n + ti]; pz = x[2 * n + ti]; }
    const Real eps2 = (Real)eps2d;
    const int64_t j0 = jbeg + blockIdx.y * chunk;
    const int64_t j1 = min(jend, j0 + chunk);
    Real sum[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
    for (int64_t jb = j0; jb < j1; jb += kDirThreads) {
        const int64_t j = jb + threadIdx.x;
        V4 s;
        if (j < j1) { s.x = x[j]; s.y = x[n + j]; s.z = x[2 * n + j]; s.w = m[j]; }
        else { s.x = s.y = s.z = s.w = 0; }
        __syncthreads();
        src[threadIdx.x] = s;
        __syncthreads();
        const int ns = (int)min((int64_t)kDirThreads, j1 - jb);
        Real part_[4] = {0, 0, 0, 0};
        for (int k = 0; k < ns; ++k) {
            if (jb + k == ti) continue;
            const V4 q = src[k];
            const Real dx = q.x - px, dy = q.y - py, dz = q.z - pz;
            const Real r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (!(r2 > Real(0))) continue;
            const Real ri = sizeof(Real) == 8 ? (Real)rsqrt((double)r2) : (Real)rsqrtf((float)r2);
            const Real mr = q.w * ri;
            const Real w = mr * (ri * ri);
            part_[0] += w * dx; part_[1] += w * dy; part_[2] += w * dz;
            part_[3] -= mr;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const Real y = part_[c] - cmp[c];
            const Real tt = sum[c] + y;
            cmp[c] = (tt - sum[c]) - y;
            sum[c] = tt;
        }
    }
    if (t < nt) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            part[((int64_t)blockIdx.y * 4 + c) * nt + t] = valid ? (double)sum[c] - (double)cmp[c] : (double)NAN;
    }
}

__global__ void k_direct_final(const double *__restrict__ part, int64_t nt, int nchunks, double G,
                               double *__restrict__ a_out, double *__restrict__ phi_out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double r[4] = {0, 0, 0, 0};
    for (int c = 0; c < nchunks; ++c)
        for (int k = 0; k < 4; ++k) r[k] += part[((int64_t)c * 4 + k) * nt + t];
    a_out[t] = G * r[0];
    a_out[nt + t] = G * r[1];
    a_out[2 * nt + t] = G * r[2];
    if (phi_out) phi_out[t] = G * r[3];
}

// Chunking of the sources [jbeg, jend) for nt targets: about 16 blocks per SM
// in all, chunks a multiple of the block's 128 sources, at most max_chunks.
static void direct_chunks(int64_t nsrc, int64_t nt, int64_t max_chunks, int64_t *chunk_out, int64_t *nch_out) {
    const int64_t tt = (nt + kDirThreads - 1) / kDirThreads;
    int64_t nch = (152 * 16 + tt - 1) / tt;
    const int64_t maxch = (nsrc + kDirThreads - 1) / kDirThreads;
    if (nch > maxch) nch = maxch;
    if (nch > max_chunks) nch = max_chunks;
    if (nch > 65535) nch = 65535;
    if (nch < 1) nch = 1;
    int64_t chunk = (nsrc + nch - 1) / nch;
    chunk = ((chunk + kDirThreads - 1) / kDirThreads) * kDirThreads;
    if (chunk < kDirThreads) chunk = kDirThreads;
    nch = (nsrc + chunk - 1) / chunk;
    if (nch < 1) nch = 1;
    *chunk_out = chunk;
    *nch_out = nch;
}

// Direct sum for nt targets over the sources [jbeg, jend) of x (stride n).
cudaError_t launch_direct_range(TreeWorkspace *ws, const void *x, const void *m, int64_t n, int64_t jbeg,
                                int64_t jend, int dtype, double G, double eps, const int64_t *targets, int64_t nt,
                                double *a_out, double *phi_out, cudaStream_t s) {
    int64_t chunk = 0, nch = 1;
    direct_chunks(jend - jbeg, nt, INT64_MAX, &chunk, &nch);
    const size_t need = (size_t)nch * 4 * (size_t)nt * sizeof(double);
    if (need > ws->direct_part_bytes) {
        if (ws->direct_part) cudaFree(ws->direct_part);
        ws->direct_part = nullptr;
        ws->direct_part_bytes = 0;
        cudaError_t e = cudaMalloc(&ws->direct_part, need);
        if (e != cudaSuccess) return e;
        ws->direct_part_bytes = need;
    }
    const int64_t tt = (nt + kDirThreads - 1) / kDirThreads;
    dim3 grid((unsigned)tt, (unsigned)nch);
    const double eps2 = eps * eps;
    if (dtype == TREE_F64)
        k_direct<double><<<grid, kDirThreads, 0, s>>>((const double *)x, (const double *)m, n, jbeg, jend, targets,
                                                      nt, chunk, eps2, ws->direct_part);
    else
        k_direct<float><<<grid, kDirThreads, 0, s>>>((const float *)x, (const float *)m, n, jbeg, jend, targets, nt,
                                                     chunk, eps2, ws->direct_part);
    k_direct_final<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(ws->direct_part, nt, (int)nch, G, a_out, phi_out);
    ws->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_direct(TreeWorkspace *ws, const void *x, const void *m, int64_t n, int dtype,
                          const int64_t *targets, int64_t nt, double *a_out, double *phi_out,
                          cudaStream_t s) {
    return launch_direct_range(ws, x, m, n, 0, n, dtype, ws->p.G, ws->p.eps, targets, nt, a_out, phi_out, s);
}

// Widen FP32 positions / masses to FP64 (exact).
__global__ void k_widen(const float *__restrict__ in, int64_t count, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

cudaError_t launch_widen(TreeWorkspace *ws, const float *in, int64_t count, double *out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_widen<<<grid_for(count, 256, 152 * 8), 256, 0, s>>>(in, count, out);
    ws->launches += 1;
    return cudaGetLastError();
}

// err[t] = |a[:, tgt[t]] - ref[:, t]| / |ref[:, t]| (a: [3][n] of Real, ref: [3][nt] FP64).
template <typename Real>
__global__ void k_rel_err(const Real *__restrict__ a, int64_t n, const int64_t *__restrict__ tgt,
                          const double *__restrict__ ref, int64_t nt, double *__restrict__ err) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int64_t i = tgt[t];
    double d2 = 0.0, r2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double r = ref[c * nt + t];
        const double d = (double)a[c * n + i] - r;
        d2 += d * d;
        r2 += r * r;
    }
    err[t] = r2 > 0.0 ? sqrt(d2 / r2) : (d2 > 0.0 ? (double)INFINITY : 0.0);
}

cudaError_t launch_rel_err(TreeWorkspace *ws, const void *a, int64_t n, int dtype, const int64_t *tgt,
                           const double *ref, int64_t nt, double *err, cudaStream_t s) {
    if (nt <= 0) return cudaSuccess;
    if (dtype == TREE_F64)
        k_rel_err<double><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>((const double *)a, n, tgt, ref, nt, err);
    else
        k_rel_err<float><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>((const float *)a, n, tgt, ref, nt, err);
    ws->launches += 1;
    return cudaGetLastError();
}

// ============================================================== walk order of the groups
// Groups whose boxes are wide (sparse regions, or a run of the Morton curve
// that jumps between distant cells) cost far more than the rest.  Walking
// them first keeps them off the end of the launch.  Key: 21 - floor(log2 of
// the box's largest side in grid units); a counting sort by key (the order
// inside a key class is arbitrary; each group's result does not depend on it).
__global__ void __launch_bounds__(256) k_group_key(const uint64_t *__restrict__ skey, const uint32_t *__restrict__ gfirst,
                                                   const uint32_t *__restrict__ ctr, uint32_t *__restrict__ gkey,
                                                   uint32_t *bucket) {
    __shared__ uint32_t h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t ng = ctr[kCtrGroups];
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const uint32_t s0 = gfirst[g], s1 = gfirst[g + 1];
        uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
        for (uint32_t i = s0; i < s1; ++i) {
            const uint64_t k = skey[i];
            const uint32_t q[3] = {compact3(k >> 2), compact3(k >> 1), compact3(k)};
            for (int d = 0; d < 3; ++d) { lo[d] = min(lo[d], q[d]); hi[d] = max(hi[d], q[d]); }
        }
        const uint32_t e = max(hi[0] - lo[0], max(hi[1] - lo[1], hi[2] - lo[2]));
        const uint32_t key = 21u - (31u - (uint32_t)__clz(e | 1u));
        gkey[g] = key;
        atomicAdd(&h[key], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(bucket + threadIdx.x, h[threadIdx.x]);
}

__global__ void k_group_scan(uint32_t *bucket) {
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int k = 0; k < 32; ++k) {
            const uint32_t c = bucket[k];
            bucket[32 + k] = s;
            s += c;
        }
    }
}

__global__ void __launch_bounds__(256) k_group_scatter(const uint32_t *__restrict__ gkey, const uint32_t *__restrict__ ctr,
                                                       uint32_t *bucket, uint32_t *__restrict__ order) {
    const uint32_t ng = ctr[kCtrGroups];
    const int lane = threadIdx.x & 31;
    // warp-uniform trip count, one atomic per distinct key in a warp
    for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; b < ng; b += gridDim.x * blockDim.x) {
        const uint32_t g = b + lane;
        const uint32_t k = g < ng ? gkey[g] : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (g < ng && lane == leader) base = atomicAdd(bucket + 32 + k, (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (g < ng) order[base + __popc(peers & lanemask_lt())] = g;
    }
}

cudaError_t launch_group_order(TreeWorkspace *ws, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ws->gbucket, 0, 64 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int nb = grid_for(ws->n / 8 + 1, 256, 152 * 8);
    k_group_key<<<nb, 256, 0, s>>>(ws->key, ws->gfirst, ws->ctr, ws->gkey, ws->gbucket);
    k_group_scan<<<1, 32, 0, s>>>(ws->gbucket);
    k_group_scatter<<<nb, 256, 0, s>>>(ws->gkey, ws->ctr, ws->gbucket, ws->gorder);
    ws->launches += 3;
    return cudaGetLastError();
}

// ============================================================== direct sum without allocation
// tree_direct_forces needs a workspace, and the workspace allocates its
// scratch with cudaMalloc.  Callers that must not allocate device memory
// (for example an application whose memory pool owns the whole GPU, or code
// that may only use buffers it was handed) call tree_direct_forces_noalloc
// instead: the per-chunk partial sums live in this fixed module array, which
// every GPU that loads the library holds (4 MiB) until the process exits.
constexpr int64_t kNoAllocScratchDoubles = 524288;  // 4 MiB
static_assert(kNoAllocScratchDoubles >= 4 * (int64_t)TREE_NOALLOC_MAX_TARGETS, "scratch too small");
__device__ __align__(256) double g_noalloc_part[kNoAllocScratchDoubles];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_part on the current device (looked up once per
// device; host code cannot use the array's name as a device pointer).
cudaError_t noalloc_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}
}  // namespace

// ============================================================== per-group walk records
// gstat[g] = {n_pc cells, n_pp particles, max stack, n_pp leaves}.
// Pair totals: sum_g |g| n_pc and sum_g |g| n_pp; deepest stack.
__global__ void __launch_bounds__(256) k_gstat_reduce(const uint4 *__restrict__ gstat, const uint32_t *__restrict__ gfirst,
                                                      const uint32_t *__restrict__ ctr, unsigned long long *stats) {
    unsigned long long pp = 0, pc = 0, ms = 0;
    const uint32_t ng = ctr[kCtrGroups];
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const uint4 r = gstat[g];
        const unsigned long long c = (unsigned long long)(gfirst[g + 1] - gfirst[g]);
        pc += c * r.x;
        pp += c * r.y;
        ms = ms > r.z ? ms : r.z;
    }
    for (int o = 16; o > 0; o >>= 1) {
        pp += __shfl_xor_sync(0xffffffffu, pp, o);
        pc += __shfl_xor_sync(0xffffffffu, pc, o);
        unsigned long long t = __shfl_xor_sync(0xffffffffu, ms, o);
        ms = ms > t ? ms : t;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(stats + kStatPP, pp);
        atomicAdd(stats + kStatPC, pc);
        atomicMax(stats + kStatMaxStack, ms);
    }
}

// Exclusive scans of the per-group list lengths (x: PC cells, w: PP leaves)
// into list_off[0..ng] and list_off[ng+1 .. 2ng+1].  Single block: the list
// path is a test/adjoint path, not the force hot path.
__global__ void __launch_bounds__(1024) k_list_scan(const uint4 *__restrict__ gstat, int64_t ng,
                                                    int64_t *__restrict__ off) {
    __shared__ unsigned long long wt[2][32];
    __shared__ unsigned long long carry[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 2) carry[tid] = 0;
    __syncthreads();
    for (int64_t b = 0; b < ng; b += 1024) {
        const int64_t g = b + tid;
        unsigned long long v[2] = {0, 0};
        if (g < ng) { const uint4 r = gstat[g]; v[0] = r.x; v[1] = r.w; }
        unsigned long long x[2] = {v[0], v[1]};
        for (int o = 1; o < 32; o <<= 1) {
            for (int c = 0; c < 2; ++c) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, x[c], o);
                if (lane >= o) x[c] += y;
            }
        }
        if (lane == 31) { wt[0][warp] = x[0]; wt[1][warp] = x[1]; }
        __syncthreads();
        if (warp == 0) {
            for (int c = 0; c < 2; ++c) {
                unsigned long long t = wt[c][lane];
                for (int o = 1; o < 32; o <<= 1) {
                    unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o) t += y;
                }
                wt[c][lane] = t;
            }
        }
        __syncthreads();
        for (int c = 0; c < 2; ++c) {
            const unsigned long long before = (warp ? wt[c][warp - 1] : 0ull) + carry[c];
            if (g < ng) off[c * (ng + 1) + g] = (int64_t)(before + x[c] - v[c]);
        }
        __syncthreads();
        if (tid < 2) carry[tid] += wt[tid][31];
        __syncthreads();
    }
    if (tid < 2) off[tid * (ng + 1) + ng] = (int64_t)carry[tid];
}

__global__ void k_export_gstat(const uint4 *__restrict__ gstat, int64_t ng, uint32_t *__restrict__ out) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = gstat[g];
        out[g] = r.x; out[ng + g] = r.y; out[2 * ng + g] = r.z; out[3 * ng + g] = r.w;
    }
}

cudaError_t launch_export_gstat(TreeWorkspace *ws, int64_t ngroups, uint32_t *out, cudaStream_t s) {
    if (ngroups <= 0) return cudaSuccess;
    k_export_gstat<<<grid_for(ngroups, 256, 152 * 8), 256, 0, s>>>(ws->gstat, ngroups, out);
    ws->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_scan_lists(TreeWorkspace *ws, int64_t ngroups, cudaStream_t s) {
    k_list_scan<<<1, 1024, 0, s>>>(ws->gstat, ngroups, ws->list_cnt);
    ws->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gstat_reduce(TreeWorkspace *ws, int64_t ngroups, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ws->stats, 0, kStatCount * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_gstat_reduce<<<grid_for(ngroups, 256, 152 * 4), 256, 0, s>>>(ws->gstat, ws->gfirst, ws->ctr, ws->stats);
    ws->launches += 1;
    return cudaGetLastError();
}

}  // namespace treegb

extern "C" tree_status_t tree_direct_forces_noalloc(const void *x, const void *m, int64_t n, int32_t dtype,
                                                    double G, double eps, const int64_t *targets, int64_t nt,
                                                    double *a_out, double *phi_out, void *stream) {
    using namespace treegb;
    if (n < 0 || nt < 0) return TREE_ERR_ARG;
    if (dtype != TREE_F32 && dtype != TREE_F64) return TREE_ERR_ARG;
    if (!(eps >= 0.0) || !isfinite(eps) || !isfinite(G)) return TREE_ERR_ARG;
    if (nt > TREE_NOALLOC_MAX_TARGETS) return TREE_ERR_CAPACITY;
    if (nt == 0) return TREE_OK;
    if (!x || !m || !targets || !a_out || n < 1) return TREE_ERR_ARG;
    double *part = nullptr;
    if (noalloc_scratch(&part) != cudaSuccess) return TREE_ERR_CUDA;
    // same chunking as tree_direct_forces, capped so the partials fit the array
    const int64_t fit = kNoAllocScratchDoubles / (4 * nt);
    int64_t chunk = 0, nch = 1;
    direct_chunks(n, nt, fit, &chunk, &nch);
    // every partial slot [chunk][component][target] is written exactly once
    // before it is read, so the array needs no clearing between calls
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t tt = (nt + kDirThreads - 1) / kDirThreads;
    dim3 grid((unsigned)tt, (unsigned)nch);
    const double eps2 = eps * eps;
    if (dtype == TREE_F64)
        k_direct<double><<<grid, kDirThreads, 0, s>>>((const double *)x, (const double *)m, n, 0, n, targets, nt,
                                                      chunk, eps2, part);
    else
        k_direct<float><<<grid, kDirThreads, 0, s>>>((const float *)x, (const float *)m, n, 0, n, targets, nt, chunk,
                                                     eps2, part);
    k_direct_final<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(part, nt, (int)nch, G, a_out, phi_out);
    return cudaGetLastError() == cudaSuccess ? TREE_OK : TREE_ERR_CUDA;
}
