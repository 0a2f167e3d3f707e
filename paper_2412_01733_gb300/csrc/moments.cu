// moments.cu -- cell moments in FP64 (Sec. 2: a far cell acts through its
// total mass at its centre of mass; the quadrupole is the next term of the
// expansion).
//
// Every cell sums its sources k (its particles, or its children as point
// masses at their centres of mass R_k) about a fixed point c near the cell's
// geometric centre (u_k = r_k - c, |u_k| <= sqrt(3) s, so no large
// cancellation):
//   M = sum m_k,  S = sum m_k u_k,  T = sum m_k u_k u_k^T,
//   R = c + S / M,  T_R = T - S S^T / M  (= sum m_k d_k d_k^T, d_k = r_k - R),
//   Q = sum_k Q_k + 3 T_R - tr(T_R) I,
// Q_k = 0 for particles: the parallel-axis theorem of the traceless
// quadrupole.  Massless cells get R = c, Q = 0.  M, S, T and Q are
// accumulated in FP64; rounded copies in the walk's precision are packed for
// the walk (FP32: -Q).
//
// Work order.  The FP64 pipe runs at 1/64 of the FP32 rate, and a warp
// issues its FP64 loop for its longest cell, so cells are first bucketed:
// leaves by particle count (one launch for all leaves, since they only need
// particles), internal cells by (level, number of children) (one launch per
// level, finest first).  A warp then mostly holds cells with equal trip
// counts.  The order inside a bucket is arbitrary; every cell's arithmetic
// is its own, so the results do not depend on it.
#include "common.cuh"

namespace treegb {

// bucket of a node: leaves 0..kMomLeafBuckets-1 by min(count, 17) (count 0
// with count 1), internal cells kMomLeafBuckets + 8 level + (nchild - 1)
__device__ __forceinline__ uint32_t mom_bucket(uint4 g, uint2 l) {
    if ((g.w >> 8) & 1u) return min(max(l.y, 1u), (uint32_t)kMomLeafBuckets) - 1u;
    return (uint32_t)kMomLeafBuckets + 8u * (g.w & 0xffu) + (l.y - 1u);
}

// Bucket counts of all nodes.
__global__ void __launch_bounds__(256) k_mom_hist(const uint32_t *__restrict__ ctr, const uint4 *__restrict__ ngeo,
                                                  const uint2 *__restrict__ nlink, uint32_t *__restrict__ cnt) {
    // after a given-up wait the buckets stay empty, so no later moment kernel does any work
    if (aborted(ctr, kStageAfter)) return;
    __shared__ uint32_t sh[kMomBuckets];
    for (int i = threadIdx.x; i < kMomBuckets; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t nn = ctr[kCtrLevelStart + kLevels];
    for (uint32_t node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x)
        atomicAdd(&sh[mom_bucket(ngeo[node], nlink[node])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kMomBuckets; i += blockDim.x)
        if (sh[i]) atomicAdd(cnt + i, sh[i]);
}

// Bucket offsets (every block scans the counts; block 0 stores them, with
// the total at [kMomBuckets]), then each tile of 256 nodes reserves its
// slots per bucket with one atomic per bucket and writes the node indices.
__global__ void __launch_bounds__(256) k_mom_scatter(const uint32_t *__restrict__ ctr, const uint4 *__restrict__ ngeo,
                                                     const uint2 *__restrict__ nlink, const uint32_t *__restrict__ cnt,
                                                     uint32_t *__restrict__ off, uint32_t *__restrict__ cursor,
                                                     uint32_t *__restrict__ order) {
    if (aborted(ctr, kStageAfter)) return;
    __shared__ uint32_t s_off[kMomBuckets + 1], s_cnt[kMomBuckets], s_base[kMomBuckets];
    for (int b = threadIdx.x; b < kMomBuckets; b += blockDim.x) s_cnt[b] = cnt[b];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < kMomBuckets; ++b) {
            s_off[b] = run;
            run += s_cnt[b];
        }
        s_off[kMomBuckets] = run;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int b = threadIdx.x; b <= kMomBuckets; b += blockDim.x) off[b] = s_off[b];
    const uint32_t nn = ctr[kCtrLevelStart + kLevels];
    for (uint32_t base = blockIdx.x * blockDim.x; base < nn; base += gridDim.x * blockDim.x) {
        for (int b = threadIdx.x; b < kMomBuckets; b += blockDim.x) s_cnt[b] = 0;
        __syncthreads();
        const uint32_t node = base + threadIdx.x;
        const bool valid = node < nn;
        uint32_t b = 0, rank = 0;
        if (valid) {
            b = mom_bucket(ngeo[node], nlink[node]);
            rank = atomicAdd(&s_cnt[b], 1u);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kMomBuckets; q += blockDim.x)
            if (s_cnt[q]) s_base[q] = atomicAdd(cursor + q, s_cnt[q]);
        __syncthreads();
        if (valid) order[s_off[b] + s_base[b] + rank] = node;
        __syncthreads();
    }
}

// FP64 sums of one cell about c and its finished moments.
struct MomSums {
    double M = 0, sx = 0, sy = 0, sz = 0, txx = 0, tyy = 0, tzz = 0, txy = 0, txz = 0, tyz = 0;
    double qxx = 0, qyy = 0, qzz = 0, qxy = 0, qxz = 0, qyz = 0;  // sum of the sources' own Q
    __device__ __forceinline__ void add(double m, double ux, double uy, double uz) {
        M += m;
        const double mx = m * ux, my = m * uy, mz = m * uz;
        sx += mx; sy += my; sz += mz;
        txx = fma(mx, ux, txx); tyy = fma(my, uy, tyy); tzz = fma(mz, uz, tzz);
        txy = fma(mx, uy, txy); txz = fma(mx, uz, txz); tyz = fma(my, uz, tyz);
    }
};

template <typename Real>
__device__ __forceinline__ void mom_store(const MomSums &a, double cx, double cy, double cz, uint32_t node,
                                          double *__restrict__ mom64, int64_t cap,
                                          typename Vec4<Real>::T *__restrict__ mom_a,
                                          typename Vec4<Real>::T *__restrict__ mom_b,
                                          typename Vec2<Real>::T *__restrict__ mom_c) {
    double Rx = cx, Ry = cy, Rz = cz, qxx = 0, qyy = 0, qzz = 0, qxy = 0, qxz = 0, qyz = 0;
    if (a.M != 0.0) {
        const double iM = 1.0 / a.M;
        Rx = cx + a.sx * iM; Ry = cy + a.sy * iM; Rz = cz + a.sz * iM;
        const double txx = a.txx - a.sx * a.sx * iM, tyy = a.tyy - a.sy * a.sy * iM, tzz = a.tzz - a.sz * a.sz * iM;
        const double txy = a.txy - a.sx * a.sy * iM, txz = a.txz - a.sx * a.sz * iM, tyz = a.tyz - a.sy * a.sz * iM;
        const double tr = txx + tyy + tzz;
        qxx = a.qxx + (3.0 * txx - tr); qyy = a.qyy + (3.0 * tyy - tr); qzz = a.qzz + (3.0 * tzz - tr);
        qxy = a.qxy + 3.0 * txy; qxz = a.qxz + 3.0 * txz; qyz = a.qyz + 3.0 * tyz;
    }
    mom64[node] = a.M; mom64[cap + node] = Rx; mom64[2 * cap + node] = Ry; mom64[3 * cap + node] = Rz;
    mom64[4 * cap + node] = qxx; mom64[5 * cap + node] = qyy; mom64[6 * cap + node] = qzz;
    mom64[7 * cap + node] = qxy; mom64[8 * cap + node] = qxz; mom64[9 * cap + node] = qyz;
    // the FP32 walk copies hold -Q (the sign its packed pair terms want)
    const double qs = sizeof(Real) == 4 ? -1.0 : 1.0;
    typename Vec4<Real>::T A, B;
    typename Vec2<Real>::T C;
    A.x = (Real)Rx; A.y = (Real)Ry; A.z = (Real)Rz; A.w = (Real)a.M;
    B.x = (Real)(qs * qxx); B.y = (Real)(qs * qyy); B.z = (Real)(qs * qzz); B.w = (Real)(qs * qxy);
    C.x = (Real)(qs * qxz); C.y = (Real)(qs * qyz);
    mom_a[node] = A; mom_b[node] = B; mom_c[node] = C;
}

// Expansion point c of a node: its geometric centre, in the frame of the
// node's own segment.  The FP32 path rounds it to FP32 with one FP32 fused
// multiply-add (any point near the cell serves; the FP32 particle
// coordinates then differ from it by exactly representable FP64 values).
template <typename Real>
__device__ __forceinline__ void mom_centre(uint4 g, uint32_t node, const DevBox *__restrict__ box,
                                           const uint32_t *__restrict__ nfirst, const int64_t *__restrict__ seg_off,
                                           int64_t nseg, double &cx, double &cy, double &cz) {
    const DevBox *bx = nseg > 1 ? box + seg_find(seg_off, nseg, nfirst[node]) : box;
    const int lvl = (int)(g.w & 0xffu);
    if (sizeof(Real) == 4) {
        const float half = 0.5f * (float)(1u << (kBits - lvl)), unit = (float)bx->unit;
        cx = (double)__fmaf_rn((float)g.x + half, unit, (float)bx->lo[0]);
        cy = (double)__fmaf_rn((float)g.y + half, unit, (float)bx->lo[1]);
        cz = (double)__fmaf_rn((float)g.z + half, unit, (float)bx->lo[2]);
    } else {
        const double half = 0.5 * (double)(1u << (kBits - lvl)), unit = bx->unit;
        cx = bx->lo[0] + ((double)g.x + half) * unit;
        cy = bx->lo[1] + ((double)g.y + half) * unit;
        cz = bx->lo[2] + ((double)g.z + half) * unit;
    }
}

// All leaves, in bucket order: sums over the cell's particles.
template <typename Real>
__global__ void __launch_bounds__(256) k_moments_leaves(
    const uint32_t *__restrict__ off, const uint32_t *__restrict__ order, const uint4 *__restrict__ ngeo,
    const uint2 *__restrict__ nlink, const typename Vec4<Real>::T *__restrict__ spos, const DevBox *__restrict__ box,
    const uint32_t *__restrict__ nfirst, const int64_t *__restrict__ seg_off, int64_t nseg, double *__restrict__ mom64,
    int64_t cap, typename Vec4<Real>::T *__restrict__ mom_a, typename Vec4<Real>::T *__restrict__ mom_b,
    typename Vec2<Real>::T *__restrict__ mom_c) {
    const uint32_t end = off[kMomLeafBuckets];
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < end; t += gridDim.x * blockDim.x) {
        const uint32_t node = order[t];
        const uint4 g = ngeo[node];
        const uint2 lk = nlink[node];
        double cx, cy, cz;
        mom_centre<Real>(g, node, box, nfirst, seg_off, nseg, cx, cy, cz);
        MomSums a;
        for (uint32_t j = lk.x; j < lk.x + lk.y; ++j) {
            const typename Vec4<Real>::T p = spos[j];
            a.add((double)p.w, (double)p.x - cx, (double)p.y - cy, (double)p.z - cz);
        }
        mom_store<Real>(a, cx, cy, cz, node, mom64, cap, mom_a, mom_b, mom_c);
    }
}

// Internal cells of level L: sums over the children's (M_k, R_k, Q_k).
template <typename Real>
__global__ void __launch_bounds__(256) k_moments_level(
    int L, const uint32_t *__restrict__ off, const uint32_t *__restrict__ order, const uint4 *__restrict__ ngeo,
    const uint2 *__restrict__ nlink, const DevBox *__restrict__ box, const uint32_t *__restrict__ nfirst,
    const int64_t *__restrict__ seg_off, int64_t nseg, double *__restrict__ mom64, int64_t cap,
    typename Vec4<Real>::T *__restrict__ mom_a, typename Vec4<Real>::T *__restrict__ mom_b,
    typename Vec2<Real>::T *__restrict__ mom_c) {
    const uint32_t b0 = kMomLeafBuckets + 8 * L;
    const uint32_t start = off[b0], end = off[b0 + 8];
    const double *M_ = mom64, *Rx_ = mom64 + cap, *Ry_ = mom64 + 2 * cap, *Rz_ = mom64 + 3 * cap;
    for (uint32_t t = start + blockIdx.x * blockDim.x + threadIdx.x; t < end; t += gridDim.x * blockDim.x) {
        const uint32_t node = order[t];
        const uint4 g = ngeo[node];
        const uint2 lk = nlink[node];
        double cx, cy, cz;
        mom_centre<Real>(g, node, box, nfirst, seg_off, nseg, cx, cy, cz);
        MomSums a;
        for (uint32_t k = lk.x; k < lk.x + lk.y; ++k) {
            a.add(M_[k], Rx_[k] - cx, Ry_[k] - cy, Rz_[k] - cz);
            a.qxx += mom64[4 * cap + k]; a.qyy += mom64[5 * cap + k]; a.qzz += mom64[6 * cap + k];
            a.qxy += mom64[7 * cap + k]; a.qxz += mom64[8 * cap + k]; a.qyz += mom64[9 * cap + k];
        }
        mom_store<Real>(a, cx, cy, cz, node, mom64, cap, mom_a, mom_b, mom_c);
    }
}

// Per segment b (its root is node b), whether the FP32 walk may take its
// r^-5 far-cell form: pc_r5_fits of the segment's cube and root mass.
__global__ void __launch_bounds__(256) k_r5_flags(const uint32_t *__restrict__ ctr, DevBox *box,
                                                  const float4 *__restrict__ mom_a, int64_t nseg) {
    if (aborted(ctr, kStageAfter)) return;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nseg; b += (int64_t)gridDim.x * blockDim.x)
        box[b].r5fit = pc_r5_fits(box[b].k, mom_a[b].w) ? 1 : 0;
}

template <typename Real>
static cudaError_t moments_impl(TreeWorkspace *ws, cudaStream_t s) {
    using V4 = typename Vec4<Real>::T;
    using V2 = typename Vec2<Real>::T;
    uint32_t *cnt = ws->mbucket, *off = ws->mbucket + kMomBuckets, *cursor = ws->mbucket + 2 * kMomBuckets + 1;
    cudaError_t e = cudaMemsetAsync(ws->mbucket, 0, (3 * kMomBuckets + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int64_t cap = ws->node_cap;
    k_mom_hist<<<grid_for(cap, 256, 152 * 8), 256, 0, s>>>(ws->ctr, ws->ngeo, ws->nlink, cnt);
    k_mom_scatter<<<grid_for(cap, 256, 152 * 8), 256, 0, s>>>(ws->ctr, ws->ngeo, ws->nlink, cnt, off,
                                                                             cursor, ws->morder);
    k_moments_leaves<Real><<<grid_for(cap, 256, 152 * 8), 256, 0, s>>>(
        off, ws->morder, ws->ngeo, ws->nlink, (const V4 *)ws->spos, ws->box, ws->nfirst, ws->seg_off, ws->nseg,
        ws->mom64, cap, (V4 *)ws->mom_a, (V4 *)ws->mom_b, (V2 *)ws->mom_c);
    const int nbl = grid_for(cap, 256, 152 * 8);
    for (int L = kMaxLevel - 1; L >= 0; --L)
        k_moments_level<Real><<<nbl, 256, 0, s>>>(L, off, ws->morder, ws->ngeo, ws->nlink, ws->box, ws->nfirst,
                                                 ws->seg_off, ws->nseg, ws->mom64, ws->node_cap, (V4 *)ws->mom_a,
                                                 (V4 *)ws->mom_b, (V2 *)ws->mom_c);
    ws->launches += 3 + kMaxLevel;
    if (sizeof(Real) == 4) {
        k_r5_flags<<<grid_for(ws->nseg, 256, 152), 256, 0, s>>>(ws->ctr, ws->box, (const float4 *)ws->mom_a,
                                                               ws->nseg);
        ws->launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_moments(TreeWorkspace *ws, cudaStream_t s) {
    if (ws->p.precision == TREE_F64) return moments_impl<double>(ws, s);
    return moments_impl<float>(ws, s);
}

}  // namespace treegb
