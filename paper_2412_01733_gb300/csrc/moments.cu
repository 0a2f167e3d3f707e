// moments.cu -- cell moments, bottom-up, in FP64 (Sec. 2: a far cell acts
// through its total mass at its centre of mass; the quadrupole is the next
// term of the expansion).
//
// Leaves sum their members about the cell's geometric centre c
// (u = r - c, |u| <= sqrt(3) s, so no large cancellation):
//   M = sum m,  S = sum m u,  T = sum m u u^T,
//   R = c + S / M,  T_R = T - S S^T / M,  Q = 3 T_R - tr(T_R) I.
// Internal cells combine their children (parallel-axis theorem of the
// traceless quadrupole), with d_k = R_k - R:
//   M = sum M_k,  R = c + sum M_k (R_k - c) / M,
//   Q = sum_k [Q_k + M_k (3 d_k d_k^T - |d_k|^2 I)].
// Massless cells get R = c, Q = 0.  The FP64 results are kept, and rounded
// copies in the walk's precision are packed for the walk (FP32: -Q).
#include "common.cuh"

namespace treegb {

template <typename Real>
__global__ void __launch_bounds__(256) k_moments_level(
    int L, const uint32_t *__restrict__ ctr, const uint4 *__restrict__ ngeo, const uint2 *__restrict__ nlink,
    const typename Vec4<Real>::T *__restrict__ spos, const DevBox *__restrict__ box,
    const uint32_t *__restrict__ nfirst, const int64_t *__restrict__ seg_off, int64_t nseg, double *__restrict__ mom64,
    int64_t cap, typename Vec4<Real>::T *__restrict__ mom_a, typename Vec4<Real>::T *__restrict__ mom_b,
    typename Vec2<Real>::T *__restrict__ mom_c) {
    const uint32_t start = ctr[kCtrLevelStart + L], end = ctr[kCtrLevelStart + L + 1];
    double *M_ = mom64, *Rx_ = mom64 + cap, *Ry_ = mom64 + 2 * cap, *Rz_ = mom64 + 3 * cap;
    double *Q_[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) Q_[c] = mom64 + (4 + c) * cap;
    for (uint32_t node = start + blockIdx.x * blockDim.x + threadIdx.x; node < end;
         node += gridDim.x * blockDim.x) {
        const uint4 g = ngeo[node];
        const uint2 lk = nlink[node];
        const int lvl = (int)(g.w & 0xffu);
        const bool leaf = (g.w >> 8) & 1u;
        // cell centre in the frame of the node's own segment
        const DevBox *bx = nseg > 1 ? box + seg_find(seg_off, nseg, nfirst[node]) : box;
        const double lo0 = bx->lo[0], lo1 = bx->lo[1], lo2 = bx->lo[2], unit = bx->unit;
        const double half = 0.5 * (double)(1u << (kBits - lvl));
        const double cx = lo0 + ((double)g.x + half) * unit;
        const double cy = lo1 + ((double)g.y + half) * unit;
        const double cz = lo2 + ((double)g.z + half) * unit;
        double M = 0, Rx, Ry, Rz, qxx = 0, qyy = 0, qzz = 0, qxy = 0, qxz = 0, qyz = 0;
        if (leaf) {
            double sx = 0, sy = 0, sz = 0, txx = 0, tyy = 0, tzz = 0, txy = 0, txz = 0, tyz = 0;
            for (uint32_t j = lk.x; j < lk.x + lk.y; ++j) {
                const typename Vec4<Real>::T p = spos[j];
                const double m = (double)p.w;
                const double ux = (double)p.x - cx, uy = (double)p.y - cy, uz = (double)p.z - cz;
                M += m;
                sx += m * ux; sy += m * uy; sz += m * uz;
                txx += m * ux * ux; tyy += m * uy * uy; tzz += m * uz * uz;
                txy += m * ux * uy; txz += m * ux * uz; tyz += m * uy * uz;
            }
            if (M != 0.0) {
                const double iM = 1.0 / M;
                Rx = cx + sx * iM; Ry = cy + sy * iM; Rz = cz + sz * iM;
                txx -= sx * sx * iM; tyy -= sy * sy * iM; tzz -= sz * sz * iM;
                txy -= sx * sy * iM; txz -= sx * sz * iM; tyz -= sy * sz * iM;
                const double tr = txx + tyy + tzz;
                qxx = 3.0 * txx - tr; qyy = 3.0 * tyy - tr; qzz = 3.0 * tzz - tr;
                qxy = 3.0 * txy; qxz = 3.0 * txz; qyz = 3.0 * tyz;
            } else {
                Rx = cx; Ry = cy; Rz = cz;
            }
        } else {
            double sx = 0, sy = 0, sz = 0;
            for (uint32_t c = lk.x; c < lk.x + lk.y; ++c) {
                const double mc = M_[c];
                M += mc;
                sx += mc * (Rx_[c] - cx); sy += mc * (Ry_[c] - cy); sz += mc * (Rz_[c] - cz);
            }
            if (M != 0.0) {
                const double iM = 1.0 / M;
                Rx = cx + sx * iM; Ry = cy + sy * iM; Rz = cz + sz * iM;
                for (uint32_t c = lk.x; c < lk.x + lk.y; ++c) {
                    const double mc = M_[c];
                    const double dx = Rx_[c] - Rx, dy = Ry_[c] - Ry, dz = Rz_[c] - Rz;
                    const double d2 = dx * dx + dy * dy + dz * dz;
                    qxx += Q_[0][c] + mc * (3.0 * dx * dx - d2);
                    qyy += Q_[1][c] + mc * (3.0 * dy * dy - d2);
                    qzz += Q_[2][c] + mc * (3.0 * dz * dz - d2);
                    qxy += Q_[3][c] + mc * (3.0 * dx * dy);
                    qxz += Q_[4][c] + mc * (3.0 * dx * dz);
                    qyz += Q_[5][c] + mc * (3.0 * dy * dz);
                }
            } else {
                Rx = cx; Ry = cy; Rz = cz;
            }
        }
        M_[node] = M; Rx_[node] = Rx; Ry_[node] = Ry; Rz_[node] = Rz;
        Q_[0][node] = qxx; Q_[1][node] = qyy; Q_[2][node] = qzz;
        Q_[3][node] = qxy; Q_[4][node] = qxz; Q_[5][node] = qyz;
        typename Vec4<Real>::T a, b;
        typename Vec2<Real>::T c;
        // the FP32 walk copies hold -Q (the sign its packed pair terms want)
        const double qs = sizeof(Real) == 4 ? -1.0 : 1.0;
        a.x = (Real)Rx; a.y = (Real)Ry; a.z = (Real)Rz; a.w = (Real)M;
        b.x = (Real)(qs * qxx); b.y = (Real)(qs * qyy); b.z = (Real)(qs * qzz); b.w = (Real)(qs * qxy);
        c.x = (Real)(qs * qxz); c.y = (Real)(qs * qyz);
        mom_a[node] = a; mom_b[node] = b; mom_c[node] = c;
    }
}

template <typename Real>
static cudaError_t moments_impl(TreeWorkspace *ws, cudaStream_t s) {
    int nb = grid_for(ws->node_cap, 256, 152 * 8);
    for (int L = kMaxLevel; L >= 0; --L) {
        k_moments_level<Real><<<nb, 256, 0, s>>>(
            L, ws->ctr, ws->ngeo, ws->nlink, (const typename Vec4<Real>::T *)ws->spos, ws->box, ws->nfirst,
            ws->seg_off, ws->nseg, ws->mom64,
            ws->node_cap, (typename Vec4<Real>::T *)ws->mom_a, (typename Vec4<Real>::T *)ws->mom_b,
            (typename Vec2<Real>::T *)ws->mom_c);
    }
    ws->launches += kLevels;
    return cudaGetLastError();
}

cudaError_t launch_moments(TreeWorkspace *ws, cudaStream_t s) {
    if (ws->p.precision == TREE_F64) return moments_impl<double>(ws, s);
    return moments_impl<float>(ws, s);
}

}  // namespace treegb
