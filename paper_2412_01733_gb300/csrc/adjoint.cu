// adjoint.cu -- vector-Jacobian product of the tree force (Sec. 2 TreeCode,
// Eq. 1) with the tree structure of the last build held fixed: key order,
// cells, walk groups and the stored interaction lists.  Moments are
// functions of (x, m), so cell cotangents are carried back to the particles.
//
// Given cotangents abar (of the accelerations) and phibar (of the
// potentials), adds to xbar and mbar:
//   PP pair (source j, target i, d = r_j - r_i, s^2 = |d|^2 + eps^2):
//     g = G m_j (abar_i s^-3 - 3 d (d.abar_i) s^-5) + G m_j phibar_i d s^-3,
//     xbar_j += g, xbar_i -= g, mbar_j += G (d.abar_i) s^-3 - G phibar_i s^-1.
//   PC pair (cell C, y = r_i - R): derivative of the cell expansion with
//     respect to y (xbar_i += ybar, Rbar_C -= ybar), M and the six stored
//     quadrupole components.
//   Cell cotangents travel down the moment tree: with d = R_child - R_parent
//     (or r_j - R for the members of a leaf), Qf the symmetric matrix of the
//     stored-component cotangent (off-diagonals halved) and
//     f(d) = 3 d.Qf.d - |d|^2 tr Qf:
//       Mbar_child += Mbar + d.Rbar / M + f(d),
//       Rbar_child += (M_child / M) Rbar + M_child (6 Qf d - 2 tr(Qf) d),
//       Qbar_child += Qbar  (the children's quadrupoles enter Q linearly);
//     a massless cell passes only Mbar.
// One warp per group walks the group's stored lists, 32 sources (cells or
// particles) at a time, one source per lane.  Each (target, source) pair is
// evaluated once: the source-side cotangents (cell or particle) are summed in
// the lane and added to global FP64 accumulators with one atomic per
// quantity per source per group; the target-side sums rotate through the
// lanes with the targets.
#include <cfloat>

#include "common.cuh"

namespace treegb {

constexpr int kAdjWarps = 4;
constexpr int kAdjMaxTargets = 64;

struct AdjArgs {
    int64_t n;
    int64_t ngroups;
    const uint32_t *gfirst;
    const void *spos;      // Vec4 (x, y, z, m), key order
    const void *cot;       // Vec4 (abar, phibar), key order
    const uint2 *nlink;
    const void *mom_a, *mom_b, *mom_c;
    const int64_t *list_off;  // [2][ngroups + 1]
    const int32_t *pc_list, *pp_list;
    double G, eps2;
    double *xt;            // [3][n] target-side xbar (plain stores), key order
    double *xg;            // [3][n] source-side xbar (atomics), key order
    double *mg;            // [n]    source-side mbar (atomics), key order
    double *ccot;          // [10][cap] cell cotangents: Mbar, Rbar(3), Qbar(6)
    int64_t cap;
};

template <typename Real> struct AdjVec;
template <> struct AdjVec<float> { using V4 = float4; using V2 = float2; };
template <> struct AdjVec<double> { using V4 = double4a; using V2 = double2a; };

template <typename Real> __device__ __forceinline__ Real rs_(Real x);
template <> __device__ __forceinline__ float rs_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rs_<double>(double x) { return rsqrt(x); }

// 1/r of a pair.  Softened FP32 (SOFT, taken only when eps^2 is a normal FP32
// number): r^2 >= eps^2 is never subnormal, so the PTX reciprocal square root
// with subnormal inputs flushed serves, as in the walk's pair terms.
// Otherwise the guarded form: a pair at r^2 = 0 contributes nothing.
template <typename Real, bool SOFT>
__device__ __forceinline__ Real inv_r(Real r2) {
    if constexpr (SOFT && sizeof(Real) == 4) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
        return y;
    } else {
        return r2 > Real(0) ? rs_<Real>(r2) : Real(0);
    }
}

// Derivatives of abar.a_PC + pb phi_PC for one (target, cell) pair.
// y = target - R.  Outputs: gy (d/dy), mb (d/dM), qb (d/dQ stored components).
template <typename Real, bool QUAD, bool SOFT>
__device__ __forceinline__ void pc_vjp(Real yx, Real yy, Real yz, Real bx, Real by, Real bz, Real pb, Real Mc,
                                       const Real (&q)[6], Real eps2, Real &gx, Real &gy, Real &gz, Real &mb,
                                       Real (&qb)[6]) {
    const Real r2 = yx * yx + yy * yy + yz * yz + eps2;
    const Real i1 = inv_r<Real, SOFT>(r2);
    const Real i2 = i1 * i1;
    const Real i3 = i1 * i2, i5 = i3 * i2, i7 = i5 * i2, i9 = i7 * i2;
    const Real yb = yx * bx + yy * by + yz * bz;
    gx = -Mc * (bx * i3 - Real(3) * yx * yb * i5) + Mc * pb * yx * i3;
    gy = -Mc * (by * i3 - Real(3) * yy * yb * i5) + Mc * pb * yy * i3;
    gz = -Mc * (bz * i3 - Real(3) * yz * yb * i5) + Mc * pb * yz * i3;
    mb = -yb * i3 - pb * i1;
    if (QUAD) {
        const Real Qx = q[0] * yx + q[3] * yy + q[4] * yz;
        const Real Qy = q[3] * yx + q[1] * yy + q[5] * yz;
        const Real Qz = q[4] * yx + q[5] * yy + q[2] * yz;
        const Real yQy = yx * Qx + yy * Qy + yz * Qz;
        const Real Qb = Qx * bx + Qy * by + Qz * bz;
        const Real Qbx = q[0] * bx + q[3] * by + q[4] * bz;
        const Real Qby = q[3] * bx + q[1] * by + q[5] * bz;
        const Real Qbz = q[4] * bx + q[5] * by + q[2] * bz;
        const Real c1 = Real(17.5) * yQy * yb * i9 - Real(5) * Qb * i7 + Real(2.5) * pb * yQy * i7;
        const Real c2 = -Real(5) * yb * i7 - pb * i5;
        const Real c3 = -Real(2.5) * yQy * i7;
        gx += Qbx * i5 + c2 * Qx + c3 * bx + c1 * yx;
        gy += Qby * i5 + c2 * Qy + c3 * by + c1 * yy;
        gz += Qbz * i5 + c2 * Qz + c3 * bz + c1 * yz;
        const Real ca = i5, cb = -Real(2.5) * i7 * yb - Real(0.5) * pb * i5;
        qb[0] = ca * yx * bx + cb * yx * yx;
        qb[1] = ca * yy * by + cb * yy * yy;
        qb[2] = ca * yz * bz + cb * yz * yz;
        qb[3] = ca * (yx * by + yy * bx) + cb * Real(2) * yx * yy;
        qb[4] = ca * (yx * bz + yz * bx) + cb * Real(2) * yx * yz;
        qb[5] = ca * (yy * bz + yz * by) + cb * Real(2) * yy * yz;
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) qb[k] = Real(0);
    }
}

// PP pair: d = source - target.  g as in the header; dm = d/dm_j (without G).
template <typename Real, bool SOFT>
__device__ __forceinline__ void pp_vjp(Real dx, Real dy, Real dz, Real bx, Real by, Real bz, Real pb, Real mj,
                                       Real eps2, Real &gx, Real &gy, Real &gz, Real &dm) {
    const Real r2 = dx * dx + dy * dy + dz * dz + eps2;
    const Real i1 = inv_r<Real, SOFT>(r2);
    const Real i3 = i1 * i1 * i1, i5 = i3 * i1 * i1;
    const Real db = dx * bx + dy * by + dz * bz;
    gx = mj * (bx * i3 - Real(3) * dx * db * i5 + pb * dx * i3);
    gy = mj * (by * i3 - Real(3) * dy * db * i5 + pb * dy * i3);
    gz = mj * (bz * i3 - Real(3) * dz * db * i5 + pb * dz * i3);
    dm = db * i3 - pb * i1;
}

template <typename Real, bool QUAD, bool SOFT>
__global__ void __launch_bounds__(kAdjWarps * 32) k_force_vjp(const AdjArgs A) {
    using V4 = typename AdjVec<Real>::V4;
    using V2 = typename AdjVec<Real>::V2;
    __shared__ V4 s_tp[kAdjWarps][kAdjMaxTargets];   // target position + mass
    __shared__ V4 s_tc[kAdjWarps][kAdjMaxTargets];   // target cotangent
    __shared__ uint32_t s_buf[kAdjWarps][32 + 32 * kMaxLeafSmall];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int next = (lane + 1) & 31;
    const int64_t g = (int64_t)blockIdx.x * kAdjWarps + w;
    if (g >= A.ngroups) return;
    const V4 *spos = reinterpret_cast<const V4 *>(A.spos);
    const V4 *cot = reinterpret_cast<const V4 *>(A.cot);
    const V4 *momA = reinterpret_cast<const V4 *>(A.mom_a);
    const V4 *momB = reinterpret_cast<const V4 *>(A.mom_b);
    const V2 *momC = reinterpret_cast<const V2 *>(A.mom_c);
    const Real eps2 = (Real)A.eps2;
    const uint32_t s0 = A.gfirst[g];
    const int cnt = (int)(A.gfirst[g + 1] - s0);
    for (int t = lane; t < cnt; t += 32) {
        s_tp[w][t] = spos[s0 + t];
        s_tc[w][t] = cot[s0 + t];
    }
    __syncwarp();
    double xt[2][3] = {{0, 0, 0}, {0, 0, 0}};

    // Every pair of a tile is evaluated once.  Lane l holds source l (a cell
    // or a particle) and, at step k, meets target (l + k) mod 32 of the
    // current half of the group: the source-side sums stay in the lane, the
    // target-side partial sums travel with their target (one shuffle per step
    // passes each to the lane that meets it next; after 32 steps a final
    // shuffle brings target l's total to lane l).

    // ---- far cells ----
    const int64_t pc0 = A.list_off[g], pc1 = A.list_off[g + 1];
    for (int64_t base = pc0; base < pc1; base += 32) {
        const int nt = (int)min((int64_t)32, pc1 - base);
        uint32_t cid = 0;
        V4 ca{};
        Real cq[6] = {0, 0, 0, 0, 0, 0};
        if (lane < nt) {
            cid = (uint32_t)A.pc_list[base + lane];
            ca = momA[cid];
            if (QUAD) {
                const V4 b = momB[cid];
                const V2 cc = momC[cid];
                const Real qs = sizeof(Real) == 4 ? Real(-1) : Real(1);  // FP32 walk copies hold -Q
                cq[0] = qs * b.x; cq[1] = qs * b.y; cq[2] = qs * b.z;
                cq[3] = qs * b.w; cq[4] = qs * cc.x; cq[5] = qs * cc.y;
            }
        }
        // the group's (at most 64) targets are summed in the working precision;
        // the per-group totals go to the FP64 accumulators
        Real acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (32 * h >= cnt) break;
            const int ch = min(32, cnt - 32 * h);
            Real tx = 0, ty = 0, tz = 0;
            for (int k = 0; k < 32; ++k) {
                if (k > 0) {
                    tx = __shfl_sync(0xffffffffu, tx, next);
                    ty = __shfl_sync(0xffffffffu, ty, next);
                    tz = __shfl_sync(0xffffffffu, tz, next);
                }
                const int t = (lane + k) & 31;
                if (lane < nt && t < ch) {
                    const V4 p = s_tp[w][32 * h + t];
                    const V4 b = s_tc[w][32 * h + t];
                    Real gx, gy, gz, mb, qb[6];
                    pc_vjp<Real, QUAD, SOFT>(p.x - ca.x, p.y - ca.y, p.z - ca.z, b.x, b.y, b.z, b.w, ca.w, cq, eps2, gx,
                                       gy, gz, mb, qb);
                    tx += gx; ty += gy; tz += gz;
                    acc[0] += mb;
                    acc[1] -= gx; acc[2] -= gy; acc[3] -= gz;
#pragma unroll
                    for (int q = 0; q < 6; ++q) acc[4 + q] += qb[q];
                }
            }
            tx = __shfl_sync(0xffffffffu, tx, next);
            ty = __shfl_sync(0xffffffffu, ty, next);
            tz = __shfl_sync(0xffffffffu, tz, next);
            if (lane < ch) { xt[h][0] += (double)tx; xt[h][1] += (double)ty; xt[h][2] += (double)tz; }
        }
        if (lane < nt) {
#pragma unroll
            for (int q = 0; q < (QUAD ? 10 : 4); ++q)
                if (acc[q] != Real(0)) atomicAdd(A.ccot + (int64_t)q * A.cap + cid, A.G * (double)acc[q]);
        }
    }

    // ---- near leaves: expand particles into the buffer, tiles of 32 ----
    const int64_t pp0 = A.list_off[A.ngroups + 1 + g], pp1 = A.list_off[A.ngroups + 1 + g + 1];
    auto pp_tile = [&](const uint32_t *src, int nt) {
        uint32_t sj = 0;
        V4 sa{};
        if (lane < nt) {
            sj = src[lane];
            sa = spos[sj];
        }
        __syncwarp();
        Real gxs = 0, gys = 0, gzs = 0, dms = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (32 * h >= cnt) break;
            const int ch = min(32, cnt - 32 * h);
            Real tx = 0, ty = 0, tz = 0;
            for (int k = 0; k < 32; ++k) {
                if (k > 0) {
                    tx = __shfl_sync(0xffffffffu, tx, next);
                    ty = __shfl_sync(0xffffffffu, ty, next);
                    tz = __shfl_sync(0xffffffffu, tz, next);
                }
                const int t = (lane + k) & 31;
                // the self pair is excluded by index
                if (lane < nt && t < ch && s0 + (uint32_t)(32 * h + t) != sj) {
                    const V4 p = s_tp[w][32 * h + t];
                    const V4 b = s_tc[w][32 * h + t];
                    Real gx, gy, gz, dm;
                    pp_vjp<Real, SOFT>(sa.x - p.x, sa.y - p.y, sa.z - p.z, b.x, b.y, b.z, b.w, sa.w, eps2, gx, gy, gz,
                                 dm);
                    tx -= gx; ty -= gy; tz -= gz;
                    gxs += gx; gys += gy; gzs += gz; dms += dm;
                }
            }
            tx = __shfl_sync(0xffffffffu, tx, next);
            ty = __shfl_sync(0xffffffffu, ty, next);
            tz = __shfl_sync(0xffffffffu, tz, next);
            if (lane < ch) { xt[h][0] += (double)tx; xt[h][1] += (double)ty; xt[h][2] += (double)tz; }
        }
        if (lane < nt) {
            atomicAdd(A.xg + sj, A.G * (double)gxs);
            atomicAdd(A.xg + A.n + sj, A.G * (double)gys);
            atomicAdd(A.xg + 2 * A.n + sj, A.G * (double)gzs);
            atomicAdd(A.mg + sj, A.G * (double)dms);
        }
        __syncwarp();
    };
    uint32_t *buf = s_buf[w];
    int nb = 0;
    for (int64_t base = pp0; base < pp1; base += 32) {
        const int nl = (int)min((int64_t)32, pp1 - base);
        uint2 lk = make_uint2(0, 0);
        if (lane < nl) lk = A.nlink[(uint32_t)A.pp_list[base + lane]];
        const bool big = lk.y > (uint32_t)kMaxLeafSmall;
        const uint32_t sc = big ? 0u : lk.y;
        uint32_t incl = sc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t c = 0; c < sc; ++c) buf[nb + (incl - sc) + c] = lk.x + c;
        nb += (int)tot;
        __syncwarp();
        uint32_t bm = __ballot_sync(0xffffffffu, big);
        while (bm) {
            const int b = __ffs(bm) - 1;
            bm &= bm - 1;
            const uint32_t f = __shfl_sync(0xffffffffu, lk.x, b), c = __shfl_sync(0xffffffffu, lk.y, b);
            for (uint32_t o = 0; o < c; o += 32) {
                const int k = (int)min(32u, c - o);
                __shared__ uint32_t s_rng[kAdjWarps][32];
                if (lane < k) s_rng[w][lane] = f + o + lane;
                __syncwarp();
                pp_tile(s_rng[w], k);
            }
        }
        int done = 0;
        while (nb - done >= 32) {
            pp_tile(buf + done, 32);
            done += 32;
        }
        const int r = nb - done;
        const uint32_t keep = lane < r ? buf[done + lane] : 0u;
        __syncwarp();
        if (lane < r) buf[lane] = keep;
        __syncwarp();
        nb = r;
    }
    if (nb > 0) pp_tile(buf, nb);

    for (int tt = 0; tt < 2; ++tt) {
        const int t = lane + 32 * tt;
        if (t < cnt) {
            A.xt[s0 + t] = A.G * xt[tt][0];
            A.xt[A.n + s0 + t] = A.G * xt[tt][1];
            A.xt[2 * A.n + s0 + t] = A.G * xt[tt][2];
        }
    }
}

// Cotangents (abar, phibar) from the caller's order into key order.
template <typename Real>
__global__ void __launch_bounds__(256) k_cot_gather(const Real *__restrict__ abar, const Real *__restrict__ phibar,
                                                    const uint32_t *__restrict__ perm, int64_t n,
                                                    typename AdjVec<Real>::V4 *__restrict__ cot,
                                                    const uint32_t *__restrict__ ctr) {
    if (aborted(ctr, kStageAfter)) return;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = perm[s];
        typename AdjVec<Real>::V4 c;
        c.x = abar[i]; c.y = abar[n + i]; c.z = abar[2 * n + i];
        c.w = phibar ? phibar[i] : Real(0);
        cot[s] = c;
    }
}

// Level L of the top-down cotangent push (see the header comment).
template <typename Real>
__global__ void __launch_bounds__(256) k_cot_push(int L, const uint32_t *__restrict__ ctr,
                                                  const uint4 *__restrict__ ngeo, const uint2 *__restrict__ nlink,
                                                  const double *__restrict__ mom64, int64_t cap,
                                                  const typename AdjVec<Real>::V4 *__restrict__ spos,
                                                  double *__restrict__ ccot, double *__restrict__ xg,
                                                  double *__restrict__ mg, int64_t n) {
    if (aborted(ctr, kStageAfter)) return;
    const uint32_t start = ctr[kCtrLevelStart + L], end = ctr[kCtrLevelStart + L + 1];
    for (uint32_t node = start + blockIdx.x * blockDim.x + threadIdx.x; node < end;
         node += gridDim.x * blockDim.x) {
        double cb[10];
        bool nz = false;
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            cb[k] = ccot[(int64_t)k * cap + node];
            nz |= cb[k] != 0.0;
        }
        if (!nz) continue;
        const uint4 geo = ngeo[node];
        const uint2 lk = nlink[node];
        const bool leaf = (geo.w >> 8) & 1u;
        const double M = mom64[node];
        const double Rx = mom64[cap + node], Ry = mom64[2 * cap + node], Rz = mom64[3 * cap + node];
        const double fxx = cb[4], fyy = cb[5], fzz = cb[6];
        const double fxy = 0.5 * cb[7], fxz = 0.5 * cb[8], fyz = 0.5 * cb[9];
        const double tr = fxx + fyy + fzz;
        const bool massive = M != 0.0;
        const double iM = massive ? 1.0 / M : 0.0;
        for (uint32_t k = lk.x; k < lk.x + lk.y; ++k) {
            double mk, dx, dy, dz;
            if (leaf) {
                const typename AdjVec<Real>::V4 p = spos[k];
                mk = (double)p.w;
                dx = (double)p.x - Rx; dy = (double)p.y - Ry; dz = (double)p.z - Rz;
            } else {
                mk = mom64[k];
                dx = mom64[cap + k] - Rx; dy = mom64[2 * cap + k] - Ry; dz = mom64[3 * cap + k] - Rz;
            }
            double dM = cb[0], gx = 0, gy = 0, gz = 0;
            if (massive) {
                const double Fx = fxx * dx + fxy * dy + fxz * dz;
                const double Fy = fxy * dx + fyy * dy + fyz * dz;
                const double Fz = fxz * dx + fyz * dy + fzz * dz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                dM += (dx * cb[1] + dy * cb[2] + dz * cb[3]) * iM + 3.0 * (dx * Fx + dy * Fy + dz * Fz) - d2 * tr;
                const double wgt = mk * iM;
                gx = wgt * cb[1] + mk * (6.0 * Fx - 2.0 * tr * dx);
                gy = wgt * cb[2] + mk * (6.0 * Fy - 2.0 * tr * dy);
                gz = wgt * cb[3] + mk * (6.0 * Fz - 2.0 * tr * dz);
            }
            if (leaf) {
                mg[k] += dM;
                xg[k] += gx; xg[n + k] += gy; xg[2 * n + k] += gz;
            } else {
                ccot[k] += dM;
                ccot[cap + k] += gx; ccot[2 * cap + k] += gy; ccot[3 * cap + k] += gz;
                if (massive)
                    for (int q = 0; q < 6; ++q) ccot[(int64_t)(4 + q) * cap + k] += cb[4 + q];
            }
        }
    }
}

// xbar[i] += xt + xg, mbar[i] += mg (key order -> caller order)
template <typename Real>
__global__ void __launch_bounds__(256) k_grad_scatter(const double *__restrict__ xt, const double *__restrict__ xg,
                                                      const double *__restrict__ mg, const uint32_t *__restrict__ perm,
                                                      int64_t n, Real *__restrict__ xbar, Real *__restrict__ mbar,
                                                      const uint32_t *__restrict__ ctr) {
    if (aborted(ctr, kStageAfter)) return;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = perm[s];
        if (xbar) {
            xbar[i] += (Real)(xt[s] + xg[s]);
            xbar[n + i] += (Real)(xt[n + s] + xg[n + s]);
            xbar[2 * n + i] += (Real)(xt[2 * n + s] + xg[2 * n + s]);
        }
        if (mbar) mbar[i] += (Real)mg[s];
    }
}

template <typename Real>
static cudaError_t adjoint_impl(TreeWorkspace *ws, const void *abar, const void *phibar, void *xbar, void *mbar,
                                cudaStream_t s) {
    const int64_t n = ws->n, cap = ws->node_cap;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ws->adj_xg, 0, 3 * n * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws->adj_mg, 0, n * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws->adj_ccot, 0, 10 * cap * sizeof(double), s)) != cudaSuccess) return e;
    const int nb = grid_for(n, 256, 152 * 8);
    k_cot_gather<Real><<<nb, 256, 0, s>>>((const Real *)abar, (const Real *)phibar, ws->idx, n,
                                          (typename AdjVec<Real>::V4 *)ws->adj_cot, ws->ctr);
    AdjArgs A;
    A.n = n;
    A.ngroups = ws->list_groups;
    A.gfirst = ws->gfirst;
    A.spos = ws->spos;
    A.cot = ws->adj_cot;
    A.nlink = ws->nlink;
    A.mom_a = ws->mom_a; A.mom_b = ws->mom_b; A.mom_c = ws->mom_c;
    A.list_off = ws->list_cnt;
    A.pc_list = ws->pc_list; A.pp_list = ws->pp_list;
    A.G = ws->p.G;
    A.eps2 = ws->p.eps * ws->p.eps;
    A.xt = ws->adj_xt; A.xg = ws->adj_xg; A.mg = ws->adj_mg; A.ccot = ws->adj_ccot;
    A.cap = cap;
    const unsigned gb = (unsigned)((A.ngroups + kAdjWarps - 1) / kAdjWarps);
    if (A.ngroups > 0) {
        const bool quad = ws->p.order == 2;
        bool done = false;
        if constexpr (sizeof(Real) == 4) {
            if ((float)(ws->p.eps * ws->p.eps) >= FLT_MIN) {  // softened FP32 pairs (inv_r)
                if (quad) k_force_vjp<Real, true, true><<<gb, kAdjWarps * 32, 0, s>>>(A);
                else k_force_vjp<Real, false, true><<<gb, kAdjWarps * 32, 0, s>>>(A);
                done = true;
            }
        }
        if (!done) {
            if (quad) k_force_vjp<Real, true, false><<<gb, kAdjWarps * 32, 0, s>>>(A);
            else k_force_vjp<Real, false, false><<<gb, kAdjWarps * 32, 0, s>>>(A);
        }
    }
    const int nbn = grid_for(ws->node_cap, 256, 152 * 8);
    for (int L = 0; L < kLevels; ++L)
        k_cot_push<Real><<<nbn, 256, 0, s>>>(L, ws->ctr, ws->ngeo, ws->nlink, ws->mom64, cap,
                                             (const typename AdjVec<Real>::V4 *)ws->spos, ws->adj_ccot, ws->adj_xg,
                                             ws->adj_mg, n);
    k_grad_scatter<Real><<<nb, 256, 0, s>>>(ws->adj_xt, ws->adj_xg, ws->adj_mg, ws->idx, n, (Real *)xbar,
                                            (Real *)mbar, ws->ctr);
    ws->launches += 3 + kLevels;
    return cudaGetLastError();
}

// One reverse step of Eqs. 2-5 (see leapfrog_adjoint_step in treegb.h).
template <typename Real>
__global__ void __launch_bounds__(256) k_adj_kick(Real *__restrict__ abar, const Real *__restrict__ vbar, Real h,
                                                  int64_t n3) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
        abar[i] += h * vbar[i];
}
template <typename Real>
__global__ void __launch_bounds__(256) k_adj_drift(Real *__restrict__ abar, Real *__restrict__ vbar,
                                                   const Real *__restrict__ xbar, Real h, Real tau, int64_t n3) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const Real vb = vbar[i] + tau * xbar[i];
        vbar[i] = vb;
        abar[i] = h * vb;
    }
}

template <typename Real>
static cudaError_t adjoint_step_impl(TreeWorkspace *ws, Real *xbar, Real *vbar, Real *abar, Real *mbar,
                                     const Real *phibar, double tau, cudaStream_t s) {
    const int64_t n3 = 3 * ws->n;
    const int nb = grid_for(n3, 256, 152 * 8);
    k_adj_kick<Real><<<nb, 256, 0, s>>>(abar, vbar, (Real)(0.5 * tau), n3);
    cudaError_t e = adjoint_impl<Real>(ws, abar, phibar, xbar, mbar, s);
    if (e != cudaSuccess) return e;
    k_adj_drift<Real><<<nb, 256, 0, s>>>(abar, vbar, xbar, (Real)(0.5 * tau), (Real)tau, n3);
    ws->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(TreeWorkspace *ws, void *xbar, void *vbar, void *abar, void *mbar,
                                const void *phibar, double tau, cudaStream_t s) {
    if (ws->p.precision == TREE_F64)
        return adjoint_step_impl<double>(ws, (double *)xbar, (double *)vbar, (double *)abar, (double *)mbar,
                                         (const double *)phibar, tau, s);
    return adjoint_step_impl<float>(ws, (float *)xbar, (float *)vbar, (float *)abar, (float *)mbar,
                                    (const float *)phibar, tau, s);
}

// Cotangents of W = 1/2 sum m phi (tree_energy_vjp): phi_bar = w_bar m / 2,
// m_bar += w_bar phi / 2.
template <typename Real>
__global__ void __launch_bounds__(256) k_energy_vjp(const Real *__restrict__ m, const Real *__restrict__ phi,
                                                    const double *__restrict__ wbar, int64_t n,
                                                    Real *__restrict__ phibar, Real *__restrict__ mbar) {
    const Real h = (Real)(0.5 * wbar[0]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (phibar) phibar[i] = h * m[i];
        if (mbar) mbar[i] += h * phi[i];
    }
}

cudaError_t launch_energy_vjp(TreeWorkspace *ws, const void *m, const void *phi, const double *wbar, int64_t n,
                              void *phibar, void *mbar, cudaStream_t s) {
    const int nb = grid_for(n, 256, 152 * 8);
    if (ws->p.precision == TREE_F64)
        k_energy_vjp<double><<<nb, 256, 0, s>>>((const double *)m, (const double *)phi, wbar, n, (double *)phibar,
                                                (double *)mbar);
    else
        k_energy_vjp<float><<<nb, 256, 0, s>>>((const float *)m, (const float *)phi, wbar, n, (float *)phibar,
                                               (float *)mbar);
    ws->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_adjoint(TreeWorkspace *ws, const void *abar, const void *phibar, void *xbar, void *mbar,
                           cudaStream_t s) {
    if (ws->p.precision == TREE_F64) return adjoint_impl<double>(ws, abar, phibar, xbar, mbar, s);
    return adjoint_impl<float>(ws, abar, phibar, xbar, mbar, s);
}

}  // namespace treegb
