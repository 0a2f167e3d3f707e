// walk.cuh -- the tree walk and force evaluation (Sec. 2 TreeCode; Eq. 1 for
// the near part), one warp per group of Gs key-ordered particles.
//
// Traversal (per warp, depth first, stack in shared memory):
//   the stack holds ranges of sibling nodes (children are contiguous in the
//   breadth-first numbering), one entry per opened cell.  Each step pops up
//   to 32 nodes from the top ranges (splitting the last one if needed), one
//   node per lane, and tests each against the group box with the integer
//   opening criterion d2 >= D[level] (D from tree_mac_table): far nodes go
//   to the PC buffer, near leaves' particles to the PP buffer, near internal
//   nodes push their child range.  Compaction uses warp ballots and scans.
// Evaluation: whenever a buffer holds 32 entries, the warp stages the 32
//   sources (float4 position+mass, or the cell's mass, COM and quadrupole)
//   in shared memory and every lane applies all 32 to its own target(s)
//   (each source is a broadcast shared-memory read; the arithmetic is plain
//   FP32 FMA plus one rsqrt per pair).  Per-tile partial sums are folded into
//   the running sums with Kahan compensation.
// The self pair i = j is excluded by index: a tile of near particles that
// holds some of the group's own particles is evaluated with the mass of each
// lane's own particle set to zero (removing -m_i/eps afterwards instead would
// cancel in FP32 against a potential that can be far smaller than m_i/eps);
// with eps = 0 a guarded variant also skips other r = 0 pairs.
#pragma once

#include "common.cuh"

namespace treegb {

constexpr int kWalkWarps = 4;                      // warps per block
constexpr int kPPCap = 32 + 32 * kMaxLeafSmall;    // PP buffer entries per warp
constexpr int kPCCap = 32 + 32 * 8;                // PC buffer entries per warp (a step adds <= 32 x 8)

struct WalkArgs {
    int64_t n;
    int32_t gs;
    int64_t ngroups;
    const void *spos;
    const uint64_t *skey;
    const uint32_t *perm;
    const uint4 *ngeo;
    const uint2 *nlink;
    const void *mom_a, *mom_b, *mom_c;
    const int64_t *dmac;
    double G, eps, eps2;
    void *a, *phi, *v;
    double half_tau;
    void *v2, *phi2;      // mirrors of the kicked v and of phi, or NULL
    int32_t stack_depth;
    uint4 *gstat;          // per group: {n_pc cells, n_pp particles, max stack, n_pp leaves}
    int32_t *dstatus;
    const int64_t *list_off;  // [2][ngroups+1] (emit mode)
    int32_t *pc_list, *pp_list;
    const uint32_t *order;    // processing order of the groups (widest boxes first), or NULL
    const uint32_t *gfirst;   // group g = sorted particles [gfirst[g], gfirst[g+1])
    uint32_t *ctr;            // counter block: group count and the walk's group ticket
    const int64_t *seg_off;   // segment offsets (nseg > 1): a group walks its own segment's tree
    int64_t nseg;
    const DevBox *box;        // per segment: the tree's cube (side 2^k)
};

template <typename Real> __device__ __forceinline__ Real rsqrt_r(Real x);
template <> __device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_r<double>(double x) { return rsqrt(x); }

// Source staging per warp: FP32 uses 16 source pairs x 5 float4 (pair-
// interleaved, see pp_pair / pc_pair); FP64 uses 32 x (double4, double4, double2).
template <typename Real>
__host__ __device__ constexpr size_t walk_stage_bytes() {
    return sizeof(Real) == 4 ? 80 * sizeof(float4)
                             : 32 * (sizeof(typename Vec4<Real>::T) * 2 + sizeof(typename Vec2<Real>::T));
}

// Per-warp shared-memory slice, rounded up to 32 bytes so that every warp's
// staging arrays (float4 / 32-byte double4) stay aligned.
template <typename Real>
__host__ __device__ constexpr size_t walk_warp_bytes(int stack_depth) {
    return (((size_t)(stack_depth + kPPCap + kPCCap + 32) * 4 + walk_stage_bytes<Real>()) + 31) & ~(size_t)31;
}

// --- pair terms ------------------------------------------------------------
// PP: source s = (x, y, z, m); d = r_s - r_i; accumulates m d / r^3 and -m / r.
template <typename Real, bool SOFT>
__device__ __forceinline__ void pp_term(Real px, Real py, Real pz, const typename Vec4<Real>::T &s,
                                        Real eps2, Real (&acc)[4]) {
    const Real dx = s.x - px, dy = s.y - py, dz = s.z - pz;
    const Real r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    Real rinv = rsqrt_r<Real>(r2);
    if (!SOFT) rinv = r2 > Real(0) ? rinv : Real(0);
    const Real mr = s.w * rinv;
    const Real mr3 = mr * (rinv * rinv);
    acc[0] = fma(mr3, dx, acc[0]);
    acc[1] = fma(mr3, dy, acc[1]);
    acc[2] = fma(mr3, dz, acc[2]);
    acc[3] -= mr;
}

// PC: y = r_i - R, r_s^2 = |y|^2 + eps^2;
//   a += -M y / r_s^3 + Q y / r_s^5 - 5/2 (y.Q.y) y / r_s^7
//   phi += -M / r_s - 1/2 (y.Q.y) / r_s^5
// A = (Rx, Ry, Rz, M), B = (Qxx, Qyy, Qzz, Qxy), C = (Qxz, Qyz).
template <typename Real, bool QUAD, bool SOFT>
__device__ __forceinline__ void pc_term(Real px, Real py, Real pz, const typename Vec4<Real>::T &A,
                                        const typename Vec4<Real>::T &B, const typename Vec2<Real>::T &C,
                                        Real eps2, Real (&acc)[4]) {
    const Real yx = px - A.x, yy = py - A.y, yz = pz - A.z;
    const Real r2 = fma(yx, yx, fma(yy, yy, fma(yz, yz, eps2)));
    Real rinv = rsqrt_r<Real>(r2);
    if (!SOFT) rinv = r2 > Real(0) ? rinv : Real(0);
    const Real rinv2 = rinv * rinv;
    const Real Mr = A.w * rinv;
    const Real Mr3 = Mr * rinv2;
    if (QUAD) {
        const Real Qx = fma(B.x, yx, fma(B.w, yy, C.x * yz));
        const Real Qy = fma(B.w, yx, fma(B.y, yy, C.y * yz));
        const Real Qz = fma(C.x, yx, fma(C.y, yy, B.z * yz));
        const Real yQy = fma(yx, Qx, fma(yy, Qy, yz * Qz));
        const Real r3 = rinv * rinv2;
        const Real r5 = r3 * rinv2;
        const Real qr5 = yQy * r5;
        const Real c = fma(Real(-2.5) * qr5, rinv2, -Mr3);
        acc[0] = fma(c, yx, fma(r5, Qx, acc[0]));
        acc[1] = fma(c, yy, fma(r5, Qy, acc[1]));
        acc[2] = fma(c, yz, fma(r5, Qz, acc[2]));
        acc[3] -= fma(Real(0.5), qr5, Mr);
    } else {
        acc[0] = fma(-Mr3, yx, acc[0]);
        acc[1] = fma(-Mr3, yy, acc[1]);
        acc[2] = fma(-Mr3, yz, acc[2]);
        acc[3] -= Mr;
    }
}

// --- packed FP32 pair terms: two sources per instruction ---------------------
// 1/r for two pairs.  Softened (SOFT): r^2 >= eps^2, and the FP32 walk takes
// this variant only when eps^2 is a normal FP32 number, so r^2 is never
// subnormal and the PTX approximate reciprocal square root with subnormal
// inputs flushed (rsqrt.approx.ftz.f32) serves; for normal inputs it gave the
// same bits as rsqrtf on sm_103a over a sweep of all normal exponents, and it
// saves rsqrtf's handling of subnormal inputs (the far-cell loop ran 6.6 %
// faster).  Unsoftened: rsqrtf, and a coincident pair (r^2 = 0) contributes
// nothing.
template <bool SOFT>
__device__ __forceinline__ float2 rsqrt_pair(float2 r2) {
    float2 ri;
    if (SOFT) {
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ri.x) : "f"(r2.x));
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ri.y) : "f"(r2.y));
    } else {
        ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        ri.x = r2.x > 0.f ? ri.x : 0.f;
        ri.y = r2.y > 0.f ? ri.y : 0.f;
    }
    return ri;
}

// Each float2 holds one quantity of two sources (or two cells); the target is
// held negated and duplicated, nP = (-p, -p), so every difference is an add.
// PP: d = r_s - r_i, accumulates m d / r^3 and -m / r for both sources.
template <bool SOFT>
__device__ __forceinline__ void pp_pair(float2 nx, float2 ny, float2 nz, float2 X, float2 Y, float2 Z, float2 M,
                                        float2 eps2, float2 neg1, float2 (&acc)[4]) {
    const float2 dx = __fadd2_rn(X, nx), dy = __fadd2_rn(Y, ny), dz = __fadd2_rn(Z, nz);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
    const float2 ri = rsqrt_pair<SOFT>(r2);
    const float2 ri2 = __fmul2_rn(ri, ri);
    const float2 mr = __fmul2_rn(M, ri);
    const float2 mr3 = __fmul2_rn(mr, ri2);
    acc[0] = __ffma2_rn(mr3, dx, acc[0]);
    acc[1] = __ffma2_rn(mr3, dy, acc[1]);
    acc[2] = __ffma2_rn(mr3, dz, acc[2]);
    acc[3] = __ffma2_rn(neg1, mr, acc[3]);
}

// PC for two cells.  With u = R - r_i (= -y) and the negated quadrupole
// Qn = -Q (the FP32 cell copies store -Q), w = Qn u equals Q y, u.w = -(y.Q.y), and the terms of
// pc_term become a = [M/r^3 - 5/2 (u.w)/r^7] u + w/r^5, phi = -M/r + 1/2 (u.w)/r^5.
// R5 (quadrupole only) takes r^-5 out of the acceleration, a = r^-5 (k u + w) with
// k = M r^2 - 5/2 (u.w)/r^2, and accumulates -phi = [M - 1/2 (u.w)/r^4] / r in acc[3]
// (neg1 must then hold -1/2): 33 packed operations for two cells instead of 34.  It forms
// r^-5 and M r^2 u, so the walk takes it only where pc_r5_fits holds.
template <bool QUAD, bool SOFT, bool R5 = false>
__device__ __forceinline__ void pc_pair(float2 nx, float2 ny, float2 nz, const float4 &A, const float4 &B,
                                        const float4 &C, const float4 &D, const float4 &E, float2 eps2,
                                        float2 neg1, float2 half, float2 m25, float2 (&acc)[4]) {
    const float2 ux = __fadd2_rn(make_float2(A.x, A.y), nx);
    const float2 uy = __fadd2_rn(make_float2(A.z, A.w), ny);
    const float2 uz = __fadd2_rn(make_float2(B.x, B.y), nz);
    const float2 M = make_float2(B.z, B.w);
    const float2 r2 = __ffma2_rn(ux, ux, __ffma2_rn(uy, uy, __ffma2_rn(uz, uz, eps2)));
    const float2 ri = rsqrt_pair<SOFT>(r2);
    const float2 ri2 = __fmul2_rn(ri, ri);
    const float2 Mr = __fmul2_rn(M, ri);
    const float2 Mr3 = __fmul2_rn(Mr, ri2);
    if (QUAD) {
        const float2 qxx = make_float2(C.x, C.y), qyy = make_float2(C.z, C.w);
        const float2 qzz = make_float2(D.x, D.y), qxy = make_float2(D.z, D.w);
        const float2 qxz = make_float2(E.x, E.y), qyz = make_float2(E.z, E.w);
        const float2 wx = __ffma2_rn(qxx, ux, __ffma2_rn(qxy, uy, __fmul2_rn(qxz, uz)));
        const float2 wy = __ffma2_rn(qxy, ux, __ffma2_rn(qyy, uy, __fmul2_rn(qyz, uz)));
        const float2 wz = __ffma2_rn(qxz, ux, __ffma2_rn(qyz, uy, __fmul2_rn(qzz, uz)));
        const float2 uw = __ffma2_rn(ux, wx, __ffma2_rn(uy, wy, __fmul2_rn(uz, wz)));
        if (R5) {
            const float2 ri4 = __fmul2_rn(ri2, ri2);
            const float2 r5 = __fmul2_rn(ri4, ri);
            const float2 k = __ffma2_rn(m25, __fmul2_rn(uw, ri2), __fmul2_rn(M, r2));
            acc[0] = __ffma2_rn(r5, __ffma2_rn(k, ux, wx), acc[0]);
            acc[1] = __ffma2_rn(r5, __ffma2_rn(k, uy, wy), acc[1]);
            acc[2] = __ffma2_rn(r5, __ffma2_rn(k, uz, wz), acc[2]);
            acc[3] = __ffma2_rn(ri, __ffma2_rn(uw, __fmul2_rn(ri4, neg1), M), acc[3]);
        } else {
            const float2 r3 = __fmul2_rn(ri, ri2);
            const float2 r5 = __fmul2_rn(r3, ri2);
            const float2 t = __fmul2_rn(uw, r5);
            const float2 c = __ffma2_rn(t, __fmul2_rn(ri2, m25), Mr3);
            acc[0] = __ffma2_rn(c, ux, __ffma2_rn(r5, wx, acc[0]));
            acc[1] = __ffma2_rn(c, uy, __ffma2_rn(r5, wy, acc[1]));
            acc[2] = __ffma2_rn(c, uz, __ffma2_rn(r5, wz, acc[2]));
            acc[3] = __ffma2_rn(neg1, Mr, __ffma2_rn(half, t, acc[3]));
        }
    } else {
        acc[0] = __ffma2_rn(Mr3, ux, acc[0]);
        acc[1] = __ffma2_rn(Mr3, uy, acc[1]);
        acc[2] = __ffma2_rn(Mr3, uz, acc[2]);
        acc[3] = __ffma2_rn(neg1, Mr, acc[3]);
    }
}

template <typename Real, bool KAHAN>
__device__ __forceinline__ void fold(Real (&sum)[4], Real (&cmp)[4], const Real (&part)[4]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (KAHAN) {
            const Real y = part[c] - cmp[c];
            const Real t = sum[c] + y;
            cmp[c] = (t - sum[c]) - y;
            sum[c] = t;
        } else {
            sum[c] += part[c];
        }
    }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

template <typename Real, int TPL, bool QUAD, bool KAHAN, bool SOFT, int MODE>
__global__ void __launch_bounds__(kWalkWarps * 32, TPL == 2 ? 4 : sizeof(Real) == 4 ? 6 : 5) k_walk(const WalkArgs A) {
    using V4 = typename Vec4<Real>::T;
    using V2 = typename Vec2<Real>::T;
    extern __shared__ __align__(32) unsigned char smem[];
    __shared__ long long sD[kLevels];
    if (aborted(A.ctr, kStageAfter)) return;  // the build gave up a wait: no valid tree
    if (threadIdx.x < kLevels) sD[threadIdx.x] = A.dmac[threadIdx.x];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int SD = A.stack_depth;
    unsigned char *wb = smem + (size_t)warp * walk_warp_bytes<Real>(SD);
    V4 *stA = reinterpret_cast<V4 *>(wb);            // FP64 layout
    V4 *stB = stA + 32;
    V2 *stC = reinterpret_cast<V2 *>(stB + 32);
    float4 *stF = reinterpret_cast<float4 *>(wb);    // FP32 pair-interleaved layout
    uint32_t *stack = reinterpret_cast<uint32_t *>(wb + walk_stage_bytes<Real>());
    uint32_t *ppbuf = stack + SD;
    uint32_t *pcbuf = ppbuf + kPPCap;
    uint32_t *sidx = pcbuf + kPCCap;  // sorted index of each staged near source
    const uint32_t lt = lanemask_lt();

    const V4 *__restrict__ spos = reinterpret_cast<const V4 *>(A.spos);
    const V4 *__restrict__ momA = reinterpret_cast<const V4 *>(A.mom_a);
    const V4 *__restrict__ momB = reinterpret_cast<const V4 *>(A.mom_b);
    const V2 *__restrict__ momC = reinterpret_cast<const V2 *>(A.mom_c);
    const Real eps2 = (Real)A.eps2;

    // full far-cell tiles of one-target-per-lane groups take pc_pair's R5 form
    // where it fits the segment's cube (flag set per segment after the moments)
    constexpr bool kR5 = sizeof(Real) == 4 && QUAD && TPL == 1;

    // persistent warps: each takes the next group slot until all are done
    const uint32_t ngroups = A.ctr[kCtrGroups];
    for (;;) {
    uint32_t slot = 0;
    if (lane == 0) slot = atomicAdd(A.ctr + kCtrWalkTicket, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= ngroups) break;
    const int64_t g = A.order ? (int64_t)A.order[slot] : (int64_t)slot;
    const int64_t s0 = A.gfirst[g];
    const int cnt = (int)(A.gfirst[g + 1] - A.gfirst[g]);
    // the group's segment b (its tree's root is node b)
    const uint32_t gseg = A.nseg > 1 ? seg_find(A.seg_off, A.nseg, s0) : 0u;

    // targets and the group's integer box
    Real px[TPL], py[TPL], pz[TPL], pm[TPL];
    uint32_t lo0 = 0xffffffffu, lo1 = 0xffffffffu, lo2 = 0xffffffffu, hi0 = 0, hi1 = 0, hi2 = 0;
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int li = lane + 32 * t;
        px[t] = py[t] = pz[t] = pm[t] = Real(0);
        if (li < cnt) {
            const V4 p = spos[s0 + li];
            px[t] = p.x; py[t] = p.y; pz[t] = p.z; pm[t] = p.w;
            const uint64_t k = A.skey[s0 + li];
            const uint32_t qx = compact3(k >> 2), qy = compact3(k >> 1), qz = compact3(k);
            lo0 = min(lo0, qx); lo1 = min(lo1, qy); lo2 = min(lo2, qz);
            hi0 = max(hi0, qx); hi1 = max(hi1, qy); hi2 = max(hi2, qz);
        }
    }
    const int glo0 = (int)__reduce_min_sync(0xffffffffu, lo0), glo1 = (int)__reduce_min_sync(0xffffffffu, lo1),
              glo2 = (int)__reduce_min_sync(0xffffffffu, lo2);
    const int ghi0 = (int)__reduce_max_sync(0xffffffffu, hi0) + 1, ghi1 = (int)__reduce_max_sync(0xffffffffu, hi1) + 1,
              ghi2 = (int)__reduce_max_sync(0xffffffffu, hi2) + 1;

    Real sum[TPL][4], cmp[TPL][4];
#pragma unroll
    for (int t = 0; t < TPL; ++t)
#pragma unroll
        for (int c = 0; c < 4; ++c) { sum[t][c] = Real(0); cmp[t][c] = Real(0); }

    // --- evaluation helpers (whole warp) ---
    // FP32: sources are staged as pairs, pair k in stF[5k .. 5k+4]:
    //   PP: (x0, x1, y0, y1), (z0, z1, m0, m1)
    //   PC: (Rx0, Rx1, Ry0, Ry1), (Rz0, Rz1, M0, M1), -(Qxx, Qyy), -(Qzz, Qxy), -(Qxz, Qyz)
    // with an odd count padded by a massless source at the origin.
    float2 nX[TPL], nY[TPL], nZ[TPL];
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        nX[t] = make_float2(-(float)px[t], -(float)px[t]);
        nY[t] = make_float2(-(float)py[t], -(float)py[t]);
        nZ[t] = make_float2(-(float)pz[t], -(float)pz[t]);
    }
    const float2 eps2v = make_float2((float)A.eps2, (float)A.eps2);
    const float2 neg1 = make_float2(-1.f, -1.f), halfv = make_float2(0.5f, 0.5f), m25 = make_float2(-2.5f, -2.5f),
                 mhalf = make_float2(-0.5f, -0.5f);
    const bool r5 = kR5 && A.box[gseg].r5fit != 0;

    // true when some staged source is one of the group's own particles
    auto stage_pp = [&](const V4 &src, uint32_t si, int ns) -> bool {
        sidx[lane] = lane < ns ? si : 0xffffffffu;
        const bool own = __any_sync(0xffffffffu, lane < ns && si - (uint32_t)s0 < (uint32_t)cnt);
        if constexpr (sizeof(Real) == 4) {
            const int ne = (ns + 1) & ~1;
            if (lane < ne) {
                float *a = reinterpret_cast<float *>(stF + 5 * (lane >> 1));
                const int sl = lane & 1;
                const bool v = lane < ns;
                a[sl] = v ? (float)src.x : 0.f;
                a[2 + sl] = v ? (float)src.y : 0.f;
                a[4 + sl] = v ? (float)src.z : 0.f;
                a[6 + sl] = v ? (float)src.w : 0.f;
            }
        } else {
            if (lane < ns) stA[lane] = src;
        }
        return own;
    };
    auto eval_pp_stage = [&](int ns, bool own) {
        if constexpr (sizeof(Real) == 4) {
            float2 part[TPL][4];
#pragma unroll
            for (int t = 0; t < TPL; ++t)
#pragma unroll
                for (int c = 0; c < 4; ++c) part[t][c] = make_float2(0.f, 0.f);
            const int np = (ns + 1) >> 1;
            if (own) {
                // the group's own particles are in this tile: each lane drops its own index
                for (int k = 0; k < np; ++k) {
                    const float4 a = stF[5 * k], b = stF[5 * k + 1];
                    const uint32_t i0 = sidx[2 * k], i1 = sidx[2 * k + 1];
#pragma unroll
                    for (int t = 0; t < TPL; ++t) {
                        const uint32_t me = (uint32_t)s0 + (uint32_t)(lane + 32 * t);
                        const float2 mm = make_float2(i0 == me ? 0.f : b.z, i1 == me ? 0.f : b.w);
                        pp_pair<SOFT>(nX[t], nY[t], nZ[t], make_float2(a.x, a.y), make_float2(a.z, a.w),
                                      make_float2(b.x, b.y), mm, eps2v, neg1, part[t]);
                    }
                }
            } else if (np == 16) {
#pragma unroll 16
                for (int k = 0; k < 16; ++k) {
                    const float4 a = stF[5 * k], b = stF[5 * k + 1];
#pragma unroll
                    for (int t = 0; t < TPL; ++t)
                        pp_pair<SOFT>(nX[t], nY[t], nZ[t], make_float2(a.x, a.y), make_float2(a.z, a.w),
                                      make_float2(b.x, b.y), make_float2(b.z, b.w), eps2v, neg1, part[t]);
                }
            } else {
                for (int k = 0; k < np; ++k) {
                    const float4 a = stF[5 * k], b = stF[5 * k + 1];
#pragma unroll
                    for (int t = 0; t < TPL; ++t)
                        pp_pair<SOFT>(nX[t], nY[t], nZ[t], make_float2(a.x, a.y), make_float2(a.z, a.w),
                                      make_float2(b.x, b.y), make_float2(b.z, b.w), eps2v, neg1, part[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                Real p1[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) p1[c] = (Real)(part[t][c].x + part[t][c].y);
                fold<Real, KAHAN>(sum[t], cmp[t], p1);
            }
        } else {
            Real part[TPL][4];
#pragma unroll
            for (int t = 0; t < TPL; ++t)
#pragma unroll
                for (int c = 0; c < 4; ++c) part[t][c] = Real(0);
            for (int j = 0; j < ns; ++j) {
                const V4 s = stA[j];
                const uint32_t sj = sidx[j];
#pragma unroll
                for (int t = 0; t < TPL; ++t) {
                    V4 st = s;
                    if (own && sj == (uint32_t)s0 + (uint32_t)(lane + 32 * t)) st.w = Real(0);
                    pp_term<Real, SOFT>(px[t], py[t], pz[t], st, eps2, part[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < TPL; ++t) fold<Real, KAHAN>(sum[t], cmp[t], part[t]);
        }
    };
    auto eval_pp_list = [&](const uint32_t *buf, int ns) {
        V4 s{};
        uint32_t si = 0xffffffffu;
        if (lane < ns) { si = buf[lane]; s = spos[si]; }
        __syncwarp();
        const bool own = stage_pp(s, si, ns);
        __syncwarp();
        eval_pp_stage(ns, own);
        __syncwarp();
    };
    auto eval_pp_range = [&](uint32_t first, int ns) {
        V4 s{};
        if (lane < ns) s = spos[first + lane];
        __syncwarp();
        const bool own = stage_pp(s, first + (uint32_t)lane, ns);
        __syncwarp();
        eval_pp_stage(ns, own);
        __syncwarp();
    };
    auto eval_pc_list = [&](const uint32_t *buf, int ns) {
        if constexpr (sizeof(Real) == 4) {
            const int ne = (ns + 1) & ~1;
            if (lane < ne) {
                float *q = reinterpret_cast<float *>(stF + 5 * (lane >> 1));
                const int sl = lane & 1;
                V4 a{};
                V4 b{};
                V2 c{};
                if (lane < ns) {
                    const uint32_t cell = buf[lane];
                    a = momA[cell];
                    if (QUAD) { b = momB[cell]; c = momC[cell]; }
                }
                q[sl] = a.x; q[2 + sl] = a.y; q[4 + sl] = a.z; q[6 + sl] = a.w;
                if (QUAD) {  // the FP32 cell copies already hold -Q
                    q[8 + sl] = b.x; q[10 + sl] = b.y; q[12 + sl] = b.z; q[14 + sl] = b.w;
                    q[16 + sl] = c.x; q[18 + sl] = c.y;
                }
            }
            __syncwarp();
            float2 part[TPL][4];
#pragma unroll
            for (int t = 0; t < TPL; ++t)
#pragma unroll
                for (int c = 0; c < 4; ++c) part[t][c] = make_float2(0.f, 0.f);
            const int np = (ns + 1) >> 1;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const bool tile_r5 = np == 16 && r5;  // part[t][3] then holds -phi
            if (tile_r5) {
#pragma unroll 16
                for (int k = 0; k < 16; ++k) {
                    const float4 a = stF[5 * k], b = stF[5 * k + 1];
                    const float4 c = stF[5 * k + 2], d = stF[5 * k + 3], e = stF[5 * k + 4];
#pragma unroll
                    for (int t = 0; t < TPL; ++t)
                        pc_pair<QUAD, SOFT, true>(nX[t], nY[t], nZ[t], a, b, c, d, e, eps2v, mhalf, halfv, m25,
                                                  part[t]);
                }
            } else if (np == 16) {
#pragma unroll 4
                for (int k = 0; k < 16; ++k) {
                    const float4 a = stF[5 * k], b = stF[5 * k + 1];
                    const float4 c = QUAD ? stF[5 * k + 2] : z4, d = QUAD ? stF[5 * k + 3] : z4,
                                 e = QUAD ? stF[5 * k + 4] : z4;
#pragma unroll
                    for (int t = 0; t < TPL; ++t)
                        pc_pair<QUAD, SOFT>(nX[t], nY[t], nZ[t], a, b, c, d, e, eps2v, neg1, halfv, m25, part[t]);
                }
            } else {
                for (int k = 0; k < np; ++k) {
                    const float4 a = stF[5 * k], b = stF[5 * k + 1];
                    const float4 c = QUAD ? stF[5 * k + 2] : z4, d = QUAD ? stF[5 * k + 3] : z4,
                                 e = QUAD ? stF[5 * k + 4] : z4;
#pragma unroll
                    for (int t = 0; t < TPL; ++t)
                        pc_pair<QUAD, SOFT>(nX[t], nY[t], nZ[t], a, b, c, d, e, eps2v, neg1, halfv, m25, part[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                Real p1[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) p1[c] = (Real)(part[t][c].x + part[t][c].y);
                if (tile_r5) p1[3] = -p1[3];
                fold<Real, KAHAN>(sum[t], cmp[t], p1);
            }
            __syncwarp();
        } else {
            if (lane < ns) {
                const uint32_t c = buf[lane];
                stA[lane] = momA[c];
                if (QUAD) { stB[lane] = momB[c]; stC[lane] = momC[c]; }
            }
            __syncwarp();
            Real part[TPL][4];
#pragma unroll
            for (int t = 0; t < TPL; ++t)
#pragma unroll
                for (int c = 0; c < 4; ++c) part[t][c] = Real(0);
            V4 b0{};
            V2 c0{};
            for (int j = 0; j < ns; ++j) {
                const V4 a = stA[j];
                const V4 b = QUAD ? stB[j] : b0;
                const V2 c = QUAD ? stC[j] : c0;
#pragma unroll
                for (int t = 0; t < TPL; ++t) pc_term<Real, QUAD, SOFT>(px[t], py[t], pz[t], a, b, c, eps2, part[t]);
            }
#pragma unroll
            for (int t = 0; t < TPL; ++t) fold<Real, KAHAN>(sum[t], cmp[t], part[t]);
            __syncwarp();
        }
    };

    // --- traversal ---
    int64_t pc_base = 0, pp_base = 0;
    if (MODE == kWalkEmit) {
        pc_base = A.list_off[g];
        pp_base = A.list_off[A.ngroups + 1 + g];
    }
    uint32_t n_pc = 0, n_pp = 0, n_ppl = 0, max_top = 1;
    int top = 1, npc = 0, npp = 0;
    // Stack entries are child ranges: first node | (count - 1) << 29.
    // the root of the group's segment (node b at level 0): range (node b, 1 node)
    if (lane == 0) stack[0] = gseg;
    __syncwarp();
    bool overflow = false;
    while (top > 0) {
        // pop up to 32 nodes from the top ranges; the last range may be split
        const int nr = top < 32 ? top : 32;
        uint32_t e = 0, sz = 0;
        if (lane < nr) {
            e = stack[top - 1 - lane];
            sz = (e >> 29) + 1u;
        }
        const uint32_t incl0 = warp_incl_scan(sz, lane);
        const uint32_t excl0 = incl0 - sz;
        const uint32_t avail = __shfl_sync(0xffffffffu, incl0, 31);
        const uint32_t take = avail < 32u ? avail : 32u;
        const bool contrib = lane < nr && excl0 < take;
        const int nfull = __popc(__ballot_sync(0xffffffffu, lane < nr && incl0 <= take));
        // the contributing ranges are lanes 0..k-1 with increasing starts excl0:
        // lane t belongs to the last one whose start is <= t
        const uint32_t starts = __reduce_or_sync(0xffffffffu, contrib ? (1u << excl0) : 0u);
        const int owner = __popc(starts & (lt | (1u << lane))) - 1;
        const uint32_t e_own = __shfl_sync(0xffffffffu, e, owner & 31);
        const uint32_t x_own = __shfl_sync(0xffffffffu, excl0, owner & 31);
        const bool act = (uint32_t)lane < take;
        const uint32_t node = act ? (e_own & 0x1fffffffu) + ((uint32_t)lane - x_own) : 0u;
        if (contrib && incl0 > take) {
            // partially used range (lane == nfull): keep its unused tail on the stack
            const uint32_t used = take - excl0;
            stack[top - 1 - lane] = ((e & 0x1fffffffu) + used) | ((sz - used - 1u) << 29);
        }
        top -= nfull;
        __syncwarp();
        uint4 geo = make_uint4(0, 0, 0, 0);
        uint2 lk = make_uint2(0, 0);
        if (act) { geo = A.ngeo[node]; lk = A.nlink[node]; }
        const int level = (int)(geo.w & 0xffu);
        const bool leaf = (geo.w >> 8) & 1u;
        const int s = 1 << (kBits - level);
        const int cx = (int)geo.x, cy = (int)geo.y, cz = (int)geo.z;
        const int gx = max(0, max(cx - ghi0, glo0 - (cx + s)));
        const int gy = max(0, max(cy - ghi1, glo1 - (cy + s)));
        const int gz = max(0, max(cz - ghi2, glo2 - (cz + s)));
        const long long d2 = (long long)gx * gx + (long long)gy * gy + (long long)gz * gz;
        const bool far = act && d2 >= sD[level];
        const bool nleaf = act && !far && leaf;
        const bool open = act && !far && !leaf;
        // A child's box lies inside its parent's, so it is at least as far from
        // the group: when an opened cell already meets its children's threshold
        // (d2 >= D[level + 1]), all its children are far and go to the far list
        // without being popped and tested one by one.
        const bool allfar = open && d2 >= sD[min(level + 1, kMaxLevel)];

        // far cells
        const uint32_t fm = __ballot_sync(0xffffffffu, far);
        const uint32_t nf = __popc(fm);
        if (MODE == kWalkForce) {
            if (far) pcbuf[npc + __popc(fm & lt)] = node;
            npc += nf;
        } else if (MODE == kWalkEmit) {
            if (far) A.pc_list[pc_base + n_pc + __popc(fm & lt)] = (int32_t)node;
        }
        n_pc += nf;
        const uint32_t am = __ballot_sync(0xffffffffu, allfar);
        if (am) {
            const uint32_t cc = allfar ? lk.y : 0u;
            const uint32_t incl = warp_incl_scan(cc, lane);
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            if (MODE == kWalkForce) {
                if (allfar)
                    for (uint32_t c = 0; c < cc; ++c) pcbuf[npc + (incl - cc) + c] = lk.x + c;
                npc += (int)tot;
            } else if (MODE == kWalkEmit) {
                if (allfar)
                    for (uint32_t c = 0; c < cc; ++c) A.pc_list[pc_base + n_pc + (incl - cc) + c] = (int32_t)(lk.x + c);
            }
            n_pc += tot;
        }

        // children of the other opened cells: one stack entry per opened cell
        const bool push = open && !allfar;
        const uint32_t om = __ballot_sync(0xffffffffu, push);
        if (om) {
            const int no = __popc(om);
            if (top + no > SD) {
                overflow = true;
            } else {
                if (push) stack[top + __popc(om & lt)] = lk.x | ((lk.y - 1u) << 29);
                top += no;
            }
            max_top = max(max_top, (uint32_t)top);
        }

        // near leaves (most steps of a deep walk have none)
        const uint32_t lm = __ballot_sync(0xffffffffu, nleaf);
        if (lm) {
            if (MODE == kWalkEmit) {
                if (nleaf) A.pp_list[pp_base + n_ppl + __popc(lm & lt)] = (int32_t)node;
            }
            n_ppl += __popc(lm);
            const uint32_t lc = nleaf ? lk.y : 0u;
            const bool big = lc > (uint32_t)kMaxLeafSmall;
            const uint32_t sc = big ? 0u : lc;
            const uint32_t incl2 = warp_incl_scan(sc, lane);
            const uint32_t tot2 = __shfl_sync(0xffffffffu, incl2, 31);
            n_pp += __reduce_add_sync(0xffffffffu, lc);
            if (MODE == kWalkForce) {
                if (nleaf && !big)
                    for (uint32_t c = 0; c < lc; ++c) ppbuf[npp + (incl2 - lc) + c] = lk.x + c;
                npp += (int)tot2;
                __syncwarp();
                uint32_t bm = __ballot_sync(0xffffffffu, big);
                while (bm) {
                    const int b = __ffs(bm) - 1;
                    bm &= bm - 1;
                    const uint32_t f = __shfl_sync(0xffffffffu, lk.x, b);
                    const uint32_t c = __shfl_sync(0xffffffffu, lk.y, b);
                    for (uint32_t o = 0; o < c; o += 32) eval_pp_range(f + o, (int)min(32u, c - o));
                }
            }
        }
        if (MODE == kWalkForce) {
            if (npc >= 32) {
                __syncwarp();
                const int ntile = npc >> 5;
                for (int t = 0; t < ntile; ++t) eval_pc_list(pcbuf + 32 * t, 32);
                const int r = npc & 31;
                uint32_t t = lane < r ? pcbuf[32 * ntile + lane] : 0;
                __syncwarp();
                if (lane < r) pcbuf[lane] = t;
                __syncwarp();
                npc = r;
            }
            if (npp >= 32) {
                const int ntile = npp >> 5;
                for (int t = 0; t < ntile; ++t) eval_pp_list(ppbuf + 32 * t, 32);
                const int r = npp & 31;
                uint32_t t = lane < r ? ppbuf[32 * ntile + lane] : 0;
                __syncwarp();
                if (lane < r) ppbuf[lane] = t;
                __syncwarp();
                npp = r;
            }
        } else {
            __syncwarp();
        }
    }
    if (MODE == kWalkForce) {
        // every traversal step evaluates the whole tiles, so fewer than 32
        // entries are left here: the staging holds at most 32 sources
        if (npc > 0) eval_pc_list(pcbuf, npc);
        if (npp > 0) eval_pp_list(ppbuf, npp);
    }
    if (overflow && lane == 0) set_status(A.dstatus, TREE_DEV_STACK);
    if (lane == 0 && A.gstat) A.gstat[g] = make_uint4(n_pc, n_pp, max_top, n_ppl);

    if (MODE == kWalkForce) {
        const Real G = (Real)A.G;
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
            const int li = lane + 32 * t;
            if (li < cnt) {
                const uint32_t i = A.perm[s0 + li];
                Real ax, ay, az, ph;
                if (KAHAN) {
                    ax = sum[t][0] - cmp[t][0]; ay = sum[t][1] - cmp[t][1];
                    az = sum[t][2] - cmp[t][2]; ph = sum[t][3] - cmp[t][3];
                } else {
                    ax = sum[t][0]; ay = sum[t][1]; az = sum[t][2]; ph = sum[t][3];
                }
                ax *= G; ay *= G; az *= G; ph *= G;
                Real *a = reinterpret_cast<Real *>(A.a);
                const int64_t n = A.n;
                a[i] = ax; a[n + i] = ay; a[2 * n + i] = az;
                if (A.phi) reinterpret_cast<Real *>(A.phi)[i] = ph;
                if (A.phi2) reinterpret_cast<Real *>(A.phi2)[i] = ph;
                if (A.v) {
                    Real *v = reinterpret_cast<Real *>(A.v);
                    const Real ht = (Real)A.half_tau;
                    const Real vx = fma(ht, ax, v[i]), vy = fma(ht, ay, v[n + i]), vz = fma(ht, az, v[2 * n + i]);
                    v[i] = vx; v[n + i] = vy; v[2 * n + i] = vz;
                    if (A.v2) {
                        Real *w = reinterpret_cast<Real *>(A.v2);
                        w[i] = vx; w[n + i] = vy; w[2 * n + i] = vz;
                    }
                }
            }
        }
    }
    }  // group loop
}

}  // namespace treegb

namespace treegb {

// Host: walk arguments from the workspace.
inline WalkArgs make_walk_args(TreeWorkspace *ws, const WalkOut &out) {
    WalkArgs a;
    a.n = ws->n;
    a.gs = ws->p.group_size;
    a.ngroups = ws->list_groups_host;  // host copy of the group count (list emission only)
    a.spos = ws->spos;
    a.skey = ws->key;
    a.perm = ws->idx;
    a.ngeo = ws->ngeo;
    a.nlink = ws->nlink;
    a.mom_a = ws->mom_a;
    a.mom_b = ws->mom_b;
    a.mom_c = ws->mom_c;
    a.dmac = ws->dmac;
    a.G = ws->p.G;
    a.eps = ws->p.eps;
    a.eps2 = ws->p.eps * ws->p.eps;
    a.a = out.a;
    a.phi = out.phi;
    a.v = out.v;
    a.half_tau = out.half_tau;
    a.v2 = out.v_mirror;
    a.phi2 = out.phi_mirror;
    a.stack_depth = ws->p.stack_depth;
    a.gstat = ws->gstat;
    a.dstatus = ws->dstatus;
    a.list_off = ws->list_cnt;
    a.pc_list = ws->pc_list;
    a.pp_list = ws->pp_list;
    a.order = walk_widest_first(ws) ? ws->gorder : nullptr;
    a.gfirst = ws->gfirst;
    a.ctr = ws->ctr;
    a.seg_off = ws->seg_off;
    a.nseg = ws->nseg;
    a.box = ws->box;
    return a;
}

template <typename Real, int TPL, bool QUAD, bool KAHAN, bool SOFT, int MODE>
cudaError_t walk_run(TreeWorkspace *ws, const WalkArgs &a, cudaStream_t s) {
    if (ws->n <= 0) return cudaSuccess;
    auto k = k_walk<Real, TPL, QUAD, KAHAN, SOFT, MODE>;
    const size_t smem = kWalkWarps * walk_warp_bytes<Real>(a.stack_depth);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // persistent grid: the resident blocks, never more than the groups need
    int per_sm = 0, sms = 0, dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWalkWarps * 32, smem);
    if (e != cudaSuccess) return e;
    const int64_t ng_bound = (ws->n + kWalkWarps - 1) / kWalkWarps;
    int64_t nb = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
    if (nb > ng_bound) nb = ng_bound;
    if (nb < 1) nb = 1;
    e = cudaMemsetAsync(ws->ctr + kCtrWalkTicket, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)nb, kWalkWarps * 32, smem, s>>>(a);
    ws->launches += 1;
    return cudaGetLastError();
}

}  // namespace treegb
