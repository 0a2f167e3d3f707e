// walk_f32.cu -- FP32 tree walk: FP32 positions, moments and pair terms,
// optional Kahan-compensated per-particle sums.
#include <cfloat>

#include "walk.cuh"

namespace treegb {

template <int TPL, bool QUAD, bool KAHAN, bool SOFT>
static cudaError_t force_f32(TreeWorkspace *ws, const WalkArgs &a, cudaStream_t s) {
    return walk_run<float, TPL, QUAD, KAHAN, SOFT, kWalkForce>(ws, a, s);
}

template <int TPL>
static cudaError_t dispatch_f32(TreeWorkspace *ws, const WalkArgs &a, bool quad, bool kahan, bool soft, cudaStream_t s) {
    if (quad) {
        if (kahan) return soft ? force_f32<TPL, true, true, true>(ws, a, s) : force_f32<TPL, true, true, false>(ws, a, s);
        return soft ? force_f32<TPL, true, false, true>(ws, a, s) : force_f32<TPL, true, false, false>(ws, a, s);
    }
    if (kahan) return soft ? force_f32<TPL, false, true, true>(ws, a, s) : force_f32<TPL, false, true, false>(ws, a, s);
    return soft ? force_f32<TPL, false, false, true>(ws, a, s) : force_f32<TPL, false, false, false>(ws, a, s);
}

cudaError_t launch_walk_f32(TreeWorkspace *ws, int mode, const WalkOut &out, cudaStream_t s) {
    const WalkArgs a = make_walk_args(ws, out);
    const bool two = ws->p.group_size > 32;
    if (mode == kWalkCount)
        return two ? walk_run<float, 2, false, false, true, kWalkCount>(ws, a, s)
                   : walk_run<float, 1, false, false, true, kWalkCount>(ws, a, s);
    if (mode == kWalkEmit)
        return two ? walk_run<float, 2, false, false, true, kWalkEmit>(ws, a, s)
                   : walk_run<float, 1, false, false, true, kWalkEmit>(ws, a, s);
    // the softened pair terms need eps^2 to be a normal FP32 number (see
    // rsqrt_pair); a smaller eps^2 takes the unsoftened variant, which still
    // adds it to r^2 and drops coincident pairs
    const bool quad = ws->p.order == 2, kahan = ws->p.kahan != 0;
    const bool soft = (float)(ws->p.eps * ws->p.eps) >= FLT_MIN;
    return two ? dispatch_f32<2>(ws, a, quad, kahan, soft, s) : dispatch_f32<1>(ws, a, quad, kahan, soft, s);
}

}  // namespace treegb
