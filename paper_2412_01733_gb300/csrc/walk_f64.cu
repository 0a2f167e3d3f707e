// walk_f64.cu -- the "plain" FP64 tree walk: the same traversal and lists,
// FP64 positions, moments and pair terms, uncompensated sums.
#include "walk.cuh"

namespace treegb {

template <int TPL, bool QUAD, bool SOFT>
static cudaError_t force_f64(TreeWorkspace *ws, const WalkArgs &a, cudaStream_t s) {
    return walk_run<double, TPL, QUAD, false, SOFT, kWalkForce>(ws, a, s);
}

cudaError_t launch_walk_f64(TreeWorkspace *ws, int mode, const WalkOut &out, cudaStream_t s) {
    const WalkArgs a = make_walk_args(ws, out);
    const bool two = ws->p.group_size > 32;
    if (mode == kWalkCount)
        return two ? walk_run<double, 2, false, false, true, kWalkCount>(ws, a, s)
                   : walk_run<double, 1, false, false, true, kWalkCount>(ws, a, s);
    if (mode == kWalkEmit)
        return two ? walk_run<double, 2, false, false, true, kWalkEmit>(ws, a, s)
                   : walk_run<double, 1, false, false, true, kWalkEmit>(ws, a, s);
    const bool quad = ws->p.order == 2, soft = ws->p.eps > 0.0;
    if (two) {
        if (quad) return soft ? force_f64<2, true, true>(ws, a, s) : force_f64<2, true, false>(ws, a, s);
        return soft ? force_f64<2, false, true>(ws, a, s) : force_f64<2, false, false>(ws, a, s);
    }
    if (quad) return soft ? force_f64<1, true, true>(ws, a, s) : force_f64<1, true, false>(ws, a, s);
    return soft ? force_f64<1, false, true>(ws, a, s) : force_f64<1, false, false>(ws, a, s);
}

}  // namespace treegb
