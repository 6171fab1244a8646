// Grouped Procrustes kernel (R > 12): the FP64 instances (the opt-in FP64
// arm of the Procrustes step).
#include "p2_polar_grp_launch.cuh"

namespace p2 {

cudaError_t polar_grp_configure_f64(int cap) { return grp_configure_t<f64n>(cap); }

cudaError_t launch_polar_grp_f64(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                                 float *T, int64_t K, cudaStream_t s, double rtol2,
                                 const int32_t *order, int32_t *qrcnt) {
    return launch_grp_t<f64n>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
}

}  // namespace p2
