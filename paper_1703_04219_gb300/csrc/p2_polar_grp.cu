// Grouped Procrustes kernel (R > 12): the double-word instances and the
// dispatch on the context's arithmetic (the FP64 instances are in
// p2_polar_grp_f64.cu).
#include "p2_polar_grp_launch.cuh"

namespace p2 {

cudaError_t polar_grp_configure(int cap, bool fp64) {
    return fp64 ? polar_grp_configure_f64(cap) : grp_configure_t<dw>(cap);
}

cudaError_t launch_polar_grp(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             float *T, int64_t K, cudaStream_t s, double rtol2,
                             const int32_t *order, int32_t *qrcnt, const dw *mpre) {
    if (c->opt.fp64_procrustes)
        return launch_polar_grp_f64(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    return launch_grp_t<dw>(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre);
}

}  // namespace p2
