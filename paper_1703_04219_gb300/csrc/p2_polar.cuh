// Helpers shared by the Procrustes kernels (p2_polar.cu, p2_polar_grp.cu).
#pragma once

#include <stdint.h>

namespace p2 {

#ifndef FULLMASK
#define FULLMASK 0xffffffffu
#endif

// Algorithmic FP64 flops per subject of the Procrustes step (fused
// multiply-add = 2; sqrt, rsqrt and division = 1), counted on the
// lane-per-subject formulation of p2_polar.cu (the grouped kernel reports the
// same count), except the data-dependent QR part, which adds 11 per QR step
// and 27 + 6R per Givens rotation.
inline __host__ __device__ unsigned long long polar_fixed_flops(int R) {
    const unsigned long long r = (unsigned long long)R, P = r * (r + 1) / 2;
    unsigned long long f = 2 * P;                    // S G S
    f += 2 * r * r * r + r * r * (r + 1);            // M = H (S G S) H^T, lower triangle
    for (unsigned long long m = 2; m + 1 <= r; ++m) {
        f += 4 * m * m + 8 * m + 9;                  // Householder step on an m-vector
        f += m * (4 * m - 2);                        // its backward accumulation
    }
    f += 3 * r;                                      // QR scale estimate
    f += 2 * r + 1;                                  // cut and d^-1/2
    f += r + r * r;                                  // Z columns scaled by d^-1/4
    f += r * r * (r + 1);                            // C = Z Z^T (lower)
    f += 2 * r * r * r + r * r;                      // T = C H S
    return f;
}

static __device__ __forceinline__ unsigned long long qr_flops(int R, int steps, int rot) {
    return 11ull * (unsigned long long)(steps > 0 ? steps : 0) +
           (27ull + 6ull * (unsigned long long)R) * (unsigned long long)rot;
}

static __device__ __forceinline__ void add_flops(SmallState *st, unsigned long long flops) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) flops += __shfl_down_sync(FULLMASK, flops, o);
    if ((threadIdx.x & 31) == 0 && flops) atomicAdd(&st->polar_flops, flops);
}

}  // namespace p2
