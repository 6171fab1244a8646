// Stand-in for cuda_bf16.h on the host (CPU emulator): bfloat16 as a 16-bit
// pattern with round-to-nearest-even conversion from float.
#pragma once
#include <cstdint>
#include <cstring>
struct __nv_bfloat16 {
    uint16_t x;
};
inline __nv_bfloat16 __float2bfloat16_rn(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return __nv_bfloat16{(uint16_t)((u >> 16) | 0x40u)};
    u += 0x7fffu + ((u >> 16) & 1u);
    return __nv_bfloat16{(uint16_t)(u >> 16)};
}
inline float __bfloat162float(__nv_bfloat16 h) {
    const uint32_t u = (uint32_t)h.x << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}
