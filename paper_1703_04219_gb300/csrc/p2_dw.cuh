// Double-word ("float-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two binary32 numbers, |l| <=
// ulp(h) / 2 after normalisation, which carries about 48 significant bits.
// The Procrustes step (Section 3.2) runs its eigen-decomposition in this
// format: the FP64 pipe of this GPU issues one warp instruction per ~76
// cycles per SM sub-partition while the FP32 pipe issues one per cycle, so a
// double-word operation of 6 to 20 FP32 instructions is several times
// cheaper than one FP64 instruction.
//
// Building blocks (all published, none taken from a library):
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and Fast2Sum (Dekker 1971): the
//     rounding error of a sum as a float;
//   TwoProd with an FMA: the rounding error of a product as a float;
//   products and sums of double-words after Joldes, Muller and Popescu,
//     "Tight and rigorous error bounds for basic building blocks of
//     double-word arithmetic", ACM TOMS 44(2), 2017 (DWTimesDW with FMA and
//     SloppyDWPlusDW, whose error is bounded by a few u^2 (|x| + |y|), u =
//     2^-24: normwise, as the Householder and Givens error analyses need);
//   square root and reciprocal square root by one Newton correction of the
//     FP32 result, the residual evaluated in double-word arithmetic;
//   division by one correction of the FP32 quotient (Karp and Markstein,
//     "High-precision division and square root", ACM TOMS 23(4), 1997).
// Accumulations of products (dot products) keep the running sum's high part
// with TwoSum and collect every low part and rounding error in a second
// float (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26(6), 2005, Algorithm Dot2, extended to double-word operands).
//
// Every rounding below must happen as written, so the device code uses the
// __f*_rn intrinsics, which the compiler never contracts into an FMA; host
// builds must not contract either (no -ffp-contract=fast with FMA hardware).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef P2_HD
#define P2_HD __host__ __device__ __forceinline__
#endif

namespace p2 {

struct alignas(8) dw {
    float h, l;
};

P2_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
P2_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
P2_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
P2_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
// correctly rounded square root
P2_HD float f_sqrt(float a) {
#ifdef __CUDA_ARCH__
    return __fsqrt_rn(a);
#else
    return sqrtf(a);
#endif
}
// Approximations (a few ulp) whose error a following correction removes.
// The callers keep their arguments in the normal range; the host versions
// (used by the CPU checks) treat a subnormal argument as zero, the harsher
// of the behaviours a hardware approximation may have, so that a caller
// that lets one through fails there too.
P2_HD float f_rsqrt_approx(float a) {
#ifdef __CUDA_ARCH__
    return rsqrtf(a);
#else
    if (fabsf(a) < 1.17549435e-38f) a = 0.f;
    return 1.0f / sqrtf(a);
#endif
}
P2_HD float f_div_approx(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    if (fabsf(b) < 1.17549435e-38f) b = 0.f;
    return a / b;
#endif
}

// biased binary exponent field of |v| (0 for zero and subnormals)
P2_HD int f_expo(float v) {
#ifdef __CUDA_ARCH__
    return (__float_as_int(v) >> 23) & 0xff;
#else
    uint32_t b;
    memcpy(&b, &v, sizeof b);
    return (int)((b >> 23) & 0xff);
#endif
}
// 2^n as a float, n clamped to the normal range [-126, 127]
P2_HD float f_pow2(int n) {
    n = n < -126 ? -126 : (n > 127 ? 127 : n);
    const uint32_t b = (uint32_t)(n + 127) << 23;
#ifdef __CUDA_ARCH__
    return __int_as_float((int)b);
#else
    float v;
    memcpy(&v, &b, sizeof v);
    return v;
#endif
}

// count of leading zero bits of a non-zero 64-bit word
P2_HD int p2_clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return __builtin_clzll(v);
#endif
}

P2_HD dw dw_f(float h) { return dw{h, 0.f}; }

// a + b = s + e exactly (TwoSum, any a, b)
P2_HD dw two_sum(float a, float b) {
    const float s = f_add(a, b);
    const float bv = f_sub(s, a);
    const float e = f_add(f_sub(a, f_sub(s, bv)), f_sub(b, bv));
    return dw{s, e};
}
// a + b = s + e exactly when expo(a) >= expo(b) (Fast2Sum); otherwise s is
// still the rounded sum and e its error up to O(u |s|)
P2_HD dw fast_sum(float a, float b) {
    const float s = f_add(a, b);
    const float e = f_sub(b, f_sub(s, a));
    return dw{s, e};
}
// a * b = p + e exactly (TwoProd with an FMA)
P2_HD dw two_prod(float a, float b) {
    const float p = f_mul(a, b);
    return dw{p, f_fma(a, b, -p)};
}

P2_HD dw dw_neg(dw x) { return dw{-x.h, -x.l}; }
// exact scaling by a power of two p (barring underflow of l)
P2_HD dw dw_scale(dw x, float p) { return dw{f_mul(x.h, p), f_mul(x.l, p)}; }

// x + y (SloppyDWPlusDW): error <= ~2u^2 (|x| + |y|)
P2_HD dw dw_add(dw x, dw y) {
    const dw s = two_sum(x.h, y.h);
    const float v = f_add(x.l, y.l);
    return fast_sum(s.h, f_add(s.l, v));
}
P2_HD dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }

// x * y (DWTimesDW with an FMA; the l*l term is below the error bound)
P2_HD dw dw_mul(dw x, dw y) {
    const float ch = f_mul(x.h, y.h);
    float cl = f_fma(x.h, y.h, -ch);
    const float t = f_fma(x.l, y.h, f_mul(x.h, y.l));
    cl = f_add(cl, t);
    return fast_sum(ch, cl);
}
// x * y for a float y
P2_HD dw dw_mulf(dw x, float y) {
    const float ch = f_mul(x.h, y);
    float cl = f_fma(x.h, y, -ch);
    cl = f_fma(x.l, y, cl);
    return fast_sum(ch, cl);
}
// x^2
P2_HD dw dw_sqr(dw x) {
    const float ch = f_mul(x.h, x.h);
    float cl = f_fma(x.h, x.h, -ch);
    cl = f_fma(f_add(x.h, x.h), x.l, cl);
    return fast_sum(ch, cl);
}
// x * y + z with one normalisation: error <= ~4u^2 (|x y| + |z|)
P2_HD dw dw_fma(dw x, dw y, dw z) {
    const float ph = f_mul(x.h, y.h);
    float pl = f_fma(x.h, y.h, -ph);
    pl = f_fma(x.h, y.l, pl);
    pl = f_fma(x.l, y.h, pl);
    const dw s = two_sum(ph, z.h);
    return fast_sum(s.h, f_add(f_add(pl, z.l), s.l));
}

// a x + b y with one normalisation (a Givens rotation's output)
P2_HD dw dw_dot2(dw a, dw x, dw b, dw y) {
    const float p1 = f_mul(a.h, x.h);
    float e1 = f_fma(a.h, x.h, -p1);
    e1 = f_fma(a.h, x.l, e1);
    e1 = f_fma(a.l, x.h, e1);
    const float p2 = f_mul(b.h, y.h);
    float e2 = f_fma(b.h, y.h, -p2);
    e2 = f_fma(b.h, y.l, e2);
    e2 = f_fma(b.l, y.h, e2);
    const dw s = two_sum(p1, p2);
    return fast_sum(s.h, f_add(f_add(e1, e2), s.l));
}

// Running sum of products: value s + c, c collecting low parts and errors.
struct dwacc {
    float s, c;
};
P2_HD dwacc acc_zero() { return dwacc{0.f, 0.f}; }
P2_HD dwacc acc_from(dw x) { return dwacc{x.h, x.l}; }
// a += x * y
P2_HD void acc_fma(dwacc &a, dw x, dw y) {
    const float ph = f_mul(x.h, y.h);
    float pl = f_fma(x.h, y.h, -ph);
    pl = f_fma(x.h, y.l, pl);
    pl = f_fma(x.l, y.h, pl);
    const dw t = two_sum(a.s, ph);
    a.s = t.h;
    a.c = f_add(a.c, f_add(t.l, pl));
}
// a += x * y for a float y
P2_HD void acc_fmaf(dwacc &a, dw x, float y) {
    const float ph = f_mul(x.h, y);
    float pl = f_fma(x.h, y, -ph);
    pl = f_fma(x.l, y, pl);
    const dw t = two_sum(a.s, ph);
    a.s = t.h;
    a.c = f_add(a.c, f_add(t.l, pl));
}
// a += x^2
P2_HD void acc_sqr(dwacc &a, dw x) {
    const float ph = f_mul(x.h, x.h);
    float pl = f_fma(x.h, x.h, -ph);
    pl = f_fma(f_add(x.h, x.h), x.l, pl);
    const dw t = two_sum(a.s, ph);
    a.s = t.h;
    a.c = f_add(a.c, f_add(t.l, pl));
}
// a += x
P2_HD void acc_add(dwacc &a, dw x) {
    const dw t = two_sum(a.s, x.h);
    a.s = t.h;
    a.c = f_add(a.c, f_add(t.l, x.l));
}
P2_HD dw acc_val(dwacc a) { return fast_sum(a.s, a.c); }

// sqrt(x) for x >= 0 (0 otherwise): correctly rounded FP32 root s, then
// s + (x - s^2) / (2 s) with the residual in double-word arithmetic
P2_HD dw dw_sqrt(dw x) {
    if (!(x.h > 0.f)) return dw{0.f, 0.f};
    const float s = f_sqrt(x.h);
    const dw p = two_prod(s, s);
    const float r = f_add(f_sub(f_sub(x.h, p.h), p.l), x.l);
    return fast_sum(s, f_div_approx(r, f_add(s, s)));
}
// 1 / sqrt(x) for x > 0: y = rsqrt(x.h), then y + y (1 - x y^2) / 2 with
// 1 - x y^2 in double-word arithmetic (relative error ~1.5 e^2 + O(u^2) for
// an initial error e of a few ulp)
P2_HD dw dw_rsqrt(dw x) {
    const float y = f_rsqrt_approx(x.h);
    const dw m = dw_mul(x, two_prod(y, y));
    const float r = f_sub(f_sub(1.0f, m.h), m.l);
    return fast_sum(y, f_mul(f_mul(y, r), 0.5f));
}
// x / y: q = x.h / y.h, then q + (x - q y) / y.h with x - q y in
// double-word arithmetic
P2_HD dw dw_div(dw x, dw y) {
    const float q = f_div_approx(x.h, y.h);
    const dw r = dw_mulf(y, q);
    const float dh = f_sub(x.h, r.h);
    const float dl = f_sub(x.l, r.l);
    return fast_sum(q, f_div_approx(f_add(dh, dl), y.h));
}
P2_HD dw dw_recip(dw y) { return dw_div(dw{1.0f, 0.f}, y); }

// Deflation test of a sub-diagonal entry ev of a tridiagonal (binary
// exponents, integer arithmetic): negligible when expo(ev) <=
// expo(max(|d1|, |d2|)) - DW_DEFLATE_BITS or expo(ev) <= tiny_ex.  Either
// condition implies |ev| < 2^(1 - DW_DEFLATE_BITS) (|d1| + |d2|) or
// |ev| < 2 * 2^tiny_ex, a backward error of the order of the rounding the
// double-word arithmetic commits (a few 2^-48 relative), with margin so the
// iteration is not asked to resolve its own rounding noise.
constexpr int DW_DEFLATE_BITS = 44;
// squared norms below this are treated as zero by the Householder steps
// (the matrices are scaled to unit size first)
constexpr float DW_TINY2 = 1.2621774e-29f;   // 2^-96
P2_HD bool dw_negligible(dw ev, dw d1, dw d2, int tiny_ex) {
    const int x = f_expo(ev.h);
    const int a = f_expo(d1.h), b = f_expo(d2.h);
    return x == 0 || x <= (a > b ? a : b) - DW_DEFLATE_BITS || x <= tiny_ex;
}

}  // namespace p2
