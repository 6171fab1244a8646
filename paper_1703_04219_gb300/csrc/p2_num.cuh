// Number types of the Procrustes step: the double-word format of p2_dw.cuh
// (the default, on the FP32 pipe) and plain FP64 (the opt-in FP64 arm, on
// the FP64 pipe), behind one interface so that the Householder + QR code and
// the Procrustes kernels are written once and compiled for either.
//
// f64n holds one FP64 value in the field h, the field through which the
// kernels read a value's magnitude, sign and binary exponent; the dw_* and
// acc_* functions below are the FP64 counterparts of p2_dw.cuh's (each a
// correctly rounded FP64 operation, or an FMA).  NumT<D> collects what
// differs between the two types: the accumulator, the deflation threshold
// of the QR iteration and the smallest squared norm the Householder steps
// act on.
#pragma once

#include "p2_dw.cuh"

namespace p2 {

struct alignas(8) f64n {
    double h;
};

// biased binary exponent of |v| on the binary32 scale (127 for [1, 2)),
// clamped to [0, 255] like f_expo of a float: 0 for zero and for magnitudes
// below the binary32 normal range
P2_HD int f_expo(double v) {
    uint64_t b;
#ifdef __CUDA_ARCH__
    b = (uint64_t)__double_as_longlong(v);
#else
    memcpy(&b, &v, sizeof b);
#endif
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;
    const int f = e - 1023 + 127;
    return f < 0 ? 0 : (f > 255 ? 255 : f);
}
// the same exponent without the clamp (zero: a very negative value)
P2_HD int expo_wide(double v) {
    uint64_t b;
#ifdef __CUDA_ARCH__
    b = (uint64_t)__double_as_longlong(v);
#else
    memcpy(&b, &v, sizeof b);
#endif
    const int e = (int)((b >> 52) & 0x7ff);
    return e == 0 ? -100000 : e - 1023 + 127;
}

P2_HD f64n dw_neg(f64n x) { return f64n{-x.h}; }
P2_HD f64n dw_scale(f64n x, float p) { return f64n{x.h * (double)p}; }
P2_HD f64n dw_add(f64n x, f64n y) { return f64n{x.h + y.h}; }
P2_HD f64n dw_sub(f64n x, f64n y) { return f64n{x.h - y.h}; }
P2_HD f64n dw_mul(f64n x, f64n y) { return f64n{x.h * y.h}; }
P2_HD f64n dw_mulf(f64n x, float y) { return f64n{x.h * (double)y}; }
P2_HD f64n dw_sqr(f64n x) { return f64n{x.h * x.h}; }
P2_HD f64n dw_fma(f64n x, f64n y, f64n z) { return f64n{fma(x.h, y.h, z.h)}; }
P2_HD f64n dw_dot2(f64n a, f64n x, f64n b, f64n y) { return f64n{fma(a.h, x.h, b.h * y.h)}; }
P2_HD f64n dw_sqrt(f64n x) { return f64n{x.h > 0.0 ? sqrt(x.h) : 0.0}; }
P2_HD f64n dw_rsqrt(f64n x) { return f64n{1.0 / sqrt(x.h)}; }
P2_HD f64n dw_div(f64n x, f64n y) { return f64n{x.h / y.h}; }
P2_HD f64n dw_recip(f64n y) { return f64n{1.0 / y.h}; }

struct f64acc {
    double s;
};
P2_HD f64acc acc_from(f64n x) { return f64acc{x.h}; }
P2_HD void acc_fma(f64acc &a, f64n x, f64n y) { a.s = fma(x.h, y.h, a.s); }
P2_HD void acc_fmaf(f64acc &a, f64n x, float y) { a.s = fma(x.h, (double)y, a.s); }
P2_HD void acc_sqr(f64acc &a, f64n x) { a.s = fma(x.h, x.h, a.s); }
P2_HD void acc_add(f64acc &a, f64n x) { a.s += x.h; }
P2_HD f64n acc_val(f64acc a) { return f64n{a.s}; }

// Deflation of a QR sub-diagonal entry in FP64: negligible when its binary
// exponent is at least F64_DEFLATE_BITS below that of the larger adjacent
// diagonal entry (|e| < 2^-49 (|d1| + |d2|), a few FP64 roundings) or at or
// below tiny_ex.
constexpr int F64_DEFLATE_BITS = 50;
P2_HD bool dw_negligible(f64n ev, f64n d1, f64n d2, int tiny_ex) {
    if (ev.h == 0.0) return true;
    const int x = expo_wide(ev.h);
    const int a = expo_wide(d1.h), b = expo_wide(d2.h);
    return x <= (a > b ? a : b) - F64_DEFLATE_BITS || x <= tiny_ex;
}

template <class D> struct NumT;
template <> struct NumT<dw> {
    using acc = dwacc;
    static constexpr int deflate_bits = DW_DEFLATE_BITS;
    static P2_HD float tiny2() { return DW_TINY2; }
};
template <> struct NumT<f64n> {
    using acc = f64acc;
    static constexpr int deflate_bits = F64_DEFLATE_BITS;
    static P2_HD float tiny2() { return 1e-30f; }     // ~2^-100: squares far inside FP64's range
};
template <class D> using acc_t = typename NumT<D>::acc;

template <class D> P2_HD acc_t<D> acc0();
template <> P2_HD dwacc acc0<dw>() { return acc_zero(); }
template <> P2_HD f64acc acc0<f64n>() { return f64acc{0.0}; }

// the value of a float
template <class D> P2_HD D num_f(float x);
template <> P2_HD dw num_f<dw>(float x) { return dw_f(x); }
template <> P2_HD f64n num_f<f64n>(float x) { return f64n{(double)x}; }

// a double-word input (the packed Gram) in the number type, exactly
template <class D> P2_HD D from_dw(dw x);
template <> P2_HD dw from_dw<dw>(dw x) { return x; }
template <> P2_HD f64n from_dw<f64n>(dw x) { return f64n{(double)x.h + (double)x.l}; }

// the exact product of two floats
template <class D> P2_HD D num_prod(float a, float b);
template <> P2_HD dw num_prod<dw>(float a, float b) { return two_prod(a, b); }
template <> P2_HD f64n num_prod<f64n>(float a, float b) { return f64n{(double)a * (double)b}; }

// v 2^(o1 + o2) rounded to float (o1, o2 powers of two, applied one at a
// time so that no intermediate leaves the float range)
P2_HD float store_f(dw v, float o1, float o2) { return f_mul(f_mul(v.h, o1), o2); }
P2_HD float store_f(f64n v, float o1, float o2) { return (float)(v.h * (double)o1 * (double)o2); }

}  // namespace p2
