// Host driver for the double-word arithmetic (p2_dw.cuh) and the double-word
// eigen-decomposition (p2_eig_dw.cuh) of the library's Procrustes kernels,
// compiled as plain C++ (no CUDA) by tests/test_dw_host.py.  Test
// infrastructure only.
//
//   dw_check ops            reads lines "op xh xl yh yl" (hex floats) and
//                           prints "zh zl" for op in add sub mul mulf sqr fma
//                           div sqrt rsqrt dot2 acc
//   dw_check eig n          reads n*n doubles (a symmetric matrix, row-major,
//                           already scaled to unit size), prints the step
//                           count, then d (n values) and Z (n*n, row-major)
//                           as double values of the double-word results
//   dw_check eig64 n        the same decomposition compiled for FP64 (the
//                           opt-in FP64 arm of the Procrustes step)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#define P2_HD inline
#include "p2_eig_dw.cuh"

using namespace p2;

static dw rd(double x) {
    const float h = (float)x;
    return dw{h, (float)(x - (double)h)};
}
static double val(dw x) { return (double)x.h + (double)x.l; }

static int ops() {
    char op[16];
    float a[6];
    while (std::scanf("%15s %a %a %a %a %a %a", op, &a[0], &a[1], &a[2], &a[3], &a[4], &a[5]) == 7) {
        const dw x{a[0], a[1]}, y{a[2], a[3]}, z{a[4], a[5]};
        dw r{0.f, 0.f};
        if (!std::strcmp(op, "add")) r = dw_add(x, y);
        else if (!std::strcmp(op, "sub")) r = dw_sub(x, y);
        else if (!std::strcmp(op, "mul")) r = dw_mul(x, y);
        else if (!std::strcmp(op, "mulf")) r = dw_mulf(x, y.h);
        else if (!std::strcmp(op, "sqr")) r = dw_sqr(x);
        else if (!std::strcmp(op, "fma")) r = dw_fma(x, y, z);
        else if (!std::strcmp(op, "div")) r = dw_div(x, y);
        else if (!std::strcmp(op, "sqrt")) r = dw_sqrt(x);
        else if (!std::strcmp(op, "rsqrt")) r = dw_rsqrt(x);
        else if (!std::strcmp(op, "dot2")) r = dw_dot2(x, y, z, x);
        else if (!std::strcmp(op, "acc")) {          // x*y + z*x accumulated, plus y
            dwacc s = acc_from(y);
            acc_fma(s, x, y);
            acc_fma(s, z, x);
            r = acc_val(s);
        } else return 2;
        std::printf("%a %a\n", r.h, r.l);
    }
    return 0;
}

static double val(f64n x) { return x.h; }
template <class D> static D rd_t(double x);
template <> dw rd_t<dw>(double x) { return rd(x); }
template <> f64n rd_t<f64n>(double x) { return f64n{x}; }

template <class D>
static int eig(int n) {
    std::vector<double> m((size_t)n * n);
    for (auto &v : m)
        if (std::scanf("%lf", &v) != 1) return 2;
    // interleaved layout with stride 1: A (n x n), then d, e
    std::vector<D> buf((size_t)n * n + 2 * (size_t)n);
    DwMat<D> A{buf.data(), 1, n};
    DwVec<D> d{buf.data() + (size_t)n * n, 1};
    DwVec<D> e{buf.data() + (size_t)n * n + n, 1};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) A(i, j) = rd_t<D>(m[(size_t)i * n + j]);
    tridiagonalize_dw<0>(n, A, d, e);
    int rot = 0;
    const int steps = tridiagonal_qr_dw<0>(n, A, d, e, 30 * n, &rot);
    std::printf("%d\n", steps);
    for (int i = 0; i < n; ++i) std::printf("%.17g\n", val(d[i]));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) std::printf("%.17g\n", val(A(i, j)));
    return 0;
}

int main(int argc, char **argv) {
    if (argc >= 2 && !std::strcmp(argv[1], "ops")) return ops();
    if (argc >= 3 && !std::strcmp(argv[1], "eig")) return eig<dw>(std::atoi(argv[2]));
    if (argc >= 3 && !std::strcmp(argv[1], "eig64")) return eig<f64n>(std::atoi(argv[2]));
    std::fprintf(stderr, "usage: dw_check ops | dw_check eig n | dw_check eig64 n\n");
    return 2;
}
