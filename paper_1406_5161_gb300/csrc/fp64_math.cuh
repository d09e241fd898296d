// FP64 building blocks for the row passes of the FP64 mode.
//
// On this part the FP64 pipe issues about two operations per clock per SM
// (measured: 1.6 dependent-free DFMA per clock per SM), and a float -> double
// conversion instruction takes a slot of that pipe too. The RBF kernel value
// K = exp(-gamma ||x - z||^2) of Section IV-E is the bulk of the FP64 work of
// the SMO step (Algorithm 2's inner product and the exponential, twice per
// active row) and of the gradient reconstruction (Algorithm 6). These helpers
// keep the arithmetic FP64 while moving work off that pipe:
//
//   widen_f32(x)   the float x as a double, exactly (the same value as the
//                  conversion instruction), by integer operations on the bit
//                  pattern;
//   exp_tang(x, T) exp(x) by the table-driven method of P. T. P. Tang,
//                  "Table-driven implementation of the exponential function
//                  in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989:
//                  x = (256 m + j) ln2/256 + r with |r| <= ln2/512, so
//                  exp(x) = 2^m * 2^(j/256) * exp(r); 2^(j/256) from a
//                  correctly rounded table T (exp2_table.inc, 256 doubles),
//                  exp(r) - 1 by its Taylor polynomial of degree 5. Ten FP64
//                  operations in the common case; within about one unit in
//                  the last place of the exact value (checked on the host
//                  against long double exp by tests/test_fp64_math_cpu.py).
//
// Both are plain IEEE arithmetic (fma, add, multiply) plus integer
// operations, written for host and device alike: the host build computes the
// same bits, which is how the tests check them without a GPU.
#ifndef SVM_FP64_MATH_CUH
#define SVM_FP64_MATH_CUH

#include <stdint.h>
#include <math.h>
#include <string.h>

#if defined(__CUDACC__)
#define SVM_HD __host__ __device__ __forceinline__
#else
#define SVM_HD inline
#endif

namespace svmgb {

SVM_HD double bits_to_double(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
#endif
}

SVM_HD uint64_t double_to_bits(double d)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    memcpy(&b, &d, sizeof b);
    return b;
#endif
}

SVM_HD uint32_t float_to_bits(float f)
{
#if defined(__CUDA_ARCH__)
    return (uint32_t)__float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    return b;
#endif
}

SVM_HD int count_leading_zeros32(uint32_t v)
{
#if defined(__CUDA_ARCH__)
    return __clz((int)v);
#else
    return v ? __builtin_clz(v) : 32;
#endif
}

// A finite float as a double, exactly. Normal floats: the exponent is
// re-biased (127 -> 1023) and the 23 fraction bits move to the top of the 52;
// zeros keep their sign; subnormal floats (m * 2^-149) are normalised with a
// leading-zero count.
SVM_HD double widen_f32(float x)
{
    const uint32_t u = float_to_bits(x);
    const uint32_t mag = u & 0x7fffffffu;
    uint64_t b;
    if (mag >= 0x00800000u) {
        b = ((uint64_t)((mag >> 3) + (896u << 20)) << 32) | (uint64_t)(mag << 29);
    } else if (mag == 0u) {
        b = 0;
    } else {
        const int lz = count_leading_zeros32(mag);   // 9 .. 31
        b = ((uint64_t)(905 - lz) << 52) | (((uint64_t)mag << (21 + lz)) & 0x000fffffffffffffull);
    }
    return bits_to_double(b | ((uint64_t)(u & 0x80000000u) << 32));
}

// 256 / ln 2, and ln 2 / 256 split into a double and its remainder (the
// mathematical constants, rounded to nearest; computed with mpmath).
constexpr double kTangInvL = 369.3299304675746;
constexpr double kTangL1 = 2.7076061740622863e-03;
constexpr double kTangL2 = 9.058776616587108e-20;
constexpr double kTangShift = 6755399441055744.0;   // 1.5 * 2^52: rounds to an integer

// exp(x) for -707 <= x <= 700 by Tang's method; outside that range (and for
// NaN) the library exp. T: the 256 entries of exp2_table.inc.
SVM_HD double exp_tang(double x, const double *T)
{
    if (!(x >= -707.0 && x <= 700.0)) return exp(x);
    // n = round(x * 256 / ln 2): the shifted sum holds n in its low bits
    const double s = fma(x, kTangInvL, kTangShift);
    const int32_t n = (int32_t)(uint32_t)double_to_bits(s);
    const double nd = s - kTangShift;
    double r = fma(-nd, kTangL1, x);
    r = fma(-nd, kTangL2, r);
    // exp(r) - 1 = r + r^2 (1/2 + r (1/6 + r (1/24 + r / 120)))
    double q = fma(1.0 / 120.0, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(q, r * r, r);
    const double t = T[n & 255];
    const double y = fma(t, p, t);
    // times 2^m, m = floor(n / 256), on the exponent field (y stays normal)
    const int64_t m = (int64_t)(n >> 8);
    return bits_to_double(double_to_bits(y) + ((uint64_t)m << 52));
}

constexpr int kExp2TabLen = 256;

#if defined(__CUDACC__)
// The table in device memory; kernels copy it into shared memory once.
static __device__ const double kExp2Tab[kExp2TabLen] = {
#include "exp2_table.inc"
};
#endif

}  // namespace svmgb

#endif  // SVM_FP64_MATH_CUH
