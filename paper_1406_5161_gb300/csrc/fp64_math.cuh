// FP64 building blocks for the row passes of the FP64 mode.
//
// On this part the FP64 pipe issues about two operations per clock per SM
// (measured: 1.6 dependent-free DFMA per clock per SM), and a float -> double
// conversion instruction takes a slot of that pipe too. The RBF kernel value
// K = exp(-gamma ||x - z||^2) of Section IV-E is the bulk of the FP64 work of
// the SMO step (Algorithm 2's inner product and the exponential, twice per
// active row) and of the gradient reconstruction (Algorithm 6). These helpers
// give FP64 results (or better) while moving that work onto the integer
// pipes:
//
//   widen_f32(x)       the float x as a double, exactly (the same value as
//                      the conversion instruction), by integer operations on
//                      the bit pattern;
//   exp_neg_fx(y, T)   exp(-y), y >= 0, in fixed-point integer arithmetic
//                      after the table-driven method of P. T. P. Tang,
//                      "Table-driven implementation of the exponential
//                      function in IEEE floating-point arithmetic", ACM TOMS
//                      15(2), 1989; within 0.53 units in the last place;
//   xd_*               inner products of float rows, exact in 128-bit
//                      integers and rounded once to the nearest double.
//
// They are written for host and device alike: the host build computes the
// same bits, which is how tests/test_fp64_math_cpu.py checks them without a
// GPU (against the conversion, long double exp and exact rationals).
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

SVM_HD uint64_t mul_hi64(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

SVM_HD int count_leading_zeros64(uint64_t v)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

#include "expfx_table.inc"

constexpr int kExpfxTabLen = 256;
constexpr uint64_t kExpfxBits700 = 0x4085e00000000000ull;   // the bits of 700.0

// exp(-y) for 0 <= y <= 700 in fixed-point integer arithmetic, after the
// table-driven method of P. T. P. Tang (ACM TOMS 15(2), 1989):
//   y = n ln2/256 + r, n = floor(y 256 / ln 2), 0 <= r < ln2/256,
//   exp(-y) = 2^-(n div 256) * 2^-((n mod 256)/256) * exp(-r).
// y is taken exactly into Q64 (64 fraction bits; below 2^-64 it counts as
// 0); n from a 64-bit product with 256/ln 2, corrected by one from the
// remainder r = y - n ln2/256, which is formed with ln2/256 to 128 bits;
// exp(-r) by its Taylor polynomial of degree 5 in Q63 (Horner, every
// intermediate positive); 2^-(j/256) from the table T (Q63, expfx_table.inc);
// the product normalised and rounded once to a double. The fixed-point
// errors stay below 2^-58 of the result, so the result is within about 0.52
// units in the last place. y outside [0, 700] (and NaN) goes to the library
// exp(-y). No FP64 arithmetic instruction is used on the integer path.
SVM_HD double exp_neg_fx(double y, const uint64_t *T)
{
    typedef unsigned __int128 u128;
    const uint64_t b = double_to_bits(y);
    if (b > kExpfxBits700) return exp(-y);   // y < 0, y > 700 or NaN
    // y = m 2^(be - 1075); in Q64: m << (be - 1011), at most 21 here
    const int be = (int)(b >> 52);
    const uint64_t m = (b & 0x000fffffffffffffull) | (be ? 0x0010000000000000ull : 0ull);
    const int sh = be - 1011;
    uint64_t hi = 0, lo = 0;
    if (sh >= 0) {
        lo = m << sh;
        hi = sh ? m >> (64 - sh) : 0ull;
    } else if (sh > -64) {
        lo = m >> -sh;
    }
    // n: (y 2^53) (256/ln2 2^54) / 2^(64 + 43), then corrected from r
    uint32_t n = (uint32_t)(mul_hi64((hi << 53) | (lo >> 11), kExpfxInvL54) >> 43);
    const u128 yq = ((u128)hi << 64) | lo;
    u128 nl = (u128)n * kExpfxLH + (((u128)n * kExpfxLL) >> 64);
    if (yq < nl) {
        n -= 1;
        nl -= kExpfxLH;
    } else if (yq - nl >= (u128)kExpfxLH) {
        n += 1;
        nl += kExpfxLH;
    }
    const uint64_t r = (uint64_t)(yq - nl);   // Q64, below 2^56
    // exp(-r) = 1 - r (1 - r (1/2 - r (1/6 - r (1/24 - r / 120)))), Q63
    uint64_t q = kExpfxC4 - mul_hi64(r, kExpfxC5);
    q = kExpfxC3 - mul_hi64(r, q);
    q = kExpfxC2 - mul_hi64(r, q);
    q = 0x8000000000000000ull - mul_hi64(r, q);
    const uint64_t e = 0x8000000000000000ull - mul_hi64(r, q);
    // 2^-(j/256) exp(-r) in Q62: in (2^60.99, 2^62]
    const uint64_t z = mul_hi64(T[n & 255u], e);
    const int lz = count_leading_zeros64(z);   // 1 .. 3
    const uint64_t zn = z << lz;              // leading one at bit 63
    uint64_t mant = (zn >> 11) + ((zn >> 10) & 1u);
    int ex = 1 - lz - (int)(n >> 8);          // z / 2^62 = (zn / 2^63) 2^(1 - lz)
    if (mant >> 53) {
        mant >>= 1;
        ex += 1;
    }
    return bits_to_double(((uint64_t)(ex + 1023) << 52) | (mant & 0x000fffffffffffffull));
}

#if defined(__CUDACC__)
// The table in device memory; kernels copy it into shared memory once.
static __device__ const uint64_t kExpfxTab[kExpfxTabLen] = {SVM_EXPFX_TABLE};
#endif

// ---- exact inner products of float-valued rows (a fused dot product)
//
// A finite float v is m 2^(b - 150): b its biased exponent (1..254 for a
// normal number), m = 2^23 + its 23 fraction bits, with v's sign; zero has
// m = 0. Take G >= every b of the operands and s = min(63, 79 - bitlen(L)),
// L the longest row. When every nonzero value has b >= t = G - floor(s / 2),
// each product x z is the integer (m_x m_z) << k, k = b_x + b_z + s - 2G in
// [0, s], in units of 2^(2G - 300 - s): |m_x m_z| < 2^48, so a sum of up to
// L products stays below 2^(bitlen(L) + 48 + s) <= 2^127 in magnitude and a
// 128-bit two's-complement accumulator (four 32-bit limbs) holds the inner
// product exactly. xd_round then rounds it once to the nearest double (ties
// to even). The result is the exact inner product correctly rounded: at
// least as accurate as FP64 summation in any order, and the same whatever
// the order of the terms, their split over lanes, and the G and s used. All
// of it is integer arithmetic, which leaves the FP64 pipe to the
// exponentials. With k < 64 a product lands at limb offset 0 or 1, so one
// accumulation is a multiply, four shifts, four selects and a four-limb add.
struct XdFormat {
    int on;     // 1: every nonzero value lies in the window
    int bias;   // s - 2G: k = b_x + b_z + bias
    int tmin;   // t: the exponent given to zeros (their m is 0)
    int unit;   // 2G - 300 - s: the accumulator counts units of 2^unit
};

SVM_HD int bit_length32(uint32_t v)
{
    return v ? 32 - count_leading_zeros32(v) : 0;
}

// The format for operands whose nonzero values have biased exponents in
// [bmin, bmax] (bmin > bmax: no nonzero value), rows of at most maxlen
// entries; subnormal values (b = 0, m != 0) leave the format off.
SVM_HD XdFormat xd_format(int bmax, int bmin, int maxlen, bool subnormal)
{
    XdFormat f;
    int s = 79 - bit_length32((uint32_t)(maxlen > 0 ? maxlen : 1));
    if (s > 63) s = 63;
    const int G = bmin > bmax ? 127 : bmax;
    int t = G - s / 2;
    if (t < 1) t = 1;
    f.on = !subnormal && (bmin > bmax || bmin >= t) && G <= 254;
    f.bias = s - 2 * G;
    f.tmin = t;
    f.unit = 2 * G - 300 - s;
    return f;
}

// b of a value's bits, zeros raised to tmin (their product is 0 whatever k)
SVM_HD int xd_exp(uint32_t u, int tmin)
{
    const int b = (int)((u >> 23) & 0xffu);
    return b > tmin ? b : tmin;
}

// m with the value's sign (0 for zero)
SVM_HD int32_t xd_mant(uint32_t u)
{
    const int32_t m = (u & 0x7f800000u) ? (int32_t)((u & 0x007fffffu) | 0x00800000u) : 0;
    return (u >> 31) ? -m : m;
}

// 128-bit two's-complement accumulator, least significant limb first
struct XdAcc {
    uint32_t w0, w1, w2, w3;
};

SVM_HD XdAcc xd_zero()
{
    XdAcc a;
    a.w0 = a.w1 = a.w2 = a.w3 = 0u;
    return a;
}

// the high word of (hi:lo) << r, 0 <= r <= 31
SVM_HD uint32_t xd_funnel(uint32_t lo, uint32_t hi, int r)
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, (unsigned)r);
#else
    return r ? (hi << r) | (lo >> (32 - r)) : hi;
#endif
}

// a += (l3:l2:l1:l0), carries through the four limbs
SVM_HD void xd_add4(XdAcc &a, uint32_t l0, uint32_t l1, uint32_t l2, uint32_t l3)
{
#if defined(__CUDA_ARCH__)
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2), "+r"(a.w3)
        : "r"(l0), "r"(l1), "r"(l2), "r"(l3));
#else
    uint64_t t = (uint64_t)a.w0 + l0;
    a.w0 = (uint32_t)t;
    t = (uint64_t)a.w1 + l1 + (t >> 32);
    a.w1 = (uint32_t)t;
    t = (uint64_t)a.w2 + l2 + (t >> 32);
    a.w2 = (uint32_t)t;
    a.w3 = a.w3 + l3 + (uint32_t)(t >> 32);
#endif
}

SVM_HD void xd_add(XdAcc &a, const XdAcc &b)
{
    xd_add4(a, b.w0, b.w1, b.w2, b.w3);
}

// a += (mx mz) << k, 0 <= k <= 63: the product (a signed 48-bit integer)
// shifted by r = k mod 32 into three limbs, placed at limb offset k / 32
SVM_HD void xd_add(XdAcc &a, int32_t mx, int32_t mz, int k)
{
    const int64_t p = (int64_t)mx * (int64_t)mz;
    const uint32_t plo = (uint32_t)(uint64_t)p, phi = (uint32_t)((uint64_t)p >> 32);
    const uint32_t sx = (uint32_t)((int32_t)phi >> 31);   // the sign, extended
    const int r = k & 31;
    const uint32_t t0 = plo << r;
    const uint32_t t1 = xd_funnel(plo, phi, r);
    const uint32_t t2 = xd_funnel(phi, sx, r);
    if (k & 32) xd_add4(a, 0u, t0, t1, t2);
    else xd_add4(a, t0, t1, t2, sx);
}

// The double nearest to a 2^unit (a read as a signed 128-bit integer), ties
// to even. For the formats above the result is a normal number or zero.
SVM_HD double xd_round(const XdAcc &acc, int unit)
{
    typedef unsigned __int128 u128;
    const u128 a = ((u128)acc.w3 << 96) | ((u128)acc.w2 << 64) | ((u128)acc.w1 << 32) | (u128)acc.w0;
    if (a == 0) return 0.0;
    const bool neg = (acc.w3 >> 31) != 0;
    u128 mag = neg ? (u128)0 - a : a;
    const uint64_t h0 = (uint64_t)(mag >> 64);
    const int lz = h0 ? count_leading_zeros64(h0) : 64 + count_leading_zeros64((uint64_t)mag);
    mag <<= lz;   // leading one at bit 127
    const uint64_t hi = (uint64_t)(mag >> 64), lo = (uint64_t)mag;
    uint64_t m = hi >> 11;   // 53 bits
    const bool half = (hi >> 10) & 1u;
    const bool sticky = (hi & 0x3ffu) != 0 || lo != 0;
    int e = 127 - lz + unit;   // |a| 2^unit = 1.f 2^e
    if (half && (sticky || (m & 1u))) {
        m += 1;
        if (m >> 53) { m >>= 1; e += 1; }
    }
    const uint64_t bits = ((uint64_t)(e + 1023) << 52) | (m & 0x000fffffffffffffull);
    return bits_to_double(bits | (neg ? 0x8000000000000000ull : 0));
}

}  // namespace svmgb

#endif  // SVM_FP64_MATH_CUH
