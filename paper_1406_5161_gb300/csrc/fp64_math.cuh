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

SVM_HD uint32_t mul_hi32(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
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
// n comes from a 64-bit product of y 2^53 with 256/ln 2 (possibly one too
// small or too large), r from the fraction bits of y 2^64 minus those of
// n ln2/256 (ln2/256 known to 128 bits): the integer parts cancel, so the
// low 64 bits of each are enough, and the sign or size of the difference
// corrects n by one. exp(-r) by its Taylor polynomial of degree 5 in Q63
// (Horner, every intermediate positive; the innermost term, which needs
// only 2^-28, in 32 bits); 2^-(j/256) from the table T (Q63,
// expfx_table.inc); the product normalised and rounded once to a double.
// The fixed-point errors stay below 2^-58 of the result, so the result is
// within about 0.52 units in the last place. y outside [0, 700] (and NaN)
// goes to the library exp(-y). No FP64 arithmetic instruction is used on
// the integer path.
SVM_HD double exp_neg_fx(double y, const uint64_t *T)
{
    const uint64_t b = double_to_bits(y);
    if (b > kExpfxBits700) return exp(-y);   // y < 0, y > 700 or NaN
    // y = m 2^(be - 1075), so y 2^64 = m << sh, sh = be - 1011 <= 21
    const int be = (int)(b >> 52);
    const uint64_t m = (b & 0x000fffffffffffffull) | (be ? 0x0010000000000000ull : 0ull);
    const int sh = be - 1011;
    uint64_t y53, lo;   // y 2^53 (truncated) and the low 64 bits of y 2^64
    if (sh >= 11) {
        y53 = m << (sh - 11);
        lo = m << sh;
    } else if (sh >= 0) {
        y53 = m >> (11 - sh);
        lo = m << sh;
    } else {
        y53 = 0;   // y < 2^-11: n = 0
        lo = sh > -64 ? m >> -sh : 0ull;
    }
    uint32_t n = (uint32_t)(mul_hi64(y53, kExpfxInvL54) >> 43);
    // the low 64 bits of n ln2/256 in Q64: n LH + floor(n LL / 2^64)
    const uint64_t nll = ((uint64_t)n * (uint32_t)(kExpfxLL >> 32) +
                          (((uint64_t)n * (uint32_t)kExpfxLL) >> 32)) >> 32;
    uint64_t r = lo - ((uint64_t)n * kExpfxLH + nll);
    if ((int64_t)r < 0) {
        n -= 1;
        r += kExpfxLH;
    } else if (r >= kExpfxLH) {
        n += 1;
        r -= kExpfxLH;
    }
    // exp(-r) = 1 - r (1 - r (1/2 - r (1/6 - r (1/24 - r / 120)))), Q63
    const uint32_t r32 = (uint32_t)(r >> 32);   // r in Q32
    const uint32_t q4 = (uint32_t)(kExpfxC4 >> 31) - mul_hi32(r32, (uint32_t)(kExpfxC5 >> 31));
    uint64_t q = kExpfxC3 - mul_hi64(r, (uint64_t)q4 << 31);
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

// A value's (m, b - t) in one word, for rows read many times: m (signed, 25
// bits) in bits 5-31, b - t (0 .. 31 within the window) in bits 0-4.
SVM_HD uint32_t xd_word(uint32_t u, int tmin)
{
    return ((uint32_t)xd_mant(u) << 5) | (uint32_t)(xd_exp(u, tmin) - tmin);
}
SVM_HD int32_t xd_word_m(uint32_t w) { return (int32_t)w >> 5; }
SVM_HD int xd_word_e(uint32_t w) { return (int)(w & 31u); }

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
// to even. For the formats above the result is a normal number or zero. The
// magnitude is (a xor s) - s, s the sign mask; the limb holding the leading
// one and the two below it give a 96-bit window whose top 53 bits are the
// significand, the next bit the rounding bit, and the rest (with the limb
// below the window) the sticky bit.
SVM_HD double xd_round(const XdAcc &acc, int unit)
{
    const uint32_t s = (uint32_t)((int32_t)acc.w3 >> 31);
    XdAcc g;
    g.w0 = acc.w0 ^ s;
    g.w1 = acc.w1 ^ s;
    g.w2 = acc.w2 ^ s;
    g.w3 = acc.w3 ^ s;
    xd_add4(g, s & 1u, 0u, 0u, 0u);
    uint32_t a, b, c, rest;
    int top;
    if (g.w3) {
        a = g.w3; b = g.w2; c = g.w1; rest = g.w0; top = 3;
    } else if (g.w2) {
        a = g.w2; b = g.w1; c = g.w0; rest = 0u; top = 2;
    } else if (g.w1) {
        a = g.w1; b = g.w0; c = 0u; rest = 0u; top = 1;
    } else if (g.w0) {
        a = g.w0; b = 0u; c = 0u; rest = 0u; top = 0;
    } else {
        return 0.0;
    }
    const int lz = count_leading_zeros32(a);
    const uint32_t h = xd_funnel(b, a, lz), mid = xd_funnel(c, b, lz), low = c << lz;
    uint64_t mant = ((uint64_t)h << 21) | (mid >> 11);   // leading one at bit 52
    const bool half = (mid >> 10) & 1u;
    const bool sticky = ((mid & 0x3ffu) | low | rest) != 0u;
    int e = 32 * top + 31 - lz + unit;   // |a| 2^unit = 1.f 2^e
    if (half && (sticky || (mant & 1u))) {
        mant += 1;
        if (mant >> 53) { mant >>= 1; e += 1; }
    }
    const uint64_t bits = ((uint64_t)(e + 1023) << 52) | (mant & 0x000fffffffffffffull);
    return bits_to_double(bits | ((uint64_t)(s & 1u) << 63));
}

}  // namespace svmgb

#endif  // SVM_FP64_MATH_CUH
