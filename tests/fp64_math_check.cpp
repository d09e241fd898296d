// Host check of the FP64 helpers of the CUDA path (fp64_math.cuh): the same
// IEEE and integer operations the device runs, compared with the conversion
// instruction, with long double exp, and (xd mode, driven by
// test_fp64_math_cpu.py) with exact rational arithmetic.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>

#include "fp64_math.cuh"

static const uint64_t T[256] = {SVM_EXPFX_TABLE};

// "xd" mode: cases on standard input, one per line. A line
//   D n x_1 z_1 ... x_n z_n    (float bit patterns in hex)
// prints the exact inner product rounded by xd_round (as the bits of a
// double), computed three ways that must agree: in order, in reverse order,
// and split over 4 lanes whose accumulators are then added; or "off" when
// the format rejects the operands. A line
//   R hi lo unit              (a 128-bit integer and a unit exponent)
// prints xd_round(hi:lo, unit).
static int xd_mode()
{
    char tag[4];
    int bad = 0;
    while (scanf("%3s", tag) == 1) {
        if (tag[0] == 'R') {
            unsigned long long hi, lo;
            int unit;
            if (scanf("%llx %llx %d", &hi, &lo, &unit) != 3) return 2;
            svmgb::XdAcc a;
            a.w0 = (uint32_t)lo;
            a.w1 = (uint32_t)(lo >> 32);
            a.w2 = (uint32_t)hi;
            a.w3 = (uint32_t)(hi >> 32);
            const double r = svmgb::xd_round(a, unit);
            printf("%016llx\n", (unsigned long long)svmgb::double_to_bits(r));
            continue;
        }
        int n;
        if (scanf("%d", &n) != 1) return 2;
        uint32_t *x = new uint32_t[n > 0 ? n : 1], *z = new uint32_t[n > 0 ? n : 1];
        int bmax = 0, bmin = 255;
        bool sub = false;
        for (int i = 0; i < n; ++i) {
            unsigned a, b;
            if (scanf("%x %x", &a, &b) != 2) return 2;
            x[i] = a;
            z[i] = b;
            for (uint32_t u : {x[i], z[i]}) {
                const int e = (int)((u >> 23) & 0xff);
                if (e == 0 && (u & 0x7fffffu)) sub = true;
                if (e != 0) {
                    bmax = e > bmax ? e : bmax;
                    bmin = e < bmin ? e : bmin;
                }
            }
        }
        const svmgb::XdFormat f = svmgb::xd_format(bmax, bmin, n, sub);
        if (!f.on) {
            printf("off\n");
        } else {
            svmgb::XdAcc a = svmgb::xd_zero(), r = a, l[4] = {a, a, a, a};
            for (int i = 0; i < n; ++i) {
                const int k = svmgb::xd_exp(x[i], f.tmin) + svmgb::xd_exp(z[i], f.tmin) + f.bias;
                if (k < 0 || k > 63) ++bad;
                svmgb::xd_add(a, svmgb::xd_mant(x[i]), svmgb::xd_mant(z[i]), k);
                svmgb::xd_add(l[i & 3], svmgb::xd_mant(x[i]), svmgb::xd_mant(z[i]), k);
            }
            // the row-pass convention: the row side as an (m, b - t) word, the
            // target side's exponent stored as b + bias + t
            svmgb::XdAcc w = svmgb::xd_zero();
            for (int i = 0; i < n; ++i) {
                const uint32_t xw = svmgb::xd_word(x[i], f.tmin);
                const int te = svmgb::xd_exp(z[i], f.tmin) + f.bias + f.tmin;
                svmgb::xd_add(w, svmgb::xd_word_m(xw), svmgb::xd_mant(z[i]), svmgb::xd_word_e(xw) + te);
            }
            if (memcmp(&a, &w, sizeof a) != 0) ++bad;
            for (int i = n - 1; i >= 0; --i)
                svmgb::xd_add(r, svmgb::xd_mant(x[i]), svmgb::xd_mant(z[i]),
                              svmgb::xd_exp(x[i], f.tmin) + svmgb::xd_exp(z[i], f.tmin) + f.bias);
            svmgb::xd_add(l[0], l[2]);
            svmgb::xd_add(l[1], l[3]);
            svmgb::xd_add(l[0], l[1]);
            if (memcmp(&a, &r, sizeof a) != 0 || memcmp(&a, &l[0], sizeof a) != 0) ++bad;
            printf("%016llx\n", (unsigned long long)svmgb::double_to_bits(svmgb::xd_round(a, f.unit)));
        }
        delete[] x;
        delete[] z;
    }
    printf("xd bad %d\n", bad);
    return bad ? 1 : 0;
}

int main(int argc, char **argv)
{
    if (argc > 1 && strcmp(argv[1], "xd") == 0) return xd_mode();
    const long long stride = argc > 1 ? atoll(argv[1]) : 1;
    // 1. widen_f32 against the conversion, over float bit patterns
    long long checked = 0, bad = 0;
    for (unsigned long long b = 0; b < (1ull << 32); b += (b < 0x01000000u) ? 1 : stride) {
        const uint32_t u = (uint32_t)b;
        if (((u >> 23) & 0xff) == 0xff) continue;   // inf / NaN are rejected at ingest
        float f;
        memcpy(&f, &u, 4);
        const double a = (double)f, w = svmgb::widen_f32(f);
        if (memcmp(&a, &w, 8) != 0) {
            if (bad < 5) printf("widen mismatch %08x: %a vs %a\n", u, a, w);
            ++bad;
        }
        ++checked;
    }
    // all subnormal patterns with the sign bit set too
    for (uint32_t m = 0; m < 0x00800000u; m += 1) {
        const uint32_t u = 0x80000000u | m;
        float f;
        memcpy(&f, &u, 4);
        const double a = (double)f, w = svmgb::widen_f32(f);
        if (memcmp(&a, &w, 8) != 0) ++bad;
        ++checked;
    }
    printf("widen checked %lld bad %lld\n", checked, bad);
    // 2. exp_neg_fx against long double exp, in units of the last place of
    // the correctly rounded value
    double worst = 0, wx = 0;
    long long n = 0;
    auto check = [&](double y) {
        const long double ref = expl(-(long double)y);
        const double rd = (double)ref, got = svmgb::exp_neg_fx(y, T);
        if (rd == 0.0 || !std::isnormal(rd)) return;
        const double ulp = nextafter(rd, INFINITY) - rd;
        const double err = (double)fabsl((long double)got - ref) / ulp;
        if (err > worst) { worst = err; wx = y; }
        ++n;
    };
    const long long N = 20000000;
    for (long long k = 0; k <= N; ++k) check(700.0 * (double)k / (double)N);
    // small arguments on a log scale, and points around multiples of ln2/256
    for (int e = -80; e <= 9; ++e)
        for (int k = 0; k < 4096; ++k) check(ldexp(1.0 + k / 4096.0, e));
    for (int j = 0; j <= 256 * 1009; j += 97) {
        const double c = j * 0.0027076061740622863;
        check(c);
        check(nextafter(c, 0.0));
        check(nextafter(c, INFINITY));
    }
    const double sp[] = {0.0, 1e-300, 4.9e-324, 1e-17, 5.551115123125783e-17, 1.1102230246251565e-16, 0.5, 1.0,
                         0.0027076061740622863, 0.0013538, 100.25, 699.9999999999999, 700.0};
    for (double y : sp) check(y);
    printf("exp points %lld max_ulp %.4f at %.17g\n", n, worst, wx);
    if (svmgb::exp_neg_fx(0.0, T) != 1.0 || svmgb::exp_neg_fx(1e-300, T) != 1.0) ++bad;
    // outside [0, 700] and NaN: the library exp
    if (!std::isnan(svmgb::exp_neg_fx(NAN, T)) || svmgb::exp_neg_fx(800.0, T) != exp(-800.0) ||
        svmgb::exp_neg_fx(-0.5, T) != exp(0.5) || svmgb::exp_neg_fx(-0.0, T) != 1.0)
        ++bad;
    if (worst > 0.53) ++bad;   // the fixed-point errors stay far below half a unit
    return bad ? 1 : 0;
}
