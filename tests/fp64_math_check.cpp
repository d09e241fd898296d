// Host check of the FP64 helpers of the CUDA path (fp64_math.cuh): the same
// IEEE operations the device runs, compared with the conversion instruction
// and with long double exp.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fp64_math.cuh"

static const double T[256] = {
#include "exp2_table.inc"
};

int main(int argc, char **argv)
{
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
    // 2. exp_tang against long double exp, in units of the last place of the
    // correctly rounded value
    double worst = 0, wx = 0;
    long long n = 0;
    const long long N = 20000000;
    for (long long k = 0; k <= N; ++k) {
        const double x = -707.0 + 707.0 * (double)k / (double)N;
        const long double ref = expl((long double)x);
        const double got = svmgb::exp_tang(x, T);
        const double rd = (double)ref;
        if (rd == 0.0 || !std::isnormal(rd)) continue;
        const double ulp = nextafter(rd, INFINITY) - rd;
        const double err = (double)fabsl((long double)got - ref) / ulp;
        if (err > worst) { worst = err; wx = x; }
        ++n;
    }
    // special points
    const double sp[] = {0.0, -0.0, -1e-300, -1e-17, -0.5, -1.0, -0.00135, -0.0013538, -707.0, -706.99,
                         -100.25, 1e-10, 1.0, 0.6931471805599453, 700.0};
    for (double x : sp) {
        const long double ref = expl((long double)x);
        const double rd = (double)ref, got = svmgb::exp_tang(x, T);
        const double ulp = nextafter(rd, INFINITY) - rd;
        const double err = (double)fabsl((long double)got - ref) / ulp;
        if (err > worst) { worst = err; wx = x; }
    }
    printf("exp points %lld max_ulp %.4f at %.17g exp0 %a\n", n, worst, wx, svmgb::exp_tang(0.0, T));
    if (svmgb::exp_tang(0.0, T) != 1.0 || svmgb::exp_tang(-0.0, T) != 1.0) ++bad;
    // NaN and arguments outside the table range go to the library exp
    if (!std::isnan(svmgb::exp_tang(NAN, T)) || svmgb::exp_tang(-800.0, T) != exp(-800.0)) ++bad;
    if (worst > 1.0 + 1e-9) ++bad;   // faithful: within one unit in the last place
    return bad ? 1 : 0;
}
