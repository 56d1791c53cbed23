// Host check of the double-float and fixed-point primitives of the FP64 block paths
// (paper_0706_3293_gb300/csrc/ef64.cuh, compiled here as plain C++) against long double
// and exact integer arithmetic, on seeded random operands.  Prints one line per primitive
// and exits non-zero on any violation of the bound each function states.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>

#include "ef64.cuh"

using ld = long double;
static int g_bad = 0;
static void report(const char *name, long n, long bad, double worst) {
    printf("%-14s %8ld cases  %ld violations  worst %.3g\n", name, n, bad, worst);
    if (bad) g_bad = 1;
}

int main() {
    std::mt19937_64 rng(20261203);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::uniform_int_distribution<int> X(-30, 30);
    const long NC = 200000;
    // TwoSum / TwoProd: exact
    {
        long bad = 0;
        for (long i = 0; i < NC; ++i) {
            const float a = (float)std::ldexp(U(rng), X(rng)), b = (float)std::ldexp(U(rng), X(rng));
            const ef::df s = ef::two_sum(a, b);
            if ((ld)s.hi + (ld)s.lo != (ld)a + (ld)b || s.hi != a + b) ++bad;
        }
        report("two_sum", NC, bad, 0.0);
        bad = 0;
        for (long i = 0; i < NC; ++i) {
            const float a = (float)std::ldexp(U(rng), X(rng)), b = (float)std::ldexp(U(rng), X(rng));
            const ef::df p = ef::two_prod(a, b);
            if ((ld)p.hi + (ld)p.lo != (ld)a * (ld)b) ++bad;
        }
        report("two_prod", NC, bad, 0.0);
    }
    // df_from_bits: |x - (hi + lo) 2^scale| < 2^-46 |x|
    {
        long bad = 0, n = 0;
        double worst = 0;
        for (long i = 0; i < NC; ++i) {
            const double x = std::ldexp(U(rng), X(rng) * 10);
            const int scale = X(rng) * 3;
            // stated domain: scaled magnitude between 2^-100 and 2^127
            if (x == 0.0 || std::ilogb(x) - scale < -99 || std::ilogb(x) - scale > 126) continue;
            const ef::df d = ef::df_from_bits(ef::d2u(x), scale);
            const ld err = std::fabs(((ld)d.hi + (ld)d.lo) * std::ldexp((ld)1, scale) - (ld)x) / std::fabs((ld)x);
            worst = std::fmax(worst, (double)err);
            ++n;
            if (err >= std::ldexp(1.0L, -46)) ++bad;
        }
        report("df_from_bits", n, bad, worst);
    }
    // bits_from_df: the binary64 nearest to (hi + lo) 2^scale (exact pair value in long double)
    {
        long bad = 0, n = 0;
        for (long i = 0; i < NC; ++i) {
            const float hi = (float)std::ldexp(U(rng), X(rng));
            if (hi == 0.0f) continue;
            const float lo = (float)(std::ldexp(U(rng), -24) * hi);    // |lo| < ulp-ish of hi
            const int scale = X(rng) * 4;
            const ef::df n2 = ef::fast_two_sum(hi, lo);
            const ld v = ((ld)n2.hi + (ld)n2.lo) * std::ldexp((ld)1, scale);
            const uint64_t got = ef::bits_from_df({hi, lo}, scale);
            ++n;
            if (got != ef::d2u((double)v)) ++bad;
        }
        report("bits_from_df", n, bad, 0.0);
    }
    // fix_from_bits: truncation toward zero of x 2^(FIX_BITS - (E - 1022)), |X| < 2^53
    {
        long bad = 0;
        for (long i = 0; i < NC; ++i) {
            const double x = std::ldexp(U(rng), X(rng));
            const int E = ef::exp_field(ef::d2u(x)) + (int)(rng() % 40);
            const ld want = std::trunc((ld)x * std::ldexp((ld)1, ef::FIX_BITS - (E - 1022)));
            const int64_t got = ef::fix_from_bits(ef::d2u(x), E);
            if ((ld)got != want || std::llabs(got) >= (1ll << ef::FIX_BITS)) ++bad;
        }
        report("fix_from_bits", NC, bad, 0.0);
    }
    // bits_from_int: T 2^k rounded to nearest even
    {
        long bad = 0;
        for (long i = 0; i < NC; ++i) {
            int64_t T = (int64_t)(rng() >> (rng() % 63));
            if (rng() & 1) T = -T;
            const int k = X(rng) * 10;
            const uint64_t got = ef::bits_from_int(T, k);
            const double want = std::ldexp((double)(ld)T, k);           // (double)(long double T): RNE
            if (got != ef::d2u(want)) ++bad;
        }
        report("bits_from_int", NC, bad, 0.0);
    }
    // fix_from_df: within 1/2 + 2^-8 units of the value
    {
        long bad = 0;
        double worst = 0;
        for (long i = 0; i < NC; ++i) {
            const double x = std::ldexp(U(rng), X(rng));
            const int E = ef::exp_field(ef::d2u(x)) + (int)(rng() % 20);
            const int scale = X(rng);
            const ef::df d = ef::df_from_bits(ef::d2u(std::ldexp(x, -scale)), 0);
            const ld unit = std::ldexp((ld)1, E - 1022 - ef::FIX_BITS);
            const ld val = ((ld)d.hi + (ld)d.lo) * std::ldexp((ld)1, scale) / unit;
            const int64_t got = ef::fix_from_df(d, E, scale);
            const double err = (double)std::fabs((ld)got - val);
            worst = std::fmax(worst, err);
            if (err > 0.5 + std::ldexp(1.0, -8)) ++bad;
        }
        report("fix_from_df", NC, bad, worst);
    }
    // df_from_fix: relative error below 2^-46 of T 2^(E - 1022 - FIX_BITS + extra - scale)
    {
        long bad = 0, n = 0;
        double worst = 0;
        for (long i = 0; i < NC; ++i) {
            int64_t T = (int64_t)(rng() >> (1 + rng() % 62));
            if (T == 0) continue;
            if (rng() & 1) T = -T;
            const int E = 1000 + X(rng), extra = X(rng), scale = X(rng);
            const ld want = (ld)T * std::ldexp((ld)1, E - 1022 - ef::FIX_BITS + extra - scale);
            // stated domain: every 21-bit piece stays a normal float after scaling
            const int u = E - 1022 - ef::FIX_BITS + extra - scale;
            if (u < -126 || std::ilogb((double)std::fabs(want)) > 126) continue;
            const ef::df d = ef::df_from_fix(T, E, extra, scale);
            const ld err = std::fabs(((ld)d.hi + (ld)d.lo) - want) / std::fabs(want);
            worst = std::fmax(worst, (double)err);
            ++n;
            if (err >= std::ldexp(1.0L, -46)) ++bad;
        }
        report("df_from_fix", n, bad, worst);
    }
    // df_add / df_mul: relative error below 2^-44 (double-float accuracy)
    {
        long bad = 0;
        double worst = 0;
        for (long i = 0; i < NC; ++i) {
            const double x = U(rng) * std::ldexp(1.0, X(rng)), y = U(rng) * std::ldexp(1.0, X(rng) / 4);
            const ef::df a = ef::df_from_bits(ef::d2u(x), 0), b = ef::df_from_bits(ef::d2u(y), 0);
            const ld ea = (ld)a.hi + (ld)a.lo, eb = (ld)b.hi + (ld)b.lo;
            const ef::df m = ef::df_mul(a, b);
            const ld e1 = std::fabs(((ld)m.hi + (ld)m.lo) - ea * eb) / std::fabs(ea * eb);
            worst = std::fmax(worst, (double)e1);
            if (e1 >= std::ldexp(1.0L, -44)) ++bad;
            if (std::fabs(ea + eb) > std::ldexp(1.0L, -20) * (std::fabs(ea) + std::fabs(eb))) {
                const ef::df s = ef::df_add(a, b);
                const ld e2 = std::fabs(((ld)s.hi + (ld)s.lo) - (ea + eb)) / std::fabs(ea + eb);
                if (e2 >= std::ldexp(1.0L, -44)) ++bad;
            }
        }
        report("df_add/df_mul", NC, bad, worst);
    }
    return g_bad;
}
