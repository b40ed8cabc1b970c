// Host-side check of the double-float arithmetic in csrc/df64.cuh (the same
// __host__ __device__ functions the df64 kernels use), against FP64 / long
// double references.  Built with nvcc as host code and run on the CPU by
// tests/test_df64_host.py; prints one line per property and exits non-zero on
// a failure.
#include <cmath>
#include <cstdio>
#include <random>

#include "../paper_1402_7285_gb300/csrc/df64.cuh"

static std::mt19937_64 rng(1234);

static float rnd_float(int emin, int emax) {
    std::uniform_real_distribution<double> u(0.5, 1.0);
    const int e = emin + (int)(rng() % (unsigned)(emax - emin + 1));
    const double s = (rng() & 1) ? -1.0 : 1.0;
    return (float)(s * std::ldexp(u(rng), e));
}

static df rnd_df(int emin, int emax) {
    const float hi = rnd_float(emin, emax);
    // a low part below half an ulp of hi: a normalised pair
    const float lo = (float)(std::ldexp((double)rnd_float(-1, -1), std::ilogb(hi) - 25));
    return df_fast_two_sum(hi, lo);
}

static long double val(df x) { return (long double)x.hi + (long double)x.lo; }

int main() {
    int fails = 0;
    const int N = 200000;

    // TwoSum and TwoProd are error-free: s + e == a + b, p + e == a * b exactly
    long bad = 0;
    for (int i = 0; i < N; ++i) {
        const float a = rnd_float(-20, 20), b = rnd_float(-20, 20);
        const df s = df_two_sum(a, b);
        if ((double)s.hi + (double)s.lo != (double)a + (double)b) ++bad;
        const float p = DF_MUL(a, b);
        const float e = fmaf(a, b, -p);
        if ((double)p + (double)e != (double)a * (double)b) ++bad;
    }
    std::printf("error-free transformations: %ld inexact of %d\n", bad, 2 * N);
    fails += bad != 0;

    // df add / multiply / fma: relative error below 2^-44 of the exact result
    // (the magnitude of the operands for the add: cancellation is absolute)
    double worst_add = 0, worst_mul = 0, worst_fma = 0, worst_mulf = 0, worst_fmaf = 0;
    for (int i = 0; i < N; ++i) {
        const df a = rnd_df(-10, 10), b = rnd_df(-10, 10), c = rnd_df(-10, 10);
        const float f = rnd_float(-10, 10);
        const long double A = val(a), B = val(b), C = val(c), F = f;
        worst_add = std::fmax(worst_add, (double)(std::fabs(val(a + b) - (A + B)) / (std::fabs(A) + std::fabs(B))));
        worst_mul = std::fmax(worst_mul, (double)(std::fabs(val(a * b) - A * B) / std::fabs(A * B)));
        worst_fma = std::fmax(worst_fma,
                              (double)(std::fabs(val(fma(a, b, c)) - (A * B + C)) / (std::fabs(A * B) + std::fabs(C))));
        worst_mulf = std::fmax(worst_mulf, (double)(std::fabs(val(mul_f(a, f)) - A * F) / std::fabs(A * F)));
        worst_fmaf = std::fmax(worst_fmaf, (double)(std::fabs(val(fma_f(a, f, c)) - (A * F + C)) /
                                                    (std::fabs(A * F) + std::fabs(C))));
    }
    const double tol = std::ldexp(1.0, -44);
    std::printf("df add %.3g mul %.3g fma %.3g mul_f %.3g fma_f %.3g (bound %.3g)\n", worst_add, worst_mul,
                worst_fma, worst_mulf, worst_fmaf, tol);
    fails += !(worst_add < tol && worst_mul < tol && worst_fma < tol && worst_mulf < tol && worst_fmaf < tol);

    // lazy accumulation (the products' inner loop): sums of K products
    // a_k b_k, relative to sum |a_k b_k|, below K * 2^-46
    double worst_sum = 0, worst_sumf = 0;
    const int K = 64;
    for (int t = 0; t < 5000; ++t) {
        DfSum s, sf;
        s.zero();
        sf.zero();
        long double ref = 0, mag = 0, reff = 0, magf = 0;
        for (int k = 0; k < K; ++k) {
            const df a = rnd_df(-6, 6), b = rnd_df(-6, 6);
            const float f = rnd_float(-6, 6);
            s.add_prod(a, b);
            sf.add_prod(a, f);
            ref += val(a) * val(b);
            mag += std::fabs(val(a) * val(b));
            reff += val(a) * (long double)f;
            magf += std::fabs(val(a) * (long double)f);
        }
        worst_sum = std::fmax(worst_sum, (double)(std::fabs(val(s.value()) - ref) / mag));
        worst_sumf = std::fmax(worst_sumf, (double)(std::fabs(val(sf.value()) - reff) / magf));
    }
    const double tol_sum = K * std::ldexp(1.0, -46);
    std::printf("lazy sums of %d products: df %.3g, FP32 operand %.3g (bound %.3g)\n", K, worst_sum, worst_sumf,
                tol_sum);
    fails += !(worst_sum < tol_sum && worst_sumf < tol_sum);

    // an identity block's term (add_val) gives the same bits as the product
    // with 1 (and the zero entries of the block change nothing)
    long diff = 0;
    for (int t = 0; t < N / 10; ++t) {
        DfSum p, q;
        p.zero();
        q.zero();
        for (int k = 0; k < 8; ++k) {
            const df a = rnd_df(-6, 6), x = rnd_df(-6, 6);
            const float xf = rnd_float(-6, 6);
            p.add_prod(a, x);
            q.add_prod(a, x);
            p.add_prod(df(1.0f), xf);
            p.add_prod(df(0.0f), x);
            q.add_val(xf);
        }
        const df pv = p.value(), qv = q.value();
        if (pv.hi != qv.hi || pv.lo != qv.lo) ++diff;
    }
    std::printf("identity-block shortcut: %ld differing sums of %d\n", diff, N / 10);
    fails += diff != 0;

    // a double splits into hi + lo with |value - (hi + lo)| below 2^-48 relative
    double worst_split = 0;
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    for (int i = 0; i < N; ++i) {
        const double v = std::ldexp(u(rng), (int)(rng() % 40) - 20);
        if (v == 0.0) continue;
        worst_split = std::fmax(worst_split, std::fabs(((double)df(v) - v) / v));
    }
    std::printf("double to df split: %.3g (bound %.3g)\n", worst_split, std::ldexp(1.0, -48));
    fails += !(worst_split < std::ldexp(1.0, -48));

    std::printf(fails ? "FAIL\n" : "OK\n");
    return fails;
}
