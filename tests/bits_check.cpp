// Host check of the bit-pattern conversions in csrc/bits.cuh against
// independent references: the host compiler's own FP32 -> FP64 conversion
// (exact in IEEE 754), truncation toward zero formed from the rounded FP32
// conversion and nextafter, and magnitude order from fabs.  Prints one line
// per check and exits non-zero on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "bits.cuh"

using elder::d2f_trunc;
using elder::f2d_exact;
using elder::mag_bits;

static uint32_t fbits(float x) { uint32_t u; std::memcpy(&u, &x, 4); return u; }
static float ffrom(uint32_t u) { float x; std::memcpy(&x, &u, 4); return x; }
static uint64_t dbits(double x) { uint64_t u; std::memcpy(&u, &x, 8); return u; }
static double dfrom(uint64_t u) { double x; std::memcpy(&x, &u, 8); return x; }

// truncation toward zero of x to FP32, with the documented range handling:
// |x| < 2^-126 -> zero of x's sign, |x| >= 2^128 or NaN -> infinity of x's sign
static float trunc_ref(double x)
{
    const bool neg = std::signbit(x);
    if (std::isnan(x) || std::fabs(x) >= std::ldexp(1.0, 128)) return neg ? -INFINITY : INFINITY;
    if (std::fabs(x) < std::ldexp(1.0, -126)) return neg ? -0.0f : 0.0f;
    float t = (float)x;  // rounded to nearest
    if (std::fabs((double)t) > std::fabs(x)) t = std::nextafter(t, 0.0f);
    return t;
}

int main()
{
    std::mt19937_64 g(12345);
    long bad = 0, n = 0;
    // f2d_exact: every FP32 exponent and sign, random mantissas, the specials
    auto chk_w = [&](uint32_t u) {
        const float x = ffrom(u);
        const double a = f2d_exact(x), b = (double)x;
        ++n;
        if (std::isnan(b) ? !std::isnan(a) : dbits(a) != dbits(b)) {
            if (bad < 5) std::printf("f2d_exact mismatch at %08x\n", u);
            ++bad;
        }
    };
    for (uint32_t e = 0; e < 256; ++e)
        for (int k = 0; k < 2000; ++k) {
            const uint32_t m = (uint32_t)g() & 0x7FFFFFu;
            chk_w((e << 23) | m);
            chk_w(0x80000000u | (e << 23) | m);
        }
    for (uint32_t u : {0x00000000u, 0x80000000u, 0x00000001u, 0x807FFFFFu, 0x00800000u,
                       0x7F7FFFFFu, 0xFF7FFFFFu, 0x7F800000u, 0xFF800000u, 0x7FC00000u})
        chk_w(u);
    std::printf("f2d_exact: %ld values, %ld mismatches\n", n, bad);
    long bad_w = bad;

    // mag_bits: orders like |x|; NaN as +inf
    long bad_m = 0, nm = 0;
    for (int k = 0; k < 1000000; ++k) {
        const float a = ffrom((uint32_t)g()), b = ffrom((uint32_t)g());
        if (std::isnan(a) || std::isnan(b)) continue;
        ++nm;
        if ((std::fabs(a) < std::fabs(b)) != (mag_bits(a) < mag_bits(b))) ++bad_m;
        if ((std::fabs(a) == std::fabs(b)) != (mag_bits(a) == mag_bits(b))) ++bad_m;
    }
    if (mag_bits(ffrom(0x7FC00000u)) != 0x7F800000u || mag_bits(ffrom(0xFFC00001u)) != 0x7F800000u ||
        mag_bits(-0.0f) != 0u || mag_bits(-INFINITY) != 0x7F800000u)
        ++bad_m;
    std::printf("mag_bits: %ld pairs, %ld mismatches\n", nm, bad_m);

    // d2f_trunc: doubles across the FP32 range and beyond, both signs
    long bad_t = 0, nt = 0;
    std::uniform_int_distribution<int> ex(-140, 140);
    for (int k = 0; k < 2000000; ++k) {
        const double x = std::ldexp(1.0 + (double)(g() >> 11) * 0x1p-53, ex(g)) * ((g() & 1) ? -1 : 1);
        ++nt;
        if (fbits(d2f_trunc(x)) != fbits(trunc_ref(x))) {
            if (bad_t < 5) std::printf("d2f_trunc mismatch at %.17g\n", x);
            ++bad_t;
        }
    }
    for (double x : {0.0, -0.0, 1.0, -1.0, 0.5, 0x1p-126, -0x1p-127, 0x1p127, 0x1.fffffffffffffp127,
                     0x1p128, -0x1p200, 1e-300, (double)INFINITY, -(double)INFINITY, std::nan("")}) {
        ++nt;
        if (fbits(d2f_trunc(x)) != fbits(trunc_ref(x))) {
            std::printf("d2f_trunc mismatch at %.17g\n", x);
            ++bad_t;
        }
    }
    // powers of two (the line-search step length) convert exactly
    for (int k = -126; k < 128; ++k)
        if (d2f_trunc(std::ldexp(1.0, k)) != std::ldexp(1.0f, k)) ++bad_t;
    std::printf("d2f_trunc: %ld values, %ld mismatches\n", nt, bad_t);
    return (bad_w || bad_m || bad_t) ? 1 : 0;
}
