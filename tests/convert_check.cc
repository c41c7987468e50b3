// Host check of the integer float <-> double conversions of the CUDA library
// against the C conversions, bit for bit.  Prints the number of mismatches of each
// sweep; exits non-zero if there is any.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "cdbm_convert.h"

static uint64_t bits64(double v) { uint64_t b; std::memcpy(&b, &v, 8); return b; }
static uint32_t bits32(float v) { uint32_t b; std::memcpy(&b, &v, 4); return b; }
static double from64(uint64_t b) { double v; std::memcpy(&v, &b, 8); return v; }

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64()    // splitmix64
{
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static long narrow_mismatch(double v)
{
    const float want = (float)v, got = cdbm::narrow_f64(v);
    if (std::isnan(want)) return std::isnan(got) ? 0 : 1;
    return bits32(want) != bits32(got);
}

int main()
{
    // float -> double: every float bit pattern
    long bad_w = 0;
    for (uint64_t b = 0; b <= 0xffffffffull; ++b) {
        float v;
        const uint32_t b32 = (uint32_t)b;
        std::memcpy(&v, &b32, 4);
        const double want = (double)v, got = cdbm::widen_f32(v);
        if (std::isnan(want) ? !std::isnan(got) : bits64(want) != bits64(got)) ++bad_w;
    }
    // double -> float: random bit patterns, random values around the float range,
    // exact ties (both parities) and the ends of the normal float range
    long bad_r = 0, bad_e = 0, bad_t = 0, bad_b = 0;
    for (long k = 0; k < 20000000; ++k) bad_r += narrow_mismatch(from64(next_u64()));
    for (long k = 0; k < 20000000; ++k) {
        const uint64_t r = next_u64();
        const uint64_t e = 860 + (r >> 53) % 330;                 // exponents 860..1189
        bad_e += narrow_mismatch(from64((r & 0x800fffffffffffffull) | (e << 52)));
    }
    for (long k = 0; k < 4000000; ++k) {
        const uint64_t r = next_u64();
        const uint64_t e = 897 + (r >> 53) % 254;
        const uint64_t frac = (r & 0x000fffffe0000000ull) | 0x10000000ull;   // dropped bits = one half
        bad_t += narrow_mismatch(from64((r & 0x8000000000000000ull) | (e << 52) | frac));
    }
    const double edges[] = {0.0, -0.0, FLT_MAX, -FLT_MAX, FLT_MIN, -FLT_MIN, DBL_MIN, DBL_MAX, INFINITY,
                            -INFINITY, NAN, 1.0, -1.0, 0.5, 3.0};
    for (double v : edges) {
        bad_b += narrow_mismatch(v);
        for (int d = -40; d <= 40; ++d) bad_b += narrow_mismatch(from64(bits64(v) + d));
    }
    std::printf("widen %ld narrow_random %ld narrow_float_range %ld narrow_ties %ld narrow_edges %ld\n", bad_w,
                bad_r, bad_e, bad_t, bad_b);
    return (bad_w | bad_r | bad_e | bad_t | bad_b) ? 1 : 0;
}
