// Host checks of the device arithmetic helpers that the kernels share with
// the host build (common.cuh, regfft.cuh) against their plain definitions.
// Prints one line per check: "<name> <cases> <failures> [<max error>]".
#include "../../paper_2003_03931_gb300/csrc/common.cuh"
#include "../../paper_2003_03931_gb300/csrc/regfft.cuh"

#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

using namespace pmpm;

static unsigned long long rng_state = 0x9E3779B97F4A7C15ull;
static unsigned long long next_u64() {
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return rng_state;
}
static float bits_float(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// round-half-even of p 2^24 through long double arithmetic and llrint
static void check_fix24() {
    long long n = 0, bad = 0;
    auto one = [&](float p) {
        if (!(fabsf(p) < 1048576.f)) return;
        ++n;
        if (fix24_rn(p) != llrint((double)p * 16777216.0)) ++bad;
    };
    for (int i = 0; i < 4000000; ++i) one(bits_float((uint32_t)next_u64()));
    for (long long j = -200000; j < 200000; ++j) one((float)(((double)j + 0.5) / 16777216.0));
    printf("fix24 %lld %lld\n", n, bad);
}

// The 128-bit moments of the dispersion: (lo, hi) += x^2 and
// (lo, hi) += floor(S^2 / n), against unsigned __int128 arithmetic, for
// random and extreme arguments, accumulated over many terms (carries)
static void check_moments() {
    long long n = 0, bad = 0;
    unsigned long long lo = 0, hi = 0, lo2 = 0, hi2 = 0;
    unsigned __int128 ref = 0, ref2 = 0;
    for (int i = 0; i < 2000000; ++i) {
        // up to 2^45, and below 2^32 (the divisions' 32-bit path) a third of the time
        long long x = (long long)(next_u64() >> (i % 3 == 0 ? 19 : (i % 3 == 1 ? 21 : 34)));
        if (next_u64() & 1) x = -x;
        if (i % 101 == 0) x = (i & 1) ? (1ll << 44) - 1 : -((1ll << 44) - 1);
        if (i == 7 || i == 8) x = (i & 1) ? -0x7fffffffffffffffll : 0x7fffffffffffffffll;
        const unsigned __int128 ux = (unsigned __int128)(x < 0 ? -x : x);
        add_square128(x, lo, hi);
        ref += ux * ux;
        int cnt = (int)(next_u64() % 70000) + 1;
        if (i % 97 == 0) cnt = (i & 1) ? 1 : 2147483647;
        add_square_over_n128(x, cnt, lo2, hi2);
        ref2 += ux * ux / (unsigned)cnt;
        ++n;
        if (lo != (unsigned long long)ref || hi != (unsigned long long)(ref >> 64)) ++bad;
        if (lo2 != (unsigned long long)ref2 || hi2 != (unsigned long long)(ref2 >> 64)) ++bad;
    }
    // the sums pass 2^64 many times over
    if (hi == 0 || hi2 == 0) ++bad;
    // the 32-bit-digit totals the kernels add to without reading back
    unsigned long long dig[4] = {0, 0, 0, 0};
    unsigned __int128 ref3 = 0;
    for (int i = 0; i < 200000; ++i) {
        const unsigned long long a = next_u64(), b = next_u64() >> (i % 5 == 0 ? 0 : 20);
        add128_digits(dig, a, b);
        ref3 += ((unsigned __int128)b << 64) | a;
        ++n;
    }
    unsigned long long l3, h3;
    combine128(dig, l3, h3);
    if (l3 != (unsigned long long)ref3 || h3 != (unsigned long long)(ref3 >> 64)) ++bad;
    printf("moments %lld %lld\n", n, bad);
}

static void check_rhe() {
    long long n = 0, bad = 0;
    for (int bits = 1; bits <= 40; ++bits)
        for (int i = 0; i < 100000; ++i) {
            unsigned long long w = next_u64() >> 12;
            if (i % 3 == 0) w = (w >> bits << bits) | (1ull << (bits - 1));   // exact halves
            const unsigned long long q = w >> bits, rem = w - (q << bits), half = 1ull << (bits - 1);
            const unsigned long long ref = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
            ++n;
            if (round_half_even_shift(w, bits) != ref) ++bad;
        }
    printf("round_half_even %lld %lld\n", n, bad);
}

// register FFTs against the direct DFT (float32 arithmetic, relative error)
template <int N, int S>
static double dft_err() {
    float2 a[N];
    std::vector<std::complex<double>> x(N);
    for (int i = 0; i < N; ++i) {
        const float re = (float)((next_u64() >> 40) * 0x1p-24 - 0.5), im = (float)((next_u64() >> 40) * 0x1p-24 - 0.5);
        x[i] = {re, im};
        a[bitrev<N == 16 ? 4 : (N == 32 ? 5 : 3)>(i)] = make_float2(re, im);
    }
    fft_dit<N, S>(a);
    double err = 0, mx = 0;
    for (int k = 0; k < N; ++k) {
        std::complex<double> acc = 0;
        for (int j = 0; j < N; ++j) acc += x[j] * std::polar(1.0, S * 2 * M_PI * (double)j * k / N);
        err = fmax(err, std::abs(acc - std::complex<double>(a[k].x, a[k].y)));
        mx = fmax(mx, std::abs(acc));
    }
    return err / mx;
}

// the real forward transform (which returns twice the DFT) against the
// direct DFT, and the round trip through the inverse
static double rfft_err() {
    float x[32];
    double xm = 0;
    for (int i = 0; i < 32; ++i) {
        x[i] = (float)((next_u64() >> 40) * 0x1p-24 - 0.5);
        xm = fmax(xm, fabs(x[i]));
    }
    float2 X[17];
    rfft32x2(x, X);
    double err = 0, mx = 0;
    for (int k = 0; k <= 16; ++k) {
        std::complex<double> acc = 0;
        for (int j = 0; j < 32; ++j) acc += (double)x[j] * std::polar(1.0, -2 * M_PI * j * k / 32.0);
        err = fmax(err, std::abs(2.0 * acc - std::complex<double>(X[k].x, X[k].y)));
        mx = fmax(mx, 2.0 * std::abs(acc));
    }
    float2 Xh[17];
    for (int k = 0; k <= 16; ++k) Xh[k] = make_float2(0.5f * X[k].x, 0.5f * X[k].y);
    float y[32];
    irfft32(Xh, y);   // 32 x
    double rt = 0;
    for (int j = 0; j < 32; ++j) rt = fmax(rt, fabs(y[j] / 32.0 - x[j]));
    return fmax(err / mx, rt / xm);
}

// Eq. 3 encode (Eq. 4 first guess plus one edge comparison each side)
// against the definition u = #{k in 1..255 : E[k] <= t}, E[k] the float32
// rounding of tan(pi (k/256 - 1/2)): every edge and its float neighbours,
// signed zeros, infinities, the largest and smallest floats, and random
// values over the whole float range and around the edges.
static void check_encode() {
    float E[256];
    E[0] = -INFINITY;
    for (int k = 1; k < 256; ++k) E[k] = (float)tan(M_PI * (k / 256.0 - 0.5));
    auto def = [&](float t) {
        int u = 0;
        for (int k = 1; k < 256; ++k) u += E[k] <= t;
        return u;
    };
    long long n = 0, bad = 0;
    uint32_t err = 0;
    auto one = [&](float t) {
        ++n;
        bad += (int)encode_momentum(t, 0.f, 1.f, E, &err) != def(t);
    };
    for (int k = 1; k < 256; ++k) {
        float t = E[k];
        for (int s = 0; s < 4; ++s) t = nextafterf(t, -INFINITY);
        for (int s = 0; s < 9; ++s, t = nextafterf(t, INFINITY)) one(t);
    }
    const float special[] = {0.f, -0.f, INFINITY, -INFINITY, 3.4028235e38f, -3.4028235e38f,
                             1e-45f, -1e-45f, 1.f, -1.f, 1e30f, -1e30f};
    for (float t : special) one(t);
    for (int i = 0; i < 2000000; ++i) {
        uint32_t b = (uint32_t)next_u64();
        float t = bits_float(b);
        if (!(t == t) || std::isinf(t)) continue;
        one(t);
        // near an edge: a few hundred ulps either side
        const float e = E[1 + (int)(next_u64() % 255)];
        memcpy(&b, &e, 4);
        b = (uint32_t)((int32_t)b + (int32_t)(next_u64() % 601) - 300);
        const float v = bits_float(b);
        if (v == v && !std::isinf(v)) one(v);
    }
    // a NaN is flagged and gets the middle bin
    err = 0;
    ++n;
    bad += encode_momentum(NAN, 0.f, 1.f, E, &err) != 128u || err == 0u;
    printf("encode %lld %lld\n", n, bad);
}

int main() {
    check_fix24();
    check_encode();
    check_moments();
    check_rhe();
    double e = 0;
    for (int t = 0; t < 20; ++t) {
        e = fmax(e, dft_err<8, -1>());
        e = fmax(e, dft_err<16, -1>());
        e = fmax(e, dft_err<16, 1>());
        e = fmax(e, dft_err<32, -1>());
        e = fmax(e, dft_err<32, 1>());
    }
    printf("fft_dit 100 0 %.3e\n", e);
    double r = 0;
    for (int t = 0; t < 50; ++t) r = fmax(r, rfft_err());
    printf("rfft32 50 0 %.3e\n", r);
    return 0;
}
