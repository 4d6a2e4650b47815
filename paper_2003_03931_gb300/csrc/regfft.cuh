// regfft.cuh -- small FFTs held in one thread's registers (16 and 32 points),
// and the real-to-complex / complex-to-real wrappers built on them.  Used by
// the tile fine-mesh solver (Sec. II: F_s = IDFT(rho~ K~_s), Eq. 1).
//
// Twiddles exp(-+2 pi i j / 32) are written as exact symmetric constants; all
// loops have compile-time bounds so every twiddle index folds to a constant.
#pragma once

#include "common.cuh"

namespace pmpm {

// cos(2 pi j / 32) for any integer j
PMPM_HD float cos32(int j) {
    const float C1 = 0.98078528040323044913f, C2 = 0.92387953251128675613f,
                C3 = 0.83146961230254523708f, C4 = 0.70710678118654752440f,
                C5 = 0.55557023301960222474f, C6 = 0.38268343236508977173f,
                C7 = 0.19509032201612826785f;
    j &= 31;
    int q = j >> 3, r = j & 7;
    // cos over the first quadrant indexed by r = 0..8
    float v;
    int idx = (q & 1) ? 8 - r : r;           // reflect in odd quadrants
    switch (idx) {
        case 0: v = 1.f; break;
        case 1: v = C1; break;
        case 2: v = C2; break;
        case 3: v = C3; break;
        case 4: v = C4; break;
        case 5: v = C5; break;
        case 6: v = C6; break;
        case 7: v = C7; break;
        default: v = 0.f; break;
    }
    // sign: quadrants 1 and 2 negative
    return (q == 1 || q == 2) ? -v : v;
}
PMPM_HD float sin32(int j) { return cos32(8 - j); }

PMPM_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
PMPM_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// d * exp(S * 2 pi i j / 32), j a compile-time constant after unrolling;
// S = -1 forward, +1 inverse.
template <int S>
PMPM_HD float2 twiddle32(float2 d, int j) {
    j &= 31;
    if (j == 0) return d;
    if (j == 8) return S < 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
    if (j == 16) return make_float2(-d.x, -d.y);
    if (j == 24) return S < 0 ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    float c = cos32(j), s = (S < 0 ? -1.f : 1.f) * sin32(j);
    return make_float2(d.x * c - d.y * s, d.x * s + d.y * c);
}

// One radix-2 decimation-in-frequency stage of an N-point transform.
template <int N, int HALF, int S>
struct DifStage {
    static PMPM_HD void run(float2 (&a)[N]) {
#pragma unroll
        for (int g = 0; g < N; g += 2 * HALF) {
#pragma unroll
            for (int k = 0; k < HALF; ++k) {
                float2 x = a[g + k], y = a[g + k + HALF];
                a[g + k] = cadd(x, y);
                a[g + k + HALF] = twiddle32<S>(csub(x, y), k * (N / (2 * HALF)) * (32 / N));
            }
        }
        DifStage<N, HALF / 2, S>::run(a);
    }
};
template <int N, int S>
struct DifStage<N, 0, S> {
    static PMPM_HD void run(float2 (&)[N]) {}
};

template <int LOG>
PMPM_HD int bitrev(int k) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < LOG; ++b) r |= ((k >> b) & 1) << (LOG - 1 - b);
    return r;
}

// In-place unnormalised N-point DFT (N = 16 or 32): on return a[bitrev(k)]
// holds X[k] = sum_n x[n] exp(S 2 pi i n k / N).
template <int N, int S>
PMPM_HD void fft_bitrev_out(float2 (&a)[N]) {
    DifStage<N, N / 2, S>::run(a);
}

// Real 32-point forward DFT through a 16-point complex one.
// In: x[0..31] real.  Out: X[0..16] (X[0], X[16] real).
PMPM_HD void rfft32(const float (&x)[32], float2 (&X)[17]) {
    float2 z[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) z[m] = make_float2(x[2 * m], x[2 * m + 1]);
    fft_bitrev_out<16, -1>(z);
#pragma unroll
    for (int k = 0; k <= 16; ++k) {
        float2 Zk = z[bitrev<4>(k & 15)];
        float2 Zr = z[bitrev<4>((16 - k) & 15)];
        // E = (Zk + conj Zr)/2, O = -i (Zk - conj Zr)/2
        float2 E = make_float2(0.5f * (Zk.x + Zr.x), 0.5f * (Zk.y - Zr.y));
        float2 O = make_float2(0.5f * (Zk.y + Zr.y), -0.5f * (Zk.x - Zr.x));
        X[k] = cadd(E, twiddle32<-1>(O, k));
    }
}

// Inverse of rfft32 without the 1/32: x[n] = sum_k X[k] exp(+2 pi i n k/32)
// over the Hermitian-extended spectrum.  In: X[0..16]; out: x[0..31].
PMPM_HD void irfft32(const float2 (&X)[17], float (&x)[32]) {
    float2 z[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float2 Xk = X[k];
        float2 Xc = make_float2(X[16 - k].x, -X[16 - k].y);   // conj X[16-k]
        float2 E = cadd(Xk, Xc);
        float2 O = twiddle32<1>(csub(Xk, Xc), k);
        z[k] = make_float2(E.x - O.y, E.y + O.x);             // E + i O
    }
    fft_bitrev_out<16, 1>(z);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        float2 v = z[bitrev<4>(m)];
        x[2 * m] = v.x;
        x[2 * m + 1] = v.y;
    }
}

}  // namespace pmpm
