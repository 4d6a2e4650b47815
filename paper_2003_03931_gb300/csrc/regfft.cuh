// regfft.cuh -- small FFTs held in one thread's registers (8, 16 and 32
// points), and the real-to-complex / complex-to-real wrappers built on them.
// Used by the tile fine-mesh solver (Sec. II: F_s = IDFT(rho~ K~_s), Eq. 1)
// and by the two-step passes of the coarse-mesh transforms.
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

// Twiddle factor w = exp(S 2 pi i j / 32) (S = -1 forward, +1 inverse, j a
// compile-time constant after unrolling) in factored form: returns u and m
// with w d = m u.  Multiples of pi/2 are a swap and signs (m = +-1); other
// angles divide through by the larger of |cos|, |sin| (ratio t with |t| <= 1),
// u = d (1 + i t) or d (t + i), so that a later a + m u is one fused
// multiply-add per component (the FMA butterfly of Linzer and Feig).
template <int S>
PMPM_HD float2 twiddle_f(float2 d, int j, float& m) {
    j &= 31;
    if (j == 0 || j == 16) {
        m = j == 0 ? 1.f : -1.f;
        return d;
    }
    if (j == 8 || j == 24) {
        m = 1.f;   // w = -i (forward 8, inverse 24) or +i
        return ((j == 8) == (S < 0)) ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
    }
    const float wr = cos32(j), wi = (S < 0 ? -1.f : 1.f) * sin32(j);
    if (fabsf(wr) >= fabsf(wi)) {
        const float t = wi / wr;
        m = wr;
        return make_float2(d.x - t * d.y, d.y + t * d.x);
    }
    const float t = wr / wi;
    m = wi;
    return make_float2(t * d.x - d.y, t * d.y + d.x);
}

// (a, b) <- (a + w b, a - w b)
template <int S>
PMPM_HD void butterfly(float2& a, float2& b, int j) {
    float m;
    const float2 u = twiddle_f<S>(b, j, m);
    const float2 x = a;
    a = make_float2(x.x + m * u.x, x.y + m * u.y);
    b = make_float2(x.x - m * u.x, x.y - m * u.y);
}

// One radix-2 decimation-in-time stage (span 2 HALF) of an N-point transform,
// then the next larger span.
template <int N, int HALF, int S>
struct DitStage {
    static PMPM_HD void run(float2 (&a)[N]) {
#pragma unroll
        for (int g = 0; g < N; g += 2 * HALF) {
#pragma unroll
            for (int k = 0; k < HALF; ++k) butterfly<S>(a[g + k], a[g + k + HALF], k * (32 / (2 * HALF)));
        }
        DitStage<N, 2 * HALF, S>::run(a);
    }
};
template <int N, int S>
struct DitStage<N, N, S> {
    static PMPM_HD void run(float2 (&)[N]) {}
};

template <int LOG>
PMPM_HD int bitrev(int k) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < LOG; ++b) r |= ((k >> b) & 1) << (LOG - 1 - b);
    return r;
}

// In-place unnormalised N-point DFT (N = 16 or 32) by radix-2 decimation in
// time: on entry a[bitrev(n)] holds x[n]; on return a[k] holds
// X[k] = sum_n x[n] exp(S 2 pi i n k / N).
template <int N, int S>
PMPM_HD void fft_dit(float2 (&a)[N]) {
    DitStage<N, 1, S>::run(a);
}

// Real 32-point forward DFT through a 16-point complex one, scaled by 2.
// In: x[0..31] real.  Out: X[0..16] = 2 DFT(x)[0..16] (X[0], X[16] real).
PMPM_HD void rfft32x2(const float (&x)[32], float2 (&X)[17]) {
    float2 z[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) z[bitrev<4>(m)] = make_float2(x[2 * m], x[2 * m + 1]);
    fft_dit<16, -1>(z);
#pragma unroll
    for (int k = 0; k <= 16; ++k) {
        const float2 Zk = z[k & 15];
        const float2 Zr = z[(16 - k) & 15];
        // 2E = Zk + conj Zr, 2O = -i (Zk - conj Zr); 2X = 2E + w^k 2O
        const float2 E = make_float2(Zk.x + Zr.x, Zk.y - Zr.y);
        const float2 O = make_float2(Zk.y + Zr.y, Zr.x - Zk.x);
        float m;
        const float2 u = twiddle_f<-1>(O, k, m);
        X[k] = make_float2(E.x + m * u.x, E.y + m * u.y);
    }
}

// Inverse of the true DFT without the 1/32: x[n] = sum_k X[k] exp(+2 pi i n k/32)
// over the Hermitian-extended spectrum.  In: X[0..16]; out: x[0..31].
PMPM_HD void irfft32(const float2 (&X)[17], float (&x)[32]) {
    float2 z[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float2 Xk = X[k];
        const float2 Xc = make_float2(X[16 - k].x, -X[16 - k].y);   // conj X[16-k]
        const float2 E = cadd(Xk, Xc);
        float m;
        const float2 u = twiddle_f<1>(csub(Xk, Xc), k, m);         // O = m u
        z[bitrev<4>(k)] = make_float2(E.x - m * u.y, E.y + m * u.x); // E + i O
    }
    fft_dit<16, 1>(z);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        x[2 * m] = z[m].x;
        x[2 * m + 1] = z[m].y;
    }
}

}  // namespace pmpm
