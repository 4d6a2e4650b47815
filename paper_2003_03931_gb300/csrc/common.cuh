// common.cuh -- definitions shared by the PM-PM kernels: geometry constants,
// error flags, the fixed-point codec of Sec. III-A (Eq. 2-4) and integer CIC.
//
// Functions marked PMPM_HD compile for host and device so that the tile
// phases can be exercised one thread at a time on a CPU; the product path
// runs them only inside CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PMPM_HD __host__ __device__ __forceinline__

namespace pmpm {

// ---------------------------------------------------------------- geometry
constexpr int kRatio = 4;        // coarse / fine cell size (Sec. II)
constexpr int kBins = 256;       // bins per coarse cell per dimension (Eq. 2)
constexpr int kCodesPerFine = kBins / kRatio;   // 64 codes per fine cell
constexpr int kBuffer = 6;       // tile buffer = short-range cutoff, fine cells (Sec. IV-A.2)
constexpr int kTileFFT = 32;     // edge of the tile FFT box (>= 20 + 2*6)
constexpr int kTileMaxCoarse = 5;                // largest tile, coarse cells
constexpr int kTileOut = kTileMaxCoarse * kRatio + 2;   // fine nodes a tile gathers from (22)
constexpr int kGreenS = kTileFFT / 2 + 1;        // 17: |k| range of the tile Green table
constexpr int kPFixBits = 24;    // momenta rounded to 2^-24 for the cell sums
constexpr float kSigmaFloor = 5.9604644775390625e-08f;  // 2^-24

// ---------------------------------------------------------------- error flags
enum : uint32_t {
    kErrFineOverflow = 1u,    // a fine tile node exceeded 2^32 - 1 weight units
    kErrMomentum = 2u,        // |p| too large for the 2^-24 fixed-point sums
    kErrCount = 8u,           // counts do not add up to N
    kErrNaN = 16u,            // non-finite momentum or force
    kErrDrift = 32u,          // drift larger than the int32 code range
    kErrLoadCounts = 64u,     // loaded counts negative or not adding up to N
};

#ifdef __CUDA_ARCH__
PMPM_HD float fadd_rn(float a, float b) { return __fadd_rn(a, b); }
PMPM_HD float fsub_rn(float a, float b) { return __fsub_rn(a, b); }
PMPM_HD float fmul_rn(float a, float b) { return __fmul_rn(a, b); }
PMPM_HD float fdiv_rn(float a, float b) { return __fdiv_rn(a, b); }
PMPM_HD double dmul_rn(double a, double b) { return __dmul_rn(a, b); }
PMPM_HD double dadd_rn(double a, double b) { return __dadd_rn(a, b); }
PMPM_HD void flag_error(uint32_t* err, uint32_t bits) { atomicOr(err, bits); }
PMPM_HD int fetch_add_i32(int32_t* p, int32_t v) { return atomicAdd(p, v); }
#else
PMPM_HD float fadd_rn(float a, float b) { volatile float r = a + b; return r; }
PMPM_HD float fsub_rn(float a, float b) { volatile float r = a - b; return r; }
PMPM_HD float fmul_rn(float a, float b) { volatile float r = a * b; return r; }
PMPM_HD float fdiv_rn(float a, float b) { volatile float r = a / b; return r; }
PMPM_HD double dmul_rn(double a, double b) { volatile double r = a * b; return r; }
PMPM_HD double dadd_rn(double a, double b) { volatile double r = a + b; return r; }
PMPM_HD void flag_error(uint32_t* err, uint32_t bits) { *err |= bits; }
PMPM_HD int fetch_add_i32(int32_t* p, int32_t v) { int o = *p; *p = o + v; return o; }
#endif

// ---------------------------------------------------------------- codec
// Eq. 3 decode: p = v_c + sigma * T[u], each operation an IEEE float32 op.
PMPM_HD float decode_momentum(float vc, float sigma, float tu) {
    return fadd_rn(vc, fmul_rn(sigma, tu));
}

// The integer drift of one position code: q + round-half-up(fl32(p * drift))
// (drift in codes per unit momentum), wrapped into [0, M) (M = nc bins per
// side).  A shift beyond the int32 code range is flagged and dropped.  The
// tile pass and the low-memory step's re-encode both call this, so the codes
// they derive from the same momentum are the same.
PMPM_HD int drift_code(int q, float p, float drift, int M, uint32_t* err) {
    const float xq = fmul_rn(p, drift);
    // |dq| < 1e9 and codes below 2^26: the sum fits in 32 bits
    int dq = 0;
    if (fabsf(xq) < 1.0e9f) dq = (int)floorf(fadd_rn(xq, 0.5f));
    else flag_error(err, kErrDrift);
    // periodic wrap; a division only for the rare particle that crosses the
    // box boundary
    int qn = q + dq;
    if (qn < 0 || qn >= M) {
        qn %= M;
        if (qn < 0) qn += M;
    }
    return qn;
}

// Eq. 4: the paper's fast arctangent, |x| <= 1 branch and its reflection
// atan(x) = +-pi/2 - atan(1/x) for |x| > 1.  It only guesses the Eq. 3 bin
// (the edge comparisons after it decide), so the reciprocal may be the
// hardware approximation (a few ulp against a margin of 0.008 rad).
PMPM_HD float atan_eq4(float x) {
    const float q = 0.78539816339744831f;   // pi/4
    const float c = 0.273f;
    float ax = x < 0.f ? -x : x;
    if (ax <= 1.f) return q * x + c * x * (1.f - ax);
#ifdef __CUDA_ARCH__
    float inv = __fdividef(1.f, x);
#else
    float inv = 1.f / x;
#endif
    float ainv = inv < 0.f ? -inv : inv;
    float half_pi = x > 0.f ? 1.5707963267948966f : -1.5707963267948966f;
    return half_pi - q * inv - c * inv * (1.f - ainv);
}

// Eq. 3 encode: u = #{k in 1..255 : E[k] <= t}, t = fl32(fl32(p - v_c) / sigma).
// The Eq. 4 angle gives a first guess within one bin (its error 0.0038 rad is
// below the bin width pi/256); one comparison on each side against the edge
// table makes the result identical to the definition.
PMPM_HD uint32_t encode_momentum(float p, float vc, float sigma, const float* E,
                                 uint32_t* err) {
    float t = fdiv_rn(fsub_rn(p, vc), sigma);
    if (!(t == t)) {            // NaN
        flag_error(err, kErrNaN);
        return 128u;
    }
    float th = atan_eq4(t);
    float g = th * 81.487330863050417f + 128.f;   // 256/pi, bin of the angle
    int u = (int)floorf(g < 0.f ? 0.f : (g > 255.f ? 255.f : g));
    if (u < 255 && E[u + 1] <= t) ++u;
    else if (u > 0 && E[u] > t) --u;
    return (uint32_t)u;
}

// --------------------------------------------------------- 128-bit moments
// The dispersion of Eq. 3 comes from exact integer moments of the fixed-point
// momenta P (below): T = sum P^2 over particles and U = sum floor(S^2 / n)
// over cells, each kept as a (lo, hi) pair of 64-bit words.
PMPM_HD unsigned long long umulhi64(unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

// (lo, hi) += x^2 for |x| < 2^63
PMPM_HD void add_square128(long long x, unsigned long long& lo, unsigned long long& hi) {
    const unsigned long long u = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
    const unsigned long long l = u * u;
    lo += l;
    hi += umulhi64(u, u) + (lo < l ? 1ull : 0ull);
}

// (lo, hi) added to a global 128-bit total held as four 32-bit digits in
// 64-bit words (value = sum d[i] 2^(32 i)): four additions whose result is
// not read back, so no thread waits on them, and every word stays below
// 2^64 for up to 2^32 additions.  combine128 folds the digits back.
PMPM_HD void add128_digits(unsigned long long* d, unsigned long long lo, unsigned long long hi) {
#ifdef __CUDA_ARCH__
    if (lo & 0xffffffffull) atomicAdd(&d[0], lo & 0xffffffffull);
    if (lo >> 32) atomicAdd(&d[1], lo >> 32);
    if (hi & 0xffffffffull) atomicAdd(&d[2], hi & 0xffffffffull);
    if (hi >> 32) atomicAdd(&d[3], hi >> 32);
#else
    d[0] += lo & 0xffffffffull;
    d[1] += lo >> 32;
    d[2] += hi & 0xffffffffull;
    d[3] += hi >> 32;
#endif
}

PMPM_HD void combine128(const unsigned long long* d, unsigned long long& lo, unsigned long long& hi) {
    const unsigned __int128 v = (unsigned __int128)d[0] + ((unsigned __int128)d[1] << 32) +
                                ((unsigned __int128)d[2] << 64) + ((unsigned __int128)d[3] << 96);
    lo = (unsigned long long)v;
    hi = (unsigned long long)(v >> 64);
}

// (lo, hi) += floor(S^2 / n) for n >= 1 (n < 2^31): with |S| = a n + r
// (0 <= r < n), S^2 / n = a^2 n + 2 a r + r^2 / n, whose first two terms are
// integers, so floor(S^2 / n) = a^2 n + 2 a r + floor(r^2 / n).  Both
// divisions take 32-bit operands when they fit (the usual case: |S| < 2^32
// and n < 2^16), 64-bit ones otherwise.
PMPM_HD void add_square_over_n128(long long S, int n, unsigned long long& lo,
                                  unsigned long long& hi) {
    const unsigned long long u = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
    const unsigned long long d = (unsigned long long)n;
    unsigned long long a, r;
    if ((u >> 32) == 0) {
        const uint32_t a32 = (uint32_t)u / (uint32_t)n;
        a = a32;
        r = (uint32_t)u - a32 * (uint32_t)n;
    } else {
        a = u / d;
        r = u - a * d;
    }
    const unsigned long long q3 = r < 65536ull ? (unsigned long long)((uint32_t)(r * r) / (uint32_t)n)
                                               : (r * r) / d;
    // a < 2^63 / n, so a^2 n < 2^126 / n and 2 a r < 2^64: 128-bit sums
    const unsigned long long a2l = a * a, a2h = umulhi64(a, a);          // a^2
    const unsigned long long pl = a2l * d, ph = a2h * d + umulhi64(a2l, d);   // a^2 n
    const unsigned long long ar = 2ull * a * r;                          // < 2^64 (r < n)
    unsigned long long vl = pl + ar, vh = ph + (vl < pl ? 1ull : 0ull);
    vl += q3;
    vh += vl < q3 ? 1ull : 0ull;
    lo += vl;
    hi += vh + (lo < vl ? 1ull : 0ull);
}

// round-half-even(p 2^24) for a float32 p with |p| < 2^20, in integers (the
// fixed-point momentum of the cell sums): p = m 2^(E - 150) exactly, so
// p 2^24 = m 2^(E - 126) with m < 2^24; no FP64 (slow on this part).
PMPM_HD long long fix24_rn(float p) {
    union { float f; uint32_t u; } bits;
    bits.f = p;
    const uint32_t E = (bits.u >> 23) & 255u, M = bits.u & 0x7fffffu;
    const uint32_t m = E ? (M | 0x800000u) : M;
    const int sh = (E ? (int)E : 1) - 126;
    long long r;
    if (sh >= 0) {
        r = (long long)m << sh;
    } else if (sh < -24) {
        r = 0;                                       // below 1/2
    } else {
        const int k = -sh;
        const uint32_t q = m >> k, rem = m & ((1u << k) - 1u), half = 1u << (k - 1);
        r = (long long)(q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u));
    }
    return (bits.u >> 31) ? -r : r;
}

// ---------------------------------------------------------------- position format
// PB bytes per position coordinate (Sec. III-A): B = 256 (1 byte, Eq. 2) or
// 65536 (2 bytes) bins per coarse cell.  The 3-D CIC weight products of
// 2-byte codes (2^-45 fine, 2^-51 coarse) are rounded half-even to the
// 1-byte units (2^-21, 2^-27) so both formats share the integer meshes.
template <int PB>
struct PosFmt {
    static_assert(PB == 1 || PB == 2, "1- or 2-byte positions");
    static constexpr int kBins = PB == 1 ? 256 : 65536;
    static constexpr int kShift = PB == 1 ? 8 : 16;             // log2(kBins)
    static constexpr int kCodesPerFine = kBins / kRatio;         // 64 or 16384
    static constexpr int kFineW = 2 * kCodesPerFine;             // fine weight denominator
    static constexpr int kFineWBits = PB == 1 ? 7 : 15;
    static constexpr int kCoarseW = 2 * kBins;                   // coarse weight denominator
    static constexpr int kCoarseWBits = PB == 1 ? 9 : 17;
    static constexpr int kRoundBits = PB == 1 ? 0 : 24;          // product -> 1-byte units
};

// round-half-even(w / 2^bits), bits > 0
// (w + 2^(bits-1) - 1 + bit `bits` of w) >> bits: the same as comparing the
// remainder with one half, with ties to the even quotient (w < 2^63)
PMPM_HD uint64_t round_half_even_shift(uint64_t w, int bits) {
    return (w + ((1ull << (bits - 1)) - 1ull) + ((w >> bits) & 1ull)) >> bits;
}

// 3-D weight in the 1-byte units from three 1-D weights of format PB
template <int PB>
PMPM_HD uint32_t cic_weight3(uint32_t wx, uint32_t wy, uint32_t wz) {
    if (PB == 1) return wx * wy * wz;
    return (uint32_t)round_half_even_shift((uint64_t)wx * wy * wz, PosFmt<PB>::kRoundBits);
}

// position bin m of particle j from a stream of PB-byte entries
template <int PB>
PMPM_HD int load_bin(const uint8_t* stream, int64_t j) {
    if (PB == 1) return stream[j];
    return reinterpret_cast<const uint16_t*>(stream)[j];
}

// ---------------------------------------------------------------- CIC
// Nodes at cell centres.  For a mesh whose node spacing holds U position
// codes, s = 2Q + 1 - U is the particle's offset from node 0 in units of
// 1/(2U); the lower node is floor(s / 2U) and the upper weight s mod 2U.
struct Cic1 {
    int i0;      // lower node
    int w1;      // weight of node i0+1, in 1/(2U) units
};

// fine mesh: U = 64, weights in 1/128
PMPM_HD Cic1 cic_fine(int64_t Q) {
    int64_t s = 2 * Q + 1 - kCodesPerFine;
    Cic1 c;
    c.i0 = (int)(s >> 7);
    c.w1 = (int)(s & 127);
    return c;
}

// coarse mesh: U = 256, weights in 1/512
PMPM_HD Cic1 cic_coarse(int64_t Q) {
    int64_t s = 2 * Q + 1 - kBins;
    Cic1 c;
    c.i0 = (int)(s >> 9);
    c.w1 = (int)(s & 511);
    return c;
}

PMPM_HD int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// wrap for an index at most one period outside [0, n): no division
PMPM_HD int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Tile partition along one axis: n_t tiles of 4 or 5 coarse cells
// (boundary i at floor(i * nc / n_t)).
PMPM_HD int tile_count(int nc, int tile_max) {
    return (nc + tile_max - 1) / tile_max;
}
PMPM_HD int tile_bound(int i, int nc, int nt) {
    return (int)(((int64_t)i * nc) / nt);
}

}  // namespace pmpm
