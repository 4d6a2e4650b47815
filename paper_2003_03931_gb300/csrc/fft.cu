// fft.cu -- batched 1-D FFTs along the three axes of an n^3 complex array
// (n a power of two), float or double.  Used for the coarse-mesh force of
// Eq. 1, the Zel'dovich displacement field and the power spectrum.
//
// One block transforms P neighbouring pencils.  Float pencils of 64 to 1024
// points take two register steps with one shared-memory transpose
// (k_fft_pass_r); other sizes and float64 take a Stockham autosort radix-2
// sweep in shared memory (k_fft_pass; natural order in and out).  For the y
// and z axes the P pencils are adjacent in x, so every global access reads
// P consecutive complex numbers.
#include "pmpm_impl.cuh"
#include "regfft.cuh"

namespace pmpm {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// All sizes are powers of two, so every index below is a shift or a mask.
// Each thread holds at most kPassElems elements of the group; it issues all
// its global loads before storing any into shared memory.
constexpr int kPassThreads = 256;
constexpr int kPassSmem = 72 * 1024;   // two buffers of 4096 + P padded elements
// P n / threads: 4096 / 256 (float), 2048 / 256 (double)
template <typename R> constexpr int pass_elems() { return sizeof(R) == 4 ? 16 : 8; }

template <typename R>
__global__ void __launch_bounds__(kPassThreads) k_fft_pass(typename Cplx<R>::T* data, int n, int log2n,
                                                           int axis, int sign, int P, int log2P,
                                                           const typename Cplx<R>::T* tw,
                                                           int log2tw) {
    using C = typename Cplx<R>::T;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    // pencils sit n + 1 apart in shared memory: the pencils a warp touches
    // together (adjacent in x for the y and z axes) fall in different banks
    const int ps = n + 1;
    C* buf0 = reinterpret_cast<C*>(fft_smem);
    C* buf1 = buf0 + (size_t)P * ps;
    const int64_t q0 = (int64_t)blockIdx.x * P;     // first pencil of the group
    const int tid = threadIdx.x;
    const int total = P * n;
    const int nmask = n - 1;

    // pencil p of the group: base offset and element stride
    auto base_of = [&](int p) -> int64_t {
        const int64_t q = q0 + p;
        if (axis == 0) return q << log2n;
        const int64_t hi = q >> log2n, lo = q & nmask;
        if (axis == 1) return (hi << (2 * log2n)) + lo;   // (x, z) -> z n^2 + x
        return (hi << log2n) + lo;                         // (x, y) -> y n + x
    };
    const int sh = axis * log2n;                            // log2 of the element stride
    auto coords = [&](int e, int& p, int& j) {
        if (axis == 0) { p = e >> log2n; j = e & nmask; }
        else { p = e & (P - 1); j = e >> log2P; }
    };

    constexpr int kPassElems = pass_elems<R>();
    C v[kPassElems];
#pragma unroll
    for (int r = 0; r < kPassElems; ++r) {
        const int e = tid + r * kPassThreads;
        if (e < total) {
            int p, j;
            coords(e, p, j);
            v[r] = data[base_of(p) + ((int64_t)j << sh)];
        }
    }
#pragma unroll
    for (int r = 0; r < kPassElems; ++r) {
        const int e = tid + r * kPassThreads;
        if (e < total) {
            int p, j;
            coords(e, p, j);
            buf0[p * ps + j] = v[r];
        }
    }
    __syncthreads();

    C* src = buf0;
    C* dst = buf1;
    const int half = n >> 1, lhalf = log2n - 1;
    for (int ls = 0; ls < log2n; ++ls) {
        const int Ns = 1 << ls;
        const int twsh = log2tw - ls - 1;                  // k tw_n / (2 Ns) = k << twsh
        for (int e = tid; e < P * half; e += kPassThreads) {
            const int p = e >> lhalf, j = e & (half - 1);
            const int k = j & (Ns - 1);
            const int b = p * ps;
            C v0 = src[b + j];
            C v1 = src[b + j + half];
            C w = tw[(int64_t)k << twsh];
            if (sign > 0) w.y = -w.y;
            v1 = cmul(v1, w);
            const int o = ((j - k) << 1) + k;
            C a, c;
            a.x = v0.x + v1.x; a.y = v0.y + v1.y;
            c.x = v0.x - v1.x; c.y = v0.y - v1.y;
            dst[b + o] = a;
            dst[b + o + Ns] = c;
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
    }

#pragma unroll
    for (int r = 0; r < kPassElems; ++r) {
        const int e = tid + r * kPassThreads;
        if (e < total) {
            int p, j;
            coords(e, p, j);
            data[base_of(p) + ((int64_t)j << sh)] = src[p * ps + j];
        }
    }
}

constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v / 2); }

// Float pencils of n = N1 N2 points (N1, N2 in {8, 16, 32}) in two register
// steps, one shared-memory transpose between (the "four-step" split of the
// DFT): with j = N2 n1 + n2 and k = k1 + N1 k2,
//   X[k] = sum_n2 W_N2^(n2 k2) [ W_n^(n2 k1) sum_n1 W_N1^(n1 k1) x[j] ].
// Step A: one thread per (pencil, n2) does the N1-point transform and the
// twiddle; step B: one thread per (pencil, k1) does the N2-point transform.
// Each element crosses shared memory once and the block waits at one
// barrier, against log2 n sweeps and barriers in k_fft_pass.  Rows of the
// transpose buffer are N2 + 1 long and pencils N1 (N2 + 1) + 1 (odd), so
// lanes over n2, k1 or the pencil all touch distinct banks.  Loads and
// stores are coalesced as in k_fft_pass: lanes run along the pencil for the
// x axis and across adjacent pencils for y and z.
template <int N1, int N2, int S>
__global__ void __launch_bounds__(kPassThreads) k_fft_pass_r(float2* data, int axis, int P, int log2P,
                                                             const float2* tw, int twsh) {
    constexpr int n = N1 * N2;
    constexpr int L1 = clog2(N1), L2 = clog2(N2), LN = L1 + L2;
    constexpr int RS = N2 + 1, PS = N1 * RS + 1;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    float2* Y = reinterpret_cast<float2*>(fft_smem);
    const int64_t q0 = (int64_t)blockIdx.x * P;
    auto base_of = [&](int p) -> int64_t {
        const int64_t q = q0 + p;
        if (axis == 0) return q << LN;
        const int64_t hi = q >> LN, lo = q & (n - 1);
        if (axis == 1) return (hi << (2 * LN)) + lo;
        return (hi << LN) + lo;
    };
    const int sh = axis * LN;
    for (int it = threadIdx.x; it < P * N2; it += kPassThreads) {
        const int p = axis == 0 ? it >> L2 : (it & (P - 1));
        const int n2 = axis == 0 ? (it & (N2 - 1)) : (it >> log2P);
        const int64_t b = base_of(p);
        float2 a[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) a[bitrev<L1>(n1)] = data[b + ((int64_t)(N2 * n1 + n2) << sh)];
        fft_dit<N1, S>(a);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 w = tw[(n2 * k1) << twsh];
            if (S > 0) w.y = -w.y;
            Y[p * PS + k1 * RS + n2] = make_float2(a[k1].x * w.x - a[k1].y * w.y, a[k1].x * w.y + a[k1].y * w.x);
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < P * N1; it += kPassThreads) {
        const int p = axis == 0 ? it >> L1 : (it & (P - 1));
        const int k1 = axis == 0 ? (it & (N1 - 1)) : (it >> log2P);
        float2 a[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) a[bitrev<L2>(n2)] = Y[p * PS + k1 * RS + n2];
        fft_dit<N2, S>(a);
        const int64_t b = base_of(p);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) data[b + ((int64_t)(k1 + N1 * k2) << sh)] = a[k2];
    }
}

template <int N1, int N2>
static void launch_pass_r(float2* data, int n, int sign, const float2* tw, int tw_n, cudaStream_t st) {
    constexpr int P = 4096 / (N1 * N2) < 8 ? 8 : 4096 / (N1 * N2);   // 64 at n = 64 ... 8 at 512, 1024
    constexpr int PS = N1 * (N2 + 1) + 1;
    const size_t smem = (size_t)P * PS * sizeof(float2);
    int lt = 0, lp = 0;
    while ((1 << lt) < tw_n) ++lt;
    while ((1 << lp) < P) ++lp;
    int ln = 0;
    while ((1 << ln) < n) ++ln;
    const int twsh = lt - ln;                       // W_n^e = tw[e << twsh]
    const int64_t groups = (int64_t)n * n / P;
    for (int axis = 0; axis < 3; ++axis) {
        if (sign < 0)
            k_fft_pass_r<N1, N2, -1><<<(unsigned)groups, kPassThreads, smem, st>>>(data, axis, P, lp, tw, twsh);
        else
            k_fft_pass_r<N1, N2, 1><<<(unsigned)groups, kPassThreads, smem, st>>>(data, axis, P, lp, tw, twsh);
    }
}

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

template <typename R>
static int pencils_per_block(int n) {
    const int elems = sizeof(R) == 4 ? 4096 : 2048;   // 2 buffers x 32 KB
    int P = elems / n;
    if (P < 1) P = 1;
    if (P > n) P = n;
    return P;
}

template <typename R>
int fft3d(Sim& s, void* data, int n, int sign) {
    using C = typename Cplx<R>::T;
    if (n < 2 || (n & (n - 1)) || n > s.fft_max)
        return set_error(s, PMPM_EINVAL, "fft length %d not supported", n);
    if (sizeof(R) == 4 && n >= 64 && n <= 1024) {
        float2* d = reinterpret_cast<float2*>(data);
        if (n == 64) launch_pass_r<8, 8>(d, n, sign, s.tw_f, s.fft_max, s.stream);
        else if (n == 128) launch_pass_r<8, 16>(d, n, sign, s.tw_f, s.fft_max, s.stream);
        else if (n == 256) launch_pass_r<16, 16>(d, n, sign, s.tw_f, s.fft_max, s.stream);
        else if (n == 512) launch_pass_r<16, 32>(d, n, sign, s.tw_f, s.fft_max, s.stream);
        else launch_pass_r<32, 32>(d, n, sign, s.tw_f, s.fft_max, s.stream);
        s.launches += 3;
        return check_launch(s, "fft");
    }
    int log2n = 0;
    while ((1 << log2n) < n) ++log2n;
    const int P = pencils_per_block<R>(n);
    if (P * n > pass_elems<R>() * kPassThreads)
        return set_error(s, PMPM_EINVAL, "fft length %d too long for this precision", n);
    const size_t smem = 2 * (size_t)P * (n + 1) * sizeof(C);
    const C* tw = sizeof(R) == 4 ? reinterpret_cast<const C*>(s.tw_f)
                                 : reinterpret_cast<const C*>(s.tw_d);
    const int64_t groups = (int64_t)n * n / P;
    for (int axis = 0; axis < 3; ++axis) {
        k_fft_pass<R><<<(unsigned)groups, kPassThreads, smem, s.stream>>>(
            reinterpret_cast<C*>(data), n, log2n, axis, sign, P, ilog2(P), tw, ilog2(s.fft_max));
        s.launches++;
    }
    return check_launch(s, "fft");
}

template int fft3d<float>(Sim&, void*, int, int);

void fft_setup() {
    cudaFuncSetAttribute(k_fft_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
    cudaFuncSetAttribute(k_fft_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
    cudaFuncSetAttribute(k_fft_pass_r<32, 32, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
    cudaFuncSetAttribute(k_fft_pass_r<32, 32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
    cudaFuncSetAttribute(k_fft_pass_r<16, 32, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
    cudaFuncSetAttribute(k_fft_pass_r<16, 32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
}

// The same three float passes for a caller-supplied twiddle table of tw_n
// entries (n divides tw_n); used where no Sim exists.
cudaError_t fft3d_float_raw(cudaStream_t st, float2* data, int n, int sign, const float2* tw,
                            int tw_n) {
    if (n >= 64 && n <= 1024 && n <= tw_n) {   // the same passes as fft3d<float>
        if (n > 512) fft_setup();                // more than 48 KB of shared memory
        if (n == 64) launch_pass_r<8, 8>(data, n, sign, tw, tw_n, st);
        else if (n == 128) launch_pass_r<8, 16>(data, n, sign, tw, tw_n, st);
        else if (n == 256) launch_pass_r<16, 16>(data, n, sign, tw, tw_n, st);
        else if (n == 512) launch_pass_r<16, 32>(data, n, sign, tw, tw_n, st);
        else launch_pass_r<32, 32>(data, n, sign, tw, tw_n, st);
        return cudaGetLastError();
    }
    int log2n = 0;
    while ((1 << log2n) < n) ++log2n;
    const int P = pencils_per_block<float>(n);
    if (P * n > pass_elems<float>() * kPassThreads) return cudaErrorInvalidValue;
    const size_t smem = 2 * (size_t)P * (n + 1) * sizeof(float2);
    cudaFuncSetAttribute(k_fft_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmem);
    const int64_t groups = (int64_t)n * n / P;
    for (int axis = 0; axis < 3; ++axis)
        k_fft_pass<float><<<(unsigned)groups, kPassThreads, smem, st>>>(data, n, log2n, axis, sign, P,
                                                                       ilog2(P), tw, ilog2(tw_n));
    return cudaGetLastError();
}
template int fft3d<double>(Sim&, void*, int, int);

}  // namespace pmpm
