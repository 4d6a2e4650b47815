// fft.cu -- batched 1-D FFTs along the three axes of an n^3 complex array
// (n a power of two), float or double.  Used for the coarse-mesh force of
// Eq. 1, the Zel'dovich displacement field and the power spectrum.
//
// One block transforms P neighbouring pencils in shared memory with a
// Stockham autosort radix-2 sweep (natural order in and out).  For the y and
// z axes the P pencils are adjacent in x, so every global access reads P
// consecutive complex numbers.
#include "pmpm_impl.cuh"

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
}

// The same three float passes for a caller-supplied twiddle table of tw_n
// entries (n divides tw_n); used where no Sim exists.
cudaError_t fft3d_float_raw(cudaStream_t st, float2* data, int n, int sign, const float2* tw,
                            int tw_n) {
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
