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

template <typename R>
__global__ void __launch_bounds__(256) k_fft_pass(typename Cplx<R>::T* data, int n, int log2n,
                                                  int axis, int sign, int P,
                                                  const typename Cplx<R>::T* tw, int tw_n) {
    using C = typename Cplx<R>::T;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    C* buf0 = reinterpret_cast<C*>(fft_smem);
    C* buf1 = buf0 + (size_t)P * n;
    const int64_t q0 = (int64_t)blockIdx.x * P;     // first pencil of the group
    const int64_t nn = (int64_t)n * n;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int total = P * n;

    // pencil p of the group: base offset and element stride
    auto base_of = [&](int p) -> int64_t {
        const int64_t q = q0 + p;
        if (axis == 0) return q * n;
        if (axis == 1) return (q / n) * nn + (q % n);   // (x, z) -> z*n*n + x
        return (q / n) * n + (q % n);                    // (x, y) -> y*n + x
    };
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? n : nn);

    for (int e = tid; e < total; e += nth) {
        int p, j;
        if (axis == 0) { p = e / n; j = e % n; } else { p = e % P; j = e / P; }
        buf0[p * n + j] = data[base_of(p) + (int64_t)j * stride];
    }
    __syncthreads();

    C* src = buf0;
    C* dst = buf1;
    const int half = n >> 1;
    for (int Ns = 1; Ns < n; Ns <<= 1) {
        for (int e = tid; e < P * half; e += nth) {
            const int p = e / half, j = e % half;
            const int k = j & (Ns - 1);
            C v0 = src[p * n + j];
            C v1 = src[p * n + j + half];
            C w = tw[(int64_t)k * (tw_n / (2 * Ns))];
            if (sign > 0) w.y = -w.y;
            v1 = cmul(v1, w);
            const int o = ((j - k) << 1) + k;
            C a, b;
            a.x = v0.x + v1.x; a.y = v0.y + v1.y;
            b.x = v0.x - v1.x; b.y = v0.y - v1.y;
            dst[p * n + o] = a;
            dst[p * n + o + Ns] = b;
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
    }

    for (int e = tid; e < total; e += nth) {
        int p, j;
        if (axis == 0) { p = e / n; j = e % n; } else { p = e % P; j = e / P; }
        data[base_of(p) + (int64_t)j * stride] = src[p * n + j];
    }
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
    const size_t smem = 2 * (size_t)P * n * sizeof(C);
    const C* tw = sizeof(R) == 4 ? reinterpret_cast<const C*>(s.tw_f)
                                 : reinterpret_cast<const C*>(s.tw_d);
    const int64_t groups = (int64_t)n * n / P;
    for (int axis = 0; axis < 3; ++axis) {
        k_fft_pass<R><<<(unsigned)groups, 256, smem, s.stream>>>(reinterpret_cast<C*>(data), n,
                                                                 log2n, axis, sign, P, tw,
                                                                 s.fft_max);
        s.launches++;
    }
    return check_launch(s, "fft");
}

template int fft3d<float>(Sim&, void*, int, int);

void fft_setup() {
    cudaFuncSetAttribute(k_fft_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    cudaFuncSetAttribute(k_fft_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
}

// The same three float passes for a caller-supplied twiddle table of tw_n
// entries (n divides tw_n); used where no Sim exists.
cudaError_t fft3d_float_raw(cudaStream_t st, float2* data, int n, int sign, const float2* tw,
                            int tw_n) {
    int log2n = 0;
    while ((1 << log2n) < n) ++log2n;
    const int P = pencils_per_block<float>(n);
    const size_t smem = 2 * (size_t)P * n * sizeof(float2);
    cudaFuncSetAttribute(k_fft_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    const int64_t groups = (int64_t)n * n / P;
    for (int axis = 0; axis < 3; ++axis)
        k_fft_pass<float><<<(unsigned)groups, 256, smem, st>>>(data, n, log2n, axis, sign, P, tw, tw_n);
    return cudaGetLastError();
}
template int fft3d<double>(Sim&, void*, int, int);

}  // namespace pmpm
