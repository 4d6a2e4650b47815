// noalloc.cu -- a power spectrum entry point that allocates no device
// memory.  Its scratch (cell offsets, the density / spectrum mesh, shell sums
// and FFT twiddles) is one file-scope device array of fixed size, so the
// entry point serves boxes of at most kNaMaxNc coarse cells per side and
// meshes of at most kNaMaxMesh points per side.  The computation follows
// pmpm_power_spectrum step for step.
#include <mutex>

#include "pmpm_impl.cuh"

namespace pmpm {

cudaError_t fft3d_float_raw(cudaStream_t st, float2* data, int n, int sign, const float2* tw, int tw_n);

namespace {

constexpr int kNaMaxNc = 64;
constexpr int kNaMaxMesh = 64;
constexpr int kNaMaxBins = kNaMaxMesh / 2;
constexpr int kNaMaxDevices = 64;
constexpr size_t kNaOffsetsBytes = 8 * ((size_t)kNaMaxNc * kNaMaxNc * kNaMaxNc + 1);
constexpr size_t kNaMeshBytes = 8 * (size_t)kNaMaxMesh * kNaMaxMesh * kNaMaxMesh;
constexpr size_t kNaBinsBytes = 8 * 3 * kNaMaxBins;
constexpr size_t kNaTwBytes = 8 * kNaMaxMesh;
constexpr size_t kA = 256;
constexpr size_t kNaOffOffsets = 0;
constexpr size_t kNaOffMesh = (kNaOffOffsets + kNaOffsetsBytes + kA - 1) / kA * kA;
constexpr size_t kNaOffBins = (kNaOffMesh + kNaMeshBytes + kA - 1) / kA * kA;
constexpr size_t kNaOffTw = (kNaOffBins + kNaBinsBytes + kA - 1) / kA * kA;
constexpr size_t kNaBytes = (kNaOffTw + kNaTwBytes + kA - 1) / kA * kA;   // about 4.2 MB

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

std::mutex g_na_lock;
unsigned char* g_na_ptr[kNaMaxDevices] = {nullptr};

__global__ void k_na_twiddles(int n, float2* tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double sv, cv;
    sincospi(2.0 * (double)k / (double)n, &sv, &cv);
    tw[k] = make_float2((float)cv, (float)-sv);
}

// exclusive scan of the counts into offsets[0..ncells], one block
__global__ void __launch_bounds__(1024) k_na_offsets(int64_t ncells, const int32_t* __restrict__ counts,
                                                     int64_t* __restrict__ offsets) {
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const int64_t per = (ncells + 1023) / 1024;
    const int64_t lo = t * per, hi = lo + per < ncells ? lo + per : ncells;
    long long s = 0;
    for (int64_t i = lo; i < hi; ++i) s += counts[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long acc = 0;
        for (int i = 0; i < 1024; ++i) {
            const long long v = part[i];
            part[i] = acc;
            acc += v;
        }
        offsets[ncells] = acc;
    }
    __syncthreads();
    long long run = part[t];
    for (int64_t i = lo; i < hi; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
}

__global__ void k_na_deposit(int64_t n, int nc, int nmesh, int lh, const int64_t* __restrict__ offsets,
                             const uint8_t* __restrict__ m0, const uint8_t* __restrict__ m1,
                             const uint8_t* __restrict__ m2, unsigned long long* rho) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    const int lu2 = 7 + lh;
    const int64_t U = (int64_t)kCodesPerFine << lh;
    const uint8_t* st[3] = {m0, m1, m2};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = ncells;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (offsets[mid] <= j) lo = mid; else hi = mid;
        }
        const int cc[3] = {(int)(lo % nc), (int)((lo / nc) % nc), (int)(lo / ((int64_t)nc * nc))};
        int i0[3];
        int64_t w1[3];
        for (int d = 0; d < 3; ++d) {
            const int64_t Q = (int64_t)cc[d] * kBins + st[d][j];
            const int64_t s = 2 * Q + 1 - U;
            i0[d] = (int)(s >> lu2);
            w1[d] = s & ((2 * U) - 1);
        }
        const int64_t W = 2 * U;
        for (int k = 0; k < 8; ++k) {
            const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
            const unsigned long long w = (unsigned long long)((dx ? w1[0] : W - w1[0]) *
                                                              (dy ? w1[1] : W - w1[1]) *
                                                              (dz ? w1[2] : W - w1[2]));
            if (!w) continue;
            const int x = wrap(i0[0] + dx, nmesh), y = wrap(i0[1] + dy, nmesh), z = wrap(i0[2] + dz, nmesh);
            atomicAdd(&rho[x + (int64_t)nmesh * (y + (int64_t)nmesh * z)], w);
        }
    }
}

// delta = rho / rho_bar - 1 in place (each element read, then written)
__global__ void k_na_delta(int64_t m3, double inv_mean, void* mesh) {
    const unsigned long long* rho = static_cast<const unsigned long long*>(mesh);
    float2* out = static_cast<float2*>(mesh);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m3;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)rho[i];
        out[i] = make_float2((float)(v * inv_mean - 1.0), 0.f);
    }
}

__global__ void k_na_bin(int nmesh, int nbins, double L, const float2* __restrict__ dk, double* bins) {
    extern __shared__ double sb[];
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) sb[i] = 0.0;
    __syncthreads();
    const int64_t m3 = (int64_t)nmesh * nmesh * nmesh;
    const double norm = L * L * L / ((double)m3 * (double)m3);
    const int h = nmesh / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m3;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nmesh), iy = (int)((i / nmesh) % nmesh),
                  iz = (int)(i / ((int64_t)nmesh * nmesh));
        const int nx = ix < h ? ix : ix - nmesh, ny = iy < h ? iy : iy - nmesh,
                  nz = iz < h ? iz : iz - nmesh;
        const double r = sqrt((double)(nx * nx + ny * ny + nz * nz));
        const int j = (int)rint(r);
        if (j < 1 || j > nbins) continue;
        const float2 v = dk[i];
        atomicAdd(&sb[j - 1], norm * ((double)v.x * v.x + (double)v.y * v.y));
        atomicAdd(&sb[nbins + j - 1], 2.0 * 3.141592653589793238462643383279502884 * r / L);
        atomicAdd(&sb[2 * nbins + j - 1], 1.0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
        if (sb[i] != 0.0) atomicAdd(&bins[i], sb[i]);
}

char g_na_msg[256] = "";

int na_fail(int code, const char* msg) {
    snprintf(g_na_msg, sizeof(g_na_msg), "%s", msg);
    return code;
}

// One-time set-up on the current device: find the scratch array's device
// address and fill the twiddle table.  Runs on the first call per device.
int na_scratch(cudaStream_t st, unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
        return na_fail(PMPM_ECUDA, "no usable CUDA device");
    std::lock_guard<std::mutex> lock(g_na_lock);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char m[200];
            snprintf(m, sizeof(m), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return na_fail(PMPM_ECUDA, m);
        }
        unsigned char* base = static_cast<unsigned char*>(p);
        k_na_twiddles<<<1, kNaMaxMesh, 0, st>>>(kNaMaxMesh, reinterpret_cast<float2*>(base + kNaOffTw));
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            return na_fail(PMPM_ECUDA, "scratch set-up failed");
        g_na_ptr[dev] = base;
    }
    *out = g_na_ptr[dev];
    return PMPM_OK;
}

}  // namespace
}  // namespace pmpm

using namespace pmpm;

extern "C" int pmpm_power_spectrum_noalloc(int32_t nc, int64_t n, const uint8_t* d_m0,
                                           const uint8_t* d_m1, const uint8_t* d_m2,
                                           const int32_t* d_counts, int32_t nmesh, int32_t nbins,
                                           double* k, double* pk, int64_t* nmodes,
                                           void* cuda_stream) {
    if (nc < 8 || nc > kNaMaxNc || (nc & (nc - 1)))
        return na_fail(PMPM_EINVAL, "nc must be a power of two in [8, 64] for the no-allocation entry point");
    const int nf = 4 * nc;
    if (nmesh < 4 || nmesh > kNaMaxMesh || (nmesh & (nmesh - 1)) || nf % nmesh)
        return na_fail(PMPM_EINVAL, "nmesh must be a power of two dividing 4*nc, at most 64");
    int lh = 0;
    while ((nmesh << lh) < nf) ++lh;
    if (lh > 2) return na_fail(PMPM_EINVAL, "nmesh below 4*nc/4 is not supported");
    if (nbins < 1 || nbins > nmesh / 2) return na_fail(PMPM_EINVAL, "nbins must be in [1, nmesh/2]");
    if (n < 1 || !d_m0 || !d_m1 || !d_m2 || !d_counts || !k || !pk || !nmodes)
        return na_fail(PMPM_EINVAL, "null pointer or empty store");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char* base = nullptr;
    int rc = na_scratch(st, &base);
    if (rc) return rc;
    int64_t* offsets = reinterpret_cast<int64_t*>(base + kNaOffOffsets);
    void* mesh = base + kNaOffMesh;
    double* bins = reinterpret_cast<double*>(base + kNaOffBins);
    const float2* tw = reinterpret_cast<const float2*>(base + kNaOffTw);
    const int64_t ncells = (int64_t)nc * nc * nc;
    const int64_t m3 = (int64_t)nmesh * nmesh * nmesh;
    // the array keeps the previous call's contents: clear what accumulates
    cudaMemsetAsync(mesh, 0, 8 * (size_t)m3, st);
    cudaMemsetAsync(bins, 0, sizeof(double) * 3 * nbins, st);
    k_na_offsets<<<1, 1024, 0, st>>>(ncells, d_counts, offsets);
    k_na_deposit<<<grid_for(n, 256), 256, 0, st>>>(n, nc, nmesh, lh, offsets, d_m0, d_m1, d_m2,
                                                    static_cast<unsigned long long*>(mesh));
    const double U = (double)(kCodesPerFine << lh);
    const double mean = (double)n * (2 * U) * (2 * U) * (2 * U) / (double)m3;
    k_na_delta<<<grid_for(m3, 256), 256, 0, st>>>(m3, 1.0 / mean, mesh);
    cudaError_t e = fft3d_float_raw(st, static_cast<float2*>(mesh), nmesh, -1, tw, kNaMaxMesh);
    if (e != cudaSuccess) return na_fail(PMPM_ECUDA, cudaGetErrorString(e));
    k_na_bin<<<grid_for(m3, 256, 152 * 4), 256, sizeof(double) * 3 * nbins, st>>>(
        nmesh, nbins, (double)nf, static_cast<const float2*>(mesh), bins);
    double hb[3 * kNaMaxBins];
    long long total = -1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb, bins, sizeof(double) * 3 * nbins, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, offsets + ncells, sizeof(total), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(PMPM_ECUDA, cudaGetErrorString(e));
    // counts that do not add up to n put particles in the wrong cells and the
    // mean density is wrong: refuse the result
    if (total != n) {
        char m[160];
        snprintf(m, sizeof(m), "the counts add up to %lld, not n = %lld", total, (long long)n);
        return na_fail(PMPM_EINVAL, m);
    }
    for (int j = 0; j < nbins; ++j) {
        const double c = hb[2 * nbins + j];
        nmodes[j] = (int64_t)c;
        k[j] = c > 0 ? hb[nbins + j] / c : 0.0;
        pk[j] = c > 0 ? hb[j] / c : 0.0;
    }
    return PMPM_OK;
}

extern "C" const char* pmpm_noalloc_last_error(void) { return g_na_msg; }
