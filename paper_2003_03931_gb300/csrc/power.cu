// power.cu -- power spectrum of the particle density (Sec. IV-D): CIC density
// on an nmesh^3 mesh (integer weights, exact), delta = rho/rho_bar - 1, DFT,
// P(k) = L^3 / nmesh^6 |delta~|^2 averaged in shells j = round(|n|).
#include <new>

#include "pmpm_impl.cuh"

namespace pmpm {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// integer CIC at node spacing h = 2^lh fine cells: U = (B/4) h codes per node;
// 2-byte products are rounded to the 1-byte unit (2U_1)^-3
template <int PB>
__global__ void k_pk_deposit(int64_t n, int nc, int nmesh, int lh, const int64_t* __restrict__ offsets,
                             const uint8_t* __restrict__ st, unsigned long long* rho) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    const int lu2 = PosFmt<PB>::kFineWBits + lh;   // log2(2U)
    const int64_t U = (int64_t)PosFmt<PB>::kCodesPerFine << lh;
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
            const int64_t Q = (int64_t)cc[d] * PosFmt<PB>::kBins + load_bin<PB>(st + (size_t)d * PB * n, j);
            const int64_t s = 2 * Q + 1 - U;
            i0[d] = (int)(s >> lu2);
            w1[d] = s & ((2 * U) - 1);
        }
        const int64_t W = 2 * U;
        for (int k = 0; k < 8; ++k) {
            const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
            unsigned long long w = (unsigned long long)((dx ? w1[0] : W - w1[0]) *
                                                        (dy ? w1[1] : W - w1[1]) *
                                                        (dz ? w1[2] : W - w1[2]));
            if (PB == 2) w = round_half_even_shift(w, PosFmt<PB>::kRoundBits);
            if (!w) continue;
            const int x = wrap(i0[0] + dx, nmesh), y = wrap(i0[1] + dy, nmesh), z = wrap(i0[2] + dz, nmesh);
            atomicAdd(&rho[x + (int64_t)nmesh * (y + (int64_t)nmesh * z)], w);
        }
    }
}

__global__ void k_pk_delta(int64_t m3, double inv_mean, const unsigned long long* __restrict__ rho,
                           float2* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m3;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)((double)rho[i] * inv_mean - 1.0), 0.f);
}

__global__ void k_pk_bin(int nmesh, int nbins, double L, const float2* __restrict__ dk,
                         double* __restrict__ bins) {
    extern __shared__ double sb[];   // [3][nbins]: P sum, k sum, count
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
        const double p = norm * ((double)v.x * v.x + (double)v.y * v.y);
        atomicAdd(&sb[j - 1], p);
        atomicAdd(&sb[nbins + j - 1], 2.0 * kPi * r / L);
        atomicAdd(&sb[2 * nbins + j - 1], 1.0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
        if (sb[i] != 0.0) atomicAdd(&bins[i], sb[i]);
}

}  // namespace

int power_spectrum_enqueue(Sim& s, int nmesh, int nbins, double* host_bins) {
    if (nmesh < 2 || (nmesh & (nmesh - 1)) || nmesh > s.pk_max || s.nf % nmesh)
        return set_error(s, PMPM_EINVAL, "nmesh %d must be a power of two dividing %d, <= %d",
                         nmesh, s.nf, s.pk_max);
    if (nbins < 1 || nbins > nmesh / 2)
        return set_error(s, PMPM_EINVAL, "nbins %d must be in [1, nmesh/2]", nbins);
    int lh = 0;
    while ((nmesh << lh) < s.nf) ++lh;
    if (lh > 2) return set_error(s, PMPM_EINVAL, "nmesh below nf/4 is not supported");
    cudaStream_t st = s.stream;
    const int64_t m3 = (int64_t)nmesh * nmesh * nmesh;
    unsigned long long* rho = reinterpret_cast<unsigned long long*>(s.scratch);
    float2* dk = reinterpret_cast<float2*>(align_up(reinterpret_cast<uintptr_t>(rho + m3)));
    cudaMemsetAsync(rho, 0, sizeof(unsigned long long) * m3, st);
    auto kd = s.pb == 2 ? k_pk_deposit<2> : k_pk_deposit<1>;
    kd<<<grid_for(s.n, 256), 256, 0, st>>>(s.n, s.nc, nmesh, lh, s.offsets[s.cur], s.streams[s.cur], rho);
    const double U = (double)(kCodesPerFine << lh);
    const double mean = (double)s.n * (2 * U) * (2 * U) * (2 * U) / (double)m3;
    k_pk_delta<<<grid_for(m3, 256), 256, 0, st>>>(m3, 1.0 / mean, rho, dk);
    int rc = fft3d<float>(s, dk, nmesh, -1);
    if (rc) return rc;
    cudaMemsetAsync(s.pk_bins, 0, sizeof(double) * 3 * nbins, st);
    k_pk_bin<<<grid_for(m3, 256, 152 * 4), 256, sizeof(double) * 3 * nbins, st>>>(
        nmesh, nbins, (double)s.nf, dk, s.pk_bins);
    s.launches += 4;
    if ((rc = check_launch(s, "power spectrum"))) return rc;
    const cudaError_t e = cudaMemcpyAsync(host_bins, s.pk_bins, sizeof(double) * 3 * nbins,
                                          cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess)
        return set_error(s, PMPM_ECUDA, "power spectrum copy: %s", cudaGetErrorString(e));
    return PMPM_OK;
}

void power_spectrum_finish(const double* hb, int nbins, double* k, double* pk, int64_t* nm) {
    for (int j = 0; j < nbins; ++j) {
        const double c = hb[2 * nbins + j];
        nm[j] = (int64_t)c;
        k[j] = c > 0 ? hb[nbins + j] / c : 0.0;
        pk[j] = c > 0 ? hb[j] / c : 0.0;
    }
}

int power_spectrum(Sim& s, int nmesh, int nbins, double* k, double* pk, int64_t* nm) {
    double* hb = new (std::nothrow) double[3 * (size_t)(nbins > 0 ? nbins : 1)];
    if (!hb) return set_error(s, PMPM_ENOMEM, "host bins");
    int rc = power_spectrum_enqueue(s, nmesh, nbins, hb);
    if (!rc) {
        const cudaError_t e = cudaStreamSynchronize(s.stream);
        if (e != cudaSuccess) rc = set_error(s, PMPM_ECUDA, "power spectrum: %s", cudaGetErrorString(e));
    }
    if (!rc) power_spectrum_finish(hb, nbins, k, pk, nm);
    delete[] hb;
    return rc;
}

}  // namespace pmpm
