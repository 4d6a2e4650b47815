// ic.cu -- Zel'dovich initial conditions (Sec. IV-A.2) for a power-law
// spectrum P(k) = k^slope exp(-(k/k_c)^2), in float64 on the device:
//   white noise (SplitMix64 counters 2i, 2i+1; Box-Muller) -> DFT ->
//   Psi~_d = i k_d / k^2 sqrt(P) w~ (k = 0 and Nyquist planes zeroed) ->
//   inverse DFT -> rms normalisation -> x = q + a Psi, p = a^(3/2) Psi (EdS; a^2 E f a Psi
//   in LambdaCDM) ->
//   Q = floor(64 x) mod (256 nc), p in float32 -> cell-ordered encode.
#include "pmpm_impl.cuh"

namespace pmpm {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// SplitMix64 output for counter j (Steele, Lea & Flood 2014)
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long j) {
    unsigned long long z = seed + (j + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_ic_noise(int64_t n, unsigned long long seed, double2* w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long z1 = splitmix64(seed, 2ull * i);
        const unsigned long long z2 = splitmix64(seed, 2ull * i + 1ull);
        const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1p-53;
        const double u2 = (double)(z2 >> 11) * 0x1p-53;
        w[i] = make_double2(sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2), 0.0);
    }
}

// sqrt(P(k)) / k^2 of every mode (0 on the k = 0 and Nyquist planes), shared
// by the three displacement components
// The amplitude depends on the mode only through m = nx^2 + ny^2 + nz^2
// (k^2 = kf^2 m): one table entry per m, so the float64 pow, exp and sqrt run
// 3 (np/2)^2 times instead of np^3 times.
__global__ void k_ic_amp_table(int mmax, int nf, double slope, double kc, double* __restrict__ tab) {
    const double kf = 2.0 * kPi / nf;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m <= mmax; m += gridDim.x * blockDim.x) {
        double c = 0.0;
        if (m > 0) {
            const double k2 = kf * kf * (double)m;
            const double k = sqrt(k2);
            c = sqrt(pow(k, slope) * exp(-(k / kc) * (k / kc))) / k2;
        }
        tab[m] = c;
    }
}

__global__ void k_ic_amplitude(int np, const double* __restrict__ tab, double* __restrict__ amp) {
    const int64_t n = (int64_t)np * np * np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % np), iy = (int)((i / np) % np), iz = (int)(i / ((int64_t)np * np));
        const int h = np / 2;
        const int nx = ix < h ? ix : ix - np, ny = iy < h ? iy : iy - np, nz = iz < h ? iz : iz - np;
        const bool zero = nx == -h || ny == -h || nz == -h;   // the Nyquist planes; m = 0 gives 0
        amp[i] = zero ? 0.0 : tab[nx * nx + ny * ny + nz * nz];
    }
}

// Psi~_d = i k_d amp w~
__global__ void k_ic_component(int np, int nf, int d, const double* __restrict__ amp,
                               const double2* __restrict__ w, double2* __restrict__ out) {
    const int64_t n = (int64_t)np * np * np;
    const double kf = 2.0 * kPi / nf;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % np), iy = (int)((i / np) % np), iz = (int)(i / ((int64_t)np * np));
        const int h = np / 2;
        const int nd = d == 0 ? (ix < h ? ix : ix - np) : (d == 1 ? (iy < h ? iy : iy - np)
                                                                  : (iz < h ? iz : iz - np));
        const double c = kf * nd * amp[i];
        const double2 a = w[i];
        out[i] = make_double2(-c * a.y, c * a.x);   // i c a
    }
}

__global__ void k_ic_store(int64_t n, int d, const double2* __restrict__ in, double* __restrict__ psi,
                           double* __restrict__ partial) {
    double acc = 0.0;
    const double inv_n = 1.0 / (double)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = in[i].x * inv_n;
        psi[d * n + i] = v;
        acc += v * v;
    }
    // deterministic block sum (fixed grid and order)
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[d * gridDim.x + blockIdx.x] += sh[0];
}

__global__ void k_ic_scale(int nblk, int64_t n, double a_init, double rms_disp, const double* partial,
                           double* scale) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int b = 0; b < nblk; ++b) s += partial[d * nblk + b];
    const double rms = sqrt(s / (double)n);
    *scale = rms > 0.0 ? rms_disp / (a_init * rms) : 0.0;
}

template <int PB>
__global__ void k_ic_particles(int np, int nc, double a_init, double pfac, const double* __restrict__ psi,
                               const double* __restrict__ scale_p, int32_t* __restrict__ Qn,
                               float* __restrict__ Pn) {
    const int64_t n = (int64_t)np * np * np;
    const double scale = *scale_p;
    const double spacing = 4.0 * nc / (double)np;
    const int64_t M = (int64_t)nc * PosFmt<PB>::kBins;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int li[3] = {(int)(i % np), (int)((i / np) % np), (int)(i / ((int64_t)np * np))};
        for (int d = 0; d < 3; ++d) {
            const double ps = psi[d * n + i] * scale;
            const double q = ((double)li[d] + 0.5) * spacing;
            const double x = q + a_init * ps;
            int64_t Q = (int64_t)floor(x * (double)PosFmt<PB>::kCodesPerFine) % M;
            if (Q < 0) Q += M;
            Qn[d * n + i] = (int32_t)Q;
            Pn[d * n + i] = (float)(pfac * ps);
        }
    }
}

// float32 variants for low-memory sims: the same noise, spectrum and
// normalisation, one float2 work array (noise regenerated per component) and
// a float32 displacement field
__global__ void k_ic_noise_f(int64_t n, unsigned long long seed, float2* w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long z1 = splitmix64(seed, 2ull * i);
        const unsigned long long z2 = splitmix64(seed, 2ull * i + 1ull);
        const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1p-53;
        const double u2 = (double)(z2 >> 11) * 0x1p-53;
        w[i] = make_float2((float)(sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2)), 0.f);
    }
}
__global__ void k_ic_amplitude_f(int np, int nf, double slope, double kc, float* __restrict__ amp) {
    const int64_t n = (int64_t)np * np * np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % np), iy = (int)((i / np) % np), iz = (int)(i / ((int64_t)np * np));
        const int h = np / 2;
        const int nx = ix < h ? ix : ix - np, ny = iy < h ? iy : iy - np, nz = iz < h ? iz : iz - np;
        double c = 0.0;
        if (!(nx == -h || ny == -h || nz == -h) && (nx | ny | nz)) {
            const double kf = 2.0 * kPi / nf;
            const double kx = kf * nx, ky = kf * ny, kz = kf * nz;
            const double k2 = kx * kx + ky * ky + kz * kz;
            const double k = sqrt(k2);
            c = sqrt(pow(k, slope) * exp(-(k / kc) * (k / kc))) / k2;
        }
        amp[i] = (float)c;
    }
}
// in place: w = i k_d amp w
__global__ void k_ic_component_f(int np, int nf, int d, const float* __restrict__ amp, float2* w) {
    const int64_t n = (int64_t)np * np * np;
    const double kf = 2.0 * kPi / nf;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % np), iy = (int)((i / np) % np), iz = (int)(i / ((int64_t)np * np));
        const int h = np / 2;
        const int nd = d == 0 ? (ix < h ? ix : ix - np) : (d == 1 ? (iy < h ? iy : iy - np)
                                                                  : (iz < h ? iz : iz - np));
        const double c = kf * nd * (double)amp[i];
        const float2 a = w[i];
        w[i] = make_float2((float)(-c * a.y), (float)(c * a.x));   // i c a
    }
}
__global__ void k_ic_store_f(int64_t n, int d, const float2* __restrict__ in, float* __restrict__ psi,
                             double* __restrict__ partial) {
    double acc = 0.0;
    const double inv_n = 1.0 / (double)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)((double)in[i].x * inv_n);
        psi[d * n + i] = v;
        acc += (double)v * v;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[d * gridDim.x + blockIdx.x] += sh[0];
}

}  // namespace

static int ic_zeldovich_lowmem(Sim& s, uint64_t seed, double slope, double kc, double rms) {
    const int np = s.np;
    const int64_t n = s.n;
    cudaStream_t st = s.stream;
    float2* w = s.ic_work;
    double* partial = s.ic_partial;
    const int nblk = 1024;
    cudaMemsetAsync(partial, 0, sizeof(double) * (3 * nblk + 1), st);
    int rc;
    // the amplitude lives in psi's last component until that component is stored
    float* amp = s.ic_psi + 2 * n;
    k_ic_amplitude_f<<<grid_for(n, 256), 256, 0, st>>>(np, s.nf, slope, kc, amp);
    for (int d = 0; d < 3; ++d) {
        k_ic_noise_f<<<grid_for(n, 256), 256, 0, st>>>(n, (unsigned long long)seed, w);
        if ((rc = fft3d<float>(s, w, np, -1))) return rc;
        k_ic_component_f<<<grid_for(n, 256), 256, 0, st>>>(np, s.nf, d, amp, w);
        if ((rc = fft3d<float>(s, w, np, 1))) return rc;
        k_ic_store_f<<<nblk, 256, 0, st>>>(n, d, w, s.ic_psi, partial);
    }
    double* scale = partial + 3 * nblk;
    k_ic_scale<<<1, 1, 0, st>>>(nblk, n, s.cfg.a_init, rms, partial, scale);
    s.launches += 3 * 3 + 2;
    if ((rc = check_launch(s, "ic"))) return rc;
    s.a = s.cfg.a_init;
    s.step = 0;
    set_device_step(s, 0);
    return encode_from_psi(s, scale);
}

int ic_zeldovich(Sim& s, uint64_t seed, double slope, double kc, double rms) {
    if (s.lowmem) return ic_zeldovich_lowmem(s, seed, slope, kc, rms);
    const int np = s.np;
    const int64_t n = s.n;
    cudaStream_t st = s.stream;
    // scratch: w~ [n] double2, work [n] double2, psi [3][n] double; Q/P alias the first two
    double2* w = reinterpret_cast<double2*>(s.scratch);
    double2* work = w + n;
    double* psi = reinterpret_cast<double*>(work + n);
    double* partial = s.ic_partial;
    const int nblk = 1024;
    cudaMemsetAsync(partial, 0, sizeof(double) * (3 * nblk + 1), st);
    k_ic_noise<<<grid_for(n, 256), 256, 0, st>>>(n, (unsigned long long)seed, w);
    int rc = fft3d<double>(s, w, np, -1);
    if (rc) return rc;
    // the amplitude lives in psi's last component until that component is stored
    double* amp = psi + 2 * n;
    // the amplitude table lives in the component buffer until the first component
    const int mmax = 3 * (np / 2) * (np / 2);
    double* tab = reinterpret_cast<double*>(work);
    k_ic_amp_table<<<grid_for(mmax + 1, 256), 256, 0, st>>>(mmax, s.nf, slope, kc, tab);
    k_ic_amplitude<<<grid_for(n, 256), 256, 0, st>>>(np, tab, amp);
    for (int d = 0; d < 3; ++d) {
        k_ic_component<<<grid_for(n, 256), 256, 0, st>>>(np, s.nf, d, amp, w, work);
        if ((rc = fft3d<double>(s, work, np, 1))) return rc;
        k_ic_store<<<nblk, 256, 0, st>>>(n, d, work, psi, partial);
    }
    double* scale = partial + 3 * nblk;
    k_ic_scale<<<1, 1, 0, st>>>(nblk, n, s.cfg.a_init, rms, partial, scale);
    auto kp = s.pb == 2 ? k_ic_particles<2> : k_ic_particles<1>;
    kp<<<grid_for(n, 256), 256, 0, st>>>(np, s.nc, s.cfg.a_init, s.ic_pfac, psi, scale, s.Qn, s.Pn);
    s.launches += 6 + 3 * 2;
    if ((rc = check_launch(s, "ic"))) return rc;
    s.a = s.cfg.a_init;
    s.step = 0;
    set_device_step(s, 0);
    return encode_from_qp(s, false);
}

}  // namespace pmpm
