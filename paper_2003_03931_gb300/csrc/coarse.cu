// coarse.cu -- long-range force on the coarse mesh (Sec. II: "F_l is usually
// computed on a 4-times-coarser mesh"; Eq. 1 with K~_l).
//
//  1. integer CIC of all particles on the nc^3 coarse mesh (int64, units
//     2^-27 per particle), accumulated per 8x8x4-cell brick in shared memory
//     and flushed with one global atomic per touched node;
//  2. delta = rho - mean (float64 subtraction, float32 storage), 3-D FFT;
//  3. Green multiply: B1 = rho~ (K~_x + i K~_y), B2 = rho~ K~_z (K~ = -i S);
//  4. two inverse FFTs give F_x + i F_y and F_z.
#include "pmpm_impl.cuh"

namespace pmpm {

namespace {

constexpr int kBX = 8, kBY = 8, kBZ = 4;
constexpr int kNX = kBX + 2, kNY = kBY + 2, kNZ = kBZ + 2;

__global__ void __launch_bounds__(256) k_coarse_deposit(int nc, const int32_t* __restrict__ counts,
                                                        const int64_t* __restrict__ offsets,
                                                        const uint8_t* __restrict__ m0,
                                                        const uint8_t* __restrict__ m1,
                                                        const uint8_t* __restrict__ m2,
                                                        unsigned long long* rho) {
    __shared__ unsigned long long acc[kNX * kNY * kNZ];
    const int nbx = nc / kBX, nby = nc / kBY;
    const int bx = blockIdx.x % nbx, by = (blockIdx.x / nbx) % nby, bz = blockIdx.x / (nbx * nby);
    const int x0 = bx * kBX, y0 = by * kBY, z0 = bz * kBZ;
    for (int i = threadIdx.x; i < kNX * kNY * kNZ; i += blockDim.x) acc[i] = 0ull;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < kBY * kBZ; r += blockDim.x / 32) {
        const int y = y0 + r % kBY, z = z0 + r / kBY;
        const int64_t base = (int64_t)nc * (y + (int64_t)nc * z) + x0;
        int64_t st[kBX + 1];
#pragma unroll
        for (int i = 0; i <= kBX; ++i) st[i] = offsets[base + i];
        const int64_t total = st[kBX] - st[0];
        for (int64_t v = lane; v < total; v += 32) {
            const int64_t j = st[0] + v;
            int cx = 0;
#pragma unroll
            for (int i = 1; i < kBX; ++i)
                if (st[i] <= j) cx = i;
            const int64_t Q[3] = {(int64_t)(x0 + cx) * kBins + m0[j], (int64_t)y * kBins + m1[j],
                                  (int64_t)z * kBins + m2[j]};
            Cic1 c[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) c[e] = cic_coarse(Q[e]);
            const int lx = c[0].i0 - (x0 - 1), ly = c[1].i0 - (y0 - 1), lz = c[2].i0 - (z0 - 1);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
                const unsigned long long w =
                    (unsigned long long)((dx ? c[0].w1 : 512 - c[0].w1) *
                                         (dy ? c[1].w1 : 512 - c[1].w1)) *
                    (unsigned long long)(dz ? c[2].w1 : 512 - c[2].w1);
                if (w) atomicAdd(&acc[(lx + dx) + kNX * ((ly + dy) + kNY * (lz + dz))], w);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kNX * kNY * kNZ; i += blockDim.x) {
        const unsigned long long v = acc[i];
        if (!v) continue;
        const int lx = i % kNX, ly = (i / kNX) % kNY, lz = i / (kNX * kNY);
        const int gx = wrap(x0 - 1 + lx, nc), gy = wrap(y0 - 1 + ly, nc), gz = wrap(z0 - 1 + lz, nc);
        atomicAdd(&rho[gx + (int64_t)nc * (gy + (int64_t)nc * gz)], v);
    }
}

__global__ void k_coarse_delta(int64_t ncells, double mean, const long long* __restrict__ rho,
                               float2* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)((double)rho[i] - mean), 0.f);
}

__device__ __forceinline__ void kfold(int k, int nc, int& a, float& sg) {
    if (k == 0) { a = 0; sg = 0.f; }
    else if (k <= nc / 2) { a = k; sg = 1.f; }
    else { a = nc - k; sg = -1.f; }
}

__global__ void k_coarse_green(int nc, const float* __restrict__ table,
                               const float2* __restrict__ A, float2* __restrict__ B1,
                               float2* __restrict__ B2) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    const int h = nc / 2 + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nc), ky = (int)((i / nc) % nc), kz = (int)(i / ((int64_t)nc * nc));
        int ax, ay, az;
        float sx, sy, sz;
        kfold(kx, nc, ax, sx);
        kfold(ky, nc, ay, sy);
        kfold(kz, nc, az, sz);
        const float Sx = sx * table[((int64_t)ax * h + ay) * h + az];
        const float Sy = sy * table[((int64_t)ay * h + ax) * h + az];
        const float Sz = sz * table[((int64_t)az * h + ay) * h + ax];
        const float2 a = A[i];
        // B1 = a (S_y - i S_x),  B2 = a (-i S_z)
        B1[i] = make_float2(a.x * Sy + a.y * Sx, a.y * Sy - a.x * Sx);
        B2[i] = make_float2(a.y * Sz, -a.x * Sz);
    }
}

__global__ void k_coarse_extract(int64_t ncells, const float2* __restrict__ B1,
                                 const float2* __restrict__ B2, float* __restrict__ Fl) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 b1 = B1[i];
        Fl[i] = b1.x;
        Fl[ncells + i] = b1.y;
        Fl[2 * ncells + i] = B2[i].x;
    }
}

}  // namespace

int coarse_deposit(Sim& s) {
    cudaMemsetAsync(s.rho_c, 0, sizeof(long long) * s.ncells, s.stream);
    const int nb = (s.nc / kBX) * (s.nc / kBY) * (s.nc / kBZ);
    k_coarse_deposit<<<nb, 256, 0, s.stream>>>(
        s.nc, s.counts[s.cur], s.offsets[s.cur], cur_stream(s, 0), cur_stream(s, 1),
        cur_stream(s, 2), reinterpret_cast<unsigned long long*>(s.rho_c));
    s.launches++;
    return check_launch(s, "coarse deposit");
}

int coarse_force(Sim& s) {
    const int64_t nc3 = s.ncells;
    const double mean = (double)s.n * 134217728.0 / (double)nc3;   // N 2^27 / nc^3
    k_coarse_delta<<<grid_for(nc3, 256), 256, 0, s.stream>>>(nc3, mean, s.rho_c, s.cA);
    s.launches++;
    int rc = fft3d<float>(s, s.cA, s.nc, -1);
    if (rc) return rc;
    k_coarse_green<<<grid_for(nc3, 256), 256, 0, s.stream>>>(s.nc, s.green_coarse, s.cA, s.cB1,
                                                            s.cB2);
    s.launches++;
    if ((rc = fft3d<float>(s, s.cB1, s.nc, 1))) return rc;
    if ((rc = fft3d<float>(s, s.cB2, s.nc, 1))) return rc;
    k_coarse_extract<<<grid_for(nc3, 256), 256, 0, s.stream>>>(nc3, s.cB1, s.cB2, s.Fl);
    s.launches++;
    return check_launch(s, "coarse force");
}

}  // namespace pmpm
