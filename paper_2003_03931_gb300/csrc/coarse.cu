// coarse.cu -- long-range force on the coarse mesh (Sec. II: the long-range
// part lives on a mesh four times coarser than the fine one; Eq. 1 with
// K~_l).
//
//  1. integer CIC of all particles on the nc^3 coarse mesh (int64, units
//     2^-27 per particle): one thread per cell sums its particles' weights on
//     the 27 surrounding nodes in 32-bit registers, an 8x8x4-cell brick
//     collects them in shared memory (64-bit sums kept as two 32-bit words)
//     and flushes one global atomic per touched node;
//  2. delta = rho - mean (float64 subtraction, float32 storage), 3-D FFT;
//  3. Green multiply: B1 = rho~ (K~_x + i K~_y), B2 = rho~ K~_z (K~ = -i S);
//  4. two inverse FFTs give F_x + i F_y and F_z.
#include "pmpm_impl.cuh"

namespace pmpm {

namespace {

constexpr int kBX = 8, kBY = 8, kBZ = 4;
constexpr int kNX = kBX + 2, kNY = kBY + 2, kNZ = kBZ + 2;

// One thread per coarse cell: the cell's particles reach only the 3^3 nodes
// around it, so their weights are summed in 27 registers and added to the
// brick's shared accumulator once per cell.
template <int PB>
__global__ void __launch_bounds__(256) k_coarse_deposit(int nc, const int32_t* __restrict__ counts,
                                                        const int64_t* __restrict__ offsets,
                                                        const uint8_t* __restrict__ m0,
                                                        const uint8_t* __restrict__ m1,
                                                        const uint8_t* __restrict__ m2,
                                                        unsigned long long* rho) {
    // the brick's node sums as 32-bit halves: a native 32-bit shared atomic on
    // the low word, and the high word counts its wraps (at most one per add)
    __shared__ uint32_t acc_lo[kNX * kNY * kNZ], acc_hi[kNX * kNY * kNZ];
    const int nbx = nc / kBX, nby = nc / kBY;
    const int bx = blockIdx.x % nbx, by = (blockIdx.x / nbx) % nby, bz = blockIdx.x / (nbx * nby);
    const int x0 = bx * kBX, y0 = by * kBY, z0 = bz * kBZ;
    for (int i = threadIdx.x; i < kNX * kNY * kNZ; i += blockDim.x) {
        acc_lo[i] = 0u;
        acc_hi[i] = 0u;
    }
    __syncthreads();
    const int lx = threadIdx.x % kBX, ly = (threadIdx.x / kBX) % kBY, lz = threadIdx.x / (kBX * kBY);
    const int cx = x0 + lx, cy = y0 + ly, cz = z0 + lz;
    const int64_t cell = cx + (int64_t)nc * (cy + (int64_t)nc * cz);
    const int64_t j0 = offsets[cell];
    const int cnt = counts[cell];
    // A particle's weight on one node is at most its whole mass, 2^27 units,
    // so 31 particles sum below 2^32: 32-bit accumulators (one multiply-add
    // per node), added to the brick every kChunk particles.
    constexpr int kChunk = 31;
    for (int q0 = 0; q0 < cnt; q0 += kChunk) {
        uint32_t a[27];
#pragma unroll
        for (int k = 0; k < 27; ++k) a[k] = 0u;
        const int qe = min(cnt, q0 + kChunk);
#pragma unroll 2
        for (int q = q0; q < qe; ++q) {
            const int64_t j = j0 + q;
            // per axis: weights of nodes c-1, c, c+1 (in 1/(2B)); the bins in the
            // lower half lie left of the cell centre
            constexpr int B = PosFmt<PB>::kBins;
            uint32_t w[3][3];
            const int mm[3] = {load_bin<PB>(m0, j), load_bin<PB>(m1, j), load_bin<PB>(m2, j)};
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const int s = 2 * mm[e] + 1 - B;     // offset from the centre, 1/(2B)
                w[e][0] = s < 0 ? (uint32_t)(-s) : 0u;
                w[e][1] = (uint32_t)(2 * B) - (uint32_t)(s < 0 ? -s : s);
                w[e][2] = s > 0 ? (uint32_t)s : 0u;
            }
#pragma unroll
            for (int kz = 0; kz < 3; ++kz)
#pragma unroll
                for (int ky = 0; ky < 3; ++ky) {
                    if (PB == 1) {
                        // 1-byte bins: products below 2^27
                        const uint32_t wyz = w[1][ky] * w[2][kz];
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) a[kx + 3 * (ky + 3 * kz)] += wyz * w[0][kx];
                    } else {
                        // 2-byte bins: the 2^-51 product rounded to the 2^-27 unit
                        const unsigned long long wyz = (unsigned long long)w[1][ky] * w[2][kz];
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
                            a[kx + 3 * (ky + 3 * kz)] +=
                                (uint32_t)round_half_even_shift(wyz * w[0][kx], PosFmt<PB>::kRoundBits);
                    }
                }
        }
#pragma unroll
        for (int k = 0; k < 27; ++k) {
            if (!a[k]) continue;
            const int dx = k % 3, dy = (k / 3) % 3, dz = k / 9;
            const int i = (lx + dx) + kNX * ((ly + dy) + kNY * (lz + dz));
            const uint32_t old = atomicAdd(&acc_lo[i], a[k]);
            if (old + a[k] < old) atomicAdd(&acc_hi[i], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kNX * kNY * kNZ; i += blockDim.x) {
        const unsigned long long v = ((unsigned long long)acc_hi[i] << 32) | acc_lo[i];
        if (!v) continue;
        const int ix = i % kNX, iy = (i / kNX) % kNY, iz = i / (kNX * kNY);
        const int gx = wrap(x0 - 1 + ix, nc), gy = wrap(y0 - 1 + iy, nc), gz = wrap(z0 - 1 + iz, nc);
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

__global__ void k_coarse_green(int nc, const float4* __restrict__ table,
                               const float2* __restrict__ A, float2* __restrict__ B1,
                               float2* __restrict__ B2) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    const int64_t h = nc / 2 + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nc), ky = (int)((i / nc) % nc), kz = (int)(i / ((int64_t)nc * nc));
        int ax, ay, az;
        float sx, sy, sz;
        kfold(kx, nc, ax, sx);
        kfold(ky, nc, ay, sy);
        kfold(kz, nc, az, sz);
        // the three components' kernels at (|kx|, |ky|, |kz|), |kx| fastest
        const float4 g = table[(az * h + ay) * h + ax];
        const float Sx = sx * g.x, Sy = sy * g.y, Sz = sz * g.z;
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
    auto k = s.pb == 2 ? k_coarse_deposit<2> : k_coarse_deposit<1>;
    k<<<nb, 256, 0, s.stream>>>(s.nc, s.counts[s.cur], s.offsets[s.cur], m_stream(s, s.cur, 0),
                                m_stream(s, s.cur, 1), m_stream(s, s.cur, 2),
                                reinterpret_cast<unsigned long long*>(s.rho_c));
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
