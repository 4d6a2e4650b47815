// sort.cu -- cell-ordered re-encode of the particles (Sec. III-A: the bins
// m^i only locate a particle once the store is ordered by cell), with the
// per-cell counts, the cell-mean velocity v_c and the dispersion sigma of
// Eq. 3.
//
// Input: new codes Q [3][N] and momenta p [3][N] (float32), any order (the
// default step), or the old store and the new momenta (the low-memory step,
// which derives Q again with the tile pass's integer drift).
//   hist    counts[c], fixed-point momentum sums S[d][c] (int64, P = p
//           rounded to 2^-24) and T = sum P^2 (128 bits): exact integers,
//           independent of order (fused into the tile pass in a step)
//   scan    offsets = exclusive scan of counts (int64); v_c = fl32(fl32(S)
//           2^-24 / n)
//   sigma   U = sum over cells of floor(S^2 / n) (128 bits); sigma =
//           fl32(sqrt((T - U) 2^-48 / 3N)), the dispersion about the exact
//           cell means
//   scatter slot = offsets[c] + rank (atomic per cell); m = Q mod 256 and the
//           Eq. 3 code u (Eq. 4 guess + edge fix-up) written to the new store
// Within-cell order is not specified; every quantity above is independent of
// it, so the encoded store is the same multiset per cell on every run.
#include "pmpm_impl.cuh"

namespace pmpm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096 cells per block

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* sh, long long& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const long long before = warp > 0 ? sh[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(int64_t ncells, const int32_t* __restrict__ counts,
                                                              long long* __restrict__ blocksums) {
    __shared__ long long sh[32];
    const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
    long long acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = b0 + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < ncells) acc += counts[i];
    }
    long long total;
    block_exclusive_scan(acc, sh, total);
    if (threadIdx.x == 0) blocksums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(int64_t nb, long long* blocksums, int64_t n,
                                                   int64_t* offsets_end, uint32_t* err) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const long long v = i < nb ? blocksums[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, sh, total);
        if (i < nb) blocksums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        *offsets_end = carry;
        if (carry != n) atomicOr(err, kErrCount);
    }
}

// One tile of kScanTile cells per block.  Global loads and stores are
// striped (consecutive threads, consecutive cells); the scan runs over each
// thread's kScanItems consecutive cells, and shared memory, padded by one
// word in 16 against bank conflicts, transposes between the two orders.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int64_t ncells, const int32_t* __restrict__ counts,
                                                             const long long* __restrict__ blocksums,
                                                             int64_t* __restrict__ offsets,
                                                             const unsigned long long* __restrict__ S,
                                                             float* __restrict__ vc,
                                                             int32_t* __restrict__ fill) {
    __shared__ long long sh[32];
    __shared__ long long buf[kScanTile + kScanTile / 16];
    int* cbuf = reinterpret_cast<int*>(buf);
    const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
    const int t = threadIdx.x;
    int cst[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int p = k * kScanThreads + t;
        const int64_t i = b0 + p;
        cst[k] = i < ncells ? counts[i] : 0;
        cbuf[p + (p >> 4)] = cst[k];
    }
    // slot counters and cell means, in the striped order
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = b0 + k * kScanThreads + t;
        if (i >= ncells) break;
        if (fill) fill[i] = 0;
        if (S) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float v = 0.f;
                if (cst[k] > 0) {
                    const float sum = __fmul_rn(__ll2float_rn((long long)S[d * ncells + i]), 0x1p-24f);
                    v = __fdiv_rn(sum, (float)cst[k]);
                }
                vc[d * ncells + i] = v;
            }
        }
    }
    __syncthreads();
    int c[kScanItems];
    long long acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int p = t * kScanItems + k;
        c[k] = cbuf[p + (p >> 4)];
        acc += c[k];
    }
    long long total;
    // (its barriers also order the reads of cbuf before the writes to buf)
    long long run = blocksums[blockIdx.x] + block_exclusive_scan(acc, sh, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int p = t * kScanItems + k;
        buf[p + (p >> 4)] = run;
        run += c[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int p = k * kScanThreads + t;
        const int64_t i = b0 + p;
        if (i < ncells) offsets[i] = buf[p + (p >> 4)];
    }
}

// Where the encode kernels read each particle's new codes Q and momenta p:
// the per-particle buffers of the default step, or, for the low-memory
// initial conditions, the float32 displacement field (x = q + a Psi,
// p = a^(3/2) Psi in EdS (a^2 E f a Psi in LambdaCDM), Q = floor(64 x) mod 256 nc;
// Sec. IV-A.2).
struct QPArrays {
    const int32_t* Q;
    const float* P;
    int64_t n;
    __device__ __forceinline__ void load(int64_t i, int32_t (&q)[3], float (&p)[3]) const {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            q[d] = Q[d * n + i];
            p[d] = P[d * n + i];
        }
    }
};

struct QPFromPsi {
    const float* psi;      // [3][N]
    const double* scale;   // device scalar: rms normalisation
    int np, nc;
    double a, a15, spacing;
    int64_t n;
    __device__ __forceinline__ void load(int64_t i, int32_t (&q)[3], float (&p)[3]) const {
        const double sc = *scale;
        const int li[3] = {(int)(i % np), (int)((i / np) % np), (int)(i / ((int64_t)np * np))};
        const int64_t M = (int64_t)nc * kBins;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double ps = (double)psi[d * n + i] * sc;
            const double x = ((double)li[d] + 0.5) * spacing + a * ps;
            int64_t Q = (int64_t)floor(x * (double)kCodesPerFine) % M;
            if (Q < 0) Q += M;
            q[d] = (int32_t)Q;
            p[d] = (float)(a15 * ps);
        }
    }
};

// flat cell index of codes q (nc^3 <= 2^30: 32-bit)
template <int PB>
__device__ __forceinline__ int key3(const int32_t (&q)[3], int nc) {
    constexpr int sh = PosFmt<PB>::kShift;
    return (q[0] >> sh) + nc * ((q[1] >> sh) + nc * (q[2] >> sh));
}

// (lo, hi) of every thread of the block added to the 128-bit total held as
// digits in dst[0..3]: a warp then a block reduction, then add128_digits
__device__ __forceinline__ void block_add128(unsigned long long lo, unsigned long long hi,
                                             unsigned long long* dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, o);
        lo += l2;
        hi += h2 + (lo < l2 ? 1ull : 0ull);
    }
    __shared__ unsigned long long shl[32], shh[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { shl[warp] = lo; shh[warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        lo = 0; hi = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            lo += shl[w];
            hi += shh[w] + (lo < shl[w] ? 1ull : 0ull);
        }
        add128_digits(dst, lo, hi);
    }
}

// New-cell counts, fixed-point momentum sums S and the second moment
// T = sum P^2 of Eq. 3's dispersion (digits d2[0..3]).  Each thread takes kHistIlp
// particles at a time and issues all their loads before the atomics; the
// sums are integers, so their order does not matter.  (Grouping the lanes of
// a warp by cell before the atomics measured no faster: the kernel waits on
// its loads, not on atomic throughput.)
constexpr int kHistIlp = 4;
template <int PB, class Src>
__global__ void __launch_bounds__(256) k_hist(Src src, int64_t n, int nc, int32_t* counts,
                                              unsigned long long* S, unsigned long long* d2,
                                              uint32_t* err) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long tlo = 0, thi = 0;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n;
         i0 += stride * kHistIlp) {
        int32_t q[kHistIlp][3];
        float p[kHistIlp][3];
#pragma unroll
        for (int u = 0; u < kHistIlp; ++u) {
            const int64_t i = i0 + u * stride;
            q[u][0] = q[u][1] = q[u][2] = 0;
            p[u][0] = p[u][1] = p[u][2] = 0.f;
            if (i < n) src.load(i, q[u], p[u]);
        }
#pragma unroll
        for (int u = 0; u < kHistIlp; ++u) {
            if (i0 + u * stride >= n) continue;
            const int64_t key = key3<PB>(q[u], nc);
            atomicAdd(&counts[key], 1);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                long long fx = 0;
                if (fabsf(p[u][d]) < 1048576.f) fx = fix24_rn(p[u][d]);
                else atomicOr(err, p[u][d] == p[u][d] ? kErrMomentum : kErrNaN);
                atomicAdd(&S[d * ncells + key], (unsigned long long)fx);
                add_square128(fx, tlo, thi);
            }
        }
    }
    block_add128(tlo, thi, d2);
}

// U = sum over cells and axes of floor(S^2 / n) into the digits d2[4..7]
// (the cell-mean part of Eq. 3's dispersion; the new counts and sums S)
__global__ void __launch_bounds__(256) k_cell_moment(int64_t ncells, const int32_t* __restrict__ counts,
                                                     const unsigned long long* __restrict__ S,
                                                     unsigned long long* d2) {
    unsigned long long lo = 0, hi = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int cnt = counts[c];
        if (cnt <= 0) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) add_square_over_n128((long long)S[d * ncells + c], cnt, lo, hi);
    }
    block_add128(lo, hi, d2 + 4);
}

// sigma = fl32(sqrt((T - U) 2^-48 / 3N)), 2^-24 when T - U = 0 (T and U
// from the digits d2[0..3] and d2[4..7]; Eq. 3's dispersion about the exact
// cell means)
__global__ void k_sigma_final(const unsigned long long* d2, int64_t n, float* sigma) {
    unsigned long long tl, th, ul, uh;
    combine128(d2, tl, th);
    combine128(d2 + 4, ul, uh);
    const unsigned long long lo = tl - ul;
    const unsigned long long hi = th - uh - (tl < ul ? 1ull : 0ull);
    float s;
    if (lo == 0 && hi == 0) {
        s = kSigmaFloor;
    } else {
        const double v = __dadd_rn(__dmul_rn(__ull2double_rn(hi), 18446744073709551616.0),
                                   __ull2double_rn(lo));
        const double s2 = __ddiv_rn(__dmul_rn(v, 0x1p-48), (double)(3 * n));
        s = __double2float_rn(__dsqrt_rn(s2));
    }
    *sigma = s;
}

// The dispersion after the counts, sums S and T of the new cells: U per
// cell, then sigma of buffer nxt.
static void finish_sigma(Sim& s, int nxt) {
    k_cell_moment<<<grid_for(s.ncells, 256, 152 * 8), 256, 0, s.stream>>>(s.ncells, s.counts[nxt], s.S,
                                                                           s.d2);
    k_sigma_final<<<1, 1, 0, s.stream>>>(s.d2, s.n, s.sigma_d[nxt]);
    s.launches += 2;
}

// Slots and Eq. 2-3 codes of two particles per lane: slot = offsets[cell] +
// rank, m = Q mod 256 (or 65536) and the Eq. 3 code u.  Every lane of the warp
// calls (live[u] false: no particle).  Lanes with the same new cell take
// consecutive ranks from one atomic; the cell's offset range and mean
// momentum are loaded before the rank atomic returns.  A rank past the
// cell's count (counts that do not match the codes) is flagged, not written.
template <int PB>
__device__ __forceinline__ void scatter_two(const int32_t (&q)[2][3], const float (&p)[2][3],
                                            const bool (&live)[2], int64_t n, int nc,
                                            const float* const (&vcd)[3],
                                            const int64_t* __restrict__ offsets, int32_t* fill,
                                            float sigma, const float* Es, uint8_t* __restrict__ out,
                                            uint32_t* err) {
    const int lane = threadIdx.x & 31;
    int64_t off[2], end[2];
    int key[2];
    float v[2][3];
    int first[2];
    unsigned peers[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) key[u] = live[u] ? key3<PB>(q[u], nc) : -1 - lane;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const bool l = key[u] >= 0;
        off[u] = l ? offsets[key[u]] : 0;
        end[u] = l ? offsets[key[u] + 1] : 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) v[u][d] = l ? vcd[d][key[u]] : 0.f;
        peers[u] = __match_any_sync(0xffffffffu, key[u]);
        first[u] = 0;
        if (l && lane == __ffs(peers[u]) - 1) first[u] = atomicAdd(&fill[key[u]], __popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        first[u] = __shfl_sync(0xffffffffu, first[u], __ffs(peers[u]) - 1);
        if (key[u] < 0) continue;
        const int64_t slot = off[u] + first[u] + __popc(peers[u] & ((1u << lane) - 1u));
        if (slot >= end[u]) {
            atomicOr(err, kErrCount);
            continue;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (PB == 1) out[d * n + slot] = (uint8_t)(q[u][d] & 255);
            else reinterpret_cast<uint16_t*>(out + 2 * d * n)[slot] = (uint16_t)(q[u][d] & 65535);
            out[(3 * PB + d) * n + slot] = (uint8_t)encode_momentum(p[u][d], v[u][d], sigma, Es, err);
        }
    }
}

// Re-encode (Eq. 2-3) of the particles a source gives, in any order.  Each
// warp handles two particles per lane at a time.
template <int PB, class Src>
__global__ void k_scatter(Src src, int64_t n, int nc, const float* __restrict__ vc,
                          const int64_t* __restrict__ offsets, int32_t* fill,
                          const float* __restrict__ sigma_p, const float* __restrict__ E,
                          uint8_t* __restrict__ out, uint32_t* err) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    const float sigma = *sigma_p;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float* const vcd[3] = {vc, vc + ncells, vc + 2 * ncells};
    // the Eq. 3 bin edges, looked up once or twice per component
    __shared__ float Es[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) Es[k] = E[k];
    __syncthreads();
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n;
         base += 2 * stride) {
        int32_t q[2][3];
        float p[2][3];
        bool live[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = base + u * stride + lane;
            live[u] = i < n;
            q[u][0] = q[u][1] = q[u][2] = 0;
            p[u][0] = p[u][1] = p[u][2] = 0.f;
            if (live[u]) src.load(i, q[u], p[u]);
        }
        scatter_two<PB>(q, p, live, n, nc, vcd, offsets, fill, sigma, Es, out, err);
    }
}

constexpr int kParkThreads = 256;
constexpr int kParkSpan = 64;   // particles per warp iteration (two per lane)

// Low-memory step: re-encode from the old store and the new momenta Pn the
// tile pass left (no new codes were stored).  Particle j of the old store,
// in old cell c with bins m, moves to Q = drift_code(256 c + m, p) per axis:
// the same integer drift as the tile pass, so the same codes.  Each warp
// takes whole rows of cells (x fastest), row r in turn by warp r mod W, so
// the rows in flight at any time span several planes: a new cell's
// particles, which come from its old neighbours, are scattered while its
// part of the new store is still in L2.  Within a row, each particle's old
// cell comes from a window of 32 old offsets, one per lane, searched
// through shuffles (the next window only where a particle lies beyond it).
__global__ void __launch_bounds__(kParkThreads, 4)
k_scatter_parked(int64_t n, int nc, const int64_t* __restrict__ offs_old,
                 const uint8_t* __restrict__ st_old, const float* __restrict__ Pn,
                 const float* __restrict__ kd, const float* __restrict__ vc,
                 const int64_t* __restrict__ offsets, int32_t* fill,
                 const float* __restrict__ sigma_p, const float* __restrict__ E,
                 uint8_t* __restrict__ out, uint32_t* err) {
    __shared__ float Es[256];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int k = tid; k < 256; k += kParkThreads) Es[k] = E[k];
    __syncthreads();
    const int64_t ncells = (int64_t)nc * nc * nc, nrows = (int64_t)nc * nc;
    const float drift = kd[1], sigma = *sigma_p;
    const int M = nc * kBins;
    const float* const vcd[3] = {vc, vc + ncells, vc + 2 * ncells};
    const int64_t warps = (int64_t)gridDim.x * (kParkThreads / 32);
    for (int64_t row = (int64_t)blockIdx.x * (kParkThreads / 32) + (tid >> 5); row < nrows; row += warps) {
        // the row's particles; cw and (wx, wy, wz): the window's first cell
        int64_t cw = row * nc;
        const int64_t j1 = offs_old[cw + nc];
        int wx = 0, wy = (int)(row % nc), wz = (int)(row / nc);
        for (int64_t base = offs_old[cw]; base < j1; base += kParkSpan) {
            int64_t j[2];
            int cell[2], cc[2][3];   // cells below nc^3 <= 2^30
            bool live[2];
            int32_t q[2][3];
            float p[2][3];
            // the particles' bins and new momenta, loaded before the cell search
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                j[u] = base + 32 * u + lane;
                live[u] = j[u] < j1;
                cell[u] = -1;
                cc[u][0] = cc[u][1] = cc[u][2] = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    q[u][d] = live[u] ? st_old[d * n + j[u]] : 0;
                    p[u][d] = live[u] ? Pn[d * n + j[u]] : 0.f;
                }
            }
            // every particle of this span lies in cell cw or after it
            for (;;) {
                const int64_t wv = offs_old[cw + lane < ncells ? cw + lane : ncells];
                const int64_t wend = offs_old[cw + 32 < ncells ? cw + 32 : ncells];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    // the largest k with offsets[cw + k] <= j (all lanes shuffle)
                    int k = 0;
#pragma unroll
                    for (int b = 16; b > 0; b >>= 1) {
                        const int64_t w = __shfl_sync(0xffffffffu, wv, k + b);
                        if (w <= j[u]) k += b;
                    }
                    if (live[u] && cell[u] < 0 && j[u] < wend) {
                        // a particle of this row lies in a cell of this row
                        cell[u] = (int)(cw + k);
                        cc[u][0] = wx + k;
                        cc[u][1] = wy;
                        cc[u][2] = wz;
                    }
                }
                const bool need = (live[0] && cell[0] < 0) || (live[1] && cell[1] < 0);
                if (!__any_sync(0xffffffffu, need)) break;
                cw += 32;
                wx += 32;
            }
            // the next span starts in the cell of this span's last particle
            const int last = (int)((j1 < base + kParkSpan ? j1 : base + kParkSpan) - 1 - base);
            const int hi = last >= 32;
            cw = __shfl_sync(0xffffffffu, hi ? cell[1] : cell[0], last & 31);
            wx = __shfl_sync(0xffffffffu, hi ? cc[1][0] : cc[0][0], last & 31);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (!live[u]) continue;
#pragma unroll
                for (int d = 0; d < 3; ++d) q[u][d] = drift_code(cc[u][d] * kBins + q[u][d], p[u][d], drift, M, err);
            }
            scatter_two<1>(q, p, live, n, nc, vcd, offsets, fill, sigma, Es, out, err);
        }
    }
}

// decoded codes and momenta of the current store, storage order
template <int PB>
__global__ void k_decode(int64_t n, int nc, const int64_t* __restrict__ offsets,
                         const uint8_t* __restrict__ st, const float* __restrict__ vc,
                         const float* __restrict__ sigma_p, const float* __restrict__ T,
                         int32_t* __restrict__ Qn, float* __restrict__ Pn) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    const float sigma = *sigma_p;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        // cell c with offsets[c] <= j < offsets[c+1]
        int64_t lo = 0, hi = ncells;   // invariant offsets[lo] <= j < offsets[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (offsets[mid] <= j) lo = mid; else hi = mid;
        }
        const int64_t c = lo;
        const int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        const int cc[3] = {cx, cy, cz};
        for (int d = 0; d < 3; ++d) {
            Qn[d * n + j] = cc[d] * PosFmt<PB>::kBins + load_bin<PB>(st + (size_t)d * PB * n, j);
            Pn[d * n + j] = decode_momentum(vc[d * ncells + c], sigma, T[st[(3 * PB + d) * n + j]]);
        }
    }
}

}  // namespace

int scan_counts(Sim& s, const int32_t* counts, int64_t* offsets) {
    const int64_t nb = (s.ncells + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s.stream>>>(s.ncells, counts, s.blocksums);
    k_scan_top<<<1, 1024, 0, s.stream>>>(nb, s.blocksums, s.n, offsets + s.ncells, s.err);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s.stream>>>(s.ncells, counts, s.blocksums, offsets,
                                                             nullptr, nullptr, nullptr);
    s.launches += 3;
    return check_launch(s, "scan");
}

// Check of loaded counts on the device, before any kernel indexes the store
// through them: every count >= 0 and their sum N.  acc[0] gathers the sum,
// acc[1] the negative counts; the verdict sets kErrLoadCounts.
__global__ void __launch_bounds__(256) k_counts_sum(int64_t ncells, const int32_t* __restrict__ counts,
                                                    unsigned long long* acc) {
    __shared__ long long ssum[8];
    __shared__ unsigned sneg[8];
    long long sum = 0;
    unsigned neg = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = counts[i];
        sum += c;
        neg += c < 0 ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        neg += __shfl_down_sync(0xffffffffu, neg, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        ssum[warp] = sum;
        sneg[warp] = neg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            sum += ssum[w];
            neg += sneg[w];
        }
        atomicAdd(&acc[0], (unsigned long long)sum);
        if (neg) atomicAdd(&acc[1], (unsigned long long)neg);
    }
}

__global__ void k_counts_verdict(const unsigned long long* acc, int64_t n, uint32_t* err) {
    if ((long long)acc[0] != (long long)n || acc[1] != 0ull) atomicOr(err, kErrLoadCounts);
}

void check_loaded_counts(Sim& s) {
    cudaMemsetAsync(s.d2, 0, 16, s.stream);
    k_counts_sum<<<grid_for(s.ncells, 256, 152 * 8), 256, 0, s.stream>>>(s.ncells, s.counts[s.cur], s.d2);
    k_counts_verdict<<<1, 1, 0, s.stream>>>(s.d2, s.n, s.err);
    s.launches += 2;
}

// Offsets of the new counts, zeroed slot counters, and the new cell means
// v_c = fl32(fl32(S 2^-24) / count) of buffer nxt.
int scan_and_means(Sim& s, int nxt) {
    const int64_t nb = (s.ncells + kScanTile - 1) / kScanTile;
    cudaStream_t st = s.stream;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(s.ncells, s.counts[nxt], s.blocksums);
    k_scan_top<<<1, 1024, 0, st>>>(nb, s.blocksums, s.n, s.offsets[nxt] + s.ncells, s.err);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(s.ncells, s.counts[nxt], s.blocksums,
                                                        s.offsets[nxt], s.S, s.vc[nxt], s.fill);
    s.launches += 3;
    return check_launch(s, "scan");
}

// Encode s.Qn / s.Pn into the other store buffer and make it current.  With
// counts_ready the new counts and momentum sums were accumulated already
// (by the tile pass).
int encode_from_qp(Sim& s, bool counts_ready) {
    const int nxt = 1 - s.cur;
    cudaStream_t st = s.stream;
    if (!counts_ready) {
        cudaMemsetAsync(s.counts[nxt], 0, sizeof(int32_t) * s.ncells, st);
        cudaMemsetAsync(s.S, 0, sizeof(unsigned long long) * 3 * s.ncells, st);
        cudaMemsetAsync(s.d2, 0, 64, st);
        auto kh = s.pb == 2 ? k_hist<2, QPArrays> : k_hist<1, QPArrays>;
        kh<<<grid_for(s.n, 256, 152 * 8), 256, 0, st>>>(QPArrays{s.Qn, s.Pn, s.n}, s.n, s.nc,
                                                         s.counts[nxt], s.S, s.d2, s.err);
        s.launches++;
    }
    int rc = scan_and_means(s, nxt);
    if (rc) return rc;
    prof_mark(s, 3);
    finish_sigma(s, nxt);
    prof_mark(s, 4);
    auto kc = s.pb == 2 ? k_scatter<2, QPArrays> : k_scatter<1, QPArrays>;
    kc<<<grid_for(s.n, 256), 256, 0, st>>>(QPArrays{s.Qn, s.Pn, s.n}, s.n, s.nc, s.vc[nxt],
                                           s.offsets[nxt], s.fill, s.sigma_d[nxt], s.Eedge,
                                           s.streams[nxt], s.err);
    s.launches++;
    prof_mark(s, 5);
    s.cur = nxt;
    s.offsets_valid = true;
    s.have_state = true;
    s.loaded = 15;
    return check_launch(s, "encode");
}

// Low-memory initial conditions: encode (Q, p) computed from the float32
// displacement field straight into store 0 (the same kernels as the step's
// re-encode, reading the field instead of per-particle buffers).
int encode_from_psi(Sim& s, const double* scale) {
    cudaStream_t st = s.stream;
    const QPFromPsi src{s.ic_psi, scale, s.np, s.nc, s.cfg.a_init, s.ic_pfac,
                        4.0 * s.nc / (double)s.np, s.n};
    s.cur = 1;
    const int nxt = 0;
    lowmem_bind(s, nxt);   // S in store 0's region until the scatter writes it
    cudaMemsetAsync(s.counts[nxt], 0, sizeof(int32_t) * s.ncells, st);
    cudaMemsetAsync(s.S, 0, sizeof(unsigned long long) * 3 * s.ncells, st);
    cudaMemsetAsync(s.d2, 0, 64, st);
    k_hist<1><<<grid_for(s.n, 256, 152 * 8), 256, 0, st>>>(src, s.n, s.nc, s.counts[nxt], s.S, s.d2,
                                                           s.err);
    s.launches++;
    int rc = scan_and_means(s, nxt);
    if (rc) return rc;
    finish_sigma(s, nxt);
    k_scatter<1><<<grid_for(s.n, 256), 256, 0, st>>>(src, s.n, s.nc, s.vc[nxt], s.offsets[nxt], s.fill,
                                                  s.sigma_d[nxt], s.Eedge, s.streams[nxt], s.err);
    s.launches += 1;
    s.cur = nxt;
    s.offsets_valid = true;
    s.have_state = true;
    s.loaded = 15;
    return check_launch(s, "encode");
}

// The rest of a low-memory step (PMPM_FLAG_LOWMEM) after its tile pass,
// which counted the new cells, summed their momenta and left the new
// momenta in s.Pn: scan, cell means and the dispersion of Eq. 3, then the
// re-encode from the old store into the other store buffer.
int encode_from_parked(Sim& s) {
    const int nxt = 1 - s.cur;
    int rc = scan_and_means(s, nxt);
    if (rc) return rc;
    prof_mark(s, 3);
    finish_sigma(s, nxt);
    prof_mark(s, 4);
    const int grid = grid_for((int64_t)s.nc * s.nc, kParkThreads / 32, 152 * 4);
    k_scatter_parked<<<grid, kParkThreads, 0, s.stream>>>(
        s.n, s.nc, s.offsets[s.cur], s.streams[s.cur], s.Pn, s.d_kd, s.vc[nxt], s.offsets[nxt],
        s.fill, s.sigma_d[nxt], s.Eedge, s.streams[nxt], s.err);
    s.launches++;
    prof_mark(s, 5);
    s.cur = nxt;
    s.offsets_valid = true;
    s.have_state = true;
    s.loaded = 15;
    return check_launch(s, "low-memory encode");
}

int decode_state(Sim& s) {
    auto k = s.pb == 2 ? k_decode<2> : k_decode<1>;
    k<<<grid_for(s.n, 256), 256, 0, s.stream>>>(s.n, s.nc, s.offsets[s.cur], s.streams[s.cur],
                                                s.vc[s.cur], s.sigma_d[s.cur], s.Tdec, s.Qn, s.Pn);
    s.launches++;
    return check_launch(s, "decode");
}

}  // namespace pmpm
