// tile.cu -- the tile pass: for every tile, the short-range fine-mesh PM of
// Sec. II (deposit, FFT, Green multiply, inverse FFT) followed by the force
// interpolation and, in step mode, the kick and the integer drift.  One CTA
// of 512 threads per tile holds the whole 32^3 tile spectrum in shared
// memory (see tile_core.cuh).
#include "pmpm_impl.cuh"
#include "tile_core.cuh"

namespace pmpm {

// Optional per-phase clock stamps of thread 0 (compiled only with
// -DPMPM_PHASE_CLOCKS; read back through pmpm_debug_phases).
#ifdef PMPM_PHASE_CLOCKS
constexpr int kMarks = 24;
__device__ unsigned long long g_phase[4096 * kMarks];
#define PMPM_MARK(k)                                                                    \
    do {                                                                                \
        if (threadIdx.x == 0 && blockIdx.x < 4096) g_phase[blockIdx.x * kMarks + (k)] = clock64(); \
    } while (0)
#else
#define PMPM_MARK(k) \
    do {             \
    } while (0)
#endif

template <int D, bool LM, int PB, typename CT>
__device__ __forceinline__ void tile_component(int tid, const TileGeom& g, const TileParams& P,
                                               const float* gS, const CT* C, float2* W,
                                               TileCells cells,
                                               unsigned long long& lo, unsigned long long& hi,
                                               float gscale) {
    __syncthreads();
    PMPM_MARK(7 + 4 * D);
    if (D > 0) {   // the x force's inverse z ran with the forward z pass
        tile_inv_z<D>(tid, g, gS, C, W);
        __syncthreads();
    }
    PMPM_MARK(8 + 4 * D);
    tile_inv_y(tid, g, W);
    __syncthreads();
    PMPM_MARK(9 + 4 * D);
    tile_inv_x(tid, g, W);
    __syncthreads();
    PMPM_MARK(10 + 4 * D);
    tile_interp<D, LM, PB>(tid, g, P, W, cells, lo, hi, gscale);
}

// 128-bit block sum of the second moment T = sum P^2 of the tile's own
// particles' new momenta (the fused sums of mode 1), staged in the free W
// area, added to the digits d2[0..3] by thread 0 (no atomic is waited for:
// the CTA ends right after).
__device__ __forceinline__ void tile_sigma_flush(int tid, const TileParams& P, float2* W,
                                                 unsigned long long lo, unsigned long long hi) {
    unsigned long long* sh = reinterpret_cast<unsigned long long*>(W);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, o);
        lo += l2;
        hi += h2 + (lo < l2 ? 1ull : 0ull);
    }
    __syncthreads();
    if ((tid & 31) == 0) {
        sh[2 * (tid >> 5)] = lo;
        sh[2 * (tid >> 5) + 1] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        lo = 0;
        hi = 0;
        for (int w = 0; w < kTileThreads / 32; ++w) {
            lo += sh[2 * w];
            hi += sh[2 * w + 1] + (lo < sh[2 * w] ? 1ull : 0ull);
        }
        add128_digits(P.d2, lo, hi);
    }
}

// The whole tile: prologue, cell tables, deposit, forward transform, then
// per force component the Green multiply, inverse transform and
// interpolation (phases of tile_core.cuh with a block barrier between).
// CT: storage of the tile spectrum, float2 or (FP16 storage option) __half2.
// LM: the low-memory step (new codes not stored).
template <bool LM, int PB, typename CT = float2>
__device__ __forceinline__ void tile_body(int tile, const TileParams& P,
                                          unsigned char* tile_smem) {
    uint32_t* R = reinterpret_cast<uint32_t*>(tile_smem);
    CT* C = reinterpret_cast<CT*>(tile_smem);
    float2* W = reinterpret_cast<float2*>(tile_smem + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(tile_smem + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    const int tid = threadIdx.x;
    const TileGeom g = tile_geom(tile, P.nc, P.nt);
    const TileCells cells = tile_cells(W, O);   // W is free until phase 5
    PMPM_MARK(0);
    tile_prologue(tid, g, P, cells, R, gS);
    __syncthreads();
    PMPM_MARK(1);
    tile_cells_scan(tid, g, cells);
    __syncthreads();
    tile_cells_map(tid, g, cells);
    __syncthreads();
    PMPM_MARK(2);
    tile_deposit_flat<PB>(tid, g, P, R, cells);
    __syncthreads();
    PMPM_MARK(3);
    // FP16 storage: the density less its mean over the halo box (the k = 0
    // mode, where the short-range kernel vanishes) is scaled by 2^-e so that
    // every spectrum value, at most 2 x 2^22 per particle of the box (the
    // forward x transform doubles), stays below 2^15; the interpolation
    // undoes the scale exactly
    float scale = 1.f, gscale = 2.384185791015625e-07f, mean = 0.f;
    if (!std::is_same<CT, float2>::value) {
        const int total = cells.pre[kHaloMax];
        const int e = 8 + (total > 1 ? 32 - __clz(total - 1) : 0);
        scale = ldexpf(1.f, -e);
        gscale = ldexpf(1.f, e - 22);
        const int hx = g.c1[0] - g.c0[0] + 4, hy = g.c1[1] - g.c0[1] + 4, hz = g.c1[2] - g.c0[2] + 4;
        mean = (float)total * 2097152.f / (64.f * (float)(hx * hy * hz));
    }
    tile_fwd_x<CT>(tid, R, scale, mean);
    __syncthreads();
    PMPM_MARK(4);
    tile_fwd_y(tid, C);
    __syncthreads();
    PMPM_MARK(5);
    tile_fwd_z_inv_z0(tid, g, gS, C, W);
    unsigned long long lo = 0, hi = 0;
    tile_component<0, LM, PB>(tid, g, P, gS, C, W, cells, lo, hi, gscale);
    tile_component<1, LM, PB>(tid, g, P, gS, C, W, cells, lo, hi, gscale);
    tile_component<2, LM, PB>(tid, g, P, gS, C, W, cells, lo, hi, gscale);
    if (P.mode == 1 && P.counts_new != nullptr) tile_sigma_flush(tid, P, W, lo, hi);
    __syncthreads();
    PMPM_MARK(19);
}

// One CTA per tile; one fits an SM at a time (the tile needs 232 KB of shared
// memory).
// PB: bytes per position bin; CT: storage of the tile spectrum; LM: the
// low-memory step.
template <int PB, typename CT, bool LM = false>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile(TileParams P) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    tile_body<LM, PB, CT>((int)blockIdx.x, P, tile_smem);
}

// One tile's fine-mesh box right after the deposit, written out in x-fastest
// node order (a check of the integer CIC; not part of a step).
template <int PB>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile_density(TileParams P, int tile,
                                                                   uint32_t* out) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    uint32_t* R = reinterpret_cast<uint32_t*>(tile_smem);
    float2* W = reinterpret_cast<float2*>(tile_smem + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(tile_smem + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    const int tid = threadIdx.x;
    const TileGeom g = tile_geom(tile, P.nc, P.nt);
    const TileCells cells = tile_cells(W, O);
    tile_prologue(tid, g, P, cells, R, gS);
    __syncthreads();
    tile_cells_scan(tid, g, cells);
    __syncthreads();
    tile_cells_map(tid, g, cells);
    __syncthreads();
    tile_deposit_halo<PB>(tid, g, P, R, cells);
    __syncthreads();
    for (int i = tid; i < kTileR; i += kTileThreads) out[i] = R[ridx(i & 31, (i >> 5) & 31, i >> 10)];
}

void tile_setup() {
    cudaFuncSetAttribute(k_tile<1, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
    cudaFuncSetAttribute(k_tile<2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
    cudaFuncSetAttribute(k_tile<1, __half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
    cudaFuncSetAttribute(k_tile<2, __half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
    cudaFuncSetAttribute(k_tile<1, float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTileSmemBytes);
    cudaFuncSetAttribute(k_tile_density<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
    cudaFuncSetAttribute(k_tile_density<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
}

// the parameters every tile kernel reads: the current store, the tables and F_l
static TileParams base_params(Sim& s) {
    TileParams P{};
    P.nc = s.nc;
    P.nt = s.nt;
    P.n = s.n;
    P.counts = s.counts[s.cur];
    P.offsets = s.offsets[s.cur];
    P.m0 = m_stream(s, s.cur, 0);
    P.m1 = m_stream(s, s.cur, 1);
    P.m2 = m_stream(s, s.cur, 2);
    P.u0 = u_stream(s, s.cur, 0);
    P.u1 = u_stream(s, s.cur, 1);
    P.u2 = u_stream(s, s.cur, 2);
    P.vc = s.vc[s.cur];
    P.sigma = s.sigma_d[s.cur];
    P.Tdec = s.Tdec;
    P.green = s.green_packed;
    P.Fl = s.Fl;
    P.kd = s.d_kd;
    P.Qn = s.Qn;
    P.Pn = s.Pn;
    P.err = s.err;
    return P;
}

int tile_pass(Sim& s, int mode, float* G) {
    TileParams P = base_params(s);
    P.mode = mode;
    P.G = G;
    const int grid = s.nt * s.nt * s.nt;
    if (mode == 1) {
        P.counts_new = s.counts[1 - s.cur];
        P.S = s.S;
        P.d2 = s.d2;
    }
    if (s.lowmem) {
        // the low-memory step keeps the new momenta only (s.Pn); the new codes
        // are derived again by its re-encode
        P.Qn = nullptr;
        k_tile<1, float2, true><<<grid, kTileThreads, kTileSmemBytes, s.stream>>>(P);
    } else if (s.fp16 && s.pb == 2) k_tile<2, __half2><<<grid, kTileThreads, kTileSmemBytes, s.stream>>>(P);
    else if (s.fp16) k_tile<1, __half2><<<grid, kTileThreads, kTileSmemBytes, s.stream>>>(P);
    else if (s.pb == 2) k_tile<2, float2><<<grid, kTileThreads, kTileSmemBytes, s.stream>>>(P);
    else k_tile<1, float2><<<grid, kTileThreads, kTileSmemBytes, s.stream>>>(P);
    s.launches++;
    return check_launch(s, "tile pass");
}

int tile_density(Sim& s, int tile, uint32_t* d_out) {
    TileParams P = base_params(s);
    P.mode = 0;
    if (s.pb == 2) k_tile_density<2><<<1, kTileThreads, kTileSmemBytes, s.stream>>>(P, tile, d_out);
    else k_tile_density<1><<<1, kTileThreads, kTileSmemBytes, s.stream>>>(P, tile, d_out);
    s.launches++;
    return check_launch(s, "tile density");
}

}  // namespace pmpm

#ifdef PMPM_PHASE_CLOCKS
extern "C" int pmpm_debug_phases(unsigned long long* out, int n) {
    return (int)cudaMemcpyFromSymbol(out, pmpm::g_phase, sizeof(unsigned long long) * n);
}
#endif
