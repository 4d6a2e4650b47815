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

template <int D>
__device__ __forceinline__ void tile_component(int tid, const TileGeom& g, const TileParams& P,
                                               const float* gS, const float2* C, float2* W,
                                               TileCells cells) {
    __syncthreads();
    PMPM_MARK(7 + 4 * D);
    tile_inv_z<D>(tid, g, gS, C, W);
    __syncthreads();
    PMPM_MARK(8 + 4 * D);
    tile_inv_y(tid, g, W);
    __syncthreads();
    PMPM_MARK(9 + 4 * D);
    tile_inv_x(tid, g, W);
    __syncthreads();
    PMPM_MARK(10 + 4 * D);
    tile_interp<D>(tid, g, P, W, cells);
}

__global__ void __launch_bounds__(kTileThreads, 1) k_tile(TileParams P) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    uint32_t* R = reinterpret_cast<uint32_t*>(tile_smem);
    float2* C = reinterpret_cast<float2*>(tile_smem);
    float2* W = reinterpret_cast<float2*>(tile_smem + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(tile_smem + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    const int tid = threadIdx.x;
    const TileGeom g = tile_geom(blockIdx.x, P.nc, P.nt);

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
    tile_deposit_flat(tid, g, P, R, cells);
    __syncthreads();
    PMPM_MARK(3);
    tile_fwd_x(tid, R);
    __syncthreads();
    PMPM_MARK(4);
    tile_fwd_y(tid, C);
    __syncthreads();
    PMPM_MARK(5);
    tile_fwd_z(tid, C);
    tile_component<0>(tid, g, P, gS, C, W, cells);
    tile_component<1>(tid, g, P, gS, C, W, cells);
    tile_component<2>(tid, g, P, gS, C, W, cells);
    __syncthreads();
    PMPM_MARK(19);
}

void tile_setup() {
    cudaFuncSetAttribute(k_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
}

int tile_pass(Sim& s, int mode, float* G) {
    TileParams P;
    P.nc = s.nc;
    P.nt = s.nt;
    P.n = s.n;
    P.counts = s.counts[s.cur];
    P.offsets = s.offsets[s.cur];
    P.m0 = cur_stream(s, 0);
    P.m1 = cur_stream(s, 1);
    P.m2 = cur_stream(s, 2);
    P.u0 = cur_stream(s, 3);
    P.u1 = cur_stream(s, 4);
    P.u2 = cur_stream(s, 5);
    P.vc = s.vc[s.cur];
    P.sigma = s.sigma_d[s.cur];
    P.Tdec = s.Tdec;
    P.green = s.green_packed;
    P.Fl = s.Fl;
    P.mode = mode;
    P.kd = s.d_kd;
    P.G = G;
    P.Qn = s.Qn;
    P.Pn = s.Pn;
    P.err = s.err;
    const int ntiles = s.nt * s.nt * s.nt;
    k_tile<<<ntiles, kTileThreads, kTileSmemBytes, s.stream>>>(P);
    s.launches++;
    return check_launch(s, "tile pass");
}

}  // namespace pmpm

#ifdef PMPM_PHASE_CLOCKS
extern "C" int pmpm_debug_phases(unsigned long long* out, int n) {
    return (int)cudaMemcpyFromSymbol(out, pmpm::g_phase, sizeof(unsigned long long) * n);
}
#endif
