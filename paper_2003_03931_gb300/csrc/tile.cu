// tile.cu -- the tile pass: for every tile, the short-range fine-mesh PM of
// Sec. II (deposit, FFT, Green multiply, inverse FFT) followed by the force
// interpolation and, in step mode, the kick and the integer drift.  One CTA
// of 512 threads per tile holds the whole 32^3 tile spectrum in shared
// memory (see tile_core.cuh).
#include "pmpm_impl.cuh"
#include "tile_core.cuh"

namespace pmpm {

__global__ void __launch_bounds__(kTileThreads, 1) k_tile(TileParams P) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    uint32_t* R = reinterpret_cast<uint32_t*>(tile_smem);
    float2* C = reinterpret_cast<float2*>(tile_smem);
    float2* W = reinterpret_cast<float2*>(tile_smem + (size_t)kTileR * 4);
    const int tid = threadIdx.x;
    const TileGeom g = tile_geom(blockIdx.x, P.nc, P.nt);

    tile_zero(tid, R);
    __syncthreads();
    tile_deposit(tid, g, P, R);
    __syncthreads();
    tile_fwd_x(tid, R);
    __syncthreads();
    tile_fwd_y(tid, C);
    __syncthreads();
    tile_fwd_z(tid, C);
    for (int d = 0; d < 3; ++d) {
        __syncthreads();
        tile_inv_z(tid, d, g, P.green, C, W);
        __syncthreads();
        tile_inv_y(tid, g, W);
        __syncthreads();
        tile_inv_x(tid, g, W);
        __syncthreads();
        tile_interp(tid, d, g, P, W);
    }
}

int tile_pass(Sim& s, int mode, float kick, float drift, float* G) {
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
    P.green = s.green_fine;
    P.Fl = s.Fl;
    P.mode = mode;
    P.kick = kick;
    P.drift = drift;
    P.G = G;
    P.Qn = s.Qn;
    P.Pn = s.Pn;
    P.counts_new = s.counts[1 - s.cur];
    P.S_new = s.S;
    P.err = s.err;
    cudaFuncSetAttribute(k_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
    const int ntiles = s.nt * s.nt * s.nt;
    k_tile<<<ntiles, kTileThreads, kTileSmemBytes, s.stream>>>(P);
    s.launches++;
    return check_launch(s, "tile pass");
}

}  // namespace pmpm
