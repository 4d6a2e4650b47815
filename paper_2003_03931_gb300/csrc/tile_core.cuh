// tile_core.cuh -- the fine-mesh (short-range) PM of one tile, Sec. II:
// "F_s on each V_tile is computed by a fine-mesh PM on a slightly enlarged
// volume (L/N_tile + 2 r_cutoff)^3".  One CTA of 512 threads owns one tile.
//
// Tile geometry.  A tile is a box of whole coarse cells, 4 or 5 per side
// (T = 16 or 20 fine cells).  Its FFT box is 32^3 fine nodes starting at
// fine node 4*c0 - 6, so it holds the tile plus a 6-cell buffer on each side
// (T + 12 <= 32).  The short-range kernel vanishes beyond 6 fine cells, so the
// circular convolution on the 32^3 box equals the whole-box convolution on
// the fine nodes [-1, T] that the tile's particles gather from.
//
// Shared memory (one CTA per SM):
//   R  32 KB x 4 B = 128 KB: integer density (uint32, units 2^-21 per
//      particle), then its 3-D spectrum packed as 16 x 32 x 32 complex with
//      the kx = 16 (Nyquist) plane folded into the imaginary part of kx = 0;
//   W  22 x 32 x 16 complex = 88 KB: one force component on its way back,
//      pruned to the 22 output planes that are needed.
// Index swizzles (x ^ y) make every pencil pass free of bank conflicts.
//
// Each phase is a per-thread function; the kernel calls them with a block
// barrier between phases.
#pragma once

#include "common.cuh"
#include "regfft.cuh"

namespace pmpm {

constexpr int kTileThreads = 512;
constexpr int kTileR = kTileFFT * kTileFFT * kTileFFT;          // 32768 words
constexpr int kTileW = kTileOut * kTileFFT * (kTileFFT / 2);    // 11264 complex
constexpr size_t kTileSmemBytes = (size_t)kTileR * 4 + (size_t)kTileW * 8;

struct TileParams {
    int nc;                       // coarse cells per side
    int nt;                       // tiles per side
    int64_t n;                    // particles
    const int32_t* counts;        // [nc^3]
    const int64_t* offsets;       // [nc^3 + 1]
    const uint8_t* m0;            // position bins (Eq. 2), storage order
    const uint8_t* m1;
    const uint8_t* m2;
    const uint8_t* u0;            // velocity bins (Eq. 3)
    const uint8_t* u1;
    const uint8_t* u2;
    const float* vc;              // [3][nc^3]
    const float* sigma;           // device scalar
    const float* Tdec;            // [256] decode table
    const float* green;           // [17][17][17] short-range Green table (scaled)
    const float* Fl;              // [3][nc^3] long-range force on the coarse mesh
    int mode;                     // 0: write g; 1: kick + drift
    float kick;                   // fl32 kick factor (multiplies g)
    float drift;                  // fl32 drift factor in position codes (multiplies p)
    float* G;                     // [3][N] (mode 0)
    int32_t* Qn;                  // [3][N] new codes (mode 1)
    float* Pn;                    // [3][N] new momenta (mode 1)
    int32_t* counts_new;          // [nc^3] (mode 1)
    unsigned long long* S_new;    // [3][nc^3] fixed-point momentum sums (mode 1)
    uint32_t* err;
};

struct TileGeom {
    int c0[3], c1[3];   // coarse-cell range [c0, c1) of the tile
    int T[3];           // fine cells per side
    int o[3];           // fine node of mesh index 0: 4*c0 - 6
};

PMPM_HD TileGeom tile_geom(int b, int nc, int nt) {
    TileGeom g;
    int t[3] = {b % nt, (b / nt) % nt, b / (nt * nt)};
    for (int d = 0; d < 3; ++d) {
        g.c0[d] = tile_bound(t[d], nc, nt);
        g.c1[d] = tile_bound(t[d] + 1, nc, nt);
        g.T[d] = kRatio * (g.c1[d] - g.c0[d]);
        g.o[d] = kRatio * g.c0[d] - kBuffer;
    }
    return g;
}

// --- shared-memory index maps ------------------------------------------------
PMPM_HD int ridx(int x, int y, int z) { return ((z << 5) + y) * 32 + (x ^ y); }
PMPM_HD int cidx(int kx, int ky, int kz) { return ((kz << 5) + ky) * 16 + (kx ^ (ky & 15)); }
PMPM_HD int widx(int kx, int ky, int zo) { return ((zo << 5) + ky) * 16 + (kx ^ (ky & 15)); }
PMPM_HD int wfidx(int xo, int yo, int zo) {
    return 2 * (((zo << 5) + yo) * 16 + ((xo >> 1) ^ (yo & 15))) + (xo & 1);
}

#ifdef __CUDA_ARCH__
PMPM_HD uint32_t smem_add_u32(uint32_t* p, uint32_t v) { return atomicAdd(p, v); }
PMPM_HD void gmem_add_i32(int32_t* p, int32_t v) { atomicAdd(p, v); }
PMPM_HD void gmem_add_u64(unsigned long long* p, unsigned long long v) { atomicAdd(p, v); }
PMPM_HD float u32_to_f32(uint32_t v) { return __uint2float_rn(v); }
PMPM_HD long long f64_to_ll_rn(double v) { return __double2ll_rn(v); }
#else
PMPM_HD uint32_t smem_add_u32(uint32_t* p, uint32_t v) { uint32_t o = *p; *p = o + v; return o; }
PMPM_HD void gmem_add_i32(int32_t* p, int32_t v) { *p += v; }
PMPM_HD void gmem_add_u64(unsigned long long* p, unsigned long long v) { *p += v; }
PMPM_HD float u32_to_f32(uint32_t v) { return (float)v; }
PMPM_HD long long f64_to_ll_rn(double v) { return llrint(v); }
#endif

// --- phase 0: clear the density --------------------------------------------
PMPM_HD void tile_zero(int tid, uint32_t* R) {
    for (int i = tid; i < kTileR; i += kTileThreads) R[i] = 0u;
}

// Per-lane table of up to 9 consecutive cells of one row: prefix counts and
// storage offsets, held in registers (fixed-size, fully unrolled).
struct RowCells {
    int pc[10];          // pc[i] = particles in cells before i; pc[n] = total
    int64_t st[9];       // storage offset of cell i
    int n;
};

PMPM_HD void row_cells(RowCells& rc, const TileParams& P, int base, int x_first, int ncell) {
    rc.n = ncell;
    int acc = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        rc.pc[i] = acc;
        rc.st[i] = 0;
        if (i < ncell) {
            int cell = base + wrap(x_first + i, P.nc);
            rc.st[i] = P.offsets[cell];
            acc += P.counts[cell];
        }
    }
    rc.pc[9] = acc;
    if (ncell < 9) {
#pragma unroll
        for (int i = 0; i < 10; ++i)
            if (i > ncell) rc.pc[i] = acc;
    }
}

PMPM_HD int row_find(const RowCells& rc, int v) {
    int c = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i)
        if (i < rc.n && rc.pc[i] <= v) c = i;
    return c;
}

// --- phase 1: integer CIC of the tile and its 2-coarse-cell halo ------------
// Particles in coarse cells [c0 - 2, c1 + 2) can reach the mesh nodes
// [-6, T + 5]; their contributions outside the 32^3 box are clipped.
PMPM_HD void tile_deposit(int tid, const TileGeom& g, const TileParams& P, uint32_t* R) {
    const int warp = tid >> 5, lane = tid & 31;
    const int hx = g.c1[0] - g.c0[0] + 4, hy = g.c1[1] - g.c0[1] + 4, hz = g.c1[2] - g.c0[2] + 4;
    const int nrows = hy * hz;
    for (int r = warp; r < nrows; r += kTileThreads / 32) {
        const int yu = g.c0[1] - 2 + r % hy, zu = g.c0[2] - 2 + r / hy;
        const int base = P.nc * (wrap(yu, P.nc) + P.nc * wrap(zu, P.nc));
        RowCells rc;
        row_cells(rc, P, base, g.c0[0] - 2, hx);
        const int total = rc.pc[9];
        for (int v = lane; v < total; v += 32) {
            const int i = row_find(rc, v);
            const int64_t j = rc.st[i] + (v - rc.pc[i]);
            const int cu[3] = {g.c0[0] - 2 + i, yu, zu};
            const int m[3] = {P.m0[j], P.m1[j], P.m2[j]};
            int li[3], w1[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                // s = 2Q + 1 - 64 relative to the mesh origin, units 1/128
                int s = 2 * (cu[d] * kBins + m[d]) + 1 - kCodesPerFine - 128 * g.o[d];
                li[d] = s >> 7;
                w1[d] = s & 127;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
                const int x = li[0] + dx, y = li[1] + dy, z = li[2] + dz;
                if ((unsigned)x >= 32u || (unsigned)y >= 32u || (unsigned)z >= 32u) continue;
                const uint32_t w = (uint32_t)((dx ? w1[0] : 128 - w1[0]) *
                                              (dy ? w1[1] : 128 - w1[1]) *
                                              (dz ? w1[2] : 128 - w1[2]));
                if (w == 0u) continue;
                const uint32_t old = smem_add_u32(&R[ridx(x, y, z)], w);
                if (old + w < old) flag_error(P.err, kErrFineOverflow);
            }
        }
    }
}

// --- phase 2: forward real transform along x (1024 rows, 2 per thread) -----
PMPM_HD void tile_fwd_x(int tid, uint32_t* R) {
    float2* C = reinterpret_cast<float2*>(R);
    for (int r = tid; r < 1024; r += kTileThreads) {
        const int y = r & 31, z = r >> 5;
        float x[32];
#pragma unroll
        for (int n = 0; n < 32; ++n) x[n] = u32_to_f32(R[ridx(n, y, z)]);
        float2 X[17];
        rfft32(x, X);
        C[cidx(0, y, z)] = make_float2(X[0].x, X[16].x);   // pack Nyquist
#pragma unroll
        for (int k = 1; k < 16; ++k) C[cidx(k, y, z)] = X[k];
    }
}

// --- phase 3/4: forward complex transforms along y and z (512 pencils) ------
PMPM_HD void tile_fwd_y(int tid, float2* C) {
    const int kx = tid & 15, z = tid >> 4;
    float2 a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = C[cidx(kx, k, z)];
    fft_bitrev_out<32, -1>(a);
#pragma unroll
    for (int k = 0; k < 32; ++k) C[cidx(kx, k, z)] = a[bitrev<5>(k)];
}

PMPM_HD void tile_fwd_z(int tid, float2* C) {
    const int kx = tid & 15, ky = tid >> 4;
    float2 a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = C[cidx(kx, ky, k)];
    fft_bitrev_out<32, -1>(a);
#pragma unroll
    for (int k = 0; k < 32; ++k) C[cidx(kx, ky, k)] = a[bitrev<5>(k)];
}

// |signed frequency| and its sign for a 32-point index
PMPM_HD int kabs32(int i) { return i <= 16 ? i : 32 - i; }
PMPM_HD float ksgn32(int i) { return i == 0 ? 0.f : (i < 16 ? 1.f : (i == 16 ? 1.f : -1.f)); }

// Green coefficient S_d(kx, ky, kz) with K~_d = -i S_d; table index
// [own axis][other][other], symmetric in the last two.
PMPM_HD float green_S(const float* Gt, int d, int kx, int ky, int kz) {
    const int ax = kabs32(kx), ay = kabs32(ky), az = kabs32(kz);
    if (d == 0) return ksgn32(kx) * Gt[(ax * kGreenS + ay) * kGreenS + az];
    if (d == 1) return ksgn32(ky) * Gt[(ay * kGreenS + ax) * kGreenS + az];
    return ksgn32(kz) * Gt[(az * kGreenS + ay) * kGreenS + ax];
}

// --- phase 5a: Green multiply (Eq. 1) and inverse transform along z -------
// For kx = 1..15: G = rho~ K~_d = -i S rho~.  For the packed kx = 0 pencil,
// Z = A + iB holds the kx = 0 (A) and kx = 16 (B) planes; with the partner
// Z' = Z(-ky, -kz): A = (Z + conj Z')/2, B = (Z - conj Z')/(2i), and the packed
// product A K~_d(0) + i B K~_d(16) = -i[(s0+s16)/2 Z + (s0-s16)/2 conj Z'].
PMPM_HD void tile_inv_z(int tid, int d, const TileGeom& g, const float* Gt, const float2* C,
                        float2* W) {
    const int kx = tid & 15, ky = tid >> 4;
    float2 a[32];
#pragma unroll
    for (int kz = 0; kz < 32; ++kz) {
        const float2 Z = C[cidx(kx, ky, kz)];
        float cA, cB;
        float2 Zp = make_float2(0.f, 0.f);
        if (kx != 0) {
            cA = green_S(Gt, d, kx, ky, kz);
            cB = 0.f;
        } else {
            const float s0 = green_S(Gt, d, 0, ky, kz);
            const float s16 = green_S(Gt, d, 16, ky, kz);
            cA = 0.5f * (s0 + s16);
            cB = 0.5f * (s0 - s16);
            Zp = C[cidx(0, (32 - ky) & 31, (32 - kz) & 31)];
        }
        // V = cA Z + cB conj(Zp);  G = -i V
        const float vx = cA * Z.x + cB * Zp.x;
        const float vy = cA * Z.y - cB * Zp.y;
        a[kz] = make_float2(vy, -vx);
    }
    fft_bitrev_out<32, 1>(a);
    const int nz = g.T[2] + 2;
#pragma unroll
    for (int zo = 0; zo < kTileOut; ++zo)
        if (zo < nz) W[widx(kx, ky, zo)] = a[bitrev<5>(zo + kBuffer - 1)];
}

// --- phase 5b: inverse transform along y, pruned to T + 2 output rows -----
PMPM_HD void tile_inv_y(int tid, const TileGeom& g, float2* W) {
    const int nz = g.T[2] + 2, ny = g.T[1] + 2;
    if (tid >= 16 * nz) return;
    const int kx = tid & 15, zo = tid >> 4;
    float2 a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = W[widx(kx, k, zo)];
    fft_bitrev_out<32, 1>(a);
#pragma unroll
    for (int yo = 0; yo < kTileOut; ++yo)
        if (yo < ny) W[widx(kx, yo, zo)] = a[bitrev<5>(yo + kBuffer - 1)];
}

// --- phase 5c: inverse real transform along x, pruned to T + 2 columns ----
PMPM_HD void tile_inv_x(int tid, const TileGeom& g, float2* W) {
    const int ny = g.T[1] + 2, nz = g.T[2] + 2, nx = g.T[0] + 2;
    float* Wf = reinterpret_cast<float*>(W);
    for (int r = tid; r < ny * nz; r += kTileThreads) {
        const int yo = r % ny, zo = r / ny;
        float2 X[17];
        const float2 p0 = W[widx(0, yo, zo)];
        X[0] = make_float2(p0.x, 0.f);
        X[16] = make_float2(p0.y, 0.f);
#pragma unroll
        for (int k = 1; k < 16; ++k) X[k] = W[widx(k, yo, zo)];
        float x[32];
        irfft32(X, x);
#pragma unroll
        for (int xo = 0; xo < kTileOut; ++xo)
            if (xo < nx) Wf[wfidx(xo, yo, zo)] = x[xo + kBuffer - 1];
    }
}

// --- phase 5d: interpolate component d to the tile's own particles, then
// (mode 1) kick and drift that component; after the last component, update
// the new-cell counts and fixed-point momentum sums.
PMPM_HD void tile_interp(int tid, int d, const TileGeom& g, const TileParams& P, const float2* W) {
    const float* Wf = reinterpret_cast<const float*>(W);
    const int warp = tid >> 5, lane = tid & 31;
    const int nx = g.c1[0] - g.c0[0], ny = g.c1[1] - g.c0[1], nz = g.c1[2] - g.c0[2];
    const int64_t ncells = (int64_t)P.nc * P.nc * P.nc;
    const int64_t n = P.n;
    const float sigma = *P.sigma;
    const uint8_t* ud = d == 0 ? P.u0 : (d == 1 ? P.u1 : P.u2);
    const float* Fl = P.Fl + d * ncells;
    for (int r = warp; r < ny * nz; r += kTileThreads / 32) {
        const int y = g.c0[1] + r % ny, z = g.c0[2] + r / ny;
        const int base = P.nc * (y + P.nc * z);
        RowCells rc;
        row_cells(rc, P, base, g.c0[0], nx);
        const int total = rc.pc[9];
        for (int v = lane; v < total; v += 32) {
            const int i = row_find(rc, v);
            const int64_t j = rc.st[i] + (v - rc.pc[i]);
            const int cell = base + g.c0[0] + i;
            const int64_t Q[3] = {(int64_t)(g.c0[0] + i) * kBins + P.m0[j],
                                  (int64_t)y * kBins + P.m1[j], (int64_t)z * kBins + P.m2[j]};
            // fine gather
            int lo[3], w1[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                int s = (int)(2 * Q[e] + 1 - kCodesPerFine - 128 * (int64_t)g.o[e]);
                lo[e] = (s >> 7) - (kBuffer - 1);
                w1[e] = s & 127;
            }
            float gf = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
                const float w = (float)((dx ? w1[0] : 128 - w1[0]) * (dy ? w1[1] : 128 - w1[1]) *
                                        (dz ? w1[2] : 128 - w1[2]));
                gf += w * Wf[wfidx(lo[0] + dx, lo[1] + dy, lo[2] + dz)];
            }
            // coarse gather
            Cic1 cc[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) cc[e] = cic_coarse(Q[e]);
            float gc = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
                const int ix = wrap(cc[0].i0 + dx, P.nc), iy = wrap(cc[1].i0 + dy, P.nc),
                          iz = wrap(cc[2].i0 + dz, P.nc);
                const float w = (float)((dx ? cc[0].w1 : 512 - cc[0].w1) *
                                        (dy ? cc[1].w1 : 512 - cc[1].w1)) *
                                (float)(dz ? cc[2].w1 : 512 - cc[2].w1);
                gc += w * Fl[(int64_t)ix + P.nc * ((int64_t)iy + (int64_t)P.nc * iz)];
            }
            const float gval = gf * 4.76837158203125e-07f      // 2^-21
                             + gc * 7.450580596923828e-09f;    // 2^-27
            if (P.mode == 0) {
                P.G[d * n + j] = gval;
                continue;
            }
            // kick (Eq. 3 decode, then p += kick * g) and integer drift
            const float p = decode_momentum(P.vc[d * ncells + cell], sigma, P.Tdec[ud[j]]);
            const float pn = fadd_rn(p, fmul_rn(P.kick, gval));
            if (!(pn == pn) || !(gval == gval)) flag_error(P.err, kErrNaN);
            if (fabsf(pn) >= 1048576.f) flag_error(P.err, kErrMomentum);
            const float xq = fmul_rn(pn, P.drift);
            if (!(fabsf(xq) < 1.0e9f)) flag_error(P.err, kErrDrift);
            const int64_t dq = (int64_t)floorf(fadd_rn(xq, 0.5f));
            const int64_t M = (int64_t)P.nc * kBins;
            int64_t qn = (Q[d] + dq) % M;
            if (qn < 0) qn += M;
            P.Qn[d * n + j] = (int32_t)qn;
            P.Pn[d * n + j] = pn;
            if (d == 2) {
                const int32_t q0 = P.Qn[j], q1 = P.Qn[n + j];
                const int64_t key = (int64_t)(q0 >> 8) +
                                    P.nc * ((int64_t)(q1 >> 8) + (int64_t)P.nc * (qn >> 8));
                gmem_add_i32(&P.counts_new[key], 1);
                const float pp[3] = {P.Pn[j], P.Pn[n + j], pn};
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const long long fx = f64_to_ll_rn((double)pp[e] * 16777216.0);
                    gmem_add_u64(&P.S_new[e * ncells + key], (unsigned long long)fx);
                }
            }
        }
    }
}

}  // namespace pmpm
