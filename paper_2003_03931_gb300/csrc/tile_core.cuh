// tile_core.cuh -- the fine-mesh (short-range) PM of one tile, Sec. II:
// each tile's short-range force comes from a fine-mesh PM over the tile
// grown by the cutoff radius on every side.  One CTA of 512 threads owns one
// tile.
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
//      particle), then twice its 3-D spectrum packed as 16 x 32 x 32 complex with
//      the kx = 16 (Nyquist) plane folded into the imaginary part of kx = 0;
//   W  22 x 32 x 16 complex = 88 KB: one force component on its way back,
//      pruned to the 22 output planes that are needed (during the deposit it
//      holds the table of the halo box's cells and the coarse force on the
//      7^3 coarse nodes around the tile);
//   G  the short-range Green table, 15 x 153 floats (9 KB): S(a, b, c) is
//      symmetric in (b, c), so only b <= c is kept, and it vanishes for own-
//      axis |k| = 0 and 16, so those rows are not stored;
//   O  the tile's own-cell table (prefix counts and storage offsets), built
//      during the deposit and used by every interpolation phase, a few
//      per-tile scalars, and the velocity decode table T of Eq. 3 (2 KB).
// Index swizzles (x ^ y) make every pencil pass free of bank conflicts.  The
// data-dependent accesses are not: the deposit's atomics and the force
// gathers at particle positions meet about 3 extra wavefronts per warp access
// (32 random addresses would meet 2.5), and the Green-table reads of the
// inverse z passes fewer; together they account for the conflicts a profile
// of the tile pass counts.  The transforms are the register FFTs of
// regfft.cuh (decimation in time with fused multiply-add butterflies).
//
// Each phase is a per-thread function; the kernel calls them with a block
// barrier between phases.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "regfft.cuh"

namespace pmpm {

constexpr int kTileThreads = 512;
constexpr int kTileR = kTileFFT * kTileFFT * kTileFFT;          // 32768 words
constexpr int kTileW = kTileOut * kTileFFT * (kTileFFT / 2);    // 11264 complex
constexpr int kGreenTri = kGreenS * (kGreenS + 1) / 2;          // 153 pairs b <= c
constexpr int kGreenRows = kGreenS - 2;                         // own-axis |k| = 1..15
constexpr int kGreenPacked = kGreenRows * kGreenTri;            // 2295 floats
constexpr int kOwnTail = 126 + 125 + 8;                         // own-cell table, ints
constexpr size_t kTileSmemBytes = (size_t)kTileR * 4 + (size_t)kTileW * 8 +
                                  (size_t)kGreenPacked * 4 + (size_t)kOwnTail * 4 + 256 * 4;

struct TileParams {
    int nc;                       // coarse cells per side
    int nt;                       // tiles per side
    int64_t n;                    // particles
    const int32_t* counts;        // [nc^3]
    const int64_t* offsets;       // [nc^3 + 1]
    const uint8_t* m0;            // position bins (Eq. 2; 1 or 2 bytes each), storage order
    const uint8_t* m1;
    const uint8_t* m2;
    const uint8_t* u0;            // velocity bins (Eq. 3)
    const uint8_t* u1;
    const uint8_t* u2;
    const float* vc;              // [3][nc^3]
    const float* sigma;           // device scalar
    const float* Tdec;            // [256] decode table
    const float* green;           // packed short-range Green table, 17 x 153 (scaled)
    const float* Fl;              // [3][nc^3] long-range force on the coarse mesh
    int mode;                     // 0: write g; 1: kick + drift
    const float* kd;              // [2] of the current step: fl32 kick factor (multiplies g)
                                  // and drift factor in position codes (multiplies p)
    float* G;                     // [3][N] (mode 0)
    int32_t* Qn;                  // [3][N] new codes (mode 1; null in the low-memory step,
                                  // whose re-encode derives them from the old store and Pn)
    float* Pn;                    // [3][N] new momenta (mode 1)
    uint32_t* err;
    // mode 1 with counts_new: the last interpolation also adds each particle
    // to its new cell's count, momentum sums and the second moment
    int32_t* counts_new;          // [nc^3]
    unsigned long long* S;        // [3][nc^3] momentum sums in units of 2^-24
    unsigned long long* d2;       // [4] digits of T = sum P^2 of the new momenta
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
// the float view of widx: word xo of the pair (xo >> 1) ^ (yo & 15), i.e.
// xo ^ 2 (yo & 15) (an even XOR keeps the low bit)
PMPM_HD int wfidx(int xo, int yo, int zo) { return ((zo << 5) + yo) * 32 + (xo ^ ((yo & 15) << 1)); }

// The tile spectrum C is stored as float2 (the default) or, with the FP16
// storage option, as __half2 at the same index (half the bytes; every
// transform still computes in float32 registers).
PMPM_HD float2 cload(const float2* C, int i) { return C[i]; }
PMPM_HD void cstore(float2* C, int i, float2 v) { C[i] = v; }
#ifdef __CUDA_ARCH__
__device__ __forceinline__ float2 cload(const __half2* C, int i) { return __half22float2(C[i]); }
__device__ __forceinline__ void cstore(__half2* C, int i, float2 v) { C[i] = __float22half2_rn(v); }
#endif

#ifdef __CUDA_ARCH__
PMPM_HD uint32_t smem_add_u32(uint32_t* p, uint32_t v) { return atomicAdd(p, v); }
PMPM_HD void gmem_add_i32(int32_t* p, int32_t v) { atomicAdd(p, v); }
PMPM_HD void gmem_add_u64(unsigned long long* p, unsigned long long v) { atomicAdd(p, v); }
PMPM_HD float u32_to_f32(uint32_t v) { return __uint2float_rn(v); }
#else
PMPM_HD uint32_t smem_add_u32(uint32_t* p, uint32_t v) { uint32_t o = *p; *p = o + v; return o; }
PMPM_HD void gmem_add_i32(int32_t* p, int32_t v) { *p += v; }
PMPM_HD void gmem_add_u64(unsigned long long* p, unsigned long long v) { *p += v; }
PMPM_HD float u32_to_f32(uint32_t v) { return (float)v; }
#endif

// --- phase 0: clear the density --------------------------------------------
PMPM_HD void tile_zero(int tid, uint32_t* R) {
    uint4* R4 = reinterpret_cast<uint4*>(R);
    for (int i = tid; i < kTileR / 4; i += kTileThreads) R4[i] = make_uint4(0u, 0u, 0u, 0u);
}

// shared-memory add without a returned value
PMPM_HD void smem_red_u32(uint32_t* p, uint32_t v) {
#ifdef __CUDA_ARCH__
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v)
                 : "memory");
#else
    *p += v;
#endif
}

// CIC of one particle (unwrapped coarse cell cu, bins m) into the tile box.
// A node gathers from the particles of at most 8 coarse cells, each weighing
// at most 2^21; with at most 255 particles per cell no node can pass 2^32, so
// CHECK (overflow detection on the returned old value) is needed only when
// some halo cell holds more.
template <bool CHECK, int PB>
PMPM_HD void deposit_one(const TileGeom& g, const int (&cu)[3], const int (&m)[3], uint32_t* R,
                         uint32_t* err) {
    using F = PosFmt<PB>;
    constexpr int W = F::kFineW;
    int li[3], w1[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // s = 2Q + 1 - B/4 relative to the mesh origin, units 1/W (W = B/2)
        const int s = 2 * (cu[d] * F::kBins + m[d]) + 1 - F::kCodesPerFine - W * g.o[d];
        li[d] = s >> F::kFineWBits;
        w1[d] = s & (W - 1);
    }
    // a cloud whose lower node is below -1 or above 31 on some axis misses the box
    if ((unsigned)(li[0] + 1) > 32u || (unsigned)(li[1] + 1) > 32u || (unsigned)(li[2] + 1) > 32u) return;
    const bool inside = (unsigned)li[0] < 31u && (unsigned)li[1] < 31u && (unsigned)li[2] < 31u;
    const uint32_t wyz[4] = {(uint32_t)((W - w1[1]) * (W - w1[2])), (uint32_t)(w1[1] * (W - w1[2])),
                             (uint32_t)((W - w1[1]) * w1[2]), (uint32_t)(w1[1] * w1[2])};
    if (!CHECK && inside) {
        // the common case, all eight nodes in the box: straight-line adds
        // (a zero weight adds nothing)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
            const uint32_t w = PB == 1 ? (uint32_t)(dx ? w1[0] : W - w1[0]) * wyz[dy + 2 * dz]
                                       : cic_weight3<PB>(dx ? w1[0] : W - w1[0], dy ? w1[1] : W - w1[1],
                                                         dz ? w1[2] : W - w1[2]);
            smem_red_u32(&R[ridx(li[0] + dx, li[1] + dy, li[2] + dz)], w);
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        const int x = li[0] + dx, y = li[1] + dy, z = li[2] + dz;
        if (!inside && ((unsigned)x >= 32u || (unsigned)y >= 32u || (unsigned)z >= 32u)) continue;
        // 1-byte: exact in 2^-21; 2-byte: the 2^-45 product rounded to 2^-21
        const uint32_t w = PB == 1 ? (uint32_t)(dx ? w1[0] : W - w1[0]) * wyz[dy + 2 * dz]
                                   : cic_weight3<PB>(dx ? w1[0] : W - w1[0], dy ? w1[1] : W - w1[1],
                                                     dz ? w1[2] : W - w1[2]);
        if (w == 0u) continue;
        if (CHECK) {
            const uint32_t old = smem_add_u32(&R[ridx(x, y, z)], w);
            if (old + w < old) flag_error(err, kErrFineOverflow);
        } else {
            smem_red_u32(&R[ridx(x, y, z)], w);
        }
    }
}

// --- phase 1: integer CIC of the tile and its 2-coarse-cell halo ------------
// Particles in coarse cells [c0 - 2, c1 + 2) can reach the mesh nodes
// [-6, T + 5]; their contributions outside the 32^3 box are clipped.
// 1a: table of the halo box's cells (storage offset, count) in the free W
//     area; 1b: exclusive prefix sums over the box cells and over the tile's
//     own cells; 1c: every thread takes particles by flattened index, so the
//     work is balanced however the particles cluster, and consecutive threads
//     read consecutive particles.  1c also gathers the long-range force of
//     the tile's own particles (it needs only F_l) and parks it in their
//     output slots, where the component phases pick it up.
// The halo box is laid out as 9 x 9 x 9 cells and the tile's own cells as
// 5 x 5 x 5 whatever the tile size (cells outside a smaller tile's box count
// as empty), so cell coordinates follow from divisions by constants.
constexpr int kHaloDim = kTileMaxCoarse + 4;                  // 9
constexpr int kHaloMax = kHaloDim * kHaloDim * kHaloDim;       // 729
constexpr int kOwnDim = kTileMaxCoarse;                       // 5
constexpr int kOwnMax = kOwnDim * kOwnDim * kOwnDim;           // 125
// The long-range force on the 7^3 coarse nodes the tile's own particles
// gather from (own cells [c0, c1) reach nodes [c0 - 1, c1]) is staged in
// shared memory by the prologue, behind the map, which gives up that room.
constexpr int kFlWin = kTileMaxCoarse + 2;                           // 7
constexpr int kFlWinNodes = kFlWin * kFlWin * kFlWin;                // 343
constexpr int kFlWinEntries = (3 * kFlWinNodes * 4 + 15) / 16 * 8;   // in map entries (4128 B)
constexpr int kMapCap = 32768 - kFlWinEntries;   // particles whose cell is looked up by table
constexpr int kPMapCap = 8192;
constexpr int kHaloChunks = (kHaloMax + 31) / 32;               // 23

struct TileCells {
    int64_t* st;       // [kHaloMax] storage offset of each halo-box cell (W)
    int* cnt;          // [kHaloMax] particles in it (W)
    int* pre;          // [kHaloMax + 1] exclusive prefix over the box cells (W)
    uint16_t* map;     // [kMapCap] halo cell of the v-th box particle (W)
    uint8_t* pmap;     // [kPMapCap] own cell of the v-th own particle (W)
    int* ppre;         // [kOwnMax + 1] exclusive prefix over the tile's own cells (O)
    int* prel;         // [kOwnMax] storage offset of own cell p minus own_base (O)
    int* misc;         // [0..1] own_base (int64), [2] largest halo-cell count,
                       // [4] sigma, [5] kick, [6] drift, [7] new sigma as float bits (O)
    float* Td;         // [256] velocity decode table T of Eq. 3 (after O)
    int* tot;          // [kHaloChunks] particles per 32-cell chunk of the halo box (W)
    int* cmax;         // [kHaloChunks] largest cell count per chunk (W)
};

PMPM_HD TileCells tile_cells(float2* W, int* O) {
    TileCells c;
    c.st = reinterpret_cast<int64_t*>(W);
    c.cnt = reinterpret_cast<int*>(c.st + kHaloMax);
    c.pre = c.cnt + kHaloMax;
    c.map = reinterpret_cast<uint16_t*>(c.pre + kHaloMax + 1 + 1);
    c.pmap = reinterpret_cast<uint8_t*>(c.map + kMapCap + kFlWinEntries);
    c.ppre = O;
    c.prel = O + 126;
    c.misc = O + 126 + 125;
    c.Td = reinterpret_cast<float*>(O + kOwnTail);
    c.tot = reinterpret_cast<int*>(c.pmap + kPMapCap);
    c.cmax = c.tot + 32;
    return c;
}
static_assert(kHaloMax * 8 + (2 * kHaloMax + 2) * 4 + (kMapCap + kFlWinEntries) * 2 + kPMapCap + 64 * 4 <=
                  kTileW * 8,
              "tile cell tables must fit in W");

// the staged F_l window, [3][kFlWin^3], x fastest (derived, holds no register)
PMPM_HD float* fl_window(const TileCells& c) { return reinterpret_cast<float*>(c.map + kMapCap); }

// Coarse-mesh force (all three components) at one of the tile's own
// particles from the staged window: the same nodes, weights and order of
// accumulation as a gather from global memory
template <int PB>
PMPM_HD void coarse_gather_win(const float* flw, const TileGeom& g, const int (&Q)[3], float (&gc)[3]) {
    using F = PosFmt<PB>;
    constexpr int W = F::kCoarseW;
    Cic1 cc[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int sc = 2 * Q[e] + 1 - F::kBins;     // units 1/(2B) of a coarse cell (< 2^28)
        cc[e].i0 = (int)(sc >> F::kCoarseWBits) - (g.c0[e] - 1);   // window node, 0..5
        cc[e].w1 = (int)(sc & (W - 1));
    }
    gc[0] = gc[1] = gc[2] = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        const int node = (cc[0].i0 + dx) + kFlWin * ((cc[1].i0 + dy) + kFlWin * (cc[2].i0 + dz));
        const float w = PB == 1
            ? (float)((dx ? cc[0].w1 : W - cc[0].w1) * (dy ? cc[1].w1 : W - cc[1].w1)) *
                  (float)(dz ? cc[2].w1 : W - cc[2].w1)
            : (float)cic_weight3<PB>(dx ? cc[0].w1 : W - cc[0].w1, dy ? cc[1].w1 : W - cc[1].w1,
                                     dz ? cc[2].w1 : W - cc[2].w1);
#pragma unroll
        for (int e = 0; e < 3; ++e) gc[e] += w * flw[e * kFlWinNodes + node];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) gc[e] *= 7.450580596923828e-09f;   // 2^-27
}
static_assert(kHaloChunks <= 32, "one lane per halo chunk");

PMPM_HD float bits_to_f32(int v) {
    union { int i; float f; } u;
    u.i = v;
    return u.f;
}
PMPM_HD int f32_to_bits(float v) {
    union { int i; float f; } u;
    u.f = v;
    return u.i;
}
PMPM_HD int64_t own_base(const TileCells& c) {
    return (int64_t)(((uint64_t)(uint32_t)c.misc[1] << 32) | (uint32_t)c.misc[0]);
}

// own cell p lies inside the tile (tiles of 4 coarse cells leave the fifth
// row, column and plane of the 5^3 layout empty)
PMPM_HD bool own_valid(const TileGeom& g, int p) {
    return p % kOwnDim < g.c1[0] - g.c0[0] && (p / kOwnDim) % kOwnDim < g.c1[1] - g.c0[1] &&
           p / (kOwnDim * kOwnDim) < g.c1[2] - g.c0[2];
}

PMPM_HD int own_to_halo(int p) {
    return (2 + p % kOwnDim) + kHaloDim * ((2 + (p / kOwnDim) % kOwnDim) + kHaloDim * (2 + p / (kOwnDim * kOwnDim)));
}

// 1a: every global load of the prologue (the halo cells' offsets and counts,
// the packed Green table, sigma and the step factors) is issued before the
// first shared-memory store, so the tile waits for one memory round trip.
PMPM_HD void tile_prologue(int tid, const TileGeom& g, const TileParams& P, TileCells c,
                           uint32_t* R, float* gS) {
    const int hx = g.c1[0] - g.c0[0] + 4, hy = g.c1[1] - g.c0[1] + 4, hz = g.c1[2] - g.c0[2] + 4;
    int64_t st[2] = {0, 0};
    int cnt[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int b = tid + u * kTileThreads;
        const int bx = b % kHaloDim, by = (b / kHaloDim) % kHaloDim, bz = b / (kHaloDim * kHaloDim);
        if (b < kHaloMax && bx < hx && by < hy && bz < hz) {
            const int cx = wrap1(g.c0[0] - 2 + bx, P.nc), cy = wrap1(g.c0[1] - 2 + by, P.nc),
                      cz = wrap1(g.c0[2] - 2 + bz, P.nc);
            const int64_t cell = cx + (int64_t)P.nc * (cy + (int64_t)P.nc * cz);
            st[u] = P.offsets[cell];
            cnt[u] = P.counts[cell];
        }
    }
    // the F_l window (three values per thread at most)
    constexpr int kWinPer = (3 * kFlWinNodes + kTileThreads - 1) / kTileThreads;
    float fw[kWinPer];
    {
        const int64_t ncells = (int64_t)P.nc * P.nc * P.nc;
#pragma unroll
        for (int k = 0; k < kWinPer; ++k) {
            const int i = tid + k * kTileThreads;
            fw[k] = 0.f;
            if (i < 3 * kFlWinNodes) {
                const int e = i / kFlWinNodes, w = i % kFlWinNodes;
                const int x = wrap1(g.c0[0] - 1 + w % kFlWin, P.nc);
                const int y = wrap1(g.c0[1] - 1 + (w / kFlWin) % kFlWin, P.nc);
                const int z = wrap1(g.c0[2] - 1 + w / (kFlWin * kFlWin), P.nc);
                fw[k] = P.Fl[e * ncells + x + P.nc * (y + P.nc * z)];
            }
        }
    }
    float gv[(kGreenPacked + kTileThreads - 1) / kTileThreads];
#pragma unroll
    for (int u = 0; u < (kGreenPacked + kTileThreads - 1) / kTileThreads; ++u) {
        const int i = tid + u * kTileThreads;
        gv[u] = i < kGreenPacked ? P.green[i] : 0.f;
    }
    const float td = tid < 256 ? P.Tdec[tid] : 0.f;
    float sc[3] = {0.f, 0.f, 0.f};
    if (tid == 0) {
        sc[0] = *P.sigma;
        if (P.mode >= 1) {
            sc[1] = P.kd[0];
            sc[2] = P.kd[1];
        }
    }
    tile_zero(tid, R);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int b = tid + u * kTileThreads;
        if (b < kHaloMax) {
            c.st[b] = st[u];
            c.cnt[b] = cnt[u];
        }
    }
#pragma unroll
    for (int u = 0; u < (kGreenPacked + kTileThreads - 1) / kTileThreads; ++u) {
        const int i = tid + u * kTileThreads;
        if (i < kGreenPacked) gS[i] = gv[u];
    }
    if (tid < 256) c.Td[tid] = td;
    float* flw = fl_window(c);
#pragma unroll
    for (int k = 0; k < kWinPer; ++k) {
        const int i = tid + k * kTileThreads;
        if (i < 3 * kFlWinNodes) flw[i] = fw[k];
    }
    if (tid == 0) {
        c.misc[4] = f32_to_bits(sc[0]);
        c.misc[5] = f32_to_bits(sc[1]);
        c.misc[6] = f32_to_bits(sc[2]);
    }
}

// Exclusive prefix of n counts produced by cnt_of(i), written to out[0..n].
template <typename F>
PMPM_HD void warp_prefix(int lane, int n, F cnt_of, int* out) {
#ifdef __CUDA_ARCH__
    int carry = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const int v = i < n ? cnt_of(i) : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (i < n) out[i] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) out[n] = carry;
#else
    if (lane != 0) return;
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        out[i] = acc;
        acc += cnt_of(i);
    }
    out[n] = acc;
#endif
}

// 1b: exclusive prefix over the halo box's cells in 32-cell chunks, one warp
// per chunk (chunk-local prefix, chunk total and largest count); the last
// two warps also build the own-cell prefix and the own cells' offsets.
PMPM_HD void tile_cells_scan(int tid, const TileGeom& g, TileCells c) {
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int kWarps = kTileThreads / 32;
#ifdef __CUDA_ARCH__
    for (int ch = warp; ch < kHaloChunks; ch += kWarps) {
        const int i = ch * 32 + lane;
        const int v = i < kHaloMax ? c.cnt[i] : 0;
        int incl = v, mx = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (i < kHaloMax) c.pre[i] = incl - v;
        if (lane == 31) c.tot[ch] = incl;
        if (lane == 0) c.cmax[ch] = mx;
    }
#else
    if (lane == 0) {
        for (int ch = warp; ch < kHaloChunks; ch += kWarps) {
            int acc = 0, mx = 0;
            for (int l = 0; l < 32; ++l) {
                const int i = ch * 32 + l;
                const int v = i < kHaloMax ? c.cnt[i] : 0;
                if (i < kHaloMax) c.pre[i] = acc;
                acc += v;
                mx = v > mx ? v : mx;
            }
            c.tot[ch] = acc;
            c.cmax[ch] = mx;
        }
    }
#endif
    const int* cnt = c.cnt;
    if (warp == kWarps - 1) {
        const TileGeom gg = g;
        warp_prefix(lane, kOwnMax,
                    [cnt, gg](int p) { return own_valid(gg, p) ? cnt[own_to_halo(p)] : 0; }, c.ppre);
    } else if (warp == kWarps - 2) {
        // storage offsets of the own cells relative to own cell 0 (increasing
        // in flat cell order, spanning less than 2^31 particles)
        const int64_t base = c.st[own_to_halo(0)];
        for (int p = lane; p < kOwnMax; p += 32)
            c.prel[p] = own_valid(g, p) ? (int)(c.st[own_to_halo(p)] - base) : 0;
        if (lane == 0) {
            c.misc[0] = (int)(uint32_t)((uint64_t)base & 0xffffffffu);
            c.misc[1] = (int)(uint32_t)((uint64_t)base >> 32);
        }
    }
}

// 1c: the chunk bases turn the chunk-local prefix into the box prefix, and
// the particle -> cell maps (first kMapCap / kPMapCap particles) are filled:
// each warp takes 32 cells at a time, one per lane; a lane writes its own
// cell when it holds at most kMapLane particles, and the whole warp writes
// each larger cell in turn, so a crowded cell is shared by 32 lanes.
constexpr int kMapLane = 16;
PMPM_HD void tile_cells_map(int tid, const TileGeom& g, TileCells c) {
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int kWarps = kTileThreads / 32;
    constexpr int kOwnGroups = (kOwnMax + 31) / 32;
#ifdef __CUDA_ARCH__
    const int t = lane < kHaloChunks ? c.tot[lane] : 0;
    int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int base = incl - t;
    if (warp == 0) {
        int mx = lane < kHaloChunks ? c.cmax[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 31) c.pre[kHaloMax] = incl;
        if (lane == 0) c.misc[2] = mx;
    }
    for (int b0 = warp * 32; b0 < kHaloMax; b0 += kTileThreads) {
        const int b = b0 + lane;
        const int n = b < kHaloMax ? c.cnt[b] : 0;
        const int p = (b < kHaloMax ? c.pre[b] : 0) + __shfl_sync(0xffffffffu, base, b0 >> 5);
        if (b < kHaloMax) c.pre[b] = p;
        if (n <= kMapLane)
            for (int q = 0; q < n && p + q < kMapCap; ++q) c.map[p + q] = (uint16_t)b;
        unsigned live = __ballot_sync(0xffffffffu, n > kMapLane && p < kMapCap);
        while (live) {
            const int src = __ffs(live) - 1;
            live &= live - 1u;
            const int nn = __shfl_sync(0xffffffffu, n, src), pp = __shfl_sync(0xffffffffu, p, src);
            for (int q = lane; q < nn && pp + q < kMapCap; q += 32) c.map[pp + q] = (uint16_t)(b0 + src);
        }
    }
    if (warp >= kWarps - kOwnGroups) {
        const int p0 = (warp - (kWarps - kOwnGroups)) * 32, p = p0 + lane;
        const int n = (p < kOwnMax && own_valid(g, p)) ? c.cnt[own_to_halo(p)] : 0;
        const int pp = p < kOwnMax ? c.ppre[p] : 0;
        if (n <= kMapLane)
            for (int q = 0; q < n && pp + q < kPMapCap; ++q) c.pmap[pp + q] = (uint8_t)p;
        unsigned live = __ballot_sync(0xffffffffu, n > kMapLane && pp < kPMapCap);
        while (live) {
            const int src = __ffs(live) - 1;
            live &= live - 1u;
            const int nn = __shfl_sync(0xffffffffu, n, src), q0 = __shfl_sync(0xffffffffu, pp, src);
            for (int q = lane; q < nn && q0 + q < kPMapCap; q += 32) c.pmap[q0 + q] = (uint8_t)(p0 + src);
        }
    }
#else
    if (lane != 0) return;
    int base[32], acc = 0, mx = 0;
    for (int l = 0; l < 32; ++l) {
        base[l] = acc;
        acc += l < kHaloChunks ? c.tot[l] : 0;
        if (l < kHaloChunks && c.cmax[l] > mx) mx = c.cmax[l];
    }
    if (warp == 0) {
        c.pre[kHaloMax] = acc;
        c.misc[2] = mx;
    }
    for (int b0 = warp * 32; b0 < kHaloMax; b0 += kTileThreads)
        for (int b = b0; b < b0 + 32 && b < kHaloMax; ++b) {
            const int n = c.cnt[b], p = c.pre[b] + base[b0 >> 5];
            c.pre[b] = p;
            for (int q = 0; q < n && p + q < kMapCap; ++q) c.map[p + q] = (uint16_t)b;
        }
    if (warp >= kWarps - kOwnGroups) {
        const int p0 = (warp - (kWarps - kOwnGroups)) * 32;
        for (int p = p0; p < p0 + 32 && p < kOwnMax; ++p) {
            const int n = own_valid(g, p) ? c.cnt[own_to_halo(p)] : 0, q0 = c.ppre[p];
            for (int q = 0; q < n && q0 + q < kPMapCap; ++q) c.pmap[q0 + q] = (uint8_t)p;
        }
    }
#endif
}

// largest i in [0, N) with pre[i] <= v (pre non-decreasing, pre[0] = 0 <= v):
// a fixed number of halving steps with no branch, so that searches of
// several particles interleave
template <int N>
PMPM_HD int prefix_find(const int* pre, int v) {
    int pos = 0;
#pragma unroll
    for (int step = 1 << 10; step > 0; step >>= 1) {
        if (step >= N) continue;
        const int t = pos + step;
        pos = (t < N && pre[t < N ? t : 0] <= v) ? t : pos;
    }
    return pos;
}

// the same search as a loop (compact code for the rare lookups past the maps)
PMPM_HD int prefix_find_loop(const int* pre, int n, int v) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

PMPM_HD int halo_of(const TileCells& c, int v) {
    return v < kMapCap ? (int)c.map[v] : prefix_find_loop(c.pre, kHaloMax, v);
}
PMPM_HD int own_of(const TileCells& c, int v) {
    return v < kPMapCap ? (int)c.pmap[v] : prefix_find_loop(c.ppre, kOwnMax, v);
}

constexpr int kDepositIlp = 4;   // halo particles per thread per iteration
constexpr int kGatherIlp = 2;    // own particles per thread per iteration

// the integer CIC of the halo box's particles into R
template <int PB>
PMPM_HD void tile_deposit_halo(int tid, const TileGeom& g, const TileParams& P, uint32_t* R,
                               TileCells c) {
    const int total = c.pre[kHaloMax];
    const bool check = c.misc[2] > 255;
    for (int v0 = tid; v0 < total; v0 += kDepositIlp * kTileThreads) {
        int b[kDepositIlp], m[kDepositIlp][3];
        bool ok[kDepositIlp];
#pragma unroll
        for (int u = 0; u < kDepositIlp; ++u) {
            const int v = v0 + u * kTileThreads;
            ok[u] = v < total;
            b[u] = ok[u] ? halo_of(c, v) : 0;
            const int64_t j = c.st[b[u]] + (v - c.pre[b[u]]);
            if (ok[u]) {
                m[u][0] = load_bin<PB>(P.m0, j);
                m[u][1] = load_bin<PB>(P.m1, j);
                m[u][2] = load_bin<PB>(P.m2, j);
            }
        }
#pragma unroll
        for (int u = 0; u < kDepositIlp; ++u) {
            if (!ok[u]) continue;
            const int cu[3] = {g.c0[0] - 2 + b[u] % kHaloDim, g.c0[1] - 2 + (b[u] / kHaloDim) % kHaloDim,
                               g.c0[2] - 2 + b[u] / (kHaloDim * kHaloDim)};
            if (check) deposit_one<true, PB>(g, cu, m[u], R, P.err);
            else deposit_one<false, PB>(g, cu, m[u], R, P.err);
        }
    }
}

// the long-range force of the tile's own particles, parked in their output
// slots
template <int PB>
PMPM_HD void tile_gather_coarse(int tid, const TileGeom& g, const TileParams& P, TileCells c) {
    float* slot = P.mode == 0 ? P.G : P.Pn;
    const int ptotal = c.ppre[kOwnMax];
    const int64_t obase = own_base(c);
    for (int v0 = tid; v0 < ptotal; v0 += kGatherIlp * kTileThreads) {
        int64_t j[kGatherIlp];
        int Q[kGatherIlp][3];   // codes, below nc 65536 <= 2^26
#pragma unroll
        for (int u = 0; u < kGatherIlp; ++u) {
            const int v = v0 + u * kTileThreads;
            const int p = v < ptotal ? own_of(c, v) : 0;
            j[u] = v < ptotal ? obase + c.prel[p] + (v - c.ppre[p]) : -1;
            if (j[u] >= 0) {
                constexpr int B = PosFmt<PB>::kBins;
                Q[u][0] = (g.c0[0] + p % kOwnDim) * B + load_bin<PB>(P.m0, j[u]);
                Q[u][1] = (g.c0[1] + (p / kOwnDim) % kOwnDim) * B + load_bin<PB>(P.m1, j[u]);
                Q[u][2] = (g.c0[2] + p / (kOwnDim * kOwnDim)) * B + load_bin<PB>(P.m2, j[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kGatherIlp; ++u) {
            if (j[u] < 0) continue;
            float gc[3];
            coarse_gather_win<PB>(fl_window(c), g, Q[u], gc);
#pragma unroll
            for (int e = 0; e < 3; ++e) slot[e * P.n + j[u]] = gc[e];
        }
    }
}

template <int PB>
PMPM_HD void tile_deposit_flat(int tid, const TileGeom& g, const TileParams& P, uint32_t* R,
                               TileCells c) {
    tile_deposit_halo<PB>(tid, g, P, R, c);
    tile_gather_coarse<PB>(tid, g, P, c);
}

// --- phase 2: forward real transform along x (1024 rows, 2 per thread) -----
// A float2 row of C takes the bytes of its own density row, so each thread
// transforms in place.  A __half2 row takes half of them, landing on another
// thread's row: the rows are then read, transformed and, after a barrier,
// written, one row per thread at a time.  There the density less `mean` (an
// estimate of the box's mean; it only moves the k = 0 mode, where the
// short-range kernel vanishes) is scaled by the power of two `scale`, so that
// FP16 holds the fluctuations, not the mean, within its range.
template <typename CT = float2>
PMPM_HD void tile_fwd_x(int tid, uint32_t* R, float scale = 1.f, float mean = 0.f) {
    CT* C = reinterpret_cast<CT*>(R);
    constexpr bool kHalf = !std::is_same<CT, float2>::value;
    for (int r = tid; r < 1024; r += kTileThreads) {
        const int y = r & 31, z = r >> 5;
        float x[32];
#pragma unroll
        for (int n = 0; n < 32; ++n) x[n] = kHalf ? (u32_to_f32(R[ridx(n, y, z)]) - mean) * scale
                                                  : u32_to_f32(R[ridx(n, y, z)]);
        float2 X[17];
        rfft32x2(x, X);
#ifdef __CUDA_ARCH__
        if (kHalf) __syncthreads();
#endif
        cstore(C, cidx(0, y, z), make_float2(X[0].x, X[16].x));   // pack Nyquist
#pragma unroll
        for (int k = 1; k < 16; ++k) cstore(C, cidx(k, y, z), X[k]);
    }
}

// --- phase 3: forward complex transform along y (512 pencils) --------------
template <typename CT>
PMPM_HD void tile_fwd_y(int tid, CT* C) {
    const int kx = tid & 15, z = tid >> 4;
    float2 a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[bitrev<5>(k)] = cload(C, cidx(kx, k, z));
    fft_dit<32, -1>(a);
#pragma unroll
    for (int k = 0; k < 32; ++k) cstore(C, cidx(kx, k, z), a[k]);
}

// |signed frequency| and its sign for a 32-point index
PMPM_HD int kabs32(int i) { return i <= 16 ? i : 32 - i; }
PMPM_HD float ksgn32(int i) { return i == 0 ? 0.f : (i < 16 ? 1.f : (i == 16 ? 1.f : -1.f)); }

// Packed index of the symmetric pair (b, c): row b holds c = b..16.
PMPM_HD int green_off(int b) { return b * kGreenS - (b * (b - 1)) / 2 - b; }
PMPM_HD int green_tri(int b, int c) {
    return b <= c ? green_off(b) + c : green_off(c) + b;
}


// --- phase 5a: Green multiply (Eq. 1) and inverse transform along z -------
// For kx = 1..15: G = rho~ K~_d = -i S rho~.  For the packed kx = 0 pencil,
// Z = A + iB holds the kx = 0 (A) and kx = 16 (B) planes; with the partner
// Z' = Z(-ky, -kz): A = (Z + conj Z')/2, B = (Z - conj Z')/(2i), and the packed
// product A K~_d(0) + i B K~_d(16) = -i[(s0+s16)/2 Z + (s0-s16)/2 conj Z'].
// Thread mapping of the z passes: warp w owns kx = w and lane l owns ky = l,
// so warp 0 alone carries the packed kx = 0 / 16 pencils and the other warps
// run without divergence; every half-warp touches 16 distinct bank pairs.
template <int D, typename Spec, typename CT>
PMPM_HD void inv_z_pencil(int kx, int ky, int nz, const float* gS, Spec spec, const CT* C,
                          float2* W) {
    const int ay = kabs32(ky);
    float2 a[32];
    if (D == 0 && kx == 0) {
        // S_x vanishes on both planes kx = 0 and kx = 16 (odd in x, zero at Nyquist)
#pragma unroll
        for (int zo = 0; zo < kTileOut; ++zo)
            if (zo < nz) W[widx(0, ky, zo)] = make_float2(0.f, 0.f);
        return;
    }
    // Each case has its own unrolled kz loop with no branch inside, so the
    // loads of all 32 iterations can be scheduled ahead of their use.
    // Per-thread parts of the table index (own-axis row a is stored at a - 1);
    // the third index |kz| is a compile-time constant in the unrolled loop.
    if (D == 0 || kx != 0) {
        const float sgy = (D == 1 && (ay == 0 || ay == 16)) ? 0.f : ksgn32(ky);
        const int bfix = D == 0 ? ay : kx;                   // pair (b, c) with b fixed
        const int offA = green_off(bfix);
        const int rowA = D == 0 ? (kx - 1) * kGreenTri : (ay >= 1 && ay <= 15 ? ay - 1 : 0) * kGreenTri;
        const int txy = green_tri(kx, ay);
#pragma unroll
        for (int kz = 0; kz < 32; ++kz) {
            const int az = kabs32(kz);
            const float2 Z = spec(kz);
            float cA;
            if (D == 2) {
                const float sz = (az == 0 || az == 16) ? 0.f : ksgn32(kz);
                const int rz = (az >= 1 && az <= 15 ? az - 1 : 0) * kGreenTri;
                cA = sz * gS[rz + txy];
            } else {
                const int idx = bfix <= az ? offA + az : green_off(az) + bfix;
                cA = (D == 0 ? 1.f : sgy) * gS[rowA + idx];
            }
            a[bitrev<5>(kz)] = make_float2(cA * Z.y, -(cA * Z.x));   // G = -i cA Z
        }
    } else {
        // packed kx = 0 / 16 pencil (y and z forces): b = 0 and b = 16
        const float sgy = (D == 1 && (ay == 0 || ay == 16)) ? 0.f : ksgn32(ky);
        const int rowA = (ay >= 1 && ay <= 15 ? ay - 1 : 0) * kGreenTri;
        const int t0 = green_tri(0, ay), t16 = green_tri(16, ay);
#pragma unroll
        for (int kz = 0; kz < 32; ++kz) {
            const int az = kabs32(kz);
            const float2 Z = spec(kz);
            const float2 Zp = cload(C, cidx(0, (32 - ky) & 31, (32 - kz) & 31));
            float s0, s16;
            if (D == 2) {
                const float sz = (az == 0 || az == 16) ? 0.f : ksgn32(kz);
                const int rz = (az >= 1 && az <= 15 ? az - 1 : 0) * kGreenTri;
                s0 = sz * gS[rz + t0];
                s16 = sz * gS[rz + t16];
            } else {
                s0 = sgy * gS[rowA + green_off(0) + az];
                s16 = sgy * gS[rowA + green_off(az) + 16];
            }
            const float cA = 0.5f * (s0 + s16), cB = 0.5f * (s0 - s16);
            // V = cA Z + cB conj(Zp);  G = -i V
            const float vx = cA * Z.x + cB * Zp.x;
            const float vy = cA * Z.y - cB * Zp.y;
            a[bitrev<5>(kz)] = make_float2(vy, -vx);
        }
    }
    fft_dit<32, 1>(a);
#pragma unroll
    for (int zo = 0; zo < kTileOut; ++zo)
        if (zo < nz) W[widx(kx, ky, zo)] = a[zo + kBuffer - 1];
}

template <int D, typename CT>
PMPM_HD void tile_inv_z(int tid, const TileGeom& g, const float* gS, const CT* C, float2* W) {
    const int kx = tid >> 5, ky = tid & 31;
    inv_z_pencil<D>(kx, ky, g.T[2] + 2, gS, [&](int kz) { return cload(C, cidx(kx, ky, kz)); }, C, W);
}

// --- phase 4 + 5a of the x force: forward transform along z, then at once
// the x-force Green multiply and inverse z of the same pencil from the
// registers (the stored spectrum serves the y and z forces).  Same thread
// mapping as the inverse z passes; every half-warp touches 16 distinct bank
// pairs of the (kx ^ ky) swizzle.
template <typename CT>
PMPM_HD void tile_fwd_z_inv_z0(int tid, const TileGeom& g, const float* gS, CT* C, float2* W) {
    const int kx = tid >> 5, ky = tid & 31;
    float2 a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[bitrev<5>(k)] = cload(C, cidx(kx, ky, k));
    fft_dit<32, -1>(a);
#pragma unroll
    for (int k = 0; k < 32; ++k) cstore(C, cidx(kx, ky, k), a[k]);
    inv_z_pencil<0>(kx, ky, g.T[2] + 2, gS, [&](int kz) { return a[kz]; }, C, W);
}

// --- phase 5b: inverse transform along y, pruned to T + 2 output rows -----
// The inverse y and x passes are the same for the three force components;
// one out-of-line copy each keeps the kernel's code within the instruction
// cache (measured: 1.2% faster than three inlined copies).
__host__ __device__ __noinline__ void tile_inv_y(int tid, const TileGeom& g, float2* W) {
    const int nz = g.T[2] + 2, ny = g.T[1] + 2;
    if (tid >= 16 * nz) return;
    const int kx = tid & 15, zo = tid >> 4;
    float2 a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[bitrev<5>(k)] = W[widx(kx, k, zo)];
    fft_dit<32, 1>(a);
#pragma unroll
    for (int yo = 0; yo < kTileOut; ++yo)
        if (yo < ny) W[widx(kx, yo, zo)] = a[yo + kBuffer - 1];
}

// --- phase 5c: inverse real transform along x, pruned to T + 2 columns ----
__host__ __device__ __noinline__ void tile_inv_x(int tid, const TileGeom& g, float2* W) {
    const int ny = g.T[1] + 2, nz = g.T[2] + 2, nx = g.T[0] + 2;   // all even
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
        // outputs xo, xo + 1 as one 8-byte store (the pair wfidx(xo), wfidx(xo + 1))
#pragma unroll
        for (int xo = 0; xo < kTileOut; xo += 2)
            if (xo < nx) W[widx(xo >> 1, yo, zo)] = make_float2(x[xo + kBuffer - 1], x[xo + kBuffer]);
    }
}

// --- phase 5d: interpolate component D to the tile's own particles, add the
// parked long-range part, then (mode 1) kick and drift that component.  The
// last component also adds each particle to its new cell's count and sums
// (the re-encode's histogram, fused here so that the codes and momenta are
// not read back by another pass).  LM (the low-memory step): the new codes
// are not stored; the fused sums derive the codes of the first two
// components from the old codes and the new momenta, as the re-encode does.
template <int D, bool LM, int PB>
PMPM_HD void tile_interp(int tid, const TileGeom& g, const TileParams& P, const float2* W,
                         TileCells c, unsigned long long& lo, unsigned long long& hi,
                         float gscale = 2.384185791015625e-07f) {
    using F = PosFmt<PB>;
    constexpr int U = 2;   // particles per thread per iteration, loads issued together
    const float* Wf = reinterpret_cast<const float*>(W);
    const int64_t ncells = (int64_t)P.nc * P.nc * P.nc;
    const int64_t n = P.n;
    const int M = P.nc * F::kBins;
    const float sigma = bits_to_f32(c.misc[4]);
    const float kick = bits_to_f32(c.misc[5]), drift = bits_to_f32(c.misc[6]);
    const uint8_t* ud = D == 0 ? P.u0 : (D == 1 ? P.u1 : P.u2);
    float* slot = P.mode == 0 ? P.G : P.Pn;
    const int ptotal = c.ppre[kOwnMax];
    const int64_t base = own_base(c);
    const float* vcD = P.vc + D * ncells;
    const bool fuse = D == 2 && P.mode == 1 && P.counts_new != nullptr;
    for (int v0 = tid; v0 < ptotal; v0 += U * kTileThreads) {
        int64_t j[U];
        int Q[U][3], cell[U];   // codes below nc 65536 <= 2^26, cells below 2^30
        float gcd[U], vcd[U];
        int u8[U];
        int32_t q01[U][2];
        float p01[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * kTileThreads;
            const int p = prefix_find<kOwnMax>(c.ppre, v < ptotal ? v : 0);
            j[u] = v < ptotal ? base + c.prel[p] + (v - c.ppre[p]) : -1;
            const int cx = g.c0[0] + p % kOwnDim, cy = g.c0[1] + (p / kOwnDim) % kOwnDim,
                      cz = g.c0[2] + p / (kOwnDim * kOwnDim);
            cell[u] = cx + P.nc * (cy + P.nc * cz);
            if (j[u] >= 0) {
                Q[u][0] = cx * F::kBins + load_bin<PB>(P.m0, j[u]);
                Q[u][1] = cy * F::kBins + load_bin<PB>(P.m1, j[u]);
                Q[u][2] = cz * F::kBins + load_bin<PB>(P.m2, j[u]);
                gcd[u] = slot[D * n + j[u]];
                if (P.mode >= 1) {
                    u8[u] = ud[j[u]];
                    vcd[u] = vcD[cell[u]];
                }
                if (fuse) {
                    if (!LM) {
                        q01[u][0] = P.Qn[j[u]];
                        q01[u][1] = P.Qn[n + j[u]];
                    }
                    p01[u][0] = P.Pn[j[u]];
                    p01[u][1] = P.Pn[n + j[u]];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j[u] < 0) continue;
            // fine gather
            int lo3[3], w1[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const int s = 2 * Q[u][e] + 1 - F::kCodesPerFine - F::kFineW * g.o[e];
                lo3[e] = (s >> F::kFineWBits) - (kBuffer - 1);
                w1[e] = s & (F::kFineW - 1);
            }
            float gf = 0.f;
            constexpr int W = F::kFineW;
            // 1-byte weights: products of integers <= 128, exact in float
            const float fx[2] = {(float)(W - w1[0]), (float)w1[0]};
            const float fy[2] = {(float)(W - w1[1]), (float)w1[1]};
            const float fz[2] = {(float)(W - w1[2]), (float)w1[2]};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
                const float w = PB == 1 ? fx[dx] * (fy[dy] * fz[dz])
                                        : (float)cic_weight3<PB>(dx ? w1[0] : W - w1[0], dy ? w1[1] : W - w1[1],
                                                                 dz ? w1[2] : W - w1[2]);
                gf += w * Wf[wfidx(lo3[0] + dx, lo3[1] + dy, lo3[2] + dz)];
            }
            // weights in units of 2^-21, and the forward x transform (rfft32x2)
            // leaves the whole spectrum doubled: gscale = 2^-22 (over the
            // density's scale with FP16 spectrum storage; a power of two)
            const float gval = gf * gscale + gcd[u];
            if (P.mode == 0) {
                slot[D * n + j[u]] = gval;
                continue;
            }
            // kick (Eq. 3 decode, then p += kick * g) and integer drift
            const float pv = decode_momentum(vcd[u], sigma, c.Td[u8[u]]);
            const float pn = fadd_rn(pv, fmul_rn(kick, gval));
            if (!(pn == pn) || !(gval == gval)) flag_error(P.err, kErrNaN);
            if (fabsf(pn) >= 1048576.f) flag_error(P.err, kErrMomentum);
            const int qn = drift_code(Q[u][D], pn, drift, M, P.err);
            if (!LM) P.Qn[D * n + j[u]] = (int32_t)qn;
            P.Pn[D * n + j[u]] = pn;
            if (!fuse) continue;
            if (LM) {
                q01[u][0] = drift_code(Q[u][0], p01[u][0], drift, M, P.err);
                q01[u][1] = drift_code(Q[u][1], p01[u][1], drift, M, P.err);
            }
            const int32_t qa[3] = {q01[u][0], q01[u][1], qn};
            const float pa[3] = {p01[u][0], p01[u][1], pn};
            const int key = (qa[0] >> F::kShift) + P.nc * ((qa[1] >> F::kShift) + P.nc * (qa[2] >> F::kShift));
            gmem_add_i32(&P.counts_new[key], 1);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                long long fx = 0;
                if (fabsf(pa[d]) < 1048576.f) fx = fix24_rn(pa[d]);
                else flag_error(P.err, pa[d] == pa[d] ? kErrMomentum : kErrNaN);
                gmem_add_u64(&P.S[d * ncells + key], (unsigned long long)fx);
                add_square128(fx, lo, hi);
            }
        }
    }
}

}  // namespace pmpm
