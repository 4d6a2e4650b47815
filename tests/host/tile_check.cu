// Host checks of the tile kernel's index arithmetic (tile_core.cuh, built for
// the host): the shared-memory swizzles, the tiling of the coarse mesh, the
// own-cell and halo-cell maps, the carving of shared memory into the cell
// tables, the prologue's staging of the halo table and of the long-range
// force window, the deposit phases (cell prefix sums, particle maps, integer
// CIC, parked long-range force) against a plain deposit and gather of a
// clustered box, and the transform phases (forward x, y, z, Green multiply
// with the packed table, pruned inverse z, y, x) against a plain DFT
// convolution, the interpolation with kick, drift and the fused new-cell
// histogram against a plain gather and the Eq. 3 decode, and the
// low-memory passes (counts, dispersion, scatter) against the default
// pass.  Nothing here needs a GPU.  Prints one line per check: "<name> <cases> <failures> [<max
// error>]".
#include "../../paper_2003_03931_gb300/csrc/tile_core.cuh"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

using namespace pmpm;

static unsigned long long rng_state = 0x2545F4914F6CDD1Dull;
static unsigned long long next_u64() {
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return rng_state;
}
static int pmod(long long a, long long n) { return (int)(((a % n) + n) % n); }

// Every index map is a bijection onto its array, and 32 consecutive words
// (16 consecutive float2) along the axes the pencil passes walk fall in
// distinct banks.
static void check_swizzles() {
    long long n = 0, bad = 0;
    std::vector<int> hit(2 * kTileR);
    auto bijective = [&](int range, auto f, int nx, int ny, int nz) {
        std::fill(hit.begin(), hit.end(), 0);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const int i = f(x, y, z);
                    ++n;
                    if (i < 0 || i >= range) ++bad;
                    else ++hit[i];
                }
        for (int i = 0; i < range; ++i) bad += hit[i] != 1;
    };
    bijective(kTileR, [](int x, int y, int z) { return ridx(x, y, z); }, 32, 32, 32);
    bijective(kTileR / 2, [](int x, int y, int z) { return cidx(x, y, z); }, 16, 32, 32);
    bijective(kTileW, [](int x, int y, int z) { return widx(x, y, z); }, 16, 32, kTileOut);
    bijective(2 * kTileW, [](int x, int y, int z) { return wfidx(x, y, z); }, 32, 32, kTileOut);
    // the float view addresses the same pair as the complex view
    for (int zo = 0; zo < kTileOut; ++zo)
        for (int yo = 0; yo < 32; ++yo)
            for (int xo = 0; xo < 32; ++xo, ++n)
                bad += wfidx(xo, yo, zo) != 2 * widx(xo >> 1, yo, zo) + (xo & 1);
    // banks: word maps mod 32 along x and y, float2 maps mod 16 along kx and
    // along each half of ky
    auto distinct = [&](int mod, auto idx, int len) {
        unsigned long long seen = 0;
        for (int t = 0; t < len; ++t) seen |= 1ull << (idx(t) % mod);
        ++n;
        bad += __builtin_popcountll(seen) != len;
    };
    for (int z = 0; z < 32; ++z)
        for (int a = 0; a < 32; ++a) {
            distinct(32, [&](int t) { return ridx(t, a, z); }, 32);
            distinct(32, [&](int t) { return ridx(a, t, z); }, 32);
        }
    for (int z = 0; z < 32; ++z)
        for (int a = 0; a < 32; ++a) {
            distinct(16, [&](int t) { return cidx(t, a, z); }, 16);
            if (a < 16)
                for (int h = 0; h < 2; ++h) {
                    distinct(16, [&](int t) { return cidx(a, 16 * h + t, z); }, 16);
                    if (z < kTileOut) distinct(16, [&](int t) { return widx(a, 16 * h + t, z); }, 16);
                }
        }
    printf("swizzles %lld %lld\n", n, bad);
}

// Every allowed mesh (nc a power of two from 8 to 1024, tiles of at most 4
// or 5 cells): the tiles partition each axis into runs of 4 or 5 cells; a
// tile's halo box (two cells each side) never holds a cell twice; the tile
// and its buffer fit the FFT box; each coarse cell belongs to one tile.
static void check_tiling() {
    long long n = 0, bad = 0;
    for (int nc = 8; nc <= 1024; nc *= 2)
        for (int tm = 4; tm <= 5; ++tm) {
            const int nt = tile_count(nc, tm);
            ++n;
            bad += (long long)nt * nt * nt > 2147483647ll;   // grid.x limit
            bad += tile_bound(0, nc, nt) != 0 || tile_bound(nt, nc, nt) != nc;
            for (int t = 0; t < nt; ++t) {
                const int s = tile_bound(t + 1, nc, nt) - tile_bound(t, nc, nt);
                ++n;
                bad += s < 4 || s > kTileMaxCoarse || s + 4 > nc || kRatio * s + 2 * kBuffer > kTileFFT ||
                       kRatio * s + 2 > kTileOut;
            }
            if (nc > 64) continue;
            std::vector<int> owner(nc * nc * nc, 0);
            for (int b = 0; b < nt * nt * nt; ++b) {
                const TileGeom g = tile_geom(b, nc, nt);
                for (int z = g.c0[2]; z < g.c1[2]; ++z)
                    for (int y = g.c0[1]; y < g.c1[1]; ++y)
                        for (int x = g.c0[0]; x < g.c1[0]; ++x) ++owner[x + nc * (y + nc * z)];
                for (int d = 0; d < 3; ++d) {
                    ++n;
                    bad += g.T[d] != kRatio * (g.c1[d] - g.c0[d]) || g.o[d] != kRatio * g.c0[d] - kBuffer;
                }
            }
            for (int c : owner) {
                ++n;
                bad += c != 1;
            }
        }
    printf("tiling %lld %lld\n", n, bad);
}

// The 32^3 box's circular convolution equals the linear one on the output
// nodes [-1, T] for any density on the box's nodes [-6, T + 5] and a kernel
// that vanishes beyond 5 nodes per axis: no pair aliases into the support.
static void check_no_alias() {
    long long n = 0, bad = 0;
    for (int T = 16; T <= 20; T += 4)
        for (int y = kBuffer - 1; y <= kBuffer + T; ++y)
            for (int x = 0; x < T + 2 * kBuffer; ++x) {
                int c = pmod(y - x, kTileFFT);
                if (c >= kTileFFT / 2) c -= kTileFFT;
                ++n;
                if (std::abs(c) <= kBuffer - 1) bad += c != y - x;
            }
    printf("no_alias %lld %lld\n", n, bad);
}

// Own cells: for each tile shape, own_valid accepts exactly the tile's cells
// and own_to_halo sends them to distinct halo cells two cells in from the
// halo box's corner.
static void check_own_cells() {
    long long n = 0, bad = 0;
    for (int sz = 4; sz <= 5; ++sz)
        for (int sy = 4; sy <= 5; ++sy)
            for (int sx = 4; sx <= 5; ++sx) {
                TileGeom g{};
                g.c0[0] = 8; g.c1[0] = 8 + sx;
                g.c0[1] = 4; g.c1[1] = 4 + sy;
                g.c0[2] = 0; g.c1[2] = sz;
                std::vector<int> seen(kHaloMax, 0);
                int valid = 0;
                for (int p = 0; p < kOwnMax; ++p) {
                    const int px = p % kOwnDim, py = (p / kOwnDim) % kOwnDim, pz = p / (kOwnDim * kOwnDim);
                    const bool inside = px < sx && py < sy && pz < sz;
                    ++n;
                    bad += own_valid(g, p) != inside;
                    if (!inside) continue;
                    ++valid;
                    const int h = own_to_halo(p);
                    if (h < 0 || h >= kHaloMax) { ++bad; continue; }
                    const int hx = h % kHaloDim, hy = (h / kHaloDim) % kHaloDim, hz = h / (kHaloDim * kHaloDim);
                    bad += hx != px + 2 || hy != py + 2 || hz != pz + 2 || seen[h]++ != 0;
                    // inside the halo box that the prologue fills (sides s + 4)
                    bad += hx >= sx + 4 || hy >= sy + 4 || hz >= sz + 4;
                }
                bad += valid != sx * sy * sz;
            }
    printf("own_cells %lld %lld\n", n, bad);
}

// The carving of shared memory: R, W, the Green table, the own-cell table and
// the decode table end at kTileSmemBytes (at most 227 KB per CTA); inside W
// the cell tables, the map, the long-range window, the own-particle map and
// the chunk sums neither overlap nor leave W, each aligned for its type.
static void check_smem_layout() {
    long long n = 0, bad = 0;
    std::vector<unsigned char> smem(kTileSmemBytes + 64);
    unsigned char* base = smem.data();
    float2* W = reinterpret_cast<float2*>(base + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(base + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    const TileCells c = tile_cells(W, O);
    const float* flw = fl_window(c);
    struct Region { const char* name; const void* p; size_t bytes; size_t align; };
    const Region w[] = {
        {"st", c.st, kHaloMax * 8, 8},
        {"cnt", c.cnt, kHaloMax * 4, 4},
        {"pre", c.pre, (kHaloMax + 1) * 4, 4},
        {"map", c.map, (size_t)kMapCap * 2, 2},
        {"flw", flw, 3 * kFlWinNodes * 4, 4},
        {"pmap", c.pmap, kPMapCap, 1},
        {"tot", c.tot, kHaloChunks * 4, 4},
        {"cmax", c.cmax, kHaloChunks * 4, 4},
    };
    const Region o[] = {
        {"ppre", c.ppre, (kOwnMax + 1) * 4, 4},
        {"prel", c.prel, kOwnMax * 4, 4},
        {"misc", c.misc, 8 * 4, 4},
        {"Td", c.Td, 256 * 4, 4},
    };
    auto inside = [&](const Region* r, int k, const unsigned char* lo, const unsigned char* hi) {
        for (int i = 0; i < k; ++i) {
            const unsigned char* p = static_cast<const unsigned char*>(r[i].p);
            ++n;
            bad += p < lo || p + r[i].bytes > hi || ((size_t)(p - base) % r[i].align) != 0;
            for (int j = 0; j < i; ++j) {
                const unsigned char* q = static_cast<const unsigned char*>(r[j].p);
                ++n;
                bad += p < q + r[j].bytes && q < p + r[i].bytes;
            }
        }
    };
    inside(w, 8, reinterpret_cast<unsigned char*>(W), reinterpret_cast<unsigned char*>(W + kTileW));
    inside(o, 4, reinterpret_cast<unsigned char*>(O), base + kTileSmemBytes);
    ++n;
    bad += reinterpret_cast<unsigned char*>(c.Td + 256) != base + kTileSmemBytes;
    ++n;
    bad += kTileSmemBytes > 227u * 1024u;
    // the float2 spectrum view of R and the uint4 clear stay inside R
    ++n;
    bad += (size_t)kTileR * 4 % 16 != 0 || (size_t)(kTileR / 2) * 8 != (size_t)kTileR * 4;
    printf("smem_layout %lld %lld\n", n, bad);
}

// The prologue, run for all 512 threads of one tile on host arrays: the halo
// table holds the offsets and counts of the wrapped cells around the tile
// (zero count outside a smaller tile's box), and the staged window gives, for
// particles anywhere in the tile's own cells, the same long-range force as a
// plain periodic CIC gather from the whole coarse mesh.
template <int PB>
static void check_prologue(long long& n, long long& bad, double& err, int nc, int tm) {
    using F = PosFmt<PB>;
    const int nt = tile_count(nc, tm);
    const int64_t nc3 = (int64_t)nc * nc * nc;
    std::vector<int32_t> counts(nc3);
    std::vector<int64_t> offsets(nc3 + 1);
    std::vector<float> Fl(3 * nc3), green(kGreenPacked), Td(256);
    for (int64_t i = 0; i < nc3; ++i) {
        counts[i] = (int32_t)(1 + i % 13);
        offsets[i] = 7 * i + 3;
    }
    float fmax = 0.f;
    for (auto& v : Fl) {
        v = (float)((double)(next_u64() >> 11) * 0x1p-53 * 2.0 - 1.0);
        fmax = std::fmax(fmax, std::fabs(v));
    }
    for (int i = 0; i < kGreenPacked; ++i) green[i] = (float)i;
    for (int i = 0; i < 256; ++i) Td[i] = (float)(i - 128);
    const float sigma = 0.25f;
    TileParams P{};
    P.nc = nc;
    P.nt = nt;
    P.counts = counts.data();
    P.offsets = offsets.data();
    P.Fl = Fl.data();
    P.green = green.data();
    P.Tdec = Td.data();
    P.sigma = &sigma;
    P.mode = 0;
    constexpr size_t kGuard = 256;
    std::vector<unsigned char> smem(kTileSmemBytes + kGuard);
    unsigned char* base = smem.data();
    uint32_t* R = reinterpret_cast<uint32_t*>(base);
    float2* W = reinterpret_cast<float2*>(base + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(base + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    const int ntiles = nt * nt * nt;
    for (int b = 0; b < ntiles; b += 1 + ntiles / 40) {
        memset(base, 0xA5, smem.size());
        const TileGeom g = tile_geom(b, nc, nt);
        const TileCells c = tile_cells(W, O);
        for (int t = 0; t < kTileThreads; ++t) tile_prologue(t, g, P, c, R, gS);
        for (size_t i = kTileSmemBytes; i < smem.size(); ++i) {
            ++n;
            bad += base[i] != 0xA5;   // nothing written past the end
        }
        // halo table
        const int hx = g.c1[0] - g.c0[0] + 4, hy = g.c1[1] - g.c0[1] + 4, hz = g.c1[2] - g.c0[2] + 4;
        for (int h = 0; h < kHaloMax; ++h) {
            const int bx = h % kHaloDim, by = (h / kHaloDim) % kHaloDim, bz = h / (kHaloDim * kHaloDim);
            ++n;
            if (bx < hx && by < hy && bz < hz) {
                const int64_t cell = pmod(g.c0[0] - 2 + bx, nc) +
                                     (int64_t)nc * (pmod(g.c0[1] - 2 + by, nc) + (int64_t)nc * pmod(g.c0[2] - 2 + bz, nc));
                bad += c.st[h] != offsets[cell] || c.cnt[h] != counts[cell];
            } else {
                bad += c.cnt[h] != 0;
            }
        }
        for (int i = 0; i < kGreenPacked; ++i) bad += gS[i] != green[i];
        for (int i = 0; i < 256; ++i) bad += c.Td[i] != Td[i];
        for (int i = 0; i < kTileR; ++i) bad += R[i] != 0u;
        n += kGreenPacked + 256 + kTileR;
        // the window against a plain periodic gather, at random particles of
        // the own cells and at the extreme codes of the first and last cells
        const float* flw = fl_window(c);
        for (int k = 0; k < 400; ++k) {
            int Q[3];
            for (int e = 0; e < 3; ++e) {
                const int s = g.c1[e] - g.c0[e];
                int cell = g.c0[e] + (int)(next_u64() % s), m = (int)(next_u64() % F::kBins);
                if (k < 8) {
                    cell = (k >> e) & 1 ? g.c1[e] - 1 : g.c0[e];
                    m = (k >> e) & 1 ? F::kBins - 1 : 0;
                }
                Q[e] = cell * F::kBins + m;
            }
            float gc[3];
            coarse_gather_win<PB>(flw, g, Q, gc);
            int i0[3];
            double f[3];
            for (int e = 0; e < 3; ++e) {
                const double d = ((double)Q[e] + 0.5) / F::kBins - 0.5;   // from node 0, in cells
                i0[e] = (int)std::floor(d);
                f[e] = d - i0[e];
            }
            for (int e = 0; e < 3; ++e) {
                double ref = 0.0;
                for (int cn = 0; cn < 8; ++cn) {
                    const int dx = cn & 1, dy = (cn >> 1) & 1, dz = cn >> 2;
                    const double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                    const int64_t node = pmod(i0[0] + dx, nc) +
                                         (int64_t)nc * (pmod(i0[1] + dy, nc) + (int64_t)nc * pmod(i0[2] + dz, nc));
                    ref += w * Fl[e * nc3 + node];
                }
                const double d = std::fabs((double)gc[e] - ref) / fmax;
                ++n;
                if (!(d <= 2e-6)) ++bad;
                if (d > err || d != d) err = d;
            }
        }
    }
}

static void run_prologue_checks() {
    long long n = 0, bad = 0;
    double err = 0.0;
    for (int nc = 8; nc <= 64; nc *= 2)
        for (int tm = 4; tm <= 5; ++tm) {
            check_prologue<1>(n, bad, err, nc, tm);
            check_prologue<2>(n, bad, err, nc, tm);
        }
    printf("prologue %lld %lld %.3e\n", n, bad, err);
}

// A clustered periodic box (cell-ordered store, counts, offsets) for the
// deposit check: a few particles in every cell, a crowded block of cells
// around one tile (more halo particles than the cell map holds, more own
// particles than the own-particle map holds) and one cell above 255 particles
// (the checked deposit path); optionally an empty block of 9^3 cells.
template <int PB>
struct Box {
    int nc;
    int64_t n = 0;
    std::vector<int32_t> counts;
    std::vector<int64_t> offsets;
    std::vector<uint16_t> m[3];   // bins, PB bytes used
    std::vector<uint8_t> s[3];    // the same bins as PB-byte streams
    Box(int nc_, int crowd_x, int crowd_y, int crowd_z, int empty = -100) : nc(nc_) {
        const int64_t nc3 = (int64_t)nc * nc * nc;
        counts.resize(nc3);
        offsets.resize(nc3 + 1);
        for (int z = 0; z < nc; ++z)
            for (int y = 0; y < nc; ++y)
                for (int x = 0; x < nc; ++x) {
                    int k = (int)(next_u64() % 5);
                    if (std::abs(x - crowd_x) <= 4 && std::abs(y - crowd_y) <= 4 && std::abs(z - crowd_z) <= 4)
                        k = 130 + (int)(next_u64() % 9);
                    if (x == crowd_x + 1 && y == crowd_y && z == crowd_z) k = 400;
                    if (std::abs(x - empty) <= 4 && std::abs(y - empty) <= 4 && std::abs(z - empty) <= 4) k = 0;
                    counts[x + (int64_t)nc * (y + (int64_t)nc * z)] = k;
                }
        for (int64_t i = 0; i < nc3; ++i) {
            offsets[i] = n;
            n += counts[i];
        }
        offsets[nc3] = n;
        for (int e = 0; e < 3; ++e) {
            m[e].resize(n);
            for (int64_t j = 0; j < n; ++j) m[e][j] = (uint16_t)(next_u64() % PosFmt<PB>::kBins);
            s[e].resize(n * PB);
            for (int64_t j = 0; j < n; ++j) memcpy(&s[e][j * PB], &m[e][j], PB);   // little endian
        }
    }
};

// 3-D CIC weight in units of 2^-21 from per-axis weights in units of 1/(2U)
// of a fine cell (U position codes per fine cell): exact for 1-byte codes,
// rounded half to even from the exact product for 2-byte codes
template <int PB>
static uint32_t weight_ref(uint64_t wx, uint64_t wy, uint64_t wz) {
    const uint64_t prod = wx * wy * wz;
    if (PB == 1) return (uint32_t)prod;
    const uint64_t unit = 1ull << 24, q = prod / unit, r = prod % unit;
    return (uint32_t)(r * 2 > unit || (r * 2 == unit && (q & 1)) ? q + 1 : q);
}

// Phases 1a-1c of the tile kernel run thread by thread on host arrays: the
// fine density in shared memory equals a plain integer CIC deposit of every
// particle of the 5^3-cell halo box, clipped to the 32^3 box, node by node;
// every own particle's long-range force slot holds the plain periodic gather.
template <int PB>
static void check_deposit(long long& n, long long& bad, double& err) {
    using F = PosFmt<PB>;
    const int nc = 32, tm = 5, nt = tile_count(nc, tm);
    const int crowd = 11;   // tile 2 spans cells 9..12 along each axis
    Box<PB> box(nc, crowd, crowd, crowd, 24);   // tile 5's halo box (cells 20..28) is empty
    const int64_t nc3 = (int64_t)nc * nc * nc;
    std::vector<float> Fl(3 * nc3), green(kGreenPacked, 0.f), Td(256, 0.f);
    for (auto& v : Fl) v = (float)((double)(next_u64() >> 11) * 0x1p-53 * 2.0 - 1.0);
    std::vector<float> G(3 * box.n);
    const float sigma = 1.f;
    uint32_t errw = 0;
    TileParams P{};
    P.nc = nc;
    P.nt = nt;
    P.n = box.n;
    P.counts = box.counts.data();
    P.offsets = box.offsets.data();
    P.m0 = box.s[0].data();
    P.m1 = box.s[1].data();
    P.m2 = box.s[2].data();
    P.Fl = Fl.data();
    P.green = green.data();
    P.Tdec = Td.data();
    P.sigma = &sigma;
    P.mode = 0;
    P.G = G.data();
    P.err = &errw;
    std::vector<unsigned char> smem(kTileSmemBytes);
    unsigned char* base = smem.data();
    uint32_t* R = reinterpret_cast<uint32_t*>(base);
    float2* W = reinterpret_cast<float2*>(base + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(base + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    // the crowded tile, a neighbour, a ragged tile, the corner tile (wrap)
    // and a tile with no particle in its halo box
    const int tiles[5][3] = {{2, 2, 2}, {3, 2, 2}, {1, 4, 6}, {nt - 1, 0, nt - 1}, {5, 5, 5}};
    for (const auto& tt : tiles) {
        const int b = tt[0] + nt * (tt[1] + nt * tt[2]);
        const TileGeom g = tile_geom(b, nc, nt);
        const TileCells c = tile_cells(W, O);
        std::fill(G.begin(), G.end(), NAN);
        for (int t = 0; t < kTileThreads; ++t) tile_prologue(t, g, P, c, R, gS);
        for (int t = 0; t < kTileThreads; ++t) tile_cells_scan(t, g, c);
        for (int t = 0; t < kTileThreads; ++t) tile_cells_map(t, g, c);
        for (int t = 0; t < kTileThreads; ++t)
            tile_deposit_flat<PB>(t, g, P, R, c);
        // the same phases with the threads in reverse order (another order
        // of the integer adds) leave the same density, word for word
        {
            const std::vector<uint32_t> first(R, R + kTileR);
            for (int t = kTileThreads - 1; t >= 0; --t) tile_prologue(t, g, P, c, R, gS);
            for (int t = kTileThreads - 1; t >= 0; --t) tile_cells_scan(t, g, c);
            for (int t = kTileThreads - 1; t >= 0; --t) tile_cells_map(t, g, c);
            for (int t = kTileThreads - 1; t >= 0; --t)
                tile_deposit_flat<PB>(t, g, P, R, c);
            ++n;
            bad += memcmp(first.data(), R, sizeof(uint32_t) * kTileR) != 0;
        }
        // plain deposit of the halo box's particles
        std::vector<uint32_t> ref(kTileR, 0u);
        int64_t halo_particles = 0, own_particles = 0;
        for (int hz = g.c0[2] - 2; hz < g.c1[2] + 2; ++hz)
            for (int hy = g.c0[1] - 2; hy < g.c1[1] + 2; ++hy)
                for (int hx = g.c0[0] - 2; hx < g.c1[0] + 2; ++hx) {
                    const int64_t cell = pmod(hx, nc) + (int64_t)nc * (pmod(hy, nc) + (int64_t)nc * pmod(hz, nc));
                    const bool own = hx >= g.c0[0] && hx < g.c1[0] && hy >= g.c0[1] && hy < g.c1[1] &&
                                     hz >= g.c0[2] && hz < g.c1[2];
                    const int hc[3] = {hx, hy, hz};
                    for (int64_t j = box.offsets[cell]; j < box.offsets[cell + 1]; ++j) {
                        ++halo_particles;
                        // fine position (unwrapped, in fine cells) of the bin
                        // centre, and its offset from box node 0's centre
                        int lo[3];
                        uint64_t w1[3];
                        for (int e = 0; e < 3; ++e) {
                            const double x = ((double)hc[e] * F::kBins + box.m[e][j] + 0.5) / F::kCodesPerFine;
                            const double d = x - 0.5 - g.o[e];
                            lo[e] = (int)std::floor(d);
                            w1[e] = (uint64_t)((d - lo[e]) * F::kFineW);   // exact
                        }
                        for (int cn = 0; cn < 8; ++cn) {
                            const int dx = cn & 1, dy = (cn >> 1) & 1, dz = cn >> 2;
                            const int x = lo[0] + dx, y = lo[1] + dy, z = lo[2] + dz;
                            if (x < 0 || x >= 32 || y < 0 || y >= 32 || z < 0 || z >= 32) continue;
                            ref[(z * 32 + y) * 32 + x] +=
                                weight_ref<PB>(dx ? w1[0] : F::kFineW - w1[0], dy ? w1[1] : F::kFineW - w1[1],
                                               dz ? w1[2] : F::kFineW - w1[2]);
                        }
                        if (!own) continue;
                        ++own_particles;
                        // its parked long-range force against a plain gather
                        int i0[3];
                        double f[3];
                        for (int e = 0; e < 3; ++e) {
                            const double d = ((double)hc[e] * F::kBins + box.m[e][j] + 0.5) / F::kBins - 0.5;
                            i0[e] = (int)std::floor(d);
                            f[e] = d - i0[e];
                        }
                        for (int e = 0; e < 3; ++e) {
                            double r = 0.0;
                            for (int cn = 0; cn < 8; ++cn) {
                                const int dx = cn & 1, dy = (cn >> 1) & 1, dz = cn >> 2;
                                const double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                                r += w * Fl[e * nc3 + pmod(i0[0] + dx, nc) +
                                            (int64_t)nc * (pmod(i0[1] + dy, nc) + (int64_t)nc * pmod(i0[2] + dz, nc))];
                            }
                            const double d = std::fabs((double)G[e * box.n + j] - r);
                            ++n;
                            if (!(d <= 2e-6)) ++bad;
                            if (d > err || d != d) err = d;
                        }
                    }
                }
        for (int z = 0; z < 32; ++z)
            for (int y = 0; y < 32; ++y)
                for (int x = 0; x < 32; ++x) {
                    ++n;
                    bad += R[ridx(x, y, z)] != ref[(z * 32 + y) * 32 + x];
                }
        // the crowded tile must take the paths past both maps and the
        // checked deposit
        ++n;
        bad += c.pre[kHaloMax] != halo_particles || c.ppre[kOwnMax] != own_particles;
        if (tt[0] == 2 && tt[1] == 2 && tt[2] == 2) {
            ++n;
            bad += !(halo_particles > kMapCap && own_particles > kPMapCap && c.misc[2] > 255);
        }
        if (tt[0] == 5) {
            ++n;
            bad += halo_particles != 0;
        }
    }
    ++n;
    bad += errw != 0u;
}

// A short-range table S(a; b, c) for the spectral check: any values serve
// (the transforms are linear in them); symmetric in the pair (b, c) as the
// packed table requires, and unlike in a and the pair.
static double s_table(int a, int b, int c) {
    return (1.0 + 0.3 * a - 0.02 * a * a) / (1.0 + 0.05 * (b * b + c * c) + 0.013 * b * c + 0.11 * a * (b + c));
}

// Phases 2-5c of the tile kernel (forward real x, complex y, z, then per
// force component the Green multiply with the packed table and the pruned
// inverse z, y, x) run thread by thread on a random density, against a plain
// float64 DFT convolution on the output nodes: F_d = 2 IDFT(K_d DFT(rho))
// (the factor 2 is the forward x transform's doubling, and the inverse
// transforms carry no 1/32), K_d(k) = -i sgn(k_d) S(|k_d|; |k_e|, |k_f|),
// zero where |k_d| is 0 or 16.  Output node o of an axis is box node
// o + 5 (fine node -1 of the tile).
static void check_spectral() {
    long long n = 0, bad = 0;
    double err = 0.0;
    std::vector<unsigned char> smem(kTileSmemBytes);
    unsigned char* base = smem.data();
    uint32_t* R = reinterpret_cast<uint32_t*>(base);
    float2* C = reinterpret_cast<float2*>(base);
    float2* W = reinterpret_cast<float2*>(base + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(base + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    // the packed table: rows a = 1..15, each the pairs b <= c in order
    // (row b holds c = b..16)
    {
        int i = 0;
        for (int a = 1; a <= 15; ++a)
            for (int b = 0; b <= 16; ++b)
                for (int c = b; c <= 16; ++c) gS[i++] = (float)s_table(a, b, c);
        ++n;
        bad += i != kGreenPacked;
    }
    typedef std::complex<double> cd;
    std::vector<cd> tw(32);
    for (int j = 0; j < 32; ++j) tw[j] = std::polar(1.0, -2.0 * M_PI * j / 32.0);
    // separable 32^3 DFT along one axis, sign -1 (forward) or +1
    auto dft_axis = [&](std::vector<cd>& a, int axis, int sign) {
        std::vector<cd> line(32);
        const int st = axis == 0 ? 1 : (axis == 1 ? 32 : 1024);
        for (int u = 0; u < 32; ++u)
            for (int v = 0; v < 32; ++v) {
                const int b0 = axis == 0 ? 32 * u + 1024 * v : (axis == 1 ? u + 1024 * v : u + 32 * v);
                for (int k = 0; k < 32; ++k) {
                    cd acc = 0.0;
                    for (int x = 0; x < 32; ++x) {
                        const cd w = tw[(k * x) & 31];
                        acc += a[b0 + st * x] * (sign < 0 ? w : std::conj(w));
                    }
                    line[k] = acc;
                }
                for (int k = 0; k < 32; ++k) a[b0 + st * k] = line[k];
            }
    };
    auto kabs = [](int k) { return k <= 16 ? k : 32 - k; };
    const int shapes[2][3] = {{0, 1, 2}, {1, 0, 6}};   // tiles (4,5,4) and (5,4,5) cells of nc = 32
    for (const auto& sh : shapes) {
        const int nc = 32, nt = tile_count(nc, 5);
        const TileGeom g = tile_geom(sh[0] + nt * (sh[1] + nt * sh[2]), nc, nt);
        std::vector<cd> rho(kTileR);
        for (int z = 0; z < 32; ++z)
            for (int y = 0; y < 32; ++y)
                for (int x = 0; x < 32; ++x) {
                    const uint32_t v = (uint32_t)(next_u64() % (1u << 22));
                    R[ridx(x, y, z)] = v;
                    rho[(z * 32 + y) * 32 + x] = (double)v;
                }
        for (int ax = 0; ax < 3; ++ax) dft_axis(rho, ax, -1);
        for (int t = 0; t < kTileThreads; ++t) tile_fwd_x(t, R);
        for (int t = 0; t < kTileThreads; ++t) tile_fwd_y(t, C);
        for (int t = 0; t < kTileThreads; ++t) tile_fwd_z_inv_z0(t, g, gS, C, W);
        for (int D = 0; D < 3; ++D) {
            if (D == 1)
                for (int t = 0; t < kTileThreads; ++t) tile_inv_z<1>(t, g, gS, C, W);
            if (D == 2)
                for (int t = 0; t < kTileThreads; ++t) tile_inv_z<2>(t, g, gS, C, W);
            for (int t = 0; t < kTileThreads; ++t) tile_inv_y(t, g, W);
            for (int t = 0; t < kTileThreads; ++t) tile_inv_x(t, g, W);
            std::vector<cd> f(kTileR);
            for (int kz = 0; kz < 32; ++kz)
                for (int ky = 0; ky < 32; ++ky)
                    for (int kx = 0; kx < 32; ++kx) {
                        const int k[3] = {kx, ky, kz};
                        const int a = kabs(k[D]), b = kabs(k[(D + 1) % 3]), c = kabs(k[(D + 2) % 3]);
                        const double sg = k[D] == 0 || k[D] == 16 ? 0.0 : (k[D] < 16 ? 1.0 : -1.0);
                        const double S = sg == 0.0 ? 0.0 : s_table(a, b < c ? b : c, b < c ? c : b);
                        const int i = (kz * 32 + ky) * 32 + kx;
                        f[i] = cd(0.0, -sg * S) * rho[i];
                    }
            for (int ax = 0; ax < 3; ++ax) dft_axis(f, ax, +1);
            const float* Wf = reinterpret_cast<const float*>(W);
            double fmax = 0.0;
            for (const cd& v : f) fmax = std::fmax(fmax, std::abs(v.real()));
            for (int zo = 0; zo < g.T[2] + 2; ++zo)
                for (int yo = 0; yo < g.T[1] + 2; ++yo)
                    for (int xo = 0; xo < g.T[0] + 2; ++xo) {
                        const cd ref = 2.0 * f[((zo + 5) * 32 + yo + 5) * 32 + xo + 5];
                        const double d = std::fabs((double)Wf[wfidx(xo, yo, zo)] - ref.real()) / (2.0 * fmax);
                        ++n;
                        if (!(d <= 1e-5)) ++bad;
                        if (d > err || d != d) err = d;
                    }
        }
    }
    printf("spectral %lld %lld %.3e\n", n, bad, err);
}

// Phase 5d (interpolation) run thread by thread after the deposit phases,
// with W holding a random force field on the output nodes [0, T + 2) of
// each axis and NaN everywhere else (a read outside the pruned output would
// show).  Mode 0: each own particle's slot holds half the plain CIC gather
// of the field (the transforms leave the field doubled) plus its parked
// long-range force.  Mode 1: the momentum is the Eq. 3 decode plus the kick
// times that force, the new code is the old one plus the rounded drift,
// wrapped into the box, and the fused histogram's counts and momentum sums
// match the tile's new codes and momenta.
template <int D, int PB>
static void run_interp(const TileGeom& g, const TileParams& P, const float2* W, TileCells c) {
    unsigned long long lo = 0, hi = 0;
    for (int t = 0; t < kTileThreads; ++t)
        tile_interp<D, false, PB>(t, g, P, W, c, lo, hi);
}

template <int PB>
static void check_interp(long long& n, long long& bad, double& err, int mode) {
    using F = PosFmt<PB>;
    const int nc = 32, nt = tile_count(nc, 5);
    Box<PB> box(nc, 11, 11, 11);
    const int64_t nc3 = (int64_t)nc * nc * nc, np = box.n;
    std::vector<float> Fl(3 * nc3), green(kGreenPacked, 0.f), Td(256), vc(3 * nc3);
    for (auto& v : Fl) v = (float)((double)(next_u64() >> 11) * 0x1p-53 * 2.0 - 1.0);
    for (auto& v : vc) v = (float)((double)(next_u64() >> 11) * 0x1p-53 * 40.0 - 20.0);
    for (int i = 0; i < 256; ++i) Td[i] = (float)(std::tan(M_PI * ((i + 0.5) / 256.0 - 0.5)) * 0.25);
    std::vector<uint8_t> u[3];
    for (int e = 0; e < 3; ++e) {
        u[e].resize(np);
        for (auto& x : u[e]) x = (uint8_t)(next_u64() & 255);
    }
    std::vector<float> G(3 * np), Pn(3 * np);
    std::vector<int32_t> Qn(3 * np), cnew(nc3);
    std::vector<unsigned long long> S(3 * nc3);
    const float sigma = 2.0f, kd[2] = {0.75f, 3.3f};
    uint32_t errw = 0;
    TileParams P{};
    P.nc = nc;
    P.nt = nt;
    P.n = np;
    P.counts = box.counts.data();
    P.offsets = box.offsets.data();
    P.m0 = box.s[0].data();
    P.m1 = box.s[1].data();
    P.m2 = box.s[2].data();
    P.u0 = u[0].data();
    P.u1 = u[1].data();
    P.u2 = u[2].data();
    P.vc = vc.data();
    P.sigma = &sigma;
    P.Tdec = Td.data();
    P.green = green.data();
    P.Fl = Fl.data();
    P.mode = mode;
    P.kd = kd;
    P.G = G.data();
    P.Qn = Qn.data();
    P.Pn = Pn.data();
    P.err = &errw;
    if (mode == 1) {
        P.counts_new = cnew.data();
        P.S = S.data();
    }
    std::vector<unsigned char> smem(kTileSmemBytes);
    unsigned char* base = smem.data();
    uint32_t* R = reinterpret_cast<uint32_t*>(base);
    float2* W = reinterpret_cast<float2*>(base + (size_t)kTileR * 4);
    float* Wf = reinterpret_cast<float*>(W);
    float* gS = reinterpret_cast<float*>(base + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    float* slot = mode == 0 ? G.data() : Pn.data();
    const int M = nc * F::kBins;
    const int tiles[3][3] = {{2, 2, 2}, {1, 4, 6}, {nt - 1, 0, nt - 1}};
    for (const auto& tt : tiles) {
        const TileGeom g = tile_geom(tt[0] + nt * (tt[1] + nt * tt[2]), nc, nt);
        const TileCells c = tile_cells(W, O);
        std::fill(cnew.begin(), cnew.end(), 0);
        std::fill(S.begin(), S.end(), 0ull);
        for (int t = 0; t < kTileThreads; ++t) tile_prologue(t, g, P, c, R, gS);
        for (int t = 0; t < kTileThreads; ++t) tile_cells_scan(t, g, c);
        for (int t = 0; t < kTileThreads; ++t) tile_cells_map(t, g, c);
        for (int t = 0; t < kTileThreads; ++t)
            tile_deposit_flat<PB>(t, g, P, R, c);
        // the tile's own particles and their cells
        std::vector<int64_t> own;
        std::vector<int> ocell;
        for (int z = g.c0[2]; z < g.c1[2]; ++z)
            for (int y = g.c0[1]; y < g.c1[1]; ++y)
                for (int x = g.c0[0]; x < g.c1[0]; ++x) {
                    const int cell = x + nc * (y + nc * z);
                    for (int64_t j = box.offsets[cell]; j < box.offsets[cell + 1]; ++j) {
                        own.push_back(j);
                        ocell.push_back(cell);
                    }
                }
        std::vector<float> field(32 * 32 * 32);
        for (int D = 0; D < 3; ++D) {
            std::fill(Wf, Wf + 2 * kTileW, NAN);
            for (int zo = 0; zo < g.T[2] + 2; ++zo)
                for (int yo = 0; yo < g.T[1] + 2; ++yo)
                    for (int xo = 0; xo < g.T[0] + 2; ++xo) {
                        const float v = (float)((double)(next_u64() >> 11) * 0x1p-53 * 2e3 - 1e3);
                        field[(zo * 32 + yo) * 32 + xo] = v;
                        Wf[wfidx(xo, yo, zo)] = v;
                    }
            std::vector<float> parked(own.size());
            for (size_t i = 0; i < own.size(); ++i) parked[i] = slot[D * np + own[i]];
            if (D == 0) run_interp<0, PB>(g, P, W, c);
            if (D == 1) run_interp<1, PB>(g, P, W, c);
            if (D == 2) run_interp<2, PB>(g, P, W, c);
            for (size_t i = 0; i < own.size(); ++i) {
                const int64_t j = own[i];
                const int cc[3] = {ocell[i] % nc, (ocell[i] / nc) % nc, ocell[i] / (nc * nc)};
                // fine position of the bin centre from output node 0 (fine
                // node -1 of the tile, centre at fine 4 c0 - 0.5)
                int lo[3], q[3];
                double f[3];
                for (int e = 0; e < 3; ++e) {
                    q[e] = cc[e] * F::kBins + box.m[e][j];
                    const double d = ((double)q[e] + 0.5) / F::kCodesPerFine - (kRatio * g.c0[e] - 0.5);
                    lo[e] = (int)std::floor(d);
                    f[e] = d - lo[e];
                }
                double gf = 0.0;
                for (int cn = 0; cn < 8; ++cn) {
                    const int dx = cn & 1, dy = (cn >> 1) & 1, dz = cn >> 2;
                    const double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                    const int x = lo[0] + dx, y = lo[1] + dy, z = lo[2] + dz;
                    gf += w * (x < 0 || y < 0 || z < 0 || x >= 32 || y >= 32 || z >= 32
                                   ? NAN : (double)field[(z * 32 + y) * 32 + x]);
                }
                const double gref = 0.5 * gf + parked[i];
                if (mode == 0) {
                    const double d = std::fabs((double)G[D * np + j] - gref) / 1e3;
                    ++n;
                    if (!(d <= 1e-6)) ++bad;
                    if (d > err || d != d) err = d;
                    continue;
                }
                // mode 1: Eq. 3 decode, kick (float32 operations), drift
                const float pv = vc[D * nc3 + ocell[i]] + sigma * Td[u[D][j]];
                const double pref = (double)pv + (double)kd[0] * gref;
                const float pn = Pn[D * np + j];
                const double d = std::fabs((double)pn - pref) / 1e3;
                ++n;
                if (!(d <= 1e-6)) ++bad;
                if (d > err || d != d) err = d;
                // the new code from the kernel's own momentum: exact
                const float xq = pn * kd[1];
                const long long dq = (long long)std::floor((double)(xq + 0.5f));
                const int qn = pmod((long long)q[D] + dq, M);
                ++n;
                bad += Qn[D * np + j] != qn;
            }
        }
        if (mode == 1) {
            // the fused histogram of the tile's particles in their new cells
            std::vector<int32_t> cref(nc3, 0);
            std::vector<unsigned long long> sref(3 * nc3, 0ull);
            for (int64_t j : own) {
                const int key = Qn[j] / F::kBins + nc * (Qn[np + j] / F::kBins + nc * (Qn[2 * np + j] / F::kBins));
                ++cref[key];
                for (int d = 0; d < 3; ++d)
                    sref[d * nc3 + key] += (unsigned long long)std::llrint((double)Pn[d * np + j] * 16777216.0);
            }
            for (int64_t i = 0; i < nc3; ++i) {
                ++n;
                bad += cnew[i] != cref[i] || S[i] != sref[i] || S[nc3 + i] != sref[nc3 + i] ||
                       S[2 * nc3 + i] != sref[2 * nc3 + i];
            }
        }
    }
    ++n;
    bad += errw != 0u;
}

// The low-memory tile pass (mode 1 without stored codes) against the default
// pass of the same tile with the same force fields: the same new momenta
// bit for bit, the same new-cell counts and momentum sums, the same 128-bit
// second moment sum P^2 (equal to the exact sum over the momenta, past 2^64
// in the crowded tile); and the codes the low-memory re-encode derives from
// the old store and those momenta (drift_code) are the default pass's codes.
template <int D, bool LM>
static void run_interp_lm(const TileGeom& g, const TileParams& P, const float2* W, TileCells c,
                          unsigned long long& lo, unsigned long long& hi) {
    for (int t = 0; t < kTileThreads; ++t) tile_interp<D, LM, 1>(t, g, P, W, c, lo, hi);
}

static void check_lowmem(long long& n, long long& bad) {
    const int nc = 32, nt = tile_count(nc, 5);
    Box<1> box(nc, 20, 4, 27);
    const int64_t nc3 = (int64_t)nc * nc * nc, np = box.n;
    std::vector<float> Fl(3 * nc3), green(kGreenPacked, 0.f), Td(256), vc(3 * nc3);
    for (auto& v : Fl) v = (float)((double)(next_u64() >> 11) * 0x1p-53 * 2.0 - 1.0);
    for (auto& v : vc) v = (float)((double)(next_u64() >> 11) * 0x1p-53 * 40.0 - 20.0);
    for (int i = 0; i < 256; ++i) Td[i] = (float)(std::tan(M_PI * ((i + 0.5) / 256.0 - 0.5)) * 0.25);
    std::vector<uint8_t> u[3];
    for (int e = 0; e < 3; ++e) {
        u[e].resize(np);
        for (auto& x : u[e]) x = (uint8_t)(next_u64() & 255);
    }
    std::vector<float> Pn(3 * np), Pn2(3 * np);
    std::vector<int32_t> Qn(3 * np), cnew(nc3), cnew2(nc3);
    std::vector<unsigned long long> S(3 * nc3), S2(3 * nc3);
    const float sigma = 2.0f, kd[2] = {0.75f, 3.3f};
    uint32_t errw = 0;
    TileParams P{};
    P.nc = nc;
    P.nt = nt;
    P.n = np;
    P.counts = box.counts.data();
    P.offsets = box.offsets.data();
    P.m0 = box.s[0].data();
    P.m1 = box.s[1].data();
    P.m2 = box.s[2].data();
    P.u0 = u[0].data();
    P.u1 = u[1].data();
    P.u2 = u[2].data();
    P.vc = vc.data();
    P.sigma = &sigma;
    P.Tdec = Td.data();
    P.green = green.data();
    P.Fl = Fl.data();
    P.kd = kd;
    P.mode = 1;
    P.err = &errw;
    std::vector<unsigned char> smem(kTileSmemBytes);
    unsigned char* base = smem.data();
    uint32_t* R = reinterpret_cast<uint32_t*>(base);
    float2* W = reinterpret_cast<float2*>(base + (size_t)kTileR * 4);
    float* Wf = reinterpret_cast<float*>(W);
    float* gS = reinterpret_cast<float*>(base + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    // one tile body, the force fields drawn from seed
    auto run = [&](const TileGeom& g, bool lm, unsigned long long seed, unsigned long long& lo,
                   unsigned long long& hi) {
        const TileCells c = tile_cells(W, O);
        for (int t = 0; t < kTileThreads; ++t) tile_prologue(t, g, P, c, R, gS);
        for (int t = 0; t < kTileThreads; ++t) tile_cells_scan(t, g, c);
        for (int t = 0; t < kTileThreads; ++t) tile_cells_map(t, g, c);
        for (int t = 0; t < kTileThreads; ++t) tile_deposit_flat<1>(t, g, P, R, c);
        const unsigned long long saved = rng_state;
        rng_state = seed;
        for (int D = 0; D < 3; ++D) {
            std::fill(Wf, Wf + 2 * kTileW, NAN);
            for (int zo = 0; zo < g.T[2] + 2; ++zo)
                for (int yo = 0; yo < g.T[1] + 2; ++yo)
                    for (int xo = 0; xo < g.T[0] + 2; ++xo)
                        Wf[wfidx(xo, yo, zo)] = (float)((double)(next_u64() >> 11) * 0x1p-53 * 2e3 - 1e3);
            if (D == 0) lm ? run_interp_lm<0, true>(g, P, W, c, lo, hi) : run_interp_lm<0, false>(g, P, W, c, lo, hi);
            if (D == 1) lm ? run_interp_lm<1, true>(g, P, W, c, lo, hi) : run_interp_lm<1, false>(g, P, W, c, lo, hi);
            if (D == 2) lm ? run_interp_lm<2, true>(g, P, W, c, lo, hi) : run_interp_lm<2, false>(g, P, W, c, lo, hi);
        }
        rng_state = saved;
    };
    const int tiles[3][3] = {{4, 0, 5}, {0, 3, 1}, {nt - 1, nt - 1, 0}};
    for (const auto& tt : tiles) {
        const TileGeom g = tile_geom(tt[0] + nt * (tt[1] + nt * tt[2]), nc, nt);
        const unsigned long long seed = next_u64() | 1ull;
        unsigned long long lo = 0, hi = 0, lo2 = 0, hi2 = 0;
        // default pass: new codes, momenta and fused sums
        P.Qn = Qn.data();
        P.Pn = Pn.data();
        P.counts_new = cnew.data();
        P.S = S.data();
        std::fill(cnew.begin(), cnew.end(), 0);
        std::fill(S.begin(), S.end(), 0ull);
        run(g, false, seed, lo, hi);
        // low-memory pass: momenta and the same sums, no codes
        P.Qn = nullptr;
        P.Pn = Pn2.data();
        P.counts_new = cnew2.data();
        P.S = S2.data();
        std::fill(cnew2.begin(), cnew2.end(), 0);
        std::fill(S2.begin(), S2.end(), 0ull);
        run(g, true, seed, lo2, hi2);
        for (int64_t i = 0; i < nc3; ++i) {
            ++n;
            bad += cnew2[i] != cnew[i] || S2[i] != S[i] || S2[nc3 + i] != S[nc3 + i] || S2[2 * nc3 + i] != S[2 * nc3 + i];
        }
        // the tile's own particles
        std::vector<int64_t> own;
        std::vector<int> own_cell;
        for (int z = g.c0[2]; z < g.c1[2]; ++z)
            for (int y = g.c0[1]; y < g.c1[1]; ++y)
                for (int x = g.c0[0]; x < g.c1[0]; ++x) {
                    const int cell = x + nc * (y + nc * z);
                    for (int64_t j = box.offsets[cell]; j < box.offsets[cell + 1]; ++j) {
                        own.push_back(j);
                        own_cell.push_back(cell);
                    }
                }
        int moved = 0;
        for (size_t k = 0; k < own.size(); ++k) {
            const int64_t j = own[k];
            const int cc[3] = {own_cell[k] % nc, (own_cell[k] / nc) % nc, own_cell[k] / (nc * nc)};
            for (int d = 0; d < 3; ++d) {
                ++n;
                const float p = Pn2[d * np + j];
                bad += std::memcmp(&p, &Pn[d * np + j], 4) != 0;
                const int q = drift_code(cc[d] * 256 + box.s[d][j], p, kd[1], nc * 256, &errw);
                ++n;
                bad += q != Qn[d * np + j];
                moved += q / 256 != cc[d];
            }
        }
        ++n;
        bad += moved == 0;   // some particles change cell, so the check covers the wrap too
        // the second moment T = sum P^2 of the new momenta (P = round(p 2^24)),
        // the same from both passes and equal to the exact sum
        unsigned __int128 ref = 0;
        for (int64_t j : own)
            for (int d = 0; d < 3; ++d) {
                const long long fx = fix24_rn(Pn[d * np + j]);
                const unsigned __int128 v = (unsigned __int128)(fx < 0 ? -fx : fx);
                ref += v * v;
            }
        ++n;
        bad += lo != (unsigned long long)ref || hi != (unsigned long long)(ref >> 64);
        ++n;
        bad += lo2 != lo || hi2 != hi;
        if (&tt == &tiles[0]) {   // the crowded tile's sum passes 2^64
            ++n;
            bad += hi == 0;
        }
    }
    ++n;
    bad += errw != 0u;
}

// Error path of the tile body that real inputs rarely reach: a fine node
// whose weight passes 2^32 - 1 units (over 2048 particles on one node).  The
// checked deposit path, taken when a cell holds more than 255 particles,
// flags kErrFineOverflow; the long-range force of every own particle (70,400
// of them) is still parked in its slot and no other slot is written.
static void check_error_paths(long long& n, long long& bad) {
    const int nc = 16, nt = tile_count(nc, 5);
    const int64_t nc3 = (int64_t)nc * nc * nc;
    std::vector<int32_t> counts(nc3, 0);
    std::vector<int64_t> offsets(nc3 + 1);
    // tile 0 owns cells 0..3 per axis: 64 cells of 1100 particles; cell
    // (1,1,1) holds 2,600 particles in one bin, whose nodes pass 2^32 units;
    // one cell outside the tile holds 10 particles
    for (int z = 0; z < 4; ++z)
        for (int y = 0; y < 4; ++y)
            for (int x = 0; x < 4; ++x) counts[x + nc * (y + nc * z)] = 1100;
    counts[1 + nc * (1 + nc)] = 2600;
    counts[8 + nc * (8 + nc * 8)] = 10;
    int64_t np = 0;
    for (int64_t i = 0; i < nc3; ++i) {
        offsets[i] = np;
        np += counts[i];
    }
    offsets[nc3] = np;
    std::vector<uint8_t> m[3];
    for (int e = 0; e < 3; ++e) {
        m[e].resize(np);
        for (int64_t j = 0; j < np; ++j) m[e][j] = (uint8_t)(next_u64() & 255);
        for (int64_t j = offsets[1 + nc * (1 + nc)]; j < offsets[2 + nc * (1 + nc)]; ++j) m[e][j] = 100;
    }
    std::vector<float> Fl(3 * nc3, 0.5f), green(kGreenPacked, 0.f), Td(256, 0.f);
    const float sigma = 1.f, kd[2] = {0.f, 0.f};
    std::vector<float> Pn(3 * (size_t)np, -7.f);
    uint32_t errw = 0;
    TileParams P{};
    P.nc = nc;
    P.nt = nt;
    P.n = np;
    P.counts = counts.data();
    P.offsets = offsets.data();
    P.m0 = m[0].data();
    P.m1 = m[1].data();
    P.m2 = m[2].data();
    P.Fl = Fl.data();
    P.green = green.data();
    P.Tdec = Td.data();
    P.sigma = &sigma;
    P.kd = kd;
    P.mode = 1;
    P.Pn = Pn.data();
    P.err = &errw;
    std::vector<unsigned char> smem(kTileSmemBytes);
    unsigned char* base = smem.data();
    uint32_t* R = reinterpret_cast<uint32_t*>(base);
    float2* W = reinterpret_cast<float2*>(base + (size_t)kTileR * 4);
    float* gS = reinterpret_cast<float*>(base + (size_t)kTileR * 4 + (size_t)kTileW * 8);
    int* O = reinterpret_cast<int*>(gS + kGreenPacked);
    const TileGeom g = tile_geom(0, nc, nt);
    const TileCells c = tile_cells(W, O);
    for (int t = 0; t < kTileThreads; ++t) tile_prologue(t, g, P, c, R, gS);
    for (int t = 0; t < kTileThreads; ++t) tile_cells_scan(t, g, c);
    for (int t = 0; t < kTileThreads; ++t) tile_cells_map(t, g, c);
    for (int t = 0; t < kTileThreads; ++t) tile_deposit_flat<1>(t, g, P, R, c);
    ++n;
    bad += c.ppre[kOwnMax] != 64 * 1100 + 1500 || c.misc[2] <= 255;   // the case is what it claims
    ++n;
    bad += (errw & kErrFineOverflow) == 0u;
    // parked forces: every own slot of each component holds F_l = 0.5
    // (gathered from a constant field), the outside cell's slots untouched
    const int64_t own_end = offsets[nc3] - 10;
    for (int e = 0; e < 3; ++e) {
        for (int64_t j = 0; j < own_end; j += 97) {
            ++n;
            bad += std::fabs(Pn[(size_t)e * np + j] - 0.5f) > 1e-6f;
        }
        for (int64_t j = own_end; j < np; ++j) {
            ++n;
            bad += Pn[(size_t)e * np + j] != -7.f;
        }
    }
}

int main() {
    check_swizzles();
    check_tiling();
    check_no_alias();
    check_own_cells();
    check_smem_layout();
    run_prologue_checks();
    {
        long long n = 0, bad = 0;
        double err = 0.0;
        check_deposit<1>(n, bad, err);
        check_deposit<2>(n, bad, err);
        printf("deposit %lld %lld %.3e\n", n, bad, err);
    }
    check_spectral();
    for (int mode = 0; mode <= 1; ++mode) {
        long long n = 0, bad = 0;
        double err = 0.0;
        check_interp<1>(n, bad, err, mode);
        check_interp<2>(n, bad, err, mode);
        printf("interp_mode%d %lld %lld %.3e\n", mode, n, bad, err);
    }
    {
        long long n = 0, bad = 0;
        check_lowmem(n, bad);
        printf("lowmem %lld %lld\n", n, bad);
    }
    {
        long long n = 0, bad = 0;
        check_error_paths(n, bad);
        printf("error_paths %lld %lld\n", n, bad);
    }
    return 0;
}
