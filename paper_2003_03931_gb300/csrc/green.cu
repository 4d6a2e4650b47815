// green.cu -- the force kernels of the PM-PM split (Sec. II, Eq. 1), built
// once per sim on the device in float64.
//
// Sec. II: F_G = F_s + F_l with F_s(r >= r_cut) = 0 and F_l(r >= r_cut) =
// F_G(r).  In a periodic box F_G is the periodic pair force (a unit mass, its
// images and the removed mean), evaluated here by the Ewald split: screened
// real-space images plus a Gaussian-damped Fourier sum.
//
//  * Long-range kernel K_l: the periodic force at coarse separations 4D.  Its
//    DFT on the coarse mesh is the Fourier part taken exactly (it is band
//    limited to |h| < nc/2) plus the FFT of the real-space part.  Stored as
//    S_l(a, b, c) = -Im K~_l^x at |kx| = a, |ky| = b, |kz| = c, a, b, c in
//    [0, nc/2]; the y and z kernels follow by axis permutation.
//  * Matching A(d): coarse-mesh force between fine-cell centres a fine
//    separation d apart, averaged over the 64 centres of a coarse cell.
//  * Short-range kernel K_s(d) = K_per(d) - A(d) for 0 < |d| < 6, and its
//    32^3 DFT stored the same way in a 17^3 table.
#include "pmpm_impl.cuh"

namespace pmpm {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kEwaldKExp = 38.0;   // exp(-k^2 / 4 alpha^2) < e^-38 beyond the cutoff
constexpr double kEwaldRCut = 6.5;    // alpha r beyond which the real-space term is dropped

struct Ewald {
    double L, alpha, rs;
    int n_img, h_max;
};

__host__ __device__ Ewald make_ewald(double L, int h_max) {
    Ewald e;
    e.L = L;
    e.h_max = h_max;
    e.alpha = (2.0 * kPi * h_max / L) / (2.0 * sqrt(kEwaldKExp));
    e.rs = kEwaldRCut / e.alpha;
    e.n_img = (int)ceil(e.rs / L + 0.5);
    return e;
}

// real-space screened sum over images within rs; skips the self term
__device__ void ewald_real(const Ewald& e, double x, double y, double z, double out[3]) {
    const double two_over_sqrt_pi = 1.1283791670955126;
    for (int nz = -e.n_img; nz <= e.n_img; ++nz)
        for (int ny = -e.n_img; ny <= e.n_img; ++ny)
            for (int nx = -e.n_img; nx <= e.n_img; ++nx) {
                const double rx = x + nx * e.L, ry = y + ny * e.L, rz = z + nz * e.L;
                const double r2 = rx * rx + ry * ry + rz * rz;
                if (r2 == 0.0 || r2 > e.rs * e.rs) continue;
                const double r = sqrt(r2);
                const double ar = e.alpha * r;
                const double screen = erfc(ar) + two_over_sqrt_pi * ar * exp(-ar * ar);
                const double f = screen / (r2 * r);
                out[0] -= rx * f;
                out[1] -= ry * f;
                out[2] -= rz * f;
            }
}

// Fourier sum over |h| <= h_max, h != 0
__device__ void ewald_fourier(const Ewald& e, double x, double y, double z, double out[3]) {
    const double pref = 4.0 * kPi / (e.L * e.L * e.L);
    const double kf = 2.0 * kPi / e.L;
    const int H = e.h_max;
    for (int hz = -H; hz <= H; ++hz)
        for (int hy = -H; hy <= H; ++hy)
            for (int hx = -H; hx <= H; ++hx) {
                const int h2 = hx * hx + hy * hy + hz * hz;
                if (h2 == 0 || h2 > H * H) continue;
                const double kx = kf * hx, ky = kf * hy, kz = kf * hz;
                const double k2 = kx * kx + ky * ky + kz * kz;
                const double c = pref * exp(-k2 / (4.0 * e.alpha * e.alpha)) / k2 *
                                 sin(kx * x + ky * y + kz * z);
                out[0] -= c * kx;
                out[1] -= c * ky;
                out[2] -= c * kz;
            }
}

__device__ void ewald_force(const Ewald& e, double x, double y, double z, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (x == 0.0 && y == 0.0 && z == 0.0) return;
    ewald_real(e, x, y, z, out);
    ewald_fourier(e, x, y, z, out);
}

// The x component of the same force, evaluated by one warp: lane l takes the
// images and Fourier vectors with flat index l, l + 32, ...; the lane sums
// are combined in a fixed order (every lane returns the total).
__device__ double ewald_force_x_warp(const Ewald& e, double x, double y, double z, int lane) {
    double fx = 0.0;
    if (!(x == 0.0 && y == 0.0 && z == 0.0)) {
        const double two_over_sqrt_pi = 1.1283791670955126;
        const int ni = 2 * e.n_img + 1;
        for (int t = lane; t < ni * ni * ni; t += 32) {
            const int nx = t % ni - e.n_img, ny = (t / ni) % ni - e.n_img, nz = t / (ni * ni) - e.n_img;
            const double rx = x + nx * e.L, ry = y + ny * e.L, rz = z + nz * e.L;
            const double r2 = rx * rx + ry * ry + rz * rz;
            if (r2 == 0.0 || r2 > e.rs * e.rs) continue;
            const double r = sqrt(r2);
            const double ar = e.alpha * r;
            const double screen = erfc(ar) + two_over_sqrt_pi * ar * exp(-ar * ar);
            fx -= rx * screen / (r2 * r);
        }
        const double pref = 4.0 * kPi / (e.L * e.L * e.L);
        const double kf = 2.0 * kPi / e.L;
        const int H = e.h_max, nh = 2 * H + 1;
        for (int t = lane; t < nh * nh * nh; t += 32) {
            const int hx = t % nh - H, hy = (t / nh) % nh - H, hz = t / (nh * nh) - H;
            const int h2 = hx * hx + hy * hy + hz * hz;
            if (h2 == 0 || h2 > H * H) continue;
            const double kx = kf * hx, ky = kf * hy, kz = kf * hz;
            const double k2 = kx * kx + ky * ky + kz * kz;
            fx -= pref * exp(-k2 / (4.0 * e.alpha * e.alpha)) / k2 * sin(kx * x + ky * y + kz * z) * kx;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fx += __shfl_xor_sync(0xffffffffu, fx, o);
    return fx;
}

// x-component of the coarse kernel at coarse offsets D in [-3, 3]^3
// one warp per entry
__global__ void k_coarse_small(double L, double* Tsmall) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= 343) return;
    const int Dx = i % 7 - 3, Dy = (i / 7) % 7 - 3, Dz = i / 49 - 3;
    const Ewald e = make_ewald(L, 8);
    const double fx = ewald_force_x_warp(e, 4.0 * Dx, 4.0 * Dy, 4.0 * Dz, lane);
    if (lane == 0) Tsmall[i] = fx;
}

// coarse CIC weights of a point at pos (fine units, relative to the left edge
// of coarse cell 0), nodes at 4a + 2
__device__ void cw1(double pos, int& a0, double& w0, double& w1) {
    const double t = (pos - 2.0) / 4.0;
    a0 = (int)floor(t);
    w1 = t - a0;
    w0 = 1.0 - w1;
}

// K_s^x(d) = K_per^x(d) - A^x(d) over d in [-5, 5]^3 (zero off the support);
// one warp per entry, the lanes splitting the Ewald sum and the 64 centres
__global__ void k_fine_values(double L, const double* Tsmall, double* Ks) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= 1331) return;
    const int dx = i % 11 - 5, dy = (i / 11) % 11 - 5, dz = i / 121 - 5;
    const int r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0 || r2 >= kBuffer * kBuffer) {
        if (lane == 0) Ks[i] = 0.0;
        return;
    }
    const Ewald e = make_ewald(L, 8);
    const double fx = ewald_force_x_warp(e, dx, dy, dz, lane);
    // A^x(d): average over the 64 fine-cell centres s of one coarse cell
    double A = 0.0;
    for (int s = lane; s < 64; s += 32) {
        const double sx = (s & 3) + 0.5, sy = ((s >> 2) & 3) + 0.5, sz = (s >> 4) + 0.5;
        int a0[3], b0[3];
        double aw[3][2], bw[3][2];
        cw1(sx, a0[0], aw[0][0], aw[0][1]);
        cw1(sy, a0[1], aw[1][0], aw[1][1]);
        cw1(sz, a0[2], aw[2][0], aw[2][1]);
        cw1(sx + dx, b0[0], bw[0][0], bw[0][1]);
        cw1(sy + dy, b0[1], bw[1][0], bw[1][1]);
        cw1(sz + dz, b0[2], bw[2][0], bw[2][1]);
        for (int ca = 0; ca < 8; ++ca) {
            const int ax = ca & 1, ay = (ca >> 1) & 1, az = ca >> 2;
            const double wa = aw[0][ax] * aw[1][ay] * aw[2][az];
            for (int cb = 0; cb < 8; ++cb) {
                const int bx = cb & 1, by = (cb >> 1) & 1, bz = cb >> 2;
                const double wb = bw[0][bx] * bw[1][by] * bw[2][bz];
                const int Dx = b0[0] + bx - a0[0] - ax, Dy = b0[1] + by - a0[1] - ay,
                          Dz = b0[2] + bz - a0[2] - az;
                A += wa * wb * Tsmall[(Dx + 3) + 7 * ((Dy + 3) + 7 * (Dz + 3))];
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) A += __shfl_xor_sync(0xffffffffu, A, o);
    if (lane == 0) Ks[i] = fx - A / 64.0;
}

// S_s(a, b, c) = sum_d K_s^x(d) sin(2 pi a dx/32) cos(2 pi b dy/32) cos(2 pi c dz/32),
// times 2^-21 (density units) and 2^-15 (unnormalised inverse 32^3 DFT)
// one warp per entry, the lanes splitting the 1331 separations
__global__ void k_fine_table(const double* Ks, float* table) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= kGreenS * kGreenS * kGreenS) return;
    const int a = i / (kGreenS * kGreenS), b = (i / kGreenS) % kGreenS, c = i % kGreenS;
    if (a == 0 || a == 16) {
        if (lane == 0) table[i] = 0.f;   // odd in its own axis: zero at k = 0 and at Nyquist
        return;
    }
    double acc = 0.0;
    for (int j = lane; j < 1331; j += 32) {
        const double k = Ks[j];
        if (k == 0.0) continue;
        const int dx = j % 11 - 5, dy = (j / 11) % 11 - 5, dz = j / 121 - 5;
        acc += k * sinpi((double)(2 * a * dx) / 32.0) * cospi((double)(2 * b * dy) / 32.0) *
               cospi((double)(2 * c * dz) / 32.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) table[i] = (float)(acc * 0x1p-36);
}

// b <= c half of the 17^3 table for own-axis rows a = 1..15 (rows 0 and 16
// vanish), row-major over (a - 1, b, c = b..16)
__global__ void k_pack_fine(const float* table, float* packed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int tri = kGreenS * (kGreenS + 1) / 2;
    if (i >= (kGreenS - 2) * tri) return;
    const int a = 1 + i / tri;
    int r = i % tri, b = 0;
    while (r >= kGreenS - b) { r -= kGreenS - b; ++b; }
    packed[i] = table[(a * kGreenS + b) * kGreenS + (b + r)];
}

// real-space part of the coarse kernel (x component) on the whole mesh,
// nearest image of D plus further images within rs
__global__ void k_coarse_real(int nc, Ewald e, double2* out) {
    const int64_t ncells = (int64_t)nc * nc * nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nc), iy = (int)((i / nc) % nc), iz = (int)(i / ((int64_t)nc * nc));
        const int Dx = ix < nc / 2 ? ix : ix - nc, Dy = iy < nc / 2 ? iy : iy - nc,
                  Dz = iz < nc / 2 ? iz : iz - nc;
        double f[3] = {0.0, 0.0, 0.0};
        const double x = 4.0 * Dx, y = 4.0 * Dy, z = 4.0 * Dz;
        // the nearest image is at least |x| away; skip points that no image reaches
        const double r2min = x * x + y * y + z * z;
        if (e.n_img > 1 || r2min <= e.rs * e.rs) ewald_real(e, x, y, z, f);
        out[i] = make_double2(f[0], 0.0);
    }
}

// S_l octant from the FFT of the real-space part plus the exact Fourier part,
// scaled by 2^-27 (density units) and 1/nc^3 (unnormalised inverse DFT)
__global__ void k_coarse_table(int nc, Ewald e, const double2* X, float* table) {
    const int h = nc / 2 + 1;
    const int64_t total = (int64_t)h * h * h;
    const double kf = 2.0 * kPi / e.L;
    const double pref = 4.0 * kPi / (e.L * e.L * e.L) * (double)nc * nc * nc;
    const double scale = 0x1p-27 / ((double)nc * nc * nc);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i / ((int64_t)h * h)), b = (int)((i / h) % h), c = (int)(i % h);
        const double2 v = X[(int64_t)a + nc * ((int64_t)b + (int64_t)nc * c)];
        double S = -v.y;
        const int h2 = a * a + b * b + c * c;
        if (h2 > 0 && h2 <= e.h_max * e.h_max) {
            const double kx = kf * a, k2 = kf * kf * h2;
            S -= pref * kx / k2 * exp(-k2 / (4.0 * e.alpha * e.alpha));
        }
        if (a == 0 || 2 * a == nc) S = 0.0;   // odd in its own axis
        table[i] = (float)(S * scale);
    }
}

// The three components' coarse kernels per folded wavenumber, gathered for
// the Green multiply: G[(az h + ay) h + ax] = (S(ax; ay, az), S(ay; ax, az),
// S(az; ay, ax), 0) from the own-axis-first table T[(a h + b) h + c] =
// S(a; b, c), so that a pass over the mesh (kx fastest) reads G in order.
__global__ void k_coarse_table4(int nc, const float* __restrict__ T, float4* __restrict__ G) {
    const int64_t h = nc / 2 + 1;
    const int64_t total = h * h * h;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t az = i / (h * h), ay = (i / h) % h, ax = i % h;
        G[i] = make_float4(T[(ax * h + ay) * h + az], T[(ay * h + ax) * h + az], T[(az * h + ay) * h + ax],
                           0.f);
    }
}

}  // namespace

int build_green_tables(Sim& s) {
    const int nc = s.nc;
    const double L = 4.0 * nc;
    cudaStream_t st = s.stream;
    // scratch: Tsmall[343], Ks[1331], coarse mesh complex [nc^3] (float64),
    // then the own-axis-first coarse table [(nc/2+1)^3] (float32)
    double* Tsmall = reinterpret_cast<double*>(s.scratch);
    double* Ks = Tsmall + 343;
    double2* mesh = reinterpret_cast<double2*>(align_up(reinterpret_cast<uintptr_t>(Ks + 1331)));
    float* T1 = reinterpret_cast<float*>(mesh + (size_t)nc * nc * nc);
    k_coarse_small<<<(343 * 32 + 255) / 256, 256, 0, st>>>(L, Tsmall);
    k_fine_values<<<(1331 * 32 + 255) / 256, 256, 0, st>>>(L, Tsmall, Ks);
    k_fine_table<<<(kGreenS * kGreenS * kGreenS * 32 + 255) / 256, 256, 0, st>>>(Ks, s.green_fine);
    k_pack_fine<<<((kGreenS - 2) * kGreenS * (kGreenS + 1) / 2 + 255) / 256, 256, 0, st>>>(s.green_fine,
                                                                                   s.green_packed);
    const Ewald e = make_ewald(L, nc / 2 - 1);
    k_coarse_real<<<grid_for(s.ncells, 256), 256, 0, st>>>(nc, e, mesh);
    int rc = fft3d<double>(s, mesh, nc, -1);
    if (rc) return rc;
    const int64_t h = nc / 2 + 1;
    k_coarse_table<<<grid_for(h * h * h, 256), 256, 0, st>>>(nc, e, mesh, T1);
    k_coarse_table4<<<grid_for(h * h * h, 256), 256, 0, st>>>(nc, T1, s.green_coarse);
    return check_launch(s, "green tables");
}

size_t green_scratch_bytes(int nc) {
    const size_t h = (size_t)(nc / 2 + 1);
    return 343 * 8 + 1331 * 8 + 512 + (size_t)nc * nc * nc * 16 + 4 * h * h * h;
}

}  // namespace pmpm
