// abi.cu -- the C ABI of pmpm.h: workspace layout, set-up, the step sequence
// and the state transfers.
//
// One step (Sec. II, Sec. III):
//   0 coarse CIC deposit of the current store
//   1 coarse FFT, Green multiply (K~_l), two inverse FFTs -> F_l
//   2 tile pass: fine CIC + FFT + K~_s + inverse per tile; interpolate F_s +
//     F_l; kick; integer drift
//   3 new-cell counts and momentum sums, scan, cell means v_c
//   4 dispersion sigma
//   5 encode + scatter into the other store buffer; swap
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <new>

#include "pmpm_impl.cuh"
#include "cosmo.h"

namespace pmpm {

static char g_init_msg[512] = "";

int set_error(Sim& s, int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s.msg, sizeof(s.msg), fmt, ap);
    va_end(ap);
    return code;
}

int check_launch(Sim& s, const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return PMPM_OK;
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static int validate(const pmpm_config* c, char* msg, size_t len) {
    if (!c) return snprintf(msg, len, "null config"), PMPM_EINVAL;
    if (!pow2(c->np) || c->np < 4 || c->np > 4096)
        return snprintf(msg, len, "np=%d must be a power of two in [4, 4096]", c->np), PMPM_EINVAL;
    if (!pow2(c->nc) || c->nc < 8 || c->nc > 1024)
        return snprintf(msg, len, "nc=%d must be a power of two in [8, 1024]", c->nc), PMPM_EINVAL;
    if (c->tile_max != 4 && c->tile_max != 5)
        return snprintf(msg, len, "tile_max=%d must be 4 or 5", c->tile_max), PMPM_EINVAL;
    if (c->buffer != kBuffer)
        return snprintf(msg, len, "buffer=%d: only %d is supported", c->buffer, kBuffer), PMPM_EINVAL;
    if ((c->pos_bytes != 1 && c->pos_bytes != 2) || c->vel_bytes != 1)
        return snprintf(msg, len, "positions take 1 or 2 bytes, velocities 1 byte"), PMPM_EINVAL;
    if (c->pos_bytes == 2 && (c->flags & PMPM_FLAG_LOWMEM))
        return snprintf(msg, len, "the low-memory step stores 1-byte positions"), PMPM_EINVAL;
    const int nf = 4 * c->nc;
    if (c->pk_mesh_max && (!pow2(c->pk_mesh_max) || c->pk_mesh_max > nf || c->pk_mesh_max < 4))
        return snprintf(msg, len, "pk_mesh_max=%d must be a power of two <= %d", c->pk_mesh_max, nf),
               PMPM_EINVAL;
    if (!(c->a_init > 0.0) || !(c->a_final >= c->a_init) || c->n_steps < 1)
        return snprintf(msg, len, "need 0 < a_init <= a_final and n_steps >= 1"), PMPM_EINVAL;
    if (c->flags & ~(PMPM_FLAG_LOWMEM | PMPM_FLAG_FINE_FP16))
        return snprintf(msg, len, "unknown flags 0x%x", (unsigned)c->flags), PMPM_EINVAL;
    if ((c->flags & PMPM_FLAG_LOWMEM) && (c->flags & PMPM_FLAG_FINE_FP16))
        return snprintf(msg, len, "FP16 tile storage is an option of the default step"), PMPM_EINVAL;
    if (!(c->omega_m >= 0.0) || !(c->omega_l >= 0.0) || (c->omega_m == 0.0 && c->omega_l != 0.0))
        return snprintf(msg, len, "need omega_m > 0 and omega_l >= 0, or both 0 (Einstein-de Sitter)"),
               PMPM_EINVAL;
    if (c->omega_m > 0.0) {
        const Background b = background_of(c->omega_m, c->omega_l);
        for (int i = 0; i <= 64; ++i) {
            const double a = c->a_init * pow(c->a_final / c->a_init, i / 64.0);
            if (!(bg_E2(b, a) > 0.0))
                return snprintf(msg, len, "no expanding background at a = %g", a), PMPM_EINVAL;
        }
    }
    return PMPM_OK;
}

static void derive(Sim& s, const pmpm_config* c) {
    s.cfg = *c;
    s.np = c->np;
    s.nc = c->nc;
    s.nf = 4 * c->nc;
    s.n = (int64_t)c->np * c->np * c->np;
    s.ncells = (int64_t)c->nc * c->nc * c->nc;
    s.tile_max = c->tile_max;
    s.nt = tile_count(c->nc, c->tile_max);
    s.pk_max = c->pk_mesh_max ? c->pk_mesh_max : (s.nf < 512 ? s.nf : 512);
    s.fft_max = s.nc;
    if (s.np > s.fft_max) s.fft_max = s.np;
    if (s.pk_max > s.fft_max) s.fft_max = s.pk_max;
    s.nblocks_scan = (s.ncells + 4095) / 4096;
    s.lowmem = (c->flags & PMPM_FLAG_LOWMEM) != 0;
    s.fp16 = (c->flags & PMPM_FLAG_FINE_FP16) != 0;
    s.pb = c->pos_bytes == 2 ? 2 : 1;
    s.ic_pfac = c->a_init * bg_ic_momentum_factor(background_of(c->omega_m, c->omega_l), c->a_init);
}

// Low-memory layout (PMPM_FLAG_LOWMEM).  The new codes are never stored (the
// re-encode derives them from the old store and the new momenta), and the
// buffers of the different phases share space:
//   [small][P0: store 0, counts 0, offsets 0, v_c 0][P1: the same for 1][fill][U]
//   Store b's region, max(6N, 36C) bytes, also holds the momentum sums S and
//   F_l of a step whose next buffer is b (lowmem_bind): both are dead before
//   the re-encode writes the store.
//   U holds, at different times: the coarse mesh and spectra (coarse force),
//   the new momenta Pn (tile pass to re-encode), the float32 displacement
//   field (ICs), the power-spectrum mesh, the force-table scratch (init).
//   ICs: the transform work array (8N) starts at P0 (P0 + P1 >= 12N).
static size_t lowmem_sf_bytes(int64_t C) { return align_up(24 * (size_t)C) + 12 * (size_t)C; }

void lowmem_bind(Sim& s, int nxt) {
    uint8_t* r = s.streams[nxt];
    s.S = reinterpret_cast<unsigned long long*>(r);
    s.Fl = reinterpret_cast<float*>(r + align_up(24 * (size_t)s.ncells));
}

static size_t layout_lowmem(Sim& s, uint8_t* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> uint8_t* {
        off = align_up(off);
        uint8_t* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const int64_t N = s.n, C = s.ncells;
    // small persistent items
    const size_t h = s.nc / 2 + 1;
    s.green_coarse = reinterpret_cast<float4*>(take(16 * h * h * h));
    s.green_fine = reinterpret_cast<float*>(take(4 * (size_t)kGreenS * kGreenS * kGreenS));
    s.green_packed = reinterpret_cast<float*>(take(4 * (size_t)kGreenS * kGreenS * (kGreenS + 1) / 2));
    s.Tdec = reinterpret_cast<float*>(take(4 * 256));
    s.Eedge = reinterpret_cast<float*>(take(4 * 256));
    s.tw_f = reinterpret_cast<float2*>(take(8 * (size_t)s.fft_max));
    s.tw_d = reinterpret_cast<double2*>(take(16 * (size_t)s.fft_max));
    s.err = reinterpret_cast<uint32_t*>(take(4));
    s.blocksums = reinterpret_cast<long long*>(take(8 * (size_t)(s.nblocks_scan + 1)));
    s.ic_partial = reinterpret_cast<double*>(take(8 * (3 * 1024 + 1)));
    s.pk_bins = reinterpret_cast<double*>(take(8 * 3 * (size_t)(s.pk_max / 2 + 1)));
    s.d_factors = reinterpret_cast<float*>(take(8 * (size_t)s.cfg.n_steps));
    s.d_step = reinterpret_cast<int*>(take(4));
    s.d_kd = reinterpret_cast<float*>(take(8));
    s.d2 = reinterpret_cast<unsigned long long*>(take(64));
    for (int b = 0; b < 2; ++b) s.sigma_d[b] = reinterpret_cast<float*>(take(4));
    off = align_up(off);
    const size_t p0 = off;
    // P0, P1 (low-memory sims store 1-byte positions)
    size_t store_b = 6 * (size_t)N;
    if (lowmem_sf_bytes(C) > store_b) store_b = lowmem_sf_bytes(C);
    for (int b = 0; b < 2; ++b) {
        s.streams[b] = take(store_b);
        s.counts[b] = reinterpret_cast<int32_t*>(take(4 * (size_t)C));
        s.offsets[b] = reinterpret_cast<int64_t*>(take(8 * (size_t)(C + 1)));
        s.vc[b] = reinterpret_cast<float*>(take(12 * (size_t)C));
    }
    s.fill = reinterpret_cast<int32_t*>(take(4 * (size_t)C));
    off = align_up(off);
    // U
    const size_t u0 = off;
    const size_t coarse_b = 4 * align_up(8 * (size_t)C);
    const size_t pk3 = (size_t)s.pk_max * s.pk_max * s.pk_max;
    const size_t pk_b = 16 * pk3 + 512;
    const size_t green_b = green_scratch_bytes(s.nc);
    size_t ub = 12 * (size_t)N;
    if (coarse_b > ub) ub = coarse_b;
    if (pk_b > ub) ub = pk_b;
    if (green_b > ub) ub = green_b;
    if (base) {
        uint8_t* u = base + u0;
        s.rho_c = reinterpret_cast<long long*>(u);
        s.cA = reinterpret_cast<float2*>(u + align_up(8 * (size_t)C));
        s.cB1 = reinterpret_cast<float2*>(u + 2 * align_up(8 * (size_t)C));
        s.cB2 = reinterpret_cast<float2*>(u + 3 * align_up(8 * (size_t)C));
        s.scratch = u;
        s.Pn = reinterpret_cast<float*>(u);
        s.ic_psi = reinterpret_cast<float*>(u);
        s.ic_work = reinterpret_cast<float2*>(base + p0);
        lowmem_bind(s, 1);
    }
    s.scratch_bytes = ub;
    s.Qn = nullptr;
    off = u0 + ub;
    return align_up(off);
}

size_t layout(Sim& s, uint8_t* base) {
    if (s.lowmem) return layout_lowmem(s, base);
    size_t off = 0;
    auto take = [&](size_t bytes) -> uint8_t* {
        off = align_up(off);
        uint8_t* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const int64_t N = s.n, C = s.ncells;
    for (int b = 0; b < 2; ++b) {
        s.streams[b] = take((size_t)(3 * s.pb + 3) * N);
        s.counts[b] = reinterpret_cast<int32_t*>(take(4 * (size_t)C));
        s.offsets[b] = reinterpret_cast<int64_t*>(take(8 * (size_t)(C + 1)));
        s.vc[b] = reinterpret_cast<float*>(take(12 * (size_t)C));
        s.sigma_d[b] = reinterpret_cast<float*>(take(4));
    }
    s.fill = reinterpret_cast<int32_t*>(take(4 * (size_t)C));
    s.S = reinterpret_cast<unsigned long long*>(take(24 * (size_t)C));
    s.d2 = reinterpret_cast<unsigned long long*>(take(64));
    s.rho_c = reinterpret_cast<long long*>(take(8 * (size_t)C));
    s.cA = reinterpret_cast<float2*>(take(8 * (size_t)C));
    s.cB1 = reinterpret_cast<float2*>(take(8 * (size_t)C));
    s.cB2 = reinterpret_cast<float2*>(take(8 * (size_t)C));
    s.Fl = reinterpret_cast<float*>(take(12 * (size_t)C));
    const size_t h = s.nc / 2 + 1;
    s.green_coarse = reinterpret_cast<float4*>(take(16 * h * h * h));
    s.green_fine = reinterpret_cast<float*>(take(4 * (size_t)kGreenS * kGreenS * kGreenS));
    s.green_packed = reinterpret_cast<float*>(take(4 * (size_t)kGreenS * kGreenS * (kGreenS + 1) / 2));
    s.Tdec = reinterpret_cast<float*>(take(4 * 256));
    s.Eedge = reinterpret_cast<float*>(take(4 * 256));
    s.tw_f = reinterpret_cast<float2*>(take(8 * (size_t)s.fft_max));
    s.tw_d = reinterpret_cast<double2*>(take(16 * (size_t)s.fft_max));
    s.err = reinterpret_cast<uint32_t*>(take(4));
    s.blocksums = reinterpret_cast<long long*>(take(8 * (size_t)(s.nblocks_scan + 1)));
    s.ic_partial = reinterpret_cast<double*>(take(8 * (3 * 1024 + 1)));
    s.pk_bins = reinterpret_cast<double*>(take(8 * 3 * (size_t)(s.pk_max / 2 + 1)));
    s.d_factors = reinterpret_cast<float*>(take(8 * (size_t)s.cfg.n_steps));
    s.d_step = reinterpret_cast<int*>(take(4));
    s.d_kd = reinterpret_cast<float*>(take(8));
    // transient scratch
    const size_t step_b = 24 * (size_t)N + 512;
    const size_t ic_b = 56 * (size_t)N + 1024;
    const size_t green_b = green_scratch_bytes(s.nc);
    const size_t pk3 = (size_t)s.pk_max * s.pk_max * s.pk_max;
    const size_t pk_b = 16 * pk3 + 512;
    size_t sb = step_b;
    if (ic_b > sb) sb = ic_b;
    if (green_b > sb) sb = green_b;
    if (pk_b > sb) sb = pk_b;
    s.scratch_bytes = sb;
    s.scratch = take(sb);
    if (base) {
        s.Qn = reinterpret_cast<int32_t*>(s.scratch);
        s.Pn = reinterpret_cast<float*>(align_up(reinterpret_cast<uintptr_t>(s.Qn + 3 * N)));
    }
    return align_up(off);
}

void prof_mark(Sim& s, int stage) {
    if (!s.prof || !s.in_step) return;
    if (s.ev_count >= kEventRing) return;   // full: further marks are dropped until read
    cudaEventRecord(s.ev[s.ev_count], s.stream);
    s.ev_stage[s.ev_count] = stage;
    s.ev_count++;
}

static void prof_fold(Sim& s) {
    if (s.ev_count == 0) return;
    cudaEventSynchronize(s.ev[s.ev_count - 1]);
    for (int i = 1; i < s.ev_count; ++i) {
        const int st = s.ev_stage[i];
        if (st < 0 || st >= kStages) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s.ev[i - 1], s.ev[i]) == cudaSuccess) s.stage_ms[st] += ms;
    }
    s.ev_count = 0;
}

// host-side float64 tables of Eq. 3: bin centres T[u] and edges E[k]
static void codec_tables(float* T, float* E) {
    const double pi = 3.141592653589793238462643383279502884;
    for (int u = 0; u < 256; ++u) T[u] = (float)tan(pi * ((u + 0.5) / 256.0 - 0.5));
    E[0] = -INFINITY;
    for (int k = 1; k < 256; ++k) E[k] = (float)tan(pi * (k / 256.0 - 0.5));
}

__global__ void k_twiddles(int n, float2* tf, double2* td) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double sv, cv;
        sincospi(2.0 * (double)k / (double)n, &sv, &cv);
        td[k] = make_double2(cv, -sv);
        tf[k] = make_float2((float)cv, (float)-sv);
    }
}

static int sync_and_check(Sim& s) {
    cudaError_t e = cudaStreamSynchronize(s.stream);
    if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "stream: %s", cudaGetErrorString(e));
    uint32_t flags = 0;
    e = cudaMemcpyAsync(&flags, s.err, 4, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
    if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "error word: %s", cudaGetErrorString(e));
    if (flags) {
        cudaMemsetAsync(s.err, 0, 4, s.stream);
        cudaStreamSynchronize(s.stream);
        if (flags & kErrLoadCounts)
            return set_error(s, PMPM_EINVAL, "loaded counts negative or not adding up to N");
        if (flags & kErrCount) return set_error(s, PMPM_ECOUNT, "particle count not conserved");
        return set_error(s, PMPM_EOVERFLOW,
                         "device range check failed (flags 0x%x: 1 fine density, 2 momentum, "
                         "16 non-finite, 32 drift)", flags);
    }
    return PMPM_OK;
}

static double sched_a(const Sim& s, int64_t n) {
    return s.cfg.a_init * pow(s.cfg.a_final / s.cfg.a_init, (double)n / (double)s.cfg.n_steps);
}

// The device step counter and the kick/drift factors of that step, which
// the tile pass reads (one pair per step, so a captured step replays as is).
__global__ void k_step_set(int* step, float* kd, const float* factors, int n_steps, int v) {
    *step = v;
    kd[0] = v < n_steps ? factors[2 * v] : 0.f;
    kd[1] = v < n_steps ? factors[2 * v + 1] : 0.f;
}
__global__ void k_step_advance(int* step, float* kd, const float* factors, int n_steps) {
    const int v = *step + 1;
    *step = v;
    kd[0] = v < n_steps ? factors[2 * v] : 0.f;
    kd[1] = v < n_steps ? factors[2 * v + 1] : 0.f;
}

static double cfg_a(const pmpm_config& c, int64_t n) {
    return c.a_init * pow(c.a_final / c.a_init, (double)n / (double)c.n_steps);
}

// float64 kick factor (multiplies g) and drift factor (multiplies p, fine
// cells) of step n: momenta at the half steps a_{n+1/2} = sqrt(a_n a_{n+1}),
// the first kick from a_0; the integrals of the background (cosmo.h)
static void step_factors(const pmpm_config& c, int64_t np3, int n, double* kick, double* drift) {
    const Background b = background_of(c.omega_m, c.omega_l);
    const double nf = 4.0 * c.nc;
    const double rho_bar = (double)np3 / (nf * nf * nf);
    const double an = cfg_a(c, n), an1 = cfg_a(c, n + 1);
    const double a_lo = n == 0 ? c.a_init : sqrt(cfg_a(c, n - 1) * an);
    const double a_hi = sqrt(an * an1);
    *kick = 3.0 * b.om / (8.0 * 3.141592653589793238462643383279502884 * rho_bar) *
            bg_kick_integral(b, a_lo, a_hi);
    *drift = bg_drift_integral(b, an, an1);
}

// float32 kick and drift factors of every step of the schedule (R7), in
// device memory so that a captured step can replay at any step index
static void fill_factors(Sim& s) {
    const int S = s.cfg.n_steps;
    float* f = new float[2 * S];
    for (int n = 0; n < S; ++n) {
        double kick, drift;
        step_factors(s.cfg, s.n, n, &kick, &drift);
        f[2 * n] = (float)kick;
        f[2 * n + 1] = (float)(drift * (s.pb == 2 ? PosFmt<2>::kCodesPerFine : PosFmt<1>::kCodesPerFine));
    }
    cudaMemcpyAsync(s.d_factors, f, sizeof(float) * 2 * S, cudaMemcpyHostToDevice, s.stream);
    cudaStreamSynchronize(s.stream);
    delete[] f;
}

void set_device_step(Sim& s, int64_t step) {
    k_step_set<<<1, 1, 0, s.stream>>>(s.d_step, s.d_kd, s.d_factors, s.cfg.n_steps, (int)step);
}

// Device work of one step; swaps the store buffers (s.cur).
static int enqueue_step(Sim& s) {
    int rc;
    prof_mark(s, -1);
    if (s.lowmem) lowmem_bind(s, 1 - s.cur);   // S and F_l in the next store's region
    if ((rc = coarse_deposit(s))) return rc;
    prof_mark(s, 0);
    if ((rc = coarse_force(s))) return rc;
    prof_mark(s, 1);
    cudaMemsetAsync(s.counts[1 - s.cur], 0, sizeof(int32_t) * s.ncells, s.stream);
    cudaMemsetAsync(s.S, 0, sizeof(unsigned long long) * 3 * s.ncells, s.stream);
    cudaMemsetAsync(s.d2, 0, 64, s.stream);
    if ((rc = tile_pass(s, 1, nullptr))) return rc;
    prof_mark(s, 2);
    if ((rc = s.lowmem ? encode_from_parked(s) : encode_from_qp(s, true))) return rc;
    k_step_advance<<<1, 1, 0, s.stream>>>(s.d_step, s.d_kd, s.d_factors, s.cfg.n_steps);
    s.launches++;
    return check_launch(s, "step");
}

static int one_step(Sim& s) {
    if (s.step >= s.cfg.n_steps) return set_error(s, PMPM_EINVAL, "schedule exhausted");
    int rc;
    if (!s.offsets_valid) {
        if ((rc = scan_counts(s, s.counts[s.cur], s.offsets[s.cur]))) return rc;
        s.offsets_valid = true;
    }
    s.in_step = true;
    if (s.graphs) {
        const int c = s.cur;
        if (!s.graph_ready[c]) {
            const bool prof = s.prof;
            const int64_t l0 = s.launches;
            s.prof = false;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "capture: %s", cudaGetErrorString(e));
            rc = enqueue_step(s);
            e = cudaStreamEndCapture(s.stream, &g);
            s.prof = prof;
            s.cur = c;   // capturing ran nothing
            s.graph_launches[c] = s.launches - l0;
            s.launches = l0;
            if (rc || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return rc ? rc : set_error(s, PMPM_ECUDA, "capture: %s", cudaGetErrorString(e));
            }
            e = cudaGraphInstantiate(&s.graph_exec[c], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "instantiate: %s", cudaGetErrorString(e));
            s.graph_ready[c] = true;
        }
        const cudaError_t e = cudaGraphLaunch(s.graph_exec[c], s.stream);
        if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "graph launch: %s", cudaGetErrorString(e));
        s.launches += s.graph_launches[c];
        s.cur = 1 - c;
    } else {
        if ((rc = enqueue_step(s))) return rc;
    }
    s.in_step = false;
    s.step += 1;
    s.a = sched_a(s, s.step);
    return PMPM_OK;
}

// Shared by pmpm_init and pmpm_init_like: everything but the force tables.
static pmpm_sim* init_common(const pmpm_config* cfg, void* d_workspace, size_t bytes,
                             void* cuda_stream, int* rc_out) {
    char msg[256];
    int rc = validate(cfg, msg, sizeof(msg));
    if (rc) {
        snprintf(g_init_msg, sizeof(g_init_msg), "%s", msg);
        *rc_out = rc;
        return nullptr;
    }
    if (!d_workspace) {
        snprintf(g_init_msg, sizeof(g_init_msg), "null workspace");
        *rc_out = PMPM_EINVAL;
        return nullptr;
    }
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256) {
        snprintf(g_init_msg, sizeof(g_init_msg), "workspace must be 256-byte aligned");
        *rc_out = PMPM_EINVAL;
        return nullptr;
    }
    pmpm_sim* h = new (std::nothrow) pmpm_sim();
    if (!h) {
        *rc_out = PMPM_ENOMEM;
        return nullptr;
    }
    Sim& s = h->s;
    derive(s, cfg);
    const size_t need = layout(s, nullptr);
    if (bytes < need) {
        snprintf(g_init_msg, sizeof(g_init_msg), "workspace %zu bytes < required %zu", bytes, need);
        delete h;
        *rc_out = PMPM_ENOMEM;
        return nullptr;
    }
    s.ws = static_cast<uint8_t*>(d_workspace);
    s.ws_bytes = bytes;
    s.stream = static_cast<cudaStream_t>(cuda_stream);
    layout(s, s.ws);
    cudaGetDevice(&s.device);
    tile_setup();
    fft_setup();
    cudaMemsetAsync(s.err, 0, 4, s.stream);
    float T[256], E[256];
    codec_tables(T, E);
    cudaMemcpyAsync(s.Tdec, T, sizeof(T), cudaMemcpyHostToDevice, s.stream);
    cudaMemcpyAsync(s.Eedge, E, sizeof(E), cudaMemcpyHostToDevice, s.stream);
    k_twiddles<<<grid_for(s.fft_max, 256), 256, 0, s.stream>>>(s.fft_max, s.tw_f, s.tw_d);
    fill_factors(s);
    set_device_step(s, 0);
    s.a = cfg->a_init;
    *rc_out = check_launch(s, "init");
    return h;
}

static int init_finish(pmpm_sim* h, pmpm_sim** out) {
    int rc = sync_and_check(h->s);
    if (rc) {
        snprintf(g_init_msg, sizeof(g_init_msg), "%s", h->s.msg);
        delete h;
        return rc;
    }
    *out = h;
    return PMPM_OK;
}


GreenRefs sim_tables(const Sim& s) {
    return GreenRefs{s.green_coarse, s.green_fine, s.green_packed};
}

size_t green_table_bytes(int nc, size_t part[3]) {
    const size_t hc = (size_t)(nc / 2 + 1);
    part[0] = 16 * hc * hc * hc;
    part[1] = 4 * (size_t)kGreenS * kGreenS * kGreenS;
    part[2] = 4 * (size_t)(kGreenS - 2) * kGreenS * (kGreenS + 1) / 2;
    return part[0] + part[1] + part[2];
}

int copy_tables(cudaStream_t st, const GreenRefs& dst, const GreenRefs& src, int nc) {
    size_t part[3];
    green_table_bytes(nc, part);
    cudaError_t e = cudaMemcpyAsync(const_cast<float4*>(dst.coarse), src.coarse, part[0],
                                    cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<float*>(dst.fine), src.fine, part[1], cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<float*>(dst.packed), src.packed, part[2],
                            cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? PMPM_OK : PMPM_ECUDA;
}

pmpm_sim* sim_create(const pmpm_config* cfg, void* d_workspace, size_t bytes, cudaStream_t st,
                     const GreenRefs* tables, int* rc_out) {
    int rc = PMPM_OK;
    pmpm_sim* h = init_common(cfg, d_workspace, bytes, st, &rc);
    if (!h) {
        *rc_out = rc;
        return nullptr;
    }
    if (!rc) {
        if (tables) {
            rc = copy_tables(h->s.stream, sim_tables(h->s), *tables, h->s.nc);
            if (rc) set_error(h->s, rc, "table copy: %s", cudaGetErrorString(cudaGetLastError()));
        } else {
            rc = build_green_tables(h->s);
        }
    }
    if (rc) {
        snprintf(g_init_msg, sizeof(g_init_msg), "%s", h->s.msg);
        delete h;
        *rc_out = rc;
        return nullptr;
    }
    pmpm_sim* out = nullptr;
    *rc_out = init_finish(h, &out);
    return out;
}

const char* init_message() { return g_init_msg; }

}  // namespace pmpm

using namespace pmpm;

extern "C" {

int pmpm_workspace_bytes(const pmpm_config* cfg, size_t* bytes) {
    char msg[256];
    int rc = validate(cfg, msg, sizeof(msg));
    if (rc) {
        snprintf(g_init_msg, sizeof(g_init_msg), "%s", msg);
        return rc;
    }
    if (!bytes) return PMPM_EINVAL;
    Sim* s = new (std::nothrow) Sim();
    if (!s) return PMPM_ENOMEM;
    derive(*s, cfg);
    *bytes = layout(*s, nullptr);
    delete s;
    return PMPM_OK;
}

int pmpm_step_factors(const pmpm_config* cfg, int32_t step, double* kick, double* drift,
                      double* ic_momentum) {
    char msg[256];
    int rc = validate(cfg, msg, sizeof(msg));
    if (rc) {
        snprintf(g_init_msg, sizeof(g_init_msg), "%s", msg);
        return rc;
    }
    if (step < 0 || step >= cfg->n_steps || !kick || !drift || !ic_momentum) return PMPM_EINVAL;
    const int64_t np3 = (int64_t)cfg->np * cfg->np * cfg->np;
    step_factors(*cfg, np3, step, kick, drift);
    *ic_momentum = bg_ic_momentum_factor(background_of(cfg->omega_m, cfg->omega_l), cfg->a_init);
    return PMPM_OK;
}

int pmpm_init(const pmpm_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
              pmpm_sim** out) {
    if (!out) return PMPM_EINVAL;
    int rc = PMPM_OK;
    *out = sim_create(cfg, d_workspace, bytes, static_cast<cudaStream_t>(cuda_stream), nullptr, &rc);
    return rc;
}

int pmpm_init_like(const pmpm_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
                   const pmpm_sim* donor, pmpm_sim** out) {
    if (!out || !donor || !cfg) return PMPM_EINVAL;
    if (donor->s.nc != cfg->nc) {
        snprintf(g_init_msg, sizeof(g_init_msg), "donor has nc=%d, config nc=%d", donor->s.nc, cfg->nc);
        return PMPM_EINVAL;
    }
    const GreenRefs t = sim_tables(donor->s);
    int rc = PMPM_OK;
    *out = sim_create(cfg, d_workspace, bytes, static_cast<cudaStream_t>(cuda_stream), &t, &rc);
    return rc;
}

int pmpm_graph_mode(pmpm_sim* h, int32_t enable) {
    if (!h) return PMPM_EINVAL;
    Sim& s = h->s;
    const cudaStream_t st = s.stream;
    if (enable && (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread))
        return set_error(s, PMPM_EINVAL, "graph mode needs a created stream, not a default stream");
    s.graphs = enable != 0;
    return PMPM_OK;
}

int pmpm_ic_zeldovich(pmpm_sim* h, uint64_t seed, double slope, double k_c, double rms_disp) {
    if (!h) return PMPM_EINVAL;
    Sim& s = h->s;
    if (!(k_c > 0.0) || !(rms_disp >= 0.0)) return set_error(s, PMPM_EINVAL, "bad spectrum");
    s.qp_step = false;
    return ic_zeldovich(s, seed, slope, k_c, rms_disp);
}

int pmpm_step(pmpm_sim* h, int32_t nsteps) {
    if (!h) return PMPM_EINVAL;
    Sim& s = h->s;
    if (!s.have_state) return set_error(s, PMPM_ESTATE, "no particle state");
    if (nsteps < 0 || s.step + nsteps > s.cfg.n_steps)
        return set_error(s, PMPM_EINVAL, "%d steps exceed the schedule (%lld of %d taken)", nsteps,
                         (long long)s.step, s.cfg.n_steps);
    for (int i = 0; i < nsteps; ++i) {
        s.qp_step = false;
        const int rc = one_step(s);
        if (rc) return rc;
        if (s.prof && s.ev_count > kEventRing - 16) prof_fold(s);
        s.qp_step = !s.lowmem;
    }
    return PMPM_OK;
}

int pmpm_power_spectrum(pmpm_sim* h, int32_t nmesh, int32_t nbins, double* k, double* pk,
                        int64_t* nmodes) {
    if (!h || !k || !pk || !nmodes) return PMPM_EINVAL;
    Sim& s = h->s;
    if (!s.have_state) return set_error(s, PMPM_ESTATE, "no particle state");
    if (!s.offsets_valid) {
        int rc = scan_counts(s, s.counts[s.cur], s.offsets[s.cur]);
        if (rc) return rc;
        s.offsets_valid = true;
    }
    s.qp_step = false;
    int rc = power_spectrum(s, nmesh, nbins, k, pk, nmodes);
    if (rc) return rc;
    return sync_and_check(s);
}

static int copy_out(Sim& s, void* dst, const void* src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s.stream);
    if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "fetch: %s", cudaGetErrorString(e));
    return PMPM_OK;
}

int pmpm_fetch(pmpm_sim* h, int32_t what, void* dst, size_t bytes) {
    if (!h || !dst) return PMPM_EINVAL;
    Sim& s = h->s;
    const size_t N = (size_t)s.n, C = (size_t)s.ncells;
    size_t need = 0;
    switch (what) {
        case PMPM_STREAMS: need = store_bytes(s); break;
        case PMPM_COUNTS: need = 4 * C; break;
        case PMPM_VC: need = 12 * C; break;
        case PMPM_SCALARS: need = sizeof(pmpm_scalars); break;
        case PMPM_DECODED_Q: case PMPM_DECODED_P: case PMPM_FORCE: need = 12 * N; break;
        case PMPM_COARSE_DENSITY: need = 8 * C; break;
        case PMPM_STEP_QP: need = 24 * N; break;
        default: return set_error(s, PMPM_EINVAL, "unknown fetch item %d", what);
    }
    if (s.lowmem && (what == PMPM_DECODED_Q || what == PMPM_DECODED_P || what == PMPM_FORCE ||
                     what == PMPM_STEP_QP))
        return set_error(s, PMPM_EINVAL, "fetch %d needs the per-particle buffers a low-memory sim "
                         "does not have", what);
    if (bytes != need) return set_error(s, PMPM_EINVAL, "fetch %d needs %zu bytes, got %zu", what, need, bytes);
    if (!s.have_state) return set_error(s, PMPM_ESTATE, "no particle state");
    if (what == PMPM_STEP_QP && !s.qp_step)
        return set_error(s, PMPM_ESTATE, "no step result: fetch STEP_QP right after pmpm_step");
    if (what == PMPM_DECODED_Q || what == PMPM_DECODED_P || what == PMPM_FORCE) s.qp_step = false;
    int rc = PMPM_OK;
    if (!s.offsets_valid && what != PMPM_STREAMS && what != PMPM_COUNTS && what != PMPM_VC &&
        what != PMPM_SCALARS) {
        if ((rc = scan_counts(s, s.counts[s.cur], s.offsets[s.cur]))) return rc;
        s.offsets_valid = true;
    }
    switch (what) {
        case PMPM_STREAMS: rc = copy_out(s, dst, s.streams[s.cur], need); break;
        case PMPM_COUNTS: rc = copy_out(s, dst, s.counts[s.cur], need); break;
        case PMPM_VC: rc = copy_out(s, dst, s.vc[s.cur], need); break;
        case PMPM_SCALARS: {
            float sig = 0.f;
            cudaError_t e = cudaMemcpyAsync(&sig, s.sigma_d[s.cur], 4, cudaMemcpyDeviceToHost, s.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
            if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "fetch: %s", cudaGetErrorString(e));
            pmpm_scalars sc;
            sc.a = s.a;
            sc.sigma = sig;
            sc.step = s.step;
            sc.n = s.n;
            memcpy(dst, &sc, sizeof(sc));
            break;
        }
        case PMPM_DECODED_Q:
        case PMPM_DECODED_P:
            if ((rc = decode_state(s))) return rc;
            rc = copy_out(s, dst, what == PMPM_DECODED_Q ? (const void*)s.Qn : (const void*)s.Pn, need);
            break;
        case PMPM_FORCE:
            if ((rc = coarse_deposit(s))) return rc;
            if ((rc = coarse_force(s))) return rc;
            if ((rc = tile_pass(s, 0, s.Pn))) return rc;
            rc = copy_out(s, dst, s.Pn, need);
            break;
        case PMPM_COARSE_DENSITY:
            if ((rc = coarse_deposit(s))) return rc;
            rc = copy_out(s, dst, s.rho_c, need);
            break;
        case PMPM_STEP_QP:
            rc = copy_out(s, dst, s.Qn, 12 * N);
            if (!rc) rc = copy_out(s, static_cast<uint8_t*>(dst) + 12 * N, s.Pn, 12 * N);
            break;
    }
    if (rc) return rc;
    return sync_and_check(s);
}

int pmpm_fetch_tile_density(pmpm_sim* h, int32_t tile, uint32_t* dst, size_t bytes, int32_t* origin,
                            int32_t* tile_edge) {
    if (!h || !dst) return PMPM_EINVAL;
    Sim& s = h->s;
    const int64_t ntiles = (int64_t)s.nt * s.nt * s.nt;
    if (tile < 0 || tile >= ntiles)
        return set_error(s, PMPM_EINVAL, "tile %d outside [0, %lld)", tile, (long long)ntiles);
    const size_t need = sizeof(uint32_t) * kTileFFT * kTileFFT * kTileFFT;
    if (bytes != need) return set_error(s, PMPM_EINVAL, "a tile box needs %zu bytes, got %zu", need, bytes);
    if (s.scratch_bytes < need)
        return set_error(s, PMPM_EINVAL, "the workspace scratch (%zu bytes) cannot hold a tile box",
                         s.scratch_bytes);
    if (!s.have_state) return set_error(s, PMPM_ESTATE, "no particle state");
    int rc = PMPM_OK;
    if (!s.offsets_valid) {
        if ((rc = scan_counts(s, s.counts[s.cur], s.offsets[s.cur]))) return rc;
        s.offsets_valid = true;
    }
    s.qp_step = false;
    uint32_t* d = reinterpret_cast<uint32_t*>(s.scratch);
    if ((rc = tile_density(s, tile, d))) return rc;
    if ((rc = copy_out(s, dst, d, need))) return rc;
    const int t[3] = {tile % s.nt, (tile / s.nt) % s.nt, tile / (s.nt * s.nt)};
    for (int d3 = 0; d3 < 3; ++d3) {
        const int c0 = tile_bound(t[d3], s.nc, s.nt), c1 = tile_bound(t[d3] + 1, s.nc, s.nt);
        if (origin) origin[d3] = kRatio * c0 - kBuffer;
        if (tile_edge) tile_edge[d3] = kRatio * (c1 - c0);
    }
    return sync_and_check(s);
}

int pmpm_load(pmpm_sim* h, int32_t what, const void* src, size_t bytes) {
    if (!h || !src) return PMPM_EINVAL;
    Sim& s = h->s;
    s.qp_step = false;
    const size_t N = (size_t)s.n, C = (size_t)s.ncells;
    cudaError_t e = cudaSuccess;
    switch (what) {
        case PMPM_STREAMS:
            if (bytes != store_bytes(s))
                return set_error(s, PMPM_EINVAL, "streams need %zu bytes", store_bytes(s));
            e = cudaMemcpyAsync(s.streams[s.cur], src, bytes, cudaMemcpyHostToDevice, s.stream);
            s.loaded |= 1;
            break;
        case PMPM_COUNTS: {
            if (bytes != 4 * C) return set_error(s, PMPM_EINVAL, "counts need %zu bytes", 4 * C);
            // the kernels index the particle streams through these counts:
            // they must be non-negative and add up to N, checked on the
            // device right after the copy (before anything else on the
            // stream); a refused load leaves no state
            e = cudaMemcpyAsync(s.counts[s.cur], src, bytes, cudaMemcpyHostToDevice, s.stream);
            s.offsets_valid = false;
            s.loaded &= ~2;
            if (e != cudaSuccess) break;
            check_loaded_counts(s);
            const int rc = sync_and_check(s);
            if (rc) {
                s.have_state = false;
                return rc;
            }
            s.loaded |= 2;
            break;
        }
        case PMPM_VC:
            if (bytes != 12 * C) return set_error(s, PMPM_EINVAL, "v_c needs %zu bytes", 12 * C);
            e = cudaMemcpyAsync(s.vc[s.cur], src, bytes, cudaMemcpyHostToDevice, s.stream);
            s.loaded |= 4;
            break;
        case PMPM_SCALARS: {
            if (bytes != sizeof(pmpm_scalars)) return set_error(s, PMPM_EINVAL, "scalars size");
            pmpm_scalars sc;
            memcpy(&sc, src, sizeof(sc));
            if (sc.n != s.n) return set_error(s, PMPM_EINVAL, "scalars n=%lld != %lld", (long long)sc.n, (long long)s.n);
            if (sc.step < 0 || sc.step > s.cfg.n_steps) return set_error(s, PMPM_EINVAL, "scalars step");
            const float sig = (float)sc.sigma;
            e = cudaMemcpyAsync(s.sigma_d[s.cur], &sig, 4, cudaMemcpyHostToDevice, s.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
            s.a = sc.a;
            s.step = sc.step;
            set_device_step(s, sc.step);
            s.loaded |= 8;
            break;
        }
        case PMPM_QP: {
            if (s.lowmem)
                return set_error(s, PMPM_EINVAL, "loading Q/P needs the per-particle buffers a "
                                 "low-memory sim does not have");
            if (bytes != 24 * N) return set_error(s, PMPM_EINVAL, "Q/P need %zu bytes", 24 * N);
            e = cudaMemcpyAsync(s.Qn, src, 12 * N, cudaMemcpyHostToDevice, s.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s.Pn, static_cast<const uint8_t*>(src) + 12 * N, 12 * N,
                                    cudaMemcpyHostToDevice, s.stream);
            if (e != cudaSuccess) break;
            // the codes index cells: check their range before any kernel uses them
            const int32_t* q = static_cast<const int32_t*>(src);
            const int64_t M = (int64_t)s.nc * (s.pb == 2 ? PosFmt<2>::kBins : PosFmt<1>::kBins);
            for (size_t i = 0; i < 3 * N; ++i)
                if (q[i] < 0 || q[i] >= M) {
                    cudaStreamSynchronize(s.stream);
                    return set_error(s, PMPM_EINVAL, "code out of range");
                }
            int rc = encode_from_qp(s, false);
            if (rc) return rc;
            s.loaded = 15;
            break;
        }
        default:
            return set_error(s, PMPM_EINVAL, "unknown load item %d", what);
    }
    if (e != cudaSuccess) return set_error(s, PMPM_ECUDA, "load: %s", cudaGetErrorString(e));
    // a store is usable once streams, counts, v_c and scalars are all present
    s.have_state = s.loaded == 15;
    return sync_and_check(s);
}

int pmpm_sync(pmpm_sim* h) {
    if (!h) return PMPM_EINVAL;
    return sync_and_check(h->s);
}

int pmpm_stage_times(pmpm_sim* h, int32_t enable, double* times, int32_t n, int64_t* launches) {
    if (!h) return PMPM_EINVAL;
    Sim& s = h->s;
    if (!s.ev_made) {
        for (int i = 0; i < kEventRing; ++i) cudaEventCreate(&s.ev[i]);
        s.ev_made = true;
    }
    prof_fold(s);
    if (times) {
        for (int i = 0; i < n && i < kStages; ++i) times[i] = s.stage_ms[i];
        if (launches) *launches = s.launches;
    } else {
        for (int i = 0; i < kStages; ++i) s.stage_ms[i] = 0.0;
        s.launches = 0;
    }
    s.prof = enable != 0;
    return PMPM_OK;
}

void pmpm_destroy(pmpm_sim* h) {
    if (!h) return;
    Sim& s = h->s;
    cudaStreamSynchronize(s.stream);
    for (int c = 0; c < 2; ++c)
        if (s.graph_ready[c]) cudaGraphExecDestroy(s.graph_exec[c]);
    if (s.ev_made)
        for (int i = 0; i < kEventRing; ++i) cudaEventDestroy(s.ev[i]);
    delete h;
}

const char* pmpm_last_error(const pmpm_sim* h) {
    if (!h) return g_init_msg;
    return h->s.msg;
}

int pmpm_codec_tables(float* T, float* E) {
    if (!T || !E) return PMPM_EINVAL;
    codec_tables(T, E);
    return PMPM_OK;
}

}  // extern "C"
