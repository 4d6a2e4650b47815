// pmpm_impl.cuh -- the sim object, its workspace layout and the host-side
// helpers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/pmpm.h"
#include "common.cuh"

namespace pmpm {

constexpr int kStages = 6;          // see pmpm_stage_times
constexpr int kEventRing = 4096;

struct Sim {
    pmpm_config cfg;
    int device = 0;
    int nc = 0, nf = 0, np = 0, nt = 0, tile_max = 0, pk_max = 0, fft_max = 0;
    int pb = 1;                                 // bytes per position bin (1 or 2)
    double ic_pfac = 0.0;                       // Zel'dovich p per unit of a_init Psi (a_init^1.5 in EdS)
    int64_t n = 0, ncells = 0;
    cudaStream_t stream = nullptr;
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;

    // particle store, double-buffered (Sec. III-A)
    uint8_t* streams[2] = {nullptr, nullptr};   // m0 m1 m2 [N] (pb bytes each), u0 u1 u2 [N]
    int32_t* counts[2] = {nullptr, nullptr};    // [nc^3]
    int64_t* offsets[2] = {nullptr, nullptr};   // [nc^3 + 1]
    float* vc[2] = {nullptr, nullptr};          // [3][nc^3]
    float* sigma_d[2] = {nullptr, nullptr};     // device scalar
    int cur = 0;
    bool have_state = false;
    int loaded = 0;                              // bits: streams, counts, v_c, scalars
    bool offsets_valid = false;
    bool qp_step = false;                        // Qn/Pn hold the last step's new codes/momenta
    double a = 0.0;
    int64_t step = 0;

    // step buffers
    int32_t* fill = nullptr;                    // [nc^3]
    unsigned long long* S = nullptr;            // [3][nc^3] fixed-point momentum sums
    unsigned long long* d2 = nullptr;           // [8] T = sum P^2, U = sum floor(S^2/n), 32-bit digits
    long long* rho_c = nullptr;                 // [nc^3]
    float2* cA = nullptr;                       // [nc^3] coarse spectra
    float2* cB1 = nullptr;
    float2* cB2 = nullptr;
    float* Fl = nullptr;                        // [3][nc^3]
    float4* green_coarse = nullptr;             // [(nc/2+1)^3] (S_x, S_y, S_z, 0), |kx| fastest
    float* green_fine = nullptr;                // [17^3]
    float* green_packed = nullptr;              // [17 x 153] b <= c half of green_fine
    float* Tdec = nullptr;                      // [256]
    float* Eedge = nullptr;                     // [256]
    float2* tw_f = nullptr;                     // [fft_max] exp(-2 pi i k / fft_max)
    double2* tw_d = nullptr;
    uint32_t* err = nullptr;
    long long* blocksums = nullptr;
    int64_t nblocks_scan = 0;
    double* ic_partial = nullptr;               // [3*1024 + 1] IC rms partial sums
    float* d_factors = nullptr;                 // [2 n_steps] kick, drift (codes) per step
    int* d_step = nullptr;                      // device copy of the step counter
    float* d_kd = nullptr;                      // [2] kick and drift factors of that step
    double* pk_bins = nullptr;                  // [3][pk_max/2 + 1] power-spectrum sums

    // transient scratch (step, init, ICs and power spectrum share it)
    uint8_t* scratch = nullptr;
    size_t scratch_bytes = 0;
    int32_t* Qn = nullptr;                      // [3][N] (aliases scratch; default step)
    float* Pn = nullptr;                        // [3][N] (aliases scratch)

    // low-memory step (PMPM_FLAG_LOWMEM)
    bool fp16 = false;                          // PMPM_FLAG_FINE_FP16: tile spectrum stored as FP16
    bool lowmem = false;
    float2* ic_work = nullptr;                  // [N] float32 IC transform (overlays the store)
    float* ic_psi = nullptr;                    // [3][N] float32 displacement field

    // captured steps, one per buffer parity
    bool graphs = false;
    bool graph_ready[2] = {false, false};
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
    int64_t graph_launches[2] = {0, 0};

    // stage timing
    bool in_step = false;
    bool prof = false;
    cudaEvent_t ev[kEventRing];
    int ev_stage[kEventRing];
    int ev_count = 0;
    bool ev_made = false;
    double stage_ms[kStages] = {0, 0, 0, 0, 0, 0};
    int64_t launches = 0;

    char msg[512] = {0};
};

inline uintptr_t align_up(uintptr_t p, uintptr_t a = 256) { return (p + a - 1) & ~(a - 1); }

inline int grid_for(int64_t n, int block, int cap = 152 * 64) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

int set_error(Sim& s, int code, const char* fmt, ...);
int check_launch(Sim& s, const char* what);

// workspace layout: fills the Sim's pointers when base != nullptr; returns bytes
size_t layout(Sim& s, uint8_t* base);

// kernels, by translation unit
int build_green_tables(Sim& s);
size_t green_scratch_bytes(int nc);
template <typename R>
int fft3d(Sim& s, void* data, int n, int sign);
int fft_pass_count(int n);
int coarse_force(Sim& s);             // deposit + FFT + Green -> s.Fl
int coarse_deposit(Sim& s);           // -> s.rho_c
int tile_pass(Sim& s, int mode, float* G);
int tile_density(Sim& s, int tile, uint32_t* d_out);   // one tile's fine box after the deposit
void tile_setup();
void fft_setup();
int scan_counts(Sim& s, const int32_t* counts, int64_t* offsets);
int encode_from_qp(Sim& s, bool counts_ready);
int scan_and_means(Sim& s, int nxt);
void check_loaded_counts(Sim& s);    // device check of loaded counts (kErrLoadCounts)
int encode_from_parked(Sim& s);       // low-memory step: re-encode from the old store and Pn
void lowmem_bind(Sim& s, int nxt);    // low-memory layout: S and F_l in store nxt's region
int encode_from_psi(Sim& s, const double* scale);   // low-memory ICs -> store 0
int decode_state(Sim& s);              // -> s.Qn, s.Pn
int ic_zeldovich(Sim& s, uint64_t seed, double slope, double kc, double rms);
int power_spectrum(Sim& s, int nmesh, int nbins, double* k, double* pk, int64_t* nm);
// The same in two halves: enqueue the kernels and an async copy of the raw
// [3][nbins] sums into host_bins (pinned for a truly async copy), then, once
// the stream has reached that point, turn the sums into k, P(k), mode counts.
int power_spectrum_enqueue(Sim& s, int nmesh, int nbins, double* host_bins);
void power_spectrum_finish(const double* host_bins, int nbins, double* k, double* pk, int64_t* nm);
void prof_mark(Sim& s, int stage);     // records an event closing `stage` (-1: opening)
void set_device_step(Sim& s, int64_t step);

// The store of buffer b: position bins m_d (pb bytes each) then velocity
// bins u_d (1 byte each), every stream N entries long.
inline uint8_t* m_stream(Sim& s, int b, int d) { return s.streams[b] + (size_t)d * s.pb * s.n; }
inline uint8_t* u_stream(Sim& s, int b, int d) {
    return s.streams[b] + (size_t)3 * s.pb * s.n + (size_t)d * s.n;
}
inline size_t store_bytes(const Sim& s) { return (size_t)(3 * s.pb + 3) * s.n; }

}  // namespace pmpm

namespace pmpm {

// Device pointers of the three force tables (Sec. II): the coarse-kernel
// spectrum, the fine kernel K_s spectrum and its packed tile copy.
struct GreenRefs {
    const float4* coarse;
    const float* fine;
    const float* packed;
};

GreenRefs sim_tables(const Sim& s);
size_t green_table_bytes(int nc, size_t part[3]);     // bytes of the three tables for this nc
int copy_tables(cudaStream_t st, const GreenRefs& dst, const GreenRefs& src, int nc);
// Create a sim on `st`; force tables copied from `tables` when non-null, else
// built.  Returns null with *rc set on failure (message: init_message()).
struct ::pmpm_sim* sim_create(const pmpm_config* cfg, void* d_workspace, size_t bytes,
                              cudaStream_t st, const GreenRefs* tables, int* rc);
const char* init_message();

}  // namespace pmpm

struct pmpm_sim {
    pmpm::Sim s;
};
