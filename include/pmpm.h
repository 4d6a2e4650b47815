/*
 * pmpm.h -- C ABI of the GB300 two-level particle-mesh (PM-PM) library.
 *
 * The library evolves cosmological N-body particles stored in the
 * fixed-point format of CUBE (Cheng et al., arXiv:2003.03931): six 1-byte
 * integers per particle (Sec. III-A, Eq. 2 and Eq. 3), grouped by coarse
 * cell, with per-cell counts and a per-cell mean velocity.  One step decodes
 * the particles, deposits them on a coarse mesh and on buffered fine-mesh
 * tiles, multiplies by the force kernels in Fourier space (Sec. II, Eq. 1),
 * interpolates the force, kicks and drifts, and re-encodes and re-sorts the
 * particles by cell.
 *
 * Conventions
 *  - Lengths are in fine cells; the box is 4*nc fine cells per side (the
 *    coarse mesh is 4x coarser, Sec. II).  Cell indices are 0-based, flat
 *    index cx + nc*(cy + nc*cz) (x fastest).
 *  - Position code Q = c*B + m with B = 256 bins per coarse cell (1-byte m,
 *    Eq. 2) or 65536 (2-byte m, Sec. III-A); decoded position (Q + 1/2)/(B/4).
 *  - Velocity p = a^2 dx/dt; decoded p = v_c + sigma*T[u] in float32, T the
 *    tangent of the bin-centre angle of 256 equal angle bins (Eq. 3; the
 *    map f is the arctangent form of Sec. III-B.2).
 *  - Memory: the caller owns all device memory.  pmpm_init borrows a device
 *    workspace of pmpm_workspace_bytes() bytes and a CUDA stream; the library
 *    allocates no device memory of its own.  Host buffers passed to fetch/
 *    load are caller-owned and only read/written during the call.
 *  - Every call returns PMPM_OK (0) or a negative error code; no exception
 *    crosses the ABI.  pmpm_last_error(sim) describes the last failure.
 *  - Calls enqueue work on the sim's stream and return without waiting,
 *    except pmpm_fetch, pmpm_load, pmpm_power_spectrum and pmpm_sync, which
 *    synchronise the stream and report device-side error flags
 *    (PMPM_EOVERFLOW, PMPM_ECOUNT).  One sim must not be used from two
 *    threads at once.
 */
#ifndef PMPM_H
#define PMPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define PMPM_OK         0
#define PMPM_EINVAL    -1   /* bad argument or configuration */
#define PMPM_ENOMEM    -2   /* workspace smaller than pmpm_workspace_bytes() */
#define PMPM_ECUDA     -3   /* a CUDA runtime call failed */
#define PMPM_EOVERFLOW -4   /* a fixed-point or integer range was exceeded */
#define PMPM_ECOUNT    -5   /* particle count not conserved (internal error) */
#define PMPM_ESTATE    -6   /* no particle state loaded yet */
#define PMPM_ETIMEOUT  -7   /* a host-side time limit ran out; the work goes on */

/* what to fetch / load */
#define PMPM_STREAMS          1  /* the store in storage order: m0 m1 m2 [N] of pos_bytes
                                    each (little-endian), then u0 u1 u2 [N] uint8;
                                    (3 pos_bytes + 3) N bytes */
#define PMPM_COUNTS           2  /* int32 [nc^3] particles per coarse cell */
#define PMPM_VC               3  /* float [3][nc^3] per-cell mean momentum v_c */
#define PMPM_SCALARS          4  /* pmpm_scalars */
#define PMPM_DECODED_Q        5  /* int32 [3][N] position codes Q (fetch only) */
#define PMPM_DECODED_P        6  /* float [3][N] decoded momenta (fetch only) */
#define PMPM_FORCE            7  /* float [3][N] unit-G field g at the particles,
                                    current state, storage order (fetch only) */
#define PMPM_COARSE_DENSITY   8  /* int64 [nc^3] integer CIC density, units 2^-27
                                    per particle (fetch only) */
#define PMPM_QP               9  /* load only: int32 Q[3][N] then float p[3][N];
                                    encodes them into the store (Sec. III-A) */
#define PMPM_STEP_QP         10  /* fetch only: int32 Q'[3][N] then float p'[3][N], the
                                    drifted position codes and kicked momenta of the
                                    last step (Sec. II), in the storage order of the
                                    state that step started from; 24 N bytes.
                                    Available after pmpm_step on a default sim until
                                    the next call that loads, initialises, fetches
                                    DECODED_Q/P or FORCE, or computes a power spectrum
                                    (they reuse the buffer): PMPM_ESTATE otherwise */
#define PMPM_FINE_TILE_DENSITY 11 /* fetch only (pmpm_fetch_tile_density): uint32
                                    [32][32][32], x fastest, the integer CIC density
                                    of one tile's fine-mesh box, units 2^-21 per
                                    particle (Sec. II) */

/* pmpm_config.flags */
#define PMPM_FLAG_LOWMEM 1   /* Low-memory step for the largest boxes.  The tile
                                pass (Sec. II) keeps only the new momenta (float32,
                                12 bytes per particle, in the space the coarse mesh
                                uses earlier in the step), not the new codes, and
                                counts the new cells and sums their momenta and
                                squared momenta (which give v_c and sigma, Eq. 3).
                                The re-encode (Sec. III-A) then derives each
                                particle's new codes again from its old codes and
                                new momentum, with the same integer drift, so the
                                new store is the one the default step writes.
                                The momentum sums and F_l share the next store's
                                space.  About 31 bytes per particle of workspace
                                instead of 83 (2048^3 particles: 264 GB, which
                                fits one GB300).
                                Initial conditions use float32 transforms and a
                                float32 displacement field (the default uses
                                float64).  PMPM_DECODED_Q/P, PMPM_FORCE,
                                PMPM_STEP_QP and loading PMPM_QP are not
                                available. */
#define PMPM_FLAG_FINE_FP16 2 /* Precision option (Sec. III-A stores particles in
                                1 or 2 bytes; this stores the fine-mesh field
                                compactly too): the tile pass keeps each tile's
                                density spectrum in FP16 (the density scaled by a
                                power of two per tile to stay in range) while every
                                transform, Green multiply and force sum runs in
                                float32.  Results differ from the default step by the
                                FP16 rounding (about 1e-3 of the force); default
                                step only (not with PMPM_FLAG_LOWMEM). */

typedef struct pmpm_config {
    int32_t np;              /* particles per side of the initial lattice, N = np^3 */
    int32_t nc;              /* coarse cells per side (>= 8); fine mesh 4*nc */
    int32_t tile_max;        /* largest tile edge in coarse cells: 4 or 5 */
    int32_t buffer;          /* tile buffer in fine cells; must be 6 (Sec. IV-A.2) */
    int32_t pos_bytes;       /* bytes per position coordinate: 1 (Eq. 2) or 2 (Sec. III-A;
                                CIC weight products rounded to the 1-byte units) */
    int32_t vel_bytes;       /* bytes per velocity coordinate; must be 1 (Eq. 3) */
    int32_t pk_mesh_max;     /* largest power-spectrum mesh; 0 = min(4*nc, 512) */
    int32_t flags;           /* PMPM_FLAG_* below; 0 = default */
    double  a_init;          /* first scale factor of the equal-log-a schedule */
    double  a_final;         /* last scale factor */
    int32_t n_steps;         /* steps of the schedule */
    int32_t reserved2;
    double  omega_m;         /* background (Sec. IV-A.2; H0 = 1): matter density today;
                                0 with omega_l 0 = Einstein-de Sitter (Omega_m = 1) */
    double  omega_l;         /* cosmological constant today; curvature 1 - omega_m - omega_l.
                                The kick and drift factors are integrals of 1/(a^2 E) and
                                1/(a^3 E) over the step, E(a) = H(a)/H0, and the
                                Zel'dovich momenta follow the growing mode */
} pmpm_config;

typedef struct pmpm_scalars {
    double  a;               /* scale factor of the stored positions */
    double  sigma;           /* velocity scale of Eq. 3 (a float32 value) */
    int64_t step;            /* steps taken on the schedule */
    int64_t n;               /* particles */
} pmpm_scalars;

typedef struct pmpm_sim pmpm_sim;

/* Device bytes a sim of this configuration needs.  Host-only, no GPU call.
 * Returns PMPM_EINVAL for unsupported configurations. */
int pmpm_workspace_bytes(const pmpm_config* cfg, size_t* bytes);

/* The float64 factors of step `step` (0 <= step < n_steps) of a
 * configuration's schedule, host only: *kick multiplies the unit-G field g
 * (3 Omega_m / (8 pi rho_bar) times the integral of 1/(a^2 E) from the
 * previous half step to the next), *drift multiplies p to give the
 * displacement in fine cells (the integral of 1/(a^3 E) over the step), and
 * *ic_momentum is the Zel'dovich momentum per unit displacement at a_init
 * (a^2 E f; sqrt(a_init) for Einstein-de Sitter).  Sec. IV-A.2's background;
 * the integrator itself is not given by the paper (kick-drift leapfrog, steps
 * equal in log a).  PMPM_EINVAL for a bad configuration or step. */
int pmpm_step_factors(const pmpm_config* cfg, int32_t step, double* kick, double* drift,
                      double* ic_momentum);

/* Create a sim on the current CUDA device.  d_workspace: device pointer,
 * 256-byte aligned, at least pmpm_workspace_bytes() bytes, owned by the
 * caller and borrowed until pmpm_destroy.  cuda_stream: a cudaStream_t (or
 * NULL for the legacy default stream).  Builds the force-kernel tables
 * (Sec. II) on the stream.  *out receives the handle. */
int pmpm_init(const pmpm_config* cfg, void* d_workspace, size_t bytes,
              void* cuda_stream, pmpm_sim** out);

/* As pmpm_init, but the force-kernel tables (Sec. II) are copied from a live
 * sim `donor` of the same nc instead of being computed again; the donor is
 * only read, on cuda_stream, during the call. */
int pmpm_init_like(const pmpm_config* cfg, void* d_workspace, size_t bytes,
                   void* cuda_stream, const pmpm_sim* donor, pmpm_sim** out);

/* enable != 0: each step is captured once per store buffer into a CUDA graph
 * and replayed (one launch per step instead of ~30).  Stage timing is not
 * recorded for replayed steps.  The sim's stream must be one the caller
 * created: a legacy or per-thread default stream cannot be captured, and
 * enabling on one returns PMPM_EINVAL. */
int pmpm_graph_mode(pmpm_sim* sim, int32_t enable);

/* Zel'dovich initial conditions at a_init (Sec. IV-A.2) for a power-law
 * spectrum P(k) = k^slope exp(-(k/k_c)^2), k in radians per fine cell;
 * white noise from counter-based SplitMix64 at `seed`; displacements scaled
 * so that their 3-D rms is rms_disp fine cells. */
int pmpm_ic_zeldovich(pmpm_sim* sim, uint64_t seed, double slope, double k_c,
                      double rms_disp);

/* Advance nsteps kick-drift steps of the schedule (Sec. II).  Asynchronous. */
int pmpm_step(pmpm_sim* sim, int32_t nsteps);

/* Power spectrum of the CIC density on an nmesh^3 mesh (nmesh = 4*nc / 2^j,
 * <= pk_mesh_max), Sec. IV-D: P(k) = L^3/nmesh^6 |DFT(delta)|^2 in shells
 * j = round(|n|), j = 1..nbins (nbins <= nmesh/2).  Host arrays of nbins
 * entries receive the mean |k|, mean P and mode count.  Synchronises. */
int pmpm_power_spectrum(pmpm_sim* sim, int32_t nmesh, int32_t nbins,
                        double* k, double* pk, int64_t* nmodes);

/* Copy part of the state (see PMPM_* above) into a host buffer of exactly
 * the listed size.  Synchronises. */
int pmpm_fetch(pmpm_sim* sim, int32_t what, void* host_dst, size_t bytes);

/* The fine-mesh box of one tile (Sec. II) as the tile pass deposits it,
 * for checking the integer CIC density node by node.  tile: flat tile index,
 * tx + nt (ty + nt tz), nt = ceil(nc / tile_max) tiles per side (tile t of
 * an axis spans coarse cells [floor(t nc / nt), floor((t + 1) nc / nt))).
 * host_dst: uint32 [32][32][32] (x fastest, 131072 bytes); box node i of an
 * axis is fine node o + i (periodic), o = 4 c0 - 6 with c0 the tile's first
 * coarse cell; origin (may be NULL) receives o for x, y, z and tile_edge
 * (may be NULL) the tile's edge in fine cells per axis.  The box holds the
 * deposit of the particles of coarse cells [c0 - 2, c1 + 2) clipped to the
 * box, so nodes i <= T + 12 (T the tile edge) carry the whole density and
 * the last nodes of a 16-cell tile only part of it.  Runs the deposit of
 * the current state (default and low-memory sims alike; the step's buffers
 * are reused, see PMPM_STEP_QP); synchronises.  PMPM_EINVAL for a tile out
 * of range, a buffer of another size, or a workspace whose scratch is
 * smaller than one box (tiny boxes with a small pk_mesh_max). */
int pmpm_fetch_tile_density(pmpm_sim* sim, int32_t tile, uint32_t* host_dst, size_t bytes,
                            int32_t* origin, int32_t* tile_edge);

/* Replace part of the state from a host buffer (PMPM_STREAMS, PMPM_COUNTS,
 * PMPM_VC, PMPM_SCALARS, or PMPM_QP which encodes raw codes and momenta).
 * Synchronises.  Counts are checked on the device right after their copy
 * (every count >= 0, sum N) and codes on the host (inside the box), before
 * any kernel indexes with them: PMPM_EINVAL, and the sim holds no state
 * until a valid one is loaded. */
int pmpm_load(pmpm_sim* sim, int32_t what, const void* host_src, size_t bytes);

/* Wait for the sim's stream and report device-side error flags. */
int pmpm_sync(pmpm_sim* sim);

/* Per-stage device time (ms) accumulated since the last reset, measured
 * with CUDA events on the sim's stream when enable != 0.  Stage order:
 * 0 coarse deposit, 1 coarse FFT + Green multiply, 2 tile fine PM + kick +
 * drift, 3 new-cell counts + scan + cell means, 4 dispersion, 5 encode +
 * scatter.  Calling with times == NULL sets the switch and resets the
 * totals. */
int pmpm_stage_times(pmpm_sim* sim, int32_t enable, double* times, int32_t n,
                     int64_t* launches);

/* Release the handle (not the caller's workspace or stream). */
void pmpm_destroy(pmpm_sim* sim);

/* Text of the last error on this sim (or of the last failed pmpm_init when
 * sim is NULL). */
const char* pmpm_last_error(const pmpm_sim* sim);

/* Power spectrum without any device allocation, for callers that may not
 * allocate GPU memory themselves: for example code running inside a host
 * application that owns a fixed device-memory budget, or a loop that cannot
 * afford the device-wide synchronisation an allocation may cause.  The paper
 * has no counterpart; it computes the same P(k) as pmpm_power_spectrum for
 * a cell-ordered store the caller already holds on the device:
 *   nc         coarse cells per side, a power of two in [8, 64]
 *   n          particles; d_m0..d_m2 their 1-byte position bins (Eq. 2; stores
 *              with 2-byte bins are not accepted), n bytes each, and d_counts
 *              the nc^3 per-cell counts (device pointers); counts that do not
 *              add up to n return PMPM_EINVAL
 *   nmesh      power of two dividing 4*nc, 4*nc/4 <= nmesh <= 64
 *   nbins      in [1, nmesh/2]; k, pk, nmodes are host arrays of nbins
 *   cuda_stream the stream to run on (NULL: legacy default stream)
 * Its scratch is one fixed array of about 4.2 MB in the library's device
 * memory, held by every GPU that loads the library until the process exits.
 * The first call on a device looks up that array's address and fills a
 * twiddle table there, synchronising the stream.  Every call copies its
 * result to the host arrays and waits for the stream before it returns.
 * All calls share the array: calls whose GPU work overlaps (other streams,
 * other host threads) race and give wrong results.  Larger sizes return
 * PMPM_EINVAL; pmpm_noalloc_last_error() explains. */
int pmpm_power_spectrum_noalloc(int32_t nc, int64_t n, const uint8_t* d_m0,
                                const uint8_t* d_m1, const uint8_t* d_m2,
                                const int32_t* d_counts, int32_t nmesh, int32_t nbins,
                                double* k, double* pk, int64_t* nmodes,
                                void* cuda_stream);

/* Text of the last failure of pmpm_power_spectrum_noalloc.  One buffer for
 * the whole process, written without a lock: with calls failing on several
 * host threads at once the text may belong to any of them. */
const char* pmpm_noalloc_last_error(void);

/* ------------------------------------------------------------------------
 * Serving many boxes on one GPU.  The paper runs one box and processes its
 * fine-mesh tiles as independent units in turn (Sec. II, Sec. IV-A); it has
 * no serving layer.  These calls hold many independent boxes on the device
 * at once: each request is a whole simulation (Zel'dovich ICs, n_steps
 * steps, the final power spectrum, Sec. IV-D), admitted when a slot and
 * enough of one caller-owned device arena are free, in arrival order, and
 * stepped with exactly the calls above, so its result is bit for bit the
 * one it would give alone.
 * ------------------------------------------------------------------------ */

/* Offset allocator over a device range the caller owns; host bookkeeping
 * only, no CUDA call.  Sizes round up to 256 bytes, offsets are multiples of
 * 256; first fit in address order; freed neighbours merge. */
typedef struct pmpm_arena pmpm_arena;
int pmpm_arena_create(size_t bytes, pmpm_arena** out);      /* EINVAL if bytes < 256 */
int pmpm_arena_alloc(pmpm_arena* arena, size_t bytes, size_t* offset);  /* ENOMEM: no range fits */
int pmpm_arena_free(pmpm_arena* arena, size_t offset);      /* EINVAL: not a live allocation */
int pmpm_arena_stats(const pmpm_arena* arena, size_t* used, size_t* largest_free,
                     int64_t* live);
void pmpm_arena_destroy(pmpm_arena* arena);

typedef struct pmpm_request {
    int32_t np, nc;          /* as pmpm_config; tile_max 5, buffer 6, 1-byte codes */
    int32_t n_steps;         /* steps of the equal-log-a schedule a_init -> a_final */
    int32_t pk_nmesh;        /* final P(k) mesh: power of two in [nc, 4*nc]; 0 = min(np, 4*nc) */
    int32_t pk_nbins;        /* 1..pk_nmesh/2; 0 = pk_nmesh/2 */
    int32_t flags;           /* 0 or PMPM_FLAG_LOWMEM (the low-memory step) */
    double  a_init, a_final;
    uint64_t seed;           /* initial conditions as pmpm_ic_zeldovich */
    double  slope, k_c, rms_disp;
    double  arrival;         /* engine clock (s): not admitted before this time */
    double*  k;              /* host, pk_nbins entries: mean |k| per shell (required) */
    double*  pk;             /* host, pk_nbins entries: P(k) (required) */
    int64_t* nmodes;         /* host, pk_nbins entries: modes per shell (required) */
    uint8_t* streams;        /* host, 6*np^3 bytes: final store, or NULL */
    int32_t* counts;         /* host, nc^3 entries: final per-cell counts, or NULL */
} pmpm_request;

typedef struct pmpm_result {
    int64_t id;              /* as returned by pmpm_batch_submit */
    int32_t status;          /* PMPM_OK or the error code of the failing call */
    int32_t reserved;
    double  t_arrival, t_admit, t_done;   /* engine clock (s) */
    double  a, sigma;        /* final scale factor and velocity scale (Eq. 3) */
    int64_t particle_steps;  /* np^3 * n_steps when status is PMPM_OK */
} pmpm_result;

typedef struct pmpm_batch_config {
    int32_t max_active;      /* boxes resident at once, 1..1024 (1 = one after another) */
    int32_t share_tables;    /* 1: force tables built once per nc, kept in the arena */
    int32_t graphs;          /* 1: steps replayed as CUDA graphs (pmpm_graph_mode) */
    int32_t priorities;      /* 0: one priority; 1: smaller boxes on higher-priority
                                streams; 2: larger boxes on higher-priority streams */
    int32_t steps_per_chunk; /* steps enqueued at a time per box (>= 1) */
    int32_t chunks_in_flight;/* chunks a box may have queued ahead (>= 1) */
    int32_t large_np;        /* boxes with np >= large_np are "large" (0: none is) */
    int32_t max_large;       /* large boxes resident at once (0: no limit); an arrived
                                large request over the limit is passed over by later
                                requests that can start, and keeps its place for the
                                next free large slot */
} pmpm_batch_config;

typedef struct pmpm_batch_stats {
    int64_t submitted, admitted, completed, failed;
    int64_t table_builds;    /* force-table computations (once per nc when shared) */
    int64_t launches;        /* library kernels launched for completed boxes */
    int64_t particle_steps;  /* of completed boxes */
    int64_t active;          /* boxes resident now */
    size_t  arena_used, arena_peak;
} pmpm_batch_stats;

typedef struct pmpm_batch pmpm_batch;

/* d_arena: device memory of arena_bytes, 256-byte aligned, owned by the
 * caller and borrowed until pmpm_batch_destroy.  Each admitted box takes
 * pmpm_workspace_bytes() of it; shared force tables stay in it for the
 * engine's life.  Every box gets its own non-blocking stream; set
 * CUDA_DEVICE_MAX_CONNECTIONS (up to 32) before the CUDA context exists so
 * that these streams do not share hardware queues.  The engine allocates
 * pinned host staging (max_active blocks of 49 KB) and no device memory. */
int pmpm_batch_create(const pmpm_batch_config* cfg, void* d_arena, size_t arena_bytes,
                      pmpm_batch** out);

/* Queue a request (copied; its host arrays must stay valid until its result
 * is polled).  PMPM_EINVAL for an invalid request, PMPM_ENOMEM when its
 * workspace is larger than the whole arena.  *id receives its id. */
int pmpm_batch_submit(pmpm_batch* batch, const pmpm_request* request, int64_t* id);

/* One scheduling pass without blocking on the device: retire finished
 * work, admit arrived requests (FIFO; the head waits for arena space), and
 * queue more steps.  *n_unfinished: requests queued or active. */
int pmpm_batch_progress(pmpm_batch* batch, int32_t* n_unfinished);

/* Call pmpm_batch_progress until every submitted request is finished, or
 * return PMPM_ETIMEOUT after max_seconds (the requests stay queued). */
int pmpm_batch_run(pmpm_batch* batch, double max_seconds);

/* Move up to max finished results into out; *n receives how many.  A request
 * that failed has a negative status (its message: pmpm_batch_last_error). */
int pmpm_batch_poll(pmpm_batch* batch, pmpm_result* out, int32_t max, int32_t* n);

/* Seconds since pmpm_batch_create on the engine's steady clock. */
double pmpm_batch_clock(const pmpm_batch* batch);

int pmpm_batch_get_stats(const pmpm_batch* batch, pmpm_batch_stats* out);

/* Wait for and release every box still resident; the arena is not freed. */
void pmpm_batch_destroy(pmpm_batch* batch);

/* Text of the last failure on this engine (or of pmpm_batch_create when NULL). */
const char* pmpm_batch_last_error(const pmpm_batch* batch);

/* sizeof pmpm_config, pmpm_scalars, pmpm_request, pmpm_result,
 * pmpm_batch_config, pmpm_batch_stats, for binding checks.  Host only. */
int pmpm_abi_sizes(int64_t* sizes, int32_t n);

/* Measurement only: FP32 fused multiply-add throughput of the current
 * device.  Launches out_len / 256 blocks of 256 threads on `stream` (a
 * cudaStream_t, NULL for the default stream); each thread runs 8
 * independent chains of `iters` FMAs and writes one float to d_out
 * (caller-owned device memory, out_len floats, out_len a multiple of 256).
 * Waits for the kernel; *flops receives 2 * 8 * iters * out_len and *ms the
 * kernel's duration between two events on the stream.  PMPM_EINVAL for bad
 * arguments, PMPM_ECUDA if a CUDA call fails. */
int pmpm_probe_fma(float* d_out, int64_t out_len, void* stream, int32_t iters, double* flops,
                   float* ms);

/* Host copies of the float32 velocity tables the library uses: T[256]
 * bin-centre values and E[256] bin edges (E[0] = -inf), Eq. 3.  Host only. */
int pmpm_codec_tables(float* T, float* E);

#ifdef __cplusplus
}
#endif

#endif /* PMPM_H */
