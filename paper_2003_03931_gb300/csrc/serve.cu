// serve.cu -- many independent PM-PM simulations resident on one GPU.
//
// The paper steps one box whose tiles are independent units processed in
// turn (Sec. II, Sec. IV-A).  A serving GPU holds many small boxes at once:
// each admitted request gets a workspace cut from one caller-owned device
// arena, its own stream, and the force tables of its coarse-mesh size
// (Sec. II), which are built once per nc and then copied.  Its steps are the
// same calls as pmpm_step, so a box evolves bit for bit as it would alone;
// only the interleaving on the device differs.
//
// Host side: one thread calls pmpm_batch_progress (or pmpm_batch_run).  Each
// call retires finished work (event queries, never a device-wide sync),
// admits arrived requests in FIFO order while a slot and arena space are
// free, and keeps every active box a bounded number of step chunks ahead.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <thread>
#include <vector>

#include "pmpm_impl.cuh"

// ------------------------------------------------------------------ arena
// Host-only bookkeeping of offsets into a device range.
struct pmpm_arena {
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;   // offset -> length, disjoint, never adjacent
    std::map<size_t, size_t> live;    // offset -> length
};

namespace pmpm {
namespace serve {

constexpr size_t kArenaAlign = 256;

int arena_init(pmpm_arena& a, size_t bytes) {
    a.size = bytes / kArenaAlign * kArenaAlign;
    a.used = a.peak = 0;
    a.free_.clear();
    a.live.clear();
    if (!a.size) return PMPM_EINVAL;
    a.free_[0] = a.size;
    return PMPM_OK;
}

int arena_alloc(pmpm_arena& a, size_t bytes, size_t* off) {
    if (bytes > a.size) return PMPM_ENOMEM;
    bytes = bytes ? (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign : kArenaAlign;
    for (auto it = a.free_.begin(); it != a.free_.end(); ++it) {
        if (it->second < bytes) continue;
        const size_t o = it->first, len = it->second;
        a.free_.erase(it);
        if (len > bytes) a.free_[o + bytes] = len - bytes;
        a.live[o] = bytes;
        a.used += bytes;
        a.peak = std::max(a.peak, a.used);
        *off = o;
        return PMPM_OK;
    }
    return PMPM_ENOMEM;
}

int arena_free(pmpm_arena& a, size_t off) {
    auto it = a.live.find(off);
    if (it == a.live.end()) return PMPM_EINVAL;
    size_t start = off, end = off + it->second;
    a.used -= it->second;
    a.live.erase(it);
    auto nx = a.free_.lower_bound(start);
    if (nx != a.free_.end() && nx->first == end) {
        end += nx->second;
        nx = a.free_.erase(nx);
    }
    if (nx != a.free_.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == start) {
            start = pv->first;
            a.free_.erase(pv);
        }
    }
    a.free_[start] = end - start;
    return PMPM_OK;
}

size_t arena_largest(const pmpm_arena& a) {
    size_t m = 0;
    for (const auto& f : a.free_) m = std::max(m, f.second);
    return m;
}

// ------------------------------------------------------------------ engine
constexpr int kPinDoubles = 3 * 2048 + 8;   // raw P(k) sums for nbins <= 2048, then sigma

struct Job {
    int64_t id = 0;
    pmpm_request r{};
    pmpm_config cfg{};
    size_t ws_bytes = 0, off = 0;
    bool has_ws = false;
    double t_admit = 0;
    pmpm_sim* sim = nullptr;
    cudaStream_t st = nullptr;
    int enq = 0;                        // steps enqueued
    std::deque<cudaEvent_t> inflight;   // one event after each enqueued chunk
    bool finishing = false;
    cudaEvent_t done_ev = nullptr;
    double* pin = nullptr;
};

struct Table {
    size_t off = 0;
    GreenRefs refs{};
};

}  // namespace serve
}  // namespace pmpm

struct pmpm_batch {
    pmpm_batch_config c{};
    uint8_t* base = nullptr;
    pmpm_arena arena;
    std::chrono::steady_clock::time_point t0;
    std::multimap<std::pair<double, int64_t>, pmpm::serve::Job*> queue;   // (arrival, id)
    std::vector<pmpm::serve::Job*> active;
    std::deque<pmpm_result> done;
    std::map<int, pmpm::serve::Table> tables;
    std::vector<cudaEvent_t> events;   // free completion events
    std::vector<double*> pins;         // free pinned staging blocks
    std::vector<double*> pins_all;
    int prio_least = 0, prio_greatest = 0;
    int device = 0;
    int64_t next_id = 1;
    pmpm_batch_stats stats{};
    char msg[512] = "";
};

namespace pmpm {
namespace serve {

char g_batch_msg[512] = "";

double now_s(const pmpm_batch& b) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - b.t0).count();
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool is_large(const pmpm_batch& b, int np) { return b.c.large_np > 0 && np >= b.c.large_np; }

// pmpm_config of a request; PMPM_OK when the sim and its P(k) mesh are valid
int request_config(const pmpm_request& r, pmpm_config* c, int* nmesh, int* nbins, char* msg,
                   size_t len) {
    memset(c, 0, sizeof(*c));
    c->np = r.np;
    c->nc = r.nc;
    c->tile_max = 5;
    c->buffer = kBuffer;
    c->pos_bytes = 1;
    c->vel_bytes = 1;
    c->a_init = r.a_init;
    c->a_final = r.a_final;
    c->n_steps = r.n_steps;
    if (r.flags & ~PMPM_FLAG_LOWMEM) return snprintf(msg, len, "unknown flags 0x%x", r.flags), PMPM_EINVAL;
    c->flags = r.flags;
    const int nf = 4 * r.nc;
    int m = r.pk_nmesh ? r.pk_nmesh : std::min(r.np, nf);
    if (!pow2(m) || m > nf || m < 4 || nf % m || nf / m > 4)
        return snprintf(msg, len, "pk_nmesh=%d must be a power of two in [4*nc/4, 4*nc]", m),
               PMPM_EINVAL;
    const int nb = r.pk_nbins ? r.pk_nbins : m / 2;
    if (nb < 1 || nb > m / 2)
        return snprintf(msg, len, "pk_nbins=%d must be in [1, %d]", nb, m / 2), PMPM_EINVAL;
    if (!r.k || !r.pk || !r.nmodes)
        return snprintf(msg, len, "k, pk and nmodes host arrays are required"), PMPM_EINVAL;
    if (r.n_steps < 1) return snprintf(msg, len, "n_steps must be >= 1"), PMPM_EINVAL;
    c->pk_mesh_max = m;
    *nmesh = m;
    *nbins = nb;
    return PMPM_OK;
}

cudaEvent_t take_event(pmpm_batch& b) {
    if (!b.events.empty()) {
        cudaEvent_t e = b.events.back();
        b.events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

// priorities 1: the smaller the box, the higher its stream's priority (short
// requests are not held up behind a large box's tile pass); 2: the larger the
// box, the higher (the large boxes, which make the latency tail, keep the
// GPU and the small ones fill the gaps)
int stream_priority(const pmpm_batch& b, int np) {
    if (!b.c.priorities) return 0;
    int level = 0;
    for (int v = np; v > 32; v >>= 1) ++level;
    if (b.c.priorities == 2) level = std::max(0, 3 - level);
    return std::min(b.prio_least, b.prio_greatest + level);   // greatest is numerically lowest
}

void release(pmpm_batch& b, Job* j) {
    if (j->st) cudaStreamSynchronize(j->st);
    for (cudaEvent_t e : j->inflight) b.events.push_back(e);
    j->inflight.clear();
    if (j->done_ev) b.events.push_back(j->done_ev);
    j->done_ev = nullptr;
    if (j->sim) pmpm_destroy(j->sim);
    j->sim = nullptr;
    if (j->st) cudaStreamDestroy(j->st);
    j->st = nullptr;
    if (j->has_ws) arena_free(b.arena, j->off);
    j->has_ws = false;
    if (j->pin) b.pins.push_back(j->pin);
    j->pin = nullptr;
}

void finish(pmpm_batch& b, Job* j, int status) {
    pmpm_result res{};
    res.id = j->id;
    res.status = status;
    res.t_arrival = j->r.arrival;
    res.t_admit = j->t_admit;
    if (status == PMPM_OK && j->sim) {
        int nmesh = 0, nbins = 0;
        pmpm_config c;
        char m[8];
        request_config(j->r, &c, &nmesh, &nbins, m, sizeof(m));
        power_spectrum_finish(j->pin, nbins, j->r.k, j->r.pk, j->r.nmodes);
        float sigma;
        memcpy(&sigma, j->pin + 3 * nbins, sizeof(float));
        res.sigma = sigma;
        res.a = j->sim->s.a;
        res.particle_steps = (int64_t)j->sim->s.n * j->r.n_steps;
        if (j->r.streams)
            status = pmpm_fetch(j->sim, PMPM_STREAMS, j->r.streams, 6 * (size_t)j->sim->s.n);
        if (!status && j->r.counts)
            status = pmpm_fetch(j->sim, PMPM_COUNTS, j->r.counts, 4 * (size_t)j->sim->s.ncells);
        if (status) snprintf(b.msg, sizeof(b.msg), "request %lld: %s", (long long)j->id,
                             pmpm_last_error(j->sim));
        res.status = status;
        b.stats.launches += j->sim->s.launches;
    }
    if (res.status == PMPM_OK) {
        b.stats.completed += 1;
        b.stats.particle_steps += res.particle_steps;
    } else {
        b.stats.failed += 1;
    }
    release(b, j);
    res.t_done = now_s(b);
    b.done.push_back(res);
    delete j;
}

void fail(pmpm_batch& b, Job* j, int rc, const char* what) {
    snprintf(b.msg, sizeof(b.msg), "request %lld: %s: %s", (long long)j->id, what,
             j->sim ? pmpm_last_error(j->sim) : init_message());
    finish(b, j, rc ? rc : PMPM_ECUDA);
}

// Workspace, stream and sim for the head request; false when it must wait.
// A request that cannot run at all is finished with its error here.
bool admit(pmpm_batch& b, Job* j) {
    if (arena_alloc(b.arena, j->ws_bytes, &j->off) != PMPM_OK) {
        if (!b.active.empty()) return false;
        // nothing left to free: the cached tables leave too little room
        snprintf(b.msg, sizeof(b.msg), "request %lld: %zu bytes never fit beside the cached tables",
                 (long long)j->id, j->ws_bytes);
        b.stats.admitted += 1;
        finish(b, j, PMPM_ENOMEM);
        return true;
    }
    j->has_ws = true;
    j->t_admit = now_s(b);
    b.stats.admitted += 1;
    if (cudaStreamCreateWithPriority(&j->st, cudaStreamNonBlocking, stream_priority(b, j->r.np)) !=
        cudaSuccess) {
        j->st = nullptr;
        fail(b, j, PMPM_ECUDA, "stream");
        return true;
    }
    j->pin = b.pins.back();
    b.pins.pop_back();
    int rc = PMPM_OK;
    auto t = b.tables.find(j->r.nc);
    const GreenRefs* refs = (b.c.share_tables && t != b.tables.end()) ? &t->second.refs : nullptr;
    j->sim = sim_create(&j->cfg, b.base + j->off, j->ws_bytes, j->st, refs, &rc);
    if (!j->sim) {
        fail(b, j, rc, "init");
        return true;
    }
    if (!refs) {
        b.stats.table_builds += 1;
        size_t part[3], off = 0;
        const size_t bytes = green_table_bytes(j->r.nc, part) + 2 * kArenaAlign;
        if (b.c.share_tables && arena_alloc(b.arena, bytes, &off) == PMPM_OK) {
            Table tb;
            tb.off = off;
            uint8_t* p = b.base + off;
            tb.refs.coarse = reinterpret_cast<const float4*>(p);
            p += (part[0] + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
            tb.refs.fine = reinterpret_cast<const float*>(p);
            p += (part[1] + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
            tb.refs.packed = reinterpret_cast<const float*>(p);
            rc = copy_tables(j->st, tb.refs, sim_tables(j->sim->s), j->r.nc);
            if (!rc && cudaStreamSynchronize(j->st) != cudaSuccess) rc = PMPM_ECUDA;
            if (rc) {
                arena_free(b.arena, off);
                fail(b, j, rc, "table cache");
                return true;
            }
            b.tables[j->r.nc] = tb;
        }
    }
    if (b.c.graphs && (rc = pmpm_graph_mode(j->sim, 1))) {
        fail(b, j, rc, "graph mode");
        return true;
    }
    if ((rc = pmpm_ic_zeldovich(j->sim, j->r.seed, j->r.slope, j->r.k_c, j->r.rms_disp))) {
        fail(b, j, rc, "initial conditions");
        return true;
    }
    b.active.push_back(j);
    return true;
}

// Queue more chunks for one active job, or its final P(k).  Returns false on failure
// (the job is then finished with its error).
bool advance(pmpm_batch& b, Job* j, bool* did) {
    while (!j->finishing && j->enq < j->r.n_steps && (int)j->inflight.size() < b.c.chunks_in_flight) {
        const int k = std::min(b.c.steps_per_chunk, j->r.n_steps - j->enq);
        int rc = pmpm_step(j->sim, k);
        cudaEvent_t e = rc ? nullptr : take_event(b);
        if (!rc && (!e || cudaEventRecord(e, j->st) != cudaSuccess)) rc = PMPM_ECUDA;
        if (rc) {
            if (e) b.events.push_back(e);
            fail(b, j, rc, "step");
            return false;
        }
        j->inflight.push_back(e);
        j->enq += k;
        *did = true;
    }
    if (!j->finishing && j->enq == j->r.n_steps) {
        int nmesh = 0, nbins = 0;
        pmpm_config c;
        char m[8];
        request_config(j->r, &c, &nmesh, &nbins, m, sizeof(m));
        Sim& s = j->sim->s;
        int rc = power_spectrum_enqueue(s, nmesh, nbins, j->pin);
        if (!rc && cudaMemcpyAsync(j->pin + 3 * nbins, s.sigma_d[s.cur], sizeof(float),
                                   cudaMemcpyDeviceToHost, j->st) != cudaSuccess)
            rc = PMPM_ECUDA;
        j->done_ev = rc ? nullptr : take_event(b);
        if (!rc && (!j->done_ev || cudaEventRecord(j->done_ev, j->st) != cudaSuccess)) rc = PMPM_ECUDA;
        if (rc) {
            fail(b, j, rc, "power spectrum");
            return false;
        }
        j->finishing = true;
        *did = true;
    }
    return true;
}

int progress(pmpm_batch& b, bool* did) {
    // 1. retire completed chunks; finish jobs whose result has landed
    for (size_t i = 0; i < b.active.size();) {
        Job* j = b.active[i];
        bool gone = false;
        while (!j->inflight.empty()) {
            const cudaError_t q = cudaEventQuery(j->inflight.front());
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) {
                b.active.erase(b.active.begin() + i);
                fail(b, j, PMPM_ECUDA, "event");
                gone = true;
                break;
            }
            b.events.push_back(j->inflight.front());
            j->inflight.pop_front();
            *did = true;
        }
        if (gone) continue;
        if (j->finishing) {
            const cudaError_t q = cudaEventQuery(j->done_ev);
            if (q != cudaErrorNotReady) {
                b.active.erase(b.active.begin() + i);
                const int rc = q == cudaSuccess ? pmpm_sync(j->sim) : PMPM_ECUDA;
                if (rc) fail(b, j, rc, "device");
                else finish(b, j, PMPM_OK);
                *did = true;
                continue;
            }
        }
        ++i;
    }
    // 2. admit arrived requests in FIFO order; a large request over the
    // large-box limit is passed over (it keeps its place in the queue)
    const double t = now_s(b);
    int n_large = 0;
    if (b.c.max_large > 0)
        for (Job* a : b.active) n_large += is_large(b, a->r.np);
    auto head = b.queue.begin();
    while ((int)b.active.size() < b.c.max_active && head != b.queue.end()) {
        if (head->first.first > t) break;
        Job* j = head->second;
        const bool large = b.c.max_large > 0 && is_large(b, j->r.np);
        if (large && n_large >= b.c.max_large) {
            ++head;
            continue;
        }
        if (!admit(b, j)) break;    // waits for arena space
        n_large += large;
        head = b.queue.erase(head);
        *did = true;
    }
    // 3. keep every active job chunks_in_flight chunks ahead
    for (size_t i = 0; i < b.active.size();) {
        Job* j = b.active[i];
        if (!advance(b, j, did)) {
            b.active.erase(std::find(b.active.begin(), b.active.end(), j));
            continue;
        }
        ++i;
    }
    b.stats.active = (int64_t)b.active.size();
    b.stats.arena_used = b.arena.used;
    b.stats.arena_peak = b.arena.peak;
    return PMPM_OK;
}

}  // namespace serve
}  // namespace pmpm

using namespace pmpm;
using namespace pmpm::serve;

extern "C" {

int pmpm_arena_create(size_t bytes, pmpm_arena** out) {
    if (!out) return PMPM_EINVAL;
    pmpm_arena* a = new (std::nothrow) pmpm_arena();
    if (!a) return PMPM_ENOMEM;
    if (arena_init(*a, bytes)) {
        delete a;
        return PMPM_EINVAL;
    }
    *out = a;
    return PMPM_OK;
}

int pmpm_arena_alloc(pmpm_arena* a, size_t bytes, size_t* offset) {
    if (!a || !offset) return PMPM_EINVAL;
    return arena_alloc(*a, bytes, offset);
}

int pmpm_arena_free(pmpm_arena* a, size_t offset) {
    if (!a) return PMPM_EINVAL;
    return arena_free(*a, offset);
}

int pmpm_arena_stats(const pmpm_arena* a, size_t* used, size_t* largest_free, int64_t* live) {
    if (!a) return PMPM_EINVAL;
    if (used) *used = a->used;
    if (largest_free) *largest_free = arena_largest(*a);
    if (live) *live = (int64_t)a->live.size();
    return PMPM_OK;
}

void pmpm_arena_destroy(pmpm_arena* a) { delete a; }

int pmpm_batch_create(const pmpm_batch_config* cfg, void* d_arena, size_t arena_bytes,
                      pmpm_batch** out) {
    if (!cfg || !out || !d_arena) return PMPM_EINVAL;
    if (cfg->max_active < 1 || cfg->max_active > 1024 || cfg->steps_per_chunk < 1 ||
        cfg->chunks_in_flight < 1 || cfg->priorities < 0 || cfg->priorities > 2 ||
        cfg->large_np < 0 || cfg->max_large < 0) {
        snprintf(g_batch_msg, sizeof(g_batch_msg),
                 "max_active in [1, 1024], steps_per_chunk >= 1, chunks_in_flight >= 1, "
                 "priorities 0, 1 or 2, large_np and max_large >= 0");
        return PMPM_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(d_arena) % kArenaAlign) {
        snprintf(g_batch_msg, sizeof(g_batch_msg), "arena must be 256-byte aligned");
        return PMPM_EINVAL;
    }
    pmpm_batch* b = new (std::nothrow) pmpm_batch();
    if (!b) return PMPM_ENOMEM;
    b->c = *cfg;
    b->base = static_cast<uint8_t*>(d_arena);
    if (arena_init(b->arena, arena_bytes)) {
        snprintf(g_batch_msg, sizeof(g_batch_msg), "arena smaller than 256 bytes");
        delete b;
        return PMPM_EINVAL;
    }
    cudaGetDevice(&b->device);
    cudaDeviceGetStreamPriorityRange(&b->prio_least, &b->prio_greatest);
    for (int i = 0; i < cfg->max_active; ++i) {
        double* p = nullptr;
        if (cudaHostAlloc(reinterpret_cast<void**>(&p), sizeof(double) * kPinDoubles,
                          cudaHostAllocDefault) != cudaSuccess) {
            snprintf(g_batch_msg, sizeof(g_batch_msg), "pinned staging allocation failed");
            for (double* q : b->pins_all) cudaFreeHost(q);
            delete b;
            return PMPM_ECUDA;
        }
        b->pins.push_back(p);
        b->pins_all.push_back(p);
    }
    b->t0 = std::chrono::steady_clock::now();
    *out = b;
    return PMPM_OK;
}

int pmpm_batch_submit(pmpm_batch* b, const pmpm_request* r, int64_t* id) {
    if (!b || !r) return PMPM_EINVAL;
    Job* j = new (std::nothrow) Job();
    if (!j) return PMPM_ENOMEM;
    j->r = *r;
    int nmesh = 0, nbins = 0;
    int rc = request_config(*r, &j->cfg, &nmesh, &nbins, b->msg, sizeof(b->msg));
    if (!rc && (rc = pmpm_workspace_bytes(&j->cfg, &j->ws_bytes)))
        snprintf(b->msg, sizeof(b->msg), "%s", pmpm_last_error(nullptr));
    if (!rc && j->ws_bytes > b->arena.size) {
        snprintf(b->msg, sizeof(b->msg), "request needs %zu bytes, arena holds %zu", j->ws_bytes,
                 b->arena.size);
        rc = PMPM_ENOMEM;
    }
    if (rc) {
        delete j;
        return rc;
    }
    j->id = b->next_id++;
    b->queue.emplace(std::make_pair(r->arrival, j->id), j);
    b->stats.submitted += 1;
    if (id) *id = j->id;
    return PMPM_OK;
}

int pmpm_batch_progress(pmpm_batch* b, int32_t* n_unfinished) {
    if (!b) return PMPM_EINVAL;
    bool did = false;
    const int rc = progress(*b, &did);
    if (n_unfinished) *n_unfinished = (int32_t)(b->queue.size() + b->active.size());
    return rc;
}

int pmpm_batch_run(pmpm_batch* b, double max_seconds) {
    if (!b) return PMPM_EINVAL;
    const double t_end = now_s(*b) + max_seconds;
    for (;;) {
        bool did = false;
        const int rc = progress(*b, &did);
        if (rc) return rc;
        if (b->queue.empty() && b->active.empty()) return PMPM_OK;
        if (now_s(*b) > t_end) {
            snprintf(b->msg, sizeof(b->msg), "pmpm_batch_run: %g s elapsed, %zu requests unfinished",
                     max_seconds, b->queue.size() + b->active.size());
            return PMPM_ETIMEOUT;
        }
        if (!did) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int pmpm_batch_poll(pmpm_batch* b, pmpm_result* out, int32_t max, int32_t* n) {
    if (!b || !n || (max > 0 && !out)) return PMPM_EINVAL;
    int32_t k = 0;
    while (k < max && !b->done.empty()) {
        out[k++] = b->done.front();
        b->done.pop_front();
    }
    *n = k;
    return PMPM_OK;
}

double pmpm_batch_clock(const pmpm_batch* b) { return b ? now_s(*b) : 0.0; }

int pmpm_batch_get_stats(const pmpm_batch* b, pmpm_batch_stats* out) {
    if (!b || !out) return PMPM_EINVAL;
    *out = b->stats;
    out->arena_used = b->arena.used;
    out->arena_peak = b->arena.peak;
    out->active = (int64_t)b->active.size();
    return PMPM_OK;
}

void pmpm_batch_destroy(pmpm_batch* b) {
    if (!b) return;
    for (Job* j : b->active) {
        release(*b, j);
        delete j;
    }
    for (auto& q : b->queue) delete q.second;
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    for (double* p : b->pins_all) cudaFreeHost(p);
    delete b;
}

const char* pmpm_batch_last_error(const pmpm_batch* b) { return b ? b->msg : g_batch_msg; }

int pmpm_abi_sizes(int64_t* sizes, int32_t n) {
    const int64_t v[] = {(int64_t)sizeof(pmpm_config), (int64_t)sizeof(pmpm_scalars),
                         (int64_t)sizeof(pmpm_request), (int64_t)sizeof(pmpm_result),
                         (int64_t)sizeof(pmpm_batch_config), (int64_t)sizeof(pmpm_batch_stats)};
    const int m = (int)(sizeof(v) / sizeof(v[0]));
    if (!sizes || n < m) return PMPM_EINVAL;
    for (int i = 0; i < m; ++i) sizes[i] = v[i];
    return PMPM_OK;
}

}  // extern "C"
