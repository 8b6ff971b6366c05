// Serving: simulation requests (print parameters: ink viscosity law,
// extrusion rate, head velocity, nozzle size; Sec. III) arrive over time, are
// admitted in arrival order while their device memory fits an HBM budget and
// an active slot is free, and advance together as one batch (continuous
// batching: the batch's members are replaced whenever a request joins or
// leaves). A finished request's fields are copied to host memory and its slot
// goes to the next waiting request at once. Its lattice goes to a pool: a
// later request with the same lattice and model constants reuses it (new
// geometry, rheology and initial state), which spares the device allocation
// and release; pooled lattices count against the budget and are released,
// oldest first, when a request needs their memory.
//
// A client of the public C ABI only (lattices, batches); the caller drives it
// by submitting requests and calling lbm_server_poll.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "../../include/lbm.h"

namespace {

struct Request {
    long long id = 0;
    lbm_config cfg;
    lbm_geometry geom;
    lbm_rheology rheo;
    long long nsteps = 0, done = 0;
    long long bytes = 0;
    lbm_handle* h = nullptr;
    lbm_status status = LBM_OK;
    double t_submit = 0, t_admit = -1, t_done = -1;
    std::vector<unsigned char> fields;  // rho_ink, rho_amb, ux, uy, uz of the last step
    lbm_diag diag;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct Pooled {
    lbm_handle* h;
    lbm_config cfg;
    long long bytes;
};

struct lbm_server {
    lbm_server_config cfg;
    std::deque<Pooled> pool;                 // idle lattices, oldest first
    std::chrono::steady_clock::time_point t0;
    std::deque<Request*> waiting;
    std::vector<Request*> active;
    std::map<long long, Request*> finished;  // not yet collected
    long long used = 0;                      // device bytes of the active lattices
    lbm_batch* batch = nullptr;
    bool dirty = true;
    long long next_id = 1, rounds = 0, steps = 0, site_steps = 0, rebuilds = 0, reused = 0;
    int peak_active = 0;
    char err[256] = "";
};

namespace {

char g_server_error[256] = "";

lbm_status sfail(lbm_server* s, lbm_status st, const char* fmt, ...) {
    char* dst = s ? s->err : g_server_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

// release a request's lattice and give its memory back to the budget
void release(lbm_server* s, Request* r) {
    if (r->h) {
        lbm_destroy(r->h);
        r->h = nullptr;
        s->used -= r->bytes;
    }
}

// a lattice built for a can serve b: same sizes, velocity set, storage and
// model constants (geometry and rheology are set per request)
bool same_model(const lbm_config& a, const lbm_config& b) {
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.velset == b.velset && a.storage == b.storage &&
           a.tau_ambient == b.tau_ambient && a.rho0_ink == b.rho0_ink && a.rho0_amb == b.rho0_amb &&
           a.alpha_ink == b.alpha_ink && a.alpha_amb == b.alpha_amb && a.A == b.A && a.beta == b.beta &&
           a.zeta_ink == b.zeta_ink && a.zeta_amb == b.zeta_amb && a.drag_gamma == b.drag_gamma &&
           a.drag_height == b.drag_height && a.body_force[0] == b.body_force[0] &&
           a.body_force[1] == b.body_force[1] && a.body_force[2] == b.body_force[2];
}

// release pooled lattices, oldest first, until `need` more bytes fit
void evict(lbm_server* s, long long need) {
    while (!s->pool.empty() && s->used + need > (long long)s->cfg.hbm_budget) {
        lbm_destroy(s->pool.front().h);
        s->used -= s->pool.front().bytes;
        s->pool.pop_front();
    }
}

void finish(lbm_server* s, Request* r, lbm_status st) {
    r->status = st;
    r->t_done = now_s(s->t0);
    s->finished[r->id] = r;
}

// copy the fields of a finished request to host memory, then free its lattice
void retire(lbm_server* s, Request* r) {
    const size_t N = (size_t)r->cfg.nx * r->cfg.ny * r->cfg.nz;
    const size_t es = r->cfg.storage == LBM_F64 ? 8 : 4;
    r->fields.resize(5 * N * es);
    void* dst[5];
    for (int k = 0; k < 5; ++k) dst[k] = r->fields.data() + k * N * es;
    memset(&r->diag, 0, sizeof(r->diag));
    const lbm_status st = lbm_fields(r->h, LBM_FIELD_RHO_INK | LBM_FIELD_RHO_AMB | LBM_FIELD_U, dst, 0, &r->diag);
    if (st == LBM_OK) {
        s->pool.push_back(Pooled{r->h, r->cfg, r->bytes});  // still counted in `used`
        r->h = nullptr;
    } else {
        release(s, r);
    }
    finish(s, r, st);
}

lbm_status admit(lbm_server* s) {
    while (!s->waiting.empty() && (int)s->active.size() < s->cfg.max_active) {
        Request* r = s->waiting.front();
        if (r->bytes > (long long)s->cfg.hbm_budget) {
            s->waiting.pop_front();
            finish(s, r, sfail(s, LBM_ENOMEM, "request %lld needs %lld bytes, over the budget", r->id, r->bytes));
            continue;
        }
        lbm_handle* h = nullptr;
        bool reuse = false;
        for (auto it = s->pool.begin(); it != s->pool.end(); ++it)
            if (same_model(it->cfg, r->cfg)) {
                h = it->h;
                s->used -= it->bytes;  // counted again below as the request's
                s->pool.erase(it);
                reuse = true;
                break;
            }
        if (!reuse) {
            evict(s, r->bytes);
            if (s->used + r->bytes > (long long)s->cfg.hbm_budget) break;  // waits for memory
        }
        lbm_status st = reuse ? LBM_OK : lbm_create(&r->cfg, &h);
        if (st == LBM_OK) st = lbm_set_ink_rheology(h, &r->rheo);
        if (st == LBM_OK) st = lbm_set_geometry(h, &r->geom);
        if (reuse) s->reused += 1;
        if (st == LBM_ENOMEM && !s->active.empty()) {
            lbm_destroy(h);
            break;  // the device is fuller than the budget says: wait for a release
        }
        s->waiting.pop_front();
        if (st != LBM_OK) {
            sfail(s, st, "request %lld: %s", r->id, h ? lbm_last_error(h) : lbm_last_error(nullptr));
            lbm_destroy(h);
            finish(s, r, st);
            continue;
        }
        r->h = h;
        r->t_admit = now_s(s->t0);
        s->used += r->bytes;
        s->active.push_back(r);
        s->dirty = true;
    }
    s->peak_active = std::max(s->peak_active, (int)s->active.size());
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_server_create(const lbm_server_config* cfg, lbm_server** out) {
    if (!out) return sfail(nullptr, LBM_EINVAL, "lbm_server_create: out is NULL");
    *out = nullptr;
    if (!cfg || cfg->hbm_budget == 0 || cfg->quantum < 1 || cfg->max_active < 1)
        return sfail(nullptr, LBM_EINVAL, "lbm_server_create: budget, quantum and max_active must be positive");
    if (cfg->storage < LBM_F64 || cfg->storage > LBM_BF16DEV)
        return sfail(nullptr, LBM_EINVAL, "lbm_server_create: unknown storage %d", cfg->storage);
    lbm_server* s = new (std::nothrow) lbm_server();
    if (!s) return sfail(nullptr, LBM_ENOMEM, "lbm_server_create: host allocation failed");
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return LBM_OK;
}

lbm_status lbm_server_submit(lbm_server* s, const lbm_config* cfg, const lbm_geometry* g, const lbm_rheology* r,
                             long long nsteps, long long* id) {
    if (!s || !cfg || !g || !r) return sfail(s, LBM_EINVAL, "lbm_server_submit: NULL argument");
    if (nsteps < 1) return sfail(s, LBM_EINVAL, "lbm_server_submit: nsteps must be >= 1");
    Request* q = new (std::nothrow) Request();
    if (!q) return sfail(s, LBM_ENOMEM, "lbm_server_submit: host allocation failed");
    q->cfg = *cfg;
    // every request runs on the server's device, storage and the fused path,
    // with a stream and device memory of the library's own
    q->cfg.device = s->cfg.device;
    q->cfg.storage = s->cfg.storage;
    q->cfg.path = LBM_PATH_FUSED;
    q->cfg.cuda_stream = nullptr;
    q->cfg.alloc = nullptr;
    q->cfg.free = nullptr;
    q->cfg.alloc_ctx = nullptr;
    if (q->cfg.velset != LBM_D3Q19 || g->z_mode != LBM_Z_WALLS || g->top_mode != LBM_TOP_OPEN) {
        delete q;
        return sfail(s, LBM_EINVAL, "lbm_server_submit: requests are D3Q19 print runs (substrate, open top)");
    }
    q->geom = *g;
    q->rheo = *r;
    q->nsteps = nsteps;
    q->bytes = lbm_lattice_bytes(&q->cfg);
    if (q->bytes < 0) {
        delete q;
        return sfail(s, LBM_EINVAL, "lbm_server_submit: invalid lattice");
    }
    q->id = s->next_id++;
    q->t_submit = now_s(s->t0);
    s->waiting.push_back(q);
    if (id) *id = q->id;
    return LBM_OK;
}

lbm_status lbm_server_poll(lbm_server* s, int* n_finished) {
    if (!s) return sfail(nullptr, LBM_EINVAL, "lbm_server_poll: NULL server");
    const size_t before = s->finished.size();
    admit(s);
    if (!s->active.empty()) {
        if (s->dirty) {
            std::vector<lbm_handle*> hs;
            for (Request* r : s->active) hs.push_back(r->h);
            lbm_status st = s->batch ? lbm_batch_reset(s->batch, hs.data(), (int)hs.size())
                                     : lbm_batch_create(hs.data(), (int)hs.size(), &s->batch);
            if (st != LBM_OK)
                return sfail(s, st, "lbm_server_poll: batch: %s", lbm_batch_last_error(s->batch));
            s->dirty = false;
            s->rebuilds += 1;
        }
        // advance together, never past the nearest request's last step
        long long q = s->cfg.quantum;
        for (Request* r : s->active) q = std::min(q, r->nsteps - r->done);
        lbm_status st = lbm_batch_step(s->batch, (int)q);
        if (st == LBM_OK) st = lbm_batch_sync(s->batch);
        if (st != LBM_OK) return sfail(s, st, "lbm_server_poll: %s", lbm_batch_last_error(s->batch));
        s->rounds += 1;
        s->steps += q;
        std::vector<Request*> keep;
        for (Request* r : s->active) {
            r->done += q;
            s->site_steps += q * (long long)r->cfg.nx * r->cfg.ny * r->cfg.nz;
            if (r->done >= r->nsteps) {
                retire(s, r);
                s->dirty = true;
            } else {
                keep.push_back(r);
            }
        }
        s->active.swap(keep);
        admit(s);  // freed memory and slots go to waiting requests at once
    }
    if (n_finished) *n_finished = (int)(s->finished.size() - before);
    return LBM_OK;
}

int lbm_server_finished(const lbm_server* s, long long* ids, int cap) {
    if (!s) return 0;
    int n = 0;
    for (const auto& kv : s->finished) {
        if (ids && n < cap) ids[n] = kv.first;
        ++n;
    }
    return n;
}

lbm_status lbm_server_result(lbm_server* s, long long id, void* const* host_dst, lbm_diag* diag,
                             lbm_server_timing* timing) {
    if (!s) return sfail(nullptr, LBM_EINVAL, "lbm_server_result: NULL server");
    auto it = s->finished.find(id);
    if (it == s->finished.end()) return sfail(s, LBM_ESTATE, "lbm_server_result: request %lld not finished", id);
    Request* r = it->second;
    if (r->status == LBM_OK && host_dst) {
        const size_t N = (size_t)r->cfg.nx * r->cfg.ny * r->cfg.nz;
        const size_t es = r->cfg.storage == LBM_F64 ? 8 : 4;
        for (int k = 0; k < 5; ++k)
            if (host_dst[k]) memcpy(host_dst[k], r->fields.data() + k * N * es, N * es);
    }
    if (diag) *diag = r->diag;
    if (timing) {
        timing->t_submit = r->t_submit;
        timing->t_admit = r->t_admit;
        timing->t_done = r->t_done;
        timing->steps = r->done;
    }
    const lbm_status st = r->status;
    s->finished.erase(it);
    delete r;
    return st;
}

lbm_status lbm_server_stats(const lbm_server* s, lbm_server_counters* out) {
    if (!s || !out) return LBM_EINVAL;
    out->waiting = (int)s->waiting.size();
    out->active = (int)s->active.size();
    out->finished = (int)s->finished.size();
    out->peak_active = s->peak_active;
    out->bytes_in_use = s->used;
    out->rounds = s->rounds;
    out->batch_steps = s->steps;
    out->site_steps = s->site_steps;
    out->batch_rebuilds = s->rebuilds;
    out->reused = s->reused;
    out->pooled = (int)s->pool.size();
    out->clock = now_s(s->t0);
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* s) {
    if (!s) return;
    lbm_batch_destroy(s->batch);
    for (Request* r : s->active) {
        release(s, r);
        delete r;
    }
    for (Request* r : s->waiting) delete r;
    for (Pooled& p : s->pool) lbm_destroy(p.h);
    for (auto& kv : s->finished) delete kv.second;
    delete s;
}

const char* lbm_server_last_error(const lbm_server* s) { return s ? s->err : g_server_error; }

}  // extern "C"
