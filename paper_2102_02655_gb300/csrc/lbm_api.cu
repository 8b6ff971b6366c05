// Host side of the C ABI declared in include/lbm.h: argument checks, device
// state, the nozzle position per step (fixed point), and kernel enqueueing.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <type_traits>

#include "../../include/lbm.h"
#include "lbm_launch.h"

using namespace cglbm;

namespace {

constexpr double kFx = 1048576.0;  // 2^20: fixed-point unit of the nozzle position
constexpr int kBoxMargin = 3;      // sites kept in the nozzle box around the wall

char g_create_error[256] = "";

long long q20(double v) { return (long long)llround(v * kFx); }

long long mod_ll(long long a, long long m) {
    a %= m;
    return a < 0 ? a + m : a;
}

long long floor_div(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

}  // namespace

struct lbm_handle {
    lbm_config cfg;
    lbm_geometry geom;
    lbm_rheology rheo;
    bool have_geom = false, have_rheo = false;
    bool dead = false;  // sticky CUDA error
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the nozzle-box kernels run on a second stream, concurrently with the
    // bulk kernel (disjoint writes, shared read-only input), joined per step
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int Q = 19;
    long long N = 0, plane = 0;
    size_t esize = 8;  // bytes per real (compute type)
    size_t psize = 8;  // bytes per stored population
    size_t fdata = 0;  // bytes of populations in a buffer; 16-bit storage keeps the ink-fraction array after them
    // device buffers
    void* f[2] = {nullptr, nullptr};
    void* rho[2] = {nullptr, nullptr};
    void* u[2] = {nullptr, nullptr};
    void* fields = nullptr;
    double* acc = nullptr;
    int* flags = nullptr;
    int cur = 0;        // f[cur], rho[cur], u[cur] hold the latest state
    long long step = 0; // steps since lbm_set_geometry
    long long launches = 0;
    int zchunk = 32;
    int variant = 0;  // fused-kernel configuration (tuning knob CGLBM_FUSED_VARIANT)
    char err[256] = "";
    // event timing (lbm_profile)
    bool profiling = false;
    static constexpr int kMaxEv = 1024;
    cudaEvent_t ev[2][kMaxEv][2] = {};  // [bulk|plain][k][begin|end]
    int nev[2] = {0, 0};
    long long ev_sites[2][kMaxEv] = {};
    lbm_timing tot = {};
};

namespace {

lbm_status fail(lbm_handle* h, lbm_status st, const char* fmt, ...) {
    char* dst = h ? h->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

lbm_status cuda_check(lbm_handle* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LBM_OK;
    if (h) h->dead = true;
    return fail(h, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* dev_alloc(lbm_handle* h, size_t bytes) {
    void* p = nullptr;
    if (h->cfg.alloc) {
        p = h->cfg.alloc(bytes, h->cfg.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(lbm_handle* h, void* p) {
    if (!p) return;
    if (h->cfg.alloc) {
        if (h->cfg.free) h->cfg.free(p, h->cfg.alloc_ctx);
    } else {
        cudaFree(p);
    }
}

bool is_fused(const lbm_handle* h) {
    if (h->cfg.velset != LBM_D3Q19) return false;
    if (38.0 * (double)h->N >= 2147483647.0) return false;  // the fused kernel indexes in 32 bits
    if (h->geom.z_mode != LBM_Z_WALLS || h->geom.top_mode != LBM_TOP_OPEN) return false;
    return h->cfg.path != LBM_PATH_PLAIN;
}

template <typename real>
void fill_model(const lbm_handle* h, StepArgs<real>& p) {
    const lbm_config& c = h->cfg;
    p.nx = c.nx; p.ny = c.ny; p.nz = c.nz;
    p.N = h->N;
    p.plane = h->plane;
    p.rho0[0] = (real)c.rho0_ink;
    p.rho0[1] = (real)c.rho0_amb;
    p.zeta[0] = (real)c.zeta_ink;
    p.zeta[1] = (real)c.zeta_amb;
    p.A = (real)c.A;
    p.beta = (real)c.beta;
    p.rho_ref = (real)c.rho0_amb;
    p.nuB = (real)((c.tau_ambient - 0.5) / 3.0);
    for (int a = 0; a < 3; ++a) p.g[a] = (real)c.body_force[a];
    p.drag_gamma = (real)c.drag_gamma;
    p.drag_height = (real)c.drag_height;
    const bool d3 = c.velset == LBM_D3Q19;
    const double w0 = d3 ? 1.0 / 3.0 : 4.0 / 9.0;
    const double alpha[2] = {c.alpha_ink > 0 ? c.alpha_ink : w0, c.alpha_amb > 0 ? c.alpha_amb : w0};
    p.unit = (c.rho0_ink == c.rho0_amb && alpha[0] == w0 && alpha[1] == w0) ? 1 : 0;
    for (int k = 0; k < 2; ++k) {
        double pf = 0.0;
        for (int i = 0; i < h->Q; ++i) {
            const double share = d3 ? D3Q19::phi_share(i) : D2Q9::phi_share(i);
            const double ph = i == 0 ? alpha[k] : (1.0 - alpha[k]) * share;
            p.phi[k][i] = (real)ph;
            p.dphi[k][i] = (real)(ph - (d3 ? D3Q19::w(i) : D2Q9::w(i)));
            const int cx = d3 ? D3Q19::c(i, 0) : D2Q9::c(i, 0);
            pf += ph * cx * cx;
        }
        for (int i = h->Q; i < kMaxQ; ++i) p.phi[k][i] = p.dphi[k][i] = 0;
        p.pfac[k] = (real)pf;
    }
    const lbm_rheology& r = h->rheo;
    p.law = r.law;
    p.nu0 = (real)r.nu0;
    p.nu_inf = (real)r.nu_inf;
    p.lambda = (real)r.lambda;
    p.n_exp = (real)r.n;
    p.K = (real)r.K;
    p.tau_min = (real)r.tau_min;
    p.tau_max = (real)r.tau_max;
    const double tol_default = sizeof(real) == 8 ? 1e-14 : 1e-6;
    p.tol = (real)(r.tol > 0 ? std::max(r.tol, tol_default) : tol_default);
    p.max_iter = r.max_iter > 0 ? r.max_iter : 60;
}

// geometry of step n-1 (index 0) and step n (index 1)
template <typename real>
void fill_geometry(const lbm_handle* h, StepArgs<real>& p, long long n) {
    const lbm_geometry& g = h->geom;
    p.z_mode = g.z_mode;
    p.top_mode = g.top_mode;
    p.nozzle = (g.nozzle && g.z_mode == LBM_Z_WALLS) ? 1 : 0;
    p.gap = g.gap;
    p.px = (long long)h->cfg.nx * (long long)kFx;
    p.py = (long long)h->cfg.ny * (long long)kFx;
    const long long hx0 = q20(g.head_pos[0]), hy0 = q20(g.head_pos[1]);
    const long long vx = q20(g.head_vel[0]), vy = q20(g.head_vel[1]);
    const long long steps[2] = {n - 1 < 0 ? 0 : n - 1, n};
    for (int w = 0; w < 2; ++w) {
        p.hx[w] = mod_ll(hx0 + vx * steps[w], p.px);
        p.hy[w] = mod_ll(hy0 + vy * steps[w], p.py);
    }
    const long long ri = q20(g.r_inner), ro = q20(g.r_inner + g.wall_thickness);
    p.rin2 = ri * ri;
    p.rout2 = ro * ro;
    // bounds for "no neighbour can be a wall node": 3/2 l.u. (> sqrt 2) clear
    const long long rci = q20(std::max(0.0, g.r_inner - 1.5)), rco = q20(g.r_inner + g.wall_thickness + 1.5);
    p.rclear_in2 = g.r_inner > 1.5 ? rci * rci : -1;
    p.rclear_out2 = rco * rco;
    p.vn[0] = (real)((double)vx / kFx);
    p.vn[1] = (real)((double)vy / kFx);
    p.vn[2] = real(0);
    p.uin[0] = p.vn[0];
    p.uin[1] = p.vn[1];
    p.uin[2] = (real)(-g.u_ink);
    for (int a = 0; a < 3; ++a) p.utop[a] = (real)g.top_vel[a];
    p.rho_top = (real)g.rho_top_amb;
}

template <typename real>
void fill_buffers(lbm_handle* h, StepArgs<real>& p, int src) {
    const int dst = 1 - src;
    p.fin = h->f[src];
    p.fout = h->f[dst];
    if (h->psize == 2) {
        p.ref_in = (const real*)((const char*)h->f[src] + h->fdata);
        p.ref_out = (real*)((char*)h->f[dst] + h->fdata);
    }
    p.rho_prev = (const real*)h->rho[src];
    p.rho_cur = (real*)h->rho[dst];
    p.u_prev = (const real*)h->u[src];
    p.u_cur = (real*)h->u[dst];
    p.fields = (real*)h->fields;
    p.acc = h->acc;
    p.flags = h->flags;
    p.write_fields = 0;
    p.box = Region{0, 0, 0, 0, 0, 0};
}

Region full_region(const lbm_handle* h) { return Region{0, h->cfg.nx, 0, h->cfg.ny, 0, h->cfg.nz}; }

Region grow(const Region& r, int k, int nx, int ny, int nz) {
    Region o = r;
    if (r.wx + 2 * k >= nx) { o.x0 = 0; o.wx = nx; }
    else { o.x0 = (int)mod_ll(r.x0 - k, nx); o.wx = r.wx + 2 * k; }
    if (r.wy + 2 * k >= ny) { o.y0 = 0; o.wy = ny; }
    else { o.y0 = (int)mod_ll(r.y0 - k, ny); o.wy = r.wy + 2 * k; }
    o.z0 = std::max(0, r.z0 - k);
    o.z1 = std::min(nz, r.z1 + k);
    return o;
}

// box around the nozzle wall at steps n-1 and n, with kBoxMargin sites of margin
template <typename real>
Region nozzle_box(const lbm_handle* h, const StepArgs<real>& p) {
    const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
    if (!p.nozzle) return Region{0, 0, 0, 0, 0, 0};
    const long long ro = q20(h->geom.r_inner + h->geom.wall_thickness);
    const long long fx = (long long)kFx;
    const lbm_geometry& g = h->geom;
    const long long hx0 = q20(g.head_pos[0]), hy0 = q20(g.head_pos[1]);
    const long long vx = q20(g.head_vel[0]), vy = q20(g.head_vel[1]);
    const long long n1 = h->step + 1, n0 = h->step;
    const long long ax[2] = {hx0 + vx * n0, hx0 + vx * n1}, ay[2] = {hy0 + vy * n0, hy0 + vy * n1};
    const long long xlo = floor_div(std::min(ax[0], ax[1]) - ro, fx) - kBoxMargin;
    const long long xhi = floor_div(std::max(ax[0], ax[1]) + ro, fx) + 1 + kBoxMargin;
    const long long ylo = floor_div(std::min(ay[0], ay[1]) - ro, fx) - kBoxMargin;
    const long long yhi = floor_div(std::max(ay[0], ay[1]) + ro, fx) + 1 + kBoxMargin;
    Region b;
    if (xhi - xlo + 1 >= nx) { b.x0 = 0; b.wx = nx; }
    else { b.x0 = (int)mod_ll(xlo, nx); b.wx = (int)(xhi - xlo + 1); }
    if (yhi - ylo + 1 >= ny) { b.y0 = 0; b.wy = ny; }
    else { b.y0 = (int)mod_ll(ylo, ny); b.wy = (int)(yhi - ylo + 1); }
    b.z0 = std::max(0, g.gap - kBoxMargin);
    b.z1 = nz;
    return b;
}

// fold recorded events into the totals (waits for them)
lbm_status fold_events(lbm_handle* h) {
    for (int g = 0; g < 2; ++g) {
        for (int k = 0; k < h->nev[g]; ++k) {
            cudaError_t e = cudaEventSynchronize(h->ev[g][k][1]);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev[g][k][0], h->ev[g][k][1]);
            if (e != cudaSuccess) return cuda_check(h, e, "event timing");
            if (g == 0) {
                h->tot.bulk_ms += ms;
                h->tot.bulk_launches += 1;
                h->tot.bulk_sites += h->ev_sites[g][k];
            } else {
                h->tot.plain_ms += ms;
                h->tot.plain_groups += 1;
                h->tot.plain_sites += h->ev_sites[g][k];
            }
        }
        h->nev[g] = 0;
    }
    return LBM_OK;
}

// record the begin (end = false) or end event of a timed group on stream st
lbm_status mark(lbm_handle* h, int g, bool end, long long sites, cudaStream_t st) {
    if (!h->profiling) return LBM_OK;
    if (!end && h->nev[g] == lbm_handle::kMaxEv) {
        lbm_status st = fold_events(h);
        if (st != LBM_OK) return st;
    }
    const int k = h->nev[g];
    for (int b = 0; b < 2; ++b)
        if (!h->ev[g][k][b]) {
            cudaError_t e = cudaEventCreate(&h->ev[g][k][b]);
            if (e != cudaSuccess) return cuda_check(h, e, "cudaEventCreate");
        }
    cudaError_t e = cudaEventRecord(h->ev[g][k][end ? 1 : 0], st);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaEventRecord");
    if (end) {
        h->ev_sites[g][k] = sites;
        h->nev[g] = k + 1;
    }
    return LBM_OK;
}

template <class VS, typename real, typename S>
lbm_status do_steps(lbm_handle* h, int nsteps) {
    for (int t = 0; t < nsteps; ++t) {
        StepArgs<real> p;
        memset(&p, 0, sizeof(p));
        fill_model(h, p);
        fill_geometry(h, p, h->step + 1);
        fill_buffers(h, p, h->cur);
        const bool last = (t == nsteps - 1);
        if (last) {
            p.write_fields = 1;
            cudaError_t e = cudaMemsetAsync(h->acc + kAccMass, 0, 5 * sizeof(double), h->stream);
            if (e != cudaSuccess) return cuda_check(h, e, "cudaMemsetAsync");
        }
        const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
        int launched = 0;
        lbm_status st = LBM_OK;
        if (std::is_same<VS, D3Q19>::value && is_fused(h)) {
            const Region box = nozzle_box(h, p);
            p.box = box;
            const long long box_sites = (long long)box.wx * box.wy * (box.z1 - box.z0);
            if (box.wx > 0) {
                cudaError_t e = cudaEventRecord(h->fork, h->stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->fork, 0);
                if (e != cudaSuccess) return cuda_check(h, e, "fork");
                if ((st = mark(h, 1, false, 0, h->side)) != LBM_OK) return st;
                launched += launch_plain<VS, real, S>(p, box, grow(box, 1, nx, ny, nz), grow(box, 2, nx, ny, nz),
                                                      h->side);
                if ((st = mark(h, 1, true, box_sites, h->side)) != LBM_OK) return st;
            }
            if ((st = mark(h, 0, false, 0, h->stream)) != LBM_OK) return st;
            launched += launch_fused<real, S>(p, h->zchunk, h->stream, h->variant);
            if ((st = mark(h, 0, true, h->N - box_sites, h->stream)) != LBM_OK) return st;
            if (box.wx > 0) {
                cudaError_t e = cudaEventRecord(h->join, h->side);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->join, 0);
                if (e != cudaSuccess) return cuda_check(h, e, "join");
            }
        } else {
            const Region R = full_region(h);
            if ((st = mark(h, 1, false, 0, h->stream)) != LBM_OK) return st;
            launched += launch_plain<VS, real, S>(p, R, R, R, h->stream);
            if ((st = mark(h, 1, true, h->N, h->stream)) != LBM_OK) return st;
        }
        h->launches += launched;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(h, e, "kernel launch");
        h->cur = 1 - h->cur;
        h->step += 1;
    }
    return LBM_OK;
}

template <class VS, typename real, typename S>
lbm_status do_init(lbm_handle* h, int staged, int have_u) {
    StepArgs<real> p;
    memset(&p, 0, sizeof(p));
    fill_model(h, p);
    fill_geometry(h, p, h->step);
    fill_buffers(h, p, 1 - h->cur);  // writes go to buffer index cur
    cudaError_t e = cudaMemsetAsync(h->acc, 0, kAccN * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaMemsetAsync");
    h->launches += launch_init<VS, real, S>(p, staged, have_u, h->stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(h, e, "init launch");
    return LBM_OK;
}

lbm_status dispatch_init(lbm_handle* h, int staged, int have_u) {
    const bool d3 = h->cfg.velset == LBM_D3Q19;
    switch (h->cfg.storage) {
    case LBM_F64:
        return d3 ? do_init<D3Q19, double, double>(h, staged, have_u) : do_init<D2Q9, double, double>(h, staged, have_u);
    case LBM_F16DEV:
        return d3 ? do_init<D3Q19, float, __half>(h, staged, have_u) : do_init<D2Q9, float, __half>(h, staged, have_u);
    case LBM_BF16DEV:
        return d3 ? do_init<D3Q19, float, __nv_bfloat16>(h, staged, have_u)
                  : do_init<D2Q9, float, __nv_bfloat16>(h, staged, have_u);
    default:
        return d3 ? do_init<D3Q19, float, float>(h, staged, have_u) : do_init<D2Q9, float, float>(h, staged, have_u);
    }
}

lbm_status check_usable(lbm_handle* h) {
    if (!h) return LBM_EINVAL;
    if (h->dead) return fail(h, LBM_ECUDA, "handle unusable after an earlier CUDA error");
    cudaError_t e = cudaSetDevice(h->cfg.device);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaSetDevice");
    return LBM_OK;
}

bool finite_d(double v) { return std::isfinite(v); }

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_config* cfg, lbm_handle** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "lbm_create: out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, LBM_EINVAL, "lbm_create: cfg is NULL");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1)
        return fail(nullptr, LBM_EINVAL, "lbm_create: lattice sizes must be >= 1");
    if (cfg->velset != LBM_D2Q9 && cfg->velset != LBM_D3Q19)
        return fail(nullptr, LBM_EINVAL, "lbm_create: unknown velocity set %d", cfg->velset);
    if (cfg->velset == LBM_D2Q9 && cfg->ny != 1)
        return fail(nullptr, LBM_EINVAL, "lbm_create: D2Q9 lattices lie in the x-z plane, ny must be 1");
    if (cfg->storage < LBM_F64 || cfg->storage > LBM_BF16DEV)
        return fail(nullptr, LBM_EINVAL, "lbm_create: unknown storage %d", cfg->storage);
    if (cfg->path < LBM_PATH_AUTO || cfg->path > LBM_PATH_FUSED)
        return fail(nullptr, LBM_EINVAL, "lbm_create: unknown path %d", cfg->path);
    if (cfg->path == LBM_PATH_FUSED && cfg->velset != LBM_D3Q19)
        return fail(nullptr, LBM_EINVAL, "lbm_create: the fused path needs D3Q19");
    const double N = (double)cfg->nx * cfg->ny * cfg->nz;
    if (N > 4.0e9) return fail(nullptr, LBM_EINVAL, "lbm_create: lattice too large");
    if (!(cfg->tau_ambient > 0.5) || !finite_d(cfg->tau_ambient))
        return fail(nullptr, LBM_EINVAL, "lbm_create: tau_ambient must be > 1/2");
    if (!(cfg->rho0_ink > 0) || !(cfg->rho0_amb > 0))
        return fail(nullptr, LBM_EINVAL, "lbm_create: reference densities must be > 0");
    if (cfg->alpha_ink >= 1.0 || cfg->alpha_amb >= 1.0)
        return fail(nullptr, LBM_EINVAL, "lbm_create: alpha must be < 1");
    if (!(cfg->beta >= 0.0 && cfg->beta <= 1.0))
        return fail(nullptr, LBM_EINVAL, "lbm_create: beta must be in [0, 1]");
    if (!finite_d(cfg->A) || !(cfg->zeta_ink > 0) || !(cfg->zeta_amb > 0) || !finite_d(cfg->drag_gamma))
        return fail(nullptr, LBM_EINVAL, "lbm_create: invalid A, zeta or drag");
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
        return fail(nullptr, LBM_EINVAL, "lbm_create: alloc and free must be given together");

    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ENOMEM, "lbm_create: host allocation failed");
    h->cfg = *cfg;
    h->Q = cfg->velset == LBM_D3Q19 ? 19 : 9;
    h->plane = (long long)cfg->nx * cfg->ny;
    h->N = h->plane * cfg->nz;
    h->esize = cfg->storage == LBM_F64 ? 8 : 4;
    h->psize = cfg->storage == LBM_F64 ? 8 : (cfg->storage == LBM_F32 ? 4 : 2);
    {
        // z-planes per CTA of the fused kernel: about six waves of two CTAs
        // per SM (measured best on the 512x128x128 lattice: 16 planes), at
        // least 4 planes so the two-plane prologue stays amortised
        const long long tiles = (long long)((cfg->nx + 31) / 32) * ((cfg->ny + 7) / 8);
        long long chunks = (152LL * 12 + tiles - 1) / tiles;
        chunks = std::max(1LL, std::min<long long>(chunks, cfg->nz));
        h->zchunk = std::max(4, (int)((cfg->nz + chunks - 1) / chunks));
        if (const char* e = getenv("CGLBM_ZCHUNK")) h->zchunk = std::max(1, atoi(e));
        if (const char* e = getenv("CGLBM_FUSED_VARIANT")) h->variant = atoi(e);
    }

    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) {
        fail(nullptr, LBM_ECUDA, "lbm_create: cudaSetDevice(%d): %s", cfg->device, cudaGetErrorString(e));
        delete h;
        return LBM_ECUDA;
    }
    if (cfg->cuda_stream) {
        h->stream = (cudaStream_t)cfg->cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            fail(nullptr, LBM_ECUDA, "lbm_create: cudaStreamCreate: %s", cudaGetErrorString(e));
            delete h;
            return LBM_ECUDA;
        }
        h->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        fail(nullptr, LBM_ECUDA, "lbm_create: side stream: %s", cudaGetErrorString(e));
        lbm_destroy(h);
        return LBM_ECUDA;
    }
    h->fdata = ((size_t)2 * h->Q * h->N * h->psize + 255) & ~(size_t)255;
    const size_t fbytes = h->fdata + (h->psize == 2 ? (size_t)h->N * h->esize : 0);
    const size_t rbytes = (size_t)2 * (h->N + 2 * h->plane) * h->esize;
    const size_t ubytes = (size_t)3 * 2 * h->plane * h->esize;
    const size_t fldbytes = (size_t)kNFields * h->N * h->esize;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        ok = (h->f[b] = dev_alloc(h, fbytes)) && (h->rho[b] = dev_alloc(h, rbytes)) &&
             (h->u[b] = dev_alloc(h, ubytes));
    }
    ok = ok && (h->fields = dev_alloc(h, fldbytes)) && (h->acc = (double*)dev_alloc(h, kAccN * sizeof(double))) &&
         (h->flags = (int*)dev_alloc(h, 256));
    if (!ok) {
        lbm_destroy(h);
        return fail(nullptr, LBM_ENOMEM, "lbm_create: device allocation of %.3f GB failed",
                    (2.0 * fbytes + 2.0 * rbytes + 2.0 * ubytes + fldbytes) / 1e9);
    }
    for (int b = 0; b < 2; ++b) {
        e = cudaMemsetAsync(h->u[b], 0, ubytes, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->rho[b], 0, rbytes, h->stream);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->acc, 0, kAccN * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) {
        fail(nullptr, LBM_ECUDA, "lbm_create: cudaMemsetAsync: %s", cudaGetErrorString(e));
        lbm_destroy(h);
        return LBM_ECUDA;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_handle* h, const lbm_geometry* g) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (!g) return fail(h, LBM_EINVAL, "lbm_set_geometry: g is NULL");
    if (g->z_mode != LBM_Z_PERIODIC && g->z_mode != LBM_Z_WALLS)
        return fail(h, LBM_EINVAL, "lbm_set_geometry: unknown z_mode");
    if (g->top_mode != LBM_TOP_OPEN && g->top_mode != LBM_TOP_WALL)
        return fail(h, LBM_EINVAL, "lbm_set_geometry: unknown top_mode");
    for (int a = 0; a < 2; ++a)
        if (!finite_d(g->head_pos[a]) || !finite_d(g->head_vel[a]) || std::fabs(g->head_vel[a]) > 0.5)
            return fail(h, LBM_EINVAL, "lbm_set_geometry: head position/velocity invalid (|v| <= 0.5)");
    if (g->nozzle) {
        if (g->z_mode != LBM_Z_WALLS) return fail(h, LBM_EINVAL, "lbm_set_geometry: the nozzle needs z walls");
        if (g->gap < 1 || g->gap >= h->cfg.nz)
            return fail(h, LBM_EINVAL, "lbm_set_geometry: gap must be in [1, nz)");
        if (!(g->r_inner > 0) || !(g->wall_thickness > 0) || g->r_inner + g->wall_thickness > 1e5)
            return fail(h, LBM_EINVAL, "lbm_set_geometry: radii must be positive");
        if (!finite_d(g->u_ink) || std::fabs(g->u_ink) > 0.5)
            return fail(h, LBM_EINVAL, "lbm_set_geometry: |u_ink| must be <= 0.5");
    }
    if (!(g->rho_top_amb > 0) && g->z_mode == LBM_Z_WALLS && g->top_mode == LBM_TOP_OPEN)
        return fail(h, LBM_EINVAL, "lbm_set_geometry: rho_top_amb must be > 0");
    h->geom = *g;
    h->have_geom = true;
    h->step = 0;
    return dispatch_init(h, 0, 0);
}

lbm_status lbm_set_ink_rheology(lbm_handle* h, const lbm_rheology* r) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (!r) return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: r is NULL");
    if (!(r->tau_min > 0.5) || !(r->tau_max >= r->tau_min) || !finite_d(r->tau_max))
        return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: need 1/2 < tau_min <= tau_max");
    switch (r->law) {
    case LBM_NEWTONIAN:
        if (!(r->nu0 > 0)) return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: nu0 must be > 0");
        break;
    case LBM_CROSS:
        if (!(r->nu0 > 0) || !(r->nu_inf >= 0) || !(r->lambda > 0) || !(r->n > 0))
            return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: Cross needs nu0 > 0, nu_inf >= 0, lambda > 0, n > 0");
        break;
    case LBM_POWER_LAW:
        if (!(r->K > 0) || !(r->n > 0))
            return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: power law needs K > 0, n > 0");
        break;
    default:
        return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: unknown law %d", r->law);
    }
    h->rheo = *r;
    h->have_rheo = true;
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_handle* h, const void* rho_ink, const void* rho_amb, const void* u, int on_device) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (!h->have_geom) return fail(h, LBM_ESTATE, "lbm_set_fields: set the geometry first");
    if (!rho_ink || !rho_amb) return fail(h, LBM_EINVAL, "lbm_set_fields: densities are NULL");
    const size_t bytes = (size_t)h->N * h->esize;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    char* stage = (char*)h->fields;
    cudaError_t e = cudaMemcpyAsync(stage + kFRhoInk * bytes, rho_ink, bytes, kind, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + kFRhoAmb * bytes, rho_amb, bytes, kind, h->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(stage + kFUx * bytes, u, 3 * bytes, kind, h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "lbm_set_fields: copy");
    return dispatch_init(h, 1, u != nullptr);
}

lbm_status lbm_step(lbm_handle* h, int nsteps) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (!h->have_geom || !h->have_rheo) return fail(h, LBM_ESTATE, "lbm_step: geometry and rheology must be set");
    if (nsteps < 0) return fail(h, LBM_EINVAL, "lbm_step: nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    const bool d3 = h->cfg.velset == LBM_D3Q19;
    switch (h->cfg.storage) {
    case LBM_F64: return d3 ? do_steps<D3Q19, double, double>(h, nsteps) : do_steps<D2Q9, double, double>(h, nsteps);
    case LBM_F16DEV: return d3 ? do_steps<D3Q19, float, __half>(h, nsteps) : do_steps<D2Q9, float, __half>(h, nsteps);
    case LBM_BF16DEV:
        return d3 ? do_steps<D3Q19, float, __nv_bfloat16>(h, nsteps) : do_steps<D2Q9, float, __nv_bfloat16>(h, nsteps);
    default: return d3 ? do_steps<D3Q19, float, float>(h, nsteps) : do_steps<D2Q9, float, float>(h, nsteps);
    }
}

lbm_status lbm_sync(lbm_handle* h, int timeout_ms) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (timeout_ms <= 0) return cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(h->stream);
        if (e == cudaSuccess) return LBM_OK;
        if (e != cudaErrorNotReady) return cuda_check(h, e, "cudaStreamQuery");
        const auto dt = std::chrono::steady_clock::now() - t0;
        if (std::chrono::duration_cast<std::chrono::milliseconds>(dt).count() >= timeout_ms)
            return fail(h, LBM_ETIMEOUT, "lbm_sync: work still running after %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

lbm_status lbm_fields(lbm_handle* h, unsigned mask, void* const* dst, int dst_on_device, lbm_diag* diag) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (!h->have_geom) return fail(h, LBM_ESTATE, "lbm_fields: no state yet");
    if (mask & ~0x7Fu) return fail(h, LBM_EINVAL, "lbm_fields: unknown bits in mask");
    if (mask && !dst) return fail(h, LBM_EINVAL, "lbm_fields: dst is NULL");
    const size_t bytes = (size_t)h->N * h->esize;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const char* src = (const char*)h->fields;
    int slot = 0;
    struct { unsigned bit; int plane; int count; } tbl[] = {
        {LBM_FIELD_RHO_INK, kFRhoInk, 1}, {LBM_FIELD_RHO_AMB, kFRhoAmb, 1}, {LBM_FIELD_U, kFUx, 3},
        {LBM_FIELD_NU, kFNu, 1},          {LBM_FIELD_P, kFP, 1},            {LBM_FIELD_PHI, kFPhi, 1},
        {LBM_FIELD_SOLID, kFSolid, 1}};
    for (auto& t : tbl) {
        if (!(mask & t.bit)) continue;
        for (int c = 0; c < t.count; ++c, ++slot) {
            if (!dst[slot]) return fail(h, LBM_EINVAL, "lbm_fields: dst[%d] is NULL", slot);
            cudaError_t e = cudaMemcpyAsync(dst[slot], src + (size_t)(t.plane + c) * bytes, bytes, kind, h->stream);
            if (e != cudaSuccess) return cuda_check(h, e, "lbm_fields: copy");
        }
    }
    double acc[kAccN];
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(acc, h->acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "lbm_fields: sync");
    if (diag) {
        for (int k = 0; k < 2; ++k) {
            diag->mass[k] = acc[kAccMass + k];
            diag->bc_flux[k] = acc[kAccBc + k];
            diag->created[k] = acc[kAccCreated + k];
            diag->destroyed[k] = acc[kAccDestroyed + k];
        }
        for (int a = 0; a < 3; ++a) diag->momentum[a] = acc[kAccMom + a];
        diag->step = h->step;
        diag->unstable = flag ? 1 : 0;
    }
    if (flag) return fail(h, LBM_EUNSTABLE, "lbm_fields: a site's total density was not finite and positive");
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    cudaSetDevice(h->cfg.device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int b = 0; b < 2; ++b) {
        dev_free(h, h->f[b]);
        dev_free(h, h->rho[b]);
        dev_free(h, h->u[b]);
    }
    dev_free(h, h->fields);
    dev_free(h, h->acc);
    dev_free(h, h->flags);
    for (int g = 0; g < 2; ++g)
        for (int k = 0; k < lbm_handle::kMaxEv; ++k)
            for (int b = 0; b < 2; ++b)
                if (h->ev[g][k][b]) cudaEventDestroy(h->ev[g][k][b]);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err : g_create_error; }

long long lbm_kernel_launches(const lbm_handle* h) { return h ? h->launches : 0; }

lbm_status lbm_profile(lbm_handle* h, int enable) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (enable) {
        h->nev[0] = h->nev[1] = 0;
        h->tot = lbm_timing{};
    }
    h->profiling = enable != 0;
    return LBM_OK;
}

lbm_status lbm_timings(lbm_handle* h, lbm_timing* out) {
    lbm_status st = check_usable(h);
    if (st != LBM_OK) return st;
    if (!out) return fail(h, LBM_EINVAL, "lbm_timings: out is NULL");
    st = fold_events(h);
    if (st != LBM_OK) return st;
    *out = h->tot;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// lbm_step_noalloc: the work space of the step in a static device array
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[LBM_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[64] = {};  // device address of g_noalloc_scratch, per device

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory: the kernels get the address that the runtime reports for the
// current device, looked up once per device.
lbm_status noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(nullptr, LBM_ECUDA, "lbm_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = ptr;
    }
    *out = (unsigned char*)g_noalloc_addr[dev];
    return LBM_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

template <class VS, typename real>
lbm_status noalloc_step(lbm_handle* tmp, long long step, const void* f_in, void* f_out, void* fields, lbm_diag* diag,
                        unsigned char* scratch, cudaStream_t st) {
    StepArgs<real> p;
    memset(&p, 0, sizeof(p));
    fill_model(tmp, p);
    fill_geometry(tmp, p, step);
    const size_t es = sizeof(real);
    const size_t rbytes = round256(2 * (size_t)(tmp->N + 2 * tmp->plane) * es);
    const size_t ubytes = round256(6 * (size_t)tmp->plane * es);
    double* acc = (double*)scratch;
    int* flags = (int*)(scratch + 256);
    real* rho_prev = (real*)(scratch + 512);
    real* rho_cur = (real*)(scratch + 512 + rbytes);
    real* u_prev = (real*)(scratch + 512 + 2 * rbytes);
    real* u_cur = (real*)(scratch + 512 + 2 * rbytes + ubytes);
    // the accumulators and the flag must start at zero; the density and
    // velocity arrays are written before they are read
    cudaError_t e = cudaMemsetAsync(scratch, 0, 512, st);
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "lbm_step_noalloc: cudaMemsetAsync: %s", cudaGetErrorString(e));
    p.fin = f_in;
    p.fout = f_out;
    p.rho_prev = rho_prev;
    p.rho_cur = rho_cur;
    p.u_prev = u_prev;
    p.u_cur = u_cur;
    p.fields = (real*)fields;
    p.acc = acc;
    p.flags = flags;
    p.write_fields = fields ? 1 : 0;
    p.box = Region{0, 0, 0, 0, 0, 0};
    launch_prev_from_f<VS, real>(p, rho_prev, u_prev, st);
    const Region R = full_region(tmp);
    launch_plain<VS, real, real>(p, R, R, R, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "lbm_step_noalloc: launch: %s", cudaGetErrorString(e));
    if (!diag) return LBM_OK;
    double a[kAccN];
    int flag = 0;
    e = cudaMemcpyAsync(a, acc, sizeof(a), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "lbm_step_noalloc: diag: %s", cudaGetErrorString(e));
    for (int k = 0; k < 2; ++k) {
        diag->mass[k] = a[kAccMass + k];
        diag->bc_flux[k] = a[kAccBc + k];
        diag->created[k] = a[kAccCreated + k];
        diag->destroyed[k] = a[kAccDestroyed + k];
    }
    for (int c = 0; c < 3; ++c) diag->momentum[c] = a[kAccMom + c];
    diag->step = step;
    diag->unstable = flag ? 1 : 0;
    if (flag) return fail(nullptr, LBM_EUNSTABLE, "lbm_step_noalloc: a site's total density was not finite and positive");
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_config* cfg, const lbm_geometry* g, const lbm_rheology* r,
                                       long long step, const void* f_in, void* f_out, void* fields, lbm_diag* diag) {
    if (!cfg || !g || !r) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: cfg, g and r are required");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || (cfg->velset != LBM_D2Q9 && cfg->velset != LBM_D3Q19) ||
        (cfg->velset == LBM_D2Q9 && cfg->ny != 1) || (cfg->storage != LBM_F64 && cfg->storage != LBM_F32))
        return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: invalid lattice sizes, velocity set or storage");
    if (!(cfg->tau_ambient > 0.5) || !(cfg->rho0_ink > 0) || !(cfg->rho0_amb > 0) || cfg->alpha_ink >= 1.0 ||
        cfg->alpha_amb >= 1.0 || !(cfg->beta >= 0.0 && cfg->beta <= 1.0))
        return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: invalid model constants");
    if (!(r->tau_min > 0.5) || !(r->tau_max >= r->tau_min) || r->law < LBM_NEWTONIAN || r->law > LBM_POWER_LAW)
        return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: invalid rheology");
    if ((g->z_mode != LBM_Z_PERIODIC && g->z_mode != LBM_Z_WALLS) || (g->top_mode != LBM_TOP_OPEN && g->top_mode != LBM_TOP_WALL) ||
        (g->nozzle && (g->z_mode != LBM_Z_WALLS || g->gap < 1 || g->gap >= cfg->nz || !(g->r_inner > 0) ||
                       !(g->wall_thickness > 0))))
        return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: invalid geometry");
    if (step < 1) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: step must be >= 1");
    if (!f_in || !f_out) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: f_in and f_out are required");
    const int Q = cfg->velset == LBM_D3Q19 ? 19 : 9;
    const size_t es = cfg->storage == LBM_F64 ? 8 : 4;
    const long long plane = (long long)cfg->nx * cfg->ny, N = plane * cfg->nz;
    const size_t fbytes = (size_t)2 * Q * N * es;
    const char* a = (const char*)f_in;
    const char* b = (const char*)f_out;
    if (a < b + fbytes && b < a + fbytes) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: f_in and f_out overlap");
    const size_t need = 512 + 2 * round256(2 * (size_t)(N + 2 * plane) * es) + 2 * round256(6 * (size_t)plane * es);
    if (need > (size_t)LBM_NOALLOC_SCRATCH_BYTES)
        return fail(nullptr, LBM_EINVAL,
                    "lbm_step_noalloc: the lattice needs %zu bytes of work space, the static array holds %u", need,
                    (unsigned)LBM_NOALLOC_SCRATCH_BYTES);
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "lbm_step_noalloc: cudaSetDevice: %s", cudaGetErrorString(e));
    unsigned char* scratch = nullptr;
    lbm_status st = noalloc_scratch(cfg->device, &scratch);
    if (st != LBM_OK) return st;
    // the constants come from the same host code as lbm_step's, through a
    // handle object on the stack that owns no device memory
    lbm_handle tmp;
    tmp.cfg = *cfg;
    tmp.geom = *g;
    tmp.rheo = *r;
    tmp.Q = Q;
    tmp.plane = plane;
    tmp.N = N;
    tmp.esize = es;
    cudaStream_t stream = (cudaStream_t)cfg->cuda_stream;
    if (cfg->velset == LBM_D3Q19)
        return cfg->storage == LBM_F64 ? noalloc_step<D3Q19, double>(&tmp, step, f_in, f_out, fields, diag, scratch, stream)
                                       : noalloc_step<D3Q19, float>(&tmp, step, f_in, f_out, fields, diag, scratch, stream);
    return cfg->storage == LBM_F64 ? noalloc_step<D2Q9, double>(&tmp, step, f_in, f_out, fields, diag, scratch, stream)
                                   : noalloc_step<D2Q9, float>(&tmp, step, f_in, f_out, fields, diag, scratch, stream);
}
