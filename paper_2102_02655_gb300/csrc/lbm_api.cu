// Host side of the C ABI declared in include/lbm.h: argument checks, device
// state, the nozzle position per step (fixed point), and kernel enqueueing.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_launch.h"

using namespace cglbm;

namespace {

constexpr double kFx = 1048576.0;  // 2^20: fixed-point unit of the nozzle position
constexpr int kBoxMargin = 3;      // sites kept in the nozzle box around the wall

char g_create_error[256] = "";

long long q20(double v) { return (long long)llround(v * kFx); }

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// The nozzle-box kernels run on a stream of the highest priority: their small
// grids then take SM slots first as the bulk kernel's CTAs retire, and the box
// chain ends before the bulk kernel instead of after it.
cudaError_t create_box_stream(cudaStream_t* st) {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return e;
    return cudaStreamCreateWithPriority(st, cudaStreamNonBlocking, greatest);
}

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
    unsigned char* geo = nullptr;  // per-column nozzle flags (nx * ny bytes)
    double* acc = nullptr;
    int* flags = nullptr;
    int cur = 0;        // f[cur], rho[cur], u[cur] hold the latest state
    long long step = 0; // steps since lbm_set_geometry
    long long launches = 0;
    int zchunk = 32;
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
    {
        // w_i rho_ref as the kernels round it, and the exact rounding offset of
        // their sums that the FP32 ink-stress split needs (see moments())
        double sw = 0.0, swx = 0.0;
        const double R = (double)p.rho_ref;
        for (int i = 0; i < h->Q; ++i) {
            const double w = c.velset == LBM_D3Q19 ? D3Q19::w(i) : D2Q9::w(i);
            const int cx = c.velset == LBM_D3Q19 ? D3Q19::c(i, 0) : D2Q9::c(i, 0);
            p.wref[i] = (real)(w * R);
            sw += (double)p.wref[i];
            swx += (double)p.wref[i] * cx * cx;
        }
        for (int i = h->Q; i < kMaxQ; ++i) p.wref[i] = 0;
        p.kappa_w = (real)((swx - R / 3.0) - (sw - R) / 3.0);
    }
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
    p.geo = h->geo;
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

// box around the nozzle wall at steps n0 and n0 + 1 (the step that n0 + 1
// completes), with kBoxMargin sites of margin
template <typename real>
Region nozzle_box(const lbm_handle* h, const StepArgs<real>& p, long long n0) {
    const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
    if (!p.nozzle) return Region{0, 0, 0, 0, 0, 0};
    const long long ro = q20(h->geom.r_inner + h->geom.wall_thickness);
    const long long fx = (long long)kFx;
    const lbm_geometry& g = h->geom;
    const long long hx0 = q20(g.head_pos[0]), hy0 = q20(g.head_pos[1]);
    const long long vx = q20(g.head_vel[0]), vy = q20(g.head_vel[1]);
    const long long n1 = n0 + 1;
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
            const Region box = nozzle_box(h, p, h->step);
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
            launched += launch_fused<real, S>(p, h->zchunk, h->stream);
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

// Makes a handle's device current for the duration of an API call and gives
// the caller's current device back on return.
struct DeviceScope {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) err = cudaSetDevice(dev);
        else prev = -1;  // nothing to give back
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

lbm_status check_usable(lbm_handle* h, const DeviceScope& ds) {
    if (h->dead) return fail(h, LBM_ECUDA, "handle unusable after an earlier CUDA error");
    if (ds.err != cudaSuccess) return cuda_check(h, ds.err, "cudaSetDevice");
    return LBM_OK;
}

bool finite_d(double v) { return std::isfinite(v); }
bool all_finite(const double* v, int n) {
    for (int k = 0; k < n; ++k)
        if (!finite_d(v[k])) return false;
    return true;
}

// Largest lattice side (x, y) and nozzle radius r_inner + wall_thickness
// (lattice units) of a run with a nozzle: the fixed-point geometry squares
// distances of up to half a side, and the radii, in units of 2^-20 in 64-bit
// integers, which stays exact below these bounds (2 (2000 * 2^20)^2 < 2^63).
constexpr int kMaxNozzleSide = 4000;
constexpr double kMaxNozzleRadius = 2000.0;

// The checks every entry point applies to a configuration, a geometry and a
// rheology. Each returns nullptr when the argument is valid, else what is
// wrong with it.
const char* config_problem(const lbm_config* c) {
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return "lattice sizes must be >= 1";
    if (c->velset != LBM_D2Q9 && c->velset != LBM_D3Q19) return "unknown velocity set";
    if (c->velset == LBM_D2Q9 && c->ny != 1) return "D2Q9 lattices lie in the x-z plane, ny must be 1";
    if (c->storage < LBM_F64 || c->storage > LBM_BF16DEV) return "unknown storage";
    if (c->path < LBM_PATH_AUTO || c->path > LBM_PATH_FUSED) return "unknown path";
    if (c->path == LBM_PATH_FUSED && c->velset != LBM_D3Q19) return "the fused path needs D3Q19";
    if ((double)c->nx * c->ny * c->nz > 4.0e9) return "lattice too large";
    if (!(c->tau_ambient > 0.5) || !finite_d(c->tau_ambient)) return "tau_ambient must be > 1/2 and finite";
    if (!(c->rho0_ink > 0) || !(c->rho0_amb > 0) || !finite_d(c->rho0_ink) || !finite_d(c->rho0_amb))
        return "reference densities must be > 0 and finite";
    if (!(c->alpha_ink < 1.0) || !(c->alpha_amb < 1.0)) return "alpha must be < 1";
    if (!(c->beta >= 0.0 && c->beta <= 1.0)) return "beta must be in [0, 1]";
    if (!finite_d(c->A) || !(c->zeta_ink > 0) || !(c->zeta_amb > 0) || !finite_d(c->zeta_ink) ||
        !finite_d(c->zeta_amb) || !finite_d(c->drag_gamma) || !finite_d(c->drag_height) ||
        !all_finite(c->body_force, 3))
        return "invalid A, zeta, drag or body force";
    if ((c->alloc == nullptr) != (c->free == nullptr)) return "alloc and free must be given together";
    return nullptr;
}

const char* geometry_problem(const lbm_config* c, const lbm_geometry* g) {
    if (g->z_mode != LBM_Z_PERIODIC && g->z_mode != LBM_Z_WALLS) return "unknown z_mode";
    if (g->top_mode != LBM_TOP_OPEN && g->top_mode != LBM_TOP_WALL) return "unknown top_mode";
    for (int a = 0; a < 2; ++a)
        if (!finite_d(g->head_pos[a]) || !finite_d(g->head_vel[a]) || std::fabs(g->head_vel[a]) > 0.5)
            return "head position/velocity invalid (finite, |v| <= 0.5)";
    if (!all_finite(g->top_vel, 3)) return "top_vel must be finite";
    if (g->nozzle) {
        if (g->z_mode != LBM_Z_WALLS) return "the nozzle needs z walls";
        if (g->gap < 1 || g->gap >= c->nz) return "gap must be in [1, nz)";
        if (!(g->r_inner > 0) || !(g->wall_thickness > 0) || !(g->r_inner + g->wall_thickness <= kMaxNozzleRadius))
            return "radii must be positive with r_inner + wall_thickness <= 2000";
        if (c->nx > kMaxNozzleSide || c->ny > kMaxNozzleSide) return "a nozzle run needs nx, ny <= 4000";
        if (!finite_d(g->u_ink) || std::fabs(g->u_ink) > 0.5) return "|u_ink| must be <= 0.5";
    }
    if (g->z_mode == LBM_Z_WALLS && g->top_mode == LBM_TOP_OPEN && !(g->rho_top_amb > 0 && finite_d(g->rho_top_amb)))
        return "rho_top_amb must be > 0 and finite";
    return nullptr;
}

const char* rheology_problem(const lbm_rheology* r) {
    if (!(r->tau_min > 0.5) || !(r->tau_max >= r->tau_min) || !finite_d(r->tau_max))
        return "need 1/2 < tau_min <= tau_max, finite";
    if (!finite_d(r->tol) || r->tol < 0 || r->max_iter < 0) return "tol and max_iter must be >= 0";
    switch (r->law) {
    case LBM_NEWTONIAN:
        if (!(r->nu0 > 0) || !finite_d(r->nu0)) return "nu0 must be > 0 and finite";
        return nullptr;
    case LBM_CROSS:
        if (!(r->nu0 > 0) || !(r->nu_inf >= 0) || !(r->lambda > 0) || !(r->n > 0) || !finite_d(r->nu0) ||
            !finite_d(r->nu_inf) || !finite_d(r->lambda) || !finite_d(r->n))
            return "Cross needs finite nu0 > 0, nu_inf >= 0, lambda > 0, n > 0";
        return nullptr;
    case LBM_POWER_LAW:
        if (!(r->K > 0) || !(r->n > 0) || !finite_d(r->K) || !finite_d(r->n))
            return "power law needs finite K > 0, n > 0";
        return nullptr;
    default:
        return "unknown law";
    }
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_config* cfg, lbm_handle** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "lbm_create: out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, LBM_EINVAL, "lbm_create: cfg is NULL");
    if (const char* m = config_problem(cfg)) return fail(nullptr, LBM_EINVAL, "lbm_create: %s", m);

    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ENOMEM, "lbm_create: host allocation failed");
    h->cfg = *cfg;
    h->Q = cfg->velset == LBM_D3Q19 ? 19 : 9;
    h->plane = (long long)cfg->nx * cfg->ny;
    h->N = h->plane * cfg->nz;
    h->esize = cfg->storage == LBM_F64 ? 8 : 4;
    h->psize = cfg->storage == LBM_F64 ? 8 : (cfg->storage == LBM_F32 ? 4 : 2);
    {
        // z-planes per CTA of the fused kernel: about four waves of CTAs
        // (152 SMs), at least 4 planes so the two-plane prologue stays
        // amortised
        const bool fp64 = cfg->storage == LBM_F64;
        const long long tiles = (long long)((cfg->nx + 31) / 32) * ((cfg->ny + kFusedTileH - 1) / kFusedTileH);
        long long chunks = (152LL * 4 * fused_ctas_per_sm(fp64) + tiles - 1) / tiles;
        chunks = std::max(1LL, std::min<long long>(chunks, cfg->nz));
        h->zchunk = std::max(4, (int)((cfg->nz + chunks - 1) / chunks));
        if (const char* e = getenv("CGLBM_ZCHUNK")) h->zchunk = std::max(1, atoi(e));
    }

    DeviceScope ds(cfg->device);
    cudaError_t e = ds.err;
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
    e = create_box_stream(&h->side);
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
    ok = ok && (h->geo = (unsigned char*)dev_alloc(h, round256((size_t)h->plane))) &&
         (h->fields = dev_alloc(h, fldbytes)) && (h->acc = (double*)dev_alloc(h, kAccN * sizeof(double))) &&
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
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
    if (st != LBM_OK) return st;
    if (!g) return fail(h, LBM_EINVAL, "lbm_set_geometry: g is NULL");
    if (const char* m = geometry_problem(&h->cfg, g)) return fail(h, LBM_EINVAL, "lbm_set_geometry: %s", m);
    h->geom = *g;
    h->have_geom = true;
    h->step = 0;
    return dispatch_init(h, 0, 0);
}

lbm_status lbm_set_ink_rheology(lbm_handle* h, const lbm_rheology* r) {
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
    if (st != LBM_OK) return st;
    if (!r) return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: r is NULL");
    if (const char* m = rheology_problem(r)) return fail(h, LBM_EINVAL, "lbm_set_ink_rheology: %s", m);
    h->rheo = *r;
    h->have_rheo = true;
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_handle* h, const void* rho_ink, const void* rho_amb, const void* u, int on_device) {
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
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
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
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
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
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
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
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
        diag->unstable = (flag & 1) ? 1 : 0;
    }
    if (flag & 2) {
        h->dead = true;  // a kernel left its step unfinished
        return fail(h, LBM_ETIMEOUT, "lbm_fields: a bounded wait inside a kernel ran out; the state is lost");
    }
    if (flag) return fail(h, LBM_EUNSTABLE, "lbm_fields: a site's total density was not finite and positive");
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    DeviceScope ds(h->cfg.device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int b = 0; b < 2; ++b) {
        dev_free(h, h->f[b]);
        dev_free(h, h->rho[b]);
        dev_free(h, h->u[b]);
    }
    dev_free(h, h->fields);
    dev_free(h, h->geo);
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
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
    if (st != LBM_OK) return st;
    if (enable) {
        h->nev[0] = h->nev[1] = 0;
        h->tot = lbm_timing{};
    }
    h->profiling = enable != 0;
    return LBM_OK;
}

lbm_status lbm_timings(lbm_handle* h, lbm_timing* out) {
    if (!h) return LBM_EINVAL;
    DeviceScope ds(h->cfg.device);
    lbm_status st = check_usable(h, ds);
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

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory: the kernels get the address the runtime reports for the current
// device, looked up on every call (no allocation; a device reset between
// calls cannot leave a stale address behind).
lbm_status noalloc_scratch(unsigned char** out) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
        return fail(nullptr, LBM_ECUDA, "lbm_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    *out = (unsigned char*)ptr;
    return LBM_OK;
}


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
    unsigned char* geo = scratch + 512 + 2 * rbytes + 2 * ubytes;  // nx * ny bytes
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
    p.geo = geo;
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
    // the same checks as lbm_create, lbm_set_geometry and lbm_set_ink_rheology
    lbm_config c = *cfg;
    c.path = LBM_PATH_PLAIN;
    c.alloc = nullptr;
    c.free = nullptr;
    if (const char* m = config_problem(&c)) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: %s", m);
    if (cfg->storage != LBM_F64 && cfg->storage != LBM_F32)
        return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: storage must be LBM_F64 or LBM_F32");
    if (const char* m = geometry_problem(cfg, g)) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: %s", m);
    if (const char* m = rheology_problem(r)) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: %s", m);
    if (step < 1) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: step must be >= 1");
    if (!f_in || !f_out) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: f_in and f_out are required");
    const int Q = cfg->velset == LBM_D3Q19 ? 19 : 9;
    const size_t es = cfg->storage == LBM_F64 ? 8 : 4;
    const long long plane = (long long)cfg->nx * cfg->ny, N = plane * cfg->nz;
    const size_t fbytes = (size_t)2 * Q * N * es;
    const char* a = (const char*)f_in;
    const char* b = (const char*)f_out;
    if (a < b + fbytes && b < a + fbytes) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: f_in and f_out overlap");
    const size_t need = 512 + 2 * round256(2 * (size_t)(N + 2 * plane) * es) + 2 * round256(6 * (size_t)plane * es) +
                        round256((size_t)plane);
    if (need > (size_t)LBM_NOALLOC_SCRATCH_BYTES)
        return fail(nullptr, LBM_EINVAL,
                    "lbm_step_noalloc: the lattice needs %zu bytes of work space, the static array holds %u", need,
                    (unsigned)LBM_NOALLOC_SCRATCH_BYTES);
    DeviceScope ds(cfg->device);
    if (ds.err != cudaSuccess)
        return fail(nullptr, LBM_ECUDA, "lbm_step_noalloc: cudaSetDevice: %s", cudaGetErrorString(ds.err));
    unsigned char* scratch = nullptr;
    lbm_status st = noalloc_scratch(&scratch);
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

// ---------------------------------------------------------------------------
// Batches: many lattices advanced together. Per step, one persistent launch
// covers the bulk of every lattice (a work list of tile columns), and one
// launch per phase covers the nozzle boxes of every lattice; G steps are
// captured once in a CUDA graph and replayed, each replay reading the step
// arguments of its G steps from a device table the host refreshes.
// ---------------------------------------------------------------------------

struct lbm_batch {
    std::vector<lbm_handle*> lat;
    int device = 0, storage = LBM_F32, unit = 1;
    cudaStream_t stream = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, done = nullptr, t0 = nullptr, t1 = nullptr;
    std::vector<cudaEvent_t> hev;  // one per lattice: its stream's work before the batch's
    // plan: fused-kernel variant, z-planes per column for each lattice
    int variant = 0;
    std::vector<int> zchunk;
    int4* d_items = nullptr;
    size_t items_cap = 0;
    int* d_queue = nullptr;  // one work-queue counter per captured step
    int n_items = 0, grid = 0;
    int occ = 0;          // resident CTAs per SM of the bulk kernel's configuration
    int ctas_per_sm = 0;  // CTAs per SM the persistent grid uses (0: all of occ)
    unsigned box_gx = 0, box_gy = 0;
    // step tables: [G][L] StepArgs, then [G][L] BoxArgs
    int G = 16;
    size_t args_bytes = 0, box_bytes = 0;
    void* d_tab = nullptr;
    void* h_tab[2] = {nullptr, nullptr};
    cudaEvent_t h_ev[2] = {nullptr, nullptr};
    int hbuf = 0;
    // captured graphs: [0] for G steps, [1] for the last remainder size
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int exec_g[2] = {0, 0};
    bool exec_valid = false;
    long long launches = 0, steps = 0;
    bool dead = false;
    char err[256] = "";
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const char* fmt, ...) {
    char* dst = b ? b->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

lbm_status bcuda(lbm_batch* b, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LBM_OK;
    b->dead = true;
    return bfail(b, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Work list of the persistent bulk kernel: for each lattice, its tile columns
// (32 x tile_h sites) of each z-chunk, lattice-major then chunk, row, column,
// so that the CTAs running at one time work on neighbouring columns of one
// lattice (their halo re-reads then hit L2). Returns the item count; writes
// at most cap items.
long long plan_items(const int* dims, int n, int tile_h, const int* zchunk, int* out, long long cap) {
    long long k = 0;
    for (int l = 0; l < n; ++l) {
        const int nx = dims[3 * l], ny = dims[3 * l + 1], nz = dims[3 * l + 2];
        const int nch = z_chunks(nz, std::max(1, zchunk[l]));
        for (int c = 0; c < nch; ++c)
            for (int y0 = 0; y0 < ny; y0 += tile_h)
                for (int x0 = 0; x0 < nx; x0 += 32) {
                    if (k < cap && out) {
                        out[4 * k] = l;
                        out[4 * k + 1] = x0 | (y0 << 16);
                        out[4 * k + 2] = z_chunk_begin(nz, nch, c);
                        out[4 * k + 3] = z_chunk_begin(nz, nch, c + 1);
                    }
                    ++k;
                }
    }
    return k;
}

template <typename real, typename S>
lbm_status batch_plan(lbm_batch* b, int variant, const std::vector<int>& zc) {
    const int L = (int)b->lat.size();
    const int th = kFusedTileH;
    std::vector<int> dims(3 * L);
    for (int l = 0; l < L; ++l) {
        dims[3 * l] = b->lat[l]->cfg.nx;
        dims[3 * l + 1] = b->lat[l]->cfg.ny;
        dims[3 * l + 2] = b->lat[l]->cfg.nz;
    }
    const long long n = plan_items(dims.data(), L, th, zc.data(), nullptr, 0);
    if (n > 0x7fffffffLL) return bfail(b, LBM_EINVAL, "lbm_batch: work list too long");
    std::vector<int> items(4 * n);
    plan_items(dims.data(), L, th, zc.data(), items.data(), n);
    cudaError_t e = cudaSuccess;
    if ((size_t)n > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        e = cudaMalloc(&b->d_items, (size_t)n * sizeof(int4));
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->items_cap = 0;
            return bfail(b, LBM_ENOMEM, "lbm_batch: work list allocation failed");
        }
        b->items_cap = (size_t)n;
    }
    e = cudaMemcpyAsync(b->d_items, items.data(), (size_t)n * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch: work list upload");
    int occ = 0, sms = 0;
    launch_fused_batch<real, S>(nullptr, nullptr, 0, nullptr, 0, b->unit, b->stream, &occ);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return bcuda(b, e, "cudaDeviceGetAttribute");
    b->n_items = (int)n;
    // fewer CTAs per SM than fit leave room for the box kernels beside the
    // persistent bulk kernel (a tuning choice)
    b->occ = std::max(1, occ);
    const int use = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, b->occ) : b->occ;
    b->grid = (int)std::max(1LL, std::min<long long>(n, (long long)use * sms));
    b->variant = variant;
    b->zchunk = zc;
    b->exec_valid = false;
    return LBM_OK;
}

// grid of the batched box kernels: the largest grown box (columns, planes)
// with two sites of slack per side, so that the box can move for a while
// before the captured graph needs a larger grid
void box_grid(const Region& R2, const Region& R1g, unsigned* gx, unsigned* gy) {
    const long long cols = (long long)(R2.wx + 4) * (R2.wy + 4);
    *gx = std::max(*gx, (unsigned)((cols + kBoxThreads - 1) / kBoxThreads));
    *gy = std::max(*gy, (unsigned)std::max(R2.z1 - R2.z0, R1g.z1 - R1g.z0));
}

template <typename real, typename S>
lbm_status batch_capture(lbm_batch* b, int slot, int g) {
    if (b->exec[slot]) {
        cudaGraphExecDestroy(b->exec[slot]);
        b->exec[slot] = nullptr;
    }
    const int L = (int)b->lat.size();
    const StepArgs<real>* args = (const StepArgs<real>*)b->d_tab;
    const BoxArgs<real>* box = (const BoxArgs<real>*)((const char*)b->d_tab + (size_t)b->G * L * sizeof(StepArgs<real>));
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch: begin capture");
    for (int k = 0; k < g && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->fork, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
        if (e != cudaSuccess) break;
        launch_plain_batch<D3Q19, real, S>(box + (size_t)k * L, L, b->box_gx, b->box_gy, b->unit, b->side);
        e = cudaMemsetAsync(b->d_queue + k, 0, sizeof(int), b->stream);
        if (e != cudaSuccess) break;
        launch_fused_batch<real, S>(args + (size_t)k * L, b->d_items, b->n_items, b->d_queue + k, b->grid, b->unit,
                                    b->stream, nullptr);
        e = cudaEventRecord(b->join, b->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[slot], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch: graph capture");
    b->exec_g[slot] = g;
    return LBM_OK;
}

template <typename real, typename S>
lbm_status batch_steps(lbm_batch* b, int nsteps) {
    const int L = (int)b->lat.size();
    cudaError_t e = cudaSuccess;
    // the batch's work follows whatever was enqueued on each lattice's stream
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        e = cudaEventRecord(b->hev[l], b->lat[l]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->hev[l], 0);
    }
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step: order after the lattices' streams");
    int remaining = nsteps;
    while (remaining > 0) {
        const int g = std::min(b->G, remaining);
        const bool last = remaining == g;
        const int buf = b->hbuf;
        e = cudaEventSynchronize(b->h_ev[buf]);  // the previous upload from this host buffer is done
        if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step: host table");
        StepArgs<real>* ha = (StepArgs<real>*)b->h_tab[buf];
        BoxArgs<real>* hb = (BoxArgs<real>*)((char*)b->h_tab[buf] + (size_t)b->G * L * sizeof(StepArgs<real>));
        unsigned gx = b->box_gx, gy = b->box_gy;
        for (int k = 0; k < g; ++k) {
            for (int l = 0; l < L; ++l) {
                lbm_handle* h = b->lat[l];
                StepArgs<real>& p = ha[(size_t)k * L + l];
                memset(&p, 0, sizeof(p));
                fill_model(h, p);
                fill_geometry(h, p, h->step + 1 + k);
                fill_buffers(h, p, h->cur ^ (k & 1));
                p.write_fields = (last && k == g - 1) ? 1 : 0;
                const Region box = nozzle_box(h, p, h->step + k);
                p.box = box;
                BoxArgs<real>& q = hb[(size_t)k * L + l];
                memset(&q, 0, sizeof(q));
                q.p = p;
                q.R = box;
                if (box.wx > 0) {
                    const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
                    q.R1 = grow(box, 1, nx, ny, nz);
                    q.R2 = grow(box, 2, nx, ny, nz);
                    q.R1g = q.R1;
                    if (q.R1g.z0 <= 0) q.R1g.z0 = -1;
                    if (q.R1g.z1 >= nz) q.R1g.z1 = nz + 1;
                    q.Rg = grow(q.R2, 2, nx, ny, nz);
                    box_grid(q.R2, q.R1g, &gx, &gy);
                }
            }
        }
        if (gx > b->box_gx || gy > b->box_gy) {
            // a box outgrew the captured grid: widen it (with slack) and recapture
            b->box_gx = gx + gx / 4 + 1;
            b->box_gy = gy;
            b->exec_valid = false;
        }
        const size_t tab_bytes = (size_t)b->G * L * (sizeof(StepArgs<real>) + sizeof(BoxArgs<real>));
        e = cudaMemcpyAsync(b->d_tab, b->h_tab[buf], tab_bytes, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->h_ev[buf], b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step: table upload");
        b->hbuf ^= 1;
        if (last) {
            for (int l = 0; l < L && e == cudaSuccess; ++l)
                e = cudaMemsetAsync(b->lat[l]->acc + kAccMass, 0, 5 * sizeof(double), b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "cudaMemsetAsync");
        }
        if (!b->exec_valid) b->exec_g[0] = b->exec_g[1] = 0;
        b->exec_valid = true;
        const int slot = g == b->G ? 0 : 1;
        if (b->exec_g[slot] != g) {
            lbm_status st = batch_capture<real, S>(b, slot, g);
            if (st != LBM_OK) return st;
        }
        e = cudaGraphLaunch(b->exec[slot], b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
        for (int l = 0; l < L; ++l) {
            lbm_handle* h = b->lat[l];
            h->step += g;
            h->cur ^= (g & 1);
        }
        b->launches += 6LL * g;  // column flags, four box phases, bulk
        b->steps += g;
        remaining -= g;
    }
    // later work on each lattice's stream (lbm_fields, lbm_step) follows the batch
    e = cudaEventRecord(b->done, b->stream);
    for (int l = 0; l < L && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->lat[l]->stream, b->done, 0);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step: order before the lattices' streams");
    return LBM_OK;
}

template <typename real, typename S>
lbm_status batch_alloc_tables(lbm_batch* b) {
    const int L = (int)b->lat.size();
    b->args_bytes = (size_t)b->G * L * sizeof(StepArgs<real>);
    b->box_bytes = (size_t)b->G * L * sizeof(BoxArgs<real>);
    const size_t bytes = b->args_bytes + b->box_bytes;
    cudaError_t e = cudaMalloc(&b->d_tab, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, (size_t)b->G * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_tab[0], bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_tab[1], bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LBM_ENOMEM, "lbm_batch_create: step tables (%.1f MB)", 3.0 * bytes / 1e6);
    }
    return LBM_OK;
}

// dispatch on the batch's storage (all lattices share it)
template <template <typename, typename> class F, typename... A>
lbm_status batch_dispatch(lbm_batch* b, A... a) {
    switch (b->storage) {
    case LBM_F64: return F<double, double>::run(b, a...);
    case LBM_F16DEV: return F<float, __half>::run(b, a...);
    case LBM_BF16DEV: return F<float, __nv_bfloat16>::run(b, a...);
    default: return F<float, float>::run(b, a...);
    }
}
template <typename real, typename S>
struct RunSteps {
    static lbm_status run(lbm_batch* b, int n) { return batch_steps<real, S>(b, n); }
};
template <typename real, typename S>
struct RunPlan {
    static lbm_status run(lbm_batch* b, int variant, const std::vector<int>* zc) { return batch_plan<real, S>(b, variant, *zc); }
};
template <typename real, typename S>
struct RunAlloc {
    static lbm_status run(lbm_batch* b) { return batch_alloc_tables<real, S>(b); }
};

lbm_status batch_usable(lbm_batch* b, const DeviceScope& ds) {
    if (b->dead) return bfail(b, LBM_ECUDA, "batch unusable after an earlier CUDA error");
    if (ds.err != cudaSuccess) return bcuda(b, ds.err, "cudaSetDevice");
    for (lbm_handle* h : b->lat)
        if (h->dead) return bfail(b, LBM_ECUDA, "a lattice of the batch is unusable after a CUDA error");
    return LBM_OK;
}

}  // namespace

extern "C" {

long long lbm_lattice_bytes(const lbm_config* cfg) {
    if (!cfg || cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return -1;
    if (cfg->velset != LBM_D2Q9 && cfg->velset != LBM_D3Q19) return -1;
    if (cfg->storage < LBM_F64 || cfg->storage > LBM_BF16DEV) return -1;
    const long long Q = cfg->velset == LBM_D3Q19 ? 19 : 9;
    const long long plane = (long long)cfg->nx * cfg->ny, N = plane * cfg->nz;
    const long long es = cfg->storage == LBM_F64 ? 8 : 4;
    const long long ps = cfg->storage == LBM_F64 ? 8 : (cfg->storage == LBM_F32 ? 4 : 2);
    const long long fdata = (2 * Q * N * ps + 255) & ~255LL;
    const long long fbytes = fdata + (ps == 2 ? N * es : 0);
    const long long rbytes = 2 * (N + 2 * plane) * es, ubytes = 3 * 2 * plane * es;
    return 2 * (fbytes + rbytes + ubytes) + (long long)kNFields * N * es + kAccN * 8 + 256 + ((plane + 255) & ~255LL);
}

long long lbm_batch_plan(const int* dims, int n, int tile_h, const int* zchunk, int* items, long long cap) {
    if (!dims || !zchunk || n < 0 || tile_h < 1) return -1;
    for (int l = 0; l < n; ++l)
        if (dims[3 * l] < 1 || dims[3 * l + 1] < 1 || dims[3 * l + 2] < 1 || dims[3 * l] > 65535 ||
            dims[3 * l + 1] > 32767)
            return -1;
    return plan_items(dims, n, tile_h, zchunk, items, items ? cap : 0);
}

}  // extern "C"

namespace {

// the members' conditions of lbm_batch_create; *unit: their density-ratio class
lbm_status batch_check(lbm_batch* b, lbm_handle* const* lattices, int n, int* unit) {
    if (!lattices || n < 1) return bfail(b, LBM_EINVAL, "lbm_batch: need at least one lattice");
    int unit0 = -1;
    for (int l = 0; l < n; ++l) {
        lbm_handle* h = lattices[l];
        if (!h) return bfail(b, LBM_EINVAL, "lbm_batch: lattice %d is NULL", l);
        if (h->dead) return bfail(b, LBM_ECUDA, "lbm_batch: lattice %d is unusable", l);
        if (!h->have_geom || !h->have_rheo)
            return bfail(b, LBM_ESTATE, "lbm_batch: lattice %d has no geometry or rheology", l);
        if (!is_fused(h))
            return bfail(b, LBM_EINVAL, "lbm_batch: lattice %d is not a fused-path lattice (D3Q19, substrate + open top)",
                         l);
        if (h->cfg.nx > 65535 || h->cfg.ny > 32767)
            return bfail(b, LBM_EINVAL, "lbm_batch: lattice %d too wide for the work list", l);
        if (h->cfg.device != lattices[0]->cfg.device || h->cfg.storage != lattices[0]->cfg.storage)
            return bfail(b, LBM_EINVAL, "lbm_batch: lattices must share device and storage");
        if (b && (h->cfg.device != b->device || h->cfg.storage != b->storage))
            return bfail(b, LBM_EINVAL, "lbm_batch_reset: lattices must keep the batch's device and storage");
        for (int m = 0; m < l; ++m)
            if (lattices[m] == h) return bfail(b, LBM_EINVAL, "lbm_batch: lattice %d given twice", l);
        StepArgs<double> p;
        memset(&p, 0, sizeof(p));
        fill_model(h, p);
        if (unit0 < 0) unit0 = p.unit;
        if (p.unit != unit0) return bfail(b, LBM_EINVAL, "lbm_batch: lattices must all have density ratio one or none");
    }
    *unit = unit0;
    return LBM_OK;
}

// members, per-member events, step tables for n lattices, default plan
lbm_status batch_members(lbm_batch* b, lbm_handle* const* lattices, int n, int unit) {
    const size_t old_cap = b->hev.size();
    b->lat.assign(lattices, lattices + n);
    b->unit = unit;
    cudaError_t e = cudaSuccess;
    while (b->hev.size() < (size_t)n && e == cudaSuccess) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->hev.push_back(ev);
    }
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch: events");
    if (!b->d_tab || (size_t)n > old_cap) {
        // tables sized for the members (capacity grows, never shrinks)
        if (b->d_tab) cudaFree(b->d_tab);
        if (b->d_queue) cudaFree(b->d_queue);
        for (int k = 0; k < 2; ++k)
            if (b->h_tab[k]) cudaFreeHost(b->h_tab[k]);
        b->d_tab = b->h_tab[0] = b->h_tab[1] = nullptr;
        b->d_queue = nullptr;
        lbm_status st = batch_dispatch<RunAlloc>(b);
        if (st != LBM_OK) return st;
    }
    // default plan: the single-lattice heuristic's z-chunk for each lattice
    std::vector<int> zc(n);
    for (int l = 0; l < n; ++l) zc[l] = lattices[l]->zchunk;
    b->box_gx = b->box_gy = 0;
    return batch_dispatch<RunPlan>(b, 0, &zc);
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_handle* const* lattices, int n, lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: out is NULL");
    *out = nullptr;
    int unit = 1;
    lbm_status st = batch_check(nullptr, lattices, n, &unit);
    if (st != LBM_OK) return st;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "lbm_batch_create: host allocation failed");
    b->device = lattices[0]->cfg.device;
    b->storage = lattices[0]->cfg.storage;
    DeviceScope ds(b->device);
    cudaError_t e = ds.err;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = create_box_stream(&b->side);
    for (cudaEvent_t* ev : {&b->fork, &b->join, &b->done, &b->h_ev[0], &b->h_ev[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
    if (e != cudaSuccess) {
        bfail(nullptr, LBM_ECUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
        lbm_batch_destroy(b);
        return LBM_ECUDA;
    }
    st = batch_members(b, lattices, n, unit);
    if (st != LBM_OK) {
        snprintf(g_create_error, sizeof(g_create_error), "%s", b->err);
        lbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_reset(lbm_batch* b, lbm_handle* const* lattices, int n) {
    if (!b) return LBM_EINVAL;
    DeviceScope ds(b->device);
    lbm_status st = batch_usable(b, ds);
    if (st != LBM_OK) return st;
    int unit = 1;
    if ((st = batch_check(b, lattices, n, &unit)) != LBM_OK) return st;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->side);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_reset: sync");
    return batch_members(b, lattices, n, unit);
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
    if (!b) return LBM_EINVAL;
    DeviceScope ds(b->device);
    lbm_status st = batch_usable(b, ds);
    if (st != LBM_OK) return st;
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "lbm_batch_step: nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    return batch_dispatch<RunSteps>(b, nsteps);
}

lbm_status lbm_batch_set_plan(lbm_batch* b, int variant, const int* zchunk) {
    if (!b) return LBM_EINVAL;
    DeviceScope ds(b->device);
    lbm_status st = batch_usable(b, ds);
    if (st != LBM_OK) return st;
    if (variant != 0) return bfail(b, LBM_EINVAL, "lbm_batch_set_plan: variant must be 0");
    if (!zchunk) return bfail(b, LBM_EINVAL, "lbm_batch_set_plan: zchunk is NULL");
    std::vector<int> zc(zchunk, zchunk + b->lat.size());
    for (int v : zc)
        if (v < 1) return bfail(b, LBM_EINVAL, "lbm_batch_set_plan: z-chunks must be >= 1");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_set_plan: sync");
    return batch_dispatch<RunPlan>(b, variant, &zc);
}

lbm_status lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_tuning* out) {
    if (!b) return LBM_EINVAL;
    DeviceScope ds(b->device);
    lbm_status st = batch_usable(b, ds);
    if (st != LBM_OK) return st;
    if (trial_steps < 1) return bfail(b, LBM_EINVAL, "lbm_batch_autotune: trial_steps < 1");
    const int L = (int)b->lat.size();
    int max_nz = 1;
    for (lbm_handle* h : b->lat) max_nz = std::max(max_nz, h->cfg.nz);
    const int chunks[] = {8, 12, 16, 24, 32, 48, 64, 96, 128};
    const int nvar = 1;  // one bulk-kernel configuration
    lbm_batch_tuning res;
    memset(&res, 0, sizeof(res));
    res.ms_per_step = 1e30;
    for (int v = 0; v < nvar; ++v) {
      // resident CTAs per SM of this variant (the plan records it)
      b->ctas_per_sm = 0;
      {
          std::vector<int> zc(L, chunks[0]);
          cudaError_t e = cudaStreamSynchronize(b->stream);
          if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_autotune: sync");
          if ((st = batch_dispatch<RunPlan>(b, v, &zc)) != LBM_OK) return st;
      }
      const int occ = b->occ;
      for (int k = occ; k >= std::max(1, occ - 1); --k) {
        for (int c : chunks) {
            if (c > max_nz && c != chunks[0]) continue;
            std::vector<int> zc(L, c);
            cudaError_t e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_autotune: sync");
            b->ctas_per_sm = k;
            if ((st = batch_dispatch<RunPlan>(b, v, &zc)) != LBM_OK) return st;
            // the first call captures the graph; the second is timed
            const int g = std::min(b->G, trial_steps);
            if ((st = lbm_batch_step(b, g)) != LBM_OK) return st;
            e = cudaEventRecord(b->t0, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "cudaEventRecord");
            if ((st = lbm_batch_step(b, trial_steps)) != LBM_OK) return st;
            e = cudaEventRecord(b->t1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(b->t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->t0, b->t1);
            if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_autotune: timing");
            const double per = ms / trial_steps;
            if (res.n_tried < LBM_TUNE_MAX) {
                res.tried_variant[res.n_tried] = v;
                res.tried_zchunk[res.n_tried] = c;
                res.tried_ctas[res.n_tried] = k;
                res.tried_ms[res.n_tried] = per;
            }
            res.n_tried += 1;
            if (per < res.ms_per_step) {
                res.ms_per_step = per;
                res.variant = v;
                res.zchunk = c;
                res.ctas_per_sm = k;
            }
        }
      }
    }
    std::vector<int> zc(L, res.zchunk);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_autotune: sync");
    b->ctas_per_sm = res.ctas_per_sm;
    if ((st = batch_dispatch<RunPlan>(b, res.variant, &zc)) != LBM_OK) return st;
    if (out) *out = res;
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch* b, lbm_batch_plan_info* out) {
    if (!b || !out) return LBM_EINVAL;
    out->n_lattices = (int)b->lat.size();
    out->variant = b->variant;
    out->tile_h = kFusedTileH;
    out->n_items = b->n_items;
    out->grid = b->grid;
    out->steps_per_graph = b->G;
    out->steps = b->steps;
    out->launches = b->launches;
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return LBM_EINVAL;
    DeviceScope ds(b->device);
    lbm_status st = batch_usable(b, ds);
    if (st != LBM_OK) return st;
    return bcuda(b, cudaStreamSynchronize(b->stream), "lbm_batch_sync");
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    DeviceScope ds(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->side) cudaStreamSynchronize(b->side);
    for (cudaGraphExec_t x : b->exec)
        if (x) cudaGraphExecDestroy(x);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_tab) cudaFree(b->d_tab);
    if (b->d_queue) cudaFree(b->d_queue);
    for (int k = 0; k < 2; ++k) {
        if (b->h_tab[k]) cudaFreeHost(b->h_tab[k]);
        if (b->h_ev[k]) cudaEventDestroy(b->h_ev[k]);
    }
    for (cudaEvent_t ev : {b->fork, b->join, b->done, b->t0, b->t1})
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : b->hev)
        if (ev) cudaEventDestroy(ev);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_create_error; }

}  // extern "C"
