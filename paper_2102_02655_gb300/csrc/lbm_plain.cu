// Phase-by-phase kernels: the direct form of one time step, used over the
// whole lattice (plain path) or only in the box around the nozzle (fused
// path). Order of a step (Sec. II A-B): stream on the step-(n-1) geometry with
// the boundary rules, delete/create the nodes the nozzle covers/uncovers, take
// moments, fill the fictitious wall densities, then collide.
#include "lbm_launch.h"

namespace cglbm {

namespace {

constexpr int kThreads = kBoxThreads;

// Launch shape of a region: blockIdx.x covers the region's columns (32-bit),
// blockIdx.y its planes. Returns false for threads past the last column or
// plane (a batched launch covers the largest region of its lattices).
__device__ __forceinline__ bool region_site(const Region& r, int nx, int ny, int* x, int* y, int* z) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= r.wx * r.wy || (int)blockIdx.y >= r.z1 - r.z0) return false;
    const int j = t / r.wx;
    const int i = t - j * r.wx;
    *x = wrapn(r.x0 + i, nx);
    *y = wrapn(r.y0 + j, ny);
    *z = r.z0 + (int)blockIdx.y;
    return true;
}

__device__ __forceinline__ bool in_region(const Region& r, int x, int y, int z, int nx, int ny) {
    if (z < r.z0 || z >= r.z1) return false;
    int dx = x - r.x0;
    if (dx < 0) dx += nx;
    int dy = y - r.y0;
    if (dy < 0) dy += ny;
    return dx < r.wx && dy < r.wy;
}

// sum over the warp, one atomic per warp
__device__ __forceinline__ void warp_add(double* dst, double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

__host__ __device__ inline long long region_sites(const Region& r) { return (long long)r.wx * r.wy * (r.z1 - r.z0); }

inline int blocks_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152LL * 16) b = 152LL * 16;
    return (int)(b < 1 ? 1 : b);
}

// one thread per column of the region, one grid row per plane
inline dim3 region_grid(const Region& r) {
    const long long cols = (long long)r.wx * r.wy;
    return dim3((unsigned)((cols + kThreads - 1) / kThreads), (unsigned)(r.z1 - r.z0 > 0 ? r.z1 - r.z0 : 1));
}

// 0. per-column nozzle flags of this step over region G (columns only)
template <typename real>
__device__ __forceinline__ void geo_body(const StepArgs<real>& p, const Region& G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.y != 0 || t >= G.wx * G.wy) return;
    const int j = t / G.wx, i = t - j * G.wx;
    const int x = wrapn(G.x0 + i, p.nx), y = wrapn(G.y0 + j, p.ny);
    p.geo[y * p.nx + x] = (unsigned char)geo_flags(p, x, y);
}

template <typename real>
__global__ void __launch_bounds__(kThreads) k_geo(StepArgs<real> p, Region G) {
    geo_body(p, G);
}

template <typename real>
__global__ void __launch_bounds__(kThreads) k_geo_b(const BoxArgs<real>* __restrict__ t) {
    const BoxArgs<real>& b = t[blockIdx.z];
    if (b.R.wx == 0) return;
    geo_body(b.p, b.Rg);
}

// the columns the boundary kernels query around region R2: two more rings
// (neighbours, and the wall-density extrapolation two links out)
__host__ __device__ inline Region geo_region(const Region& R2, int nx, int ny) {
    Region g = R2;
    if (R2.wx + 4 >= nx) { g.x0 = 0; g.wx = nx; }
    else { g.x0 = R2.x0 - 2 < 0 ? R2.x0 - 2 + nx : R2.x0 - 2; g.wx = R2.wx + 4; }
    if (R2.wy + 4 >= ny) { g.y0 = 0; g.wy = ny; }
    else { g.y0 = R2.y0 - 2 < 0 ? R2.y0 - 2 + ny : R2.y0 - 2; g.wy = R2.wy + 4; }
    g.z0 = 0;
    g.z1 = 1;
    return g;
}

inline dim3 geo_grid(const Region& G) {
    return dim3((unsigned)(((long long)G.wx * G.wy + kThreads - 1) / kThreads), 1);
}

// 1. stream + densities (post-streaming) of every fluid node of step n-1 in R2
template <class VS, typename real, typename S>
__device__ __forceinline__ void stream_density_body(const StepArgs<real>& p, const Region& R2, const Region& R) {
    const long long comp = p.N + 2 * p.plane;
    double bc0 = 0, bc1 = 0, de0 = 0, de1 = 0;
    int x, y, z;
    if (region_site(R2, p.nx, p.ny, &x, &y, &z) && !solid_at(p, x, y, z, 0)) {
        real f[2][VS::Q];
        real bc[2] = {real(0), real(0)};
        pull_general<VS, S>(p, x, y, z, f, bc);
        real rY = 0, sd = 0;
#pragma unroll
        for (int i = 0; i < VS::Q; ++i) { rY += f[0][i]; sd += f[1][i]; }
        const real rB = (p.rho_ref + sd) - rY;
        const long long r = ridx(p, x, y, z);
        p.rho_cur[r] = rY;
        p.rho_cur[comp + r] = rB;
        if (in_region(R, x, y, z, p.nx, p.ny)) {
            bc0 += (double)bc[0];
            bc1 += (double)bc[1];
            if (solid_at(p, x, y, z, 1)) {
                de0 += (double)rY;
                de1 += (double)rB;
            } else {
                // the collision of this site reads these in place (step 4)
                const long long s = sidx(p, x, y, z);
                const real c = ref_frac(rY, rB);
#pragma unroll
                for (int i = 0; i < VS::Q; ++i) pop_put<VS, S>(p, i, s, p.N, f[0][i], f[1][i], c);
                ref_put<S>(p, s, c);
            }
        }
    }
    warp_add(p.acc + kAccBc, bc0);
    warp_add(p.acc + kAccBc + 1, bc1);
    warp_add(p.acc + kAccDestroyed, de0);
    warp_add(p.acc + kAccDestroyed + 1, de1);
}

template <class VS, typename real, typename S>
__global__ void __launch_bounds__(kThreads, 2) k_stream_density(StepArgs<real> p, Region R2, Region R) {
    stream_density_body<VS, real, S>(p, R2, R);
}

template <class VS, typename real, typename S>
__global__ void __launch_bounds__(kThreads, 2) k_stream_density_b(const BoxArgs<real>* __restrict__ t) {
    const BoxArgs<real>& b = t[blockIdx.z];
    if (b.R.wx == 0) return;  // no box for this lattice
    stream_density_body<VS, real, S>(b.p, b.R2, b.R);
}

// 2. nodes the nozzle uncovered: mean density of the neighbours that are fluid
//    at both steps (Sec. II B)
template <class VS, typename real, typename S>
__device__ __forceinline__ void created_body(const StepArgs<real>& p, const Region& R1, const Region& R) {
    const long long comp = p.N + 2 * p.plane;
    double c0 = 0, c1 = 0;
    int x, y, z;
    if (region_site(R1, p.nx, p.ny, &x, &y, &z) && solid_at(p, x, y, z, 0) && !solid_at(p, x, y, z, 1)) {
        real s0 = 0, s1 = 0;
        int cnt = 0;
#pragma unroll
        for (int i = 1; i < VS::Q; ++i) {
            const int x1 = wrapn(x + VS::c(i, 0), p.nx), y1 = wrapn(y + VS::c(i, 1), p.ny);
            int z1 = z + VS::c(i, 2);
            if (p.z_mode == kZPeriodic) z1 = wrapn(z1, p.nz);
            else if (z1 < 0 || z1 >= p.nz) continue;
            if (solid_at(p, x1, y1, z1, 0) || solid_at(p, x1, y1, z1, 1)) continue;
            const long long r1 = ridx(p, x1, y1, z1);
            s0 += p.rho_cur[r1];
            s1 += p.rho_cur[comp + r1];
            ++cnt;
        }
        real m0, m1;
        if (cnt > 0) { m0 = s0 / real(cnt); m1 = s1 / real(cnt); }
        else { m0 = real(0); m1 = p.rho0[1]; }
        const long long r = ridx(p, x, y, z);
        p.rho_cur[r] = m0;
        p.rho_cur[comp + r] = m1;
        if (in_region(R, x, y, z, p.nx, p.ny)) {
            c0 += (double)m0;
            c1 += (double)m1;
            // populations of the created node: equilibrium at the nozzle velocity
            const long long s = sidx(p, x, y, z);
            const real uu = p.vn[0] * p.vn[0] + p.vn[1] * p.vn[1] + p.vn[2] * p.vn[2];
            const real c = ref_frac(m0, m1);
#pragma unroll
            for (int i = 0; i < VS::Q; ++i) {
                real eY, eD;
                feq_pair<VS>(p, i, m0, m1, p.vn[0], p.vn[1], p.vn[2], uu, &eY, &eD);
                pop_put<VS, S>(p, i, s, p.N, eY, eD, c);
            }
            ref_put<S>(p, s, c);
        }
    }
    warp_add(p.acc + kAccCreated, c0);
    warp_add(p.acc + kAccCreated + 1, c1);
}

template <class VS, typename real, typename S>
__global__ void __launch_bounds__(kThreads) k_created(StepArgs<real> p, Region R1, Region R) {
    created_body<VS, real, S>(p, R1, R);
}

template <class VS, typename real, typename S>
__global__ void __launch_bounds__(kThreads) k_created_b(const BoxArgs<real>* __restrict__ t) {
    const BoxArgs<real>& b = t[blockIdx.z];
    if (b.R.wx == 0) return;  // no box for this lattice
    created_body<VS, real, S>(b.p, b.R1, b.R);
}

// fictitious density of solid node (x, y, z) of step n (Eq. 18): the
// zeta-scaled, w-weighted mean over its fluid neighbours
template <class VS, typename real>
__device__ __forceinline__ void wall_rho(const StepArgs<real>& p, int x, int y, int z, real* o0, real* o1) {
    const long long comp = p.N + 2 * p.plane;
    real n0 = 0, n1 = 0, den = 0;
#pragma unroll
    for (int i = 1; i < VS::Q; ++i) {
        const int x1 = wrapn(x + VS::c(i, 0), p.nx), y1 = wrapn(y + VS::c(i, 1), p.ny);
        int z1 = z + VS::c(i, 2);
        if (p.z_mode == kZPeriodic) z1 = wrapn(z1, p.nz);
        else if (z1 < 0 || z1 >= p.nz) continue;
        if (solid_at(p, x1, y1, z1, 1)) continue;
        const long long r1 = ridx(p, x1, y1, z1);
        const real w = (real)VS::w(i);
        n0 += w * p.rho_cur[r1];
        n1 += w * p.rho_cur[comp + r1];
        den += w;
    }
    *o0 = den > real(0) ? p.zeta[0] * n0 / den : real(0);
    *o1 = den > real(0) ? p.zeta[1] * n1 / den : real(0);
}

// 3. wall densities on solid nodes of R1 and the ghost planes z = -1, z = nz
template <class VS, typename real>
__device__ __forceinline__ void wall_body(const StepArgs<real>& p, const Region& R1g) {
    const long long comp = p.N + 2 * p.plane;
    int x, y, z;
    if (!region_site(R1g, p.nx, p.ny, &x, &y, &z)) return;
    {
        real o0, o1;
        if (z < 0 || z >= p.nz) {
            if (p.z_mode != kZWalls) return;
            if (z >= p.nz && p.top_mode == kTopOpen) {
                // open top: zero normal gradient, copy of the top plane
                const int zt = p.nz - 1;
                if (solid_at(p, x, y, zt, 1)) {
                    wall_rho<VS>(p, x, y, zt, &o0, &o1);
                } else {
                    const long long rt = ridx(p, x, y, zt);
                    o0 = p.rho_cur[rt];
                    o1 = p.rho_cur[comp + rt];
                }
            } else {
                wall_rho<VS>(p, x, y, z, &o0, &o1);  // substrate or lid
            }
        } else {
            if (!solid_at(p, x, y, z, 1)) return;
            wall_rho<VS>(p, x, y, z, &o0, &o1);
        }
        const long long r = ridx(p, x, y, z);
        p.rho_cur[r] = o0;
        p.rho_cur[comp + r] = o1;
    }
}

template <class VS, typename real>
__global__ void __launch_bounds__(kThreads) k_wall(StepArgs<real> p, Region R1g) {
    wall_body<VS, real>(p, R1g);
}

template <class VS, typename real>
__global__ void __launch_bounds__(kThreads) k_wall_b(const BoxArgs<real>* __restrict__ t) {
    const BoxArgs<real>& b = t[blockIdx.z];
    if (b.R.wx == 0) return;  // no box for this lattice
    wall_body<VS, real>(b.p, b.R1g);
}

// neighbour accessors over the density array of the step: the ink fraction
// (density ratio one), or ink and ambient fractions and the phase field
template <class VS, typename real>
struct ArrayNbUnit {
    const StepArgs<real>* p;
    int x, y, z;
    __device__ __forceinline__ real operator()(int i) const {
        const long long comp = p->N + 2 * p->plane;
        const int x1 = wrapn(x + VS::c(i, 0), p->nx), y1 = wrapn(y + VS::c(i, 1), p->ny);
        int z1 = z + VS::c(i, 2);
        if (p->z_mode == kZPeriodic) z1 = wrapn(z1, p->nz);
        const long long r1 = ridx(*p, x1, y1, z1);
        const real a = p->rho_cur[r1], b = p->rho_cur[comp + r1];
        return colour_frac(a, b);
    }
};

template <class VS, typename real>
struct ArrayNb {
    const StepArgs<real>* p;
    int x, y, z;
    __device__ __forceinline__ void operator()(int i, real* cY, real* cB, real* rn) const {
        const long long comp = p->N + 2 * p->plane;
        const int x1 = wrapn(x + VS::c(i, 0), p->nx), y1 = wrapn(y + VS::c(i, 1), p->ny);
        int z1 = z + VS::c(i, 2);
        if (p->z_mode == kZPeriodic) z1 = wrapn(z1, p->nz);
        const long long r1 = ridx(*p, x1, y1, z1);
        const real a = p->rho_cur[r1], b = p->rho_cur[comp + r1];
        *cY = colour_frac(a, b);
        *cB = colour_frac(b, a);
        *rn = phase_field(*p, a, b);
    }
};

template <typename real>
__device__ __forceinline__ void store_fields(const StepArgs<real>& p, long long s, const SiteOut<real>& so,
                                             real solid) {
    real* F = p.fields;
    F[kFRhoInk * p.N + s] = so.rhoY;
    F[kFRhoAmb * p.N + s] = so.rhoB;
    F[kFUx * p.N + s] = so.u[0];
    F[kFUy * p.N + s] = so.u[1];
    F[kFUz * p.N + s] = so.u[2];
    F[kFNu * p.N + s] = so.tau > real(0) ? (so.tau - real(0.5)) * real(1.0 / 3.0) : real(0);
    F[kFP * p.N + s] = p.pfac[0] * so.rhoY + p.pfac[1] * so.rhoB;
    F[kFPhi * p.N + s] = so.rn;
    F[kFSolid * p.N + s] = solid;
}

// 4. collision at every fluid node of step n in R, in place: steps 1 and 2
//    left the post-streaming (or created) populations in fout
template <class VS, typename real, bool kUnit, typename S>
__device__ __forceinline__ void collide_body(const StepArgs<real>& p, const Region& R) {
    const long long comp = p.N + 2 * p.plane;
    double m0 = 0, m1 = 0, px = 0, py = 0, pz = 0;
    int bad = 0;
    int x, y, z;
    const bool active = region_site(R, p.nx, p.ny, &x, &y, &z);
    const long long s = active ? sidx(p, x, y, z) : 0;
    if (active && solid_at(p, x, y, z, 1)) {
        if (p.write_fields) {
            SiteOut<real> so = {0, 0, {0, 0, 0}, 0, 0};
            store_fields(p, s, so, real(1));
        }
    } else if (active) {
        real f[2][VS::Q];
#pragma unroll
        for (int i = 0; i < VS::Q; ++i) pop_get<VS, S>(p, p.fout, p.ref_out, i, s, p.N, &f[0][i], &f[1][i]);
        SiteOut<real> so;
        const real zd = p.z_mode == kZWalls ? real(z) + real(0.5) : real(-1);
        if constexpr (kUnit) {
            ArrayNbUnit<VS, real> nb{&p, x, y, z};
            collide<VS, real, true>(p, f, nb, zd, &so);
        } else {
            ArrayNb<VS, real> nb{&p, x, y, z};
            collide<VS, real, false>(p, f, nb, zd, &so);
        }
#pragma unroll
        for (int i = 0; i < VS::Q; ++i) pop_put<VS, S>(p, i, s, p.N, f[0][i], f[1][i], so.cY);
        ref_put<S>(p, s, so.cY);
        if (z >= p.nz - 2)
            for (int a = 0; a < 3; ++a) p.u_cur[utop_idx(p, a, x, y, z)] = so.u[a];
        if (unstable_site(so.rhoY, so.rhoB)) bad = 1;
        if (p.write_fields) {
            store_fields(p, s, so, real(0));
            m0 += (double)so.rhoY;
            m1 += (double)so.rhoB;
            const double rr = (double)so.rhoY + (double)so.rhoB;
            px += rr * (double)so.u[0];
            py += rr * (double)so.u[1];
            pz += rr * (double)so.u[2];
        }
    }
    if (p.write_fields) {
        warp_add(p.acc + kAccMass, m0);
        warp_add(p.acc + kAccMass + 1, m1);
        warp_add(p.acc + kAccMom, px);
        warp_add(p.acc + kAccMom + 1, py);
        warp_add(p.acc + kAccMom + 2, pz);
    }
    if (bad) atomicOr(p.flags, 1);
}

// CTAs per SM the collision kernels are compiled for: in FP32 six (at most 85
// registers), so that the nozzle box's collision runs in one wave
template <typename real>
constexpr int collide_min_blocks() {
    return sizeof(real) == 4 ? 6 : 2;
}

template <class VS, typename real, bool kUnit, typename S>
__global__ void __launch_bounds__(kThreads, collide_min_blocks<real>()) k_collide(StepArgs<real> p, Region R) {
    collide_body<VS, real, kUnit, S>(p, R);
}

template <class VS, typename real, bool kUnit, typename S>
__global__ void __launch_bounds__(kThreads, collide_min_blocks<real>())
    k_collide_b(const BoxArgs<real>* __restrict__ t) {
    const BoxArgs<real>& b = t[blockIdx.z];
    if (b.R.wx == 0) return;  // no box for this lattice
    collide_body<VS, real, kUnit, S>(b.p, b.R);
}

// initial equilibrium state
template <class VS, typename real, typename S>
__global__ void __launch_bounds__(kThreads) k_init(StepArgs<real> p, int staged, int have_u) {
    const long long comp = p.N + 2 * p.plane;
    double m0 = 0, m1 = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < p.N;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % p.nx);
        const int y = (int)((s / p.nx) % p.ny);
        const int z = (int)(s / p.plane);
        const long long r = ridx(p, x, y, z);
        SiteOut<real> so = {0, 0, {0, 0, 0}, 0, 0};
        if (solid_at(p, x, y, z, 1)) {
            p.rho_cur[r] = real(0);
            p.rho_cur[comp + r] = real(0);
            store_fields(p, s, so, real(1));
            continue;
        }
        real rY, rB, u[3] = {0, 0, 0};
        if (staged) {
            rY = p.fields[kFRhoInk * p.N + s];
            rB = p.fields[kFRhoAmb * p.N + s];
            if (have_u) {
                u[0] = p.fields[kFUx * p.N + s];
                u[1] = p.fields[kFUy * p.N + s];
                u[2] = p.fields[kFUz * p.N + s];
            }
        } else {
            const bool ink = p.nozzle && z >= p.gap && (geo_at(p, x, y) & kGeoIn1);
            rY = ink ? p.rho0[0] : real(0);
            rB = ink ? real(0) : p.rho0[1];
        }
        const real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const real c = ref_frac(rY, rB);
#pragma unroll
        for (int i = 0; i < VS::Q; ++i) {
            real eY, eD;
            feq_pair<VS>(p, i, rY, rB, u[0], u[1], u[2], uu, &eY, &eD);
            pop_put<VS, S>(p, i, s, p.N, eY, eD, c);
        }
        ref_put<S>(p, s, c);
        p.rho_cur[r] = rY;
        p.rho_cur[comp + r] = rB;
        if (z >= p.nz - 2)
            for (int a = 0; a < 3; ++a) p.u_cur[utop_idx(p, a, x, y, z)] = u[a];
        so.rhoY = rY;
        so.rhoB = rB;
        so.u[0] = u[0]; so.u[1] = u[1]; so.u[2] = u[2];
        so.tau = real(0);
        so.rn = phase_field(p, rY, rB);
        store_fields(p, s, so, real(0));
        m0 += (double)rY;
        m1 += (double)rB;
    }
    warp_add(p.acc + kAccMass, m0);
    warp_add(p.acc + kAccMass + 1, m1);
}

template <class VS, typename real>
__global__ void __launch_bounds__(kThreads) k_prev_from_f(StepArgs<real> p, real* rho_prev, real* u_prev) {
    const long long comp = p.N + 2 * p.plane;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < p.N;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % p.nx);
        const int y = (int)((s / p.nx) % p.ny);
        const int z = (int)(s / p.plane);
        if (solid_at(p, x, y, z, 0)) continue;
        real rY = 0, sd = 0, m[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < VS::Q; ++i) {
            real a, d;
            pop_get<VS, real>(p, p.fin, p.ref_in, i, s, p.N, &a, &d);
            rY += a;
            sd += d;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (VS::c(i, c)) m[c] += VS::c(i, c) > 0 ? d : -d;
        }
        const real rho = p.rho_ref + sd;
        const long long r = ridx(p, x, y, z);
        rho_prev[r] = rY;
        rho_prev[comp + r] = rho - rY;
        if (z >= p.nz - 2) {
            // m = rho u + F with F = rho g - gamma rho_Y u in the drag zone
            const bool zone = p.z_mode == kZWalls && p.drag_gamma != real(0) && real(z) + real(0.5) < p.drag_height;
            const real den = zone ? rho - p.drag_gamma * rY : rho;
            for (int a = 0; a < 3; ++a) {
                const real ub = (m[a] - rho * p.g[a]) / den;
                const real F = rho * p.g[a] - (zone ? p.drag_gamma * rY * ub : real(0));
                u_prev[utop_idx(p, a, x, y, z)] = ub + real(0.5) * F / rho;
            }
        }
    }
}

}  // namespace

template <class VS, typename real>
int launch_prev_from_f(const StepArgs<real>& p, real* rho_prev, real* u_prev, cudaStream_t st) {
    int n = 0;
    if (p.nozzle) {
        const Region G{0, p.nx, 0, p.ny, 0, 1};
        k_geo<real><<<geo_grid(G), kThreads, 0, st>>>(p, G);
        n = 1;
    }
    k_prev_from_f<VS, real><<<blocks_for(p.N), kThreads, 0, st>>>(p, rho_prev, u_prev);
    return 1 + n;
}

template int launch_plain_batch<D3Q19, float, float>(const BoxArgs<float>*, int, unsigned, unsigned, int, cudaStream_t);
template int launch_plain_batch<D3Q19, double, double>(const BoxArgs<double>*, int, unsigned, unsigned, int, cudaStream_t);
template int launch_plain_batch<D3Q19, float, __half>(const BoxArgs<float>*, int, unsigned, unsigned, int, cudaStream_t);
template int launch_plain_batch<D3Q19, float, __nv_bfloat16>(const BoxArgs<float>*, int, unsigned, unsigned, int, cudaStream_t);
template int launch_prev_from_f<D3Q19, float>(const StepArgs<float>&, float*, float*, cudaStream_t);
template int launch_prev_from_f<D3Q19, double>(const StepArgs<double>&, double*, double*, cudaStream_t);
template int launch_prev_from_f<D2Q9, float>(const StepArgs<float>&, float*, float*, cudaStream_t);
template int launch_prev_from_f<D2Q9, double>(const StepArgs<double>&, double*, double*, cudaStream_t);

template <class VS, typename real, typename S>
int launch_plain(const StepArgs<real>& p, const Region& R, const Region& R1, const Region& R2, cudaStream_t st) {
    if (region_sites(R) == 0) return 0;
    int n = 0;
    if (p.nozzle) {
        const Region G = geo_region(R2, p.nx, p.ny);
        k_geo<real><<<geo_grid(G), kThreads, 0, st>>>(p, G);
        n = 1;
    }
    k_stream_density<VS, real, S><<<region_grid(R2), kThreads, 0, st>>>(p, R2, R);
    k_created<VS, real, S><<<region_grid(R1), kThreads, 0, st>>>(p, R1, R);
    Region R1g = R1;
    if (p.z_mode == kZWalls) {
        if (R1g.z0 <= 0) R1g.z0 = -1;
        if (R1g.z1 >= p.nz) R1g.z1 = p.nz + 1;
    }
    k_wall<VS, real><<<region_grid(R1g), kThreads, 0, st>>>(p, R1g);
    if (p.unit) k_collide<VS, real, true, S><<<region_grid(R), kThreads, 0, st>>>(p, R);
    else k_collide<VS, real, false, S><<<region_grid(R), kThreads, 0, st>>>(p, R);
    return 4 + n;
}

template <class VS, typename real, typename S>
int launch_plain_batch(const BoxArgs<real>* t, int n, unsigned gx, unsigned gy, int unit, cudaStream_t st) {
    if (n <= 0 || gx == 0 || gy == 0) return 0;
    const dim3 grid(gx, gy, (unsigned)n);
    k_geo_b<real><<<dim3(gx, 1, (unsigned)n), kThreads, 0, st>>>(t);
    k_stream_density_b<VS, real, S><<<grid, kThreads, 0, st>>>(t);
    k_created_b<VS, real, S><<<grid, kThreads, 0, st>>>(t);
    k_wall_b<VS, real><<<grid, kThreads, 0, st>>>(t);
    if (unit) k_collide_b<VS, real, true, S><<<grid, kThreads, 0, st>>>(t);
    else k_collide_b<VS, real, false, S><<<grid, kThreads, 0, st>>>(t);
    return 5;
}

template <class VS, typename real, typename S>
int launch_init(const StepArgs<real>& p, int staged, int have_u, cudaStream_t st) {
    int n = 0;
    if (p.nozzle) {
        const Region G{0, p.nx, 0, p.ny, 0, 1};
        k_geo<real><<<geo_grid(G), kThreads, 0, st>>>(p, G);
        n = 1;
    }
    k_init<VS, real, S><<<blocks_for(p.N), kThreads, 0, st>>>(p, staged, have_u);
    return 1 + n;
}

template int launch_plain<D3Q19, float, float>(const StepArgs<float>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D3Q19, float, float>(const StepArgs<float>&, int, int, cudaStream_t);
template int launch_plain<D3Q19, double, double>(const StepArgs<double>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D3Q19, double, double>(const StepArgs<double>&, int, int, cudaStream_t);
template int launch_plain<D3Q19, float, __half>(const StepArgs<float>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D3Q19, float, __half>(const StepArgs<float>&, int, int, cudaStream_t);
template int launch_plain<D3Q19, float, __nv_bfloat16>(const StepArgs<float>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D3Q19, float, __nv_bfloat16>(const StepArgs<float>&, int, int, cudaStream_t);
template int launch_plain<D2Q9, float, float>(const StepArgs<float>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D2Q9, float, float>(const StepArgs<float>&, int, int, cudaStream_t);
template int launch_plain<D2Q9, double, double>(const StepArgs<double>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D2Q9, double, double>(const StepArgs<double>&, int, int, cudaStream_t);
template int launch_plain<D2Q9, float, __half>(const StepArgs<float>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D2Q9, float, __half>(const StepArgs<float>&, int, int, cudaStream_t);
template int launch_plain<D2Q9, float, __nv_bfloat16>(const StepArgs<float>&, const Region&, const Region&, const Region&,
                                               cudaStream_t);
template int launch_init<D2Q9, float, __nv_bfloat16>(const StepArgs<float>&, int, int, cudaStream_t);

}  // namespace cglbm
