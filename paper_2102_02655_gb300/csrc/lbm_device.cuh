// Device-side building blocks of the two-component regularised colour-gradient
// lattice Boltzmann step (Monteferrante et al., arXiv 2102.02655, Sec. II):
// lattice constants, the nozzle template in fixed point, streaming with the
// boundary rules, and the collision at one site. Shared by the phase-by-phase
// kernels and the fused bulk kernel so that both compute the same arithmetic.
//
// Storage of a site: slot 0 holds the ink populations f^Y_i; slot 1 holds the
// deviation of the total populations from rest, d_i = f^Y_i + f^B_i - w_i
// rho_ref. Every step is linear in the populations, so streaming and the
// boundary rules act on d directly; moments and stresses of the mixture come
// from the small numbers d_i, and the ink mass in the ambient stays exact
// (its populations are tiny there). This keeps FP32 storage accurate.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace cglbm {

constexpr int kMaxQ = 19;

// ---------------------------------------------------------------------------
// Velocity sets. Direction pairs (1,2), (3,4), ... are opposite.
// ---------------------------------------------------------------------------

// D3Q19: rest, 6 axis links (w = 1/18), 12 face diagonals (w = 1/36).
struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr bool kPlanar = false;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : (i <= 6 ? 1 : 2); }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    // Perturbation coefficients (Eq. 10) for D3Q19: B_i = w_i (|c_i|^2 - 2/3),
    // the one choice proportional to w_i and quadratic in |c_i| that keeps the
    // two properties of the paper's D2Q9 values: sum_i B_i = c_s^2 and
    // sum_i B_i c_i c_i = I/3.
    __host__ __device__ static constexpr double B(int i) {
        return i == 0 ? -2.0 / 9.0 : (i <= 6 ? 1.0 / 54.0 : 1.0 / 27.0);
    }
    // phi^k_i share of the moving links (Eq. 7 generalised): (1 - alpha)/12 on
    // axes, (1 - alpha)/24 on diagonals.
    __host__ __device__ static constexpr double phi_share(int i) {
        return i == 0 ? 0.0 : (i <= 6 ? 1.0 / 12.0 : 1.0 / 24.0);
    }
    __host__ __device__ static constexpr double inv_norm(int i) {
        return i == 0 ? 0.0 : (i <= 6 ? 1.0 : 0.70710678118654752440);
    }
};

// D2Q9 of Sec. II A, laid in the x-z plane: rest (4/9), 4 axis links (1/9),
// 4 diagonals (1/36), B_i = -4/27, 2/27, 5/108 as printed after Eq. 12.
struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr bool kPlanar = true;
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 0, 1}, {0, 0, -1},
                                 {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : (i <= 4 ? 1 : 2); }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr double B(int i) {
        return i == 0 ? -4.0 / 27.0 : (i <= 4 ? 2.0 / 27.0 : 5.0 / 108.0);
    }
    // Eq. 7: (1 - alpha)/5 on axes, (1 - alpha)/20 on diagonals
    __host__ __device__ static constexpr double phi_share(int i) {
        return i == 0 ? 0.0 : (i <= 4 ? 1.0 / 5.0 : 1.0 / 20.0);
    }
    __host__ __device__ static constexpr double inv_norm(int i) {
        return i == 0 ? 0.0 : (i <= 4 ? 1.0 : 0.70710678118654752440);
    }
};

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Link vectors for loops that index the velocity set at run time (the
// compact boundary path); same order as the constexpr tables above.
static __constant__ signed char kLinkD3Q19[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static __constant__ signed char kLinkD2Q9[9][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 0, 1}, {0, 0, -1},
                                                   {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}};
template <class VS>
__device__ __forceinline__ int link(int i, int a) {
    if constexpr (VS::Q == 19) return kLinkD3Q19[i][a];
    else return kLinkD2Q9[i][a];
}

enum { kZPeriodic = 0, kZWalls = 1 };
enum { kTopOpen = 0, kTopWall = 1 };
enum { kLawNewtonian = 0, kLawCross = 1, kLawPower = 2 };

// accumulator slots (FP64, device)
enum { kAccBc = 0, kAccDestroyed = 2, kAccCreated = 4, kAccMass = 6, kAccMom = 8, kAccN = 16 };
// field planes written on the last step of an lbm_step call
enum { kFRhoInk = 0, kFRhoAmb, kFUx, kFUy, kFUz, kFNu, kFP, kFPhi, kFSolid, kNFields };

// An axis-aligned region of sites with periodic x, y: x = (x0 + i) mod nx for
// 0 <= i < wx, likewise y, and z0 <= z < z1.
struct Region {
    int x0, wx, y0, wy, z0, z1;
};

// Everything a kernel needs for one step. Passed by value (or, for batches of
// lattices, read from a device table; 16-byte aligned for vector copies).
template <typename real>
struct __align__(16) StepArgs {
    int nx, ny, nz;
    long long N;       // sites
    long long plane;   // nx * ny
    int z_mode, top_mode, nozzle, gap;
    // nozzle axis at step n-1 (index 0) and step n (index 1), in 2^-20 lattice
    // units, reduced into [0, period)
    long long hx[2], hy[2];
    long long rin2, rout2, px, py;  // squared radii (fixed point^2), periods
    long long rclear_in2, rclear_out2;  // radii 3/2 inside and outside the wall, squared
    real vn[3];        // nozzle velocity (moving-wall rule and node creation)
    real uin[3];       // inlet velocity u_ink + v_nozzle (Eq. 27)
    real utop[3];      // lid velocity
    real rho_top;      // imposed ambient density at the open top
    real rho0[2], zeta[2], A, beta, nuB, g[3], drag_gamma, drag_height;
    real phi[2][kMaxQ];
    real dphi[2][kMaxQ];  // phi^k_i - w_i (zero at density ratio one)
    real pfac[2];      // p^k = pfac[k] rho^k (Eq. 9)
    real rho_ref;      // reference total density of the stored deviation
    real wref[kMaxQ];  // w_i rho_ref, rounded to the compute type
    real kappa_w;      // sum_i wref_i c_ix^2 - rho_ref/3 - (sum_i wref_i - rho_ref)/3, exact
    int unit;          // rho0_ink == rho0_amb and phi = w for both (density ratio one)
    int law, max_iter;
    real nu0, nu_inf, lambda, n_exp, K, tau_min, tau_max, tol;
    // state: populations in the stored type S of the kernels (see Stored)
    const void* fin;
    void* fout;
    const real* ref_in;    // 16-bit storage: ink fraction of each site of fin
    real* ref_out;         // and of fout
    real* rho_cur;         // (nz + 2) planes, z = -1 .. nz
    const real* rho_prev;
    const real* u_prev;    // physical velocity of the last two planes, 3 x 2 x plane
    real* u_cur;
    real* fields;          // kNFields x N
    double* acc;
    int* flags;
    int write_fields;
    Region box;            // nozzle box (fused path); wx = 0 when unused
    // per-column nozzle flags of this step ([y][x], kGeo* bits), written by
    // k_geo over the columns the boundary kernels query (nozzle runs only)
    unsigned char* geo;
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------

// Population storage. S is the stored type: the compute type itself (FP64 or
// FP32), or a 16-bit type (FP16, BF16) that holds deviations from a local
// rest state, so that its 11 or 8 significant bits resolve the dynamics
// rather than the rest populations. Slot 1 holds the total deviation
// d_i = f^Y_i + f^B_i - w_i rho_ref in every case. With 16-bit storage slot 0
// holds f^Y_i - c w_i rho_ref, c the ink fraction rho_Y / rho of the site
// that wrote the value; c is kept per site (compute type) beside each
// population buffer, so a pull from x - c_i adds back c(x - c_i) w_i rho_ref.
template <typename S>
struct Stored {
    static constexpr bool kDev = false;
};
template <>
struct Stored<__half> {
    static constexpr bool kDev = true;
};
template <>
struct Stored<__nv_bfloat16> {
    static constexpr bool kDev = true;
};

// FP16 values are stored times 2^13: the deviations (|d| < 8) keep clear of
// FP16's largest value, and the small ones (ink diffusing into the ambient,
// 1e-6 .. 1e-9) stay above its subnormal range, where rounding of a
// positive quantity trailing off to zero loses mass. The scaling is exact.
constexpr float kF16Scale = 8192.0f, kF16Unscale = 1.0f / 8192.0f;

// The two slots of element k = i N + s (direction i, site s of N) as
// stored: FP64 and FP32 keep the slots in two arrays Q N elements apart
// (slot-major, [2][Q][N]); the 16-bit types keep them side by side, one
// 32-bit word per direction and site ([Q][N][2]), so that a pull or a store
// moves both slots in one access and converts them in one instruction.
template <class VS, typename S, typename real, typename Idx>
__device__ __forceinline__ void slots_get(const void* b, Idx k, Idx N, real* a, real* d) {
    if constexpr (std::is_same<S, __half>::value) {
        const float2 v = __half22float2(static_cast<const __half2*>(b)[k]);
        *a = v.x * kF16Unscale;
        *d = v.y * kF16Unscale;
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        const float2 v = __bfloat1622float2(static_cast<const __nv_bfloat162*>(b)[k]);
        *a = v.x;
        *d = v.y;
    } else {
        *a = static_cast<const real*>(b)[k];
        *d = static_cast<const real*>(b)[k + (Idx)VS::Q * N];
    }
}

template <class VS, typename S, typename real, typename Idx>
__device__ __forceinline__ void slots_put(void* b, Idx k, Idx N, real a, real d) {
    if constexpr (std::is_same<S, __half>::value) {
        static_cast<__half2*>(b)[k] = __floats2half2_rn(a * kF16Scale, d * kF16Scale);
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        static_cast<__nv_bfloat162*>(b)[k] = __floats2bfloat162_rn(a, d);
    } else {
        static_cast<real*>(b)[k] = a;
        static_cast<real*>(b)[k + (Idx)VS::Q * N] = d;
    }
}

// Both slots of direction i written at site s (of N) into buffer b with
// ink-fraction array ref: the post-collision populations of step n-1 when
// b = fin, or this step's values at s when b = fout (in place).
template <class VS, typename S, typename real, typename Idx>
__device__ __forceinline__ void pop_get(const StepArgs<real>& p, const void* b, const real* ref, int i, Idx s, Idx N,
                                        real* fY, real* fD) {
    slots_get<VS, S>(b, (Idx)i * N + s, N, fY, fD);
    if constexpr (Stored<S>::kDev) *fY += (real)VS::w(i) * p.rho_ref * ref[s];
}

// Store both slots of direction i at site s of fout; c is the site's ink
// fraction (written once per site with ref_put).
template <class VS, typename S, typename real, typename Idx>
__device__ __forceinline__ void pop_put(const StepArgs<real>& p, int i, Idx s, Idx N, real fY, real fD, real c) {
    if constexpr (Stored<S>::kDev) fY -= (real)VS::w(i) * p.rho_ref * c;
    slots_put<VS, S>(p.fout, (Idx)i * N + s, N, fY, fD);
}

template <typename S, typename real, typename Idx>
__device__ __forceinline__ void ref_put(const StepArgs<real>& p, Idx s, real c) {
    if constexpr (Stored<S>::kDev) p.ref_out[s] = c;
}

// ink fraction used as the 16-bit reference (0 for an empty site)
template <typename real>
__device__ __forceinline__ real ref_frac(real rY, real rB) {
    const real t = rY + rB;
    return t > real(0) ? rY / t : real(0);
}

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
// periodic wrap of any offset; the modulo runs only when a leaves [0, n)
__device__ __forceinline__ int wrapn(int a, int n) {
    if (a >= 0 && a < n) return a;
    a %= n;
    return a < 0 ? a + n : a;
}

template <typename real>
__device__ __forceinline__ real clampr(real v, real lo, real hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

template <typename real>
__device__ __forceinline__ long long ridx(const StepArgs<real>& p, int x, int y, int z) {
    return (long long)(z + 1) * p.plane + (long long)y * p.nx + x;
}

template <typename real>
__device__ __forceinline__ long long sidx(const StepArgs<real>& p, int x, int y, int z) {
    return (long long)z * p.plane + (long long)y * p.nx + x;
}

// ---------------------------------------------------------------------------
// Nozzle template (Sec. II B), fixed point
// ---------------------------------------------------------------------------

__device__ __forceinline__ long long near_image(long long d, long long period) {
    // d in (-period, period) because the head coordinate is reduced on the host
    if (2 * d >= period) d -= period;
    else if (2 * d < -period) d += period;
    return d;
}

template <typename real>
__device__ __forceinline__ long long axis_d2(const StepArgs<real>& p, int x, int y, int which) {
    long long dx = near_image((long long)x * 1048576LL - p.hx[which], p.px);
    long long dy = near_image((long long)y * 1048576LL - p.hy[which], p.py);
    return dx * dx + dy * dy;
}

// The nozzle is a vertical annulus above the gap, so a column's relation to it
// does not depend on z: k_geo classifies each queried column once per step
// (exact fixed-point arithmetic) and the per-site tests read a byte.
enum {
    kGeoSolid0 = 1,   // r_in <= r <= r_out at step n-1
    kGeoSolid1 = 2,   // same at step n
    kGeoIn0 = 4,      // r < r_in at step n-1 (inlet above the top)
    kGeoIn1 = 8,      // r < r_in at step n (ink of the initial fill)
    kGeoClear0 = 16,  // 3/2 clear of the wall's radii at step n-1
};

template <typename real>
__device__ __forceinline__ unsigned geo_flags(const StepArgs<real>& p, int x, int y) {
    const long long d0 = axis_d2(p, x, y, 0), d1 = axis_d2(p, x, y, 1);
    unsigned g = 0;
    if (d0 >= p.rin2 && d0 <= p.rout2) g |= kGeoSolid0;
    if (d1 >= p.rin2 && d1 <= p.rout2) g |= kGeoSolid1;
    if (d0 < p.rin2) g |= kGeoIn0;
    if (d1 < p.rin2) g |= kGeoIn1;
    if (d0 < p.rclear_in2 || d0 > p.rclear_out2) g |= kGeoClear0;
    return g;
}

template <typename real>
__device__ __forceinline__ unsigned geo_at(const StepArgs<real>& p, int x, int y) {
    return p.geo[y * p.nx + x];
}

// nozzle wall node (z >= gap, r_in <= r <= r_out) on the geometry of step n-1 (0) or n (1)
template <typename real>
__device__ __forceinline__ bool solid_at(const StepArgs<real>& p, int x, int y, int z, int which) {
    if (!p.nozzle || z < p.gap) return false;
    return (geo_at(p, x, y) & (which ? kGeoSolid1 : kGeoSolid0)) != 0;
}

// ---------------------------------------------------------------------------
// Streaming with the boundary rules (Eq. 1, 26-28), full generality.
// Pulls the populations of fluid site (x, y, z) of the step-(n-1) geometry.
// bc[k] accumulates the mass change of the boundary links.
// ---------------------------------------------------------------------------

template <typename real>
__device__ __forceinline__ real wall_density(const StepArgs<real>& p, int k, int x, int y, int z, int cx, int cy,
                                             int cz, long long s_self) {
    // Eq. 26: density at the wall by quadratic extrapolation along +c_i from
    // x (distance 1/2), x + c_i (3/2), x + 2 c_i (5/2), using the step-(n-1)
    // densities; falls back to the node's own density if either is not fluid.
    const real r0 = p.rho_prev[(long long)k * (p.N + 2 * p.plane) + s_self + p.plane];
    const int x1 = wrapn(x + cx, p.nx), y1 = wrapn(y + cy, p.ny);
    const int x2 = wrapn(x + 2 * cx, p.nx), y2 = wrapn(y + 2 * cy, p.ny);
    int z1 = z + cz, z2 = z + 2 * cz;
    if (p.z_mode == kZPeriodic) {
        z1 = wrapn(z1, p.nz);
        z2 = wrapn(z2, p.nz);
    } else if (z1 < 0 || z1 >= p.nz || z2 < 0 || z2 >= p.nz) {
        return r0;
    }
    if (solid_at(p, x1, y1, z1, 0) || solid_at(p, x2, y2, z2, 0)) return r0;
    const long long off = (long long)k * (p.N + 2 * p.plane);
    const real r1 = p.rho_prev[off + ridx(p, x1, y1, z1)];
    const real r2 = p.rho_prev[off + ridx(p, x2, y2, z2)];
    return (real(15) * r0 - real(10) * r1 + real(3) * r2) * real(0.125);
}

// index of the velocity of the top two planes (z = nz-2, nz-1)
template <typename real>
__device__ __forceinline__ long long utop_idx(const StepArgs<real>& p, int a, int x, int y, int z) {
    return ((long long)a * 2 + (z - (p.nz - 2))) * p.plane + (long long)y * p.nx + x;
}

template <typename real>
__device__ __forceinline__ void anti_bb_velocity(const StepArgs<real>& p, int x, int y, int z, int cx, int cy, int cz,
                                                 real uw[3]) {
    // Eq. 28: half-way velocity by second-order extrapolation
    // 1.5 u(x) - 0.5 u(x + c_i), step n-1 values; u(x) alone if x + c_i is not fluid
    for (int a = 0; a < 3; ++a) uw[a] = p.u_prev[utop_idx(p, a, x, y, z)];
    const int z1 = z + cz;
    if (z1 < 0 || z1 < p.nz - 2) return;
    const int x1 = wrapn(x + cx, p.nx), y1 = wrapn(y + cy, p.ny);
    if (solid_at(p, x1, y1, z1, 0)) return;
    for (int a = 0; a < 3; ++a) uw[a] = real(1.5) * uw[a] - real(0.5) * p.u_prev[utop_idx(p, a, x1, y1, z1)];
}

enum { kLinkFluid = 0, kLinkRest, kLinkMoving, kLinkOpen };

template <typename real>
__device__ __forceinline__ int classify(const StepArgs<real>& p, int x, int y, int z, int cx, int cy, int cz,
                                        long long* src, real uw[3]) {
    const int sx = wrapn(x - cx, p.nx), sy = wrapn(y - cy, p.ny);
    int sz = z - cz;
    uw[0] = uw[1] = uw[2] = real(0);
    if (p.z_mode == kZPeriodic) {
        *src = sidx(p, sx, sy, wrapn(sz, p.nz));
        return kLinkFluid;
    }
    if (sz < 0) return kLinkRest;  // substrate: resting wall half-way below z = 0
    if (sz >= p.nz) {
        if (p.top_mode == kTopWall) {
            uw[0] = p.utop[0]; uw[1] = p.utop[1]; uw[2] = p.utop[2];
            return kLinkMoving;
        }
        if (p.nozzle) {
            const unsigned g = geo_at(p, sx, sy);
            if (g & kGeoSolid0) {
                uw[0] = p.vn[0]; uw[1] = p.vn[1]; uw[2] = p.vn[2];
                return kLinkMoving;
            }
            if (g & kGeoIn0) {  // inlet, Eq. 27
                uw[0] = p.uin[0]; uw[1] = p.uin[1]; uw[2] = p.uin[2];
                return kLinkMoving;
            }
        }
        return kLinkOpen;
    }
    if (solid_at(p, sx, sy, sz, 0)) {
        uw[0] = p.vn[0]; uw[1] = p.vn[1]; uw[2] = p.vn[2];
        return kLinkMoving;
    }
    *src = sidx(p, sx, sy, sz);
    return kLinkFluid;
}

// true if no lattice neighbour of (x, y, z) can be a nozzle node of the
// step-(n-1) geometry: every neighbour lies within sqrt(2) of the site in the
// x-y plane, so the site's distance to the axis must stay 3/2 clear of the
// wall's radii (squared radii padded in fixed point), or it lies below gap - 1
template <typename real>
__device__ __forceinline__ bool clear_of_nozzle(const StepArgs<real>& p, int x, int y, int z) {
    if (!p.nozzle || z < p.gap - 1) return true;
    return (geo_at(p, x, y) & kGeoClear0) != 0;
}

template <class VS, typename S, typename real>
__device__ __forceinline__ void pull_general(const StepArgs<real>& p, int x, int y, int z, real f[2][VS::Q],
                                             real bc[2]) {
    const long long s = sidx(p, x, y, z);
    if (p.z_mode == kZPeriodic || (z < p.nz - 1 && clear_of_nozzle(p, x, y, z))) {
        // plain streaming: every source is a fluid node, except across the
        // substrate (resting half-way wall, identity on the own population)
        const int xm = wrapn(x - 1, p.nx), xp = wrapn(x + 1, p.nx);
        const int ym = wrapn(y - 1, p.ny), yp = wrapn(y + 1, p.ny);
#pragma unroll
        for (int i = 0; i < VS::Q; ++i) {
            const int cx = VS::c(i, 0), cy = VS::c(i, 1), cz = VS::c(i, 2);
            int sz = z - cz;
            long long src;
            if (p.z_mode == kZPeriodic) sz = wrapn(sz, p.nz);
            if (sz < 0) {
                pop_get<VS, S>(p, p.fin, p.ref_in, opp(i), s, p.N, &f[0][i], &f[1][i]);
                continue;
            }
            src = sidx(p, cx > 0 ? xm : (cx < 0 ? xp : x), cy > 0 ? ym : (cy < 0 ? yp : y), sz);
            pop_get<VS, S>(p, p.fin, p.ref_in, i, src, p.N, &f[0][i], &f[1][i]);
        }
        return;
    }
    // near the nozzle or on the top plane: every link classified, in a
    // compact loop (this path is rare; its code stays small)
#pragma unroll 1
    for (int i = 0; i < VS::Q; ++i) {
        const int cx = link<VS>(i, 0), cy = link<VS>(i, 1), cz = link<VS>(i, 2);
        long long src = 0;
        real uw[3];
        const int kind = classify(p, x, y, z, cx, cy, cz, &src, uw);
        const int ib = opp(i);
        if (kind == kLinkFluid) {
            pop_get<VS, S>(p, p.fin, p.ref_in, i, src, p.N, &f[0][i], &f[1][i]);
            continue;
        }
        real oY, oD;  // f*^Y_ib(x) and d*_ib(x), heading to the boundary
        pop_get<VS, S>(p, p.fin, p.ref_in, ib, s, p.N, &oY, &oD);
        const real w = (real)VS::w(ib);
        real vY, vD;
        if (kind == kLinkRest) {
            vY = oY;
            vD = oD;
        } else if (kind == kLinkMoving) {
            // Eq. 26 per component; for the total the wall densities add up
            const real rwY = wall_density(p, 0, x, y, z, cx, cy, cz, s);
            const real rwB = wall_density(p, 1, x, y, z, cx, cy, cz, s);
            const real ucb = -((real)cx * uw[0] + (real)cy * uw[1] + (real)cz * uw[2]);
            vY = oY - real(6) * w * rwY * ucb;
            vD = oD - real(6) * w * (rwY + rwB) * ucb;
        } else {
            // Eq. 28 with imposed densities 0 (ink) and rho_top (ambient)
            real u2[3];
            anti_bb_velocity(p, x, y, z, cx, cy, cz, u2);
            const real cu = -((real)cx * u2[0] + (real)cy * u2[1] + (real)cz * u2[2]);  // c_ib . u
            const real uu = u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2];
            const real q = real(4.5) * cu * cu - real(1.5) * uu;
            vY = -oY;
            vD = -oD + real(2) * (p.rho_top * p.dphi[1][ib] + w * (p.rho_top - p.rho_ref) + p.rho_top * w * q);
        }
        f[0][i] = vY;
        f[1][i] = vD;
        bc[0] += vY - oY;
        bc[1] += (vD - oD) - (vY - oY);
    }
}

// ink population and total deviation of the equilibrium pair at density
// (rY, rB) and velocity u (Eq. 6): f^Y_i and sum_k f^k,eq_i - w_i rho_ref
template <class VS, typename real>
__device__ __forceinline__ void feq_pair(const StepArgs<real>& p, int i, real rY, real rB, real ux, real uy, real uz,
                                         real uu, real* eY, real* eD) {
    const real cu = (real)VS::c(i, 0) * ux + (real)VS::c(i, 1) * uy + (real)VS::c(i, 2) * uz;
    const real w = (real)VS::w(i);
    const real base = real(3) * cu + real(4.5) * cu * cu - real(1.5) * uu;
    *eY = rY * (p.phi[0][i] + w * base);
    *eD = rY * p.dphi[0][i] + rB * p.dphi[1][i] + w * ((rY + rB) - p.rho_ref) + (rY + rB) * w * base;
}

// ---------------------------------------------------------------------------
// Local relaxation time (Eq. 17, 23-25)
// ---------------------------------------------------------------------------

template <typename real>
__device__ __forceinline__ real rpow(real a, real b);
template <>
__device__ __forceinline__ double rpow<double>(double a, double b) { return pow(a, b); }
template <>
__device__ __forceinline__ float rpow<float>(float a, float b) { return powf(a, b); }

// Quotient, square root and reciprocal square root for the collision's smooth
// coefficients (velocity, colour fraction, mixture viscosity, perturbation and
// recolouring amplitudes). FP64 keeps the IEEE operations; FP32 takes the
// hardware approximations (within 2 ulp), far below the FP32 storage rounding
// that already bounds the single-precision path.
template <typename real>
__device__ __forceinline__ real qdiv(real a, real b);
template <>
__device__ __forceinline__ double qdiv<double>(double a, double b) { return a / b; }
template <>
__device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

template <typename real>
__device__ __forceinline__ real qrsqrt(real a);  // a > 0
template <>
__device__ __forceinline__ double qrsqrt<double>(double a) { return 1.0 / sqrt(a); }
template <>
__device__ __forceinline__ float qrsqrt<float>(float a) { return rsqrtf(a); }

template <typename real>
__device__ __forceinline__ real qsqrt(real a);  // a >= 0
template <>
__device__ __forceinline__ double qsqrt<double>(double a) { return sqrt(a); }
template <>
__device__ __forceinline__ float qsqrt<float>(float a) { return a > 0.0f ? a * rsqrtf(a) : 0.0f; }

// Square of the |grad rho^N| at or below which the recolouring direction of
// Eq. 16 is undefined: 2^8 units of rounding of the arithmetic, 2^-45 in FP64
// and 2^-16 in FP32 (the colour fractions the gradient is formed from carry a
// few units of rounding each).
template <typename real>
__device__ __forceinline__ constexpr real grad_floor2();
template <>
__device__ __forceinline__ constexpr double grad_floor2<double>() { return 0x1p-90; }
template <>
__device__ __forceinline__ constexpr float grad_floor2<float>() { return 0x1p-32f; }

// ink fraction rho_Y / (rho_Y + rho_B) of a site's densities
template <typename real>
__device__ __forceinline__ real colour_frac(real a, real b) { return qdiv(a, a + b); }

// tau of the ink law at shear rate g (unclamped) and d tau / d g
template <typename real>
__device__ __forceinline__ void tau_law(const StepArgs<real>& p, real g, real* t, real* dt) {
    if (p.law == kLawCross) {
        const real xg = rpow(p.lambda * g, p.n_exp);
        const real inv = real(1) / (real(1) + xg);
        const real nu = p.nu_inf + (p.nu0 - p.nu_inf) * inv;
        *t = real(0.5) + real(3) * nu;
        *dt = g > real(0) ? -real(3) * (p.nu0 - p.nu_inf) * p.n_exp * xg * inv * inv / g : real(0);
    } else {  // power law
        const real nu = p.K * rpow(g, p.n_exp - real(1));
        *t = real(0.5) + real(3) * nu;
        *dt = real(3) * (p.n_exp - real(1)) * nu / g;
    }
}

// tau of the ink at zero shear rate (clamped)
template <typename real>
__device__ __forceinline__ real tau_zero_shear(const StepArgs<real>& p) {
    if (p.law == kLawPower) {
        if (p.n_exp < real(1)) return p.tau_max;
        if (p.n_exp > real(1)) return p.tau_min;
        return clampr(real(0.5) + real(3) * p.K, p.tau_min, p.tau_max);
    }
    return clampr(real(0.5) + real(3) * p.nu0, p.tau_min, p.tau_max);
}

// The ink's largest weight in the mixture's relaxation time (Eq. 17), with
// its viscosity at least nu_min (that at tau_min): (c_Y/nu_min) / (c_Y/nu_min +
// c_B/nu_B). cY, cB: the site's colour fractions.
template <typename real>
__device__ __forceinline__ real ink_weight(const StepArgs<real>& p, real cY, real cB) {
    const real aYm = qdiv(cY * real(3), p.tau_min - real(0.5)), aBm = qdiv(cB, p.nuB);
    return qdiv(aYm, aYm + aBm);
}

// Root of g tau_Y(g) = S / (rho_Y c_s^2) (Eq. 24-25) by Newton's method kept
// inside the bracket [s / tau_max, s / tau_min] (bisection when a step leaves
// it). Returns the clamped tau_Y.
//
// The root serves the mixture's relaxation time (Eq. 17), in which the ink's
// viscosity enters with at most the weight w = (c_Y/nu_min) / (c_Y/nu_min +
// c_B/nu_B) (nu_min: the viscosity at tau_min). A relative error e in tau_Y
// moves the mixture's tau by at most about w e, so the iteration stops when
// its relative step is below tol / w (tol when w = 1, at most 1e-2), and where
// w <= tol the ink's viscosity cannot move tau by tol at all and its
// zero-shear value is taken. Either way the mixture's tau is within tol
// (relative) of the one the exact root gives.
template <typename real>
__device__ __forceinline__ real solve_tau_ink(const StepArgs<real>& p, real S, real rhoY, real rho, real wmax) {
    if (p.law == kLawNewtonian) return clampr(real(0.5) + real(3) * p.nu0, p.tau_min, p.tau_max);
    if (!(rhoY > real(1e-12) * rho) || !(S > real(0)) || !(wmax > p.tol)) return tau_zero_shear(p);
    const real tol = fmin(p.tol / wmax, real(1e-2));
    const real s = real(3) * S / rhoY;
    real lo = s / p.tau_max, hi = s / p.tau_min;
    real t, dt;
    tau_law(p, lo, &t, &dt);
    if (t >= p.tau_max) return p.tau_max;  // root on the tau_max branch
    tau_law(p, hi, &t, &dt);
    if (t <= p.tau_min) return p.tau_min;  // root on the tau_min branch
    // start near the root: for the power law, the root of its larger term
    // alone (g/2 = s or 3K g^n = s; an upper bound of the root, since both
    // terms are positive); for the Cross law, one fixed-point step from the
    // zero-shear relaxation time
    real g;
    if (p.law == kLawPower) {
        g = fmin(real(2) * s, rpow(s * qdiv(real(1), real(3) * p.K), qdiv(real(1), p.n_exp)));
    } else {
        tau_law(p, s / tau_zero_shear(p), &t, &dt);
        g = s / clampr(t, p.tau_min, p.tau_max);
    }
    g = clampr(g, lo, hi);
    for (int it = 0; it < p.max_iter; ++it) {
        tau_law(p, g, &t, &dt);
        if (t > p.tau_max) { t = p.tau_max; dt = real(0); }
        else if (t < p.tau_min) { t = p.tau_min; dt = real(0); }
        const real h = g * t - s;
        if (h < real(0)) lo = g; else hi = g;
        real gn = g - h / (t + g * dt);
        if (!(gn > lo && gn < hi)) gn = real(0.5) * (lo + hi);
        const real step = gn - g;
        g = gn;
        if (fabs(step) <= tol * g) break;
    }
    tau_law(p, g, &t, &dt);
    return clampr(t, p.tau_min, p.tau_max);
}

// ---------------------------------------------------------------------------
// Collision at one fluid site (Eq. 4-20, 29).
//   f[k][i]: populations after streaming, replaced by the post-collision ones.
//   nb(i, &cY, &cB, &rn): colour fractions rho_Y/rho, rho_B/rho and phase
//   field rho^N of the neighbour x + c_i (fluid, wall or ghost node).
//   zdist: distance to the substrate (drag zone), < 0 when there is none.
// Outputs the physical velocity and tau for the fields.
// ---------------------------------------------------------------------------

template <typename real>
struct SiteOut {
    real rhoY, rhoB, u[3], tau, rn;
    real cY;  // ink fraction rho_Y / rho after streaming
};

template <typename real>
__device__ __forceinline__ real phase_field(const StepArgs<real>& p, real rY, real rB) {
    const real aY = rY / p.rho0[0], aB = rB / p.rho0[1];
    return (aY - aB) / (aY + aB);
}

// Collision at one fluid site (Eq. 4-20, 29).
//   f[0][i]: ink populations, f[1][i]: total deviation d_i (see the storage
//   note at the top); both replaced by the post-collision values.
//   kUnit: reference densities equal and phi = w (density ratio one); the
//   neighbour accessor then returns the ink fraction cY only, since
//   rho_B/rho = 1 - cY and rho^N = 2 cY - 1. Otherwise it returns
//   (cY, cB, rho^N).
//   zdist: distance to the substrate (drag zone), < 0 when there is none.
//
// The regularised collision (Eq. 20) rebuilds every population from the
// moments, so the step splits in two: moments() takes what the site's own
// populations after streaming give (ink density, total deviation, momentum,
// the two non-equilibrium stresses: 17 numbers), collide_out() adds the
// neighbours' colour fractions and writes the new populations, each pair of
// opposite directions (2p-1, 2p) sharing its even part. collide() is the two
// in sequence.

template <typename real>
struct Moments {
    real rY, sd;   // ink density, sum of the total deviations
    real m[3];     // momentum sum_i c_i d_i
    real PY[6];    // ink non-equilibrium stress (Eq. 20): xx yy zz xy xz yz
    real PT[6];    // mixture non-equilibrium stress
};

// Moments of a site after streaming (Eq. 2-3, 20).
//
// The ink's non-equilibrium stress Pi^Y = sum_i f^Y_i c_i c_i - rho_Y (p_Y I
// + u u) is a difference of O(rho_Y) numbers that is 10^-3..10^-4 of them in
// the print flow, and the shear rate of Eq. 24 is read from it. In FP64 it is
// summed as written. In FP32 the direct sum would lose about 3 digits to that
// cancellation, so the stress is taken apart exactly: with c = rho_Y / rho
// and the ink's excess over its share of the total, h_i = f^Y_i - c f_i
// (f_i = W_i + d_i, W_i = w_i rho_ref as rounded in p.wref),
//   sum_i f^Y_i c_i c_i = c (sum_i W_i c_i c_i + sum_i d_i c_i c_i) + sum_i h_i c_i c_i,
// which for any c gives
//   Pi^Y = c Pi + H - (sum_i h_i)(I/3 + u u) + c kappa I   (density ratio one),
// Pi the mixture stress (formed from the small deviations d_i), H the second
// moment of h and kappa the rounding of the weights, sum_i W_i c_x^2 - rho_ref/3
// - (sum_i W_i - rho_ref)/3 (p.kappa_w, exact on the host). h_i is small
// (the recolouring term and the rounding of the stored values), so the sums
// carry no cancellation and every operation stays in FP32.
template <typename T>
__device__ __forceinline__ T rfma(T a, T b, T c) { return fma(a, b, c); }

template <class VS, typename real>
__device__ __forceinline__ void moments(const StepArgs<real>& p, const real f[2][VS::Q], Moments<real>* M) {
    constexpr int Q = VS::Q;
    constexpr bool kSplit = sizeof(real) < sizeof(double);
    // moments (Eq. 2-3) and the second moments of the total deviation (and,
    // in FP64, of the ink), accumulated direction by direction: ink density
    // from slot 0, total density and momentum from the deviation slot
    // (sum_i w_i c_i = 0). The densities are summed in direction order, as
    // every density of the step is, so that a site's colour fraction is the
    // same bit for bit wherever it is computed.
    real rY = 0, sd = 0, mx = 0, my = 0, mz = 0;
    real a[6] = {0, 0, 0, 0, 0, 0}, b[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rY += f[0][i];
        sd += f[1][i];
    }
    // first and second moments over pairs of opposite directions (2q-1, 2q):
    // the pair's sum carries the second moments, its difference the momentum
#pragma unroll
    for (int q = 0; q < (Q - 1) / 2; ++q) {
        const int i = 2 * q + 1;
        const int cx = VS::c(i, 0), cy = VS::c(i, 1), cz = VS::c(i, 2);
        const real ds = f[1][i] + f[1][i + 1], dd = f[1][i] - f[1][i + 1];
        if (cx) mx += cx > 0 ? dd : -dd;
        if (cy) my += cy > 0 ? dd : -dd;
        if (cz) mz += cz > 0 ? dd : -dd;
        if (cx) b[0] += ds;
        if (cy) b[1] += ds;
        if (cz) b[2] += ds;
        if (cx && cy) b[3] += (cx == cy) ? ds : -ds;
        if (cx && cz) b[4] += (cx == cz) ? ds : -ds;
        if (cy && cz) b[5] += (cy == cz) ? ds : -ds;
        if constexpr (!kSplit) {
            const real ys = f[0][i] + f[0][i + 1];
            if (cx) a[0] += ys;
            if (cy) a[1] += ys;
            if (cz) a[2] += ys;
            if (cx && cy) a[3] += (cx == cy) ? ys : -ys;
            if (cx && cz) a[4] += (cx == cz) ? ys : -ys;
            if (cy && cz) a[5] += (cy == cz) ? ys : -ys;
        }
    }
    const real rho = p.rho_ref + sd;
    const real rB = rho - rY;
    const real irho = qdiv(real(1), rho);
    const real ux = mx * irho, uy = my * irho, uz = mz * irho;

    // mixture non-equilibrium stress (Eq. 20):
    // Pi = sum d c c - [sum_k rho_k pfac_k - rho_ref c_s^2] I - rho u u
    real* PY = M->PY;
    real* PT = M->PT;
    // (rho - rho_ref) c_s^2 formed from sd itself, not from the rounded rho
    real pT = sd * real(1.0 / 3.0);
    if (!p.unit) pT += rY * (p.pfac[0] - real(1.0 / 3.0)) + rB * (p.pfac[1] - real(1.0 / 3.0));
    PT[0] = b[0] - (pT + rho * ux * ux);
    PT[1] = b[1] - (pT + rho * uy * uy);
    PT[2] = b[2] - (pT + rho * uz * uz);
    PT[3] = b[3] - rho * ux * uy;
    PT[4] = b[4] - rho * ux * uz;
    PT[5] = b[5] - rho * uy * uz;
    if constexpr (kSplit) {
        // ink stress by the split above: c Pi + H - h0 (I/3 + u u) + c kappa I
        const real c = rY * irho;
        real h0 = rfma(-c, f[1][0], rfma(-c, p.wref[0], f[0][0])), H[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < (Q - 1) / 2; ++q) {
            const int i = 2 * q + 1;
            const int cx = VS::c(i, 0), cy = VS::c(i, 1), cz = VS::c(i, 2);
            // opposite directions share w_i, so wref too
            const real h = rfma(-c, f[1][i], rfma(-c, p.wref[i], f[0][i])) +
                           rfma(-c, f[1][i + 1], rfma(-c, p.wref[i], f[0][i + 1]));
            h0 += h;
            if (cx) H[0] += h;
            if (cy) H[1] += h;
            if (cz) H[2] += h;
            if (cx && cy) H[3] += (cx == cy) ? h : -h;
            if (cx && cz) H[4] += (cx == cz) ? h : -h;
            if (cy && cz) H[5] += (cy == cz) ? h : -h;
        }
        // isotropic part: -h0/3 + c kappa, and away from density ratio one the
        // partial-pressure terms (c - 1) rho_Y (p_Y - 1/3) + c rho_B (p_B - 1/3)
        real iso = rfma(c, p.kappa_w, -h0 * real(1.0 / 3.0));
        if (!p.unit)
            iso += (c - real(1)) * rY * (p.pfac[0] - real(1.0 / 3.0)) + c * rB * (p.pfac[1] - real(1.0 / 3.0));
        PY[0] = rfma(c, PT[0], H[0]) + (iso - h0 * ux * ux);
        PY[1] = rfma(c, PT[1], H[1]) + (iso - h0 * uy * uy);
        PY[2] = rfma(c, PT[2], H[2]) + (iso - h0 * uz * uz);
        PY[3] = rfma(c, PT[3], H[3]) - h0 * ux * uy;
        PY[4] = rfma(c, PT[4], H[4]) - h0 * ux * uz;
        PY[5] = rfma(c, PT[5], H[5]) - h0 * uy * uz;
    } else {
        // ink non-equilibrium stress as written: sum f^Y c c - rY (pfac_Y I + u u)
        const real pY = p.pfac[0] * rY;
        PY[0] = a[0] - (pY + rY * ux * ux);
        PY[1] = a[1] - (pY + rY * uy * uy);
        PY[2] = a[2] - (pY + rY * uz * uz);
        PY[3] = a[3] - rY * ux * uy;
        PY[4] = a[4] - rY * ux * uz;
        PY[5] = a[5] - rY * uy * uz;
    }
    if (VS::kPlanar) { PY[1] = PY[3] = PY[5] = 0; PT[1] = PT[3] = PT[5] = 0; }
    M->rY = rY;
    M->sd = sd;
    M->m[0] = mx;
    M->m[1] = my;
    M->m[2] = mz;
}

// The collision from the moments and the neighbours' colour fractions
// (Eq. 5-17, 20, 29): out(i, fY_i, d_i, cY) receives the post-collision ink
// population and total deviation of each direction i (cY: the site's ink
// fraction, for the 16-bit storage reference).
template <class VS, typename real, bool kUnit, typename Nb, typename Out>
__device__ __forceinline__ void collide_out(const StepArgs<real>& p, const Moments<real>& M, const Nb& nb, real zdist,
                                            SiteOut<real>* so, Out&& out) {
    constexpr int Q = VS::Q;
    constexpr int NP = (Q - 1) / 2;
    const real rY = M.rY;
    const real rho = p.rho_ref + M.sd;
    const real rB = rho - rY;
    const real irho = qdiv(real(1), rho);
    const real ux = M.m[0] * irho, uy = M.m[1] * irho, uz = M.m[2] * irho;
    const real cY0 = rY * irho, cB0 = rB * irho;
    const real* PY = M.PY;
    const real* PT = M.PT;

    // colour-gradient force (Eq. 11) and grad rho^N by the isotropic stencil
    // (Eq. 12), as pair differences 3 sum_p w_p c_p [chi(x + c_p) - chi(x - c_p)]:
    // equal to the printed form (sum_i w_i c_i = 0) and exactly zero on a
    // uniform field
    real F[3], gN[3], rn0;
    if constexpr (kUnit) {
        real g[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int i = 2 * q + 1;
            const real dd = (real)VS::w(i) * (nb(i) - nb(i + 1));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (VS::c(i, a) > 0) g[a] += dd;
                else if (VS::c(i, a) < 0) g[a] -= dd;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F[a] = real(3) * g[a];            // grad(rho_Y/rho); F = (cB0 + cY0) grad cY
            gN[a] = real(6) * g[a];           // rho^N = 2 cY - 1
        }
        rn0 = cY0 - cB0;
    } else {
        real gY[3] = {0, 0, 0}, gB[3] = {0, 0, 0}, gR[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int i = 2 * q + 1;
            real aY, aB, aN, bY, bB, bN;
            nb(i, &aY, &aB, &aN);
            nb(i + 1, &bY, &bB, &bN);
            const real w = (real)VS::w(i);
            const real dY = w * (aY - bY), dB = w * (aB - bB), dN = w * (aN - bN);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (VS::c(i, a) > 0) { gY[a] += dY; gB[a] += dB; gR[a] += dN; }
                else if (VS::c(i, a) < 0) { gY[a] -= dY; gB[a] -= dB; gR[a] -= dN; }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F[a] = real(3) * (cB0 * gY[a] - cY0 * gB[a]);
            gN[a] = real(3) * gR[a];
        }
        rn0 = phase_field(p, rY, rB);
    }
    const real Fn2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    const real gN2 = gN[0] * gN[0] + gN[1] * gN[1] + gN[2] * gN[2];
    const real gNn = qsqrt(gN2);

    // local relaxation time: ink viscosity from Eq. 24-25, harmonic mixing
    // by mass fraction (Eq. 17), clamp
    const real S = qsqrt(PY[0] * PY[0] + PY[1] * PY[1] + PY[2] * PY[2] +
                         real(2) * (PY[3] * PY[3] + PY[4] * PY[4] + PY[5] * PY[5]));
    const real tauY = solve_tau_ink(p, S, rY, rho, ink_weight(p, cY0, cB0));
    const real nuY = (tauY - real(0.5)) * real(1.0 / 3.0);
    const real inv_nu = qdiv(cY0, nuY) + qdiv(cB0, p.nuB);
    const real tau = clampr(real(0.5) + qdiv(real(3), inv_nu), p.tau_min, p.tau_max);
    const real om45 = (real(1) - qdiv(real(1), tau)) * real(4.5);

    // body force and drag by the exact difference method (Eq. 29): the
    // equilibrium is taken at v = u + F/rho, f^eq(u) + [f^eq(v) - f^eq(u)]
    real Fb[3] = {rho * p.g[0], rho * p.g[1], rho * p.g[2]};
    if (p.drag_gamma != real(0) && zdist >= real(0) && zdist < p.drag_height) {
        Fb[0] -= p.drag_gamma * rY * ux;
        Fb[1] -= p.drag_gamma * rY * uy;
        Fb[2] -= p.drag_gamma * rY * uz;
    }
    const real vx = ux + Fb[0] * irho, vy = uy + Fb[1] * irho, vz = uz + Fb[2] * irho;
    const real vv15 = real(1.5) * (vx * vx + vy * vy + vz * vz);

    // perturbation (Eq. 10) once on the total; recolouring (Eq. 14-16) with
    // cos(phi_i) = c.grad / (|c| |grad|) as printed (Eq. 16), taken as 0 where
    // |grad rho^N| is at or below the rounding level of the arithmetic (the
    // 0/0 case: such a gradient has no meaningful direction)
    const bool pert = gNn > real(0) && Fn2 > real(0);
    const real pA = pert ? real(0.5) * p.A * gNn : real(0);
    const real pAF = pert ? qdiv(pA, Fn2) : real(0);
    const real rec = gN2 > grad_floor2<real>() ? p.beta * rY * rB * irho * irho * qrsqrt(gN2) : real(0);
    const real tr3 = (PT[0] + PT[1] + PT[2]) * real(1.0 / 3.0);
    const real drho = M.sd;  // rho - rho_ref, the deviation sum itself

    // The collision conserves each component's mass (Eq. 5, 10, 14-15, 20,
    // 29 each add zero mass), so the rest direction is written last as what
    // that leaves: f^Y_0 = rho_Y - sum_{i>0} f^Y_i and d_0 = sd - sum_{i>0} d_i.
    // In exact arithmetic this is the rest direction's formula; in FP32 it
    // keeps the rounding of c_Y rho and of the weights (sum_i fl(w_i) != 1)
    // from adding the same error to a site's mass at every step.
    real sY = 0, sD = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int i = 2 * q + 1;
        const int cx = VS::c(i, 0), cy = VS::c(i, 1), cz = VS::c(i, 2);
        const real w = (real)VS::w(i);
        const real cv = cx * vx + cy * vy + cz * vz;
        // even part: rest-frame share, quadratic equilibrium terms,
        // regularised non-equilibrium (1 - 1/tau) w/(2 c_s^4) (c.Pi.c - c_s^2 tr Pi)
        // and the perturbation; odd part: the linear equilibrium term
        const real qT = cx * cx * PT[0] + cy * cy * PT[1] + cz * cz * PT[2] +
                        real(2) * (cx * cy * PT[3] + cx * cz * PT[4] + cy * cz * PT[5]) - tr3;
        const real Fc = cx * F[0] + cy * F[1] + cz * F[2];
        real e = w * drho + rho * w * (real(4.5) * cv * cv - vv15) + om45 * w * qT +
                 (pert ? pAF * w * Fc * Fc - pA * (real)VS::B(i) : real(0));
        if constexpr (!kUnit) e += rY * p.dphi[0][i] + rB * p.dphi[1][i];
        const real o = real(3) * rho * w * cv;
        const real cg = (cx * gN[0] + cy * gN[1] + cz * gN[2]) * (real)VS::inv_norm(i);
        real e0;
        if constexpr (kUnit) e0 = rho * w;
        else e0 = rY * p.phi[0][i] + rB * p.phi[1][i];
        const real G = rec * cg * e0;
        const real dp = e + o, dm = e - o;
        const real yp = cY0 * (w * p.rho_ref + dp) + G, ym = cY0 * (w * p.rho_ref + dm) - G;
        out(i, yp, dp, cY0);
        out(i + 1, ym, dm, cY0);
        sY += yp + ym;
        sD += dp + dm;
    }
    // rest direction
    out(0, rY - sY, M.sd - sD, cY0);

    so->rhoY = rY;
    so->rhoB = rB;
    so->u[0] = ux + real(0.5) * Fb[0] * irho;
    so->u[1] = uy + real(0.5) * Fb[1] * irho;
    so->u[2] = uz + real(0.5) * Fb[2] * irho;
    so->tau = tau;
    so->rn = rn0;
    so->cY = cY0;
}

template <class VS, typename real, bool kUnit, typename Nb>
__device__ __forceinline__ void collide(const StepArgs<real>& p, real f[2][VS::Q], const Nb& nb, real zdist,
                                        SiteOut<real>* so) {
    Moments<real> M;
    moments<VS>(p, f, &M);
    collide_out<VS, real, kUnit>(p, M, nb, zdist, so, [&](int i, real fY, real fD, real) {
        f[0][i] = fY;
        f[1][i] = fD;
    });
}

// unstable: the total density is not finite and positive (a vanishing
// component may dip slightly below zero at moving walls; that is not flagged)
template <typename real>
__device__ __forceinline__ bool unstable_site(real rY, real rB) {
    const real rho = rY + rB;
    return !(rho > real(0) && rho < real(1e6));
}

}  // namespace cglbm
