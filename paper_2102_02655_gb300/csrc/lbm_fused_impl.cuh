// Fused bulk step (templates; lbm_fused_<storage>.cu instantiate them, one
// translation unit per storage type): one kernel does streaming, moments, colour gradient, local
// relaxation time, regularised collision, perturbation and recolouring for
// every site outside the nozzle box (D3Q19, substrate below, open top).
//
// Each CTA owns a 32 x 8 column tile and marches up a chunk of z-planes. The
// colour gradient (Eq. 12) needs this step's densities at the 18 neighbours,
// which other CTAs produce, so for the plane ahead the CTA pulls:
//   - the populations of its own sites, kept in shared memory until the
//     collision of that plane (one iteration later), and their densities;
//   - the densities of the one-site halo ring around the tile (these re-reads
//     of neighbouring tiles' populations are served by L2);
// and keeps four planes of colour fractions in shared memory (a ring: the
// plane written for z + 1 is never one that a collision of plane z - 1 still
// reads, so one barrier per plane suffices). HBM traffic is one read and one
// write of the populations per site update.
//
// Indices are 32-bit (the host selects this kernel only when 38 N < 2^31);
// the periodic wrap in x and y is resolved once per site into the source
// column and row of each direction.
#pragma once

#include "lbm_launch.h"

namespace cglbm {

namespace {

// Tile geometry: TX x TY sites, one thread each, plus halo rings.
template <int TY_, int TX_ = 32>
struct Tile {
    static constexpr int TX = TX_, TY = TY_, NT = TX * TY;
    static constexpr int HX = TX + 2, HY = TY + 2, HS = HX * HY;  // tile + one-site halo
    static constexpr int NRING = HS - NT;                         // halo sites
    static constexpr int SX = TX + 4, SY = TY + 4, SS = SX * SY;  // tile + two rings (substrate ghost)
    static_assert(SS - HS <= NT && NRING <= NT, "ring sites must fit one item per thread");
};

__device__ __forceinline__ int slot_of(int z) { return (z + 4) & 3; }  // z >= -1

// Streaming for a site away from the nozzle on a plane below the top
// (0 <= zz <= nz - 2): every source is a fluid site except across the
// substrate, where the resting half-way wall bounces the population back
// (the pull then reads the opposite direction at the site itself). Branch-free:
// the substrate case is an address select on the upward directions only.
//
// With 16-bit storage the pull adds back c(x - c_i) w_i rho_ref (see Stored)
// from the source sites' ink fractions: read from p.ref_in, or, when rs is
// given, from shared memory: rs[k] holds plane zz - 1 + k of the tile's
// ink fractions on a box of row width W, and the site is entry rj of it.
template <typename S, typename real, int W = 0>
__device__ __forceinline__ void pull_interior(const StepArgs<real>& p, int gx, int gy, int zz, real f[2][19],
                                              const real* const* rs = nullptr, int rj = 0) {
    using VS = D3Q19;
    const int nx = p.nx, ny = p.ny, pl = (int)p.plane, N = (int)p.N;
    const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
    const int r0 = gy * nx;
    const int rm = (gy == 0 ? ny - 1 : gy - 1) * nx, rp = (gy == ny - 1 ? 0 : gy + 1) * nx;
    const int s = zz * pl + r0 + gx;
    const bool bottom = zz == 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = VS::c(i, 0), cy = VS::c(i, 1), cz = VS::c(i, 2);
        const int sx = cx > 0 ? xm : (cx < 0 ? xp : gx);
        const int sy = cy > 0 ? rm : (cy < 0 ? rp : r0);
        int src = zz * pl - cz * pl + sy + sx;
        int idx = i * N + src;
        if (cz > 0) {
            idx = bottom ? opp(i) * N + s : idx;
            src = bottom ? s : src;
        }
        slots_get<VS, S>(p.fin, idx, N, &f[0][i], &f[1][i]);
        if constexpr (Stored<S>::kDev) {
            real c;
            if constexpr (W > 0) c = rs[1 - cz][rj - cy * W - cx];
            else c = p.ref_in[src];
            f[0][i] += (real)VS::w(i) * p.rho_ref * c;
        }
    }
}

// Streaming on the top plane (zz = nz - 1; also the substrate when nz = 1):
// links leaving through the open top take the anti-bounce-back value of
// Eq. 28 with rho_Y = 0 and rho_B = rho_top, the wall velocity extrapolated
// from the last two planes of the previous step, u_w = 1.5 u(x) - 0.5 u(x + c_i).
// Writes the 38 populations to f and returns the densities after streaming
// and, when ledger, the boundary-link mass change of each component. Every
// population and velocity is loaded before the boundary rules use them, so
// the plane costs one memory round trip more than an interior one.
template <typename real>
struct TopPull {
    real rY, rB;
    double b0, b1;
};
template <typename S, typename real>
__device__ __forceinline__ TopPull<real> pull_top(const StepArgs<real>& p, int gx, int gy, real f[2][19],
                                                  bool ledger) {
    using VS = D3Q19;
    const int zz = p.nz - 1;
    const int nx = p.nx, ny = p.ny, pl = (int)p.plane, N = (int)p.N;
    const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
    const int r0 = gy * nx;
    const int rm = (gy == 0 ? ny - 1 : gy - 1) * nx, rp = (gy == ny - 1 ? 0 : gy + 1) * nx;
    const int zoff = zz * pl;
    const int s = zoff + r0 + gx;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = VS::c(i, 0), cy = VS::c(i, 1), cz = VS::c(i, 2);
        // a link from below the substrate (nz = 1) or from above the top
        // starts from the site's own opposite population
        const bool bnd = cz < 0 || (cz > 0 && zz == 0);
        const int sx = cx > 0 ? xm : (cx < 0 ? xp : gx);
        const int sy = cy > 0 ? rm : (cy < 0 ? rp : r0);
        const int src = bnd ? s : zoff - cz * pl + sy + sx;
        const int a = (bnd ? opp(i) : i) * N + src;  // w_i = w_opp(i)
        slots_get<VS, S>(p.fin, a, N, &f[0][i], &f[1][i]);
        if constexpr (Stored<S>::kDev) f[0][i] += (real)VS::w(i) * p.rho_ref * p.ref_in[src];
    }
    real u0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u0[c] = p.u_prev[c * 2 * pl + pl + r0 + gx];
    TopPull<real> r{real(0), real(0), 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = VS::c(i, 0), cy = VS::c(i, 1), cz = VS::c(i, 2);
        if (cz >= 0) continue;  // resting substrate (nz = 1): the bounced-back value as loaded
        const int ib = opp(i);
        const int x1 = cx > 0 ? xp : (cx < 0 ? xm : gx), y1 = cy > 0 ? rp : (cy < 0 ? rm : r0);
        real uw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const real un = p.u_prev[c * 2 * pl + y1 + x1];  // plane nz - 2 (slot 0 exists for nz = 1 too)
            uw[c] = p.nz >= 2 ? real(1.5) * u0[c] - real(0.5) * un : u0[c];
        }
        const real cu = -(real)(cx * uw[0] + cy * uw[1] + cz * uw[2]);  // c_ib . u_w
        const real q = real(4.5) * cu * cu - real(1.5) * (uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2]);
        const real w = (real)VS::w(i);
        const real oY = f[0][i], oD = f[1][i];
        const real fY = -oY;  // imposed ink density 0
        const real fD = -oD + real(2) * (p.rho_top * p.dphi[1][ib] + w * (p.rho_top - p.rho_ref) + p.rho_top * w * q);
        if (ledger) {
            r.b0 += (double)(fY - oY);
            r.b1 += (double)((fD - oD) - (fY - oY));
        }
        f[0][i] = fY;
        f[1][i] = fD;
    }
    real sumD = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        r.rY += f[0][i];
        sumD += f[1][i];
    }
    r.rB = (p.rho_ref + sumD) - r.rY;
    return r;
}

__device__ __forceinline__ void warp_add(double* dst, double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const unsigned lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;  // tiles narrower than a warp too
    if (lane == 0 && v != 0.0) atomicAdd(dst, v);
}

// column (x, y) inside the nozzle box's columns (any plane)
template <typename real>
__device__ __forceinline__ bool in_box_xy(const StepArgs<real>& p, int x, int y) {
    const Region& b = p.box;
    if (b.wx == 0) return false;
    int dx = x - b.x0;
    if (dx < 0) dx += p.nx;
    int dy = y - b.y0;
    if (dy < 0) dy += p.ny;
    return dx < b.wx && dy < b.wy;
}

template <typename real>
__device__ __forceinline__ bool in_box(const StepArgs<real>& p, int x, int y, int z) {
    return z >= p.box.z0 && z < p.box.z1 && in_box_xy(p, x, y);
}

template <typename real, bool kUnit, int HS>
struct Colour {
    static constexpr int NV = kUnit ? 1 : 3;
    real* col;  // [3 slots][NV][HS]
    __device__ __forceinline__ void put(const StepArgs<real>& p, int slot, int j, real rY, real rB) const {
        if constexpr (kUnit) {
            col[slot * HS + j] = colour_frac(rY, rB);
        } else {
            col[(slot * 3 + 0) * HS + j] = colour_frac(rY, rB);
            col[(slot * 3 + 1) * HS + j] = colour_frac(rB, rY);
            col[(slot * 3 + 2) * HS + j] = phase_field(p, rY, rB);
        }
    }
};

template <typename real, bool kUnit, int HX, int HS>
struct SmemNb;
template <typename real, int HX, int HS>
struct SmemNb<real, true, HX, HS> {
    const real* col;
    int slot[3], hidx;
    __device__ __forceinline__ real operator()(int i) const {
        return col[slot[1 + D3Q19::c(i, 2)] * HS + hidx + D3Q19::c(i, 0) + D3Q19::c(i, 1) * HX];
    }
};
template <typename real, int HX, int HS>
struct SmemNb<real, false, HX, HS> {
    const real* col;
    int slot[3], hidx;
    __device__ __forceinline__ void operator()(int i, real* cY, real* cB, real* rn) const {
        const int j = hidx + D3Q19::c(i, 0) + D3Q19::c(i, 1) * HX;
        const int sl = slot[1 + D3Q19::c(i, 2)];
        *cY = col[(sl * 3 + 0) * HS + j];
        *cB = col[(sl * 3 + 1) * HS + j];
        *rn = col[(sl * 3 + 2) * HS + j];
    }
};

template <int HX, int HY>
__device__ __forceinline__ void ring_coord(int r, int* hx, int* hy) {
    if (r < HX) { *hx = r; *hy = 0; }
    else if (r < 2 * HX) { *hx = r - HX; *hy = HY - 1; }
    else if (r < 2 * HX + HY - 2) { *hx = 0; *hy = 1 + r - 2 * HX; }
    else { *hx = HX - 1; *hy = 1 + r - 2 * HX - (HY - 2); }
}

template <typename real>
__device__ __forceinline__ void density(const real f[2][19], const StepArgs<real>& p, real* rY, real* rB) {
    real a = 0, b = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) { a += f[0][i]; b += f[1][i]; }
    *rY = a;
    *rB = (p.rho_ref + b) - a;
}

// One tile column (x0, y0) of planes [za, zb) of one lattice; shared memory
// as laid out by fused_smem. Used by the single-lattice kernel (one column
// per CTA) and by the persistent batched kernel (a list of columns per CTA).
// The CTA has 32 x 8 threads, one site of the 32 x 8 tile each (two sites per
// thread, on 32 x 16 tiles at two CTAs per SM, measured 20% slower). The own
// sites wait for their collision as their 17 moments
// (see moments()) rather than their 38 populations: less than half the
// shared memory and none of the populations' registers across the plane.
template <typename real, typename S, bool kUnit>
__device__ __forceinline__ void fused_column(const StepArgs<real>& p, unsigned char* smraw, int x0, int y0, int za,
                                             int zb) {
    using T = Tile<8, 32>;
    constexpr int NT = T::NT, HX = T::HX, HY = T::HY, HS = T::HS;
    constexpr int NRING = T::NRING, SX = T::SX, SY = T::SY, SS = T::SS;
    constexpr int NTH = 256;                        // threads
    constexpr int NS = 17;                          // moments staged per site
    static_assert(NRING <= NTH && SS - HS <= NTH, "one ring site per thread");
    real* pops = reinterpret_cast<real*>(smraw);   // [2 buffers][NS][NT]
    Colour<real, kUnit, HS> C{pops + 2 * NS * NT};  // [4 slots][NV][HS]
    // 16-bit storage: the ink fractions of the source sites, four planes of
    // the tile grown by two rings ([4 slots][SS], plane q in slot q mod 4)
    constexpr bool kRef = Stored<S>::kDev;
    real* refs = C.col + 4 * Colour<real, kUnit, HS>::NV * HS;
    // substrate prologue scratch [2][SS]: staging buffer 1, first written
    // after the prologue's last read of it
    real* sub = pops + NS * NT;
    static_assert(NS * NT >= 2 * SS, "substrate scratch");
    // a site waits for its collision as its 17 moments (see moments()); its
    // densities after streaming, for the colour plane, come with them
    auto stage = [&](real* b, const real f[2][19], real* rY, real* rB) {
        Moments<real> M;
        moments<D3Q19>(p, f, &M);
        *rY = M.rY;
        *rB = (p.rho_ref + M.sd) - M.rY;
        b[0] = M.rY;
        b[NT] = M.sd;
#pragma unroll
        for (int k = 0; k < 3; ++k) b[(2 + k) * NT] = M.m[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            b[(5 + k) * NT] = M.PY[k];
            b[(11 + k) * NT] = M.PT[k];
        }
    };

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    // the own site: (xs, ys), periodic image (gxs, gys), colour-ring index hidx
    const int xs = x0 + tx, ys = y0 + ty;
    const bool in_xy = xs < p.nx && ys < p.ny;
    const int gxs = in_xy ? xs : wrapn(xs, p.nx), gys = in_xy ? ys : wrapn(ys, p.ny);
    const int hidx = (ty + 1) * HX + (tx + 1);
    // the nozzle box's column test, once per column (its planes per plane)
    const bool box_xy = in_box_xy(p, xs, ys);
    double bc[2] = {0.0, 0.0};

    // Densities after streaming on plane zz for the tile (item 0, the own
    // sites) and its halo ring (item 1), and with outer also the second ring
    // (item 2, the substrate prologue). The own sites' moments go to
    // buffer zz & 1 and their boundary-link mass is booked once, for this
    // chunk's planes. One pull body serves every item.
    auto load_plane = [&](int zz, bool keep, bool outer) {
        const int nitems = outer ? 3 : 2;
        for (int it = 0; it < nitems; ++it) {
            int hx, hy;  // coordinates in the tile grown by two rings
            const bool own = it == 0;
            if (own) {
                hx = tx + 2;
                hy = ty + 2;
            } else if (it == 1) {
                if (tid >= NRING) continue;
                ring_coord<HX, HY>(tid, &hx, &hy);
                hx += 1;
                hy += 1;
            } else {
                if (tid >= SS - HS) continue;
                // the sites of the second ring
                const int j = tid;
                if (j < SX) { hx = j; hy = 0; }
                else if (j < 2 * SX) { hx = j - SX; hy = SY - 1; }
                else { const int k = j - 2 * SX; hy = 1 + (k >> 1); hx = (k & 1) ? SX - 1 : 0; }
            }
            const int px = wrapn(x0 - 2 + hx, p.nx), py = wrapn(y0 - 2 + hy, p.ny);
            real* dst = own && keep ? pops + (zz & 1) * NS * NT + tid : nullptr;
            real rY, rB;
            if (zz == p.nz - 1) {
                const bool led = own && keep && in_xy && zz < zb && !in_box(p, xs, ys, zz);
                real ft[2][19];
                const TopPull<real> res = pull_top<S>(p, px, py, ft, led);
                if (dst) stage(dst, ft, &rY, &rB);
                rY = res.rY;
                rB = res.rB;
                bc[0] += res.b0;
                bc[1] += res.b1;
            } else {
                real f[2][19];
                pull_interior<S>(p, px, py, zz, f);
                if (dst) stage(dst, f, &rY, &rB);
                else density(f, p, &rY, &rB);
            }
            if (outer) {
                sub[hy * SX + hx] = rY;
                sub[SS + hy * SX + hx] = rB;
            }
            if (it <= 1) C.put(p, slot_of(zz), (hy - 1) * HX + (hx - 1), rY, rB);
        }
    };

    // Plane zz below the top (1 <= zz <= nz - 2): the own site's pull, then
    // (warps 0-2) the halo site's.
    const bool has_halo = tid < NRING;
    int rx = 0, ry = 0;
    if (has_halo) ring_coord<HX, HY>(tid, &rx, &ry);
    const int hgx = wrapn(x0 - 1 + rx, p.nx), hgy = wrapn(y0 - 1 + ry, p.ny);
    const int hj = ry * HX + rx;
    // ink fractions of plane q on the tile grown by two rings (16-bit storage)
    auto load_ref = [&](int q) {
        for (int j = tid; j < SS; j += NTH) {
            const int gx = wrapn(x0 - 2 + j % SX, p.nx), gy = wrapn(y0 - 2 + j / SX, p.ny);
            refs[(q & 3) * SS + j] = p.ref_in[(long long)q * p.plane + (long long)gy * p.nx + gx];
        }
    };
    auto load_interior = [&](int zz) {
        real rY, rB;
        const real* rs[3] = {refs + ((zz - 1) & 3) * SS, refs + (zz & 3) * SS, refs + ((zz + 1) & 3) * SS};
        {
            real f[2][19];
            if constexpr (kRef)
                pull_interior<S, real, SX>(p, gxs, gys, zz, f, rs, (ty + 2) * SX + tx + 2);
            else
                pull_interior<S>(p, gxs, gys, zz, f);
            stage(pops + (zz & 1) * NS * NT + tid, f, &rY, &rB);
            C.put(p, slot_of(zz), hidx, rY, rB);
        }
        if (has_halo) {
            real h[2][19];
            if constexpr (kRef)
                pull_interior<S, real, SX>(p, hgx, hgy, zz, h, rs, (ry + 1) * SX + rx + 1);
            else
                pull_interior<S>(p, hgx, hgy, zz, h);
            density(h, p, &rY, &rB);
            C.put(p, slot_of(zz), hj, rY, rB);
        }
    };

    // 16-bit storage: the pull of interior plane zz (1 <= zz <= nz - 2) reads
    // the ink fractions of planes zz - 1 .. zz + 1 from shared memory. Planes
    // za .. za + 2 are loaded here, and iteration z loads plane z + 3 into the
    // slot of plane z - 1, whose last reader (the pull of plane z, one
    // iteration earlier) is behind that iteration's barrier.
    const int zref_end = min(zb + 1, p.nz - 1);  // last plane an interior pull reads
    if constexpr (kRef)
        for (int q = za; q <= min(za + 2, zref_end); ++q) load_ref(q);

    // prologue: planes za - 1 and za
    if (za == 0) {
        // plane 0 with two rings, for the substrate ghost plane z = -1 built by
        // the fictitious-density rule (Eq. 18) from its five fluid neighbours
        load_plane(0, true, true);
        __syncthreads();
        for (int j = tid; j < HS; j += NTH) {
            const int hx = j % HX, hy = j / HX;
            const int c = (hy + 1) * SX + (hx + 1);
            real n0 = 0, n1 = 0, den = 0;
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                if (D3Q19::c(i, 2) != 1) continue;
                const real w = (real)D3Q19::w(i);
                const int cc = c + D3Q19::c(i, 0) + D3Q19::c(i, 1) * SX;
                n0 += w * sub[cc];
                n1 += w * sub[SS + cc];
                den += w;
            }
            C.put(p, slot_of(-1), j, p.zeta[0] * n0 / den, p.zeta[1] * n1 / den);
        }
        __syncthreads();  // the scratch in buffer 1 is read; plane 1 goes there next
    } else {
        load_plane(za - 1, false, false);
        load_plane(za, true, false);
        if constexpr (kRef) __syncthreads();  // the ink fractions loaded above
    }

    double m0 = 0, m1 = 0, mx = 0, my = 0, mz = 0;
    int bad = 0;
    const int N = (int)p.N;
    for (int z = za; z < zb; ++z) {
        // plane z + 1 goes to colour slot (z + 1) mod 4 and moment buffer
        // (z + 1) & 1: no collision still running (plane z - 1, other threads)
        // reads that slot, and the buffer's previous plane was read by this
        // thread only
        if constexpr (kRef)
            if (z + 3 <= zref_end) load_ref(z + 3);
        if (z + 1 < p.nz - 1) load_interior(z + 1);
        else if (z + 1 == p.nz - 1) load_plane(z + 1, true, false);
        __syncthreads();
        // open top: zero normal gradient, the ghost plane above is the top plane
        const int sup = z + 1 < p.nz ? slot_of(z + 1) : slot_of(z);
        // the own site if it belongs to this kernel (not outside the lattice,
        // not in the nozzle box, whose sites pull from wall nodes here)
        if (in_xy && !(box_xy && z >= p.box.z0 && z < p.box.z1)) {
            SmemNb<real, kUnit, HX, HS> nb{C.col, {slot_of(z - 1), slot_of(z), sup}, hidx};
            SiteOut<real> so;
            const int s = z * (int)p.plane + gys * p.nx + gxs;
            const real* b = pops + (z & 1) * NS * NT + tid;
            Moments<real> M;
            M.rY = b[0];
            M.sd = b[NT];
#pragma unroll
            for (int k = 0; k < 3; ++k) M.m[k] = b[(2 + k) * NT];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                M.PY[k] = b[(5 + k) * NT];
                M.PT[k] = b[(11 + k) * NT];
            }
            collide_out<D3Q19, real, kUnit>(p, M, nb, real(z) + real(0.5), &so,
                                            [&](int i, real fY, real fD, real c) {
                                                pop_put<D3Q19, S>(p, i, s, N, fY, fD, c);
                                            });
            ref_put<S>(p, s, so.cY);
            if (z >= p.nz - 2)
                for (int a = 0; a < 3; ++a) p.u_cur[utop_idx(p, a, xs, ys, z)] = so.u[a];
            if (unstable_site(so.rhoY, so.rhoB)) bad = 1;
            if (p.write_fields) {
                real* F = p.fields;
                F[kFRhoInk * p.N + s] = so.rhoY;
                F[kFRhoAmb * p.N + s] = so.rhoB;
                F[kFUx * p.N + s] = so.u[0];
                F[kFUy * p.N + s] = so.u[1];
                F[kFUz * p.N + s] = so.u[2];
                F[kFNu * p.N + s] = (so.tau - real(0.5)) * real(1.0 / 3.0);
                F[kFP * p.N + s] = p.pfac[0] * so.rhoY + p.pfac[1] * so.rhoB;
                F[kFPhi * p.N + s] = so.rn;
                F[kFSolid * p.N + s] = real(0);
                m0 += (double)so.rhoY;
                m1 += (double)so.rhoB;
                const double rr = (double)so.rhoY + (double)so.rhoB;
                mx += rr * (double)so.u[0];
                my += rr * (double)so.u[1];
                mz += rr * (double)so.u[2];
            }
        }
    }
    warp_add(p.acc + kAccBc, bc[0]);
    warp_add(p.acc + kAccBc + 1, bc[1]);
    if (p.write_fields) {
        warp_add(p.acc + kAccMass, m0);
        warp_add(p.acc + kAccMass + 1, m1);
        warp_add(p.acc + kAccMom, mx);
        warp_add(p.acc + kAccMom + 1, my);
        warp_add(p.acc + kAccMom + 2, mz);
    }
    if (bad) atomicOr(p.flags, 1);
}

template <typename real, typename S, bool kUnit>
constexpr size_t fused_smem() {
    using T = Tile<8, 32>;
    return sizeof(real) * (2 * 17 * T::NT + 4 * Colour<real, kUnit, T::HS>::NV * T::HS +
                           (Stored<S>::kDev ? 4 * T::SS : 0));
}

// Configuration of the single-lattice bulk kernel: one site per thread
// (32 x 8 tiles), three CTAs of 256 threads per SM in FP32 arithmetic (80
// registers), one in FP64.
template <typename real>
constexpr int fused_minb() { return sizeof(real) == 8 ? 1 : 3; }
constexpr int kTileH = 8;  // rows of the batched kernel's tiles (one site per thread)

template <typename real, typename S, bool kUnit>
__global__ void __launch_bounds__(256, fused_minb<real>()) k_fused(StepArgs<real> p, int zchunk) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = z_chunks(p.nz, zchunk);
    fused_column<real, S, kUnit>(p, smraw, blockIdx.x * 32, blockIdx.y * 8, z_chunk_begin(p.nz, n, blockIdx.z),
                                 z_chunk_begin(p.nz, n, blockIdx.z + 1));
}

// Persistent form over many lattices: the CTAs take columns of the work list
// (lattice, x0 | y0 << 16, za, zb) in order from a queue (an atomic counter,
// zero at launch), so CTAs that become resident late, behind other kernels,
// simply take fewer columns. Each lattice's step arguments are copied to
// shared memory when a CTA's column changes lattice.
// the batched kernel keeps one site per thread at three CTAs per SM (FP32),
// leaving room on the SMs for the batched box kernels beside it
template <typename real>
constexpr int batch_minb() { return sizeof(real) == 8 ? 1 : 3; }

template <typename real, typename S, bool kUnit>
__global__ void __launch_bounds__(Tile<kTileH>::NT, batch_minb<real>())
    k_fused_batch(const StepArgs<real>* __restrict__ args, const int4* __restrict__ items, int n_items,
                  int* __restrict__ queue) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(16) StepArgs<real> sp;
    __shared__ int next;
    constexpr int NT = Tile<kTileH>::NT;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    int last = -1;
    for (;;) {
        __syncthreads();  // the previous column's shared state and `next` are free
        if (tid == 0) next = atomicAdd(queue, 1);
        __syncthreads();
        const int w = next;
        if (w >= n_items) break;
        const int4 it = items[w];
        if (it.x != last) {
            const int4* src = reinterpret_cast<const int4*>(args + it.x);
            int4* dst = reinterpret_cast<int4*>(&sp);
            for (int k = tid; k < (int)(sizeof(StepArgs<real>) / 16); k += NT) dst[k] = src[k];
            last = it.x;
            __syncthreads();
        }
        fused_column<real, S, kUnit>(sp, smraw, it.y & 0xffff, it.y >> 16, it.z, it.w);
    }
}

// the kernel's dynamic shared memory limit is set once per device (context)
template <typename K>
void set_smem_once(K kernel, size_t smem, unsigned* configured) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 32 && !(*configured & (1u << dev))) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        *configured |= 1u << dev;
    }
}

template <typename real, typename S, bool kUnit>
int launch_one(const StepArgs<real>& p, int zchunk, cudaStream_t st) {
    constexpr size_t smem = fused_smem<real, S, kUnit>();
    static_assert(smem * fused_minb<real>() <= 227 * 1024, "CTAs per SM");
    static unsigned configured = 0;
    set_smem_once(k_fused<real, S, kUnit>, smem, &configured);
    dim3 block(32, 8);
    dim3 grid((p.nx + 31) / 32, (p.ny + 7) / 8, z_chunks(p.nz, zchunk));
    k_fused<real, S, kUnit><<<grid, block, smem, st>>>(p, zchunk);
    return 1;
}

template <typename real, typename S, bool kUnit>
int launch_batch_one(const StepArgs<real>* args, const int4* items, int n_items, int* queue, int grid,
                     cudaStream_t st, int* occupancy) {
    constexpr size_t smem = fused_smem<real, S, kUnit>();
    static unsigned configured = 0;
    set_smem_once(k_fused_batch<real, S, kUnit>, smem, &configured);
    if (occupancy) {
        *occupancy = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, k_fused_batch<real, S, kUnit>, Tile<kTileH>::NT,
                                                      smem);
        return 0;
    }
    if (n_items <= 0) return 0;
    k_fused_batch<real, S, kUnit><<<grid, dim3(32, kTileH), smem, st>>>(args, items, n_items, queue);
    return 1;
}

}  // namespace

template <typename real, typename S>
int launch_fused(const StepArgs<real>& p, int zchunk, cudaStream_t st) {
    return p.unit ? launch_one<real, S, true>(p, zchunk, st) : launch_one<real, S, false>(p, zchunk, st);
}

template <typename real, typename S>
int launch_fused_batch(const StepArgs<real>* args, const int4* items, int n_items, int* queue, int grid, int unit,
                       cudaStream_t st, int* occupancy) {
    return unit ? launch_batch_one<real, S, true>(args, items, n_items, queue, grid, st, occupancy)
                : launch_batch_one<real, S, false>(args, items, n_items, queue, grid, st, occupancy);
}

}  // namespace cglbm
