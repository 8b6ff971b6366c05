// Fused bulk step: one kernel does streaming, moments, colour gradient, local
// relaxation time, regularised collision, perturbation and recolouring for
// every site outside the nozzle box (D3Q19, substrate below, open top).
//
// Each CTA owns a TX x TY column tile and marches up a chunk of z-planes. The
// colour gradient (Eq. 12) needs the densities of this step at the 18
// neighbours, which other CTAs produce; the CTA therefore recomputes, for the
// plane ahead, the post-streaming densities of its tile plus a one-site halo
// from the populations in HBM (the re-reads hit L2), and keeps three planes
// of colour fractions in shared memory. HBM traffic stays at one read and one
// write of the populations per site update.
#include "lbm_launch.h"

namespace cglbm {

namespace {

// streaming for a site away from the nozzle: every source is fluid except
// across the substrate (resting half-way wall) and the open top
// (anti-bounce-back, Eq. 28)
template <typename real, bool kLedger>
__device__ __forceinline__ void pull_bulk(const StepArgs<real>& p, int x, int y, int z, real f[2][19],
                                          real bc[2]) {
    using VS = D3Q19;
    const long long s = sidx(p, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sz = z - VS::c(i, 2);
        const int ib = opp(i);
        if (sz < 0) {
            f[0][i] = p.fin[(long long)ib * p.N + s];
            f[1][i] = p.fin[(long long)(19 + ib) * p.N + s];
        } else if (sz >= p.nz) {
            real u2[3];
            anti_bb_velocity<VS>(p, x, y, z, i, u2);
            const real cu = (real)VS::c(ib, 0) * u2[0] + (real)VS::c(ib, 1) * u2[1] + (real)VS::c(ib, 2) * u2[2];
            const real uu = u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2];
            const real q = real(4.5) * cu * cu - real(1.5) * uu;
            const real w = (real)VS::w(ib);
            const real oY = p.fin[(long long)ib * p.N + s];
            const real oD = p.fin[(long long)(19 + ib) * p.N + s];
            // imposed densities: ink 0, ambient rho_top
            f[0][i] = -oY;
            f[1][i] = -oD + real(2) * (p.rho_top * p.dphi[1][ib] + w * (p.rho_top - p.rho_ref) + p.rho_top * w * q);
            if (kLedger) {
                bc[0] += f[0][i] - oY;
                bc[1] += (f[1][i] - oD) - (f[0][i] - oY);
            }
        } else {
            const int sx = wrap1(x - VS::c(i, 0), p.nx), sy = wrap1(y - VS::c(i, 1), p.ny);
            const long long src = sidx(p, sx, sy, sz);
            f[0][i] = p.fin[(long long)i * p.N + src];
            f[1][i] = p.fin[(long long)(19 + i) * p.N + src];
        }
    }
}

template <typename real>
__device__ __forceinline__ void pull_bulk_density(const StepArgs<real>& p, int x, int y, int z, real* rY, real* rB) {
    real f[2][19];
    real bc[2];
    pull_bulk<real, false>(p, x, y, z, f, bc);
    real a = 0, b = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) { a += f[0][i]; b += f[1][i]; }
    *rY = a;
    *rB = (p.rho_ref + b) - a;
}

__device__ __forceinline__ void warp_add(double* dst, double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

template <typename real>
__device__ __forceinline__ bool in_box(const StepArgs<real>& p, int x, int y, int z) {
    const Region& b = p.box;
    if (b.wx == 0 || z < b.z0 || z >= b.z1) return false;
    int dx = x - b.x0;
    if (dx < 0) dx += p.nx;
    int dy = y - b.y0;
    if (dy < 0) dy += p.ny;
    return dx < b.wx && dy < b.wy;
}

template <typename real, int TX, int TY>
struct SmemNb {
    const real (*sm)[3][(TX + 2) * (TY + 2)];
    int slot[3];  // slots of planes z-1, z, z+1
    int hidx;     // halo-tile index of the site
    __device__ __forceinline__ void operator()(int i, real* cY, real* cB, real* rn) const {
        const int j = hidx + D3Q19::c(i, 0) + D3Q19::c(i, 1) * (TX + 2);
        const int sl = slot[1 + D3Q19::c(i, 2)];
        *cY = sm[sl][0][j];
        *cB = sm[sl][1][j];
        *rn = sm[sl][2][j];
    }
};

template <typename real, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) k_fused(StepArgs<real> p, int zchunk) {
    constexpr int HX = TX + 2, HY = TY + 2, HS = HX * HY;
    constexpr int SX = TX + 4, SY = TY + 4, SS = SX * SY;
    constexpr int NT = TX * TY;
    __shared__ real sm[3][3][HS];
    __shared__ real sub[2][SS];

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int za = blockIdx.z * zchunk;
    const int zb = min(p.nz, za + zchunk);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x = x0 + tx, y = y0 + ty;
    const bool in_xy = x < p.nx && y < p.ny;

    auto put = [&](int slot, int j, real rY, real rB) {
        const real tot = rY + rB;
        sm[slot][0][j] = rY / tot;
        sm[slot][1][j] = rB / tot;
        sm[slot][2][j] = phase_field(p, rY, rB);
    };
    // densities after streaming of plane zz over the tile and its halo
    auto load_plane = [&](int zz, int slot) {
        if (zz >= p.nz) {  // open top: copy of the top plane
            const int src = (zz - 1 + 3) % 3;
            for (int j = tid; j < HS; j += NT) {
                sm[slot][0][j] = sm[src][0][j];
                sm[slot][1][j] = sm[src][1][j];
                sm[slot][2][j] = sm[src][2][j];
            }
            return;
        }
        for (int j = tid; j < HS; j += NT) {
            const int hx = j % HX, hy = j / HX;
            const int gx = wrapn(x0 - 1 + hx, p.nx), gy = wrapn(y0 - 1 + hy, p.ny);
            real rY, rB;
            pull_bulk_density(p, gx, gy, zz, &rY, &rB);
            put(slot, j, rY, rB);
        }
    };

    // prologue: planes za - 1 and za
    if (za == 0) {
        // plane 0 with two rings, then the substrate ghost plane z = -1 from
        // the fictitious-density rule (Eq. 18) over its five fluid neighbours
        for (int j = tid; j < SS; j += NT) {
            const int sx = j % SX, sy = j / SX;
            const int gx = wrapn(x0 - 2 + sx, p.nx), gy = wrapn(y0 - 2 + sy, p.ny);
            real rY, rB;
            pull_bulk_density(p, gx, gy, 0, &rY, &rB);
            sub[0][j] = rY;
            sub[1][j] = rB;
        }
        __syncthreads();
        for (int j = tid; j < HS; j += NT) {
            const int hx = j % HX, hy = j / HX;
            const int c = (hy + 1) * SX + (hx + 1);
            put(0, j, sub[0][c], sub[1][c]);  // plane 0 -> slot 0
            real n0 = 0, n1 = 0, den = 0;
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                if (D3Q19::c(i, 2) != 1) continue;
                const real w = (real)D3Q19::w(i);
                const int cc = c + D3Q19::c(i, 0) + D3Q19::c(i, 1) * SX;
                n0 += w * sub[0][cc];
                n1 += w * sub[1][cc];
                den += w;
            }
            put(2, j, p.zeta[0] * n0 / den, p.zeta[1] * n1 / den);  // plane -1 -> slot 2
        }
    } else {
        load_plane(za - 1, (za - 1) % 3);
        load_plane(za, za % 3);
    }

    double bc0 = 0, bc1 = 0, m0 = 0, m1 = 0, mx = 0, my = 0, mz = 0;
    int bad = 0;
    const int hidx = (ty + 1) * HX + (tx + 1);

    for (int z = za; z < zb; ++z) {
        __syncthreads();  // plane z-2's slot is free, plane z's writes visible
        load_plane(z + 1, (z + 1) % 3);
        __syncthreads();
        if (in_xy && !in_box(p, x, y, z)) {
            real f[2][19];
            real bc[2] = {real(0), real(0)};
            pull_bulk<real, true>(p, x, y, z, f, bc);
            bc0 += (double)bc[0];
            bc1 += (double)bc[1];
            SmemNb<real, TX, TY> nb{sm, {(z + 2) % 3, z % 3, (z + 1) % 3}, hidx};
            SiteOut<real> so;
            collide<D3Q19>(p, f, nb, real(z) + real(0.5), &so);
            const long long s = sidx(p, x, y, z);
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                p.fout[(long long)i * p.N + s] = f[0][i];
                p.fout[(long long)(19 + i) * p.N + s] = f[1][i];
            }
            if (z >= p.nz - 2)
                for (int a = 0; a < 3; ++a) p.u_cur[utop_idx(p, a, x, y, z)] = so.u[a];
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
    warp_add(p.acc + kAccBc, bc0);
    warp_add(p.acc + kAccBc + 1, bc1);
    if (p.write_fields) {
        warp_add(p.acc + kAccMass, m0);
        warp_add(p.acc + kAccMass + 1, m1);
        warp_add(p.acc + kAccMom, mx);
        warp_add(p.acc + kAccMom + 1, my);
        warp_add(p.acc + kAccMom + 2, mz);
    }
    if (bad) atomicOr(p.flags, 1);
}

}  // namespace

template <typename real>
int launch_fused(const StepArgs<real>& p, int zchunk, cudaStream_t st) {
    constexpr int TX = 32, TY = 8;
    dim3 block(TX, TY);
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.nz + zchunk - 1) / zchunk);
    if (sizeof(real) == 4)
        k_fused<real, TX, TY, 2><<<grid, block, 0, st>>>(p, zchunk);
    else
        k_fused<real, TX, TY, 1><<<grid, block, 0, st>>>(p, zchunk);
    return 1;
}

template int launch_fused<float>(const StepArgs<float>&, int, cudaStream_t);
template int launch_fused<double>(const StepArgs<double>&, int, cudaStream_t);

}  // namespace cglbm
