/*
 * Plain FP64 CPU oracle: two-component regularised colour-gradient lattice
 * Boltzmann step with a shear-thinning ink and a moving print head.
 * Monteferrante, Montessori, Succi, Pisignano, Lauricella (arXiv 2102.02655).
 *
 * TEST INFRASTRUCTURE (see cglbm_oracle.h). Shares nothing with the CUDA path.
 *
 * One time step n (state: post-collision populations f* of step n-1):
 *   1. stream f* on the geometry of step n-1, applying the boundary rules on
 *      every link whose source is not a fluid node (Eq. 1, 26-28);
 *   2. move the nozzle to its step-n position; delete the populations of
 *      nodes that became solid and create nodes that became fluid (Sec. II B);
 *   3. moments rho^k, rho u (Eq. 2-3);
 *   4. fictitious wall densities on solid nodes (Eq. 18);
 *   5. colour field and its isotropic gradient (Eq. 11-12);
 *   6. local relaxation time from the ink rheology (Eq. 17, 23-25);
 *   7. regularised BGK per component (Eq. 5-6, 20) plus the drag/body force
 *      by the exact difference method (Eq. 29);
 *   8. perturbation once on the total (Eq. 10);
 *   9. recolouring (Eq. 14-16), giving f* of step n.
 * Readings of silent or garbled passages are listed where they are used.
 */
#include "cglbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXQ 19
#define CS2 (1.0 / 3.0)
#define CS4 (1.0 / 9.0)

struct or_lattice {
    or_params p;
    or_geom g;
    or_rheo r;
    int have_geom, have_rheo;
    int Q;
    int c[MAXQ][3];
    double w[MAXQ], B[MAXQ], phi[2][MAXQ], cnorm[MAXQ];
    double pfac[2]; /* sum_i phi^k_i c_ix^2: partial pressure factor, Eq. 9 */
    int opp[MAXQ];
    int nx, ny, nz;
    long N;
    double *fstar, *fpost, *rho_prev, *u_prev, *rho_all, *fields;
    unsigned char *fluid_prev, *fluid_now;
    double *plane_acc; /* per-plane partial sums, summed serially (deterministic) */
    long long step;
    int64_t hq[2], vq[2], rin2q, rout2q; /* fixed-point geometry, set with the geometry */
    double bc_flux[2], created[2], destroyed[2];
    double mass[2], mom[3];
};

/* ------------------------------------------------------------------------ */
/* Velocity sets                                                              */
/* ------------------------------------------------------------------------ */

/* D2Q9 (Sec. II A: rest + 8 directions, weights 4/9, 1/9, 1/36) is laid in the
 * x-z plane so that z stays the vertical axis of the print setup. D3Q19 (the
 * standard 3D set, not in the paper) keeps the 18 links with |c|^2 <= 2.
 * The sets are enumerated by brute force over {-1,0,1}^3. */
static int build_velset(int velset, int c[MAXQ][3], double w[MAXQ], double B[MAXQ])
{
    int q = 1;
    c[0][0] = c[0][1] = c[0][2] = 0;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int n2 = cx * cx + cy * cy + cz * cz;
                if (n2 == 0 || n2 > 2) continue;
                if (velset == OR_D2Q9 && cy != 0) continue;
                c[q][0] = cx; c[q][1] = cy; c[q][2] = cz; ++q;
            }
    for (int i = 0; i < q; ++i) {
        int n2 = c[i][0] * c[i][0] + c[i][1] * c[i][1] + c[i][2] * c[i][2];
        if (velset == OR_D2Q9) w[i] = n2 == 0 ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else                   w[i] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    /* B_i of the perturbation operator (Eq. 10). The paper prints the D2Q9
     * values. Both sets here take B_i = w_i (a |c_i|^2 + b) with (a, b) fixed
     * by the two conditions the printed D2Q9 values satisfy: the perturbation
     * conserves mass, sum_i B_i = c_s^2, and its stress is proportional to
     * (n n - I), sum_i B_i c_ix^2 = c_s^2. For D2Q9 this reproduces the printed
     * -4/27, 2/27, 5/108 (checked by a test). */
    double m11 = 0, m12 = 0, m21 = 0, m22 = 0;
    for (int i = 0; i < q; ++i) {
        double n2 = c[i][0] * c[i][0] + c[i][1] * c[i][1] + c[i][2] * c[i][2];
        double cx2 = c[i][0] * c[i][0];
        m11 += w[i] * n2;  m12 += w[i];
        m21 += w[i] * n2 * cx2; m22 += w[i] * cx2;
    }
    double det = m11 * m22 - m12 * m21;
    double a = (CS2 * m22 - m12 * CS2) / det;
    double b = (m11 * CS2 - m21 * CS2) / det;
    for (int i = 0; i < q; ++i) {
        double n2 = c[i][0] * c[i][0] + c[i][1] * c[i][1] + c[i][2] * c[i][2];
        B[i] = w[i] * (a * n2 + b);
    }
    return q;
}

int or_velset(int velset, int* c, double* w, double* B)
{
    int cc[MAXQ][3]; double ww[MAXQ], bb[MAXQ];
    int q = build_velset(velset, cc, ww, bb);
    for (int i = 0; i < q; ++i) {
        if (c) { c[3 * i] = cc[i][0]; c[3 * i + 1] = cc[i][1]; c[3 * i + 2] = cc[i][2]; }
        if (w) w[i] = ww[i];
        if (B) B[i] = bb[i];
    }
    return q;
}

/* phi^k_i (Eq. 7): alpha_k at rest, and the moving weight share of 1 - alpha_k
 * in proportion to w_i. For D2Q9 this is (1-alpha)/5 on axes and (1-alpha)/20
 * on diagonals, as printed; with alpha = w_0 it gives phi_i = w_i. */
double or_phi(int velset, double alpha, int i)
{
    int c[MAXQ][3]; double w[MAXQ], B[MAXQ];
    build_velset(velset, c, w, B);
    if (i == 0) return alpha;
    return (1.0 - alpha) * w[i] / (1.0 - w[0]);
}

/* ------------------------------------------------------------------------ */
/* Geometry: the nozzle template (Sec. II B) in fixed point                   */
/* ------------------------------------------------------------------------ */

/* Reading (the 3D geometry is not in the paper): the nozzle is a vertical
 * annular wall r_inner <= r <= r_inner + wall_thickness around the axis
 * through the head position, for z >= gap, open at the top. Positions are
 * tracked in units of 2^-20 lattice units so that the solid/fluid decision for
 * every node is exact integer arithmetic, independent of rounding. */
#define FX 1048576.0
static int64_t q20(double v) { return (int64_t)llround(v * FX); }

static int64_t min_image(int64_t d, int64_t period)
{
    d %= period;
    if (d < 0) d += period;
    if (2 * d >= period) d -= period;
    return d;
}

/* squared horizontal distance (fixed point^2) from node (x, y) to the axis at step n */
static int64_t axis_d2(const or_lattice* L, int x, int y, long long n)
{
    int64_t hx = L->hq[0] + L->vq[0] * n;
    int64_t hy = L->hq[1] + L->vq[1] * n;
    int64_t dx = min_image((int64_t)x * (int64_t)FX - hx, (int64_t)L->nx * (int64_t)FX);
    int64_t dy = min_image((int64_t)y * (int64_t)FX - hy, (int64_t)L->ny * (int64_t)FX);
    return dx * dx + dy * dy;
}

static int64_t rin2(const or_lattice* L) { return L->rin2q; }
static int64_t rout2(const or_lattice* L) { return L->rout2q; }

static int nozzle_active(const or_lattice* L) { return L->g.nozzle && L->g.z_mode == OR_Z_WALLS; }

/* solid nozzle node at step n (z may be nz for the column above the top) */
static int is_solid(const or_lattice* L, int x, int y, int z, long long n)
{
    if (!nozzle_active(L) || z < L->g.gap) return 0;
    int64_t d2 = axis_d2(L, x, y, n);
    return d2 >= rin2(L) && d2 <= rout2(L);
}

static int inside_nozzle(const or_lattice* L, int x, int y, long long n)
{
    return nozzle_active(L) && axis_d2(L, x, y, n) < rin2(L);
}

/* head velocity as used by the wall rule: the fixed-point step, exactly */
static void head_velocity(const or_lattice* L, double v[3])
{
    v[0] = (double)q20(L->g.head_vel[0]) / FX;
    v[1] = (double)q20(L->g.head_vel[1]) / FX;
    v[2] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Small helpers                                                               */
/* ------------------------------------------------------------------------ */

static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

static long sidx(const or_lattice* L, int x, int y, int z) { return ((long)z * L->ny + y) * L->nx + x; }

/* index into rho_all, which has a ghost plane below (z = -1) and above (z = nz) */
static long ridx(const or_lattice* L, int x, int y, int z) { return ((long)(z + 1) * L->ny + y) * L->nx + x; }

/* neighbour of (x,y,z) along +d*c_i; returns 0 if it leaves the domain in z */
static int step_to(const or_lattice* L, int x, int y, int z, const int* c, int d, int* ox, int* oy, int* oz)
{
    *ox = wrap(x + d * c[0], L->nx);
    *oy = wrap(y + d * c[1], L->ny);
    int zz = z + d * c[2];
    if (L->g.z_mode == OR_Z_PERIODIC) zz = wrap(zz, L->nz);
    else if (zz < 0 || zz >= L->nz) return 0;
    *oz = zz;
    return 1;
}

/* Equilibrium of component k (Eq. 6). The paper prints 2 c_s^2 under the
 * quadratic term (c.u)^2; the anti-bounce-back rule (Eq. 28) and the standard
 * form use 2 c_s^4, which is the reading taken here. */
static double feq(const or_lattice* L, int k, int i, double rho, const double* u)
{
    double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return rho * (L->phi[k][i] + L->w[i] * (cu / CS2 + cu * cu / (2.0 * CS4) - uu / (2.0 * CS2)));
}

/* Wall density by quadratic extrapolation to the half-way point from the
 * values at distances 1/2, 3/2, 5/2 (Sec. II B, "third order interpolation in
 * the direction -c_i"; the stencil is not given: reading = the three-point
 * Lagrange extrapolation). */
double or_wall_interp(double r0, double r1, double r2)
{
    return (15.0 * r0 - 10.0 * r1 + 3.0 * r2) / 8.0;
}

/* ------------------------------------------------------------------------ */
/* Rheology: Eq. 23-25 and the implicit shear-rate equation (Eq. 24)          */
/* ------------------------------------------------------------------------ */

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* kinematic ink viscosity from the constitutive law at shear rate gdot */
static double nu_law(const or_rheo* r, double gdot)
{
    switch (r->law) {
    case OR_LAW_CROSS:
        return r->nu_inf + (r->nu0 - r->nu_inf) / (1.0 + pow(r->lambda * gdot, r->n));
    case OR_LAW_POWER:
        if (gdot <= 0.0) return r->n < 1.0 ? INFINITY : (r->n > 1.0 ? 0.0 : r->K);
        return r->K * pow(gdot, r->n - 1.0);
    default:
        return r->nu0;
    }
}

/* tau_Y(gdot) = 1/2 + nu(gdot)/c_s^2 (Eq. 25), clamped to [tau_min, tau_max] */
static double tau_law(const or_rheo* r, double gdot)
{
    double nu = nu_law(r, gdot);
    double t = isinf(nu) ? r->tau_max : 0.5 + nu / CS2;
    return clampd(t, r->tau_min, r->tau_max);
}

/* Root of gdot = S / (rho_Y tau_Y(gdot) c_s^2) (Eq. 24 with Eq. 25).
 * The paper solves it "iteratively until converged below a threshold" and
 * gives neither method nor threshold. The oracle takes the plain definition,
 * the root itself: h(g) = g tau_Y(g) - S/(rho_Y c_s^2) is continuous and
 * increasing (tau_Y is clamped), negative at S/(rho_Y c_s^2 tau_max) and
 * positive at S/(rho_Y c_s^2 tau_min), so bisection on that bracket until the
 * bracket stops shrinking finds it. Returns tau_Y; gdot_out gets the root. */
double or_solve_tau_ink(const or_rheo* r, double S, double rho_ink, double* gdot_out)
{
    if (r->law == OR_LAW_NEWTONIAN) {
        if (gdot_out) *gdot_out = 0.0;
        return tau_law(r, 0.0);
    }
    if (!(S > 0.0) || !(rho_ink > 0.0)) {
        if (gdot_out) *gdot_out = 0.0;
        return tau_law(r, 0.0);
    }
    double s = S / (rho_ink * CS2);
    double lo = s / r->tau_max, hi = s / r->tau_min;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double h = mid * tau_law(r, mid) - s;
        if (h < 0.0) lo = mid; else hi = mid;
    }
    double g = 0.5 * (lo + hi);
    if (gdot_out) *gdot_out = g;
    return tau_law(r, g);
}

/* ------------------------------------------------------------------------ */
/* Collision at one fluid site                                                 */
/* ------------------------------------------------------------------------ */

/* fin[k*Q+i]: populations after streaming. nbr[k*Q+i]: density of component k
 * at x + c_i (fluid density, fictitious wall density or ghost value).
 * z_wall_dist: distance to the substrate wall (drag zone test), < 0 if none.
 * out[k*Q+i]: post-collision populations. aux: tau, |grad rhoN|, physical u. */
static void collide_site(const or_lattice* L, const double* fin, const double* nbr,
                         double z_wall_dist, double* out, double* aux)
{
    const int Q = L->Q;
    const double rY0 = L->p.rho0_ink, rB0 = L->p.rho0_amb;

    /* moments (Eq. 2-3) */
    double rho_k[2] = {0, 0}, mom[3] = {0, 0, 0};
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < Q; ++i) {
            double f = fin[k * Q + i];
            rho_k[k] += f;
            for (int a = 0; a < 3; ++a) mom[a] += f * L->c[i][a];
        }
    double rho = rho_k[0] + rho_k[1];
    double u[3] = {mom[0] / rho, mom[1] / rho, mom[2] / rho};
    double phY = rho_k[0] / rho, phB = rho_k[1] / rho;

    /* colour-gradient force (Eq. 11) with the isotropic gradient (Eq. 12),
     * and the gradient of the phase field rho^N. rho^N is used by the paper but
     * never defined; reading: the usual colour-gradient phase field
     * (a_Y - a_B)/(a_Y + a_B), a_k = rho_k/rho_k0.
     * Eq. 12 is evaluated as (1/c_s^2) sum_i w_i [chi(x + c_i) - chi(x)] c_i,
     * equal to the printed form because sum_i w_i c_i = 0, and exactly zero on
     * a uniform field (the printed form leaves rounding noise there).
     * The phase-field difference rho^N(x + c_i) - rho^N(x) is written as one
     * fraction, 2 (a_Y,i a_B,0 - a_B,i a_Y,0) / ((a_Y,i + a_B,i)(a_Y,0 + a_B,0)),
     * an exact rewriting that keeps its relative precision where the ink
     * density is tiny: there rho^N = -1 + O(rho_Y) would lose every digit of
     * the difference, and the direction of Eq. 16 is read from it. */
    double gY[3] = {0, 0, 0}, gB[3] = {0, 0, 0}, gN[3] = {0, 0, 0};
    const double cY0 = phY, cB0 = phB;
    const double aY0 = rho_k[0] / rY0, aB0 = rho_k[1] / rB0;
    const double rn0 = (aY0 - aB0) / (aY0 + aB0);
    for (int i = 1; i < Q; ++i) {
        double nY = nbr[i], nB = nbr[Q + i];
        double tot = nY + nB;
        double cY = nY / tot, cB = nB / tot;
        double aY = nY / rY0, aB = nB / rB0;
        double drn = 2.0 * (aY * aB0 - aB * aY0) / ((aY + aB) * (aY0 + aB0));
        for (int a = 0; a < 3; ++a) {
            gY[a] += L->w[i] * (cY - cY0) * L->c[i][a] / CS2;
            gB[a] += L->w[i] * (cB - cB0) * L->c[i][a] / CS2;
            gN[a] += L->w[i] * drn * L->c[i][a] / CS2;
        }
    }
    double F[3];
    for (int a = 0; a < 3; ++a) F[a] = phB * gY[a] - phY * gB[a];
    double Fn2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    double gNn = sqrt(gN[0] * gN[0] + gN[1] * gN[1] + gN[2] * gN[2]);

    /* equilibria and non-equilibrium stress of each component (Eq. 6, 20) */
    double fe[2][MAXQ], Pi[2][3][3];
    for (int k = 0; k < 2; ++k) {
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Pi[k][a][b] = 0.0;
        for (int i = 0; i < Q; ++i) {
            fe[k][i] = feq(L, k, i, rho_k[k], u);
            double d = fin[k * Q + i] - fe[k][i];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Pi[k][a][b] += d * L->c[i][a] * L->c[i][b];
        }
    }

    /* local relaxation time (Eq. 17, 24-25): ink viscosity from the implicit
     * shear-rate equation with the ink's own stress |Pi^Y|, ambient viscosity
     * from tau_amb, mixed harmonically by mass fraction, then clamped. */
    double S = 0.0;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) S += Pi[0][a][b] * Pi[0][a][b];
    S = sqrt(S);
    double tauY;
    if (rho_k[0] > 1e-12 * rho) tauY = or_solve_tau_ink(&L->r, S, rho_k[0], NULL);
    else                        tauY = tau_law(&L->r, 0.0);
    double nuY = CS2 * (tauY - 0.5);
    double nuB = CS2 * (L->p.tau_amb - 0.5);
    double inv_nu = phY / nuY + phB / nuB;
    double tau = clampd(0.5 + (1.0 / inv_nu) / CS2, L->r.tau_min, L->r.tau_max);

    /* body force and drag (Eq. 29) by the exact difference method: each
     * component gets f^eq(rho_k, u + F/rho) - f^eq(rho_k, u). Reading: the
     * drag uses the pre-force velocity u, and acts within drag_height of the
     * substrate wall. */
    double Fb[3];
    for (int a = 0; a < 3; ++a) Fb[a] = rho * L->p.g[a];
    if (L->p.drag_gamma != 0.0 && z_wall_dist >= 0.0 && z_wall_dist < L->p.drag_height)
        for (int a = 0; a < 3; ++a) Fb[a] += -L->p.drag_gamma * rho_k[0] * u[a];
    int forced = (Fb[0] != 0.0 || Fb[1] != 0.0 || Fb[2] != 0.0);
    double u2[3] = {u[0] + Fb[0] / rho, u[1] + Fb[1] / rho, u[2] + Fb[2] / rho};

    /* regularised BGK per component (Eq. 5 with Eq. 20):
     * f^reg = f^eq + w_i/(2 c_s^4) Q_i:Pi^neq, then f^reg - (f^reg - f^eq)/tau */
    double fs[MAXQ];
    for (int i = 0; i < Q; ++i) fs[i] = 0.0;
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < Q; ++i) {
            double qp = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    qp += (L->c[i][a] * L->c[i][b] - (a == b ? CS2 : 0.0)) * Pi[k][a][b];
            double freg = fe[k][i] + L->w[i] / (2.0 * CS4) * qp;
            double v = freg - (freg - fe[k][i]) / tau;
            if (forced) v += feq(L, k, i, rho_k[k], u2) - fe[k][i];
            fs[i] += v;
        }

    /* perturbation operator (Eq. 10), applied once to the total. Reading: the
     * paper's per-component superscript k notwithstanding, applying it once
     * is what gives sigma = 2 tau A / 9 (Eq. 13), which a test checks. */
    if (gNn > 0.0 && Fn2 > 0.0)
        for (int i = 0; i < Q; ++i) {
            double Fc = F[0] * L->c[i][0] + F[1] * L->c[i][1] + F[2] * L->c[i][2];
            fs[i] += 0.5 * L->p.A * gNn * (L->w[i] * Fc * Fc / Fn2 - L->B[i]);
        }

    /* recolouring (Eq. 14-16). Both lines use the zero-velocity equilibria
     * sum_k rho_k phi^k_i (Eq. 15 prints u; reading: u = 0 as in Eq. 14).
     * cos(phi_i) is Eq. 16 as printed. It is undefined where grad rho^N = 0;
     * a computed gradient at or below the rounding level of the arithmetic
     * (grad_floor) has no meaningful direction either, so there, and only
     * there, cos(phi_i) = 0. */
    const int has_dir = gNn > L->p.grad_floor;
    for (int i = 0; i < Q; ++i) {
        double cosp = 0.0;
        if (i != 0 && has_dir)
            cosp = (L->c[i][0] * gN[0] + L->c[i][1] * gN[1] + L->c[i][2] * gN[2]) / (L->cnorm[i] * gNn);
        double e0 = rho_k[0] * L->phi[0][i] + rho_k[1] * L->phi[1][i];
        double g = L->p.beta * rho_k[0] * rho_k[1] / (rho * rho) * cosp * e0;
        out[i] = phY * fs[i] + g;
        out[Q + i] = phB * fs[i] - g;
    }

    if (aux) {
        aux[0] = tau;
        aux[1] = gNn;
        for (int a = 0; a < 3; ++a) aux[2 + a] = u[a] + Fb[a] / (2.0 * rho);
    }
}

void or_collide_one(const or_lattice* L, const double* fin, const double* nbr,
                    double z_wall_dist, double* out, double* aux)
{
    collide_site(L, fin, nbr, z_wall_dist, out, aux);
}

/* ------------------------------------------------------------------------ */
/* Lattice                                                                     */
/* ------------------------------------------------------------------------ */

or_lattice* or_create(const or_params* p)
{
    if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->velset == OR_D2Q9 && p->ny != 1) return NULL;
    or_lattice* L = (or_lattice*)calloc(1, sizeof(or_lattice));
    if (!L) return NULL;
    L->p = *p;
    if (!(L->p.grad_floor > 0.0)) L->p.grad_floor = 0x1p-45;
    L->nx = p->nx; L->ny = p->ny; L->nz = p->nz;
    L->N = (long)p->nx * p->ny * p->nz;
    L->Q = build_velset(p->velset, L->c, L->w, L->B);
    for (int i = 0; i < L->Q; ++i) {
        for (int j = 0; j < L->Q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2]) L->opp[i] = j;
        L->cnorm[i] = sqrt((double)(L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] + L->c[i][2] * L->c[i][2]));
    }
    double alpha[2] = {p->alpha_ink, p->alpha_amb};
    for (int k = 0; k < 2; ++k) {
        L->pfac[k] = 0.0;
        for (int i = 0; i < L->Q; ++i) {
            L->phi[k][i] = i == 0 ? alpha[k] : (1.0 - alpha[k]) * L->w[i] / (1.0 - L->w[0]);
            L->pfac[k] += L->phi[k][i] * L->c[i][0] * L->c[i][0];
        }
    }
    long N = L->N, Q = L->Q;
    long NR = (long)(p->nz + 2) * p->nx * p->ny;
    L->fstar = (double*)calloc(2 * Q * N, sizeof(double));
    L->fpost = (double*)calloc(2 * Q * N, sizeof(double));
    L->rho_prev = (double*)calloc(2 * N, sizeof(double));
    L->u_prev = (double*)calloc(3 * N, sizeof(double));
    L->rho_all = (double*)calloc(2 * NR, sizeof(double));
    L->fields = (double*)calloc((long)OR_NFIELDS * N, sizeof(double));
    L->fluid_prev = (unsigned char*)calloc(N, 1);
    L->fluid_now = (unsigned char*)calloc(N, 1);
    L->plane_acc = (double*)calloc((long)p->nz * 16, sizeof(double));
    if (!L->fstar || !L->fpost || !L->rho_prev || !L->u_prev || !L->rho_all || !L->fields ||
        !L->fluid_prev || !L->fluid_now || !L->plane_acc) {
        or_destroy(L);
        return NULL;
    }
    return L;
}

void or_destroy(or_lattice* L)
{
    if (!L) return;
    free(L->fstar); free(L->fpost); free(L->rho_prev); free(L->u_prev);
    free(L->rho_all); free(L->fields); free(L->fluid_prev); free(L->fluid_now); free(L->plane_acc);
    free(L);
}

int or_set_rheology(or_lattice* L, const or_rheo* r)
{
    if (!L || !r) return 1;
    if (!(r->tau_min > 0.5) || !(r->tau_max >= r->tau_min)) return 1;
    L->r = *r;
    L->have_rheo = 1;
    return 0;
}

static void mark_fluid(or_lattice* L, unsigned char* fl, long long n)
{
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) fl[sidx(L, x, y, z)] = !is_solid(L, x, y, z, n);
}

/* macroscopic output at one site from given densities and velocity */
static void write_fields(or_lattice* L, long s, double rY, double rB, const double* u, double tau, double solid)
{
    long N = L->N;
    double aY = rY / L->p.rho0_ink, aB = rB / L->p.rho0_amb;
    L->fields[OR_F_RHO_INK * N + s] = rY;
    L->fields[OR_F_RHO_AMB * N + s] = rB;
    L->fields[OR_F_UX * N + s] = u[0];
    L->fields[OR_F_UY * N + s] = u[1];
    L->fields[OR_F_UZ * N + s] = u[2];
    L->fields[OR_F_NU * N + s] = tau > 0.0 ? CS2 * (tau - 0.5) : 0.0;
    L->fields[OR_F_P * N + s] = L->pfac[0] * rY + L->pfac[1] * rB;
    L->fields[OR_F_RHON * N + s] = (aY + aB) > 0.0 ? (aY - aB) / (aY + aB) : 0.0;
    L->fields[OR_F_SOLID * N + s] = solid;
}

static void init_state(or_lattice* L, const double* rY, const double* rB, const double* u)
{
    const int Q = L->Q;
    long N = L->N;
    mark_fluid(L, L->fluid_now, L->step);
    memset(L->fields, 0, sizeof(double) * OR_NFIELDS * N);
    L->mass[0] = L->mass[1] = 0.0;
    L->mom[0] = L->mom[1] = L->mom[2] = 0.0;
    for (long s = 0; s < N; ++s) {
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < Q; ++i) L->fstar[(k * Q + i) * N + s] = 0.0;
        if (!L->fluid_now[s]) {
            L->rho_prev[s] = L->rho_prev[N + s] = 0.0;
            L->u_prev[s] = L->u_prev[N + s] = L->u_prev[2 * N + s] = 0.0;
            double zero[3] = {0, 0, 0};
            write_fields(L, s, 0.0, 0.0, zero, 0.0, 1.0);
            L->fields[OR_F_RHON * N + s] = 0.0;
            continue;
        }
        double uu[3] = {u ? u[3 * s] : 0.0, u ? u[3 * s + 1] : 0.0, u ? u[3 * s + 2] : 0.0};
        double rk[2] = {rY[s], rB[s]};
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < Q; ++i) L->fstar[(k * Q + i) * N + s] = feq(L, k, i, rk[k], uu);
        L->rho_prev[s] = rk[0];
        L->rho_prev[N + s] = rk[1];
        for (int a = 0; a < 3; ++a) L->u_prev[a * N + s] = uu[a];
        write_fields(L, s, rk[0], rk[1], uu, 0.0, 0.0);
    }
    for (long s = 0; s < N; ++s) {
        if (!L->fluid_now[s]) continue;
        double rr = L->rho_prev[s] + L->rho_prev[N + s];
        L->mass[0] += L->rho_prev[s];
        L->mass[1] += L->rho_prev[N + s];
        for (int a = 0; a < 3; ++a) L->mom[a] += rr * L->u_prev[a * N + s];
    }
    L->bc_flux[0] = L->bc_flux[1] = 0.0;
    L->created[0] = L->created[1] = 0.0;
    L->destroyed[0] = L->destroyed[1] = 0.0;
}

/* Initial state (Sec. III): the nozzle filled with ink, ambient elsewhere, at
 * rest, populations at equilibrium. */
int or_set_geometry(or_lattice* L, const or_geom* g)
{
    if (!L || !g) return 1;
    if (g->nozzle && g->z_mode != OR_Z_WALLS) return 1;
    if (g->nozzle && (g->gap < 1 || g->gap >= L->nz || !(g->r_inner > 0.0) || !(g->wall_thickness > 0.0))) return 1;
    /* the fixed-point distances below are squared in 64 bits: exact for
     * lattice sides up to 4000 and radii up to 2000 */
    if (g->nozzle && (L->nx > 4000 || L->ny > 4000 || !(g->r_inner + g->wall_thickness <= 2000.0))) return 1;
    L->g = *g;
    L->have_geom = 1;
    L->step = 0;
    for (int a = 0; a < 2; ++a) { L->hq[a] = q20(g->head_pos[a]); L->vq[a] = q20(g->head_vel[a]); }
    {
        int64_t ri = q20(g->r_inner), ro = q20(g->r_inner + g->wall_thickness);
        L->rin2q = ri * ri;
        L->rout2q = ro * ro;
    }
    long N = L->N;
    double* rY = (double*)calloc(N, sizeof(double));
    double* rB = (double*)calloc(N, sizeof(double));
    if (!rY || !rB) { free(rY); free(rB); return 2; }
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                long s = sidx(L, x, y, z);
                int ink = nozzle_active(L) && z >= g->gap && inside_nozzle(L, x, y, 0);
                rY[s] = ink ? L->p.rho0_ink : 0.0;
                rB[s] = ink ? 0.0 : L->p.rho0_amb;
            }
    init_state(L, rY, rB, NULL);
    free(rY); free(rB);
    return 0;
}

int or_set_fields(or_lattice* L, const double* rho_ink, const double* rho_amb, const double* u)
{
    if (!L || !L->have_geom || !rho_ink || !rho_amb) return 1;
    init_state(L, rho_ink, rho_amb, u);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Streaming with the boundary rules (Eq. 1, 26-28)                           */
/* ------------------------------------------------------------------------ */

enum { LINK_FLUID = 0, LINK_REST_WALL, LINK_MOVING_WALL, LINK_OPEN };

/* Classify the source x - c_i of the population pulled into (x,y,z) along i,
 * on the geometry of step n-1. For moving walls uw gets the wall velocity. */
static int classify_source(const or_lattice* L, int x, int y, int z, int i, long long nprev, double* uw, long* src)
{
    int sx, sy, sz;
    const int* c = L->c[i];
    sx = wrap(x - c[0], L->nx);
    sy = wrap(y - c[1], L->ny);
    sz = z - c[2];
    uw[0] = uw[1] = uw[2] = 0.0;
    if (L->g.z_mode == OR_Z_PERIODIC) {
        *src = sidx(L, sx, sy, wrap(sz, L->nz));
        return LINK_FLUID;
    }
    if (sz < 0) return LINK_REST_WALL; /* substrate: no-slip wall half-way below z = 0 */
    if (sz >= L->nz) {
        if (L->g.top_mode == OR_TOP_WALL) {
            for (int a = 0; a < 3; ++a) uw[a] = L->g.top_vel[a];
            return LINK_MOVING_WALL;
        }
        if (nozzle_active(L)) {
            int64_t d2 = axis_d2(L, sx, sy, nprev);
            if (d2 >= rin2(L) && d2 <= rout2(L)) { head_velocity(L, uw); return LINK_MOVING_WALL; }
            if (d2 < rin2(L)) {
                /* inlet (Eq. 27): u_Inlet = u_ink + v_nozzle, with u_ink along -z */
                head_velocity(L, uw);
                uw[2] -= L->g.u_ink;
                return LINK_MOVING_WALL;
            }
        }
        return LINK_OPEN;
    }
    *src = sidx(L, sx, sy, sz);
    if (!L->fluid_prev[*src]) { head_velocity(L, uw); return LINK_MOVING_WALL; } /* nozzle wall at step n-1 */
    return LINK_FLUID;
}

/* populations after streaming at fluid node (x,y,z) of step n-1; adds the
 * boundary-link mass changes to acc[0..1] */
static void pull_site(or_lattice* L, int x, int y, int z, long long nprev, double* fo, double* acc)
{
    const int Q = L->Q;
    long N = L->N, s = sidx(L, x, y, z);
    for (int i = 0; i < Q; ++i) {
        double uw[3]; long src = -1;
        int kind = classify_source(L, x, y, z, i, nprev, uw, &src);
        int ib = L->opp[i];
        for (int k = 0; k < 2; ++k) {
            double out_own = L->fstar[(k * Q + ib) * N + s]; /* f*_ib(x) heading to the boundary */
            double v;
            if (kind == LINK_FLUID) {
                fo[k * Q + i] = L->fstar[(k * Q + i) * N + src];
                continue;
            } else if (kind == LINK_REST_WALL) {
                v = out_own;
            } else if (kind == LINK_MOVING_WALL) {
                /* Eq. 26: f_i(x) = f*_ib(x) - 2 w rho_w (u_w . c_ib)/c_s^2 with the
                 * wall density extrapolated along +c_i into the fluid */
                double r0 = L->rho_prev[k * N + s], rw = r0;
                int x1, y1, z1, x2, y2, z2;
                if (step_to(L, x, y, z, L->c[i], 1, &x1, &y1, &z1) && step_to(L, x, y, z, L->c[i], 2, &x2, &y2, &z2)) {
                    long s1 = sidx(L, x1, y1, z1), s2 = sidx(L, x2, y2, z2);
                    if (L->fluid_prev[s1] && L->fluid_prev[s2])
                        rw = or_wall_interp(r0, L->rho_prev[k * N + s1], L->rho_prev[k * N + s2]);
                }
                double ucb = -(uw[0] * L->c[i][0] + uw[1] * L->c[i][1] + uw[2] * L->c[i][2]);
                v = out_own - 2.0 * L->w[ib] * rw * ucb / CS2;
            } else {
                /* anti-bounce-back (Eq. 28) with the imposed densities (ink 0,
                 * ambient rho_top_amb) and the half-way velocity from a
                 * second-order extrapolation 1.5 u(x) - 0.5 u(x + c_i) */
                double u0[3], uw2[3];
                for (int a = 0; a < 3; ++a) u0[a] = L->u_prev[a * N + s];
                for (int a = 0; a < 3; ++a) uw2[a] = u0[a];
                int x1, y1, z1;
                if (step_to(L, x, y, z, L->c[i], 1, &x1, &y1, &z1)) {
                    long s1 = sidx(L, x1, y1, z1);
                    if (L->fluid_prev[s1])
                        for (int a = 0; a < 3; ++a) uw2[a] = 1.5 * u0[a] - 0.5 * L->u_prev[a * N + s1];
                }
                double rw = k == 0 ? 0.0 : L->g.rho_top_amb;
                double cu = uw2[0] * L->c[ib][0] + uw2[1] * L->c[ib][1] + uw2[2] * L->c[ib][2];
                double uu = uw2[0] * uw2[0] + uw2[1] * uw2[1] + uw2[2] * uw2[2];
                v = -out_own + 2.0 * rw * (L->phi[k][ib] + L->w[ib] * (cu * cu / (2.0 * CS4) - uu / (2.0 * CS2)));
            }
            fo[k * Q + i] = v;
            acc[k] += v - out_own;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One step                                                                    */
/* ------------------------------------------------------------------------ */

static void one_step(or_lattice* L)
{
    const int Q = L->Q, nx = L->nx, ny = L->ny, nz = L->nz;
    const long N = L->N;
    const long long nprev = L->step, ncur = L->step + 1;
    double* acc = L->plane_acc; /* per plane: [0..1] bc, [2..3] destroyed, [4..5] created, [6..7] mass, [8..10] mom */
    memset(acc, 0, sizeof(double) * 16 * nz);

    /* geometry of step n-1 and step n */
    mark_fluid(L, L->fluid_prev, nprev);
    mark_fluid(L, L->fluid_now, ncur);

    /* 1. stream on the geometry of step n-1 */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        double fo[2 * MAXQ];
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long s = sidx(L, x, y, z);
                if (!L->fluid_prev[s]) continue;
                pull_site(L, x, y, z, nprev, fo, acc + 16 * z);
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < Q; ++i) L->fpost[(k * Q + i) * N + s] = fo[k * Q + i];
            }
    }

    /* 2-3. moments after streaming; destroy nodes that became solid (their
     * populations are deleted, Sec. II B) */
    double* rho_cur = L->rho_all; /* with ghost planes */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long s = sidx(L, x, y, z), r = ridx(L, x, y, z);
                long NR = (long)(nz + 2) * nx * ny;
                rho_cur[r] = rho_cur[NR + r] = 0.0;
                if (!L->fluid_prev[s]) continue;
                double rk[2] = {0, 0};
                for (int k = 0; k < 2; ++k)
                    for (int i = 0; i < Q; ++i) rk[k] += L->fpost[(k * Q + i) * N + s];
                rho_cur[r] = rk[0];
                rho_cur[NR + r] = rk[1];
                if (!L->fluid_now[s]) {
                    acc[16 * z + 2] += rk[0];
                    acc[16 * z + 3] += rk[1];
                }
            }

    /* created nodes: equilibrium at the nozzle velocity with the mean density
     * of the neighbouring fluid nodes (Sec. II B). Reading: neighbours are the
     * Q-1 lattice neighbours that were fluid at both steps; their densities
     * are the ones after this step's streaming. */
    {
        double vn[3];
        head_velocity(L, vn);
        long NR = (long)(nz + 2) * nx * ny;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    long s = sidx(L, x, y, z);
                    if (!(L->fluid_now[s] && !L->fluid_prev[s])) continue;
                    double sum[2] = {0, 0};
                    int cnt = 0;
                    for (int i = 1; i < Q; ++i) {
                        int x1, y1, z1;
                        if (!step_to(L, x, y, z, L->c[i], 1, &x1, &y1, &z1)) continue;
                        long s1 = sidx(L, x1, y1, z1);
                        if (!(L->fluid_prev[s1] && L->fluid_now[s1])) continue;
                        long r1 = ridx(L, x1, y1, z1);
                        sum[0] += rho_cur[r1];
                        sum[1] += rho_cur[NR + r1];
                        ++cnt;
                    }
                    double rb[2];
                    if (cnt > 0) { rb[0] = sum[0] / cnt; rb[1] = sum[1] / cnt; }
                    else { rb[0] = 0.0; rb[1] = L->p.rho0_amb; }
                    for (int k = 0; k < 2; ++k)
                        for (int i = 0; i < Q; ++i) L->fpost[(k * Q + i) * N + s] = feq(L, k, i, rb[k], vn);
                    acc[16 * z + 4] += rb[0];
                    acc[16 * z + 5] += rb[1];
                }
        /* their densities, written after all means are taken */
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    long s = sidx(L, x, y, z);
                    if (!(L->fluid_now[s] && !L->fluid_prev[s])) continue;
                    double rk[2] = {0, 0};
                    for (int k = 0; k < 2; ++k)
                        for (int i = 0; i < Q; ++i) rk[k] += L->fpost[(k * Q + i) * N + s];
                    long r = ridx(L, x, y, z);
                    rho_cur[r] = rk[0];
                    rho_cur[NR + r] = rk[1];
                }
    }

    /* 4. fictitious wall densities (Eq. 18): on every solid node (nozzle,
     * substrate plane z = -1, lid plane z = nz) the zeta-scaled, w-weighted mean
     * of the fluid neighbours. The paper prints the switch s outside the sum;
     * reading: s weights each term inside both sums. At the open top the ghost
     * plane z = nz copies z = nz-1 (zero normal gradient; not in the paper). */
    {
        long NR = (long)(nz + 2) * nx * ny;
        double zeta[2] = {L->p.zeta_ink, L->p.zeta_amb};
        int zlo = L->g.z_mode == OR_Z_WALLS ? -1 : 0;
        int zhi = L->g.z_mode == OR_Z_WALLS ? nz : nz - 1;
        for (int z = zlo; z <= zhi; ++z) {
            if (z == nz && L->g.top_mode == OR_TOP_OPEN) continue;
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int solid = (z < 0 || z >= nz) ? 1 : !L->fluid_now[sidx(L, x, y, z)];
                    if (!solid) continue;
                    double num[2] = {0, 0}, den = 0.0;
                    for (int i = 1; i < Q; ++i) {
                        int x1 = wrap(x + L->c[i][0], nx), y1 = wrap(y + L->c[i][1], ny), z1 = z + L->c[i][2];
                        if (L->g.z_mode == OR_Z_PERIODIC) z1 = wrap(z1, nz);
                        else if (z1 < 0 || z1 >= nz) continue;
                        if (!L->fluid_now[sidx(L, x1, y1, z1)]) continue;
                        long r1 = ridx(L, x1, y1, z1);
                        num[0] += L->w[i] * rho_cur[r1];
                        num[1] += L->w[i] * rho_cur[NR + r1];
                        den += L->w[i];
                    }
                    long r = ridx(L, x, y, z);
                    rho_cur[r] = den > 0.0 ? zeta[0] * num[0] / den : 0.0;
                    rho_cur[NR + r] = den > 0.0 ? zeta[1] * num[1] / den : 0.0;
                }
        }
        if (L->g.z_mode == OR_Z_WALLS && L->g.top_mode == OR_TOP_OPEN)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    rho_cur[ridx(L, x, y, nz)] = rho_cur[ridx(L, x, y, nz - 1)];
                    rho_cur[NR + ridx(L, x, y, nz)] = rho_cur[NR + ridx(L, x, y, nz - 1)];
                }
    }

    /* 5-9. collision at every fluid node of step n */
    {
        long NR = (long)(nz + 2) * nx * ny;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z) {
            double fin[2 * MAXQ], nbr[2 * MAXQ], out[2 * MAXQ], aux[5];
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    long s = sidx(L, x, y, z);
                    if (!L->fluid_now[s]) {
                        for (int k = 0; k < 2; ++k)
                            for (int i = 0; i < Q; ++i) L->fstar[(k * Q + i) * N + s] = 0.0;
                        double zero[3] = {0, 0, 0};
                        write_fields(L, s, 0.0, 0.0, zero, 0.0, 1.0);
                        L->fields[OR_F_RHON * N + s] = 0.0;
                        continue;
                    }
                    for (int k = 0; k < 2; ++k)
                        for (int i = 0; i < Q; ++i) fin[k * Q + i] = L->fpost[(k * Q + i) * N + s];
                    for (int i = 0; i < Q; ++i) {
                        int x1 = wrap(x + L->c[i][0], nx), y1 = wrap(y + L->c[i][1], ny), z1 = z + L->c[i][2];
                        if (L->g.z_mode == OR_Z_PERIODIC) z1 = wrap(z1, nz);
                        long r1 = ridx(L, x1, y1, z1);
                        nbr[i] = rho_cur[r1];
                        nbr[Q + i] = rho_cur[NR + r1];
                    }
                    double zd = L->g.z_mode == OR_Z_WALLS ? z + 0.5 : -1.0;
                    collide_site(L, fin, nbr, zd, out, aux);
                    for (int k = 0; k < 2; ++k)
                        for (int i = 0; i < Q; ++i) L->fstar[(k * Q + i) * N + s] = out[k * Q + i];
                    long r = ridx(L, x, y, z);
                    double rY = rho_cur[r], rB = rho_cur[NR + r];
                    write_fields(L, s, rY, rB, aux + 2, aux[0], 0.0);
                    L->rho_prev[s] = rY;
                    L->rho_prev[N + s] = rB;
                    for (int a = 0; a < 3; ++a) L->u_prev[a * N + s] = aux[2 + a];
                    double* a = acc + 16 * z;
                    a[6] += rY;
                    a[7] += rB;
                    for (int d = 0; d < 3; ++d) a[8 + d] += (rY + rB) * aux[2 + d];
                }
        }
    }

    L->mass[0] = L->mass[1] = 0.0;
    L->mom[0] = L->mom[1] = L->mom[2] = 0.0;
    for (int z = 0; z < nz; ++z) {
        const double* a = acc + 16 * z;
        for (int k = 0; k < 2; ++k) {
            L->bc_flux[k] += a[k];
            L->destroyed[k] += a[2 + k];
            L->created[k] += a[4 + k];
            L->mass[k] += a[6 + k];
        }
        for (int d = 0; d < 3; ++d) L->mom[d] += a[8 + d];
    }
    L->step = ncur;
}

int or_step(or_lattice* L, int nsteps)
{
    if (!L || !L->have_geom || !L->have_rheo || nsteps < 0) return 1;
    for (int t = 0; t < nsteps; ++t) one_step(L);
    return 0;
}

void or_fields(const or_lattice* L, double* out)
{
    memcpy(out, L->fields, sizeof(double) * OR_NFIELDS * L->N);
}

void or_get_diag(const or_lattice* L, or_diag* d)
{
    for (int k = 0; k < 2; ++k) {
        d->mass[k] = L->mass[k];
        d->bc_flux[k] = L->bc_flux[k];
        d->created[k] = L->created[k];
        d->destroyed[k] = L->destroyed[k];
    }
    for (int a = 0; a < 3; ++a) d->momentum[a] = L->mom[a];
    d->step = L->step;
}

int or_get_populations(const or_lattice* L, double* out)
{
    memcpy(out, L->fstar, sizeof(double) * 2 * L->Q * L->N);
    return L->Q;
}

int or_get_post_stream(const or_lattice* L, double* out)
{
    memcpy(out, L->fpost, sizeof(double) * 2 * L->Q * L->N);
    return L->Q;
}

int or_get_densities(const or_lattice* L, double* out)
{
    memcpy(out, L->rho_all, sizeof(double) * 2 * (L->nz + 2) * L->nx * L->ny);
    return L->Q;
}
