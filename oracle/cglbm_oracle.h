/*
 * Plain FP64 CPU oracle for the two-component regularised colour-gradient
 * lattice Boltzmann step of Monteferrante et al., "Lattice Boltzmann
 * multicomponent model for direct-writing printing" (Sec. II A, II B, III).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * All arithmetic is double precision. Every step is a plain loop over the
 * lattice in the order the method states (stream, node flips, moments, wall
 * densities, colour gradient, local relaxation time, regularised BGK,
 * perturbation, recolouring). Each function cites the passage it follows.
 *
 * Parity status of each part (what pins it) is listed in the test suite
 * (tests/test_oracle_*.py). The full coupled print run has no external
 * reference: parity unpinned for that composition as a whole; its parts are
 * pinned one by one.
 */
#ifndef CGLBM_ORACLE_H
#define CGLBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_D2Q9 = 0, OR_D3Q19 = 1 };
enum { OR_LAW_NEWTONIAN = 0, OR_LAW_CROSS = 1, OR_LAW_POWER = 2 };
enum { OR_Z_PERIODIC = 0, OR_Z_WALLS = 1 };
enum { OR_TOP_OPEN = 0, OR_TOP_WALL = 1 };

/* Fields written by or_fields, in this order, each nx*ny*nz doubles. */
enum { OR_F_RHO_INK = 0, OR_F_RHO_AMB, OR_F_UX, OR_F_UY, OR_F_UZ, OR_F_NU, OR_F_P, OR_F_RHON, OR_F_SOLID, OR_NFIELDS };

typedef struct {
    int nx, ny, nz;
    int velset;                 /* OR_D2Q9 (x-z plane, ny must be 1) or OR_D3Q19 */
    double tau_amb;             /* ambient (blue) relaxation time, Sec. III */
    double rho0_ink, rho0_amb;  /* reference densities entering rho^N */
    double alpha_ink, alpha_amb;/* phi_0 of each component, Eq. 7 */
    double A, beta;             /* perturbation strength (Eq. 10), recolouring (Eq. 14-15) */
    double zeta_ink, zeta_amb;  /* wall affinities, Eq. 18 */
    double drag_gamma, drag_height; /* drag near the substrate, Eq. 29 */
    double g[3];                /* body acceleration (for channel-flow checks) */
    double grad_floor;          /* |grad rho^N| at or below which cos(phi_i) of Eq. 16 is
                                   taken as 0 (the 0/0 case): the rounding level of the
                                   arithmetic that computes the gradient; 0 selects
                                   2^-45 (2^8 units of FP64 rounding) */
} or_params;

typedef struct {
    int z_mode;                 /* OR_Z_PERIODIC or OR_Z_WALLS */
    int top_mode;               /* OR_TOP_OPEN (anti-bounce-back, Eq. 28) or OR_TOP_WALL */
    int nozzle;                 /* 1: moving nozzle present (needs OR_Z_WALLS) */
    double head_pos[2];         /* nozzle axis (x, y) at step 0 */
    double head_vel[2];         /* nozzle velocity, Eq. 26-27 */
    double r_inner, wall_thickness;
    int gap;                    /* lowest z of the nozzle wall */
    double u_ink;               /* extrusion speed in the head frame, Eq. 27 */
    double top_vel[3];          /* lid velocity when top_mode == OR_TOP_WALL */
    double rho_top_amb;         /* imposed ambient density at the open top */
} or_geom;

typedef struct {
    int law;                    /* OR_LAW_* */
    double nu0, nu_inf, lambda, n;  /* Cross law, Eq. 23 (kinematic form, Eq. 25) */
    double K;                   /* power law nu = K gdot^(n-1) */
    double tau_min, tau_max;    /* clamps on the relaxation time */
} or_rheo;

typedef struct {
    double mass[2];       /* sum of rho^k over fluid nodes at the last step */
    double momentum[3];   /* sum of rho u (physical velocity) */
    double bc_flux[2];    /* cumulative mass in minus out at boundary links */
    double created[2];    /* cumulative mass of created nodes */
    double destroyed[2];  /* cumulative mass of destroyed nodes */
    long long step;
} or_diag;

typedef struct or_lattice or_lattice;

or_lattice* or_create(const or_params* p);
void        or_destroy(or_lattice* L);
int         or_set_geometry(or_lattice* L, const or_geom* g);
int         or_set_rheology(or_lattice* L, const or_rheo* r);
int         or_set_fields(or_lattice* L, const double* rho_ink, const double* rho_amb, const double* u);
int         or_step(or_lattice* L, int nsteps);
void        or_fields(const or_lattice* L, double* out);   /* OR_NFIELDS * nx*ny*nz */
void        or_get_diag(const or_lattice* L, or_diag* d);
int         or_get_populations(const or_lattice* L, double* out); /* 2*Q*N post-collision */
/* State inside the last step, for the pin tests: the populations after
 * streaming and node creation, before the collision (2*Q*N; meaningful at the
 * fluid nodes of the step), and the densities the colour gradient read
 * (2 components x (nz+2) planes z = -1..nz x ny x nx: fluid nodes after
 * streaming, created nodes, the fictitious densities of Eq. 18 on solid nodes
 * and on the substrate or lid plane, the copied ghost plane of an open top). */
int         or_get_post_stream(const or_lattice* L, double* out);
int         or_get_densities(const or_lattice* L, double* out);

/* Unit-level entry points used by the pin tests. */
int    or_velset(int velset, int* c, double* w, double* B);        /* returns Q */
double or_phi(int velset, double alpha, int i);
double or_solve_tau_ink(const or_rheo* r, double S, double rho_ink, double* gdot_out);
double or_wall_interp(double r0, double r1, double r2);
/* One collision at one site. fin: 2*Q populations; nbr: 2*Q neighbour
 * densities (component-major, entry i = density at x + c_i, i = 0 ignored);
 * out: 2*Q post-collision populations; aux[0..4] = tau, |grad rhoN|, ux, uy, uz. */
void   or_collide_one(const or_lattice* L, const double* fin, const double* nbr,
                      double z_wall_dist, double* out, double* aux);

#ifdef __cplusplus
}
#endif
#endif
