/*
 * lbm.h - C ABI of the GB300 library for the two-component regularised
 * colour-gradient lattice Boltzmann step with a shear-thinning ink and a
 * moving print head (Monteferrante et al., arXiv 2102.02655, Sec. II-III).
 *
 * One handle owns one lattice resident in device memory. All compute runs in
 * the library's CUDA kernels on the handle's stream; the host side only
 * validates arguments, computes the nozzle position per step and enqueues
 * kernels.
 *
 * Conventions
 *  - Lattice indices: site (x, y, z), x fastest, z the vertical axis (the
 *    substrate is below z = 0, the open top above z = nz - 1). Field arrays
 *    are [z][y][x] contiguous.
 *  - Every call returns an lbm_status; nothing aborts. A failing call stores a
 *    message readable with lbm_last_error. An LBM_ECUDA error is sticky: the
 *    handle refuses further work and must be destroyed.
 *  - Pointers named *_dev or passed with on_device = 1 are device pointers on
 *    the handle's device; others are host pointers. Field values are double
 *    for LBM_F64 storage and float otherwise (F32, F16DEV, BF16DEV).
 *  - Calls on one handle must not overlap (one host thread at a time).
 *  - A call that touches the GPU makes the handle's device (cfg->device)
 *    current while it runs and gives the caller's current device back on
 *    return.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* invalid argument or configuration */
    LBM_ENOMEM = 2,     /* device allocation failed */
    LBM_ECUDA = 3,      /* CUDA runtime error (sticky) */
    LBM_EUNSTABLE = 4,  /* a site's total density was not finite and positive */
    LBM_ETIMEOUT = 5,   /* a bounded wait ran out (host wait; or, sticky, a kernel's internal wait) */
    LBM_ESTATE = 6      /* call out of order (e.g. lbm_step before geometry and rheology) */
} lbm_status;

/* Velocity set. D2Q9 is the paper's lattice (Sec. II A), laid in the x-z
 * plane (ny must be 1); D3Q19 is the standard 3D set used for 3D lattices. */
typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_velset;

/* Storage of the populations. F64 and F32 store and compute in that type.
 * F16DEV and BF16DEV store 16-bit deviations from a local rest state and
 * compute in FP32 (reductions in FP64): slot 1 holds the total deviation
 * f^Y_i + f^B_i - w_i rho0_amb, slot 0 the ink population minus
 * c w_i rho0_amb, c the ink fraction of the site that wrote it (kept per site
 * in FP32 beside each population buffer). 2 x Q x 2 bytes + 4 bytes per site
 * and buffer instead of 2 x Q x 4. Fields and diagnostics are FP32/FP64 as for
 * F32. Not accepted by lbm_step_noalloc. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16DEV = 2, LBM_BF16DEV = 3 } lbm_storage;

/* Execution path: PLAIN runs the phase-by-phase kernels over the whole
 * lattice; FUSED runs the fused z-marching kernel over the bulk and the
 * phase-by-phase kernels only in a box around the nozzle (D3Q19 only).
 * AUTO picks FUSED where it applies. Both give the same result. */
typedef enum { LBM_PATH_AUTO = 0, LBM_PATH_PLAIN = 1, LBM_PATH_FUSED = 2 } lbm_path;

typedef enum { LBM_Z_PERIODIC = 0, LBM_Z_WALLS = 1 } lbm_zmode;
typedef enum { LBM_TOP_OPEN = 0, LBM_TOP_WALL = 1 } lbm_topmode;
typedef enum { LBM_NEWTONIAN = 0, LBM_CROSS = 1, LBM_POWER_LAW = 2 } lbm_law;

/* Lattice and model constants (Sec. II A). */
typedef struct {
    int nx, ny, nz;
    int velset;            /* lbm_velset */
    int storage;           /* lbm_storage */
    int path;              /* lbm_path */
    double tau_ambient;    /* relaxation time of the Newtonian ambient (blue) fluid */
    double rho0_ink, rho0_amb;    /* reference densities in the phase field rho^N */
    double alpha_ink, alpha_amb;  /* phi_0 of each component (Eq. 7); <= 0 selects w_0 */
    double A;              /* perturbation strength, sigma = 2 tau A / 9 (Eq. 10, 13) */
    double beta;           /* recolouring parameter (Eq. 14-15) */
    double zeta_ink, zeta_amb;    /* wall affinities in the fictitious densities (Eq. 18) */
    double drag_gamma;     /* friction coefficient of the substrate drag (Eq. 29) */
    double drag_height;    /* the drag acts closer than this to the substrate */
    double body_force[3];  /* body acceleration (0 in the print runs) */
    int device;            /* CUDA device ordinal */
    void* cuda_stream;     /* cudaStream_t to enqueue on; NULL = a stream the library creates */
    /* Optional device allocator. NULL alloc = cudaMalloc/cudaFree. The
     * callbacks run inside lbm_create and lbm_destroy only. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* alloc_ctx;
} lbm_config;

/* Print-head geometry and boundaries (Sec. II B, Sec. III). */
typedef struct {
    int z_mode;            /* lbm_zmode: periodic in z, or substrate below and a top boundary */
    int top_mode;          /* lbm_topmode: open (anti-bounce-back, Eq. 28) or a moving lid */
    int nozzle;            /* 1: annular nozzle present (requires LBM_Z_WALLS) */
    double head_pos[2];    /* nozzle axis (x, y) at step 0, lattice units */
    double head_vel[2];    /* nozzle velocity v_nozzle in the x-y plane (Eq. 26) */
    double r_inner;        /* inner radius of the nozzle wall */
    double wall_thickness; /* the wall spans r_inner <= r <= r_inner + wall_thickness */
    int gap;               /* lowest z of the nozzle wall; the substrate is at z = -1/2 */
    double u_ink;          /* extrusion speed in the head frame, along -z (Eq. 27) */
    double top_vel[3];     /* lid velocity when top_mode = LBM_TOP_WALL */
    double rho_top_amb;    /* ambient density imposed at the open top (Eq. 28) */
} lbm_geometry;

/* Ink rheology (Eq. 23-25): kinematic viscosity of the ink as a function of
 * the shear rate from the implicit equation Eq. 24. */
typedef struct {
    int law;               /* lbm_law */
    double nu0, nu_inf, lambda, n;  /* Cross: nu = nu_inf + (nu0 - nu_inf)/(1 + (lambda gdot)^n) */
    double K;              /* power law: nu = K gdot^(n-1) */
    double tau_min, tau_max;        /* clamps of the ink and mixture relaxation times */
    double tol;            /* relative tolerance of the shear-rate iteration (<= 0: default) */
    int max_iter;          /* iteration cap (<= 0: default 60) */
} lbm_rheology;

/* Diagnostics, accumulated in FP64 on the device. */
typedef struct {
    double mass[2];        /* sum of rho^ink, rho^amb over fluid nodes at the last step */
    double momentum[3];    /* sum of rho u (physical velocity) at the last step */
    double bc_flux[2];     /* cumulative mass entering minus leaving at boundary links */
    double created[2];     /* cumulative mass of nodes uncovered by the nozzle */
    double destroyed[2];   /* cumulative mass of nodes covered by the nozzle */
    long long step;        /* steps since lbm_set_geometry */
    int unstable;          /* 1 if any site's total density was not finite and positive */
} lbm_diag;

/* Field selection bits for lbm_fields; the buffers are taken in this order. */
enum {
    LBM_FIELD_RHO_INK = 1 << 0,  /* rho^Y (Eq. 2) */
    LBM_FIELD_RHO_AMB = 1 << 1,  /* rho^B */
    LBM_FIELD_U = 1 << 2,        /* physical velocity, 3 arrays ux, uy, uz (Eq. 3) */
    LBM_FIELD_NU = 1 << 3,       /* mixture kinematic viscosity c_s^2 (tau - 1/2) (Eq. 17) */
    LBM_FIELD_P = 1 << 4,        /* pressure sum_k p^k (Eq. 9) */
    LBM_FIELD_PHI = 1 << 5,      /* phase field rho^N */
    LBM_FIELD_SOLID = 1 << 6     /* 1 on nozzle nodes, 0 on fluid nodes */
};

/* Create a lattice (Sec. II A constants). Allocates the device state through
 * cfg->alloc (or cudaMalloc). Returns LBM_EINVAL for bad sizes/values,
 * LBM_ENOMEM if an allocation fails. *out is NULL on failure. */
lbm_status lbm_create(const lbm_config* cfg, struct lbm_handle** out);

/* Set the print-head geometry and boundaries, reset the step counter and the
 * diagnostics, and initialise the state of Sec. III: the nozzle interior
 * above the gap filled with ink, ambient fluid elsewhere, all at rest, with
 * equilibrium populations. LBM_EINVAL for an inconsistent geometry: non-finite
 * values, |head_vel| or |u_ink| above 0.5, a gap outside [1, nz), and, with a
 * nozzle, r_inner + wall_thickness above 2000 or nx, ny above 4000 (the
 * fixed-point geometry of the nozzle squares distances in 64-bit integers). */
lbm_status lbm_set_geometry(struct lbm_handle* h, const lbm_geometry* g);

/* Set the ink rheology (Eq. 23-25). LBM_EINVAL if tau_min <= 1/2 or
 * tau_max < tau_min or the law's parameters are out of range. */
lbm_status lbm_set_ink_rheology(struct lbm_handle* h, const lbm_rheology* r);

/* Replace the state by equilibrium populations of the given densities and
 * velocity (u = NULL: at rest) on every fluid node; solid nodes are ignored.
 * rho_ink, rho_amb: nx*ny*nz values; u: 3 arrays (ux, uy, uz) back to back.
 * on_device selects device or host pointers. Resets the ledger. */
lbm_status lbm_set_fields(struct lbm_handle* h, const void* rho_ink, const void* rho_amb,
                          const void* u, int on_device);

/* Enqueue nsteps time steps (Eq. 1) on the handle's stream and return. The
 * macroscopic fields of the last step are kept for lbm_fields. LBM_ESTATE if
 * geometry or rheology are missing. */
lbm_status lbm_step(struct lbm_handle* h, int nsteps);

/* Copy the fields selected by mask (LBM_FIELD_*) of the last completed step
 * into dst[0..] (one nx*ny*nz buffer per field, three for LBM_FIELD_U), on the
 * device or host per dst_on_device, and fill *diag if not NULL. Waits for the
 * stream. Returns LBM_EUNSTABLE (after copying) if the unstable flag is set, and LBM_ETIMEOUT
 * (sticky) if a kernel's bounded internal wait ran out (the state is then lost). */
lbm_status lbm_fields(struct lbm_handle* h, unsigned mask, void* const* dst, int dst_on_device,
                      lbm_diag* diag);

/* Wait for all enqueued work, giving up after timeout_ms (<= 0: no limit);
 * LBM_ETIMEOUT if it did not finish in time. */
lbm_status lbm_sync(struct lbm_handle* h, int timeout_ms);

/* Release the lattice and its device memory. NULL is accepted. */
void lbm_destroy(struct lbm_handle* h);

/* Message of the last failing call on h (or of the last lbm_create failure
 * when h is NULL). Valid until the next call on h. */
const char* lbm_last_error(const struct lbm_handle* h);

/* Number of kernel launches enqueued on h since its creation. */
long long lbm_kernel_launches(const struct lbm_handle* h);

/* Device time of the library's kernels, measured with CUDA events recorded
 * on the handle's stream around the fused bulk kernel and around the group of
 * phase-by-phase kernels of every step while profiling is on. */
typedef struct {
    double bulk_ms;            /* summed duration of the fused bulk kernel launches */
    double plain_ms;           /* summed duration of the phase-by-phase kernel groups */
    long long bulk_launches, plain_groups;
    long long bulk_sites;      /* site updates done by the fused bulk kernel */
    long long plain_sites;     /* site updates done by the phase-by-phase kernels */
} lbm_timing;

/* Turn event timing on (1) or off (0); turning it on clears the totals. */
lbm_status lbm_profile(struct lbm_handle* h, int enable);

/* Wait for the stream and return the totals since profiling was turned on. */
lbm_status lbm_timings(struct lbm_handle* h, lbm_timing* out);

/* One time step on population buffers the caller owns, with no device
 * allocation at all. This entry point has no counterpart in the paper: it is
 * for callers that cannot call cudaMalloc, such as code running inside
 * another framework's memory pool or a pre-sized arena that forbids new
 * allocations, and real-time loops where an allocation could stall or fail.
 * lbm_create allocates the lattice state; this call does not: every device
 * buffer comes from the caller, and the work space lives in one fixed static
 * device array of LBM_NOALLOC_SCRATCH_BYTES inside the library (held by every
 * GPU that loads the library, until the process exits).
 *
 * It runs the phase-by-phase kernels of lbm_step over the whole lattice.
 *  cfg, g, r  lattice constants, geometry and rheology as for lbm_create,
 *             lbm_set_geometry and lbm_set_ink_rheology; cfg->device selects
 *             the GPU, cfg->cuda_stream the stream (NULL = the legacy default
 *             stream); cfg->path, alloc, free and alloc_ctx are ignored.
 *  step       index n >= 1 of the step taken: the nozzle moves from its step
 *             n-1 to its step n position.
 *  f_in       device buffer of 2*Q*N values (double for LBM_F64, else float):
 *             the post-collision populations of step n-1, value (k*Q + i)*N +
 *             site with site = (z*ny + y)*nx + x; slot k = 0 holds the ink
 *             populations f^Y_i, slot k = 1 holds f^Y_i + f^B_i - w_i rho0_amb.
 *             At rest with phi = w: slot 0 = w_i rho_ink, slot 1 =
 *             w_i (rho_ink + rho_amb - rho0_amb).
 *  f_out      device buffer of the same size for step n; must not overlap f_in.
 *  fields     optional device buffer of 9*N values: rho_ink, rho_amb, ux, uy,
 *             uz, nu, p, rho^N, solid of step n (NULL: not written).
 *  diag       optional host struct: mass and momentum of step n (only when
 *             fields is given, else 0) and this step's boundary flux and
 *             created/destroyed mass; filling it waits for the stream.
 * The previous step's densities and top-plane velocities are rebuilt from
 * f_in (collision conserves each component's mass), so the result equals
 * lbm_step's up to rounding. Arguments pass the same checks as in lbm_create,
 * lbm_set_geometry and lbm_set_ink_rheology. Each call looks up the static
 * array's device address on cfg->device (no allocation); the first call on a
 * device also loads the library's kernels there, so make that first call
 * before any stream capture. The caller's current device is kept.
 * All calls share the one array and it keeps the last call's contents (the
 * call clears what must start at zero): calls that overlap on the GPU race,
 * so issue them on one stream or wait between them. Returns LBM_EINVAL for
 * invalid arguments or a lattice whose work space (four densities per site,
 * the top planes' velocities and one byte per column) exceeds the array, about 500k sites in
 * FP64 and 1M in FP32, LBM_ECUDA on a CUDA error,
 * LBM_EUNSTABLE (diag requested) if a site's total density was not finite
 * and positive. */
#define LBM_NOALLOC_SCRATCH_BYTES (16u << 20)
lbm_status lbm_step_noalloc(const lbm_config* cfg, const lbm_geometry* g, const lbm_rheology* r, long long step,
                            const void* f_in, void* f_out, void* fields, lbm_diag* diag);

typedef struct lbm_handle lbm_handle;

/* ---------------------------------------------------------------------------
 * Batches: many independent lattices (a parameter sweep of print runs,
 * Sec. III) advanced together on one device. Each lattice keeps its own
 * handle, state and parameters; per time step (Eq. 1) one persistent launch
 * covers the bulk of every lattice and one launch per phase covers every
 * nozzle box, and G steps at a time run as one replayed CUDA graph. Every
 * lattice computes exactly what lbm_step computes on it alone, whatever the
 * plan (tile height, z-planes per column).
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* Group n lattices (host array of handles, not copied beyond this call;
 * the handles stay owned by the caller and must outlive the batch). Every
 * lattice must be configured (geometry and rheology set), take the fused path
 * (D3Q19, substrate below, open top, 38 N < 2^31), and share the device, the
 * storage and the density-ratio class (ratio one or not) with the others;
 * nx <= 65535, ny <= 32767. Returns LBM_EINVAL / LBM_ESTATE otherwise (message
 * from lbm_batch_last_error(NULL)), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_batch_create(lbm_handle* const* lattices, int n, lbm_batch** out);

/* Replace the batch's lattices (same conditions as lbm_batch_create, and the
 * batch's device and storage), keeping its streams and reusing its step
 * tables where they are large enough; the plan returns to the default. Waits
 * for the batch's stream. For continuous batching, where members come and go. */
lbm_status lbm_batch_reset(lbm_batch* b, lbm_handle* const* lattices, int n);

/* Advance every lattice of the batch by nsteps steps (asynchronous on the
 * batch's own stream, ordered after work already enqueued on each lattice's
 * stream and before work enqueued there later). The fields of the last step
 * are kept for lbm_fields on each handle. */
lbm_status lbm_batch_step(lbm_batch* b, int nsteps);

/* Wait for the batch's stream. */
lbm_status lbm_batch_sync(lbm_batch* b);

/* Set the plan: variant 0 (32 x 8 tile columns, the one bulk-kernel
 * configuration; any other value is LBM_EINVAL) and, per lattice (host array of n ints), at most how many z-planes
 * one CTA of the bulk kernel marches up a column (the column's nz planes are
 * split into ceil(nz / zchunk) chunks whose lengths differ by at most one).
 * Waits for the batch's stream. */
lbm_status lbm_batch_set_plan(lbm_batch* b, int variant, const int* zchunk);

/* Autotuner: times trial_steps real steps of the batch (after one untimed
 * graph capture) for each candidate plan (variant x CTAs per SM of the
 * persistent bulk kernel, all that fit or one fewer, which leaves room for the
 * box kernels beside it x z-planes per column in 8 .. 128 up to the tallest
 * lattice) and keeps the fastest. The trial steps advance the lattices (every
 * candidate computes the same result). */
#define LBM_TUNE_MAX 40
typedef struct {
    int variant, zchunk, ctas_per_sm;  /* chosen plan */
    double ms_per_step;                /* its time per batch step */
    int n_tried;                       /* candidates timed */
    int tried_variant[LBM_TUNE_MAX], tried_zchunk[LBM_TUNE_MAX], tried_ctas[LBM_TUNE_MAX];
    double tried_ms[LBM_TUNE_MAX];
} lbm_batch_tuning;
lbm_status lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_tuning* out);

typedef struct {
    int n_lattices, variant, tile_h, n_items, grid, steps_per_graph;
    long long steps, launches;  /* batch steps taken, kernels launched by them */
} lbm_batch_plan_info;
lbm_status lbm_batch_info(const lbm_batch* b, lbm_batch_plan_info* out);

/* Release the batch (not its lattices). NULL is accepted. */
void lbm_batch_destroy(lbm_batch* b);

/* Message of the last failing call on b (NULL: of the last lbm_batch_create). */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Host-only helper (no device work): the work list of the persistent bulk
 * kernel for n lattices of sizes dims[3l..3l+2] = (nx, ny, nz), tile height
 * tile_h and at most zchunk[l] z-planes per item (each column's nz planes in
 * ceil(nz / zchunk[l]) chunks whose lengths differ by at most one). Writes up
 * to cap items of four ints (lattice, x0 | y0 << 16, za, zb) to items (may be
 * NULL) and returns
 * the item count, or -1 for invalid arguments. */
long long lbm_batch_plan(const int* dims, int n, int tile_h, const int* zchunk, int* items, long long cap);

/* Device bytes lbm_create allocates for cfg (host-only; -1 if cfg is
 * invalid): both population buffers (with the 16-bit storage's ink-fraction
 * arrays), the density and top-velocity arrays, the field planes and the
 * accumulators. */
long long lbm_lattice_bytes(const lbm_config* cfg);

/* ---------------------------------------------------------------------------
 * Serving: print-run simulation requests (ink law, extrusion rate, head
 * velocity, nozzle size: the parameters of Sec. III) arriving over time.
 * Requests wait in arrival order; each lbm_server_poll admits the waiting
 * ones while an active slot is free and their lbm_lattice_bytes fit the HBM
 * budget, advances all active requests together as one batch (lbm_batch_*)
 * by min(quantum, the fewest remaining steps), and retires the ones that
 * reached their step count: their rho_ink, rho_amb, ux, uy, uz are copied to
 * host memory and their slot is free at once, so the next waiting request
 * can join in the same call (continuous batching). A retired lattice is kept
 * in a pool for a later request with the same sizes and model constants
 * (pooled lattices count against the budget and are freed, oldest first,
 * when a request needs their memory). A result equals what the
 * same request computes alone (lbm_create + lbm_step) to rounding.
 * ------------------------------------------------------------------------- */
typedef struct lbm_server lbm_server;
typedef struct {
    unsigned long long hbm_budget;  /* device bytes the active lattices may hold */
    int device;                     /* CUDA device of every request */
    int storage;                    /* lbm_storage of every request */
    int quantum;                    /* steps per poll at most */
    int max_active;                 /* requests advanced together at most */
} lbm_server_config;
typedef struct {
    double t_submit, t_admit, t_done;  /* seconds since lbm_server_create */
    long long steps;
} lbm_server_timing;
typedef struct {
    int waiting, active, finished, peak_active;
    long long bytes_in_use;    /* device bytes of active and pooled lattices */
    long long rounds, batch_steps, site_steps, batch_rebuilds;
    long long reused;          /* admissions served by a pooled lattice */
    int pooled;                /* idle lattices kept for reuse */
    double clock;              /* seconds since lbm_server_create */
} lbm_server_counters;

lbm_status lbm_server_create(const lbm_server_config* cfg, lbm_server** out);

/* Queue a request: a D3Q19 print run (z_mode walls, open top) of nsteps >= 1
 * steps from the print setup's initial state (nozzle filled with ink). The
 * server sets cfg's device, storage, path (fused), stream and allocator.
 * Writes the request id to *id. The structs are copied. */
lbm_status lbm_server_submit(lbm_server* s, const lbm_config* cfg, const lbm_geometry* g, const lbm_rheology* r,
                             long long nsteps, long long* id);

/* One scheduling round (blocks while the round's steps run on the device).
 * *n_finished: requests finished in this round. */
lbm_status lbm_server_poll(lbm_server* s, int* n_finished);

/* Ids of finished, uncollected requests (up to cap written); returns how
 * many there are. */
int lbm_server_finished(const lbm_server* s, long long* ids, int cap);

/* Collect a finished request: copies its five field planes (nx*ny*nz values
 * each, double for LBM_F64 else float; NULL entries skipped) to the host
 * buffers host_dst[0..4] = rho_ink, rho_amb, ux, uy, uz, its diagnostics and
 * timing, and forgets it. Returns the request's own status (e.g.
 * LBM_EUNSTABLE, LBM_ENOMEM if it could never fit the budget), LBM_ESTATE
 * if it has not finished. */
lbm_status lbm_server_result(lbm_server* s, long long id, void* const* host_dst, lbm_diag* diag,
                             lbm_server_timing* timing);

lbm_status lbm_server_stats(const lbm_server* s, lbm_server_counters* out);

/* Release the server, its active lattices and uncollected results. */
void lbm_server_destroy(lbm_server* s);

const char* lbm_server_last_error(const lbm_server* s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
