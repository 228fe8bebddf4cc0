/*
 * mps.h -- C ABI of the GB300 MPS time-step library.
 *
 * One Moving Particle Semi-implicit (MPS) time step, after Vieira-e-Silva et al., "A fluid
 * simulation system based on the MPS method" (arXiv 2105.01677):
 *   - cell-linked-list neighbour search (Sec. 4.1), here a Morton-sorted bucket grid;
 *   - particle number density (Eq. 5), Laplacian model (Eq. 7) and pressure gradient
 *     (difference form of the multi-density gradient, Sec. 3.2.1) with w(r) = re/r - 1 (Eq. 4);
 *   - the pressure Poisson equation (Eq. 13) assembled as in the CUDA PPE listing (Listing 2) of Sec. 4.3
 *     and solved by conjugate gradients (Sec. 3.1.2), or
 *   - the weakly-compressible equation-of-state pressure (Eq. 16).
 *
 * Conventions for every call:
 *   - Return 0 (MPS_OK) on success or a negative MPS_E* code; mps_strerror() names it.
 *   - Host pointers are ordinary (pageable or pinned) host memory owned by the caller; the
 *     library only reads or writes them during the call.
 *   - Particle arrays are indexed by the caller's particle id 0..n-1 ("original order").
 *     Vector quantities are array-of-structs with `dim` doubles per particle (x, y[, z]).
 *   - Particle kinds (int8): MPS_FLUID, MPS_WALL, MPS_DUMMY, MPS_GHOST.  WALL particles take
 *     part in the PPE but never move; DUMMY particles only count towards the number density
 *     (the "bcon == -1" particles of the PPE listing); GHOST particles are out of the domain
 *     and ignored.  A particle that leaves the cell grid becomes a GHOST (not an error).
 *   - Calls on one context are not thread-safe; different contexts are independent.
 *   - Every call is synchronous with respect to the host: when it returns, its device work
 *     is complete.
 *   - The context owns all device memory it allocates (from `alloc`/`release` if given,
 *     else cudaMalloc/cudaFree) until mps_destroy().
 */
#ifndef MPS_GB300_H
#define MPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Particle kinds. */
#define MPS_FLUID 0
#define MPS_WALL 1
#define MPS_DUMMY 2
#define MPS_GHOST 3

/* Status codes. */
#define MPS_OK 0
#define MPS_EINVAL -1       /* bad argument: dim, radii, sizes, non-positive n, grid too large */
#define MPS_ENOMEM -2       /* device or host allocation failed                              */
#define MPS_ECG_NOCONV -3   /* CG did not reach cg_tol within cg_max_iter (report filled)    */
#define MPS_ENONFINITE -4   /* NaN or Inf in a position or velocity                          */
#define MPS_ESKIN -5        /* more than max(64, n/256) particles moved more than half the   *
                             * cell skin within a step (fewer: their lists are completed)     */
#define MPS_ECOINCIDENT -6  /* two neighbouring particles at distance 0 (w infinite, Eq. 4)  */
#define MPS_ECAP -7         /* a caller buffer or the per-particle neighbour cap is too small */
#define MPS_EDEVICE -8      /* a CUDA call failed or a device-side wait gave up              */

/* Device memory hooks: alloc returns a device pointer of >= bytes (256-byte aligned) or
 * NULL; release frees it.  Both receive `user`.  Both NULL: cudaMalloc / cudaFree. */
typedef void* (*mps_alloc_fn)(size_t bytes, void* user);
typedef void (*mps_release_fn)(void* ptr, void* user);

typedef struct {
    int32_t dim;              /* 2 or 3                                                        */
    int32_t pressure_mode;    /* 0: PPE solved by CG (Eq. 13); 1: equation of state (Eq. 16)  */
    double l0;                /* average particle distance [m]                                */
    double re_n;              /* influence radius of number density, gradient, p_hat [m]      */
    double re_lap;            /* influence radius of the Laplacian (viscosity, PPE) [m]       */
    double rho;               /* density [kg/m^3]                                             */
    double nu;                /* kinematic viscosity [m^2/s]                                  */
    double dt;                /* time step [s]                                                */
    double beta;              /* free-surface threshold of Eq. 15 (paper: 0.97)               */
    double g[3];              /* external acceleration [m/s^2]                                */
    double c0;                /* speed of sound of Eq. 16 [m/s]                               */
    double gamma;             /* exponent of Eq. 16 (paper: 7)                                */
    double alpha_c;           /* PPE diagonal term alpha_c/dt^2 (listing of Sec. 4.3: 1e-7)   */
    double cg_tol;            /* stop when ||b - A p|| / ||b|| <= cg_tol (FP64 residual)       */
    int32_t cg_max_iter;      /* total CG iteration cap per solve; <= 0: 10 n                 */
    int32_t precision;        /* 0: FP64 throughout; 1: mixed (FP32 pair terms and inner CG,   *
                               *    FP64 number density, dot products, residual, refinement)  */
    int32_t clamp_negative_p; /* PPE only: p = max(p, 0) after the solve (default 1)          */
    int32_t nbr_cap;          /* max stored non-dummy neighbours per particle within re_lap;   *
                               * <= 0: 1.5x the ideal-lattice count, rounded up to 32          */
    double cell_skin;         /* s: cell side h = max(re_n, re_lap) (1 + s); a step fails with *
                               * MPS_ESKIN if a particle moves more than s max(re)/2           */
    double box_min[3];        /* cell grid origin [m]; unused axes ignored                    */
    double box_max[3];        /* cell grid extent: ncell = floor((max - min)/h) + 1 per axis  */
    double inner_tol;         /* mixed: relative residual reduction of an FP32 inner CG that   *
                               * cannot finish the solve; the sweep that can (the reduction    *
                               * still needed, with a margin of 2, is >= 1e-6) asks for that   */
    int32_t max_outer;        /* mixed: cap on FP64 refinement sweeps                          */
    int32_t ppe_operator;     /* mixed inner operator: 0 stored FP32 coefficients,             *
                               * 1 matrix-free (coefficients recomputed from positions)        */
    int32_t device;           /* CUDA device ordinal                                           */
    int32_t gather_block;     /* threads per cell block of the candidate gather (warps that   *
                               * share a cell's candidates): 32, 64, 96 or 128; 0 chooses by   *
                               * dimension (tuning only, results identical)                    */
    int32_t list_every;       /* candidate lists (cell gather within h): 0 or 1 gathers them  *
                               * every step; K > 1 keeps them for up to K steps, gathering    *
                               * afresh earlier as soon as a particle has moved more than     *
                               * s max(re)/2 from where they were gathered or leaves the grid. *
                               * Neighbour sets stay exact either way (Sec. 5.6.3 runs the    *
                               * paper's fast mode with a refresh every 4 steps).              */
    int32_t kernel;           /* weight w(r): 0 the kernel of Eq. 4, re/r - 1 (default);       *
                               * 1 (1 - r/re)^3, the kernel the paper recommends with the      *
                               * equation of state (Sec. 3.1); n0 and lambda follow it          */
    int32_t gradient_form;    /* 0 difference form (p_j - p_hat_i) (default); 1 CMPS, Eq. 18: *
                               * ((p_i + p_j) - (p_hat_i + p_hat_j)), momentum-conserving;     *
                               * p_hat is then the neighbourhood minimum on both paths         */
    int32_t source_term;      /* PPE source: 0 Eq. 13, (n* - n0)/(n0 dt^2) (default); 1 HS,    *
                               * Eq. 21, (Dn/Dt)* / (n0 dt) from the predicted velocities over *
                               * the number-density neighbours; 2 HS plus the error-           *
                               * compensating source of Eq. 24-25, ECS / dt, from n and Dn/Dt  *
                               * at the step's start (1 and 2 require kernel 0; with           *
                               * pressure_mode 1 there is no PPE and the value is ignored)      */
    int32_t ppe_host_loop;    /* mixed PPE of one scene: 0 (default) runs the refinement and   *
                               * inner CG loops on the device as one CUDA graph with           *
                               * conditional nodes (one launch and one read per solve); 1     *
                               * drives them from the host, polling per chunk of iterations.  *
                               * Results are identical.                                        */
    int32_t cg_x0;            /* PPE initial guess from the previous steps' solutions before  *
                               * the clamp (carried with the particles): 0 (default) x0 = 0;  *
                               * 1 the previous solution; 2 its linear, 3 its quadratic, 4    *
                               * its cubic extrapolation in time from the last 2, 3 or 4      *
                               * solutions (the polynomial through them at equal steps; lower *
                               * orders while fewer exist; none before the first solve and    *
                               * after mps_write_state).  The stop rule is unchanged (FP64    *
                               * ||b - A p|| / ||b|| <= cg_tol); a step then depends on the   *
                               * previous steps' solves at the level of the tolerance          */
    int32_t step_graph;       /* 1 (default): a step on the mixed path (device-driven PPE) or  *
                               * the equation-of-state path, with candidate lists gathered    *
                               * every step and the stage timers off, runs as one CUDA graph: *
                               * one launch and one synchronisation; 0: launch by launch (the *
                               * bucket build still one graph); 2: every kernel launched one  *
                               * by one, the bucket build included (for kernel profilers; the *
                               * mixed PPE solve's own graph follows ppe_host_loop).           *
                               * Results are identical.                                        */
    int32_t inner_cg;         /* mixed inner CG of the device-driven solve: 0 (default) three  *
                               * kernels per iteration; 1 two (fused: the recurrences of      *
                               * Chronopoulos and Gear; rounds differently, same stop rule)    */
    int32_t spmv_block;       /* threads per block of the FP32 SpMV: 256 or 512; 0: 512         */
    int32_t build_block;      /* threads per block of the row build (n*, flags, PPE rows): 64, *
                               * 128 or 256; 0: 128 on the mixed PPE path (whose blocks stage  *
                               * their output rows in shared memory), 256 elsewhere (tuning    *
                               * only, results identical)                                      */
    int32_t bucket_sort;      /* graph-run bucket builds: 0 (default) sort the particles whose *
                               * cell changed and merge them into the previous order when it   *
                               * holds (the radix sort otherwise); 1 always the radix sort.    *
                               * Both give the stable order by cell key: results identical.   */
    int32_t cg_unroll;        /* device-driven mixed solve: inner CG iterations per pass of its *
                               * conditional loop (1, 2 or 4; 0: 1); the iterations after     *
                               * convergence return at once (results identical)                */
    int32_t predict_tpr;      /* threads per FLUID row of the prediction: 1, 2 or 4 (0: 1); the *
                               * row's viscosity sums are added across them, so the rounding   *
                               * changes (well within the parity bounds)                        */
    void* stream;             /* cudaStream_t to run on, or NULL for a library-owned stream    */
    mps_alloc_fn alloc;       /* optional device allocator (see above)                        */
    mps_release_fn release;
    void* alloc_user;
} mps_params;

/* Per-step diagnostics (values of the last step of a call). */
typedef struct {
    int32_t status;           /* MPS_OK or the first error seen                               */
    int32_t cg_iters;         /* CG iterations (mixed: FP32 inner iterations, all sweeps)     */
    int32_t cg_outer;         /* mixed: FP64 refinement sweeps; FP64: restarts                 */
    int32_t list_gathered;    /* 1 if the step gathered its candidate lists afresh            */
    double cg_resid;          /* FP64 relative residual ||b - A p|| / ||b|| at exit            */
    int64_t n_surface;        /* FLUID/WALL particles with n* < beta n0 (Eq. 15)               */
    int64_t n_ghost;
    int64_t n_ppe_rows;       /* unknowns of the PPE                                          */
    double max_disp;          /* max |r* - r_b| over FLUID particles [m], r_b the positions   *
                               * the candidate lists were gathered at (r^k when every step)    */
    double n0_pnd;            /* reference number density at re_n (ideal lattice)             */
    double n0_lap;            /* reference number density at re_lap                           */
    double lambda;            /* lambda of Eq. 7 at re_lap [m^2]                               */
    int64_t steps_done;       /* steps completed by this context so far                       */
    int64_t cand_tests;       /* distance tests of the cell gather (candidate lists)          */
    int64_t pairs_ppe;        /* PPE coefficients evaluated (non-dummy pairs within re_lap)   */
    int64_t pairs_pnd;        /* number-density terms evaluated (pairs within re_n)           */
    int64_t list_tests;       /* candidate-list entries classified at r* (distance tests of  *
                               * the number-density / PPE assembly)                           */
    int32_t step_graph;       /* 1 if the step ran as one CUDA graph launch                    */
    int32_t n_fast;           /* FLUID particles that moved more than half the cell skin: their *
                               * candidate lists were completed by a direct search at r*      */
    int32_t bucket_merged;    /* the step's bucket build: 1 merged the particles whose cell    *
                               * changed into the previous order, 0 radix-sorted, -1 none (kept *
                               * lists)                                                        */
    int64_t n_moved;          /* particles whose cell key changed since the previous build     *
                               * (counted by graph-run builds; 0 launched kernel by kernel)     */
} mps_report;

/* Opaque context: device buffers, stream and derived constants of one particle system. */
typedef struct mps_ctx mps_ctx;

/* Fill *p with the defaults: dim 2, l0 0.01, re_n 2.1 l0, re_lap 4 l0, rho 1000, nu 1e-6,
 * dt 1e-4, beta 0.97, g (0, -9.81, 0), c0 20, gamma 7, alpha_c 1e-7, cg_tol 1e-8,
 * cg_max_iter 0, precision 0, clamp 1, nbr_cap 0, cell_skin 0.1, box [0,1]^dim,
 * inner_tol 1e-4, max_outer 30, ppe_operator 0, device 0, cg_x0 0, step_graph 1, no stream,
 * no hooks. */
void mps_params_default(mps_params* p);

/* Create a context from n particles (the problem statement of Sec. 3 and the particle kinds
 * of the PPE listing, Sec. 4.3).
 * pos: n*dim doubles; vel: n*dim doubles or NULL (zero); types: n int8 kinds.
 * The reference densities n0 (at re_n and re_lap) and lambda (at re_lap) are computed on the
 * host from an ideal lattice of spacing l0: all offsets o with 0 < |o| l0 < re (Eq. 5 and the
 * weighted mean of r^2 under Eq. 7).
 * Errors: MPS_EINVAL (params, n <= 0 or n >= 2^31, unknown kind, grid over 2^10 cells per
 * axis in 3D or 2^16 in 2D), MPS_ENONFINITE, MPS_ENOMEM, MPS_EDEVICE.
 * *out is written only on success; the caller's arrays are copied and not retained. */
int mps_create(const double* pos, const double* vel, const int8_t* types, int64_t n,
               const mps_params* params, mps_ctx** out);

/* Advance nsteps time steps (Sec. 3, semi-implicit predictor-corrector):
 *   1. bucket build at r^k: cell keys, Morton radix sort, cell table by scan (Sec. 4.1);
 *   2. predict FLUID u* = u + dt (nu lap(u) + g) (Eq. 2, Eq. 7 over re_lap), r* = r + dt u*;
 *   3. number density n* at r* (Eq. 5, re_n); free surface n* < beta n0 (Eq. 15);
 *   4. pressure: PPE A p = b (Eq. 13; A = -(1/rho) Lap + alpha_c/dt^2 I on FLUID/WALL rows
 *      off the surface, b = (n* - n0)/(n0 dt^2)) by CG, or the equation of state (Eq. 16);
 *   5. PPE: clamp p >= 0, p_hat_i = min of p over i and its non-dummy re_n neighbours;
 *   6. FLUID u = u* - (dt/rho) grad p, r = r* + dt (u - u*), gradient over re_n at r*.
 * last (nullable) receives the report of the final step.  On an error the remaining steps
 * are skipped and the state is unspecified (read it only to diagnose).
 * Errors: MPS_ECG_NOCONV, MPS_ESKIN, MPS_ECOINCIDENT, MPS_ECAP, MPS_ENONFINITE, MPS_EDEVICE. */
int mps_step(mps_ctx* ctx, int32_t nsteps, mps_report* last);

/* Steps 1-4 (and 5) of mps_step at the current state without advancing it: afterwards
 * mps_read_state returns the new p, n* and flags while positions and velocities are
 * unchanged.  Errors as mps_step. */
int mps_solve_ppe(mps_ctx* ctx, mps_report* out);

/* Copy the state to caller buffers in original particle order; any pointer may be NULL.
 * pos, vel: n*dim doubles; p, n_star: n doubles (of the last step or solve; 0 before any;
 * n_star is 0 for DUMMY and GHOST particles, whose own density enters no equation);
 * flags: n bytes, bit 0 = free surface; types: n int8 (GHOST for particles that left). */
int mps_read_state(mps_ctx* ctx, double* pos, double* vel, double* p, double* n_star,
                   uint8_t* flags, int8_t* types);

/* Replace positions, velocities and kinds (original order; vel or types may be NULL to keep
 * them).  Same checks as mps_create.  Used to restart from a saved state: the next PPE solve
 * starts from zero (cg_x0's history is cleared) and p, n* and flags read 0 until the next
 * step.  Writing back, bit for bit, the state the context already holds (for instance a
 * host loop that reads the state after each step and writes it back before the next)
 * changes nothing at all: the call returns without touching the context. */
int mps_write_state(mps_ctx* ctx, const double* pos, const double* vel, const int8_t* types);

/* Clear the PPE initial-guess history (cg_x0): the next solve starts from zero, as after
 * writing a new state.  For callers that replay a trajectory from a saved state and need
 * the replay to repeat the original bit for bit (a checkpointed rollout).  Errors:
 * MPS_EINVAL (NULL). */
int mps_clear_history(mps_ctx* ctx);

/* Set the external acceleration g [m/s^2] (3 doubles; the unused axis of 2D is ignored)
 * for the following steps.  A time-dependent body force -- for instance the inertial
 * acceleration -X''(t) of a tank shaken by X(t), in the tank's frame -- is applied by
 * setting it before each step.  Errors: MPS_EINVAL (NULL or not finite). */
int mps_set_gravity(mps_ctx* ctx, const double* g);

/* ---------------------------------------------------------------- reverse step
 * Vector-Jacobian product of one step (the reverse mode of the step map; the paper has no
 * counterpart).  The step is the map (r^k, u^k, g) -> (r^{k+1}, u^{k+1}) that mps_step
 * would apply to the context's current state.  Its discrete choices are held at their
 * values in that step: neighbour sets, GHOST and free-surface sets (Eq. 15), the clamp's
 * active set and the neighbour giving p_hat_i.  Within them the step is smooth and this
 * is its exact derivative.  The PPE path solves the adjoint system A lam = dL/dp on the
 * step's own symmetric matrix (Eq. 13 as assembled in Listing 2 of Sec. 4.3) with the same
 * solver, precision and cg_tol; the equation-of-state path differentiates Eq. 16.
 *   g_pos, g_vel    dL/dr^{k+1}, dL/du^{k+1}: n*dim doubles each (original order);
 *   out_pos, out_vel dL/dr^k, dL/du^k: n*dim doubles each (caller-allocated);
 *   out_g           dL/dg: 3 doubles (nullable; 0 on the unused axis of 2D);
 *   out_nu          dL/dnu_i: n doubles (nullable; original order), the cotangent of every
 *                   particle's kinematic viscosity in the prediction u* = u + dt (nu_i
 *                   lap(u)_i + g) (Eq. 7): dt lap(u)_i . dL/du*_i for FLUID particles, 0 for
 *                   the others.  With one viscosity for all (params.nu), dL/dnu is their sum.
 * GHOST particles carry their cotangents through, except that a particle turned GHOST
 * by this step (its velocity is reset) gets dL/du^k = 0.
 * The state is not advanced: afterwards positions and velocities are unchanged and
 * mps_read_state returns p, n* and flags of the step (as after mps_solve_ppe).
 * Supported: one scene, kernel 0, gradient_form 0, source_term 0 (one or two phases,
 * either precision, either pressure mode); otherwise MPS_EINVAL.
 * Errors: as mps_step (forward) and MPS_ECG_NOCONV of the adjoint solve. */
typedef struct {
    int32_t status;          /* MPS_OK or the error                                         */
    int32_t cg_iters;        /* adjoint PPE solve: CG iterations (mixed: FP32 inner ones)   */
    int32_t cg_outer;        /* adjoint PPE solve: refinement sweeps                         */
    int32_t pad;
    double cg_resid;         /* adjoint PPE solve: relative residual at exit               */
    mps_report forward;      /* the repeated forward step                                   */
} mps_vjp_report;
int mps_step_vjp(mps_ctx* ctx, const double* g_pos, const double* g_vel, double* out_pos,
                 double* out_vel, double* out_g, double* out_nu, mps_vjp_report* report);

/* Device-memory variants: the same calls with the caller's particle arrays (every pointer
 * argument except out_g and report) in device memory of the context's device, in the same
 * original-order layouts; no host copies are made.  Work runs on the context's stream and
 * the calls are synchronous at return like the host ones.  For callers whose data already
 * lives on the GPU (PyTorch tensors, a rollout's checkpoints). */
int mps_read_state_device(mps_ctx* ctx, double* pos, double* vel, double* p, double* n_star,
                          uint8_t* flags, int8_t* types);
int mps_write_state_device(mps_ctx* ctx, const double* pos, const double* vel, const int8_t* types);
int mps_step_vjp_device(mps_ctx* ctx, const double* g_pos, const double* g_vel, double* out_pos,
                        double* out_vel, double* out_g, double* out_nu, mps_vjp_report* report);

/* Two-phase (multi-density, multi-viscosity) flow of Sec. 3.2.1: a density rho_i [kg/m^3]
 * and a kinematic viscosity nu_i [m^2/s] per particle, n doubles each in the original
 * particle order (copied; the caller keeps its arrays).  NULL leaves that property uniform
 * (params->rho or params->nu); both NULL returns to single-phase flow.  With densities:
 *   equation of state (Eq. 16)   p_i = rho_i c0^2/gamma ((n*_i/n0)^gamma - 1);
 *   pressure correction          u'_i = -(dt/rho_i) grad p_i  (the multi-density pressure
 *                                term, (rho_j/rho_i) alpha_j - alpha_i = (p_j - p_i)/rho_i);
 *   PPE (Eq. 13, Listing 2)      c_ij = 2d/(n0 lambda) * 2/(rho_i + rho_j) * w(r_ij), the
 *                                1/rho of one phase replaced by the pair's mean density;
 * with viscosities the prediction uses the particle's own nu_i.  The properties stay with
 * their particles across steps and mps_write_state.
 * Errors: MPS_EINVAL (a density not finite and > 0, a viscosity not finite and >= 0, or
 * densities with the matrix-free inner operator, ppe_operator 1), MPS_ENOMEM. */
int mps_set_fluid_properties(mps_ctx* ctx, const double* rho, const double* nu);

/* Cell key of every particle at the current positions (original order): the Morton code
 * (x in bit 0) of c = floor((x - box_min)/h) per axis, or 0xFFFFFFFF for a particle outside
 * the grid or a GHOST.  Bit-exact with the floor definition. */
int mps_debug_cells(mps_ctx* ctx, uint32_t* cell_key);

/* Neighbour sets at the current positions through the GPU bucket grid and gather:
 * which = 0: radius re_n, 1: radius re_lap.  j is a neighbour of i iff j != i, neither is a
 * GHOST and ((dx*dx)+(dy*dy))+(dz*dz) < re*re in binary64.  offsets: n+1 int64; ids: cap
 * int32, rows in ascending original id.  If ids is NULL or cap is too small only offsets
 * are written and MPS_ECAP is returned when ids was given. */
int mps_debug_neighbors(mps_ctx* ctx, int32_t which, int64_t* offsets, int32_t* ids,
                        int64_t cap);

/* ---------------------------------------------------------------- batched ensemble
 * Many independent scenes in one context, stepped together by the same kernel launches
 * (the paper runs one scene at a time; this batching has no counterpart there).  Scene s
 * has its own particle spacing l0 and cell grid box, in its own coordinates; the radii
 * scale with l0 (re_n = (params->re_n / params->l0) l0_s, likewise re_lap), and so do
 * lambda, the PPE and Laplacian coefficients and the cell side; every other parameter
 * (dt, rho, nu, g, beta, c0, gamma, alpha_c, tolerances, options) is common.  Particles
 * of different scenes never interact.  Each scene's PPE is solved to cg_tol relative to
 * its own right-hand side (one CG over the block-diagonal system, stopped when every
 * scene meets its tolerance).  A step fails with MPS_ESKIN if any particle moves more
 * than s max(re)/2 of the scene with the smallest spacing. */
typedef struct {
    double l0;          /* particle spacing [m] */
    double box_min[3];  /* cell grid origin of the scene [m] (its own coordinates) */
    double box_max[3];  /* cell grid extent: outside -> GHOST, as in mps_params */
} mps_scene;

/* pos, vel, types as mps_create; scene: n scene indices in [0, n_scenes).  params->box_*
 * are ignored.  mps_debug_cells / mps_debug_neighbors are not available on an ensemble
 * (MPS_EINVAL); everything else is.
 * Errors: as mps_create, and MPS_EINVAL for n_scenes < 1 or > 65535, a scene index out of
 * range, or a scene with l0 <= 0 or an empty box. */
int mps_create_ensemble(const double* pos, const double* vel, const int8_t* types,
                        const int32_t* scene, int64_t n, const mps_params* params,
                        const mps_scene* scenes, int32_t n_scenes, mps_ctx** out);

/* Autotuning (a tool of this library; the paper has none): times the launch shapes and the
 * inner solver's form on the current state with CUDA events on the context's stream
 * (`repeats` timed runs each after one untimed run) and keeps the fastest:
 *   - after at least one step, the cell side h = max(re)(1 + s) (Sec. 4.1's bucket size):
 *     the cell skin s among 0.05, 0.1, 0.15, 0.2, 0.3 and the context's own, no smaller
 *     than twice the candidate-list skin the last step's motion asked for, timed as a
 *     bucket build plus a candidate gather; the grid (cells per axis, cell table, candidate
 *     list capacity) is derived again for each, and afterwards params.cell_skin is the
 *     chosen s (so a step's MPS_ESKIN limit is s max(re)/2 of that s);
 *   - the candidate gather's cell block: 32, 64, 96 or 128 threads (params.gather_block);
 *   - the prediction's threads per FLUID row: 1, 2 or 4 (each takes every 2nd or 4th
 *     candidate of the row's list; the row's sums are added across them);
 *   - the row build's block: 64, 128 or 256 threads (params.build_block);
 *   - mixed PPE only, on the system of a solve at the current state: the FP32 SpMV's block,
 *     256 or 512 threads, and the inner CG as three kernels per iteration (SpMV; x, r
 *     update; direction update) or two (the recurrences of Chronopoulos and Gear: SpMV of
 *     the residual; one pass updating direction, A-direction, x and r), the latter for the
 *     device-driven solve only, with 1, 2 or 4 inner iterations per pass of the solve's
 *     conditional loop (params.cg_unroll).
 * Neighbour sets and the solve's stop rule are the same whatever the choice; the fused CG,
 * and another cell side (its candidates come in another order), round differently, so a
 * solve's result changes within its tolerance.  Afterwards the
 * state is reordered as by a step's bucket build and p, n* and flags are those of a solve at
 * the current state (positions and velocities are not advanced).  *out (nullable) receives
 * the choice and its times.  Errors: MPS_EINVAL (repeats < 1), MPS_ENOMEM (the cell table
 * or candidate lists of another cell side; the context keeps its cells then), MPS_EDEVICE,
 * and the errors of the solve. */
typedef struct {
    int32_t gather_block;   /* threads per cell block of the candidate gather                */
    int32_t spmv_block;     /* threads per block of the FP32 SpMV of the mixed inner CG      */
    int32_t cg_fused;       /* 1: the inner CG in two kernels per iteration, 0: three        */
    int32_t build_block;    /* threads per block of the row build                            */
    int32_t cg_unroll;      /* inner CG iterations per pass of the solve's conditional loop   */
    int32_t predict_tpr;    /* threads per FLUID row of the prediction                        */
    double gather_ms;       /* the chosen gather's time [ms]                                 */
    double spmv_ms;         /* the chosen SpMV's time [ms] (0 without a mixed PPE)            */
    double solve_ms;        /* a mixed solve's time with the chosen form [ms] (0 without)     */
    double build_ms;        /* the chosen row build's time [ms]                              */
    double cell_skin;       /* the chosen cell skin s (cell side h = max(re)(1 + s))         */
    double cell_ms;         /* bucket build + candidate gather with the chosen cells [ms]    */
    double predict_ms;      /* the chosen prediction's time [ms]                             */
} mps_tuning;
int mps_autotune(mps_ctx* ctx, int32_t repeats, mps_tuning* out);

/* Relative PPE residual ||b_s - A_s p_s|| / ||b_s|| of every scene after the last step
 * (n_scenes doubles; 0 for a scene with b_s = 0); a single-scene context writes one. */
int mps_scene_residuals(mps_ctx* ctx, double* out);

/* Derived constants: out[0] n0 at re_n, out[1] n0 at re_lap, out[2] lambda [m^2],
 * out[3] cell side h [m], out[4] cells per axis x, out[5] y, out[6] z, out[7] nbr_cap. */
int mps_get_constants(mps_ctx* ctx, double* out);

/* Stage timers (CUDA events recorded on the context's stream around each stage of a step)
 * and a count of the kernel launches the context issued.  Stages: */
#define MPS_STAGE_BUCKET 0   /* cell keys, radix sort, cell table, permutation        */
#define MPS_STAGE_GATHER 1   /* candidate lists from the cell grid (one kernel)       */
#define MPS_STAGE_PREDICT 2  /* viscosity + gravity prediction (one kernel)           */
#define MPS_STAGE_BUILD 3    /* number density, flags, PPE rows, lists (one kernel)   */
#define MPS_STAGE_PPE 4      /* CG solve (includes the host's convergence polls)      */
#define MPS_STAGE_UPDATE 5   /* clamp, minimum pressure, gradient correction          */
#define MPS_NSTAGES 6
/* on != 0 enables the stage timers (off by default) and resets timers and counter. */
int mps_set_profiling(mps_ctx* ctx, int32_t on);
/* stage_ms[MPS_NSTAGES]: accumulated milliseconds; stage_calls[MPS_NSTAGES]: stages timed;
 * launches: kernels launched since the last reset.  Any pointer may be NULL. */
int mps_get_profile(mps_ctx* ctx, double* stage_ms, int64_t* stage_calls, int64_t* launches);

/* Kernel timing (a tool of this library): after a step or solve of a PPE context, launch
 * one kernel of the PPE solve `repeats` times on the system that step built (CUDA events
 * on the context's stream, one launch at a time) and report its mean duration [ms] and its
 * algorithmic bytes per launch (per row of the system the stored coefficients and the
 * row's own vector entries, per other row its diagonal read and output write; gathers of
 * neighbour entries, which stay in cache, are not counted).  Only scratch vectors change:
 * the state, p, n* and flags stay as the step left them.
 *   MPS_KERNEL_SPMV32   the FP32 SpMV of the mixed inner CG (column + FP32 value: 8 B per
 *                       coefficient);
 *   MPS_KERNEL_RESID_FF the mixed float-float residual (12 B per coefficient);
 *   MPS_KERNEL_SPMV64   the FP64 SpMV (12 B per coefficient).
 * Errors: MPS_EINVAL (equation-of-state context, repeats < 1, or a kernel of the other
 * precision), MPS_EDEVICE. */
#define MPS_KERNEL_SPMV32 0
#define MPS_KERNEL_RESID_FF 1
#define MPS_KERNEL_SPMV64 2
int mps_time_kernel(mps_ctx* ctx, int32_t which, int32_t repeats, double* ms_per_launch,
                    double* bytes_per_launch);

/* Measured arithmetic peak of a device (a measuring tool of this library; the paper has no
 * counterpart): the pair sums of the step are bound by FP32 arithmetic in the mixed path
 * and by FP64 arithmetic in the FP64 path, and their rooflines are taken against these
 * rates.  Launches `repeats` timed kernels (after two untimed ones) of independent chains
 * of fused multiply-adds over whole waves of the device's SMs, timed with CUDA events on
 * `stream` (cudaStream_t, NULL: the legacy default stream), and returns the rate in
 * TFLOP/s (one fused multiply-add = 2 flops) and the mean launch time [ms] (nullable).
 *   MPS_PEAK_FFMA   scalar FP32 FFMA;
 *   MPS_PEAK_FFMA2  packed two-lane FP32 FFMA (one instruction, two fused multiply-adds);
 *   MPS_PEAK_DFMA   FP64 DFMA.
 * The device is made current for the call and the previous one restored.  Synchronous.
 * Errors: MPS_EINVAL (unknown `which`, repeats < 1, tflops NULL), MPS_EDEVICE (a CUDA call
 * failed, or a launch error was already pending on entry, which is left pending). */
#define MPS_PEAK_FFMA 0
#define MPS_PEAK_FFMA2 1
#define MPS_PEAK_DFMA 2
int mps_measure_peak(int32_t device, int32_t which, int32_t repeats, void* stream, double* tflops,
                     double* ms_per_launch);

/* Solve A x = b by FP64 conjugate gradients WITHOUT ALLOCATING any memory.
 * No counterpart in the paper: this is an entry point for callers that are not allowed to
 * call cudaMalloc -- for instance a host application whose device memory is entirely
 * managed by its own pool and that forbids other allocators, or a real-time loop where
 * cudaMalloc/cudaFree (which can synchronise the device and take milliseconds) are off
 * limits after start-up.  Such a caller passes its own inputs and outputs; the CG's scratch
 * vectors, partial sums and scalars live in one fixed array of device memory that belongs
 * to the loaded library (about 6.3 MB on every GPU that loads it, held until process exit).
 *
 * The system uses the row layout of the library's PPE operator:
 *   (A x)_i = diag[i] x_i - sum_{k < cnt[i]} val[i*cap + k] x[col[i*cap + k]]  if diag[i] != 0,
 *   and rows with diag[i] == 0 are outside the system (x_i = 0, b_i must be 0).
 * A must be symmetric positive definite on its rows.  col, cnt, val, diag, b and x are
 * device pointers owned by the caller (col/val: n*cap entries, the others n); x is
 * overwritten with the solution.  CG starts from x = 0 and stops when the recomputed true
 * residual satisfies ||b - A x|| <= tol ||b|| (restarting from it if the recurrence drifted,
 * at most 30 times), or with MPS_ECG_NOCONV after max_iter iterations in total (<= 0: 10 n)
 * or 30 restarts (a tol below what FP64 can attain on the system).
 * A CUDA launch error already pending in the calling thread on entry is reported as
 * MPS_EDEVICE and left pending (not cleared) for its owner; nothing is launched then.
 * stream: cudaStream_t (NULL: the legacy default stream); the call is synchronous.
 * iters_out, resid_out (nullable): iterations and final relative residual.
 * Limits: 1 <= n <= MPS_NOALLOC_MAX_ROWS, else MPS_EINVAL.
 * Every call shares the one scratch array of the current device: two calls whose work
 * overlaps on a GPU (different streams, threads or processes sharing the library instance)
 * race and corrupt each other; serialise them.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Calls no cudaMalloc, cudaFree or allocating library
 * routine. */
#define MPS_NOALLOC_MAX_ROWS 262144
int mps_ppe_cg_noalloc(int64_t n, int32_t cap, const int32_t* col, const int32_t* cnt,
                       const double* val, const double* diag, const double* b, double* x,
                       double tol, int32_t max_iter, void* stream, int32_t* iters_out,
                       double* resid_out);

/* Release every device buffer and the owned stream.  NULL is ignored. */
void mps_destroy(mps_ctx* ctx);

/* Static string naming a status code. */
const char* mps_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif
