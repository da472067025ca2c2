/*
 * lbm.h -- C ABI of the GB300 (sm_103a) implementation of the per-time-step
 * fused collide-and-stream update of the coupled central-moment lattice
 * Boltzmann system of Elbousefi, Schupbach, Premnath & Welch, "Investigation
 * of Surfactant-Laden Bubble Migration Dynamics in Self-Rewetting Fluids
 * using Lattice Boltzmann Method" (arXiv 2408.00146).
 *
 * One simulation ("sim") evolves four D2Q9 distributions on an nx x ny
 * lattice: f (conservative Allen-Cahn phase field, App. B), g (pressure-based
 * two-fluid flow with capillary and Marangoni forces, App. C), h (energy,
 * App. D) and q (surfactant, App. E), coupled through the surface-tension
 * law sigma(T, psi) of Eq. (6) and the isotropic finite-difference stencils
 * of Sec. 3.
 *
 * Geometry: x is periodic.  With walls != 0, rows y = 0 and y = ny-1 are solid
 * (halfway bounce-back for f, g and, by default, q; anti-bounce-back Dirichlet
 * temperature T_H at y = 0 and T_C at y = ny-1 for h, and for q when psi is
 * held at psi_L / psi_R, see psi_bc) and rows 1..ny-2 are fluid; with
 * walls == 0, y is periodic too.  phi = 0 is the ambient fluid A, phi = 1
 * the bubble B (Sec. 3).
 *
 * Conventions for every call:
 *   - every entry point returns an lbm_status; nothing aborts or exits;
 *     on failure lbm_last_error() returns a message for the calling thread;
 *   - host pointers are read or written before the call returns (the call
 *     synchronises the sim's stream where it touches host memory); the
 *     caller keeps ownership of every buffer it passes;
 *   - device work is issued on the CUDA stream given to lbm_create; calls on
 *     one sim must not run concurrently from several threads.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sim lbm_sim;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,    /* invalid argument or parameter out of range       */
    LBM_ENOMEM = -2,    /* device or host allocation failed / too small     */
    LBM_ECUDA = -3,     /* a CUDA runtime call failed                       */
    LBM_EUNSTABLE = -4, /* a NaN or Inf was found by lbm_observe            */
    LBM_ETIMEOUT = -5,  /* reserved: a bounded device wait gave up          */
    LBM_ESTATE = -6     /* call out of order (e.g. lbm_step before init)    */
} lbm_status;

/* Population storage precision (lbm_params.precision).  The arithmetic is
 * FP32 in every mode; the paper fixes no storage format (its method is stated
 * in exact arithmetic).
 *   LBM_FP32: the 36 populations of each node in FP32 (144 B per node and
 *     buffer).
 *   LBM_FP16, LBM_BF16: per node, m = M/36 in FP32 for the zeroth moments
 *     M = (M_f, M_g, M_h, M_q) of the populations it pushed at the last step
 *     (16 B), and per population its deviation from k_a m of the node that
 *     pushed it (the source y - e_a, or the node itself for a population that
 *     bounced back), stored in IEEE binary16 or bfloat16 (72 B per node and
 *     buffer; the sets in pairs, (f, g) and (h, q), the two deviations of a
 *     population side by side in one 32-bit word); k_a = 36 w_a = 16, 4, 1
 *     are exact integer weights.  The rest
 *     part carries the conserved scalars phi, T, psi in FP32; the rounding
 *     errors of the nine deviations a node pushes are folded into its m, so
 *     the populations it pushes sum to their FP32 values.  Populations at the
 *     API (lbm_init, lbm_get_populations) stay FP32 arrays. */
enum { LBM_FP32 = 0, LBM_FP16 = 1, LBM_BF16 = 2 };

/* Problem parameters, named as in the paper's problem statement (Sec. 2,
 * Sec. 6).  Lattice units throughout.  The lattice parameters derived from
 * them are listed under lbm_get_derived. */
typedef struct {
    int32_t nx, ny;        /* lattice size; nx periodic axis, ny wall-bounded  */
    int32_t walls;         /* 1: solid rows y=0, ny-1; 0: periodic y            */
    double R;              /* bubble radius (length scale of Eq. (8), Eq. (21)) */
    double xb, yb;         /* bubble centre, used by the analytic initial state */
    double W;              /* interface width (Sec. 3)                          */
    double M_phi;          /* ACE mobility, Eq. (12); omega_phi by App. B       */
    double rho_A;          /* ambient density                                   */
    double rho_ratio;      /* rho_A / rho_B, Eq. (9)                            */
    double mu_ratio;       /* mu_A / mu_B, Eq. (9)                              */
    double alpha_ratio;    /* alpha_A / alpha_B (thermal diffusivities)         */
    double Re, Ma;         /* Eq. (8) with U = U_o of Eq. (21)                  */
    double sigma0;         /* surface tension at T_ref, clean interface, Eq. (6)*/
    double sigma_T;        /* linear sensitivity, Eq. (6) (normal fluids)       */
    double sigma_TT;       /* quadratic sensitivity, Eq. (6) (self-rewetting)   */
    double T_ref;          /* reference temperature, Eq. (6)                    */
    double T_H, T_C;       /* wall temperatures at y = 0 and y = ny-1           */
    double beta;           /* Gibbs elasticity, Eq. (6)-(7)                     */
    double Pi, Ex;         /* surfactant groups defined after Eq. (11)          */
    double M_psi;          /* surfactant diffusivity of the q scheme (App. E)   */
    double psi0;           /* uniform initial surfactant (analytic init)        */
    double Fext_x, Fext_y; /* uniform external body force F_ext (Eq. (14))      */
    double gravity;        /* buoyancy -(rho - rho_A) g along y (Sec. 5.3)      */
    double nu_A;           /* > 0: ambient kinematic viscosity given directly   */
    double alpha_A;        /* > 0: ambient thermal diffusivity given directly   */
    int32_t precision;     /* LBM_FP32, LBM_FP16 or LBM_BF16 (storage, above)   */
    double psi_L, psi_R;   /* surfactant at the y=0 and y=ny-1 ends, in [0, 1)  */
    int32_t psi_bc;        /* walls for psi (Sec. 2, Sec. 6): 0 zero flux (halfway
                              bounce-back for q) and uniform initial psi0; 1 psi
                              held at psi_L, psi_R on the wall planes (anti-
                              bounce-back for q with 2 w_a psi_w, stencil ghosts
                              odd about psi_w), the paper's main cases; 2 zero
                              flux with psi_L -> psi_R only as the linear
                              initial profile (the variant at the end of
                              Sec. 6).  1 and 2 set the analytic initial psi
                              linear between the wall planes.  Needs walls = 1
                              to have an effect.                               */
} lbm_params;

/* Observables (Sec. 5.3, Sec. 6): phi-weighted bubble centroid ("mass
 * center") and migration velocity ("average velocity inside the bubble"),
 * phase-field and surfactant masses, reduced in FP64 over fluid nodes. */
typedef struct {
    double t;         /* time steps taken since lbm_init                       */
    double mass_phi;  /* sum of phi                                            */
    double mass_psi;  /* sum of psi                                            */
    double xc, yc;    /* sum(phi x)/sum(phi), sum(phi y)/sum(phi)              */
    double ux_bub;    /* sum(phi u_x)/sum(phi)                                 */
    double uy_bub;    /* sum(phi u_y)/sum(phi)                                 */
    double U_o;       /* characteristic thermocapillary velocity, Eq. (21)     */
    double t_star;    /* t U_o / R                                             */
    int32_t nan_flag; /* number of fluid nodes with a non-finite field value   */
} lbm_obs;

/* Number of doubles written by lbm_get_derived, in this order:
 * dT, M1, M2, L, U_o, rho_A, rho_B, mu_A, mu_B, nu_A, nu_B, alpha_A, alpha_B,
 * omega_phi, omega_psi, lambda, s, w, m_psi, D_psi. */
#define LBM_NDERIVED 20

/* Validates p and writes the LBM_NDERIVED lattice parameters listed above
 * without creating a sim (host only; no CUDA call).  Errors: LBM_EINVAL. */
lbm_status lbm_derive(const lbm_params* p, double* out);

/* Bytes of device workspace one sim needs (two population buffers -- 36
 * floats per node for LBM_FP32; 36 16-bit deviations and 4 floats per node for
 * LBM_FP16/LBM_BF16 -- one field buffer of 6 floats per node, reduction
 * scratch).  Errors: LBM_EINVAL for invalid parameters. */
lbm_status lbm_workspace_bytes(const lbm_params* p, size_t* bytes);

/* Creates a sim and allocates its device workspace with cudaMalloc on the
 * current device.  stream: a cudaStream_t, or NULL for the default stream.
 * The parameters are validated and the lattice parameters derived as in
 * Sec. 2 and Sec. 6 (Eqs. (8)-(10), (21); App. B-E relaxation rates); every
 * relaxation rate must lie in (0, 2), nx >= 4, ny >= 5 with walls (4
 * without).  Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_create(const lbm_params* p, void* stream, lbm_sim** out);

/* As lbm_create, but the caller supplies the device workspace: a pointer
 * into device memory of at least lbm_workspace_bytes() bytes, 256-byte
 * aligned, that stays valid and untouched by the caller until lbm_destroy.
 * The sim never frees it.  Errors: as lbm_create; LBM_ENOMEM if bytes is too
 * small. */
lbm_status lbm_create_ex(const lbm_params* p, void* stream, void* workspace,
                         size_t workspace_bytes, lbm_sim** out);

/* Sets the state at t = 0.
 *   populations != NULL: host float array [4][9][ny][nx] (sets f, g, h, q;
 *     directions in the order e_0..e_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),
 *     (1,1),(-1,1),(-1,-1),(1,-1); wall rows are ignored), copied as the
 *     post-streaming populations of t = 0 (16-bit storage: each node's M is
 *     set to the sums of its own nine populations, and the deviations are
 *     rounded from the given values);
 *   else fields != NULL: host double array [6][ny][nx] of phi, u_x, u_y, p,
 *     T, psi; every population is set to the equilibrium of App. B-E built
 *     from these fields (n and R from the isotropic stencils of phi);
 *   else: the analytic state of Sec. 2 -- bubble of radius R at (xb, yb) with
 *     the tanh profile of Sec. 3, fluid at rest (p = 0), T linear from T_H
 *     on the plane y = 1/2 to T_C on y = ny - 3/2 (T_ref without walls),
 *     psi = psi0 (or the psi_L -> psi_R profile, see psi_bc), then the
 *     equilibria as above.
 * Errors: LBM_EINVAL (NULL sim), LBM_ECUDA. */
lbm_status lbm_init(lbm_sim* sim, const double* fields, const float* populations);

/* Advances nsteps time steps: each is one launch of a fused kernel that
 * reads the populations, builds phi, T, psi, p* and the forces of Sec. 3 and
 * App. C from them with the isotropic stencils (a two-node halo), collides f,
 * g, h, q (App. B-E) and streams the results to the neighbours (Eqs. (27)-(28),
 * (33)-(34), (38)-(39), (43)-(44)).  Lattices with nx >= 32, nx a multiple of
 * 4 (FP32) or 8 (16-bit storage), at least 16 fluid rows and walls (or, FP32,
 * a periodic y axis of whole 8-row chunks) take the streaming kernels (see
 * lbm_batch_plan); the others a tile kernel.  Asynchronous on the sim's
 * stream; long runs replay a captured CUDA graph.  nsteps = 0 is a no-op.
 * Errors: LBM_EINVAL (nsteps < 0), LBM_ESTATE (not initialised), LBM_ECUDA. */
lbm_status lbm_step(lbm_sim* sim, int64_t nsteps);

/* Advances n simulations (1 <= n <= 64) by nsteps time steps with one kernel
 * launch per step and kernel family: the streaming kernel of each storage
 * precision (at most 48 16-bit sims per launch) and the tile kernel of each
 * precision, each launch covering all the sims it takes; the simulations may
 * differ in size, parameters and precision.  Each step is the same fused update as
 * lbm_step, so the result of every simulation equals what lbm_step gives it
 * alone.  All sims must be initialised, distinct, and created on the same
 * device and stream; the launches are issued on that stream (asynchronous)
 * and counted by lbm_launch_count of sims[0].  Every 64 steps of a call, and
 * a remaining run of 8 to 63 steps, replay a CUDA graph of that many steps,
 * captured on first use and cached per host thread for that list of sims,
 * their current buffers, the strip plan and the step count (8 graphs; a
 * destroyed sim's graphs are never replayed); a remainder under 8 steps is
 * launched step by step.  Errors: LBM_EINVAL, LBM_ESTATE, LBM_ECUDA. */
lbm_status lbm_step_batch(lbm_sim* const* sims, int32_t n, int64_t nsteps);

/* Strip plan of a batch.  Sims eligible for the streaming kernels (see
 * lbm_step) are stepped by blocks of 256 threads that each walk one column of
 * up to W nodes over a strip of chunks of H rows, in one of two compiled tile
 * shapes W x H: 32 x 8, or 64 x 4 for FP32 storage (lbm_batch_tiles).  strip_chunks[i]
 * (caller's array of n) receives the strip length, in chunks, that
 * lbm_step_batch uses for sims[i] in this batch (0 for sims stepped by a tile
 * kernel).  Without tuning it comes from a cost model of each streaming
 * launch in the 32 x 8 shape (one strip per block slot, resident blocks x SMs
 * slots, longest first).  Host only; arguments as lbm_step_batch.  The
 * paper has no counterpart (it fixes no GPU work decomposition).  Errors:
 * LBM_EINVAL, LBM_ESTATE. */
lbm_status lbm_batch_plan(lbm_sim* const* sims, int32_t n, int32_t* strip_chunks);

/* Tile shape of the batch's plan: tile_w[i] and tile_h[i] (caller's arrays of
 * n; either may be NULL) receive the column width W and chunk height H of the
 * streaming launch that steps sims[i] (0 for sims stepped by a tile kernel).
 * Every sim of one streaming launch has the same shape.  Host only;
 * arguments as lbm_step_batch.  The paper has no counterpart.  Errors:
 * LBM_EINVAL, LBM_ESTATE. */
lbm_status lbm_batch_tiles(lbm_sim* const* sims, int32_t n, int32_t* tile_w, int32_t* tile_h);

/* Sets the plan of a batch, as lbm_tune_batch would after measuring it:
 * tile_w[i] (32, or 64 for FP32 storage) and strip_chunks[i] (>= 4 chunks) for every sim the
 * streaming kernels step (entries of the others are ignored); the sims of one
 * streaming launch (one storage precision, see lbm_step_batch) must share a
 * tile width.  Kept for later lbm_step_batch calls on sims of the same sizes
 * in the same order on this host thread.  The result of a step does not
 * depend on the plan.  Host only.  The paper has no counterpart.  Errors:
 * LBM_EINVAL (NULL arrays, unknown width, strip_chunks < 4, mixed widths in
 * one launch, batch arguments), LBM_ESTATE. */
lbm_status lbm_pin_batch_plan(lbm_sim* const* sims, int32_t n, const int32_t* tile_w,
                              const int32_t* strip_chunks);

/* Measured choice of the strip plan of a batch (autotuner).  For each
 * distinct plan among the tile shapes and candidate strip lengths (the cost
 * model's first),
 * advances the whole batch trial_steps steps and times them with CUDA events
 * on the batch's stream; the fastest plan is kept and used by later
 * lbm_step_batch calls on sims of the same sizes in the same order, on this
 * host thread (a plan cache of 16 size lists; tuned plans are evicted last).
 * The trial steps are real steps: a step's result does not depend on the
 * plan, so every sim advances *steps_taken steps (1 untimed warm-up step +
 * trial_steps per candidate), as if by lbm_step_batch; on failure it still
 * counts the steps taken.  A batch with no streaming sim takes no step.  Uses
 * the caller's current device, as every call does.  Synchronises the stream.
 * The paper has no counterpart.  Errors: LBM_EINVAL (trial_steps < 1, steps_taken NULL, batch
 * arguments), LBM_ESTATE, LBM_ECUDA. */
lbm_status lbm_tune_batch(lbm_sim* const* sims, int32_t n, int32_t trial_steps,
                          int64_t* steps_taken);

/* Computes the observables of the current state (out may be NULL) and, if
 * host_fields != NULL, copies the macroscopic fields phi, u_x, u_y, p, T, psi
 * into the host double array [6][ny][nx] (wall rows set to 0).  Synchronises
 * the stream.  Errors: LBM_ESTATE, LBM_ECUDA, LBM_EUNSTABLE if a non-finite
 * value was found (out and host_fields are still written). */
lbm_status lbm_observe(lbm_sim* sim, lbm_obs* out, double* host_fields);

/* Observables of several simulations with one wait, for serving loops that
 * keep the GPU busy while they read results.  lbm_observe_enqueue enqueues,
 * for each of sims[0..n-1] (1 <= n <= 64; distinct, initialised, one device
 * and stream, as lbm_step_batch), the evaluation lbm_observe performs -- the
 * fields of the current state, the FP64 reductions, and the copy of their
 * result into the sim's pinned host buffer -- and returns without waiting;
 * later work on the stream (further steps) does not change the result.
 * lbm_observe_collect waits for those evaluations and writes out[i] (caller's
 * array of n) for sims[i], with t the step count at enqueue time; status
 * (caller's array of n, may be NULL) receives each sim's lbm_observe status
 * (LBM_OK, LBM_EUNSTABLE, LBM_ETIMEOUT).  A second enqueue before the collect
 * replaces the first.  The paper has no counterpart.
 * Errors: LBM_EINVAL, LBM_ESTATE (collect without an enqueued evaluation),
 * LBM_ECUDA. */
lbm_status lbm_observe_enqueue(lbm_sim* const* sims, int32_t n);
lbm_status lbm_observe_collect(lbm_sim* const* sims, int32_t n, lbm_obs* out, int32_t* status);

/* Copies the current post-streaming populations into the host float array
 * [4][9][ny][nx] (the layout lbm_init accepts back: checkpoint/restart; wall
 * rows hold 0).  16-bit storage: the populations are rebuilt as
 * k_a m(source) + deviation in FP32.  Synchronises the stream.  Errors:
 * LBM_ESTATE, LBM_ECUDA. */
lbm_status lbm_get_populations(lbm_sim* sim, float* host_pops);

/* Writes the LBM_NDERIVED lattice parameters listed above.  Errors:
 * LBM_EINVAL. */
lbm_status lbm_get_derived(const lbm_sim* sim, double* out);

/* Number of kernel launches this sim has issued since creation (every
 * launch, including those replayed inside CUDA graphs). */
int64_t lbm_launch_count(const lbm_sim* sim);

/* Frees the sim and, for lbm_create, its workspace.  NULL is a no-op. */
void lbm_destroy(lbm_sim* sim);

/* Message describing the last failure on the calling thread ("" if none). */
const char* lbm_last_error(void);

/* Diagnostic of the failure path of the kernels' waits: launches one block
 * that waits, with the same bounded wait the step kernels use for their tile
 * copies, on a barrier that nothing ever completes, giving up after limit_ns
 * nanoseconds of wall time (0 < limit_ns <= 1e10; the step kernels use 1 s).
 * *gave_up = 1 when the block abandoned the wait and returned -- what lets a
 * step whose copy never lands report LBM_ETIMEOUT through lbm_observe instead
 * of hanging the GPU -- and 0 otherwise.  Uses the current device and default
 * stream and synchronises it.  The paper has no counterpart.
 * Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_probe_bounded_wait(int64_t limit_ns, int32_t* gave_up);

/* FP64 observable sums over the fluid nodes of a caller-provided device field
 * array, for callers that cannot allocate device memory where they call it:
 * code recording a stream into a CUDA graph, latency-critical loops that must
 * not take the device-wide synchronisation of cudaMalloc/cudaFree, and hosts
 * whose device memory is fully budgeted in advance.  The paper has no
 * counterpart: it is plumbing around the reduction lbm_observe performs.
 *   d_fields: device float array [6][ny][nx] (phi, u_x, u_y, p, T, psi; the
 *     layout lbm_observe copies out), read only; with walls != 0 rows 0 and
 *     ny-1 are skipped.
 *   d_sums: device double array of 8, written: sum phi, sum psi, sum phi x,
 *     sum phi y, sum phi u_x, sum phi u_y, number of nodes holding a
 *     non-finite value, number of fluid nodes.
 *   stream: cudaStream_t (NULL = default stream); the call only enqueues two
 *     kernels and returns without synchronising.
 * No allocation: the block partial sums live in a fixed 256 KiB array inside
 * the library's device image, present on every device that loads the
 * library until the process exits.  That caps the lattice at 16,777,216
 * fluid nodes; larger ones return LBM_EINVAL with a message saying so.  The
 * first call on a device looks the array's device address up (a host-side
 * runtime query, no allocation); make that first call before any stream
 * capture.  Every call shares the one array, so calls whose kernels overlap
 * on the GPU (different streams without ordering) race and return garbage;
 * order them on one stream or with events.  Each call writes every partial
 * it reads, so nothing has to be cleared between calls.
 * Errors: LBM_EINVAL, LBM_ECUDA (message in lbm_last_error()). */
lbm_status lbm_reduce_observables_noalloc(const float* d_fields, int32_t nx, int32_t ny,
                                          int32_t walls, double* d_sums, void* stream);

#ifdef __cplusplus
}
#endif
#endif
