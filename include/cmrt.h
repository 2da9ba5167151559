/*
 * libcmrt -- two-colour D2Q9 chromodynamic multi-relaxation-time lattice
 * Boltzmann step on NVIDIA GB300 (sm_103a).
 *
 * Method: J. Spendlove, X. Xu, O. J. Halliday, T. Schenkel, I. Halliday,
 * "Chromodynamic multi-relaxation time lattice Boltzmann scheme for fluids
 * with density difference", arXiv 2005.04642.
 *
 *   Sec. 2   two-colour populations R_i, B_i, density-contrast equilibrium
 *            (Eqs. equ_equ, eq_phi), colour index (Eq. equ_rhoN_def),
 *            Lishchuk force G = sigma K grad(rho^N) / 2 (Eq. equ_stforce),
 *            force-adjusted velocity (Eq. equ_u_def), d'Ortona recolour
 *            (Eq. eq_re_color), streaming (Eq. equ_evolution).
 *   Sec. 3 / App. A   Dellar MRT collision in moment space: modes m = M f,
 *            equilibria h^(p).f^(0), sources S^(p) from F_1 + F_2 with the
 *            correction tensor C (Eq. Correction), forced scalar relaxation
 *            (Eq. 38) and explicit reconstruction f+ = M^{-1} m+.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Lattice nx * ny, x fastest: a field is float[ny][nx] (row-major).
 * - Link order: i = 0 rest; i = 1..8 counter-clockwise from (1, 1), so odd i
 *   are the diagonal ("longer") links: 1 (1,1) 2 (0,1) 3 (-1,1) 4 (-1,0)
 *   5 (-1,-1) 6 (0,-1) 7 (1,-1) 8 (1,0).
 * - Population arrays are float[2][9][ny][nx]: colour (0 = red, 1 = blue),
 *   link, row, column.
 * - x is periodic.  y is periodic (wall_y = 0) or bounded by half-way
 *   bounce-back walls at y = -1/2 and y = ny - 1/2 (wall_y = 1).
 * - Every pointer argument may point to host memory or to device memory of
 *   the context's device; the library detects which (cudaPointerGetAttributes).
 *   Page-locked host memory mapped for the device is read and written by the
 *   kernels in place; other host memory is copied through the state buffer
 *   that does not hold the current state (dead between steps) or, where that
 *   is too small, through the library's own staging buffer.  The
 *   caller owns every buffer it passes; the library owns everything it
 *   allocates and frees it in cmrt_destroy.
 * - Calls are asynchronous on the context's stream unless stated; a call
 *   that reads results into host memory synchronises that stream.
 * - No call aborts or throws.  Each returns a cmrt_status; the message of the
 *   last failure is available from cmrt_last_error.  After CMRT_ECUDA or
 *   CMRT_ENONFINITE a context is failed: every later call on it except
 *   cmrt_last_error and cmrt_destroy returns CMRT_ESTATE.
 * - A context is used from one host thread at a time.
 */
#ifndef CMRT_H
#define CMRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Raised whenever cmrt_params changes layout or a call is added or changes
 * meaning; bindings check it (cmrt_abi_version) before use.  6: per-context
 * step graphs (cmrt_set_graph_steps, cmrt_get_graph_steps).  7: checkpoint
 * and restart (cmrt_save_bytes, cmrt_save, cmrt_load).  8: precision_reference
 * 0 is the node-mixture reference, the pure-colour one moved to 2.  9: the
 * 16-bit record carries reference dipoles and the rest populations (64 B/node).
 * 10: each 16-bit record carries its reference shape (a flag in D_0). */
#define CMRT_ABI_VERSION 10

typedef struct cmrt_ctx cmrt_ctx;     /* opaque, owned by the library */
typedef struct cmrt_batch cmrt_batch; /* opaque, owned by the library */

typedef enum {
    CMRT_OK = 0,
    CMRT_EINVAL = 1,     /* bad parameter, size or pointer                      */
    CMRT_ENOMEM = 2,     /* device or host allocation failed                    */
    CMRT_ECUDA = 3,      /* a CUDA runtime call failed (message has the reason) */
    CMRT_ENONFINITE = 4, /* a non-finite density appeared in the state          */
    CMRT_ESTATE = 5,     /* context already failed, or NULL context             */
    CMRT_ETIMEOUT = 6    /* a bounded device-side wait gave up                  */
} cmrt_status;

/* Parameters of the scheme (Sec. 2, Sec. 3, App. A).  Fill with
 * cmrt_params_default, then override. */
typedef struct {
    int32_t nx, ny;          /* lattice size, each >= 1                                         */
    int32_t wall_y;          /* 0: periodic in y; 1: half-way bounce-back walls in y             */
    double rho0_r, rho0_b;   /* bulk densities; Lambda = rho0_r / rho0_b (Eq. equ_fred)         */
    double alpha_r, alpha_b; /* rest fractions in phi_i (Eq. eq_phi); must satisfy
                                (1 - alpha_b) / (1 - alpha_r) = Lambda to 1e-9 relative         */
    double sigma;            /* interfacial tension in G = sigma K grad(rho^N) / 2 (Eq. equ_stforce) */
    double beta;             /* segregation parameter of the recolour (Eq. eq_re_color)         */
    double lambda3_r;        /* shear eigenvalue of pure red, in (0, 2): nu = (2/lambda3 - 1)/6   */
    double lambda3_b;        /* shear eigenvalue of pure blue                                    */
    double lambda6;          /* ghost eigenvalue of N, in (0, 2] (default 1)                     */
    double lambda7;          /* ghost eigenvalue of J_x, J_y, in (0, 2] (default 1, Sec. 4)       */
    double g_acc[2];         /* body acceleration: adds rho * g_acc to G                          */
    double g_vol[2];         /* force per unit volume: adds g_vol to G (App. D pressure gradient) */
    int32_t visc_mode;       /* 0: nu linear in rho^N between the pure fluids;
                                1: constant shear viscosity eta, nu = eta / rho                  */
    double eta;              /* shear viscosity for visc_mode 1                                   */
    int32_t stencil_order;   /* 2: compact isotropic gradients (Sec. 2), fused one-kernel step;
                                6: App. B's order-6 stencil for grad rho^N and grad Phi' (radius 3;
                                K and div u stay compact), run as four plane passes; FP32 storage
                                only, ny >= 3 with walls, not in batches or
                                cmrt_diagnostics_noalloc                                         */
    int32_t curvature_mode;  /* 0: K = div n-hat; 1: K = fixed_K (Sec. 4.2)                        */
    double fixed_K;
    int32_t ghost_N_mode;    /* 0: N relaxes to h^(6).f^(0) (App. A); 1: N relaxes to 0 (Table 1) */
    int32_t precision;       /* population storage in HBM: 0 = FP32 (72 B/node); 1 = BF16, 2 = FP16
                                (64 B/node: rho_R, rho_B and the rest populations R_0, B_0 in
                                FP32; four 16-bit (red, blue) pairs of reference dipoles -- the
                                equilibrium's velocity term and the recolour's segregation term
                                (Eq. eq_re_color) per link direction; eight 16-bit pairs of
                                deviations C_i - rho_C psi_i -/+ D_C of the moving links, FP16
                                ones times 2^k with k = 14 for bulk densities up to 1; the
                                lowest bit of D_0's red half selects the shape of psi: the
                                equilibrium's, psi_d = psi_a / 4, or the one with ghost moment
                                N = 0 that the step writes under ghost_N_mode 1);
                                arithmetic is FP32 in all cases                                   */
    int32_t diag_every;      /* cmrt_step checks the non-finite flag every diag_every steps
                                (synchronising the stream then); 0 = only at cmrt_diagnostics    */
    int32_t precision_reference; /* 16-bit storage reference psi_i: 0 = phi_i of Eq. eq_phi at the
                                node's own mixture (from its stored densities; default);
                                1 = the lattice weights w_i; 2 = phi_i of the pure colour C  */
    int32_t adjoint_fused;   /* kernels of one reverse step of cmrt_adjoint / cmrt_step_vjp
                                (compact stencil; App. B's stencil always uses plane passes):
                                0 = automatic -- in cmrt_adjoint the fused kernels whenever its
                                forward steps can write the forward fields the reverse steps read
                                (one set of 14 planes per recomputed or kept state, allocated where
                                memory allows); otherwise, and in cmrt_step_vjp, the fused kernels
                                where the lattice fills 16-row segments in two waves of the GPU and
                                eight per-node plane passes on smaller lattices; 1 = always the
                                fused kernels; 2 = always the plane passes.  Both compute the same
                                values (rounding order aside)                                     */
} cmrt_params;

/* ABI version of the loaded library (CMRT_ABI_VERSION). */
int32_t cmrt_abi_version(void);

/* sizeof(cmrt_params) as compiled into the library, for binding checks. */
size_t cmrt_params_size(void);

/* Defaults of the paper's static-drop setting for an nx * ny periodic lattice:
 * rho0 = (1, 0.1), alpha = (0.95, 0.5), sigma = 0.005, beta = 0.67,
 * lambda3 = 1 (nu = 1/6), lambda6 = lambda7 = 1, no body force, diag_every 0.
 * Returns CMRT_EINVAL if p is NULL.  Touches no GPU. */
cmrt_status cmrt_params_default(cmrt_params* p, int32_t nx, int32_t ny);

/* Checks a parameter set without touching the GPU.  Returns CMRT_OK or
 * CMRT_EINVAL; the reason is available from cmrt_last_error(NULL). */
cmrt_status cmrt_validate(const cmrt_params* p);

/* Creates a context on the current CUDA device and stream `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream) and initialises the
 * state at t = 0 from a colour field and a velocity field:
 *   rho_R = rho0_r (1 + rho^N_0)/2,  rho_B = rho0_b (1 - rho^N_0)/2,
 *   C_i = (rho_C / rho) f^(0)_i(rho, u_0)          (Eqs. equ_rhoN_def, equ_equ)
 * rho_n0: float[ny][nx] with values in [-1, 1]; NULL means -1 (all blue).
 * u0:     float[2][ny][nx] (u_x then u_y); NULL means 0.
 * On success *out receives the context (caller frees it with cmrt_destroy).
 * Errors: CMRT_EINVAL (parameters, out == NULL), CMRT_ENOMEM, CMRT_ECUDA. */
cmrt_status cmrt_init(const cmrt_params* p, const float* rho_n0, const float* u0,
                      void* cuda_stream, cmrt_ctx** out);

/* Advances the state by n >= 0 time steps t -> t + n.  One step is the whole
 * per-node update of Sec. 2 / App. A: colour gradient, unit normal and
 * curvature, force and force-adjusted velocity, correction tensor, MRT
 * collision in moment space, recolour and streaming, fused in one kernel.
 * Asynchronous, except every diag_every steps (see cmrt_params). */
cmrt_status cmrt_step(cmrt_ctx* c, int64_t n);

/* Steps per CUDA graph in cmrt_step (and in cmrt_adjoint's forward run).
 * An even count > 0 (default 32) records that many steps once per buffer
 * parity, on a private stream, at their first use, and replays the graph for
 * each whole group of steps (single launches for the rest); 0 launches every
 * step on its own.  Results are bit-identical either way; the graphs take the
 * gaps between launches off small lattices (64^2: 8.2 -> 5.4 us per step).
 * Synchronises the stream and drops recorded graphs.  CMRT_EINVAL for an odd
 * or negative count or a batch member view. */
cmrt_status cmrt_set_graph_steps(cmrt_ctx* c, int32_t steps);
/* The current steps per graph, or -1 for NULL. */
int32_t cmrt_get_graph_steps(const cmrt_ctx* c);

/* Macroscopic fields at the current time: rho_R, rho_B (Eq. equ_u_def), the
 * force-adjusted velocity u = (sum_i f_i c_i + G/2)/rho (Eq. equ_u_def) and
 * the pressure p = 3/5 [(1 - alpha_r) rho_R + (1 - alpha_b) rho_B] (App. A,
 * isotropic part of the equilibrium second moment).  Each pointer is a
 * float[ny][nx] buffer or NULL (skipped). */
cmrt_status cmrt_fields(cmrt_ctx* c, float* rho_r, float* rho_b, float* ux, float* uy, float* p);

/* Diagnostics of the current state, reduced in FP64:
 * out[0] = sum rho_R, out[1] = sum rho_B, out[2..3] = sum_r sum_i f_i c_i
 * (colour-blind lattice momentum), out[4] = max |u| (force-adjusted),
 * out[5] = number of nodes whose density is not finite.
 * Synchronises the stream.  Returns CMRT_ENONFINITE (and fails the context)
 * when out[5] > 0. */
cmrt_status cmrt_diagnostics(cmrt_ctx* c, double out[6]);

/* Copies the pre-collision populations R_i(r, t), B_i(r, t) of the current
 * time into dst, float[2][9][ny][nx]. */
cmrt_status cmrt_get_populations(cmrt_ctx* c, float* dst);

/* Replaces the state by the pre-collision populations in src,
 * float[2][9][ny][nx], taken as the state at the current time. */
cmrt_status cmrt_set_populations(cmrt_ctx* c, const float* src);

/* Checkpoint and restart.  cmrt_save writes the context's state exactly as
 * stored (FP32 populations, or the 16-bit records with their FP32 densities)
 * with the time step and the lattice's size and storage form, so that
 * cmrt_load on a context of the same size and storage form resumes the run
 * bit for bit -- unlike a population export and import, which for 16-bit
 * storage re-encodes.  The layout of the bytes is private to this library
 * version (ABI version, sizes and a format tag are checked on load).
 * dst/src: host or device memory of at least cmrt_save_bytes(c) bytes;
 * CMRT_EINVAL if smaller, or on load if the record does not match the
 * context.  Synchronises the stream. */
size_t cmrt_save_bytes(const cmrt_ctx* c);
cmrt_status cmrt_save(cmrt_ctx* c, void* dst, size_t bytes);
cmrt_status cmrt_load(cmrt_ctx* c, const void* src, size_t bytes);

/* Waits for all work queued on the context's stream. */
cmrt_status cmrt_synchronize(cmrt_ctx* c);

/* Number of time steps taken since cmrt_init; -1 for NULL. */
int64_t cmrt_time(const cmrt_ctx* c);

/* Number of kernels this context has launched; -1 for NULL. */
int64_t cmrt_launch_count(const cmrt_ctx* c);

/* Bytes of device memory the context holds. */
size_t cmrt_device_bytes(const cmrt_ctx* c);

/* Diagnostics of caller-owned populations that allocate nothing.
 *
 * The paper has no counterpart: this is a library facility.  It is for
 * callers that cannot allocate device memory when they need the reduction:
 * code under a hard device-memory cap or a custom allocator that forbids
 * ad-hoc allocations, and code that must not let cudaMalloc/cudaFree
 * synchronise the whole device in the middle of a pipeline.  It needs no
 * context and calls no allocating routine.
 *
 * p:     parameters of the lattice (validated as for cmrt_init);
 *        stencil_order 6 is rejected (its passes need a context's planes).
 * pops:  pre-collision populations float[2][9][ny][nx] in DEVICE memory of
 *        the current device (e.g. from cmrt_get_populations), 16-byte aligned
 *        when nx is a multiple of 4 and 4-byte aligned otherwise.  Host
 *        memory (copying it would need a buffer), memory of another device
 *        and a misaligned address are rejected with CMRT_EINVAL before any
 *        launch.
 * out:   host double[6], the same quantities as cmrt_diagnostics.
 * cuda_stream: stream the reduction runs on.  The call waits for this
 *        stream before it returns (the result is copied to the host), so a
 *        stream that is capturing a CUDA graph is rejected with CMRT_EINVAL
 *        before anything is enqueued.
 *
 * Scratch: a fixed area compiled into the library (384 KiB of device memory
 * on every GPU that loads it, held until exit) with room for 8192 partial
 * blocks, i.e. lattices up to 983,040 columns wide and any height.  Wider
 * lattices are rejected with CMRT_EINVAL.  All calls share that area: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  The first call on a device looks up the
 * area's device address (cudaGetSymbolAddress) and keeps it for the life of
 * the process: make that first call before any stream capture, and do not
 * use this entry point on a device after cudaDeviceReset.  Returns
 * CMRT_ENONFINITE when out[5] > 0. */
cmrt_status cmrt_diagnostics_noalloc(const cmrt_params* p, const float* pops, double out[6], void* cuda_stream);

/* ------------------------------------------------------------------------
 * Discrete adjoint (reverse mode) of the step, FP32 storage only.
 *
 * The step f(t+1) = S(f(t); theta) is the composition streaming o recolour
 * o collision o (force, curvature, normal, gradients) o moments of Sec. 2 and
 * App. A; its adjoint applies the transposed Jacobian of every one of those
 * operations in reverse order (transposed gather with bounce-back,
 * transposed MRT reconstruction and relaxation with the Jacobians of the
 * equilibria, sources and correction tensor, adjoint recolour including the
 * derivative of the unit normal and its eps-regularisation, the transposed
 * compact stencils with their wall mirrors).  The paper has no adjoint: this
 * is a library facility.  Parameters theta, in this order:
 *   sigma, beta, lambda3_r, lambda3_b, g_acc[0], g_acc[1].
 * Parameter gradients are accumulated in FP64, the adjoint fields in FP32.
 * ------------------------------------------------------------------------ */

/* Vector-Jacobian product of one step at the current state f(t) (the state
 * is not advanced).
 * lam_next: dJ/df(t+1), float[2][9][ny][nx] (pre-collision layout, host or
 *           device).
 * lam:      receives dJ/df(t) through this step, same layout.
 * grad_params: NULL, or double[6] to which this step's dJ/dtheta is ADDED.
 * Synchronises the stream.  CMRT_EINVAL for 16-bit storage. */
cmrt_status cmrt_step_vjp(cmrt_ctx* c, const float* lam_next, float* lam, double grad_params[6]);

/* Gradient of the colour-field mismatch after nsteps steps,
 *   J = 1/2 sum_r (rho^N(r, t0 + nsteps) - target(r))^2,
 * t0 the current time.  Runs the nsteps forward steps (the context ends at
 * t0 + nsteps, as after cmrt_step), keeping a checkpoint every ckpt_every
 * steps, then sweeps the segments backwards, recomputing each from its
 * checkpoint.  ckpt_every = 1 keeps every state, written in place by the
 * forward steps, and recomputes nothing: the cheapest sweep where HBM holds
 * nsteps states.  Device memory: (ceil(nsteps/ckpt_every) + ckpt_every + 1)
 * states of 72 B per node plus 38 scratch planes, kept for later calls.
 * target:  float[ny][nx] (host or device).
 * J:       NULL or receives J (FP64 sum).
 * grad_params: NULL or receives dJ/dtheta (double[6]).
 * grad_rho_n0: NULL or float[ny][nx] receiving dJ/drho^N_0, the gradient
 *          with respect to the initial colour field given to cmrt_init (the
 *          initial velocity held fixed); only at time 0 (else CMRT_EINVAL).
 * Synchronises.  CMRT_EINVAL for 16-bit storage, nsteps < 1 or
 * ckpt_every < 1, or on a batch member view; CMRT_ENONFINITE if the forward
 * run produced a non-finite density. */
cmrt_status cmrt_adjoint(cmrt_ctx* c, int64_t nsteps, int32_t ckpt_every, const float* target, double* J,
                         double grad_params[6], float* grad_rho_n0);

/* Frees the context and everything it allocated.  NULL is a no-op. */
void cmrt_destroy(cmrt_ctx* c);

/* Message of the last failure on c, or of the last failure in this thread
 * when c is NULL.  The string is owned by the library and stays valid until
 * the next call on the same context (or thread). */
const char* cmrt_last_error(const cmrt_ctx* c);

/* ------------------------------------------------------------------------
 * Batched ensembles.
 *
 * The paper steps one lattice at a time; these calls are a library
 * facility for running many independent lattices of uneven sizes, each the
 * scheme above with its own parameters (sigma, Lambda, alpha, relaxation
 * rates, forces, walls), in ONE persistent kernel launch per time step.  The
 * launch drains a work list of tiles (member, 120-column strip, segment of
 * rows), longest segments first; no CTA ever waits on another, so there is
 * no device-side wait that could time out.  Steps are replayed from CUDA
 * graphs recorded on first use.  Each member's results are bit-identical to
 * stepping it alone with cmrt_step.
 * ------------------------------------------------------------------------ */

/* cmrt_batch_tune flag: measure even when the cache holds an entry. */
#define CMRT_TUNE_FORCE 1

/* Creates an ensemble of n >= 1 lattices on the current device and stream.
 * params:  cmrt_params[n]; every entry is validated as for cmrt_init, and
 *          all must share one `precision`.
 * rho_n0:  array of n pointers (host array), each as rho_n0 of cmrt_init
 *          for that member (host or device float[ny][nx], or NULL); the
 *          array itself may be NULL (all members -1).
 * u0:      likewise, float[2][ny][nx] per member, or NULL.
 * The batch holds both state buffers of every member in two arenas
 * (member offsets aligned to 256 B).  Rows per work item start at
 * min(64, ny) for each size class.  The batch checks the members'
 * non-finite flags every d steps, d the smallest positive diag_every of the
 * members (0 everywhere: only at cmrt_batch_diagnostics).
 * Errors: CMRT_EINVAL (with the member index in the message), CMRT_ENOMEM,
 * CMRT_ECUDA. */
cmrt_status cmrt_batch_init(int32_t n, const cmrt_params* params, const float* const* rho_n0,
                            const float* const* u0, void* cuda_stream, cmrt_batch** out);

/* Advances every member by n >= 0 steps.  Whole blocks of graph_steps steps
 * are launched as one recorded CUDA graph, the rest one launch per step.
 * Asynchronous except at the non-finite checks; CMRT_ENONFINITE names the
 * first member that failed and fails the batch. */
cmrt_status cmrt_batch_step(cmrt_batch* b, int64_t n);

/* Autotuner: picks the rows per work item of each size class (nx, ny,
 * wall_y) by coordinate descent over {8, 16, ..., 512} (capped at ny),
 * two passes, timing whole batched launches (2 warm-up + 5 timed, CUDA
 * events) that read the current state and write the other buffer, so the
 * state does not advance.  cache_path (may be NULL): a JSON array, one
 * object per line, keyed by device name, SM count and the batch signature
 * (precision, vector path, size classes with their counts); a matching
 * entry is applied without measuring unless flags has CMRT_TUNE_FORCE, and
 * a measurement replaces it.  us_per_step (may be NULL) receives the best
 * time of one batched step in microseconds (the cached one on a hit). */
cmrt_status cmrt_batch_tune(cmrt_batch* b, const char* cache_path, int32_t flags, double* us_per_step);

/* Sets the rows per work item of the members of size nx x ny with the given
 * wall_y (CMRT_EINVAL if there are none, or rows < 1).  Rebuilds the work
 * list after the work queued so far has finished. */
cmrt_status cmrt_batch_set_rows(cmrt_batch* b, int32_t nx, int32_t ny, int32_t wall_y, int32_t rows);

/* Rows per work item of a size class, -1 if the batch has no such class. */
int32_t cmrt_batch_get_rows(const cmrt_batch* b, int32_t nx, int32_t ny, int32_t wall_y);

/* Steps per recorded graph: 0 (no graphs) or a positive even number
 * (default 32). */
cmrt_status cmrt_batch_set_graph_steps(cmrt_batch* b, int32_t steps);

/* A view of member k as a context: cmrt_fields, cmrt_diagnostics,
 * cmrt_get_populations, cmrt_set_populations, cmrt_synchronize, cmrt_time
 * work on it and act on that member's state inside the batch.  cmrt_step on
 * a view returns CMRT_EINVAL (members advance with cmrt_batch_step), and
 * cmrt_destroy on a view does nothing: the view belongs to the batch and is
 * freed by cmrt_batch_destroy.  The same view is returned on every call. */
cmrt_status cmrt_batch_member(cmrt_batch* b, int32_t k, cmrt_ctx** view);

/* cmrt_diagnostics of every member into out[n][6].  Synchronises. */
cmrt_status cmrt_batch_diagnostics(cmrt_batch* b, double* out);

/* Waits for all work queued on the batch's stream. */
cmrt_status cmrt_batch_synchronize(cmrt_batch* b);

/* Number of members, steps taken, kernels launched (every batched step is
 * one launch, also inside a graph), and work items per step; -1 for NULL. */
int32_t cmrt_batch_size(const cmrt_batch* b);
int64_t cmrt_batch_time(const cmrt_batch* b);
int64_t cmrt_batch_launch_count(const cmrt_batch* b);
int64_t cmrt_batch_work_items(const cmrt_batch* b);

/* Bytes of device memory the batch holds (arenas, work list, views). */
size_t cmrt_batch_device_bytes(const cmrt_batch* b);

/* Frees the batch, its member views and everything it allocated.  NULL is a
 * no-op. */
void cmrt_batch_destroy(cmrt_batch* b);

/* Message of the last failure on b, or of the last failure in this thread
 * when b is NULL. */
const char* cmrt_batch_last_error(const cmrt_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* CMRT_H */
