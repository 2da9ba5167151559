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
 *   the context's device; the library detects which (cudaPointerGetAttributes)
 *   and copies through its own staging buffer when it is host memory.  The
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

#define CMRT_ABI_VERSION 2

typedef struct cmrt_ctx cmrt_ctx; /* opaque, owned by the library */

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
    int32_t stencil_order;   /* 2: compact isotropic gradients (Sec. 2) -- the only order built   */
    int32_t curvature_mode;  /* 0: K = div n-hat; 1: K = fixed_K (Sec. 4.2)                        */
    double fixed_K;
    int32_t ghost_N_mode;    /* 0: N relaxes to h^(6).f^(0) (App. A); 1: N relaxes to 0 (Table 1) */
    int32_t precision;       /* population storage in HBM: 0 = FP32 (72 B/node); 1 = BF16, 2 = FP16
                                (44 B/node: rho_R, rho_B in FP32 plus nine 16-bit pairs of
                                deviations C_i - rho_C psi^C_i); arithmetic is FP32 in all cases */
    int32_t diag_every;      /* cmrt_step checks the non-finite flag every diag_every steps
                                (synchronising the stream then); 0 = only at cmrt_diagnostics    */
    int32_t precision_reference; /* 16-bit storage reference psi^C_i: 0 = phi_i of pure colour C
                                (Eq. eq_phi at alpha_C); 1 = the lattice weights w_i            */
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
 * code recording a CUDA graph, code under a hard device-memory cap or a
 * custom allocator, code that must not let cudaMalloc/cudaFree synchronise
 * the device.  It needs no context and calls no allocating routine.
 *
 * p:     parameters of the lattice (validated as for cmrt_init).
 * pops:  pre-collision populations float[2][9][ny][nx] in DEVICE memory of
 *        the current device (e.g. from cmrt_get_populations); host memory is
 *        rejected with CMRT_EINVAL, since copying it would need a buffer.
 * out:   host double[6], the same quantities as cmrt_diagnostics.
 * cuda_stream: stream the reduction runs on; the call synchronises it.
 *
 * Scratch: a fixed area compiled into the library (384 KiB of device memory
 * on every GPU that loads it, held until exit) with room for 8192 partial
 * blocks, i.e. lattices up to 983,040 columns wide and any height.  Wider
 * lattices are rejected with CMRT_EINVAL.  All calls share that area: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  The first call on a device looks up the
 * area's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Returns CMRT_ENONFINITE when out[5] > 0. */
cmrt_status cmrt_diagnostics_noalloc(const cmrt_params* p, const float* pops, double out[6], void* cuda_stream);

/* Frees the context and everything it allocated.  NULL is a no-op. */
void cmrt_destroy(cmrt_ctx* c);

/* Message of the last failure on c, or of the last failure in this thread
 * when c is NULL.  The string is owned by the library and stays valid until
 * the next call on the same context (or thread). */
const char* cmrt_last_error(const cmrt_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* CMRT_H */
