// Internal interface between the C ABI (cmrt_api.cu) and the kernels
// (cmrt_step.cu, cmrt_aux.cu) of libcmrt.  Not installed, not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

namespace cmrt {

// Launches `kernel` with programmatic stream serialisation: the launch may
// overlap the tail of the previous kernel on the stream, which removes the
// gap between back-to-back kernels on small lattices.  Every kernel launched
// this way starts with pdl_begin() (cmrt_device.cuh).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the arguments, converted to the kernel's parameter types, by address
    return [&](std::remove_cv_t<std::remove_reference_t<KArgs>>... a) {
        void* ptrs[] = {static_cast<void*>(&a)...};
        return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(kernel), ptrs);
    }(static_cast<Args&&>(args)...);
}

// Parameters of one step in the form the kernels use: FP32 coefficients
// derived once on the host (in FP64) from cmrt_params.
// Population storage in HBM (cmrt_params.precision).
constexpr int kPrecF32 = 0;
constexpr int kPrecB16 = 1;
constexpr int kPrecF16 = 2;

struct StepParams {
    int nx, ny, wall_y;
    int precision;                 // kPrecF32 / kPrecB16 / kPrecF16
    int precision_reference;       // 16-bit storage reference: 0 node mixture, 1 w_i, 2 pure colour
    float psi_r[3], psi_b[3];      // constant reference weights (rest, axis, diagonal), references 1 and 2
    float mix_r, mix_b;            // (1 - alpha_C) / 5: psi_axis of the node mixture (reference 0)
    float dev_scale, dev_unscale;  // 16-bit deviations are stored as d * dev_scale (a power of two)
    int visc_mode, curvature_mode, ghost_N_mode;
    int stencil_order;             // 2: compact gradients; 6: App. B for grad rho^N and grad Phi'
    int adjoint_fused;              // 0: automatic, 1: fused reverse tail, 2: plane passes
    float inv_rho0_r, inv_rho0_b;  // colour index (Eq. equ_rhoN_def)
    float alpha_r, alpha_b;        // rest weights phi_0 (Eq. eq_phi)
    float kphi_r, kphi_b;          // 9/5 (1 - alpha_C): phi_i = w_i (kphi_r rho_R + kphi_b rho_B) / rho
    float cs2_r, cs2_b;            // 3/5 (1 - alpha_C): pressure (App. A)
    float phip_r, phip_b;          // Phi' = phip_r rho_R + phip_b rho_B (App. A)
    float neq_r, neq_b;            // h^(6).f^(0) = neq_r rho_R + neq_b rho_B (App. A)
    float half_sigma, beta;
    float nu_r, nu_b, eta;         // viscosity model (Sec. 2)
    float lambda6, lambda7;
    float gacc_x, gacc_y, gvol_x, gvol_y;
    float fixed_K;
};

// Output buffers of the field pass (any may be null); `fwd` receives the
// forward fields of a step's input state (Pass::StepFields), kFwdPlanes planes
// float[kFwdPlanes][ny][nx] in the order of FwdPlane.
struct FieldOut {
    float* rho_r;
    float* rho_b;
    float* ux;
    float* uy;
    float* p;
    float* fwd;
};

// The forward fields of a state that one reverse step of the adjoint reads,
// as planes: colour densities, colour fractions, Phi', grad rho^N, K, the
// force G and the force-adjusted velocity u (the first planes of the
// adjoint's scratch, and the layout Pass::StepFields writes).  The momentum
// planes between them are holes in a set the step writes (the plane passes
// use them): with the twelve planes packed the reverse collision pass ran
// 4 % slower at 2048^2, measured, so the sets keep these offsets.
enum FwdPlane : int {
    kFwdRR = 0, kFwdRB, kFwdJX, kFwdJY, kFwdCHR, kFwdCHB, kFwdPHIP, kFwdGX, kFwdGY, kFwdK, kFwdGFX, kFwdGFY, kFwdUX,
    kFwdUY, kFwdPlanes
};

// Geometry of the fused row-marching kernel: a CTA owns a strip of kTileX
// columns (plus a 4-column halo on each side, kWin columns in all) and marches
// down a segment of rows of it (chain_rows); each of its thread groups has
// kThreads threads, one per window column.
constexpr int kThreads = 128;
constexpr int kWin = 128;
constexpr int kHalo = 4;
constexpr int kTileX = kWin - 2 * kHalo;  // 120
constexpr int kRing = 9;                  // rows of post-collision populations kept in shared memory

// Step: one time step; StepFields: the same step, also writing the forward
// fields of its input state (FP32 storage, for the adjoint's segment replay).
enum class Pass : int { Step = 0, Fields = 1, Diag = 2, StepFields = 3 };

// Number of FP64 partial sums each CTA of the diagnostics pass writes.
constexpr int kDiagSlots = 6;  // mass_r, mass_b, mom_x, mom_y, max|u|^2, non-finite count

// Bytes of one node of the state for a storage precision (72 FP32, 64 16-bit).
size_t state_node_bytes(int precision);
// grid of the chain kernel for a lattice, with `rows` rows per CTA
dim3 chain_grid(int nx, int ny, int rows);
// rows per CTA chosen for a lattice on a device with `sms` multiprocessors
int chain_rows(int nx, int ny, int sms, int precision);

// One fused step: src holds the post-collision state P_{t-1} in the layout of
// P.precision, dst receives P_t.  flag is set non-zero if a node has a
// non-finite density.
cudaError_t launch_step(const void* src, void* dst, const StepParams& P, int rows, unsigned* flag, cudaStream_t s);
// The same step (FP32 storage, compact stencil) also writing the forward
// fields of src (the state P_{t-1}) into fwd[kFwdPlanes][ny][nx], bit for bit
// the values the adjoint's own forward recomputation gives.
cudaError_t launch_step_fields(const float* src, float* dst, const StepParams& P, int rows, unsigned* flag,
                               float* fwd, cudaStream_t s);
// Fields of the state whose post-collision populations are in src.
cudaError_t launch_fields(const void* src, const StepParams& P, int rows, FieldOut out, cudaStream_t s);
// Per-CTA FP64 partial diagnostics into partials[grid][kDiagSlots].
cudaError_t launch_diag_partials(const void* src, const StepParams& P, int rows, double* partials, cudaStream_t s);
// Same, from pre-collision FP32 populations in the public layout float[2][9][ny][nx].
cudaError_t launch_diag_partials_pre(const float* pre, const StepParams& P, int rows,
                                     double* partials, cudaStream_t s);
// Reduces nblocks partial rows into out[kDiagSlots] (one CTA).
cudaError_t launch_diag_reduce(const double* partials, int nblocks, double* out, cudaStream_t s);

// Batched ensembles: one work item is the strip [x0, x0 + kTileX) of rows
// [y0, y0 + rows) of lattice `member`.
struct BatchItem {
    int member, x0, y0, rows;
};

// Arguments of one persistent batched launch (all pointers are device memory).
struct BatchArgs {
    const BatchItem* items;     // work list, in the order the CTAs take it
    int nitems;
    const StepParams* params;   // [members]
    const size_t* offsets;      // [members] byte offset of a member's state in src and dst
    const char* src;            // post-collision states P_{t-1} of all members
    char* dst;                  // receives P_t
    unsigned* flags;            // [members] non-finite flags
    unsigned* counters;         // [2] next item, CTAs finished; zero between launches
};

// Sets up the batched kernel for a storage precision on the current device
// and reports how many of its CTAs fit on one SM.
cudaError_t prepare_batch(int precision, bool vec, int* ctas_per_sm);
// One step of every member of a batch: `grid` persistent CTAs drain the work list.
cudaError_t launch_batch(const BatchArgs& A, int precision, bool vec, int grid, cudaStream_t s);

// Plane passes (cmrt_planes.cu), FP32 storage: one thread per node, the
// intermediate fields in scratch planes float[kAdjPlanes][ny][nx].
// The step, fields and diagnostics with the order-6 gradient (App. B); each
// launches 4 kernels, diagnostics write partials[adj_blocks][kDiagSlots].
cudaError_t launch_step_planes(const float* post, float* dst, const StepParams& P, float* scratch, unsigned* flag,
                               cudaStream_t s);
cudaError_t launch_fields_planes(const float* post, const StepParams& P, float* scratch, FieldOut out,
                                 cudaStream_t s);
cudaError_t launch_diag_planes(const float* post, const StepParams& P, float* scratch, double* partials,
                               cudaStream_t s);

// Discrete adjoint (cmrt_planes.cu), FP32 storage.  scratch: float[kAdjPlanes][ny][nx];
// partials: double[adj_blocks][kAdjSlots], accumulated by every launch (zero it
// before the first): slots 0..5 = dJ/d(sigma, beta, lambda3_r, lambda3_b,
// g_acc_x, g_acc_y), slot 6 = J.
constexpr int kAdjPlanes = 38;
constexpr int kAdjSlots = 8;
int adj_blocks(int nx, int ny);
int adj_launches_per_step(const StepParams& P);
// lam_post: adjoint of P_t; post: P_{t-1}; writes the adjoint of P_{t-1} into lam_prev.
// fwd: the forward fields of post written by launch_step_fields, or null to
// recompute them (used only where adj_fused(P)).
cudaError_t launch_adjoint_step(const float* post, const float* lam_post, const StepParams& P, float* scratch,
                                double* partials, float* lam_prev, cudaStream_t s, const float* fwd = nullptr);
// whether one reverse step runs as the fused kernels (compact stencil, lattice large enough or asked for)
bool adj_fused(const StepParams& P);
// whether the fused kernels may read forward fields written by the forward
// steps (compact stencil, plane passes not asked for); a call that uses such
// fields runs all its reverse steps fused
bool adj_fields_usable(const StepParams& P);
// same, but writes dJ/df(t) (pre-collision, float[2][9][ny][nx]) into lam_pre
cudaError_t launch_adjoint_step_pre(const float* post, const float* lam_post, const StepParams& P, float* scratch,
                                    double* partials, float* lam_pre, cudaStream_t s);
// J of f(T) = gather(post) against target, and the adjoint of post (P_{T-1}) in lam_post
cudaError_t launch_adjoint_seed(const float* post, const float* target, const StepParams& P, float* scratch,
                                double* partials, float* lam_post, cudaStream_t s);
// dJ/drho^N_0 from the initial pre-collision state and its adjoint
cudaError_t launch_adjoint_init(const float* pre0, const float* lam_pre0, const StepParams& P, float* grad_rho_n0,
                                cudaStream_t s);
cudaError_t launch_adjoint_reduce(const double* partials, int nblocks, double* out, cudaStream_t s);

// 16-bit storage: FP32 post-collision planes float[18][ny][nx] <-> the
// deviation layout of P.precision (see cmrt_step.cu).
cudaError_t launch_encode(const float* post32, const StepParams& P, void* state, cudaStream_t s);
cudaError_t launch_decode(const void* state, const StepParams& P, float* post32, cudaStream_t s);

// Initial state: writes into post the populations P_{-1} whose streaming gives
// the equilibrium state of Eq. equ_equ at t = 0.
cudaError_t launch_init_fp64(const float* rho_n0, const float* u0, int nx, int ny, int walls, double rho0_r,
                             double rho0_b, double alpha_r, double alpha_b, float* post, cudaStream_t s);
// Pre-collision populations f(t) = stream(P_{t-1}) into pre[18][ny][nx].
cudaError_t launch_stream_out(const float* post, const StepParams& P, float* pre, cudaStream_t s);
// Inverse: post P_{t-1} such that stream(P_{t-1}) = pre.
cudaError_t launch_unstream_in(const float* pre, const StepParams& P, float* post, cudaStream_t s);

}  // namespace cmrt
