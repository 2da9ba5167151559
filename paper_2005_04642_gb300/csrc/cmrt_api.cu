// C ABI of libcmrt (include/cmrt.h): parameter validation, context and
// device-memory management, host/device pointer handling and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cmrt.h"
#include "cmrt_internal.h"

using cmrt::StepParams;

namespace {

// NVTX range over one library call (step, fields, diagnostics, adjoint,
// batch step), for timelines taken with a profiler attached.  NVTX v3 is
// header-only and costs a few nanoseconds when no tool is loaded.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

thread_local std::string g_thread_error;

struct Batch;

// Device staging for host-pointer arguments (grown on demand).
struct Staging {
    float* ptr = nullptr;
    size_t bytes = 0;
};

struct Ctx {
    cmrt_params p{};
    StepParams sp{};
    int device = 0;
    cudaStream_t stream = nullptr;
    void* buf[2] = {nullptr, nullptr};   // post-collision state, A/B (layout of p.precision)
    int cur = 0;                         // buf[cur] holds P_{t-1}
    unsigned* d_flag = nullptr;          // non-finite flag written by the step kernel
    double* d_partials = nullptr;        // per-CTA partial diagnostics
    double* d_diag = nullptr;            // reduced diagnostics
    int n_partials = 0;
    Staging own_staging;
    Staging* stg = &own_staging;         // a batch member uses its batch's staging
    Batch* owner = nullptr;              // batch whose arena holds buf[] (member views)
    int member = -1;
    // discrete adjoint workspace (allocated on first use)
    float* adj_scratch = nullptr;        // float[kAdjPlanes][n]
    double* adj_partials = nullptr;      // double[adj_blocks][kAdjSlots]
    double* adj_out = nullptr;           // double[kAdjSlots]
    float* adj_lam[2] = {nullptr, nullptr};
    float* adj_ckpt = nullptr;           // checkpoints, float[cap][18][n]
    size_t adj_ckpt_cap = 0;
    float* adj_seg = nullptr;            // segment states (slot 0: the checkpoint), float[cap][18][n]
    size_t adj_seg_cap = 0;
    // forward fields of states 0 .. cap - 1 of a segment (written by the
    // replayed steps) or of every kept state (written by the forward run), for
    // the reverse steps, float[cap][kFwdPlanes][n]; null where the reverse
    // step recomputes them (plane passes, or no memory for them)
    float* adj_fields = nullptr;
    size_t adj_fields_cap = 0;
    // CUDA graphs of one checkpoint segment (replay + reverse steps), keyed by
    // the segment length and the adjoint buffer it starts from; recorded on a
    // private stream and valid while the workspace pointers stay put
    struct AdjGraph {
        int64_t len;
        int a;
        bool fields;       // the replayed steps write the forward fields
        cudaGraphExec_t exec;
        int64_t launches;  // kernels one replay of the graph launches
    };
    std::vector<AdjGraph> adj_graphs;
    cudaStream_t adj_capture = nullptr;  // private stream on which graphs are recorded
    // CUDA graphs of graph_steps plain steps starting from buffer parity 0 / 1
    int graph_steps = 32;
    cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
    size_t adj_bytes = 0;
    int rows = 128;                      // rows per CTA of the chain kernel
    int64_t t = 0;
    int64_t launches = 0;
    size_t dev_bytes = 0;
    bool failed = false;
    std::string err;
};

}  // namespace

struct cmrt_ctx {
    Ctx c;
};

namespace {

// An ensemble of independent lattices stepped together by the persistent
// batched kernel.  All members share one storage precision; their states
// live in two arenas (A-B), member m at byte offset off[m] of each.
struct Batch {
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;      // private stream on which graphs are recorded
    int precision = 0;
    bool vec = true;                     // every member has nx % 4 == 0
    std::vector<cmrt_params> p;
    std::vector<StepParams> sp;
    std::vector<size_t> off;
    size_t arena_bytes = 0;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t t = 0;
    int64_t launches = 0;
    size_t dev_bytes = 0;
    StepParams* d_params = nullptr;
    size_t* d_off = nullptr;
    unsigned* d_flags = nullptr;
    unsigned* d_counters = nullptr;
    cmrt::BatchItem* d_items = nullptr;
    size_t items_cap = 0;
    int nitems = 0;
    int grid = 0;                        // persistent CTAs
    int diag_every = 0;                  // smallest positive diag_every of the members
    std::map<std::string, int> rows;     // size class -> rows per work item
    int graph_steps = 32;                // steps per recorded graph (even), 0 = none
    cudaGraphExec_t exec[2] = {nullptr, nullptr};  // graphs starting from parity 0 / 1
    std::vector<cmrt_ctx*> views;
    Staging staging;
    bool failed = false;
    std::string err;
};

}  // namespace

struct cmrt_batch {
    Batch b;
};

namespace {

cmrt_status fail(Ctx* c, cmrt_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (st == CMRT_ECUDA || st == CMRT_ENONFINITE) c->failed = true;
    }
    g_thread_error = buf;
    return st;
}

#define CK(ctx, call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail((ctx), CMRT_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool finite(double v) { return std::isfinite(v); }

cmrt_status validate(const cmrt_params* p) {
    if (!p) return fail(nullptr, CMRT_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(nullptr, CMRT_EINVAL, "nx, ny must be >= 1 (got %d, %d)", p->nx, p->ny);
    const double cells = static_cast<double>(p->nx) * p->ny;
    if (cells * 18.0 * 4.0 > 9.0e18) return fail(nullptr, CMRT_EINVAL, "lattice too large");
    if (p->wall_y != 0 && p->wall_y != 1) return fail(nullptr, CMRT_EINVAL, "wall_y must be 0 or 1");
    if (!(p->rho0_r > 0) || !(p->rho0_b > 0) || !finite(p->rho0_r) || !finite(p->rho0_b))
        return fail(nullptr, CMRT_EINVAL, "rho0_r, rho0_b must be finite and > 0");
    if (!(p->alpha_r >= 0 && p->alpha_r < 1) || !(p->alpha_b >= 0 && p->alpha_b < 1))
        return fail(nullptr, CMRT_EINVAL, "alpha_r, alpha_b must lie in [0, 1)");
    const double Lam = p->rho0_r / p->rho0_b;
    const double Lam_a = (1.0 - p->alpha_b) / (1.0 - p->alpha_r);
    if (std::fabs(Lam_a - Lam) > 1e-9 * Lam)
        return fail(nullptr, CMRT_EINVAL,
                    "density ratio rho0_r/rho0_b = %.12g but (1-alpha_b)/(1-alpha_r) = %.12g (Eq. equ_fred)", Lam,
                    Lam_a);
    if (!finite(p->sigma) || p->sigma < 0) return fail(nullptr, CMRT_EINVAL, "sigma must be finite and >= 0");
    if (!finite(p->beta) || p->beta < 0) return fail(nullptr, CMRT_EINVAL, "beta must be finite and >= 0");
    if (!(p->lambda3_r > 0 && p->lambda3_r < 2) || !(p->lambda3_b > 0 && p->lambda3_b < 2))
        return fail(nullptr, CMRT_EINVAL, "lambda3_r, lambda3_b must lie in (0, 2)");
    if (!(p->lambda6 > 0 && p->lambda6 <= 2) || !(p->lambda7 > 0 && p->lambda7 <= 2))
        return fail(nullptr, CMRT_EINVAL, "lambda6, lambda7 must lie in (0, 2]");
    for (int k = 0; k < 2; ++k)
        if (!finite(p->g_acc[k]) || !finite(p->g_vol[k]))
            return fail(nullptr, CMRT_EINVAL, "body forces must be finite");
    if (p->visc_mode != 0 && p->visc_mode != 1) return fail(nullptr, CMRT_EINVAL, "visc_mode must be 0 or 1");
    if (p->visc_mode == 1 && !(p->eta > 0 && finite(p->eta)))
        return fail(nullptr, CMRT_EINVAL, "eta must be finite and > 0 for visc_mode 1");
    if (p->stencil_order != 2 && p->stencil_order != 6)
        return fail(nullptr, CMRT_EINVAL, "stencil_order must be 2 (compact) or 6 (App. B), got %d", p->stencil_order);
    if (p->stencil_order == 6 && p->precision != 0)
        return fail(nullptr, CMRT_EINVAL, "stencil_order 6 needs FP32 storage (precision 0)");
    if (p->stencil_order == 6 && p->wall_y && p->ny < 3)
        return fail(nullptr, CMRT_EINVAL, "stencil_order 6 with walls needs ny >= 3 (mirror rows of the radius-3 stencil)");
    if (p->curvature_mode != 0 && p->curvature_mode != 1)
        return fail(nullptr, CMRT_EINVAL, "curvature_mode must be 0 or 1");
    if (!finite(p->fixed_K)) return fail(nullptr, CMRT_EINVAL, "fixed_K must be finite");
    if (p->ghost_N_mode != 0 && p->ghost_N_mode != 1)
        return fail(nullptr, CMRT_EINVAL, "ghost_N_mode must be 0 or 1");
    if (p->precision < 0 || p->precision > 2)
        return fail(nullptr, CMRT_EINVAL, "precision must be 0 (FP32), 1 (BF16) or 2 (FP16)");
    if (p->precision_reference < 0 || p->precision_reference > 2)
        return fail(nullptr, CMRT_EINVAL, "precision_reference must be 0, 1 or 2");
    if (p->adjoint_fused < 0 || p->adjoint_fused > 2)
        return fail(nullptr, CMRT_EINVAL, "adjoint_fused must be 0 (automatic), 1 (fused kernels) or 2 (plane passes)");
    if (p->diag_every < 0) return fail(nullptr, CMRT_EINVAL, "diag_every must be >= 0");
    return CMRT_OK;
}

StepParams derive(const cmrt_params& p) {
    StepParams s{};
    s.nx = p.nx;
    s.ny = p.ny;
    s.wall_y = p.wall_y;
    s.visc_mode = p.visc_mode;
    s.curvature_mode = p.curvature_mode;
    s.ghost_N_mode = p.ghost_N_mode;
    s.stencil_order = p.stencil_order;
    s.adjoint_fused = p.adjoint_fused;
    const double Lam = p.rho0_r / p.rho0_b;
    s.inv_rho0_r = static_cast<float>(1.0 / p.rho0_r);
    s.inv_rho0_b = static_cast<float>(1.0 / p.rho0_b);
    s.alpha_r = static_cast<float>(p.alpha_r);
    s.alpha_b = static_cast<float>(p.alpha_b);
    s.kphi_r = static_cast<float>(1.8 * (1.0 - p.alpha_r));
    s.kphi_b = static_cast<float>(1.8 * (1.0 - p.alpha_b));
    s.cs2_r = static_cast<float>(0.6 * (1.0 - p.alpha_r));
    s.cs2_b = static_cast<float>(0.6 * (1.0 - p.alpha_b));
    // Phi' = 3/5 (1 - alpha_R)(rho_R + Lambda rho_B) - rho/3 (App. A)
    s.phip_r = static_cast<float>(0.6 * (1.0 - p.alpha_r) - 1.0 / 3.0);
    s.phip_b = static_cast<float>(0.6 * (1.0 - p.alpha_r) * Lam - 1.0 / 3.0);
    // h^(6).f^(0) = 9/5 alpha_R rho_R + 9/5 alpha_B rho_B - 4/5 rho (App. A)
    s.neq_r = static_cast<float>(1.8 * p.alpha_r - 0.8);
    s.neq_b = static_cast<float>(1.8 * p.alpha_b - 0.8);
    s.half_sigma = static_cast<float>(0.5 * p.sigma);
    s.beta = static_cast<float>(p.beta);
    s.nu_r = static_cast<float>((2.0 / p.lambda3_r - 1.0) / 6.0);
    s.nu_b = static_cast<float>((2.0 / p.lambda3_b - 1.0) / 6.0);
    s.eta = static_cast<float>(p.eta);
    s.lambda6 = static_cast<float>(p.lambda6);
    s.lambda7 = static_cast<float>(p.lambda7);
    s.gacc_x = static_cast<float>(p.g_acc[0]);
    s.gacc_y = static_cast<float>(p.g_acc[1]);
    s.gvol_x = static_cast<float>(p.g_vol[0]);
    s.gvol_y = static_cast<float>(p.g_vol[1]);
    s.fixed_K = static_cast<float>(p.fixed_K);
    s.precision = p.precision;
    s.precision_reference = p.precision_reference;
    // 16-bit storage keeps C_i - rho_C psi_i -/+ D_C for the moving links.
    // Reference 0: phi_i of Eq. eq_phi at the node's own mixture (computed in
    // the kernels from the stored densities with psi_axis = mix_r rho_R +
    // mix_b rho_B over rho); reference 1: the lattice weights w_i; reference
    // 2: phi_i of the pure colour C (alpha_C).  Every reference has psi_axis a
    // multiple of 2^-24; the kernels take psi_diag = psi_axis / 4 (exact in
    // FP32) or, for records flagged N-free, the shape with ghost moment 0.
    s.mix_r = static_cast<float>((1.0 - p.alpha_r) / 5.0);
    s.mix_b = static_cast<float>((1.0 - p.alpha_b) / 5.0);
    // FP16 deviations are stored scaled by 2^k so that small ones stay in
    // FP16's normal range (below 6.1e-5 it keeps only an absolute step of
    // 6e-8, which is about 1 % of a light fluid's deviations): k = 14 for bulk
    // densities up to 1, one less per doubling above, so that deviations up
    // to 4 rho0 stay finite (FP16's largest value is 65504).  Scaling by a
    // power of two commutes exactly with FP32 rounding.  BF16 has FP32's
    // exponent range and is stored unscaled.
    int k = 0;
    if (p.precision == 2) {
        const double rho_max = std::max(p.rho0_r, p.rho0_b);
        k = 14 - std::max(0, static_cast<int>(std::ceil(std::log2(rho_max))));
        k = std::max(k, 0);
    }
    s.dev_scale = static_cast<float>(std::ldexp(1.0, k));
    s.dev_unscale = static_cast<float>(std::ldexp(1.0, -k));
    auto weights = [&](double alpha, float out[3]) {
        const double axis = p.precision_reference == 1 ? 1.0 / 9.0 : (1.0 - alpha) / 5.0;
        const double pa = std::ldexp(std::nearbyint(std::ldexp(axis, 24)), -24);  // a multiple of 2^-24
        out[1] = static_cast<float>(pa);
        out[2] = static_cast<float>(pa / 4.0);        // exact
        out[0] = static_cast<float>(1.0 - 5.0 * pa);  // the rest link's share (the record stores it directly)
    };
    weights(p.alpha_r, s.psi_r);
    weights(p.alpha_b, s.psi_b);
    return s;
}

size_t cells(const Ctx& c) { return static_cast<size_t>(c.p.nx) * c.p.ny; }

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unregistered host pointer
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device-side address of page-locked host memory (cudaHostAlloc,
// cudaHostRegister) mapped for the context's device, or null for any other
// memory.  Kernels read and write such memory directly over the host link
// (NVLink-C2C on Grace), which needs no staging buffer and no copy-engine
// transfer.
void* mapped_host(const Ctx* c, const void* ptr) {
    if (!ptr) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer && a.device == c->device) ? a.devicePointer : nullptr;
}

cmrt_status ensure_staging(Ctx* c, size_t bytes) {
    Staging& st = *c->stg;
    if (st.bytes >= bytes) return CMRT_OK;
    if (st.ptr) {
        cudaStreamSynchronize(c->stream);
        cudaFree(st.ptr);
        st.ptr = nullptr;
        st.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&st.ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        st.ptr = nullptr;
        return fail(c, CMRT_ENOMEM, "cudaMalloc of %zu staging bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    st.bytes = bytes;
    return CMRT_OK;
}

Ctx* live(cmrt_ctx* h) {
    if (!h) {
        fail(nullptr, CMRT_ESTATE, "NULL context");
        return nullptr;
    }
    if (h->c.failed) {
        g_thread_error = "context has failed earlier: " + h->c.err;
        return nullptr;
    }
    Ctx* c = &h->c;
    if (c->owner) {  // a member view follows its batch's time and buffer parity
        if (c->owner->failed) {
            g_thread_error = "batch has failed earlier: " + c->owner->err;
            return nullptr;
        }
        c->cur = c->owner->cur;
        c->t = c->owner->t;
    }
    return c;
}

cmrt_status set_device(Ctx* c) {
    int cur = -1;
    CK(c, cudaGetDevice(&cur));
    if (cur != c->device) CK(c, cudaSetDevice(c->device));
    return CMRT_OK;
}

void drop_adj_graphs(Ctx* c) {
    for (Ctx::AdjGraph& g : c->adj_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    c->adj_graphs.clear();
}

void drop_step_graphs(Ctx* c) {
    for (cudaGraphExec_t& g : c->step_exec)
        if (g) cudaGraphExecDestroy(g), g = nullptr;
}

void free_all(Ctx* c) {
    if (!c->owner) {  // a member view borrows its state and flag from the batch
        for (void*& b : c->buf)
            if (b) cudaFree(b), b = nullptr;
        if (c->d_flag) cudaFree(c->d_flag), c->d_flag = nullptr;
    }
    if (c->d_partials) cudaFree(c->d_partials), c->d_partials = nullptr;
    if (c->d_diag) cudaFree(c->d_diag), c->d_diag = nullptr;
    if (c->own_staging.ptr) cudaFree(c->own_staging.ptr), c->own_staging.ptr = nullptr;
    if (c->adj_scratch) cudaFree(c->adj_scratch), c->adj_scratch = nullptr;
    if (c->adj_partials) cudaFree(c->adj_partials), c->adj_partials = nullptr;
    if (c->adj_out) cudaFree(c->adj_out), c->adj_out = nullptr;
    for (float*& l : c->adj_lam)
        if (l) cudaFree(l), l = nullptr;
    if (c->adj_ckpt) cudaFree(c->adj_ckpt), c->adj_ckpt = nullptr;
    if (c->adj_seg) cudaFree(c->adj_seg), c->adj_seg = nullptr;
    if (c->adj_fields) cudaFree(c->adj_fields), c->adj_fields = nullptr;
    c->adj_bytes = 0;
    c->adj_ckpt_cap = c->adj_seg_cap = c->adj_fields_cap = 0;
    drop_adj_graphs(c);
    drop_step_graphs(c);
    if (c->adj_capture) cudaStreamDestroy(c->adj_capture), c->adj_capture = nullptr;
}

cmrt_status check_flag(Ctx* c) {
    unsigned h = 0;
    CK(c, cudaMemcpyAsync(&h, c->d_flag, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (h) return fail(c, CMRT_ENONFINITE, "non-finite density in the state before step %lld", (long long)c->t);
    return CMRT_OK;
}

// One step src -> dst: the fused kernel, or the plane passes for the order-6
// stencil.  Returns the number of kernels launched, or -1 on a launch error.
int step_once(Ctx* c, const void* src, void* dst, cudaError_t* err) {
    if (c->p.stencil_order == 6) {
        *err = cmrt::launch_step_planes(static_cast<const float*>(src), static_cast<float*>(dst), c->sp,
                                        c->adj_scratch, c->d_flag, c->stream);
        return *err == cudaSuccess ? 4 : -1;
    }
    *err = cmrt::launch_step(src, dst, c->sp, c->rows, c->d_flag, c->stream);
    return *err == cudaSuccess ? 1 : -1;
}

#define STEP(ctx, src, dst)                                                                          \
    do {                                                                                             \
        cudaError_t e_ = cudaSuccess;                                                                \
        const int k_ = step_once((ctx), (src), (dst), &e_);                                          \
        if (k_ < 0) return fail((ctx), CMRT_ECUDA, "step launch failed: %s", cudaGetErrorString(e_)); \
        (ctx)->launches += k_;                                                                       \
    } while (0)

// The state buffer that does not hold the current state.  Between steps it
// is dead (the next step overwrites all of it), so a call that moves data
// between host memory and the device stages through its first `floats`
// floats instead of allocating: nothing is allocated on the device after
// cmrt_init for host inputs of an FP32 state or for host outputs of
// cmrt_fields.  Null when the buffer is smaller than that.
float* idle_buffer(Ctx* c, size_t floats) {
    const size_t have = cells(*c) * cmrt::state_node_bytes(c->p.precision);
    return floats * sizeof(float) <= have ? static_cast<float*>(c->buf[c->cur ^ 1]) : nullptr;
}

// Records graph_steps plain steps starting from buffer parity `parity` on
// the private capture stream (the launchers enqueue on c->stream, which is
// swapped for the recording).
cmrt_status build_step_graph(Ctx* c, int parity) {
    if (!c->adj_capture) CK(c, cudaStreamCreateWithFlags(&c->adj_capture, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    c->stream = c->adj_capture;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->adj_capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < c->graph_steps && e == cudaSuccess; ++k)
            step_once(c, c->buf[(parity + k) & 1], c->buf[(parity + k + 1) & 1], &e);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c->adj_capture, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    c->stream = user;
    if (e != cudaSuccess) return fail(c, CMRT_ECUDA, "recording the step graph failed: %s", cudaGetErrorString(e));
    c->step_exec[parity] = exec;
    return CMRT_OK;
}

// n plain steps on the context's stream: whole graphs of graph_steps steps
// (an even count, so the buffer parity is unchanged), then single launches.
cmrt_status advance(Ctx* c, int64_t n) {
    const int per_step = c->p.stencil_order == 6 ? 4 : 1;
    while (c->graph_steps > 0 && n >= c->graph_steps) {
        if (!c->step_exec[c->cur] && build_step_graph(c, c->cur) != CMRT_OK) return CMRT_ECUDA;
        CK(c, cudaGraphLaunch(c->step_exec[c->cur], c->stream));
        c->t += c->graph_steps;
        c->launches += static_cast<int64_t>(c->graph_steps) * per_step;
        n -= c->graph_steps;
    }
    for (; n > 0; --n) {
        STEP(c, c->buf[c->cur], c->buf[c->cur ^ 1]);
        c->cur ^= 1;
        c->t++;
    }
    return CMRT_OK;
}

// Writes the state at t = 0 into c->buf[c->cur] (Eqs. equ_rhoN_def, equ_equ):
// the equilibrium of the colour field rho_n0 and velocity u0 (host or device
// pointers, NULL for -1 and 0).
cmrt_status init_state(Ctx* c, const float* rho_n0, const float* u0) {
    const cmrt_params* p = &c->p;
    const size_t n = cells(*c);
    // inputs: device memory and mapped page-locked host memory are read by
    // the kernel in place; other host memory is copied into the idle state
    // buffer (FP32 storage) or into staging after an FP32 state area (16-bit
    // storage, encoded from FP32)
    const float* d_rn = rho_n0;
    const float* d_u = u0;
    const bool rn_host = rho_n0 && !is_device_ptr(rho_n0);
    const bool u_host = u0 && !is_device_ptr(u0);
    if (rn_host) d_rn = static_cast<const float*>(mapped_host(c, rho_n0));
    if (u_host) d_u = static_cast<const float*>(mapped_host(c, u0));
    const bool rn_copy = rn_host && !d_rn, u_copy = u_host && !d_u;
    const bool packed = p->precision != 0;
    const size_t need = packed ? 18 * n + ((rn_copy || u_copy) ? 3 * n : 0) : 0;
    if (need && ensure_staging(c, need * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
    if (rn_copy || u_copy) {
        float* in = packed ? c->stg->ptr + 18 * n : idle_buffer(c, 3 * n);
        if (rn_copy) {
            CK(c, cudaMemcpyAsync(in, rho_n0, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            d_rn = in;
        }
        if (u_copy) {
            CK(c, cudaMemcpyAsync(in + n, u0, 2 * n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            d_u = in + n;
        }
    }
    float* post32 = packed ? c->stg->ptr : static_cast<float*>(c->buf[c->cur]);
    CK(c, cmrt::launch_init_fp64(d_rn, d_u, p->nx, p->ny, p->wall_y, p->rho0_r, p->rho0_b, p->alpha_r, p->alpha_b,
                                 post32, c->stream));
    c->launches++;
    if (packed) {
        CK(c, cmrt::launch_encode(post32, c->sp, c->buf[c->cur], c->stream));
        c->launches++;
    }
    // host buffers may be reused by the caller as soon as we return, and the
    // staging area by the next call
    if (rn_host || u_host || packed) CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

}  // namespace

extern "C" {

int32_t cmrt_abi_version(void) { return CMRT_ABI_VERSION; }

size_t cmrt_params_size(void) { return sizeof(cmrt_params); }

cmrt_status cmrt_params_default(cmrt_params* p, int32_t nx, int32_t ny) {
    if (!p) return fail(nullptr, CMRT_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof *p);
    p->nx = nx;
    p->ny = ny;
    p->wall_y = 0;
    p->rho0_r = 1.0;
    p->rho0_b = 0.1;
    p->alpha_r = 0.95;
    p->alpha_b = 0.5;
    p->sigma = 0.005;
    p->beta = 0.67;
    p->lambda3_r = 1.0;
    p->lambda3_b = 1.0;
    p->lambda6 = 1.0;
    p->lambda7 = 1.0;
    p->visc_mode = 0;
    p->eta = 1.0 / 6.0;
    p->stencil_order = 2;
    p->curvature_mode = 0;
    p->fixed_K = 0.0;
    p->ghost_N_mode = 0;
    p->precision = 0;
    p->diag_every = 0;
    return CMRT_OK;
}

cmrt_status cmrt_validate(const cmrt_params* p) { return validate(p); }

cmrt_status cmrt_init(const cmrt_params* p, const float* rho_n0, const float* u0, void* cuda_stream,
                      cmrt_ctx** out) {
    NvtxRange nvtx_range("cmrt_init");
    if (!out) return fail(nullptr, CMRT_EINVAL, "out is NULL");
    *out = nullptr;
    cmrt_status st = validate(p);
    if (st != CMRT_OK) return st;
    cmrt_ctx* h = new (std::nothrow) cmrt_ctx;
    if (!h) return fail(nullptr, CMRT_ENOMEM, "host allocation of the context failed");
    Ctx* c = &h->c;
    c->p = *p;
    c->sp = derive(*p);
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    auto bail = [&](cmrt_status s) {
        g_thread_error = c->err.empty() ? g_thread_error : c->err;
        free_all(c);
        delete h;
        return s;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        fail(c, CMRT_ECUDA, "no CUDA device");
        return bail(CMRT_ECUDA);
    }
    const size_t n = cells(*c);
    const size_t state_bytes = n * cmrt::state_node_bytes(p->precision);
    for (void*& b : c->buf) {
        cudaError_t e = cudaMalloc(&b, state_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b = nullptr;
            fail(c, CMRT_ENOMEM, "cudaMalloc of %zu state bytes failed: %s", state_bytes, cudaGetErrorString(e));
            return bail(CMRT_ENOMEM);
        }
        c->dev_bytes += state_bytes;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        sms = 1;
    }
    c->rows = cmrt::chain_rows(p->nx, p->ny, sms, p->precision);
    const dim3 g = cmrt::chain_grid(p->nx, p->ny, c->rows);
    c->n_partials = static_cast<int>(g.x * g.y);
    if (p->stencil_order == 6) {
        // the order-6 passes keep their fields in the scratch planes and write
        // one partial row per 128-column block of a lattice row
        c->n_partials = std::max(c->n_partials, cmrt::adj_blocks(p->nx, p->ny));
        const size_t bytes = cmrt::kAdjPlanes * cells(*c) * sizeof(float);
        if (cudaMalloc(&c->adj_scratch, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->adj_scratch = nullptr;
            fail(c, CMRT_ENOMEM, "cudaMalloc of %zu scratch bytes for the order-6 step failed", bytes);
            return bail(CMRT_ENOMEM);
        }
        c->adj_bytes += bytes;
    }
    if (cudaMalloc(&c->d_flag, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&c->d_partials, sizeof(double) * cmrt::kDiagSlots * c->n_partials) != cudaSuccess ||
        cudaMalloc(&c->d_diag, sizeof(double) * cmrt::kDiagSlots) != cudaSuccess) {
        cudaGetLastError();
        fail(c, CMRT_ENOMEM, "cudaMalloc of diagnostics buffers failed");
        return bail(CMRT_ENOMEM);
    }
    c->dev_bytes += sizeof(unsigned) + sizeof(double) * cmrt::kDiagSlots * (c->n_partials + 1);
    if (cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned), c->stream) != cudaSuccess) {
        fail(c, CMRT_ECUDA, "cudaMemsetAsync failed");
        return bail(CMRT_ECUDA);
    }
    c->cur = 0;
    st = init_state(c, rho_n0, u0);
    if (st != CMRT_OK) return bail(st);
    c->cur = 0;
    c->t = 0;
    *out = h;
    return CMRT_OK;
}

cmrt_status cmrt_step(cmrt_ctx* h, int64_t n) {
    NvtxRange nvtx_range("cmrt_step");
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (n < 0) return fail(c, CMRT_EINVAL, "n must be >= 0");
    if (c->owner) return fail(c, CMRT_EINVAL, "member %d of a batch is stepped by cmrt_batch_step", c->member);
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    int64_t left = n;
    while (left > 0) {
        // up to the next non-finite check
        int64_t chunk = left;
        if (c->p.diag_every > 0) chunk = std::min<int64_t>(chunk, c->p.diag_every - c->t % c->p.diag_every);
        left -= chunk;
        cmrt_status st = advance(c, chunk);
        if (st != CMRT_OK) return st;
        if (c->p.diag_every > 0 && (c->t % c->p.diag_every) == 0 && (st = check_flag(c)) != CMRT_OK) return st;
    }
    return CMRT_OK;
}

cmrt_status cmrt_set_graph_steps(cmrt_ctx* h, int32_t steps) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (steps < 0 || steps % 2 != 0) return fail(c, CMRT_EINVAL, "graph steps must be 0 or a positive even number");
    if (c->owner) return fail(c, CMRT_EINVAL, "member %d of a batch is stepped by cmrt_batch_step", c->member);
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    CK(c, cudaStreamSynchronize(c->stream));
    drop_step_graphs(c);
    c->graph_steps = steps;
    return CMRT_OK;
}

int32_t cmrt_get_graph_steps(const cmrt_ctx* h) { return h ? h->c.graph_steps : -1; }

cmrt_status cmrt_fields(cmrt_ctx* h, float* rho_r, float* rho_b, float* ux, float* uy, float* p) {
    NvtxRange nvtx_range("cmrt_fields");
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    const size_t n = cells(*c);
    float* outs[5] = {rho_r, rho_b, ux, uy, p};
    float* dev[5];
    bool any_host = false;
    // device memory and mapped page-locked host memory are written by the
    // kernel in place; other host outputs go to the idle state buffer (5 of
    // its 11 or 18 floats per node) and are copied out
    bool copy[5] = {false, false, false, false, false};
    for (int k = 0; k < 5; ++k) {
        dev[k] = outs[k];
        if (outs[k] && !is_device_ptr(outs[k])) {
            dev[k] = static_cast<float*>(mapped_host(c, outs[k]));
            copy[k] = !dev[k];
            any_host = true;
        }
    }
    float* scratch = nullptr;
    if (copy[0] || copy[1] || copy[2] || copy[3] || copy[4]) {
        scratch = idle_buffer(c, 5 * n);
        if (!scratch) {
            if (ensure_staging(c, 5 * n * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
            scratch = c->stg->ptr;
        }
        for (int k = 0; k < 5; ++k)
            if (copy[k]) dev[k] = scratch + k * n;
    }
    const cmrt::FieldOut fo{dev[0], dev[1], dev[2], dev[3], dev[4]};
    if (c->p.stencil_order == 6) {
        CK(c, cmrt::launch_fields_planes(static_cast<const float*>(c->buf[c->cur]), c->sp, c->adj_scratch, fo,
                                         c->stream));
        c->launches += 4;
    } else {
        CK(c, cmrt::launch_fields(c->buf[c->cur], c->sp, c->rows, fo, c->stream));
        c->launches++;
    }
    if (any_host) {
        for (int k = 0; k < 5; ++k)
            if (copy[k]) CK(c, cudaMemcpyAsync(outs[k], dev[k], n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return CMRT_OK;
}

cmrt_status cmrt_diagnostics(cmrt_ctx* h, double out[6]) {
    NvtxRange nvtx_range("cmrt_diagnostics");
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (!out) return fail(c, CMRT_EINVAL, "out is NULL");
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    if (c->p.stencil_order == 6) {
        CK(c, cmrt::launch_diag_planes(static_cast<const float*>(c->buf[c->cur]), c->sp, c->adj_scratch,
                                       c->d_partials, c->stream));
        CK(c, cmrt::launch_diag_reduce(c->d_partials, cmrt::adj_blocks(c->p.nx, c->p.ny), c->d_diag, c->stream));
        c->launches += 5;
    } else {
        CK(c, cmrt::launch_diag_partials(c->buf[c->cur], c->sp, c->rows, c->d_partials, c->stream));
        CK(c, cmrt::launch_diag_reduce(c->d_partials, c->n_partials, c->d_diag, c->stream));
        c->launches += 2;
    }
    double h6[cmrt::kDiagSlots];
    CK(c, cudaMemcpyAsync(h6, c->d_diag, sizeof h6, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    out[0] = h6[0];
    out[1] = h6[1];
    out[2] = h6[2];
    out[3] = h6[3];
    out[4] = std::sqrt(h6[4]);
    out[5] = h6[5];
    if (h6[5] > 0) return fail(c, CMRT_ENONFINITE, "%.0f nodes have a non-finite density at t = %lld", h6[5], (long long)c->t);
    return CMRT_OK;
}

cmrt_status cmrt_get_populations(cmrt_ctx* h, float* dst) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (!dst) return fail(c, CMRT_EINVAL, "dst is NULL");
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    const size_t n18 = cells(*c) * 18;
    const size_t bytes = n18 * sizeof(float);
    const bool host = !is_device_ptr(dst);
    float* mapped = host ? static_cast<float*>(mapped_host(c, dst)) : nullptr;
    const bool copy = host && !mapped;
    const bool packed = c->p.precision != 0;
    // staging: [FP32 post-collision planes (16-bit storage)] [pre-collision copy (unmapped host dst)];
    // an FP32 state copies out through the idle state buffer instead
    const size_t need = packed ? n18 + (copy ? n18 : 0) : 0;
    if (need && ensure_staging(c, need * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
    const float* post32 = static_cast<const float*>(c->buf[c->cur]);
    if (packed) {
        CK(c, cmrt::launch_decode(c->buf[c->cur], c->sp, c->stg->ptr, c->stream));
        c->launches++;
        post32 = c->stg->ptr;
    }
    float* d = copy ? (packed ? c->stg->ptr + n18 : idle_buffer(c, n18)) : (mapped ? mapped : dst);
    CK(c, cmrt::launch_stream_out(post32, c->sp, d, c->stream));
    c->launches++;
    if (copy) CK(c, cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (host) CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

cmrt_status cmrt_set_populations(cmrt_ctx* h, const float* src) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (!src) return fail(c, CMRT_EINVAL, "src is NULL");
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    const size_t n18 = cells(*c) * 18;
    const size_t bytes = n18 * sizeof(float);
    const float* s = src;
    const bool host = !is_device_ptr(src);
    const float* mapped = host ? static_cast<const float*>(mapped_host(c, src)) : nullptr;
    const bool copy = host && !mapped;
    const bool packed = c->p.precision != 0;
    // staging: [FP32 post-collision planes (16-bit storage)] [pre-collision copy (unmapped host src)];
    // an FP32 state copies in through the idle state buffer instead
    const size_t need = packed ? n18 + (copy ? n18 : 0) : 0;
    if (need && ensure_staging(c, need * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
    if (mapped) s = mapped;
    if (copy) {
        float* hs = packed ? c->stg->ptr + n18 : idle_buffer(c, n18);
        CK(c, cudaMemcpyAsync(hs, src, bytes, cudaMemcpyHostToDevice, c->stream));
        s = hs;
    }
    float* post32 = packed ? c->stg->ptr : static_cast<float*>(c->buf[c->cur]);
    CK(c, cmrt::launch_unstream_in(s, c->sp, post32, c->stream));
    c->launches++;
    if (packed) {
        CK(c, cmrt::launch_encode(post32, c->sp, c->buf[c->cur], c->stream));
        c->launches++;
    }
    if (host || packed) CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

// Checkpoint record: this header, then the state buffer's bytes as stored.
struct SaveHeader {
    uint64_t tag;
    int32_t abi, nx, ny, precision, wall_y, stencil_order;
    int64_t t;
    uint64_t state_bytes;
};
constexpr uint64_t kSaveTag = 0x3156415354524d43ull;  // "CMRTSAV1"

size_t cmrt_save_bytes(const cmrt_ctx* h) {
    if (!h) return 0;
    return sizeof(SaveHeader) + cells(h->c) * cmrt::state_node_bytes(h->c.p.precision);
}

cmrt_status cmrt_save(cmrt_ctx* h, void* dst, size_t bytes) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (!dst) return fail(c, CMRT_EINVAL, "dst is NULL");
    const size_t state = cells(*c) * cmrt::state_node_bytes(c->p.precision);
    if (bytes < sizeof(SaveHeader) + state)
        return fail(c, CMRT_EINVAL, "a checkpoint needs %zu bytes, got %zu", sizeof(SaveHeader) + state, bytes);
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    const SaveHeader hd{kSaveTag, CMRT_ABI_VERSION, c->p.nx, c->p.ny, c->p.precision, c->p.wall_y,
                        c->p.stencil_order, c->t, static_cast<uint64_t>(state)};
    char* out = static_cast<char*>(dst);
    if (is_device_ptr(dst)) CK(c, cudaMemcpyAsync(out, &hd, sizeof hd, cudaMemcpyHostToDevice, c->stream));
    else std::memcpy(out, &hd, sizeof hd);
    CK(c, cudaMemcpyAsync(out + sizeof hd, c->buf[c->cur], state, cudaMemcpyDefault, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

cmrt_status cmrt_load(cmrt_ctx* h, const void* src, size_t bytes) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (!src) return fail(c, CMRT_EINVAL, "src is NULL");
    if (c->owner) return fail(c, CMRT_EINVAL, "member %d of a batch follows the batch's time", c->member);
    if (bytes < sizeof(SaveHeader)) return fail(c, CMRT_EINVAL, "%zu bytes hold no checkpoint", bytes);
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    SaveHeader hd{};
    const char* in = static_cast<const char*>(src);
    if (is_device_ptr(src)) {
        CK(c, cudaMemcpyAsync(&hd, in, sizeof hd, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(&hd, in, sizeof hd);
    }
    const size_t state = cells(*c) * cmrt::state_node_bytes(c->p.precision);
    if (hd.tag != kSaveTag || hd.abi != CMRT_ABI_VERSION)
        return fail(c, CMRT_EINVAL, "not a checkpoint of this library version");
    if (hd.nx != c->p.nx || hd.ny != c->p.ny || hd.precision != c->p.precision || hd.wall_y != c->p.wall_y ||
        hd.stencil_order != c->p.stencil_order || hd.state_bytes != state)
        return fail(c, CMRT_EINVAL, "the checkpoint is of a %d x %d lattice (storage %d, walls %d, order %d)", hd.nx,
                    hd.ny, hd.precision, hd.wall_y, hd.stencil_order);
    if (bytes < sizeof hd + state) return fail(c, CMRT_EINVAL, "the checkpoint is cut short (%zu bytes)", bytes);
    CK(c, cudaMemcpyAsync(c->buf[c->cur], in + sizeof hd, state, cudaMemcpyDefault, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->t = hd.t;
    return CMRT_OK;
}

cmrt_status cmrt_synchronize(cmrt_ctx* h) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

int64_t cmrt_time(const cmrt_ctx* h) {
    if (!h) return -1;
    return h->c.owner ? h->c.owner->t : h->c.t;  // a member view follows its batch
}

int64_t cmrt_launch_count(const cmrt_ctx* h) { return h ? h->c.launches : -1; }

size_t cmrt_device_bytes(const cmrt_ctx* h) {
    return h ? h->c.dev_bytes + h->c.own_staging.bytes + h->c.adj_bytes : 0;
}

void cmrt_destroy(cmrt_ctx* h) {
    if (!h || h->c.owner) return;  // member views are freed with their batch
    Ctx* c = &h->c;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != c->device) cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    cudaGetLastError();
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    delete h;
}

const char* cmrt_last_error(const cmrt_ctx* h) {
    if (h) return h->c.err.c_str();
    return g_thread_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Diagnostics without any allocation.
//
// Some callers cannot allocate device memory at the point where they want a
// reduction of the state: code under a hard device-memory cap or a custom
// allocator that forbids ad-hoc allocations, and code that must not let
// cudaMalloc/cudaFree synchronise the whole device in the middle of a
// pipeline.  For them this entry point works on caller-owned populations and
// uses a fixed scratch area compiled into the library instead of a context.
// It waits for its own stream (the result is copied to the host), so a
// stream that is recording a CUDA graph is refused before anything is
// enqueued.
// ---------------------------------------------------------------------------
namespace {

// Per-CTA FP64 partial sums, then the reduced result in the last slot.
// Sized for up to kNoAllocMaxBlocks CTAs of the diagnostics pass; every GPU
// that loads the library holds these 384 KiB until the process exits.
constexpr int kNoAllocMaxBlocks = 8192;
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxBlocks + 1) * cmrt::kDiagSlots];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

extern "C" cmrt_status cmrt_diagnostics_noalloc(const cmrt_params* p, const float* pops, double out[6],
                                                void* cuda_stream) {
    cmrt_status st = validate(p);
    if (st != CMRT_OK) return st;
    if (!pops || !out) return fail(nullptr, CMRT_EINVAL, "pops and out must not be NULL");
    if (p->stencil_order != 2)
        return fail(nullptr, CMRT_EINVAL, "stencil_order 6 needs a context (its passes keep fields in scratch planes)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(nullptr, CMRT_ECUDA, "no usable current CUDA device");
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the call ends by waiting for its stream, which a capturing stream does
    // not allow: refuse before anything is enqueued, leaving the capture intact
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, CMRT_EINVAL, "the stream's capture status cannot be queried");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return fail(nullptr, CMRT_EINVAL, "the stream is capturing a CUDA graph; this call waits for its stream");
    // the pass reads the planes with 16-byte copies when nx is a multiple of 4
    // (4-byte copies otherwise): the base address must allow them
    const uintptr_t align = (p->nx % 4 == 0) ? 16 : 4;
    if (reinterpret_cast<uintptr_t>(pops) % align != 0)
        return fail(nullptr, CMRT_EINVAL, "pops must be %u-byte aligned for nx = %d", static_cast<unsigned>(align),
                    p->nx);
    {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, pops) != cudaSuccess) {
            cudaGetLastError();
            return fail(nullptr, CMRT_EINVAL, "pops must be device memory of the current device");
        }
        if (a.type == cudaMemoryTypeDevice && a.device != dev)
            return fail(nullptr, CMRT_EINVAL, "pops is memory of device %d, the current device is %d", a.device, dev);
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return fail(nullptr, CMRT_EINVAL, "pops must be device memory of the current device");
    }
    double* scratch = nullptr;
    {
        // set-up, once per device, with that device current: the host-side name
        // of a __device__ array is not its device address
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return fail(nullptr, CMRT_ECUDA, "cudaGetSymbolAddress of the scratch area failed: %s",
                            cudaGetErrorString(e));
            g_noalloc_ptr[dev] = static_cast<double*>(ptr);
        }
        scratch = g_noalloc_ptr[dev];
    }
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 1;
    }
    const int strips = (p->nx + cmrt::kTileX - 1) / cmrt::kTileX;
    if (strips > kNoAllocMaxBlocks)
        return fail(nullptr, CMRT_EINVAL, "nx = %d needs %d column strips; the scratch area holds %d", p->nx, strips,
                    kNoAllocMaxBlocks);
    int rows = cmrt::chain_rows(p->nx, p->ny, sms, 0);
    const int max_segs = kNoAllocMaxBlocks / strips;
    if ((p->ny + rows - 1) / rows > max_segs) rows = (p->ny + max_segs - 1) / max_segs;
    const dim3 g = cmrt::chain_grid(p->nx, p->ny, rows);
    const int nblocks = static_cast<int>(g.x * g.y);
    if (nblocks > kNoAllocMaxBlocks)
        return fail(nullptr, CMRT_EINVAL, "lattice %d x %d needs %d partial blocks; the scratch area holds %d", p->nx,
                    p->ny, nblocks, kNoAllocMaxBlocks);
    const StepParams sp = derive(*p);
    double* result = scratch + static_cast<size_t>(kNoAllocMaxBlocks) * cmrt::kDiagSlots;
    // every partial slot used below is written by its CTA and the result by the
    // reduction, so nothing left from an earlier call is read
    CK(nullptr, cmrt::launch_diag_partials_pre(pops, sp, rows, scratch, s));
    CK(nullptr, cmrt::launch_diag_reduce(scratch, nblocks, result, s));
    double h6[cmrt::kDiagSlots];
    CK(nullptr, cudaMemcpyAsync(h6, result, sizeof h6, cudaMemcpyDeviceToHost, s));
    CK(nullptr, cudaStreamSynchronize(s));
    out[0] = h6[0];
    out[1] = h6[1];
    out[2] = h6[2];
    out[3] = h6[3];
    out[4] = std::sqrt(h6[4]);
    out[5] = h6[5];
    if (h6[5] > 0) return fail(nullptr, CMRT_ENONFINITE, "%.0f nodes have a non-finite density", h6[5]);
    return CMRT_OK;
}


// ---------------------------------------------------------------------------
// Batched ensembles (cmrt_batch_*).
//
// Hundreds of independent lattices advance together: one persistent launch
// per time step drains a work list of tiles (member, strip, row segment)
// ordered longest first.  The rows of a tile are set per size class (nx, ny,
// walls) by cmrt_batch_set_rows or by the autotuner, which times whole
// batched launches that do not advance the state and keeps the best rows per
// class (coordinate descent, results cached in a JSON file).  Steps are
// replayed from CUDA graphs of graph_steps launches recorded once per buffer
// parity.
// ---------------------------------------------------------------------------
namespace {

cmrt_status bfail(Batch* b, cmrt_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) {
        b->err = buf;
        if (st == CMRT_ECUDA || st == CMRT_ENONFINITE) b->failed = true;
    }
    g_thread_error = buf;
    return st;
}

#define BCK(b, call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail((b), CMRT_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

std::string class_key(const cmrt_params& p) {
    char k[64];
    snprintf(k, sizeof k, "%dx%dw%d", p.nx, p.ny, p.wall_y);
    return k;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Rows per work item before tuning: whole lattices up to 64 rows, else 64.
int default_rows(const cmrt_params& p) { return std::min(64, std::max(1, p.ny)); }

Batch* blive(cmrt_batch* h) {
    if (!h) {
        bfail(nullptr, CMRT_ESTATE, "NULL batch");
        return nullptr;
    }
    if (h->b.failed) {
        g_thread_error = "batch has failed earlier: " + h->b.err;
        return nullptr;
    }
    return &h->b;
}

cmrt_status bset_device(Batch* b) {
    int cur = -1;
    BCK(b, cudaGetDevice(&cur));
    if (cur != b->device) BCK(b, cudaSetDevice(b->device));
    return CMRT_OK;
}

void drop_graphs(Batch* b) {
    for (cudaGraphExec_t& e : b->exec)
        if (e) cudaGraphExecDestroy(e), e = nullptr;
}

void free_batch(Batch* b) {
    drop_graphs(b);
    for (cmrt_ctx*& v : b->views) {
        if (v) {
            free_all(&v->c);
            delete v;
            v = nullptr;
        }
    }
    for (void*& p : b->buf)
        if (p) cudaFree(p), p = nullptr;
    if (b->d_params) cudaFree(b->d_params), b->d_params = nullptr;
    if (b->d_off) cudaFree(b->d_off), b->d_off = nullptr;
    if (b->d_flags) cudaFree(b->d_flags), b->d_flags = nullptr;
    if (b->d_counters) cudaFree(b->d_counters), b->d_counters = nullptr;
    if (b->d_items) cudaFree(b->d_items), b->d_items = nullptr;
    if (b->staging.ptr) cudaFree(b->staging.ptr), b->staging.ptr = nullptr;
    if (b->capture) cudaStreamDestroy(b->capture), b->capture = nullptr;
}

// Work list for the current rows per class: every member cut into strips of
// kTileX columns and segments of its class's rows, longest segments first,
// and within equal lengths member by member, segment by segment, so that
// neighbouring strips (which share halo columns) run close together in time.
cmrt_status build_items(Batch* b) {
    std::vector<cmrt::BatchItem> items;
    for (int m = 0; m < b->n; ++m) {
        const cmrt_params& p = b->p[m];
        const int r = b->rows[class_key(p)];
        const int strips = (p.nx + cmrt::kTileX - 1) / cmrt::kTileX;
        for (int y0 = 0; y0 < p.ny; y0 += r)
            for (int s = 0; s < strips; ++s)
                items.push_back(cmrt::BatchItem{m, s * cmrt::kTileX, y0, std::min(r, p.ny - y0)});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const cmrt::BatchItem& a, const cmrt::BatchItem& c) { return a.rows > c.rows; });
    // the kernels of earlier steps may still read the old list
    BCK(b, cudaStreamSynchronize(b->stream));
    if (items.size() > b->items_cap) {
        if (b->d_items) {
            cudaFree(b->d_items);
            b->dev_bytes -= b->items_cap * sizeof(cmrt::BatchItem);
            b->d_items = nullptr;
            b->items_cap = 0;
        }
        cudaError_t e = cudaMalloc(&b->d_items, items.size() * sizeof(cmrt::BatchItem));
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->d_items = nullptr;
            return bfail(b, CMRT_ENOMEM, "cudaMalloc of the work list failed: %s", cudaGetErrorString(e));
        }
        b->items_cap = items.size();
        b->dev_bytes += b->items_cap * sizeof(cmrt::BatchItem);
    }
    BCK(b, cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(cmrt::BatchItem), cudaMemcpyHostToDevice,
                           b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->nitems = static_cast<int>(items.size());
    drop_graphs(b);  // they hold the old list length
    return CMRT_OK;
}

cudaError_t batch_launch(Batch* b, int src_parity, cudaStream_t s) {
    cmrt::BatchArgs A{b->d_items, b->nitems, b->d_params, b->d_off,
                      static_cast<const char*>(b->buf[src_parity]), static_cast<char*>(b->buf[src_parity ^ 1]),
                      b->d_flags, b->d_counters};
    return cmrt::launch_batch(A, b->precision, b->vec, b->grid, s);
}

// Records graph_steps batched steps starting from buffer parity `parity`.
cmrt_status build_graph(Batch* b, int parity) {
    BCK(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < b->graph_steps && e == cudaSuccess; ++k) e = batch_launch(b, (parity + k) & 1, b->capture);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, CMRT_ECUDA, "recording the step graph failed: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec[parity] = nullptr;
        return bfail(b, CMRT_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    }
    return CMRT_OK;
}

cmrt_status check_batch_flags(Batch* b) {
    std::vector<unsigned> h(b->n);
    BCK(b, cudaMemcpyAsync(h.data(), b->d_flags, b->n * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    for (int m = 0; m < b->n; ++m)
        if (h[m]) return bfail(b, CMRT_ENONFINITE, "member %d has a non-finite density before step %lld", m, (long long)b->t);
    return CMRT_OK;
}

// ----- autotuner cache: a JSON array with one object per line -----
std::string json_str(const std::string& line, const char* key) {
    const std::string k = std::string("\"") + key + "\": \"";
    const size_t a = line.find(k);
    if (a == std::string::npos) return "";
    const size_t b = line.find('"', a + k.size());
    if (b == std::string::npos) return "";
    return line.substr(a + k.size(), b - a - k.size());
}

std::string sanitize(std::string v) {
    for (char& ch : v)
        if (ch == '"' || ch == '\\' || static_cast<unsigned char>(ch) < 32) ch = '_';
    return v;
}

std::vector<std::string> read_lines(const char* path) {
    std::vector<std::string> out;
    FILE* f = fopen(path, "r");
    if (!f) return out;
    char buf[8192];
    while (fgets(buf, sizeof buf, f)) {
        std::string l(buf);
        while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
        if (l.find("\"signature\"") != std::string::npos) {
            if (!l.empty() && l.back() == ',') l.pop_back();
            out.push_back(l);
        }
    }
    fclose(f);
    return out;
}

bool write_lines(const char* path, const std::vector<std::string>& lines) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fputs("[\n", f);
    for (size_t i = 0; i < lines.size(); ++i) fprintf(f, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
    fputs("]\n", f);
    const bool ok = fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), path) == 0;
}

// "64x64w0=32 128x128w0=64" <-> the rows map
std::string rows_string(const std::map<std::string, int>& rows) {
    std::string s;
    for (const auto& kv : rows) s += (s.empty() ? "" : " ") + kv.first + "=" + std::to_string(kv.second);
    return s;
}

bool parse_rows(const std::string& s, std::map<std::string, int>& rows) {
    std::map<std::string, int> got;
    size_t pos = 0;
    while (pos < s.size()) {
        size_t end = s.find(' ', pos);
        if (end == std::string::npos) end = s.size();
        const std::string tok = s.substr(pos, end - pos);
        const size_t eq = tok.find('=');
        if (eq == std::string::npos) return false;
        const int r = std::atoi(tok.c_str() + eq + 1);
        if (r < 1) return false;
        got[tok.substr(0, eq)] = r;
        pos = end + 1;
    }
    for (const auto& kv : rows)
        if (!got.count(kv.first)) return false;
    for (auto& kv : rows) kv.second = got[kv.first];
    return true;
}

// Signature of what the tuned rows depend on: storage, vector path and the
// multiset of size classes.
std::string batch_signature(const Batch* b) {
    std::map<std::string, int> count;
    for (const cmrt_params& p : b->p) count[class_key(p)]++;
    std::string s = "p" + std::to_string(b->precision) + " v" + std::to_string(b->vec ? 1 : 0);
    for (const auto& kv : count) s += " " + kv.first + "*" + std::to_string(kv.second);
    return s;
}

}  // namespace

extern "C" {

cmrt_status cmrt_batch_init(int32_t n, const cmrt_params* params, const float* const* rho_n0, const float* const* u0,
                            void* cuda_stream, cmrt_batch** out) {
    if (!out) return bfail(nullptr, CMRT_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !params) return bfail(nullptr, CMRT_EINVAL, "a batch needs n >= 1 members and their params");
    for (int m = 0; m < n; ++m) {
        cmrt_status st = validate(&params[m]);
        if (st != CMRT_OK) return bfail(nullptr, st, "member %d: %s", m, g_thread_error.c_str());
        if (params[m].precision != params[0].precision)
            return bfail(nullptr, CMRT_EINVAL, "member %d: all members must share one storage precision", m);
        if (params[m].stencil_order != 2)
            return bfail(nullptr, CMRT_EINVAL, "member %d: batches run the fused compact-stencil step only", m);
    }
    cmrt_batch* h = new (std::nothrow) cmrt_batch;
    if (!h) return bfail(nullptr, CMRT_ENOMEM, "host allocation of the batch failed");
    Batch* b = &h->b;
    auto bail = [&](cmrt_status s) {
        g_thread_error = b->err.empty() ? g_thread_error : b->err;
        free_batch(b);
        delete h;
        return s;
    };
    b->n = n;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->precision = params[0].precision;
    b->p.assign(params, params + n);
    b->views.assign(n, nullptr);
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        cudaGetLastError();
        bfail(b, CMRT_ECUDA, "no CUDA device");
        return bail(CMRT_ECUDA);
    }
    const size_t node = cmrt::state_node_bytes(b->precision);
    for (int m = 0; m < n; ++m) {
        b->sp.push_back(derive(params[m]));
        b->vec = b->vec && (params[m].nx % 4) == 0;
        b->off.push_back(b->arena_bytes);
        const size_t bytes = static_cast<size_t>(params[m].nx) * params[m].ny * node;
        b->arena_bytes += (bytes + 255) / 256 * 256;  // 256-byte aligned members
        b->rows[class_key(params[m])] = default_rows(params[m]);
        if (params[m].diag_every > 0 && (b->diag_every == 0 || params[m].diag_every < b->diag_every))
            b->diag_every = params[m].diag_every;
    }
    auto dmalloc = [&](void** ptr, size_t bytes) {
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            bfail(b, CMRT_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            return false;
        }
        b->dev_bytes += bytes;
        return true;
    };
    if (!dmalloc(&b->buf[0], b->arena_bytes) || !dmalloc(&b->buf[1], b->arena_bytes) ||
        !dmalloc(reinterpret_cast<void**>(&b->d_params), n * sizeof(StepParams)) ||
        !dmalloc(reinterpret_cast<void**>(&b->d_off), n * sizeof(size_t)) ||
        !dmalloc(reinterpret_cast<void**>(&b->d_flags), n * sizeof(unsigned)) ||
        !dmalloc(reinterpret_cast<void**>(&b->d_counters), 2 * sizeof(unsigned)))
        return bail(CMRT_ENOMEM);
    auto ck = [&](cudaError_t e, const char* what) {
        if (e == cudaSuccess) return true;
        bfail(b, CMRT_ECUDA, "%s failed: %s", what, cudaGetErrorString(e));
        return false;
    };
    if (!ck(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "cudaStreamCreateWithFlags") ||
        !ck(cudaMemcpyAsync(b->d_params, b->sp.data(), n * sizeof(StepParams), cudaMemcpyHostToDevice, b->stream),
            "copy of member parameters") ||
        !ck(cudaMemcpyAsync(b->d_off, b->off.data(), n * sizeof(size_t), cudaMemcpyHostToDevice, b->stream),
            "copy of member offsets") ||
        !ck(cudaMemsetAsync(b->d_flags, 0, n * sizeof(unsigned), b->stream), "cudaMemsetAsync") ||
        !ck(cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(unsigned), b->stream), "cudaMemsetAsync"))
        return bail(CMRT_ECUDA);
    int per_sm = 0, sms = 0;
    if (!ck(cmrt::prepare_batch(b->precision, b->vec, &per_sm), "setting up the batched kernel") ||
        !ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "cudaDeviceGetAttribute"))
        return bail(CMRT_ECUDA);
    if (per_sm < 1) {
        bfail(b, CMRT_ECUDA, "the batched kernel does not fit on an SM");
        return bail(CMRT_ECUDA);
    }
    b->grid = per_sm * sms;
    // initial states, member by member, through the single-lattice path
    for (int m = 0; m < n; ++m) {
        Ctx tmp;
        tmp.p = params[m];
        tmp.sp = b->sp[m];
        tmp.device = b->device;
        tmp.stream = b->stream;
        tmp.buf[0] = static_cast<char*>(b->buf[0]) + b->off[m];
        tmp.buf[1] = static_cast<char*>(b->buf[1]) + b->off[m];
        tmp.cur = 0;
        tmp.stg = &b->staging;
        tmp.owner = b;
        cmrt_status st = init_state(&tmp, rho_n0 ? rho_n0[m] : nullptr, u0 ? u0[m] : nullptr);
        b->launches += tmp.launches;
        if (st != CMRT_OK) {
            bfail(b, st, "member %d: %s", m, tmp.err.c_str());
            return bail(st);
        }
    }
    if (build_items(b) != CMRT_OK) return bail(CMRT_ECUDA);
    *out = h;
    return CMRT_OK;
}

cmrt_status cmrt_batch_step(cmrt_batch* h, int64_t n) {
    NvtxRange nvtx_range("cmrt_batch_step");
    Batch* b = blive(h);
    if (!b) return CMRT_ESTATE;
    if (n < 0) return bfail(b, CMRT_EINVAL, "n must be >= 0");
    if (bset_device(b) != CMRT_OK) return CMRT_ECUDA;
    int64_t left = n;
    while (left > 0) {
        int64_t chunk = left;
        if (b->diag_every > 0) chunk = std::min<int64_t>(chunk, b->diag_every - b->t % b->diag_every);
        left -= chunk;
        while (b->graph_steps > 0 && chunk >= b->graph_steps) {
            if (!b->exec[b->cur] && build_graph(b, b->cur) != CMRT_OK) return CMRT_ECUDA;
            BCK(b, cudaGraphLaunch(b->exec[b->cur], b->stream));
            b->t += b->graph_steps;  // an even count: the parity is unchanged
            b->launches += b->graph_steps;
            chunk -= b->graph_steps;
        }
        for (; chunk > 0; --chunk) {
            BCK(b, batch_launch(b, b->cur, b->stream));
            b->cur ^= 1;
            b->t++;
            b->launches++;
        }
        if (b->diag_every > 0 && b->t % b->diag_every == 0) {
            cmrt_status st = check_batch_flags(b);
            if (st != CMRT_OK) return st;
        }
    }
    return CMRT_OK;
}

cmrt_status cmrt_batch_set_rows(cmrt_batch* h, int32_t nx, int32_t ny, int32_t wall_y, int32_t rows) {
    Batch* b = blive(h);
    if (!b) return CMRT_ESTATE;
    cmrt_params k{};
    k.nx = nx;
    k.ny = ny;
    k.wall_y = wall_y;
    auto it = b->rows.find(class_key(k));
    if (it == b->rows.end()) return bfail(b, CMRT_EINVAL, "no member of size %d x %d with wall_y %d", nx, ny, wall_y);
    if (rows < 1) return bfail(b, CMRT_EINVAL, "rows must be >= 1");
    if (bset_device(b) != CMRT_OK) return CMRT_ECUDA;
    it->second = rows;
    return build_items(b);
}

int32_t cmrt_batch_get_rows(const cmrt_batch* h, int32_t nx, int32_t ny, int32_t wall_y) {
    if (!h) return -1;
    cmrt_params k{};
    k.nx = nx;
    k.ny = ny;
    k.wall_y = wall_y;
    auto it = h->b.rows.find(class_key(k));
    return it == h->b.rows.end() ? -1 : it->second;
}

cmrt_status cmrt_batch_set_graph_steps(cmrt_batch* h, int32_t steps) {
    Batch* b = blive(h);
    if (!b) return CMRT_ESTATE;
    if (steps < 0 || steps % 2 != 0) return bfail(b, CMRT_EINVAL, "graph steps must be 0 or a positive even number");
    if (bset_device(b) != CMRT_OK) return CMRT_ECUDA;
    BCK(b, cudaStreamSynchronize(b->stream));
    drop_graphs(b);
    b->graph_steps = steps;
    return CMRT_OK;
}

cmrt_status cmrt_batch_tune(cmrt_batch* h, const char* cache_path, int32_t flags, double* us_per_step) {
    Batch* b = blive(h);
    if (!b) return CMRT_ESTATE;
    if (bset_device(b) != CMRT_OK) return CMRT_ECUDA;
    cudaDeviceProp prop{};
    BCK(b, cudaGetDeviceProperties(&prop, b->device));
    const std::string device = sanitize(prop.name);
    const std::string sig = batch_signature(b);
    std::vector<std::string> lines;
    if (cache_path) lines = read_lines(cache_path);
    if (cache_path && !(flags & CMRT_TUNE_FORCE)) {
        for (const std::string& l : lines) {
            if (json_str(l, "device") != device || json_str(l, "signature") != sig) continue;
            const size_t a = l.find("\"sms\": ");
            if (a == std::string::npos || std::atoi(l.c_str() + a + 7) != prop.multiProcessorCount) continue;
            std::map<std::string, int> rows = b->rows;
            if (!parse_rows(json_str(l, "rows"), rows)) continue;
            b->rows = rows;
            if (us_per_step) {
                const size_t u = l.find("\"us_per_step\": ");
                *us_per_step = u == std::string::npos ? 0.0 : std::atof(l.c_str() + u + 15);
            }
            return build_items(b);
        }
    }
    // Time whole batched launches from the current state into the other
    // buffer: the state does not advance, so tuning leaves results unchanged.
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    auto time_us = [&](double* us) -> cmrt_status {
        cmrt_status st = build_items(b);
        if (st != CMRT_OK) return st;
        constexpr int kWarm = 2, kReps = 5;
        for (int k = 0; k < kWarm; ++k) BCK(b, batch_launch(b, b->cur, b->stream));
        BCK(b, cudaEventRecord(e0, b->stream));
        for (int k = 0; k < kReps; ++k) BCK(b, batch_launch(b, b->cur, b->stream));
        BCK(b, cudaEventRecord(e1, b->stream));
        BCK(b, cudaEventSynchronize(e1));
        float ms = 0.f;
        BCK(b, cudaEventElapsedTime(&ms, e0, e1));
        b->launches += kWarm + kReps;
        *us = 1000.0 * ms / kReps;
        return CMRT_OK;
    };
    cmrt_status st = CMRT_OK;
    double best = 0.0;
    st = time_us(&best);
    for (int pass = 0; pass < 2 && st == CMRT_OK; ++pass) {
        for (auto& kv : b->rows) {
            const int ny = std::atoi(kv.first.c_str() + kv.first.find('x') + 1);
            const int keep = kv.second;
            int best_r = keep;
            for (int r = 8; r <= 512 && st == CMRT_OK; r *= 2) {
                const int rr = std::min(r, ny);
                if (rr == keep) continue;
                kv.second = rr;
                double us = 0.0;
                st = time_us(&us);
                if (st == CMRT_OK && us < best) {
                    best = us;
                    best_r = rr;
                }
                if (r >= ny) break;
            }
            kv.second = best_r;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CMRT_OK) return st;
    st = build_items(b);
    if (st != CMRT_OK) return st;
    if (us_per_step) *us_per_step = best;
    if (cache_path) {
        char line[4096];
        snprintf(line, sizeof line,
                 "{\"device\": \"%s\", \"sms\": %d, \"signature\": \"%s\", \"rows\": \"%s\", \"us_per_step\": %.1f}",
                 device.c_str(), prop.multiProcessorCount, sig.c_str(), rows_string(b->rows).c_str(), best);
        std::vector<std::string> keep;
        for (const std::string& l : lines)
            if (!(json_str(l, "device") == device && json_str(l, "signature") == sig)) keep.push_back(l);
        keep.push_back(line);
        if (!write_lines(cache_path, keep)) return bfail(b, CMRT_EINVAL, "cannot write the tuning cache %s", cache_path);
    }
    return CMRT_OK;
}

cmrt_status cmrt_batch_member(cmrt_batch* h, int32_t k, cmrt_ctx** view) {
    Batch* b = blive(h);
    if (!b) return CMRT_ESTATE;
    if (!view) return bfail(b, CMRT_EINVAL, "view is NULL");
    *view = nullptr;
    if (k < 0 || k >= b->n) return bfail(b, CMRT_EINVAL, "member %d out of range [0, %d)", k, b->n);
    if (!b->views[k]) {
        if (bset_device(b) != CMRT_OK) return CMRT_ECUDA;
        cmrt_ctx* v = new (std::nothrow) cmrt_ctx;
        if (!v) return bfail(b, CMRT_ENOMEM, "host allocation of a member view failed");
        Ctx* c = &v->c;
        c->p = b->p[k];
        c->sp = b->sp[k];
        c->device = b->device;
        c->stream = b->stream;
        c->buf[0] = static_cast<char*>(b->buf[0]) + b->off[k];
        c->buf[1] = static_cast<char*>(b->buf[1]) + b->off[k];
        c->d_flag = b->d_flags + k;
        c->stg = &b->staging;
        c->owner = b;
        c->member = k;
        int sms = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
            cudaGetLastError();
            sms = 1;
        }
        c->rows = cmrt::chain_rows(c->p.nx, c->p.ny, sms, c->p.precision);
        const dim3 g = cmrt::chain_grid(c->p.nx, c->p.ny, c->rows);
        c->n_partials = static_cast<int>(g.x * g.y);
        if (cudaMalloc(&c->d_partials, sizeof(double) * cmrt::kDiagSlots * c->n_partials) != cudaSuccess ||
            cudaMalloc(&c->d_diag, sizeof(double) * cmrt::kDiagSlots) != cudaSuccess) {
            cudaGetLastError();
            free_all(c);
            delete v;
            return bfail(b, CMRT_ENOMEM, "cudaMalloc of a member view's diagnostics buffers failed");
        }
        c->dev_bytes = sizeof(double) * cmrt::kDiagSlots * (c->n_partials + 1);
        b->dev_bytes += c->dev_bytes;
        b->views[k] = v;
    }
    *view = b->views[k];
    return CMRT_OK;
}

cmrt_status cmrt_batch_diagnostics(cmrt_batch* h, double* out) {
    Batch* b = blive(h);
    if (!b) return CMRT_ESTATE;
    if (!out) return bfail(b, CMRT_EINVAL, "out is NULL");
    for (int m = 0; m < b->n; ++m) {
        cmrt_ctx* v = nullptr;
        cmrt_status st = cmrt_batch_member(h, m, &v);
        if (st != CMRT_OK) return st;
        st = cmrt_diagnostics(v, out + 6 * static_cast<size_t>(m));
        b->launches += 2;
        if (st == CMRT_ENONFINITE) return bfail(b, st, "member %d: %s", m, v->c.err.c_str());
        if (st != CMRT_OK) return bfail(b, st, "member %d: %s", m, g_thread_error.c_str());
    }
    return CMRT_OK;
}

cmrt_status cmrt_batch_synchronize(cmrt_batch* h) {
    Batch* b = blive(h);
    if (!b) return CMRT_ESTATE;
    BCK(b, cudaStreamSynchronize(b->stream));
    return CMRT_OK;
}

int32_t cmrt_batch_size(const cmrt_batch* h) { return h ? h->b.n : -1; }

int64_t cmrt_batch_time(const cmrt_batch* h) { return h ? h->b.t : -1; }

int64_t cmrt_batch_launch_count(const cmrt_batch* h) { return h ? h->b.launches : -1; }

int64_t cmrt_batch_work_items(const cmrt_batch* h) { return h ? h->b.nitems : -1; }

size_t cmrt_batch_device_bytes(const cmrt_batch* h) { return h ? h->b.dev_bytes + h->b.staging.bytes : 0; }

void cmrt_batch_destroy(cmrt_batch* h) {
    if (!h) return;
    Batch* b = &h->b;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != b->device) cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    cudaGetLastError();
    if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
    delete h;
}

const char* cmrt_batch_last_error(const cmrt_batch* h) {
    if (h) return h->b.err.c_str();
    return g_thread_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Discrete adjoint (cmrt_step_vjp, cmrt_adjoint).
// ---------------------------------------------------------------------------
namespace {

// Grows the adjoint workspace: scratch planes, partial sums, two adjoint
// states, `ckpt` checkpoint states, `seg` recomputed segment states and,
// where the reverse step runs fused, `fields` sets of forward fields.
cmrt_status ensure_adj(Ctx* c, size_t ckpt, size_t seg, size_t fields) {
    const size_t n = cells(*c);
    const size_t state = 18 * n * sizeof(float);
    auto grow = [&](void** ptr, size_t bytes) -> cmrt_status {
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            return fail(c, CMRT_ENOMEM, "cudaMalloc of %zu adjoint bytes failed: %s", bytes, cudaGetErrorString(e));
        }
        c->adj_bytes += bytes;
        return CMRT_OK;
    };
    cmrt_status st = CMRT_OK;
    const size_t nb = static_cast<size_t>(cmrt::adj_blocks(c->p.nx, c->p.ny));
    if (!c->adj_scratch && (st = grow(reinterpret_cast<void**>(&c->adj_scratch), cmrt::kAdjPlanes * n * sizeof(float))))
        return st;
    if (!c->adj_partials &&
        (st = grow(reinterpret_cast<void**>(&c->adj_partials), nb * cmrt::kAdjSlots * sizeof(double))))
        return st;
    if (!c->adj_out && (st = grow(reinterpret_cast<void**>(&c->adj_out), cmrt::kAdjSlots * sizeof(double)))) return st;
    for (float*& l : c->adj_lam)
        if (!l && (st = grow(reinterpret_cast<void**>(&l), state))) return st;
    if (ckpt > c->adj_ckpt_cap) {
        CK(c, cudaStreamSynchronize(c->stream));
        if (c->adj_ckpt) cudaFree(c->adj_ckpt), c->adj_ckpt = nullptr, c->adj_bytes -= c->adj_ckpt_cap * state;
        c->adj_ckpt_cap = 0;
        if ((st = grow(reinterpret_cast<void**>(&c->adj_ckpt), ckpt * state))) return st;
        c->adj_ckpt_cap = ckpt;
    }
    if (seg > c->adj_seg_cap) {
        CK(c, cudaStreamSynchronize(c->stream));
        drop_adj_graphs(c);  // they name the old segment buffer
        if (c->adj_seg) cudaFree(c->adj_seg), c->adj_seg = nullptr, c->adj_bytes -= c->adj_seg_cap * state;
        c->adj_seg_cap = 0;
        if ((st = grow(reinterpret_cast<void**>(&c->adj_seg), seg * state))) return st;
        c->adj_seg_cap = seg;
    }
    // Forward fields of the states whose reverse step can read them, where the
    // reverse step runs fused.  Optional: without the memory for them the
    // reverse steps recompute the fields.
    const size_t nfields = cmrt::adj_fields_usable(c->sp) ? fields : 0;
    if (nfields > c->adj_fields_cap) {
        const size_t fstate = static_cast<size_t>(cmrt::kFwdPlanes) * n * sizeof(float);
        CK(c, cudaStreamSynchronize(c->stream));
        drop_adj_graphs(c);  // they name the old buffer, or none
        if (c->adj_fields) cudaFree(c->adj_fields), c->adj_fields = nullptr, c->adj_bytes -= c->adj_fields_cap * fstate;
        c->adj_fields_cap = 0;
        if (cudaMalloc(reinterpret_cast<void**>(&c->adj_fields), nfields * fstate) == cudaSuccess) {
            c->adj_fields_cap = nfields;
            c->adj_bytes += nfields * fstate;
        } else {
            cudaGetLastError();  // not an error: the reverse steps recompute the fields
            c->adj_fields = nullptr;
        }
    }
    return CMRT_OK;
}

// Reduces the partial sums into out[kAdjSlots] on the host (synchronises).
cmrt_status adj_collect(Ctx* c, double* out) {
    CK(c, cmrt::launch_adjoint_reduce(c->adj_partials, cmrt::adj_blocks(c->p.nx, c->p.ny), c->adj_out, c->stream));
    c->launches++;
    CK(c, cudaMemcpyAsync(out, c->adj_out, cmrt::kAdjSlots * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

cmrt_status adj_zero(Ctx* c) {
    CK(c, cudaMemsetAsync(c->adj_partials, 0,
                          static_cast<size_t>(cmrt::adj_blocks(c->p.nx, c->p.ny)) * cmrt::kAdjSlots * sizeof(double),
                          c->stream));
    return CMRT_OK;
}

}  // namespace

extern "C" cmrt_status cmrt_step_vjp(cmrt_ctx* h, const float* lam_next, float* lam, double grad_params[6]) {
    NvtxRange nvtx_range("cmrt_step_vjp");
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (!lam_next || !lam) return fail(c, CMRT_EINVAL, "lam_next and lam must not be NULL");
    if (c->p.precision != 0) return fail(c, CMRT_EINVAL, "the adjoint needs FP32 storage (precision 0)");
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    cmrt_status st = ensure_adj(c, 0, 0, 0);
    if (st != CMRT_OK) return st;
    const size_t n18 = cells(*c) * 18;
    const float* src = lam_next;
    if (!is_device_ptr(lam_next)) {
        CK(c, cudaMemcpyAsync(c->adj_lam[1], lam_next, n18 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        src = c->adj_lam[1];
    }
    // adjoint of P_t: the transpose of the gather f(t+1) = gather(P_t), a permutation
    CK(c, cmrt::launch_unstream_in(src, c->sp, c->adj_lam[0], c->stream));
    if ((st = adj_zero(c)) != CMRT_OK) return st;
    const bool host = !is_device_ptr(lam);
    float* dst = host ? c->adj_lam[1] : lam;
    CK(c, cmrt::launch_adjoint_step_pre(static_cast<const float*>(c->buf[c->cur]), c->adj_lam[0], c->sp,
                                        c->adj_scratch, c->adj_partials, dst, c->stream));
    c->launches += 1 + cmrt::adj_launches_per_step(c->sp);
    if (host) CK(c, cudaMemcpyAsync(lam, dst, n18 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    double out[cmrt::kAdjSlots];
    if ((st = adj_collect(c, out)) != CMRT_OK) return st;
    if (grad_params)
        for (int k = 0; k < 6; ++k) grad_params[k] += out[k];
    return CMRT_OK;
}

// The graph of one checkpoint segment of `len` steps whose reverse sweep
// starts from adjoint buffer `a`: recompute the states 1 .. len - 1 of the
// segment buffer from slot 0 (the checkpoint), then the reverse steps
// len - 1 .. 0.  Where the reverse step runs fused and the field buffer is
// there, the step that recomputes state j + 1 also writes the forward fields
// of state j, bit for bit those the reverse step would recompute, so that
// reverse steps len - 2 .. 0 skip that recomputation.  Recorded on the first
// use of (len, a) -- on a private stream, so the caller's stream may be any
// -- and replayed afterwards; *launches receives its kernel count.  sp: the
// call's parameters (fused reverse kernels where it uses forward fields).
cmrt_status adj_segment_graph(Ctx* c, const cmrt::StepParams& sp, int64_t len, int a, cudaGraphExec_t* out,
                              int64_t* launches) {
    const bool emit = c->adj_fields && cmrt::adj_fused(sp) && len > 1 &&
                      static_cast<size_t>(len - 1) <= c->adj_fields_cap;
    for (const Ctx::AdjGraph& g : c->adj_graphs)
        if (g.len == len && g.a == a && g.fields == emit) {
            *out = g.exec;
            *launches = g.launches;
            return CMRT_OK;
        }
    const size_t nf = static_cast<size_t>(cmrt::kFwdPlanes) * cells(*c);
    auto fields = [&](int64_t j) { return c->adj_fields + static_cast<size_t>(j) * nf; };
    int64_t count = 0;
    if (!c->adj_capture) CK(c, cudaStreamCreateWithFlags(&c->adj_capture, cudaStreamNonBlocking));
    const size_t n18 = 18 * cells(*c);
    auto slot = [&](int64_t j) { return c->adj_seg + static_cast<size_t>(j) * n18; };
    cudaStream_t user = c->stream;
    c->stream = c->adj_capture;  // the launchers enqueue on c->stream
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->adj_capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int64_t j = 1; j < len && e == cudaSuccess; ++j) {
            if (emit) {
                e = cmrt::launch_step_fields(slot(j - 1), slot(j), sp, c->rows, c->d_flag, fields(j - 1),
                                             c->stream);
                count += 1;
            } else {
                count += step_once(c, slot(j - 1), slot(j), &e);
            }
        }
        int aa = a;
        for (int64_t j = len - 1; j >= 0 && e == cudaSuccess; --j, aa ^= 1) {
            const float* fwd = emit && j < len - 1 ? fields(j) : nullptr;
            e = cmrt::launch_adjoint_step(slot(j), c->adj_lam[aa], sp, c->adj_scratch, c->adj_partials,
                                          c->adj_lam[aa ^ 1], c->stream, fwd);
            count += cmrt::adj_launches_per_step(sp) - (fwd ? 1 : 0);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c->adj_capture, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    c->stream = user;
    if (e != cudaSuccess) return fail(c, CMRT_ECUDA, "recording the adjoint segment graph failed: %s", cudaGetErrorString(e));
    c->adj_graphs.push_back({len, a, emit, exec, count});
    *out = exec;
    *launches = count;
    return CMRT_OK;
}

extern "C" cmrt_status cmrt_adjoint(cmrt_ctx* h, int64_t nsteps, int32_t ckpt_every, const float* target, double* J,
                                    double grad_params[6], float* grad_rho_n0) {
    NvtxRange nvtx_range("cmrt_adjoint");
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (c->owner) return fail(c, CMRT_EINVAL, "member %d of a batch is stepped by cmrt_batch_step", c->member);
    if (nsteps < 1 || ckpt_every < 1) return fail(c, CMRT_EINVAL, "nsteps and ckpt_every must be >= 1");
    if (!target) return fail(c, CMRT_EINVAL, "target is NULL");
    if (c->p.precision != 0) return fail(c, CMRT_EINVAL, "the adjoint needs FP32 storage (precision 0)");
    if (grad_rho_n0 && c->t != 0)
        return fail(c, CMRT_EINVAL, "grad_rho_n0 needs the initial state (time 0, now %lld)", (long long)c->t);
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    const int64_t K = ckpt_every;
    const size_t nck = static_cast<size_t>((nsteps + K - 1) / K);
    const size_t seg = static_cast<size_t>(std::min<int64_t>(K, nsteps));
    // fields: of every state with every state kept, else of a segment's
    // states but its last
    cmrt_status st = ensure_adj(c, nck, seg, K == 1 ? static_cast<size_t>(nsteps) : seg - 1);
    if (st != CMRT_OK) return st;
    const size_t n = cells(*c), n18 = 18 * n;
    const size_t state = n18 * sizeof(float);
    const float* d_target = target;
    if (!is_device_ptr(target)) {
        if (ensure_staging(c, n * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
        CK(c, cudaMemcpyAsync(c->stg->ptr, target, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        d_target = c->stg->ptr;
    }
    if ((st = adj_zero(c)) != CMRT_OK) return st;
    // forward, keeping P_{kK-1} (relative to the current time) as checkpoint k
    CK(c, cudaMemcpyAsync(c->adj_ckpt, c->buf[c->cur], state, cudaMemcpyDeviceToDevice, c->stream));
    // Forward fields from the forward steps where the field buffer could be
    // had: then every reverse step of the call runs fused (the same kernels
    // whichever source a state's fields come from, so the checkpoint interval
    // does not change the result); otherwise the lattice-size rule decides.
    const size_t need = K == 1 ? static_cast<size_t>(nsteps) : seg - 1;
    const bool use_fields = cmrt::adj_fields_usable(c->sp) && need > 0 && c->adj_fields && c->adj_fields_cap >= need;
    cmrt::StepParams spa = c->sp;
    if (use_fields) spa.adjoint_fused = 1;
    // every state kept: each forward step writes the fields of the state it reads
    const bool emit_all = K == 1 && use_fields;
    const size_t nf = static_cast<size_t>(cmrt::kFwdPlanes) * n;
    if (K == 1) {
        // every state is kept (memory permitting, the cheapest sweep): step t
        // reads slot t of the checkpoint array and writes slot t + 1 (the last
        // step the lattice's other buffer), so that the reverse sweep reads
        // each state in place -- no copies and no recomputation
        for (int64_t t = 0; t < nsteps; ++t) {
            float* src = c->adj_ckpt + static_cast<size_t>(t) * n18;
            void* dst = t + 1 < nsteps ? static_cast<void*>(c->adj_ckpt + static_cast<size_t>(t + 1) * n18)
                                       : c->buf[c->cur ^ 1];
            if (emit_all) {
                CK(c, cmrt::launch_step_fields(src, static_cast<float*>(dst), c->sp, c->rows, c->d_flag,
                                               c->adj_fields + static_cast<size_t>(t) * nf, c->stream));
                c->launches++;
            } else {
                STEP(c, src, dst);
            }
            c->t++;
        }
        c->cur ^= 1;
    }
    for (size_t k = 1; K > 1 && k <= nck; ++k) {
        if ((st = advance(c, std::min<int64_t>(static_cast<int64_t>(k) * K, nsteps) - static_cast<int64_t>(k - 1) * K)) !=
            CMRT_OK)
            return st;
        if (k < nck)
            CK(c, cudaMemcpyAsync(c->adj_ckpt + k * n18, c->buf[c->cur], state, cudaMemcpyDeviceToDevice, c->stream));
    }
    // objective and its adjoint
    int a = 0;
    CK(c, cmrt::launch_adjoint_seed(static_cast<const float*>(c->buf[c->cur]), d_target, c->sp, c->adj_scratch,
                                    c->adj_partials, c->adj_lam[a], c->stream));
    c->launches += 2;
    // reverse sweep.  K = 1: each reverse step reads its kept state.
    // Otherwise segments in reverse: the checkpoint goes to slot 0 of the
    // segment buffer, then one graph recomputes the segment's states from it
    // and runs its reverse steps
    if (K == 1) {
        for (int64_t t = nsteps - 1; t >= 0; --t, a ^= 1)
            CK(c, cmrt::launch_adjoint_step(c->adj_ckpt + static_cast<size_t>(t) * n18, c->adj_lam[a], spa,
                                            c->adj_scratch, c->adj_partials, c->adj_lam[a ^ 1], c->stream,
                                            emit_all ? c->adj_fields + static_cast<size_t>(t) * nf : nullptr));
        c->launches += nsteps * (cmrt::adj_launches_per_step(spa) - (emit_all ? 1 : 0));
    }
    for (int64_t k = static_cast<int64_t>(nck) - 1; K > 1 && k >= 0; --k) {
        const int64_t len = std::min((k + 1) * K, nsteps) - k * K;
        CK(c, cudaMemcpyAsync(c->adj_seg, c->adj_ckpt + static_cast<size_t>(k) * n18, state, cudaMemcpyDeviceToDevice,
                              c->stream));
        cudaGraphExec_t exec = nullptr;
        int64_t nl = 0;
        if ((st = adj_segment_graph(c, spa, len, a, &exec, &nl)) != CMRT_OK) return st;
        CK(c, cudaGraphLaunch(exec, c->stream));
        c->launches += nl;
        a ^= static_cast<int>(len & 1);
    }
    if (grad_rho_n0) {
        // f(0) and dJ/df(0): the gather of P_{-1} and of its adjoint (a permutation)
        float* pre0 = c->adj_lam[a ^ 1];
        float* lam0 = c->adj_scratch;  // 18 of its planes
        CK(c, cmrt::launch_stream_out(c->adj_ckpt, c->sp, pre0, c->stream));
        CK(c, cmrt::launch_stream_out(c->adj_lam[a], c->sp, lam0, c->stream));
        const bool host = !is_device_ptr(grad_rho_n0);
        float* g = grad_rho_n0;
        if (host) {
            if (ensure_staging(c, 2 * n * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
            g = c->stg->ptr + n;
        }
        CK(c, cmrt::launch_adjoint_init(pre0, lam0, c->sp, g, c->stream));
        c->launches += 3;
        if (host) CK(c, cudaMemcpyAsync(grad_rho_n0, g, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    double out[cmrt::kAdjSlots];
    if ((st = adj_collect(c, out)) != CMRT_OK) return st;
    if (J) *J = out[6];
    if (grad_params)
        for (int k = 0; k < 6; ++k) grad_params[k] = out[k];
    return check_flag(c);
}
