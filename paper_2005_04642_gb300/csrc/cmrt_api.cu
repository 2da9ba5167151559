// C ABI of libcmrt (include/cmrt.h): parameter validation, context and
// device-memory management, host/device pointer handling and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "cmrt.h"
#include "cmrt_internal.h"

using cmrt::StepParams;

namespace {

thread_local std::string g_thread_error;

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
    float* staging = nullptr;            // device staging for host-pointer arguments
    size_t staging_bytes = 0;
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
    if (p->stencil_order != 2)
        return fail(nullptr, CMRT_EINVAL, "stencil_order %d is not built (only the compact order 2 is)",
                    p->stencil_order);
    if (p->curvature_mode != 0 && p->curvature_mode != 1)
        return fail(nullptr, CMRT_EINVAL, "curvature_mode must be 0 or 1");
    if (!finite(p->fixed_K)) return fail(nullptr, CMRT_EINVAL, "fixed_K must be finite");
    if (p->ghost_N_mode != 0 && p->ghost_N_mode != 1)
        return fail(nullptr, CMRT_EINVAL, "ghost_N_mode must be 0 or 1");
    if (p->precision < 0 || p->precision > 2)
        return fail(nullptr, CMRT_EINVAL, "precision must be 0 (FP32), 1 (BF16) or 2 (FP16)");
    if (p->precision_reference != 0 && p->precision_reference != 1)
        return fail(nullptr, CMRT_EINVAL, "precision_reference must be 0 or 1");
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
    // 16-bit storage keeps C_i - rho_C psi^C_i.  Reference 0: the pure-colour
    // rest weights phi_i of Eq. eq_phi at alpha_C; reference 1: w_i.
    // The FP32 weights are adjusted so that psi_0 + 4 psi_axis + 4 psi_diag is
    // exactly 1 in real arithmetic: any reference decodes correctly, but one
    // whose weights do not sum to 1 would bias colour mass every step.
    const double wts[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    auto weights = [&](double alpha, float out[3]) {
        const double axis = p.precision_reference == 1 ? wts[1] : 1.8 * (1.0 - alpha) * wts[1];
        const double diag = p.precision_reference == 1 ? wts[2] : 1.8 * (1.0 - alpha) * wts[2];
        const double fa = static_cast<float>(axis);
        const double moving = std::ldexp(std::nearbyint(std::ldexp(4.0 * fa + 4.0 * static_cast<float>(diag), 24)), -24);
        out[1] = static_cast<float>(fa);
        out[2] = static_cast<float>((moving - 4.0 * fa) / 4.0);   // exact: a multiple of 2^-30
        out[0] = static_cast<float>(1.0 - moving);                // exact: a multiple of 2^-24
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

cmrt_status ensure_staging(Ctx* c, size_t bytes) {
    if (c->staging_bytes >= bytes) return CMRT_OK;
    if (c->staging) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->staging);
        c->dev_bytes -= c->staging_bytes;
        c->staging = nullptr;
        c->staging_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->staging, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->staging = nullptr;
        return fail(c, CMRT_ENOMEM, "cudaMalloc of %zu staging bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    c->staging_bytes = bytes;
    c->dev_bytes += bytes;
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
    return &h->c;
}

cmrt_status set_device(Ctx* c) {
    int cur = -1;
    CK(c, cudaGetDevice(&cur));
    if (cur != c->device) CK(c, cudaSetDevice(c->device));
    return CMRT_OK;
}

void free_all(Ctx* c) {
    for (void*& b : c->buf)
        if (b) cudaFree(b), b = nullptr;
    if (c->d_flag) cudaFree(c->d_flag), c->d_flag = nullptr;
    if (c->d_partials) cudaFree(c->d_partials), c->d_partials = nullptr;
    if (c->d_diag) cudaFree(c->d_diag), c->d_diag = nullptr;
    if (c->staging) cudaFree(c->staging), c->staging = nullptr;
}

cmrt_status check_flag(Ctx* c) {
    unsigned h = 0;
    CK(c, cudaMemcpyAsync(&h, c->d_flag, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (h) return fail(c, CMRT_ENONFINITE, "non-finite density in the state before step %lld", (long long)c->t);
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
    // inputs: copy host arrays into staging (after an FP32 state area when the
    // state is stored in 16 bits and has to be encoded from FP32)
    const float* d_rn = rho_n0;
    const float* d_u = u0;
    const bool rn_host = rho_n0 && !is_device_ptr(rho_n0);
    const bool u_host = u0 && !is_device_ptr(u0);
    const bool packed = p->precision != 0;
    const size_t in_off = packed ? 18 * n : 0;
    if (rn_host || u_host || packed) {
        if (ensure_staging(c, (in_off + ((rn_host || u_host) ? 3 * n : 0)) * sizeof(float)) != CMRT_OK)
            return bail(CMRT_ENOMEM);
        if (rn_host) {
            if (cudaMemcpyAsync(c->staging + in_off, rho_n0, n * sizeof(float), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess) {
                fail(c, CMRT_ECUDA, "copy of rho_n0 failed");
                return bail(CMRT_ECUDA);
            }
            d_rn = c->staging + in_off;
        }
        if (u_host) {
            if (cudaMemcpyAsync(c->staging + in_off + n, u0, 2 * n * sizeof(float), cudaMemcpyHostToDevice,
                                c->stream) != cudaSuccess) {
                fail(c, CMRT_ECUDA, "copy of u0 failed");
                return bail(CMRT_ECUDA);
            }
            d_u = c->staging + in_off + n;
        }
    }
    float* post32 = packed ? c->staging : static_cast<float*>(c->buf[0]);
    cudaError_t e = cmrt::launch_init_fp64(d_rn, d_u, p->nx, p->ny, p->wall_y, p->rho0_r, p->rho0_b, p->alpha_r,
                                           p->alpha_b, post32, c->stream);
    if (e == cudaSuccess && packed) {
        c->launches++;
        e = cmrt::launch_encode(post32, c->sp, c->buf[0], c->stream);
    }
    if (e != cudaSuccess) {
        fail(c, CMRT_ECUDA, "init kernel launch failed: %s", cudaGetErrorString(e));
        return bail(CMRT_ECUDA);
    }
    c->launches++;
    if (rn_host || u_host || packed) {
        // host buffers may be reused by the caller as soon as we return, and the
        // staging area by the next call
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            fail(c, CMRT_ECUDA, "stream synchronisation failed");
            return bail(CMRT_ECUDA);
        }
    }
    c->cur = 0;
    c->t = 0;
    *out = h;
    return CMRT_OK;
}

cmrt_status cmrt_step(cmrt_ctx* h, int64_t n) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (n < 0) return fail(c, CMRT_EINVAL, "n must be >= 0");
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    for (int64_t k = 0; k < n; ++k) {
        CK(c, cmrt::launch_step(c->buf[c->cur], c->buf[c->cur ^ 1], c->sp, c->rows, c->d_flag, c->stream));
        c->launches++;
        c->cur ^= 1;
        c->t++;
        if (c->p.diag_every > 0 && (c->t % c->p.diag_every) == 0) {
            cmrt_status st = check_flag(c);
            if (st != CMRT_OK) return st;
        }
    }
    return CMRT_OK;
}

cmrt_status cmrt_fields(cmrt_ctx* h, float* rho_r, float* rho_b, float* ux, float* uy, float* p) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    const size_t n = cells(*c);
    float* outs[5] = {rho_r, rho_b, ux, uy, p};
    float* dev[5];
    bool any_host = false;
    for (int k = 0; k < 5; ++k) any_host |= (outs[k] && !is_device_ptr(outs[k]));
    if (any_host && ensure_staging(c, 5 * n * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
    for (int k = 0; k < 5; ++k) {
        if (!outs[k]) dev[k] = nullptr;
        else dev[k] = is_device_ptr(outs[k]) ? outs[k] : c->staging + k * n;
    }
    CK(c, cmrt::launch_fields(c->buf[c->cur], c->sp, c->rows, cmrt::FieldOut{dev[0], dev[1], dev[2], dev[3], dev[4]},
                              c->stream));
    c->launches++;
    if (any_host) {
        for (int k = 0; k < 5; ++k)
            if (outs[k] && dev[k] != outs[k])
                CK(c, cudaMemcpyAsync(outs[k], dev[k], n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return CMRT_OK;
}

cmrt_status cmrt_diagnostics(cmrt_ctx* h, double out[6]) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    if (!out) return fail(c, CMRT_EINVAL, "out is NULL");
    if (set_device(c) != CMRT_OK) return CMRT_ECUDA;
    CK(c, cmrt::launch_diag_partials(c->buf[c->cur], c->sp, c->rows, c->d_partials, c->stream));
    CK(c, cmrt::launch_diag_reduce(c->d_partials, c->n_partials, c->d_diag, c->stream));
    c->launches += 2;
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
    const bool packed = c->p.precision != 0;
    // staging: [FP32 post-collision planes (16-bit storage)] [pre-collision copy (host dst)]
    const size_t need = (packed ? n18 : 0) + (host ? n18 : 0);
    if (need && ensure_staging(c, need * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
    const float* post32 = static_cast<const float*>(c->buf[c->cur]);
    if (packed) {
        CK(c, cmrt::launch_decode(c->buf[c->cur], c->sp, c->staging, c->stream));
        c->launches++;
        post32 = c->staging;
    }
    float* d = host ? c->staging + (packed ? n18 : 0) : dst;
    CK(c, cmrt::launch_stream_out(post32, c->sp, d, c->stream));
    c->launches++;
    if (host) {
        CK(c, cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
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
    const bool packed = c->p.precision != 0;
    // staging: [FP32 post-collision planes (16-bit storage)] [pre-collision copy (host src)]
    const size_t need = (packed ? n18 : 0) + (host ? n18 : 0);
    if (need && ensure_staging(c, need * sizeof(float)) != CMRT_OK) return CMRT_ENOMEM;
    if (host) {
        float* hs = c->staging + (packed ? n18 : 0);
        CK(c, cudaMemcpyAsync(hs, src, bytes, cudaMemcpyHostToDevice, c->stream));
        s = hs;
    }
    float* post32 = packed ? c->staging : static_cast<float*>(c->buf[c->cur]);
    CK(c, cmrt::launch_unstream_in(s, c->sp, post32, c->stream));
    c->launches++;
    if (packed) {
        CK(c, cmrt::launch_encode(post32, c->sp, c->buf[c->cur], c->stream));
        c->launches++;
    }
    if (host || packed) CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

cmrt_status cmrt_synchronize(cmrt_ctx* h) {
    Ctx* c = live(h);
    if (!c) return CMRT_ESTATE;
    CK(c, cudaStreamSynchronize(c->stream));
    return CMRT_OK;
}

int64_t cmrt_time(const cmrt_ctx* h) { return h ? h->c.t : -1; }

int64_t cmrt_launch_count(const cmrt_ctx* h) { return h ? h->c.launches : -1; }

size_t cmrt_device_bytes(const cmrt_ctx* h) { return h ? h->c.dev_bytes : 0; }

void cmrt_destroy(cmrt_ctx* h) {
    if (!h) return;
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
// reduction of the state: code recording a CUDA graph (cudaMalloc is not a
// capturable operation), code running under a hard device-memory cap or a
// custom allocator that forbids ad-hoc allocations, and code that must not
// let cudaMalloc/cudaFree synchronise the device in the middle of a pipeline.
// For them this entry point works on caller-owned populations and uses a
// fixed scratch area compiled into the library instead of a context.
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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(nullptr, CMRT_ECUDA, "no usable current CUDA device");
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
    if (!is_device_ptr(pops)) return fail(nullptr, CMRT_EINVAL, "pops must be device memory of the current device");
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
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
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

