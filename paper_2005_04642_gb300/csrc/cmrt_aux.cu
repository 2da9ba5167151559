// Initialisation and state import/export kernels of libcmrt.
//
// The library stores the post-collision populations P_{t-1}; the state of
// the paper at time t is the pre-collision f(t) = stream(P_{t-1})
// (Eq. equ_evolution).  These kernels translate between the two, and build
// the initial state from a colour field and a velocity field.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cmrt_device.cuh"

namespace cmrt {
namespace {

__device__ __forceinline__ int wrapx(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// Initial state (t = 0): at each node the equilibrium of Eq. equ_equ with
// phi_i of Eq. eq_phi, split by colour as C_i = (rho_C / rho) f^(0)_i, from
// rho_R = rho0_R (1 + rho^N_0)/2 and rho_B = rho0_B (1 - rho^N_0)/2 (which
// inverts Eq. equ_rhoN_def).  f^(0)_i = rho phi_i + w_i rho Q_i with the
// velocity part Q_i = 3 c.u + 9/2 (c.u)^2 - 3/2 u^2.  The colour split and
// rho phi_i (three link classes per node) are FP64; Q_i, small and taken
// from FP32 velocities, is FP32 (its rounding is far below a float ulp of
// C_i), and each C_i is one FP64 FMA rounded once to FP32.  Each node
// writes its links to where the first step's pull streaming will find them:
// f_i(r) goes to P_i(r - c_i), or to P_opp(i)(r) where r - c_i lies beyond a
// wall (half-way bounce-back).
struct InitIn {
    const float* rho_n0;
    const float* u0;
    double rho0_r, rho0_b, alpha_r, alpha_b;
};

// one thread per node: x from the block column, y from the block row (a
// stride over rows beyond the grid's y extent)
__global__ void k_init(InitIn in, int nx, int ny, int walls, float* __restrict__ post) {
    const size_t plane = static_cast<size_t>(nx) * ny;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;  // the source columns x - c_ix
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const size_t n = static_cast<size_t>(y) * nx + x;
        const double rn = in.rho_n0 ? static_cast<double>(in.rho_n0[n]) : -1.0;
        const float fux = in.u0 ? in.u0[n] : 0.0f;
        const float fuy = in.u0 ? in.u0[plane + n] : 0.0f;
        const double rr = in.rho0_r * (1.0 + rn) * 0.5;
        const double rb = in.rho0_b * (1.0 - rn) * 0.5;
        const double rho = rr + rb;
        const double inv_rho = 1.0 / rho;
        const double ar = rr * inv_rho, ab = rb * inv_rho;
        // rho phi_i and w_i rho of the rest, axis and diagonal links
        const double rphi0 = in.alpha_r * rr + in.alpha_b * rb;
        const double rphim = 1.8 * ((1.0 - in.alpha_r) * rr + (1.0 - in.alpha_b) * rb);
        const double rphi_c[3] = {rphi0, rphim * (1.0 / 9.0), rphim * (1.0 / 36.0)};
        const double wrho_c[3] = {rho * (4.0 / 9.0), rho * (1.0 / 9.0), rho * (1.0 / 36.0)};
        const float usq = fmaf(fux, fux, fuy * fuy);
        // at rest Q_i = 0 and f^(0)_i = rho phi_i: the three link classes'
        // colour parts, each rounded once, serve all nine links (the same
        // values the per-link form gives, with a third of its FP64 work)
        const bool rest = fux == 0.0f && fuy == 0.0f;
        float r_c[3], b_c[3];
        if (rest) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                r_c[c] = static_cast<float>(ar * rphi_c[c]);
                b_c[c] = static_cast<float>(ab * rphi_c[c]);
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cls = i == 0 ? 0 : ((i & 1) ? 2 : 1);
            float vr, vb;
            if (rest) {
                vr = r_c[cls];
                vb = b_c[cls];
            } else {
                const float cu = float(lcx(i)) * fux + float(lcy(i)) * fuy;
                const float Q = fmaf(4.5f * cu, cu, fmaf(3.0f, cu, -1.5f * usq));
                const double f0 = fma(wrho_c[cls], static_cast<double>(Q), rphi_c[cls]);
                vr = static_cast<float>(ar * f0);
                vb = static_cast<float>(ab * f0);
            }
            const int ty = y - lcy(i);
            size_t dst;
            int li;
            if (walls && (ty < 0 || ty >= ny)) {
                dst = n;
                li = lopp(i);
            } else {
                const int sx = lcx(i) > 0 ? xm : (lcx(i) < 0 ? xp : x);
                dst = static_cast<size_t>(ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty)) * nx + sx;
                li = i;
            }
            post[li * plane + dst] = vr;
            post[(9 + li) * plane + dst] = vb;
        }
    }
}

// pre_i(r) = P_i(r - c_i), or P_opp(i)(r) where r - c_i lies beyond a wall.
__global__ void k_stream_out(const float* __restrict__ post, int nx, int ny, int walls, float* __restrict__ pre) {
    const size_t plane = static_cast<size_t>(nx) * ny;
    for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < plane;
         n += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int y = static_cast<int>(n / nx);
        const int x = static_cast<int>(n - static_cast<size_t>(y) * nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sy = y - lcy(i);
            for (int c = 0; c < 2; ++c) {
                float v;
                if (walls && (sy < 0 || sy >= ny)) {
                    v = post[(c * 9 + lopp(i)) * plane + n];
                } else {
                    v = post[(c * 9 + i) * plane + static_cast<size_t>(wrapx(sy, ny)) * nx + wrapx(x - lcx(i), nx)];
                }
                pre[(c * 9 + i) * plane + n] = v;
            }
        }
    }
}

// Inverse of k_stream_out: P_i(s) = pre_i(s + c_i), or pre_opp(i)(s) where
// s + c_i lies beyond a wall.
__global__ void k_unstream_in(const float* __restrict__ pre, int nx, int ny, int walls, float* __restrict__ post) {
    const size_t plane = static_cast<size_t>(nx) * ny;
    for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < plane;
         n += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int y = static_cast<int>(n / nx);
        const int x = static_cast<int>(n - static_cast<size_t>(y) * nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ty = y + lcy(i);
            for (int c = 0; c < 2; ++c) {
                float v;
                if (walls && (ty < 0 || ty >= ny)) {
                    v = pre[(c * 9 + lopp(i)) * plane + n];
                } else {
                    v = pre[(c * 9 + i) * plane + static_cast<size_t>(wrapx(ty, ny)) * nx + wrapx(x + lcx(i), nx)];
                }
                post[(c * 9 + i) * plane + n] = v;
            }
        }
    }
}

// 16-bit storage (see cmrt_step.cu): a node keeps (rho'_R, rho'_B) in FP32 and,
// per link, the deviations d_C,i = C_i - rho_C psi_i as a 16-bit pair, with
// rho_C the sum of the record's own nine populations of colour C and
// rho'_C = rho_C - sum_i round(d_C,i), so that decoding conserves rho_C.
// The reference weights (rest, axis, diagonal) as (red, blue) pairs: the
// node's mixture (precision_reference 0; the same exact-sum rounding as the
// step kernel's) or per-colour constants.
__device__ __forceinline__ void ref_weights(float rr, float rb, const StepParams& P, float2 (&w)[3]) {
    if (P.precision_reference == 0) {
        float s5 = fmaf(P.mix_r, rr, P.mix_b * rb) * __fdividef(1.0f, rr + rb);
        s5 = fminf(fmaxf(s5, 0.0f), 0.25f);
        const float pa = __fsub_rn(__fadd_rn(s5, 0.5f), 0.5f);
        const float p0 = fmaf(-4.0f, pa, 1.0f - pa);
        w[0] = make_float2(p0, p0);
        w[1] = make_float2(pa, pa);
        w[2] = make_float2(0.25f * pa, 0.25f * pa);
    } else {
        for (int k = 0; k < 3; ++k) w[k] = make_float2(P.psi_r[k], P.psi_b[k]);
    }
}
__device__ __forceinline__ int ref_class(int i) { return i == 0 ? 0 : ((i & 1) ? 2 : 1); }
__device__ __forceinline__ unsigned pack2(float a, float b, int precision) {
    if (precision == kPrecF16) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned*>(&h);
}
__device__ __forceinline__ float2 unpack2(unsigned v, int precision) {
    if (precision == kPrecF16) return __half22float2(*reinterpret_cast<const __half2*>(&v));
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v));
}

__global__ void k_encode(const float* __restrict__ post, StepParams P, char* __restrict__ state) {
    const size_t nodes = static_cast<size_t>(P.nx) * P.ny;
    for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < nodes;
         n += static_cast<size_t>(gridDim.x) * blockDim.x) {
        float r[9], b[9], rr = 0.f, rb = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            r[i] = post[i * nodes + n];
            b[i] = post[(9 + i) * nodes + n];
            rr += r[i];
            rb += b[i];
        }
        unsigned* dev = reinterpret_cast<unsigned*>(state + nodes * 8);
        float2 w[3];
        ref_weights(rr, rb, P, w);
        float er = 0.f, eb = 0.f;  // rounded deviations, absorbed by the stored densities
        const float S = P.dev_scale;  // a power of two: the scaled deviation is the deviation, scaled exactly
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float2 wi = w[ref_class(i)];
            const unsigned h = pack2(fmaf(-rr * S, wi.x, r[i] * S), fmaf(-rb * S, wi.y, b[i] * S), P.precision);
            const float2 back = unpack2(h, P.precision);
            er = fmaf(back.x, P.dev_unscale, er);
            eb = fmaf(back.y, P.dev_unscale, eb);
            dev[i * nodes + n] = h;
        }
        reinterpret_cast<float2*>(state)[n] = make_float2(rr - er, rb - eb);
    }
}

__global__ void k_decode(const char* __restrict__ state, StepParams P, float* __restrict__ post) {
    const size_t nodes = static_cast<size_t>(P.nx) * P.ny;
    for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < nodes;
         n += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float2 rho = reinterpret_cast<const float2*>(state)[n];
        const unsigned* dev = reinterpret_cast<const unsigned*>(state + nodes * 8);
        float2 w[3];
        ref_weights(rho.x, rho.y, P, w);
        // the step kernel's decode: reference pair rho' psi rounded once, plus the deviation
        float2 ref[3];
        for (int k = 0; k < 3; ++k) ref[k] = make_float2(__fmul_rn(rho.x, w[k].x), __fmul_rn(rho.y, w[k].y));
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float2 d = unpack2(dev[i * nodes + n], P.precision);
            post[i * nodes + n] = __fmaf_rn(d.x, P.dev_unscale, ref[ref_class(i)].x);
            post[(9 + i) * nodes + n] = __fmaf_rn(d.y, P.dev_unscale, ref[ref_class(i)].y);
        }
    }
}

dim3 flat_grid(size_t n) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks == 0) blocks = 1;
    return dim3(static_cast<unsigned>(blocks));
}

}  // namespace

// rho0/alpha are passed through StepParams' sources in FP64 by the caller.
cudaError_t launch_init_fp64(const float* rho_n0, const float* u0, int nx, int ny, int walls, double rho0_r,
                             double rho0_b, double alpha_r, double alpha_b, float* post, cudaStream_t s) {
    InitIn in{rho_n0, u0, rho0_r, rho0_b, alpha_r, alpha_b};
    const dim3 g(static_cast<unsigned>((nx + 127) / 128), static_cast<unsigned>(ny < 65535 ? ny : 65535));
    k_init<<<g, 128, 0, s>>>(in, nx, ny, walls, post);
    return cudaGetLastError();
}

cudaError_t launch_encode(const float* post32, const StepParams& P, void* state, cudaStream_t s) {
    k_encode<<<flat_grid(static_cast<size_t>(P.nx) * P.ny), 256, 0, s>>>(post32, P, static_cast<char*>(state));
    return cudaGetLastError();
}

cudaError_t launch_decode(const void* state, const StepParams& P, float* post32, cudaStream_t s) {
    k_decode<<<flat_grid(static_cast<size_t>(P.nx) * P.ny), 256, 0, s>>>(static_cast<const char*>(state), P, post32);
    return cudaGetLastError();
}

cudaError_t launch_stream_out(const float* post, const StepParams& P, float* pre, cudaStream_t s) {
    k_stream_out<<<flat_grid(static_cast<size_t>(P.nx) * P.ny), 256, 0, s>>>(post, P.nx, P.ny, P.wall_y, pre);
    return cudaGetLastError();
}

cudaError_t launch_unstream_in(const float* pre, const StepParams& P, float* post, cudaStream_t s) {
    k_unstream_in<<<flat_grid(static_cast<size_t>(P.nx) * P.ny), 256, 0, s>>>(pre, P.nx, P.ny, P.wall_y, post);
    return cudaGetLastError();
}

}  // namespace cmrt
