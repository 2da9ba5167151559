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

// 16-bit storage (see cmrt_step.cu): a node keeps (rho_R, rho_B) and the
// rest populations (R_0, B_0) in FP32 and twelve 16-bit (red, blue) pairs:
// four reference dipoles D_j and the deviations d_C,i of links 1..8, decoded
// as C_i = rho_C psi_i +/- D_C,dip(i) + d_C,i / 2^k.  Here the dipoles are
// those of the record's own populations: their velocity j / rho and their
// segregation vector S, the antisymmetric part of the colour split C_i -
// (rho_C / rho) f_i along x and y (a state the step wrote gets its own S
// back; any other state a valid one, whose rest the deviations carry).  The
// rest populations are the remainder of rho_C after the moving links as the
// step kernel decodes them, so that decoding conserves rho_C.  The reference
// weights of the axis and diagonal links as (red, blue) pairs, with the step
// kernel's rounding (Layout16::weights): the node's mixture
// (precision_reference 0) or per-colour constants; the diagonal weight a
// quarter of the axis one (flag 0, the equilibrium's shape) or the rest
// state with the same mass and energy and ghost moment N = 0 (flag 1).  The
// flag is the lowest bit of D_0's red half; the encoder gives each record
// the shape nearer to its own N.
__device__ __forceinline__ void ref_weights(float rr, float rb, bool nfree, const StepParams& P, float2& wa,
                                            float2& wd) {
    float pr, pb;
    if (P.precision_reference == 0) {
        float s5 = fmaf(P.mix_r, rr, P.mix_b * rb) * __fdividef(1.0f, rr + rb);
        s5 = fminf(fmaxf(s5, 0.0f), 0.25f);
        pr = pb = __fsub_rn(__fadd_rn(s5, 0.5f), 0.5f);
    } else {
        pr = P.psi_r[1];
        pb = P.psi_b[1];
    }
    if (nfree) {
        wa = make_float2(__fmaf_rn(pr, 0.5f, 1.0f / 18.0f), __fmaf_rn(pb, 0.5f, 1.0f / 18.0f));
        wd = make_float2(__fmaf_rn(pr, 0.5f, -1.0f / 36.0f), __fmaf_rn(pb, 0.5f, -1.0f / 36.0f));
    } else {
        wa = make_float2(pr, pb);
        wd = make_float2(__fmul_rn(pr, 0.25f), __fmul_rn(pb, 0.25f));
    }
}
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
        float r[9], b[9], rr = 0.f, rb = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            r[i] = post[i * nodes + n];
            b[i] = post[(9 + i) * nodes + n];
            rr += r[i];
            rb += b[i];
            jx += lcx(i) * (r[i] + b[i]);
            jy += lcy(i) * (r[i] + b[i]);
        }
        const float rho = rr + rb;
        // S from the antisymmetric part of the red split a_i = R_i - (rho_R / rho) f_i:
        // a_8 - a_4 = 2 w_axis S_x, a_2 - a_6 = 2 w_axis S_y
        const float kr = rr / rho;
        const float a8 = fmaf(-kr, r[8] + b[8], r[8]), a4 = fmaf(-kr, r[4] + b[4], r[4]);
        const float a2 = fmaf(-kr, r[2] + b[2], r[2]), a6 = fmaf(-kr, r[6] + b[6], r[6]);
        unsigned* pairs = reinterpret_cast<unsigned*>(state + nodes * 16);
        // the reference shape: the one whose ghost moment N (Dellar's weights
        // 1, -2, 4 for the rest, axis and diagonal links) is nearer the record's
        // (a shape's N per unit density: 1 - 12 (psi_a - psi_d); 0 for the N-free one)
        float2 wa0, wd0;
        ref_weights(rr, rb, false, P, wa0, wd0);
        const float npl = rr * (1.0f - 12.0f * (wa0.x - wd0.x)) + rb * (1.0f - 12.0f * (wa0.y - wd0.y));
        float N = r[0] + b[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) N = fmaf((i & 1) ? 4.0f : -2.0f, r[i] + b[i], N);
        const bool nfree = fabsf(N) < fabsf(N - npl);
        float2 D[4];
        dipoles16(rr, rb, jx / rho, jy / rho, (a8 - a4) * (0.5f / lw(8)), (a2 - a6) * (0.5f / lw(2)), D);
        for (int j = 0; j < 4; ++j) {
            unsigned h = pack2(D[j].x, D[j].y, P.precision);
            if (j == 0) h = (h & ~1u) | (nfree ? 1u : 0u);  // the flag
            pairs[j * nodes + n] = h;
            D[j] = unpack2(h, P.precision);  // the dipole as stored
        }
        float2 wa, wd;
        ref_weights(rr, rb, nfree, P, wa, wd);
        const float2 refa = make_float2(__fmul_rn(rr, wa.x), __fmul_rn(rb, wa.y));  // the decoder's
        const float2 refd = make_float2(__fmul_rn(rr, wd.x), __fmul_rn(rb, wd.y));
        const float S = P.dev_scale;  // a power of two: the scaled deviation is the deviation, scaled exactly
        float sr = 0.f, sb = 0.f;     // the moving links as decoded, for the rest populations
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float wr = (i & 1) ? wd.x : wa.x, wb = (i & 1) ? wd.y : wa.y;
            const float2 Dj = D[dip_index(i)];
            const float sg = dip_neg(i) ? -1.0f : 1.0f;
            const float cr = r[i] - sg * Dj.x, cb = b[i] - sg * Dj.y;
            const unsigned h = pack2(fmaf(-rr * S, wr, cr * S), fmaf(-rb * S, wb, cb * S), P.precision);
            pairs[(3 + i) * nodes + n] = h;
            const float2 dd = unpack2(h, P.precision);
            const float2 ref = (i & 1) ? refd : refa;
            float xr = __fmaf_rn(dd.x, P.dev_unscale, ref.x);
            float xb = __fmaf_rn(dd.y, P.dev_unscale, ref.y);
            if (dip_neg(i)) {
                xr = __fmaf_rn(Dj.x, -1.0f, xr);
                xb = __fmaf_rn(Dj.y, -1.0f, xb);
            } else {
                xr = __fadd_rn(xr, Dj.x);
                xb = __fadd_rn(xb, Dj.y);
            }
            sr = __fadd_rn(sr, xr);
            sb = __fadd_rn(sb, xb);
        }
        float2* own = reinterpret_cast<float2*>(state) + n;
        own[0] = make_float2(rr, rb);
        own[nodes] = make_float2(__fsub_rn(rr, sr), __fsub_rn(rb, sb));
    }
}

__global__ void k_decode(const char* __restrict__ state, StepParams P, float* __restrict__ post) {
    const size_t nodes = static_cast<size_t>(P.nx) * P.ny;
    for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < nodes;
         n += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float2* own = reinterpret_cast<const float2*>(state) + n;
        const float2 rho = own[0], rest = own[nodes];
        const unsigned* pairs = reinterpret_cast<const unsigned*>(state + nodes * 16);
        // the step kernel's decode: the reference pair rho psi_i plus the
        // deviation, rounded once; then the dipole
        float2 wa, wd;
        ref_weights(rho.x, rho.y, (pairs[n] & 1u) != 0, P, wa, wd);
        const float2 refa = make_float2(__fmul_rn(rho.x, wa.x), __fmul_rn(rho.y, wa.y));
        const float2 refd = make_float2(__fmul_rn(rho.x, wd.x), __fmul_rn(rho.y, wd.y));
        post[n] = rest.x;
        post[9 * nodes + n] = rest.y;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float2 d = unpack2(pairs[(3 + i) * nodes + n], P.precision);
            const float2 ref = (i & 1) ? refd : refa;
            float cr = __fmaf_rn(d.x, P.dev_unscale, ref.x);
            float cb = __fmaf_rn(d.y, P.dev_unscale, ref.y);
            const float2 D = unpack2(pairs[dip_index(i) * nodes + n], P.precision);
            if (dip_neg(i)) {
                cr = __fmaf_rn(D.x, -1.0f, cr);
                cb = __fmaf_rn(D.y, -1.0f, cb);
            } else {
                cr = __fadd_rn(cr, D.x);
                cb = __fadd_rn(cb, D.y);
            }
            post[i * nodes + n] = cr;
            post[(9 + i) * nodes + n] = cb;
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
