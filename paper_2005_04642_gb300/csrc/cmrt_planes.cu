// Per-node plane passes (one thread per node, intermediate fields in global
// planes) for FP32 storage: the step with App. B's order-6 gradient stencil,
// and the discrete adjoint (reverse mode) of the step, arXiv 2005.04642,
// Sec. 2, App. A, App. B.
//
// Order-6 step.  App. B's non-compact stencil d_a X = sum_N a_N sum_i w_i
// X(r + N c_i) c_ia, (a_1, a_2, a_3) = (9/2, -9/10, 1/10), has radius 3; used
// for grad rho^N and grad Phi' it widens the step's dependency radius from 3
// to 5.  Rather than a second fused kernel with a wider halo and deeper
// rings, the order-6 step runs as four passes over planes: moments, grad
// rho^N, K / G / u (k_fwd_*, shared with the adjoint), then k_step_planes
// (grad Phi', div u, collision, recolour, store).
//
// The forward step maps the post-collision state P_{t-1} to P_t:
//   f(t) = gather(P_{t-1})                       (streaming, Eq. equ_evolution)
//   P_t  = CR(f(t))                              (collide + recolour)
// with CR built from the moments, grad rho^N, the unit normal, the curvature,
// the force and force-adjusted velocity, grad Phi', div u, the correction
// tensor, the MRT collision and the recolour.  Its adjoint is
//   lam_P(t-1) = gather^T( CR'(f(t))^T lam_P(t) ),
// evaluated here as a chain of per-node passes over whole planes (one thread
// per node), the reverse of the forward chain:
//   k_fwd_moments   rho_R, rho_B, j, colour fractions, Phi'  (recomputed)
//   k_fwd_normal    grad rho^N                             (recomputed)
//   k_fwd_force     K, G, u                                (recomputed)
//   k_rev_collide   reverse of recolour, reconstruction, relaxation,
//                   equilibria, sources, correction tensor, lambda_3
//   k_rev_force     reverse of div u and of u = (j + G/2)/rho, G
//   k_rev_normal    reverse of K = div n-hat and n-hat = -g/max(|g|, eps)
//   k_rev_moments   reverse of grad rho^N, grad Phi', rho^N, Phi'
//   k_rev_gather    transpose of the streaming gather (bounce-back included)
// The transposed compact stencils are gathers: on a periodic lattice the
// transpose of d/dx is -d/dx; next to a wall the mirrored ghost reads add
// the terms of the row's own nodes with the ghost's parity.
//
// Parameter gradients (sigma, beta, lambda3_r, lambda3_b, g_acc) are reduced
// per CTA (FP32 within a warp, FP64 from there) and accumulated across steps
// in a per-CTA FP64 slot (no atomics: every launch of a pass uses the same
// grid, and the slots are summed once at the end).
#include <atomic>
#include <type_traits>

#include "cmrt_device.cuh"

namespace cmrt {
namespace {

constexpr int kAT = 128;  // threads per CTA (along x)

// Scratch planes, each float[ny][nx].
enum Plane : int {
    kRR = 0, kRB, kJX, kJY, kCHR, kCHB, kPHIP, kGX, kGY, kK, kGFX, kGFY, kUX, kUY,  // forward
    kFB0,                                                                   // 9 planes f-bar
    kRRB = kFB0 + 9, kRBB, kUXB, kUYB, kGFXB, kGFYB, kDPXB, kDPYB, kDIVUB, kGXB, kGYB, kRNB, kJXB, kJYB, kKB,
    kNumPlanes
};
static_assert(kNumPlanes == kAdjPlanes, "scratch plane count");
static_assert(kRR == kFwdRR && kRB == kFwdRB && kCHR == kFwdCHR && kCHB == kFwdCHB && kPHIP == kFwdPHIP &&
                  kGX == kFwdGX && kGY == kFwdGY && kK == kFwdK && kGFX == kFwdGFX && kGFY == kFwdGFY &&
                  kUX == kFwdUX && kJX == kFwdJX && kJY == kFwdJY && kFB0 == kFwdPlanes,
              "the forward planes lead the scratch planes, in the order the step kernel writes them");

// periodic image of v in [0, n); the integer modulo only for images more than
// one period away (lattices narrower than a stencil's reach)
__device__ __forceinline__ int wrap_to(int v, int n) {
    if (v >= 0 && v < n) return v;
    if (v < 0 && v + n >= 0) return v + n;
    if (v >= n && v - n < n) return v - n;
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// App. B coefficients a_N of the order-6 stencil
__host__ __device__ constexpr float order6_coef(int N) { return N == 1 ? 4.5f : (N == 2 ? -0.9f : 0.1f); }

// Neighbourhood of node (x, y) out to distance R in the planes: the periodic
// images of the columns x - R .. x + R and the offsets of the rows y - R ..
// y + R -- periodic images, or with walls W the mirror rows -1 - y' below
// y = -1/2 and 2 ny - 1 - y' above y = ny - 1/2, flagged because odd fields
// change sign there.  Computed once per thread, so every stencil read is a
// plain indexed load; a CTA covers part of one row, so the row offsets and
// the wall branches are uniform across it.
template <int R, bool W>
struct Nbh {
    int nx, ny, x, y;
    size_t n, o;  // plane size; this node
    int col[2 * R + 1];
    size_t row[2 * R + 1];
    bool mir[2 * R + 1];

    __device__ __forceinline__ Nbh(const StepParams& P, int x_, int y_) : nx(P.nx), ny(P.ny), x(x_), y(y_) {
        n = static_cast<size_t>(nx) * ny;
#pragma unroll
        for (int d = -R; d <= R; ++d) {
            col[d + R] = wrap_to(x + d, nx);
            int yy = y + d;
            bool m = false;
            if (W) {
                if (yy < 0) {
                    yy = -1 - yy;
                    m = true;
                } else if (yy >= ny) {
                    yy = 2 * ny - 1 - yy;
                    m = true;
                }
            } else {
                yy = wrap_to(yy, ny);
            }
            row[d + R] = static_cast<size_t>(yy) * nx;
            mir[d + R] = m;
        }
        o = row[R] + x;
    }

    // value of a plane at (x + dx, y + dy); `parity` multiplies a mirrored value
    __device__ __forceinline__ float val(const float* a, int dx, int dy, float parity) const {
        const float v = a[row[dy + R] + col[dx + R]];
        return (W && mir[dy + R]) ? parity * v : v;
    }

    // gradient of a plane at this node: the compact stencil (Sec. 2) for
    // ORDER 2, App. B's radius-3 stencil for ORDER 6
    template <int ORDER>
    __device__ __forceinline__ void grad(const float* a, float parity, float& gx, float& gy) const {
        static_assert(R >= (ORDER == 6 ? 3 : 1), "neighbourhood too small for the stencil");
        if (ORDER == 2) {
            const float e = val(a, 1, 0, parity), w = val(a, -1, 0, parity);
            const float n_ = val(a, 0, 1, parity), s = val(a, 0, -1, parity);
            const float ne = val(a, 1, 1, parity), nw = val(a, -1, 1, parity);
            const float se = val(a, 1, -1, parity), sw = val(a, -1, -1, parity);
            gx = ddx(e, w, ne, nw, se, sw);
            gy = ddy(n_, s, ne, nw, se, sw);
        } else {
            gx = 0.0f;
            gy = 0.0f;
#pragma unroll
            for (int N = 1; N <= 3; ++N) {
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const float v = val(a, N * lcx(i), N * lcy(i), parity);
                    if (lcx(i)) gx = fmaf(order6_coef(N) * lw(i) * float(lcx(i)), v, gx);
                    if (lcy(i)) gy = fmaf(order6_coef(N) * lw(i) * float(lcy(i)), v, gy);
                }
            }
        }
    }

    // transpose of one component (XC: x, else y) of grad<ORDER>, applied to
    // a plane: sum over the stencil's reach N c_i of k a(r - N c_i) for nodes
    // of the lattice, plus, next to a wall, the nodes whose stencil read this
    // node as a mirrored ghost (mirror row -1 - y' below, 2 ny - 1 - y' above)
    template <bool XC, int ORDER>
    __device__ __forceinline__ float gradT(const float* a, float parity) const {
        static_assert(R >= (ORDER == 6 ? 3 : 1), "neighbourhood too small for the stencil");
        float acc = 0.0f;
#pragma unroll
        for (int N = 1; N <= (ORDER == 6 ? 3 : 1); ++N) {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int c = XC ? lcx(i) : lcy(i);
                if (c == 0) continue;
                const float k = (ORDER == 6 ? order6_coef(N) : 3.0f) * lw(i) * float(c);
                const int dx = -N * lcx(i), dy = -N * lcy(i);  // the node r - N c_i
                if (!W) {
                    acc = fmaf(k, a[row[dy + R] + col[dx + R]], acc);
                } else {
                    if (!mir[dy + R]) acc = fmaf(k, a[row[dy + R] + col[dx + R]], acc);
                    const int yb = -1 - y + dy;  // node whose read below y = -1/2 mirrors onto row y
                    if (yb >= 0 && yb < ny && yb - dy < 0)
                        acc = fmaf(parity * k, a[static_cast<size_t>(yb) * nx + col[dx + R]], acc);
                    const int yt = 2 * ny - 1 - y + dy;  // same above y = ny - 1/2
                    if (yt >= 0 && yt < ny && yt - dy >= ny)
                        acc = fmaf(parity * k, a[static_cast<size_t>(yt) * nx + col[dx + R]], acc);
                }
            }
        }
        return acc;
    }

    // pre-collision populations of this node: f_i(r) = P_i(r - c_i), or
    // P_opp(i)(r) where r - c_i lies beyond a wall (half-way bounce-back)
    __device__ __forceinline__ void gather(const float* __restrict__ post, float (&fr)[9], float (&fb)[9]) const {
        static_assert(R >= 1, "the gather reads the nearest neighbours");
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            size_t src;
            int li = i;
            if (W && mir[-lcy(i) + R]) {
                li = lopp(i);
                src = o;
            } else {
                src = row[-lcy(i) + R] + col[-lcx(i) + R];
            }
            fr[i] = post[static_cast<size_t>(li) * n + src];
            fb[i] = post[static_cast<size_t>(9 + li) * n + src];
        }
    }
};

// the neighbourhood a stencil of the given order needs
template <int ORDER>
constexpr int reach() { return ORDER == 6 ? 3 : 1; }

// a node's own offset in the planes (per-node passes without a stencil)
struct Own {
    size_t n, o;
    __device__ __forceinline__ Own(const StepParams& P, int x, int y)
        : n(static_cast<size_t>(P.nx) * P.ny), o(static_cast<size_t>(y) * P.nx + x) {}
};

__device__ __forceinline__ float sum9f(const float (&v)[9]) {
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
}

// adjoint of g -> g / |g| (0 below kNormalTau): (I - e e^T) b / |g| above the
// threshold, 0 below it (the map is constant there)
__device__ __forceinline__ void normalise_T(float gx, float gy, float bx, float by, float& ox, float& oy) {
    const float mag2 = fmaf(gx, gx, gy * gy);
    if (mag2 >= kNormalTau * kNormalTau) {
        const float inv = rsqrtf(mag2);
        const float ex = gx * inv, ey = gy * inv;
        const float dot = fmaf(ex, bx, ey * by);
        ox = (bx - ex * dot) * inv;
        oy = (by - ey * dot) * inv;
    } else {
        ox = 0.0f;
        oy = 0.0f;
    }
}

// CTA reduction of up to 7 per-node terms, added into this CTA's FP64 slot:
// FP32 products and warp sums of 32 terms (GB300's FP64 rate is a small
// fraction of its FP32 rate), FP64 from the warp partials on -- across the
// CTA's warps and, in the slot, across all steps of the adjoint sweep.
template <int N>
__device__ __forceinline__ void add_partials(float (&v)[N], const int* slots, double* __restrict__ partials) {
    __shared__ double red[kAT / 32][N];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < N; ++j) red[warp][j] = v[j];
    __syncthreads();
    if (threadIdx.x < N) {
        double acc = 0.0;
        for (int w = 0; w < kAT / 32; ++w) acc += red[w][threadIdx.x];
        const size_t b = static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x;
        partials[b * kAdjSlots + slots[threadIdx.x]] += acc;
    }
}

// ----------------------------------------------------------------- forward recomputation
template <bool W>
__global__ void __launch_bounds__(kAT) k_fwd_moments(const float* __restrict__ post, const StepParams P,
                                                      float* __restrict__ S) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Nbh<1, W> L(P, x, y);
    float fr[9], fb[9];
    L.gather(post, fr, fb);
    const float rr = sum9f(fr), rb = sum9f(fb);
    float f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fr[i] + fb[i];
    const size_t o = L.o;
    S[kRR * L.n + o] = rr;
    S[kRB * L.n + o] = rb;
    S[kJX * L.n + o] = ((f[1] + f[7]) + f[8]) - ((f[3] + f[5]) + f[4]);
    S[kJY * L.n + o] = ((f[1] + f[3]) + f[2]) - ((f[5] + f[7]) + f[6]);
    // colour fractions chi_R = a / (a + b), chi_B = b / (a + b), rho^N = chi_R - chi_B
    // (Eq. equ_rhoN_def); the smaller one carries the colour gradient of a
    // nearly pure region without the cancellation of rho^N near -1 or +1
    const float a = rr * P.inv_rho0_r, b = rb * P.inv_rho0_b;
    const float inv = 1.0f / (a + b);
    S[kCHR * L.n + o] = a * inv;
    S[kCHB * L.n + o] = b * inv;
    S[kPHIP * L.n + o] = fmaf(P.phip_r, rr, P.phip_b * rb);  // App. A, Phi'
}

template <int ORDER, bool W>
__global__ void __launch_bounds__(kAT) k_fwd_normal(const StepParams P, float* __restrict__ S) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Nbh<reach<ORDER>(), W> L(P, x, y);
    // grad rho^N = 2 grad chi_R = -2 grad chi_B (the stencil weights sum to
    // zero): the same stencil, evaluated on the fraction that is small here
    const size_t o = L.o;
    float gx, gy;
    const bool red_minor = S[kCHR * L.n + o] <= 0.5f;
    const float* ch = S + (red_minor ? kCHR : kCHB) * L.n;
    L.template grad<ORDER>(ch, 1.0f, gx, gy);
    gx *= red_minor ? 2.0f : -2.0f;
    gy *= red_minor ? 2.0f : -2.0f;
    S[kGX * L.n + o] = gx;
    S[kGY * L.n + o] = gy;
}

__device__ __forceinline__ void normal_of(float gx, float gy, float& nx, float& ny) {
    const float mag2 = fmaf(gx, gx, gy * gy);
    const float inv = (mag2 >= kNormalTau * kNormalTau) ? rsqrtf(mag2) : 0.0f;
    nx = -gx * inv;
    ny = -gy * inv;
}

template <bool W>
__global__ void __launch_bounds__(kAT) k_fwd_force(const StepParams P, float* __restrict__ S) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Nbh<1, W> L(P, x, y);
    float K = P.fixed_K;
    if (P.curvature_mode == 0) {
        // K = div n-hat with n-hat of the neighbours (x even, y odd beyond a wall)
        float nxv[9], nyv[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const size_t o = L.row[lcy(i) + 1] + L.col[lcx(i) + 1];
            normal_of(S[kGX * L.n + o], S[kGY * L.n + o], nxv[i], nyv[i]);
            if (W && L.mir[lcy(i) + 1]) nyv[i] = -nyv[i];
        }
        K = ddx(nxv[8], nxv[4], nxv[1], nxv[3], nxv[7], nxv[5]) + ddy(nyv[2], nyv[6], nyv[1], nyv[3], nyv[7], nyv[5]);
    }
    const size_t o = L.o;
    const float gx = S[kGX * L.n + o], gy = S[kGY * L.n + o];
    const float rho = S[kRR * L.n + o] + S[kRB * L.n + o];
    const float hk = P.half_sigma * K;
    const float Gx = fmaf(hk, gx, fmaf(rho, P.gacc_x, P.gvol_x));
    const float Gy = fmaf(hk, gy, fmaf(rho, P.gacc_y, P.gvol_y));
    S[kK * L.n + o] = K;
    S[kGFX * L.n + o] = Gx;
    S[kGFY * L.n + o] = Gy;
    S[kUX * L.n + o] = fmaf(0.5f, Gx, S[kJX * L.n + o]) / rho;
    S[kUY * L.n + o] = fmaf(0.5f, Gy, S[kJY * L.n + o]) / rho;
}

// ----------------------------------------------------------------- reverse passes
// Reverse of the per-node collision and recolour (App. A Eqs. 38, eq84;
// Eq. eq_re_color) at one node: the adjoints of the node's inputs from the
// adjoint (lamr, lamb) of its post-collision populations.  Inputs: the
// pre-collision populations f, the colour densities, the force-adjusted
// velocity, the force, grad rho^N, rho^N, grad Phi' and div u.
struct RevCollide {
    float fbar[9];  // M^T m-bar: the common part of the population adjoint
    float rrb, rbb, uxb, uyb, Gxb, Gyb, dPxb, dPyb, divub, gxb, gyb, rnb;
    float acc[3];   // dJ/d(beta, lambda3_r, lambda3_b) of this node
};
__device__ __forceinline__ void rev_collide_node(const float (&f)[9], float rr, float rb, float ux, float uy, float Gx,
                                                 float Gy, float gx, float gy, float rn, float dPx, float dPy,
                                                 float divu, const float (&lamr)[9], const float (&lamb)[9],
                                                 const StepParams& P, RevCollide& out) {
    out.acc[0] = out.acc[1] = out.acc[2] = 0.0f;  // lambda3 terms stay 0 with constant eta
    const float rho = rr + rb, ir = 1.0f / rho, ir2 = ir * ir;
    // ---- forward values at this node
    float nu, dnu_drn = 0.0f;
    if (P.visc_mode == 0) {
        nu = fmaf(0.5f * (P.nu_r - P.nu_b), rn, 0.5f * (P.nu_r + P.nu_b));
        dnu_drn = 0.5f * (P.nu_r - P.nu_b);
    } else {
        nu = P.eta * ir;
    }
    const float lam3 = 2.0f / fmaf(6.0f, nu, 1.0f);
    const float a = fmaf(-0.5f, lam3, 1.0f);
    const float hx = Gx - dPx, hy = Gy - dPy;
    const float iso = fmaf(ux, dPx, fmaf(uy, dPy, -rho * divu * (1.0f / 3.0f)));
    const float Cxx = a * fmaf(2.0f * ux, hx, -iso);
    const float Cyy = a * fmaf(2.0f * uy, hy, -iso);
    const float Cxy = a * fmaf(ux, hy, uy * hx);
    float m[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float h = p == 0 ? 1.0f : p == 1 ? float(lcx(i)) : p == 2 ? float(lcy(i))
                          : p == 3 ? float(lcx(i) * lcx(i)) : p == 4 ? float(lcy(i) * lcy(i))
                          : p == 5 ? float(lcx(i) * lcy(i)) : p == 6 ? lg(i)
                          : p == 7 ? lg(i) * float(lcx(i)) : lg(i) * float(lcy(i));
            if (h != 0.0f) s = fmaf(h, f[i], s);
        }
        m[p] = s;
    }
    const float pres = fmaf(P.cs2_r, rr, P.cs2_b * rb);
    float meq[9] = {rho, rho * ux, rho * uy, fmaf(rho * ux, ux, pres), fmaf(rho * uy, uy, pres), rho * ux * uy,
                    P.ghost_N_mode == 0 ? fmaf(P.neq_r, rr, P.neq_b * rb) : 0.0f, 0.0f, 0.0f};
    const float lamv[9] = {0.0f, 0.0f, 0.0f, lam3, lam3, lam3, P.lambda6, P.lambda7, P.lambda7};
    const float Sv[9] = {0.0f, Gx, Gy, Cxx, Cyy, Cxy, 0.0f, 0.0f, 0.0f};
    float fp[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float s = f[i];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const float k = kinv(i, p);
            if (k != 0.0f) s = fmaf(k, fmaf(lamv[p], meq[p] - m[p], Sv[p]), s);
        }
        fp[i] = s;
    }
    const float mag2 = fmaf(gx, gx, gy * gy);
    const float inv = (mag2 >= kNormalTau * kNormalTau) ? rsqrtf(mag2) : 0.0f;
    const float ex = gx * inv, ey = gy * inv;
    const float phim = fmaf(P.kphi_r, rr, P.kphi_b * rb) * ir;  // phi_i = w_i phim (i != 0)
    const float seg = P.beta * rr * rb * ir;
    // ---- recolour: C++_i = x_C f+_i +/- seg phi_i (e . c-hat_i)
    const float xR = rr * ir, xB = rb * ir;
    float fpb[9];
    float xRb = 0.0f, xBb = 0.0f, segb = 0.0f, phimb = 0.0f, exb = 0.0f, eyb = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float lr = lamr[i];
        const float lb = lamb[i];
        fpb[i] = fmaf(xR, lr, xB * lb);
        xRb = fmaf(lr, fp[i], xRb);
        xBb = fmaf(lb, fp[i], xBb);
        if (i > 0) {
            const float db = lr - lb;
            const float ec = fmaf(chx(i), ex, chy(i) * ey);
            segb = fmaf(db * lw(i) * phim, ec, segb);
            phimb = fmaf(db * seg * lw(i), ec, phimb);
            exb = fmaf(db * seg * lw(i) * phim, chx(i), exb);
            eyb = fmaf(db * seg * lw(i) * phim, chy(i), eyb);
        }
    }
    out.acc[0] = segb * (rr * rb * ir);
    float rrb = (xRb - xBb) * rb * ir2;
    float rbb = (xBb - xRb) * rr * ir2;
    rrb = fmaf(segb * P.beta, rb * rb * ir2, rrb);
    rbb = fmaf(segb * P.beta, rr * rr * ir2, rbb);
    rrb = fmaf(phimb * (P.kphi_r - P.kphi_b), rb * ir2, rrb);
    rbb = fmaf(phimb * (P.kphi_b - P.kphi_r), rr * ir2, rbb);
    float gxb, gyb;
    normalise_T(gx, gy, exb, eyb, gxb, gyb);
    // ---- reconstruction and relaxation: m+ = m + lambda (m^(0) - m) + S, f+ = M^{-1} m+
    float mpb[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float k = kinv(i, p);
            if (k != 0.0f) s = fmaf(k, fpb[i], s);
        }
        mpb[p] = s;
    }
    float lam3b = 0.0f;
#pragma unroll
    for (int p = 3; p < 6; ++p) lam3b = fmaf(mpb[p], meq[p] - m[p], lam3b);
    float mb[9], meqb[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        mb[p] = (1.0f - lamv[p]) * mpb[p];
        meqb[p] = lamv[p] * mpb[p];
    }
    // common part of the population adjoint, M^T m-bar
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float fbi = mb[0] + float(lcx(i)) * mb[1] + float(lcy(i)) * mb[2] +
                          float(lcx(i) * lcx(i)) * mb[3] + float(lcy(i) * lcy(i)) * mb[4] +
                          float(lcx(i) * lcy(i)) * mb[5] + lg(i) * (mb[6] + float(lcx(i)) * mb[7] +
                                                                    float(lcy(i)) * mb[8]);
        out.fbar[i] = fbi;
    }
    // modal equilibrium (App. A)
    float rhob = meqb[0] + meqb[1] * ux + meqb[2] * uy + meqb[3] * ux * ux + meqb[4] * uy * uy +
                 meqb[5] * ux * uy;
    float uxb = rho * (meqb[1] + 2.0f * ux * meqb[3] + uy * meqb[5]);
    float uyb = rho * (meqb[2] + 2.0f * uy * meqb[4] + ux * meqb[5]);
    const float prb = meqb[3] + meqb[4];
    rrb = fmaf(P.cs2_r, prb, rrb);
    rbb = fmaf(P.cs2_b, prb, rbb);
    if (P.ghost_N_mode == 0) {
        rrb = fmaf(P.neq_r, meqb[6], rrb);
        rbb = fmaf(P.neq_b, meqb[6], rbb);
    }
    // sources S = (0, G, C_xx, C_yy, C_xy, 0, 0, 0) and the correction tensor (Eq. Correction)
    float Gxb = mpb[1], Gyb = mpb[2];
    const float cxxb = mpb[3], cyyb = mpb[4], cxyb = mpb[5];
    const float ab = cxxb * fmaf(2.0f * ux, hx, -iso) + cyyb * fmaf(2.0f * uy, hy, -iso) +
                     cxyb * fmaf(ux, hy, uy * hx);
    lam3b = fmaf(-0.5f, ab, lam3b);
    const float isob = -a * (cxxb + cyyb);
    const float hxb = a * fmaf(2.0f * ux, cxxb, uy * cxyb);
    const float hyb = a * fmaf(2.0f * uy, cyyb, ux * cxyb);
    uxb += a * fmaf(2.0f * hx, cxxb, hy * cxyb) + isob * dPx;
    uyb += a * fmaf(2.0f * hy, cyyb, hx * cxyb) + isob * dPy;
    Gxb += hxb;
    Gyb += hyb;
    const float dPxb = fmaf(isob, ux, -hxb);
    const float dPyb = fmaf(isob, uy, -hyb);
    rhob = fmaf(-isob * (1.0f / 3.0f), divu, rhob);
    const float divub = -isob * rho * (1.0f / 3.0f);
    // lambda_3 = 2 / (6 nu + 1): d lambda_3 / d nu = -3 lambda_3^2
    const float nub = lam3b * (-3.0f * lam3 * lam3);
    float rnb = 0.0f;
    if (P.visc_mode == 0) {
        rnb = nub * dnu_drn;
        // nu_C = (2 / lambda3_C - 1) / 6: d nu_C / d lambda3_C = -(6 nu_C + 1)^2 / 12
        const float dr = fmaf(6.0f, P.nu_r, 1.0f), db = fmaf(6.0f, P.nu_b, 1.0f);
        out.acc[1] = nub * 0.5f * (1.0f + rn) * (-dr * dr * (1.0f / 12.0f));
        out.acc[2] = nub * 0.5f * (1.0f - rn) * (-db * db * (1.0f / 12.0f));
    } else {
        rhob = fmaf(nub, -P.eta * ir2, rhob);
    }
    out.rrb = rrb + rhob;
    out.rbb = rbb + rhob;
    out.uxb = uxb;
    out.uyb = uyb;
    out.Gxb = Gxb;
    out.Gyb = Gyb;
    out.dPxb = dPxb;
    out.dPyb = dPyb;
    out.divub = divub;
    out.gxb = gxb;
    out.gyb = gyb;
    out.rnb = rnb;
}

// the outputs of rev_collide_node into the planes at offset o
__device__ __forceinline__ void store_rev_collide(float* __restrict__ S, size_t n, size_t o, const RevCollide& r) {
#pragma unroll
    for (int i = 0; i < 9; ++i) S[static_cast<size_t>(kFB0 + i) * n + o] = r.fbar[i];
    S[kRRB * n + o] = r.rrb;
    S[kRBB * n + o] = r.rbb;
    S[kUXB * n + o] = r.uxb;
    S[kUYB * n + o] = r.uyb;
    S[kGFXB * n + o] = r.Gxb;
    S[kGFYB * n + o] = r.Gyb;
    S[kDPXB * n + o] = r.dPxb;
    S[kDPYB * n + o] = r.dPyb;
    S[kDIVUB * n + o] = r.divub;
    S[kGXB * n + o] = r.gxb;
    S[kGYB * n + o] = r.gyb;
    S[kRNB * n + o] = r.rnb;
}

// The reverse collision pass: lam is the adjoint of the post-collision state P_t (18 planes).
// F: the forward planes of post (the first kFwdPlanes planes of S, or those a
// replayed step wrote); S: the adjoint's scratch planes.
template <int ORDER, bool W>
__global__ void __launch_bounds__(kAT) k_rev_collide(const float* __restrict__ post, const float* __restrict__ lam,
                                                      const StepParams P, const float* __restrict__ F,
                                                      float* __restrict__ S, double* __restrict__ partials) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    float acc[3] = {0.0f, 0.0f, 0.0f};  // beta, lambda3_r, lambda3_b
    if (x < P.nx) {
        const Nbh<reach<ORDER>(), W> L(P, x, y);
        const size_t o = L.o;
        float fr[9], fb[9], f[9];
        L.gather(post, fr, fb);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fr[i] + fb[i];
        float dPx, dPy, dux, duy, t0, t1;
        L.template grad<ORDER>(F + kPHIP * L.n, 1.0f, dPx, dPy);
        L.template grad<2>(F + kUX * L.n, -1.0f, dux, t0);
        L.template grad<2>(F + kUY * L.n, -1.0f, t1, duy);
        float lr[9], lb[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            lr[i] = lam[static_cast<size_t>(i) * L.n + o];
            lb[i] = lam[static_cast<size_t>(9 + i) * L.n + o];
        }
        RevCollide r;
        rev_collide_node(f, F[kRR * L.n + o], F[kRB * L.n + o], F[kUX * L.n + o], F[kUY * L.n + o],
                         F[kGFX * L.n + o], F[kGFY * L.n + o], F[kGX * L.n + o], F[kGY * L.n + o],
                         F[kCHR * L.n + o] - F[kCHB * L.n + o], dPx, dPy, dux + duy, lr, lb, P, r);
        store_rev_collide(S, L.n, o, r);
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[j] = r.acc[j];
    }
    const int slots[3] = {1, 2, 3};
    add_partials<3>(acc, slots, partials);
}

// Reverse of div u, u = (j + G/2) / rho and G = sigma K g / 2 + rho g_acc + g_vol.
template <bool W>
__global__ void __launch_bounds__(kAT) k_rev_force(const StepParams P, float* __restrict__ S,
                                                    double* __restrict__ partials) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    float acc[3] = {0.0f, 0.0f, 0.0f};  // sigma, g_acc_x, g_acc_y
    if (x < P.nx) {
        const Nbh<1, W> L(P, x, y);
        const size_t o = L.o;
        const float uxt = S[kUXB * L.n + o] + L.template gradT<true, 2>(S + kDIVUB * L.n, -1.0f);
        const float uyt = S[kUYB * L.n + o] + L.template gradT<false, 2>(S + kDIVUB * L.n, -1.0f);
        const float rho = S[kRR * L.n + o] + S[kRB * L.n + o];
        const float ir = 1.0f / rho;
        const float ux = S[kUX * L.n + o], uy = S[kUY * L.n + o];
        const float Gxt = fmaf(0.5f * ir, uxt, S[kGFXB * L.n + o]);
        const float Gyt = fmaf(0.5f * ir, uyt, S[kGFYB * L.n + o]);
        const float gx = S[kGX * L.n + o], gy = S[kGY * L.n + o], K = S[kK * L.n + o];
        const float rhob = -(ux * uxt + uy * uyt) * ir + Gxt * P.gacc_x + Gyt * P.gacc_y;
        const float gG = fmaf(Gxt, gx, Gyt * gy);
        S[kJXB * L.n + o] = uxt * ir;
        S[kJYB * L.n + o] = uyt * ir;
        S[kKB * L.n + o] = P.half_sigma * gG;
        S[kGXB * L.n + o] += P.half_sigma * K * Gxt;
        S[kGYB * L.n + o] += P.half_sigma * K * Gyt;
        S[kRRB * L.n + o] += rhob;
        S[kRBB * L.n + o] += rhob;
        acc[0] = 0.5f * K * gG;
        acc[1] = rho * Gxt;
        acc[2] = rho * Gyt;
    }
    const int slots[3] = {0, 4, 5};
    add_partials<3>(acc, slots, partials);
}

// Reverse of K = d_x n_x + d_y n_y and n-hat = -g / max(|g|, eps).
template <bool W>
__global__ void __launch_bounds__(kAT) k_rev_normal(const StepParams P, float* __restrict__ S) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Nbh<1, W> L(P, x, y);
    const size_t o = L.o;
    const float nxb = L.template gradT<true, 2>(S + kKB * L.n, 1.0f);
    const float nyb = L.template gradT<false, 2>(S + kKB * L.n, -1.0f);
    float tx, ty;
    normalise_T(S[kGX * L.n + o], S[kGY * L.n + o], nxb, nyb, tx, ty);
    S[kGXB * L.n + o] -= tx;
    S[kGYB * L.n + o] -= ty;
}

// Reverse of grad rho^N, grad Phi', rho^N, Phi' and of the moments: leaves
// the population adjoint dJ/dC_i(r, t) = FB_i + (c_i . j-bar) + rho_C-bar.
template <int ORDER, bool W>
__global__ void __launch_bounds__(kAT) k_rev_moments(const StepParams P, float* __restrict__ S) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Nbh<reach<ORDER>(), W> L(P, x, y);
    const size_t o = L.o;
    float rnb = S[kRNB * L.n + o];
    rnb += L.template gradT<true, ORDER>(S + kGXB * L.n, 1.0f) + L.template gradT<false, ORDER>(S + kGYB * L.n, 1.0f);
    const float phb =
        L.template gradT<true, ORDER>(S + kDPXB * L.n, 1.0f) + L.template gradT<false, ORDER>(S + kDPYB * L.n, 1.0f);
    const float rr = S[kRR * L.n + o], rb = S[kRB * L.n + o];
    const float a = rr * P.inv_rho0_r, b = rb * P.inv_rho0_b;
    const float iden = 1.0f / ((a + b) * (a + b));
    S[kRRB * L.n + o] += fmaf(rnb * 2.0f * b * iden, P.inv_rho0_r, phb * P.phip_r);
    S[kRBB * L.n + o] += fmaf(rnb * -2.0f * a * iden, P.inv_rho0_b, phb * P.phip_b);
    const float jxb = S[kJXB * L.n + o], jyb = S[kJYB * L.n + o];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float v = S[static_cast<size_t>(kFB0 + i) * L.n + o];
        if (lcx(i)) v += float(lcx(i)) * jxb;
        if (lcy(i)) v += float(lcy(i)) * jyb;
        S[static_cast<size_t>(kFB0 + i) * L.n + o] = v;
    }
}

// Transpose of the streaming gather: lam_i(s) = fbar_i(s + c_i), or
// fbar_opp(i)(s) where s + c_i lies beyond a wall.
template <bool W>
__global__ void __launch_bounds__(kAT) k_rev_gather(const StepParams P, const float* __restrict__ S,
                                                     float* __restrict__ lam_out) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Nbh<1, W> L(P, x, y);
    const size_t o = L.o;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        size_t src;
        int li = i;
        if (W && L.mir[lcy(i) + 1]) {
            li = lopp(i);
            src = o;
        } else {
            src = L.row[lcy(i) + 1] + L.col[lcx(i) + 1];
        }
        const float common = S[static_cast<size_t>(kFB0 + li) * L.n + src];
        lam_out[static_cast<size_t>(i) * L.n + o] = common + S[kRRB * L.n + src];
        lam_out[static_cast<size_t>(9 + i) * L.n + o] = common + S[kRBB * L.n + src];
    }
}

// dJ/df(t) in the public pre-collision layout: fbar_i + rho_C-bar at the node.
__global__ void __launch_bounds__(kAT) k_rev_expand(const StepParams P, const float* __restrict__ S,
                                                     float* __restrict__ lam_pre) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Own L(P, x, y);
    const size_t o = L.o;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float common = S[static_cast<size_t>(kFB0 + i) * L.n + o];
        lam_pre[static_cast<size_t>(i) * L.n + o] = common + S[kRRB * L.n + o];
        lam_pre[static_cast<size_t>(9 + i) * L.n + o] = common + S[kRBB * L.n + o];
    }
}

// ----------------------------------------------------------------- fused tail of the reverse step
// The reverse of the force, of the normal, of the moments and the transposed
// gather (or, for the step VJP, the expansion at the node) in one row
// wavefront, compact stencils only.  A CTA owns the strip [x0, x0 + 120) of
// the rows [y0, y0 + rows), with 4 halo columns on each side (one thread per
// window column), and marches down the rows; iteration k (s = y0 - 4 + k)
// runs
//   L  (row s)      load div-u-bar into a ring
//   R2 (row s - 1)  reverse of div u, u = (j + G/2) / rho and G          (k_rev_force)
//   R3 (row s - 2)  reverse of K = div n-hat and of n-hat                 (k_rev_normal)
//   R4 (row s - 3)  reverse of grad rho^N, grad Phi', rho^N, Phi', j      (k_rev_moments)
//   R5 (row s - 4)  lambda of P_{t-1}: transposed gather or expansion    (k_rev_gather / k_rev_expand)
// with one barrier between stages.  Each stage reads its stencil inputs from
// rings in shared memory, which hold exactly the rows still to be read, and
// its per-node inputs from the planes, loaded into registers one iteration
// ahead so that their latency overlaps the current row: every plane row is
// read from HBM once and only lambda is written.  The arithmetic is that of
// the plane passes, term by term in the same order.
// Ring sizes: a ring written by the stage at row s - a and last read, at
// its lowest, at row s - b needs b - a + 1 rows when the writing stage runs
// before the reading one in an iteration, b - a when after -- the fewest that
// never overwrite a row still to be read, so that five CTAs fit per SM.
constexpr int kTailRows = 75;  // ring rows of shared memory, kWin floats each
enum TailRing : int {
    kTDivub = 0,                                                // L at s, R2 reads s - 2 .. s: 3 rows
    kTKb = 3, kTJxb = 6, kTJyb = 9, kTRr = 12, kTRb = 15,       // R2 at s - 1, read down to s - 3: 3 rows
    kTGxb = 18, kTGyb = 22, kTDpxb = 26, kTDpyb = 30,           // R2 at s - 1, R4 reads down to s - 4: 4 rows
    kTGx = 34, kTGy = 36,                                       // R2 at s - 1, R3 reads s - 2: 2 rows
    kTRrb = 38, kTRbb = 43,                                     // R2 at s - 1, R5 reads down to s - 5: 5 rows
    kTFb = 48                                                   // 9 links; R4 at s - 3, R5 reads down to s - 5: 3 rows
};
static_assert(kTFb + 9 * 3 == kTailRows, "tail ring layout");
constexpr int kTailSmem = kTailRows * kWin * 4;
// slot of row r (r >= -64) in an M-row ring
template <int M>
__device__ __forceinline__ int tail_slot(int r) { return static_cast<int>(static_cast<unsigned>(r + 64 * M) % M); }

template <bool W, bool EXPAND>
__global__ void __launch_bounds__(kWin, 5) k_rev_tail(const StepParams P, const float* __restrict__ F,
                                                   const float* __restrict__ S, float* __restrict__ lam,
                                                   const int rows, double* __restrict__ partials) {
    extern __shared__ __align__(16) float tsm[];
    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const size_t n = static_cast<size_t>(nx) * ny;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * rows;
    const int y_end = min(y0 + rows, ny);
    const int gx = wrap_to(x0 - kHalo + t, nx);  // this thread's lattice column
    const bool own_col = t >= kHalo && t < kWin - kHalo && x0 + t - kHalo < nx;
    auto row_ok = [&](int r) { return !W || (r >= 0 && r < ny); };
    auto node = [&](int r) { return static_cast<size_t>(wrap_to(r, ny)) * nx + gx; };
    auto ring2 = [&](int base, int r) { return tsm + (base + tail_slot<2>(r)) * kWin; };
    auto ring3 = [&](int base, int r) { return tsm + (base + tail_slot<3>(r)) * kWin; };
    auto ring4 = [&](int base, int r) { return tsm + (base + tail_slot<4>(r)) * kWin; };
    auto ring5 = [&](int base, int r) { return tsm + (base + tail_slot<5>(r)) * kWin; };
    auto fbr = [&](int i, int r) { return tsm + (kTFb + 3 * i + tail_slot<3>(r)) * kWin; };
    // transpose of one component of the compact gradient, on ring rows
    // (the tap order and wall terms of Nbh::gradT)
    auto gradT = [&](auto rowp, bool xc, int y, float parity) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const int c = xc ? lcx(i) : lcy(i);
            if (c == 0) continue;
            const float k = 3.0f * lw(i) * float(c);
            const int dx = -lcx(i), dy = -lcy(i);
            if (!W) {
                acc = fmaf(k, rowp(y + dy)[t + dx], acc);
            } else {
                if (y + dy >= 0 && y + dy < ny) acc = fmaf(k, rowp(y + dy)[t + dx], acc);
                const int yb = -1 - y + dy;
                if (yb >= 0 && yb < ny && yb - dy < 0) acc = fmaf(parity * k, rowp(yb)[t + dx], acc);
                const int yt = 2 * ny - 1 - y + dy;
                if (yt >= 0 && yt < ny && yt - dy >= ny) acc = fmaf(parity * k, rowp(yt)[t + dx], acc);
            }
        }
        return acc;
    };
    double acc_sigma = 0.0, acc_gx = 0.0, acc_gy = 0.0;
    const int iters = (y_end - y0) + 8;
    // per-node inputs, one row ahead: div-u-bar for L, 17 planes for R2, 10 for R4
    constexpr int kIn2[17] = {kUXB, kUYB, kRR, kRB, kUX, kUY, kGFXB, kGFYB, kGX, kGY, kK,
                              kGXB, kGYB, kRRB, kRBB, kDPXB, kDPYB};
    auto in_L = [&](int r) { return row_ok(r); };
    auto in_R2 = [&](int r) { return r >= y0 - 3 && r <= y_end + 2 && row_ok(r) && t >= 1 && t < kWin - 1; };
    auto in_R4 = [&](int r) { return r >= y0 - 1 && r <= y_end && row_ok(r) && t >= 3 && t < kWin - 3; };
    float dv_next = 0.0f, in2_next[17], in4_next[10];
    auto fetch = [&](int s) {  // the inputs of iteration s: L at s, R2 at s - 1, R4 at s - 3
        if (in_L(s)) dv_next = S[kDIVUB * n + node(s)];
        if (in_R2(s - 1)) {
            const size_t o = node(s - 1);
#pragma unroll
            for (int j = 0; j < 17; ++j) {
                const int pl = kIn2[j];
                in2_next[j] = (pl < kFwdPlanes ? F : S)[static_cast<size_t>(pl) * n + o];
            }
        }
        if (in_R4(s - 3)) {
            const size_t o = node(s - 3);
            in4_next[0] = S[kRNB * n + o];
#pragma unroll
            for (int i = 0; i < 9; ++i) in4_next[1 + i] = S[static_cast<size_t>(kFB0 + i) * n + o];
        }
    };
    fetch(y0 - 4);
    for (int k = 0; k < iters; ++k) {
        const int s = y0 - 4 + k;
        const float dv = dv_next;
        float in2[17], in4[10];
#pragma unroll
        for (int j = 0; j < 17; ++j) in2[j] = in2_next[j];
#pragma unroll
        for (int j = 0; j < 10; ++j) in4[j] = in4_next[j];
        if (k + 1 < iters) fetch(s + 1);
        // ---- L: div-u-bar of row s (the window: R2 reads it at t +- 1)
        if (in_L(s)) ring3(kTDivub, s)[t] = dv;
        __syncthreads();
        // ---- R2: reverse of the force at row s - 1 (k_rev_force)
        {
            const int y = s - 1;
            if (in_R2(y)) {
                const auto dvr = [&](int r) { return ring3(kTDivub, r); };
                const float uxt = in2[0] + gradT(dvr, true, y, -1.0f);
                const float uyt = in2[1] + gradT(dvr, false, y, -1.0f);
                const float rr = in2[2], rb = in2[3];
                const float rho = rr + rb;
                const float ir = 1.0f / rho;
                const float ux = in2[4], uy = in2[5];
                const float Gxt = fmaf(0.5f * ir, uxt, in2[6]);
                const float Gyt = fmaf(0.5f * ir, uyt, in2[7]);
                const float gxv = in2[8], gyv = in2[9], K = in2[10];
                const float rhob = -(ux * uxt + uy * uyt) * ir + Gxt * P.gacc_x + Gyt * P.gacc_y;
                const float gG = fmaf(Gxt, gxv, Gyt * gyv);
                ring3(kTJxb, y)[t] = uxt * ir;
                ring3(kTJyb, y)[t] = uyt * ir;
                ring3(kTKb, y)[t] = P.half_sigma * gG;
                float gxb = in2[11], gyb = in2[12], rrb = in2[13], rbb = in2[14];
                gxb += P.half_sigma * K * Gxt;
                gyb += P.half_sigma * K * Gyt;
                rrb += rhob;
                rbb += rhob;
                ring4(kTGxb, y)[t] = gxb;
                ring4(kTGyb, y)[t] = gyb;
                ring5(kTRrb, y)[t] = rrb;
                ring5(kTRbb, y)[t] = rbb;
                ring4(kTDpxb, y)[t] = in2[15];
                ring4(kTDpyb, y)[t] = in2[16];
                ring3(kTRr, y)[t] = rr;
                ring3(kTRb, y)[t] = rb;
                ring2(kTGx, y)[t] = gxv;
                ring2(kTGy, y)[t] = gyv;
                if (own_col && y >= y0 && y < y_end) {
                    acc_sigma += static_cast<double>(0.5f * K * gG);
                    acc_gx += static_cast<double>(rho * Gxt);
                    acc_gy += static_cast<double>(rho * Gyt);
                }
            }
        }
        __syncthreads();
        // ---- R3: reverse of K = div n-hat and of the regularised normal at row s - 2 (k_rev_normal)
        if (P.curvature_mode == 0) {
            const int y = s - 2;
            if (y >= y0 - 2 && y <= y_end + 1 && row_ok(y) && t >= 2 && t < kWin - 2) {
                const auto kb = [&](int r) { return ring3(kTKb, r); };
                const float nxb = gradT(kb, true, y, 1.0f);
                const float nyb = gradT(kb, false, y, -1.0f);
                float tx, ty;
                normalise_T(ring2(kTGx, y)[t], ring2(kTGy, y)[t], nxb, nyb, tx, ty);
                ring4(kTGxb, y)[t] -= tx;
                ring4(kTGyb, y)[t] -= ty;
            }
        }
        __syncthreads();
        // ---- R4: reverse of the gradients, rho^N, Phi' and the moments at row s - 3 (k_rev_moments)
        {
            const int y = s - 3;
            if (in_R4(y)) {
                float rnb = in4[0];
                rnb += gradT([&](int r) { return ring4(kTGxb, r); }, true, y, 1.0f) +
                       gradT([&](int r) { return ring4(kTGyb, r); }, false, y, 1.0f);
                const float phb = gradT([&](int r) { return ring4(kTDpxb, r); }, true, y, 1.0f) +
                                  gradT([&](int r) { return ring4(kTDpyb, r); }, false, y, 1.0f);
                const float rr = ring3(kTRr, y)[t], rb = ring3(kTRb, y)[t];
                const float a = rr * P.inv_rho0_r, b = rb * P.inv_rho0_b;
                const float iden = 1.0f / ((a + b) * (a + b));
                ring5(kTRrb, y)[t] += fmaf(rnb * 2.0f * b * iden, P.inv_rho0_r, phb * P.phip_r);
                ring5(kTRbb, y)[t] += fmaf(rnb * -2.0f * a * iden, P.inv_rho0_b, phb * P.phip_b);
                const float jxb = ring3(kTJxb, y)[t], jyb = ring3(kTJyb, y)[t];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    float v = in4[1 + i];
                    if (lcx(i)) v += float(lcx(i)) * jxb;
                    if (lcy(i)) v += float(lcy(i)) * jyb;
                    fbr(i, y)[t] = v;
                }
            }
        }
        __syncthreads();
        // ---- R5: lambda at row s - 4 (k_rev_gather / k_rev_expand)
        {
            const int y = s - 4;
            if (y >= y0 && y < y_end && own_col) {
                const size_t o = static_cast<size_t>(y) * nx + gx;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    float common, cr, cb;
                    if (EXPAND) {
                        common = fbr(i, y)[t];
                        cr = ring5(kTRrb, y)[t];
                        cb = ring5(kTRbb, y)[t];
                    } else {
                        int li = i, sy = y + lcy(i), st = t + lcx(i);
                        if (W && (sy < 0 || sy >= ny)) {  // the node's own reversed link (half-way bounce-back)
                            li = lopp(i);
                            sy = y;
                            st = t;
                        }
                        common = fbr(li, sy)[st];
                        cr = ring5(kTRrb, sy)[st];
                        cb = ring5(kTRbb, sy)[st];
                    }
                    lam[static_cast<size_t>(i) * n + o] = common + cr;
                    lam[static_cast<size_t>(9 + i) * n + o] = common + cb;
                }
            }
        }
        __syncthreads();
    }
    // parameter gradients of the owned nodes: FP64 per thread, then per CTA
    __shared__ double red[kWin / 32][3];
    double v[3] = {acc_sigma, acc_gx, acc_gy};
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], off);
    if ((t & 31) == 0)
#pragma unroll
        for (int j = 0; j < 3; ++j) red[t >> 5][j] = v[j];
    __syncthreads();
    if (t < 3) {
        double a = 0.0;
        for (int w = 0; w < kWin / 32; ++w) a += red[w][t];
        const int slot = t == 0 ? 0 : (t == 1 ? 4 : 5);  // sigma, g_acc_x, g_acc_y
        partials[(static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x) * kAdjSlots + slot] += a;
    }
}

// rows per CTA of the fused tail: enough CTAs for two waves of 152 SMs where
// the lattice allows, at most 64 rows (8 fill iterations per segment)
int tail_rows(int nx, int ny) {
    const long strips = (nx + kTileX - 1) / kTileX;
    int rows = 64;
    while (rows > 4 && strips * ((ny + rows - 1) / rows) < 2 * 152) rows /= 2;
    return rows;
}

// fused kernels or plane passes (compact stencil): as asked, else the fused
// kernels where the lattice fills 16-row segments in two waves -- on smaller
// lattices their fill rows per segment cost more than the launches they save
bool use_fused(const StepParams& P) {
    return P.adjoint_fused == 1 || (P.adjoint_fused == 0 && tail_rows(P.nx, P.ny) >= 16);
}

template <bool W, bool EXPAND>
cudaError_t launch_tail(const StepParams& P, const float* F, const float* S, float* lam, double* partials,
                        cudaStream_t s) {
    static std::atomic<unsigned long long> configured{0};  // the shared-memory opt-in, once per device (any thread)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k_rev_tail<W, EXPAND>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    const int rows = tail_rows(P.nx, P.ny);
    const dim3 g(static_cast<unsigned>((P.nx + kTileX - 1) / kTileX), static_cast<unsigned>((P.ny + rows - 1) / rows));
    k_rev_tail<W, EXPAND><<<g, kWin, kTailSmem, s>>>(P, F, S, lam, rows, partials);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- fused forward recomputation
// The forward fields of P_{t-1} that the reverse step reads (moments, colour
// fractions, Phi', grad rho^N, K, G and u) in one row wavefront, compact
// stencil only: the same tiling as k_rev_tail, iteration k (s = y0 - 2 + k)
// runs
//   A (row s - 1)  gather f, colour moments, colour fractions, Phi'        (k_fwd_moments)
//   B (row s - 2)  grad rho^N on the smaller colour fraction, n-hat       (k_fwd_normal)
//   C (row s - 3)  K = div n-hat, G, u                                    (k_fwd_force)
// with one barrier between stages, the stencil inputs in rings in shared
// memory and A's gather loaded one row ahead; every owned node's fields go
// to the planes once.  The arithmetic is that of the plane passes, term by
// term.  (Fusing the reverse collision as a fourth stage was tried: its
// registers left 12 warps per SM, and the four-stage kernel took 1.4x the
// time of the passes it replaced.)
// Only the stencil stages' inputs live in rings (4 rows each: three rows a
// stencil reads, one more for the mirrored row a wall adds ahead of the
// schedule); Phi', G and u go to the planes alone.
constexpr int kHeadRows = 40;  // ring rows of shared memory, kWin floats each
enum HeadRing : int {
    kHChr = 0, kHChb = 4, kHRr = 8, kHRb = 12, kHJx = 16, kHJy = 20, kHGx = 24, kHGy = 28, kHNx = 32, kHNy = 36
};

template <bool W>
__global__ void __launch_bounds__(kWin) k_fwd_head(const float* __restrict__ post, const StepParams P,
                                                   float* __restrict__ S, const int rows) {
    __shared__ __align__(16) float hsm[kHeadRows * kWin];
    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const size_t n = static_cast<size_t>(nx) * ny;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * rows;
    const int y_end = min(y0 + rows, ny);
    const int xm = wrap_to(x0 - kHalo + t - 1, nx), xc = wrap_to(x0 - kHalo + t, nx), xp = wrap_to(x0 - kHalo + t + 1, nx);
    const bool own_col = t >= kHalo && t < kWin - kHalo && x0 + t - kHalo < nx;
    auto row_ok = [&](int r) { return !W || (r >= 0 && r < ny); };
    auto r4 = [&](int base, int r) { return hsm + (base + (r & 3)) * kWin; };
    // pre-collision populations of node (column xc, row y): f_i(r) = P_i(r - c_i),
    // half-way bounce-back beyond a wall (Nbh::gather)
    auto gather = [&](int y, float (&fr)[9], float (&fb)[9]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sy = y - lcy(i);
            size_t src;
            int li = i;
            if (W && (sy < 0 || sy >= ny)) {
                li = lopp(i);
                src = static_cast<size_t>(y) * nx + xc;
            } else {
                src = static_cast<size_t>(wrap_to(sy, ny)) * nx + (lcx(i) > 0 ? xm : (lcx(i) < 0 ? xp : xc));
            }
            fr[i] = post[static_cast<size_t>(li) * n + src];
            fb[i] = post[static_cast<size_t>(9 + li) * n + src];
        }
    };
    // compact gradient of a ring field at (row y, column t): Nbh::grad<2>
    // (wall rows come from the mirrored ghost rows the writers add)
    auto grad = [&](auto rowp, int y, float& gxo, float& gyo) {
        const float* m = rowp(y);
        const float* a = rowp(y + 1);
        const float* b = rowp(y - 1);
        gxo = ddx(m[t + 1], m[t - 1], a[t + 1], a[t - 1], b[t + 1], b[t - 1]);
        gyo = ddy(a[t], b[t], a[t + 1], a[t - 1], b[t + 1], b[t - 1]);
    };
    auto in_A = [&](int r) { return r >= y0 - 3 && r <= y_end + 2 && row_ok(r) && t >= 1 && t < kWin - 1; };
    auto owned = [&](int r) { return r >= y0 && r < y_end && own_col; };
    float frn[9], fbn[9];  // next iteration's A gather
    auto fetch = [&](int s) {
        if (in_A(s - 1)) gather(s - 1, frn, fbn);
    };
    const int iters = (y_end - y0) + 5;
    fetch(y0 - 2);
    for (int k = 0; k < iters; ++k) {
        const int s = y0 - 2 + k;
        float fr[9], fb[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fr[i] = frn[i];
            fb[i] = fbn[i];
        }
        if (k + 1 < iters) fetch(s + 1);
        // ---- A: moments at row s - 1 (k_fwd_moments)
        {
            const int y = s - 1;
            if (in_A(y)) {
                float f[9];
                const float rr = sum9f(fr), rb = sum9f(fb);
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = fr[i] + fb[i];
                const float a = rr * P.inv_rho0_r, b = rb * P.inv_rho0_b;
                // the step kernel's arithmetic, bit for bit (its fields replace these
                // where a replayed step wrote them)
                const float inv = rcp(__fadd_rn(a, b));
                const float chr = a * inv, chb = b * inv;
                const float phip = fmaf(P.phip_r, rr, P.phip_b * rb);  // App. A, Phi'
                r4(kHChr, y)[t] = chr;
                r4(kHChb, y)[t] = chb;
                r4(kHRr, y)[t] = rr;
                r4(kHRb, y)[t] = rb;
                r4(kHJx, y)[t] = ((f[1] + f[7]) + f[8]) - ((f[3] + f[5]) + f[4]);
                r4(kHJy, y)[t] = ((f[1] + f[3]) + f[2]) - ((f[5] + f[7]) + f[6]);
                if (W && (y == 0 || y == ny - 1)) {  // even mirrors beyond the walls
                    const int g = y == 0 ? -1 : ny;
                    r4(kHChr, g)[t] = chr;
                    r4(kHChb, g)[t] = chb;
                }
                if (owned(y)) {
                    const size_t o = static_cast<size_t>(y) * nx + xc;
                    S[kRR * n + o] = rr;
                    S[kRB * n + o] = rb;
                    S[kCHR * n + o] = chr;
                    S[kCHB * n + o] = chb;
                    S[kPHIP * n + o] = phip;
                }
            }
        }
        __syncthreads();
        // ---- B: grad rho^N on the smaller colour fraction, n-hat at row s - 2 (k_fwd_normal)
        {
            const int y = s - 2;
            if (y >= y0 - 2 && y <= y_end + 1 && row_ok(y) && t >= 2 && t < kWin - 2) {
                const bool red_minor = r4(kHChr, y)[t] <= 0.5f;
                float gx, gy;
                if (red_minor) grad([&](int r) { return r4(kHChr, r); }, y, gx, gy);
                else grad([&](int r) { return r4(kHChb, r); }, y, gx, gy);
                gx *= red_minor ? 2.0f : -2.0f;
                gy *= red_minor ? 2.0f : -2.0f;
                float nhx, nhy;
                normal_of(gx, gy, nhx, nhy);
                r4(kHGx, y)[t] = gx;
                r4(kHGy, y)[t] = gy;
                r4(kHNx, y)[t] = nhx;
                r4(kHNy, y)[t] = nhy;
                if (W && (y == 0 || y == ny - 1)) {  // the normal beyond a wall: y component odd
                    const int g = y == 0 ? -1 : ny;
                    r4(kHNx, g)[t] = nhx;
                    r4(kHNy, g)[t] = -nhy;
                }
            }
        }
        __syncthreads();
        // ---- C: curvature, force, velocity at row s - 3 (k_fwd_force)
        {
            const int y = s - 3;
            if (y >= y0 - 1 && y <= y_end && row_ok(y) && t >= 3 && t < kWin - 3) {
                float K = P.fixed_K;
                if (P.curvature_mode == 0) {
                    const float* nxm = r4(kHNx, y);
                    const float* nxa = r4(kHNx, y + 1);
                    const float* nxb = r4(kHNx, y - 1);
                    const float* nym = r4(kHNy, y);
                    const float* nya = r4(kHNy, y + 1);
                    const float* nyb = r4(kHNy, y - 1);
                    K = ddx(nxm[t + 1], nxm[t - 1], nxa[t + 1], nxa[t - 1], nxb[t + 1], nxb[t - 1]) +
                        ddy(nya[t], nyb[t], nya[t + 1], nya[t - 1], nyb[t + 1], nyb[t - 1]);
                }
                const float gx = r4(kHGx, y)[t], gy = r4(kHGy, y)[t];
                const float rr = r4(kHRr, y)[t], rb = r4(kHRb, y)[t];
                const float rho = rr + rb;
                const float hk = P.half_sigma * K;
                const float Gx = fmaf(hk, gx, fmaf(rho, P.gacc_x, P.gvol_x));
                const float Gy = fmaf(hk, gy, fmaf(rho, P.gacc_y, P.gvol_y));
                const float inv_rho = rcp(rho);
                const float ux = fmaf(0.5f, Gx, r4(kHJx, y)[t]) * inv_rho;
                const float uy = fmaf(0.5f, Gy, r4(kHJy, y)[t]) * inv_rho;
                if (owned(y)) {
                    const size_t o = static_cast<size_t>(y) * nx + xc;
                    S[kGX * n + o] = gx;
                    S[kGY * n + o] = gy;
                    S[kK * n + o] = K;
                    S[kGFX * n + o] = Gx;
                    S[kGFY * n + o] = Gy;
                    S[kUX * n + o] = ux;
                    S[kUY * n + o] = uy;
                }
            }
        }
        __syncthreads();
    }
}

template <bool W>
cudaError_t launch_fwd_head(const float* post, const StepParams& P, float* S, cudaStream_t s) {
    const int rows = tail_rows(P.nx, P.ny);
    const dim3 g(static_cast<unsigned>((P.nx + kTileX - 1) / kTileX), static_cast<unsigned>((P.ny + rows - 1) / rows));
    k_fwd_head<W><<<g, kWin, 0, s>>>(post, P, S, rows);
    return cudaGetLastError();
}

// Objective J = 1/2 sum (rho^N - target)^2 of f(T) = gather(P_{T-1}) and its
// gradient dJ/dC_i = (rho^N - target) d rho^N / d rho_C, the same for every link.
template <bool W>
__global__ void __launch_bounds__(kAT) k_seed(const float* __restrict__ post, const float* __restrict__ target,
                                               const StepParams P, float* __restrict__ S,
                                               double* __restrict__ partials) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    float acc[1] = {0.0f};
    if (x < P.nx) {
        const Nbh<1, W> L(P, x, y);
        const size_t o = L.o;
        float fr[9], fb[9];
        L.gather(post, fr, fb);
        const float a = sum9f(fr) * P.inv_rho0_r, b = sum9f(fb) * P.inv_rho0_b;
        const float res = (a - b) / (a + b) - target[o];
        const float iden = 1.0f / ((a + b) * (a + b));
        acc[0] = 0.5f * res * res;
        S[kRRB * L.n + o] = res * 2.0f * b * iden * P.inv_rho0_r;
        S[kRBB * L.n + o] = res * -2.0f * a * iden * P.inv_rho0_b;
#pragma unroll
        for (int i = 0; i < 9; ++i) S[static_cast<size_t>(kFB0 + i) * L.n + o] = 0.0f;
    }
    const int slots[1] = {6};
    add_partials<1>(acc, slots, partials);
}

// dJ/drho^N_0 through the initial state C_i = (rho_C / rho) f^(0)_i(rho, u_0),
// rho_R = rho0_r (1 + rho^N_0)/2, rho_B = rho0_b (1 - rho^N_0)/2; pre0 is that
// state (pre-collision, public layout), lam0 its adjoint.
__global__ void __launch_bounds__(kAT) k_init_T(const float* __restrict__ pre0, const float* __restrict__ lam0,
                                                 const StepParams P, float* __restrict__ grad) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Own L(P, x, y);
    const size_t o = L.o;
    float R[9], B[9], f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R[i] = pre0[static_cast<size_t>(i) * L.n + o];
        B[i] = pre0[static_cast<size_t>(9 + i) * L.n + o];
        f[i] = R[i] + B[i];
    }
    const float rr = sum9f(R), rb = sum9f(B), rho = rr + rb, ir = 1.0f / rho, ir2 = ir * ir;
    const float ux = (((f[1] + f[7]) + f[8]) - ((f[3] + f[5]) + f[4])) * ir;
    const float uy = (((f[1] + f[3]) + f[2]) - ((f[5] + f[7]) + f[6])) * ir;
    const float xR = rr * ir, xB = rb * ir;
    float xRb = 0.0f, xBb = 0.0f, rrb = 0.0f, rbb = 0.0f;
    const float usq = fmaf(ux, ux, uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float lr = lam0[static_cast<size_t>(i) * L.n + o];
        const float lb = lam0[static_cast<size_t>(9 + i) * L.n + o];
        xRb = fmaf(lr, f[i], xRb);
        xBb = fmaf(lb, f[i], xBb);
        const float f0b = fmaf(xR, lr, xB * lb);
        const float cu = fmaf(float(lcx(i)), ux, float(lcy(i)) * uy);
        const float Q = fmaf(3.0f, cu, fmaf(4.5f * cu, cu, -1.5f * usq));
        // rho phi_0 = alpha_r rho_R + alpha_b rho_B; rho phi_i = k w_i ((1 - alpha_r) rho_R + (1 - alpha_b) rho_B)
        const float kr = i == 0 ? P.alpha_r : lw(i) * P.kphi_r;
        const float kb = i == 0 ? P.alpha_b : lw(i) * P.kphi_b;
        rrb = fmaf(f0b, fmaf(lw(i), Q, kr), rrb);
        rbb = fmaf(f0b, fmaf(lw(i), Q, kb), rbb);
    }
    rrb = fmaf(xRb - xBb, rb * ir2, rrb);
    rbb = fmaf(xBb - xRb, rr * ir2, rbb);
    // d rho_R / d rho^N_0 = rho0_r / 2, d rho_B / d rho^N_0 = -rho0_b / 2
    grad[o] = 0.5f * (rrb / P.inv_rho0_r - rbb / P.inv_rho0_b);
}

// ----------------------------------------------------------------- order-6 step and its outputs
// The rest of one step after k_fwd_*: grad Phi' (order of P.stencil_order),
// div u, collision in moment space, recolour and store of P_t (FP32 layout).
template <int ORDER, bool W>
__global__ void __launch_bounds__(kAT) k_step_planes(const float* __restrict__ post, float* __restrict__ dst,
                                                      const StepParams P, const float* __restrict__ S,
                                                      unsigned* __restrict__ flag) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Nbh<reach<ORDER>(), W> L(P, x, y);
    const size_t o = L.o;
    float fr[9], fb[9], f[9];
    L.gather(post, fr, fb);
    const float rr = sum9f(fr), rb = sum9f(fb);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fr[i] + fb[i];
    const float rho = rr + rb;
    if (!isfinite(rho)) atomicOr(flag, 1u);
    float dPx, dPy, dux, duy, t0, t1;
    L.template grad<ORDER>(S + kPHIP * L.n, 1.0f, dPx, dPy);
    L.template grad<2>(S + kUX * L.n, -1.0f, dux, t0);
    L.template grad<2>(S + kUY * L.n, -1.0f, t1, duy);
    const float inv_rho = rcp(rho);
    float nu;
    if (P.visc_mode == 0) {
        const float rn = S[kCHR * L.n + o] - S[kCHB * L.n + o];
        nu = fmaf(0.5f * (P.nu_r - P.nu_b), rn, 0.5f * (P.nu_r + P.nu_b));
    } else {
        nu = P.eta * inv_rho;
    }
    float fp[9];
    collide_increment(f, rr, rb, rho, nu, S[kUX * L.n + o], S[kUY * L.n + o], S[kGFX * L.n + o],
                      S[kGFY * L.n + o], dPx, dPy, dux + duy, P, fp);
    // recolour along e = grad rho^N / |grad rho^N| (Eq. eq_re_color; 0 below kNormalTau)
    const float gx = S[kGX * L.n + o], gy = S[kGY * L.n + o];
    const float mag2 = fmaf(gx, gx, gy * gy);
    const float inv = (mag2 >= kNormalTau * kNormalTau) ? rsqrtf(mag2) : 0.0f;
    const float phim = fmaf(P.kphi_r, rr, P.kphi_b * rb) * inv_rho;
    const float sg = P.beta * (rr * rb) * inv_rho * phim * inv;
    store_recoloured_f32(dst + o, L.n, fp, rr, rb, inv_rho, sg * gx, sg * gy);
}

__global__ void __launch_bounds__(kAT) k_fields_planes(const StepParams P, const float* __restrict__ S,
                                                        FieldOut fo) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx) return;
    const Own L(P, x, y);
    const size_t o = L.o;
    const float rr = S[kRR * L.n + o], rb = S[kRB * L.n + o];
    if (fo.rho_r) fo.rho_r[o] = rr;
    if (fo.rho_b) fo.rho_b[o] = rb;
    if (fo.ux) fo.ux[o] = S[kUX * L.n + o];
    if (fo.uy) fo.uy[o] = S[kUY * L.n + o];
    if (fo.p) fo.p[o] = fmaf(P.cs2_r, rr, P.cs2_b * rb);
}

// FP64 per-CTA partial diagnostics, partials[block][kDiagSlots] (slot 4 is a maximum)
__global__ void __launch_bounds__(kAT) k_diag_planes(const StepParams P, const float* __restrict__ S,
                                                      double* __restrict__ partials) {
    const int x = blockIdx.x * kAT + threadIdx.x, y = blockIdx.y;
    double v[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (x < P.nx) {
        const Own L(P, x, y);
        const size_t o = L.o;
        const float rr = S[kRR * L.n + o], rb = S[kRB * L.n + o];
        if (isfinite(rr + rb)) {
            const double ux = S[kUX * L.n + o], uy = S[kUY * L.n + o];
            v[0] = rr;
            v[1] = rb;
            v[2] = S[kJX * L.n + o];
            v[3] = S[kJY * L.n + o];
            v[4] = ux * ux + uy * uy;
        } else {
            v[5] = 1.0;
        }
    }
    __shared__ double red[kAT / 32][kDiagSlots];
#pragma unroll
    for (int j = 0; j < kDiagSlots; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v[j], off);
            v[j] = j == 4 ? fmax(v[j], w) : v[j] + w;
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < kDiagSlots; ++j) red[warp][j] = v[j];
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        double acc = red[0][threadIdx.x];
        for (int w = 1; w < kAT / 32; ++w)
            acc = threadIdx.x == 4 ? fmax(acc, red[w][threadIdx.x]) : acc + red[w][threadIdx.x];
        partials[(static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x) * kDiagSlots + threadIdx.x] = acc;
    }
}

__global__ void k_adj_reduce(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double red[kAT / 32][kAdjSlots];
    double v[kAdjSlots];
#pragma unroll
    for (int j = 0; j < kAdjSlots; ++j) v[j] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int j = 0; j < kAdjSlots; ++j) v[j] += partials[static_cast<size_t>(b) * kAdjSlots + j];
#pragma unroll
    for (int j = 0; j < kAdjSlots; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < kAdjSlots; ++j) red[warp][j] = v[j];
    __syncthreads();
    if (threadIdx.x < kAdjSlots) {
        double acc = 0.0;
        for (int w = 0; w < kAT / 32; ++w) acc += red[w][threadIdx.x];
        out[threadIdx.x] = acc;
    }
}

dim3 adj_grid(const StepParams& P) { return dim3(static_cast<unsigned>((P.nx + kAT - 1) / kAT), P.ny, 1); }

// Calls f(order, walls) with both as compile-time constants.
template <class F>
void dispatch(const StepParams& P, F&& f) {
    using O2 = std::integral_constant<int, 2>;
    using O6 = std::integral_constant<int, 6>;
    if (P.stencil_order == 6) {
        if (P.wall_y) f(O6{}, std::true_type{});
        else f(O6{}, std::false_type{});
    } else {
        if (P.wall_y) f(O2{}, std::true_type{});
        else f(O2{}, std::false_type{});
    }
}

// moments, colour fractions, Phi', grad rho^N, K, G and u of P_{t-1} into the planes
template <int O, bool W>
void forward_planes(const float* post, const StepParams& P, float* S, cudaStream_t s) {
    const dim3 g = adj_grid(P);
    k_fwd_moments<W><<<g, kAT, 0, s>>>(post, P, S);
    k_fwd_normal<O, W><<<g, kAT, 0, s>>>(P, S);
    k_fwd_force<W><<<g, kAT, 0, s>>>(P, S);
}

// One adjoint step: `lam_out` is lambda of P_{t-1} (transposed gather) or,
// with EXPAND, dJ/df(t) in the public layout.  With the compact stencil on a
// large enough lattice it is three launches (k_fwd_head: the forward fields;
// the reverse collision pass; k_rev_tail: the rest); otherwise eight plane
// passes (seven with fixed K).
template <int O, bool W, bool EXPAND>
cudaError_t reverse_step(const float* post, const float* lam_post, const StepParams& P, float* S, double* partials,
                         float* lam_out, cudaStream_t s, const float* fwd) {
    const dim3 g = adj_grid(P);
    if (O == 2 && use_fused(P)) {
        // the forward fields of post: written by the replayed step, or recomputed here
        const float* F = fwd;
        if (!F) {
            const cudaError_t e = launch_fwd_head<W>(post, P, S, s);
            if (e != cudaSuccess) return e;
            F = S;
        }
        k_rev_collide<O, W><<<g, kAT, 0, s>>>(post, lam_post, P, F, S, partials);
        return launch_tail<W, EXPAND>(P, F, S, lam_out, partials, s);
    }
    forward_planes<O, W>(post, P, S, s);
    k_rev_collide<O, W><<<g, kAT, 0, s>>>(post, lam_post, P, S, S, partials);
    k_rev_force<W><<<g, kAT, 0, s>>>(P, S, partials);
    if (P.curvature_mode == 0) k_rev_normal<W><<<g, kAT, 0, s>>>(P, S);
    k_rev_moments<O, W><<<g, kAT, 0, s>>>(P, S);
    if (EXPAND) k_rev_expand<<<g, kAT, 0, s>>>(P, S, lam_out);
    else k_rev_gather<W><<<g, kAT, 0, s>>>(P, S, lam_out);
    return cudaGetLastError();
}

}  // namespace

int adj_blocks(int nx, int ny) {
    // per-CTA partial-sum slots: the larger of the plane passes' grid and the fused tail's
    const int planes = ((nx + kAT - 1) / kAT) * ny;
    const int rows = tail_rows(nx, ny);
    const int tail = ((nx + kTileX - 1) / kTileX) * ((ny + rows - 1) / rows);
    return planes > tail ? planes : tail;
}

cudaError_t launch_step_planes(const float* post, float* dst, const StepParams& P, float* scratch, unsigned* flag,
                               cudaStream_t s) {
    dispatch(P, [&](auto o, auto w) {
        forward_planes<decltype(o)::value, decltype(w)::value>(post, P, scratch, s);
        k_step_planes<decltype(o)::value, decltype(w)::value><<<adj_grid(P), kAT, 0, s>>>(post, dst, P, scratch, flag);
    });
    return cudaGetLastError();
}

cudaError_t launch_fields_planes(const float* post, const StepParams& P, float* scratch, FieldOut out,
                                 cudaStream_t s) {
    dispatch(P, [&](auto o, auto w) { forward_planes<decltype(o)::value, decltype(w)::value>(post, P, scratch, s); });
    k_fields_planes<<<adj_grid(P), kAT, 0, s>>>(P, scratch, out);
    return cudaGetLastError();
}

cudaError_t launch_diag_planes(const float* post, const StepParams& P, float* scratch, double* partials,
                               cudaStream_t s) {
    dispatch(P, [&](auto o, auto w) { forward_planes<decltype(o)::value, decltype(w)::value>(post, P, scratch, s); });
    k_diag_planes<<<adj_grid(P), kAT, 0, s>>>(P, scratch, partials);
    return cudaGetLastError();
}

bool adj_fused(const StepParams& P) { return P.stencil_order == 2 && use_fused(P); }
bool adj_fields_usable(const StepParams& P) { return P.stencil_order == 2 && P.adjoint_fused != 2; }

int adj_launches_per_step(const StepParams& P) {
    if (adj_fused(P)) return 3;  // fused forward fields, collision pass, fused tail
    return P.curvature_mode == 0 ? 8 : 7;
}

cudaError_t launch_adjoint_step(const float* post, const float* lam_post, const StepParams& P, float* scratch,
                                double* partials, float* lam_prev, cudaStream_t s, const float* fwd) {
    if (fwd && !adj_fused(P)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    dispatch(P, [&](auto o, auto w) {
        e = reverse_step<decltype(o)::value, decltype(w)::value, false>(post, lam_post, P, scratch, partials, lam_prev,
                                                                       s, fwd);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_adjoint_step_pre(const float* post, const float* lam_post, const StepParams& P, float* scratch,
                                    double* partials, float* lam_pre, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    dispatch(P, [&](auto o, auto w) {
        e = reverse_step<decltype(o)::value, decltype(w)::value, true>(post, lam_post, P, scratch, partials, lam_pre, s,
                                                                      nullptr);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_adjoint_seed(const float* post, const float* target, const StepParams& P, float* scratch,
                                double* partials, float* lam_post, cudaStream_t s) {
    const dim3 g = adj_grid(P);
    if (P.wall_y) {
        k_seed<true><<<g, kAT, 0, s>>>(post, target, P, scratch, partials);
        k_rev_gather<true><<<g, kAT, 0, s>>>(P, scratch, lam_post);
    } else {
        k_seed<false><<<g, kAT, 0, s>>>(post, target, P, scratch, partials);
        k_rev_gather<false><<<g, kAT, 0, s>>>(P, scratch, lam_post);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_init(const float* pre0, const float* lam_pre0, const StepParams& P, float* grad_rho_n0,
                                cudaStream_t s) {
    k_init_T<<<adj_grid(P), kAT, 0, s>>>(pre0, lam_pre0, P, grad_rho_n0);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_reduce(const double* partials, int nblocks, double* out, cudaStream_t s) {
    k_adj_reduce<<<1, kAT, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace cmrt
