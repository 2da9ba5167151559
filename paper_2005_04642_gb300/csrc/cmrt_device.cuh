// Device-side building blocks of the two-colour D2Q9 chromodynamic MRT step
// (arXiv 2005.04642).  Shared by the kernels of libcmrt; host code sees only
// the parameter block and the kernel launchers declared in cmrt_internal.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cmrt_internal.h"

namespace cmrt {

// Programmatic dependent launch.  A kernel launched by launch_pdl may be
// scheduled while the kernel before it on the stream is still finishing;
// pdl_begin, its first statement, waits until that kernel has completed and
// its writes are visible, before this kernel touches global memory, and then
// lets the next kernel be scheduled likewise (one kernel ahead at most).  For
// a kernel launched without the attribute both instructions do nothing.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// D2Q9 links (Sec. 3, Fig. 1 caption: odd i are the longer links; App. A
// weights w_0 = 4/9, w_odd = 1/36, w_even = 1/9).  Link i = 1..8 runs
// counter-clockwise from (1, 1).  Written as constexpr functions so that
// every use inside an unrolled loop folds to an immediate.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int lcx(int i) {
    return (i == 1 || i == 7 || i == 8) ? 1 : ((i == 3 || i == 4 || i == 5) ? -1 : 0);
}
__host__ __device__ constexpr int lcy(int i) {
    return (i == 1 || i == 2 || i == 3) ? 1 : ((i == 5 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr float lw(int i) {
    return i == 0 ? 4.0f / 9.0f : ((i & 1) ? 1.0f / 36.0f : 1.0f / 9.0f);
}
__host__ __device__ constexpr int lopp(int i) { return i == 0 ? 0 : ((i + 3) & 7) + 1; }
// Dellar's ghost basis g_i (App. A): 1, 4 (odd), -2 (even).
__host__ __device__ constexpr float lg(int i) { return i == 0 ? 1.0f : ((i & 1) ? 4.0f : -2.0f); }

// Column k^(p)_i of M^{-1} (App. A, the k vectors):
//   k0 = w(2 - 3/2 |c|^2), k1 = 3 w c_x, k2 = 3 w c_y, k3 = w(9/2 c_x^2 - 3/2),
//   k4 = w(9/2 c_y^2 - 3/2), k5 = 9 w c_x c_y, k6 = g w / 4,
//   k7 = 3/8 g w c_x, k8 = 3/8 g w c_y.
__host__ __device__ constexpr float kinv(int i, int p) {
    return p == 0 ? lw(i) * (2.0f - 1.5f * float(lcx(i) * lcx(i) + lcy(i) * lcy(i)))
         : p == 1 ? 3.0f * lw(i) * float(lcx(i))
         : p == 2 ? 3.0f * lw(i) * float(lcy(i))
         : p == 3 ? lw(i) * (4.5f * float(lcx(i) * lcx(i)) - 1.5f)
         : p == 4 ? lw(i) * (4.5f * float(lcy(i) * lcy(i)) - 1.5f)
         : p == 5 ? 9.0f * lw(i) * float(lcx(i) * lcy(i))
         : p == 6 ? 0.25f * lg(i) * lw(i)
         : p == 7 ? 0.375f * lg(i) * lw(i) * float(lcx(i))
                  : 0.375f * lg(i) * lw(i) * float(lcy(i));
}

// Unit link vector c-hat_i = c_i / |c_i| (Eq. eq_re_color), c-hat_0 = 0.
__host__ __device__ constexpr float chx(int i) {
    return (i & 1) ? float(lcx(i)) * 0.70710678118654752f : float(lcx(i));
}
__host__ __device__ constexpr float chy(int i) {
    return (i & 1) ? float(lcy(i)) * 0.70710678118654752f : float(lcy(i));
}

// Compact isotropic first derivative (Sec. 2; App. B with N = 1):
//   d_a X = 3 sum_i w_i X(r + c_i) c_ia
// written out: axis neighbours carry 1/3, diagonals 1/12.
// (the multiply-add written out, so that every kernel rounds it alike)
__device__ __forceinline__ float ddx(float e, float w, float ne, float nw, float se, float sw) {
    return fmaf(1.0f / 3.0f, e - w, (1.0f / 12.0f) * ((ne - nw) + (se - sw)));
}
__device__ __forceinline__ float ddy(float n, float s, float ne, float nw, float se, float sw) {
    return fmaf(1.0f / 3.0f, n - s, (1.0f / 12.0f) * ((ne - se) + (nw - sw)));
}

// Guard of the unit normal n-hat = -grad rho^N / |grad rho^N| (Sec. 2), which
// has no direction where the colour gradient vanishes (at the centre of a
// symmetric drop, at the symmetry points between drops): below kNormalTau
// the normal is taken as zero, so such a node gets no recolour bias and adds
// nothing to K.  The threshold sits above the FP32 round-off of the gradient
// (taken on the minority colour fraction, whose spacing is relative) and far
// below the gradient of any resolved interface.
constexpr float kNormalTau = 1e-9f;

__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }

// Segregation term of link i, w_i (s . c-hat_i) for a vector s (Eq. eq_re_color
// with phi_i = w_i phim folded into s).
__device__ __forceinline__ void segregation(float sx, float sy, float (&seg)[9]) {
    seg[0] = 0.0f;
    seg[8] = lw(8) * sx;
    seg[4] = -seg[8];
    seg[2] = lw(2) * sy;
    seg[6] = -seg[2];
    const float d1 = lw(1) * chx(1) * (sx + sy);
    const float d3 = lw(3) * chx(1) * (sy - sx);
    seg[1] = d1;
    seg[5] = -d1;
    seg[3] = d3;
    seg[7] = -d3;
}

// Reference dipoles of the 16-bit storage (cmrt_step.cu): per (red, blue)
// pair, the velocity term of the equilibrium, 3 w_i rho_C c_i . u, plus the
// segregation term of the recolour (Eq. eq_re_color), +/- w_i S . c-hat_i
// (red +, blue -), for the links c = (1, 0) (D[0]), (0, 1) (D[1]), (1, 1)
// (D[2]) and (-1, 1) (D[3]); the opposite links carry the negatives.
__device__ __forceinline__ void dipoles16(float rr, float rb, float ux, float uy, float sx, float sy,
                                          float2 (&D)[4]) {
    const float ar = 3.0f * rr, ab = 3.0f * rb;
    D[0] = make_float2(lw(8) * fmaf(ar, ux, sx), lw(8) * fmaf(ab, ux, -sx));
    D[1] = make_float2(lw(2) * fmaf(ar, uy, sy), lw(2) * fmaf(ab, uy, -sy));
    const float up = ux + uy, um = uy - ux;
    const float sp = chx(1) * (sx + sy), sm = chx(1) * (sy - sx);
    D[2] = make_float2(lw(1) * fmaf(ar, up, sp), lw(1) * fmaf(ab, up, -sp));
    D[3] = make_float2(lw(1) * fmaf(ar, um, sm), lw(1) * fmaf(ab, um, -sm));
}
// which dipole link i >= 1 carries, and whether negated (links 4, 6, 5, 7)
__host__ __device__ constexpr int dip_index(int i) {
    return (i == 8 || i == 4) ? 0 : (i == 2 || i == 6) ? 1 : (i == 1 || i == 5) ? 2 : 3;
}
__host__ __device__ constexpr bool dip_neg(int i) { return i == 4 || i == 6 || i == 5 || i == 7; }

// Collision in moment space of one node in increment form (App. A, Eq. 38
// minus m, and the reconstruction of Eq. eq84): f+ = f + M^{-1} dm with
// dm = Lambda (m^(0) - m) + S.  Inputs: the pre-collision populations f, the
// colour densities, the local kinematic viscosity nu (Sec. 2), the
// force-adjusted velocity, the force G, grad Phi' and div u.  The increments
// are small, so FP32 rounding stays at the level of population storage.  The
// reconstruction M^{-1} dm is grouped by the parity of each column k^(p)
// under c -> -c, which the k vectors of App. A have by construction.
__device__ __forceinline__ void collide_increment(const float (&f)[9], float rr, float rb, float rho, float nu,
                                                  float ux, float uy, float Gx, float Gy, float dPx, float dPy,
                                                  float divu, const StepParams& P, float (&fp)[9]) {
    const float lam3 = 2.0f * rcp(fmaf(6.0f, nu, 1.0f));
    const float a = fmaf(-0.5f, lam3, 1.0f);
    // correction tensor C_ab (App. A, Eq. Correction)
    const float qx = Gx - dPx, qy = Gy - dPy;
    const float iso = fmaf(ux, dPx, fmaf(uy, dPy, -rho * divu * (1.0f / 3.0f)));
    const float Cxx = a * fmaf(2.0f * ux, qx, -iso);
    const float Cyy = a * fmaf(2.0f * uy, qy, -iso);
    const float Cxy = a * fmaf(ux, qy, uy * qx);
    // modes that relax (Table 1 rows 3..8, unweighted): Pi_xx, Pi_yy, Pi_xy, N, J_x, J_y
    const float dsum = (f[1] + f[5]) + (f[3] + f[7]);  // diagonals
    const float ax = f[4] + f[8], ay = f[2] + f[6];
    const float pxx = dsum + ax;
    const float pyy = dsum + ay;
    const float pxy = (f[1] + f[5]) - (f[3] + f[7]);
    const float gN = fmaf(lg(1), dsum, fmaf(lg(2), ax + ay, f[0]));
    const float gJx = fmaf(lg(1), (f[1] + f[7]) - (f[3] + f[5]), lg(8) * (f[8] - f[4]));
    const float gJy = fmaf(lg(1), (f[1] + f[3]) - (f[5] + f[7]), lg(2) * (f[2] - f[6]));
    // dm = lambda (m^(0) - m) + S with the equilibria h^(p).f^(0) and
    // sources S^(p) of App. A (S^(1,2) = G, S^(3..5) = C)
    const float pres = fmaf(P.cs2_r, rr, P.cs2_b * rb);
    const float Neq = (P.ghost_N_mode == 0) ? fmaf(P.neq_r, rr, P.neq_b * rb) : 0.0f;
    const float rux = rho * ux;
    const float dm1 = Gx, dm2 = Gy;
    const float dm3 = fmaf(lam3, fmaf(rux, ux, pres) - pxx, Cxx);
    const float dm4 = fmaf(lam3, fmaf(rho * uy, uy, pres) - pyy, Cyy);
    const float dm5 = fmaf(lam3, fmaf(rux, uy, -pxy), Cxy);
    const float dm6 = P.lambda6 * (Neq - gN);
    const float dm7 = -P.lambda7 * gJx;
    const float dm8 = -P.lambda7 * gJy;
    // f+ - f = M^{-1} dm (App. A, Eq. eq84), grouped by parity of k^(p)
    float df[9];
    df[0] = fmaf(kinv(0, 3), dm3 + dm4, kinv(0, 6) * dm6);
    const float ex8 = fmaf(kinv(8, 3), dm3, fmaf(kinv(8, 4), dm4, kinv(8, 6) * dm6));
    const float ox8 = fmaf(kinv(8, 1), dm1, kinv(8, 7) * dm7);
    const float ey2 = fmaf(kinv(2, 3), dm3, fmaf(kinv(2, 4), dm4, kinv(2, 6) * dm6));
    const float oy2 = fmaf(kinv(2, 2), dm2, kinv(2, 8) * dm8);
    df[8] = ex8 + ox8;
    df[4] = ex8 - ox8;
    df[2] = ey2 + oy2;
    df[6] = ey2 - oy2;
    const float ed = fmaf(kinv(1, 3), dm3 + dm4, kinv(1, 6) * dm6);
    const float exy = kinv(1, 5) * dm5;
    const float odx = fmaf(kinv(1, 1), dm1, kinv(1, 7) * dm7);
    const float ody = fmaf(kinv(1, 2), dm2, kinv(1, 8) * dm8);
    const float pe = ed + exy, me = ed - exy, q1 = odx + ody, q2 = odx - ody;
    df[1] = pe + q1;  // (+1, +1)
    df[5] = pe - q1;  // (-1, -1)
    df[7] = me + q2;  // (+1, -1)
    df[3] = me - q2;  // (-1, +1)
#pragma unroll
    for (int i = 0; i < 9; ++i) fp[i] = f[i] + df[i];  // f+ = f + M^{-1} dm
}

// Store of the post-collision, recoloured populations of one node (Eq.
// eq_re_color) in the FP32 layout float[18][nodes] at `out` (the node's
// address in plane 0).  The minority colour is formed directly and the
// majority as the rest of f+, so that R++ + B++ = f+ holds to one rounding of
// the majority.  (sx, sy) is the red segregation vector
// beta phi rho_R rho_B / rho e.
__device__ __forceinline__ void store_recoloured_f32(float* out, size_t nodes, const float (&fp)[9], float rr,
                                                     float rb, float inv_rho, float sx, float sy) {
    const bool red_major = rr >= rb;
    const float amin = (red_major ? rb : rr) * inv_rho;
    const float smin = red_major ? -1.0f : 1.0f;  // minority's sign of the segregation term
    float seg[9];
    segregation(smin * sx, smin * sy, seg);
    float* out_min = out + (red_major ? 9 * nodes : 0);
    float* out_maj = out + (red_major ? 0 : 9 * nodes);
    // links in pairs as packed FP32x2 FMAs (fp - cmin as cmin * -1 + fp: the
    // same single rounding as the subtraction)
    const float2 a2 = make_float2(amin, amin), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
        const float2 f2 = make_float2(fp[i], fp[i + 1]);
        const float2 cmin = __ffma2_rn(a2, f2, make_float2(seg[i], seg[i + 1]));
        const float2 cmaj = __ffma2_rn(cmin, m1, f2);
        __stcs(out_min + i * nodes, cmin.x);
        __stcs(out_min + (i + 1) * nodes, cmin.y);
        __stcs(out_maj + i * nodes, cmaj.x);
        __stcs(out_maj + (i + 1) * nodes, cmaj.y);
    }
    const float cmin8 = fmaf(amin, fp[8], seg[8]);
    __stcs(out_min + 8 * nodes, cmin8);
    __stcs(out_maj + 8 * nodes, fp[8] - cmin8);
}

}  // namespace cmrt
