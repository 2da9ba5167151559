// Device-side building blocks of the two-colour D2Q9 chromodynamic MRT step
// (arXiv 2005.04642).  Shared by the kernels of libcmrt; host code sees only
// the parameter block and the kernel launchers declared in cmrt_internal.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cmrt_internal.h"

namespace cmrt {

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
__device__ __forceinline__ float ddx(float e, float w, float ne, float nw, float se, float sw) {
    return (1.0f / 3.0f) * (e - w) + (1.0f / 12.0f) * ((ne - nw) + (se - sw));
}
__device__ __forceinline__ float ddy(float n, float s, float ne, float nw, float se, float sw) {
    return (1.0f / 3.0f) * (n - s) + (1.0f / 12.0f) * ((ne - se) + (nw - sw));
}

// Regularisation of the unit normal, n-hat = -grad rho^N / max(|grad rho^N|, eps):
// the paper's unit vector wherever an interface is resolved, shrinking smoothly
// to zero where the colour gradient vanishes (there its direction would be
// set by round-off).
constexpr float kNormalEps = 1e-4f;

}  // namespace cmrt
