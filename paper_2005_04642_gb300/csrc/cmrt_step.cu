// Fused chromodynamic MRT step (arXiv 2005.04642, Sec. 2, Sec. 3, App. A)
// as one row-marching kernel for sm_103a.
//
// Data layout in HBM: the state is the post-collision (pre-streaming)
// populations P_{t-1} as 18 planes float[18][ny][nx] (red links 0..8, then
// blue links 0..8).  One launch gathers the pre-collision populations
// f(t) = stream(P_{t-1}) on the fly ("pull"), performs the whole per-node
// update and writes P_t to the other buffer at the node itself, so every
// HBM access is coalesced: 72 B read + 72 B written per node.
//
// A CTA of 128 threads owns a strip of 120 columns (plus 4 halo columns on
// each side, 128 in all: one thread per column) and marches down a segment
// of rows.  Rows of post-collision populations stream into an 8-row ring in
// shared memory with 16-byte cp.async copies, two rows ahead of use.  Each
// iteration runs a wavefront of four stages on consecutive rows, each stage
// reading only what the previous one left in shared memory:
//   A (row s-1)  gather f, colour moments, rho^N, Phi'          (tile + 3)
//   B (row s-2)  grad rho^N and n-hat with the compact stencil   (tile + 2)
//   C (row s-3)  K = div n-hat, force G, force-adjusted u        (tile + 1)
//   D (row s-4)  grad Phi', div u, C_ab, MRT collision in moment
//                space, reconstruction, recolour, store          (tile)
// so the stencil chain of radius 3 costs only the recomputation of the halo
// moments and never re-reads HBM.
//
// The collision is written in increment form, f+ = f + M^{-1} dm with
// dm = Lambda (m^(0) - m) + S (App. A, Eq. 38 minus m): the increments are
// small, so FP32 rounding stays at the level of population storage.
#include "cmrt_device.cuh"

namespace cmrt {
namespace {

constexpr int kPlanes = 18;
constexpr int kPopFloats = kRing * kPlanes * kWin;
// ring A: rho^N, Phi', rho, j_x, j_y over 8 rows
constexpr int kAF = 5;
constexpr int kAFloats = 8 * kAF * kWin;
// ring B: grad rho^N (x, y), n-hat (x, y) over 4 rows
constexpr int kBF = 4;
constexpr int kBFloats = 4 * kBF * kWin;
// ring C: G (x, y), u (x, y) over 4 rows
constexpr int kCF = 4;
constexpr int kCFloats = 4 * kCF * kWin;
constexpr int kSmemFloats = kPopFloats + kAFloats + kBFloats + kCFloats;

struct Rings {
    float* pop;
    float* a;
    float* b;
    float* c;
    __device__ __forceinline__ float* P(int row, int q) const {
        return pop + (((row & (kRing - 1)) * kPlanes) + q) * kWin;
    }
    __device__ __forceinline__ float* A(int row, int f) const { return a + (((row & 7) * kAF) + f) * kWin; }
    __device__ __forceinline__ float* B(int row, int f) const { return b + (((row & 3) * kBF) + f) * kWin; }
    __device__ __forceinline__ float* C(int row, int f) const { return c + (((row & 3) * kCF) + f) * kWin; }
};

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrap(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// Issue the asynchronous copy of post-collision row `row` (unwrapped index)
// of the window [x0 - 4, x0 + 124) into its ring slot.
template <bool VEC>
__device__ __forceinline__ void issue_row(const Rings& R, const float* __restrict__ src, int row, int x0,
                                          int nx, int ny, size_t plane) {
    const int gy = wrap(row, ny);
    const float* base = src + static_cast<size_t>(gy) * nx;
    if (VEC) {
        constexpr int kChunks = kWin / 4;
        for (int c = threadIdx.x; c < kPlanes * kChunks; c += kThreads) {
            const int q = c / kChunks;
            const int w4 = (c - q * kChunks) * 4;
            const int gx = wrap(x0 - kHalo + w4, nx);
            cp_async16(R.P(row, q) + w4, base + q * plane + gx);
        }
    } else {
        for (int c = threadIdx.x; c < kPlanes * kWin; c += kThreads) {
            const int q = c / kWin;
            const int w = c - q * kWin;
            const int gx = wrap(x0 - kHalo + w, nx);
            cp_async4(R.P(row, q) + w, base + q * plane + gx);
        }
    }
}

// Pre-collision populations at (row y, window column t): pull from the
// post-collision ring, f_i(r) = P_i(r - c_i) (Eq. equ_evolution), with
// half-way bounce-back P_opp(i)(r) where r - c_i lies beyond a wall.
__device__ __forceinline__ void gather(const Rings& R, int y, int t, bool walls, int ny, float (&fr)[9],
                                       float (&fb)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sy = y - lcy(i);
        if (walls && (sy < 0 || sy >= ny)) {
            fr[i] = R.P(y, lopp(i))[t];
            fb[i] = R.P(y, 9 + lopp(i))[t];
        } else {
            fr[i] = R.P(sy, i)[t - lcx(i)];
            fb[i] = R.P(sy, 9 + i)[t - lcx(i)];
        }
    }
}

// Compact derivative of a ring field at (row y, column t).
template <typename Row>
__device__ __forceinline__ void grad_at(Row rowp, int y, int t, float& gx, float& gy) {
    const float* n = rowp(y + 1);
    const float* m = rowp(y);
    const float* s = rowp(y - 1);
    gx = ddx(m[t + 1], m[t - 1], n[t + 1], n[t - 1], s[t + 1], s[t - 1]);
    gy = ddy(n[t], s[t], n[t + 1], n[t - 1], s[t + 1], s[t - 1]);
}

template <bool VEC, Pass MODE>
__global__ void __launch_bounds__(kThreads, 2)
    k_chain(const float* __restrict__ src, float* __restrict__ dst, const StepParams P, const int rows,
            FieldOut fo, unsigned* __restrict__ flag, double* __restrict__ partials) {
    extern __shared__ __align__(16) float smem[];
    Rings R{smem, smem + kPopFloats, smem + kPopFloats + kAFloats, smem + kPopFloats + kAFloats + kBFloats};

    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const bool walls = P.wall_y != 0;
    const size_t plane = static_cast<size_t>(nx) * ny;
    const int x0 = blockIdx.x * kTileX;
    const int y0 = blockIdx.y * rows;
    const int y_end = min(y0 + rows, ny);
    const int s_first = y0 - 4;
    const int s_last = y_end + 3;
    const int iters = (y_end - y0) + 8;
    auto row_ok = [&](int r) { return !walls || (r >= 0 && r < ny); };

    // diagnostics accumulators (Pass::Diag)
    double acc_r = 0.0, acc_b = 0.0, acc_jx = 0.0, acc_jy = 0.0, acc_u2 = 0.0, acc_bad = 0.0;

    if (row_ok(s_first)) issue_row<VEC>(R, src, s_first, x0, nx, ny, plane);
    cp_commit();
    if (row_ok(s_first + 1)) issue_row<VEC>(R, src, s_first + 1, x0, nx, ny, plane);
    cp_commit();

    for (int k = 0; k < iters; ++k) {
        const int s = s_first + k;
        cp_wait<1>();
        __syncthreads();
        if (s + 2 <= s_last && row_ok(s + 2)) issue_row<VEC>(R, src, s + 2, x0, nx, ny, plane);
        cp_commit();

        // ---------------- stage A: moments at row ya = s - 1 (tile + 3 halo)
        {
            const int ya = s - 1;
            if (ya >= y0 - 3 && ya <= y_end + 2 && row_ok(ya) && t >= 1 && t < kWin - 1) {
                float fr[9], fb[9];
                gather(R, ya, t, walls, ny, fr, fb);
                float rr = 0.f, rb = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    rr += fr[i];
                    rb += fb[i];
                    const float f = fr[i] + fb[i];
                    if (lcx(i) != 0) jx += float(lcx(i)) * f;
                    if (lcy(i) != 0) jy += float(lcy(i)) * f;
                }
                const float a = rr * P.inv_rho0_r;
                const float b = rb * P.inv_rho0_b;
                const float rn = (a - b) / (a + b);          // Eq. equ_rhoN_def
                const float phip = P.phip_r * rr + P.phip_b * rb;  // App. A, Phi'
                R.A(ya, 0)[t] = rn;
                R.A(ya, 1)[t] = phip;
                R.A(ya, 2)[t] = rr + rb;
                R.A(ya, 3)[t] = jx;
                R.A(ya, 4)[t] = jy;
                if (walls && ya == 0) {  // even mirror beyond y = -1/2
                    R.A(-1, 0)[t] = rn;
                    R.A(-1, 1)[t] = phip;
                }
                if (walls && ya == ny - 1) {  // even mirror beyond y = ny - 1/2
                    R.A(ny, 0)[t] = rn;
                    R.A(ny, 1)[t] = phip;
                }
            }
        }
        __syncthreads();

        // ---------------- stage B: grad rho^N, n-hat at row yb = s - 2 (tile + 2)
        {
            const int yb = s - 2;
            if (yb >= y0 - 2 && yb <= y_end + 1 && row_ok(yb) && t >= 2 && t < kWin - 2) {
                float gx, gy;
                grad_at([&](int r) { return R.A(r, 0); }, yb, t, gx, gy);
                // n-hat = -grad rho^N / |grad rho^N| (Sec. 2), regularised below kNormalEps
                const float mag2 = gx * gx + gy * gy;
                const float inv = (mag2 >= kNormalEps * kNormalEps) ? rsqrtf(mag2) : (1.0f / kNormalEps);
                const float nhx = -gx * inv;
                const float nhy = -gy * inv;
                R.B(yb, 0)[t] = gx;
                R.B(yb, 1)[t] = gy;
                R.B(yb, 2)[t] = nhx;
                R.B(yb, 3)[t] = nhy;
                if (walls && yb == 0) {  // reflected normal beyond the wall
                    R.B(-1, 2)[t] = nhx;
                    R.B(-1, 3)[t] = -nhy;
                }
                if (walls && yb == ny - 1) {
                    R.B(ny, 2)[t] = nhx;
                    R.B(ny, 3)[t] = -nhy;
                }
            }
        }
        __syncthreads();

        // ---------------- stage C: curvature, force, velocity at row yc = s - 3 (tile + 1)
        {
            const int yc = s - 3;
            if (yc >= y0 - 1 && yc <= y_end && row_ok(yc) && t >= 3 && t < kWin - 3) {
                float K;
                if (P.curvature_mode == 0) {
                    float dnx, dny, unused;
                    grad_at([&](int r) { return R.B(r, 2); }, yc, t, dnx, unused);
                    grad_at([&](int r) { return R.B(r, 3); }, yc, t, unused, dny);
                    K = dnx + dny;  // K = div n-hat (Sec. 2)
                } else {
                    K = P.fixed_K;
                }
                const float gx = R.B(yc, 0)[t];
                const float gy = R.B(yc, 1)[t];
                const float rho = R.A(yc, 2)[t];
                // G = sigma K grad rho^N / 2 + rho g_acc + g_vol (Eq. equ_stforce plus body force)
                const float Gx = P.half_sigma * K * gx + rho * P.gacc_x + P.gvol_x;
                const float Gy = P.half_sigma * K * gy + rho * P.gacc_y + P.gvol_y;
                const float inv_rho = 1.0f / rho;
                // force-adjusted velocity (Eq. equ_u_def)
                const float ux = (R.A(yc, 3)[t] + 0.5f * Gx) * inv_rho;
                const float uy = (R.A(yc, 4)[t] + 0.5f * Gy) * inv_rho;
                R.C(yc, 0)[t] = Gx;
                R.C(yc, 1)[t] = Gy;
                R.C(yc, 2)[t] = ux;
                R.C(yc, 3)[t] = uy;
                if (walls && yc == 0) {  // no-slip: odd mirror of u
                    R.C(-1, 2)[t] = -ux;
                    R.C(-1, 3)[t] = -uy;
                }
                if (walls && yc == ny - 1) {
                    R.C(ny, 2)[t] = -ux;
                    R.C(ny, 3)[t] = -uy;
                }
            }
        }
        __syncthreads();

        // ---------------- stage D: collide, recolour, store at row yd = s - 4 (tile)
        {
            const int yd = s - 4;
            const int gxo = x0 + t - kHalo;
            if (yd >= y0 && yd < y_end && t >= kHalo && t < kWin - kHalo && gxo < nx) {
                float fr[9], fb[9];
                gather(R, yd, t, walls, ny, fr, fb);
                float rr = 0.f, rb = 0.f, f[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    rr += fr[i];
                    rb += fb[i];
                    f[i] = fr[i] + fb[i];
                }
                const float rho = rr + rb;
                const float ux = R.C(yd, 2)[t];
                const float uy = R.C(yd, 3)[t];
                if (MODE == Pass::Step) {
                    if (!isfinite(rho)) atomicOr(flag, 1u);
                    const float Gx = R.C(yd, 0)[t];
                    const float Gy = R.C(yd, 1)[t];
                    float dPx, dPy, dux, duy, unused;
                    grad_at([&](int r) { return R.A(r, 1); }, yd, t, dPx, dPy);
                    grad_at([&](int r) { return R.C(r, 2); }, yd, t, dux, unused);
                    grad_at([&](int r) { return R.C(r, 3); }, yd, t, unused, duy);
                    const float divu = dux + duy;
                    const float inv_rho = 1.0f / rho;
                    // local shear eigenvalue (Sec. 2: nu(rho^N) = (2/lambda_3 - 1)/6)
                    float nu;
                    if (P.visc_mode == 0) {
                        const float rn = R.A(yd, 0)[t];
                        nu = 0.5f * P.nu_r * (1.0f + rn) + 0.5f * P.nu_b * (1.0f - rn);
                    } else {
                        nu = P.eta * inv_rho;
                    }
                    const float lam3 = 2.0f / (6.0f * nu + 1.0f);
                    const float a = 1.0f - 0.5f * lam3;
                    // correction tensor C_ab (App. A, Eq. Correction)
                    const float iso = ux * dPx + uy * dPy - rho * divu * (1.0f / 3.0f);
                    const float Cxx = a * (2.0f * ux * (Gx - dPx) - iso);
                    const float Cyy = a * (2.0f * uy * (Gy - dPy) - iso);
                    const float Cxy = a * (ux * (Gy - dPy) + uy * (Gx - dPx));
                    // modes m = M f that relax (Table 1, rows 3..8; unweighted)
                    float pxx = 0.f, pyy = 0.f, pxy = 0.f, gN = 0.f, gJx = 0.f, gJy = 0.f;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (lcx(i) != 0) pxx += f[i];
                        if (lcy(i) != 0) pyy += f[i];
                        if (lcx(i) * lcy(i) != 0) pxy += float(lcx(i) * lcy(i)) * f[i];
                        gN += lg(i) * f[i];
                        if (lcx(i) != 0) gJx += lg(i) * float(lcx(i)) * f[i];
                        if (lcy(i) != 0) gJy += lg(i) * float(lcy(i)) * f[i];
                    }
                    // equilibria h^(p).f^(0) (App. A) and sources S^(p)
                    const float pres = P.cs2_r * rr + P.cs2_b * rb;
                    const float Neq = (P.ghost_N_mode == 0) ? (P.neq_r * rr + P.neq_b * rb) : 0.0f;
                    float dm[9];
                    dm[0] = 0.0f;
                    dm[1] = Gx;
                    dm[2] = Gy;
                    dm[3] = lam3 * (pres + rho * ux * ux - pxx) + Cxx;
                    dm[4] = lam3 * (pres + rho * uy * uy - pyy) + Cyy;
                    dm[5] = lam3 * (rho * ux * uy - pxy) + Cxy;
                    dm[6] = P.lambda6 * (Neq - gN);
                    dm[7] = -P.lambda7 * gJx;
                    dm[8] = -P.lambda7 * gJy;
                    // recolour (Eq. eq_re_color): red along e = grad rho^N/|grad rho^N| = -n-hat
                    const float ex = -R.B(yd, 2)[t];
                    const float ey = -R.B(yd, 3)[t];
                    const float aR = rr * inv_rho;
                    const float aB = rb * inv_rho;
                    const float phim = (P.kphi_r * rr + P.kphi_b * rb) * inv_rho;  // phi_i / w_i, i != 0
                    const float seg = P.beta * rr * rb * inv_rho * phim;
                    const bool red_major = rr >= rb;
                    const size_t o = static_cast<size_t>(yd) * nx + gxo;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        float df = 0.0f;
#pragma unroll
                        for (int p = 1; p < 9; ++p) {
                            if (kinv(i, p) != 0.0f) df = fmaf(kinv(i, p), dm[p], df);
                        }
                        const float fp = f[i] + df;  // f+ = f + M^{-1} dm
                        float d = 0.0f;
                        if (i != 0) d = seg * lw(i) * (chx(i) * ex + chy(i) * ey);
                        // the minority colour directly, the majority as the rest of f+,
                        // so that R++ + B++ = f+ holds to one rounding of the majority
                        const float r_pp = fmaf(aR, fp, d);
                        const float b_pp = fmaf(aB, fp, -d);
                        dst[i * plane + o] = red_major ? fp - b_pp : r_pp;
                        dst[(9 + i) * plane + o] = red_major ? b_pp : fp - r_pp;
                    }
                } else if (MODE == Pass::Fields) {
                    const size_t o = static_cast<size_t>(yd) * nx + gxo;
                    if (fo.rho_r) fo.rho_r[o] = rr;
                    if (fo.rho_b) fo.rho_b[o] = rb;
                    if (fo.ux) fo.ux[o] = ux;
                    if (fo.uy) fo.uy[o] = uy;
                    if (fo.p) fo.p[o] = P.cs2_r * rr + P.cs2_b * rb;
                } else {
                    float jx = 0.f, jy = 0.f;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (lcx(i) != 0) jx += float(lcx(i)) * f[i];
                        if (lcy(i) != 0) jy += float(lcy(i)) * f[i];
                    }
                    if (isfinite(rho)) {
                        acc_r += rr;
                        acc_b += rb;
                        acc_jx += jx;
                        acc_jy += jy;
                        acc_u2 = fmax(acc_u2, static_cast<double>(ux) * ux + static_cast<double>(uy) * uy);
                    } else {
                        acc_bad += 1.0;
                    }
                }
            }
        }
    }
    cp_wait<0>();

    if (MODE == Pass::Diag) {
        // warp shuffle reduction, then across the CTA's warps in shared memory
        double v[kDiagSlots] = {acc_r, acc_b, acc_jx, acc_jy, acc_u2, acc_bad};
#pragma unroll
        for (int j = 0; j < kDiagSlots; ++j) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double o = __shfl_down_sync(0xffffffffu, v[j], off);
                v[j] = (j == 4) ? fmax(v[j], o) : v[j] + o;
            }
        }
        __syncthreads();
        double* red = reinterpret_cast<double*>(smem);
        const int warp = t >> 5, lane = t & 31;
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < kDiagSlots; ++j) red[warp * kDiagSlots + j] = v[j];
        }
        __syncthreads();
        if (t < kDiagSlots) {
            double acc = red[t];
            for (int w = 1; w < kThreads / 32; ++w) {
                const double o = red[w * kDiagSlots + t];
                acc = (t == 4) ? fmax(acc, o) : acc + o;
            }
            partials[(static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x) * kDiagSlots + t] = acc;
        }
    }
}

__global__ void k_diag_reduce(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double red[kThreads / 32][kDiagSlots];
    double v[kDiagSlots] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < kDiagSlots; ++j) {
            const double o = partials[static_cast<size_t>(b) * kDiagSlots + j];
            v[j] = (j == 4) ? fmax(v[j], o) : v[j] + o;
        }
    }
#pragma unroll
    for (int j = 0; j < kDiagSlots; ++j) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v[j], off);
            v[j] = (j == 4) ? fmax(v[j], o) : v[j] + o;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kDiagSlots; ++j) red[warp][j] = v[j];
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        double acc = red[0][threadIdx.x];
        for (int w = 1; w < kThreads / 32; ++w) {
            const double o = red[w][threadIdx.x];
            acc = (threadIdx.x == 4) ? fmax(acc, o) : acc + o;
        }
        out[threadIdx.x] = acc;
    }
}

template <Pass MODE>
cudaError_t launch_chain(const float* src, float* dst, const StepParams& P, int rows, FieldOut fo,
                         unsigned* flag, double* partials, cudaStream_t s) {
    const bool vec = (P.nx % 4) == 0;
    const size_t smem = chain_smem_bytes();
    const dim3 grid = chain_grid(P.nx, P.ny, rows);
    cudaError_t e;
    if (vec) {
        e = cudaFuncSetAttribute(k_chain<true, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_chain<true, MODE><<<grid, kThreads, smem, s>>>(src, dst, P, rows, fo, flag, partials);
    } else {
        e = cudaFuncSetAttribute(k_chain<false, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_chain<false, MODE><<<grid, kThreads, smem, s>>>(src, dst, P, rows, fo, flag, partials);
    }
    return cudaGetLastError();
}

}  // namespace

size_t chain_smem_bytes() { return sizeof(float) * static_cast<size_t>(kSmemFloats); }

dim3 chain_grid(int nx, int ny, int rows) {
    return dim3(static_cast<unsigned>((nx + kTileX - 1) / kTileX), static_cast<unsigned>((ny + rows - 1) / rows), 1);
}

cudaError_t launch_step(const float* src, float* dst, const StepParams& P, int rows, unsigned* flag,
                        cudaStream_t s) {
    return launch_chain<Pass::Step>(src, dst, P, rows, FieldOut{}, flag, nullptr, s);
}

cudaError_t launch_fields(const float* src, const StepParams& P, int rows, FieldOut out, cudaStream_t s) {
    return launch_chain<Pass::Fields>(src, nullptr, P, rows, out, nullptr, nullptr, s);
}

cudaError_t launch_diag_partials(const float* src, const StepParams& P, int rows, double* partials,
                                 cudaStream_t s) {
    return launch_chain<Pass::Diag>(src, nullptr, P, rows, FieldOut{}, nullptr, partials, s);
}

cudaError_t launch_diag_reduce(const double* partials, int nblocks, double* out, cudaStream_t s) {
    k_diag_reduce<<<1, kThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace cmrt
