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
// small, so FP32 rounding stays at the level of population storage.  The
// reconstruction M^{-1} dm is grouped by the parity of each column k^(p)
// under c -> -c, which the k vectors of App. A have by construction.
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
// 16-byte chunks of one ring row (18 planes x 128 columns) and chunks per thread
constexpr int kChunksPerPlane = kWin / 4;
constexpr int kRowChunks = kPlanes * kChunksPerPlane;
constexpr int kChunkIters = (kRowChunks + kThreads - 1) / kThreads;

// The reconstruction below relies on these symmetries of App. A's k vectors.
static_assert(kinv(4, 3) == kinv(8, 3) && kinv(4, 4) == kinv(8, 4) && kinv(4, 6) == kinv(8, 6), "even x");
static_assert(kinv(4, 1) == -kinv(8, 1) && kinv(4, 7) == -kinv(8, 7), "odd x");
static_assert(kinv(6, 3) == kinv(2, 3) && kinv(6, 4) == kinv(2, 4) && kinv(6, 6) == kinv(2, 6), "even y");
static_assert(kinv(6, 2) == -kinv(2, 2) && kinv(6, 8) == -kinv(2, 8), "odd y");
static_assert(kinv(2, 3) == kinv(8, 4) && kinv(2, 4) == kinv(8, 3) && kinv(2, 2) == kinv(8, 1) &&
              kinv(2, 8) == kinv(8, 7), "x <-> y");
static_assert(kinv(1, 3) == kinv(1, 4) && kinv(1, 1) == kinv(1, 2) && kinv(1, 7) == kinv(1, 8), "diagonal");
static_assert(kinv(8, 2) == 0.f && kinv(8, 5) == 0.f && kinv(8, 8) == 0.f && kinv(0, 1) == 0.f &&
              kinv(0, 5) == 0.f && kinv(0, 7) == 0.f, "zeros");

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

__device__ __forceinline__ void cp_async16(unsigned smem_addr, const float* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned smem_addr, const float* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
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

__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }

// Per-thread plan of the asynchronous row copies: which 16-byte chunks of a
// ring row this thread fetches, as (shared offset, global offset) pairs that
// are the same for every row of the strip.
template <bool VEC>
struct CopyPlan {
    static constexpr int kN = VEC ? kChunkIters : kPlanes;
    unsigned soff[kN];  // byte offset inside a ring row
    size_t goff[kN];    // element offset inside a global row (plane * nx * ny + column)
    int n;

    __device__ __forceinline__ void init(int x0, int nx, size_t plane) {
        n = 0;
        if (VEC) {
#pragma unroll
            for (int m = 0; m < kN; ++m) {
                const int c = threadIdx.x + m * kThreads;
                const int q = c / kChunksPerPlane;
                const int w4 = (c - q * kChunksPerPlane) * 4;
                soff[m] = static_cast<unsigned>((q * kWin + w4) * sizeof(float));
                goff[m] = static_cast<size_t>(q) * plane + wrap(x0 - kHalo + w4, nx);
                if (c < kRowChunks) n = m + 1;
            }
        } else {
            const int gx = wrap(x0 - kHalo + static_cast<int>(threadIdx.x), nx);
#pragma unroll
            for (int q = 0; q < kN; ++q) {
                soff[q] = static_cast<unsigned>((q * kWin + threadIdx.x) * sizeof(float));
                goff[q] = static_cast<size_t>(q) * plane + gx;
            }
            n = kN;
        }
    }

    __device__ __forceinline__ void issue(unsigned ring_row_addr, const float* grow) const {
#pragma unroll
        for (int m = 0; m < kN; ++m) {
            if (m < n) {
                if (VEC) cp_async16(ring_row_addr + soff[m], grow + goff[m]);
                else cp_async4(ring_row_addr + soff[m], grow + goff[m]);
            }
        }
    }
};

// Pre-collision populations at (row y, window column t): pull from the
// post-collision ring, f_i(r) = P_i(r - c_i) (Eq. equ_evolution), with
// half-way bounce-back P_opp(i)(r) where r - c_i lies beyond a wall.
// With PRE the rows hold pre-collision populations f(t) already in place
// (the public layout), so the node's own column is read unshifted.
template <bool WALLS, bool PRE = false>
__device__ __forceinline__ void gather(const Rings& R, int y, int t, int ny, float (&fr)[9], float (&fb)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sy = y - lcy(i);
        if (PRE) {
            fr[i] = R.P(y, i)[t];
            fb[i] = R.P(y, 9 + i)[t];
        } else if (WALLS && (sy < 0 || sy >= ny)) {
            fr[i] = R.P(y, lopp(i))[t];
            fb[i] = R.P(y, 9 + lopp(i))[t];
        } else {
            fr[i] = R.P(sy, i)[t - lcx(i)];
            fb[i] = R.P(sy, 9 + i)[t - lcx(i)];
        }
    }
}

__device__ __forceinline__ float sum9(const float (&v)[9]) {
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
}

// Compact derivatives of a ring field around (row y, column t).
template <typename Row>
__device__ __forceinline__ float ddx_at(Row rowp, int y, int t) {
    const float* n = rowp(y + 1);
    const float* m = rowp(y);
    const float* s = rowp(y - 1);
    return ddx(m[t + 1], m[t - 1], n[t + 1], n[t - 1], s[t + 1], s[t - 1]);
}
template <typename Row>
__device__ __forceinline__ float ddy_at(Row rowp, int y, int t) {
    const float* n = rowp(y + 1);
    const float* s = rowp(y - 1);
    return ddy(n[t], s[t], n[t + 1], n[t - 1], s[t + 1], s[t - 1]);
}

template <bool VEC, bool WALLS, Pass MODE, bool PRE = false>
__global__ void __launch_bounds__(kThreads, 2)
    k_chain(const float* __restrict__ src, float* __restrict__ dst, const StepParams P, const int rows,
            FieldOut fo, unsigned* __restrict__ flag, double* __restrict__ partials) {
    extern __shared__ __align__(16) float smem[];
    Rings R{smem, smem + kPopFloats, smem + kPopFloats + kAFloats, smem + kPopFloats + kAFloats + kBFloats};
    const unsigned pop_addr = static_cast<unsigned>(__cvta_generic_to_shared(smem));

    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const size_t plane = static_cast<size_t>(nx) * ny;
    const int x0 = blockIdx.x * kTileX;
    const int y0 = blockIdx.y * rows;
    const int y_end = min(y0 + rows, ny);
    const int s_first = y0 - 4;
    const int s_last = y_end + 3;
    const int iters = (y_end - y0) + 8;
    auto row_ok = [&](int r) { return !WALLS || (r >= 0 && r < ny); };

    CopyPlan<VEC> plan;
    plan.init(x0, nx, plane);
    auto issue_row = [&](int row) {
        const unsigned ring_row = pop_addr + static_cast<unsigned>((row & (kRing - 1)) * kPlanes * kWin * 4);
        plan.issue(ring_row, src + static_cast<size_t>(wrap(row, ny)) * nx);
    };

    // diagnostics accumulators (Pass::Diag)
    double acc_r = 0.0, acc_b = 0.0, acc_jx = 0.0, acc_jy = 0.0, acc_u2 = 0.0, acc_bad = 0.0;

    if (row_ok(s_first)) issue_row(s_first);
    cp_commit();
    if (row_ok(s_first + 1)) issue_row(s_first + 1);
    cp_commit();

    for (int k = 0; k < iters; ++k) {
        const int s = s_first + k;
        cp_wait<1>();
        __syncthreads();
        if (s + 2 <= s_last && row_ok(s + 2)) issue_row(s + 2);
        cp_commit();

        // ---------------- stage A: moments at row ya = s - 1 (tile + 3 halo)
        {
            const int ya = s - 1;
            if (ya >= y0 - 3 && ya <= y_end + 2 && row_ok(ya) && t >= 1 && t < kWin - 1) {
                float fr[9], fb[9];
                gather<WALLS, PRE>(R, ya, t, ny, fr, fb);
                const float rr = sum9(fr);
                const float rb = sum9(fb);
                // colour-blind momentum sum_i f_i c_i (Eq. equ_u_def)
                const float jx = ((fr[1] + fb[1]) + (fr[7] + fb[7])) + (fr[8] + fb[8]) -
                                 (((fr[3] + fb[3]) + (fr[5] + fb[5])) + (fr[4] + fb[4]));
                const float jy = ((fr[1] + fb[1]) + (fr[3] + fb[3])) + (fr[2] + fb[2]) -
                                 (((fr[5] + fb[5]) + (fr[7] + fb[7])) + (fr[6] + fb[6]));
                const float a = rr * P.inv_rho0_r;
                const float b = rb * P.inv_rho0_b;
                const float rn = (a - b) * rcp(a + b);             // Eq. equ_rhoN_def
                const float phip = fmaf(P.phip_r, rr, P.phip_b * rb);  // App. A, Phi'
                R.A(ya, 0)[t] = rn;
                R.A(ya, 1)[t] = phip;
                R.A(ya, 2)[t] = rr + rb;
                R.A(ya, 3)[t] = jx;
                R.A(ya, 4)[t] = jy;
                if (WALLS && ya == 0) {  // even mirror beyond y = -1/2
                    R.A(-1, 0)[t] = rn;
                    R.A(-1, 1)[t] = phip;
                }
                if (WALLS && ya == ny - 1) {  // even mirror beyond y = ny - 1/2
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
                auto rn_row = [&](int r) { return R.A(r, 0); };
                const float gx = ddx_at(rn_row, yb, t);
                const float gy = ddy_at(rn_row, yb, t);
                // n-hat = -grad rho^N / |grad rho^N| (Sec. 2), regularised below kNormalEps
                const float mag2 = fmaf(gx, gx, gy * gy);
                const float inv = (mag2 >= kNormalEps * kNormalEps) ? rsqrtf(mag2) : (1.0f / kNormalEps);
                const float nhx = -gx * inv;
                const float nhy = -gy * inv;
                R.B(yb, 0)[t] = gx;
                R.B(yb, 1)[t] = gy;
                R.B(yb, 2)[t] = nhx;
                R.B(yb, 3)[t] = nhy;
                if (WALLS && yb == 0) {  // reflected normal beyond the wall
                    R.B(-1, 2)[t] = nhx;
                    R.B(-1, 3)[t] = -nhy;
                }
                if (WALLS && yb == ny - 1) {
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
                    // K = div n-hat (Sec. 2)
                    K = ddx_at([&](int r) { return R.B(r, 2); }, yc, t) + ddy_at([&](int r) { return R.B(r, 3); }, yc, t);
                } else {
                    K = P.fixed_K;
                }
                const float gx = R.B(yc, 0)[t];
                const float gy = R.B(yc, 1)[t];
                const float rho = R.A(yc, 2)[t];
                // G = sigma K grad rho^N / 2 + rho g_acc + g_vol (Eq. equ_stforce plus body force)
                const float hk = P.half_sigma * K;
                const float Gx = fmaf(hk, gx, fmaf(rho, P.gacc_x, P.gvol_x));
                const float Gy = fmaf(hk, gy, fmaf(rho, P.gacc_y, P.gvol_y));
                const float inv_rho = rcp(rho);
                // force-adjusted velocity (Eq. equ_u_def)
                const float ux = fmaf(0.5f, Gx, R.A(yc, 3)[t]) * inv_rho;
                const float uy = fmaf(0.5f, Gy, R.A(yc, 4)[t]) * inv_rho;
                R.C(yc, 0)[t] = Gx;
                R.C(yc, 1)[t] = Gy;
                R.C(yc, 2)[t] = ux;
                R.C(yc, 3)[t] = uy;
                if (WALLS && yc == 0) {  // no-slip: odd mirror of u
                    R.C(-1, 2)[t] = -ux;
                    R.C(-1, 3)[t] = -uy;
                }
                if (WALLS && yc == ny - 1) {
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
                float fr[9], fb[9], f[9];
                gather<WALLS, PRE>(R, yd, t, ny, fr, fb);
                const float rr = sum9(fr);
                const float rb = sum9(fb);
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = fr[i] + fb[i];
                const float rho = rr + rb;
                const float ux = R.C(yd, 2)[t];
                const float uy = R.C(yd, 3)[t];
                if (MODE == Pass::Step) {
                    if (!isfinite(rho)) atomicOr(flag, 1u);
                    const float Gx = R.C(yd, 0)[t];
                    const float Gy = R.C(yd, 1)[t];
                    auto phip_row = [&](int r) { return R.A(r, 1); };
                    const float dPx = ddx_at(phip_row, yd, t);
                    const float dPy = ddy_at(phip_row, yd, t);
                    const float divu = ddx_at([&](int r) { return R.C(r, 2); }, yd, t) +
                                       ddy_at([&](int r) { return R.C(r, 3); }, yd, t);
                    const float inv_rho = rcp(rho);
                    // local shear eigenvalue (Sec. 2: nu(rho^N) = (2/lambda_3 - 1)/6)
                    float nu;
                    if (P.visc_mode == 0) {
                        const float rn = R.A(yd, 0)[t];
                        nu = fmaf(0.5f * (P.nu_r - P.nu_b), rn, 0.5f * (P.nu_r + P.nu_b));
                    } else {
                        nu = P.eta * inv_rho;
                    }
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
                    // recolour (Eq. eq_re_color): red moves along e = grad rho^N / |grad rho^N| = -n-hat,
                    // by beta phi_i rho_R rho_B / rho (e . c-hat_i); phi_i = w_i phim for i != 0
                    const float ex = -R.B(yd, 2)[t];
                    const float ey = -R.B(yd, 3)[t];
                    const float phim = fmaf(P.kphi_r, rr, P.kphi_b * rb) * inv_rho;
                    const float seg = P.beta * (rr * rb) * inv_rho * phim;
                    // the minority colour is formed directly and the majority as the rest
                    // of f+, so that R++ + B++ = f+ holds to one rounding of the majority
                    const bool red_major = rr >= rb;
                    const float amin = (red_major ? rb : rr) * inv_rho;
                    const float smin = red_major ? -seg : seg;  // minority's sign of the segregation term
                    const float sx = smin * ex, sy = smin * ey;
                    float dmin[9];
                    dmin[0] = 0.0f;
                    dmin[8] = lw(8) * sx;
                    dmin[4] = -dmin[8];
                    dmin[2] = lw(2) * sy;
                    dmin[6] = -dmin[2];
                    const float dd1 = lw(1) * chx(1) * (sx + sy);
                    const float dd3 = lw(3) * chx(1) * (sy - sx);
                    dmin[1] = dd1;
                    dmin[5] = -dd1;
                    dmin[3] = dd3;
                    dmin[7] = -dd3;
                    const size_t o = static_cast<size_t>(yd) * nx + gxo;
                    float* out_min = dst + o + (red_major ? 9 * plane : 0);
                    float* out_maj = dst + o + (red_major ? 0 : 9 * plane);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const float fp = f[i] + df[i];  // f+ = f + M^{-1} dm
                        const float cmin = fmaf(amin, fp, dmin[i]);
                        __stcs(out_min + i * plane, cmin);
                        __stcs(out_maj + i * plane, fp - cmin);
                    }
                } else if (MODE == Pass::Fields) {
                    const size_t o = static_cast<size_t>(yd) * nx + gxo;
                    if (fo.rho_r) fo.rho_r[o] = rr;
                    if (fo.rho_b) fo.rho_b[o] = rb;
                    if (fo.ux) fo.ux[o] = ux;
                    if (fo.uy) fo.uy[o] = uy;
                    if (fo.p) fo.p[o] = fmaf(P.cs2_r, rr, P.cs2_b * rb);
                } else {
                    const float jx = (f[1] + f[7] + f[8]) - (f[3] + f[4] + f[5]);
                    const float jy = (f[1] + f[2] + f[3]) - (f[5] + f[6] + f[7]);
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

template <bool VEC, bool WALLS, Pass MODE, bool PRE = false>
cudaError_t launch_one(const float* src, float* dst, const StepParams& P, int rows, FieldOut fo, unsigned* flag,
                       double* partials, cudaStream_t s) {
    // the shared-memory opt-in is per kernel and per device: set it once for each
    static unsigned long long configured = 0;
    const size_t smem = chain_smem_bytes();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(k_chain<VEC, WALLS, MODE, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    k_chain<VEC, WALLS, MODE, PRE><<<chain_grid(P.nx, P.ny, rows), kThreads, smem, s>>>(src, dst, P, rows, fo, flag,
                                                                                    partials);
    return cudaGetLastError();
}

template <Pass MODE>
cudaError_t launch_chain(const float* src, float* dst, const StepParams& P, int rows, FieldOut fo,
                         unsigned* flag, double* partials, cudaStream_t s) {
    const bool vec = (P.nx % 4) == 0;
    const bool walls = P.wall_y != 0;
    if (vec && walls) return launch_one<true, true, MODE>(src, dst, P, rows, fo, flag, partials, s);
    if (vec) return launch_one<true, false, MODE>(src, dst, P, rows, fo, flag, partials, s);
    if (walls) return launch_one<false, true, MODE>(src, dst, P, rows, fo, flag, partials, s);
    return launch_one<false, false, MODE>(src, dst, P, rows, fo, flag, partials, s);
}

}  // namespace

size_t chain_smem_bytes() { return sizeof(float) * static_cast<size_t>(kSmemFloats); }

dim3 chain_grid(int nx, int ny, int rows) {
    return dim3(static_cast<unsigned>((nx + kTileX - 1) / kTileX), static_cast<unsigned>((ny + rows - 1) / rows), 1);
}

int chain_rows(int nx, int ny, int sms) {
    // Rows per CTA: each CTA spends (rows + 8) row-iterations (8 fill the
    // pipeline), and the CTAs run in waves of (SMs x 2 resident CTAs); pick
    // the segment length that minimises waves x (rows + 8).
    const int strips = (nx + kTileX - 1) / kTileX;
    const long slots = 2L * (sms > 0 ? sms : 1);
    int best = 8;
    long best_cost = -1;
    for (int rows = 8; rows <= 512; rows += 8) {
        const long segs = (ny + rows - 1) / rows;
        const long waves = (strips * segs + slots - 1) / slots;
        const long cost = waves * (rows + 8);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = rows;
        }
        if (rows >= ny) break;
    }
    return best;
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

cudaError_t launch_diag_partials_pre(const float* pre, const StepParams& P, int rows, double* partials,
                                     cudaStream_t s) {
    const bool vec = (P.nx % 4) == 0;
    const bool walls = P.wall_y != 0;
    const FieldOut none{};
    if (vec && walls) return launch_one<true, true, Pass::Diag, true>(pre, nullptr, P, rows, none, nullptr, partials, s);
    if (vec) return launch_one<true, false, Pass::Diag, true>(pre, nullptr, P, rows, none, nullptr, partials, s);
    if (walls) return launch_one<false, true, Pass::Diag, true>(pre, nullptr, P, rows, none, nullptr, partials, s);
    return launch_one<false, false, Pass::Diag, true>(pre, nullptr, P, rows, none, nullptr, partials, s);
}

cudaError_t launch_diag_reduce(const double* partials, int nblocks, double* out, cudaStream_t s) {
    k_diag_reduce<<<1, kThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace cmrt
