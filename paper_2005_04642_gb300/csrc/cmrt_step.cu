// Fused chromodynamic MRT step (arXiv 2005.04642, Sec. 2, Sec. 3, App. A)
// as one row-marching kernel for sm_103a.
//
// Data layout in HBM: the state is the post-collision (pre-streaming)
// populations P_{t-1}.  With FP32 storage they are 18 planes
// float[18][ny][nx] (red links 0..8, then blue links 0..8).  With 16-bit
// storage (FP16 or BF16) a node keeps its two colour densities and its two
// rest populations in FP32 and twelve 16-bit (red, blue) pairs: four
// reference dipoles -- the equilibrium's velocity term and the recolour's
// segregation term -- and the deviations d_{C,i} = C_i - rho_C psi_i -/+ D_C
// of the eight moving links from a reference that scales with the node's own
// colour density: planes 0 and 1 are float2[ny][nx] (rho_R, rho_B) and
// (R_0, B_0), planes 2..13 16-bit pairs.  The rest populations are the
// remainder of the densities after the decoded moving links, so a record
// decodes to populations summing to rho_C.
// One launch gathers the pre-collision populations f(t) = stream(P_{t-1})
// on the fly ("pull"), performs the whole per-node update and writes P_t to
// the other buffer at the node itself, so every HBM access is coalesced:
// 72 B (FP32) or 64 B (16-bit) read and as much written per node.
//
// A CTA owns a strip of 120 columns (plus 4 halo columns on each side, 128
// in all: one thread per column in each of its thread groups) and marches
// down a segment of rows.  Rows of the state stream into a 9-row ring in
// shared memory with 16-byte cp.async copies, two rows ahead of use.  Each
// iteration runs a wavefront of four stages on consecutive rows, each stage
// reading only what the previous one left in shared memory:
//   A (row s-1)  gather f, colour moments, red fraction, Phi'  (tile + 3)
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
#include <atomic>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cmrt_device.cuh"

namespace cmrt {
namespace {

constexpr int kPlanes = 18;
// Rings of stage results, four rows each (a row is one float per window
// column; fields x and y interleaved by row): the front's B and C write rows
// s - 2 and s - 3 of iteration k + 1 (that is, s - 1 and s - 2) while the
// back's D of iteration k may still read n-hat and G of row s - 4 and u of
// rows s - 5 .. s - 3; grad rho^N only C reads, on the front.  The mirrored
// rows beyond a wall share these slots: row -1 takes the slot of row 3, and
// row ny the slot of row ny - 4, written one row iteration after row ny - 1,
// when no stage reads row ny - 4 any more.
constexpr int kBFloats = (4 * 2 + 4 * 2) * kWin;  // grad rho^N, n-hat
constexpr int kCFloats = (4 * 2 + 4 * 2) * kWin;  // G, u

// The step runs warp-specialised: a CTA of 2 x kThreads threads, whose first
// kThreads ("front") stream the rows in and run stages A and B, and C with
// 16-bit storage, while the other kThreads ("back") run stage D, and C with
// FP32 storage, one row iteration behind them.
constexpr int kStepThreads = 2 * kThreads;
// Named barriers (0 is __syncthreads): the front among themselves; front ->
// back "the front's stages of iteration k are in shared memory" (kBarC) and
// back -> front "the back's stages of iteration k are done with their rows"
// (kBarD), each alternating between two ids by the parity of k so that no
// barrier sees arrivals of two iterations; the back among themselves between
// C and D.
constexpr int kBarFront = 1;
constexpr int kBarC = 2;  // 2, 3
constexpr int kBarD = 4;  // 4, 5
constexpr int kBarBack = 6;

template <int ID, int N>
__device__ __forceinline__ void bar_sync() {
    asm volatile("bar.sync %0, %1;\n" ::"n"(ID), "n"(N) : "memory");
}
template <int ID, int N>
__device__ __forceinline__ void bar_arrive() {
    asm volatile("bar.arrive %0, %1;\n" ::"n"(ID), "n"(N) : "memory");
}

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

__device__ __forceinline__ void cp_async16(unsigned smem_addr, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned smem_addr, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned smem_addr, const void* gmem) {
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

// (sum over links of r, of b), pairwise, as packed FP32x2 adds (one instruction per pair)
__device__ __forceinline__ float2 sum9x2(const float (&r)[9], const float (&b)[9]) {
    float2 v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = make_float2(r[i], b[i]);
    const float2 a = __fadd2_rn(__fadd2_rn(v[0], v[1]), __fadd2_rn(v[2], v[3]));
    const float2 c = __fadd2_rn(__fadd2_rn(v[4], v[5]), __fadd2_rn(v[6], v[7]));
    return __fadd2_rn(__fadd2_rn(a, c), v[8]);
}

// ---------------------------------------------------------------------------
// Storage layouts.  A layout fixes the bytes of one ring row, how a thread
// copies its share of a row from HBM, how stage A / D gather the 18
// pre-collision populations of a node from the ring, and how stage D stores
// the node's post-collision populations.
// ---------------------------------------------------------------------------

// 32-bit: 18 FP32 planes.
struct LayoutF32 {
    static constexpr bool kPrep = false;
    static constexpr bool kCFront = false;  // stage C on the back warps (see chain_tile)
    static constexpr int kSlotBytes = kPlanes * kWin * 4;
    static constexpr int kChunks = kSlotBytes / 16;
    static constexpr int kVecIters = (kChunks + kThreads - 1) / kThreads;
    static constexpr size_t node_bytes() { return kPlanes * 4; }

    template <bool VEC>
    struct Plan {
        static constexpr int kN = VEC ? kVecIters : kPlanes;
        unsigned soff[kN];  // byte offset inside a ring row
        size_t goff[kN];    // byte offset inside the state, row 0
        int n;
        __device__ __forceinline__ void init(int x0, int nx, size_t nodes) {
            n = 0;
            if (VEC) {
                constexpr int kPer = kWin / 4;
#pragma unroll
                for (int m = 0; m < kN; ++m) {
                    const int c = threadIdx.x + m * kThreads;
                    const int q = c / kPer;
                    const int w4 = (c - q * kPer) * 4;
                    soff[m] = static_cast<unsigned>((q * kWin + w4) * 4);
                    goff[m] = (static_cast<size_t>(q) * nodes + wrap(x0 - kHalo + w4, nx)) * 4;
                    if (c < kChunks) n = m + 1;
                }
            } else {
                const int gx = wrap(x0 - kHalo + static_cast<int>(threadIdx.x), nx);
#pragma unroll
                for (int q = 0; q < kN; ++q) {
                    soff[q] = static_cast<unsigned>((q * kWin + threadIdx.x) * 4);
                    goff[q] = (static_cast<size_t>(q) * nodes + gx) * 4;
                }
                n = kN;
            }
        }
        __device__ __forceinline__ void issue(unsigned slot_addr, const char* state, int gy, int nx) const {
            const char* row = state + static_cast<size_t>(gy) * nx * 4;
#pragma unroll
            for (int m = 0; m < kN; ++m) {
                if (m < n) {
                    if (VEC) cp_async16(slot_addr + soff[m], row + goff[m]);
                    else cp_async4(slot_addr + soff[m], row + goff[m]);
                }
            }
        }
    };

    __device__ __forceinline__ static void prep(char*, int, const StepParams&) {}
    __device__ __forceinline__ static const float* plane(const char* slot, int q) {
        return reinterpret_cast<const float*>(slot) + q * kWin;
    }
    // populations (red, blue) of link i of the node in column `col` of a ring row
    __device__ __forceinline__ static void pair(const char* slot, int i, int col, const StepParams&, float& r,
                                                float& b) {
        r = plane(slot, i)[col];
        b = plane(slot, 9 + i)[col];
    }

    // Store of the post-collision populations of one node.  The minority colour
    // is formed directly and the majority as the rest of f+, so that
    // R++ + B++ = f+ holds to one rounding of the majority.  (sx, sy) is the
    // red segregation vector beta phi rho_R rho_B / rho e of Eq. eq_re_color.
    __device__ __forceinline__ static void store(char* dst, size_t nodes, size_t node, const float (&fp)[9],
                                                 float rr, float rb, float inv_rho, float sx, float sy, float,
                                                 float, const StepParams&) {
        store_recoloured_f32(reinterpret_cast<float*>(dst) + node, nodes, fp, rr, rb, inv_rho, sx, sy);
    }
};

// 16-bit deviations (H = __half2 or __nv_bfloat162).
//
// Record of a node: two float2 planes -- the colour densities (rho_R,
// rho_B) and the rest populations (R_0, B_0) -- then twelve planes of 16-bit
// (red, blue) pairs -- four reference dipoles D_0..D_3, then the deviations
// d_i of the moving links i = 1..8 -- decoded as
//   C_i = rho_C psi_i + (+/-) D_C,dip(i) + d_C,i / 2^k      (i >= 1)
// (dip_index, dip_neg).  psi_i are the reference weights of the axis and
// diagonal links (weights()), of the shape that the lowest bit of D_0's red
// half selects (the record's flag).  The step stores as dipoles (dipoles16) the
// equilibrium's velocity term, with the node's post-collision velocity, and
// the recolour's segregation term (Eq. eq_re_color), so that its deviations
// are only the non-equilibrium and second-order parts of the populations:
// tens of times smaller than their deviations from rho_C psi_i, and so is
// their 16-bit rounding.  The dipoles are reference values, stored rounded
// and used as stored: their rounding only moves a little into the
// deviations.  The rest populations are the remainder of rho_C after the
// decoded moving links, so that a record decodes to populations summing to
// rho_C.  Any pair of population sets is representable.
//
// A ring row keeps, per window column, the densities as copied --
// overwritten by the thread that copied them, as soon as its copy has landed
// (prep), with the axis reference pair (rho_R psi^R_a, rho_B psi^B_a) -- the
// diagonal reference pair (prep), and the rest populations and the twelve
// 16-bit pairs as copied.
template <class H>
struct Layout16 {
    static constexpr int kRefBytes = 2 * kWin * 8;  // float2 per column: (rho_R, rho_B) -> axis pair; diagonal pair
    static constexpr int kRestBytes = kWin * 8;     // float2 per column: (R_0, B_0)
    static constexpr int kPairBytes = kWin * 4;   // one 16-bit pair per column and plane
    static constexpr int kPairOff = kRefBytes + kRestBytes;
    static constexpr int kPairPlanes = 12;        // four dipoles, eight deviations
    static constexpr int kSlotBytes = kPairOff + kPairPlanes * kPairBytes;
    // 16-byte chunks of the pair planes after D_0: each thread copies its own
    // column of D_0, which carries the record's reference flag (prep)
    static constexpr int kPairChunks = (kPairPlanes - 1) * kPairBytes / 16;
    static constexpr int kVecIters = (kPairChunks + kThreads - 1) / kThreads;
    static constexpr bool kPrep = true;
    static constexpr bool kCFront = true;  // stage C on the front warps (see chain_tile)
    static constexpr size_t node_bytes() { return 16 + kPairPlanes * 4; }

    __device__ __forceinline__ static float2 to2(H v);
    __device__ __forceinline__ static H from2(float a, float b);
    __device__ __forceinline__ static H from2x(float2 v) { return from2(v.x, v.y); }

    // Each thread copies the densities, the rest populations and the dipole
    // D_0 of its own window column (8, 8 and 4 bytes) and a share of the
    // other pair planes (16-byte chunks of four columns, or its own column's
    // four bytes per plane when nx is not a multiple of 4).
    template <bool VEC>
    struct Plan {
        static constexpr int kN = VEC ? kVecIters : kPairPlanes;
        unsigned soff[kN];
        size_t goff[kN];  // byte offset of the chunk in row 0 of its plane
        unsigned own_soff;
        size_t own_goff;  // byte offset of the column in row 0 of the densities' plane
        size_t rest_off;  // bytes from the densities' plane to the rest populations'
        int n;
        __device__ __forceinline__ void init(int x0, int nx, size_t nodes) {
            const int gx = wrap(x0 - kHalo + static_cast<int>(threadIdx.x), nx);
            own_soff = threadIdx.x * 8;
            own_goff = static_cast<size_t>(gx) * 8;
            rest_off = nodes * 8;
            n = 0;
            if (VEC) {
                constexpr int kPer = kPairBytes / 16;  // chunks per plane row
#pragma unroll
                for (int m = 0; m < kN; ++m) {
                    const int c = threadIdx.x + m * kThreads;
                    const int p = 1 + c / kPer;
                    const int w4 = (c - (p - 1) * kPer) * 4;
                    soff[m] = static_cast<unsigned>(kPairOff + p * kPairBytes + w4 * 4);
                    goff[m] = nodes * 16 + static_cast<size_t>(p) * nodes * 4 +
                              static_cast<size_t>(wrap(x0 - kHalo + w4, nx)) * 4;
                    if (c < kPairChunks) n = m + 1;
                }
            } else {
#pragma unroll
                for (int p = 0; p < kPairPlanes; ++p) {
                    soff[p] = static_cast<unsigned>(kPairOff + p * kPairBytes + threadIdx.x * 4);
                    goff[p] = nodes * 16 + static_cast<size_t>(p) * nodes * 4 + static_cast<size_t>(gx) * 4;
                }
                n = kN;
            }
        }
        __device__ __forceinline__ void issue(unsigned slot_addr, const char* state, int gy, int nx) const {
            const size_t row_nodes = static_cast<size_t>(gy) * nx;
            const char* own = state + own_goff + row_nodes * 8;
            cp_async8(slot_addr + own_soff, own);
            cp_async8(slot_addr + kRefBytes + own_soff, own + rest_off);
            if (VEC) cp_async4(slot_addr + kPairOff + own_soff / 2, state + 2 * rest_off + own_goff / 2 + row_nodes * 4);
#pragma unroll
            for (int m = 0; m < kN; ++m) {
                if (m < n) {
                    const char* g = state + goff[m] + row_nodes * 4;
                    if (VEC) cp_async16(slot_addr + soff[m], g);
                    else cp_async4(slot_addr + soff[m], g);
                }
            }
        }
    };

    // Reference weights (psi_a, psi_d) of a node's axis and diagonal links, as
    // (red, blue) pairs.  psi_a: precision_reference 0 phi_i of Eq. eq_phi at
    // the node's own mixture, ((1 - alpha_R) rho_R + (1 - alpha_B) rho_B) /
    // (5 rho) rounded to a multiple of 2^-24; otherwise per-colour constants
    // (psi_r, psi_b).  Two shapes, chosen per record by its flag (the lowest
    // bit of D_0's red half): psi_d = psi_a / 4 (flag 0), the equilibrium's
    // shape, whose ghost moment N is the equilibrium one; or (flag 1) the rest
    // state with the same mass and energy and N = 0, which is what the
    // collision leaves where N relaxes to 0 (ghost_N_mode 1): with Dellar's
    // ghost weights g = (1, -2, 4) for the rest, axis and diagonal links,
    // psi_a' = psi_a / 2 + 1/18 and psi_d' = psi_a / 2 - 1/36.  Any choice
    // decodes correctly; a reference far from the populations only makes the
    // deviations, and their 16-bit rounding, larger.
    __device__ __forceinline__ static void weights(float rr, float rb, float inv_rho, bool nfree,
                                                   const StepParams& P, float2& wa, float2& wd) {
        float2 pa;
        if (P.precision_reference == 0) {
            float s5 = fmaf(P.mix_r, rr, P.mix_b * rb) * inv_rho;
            s5 = fminf(fmaxf(s5, 0.0f), 0.25f);
            const float q = __fsub_rn(__fadd_rn(s5, 0.5f), 0.5f);  // a multiple of 2^-24
            pa = make_float2(q, q);
        } else {
            pa = make_float2(P.psi_r[1], P.psi_b[1]);
        }
        // one form for both shapes: pa * s + c, with (s, c) = (1, 0) and (1/4, 0)
        // exact for the equilibrium's
        const float sa = nfree ? 0.5f : 1.0f, ca = nfree ? 1.0f / 18.0f : 0.0f;
        const float sd = nfree ? 0.5f : 0.25f, cd = nfree ? -1.0f / 36.0f : 0.0f;
        wa = __ffma2_rn(pa, make_float2(sa, sa), make_float2(ca, ca));
        wd = __ffma2_rn(pa, make_float2(sd, sd), make_float2(cd, cd));
    }

    // Reference pairs of window column t of a ring row whose copy has landed
    // (the calling thread copied that column's densities and D_0 itself, and
    // only it reads or writes the densities).
    __device__ __forceinline__ static void prep(char* slot, int t, const StepParams& P) {
        float2* ref = reinterpret_cast<float2*>(slot);
        const float2 rho = ref[t];
        const unsigned d0 = reinterpret_cast<const unsigned*>(slot + kPairOff)[t];
        float2 wa, wd;
        weights(rho.x, rho.y, rcp(rho.x + rho.y), (d0 & 1u) != 0, P, wa, wd);
        ref[t] = __fmul2_rn(rho, wa);
        ref[kWin + t] = __fmul2_rn(rho, wd);
    }

    // link class of link i >= 1: axis (even i) or diagonal (odd i)
    __device__ __forceinline__ static constexpr bool diag(int i) { return (i & 1) != 0; }

    __device__ __forceinline__ static void pair(const char* slot, int i, int col, const StepParams& P, float& r,
                                                float& b) {
        if (i == 0) {
            const float2 z = reinterpret_cast<const float2*>(slot + kRefBytes)[col];
            r = z.x;
            b = z.y;
            return;
        }
        const float2 ref = reinterpret_cast<const float2*>(slot)[(diag(i) ? kWin : 0) + col];
        const H* pairs = reinterpret_cast<const H*>(slot + kPairOff);
        const float2 un2 = make_float2(P.dev_unscale, P.dev_unscale);
        const float2 d = to2(pairs[(3 + i) * kWin + col]);
        // reference pair plus the stored deviation times 2^-k (exact), rounded once
        float2 c = __ffma2_rn(d, un2, ref);
        const float2 D = to2(pairs[dip_index(i) * kWin + col]);
        c = dip_neg(i) ? __ffma2_rn(D, make_float2(-1.0f, -1.0f), c) : __fadd2_rn(c, D);
        r = c.x;
        b = c.y;
    }

    // (ux, uy): the node's post-collision velocity, for the dipoles.
    __device__ __forceinline__ static void store(char* dst, size_t nodes, size_t node, const float (&fp)[9],
                                                 float rr, float rb, float inv_rho, float sx, float sy, float ux,
                                                 float uy, const StepParams& P) {
        // The recoloured pair of link i is (rho_C / rho) f+_i +/- s_i (Eq.
        // eq_re_color); the record keeps it minus the dipole and the reference,
        // scaled by 2^k (dev_scale) before rounding to 16 bits (a power-of-two
        // factor commutes exactly with FP32 rounding).
        const float S = P.dev_scale;
        H* pairs = reinterpret_cast<H*>(dst + nodes * 16) + node;
        float2 D[4];
        dipoles16(rr, rb, ux, uy, sx, sy, D);
        // the reference flag: N-free shape where the collision relaxes N to 0
        const bool nfree = P.ghost_N_mode == 1;
        float2 Dq[4];  // as stored, and as the decoder will use them
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            H h = from2x(D[j]);
            if (j == 0) {
                // the flag replaces the lowest bit of D_0's red half: a reference
                // value, so the change moves into the deviations exactly
                unsigned u = *reinterpret_cast<const unsigned*>(&h);
                u = (u & ~1u) | (nfree ? 1u : 0u);
                h = *reinterpret_cast<const H*>(&u);
            }
            pairs[j * nodes] = h;
            Dq[j] = to2(h);
        }
        float seg[9];
        segregation(sx * S, sy * S, seg);
        const float2 rho2 = make_float2(rr, rb);
        float2 wa, wd;
        weights(rr, rb, inv_rho, nfree, P, wa, wd);
        const float2 refa = __fmul2_rn(rho2, wa);  // the decoder's reference pairs
        const float2 refd = __fmul2_rn(rho2, wd);
        const float2 a2 = make_float2(rr * inv_rho * S, rb * inv_rho * S), mrho = make_float2(-rr * S, -rb * S);
        const float2 mS = make_float2(-S, -S), pS = make_float2(S, S), m1 = make_float2(-1.0f, -1.0f);
        const float2 un2 = make_float2(P.dev_unscale, P.dev_unscale);
        // The rest populations are what is left of rho_R and rho_B after the
        // moving links as the decoder will see them (pair(), bit for bit), so
        // that every record decodes to exactly its colour densities: colour mass
        // is conserved through the storage to the rounding of that sum.
        float2 sum = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            float2 C = __ffma2_rn(a2, make_float2(fp[i], fp[i]), make_float2(seg[i], -seg[i]));
            const float2 Dj = Dq[dip_index(i)];
            C = __ffma2_rn(Dj, dip_neg(i) ? pS : mS, C);
            const H h = from2x(__ffma2_rn(mrho, diag(i) ? wd : wa, C));
            pairs[(3 + i) * nodes] = h;
            const float2 d = to2(h);
            float2 c = __ffma2_rn(d, un2, diag(i) ? refd : refa);
            c = dip_neg(i) ? __ffma2_rn(Dj, m1, c) : __fadd2_rn(c, Dj);
            sum = __fadd2_rn(sum, c);
        }
        float2* own = reinterpret_cast<float2*>(dst) + node;
        own[0] = rho2;
        own[nodes] = __ffma2_rn(sum, m1, rho2);
    }
};

template <>
__device__ __forceinline__ float2 Layout16<__half2>::to2(__half2 v) { return __half22float2(v); }
template <>
__device__ __forceinline__ __half2 Layout16<__half2>::from2(float a, float b) { return __floats2half2_rn(a, b); }
template <>
__device__ __forceinline__ float2 Layout16<__nv_bfloat162>::to2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <>
__device__ __forceinline__ __nv_bfloat162 Layout16<__nv_bfloat162>::from2(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}

using LayoutF16 = Layout16<__half2>;
using LayoutB16 = Layout16<__nv_bfloat162>;

// ---------------------------------------------------------------------------
// Shared-memory rings of one CTA.
// ---------------------------------------------------------------------------
template <class L>
struct Geometry {
    static constexpr int kPopBytes = kRing * L::kSlotBytes;
    // ring A: Phi' over 8 rows (ring Q; D's stencil reads it) and chi_R, rho,
    // j_x, j_y, chi_B over 4 rows (B and C read them; D recomputes rho^N)
    static constexpr int kQFloats = 8 * kWin;
    static constexpr int kAFloats = 5 * 4 * kWin;
    static constexpr int kBytes = kPopBytes + 4 * (kQFloats + kAFloats + kBFloats + kCFloats);
};

// two warp-specialised CTAs per SM (228 KB of shared memory, 1 KB reserved per CTA, 16 B of static
// shared memory in the batched kernel)
static_assert(2 * (Geometry<LayoutF32>::kBytes + 1024 + 16) <= 228 * 1024, "two FP32 step CTAs per SM");

template <class L, bool W>
struct Rings {
    char* pop;
    float* q;
    float* a;
    float* b;
    float* c;
    // population ring slot k (rows map to slots in order of arrival)
    __device__ __forceinline__ const char* slot(int k) const { return pop + k * L::kSlotBytes; }
    // ring A fields: the colour fractions chi_R = a / (a + b) and chi_B = b / (a + b)
    // (a = rho_R / rho0_r, b = rho_B / rho0_b; rho^N = chi_R - chi_B, Eq. equ_rhoN_def)
    __device__ __forceinline__ float* chiR(int row) const { return a + ((row & 3) * 5 + 0) * kWin; }
    __device__ __forceinline__ float* chiB(int row) const { return a + ((row & 3) * 5 + 4) * kWin; }
    __device__ __forceinline__ float* phip(int row) const { return q + (row & 7) * kWin; }
    __device__ __forceinline__ float* rho(int row) const { return a + ((row & 3) * 5 + 1) * kWin; }
    __device__ __forceinline__ float* jx(int row) const { return a + ((row & 3) * 5 + 2) * kWin; }
    __device__ __forceinline__ float* jy(int row) const { return a + ((row & 3) * 5 + 3) * kWin; }
    __device__ __forceinline__ float* grad(int row, int f) const { return b + ((row & 3) * 2 + f) * kWin; }
    __device__ __forceinline__ float* nh(int row, int f) const { return b + (8 + (row & 3) * 2 + f) * kWin; }
    __device__ __forceinline__ float* G(int row, int f) const { return c + ((row & 3) * 2 + f) * kWin; }
    __device__ __forceinline__ float* u(int row, int f) const { return c + (8 + (row & 3) * 2 + f) * kWin; }
};

// The rings carved out of a CTA's dynamic shared memory.
template <class L, bool W>
__device__ __forceinline__ Rings<L, W> make_rings(char* smem, int ny) {
    using G = Geometry<L>;
    Rings<L, W> R;
    R.pop = smem;
    R.q = reinterpret_cast<float*>(smem + G::kPopBytes);
    R.a = R.q + G::kQFloats;
    R.b = R.a + G::kAFloats;
    R.c = R.b + kBFloats;
    return R;
}

// Pre-collision populations at (row y, window column t): pull from the
// post-collision ring, f_i(r) = P_i(r - c_i) (Eq. equ_evolution), with
// half-way bounce-back P_opp(i)(r) where r - c_i lies beyond a wall.
// With PRE the rows hold pre-collision populations f(t) already in place
// (the public FP32 layout), so the node's own column is read unshifted.
// The ring slots of rows y - 1, y and y + 1 are passed in.
template <class L, bool WALLS, bool PRE>
__device__ __forceinline__ void gather(const char* below, const char* mid, const char* above, int y, int t, int ny,
                                       const StepParams& P, float (&fr)[9], float (&fb)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sy = y - lcy(i);
        if (PRE) {
            L::pair(mid, i, t, P, fr[i], fb[i]);
        } else if (WALLS && (sy < 0 || sy >= ny)) {
            L::pair(mid, lopp(i), t, P, fr[i], fb[i]);
        } else {
            L::pair(lcy(i) > 0 ? below : (lcy(i) < 0 ? above : mid), i, t - lcx(i), P, fr[i], fb[i]);
        }
    }
}

// slot of the row d rows before the row in slot k of a kRing-slot ring (0 <= d < kRing)
__device__ __forceinline__ int ring_back(int k, int d) { return k >= d ? k - d : k - d + kRing; }
__device__ __forceinline__ int ring_next(int k) { return k == kRing - 1 ? 0 : k + 1; }

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

template <class L>
constexpr int min_ctas_per_sm() {
    return Geometry<L>::kBytes + 1024 <= 228 * 1024 / 3 ? 3 : 2;
}
// CTA size of a pass: the step is warp-specialised (front + back)
constexpr int pass_threads(Pass m) { return m == Pass::Step || m == Pass::StepFields ? kStepThreads : kThreads; }
// resident CTAs per SM a pass is compiled for: the warp-specialised step
// keeps two CTAs (16 warps) per SM in every storage form
template <class L>
constexpr int pass_ctas_per_sm(Pass m) {
    return m == Pass::Step || m == Pass::StepFields ? 2 : min_ctas_per_sm<L>();
}

// Diagnostics accumulators of one thread (Pass::Diag).
struct DiagAcc {
    double r = 0.0, b = 0.0, jx = 0.0, jy = 0.0, u2 = 0.0, bad = 0.0;
};

// One tile: the strip [x0, x0 + 120) of rows [y0, y0 + rows) of a lattice,
// with its whole four-stage row pipeline.  Leaves no copy in flight.
//
// Row iteration k (s = y0 - 4 + k) runs stage A at row s - 1, B at s - 2, C
// at s - 3 and D at s - 4; the copy of row s + 2 is issued at its start, into
// the ring slot of row s - 7.  The fields and diagnostics passes run all four
// stages in every thread of a 128-thread CTA, one barrier between stages.
// The step is warp-specialised (2 x 128 threads): the front threads wait for
// the copies, issue the next one and run A and B of iteration k, then
// publish them with bar.arrive; the back threads run C and D of iteration k
// (a back-only barrier between them) while the front is at iteration k + 1.
// With 16-bit storage C runs on the front instead: there the back, with its
// decode and encode, sets the pace, and the move makes the step 2.6 %
// faster; FP32 (Step and StepFields) keeps C on the back, which StepFields,
// whose front also stores A's and B's forward fields, needs (5.6 % slower
// otherwise) and the FP32 step does not mind.
// D reads population rows s - 5 .. s - 3 (nine rows in flight in all: D's
// three, A's three, two copies and the row D of iteration k - 1 read), u
// rows s - 5 .. s - 3, G and n-hat of row s - 4; C on the back also reads
// n-hat rows s - 4 .. s - 2, grad rho^N and ring A of row s - 3.  Before
// leaving iteration k the front waits for the back's iteration k - 1, so
// that in iteration k + 1 nothing it writes -- ring A row s, grad rho^N and
// n-hat rows s - 1, with C on the front G and u row s - 2, the copy into the
// slot of row s - 6 -- is still being read; the mirrored wall rows ny of
// n-hat and u take the slots of row ny - 4, written at least one row
// iteration after the last stage that reads row ny - 4 has run.
template <class L, bool VEC, bool WALLS, Pass MODE, bool PRE>
__device__ __forceinline__ void chain_tile(const Rings<L, WALLS>& R, const unsigned pop_addr, const char* __restrict__ src,
                                           char* __restrict__ dst, const StepParams& P, const int x0, const int y0,
                                           const int rows, const FieldOut& fo, unsigned* __restrict__ flag,
                                           DiagAcc& acc) {
    constexpr bool kStep = MODE == Pass::Step || MODE == Pass::StepFields;
    constexpr bool kWS = kStep;
    constexpr bool kCFront = L::kCFront;
    const bool front = !kWS || threadIdx.x < kThreads;  // warp-uniform
    const int t = front ? static_cast<int>(threadIdx.x) : static_cast<int>(threadIdx.x) - kThreads;
    const int nx = P.nx, ny = P.ny;
    const size_t nodes = static_cast<size_t>(nx) * ny;
    const int y_end = min(y0 + rows, ny);
    const int s_first = y0 - 4;
    const int s_last = y_end + 3;
    const int iters = (y_end - y0) + 8;
    auto row_ok = [&](int r) { return !WALLS || (r >= 0 && r < ny); };
    // Pass::StepFields: the forward fields of the nodes this tile owns go to fo.fwd
    const int gx_own = x0 + t - kHalo;
    const bool own_col = t >= kHalo && t < kWin - kHalo && gx_own < nx;
    auto owned = [&](int r) { return MODE == Pass::StepFields && own_col && r >= y0 && r < y_end; };
    auto fwd = [&](int plane, int r) -> float& {
        return fo.fwd[static_cast<size_t>(plane) * nodes + static_cast<size_t>(r) * nx + gx_own];
    };

    typename L::template Plan<VEC> plan;
    plan.init(x0, nx, nodes);
    // population rows go to ring slots in order: row s_first + j to slot j mod kRing
    auto issue_row = [&](int row, int slot) {
        int gy = row;  // periodic image of the row (the modulo only near the lattice's ends)
        if (gy < 0 || gy >= ny) gy = wrap(gy, ny);
        plan.issue(pop_addr + static_cast<unsigned>(slot * L::kSlotBytes), src, gy, nx);
    };

    // ---------------- stage A: moments at row ya = s - 1 (tile + 3 halo); ks = slot of row s
    auto stage_a = [&](const int s, const int ks) {
        const int ya = s - 1;
        if (ya >= y0 - 3 && ya <= y_end + 2 && row_ok(ya) && t >= 1 && t < kWin - 1) {
            float fr[9], fb[9];
            gather<L, WALLS, PRE>(R.slot(ring_back(ks, 2)), R.slot(ring_back(ks, 1)), R.slot(ks), ya, t, ny, P, fr,
                                  fb);
            const float2 rrb = sum9x2(fr, fb);
            const float rr = rrb.x, rb = rrb.y;
            // colour-blind momentum sum_i f_i c_i (Eq. equ_u_def)
            const float jx = ((fr[1] + fb[1]) + (fr[7] + fb[7])) + (fr[8] + fb[8]) -
                             (((fr[3] + fb[3]) + (fr[5] + fb[5])) + (fr[4] + fb[4]));
            const float jy = ((fr[1] + fb[1]) + (fr[3] + fb[3])) + (fr[2] + fb[2]) -
                             (((fr[5] + fb[5]) + (fr[7] + fb[7])) + (fr[6] + fb[6]));
            const float a = rr * P.inv_rho0_r;
            const float b = rb * P.inv_rho0_b;
            // colour fractions: rho^N = 2 chi_R - 1 = 1 - 2 chi_B (Eq. equ_rhoN_def);
            // the smaller of the two keeps the digits that rho^N, stored in FP32
            // next to -1 or +1, would lose
            const float inv_ab = rcp(__fadd_rn(a, b));  // not contracted: the adjoint recomputes it
            const float chr = a * inv_ab;
            const float chb = b * inv_ab;
            const float phip = fmaf(P.phip_r, rr, P.phip_b * rb);  // App. A, Phi'
            R.chiR(ya)[t] = chr;
            R.chiB(ya)[t] = chb;
            R.phip(ya)[t] = phip;
            R.rho(ya)[t] = rr + rb;
            R.jx(ya)[t] = jx;
            R.jy(ya)[t] = jy;
            if (owned(ya)) {
                fwd(kFwdRR, ya) = rr;
                fwd(kFwdRB, ya) = rb;
                fwd(kFwdCHR, ya) = chr;
                fwd(kFwdCHB, ya) = chb;
                fwd(kFwdPHIP, ya) = phip;
            }
            if (WALLS && ya == 0) {  // even mirror beyond y = -1/2
                R.chiR(-1)[t] = chr;
                R.chiB(-1)[t] = chb;
                R.phip(-1)[t] = phip;
            }
            if (WALLS && ya == ny - 1) {  // even mirror beyond y = ny - 1/2
                R.chiR(ny)[t] = chr;
                R.chiB(ny)[t] = chb;
                R.phip(ny)[t] = phip;
            }
        }
    };
    // ---------------- stage B: grad rho^N, n-hat at row yb = s - 2 (tile + 2)
    auto stage_b = [&](const int s) {
        const int yb = s - 2;
        if (yb >= y0 - 2 && yb <= y_end + 1 && row_ok(yb) && t >= 2 && t < kWin - 2) {
            // grad rho^N = 2 grad chi_R = -2 grad chi_B (the stencil weights sum
            // to zero), taken on the node's minority fraction, whose FP32 spacing
            // is relative: the gradient stays accurate where it is small
            const bool use_b = R.chiR(yb)[t] > 0.5f;
            const int foff = use_b ? 4 * kWin : 0;
            auto ch_row = [&](int r) { return R.chiR(r) + foff; };
            const float two = use_b ? -2.0f : 2.0f;
            const float gx = two * ddx_at(ch_row, yb, t);
            const float gy = two * ddy_at(ch_row, yb, t);
            // n-hat = -grad rho^N / |grad rho^N| (Sec. 2); no direction below kNormalTau
            const float mag2 = fmaf(gx, gx, gy * gy);
            const float inv = (mag2 >= kNormalTau * kNormalTau) ? rsqrtf(mag2) : 0.0f;
            const float nhx = -gx * inv;
            const float nhy = -gy * inv;
            R.grad(yb, 0)[t] = gx;
            R.grad(yb, 1)[t] = gy;
            R.nh(yb, 0)[t] = nhx;
            R.nh(yb, 1)[t] = nhy;
            if (owned(yb)) {
                fwd(kFwdGX, yb) = gx;
                fwd(kFwdGY, yb) = gy;
            }
            if (WALLS && yb == 0) {  // reflected normal beyond the wall
                R.nh(-1, 0)[t] = nhx;
                R.nh(-1, 1)[t] = -nhy;
            }
        }
        if (WALLS && yb == ny && t >= 2 && t < kWin - 2) {
            // reflected normal beyond the top wall, from row ny - 1 (written by
            // this thread one iteration ago) into the slot of row ny - 4
            R.nh(ny, 0)[t] = R.nh(ny - 1, 0)[t];
            R.nh(ny, 1)[t] = -R.nh(ny - 1, 1)[t];
        }
    };
    // ---------------- stage C: curvature, force, velocity at row yc = s - 3 (tile + 1)
    auto stage_c = [&](const int s) {
        const int yc = s - 3;
        if (yc >= y0 - 1 && yc <= y_end && row_ok(yc) && t >= 3 && t < kWin - 3) {
            float K;
            if (P.curvature_mode == 0) {
                // K = div n-hat (Sec. 2)
                K = ddx_at([&](int r) { return R.nh(r, 0); }, yc, t) + ddy_at([&](int r) { return R.nh(r, 1); }, yc, t);
            } else {
                K = P.fixed_K;
            }
            const float gx = R.grad(yc, 0)[t];
            const float gy = R.grad(yc, 1)[t];
            const float rho = R.rho(yc)[t];
            // G = sigma K grad rho^N / 2 + rho g_acc + g_vol (Eq. equ_stforce plus body force)
            const float hk = P.half_sigma * K;
            const float Gx = fmaf(hk, gx, fmaf(rho, P.gacc_x, P.gvol_x));
            const float Gy = fmaf(hk, gy, fmaf(rho, P.gacc_y, P.gvol_y));
            const float inv_rho = rcp(rho);
            // force-adjusted velocity (Eq. equ_u_def)
            const float ux = fmaf(0.5f, Gx, R.jx(yc)[t]) * inv_rho;
            const float uy = fmaf(0.5f, Gy, R.jy(yc)[t]) * inv_rho;
            R.G(yc, 0)[t] = Gx;
            R.G(yc, 1)[t] = Gy;
            R.u(yc, 0)[t] = ux;
            R.u(yc, 1)[t] = uy;
            if (owned(yc)) {
                fwd(kFwdK, yc) = K;
                fwd(kFwdGFX, yc) = Gx;
                fwd(kFwdGFY, yc) = Gy;
                fwd(kFwdUX, yc) = ux;
                fwd(kFwdUY, yc) = uy;
            }
            if (WALLS && yc == 0) {  // no-slip: odd mirror of u
                R.u(-1, 0)[t] = -ux;
                R.u(-1, 1)[t] = -uy;
            }
        }
        if (WALLS && yc == ny && t >= 3 && t < kWin - 3) {
            // odd mirror of u beyond the top wall, from row ny - 1 (this thread,
            // one iteration ago) into the slot of row ny - 4
            R.u(ny, 0)[t] = -R.u(ny - 1, 0)[t];
            R.u(ny, 1)[t] = -R.u(ny - 1, 1)[t];
        }
    };
    // ---------------- stage D: collide, recolour, store at row yd = s - 4 (tile); ks = slot of row s
    auto stage_d = [&](const int s, const int ks) {
        const int yd = s - 4;
        const int gxo = x0 + t - kHalo;
        if (yd >= y0 && yd < y_end && t >= kHalo && t < kWin - kHalo && gxo < nx) {
            float fr[9], fb[9], f[9];
            gather<L, WALLS, PRE>(R.slot(ring_back(ks, 5)), R.slot(ring_back(ks, 4)), R.slot(ring_back(ks, 3)), yd,
                                  t, ny, P, fr, fb);
            const float2 rrb = sum9x2(fr, fb);
            const float rr = rrb.x, rb = rrb.y;
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = fr[i] + fb[i];
            const float rho = rr + rb;
            const float ux = R.u(yd, 0)[t];
            const float uy = R.u(yd, 1)[t];
            if (kStep) {
                if (!isfinite(rho)) atomicOr(flag, 1u);
                const float Gx = R.G(yd, 0)[t];
                const float Gy = R.G(yd, 1)[t];
                auto phip_row = [&](int r) { return R.phip(r); };
                const float dPx = ddx_at(phip_row, yd, t);
                const float dPy = ddy_at(phip_row, yd, t);
                const float divu = ddx_at([&](int r) { return R.u(r, 0); }, yd, t) +
                                   ddy_at([&](int r) { return R.u(r, 1); }, yd, t);
                const float inv_rho = rcp(rho);
                // local shear eigenvalue (Sec. 2: nu(rho^N) = (2/lambda_3 - 1)/6)
                float nu;
                if (P.visc_mode == 0) {
                    // rho^N of this node (Eq. equ_rhoN_def): ring A's four rows no longer hold row yd
                    const float ra = rr * P.inv_rho0_r, ba = rb * P.inv_rho0_b;
                    const float rn = (ra - ba) * rcp(ra + ba);
                    nu = fmaf(0.5f * (P.nu_r - P.nu_b), rn, 0.5f * (P.nu_r + P.nu_b));
                } else {
                    nu = P.eta * inv_rho;
                }
                float fp[9];
                collide_increment(f, rr, rb, rho, nu, ux, uy, Gx, Gy, dPx, dPy, divu, P, fp);
                // recolour (Eq. eq_re_color): red moves along e = grad rho^N / |grad rho^N| = -n-hat,
                // by beta phi_i rho_R rho_B / rho (e . c-hat_i); phi_i = w_i phim for i != 0
                const float ex = -R.nh(yd, 0)[t];
                const float ey = -R.nh(yd, 1)[t];
                const float phim = fmaf(P.kphi_r, rr, P.kphi_b * rb) * inv_rho;
                const float sg = P.beta * (rr * rb) * inv_rho * phim;
                // post-collision velocity u + G / (2 rho) (the 16-bit record's dipoles)
                L::store(dst, nodes, static_cast<size_t>(yd) * nx + gxo, fp, rr, rb, inv_rho, sg * ex, sg * ey,
                         fmaf(0.5f * Gx, inv_rho, ux), fmaf(0.5f * Gy, inv_rho, uy), P);
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
                    acc.r += rr;
                    acc.b += rb;
                    acc.jx += jx;
                    acc.jy += jy;
                    acc.u2 = fmax(acc.u2, static_cast<double>(ux) * ux + static_cast<double>(uy) * uy);
                } else {
                    acc.bad += 1.0;
                }
            }
        }
    };

    // the first two rows, into slots 0 and 1
    auto issue_first = [&]() {
        if (row_ok(s_first)) issue_row(s_first, 0);
        cp_commit();
        if (row_ok(s_first + 1)) issue_row(s_first + 1, 1);
        cp_commit();
    };
    if (!kWS) {
        issue_first();
        int ks = 0;  // slot of row s
        for (int k = 0; k < iters; ++k, ks = ring_next(ks)) {
            const int s = s_first + k;
            cp_wait<1>();
            if (L::kPrep && s <= s_last && row_ok(s)) L::prep(R.pop + ks * L::kSlotBytes, t, P);
            __syncthreads();
            if (s + 2 <= s_last && row_ok(s + 2)) issue_row(s + 2, ring_next(ring_next(ks)));
            cp_commit();
            stage_a(s, ks);
            __syncthreads();
            stage_b(s);
            __syncthreads();
            stage_c(s);
            __syncthreads();
            stage_d(s, ks);
        }
        cp_wait<0>();
    } else if (front) {
        issue_first();
        int ks = 0;
        for (int k = 0; k < iters; ++k, ks = ring_next(ks)) {
            const int s = s_first + k;
            cp_wait<1>();
            // row s has landed: this thread's column of it gets its reference pairs
            if (L::kPrep && s <= s_last && row_ok(s)) L::prep(R.pop + ks * L::kSlotBytes, t, P);
            bar_sync<kBarFront, kThreads>();
            // row s + 2 goes to the slot of row s - 7, last read by D of iteration k - 2
            if (s + 2 <= s_last && row_ok(s + 2)) issue_row(s + 2, ring_next(ring_next(ks)));
            cp_commit();
            stage_a(s, ks);
            bar_sync<kBarFront, kThreads>();
            stage_b(s);
            if (kCFront) {
                bar_sync<kBarFront, kThreads>();
                stage_c(s);
            }
            // publish the front's stages of iteration k, then wait until the back
            // is done with iteration k - 1, whose rows iteration k + 1 overwrites
            if (k & 1) {
                bar_arrive<kBarC + 1, kStepThreads>();
                bar_sync<kBarD + 1, kStepThreads>();
            } else {
                bar_arrive<kBarC, kStepThreads>();
                bar_sync<kBarD, kStepThreads>();
            }
        }
        cp_wait<0>();
    } else {
        bar_arrive<kBarD, kStepThreads>();  // no D before iteration 0
        int ks = 0;
        for (int k = 0; k < iters; ++k, ks = ring_next(ks)) {
            if (k & 1) bar_sync<kBarC + 1, kStepThreads>();
            else bar_sync<kBarC, kStepThreads>();
            if (!kCFront) {
                stage_c(s_first + k);
                bar_sync<kBarBack, kThreads>();  // u of row s - 3 is in shared memory
            }
            stage_d(s_first + k, ks);
            if (k + 1 < iters) {
                if (k & 1) bar_arrive<kBarD, kStepThreads>();  // D of iteration k + 1 (even) may follow
                else bar_arrive<kBarD + 1, kStepThreads>();
            }
        }
    }
}

// A tile of rows [y0, y0 + rows) touches population rows y0 - 4 .. y0 + rows + 3
// and runs its stages on rows y0 - 3 .. y0 + rows + 2.  When all of these lie
// inside [1, ny - 2] no wall condition can apply (no bounce-back link, no
// mirrored row is written or read), and the periodic form of the pipeline
// computes exactly the same values with fewer instructions.
__device__ __forceinline__ bool away_from_walls(int y0, int rows, int ny) { return y0 >= 5 && y0 + rows + 5 <= ny; }

template <class L, bool VEC, bool WALLS, Pass MODE, bool PRE>
__global__ void __launch_bounds__(pass_threads(MODE), pass_ctas_per_sm<L>(MODE))
    k_chain(const char* __restrict__ src, char* __restrict__ dst, const StepParams P, const int rows, FieldOut fo,
            unsigned* __restrict__ flag, double* __restrict__ partials) {
    pdl_begin();
    extern __shared__ __align__(16) char smem[];
    const unsigned pop_addr = static_cast<unsigned>(__cvta_generic_to_shared(smem));

    DiagAcc acc;
    const int x0 = static_cast<int>(blockIdx.x) * kTileX, y0 = static_cast<int>(blockIdx.y) * rows;
    if (WALLS && away_from_walls(y0, rows, P.ny))
        chain_tile<L, VEC, false, MODE, PRE>(make_rings<L, false>(smem, P.ny), pop_addr, src, dst, P, x0, y0, rows, fo,
                                             flag, acc);
    else
        chain_tile<L, VEC, WALLS, MODE, PRE>(make_rings<L, WALLS>(smem, P.ny), pop_addr, src, dst, P, x0, y0, rows, fo,
                                             flag, acc);
    const int t = threadIdx.x;

    if (MODE == Pass::Diag) {
        // warp shuffle reduction, then across the CTA's warps in shared memory
        double v[kDiagSlots] = {acc.r, acc.b, acc.jx, acc.jy, acc.u2, acc.bad};
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

// Batched ensemble: a persistent kernel over a work list of tiles of many
// independent lattices.  Each CTA takes the next item (member, strip, row
// segment) from a global counter until the list is exhausted; every item is
// the same four-stage row pipeline as k_chain, run with that member's own
// parameters and buffers.  No CTA waits on another: an atomicAdd hands out
// the items, and the last CTA to leave resets the counters for the next
// launch.
template <class L, bool VEC>
__global__ void __launch_bounds__(kStepThreads, pass_ctas_per_sm<L>(Pass::Step)) k_batch(const BatchArgs A) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_item;
    const unsigned pop_addr = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    for (;;) {
        __syncthreads();  // the previous item is done with the rings and s_item
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(&A.counters[0], 1u));
        __syncthreads();
        const int it = s_item;
        if (it >= A.nitems) break;
        const BatchItem w = A.items[it];
        const StepParams P = A.params[w.member];  // a register copy: stores cannot alias it
        const size_t off = A.offsets[w.member];
        DiagAcc acc;
        if (P.wall_y && !away_from_walls(w.y0, w.rows, P.ny))
            chain_tile<L, VEC, true, Pass::Step, false>(make_rings<L, true>(smem, P.ny), pop_addr, A.src + off, A.dst + off, P, w.x0, w.y0, w.rows,
                                                        FieldOut{}, A.flags + w.member, acc);
        else
            chain_tile<L, VEC, false, Pass::Step, false>(make_rings<L, false>(smem, P.ny), pop_addr, A.src + off, A.dst + off, P, w.x0, w.y0,
                                                         w.rows, FieldOut{}, A.flags + w.member, acc);
    }
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's last counter access precedes its exit count
        const unsigned done = atomicAdd(&A.counters[1], 1u);
        if (done == gridDim.x - 1) {
            A.counters[0] = 0u;
            A.counters[1] = 0u;
            __threadfence();
        }
    }
}

template <class L, bool VEC>
cudaError_t batch_configure(int dev, int* ctas_per_sm) {
    static std::atomic<unsigned long long> configured{0};  // per device, set from any host thread
    const unsigned long long bit = 1ull << (dev & 63);
    cudaError_t e = cudaSuccess;
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k_batch<L, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, Geometry<L>::kBytes);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    if (ctas_per_sm)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_batch<L, VEC>, kStepThreads,
                                                          Geometry<L>::kBytes);
    return e;
}

template <class L, bool VEC>
cudaError_t batch_launch(const BatchArgs& A, int grid, cudaStream_t s) {
    k_batch<L, VEC><<<grid, kStepThreads, Geometry<L>::kBytes, s>>>(A);
    return cudaGetLastError();
}

__global__ void k_diag_reduce(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    pdl_begin();
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

template <class L, bool VEC, bool WALLS, Pass MODE, bool PRE>
cudaError_t launch_one(const void* src, void* dst, const StepParams& P, int rows, FieldOut fo, unsigned* flag,
                       double* partials, cudaStream_t s) {
    // the shared-memory opt-in is per kernel and per device: set it once for each
    static std::atomic<unsigned long long> configured{0};  // per device, set from any host thread
    const int smem = Geometry<L>::kBytes;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k_chain<L, VEC, WALLS, MODE, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    return launch_pdl(k_chain<L, VEC, WALLS, MODE, PRE>, chain_grid(P.nx, P.ny, rows), dim3(pass_threads(MODE)), smem,
                      s, static_cast<const char*>(src), static_cast<char*>(dst), P, rows, fo, flag, partials);
}

template <class L, Pass MODE, bool PRE = false>
cudaError_t launch_layout(const void* src, void* dst, const StepParams& P, int rows, FieldOut fo, unsigned* flag,
                          double* partials, cudaStream_t s) {
    const bool vec = (P.nx % 4) == 0;
    const bool walls = P.wall_y != 0;
    if (vec && walls) return launch_one<L, true, true, MODE, PRE>(src, dst, P, rows, fo, flag, partials, s);
    if (vec) return launch_one<L, true, false, MODE, PRE>(src, dst, P, rows, fo, flag, partials, s);
    if (walls) return launch_one<L, false, true, MODE, PRE>(src, dst, P, rows, fo, flag, partials, s);
    return launch_one<L, false, false, MODE, PRE>(src, dst, P, rows, fo, flag, partials, s);
}

template <Pass MODE>
cudaError_t launch_chain(const void* src, void* dst, const StepParams& P, int rows, FieldOut fo, unsigned* flag,
                         double* partials, cudaStream_t s) {
    switch (P.precision) {
        case kPrecF16: return launch_layout<LayoutF16, MODE>(src, dst, P, rows, fo, flag, partials, s);
        case kPrecB16: return launch_layout<LayoutB16, MODE>(src, dst, P, rows, fo, flag, partials, s);
        default: return launch_layout<LayoutF32, MODE>(src, dst, P, rows, fo, flag, partials, s);
    }
}

}  // namespace

size_t state_node_bytes(int precision) {
    return precision == kPrecF32 ? LayoutF32::node_bytes() : LayoutF16::node_bytes();
}

dim3 chain_grid(int nx, int ny, int rows) {
    return dim3(static_cast<unsigned>((nx + kTileX - 1) / kTileX), static_cast<unsigned>((ny + rows - 1) / rows), 1);
}

int chain_rows(int nx, int ny, int sms, int precision) {
    // Rows per CTA: each CTA spends (rows + 8) row-iterations (8 fill the
    // pipeline), and the CTAs run in waves of (SMs x resident CTAs); pick
    // the segment length that minimises waves x (rows + 8).  Short segments
    // (1, 2, 4 rows) win on lattices too small to fill one wave.
    const int strips = (nx + kTileX - 1) / kTileX;
    const int per_sm = precision == kPrecF32 ? pass_ctas_per_sm<LayoutF32>(Pass::Step)
                                             : pass_ctas_per_sm<LayoutF16>(Pass::Step);
    const long slots = static_cast<long>(per_sm) * (sms > 0 ? sms : 1);
    int best = 8;
    long best_cost = -1;
    for (int rows = 1; rows <= 512; rows = rows < 8 ? 2 * rows : rows + 8) {
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

cudaError_t launch_step(const void* src, void* dst, const StepParams& P, int rows, unsigned* flag, cudaStream_t s) {
    return launch_chain<Pass::Step>(src, dst, P, rows, FieldOut{}, flag, nullptr, s);
}

cudaError_t launch_step_fields(const float* src, float* dst, const StepParams& P, int rows, unsigned* flag,
                               float* fwd, cudaStream_t s) {
    FieldOut fo{};
    fo.fwd = fwd;
    return launch_layout<LayoutF32, Pass::StepFields>(src, dst, P, rows, fo, flag, nullptr, s);
}

cudaError_t launch_fields(const void* src, const StepParams& P, int rows, FieldOut out, cudaStream_t s) {
    return launch_chain<Pass::Fields>(src, nullptr, P, rows, out, nullptr, nullptr, s);
}

cudaError_t launch_diag_partials(const void* src, const StepParams& P, int rows, double* partials, cudaStream_t s) {
    return launch_chain<Pass::Diag>(src, nullptr, P, rows, FieldOut{}, nullptr, partials, s);
}

cudaError_t launch_diag_partials_pre(const float* pre, const StepParams& P, int rows, double* partials,
                                     cudaStream_t s) {
    return launch_layout<LayoutF32, Pass::Diag, true>(pre, nullptr, P, rows, FieldOut{}, nullptr, partials, s);
}

cudaError_t launch_diag_reduce(const double* partials, int nblocks, double* out, cudaStream_t s) {
    return launch_pdl(k_diag_reduce, dim3(1), dim3(kThreads), 0, s, partials, nblocks, out);
}

cudaError_t prepare_batch(int precision, bool vec, int* ctas_per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    switch (precision) {
        case kPrecF16:
            return vec ? batch_configure<LayoutF16, true>(dev, ctas_per_sm)
                       : batch_configure<LayoutF16, false>(dev, ctas_per_sm);
        case kPrecB16:
            return vec ? batch_configure<LayoutB16, true>(dev, ctas_per_sm)
                       : batch_configure<LayoutB16, false>(dev, ctas_per_sm);
        default:
            return vec ? batch_configure<LayoutF32, true>(dev, ctas_per_sm)
                       : batch_configure<LayoutF32, false>(dev, ctas_per_sm);
    }
}

cudaError_t launch_batch(const BatchArgs& A, int precision, bool vec, int grid, cudaStream_t s) {
    switch (precision) {
        case kPrecF16: return vec ? batch_launch<LayoutF16, true>(A, grid, s) : batch_launch<LayoutF16, false>(A, grid, s);
        case kPrecB16: return vec ? batch_launch<LayoutB16, true>(A, grid, s) : batch_launch<LayoutB16, false>(A, grid, s);
        default: return vec ? batch_launch<LayoutF32, true>(A, grid, s) : batch_launch<LayoutF32, false>(A, grid, s);
    }
}

}  // namespace cmrt
