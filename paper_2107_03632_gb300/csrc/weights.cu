// RBF-FD Laplacian weights: one augmented PHS+polynomial system per stencil,
// held in shared memory and solved by one, two or four warps (sm_103a), in
// FP64 (the default) or in double-float arithmetic (opt-in).
//
// Sec. II, Eq. 1: (L u)(x_c) ~ sum_j w_j u(x_j) over the stencil of x_c.
// Sec. V: Phi(r) = r^3 augmented with the monomials of degree <= m, L = lap.
// The weights solve
//     [ Phi  P ] [ w ]   [ 9 |xh_j|        ]   Phi_jk = |xh_j - xh_k|^3
//     [ P^T  0 ] [ l ] = [ lap p_k(0)      ]   P_jk   = p_k(xh_j)
// in coordinates xh = (x - x_c) / delta, delta = max_j |x_j - x_c|
// (lap r^3 = 9 r in 2D); w = wh / delta^2.  Monomials in graded order
// 1, x, y, x^2, xy, y^2, ...; only x^2 and y^2 have lap p(0) = 2.
//
// Design for this chip: FP64 is the scarce pipe, everything else is nearly
// free next to it, so the kernel spends FP64 instructions only on the
// arithmetic that defines the weights:
//  * one warp owns one stencil; its (M x M+1) augmented matrix lives in
//    shared memory, row-major with an odd leading dimension (M = n + s);
//  * Gaussian elimination with partial pivoting (row of the largest |a_ik|,
//    ties to the lower row, as LAPACK's idamax); the pivot search compares
//    |a| as integer bit patterns, not with FP64 compares;
//  * the rank-1 trailing update is flattened over the (rows x cols) block so
//    all 32 lanes issue DFMAs down to the last columns (no idle lanes at the
//    narrow tail of the factorisation);
//  * the stencil coordinates are parked in the s x s zero block while Phi and
//    P are built (when it is large enough), so a warp needs no extra shared
//    memory and four m = 6 stencils (M = 84) fit on one SM.
#include "common.cuh"
#include "df32.cuh"
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace rbffd {
namespace {

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

struct WeightsGeom {
    int n, m, s, M, LD;  // stencil size, degree, monomials, system size, row stride (doubles)
    int coords_in_zero_block;
    int smem_doubles;    // per warp
};

WeightsGeom weights_geom(int n, int m) {
    WeightsGeom g;
    g.n = n;
    g.m = m;
    g.s = (m + 1) * (m + 2) / 2;
    g.M = n + g.s;
    g.LD = g.M + 1;
    if ((g.LD & 1) == 0) g.LD += 1;  // odd stride: column walks spread over banks
    g.coords_in_zero_block = (g.s * g.s >= 2 * n) ? 1 : 0;
    g.smem_doubles = g.M * g.LD + (g.coords_in_zero_block ? 0 : 2 * n);
    return g;
}

// Warp-per-stencil kernel.  Dynamic shared memory: warps_per_block *
// smem_doubles doubles.
//   op 0 (Laplacian): centres cxy = xy, weights of lap at the centre.
//   op 1 (interpolation): centres cxy are other points (N of them; the
//        stencils index the Nd points xy); weights of the value at the
//        centre, right-hand side [ |xh_j|^3 ; p_k(0) ], no rescaling.
__global__ void __launch_bounds__(128) weights_kernel(const double2* __restrict__ xy, const int* __restrict__ idx,
                                                      int N, int n, int m, int s, int M, int LD, int coords_zb,
                                                      int smem_doubles, double* __restrict__ w,
                                                      int* __restrict__ node_status,
                                                      const double2* __restrict__ cxy, int Nd, int op) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double* A = smem + (size_t)wib * smem_doubles;
    // coordinate scratch of 2n doubles past the matrix, when the zero block
    // is too small to hold it
    double* cx = A + (size_t)M * LD;
    // entry i of the warp's region (tested against it in the checked build,
    // whose first test is that the region lies in the launch's shared memory)
    (void)RB_SH(A + (size_t)smem_doubles - 1);
    auto a = [&](size_t i) -> double& { return RB_AT(A, i, smem_doubles); };
    const int total_warps = gridDim.x * wpb;

    for (int node = blockIdx.x * wpb + wib; node < N; node += total_warps) {
        const int* sten = idx + (int64_t)node * n;
        const double2 c = cxy[node];

        // ---- shift, scale --------------------------------------------------
        // Coordinates go to a linear scratch of 2n doubles.  In the zero
        // block, entry t is stored at row n + t / s, column n + t % s.
        auto cs = [&](int t) -> double& {
            if (coords_zb) return a((size_t)(n + t / s) * LD + n + t % s);
            return RB_AT(cx, t, 2 * n);
        };
        unsigned long long dmax = 0;
        int bad_index = 0;
        for (int j = lane; j < n; j += 32) {
            const int sj = sten[j];
            const bool ok = (unsigned)sj < (unsigned)Nd;  // never read outside xy
            bad_index |= ok ? 0 : 1;
            const double2 p = ok ? xy[sj] : c;
            const double dx = __dadd_rn(p.x, -c.x);
            const double dy = __dadd_rn(p.y, -c.y);
            const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            const unsigned long long b = abs_bits(d2);
            dmax = (b > dmax) ? b : dmax;
            cs(2 * j) = dx;
            cs(2 * j + 1) = dy;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, dmax, o);
            dmax = (t > dmax) ? t : dmax;
        }
        const double delta = __dsqrt_rn(__longlong_as_double((long long)dmax));
        const double delta2 = __dmul_rn(delta, delta);
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            cs(2 * j) = __ddiv_rn(cs(2 * j), delta);
            cs(2 * j + 1) = __ddiv_rn(cs(2 * j + 1), delta);
        }
        __syncwarp();

        // ---- Phi block (upper triangle pairs, mirrored) and the RHS ---------
        const int npairs = n * (n - 1) / 2;
        int coincident = 0;  // two stencil nodes at the same point: singular system
        {
            // pair p -> (j, k), j < k, enumerated row by row of the upper triangle
            for (int pidx = lane; pidx < npairs; pidx += 32) {
                // invert p = j*(2n-j-1)/2 + (k-j-1)
                int j = (int)((2.0f * n - 1.0f - sqrtf((2.0f * n - 1.0f) * (2.0f * n - 1.0f) - 8.0f * pidx)) * 0.5f);
                if (j < 0) j = 0;
                while (j > 0 && j * (2 * n - j - 1) / 2 > pidx) --j;
                while ((j + 1) * (2 * n - j - 2) / 2 <= pidx) ++j;
                const int k = pidx - j * (2 * n - j - 1) / 2 + j + 1;
                const double dx = __dadd_rn(cs(2 * j), -cs(2 * k));
                const double dy = __dadd_rn(cs(2 * j + 1), -cs(2 * k + 1));
                const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
                coincident |= (dx == 0.0 && dy == 0.0) ? 1 : 0;
                const double phi = __dmul_rn(__dmul_rn(r, r), r);
                a((size_t)j * LD + k) = phi;
                a((size_t)k * LD + j) = phi;
            }
            for (int j = lane; j < n; j += 32) {
                a((size_t)j * LD + j) = 0.0;
                const double xh = cs(2 * j), yh = cs(2 * j + 1);
                const double rj = __dsqrt_rn(__dadd_rn(__dmul_rn(xh, xh), __dmul_rn(yh, yh)));
                a((size_t)j * LD + M) = op ? __dmul_rn(__dmul_rn(rj, rj), rj) : __dmul_rn(9.0, rj);
                // monomials x^a y^b, graded order; powers by repeated products
                double xp[9], yp[9];
                xp[0] = 1.0;
                yp[0] = 1.0;
#pragma unroll
                for (int q = 1; q < 9; ++q) {
                    xp[q] = (q <= m) ? __dmul_rn(xp[q - 1], xh) : 0.0;
                    yp[q] = (q <= m) ? __dmul_rn(yp[q - 1], yh) : 0.0;
                }
                int col = 0;
                for (int d = 0; d <= m; ++d) {
                    for (int i = 0; i <= d; ++i) {
                        const double v = (d == 0) ? 1.0 : __dmul_rn(xp[d - i], yp[i]);
                        a((size_t)j * LD + n + col) = v;  // P
                        a((size_t)(n + col) * LD + j) = v;  // P^T
                        ++col;
                    }
                }
            }
        }
        __syncwarp();
        // zero block and polynomial RHS (coordinates no longer needed)
        for (int t = lane; t < s * s; t += 32) a((size_t)(n + t / s) * LD + n + t % s) = 0.0;
        {
            int col = 0;
            for (int d = 0; d <= m; ++d)
                for (int i = 0; i <= d; ++i, ++col)
                    if (lane == 0)
                        a((size_t)(n + col) * LD + M) =
                            op ? (d == 0 ? 1.0 : 0.0) : ((d == 2 && (i == 0 || i == 2)) ? 2.0 : 0.0);
        }
        __syncwarp();

        // ---- Gaussian elimination with partial pivoting ---------------------
        int singular = __any_sync(0xffffffffu, bad_index | coincident) ? 1 : 0;
        for (int k = 0; k < M && !singular; ++k) {
            // pivot: largest |a_ik|, i >= k, lowest i on ties
            unsigned long long best = 0;
            int bi = k;
            for (int i = k + lane; i < M; i += 32) {
                const unsigned long long b = abs_bits(a((size_t)i * LD + k));
                if (b > best) {  // ascending i per lane: keeps the first maximum
                    best = b;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (best == 0) {  // exactly zero column: singular
                singular = 1;
                break;
            }
            if (bi != k) {
                for (int j = k + lane; j <= M; j += 32) {
                    const double t = a((size_t)k * LD + j);
                    a((size_t)k * LD + j) = a((size_t)bi * LD + j);
                    a((size_t)bi * LD + j) = t;
                }
            }
            __syncwarp();
            // the pivot's reciprocal replaces the pivot (only the back
            // substitution reads it again, and multiplies by it)
            const double inv = rcp64(a((size_t)k * LD + k));
            for (int i = k + 1 + lane; i < M; i += 32) a((size_t)i * LD + k) = __dmul_rn(a((size_t)i * LD + k), inv);
            __syncwarp();
            if (lane == 0) a((size_t)k * LD + k) = inv;
            // trailing update, flattened over rows i in (k, M), cols j in (k, M]
            const int R = M - k - 1, C = M - k;
            if (R > 0) {
                const int total = R * C;
                int ii = lane / C, jj = lane % C;
                const int si = 32 / C, sj = 32 % C;
                const double* prow = A + (size_t)k * LD + k + 1;
                int e = lane;
                for (; e + 96 < total; e += 128) {
                    int i0 = ii, j0 = jj;
                    int i1 = i0 + si, j1 = j0 + sj;
                    if (j1 >= C) { j1 -= C; ++i1; }
                    int i2 = i1 + si, j2 = j1 + sj;
                    if (j2 >= C) { j2 -= C; ++i2; }
                    int i3 = i2 + si, j3 = j2 + sj;
                    if (j3 >= C) { j3 -= C; ++i3; }
                    ii = i3 + si;
                    jj = j3 + sj;
                    if (jj >= C) { jj -= C; ++ii; }
                    double* r0 = A + (size_t)(k + 1 + i0) * LD + k;
                    double* r1 = A + (size_t)(k + 1 + i1) * LD + k;
                    double* r2 = A + (size_t)(k + 1 + i2) * LD + k;
                    double* r3 = A + (size_t)(k + 1 + i3) * LD + k;
                    const int L = smem_doubles;
                    (void)L;  // the bound of the checked build's tests
                    const double l0 = RB_PT(r0, A, L), l1 = RB_PT(r1, A, L), l2 = RB_PT(r2, A, L),
                                 l3 = RB_PT(r3, A, L);
                    const double u0 = RB_PT(prow + j0, A, L), u1 = RB_PT(prow + j1, A, L),
                                 u2 = RB_PT(prow + j2, A, L), u3 = RB_PT(prow + j3, A, L);
                    const double a0 = RB_PT(r0 + 1 + j0, A, L), a1 = RB_PT(r1 + 1 + j1, A, L),
                                 a2 = RB_PT(r2 + 1 + j2, A, L), a3 = RB_PT(r3 + 1 + j3, A, L);
                    RB_PT(r0 + 1 + j0, A, L) = fma(-l0, u0, a0);
                    RB_PT(r1 + 1 + j1, A, L) = fma(-l1, u1, a1);
                    RB_PT(r2 + 1 + j2, A, L) = fma(-l2, u2, a2);
                    RB_PT(r3 + 1 + j3, A, L) = fma(-l3, u3, a3);
                }
                for (; e < total; e += 32) {
                    double* r0 = A + (size_t)(k + 1 + ii) * LD + k;
                    RB_PT(r0 + 1 + jj, A, smem_doubles) = fma(-RB_PT(r0, A, smem_doubles),
                                                              RB_PT(prow + jj, A, smem_doubles),
                                                              RB_PT(r0 + 1 + jj, A, smem_doubles));
                    ii += si;
                    jj += sj;
                    if (jj >= C) { jj -= C; ++ii; }
                }
            }
            __syncwarp();
        }

        // ---- back substitution on U x = b' (b' in column M) -----------------
        if (!singular) {
            for (int j = M - 1; j >= 0; --j) {
                const double xj = __dmul_rn(a((size_t)j * LD + M), a((size_t)j * LD + j));
                __syncwarp();
                for (int i = lane; i < j; i += 32)
                    a((size_t)i * LD + M) = fma(-a((size_t)i * LD + j), xj, a((size_t)i * LD + M));
                if (lane == 0) a((size_t)j * LD + M) = xj;
                __syncwarp();
            }
        }

        // ---- scale back and store ------------------------------------------
        int bad = singular;
        double* wout = w + (int64_t)node * n;
        for (int j = lane; j < n; j += 32) {
            const double v = singular ? 0.0 : (op ? a((size_t)j * LD + M) : __ddiv_rn(a((size_t)j * LD + M), delta2));
            if (!isfinite(v)) bad = 1;
            a((size_t)j * LD + M) = v;
        }
        bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
        for (int j = lane; j < n; j += 32) wout[j] = bad ? 0.0 : a((size_t)j * LD + M);
        if (node_status && lane == 0) node_status[node] = bad;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Null-space (block) elimination of the same saddle-point system.
//
// With P of full column rank, pick s pivot rows r1 of P by Gauss-Jordan
// elimination with row pivoting (the other q = n - s rows are r2) and let
// X = P[r2] P[r1]^-1 (q x s).  The columns of Z = [-X^T ; I] (rows r1, r2)
// span {z : P^T z = 0}, every solution of P^T w = g is w0 + Z y with
// w0[r1] = P[r1]^-T g, w0[r2] = 0, and the first block row reduces to
//     (Z^T Phi Z) y = Z^T (f - Phi w0).
// r^3 is conditionally positive definite of order 2 and the columns of Z
// annihilate every polynomial of degree <= m (>= 1), so Z^T Phi Z is
// symmetric positive definite: Cholesky, no pivoting.  The weights are
// the same as from the full (n+s) x (n+s) solve in exact arithmetic; the
// FP64 work is ~n s^2 (elimination) + 2 s^2 q + s q^2 (reduced matrix) +
// q^3/3 flops instead of (2/3)(n+s)^3, about half at m = 6, n = 56.
//
// Shared memory per stencil (8-byte slots unless noted), nodes in permuted
// order [r1, r2] once the pivots are known; Phi is held as its three blocks
// (Phi21 = Phi12^T is not stored):
//   A11  s x LDS     Phi11 (both triangles)
//   A12  s x LDQ     Phi12; T = Phi12 - Phi11 X^T overwrites it
//   A22  q(q+1)/2    Phi22, lower triangle packed by rows; S' = Phi22 -
//                    Phi21 X^T, then S = S' - X T = Z^T Phi Z overwrite it
//                    Before Phi is built the same region holds
//   P    (n+1) x LDS monomials, row n holds g; after the elimination rows r2
//                    hold X and row n holds w0[r1] -- copied out to
//   X    q x LDX     X compacted (row j = node r2_j), and w0 (s)
//   crd  2n          scaled coordinates (caller order)
//   fv, uv, wv  n    rhs 9|xh|, f - Phi w0, permuted weights
//   tv   n           reduced rhs / solution (q used)
//   perm, act  n int permutation and the active-row list
// (~26 KB at m = 6, n = 56: eight stencils per SM.)
struct NsGeom {
    int n, m, s, q, LDQ, LDS, LDX;
    int doubles, ints, bytes;
};

// Doubles of the region that holds Phi's blocks, and P before them.
__host__ __device__ inline int ns_phi_region(int n, int s, int LDS, int LDQ) {
    const int q = n - s;
    const int blocks = s * LDS + s * LDQ + q * (q + 1) / 2;
    return blocks > (n + 1) * LDS ? blocks : (n + 1) * LDS;
}

NsGeom ns_geom(int n, int m) {
    NsGeom g;
    g.n = n;
    g.m = m;
    g.s = (m + 1) * (m + 2) / 2;
    g.q = n - g.s;
    g.LDQ = g.q | 1;
    g.LDS = g.s | 1;
    g.LDX = g.s | 1;
    // P must fit in Phi's region while the elimination runs
    const int phi = ns_phi_region(n, g.s, g.LDS, g.LDQ);
    g.doubles = phi + g.q * g.LDX + g.s + 2 * n + 4 * n;
    g.ints = 2 * n;
    g.bytes = (int)align_up((size_t)g.doubles * 8 + (size_t)g.ints * 4, 16);
    return g;
}

// Synchronisation and reductions over the threads of one stencil: half a
// warp (NT = 16, two stencils per warp), a warp (NT = 32) or the whole block
// (NT = 64 or 128, one stencil per block).
template <int NT>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (NT >= 32) return 0xffffffffu;
    else return ((1u << NT) - 1u) << ((threadIdx.x & 31) & ~(NT - 1));
}

// Shuffle offset the in-warp reductions start from.
template <int NT>
constexpr int group_shfl_top() {
    return NT < 32 ? NT / 2 : 16;
}

template <int NT>
__device__ __forceinline__ void group_sync() {
    if (NT < 32) __syncwarp(group_mask<NT>());
    else if (NT == 32) __syncwarp();
    else __syncthreads();
}

template <int NT>
__device__ __forceinline__ int group_any(int p) {
    if (NT <= 32) return __any_sync(group_mask<NT>(), p);
    return __syncthreads_or(p);
}

// Max over the group of a per-warp maximum (already reduced within each warp).
template <int NT>
__device__ __forceinline__ unsigned long long group_max_u64(unsigned long long v, unsigned long long* sh) {
    if (NT <= 32) return v;
    constexpr int W = NT / 32;
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) RB_AT(sh, w, W) = v;
    __syncthreads();
    unsigned long long r = sh[0];
#pragma unroll
    for (int k = 1; k < W; ++k) r = sh[k] > r ? sh[k] : r;
    __syncthreads();
    return r;
}

// Pivot (largest |value|, then lowest row) over the group, from per-warp results.
template <int NT>
__device__ __forceinline__ void group_argmax(unsigned long long& best, int& bi, int& bpos, unsigned long long* shb,
                                             int* shi) {
    if (NT <= 32) return;
    constexpr int W = NT / 32;
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        RB_AT(shb, w, W) = best;
        RB_AT(shi, 2 * w, 2 * W) = bi;
        RB_AT(shi, 2 * w + 1, 2 * W) = bpos;
    }
    __syncthreads();
    best = shb[0];
    bi = shi[0];
    bpos = shi[1];
#pragma unroll
    for (int k = 1; k < W; ++k)
        if (shb[k] > best || (shb[k] == best && shi[2 * k] < bi)) {
            best = shb[k];
            bi = shi[2 * k];
            bpos = shi[2 * k + 1];
        }
    __syncthreads();
}

// Arithmetic of the null-space kernel.  F64: IEEE double throughout.  DF:
// double-float values (df32.cuh, ~48 significant bits) on the FP32 pipe,
// which on this GPU issues 64 lanes per clock per SM against the FP64
// units' 2: the elimination, the reduced matrix and its Cholesky factor run
// there; only the shift/scale of the coordinates and the final division by
// delta^2 stay in FP64.  The rounding unit is ~2^-48 instead of 2^-53; with
// the scaled PHS system's condition numbers (<= ~1e7 for m <= 6 on the
// node sets measured) the weights stay within ~1e-10 of the FP64 ones, so
// the DF form is offered for 1 <= m <= 6 only.
struct NsF64 {
    using S = double;
    using V = double;
    static __device__ __forceinline__ V ld(const S* p) { return *p; }
    static __device__ __forceinline__ void st(S* p, V v) { *p = v; }
    static __device__ __forceinline__ V from_d(double x) { return x; }
    static __device__ __forceinline__ double to_d(V v) { return v; }
    static __device__ __forceinline__ V zero() { return 0.0; }
    static __device__ __forceinline__ V cst(double x) { return x; }
    // c - a b
    static __device__ __forceinline__ V nfma(V a, V b, V c) { return fma(-a, b, c); }
    static __device__ __forceinline__ V mul(V a, V b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __dadd_rn(a, -b); }
    static __device__ __forceinline__ V rcp(V a) { return rcp64(a); }
    static __device__ __forceinline__ V sqrt(V a) { return sqrt64(a); }
    // |x|^3 of the difference (dx, dy): r^2 by one FMA, then r^2 sqrt(r^2)
    static __device__ __forceinline__ V r3(V dx, V dy) {
        const double r2 = fma(dx, dx, __dmul_rn(dy, dy));
        return __dmul_rn(r2, sqrt64(r2));
    }
    // pivot search key (monotone in |a|); tests on it and on values by
    // integer instructions (FP64 compares would occupy the FP64 units)
    static __device__ __forceinline__ unsigned long long key(V a) { return abs_bits(a); }
    static __device__ __forceinline__ bool key_small(unsigned long long k) {
        return k < 0x3d719799812dea11ull;  // |a| < 1e-12
    }
    static __device__ __forceinline__ bool key_nonfinite(unsigned long long k) { return k >= 0x7ff0000000000000ull; }
    static __device__ __forceinline__ bool is_zero(V a) { return (abs_bits(a)) == 0ull; }
    static __device__ __forceinline__ bool pos_finite(V a) { return positive_finite64(a); }
};

struct NsDF {
    using S = float2;
    using V = df;
    static __device__ __forceinline__ V ld(const S* p) { return df_load(p); }
    static __device__ __forceinline__ void st(S* p, V v) { df_store(p, v); }
    static __device__ __forceinline__ V from_d(double x) { return df_from_double(x); }
    static __device__ __forceinline__ double to_d(V v) { return df_to_double(v); }
    static __device__ __forceinline__ V zero() { return df_make(0.f, 0.f); }
    static __device__ __forceinline__ V cst(double x) { return df_make((float)x, 0.f); }  // small exact constants
    // c - a b: the product exactly to ~2^-48 (TwoProd of the leading parts,
    // cross terms by FMA), then TwoSum with c.
    static __device__ __forceinline__ V nfma(V a, V b, V c) {
        const df p = two_prod(a.hi, b.hi);
        const float pl = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
        const df s = two_sum(c.hi, -p.hi);
        const float e = __fadd_rn(__fsub_rn(c.lo, pl), s.lo);
        return fast_two_sum(s.hi, e);
    }
    static __device__ __forceinline__ V mul(V a, V b) { return df_mul(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return df_add(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return df_sub(a, b); }
    // 1/a: float reciprocal r, then one Newton step r + r (1 - a r) with the
    // residual 1 - a r formed from an exact product
    static __device__ __forceinline__ V rcp(V a) {
        const float r = __frcp_rn(a.hi);
        const df p = two_prod(a.hi, r);
        const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p.hi), p.lo), __fmul_rn(a.lo, r));
        return fast_two_sum(r, __fmul_rn(r, e));
    }
    // a^-1/2: float rsqrt, one Newton step in float (to ~1 ulp), then one in
    // double-float, y + (y/2)(1 - a y^2) with a y^2 from an exact square
    static __device__ __forceinline__ V rsqrt(V a) {
        const float y0 = rsqrtf(a.hi);
        const float y = __fmaf_rn(__fmul_rn(0.5f, y0), __fmaf_rn(-__fmul_rn(a.hi, y0), y0, 1.0f), y0);
        const df y2 = two_prod(y, y);
        const df ay2 = df_mul(a, y2);
        const float e = __fsub_rn(__fsub_rn(1.0f, ay2.hi), ay2.lo);
        return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e));
    }
    static __device__ __forceinline__ V sqrt(V a) { return (a.hi > 0.f) ? df_mul(a, rsqrt(a)) : df_make(0.f, 0.f); }
    // |x|^3 of the difference (dx, dy): r^3 = r^2 (r^2 rsqrt(r^2))
    static __device__ __forceinline__ V r3(V dx, V dy) {
        const df r2 = df_add(df_mul(dx, dx), df_mul(dy, dy));
        return df_mul(r2, df_mul(r2, rsqrt(r2)));
    }
    static __device__ __forceinline__ unsigned long long key(V a) {
        return (unsigned long long)(__float_as_uint(a.hi) & 0x7fffffffu);
    }
    static __device__ __forceinline__ bool key_small(unsigned long long k) {
        return k < 0x2b8cbcccull;  // |a| < 1e-12f
    }
    static __device__ __forceinline__ bool key_nonfinite(unsigned long long k) { return k >= 0x7f800000ull; }
    static __device__ __forceinline__ bool is_zero(V a) { return a.hi == 0.f && a.lo == 0.f; }
    static __device__ __forceinline__ bool pos_finite(V a) { return a.hi > 0.f && isfinite(a.hi); }
};

// op 0: Laplacian weights at the stencil's first node (N = Nd, cxy = xy).
// op 1: interpolation weights of the value at the query point cxy[node]
//       (stencils index the Nd points xy): right-hand side [ |xh_j|^3 ;
//       p_k(0) ], no rescaling.
//
// Scalars that one step of the elimination needs (a pivot's reciprocal, the
// next diagonal entry's reciprocal, the scale) are computed by one thread
// and handed to the others through shared memory: computed by every thread
// of the group they cost as many FP64 lane-operations as a full row update.
template <int NT, class R>
__global__ void __launch_bounds__(128) weights_ns_kernel(const double2* __restrict__ xy, const int* __restrict__ idx,
                                                         int N, int n, int m, int s, int LDQ, int LDS,
                                                         int bytes_per_warp, double* __restrict__ w,
                                                         int* __restrict__ node_status,
                                                         const double2* __restrict__ cxy, int Nd, int op) {
    using S = typename R::S;
    using V = typename R::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // NT threads per stencil: half a warp or one warp (several stencils per
    // block) or two or four warps (one stencil per block, block-wide
    // synchronisation)
    const int lane = threadIdx.x % NT;
    const int wib = threadIdx.x / NT;
    const int wpb = blockDim.x / NT;
    __shared__ unsigned long long red_u64[4];
    __shared__ int red_i[8];
    const int q = n - s;
    const int LDX = LDS;
    S* Phi = reinterpret_cast<S*>(smem_raw + (size_t)wib * bytes_per_warp);
    S* P = Phi;  // the elimination's matrix, inside Phi's region until Phi is built
    S* A11 = Phi;
    S* A12 = A11 + (size_t)s * LDS;
    S* A22 = A12 + (size_t)s * LDQ;  // lower triangle, row i at i (i + 1) / 2
    S* X = Phi + ns_phi_region(n, s, LDS, LDQ);
    S* w0 = X + (size_t)q * LDX;
    S* crd = w0 + s;
    S* fv = crd + 2 * n;
    S* uv = fv + n;
    S* wv = uv + n;
    S* tv = wv + n;
    int* perm = reinterpret_cast<int*>(tv + n);
    int* act = perm + n;
    // 8-byte slots either way (S is double or float2): raw FP64 differences
    // in crd before scaling, the scale factors in wv until the weights
    double* crdd = reinterpret_cast<double*>(crd);
    double* scal = reinterpret_cast<double*>(wv);
    const int total_warps = gridDim.x * wpb;
    // loads and stores of the group's region (tested against it in the
    // checked build, whose first test is that the region lies in the launch's
    // shared memory)
    const int region = bytes_per_warp / (int)sizeof(S);
    (void)region;  // the bound of the checked build's tests
    (void)RB_SH(smem_raw + (size_t)(wib + 1) * bytes_per_warp - 1);
    auto ldc = [&](const S* p) -> V { return R::ld(&RB_PT(p, Phi, region)); };
    auto stc = [&](S* p, V v) { R::st(&RB_PT(p, Phi, region), v); };

    for (int node = blockIdx.x * wpb + wib; node < N; node += total_warps) {
        const int* sten = idx + (int64_t)node * n;
        const double2 c = cxy[node];

        // ---- shift (FP64): differences and the largest squared distance ------
        unsigned long long dmax = 0;
        int bad = 0;
        for (int j = lane; j < n; j += NT) {
            const int sj = sten[j];
            const bool ok = (unsigned)sj < (unsigned)Nd;  // never read outside xy
            bad |= ok ? 0 : 1;
            const double2 p = ok ? xy[sj] : c;
            const double dx = __dadd_rn(p.x, -c.x);
            const double dy = __dadd_rn(p.y, -c.y);
            RB_AT(crdd, 2 * j, 2 * n) = dx;
            RB_AT(crdd, 2 * j + 1, 2 * n) = dy;
            const unsigned long long b = abs_bits(fma(dx, dx, __dmul_rn(dy, dy)));
            dmax = (b > dmax) ? b : dmax;
        }
#pragma unroll
        for (int o = group_shfl_top<NT>(); o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(group_mask<NT>(), dmax, o);
            dmax = (t > dmax) ? t : dmax;
        }
        dmax = group_max_u64<NT>(dmax, red_u64);
        // scale: 1/delta = (max d^2)^-1/2 and 1/delta^2, by one thread
        if (lane == 0) {
            const double id = rsqrt64(__longlong_as_double((long long)dmax));
            scal[0] = id;
            scal[1] = __dmul_rn(id, id);
        }
        group_sync<NT>();
        const double inv_delta = scal[0], inv_delta2 = scal[1];
        const int bad_any = group_any<NT>(bad);

        // interpolation at a point that is its own first neighbour (a fine
        // node kept on the coarse level): the weights are e_1, the value there
        if (op && !bad_any && abs_bits(RB_AT(crdd, 0, 2 * n)) == 0ull && abs_bits(RB_AT(crdd, 1, 2 * n)) == 0ull) {
            double* wo = w + (int64_t)node * n;
            for (int a = lane; a < n; a += NT) wo[a] = a == 0 ? 1.0 : 0.0;
            if (node_status && lane == 0) node_status[node] = 0;
            group_sync<NT>();
            continue;
        }

        // ---- P (rows 0..n-1: monomials at xh_j; row n: g) ------------------
        // degree d from degree d - 1 of the same row: x^(d-i) y^i = x * x^(d-1-i) y^i
        // for i < d, and y^d = y * y^(d-1)
        for (int j = lane; j < n; j += NT) {
            const V xh = R::from_d(__dmul_rn(RB_AT(crdd, 2 * j, 2 * n), inv_delta));
            const V yh = R::from_d(__dmul_rn(RB_AT(crdd, 2 * j + 1, 2 * n), inv_delta));
            stc(crd + 2 * j, xh);
            stc(crd + 2 * j + 1, yh);
            S* pr = P + (size_t)j * LDS;
            stc(pr, R::cst(1.0));
            if (m >= 1) {
                stc(pr + 1, xh);
                stc(pr + 2, yh);
            }
            for (int d = 2, prev = 1, cur = 3; d <= m; prev = cur, cur += d + 1, ++d) {
                for (int i = 0; i < d; ++i) stc(pr + cur + i, R::mul(xh, ldc(pr + prev + i)));
                stc(pr + cur + d, R::mul(yh, ldc(pr + prev + d - 1)));
            }
            RB_AT(act, j, n) = j;
        }
        for (int col = lane; col < s; col += NT) {
            // g_k = lap p_k(0): 2 for x^2 (index 3) and y^2 (index 5);
            // interpolation: p_k(0), 1 for the constant
            const bool one = op ? (col == 0) : (col == 3 || col == 5);
            stc(P + (size_t)n * LDS + col, one ? R::cst(op ? 1.0 : 2.0) : R::zero());
        }
        group_sync<NT>();

        // ---- Gauss-Jordan with row pivoting on P ------------------------------
        int na = n;  // active (not yet pivot) rows act[0..na)
        int singular = bad_any ? 1 : 0;
        for (int k = 0; k < s && !singular; ++k) {
            unsigned long long best = 0;
            int bi = 0x7fffffff, bpos = -1;
            for (int t = lane; t < na; t += NT) {
                const int r = RB_AT(act, t, n);
                const unsigned long long b = R::key(ldc(P + (size_t)r * LDS + k));
                if (b > best || (b == best && r < bi)) {
                    best = b;
                    bi = r;
                    bpos = t;
                }
            }
#pragma unroll
            for (int o = group_shfl_top<NT>(); o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(group_mask<NT>(), best, o);
                const int oi = __shfl_xor_sync(group_mask<NT>(), bi, o);
                const int op_ = __shfl_xor_sync(group_mask<NT>(), bpos, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                    bpos = op_;
                }
            }
            group_argmax<NT>(best, bi, bpos, red_u64, red_i);
            // rank deficient (pivot below 1e-12: P's entries are monomials of
            // points in the unit disk, so |P| <= 1) or non-finite
            if (R::key_small(best) || R::key_nonfinite(best)) {
                singular = 1;
                break;
            }
            const int pr = bi;
            // the pivot's reciprocal, by one thread, in tv[0] (free until the
            // substitutions); every thread has finished the search above
            // (shuffles, or the block barriers of group_argmax)
            if (lane == 0) {
                stc(tv, R::rcp(ldc(P + (size_t)pr * LDS + k)));
                RB_AT(perm, k, n) = pr;
                RB_AT(act, bpos, n) = RB_AT(act, na - 1, n);  // swap-remove the pivot row
            }
            --na;
            group_sync<NT>();
            const V inv = ldc(tv);
            // every active row and the g row: column k scaled by the pivot
            // reciprocal (pivot row -> e_k) ...
            for (int t = lane; t <= na; t += NT) {
                S* rr = P + (size_t)((t < na) ? RB_AT(act, t, n) : n) * LDS;
                stc(rr + k, R::mul(ldc(rr + k), inv));
            }
            group_sync<NT>();
            // ... then column j -= P[pr][j] * (scaled) P[r][k] for j != k,
            // flattened over (row, column) so that every lane of the group
            // has an element (one thread per row left whole warps idle once
            // fewer rows than lanes remained); the pivot row is only read
            const S* prow = P + (size_t)pr * LDS;
            const int C = s - 1, total = (na + 1) * C;
            if (C > 0) {
                int t = lane / C, jj = lane - (lane / C) * C;
                const int dt = NT / C, dj = NT - (NT / C) * C;
                for (int e = lane; e < total; e += NT) {
                    S* rr = P + (size_t)((t < na) ? RB_AT(act, t, n) : n) * LDS;
                    const int j = jj < k ? jj : jj + 1;
                    stc(rr + j, R::nfma(ldc(prow + j), ldc(rr + k), ldc(rr + j)));
                    t += dt;
                    jj += dj;
                    if (jj >= C) {
                        jj -= C;
                        ++t;
                    }
                }
            }
            group_sync<NT>();
        }
        if (!singular) {
            for (int t = lane; t < q; t += NT) RB_AT(perm, s + t, n) = RB_AT(act, t, n);
            // X (rows of the non-pivot nodes) and w0 out of P, whose region
            // Phi takes next: X[j][k] = P[act[j]][k], w0[k] = P[n][k]
            for (int e = lane; e < (q + 1) * s; e += NT) {
                const int j = e / s, k = e - (e / s) * s;
                if (j < q) stc(X + (size_t)j * LDX + k, ldc(P + (size_t)RB_AT(act, j, n) * LDS + k));
                else stc(w0 + k, ldc(P + (size_t)n * LDS + k));
            }
        }
        group_sync<NT>();

        // ---- Phi's blocks in permuted order, and f = 9 |xh| ------------------
        int coincident = 0;
        if (!singular) {
            const int npairs = n * (n - 1) / 2;
            for (int pidx = lane; pidx < npairs; pidx += NT) {
                int a = (int)((2.0f * n - 1.0f - sqrtf((2.0f * n - 1.0f) * (2.0f * n - 1.0f) - 8.0f * pidx)) * 0.5f);
                if (a < 0) a = 0;
                while (a > 0 && a * (2 * n - a - 1) / 2 > pidx) --a;
                while ((a + 1) * (2 * n - a - 2) / 2 <= pidx) ++a;
                const int b = pidx - a * (2 * n - a - 1) / 2 + a + 1;  // a < b
                const int ja = RB_AT(perm, a, n), jb = RB_AT(perm, b, n);
                const V dx = R::sub(ldc(crd + 2 * ja), ldc(crd + 2 * jb));
                const V dy = R::sub(ldc(crd + 2 * ja + 1), ldc(crd + 2 * jb + 1));
                const bool same = R::is_zero(dx) && R::is_zero(dy);
                coincident |= same ? 1 : 0;
                const V phi = same ? R::zero() : R::r3(dx, dy);
                if (b < s) {
                    stc(A11 + (size_t)a * LDS + b, phi);
                    stc(A11 + (size_t)b * LDS + a, phi);
                } else if (a < s) {
                    stc(A12 + (size_t)a * LDQ + (b - s), phi);
                } else {
                    const int i = b - s;
                    stc(A22 + (size_t)(i * (i + 1) / 2 + (a - s)), phi);
                }
            }
            for (int a = lane; a < n; a += NT) {
                if (a < s) stc(A11 + (size_t)a * LDS + a, R::zero());
                else stc(A22 + (size_t)((a - s) * (a - s + 1) / 2 + (a - s)), R::zero());
                const int ja = RB_AT(perm, a, n);
                const V xh = ldc(crd + 2 * ja), yh = ldc(crd + 2 * ja + 1);
                // f = lap |x - x_c|^3 = 9 |xh| at the centre; interpolation: |xh|^3
                const V rr = R::add(R::mul(xh, xh), R::mul(yh, yh));
                stc(fv + a, R::mul(op ? rr : R::cst(9.0), R::sqrt(rr)));
            }
        }
        singular |= group_any<NT>(coincident) ? 1 : 0;
        group_sync<NT>();

        if (!singular) {
            // ---- S' = Phi22 - Phi21 X^T (lower triangle, in place) ----------
            // (Phi21 = Phi12^T: column j of A12.)  Before T overwrites A12.
            const int nlow = q * (q + 1) / 2;
            for (int e = lane; e < nlow; e += NT) {
                int j = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                while (j * (j + 1) / 2 > e) --j;
                while ((j + 1) * (j + 2) / 2 <= e) ++j;
                const int l = e - j * (j + 1) / 2;
                const S* xl = X + (size_t)l * LDX;
                V acc = ldc(A22 + e), acc1 = R::zero();
                int k = 0;
                for (; k + 1 < s; k += 2) {
                    acc = R::nfma(ldc(A12 + (size_t)k * LDQ + j), ldc(xl + k), acc);
                    acc1 = R::nfma(ldc(A12 + (size_t)(k + 1) * LDQ + j), ldc(xl + k + 1), acc1);
                }
                if (k < s) acc = R::nfma(ldc(A12 + (size_t)k * LDQ + j), ldc(xl + k), acc);
                stc(A22 + e, R::add(acc, acc1));
            }
            // ---- u = f - Phi[:, 0..s) w0 (rows r1 from A11, rows r2 from A12^T) ----
            for (int a = lane; a < n; a += NT) {
                V acc = ldc(fv + a), acc1 = R::zero();
                int k = 0;
                if (a < s) {
                    const S* pr = A11 + (size_t)a * LDS;
                    for (; k + 1 < s; k += 2) {
                        acc = R::nfma(ldc(pr + k), ldc(w0 + k), acc);
                        acc1 = R::nfma(ldc(pr + k + 1), ldc(w0 + k + 1), acc1);
                    }
                    if (k < s) acc = R::nfma(ldc(pr + k), ldc(w0 + k), acc);
                } else {
                    const S* pc = A12 + (a - s);
                    for (; k + 1 < s; k += 2) {
                        acc = R::nfma(ldc(pc + (size_t)k * LDQ), ldc(w0 + k), acc);
                        acc1 = R::nfma(ldc(pc + (size_t)(k + 1) * LDQ), ldc(w0 + k + 1), acc1);
                    }
                    if (k < s) acc = R::nfma(ldc(pc + (size_t)k * LDQ), ldc(w0 + k), acc);
                }
                stc(uv + a, R::add(acc, acc1));
            }
            group_sync<NT>();
            // ---- T = Phi12 - Phi11 X^T (s x q, in place in A12) --------------
            for (int e = lane; e < s * q; e += NT) {
                const int a = e / q, j = e - (e / q) * q;
                const S* xr = X + (size_t)j * LDX;
                const S* pr = A11 + (size_t)a * LDS;
                // two independent chains (latency, not issue, limits a single one)
                V acc = ldc(A12 + (size_t)a * LDQ + j), acc1 = R::zero();
                int k = 0;
                for (; k + 1 < s; k += 2) {
                    acc = R::nfma(ldc(pr + k), ldc(xr + k), acc);
                    acc1 = R::nfma(ldc(pr + k + 1), ldc(xr + k + 1), acc1);
                }
                if (k < s) acc = R::nfma(ldc(pr + k), ldc(xr + k), acc);
                stc(A12 + (size_t)a * LDQ + j, R::add(acc, acc1));
            }
            // ---- t = Z^T u = u[r2] - X u[r1] -------------------------------------
            for (int j = lane; j < q; j += NT) {
                const S* xj = X + (size_t)j * LDX;
                V acc = ldc(uv + s + j), acc1 = R::zero();
                int k = 0;
                for (; k + 1 < s; k += 2) {
                    acc = R::nfma(ldc(xj + k), ldc(uv + k), acc);
                    acc1 = R::nfma(ldc(xj + k + 1), ldc(uv + k + 1), acc1);
                }
                if (k < s) acc = R::nfma(ldc(xj + k), ldc(uv + k), acc);
                stc(tv + j, R::add(acc, acc1));
            }
            group_sync<NT>();
            // ---- S = S' - X T (lower triangle, in place) ---------------------
            for (int e = lane; e < nlow; e += NT) {
                int j = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                while (j * (j + 1) / 2 > e) --j;
                while ((j + 1) * (j + 2) / 2 <= e) ++j;
                const int l = e - j * (j + 1) / 2;
                const S* xj = X + (size_t)j * LDX;
                V acc = ldc(A22 + e), acc1 = R::zero();
                int k = 0;
                for (; k + 1 < s; k += 2) {
                    acc = R::nfma(ldc(xj + k), ldc(A12 + (size_t)k * LDQ + l), acc);
                    acc1 = R::nfma(ldc(xj + k + 1), ldc(A12 + (size_t)(k + 1) * LDQ + l), acc1);
                }
                if (k < s) acc = R::nfma(ldc(xj + k), ldc(A12 + (size_t)k * LDQ + l), acc);
                stc(A22 + e, R::add(acc, acc1));
            }
            group_sync<NT>();
            // ---- S = L D L^T: unit lower L in place, 1/D in fv -----------------
            // (S is positive definite: no pivoting.)  Column c: the unscaled
            // column goes to uv (free now), L[i][c] = S[i][c] / D[c], then
            // S[i][j] -= L[i][c] S[j][c] for c < j <= i.  The thread that
            // updates the next diagonal entry also forms its reciprocal and
            // the singularity flag (act[0], free after the elimination).
            if (q > 0) {
                if (lane == 0) {
                    const V d0 = ldc(A22);
                    RB_AT(act, 0, n) = R::pos_finite(d0) ? 0 : 1;
                    stc(fv, R::rcp(d0));
                }
                group_sync<NT>();
            }
            for (int cI = 0; cI < q; ++cI) {
                if (RB_AT(act, 0, n)) {
                    singular = 1;
                    break;
                }
                const V invd = ldc(fv + cI);
                for (int i = cI + 1 + lane; i < q; i += NT) {
                    S* si = A22 + (size_t)(i * (i + 1) / 2);
                    const V v = ldc(si + cI);
                    stc(uv + i, v);
                    stc(si + cI, R::mul(v, invd));
                }
                group_sync<NT>();
                const int rem = q - cI - 1, ntr = rem * (rem + 1) / 2;
                for (int e = lane; e < ntr; e += NT) {
                    int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                    while (i * (i + 1) / 2 > e) --i;
                    while ((i + 1) * (i + 2) / 2 <= e) ++i;
                    const int j = e - i * (i + 1) / 2;
                    const int ri = cI + 1 + i;
                    S* si = A22 + (size_t)(ri * (ri + 1) / 2);
                    const V nv = R::nfma(ldc(si + cI), ldc(uv + cI + 1 + j), ldc(si + cI + 1 + j));
                    stc(si + cI + 1 + j, nv);
                    if (e == 0) {  // (i, j) = (0, 0): the next diagonal entry, final now
                        RB_AT(act, 0, n) = R::pos_finite(nv) ? 0 : 1;
                        stc(fv + cI + 1, R::rcp(nv));
                    }
                }
                group_sync<NT>();
            }
        }
        if (!singular) {
            // ---- L y = t, z = D^-1 y, L^T x = z (unit triangles) -----------------
            for (int cI = 0; cI < q; ++cI) {
                const V yc = ldc(tv + cI);
                for (int i = cI + 1 + lane; i < q; i += NT)
                    stc(tv + i, R::nfma(ldc(A22 + (size_t)(i * (i + 1) / 2 + cI)), yc, ldc(tv + i)));
                group_sync<NT>();
            }
            for (int i = lane; i < q; i += NT) stc(tv + i, R::mul(ldc(tv + i), ldc(fv + i)));
            group_sync<NT>();
            for (int cI = q - 1; cI >= 0; --cI) {
                const S* sc = A22 + (size_t)(cI * (cI + 1) / 2);
                const V zc = ldc(tv + cI);
                for (int i = lane; i < cI; i += NT) stc(tv + i, R::nfma(ldc(sc + i), zc, ldc(tv + i)));
                group_sync<NT>();
            }
            // ---- w = w0 + Z z: w[r2_j] = z_j, w[r1_k] = w0_k - sum_j X[j][k] z_j ----
            for (int k = lane; k < s; k += NT) {
                V acc = ldc(w0 + k), acc1 = R::zero();
                int j = 0;
                for (; j + 1 < q; j += 2) {
                    acc = R::nfma(ldc(X + (size_t)j * LDX + k), ldc(tv + j), acc);
                    acc1 = R::nfma(ldc(X + (size_t)(j + 1) * LDX + k), ldc(tv + j + 1), acc1);
                }
                if (j < q) acc = R::nfma(ldc(X + (size_t)j * LDX + k), ldc(tv + j), acc);
                stc(wv + k, R::add(acc, acc1));
            }
            for (int j = lane; j < q; j += NT) stc(wv + s + j, ldc(tv + j));
            group_sync<NT>();
        }

        // ---- scale back (FP64) to the caller's order -------------------------
        // (each lane rewrites its own slots of wv as doubles: 8 bytes either way)
        double* wout = w + (int64_t)node * n;
        double* wd = reinterpret_cast<double*>(wv);
        int nonfinite = 0;
        for (int a = lane; a < n; a += NT) {
            const double v = singular ? 0.0 : (op ? R::to_d(ldc(wv + a)) : __dmul_rn(R::to_d(ldc(wv + a)), inv_delta2));
            nonfinite |= finite64(v) ? 0 : 1;
            wd[a] = v;
        }
        const int fail = (singular || group_any<NT>(nonfinite)) ? 1 : 0;
        group_sync<NT>();
        for (int a = lane; a < n; a += NT) RB_AT(wout, singular ? a : RB_AT(perm, a, n), n) = fail ? 0.0 : wd[a];
        if (node_status && lane == 0) node_status[node] = fail;
        group_sync<NT>();
    }
}

// Warps per block maximising resident warps per SM for a per-warp shared
// memory footprint (228 KB per SM, 1 KB reserved per block, <= 32 blocks).
int warps_per_block_for(size_t per_warp, size_t* smem_bytes) {
    int best_w = 1, best_res = 0;
    for (int wpb = 1; wpb <= 4; ++wpb) {
        const size_t blk = per_warp * wpb;
        if (blk > 227 * 1024) break;
        int blocks = (int)(233472 / (blk + 1024));
        blocks = std::min(blocks, 32);
        const int res = std::min(blocks * wpb, 64);
        if (res >= best_res) {
            best_res = res;
            best_w = wpb;
        }
    }
    *smem_bytes = per_warp * best_w;
    return best_w;
}

int weights_warps_per_block(const WeightsGeom& g, size_t* smem_bytes) {
    return warps_per_block_for((size_t)g.smem_doubles * sizeof(double), smem_bytes);
}

}  // namespace
}  // namespace rbffd

namespace rbffd {
namespace {

// Launch configuration of the weight solve: kernel variant and warps (one
// stencil each) per block.  The default per (n, m) follows the shared-memory
// footprint; rbffd_weights_autotune replaces it with the fastest measured
// candidate, kept in a process-wide table per (device, n, m).
struct WCfg {
    int kernel;  // 0 null-space elimination (one warp per stencil), 1 full Gaussian
                 // elimination, 2 / 3 null-space elimination with two / four warps
                 // per stencil; 4 / 5 / 6: 0 / 2 / 3 in double-float arithmetic;
                 // 7 / 8: null-space elimination with half a warp per stencil,
                 // FP64 / double-float; 9 / 10: the same with a quarter warp
    int wpb;     // warps per block (kernels 2, 3: 2 or 4, one stencil)
};

std::mutex g_wcfg_mu;
std::map<std::tuple<int, int, int>, std::pair<WCfg, double>> g_wcfg;  // -> (config, ms per 1e6 stencils)

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// Shared memory per stencil.
size_t smem_per_stencil(int kernel, int n, int m) {
    if (kernel == 1) return (size_t)weights_geom(n, m).smem_doubles * sizeof(double);
    return (size_t)ns_geom(n, m).bytes;
}

// Stencils per block of a configuration, and its dynamic shared memory.
int stencils_per_block(const WCfg& c) {
    if (c.kernel >= 9) return 4 * c.wpb;
    if (c.kernel >= 7) return 2 * c.wpb;
    return (c.kernel == 2 || c.kernel == 3 || c.kernel == 5 || c.kernel == 6) ? 1 : c.wpb;
}

bool cfg_is_df(const WCfg& c) { return (c.kernel >= 4 && c.kernel <= 6) || c.kernel == 8 || c.kernel == 10; }

// The double-float null-space kernels: 1 <= m <= 6 (accuracy, see NsDF).
constexpr int kDfMaxM = 6;
size_t block_smem(const WCfg& c, int n, int m) { return smem_per_stencil(c.kernel, n, m) * stencils_per_block(c); }

bool cfg_valid(const WCfg& c, int n, int m) {
    if (c.kernel < 0 || c.kernel > 10) return false;
    if (c.kernel != 1 && m < 1) return false;  // null-space form needs the linear monomials
    if (cfg_is_df(c) && m > kDfMaxM) return false;
    if ((c.kernel == 2 || c.kernel == 5) && c.wpb != 2) return false;
    if ((c.kernel == 3 || c.kernel == 6) && c.wpb != 4) return false;
    if ((c.kernel <= 1 || c.kernel == 4 || c.kernel >= 7) && (c.wpb < 1 || c.wpb > 4))
        return false;  // __launch_bounds__(128)
    return block_smem(c, n, m) <= 227 * 1024;
}

WCfg default_cfg(int n, int m) {
    WCfg c;
    // FP64 by default: null-space elimination (m >= 1: the form needs r^3
    // positive definite on the null space of P^T, which holds once P
    // contains the linear monomials), full elimination for m = 0
    c.kernel = m < 1 ? 1 : 0;
    size_t smem = 0;
    c.wpb = warps_per_block_for(smem_per_stencil(c.kernel, n, m), &smem);
    // large systems (m >= 5): two warps per stencil, as measured fastest in
    // FP64 (m = 6, n = 56, 4M nodes: 1,346 ms against 1,595 with one warp)
    const WCfg big{2, 2};
    if (m >= 5 && cfg_valid(big, n, m)) return big;
    // the smallest systems (m <= 2, n <= 16): a quarter of a warp per stencil
    // (2M nodes, m = 2, n = 12: 6.3 ms per 1e6 stencils against 8.2 with
    // half a warp and 13.0 with a warp)
    const WCfg quarter{9, 2};
    if (m <= 2 && n <= 16 && cfg_valid(quarter, n, m)) return quarter;
    // small systems (m <= 4, n <= 32): half a warp per stencil (1M nodes:
    // m = 2, n = 12 8.3 ms against 13.0; m = 4, n = 30 45.3 against 50.4)
    const WCfg half{7, 2};
    if (m <= 4 && n <= 32 && cfg_valid(half, n, m)) return half;
    return c;
}

// The double-float kernels for the preconditioner's small systems (coarse
// operators and interpolation, n = 12, m = 2: 3.6 ms per 1e6 stencils with a
// quarter of a warp per stencil against 4.9 with half a warp and 7.7 with a
// warp), else the warp-per-stencil form.
WCfg small_df_cfg(int n, int m) {
    const WCfg quarter{10, 2};
    if (n <= 16 && m <= 2 && cfg_valid(quarter, n, m)) return quarter;
    const WCfg half{8, 2};
    if (n <= 20 && cfg_valid(half, n, m)) return half;
    WCfg c{4, 1};
    size_t smem = 0;
    c.wpb = warps_per_block_for(smem_per_stencil(4, n, m), &smem);
    return c;
}

WCfg chosen_cfg(int n, int m) {
    // RBFFD_WEIGHTS=lu forces the full Gaussian elimination (comparisons)
    // RBFFD_WEIGHTS=ns64 forces the FP64 null-space elimination, one warp
    // RBFFD_WEIGHTS=df forces its double-float form, one warp (1 <= m <= 6)
    const char* sel = std::getenv("RBFFD_WEIGHTS");
    if (sel && std::strcmp(sel, "df") == 0 && m >= 1 && m <= kDfMaxM) {
        WCfg c{4, 1};
        size_t smem = 0;
        c.wpb = warps_per_block_for(smem_per_stencil(c.kernel, n, m), &smem);
        if (cfg_valid(c, n, m)) return c;
    }
    if (sel && (std::strcmp(sel, "lu") == 0 || (std::strcmp(sel, "ns64") == 0 && m >= 1))) {
        WCfg c = default_cfg(n, m);
        size_t smem = 0;
        c.kernel = std::strcmp(sel, "lu") == 0 ? 1 : 0;
        c.wpb = warps_per_block_for(smem_per_stencil(c.kernel, n, m), &smem);
        return c;
    }
    std::lock_guard<std::mutex> lk(g_wcfg_mu);
    auto it = g_wcfg.find(std::make_tuple(current_device(), n, m));
    if (it != g_wcfg.end()) return it->second.first;
    return default_cfg(n, m);
}

template <int NT, class R>
int launch_ns(const WCfg& c, const double2* xy, const int32_t* idx, int64_t N, int n, int m, double* w,
              int32_t* node_status, cudaStream_t st, const double2* cxy = nullptr, int64_t Nd = 0, int op = 0) {
    if (!cxy) {
        cxy = xy;
        Nd = N;
    }
    NsGeom g = ns_geom(n, m);
    const int spb = stencils_per_block(c);
    const size_t smem = block_smem(c, n, m);
    auto kern = weights_ns_kernel<NT, R>;
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    RBFFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT * spb, smem));
    if (per_sm < 1) return RBFFD_ERR_INVALID_ARG;
    const int64_t need = (N + spb - 1) / spb;
    const int blocks = (int)std::min<int64_t>(need, (int64_t)per_sm * sm_count());
    kern<<<blocks, NT * spb, smem, st>>>(xy, idx, (int)N, n, m, g.s, g.LDQ, g.LDS, g.bytes, w, node_status, cxy,
                                         (int)Nd, op);
    return RBFFD_OK;
}

int launch_weights(const WCfg& c, const double* xy, const int32_t* idx, int64_t N, int n, int m, double* w,
                   int32_t* node_status, cudaStream_t st) {
    if (!cfg_valid(c, n, m)) return RBFFD_ERR_INVALID_ARG;
    const double2* p = reinterpret_cast<const double2*>(xy);
    int rc = RBFFD_OK;
    if (c.kernel == 1) {
        WeightsGeom g = weights_geom(n, m);
        const int wpb = c.wpb;
        const size_t smem = block_smem(c, n, m);
        RBFFD_CUDA_TRY(cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RBFFD_CUDA_TRY(cudaFuncSetAttribute(weights_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        int per_sm = 0;
        RBFFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, weights_kernel, 32 * wpb, smem));
        if (per_sm < 1) return RBFFD_ERR_INVALID_ARG;
        const int64_t need = (N + wpb - 1) / wpb;
        const int blocks = (int)std::min<int64_t>(need, (int64_t)per_sm * sm_count());
        weights_kernel<<<blocks, 32 * wpb, smem, st>>>(p, idx, (int)N, n, m, g.s, g.M, g.LD, g.coords_in_zero_block,
                                                       g.smem_doubles, w, node_status, p, (int)N, 0);
    } else if (c.kernel == 0) {
        rc = launch_ns<32, NsF64>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 2) {
        rc = launch_ns<64, NsF64>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 3) {
        rc = launch_ns<128, NsF64>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 4) {
        rc = launch_ns<32, NsDF>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 5) {
        rc = launch_ns<64, NsDF>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 6) {
        rc = launch_ns<128, NsDF>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 7) {
        rc = launch_ns<16, NsF64>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 8) {
        rc = launch_ns<16, NsDF>(c, p, idx, N, n, m, w, node_status, st);
    } else if (c.kernel == 9) {
        rc = launch_ns<8, NsF64>(c, p, idx, N, n, m, w, node_status, st);
    } else {
        rc = launch_ns<8, NsDF>(c, p, idx, N, n, m, w, node_status, st);
    }
    if (rc != RBFFD_OK) return rc;
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

bool weights_args_ok(const double* xy, const int32_t* idx, const double* w, int64_t N, int32_t n, int32_t m) {
    if (!xy || !idx || !w || N <= 0 || N > 0x7fffffffLL || n < 1 || n > RBFFD_MAX_STENCIL || m < 0 || m > 8)
        return false;
    if (((uintptr_t)xy & 15) != 0) return false;
    return n >= (m + 1) * (m + 2) / 2;
}

}  // namespace
}  // namespace rbffd

extern "C" int rbffd_weights(const double* xy, const int32_t* idx, int64_t N, int32_t n, int32_t m, double* w,
                             int32_t* node_status, void* stream) {
    RBFFD_NVTX("rbffd_weights");
    using namespace rbffd;
    if (!weights_args_ok(xy, idx, w, N, n, m)) return RBFFD_ERR_INVALID_ARG;
    return launch_weights(chosen_cfg(n, m), xy, idx, N, n, m, w, node_status, as_stream(stream));
}

extern "C" int rbffd_weights_autotune(const double* xy, const int32_t* idx, int64_t N, int32_t n, int32_t m,
                                      double* w, int32_t* node_status, int32_t precision,
                                      rbffd_weights_config* best, void* stream) {
    RBFFD_NVTX("rbffd_weights_autotune");
    using namespace rbffd;
    if (!weights_args_ok(xy, idx, w, N, n, m)) return RBFFD_ERR_INVALID_ARG;
    if (precision != RBFFD_WEIGHTS_FP64 && precision != RBFFD_WEIGHTS_DF && precision != RBFFD_WEIGHTS_ANY)
        return RBFFD_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    // sample: the first stencils, enough for many waves of resident stencils
    // (tail effects of a few waves decided between near-equal configurations)
    const int64_t S = std::min<int64_t>(N, (int64_t)sm_count() * 512);
    std::vector<WCfg> all;
    for (int kernel = 0; kernel <= 1; ++kernel)
        for (int wpb = 1; wpb <= 4; ++wpb) all.push_back(WCfg{kernel, wpb});
    all.push_back(WCfg{2, 2});
    all.push_back(WCfg{3, 4});
    for (int wpb = 1; wpb <= 4; ++wpb) all.push_back(WCfg{4, wpb});
    all.push_back(WCfg{5, 2});
    all.push_back(WCfg{6, 4});
    for (int wpb = 1; wpb <= 4; ++wpb) {
        all.push_back(WCfg{7, wpb});
        all.push_back(WCfg{8, wpb});
        all.push_back(WCfg{9, wpb});
        all.push_back(WCfg{10, wpb});
    }
    std::vector<WCfg> cands;
    for (const WCfg& c : all) {
        if (!cfg_valid(c, n, m)) continue;
        if (precision == RBFFD_WEIGHTS_FP64 && cfg_is_df(c)) continue;
        if (precision == RBFFD_WEIGHTS_DF && !cfg_is_df(c)) continue;
        cands.push_back(c);
    }
    if (cands.empty()) return RBFFD_ERR_INVALID_ARG;
    cudaEvent_t e0, e1;
    RBFFD_CUDA_TRY(cudaEventCreate(&e0));
    RBFFD_CUDA_TRY(cudaEventCreate(&e1));
    WCfg win = cands[0];
    double win_ms = INFINITY;
    int rc = RBFFD_OK;
    for (const WCfg& c : cands) {
        if ((rc = launch_weights(c, xy, idx, S, n, m, w, node_status, st)) != RBFFD_OK) break;  // warm-up
        float best_ms = INFINITY;  // the fastest of three timed launches
        for (int r = 0; r < 3 && rc == RBFFD_OK; ++r) {
            float ms = 0.f;
            if (cudaEventRecord(e0, st) != cudaSuccess) { rc = RBFFD_ERR_CUDA; break; }
            if ((rc = launch_weights(c, xy, idx, S, n, m, w, node_status, st)) != RBFFD_OK) break;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = RBFFD_ERR_CUDA;
                break;
            }
            best_ms = std::min(best_ms, ms);
        }
        if (rc != RBFFD_OK) break;
        const double per = best_ms * 1e6 / (double)S;  // ms per 1e6 stencils
        if (per < win_ms) {
            win_ms = per;
            win = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RBFFD_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_wcfg_mu);
        g_wcfg[std::make_tuple(current_device(), (int)n, (int)m)] = std::make_pair(win, win_ms);
    }
    if (best) {
        best->kernel = win.kernel;
        best->warps_per_block = win.wpb;
        best->ms_per_mnode = win_ms;
    }
    return RBFFD_OK;
}

extern "C" int rbffd_weights_get_config(int32_t n, int32_t m, rbffd_weights_config* cfg) {
    RBFFD_NVTX("rbffd_weights_get_config");
    using namespace rbffd;
    if (!cfg || n < 1 || n > RBFFD_MAX_STENCIL || m < 0 || m > 8 || n < (m + 1) * (m + 2) / 2)
        return RBFFD_ERR_INVALID_ARG;
    const WCfg c = chosen_cfg(n, m);
    double ms = 0.0;
    {
        std::lock_guard<std::mutex> lk(g_wcfg_mu);
        auto it = g_wcfg.find(std::make_tuple(current_device(), (int)n, (int)m));
        if (it != g_wcfg.end() && it->second.first.kernel == c.kernel && it->second.first.wpb == c.wpb)
            ms = it->second.second;
    }
    cfg->kernel = c.kernel;
    cfg->warps_per_block = c.wpb;
    cfg->ms_per_mnode = ms;
    return RBFFD_OK;
}

extern "C" int rbffd_weights_set_config(int32_t n, int32_t m, const rbffd_weights_config* cfg) {
    RBFFD_NVTX("rbffd_weights_set_config");
    using namespace rbffd;
    if (n < 1 || n > RBFFD_MAX_STENCIL || m < 0 || m > 8 || n < (m + 1) * (m + 2) / 2) return RBFFD_ERR_INVALID_ARG;
    const auto key = std::make_tuple(current_device(), (int)n, (int)m);
    std::lock_guard<std::mutex> lk(g_wcfg_mu);
    if (!cfg) {
        g_wcfg.erase(key);
        return RBFFD_OK;
    }
    if (!cfg_valid(WCfg{cfg->kernel, cfg->warps_per_block}, n, m)) return RBFFD_ERR_INVALID_ARG;
    g_wcfg[key] = std::make_pair(WCfg{cfg->kernel, cfg->warps_per_block}, 0.0);
    return RBFFD_OK;
}

// Laplacian weights of a preconditioner's coarse operator: the double-float
// null-space form where it is offered (1 <= m <= 6), FP64 otherwise.  Only
// the multigrid hierarchy uses them; its accuracy does not enter the
// solution, which the FP64 operator's residual decides.
int rbffd::coarse_weights(const double* xy, const int32_t* idx, int64_t N, int32_t n, int32_t m, double* w,
                          int32_t* node_status, cudaStream_t st) {
    if (!weights_args_ok(xy, idx, w, N, n, m)) return RBFFD_ERR_INVALID_ARG;
    WCfg c;
    size_t smem = 0;
    if (m >= 1 && m <= kDfMaxM) {
        c = small_df_cfg(n, m);
    } else {
        c.kernel = m < 1 ? 1 : 0;
        c.wpb = warps_per_block_for(smem_per_stencil(c.kernel, n, m), &smem);
    }
    return launch_weights(c, xy, idx, N, n, m, w, node_status, st);
}

// Interpolation weights (used by the multigrid transfer operators): for each
// of the Nq points q, the weights w (Nq x n) with sum_j w_j u(x_{idx_j})
// exact for polynomials of degree <= m, from the PHS r^3 + monomial system
// centred at q (the kernel above with op 1).  node_status: 1 where the
// system is singular (weights then 0).
int rbffd::interp_weights(const double* xy, int64_t Nd, const double* qxy, int64_t Nq, const int32_t* idx,
                          int32_t n, int32_t m, double* w, int32_t* node_status, cudaStream_t st) {
    if (!xy || !qxy || !idx || !w || Nq <= 0 || Nq > 0x7fffffffLL || Nd <= 0 || Nd > 0x7fffffffLL || n < 1 ||
        n > RBFFD_MAX_STENCIL || m < 0 || m > 8)
        return RBFFD_ERR_INVALID_ARG;
    const int s = (m + 1) * (m + 2) / 2;
    if (n < s) return RBFFD_ERR_INVALID_ARG;
    if (m >= 1) {
        // the null-space elimination of the same saddle system (double-float
        // for m <= 6), one warp per query point, stencils per block by the
        // shared-memory footprint
        WCfg c;
        size_t smem_b = 0;
        if (m <= kDfMaxM) {
            c = small_df_cfg(n, m);
        } else {
            c.kernel = 0;
            c.wpb = warps_per_block_for(smem_per_stencil(c.kernel, n, m), &smem_b);
        }
        if (!cfg_valid(c, n, m)) return RBFFD_ERR_INVALID_ARG;
        const double2* d2 = reinterpret_cast<const double2*>(xy);
        const double2* q2 = reinterpret_cast<const double2*>(qxy);
        const int rc = c.kernel == 10  ? launch_ns<8, NsDF>(c, d2, idx, Nq, n, m, w, node_status, st, q2, Nd, 1)
                       : c.kernel == 8 ? launch_ns<16, NsDF>(c, d2, idx, Nq, n, m, w, node_status, st, q2, Nd, 1)
                       : c.kernel == 4 ? launch_ns<32, NsDF>(c, d2, idx, Nq, n, m, w, node_status, st, q2, Nd, 1)
                                       : launch_ns<32, NsF64>(c, d2, idx, Nq, n, m, w, node_status, st, q2, Nd, 1);
        if (rc != RBFFD_OK) return rc;
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        return RBFFD_OK;
    }
    WeightsGeom g = weights_geom(n, m);
    size_t smem = 0;
    const int wpb = weights_warps_per_block(g, &smem);
    if (smem > 227 * 1024) return RBFFD_ERR_INVALID_ARG;
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RBFFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, weights_kernel, 32 * wpb, smem));
    if (per_sm < 1) return RBFFD_ERR_INVALID_ARG;
    const int64_t need = (Nq + wpb - 1) / wpb;
    const int blocks = (int)std::min<int64_t>(need, (int64_t)per_sm * sm_count());
    weights_kernel<<<blocks, 32 * wpb, smem, st>>>(reinterpret_cast<const double2*>(xy), idx, (int)Nq, n, m, g.s,
                                                   g.M, g.LD, g.coords_in_zero_block, g.smem_doubles, w, node_status,
                                                   reinterpret_cast<const double2*>(qxy), (int)Nd, 1);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}
