// RBF-FD Laplacian weights: one augmented PHS+polynomial system per stencil,
// solved in FP64 shared memory by one warp (sm_103a).
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

#include <algorithm>

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
__global__ void __launch_bounds__(128) weights_kernel(const double2* __restrict__ xy, const int* __restrict__ idx,
                                                      int N, int n, int m, int s, int M, int LD, int coords_zb,
                                                      int smem_doubles, double* __restrict__ w,
                                                      int* __restrict__ node_status) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double* A = smem + (size_t)wib * smem_doubles;
    // coordinate scratch of 2n doubles past the matrix, when the zero block
    // is too small to hold it
    double* cx = A + (size_t)M * LD;
    const int total_warps = gridDim.x * wpb;

    for (int node = blockIdx.x * wpb + wib; node < N; node += total_warps) {
        const int* sten = idx + (int64_t)node * n;
        const double2 c = xy[node];

        // ---- shift, scale --------------------------------------------------
        // Coordinates go to a linear scratch of 2n doubles.  In the zero
        // block, entry t is stored at row n + t / s, column n + t % s.
        auto cs = [&](int t) -> double& {
            if (coords_zb) return A[(size_t)(n + t / s) * LD + n + t % s];
            return cx[t];
        };
        unsigned long long dmax = 0;
        int bad_index = 0;
        for (int j = lane; j < n; j += 32) {
            const int sj = sten[j];
            const bool ok = (unsigned)sj < (unsigned)N;  // never read outside xy
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
                A[(size_t)j * LD + k] = phi;
                A[(size_t)k * LD + j] = phi;
            }
            for (int j = lane; j < n; j += 32) {
                A[(size_t)j * LD + j] = 0.0;
                const double xh = cs(2 * j), yh = cs(2 * j + 1);
                const double rj = __dsqrt_rn(__dadd_rn(__dmul_rn(xh, xh), __dmul_rn(yh, yh)));
                A[(size_t)j * LD + M] = __dmul_rn(9.0, rj);
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
                        A[(size_t)j * LD + n + col] = v;  // P
                        A[(size_t)(n + col) * LD + j] = v;  // P^T
                        ++col;
                    }
                }
            }
        }
        __syncwarp();
        // zero block and polynomial RHS (coordinates no longer needed)
        for (int t = lane; t < s * s; t += 32) A[(size_t)(n + t / s) * LD + n + t % s] = 0.0;
        {
            int col = 0;
            for (int d = 0; d <= m; ++d)
                for (int i = 0; i <= d; ++i, ++col)
                    if (lane == 0) A[(size_t)(n + col) * LD + M] = ((d == 2 && (i == 0 || i == 2)) ? 2.0 : 0.0);
        }
        __syncwarp();

        // ---- Gaussian elimination with partial pivoting ---------------------
        int singular = __any_sync(0xffffffffu, bad_index | coincident) ? 1 : 0;
        for (int k = 0; k < M && !singular; ++k) {
            // pivot: largest |a_ik|, i >= k, lowest i on ties
            unsigned long long best = 0;
            int bi = k;
            for (int i = k + lane; i < M; i += 32) {
                const unsigned long long b = abs_bits(A[(size_t)i * LD + k]);
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
                    const double t = A[(size_t)k * LD + j];
                    A[(size_t)k * LD + j] = A[(size_t)bi * LD + j];
                    A[(size_t)bi * LD + j] = t;
                }
            }
            __syncwarp();
            const double inv = __ddiv_rn(1.0, A[(size_t)k * LD + k]);
            for (int i = k + 1 + lane; i < M; i += 32) A[(size_t)i * LD + k] = __dmul_rn(A[(size_t)i * LD + k], inv);
            __syncwarp();
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
                    const double l0 = r0[0], l1 = r1[0], l2 = r2[0], l3 = r3[0];
                    const double u0 = prow[j0], u1 = prow[j1], u2 = prow[j2], u3 = prow[j3];
                    const double a0 = r0[1 + j0], a1 = r1[1 + j1], a2 = r2[1 + j2], a3 = r3[1 + j3];
                    r0[1 + j0] = fma(-l0, u0, a0);
                    r1[1 + j1] = fma(-l1, u1, a1);
                    r2[1 + j2] = fma(-l2, u2, a2);
                    r3[1 + j3] = fma(-l3, u3, a3);
                }
                for (; e < total; e += 32) {
                    double* r0 = A + (size_t)(k + 1 + ii) * LD + k;
                    r0[1 + jj] = fma(-r0[0], prow[jj], r0[1 + jj]);
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
                const double xj = __ddiv_rn(A[(size_t)j * LD + M], A[(size_t)j * LD + j]);
                __syncwarp();
                for (int i = lane; i < j; i += 32) A[(size_t)i * LD + M] = fma(-A[(size_t)i * LD + j], xj, A[(size_t)i * LD + M]);
                if (lane == 0) A[(size_t)j * LD + M] = xj;
                __syncwarp();
            }
        }

        // ---- scale back and store ------------------------------------------
        int bad = singular;
        double* wout = w + (int64_t)node * n;
        for (int j = lane; j < n; j += 32) {
            const double v = singular ? 0.0 : __ddiv_rn(A[(size_t)j * LD + M], delta2);
            if (!isfinite(v)) bad = 1;
            A[(size_t)j * LD + M] = v;
        }
        bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
        for (int j = lane; j < n; j += 32) wout[j] = bad ? 0.0 : A[(size_t)j * LD + M];
        if (node_status && lane == 0) node_status[node] = bad;
        __syncwarp();
    }
}

int weights_warps_per_block(const WeightsGeom& g, size_t* smem_bytes) {
    // one warp per block when a warp needs a lot of shared memory (m = 6),
    // four otherwise; the per-SM residency is then set by shared memory.
    const size_t per_warp = (size_t)g.smem_doubles * sizeof(double);
    int wpb = 4;
    while (wpb > 1 && per_warp * wpb > 227 * 1024) --wpb;
    *smem_bytes = per_warp * wpb;
    return wpb;
}

}  // namespace
}  // namespace rbffd

extern "C" int rbffd_weights(const double* xy, const int32_t* idx, int64_t N, int32_t n, int32_t m, double* w,
                             int32_t* node_status, void* stream) {
    using namespace rbffd;
    if (!xy || !idx || !w || N <= 0 || N > 0x7fffffffLL || n < 1 || n > RBFFD_MAX_STENCIL || m < 0 || m > 8)
        return RBFFD_ERR_INVALID_ARG;
    if (((uintptr_t)xy & 15) != 0) return RBFFD_ERR_INVALID_ARG;
    const int s = (m + 1) * (m + 2) / 2;
    if (n < s) return RBFFD_ERR_INVALID_ARG;
    WeightsGeom g = weights_geom(n, m);
    size_t smem = 0;
    const int wpb = weights_warps_per_block(g, &smem);
    if (smem > 227 * 1024) return RBFFD_ERR_INVALID_ARG;  // system too large for one SM
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBFFD_CUDA_TRY(cudaFuncSetAttribute(weights_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    RBFFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, weights_kernel, 32 * wpb, smem));
    if (per_sm < 1) return RBFFD_ERR_INVALID_ARG;
    const int64_t need = (N + wpb - 1) / wpb;
    const int blocks = (int)std::min<int64_t>(need, (int64_t)per_sm * sm_count());
    weights_kernel<<<blocks, 32 * wpb, smem, as_stream(stream)>>>(reinterpret_cast<const double2*>(xy), idx, (int)N, n,
                                                                  m, g.s, g.M, g.LD, g.coords_in_zero_block,
                                                                  g.smem_doubles, w, node_status);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}
