// Geometric multigrid preconditioner on RBF-FD node sets (sm_103a).
//
// The paper stops at an explicit time loop and names the implicit solve as
// the next step (Sec. VI); Jacobi-scaled BiCGSTAB on the RBF-FD Laplacian
// needs O(1/h) iterations (tens of thousands at 4M nodes).  This file builds
// a V-cycle whose every level is an RBF-FD discretisation of the same
// problem, made by this library's own stages:
//
//  * coarsening: the nodes of a level are binned on a uniform grid of side
//    c ~ 2x their mean spacing; each occupied cell keeps one node, a
//    Dirichlet node if the cell has one, else the node nearest the cell
//    centre (ties: lower index; one 64-bit atomicMin per node on the packed
//    key (interior?, d^2 to the centre, index), so the choice does not depend
//    on thread order).  c grows until at most half the nodes survive.
//    Survivors keep their relative order, so coarse indices inherit the
//    fine ordering's locality.
//  * coarse operator: stencils, Laplacian weights (PHS r^3 + monomials of
//    degree 2, n = 12) and the Dirichlet-row assembly of the fine problem,
//    rerun on the coarse nodes (rediscretisation; Sec. II Eq. 1, Sec. IV).
//  * prolongation P (ELL, 12 per row): PHS r^3 + degree-2 interpolation from
//    the 12 nearest coarse nodes; rows of Dirichlet nodes are zero (the
//    correction vanishes on the boundary).  Restriction R = (N_c / N_f) P^T
//    (a deterministic transpose), zero rows at coarse Dirichlet nodes.
//  * smoothing: nu damped Jacobi sweeps x += W (b - A x), W = Omega D^-1,
//    before and after the coarse correction.  The damping omega applies to
//    the interior rows; Dirichlet rows (identity rows of A, identity columns
//    of A^T) take omega = 1, so a cycle reproduces boundary data exactly.
//    With omega < 1 there, the Dirichlet values would come back off by
//    (1 - omega)^(2 nu), and the interior rows next to the boundary, whose
//    weights scale as 1/h^2, would turn that into a residual ~1/h^2 times
//    the data: at 1e6 nodes BiCGSTAB broke down in its first step on such
//    right-hand sides.  W is stored (per level, FP64 and float32) in place of
//    D^-1.  The coarsest level (<= 128 nodes) is
//    solved with its dense inverse (Gauss-Jordan with partial pivoting, one
//    block).
//
// A V-cycle is a fixed linear map (fixed sweeps, exact coarsest solve), so
// it can right-precondition BiCGSTAB.  It runs in FP64, or in float32 values
// and vectors (the mixed-precision solve: the preconditioner needs no FP64
// accuracy, the outer FP64 BiCGSTAB keeps the residual exact).
#include "common.cuh"
#include "internal.cuh"
#include "scan.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace rbffd {

static_assert(sizeof(MgHierarchy) <= sizeof(rbffd_mg), "rbffd_mg is too small for the hierarchy");

namespace {

constexpr int kT = 256;

// Rows of a CSR matrix, TPR lanes per row; every lane of a warp runs the same
// number of trips (warp-uniform loop), so full-mask shuffles are safe.
#define MG_ROWS(TPR, N, i, valid, ...)                                                 \
    {                                                                                  \
        const int64_t g0_ = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / (TPR); \
        const int64_t ng_ = ((int64_t)gridDim.x * blockDim.x) / (TPR);                \
        const int64_t off_ = (threadIdx.x & 31) / (TPR);                              \
        for (int64_t base_ = g0_ - off_; base_ < (N); base_ += ng_) {                 \
            const int64_t i = base_ + off_;                                           \
            const bool valid = i < (N);                                               \
            __VA_ARGS__                                                               \
        }                                                                             \
    }

#define MG_ELEMS(N, i) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (N); i += (int64_t)gridDim.x * blockDim.x)

template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c);
template <>
__device__ __forceinline__ double fmaT<double>(double a, double b, double c) {
    return fma(a, b, c);
}
template <>
__device__ __forceinline__ float fmaT<float>(float a, float b, float c) {
    return fmaf(a, b, c);
}

template <typename T, int TPR>
__device__ __forceinline__ T row_sum(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                     const T* __restrict__ val, const T* __restrict__ x, int64_t nx, int64_t row,
                                     int sub, bool valid) {
    (void)nx;  // length of x: bound of the checked build's tests
    int64_t a = 0, e = 0;
    if (valid) {
        a = __ldg(row_ptr + row);
        e = __ldg(row_ptr + row + 1);
    }
    T sum = T(0);
#pragma unroll 4
    for (int64_t k = a + sub; k < e; k += TPR) sum = fmaT<T>(__ldg(val + k), __ldg(&RB_AT(x, __ldg(col + k), nx)), sum);
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, TPR);
    return sum;
}

__device__ __forceinline__ bool stopped(const int* flag) { return flag && *(volatile const int*)flag != 0; }

// x = W b (the first sweep from x = 0); dinv holds W = Omega D^-1
template <typename T, typename BT>
__global__ void __launch_bounds__(kT) mg_first_kernel(int64_t N, const BT* __restrict__ b, const T* __restrict__ dinv,
                                                      T* __restrict__ x, const int* flag) {
    if (stopped(flag)) return;
    MG_ELEMS(N, i) x[i] = dinv[i] * (T)b[i];
}

// xo = xi + W (b - A xi)
template <typename T, typename BT, typename OT, int TPR>
__global__ void __launch_bounds__(kT) mg_jacobi_kernel(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                                       const T* __restrict__ val, int64_t N, const T* __restrict__ xi,
                                                       const BT* __restrict__ b, const T* __restrict__ dinv,
                                                       OT* __restrict__ xo, const int* flag) {
    if (stopped(flag)) return;
    const int sub = threadIdx.x & (TPR - 1);
    MG_ROWS(TPR, N, i, valid, {
        const T ax = row_sum<T, TPR>(row_ptr, col, val, xi, N, i, sub, valid);
        if (valid && sub == 0) xo[i] = (OT)fmaT<T>(dinv[i], (T)b[i] - ax, xi[i]);
    })
}

// r = b - A x
template <typename T, typename BT, int TPR>
__global__ void __launch_bounds__(kT) mg_resid_kernel(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                                      const T* __restrict__ val, int64_t N, const T* __restrict__ x,
                                                      const BT* __restrict__ b, T* __restrict__ r, const int* flag) {
    if (stopped(flag)) return;
    const int sub = threadIdx.x & (TPR - 1);
    MG_ROWS(TPR, N, i, valid, {
        const T ax = row_sum<T, TPR>(row_ptr, col, val, x, N, i, sub, valid);
        if (valid && sub == 0) r[i] = (T)b[i] - ax;
    })
}

// y = R r (restriction, CSR with n rows)
template <typename T, int TPR>
__global__ void __launch_bounds__(kT) mg_restrict_kernel(const int64_t* __restrict__ row_ptr,
                                                         const int* __restrict__ col, const T* __restrict__ val,
                                                         int64_t n, const T* __restrict__ r, int64_t nr,
                                                         T* __restrict__ y, const int* flag) {
    if (stopped(flag)) return;
    const int sub = threadIdx.x & (TPR - 1);
    MG_ROWS(TPR, n, i, valid, {
        const T v = row_sum<T, TPR>(row_ptr, col, val, r, nr, i, sub, valid);
        if (valid && sub == 0) y[i] = v;
    })
}

// x += P e (ELL, kMgK entries per row)
template <typename T>
__global__ void __launch_bounds__(kT) mg_prolong_kernel(int64_t N, const int32_t* __restrict__ pidx,
                                                        const T* __restrict__ pval, const T* __restrict__ e,
                                                        int64_t ne, T* __restrict__ x, const int* flag) {
    (void)ne;  // length of e: bound of the checked build's tests
    if (stopped(flag)) return;
    MG_ELEMS(N, i) {
        const int32_t* ip = pidx + i * kMgK;
        const T* vp = pval + i * kMgK;
        T acc = x[i];
#pragma unroll
        for (int j = 0; j < kMgK; ++j) acc = fmaT<T>(__ldg(vp + j), __ldg(&RB_AT(e, __ldg(ip + j), ne)), acc);
        x[i] = acc;
    }
}

// x = Minv b, one warp per row
template <typename T, typename BT, typename OT>
__global__ void __launch_bounds__(kT) mg_dense_kernel(int n, const T* __restrict__ minv, const BT* __restrict__ b,
                                                      OT* __restrict__ x, const int* flag) {
    if (stopped(flag)) return;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        T acc = T(0);
        for (int j = lane; j < n; j += 32) acc = fmaT<T>(minv[(int64_t)i * n + j], (T)b[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) x[i] = (OT)acc;
    }
}

// ------------------------------------------------------------------ setup --
struct MgBox {
    double mnx, mny, mxx, mxy;
};

__global__ void __launch_bounds__(kT) mg_bbox_kernel(const double2* __restrict__ xy, int64_t N, MgBox* out) {
    double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    MG_ELEMS(N, i) {
        const double2 p = xy[i];
        mnx = fmin(mnx, p.x);
        mny = fmin(mny, p.y);
        mxx = fmax(mxx, p.x);
        mxy = fmax(mxy, p.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fmin(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = fmin(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = fmax(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = fmax(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    __shared__ MgBox sh[kT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) RB_AT(sh, wid, kT / 32) = MgBox{mnx, mny, mxx, mxy};
    __syncthreads();
    if (threadIdx.x == 0) {
        MgBox r = sh[0];
        for (int k = 1; k < kT / 32; ++k) {
            r.mnx = fmin(r.mnx, sh[k].mnx);
            r.mny = fmin(r.mny, sh[k].mny);
            r.mxx = fmax(r.mxx, sh[k].mxx);
            r.mxy = fmax(r.mxy, sh[k].mxy);
        }
        out[blockIdx.x] = r;
    }
}

struct CellGrid {
    double x0, y0, inv_c;
    int gx, gy;
};

__device__ __forceinline__ int64_t cell_of(const CellGrid& g, double x, double y) {
    int cx = (int)floor((x - g.x0) * g.inv_c);
    int cy = (int)floor((y - g.y0) * g.inv_c);
    cx = cx < 0 ? 0 : (cx >= g.gx ? g.gx - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= g.gy ? g.gy - 1 : cy);
    return (int64_t)cy * g.gx + cx;
}

// Packed ranking key: bit 63 = interior node (Dirichlet nodes win), bits
// 62..31 = float32 bits of (d / c)^2 to the cell centre (non-negative, so
// monotone as an integer; < 2^31), bits 30..0 = node index.
__global__ void __launch_bounds__(kT) mg_mark_kernel(const double2* __restrict__ xy, const uint8_t* __restrict__ mask,
                                                     int64_t N, CellGrid g, unsigned long long* __restrict__ best) {
    MG_ELEMS(N, i) {
        const double2 p = xy[i];
        const int64_t c = cell_of(g, p.x, p.y);
        const int cx = (int)(c % g.gx), cy = (int)(c / g.gx);
        const double ux = (p.x - g.x0) * g.inv_c - (cx + 0.5);
        const double uy = (p.y - g.y0) * g.inv_c - (cy + 0.5);
        float d2 = (float)(ux * ux + uy * uy);
        if (!(d2 >= 0.f) || d2 > 1e30f) d2 = 1e30f;
        const unsigned long long key = ((unsigned long long)(mask[i] ? 0u : 1u) << 63) |
                                       ((unsigned long long)__float_as_uint(d2) << 31) | (unsigned long long)i;
        atomicMin(&RB_AT(best, c, (int64_t)g.gx * g.gy), key);
    }
}

__global__ void __launch_bounds__(kT) mg_select_kernel(const double2* __restrict__ xy, int64_t N, CellGrid g,
                                                       const unsigned long long* __restrict__ best,
                                                       int* __restrict__ sel) {
    MG_ELEMS(N, i) {
        const double2 p = xy[i];
        const int64_t c = cell_of(g, p.x, p.y);
        sel[i] = ((RB_AT(best, c, (int64_t)g.gx * g.gy) & 0x7fffffffull) == (unsigned long long)i) ? 1 : 0;
    }
}

struct SelLoad {
    const int* sel;
    __device__ int operator()(int64_t i) const { return sel[i]; }
};

__global__ void __launch_bounds__(kT) mg_gather_kernel(const double2* __restrict__ xy, const uint8_t* __restrict__ mask,
                                                       int64_t N, const int* __restrict__ sel,
                                                       const int* __restrict__ pos, int64_t Nc,
                                                       double2* __restrict__ cxy, uint8_t* __restrict__ cmask) {
    (void)Nc;  // coarse points: bound of the checked build's tests
    MG_ELEMS(N, i) {
        if (sel[i]) {
            const int k = pos[i];
            RB_AT(cxy, k, Nc) = xy[i];
            RB_AT(cmask, k, Nc) = mask[i] ? 1 : 0;
        }
    }
}

// D^-1 from the diagonal of a CSR matrix (1 where the diagonal is zero or
// missing); float copies of dinv and, if val32 != NULL, of the values.
// Dirichlet rows of level 0: y_b += W_b (r_b - (A y)_b), W_b = 1 / a_bb.
// Forward hierarchy (A's Dirichlet rows are identity rows): y_b = r_b, the
// starting guess that keeps every later residual zero on Dirichlet rows.
// Adjoint hierarchy (A^T: identity Dirichlet columns): the back substitution
// y_b = r_b - sum_i a_ib y_i over interior rows i.  In place: a Dirichlet
// row reads only interior entries of y and its own.
__global__ void __launch_bounds__(kT) mg_bfix_kernel(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                                     const double* __restrict__ val, int64_t N,
                                                     const uint8_t* __restrict__ mask, const double* __restrict__ w,
                                                     const double* __restrict__ r, double* y, const int* flag) {
    if (stopped(flag)) return;
    MG_ELEMS(N, i) {
        if (!mask[i]) continue;
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = fma(val[k], RB_AT(y, col[k], N), s);
        y[i] = fma(w[i], r[i] - s, y[i]);
    }
}

// W = Omega D^-1 of the smoother: omega / a_ii on interior rows, 1 / a_ii on
// Dirichlet rows.
__global__ void __launch_bounds__(kT) mg_diag_kernel(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                                     const double* __restrict__ val, int64_t N, int col_base,
                                                     const uint8_t* __restrict__ mask, double omega,
                                                     double* __restrict__ dinv, float* __restrict__ dinv32,
                                                     int* __restrict__ bad) {
    int nb = 0;
    MG_ELEMS(N, i) {
        double d = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col[k] - col_base == (int)i) d = val[k];
        const bool ok = d != 0.0 && isfinite(d);
        nb |= ok ? 0 : 1;
        const double iv = ok ? (mask[i] ? 1.0 : omega) / d : 1.0;
        dinv[i] = iv;
        dinv32[i] = __double2float_rn(iv);
    }
    if (nb) atomicOr(bad, 1);
}

// Interpolation rows: zero at Dirichlet nodes; where the interpolation
// system was singular (its nodes on one conic), the value of the nearest
// coarse node; float copy; CSR row pointer of the ELL layout.
__global__ void __launch_bounds__(kT) mg_pfix_kernel(int64_t N, const uint8_t* __restrict__ mask,
                                                     const int* __restrict__ pstat, double* __restrict__ pval,
                                                     float* __restrict__ pval32, int64_t* __restrict__ prow) {
    MG_ELEMS(N, i) {
        const bool dir = mask[i] != 0;
        const bool sing = pstat[i] != 0;
        for (int j = 0; j < kMgK; ++j) {
            const int64_t e = i * kMgK + j;
            const double v = dir ? 0.0 : (sing ? (j == 0 ? 1.0 : 0.0) : pval[e]);
            pval[e] = v;
            pval32[e] = __double2float_rn(v);
        }
        prow[i] = i * kMgK;
        if (i == N - 1) prow[N] = N * kMgK;
    }
}

// CSR row pointer of the ELL prolongation (kMgK entries per row).
__global__ void __launch_bounds__(kT) mg_ellrow_kernel(int64_t N, int64_t* __restrict__ prow) {
    MG_ELEMS(N + 1, i) prow[i] = i * kMgK;
}

// R = scale P^T with zero rows at coarse Dirichlet nodes; float copy.
__global__ void __launch_bounds__(kT) mg_rscale_kernel(const int64_t* __restrict__ rrow, int64_t Nc,
                                                       const uint8_t* __restrict__ cmask, double scale,
                                                       double* __restrict__ rval, float* __restrict__ rval32) {
    MG_ELEMS(Nc, c) {
        const double f = (cmask && cmask[c]) ? 0.0 : scale;
        for (int64_t k = rrow[c]; k < rrow[c + 1]; ++k) {
            const double v = rval[k] * f;
            rval[k] = v;
            rval32[k] = __double2float_rn(v);
        }
    }
}

// Adjoint hierarchy: prolongation R^T = scale P with the columns of coarse
// Dirichlet nodes zeroed (R zeroes their rows); float copy.
__global__ void __launch_bounds__(kT) mg_pscale_kernel(int64_t N, const int32_t* __restrict__ pidx,
                                                       const uint8_t* __restrict__ cmask, int64_t Nc, double scale,
                                                       double* __restrict__ pval, float* __restrict__ pval32) {
    const int64_t total = N * kMgK;
    MG_ELEMS(total, e) {
        (void)Nc;  // coarse points: bound of the checked build's tests
        const double v = RB_AT(cmask, pidx[e], Nc) ? 0.0 : scale * pval[e];
        pval[e] = v;
        pval32[e] = __double2float_rn(v);
    }
}

__global__ void __launch_bounds__(kT) mg_f32_kernel(const double* __restrict__ v, int64_t n, float* __restrict__ v32) {
    MG_ELEMS(n, i) v32[i] = __double2float_rn(v[i]);
}

// A singular stencil at an interior node (Dirichlet rows ignore weights).
__global__ void __launch_bounds__(kT) mg_count_kernel(const int* __restrict__ stat, const uint8_t* __restrict__ mask,
                                                      int64_t N, int* __restrict__ bad) {
    int nb = 0;
    MG_ELEMS(N, i) nb |= (stat[i] && !mask[i]) ? 1 : 0;
    if (nb) atomicOr(bad, 1);
}

// Dense [A | I] (n x 2n, row-major) from CSR.
__global__ void __launch_bounds__(kT) mg_dense_build_kernel(const int64_t* __restrict__ row_ptr,
                                                            const int* __restrict__ col,
                                                            const double* __restrict__ val, int n, int col_base,
                                                            double* __restrict__ aug) {
    const int64_t total = (int64_t)n * 2 * n;
    MG_ELEMS(total, e) aug[e] = 0.0;
    __syncthreads();  // (single block: the zero fill precedes the scatter)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int c = col[k] - col_base;
            if ((unsigned)c < (unsigned)n) aug[(int64_t)i * 2 * n + c] += val[k];
        }
        aug[(int64_t)i * 2 * n + n + i] = 1.0;
    }
}

// Gauss-Jordan inversion of [A | I] (n x 2n, row-major, n <= kMgCoarsest) by
// one block: for each column k, the pivot is the largest |a_ik|, i >= k
// (lowest i on ties); rows k and pivot are swapped, row k is scaled, and
// column k is eliminated from every other row with multipliers saved in
// shared memory first (the pivot row itself is not written in that phase).
// Sets *bad on a zero pivot.
constexpr int kGJ = 256;
__global__ void __launch_bounds__(kGJ) mg_gj_kernel(double* __restrict__ aug, int n, int* __restrict__ bad) {
    __shared__ double sv[kGJ];
    __shared__ int si[kGJ];
    __shared__ double f[kMgCoarsest];
    __shared__ int prow;
    __shared__ double piv;
    const int n2 = 2 * n;
    const int tid = threadIdx.x;
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += kGJ) {
            const double v = fabs(aug[(int64_t)i * n2 + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        sv[tid] = best;
        si[tid] = bi;
        __syncthreads();
        for (int o = kGJ / 2; o > 0; o >>= 1) {
            if (tid < o) {
                const double ov = sv[tid + o];
                const int oi = si[tid + o];
                if (ov > sv[tid] || (ov == sv[tid] && oi < si[tid])) {
                    sv[tid] = ov;
                    si[tid] = oi;
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            prow = si[0];
            if (!(sv[0] > 0.0) || prow >= n) {
                *bad = 1;
                prow = k;
            }
        }
        __syncthreads();
        const int p = prow;
        if (p != k)
            for (int j = tid; j < n2; j += kGJ) {
                const double t = aug[(int64_t)k * n2 + j];
                aug[(int64_t)k * n2 + j] = aug[(int64_t)p * n2 + j];
                aug[(int64_t)p * n2 + j] = t;
            }
        __syncthreads();
        if (tid == 0) {
            const double d = aug[(int64_t)k * n2 + k];
            piv = (d != 0.0) ? 1.0 / d : 0.0;
        }
        __syncthreads();
        for (int j = tid; j < n2; j += kGJ) aug[(int64_t)k * n2 + j] *= piv;
        for (int i = tid; i < n; i += kGJ) RB_AT(f, i, kMgCoarsest) = (i == k) ? 0.0 : aug[(int64_t)i * n2 + k];
        __syncthreads();
        const int64_t total = (int64_t)n * n2;
        for (int64_t e = tid; e < total; e += kGJ) {
            const int i = (int)(e / n2), j = (int)(e - (int64_t)i * n2);
            if (i != k) aug[e] = fma(-RB_AT(f, i, kMgCoarsest), aug[(int64_t)k * n2 + j], aug[e]);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kT) mg_dense_copy_kernel(const double* __restrict__ aug, int n,
                                                           double* __restrict__ minv, float* __restrict__ minv32) {
    const int64_t total = (int64_t)n * n;
    MG_ELEMS(total, e) {
        const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
        const double v = aug[(int64_t)i * 2 * n + n + j];
        minv[e] = v;
        minv32[e] = __double2float_rn(v);
    }
}

// ------------------------------------------------------------------- host --
// ---- Galerkin coarse operators (adjoint hierarchy) -------------------------
// A_{l+1} = R_l A_l P_l with R_l = P^T (the interpolation's transpose) and
// P_l = (N_c / N_f) P without the columns of coarse Dirichlet nodes; the rows
// of coarse Dirichlet nodes become identity rows (their columns are zero in
// the product, so the coarse system stays block diagonal).  One warp per
// coarse row c and two shared-memory hash tables (open addressing, linear
// probing, keys -1 when empty): first D = R_c A_l keyed by fine column, then
// the row C_c = D P_l keyed by coarse column.  Zero entries of R and P_l
// (Dirichlet rows of P, the removed columns) are skipped.  Every key's terms
// are summed in a fixed order (a batch is one A row, whose columns are
// distinct, or two P rows, one per half-warp, whose values go in one half
// after the other; batches run in sequence; D is sorted by column before its
// rows of P are read), and
// the row is sorted by column and staged at a place taken from an atomic
// counter; after a scan of the row lengths a second kernel copies each row
// to its CSR position.  The product therefore does not depend on thread
// timing.
// Two table sizes: (512, 256) slots first, four warps per block, 9 KB of
// tables per warp (24 warps per SM); a level whose rows overflow them is
// redone with (1024, 512), 18 KB per warp (12 warps per SM).
constexpr int kGalWarps = 4;
template <int H1, int H2>
constexpr size_t gal_smem_bytes() {
    return (size_t)kGalWarps * (H1 + H2) * (sizeof(int) + sizeof(double));
}

// Slot of `key` in a table of cap = mask + 1 slots (inserted if absent);
// -1 when the table is full.  *fresh is set when this call inserted it.
__device__ __forceinline__ int gal_slot(int* keys, unsigned mask, int key, int* fresh) {
    unsigned h = ((unsigned)key * 2654435761u) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int k = *(volatile int*)(keys + h);
        if (k == key) return (int)h;
        if (k == -1) {
            const int old = atomicCAS(keys + h, -1, key);
            if (old == -1) {
                *fresh = 1;
                return (int)h;
            }
            if (old == key) return (int)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Ascending sort of n <= cap (key, value) pairs held at the front of the
// arrays, by one warp (bitonic network over the next power of two, padded
// with INT_MAX keys).
__device__ __forceinline__ void gal_sort(int* keys, double* vals, int n, int cap, int lane) {
    (void)cap;  // table size: bound of the checked build's tests
    int m = 32;
    while (m < n) m <<= 1;
    for (int i = n + lane; i < m; i += 32) RB_AT(keys, i, cap) = 0x7fffffff;
    __syncwarp();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < m; i += 32) {
                const int p = i ^ j;
                if (p > i) {
                    const int a = RB_AT(keys, i, cap), b = RB_AT(keys, p, cap);
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        RB_AT(keys, i, cap) = b;
                        RB_AT(keys, p, cap) = a;
                        const double t = RB_AT(vals, i, cap);
                        RB_AT(vals, i, cap) = RB_AT(vals, p, cap);
                        RB_AT(vals, p, cap) = t;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Moves the occupied slots of a table (cap slots) to its front, in slot
// order; returns their count.  Every lane gets the count.
__device__ __forceinline__ int gal_compact(int* keys, double* vals, int cap, int lane, bool with_vals) {
    int n = 0;
    for (int base = 0; base < cap; base += 32) {
        const int i = base + lane;
        const int k = keys[i];
        const double v = with_vals ? vals[i] : 0.0;
        const unsigned occ = __ballot_sync(0xffffffffu, k != -1);
        __syncwarp();
        if (k != -1) {
            const int dst = n + __popc(occ & ((1u << lane) - 1u));
            RB_AT(keys, dst, cap) = k;
            if (with_vals) RB_AT(vals, dst, cap) = v;
        }
        n += __popc(occ);
        __syncwarp();
    }
    return n;
}

template <int kGalH1, int kGalH2>
__global__ void __launch_bounds__(kGalWarps * 32) mg_galerkin_kernel(
    int64_t Nc, const int64_t* __restrict__ rrow, const int32_t* __restrict__ rcol, const double* __restrict__ rval,
    const int64_t* __restrict__ arow, const int* __restrict__ acol, const double* __restrict__ aval,
    const int32_t* __restrict__ pidx, const double* __restrict__ pval, const uint8_t* __restrict__ cmask,
    int* __restrict__ count, int64_t* __restrict__ start, unsigned long long* __restrict__ total, int64_t cap,
    int* __restrict__ tcol, double* __restrict__ tval, int* __restrict__ bad, int64_t Nf, int64_t annz) {
    (void)Nf;  // fine points and A's entries: bounds of the checked build's tests
    (void)annz;
    extern __shared__ __align__(16) unsigned char gal_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* v1 = reinterpret_cast<double*>(gal_smem) + (size_t)wid * (kGalH1 + kGalH2);
    double* v2 = v1 + kGalH1;
    int* k1 = reinterpret_cast<int*>(reinterpret_cast<double*>(gal_smem) + (size_t)kGalWarps * (kGalH1 + kGalH2)) +
              (size_t)wid * (kGalH1 + kGalH2);
    int* k2 = k1 + kGalH1;
    (void)RB_SH(v2 + kGalH2 - 1);  // the warp's tables lie in the launch's shared memory
    (void)RB_SH(k2 + kGalH2 - 1);
    int overflow = 0;
    const int64_t nwarps = (int64_t)gridDim.x * kGalWarps;
    for (int64_t c = (int64_t)blockIdx.x * kGalWarps + wid; c < Nc; c += nwarps) {
        int m = 1;
        if (cmask[c]) {
            if (lane == 0) {  // an identity row
                k2[0] = (int)c;
                v2[0] = 1.0;
            }
        } else {
            for (int i = lane; i < kGalH1; i += 32) {
                k1[i] = -1;
                v1[i] = 0.0;
            }
            for (int i = lane; i < kGalH2; i += 32) {
                k2[i] = -1;
                v2[i] = 0.0;
            }
            __syncwarp();
            bool full = false;
            // D = R_c A_l: one row of A_l per batch of lanes.  The entries of
            // R's row and the extents of their A rows are loaded 32 at a time,
            // one per lane (independent loads), then handed out by shuffles,
            // and each A row's first batch is loaded before the previous
            // row's keys go into the table.
            const int64_t r0 = rrow[c], r1 = rrow[c + 1];
            for (int64_t e0 = r0; e0 < r1; e0 += 32) {
                double rv_l = 0.0;
                int64_t a0_l = 0, a1_l = 0;
                if (e0 + lane < r1) {
                    rv_l = rval[e0 + lane];
                    if (rv_l != 0.0) {
                        const int f = rcol[e0 + lane];
                        a0_l = RB_AT(arow, f, Nf + 1);
                        a1_l = RB_AT(arow, f + 1, Nf + 1);
                    }
                }
                const int cnt = (int)min((int64_t)32, r1 - e0);
                // the first batch of the first entry's A row
                int64_t a0 = __shfl_sync(0xffffffffu, a0_l, 0), a1 = __shfl_sync(0xffffffffu, a1_l, 0);
                int kc = (a0 + lane < a1) ? RB_AT(acol, a0 + lane, annz) : -1;
                double kv = (a0 + lane < a1) ? RB_AT(aval, a0 + lane, annz) : 0.0;
                for (int t = 0; t < cnt; ++t) {
                    const double rv = __shfl_sync(0xffffffffu, rv_l, t);
                    const int64_t b0 = a0, b1 = a1;
                    int cur_c = kc;
                    double cur_v = kv;
                    // the next entry's first batch, in flight while this row fills the table
                    if (t + 1 < cnt) {
                        a0 = __shfl_sync(0xffffffffu, a0_l, t + 1);
                        a1 = __shfl_sync(0xffffffffu, a1_l, t + 1);
                        kc = (a0 + lane < a1) ? RB_AT(acol, a0 + lane, annz) : -1;
                        kv = (a0 + lane < a1) ? RB_AT(aval, a0 + lane, annz) : 0.0;
                    }
                    if (rv == 0.0) continue;  // (warp-uniform: a Dirichlet row of P)
                    for (int64_t b = b0; b < b1; b += 32) {
                        const int64_t k = b + lane;
                        if (b > b0 && k < b1) {  // batches after the first (rows longer than 32)
                            cur_c = RB_AT(acol, k, annz);
                            cur_v = RB_AT(aval, k, annz);
                        }
                        if (k < b1) {
                            int fresh = 0;
                            const int sl = gal_slot(k1, kGalH1 - 1, cur_c, &fresh);
                            if (sl < 0) full = true;
                            else RB_AT(v1, sl, kGalH1) = fma(rv, cur_v, RB_AT(v1, sl, kGalH1));
                        }
                        __syncwarp();
                    }
                }
            }
            // D's entries at the front, sorted by column
            const int n1 = gal_compact(k1, v1, kGalH1, lane, true);
            gal_sort(k1, v1, n1, kGalH1, lane);
            // C_c = D P_l: two entries of D per batch, lanes 0-11 and 16-27;
            // the keys go in together, the values in D's order; the next
            // batch's row of P is loaded before this batch's keys go in
            const int half = lane >> 4, j = lane & 15;
            const bool jl = j < kMgK;
            int nxt_i = -1;
            double nxt_v = 0.0;
            if (half < n1 && jl) {
                const int64_t pe = (int64_t)RB_AT(k1, half, kGalH1) * kMgK + j;
                nxt_v = RB_AT(pval, pe, Nf * kMgK);
                nxt_i = RB_AT(pidx, pe, Nf * kMgK);
            }
            for (int i = 0; i < n1; i += 2) {
                const int di = i + half;
                const int pj = nxt_i;
                const double pv = nxt_v;
                if (di + 2 < n1 && jl) {
                    const int64_t pe = (int64_t)RB_AT(k1, di + 2, kGalH1) * kMgK + j;
                    nxt_v = RB_AT(pval, pe, Nf * kMgK);
                    nxt_i = RB_AT(pidx, pe, Nf * kMgK);
                }
                int sl = -1;
                double term = 0.0;
                if (di < n1 && jl && pv != 0.0) {
                    int fresh = 0;
                    sl = gal_slot(k2, kGalH2 - 1, pj, &fresh);
                    if (sl < 0) full = true;
                    term = RB_AT(v1, di, kGalH1) * pv;
                }
                __syncwarp();
                if (half == 0 && sl >= 0) RB_AT(v2, sl, kGalH2) += term;
                __syncwarp();
                if (half == 1 && sl >= 0) RB_AT(v2, sl, kGalH2) += term;
                __syncwarp();
            }
            if (__any_sync(0xffffffffu, full)) {
                overflow = 1;
                continue;
            }
            m = gal_compact(k2, v2, kGalH2, lane, true);
            gal_sort(k2, v2, m, kGalH2, lane);
        }
        // stage the row (any free place: the copy below puts rows in order)
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(total, (unsigned long long)m);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if ((int64_t)pos + m > cap) {
            overflow = 1;
            continue;
        }
        for (int i = lane; i < m; i += 32) {
            RB_AT(tcol, pos + i, cap) = RB_AT(k2, i, kGalH2);
            RB_AT(tval, pos + i, cap) = RB_AT(v2, i, kGalH2);
        }
        if (lane == 0) {
            count[c] = m;
            start[c] = (int64_t)pos;
        }
        __syncwarp();
    }
    if (overflow && lane == 0) atomicOr(bad, 2);
}

// The staged rows into the level's CSR (row c at crow[c]), with the float copy.
__global__ void __launch_bounds__(kT) mg_galerkin_place_kernel(int64_t Nc, const int64_t* __restrict__ start,
                                                               const int64_t* __restrict__ crow,
                                                               const int* __restrict__ tcol,
                                                               const double* __restrict__ tval,
                                                               int* __restrict__ ccol, double* __restrict__ cval,
                                                               float* __restrict__ cval32, int64_t tcap,
                                                               int64_t cnnz) {
    (void)tcap;  // staged and placed entries: bounds of the checked build's tests
    (void)cnnz;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < Nc; c += nw) {
        const int64_t o = crow[c], len = crow[c + 1] - o, s = start[c];
        RB_SPAN(s, len, tcap);
        RB_SPAN(o, len, cnnz);
        for (int64_t i = lane; i < len; i += 32) {
            const double v = RB_AT(tval, s + i, tcap);
            RB_AT(ccol, o + i, cnnz) = RB_AT(tcol, s + i, tcap);
            RB_AT(cval, o + i, cnnz) = v;
            RB_AT(cval32, o + i, cnnz) = __double2float_rn(v);
        }
    }
}

struct CountLoad64 {
    const int* c;
    __device__ int64_t operator()(int64_t i) const { return (int64_t)c[i]; }
};

int tpr_for(int64_t rows, int64_t nnz) {
    const double L = (double)nnz / (double)std::max<int64_t>(rows, 1);
    if (L >= 80) return 8;  // (Galerkin coarse operators)
    if (L >= 40) return 4;
    if (L >= 8) return 2;
    return 1;
}

int blocks_for(int64_t threads) {
    const int64_t b = (threads + kT - 1) / kT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 16));
}

// Upper bounds of the level sizes: each coarsening keeps at most half.
std::vector<int64_t> level_bounds(int64_t N) {
    std::vector<int64_t> nb{N};
    while (nb.back() > kMgCoarsest && (int)nb.size() < RBFFD_MG_MAX_LEVELS) nb.push_back(nb.back() / 2);
    return nb;
}

struct MgScratch {
    int64_t* a_row;  // adjoint hierarchy: the coarse operator before its transpose
    int32_t* a_col;
    double* a_val;
    unsigned long long* cells;
    int* sel;
    int* pos;
    int* sums;
    MgBox* box;
    int* flags;  // [0] singular / bad, [1] spare
    int* pstat;
    int32_t* sidx;   // coarse stencils
    double* sw;      // coarse weights
    int32_t* sstat;  // coarse weight status
    void* knn_ws;
    size_t knn_bytes;
    void* asm_ws;
    size_t asm_bytes;
    void* tr_ws;
    size_t tr_bytes;
    double* aug;
    int64_t* prow;
    int64_t* sums64;  // tile sums of 64-bit scans
    // Galerkin products: rows staged before their CSR placement (capacity
    // gal_cap entries), per-row staging offsets, the staging counter
    int* gal_col;
    double* gal_val;
    int64_t* gal_start;
    unsigned long long* gal_total;
    int64_t gal_cap;
};

constexpr int kBoxParts = 64;

// Carves the workspace; with ws == NULL only sizes it.  Levels: the given
// sizes (a built hierarchy's), else the upper bounds of level_bounds; the
// operators of levels >= 1 hold `cap` entries per row.
size_t mg_layout(void* ws, int64_t N, MgHierarchy* h, MgScratch* s, const std::vector<int64_t>* sizes = nullptr,
                 int cap = kMgCoarseN) {
    const std::vector<int64_t> nb = sizes ? *sizes : level_bounds(N);
    Carver c(ws);
    MgScratch t{};
    size_t knn_b = 0, asm_b = 0, tr_b = 0;
    for (size_t l = 0; l < nb.size(); ++l) {
        knn_b = std::max(knn_b, rbffd_stencils_workspace_size(std::max<int64_t>(nb[l], kMgCoarseN), kMgCoarseN));
        asm_b = std::max(asm_b, rbffd_assemble_workspace_size(nb[l]));
        tr_b = std::max(tr_b, rbffd_transpose_workspace_size(nb[l]));
    }
    {
        const int64_t n1b = nb.size() > 1 ? nb[1] : 1;
        t.a_row = c.take<int64_t>(n1b + 1);
        t.a_col = c.take<int32_t>((size_t)n1b * kMgCoarseN);
        t.a_val = c.take<double>((size_t)n1b * kMgCoarseN);
    }
    t.cells = c.take<unsigned long long>((size_t)(2 * N + 16));
    t.sel = c.take<int>(N);
    t.pos = c.take<int>(N + 1);
    t.sums = c.take<int>(scan_tiles(N) + 1);
    t.box = c.take<MgBox>(kBoxParts);
    t.flags = c.take<int>(64);
    t.pstat = c.take<int>(N);
    t.prow = c.take<int64_t>(N + 1);
    const int64_t n1 = nb.size() > 1 ? nb[1] : 1;
    t.sidx = c.take<int32_t>((size_t)n1 * kMgCoarseN);
    t.sw = c.take<double>((size_t)n1 * kMgCoarseN);
    t.sstat = c.take<int32_t>(n1);
    t.knn_ws = c.take<char>(knn_b);
    t.knn_bytes = knn_b;
    t.asm_ws = c.take<char>(asm_b);
    t.asm_bytes = asm_b;
    t.tr_ws = c.take<char>(tr_b);
    t.tr_bytes = tr_b;
    t.aug = c.take<double>((size_t)kMgCoarsest * 2 * kMgCoarsest);
    t.sums64 = c.take<int64_t>(scan_tiles(N) + 1);
    if (cap > kMgCoarseN && nb.size() > 1) {
        t.gal_cap = nb[1] * (int64_t)cap;
        t.gal_col = c.take<int>((size_t)t.gal_cap);
        t.gal_val = c.take<double>((size_t)t.gal_cap);
        t.gal_start = c.take<int64_t>(nb[1]);
        t.gal_total = c.take<unsigned long long>(1);
    }
    MgHierarchy hh{};
    for (size_t l = 0; l < nb.size(); ++l) {
        const int64_t n = nb[l];
        MgLevel& L = hh.lv[l];
        if (l > 0) {
            double* xy = c.take<double>((size_t)2 * n);
            L.xy = xy;
            uint8_t* mk = c.take<uint8_t>(n);
            L.mask = mk;
            int64_t* rp = c.take<int64_t>(n + 1);
            L.row_ptr = rp;
            int* cl = c.take<int>((size_t)n * cap);
            L.col = cl;
            double* v = c.take<double>((size_t)n * cap);
            L.val = v;
            float* v32 = c.take<float>((size_t)n * cap);
            L.val32 = v32;
        }
        L.dinv = c.take<double>(n);
        L.dinv32 = c.take<float>(n);
        L.x = c.take<double>(n);
        L.t = c.take<double>(n);
        L.r = c.take<double>(n);
        L.b = c.take<double>(n);
        L.x32 = c.take<float>(n);
        L.t32 = c.take<float>(n);
        L.r32 = c.take<float>(n);
        L.b32 = c.take<float>(n);
        if (l + 1 < nb.size()) {
            L.pidx = c.take<int32_t>((size_t)n * kMgK);
            L.pval = c.take<double>((size_t)n * kMgK);
            L.pval32 = c.take<float>((size_t)n * kMgK);
            L.rrow = c.take<int64_t>(n + 1);
            L.rcol = c.take<int32_t>((size_t)n * kMgK);
            L.rval = c.take<double>((size_t)n * kMgK);
            L.rval32 = c.take<float>((size_t)n * kMgK);
        }
    }
    // the dense inverse goes with whichever level ends up coarsest
    double* minv = c.take<double>((size_t)kMgCoarsest * kMgCoarsest);
    float* minv32 = c.take<float>((size_t)kMgCoarsest * kMgCoarsest);
    for (size_t l = 0; l < nb.size(); ++l) {
        hh.lv[l].minv = minv;
        hh.lv[l].minv32 = minv32;
    }
    if (h) *h = hh;
    if (s) *s = t;
    return c.off;
}

// Selects the coarse nodes of level l into level l + 1; returns their count
// in *nc.
int coarsen(const MgLevel& L, MgLevel& C, const MgScratch& s, cudaStream_t st, int64_t* nc) {
    const int64_t N = L.N;
    const double2* xy = reinterpret_cast<const double2*>(L.xy);
    mg_bbox_kernel<<<kBoxParts, kT, 0, st>>>(xy, N, s.box);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    MgBox parts[kBoxParts];
    RBFFD_CUDA_TRY(cudaMemcpyAsync(parts, s.box, sizeof(parts), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    MgBox bx = parts[0];
    for (int k = 1; k < kBoxParts; ++k) {
        bx.mnx = std::min(bx.mnx, parts[k].mnx);
        bx.mny = std::min(bx.mny, parts[k].mny);
        bx.mxx = std::max(bx.mxx, parts[k].mxx);
        bx.mxy = std::max(bx.mxy, parts[k].mxy);
    }
    const double W = bx.mxx - bx.mnx, H = bx.mxy - bx.mny;
    if (!(std::isfinite(W) && std::isfinite(H)) || !(W > 0.0 || H > 0.0)) return RBFFD_ERR_INVALID_ARG;
    double c = (W > 0.0 && H > 0.0) ? 2.0 * std::sqrt(W * H / (double)N) : 2.0 * std::max(W, H) / (double)N;
    for (int attempt = 0; attempt < 200; ++attempt, c *= 1.25) {
        CellGrid g;
        g.x0 = bx.mnx;
        g.y0 = bx.mny;
        g.inv_c = 1.0 / c;
        const double gx = std::floor(W / c) + 1.0, gy = std::floor(H / c) + 1.0;
        if (gx * gy > (double)(2 * N + 16)) continue;
        g.gx = (int)gx;
        g.gy = (int)gy;
        const int64_t cells = (int64_t)g.gx * g.gy;
        RBFFD_CUDA_TRY(cudaMemsetAsync(s.cells, 0xff, sizeof(unsigned long long) * cells, st));
        mg_mark_kernel<<<blocks_for(N), kT, 0, st>>>(xy, L.mask, N, g, s.cells);
        mg_select_kernel<<<blocks_for(N), kT, 0, st>>>(xy, N, g, s.cells, s.sel);
        note_launches(2);
        RBFFD_LAUNCH_CHECK();
        RBFFD_CUDA_TRY(exclusive_scan<int>(SelLoad{s.sel}, N, s.pos, s.sums, s.pos + N, st));
        int cnt = 0;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(&cnt, s.pos + N, sizeof(int), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        if ((int64_t)cnt > N / 2) continue;
        if (cnt <= kMgK) return RBFFD_ERR_INVALID_ARG;  // degenerate node set
        mg_gather_kernel<<<blocks_for(N), kT, 0, st>>>(xy, L.mask, N, s.sel, s.pos, (int64_t)cnt,
                                                       reinterpret_cast<double2*>(const_cast<double*>(C.xy)),
                                                       const_cast<uint8_t*>(C.mask));
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        *nc = cnt;
        return RBFFD_OK;
    }
    return RBFFD_ERR_INVALID_ARG;
}

int dense_inverse(const MgLevel& L, int col_base, const MgScratch& s, cudaStream_t st) {
    const int n = (int)L.N;
    mg_dense_build_kernel<<<1, kT, 0, st>>>(L.row_ptr, L.col, L.val, n, col_base, s.aug);
    mg_gj_kernel<<<1, kGJ, 0, st>>>(s.aug, n, s.flags);
    note_launches(2);
    mg_dense_copy_kernel<<<blocks_for((int64_t)n * n), kT, 0, st>>>(s.aug, n, L.minv, L.minv32);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

// ---- V-cycle ----------------------------------------------------------------
template <typename T>
struct Sel;
template <>
struct Sel<double> {
    static const double* val(const MgLevel& L) { return L.val; }
    static const double* dinv(const MgLevel& L) { return L.dinv; }
    static const double* pval(const MgLevel& L) { return L.pval; }
    static const double* rval(const MgLevel& L) { return L.rval; }
    static const double* minv(const MgLevel& L) { return L.minv; }
    static double* x(const MgLevel& L) { return L.x; }
    static double* t(const MgLevel& L) { return L.t; }
    static double* r(const MgLevel& L) { return L.r; }
    static double* b(const MgLevel& L) { return L.b; }
};
template <>
struct Sel<float> {
    static const float* val(const MgLevel& L) { return L.val32; }
    static const float* dinv(const MgLevel& L) { return L.dinv32; }
    static const float* pval(const MgLevel& L) { return L.pval32; }
    static const float* rval(const MgLevel& L) { return L.rval32; }
    static const float* minv(const MgLevel& L) { return L.minv32; }
    static float* x(const MgLevel& L) { return L.x32; }
    static float* t(const MgLevel& L) { return L.t32; }
    static float* r(const MgLevel& L) { return L.r32; }
    static float* b(const MgLevel& L) { return L.b32; }
};

template <typename T, typename BT, typename OT>
void jacobi(const MgLevel& L, const T* xi, const BT* b, OT* xo, const int* flag, cudaStream_t st) {
    const int g = blocks_for(L.N * L.tpr);
    const T* val = Sel<T>::val(L);
    const T* dinv = Sel<T>::dinv(L);
    switch (L.tpr) {
        case 8: mg_jacobi_kernel<T, BT, OT, 8><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, xi, b, dinv, xo, flag); break;
        case 4: mg_jacobi_kernel<T, BT, OT, 4><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, xi, b, dinv, xo, flag); break;
        case 2: mg_jacobi_kernel<T, BT, OT, 2><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, xi, b, dinv, xo, flag); break;
        default: mg_jacobi_kernel<T, BT, OT, 1><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, xi, b, dinv, xo, flag); break;
    }
}

template <typename T, typename BT>
void resid(const MgLevel& L, const T* x, const BT* b, T* r, const int* flag, cudaStream_t st) {
    const int g = blocks_for(L.N * L.tpr);
    const T* val = Sel<T>::val(L);
    switch (L.tpr) {
        case 8: mg_resid_kernel<T, BT, 8><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, x, b, r, flag); break;
        case 4: mg_resid_kernel<T, BT, 4><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, x, b, r, flag); break;
        case 2: mg_resid_kernel<T, BT, 2><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, x, b, r, flag); break;
        default: mg_resid_kernel<T, BT, 1><<<g, kT, 0, st>>>(L.row_ptr, L.col, val, L.N, x, b, r, flag); break;
    }
}

template <typename T>
void restrict_to(const MgLevel& L, int64_t nc, const T* r, T* bc, const int* flag, cudaStream_t st) {
    const int g = blocks_for(nc * L.rtpr);
    const T* val = Sel<T>::rval(L);
    switch (L.rtpr) {
        case 8: mg_restrict_kernel<T, 8><<<g, kT, 0, st>>>(L.rrow, L.rcol, val, nc, r, L.N, bc, flag); break;
        case 4: mg_restrict_kernel<T, 4><<<g, kT, 0, st>>>(L.rrow, L.rcol, val, nc, r, L.N, bc, flag); break;
        case 2: mg_restrict_kernel<T, 2><<<g, kT, 0, st>>>(L.rrow, L.rcol, val, nc, r, L.N, bc, flag); break;
        default: mg_restrict_kernel<T, 1><<<g, kT, 0, st>>>(L.rrow, L.rcol, val, nc, r, L.N, bc, flag); break;
    }
}

// One level of the cycle: b (BT) in, result in x (OT) for level 0, in the
// level's own current-iterate buffer otherwise (returned).
template <typename T>
T* cycle_level(const MgHierarchy& h, int l, const void* bin, bool b_is_double, double* out, const int* flag,
               cudaStream_t st, int* launches, std::vector<int>* ev) {
    const MgLevel& L = h.lv[l];
    const bool last_level = (l == h.n_levels - 1);
    const bool top = (l == 0);
    T* cur = Sel<T>::x(L);
    T* oth = Sel<T>::t(L);
    auto launch_first = [&](T* x) {
        const int g = blocks_for(L.N);
        if (b_is_double)
            mg_first_kernel<T, double><<<g, kT, 0, st>>>(L.N, static_cast<const double*>(bin), Sel<T>::dinv(L), x, flag);
        else
            mg_first_kernel<T, T><<<g, kT, 0, st>>>(L.N, static_cast<const T*>(bin), Sel<T>::dinv(L), x, flag);
        ++*launches;
    };
    auto sweep = [&](T* xi, T* xo, double* xo64) {
        // finest-level sweeps are timed when profiling (algorithmic bytes:
        // matrix, row pointers, iterate once, rhs, D^-1, result)
        const int e = (top && ev) ? prof_begin(st) : -1;
        if (b_is_double) {
            const double* b = static_cast<const double*>(bin);
            if (xo64) jacobi<T, double, double>(L, xi, b, xo64, flag, st);
            else jacobi<T, double, T>(L, xi, b, xo, flag, st);
        } else {
            const T* b = static_cast<const T*>(bin);
            if (xo64) jacobi<T, T, double>(L, xi, b, xo64, flag, st);
            else jacobi<T, T, T>(L, xi, b, xo, flag, st);
        }
        if (top && ev) {
            const int64_t bytes = L.nnz * (int64_t)(sizeof(T) + 4) + 8 * (L.N + 1) +
                                  L.N * (int64_t)(2 * sizeof(T) + (b_is_double ? 8 : sizeof(T)) + sizeof(T)) +
                                  (xo64 ? L.N * (int64_t)(8 - sizeof(T)) : 0);
            prof_end(e, st, kProfMg, bytes);
            ev->push_back(e);
        }
        ++*launches;
    };
    if (last_level) {
        const int g = blocks_for((int64_t)L.N * 32);
        const T* mv = Sel<T>::minv(L);
        if (top) {
            mg_dense_kernel<T, double, double><<<g, kT, 0, st>>>((int)L.N, mv, static_cast<const double*>(bin), out, flag);
        } else {
            mg_dense_kernel<T, T, T><<<g, kT, 0, st>>>((int)L.N, mv, static_cast<const T*>(bin), cur, flag);
        }
        ++*launches;
        return cur;
    }
    // pre-smoothing
    launch_first(cur);
    for (int k = 1; k < h.nu; ++k) {
        sweep(cur, oth, nullptr);
        std::swap(cur, oth);
    }
    // residual, restriction, coarse correction
    if (b_is_double) resid<T, double>(L, cur, static_cast<const double*>(bin), Sel<T>::r(L), flag, st);
    else resid<T, T>(L, cur, static_cast<const T*>(bin), Sel<T>::r(L), flag, st);
    const MgLevel& C = h.lv[l + 1];
    restrict_to<T>(L, C.N, Sel<T>::r(L), Sel<T>::b(C), flag, st);
    *launches += 2;
    T* e = cycle_level<T>(h, l + 1, Sel<T>::b(C), false, nullptr, flag, st, launches, ev);
    mg_prolong_kernel<T><<<blocks_for(L.N), kT, 0, st>>>(L.N, L.pidx, Sel<T>::pval(L), e, C.N, cur, flag);
    ++*launches;
    // post-smoothing; the last sweep of level 0 writes the FP64 output
    for (int k = 0; k < h.nu; ++k) {
        const bool final_top = top && k == h.nu - 1;
        sweep(cur, oth, final_top ? out : nullptr);
        if (!final_top) std::swap(cur, oth);
    }
    return cur;
}

}  // namespace

size_t mg_multi_coarse_floats(const MgHierarchy* h, int R) {
    if (!h) return 0;
    size_t t = 0;
    for (int l = 1; l < h->n_levels; ++l) t += (size_t)4 * h->lv[l].N * R;
    return t;
}

const MgHierarchy* mg_hierarchy(const rbffd_mg* h) {
    if (!h) return nullptr;
    const MgHierarchy* m = reinterpret_cast<const MgHierarchy*>(h);
    if (m->magic != kMgMagic || m->n_levels < 1) return nullptr;
    return m;
}

int64_t mg_fine_rows(const MgHierarchy* h) { return h ? h->lv[0].N : 0; }

bool mg_has_fp32(const MgHierarchy* h) { return h && h->has32; }

bool mg_is_transposed(const MgHierarchy* h) { return h && h->transposed; }

bool mg_is_galerkin(const MgHierarchy* h) { return h && h->galerkin; }

int mg_dirichlet_fix(const MgHierarchy* h, const double* r, double* y, const int* flag, cudaStream_t st) {
    if (!h || !r || !y || h->col_base != 0) return RBFFD_ERR_INVALID_ARG;
    const MgLevel& L = h->lv[0];
    mg_bfix_kernel<<<blocks_for(L.N), kT, 0, st>>>(L.row_ptr, L.col, L.val, L.N, L.mask, L.dinv, r, y, flag);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

__global__ void __launch_bounds__(kT) mg_zero_dirichlet_kernel(int64_t N, const uint8_t* __restrict__ mask,
                                                               double* __restrict__ y, const int* flag) {
    if (stopped(flag)) return;
    MG_ELEMS(N, i) if (mask[i]) y[i] = 0.0;
}

int mg_apply_interior(const MgHierarchy* h, bool fp32, const double* b, double* x, const int* flag, cudaStream_t st,
                      std::vector<int>* ev) {
    if (!h || !b || !x || h->col_base != 0) return RBFFD_ERR_INVALID_ARG;
    if (fp32 && !h->has32) return RBFFD_ERR_INVALID_ARG;
    int launches = 0;
    if (fp32) cycle_level<float>(*h, 0, b, true, x, flag, st, &launches, ev);
    else cycle_level<double>(*h, 0, b, true, x, flag, st, &launches, ev);
    const MgLevel& L = h->lv[0];
    mg_zero_dirichlet_kernel<<<blocks_for(L.N), kT, 0, st>>>(L.N, L.mask, x, flag);
    note_launches(launches + 1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

int mg_apply(const MgHierarchy* h, bool fp32, const double* b, double* x, const int* flag, cudaStream_t st,
             std::vector<int>* ev) {
    if (!h || !b || !x || h->col_base != 0) return RBFFD_ERR_INVALID_ARG;
    if (fp32 && !h->has32) return RBFFD_ERR_INVALID_ARG;
    int launches = 0;
    if (fp32) cycle_level<float>(*h, 0, b, true, x, flag, st, &launches, ev);
    else cycle_level<double>(*h, 0, b, true, x, flag, st, &launches, ev);
    note_launches(launches);
    RBFFD_LAUNCH_CHECK();
    // adjoint: the transpose of the boundary-eliminated forward cycle
    // E_b + B (I - A E_b) is B^T followed by the Dirichlet back substitution
    if (h->transposed) return mg_dirichlet_fix(h, b, x, flag, st);
    return RBFFD_OK;
}

}  // namespace rbffd

// ---------------------------------------------------------------- C ABI -----
extern "C" size_t rbffd_mg_workspace_size(int64_t N, int64_t nnz) {
    RBFFD_NVTX("rbffd_mg_workspace_size");
    (void)nnz;  // the fine matrix stays the caller's
    if (N <= 0 || N > 0x7fffffffLL) return 0;
    return rbffd::mg_layout(nullptr, N, nullptr, nullptr);
}

extern "C" int rbffd_mg_levels(const rbffd_mg* mg, int64_t* n_nodes) {
    RBFFD_NVTX("rbffd_mg_levels");
    const rbffd::MgHierarchy* h = rbffd::mg_hierarchy(mg);
    if (!h) return 0;
    if (n_nodes)
        for (int l = 0; l < RBFFD_MG_MAX_LEVELS; ++l) n_nodes[l] = l < h->n_levels ? h->lv[l].N : 0;
    return h->n_levels;
}

extern "C" int rbffd_mg_level(const rbffd_mg* mg, int32_t level, rbffd_mg_level_info* out) {
    RBFFD_NVTX("rbffd_mg_level");
    using namespace rbffd;
    if (!mg || !out) return RBFFD_ERR_INVALID_ARG;
    MgHierarchy h;
    std::memcpy(&h, mg, sizeof(h));
    if (h.magic != kMgMagic || level < 0 || level >= h.n_levels) return RBFFD_ERR_INVALID_ARG;
    const MgLevel& L = h.lv[level];
    const bool coarsest = level == h.n_levels - 1;
    std::memset(out, 0, sizeof(*out));
    out->n_nodes = L.N;
    out->xy = L.xy;
    out->is_dirichlet = L.mask;
    out->A.n_rows = L.N;
    out->A.nnz = L.nnz;
    out->A.row_ptr = L.row_ptr;
    out->A.col = L.col;
    out->A.val = L.val;
    out->A.dtype = 0;
    out->w = L.dinv;
    out->p_idx = coarsest ? nullptr : L.pidx;
    out->p_val = coarsest ? nullptr : L.pval;
    out->p_k = coarsest ? 0 : kMgK;
    out->minv = coarsest ? L.minv : nullptr;
    return RBFFD_OK;
}

extern "C" int rbffd_mg_adjoint_of(const rbffd_mg* fwd, const rbffd_csr* AT, const rbffd_csr* AT32, rbffd_mg* mg,
                                   void* ws, size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_mg_adjoint_of");
    using namespace rbffd;
    if (!mg) return RBFFD_ERR_INVALID_ARG;
    std::memset(mg, 0, sizeof(*mg));
    const MgHierarchy* F = mg_hierarchy(fwd);
    if (!F || !AT || !AT->row_ptr || !AT->col || !AT->val || AT->dtype != 0) return RBFFD_ERR_INVALID_ARG;
    if (AT32 && (!AT32->val || AT32->dtype != 1 || AT32->n_rows != AT->n_rows || AT32->nnz != AT->nnz ||
                 AT32->row_ptr != AT->row_ptr || AT32->col != AT->col))
        return RBFFD_ERR_INVALID_ARG;
    return mg_adjoint_of(*F, AT, AT32 ? static_cast<const float*>(AT32->val) : nullptr, mg, ws, ws_bytes,
                         as_stream(stream));
}

extern "C" size_t rbffd_mg_galerkin_workspace_size(const rbffd_mg* fwd) {
    RBFFD_NVTX("rbffd_mg_galerkin_workspace_size");
    using namespace rbffd;
    const MgHierarchy* F = mg_hierarchy(fwd);
    if (!F || F->transposed) return 0;
    return mg_galerkin_workspace(*F);
}

extern "C" int rbffd_mg_galerkin_adjoint(const rbffd_mg* fwd, const rbffd_csr* AT, const rbffd_csr* AT32,
                                         rbffd_mg* mg, void* ws, size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_mg_galerkin_adjoint");
    using namespace rbffd;
    if (!mg) return RBFFD_ERR_INVALID_ARG;
    std::memset(mg, 0, sizeof(*mg));
    const MgHierarchy* F = mg_hierarchy(fwd);
    if (!F || !AT || !AT->row_ptr || !AT->col || !AT->val || AT->dtype != 0) return RBFFD_ERR_INVALID_ARG;
    if (AT32 && (!AT32->val || AT32->dtype != 1 || AT32->n_rows != AT->n_rows || AT32->nnz != AT->nnz ||
                 AT32->row_ptr != AT->row_ptr || AT32->col != AT->col))
        return RBFFD_ERR_INVALID_ARG;
    return mg_galerkin_adjoint(*F, AT, AT32 ? static_cast<const float*>(AT32->val) : nullptr, mg, ws, ws_bytes,
                               as_stream(stream));
}

extern "C" int rbffd_mg_apply(const rbffd_mg* mg, int32_t fp32, const double* b, double* x, void* stream) {
    RBFFD_NVTX("rbffd_mg_apply");
    using namespace rbffd;
    const MgHierarchy* h = mg_hierarchy(mg);
    if (!h || !b || !x || b == x) return RBFFD_ERR_INVALID_ARG;
    return mg_apply(h, fp32 != 0, b, x, nullptr, as_stream(stream));
}

extern "C" int rbffd_mg_setup(const double* xy, const uint8_t* is_dirichlet, int64_t N, const rbffd_csr* A,
                              const rbffd_csr* A32, int32_t nu, double omega, rbffd_mg* mg, void* ws,
                              size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_mg_setup");
    using namespace rbffd;
    if (!mg) return RBFFD_ERR_INVALID_ARG;
    std::memset(mg, 0, sizeof(*mg));
    if (!xy || !is_dirichlet || !A || !A->row_ptr || !A->col || !A->val || A->dtype != 0 || N <= 0 ||
        N > 0x7fffffffLL || A->n_rows != N || A->nnz <= 0)
        return RBFFD_ERR_INVALID_ARG;
    if (A32 && (!A32->val || A32->dtype != 1 || A32->n_rows != N || A32->nnz != A->nnz || A32->row_ptr != A->row_ptr ||
                A32->col != A->col))
        return RBFFD_ERR_INVALID_ARG;
    return mg_setup_core(xy, is_dirichlet, N, A->row_ptr, A->col, static_cast<const double*>(A->val),
                         A32 ? static_cast<const float*>(A32->val) : nullptr, A->nnz, 0, nu, omega, mg, ws, ws_bytes,
                         as_stream(stream), false);
}

extern "C" int rbffd_mg_setup_geometry(const double* xy, const uint8_t* is_dirichlet, int64_t N, int32_t nu,
                                       double omega, rbffd_mg* mg, void* ws, size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_mg_setup_geometry");
    using namespace rbffd;
    if (!mg) return RBFFD_ERR_INVALID_ARG;
    std::memset(mg, 0, sizeof(*mg));
    if (!xy || !is_dirichlet || N <= 0 || N > 0x7fffffffLL) return RBFFD_ERR_INVALID_ARG;
    return mg_setup_geometry(xy, is_dirichlet, N, 0, nu, omega, mg, ws, ws_bytes, as_stream(stream), false);
}

extern "C" int rbffd_mg_setup_operator(rbffd_mg* mg, const rbffd_csr* A, const rbffd_csr* A32, void* stream) {
    RBFFD_NVTX("rbffd_mg_setup_operator");
    using namespace rbffd;
    if (!mg) return RBFFD_ERR_INVALID_ARG;
    const MgHierarchy* g = reinterpret_cast<const MgHierarchy*>(mg);
    if (g->magic != kMgGeometryMagic || g->transposed) return RBFFD_ERR_INVALID_ARG;
    const int64_t N = g->lv[0].N;
    if (!A || !A->row_ptr || !A->col || !A->val || A->dtype != 0 || A->n_rows != N || A->nnz <= 0)
        return RBFFD_ERR_INVALID_ARG;
    if (A32 && (!A32->val || A32->dtype != 1 || A32->n_rows != N || A32->nnz != A->nnz || A32->row_ptr != A->row_ptr ||
                A32->col != A->col))
        return RBFFD_ERR_INVALID_ARG;
    return mg_setup_operator(mg, A->row_ptr, A->col, static_cast<const double*>(A->val),
                             A32 ? static_cast<const float*>(A32->val) : nullptr, A->nnz, as_stream(stream));
}

extern "C" int rbffd_mg_setup_adjoint(const double* xy, const uint8_t* is_dirichlet, int64_t N, const rbffd_csr* AT,
                                      const rbffd_csr* AT32, int32_t nu, double omega, rbffd_mg* mg, void* ws,
                                      size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_mg_setup_adjoint");
    using namespace rbffd;
    if (!mg) return RBFFD_ERR_INVALID_ARG;
    std::memset(mg, 0, sizeof(*mg));
    if (!xy || !is_dirichlet || !AT || !AT->row_ptr || !AT->col || !AT->val || AT->dtype != 0 || N <= 0 ||
        N > 0x7fffffffLL || AT->n_rows != N || AT->nnz <= 0)
        return RBFFD_ERR_INVALID_ARG;
    if (AT32 && (!AT32->val || AT32->dtype != 1 || AT32->n_rows != N || AT32->nnz != AT->nnz ||
                 AT32->row_ptr != AT->row_ptr || AT32->col != AT->col))
        return RBFFD_ERR_INVALID_ARG;
    return mg_setup_core(xy, is_dirichlet, N, AT->row_ptr, AT->col, static_cast<const double*>(AT->val),
                         AT32 ? static_cast<const float*>(AT32->val) : nullptr, AT->nnz, 0, nu, omega, mg, ws,
                         ws_bytes, as_stream(stream), true);
}

// The adjoint hierarchy of a built forward one: the coarse node sets, the
// smoother weights and the interpolation are the forward ones (copied), the
// level operators are transposed, the transfers swapped, and the coarsest
// transposed operator inverted; the same arrays rbffd_mg_setup_adjoint
// builds from scratch, at the cost of the transposes.
int rbffd::mg_adjoint_of(const MgHierarchy& F, const rbffd_csr* AT, const float* val32, rbffd_mg* mg, void* ws,
                         size_t ws_bytes, cudaStream_t st) {
    std::memset(mg, 0, sizeof(*mg));
    const MgLevel& F0 = F.lv[0];
    const int64_t N = F0.N;
    if (F.transposed || F.col_base != 0 || AT->n_rows != N || AT->nnz != F0.nnz) return RBFFD_ERR_INVALID_ARG;
    if (val32 && !F.has32) return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0) return RBFFD_ERR_WORKSPACE;
    if (ws_bytes < mg_layout(nullptr, N, nullptr, nullptr)) return RBFFD_ERR_WORKSPACE;
    MgHierarchy h{};
    MgScratch s{};
    mg_layout(ws, N, &h, &s);
    h.nu = F.nu;
    h.omega = F.omega;
    h.has32 = val32 ? 1 : 0;
    h.col_base = 0;
    h.transposed = 1;
    RBFFD_CUDA_TRY(cudaMemsetAsync(s.flags, 0, sizeof(int) * 64, st));
    MgLevel& L0 = h.lv[0];
    L0.N = N;
    L0.row_ptr = AT->row_ptr;
    L0.col = AT->col;
    L0.val = static_cast<const double*>(AT->val);
    L0.val32 = val32;
    L0.nnz = AT->nnz;
    L0.tpr = tpr_for(N, AT->nnz);
    L0.xy = F0.xy;
    L0.mask = F0.mask;
    const int n_levels = F.n_levels;
    for (int l = 0; l < n_levels; ++l) {
        MgLevel& L = h.lv[l];
        const MgLevel& FL = F.lv[l];
        // W: the diagonal and the Dirichlet rows are those of the forward level
        RBFFD_CUDA_TRY(cudaMemcpyAsync(L.dinv, FL.dinv, sizeof(double) * L.N, cudaMemcpyDeviceToDevice, st));
        RBFFD_CUDA_TRY(cudaMemcpyAsync(L.dinv32, FL.dinv32, sizeof(float) * L.N, cudaMemcpyDeviceToDevice, st));
        if (l == n_levels - 1) {
            int rc = dense_inverse(L, 0, s, st);
            if (rc != RBFFD_OK) return rc;
            break;
        }
        MgLevel& C = h.lv[l + 1];
        const MgLevel& FC = F.lv[l + 1];
        const int64_t nc = FC.N;
        C.N = nc;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(C.xy), FC.xy, sizeof(double) * 2 * nc,
                                       cudaMemcpyDeviceToDevice, st));
        RBFFD_CUDA_TRY(cudaMemcpyAsync(const_cast<uint8_t*>(C.mask), FC.mask, nc, cudaMemcpyDeviceToDevice, st));
        rbffd_csr Ac{};
        Ac.n_rows = nc;
        Ac.nnz = FC.nnz;
        Ac.row_ptr = FC.row_ptr;
        Ac.col = FC.col;
        Ac.val = FC.val;
        Ac.dtype = 0;
        int rc = rbffd_transpose(&Ac, const_cast<int64_t*>(C.row_ptr), const_cast<int*>(C.col),
                                 const_cast<double*>(C.val), nullptr, s.tr_ws, s.tr_bytes, st);
        if (rc != RBFFD_OK) return rc;
        mg_f32_kernel<<<blocks_for(FC.nnz), kT, 0, st>>>(C.val, FC.nnz, const_cast<float*>(C.val32));
        C.nnz = FC.nnz;
        C.tpr = tpr_for(nc, FC.nnz);
        // transfers: R = P^T (raw), prolongation R_fwd^T = (N_c / N_f) P
        // without the coarse Dirichlet columns
        RBFFD_CUDA_TRY(cudaMemcpyAsync(L.pidx, FL.pidx, sizeof(int32_t) * L.N * kMgK, cudaMemcpyDeviceToDevice, st));
        RBFFD_CUDA_TRY(cudaMemcpyAsync(L.pval, FL.pval, sizeof(double) * L.N * kMgK, cudaMemcpyDeviceToDevice, st));
        mg_ellrow_kernel<<<blocks_for(L.N + 1), kT, 0, st>>>(L.N, s.prow);
        rbffd_csr P{};
        P.n_rows = L.N;
        P.nnz = L.N * kMgK;
        P.row_ptr = s.prow;
        P.col = L.pidx;
        P.val = L.pval;
        P.dtype = 0;
        if ((rc = rbffd_transpose(&P, L.rrow, L.rcol, L.rval, nullptr, s.tr_ws, s.tr_bytes, st)) != RBFFD_OK) return rc;
        mg_rscale_kernel<<<blocks_for(nc), kT, 0, st>>>(L.rrow, nc, nullptr, 1.0, L.rval, L.rval32);
        mg_pscale_kernel<<<blocks_for(L.N * kMgK), kT, 0, st>>>(L.N, L.pidx, C.mask, nc, (double)nc / (double)L.N,
                                                                 L.pval, L.pval32);
        note_launches(4);
        RBFFD_LAUNCH_CHECK();
        L.rtpr = tpr_for(nc, L.N * kMgK);
    }
    int flags[2] = {0, 0};
    RBFFD_CUDA_TRY(cudaMemcpyAsync(flags, s.flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags[0]) return RBFFD_ERR_SINGULAR_STENCIL;
    h.n_levels = n_levels;
    h.magic = kMgMagic;
    std::memcpy(mg, &h, sizeof(h));
    return RBFFD_OK;
}

// Level sizes of a built hierarchy (the Galerkin hierarchy's layout).
static std::vector<int64_t> level_sizes(const rbffd::MgHierarchy& F) {
    std::vector<int64_t> nb;
    for (int l = 0; l < F.n_levels; ++l) nb.push_back(F.lv[l].N);
    return nb;
}

size_t rbffd::mg_galerkin_workspace(const MgHierarchy& F) {
    const std::vector<int64_t> nb = level_sizes(F);
    return mg_layout(nullptr, F.lv[0].N, nullptr, nullptr, &nb, kMgGalerkinRow);
}

// The adjoint hierarchy of a built forward one with Galerkin coarse
// operators: node sets, interpolation and transfers as in mg_adjoint_of
// (restriction P^T, prolongation (N_c / N_f) P without the coarse Dirichlet
// columns); each coarse operator the product R A P of the level above it
// (mg_galerkin_kernel), its smoother weights from its own diagonal, the
// coarsest inverted.
int rbffd::mg_galerkin_adjoint(const MgHierarchy& F, const rbffd_csr* AT, const float* val32, rbffd_mg* mg,
                               void* ws, size_t ws_bytes, cudaStream_t st) {
    std::memset(mg, 0, sizeof(*mg));
    const MgLevel& F0 = F.lv[0];
    const int64_t N = F0.N;
    if (F.transposed || F.col_base != 0 || AT->n_rows != N || AT->nnz != F0.nnz) return RBFFD_ERR_INVALID_ARG;
    if (val32 && !F.has32) return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0) return RBFFD_ERR_WORKSPACE;
    const std::vector<int64_t> nb = level_sizes(F);
    if (ws_bytes < mg_layout(nullptr, N, nullptr, nullptr, &nb, kMgGalerkinRow)) return RBFFD_ERR_WORKSPACE;
    static bool smem_set = false;
    if (!smem_set) {
        RBFFD_CUDA_TRY(cudaFuncSetAttribute(mg_galerkin_kernel<512, 256>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)gal_smem_bytes<512, 256>()));
        RBFFD_CUDA_TRY(cudaFuncSetAttribute(mg_galerkin_kernel<1024, 512>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)gal_smem_bytes<1024, 512>()));
        smem_set = true;
    }
    MgHierarchy h{};
    MgScratch s{};
    mg_layout(ws, N, &h, &s, &nb, kMgGalerkinRow);
    h.nu = F.nu;
    h.omega = F.omega;
    h.has32 = val32 ? 1 : 0;
    h.col_base = 0;
    h.transposed = 1;
    h.galerkin = 1;
    RBFFD_CUDA_TRY(cudaMemsetAsync(s.flags, 0, sizeof(int) * 64, st));
    MgLevel& L0 = h.lv[0];
    L0.N = N;
    L0.row_ptr = AT->row_ptr;
    L0.col = AT->col;
    L0.val = static_cast<const double*>(AT->val);
    L0.val32 = val32;
    L0.nnz = AT->nnz;
    L0.tpr = tpr_for(N, AT->nnz);
    L0.xy = F0.xy;
    L0.mask = F0.mask;
    // level 0's smoother: A^T has A's diagonal and Dirichlet rows
    RBFFD_CUDA_TRY(cudaMemcpyAsync(L0.dinv, F0.dinv, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(L0.dinv32, F0.dinv32, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    const int n_levels = F.n_levels;
    for (int l = 0; l + 1 < n_levels; ++l) {
        MgLevel& L = h.lv[l];
        const MgLevel& FL = F.lv[l];
        MgLevel& C = h.lv[l + 1];
        const MgLevel& FC = F.lv[l + 1];
        const int64_t nc = FC.N;
        C.N = nc;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(C.xy), FC.xy, sizeof(double) * 2 * nc,
                                       cudaMemcpyDeviceToDevice, st));
        RBFFD_CUDA_TRY(cudaMemcpyAsync(const_cast<uint8_t*>(C.mask), FC.mask, nc, cudaMemcpyDeviceToDevice, st));
        // transfers: R = P^T (raw), prolongation (N_c / N_f) P without the
        // coarse Dirichlet columns
        RBFFD_CUDA_TRY(cudaMemcpyAsync(L.pidx, FL.pidx, sizeof(int32_t) * L.N * kMgK, cudaMemcpyDeviceToDevice, st));
        RBFFD_CUDA_TRY(cudaMemcpyAsync(L.pval, FL.pval, sizeof(double) * L.N * kMgK, cudaMemcpyDeviceToDevice, st));
        mg_ellrow_kernel<<<blocks_for(L.N + 1), kT, 0, st>>>(L.N, s.prow);
        rbffd_csr P{};
        P.n_rows = L.N;
        P.nnz = L.N * kMgK;
        P.row_ptr = s.prow;
        P.col = L.pidx;
        P.val = L.pval;
        P.dtype = 0;
        int rc = rbffd_transpose(&P, L.rrow, L.rcol, L.rval, nullptr, s.tr_ws, s.tr_bytes, st);
        if (rc != RBFFD_OK) return rc;
        mg_rscale_kernel<<<blocks_for(nc), kT, 0, st>>>(L.rrow, nc, nullptr, 1.0, L.rval, L.rval32);
        mg_pscale_kernel<<<blocks_for(L.N * kMgK), kT, 0, st>>>(L.N, L.pidx, C.mask, nc, (double)nc / (double)L.N,
                                                                 L.pval, L.pval32);
        note_launches(3);
        RBFFD_LAUNCH_CHECK();
        L.rtpr = tpr_for(nc, L.N * kMgK);
        // C = R A P: rows staged (small tables first, the large ones if a row
        // overflowed them), row pointer, rows placed
        int* cnt = s.pos;
        int* over = s.flags + 2;
        int64_t* crow = const_cast<int64_t*>(C.row_ptr);
        int64_t cnnz = 0;
        const int64_t stage_cap = std::min(s.gal_cap, nc * (int64_t)kMgGalerkinRow);
        for (int large = 0; large < 2; ++large) {
            RBFFD_CUDA_TRY(cudaMemsetAsync(s.gal_total, 0, sizeof(unsigned long long), st));
            RBFFD_CUDA_TRY(cudaMemsetAsync(over, 0, sizeof(int), st));
            if (!large)
                mg_galerkin_kernel<512, 256><<<sm_count() * 6, kGalWarps * 32, gal_smem_bytes<512, 256>(), st>>>(
                    nc, L.rrow, L.rcol, L.rval, L.row_ptr, L.col, L.val, L.pidx, L.pval, C.mask, cnt, s.gal_start,
                    s.gal_total, stage_cap, s.gal_col, s.gal_val, over, L.N, L.nnz);
            else
                mg_galerkin_kernel<1024, 512><<<sm_count() * 3, kGalWarps * 32, gal_smem_bytes<1024, 512>(), st>>>(
                    nc, L.rrow, L.rcol, L.rval, L.row_ptr, L.col, L.val, L.pidx, L.pval, C.mask, cnt, s.gal_start,
                    s.gal_total, stage_cap, s.gal_col, s.gal_val, over, L.N, L.nnz);
            note_launches(1);
            RBFFD_LAUNCH_CHECK();
            RBFFD_CUDA_TRY(exclusive_scan<int64_t>(CountLoad64{cnt}, nc, crow, s.sums64, crow + nc, st));
            int ovf = 0;
            RBFFD_CUDA_TRY(cudaMemcpyAsync(&cnnz, crow + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            RBFFD_CUDA_TRY(cudaMemcpyAsync(&ovf, over, sizeof(int), cudaMemcpyDeviceToHost, st));
            RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
            if (!ovf) break;
            // a row wider than the large tables, or more entries than the layout holds
            if (large) return RBFFD_ERR_WORKSPACE;
        }
        if (cnnz > nc * (int64_t)kMgGalerkinRow) return RBFFD_ERR_WORKSPACE;
        mg_galerkin_place_kernel<<<blocks_for(nc * 32), kT, 0, st>>>(nc, s.gal_start, crow, s.gal_col, s.gal_val,
                                                                     const_cast<int*>(C.col),
                                                                     const_cast<double*>(C.val),
                                                                     const_cast<float*>(C.val32), stage_cap, cnnz);
        C.nnz = cnnz;
        C.tpr = tpr_for(nc, cnnz);
        mg_diag_kernel<<<blocks_for(nc), kT, 0, st>>>(C.row_ptr, C.col, C.val, nc, 0, C.mask, h.omega, C.dinv,
                                                      C.dinv32, s.flags + 1);
        note_launches(2);
        RBFFD_LAUNCH_CHECK();
    }
    {
        const int rc = dense_inverse(h.lv[n_levels - 1], 0, s, st);
        if (rc != RBFFD_OK) return rc;
    }
    int flags[2] = {0, 0};
    RBFFD_CUDA_TRY(cudaMemcpyAsync(flags, s.flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags[0] || flags[1]) return RBFFD_ERR_SINGULAR_STENCIL;
    h.n_levels = n_levels;
    h.magic = kMgMagic;
    std::memcpy(mg, &h, sizeof(h));
    return RBFFD_OK;
}

int rbffd::mg_setup_geometry(const double* xy, const uint8_t* is_dirichlet, int64_t N, int col_base, int nu,
                             double omega, rbffd_mg* mg, void* ws, size_t ws_bytes, cudaStream_t st,
                             bool transposed) {
    using namespace rbffd;
    std::memset(mg, 0, sizeof(*mg));
    if (nu < 1 || nu > 8 || !(omega > 0.0 && omega < 1.0)) return RBFFD_ERR_INVALID_ARG;
    if (((uintptr_t)xy & 15) != 0) return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0) return RBFFD_ERR_WORKSPACE;
    const size_t need = mg_layout(nullptr, N, nullptr, nullptr);
    if (ws_bytes < need) return RBFFD_ERR_WORKSPACE;

    MgHierarchy h{};
    MgScratch s{};
    mg_layout(ws, N, &h, &s);
    h.magic = 0;
    h.nu = nu;
    h.omega = omega;
    h.col_base = col_base;
    h.transposed = transposed ? 1 : 0;
    h.ws = ws;
    h.ws_bytes = ws_bytes;
    RBFFD_CUDA_TRY(cudaMemsetAsync(s.flags, 0, sizeof(int) * 64, st));

    MgLevel& L0 = h.lv[0];
    L0.N = N;
    L0.xy = xy;
    L0.mask = is_dirichlet;

    int levels = 1;
    int rc = RBFFD_OK;
    for (int l = 0;; ++l) {
        MgLevel& L = h.lv[l];
        if (L.N <= kMgCoarsest || l + 1 >= RBFFD_MG_MAX_LEVELS) {
            if (L.N > kMgCoarsest) return RBFFD_ERR_INVALID_ARG;
            // (a single level is the fine operator itself: inverted by the operator phase)
            if (l > 0 && (rc = dense_inverse(L, 0, s, st)) != RBFFD_OK) return rc;
            levels = l + 1;
            break;
        }
        MgLevel& C = h.lv[l + 1];
        int64_t nc = 0;
        if ((rc = coarsen(L, C, s, st, &nc)) != RBFFD_OK) return rc;
        C.N = nc;
        // coarse operator: stencils, weights, Dirichlet-row assembly
        if ((rc = rbffd_stencils(C.xy, nc, kMgCoarseN, s.sidx, s.knn_ws, s.knn_bytes, st)) != RBFFD_OK) return rc;
        if ((rc = coarse_weights(C.xy, s.sidx, nc, kMgCoarseN, kMgCoarseM, s.sw, s.sstat, st)) != RBFFD_OK) return rc;
        mg_count_kernel<<<blocks_for(nc), kT, 0, st>>>(s.sstat, C.mask, nc, s.flags);
        note_launches(1);
        // (adjoint hierarchy: assembled into scratch, then transposed into the level)
        int64_t* crow = transposed ? s.a_row : const_cast<int64_t*>(C.row_ptr);
        if ((rc = rbffd_assemble_pattern(C.mask, nc, kMgCoarseN, crow, s.asm_ws, s.asm_bytes, st)) != RBFFD_OK)
            return rc;
        int64_t cnnz = 0;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(&cnnz, crow + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (!transposed) {
            if ((rc = rbffd_assemble(s.sidx, s.sw, C.mask, nc, kMgCoarseN, crow, cnnz, const_cast<int*>(C.col),
                                     const_cast<double*>(C.val), const_cast<float*>(C.val32), st)) != RBFFD_OK)
                return rc;
        } else {
            if ((rc = rbffd_assemble(s.sidx, s.sw, C.mask, nc, kMgCoarseN, crow, cnnz, s.a_col, s.a_val, nullptr,
                                     st)) != RBFFD_OK)
                return rc;
            rbffd_csr Ac{};
            Ac.n_rows = nc;
            Ac.nnz = cnnz;
            Ac.row_ptr = s.a_row;
            Ac.col = s.a_col;
            Ac.val = s.a_val;
            Ac.dtype = 0;
            if ((rc = rbffd_transpose(&Ac, const_cast<int64_t*>(C.row_ptr), const_cast<int*>(C.col),
                                      const_cast<double*>(C.val), nullptr, s.tr_ws, s.tr_bytes, st)) != RBFFD_OK)
                return rc;
            mg_f32_kernel<<<blocks_for(cnnz), kT, 0, st>>>(C.val, cnnz, const_cast<float*>(C.val32));
            note_launches(1);
        }
        C.nnz = cnnz;
        C.tpr = tpr_for(nc, cnnz);
        mg_diag_kernel<<<blocks_for(nc), kT, 0, st>>>(C.row_ptr, C.col, C.val, nc, 0, C.mask, omega, C.dinv, C.dinv32,
                                                      s.flags + 1);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        // prolongation: interpolation from the kMgK nearest coarse nodes
        if ((rc = knn_search(C.xy, nc, L.xy, L.N, kMgK, L.pidx, s.knn_ws, s.knn_bytes, st)) != RBFFD_OK) return rc;
        if ((rc = interp_weights(C.xy, nc, L.xy, L.N, L.pidx, kMgK, kMgInterpM, L.pval, s.pstat, st)) != RBFFD_OK)
            return rc;
        mg_pfix_kernel<<<blocks_for(L.N), kT, 0, st>>>(L.N, L.mask, s.pstat, L.pval, L.pval32, s.prow);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        // restriction: (N_c / N_f) P^T, P viewed as an N_f x N_f matrix
        rbffd_csr P{};
        P.n_rows = L.N;
        P.nnz = L.N * kMgK;
        P.row_ptr = s.prow;
        P.col = L.pidx;
        P.val = L.pval;
        P.dtype = 0;
        if ((rc = rbffd_transpose(&P, L.rrow, L.rcol, L.rval, nullptr, s.tr_ws, s.tr_bytes, st)) != RBFFD_OK) return rc;
        const double cscale = (double)nc / (double)L.N;
        if (!transposed) {
            mg_rscale_kernel<<<blocks_for(nc), kT, 0, st>>>(L.rrow, nc, C.mask, cscale, L.rval, L.rval32);
        } else {
            // the transpose of the forward cycle: restrict with P^T, prolong
            // with R^T = (N_c / N_f) P without the coarse Dirichlet columns
            mg_rscale_kernel<<<blocks_for(nc), kT, 0, st>>>(L.rrow, nc, nullptr, 1.0, L.rval, L.rval32);
            mg_pscale_kernel<<<blocks_for(L.N * kMgK), kT, 0, st>>>(L.N, L.pidx, C.mask, nc, cscale, L.pval, L.pval32);
            note_launches(1);
        }
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        L.rtpr = tpr_for(nc, L.N * kMgK);
    }
    int flags[2] = {0, 0};
    RBFFD_CUDA_TRY(cudaMemcpyAsync(flags, s.flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags[0]) return RBFFD_ERR_SINGULAR_STENCIL;
    h.n_levels = levels;
    h.magic = kMgGeometryMagic;
    std::memcpy(mg, &h, sizeof(h));
    return RBFFD_OK;
}

int rbffd::mg_setup_operator(rbffd_mg* mg, const int64_t* row_ptr, const int* col, const double* val,
                             const float* val32, int64_t nnz, cudaStream_t st) {
    using namespace rbffd;
    MgHierarchy h;
    std::memcpy(&h, mg, sizeof(h));
    if (h.magic != kMgGeometryMagic || h.n_levels < 1) return RBFFD_ERR_INVALID_ARG;
    MgScratch s{};
    mg_layout(h.ws, h.lv[0].N, nullptr, &s);  // the scratch of the geometry phase's layout
    MgLevel& L0 = h.lv[0];
    const int64_t N = L0.N;
    L0.row_ptr = row_ptr;
    L0.col = col;
    L0.val = val;
    L0.val32 = val32;
    L0.nnz = nnz;
    L0.tpr = tpr_for(N, nnz);
    h.has32 = val32 ? 1 : 0;
    mg_diag_kernel<<<blocks_for(N), kT, 0, st>>>(L0.row_ptr, L0.col, L0.val, N, h.col_base, L0.mask, h.omega, L0.dinv,
                                                 L0.dinv32, s.flags + 1);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    if (h.n_levels == 1) {  // the fine operator is the coarsest level
        int rc = dense_inverse(L0, h.col_base, s, st);
        if (rc != RBFFD_OK) return rc;
        int flag = 0;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(&flag, s.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (flag) return RBFFD_ERR_SINGULAR_STENCIL;
    }
    h.magic = kMgMagic;
    std::memcpy(mg, &h, sizeof(h));
    return RBFFD_OK;
}

int rbffd::mg_setup_core(const double* xy, const uint8_t* is_dirichlet, int64_t N, const int64_t* row_ptr,
                         const int* col, const double* val, const float* val32, int64_t nnz, int col_base, int nu,
                         double omega, rbffd_mg* mg, void* ws, size_t ws_bytes, cudaStream_t st, bool transposed) {
    int rc = mg_setup_geometry(xy, is_dirichlet, N, col_base, nu, omega, mg, ws, ws_bytes, st, transposed);
    if (rc == RBFFD_OK) rc = mg_setup_operator(mg, row_ptr, col, val, val32, nnz, st);
    if (rc != RBFFD_OK) std::memset(mg, 0, sizeof(*mg));
    return rc;
}
