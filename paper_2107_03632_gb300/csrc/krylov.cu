// BiCGSTAB for the assembled RBF-FD Poisson system: an FP64 solver and a
// mixed solver with FP32 matrix values inside FP64 refinement; plus the
// adjoint solve (sm_103a).
//
// Sec. VI names the implicit solution of the Poisson problem as the next
// step beyond the paper's explicit loop; A u = b is solved here by BiCGSTAB
// (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) with left Jacobi
// scaling D^-1 A u = D^-1 b.  Convergence is judged on the unscaled residual
// |b - A u| <= tol |b|, and a solve returns OK only after that residual has
// been recomputed explicitly from u.
//
// Hardware facts that shape the kernels: FP64 on this chip issues about
// 0.55e12 DFMA/s while HBM streams about 0.83e12 doubles/s, so an FP64
// kernel that does one FP64 operation per double it reads is as much
// FP64-bound as HBM-bound; FP32 runs ~60x faster.  Hence
//  * the FP64 SpMV gives each row TPR <= 4 lanes (few FP64 reduction adds
//    per row), and every vector kernel fuses its dot products;
//  * the mixed solver keeps its Krylov vectors as double-float pairs
//    (df32.cuh, ~48-bit) and does all inner arithmetic on the FP32 pipe, so
//    its inner iteration is bound by HBM bytes only (4-byte values).
//
// FP64 iteration (five kernels on the caller's stream):
//   update_p  p = r + beta (p - omega v)
//   spmv(v)   v = D^-1 A p, (rh, v)               -> alpha
//   update_s  s = r - alpha v
//   spmv(t)   t = D^-1 A s, (t, s), (t, t)        -> omega
//   update_xr x += alpha p + omega s, r = s - omega t, |D r|^2, (rh, r) -> rho
// Scalars live in a device state block; each reduction is finished by the
// last block to arrive (fixed summation order: deterministic for a given
// grid).  The host enqueues iterations in chunks and reads the state between
// chunks; kernels of a finished pass return at once.
//
// Both solvers run in restarted passes.  A pass starts from the explicit
// residual r = b - A x (computed in FP64) with a fresh shadow residual
// rh = r and ends when its recurrence residual has fallen by inner_tol (or
// on a breakdown); the next pass restarts from the new explicit residual.
// Long unrestarted BiCGSTAB runs on these nonsymmetric RBF-FD matrices were
// measured to stall or diverge at 4e6 nodes, while restarted passes converge.
//
// Mixed solver: the passes are the inner solves of FP64 iterative
// refinement -- r = b - A x with the FP64 matrix, the inner BiCGSTAB solves
// A d = r on the float32 values, x += d in FP64.  The inner operator is
// written in difference form
//     (A d)_i = sum_j a_ij (d_j - d_i) + sigma_i d_i,  sigma_i = sum_j a_ij,
// which is A exactly in exact arithmetic and keeps the zero row sums of the
// RBF-FD Laplacian exact after rounding a_ij to float (plain float rounding
// of a_ij would perturb the smooth modes by ~n eps_32 / h^2).
#include "common.cuh"
#include "df32.cuh"
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

namespace rbffd {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 2048;
constexpr int kSlots = 8;
constexpr int kQ = 4;

enum Flag : int { kRunning = 0, kConverged = 1, kBreakdown = 2, kMaxIter = 3, kReplace = 4, kDiverged = 5 };
// A pass whose residual has grown 1e3 above its start is ended early.
constexpr double kGrowth2 = 1e6;
enum Slot : int { kSlotResid = 0, kSlotV = 1, kSlotT = 2, kSlotXR = 3, kSlotLoad = 4 };
enum ResidMode : int { kInit = 0, kCheck = 2 };

struct KState {
    double rho, rho_new, alpha, omega;
    double bnorm2;  // |b|^2 of the system (unscaled)
    double tol2;    // converged when |r|^2 <= tol2
    double rnorm2;  // last recurrence |r|^2 (unscaled)
    double tnorm2;  // last explicit |b - A x|^2
    double rmax2;   // |r|^2 at the start of the pass
    double repl2;   // the pass ends when |r|^2 < repl2 * rmax2
    double sres2;   // last explicit Jacobi-scaled |D^-1 (b - A x)|^2
    double s0;      // scaled |r|^2 at the start of the pass (growth guard)
    int iter;       // iterations of the current run
    int max_iter;
    int flag;
    int bad;        // input validation failure
    int pad0;
    int pad;
    unsigned int counter[kSlots];
};

__device__ __forceinline__ double* part_at(double* part, int slot, int q) {
    return part + ((size_t)slot * kQ + q) * kMaxBlocks;
}

// Block-reduce NQ values, store block partials, and let the last block to
// arrive sum all partials in block order (returned in tot[]).  True there.
template <int NQ>
__device__ bool reduce_last(double (&v)[NQ], double* part, int slot, unsigned int* counter, double (&tot)[NQ]) {
    __shared__ double sh[32];
    __shared__ unsigned int is_last;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double bs = block_sum<kThreads>(v[q], sh);
        if (threadIdx.x == 0) RB_AT(part_at(part, slot, q), blockIdx.x, kMaxBlocks) = bs;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double acc = 0.0;
        const double* pq = part_at(part, slot, q);
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) acc += __ldcg(pq + b);
        tot[q] = block_sum<kThreads>(acc, sh);
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

__device__ __forceinline__ void set_alpha(KState* st, double rv) {
    if (rv == 0.0 || !finite(rv)) {
        st->flag = kBreakdown;
    } else {
        st->alpha = st->rho_new / rv;
        st->rho = st->rho_new;
    }
}

// omega = (t, s) / (t, t).  (The enlarged omega of Sleijpen & van der Vorst
// for nearly orthogonal t, s was measured to slow these solves 6x and is
// not used.)
__device__ __forceinline__ void set_omega(KState* st, double ts, double tt, double ss) {
    (void)ss;
    if (!finite(ts) || !finite(tt)) {
        st->flag = kBreakdown;
        return;
    }
    st->omega = (tt > 0.0) ? ts / tt : 0.0;
}

// Iterate rows in groups of TPR lanes with a warp-uniform loop (every lane
// of a warp runs the same number of trips, so full-mask shuffles are safe).
#define RBFFD_ROW_LOOP(TPR, N, i, valid, BODY)                                        \
    {                                                                                 \
        const int64_t g0_ = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / (TPR); \
        const int64_t ng_ = ((int64_t)gridDim.x * blockDim.x) / (TPR);                \
        const int64_t off_ = (threadIdx.x & 31) / (TPR);                              \
        for (int64_t base_ = g0_ - off_; base_ < (N); base_ += ng_) {                 \
            const int64_t i = base_ + off_;                                           \
            const bool valid = i < (N);                                               \
            BODY                                                                      \
        }                                                                             \
    }

#define RBFFD_ELEM_LOOP(N, i) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (N); i += (int64_t)gridDim.x * blockDim.x)

// ============================================================== FP64 ========
// sum_k a_k x[col_k] over one row, TPR lanes (result in every lane).
template <int TPR>
__device__ __forceinline__ double row_dot64(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                            const double* __restrict__ val, const double* __restrict__ x,
                                            int64_t nx, int64_t row, int sub, bool valid) {
    (void)nx;  // length of x: bound of the checked build's tests
    int64_t a = 0, e = 0;
    if (valid) {
        a = __ldg(row_ptr + row);
        e = __ldg(row_ptr + row + 1);
    }
    double sum = 0.0;
#pragma unroll 4
    for (int64_t k = a + sub; k < e; k += TPR) sum = fma(__ldg(val + k), __ldg(&RB_AT(x, __ldg(col + k), nx)), sum);
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, TPR);
    return sum;
}

// b_i - sum_k a_k x[col_k] for one row with compensated arithmetic: each
// product split exactly by FMA (p + e = a x) and the running sum kept as an
// unevaluated pair (TwoSum, Knuth), so the residual is accurate to about
// eps |r_i| instead of eps sum |a x| (the latter reaches 1e-10 of |b| on the
// finest m = 6 workload).  Used for the explicit residuals that decide
// convergence and restart every pass; ~10 FP64 operations per entry.
__device__ __forceinline__ void two_sum64(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    const double bb = __dadd_rn(s, -a);
    e = __dadd_rn(__dadd_rn(a, -__dadd_rn(s, -bb)), __dadd_rn(b, -bb));
}

template <int TPR>
__device__ __forceinline__ double row_residual64(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                                 const double* __restrict__ val, const double* __restrict__ x,
                                                 int64_t nx, int64_t row, int sub, bool valid, double bi) {
    (void)nx;  // length of x: bound of the checked build's tests
    int64_t a = 0, e = 0;
    if (valid) {
        a = __ldg(row_ptr + row);
        e = __ldg(row_ptr + row + 1);
    }
    double sh = 0.0, sl = 0.0;
#pragma unroll 2
    for (int64_t k = a + sub; k < e; k += TPR) {
        const double av = __ldg(val + k), xv = __ldg(&RB_AT(x, __ldg(col + k), nx));
        const double p = __dmul_rn(av, xv);
        const double pe = fma(av, xv, -p);
        double t, te;
        two_sum64(sh, p, t, te);
        sh = t;
        sl = __dadd_rn(sl, __dadd_rn(te, pe));
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) {
        const double oh = __shfl_xor_sync(0xffffffffu, sh, o, TPR);
        const double ol = __shfl_xor_sync(0xffffffffu, sl, o, TPR);
        double t, te;
        two_sum64(sh, oh, t, te);
        sh = t;
        sl = __dadd_rn(sl, __dadd_rn(ol, te));
    }
    double rh, rl;
    two_sum64(bi, -sh, rh, rl);
    return __dadd_rn(rh, __dadd_rn(rl, -sl));
}

// ---- setup: diagonal, row sums, Jacobi scaling, validation -----------------
__global__ void __launch_bounds__(kThreads) setup_kernel(const int64_t* __restrict__ row_ptr,
                                                         const int* __restrict__ col,
                                                         const double* __restrict__ val, int64_t N, int64_t nnz,
                                                         int jacobi, double* __restrict__ d,
                                                         double* __restrict__ dinv, float* __restrict__ d32,
                                                         float* __restrict__ dinv32, float* __restrict__ sigma32,
                                                         KState* st) {
    int bad = 0;
    RBFFD_ELEM_LOOP(N, i) {
        const int64_t a = row_ptr[i], e = row_ptr[i + 1];
        double di = 0.0, rs = 0.0;
        if (a < 0 || e < a || e > nnz) {
            bad = 1;
        } else {
            for (int64_t k = a; k < e; ++k) {
                const int c = col[k];
                const double v = val[k];
                if ((unsigned)c >= (unsigned)N) bad = 1;
                if (c == (int)i) di = v;
                rs += v;
            }
        }
        if (i == N - 1 && e != nnz) bad = 1;
        if (i == 0 && a != 0) bad = 1;
        const bool use = jacobi && di != 0.0 && isfinite(di);
        const double dv = use ? di : 1.0;
        const double iv = use ? 1.0 / di : 1.0;
        d[i] = dv;
        dinv[i] = iv;
        if (d32) {
            d32[i] = __double2float_rn(dv);
            dinv32[i] = __double2float_rn(iv);
            sigma32[i] = __double2float_rn(rs);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->bad, 1);
}

// kInit:  r = D^-1 (b - A x), rh = r (seed 0) or the pseudo-random shadow
//         residual of seed, p = v = 0, scalars reset: a new pass that ends
//         when |r|^2 < repl^2 |b - A x|^2.
// kCheck: r = b - A x (unscaled), |r|^2 and |b|^2 only.
template <int TPR, int MODE>
__global__ void __launch_bounds__(kThreads) resid64_kernel(const int64_t* __restrict__ row_ptr,
                                                           const int* __restrict__ col,
                                                           const double* __restrict__ val, int64_t N,
                                                           const double* __restrict__ b,
                                                           const double* __restrict__ x,
                                                           const double* __restrict__ dinv,
                                                           double* __restrict__ r, double* __restrict__ rh,
                                                           double* __restrict__ p, double* __restrict__ v,
                                                           double tol, int max_iter, double repl,
                                                           unsigned long long seed, KState* st, double* part) {
    const int sub = threadIdx.x & (TPR - 1);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    RBFFD_ROW_LOOP(TPR, N, i, valid, {
        const double bi = valid ? b[i] : 0.0;
        const double rt = row_residual64<TPR>(row_ptr, col, val, x, N, i, sub, valid, bi);
        if (valid && sub == 0) {
            acc[0] = fma(rt, rt, acc[0]);
            acc[1] = fma(bi, bi, acc[1]);
            const double ri = rt * dinv[i];
            acc[2] = fma(ri, ri, acc[2]);
            if (MODE == kCheck) {
                r[i] = rt;
            } else {
                const double hi = seed ? (double)shadow_value(seed, i) : ri;
                r[i] = ri;
                rh[i] = hi;
                p[i] = 0.0;
                v[i] = 0.0;
                acc[3] = fma(hi, ri, acc[3]);
            }
        }
    })
    double tot[4];
    if (reduce_last<4>(acc, part, kSlotResid, &st->counter[kSlotResid], tot) && threadIdx.x == 0) {
        st->tnorm2 = tot[0];
        st->sres2 = tot[2];
        if (MODE == kCheck) {
            st->bnorm2 = tot[1];
            return;
        }
        st->s0 = tot[2];
        st->bnorm2 = tot[1];
        st->tol2 = tol * tol * tot[1];
        st->rho = 1.0;
        st->alpha = 1.0;
        st->omega = 1.0;
        st->iter = 0;
        st->max_iter = max_iter;
        st->repl2 = repl * repl;
        st->rnorm2 = tot[0];
        st->rmax2 = tot[0];
        st->rho_new = tot[3];
        int flag = kRunning;
        if (tot[0] <= st->tol2) flag = kConverged;
        else if (!finite(tot[0]) || !finite(tot[2]) || !finite(tot[3]) || tot[3] == 0.0) flag = kBreakdown;
        else if (st->iter >= st->max_iter) flag = kMaxIter;
        st->flag = flag;
    }
}

__global__ void __launch_bounds__(kThreads) update_p64_kernel(int64_t N, const double* __restrict__ r,
                                                              const double* __restrict__ v, double* __restrict__ p,
                                                              const KState* st) {
    if (st->flag != kRunning) return;
    const double beta = (st->rho_new / st->rho) * (st->alpha / st->omega);
    const double omega = st->omega;
    RBFFD_ELEM_LOOP(N, i) p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
}

// y = D^-1 A xin; MODE 0: (rh, y) -> alpha.  MODE 1: (y, xin), (y, y) -> omega.
// MODE 2: the product alone.
// With right preconditioning xin is M^-1 s and the omega dots take s itself
// (dotv); dotv NULL: xin.
template <int TPR, int MODE>
__global__ void __launch_bounds__(kThreads) spmv64_kernel(const int64_t* __restrict__ row_ptr,
                                                          const int* __restrict__ col,
                                                          const double* __restrict__ val, int64_t N,
                                                          const double* __restrict__ xin,
                                                          const double* __restrict__ dinv, double* __restrict__ y,
                                                          const double* __restrict__ rh, KState* st, double* part,
                                                          const double* __restrict__ dotv) {
    if (st->flag != kRunning) return;
    const int sub = threadIdx.x & (TPR - 1);
    double acc[3] = {0.0, 0.0, 0.0};
    RBFFD_ROW_LOOP(TPR, N, i, valid, {
        const double ax = row_dot64<TPR>(row_ptr, col, val, xin, N, i, sub, valid);
        if (valid && sub == 0) {
            const double yi = ax * dinv[i];
            y[i] = yi;
            if (MODE == 0) {
                acc[0] = fma(rh[i], yi, acc[0]);
            } else if (MODE == 1) {
                const double si = dotv ? dotv[i] : xin[i];
                acc[0] = fma(yi, si, acc[0]);
                acc[1] = fma(yi, yi, acc[1]);
                acc[2] = fma(si, si, acc[2]);
            }
        }
    })
    if (MODE == 2) return;
    if (MODE == 0) {
        double a1[1] = {acc[0]}, tot[1];
        if (reduce_last<1>(a1, part, kSlotV, &st->counter[kSlotV], tot) && threadIdx.x == 0) set_alpha(st, tot[0]);
    } else {
        double tot[3];
        if (reduce_last<3>(acc, part, kSlotT, &st->counter[kSlotT], tot) && threadIdx.x == 0)
            set_omega(st, tot[0], tot[1], tot[2]);
    }
}

// Left preconditioning (the adjoint with multigrid): the reductions that the
// SpMV kernels fuse in the right-preconditioned form.  MODE 0: (rh, v) ->
// alpha.  MODE 1: (t, s), (t, t), (s, s) -> omega.
template <int MODE>
__global__ void __launch_bounds__(kThreads) dot64_kernel(int64_t N, const double* __restrict__ a,
                                                         const double* __restrict__ b, KState* st, double* part) {
    if (st->flag != kRunning) return;
    double acc[3] = {0.0, 0.0, 0.0};
    RBFFD_ELEM_LOOP(N, i) {
        const double ai = a[i], bi = b[i];
        acc[0] = fma(ai, bi, acc[0]);
        if (MODE == 1) {
            acc[1] = fma(ai, ai, acc[1]);
            acc[2] = fma(bi, bi, acc[2]);
        }
    }
    if (MODE == 0) {
        double a1[1] = {acc[0]}, tot[1];
        if (reduce_last<1>(a1, part, kSlotV, &st->counter[kSlotV], tot) && threadIdx.x == 0) set_alpha(st, tot[0]);
    } else {
        double tot[3];
        if (reduce_last<3>(acc, part, kSlotT, &st->counter[kSlotT], tot) && threadIdx.x == 0)
            set_omega(st, tot[0], tot[1], tot[2]);
    }
}

// Start of a left-preconditioned pass: r = mr (= M (b - A x), from a pass
// started by resid64 kInit), rh = r or the pseudo-random shadow of seed;
// the pass then ends on the relative reduction of |M r| alone (tol2 = 0:
// the explicit FP64 residual between passes decides convergence).
__global__ void __launch_bounds__(kThreads) left_init_kernel(int64_t N, const double* __restrict__ mr,
                                                             double* __restrict__ r, double* __restrict__ rh,
                                                             unsigned long long seed, KState* st, double* part) {
    if (st->flag != kRunning) return;
    double acc[2] = {0.0, 0.0};
    RBFFD_ELEM_LOOP(N, i) {
        const double ri = mr[i];
        const double hi = seed ? (double)shadow_value(seed, i) : ri;
        r[i] = ri;
        rh[i] = hi;
        acc[0] = fma(ri, ri, acc[0]);
        acc[1] = fma(hi, ri, acc[1]);
    }
    double tot[2];
    if (reduce_last<2>(acc, part, kSlotLoad, &st->counter[kSlotLoad], tot) && threadIdx.x == 0) {
        st->rnorm2 = tot[0];
        st->rmax2 = tot[0];
        st->s0 = tot[0];
        st->rho_new = tot[1];
        st->tol2 = 0.0;
        if (!finite(tot[0]) || !finite(tot[1]) || tot[0] == 0.0 || tot[1] == 0.0) st->flag = kBreakdown;
    }
}

__global__ void __launch_bounds__(kThreads) update_s64_kernel(int64_t N, const double* __restrict__ r,
                                                              const double* __restrict__ v, double* __restrict__ s,
                                                              const KState* st) {
    if (st->flag != kRunning) return;
    const double alpha = st->alpha;
    RBFFD_ELEM_LOOP(N, i) s[i] = fma(-alpha, v[i], r[i]);
}

// Stop test shared by both engines' update_xr.  rn2: unscaled |D r|^2 (the
// convergence measure); sn2: Jacobi-scaled |r|^2, the norm BiCGSTAB works
// on, used by the growth guard (the unscaled norm of a scaled iteration can
// swing by the spread of the diagonal).
__device__ __forceinline__ void finish_iteration(KState* st, double rn2, double rho_new, double sn2) {
    st->rnorm2 = rn2;
    st->rho_new = rho_new;
    const int it = st->iter + 1;
    st->iter = it;
    int flag = kRunning;
    if (rn2 <= st->tol2) flag = kConverged;
    else if (!finite(rn2) || !finite(rho_new) || rho_new == 0.0 || st->omega == 0.0) flag = kBreakdown;
    else if (rn2 < st->repl2 * st->rmax2) flag = kReplace;
    else if (!finite(sn2) || sn2 > kGrowth2 * st->s0) flag = kDiverged;
    else if (it >= st->max_iter) flag = kMaxIter;
    st->flag = flag;
}

// x += alpha p + omega sx (sx = M^-1 s with right preconditioning, else s),
// r = s - omega t.
__global__ void __launch_bounds__(kThreads) update_xr64_kernel(int64_t N, double* __restrict__ x,
                                                               const double* __restrict__ p,
                                                               const double* __restrict__ s,
                                                               const double* __restrict__ t, double* __restrict__ r,
                                                               const double* __restrict__ rh,
                                                               const double* __restrict__ d, KState* st,
                                                               double* part, const double* __restrict__ sx) {
    if (st->flag != kRunning) return;
    const double alpha = st->alpha, omega = st->omega;
    double acc[3] = {0.0, 0.0, 0.0};
    RBFFD_ELEM_LOOP(N, i) {
        const double si = s[i];
        x[i] = fma(omega, sx ? sx[i] : si, fma(alpha, p[i], x[i]));
        const double ri = fma(-omega, t[i], si);
        r[i] = ri;
        const double ru = ri * d[i];
        acc[0] = fma(ru, ru, acc[0]);
        acc[1] = fma(rh[i], ri, acc[1]);
        acc[2] = fma(ri, ri, acc[2]);
    }
    double tot[3];
    if (reduce_last<3>(acc, part, kSlotXR, &st->counter[kSlotXR], tot) && threadIdx.x == 0)
        finish_iteration(st, tot[0], tot[1], tot[2]);
}

// ============================================================ double-float ==
// sum_j a_ij (d_j - d_i) over one row with float a_ij; TPR lanes, df32
// accumulation (result in every lane).
template <int TPR>
__device__ __forceinline__ df row_apply_df(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                           const float* __restrict__ val, const float2* __restrict__ x,
                                           int64_t nx, int64_t row, int sub, bool valid, df xi) {
    (void)nx;  // length of x: bound of the checked build's tests
    int64_t a = 0, e = 0;
    if (valid) {
        a = __ldg(row_ptr + row);
        e = __ldg(row_ptr + row + 1);
    }
    DfAcc acc;
#pragma unroll 4
    for (int64_t k = a + sub; k < e; k += TPR) {
        const float w = __ldg(val + k);
        const df xj = df_ldg(&RB_AT(x, __ldg(col + k), nx));
        // d_j - d_i as an unnormalised pair: the rounding of the leading
        // difference is at most eps_32 of that difference (exact when the
        // two values are within a factor 2), so no cancellation is lost
        const float dh = __fsub_rn(xj.hi, xi.hi);
        const float dl = __fsub_rn(xj.lo, xi.lo);
        df pr = two_prod(w, dh);
        pr.lo = __fmaf_rn(w, dl, pr.lo);
        acc.add(pr);
    }
    df sum = acc.value();
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) sum = df_add(sum, df_shfl_xor(sum, o, TPR));
    return sum;
}

// Outer residual into the inner system: r = D^-1 r64 (df32), p = v = 0,
// correction 0, scalars reset, and the shadow residual rh: a pseudo-random
// vector (seed != 0) or r itself (seed == 0).  The outer residual of a late
// refinement pass is the float32 rounding of the matrix acting on the last
// correction; with rh = r, BiCGSTAB on it was seen to break down within ~50
// iterations (residual growth 1e3), in exact FP64 arithmetic too, while a
// random rh converged.  The pass ends when the inner residual has fallen
// below inner_tol |r64|.
__global__ void __launch_bounds__(kThreads) load_df_kernel(int64_t N, const double* __restrict__ r64,
                                                           const float* __restrict__ dinv32, float2* __restrict__ r,
                                                           float2* __restrict__ rh, float2* __restrict__ p,
                                                           float2* __restrict__ v, float2* __restrict__ xd,
                                                           double inner_tol, int max_iter, unsigned long long seed,
                                                           KState* st, double* part) {
    DfAcc a0, a1;
    RBFFD_ELEM_LOOP(N, i) {
        const df ri = df_mul_f(df_from_double(r64[i]), dinv32[i]);
        df_store(r + i, ri);
        const df hi = seed ? df_make(shadow_value(seed, i), 0.f) : ri;
        df_store(rh + i, hi);
        xd[i] = make_float2(0.f, 0.f);
        p[i] = make_float2(0.f, 0.f);
        v[i] = make_float2(0.f, 0.f);
        a0.add(df_mul(ri, ri));
        a1.add(df_mul(hi, ri));
    }
    double acc[2] = {df_to_double(a0.value()), df_to_double(a1.value())}, tot[2];
    if (reduce_last<2>(acc, part, kSlotLoad, &st->counter[kSlotLoad], tot) && threadIdx.x == 0) {
        st->rho = 1.0;
        st->alpha = 1.0;
        st->omega = 1.0;
        st->rho_new = tot[1];
        st->s0 = tot[0];
        st->iter = 0;
        st->max_iter = max_iter;
        st->tol2 = 0.0;           // inner passes end on the relative trigger
        st->rnorm2 = st->tnorm2;  // |r64|^2 from the preceding check
        st->rmax2 = st->tnorm2;
        st->repl2 = inner_tol * inner_tol;
        st->flag = (!finite(tot[0]) || tot[0] == 0.0 || !finite(tot[1]) || tot[1] == 0.0)
                       ? kBreakdown
                       : (max_iter <= 0 ? kMaxIter : kRunning);
    }
}

__global__ void __launch_bounds__(kThreads) update_p_df_kernel(int64_t N, const float2* __restrict__ r,
                                                               const float2* __restrict__ v,
                                                               float2* __restrict__ p, const KState* st) {
    if (st->flag != kRunning) return;
    const df beta = df_from_double((st->rho_new / st->rho) * (st->alpha / st->omega));
    const df nomega = df_from_double(-st->omega);
    RBFFD_ELEM_LOOP(N, i) {
        const df t = df_fma(nomega, df_load(v + i), df_load(p + i));
        df_store(p + i, df_fma(beta, t, df_load(r + i)));
    }
}

// y = D^-1 A32 xin (difference form); MODE 0: (rh, y) -> alpha; MODE 1:
// (y, xin), (y, y) -> omega.
template <int TPR, int MODE>
__global__ void __launch_bounds__(kThreads) spmv_df_kernel(const int64_t* __restrict__ row_ptr,
                                                           const int* __restrict__ col,
                                                           const float* __restrict__ val, int64_t N,
                                                           const float2* __restrict__ xin,
                                                           const float* __restrict__ sigma,
                                                           const float* __restrict__ dinv,
                                                           float2* __restrict__ y, const float2* __restrict__ rh,
                                                           KState* st, double* part) {
    if (st->flag != kRunning) return;
    const int sub = threadIdx.x & (TPR - 1);
    DfAcc a0, a1, a2;
    RBFFD_ROW_LOOP(TPR, N, i, valid, {
        const df xi = valid ? df_ldg(xin + i) : df_make(0.f, 0.f);
        df ax = row_apply_df<TPR>(row_ptr, col, val, xin, N, i, sub, valid, xi);
        if (valid && sub == 0) {
            ax = df_add(ax, df_mul_f(xi, sigma[i]));
            const df yi = df_mul_f(ax, dinv[i]);
            df_store(y + i, yi);
            if (MODE == 0) {
                a0.add(df_mul(df_load(rh + i), yi));
            } else {
                a0.add(df_mul(yi, xi));
                a1.add(df_mul(yi, yi));
                a2.add(df_mul(xi, xi));
            }
        }
    })
    if (MODE == 0) {
        double acc[1] = {df_to_double(a0.value())}, tot[1];
        if (reduce_last<1>(acc, part, kSlotV, &st->counter[kSlotV], tot) && threadIdx.x == 0) {
            const double rv = tot[0];
            if (rv == 0.0 || !finite(rv)) {
                st->flag = kBreakdown;
            } else {
                st->alpha = st->rho_new / rv;
                st->rho = st->rho_new;
            }
        }
    } else {
        double acc[3] = {df_to_double(a0.value()), df_to_double(a1.value()), df_to_double(a2.value())}, tot[3];
        if (reduce_last<3>(acc, part, kSlotT, &st->counter[kSlotT], tot) && threadIdx.x == 0)
            set_omega(st, tot[0], tot[1], tot[2]);
    }
}

__global__ void __launch_bounds__(kThreads) update_s_df_kernel(int64_t N, const float2* __restrict__ r,
                                                               const float2* __restrict__ v,
                                                               float2* __restrict__ s, const KState* st) {
    if (st->flag != kRunning) return;
    const df nalpha = df_from_double(-st->alpha);
    RBFFD_ELEM_LOOP(N, i) df_store(s + i, df_fma(nalpha, df_load(v + i), df_load(r + i)));
}

__global__ void __launch_bounds__(kThreads) update_xr_df_kernel(int64_t N, float2* __restrict__ x,
                                                                const float2* __restrict__ p,
                                                                const float2* __restrict__ s,
                                                                const float2* __restrict__ t,
                                                                float2* __restrict__ r,
                                                                const float2* __restrict__ rh,
                                                                const float* __restrict__ d, KState* st,
                                                                double* part) {
    if (st->flag != kRunning) return;
    const df alpha = df_from_double(st->alpha), omega = df_from_double(st->omega);
    const df nomega = df_from_double(-st->omega);
    DfAcc a0, a1, a2;
    RBFFD_ELEM_LOOP(N, i) {
        const df si = df_load(s + i);
        df_store(x + i, df_fma(omega, si, df_fma(alpha, df_load(p + i), df_load(x + i))));
        const df ri = df_fma(nomega, df_load(t + i), si);
        df_store(r + i, ri);
        const df ru = df_mul_f(ri, d[i]);
        a0.add(df_mul(ru, ru));
        a1.add(df_mul(df_load(rh + i), ri));
        a2.add(df_mul(ri, ri));
    }
    double acc[3] = {df_to_double(a0.value()), df_to_double(a1.value()), df_to_double(a2.value())}, tot[3];
    if (reduce_last<3>(acc, part, kSlotXR, &st->counter[kSlotXR], tot) && threadIdx.x == 0)
        finish_iteration(st, tot[0], tot[1], tot[2]);
}

// x64 += correction (df32), correction = 0.
__global__ void refine_kernel(int64_t N, double* __restrict__ x, float2* __restrict__ xd) {
    RBFFD_ELEM_LOOP(N, i) {
        const float2 c = xd[i];
        x[i] += (double)c.x + (double)c.y;
        xd[i] = make_float2(0.f, 0.f);
    }
}

__global__ void misfit_grad_kernel(int64_t N, const double* __restrict__ u, const double* __restrict__ ut,
                                   const uint8_t* __restrict__ mask, double* __restrict__ g) {
    RBFFD_ELEM_LOOP(N, i) g[i] = mask[i] ? 0.0 : 2.0 * (u[i] - ut[i]);
}

__global__ void adjoint_grad_kernel(int64_t N, const uint8_t* __restrict__ mask, const double* __restrict__ lam,
                                    double* __restrict__ dLdf, double* __restrict__ dLdg) {
    RBFFD_ELEM_LOOP(N, i) {
        const bool dir = mask[i] != 0;
        const double l = lam[i];
        if (dLdf) dLdf[i] = dir ? 0.0 : -l;
        if (dLdg) dLdg[i] = dir ? l : 0.0;
    }
}

// ---------------------------------------------------------------- host -----
struct Work {
    KState* st;
    double* part;
    double *d, *dinv;
    double* x_save;  // iterate at the start of the current pass
    // FP64 engine
    double *r, *rh, *p, *v, *s, *t;
    // multigrid right preconditioning: ph = M^-1 p, sh = M^-1 s
    double *ph, *sh;
    const MgHierarchy* mg;  // host object, NULL without multigrid
    bool mg32;              // float32 V-cycle
    bool left;              // left preconditioning on the interior (adjoint with multigrid)
    // mixed engine
    double* r64;
    float *d32, *dinv32, *sigma32;
    float2 *xd, *rd, *rhd, *pd, *vd, *sd, *td;
};

// Carves the workspace (ws may be null to size it); returns the bytes used.
// With multigrid (mg) the FP64 engine runs in both precisions (the float32
// part is the V-cycle), so `mixed` then selects nothing here.
size_t layout(void* ws, int64_t N, bool mixed, bool mg, Work* w) {
    Carver c(ws);
    Work t{};
    t.st = c.take<KState>(1);
    t.part = c.take<double>((size_t)kSlots * kQ * kMaxBlocks);
    t.d = c.take<double>(N);
    t.dinv = c.take<double>(N);
    t.x_save = c.take<double>(N);
    if (!mixed || mg) {
        t.r = c.take<double>(N);
        t.rh = c.take<double>(N);
        t.p = c.take<double>(N);
        t.v = c.take<double>(N);
        t.s = c.take<double>(N);
        t.t = c.take<double>(N);
        if (mg) {
            t.ph = c.take<double>(N);
            t.sh = c.take<double>(N);
        }
    } else {
        t.r64 = c.take<double>(N);
        t.d32 = c.take<float>(N);
        t.dinv32 = c.take<float>(N);
        t.sigma32 = c.take<float>(N);
        t.xd = c.take<float2>(N);
        t.rd = c.take<float2>(N);
        t.rhd = c.take<float2>(N);
        t.pd = c.take<float2>(N);
        t.vd = c.take<float2>(N);
        t.sd = c.take<float2>(N);
        t.td = c.take<float2>(N);
    }
    if (w) *w = t;
    return c.off;
}

int env_int(const char* name, int dflt);

// RBFFD_TRACE=1 prints one line per pass to stderr (diagnostics only).
bool shadow_random() {
    static const int on = env_int("RBFFD_SHADOW", 0);
    return on != 0;
}

bool trace_on() {
    static const int on = env_int("RBFFD_TRACE", 0);
    return on != 0;
}

int env_int(const char* name, int dflt) {
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    return std::atoi(v);
}

// Lanes per row, from sweeps on GB300: the FP64 SpMV keeps few lanes per row
// (each reduction step costs FP64 adds): 4 for ~56 entries, 2 for ~30; the
// df32 SpMV does best with 4.  RBFFD_TPR64 / RBFFD_TPR32 override for
// tuning sweeps.
int tpr64_for(int64_t N, int64_t nnz) {
    const int o = env_int("RBFFD_TPR64", 0);
    if (o == 1 || o == 2 || o == 4 || o == 8) return o;
    const double L = (double)nnz / (double)std::max<int64_t>(N, 1);
    if (L >= 40) return 4;
    if (L >= 8) return 2;
    return 1;
}

int tpr32_for(int64_t N, int64_t nnz) {
    const int o = env_int("RBFFD_TPR32", 0);
    if (o == 2 || o == 4 || o == 8 || o == 16) return o;
    const double L = (double)nnz / (double)std::max<int64_t>(N, 1);
    if (L >= 12) return 4;
    return 2;
}

// Grid of a persistent-style launch: every block resident at once (blocks
// per SM from the occupancy calculator, cached per kernel), capped at the
// partial-sum capacity.  Reductions finish in the last block of the grid, so
// each launch may use its own grid size.
template <class K>
int grid_of(K kernel) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    const void* key = reinterpret_cast<const void*>(kernel);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 4;
    const int g = std::min(kMaxBlocks, per_sm * sm_count());
    cache[key] = g;
    return g;
}


int64_t spmv_bytes(const rbffd_csr& A, int val_bytes) {
    return A.nnz * (int64_t)(val_bytes + 4) + 8 * (A.n_rows + 1) + 4 * 8 * A.n_rows;
}

template <int TPR>
struct Ops64 {
    static void resid(int mode, const rbffd_csr& A, const double* b, const double* x, const Work& w, double* r,
                      double tol, int max_iter, double repl, unsigned long long seed, cudaStream_t st) {
        const double* val = static_cast<const double*>(A.val);
        if (mode == kInit)
            resid64_kernel<TPR, kInit><<<grid_of(resid64_kernel<TPR, kInit>), kThreads, 0, st>>>(
                A.row_ptr, A.col, val, A.n_rows, b, x, w.dinv, r, w.rh, w.p, w.v, tol, max_iter, repl, seed, w.st, w.part);
        else
            resid64_kernel<TPR, kCheck><<<grid_of(resid64_kernel<TPR, kCheck>), kThreads, 0, st>>>(
                A.row_ptr, A.col, val, A.n_rows, b, x, w.dinv, r, w.rh, w.p, w.v, tol, max_iter, repl, seed, w.st, w.part);
        note_launches(1);
    }
    // Left-preconditioned iteration on the interior unknowns (see
    // solve_fp64): v = Pi B^T (A p), t = Pi B^T (A s), x += alpha p + omega s.
    static void iteration_left(const rbffd_csr& A, double* x, const Work& w, cudaStream_t st,
                               std::vector<int>& ev) {
        const int64_t N = A.n_rows;
        const double* val = static_cast<const double*>(A.val);
        const int64_t bytes = spmv_bytes(A, 8);
        const int* flag = reinterpret_cast<const int*>(reinterpret_cast<const char*>(w.st) + offsetof(KState, flag));
        update_p64_kernel<<<grid_of(update_p64_kernel), kThreads, 0, st>>>(N, w.r, w.v, w.p, w.st);
        int e = prof_begin(st);
        spmv64_kernel<TPR, 2><<<grid_of(spmv64_kernel<TPR, 2>), kThreads, 0, st>>>(
            A.row_ptr, A.col, val, N, w.p, w.dinv, w.ph, nullptr, w.st, w.part, nullptr);
        prof_end(e, st, kProfSpmv64, bytes);
        ev.push_back(e);
        mg_apply_interior(w.mg, w.mg32, w.ph, w.v, flag, st, &ev);
        dot64_kernel<0><<<grid_of(dot64_kernel<0>), kThreads, 0, st>>>(N, w.rh, w.v, w.st, w.part);
        update_s64_kernel<<<grid_of(update_s64_kernel), kThreads, 0, st>>>(N, w.r, w.v, w.s, w.st);
        e = prof_begin(st);
        spmv64_kernel<TPR, 2><<<grid_of(spmv64_kernel<TPR, 2>), kThreads, 0, st>>>(
            A.row_ptr, A.col, val, N, w.s, w.dinv, w.sh, nullptr, w.st, w.part, nullptr);
        prof_end(e, st, kProfSpmv64, bytes);
        ev.push_back(e);
        mg_apply_interior(w.mg, w.mg32, w.sh, w.t, flag, st, &ev);
        dot64_kernel<1><<<grid_of(dot64_kernel<1>), kThreads, 0, st>>>(N, w.t, w.s, w.st, w.part);
        update_xr64_kernel<<<grid_of(update_xr64_kernel), kThreads, 0, st>>>(N, x, w.p, w.s, w.t, w.r, w.rh, w.d,
                                                                             w.st, w.part, nullptr);
        note_launches(7);
    }
    static void iteration(const rbffd_csr& A, double* x, const Work& w, cudaStream_t st, std::vector<int>& ev) {
        if (w.left) return iteration_left(A, x, w, st, ev);
        const int64_t N = A.n_rows;
        const double* val = static_cast<const double*>(A.val);
        const int64_t bytes = spmv_bytes(A, 8);
        // right preconditioning: the SpMVs act on M^-1 p and M^-1 s
        const int* flag = reinterpret_cast<const int*>(reinterpret_cast<const char*>(w.st) + offsetof(KState, flag));
        const double* pin = w.mg ? w.ph : w.p;
        const double* sin_ = w.mg ? w.sh : w.s;
        update_p64_kernel<<<grid_of(update_p64_kernel), kThreads, 0, st>>>(N, w.r, w.v, w.p, w.st);
        if (w.mg) mg_apply(w.mg, w.mg32, w.p, w.ph, flag, st, &ev);
        int e = prof_begin(st);
        spmv64_kernel<TPR, 0><<<grid_of(spmv64_kernel<TPR, 0>), kThreads, 0, st>>>(
            A.row_ptr, A.col, val, N, pin, w.dinv, w.v, w.rh, w.st, w.part, nullptr);
        prof_end(e, st, kProfSpmv64, bytes);
        ev.push_back(e);
        update_s64_kernel<<<grid_of(update_s64_kernel), kThreads, 0, st>>>(N, w.r, w.v, w.s, w.st);
        if (w.mg) mg_apply(w.mg, w.mg32, w.s, w.sh, flag, st, &ev);
        e = prof_begin(st);
        spmv64_kernel<TPR, 1><<<grid_of(spmv64_kernel<TPR, 1>), kThreads, 0, st>>>(
            A.row_ptr, A.col, val, N, sin_, w.dinv, w.t, nullptr, w.st, w.part, w.mg ? w.s : nullptr);
        prof_end(e, st, kProfSpmv64, bytes);
        ev.push_back(e);
        update_xr64_kernel<<<grid_of(update_xr64_kernel), kThreads, 0, st>>>(N, x, pin, w.s, w.t, w.r, w.rh, w.d,
                                                                             w.st, w.part, w.mg ? w.sh : nullptr);
        note_launches(5);
    }
};

template <int TPR>
struct OpsDf {
    static void iteration(const rbffd_csr& A32, const Work& w, cudaStream_t st, std::vector<int>& ev) {
        const int64_t N = A32.n_rows;
        const float* val = static_cast<const float*>(A32.val);
        // algorithmic bytes: nnz (4 + 4) + row_ptr + 8-byte df32 vectors
        // (gathered once, result, dot partner) + 4-byte sigma and scale
        const int64_t bytes = spmv_bytes(A32, 4);
        update_p_df_kernel<<<grid_of(update_p_df_kernel), kThreads, 0, st>>>(N, w.rd, w.vd, w.pd, w.st);
        int e = prof_begin(st);
        spmv_df_kernel<TPR, 0><<<grid_of(spmv_df_kernel<TPR, 0>), kThreads, 0, st>>>(
            A32.row_ptr, A32.col, val, N, w.pd, w.sigma32, w.dinv32, w.vd, w.rhd, w.st, w.part);
        prof_end(e, st, kProfSpmv32, bytes);
        ev.push_back(e);
        update_s_df_kernel<<<grid_of(update_s_df_kernel), kThreads, 0, st>>>(N, w.rd, w.vd, w.sd, w.st);
        e = prof_begin(st);
        spmv_df_kernel<TPR, 1><<<grid_of(spmv_df_kernel<TPR, 1>), kThreads, 0, st>>>(
            A32.row_ptr, A32.col, val, N, w.sd, w.sigma32, w.dinv32, w.td, nullptr, w.st, w.part);
        prof_end(e, st, kProfSpmv32, bytes);
        ev.push_back(e);
        update_xr_df_kernel<<<grid_of(update_xr_df_kernel), kThreads, 0, st>>>(N, w.xd, w.pd, w.sd, w.td, w.rd,
                                                                               w.rhd, w.d32, w.st, w.part);
        note_launches(5);
    }
};

void resid64(int tpr, int mode, const rbffd_csr& A, const double* b, const double* x, const Work& w, double* r,
             double tol, int max_iter, double repl, cudaStream_t st, unsigned long long seed = 0) {
    switch (tpr) {
        case 1: Ops64<1>::resid(mode, A, b, x, w, r, tol, max_iter, repl, seed, st); break;
        case 2: Ops64<2>::resid(mode, A, b, x, w, r, tol, max_iter, repl, seed, st); break;
        case 8: Ops64<8>::resid(mode, A, b, x, w, r, tol, max_iter, repl, seed, st); break;
        default: Ops64<4>::resid(mode, A, b, x, w, r, tol, max_iter, repl, seed, st); break;
    }
}

void iter64(int tpr, const rbffd_csr& A, double* x, const Work& w, cudaStream_t st, std::vector<int>& ev) {
    switch (tpr) {
        case 1: Ops64<1>::iteration(A, x, w, st, ev); break;
        case 2: Ops64<2>::iteration(A, x, w, st, ev); break;
        case 8: Ops64<8>::iteration(A, x, w, st, ev); break;
        default: Ops64<4>::iteration(A, x, w, st, ev); break;
    }
}

void iter_df(int tpr, const rbffd_csr& A32, const Work& w, cudaStream_t st, std::vector<int>& ev) {
    switch (tpr) {
        case 2: OpsDf<2>::iteration(A32, w, st, ev); break;
        case 8: OpsDf<8>::iteration(A32, w, st, ev); break;
        case 16: OpsDf<16>::iteration(A32, w, st, ev); break;
        default: OpsDf<4>::iteration(A32, w, st, ev); break;
    }
}

int read_state(const Work& w, KState* hs, cudaStream_t st) {
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    return RBFFD_OK;
}

bool csr_ok(const rbffd_csr* A, int dtype) {
    return A && A->row_ptr && A->col && A->val && A->dtype == dtype && A->n_rows > 0 &&
           A->n_rows <= 0x7fffffffLL && A->nnz >= 0;
}

double rel_of(const KState& s) {
    if (s.bnorm2 > 0.0) return std::sqrt(s.tnorm2 / s.bnorm2);
    return std::sqrt(s.tnorm2);
}

// Iterations enqueued per host round trip.  A chunk that runs past the end
// of its pass costs the launches of every iteration after the end (kernels
// that return at once: ~90 launches, ~0.2 ms, per iteration with the
// V-cycles); one that stops short costs a round trip (tens of microseconds
// of idle device).  So the next chunk is the number of iterations the pass
// still needs at the residual reduction measured so far in it (rate2: factor
// per iteration on |r|^2), plus one, but at most ~kChunkMs of device time at
// the measured time per iteration: early BiCGSTAB iterations often reduce
// the residual slowly and would make the prediction far too long.  Without
// a measurement: 4, doubling, within the same time cap.
constexpr double kChunkMs = 4.0;

struct ChunkPlan {
    int chunk = 4;
    double rate2 = 0.0;
    double ms_per_iter = 0.0;
    int cap() const {
        if (!(ms_per_iter > 0.0)) return 64;
        return (int)std::min(64.0, std::max(2.0, std::ceil(kChunkMs / ms_per_iter)));
    }
    static int need(double from2, double to2, double rate2) {
        if (!(rate2 > 0.0 && rate2 < 1.0) || !(from2 > 0.0) || !(to2 > 0.0)) return -1;
        if (from2 <= to2) return 1;
        const double n = std::ceil(std::log(to2 / from2) / std::log(rate2));
        return (int)std::min(n, 63.0) + 1;
    }
    // first chunk of a pass starting at |r|^2 = start2 that ends at target2
    void start(double start2, double target2) {
        const int n = need(start2, target2, rate2);
        if (n > 0) chunk = std::min(std::max(n, 1), cap());
    }
    void update(const KState& hs, double start2, int ran, double ms) {
        if (ran > 0 && ms > 0.0) ms_per_iter = ms_per_iter > 0.0 ? 0.5 * (ms_per_iter + ms / ran) : ms / ran;
        const double target2 = std::max(hs.tol2, hs.repl2 * hs.rmax2);
        if (hs.iter > 0 && hs.rnorm2 > 0.0 && start2 > 0.0) {
            const double r2 = std::pow(hs.rnorm2 / start2, 1.0 / hs.iter);
            if (r2 > 0.0 && r2 < 1.0) rate2 = r2;
        }
        const int n = need(hs.rnorm2, target2, rate2);
        chunk = std::min(n > 0 ? std::max(n, 1) : chunk * 2, cap());
    }
};

// Stagnation: the relative residual must halve at least once per
// max(kStagMin, its age) iterations, its age being the iteration count at
// which it last halved; a solve that goes longer without halving stops with
// RBFFD_ERR_NOT_CONVERGED (a converging solve halves its residual steadily,
// every few iterations with multigrid, every few hundred with Jacobi
// scaling at millions of nodes; operators with spurious modes, e.g. stencils
// barely larger than the polynomial space, stall and otherwise ran to
// max_iter).  Observed at every explicit residual and, inside a pass, from
// the recurrence residual at each chunk boundary.
constexpr long long kStagMin = 2000;
struct StagMonitor {
    double anchor = -1.0;  // relative residual at the last halving
    long long at = 0;      // iteration count then
    bool stalled = false;
    void observe(double rel, long long it) {
        if (!(rel >= 0.0) || !std::isfinite(rel)) return;
        if (anchor < 0.0 || rel <= 0.5 * anchor) {
            anchor = rel;
            at = it;
            return;
        }
        if (it - at > std::max(kStagMin, at)) stalled = true;
    }
};

// Runs chunks of iterations until the state leaves kRunning (or, with a
// monitor, until it reports stagnation; the state then stays kRunning and
// the next pass restarts it); returns the flag, or minus a status on a CUDA
// error.  rel_start: the relative residual at the pass start, it_base: the
// iterations before this pass.  With profiling on, only the SpMV launches of
// iterations that ran are accounted (launches after the pass ended return at
// once and are dropped).
template <class IterFn>
int run_chunks(const Work& w, KState* hs, cudaStream_t st, ChunkPlan& plan, IterFn iter, StagMonitor* mon = nullptr,
               double rel_start = 0.0, long long it_base = 0) {
    std::vector<int> ev;
    const double start2 = hs->rnorm2;
    plan.start(start2, std::max(hs->tol2, hs->repl2 * hs->rmax2));
    while (hs->flag == kRunning) {
        const int before = hs->iter;
        const int chunk = plan.chunk;
        const auto t0 = std::chrono::steady_clock::now();
        ev.clear();
        for (int c = 0; c < chunk; ++c) iter(ev);
        RBFFD_LAUNCH_CHECK();
        const int rc = read_state(w, hs, st);
        if (rc != RBFFD_OK) return -rc;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        // every iteration brackets the same number of launches, in order
        const int per_iter = chunk > 0 ? (int)ev.size() / chunk : 0;
        if (profiling()) prof_commit(ev.data(), (int)ev.size(), per_iter * (hs->iter - before));
        plan.update(*hs, start2, hs->iter - before, ms);
        if (mon && start2 > 0.0 && hs->flag == kRunning) {
            mon->observe(rel_start * std::sqrt(hs->rnorm2 / start2), it_base + hs->iter);
            if (mon->stalled) break;
        }
    }
    return hs->flag;
}

// Pass bookkeeping shared by both solvers.  A pass that leaves the explicit
// Jacobi-scaled residual larger than at its start is undone (the iterate is
// restored from the copy taken before the pass) and later passes get half
// the iteration budget of the undone one (growing again by a quarter per
// kept pass): the early part of a BiCGSTAB pass is the part that reduces
// the residual.
struct PassGuard {
    double prev = INFINITY;  // explicit scaled |r|^2 at the start of the pass just run
    int cap = 0x7fffffff;    // iteration budget of the next pass
    int last_iters = 0;      // iterations of the pass just run
    int rejected = 0;        // passes undone in a row
    int rejected_total = 0;
    // Called when the explicit residual after a pass is not below the one
    // before it.  Returns false once retrying is pointless: the pass was a
    // single iteration already (the iterate sits at the rounding floor of
    // the explicit residual) or passes were undone 12 times in a row.
    bool reject() {
        ++rejected;
        ++rejected_total;
        prev = INFINITY;
        if (last_iters <= 1 || rejected > 12) return false;
        cap = std::max(last_iters / 2, 1);
        return true;
    }
    // A pass was kept: the budget found by halving stays in force (long
    // passes on these matrices tend to diverge again from the same kind of
    // residual) and grows by a quarter per kept pass.
    void accept() {
        rejected = 0;
        if (cap < 0x7fffffff / 2) cap += std::max(cap / 4, 1);
    }
    // Last resort once reject() gives up: if the passes used rh = r, retry
    // with pseudo-random shadow residuals (a pass that blows up in its first
    // iteration is a near-breakdown, (rh, A M p) ~ 0, of the shadow r).
    bool switch_shadow(bool& rnd) {
        if (rnd) return false;
        rnd = true;
        rejected = 0;
        cap = 0x7fffffff;
        return true;
    }
};

// Shadow residual of a pass: r itself (seed 0) by default; a pseudo-random
// one per pass once rnd is set (RBFFD_SHADOW=1 sets it from the start: better
// on late passes of small systems, worse on the long first pass of 4M-node
// systems) or after a pass that broke down with rh = r.
unsigned long long shadow_seed(bool rnd, int pass) {
    return rnd ? 0x5EED2107ull + (unsigned long long)pass : 0ull;
}

int solve_fp64(const rbffd_csr& A, const double* b, double* x, const rbffd_solve_opts& o, const Work& w,
               cudaStream_t st, rbffd_solve_info* info) {
    const int64_t N = A.n_rows;
    const int tpr = tpr64_for(N, A.nnz);
    KState hs;
    int rc;
    int total = 0, passes = 0, breakdowns = 0;
    ChunkPlan chunk;
    int status = RBFFD_ERR_NOT_CONVERGED;
    double rel = INFINITY;
    PassGuard g;
    StagMonitor mon;
    // A pass ends when its recurrence residual reaches tol; near the FP64
    // floor the recurrence drifts from the true residual by ~10 %, so a pass
    // that ended there while the explicit residual is still above tol would
    // repeat as a one-iteration pass.  After each such pass the next pass's
    // target is a quarter of the one before (down to tol / 1000).
    double tol_scale = 1.0;
    bool rnd = shadow_random();
    // Multigrid, forward: start from x_b = b_b on the Dirichlet (identity)
    // rows, so that every residual is zero there.  The right-preconditioned
    // operator A M = [I 0; (I - L_ii M_ii) L_ib  L_ii M_ii] couples the
    // Dirichlet part of a vector into the interior through a block of size
    // ~1/h^2; a residual with Dirichlet entries (nonzero boundary data) made
    // BiCGSTAB break down in its first step at 1e6 nodes.
    // Multigrid, adjoint (A here is A^T = [I L_ib^T; 0 L_ii^T]): the
    // interior unknowns solve L_ii^T x_i = b_i and x_b = b_b - L_ib^T x_i
    // follows by back substitution (the same Dirichlet-row update, done
    // here and after every pass).  The interior system runs left
    // preconditioned, B_ii^T L_ii^T = (L_ii B_ii)^T, the transpose of the
    // forward's right-preconditioned operator, whose deviation from I is
    // bounded.  Right preconditioning, L_ii^T B_ii^T = (B_ii L_ii)^T, puts
    // L^T after the cycle: RBF-FD columns do not sum to zero, so L^T turns
    // the cycle's smooth error into a rough vector ~1/h^2 larger (growth
    // ~1e3 in the first BiCGSTAB step at 1e6 nodes, and passes that failed).
    if (w.mg && (rc = mg_dirichlet_fix(w.mg, b, x, nullptr, st)) != RBFFD_OK) return rc;
    while (true) {
        // explicit residual; starts a fresh pass (rh = r or a pseudo-random
        // shadow residual, p = v = 0)
        const int budget = std::min(std::max(o.max_iter - total, 0), g.cap);
        resid64(tpr, kInit, A, b, x, w, w.r, o.tol * tol_scale, budget, o.inner_tol, st, shadow_seed(rnd, passes));
        RBFFD_LAUNCH_CHECK();
        if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
        if (passes > 0 && !(hs.sres2 <= g.prev)) {
            // the pass made things worse: undo it and retry with a shorter pass
            RBFFD_CUDA_TRY(cudaMemcpyAsync(x, w.x_save, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
            const bool retry = !mon.stalled && (g.reject() || g.switch_shadow(rnd));
            if (trace_on()) fprintf(stderr, "[rbffd fp64] pass undone, %s\n", retry ? "retry" : "stop");
            if (!retry) {
                resid64(tpr, kCheck, A, b, x, w, w.r, o.tol, 0, 0.0, st);
                RBFFD_LAUNCH_CHECK();
                if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
                rel = rel_of(hs);
                status = rel <= o.tol ? RBFFD_OK : RBFFD_ERR_NOT_CONVERGED;
                break;
            }
            continue;
        }
        g.accept();
        if (hs.bnorm2 == 0.0 && hs.tnorm2 == 0.0) {
            rel = 0.0;
            status = RBFFD_OK;
            break;
        }
        rel = rel_of(hs);
        if (rel <= o.tol) {
            status = RBFFD_OK;
            break;
        }
        if (!std::isfinite(rel)) {
            status = RBFFD_ERR_BREAKDOWN;
            break;
        }
        mon.observe(rel, total);
        if (mon.stalled) {
            if (trace_on()) fprintf(stderr, "[rbffd fp64] stagnation after %d iterations, rel %.3e\n", total, rel);
            break;
        }
        if (total >= o.max_iter || passes >= o.max_outer) break;
        ++passes;
        g.prev = hs.sres2;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(w.x_save, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        const double start2 = hs.tnorm2;
        if (w.left) {
            // r = Pi B^T (b - A x), rh, scalars of the left-preconditioned pass
            const int* flag =
                reinterpret_cast<const int*>(reinterpret_cast<const char*>(w.st) + offsetof(KState, flag));
            if ((rc = mg_apply_interior(w.mg, w.mg32, w.r, w.ph, flag, st)) != RBFFD_OK) return rc;
            left_init_kernel<<<grid_of(left_init_kernel), kThreads, 0, st>>>(N, w.ph, w.r, w.rh,
                                                                             shadow_seed(rnd, passes), w.st, w.part);
            note_launches(1);
            RBFFD_LAUNCH_CHECK();
            if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
        }
        const int f = run_chunks(w, &hs, st, chunk, [&](std::vector<int>& ev) { iter64(tpr, A, x, w, st, ev); },
                                 &mon, rel, total);
        if (f < 0) return -f;
        if (w.left && (rc = mg_dirichlet_fix(w.mg, b, x, nullptr, st)) != RBFFD_OK) return rc;
        total += hs.iter;
        if (trace_on())
            fprintf(stderr, "[rbffd fp64] pass %d: %d its, flag %d, recurrence |r|/|r0| %.3e, rel at start %.3e\n",
                    passes, hs.iter, hs.flag, std::sqrt(hs.rnorm2 / start2), rel);
        g.last_iters = hs.iter;
        if (hs.flag == kConverged) tol_scale = std::max(0.25 * tol_scale, 1e-3);
        if (hs.flag == kBreakdown) {
            rnd = true;
            if (++breakdowns >= 8) {
                status = RBFFD_ERR_BREAKDOWN;
                break;
            }
        }
    }
    if (status != RBFFD_OK && std::isfinite(rel) && total > 0) {
        resid64(tpr, kCheck, A, b, x, w, w.r, o.tol, 0, 0.0, st);
        RBFFD_LAUNCH_CHECK();
        if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
        rel = rel_of(hs);
    }
    info->status = status;
    info->iters = total;
    info->outer_sweeps = passes;
    info->restarts = g.rejected_total;
    info->rel_residual = rel;
    return status;
}

int solve_mixed(const rbffd_csr& A, const rbffd_csr& A32, const double* b, double* x, const rbffd_solve_opts& o,
                const Work& w, cudaStream_t st, rbffd_solve_info* info) {
    const int64_t N = A.n_rows;
    const int tpr64 = tpr64_for(N, A.nnz);
    const int tpr32 = tpr32_for(N, A.nnz);
    KState hs;
    int rc;
    int total = 0, outer = 0, breakdowns = 0;
    ChunkPlan chunk;
    int status = RBFFD_ERR_NOT_CONVERGED;
    double rel = INFINITY;
    PassGuard g;
    StagMonitor mon;
    bool rnd = shadow_random();
    while (true) {
        resid64(tpr64, kCheck, A, b, x, w, w.r64, o.tol, 0, 0.0, st);
        RBFFD_LAUNCH_CHECK();
        if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
        if (outer > 0 && !(hs.sres2 <= g.prev)) {
            // the correction made things worse: undo it, shorter next pass
            RBFFD_CUDA_TRY(cudaMemcpyAsync(x, w.x_save, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
            const bool retry = !mon.stalled && (g.reject() || g.switch_shadow(rnd));
            if (trace_on()) fprintf(stderr, "[rbffd mixed] pass undone, %s\n", retry ? "retry" : "stop");
            if (!retry) {
                resid64(tpr64, kCheck, A, b, x, w, w.r64, o.tol, 0, 0.0, st);
                RBFFD_LAUNCH_CHECK();
                if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
                rel = rel_of(hs);
                status = rel <= o.tol ? RBFFD_OK : RBFFD_ERR_NOT_CONVERGED;
                break;
            }
            continue;
        }
        g.accept();
        if (hs.bnorm2 == 0.0 && hs.tnorm2 == 0.0) {
            rel = 0.0;
            status = RBFFD_OK;
            break;
        }
        rel = rel_of(hs);
        if (rel <= o.tol) {
            status = RBFFD_OK;
            break;
        }
        if (!std::isfinite(rel)) {
            status = RBFFD_ERR_BREAKDOWN;
            break;
        }
        mon.observe(rel, total);
        if (mon.stalled) {
            if (trace_on()) fprintf(stderr, "[rbffd mixed] stagnation after %d iterations, rel %.3e\n", total, rel);
            break;
        }
        if (total >= o.max_iter || outer >= o.max_outer) break;
        ++outer;
        g.prev = hs.sres2;
        // relative target of this pass: inner_tol, but no deeper than the
        // outer tolerance needs
        const double inner = std::min(std::max(o.inner_tol, 0.5 * o.tol / rel), 0.5);
        const int budget = std::min(o.max_iter - total, g.cap);
        const unsigned long long seed = shadow_seed(rnd, outer);
        load_df_kernel<<<grid_of(load_df_kernel), kThreads, 0, st>>>(N, w.r64, w.dinv32, w.rd, w.rhd, w.pd, w.vd,
                                                                     w.xd, inner, budget, seed, w.st, w.part);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
        const double start2 = hs.rmax2;
        const int f = run_chunks(w, &hs, st, chunk, [&](std::vector<int>& ev) { iter_df(tpr32, A32, w, st, ev); },
                                 &mon, rel, total);
        if (f < 0) return -f;
        total += hs.iter;
        if (trace_on())
            fprintf(stderr, "[rbffd mixed] pass %d: %d its, flag %d, inner |r|/|r0| %.3e, rel at start %.3e\n", outer,
                    hs.iter, hs.flag, std::sqrt(hs.rnorm2 / start2), rel);
        g.last_iters = hs.iter;
        RBFFD_CUDA_TRY(cudaMemcpyAsync(w.x_save, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        refine_kernel<<<grid_of(refine_kernel), kThreads, 0, st>>>(N, x, w.xd);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        if (hs.flag == kBreakdown) {
            rnd = true;
            if (++breakdowns >= 8) {
                status = RBFFD_ERR_BREAKDOWN;
                break;
            }
        }
    }
    if (status != RBFFD_OK && std::isfinite(rel) && total > 0) {
        resid64(tpr64, kCheck, A, b, x, w, w.r64, o.tol, 0, 0.0, st);
        RBFFD_LAUNCH_CHECK();
        if ((rc = read_state(w, &hs, st)) != RBFFD_OK) return rc;
        rel = rel_of(hs);
    }
    info->status = status;
    info->iters = total;
    info->outer_sweeps = outer;
    info->restarts = g.rejected_total;
    info->rel_residual = rel;
    return status;
}

int solve_impl(const rbffd_csr* A, const rbffd_csr* A32, const double* b, double* x, const rbffd_solve_opts* o,
               rbffd_solve_info* info, void* ws, size_t ws_bytes, cudaStream_t st, bool adjoint) {
    if (!csr_ok(A, 0) || !b || !x || !o || !info) return RBFFD_ERR_INVALID_ARG;
    const bool mixed = o->precision == 1;
    if (o->precision != 0 && o->precision != 1) return RBFFD_ERR_INVALID_ARG;
    if (mixed && o->precond != 1 && (!csr_ok(A32, 1) || A32->n_rows != A->n_rows || A32->nnz != A->nnz ||
                  A32->row_ptr != A->row_ptr || A32->col != A->col))
        return RBFFD_ERR_INVALID_ARG;  // the float32 copy shares A's (validated) pattern
    if (!(o->tol > 0.0) || o->max_iter < 0) return RBFFD_ERR_INVALID_ARG;
    if (!(o->inner_tol > 0.0 && o->inner_tol < 1.0) || o->max_outer < 1) return RBFFD_ERR_INVALID_ARG;
    const int64_t N = A->n_rows;
    if (o->precond != 0 && o->precond != 1) return RBFFD_ERR_INVALID_ARG;
    const MgHierarchy* mg = nullptr;
    if (o->precond == 1) {
        mg = mg_hierarchy(o->mg);
        // a hierarchy built for A serves the solve, one built for A^T the adjoint
        if (!mg || mg_fine_rows(mg) != N || (mixed && !mg_has_fp32(mg)) || mg_is_transposed(mg) != adjoint)
            return RBFFD_ERR_INVALID_ARG;
    }
    Work w{};
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0 || ws_bytes < layout(nullptr, N, mixed, mg != nullptr, nullptr))
        return RBFFD_ERR_WORKSPACE;
    layout(ws, N, mixed, mg != nullptr, &w);
    w.mg = mg;
    w.mg32 = mg && mixed;
    w.left = mg && adjoint && !mg_is_galerkin(mg);
    std::memset(info, 0, sizeof(*info));

    KState hs;
    RBFFD_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(KState), st));
    // with the multigrid preconditioner the outer system is not rescaled
    const int jacobi = (o->jacobi && !mg) ? 1 : 0;
    setup_kernel<<<(int)std::min<int64_t>((N + kThreads - 1) / kThreads, sm_count() * 8), kThreads, 0, st>>>(
        A->row_ptr, A->col, static_cast<const double*>(A->val), N, A->nnz, jacobi, w.d, w.dinv, w.d32, w.dinv32,
        w.sigma32, w.st);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    int rc = read_state(w, &hs, st);
    if (rc != RBFFD_OK) return rc;
    if (hs.bad) return RBFFD_ERR_INVALID_ARG;
    // multigrid: the FP64 BiCGSTAB, its V-cycle in float32 when mixed
    if (mg) return solve_fp64(*A, b, x, *o, w, st, info);
    return mixed ? solve_mixed(*A, *A32, b, x, *o, w, st, info) : solve_fp64(*A, b, x, *o, w, st, info);
}

}  // namespace
}  // namespace rbffd

extern "C" size_t rbffd_solve_workspace_size(int64_t N, const rbffd_solve_opts* opts) {
    RBFFD_NVTX("rbffd_solve_workspace_size");
    if (N <= 0) return 0;
    const bool mixed = opts && opts->precision == 1;
    const bool mg = opts && opts->precond == 1;
    return rbffd::layout(nullptr, N, mixed, mg, nullptr);
}

extern "C" int rbffd_solve(const rbffd_csr* A, const rbffd_csr* A32, const double* b, double* x,
                           const rbffd_solve_opts* opts, rbffd_solve_info* info, void* ws, size_t ws_bytes,
                           void* stream) {
    RBFFD_NVTX("rbffd_solve");
    return rbffd::solve_impl(A, A32, b, x, opts, info, ws, ws_bytes, rbffd::as_stream(stream), false);
}

extern "C" int rbffd_solve_adjoint(const rbffd_csr* AT, const rbffd_csr* AT32, const uint8_t* is_dirichlet,
                                   const double* dLdu, double* lambda, double* dLdf, double* dLdg,
                                   const rbffd_solve_opts* opts, rbffd_solve_info* info, void* ws, size_t ws_bytes,
                                   void* stream) {
    RBFFD_NVTX("rbffd_solve_adjoint");
    using namespace rbffd;
    if (!is_dirichlet && (dLdf || dLdg)) return RBFFD_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    const int rc = solve_impl(AT, AT32, dLdu, lambda, opts, info, ws, ws_bytes, st, true);
    if (rc != RBFFD_OK) return rc;
    if (dLdf || dLdg) {
        const int64_t N = AT->n_rows;
        adjoint_grad_kernel<<<(int)std::min<int64_t>((N + 255) / 256, sm_count() * 8), 256, 0, st>>>(
            N, is_dirichlet, lambda, dLdf, dLdg);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
    }
    return RBFFD_OK;
}

extern "C" int rbffd_misfit_grad(const double* u, const double* u_target, const uint8_t* is_dirichlet, int64_t N,
                                 double* dLdu, void* stream) {
    RBFFD_NVTX("rbffd_misfit_grad");
    using namespace rbffd;
    if (!u || !u_target || !is_dirichlet || !dLdu || N <= 0) return RBFFD_ERR_INVALID_ARG;
    misfit_grad_kernel<<<(int)std::min<int64_t>((N + 255) / 256, sm_count() * 8), 256, 0, as_stream(stream)>>>(
        N, u, u_target, is_dirichlet, dLdu);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}
