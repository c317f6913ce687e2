// BiCGSTAB for the assembled RBF-FD Poisson system, FP64 and mixed
// FP32-inner / FP64-refinement, plus the adjoint solve (sm_103a).
//
// Sec. VI names the implicit solution of the Poisson problem as the next
// step beyond the paper's explicit loop; A u = b is solved here by BiCGSTAB
// (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) with left Jacobi
// scaling D^-1 A u = D^-1 b.  Convergence is always judged on the unscaled
// residual |b - A u| <= tol |b|, re-computed explicitly at the end.
//
// One iteration = five kernels on the caller's stream:
//   update_p : p = r + beta (p - omega v)            (beta from device state)
//   spmv_v   : v = D^-1 A p,  partial (rh, v)        -> alpha
//   update_s : s = r - alpha v
//   spmv_t   : t = D^-1 A s,  partials (t,s), (t,t)  -> omega
//   update_xr: x += alpha p + omega s, r = s - omega t,
//              partials |D r|^2, (rh, r)             -> rho, stop test
// Scalars live in a device state block; each reduction is finished by the
// last block to arrive (fixed order over block partials, so results are
// deterministic for a given grid), so no iteration needs the host.  The
// host enqueues iterations in chunks and reads the 100-byte state between
// chunks; kernels of a finished solve return at once.
//
// SpMV: CSR, TPR lanes per row (TPR chosen from the mean row length so each
// lane streams several entries), matrix streams read with evict-first
// hints, gathered vector through L1/L2.  Mixed precision reads the float32
// copy of the values (8 bytes per entry instead of 12).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace rbffd {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 2048;
constexpr int kSlots = 6;
constexpr int kQ = 3;

enum Flag : int { kRunning = 0, kConverged = 1, kBreakdown = 2, kMaxIter = 3 };

struct KState {
    double rho, rho_new, alpha, omega;
    double bnorm2;  // |b|^2 of the system being iterated
    double tol2;    // stop when |r|^2 <= tol2 (unscaled)
    double rnorm2;  // last recurrence |r|^2 (unscaled)
    double tnorm2;  // last explicit residual |b - A x|^2
    int iter;
    int max_iter;
    int flag;
    int bad;        // input validation failure
    unsigned int counter[kSlots];
};

struct Work {
    KState* st;
    double* part;  // [kSlots][kQ][kMaxBlocks]
    double *r, *rh, *p, *v, *s, *t;
    double *d, *dinv;
    double *r_outer, *dx;
};

enum Slot { kSlotResid = 0, kSlotV = 1, kSlotT = 2, kSlotXR = 3, kSlotDiag = 4 };

__device__ __forceinline__ double* part_at(double* part, int slot, int q) {
    return part + ((size_t)slot * kQ + q) * kMaxBlocks;
}

// Block-reduce NQ values, store block partials, and let the last block to
// arrive sum all partials (returned in tot[]).  Returns true in that block.
template <int NQ>
__device__ bool reduce_last(double (&v)[NQ], double* part, int slot, unsigned int* counter, double (&tot)[NQ]) {
    __shared__ double sh[32];
    __shared__ unsigned int is_last;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double bs = block_sum<kThreads>(v[q], sh);
        if (threadIdx.x == 0) part_at(part, slot, q)[blockIdx.x] = bs;
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

template <class VT>
__device__ __forceinline__ double ld_val(const VT* p) {
    return (double)__ldcs(p);
}

// Sum of row `row` times x, TPR lanes cooperating (result valid in all of
// them).  All 32 lanes of the warp must call it together (shuffles); a lane
// group with valid == false contributes an empty row.
template <class VT, int TPR>
__device__ __forceinline__ double row_dot(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                          const VT* __restrict__ val, const double* __restrict__ x, int64_t row,
                                          int sub, bool valid) {
    int64_t a = 0, e = 0;
    if (valid) {
        a = row_ptr[row];
        e = row_ptr[row + 1];
    }
    double sum = 0.0;
#pragma unroll 4
    for (int64_t k = a + sub; k < e; k += TPR) sum = fma(ld_val(val + k), x[__ldcs(col + k)], sum);
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, TPR);
    return sum;
}

// ---- setup: diagonal, Jacobi scaling, validation ---------------------------
__global__ void __launch_bounds__(kThreads) diag_kernel(const int64_t* __restrict__ row_ptr,
                                                        const int* __restrict__ col, const double* __restrict__ val,
                                                        int64_t N, int64_t nnz, int jacobi, double* __restrict__ d,
                                                        double* __restrict__ dinv, KState* st) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = row_ptr[i], e = row_ptr[i + 1];
        double di = 0.0;
        if (a < 0 || e < a || e > nnz) {
            bad = 1;
        } else {
            for (int64_t k = a; k < e; ++k) {
                const int c = col[k];
                if ((unsigned)c >= (unsigned)N) bad = 1;
                if (c == (int)i) di = val[k];
            }
        }
        if (i == N - 1 && e != nnz) bad = 1;
        if (i == 0 && a != 0) bad = 1;
        const bool use = jacobi && di != 0.0 && isfinite(di);
        d[i] = use ? di : 1.0;
        dinv[i] = use ? 1.0 / di : 1.0;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->bad, 1);
}

// r = D^-1 (b - A x) (or unscaled when scale_out == 0); partials |b - A x|^2,
// |b|^2, |r|^2.  With init: rh = r, p = v = 0 and the iteration scalars are
// reset (rho_new = (rh, r)).
template <class VT, int TPR>
__global__ void __launch_bounds__(kThreads) residual_kernel(const int64_t* __restrict__ row_ptr,
                                                            const int* __restrict__ col, const VT* __restrict__ val,
                                                            int64_t N, const double* __restrict__ b,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ dinv, double* __restrict__ r,
                                                            int scale_out, int init, double* __restrict__ rh,
                                                            double* __restrict__ p, double* __restrict__ v,
                                                            double tol, int max_iter, KState* st, double* part) {
    const int sub = threadIdx.x & (TPR - 1);
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPR;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / TPR;
    const int64_t gw = g0 - (threadIdx.x & 31) / TPR;  // first group of this warp: loop bound is warp-uniform
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t base = gw; base < N; base += ng) {
        const int64_t i = base + (g0 - gw);
        const bool valid = i < N;
        const double ax = row_dot<VT, TPR>(row_ptr, col, val, x, i, sub, valid);
        if (valid && sub == 0) {
            const double bi = b[i];
            const double rt = bi - ax;
            const double ri = scale_out ? rt * dinv[i] : rt;
            r[i] = ri;
            if (init) {
                rh[i] = ri;
                p[i] = 0.0;
                v[i] = 0.0;
            }
            acc[0] = fma(rt, rt, acc[0]);
            acc[1] = fma(bi, bi, acc[1]);
            acc[2] = fma(ri, ri, acc[2]);
        }
    }
    double tot[3];
    if (reduce_last<3>(acc, part, kSlotResid, &st->counter[kSlotResid], tot) && threadIdx.x == 0) {
        st->tnorm2 = tot[0];
        if (init) {
            st->bnorm2 = tot[1];
            st->tol2 = tol * tol * tot[1];
            st->rnorm2 = tot[0];
            st->rho = 1.0;
            st->alpha = 1.0;
            st->omega = 1.0;
            st->rho_new = tot[2];
            st->iter = 0;
            st->max_iter = max_iter;
            int flag = kRunning;
            if (!(tot[0] <= st->tol2)) {
                if (!finite(tot[0]) || !finite(tot[2])) flag = kBreakdown;
                else if (max_iter <= 0) flag = kMaxIter;
            } else {
                flag = kConverged;
            }
            st->flag = flag;
        }
    }
}

__global__ void __launch_bounds__(kThreads) update_p_kernel(int64_t N, const double* __restrict__ r,
                                                            const double* __restrict__ v, double* __restrict__ p,
                                                            const KState* st) {
    if (st->flag != kRunning) return;
    const double beta = (st->rho_new / st->rho) * (st->alpha / st->omega);
    const double omega = st->omega;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
}

// y = D^-1 A xin; partial (rh, y) [NQ = 1] or (y, s), (y, y) [NQ = 2].
template <class VT, int TPR, int MODE>
__global__ void __launch_bounds__(kThreads) spmv_kernel(const int64_t* __restrict__ row_ptr,
                                                        const int* __restrict__ col, const VT* __restrict__ val,
                                                        int64_t N, const double* __restrict__ xin,
                                                        const double* __restrict__ dinv, double* __restrict__ y,
                                                        const double* __restrict__ other, KState* st, double* part) {
    if (st->flag != kRunning) return;
    const int sub = threadIdx.x & (TPR - 1);
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPR;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / TPR;
    const int64_t gw = g0 - (threadIdx.x & 31) / TPR;  // warp-uniform loop bound
    double acc[2] = {0.0, 0.0};
    for (int64_t base = gw; base < N; base += ng) {
        const int64_t i = base + (g0 - gw);
        const bool valid = i < N;
        const double ax = row_dot<VT, TPR>(row_ptr, col, val, xin, i, sub, valid);
        if (valid && sub == 0) {
            const double yi = ax * dinv[i];
            y[i] = yi;
            if (MODE == 0) {
                acc[0] = fma(other[i], yi, acc[0]);  // (rh, v)
            } else {
                acc[0] = fma(yi, xin[i], acc[0]);  // (t, s)
                acc[1] = fma(yi, yi, acc[1]);      // (t, t)
            }
        }
    }
    if (MODE == 0) {
        double a1[1] = {acc[0]}, tot[1];
        if (reduce_last<1>(a1, part, kSlotV, &st->counter[kSlotV], tot) && threadIdx.x == 0) {
            const double rv = tot[0];
            if (rv == 0.0 || !finite(rv)) {
                st->flag = kBreakdown;
            } else {
                st->alpha = st->rho_new / rv;
                st->rho = st->rho_new;
            }
        }
    } else {
        double tot[2];
        if (reduce_last<2>(acc, part, kSlotT, &st->counter[kSlotT], tot) && threadIdx.x == 0) {
            const double ts = tot[0], tt = tot[1];
            if (!finite(ts) || !finite(tt)) st->flag = kBreakdown;
            else st->omega = (tt > 0.0) ? ts / tt : 0.0;
        }
    }
}

__global__ void __launch_bounds__(kThreads) update_s_kernel(int64_t N, const double* __restrict__ r,
                                                            const double* __restrict__ v, double* __restrict__ s,
                                                            const KState* st) {
    if (st->flag != kRunning) return;
    const double alpha = st->alpha;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = fma(-alpha, v[i], r[i]);
}

__global__ void __launch_bounds__(kThreads) update_xr_kernel(int64_t N, double* __restrict__ x,
                                                             const double* __restrict__ p,
                                                             const double* __restrict__ s,
                                                             const double* __restrict__ t, double* __restrict__ r,
                                                             const double* __restrict__ rh,
                                                             const double* __restrict__ d, KState* st,
                                                             double* part) {
    if (st->flag != kRunning) return;
    const double alpha = st->alpha, omega = st->omega;
    double acc[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double si = s[i];
        x[i] = fma(omega, si, fma(alpha, p[i], x[i]));
        const double ri = fma(-omega, t[i], si);
        r[i] = ri;
        const double ru = ri * d[i];
        acc[0] = fma(ru, ru, acc[0]);
        acc[1] = fma(rh[i], ri, acc[1]);
    }
    double tot[2];
    if (reduce_last<2>(acc, part, kSlotXR, &st->counter[kSlotXR], tot) && threadIdx.x == 0) {
        const double rn2 = tot[0], rho_new = tot[1];
        st->rnorm2 = rn2;
        st->rho_new = rho_new;
        const int it = st->iter + 1;
        st->iter = it;
        int flag = kRunning;
        if (rn2 <= st->tol2) flag = kConverged;
        else if (!finite(rn2) || !finite(rho_new) || rho_new == 0.0 || st->omega == 0.0) flag = kBreakdown;
        else if (it >= st->max_iter) flag = kMaxIter;
        st->flag = flag;
    }
}

__global__ void axpy_kernel(int64_t N, double* __restrict__ x, const double* __restrict__ dx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += dx[i];
}

__global__ void adjoint_grad_kernel(int64_t N, const uint8_t* __restrict__ mask, const double* __restrict__ lam,
                                    double* __restrict__ dLdf, double* __restrict__ dLdg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const bool dir = mask[i] != 0;
        const double l = lam[i];
        if (dLdf) dLdf[i] = dir ? 0.0 : -l;
        if (dLdg) dLdg[i] = dir ? l : 0.0;
    }
}

// ---------------------------------------------------------------- host -----
Work carve(void* ws, int64_t N, bool mixed) {
    Carver c(ws);
    Work w;
    w.st = c.take<KState>(1);
    w.part = c.take<double>((size_t)kSlots * kQ * kMaxBlocks);
    w.r = c.take<double>(N);
    w.rh = c.take<double>(N);
    w.p = c.take<double>(N);
    w.v = c.take<double>(N);
    w.s = c.take<double>(N);
    w.t = c.take<double>(N);
    w.d = c.take<double>(N);
    w.dinv = c.take<double>(N);
    w.r_outer = mixed ? c.take<double>(N) : nullptr;
    w.dx = mixed ? c.take<double>(N) : nullptr;
    return w;
}

size_t work_bytes(int64_t N, bool mixed) {
    Carver c(nullptr);
    c.take<KState>(1);
    c.take<double>((size_t)kSlots * kQ * kMaxBlocks);
    for (int k = 0; k < 8; ++k) c.take<double>(N);
    if (mixed) {
        c.take<double>(N);
        c.take<double>(N);
    }
    return c.off;
}

int tpr_for(int64_t N, int64_t nnz) {
    const double L = (double)nnz / (double)std::max<int64_t>(N, 1);
    if (L <= 8) return 2;
    if (L <= 24) return 4;
    if (L <= 48) return 8;
    if (L <= 96) return 16;
    return 32;
}

int nblocks() { return std::min(kMaxBlocks, sm_count() * 8); }

template <class VT, int TPR>
struct Ops {
    static void residual(const rbffd_csr& A, const double* b, const double* x, const Work& w, double* r, int scale,
                         int init, double tol, int max_iter, cudaStream_t st) {
        residual_kernel<VT, TPR><<<nblocks(), kThreads, 0, st>>>(A.row_ptr, A.col, static_cast<const VT*>(A.val),
                                                                 A.n_rows, b, x, w.dinv, r, scale, init, w.rh, w.p,
                                                                 w.v, tol, max_iter, w.st, w.part);
        note_launches(1);
    }
    // Algorithmic bytes of one SpMV launch (see rbffd_profile in rbffd.h).
    static int64_t spmv_bytes(const rbffd_csr& A) {
        return A.nnz * (int64_t)(sizeof(VT) + 4) + 8 * (A.n_rows + 1) + 4 * 8 * A.n_rows;
    }
    static void iteration(const rbffd_csr& A, double* x, const Work& w, cudaStream_t st) {
        const int64_t N = A.n_rows;
        const int nb = nblocks();
        const VT* val = static_cast<const VT*>(A.val);
        const int kind = sizeof(VT) == 8 ? kProfSpmv64 : kProfSpmv32;
        const int64_t bytes = spmv_bytes(A);
        update_p_kernel<<<nb, kThreads, 0, st>>>(N, w.r, w.v, w.p, w.st);
        int ev = prof_begin(st);
        spmv_kernel<VT, TPR, 0><<<nb, kThreads, 0, st>>>(A.row_ptr, A.col, val, N, w.p, w.dinv, w.v, w.rh, w.st,
                                                         w.part);
        prof_end(ev, st, kind, bytes);
        update_s_kernel<<<nb, kThreads, 0, st>>>(N, w.r, w.v, w.s, w.st);
        ev = prof_begin(st);
        spmv_kernel<VT, TPR, 1><<<nb, kThreads, 0, st>>>(A.row_ptr, A.col, val, N, w.s, w.dinv, w.t, nullptr,
                                                         w.st, w.part);
        prof_end(ev, st, kind, bytes);
        update_xr_kernel<<<nb, kThreads, 0, st>>>(N, x, w.p, w.s, w.t, w.r, w.rh, w.d, w.st, w.part);
        note_launches(5);
    }
};

template <class VT>
void residual_dispatch(int tpr, const rbffd_csr& A, const double* b, const double* x, const Work& w, double* r,
                       int scale, int init, double tol, int max_iter, cudaStream_t st) {
    switch (tpr) {
        case 2: Ops<VT, 2>::residual(A, b, x, w, r, scale, init, tol, max_iter, st); break;
        case 4: Ops<VT, 4>::residual(A, b, x, w, r, scale, init, tol, max_iter, st); break;
        case 8: Ops<VT, 8>::residual(A, b, x, w, r, scale, init, tol, max_iter, st); break;
        case 16: Ops<VT, 16>::residual(A, b, x, w, r, scale, init, tol, max_iter, st); break;
        default: Ops<VT, 32>::residual(A, b, x, w, r, scale, init, tol, max_iter, st); break;
    }
}

template <class VT>
void iteration_dispatch(int tpr, const rbffd_csr& A, double* x, const Work& w, cudaStream_t st) {
    switch (tpr) {
        case 2: Ops<VT, 2>::iteration(A, x, w, st); break;
        case 4: Ops<VT, 4>::iteration(A, x, w, st); break;
        case 8: Ops<VT, 8>::iteration(A, x, w, st); break;
        case 16: Ops<VT, 16>::iteration(A, x, w, st); break;
        default: Ops<VT, 32>::iteration(A, x, w, st); break;
    }
}

int read_state(const Work& w, KState* hs, cudaStream_t st) {
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (profiling()) prof_collect();
    return RBFFD_OK;
}

// One BiCGSTAB run on A (values VT) for A x = b from the given x, to
// |b - A x| <= tol |b| by the recurrence residual.  Returns the final flag.
template <class VT>
int bicgstab_run(const rbffd_csr& A, const double* b, double* x, double tol, int max_iter, const Work& w,
                 cudaStream_t st, KState* hs) {
    const int tpr = tpr_for(A.n_rows, A.nnz);
    residual_dispatch<VT>(tpr, A, b, x, w, w.r, 1, 1, tol, max_iter, st);
    RBFFD_LAUNCH_CHECK();
    int chunk = 4;
    int rc = read_state(w, hs, st);
    if (rc != RBFFD_OK) return -rc;
    while (hs->flag == kRunning) {
        for (int c = 0; c < chunk; ++c) iteration_dispatch<VT>(tpr, A, x, w, st);
        RBFFD_LAUNCH_CHECK();
        rc = read_state(w, hs, st);
        if (rc != RBFFD_OK) return -rc;
        chunk = std::min(chunk * 2, 64);
    }
    return hs->flag;
}

bool csr_ok(const rbffd_csr* A, int dtype) {
    return A && A->row_ptr && A->col && A->val && A->dtype == dtype && A->n_rows > 0 &&
           A->n_rows <= 0x7fffffffLL && A->nnz >= 0;
}

int solve_impl(const rbffd_csr* A, const rbffd_csr* A32, const double* b, double* x, const rbffd_solve_opts* o,
               rbffd_solve_info* info, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!csr_ok(A, 0) || !b || !x || !o || !info) return RBFFD_ERR_INVALID_ARG;
    const bool mixed = o->precision == 1;
    if (o->precision != 0 && o->precision != 1) return RBFFD_ERR_INVALID_ARG;
    if (mixed && (!csr_ok(A32, 1) || A32->n_rows != A->n_rows || A32->nnz != A->nnz ||
                  A32->row_ptr != A->row_ptr || A32->col != A->col))
        return RBFFD_ERR_INVALID_ARG;  // the float32 copy shares A's (validated) pattern
    if (!(o->tol > 0.0) || o->max_iter < 0) return RBFFD_ERR_INVALID_ARG;
    if (mixed && (!(o->inner_tol > 0.0 && o->inner_tol < 1.0) || o->max_outer < 1)) return RBFFD_ERR_INVALID_ARG;
    const int64_t N = A->n_rows;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0 || ws_bytes < work_bytes(N, mixed)) return RBFFD_ERR_WORKSPACE;
    Work w = carve(ws, N, mixed);
    std::memset(info, 0, sizeof(*info));

    KState hs;
    RBFFD_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(KState), st));
    diag_kernel<<<std::min<int64_t>((N + kThreads - 1) / kThreads, sm_count() * 8), kThreads, 0, st>>>(
        A->row_ptr, A->col, static_cast<const double*>(A->val), N, A->nnz, o->jacobi ? 1 : 0, w.d, w.dinv, w.st);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    int rc = read_state(w, &hs, st);
    if (rc != RBFFD_OK) return rc;
    if (hs.bad) return RBFFD_ERR_INVALID_ARG;

    const int tpr = tpr_for(N, A->nnz);
    int total_iters = 0, restarts = 0, breakdowns = 0, outer = 0;
    const int max_outer = mixed ? o->max_outer : std::max(4, o->max_outer);
    int status = RBFFD_ERR_NOT_CONVERGED;
    double last_rel = INFINITY;
    while (true) {
        // explicit FP64 residual of the current x
        residual_dispatch<double>(tpr, *A, b, x, w, mixed ? w.r_outer : w.r, 0, 1, o->tol, 1, st);
        RBFFD_LAUNCH_CHECK();
        rc = read_state(w, &hs, st);
        if (rc != RBFFD_OK) return rc;
        const double rel = hs.bnorm2 > 0.0 ? std::sqrt(hs.tnorm2 / hs.bnorm2) : std::sqrt(hs.tnorm2);
        last_rel = rel;
        if (hs.bnorm2 == 0.0 && hs.tnorm2 == 0.0) { status = RBFFD_OK; last_rel = 0.0; break; }
        if (rel <= o->tol) { status = RBFFD_OK; break; }
        if (!std::isfinite(rel)) { status = RBFFD_ERR_BREAKDOWN; break; }
        if (total_iters >= o->max_iter || outer >= max_outer) { status = RBFFD_ERR_NOT_CONVERGED; break; }
        ++outer;
        int flag;
        const int budget = o->max_iter - total_iters;
        if (!mixed) {
            flag = bicgstab_run<double>(*A, b, x, o->tol, budget, w, st, &hs);
        } else {
            RBFFD_CUDA_TRY(cudaMemsetAsync(w.dx, 0, sizeof(double) * N, st));
            flag = bicgstab_run<float>(*A32, w.r_outer, w.dx, o->inner_tol, budget, w, st, &hs);
            if (flag >= 0) {
                axpy_kernel<<<nblocks(), kThreads, 0, st>>>(N, x, w.dx);
                note_launches(1);
                RBFFD_LAUNCH_CHECK();
            }
        }
        if (flag < 0) return -flag;
        total_iters += hs.iter;
        if (flag == kBreakdown) {
            if (++breakdowns >= 2) {
                // measure where we are before reporting
                residual_dispatch<double>(tpr, *A, b, x, w, w.r, 0, 1, o->tol, 1, st);
                rc = read_state(w, &hs, st);
                if (rc != RBFFD_OK) return rc;
                last_rel = hs.bnorm2 > 0.0 ? std::sqrt(hs.tnorm2 / hs.bnorm2) : std::sqrt(hs.tnorm2);
                status = last_rel <= o->tol ? RBFFD_OK : RBFFD_ERR_BREAKDOWN;
                break;
            }
            ++restarts;
        } else {
            breakdowns = 0;
            if (!mixed && flag == kConverged && outer > 1) ++restarts;
        }
    }
    info->status = status;
    info->iters = total_iters;
    info->outer_sweeps = outer;
    info->restarts = restarts;
    info->rel_residual = last_rel;
    return status;
}

}  // namespace
}  // namespace rbffd

extern "C" size_t rbffd_solve_workspace_size(int64_t N, const rbffd_solve_opts* opts) {
    if (N <= 0) return 0;
    const bool mixed = opts && opts->precision == 1;
    return rbffd::work_bytes(N, mixed);
}

extern "C" int rbffd_solve(const rbffd_csr* A, const rbffd_csr* A32, const double* b, double* x,
                           const rbffd_solve_opts* opts, rbffd_solve_info* info, void* ws, size_t ws_bytes,
                           void* stream) {
    return rbffd::solve_impl(A, A32, b, x, opts, info, ws, ws_bytes, rbffd::as_stream(stream));
}

extern "C" int rbffd_solve_adjoint(const rbffd_csr* AT, const rbffd_csr* AT32, const uint8_t* is_dirichlet,
                                   const double* dLdu, double* lambda, double* dLdf, double* dLdg,
                                   const rbffd_solve_opts* opts, rbffd_solve_info* info, void* ws, size_t ws_bytes,
                                   void* stream) {
    using namespace rbffd;
    if (!is_dirichlet && (dLdf || dLdg)) return RBFFD_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    const int rc = solve_impl(AT, AT32, dLdu, lambda, opts, info, ws, ws_bytes, st);
    if (rc != RBFFD_OK) return rc;
    if (dLdf || dLdg) {
        const int64_t N = AT->n_rows;
        adjoint_grad_kernel<<<std::min<int64_t>((N + 255) / 256, sm_count() * 8), 256, 0, st>>>(N, is_dirichlet,
                                                                                               lambda, dLdf, dLdg);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
    }
    return RBFFD_OK;
}
