// Batched pipeline: many independent node sets ("instances") of uneven size
// and degree, each with up to 64 right-hand sides, solved together (sm_103a).
//
// Per instance the method is the paper's (stencils, RBF-FD weights, the
// Poisson operator with Dirichlet rows; Sec. II Eq. 1, Sec. IV Eqs. 2-3, the
// implicit solve of Sec. VI); batching is this library's addition.
//
// Setup: stencils and weights per instance (the single-instance kernels on
// sub-arrays), then one block-diagonal CSR over all instances (a row-length
// scan and a warp-per-row fill that turns instance-local stencil indices
// into global columns) with float32 values, and b = -f | g for every rhs.
//
// Solve: the mixed solver of rbffd_solve -- an FP64 residual per (instance,
// rhs) pair, inner BiCGSTAB passes on the float32 matrix in difference form
// with double-float (2 x float32) vectors, x += correction in FP64 -- run for
// all pairs at once.  Vectors are node-major, [node][rhs]: a warp owns a row
// and its lanes own right-hand sides (lane, lane + 32), so every matrix entry
// is read once for all of an instance's right-hand sides and every gathered
// neighbour value is a coalesced 256-byte segment.  Rows are grouped in units
// of 256 consecutive rows of one instance; a block reduces its unit's dot
// products per rhs, and the last unit of an instance to finish turns the
// instance's unit partials (summed in unit order: deterministic) into that
// instance's per-rhs BiCGSTAB scalars.  Each pair has its own scalars and
// pass state; units of instances with no running pair return at once.  The
// host replays a CUDA graph of a chunk of inner iterations and reads one
// counter of running pairs between chunks -- no kernel ever waits on another
// block.
#include "common.cuh"
#include "df32.cuh"
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "scan.cuh"

#define RBFFD_CUDA_TRY_NEG(call)               \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) {               \
            ::rbffd::set_cuda_error(e_);       \
            return -(int)RBFFD_ERR_CUDA;       \
        }                                      \
    } while (0)

namespace rbffd {
namespace {

constexpr int kBT = 256;          // threads per block (8 warps)
constexpr int kSetupStreams = 8;  // instances' stencils and weights run on this many streams
constexpr int kUnitRows = 256;    // rows per unit (32 per warp)
constexpr int kMaxRhs = 64;
constexpr int kPassCap = 1500;    // inner iterations per pass at most
constexpr double kGrowth2 = 1e6;  // a pass whose scaled residual grows 1e3 ends

// Pair flags.
enum : int { kRun = 0, kPassEnd = 1, kDone = 2, kFail = 3 };

struct Inst {
    int64_t node_off, n_nodes, idx_off;
    int32_t n, m, unit_off, n_units;
};

struct Unit {
    int32_t inst;
    int32_t pad;
    int64_t row_lo, row_hi;  // global rows
};

// Per-pair state (structure of arrays, P = n_inst * R).
struct Pairs {
    double *rho, *rho_new, *alpha, *omega, *bn2, *tol2, *rn2, *tn2, *s0, *rstart2, *repl2;
    int *flag, *iters, *pass_iters;
};

struct Ctl {
    int running;      // pairs in an inner pass (all instances)
    int active;       // pairs not converged / failed
    int pad[2];
};

struct BWork {
    Inst* inst;
    Unit* units;
    int* inst_running;   // per instance: pairs in an inner pass
    unsigned* inst_cnt;  // per instance: units done in the current launch
    Ctl* ctl;
    double* part;        // [3][n_units][R]
    Pairs pr;
    int32_t* idx;
    double* w;
    int32_t* nstat;
    int64_t* row_ptr;
    int32_t* col;
    double* val;
    float* val32;
    int64_t* scan_sums;
    void* knn_ws;
    double *b, *r64;
    double *d, *dinv;
    float *d32, *dinv32, *sig32;
    float2 *xd, *r, *rh, *p, *v, *s, *t;
    // multigrid mode: FP64 Krylov vectors (r is r64), the preconditioned
    // directions, the float V-cycle's level-0 work vectors, the coarse-level
    // vectors and the per-instance hierarchies' workspaces
    double *mrh, *mp, *mv, *ms, *mt, *mph, *msh;  // used as float2 (double-float) vectors
    float2* mr;                                   // double-float residual
    float* val_lo;                                // val - val32, as float (val32 holds the leading part)
    float *f0, *f1, *f2;
    float* coarse;
    char* mgws;
    char* mbtab;  // device tables of the batched V-cycle
    size_t mbtab_bytes;
    int* loop;    // counters of the device-side loop (8 ints)
};

__device__ __forceinline__ int find_inst(const Inst* inst, int n_inst, int64_t row) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].node_off <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- setup ----
struct BRowLen {
    const Inst* inst;
    int n_inst;
    const uint8_t* mask;
    __device__ int64_t operator()(int64_t r) const {
        return mask[r] ? (int64_t)1 : (int64_t)inst[find_inst(inst, n_inst, r)].n;
    }
};

__global__ void __launch_bounds__(kBT) b_fill_kernel(const Inst* __restrict__ inst, int n_inst, int64_t N,
                                                     const uint8_t* __restrict__ mask,
                                                     const int32_t* __restrict__ idx, const double* __restrict__ w,
                                                     const int64_t* __restrict__ row_ptr, int64_t nnz_cap,
                                                     int32_t* __restrict__ col, double* __restrict__ val,
                                                     float* __restrict__ val32) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp0; r < N; r += nwarps) {
        const int ii = find_inst(inst, n_inst, r);
        const Inst in = inst[ii];
        const int64_t a = row_ptr[r];
        const bool dir = mask[r] != 0;
        const int len = dir ? 1 : in.n;
        if (a < 0 || a + len > nnz_cap) continue;
        if (dir) {
            if (lane == 0) {
                col[a] = (int32_t)r;
                val[a] = 1.0;
                val32[a] = 1.0f;
            }
        } else {
            const int64_t lr = r - in.node_off;
            const int32_t* si = idx + in.idx_off + lr * in.n;
            const double* wi = w + in.idx_off + lr * in.n;
            for (int j = lane; j < in.n; j += 32) {
                const double v = wi[j];
                col[a + j] = (int32_t)(si[j] + in.node_off);
                val[a + j] = v;
                val32[a + j] = __double2float_rn(v);
            }
        }
    }
}

__global__ void b_rhs_kernel(int64_t N, int R, const uint8_t* __restrict__ mask, const double* __restrict__ f,
                             const double* __restrict__ g, double* __restrict__ b) {
    const int64_t total = N * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = mask[e / R] ? g[e] : -f[e];
}

// Starting guess on the Dirichlet (identity) rows: u_b = b_b, so every
// residual is zero there (with nonzero boundary data, a Dirichlet part of
// the residual is coupled into the interior by a block of size ~1/h^2 of
// the preconditioned operator).
__global__ void b_dstart_kernel(int64_t N, int R, const uint8_t* __restrict__ mask, const double* __restrict__ b,
                                double* __restrict__ u) {
    const int64_t total = N * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        if (mask[e / R]) u[e] = b[e];
}

__global__ void b_diag_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, int64_t N, double* __restrict__ d,
                              double* __restrict__ dinv, float* __restrict__ d32, float* __restrict__ dinv32,
                              float* __restrict__ sig32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double di = 0.0, rs = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const double v = val[k];
            if (col[k] == (int32_t)i) di = v;
            rs += v;
        }
        const bool use = di != 0.0 && isfinite(di);
        d[i] = use ? di : 1.0;
        dinv[i] = use ? 1.0 / di : 1.0;
        d32[i] = __double2float_rn(use ? di : 1.0);
        dinv32[i] = __double2float_rn(use ? 1.0 / di : 1.0);
        sig32[i] = __double2float_rn(rs);
    }
}

// ------------------------------------------------------------- reductions --
// Reduce NQ per-lane values (for rhs lane and lane + 32) over the block's 8
// warps and store them as the unit's partials [q][unit][rhs].
template <int NQ>
__device__ void unit_store(const double (&v0)[NQ], const double (&v1)[NQ], double* part, int n_units, int R,
                           int unit) {
    __shared__ double sh[NQ][8][kMaxRhs];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        sh[q][wid][lane] = v0[q];
        sh[q][wid][lane + 32] = v1[q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NQ * R; e += blockDim.x) {
        const int q = e / R, k = e - (e / R) * R;
        double acc = 0.0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) acc += sh[q][ww][k];
        part[((size_t)q * n_units + unit) * R + k] = acc;
    }
    __syncthreads();
}

// True in the block that finished the last unit of instance `ii`.
__device__ bool last_unit(unsigned* cnt, int n_units_inst) {
    __shared__ unsigned last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(cnt, 1u) == (unsigned)n_units_inst - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    if (threadIdx.x == 0) *cnt = 0u;
    return true;
}

// Sum of the instance's unit partials for quantity q, rhs k (unit order).
__device__ __forceinline__ double inst_sum(const double* part, int n_units, int R, int q, const Inst& in, int k) {
    double acc = 0.0;
    for (int u = 0; u < in.n_units; ++u) acc += __ldcg(part + ((size_t)q * n_units + in.unit_off + u) * R + k);
    return acc;
}

// --------------------------------------------------------------- kernels ---
// FP64 residual r64 = b - A x for every pair of instances with active pairs;
// finalises per pair: converged when |r|^2 <= tol^2 |b|^2.
__global__ void __launch_bounds__(kBT) b_check_kernel(const Unit* __restrict__ units, int n_units,
                                                      const Inst* __restrict__ inst, const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, const double* __restrict__ val,
                                                      int R, const double* __restrict__ b,
                                                      const double* __restrict__ x, const double* __restrict__ dinv,
                                                      double* __restrict__ r64, Pairs pr, unsigned* inst_cnt,
                                                      Ctl* ctl, double* part, double tol) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k0 = lane, k1 = lane + 32;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        const Inst in = inst[un.inst];
        RB_SPAN(un.row_lo - in.node_off, un.row_hi - un.row_lo, in.n_nodes);
        // the instance's block of x (the bound of the checked build's tests)
        const double* xb = x + in.node_off * R;
        const int64_t xn = in.n_nodes * R;
        (void)xb;
        (void)xn;
        // skip instances whose pairs are all finished
        bool any = false;
        for (int k = 0; k < R; ++k) {
            const int f = pr.flag[un.inst * R + k];
            any |= (f != kDone && f != kFail);
        }
        if (!any) continue;
        double a0[3] = {0.0, 0.0, 0.0}, a1[3] = {0.0, 0.0, 0.0};
        for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
            const int64_t lo = row_ptr[row], hi = row_ptr[row + 1];
            double s0 = 0.0, s1 = 0.0;
            for (int64_t q = lo; q < hi; ++q) {
                const double a = __ldg(val + q);
                const int64_t c = (int64_t)__ldg(col + q) * R;
                if (k0 < R) s0 = fma(a, RB_PT(x + c + k0, xb, xn), s0);
                if (k1 < R) s1 = fma(a, RB_PT(x + c + k1, xb, xn), s1);
            }
            const double di = dinv[row];
            if (k0 < R) {
                const double bi = b[row * R + k0], rt = bi - s0, rs = rt * di;
                r64[row * R + k0] = rt;
                a0[0] = fma(rt, rt, a0[0]);
                a0[1] = fma(bi, bi, a0[1]);
                a0[2] = fma(rs, rs, a0[2]);
            }
            if (k1 < R) {
                const double bi = b[row * R + k1], rt = bi - s1, rs = rt * di;
                r64[row * R + k1] = rt;
                a1[0] = fma(rt, rt, a1[0]);
                a1[1] = fma(bi, bi, a1[1]);
                a1[2] = fma(rs, rs, a1[2]);
            }
        }
        unit_store<3>(a0, a1, part, n_units, R, u);
        if (last_unit(&inst_cnt[un.inst], in.n_units)) {
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int pi = un.inst * R + k;
                const int f = pr.flag[pi];
                if (f == kDone || f == kFail) continue;
                const double tn = inst_sum(part, n_units, R, 0, in, k), bn = inst_sum(part, n_units, R, 1, in, k);
                pr.tn2[pi] = tn;
                pr.bn2[pi] = bn;
                pr.rstart2[pi] = inst_sum(part, n_units, R, 2, in, k);
                pr.tol2[pi] = tol * tol * bn;
                const bool conv = tn <= tol * tol * bn;
                pr.flag[pi] = conv ? kDone : (isfinite(tn) ? kPassEnd : kFail);
                if (!conv && isfinite(tn)) atomicAdd(&ctl->active, 1);
            }
        }
    }
}

// Inner pass start for active pairs: r = D^-1 r64 (df32), rh pseudo-random, p = v = 0,
// correction 0; scalars reset; the pass ends when |D r| < inner_tol |r64|.
__global__ void __launch_bounds__(kBT) b_load_kernel(const Unit* __restrict__ units, int n_units,
                                                     const Inst* __restrict__ inst, int R,
                                                     const double* __restrict__ r64,
                                                     const float* __restrict__ dinv32, float2* __restrict__ rr,
                                                     float2* __restrict__ rh, float2* __restrict__ p,
                                                     float2* __restrict__ v, float2* __restrict__ xd, Pairs pr,
                                                     unsigned* inst_cnt, int* inst_running, Ctl* ctl, double* part,
                                                     double inner_tol, int max_iter, unsigned long long seed) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k0 = lane, k1 = lane + 32;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        const Inst in = inst[un.inst];
        RB_SPAN(un.row_lo - in.node_off, un.row_hi - un.row_lo, in.n_nodes);
        bool any = false;
        for (int k = 0; k < R; ++k) any |= pr.flag[un.inst * R + k] == kPassEnd;
        if (!any) continue;
        const bool on0 = k0 < R && pr.flag[un.inst * R + k0] == kPassEnd;
        const bool on1 = k1 < R && pr.flag[un.inst * R + k1] == kPassEnd;
        // shadow residual: pseudo-random per (row, rhs) -- see load_df_kernel
        DfAcc c0, c1, h0, h1;
        for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
            const float di = dinv32[row];
            if (on0) {
                const int64_t e = row * R + k0;
                const df ri = df_mul_f(df_from_double(r64[e]), di);
                const df hi = df_make(shadow_value(seed, e), 0.f);
                df_store(rr + e, ri);
                df_store(rh + e, hi);
                p[e] = v[e] = xd[e] = make_float2(0.f, 0.f);
                c0.add(df_mul(ri, ri));
                h0.add(df_mul(hi, ri));
            }
            if (on1) {
                const int64_t e = row * R + k1;
                const df ri = df_mul_f(df_from_double(r64[e]), di);
                const df hi = df_make(shadow_value(seed, e), 0.f);
                df_store(rr + e, ri);
                df_store(rh + e, hi);
                p[e] = v[e] = xd[e] = make_float2(0.f, 0.f);
                c1.add(df_mul(ri, ri));
                h1.add(df_mul(hi, ri));
            }
        }
        double a0[2] = {df_to_double(c0.value()), df_to_double(h0.value())};
        double a1[2] = {df_to_double(c1.value()), df_to_double(h1.value())};
        unit_store<2>(a0, a1, part, n_units, R, u);
        if (last_unit(&inst_cnt[un.inst], in.n_units)) {
            int running = 0;
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int pi = un.inst * R + k;
                if (pr.flag[pi] != kPassEnd) continue;
                if (pr.iters[pi] >= max_iter) {
                    pr.flag[pi] = kFail;
                    continue;
                }
                const double rr2 = inst_sum(part, n_units, R, 0, in, k);
                const double hr = inst_sum(part, n_units, R, 1, in, k);
                pr.rho[pi] = pr.alpha[pi] = pr.omega[pi] = 1.0;
                pr.rho_new[pi] = hr;
                pr.s0[pi] = rr2;
                pr.rn2[pi] = pr.tn2[pi];
                pr.repl2[pi] = inner_tol * inner_tol;
                pr.pass_iters[pi] = 0;
                pr.flag[pi] = (rr2 > 0.0 && isfinite(rr2) && hr != 0.0 && isfinite(hr)) ? kRun : kFail;
                running += pr.flag[pi] == kRun;
            }
            // per-instance running count (threads < R each handled one pair)
            __shared__ int cnt;
            if (threadIdx.x == 0) cnt = 0;
            __syncthreads();
            if (running) atomicAdd(&cnt, running);
            __syncthreads();
            if (threadIdx.x == 0) {
                inst_running[un.inst] = cnt;
                atomicAdd(&ctl->running, cnt);
            }
        }
    }
}

__device__ __forceinline__ bool inst_live(const int* inst_running, int ii) { return inst_running[ii] > 0; }

// Block-wide: `ended` pairs (summed over threads) left their inner pass.
__device__ void end_pairs(int ended, int* inst_running, Ctl* ctl) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    if (ended) atomicAdd(&cnt, ended);
    __syncthreads();
    if (threadIdx.x == 0 && cnt) {
        *inst_running -= cnt;
        atomicSub(&ctl->running, cnt);
    }
}

__global__ void __launch_bounds__(kBT) b_update_p_kernel(const Unit* __restrict__ units, int n_units, int R,
                                                         const float2* __restrict__ rr, const float2* __restrict__ v,
                                                         float2* __restrict__ p, Pairs pr,
                                                         const int* __restrict__ inst_running) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= R) continue;
            const int pi = un.inst * R + k;
            if (pr.flag[pi] != kRun) continue;
            const df beta = df_from_double((pr.rho_new[pi] / pr.rho[pi]) * (pr.alpha[pi] / pr.omega[pi]));
            const df nom = df_from_double(-pr.omega[pi]);
            for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
                const int64_t e = row * R + k;
                const df t = df_fma(nom, df_load(v + e), df_load(p + e));
                df_store(p + e, df_fma(beta, t, df_load(rr + e)));
            }
        }
    }
}

// y = D^-1 A32 xin (difference form), MODE 0: (rh, y) -> alpha; MODE 1:
// (y, xin), (y, y) -> omega.
template <int MODE>
__global__ void __launch_bounds__(kBT) b_spmm_kernel(const Unit* __restrict__ units, int n_units,
                                                     const Inst* __restrict__ inst,
                                                     const int64_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col, const float* __restrict__ val,
                                                     int R, const float2* __restrict__ xin,
                                                     const float* __restrict__ sig, const float* __restrict__ dinv,
                                                     float2* __restrict__ y, const float2* __restrict__ rh, Pairs pr,
                                                     int* __restrict__ inst_running, unsigned* inst_cnt, Ctl* ctl,
                                                     double* part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k0 = lane, k1 = lane + 32;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
        const Inst in = inst[un.inst];
        RB_SPAN(un.row_lo - in.node_off, un.row_hi - un.row_lo, in.n_nodes);
        // the instance's block of xin (the bound of the checked build's tests)
        const float2* xb = xin + in.node_off * R;
        const int64_t xn = in.n_nodes * R;
        (void)xb;
        (void)xn;
        const bool on0 = k0 < R && pr.flag[un.inst * R + k0] == kRun;
        const bool on1 = k1 < R && pr.flag[un.inst * R + k1] == kRun;
        DfAcc c0a, c0b, c1a, c1b;
        for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
            const int64_t lo = row_ptr[row], hi = row_ptr[row + 1];
            const df x0 = on0 ? df_load(xin + row * R + k0) : df_make(0.f, 0.f);
            const df x1 = on1 ? df_load(xin + row * R + k1) : df_make(0.f, 0.f);
            DfAcc s0, s1;
            for (int64_t q = lo; q < hi; ++q) {
                const float w = __ldg(val + q);
                const int64_t c = (int64_t)__ldg(col + q) * R;
                if (on0) {
                    const df xj = df_load(&RB_PT(xin + c + k0, xb, xn));
                    df pp = two_prod(w, __fsub_rn(xj.hi, x0.hi));
                    pp.lo = __fmaf_rn(w, __fsub_rn(xj.lo, x0.lo), pp.lo);
                    s0.add(pp);
                }
                if (on1) {
                    const df xj = df_load(&RB_PT(xin + c + k1, xb, xn));
                    df pp = two_prod(w, __fsub_rn(xj.hi, x1.hi));
                    pp.lo = __fmaf_rn(w, __fsub_rn(xj.lo, x1.lo), pp.lo);
                    s1.add(pp);
                }
            }
            const float sg = sig[row], di = dinv[row];
            if (on0) {
                const df yv = df_mul_f(df_add(s0.value(), df_mul_f(x0, sg)), di);
                df_store(y + row * R + k0, yv);
                if (MODE == 0) c0a.add(df_mul(df_load(rh + row * R + k0), yv));
                else {
                    c0a.add(df_mul(yv, x0));
                    c0b.add(df_mul(yv, yv));
                }
            }
            if (on1) {
                const df yv = df_mul_f(df_add(s1.value(), df_mul_f(x1, sg)), di);
                df_store(y + row * R + k1, yv);
                if (MODE == 0) c1a.add(df_mul(df_load(rh + row * R + k1), yv));
                else {
                    c1a.add(df_mul(yv, x1));
                    c1b.add(df_mul(yv, yv));
                }
            }
        }
        double a0[2] = {df_to_double(c0a.value()), df_to_double(c0b.value())};
        double a1[2] = {df_to_double(c1a.value()), df_to_double(c1b.value())};
        unit_store<2>(a0, a1, part, n_units, R, u);
        if (last_unit(&inst_cnt[un.inst], in.n_units)) {
            int ended = 0;
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int pi = un.inst * R + k;
                if (pr.flag[pi] != kRun) continue;
                const double q0 = inst_sum(part, n_units, R, 0, in, k);
                bool brk = false;
                if (MODE == 0) {
                    if (q0 == 0.0 || !isfinite(q0)) {
                        brk = true;
                    } else {
                        pr.alpha[pi] = pr.rho_new[pi] / q0;
                        pr.rho[pi] = pr.rho_new[pi];
                    }
                } else {
                    const double q1 = inst_sum(part, n_units, R, 1, in, k);
                    if (!isfinite(q0) || !isfinite(q1)) brk = true;
                    else pr.omega[pi] = (q1 > 0.0) ? q0 / q1 : 0.0;
                }
                if (brk) {  // breakdown: the pass ends here
                    pr.flag[pi] = kPassEnd;
                    ++ended;
                }
            }
            end_pairs(ended, inst_running + un.inst, ctl);
        }
    }
}

__global__ void __launch_bounds__(kBT) b_update_s_kernel(const Unit* __restrict__ units, int n_units, int R,
                                                         const float2* __restrict__ rr, const float2* __restrict__ v,
                                                         float2* __restrict__ s, Pairs pr,
                                                         const int* __restrict__ inst_running) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= R) continue;
            const int pi = un.inst * R + k;
            if (pr.flag[pi] != kRun) continue;
            const df na = df_from_double(-pr.alpha[pi]);
            for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
                const int64_t e = row * R + k;
                df_store(s + e, df_fma(na, df_load(v + e), df_load(rr + e)));
            }
        }
    }
}

__global__ void __launch_bounds__(kBT) b_update_xr_kernel(const Unit* __restrict__ units, int n_units,
                                                          const Inst* __restrict__ inst, int R,
                                                          float2* __restrict__ xd, const float2* __restrict__ p,
                                                          const float2* __restrict__ s, const float2* __restrict__ t,
                                                          float2* __restrict__ rr, const float2* __restrict__ rh,
                                                          const float* __restrict__ d32, Pairs pr,
                                                          int* __restrict__ inst_running, unsigned* inst_cnt, Ctl* ctl,
                                                          double* part, int max_iter) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
        const Inst in = inst[un.inst];
        RB_SPAN(un.row_lo - in.node_off, un.row_hi - un.row_lo, in.n_nodes);
        double a[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= R) continue;
            const int pi = un.inst * R + k;
            if (pr.flag[pi] != kRun) continue;
            const df al = df_from_double(pr.alpha[pi]), om = df_from_double(pr.omega[pi]);
            const df nom = df_from_double(-pr.omega[pi]);
            DfAcc c0, c1, c2;
            for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
                const int64_t e = row * R + k;
                const df si = df_load(s + e);
                df_store(xd + e, df_fma(om, si, df_fma(al, df_load(p + e), df_load(xd + e))));
                const df ri = df_fma(nom, df_load(t + e), si);
                df_store(rr + e, ri);
                const df ru = df_mul_f(ri, d32[row]);
                c0.add(df_mul(ru, ru));
                c1.add(df_mul(df_load(rh + e), ri));
                c2.add(df_mul(ri, ri));
            }
            a[h][0] = df_to_double(c0.value());
            a[h][1] = df_to_double(c1.value());
            a[h][2] = df_to_double(c2.value());
        }
        unit_store<3>(a[0], a[1], part, n_units, R, u);
        if (last_unit(&inst_cnt[un.inst], in.n_units)) {
            int ended = 0;
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int pi = un.inst * R + k;
                if (pr.flag[pi] != kRun) continue;
                const double rn2 = inst_sum(part, n_units, R, 0, in, k);
                const double rho_new = inst_sum(part, n_units, R, 1, in, k);
                const double sn2 = inst_sum(part, n_units, R, 2, in, k);
                pr.rn2[pi] = rn2;
                pr.rho_new[pi] = rho_new;
                pr.iters[pi] += 1;
                pr.pass_iters[pi] += 1;
                bool end = false;
                if (!isfinite(rn2) || !isfinite(rho_new) || rho_new == 0.0 || pr.omega[pi] == 0.0) end = true;
                else if (rn2 < pr.repl2[pi] * pr.tn2[pi]) end = true;
                else if (!(sn2 <= kGrowth2 * pr.s0[pi])) end = true;
                else if (pr.pass_iters[pi] >= kPassCap || pr.iters[pi] >= max_iter) end = true;
                if (end) {
                    pr.flag[pi] = kPassEnd;
                    ++ended;
                }
            }
            end_pairs(ended, inst_running + un.inst, ctl);
        }
    }
}

// x += correction for pairs whose pass just ended; correction = 0.
__global__ void __launch_bounds__(kBT) b_refine_kernel(const Unit* __restrict__ units, int n_units, int R,
                                                       double* __restrict__ x, float2* __restrict__ xd, Pairs pr) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= R) continue;
            const int pi = un.inst * R + k;
            if (pr.flag[pi] != kPassEnd) continue;
            for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
                const int64_t e = row * R + k;
                const float2 c = xd[e];
                x[e] += (double)c.x + (double)c.y;
                xd[e] = make_float2(0.f, 0.f);
            }
        }
    }
}

// ------------------------------------------------------ multigrid mode -----
// Every (instance, rhs) pair runs BiCGSTAB right-preconditioned by its
// instance's float32 V-cycle (applied to all of the instance's right-hand
// sides at once); passes start from the explicit FP64 residual of b_check
// (r = r64, rh = r, p = v = 0).

// ---- double-float outer solve (multigrid mode) ----------------------------
// The outer BiCGSTAB of the multigrid mode keeps its vectors as double-float
// pairs and reads the matrix as (val32, val_lo) float pairs, so the 64-rhs
// SpMM runs on the FP32 pipe (one FP64 multiply-add per matrix entry and rhs
// would make it FP64-bound on this chip) at ~1e-14 relative accuracy; the
// solution x stays FP64 and the explicit FP64 residual of b_check decides
// convergence.

__global__ void __launch_bounds__(kBT) md_split_kernel(const double* __restrict__ val, const float* __restrict__ hi,
                                                       int64_t nnz, float* __restrict__ lo) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        lo[k] = __double2float_rn(val[k] - (double)hi[k]);
}

__global__ void __launch_bounds__(kBT) md_load_kernel(const Unit* __restrict__ units, int n_units,
                                                      const Inst* __restrict__ inst, int R,
                                                      const double* __restrict__ r64, float2* __restrict__ rr,
                                                      float2* __restrict__ rh, float2* __restrict__ p,
                                                      float2* __restrict__ v, Pairs pr, unsigned* inst_cnt,
                                                      int* inst_running, Ctl* ctl, double* part, double inner_tol,
                                                      int max_iter, const int* gate) {
    if (gate && *(volatile const int*)gate == 0) return;  // the device loop decided to stop
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k0 = lane, k1 = lane + 32;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        const Inst in = inst[un.inst];
        RB_SPAN(un.row_lo - in.node_off, un.row_hi - un.row_lo, in.n_nodes);
        bool any = false;
        for (int k = 0; k < R; ++k) any |= pr.flag[un.inst * R + k] == kPassEnd;
        if (!any) continue;
        const bool on0 = k0 < R && pr.flag[un.inst * R + k0] == kPassEnd;
        const bool on1 = k1 < R && pr.flag[un.inst * R + k1] == kPassEnd;
        DfAcc c0, c1;
        for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
            if (on0) {
                const int64_t e = row * R + k0;
                const df ri = df_from_double(r64[e]);
                df_store(rr + e, ri);
                df_store(rh + e, ri);
                p[e] = v[e] = make_float2(0.f, 0.f);
                c0.add(df_mul(ri, ri));
            }
            if (on1) {
                const int64_t e = row * R + k1;
                const df ri = df_from_double(r64[e]);
                df_store(rr + e, ri);
                df_store(rh + e, ri);
                p[e] = v[e] = make_float2(0.f, 0.f);
                c1.add(df_mul(ri, ri));
            }
        }
        double a0[1] = {df_to_double(c0.value())}, a1[1] = {df_to_double(c1.value())};
        unit_store<1>(a0, a1, part, n_units, R, u);
        if (last_unit(&inst_cnt[un.inst], in.n_units)) {
            int running = 0;
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int pi = un.inst * R + k;
                if (pr.flag[pi] != kPassEnd) continue;
                if (pr.iters[pi] >= max_iter) {
                    pr.flag[pi] = kFail;
                    continue;
                }
                const double rr2 = inst_sum(part, n_units, R, 0, in, k);
                pr.rho[pi] = pr.alpha[pi] = pr.omega[pi] = 1.0;
                pr.rho_new[pi] = rr2;
                pr.s0[pi] = rr2;
                pr.rn2[pi] = pr.tn2[pi];
                pr.repl2[pi] = inner_tol * inner_tol;
                pr.pass_iters[pi] = 0;
                pr.flag[pi] = (rr2 > 0.0 && isfinite(rr2)) ? kRun : kFail;
                running += pr.flag[pi] == kRun;
            }
            __shared__ int cnt;
            if (threadIdx.x == 0) cnt = 0;
            __syncthreads();
            if (running) atomicAdd(&cnt, running);
            __syncthreads();
            if (threadIdx.x == 0) {
                inst_running[un.inst] = cnt;
                atomicAdd(&ctl->running, cnt);
            }
        }
    }
}

__global__ void __launch_bounds__(kBT) md_update_p_kernel(const Unit* __restrict__ units, int n_units, int R,
                                                          const float2* __restrict__ rr, const float2* __restrict__ v,
                                                          float2* __restrict__ p, Pairs pr,
                                                          const int* __restrict__ inst_running) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= R) continue;
            const int pi = un.inst * R + k;
            if (pr.flag[pi] != kRun) continue;
            const df beta = df_from_double((pr.rho_new[pi] / pr.rho[pi]) * (pr.alpha[pi] / pr.omega[pi]));
            const df nom = df_from_double(-pr.omega[pi]);
            for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
                const int64_t e = row * R + k;
                const df t = df_fma(nom, df_load(v + e), df_load(p + e));
                df_store(p + e, df_fma(beta, t, df_load(rr + e)));
            }
        }
    }
}

// y = A xin with A as (hi, lo) float pairs; MODE 0: (rh, y) -> alpha;
// MODE 1: (y, s), (y, y) -> omega.
template <int MODE>
__global__ void __launch_bounds__(kBT) md_spmm_kernel(const Unit* __restrict__ units, int n_units,
                                                      const Inst* __restrict__ inst,
                                                      const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, const float* __restrict__ vhi,
                                                      const float* __restrict__ vlo, int R,
                                                      const float2* __restrict__ xin, float2* __restrict__ y,
                                                      const float2* __restrict__ dotv, Pairs pr,
                                                      int* __restrict__ inst_running, unsigned* inst_cnt, Ctl* ctl,
                                                      double* part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k0 = lane, k1 = lane + 32;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
        const Inst in = inst[un.inst];
        RB_SPAN(un.row_lo - in.node_off, un.row_hi - un.row_lo, in.n_nodes);
        // the instance's block of xin (the bound of the checked build's tests)
        const float2* xb = xin + in.node_off * R;
        const int64_t xn = in.n_nodes * R;
        (void)xb;
        (void)xn;
        const bool on0 = k0 < R && pr.flag[un.inst * R + k0] == kRun;
        const bool on1 = k1 < R && pr.flag[un.inst * R + k1] == kRun;
        DfAcc c0a, c0b, c1a, c1b;
        for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
            const int64_t lo = row_ptr[row], hi = row_ptr[row + 1];
            DfAcc s0, s1;
            int64_t q = lo;
            // four entries at a time: their indices, then their gathers in
            // flight together (the same sums, in the same order)
            for (; q + 4 <= hi; q += 4) {
                float ah[4], al[4];
                int64_t c[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ah[i] = __ldg(vhi + q + i);
                    al[i] = __ldg(vlo + q + i);
                    c[i] = (int64_t)__ldg(col + q + i) * R;
                }
                df x0[4], x1[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    x0[i] = on0 ? df_load(&RB_PT(xin + c[i] + k0, xb, xn)) : df_make(0.f, 0.f);
                    x1[i] = on1 ? df_load(&RB_PT(xin + c[i] + k1, xb, xn)) : df_make(0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (on0) {
                        df pp = two_prod(ah[i], x0[i].hi);
                        pp.lo = __fmaf_rn(ah[i], x0[i].lo, __fmaf_rn(al[i], x0[i].hi, pp.lo));
                        s0.add(pp);
                    }
                    if (on1) {
                        df pp = two_prod(ah[i], x1[i].hi);
                        pp.lo = __fmaf_rn(ah[i], x1[i].lo, __fmaf_rn(al[i], x1[i].hi, pp.lo));
                        s1.add(pp);
                    }
                }
            }
            for (; q < hi; ++q) {
                const float ah = __ldg(vhi + q), al = __ldg(vlo + q);
                const int64_t c = (int64_t)__ldg(col + q) * R;
                if (on0) {
                    const df xj = df_load(&RB_PT(xin + c + k0, xb, xn));
                    df pp = two_prod(ah, xj.hi);
                    pp.lo = __fmaf_rn(ah, xj.lo, __fmaf_rn(al, xj.hi, pp.lo));
                    s0.add(pp);
                }
                if (on1) {
                    const df xj = df_load(&RB_PT(xin + c + k1, xb, xn));
                    df pp = two_prod(ah, xj.hi);
                    pp.lo = __fmaf_rn(ah, xj.lo, __fmaf_rn(al, xj.hi, pp.lo));
                    s1.add(pp);
                }
            }
            if (on0) {
                const int64_t e = row * R + k0;
                const df yv = s0.value();
                df_store(y + e, yv);
                if (MODE == 0) c0a.add(df_mul(df_load(dotv + e), yv));
                else {
                    c0a.add(df_mul(yv, df_load(dotv + e)));
                    c0b.add(df_mul(yv, yv));
                }
            }
            if (on1) {
                const int64_t e = row * R + k1;
                const df yv = s1.value();
                df_store(y + e, yv);
                if (MODE == 0) c1a.add(df_mul(df_load(dotv + e), yv));
                else {
                    c1a.add(df_mul(yv, df_load(dotv + e)));
                    c1b.add(df_mul(yv, yv));
                }
            }
        }
        double a0[2] = {df_to_double(c0a.value()), df_to_double(c0b.value())};
        double a1[2] = {df_to_double(c1a.value()), df_to_double(c1b.value())};
        unit_store<2>(a0, a1, part, n_units, R, u);
        if (last_unit(&inst_cnt[un.inst], in.n_units)) {
            int ended = 0;
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int pi = un.inst * R + k;
                if (pr.flag[pi] != kRun) continue;
                const double q0 = inst_sum(part, n_units, R, 0, in, k);
                bool brk = false;
                if (MODE == 0) {
                    if (q0 == 0.0 || !isfinite(q0)) {
                        brk = true;
                    } else {
                        pr.alpha[pi] = pr.rho_new[pi] / q0;
                        pr.rho[pi] = pr.rho_new[pi];
                    }
                } else {
                    const double q1 = inst_sum(part, n_units, R, 1, in, k);
                    if (!isfinite(q0) || !isfinite(q1)) brk = true;
                    else pr.omega[pi] = (q1 > 0.0) ? q0 / q1 : 0.0;
                }
                if (brk) {
                    pr.flag[pi] = kPassEnd;
                    ++ended;
                }
            }
            end_pairs(ended, inst_running + un.inst, ctl);
        }
    }
}

__global__ void __launch_bounds__(kBT) md_update_s_kernel(const Unit* __restrict__ units, int n_units, int R,
                                                          const float2* __restrict__ rr, const float2* __restrict__ v,
                                                          float2* __restrict__ s, Pairs pr,
                                                          const int* __restrict__ inst_running) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= R) continue;
            const int pi = un.inst * R + k;
            if (pr.flag[pi] != kRun) continue;
            const df na = df_from_double(-pr.alpha[pi]);
            for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
                const int64_t e = row * R + k;
                df_store(s + e, df_fma(na, df_load(v + e), df_load(rr + e)));
            }
        }
    }
}

// x (FP64) += alpha ph + omega sh, r = s - omega t (double-float).
__global__ void __launch_bounds__(kBT) md_update_xr_kernel(const Unit* __restrict__ units, int n_units,
                                                           const Inst* __restrict__ inst, int R,
                                                           double* __restrict__ x, const float2* __restrict__ ph,
                                                           const float2* __restrict__ sh, const float2* __restrict__ s,
                                                           const float2* __restrict__ t, float2* __restrict__ rr,
                                                           const float2* __restrict__ rh, Pairs pr,
                                                           int* __restrict__ inst_running, unsigned* inst_cnt,
                                                           Ctl* ctl, double* part, int max_iter) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        if (!inst_live(inst_running, un.inst)) continue;
        const Inst in = inst[un.inst];
        RB_SPAN(un.row_lo - in.node_off, un.row_hi - un.row_lo, in.n_nodes);
        double a[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= R) continue;
            const int pi = un.inst * R + k;
            if (pr.flag[pi] != kRun) continue;
            const double al = pr.alpha[pi], om = pr.omega[pi];
            const df nom = df_from_double(-om);
            DfAcc c0, c1;
            for (int64_t row = un.row_lo + wid; row < un.row_hi; row += 8) {
                const int64_t e = row * R + k;
                const float2 pv = ph[e], sv = sh[e];
                x[e] = fma(om, (double)sv.x + (double)sv.y, fma(al, (double)pv.x + (double)pv.y, x[e]));
                const df ri = df_fma(nom, df_load(t + e), df_load(s + e));
                df_store(rr + e, ri);
                c0.add(df_mul(ri, ri));
                c1.add(df_mul(df_load(rh + e), ri));
            }
            a[h][0] = df_to_double(c0.value());
            a[h][1] = df_to_double(c1.value());
        }
        unit_store<2>(a[0], a[1], part, n_units, R, u);
        if (last_unit(&inst_cnt[un.inst], in.n_units)) {
            int ended = 0;
            for (int k = threadIdx.x; k < R; k += blockDim.x) {
                const int pi = un.inst * R + k;
                if (pr.flag[pi] != kRun) continue;
                const double rn2 = inst_sum(part, n_units, R, 0, in, k);
                const double rho_new = inst_sum(part, n_units, R, 1, in, k);
                pr.rn2[pi] = rn2;
                pr.rho_new[pi] = rho_new;
                pr.iters[pi] += 1;
                pr.pass_iters[pi] += 1;
                bool end = false;
                if (!isfinite(rn2) || !isfinite(rho_new) || rho_new == 0.0 || pr.omega[pi] == 0.0) end = true;
                else if (rn2 <= pr.tol2[pi] || rn2 < pr.repl2[pi] * pr.tn2[pi]) end = true;
                else if (!(rn2 <= kGrowth2 * pr.s0[pi])) end = true;
                else if (pr.pass_iters[pi] >= kPassCap || pr.iters[pi] >= max_iter) end = true;
                if (end) {
                    pr.flag[pi] = kPassEnd;
                    ++ended;
                }
            }
            end_pairs(ended, inst_running + un.inst, ctl);
        }
    }
}

// ------------------------------------------------- the device-side loop ---
// The multigrid mode's rounds (explicit FP64 residual, then BiCGSTAB passes)
// run as one graph launch: an outer WHILE node over rounds and an inner
// WHILE node over iterations, their conditions set by the two kernels below.
// loop[0]: this round runs, loop[1]: rounds started, loop[2]: iterations
// started, loop[3]: iterations of this round, loop[4..5]: (instance, rhs)
// pair-iterations (a 64-bit count).  Each condition is also capped by those
// counters -- max_outer rounds, and per round the per-pass cap every pair
// obeys (kPassCap, max_iter) plus one -- so both loops end whatever the
// solver's flags say.
__global__ void b_reset_ctl_kernel(Ctl* ctl) {
    if (threadIdx.x == 0) {
        ctl->running = 0;
        ctl->active = 0;
    }
}

__global__ void b_decide_outer_kernel(const Ctl* ctl, int* loop, int max_outer, const int* stop,
                                      cudaGraphConditionalHandle outer) {
    if (threadIdx.x != 0) return;
    const bool halt = stop && *(volatile const int*)stop != 0;
    const int go = (!halt && ctl->active > 0 && loop[1] < max_outer) ? 1 : 0;
    loop[0] = go;
    loop[3] = 0;
    if (go) loop[1] += 1;
    cudaGraphSetConditional(outer, go);
}

__global__ void b_decide_inner_kernel(const Ctl* ctl, int* loop, int round_cap, const int* stop,
                                      cudaGraphConditionalHandle inner) {
    if (threadIdx.x != 0) return;
    const bool halt = stop && *(volatile const int*)stop != 0;
    const int run = ctl->running;
    const int go = (!halt && loop[0] != 0 && run > 0 && loop[3] < round_cap) ? 1 : 0;
    if (go) {
        loop[2] += 1;
        loop[3] += 1;
        *reinterpret_cast<unsigned long long*>(loop + 4) += (unsigned long long)run;
    }
    cudaGraphSetConditional(inner, go);
}

// ------------------------------------------------------------------ host ---
struct Plan {
    int n_inst = 0, R = 0, n_units = 0;
    int64_t N = 0, idx_total = 0, nnz_cap = 0;
    size_t knn_ws = 0;
    std::vector<Inst> inst;
    std::vector<Unit> units;
    // multigrid mode: per instance its hierarchy's workspace and its
    // coarse-level multi-rhs vectors (bounds), as offsets into two areas
    bool mg = false;
    std::vector<size_t> mg_off, mg_bytes, coarse_off;
    size_t mg_total = 0, coarse_total = 0;
};

bool make_plan(const rbffd_batch_desc* desc, int32_t n_inst, int32_t R, bool mg, Plan* pl) {
    if (!desc || n_inst < 1 || R < 1 || R > kMaxRhs) return false;
    pl->n_inst = n_inst;
    pl->R = R;
    pl->mg = mg;
    int64_t off = 0, idx_off = 0;
    int uoff = 0;
    for (int i = 0; i < n_inst; ++i) {
        const rbffd_batch_desc& d = desc[i];
        const int s = (d.m + 1) * (d.m + 2) / 2;
        if (d.node_offset != off || d.n_nodes < 1 || d.n < 1 || d.n > RBFFD_MAX_STENCIL || d.n > d.n_nodes ||
            d.m < 0 || d.m > 8 || d.n < s)
            return false;
        Inst in;
        in.node_off = off;
        in.n_nodes = d.n_nodes;
        in.idx_off = idx_off;
        in.n = d.n;
        in.m = d.m;
        in.unit_off = uoff;
        in.n_units = (int)((d.n_nodes + kUnitRows - 1) / kUnitRows);
        for (int u = 0; u < in.n_units; ++u) {
            Unit un;
            un.inst = i;
            un.pad = 0;
            un.row_lo = off + (int64_t)u * kUnitRows;
            un.row_hi = std::min(off + d.n_nodes, un.row_lo + kUnitRows);
            pl->units.push_back(un);
        }
        uoff += in.n_units;
        pl->inst.push_back(in);
        if (mg) {
            const size_t b = align_up(rbffd_mg_workspace_size(d.n_nodes, 0));
            if (b == 0) return false;
            pl->mg_off.push_back(pl->mg_total);
            pl->mg_bytes.push_back(b);
            pl->mg_total += b;
            // coarse levels hold at most half the nodes of the level above:
            // 4 vectors x R x (N/2 + N/4 + ...) < 4 R N floats
            pl->coarse_off.push_back(pl->coarse_total);
            pl->coarse_total += align_up((size_t)4 * R * d.n_nodes * sizeof(float)) / sizeof(float);
        }
        pl->knn_ws = std::max(pl->knn_ws, rbffd_stencils_workspace_size(d.n_nodes, d.n));
        off += d.n_nodes;
        idx_off += d.n_nodes * d.n;
    }
    if (off > 0x7fffffffLL) return false;
    pl->N = off;
    pl->idx_total = idx_off;
    pl->nnz_cap = idx_off;  // every row at most n_i entries
    pl->n_units = uoff;
    return true;
}

size_t layout(void* ws, const Plan& pl, BWork* w) {
    Carver c(ws);
    BWork t{};
    const int64_t N = pl.N, NR = pl.N * pl.R;
    const int P = pl.n_inst * pl.R;
    t.inst = c.take<Inst>(pl.n_inst);
    t.units = c.take<Unit>(pl.n_units);
    t.inst_running = c.take<int>(pl.n_inst);
    t.inst_cnt = c.take<unsigned>(pl.n_inst);
    t.ctl = c.take<Ctl>(1);
    t.part = c.take<double>((size_t)3 * pl.n_units * pl.R);
    double** dd[] = {&t.pr.rho, &t.pr.rho_new, &t.pr.alpha, &t.pr.omega, &t.pr.bn2, &t.pr.tol2,
                     &t.pr.rn2, &t.pr.tn2, &t.pr.s0, &t.pr.rstart2, &t.pr.repl2};
    for (double** q : dd) *q = c.take<double>(P);
    t.pr.flag = c.take<int>(P);
    t.pr.iters = c.take<int>(P);
    t.pr.pass_iters = c.take<int>(P);
    t.idx = c.take<int32_t>(pl.idx_total);
    t.w = c.take<double>(pl.idx_total);
    t.nstat = c.take<int32_t>(N);
    t.row_ptr = c.take<int64_t>(N + 1);
    t.col = c.take<int32_t>(pl.nnz_cap);
    t.val = c.take<double>(pl.nnz_cap);
    t.val32 = c.take<float>(pl.nnz_cap);
    t.scan_sums = c.take<int64_t>(scan_tiles(N) + 1);
    t.knn_ws = c.take<char>(align_up(pl.knn_ws) * kSetupStreams);
    t.b = c.take<double>(NR);
    t.r64 = c.take<double>(NR);
    t.d = c.take<double>(N);
    t.dinv = c.take<double>(N);
    t.d32 = c.take<float>(N);
    t.dinv32 = c.take<float>(N);
    t.sig32 = c.take<float>(N);
    if (!pl.mg) {
        float2** vv[] = {&t.xd, &t.r, &t.rh, &t.p, &t.v, &t.s, &t.t};
        for (float2** q : vv) *q = c.take<float2>(NR);
    } else {
        double** mm[] = {&t.mrh, &t.mp, &t.mv, &t.ms, &t.mt, &t.mph, &t.msh};
        for (double** q : mm) *q = c.take<double>(NR);
        t.mr = c.take<float2>(NR);
        t.val_lo = c.take<float>(pl.nnz_cap);
        t.f0 = c.take<float>(NR);
        t.f1 = c.take<float>(NR);
        t.f2 = c.take<float>(NR);
        t.coarse = c.take<float>(pl.coarse_total);
        t.mgws = c.take<char>(pl.mg_total);
        t.mbtab_bytes = mg_batch_table_bytes(pl.n_inst, pl.N);
        t.mbtab = c.take<char>(t.mbtab_bytes);
        t.loop = c.take<int>(8);
    }
    if (w) *w = t;
    return c.off;
}

// one block per unit: a grid-stride loop over more units than resident
// blocks runs in uneven waves
int grid_units(int n_units) { return std::max(1, n_units); }

// RBFFD_TRACE=1: phase times of the batched solve on stderr (host clock
// after a stream synchronisation; diagnostics only).
struct PhaseClock {
    bool on;
    cudaStream_t st;
    std::chrono::steady_clock::time_point t0;
    explicit PhaseClock(cudaStream_t s) : st(s) {
        const char* v = std::getenv("RBFFD_TRACE");
        on = v && *v && std::atoi(v) != 0;
        t0 = std::chrono::steady_clock::now();
    }
    void mark(const char* what) {
        if (!on) return;
        cudaStreamSynchronize(st);
        const auto t = std::chrono::steady_clock::now();
        fprintf(stderr, "[rbffd batched] %s: %.1f ms\n", what,
                std::chrono::duration<double, std::milli>(t - t0).count());
        t0 = t;
    }
};

int finish_info(const Plan& pl, const BWork& w, int rounds, const std::vector<int>& inst_bad, rbffd_solve_info* info,
                cudaStream_t st);

// Multigrid mode: one hierarchy per instance (its fine level is the
// instance's block of the batched matrix), then rounds of (explicit FP64
// residual per pair, BiCGSTAB passes); one iteration for all instances --
// the outer kernels and every instance's two V-cycles -- is one CUDA graph,
// replayed while any pair is in a pass.  Returns the rounds run, or minus
// an error status.
int solve_mg(const Plan& pl, const BWork& w, const double* xy, const uint8_t* mask, double* u,
             const rbffd_solve_opts* o, cudaStream_t st) {
    const int R = pl.R;
    const int gu = grid_units(pl.n_units);
    PhaseClock clk(st);
    std::vector<rbffd_mg> hs(pl.n_inst);
    std::vector<const MgHierarchy*> H(pl.n_inst);
    {
        // The hierarchy setups read level sizes back to the host, so each
        // blocks its thread: kSetupStreams host threads, each on its own
        // stream, build disjoint sets of instances; `st` then waits for them.
        if (cudaStreamSynchronize(st) != cudaSuccess) return -(int)RBFFD_ERR_CUDA;
        int dev = 0;
        cudaGetDevice(&dev);
        std::vector<int> rcs(kSetupStreams, RBFFD_OK);
        std::vector<std::thread> th;
        for (int t = 0; t < kSetupStreams; ++t) {
            th.emplace_back([&, t]() {
                cudaSetDevice(dev);
                cudaStream_t ts;
                if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
                    rcs[t] = RBFFD_ERR_CUDA;
                    return;
                }
                for (int i = t; i < pl.n_inst && rcs[t] == RBFFD_OK; i += kSetupStreams) {
                    const Inst& in = pl.inst[i];
                    rcs[t] = mg_setup_core(xy + 2 * in.node_off, mask + in.node_off, in.n_nodes,
                                           w.row_ptr + in.node_off, w.col, w.val, w.val32,
                                           in.n_nodes * (int64_t)in.n, (int)in.node_off, 2, 0.6, &hs[i],
                                           w.mgws + pl.mg_off[i], pl.mg_bytes[i], ts);
                }
                if (cudaStreamSynchronize(ts) != cudaSuccess && rcs[t] == RBFFD_OK) rcs[t] = RBFFD_ERR_CUDA;
                cudaStreamDestroy(ts);
            });
        }
        for (auto& x : th) x.join();
        for (int t = 0; t < kSetupStreams; ++t)
            if (rcs[t] != RBFFD_OK) return -rcs[t];
    }
    for (int i = 0; i < pl.n_inst; ++i) {
        H[i] = mg_hierarchy(&hs[i]);
        if (!H[i] || mg_multi_coarse_floats(H[i], R) * sizeof(float) >
                         (i + 1 < pl.n_inst ? pl.coarse_off[i + 1] - pl.coarse_off[i]
                                            : pl.coarse_total - pl.coarse_off[i]) *
                             sizeof(float))
            return -RBFFD_ERR_WORKSPACE;
    }
    clk.mark("multigrid hierarchies");
    // the batched V-cycle: one launch per (level, operation) over all instances
    MgBatch mb{};
    {
        std::vector<int64_t> noff(pl.n_inst);
        for (int i = 0; i < pl.n_inst; ++i) noff[i] = pl.inst[i].node_off;
        const int rc = mg_batch_build(H.data(), noff.data(), pl.n_inst, R, w.f0, w.f1, w.f2, w.coarse,
                                      pl.coarse_off.data(), w.mbtab, w.mbtab_bytes, o->persistent,
                                      (long long)o->spin_limit, o->wait_test, st, &mb);
        if (rc != RBFFD_OK) return -rc;
    }
    int vlaunch = 0;
    // double-float views of the outer vectors
    float2* vr = w.mr;
    float2* vrh = reinterpret_cast<float2*>(w.mrh);
    float2* vp = reinterpret_cast<float2*>(w.mp);
    float2* vv = reinterpret_cast<float2*>(w.mv);
    float2* vsv = reinterpret_cast<float2*>(w.ms);
    float2* vt = reinterpret_cast<float2*>(w.mt);
    float2* vph = reinterpret_cast<float2*>(w.mph);
    float2* vsh = reinterpret_cast<float2*>(w.msh);
    // one BiCGSTAB iteration of every running pair (with its two batched
    // V-cycles), captured on `cap`
    auto capture_iteration = [&](cudaStream_t cap) -> int {
        md_update_p_kernel<<<gu, kBT, 0, cap>>>(w.units, pl.n_units, R, vr, vv, vp, w.pr, w.inst_running);
        int rc = mg_batch_apply_df(mb, R, vp, vph, w.inst_running, cap, &vlaunch);
        md_spmm_kernel<0><<<gu, kBT, 0, cap>>>(w.units, pl.n_units, w.inst, w.row_ptr, w.col, w.val32, w.val_lo, R,
                                               vph, vv, vrh, w.pr, w.inst_running, w.inst_cnt, w.ctl, w.part);
        md_update_s_kernel<<<gu, kBT, 0, cap>>>(w.units, pl.n_units, R, vr, vv, vsv, w.pr, w.inst_running);
        if (rc == RBFFD_OK) rc = mg_batch_apply_df(mb, R, vsv, vsh, w.inst_running, cap, &vlaunch);
        md_spmm_kernel<1><<<gu, kBT, 0, cap>>>(w.units, pl.n_units, w.inst, w.row_ptr, w.col, w.val32, w.val_lo, R,
                                               vsh, vt, vsv, w.pr, w.inst_running, w.inst_cnt, w.ctl, w.part);
        md_update_xr_kernel<<<gu, kBT, 0, cap>>>(w.units, pl.n_units, w.inst, R, u, vph, vsh, vsv, vt, vr, vrh, w.pr,
                                                 w.inst_running, w.inst_cnt, w.ctl, w.part, o->max_iter);
        return rc;
    };
    const bool device_loop = o->device_loop != 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int round_cap = std::min(std::max(o->max_iter, 1), kPassCap) + 1;
    int* stop = mb.status;  // a bounded wait of the batched V-cycle ran out
    {
        cudaStream_t cap;
        RBFFD_CUDA_TRY_NEG(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        int rc = RBFFD_OK;
        cudaError_t e = cudaSuccess;
        if (!device_loop) {
            // one graph per iteration, launched by the host loop below
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = capture_iteration(cap);
                e = cudaStreamEndCapture(cap, &graph);
            }
        } else {
            // the whole solve as one graph: WHILE (rounds) { FP64 residual
            // check, pass start, WHILE (iterations) { one iteration } }
            e = cudaGraphCreate(&graph, 0);
            cudaGraphConditionalHandle h_out = 0, h_in = 0;
            cudaGraph_t body_out = nullptr, body_in = nullptr;
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_out, graph, 1, cudaGraphCondAssignDefault);
            if (e == cudaSuccess) {
                cudaGraphNodeParams cp{};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = h_out;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                cudaGraphNode_t n_out;
                e = cudaGraphAddNode(&n_out, graph, nullptr, nullptr, 0, &cp);
                if (e == cudaSuccess) body_out = cp.conditional.phGraph_out[0];
            }
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_in, body_out, 0, 0);
            // outer body: residual check, decision, pass start, first inner
            // decision, inner loop
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(cap, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                b_reset_ctl_kernel<<<1, 32, 0, cap>>>(w.ctl);
                b_check_kernel<<<gu, kBT, 0, cap>>>(w.units, pl.n_units, w.inst, w.row_ptr, w.col, w.val, R, w.b, u,
                                                    w.dinv, w.r64, w.pr, w.inst_cnt, w.ctl, w.part, o->tol);
                b_decide_outer_kernel<<<1, 32, 0, cap>>>(w.ctl, w.loop, o->max_outer, stop, h_out);
                md_load_kernel<<<gu, kBT, 0, cap>>>(w.units, pl.n_units, w.inst, R, w.r64, vr, vrh, vp, vv, w.pr,
                                                    w.inst_cnt, w.inst_running, w.ctl, w.part, o->inner_tol,
                                                    o->max_iter, w.loop);
                b_decide_inner_kernel<<<1, 32, 0, cap>>>(w.ctl, w.loop, round_cap, stop, h_in);
                cudaStreamCaptureStatus cs;
                cudaGraph_t cg = nullptr;
                const cudaGraphNode_t* deps = nullptr;
                size_t nd = 0;
                e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &cg, &deps, nullptr, &nd);
                if (e == cudaSuccess) {
                    cudaGraphNodeParams cp{};
                    cp.type = cudaGraphNodeTypeConditional;
                    cp.conditional.handle = h_in;
                    cp.conditional.type = cudaGraphCondTypeWhile;
                    cp.conditional.size = 1;
                    cudaGraphNode_t n_in;
                    e = cudaGraphAddNode(&n_in, cg, deps, nullptr, nd, &cp);
                    if (e == cudaSuccess) {
                        body_in = cp.conditional.phGraph_out[0];
                        e = cudaStreamUpdateCaptureDependencies(cap, &n_in, nullptr, 1,
                                                                cudaStreamSetCaptureDependencies);
                    }
                }
                cudaGraph_t got = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(cap, &got);
                if (e == cudaSuccess) e = e2;
            }
            // inner body: one iteration, then the next inner decision
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(cap, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = capture_iteration(cap);
                b_decide_inner_kernel<<<1, 32, 0, cap>>>(w.ctl, w.loop, round_cap, stop, h_in);
                cudaGraph_t got = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(cap, &got);
                if (e == cudaSuccess) e = e2;
            }
        }
        if (e == cudaSuccess && rc == RBFFD_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess || rc != RBFFD_OK) {
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) set_cuda_error(e);
            return -(rc != RBFFD_OK ? rc : (int)RBFFD_ERR_CUDA);
        }
    }
    const int per_iter = 5 + vlaunch + (device_loop ? 1 : 0);  // + the inner decision on the device
    // algorithmic bytes of one iteration with every pair running (see the
    // profiling hooks in rbffd.h)
    int64_t nnz = 0;
    if (cudaMemcpyAsync(&nnz, w.row_ptr + pl.N, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -(int)RBFFD_ERR_CUDA;
    const int64_t iter_bytes = (int64_t)(168 + 2 * 118) * pl.N * R + 2 * 12 * nnz + 2 * 4 * 8 * nnz;
    // the matrix's trailing float parts for the double-float SpMM
    md_split_kernel<<<std::max(1, std::min((int)((nnz + kBT - 1) / kBT), sm_count() * 16)), kBT, 0, st>>>(
        w.val, w.val32, nnz, w.val_lo);
    note_launches(1);
    clk.mark("iteration graph capture");
    int err = RBFFD_OK;
    int rounds = 0;
    bool timed_out = false;
    if (device_loop) {
        int hl[8] = {0};
        if (cudaMemsetAsync(w.loop, 0, sizeof(int) * 8, st) != cudaSuccess) err = RBFFD_ERR_CUDA;
        const int ev = prof_begin(st);
        if (err == RBFFD_OK && cudaGraphLaunch(exec, st) != cudaSuccess) err = RBFFD_ERR_CUDA;
        prof_end(ev, st, kProfBatchIter, 0);
        if (err == RBFFD_OK && (cudaMemcpyAsync(hl, w.loop, sizeof(hl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                                cudaStreamSynchronize(st) != cudaSuccess))
            err = RBFFD_ERR_CUDA;
        rounds = hl[1];
        const int iters = hl[2];
        unsigned long long pair_iters = 0;
        std::memcpy(&pair_iters, hl + 4, sizeof(pair_iters));
        // the loop ran on the device: its time counts as `iters` iterations,
        // bytes in proportion to the pairs that were in a pass
        prof_commit_as(ev, iters, (int64_t)((double)iter_bytes * (double)pair_iters / (pl.n_inst * (double)R)));
        note_launches((int)std::min<long long>((long long)iters * per_iter + rounds * 4LL, 1LL << 30));
        if (err == RBFFD_OK && mg_batch_timed_out(mb, st, &timed_out) != RBFFD_OK) err = RBFFD_ERR_CUDA;
    } else {
        Ctl hc;
        for (;;) {
            if (cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st) != cudaSuccess) { err = RBFFD_ERR_CUDA; break; }
            b_check_kernel<<<gu, kBT, 0, st>>>(w.units, pl.n_units, w.inst, w.row_ptr, w.col, w.val, R, w.b, u,
                                               w.dinv, w.r64, w.pr, w.inst_cnt, w.ctl, w.part, o->tol);
            note_launches(1);
            if (cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                err = RBFFD_ERR_CUDA;
                break;
            }
            if (hc.active == 0 || rounds >= o->max_outer) break;
            ++rounds;
            md_load_kernel<<<gu, kBT, 0, st>>>(w.units, pl.n_units, w.inst, R, w.r64, vr, vrh, vp, vv, w.pr,
                                               w.inst_cnt, w.inst_running, w.ctl, w.part, o->inner_tol, o->max_iter,
                                               nullptr);
            note_launches(1);
            for (int guard = 0; guard < round_cap; ++guard) {
                if (cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    err = RBFFD_ERR_CUDA;
                    break;
                }
                if (hc.running <= 0) break;
                const int ev = prof_begin(st);
                if (cudaGraphLaunch(exec, st) != cudaSuccess) {
                    err = RBFFD_ERR_CUDA;
                    break;
                }
                // bytes in proportion to the pairs still in a pass
                prof_end(ev, st, kProfBatchIter,
                         (int64_t)((double)iter_bytes * hc.running / (pl.n_inst * (double)R)));
                note_launches(per_iter);
                if (mb.persistent) {
                    if (mg_batch_timed_out(mb, st, &timed_out) != RBFFD_OK) err = RBFFD_ERR_CUDA;
                    if (err != RBFFD_OK || timed_out) break;
                }
            }
            if (err != RBFFD_OK || timed_out) break;
        }
    }
    if (err == RBFFD_OK && timed_out) err = RBFFD_ERR_TIMEOUT;
    clk.mark("solve");
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (err == RBFFD_OK) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_cuda_error(e);
            err = RBFFD_ERR_CUDA;
        }
    }
    return err != RBFFD_OK ? -err : rounds;
}

}  // namespace
}  // namespace rbffd

extern "C" size_t rbffd_batched_workspace_size(const rbffd_batch_desc* desc, int32_t n_inst, int32_t n_rhs,
                                               const rbffd_solve_opts* opts) {
    RBFFD_NVTX("rbffd_batched_workspace_size");
    rbffd::Plan pl;
    if (opts && opts->precond != 0 && opts->precond != 1) return 0;
    if (!rbffd::make_plan(desc, n_inst, n_rhs, opts && opts->precond == 1, &pl)) return 0;
    return rbffd::layout(nullptr, pl, nullptr);
}

extern "C" int rbffd_solve_batched(const rbffd_batch_desc* desc, int32_t n_inst, const double* xy,
                                   const uint8_t* is_dirichlet, const double* f, const double* g, int32_t n_rhs,
                                   double* u, const rbffd_solve_opts* o, rbffd_solve_info* info, void* ws,
                                   size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_solve_batched");
    using namespace rbffd;
    Plan pl;
    if (!o || (o->precond != 0 && o->precond != 1)) return RBFFD_ERR_INVALID_ARG;
    const bool use_mg = o->precond == 1;
    if (!xy || !is_dirichlet || !f || !g || !u || !info || !make_plan(desc, n_inst, n_rhs, use_mg, &pl))
        return RBFFD_ERR_INVALID_ARG;
    if (((uintptr_t)xy & 15) != 0) return RBFFD_ERR_INVALID_ARG;
    if (!(o->tol > 0.0) || o->max_iter < 0 || !(o->inner_tol > 0.0 && o->inner_tol < 1.0) || o->max_outer < 1)
        return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0 || ws_bytes < layout(nullptr, pl, nullptr))
        return RBFFD_ERR_WORKSPACE;
    BWork w;
    layout(ws, pl, &w);
    cudaStream_t st = as_stream(stream);
    const int R = pl.R, P = pl.n_inst * pl.R;
    const int64_t N = pl.N;

    RBFFD_CUDA_TRY(cudaMemcpyAsync(w.inst, pl.inst.data(), sizeof(Inst) * pl.n_inst, cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(w.units, pl.units.data(), sizeof(Unit) * pl.n_units, cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(w.inst_cnt, 0, sizeof(unsigned) * pl.n_inst, st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(w.pr.flag, 0, sizeof(int) * P, st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(w.pr.iters, 0, sizeof(int) * P, st));

    // ---- setup: stencils and weights per instance, then one CSR -----------
    PhaseClock clk(st);
    {
        // independent instances: spread over streams (each with its own
        // stencil workspace), forked from and joined back to `st`
        cudaStream_t ss[kSetupStreams];
        cudaEvent_t fork_ev, join_ev[kSetupStreams];
        RBFFD_CUDA_TRY(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
        for (int k = 0; k < kSetupStreams; ++k) {
            RBFFD_CUDA_TRY(cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking));
            RBFFD_CUDA_TRY(cudaEventCreateWithFlags(&join_ev[k], cudaEventDisableTiming));
        }
        RBFFD_CUDA_TRY(cudaEventRecord(fork_ev, st));
        int rc = RBFFD_OK;
        for (int k = 0; k < kSetupStreams && rc == RBFFD_OK; ++k)
            if (cudaStreamWaitEvent(ss[k], fork_ev, 0) != cudaSuccess) rc = RBFFD_ERR_CUDA;
        const size_t kws = align_up(pl.knn_ws);
        for (int i = 0; i < pl.n_inst && rc == RBFFD_OK; ++i) {
            const Inst& in = pl.inst[i];
            const int k = i % kSetupStreams;
            const double* xy_i = xy + 2 * in.node_off;
            rc = rbffd_stencils(xy_i, in.n_nodes, in.n, w.idx + in.idx_off, static_cast<char*>(w.knn_ws) + k * kws,
                                pl.knn_ws, ss[k]);
            if (rc == RBFFD_OK)
                rc = rbffd_weights(xy_i, w.idx + in.idx_off, in.n_nodes, in.n, in.m, w.w + in.idx_off,
                                   w.nstat + in.node_off, ss[k]);
        }
        for (int k = 0; k < kSetupStreams; ++k) {
            if (cudaEventRecord(join_ev[k], ss[k]) != cudaSuccess || cudaStreamWaitEvent(st, join_ev[k], 0) != cudaSuccess)
                rc = RBFFD_ERR_CUDA;
        }
        for (int k = 0; k < kSetupStreams; ++k) {
            cudaStreamDestroy(ss[k]);
            cudaEventDestroy(join_ev[k]);
        }
        cudaEventDestroy(fork_ev);
        if (rc != RBFFD_OK) return rc;
    }
    RBFFD_CUDA_TRY(exclusive_scan<int64_t>(BRowLen{w.inst, pl.n_inst, is_dirichlet}, N, w.row_ptr, w.scan_sums,
                                           w.row_ptr + N, st));
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((N * 32 + 255) / 256, sm_count() * 16));
    b_fill_kernel<<<gb, 256, 0, st>>>(w.inst, pl.n_inst, N, is_dirichlet, w.idx, w.w, w.row_ptr, pl.nnz_cap, w.col,
                                      w.val, w.val32);
    b_rhs_kernel<<<sm_count() * 8, 256, 0, st>>>(N, R, is_dirichlet, f, g, w.b);
    b_dstart_kernel<<<sm_count() * 8, 256, 0, st>>>(N, R, is_dirichlet, w.b, u);
    b_diag_kernel<<<(int)std::min<int64_t>((N + 255) / 256, sm_count() * 8), 256, 0, st>>>(
        w.row_ptr, w.col, w.val, N, w.d, w.dinv, w.d32, w.dinv32, w.sig32);
    note_launches(4);
    RBFFD_LAUNCH_CHECK();

    // per-node weight status: any singular stencil fails the instance
    clk.mark("stencils, weights, matrix");
    std::vector<int32_t> hstat(N);
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hstat.data(), w.nstat, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> inst_bad(pl.n_inst, 0);
    for (int i = 0; i < pl.n_inst; ++i)
        for (int64_t k = 0; k < pl.inst[i].n_nodes; ++k)
            if (hstat[pl.inst[i].node_off + k]) {
                inst_bad[i] = 1;
                break;
            }

    const int gu = grid_units(pl.n_units);
    if (use_mg) {
        const int rc = solve_mg(pl, w, xy, is_dirichlet, u, o, st);
        return finish_info(pl, w, rc, inst_bad, info, st);
    }

    // ---- solve: rounds of (FP64 residual, inner passes, refinement) --------
    const int chunk = 16;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto enqueue_chunk = [&](cudaStream_t s) {
        for (int c = 0; c < chunk; ++c) {
            b_update_p_kernel<<<gu, kBT, 0, s>>>(w.units, pl.n_units, R, w.r, w.v, w.p, w.pr, w.inst_running);
            b_spmm_kernel<0><<<gu, kBT, 0, s>>>(w.units, pl.n_units, w.inst, w.row_ptr, w.col, w.val32, R, w.p,
                                                w.sig32, w.dinv32, w.v, w.rh, w.pr, w.inst_running, w.inst_cnt,
                                                w.ctl, w.part);
            b_update_s_kernel<<<gu, kBT, 0, s>>>(w.units, pl.n_units, R, w.r, w.v, w.s, w.pr, w.inst_running);
            b_spmm_kernel<1><<<gu, kBT, 0, s>>>(w.units, pl.n_units, w.inst, w.row_ptr, w.col, w.val32, R, w.s,
                                                w.sig32, w.dinv32, w.t, nullptr, w.pr, w.inst_running, w.inst_cnt,
                                                w.ctl, w.part);
            b_update_xr_kernel<<<gu, kBT, 0, s>>>(w.units, pl.n_units, w.inst, R, w.xd, w.p, w.s, w.t, w.r, w.rh,
                                                  w.d32, w.pr, w.inst_running, w.inst_cnt, w.ctl, w.part,
                                                  o->max_iter);
        }
    };
    // one graph of a chunk of inner iterations, replayed
    {
        cudaStream_t cap;
        RBFFD_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_chunk(cap);
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            set_cuda_error(e);
            return RBFFD_ERR_CUDA;
        }
    }
    int rc = RBFFD_OK;
    int rounds = 0;
    Ctl hc;
    std::vector<int> hflag(P);
    for (;;) {
        RBFFD_CUDA_TRY(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st));
        b_check_kernel<<<gu, kBT, 0, st>>>(w.units, pl.n_units, w.inst, w.row_ptr, w.col, w.val, R, w.b, u, w.dinv,
                                           w.r64, w.pr, w.inst_cnt, w.ctl, w.part, o->tol);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        RBFFD_CUDA_TRY(cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (hc.active == 0 || rounds >= o->max_outer) break;
        ++rounds;
        b_load_kernel<<<gu, kBT, 0, st>>>(w.units, pl.n_units, w.inst, R, w.r64, w.dinv32, w.r, w.rh, w.p, w.v, w.xd,
                                          w.pr, w.inst_cnt, w.inst_running, w.ctl, w.part, o->inner_tol, o->max_iter,
                                          0x5EED2107ull + (unsigned long long)rounds);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
        for (int guard = 0; guard < 1 << 20; ++guard) {
            RBFFD_CUDA_TRY(cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
            RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
            if (hc.running <= 0) break;
            RBFFD_CUDA_TRY(cudaGraphLaunch(exec, st));
            note_launches(5 * chunk);
        }
        b_refine_kernel<<<gu, kBT, 0, st>>>(w.units, pl.n_units, R, u, w.xd, w.pr);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);

    (void)hflag;
    return finish_info(pl, w, rounds, inst_bad, info, st);
}

namespace rbffd {
namespace {
// Per-instance summary: the worst right-hand side of each instance.
int finish_info(const Plan& pl, const BWork& w, int rounds, const std::vector<int>& inst_bad, rbffd_solve_info* info,
                cudaStream_t st) {
    const int R = pl.R, P = pl.n_inst * pl.R;
    if (rounds < 0) return -rounds;  // an error code from the solve
    int rc = RBFFD_OK;
    std::vector<int> hflag(P);
    std::vector<double> tn(P), bn(P);
    std::vector<int> it(P);
    RBFFD_CUDA_TRY(cudaMemcpyAsync(hflag.data(), w.pr.flag, sizeof(int) * P, cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(tn.data(), w.pr.tn2, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(bn.data(), w.pr.bn2, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(it.data(), w.pr.iters, sizeof(int) * P, cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < pl.n_inst; ++i) {
        rbffd_solve_info& inf = info[i];
        std::memset(&inf, 0, sizeof(inf));
        int status = RBFFD_OK;
        for (int k = 0; k < R; ++k) {
            const int pi = i * R + k;
            const double rel = bn[pi] > 0.0 ? std::sqrt(tn[pi] / bn[pi]) : std::sqrt(tn[pi]);
            inf.rel_residual = std::max(inf.rel_residual, rel);
            inf.iters = std::max(inf.iters, it[pi]);
            if (hflag[pi] != kDone) status = (hflag[pi] == kFail && !std::isfinite(rel)) ? RBFFD_ERR_BREAKDOWN
                                                                                           : RBFFD_ERR_NOT_CONVERGED;
        }
        if (inst_bad[i]) status = RBFFD_ERR_SINGULAR_STENCIL;
        inf.status = status;
        inf.outer_sweeps = rounds;
        if (status != RBFFD_OK && rc == RBFFD_OK) rc = status;
    }
    return rc;
}
}  // namespace
}  // namespace rbffd
