// Batched multi-right-hand-side V-cycle over many instances' hierarchies
// (sm_103a): the preconditioner of the batched solve (rbffd_solve_batched).
//
// Each instance has its own multigrid hierarchy (mg.cu: rediscretised RBF-FD
// coarse levels, PHS interpolation, damped Jacobi smoothing, dense coarsest
// solve), and every instance's V-cycle is the same sequence of operations on
// levels 0, 1, ... .  Instead of issuing each instance's coarse-level kernels
// separately (hundreds of tiny launches per instance and cycle), one launch
// per (level, operation) covers every instance that has that level: a
// device table holds one descriptor per (instance, level) -- the level's
// operator, transfers and vectors -- and a unit table lists tiles of rows
// (instance, level, row range).  A block walks units, a warp owns a row,
// and lanes k and k + 32 own right-hand sides k and k + 32 of node-major
// [row][R] vectors, so a matrix entry is read once for all right-hand sides.
// Units of instances with no running (instance, rhs) pair return at once.
//
// Schedule of one cycle (nu pre- and post-sweeps):
//   descend, l = 0, 1, ...: the instances whose coarsest level is l solve it
//     (dense inverse); the others smooth (x = W b, nu - 1 sweeps), form the
//     residual and restrict it to level l + 1;
//   ascend, l = ..., 1, 0: prolongate the next level's result and add it,
//     then nu post-sweeps; the last level-0 sweep writes the output.
// In exact arithmetic this is the recursive V-cycle of each instance.
//
// Optionally (the persistent mode), levels 1 and below (every instance's
// coarse levels) run as one persistent launch (mb_coarse_kernel) from a
// device work queue of tasks (instance,
// level, operation, tile of rows) in a topological order: phase k of every
// instance after phase k - 1 of every instance.  A block takes the next
// task with an atomic ticket and waits until every tile of the same
// instance's previous phase is done (a per-(instance, phase) counter); the
// tasks it can wait on were all handed out earlier to running blocks, so
// the waits end.  Each wait is bounded (spin_limit polls): past it the
// kernel records a timeout, every block stops at its next task, and the
// solve returns RBFFD_ERR_TIMEOUT.  Vectors written inside this launch are
// read with coherent loads (the read-only cache path is not coherent with
// writes of other blocks of the same launch).  Measured on 256 disks x 64
// rhs, the per-operation launches are faster (a solve of 4.13 s against
// 4.57 s), so they are the default.
#include "common.cuh"
#include "internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace rbffd {

struct MbLevel {
    const int64_t* row_ptr;
    const int* col;
    const float* val;
    const float* dinv;  // W = Omega D^-1
    const int32_t* pidx;  // prolongation from level l + 1 (ELL, kMgK per row)
    const float* pval;
    const int64_t* rrow;  // restriction to level l + 1 (CSR, N_next rows)
    const int* rcol;
    const float* rval;
    const float* minv;  // coarsest: dense inverse
    float *x, *t, *r, *b;  // level vectors; level 0: the caller's global arrays (rows row_off ..)
    float* b_next;         // the next level's b (restriction target)
    const float* e_next;   // the next level's result (its x if coarsest there, else its t)
    int64_t N, N_next, row_off;
    int32_t inst, pad;
};

struct MbUnit {
    int32_t desc;
    int32_t pad;
    int64_t lo, hi;  // rows of the descriptor's level
};

// A task of the persistent coarse-level kernel: one tile of one operation.
struct MbTask {
    int32_t desc;
    int8_t op;   // kOpFirst .. kOpDense
    int8_t dir;  // which level vector holds the current iterate
    int16_t pad;
    int64_t lo, hi;
    int32_t wait;  // counter of the instance's previous phase (-1: none)
    int32_t need;  // its tiles
    int32_t post;  // counter of this task's phase
    int32_t pad2;
};

namespace {

constexpr int kMbT = 256;         // threads per block (8 warps)
constexpr int kMbTileRows = 256;  // rows per unit
constexpr int kMbDenseRows = 16;  // rows per unit of the dense coarsest solves
enum : int8_t { kOpFirst = 0, kOpSweep = 1, kOpResid = 2, kOpRestrict = 3, kOpProlong = 4, kOpDense = 5 };
constexpr long long kMbDefaultSpin = 1LL << 26;  // polls of a bounded wait (~seconds with the back-off)

__device__ __forceinline__ float mb_f(double v) { return (float)v; }
__device__ __forceinline__ float mb_f(float v) { return v; }
__device__ __forceinline__ float mb_f(float2 v) { return v.x; }
template <typename OT>
__device__ __forceinline__ OT mb_out(float v);
template <>
__device__ __forceinline__ float mb_out<float>(float v) {
    return v;
}
template <>
__device__ __forceinline__ float2 mb_out<float2>(float v) {
    return make_float2(v, 0.f);
}
// Level vectors: read-only cache path (NC) in the per-operation kernels,
// where no block of the launch writes them; coherent loads in the
// persistent kernel, where earlier phases of the same launch did.
template <bool NC, typename T>
__device__ __forceinline__ T ldv(const T* p) {
    if (NC) return __ldg(p);
    return *p;
}

#define MB_ROW_LOOP(i) for (int64_t i = U.lo + (threadIdx.x >> 5); i < U.hi; i += kMbT / 32)

// s = sum_q val[q] x[col[q]] for right-hand sides lane and lane + 32 over
// the entries [a, e) of a row, eight entries at a time, then four (their
// indices, then their gathers, are independent loads in flight together:
// the sweeps are bound by the latency of these gathers, and eight entries
// instead of four took the batched solve from 4.19 to 3.90 s).
template <bool NC>
__device__ __forceinline__ void row_dot(const int* __restrict__ col, const float* __restrict__ val,
                                        const float* __restrict__ x, int64_t a, int64_t e, int R, int lane,
                                        bool on0, bool on1, float& s0, float& s1, const float* xlo, int64_t nx) {
    // (xlo, nx: the gathered entries lie in xlo[0 .. nx), the bound of the
    // checked build's tests)
    (void)xlo;
    (void)nx;
    float t0 = 0.f, t1 = 0.f, u0 = 0.f, u1 = 0.f;
    int64_t q = a;
    for (; q + 8 <= e; q += 8) {
        int64_t c[8];
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            c[i] = (int64_t)__ldg(col + q + i) * R;
            v[i] = __ldg(val + q + i);
        }
        float x0[8], x1[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            x0[i] = on0 ? ldv<NC>(&RB_PT(x + c[i] + lane, xlo, nx)) : 0.f;
            x1[i] = on1 ? ldv<NC>(&RB_PT(x + c[i] + lane + 32, xlo, nx)) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            t0 = fmaf(v[i], x0[i], t0);
            u0 = fmaf(v[i + 1], x0[i + 1], u0);
            t1 = fmaf(v[i], x1[i], t1);
            u1 = fmaf(v[i + 1], x1[i + 1], u1);
        }
    }
    for (; q + 4 <= e; q += 4) {
        const int64_t c0 = (int64_t)__ldg(col + q) * R, c1 = (int64_t)__ldg(col + q + 1) * R;
        const int64_t c2 = (int64_t)__ldg(col + q + 2) * R, c3 = (int64_t)__ldg(col + q + 3) * R;
        const float v0 = __ldg(val + q), v1 = __ldg(val + q + 1), v2 = __ldg(val + q + 2), v3 = __ldg(val + q + 3);
        if (on0) {
            const float x0 = ldv<NC>(&RB_PT(x + c0 + lane, xlo, nx)), x1 = ldv<NC>(&RB_PT(x + c1 + lane, xlo, nx));
            const float x2 = ldv<NC>(&RB_PT(x + c2 + lane, xlo, nx)), x3 = ldv<NC>(&RB_PT(x + c3 + lane, xlo, nx));
            t0 = fmaf(v0, x0, t0);
            u0 = fmaf(v1, x1, u0);
            t0 = fmaf(v2, x2, t0);
            u0 = fmaf(v3, x3, u0);
        }
        if (on1) {
            const float x0 = ldv<NC>(&RB_PT(x + c0 + lane + 32, xlo, nx));
            const float x1 = ldv<NC>(&RB_PT(x + c1 + lane + 32, xlo, nx));
            const float x2 = ldv<NC>(&RB_PT(x + c2 + lane + 32, xlo, nx));
            const float x3 = ldv<NC>(&RB_PT(x + c3 + lane + 32, xlo, nx));
            t1 = fmaf(v0, x0, t1);
            u1 = fmaf(v1, x1, u1);
            t1 = fmaf(v2, x2, t1);
            u1 = fmaf(v3, x3, u1);
        }
    }
    for (; q < e; ++q) {
        const float v = __ldg(val + q);
        const int64_t c = (int64_t)__ldg(col + q) * R;
        if (on0) t0 = fmaf(v, ldv<NC>(&RB_PT(x + c + lane, xlo, nx)), t0);
        if (on1) t1 = fmaf(v, ldv<NC>(&RB_PT(x + c + lane + 32, xlo, nx)), t1);
    }
    s0 = t0 + u0;
    s1 = t1 + u1;
}

// ---- one tile (rows [U.lo, U.hi) of descriptor Dp) of each operation -------
// x = W b (the first pre-sweep from x = 0).  TOP: b is the caller's array.
template <bool TOP, bool NC, typename BT>
__device__ __forceinline__ void tile_first(const MbUnit& U, const MbLevel* Dp, int R, const BT* __restrict__ bin) {
    const int lane = threadIdx.x & 31;
    const float* __restrict__ dinv = Dp->dinv;
    const float* __restrict__ b = Dp->b;
    float* __restrict__ x = Dp->x;
    const int64_t roff = Dp->row_off;
    RB_SPAN(U.lo, U.hi - U.lo, Dp->N);
    MB_ROW_LOOP(i) {
        const int64_t g = (roff + i) * R;
        const float di = __ldg(dinv + i);
        if (lane < R) x[g + lane] = di * (TOP ? mb_f(__ldg(bin + g + lane)) : ldv<NC>(b + g + lane));
        if (lane + 32 < R) x[g + lane + 32] = di * (TOP ? mb_f(__ldg(bin + g + lane + 32)) : ldv<NC>(b + g + lane + 32));
    }
}

// MODE 0: xo = xi + W (b - A xi) into the level's other vector; MODE 1:
// r = b - A xi; MODE 2: the final level-0 sweep, into the caller's output.
// dir 0: xi = x (xo = t); dir 1: xi = t (xo = x).
template <bool TOP, bool NC, typename BT, typename OT, int MODE>
__device__ __forceinline__ void tile_sweep(const MbUnit& U, const MbLevel* Dp, int R, int dir,
                                           const BT* __restrict__ bin, OT* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    const int64_t* __restrict__ row_ptr = Dp->row_ptr;
    const int* __restrict__ col = Dp->col;
    const float* __restrict__ val = Dp->val;
    const float* __restrict__ dinv = Dp->dinv;
    const float* __restrict__ xi = dir ? Dp->t : Dp->x;
    float* __restrict__ xo = MODE == 1 ? Dp->r : (dir ? Dp->x : Dp->t);
    const float* __restrict__ b = Dp->b;
    const int64_t roff = Dp->row_off;
    RB_SPAN(U.lo, U.hi - U.lo, Dp->N);
    MB_ROW_LOOP(i) {
        const int64_t a = __ldg(row_ptr + i), e = __ldg(row_ptr + i + 1);
        float s0, s1;
        row_dot<NC>(col, val, xi, a, e, R, lane, on0, on1, s0, s1, xi + roff * R, Dp->N * R);
        const int64_t g = (roff + i) * R;
        const float di = __ldg(dinv + i);
        if (on0) {
            const float r = (TOP ? mb_f(__ldg(bin + g + lane)) : ldv<NC>(b + g + lane)) - s0;
            if (MODE == 1) xo[g + lane] = r;
            else if (MODE == 2) out[g + lane] = mb_out<OT>(fmaf(di, r, ldv<NC>(xi + g + lane)));
            else xo[g + lane] = fmaf(di, r, ldv<NC>(xi + g + lane));
        }
        if (on1) {
            const float r = (TOP ? mb_f(__ldg(bin + g + lane + 32)) : ldv<NC>(b + g + lane + 32)) - s1;
            if (MODE == 1) xo[g + lane + 32] = r;
            else if (MODE == 2) out[g + lane + 32] = mb_out<OT>(fmaf(di, r, ldv<NC>(xi + g + lane + 32)));
            else xo[g + lane + 32] = fmaf(di, r, ldv<NC>(xi + g + lane + 32));
        }
    }
}

// b_next = R r: rows of the next level, descriptor of level l.
template <bool NC>
__device__ __forceinline__ void tile_restrict(const MbUnit& U, const MbLevel* Dp, int R) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    const int64_t* __restrict__ rrow = Dp->rrow;
    const int* __restrict__ rcol = Dp->rcol;
    const float* __restrict__ rval = Dp->rval;
    const float* __restrict__ r = Dp->r + Dp->row_off * R;
    float* __restrict__ y = Dp->b_next;
    RB_SPAN(U.lo, U.hi - U.lo, Dp->N_next);
    MB_ROW_LOOP(i) {
        const int64_t a = __ldg(rrow + i), e = __ldg(rrow + i + 1);
        float s0, s1;
        row_dot<NC>(rcol, rval, r, a, e, R, lane, on0, on1, s0, s1, r, Dp->N * R);
        if (on0) y[i * R + lane] = s0;
        if (on1) y[i * R + lane + 32] = s1;
    }
}

// x += P e_next on the level's current vector (dir 0: x, 1: t).
template <bool NC>
__device__ __forceinline__ void tile_prolong(const MbUnit& U, const MbLevel* Dp, int R, int dir) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    const int32_t* __restrict__ pidx = Dp->pidx;
    const float* __restrict__ pval = Dp->pval;
    const float* __restrict__ en = Dp->e_next;
    float* __restrict__ xb = (dir ? Dp->t : Dp->x) + Dp->row_off * R;
    RB_SPAN(U.lo, U.hi - U.lo, Dp->N);
    MB_ROW_LOOP(i) {
        float* x = xb + i * R;
        float s0 = on0 ? x[lane] : 0.f, s1 = on1 ? x[lane + 32] : 0.f;
#pragma unroll
        for (int j = 0; j < kMgK; ++j) {
            const float a = __ldg(pval + i * kMgK + j);
            const int64_t c = (int64_t)__ldg(pidx + i * kMgK + j) * R;
            if (on0) s0 = fmaf(a, ldv<NC>(&RB_PT(en + c + lane, en, Dp->N_next * R)), s0);
            if (on1) s1 = fmaf(a, ldv<NC>(&RB_PT(en + c + lane + 32, en, Dp->N_next * R)), s1);
        }
        if (on0) x[lane] = s0;
        if (on1) x[lane + 32] = s1;
    }
}

// Coarsest level: x = Minv b (dense N x N, N <= kMgCoarsest).  TOP: a
// one-level instance, b and the output are the caller's arrays.
template <bool TOP, bool NC, typename BT, typename OT>
__device__ __forceinline__ void tile_dense(const MbUnit& U, const MbLevel* Dp, int R, const BT* __restrict__ bin,
                                           OT* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    const float* __restrict__ minv = Dp->minv;
    const float* __restrict__ b = Dp->b;
    float* __restrict__ x = Dp->x;
    const int64_t n = Dp->N, roff = Dp->row_off;
    RB_SPAN(U.lo, U.hi - U.lo, n);
    MB_ROW_LOOP(i) {
        float s0 = 0.f, s1 = 0.f;
        for (int64_t j = 0; j < n; ++j) {
            const float a = __ldg(minv + i * n + j);
            const int64_t c = (roff + j) * R;
            if (on0) s0 = fmaf(a, TOP ? mb_f(__ldg(bin + c + lane)) : ldv<NC>(b + c + lane), s0);
            if (on1) s1 = fmaf(a, TOP ? mb_f(__ldg(bin + c + lane + 32)) : ldv<NC>(b + c + lane + 32), s1);
        }
        const int64_t g = (roff + i) * R;
        if (TOP) {
            if (on0) out[g + lane] = mb_out<OT>(s0);
            if (on1) out[g + lane + 32] = mb_out<OT>(s1);
        } else {
            if (on0) x[g + lane] = s0;
            if (on1) x[g + lane + 32] = s1;
        }
    }
}

// ---- per-operation kernels (level 0): a block per unit -------------------
__device__ __forceinline__ bool unit_live(const MbLevel* Dp, const int* live) {
    return !live || *(volatile const int*)(live + Dp->inst) != 0;
}

template <bool TOP, typename BT>
__global__ void __launch_bounds__(kMbT) mb_first_kernel(const MbUnit* __restrict__ units, int n_units,
                                                        const MbLevel* __restrict__ descs, int R,
                                                        const BT* __restrict__ bin, const int* live) {
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const MbUnit U = units[u];
        const MbLevel* Dp = descs + U.desc;
        if (unit_live(Dp, live)) tile_first<TOP, true, BT>(U, Dp, R, bin);
    }
}

template <bool TOP, typename BT, typename OT, int MODE>
__global__ void __launch_bounds__(kMbT) mb_sweep_kernel(const MbUnit* __restrict__ units, int n_units,
                                                        const MbLevel* __restrict__ descs, int R, int dir,
                                                        const BT* __restrict__ bin, OT* __restrict__ out,
                                                        const int* live) {
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const MbUnit U = units[u];
        const MbLevel* Dp = descs + U.desc;
        if (unit_live(Dp, live)) tile_sweep<TOP, true, BT, OT, MODE>(U, Dp, R, dir, bin, out);
    }
}

__global__ void __launch_bounds__(kMbT) mb_restrict_kernel(const MbUnit* __restrict__ units, int n_units,
                                                           const MbLevel* __restrict__ descs, int R, const int* live) {
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const MbUnit U = units[u];
        const MbLevel* Dp = descs + U.desc;
        if (unit_live(Dp, live)) tile_restrict<true>(U, Dp, R);
    }
}

__global__ void __launch_bounds__(kMbT) mb_prolong_kernel(const MbUnit* __restrict__ units, int n_units,
                                                          const MbLevel* __restrict__ descs, int R, int dir,
                                                          const int* live) {
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const MbUnit U = units[u];
        const MbLevel* Dp = descs + U.desc;
        if (unit_live(Dp, live)) tile_prolong<true>(U, Dp, R, dir);
    }
}

template <bool TOP, typename BT, typename OT>
__global__ void __launch_bounds__(kMbT) mb_dense_kernel(const MbUnit* __restrict__ units, int n_units,
                                                        const MbLevel* __restrict__ descs, int R,
                                                        const BT* __restrict__ bin, OT* __restrict__ out,
                                                        const int* live) {
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const MbUnit U = units[u];
        const MbLevel* Dp = descs + U.desc;
        if (unit_live(Dp, live)) tile_dense<TOP, true, BT, OT>(U, Dp, R, bin, out);
    }
}

// ---- the persistent kernel of levels >= 1 --------------------------------
// status[0]: stop (set on a timeout); status[1]: a wait ran out.
__global__ void __launch_bounds__(kMbT) mb_coarse_kernel(const MbTask* __restrict__ tasks, int ntasks,
                                                         const MbLevel* __restrict__ descs, int R, int* head,
                                                         int* done, int ncount, int* status, long long spin_limit,
                                                         const int* live) {
    (void)ncount;  // counters: bound of the checked build's tests
    __shared__ int s_task, s_go;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(head, 1);
            int go = t < ntasks && *(volatile int*)status == 0;
            if (go && tasks[t].wait >= 0) {
                const int* c = &RB_AT(done, tasks[t].wait, ncount);
                const int need = tasks[t].need;
                long long polls = 0;
                while (*(volatile const int*)c < need) {
                    if (*(volatile int*)status != 0) {
                        go = 0;
                        break;
                    }
                    if (++polls > spin_limit) {
                        atomicExch(status + 1, 1);
                        atomicExch(status, 1);
                        go = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();  // the producers' writes are visible past this point
            s_task = t;
            s_go = go;
        }
        __syncthreads();
        if (!s_go) return;
        const MbTask T = tasks[s_task];
        const MbLevel* Dp = descs + T.desc;
        if (unit_live(Dp, live)) {
            MbUnit U;
            U.desc = T.desc;
            U.pad = 0;
            U.lo = T.lo;
            U.hi = T.hi;
            switch (T.op) {
                case kOpFirst: tile_first<false, false, float>(U, Dp, R, nullptr); break;
                case kOpSweep: tile_sweep<false, false, float, float, 0>(U, Dp, R, T.dir, nullptr, nullptr); break;
                case kOpResid: tile_sweep<false, false, float, float, 1>(U, Dp, R, T.dir, nullptr, nullptr); break;
                case kOpRestrict: tile_restrict<false>(U, Dp, R); break;
                case kOpProlong: tile_prolong<false>(U, Dp, R, T.dir); break;
                default: tile_dense<false, false, float, float>(U, Dp, R, nullptr, nullptr); break;
            }
        }
        __syncthreads();  // every thread's writes of the tile ...
        if (threadIdx.x == 0) {
            __threadfence();  // ... before the tile counts as done
            atomicAdd(&RB_AT(done, T.post, ncount), 1);
        }
    }
}

}  // namespace

namespace {
// Tasks of the coarse levels: per level (at most 2 nu + 3 operations of
// kMbTileRows rows; the levels >= 1 of an instance hold fewer rows than its
// level 0) plus partial tiles and the dense tiles; nu <= 4.
int64_t coarse_task_bound(int n_inst, int64_t total_nodes) {
    return 11 * (total_nodes / kMbTileRows + (int64_t)n_inst * RBFFD_MG_MAX_LEVELS) +
           (int64_t)n_inst * (kMgCoarsest / kMbDenseRows + 1);
}
int64_t counter_bound(int n_inst) { return (int64_t)n_inst * (11 * RBFFD_MG_MAX_LEVELS + 2); }
}  // namespace

size_t mg_batch_table_bytes(int n_inst, int64_t total_nodes) {
    // units of every level (the levels of one instance hold fewer than twice
    // its nodes; the restriction's sets fewer than its nodes), plus partial
    // tiles and the dense tiles
    const int64_t units = 3 * (total_nodes / kMbTileRows + 1) + 3 * (int64_t)n_inst * RBFFD_MG_MAX_LEVELS +
                          (int64_t)n_inst * (kMgCoarsest / kMbDenseRows + 1);
    return align_up((size_t)n_inst * RBFFD_MG_MAX_LEVELS * sizeof(MbLevel)) + align_up((size_t)units * sizeof(MbUnit)) +
           align_up((size_t)coarse_task_bound(n_inst, total_nodes) * sizeof(MbTask)) +
           align_up((size_t)(counter_bound(n_inst) + 4) * sizeof(int));
}

int mg_batch_build(const MgHierarchy* const* H, const int64_t* node_off, int n_inst, int R, float* x0, float* t0,
                   float* r0, float* coarse, const size_t* coarse_off, void* tables, size_t table_bytes,
                   int persistent, long long spin_limit, int wait_test, cudaStream_t st, MgBatch* out) {
    if (!H || !node_off || n_inst < 1 || R < 1 || R > 64 || !x0 || !t0 || !r0 || !tables || !out)
        return RBFFD_ERR_INVALID_ARG;
    int64_t total = 0;
    int nu = -1;
    int lmax = 0;
    for (int i = 0; i < n_inst; ++i) {
        if (!H[i] || !H[i]->has32 || H[i]->col_base != (int)node_off[i]) return RBFFD_ERR_INVALID_ARG;
        if (nu >= 0 && H[i]->nu != nu) return RBFFD_ERR_INVALID_ARG;  // one schedule for all
        nu = H[i]->nu;
        total += H[i]->lv[0].N;
        lmax = std::max(lmax, H[i]->n_levels);
        if (H[i]->n_levels > 1 && !coarse) return RBFFD_ERR_INVALID_ARG;
    }
    if (nu < 1 || nu > 4 || table_bytes < mg_batch_table_bytes(n_inst, total)) return RBFFD_ERR_WORKSPACE;
    constexpr int ML = RBFFD_MG_MAX_LEVELS;
    std::vector<MbLevel> desc((size_t)n_inst * ML);
    std::memset(desc.data(), 0, desc.size() * sizeof(MbLevel));
    for (int i = 0; i < n_inst; ++i) {
        const MgHierarchy& h = *H[i];
        size_t off = coarse_off ? coarse_off[i] : 0;
        for (int l = 0; l < h.n_levels; ++l) {
            const MgLevel& L = h.lv[l];
            MbLevel& D = desc[(size_t)i * ML + l];
            D.row_ptr = L.row_ptr;
            D.col = L.col;
            D.val = L.val32;
            D.dinv = L.dinv32;
            D.minv = L.minv32;
            D.N = L.N;
            D.inst = i;
            if (l == 0) {
                D.x = x0;
                D.t = t0;
                D.r = r0;
                D.b = nullptr;
                D.row_off = node_off[i];
            } else {
                const size_t n = (size_t)L.N * R;
                D.x = coarse + off;
                D.t = coarse + off + n;
                D.r = coarse + off + 2 * n;
                D.b = coarse + off + 3 * n;
                D.row_off = 0;
                off += 4 * n;
            }
        }
        for (int l = 0; l + 1 < h.n_levels; ++l) {
            const MgLevel& L = h.lv[l];
            MbLevel& D = desc[(size_t)i * ML + l];
            const MbLevel& C = desc[(size_t)i * ML + l + 1];
            D.pidx = L.pidx;
            D.pval = L.pval32;
            D.rrow = L.rrow;
            D.rcol = L.rcol;
            D.rval = L.rval32;
            D.N_next = C.N;
            D.b_next = C.b;
            // the next level's result: its dense solve writes x; a smoothed
            // level ends after 2 nu - 1 vector swaps, in t
            D.e_next = (l + 1 == h.n_levels - 1) ? C.x : C.t;
        }
    }
    MgBatch B{};
    B.levels = lmax;
    B.nu = nu;
    B.persistent = persistent ? 1 : 0;
    const int pre_dir = (nu - 1) & 1;  // the vector holding the iterate after the pre-sweeps
    // units per level: the instances going deeper (a), those whose coarsest
    // level it is (d), and the next level's rows of the former (c, the
    // restriction)
    std::vector<MbUnit> units;
    auto tiles = [&](std::vector<MbUnit>& v, int i, int l, int64_t rows, int per) {
        for (int64_t lo = 0; lo < rows; lo += per) {
            MbUnit u{};
            u.desc = i * ML + l;
            u.lo = lo;
            u.hi = std::min<int64_t>(rows, lo + per);
            v.push_back(u);
        }
    };
    for (int l = 0; l < lmax; ++l) {
        B.a_off[l] = (int)units.size();
        for (int i = 0; i < n_inst; ++i)
            if (H[i]->n_levels - 1 > l) tiles(units, i, l, H[i]->lv[l].N, kMbTileRows);
        B.a_n[l] = (int)units.size() - B.a_off[l];
        B.d_off[l] = (int)units.size();
        for (int i = 0; i < n_inst; ++i)
            if (H[i]->n_levels - 1 == l) tiles(units, i, l, H[i]->lv[l].N, kMbDenseRows);
        B.d_n[l] = (int)units.size() - B.d_off[l];
        B.c_off[l] = (int)units.size();
        for (int i = 0; i < n_inst; ++i)
            if (H[i]->n_levels - 1 > l) tiles(units, i, l, H[i]->lv[l + 1].N, kMbTileRows);
        B.c_n[l] = (int)units.size() - B.c_off[l];
    }
    // the coarse levels' phases per instance (levels 1 .. L-1): descend --
    // first sweep, nu - 1 sweeps, residual, restriction per level, the dense
    // solve at the coarsest; ascend -- prolongation and nu sweeps per level
    struct Phase {
        int8_t op, dir;
        int level;
        int64_t rows;
    };
    std::vector<std::vector<Phase>> ph(n_inst);
    size_t kmax = 0;
    for (int i = 0; i < n_inst; ++i) {
        const MgHierarchy& h = *H[i];
        const int L = h.n_levels;
        if (L < 2) continue;
        std::vector<Phase>& P = ph[i];
        for (int l = 1; l < L - 1; ++l) {
            P.push_back({kOpFirst, 0, l, h.lv[l].N});
            for (int k = 1; k < nu; ++k) P.push_back({kOpSweep, (int8_t)((k - 1) & 1), l, h.lv[l].N});
            P.push_back({kOpResid, (int8_t)pre_dir, l, h.lv[l].N});
            P.push_back({kOpRestrict, 0, l, h.lv[l + 1].N});
        }
        P.push_back({kOpDense, 0, L - 1, h.lv[L - 1].N});
        for (int l = L - 2; l >= 1; --l) {
            P.push_back({kOpProlong, (int8_t)pre_dir, l, h.lv[l].N});
            for (int k = 0; k < nu; ++k) P.push_back({kOpSweep, (int8_t)((pre_dir + k) & 1), l, h.lv[l].N});
        }
        kmax = std::max(kmax, P.size());
    }
    // counters: one per (instance, phase), plus a sentinel nothing increments
    std::vector<int> cbase(n_inst, 0);
    int ncount = 0;
    for (int i = 0; i < n_inst; ++i) {
        cbase[i] = ncount;
        ncount += (int)ph[i].size();
    }
    const int sentinel = ncount++;
    auto ntiles = [&](const Phase& p) {
        const int per = p.op == kOpDense ? kMbDenseRows : kMbTileRows;
        return (int)((p.rows + per - 1) / per);
    };
    std::vector<MbTask> tasks;
    if (!persistent) kmax = 0;  // the per-operation launches need no task queue
    for (size_t k = 0; k < kmax; ++k)
        for (int i = 0; i < n_inst; ++i) {
            if (k >= ph[i].size()) continue;
            const Phase& p = ph[i][k];
            const int per = p.op == kOpDense ? kMbDenseRows : kMbTileRows;
            // (the restriction's rows are level l + 1's, read with level l's
            // descriptor)
            for (int64_t lo = 0; lo < p.rows; lo += per) {
                MbTask t{};
                t.desc = i * ML + p.level;
                t.op = p.op;
                t.dir = p.dir;
                t.lo = lo;
                t.hi = std::min<int64_t>(p.rows, lo + per);
                t.wait = k > 0 ? cbase[i] + (int)k - 1 : -1;
                t.need = k > 0 ? ntiles(ph[i][k - 1]) : 0;
                t.post = cbase[i] + (int)k;
                if (wait_test && tasks.empty()) {  // tests only: a wait nothing ends
                    t.wait = sentinel;
                    t.need = 1;
                }
                tasks.push_back(t);
            }
        }
    Carver c(tables);
    MbLevel* ddesc = c.take<MbLevel>(desc.size());
    MbUnit* dunits = c.take<MbUnit>(std::max<size_t>(units.size(), 1));
    MbTask* dtasks = c.take<MbTask>(std::max<size_t>(tasks.size(), 1));
    int* ints = c.take<int>((size_t)ncount + 4);
    if (c.off > table_bytes || (int64_t)tasks.size() > coarse_task_bound(n_inst, total) ||
        ncount > counter_bound(n_inst) + 1)
        return RBFFD_ERR_WORKSPACE;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(ddesc, desc.data(), desc.size() * sizeof(MbLevel), cudaMemcpyHostToDevice, st));
    if (!units.empty())
        RBFFD_CUDA_TRY(cudaMemcpyAsync(dunits, units.data(), units.size() * sizeof(MbUnit), cudaMemcpyHostToDevice, st));
    if (!tasks.empty())
        RBFFD_CUDA_TRY(cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(MbTask), cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaMemsetAsync(ints, 0, sizeof(int) * ((size_t)ncount + 4), st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));  // the host tables go out of scope
    B.desc = ddesc;
    B.units = dunits;
    B.tasks = dtasks;
    B.ntasks = (int)tasks.size();
    B.status = ints;          // [0] stop, [1] a wait ran out
    B.head = ints + 2;
    B.done = ints + 4;
    B.ncount = ncount;
    B.spin_limit = spin_limit > 0 ? spin_limit : kMbDefaultSpin;
    int per_sm = 0;
    RBFFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mb_coarse_kernel, kMbT, 0));
    B.coarse_grid = std::max(1, std::min(B.ntasks, std::max(per_sm, 1) * sm_count()));
    *out = B;
    return RBFFD_OK;
}

int mg_batch_apply_df(const MgBatch& B, int R, const float2* b, float2* x, const int* live, cudaStream_t st,
                      int* launches) {
    if (!B.desc || !b || !x || R < 1 || R > 64) return RBFFD_ERR_INVALID_ARG;
    int n = 0;
    const MbLevel* D = B.desc;
    const int pre_dir = (B.nu - 1) & 1;
    const bool pers = B.persistent && B.ntasks > 0;
    // descend: level by level (only level 0 in the persistent mode)
    for (int l = 0; l < (pers ? 1 : B.levels); ++l) {
        const bool top = l == 0;
        if (B.d_n[l]) {
            const MbUnit* u = B.units + B.d_off[l];
            if (top) mb_dense_kernel<true, float2, float2><<<B.d_n[l], kMbT, 0, st>>>(u, B.d_n[l], D, R, b, x, live);
            else mb_dense_kernel<false, float2, float2><<<B.d_n[l], kMbT, 0, st>>>(u, B.d_n[l], D, R, b, x, live);
            ++n;
        }
        if (!B.a_n[l]) continue;
        const MbUnit* u = B.units + B.a_off[l];
        const int g = B.a_n[l];
        if (top) mb_first_kernel<true, float2><<<g, kMbT, 0, st>>>(u, g, D, R, b, live);
        else mb_first_kernel<false, float2><<<g, kMbT, 0, st>>>(u, g, D, R, b, live);
        for (int k = 1; k < B.nu; ++k) {
            const int dir = (k - 1) & 1;
            if (top) mb_sweep_kernel<true, float2, float2, 0><<<g, kMbT, 0, st>>>(u, g, D, R, dir, b, x, live);
            else mb_sweep_kernel<false, float2, float2, 0><<<g, kMbT, 0, st>>>(u, g, D, R, dir, b, x, live);
        }
        if (top) mb_sweep_kernel<true, float2, float2, 1><<<g, kMbT, 0, st>>>(u, g, D, R, pre_dir, b, x, live);
        else mb_sweep_kernel<false, float2, float2, 1><<<g, kMbT, 0, st>>>(u, g, D, R, pre_dir, b, x, live);
        mb_restrict_kernel<<<B.c_n[l], kMbT, 0, st>>>(B.units + B.c_off[l], B.c_n[l], D, R, live);
        n += B.nu + 2;
    }
    // levels >= 1 of every instance: one persistent launch
    if (pers && B.a_n[0]) {
        RBFFD_CUDA_TRY(cudaMemsetAsync(B.head, 0, sizeof(int) * (2 + (size_t)B.ncount), st));
        mb_coarse_kernel<<<B.coarse_grid, kMbT, 0, st>>>(B.tasks, B.ntasks, D, R, B.head, B.done, B.ncount,
                                                          B.status, B.spin_limit, live);
        ++n;
    }
    // ascend
    for (int l = (pers ? 0 : B.levels - 2); l >= 0; --l) {
        if (!B.a_n[l]) continue;
        const bool top = l == 0;
        const MbUnit* u = B.units + B.a_off[l];
        const int g = B.a_n[l];
        mb_prolong_kernel<<<g, kMbT, 0, st>>>(u, g, D, R, pre_dir, live);
        ++n;
        for (int k = 0; k < B.nu; ++k) {
            const int dir = (pre_dir + k) & 1;
            if (top && k == B.nu - 1)
                mb_sweep_kernel<true, float2, float2, 2><<<g, kMbT, 0, st>>>(u, g, D, R, dir, b, x, live);
            else if (top)
                mb_sweep_kernel<true, float2, float2, 0><<<g, kMbT, 0, st>>>(u, g, D, R, dir, b, x, live);
            else
                mb_sweep_kernel<false, float2, float2, 0><<<g, kMbT, 0, st>>>(u, g, D, R, dir, b, x, live);
            ++n;
        }
    }
    if (launches) *launches += n;  // (the caller accounts them: they may be captured, not run)
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

int mg_batch_timed_out(const MgBatch& B, cudaStream_t st, bool* out) {
    int h[2] = {0, 0};
    RBFFD_CUDA_TRY(cudaMemcpyAsync(h, B.status, sizeof(h), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    *out = h[1] != 0;
    return RBFFD_OK;
}

}  // namespace rbffd
