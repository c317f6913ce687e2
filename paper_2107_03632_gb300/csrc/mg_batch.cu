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

namespace {

constexpr int kMbT = 256;        // threads per block (8 warps)
constexpr int kMbTileRows = 256; // rows per unit
constexpr int kMbDenseRows = 16; // rows per unit of the dense coarsest solves

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

// Grid-stride over units (a block per unit); the body sees the unit U and
// its descriptor Dp; warp w of the block takes rows lo + w, lo + w + 8, ...
#define MB_UNITS(units, n_units, live, ...)                                         \
    for (int u_ = blockIdx.x; u_ < (n_units); u_ += gridDim.x) {                   \
        const MbUnit U = (units)[u_];                                               \
        const MbLevel* Dp = descs + U.desc;                                         \
        if ((live) && *(volatile const int*)((live) + Dp->inst) == 0) continue;      \
        __VA_ARGS__                                                                 \
    }
#define MB_ROW_LOOP(i) for (int64_t i = U.lo + (threadIdx.x >> 5); i < U.hi; i += kMbT / 32)

// s = sum_q val[q] x[col[q]] for right-hand sides lane and lane + 32 over
// the entries [a, e) of a row, four entries at a time (their indices, then
// their gathers, are independent loads in flight together).
__device__ __forceinline__ void row_dot(const int* __restrict__ col, const float* __restrict__ val,
                                        const float* __restrict__ x, int64_t a, int64_t e, int R, int lane,
                                        bool on0, bool on1, float& s0, float& s1) {
    float t0 = 0.f, t1 = 0.f, u0 = 0.f, u1 = 0.f;
    int64_t q = a;
    for (; q + 4 <= e; q += 4) {
        const int64_t c0 = (int64_t)__ldg(col + q) * R, c1 = (int64_t)__ldg(col + q + 1) * R;
        const int64_t c2 = (int64_t)__ldg(col + q + 2) * R, c3 = (int64_t)__ldg(col + q + 3) * R;
        const float v0 = __ldg(val + q), v1 = __ldg(val + q + 1), v2 = __ldg(val + q + 2), v3 = __ldg(val + q + 3);
        if (on0) {
            const float x0 = __ldg(x + c0 + lane), x1 = __ldg(x + c1 + lane);
            const float x2 = __ldg(x + c2 + lane), x3 = __ldg(x + c3 + lane);
            t0 = fmaf(v0, x0, t0);
            u0 = fmaf(v1, x1, u0);
            t0 = fmaf(v2, x2, t0);
            u0 = fmaf(v3, x3, u0);
        }
        if (on1) {
            const float x0 = __ldg(x + c0 + lane + 32), x1 = __ldg(x + c1 + lane + 32);
            const float x2 = __ldg(x + c2 + lane + 32), x3 = __ldg(x + c3 + lane + 32);
            t1 = fmaf(v0, x0, t1);
            u1 = fmaf(v1, x1, u1);
            t1 = fmaf(v2, x2, t1);
            u1 = fmaf(v3, x3, u1);
        }
    }
    for (; q < e; ++q) {
        const float v = __ldg(val + q);
        const int64_t c = (int64_t)__ldg(col + q) * R;
        if (on0) t0 = fmaf(v, __ldg(x + c + lane), t0);
        if (on1) t1 = fmaf(v, __ldg(x + c + lane + 32), t1);
    }
    s0 = t0 + u0;
    s1 = t1 + u1;
}

// x = W b (the first pre-sweep from x = 0).  TOP: b is the caller's array.
template <bool TOP, typename BT>
__global__ void __launch_bounds__(kMbT) mb_first_kernel(const MbUnit* __restrict__ units, int n_units,
                                                        const MbLevel* __restrict__ descs, int R,
                                                        const BT* __restrict__ bin, const int* live) {
    const int lane = threadIdx.x & 31;
    MB_UNITS(units, n_units, live, {
        const float* __restrict__ dinv = Dp->dinv;
        const float* __restrict__ b = Dp->b;
        float* __restrict__ x = Dp->x;
        const int64_t roff = Dp->row_off;
        MB_ROW_LOOP(i) {
            const int64_t g = (roff + i) * R;
            const float di = __ldg(dinv + i);
            if (lane < R) x[g + lane] = di * (TOP ? mb_f(__ldg(bin + g + lane)) : __ldg(b + g + lane));
            if (lane + 32 < R) x[g + lane + 32] = di * (TOP ? mb_f(__ldg(bin + g + lane + 32)) : __ldg(b + g + lane + 32));
        }
    })
}

// MODE 0: xo = xi + W (b - A xi) into the level's other vector; MODE 1:
// r = b - A xi; MODE 2: the final level-0 sweep, into the caller's output.
// dir 0: xi = x (xo = t); dir 1: xi = t (xo = x).  xi is only read here
// (every write goes to another vector), hence the read-only loads.
template <bool TOP, typename BT, typename OT, int MODE>
__global__ void __launch_bounds__(kMbT) mb_sweep_kernel(const MbUnit* __restrict__ units, int n_units,
                                                        const MbLevel* __restrict__ descs, int R, int dir,
                                                        const BT* __restrict__ bin, OT* __restrict__ out,
                                                        const int* live) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    MB_UNITS(units, n_units, live, {
        const int64_t* __restrict__ row_ptr = Dp->row_ptr;
        const int* __restrict__ col = Dp->col;
        const float* __restrict__ val = Dp->val;
        const float* __restrict__ dinv = Dp->dinv;
        const float* __restrict__ xi = dir ? Dp->t : Dp->x;
        float* __restrict__ xo = MODE == 1 ? Dp->r : (dir ? Dp->x : Dp->t);
        const float* __restrict__ b = Dp->b;
        const int64_t roff = Dp->row_off;
        MB_ROW_LOOP(i) {
            const int64_t a = __ldg(row_ptr + i), e = __ldg(row_ptr + i + 1);
            float s0, s1;
            row_dot(col, val, xi, a, e, R, lane, on0, on1, s0, s1);
            const int64_t g = (roff + i) * R;
            const float di = __ldg(dinv + i);
            if (on0) {
                const float r = (TOP ? mb_f(__ldg(bin + g + lane)) : __ldg(b + g + lane)) - s0;
                if (MODE == 1) xo[g + lane] = r;
                else if (MODE == 2) out[g + lane] = mb_out<OT>(fmaf(di, r, __ldg(xi + g + lane)));
                else xo[g + lane] = fmaf(di, r, __ldg(xi + g + lane));
            }
            if (on1) {
                const float r = (TOP ? mb_f(__ldg(bin + g + lane + 32)) : __ldg(b + g + lane + 32)) - s1;
                if (MODE == 1) xo[g + lane + 32] = r;
                else if (MODE == 2) out[g + lane + 32] = mb_out<OT>(fmaf(di, r, __ldg(xi + g + lane + 32)));
                else xo[g + lane + 32] = fmaf(di, r, __ldg(xi + g + lane + 32));
            }
        }
    })
}

// b_next = R r: units over the next level's rows, descriptors of level l.
__global__ void __launch_bounds__(kMbT) mb_restrict_kernel(const MbUnit* __restrict__ units, int n_units,
                                                           const MbLevel* __restrict__ descs, int R,
                                                           const int* live) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    MB_UNITS(units, n_units, live, {
        const int64_t* __restrict__ rrow = Dp->rrow;
        const int* __restrict__ rcol = Dp->rcol;
        const float* __restrict__ rval = Dp->rval;
        const float* __restrict__ r = Dp->r + Dp->row_off * R;
        float* __restrict__ y = Dp->b_next;
        MB_ROW_LOOP(i) {
            const int64_t a = __ldg(rrow + i), e = __ldg(rrow + i + 1);
            float s0, s1;
            row_dot(rcol, rval, r, a, e, R, lane, on0, on1, s0, s1);
            if (on0) y[i * R + lane] = s0;
            if (on1) y[i * R + lane + 32] = s1;
        }
    })
}

// x += P e_next on the level's current vector (dir 0: x, 1: t).
__global__ void __launch_bounds__(kMbT) mb_prolong_kernel(const MbUnit* __restrict__ units, int n_units,
                                                          const MbLevel* __restrict__ descs, int R, int dir,
                                                          const int* live) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    MB_UNITS(units, n_units, live, {
        const int32_t* __restrict__ pidx = Dp->pidx;
        const float* __restrict__ pval = Dp->pval;
        const float* __restrict__ en = Dp->e_next;
        float* __restrict__ xb = (dir ? Dp->t : Dp->x) + Dp->row_off * R;
        MB_ROW_LOOP(i) {
            float* x = xb + i * R;
            float s0 = on0 ? x[lane] : 0.f, s1 = on1 ? x[lane + 32] : 0.f;
#pragma unroll
            for (int j = 0; j < kMgK; ++j) {
                const float a = __ldg(pval + i * kMgK + j);
                const int64_t c = (int64_t)__ldg(pidx + i * kMgK + j) * R;
                if (on0) s0 = fmaf(a, __ldg(en + c + lane), s0);
                if (on1) s1 = fmaf(a, __ldg(en + c + lane + 32), s1);
            }
            if (on0) x[lane] = s0;
            if (on1) x[lane + 32] = s1;
        }
    })
}

// Coarsest level: x = Minv b (dense N x N, N <= kMgCoarsest).  TOP: a
// one-level instance, b and the output are the caller's arrays.
template <bool TOP, typename BT, typename OT>
__global__ void __launch_bounds__(kMbT) mb_dense_kernel(const MbUnit* __restrict__ units, int n_units,
                                                        const MbLevel* __restrict__ descs, int R,
                                                        const BT* __restrict__ bin, OT* __restrict__ out,
                                                        const int* live) {
    const int lane = threadIdx.x & 31;
    const bool on0 = lane < R, on1 = lane + 32 < R;
    MB_UNITS(units, n_units, live, {
        const float* __restrict__ minv = Dp->minv;
        const float* __restrict__ b = Dp->b;
        float* __restrict__ x = Dp->x;
        const int64_t n = Dp->N, roff = Dp->row_off;
        MB_ROW_LOOP(i) {
            float s0 = 0.f, s1 = 0.f;
            for (int64_t j = 0; j < n; ++j) {
                const float a = __ldg(minv + i * n + j);
                const int64_t c = (roff + j) * R;
                if (on0) s0 = fmaf(a, TOP ? mb_f(__ldg(bin + c + lane)) : __ldg(b + c + lane), s0);
                if (on1) s1 = fmaf(a, TOP ? mb_f(__ldg(bin + c + lane + 32)) : __ldg(b + c + lane + 32), s1);
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
    })
}

// one block per unit (a grid-stride loop over more units than resident
// blocks would run in uneven waves)
int mb_grid(int n_units) { return std::max(1, n_units); }

}  // namespace

size_t mg_batch_table_bytes(int n_inst, int64_t total_nodes) {
    // descriptors: n_inst x max levels; units: every level's tiles (the
    // levels of one instance hold fewer than twice its nodes) in the three
    // sets, plus one partial tile per (instance, level, set)
    const int64_t tiles = 2 * (2 * total_nodes / kMbTileRows + 2) + 3 * (int64_t)n_inst * RBFFD_MG_MAX_LEVELS +
                          (int64_t)n_inst * (kMgCoarsest / kMbDenseRows + 1);
    return align_up((size_t)n_inst * RBFFD_MG_MAX_LEVELS * sizeof(MbLevel)) + align_up((size_t)tiles * sizeof(MbUnit));
}

int mg_batch_build(const MgHierarchy* const* H, const int64_t* node_off, int n_inst, int R, float* x0, float* t0,
                   float* r0, float* coarse, const size_t* coarse_off, void* tables, size_t table_bytes,
                   cudaStream_t st, MgBatch* out) {
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
    if (nu < 1 || table_bytes < mg_batch_table_bytes(n_inst, total)) return RBFFD_ERR_WORKSPACE;
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
    // unit tables: per level, the instances going deeper (A), those whose
    // coarsest level it is (D), and the next level's rows of A (restriction)
    std::vector<MbUnit> units;
    MgBatch B{};
    B.levels = lmax;
    B.nu = nu;
    auto tiles = [&](int i, int l, int64_t rows, int per) {
        for (int64_t lo = 0; lo < rows; lo += per) {
            MbUnit u{};
            u.desc = i * ML + l;
            u.lo = lo;
            u.hi = std::min<int64_t>(rows, lo + per);
            units.push_back(u);
        }
    };
    for (int l = 0; l < lmax; ++l) {
        B.a_off[l] = (int)units.size();
        for (int i = 0; i < n_inst; ++i)
            if (H[i]->n_levels - 1 > l) tiles(i, l, H[i]->lv[l].N, kMbTileRows);
        B.a_n[l] = (int)units.size() - B.a_off[l];
        B.d_off[l] = (int)units.size();
        for (int i = 0; i < n_inst; ++i)
            if (H[i]->n_levels - 1 == l) tiles(i, l, H[i]->lv[l].N, kMbDenseRows);
        B.d_n[l] = (int)units.size() - B.d_off[l];
        B.c_off[l] = (int)units.size();
        for (int i = 0; i < n_inst; ++i)
            if (H[i]->n_levels - 1 > l) tiles(i, l, H[i]->lv[l + 1].N, kMbTileRows);
        B.c_n[l] = (int)units.size() - B.c_off[l];
    }
    Carver c(tables);
    MbLevel* ddesc = c.take<MbLevel>(desc.size());
    MbUnit* dunits = c.take<MbUnit>(units.size());
    if (c.off > table_bytes) return RBFFD_ERR_WORKSPACE;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(ddesc, desc.data(), desc.size() * sizeof(MbLevel), cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaMemcpyAsync(dunits, units.data(), units.size() * sizeof(MbUnit), cudaMemcpyHostToDevice, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));  // the host tables go out of scope
    B.desc = ddesc;
    B.units = dunits;
    *out = B;
    return RBFFD_OK;
}

int mg_batch_apply_df(const MgBatch& B, int R, const float2* b, float2* x, const int* live, cudaStream_t st,
                      int* launches) {
    if (!B.desc || !B.units || !b || !x || R < 1 || R > 64) return RBFFD_ERR_INVALID_ARG;
    int n = 0;
    const MbLevel* D = B.desc;
    const int pre_dir = (B.nu - 1) & 1;  // the vector holding the iterate after the pre-sweeps
    for (int l = 0; l < B.levels; ++l) {
        const bool top = l == 0;
        if (B.d_n[l]) {
            const MbUnit* u = B.units + B.d_off[l];
            if (top)
                mb_dense_kernel<true, float2, float2><<<mb_grid(B.d_n[l]), kMbT, 0, st>>>(u, B.d_n[l], D, R, b, x, live);
            else
                mb_dense_kernel<false, float2, float2><<<mb_grid(B.d_n[l]), kMbT, 0, st>>>(u, B.d_n[l], D, R, b, x,
                                                                                          live);
            ++n;
        }
        if (!B.a_n[l]) continue;
        const MbUnit* u = B.units + B.a_off[l];
        const int g = mb_grid(B.a_n[l]);
        if (top) mb_first_kernel<true, float2><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, b, live);
        else mb_first_kernel<false, float2><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, b, live);
        ++n;
        for (int k = 1; k < B.nu; ++k) {
            const int dir = (k - 1) & 1;
            if (top) mb_sweep_kernel<true, float2, float2, 0><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, dir, b, x, live);
            else mb_sweep_kernel<false, float2, float2, 0><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, dir, b, x, live);
            ++n;
        }
        if (top) mb_sweep_kernel<true, float2, float2, 1><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, pre_dir, b, x, live);
        else mb_sweep_kernel<false, float2, float2, 1><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, pre_dir, b, x, live);
        mb_restrict_kernel<<<mb_grid(B.c_n[l]), kMbT, 0, st>>>(B.units + B.c_off[l], B.c_n[l], D, R, live);
        n += 2;
    }
    for (int l = B.levels - 2; l >= 0; --l) {
        if (!B.a_n[l]) continue;
        const bool top = l == 0;
        const MbUnit* u = B.units + B.a_off[l];
        const int g = mb_grid(B.a_n[l]);
        mb_prolong_kernel<<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, pre_dir, live);
        ++n;
        for (int k = 0; k < B.nu; ++k) {
            const int dir = (pre_dir + k) & 1;
            if (top && k == B.nu - 1)
                mb_sweep_kernel<true, float2, float2, 2><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, dir, b, x, live);
            else if (top)
                mb_sweep_kernel<true, float2, float2, 0><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, dir, b, x, live);
            else
                mb_sweep_kernel<false, float2, float2, 0><<<g, kMbT, 0, st>>>(u, B.a_n[l], D, R, dir, b, x, live);
            ++n;
        }
    }
    if (launches) *launches += n;
    note_launches(n);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

}  // namespace rbffd
