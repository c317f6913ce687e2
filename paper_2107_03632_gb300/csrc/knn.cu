// Exact n-nearest-neighbour stencils on a uniform cell grid (sm_103a).
//
// Sec. II, Eq. 1: the operator at node x is approximated from the values on
// N(x), the nodes neighbouring x; Sec. V takes the n nearest nodes.  Order of
// a stencil: key (d^2, j) ascending, where d^2 = dx*dx + dy*dy is rounded
// product by product (no FMA: __dmul_rn / __dadd_rn) and j is the caller's
// node index; node x itself comes first (d^2 = 0).
//
// Pipeline (all on the stream, no host synchronisation):
//   1. bounding box (block partials, then one block)         -> GridParams
//   2. cell key per node, histogram of keys (atomics)
//   3. exclusive scan of the histogram                       -> cell_start
//   4. scatter nodes into cell order (SoA double2 + original index)
//   5. one warp per query, in cell order: scan cells ring by ring around the
//      query's cell, keep a sorted top-n list of keys distributed over the
//      warp's registers (entry e at lane e%32, slot e/32), prune cells whose
//      nearest point cannot beat the current n-th key, and stop once the
//      unvisited region is provably farther than the n-th key.
// Distances are compared as the IEEE bit patterns of non-negative doubles
// (monotone as unsigned integers), so ranking never touches the FP64 pipe.
#include "common.cuh"
#include "internal.cuh"
#include "scan.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <map>
#include <mutex>

namespace rbffd {
namespace {

struct GridParams {
    double x0, y0;      // lower-left corner of the grid
    double cell;        // cell side
    double inv_cell;    // 1 / cell
    double margin;      // absolute slack for the geometric pruning tests
    int G;              // cells per axis (G x G cells)
    int pad;
};

struct Box {
    double mnx, mny, mxx, mxy;
};

constexpr int kBoxBlocks = 256;
constexpr int kBoxThreads = 256;

__global__ void __launch_bounds__(kBoxThreads) bbox_partial_kernel(const double2* __restrict__ xy, int64_t N,
                                                                   Box* __restrict__ part) {
    double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
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
    __shared__ Box sh[kBoxThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) RB_AT(sh, wid, kBoxThreads / 32) = Box{mnx, mny, mxx, mxy};
    __syncthreads();
    if (threadIdx.x == 0) {
        Box r = sh[0];
        for (int k = 1; k < kBoxThreads / 32; ++k) {
            r.mnx = fmin(r.mnx, sh[k].mnx);
            r.mny = fmin(r.mny, sh[k].mny);
            r.mxx = fmax(r.mxx, sh[k].mxx);
            r.mxy = fmax(r.mxy, sh[k].mxy);
        }
        part[blockIdx.x] = r;
    }
}

__global__ void grid_setup_kernel(const Box* __restrict__ part, int nparts, int G, GridParams* gp) {
    if (threadIdx.x != 0) return;
    Box r = part[0];
    for (int k = 1; k < nparts; ++k) {
        r.mnx = fmin(r.mnx, part[k].mnx);
        r.mny = fmin(r.mny, part[k].mny);
        r.mxx = fmax(r.mxx, part[k].mxx);
        r.mxy = fmax(r.mxy, part[k].mxy);
    }
    double x0 = r.mnx, y0 = r.mny;
    double span = fmax(r.mxx - r.mnx, r.mxy - r.mny);
    if (!(x0 > -INFINITY && x0 < INFINITY)) x0 = 0.0;  // no finite point
    if (!(y0 > -INFINITY && y0 < INFINITY)) y0 = 0.0;
    if (!(span > 0.0 && span < INFINITY)) span = 1.0;    // single point / degenerate
    GridParams p;
    p.x0 = x0;
    p.y0 = y0;
    p.cell = span / G;
    p.inv_cell = G / span;
    p.margin = 1e-12 * (span + fabs(x0) + fabs(y0));
    p.G = G;
    p.pad = 0;
    *gp = p;
}

__device__ __forceinline__ int cell_coord(double v, double v0, double inv, int G) {
    const double t = floor((v - v0) * inv);
    // NaN and out-of-range values are clamped (NaN compares false).
    int c = (t >= 0.0) ? ((t < (double)G) ? (int)t : G - 1) : 0;
    return c;
}

__global__ void cell_count_kernel(const double2* __restrict__ xy, int64_t N, const GridParams* __restrict__ gp,
                                  int* __restrict__ keys, int* __restrict__ counts) {
    const GridParams p = *gp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 q = xy[i];
        const int cx = cell_coord(q.x, p.x0, p.inv_cell, p.G);
        const int cy = cell_coord(q.y, p.y0, p.inv_cell, p.G);
        const int key = cy * p.G + cx;
        keys[i] = key;
        atomicAdd(&RB_AT(counts, key, p.G * p.G), 1);
    }
}

// counts[key] runs from the cell size down to 1, so positions fill
// [start[key], start[key+1]) exactly once.  Order inside a cell is arbitrary;
// stencils do not depend on it because the ranking key is a total order.
__global__ void cell_scatter_kernel(const double2* __restrict__ xy, int64_t N, const int* __restrict__ keys,
                                    const int* __restrict__ cell_start, int* __restrict__ counts, int64_t cells,
                                    double2* __restrict__ sxy, int* __restrict__ sorig) {
    (void)cells;  // bound of the checked build's tests
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int key = keys[i];
        const int pos = RB_AT(cell_start, key + 1, cells + 1) - atomicSub(&RB_AT(counts, key, cells), 1);
        RB_AT(sxy, pos, N) = xy[i];
        RB_AT(sorig, pos, N) = (int)i;
    }
}

struct Key {
    unsigned long long d;  // bit pattern of d^2 (non-negative double)
    unsigned int j;        // caller index
};

__device__ __forceinline__ bool key_less(unsigned long long ad, unsigned int aj, unsigned long long bd,
                                         unsigned int bj) {
    return (ad < bd) || (ad == bd && aj < bj);
}

__device__ __forceinline__ double key_d2(unsigned long long d) { return __longlong_as_double((long long)d); }

// Distributed sorted list of SLOTS*32 keys (entry e: lane e & 31, slot e >> 5).
template <int SLOTS>
struct TopList {
    unsigned long long d[SLOTS];
    unsigned int j[SLOTS];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            d[s] = ~0ull;
            j[s] = ~0u;
        }
    }

    // Insert key (kd, kj), which is known to be smaller than entry n-1.
    __device__ __forceinline__ void insert(unsigned long long kd, unsigned int kj, int lane) {
        int p = 0;
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) p += __popc(__ballot_sync(0xffffffffu, key_less(d[s], j[s], kd, kj)));
        unsigned long long up_d[SLOTS];
        unsigned int up_j[SLOTS];
        unsigned long long top_d[SLOTS];
        unsigned int top_j[SLOTS];
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            up_d[s] = __shfl_up_sync(0xffffffffu, d[s], 1);
            up_j[s] = __shfl_up_sync(0xffffffffu, j[s], 1);
            top_d[s] = __shfl_sync(0xffffffffu, d[s], 31);
            top_j[s] = __shfl_sync(0xffffffffu, j[s], 31);
        }
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            const int e = s * 32 + lane;
            unsigned long long pd;
            unsigned int pj;
            if (lane > 0) {
                pd = up_d[s];
                pj = up_j[s];
            } else if (s > 0) {
                pd = top_d[s > 0 ? s - 1 : 0];
                pj = top_j[s > 0 ? s - 1 : 0];
            } else {
                pd = ~0ull;
                pj = ~0u;
            }
            if (e == p) {
                d[s] = kd;
                j[s] = kj;
            } else if (e > p) {
                d[s] = pd;
                j[s] = pj;
            }
        }
    }

    // Merge a batch of 32 keys (one per lane, sorted ascending over the
    // lanes): afterwards the list holds the SLOTS*32 smallest of the list
    // and the batch, sorted.  Classic bitonic merge: the last slot against
    // the reversed batch keeps the smaller key of each pair, which leaves the
    // list a bitonic sequence of the smallest keys; compare-exchange stages of
    // halving distance then sort it (between slots in registers, within a
    // slot by shuffles).
    __device__ __forceinline__ void merge(unsigned long long bd, unsigned int bj, int lane) {
        const unsigned long long rd = __shfl_sync(0xffffffffu, bd, 31 - lane);
        const unsigned int rj = __shfl_sync(0xffffffffu, bj, 31 - lane);
        if (key_less(rd, rj, d[SLOTS - 1], j[SLOTS - 1])) {
            d[SLOTS - 1] = rd;
            j[SLOTS - 1] = rj;
        }
#pragma unroll
        for (int h = SLOTS / 2; h > 0; h >>= 1)  // distance 32 h: slot s against slot s + h
#pragma unroll
            for (int s = 0; s < SLOTS; ++s)
                if ((s & h) == 0 && key_less(d[s + h], j[s + h], d[s], j[s])) {
                    const unsigned long long td = d[s];
                    const unsigned int tj = j[s];
                    d[s] = d[s + h];
                    j[s] = j[s + h];
                    d[s + h] = td;
                    j[s + h] = tj;
                }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const bool lower = (lane & o) == 0;
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                const unsigned long long pd = __shfl_xor_sync(0xffffffffu, d[s], o);
                const unsigned int pj = __shfl_xor_sync(0xffffffffu, j[s], o);
                if (lower ? key_less(pd, pj, d[s], j[s]) : key_less(d[s], j[s], pd, pj)) {
                    d[s] = pd;
                    j[s] = pj;
                }
            }
        }
    }

    // Entry e broadcast to the warp.
    __device__ __forceinline__ void get(int e, unsigned long long& od, unsigned int& oj) const {
        const int s = e >> 5, l = e & 31;
        unsigned long long v = d[0];
        unsigned int w = j[0];
#pragma unroll
        for (int t = 1; t < SLOTS; ++t)
            if (t == s) {
                v = d[t];
                w = j[t];
            }
        od = __shfl_sync(0xffffffffu, v, l);
        oj = __shfl_sync(0xffffffffu, w, l);
    }
};

// Ascending bitonic sort of 32 keys, one per lane.
__device__ __forceinline__ void warp_sort32(unsigned long long& d, unsigned int& j, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int o = k >> 1; o > 0; o >>= 1) {
            const unsigned long long pd = __shfl_xor_sync(0xffffffffu, d, o);
            const unsigned int pj = __shfl_xor_sync(0xffffffffu, j, o);
            const bool up = (lane & k) == 0 || k == 32;  // this run ascending
            const bool lower = (lane & o) == 0;
            if (lower == up ? key_less(pd, pj, d, j) : key_less(d, j, pd, pj)) {
                d = pd;
                j = pj;
            }
        }
    }
}

// Batches with more accepted candidates than this are sorted and merged into
// the list at once; fewer are inserted one by one (4M nodes, n = 56: 24.9 /
// 24.4 / 24.0 / 23.6 / 23.1 ms of stencils with 1 / 2 / 4 / 8 / 16 here,
// 34.3 ms inserting every candidate).
constexpr int kMergeBatch = 16;

// Queries: the indexed points themselves in cell order (qxy = sxy, qorig =
// sorig: stencils), or separate points in their own order (qorig = NULL:
// output row q).
//
// Search order: first the (2 R0 + 1)^2 block of cells around the query's
// cell, R0 chosen on the host so that the block holds about n points, row
// by row from the query's row outwards -- the points of a row of cells are
// contiguous in the cell-sorted arrays, so a warp reads 32 candidates at a
// time instead of one cell's few; then rings of cells until the gap to the
// unvisited cells exceeds the n-th key.  The candidate keys (d^2, index) are
// FP64 and exact; the pruning bounds for groups of cells are FP32, taken
// relative to the query and shrunk by a slack, so they only ever keep a cell
// that an exact bound would have skipped.  (On this chip the FP64 units issue
// 2 lanes per clock per SM: per-cell FP64 bounds and one-cell candidate
// batches made the search FP64-bound.)
template <int SLOTS>
__global__ void __launch_bounds__(256) knn_kernel(const double2* __restrict__ sxy, const int* __restrict__ sorig,
                                                  const int* __restrict__ cell_start, int Np,
                                                  const GridParams* __restrict__ gp, int Nq,
                                                  const double2* __restrict__ qxy, const int* __restrict__ qorig,
                                                  int n, int R0, int* __restrict__ idx) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= Nq) return;
    const GridParams p = *gp;
    const double2 Q = qxy[q];
    const int qo = qorig ? qorig[q] : q;
    const int G = p.G;
    (void)Np;  // bound of the checked build's tests
    const int cx = cell_coord(Q.x, p.x0, p.inv_cell, G);
    const int cy = cell_coord(Q.y, p.y0, p.inv_cell, G);

    TopList<SLOTS> top;
    top.init();
    unsigned long long thr_d = ~0ull;  // key of entry n-1 (all-ones: list not full)
    unsigned int thr_j = ~0u;

    // one batch: lane's candidate at sorted position jj (none: jj < 0)
    auto eval = [&](int jj) {
        unsigned long long kd = ~0ull;
        unsigned int kj = ~0u;
        if (jj >= 0) {
            const double2 P = RB_AT(sxy, jj, Np);
            const double dx = __dadd_rn(P.x, -Q.x);
            const double dy = __dadd_rn(P.y, -Q.y);
            const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            kd = (unsigned long long)__double_as_longlong(d2) & 0x7fffffffffffffffull;
            kj = (unsigned int)RB_AT(sorig, jj, Np);
        }
        const bool acc = key_less(kd, kj, thr_d, thr_j);
        unsigned int m = __ballot_sync(0xffffffffu, acc);
        if (__popc(m) > kMergeBatch) {  // many at once (the first batches of a query)
            unsigned long long md = acc ? kd : ~0ull;
            unsigned int mj = acc ? kj : ~0u;
            warp_sort32(md, mj, lane);
            top.merge(md, mj, lane);
            top.get(n - 1, thr_d, thr_j);
            return;
        }
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const unsigned long long id = __shfl_sync(0xffffffffu, kd, src);
            const unsigned int ij = __shfl_sync(0xffffffffu, kj, src);
            if (!key_less(id, ij, thr_d, thr_j)) continue;  // threshold moved
            top.insert(id, ij, lane);
            top.get(n - 1, thr_d, thr_j);
        }
    };
    // candidates at sorted positions [beg, end)
    auto scan = [&](int beg, int end) {
        for (int base = beg; base < end; base += 32) eval(base + lane < end ? base + lane : -1);
    };
    // FP32 lower bound of d^2 from the query to the cells [xl, xh] of row yy,
    // relative to the query's cell corner (exact in FP64), shrunk by a slack;
    // true when all of them lie beyond the n-th key
    const float fx = (float)(Q.x - (p.x0 + cx * p.cell));
    const float fy = (float)(Q.y - (p.y0 + cy * p.cell));
    const float cf = (float)p.cell;
    const float slack = (float)p.margin + 1e-4f * cf;
    auto beyond = [&](int xl, int xh, int yy) -> bool {
        if (thr_d == ~0ull) return false;
        const float lx = (float)(xl - cx) * cf - fx, hx = (float)(xh + 1 - cx) * cf - fx;
        const float ly = (float)(yy - cy) * cf - fy, hy = ly + cf;
        const float dx = fmaxf(fmaxf(fmaxf(lx, -hx), 0.f) - slack, 0.f);
        const float dy = fmaxf(fmaxf(fmaxf(ly, -hy), 0.f) - slack, 0.f);
        return (dx * dx + dy * dy) * (1.0f - 1e-4f) > (float)key_d2(thr_d);
    };
    auto row_range = [&](int xl, int xh, int yy) {
        if (!beyond(xl, xh, yy))
            scan(RB_AT(cell_start, yy * G + xl, G * G + 1), RB_AT(cell_start, yy * G + xh + 1, G * G + 1));
    };
    // true when the cells within ring r hold the n nearest: whole grid
    // visited, or the gap from Q to the unvisited cells exceeds the n-th key
    auto done = [&](int r) -> bool {
        if (cx - r <= 0 && cy - r <= 0 && cx + r >= G - 1 && cy + r >= G - 1) return true;
        if (thr_d == ~0ull) return false;
        double gap = INFINITY;
        if (cx - r > 0) gap = fmin(gap, Q.x - (p.x0 + (cx - r) * p.cell));
        if (cx + r < G - 1) gap = fmin(gap, (p.x0 + (cx + r + 1) * p.cell) - Q.x);
        if (cy - r > 0) gap = fmin(gap, Q.y - (p.y0 + (cy - r) * p.cell));
        if (cy + r < G - 1) gap = fmin(gap, (p.y0 + (cy + r + 1) * p.cell) - Q.y);
        gap -= p.margin;
        return gap > 0.0 && gap * gap > key_d2(thr_d);
    };

    // the block, rows from the query's outwards, their candidates packed into
    // batches of 32 across row boundaries (a row is tested against the n-th
    // key when the batch that would start it is filled)
    {
        const int xlo = max(cx - R0, 0), xhi = min(cx + R0, G - 1);
        int k = 0, sb = 0, sl = 0;  // next row; the current row's unread range [sb, sb + sl)
        for (;;) {
            int mine = -1, fill = 0;
            while (fill < 32) {
                if (sl == 0) {
                    bool got = false;
                    while (k <= 2 * R0 && !got) {
                        const int yy = cy + ((k & 1) ? -((k + 1) >> 1) : (k >> 1));
                        ++k;
                        if (yy < 0 || yy >= G || beyond(xlo, xhi, yy)) continue;
                        sb = RB_AT(cell_start, yy * G + xlo, G * G + 1);
                        sl = RB_AT(cell_start, yy * G + xhi + 1, G * G + 1) - sb;
                        got = sl > 0;
                    }
                    if (!got) break;
                }
                const int t = min(32 - fill, sl);
                if (lane >= fill && lane < fill + t) mine = sb + lane - fill;
                sb += t;
                sl -= t;
                fill += t;
            }
            if (fill == 0) break;
            eval(mine);
        }
    }
    // then rings: the two edge rows as ranges, the side cells one by one
    for (int r = R0; !done(r) && r <= G; ) {
        ++r;
        for (int yy = cy - r; yy <= cy + r; ++yy) {
            if (yy < 0 || yy >= G) continue;
            if (yy == cy - r || yy == cy + r) {
                row_range(max(cx - r, 0), min(cx + r, G - 1), yy);
            } else {
                if (cx - r >= 0) row_range(cx - r, cx - r, yy);
                if (cx + r < G) row_range(cx + r, cx + r, yy);
            }
        }
    }

    RB_SPAN((int64_t)qo * n, n, (int64_t)Nq * n);
    int* out = idx + (int64_t)qo * n;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const int e = s * 32 + lane;
        if (e < n) out[e] = (int)top.j[s];
    }
}

// Block radius of the first search phase: about n points in (2 R0 + 1)^2
// cells at ~3 points per cell, plus half a cell.
int block_radius(int n) { return std::max(1, (int)std::ceil(std::sqrt((double)n / (3.0 * 3.14159265358979)) + 0.5)); }

// Cells per axis: about kOcc nodes per cell on a square domain, capped.
int grid_side(int64_t N, int n) {
    (void)n;
    const double occ = 3.0;
    int G = (int)std::ceil(std::sqrt((double)N / occ));
    if (G < 1) G = 1;
    if (G > 4096) G = 4096;
    return G;
}

struct KnnLayout {
    GridParams* gp;
    Box* part;
    int* keys;
    int* counts;
    int* cell_start;
    int* sums;
    double2* sxy;
    int* sorig;
    size_t bytes;
};

KnnLayout knn_layout(void* ws, int64_t N, int n) {
    const int G = grid_side(N, n);
    const int64_t cells = (int64_t)G * G;
    Carver c(ws);
    KnnLayout L;
    L.gp = c.take<GridParams>(1);
    L.part = c.take<Box>(kBoxBlocks);
    L.keys = c.take<int>(N);
    L.counts = c.take<int>(cells);
    L.cell_start = c.take<int>(cells + 1);
    L.sums = c.take<int>(scan_tiles(cells) + 1);
    L.sxy = c.take<double2>(N);
    L.sorig = c.take<int>(N);
    L.bytes = c.off;
    return L;
}

struct CountLoad {
    const int* counts;
    __device__ int operator()(int64_t i) const { return counts[i]; }
};

}  // namespace
}  // namespace rbffd

extern "C" size_t rbffd_stencils_workspace_size(int64_t N, int32_t n) {
    RBFFD_NVTX("rbffd_stencils_workspace_size");
    if (N <= 0 || n <= 0) return 0;
    return rbffd::knn_layout(nullptr, N, n).bytes;
}

extern "C" int rbffd_stencils(const double* xy, int64_t N, int32_t n, int32_t* idx, void* ws, size_t ws_bytes,
                              void* stream) {
    RBFFD_NVTX("rbffd_stencils");
    using namespace rbffd;
    if (!xy || !idx || N <= 0 || N > 0x7fffffffLL || n < 1 || n > RBFFD_MAX_STENCIL || (int64_t)n > N)
        return RBFFD_ERR_INVALID_ARG;
    if (((uintptr_t)xy & 15) != 0) return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0) return RBFFD_ERR_WORKSPACE;
    return knn_search(xy, N, nullptr, N, n, idx, ws, ws_bytes, as_stream(stream));
}

int rbffd::knn_search(const double* xy, int64_t N, const double* qxy, int64_t Nq, int32_t n, int32_t* idx, void* ws,
                      size_t ws_bytes, cudaStream_t st) {
    KnnLayout L = knn_layout(ws, N, n);
    if (ws_bytes < L.bytes) return RBFFD_ERR_WORKSPACE;
    if (Nq <= 0 || Nq > 0x7fffffffLL) return RBFFD_ERR_INVALID_ARG;
    const int G = grid_side(N, n);
    const int64_t cells = (int64_t)G * G;
    const double2* p = reinterpret_cast<const double2*>(xy);
    const int grid_pts = (int)std::min<int64_t>((N + 255) / 256, (int64_t)sm_count() * 8);

    bbox_partial_kernel<<<kBoxBlocks, kBoxThreads, 0, st>>>(p, N, L.part);
    grid_setup_kernel<<<1, 32, 0, st>>>(L.part, kBoxBlocks, G, L.gp);
    RBFFD_CUDA_TRY(cudaMemsetAsync(L.counts, 0, sizeof(int) * cells, st));
    cell_count_kernel<<<grid_pts, 256, 0, st>>>(p, N, L.gp, L.keys, L.counts);
    RBFFD_CUDA_TRY(exclusive_scan<int>(CountLoad{L.counts}, cells, L.cell_start, L.sums, L.cell_start + cells, st));
    cell_scatter_kernel<<<grid_pts, 256, 0, st>>>(p, N, L.keys, L.cell_start, L.counts, cells, L.sxy, L.sorig);
    const int warps_per_block = 8;
    const int blocks = (int)((Nq + warps_per_block - 1) / warps_per_block);
    const double2* q = qxy ? reinterpret_cast<const double2*>(qxy) : L.sxy;
    const int* qo = qxy ? nullptr : L.sorig;
    const int R0 = block_radius(n);
    if (n <= 32)
        knn_kernel<1><<<blocks, 256, 0, st>>>(L.sxy, L.sorig, L.cell_start, (int)N, L.gp, (int)Nq, q, qo, n, R0, idx);
    else if (n <= 64)
        knn_kernel<2><<<blocks, 256, 0, st>>>(L.sxy, L.sorig, L.cell_start, (int)N, L.gp, (int)Nq, q, qo, n, R0, idx);
    else
        knn_kernel<4><<<blocks, 256, 0, st>>>(L.sxy, L.sorig, L.cell_start, (int)N, L.gp, (int)Nq, q, qo, n, R0, idx);
    note_launches(5);  // bbox, setup, count, scatter, knn (+3 in the scan)
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

// ---------------------------------------------------------------------------
// Stencils without any device allocation, for callers that cannot call
// cudaMalloc (or any allocating routine) on the path -- for example code
// running inside a CUDA stream capture, a custom memory arena that owns all
// device memory, or a real-time loop that must not allocate -- and cannot
// provide a workspace either.  The scratch of rbffd_stencils lives in one
// file-scope device array sized for RBFFD_STENCILS_NOALLOC_MAX_NODES nodes;
// every GPU that loads this library keeps that array until the process
// exits.  In host code the array's name is only a host-side stand-in, so
// its device address is looked up with cudaGetSymbolAddress, with the
// device current, on the first call in each CUDA context; the address is
// cached under the context's unique ID (cuCtxGetId, reached through the
// runtime's driver entry points), so a context rebuilt after
// cudaDeviceReset gets a fresh lookup instead of a stale address.
static __device__ __align__(256) unsigned char g_stencils_noalloc_scratch[RBFFD_STENCILS_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
std::map<unsigned long long, void*> g_noalloc_ptr;  // context ID -> device address of the array
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

// Unique ID of the calling thread's current context; makes device `dev`'s
// primary context current first if the thread has none.
int current_context_id(int dev, unsigned long long* id) {
    if (!g_ctx_current || !g_ctx_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return RBFFD_ERR_CUDA;
        g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
        g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return RBFFD_ERR_CUDA;
    if (!ctx) {
        if (cudaSetDevice(dev) != cudaSuccess || g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return RBFFD_ERR_CUDA;
    }
    if (g_ctx_id(ctx, id) != CUDA_SUCCESS) return RBFFD_ERR_CUDA;
    return RBFFD_OK;
}
}  // namespace

extern "C" int rbffd_stencils_noalloc(const double* xy, int64_t N, int32_t n, int32_t* idx, void* stream) {
    RBFFD_NVTX("rbffd_stencils_noalloc");
    using namespace rbffd;
    if (N > RBFFD_STENCILS_NOALLOC_MAX_NODES || N <= 0) return RBFFD_ERR_INVALID_ARG;
    const size_t need = rbffd_stencils_workspace_size(N, n);
    if (need == 0 || need > (size_t)RBFFD_STENCILS_NOALLOC_SCRATCH_BYTES) return RBFFD_ERR_INVALID_ARG;
    int dev = 0;
    RBFFD_CUDA_TRY(cudaGetDevice(&dev));
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        unsigned long long cid = 0;
        if (current_context_id(dev, &cid) != RBFFD_OK) return RBFFD_ERR_CUDA;
        auto it = g_noalloc_ptr.find(cid);
        if (it == g_noalloc_ptr.end()) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_stencils_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
                return RBFFD_ERR_CUDA;
            }
            it = g_noalloc_ptr.emplace(cid, p).first;
        }
        ptr = it->second;
    }
    // rbffd_stencils clears the cell histogram before use; everything else in
    // the scratch is overwritten, so leftovers of earlier calls do no harm
    return rbffd_stencils(xy, N, n, idx, ptr, (size_t)RBFFD_STENCILS_NOALLOC_SCRATCH_BYTES, stream);
}
