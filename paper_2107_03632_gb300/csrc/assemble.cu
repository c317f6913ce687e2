// Assembly of the discrete Poisson operator (CSR, Dirichlet rows), the
// right-hand side, and the CSR transpose used by the adjoint solve.
//
// Sec. IV, Eqs. 2-4 at steady state: interior rows hold the RBF-FD Laplacian
// weights of the node's stencil (A[i, idx[i,j]] = w[i,j], stencil order),
// Dirichlet rows the identity; b = -f inside, g on the boundary.
#include "common.cuh"
#include "scan.cuh"

#include <algorithm>

namespace rbffd {
namespace {

struct RowLenLoad {
    const uint8_t* mask;
    int64_t n;
    __device__ int64_t operator()(int64_t i) const { return mask[i] ? (int64_t)1 : n; }
};

// One warp per row: copy the stencil and its weights into the row's range.
__global__ void __launch_bounds__(256) assemble_fill_kernel(const int* __restrict__ idx, const double* __restrict__ w,
                                                            const uint8_t* __restrict__ mask, int64_t N, int n,
                                                            const int64_t* __restrict__ row_ptr, int64_t nnz,
                                                            int* __restrict__ col, double* __restrict__ val,
                                                            float* __restrict__ val32) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < N; i += nwarps) {
        const int64_t a = row_ptr[i];
        const bool dir = mask[i] != 0;
        const int len = dir ? 1 : n;
        if (a < 0 || a + len > nnz) continue;  // inconsistent row_ptr: never write past nnz
        if (dir) {
            if (lane == 0) {
                col[a] = (int)i;
                val[a] = 1.0;
                if (val32) val32[a] = 1.0f;
            }
        } else {
            const int* si = idx + i * n;
            const double* wi = w + i * n;
            for (int j = lane; j < n; j += 32) {
                const double v = wi[j];
                col[a + j] = si[j];
                val[a + j] = v;
                if (val32) val32[a + j] = __double2float_rn(v);
            }
        }
    }
}

__global__ void rhs_kernel(const double* __restrict__ f, const double* __restrict__ g,
                           const uint8_t* __restrict__ mask, int64_t N, double* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = mask[i] ? g[i] : -f[i];
}

// ---- transpose ------------------------------------------------------------
// count entries per column (warp per row, lanes over the row's entries)
__global__ void col_count_kernel(const int64_t* __restrict__ row_ptr, const int* __restrict__ col, int64_t N,
                                 int64_t nnz, int* __restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp0; r < N; r += nwarps) {
        const int64_t a = max(row_ptr[r], (int64_t)0), e = min(row_ptr[r + 1], nnz);
        for (int64_t k = a + lane; k < e; k += 32) {
            const int c = col[k];
            if ((unsigned)c < (unsigned)N) atomicAdd(&counts[c], 1);
        }
    }
}

struct CountLoad64 {
    const int* counts;
    __device__ int64_t operator()(int64_t i) const { return (int64_t)counts[i]; }
};

// counts[c] runs down from the column length to 1: positions fill
// [row_ptr_t[c], row_ptr_t[c+1]) once each (order fixed afterwards).
__global__ void transpose_scatter_kernel(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                                         const double* __restrict__ val, int64_t N, int64_t nnz,
                                         const int64_t* __restrict__ row_ptr_t, int* __restrict__ counts,
                                         int* __restrict__ col_t, double* __restrict__ val_t) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp0; r < N; r += nwarps) {
        const int64_t a = max(row_ptr[r], (int64_t)0), e = min(row_ptr[r + 1], nnz);
        for (int64_t k = a + lane; k < e; k += 32) {
            const int c = col[k];
            if ((unsigned)c >= (unsigned)N) continue;
            const int64_t pos = row_ptr_t[c + 1] - atomicSub(&counts[c], 1);
            RB_AT(col_t, pos, nnz) = (int)r;
            RB_AT(val_t, pos, nnz) = val[k];
        }
    }
}

// Sort each row of A^T by column index: one warp per row, a bitonic network
// over the row's entries held in registers (up to 128 entries, four per
// lane); a longer row is sorted by one thread (insertion sort).  With
// val32_t, also write the row's float32 copy (rounded to nearest).  Columns
// within a row are distinct, so the order is unique.
__global__ void __launch_bounds__(256) row_sort_kernel(const int64_t* __restrict__ row_ptr_t, int64_t N,
                                                       int64_t nnz, int* __restrict__ col_t,
                                                       double* __restrict__ val_t, float* __restrict__ val32_t) {
    (void)nnz;  // bound of the checked build's tests (the transpose has at most nnz entries)
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N; r += nw) {
        const int64_t a = row_ptr_t[r], e = row_ptr_t[r + 1];
        const int len = (int)(e - a);
        RB_SPAN(a, len, nnz);
        if (len > 128) {
            if (lane == 0) {
                for (int64_t k = a + 1; k < e; ++k) {
                    const int c = col_t[k];
                    const double v = val_t[k];
                    int64_t q = k - 1;
                    while (q >= a && col_t[q] > c) {
                        col_t[q + 1] = col_t[q];
                        val_t[q + 1] = val_t[q];
                        --q;
                    }
                    col_t[q + 1] = c;
                    val_t[q + 1] = v;
                }
            }
            __syncwarp();
            if (val32_t)
                for (int64_t k = a + lane; k < e; k += 32) val32_t[k] = __double2float_rn(val_t[k]);
            continue;
        }
        // element i = lane + 32 q in register q; padding keys sort last
        int key[4];
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            key[q] = i < len ? col_t[a + i] : 0x7fffffff;
            v[q] = i < len ? val_t[a + i] : 0.0;
        }
        const int m = len <= 32 ? 32 : (len <= 64 ? 64 : 128);  // warp-uniform
        if (len > 1) {
            for (int k = 2; k <= m; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    if (j >= 32) {
                        // partner in register q ^ (j / 32) of the same lane
                        // (registers named at compile time, so they stay registers)
                        auto cx = [&](int& ka, double& va, int& kb, double& vb, int q) {
                            const bool up = ((lane + 32 * q) & k) == 0;
                            if (ka != kb && (ka > kb) == up) {
                                const int tk = ka;
                                ka = kb;
                                kb = tk;
                                const double tv = va;
                                va = vb;
                                vb = tv;
                            }
                        };
                        if (j == 32) {
                            cx(key[0], v[0], key[1], v[1], 0);
                            if (m == 128) cx(key[2], v[2], key[3], v[3], 2);
                        } else {  // j == 64, m == 128
                            cx(key[0], v[0], key[2], v[2], 0);
                            cx(key[1], v[1], key[3], v[3], 1);
                        }
                    } else {
                        // partner in lane ^ j, same register
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (32 * q < m) {
                                const int pk = __shfl_xor_sync(0xffffffffu, key[q], j);
                                const double pv = __shfl_xor_sync(0xffffffffu, v[q], j);
                                const bool up = ((lane + 32 * q) & k) == 0;
                                const bool lower = (lane & j) == 0;
                                // the lower position keeps the smaller key when ascending
                                const bool take = (lower == up) ? (pk < key[q]) : (pk > key[q]);
                                if (take) {
                                    key[q] = pk;
                                    v[q] = pv;
                                }
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            if (i < len) {
                col_t[a + i] = key[q];
                val_t[a + i] = v[q];
                if (val32_t) val32_t[a + i] = __double2float_rn(v[q]);
            }
        }
    }
}

int grid_for(int64_t work, int per_block) {
    const int64_t b = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 16));
}

}  // namespace
}  // namespace rbffd

extern "C" size_t rbffd_assemble_workspace_size(int64_t N) {
    RBFFD_NVTX("rbffd_assemble_workspace_size");
    if (N <= 0) return 0;
    rbffd::Carver c(nullptr);
    c.take<int64_t>(rbffd::scan_tiles(N) + 1);
    return c.off;
}

extern "C" int rbffd_assemble_pattern(const uint8_t* is_dirichlet, int64_t N, int32_t n, int64_t* row_ptr, void* ws,
                                      size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_assemble_pattern");
    using namespace rbffd;
    if (!is_dirichlet || !row_ptr || N <= 0 || N > 0x7fffffffLL || n < 1 || n > RBFFD_MAX_STENCIL)
        return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0 || ws_bytes < rbffd_assemble_workspace_size(N))
        return RBFFD_ERR_WORKSPACE;
    int64_t* sums = static_cast<int64_t*>(ws);
    RBFFD_CUDA_TRY(exclusive_scan<int64_t>(RowLenLoad{is_dirichlet, (int64_t)n}, N, row_ptr, sums, row_ptr + N,
                                           as_stream(stream)));
    return RBFFD_OK;
}

extern "C" int rbffd_assemble(const int32_t* idx, const double* w, const uint8_t* is_dirichlet, int64_t N, int32_t n,
                              const int64_t* row_ptr, int64_t nnz, int32_t* col, double* val, float* val32,
                              void* stream) {
    RBFFD_NVTX("rbffd_assemble");
    using namespace rbffd;
    if (!idx || !w || !is_dirichlet || !row_ptr || !col || !val || N <= 0 || N > 0x7fffffffLL || n < 1 ||
        n > RBFFD_MAX_STENCIL || nnz < 0)
        return RBFFD_ERR_INVALID_ARG;
    assemble_fill_kernel<<<grid_for(N * 32, 256), 256, 0, as_stream(stream)>>>(idx, w, is_dirichlet, N, n, row_ptr,
                                                                               nnz, col, val, val32);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

extern "C" int rbffd_rhs(const double* f, const double* g, const uint8_t* is_dirichlet, int64_t N, double* b,
                         void* stream) {
    RBFFD_NVTX("rbffd_rhs");
    using namespace rbffd;
    if (!f || !g || !is_dirichlet || !b || N <= 0) return RBFFD_ERR_INVALID_ARG;
    rhs_kernel<<<grid_for(N, 256), 256, 0, as_stream(stream)>>>(f, g, is_dirichlet, N, b);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

extern "C" size_t rbffd_transpose_workspace_size(int64_t n_rows) {
    RBFFD_NVTX("rbffd_transpose_workspace_size");
    if (n_rows <= 0) return 0;
    rbffd::Carver c(nullptr);
    c.take<int>(n_rows);
    c.take<int64_t>(rbffd::scan_tiles(n_rows) + 1);
    return c.off;
}

extern "C" int rbffd_transpose(const rbffd_csr* A, int64_t* row_ptr_t, int32_t* col_t, double* val_t,
                               float* val32_t, void* ws, size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_transpose");
    using namespace rbffd;
    if (!A || !A->row_ptr || !A->col || !A->val || A->dtype != 0 || !row_ptr_t || !col_t || !val_t ||
        A->n_rows <= 0 || A->n_rows > 0x7fffffffLL || A->nnz < 0)
        return RBFFD_ERR_INVALID_ARG;
    const int64_t N = A->n_rows;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0 || ws_bytes < rbffd_transpose_workspace_size(N))
        return RBFFD_ERR_WORKSPACE;
    Carver c(ws);
    int* counts = c.take<int>(N);
    int64_t* sums = c.take<int64_t>(scan_tiles(N) + 1);
    cudaStream_t st = as_stream(stream);
    const double* val = static_cast<const double*>(A->val);
    RBFFD_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * N, st));
    col_count_kernel<<<grid_for(N * 32, 256), 256, 0, st>>>(A->row_ptr, A->col, N, A->nnz, counts);
    RBFFD_CUDA_TRY(exclusive_scan<int64_t>(CountLoad64{counts}, N, row_ptr_t, sums, row_ptr_t + N, st));
    transpose_scatter_kernel<<<grid_for(N * 32, 256), 256, 0, st>>>(A->row_ptr, A->col, val, N, A->nnz, row_ptr_t, counts,
                                                                    col_t, val_t);
    row_sort_kernel<<<grid_for(N * 32, 256), 256, 0, st>>>(row_ptr_t, N, A->nnz, col_t, val_t, val32_t);
    note_launches(3);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}
