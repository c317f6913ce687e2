// The paper's explicit time loop on the GPU (sm_103a).
//
// Sec. IV, Eq. 4: forward Euler for u_t = lap u + f,
//     u_2(x_i) = u_1(x_i) + dt ( f(x_i) + sum_j w_ij u_1(x_{idx_ij}) )
// on interior nodes; Dirichlet nodes keep their values.  Sec. V's data model
// holds, per node, the weights and support indices of its stencil and, per
// interior node, its index (the interior list); the loop itself is the
// paper's only GPU workload (1e5 steps of dt = 1e-6).
//
// Layout for this chip: the interior rows are packed once into an ELL array
// stored column-major, [j][r] for stencil entry j of interior row r, so a
// warp's 32 rows read 32 consecutive weights (and indices) per entry: every
// load is one coalesced 256-byte (128-byte) segment.  One launch per step,
// one thread per interior row, ping-pong between two u buffers (both hold
// the Dirichlet values, which no step writes); the steps are captured once
// into a CUDA graph of kGraphSteps launches and replayed, so a step costs
// its memory traffic and not a host launch.
#include "common.cuh"
#include "scan.cuh"

#include <algorithm>

namespace rbffd {
namespace {

constexpr int kT = 256;
constexpr int kGraphSteps = 64;  // even: a replay leaves the result where it started

struct ExplicitLayout {
    int32_t* rows;  // interior node ids, N_i
    int32_t* idx;   // [n][N_i] column-major
    double* w;      // [n][N_i]
    double* u2;     // second time level, N
    int* pos;       // scan of the interior flags, N + 1
    int* sums;
    int* bad;       // out-of-range stencil index seen by the packing
    size_t bytes;
};

ExplicitLayout explicit_layout(void* ws, int64_t N, int n) {
    Carver c(ws);
    ExplicitLayout L;
    L.rows = c.take<int32_t>(N);
    L.idx = c.take<int32_t>((size_t)N * n);
    L.w = c.take<double>((size_t)N * n);
    L.u2 = c.take<double>(N);
    L.pos = c.take<int>(N + 1);
    L.sums = c.take<int>(scan_tiles(N) + 1);
    L.bad = c.take<int>(1);
    L.bytes = c.off;
    return L;
}

struct InteriorLoad {
    const uint8_t* mask;
    __device__ int operator()(int64_t i) const { return mask[i] ? 0 : 1; }
};

__global__ void __launch_bounds__(kT) explicit_pack_kernel(const int32_t* __restrict__ idx,
                                                           const double* __restrict__ w,
                                                           const uint8_t* __restrict__ mask, int64_t N, int n,
                                                           const int* __restrict__ pos, int64_t Ni,
                                                           int32_t* __restrict__ rows, int32_t* __restrict__ idxT,
                                                           double* __restrict__ wT, int* __restrict__ bad) {
    int nb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        if (mask[i]) continue;
        const int64_t r = pos[i];
        RB_AT(rows, r, Ni) = (int32_t)i;
        for (int j = 0; j < n; ++j) {
            int32_t c = idx[i * n + j];
            if ((uint32_t)c >= (uint32_t)N) {  // never let the loop read outside u
                nb = 1;
                c = (int32_t)i;
            }
            RB_AT(idxT, (int64_t)j * Ni + r, (int64_t)n * Ni) = c;
            RB_AT(wT, (int64_t)j * Ni + r, (int64_t)n * Ni) = w[i * n + j];
        }
    }
    if (nb) atomicOr(bad, 1);
}

// One forward-Euler step on the interior rows.
__global__ void __launch_bounds__(kT) explicit_step_kernel(const int32_t* __restrict__ rows,
                                                           const int32_t* __restrict__ idxT,
                                                           const double* __restrict__ wT, int64_t Ni, int n,
                                                           const double* __restrict__ f, double dt,
                                                           const double* __restrict__ u1, double* __restrict__ u2,
                                                           int64_t N) {
    (void)N;  // nodes: bound of the checked build's tests
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Ni; r += (int64_t)gridDim.x * blockDim.x) {
        double lap = 0.0;
        for (int j = 0; j < n; ++j)
            lap = fma(__ldg(wT + (int64_t)j * Ni + r), __ldg(&RB_AT(u1, __ldg(idxT + (int64_t)j * Ni + r), N)), lap);
        const int i = __ldg(rows + r);
        RB_AT(u2, i, N) = fma(dt, __ldg(&RB_AT(f, i, N)) + lap, RB_AT(u1, i, N));
    }
}

int step_blocks(int64_t Ni) {
    const int64_t b = (Ni + kT - 1) / kT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 32));
}

}  // namespace
}  // namespace rbffd

extern "C" size_t rbffd_explicit_workspace_size(int64_t N, int32_t n) {
    RBFFD_NVTX("rbffd_explicit_workspace_size");
    if (N <= 0 || N > 0x7fffffffLL || n < 1 || n > RBFFD_MAX_STENCIL) return 0;
    return rbffd::explicit_layout(nullptr, N, n).bytes;
}

extern "C" int rbffd_explicit_pack(const int32_t* idx, const double* w, const uint8_t* is_dirichlet, int64_t N,
                                   int32_t n, int64_t* n_interior, void* ws, size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_explicit_pack");
    using namespace rbffd;
    if (!idx || !w || !is_dirichlet || !n_interior || N <= 0 || N > 0x7fffffffLL || n < 1 ||
        n > RBFFD_MAX_STENCIL)
        return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0) return RBFFD_ERR_WORKSPACE;
    ExplicitLayout L = explicit_layout(ws, N, n);
    if (ws_bytes < L.bytes) return RBFFD_ERR_WORKSPACE;
    cudaStream_t st = as_stream(stream);
    RBFFD_CUDA_TRY(cudaMemsetAsync(L.bad, 0, sizeof(int), st));
    RBFFD_CUDA_TRY(exclusive_scan<int>(InteriorLoad{is_dirichlet}, N, L.pos, L.sums, L.pos + N, st));
    int ni = 0;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(&ni, L.pos + N, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (ni > 0) {
        explicit_pack_kernel<<<step_blocks(N), kT, 0, st>>>(idx, w, is_dirichlet, N, n, L.pos, ni, L.rows, L.idx, L.w,
                                                            L.bad);
        note_launches(1);
        RBFFD_LAUNCH_CHECK();
    }
    int bad = 0;
    RBFFD_CUDA_TRY(cudaMemcpyAsync(&bad, L.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBFFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) return RBFFD_ERR_INVALID_ARG;
    *n_interior = ni;
    return RBFFD_OK;
}

extern "C" int rbffd_explicit_run(const double* f, double* u, int64_t N, int32_t n, int64_t n_interior, double dt,
                                  int64_t steps, void* ws, size_t ws_bytes, void* stream) {
    RBFFD_NVTX("rbffd_explicit_run");
    using namespace rbffd;
    if (!f || !u || N <= 0 || N > 0x7fffffffLL || n < 1 || n > RBFFD_MAX_STENCIL || n_interior < 0 ||
        n_interior > N || steps < 0 || !(dt == dt))
        return RBFFD_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0) return RBFFD_ERR_WORKSPACE;
    ExplicitLayout L = explicit_layout(ws, N, n);
    if (ws_bytes < L.bytes) return RBFFD_ERR_WORKSPACE;
    if (steps == 0 || n_interior == 0) return RBFFD_OK;
    cudaStream_t st = as_stream(stream);
    const int64_t Ni = n_interior;
    const int g = step_blocks(Ni);
    // both levels hold the Dirichlet values
    RBFFD_CUDA_TRY(cudaMemcpyAsync(L.u2, u, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    double* a = u;
    double* b = L.u2;
    int64_t done = 0;
    if (steps >= 2 * kGraphSteps) {
        cudaStream_t cap;
        RBFFD_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < kGraphSteps; ++k) {
                explicit_step_kernel<<<g, kT, 0, cap>>>(L.rows, L.idx, L.w, Ni, n, f, dt, (k & 1) ? b : a,
                                                        (k & 1) ? a : b, N);
            }
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            set_cuda_error(e);
            return RBFFD_ERR_CUDA;
        }
        const int64_t reps = steps / kGraphSteps;
        for (int64_t k = 0; k < reps && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, st);
        note_launches((int)std::min<int64_t>(reps * kGraphSteps, 0x7fffffff));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            set_cuda_error(e);
            return RBFFD_ERR_CUDA;
        }
        done = reps * kGraphSteps;  // even: the current level is back in a
    }
    for (int64_t k = done; k < steps; ++k) {
        explicit_step_kernel<<<g, kT, 0, st>>>(L.rows, L.idx, L.w, Ni, n, f, dt, a, b, N);
        std::swap(a, b);
        note_launches(1);
    }
    RBFFD_LAUNCH_CHECK();
    if (a != u) RBFFD_CUDA_TRY(cudaMemcpyAsync(u, a, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    return RBFFD_OK;
}
