// Shared device/host helpers of the RBF-FD library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "rbffd.h"

namespace rbffd {

// Records the CUDA error text for rbffd_last_cuda_error().
void set_cuda_error(cudaError_t e);

#define RBFFD_LAUNCH_CHECK()                                   \
    do {                                                       \
        cudaError_t e_ = cudaGetLastError();                   \
        if (e_ != cudaSuccess) {                               \
            ::rbffd::set_cuda_error(e_);                       \
            return RBFFD_ERR_CUDA;                             \
        }                                                      \
    } while (0)

#define RBFFD_CUDA_TRY(call)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) {                               \
            ::rbffd::set_cuda_error(e_);                       \
            return RBFFD_ERR_CUDA;                             \
        }                                                      \
    } while (0)

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// Carves consecutive 256-byte aligned slices out of a workspace.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* p) : base(static_cast<char*>(p)) {}
    template <class T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off = align_up(off + count * sizeof(T));
        return p;
    }
};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Number of SMs of the current device (cached per device).
int sm_count();

// Launch accounting and optional kernel timing (rbffd_profile_*).
void note_launches(int count);
bool profiling();
enum ProfKind { kProfSpmv64 = 0, kProfSpmv32 = 1, kProfMg = 2, kProfBatchIter = 3, kProfKinds = 4 };
// Brackets one launch with events when profiling is on: call prof_begin
// before and prof_end after the launch (both on stream `st`).
int prof_begin(cudaStream_t st);
void prof_end(int slot, cudaStream_t st, int kind, int64_t bytes);
// Adds the device time of completed bracketed launches (call after the
// stream has been synchronised).
void prof_collect();
// After a synchronisation: accounts the first `keep` of `count` bracketed
// launches and drops the rest (launches that returned without work).
void prof_commit(const int* slots, int count, int keep);

// ---------------------------------------------------------------- device --
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Entry i of a pseudo-random shadow residual for BiCGSTAB: uniform in
// [-1, 1), exact in float32, from the SplitMix64 finaliser (Steele, Lea and
// Flood, 2014) of seed + (i + 1) * golden.  A shadow residual drawn this way
// instead of the starting residual keeps the bi-orthogonality coefficient
// (r^, r) away from zero when the starting residual is concentrated in a few
// modes, as it is in late refinement passes.
__device__ __forceinline__ float shadow_value(unsigned long long seed, long long i) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)(z >> 40) * 0x1p-23f - 1.0f;
}

// FP64 reciprocal and reciprocal square root by Newton-Raphson refinement of
// a float32 seed (Newton's method on f(y) = 1/y - a and f(y) = 1/y^2 - a:
// y <- y + y (1 - a y) and y <- y + y (1/2 - (a/2) y^2), each step doubling
// the correct bits: ~22 -> ~44 -> full double precision, within about one
// ulp of the correctly rounded result).  Two FMAs per step against the much
// longer correctly rounded division and square root; the weight solves call
// them on scalars that every lane of a warp computes.  Outside the float32
// normal range the seeds are meaningless, so there the IEEE operations run.
__device__ __forceinline__ double rcp64(double a) {
    const double m = fabs(a);
    if (!(m > 1e-30 && m < 1e30)) return __ddiv_rn(1.0, a);
    double y = (double)__frcp_rn((float)a);
    double e = fma(-a, y, 1.0);
    y = fma(y, e, y);
    e = fma(-a, y, 1.0);
    return fma(y, e, y);
}

__device__ __forceinline__ double rsqrt64(double a) {
    if (!(a > 1e-30 && a < 1e30)) return __ddiv_rn(1.0, __dsqrt_rn(a));
    double y = (double)rsqrtf((float)a);
    const double h = 0.5 * a;
    double e = fma(-h * y, y, 0.5);
    y = fma(y, e, y);
    e = fma(-h * y, y, 0.5);
    return fma(y, e, y);
}

// Block-wide sum; every thread gets the result.  `sh` needs 32 doubles.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    constexpr int W = BLOCK / 32;
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = (lane < W) ? sh[lane] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    return sh[0];
}

}  // namespace rbffd
