// Shared device/host helpers of the RBF-FD library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stddef.h>

#include "checked.cuh"
#include "rbffd.h"

namespace rbffd {

// NVTX range over one C-ABI call (header-only NVTX; a no-op unless a
// profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define RBFFD_NVTX(name) ::rbffd::NvtxRange rbffd_nvtx_range_(name)

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
// After a synchronisation: accounts the bracketed launch `slot` (a graph
// that looped on the device) as `count` launches of `bytes` in all.
void prof_commit_as(int slot, int count, int64_t bytes);

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

// ---- FP64 scalars with few FP64 instructions ----------------------------
// On this GPU the FP64 units issue 2 lanes per clock per SM (the FP32 pipe
// 128), and conversions between float and double and FP64 compares occupy
// them like a DFMA.  The helpers below move a double's leading bits into a
// float seed, and a float seed back into a double, with integer
// instructions only, and finish with FMA-based Newton-type corrections.

// Exponent field of a within [1023 - 100, 1023 + 100], i.e. 2^-100 <= |a| <
// 2^101: the range where the float seeds below are normal floats.
__device__ __forceinline__ bool seed_range(double a) {
    const unsigned e = ((unsigned)__double2hiint(a) >> 20) & 0x7ffu;
    return e - (1023u - 100u) <= 200u;
}
// Sign bit of a clear (a >= +0, or a NaN with the sign clear).
__device__ __forceinline__ bool sign_clear(double a) { return __double2hiint(a) >= 0; }
// a truncated to float (sign, exponent rebiased, leading 23 fraction bits);
// valid where seed_range(a).
__device__ __forceinline__ float f32_trunc(double a) {
    const unsigned hi = (unsigned)__double2hiint(a), lo = (unsigned)__double2loint(a);
    const unsigned mag = __funnelshift_l(lo, (hi & 0x7fffffffu) - (896u << 20), 3);
    return __uint_as_float(mag | (hi & 0x80000000u));
}
// A normal float as a double (exact).
__device__ __forceinline__ double f64_of(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned hi = (((b & 0x7fffffffu) >> 3) + (896u << 20)) | (b & 0x80000000u);
    return __hiloint2double((int)hi, (int)(b << 29));
}
// IEEE bit tests without FP64 compares.
__device__ __forceinline__ bool finite64(double a) {
    return (((unsigned)__double2hiint(a) >> 20) & 0x7ffu) != 0x7ffu;
}
__device__ __forceinline__ bool positive_finite64(double a) {  // 0 < a < inf
    return (unsigned long long)__double_as_longlong(a) - 1ull < 0x7fefffffffffffffull;
}

// FP64 reciprocal, reciprocal square root and square root from a float
// seed y0 (relative error e0 <= ~2^-21: the float function's own error plus
// the truncation of a to float).
//  1/a:      e = 1 - a y0, y = y0 (1 + e + e^2)          error ~e0^3 ~ 2^-63
//  a^-1/2:   e = 1 - a y0^2, y = y0 (1 + e/2 + 3e^2/8)    error ~(5/16) e0^3
//  sqrt(a):  s = a y0, then twice s += (a - s^2) y0/2     error ~(3/2) e0^3
// (the truncated Taylor series of (1 - e)^-1 and (1 - e)^-1/2, and Newton's
// iteration for s^2 = a with the derivative 2 s frozen at 2/y0).  Each ends
// with one rounding: within about one ulp of the correctly rounded result.
// Outside seed_range (and for a <= 0 where the root is asked) the IEEE
// operations run.
__device__ __forceinline__ double rcp64(double a) {
    if (!seed_range(a)) return __ddiv_rn(1.0, a);
    const double y = f64_of(__frcp_rn(f32_trunc(a)));
    const double e = fma(-a, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

__device__ __forceinline__ double rsqrt64(double a) {
    if (!(seed_range(a) && sign_clear(a))) return __ddiv_rn(1.0, __dsqrt_rn(a));
    const double y = f64_of(rsqrtf(f32_trunc(a)));
    const double e = fma(-(a * y), y, 1.0);
    return fma(y * e, fma(0.375, e, 0.5), y);
}

__device__ __forceinline__ double sqrt64(double a) {
    if (!(seed_range(a) && sign_clear(a))) return __dsqrt_rn(a);
    const float yf = rsqrtf(f32_trunc(a));
    const double hy = f64_of(0.5f * yf);
    double s = a * f64_of(yf);
    s = fma(fma(-s, s, a), hy, s);
    return fma(fma(-s, s, a), hy, s);
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
