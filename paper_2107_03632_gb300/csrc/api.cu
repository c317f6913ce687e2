// Status strings, error bookkeeping and device queries of the C ABI.
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

namespace rbffd {

static thread_local char g_last_error[256] = "no error";

void set_cuda_error(cudaError_t e) {
    const char* name = cudaGetErrorName(e);
    const char* msg = cudaGetErrorString(e);
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", name ? name : "?", msg ? msg : "?");
}

int sm_count() {
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    std::call_once(once[dev], [&] {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cached[dev] = v;
    });
    return cached[dev];
}

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_profiling{0};

struct ProfPair {
    cudaEvent_t a = nullptr, b = nullptr;
    int kind = 0;
    int64_t bytes = 0;
    bool pending = false;
};

static std::mutex g_prof_mu;
static std::vector<ProfPair> g_pairs;
static long long g_prof_launches[kProfKinds];
static double g_prof_ms[kProfKinds];
static long long g_prof_bytes[kProfKinds];

void note_launches(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

bool profiling() { return g_profiling.load(std::memory_order_relaxed) != 0; }

int prof_begin(cudaStream_t st) {
    if (!profiling()) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int slot = -1;
    for (size_t k = 0; k < g_pairs.size(); ++k)
        if (!g_pairs[k].pending) {
            slot = (int)k;
            break;
        }
    if (slot < 0) {
        ProfPair p;
        if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return -1;
        g_pairs.push_back(p);
        slot = (int)g_pairs.size() - 1;
    }
    if (cudaEventRecord(g_pairs[slot].a, st) != cudaSuccess) return -1;
    g_pairs[slot].pending = true;
    return slot;
}

void prof_end(int slot, cudaStream_t st, int kind, int64_t bytes) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfPair& p = g_pairs[slot];
    p.kind = kind;
    p.bytes = bytes;
    if (cudaEventRecord(p.b, st) != cudaSuccess) p.pending = false;
}

void prof_commit(const int* slots, int count, int keep) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int k = 0; k < count; ++k) {
        const int sl = slots[k];
        if (sl < 0 || sl >= (int)g_pairs.size()) continue;
        ProfPair& p = g_pairs[sl];
        if (!p.pending) continue;
        float ms = 0.f;
        if (k < keep && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_prof_launches[p.kind] += 1;
            g_prof_ms[p.kind] += ms;
            g_prof_bytes[p.kind] += p.bytes;
        }
        p.pending = false;
    }
}

void prof_commit_as(int slot, int count, int64_t bytes) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (slot < 0 || slot >= (int)g_pairs.size()) return;
    ProfPair& p = g_pairs[slot];
    if (!p.pending) return;
    float ms = 0.f;
    if (count > 0 && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        g_prof_launches[p.kind] += count;
        g_prof_ms[p.kind] += ms;
        g_prof_bytes[p.kind] += bytes;
    }
    p.pending = false;
}

void prof_collect() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (ProfPair& p : g_pairs) {
        if (!p.pending) continue;
        if (cudaEventQuery(p.b) != cudaSuccess) continue;  // not finished yet: keep for later
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_prof_launches[p.kind] += 1;
            g_prof_ms[p.kind] += ms;
            g_prof_bytes[p.kind] += p.bytes;
        }
        p.pending = false;
    }
}

// Readers of the bounds-checked build's per-unit violation records (each
// unit registers one while the library loads; none in the normal build).
static std::vector<CheckedReader>& checked_readers() {
    static std::vector<CheckedReader> v;
    return v;
}
static std::mutex& checked_mu() {
    static std::mutex mu;
    return mu;
}

void checked_register(CheckedReader read) {
    std::lock_guard<std::mutex> lk(checked_mu());
    checked_readers().push_back(read);
}

// Source files whose lines the records may name.
static const char* const kCheckedFiles[] = {"api.cu",     "knn.cu",      "weights.cu",  "assemble.cu",
                                             "krylov.cu",  "batched.cu",  "mg.cu",       "mg_batch.cu",
                                             "explicit.cu", "common.cuh", "scan.cuh",    "internal.cuh",
                                             "df32.cuh",   "checked.cuh"};

}  // namespace rbffd

extern "C" {

int rbffd_profile_enable(int on) {
    RBFFD_NVTX("rbffd_profile_enable");
    rbffd::g_profiling.store(on ? 1 : 0);
    return RBFFD_OK;
}

int rbffd_profile_read(rbffd_profile* out, int reset) {
    using namespace rbffd;
    RBFFD_NVTX("rbffd_profile_read");
    if (!out) return RBFFD_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (ProfPair& p : g_pairs)
            if (p.pending) cudaEventSynchronize(p.b);
    }
    prof_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    out->launches = g_launches.load();
    out->spmv64_launches = g_prof_launches[kProfSpmv64];
    out->spmv64_ms = g_prof_ms[kProfSpmv64];
    out->spmv64_bytes = g_prof_bytes[kProfSpmv64];
    out->spmv32_launches = g_prof_launches[kProfSpmv32];
    out->spmv32_ms = g_prof_ms[kProfSpmv32];
    out->spmv32_bytes = g_prof_bytes[kProfSpmv32];
    out->mg_launches = g_prof_launches[kProfMg];
    out->mg_ms = g_prof_ms[kProfMg];
    out->mg_bytes = g_prof_bytes[kProfMg];
    out->batch_iter_launches = g_prof_launches[kProfBatchIter];
    out->batch_iter_ms = g_prof_ms[kProfBatchIter];
    out->batch_iter_bytes = g_prof_bytes[kProfBatchIter];
    if (reset) {
        g_launches.store(0);
        for (int k = 0; k < kProfKinds; ++k) {
            g_prof_launches[k] = 0;
            g_prof_ms[k] = 0.0;
            g_prof_bytes[k] = 0;
        }
    }
    return RBFFD_OK;
}


int rbffd_checked_read(rbffd_checked_report* out, int reset) {
    using namespace rbffd;
    RBFFD_NVTX("rbffd_checked_read");
    if (!out) return RBFFD_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
#ifdef RBFFD_CHECKED
    out->checked = 1;
#endif
    std::lock_guard<std::mutex> lk(checked_mu());
    for (CheckedReader read : checked_readers()) {
        CheckedRecord r{};
        const int e = read(&r, reset);
        if (e != (int)cudaSuccess) {
            set_cuda_error((cudaError_t)e);
            return RBFFD_ERR_CUDA;
        }
        if (r.count && !out->violations) {
            out->line = (int32_t)r.line;
            out->index = r.index;
            out->bound = r.bound;
            const char* name = "?";
            for (const char* f : kCheckedFiles)
                if ((long long)chk_name_hash(f) == r.file_hash) name = f;
            snprintf(out->file, sizeof(out->file), "%s", name);
        }
        out->violations += (int64_t)r.count;
    }
    return RBFFD_OK;
}

const char* rbffd_status_string(int s) {
    switch (s) {
        case RBFFD_OK: return "RBFFD_OK";
        case RBFFD_ERR_INVALID_ARG: return "RBFFD_ERR_INVALID_ARG";
        case RBFFD_ERR_CUDA: return "RBFFD_ERR_CUDA";
        case RBFFD_ERR_SINGULAR_STENCIL: return "RBFFD_ERR_SINGULAR_STENCIL";
        case RBFFD_ERR_NOT_CONVERGED: return "RBFFD_ERR_NOT_CONVERGED";
        case RBFFD_ERR_BREAKDOWN: return "RBFFD_ERR_BREAKDOWN";
        case RBFFD_ERR_TIMEOUT: return "RBFFD_ERR_TIMEOUT";
        case RBFFD_ERR_WORKSPACE: return "RBFFD_ERR_WORKSPACE";
        default: return "RBFFD_UNKNOWN_STATUS";
    }
}

const char* rbffd_last_cuda_error(void) { return rbffd::g_last_error; }

int rbffd_version(void) { return 100; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Diagnostics: the library's FP64 reciprocal and reciprocal square root
// (Newton-Raphson on float seeds, used inside the weight solves), evaluated
// elementwise so that tests can hold them against IEEE results.
namespace rbffd {
namespace {
__global__ void diag_recip_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ rcp,
                                  double* __restrict__ rsq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (rcp) rcp[i] = rcp64(x[i]);
        if (rsq) rsq[i] = rsqrt64(x[i]);
    }
}
}  // namespace
}  // namespace rbffd

// ---------------------------------------------------------------------------
// Self-check of the bounds-checked build: one thread reads entry `index` of
// a 64-entry table with RB_AT against `bound`, tests the sub-array [span_off,
// span_off + span_len) against `bound` with RB_SPAN, and stores the value at
// byte `smem_off` of 64 bytes of dynamic shared memory through RB_SH.  In
// the checked build an index outside its bound is recorded and redirected
// (never performed); the normal build takes only in-range arguments, tested
// on the host before anything is launched.
namespace rbffd {
namespace {
constexpr int kProbeTable = 64;
constexpr int kProbeSmem = 64;
__device__ double g_probe_table[kProbeTable];

__global__ void checked_probe_kernel(int64_t index, int64_t bound, int64_t span_off, int64_t span_len,
                                     int64_t smem_off, double* out) {
    extern __shared__ __align__(16) unsigned char probe_smem[];
    const double v = RB_AT(g_probe_table, index, bound) + 1.0;
    RB_SPAN(span_off, span_len, bound);
    double* slot = reinterpret_cast<double*>(probe_smem + smem_off);
    *RB_SH(slot) = v;
    __syncwarp();
    out[0] = *RB_SH(slot);
}
}  // namespace
}  // namespace rbffd

extern "C" int rbffd_checked_probe(int64_t index, int64_t bound, int64_t span_off, int64_t span_len,
                                   int64_t smem_off, double* out, void* stream) {
    RBFFD_NVTX("rbffd_checked_probe");
    using namespace rbffd;
    if (!out || bound < 0 || bound > kProbeTable || smem_off % 8 != 0) return RBFFD_ERR_INVALID_ARG;
#ifndef RBFFD_CHECKED
    // the normal build performs only in-range accesses
    if (index < 0 || index >= bound || span_off < 0 || span_len < 0 || span_off > bound - span_len ||
        smem_off < 0 || smem_off > kProbeSmem - 8)
        return RBFFD_ERR_INVALID_ARG;
#endif
    checked_probe_kernel<<<1, 1, kProbeSmem, as_stream(stream)>>>(index, bound, span_off, span_len, smem_off, out);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}

extern "C" int rbffd_diag_recip(const double* x, int64_t n, double* rcp, double* rsqrt, void* stream) {
    RBFFD_NVTX("rbffd_diag_recip");
    using namespace rbffd;
    if (!x || n <= 0 || (!rcp && !rsqrt)) return RBFFD_ERR_INVALID_ARG;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    diag_recip_kernel<<<blocks, 256, 0, as_stream(stream)>>>(x, n, rcp, rsqrt);
    note_launches(1);
    RBFFD_LAUNCH_CHECK();
    return RBFFD_OK;
}
