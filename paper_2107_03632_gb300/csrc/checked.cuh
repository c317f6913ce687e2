// Bounds-checked build of the library (compiled with -DRBFFD_CHECKED).
//
// In the checked build every index a kernel computes is tested before the
// access it addresses:
//   RB_AT(p, i, n)        p[i] when 0 <= i < n.  Otherwise the violation is
//                         recorded and the access goes to a private sink of
//                         this translation unit (a read returns its bytes, a
//                         write lands there), so a wrong index never reaches
//                         memory outside the array.
//   RB_SPAN(off, len, n)  records a violation unless [off, off + len) lies in
//                         [0, n): a sub-array carved out of a larger one (a
//                         stencil's row of idx, a row of a CSR matrix), whose
//                         own accesses RB_AT then checks against len.
//   RB_PT(p, base, n)     *p, p a pointer into the array base[0 .. n): the
//                         same test as RB_AT(base, p - base, n)
//   RB_SH(p)              p, a pointer into the block's dynamic shared
//                         memory, when the whole object at p lies inside the
//                         launch's dynamic shared memory; otherwise the sink.
// A violation never stops a kernel (no trap, no device assert): it counts in
// the unit's device record, which also keeps the source file, line, index
// and bound of the unit's first violation; rbffd_checked_read gathers the
// records of all units.  In the normal build the macros are the plain
// expressions, so the normal build's code is the same as without them.
//
// Accesses that are not wrapped are those whose index is the loop variable
// of an enclosing loop bounded by the same array's extent (a grid-stride
// "for (i = ...; i < n; ...) y[i] = ..." over an array of n entries), and
// accesses at compile-time constant indices of fixed-size arrays.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace rbffd {

// FNV-1a (32-bit) hash of the base name of a path: identifies the source
// file of a violation in the device record.
constexpr uint32_t chk_name_hash(const char* path) {
    const char* b = path;
    for (const char* p = path; *p; ++p)
        if (*p == '/' || *p == '\\') b = p + 1;
    uint32_t h = 2166136261u;
    for (; *b; ++b) h = (h ^ (uint32_t)(unsigned char)*b) * 16777619u;
    return h;
}

// One translation unit's record, as read back on the host.
struct CheckedRecord {
    unsigned long long count;  // violations since the last reset
    long long file_hash, line, index, bound;  // the first violation
};
using CheckedReader = int (*)(CheckedRecord* out, int reset);
// Registers a unit's reader (host; called during library load).
void checked_register(CheckedReader read);

}  // namespace rbffd

#ifdef RBFFD_CHECKED

namespace {

__device__ unsigned long long rb_chk_count;
__device__ long long rb_chk_first[4];  // file hash, line, index, bound
__device__ __align__(16) unsigned char rb_chk_sink[256];

__device__ __noinline__ void rb_chk_fail(uint32_t file, int line, long long i, long long n) {
    if (atomicAdd(&rb_chk_count, 1ull) == 0ull) {
        rb_chk_first[0] = (long long)file;
        rb_chk_first[1] = line;
        rb_chk_first[2] = i;
        rb_chk_first[3] = n;
    }
}

template <class T, class I>
__device__ __forceinline__ T& rb_chk_at(T* p, I i, long long n, uint32_t file, int line) {
    static_assert(sizeof(T) <= sizeof(rb_chk_sink), "element larger than the sink");
    const long long k = (long long)i;
    if ((unsigned long long)k < (unsigned long long)n) return p[k];
    rb_chk_fail(file, line, k, n);
    return *reinterpret_cast<T*>(rb_chk_sink);
}

__device__ __forceinline__ void rb_chk_span(long long off, long long len, long long n, uint32_t file, int line) {
    if (off < 0 || len < 0 || off > n - len) rb_chk_fail(file, line, off + len, n);
}

template <class T>
__device__ __forceinline__ T* rb_chk_sh(T* p, uint32_t file, int line) {
    static_assert(sizeof(T) <= sizeof(rb_chk_sink), "element larger than the sink");
    extern __shared__ __align__(16) unsigned char rb_chk_dyn[];
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    // below the base the difference wraps to a huge unsigned offset
    const unsigned long long off =
        (unsigned long long)(reinterpret_cast<const char*>(p) - reinterpret_cast<const char*>(rb_chk_dyn));
    if (off + sizeof(T) <= (unsigned long long)dyn) return p;
    rb_chk_fail(file, line, (long long)off, (long long)dyn);
    return reinterpret_cast<T*>(rb_chk_sink);
}

int rb_chk_read(::rbffd::CheckedRecord* out, int reset) {
    cudaError_t e = cudaMemcpyFromSymbol(&out->count, rb_chk_count, sizeof(unsigned long long));
    long long first[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(first, rb_chk_first, sizeof(first));
    out->file_hash = first[0];
    out->line = first[1];
    out->index = first[2];
    out->bound = first[3];
    if (e == cudaSuccess && reset) {
        const unsigned long long zc = 0;
        const long long zf[4] = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(rb_chk_count, &zc, sizeof(zc));
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(rb_chk_first, zf, sizeof(zf));
    }
    return (int)e;
}

struct RbChkRegistration {
    RbChkRegistration() { ::rbffd::checked_register(&rb_chk_read); }
};
RbChkRegistration rb_chk_registration_;

}  // namespace

#define RB_FILE_HASH_ (::std::integral_constant<uint32_t, ::rbffd::chk_name_hash(__FILE__)>::value)
#define RB_AT(p, i, n) (rb_chk_at((p), (i), (long long)(n), RB_FILE_HASH_, __LINE__))
#define RB_SPAN(off, len, n) \
    rb_chk_span((long long)(off), (long long)(len), (long long)(n), RB_FILE_HASH_, __LINE__)
#define RB_PT(p, base, n) (rb_chk_at((base), (p) - (base), (long long)(n), RB_FILE_HASH_, __LINE__))
#define RB_SH(p) (rb_chk_sh((p), RB_FILE_HASH_, __LINE__))

#else

#define RB_AT(p, i, n) ((p)[i])
#define RB_SPAN(off, len, n) ((void)0)
#define RB_PT(p, base, n) (*(p))
#define RB_SH(p) (p)

#endif
