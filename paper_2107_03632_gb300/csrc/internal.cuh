// Library-internal entry points shared between translation units (not part
// of the C ABI).
#pragma once

#include "common.cuh"

#include <vector>

namespace rbffd {

// n nearest of the N points xy for each of the Nq points qxy (or, with qxy
// NULL, for each of the N points themselves, i.e. the stencils): rows of
// idx in query order, ordered by (d^2, index).  ws: the stencil workspace
// of N points.
int knn_search(const double* xy, int64_t N, const double* qxy, int64_t Nq, int32_t n, int32_t* idx, void* ws,
               size_t ws_bytes, cudaStream_t st);

// Interpolation weights at the Nq points qxy from their stencils idx (Nq x n,
// indices into the Nd points xy): PHS r^3 + monomials of degree <= m, exact
// for those monomials.  node_status (may be NULL): 1 where singular.
int interp_weights(const double* xy, int64_t Nd, const double* qxy, int64_t Nq, const int32_t* idx, int32_t n,
                   int32_t m, double* w, int32_t* node_status, cudaStream_t st);

// Multigrid hierarchy built by rbffd_mg_setup (lives in the caller's rbffd_mg).
struct MgHierarchy;
const MgHierarchy* mg_hierarchy(const rbffd_mg* h);
int64_t mg_fine_rows(const MgHierarchy* h);
bool mg_has_fp32(const MgHierarchy* h);
// Enqueues x = M^-1 b, one V-cycle (FP64, or float32 values and vectors when
// fp32), on st; every kernel returns at once while *flag != 0.  With
// profiling on and ev given, the finest-level sweeps are bracketed with
// events (their slots appended to ev).
int mg_apply(const MgHierarchy* h, bool fp32, const double* b, double* x, const int* flag, cudaStream_t st,
             std::vector<int>* ev = nullptr);

}  // namespace rbffd
