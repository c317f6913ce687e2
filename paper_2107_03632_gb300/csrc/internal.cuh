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

// Laplacian weights of a multigrid coarse level (double-float null-space
// solve for 1 <= m <= 6, FP64 otherwise): the preconditioner's operators.
int coarse_weights(const double* xy, const int32_t* idx, int64_t N, int32_t n, int32_t m, double* w,
                   int32_t* node_status, cudaStream_t st);

// Interpolation weights at the Nq points qxy from their stencils idx (Nq x n,
// indices into the Nd points xy): PHS r^3 + monomials of degree <= m, exact
// for those monomials.  node_status (may be NULL): 1 where singular.
int interp_weights(const double* xy, int64_t Nd, const double* qxy, int64_t Nq, const int32_t* idx, int32_t n,
                   int32_t m, double* w, int32_t* node_status, cudaStream_t st);

// Multigrid hierarchy built by rbffd_mg_setup (lives in the caller's rbffd_mg).
constexpr int kMgCoarsest = 128;  // dense inverse (one-block Gauss-Jordan) at or below this size
constexpr int kMgK = 12;          // coarse nodes per interpolation stencil
constexpr int kMgInterpM = 2;     // interpolation degree
constexpr int kMgCoarseN = 12;    // coarse operator: stencil size
constexpr int kMgCoarseM = 2;     //                  and degree
constexpr uint32_t kMgMagic = 0x4D475242u;

struct MgLevel {
    int64_t N;
    // operator of this level (level 0: the caller's matrix)
    const int64_t* row_ptr;
    const int* col;
    const double* val;
    const float* val32;
    int64_t nnz;
    int tpr;
    double* dinv;
    float* dinv32;
    // geometry of coarse levels (level 0: the caller's arrays)
    const double* xy;
    const uint8_t* mask;
    // transfer to the next level: P (N x kMgK, ELL row-major), R (CSR)
    int32_t* pidx;
    double* pval;
    float* pval32;
    int64_t* rrow;
    int32_t* rcol;
    double* rval;
    float* rval32;
    int rtpr;
    // vectors (x and t alternate as the current iterate)
    double *x, *t, *r, *b;
    float *x32, *t32, *r32, *b32;
    // coarsest: dense inverse, row-major N x N
    double* minv;
    float* minv32;
};

struct MgHierarchy {
    uint32_t magic;
    int n_levels;
    int nu;
    int has32;
    int col_base;  // level-0 column indices are offset by this (rows local)
    int transposed;  // built for A^T (rbffd_mg_setup_adjoint)
    double omega;
    MgLevel lv[RBFFD_MG_MAX_LEVELS];
};
const MgHierarchy* mg_hierarchy(const rbffd_mg* h);
int64_t mg_fine_rows(const MgHierarchy* h);
bool mg_has_fp32(const MgHierarchy* h);
bool mg_is_transposed(const MgHierarchy* h);
// Enqueues x = M^-1 b, one V-cycle (FP64, or float32 values and vectors when
// fp32), on st; every kernel returns at once while *flag != 0.  With
// profiling on and ev given, the finest-level sweeps are bracketed with
// events (their slots appended to ev).
// Forward hierarchies: B, the V-cycle.  Adjoint hierarchies: B^T, then the
// Dirichlet back substitution (mg_dirichlet_fix), i.e. the transpose of
// M = E_b + B (I - A E_b) (E_b: the Dirichlet rows' selector), which equals
// B on the residuals a forward solve started by mg_dirichlet_fix produces.
// With A = [I 0; L_ib L_ii] (Dirichlet rows first) M A = diag(I, B_ii L_ii),
// so the adjoint's preconditioned operator is block diagonal.
int mg_apply(const MgHierarchy* h, bool fp32, const double* b, double* x, const int* flag, cudaStream_t st,
             std::vector<int>* ev = nullptr);
// x = Pi B b: the V-cycle alone, Dirichlet entries of the result zeroed
// (Pi); with the adjoint hierarchy, on boundary-free b, B_ii^T b_i (the left
// preconditioner of the adjoint's interior system).
int mg_apply_interior(const MgHierarchy* h, bool fp32, const double* b, double* x, const int* flag, cudaStream_t st,
                      std::vector<int>* ev = nullptr);
// y_b += W_b (r_b - (A y)_b) on the Dirichlet rows of level 0 (see
// mg_bfix_kernel); one launch on st.
int mg_dirichlet_fix(const MgHierarchy* h, const double* r, double* y, const int* flag, cudaStream_t st);

// rbffd_mg_setup for a fine operator given by arrays: row_ptr points at the
// fine rows' first entry (values are offsets into col/val), and column
// indices are offset by col_base (a block of a larger block-diagonal matrix).
int mg_setup_core(const double* xy, const uint8_t* mask, int64_t N, const int64_t* row_ptr, const int* col,
                  const double* val, const float* val32, int64_t nnz, int col_base, int nu, double omega,
                  rbffd_mg* mg, void* ws, size_t ws_bytes, cudaStream_t st, bool transposed = false);

// The adjoint hierarchy of the forward hierarchy F for AT = A^T
// (rbffd_mg_adjoint_of).
int mg_adjoint_of(const MgHierarchy& F, const rbffd_csr* AT, const float* val32, rbffd_mg* mg, void* ws,
                  size_t ws_bytes, cudaStream_t st);

// Multi-right-hand-side float32 V-cycle on node-major vectors [row][R]
// (R <= 64): x = M^-1 b for every column.  Level 0 works on rows
// [row_off, row_off + N) of the caller's arrays b (FP64), x (FP64 output)
// and the float work vectors x0, t0, r0 (all with the same row numbering,
// which the level-0 column indices, offset by the hierarchy's col_base,
// also use); the coarse levels use `coarse` (mg_multi_coarse_floats floats).
// Every kernel returns at once while *live == 0 (live may be NULL).
size_t mg_multi_coarse_floats(const MgHierarchy* h, int R);
int mg_apply_multi(const MgHierarchy* h, int64_t row_off, int R, const double* b, double* x, float* x0, float* t0,
                   float* r0, float* coarse, const int* live, cudaStream_t st, int* launches);
// The same with double-float (float2: leading, trailing) right-hand sides
// and results (the result's trailing part is zero).
int mg_apply_multi_df(const MgHierarchy* h, int64_t row_off, int R, const float2* b, float2* x, float* x0, float* t0,
                      float* r0, float* coarse, const int* live, cudaStream_t st, int* launches);

}  // namespace rbffd
