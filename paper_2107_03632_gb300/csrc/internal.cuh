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
constexpr uint32_t kMgGeometryMagic = 0x4D474753u;  // geometry built, fine operator not attached yet
constexpr int kMgGalerkinRow = 256;  // Galerkin coarse operators: mean entries per row the layout holds

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
    int galerkin;    // adjoint hierarchy with Galerkin coarse operators (rbffd_mg_galerkin_adjoint)
    double omega;
    void* ws;         // the workspace the hierarchy lives in
    size_t ws_bytes;
    MgLevel lv[RBFFD_MG_MAX_LEVELS];
};
const MgHierarchy* mg_hierarchy(const rbffd_mg* h);
int64_t mg_fine_rows(const MgHierarchy* h);
bool mg_has_fp32(const MgHierarchy* h);
bool mg_is_transposed(const MgHierarchy* h);
bool mg_is_galerkin(const MgHierarchy* h);
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

// The two phases of mg_setup_core.  Geometry: everything that depends on
// the nodes and the mask only -- the coarse node sets, their operators and
// smoother weights, interpolation and restriction, the coarsest level's
// dense inverse -- and level 0's geometry; synchronises st.  Operator: the
// fine operator attached to level 0 (its smoother weights; its dense
// inverse when it is the only level, which synchronises st).
int mg_setup_geometry(const double* xy, const uint8_t* mask, int64_t N, int col_base, int nu, double omega,
                      rbffd_mg* mg, void* ws, size_t ws_bytes, cudaStream_t st, bool transposed = false);
int mg_setup_operator(rbffd_mg* mg, const int64_t* row_ptr, const int* col, const double* val, const float* val32,
                      int64_t nnz, cudaStream_t st);

// The adjoint hierarchy of the forward hierarchy F for AT = A^T
// (rbffd_mg_adjoint_of).
int mg_adjoint_of(const MgHierarchy& F, const rbffd_csr* AT, const float* val32, rbffd_mg* mg, void* ws,
                  size_t ws_bytes, cudaStream_t st);
// The adjoint hierarchy of F with Galerkin coarse operators
// (rbffd_mg_galerkin_adjoint) and its workspace.
size_t mg_galerkin_workspace(const MgHierarchy& F);
int mg_galerkin_adjoint(const MgHierarchy& F, const rbffd_csr* AT, const float* val32, rbffd_mg* mg, void* ws,
                        size_t ws_bytes, cudaStream_t st);

// Coarse-level vectors of the multi-right-hand-side V-cycle (4 float
// vectors of N_l x R per coarse level l).
size_t mg_multi_coarse_floats(const MgHierarchy* h, int R);

// Batched multi-right-hand-side float32 V-cycle over many instances'
// hierarchies (mg_batch.cu): one launch per (level, operation) over every
// instance with that level, from device tables of (instance, level)
// descriptors and row tiles.  Vectors are node-major [row][R] (R <= 64).
struct MbLevel;
struct MbUnit;
struct MbTask;
struct MgBatch {
    const MbLevel* desc;
    const MbUnit* units;
    int levels, nu, persistent;
    // per level: units of the instances going deeper (a), of those whose
    // coarsest level it is (d), and of the next level's rows of the former (c)
    int a_off[RBFFD_MG_MAX_LEVELS], a_n[RBFFD_MG_MAX_LEVELS];
    int d_off[RBFFD_MG_MAX_LEVELS], d_n[RBFFD_MG_MAX_LEVELS];
    int c_off[RBFFD_MG_MAX_LEVELS], c_n[RBFFD_MG_MAX_LEVELS];
    // the persistent mode's task queue for levels >= 1 and its counters
    const MbTask* tasks;
    int ntasks, ncount, coarse_grid;
    int *head, *done, *status;
    long long spin_limit;
};
// Device bytes of the tables for n_inst instances of total_nodes nodes.
size_t mg_batch_table_bytes(int n_inst, int64_t total_nodes);
// Fills the tables (synchronises st).  H[i]: instance i's hierarchy, built
// with col_base = node_off[i] on its block of the batched matrix; x0, t0,
// r0: level-0 work vectors over all rows [N_total][R]; coarse +
// coarse_off[i]: instance i's coarse-level vectors (mg_multi_coarse_floats).
// persistent: levels >= 1 as one persistent launch from a task queue (else
// one launch per level and operation); spin_limit: polls of its bounded
// waits (0: the default); wait_test (tests only): the first coarse task
// waits on a counter that nothing increments, so the wait runs out.
int mg_batch_build(const MgHierarchy* const* H, const int64_t* node_off, int n_inst, int R, float* x0, float* t0,
                   float* r0, float* coarse, const size_t* coarse_off, void* tables, size_t table_bytes,
                   int persistent, long long spin_limit, int wait_test, cudaStream_t st, MgBatch* out);
// x = M^-1 b for every instance and right-hand side, b and x double-float
// pairs (the leading float is used; the result's trailing part is zero).
// Units of instance i return at once while live[i] == 0.
int mg_batch_apply_df(const MgBatch& B, int R, const float2* b, float2* x, const int* live, cudaStream_t st,
                      int* launches);
// Whether a bounded wait of the persistent kernel ran out (synchronises st).
int mg_batch_timed_out(const MgBatch& B, cudaStream_t st, bool* out);

}  // namespace rbffd
