/*
 * rbffd.h -- C ABI of the GB300 RBF-FD Poisson library.
 *
 * The library computes, on one GPU, the pipeline of the RBF-FD solution of
 * Poisson's equation on scattered 2D nodes (Jancic, Slak, Kosec, "GPU
 * accelerated RBF-FD solution of Poisson's equation", arXiv 2107.03632):
 *
 *   stencils  -> for every node, its n nearest nodes        (Sec. II, Eq. 1)
 *   weights   -> RBF-FD Laplacian weights, PHS r^3 + monomials of degree
 *                <= m, one augmented system per stencil      (Sec. II Eq. 1, Sec. V)
 *   assemble  -> the discrete Poisson operator, Dirichlet rows  (Sec. IV, Eqs. 2-4)
 *   rhs       -> b = -f on interior rows, g on Dirichlet rows   (Sec. IV, Eqs. 2-3)
 *   solve     -> BiCGSTAB on A u = b, FP64 or FP32-inner/FP64
 *                refinement (the implicit solve of Sec. VI)
 *   solve_adjoint -> A^T lambda = dL/du and the gradients dL/df, dL/dg
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers owned by the caller, unless a
 *    comment says "host".  The library makes no device-memory allocation of
 *    its own (no cudaMalloc): scratch space is a caller-provided workspace
 *    whose size the matching *_workspace_size function returns (workspace
 *    pointers must be 256-byte aligned).  Exceptions, where the CUDA runtime
 *    allocates on the library's behalf: rbffd_solve_batched creates its
 *    streams, events and CUDA graphs (captured, instantiated and destroyed
 *    within the call), and rbffd_explicit_run instantiates a CUDA graph of
 *    its steps on every call; graph instantiation reserves device memory.
 *    rbffd_stencils_noalloc uses a static device array (below).
 *  - Every entry point opens an NVTX range named after it (visible in
 *    profilers; free when no profiler is attached).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on that stream; calls return before it completes unless
 *    the comment says the call blocks.
 *  - Node coordinates xy are an N x 2 row-major float64 array (x0, y0, x1, ...).
 *    Stencils idx and weights w are N x n row-major (row i = node i).
 *  - Node indices are int32 (N < 2^31).
 *  - Return value: an rbffd_status.  Argument errors are detected on the host
 *    before anything is enqueued and nothing is written.  RBFFD_ERR_CUDA means
 *    a launch failed; the CUDA error string is available from
 *    rbffd_last_cuda_error().
 */
#ifndef RBFFD_H
#define RBFFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rbffd_status {
    RBFFD_OK = 0,
    RBFFD_ERR_INVALID_ARG = 1,      /* bad size, null pointer, unsupported m/n */
    RBFFD_ERR_CUDA = 2,             /* a CUDA call or launch failed */
    RBFFD_ERR_SINGULAR_STENCIL = 3, /* reported per node in node_status */
    RBFFD_ERR_NOT_CONVERGED = 4,    /* iteration cap reached, or the residual stagnated */
    RBFFD_ERR_BREAKDOWN = 5,        /* BiCGSTAB breakdown persisted after a restart */
    RBFFD_ERR_TIMEOUT = 6,          /* a bounded device wait gave up */
    RBFFD_ERR_WORKSPACE = 7         /* workspace too small or misaligned */
} rbffd_status;

/* Human-readable name of a status code (static string, host). */
const char* rbffd_status_string(int status);

/* Text of the last CUDA error seen by this library on the calling thread (host). */
const char* rbffd_last_cuda_error(void);

/* ABI version: 100 * major + minor. */
int rbffd_version(void);

/* Largest supported stencil size n. */
#define RBFFD_MAX_STENCIL 128

/* ------------------------------------------------------------------------ */
/* Stencil (support) selection -- Sec. II, Eq. 1: N(x) is the set of nodes   */
/* whose values approximate the operator at x; Sec. V uses the n nearest     */
/* nodes.                                                                    */
/*                                                                           */
/* For every node i, idx[i*n + 0 .. n-1] receives the n nodes nearest to     */
/* node i among all N nodes, node i itself included (first, distance 0),     */
/* ordered by squared distance d^2 = dx*dx + dy*dy (each product rounded,    */
/* no fused multiply-add) and, for equal d^2, by the smaller node index.     */
/* The result is exact (identical to brute force).                           */
/*   xy  : N x 2 float64, read only.                                         */
/*   n   : 1 <= n <= min(N, RBFFD_MAX_STENCIL).                              */
/*   idx : N x n int32, written.                                             */
/*   ws  : rbffd_stencils_workspace_size(N, n) bytes of device scratch.      */
/* Non-finite coordinates give unspecified stencils for those nodes (finite  */
/* nodes never select them).                                                 */
/* ------------------------------------------------------------------------ */
size_t rbffd_stencils_workspace_size(int64_t N, int32_t n);
int rbffd_stencils(const double* xy, int64_t N, int32_t n, int32_t* idx,
                   void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* rbffd_stencils without any device allocation and without a workspace.    */
/* (The paper has no counterpart: this serves callers that cannot allocate  */
/* device memory on their path -- code inside a CUDA stream capture, a      */
/* memory arena that owns all device memory, a loop that must not allocate  */
/* -- and cannot hand over scratch space either.)                           */
/* Same arguments, results and errors as rbffd_stencils, for N up to        */
/* RBFFD_STENCILS_NOALLOC_MAX_NODES; larger N returns RBFFD_ERR_INVALID_ARG  */
/* before anything is enqueued.  The scratch is one fixed device array of   */
/* RBFFD_STENCILS_NOALLOC_SCRATCH_BYTES inside the library, held by every   */
/* GPU that loads the library until the process exits.  The first call in  */
/* each CUDA context (per device, and again after cudaDeviceReset rebuilds  */
/* the context) looks up that array's device address                        */
/* (cudaGetSymbolAddress, with the device current) and caches it under the  */
/* context's unique ID: make that first call before any stream capture.     */
/* All calls share the array: calls whose work overlaps on the              */
/* GPU (other streams, other threads) race and give wrong stencils; calls   */
/* ordered on one stream are safe.  It calls no cudaMalloc, cudaFree or     */
/* other allocating routine.                                                 */
/* ------------------------------------------------------------------------ */
#define RBFFD_STENCILS_NOALLOC_MAX_NODES (1LL << 20)
#define RBFFD_STENCILS_NOALLOC_SCRATCH_BYTES (28u << 20)
int rbffd_stencils_noalloc(const double* xy, int64_t N, int32_t n, int32_t* idx, void* stream);

/* ------------------------------------------------------------------------ */
/* RBF-FD Laplacian weights -- Sec. II, Eq. 1 with the basis of Sec. V:      */
/* Phi(r) = r^3 augmented with all 2D monomials of degree <= m.              */
/*                                                                           */
/* For each node i with stencil idx[i*n ..], the augmented system            */
/*      [ Phi  P ] [ w ]   [ lap phi_j(x_i) ]      Phi_jk = |x_j - x_k|^3    */
/*      [ P^T  0 ] [ l ] = [ lap p_k(x_i)   ]      P_jk   = p_k(x_j)         */
/* is formed in coordinates shifted to x_i and scaled by delta_i (the        */
/* largest |x_j - x_i| in the stencil), solved, and                          */
/* w[i*n + j] = wh_j / delta_i^2.  The system of one stencil lives in shared */
/* memory and one, two or four warps solve it.  Solvers: null-space         */
/* elimination (Gauss-Jordan with row pivoting on P, then an L D L^T        */
/* factorisation of the positive definite Z^T Phi Z; m >= 1) and Gaussian   */
/* elimination with partial pivoting of the whole system (any m, the only   */
/* one for m = 0).  Arithmetic: FP64 by default; a double-float form of the */
/* null-space solver (pairs of floats, ~48 significant bits, on the FP32    */
/* pipe) is used only when selected through rbffd_weights_set_config or     */
/* rbffd_weights_autotune with RBFFD_WEIGHTS_DF / _ANY.                      */
/* Monomials are in graded order 1, x, y, x^2, xy, y^2, ...; s = (m+1)(m+2)/2.*/
/*   m           : 0 <= m <= 8 and s <= n (the system needs n >= s nodes).   */
/*   w           : N x n float64, written (rows of singular stencils: 0).    */
/*   node_status : N int32 or NULL; 0 = ok, 1 = singular/non-finite system.  */
/* No workspace.                                                             */
/* ------------------------------------------------------------------------ */
int rbffd_weights(const double* xy, const int32_t* idx, int64_t N, int32_t n, int32_t m,
                  double* w, int32_t* node_status, void* stream);

/* Weight-solve launch configuration ("tile shape") per (n, m): the solver   */
/* and its threads per stencil -- 0 null-space elimination, one warp per    */
/* stencil, 1..4 stencils (warps) per block; 1 full Gaussian elimination,  */
/* likewise; 2 / 3 null-space elimination with two / four warps per        */
/* stencil, one stencil per block (warps_per_block = 2 / 4); all in FP64.  */
/* 4 / 5 / 6: the same three null-space forms in double-float arithmetic   */
/* (FP64 only for the coordinate shift/scale and the final scaling),       */
/* offered for 1 <= m <= 6, where the scaled systems' conditioning keeps    */
/* the weights within ~1e-10 of FP64.  7 / 8: the null-space form with     */
/* half a warp (16 threads) per stencil, two stencils per warp, FP64 /      */
/* double-float (warps_per_block 1..4: 2..8 stencils per block); 9 / 10:    */
/* a quarter of a warp (8 threads), four stencils per warp (4..16 per      */
/* block).                                                                  */
/* The default is FP64: 2 (two warps per stencil) for m >= 5 when it fits,  */
/* 9 (a quarter warp, warps_per_block 2) for m <= 2 with n <= 16, 7 (half a */
/* warp, warps_per_block 2) for other m <= 4 with n <= 32, 0 for other     */
/* m >= 1, 1 for m = 0.                                                      */
/* RBFFD_WEIGHTS=ns64 (environment) forces the FP64 null-space form with    */
/* one warp per stencil, =df its double-float form (1 <= m <= 6), =lu the   */
/* Gaussian elimination.                                                     */
/* rbffd_weights_autotune times every candidate of the given precision      */
/* (RBFFD_WEIGHTS_FP64: kernels 0-3, 7, 9; RBFFD_WEIGHTS_DF: 4-6, 8, 10;    */
/* _ANY: all)                                                               */
/* that                                                                     */
/* fits in shared memory on the first min(N, 512 x SMs) stencils of the     */
/* given set (the fastest of 3 launches after one warm-up, CUDA events),    */
/* records the                                                               */
/* fastest for (current device, n, m) in a process-wide table that          */
/* rbffd_weights and rbffd_solve_batched then use, and returns it in *best   */
/* (may be NULL).  w and node_status serve as its scratch (their first rows */
/* are overwritten).  Synchronises `stream`.  (Autotuning has no            */
/* counterpart in the paper.)  rbffd_weights_get_config returns the          */
/* configuration in force; rbffd_weights_set_config pins one (NULL: back to  */
/* the default above, warps per block from the shared-memory footprint).   */
#define RBFFD_WEIGHTS_FP64 0
#define RBFFD_WEIGHTS_DF 1
#define RBFFD_WEIGHTS_ANY 2
typedef struct rbffd_weights_config {
    int32_t kernel;          /* 0 null-space (1 warp/stencil), 1 Gaussian, 2 / 3 null-space (2 / 4 warps), */
                             /* 4 / 5 / 6 as 0 / 2 / 3 in double-float arithmetic; 7 / 8 null-space     */
                             /* with half a warp per stencil, FP64 / double-float; 9 / 10 the same     */
                             /* with a quarter of a warp                                                 */
    int32_t warps_per_block; /* kernels 0, 1, 4: stencils (warps) per block; 2, 5: 2; 3, 6: 4;          */
                             /* 7, 8: warps per block (two stencils per warp); 9, 10: four per warp     */
    double ms_per_mnode;     /* autotune: measured ms per 1e6 stencils (0 otherwise) */
} rbffd_weights_config;
int rbffd_weights_autotune(const double* xy, const int32_t* idx, int64_t N, int32_t n, int32_t m,
                           double* w, int32_t* node_status, int32_t precision, rbffd_weights_config* best,
                           void* stream);
int rbffd_weights_get_config(int32_t n, int32_t m, rbffd_weights_config* cfg);
int rbffd_weights_set_config(int32_t n, int32_t m, const rbffd_weights_config* cfg);

/* ------------------------------------------------------------------------ */
/* Assembly -- Sec. IV, Eqs. 2-4 at steady state: interior rows carry the    */
/* RBF-FD Laplacian (A[i, idx[i,j]] = w[i,j], stencil order), Dirichlet rows */
/* carry the identity (A[i,i] = 1).  CSR with int64 row pointers.            */
/*                                                                           */
/* rbffd_assemble_pattern writes row_ptr (N+1 int64): rows have n entries,  */
/* Dirichlet rows 1.  nnz = row_ptr[N] = (N - N_dirichlet) * n + N_dirichlet.*/
/* rbffd_assemble then writes col (nnz int32) and val (nnz float64) and, if  */
/* val32 is not NULL, a float32 copy of val.  Rows whose range in row_ptr    */
/* would pass nnz are not written.                                           */
/*   is_dirichlet : N uint8 (nonzero = boundary node with a Dirichlet row).  */
/*   ws           : rbffd_assemble_workspace_size(N) bytes.                  */
/* ------------------------------------------------------------------------ */
size_t rbffd_assemble_workspace_size(int64_t N);
int rbffd_assemble_pattern(const uint8_t* is_dirichlet, int64_t N, int32_t n,
                           int64_t* row_ptr, void* ws, size_t ws_bytes, void* stream);
int rbffd_assemble(const int32_t* idx, const double* w, const uint8_t* is_dirichlet,
                   int64_t N, int32_t n, const int64_t* row_ptr, int64_t nnz,
                   int32_t* col, double* val, float* val32, void* stream);

/* Right-hand side -- Sec. IV, Eqs. 2-3 at steady state (-lap u = f inside,  */
/* u = g on the boundary): b[i] = g[i] if is_dirichlet[i] else -f[i].        */
int rbffd_rhs(const double* f, const double* g, const uint8_t* is_dirichlet, int64_t N,
              double* b, void* stream);

/* CSR descriptor (host struct holding device pointers). */
typedef struct rbffd_csr {
    int64_t n_rows;          /* square matrix: n_rows x n_rows */
    int64_t nnz;
    const int64_t* row_ptr;  /* n_rows + 1 */
    const int32_t* col;      /* nnz */
    const void* val;         /* nnz, float64 (dtype 0) or float32 (dtype 1) */
    int32_t dtype;
} rbffd_csr;

/* Transpose A (float64 values) into CSR of A^T (the operator of the       */
/* adjoint solve, rbffd_solve_adjoint).  Within a row of A^T the entries    */
/* are in increasing column order (deterministic).                          */
/*   row_ptr_t : n_rows + 1 int64, col_t : nnz int32, val_t : nnz float64.   */
/*   val32_t   : nnz float32 (val_t rounded to nearest), or NULL: the       */
/*               float32 copy the mixed-precision adjoint solve reads.       */
/*   ws        : rbffd_transpose_workspace_size(n_rows) bytes.               */
/* Asynchronous on `stream`; argument errors return before anything is      */
/* enqueued (RBFFD_ERR_INVALID_ARG, RBFFD_ERR_WORKSPACE).                    */
size_t rbffd_transpose_workspace_size(int64_t n_rows);
int rbffd_transpose(const rbffd_csr* A, int64_t* row_ptr_t, int32_t* col_t, double* val_t, float* val32_t,
                    void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Explicit time loop -- Sec. IV, Eq. 4, the paper's GPU workload: forward  */
/* Euler for u_t = lap u + f,                                               */
/*   u_2[i] = u_1[i] + dt (f[i] + sum_j w[i,j] u_1[idx[i,j]])   (interior), */
/* Dirichlet nodes unchanged.                                                */
/* rbffd_explicit_pack copies the interior rows of (idx, w) (N x n, as from  */
/* rbffd_stencils / rbffd_weights) into the workspace as column-major ELL    */
/* arrays with the interior list (Sec. V's data model), returns the         */
/* interior count in *n_interior (host) and synchronises `stream`;          */
/* RBFFD_ERR_INVALID_ARG if a stencil index of an interior row is outside   */
/* [0, N).  rbffd_explicit_run then advances u (device, N float64, in/out)   */
/* by `steps` steps of size dt on the stream (asynchronous; the steps run as */
/* replays of a CUDA graph of 64 launches).  f: N float64 (device).          */
/*   ws : rbffd_explicit_workspace_size(N, n) bytes, the same for both calls.*/
/* ------------------------------------------------------------------------ */
size_t rbffd_explicit_workspace_size(int64_t N, int32_t n);
int rbffd_explicit_pack(const int32_t* idx, const double* w, const uint8_t* is_dirichlet, int64_t N,
                        int32_t n, int64_t* n_interior, void* ws, size_t ws_bytes, void* stream);
int rbffd_explicit_run(const double* f, double* u, int64_t N, int32_t n, int64_t n_interior, double dt,
                       int64_t steps, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Multigrid preconditioner (an addition of this library: the paper has no  */
/* implicit solver, Sec. VI names one as the next step).  A geometric       */
/* V-cycle on the node sets themselves, built from the pieces of this      */
/* header:                                                                   */
/*  * coarsening: one node per cell of a uniform grid of side ~2x the mean   */
/*    spacing (a Dirichlet node where the cell has one, else the node        */
/*    nearest the cell centre; ties to the lower index), so each level has   */
/*    at most half the nodes of the one above; down to <= 128 nodes;         */
/*  * coarse operators: rediscretised -- stencils, RBF-FD Laplacian weights  */
/*    (r^3 + monomials of degree 2, n = 12) and Dirichlet rows on the coarse */
/*    nodes, as in Sec. II Eq. 1 / Sec. IV;                                  */
/*  * prolongation P: PHS r^3 + degree-2 interpolation from the 12 nearest   */
/*    coarse nodes (zero rows at Dirichlet nodes); restriction R = (N_c/N_f) */
/*    P^T with zero rows at coarse Dirichlet nodes;                          */
/*  * smoothing: nu Jacobi sweeps, weight omega on interior rows and 1 on   */
/*    Dirichlet rows, before and after;                                     */
/*    coarsest level: a dense inverse (Gauss-Jordan, partial pivoting).     */
/* With opts->precond = 1, rbffd_solve runs BiCGSTAB right-preconditioned by */
/* one V-cycle per application (FP64 V-cycle in precision 0; in precision 1 */
/* the V-cycle runs in float32 values and vectors inside the FP64 BiCGSTAB, */
/* which needs A32), from x_b = b_b on the Dirichlet rows (A's Dirichlet    */
/* rows must be identity rows, as rbffd_assemble writes them).  The adjoint */
/* solve takes the hierarchy of rbffd_mg_setup_adjoint / _adjoint_of: it    */
/* solves the interior block L_ii^T x_i = b_i left-preconditioned by the    */
/* transposed cycle and sets x_b = b_b - L_ib^T x_i after every pass; with  */
/* a hierarchy of rbffd_mg_galerkin_adjoint it runs right-preconditioned    */
/* (below).                                                                  */
/*   mg       : host object filled here; read by rbffd_solve.  It points     */
/*              into ws, which must stay allocated and unchanged meanwhile.  */
/*   A, A32   : the fine-level operator (as passed to rbffd_solve; A32 may   */
/*              be NULL, then only the FP64 V-cycle is available).           */
/*   nu       : 1..8 sweeps; omega: 0 < omega < 1 (e.g. nu 2, omega 0.6).   */
/*   ws       : rbffd_mg_workspace_size(N, A->nnz) bytes (a bound).          */
/* Synchronises `stream` (level sizes are read back).  Errors: invalid       */
/* arguments, RBFFD_ERR_SINGULAR_STENCIL if a coarse stencil or the coarsest */
/* matrix is singular.                                                       */
/* ------------------------------------------------------------------------ */
#define RBFFD_MG_MAX_LEVELS 24
typedef struct rbffd_mg {
    uint64_t opaque[2048];
} rbffd_mg;

size_t rbffd_mg_workspace_size(int64_t N, int64_t nnz);
int rbffd_mg_setup(const double* xy, const uint8_t* is_dirichlet, int64_t N, const rbffd_csr* A,
                   const rbffd_csr* A32, int32_t nu, double omega, rbffd_mg* mg, void* ws, size_t ws_bytes,
                   void* stream);
/* The same hierarchy as rbffd_mg_setup, built in two calls.  Everything   */
/* but the fine level's operator depends only on the nodes and the mask --  */
/* the coarse node sets, their operators and smoother weights, the          */
/* interpolation and restriction, the coarsest level's dense inverse -- so  */
/* rbffd_mg_setup_geometry builds it, and synchronises `stream`, while the  */
/* fine operator may still be computed on another stream (the weight solve, */
/* assembly).  rbffd_mg_setup_operator then attaches A (and A32, as in      */
/* rbffd_mg_setup) to level 0: its smoother weights, asynchronous on        */
/* `stream`; when the node set is a single level (N <= 128) also its dense  */
/* inverse, which synchronises `stream`.  Between the calls the hierarchy   */
/* serves nothing (rbffd_solve refuses it).  Forward hierarchies only.      */
/* ws: rbffd_mg_workspace_size(N, nnz) bytes (the size depends on N only). */
/* Errors: as rbffd_mg_setup; rbffd_mg_setup_operator returns               */
/* RBFFD_ERR_INVALID_ARG unless mg holds a geometry of N = A->n_rows nodes.  */
/* (The split has no counterpart in the paper.)                             */
int rbffd_mg_setup_geometry(const double* xy, const uint8_t* is_dirichlet, int64_t N, int32_t nu, double omega,
                            rbffd_mg* mg, void* ws, size_t ws_bytes, void* stream);
int rbffd_mg_setup_operator(rbffd_mg* mg, const rbffd_csr* A, const rbffd_csr* A32, void* stream);
/* rbffd_mg_setup_adjoint: the same hierarchy for the adjoint operator AT  */
/* = A^T (as passed to rbffd_solve_adjoint): every level's operator is the  */
/* transpose of the forward one (coarse levels rediscretised, then          */
/* transposed), restriction P^T and prolongation R^T = (N_c / N_f) P with   */
/* the coarse Dirichlet columns zeroed -- the exact transpose of the        */
/* forward V-cycle.  rbffd_solve takes only forward hierarchies,           */
/* rbffd_solve_adjoint only adjoint ones (else RBFFD_ERR_INVALID_ARG).      */
int rbffd_mg_setup_adjoint(const double* xy, const uint8_t* is_dirichlet, int64_t N, const rbffd_csr* AT,
                           const rbffd_csr* AT32, int32_t nu, double omega, rbffd_mg* mg, void* ws,
                           size_t ws_bytes, void* stream);
/* rbffd_mg_adjoint_of: the adjoint hierarchy of a built forward hierarchy */
/* `fwd` for AT = A^T (the matrix rbffd_solve_adjoint gets): the coarse      */
/* node sets, smoother weights and interpolation are fwd's (copied into ws, */
/* so fwd may be rebuilt or freed afterwards), the operators transposed,    */
/* the coarsest transposed operator inverted.  The result holds the same    */
/* values as rbffd_mg_setup_adjoint on the same inputs; it costs the        */
/* transposes instead of a second coarsening, kNN and weight solve.         */
/*   AT, AT32 : as for rbffd_mg_setup_adjoint (AT32 needs fwd built with a  */
/*              float32 copy).  ws: rbffd_mg_workspace_size(N, AT->nnz).     */
/* Synchronises `stream`.  Errors: RBFFD_ERR_INVALID_ARG (fwd not a built    */
/* forward hierarchy, sizes differ), RBFFD_ERR_WORKSPACE.                    */
int rbffd_mg_adjoint_of(const rbffd_mg* fwd, const rbffd_csr* AT, const rbffd_csr* AT32, rbffd_mg* mg, void* ws,
                        size_t ws_bytes, void* stream);
/* rbffd_mg_galerkin_adjoint: the adjoint hierarchy of a built forward     */
/* hierarchy `fwd` with GALERKIN coarse operators: node sets, interpolation */
/* and transfers as rbffd_mg_adjoint_of (restriction R = P^T, prolongation  */
/* (N_c / N_f) P without the coarse Dirichlet columns), but each coarse     */
/* operator is the product R A_l P of the level above (A_0 = AT), its rows  */
/* at coarse Dirichlet nodes replaced by identity rows, its columns sorted; */
/* smoother weights from its own diagonal; the coarsest inverted.  The      */
/* product is computed on the device in a fixed summation order (the same   */
/* bits on every run: rows are staged, then placed in CSR order).           */
/* rbffd_solve_adjoint runs with such a hierarchy                            */
/* RIGHT-preconditioned on the whole system: M = the cycle followed by the  */
/* Dirichlet back substitution, from x_b = b_b - L_ib^T x_i, so A^T M is    */
/* block diagonal with an identity Dirichlet block.                         */
/*   AT, AT32 : as for rbffd_mg_adjoint_of.                                  */
/*   ws       : rbffd_mg_galerkin_workspace_size(fwd) bytes: the layout of   */
/*              rbffd_mg_adjoint_of with room for 256 entries per coarse row */
/*              on average, plus as much staging room for the largest coarse */
/*              level (0 if fwd is not a built forward hierarchy).           */
/* Synchronises `stream`.  Errors: RBFFD_ERR_INVALID_ARG (as                 */
/* rbffd_mg_adjoint_of), RBFFD_ERR_WORKSPACE (ws too small; or a coarse row  */
/* with more than 512 entries, or one with more than 1024 distinct columns  */
/* in R_c A_l, or more entries on a level than the layout holds),           */
/* RBFFD_ERR_SINGULAR_STENCIL (a zero diagonal, a singular coarsest         */
/* matrix).                                                                  */
size_t rbffd_mg_galerkin_workspace_size(const rbffd_mg* fwd);
int rbffd_mg_galerkin_adjoint(const rbffd_mg* fwd, const rbffd_csr* AT, const rbffd_csr* AT32, rbffd_mg* mg,
                              void* ws, size_t ws_bytes, void* stream);
/* Levels of a built hierarchy (finest first); n_nodes: RBFFD_MG_MAX_LEVELS  */
/* entries, may be NULL.  Returns the level count, 0 if mg was not built.    */
int rbffd_mg_levels(const rbffd_mg* mg, int64_t* n_nodes);
/* rbffd_mg_level: read-only view of one level of a built hierarchy, for     */
/* inspection.  Every pointer is a device pointer into the hierarchy's       */
/* workspace (level 0: the caller's xy, mask and matrix), valid until the    */
/* workspace is rebuilt or freed.                                            */
/*   A      : the level's operator (FP64; the adjoint hierarchy: the         */
/*            transposed operator).                                          */
/*   w      : smoother weights W = Omega D^-1 (omega / a_ii on interior      */
/*            rows, 1 / a_ii on Dirichlet rows).                             */
/*   p_idx, p_val : the prolongation from level + 1 into this level, ELL    */
/*            n_nodes x p_k (coarse indices); forward hierarchy: P, the     */
/*            interpolation; adjoint: R^T = (N_c / N_f) P without the coarse */
/*            Dirichlet columns.  NULL (p_k 0) at the coarsest level.        */
/*   minv   : coarsest level only: its dense inverse, row-major.            */
/* Errors: RBFFD_ERR_INVALID_ARG (mg not built, level out of range).        */
typedef struct rbffd_mg_level_info {
    int64_t n_nodes;
    const double* xy;
    const uint8_t* is_dirichlet;
    rbffd_csr A;
    const double* w;
    const int32_t* p_idx;
    const double* p_val;
    int32_t p_k;
    const double* minv;
} rbffd_mg_level_info;
int rbffd_mg_level(const rbffd_mg* mg, int32_t level, rbffd_mg_level_info* out);
/* rbffd_mg_apply: x = M b, one application of the preconditioner on        */
/* `stream` (b, x: device, N float64 each, distinct).  Forward hierarchy:   */
/* one V-cycle B from x = 0.  Adjoint hierarchy: the transpose of the       */
/* forward preconditioner E_b + B (I - A E_b) (E_b selects the Dirichlet    */
/* entries), i.e. B^T followed by the Dirichlet back substitution           */
/* x_b = b_b - sum_i a_ib x_i.  fp32 != 0: float32 V-cycle (needs a         */
/* hierarchy built with A32).  Errors: RBFFD_ERR_INVALID_ARG.               */
int rbffd_mg_apply(const rbffd_mg* mg, int32_t fp32, const double* b, double* x, void* stream);

/* ------------------------------------------------------------------------ */
/* Krylov solve -- the implicit solution named in Sec. VI: A x = b by       */
/* BiCGSTAB (van der Vorst 1992) with left Jacobi scaling D^-1 A x = D^-1 b. */
/* Convergence is judged on the unscaled system: |b - A x|_2 <= tol |b|_2,   */
/* confirmed by an explicitly recomputed residual before returning OK.       */
/* BiCGSTAB runs in restarted passes: each pass starts from the explicit    */
/* residual (shadow residual = residual) and ends when its residual has     */
/* fallen by inner_tol, or when its recurrence residual reaches tol (after  */
/* a pass that ended so while the explicit residual stayed above tol, the   */
/* next pass aims 4 times lower, down to tol / 1000); at most max_outer     */
/* passes.                                                                   */
/*                                                                           */
/* precision 0 (FP64): matrix, vectors and scalars in float64.               */
/* precision 1 (mixed): an FP64 refinement loop (r = b - A x with the FP64   */
/*   matrix, x += correction in FP64) around inner BiCGSTAB iterations that  */
/*   read the float32 copy of the matrix (A32: same row_ptr and col arrays  */
/*   as A, float32 values) in difference form sum_j a_ij (d_j - d_i) +       */
/*   (sum_j a_ij) d_i, with double-float (2 x float32) Krylov vectors; an   */
/*   inner pass ends when its residual has fallen by inner_tol.             */
/*                                                                           */
/* x is in/out: the initial guess on entry, the solution on exit (warm       */
/* start).  The call BLOCKS the host until the solve ends and synchronises   */
/* `stream`; *info (host) receives the outcome.  A breakdown (rho or omega  */
/* zero or non-finite) restarts once from the true residual before           */
/* RBFFD_ERR_BREAKDOWN is returned.  Stagnation ends the solve early with   */
/* RBFFD_ERR_NOT_CONVERGED: the relative residual (explicit between passes, */
/* the recurrence estimate inside a pass) must halve at least once per      */
/* max(2000, k) iterations, k being the iteration count at its last halving */
/* (operators with spurious modes, e.g. stencils barely larger than the    */
/* polynomial space, otherwise ran to max_iter).                            */
/* ------------------------------------------------------------------------ */
typedef struct rbffd_solve_opts {
    double tol;          /* relative residual target, e.g. 1e-10 */
    int32_t max_iter;    /* cap on (inner) BiCGSTAB iterations in total */
    int32_t precision;   /* 0 = FP64, 1 = mixed FP32-inner / FP64 refinement */
    double inner_tol;    /* residual reduction per restarted pass, 0 < inner_tol < 1 */
    int32_t max_outer;   /* cap on passes (refinement steps in mixed mode) */
    int32_t jacobi;      /* 1 = left Jacobi scaling (default), 0 = none */
    int32_t precond;     /* 0 = none / Jacobi as above, 1 = multigrid (mg) */
    const rbffd_mg* mg;  /* hierarchy from rbffd_mg_setup when precond = 1 */
    /* rbffd_solve_batched with multigrid only (others ignore them): */
    int64_t spin_limit;  /* polls of each bounded device wait of the persistent coarse-level kernel */
                         /* before the solve stops with RBFFD_ERR_TIMEOUT; 0 = default (2^26) */
    int32_t wait_test;   /* tests of the timeout path: 1 = the first coarse-level task waits on a */
                         /* counter that nothing increments (the wait runs out); 0 otherwise */
    int32_t persistent;  /* 1 = every instance's coarse levels as one persistent launch from a */
                         /* device task queue; 0 (default) = one launch per level and operation */
    int32_t device_loop; /* 1 = the whole solve as one CUDA graph launch whose loops run on the */
                         /* device; 0 (default) = one graph launch per iteration, host-driven */
} rbffd_solve_opts;

typedef struct rbffd_solve_info {
    int32_t status;       /* rbffd_status of the solve */
    int32_t iters;        /* BiCGSTAB iterations performed (inner, in total) */
    int32_t outer_sweeps; /* refinement passes (mixed) or residual checks (FP64) */
    int32_t restarts;     /* breakdown or residual-drift restarts */
    double rel_residual;  /* final |b - A x| / |b| with the FP64 matrix */
} rbffd_solve_info;

size_t rbffd_solve_workspace_size(int64_t N, const rbffd_solve_opts* opts);
int rbffd_solve(const rbffd_csr* A, const rbffd_csr* A32, const double* b, double* x,
                const rbffd_solve_opts* opts, rbffd_solve_info* info,
                void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Adjoint solve -- gradient of a loss L(u) of the solution u = A^{-1} b.    */
/* Solves A^T lambda = dLdu with the same solver as rbffd_solve, given AT =  */
/* A^T (from rbffd_transpose), then, since b = -f inside and b = g on the    */
/* boundary:  dLdf[i] = -lambda[i] (interior), 0 (Dirichlet);                */
/*            dLdg[i] = lambda[i] (Dirichlet), 0 (interior).                 */
/* dLdf and dLdg may be NULL.  lambda is in/out (initial guess).  Blocks    */
/* like rbffd_solve.  Workspace: rbffd_solve_workspace_size.                 */
/* ------------------------------------------------------------------------ */
int rbffd_solve_adjoint(const rbffd_csr* AT, const rbffd_csr* AT32, const uint8_t* is_dirichlet,
                        const double* dLdu, double* lambda, double* dLdf, double* dLdg,
                        const rbffd_solve_opts* opts, rbffd_solve_info* info,
                        void* ws, size_t ws_bytes, void* stream);

/* Gradient of the misfit L(u) = sum over interior nodes of (u - u_target)^2 */
/* (the loss of the differentiable solve; no counterpart in the paper,     */
/* which has no loss and no gradient):                                      */
/* dLdu = 2 (u - u_target) on interior nodes, 0 on Dirichlet nodes.          */
/*   u, u_target, dLdu : device, N float64 each; is_dirichlet : N uint8.     */
/* Asynchronous on `stream`.  Errors: RBFFD_ERR_INVALID_ARG (null pointer,   */
/* N <= 0), returned before anything is enqueued.                            */
int rbffd_misfit_grad(const double* u, const double* u_target, const uint8_t* is_dirichlet, int64_t N,
                      double* dLdu, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched solve -- many independent node sets (instances) of uneven size   */
/* and degree, each with several right-hand sides, through the whole        */
/* pipeline of this header at once (the paper's method applied per          */
/* instance; batching has no counterpart in the paper).                     */
/*                                                                           */
/* Instances are stored back to back: instance i owns nodes                 */
/* [node_offset_i, node_offset_i + n_nodes_i) of xy (N_total x 2) and        */
/* is_dirichlet, and the same rows of the node-major right-hand-side and    */
/* solution arrays f, g, u (N_total x n_rhs, entry [node * n_rhs + k]).     */
/* Per instance: stencils, weights (degree m_i, stencil size n_i), the      */
/* block of the block-diagonal CSR, and n_rhs right-hand sides b = -f | g.  */
/* With opts->precond = 0 the solve is the Jacobi mixed one of rbffd_solve */
/* (float32 inner BiCGSTAB in double-float vectors, FP64 refinement), run   */
/* for all (instance, rhs) pairs together; the inner iterations are         */
/* replayed as one CUDA graph per chunk of iterations.  With                */
/* opts->precond = 1 (opts->mg is not used) each instance gets its own      */
/* multigrid hierarchy (as rbffd_mg_setup, V(2,2), omega 0.6) and every     */
/* pair runs BiCGSTAB right-preconditioned by the instance's float32        */
/* V-cycle, applied to all of its right-hand sides at once, with            */
/* double-float (2 x float32) Krylov vectors and the matrix read as float32 */
/* (leading, trailing) pairs, the solution kept in FP64.  The instances'    */
/* V-cycles run as one launch per (level, operation) over all instances,    */
/* or (opts->persistent = 1) as launches on level 0 and ONE persistent     */
/* launch for every instance's levels >= 1 (a device work queue of          */
/* (instance, level, operation, tile) tasks; each dependency wait is        */
/* bounded by opts->spin_limit polls, past which the solve stops with       */
/* RBFFD_ERR_TIMEOUT).  Each iteration (both V-cycles and the BiCGSTAB     */
/* kernels of every running pair) is one CUDA graph launch, the host       */
/* reading the count of running pairs in between; with opts->device_loop = */
/* 1 the whole solve -- rounds of (explicit FP64 residual, BiCGSTAB pass)  */
/* -- is ONE graph launch whose loops run on the device (conditional WHILE */
/* nodes, capped by max_outer and the per-pass iteration cap).             */
/* Either way each pair has its own                                          */
/* BiCGSTAB scalars and stops on its own relative residual (explicit FP64   */
/* residual with the FP64 matrix, tol).  Blocks the host like rbffd_solve.  */
/*   desc    : host array of n_inst descriptors (offsets contiguous, in      */
/*             order: node_offset_0 = 0, node_offset_{i+1} = node_offset_i + */
/*             n_nodes_i).                                                  */
/*   n_rhs   : 1 <= n_rhs <= 64.                                             */
/*   u       : N_total x n_rhs float64, in: initial guess, out: solution.    */
/*   info    : host array of n_inst; per instance the worst right-hand side */
/*             (largest final relative residual, most iterations).          */
/* Returns RBFFD_OK when every pair converged, else the worst status.       */
/* ------------------------------------------------------------------------ */
typedef struct rbffd_batch_desc {
    int64_t node_offset;
    int64_t n_nodes;
    int32_t m;
    int32_t n;
} rbffd_batch_desc;

/* Workspace of rbffd_solve_batched for these instances and the solver     */
/* options it will get (opts NULL: precond 0).                               */
size_t rbffd_batched_workspace_size(const rbffd_batch_desc* desc, int32_t n_inst, int32_t n_rhs,
                                    const rbffd_solve_opts* opts);
int rbffd_solve_batched(const rbffd_batch_desc* desc, int32_t n_inst, const double* xy,
                        const uint8_t* is_dirichlet, const double* f, const double* g, int32_t n_rhs,
                        double* u, const rbffd_solve_opts* opts, rbffd_solve_info* info, void* ws,
                        size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Measurement hooks (no counterpart in the paper; used to report roofline   */
/* fractions).  The library counts every kernel it launches.  With profiling */
/* enabled it also brackets each SpMV launch of the Krylov iteration with    */
/* CUDA events on the solve's stream and sums their device time together     */
/* with the launch's algorithmic bytes:                                      */
/*   nnz * (value bytes + 4) + 8 (N + 1) [row_ptr] + 8 N [gathered vector,   */
/*   read once] + 8 N [result] + 8 N [Jacobi scale] + 8 N [dot partner].     */
/* With the multigrid preconditioner it also brackets the finest level's     */
/* Jacobi sweeps of every V-cycle (mg_*): nnz * (value bytes + 4) +          */
/* 8 (N + 1) + N * (2 x vector bytes [iterate gathered once, result] +      */
/* right-hand-side bytes + value bytes [D^-1]).  The batched multigrid     */
/* solve brackets each iteration (one graph replay for all instances) with  */
/* its algorithmic bytes for all pairs: 168 B per (node, rhs) for the outer */
/* FP64 kernels + 2 x 12 nnz (FP64 matrix, once per rhs block) and, per     */
/* V-cycle, 118 B per (node, rhs) + 4 passes x 8 nnz on the finest level.   */
/* Profiling is process-wide, off by default, and meant for one thread and   */
/* one device.  rbffd_profile_read waits for bracketed launches to finish.   */
/* ------------------------------------------------------------------------ */
typedef struct rbffd_profile {
    int64_t launches;         /* kernels launched since the last reset */
    int64_t spmv64_launches;  /* timed SpMV launches, float64 values */
    double spmv64_ms;
    int64_t spmv64_bytes;
    int64_t spmv32_launches;  /* timed SpMV launches, float32 values */
    double spmv32_ms;
    int64_t spmv32_bytes;
    int64_t mg_launches;      /* timed finest-level V-cycle sweeps */
    double mg_ms;
    int64_t mg_bytes;
    int64_t batch_iter_launches;  /* timed iterations (graph replays) of the batched multigrid solve */
    double batch_iter_ms;
    int64_t batch_iter_bytes;
} rbffd_profile;

/* Diagnostics (no counterpart in the paper): evaluates on the device, for   */
/* each of the n float64 values x (device), the library's own FP64           */
/* reciprocal and reciprocal square root -- Newton-Raphson refinement of a   */
/* float32 seed, used inside the weight solves -- into rcp and rsqrt        */
/* (device, n float64 each; either may be NULL).  Asynchronous on stream.    */
int rbffd_diag_recip(const double* x, int64_t n, double* rcp, double* rsqrt, void* stream);

int rbffd_profile_enable(int on);
int rbffd_profile_read(rbffd_profile* out, int reset);

/* Bounds-checked build (no counterpart in the paper; a testing aid).  The   */
/* library compiled with -DRBFFD_CHECKED (librbffd_checked.so) tests every    */
/* index its kernels compute -- global gathers and scatters, sub-arrays of   */
/* larger arrays (stencil rows, CSR rows), and pointers into shared memory   */
/* -- before the access.  An index out of range does not stop the kernel:    */
/* the access goes to a private scratch location instead (a read returns     */
/* its bytes, a write lands there) and the violation is counted in a device  */
/* record per source unit.  rbffd_checked_read gathers those records into    */
/* *out: checked = 1 in the checked build (0 and no violations otherwise),   */
/* violations = their total since the last reset, and file / line / index /  */
/* bound of the first violation of the first unit that has one (index is    */
/* the offending index, or the end of the offending sub-array, or the byte   */
/* offset into shared memory; bound the extent it broke).  Call it after the */
/* work has completed (synchronise the streams first); reset != 0 clears     */
/* the records.  Errors: RBFFD_ERR_INVALID_ARG (out NULL), RBFFD_ERR_CUDA.   */
typedef struct rbffd_checked_report {
    int32_t checked;     /* 1: this library is the bounds-checked build */
    int32_t line;        /* first violation: source line */
    char file[32];       /* first violation: source file (base name) */
    int64_t violations;  /* violations since the last reset */
    int64_t index;       /* first violation: the index (or end, or byte offset) */
    int64_t bound;       /* first violation: the extent it broke */
} rbffd_checked_report;
int rbffd_checked_read(rbffd_checked_report* out, int reset);
/* Self-check of the bounds-checked build: one thread reads entry `index` of */
/* a 64-entry zero-filled device table tested against `bound` (<= 64), tests */
/* the sub-array [span_off, span_off + span_len) against `bound`, and stores */
/* 1 + that entry at byte smem_off (a multiple of 8) of 64 bytes of dynamic  */
/* shared memory, then reads it back into *out (device, 1 double).  The      */
/* checked build records (and redirects) each access outside its bound, so  */
/* out-of-range arguments show up in rbffd_checked_read; the normal build    */
/* returns RBFFD_ERR_INVALID_ARG for them before launching anything.         */
/* Asynchronous on `stream`.                                                 */
int rbffd_checked_probe(int64_t index, int64_t bound, int64_t span_off, int64_t span_len, int64_t smem_off,
                        double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RBFFD_H */
