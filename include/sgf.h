/*
 * sgf.h - C ABI of the GB300 Sparse Geometric Factorization (SGF) library.
 *
 * The library builds the approximate factorization A ~ A_l of Algorithm 4.1
 * (Klockiewicz & Darve, "Sparse Hierarchical Preconditioners Using Piecewise
 * Smooth Approximations of Eigenvectors") for SPD matrices that come from a
 * stencil discretization on a cartesian grid, applies A_l^{-1} (Sec. 4.7) and
 * runs conjugate gradients preconditioned with it (Sec. 7).
 *
 * Conventions shared by every call:
 *  - Every call returns an int status: SGF_OK (0) or a negative SGF_ERR_*.
 *    No exception crosses the ABI.  sgf_status_string() names a status.
 *  - Handles (sgf_plan, sgf_factor_t) are opaque and owned by the library; free
 *    them with sgf_plan_destroy / sgf_factor_destroy.
 *  - Pointers named *_dev are device pointers (any allocation of the current
 *    CUDA device, e.g. a torch tensor's data_ptr()); *_host are host pointers.
 *    Caller buffers are borrowed for the duration of the call: the calls that
 *    take a stream enqueue their device work on it and return once it is
 *    enqueued unless the description says the call synchronizes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Vectors of the unknowns use the natural order: grid point (x, y, z) has
 *    number x + nx*(y + ny*z), and DOF c of a vector problem is 3*point + c.
 *    Several right-hand sides are stored one after the other (nrhs x n,
 *    row-major: RHS j starts at j*n).
 *  - Coefficient arrays are FP64 per cell in the same natural order; for Q1
 *    elasticity one Young's modulus per hexahedral element (ex x ey x ez,
 *    x fastest) where the point grid is ex x (ey+1) x (ez+1) free nodes (the
 *    nodes of the clamped x = 0 face are removed; point x index i is node
 *    x = i + 1).
 */
#ifndef SGF_H_
#define SGF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
  SGF_OK = 0,
  SGF_ERR_INVALID_ARG = -1,    /* a pointer, size or option is out of range   */
  SGF_ERR_NOT_SPD = -2,        /* a Cholesky pivot was <= 0 (node in info)     */
  SGF_ERR_NONFINITE = -3,      /* NaN/Inf in an input or a pivot               */
  SGF_ERR_OOM = -4,            /* device allocation failed                     */
  SGF_ERR_NO_CONVERGENCE = -5, /* PCG reached maxit before rtol                */
  SGF_ERR_TIMEOUT = -6,        /* a bounded device wait gave up                */
  SGF_ERR_CUDA = -7,           /* a CUDA runtime call failed                   */
  SGF_ERR_UNSUPPORTED = -8     /* valid request this build does not implement  */
};

/* ---- problem description (Sec. 5 cartesian grids, Sec. 7.1 problems) --- */
typedef enum {
  SGF_STENCIL_5PT_2D = 0,    /* FD Laplacian -div(k grad u), ghost Dirichlet (weight 1)   */
  SGF_STENCIL_7PT_3D = 1,    /* FD 7-point, ghost Dirichlet (weight 1)                    */
  SGF_STENCIL_7PT_FV_3D = 2, /* two-point-flux finite volume, half-cell Dirichlet (w 2)   */
  SGF_STENCIL_Q1_ELASTIC_3D = 3 /* trilinear hexahedra, 3 DOF / node, x- face clamped    */
} sgf_stencil;

/* Dirichlet face bits; every other face is natural (Neumann / no flow). */
enum { SGF_FACE_XM = 1, SGF_FACE_XP = 2, SGF_FACE_YM = 4, SGF_FACE_YP = 8,
       SGF_FACE_ZM = 16, SGF_FACE_ZP = 32 };

typedef struct sgf_grid {
  int dim;           /* 2 or 3                                              */
  int n[3];          /* unknowns (cells / points) per axis; n[2] = 1 in 2D  */
  int dof;           /* unknowns per point: 1 (scalar)                      */
  unsigned dirichlet;/* OR of SGF_FACE_* bits                               */
} sgf_grid;

/* Which separators get compressed (Sec. 5.1). */
typedef enum {
  SGF_SCHEME_NEST_ALL_ALL = 0, /* every separator cell of dimension >= 1      */
  SGF_SCHEME_NEST_2_ALL = 1,   /* codimension-1 separators only               */
  SGF_SCHEME_NONE = 2,         /* no compression: exact block Cholesky        */
  SGF_SCHEME_GEN_ALL_ALL = 3,  /* general partitions (Sec. 5.2): cells of      */
                               /* (b 2^(t-1))^3 vertices, no interiors, every  */
                               /* node compressed                              */
  SGF_SCHEME_NEST_2_2 = 4      /* codimension-1 separators, their blocks to the*/
                               /* lower-dimensional separators on their rim    */
                               /* (boxes at most one grid step apart) kept     */
                               /* exactly in span(Q1)                          */
} sgf_scheme;

typedef enum { SGF_BASIS_POLY = 0, SGF_BASIS_RBM = 1 } sgf_basis;
typedef enum { SGF_PREC_FP64 = 0, SGF_PREC_MIXED = 1 } sgf_precision;

typedef struct sgf_opts {
  int scheme;              /* sgf_scheme                                        */
  int leaf;                /* b: level-1 cut spacing (Sec. 5.1), >= 2            */
  int degree;              /* j of Pi^j: 0, 1 or 2 (Sec. 3.1)                    */
  int basis;               /* sgf_basis                                         */
  int precision;           /* sgf_precision                                     */
  double tau;              /* rank tolerance: keep |R_kk| > tau |R_11|; <=0 = default */
  int compress_from_level; /* first level whose separators may compress (>= 1)  */
  double nu;               /* Poisson ratio for Q1 elasticity (<= 0: 0.3)       */
} sgf_opts;

typedef struct sgf_plan sgf_plan;
typedef struct sgf_factor_s sgf_factor_t;

/* ---- analysis ------------------------------------------------------------
 * sgf_analyze: geometric nested dissection of Sec. 5.1 (cut spacing
 * d = leaf * 2^(t-1) at level t, one separator layer every d unknowns), the
 * node orders, parent/child maps and block sparsity of every level, the
 * node-local polynomial bases Pi^j of Sec. 3.1 and the re-expansion matrices
 * used when nodes merge (Sec. 4.4).  Host only; no device work.
 * Q1 elasticity (Sec. 7.1.3 on hexahedra): dof = 3, the rigid-body-mode
 * basis (Sec. 7.2), the x- face clamped.
 * Errors: INVALID_ARG for bad sizes/options, UNSUPPORTED for combinations
 * this build does not implement.                                            */
int sgf_analyze(const sgf_grid* grid, int stencil, const sgf_opts* opts, sgf_plan** out);
void sgf_plan_destroy(sgf_plan* plan);

/* Level summary: number of levels (top included) and unknowns. */
int sgf_plan_info(const sgf_plan* plan, int* nlevels, int64_t* n_unknowns);

/* Symbolic export for bit-exact comparison, one level at a time (0-based
 * `level`).  Every array argument may be NULL; counts are always written.
 *  nnodes, npairs, npost: node count, pre-elimination block pairs (u < v),
 *  post-elimination separator pairs.
 *  codes: 3 ints per node (z, y, x cell codes: 2k interval k, 2k+1 separator k)
 *  flags: per node, bit 0 = interior, bits 4..7 = cell dimension
 *  child_ptr (nnodes+1), child_idx: children in the previous level (level>0)
 *  pairs (2*npairs), post (2*npost).                                        */
int sgf_plan_export_level(const sgf_plan* plan, int level, int* nnodes, int* npairs,
                          int* npost, int* codes, int* flags, int* child_ptr,
                          int* child_idx, int* pairs, int* post);

/* Bytes of device memory sgf_factor needs (upper bound from the structural
 * node sizes), for FP64 and for mixed precision; used for admission.        */
int sgf_plan_footprint(const sgf_plan* plan, size_t* bytes_fp64, size_t* bytes_mixed);

/* ---- launch-shape tuning ---------------------------------------------------
 * Parameters of the batched launches that change speed and the order of
 * floating-point sums, not the method (Sec. 4 is unchanged by them).  Kept per
 * plan; every later sgf_factor of the plan uses them.
 *   gemv_min_elems, gemv_max_elems: element budget of one apply GEMV task
 *     (a launch's elements spread over about eight tasks per SM, clamped to
 *     this range); 256 <= min <= max <= 1 << 20.
 *   front_small: largest front (rows) the one-CTA elimination kernel takes in
 *     a batch of at least one front per SM (single precision); 64..512.
 *   tensor_cores: single-precision factor GEMMs on the tensor cores with
 *     every FP32 operand split into TF32 parts: 1 = two parts and three
 *     products (the 3xTF32 scheme), 2 = three parts and six products; both
 *     flush the tensor-core partial sums to FP32 registers every 32 terms of
 *     K (the tensor cores accumulate with truncation); 0 = FP32 CUDA cores
 *     only.
 *   gemv_cols: outputs per apply GEMV task of the transposed (column dot
 *     product) form, 32 or 64 (single precision; double precision uses 32).
 *   tc_min_dim: a product goes to the tensor cores (128 x 128 tiles) only
 *     when both dimensions of its output block are at least this, else to
 *     64 x 64 CUDA-core tiles (small blocks would leave most of a tensor-core
 *     tile empty); 1..4096.
 * Defaults: 4096, 32768, 512, 1, 32, 64.                                     */
typedef struct {
  int gemv_min_elems;
  int gemv_max_elems;
  int front_small;
  int tensor_cores;
  int gemv_cols;
  int tc_min_dim;
} sgf_tuning;

/* Current tuning of a plan (INVALID_ARG on NULL). */
int sgf_plan_get_tuning(const sgf_plan* plan, sgf_tuning* out);
/* Replace the tuning of a plan; INVALID_ARG (plan unchanged) when a field is
 * outside the ranges above.  Factors made before keep their launch shapes.  */
int sgf_plan_set_tuning(sgf_plan* plan, const sgf_tuning* t);
/* Autotuner: searches the launch shapes with CUDA events on `stream`, after
 * one untimed warm-up factorization of coeffs_dev.  First, in single
 * precision, front_small (512, 256) x tc_min_dim (32, 64, 128) with the
 * plan's tensor-core mode (1 when it is 0), each timed as the faster of two
 * sgf_factor calls; then, with the fastest of those, five GEMV
 * budgets (4K-32K, 8K-64K, 16K-128K, 32K-128K, 32K-256K elements per task),
 * in single precision each with gemv_cols 32 and 64, each timed on napply
 * applications of A_l^{-1} to a fixed vector (skipped
 * when napply = 0: the budgets stay as they were).  The two groups are
 * independent (the first changes only the factorization, the second only
 * the apply).  Keeps the result in the plan, writes it to *best and the sum
 * of the two best times (ms) to *best_ms when not NULL.  Allocates and frees
 * device memory; synchronizes the stream.  Errors: those of sgf_factor; on
 * error the plan keeps its previous tuning.                                 */
int sgf_autotune(sgf_plan* plan, const double* coeffs_dev, void* stream, int napply, sgf_tuning* best,
                 double* best_ms);

/* ---- numeric factorization ----------------------------------------------
 * sgf_factor: Algorithm 4.1 on the device.  coeffs_dev holds one FP64
 * coefficient per cell (natural order).  Per level: batched elimination of
 * the interiors (Eq. (elimination)), compression of the selected separators
 * (Sec. 3.2: scaling, filtered interaction matrix Eq. (N-definition),
 * column-pivoted QR Eq. (QR), rank, Eq. (M') and Eq. (phi-update)), merge
 * into the next level (Sec. 4.3-4.4), then the top Cholesky (Sec. 4.5).
 * Synchronizes the stream once per level to read the numeric ranks.
 * Errors: NOT_SPD / NONFINITE (bad pivot; the node is reported by
 * sgf_factor_status), OOM, CUDA.  On error *out is NULL.                   */
int sgf_factor(const sgf_plan* plan, const double* coeffs_dev, void* stream, sgf_factor_t** out);
void sgf_factor_destroy(sgf_factor_t* f);

/* Per-level statistics: for `level`, the number of compressed separators,
 * the summed node sizes before and after compression, and the factor bytes. */
int sgf_factor_level_stats(const sgf_factor_t* f, int level, int* ncompressed,
                           int64_t* size_before, int64_t* size_after, int64_t* bytes);
/* Ranks of the level's nodes: m[i] (size when compressed) and r[i] (kept
 * rank, = m[i] when the node was not compressed).  Arrays of nnodes ints.   */
int sgf_factor_ranks(const sgf_factor_t* f, int level, int* m, int* r);
/* Last device status: node index of a failed pivot (or -1) and status.     */
int sgf_factor_status(const sgf_factor_t* f, int* bad_level, int* bad_node);
/* Precision the factor holds: SGF_PREC_FP64 or SGF_PREC_MIXED.  A mixed
 * request whose FP32 factorization met a non-positive or non-finite pivot is
 * factored again entirely in FP64 (the mixed-precision policy: CG then runs
 * on an FP64 preconditioner); it reports SGF_PREC_FP64.  -1 on NULL.       */
int sgf_factor_precision(const sgf_factor_t* f);

/* ---- apply (Sec. 4.7) and products ----------------------------------------
 * y = A_l^{-1} x (sgf_apply) or y = A_l x (sgf_apply_forward); nrhs vectors,
 * natural order, FP64 in and out.  x and y may not alias.                   */
int sgf_apply(const sgf_factor_t* f, const double* x_dev, double* y_dev, int nrhs, void* stream);
int sgf_apply_forward(const sgf_factor_t* f, const double* x_dev, double* y_dev, int nrhs,
                      void* stream);
/* y = A x with the assembled operator (FP64 stencil SpMV).                  */
int sgf_spmv(const sgf_factor_t* f, const double* x_dev, double* y_dev, int nrhs, void* stream);

/* ---- PCG (Sec. 7) -----------------------------------------------------------
 * Solves A x = b with CG preconditioned by A_l^{-1}, x0 = 0, until
 * ||r||_2 <= rtol ||b||_2 (recursive residual) or maxit.  The residual,
 * SpMV and dot products are FP64; with a mixed-precision factor the beta is
 * the flexible (Polak-Ribiere) one.  Synchronizes the stream.  info (may be
 * NULL) receives iterations, the true relative residual ||b - A x|| / ||b||
 * and the device time.  Returns NO_CONVERGENCE when maxit was reached.      */
typedef struct sgf_solve_info {
  int iterations;      /* max over right-hand sides                          */
  double rel_residual; /* max over right-hand sides                          */
  double seconds;      /* time of the solve: device time (CUDA events) for   */
                       /* sgf_pcg_solve, host wall time for                  */
                       /* sgf_pcg_solve_noalloc                              */
} sgf_solve_info;

int sgf_pcg_solve(const sgf_factor_t* f, const double* b_dev, double* x_dev, int nrhs,
                  double rtol, int maxit, void* stream, sgf_solve_info* info);

/* ---- allocation-free PCG ---------------------------------------------------
 * sgf_pcg_solve_noalloc: the PCG of sgf_pcg_solve (one right-hand side) for
 * callers that cannot let the library allocate device memory while solving:
 * a process that reserves its whole memory budget up front and treats any
 * later cudaMalloc as a violation, code that owns all device memory through
 * its own arena, or a latency-critical loop that cannot afford an allocator
 * call.  The paper has no counterpart; this is a deployment interface.
 * Its work vectors and dot-product partial sums live in one fixed device
 * array of 5 * SGF_NOALLOC_MAX_UNKNOWNS + 368 doubles (about 10 MiB) that
 * every GPU loading the library keeps until the process exits; factors with
 * more than SGF_NOALLOC_MAX_UNKNOWNS unknowns are rejected with
 * SGF_ERR_INVALID_ARG, and so is a call whose current device is not the
 * factor's.  It calls no allocator: sgf_factor builds and instantiates the
 * single-RHS apply graph this solve replays, so nothing is captured or
 * instantiated here either (sgf_memory_stats shows no new allocation event
 * across a call).  The first call on a device looks up the array's device
 * address (once per device, with that device current): make that first
 * call before any stream capture.  Every call shares the one array and
 * writes each word it reads, so nothing carries over between calls, but
 * calls that overlap on the GPU (other streams or threads) race on it and
 * must not be issued.  Synchronizes the stream; info->seconds is host wall
 * time.                                                                    */
#define SGF_NOALLOC_MAX_UNKNOWNS 262144
int sgf_pcg_solve_noalloc(const sgf_factor_t* f, const double* b_dev, double* x_dev, double rtol,
                          int maxit, void* stream, sgf_solve_info* info);

/* Host-buffer convenience path: copies coeffs/b from host memory, factors,
 * solves and copies x back (the end-to-end call of the serving loop).      */
int sgf_solve_host(const sgf_plan* plan, const double* coeffs_host, const double* b_host,
                   double* x_host, int nrhs, double rtol, int maxit, void* stream,
                   sgf_solve_info* info);

/* ---- asynchronous status ---------------------------------------------------
 * sgf_sync: waits for the current device (the factor's; INVALID_ARG when
 * another device is current) and surfaces what the asynchronous work issued
 * for this factor found (Sec. 4.7 applies and products are enqueued and
 * return before the device has run them): SGF_ERR_CUDA for a sticky CUDA
 * error, the factorization's pivot status (NOT_SPD / NONFINITE), then
 * SGF_ERR_NONFINITE when an sgf_apply or sgf_apply_forward since the last
 * sgf_sync wrote a NaN or infinity into its output (that flag is cleared by
 * this call), else SGF_OK.  The check is folded into the final copy of every
 * apply and multiply, so it costs no extra pass over the vectors.          */
int sgf_sync(const sgf_factor_t* f);

/* Device-memory accounting: *alloc_events (may be NULL) = how many times
 * this library has asked the CUDA runtime or driver for device memory since
 * the process started (cudaMalloc, stream-ordered allocations, stream
 * creation and graph instantiation each count one); *pool_used_bytes (may be
 * NULL) = bytes in use from the current device's default stream-ordered pool
 * (every user of that pool counted).  Host only, no synchronization.       */
int sgf_memory_stats(int64_t* alloc_events, int64_t* pool_used_bytes);

const char* sgf_status_string(int status);
/* Human-readable message of the last failed call on the calling thread.   */
const char* sgf_last_error(void);

/* Host-only validation mode.  With SGF_DRY_RUN=1 in the environment,
 * sgf_factor / sgf_apply / sgf_apply_forward make no CUDA call: device
 * allocations become address ranges in a table and every batched task is
 * checked to read and write inside one allocation instead of being launched
 * (numeric ranks are replaced by a deterministic stand-in).  These two calls
 * report what the checks found: the number of out-of-range accesses since
 * the last reset (reset != 0 clears it) and a text log of the first ones.  */
int64_t sgf_dry_run_violations(int reset);
const char* sgf_dry_run_report(void);

/* Device memory.  Factors, their apply programs and solver work buffers are
 * allocated from the current device's default stream-ordered pool, which
 * keeps blocks freed by sgf_factor_destroy cached for the next factorization
 * (no driver allocation or unmapping per factorization).  The cache counts
 * as used memory for other allocators in the process (e.g. PyTorch's);
 * sgf_release_cached_memory synchronizes the current device and hands the
 * unused cached blocks back.  An allocation of this library that fails does
 * the same once before it reports SGF_ERR_OOM.  Returns SGF_OK or
 * SGF_ERR_CUDA.                                                           */
int sgf_release_cached_memory(void);

/* Launch accounting for benchmarks.  Kinds 0..11 are named by
 * sgf_profile_kind_name (k_gemm, k_diag, k_copy, k_qrcp, k_gemv_n, k_gemv_t,
 * k_veccopy, k_assemble, k_spmv, k_dot, k_vector, apply); "apply" is one
 * replay of the graph that applies A_l^{-1} (Sec. 4.7), whose kernels are
 * also counted, untimed, under their own kinds.  sgf_profile_reset clears
 * the counters; with timing = 1 every later launch is bracketed by CUDA
 * events on its own stream, with timing = 2 only the factor's contraction
 * launches (k_gemm, k_diag, k_qrcp) and the apply replays (far fewer, so the
 * events barely perturb a timed step), with 0 none.  sgf_profile_read (synchronizes on the recorded
 * events) returns, for one kind, the launches since the reset, their summed
 * device time in ms (0 without timing) and the algorithmic flops and bytes
 * the host attached to them.  Not thread-safe with concurrent factors.      */
void sgf_profile_reset(int timing);
int sgf_profile_read(int kind, int64_t* launches, double* ms, double* flops, double* bytes);
const char* sgf_profile_kind_name(int kind);

#ifdef __cplusplus
}
#endif
#endif /* SGF_H_ */
