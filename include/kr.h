/*
 * kr.h -- C interface of the GB300 simultaneous short-recurrence Krylov solvers.
 *
 * Solves A X = B for a sparse non-Hermitian A in C^{n x n} and s right-hand sides
 * B in C^{n x s} with the simultaneous methods of Rashedi, Birk, Frommer, Ebadi,
 * "On short recurrence Krylov type methods for linear systems with many
 * right-hand sides" (Sec. 1 states the problem; Secs. 2 and 4 the methods).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Complex numbers are (re, im) pairs of doubles.  An n x s block is n*s
 * consecutive pairs, row i holding the s entries of unknown i (row-interleaved:
 * the storage of a C-contiguous (n, s) complex128 array).  An n-vector is n
 * consecutive pairs.  Device pointers must be 16-byte aligned.
 *
 * Every function returns a kr_status; 0 is success.  On any non-zero return a
 * human-readable message is available from kr_last_error() (thread-local).
 * Nothing is thrown across the interface and no call traps or aborts.
 *
 * `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 * enqueued on it; kr_solve and kr_adjoint_solve additionally synchronise with it
 * to read the convergence state.  The library is not re-entrant for one kr_op:
 * do not run two calls on the same operator concurrently.
 *
 * Ownership: the library owns an operator's device copies of A and A^H and the
 * solver workspace cached inside the operator (allocated at the first solve for
 * a given s and precision, freed by kr_op_destroy).  The caller owns every
 * B, X, G, Lambda, V, Y and output buffer passed in.
 */
#ifndef KR_H_
#define KR_H_

#include <stdint.h>

#if defined(__GNUC__)
#define KR_API __attribute__((visibility("default")))
#else
#define KR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KR_OK = 0,          /* converged: ||R_k||_F <= tol * ||R_0||_F (or call succeeded) */
  KR_BREAKDOWN = 1,   /* a scalar denominator vanished or an s x s matrix was singular (Sec. 2) */
  KR_DIVERGED = 2,    /* relative residual above 1e8, or above 1 at the end ("div." in Table 2) */
  KR_NAN = 3,         /* a non-finite value appeared */
  KR_MAXIT = 4,       /* iteration limit reached */
  KR_TIMEOUT = 5,     /* wall-clock limit reached */
  KR_BAD_ARG = 6,     /* invalid argument (size, pointer, method) */
  KR_OOM = 7,         /* device allocation failed */
  KR_CUDA_ERROR = 8,  /* a CUDA call failed */
  KR_UNSUPPORTED = 9  /* combination not supported (e.g. s > 32) */
} kr_status;

typedef enum {
  KR_BL_BICG = 0,         /* Bl-BiCG, Algorithm 3 (Sec. 2) */
  KR_BL_BICG_RQ = 1,      /* Bl-BiCG-rQ, Algorithm 5 (Sec. 4) */
  KR_GL_BICG = 2,         /* Gl-BiCG, Algorithm 2 (Sec. 2) */
  KR_EGL_BICG = 3,        /* eGl-BiCG, Algorithm 4 (Sec. 4) */
  KR_BL_BICGSTAB = 4,     /* Bl-BiCGStab (Sec. 2; El Guennouni-Jbilou-Sadok) */
  KR_BL_BICGSTAB_RQ = 5,  /* Bl-BiCGStab-rQ (Sec. 4, last remark) */
  KR_GL_BICGSTAB = 6,     /* Gl-BiCGStab (Sec. 2, global principle) */
  KR_BL_QMR = 7,          /* Bl-QMR with block products, no look-ahead (Sec. 2) */
  KR_GL_QMR = 8,          /* Gl-QMR (Sec. 2, global principle) */
  KR_EGL_QMR = 9,         /* eGl-QMR (Sec. 4) */
  KR_LI_BICG = 10,        /* Li-BiCG, Algorithm 1 (Sec. 2) */
  KR_LI_BICGSTAB = 11,    /* Li-BiCGStab: loop interchange (Sec. 2) applied to BiCGStab */
  KR_LI_QMR = 12          /* Li-QMR: loop interchange (Sec. 2) applied to QMR (no look-ahead) */
} kr_method;

typedef enum {
  KR_FP64 = 0,        /* complex128 everywhere */
  KR_FP32_REFINE = 1  /* complex64 inner solves inside an FP64 defect-correction loop */
} kr_precision;

typedef enum {
  KR_SHADOW_DEFAULT = 0, /* R^_0 = R_0 (block, global, Li), r^_0 = mean of R_0's columns (economic): Sec. 5 */
  KR_SHADOW_CONJ = 1,    /* R^_0 = conj(R_0) (Sec. 4) */
  KR_SHADOW_USER = 2     /* kr_options.shadow holds R^_0 (n x s) or r^_0 (n-vector, economic methods) */
} kr_shadow;

typedef struct kr_op_s* kr_op;

typedef struct {
  double tol;             /* relative tolerance on ||R||_F / ||R_0||_F (Sec. 5 uses 1e-10) */
  int32_t maxit;          /* iteration limit (Sec. 5: 500, 1200 for Example 5) */
  int32_t precision;      /* kr_precision */
  double inner_tol;       /* KR_FP32_REFINE: relative tolerance of each inner complex64 solve */
  int32_t max_outer;      /* KR_FP32_REFINE: limit on defect-correction steps (0 = 30) */
  int32_t shadow_mode;    /* kr_shadow */
  const double* shadow;   /* KR_SHADOW_USER: device pointer, layout as B (or an n-vector) */
  int32_t check_every;    /* read the convergence state back every this many iterations (0 = 8) */
  int32_t host_buffers;   /* 1: B and X are host pointers (copied to and from the device inside the call) */
  double* history;        /* optional host array of maxit+1 doubles: ||R_k||_F / ||R_0||_F, k = 0..iters */
  double time_limit_s;    /* optional wall-clock limit (0 = none) -> KR_TIMEOUT */
  int32_t graphs;         /* CUDA-graph replay of the iterations: 0 = automatic (on when n*s <= 2^22,
                             where kernel launches rather than kernels take the time, and whenever a
                             preconditioner is set), 1 = on, 2 = off.
                             Two iterations are captured once and replayed until convergence; the
                             results are bitwise those of the eager launches.  Off while the launch
                             profile times kernels. */
  int32_t orthonormalize_B; /* 1: the set-up of Sec. 5, right-hand sides replaced by the orthonormal
                             factor of a thin QR: R_0 = B - A X_0 = Q S (Q^H Q = I, S upper triangular
                             with real positive diagonal), the method solves A Y = Q from Y = 0 and
                             X = X_0 + Y S is returned.  tol, history and relres_recursive refer to
                             the system with Q; relres_true to the caller's system.  KR_BREAKDOWN
                             (breakdown_iter 1) when R_0 is numerically rank deficient.  Not with a
                             preconditioner (KR_UNSUPPORTED).  0 (default): B as given. */
  int32_t deterministic;  /* 0 or 1.  Every reduction of the library sums its per-CTA partial sums in
                             a fixed order over a grid fixed by (n, s, device), so results are bitwise
                             reproducible on a given device with either value; the field records the
                             caller's requirement and rejects other values (KR_BAD_ARG). */
  int32_t reserved;
} kr_options;

typedef struct {
  int32_t iters;            /* iterations performed (inner iterations summed for KR_FP32_REFINE) */
  int32_t matvecs;          /* single-vector matrix products (2s per Bl/Gl BiCG or QMR iteration) */
  double relres_recursive;  /* last recursively updated ||R||_F / ||R_0||_F (||C||_F for -rQ) */
  double relres_true;       /* ||B - A X||_F / ||R_0||_F recomputed in FP64 at exit */
  int32_t status;           /* kr_status of the iteration */
  int32_t outer_iters;      /* KR_FP32_REFINE: defect-correction steps */
  int32_t fp64_iters;       /* KR_FP32_REFINE: iterations of the FP64 solve that finishes the job when a
                               complex64 inner solve failed to reduce the FP64 residual (0: none) */
  int32_t breakdown_iter;   /* status KR_BREAKDOWN: the iteration (1-based; iters + 1) whose scalar
                               denominator vanished or whose s x s matrix was singular (Secs. 2, 4);
                               X and the residuals are those after iters iterations.  0 otherwise */
} kr_info;

/* Fill *opt with defaults: tol 1e-8, maxit 500, FP64, default shadow, check_every 8,
 * B as given (orthonormalize_B 0), deterministic 1. */
KR_API void kr_options_default(kr_options* opt);

/* Build an operator from a CSR matrix (Sec. 1: A sparse, used only through
 * matrix-block-vector products A V and A^H W).
 *   n, nnz        : order and number of stored entries;
 *   rowptr[n+1]   : int64 row offsets (host), rowptr[0] = 0, rowptr[n] = nnz;
 *   colidx[nnz]   : int32 column indices (host), each in [0, n);
 *   vals[2*nnz]   : interleaved (re, im) entries (host);
 *   device        : CUDA device ordinal that will hold the operator.
 * The library copies the arrays (the caller keeps ownership), builds A^H as an
 * explicit CSR, and stores real off-diagonal entries in real form when every
 * off-diagonal entry has a zero imaginary part.  Returns KR_BAD_ARG for
 * malformed CSR (checked on the host), KR_OOM when device memory runs out. */
KR_API kr_status kr_op_create_csr(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                           const double* vals, int32_t device, kr_op* out);

/* kr_op_create_csr for arrays that may live on the device: with on_device != 0, rowptr,
 * colidx and vals are device pointers of the device that `stream` belongs to (the current
 * device when stream is NULL), copied on `stream` (the call waits for the copies); with
 * on_device == 0 they are host pointers and the operator is built on the current device.
 * The caller keeps ownership.  Validation, the explicit A^H and the storage choice are those
 * of kr_op_create_csr (made on the host from the copied arrays); errors as there. */
KR_API kr_status kr_op_create_csr_async(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                        const double* vals, int32_t on_device, void* stream, kr_op* out);

/* Matrix-free operator of a (2d+1)-point stencil on a d-dimensional grid (d = 1, 2, 3)
 * with Dirichlet boundaries (the convection-diffusion discretisations of Sec. 5,
 * Examples 1-3): unknown i = x_0 + N_0 x_1 + N_0 N_1 x_2 and
 *   (A v)_i = c v_i + sum_a ( m_a v_{i - st_a} [x_a > 0] + p_a v_{i + st_a} [x_a < N_a - 1] ),
 * st_a = N_0 ... N_{a-1}.  dims[d]: grid extents; coeffs[2 + 4d]: (re, im) of c, then for
 * each axis a the pairs m_a, p_a.  No matrix is stored: a product reads only the
 * vectors.  A^H uses the conjugated, mirrored coefficients.  kr_grad_values and
 * kr_op_update_values need a CSR operator and return KR_UNSUPPORTED here. */
KR_API kr_status kr_op_create_stencil(int32_t dim, const int64_t* dims, const double* coeffs, int32_t device,
                                      kr_op* out);

/* Matrix-free 4D lattice operator (Sec. 5, Example 4: a Wilson-type nearest-neighbour
 * operator, 12 unknowns per site).  Sites x = x_0 + L_0 x_1 + L_0 L_1 x_2 + L_0 L_1 L_2 x_3
 * on a periodic lattice, unknown (x * 4 + spin) * 3 + colour, and
 *   (A v)_x = d v_x + hop * sum_mu [ (I - gamma_mu) (x) U_mu(x) v_{x+mu}
 *                                    + (I + gamma_mu) (x) U_mu(x-mu)^H v_{x-mu} ].
 * dims[4]: extents L_mu (each >= 3); diag[2]: (re, im) of d; hop: real coefficient;
 * gamma[4*4*4*2]: the four 4 x 4 matrices gamma_mu, row-major, interleaved (re, im), each
 * Hermitian with exactly one entry of modulus 1 per row, off the diagonal (a chiral
 * basis; checked on the host); links[4*sites*9*2]: host array of the 3 x 3 link matrices
 * U_mu(x), row-major, interleaved, indexed [mu][x].  The caller's arrays are copied.
 * A product reads the vectors and the links only; each neighbour spinor is projected on
 * the two independent spin components of (I -+ gamma_mu) before the link multiplies it.
 * A^H is the same form with gamma_mu -> -gamma_mu and d -> conj(d).  kr_op_info reports
 * nnz = 49 n (the entries of the equivalent sparse matrix).  kr_grad_values and
 * kr_op_update_values return KR_UNSUPPORTED. */
KR_API kr_status kr_op_create_lattice4d(const int64_t* dims, const double* diag, double hop, const double* gamma,
                                        const double* links, int32_t device, kr_op* out);

/* Preconditioners (kr_op_set_preconditioner). */
typedef enum {
  KR_PREC_NONE = 0,
  KR_PREC_ILU0 = 1  /* incomplete LU without fill-in (Sec. 5, second set of experiments) */
} kr_preconditioner;

/* Set (or with KR_PREC_NONE remove) a right preconditioner of a CSR operator: later kr_solve
 * calls solve A M^{-1} Y = B - A X_0 from Y = 0 and return X = X_0 + M^{-1} Y, with every
 * iteration's products A M^{-1} V and M^{-H} A^H W (the methods are unchanged; the reported
 * residuals are those of the original system).  ILU(0): M = L U, L unit lower and U upper
 * triangular with the sparsity pattern of A and (L U)_ij = A_ij on it, factorised once in
 * FP64 on the host; each triangular solve is level-scheduled (one launch per level of row
 * dependencies).  Requires every diagonal entry stored; KR_BREAKDOWN on a zero pivot;
 * KR_UNSUPPORTED for matrix-free operators.  kr_adjoint_solve and KR_FP32_REFINE return
 * KR_UNSUPPORTED while a preconditioner is set.  kr_op_update_values removes it. */
KR_API kr_status kr_op_set_preconditioner(kr_op op, int32_t kind);

/* Y = M^{-1} V (adjoint = 0) or M^{-H} V (adjoint = 1) with the operator's preconditioner;
 * V, Y: device n x s complex128 blocks (Y may equal V). */
KR_API kr_status kr_op_apply_precond(kr_op op, int32_t adjoint, int32_t s, const double* V, double* Y,
                                     void* stream);

/* Replace the stored entries of A (same sparsity pattern, same order as given to
 * kr_op_create_csr): vals[2*nnz] interleaved (re, im), a host pointer
 * (on_device = 0) or a device pointer (on_device != 0).  A^H, the real/complex
 * storage choice and the complex64 copy are rebuilt; cached workspace is kept.
 * Used when A depends on parameters that are being optimised (differentiation
 * through the solve). */
KR_API kr_status kr_op_update_values(kr_op op, const double* vals, int32_t on_device);

/* Release the operator, its device arrays and its cached workspace.  NULL is accepted. */
KR_API kr_status kr_op_destroy(kr_op op);

/* Order, stored entries, and whether the real-off-diagonal storage is in use. */
KR_API kr_status kr_op_info(kr_op op, int64_t* n, int64_t* nnz, int32_t* real_offdiag);

/* Matrix-block-vector product (Sec. 1; Algorithms 1-5, first line of the loop):
 * Y = A V (adjoint = 0) or Y = A^H V (adjoint = 1), V and Y device n x s blocks,
 * 1 <= s <= 32, V and Y must not overlap. */
KR_API kr_status kr_op_apply(kr_op op, int32_t adjoint, int32_t s, const double* V, double* Y, void* stream);

/* Reduction kinds of kr_op_apply_reduce and kr_block_reduce. */
typedef enum {
  KR_RED_GRAM = 1,   /* s x s  U^H Y  (Algorithm 3: (Ph^H Q), Algorithm 5: (Vh^H W)) */
  KR_RED_TRACE = 2,  /* 1      tr(U^H Y)  (Algorithm 2) */
  KR_RED_SUMV = 3,   /* 1      sum(u^H Y), u an n-vector (Algorithm 4) */
  KR_RED_NORM2 = 4   /* 1      ||Y||_F^2 (U ignored; result in the real part) */
} kr_reduction;

/* Block product fused with one reduction of its output: Y = op(A) V and
 * out = reduce(U, Y).  Y may be NULL (product not stored).  U is a device n x s
 * block (GRAM, TRACE) or n-vector (SUMV).  out is a device array of s*s (GRAM)
 * or 1 complex entries, row-major.  Summation order is fixed: repeated calls
 * give bitwise identical results. */
KR_API kr_status kr_op_apply_reduce(kr_op op, int32_t adjoint, int32_t s, const double* V, double* Y, const double* U,
                             int32_t kind, double* out, void* stream);

/* Stand-alone reduction of two device blocks: out = reduce(U, Y) as above. */
KR_API kr_status kr_block_reduce(int64_t n, int32_t s, const double* U, const double* Y, int32_t kind, double* out,
                          void* stream);

/* Complex64 variants of kr_op_apply_reduce and kr_block_reduce: the product and
 * reduction kernels of the complex64 inner solves of KR_FP32_REFINE, exposed for
 * testing and for callers that keep their blocks in complex64.  V, Y and U are device
 * n x s complex64 blocks (interleaved float re, im; U an n-vector for SUMV); the
 * products and the per-CTA partial sums are formed in FP32, the partial sums are added
 * in FP64 and out is complex128 (s*s or 1 entries, as above).  kind == 0 in
 * kr_op_apply_reduce_c64 is a plain product (Y required).  The first complex64 call on
 * a CSR operator uploads its complex64 copy (kept until kr_op_destroy). */
KR_API kr_status kr_op_apply_reduce_c64(kr_op op, int32_t adjoint, int32_t s, const float* V, float* Y,
                                        const float* U, int32_t kind, double* out, void* stream);
KR_API kr_status kr_block_reduce_c64(int64_t n, int32_t s, const float* U, const float* Y, int32_t kind,
                                     double* out, void* stream);

/* The reduction of kr_block_reduce without any device allocation by the library,
 * for callers that cannot let a library allocate device memory (an application
 * whose own pool allocator owns all device memory, or a latency-critical loop
 * that cannot afford cudaMalloc's possible device synchronisation).  The paper
 * has no counterpart: this is an interface variant, not a step of the method.
 * Arguments and result as kr_block_reduce; out is caller-owned device memory.
 * Limit: 1 <= s <= 16, otherwise KR_UNSUPPORTED before any GPU work.  The
 * scratch (per-CTA partial sums) is a 1 MiB statically sized device array held
 * by every GPU that loads the library until process exit.  The call runs on the
 * device that holds Y (made current for the call, the previous device restored);
 * U, out and a non-null stream on another device give KR_BAD_ARG.  The array's
 * device address is looked up on every call made outside a stream capture; a call
 * made while its stream is being captured reuses the address of the last
 * uncaptured call on that device, so call once on each device before capturing.
 * The grid is capped at 256 CTAs, so for large n the result agrees with
 * kr_block_reduce to rounding, not bitwise.  All calls share the array (each
 * fully overwrites what it reads, so nothing needs clearing); calls whose GPU work
 * overlaps race on it. */
KR_API kr_status kr_block_reduce_noalloc(int64_t n, int32_t s, const double* U, const double* Y, int32_t kind,
                                         double* out, void* stream);

/* Thin QR of a device n x s block (Sec. 4, Eq. (QR)): Z = Q S, Q^H Q = I, S upper
 * triangular with real positive diagonal (CholQR2, shifted first pass when the
 * Gram matrix is not numerically positive definite).  Q (device n x s, may equal
 * Z) and S (device s x s, row-major) are written.  KR_BREAKDOWN if Z is
 * numerically rank deficient. */
KR_API kr_status kr_thin_qr(int64_t n, int32_t s, const double* Z, double* Q, double* S, void* stream);

/* Solve A X = B with `method` (kr_method) for s right-hand sides, 1 <= s <= 32.
 * B, X: n x s blocks; device pointers unless opt->host_buffers.  X holds the
 * initial guess X_0 on entry (the paper uses X_0 = 0, Sec. 5) and the final
 * iterate on return.  opt may be NULL (defaults).  info may be NULL.
 * The return value is the iteration status (KR_OK when converged) or an error. */
KR_API kr_status kr_solve(kr_op op, int32_t method, int32_t s, const double* B, double* X, const kr_options* opt,
                   void* stream, kr_info* info);

/* Solve the adjoint system A^H Lambda = G with the same simultaneous methods
 * (roles of A and A^H exchanged); arguments as kr_solve.  Used by reverse-mode
 * differentiation: for L(X) with X = A^{-1} B, dL/dB = Lambda where
 * A^H Lambda = dL/dX. */
KR_API kr_status kr_adjoint_solve(kr_op op, int32_t method, int32_t s, const double* G, double* Lambda,
                           const kr_options* opt, void* stream, kr_info* info);

/* Gradient with respect to the stored entries of A for X = A^{-1} B and
 * Lambda = A^{-H} dL/dX:  dL/dA_ij = - sum_c Lambda_ic conj(X_jc) for every stored
 * (i, j), written as nnz complex values in the order of the CSR given to
 * kr_op_create_csr (device pointers, dvals of 2*nnz doubles). */
KR_API kr_status kr_grad_values(kr_op op, int32_t s, const double* Lambda, const double* X, double* dvals, void* stream);

/* Kernel classes of the launch profile. */
typedef enum {
  KR_K_SPMM = 0,     /* block sparse products A V, A^H W with fused reductions */
  KR_K_LINCOMB = 1,  /* row-local block updates with fused reductions */
  KR_K_REDUCE = 2,   /* fixed-order sums of per-CTA partial reductions */
  KR_K_COEF = 3,     /* one-CTA FP64 coefficient algebra (s x s solves, QR factors, rotations) */
  KR_K_OTHER = 4,    /* precision conversions, gradient */
  KR_K_SPMM_C64 = 5,     /* block sparse products in complex64 (mixed-precision inner solves) */
  KR_K_LINCOMB_C64 = 6,  /* row-local block updates in complex64 */
  KR_K_CLASSES = 7
} kr_kernel_class;

typedef struct {
  int64_t launches[8];  /* kernel launches per class since the last reset */
  double ms[8];         /* summed CUDA-event durations per class (when timing is on) */
  double flops[8];      /* algorithmic floating-point operations per class */
  double bytes[8];      /* algorithmic DRAM bytes per class (each operand read or written once) */
} kr_profile;

/* Turn launch counting on or off (process-wide, default off).  With
 * time_kernels != 0 every launch is bracketed by CUDA events on its stream and
 * the durations are summed when kr_profile_read is called (which synchronises
 * with the recorded events).  Profiling adds no kernels of its own. */
KR_API kr_status kr_profile_enable(int32_t enable, int32_t time_kernels);

/* Copy the counters into *out; reset them when reset != 0. */
KR_API kr_status kr_profile_read(kr_profile* out, int32_t reset);

/* Kernel choice for complex64 blocks (the inner solves of KR_FP32_REFINE); the paper
 * has no counterpart.  With enable != 0 (the default), complex64 launches with even s
 * and no s x s Gram or s x s coefficient matrix run on kernels in which one thread owns
 * two adjacent columns of a row (16-byte loads and stores); enable == 0 keeps every
 * launch on the one-column kernels.  Both compute each output entry with the same
 * operations in the same order; only the grouping of the fused reductions' partial sums
 * differs.  Process-wide; takes effect for launches issued after the call.  Always
 * returns KR_OK. */
KR_API kr_status kr_set_column_pairs(int32_t enable);

/* Kernel choice for staged complex64 products (the paper has no counterpart).  With enable != 0
 * (the default):
 *  - complex64 products of a CSR operator with s in {4, 8, 16, 32}, at most 1024 stored entries
 *    per tile of rows (128, 64, 32 or 16 rows for s = 4, 8, 16, 32), at most two fused s x s Grams and
 *    two distinct block operands of the fused reductions run on a kernel that stages each row
 *    tile's row pointers, diagonal, indices, values and reduction operands in shared memory with
 *    bulk asynchronous copies and forms the fused Grams from shared memory;
 *  - complex64 products of a matrix-free 2D or 3D stencil operator with s in {2, 4, 8, 16, 32}
 *    and at most one distinct block operand run on a kernel that marches the grid's planes
 *    through shared memory, one TMA tensor copy per halo'd plane of an x-y tile.
 * enable == 0 leaves them to the column-pair and one-column kernels (kr_set_column_pairs).
 * Products are bitwise the same on all of them; reductions agree to FP32 rounding.
 * Process-wide; always returns KR_OK. */
KR_API kr_status kr_set_tile_kernels(int32_t enable);

/* Schedule of Gl-BiCG (Algorithm 2) and eGl-BiCG (Algorithm 4); the paper has no counterpart.
 * With enable != 0 (the default), alpha's denominator tr(Ph^H A P) is taken as tr((A^H Ph)^H P),
 * a reduction of the direction update of P once A^H Ph is formed, and the update X += alpha P,
 * R -= alpha A P, Rh -= conj(alpha) A^H Ph runs in one pass, which for CSR operators without
 * preconditioner forms A P row by row without storing it (for the matrix-free lattice and with a
 * preconditioner A P is stored first).  The matrix-free stencil runs the algorithms' own order.
 * Per iteration that reads and writes 2M + 8 Bv instead of 2M + 11 Bv for eGl-BiCG and
 * 2M + 17 Bv instead of 2M + 19 Bv for Gl-BiCG (M: one read of A, Bv: one n x s block).  The
 * iterates are those of the algorithms in exact arithmetic; rounding differs.  enable == 0
 * runs the algorithms' own order.  Process-wide; always returns KR_OK. */
KR_API kr_status kr_set_fused_products(int32_t enable);

/* Number of bounded waits of the tile kernels (kr_set_tile_kernels) that ran out since the last
 * reset, for the current device.  A wait that runs out means the copies it waited for did not
 * arrive within about a second; the kernel then stops without computing the rest of its tiles and
 * writes NaN into its partial reductions, so the affected results are not silently wrong.  With
 * reset != 0 the counter is cleared.  KR_BAD_ARG if count is NULL. */
KR_API kr_status kr_take_device_timeouts(int32_t reset, int64_t* count);

/* Kernel choice for the matrix-free lattice product (kr_op_create_lattice4d); the paper
 * has no counterpart.  rows = 4: a thread forms the 4 rows of one (site, colour) pair of
 * one column (fewer registers, the spin projection repeated per colour); rows = 12: a
 * thread forms all 12 rows of a site (a quarter fewer flops, a third of the gathers, more
 * registers); rows = 0 (the default): 12, measured faster in both precisions.
 * Process-wide; returns KR_BAD_ARG for other values. */
KR_API kr_status kr_set_lattice_rows_per_thread(int32_t rows);

/* Arithmetic-throughput probe (a diagnostic; the paper has no counterpart): one launch of
 * 4 CTAs x 256 threads per SM, each thread running 16 independent FMA chains of `iters` steps
 * in FP64 (precision = KR_FP64) or FP32 (precision = 2), enqueued on `stream`.  *flops receives
 * the launch's floating-point operations (2 per FMA), so that the caller's CUDA-event time
 * gives the device's FMA rate: the denominator of the FP64 path's roofline.  out: device
 * buffer of one double (written by one thread).  KR_BAD_ARG for other arguments. */
KR_API kr_status kr_probe_fma(int32_t precision, int64_t iters, double* out, double* flops, void* stream);

/* Message describing the last failure on the calling thread ("" if none). */
KR_API const char* kr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KR_H_ */
