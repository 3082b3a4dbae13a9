/*
 * hmat.h -- C ABI of a GB300 (sm_103a) library for the H-matrix vector product
 * and the BiCG-STAB solve of a collocation BEM system, after Ooi, Iwashita,
 * Fukaya, Ida, Yokota, "Effect of Mixed Precision Computing on H-Matrix Vector
 * Multiplication in BEM Analysis" (arXiv:1911.00093).
 *
 * The operation (Section 2.1, eq. 5-10 and 21-25): y~ = A~ x, where A~ is a
 * block partition M of I x J (eq. 1-2) whose blocks are either dense A|^m or
 * low rank V_m W_m (eq. 3-4); a dense block adds A|^m x_m to y~ (eq. 21), a
 * low-rank block adds V_m (W_m x_m) (eq. 9-10, 22-24); every block's result
 * is scattered into y~ (eq. 7-8, 25).  The solver is BiCG-STAB (Algorithm 1),
 * accepted only when the true residual with the FP64 H-matrix meets the
 * tolerance (Section 4.1.3).
 *
 * Conventions for every function:
 *   - the return value is an hmat_status; 0 is success; no C++ exception
 *     crosses this interface;
 *   - vectors are FP64, length N, in the ORIGINAL panel order (the order of the
 *     builder's inputs); a block of nrhs vectors is column-major N x nrhs;
 *   - vector arguments may be device pointers (cudaMalloc, torch tensors) or
 *     host pointers (pageable or pinned); host data is staged through the
 *     handle's own device buffers and the call returns after the result is
 *     back in host memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is enqueued on it;
 *   - a handle is used by one host thread at a time.
 */
#ifndef HMAT_H
#define HMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hmat_status {
    HMAT_OK = 0,
    HMAT_ERR_ARG = 1,              /* null pointer, nrhs < 1, unknown precision, bad option    */
    HMAT_ERR_BAD_LAYOUT = 2,       /* blob fails validation (magic, sizes, cover of eq. 1-2)   */
    HMAT_ERR_NOMEM = 3,            /* host or device allocation failed                         */
    HMAT_ERR_CUDA = 4,             /* a CUDA runtime call failed (hmat_last_cuda_error)        */
    HMAT_ERR_BREAKDOWN_RHO = 5,    /* Algorithm 1: rho_{i-1} = r~^T r_{i-1} = 0 ("method fails") */
    HMAT_ERR_BREAKDOWN_OMEGA = 6,  /* Algorithm 1: omega_i = 0 prevents continuation           */
    HMAT_ERR_MAXIT = 7,            /* iteration or restart budget spent before the tolerance   */
    HMAT_ERR_NONFINITE = 8,        /* NaN/Inf in a residual norm or an input vector            */
    HMAT_ERR_RANGE = 9,            /* a panel value cannot be held by the precision form       */
    HMAT_ERR_UNSUPPORTED = 10,     /* valid request outside this build's limits (e.g. leaf>64) */
    HMAT_ERR_TIMEOUT = 11          /* a bounded wait inside a kernel ran out; the kernel gave up
                                      its work (the result of that product is not valid)        */
} hmat_status;

/*
 * Precision forms of the uploaded H-matrix.  Every form keeps y~ in FP64.
 *
 *  HMAT_FP64       FP64 panels (8 bytes per entry, stored as the exact pair
 *                  hi = fl32(a), lo = fl32(a - hi)); products and sums run in
 *                  double-float arithmetic (about 2^-48 relative) on the FP32
 *                  pipe.  Method 1-Double of Section 3.1 at FP64-class accuracy;
 *                  relative product error <= 1e-13 against an FP64 evaluation.
 *  HMAT_FP64_DFMA  IEEE FP64 panels and FP64 FMA arithmetic, literally Method
 *                  1-Double; on GB300 bound by the FP64 pipe, not by HBM.
 *  HMAT_FP32       FP32 panels, FP32 copy of the source vector (Section 3.5),
 *                  FP32 sums over chunks of 8 products, compensated (double-
 *                  float) sums across chunks, FP64 into y~; <= 1e-6 relative.
 *  HMAT_BF16       BF16 panels, each dense block and each low-rank factor
 *                  scaled by a power of two, FP32 source copy, FP32 chunk sums,
 *                  compensated sums across chunks, FP64 into y~; <= 1e-2
 *                  relative; meant to be wrapped in FP64 iterative refinement
 *                  (hmat_solve_opts.inner_tol).
 *
 * The four forms above store each array (dense block, V_m, W_m) divided by a
 * power of two (2^floor(log2 max|array|)), which is exact and undone on the fly.
 *
 * The paper's own variants (Section 3, Table 1), reproduced literally as
 * baselines: every operation Table 1 puts in FP64 runs in IEEE FP64 (multiply,
 * then add), every product of two FP32 operands is rounded to FP32, and the
 * source vector is rounded to FP32 where Table 1 says FP32 (Section 3.5).
 * Method 1-Double is HMAT_FP64_DFMA.
 *  HMAT_M1_SINGLE  FP32 A|^m, V_m, W_m; FP32 x; z_m accumulated in FP32;
 *                  y^_m in FP64 (Method 1-Single).
 *  HMAT_M1_MIXED   FP32 A|^m, V_m, W_m; FP64 x; z_m = fl32(z_m + W_m x) with the
 *                  right side in FP64; y^_m in FP64 (Method 1-Mixed).
 *  HMAT_M2_DOUBLE  V'_m D_m W'_m (eq. 11-16) in FP64 (Method 2-Double).
 *  HMAT_M2_SINGLE  FP32 A|^m, V'_m, W'_m, FP64 D_m; FP32 x; z_m in FP64
 *                  (Method 2-Single).
 *  HMAT_M2_MIXED   FP32 A|^m, V'_m, W'_m, FP64 D_m; FP64 x; z_m in FP64
 *                  (Method 2-Mixed).
 *  HMAT_M3         FP64 A|^m; rank i of a low-rank block in FP64 when
 *                  d_i >= d_max 10^-c, else in FP32 (eq. 17-20); the FP64 ranks
 *                  follow Method 2-Double, the FP32 ranks Method 2-Mixed, the two
 *                  parts are added (Section 3.4).  Upload with hmat_upload_ex.
 *  HMAT_M3_TRUNC   Section 4.5's alternative: the ranks Method 3 would store in
 *                  FP32 (d_i < d_max 10^-c) are deleted with their column of V'_m
 *                  and row of W'_m; the rest as Method 2-Double.  Upload with
 *                  hmat_upload_ex.
 *  HMAT_M3_DENSE   Section 4.5's multi-level dense blocks: column j of a dense
 *                  block stays FP64 when max_i |a_ij| >= d_max 10^-c, d_max the
 *                  largest entry of all dense blocks (Method 3's rule, eq. 19-20,
 *                  on the form A|^m = A|^m I); the other columns and every
 *                  low-rank block follow Method 2-Mixed; the parts are added.
 *                  c = -1 is Method 2-Mixed, c >= 2 keeps the collocation near
 *                  field all FP64.  Upload with hmat_upload_ex.
 * These variants carry FP64 arithmetic per entry and are bound by the FP64 pipe
 * of GB300, not by HBM.
 */
typedef enum hmat_precision {
    HMAT_FP64 = 0,
    HMAT_FP64_DFMA = 1,
    HMAT_FP32 = 2,
    HMAT_BF16 = 3,
    HMAT_M1_SINGLE = 4,
    HMAT_M1_MIXED = 5,
    HMAT_M2_DOUBLE = 6,
    HMAT_M2_SINGLE = 7,
    HMAT_M2_MIXED = 8,
    HMAT_M3 = 9,
    HMAT_M3_TRUNC = 10,
    HMAT_M3_DENSE = 11
} hmat_precision;

typedef struct hmat_t *hmat_handle;

/* ------------------------------------------------------------------------- */
/* Host builder: collocation BEM kernel -> serialized H-matrix ("blob")        */
/* ------------------------------------------------------------------------- */
/*
 * hmat_build -- build the FP64 H-matrix of the single-layer collocation matrix
 *   a_ij = area_j / (4 pi |c_i - c_j|)   (i != j),   a_ii = sqrt(area_i / pi) / 2
 * on n flat panels, on the host (the paper builds it with the HACApK library,
 * Section 4.1.3; this builder follows the same recipe):
 *   cluster tree  longest-axis bisection of the collocation points at the
 *                 bounding-box midpoint (points <= midpoint go left; an empty side
 *                 falls back to a median split in (coordinate, index) order);
 *                 clusters with <= leaf points are leaves;
 *   partition     (tau, sigma) is low rank iff dist(tau, sigma) > 0 and
 *                 min(diam tau, diam sigma) <= eta dist(tau, sigma) (boxes of the
 *                 collocation points); two leaves that fail it are dense; otherwise
 *                 every non-leaf side is split;
 *   low rank      ACA with partial pivoting to relative accuracy aca_eps; a block
 *                 whose factors are not smaller than the block is stored dense.
 * centroids: host, n x 3 row-major FP64 collocation points; areas: host, n FP64.
 * On success *blob receives a malloc'ed buffer of *blob_bytes bytes owned by the
 * caller (free it with hmat_blob_free).  Errors: HMAT_ERR_ARG (null, n < 1,
 * leaf < 1 or > 64, eta < 0, aca_eps <= 0, non-finite input), HMAT_ERR_NOMEM.
 * Uses OpenMP threads on the host; the result does not depend on their number.
 */
int hmat_build(int64_t n, const double *centroids, const double *areas, int32_t leaf, double eta,
               double aca_eps, void **blob, size_t *blob_bytes);

void hmat_blob_free(void *blob);

/*
 * hmat_build_device -- hmat_build with the entries computed on the current CUDA
 * device: the cluster tree and block partition are planned on the host, then one
 * CTA per admissible block runs the same ACA with partial pivoting and another
 * launch writes the dense blocks and the factors, which are copied into the host
 * blob.  Every floating-point operation is the host builder's in the same order
 * (no contraction; IEEE division and square root), so the blob equals
 * hmat_build's byte for byte.  A block whose ACA needs more than 64 ranks
 * without becoming dense is finished by the host builder's own code.  The
 * paper takes this step from HACApK on the CPU (Section 4.1.3); it is not on
 * the product's path.  Arguments, ownership and errors as hmat_build, plus
 * HMAT_ERR_CUDA; `info` (may be NULL) receives counts and host-clock times.
 * Synchronous; the device memory it uses is freed before it returns.
 */
typedef struct hmat_build_device_info {
    int64_t aca_blocks;        /* admissible blocks approximated on the device            */
    int64_t host_blocks;       /* of those, finished on the host (ranks above 64)        */
    int64_t workspace_bytes;   /* device workspace of the ACA (factors and pivot flags)  */
    double plan_ms;            /* host: cluster tree and block partition                 */
    double alloc_ms;           /* device buffers (ACA workspace) and input uploads        */
    double aca_ms;             /* the ACA launch, up to the ranks on the host             */
    double pack_ms;            /* block kinds, blob index, dense entries and factor pack  */
    double copy_ms;            /* the blob's values, device to host                      */
} hmat_build_device_info;

int hmat_build_device(int64_t n, const double *centroids, const double *areas, int32_t leaf, double eta,
                      double aca_eps, void **blob, size_t *blob_bytes, hmat_build_device_info *info);

/*
 * Serialized H-matrix, version 1 (all integers little-endian int64, all values
 * FP64; sections start on 64-byte boundaries; offsets are bytes from the start):
 *   header (256 bytes): magic "HMATBLB1", u32 version = 1, u32 header bytes = 256,
 *     n, nclusters, nblocks, ndata, leaf, eta (f64), aca_eps (f64), off_perm,
 *     off_clusters, off_blocks, off_data, total_bytes, dense_entries,
 *     lr_entries, rank_sum, rank_max, zero padding;
 *   perm[n]            perm[p] = original index of the p-th point of the cluster order;
 *   clusters[nc][4]    begin, end (a range of the cluster order), child0, child1 (-1 for
 *                      a leaf); cluster 0 is the root [0, n);
 *   blocks[nb][8]      i_s, i_e, j_s, j_e (ranges of the cluster order), kind (0 dense,
 *                      1 low rank), rank r, data offset (in values), 0;
 *   data[ndata]        dense block: A|^m, #I x #J row-major; low-rank block: V_m (#I x r
 *                      row-major) followed by W_m (r x #J row-major), eq. (3).
 */
typedef struct hmat_blob_stats {
    int64_t n, nclusters, nblocks, nleaves;
    int64_t dense_blocks, lr_blocks;
    int64_t dense_entries;   /* sum over dense blocks of #I #J       */
    int64_t lr_entries;      /* sum over low-rank blocks of r(#I+#J) */
    int64_t rank_sum, rank_max;
} hmat_blob_stats;

/* Validate a blob (the same checks as hmat_upload) and report its sizes. */
int hmat_blob_stats_get(const void *blob, size_t blob_bytes, hmat_blob_stats *out);

/*
 * hmat_form_stats_get -- what hmat_upload_ex would store for `precision` (and
 * Method 3's c), on the host only (no device is touched): the segments of a
 * paper variant (Table 1 / Section 4.5 derivation) or the one segment of a
 * GPU-native form, each packed and checked as at upload, with per-segment
 * counts.  Errors as hmat_upload_ex, without HMAT_ERR_CUDA / HMAT_ERR_NOMEM
 * from the device.
 */
typedef struct hmat_form_stats {
    int32_t segments;              /* 1 or 2                                                   */
    int32_t pad;
    int64_t blocks[2];             /* derived blocks per segment                               */
    int64_t dense_entries[2];      /* dense-block entries stored per segment                   */
    int64_t lr_ranks[2];           /* low-rank columns (ranks) stored per segment               */
    int64_t lr_entries[2];         /* low-rank factor entries stored per segment                */
    int64_t column_subsets[2];     /* dense blocks stored as column subsets per segment         */
    int64_t selected_operands[2];  /* entries of the operand selection lists per segment        */
} hmat_form_stats;
int hmat_form_stats_get(const void *blob, size_t blob_bytes, int32_t precision, int32_t method3_c,
                        hmat_form_stats *out);

/* ------------------------------------------------------------------------- */
/* Device H-matrix                                                            */
/* ------------------------------------------------------------------------- */
/*
 * hmat_upload -- validate `blob` (host memory, caller-owned, not retained),
 * convert its panels to `precision` on the host (Section 4.1.3: the FP64
 * H-matrix is generated first, then each submatrix is converted) and copy the
 * packed result to the current CUDA device.  Forms other than HMAT_FP64 and
 * HMAT_FP64_DFMA also keep an HMAT_FP64 copy for the true residual.  The handle
 * owns every device buffer it allocates.  The call is synchronous.
 * Errors: HMAT_ERR_ARG, HMAT_ERR_BAD_LAYOUT (bad magic/version/sizes, a non-
 * permutation, blocks that do not cover I x J exactly once, rank > min(#I,#J),
 * non-finite values), HMAT_ERR_UNSUPPORTED (a leaf with more than 64 points),
 * HMAT_ERR_RANGE, HMAT_ERR_NOMEM, HMAT_ERR_CUDA.
 */
int hmat_upload(const void *blob, size_t blob_bytes, int32_t precision, hmat_handle *out);

/* hmat_upload with Method 3's c (eq. 19-20) for HMAT_M3, HMAT_M3_TRUNC and
 * HMAT_M3_DENSE (-1..16, else HMAT_ERR_ARG); ignored by the other forms. */
int hmat_upload_ex(const void *blob, size_t blob_bytes, int32_t precision, int32_t method3_c, hmat_handle *out);

/* Free every device and host resource of the handle (NULL is accepted). */
int hmat_destroy(hmat_handle h);

/*
 * hmat_matvec -- y = A~ x (overwrite) for nrhs vectors, column-major N x nrhs,
 * original panel order, in the handle's precision form.  x and y must not
 * overlap.  Asynchronous on `stream` for device pointers.  For a HMAT_BF16 or
 * HMAT_FP32 handle and nrhs >= 2 the columns go through the tensor-core
 * product, 64 per pass (tcgen05 MMAs, FP32 accumulation in tensor memory; one
 * GEMM per column cluster for t, one per leaf row cluster for y): BF16 panels
 * (kind::f16) times x and t split into two BF16 parts, within 2e-5 of the same
 * panels' exact product; FP32 panels and operands each split into two TF32
 * parts (kind::tf32, two MMAs per step), within 1e-5 -- the tensor cores' FP32
 * accumulation, where one column at a time (nrhs = 1) keeps the FP32 form's
 * 2e-7.  For a double-float operator (an HMAT_FP64 handle, and the FP64 copy
 * that hmat_matvec_fp64 applies for HMAT_FP64, HMAT_BF16 and HMAT_FP32
 * handles) and nrhs >= 2 the columns go through the many-column double-float
 * product, 16 per pass: each panel vector loaded is applied to several columns,
 * and every column's result is bit for bit that of a one-column product.  The
 * many-column products allocate their buffers on first use.  x and y may be host
 * memory (staged through the handle's buffers) or device memory of the handle's
 * GPU; device memory of another GPU is rejected (HMAT_ERR_ARG), and so it is for
 * b and x of the solvers.
 * Errors: HMAT_ERR_ARG, HMAT_ERR_NOMEM, HMAT_ERR_CUDA.
 */
int hmat_matvec(hmat_handle h, const double *x, double *y, int32_t nrhs, void *stream);

/* Same product with the handle's FP64 copy (the operator of the true residual). */
int hmat_matvec_fp64(hmat_handle h, const double *x, double *y, int32_t nrhs, void *stream);

typedef struct hmat_solve_opts {
    double tol;            /* accept when ||b - A~64 x||_2 <= tol ||b||_2 (Section 4.1.3)      */
    double inner_tol;      /* a run of Algorithm 1 stops at ||r_i|| <= max(tol ||b||,
                              inner_tol ||r_start||); 0 = the paper's criterion; > 0 turns the
                              restarts into FP64 iterative refinement of a low-precision solve */
    int32_t maxit;         /* total Algorithm 1 iterations over all runs                        */
    int32_t max_restarts;  /* runs after the first one                                          */
    int32_t check_every;   /* iterations per graph batch (>= 1): between host reads of the stop
                              flag (use_graph 1), per body of the device loop (use_graph 2)     */
    int32_t use_graph;     /* 1: replay check_every iterations as one CUDA graph, the host
                              reading the stop flag between replays; 2: a whole run as one graph
                              launch (a conditional WHILE node over those batches; the device
                              decides when the run ends); 0: plain launches                     */
} hmat_solve_opts;

typedef struct hmat_solve_info {
    int32_t status;        /* hmat_status of the solve                                          */
    int32_t iters;         /* Algorithm 1 iterations (each with up to two products)             */
    int32_t restarts;      /* runs started from a true residual after the first                 */
    int32_t matvecs;       /* products in the handle's precision form                           */
    int32_t matvecs_fp64;  /* FP64 products for true residuals                                  */
    int32_t launches;      /* kernels this call enqueued (skipped ones inside graph batches too) */
    double relres_true;    /* ||b - A~64 x||_2 / ||b||_2 at exit                                 */
    double relres_inner;   /* last recursive ||r_i||_2 / ||b||_2                                */
} hmat_solve_info;

/* Defaults: tol 1e-8, inner_tol 0, maxit 1000, max_restarts 30, check_every 1, use_graph 2. */
void hmat_solve_opts_default(hmat_solve_opts *opts);

/*
 * hmat_bicgstab -- solve A~ x = b by BiCG-STAB (Algorithm 1) with the handle's
 * precision form for the products v = A~ p and t = A~ s, FP64 for every inner
 * product, the alpha/beta/omega updates and the vectors, and the FP64 true
 * residual for acceptance.  x is the initial guess on entry and the solution on
 * exit (x = 0 on exit when b = 0).  b and x are N vectors in original order.
 * Returns info->status (also when it is not HMAT_OK).  Synchronises `stream`.
 * Errors: HMAT_ERR_ARG, HMAT_ERR_CUDA, HMAT_ERR_BREAKDOWN_RHO,
 * HMAT_ERR_BREAKDOWN_OMEGA, HMAT_ERR_MAXIT, HMAT_ERR_NONFINITE.
 */
int hmat_bicgstab(hmat_handle h, const double *b, double *x, double tol, int32_t maxit, void *stream,
                  hmat_solve_info *info);

/* hmat_bicgstab with every option explicit (opts NULL = defaults). */
int hmat_bicgstab_ex(hmat_handle h, const double *b, double *x, const hmat_solve_opts *opts, void *stream,
                     hmat_solve_info *info);

/*
 * hmat_gmres -- solve A~ x = b with restarted GMRES(m) (1 <= m <= 64) on the same
 * products (Section 4.5 names other solvers as the next use of the mixed
 * products): Arnoldi with classical Gram-Schmidt applied twice, Givens
 * rotations, x += V y after each cycle of at most m steps; a cycle is one graph
 * launch.  Runs, the FP64 true residual and restarts as hmat_bicgstab_ex
 * (`check_every` and `use_graph` of opts are not used); `iters` counts Arnoldi
 * steps.  Allocates its Krylov basis (N x (m + 1) doubles) on first use.
 */
int hmat_gmres(hmat_handle h, const double *b, double *x, int32_t m, const hmat_solve_opts *opts, void *stream,
               hmat_solve_info *info);

/* ------------------------------------------------------------------------- */
/* Many systems at once                                                       */
/* ------------------------------------------------------------------------- */
/*
 * hmat_upload_batch -- one handle over `count` independent problems (blobs as for
 * hmat_upload, each validated alone), held as one block-diagonal operator: the
 * problems' index spaces are concatenated in the given order, so x and y of
 * every call on the handle are the concatenation of the problems' vectors (each
 * in its own original panel order), and one product is one launch sequence over
 * all problems.  `method3_c` as for hmat_upload_ex.  Errors as hmat_upload.
 */
int hmat_upload_batch(const void *const *blobs, const size_t *blob_bytes, int32_t count, int32_t precision,
                      int32_t method3_c, hmat_handle *out);

/* Problems of a handle (1 unless made by hmat_upload_batch); `offsets`
 * (count + 1 entries, may be NULL) receives their first rows and the total. */
int hmat_problems(hmat_handle h, int32_t *count, int64_t *offsets);

/*
 * hmat_bicgstab_multi -- solve every (problem, right-hand side) system of a
 * handle with its own BiCG-STAB recurrence (Algorithm 1), all advanced together:
 * one product launch sequence per right-hand side and iteration serves every
 * problem, the vector kernels run over all systems at once with per-system
 * inner products, and every decision (stop, breakdown, true residual with the
 * FP64 H-matrix, restart from it) is taken per system on the device.  The
 * products of several columns go through the many-column products of
 * hmat_matvec, and the work of a system whose run has stopped is skipped
 * inside the iterations.  With nrhs >= 2 and a double-float FP64 copy (every
 * form but the paper's Table 1 variants) the true residuals of the systems
 * whose run stopped are taken at the next host read (every check_every
 * iterations), over those systems' columns only, and a system that restarts
 * iterates on with the others; otherwise they are taken once no system
 * iterates.  A system's results do not depend on the other systems'.
 * b, x: N_total x nrhs column-major (N_total = the handle's N), host or device;
 * x holds the initial guess and receives the solution.  `opts` as for
 * hmat_bicgstab_ex (NULL: defaults).  infos (may be NULL): count x nrhs entries,
 * system (p, k) at index k * count + p; `launches` is the whole call's.
 * Returns HMAT_OK when every system converged, else the first system's error.
 */
int hmat_bicgstab_multi(hmat_handle h, const double *b, double *x, int32_t nrhs, const hmat_solve_opts *opts,
                        void *stream, hmat_solve_info *infos);

/* ------------------------------------------------------------------------- */
/* Product without allocation (an addition of this library; the paper has no  */
/* counterpart)                                                               */
/* ------------------------------------------------------------------------- */
/* Bytes of the static device array the allocation-free product uses. */
#define HMAT_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/*
 * hmat_matvec_noalloc -- y = A~ x for one vector, like hmat_matvec, but the call
 * allocates no memory at all.  The paper has no counterpart: it exists for
 * callers that cannot call cudaMalloc when they run the product --
 * latency-critical loops that cannot pay for an allocation (it may synchronise
 * the device), and hosts or plugins whose device memory belongs to another
 * allocator or budget.  Such a caller creates the handle once at set-up
 * (hmat_upload allocates then) and afterwards only calls this function.
 *
 * x and y: device pointers (N doubles, original panel order; host pointers are
 * rejected with HMAT_ERR_ARG because staging them would need buffers), on the
 * handle's device, which must be current; device memory of another GPU is
 * rejected with HMAT_ERR_ARG.  The product's scratch (source
 * operand copy, partial sums, operand buffers) lives in one static device array
 * of HMAT_NOALLOC_SCRATCH_BYTES compiled into the library; every GPU that loads
 * the library holds that array until the process exits.  A handle whose scratch
 * does not fit (roughly N above 20,000 panels for the FP64 form), and a handle of
 * one of the paper's two-segment variants (HMAT_M1_MIXED, HMAT_M2_SINGLE,
 * HMAT_M3), is rejected with HMAT_ERR_UNSUPPORTED.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls, on every handle, share the one array: calls that overlap on the GPU
 * (different streams without ordering) race and give wrong results.  The call
 * clears what must start at zero and is asynchronous on `stream`.
 */
int hmat_matvec_noalloc(hmat_handle h, const double *x, double *y, void *stream);

/*
 * Failure detection of the tensor-core product for many right-hand sides (no
 * counterpart in the paper; it guards the GPU path).  Its kernels hand shared-
 * memory buffers between the copy engine, the tensor cores and the threads
 * through mbarriers; every such wait is bounded (default about one second of SM
 * clock).  A wait that runs out makes the kernel give up its work, write
 * HMAT_ERR_TIMEOUT into the handle's status word (host memory the kernel can
 * write), let the copies and MMAs it issued finish, free its tensor memory and
 * return; the CUDA context stays usable.  The status is reported, and cleared,
 * by the next call on the handle (hmat_matvec, the solvers,
 * hmat_matvec_noalloc, hmat_time_matvec) or by hmat_check.
 *
 * hmat_check -- synchronise `stream` and return HMAT_ERR_TIMEOUT if a bounded
 * wait of one of the handle's kernels ran out since the last report (clearing
 * it), else HMAT_OK (HMAT_ERR_CUDA if the synchronisation fails).
 */
int hmat_check(hmat_handle h, void *stream);

/*
 * hmat_set_wait_limit -- the bound of those waits, in SM clock cycles (>= 1),
 * for the products enqueued after the call (a cached solver graph is captured
 * again).  withhold = 1 makes the projection issue none of its panel copies, so
 * its waits run out: a test of the timeout path that needs no fault; 0 is
 * normal operation.  Errors: HMAT_ERR_ARG.
 */
int hmat_set_wait_limit(hmat_handle h, int64_t cycles, int32_t withhold);

/* ------------------------------------------------------------------------- */
/* Introspection                                                              */
/* ------------------------------------------------------------------------- */
typedef struct hmat_handle_info {
    int64_t n;
    int32_t precision;
    int32_t nleaves;
    int64_t panel_bytes;         /* device bytes of the form's panels (algorithmic bytes read per product) */
    int64_t panel_bytes_fp64;    /* device bytes of the FP64 H-matrix of the true residual                  */
    int64_t index_bytes;         /* device bytes of the packing indices                                     */
    int64_t stored_entries;      /* dense_entries + lr_entries of the blob                                  */
    int64_t phase1_entries;      /* entries streamed by the projection t = W x                              */
    int64_t phase2_entries;      /* entries streamed by the expansion y = D x + V t                         */
    int64_t partials;            /* projection outputs T (per leaf column cluster, padded), summed per block */
    int64_t rank_sum;
    int64_t stored_bytes;        /* stored entries times their element bytes (no padding): the bytes one   */
                                 /* product must read at least                                              */
    int64_t phase1_bytes;        /* the projection's share of stored_bytes                                  */
    int64_t phase2_bytes;        /* the expansion's share                                                   */
    int32_t segments;            /* 1, or 2 for a paper variant whose product adds two expansions           */
    int32_t method3_c;           /* c of eq. (19)-(20) for HMAT_M3, _TRUNC and _DENSE, else 0               */
} hmat_handle_info;

int hmat_info(hmat_handle h, hmat_handle_info *out);

/*
 * hmat_autotune -- choose the projection's CTA size per panel-width bucket by
 * measurement (the paper has no counterpart: it concerns how the GPU runs the
 * product of eq. 9, not what it computes).  The leaf column clusters are
 * bucketed by the width of their panels (16-byte column vectors per row: at
 * most 32, 64, 128, 256, more); each bucket can run with CTAs of 64, 128 or 256
 * threads.  Starting from one launch over the clusters in cluster order at the
 * store's default size, the tuner times whole projections (reps launches each,
 * CUDA events on `stream`) with the work list sorted by bucket and one size per
 * bucket, changing one bucket at a time while that helps (two passes), and keeps
 * the sorted plan only if it beats the default by more than 2 %; the plan is
 * stored in the handle (also for the FP64 operator of the true residuals).  The
 * products give the same bits under any plan (each column's sum is one thread's
 * sum in row order).  The paper's variants keep their single launch.  Do not
 * overlap it with other calls on the handle; cached solver graphs are captured
 * again.  `out` (may be NULL) receives the report of the iterated operator.
 * Errors: HMAT_ERR_ARG, HMAT_ERR_NOMEM, HMAT_ERR_CUDA.
 */
typedef struct hmat_tune_bucket {
    int32_t vec_max;   /* the bucket's panels have at most this many column vectors per row (0: no bound) */
    int32_t clusters;  /* leaf column clusters in the bucket                                            */
    int32_t threads;   /* the chosen CTA size                                                            */
    int32_t pad;
    double us[3];      /* projection microseconds with this bucket at 64, 128, 256 threads (the others
                          as chosen; 0 if not measured)                                                   */
} hmat_tune_bucket;

typedef struct hmat_tune_report {
    int32_t nbuckets;  /* 5                                                                             */
    int32_t sorted;    /* 1: the projection runs the bucket-sorted work list, one launch per size run    */
    double default_us; /* one launch over the clusters in cluster order at the default CTA size          */
    double tuned_us;   /* the plan kept                                                                  */
    hmat_tune_bucket bucket[5];
} hmat_tune_report;

int hmat_autotune(hmat_handle h, int32_t reps, void *stream, hmat_tune_report *out);

/*
 * hmat_time_matvec -- enqueue `iters` products of a fixed internal vector on
 * `stream` and time each kernel of the product with CUDA events recorded on
 * that stream; ms_out[0..3] receive the mean milliseconds per launch of the
 * source-vector preparation, the projection (t = W x and the operand scatter),
 * the reduction of the blocks spanning several leaf clusters and the expansion
 * (y = D x + V t); ms_out[4] the mean per whole product.  The expansion runs as
 * in a solver product, with the fused inner products of Algorithm 1, so it
 * writes the handle's solver scalars: do not overlap it with a solve on the same
 * handle.  For a paper variant of two segments each entry sums both segments'
 * launches.  `fp64` = 1 times the FP64 H-matrix of the true residual.
 * Synchronises `stream`.
 */
int hmat_time_matvec(hmat_handle h, int32_t iters, int32_t fp64, void *stream, double *ms_out);

/* Message for a status code (static storage). */
const char *hmat_strerror(int status);

/* Text of the last CUDA error seen by this library in the calling thread. */
const char *hmat_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HMAT_H */
