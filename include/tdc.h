/*
 * tdc.h -- C ABI of the GB300 divide-and-conquer (DC) tridiagonal eigensolver.
 *
 * The library computes T = Q diag(lambda) Q^T for a real symmetric tridiagonal
 * T = tridiag(e, d, e) (the matrix of Eq. (1) of Li, Rouet, Liu, Huang, Gao and Chi,
 * "An efficient hybrid tridiagonal divide-and-conquer algorithm on distributed
 * memory architectures") by Cuppen's method: tearing (Eq. 2), recursive solution of
 * the two halves, and the rank-one merge of Eqs. (3)-(6), with deflation (Eq. 5),
 * FP64 secular-equation roots, the Loewner-theorem recomputation of z (Remark 1)
 * and the eigenvector product U = Q (G P) diag(Qhat, I) of Eq. (6).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers unless the name ends in _host.
 *    The caller owns every buffer; the library allocates nothing except where an
 *    entry point says so.
 *  - Matrices are column-major FP64 with a leading dimension ld >= rows.
 *  - Eigenvalues are returned in ascending order.  syev-type entry points make the
 *    largest-magnitude entry of every eigenvector positive (first such entry on ties).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    asynchronous with respect to the host unless stated otherwise.
 *  - Return value: 0 = launched; -i = argument i is invalid (LAPACK convention,
 *    nothing launched); 3 = workspace too small; 4 = a CUDA error was reported at
 *    launch.  Conditions found on the device are OR-ed into *dev_status (a device
 *    int the call zeroes first): bit 0 (1) = a secular root hit the iteration cap,
 *    bit 1 (2) = non-finite input, bit 2 (4) = a leaf QL iteration hit its cap,
 *    bit 3 (8) = a bounded device wait timed out.
 *    dev_status may be NULL (the status is then kept in the workspace).
 *  - No entry point aborts, throws, traps the device, or reads host memory from a
 *    kernel.
 */
#ifndef TDC_H_
#define TDC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Which form of the eigenvector product U = Q_sel Qhat (Eq. 6) a merge uses. */
enum tdc_path {
  TDC_PATH_DENSE_FP64 = 0,   /* FP64 GEMM, Qhat tiles generated inside the kernel      */
  TDC_PATH_DENSE_OZAKI = 1,  /* split-precision FP64 emulation on bf16 tensor cores    */
  TDC_PATH_HSS = 2,          /* randomized HSS approximation of Qhat (Algorithm 1)     */
  TDC_PATH_AUTO = 3          /* HSS when K >= k_threshold, else DENSE_OZAKI           */
};

typedef struct tdc_opts {
  int32_t path;              /* enum tdc_path                                           */
  int32_t leaf;              /* leaf size, 1..32 (default 32)                           */
  double hss_tol;            /* relative ID tolerance for the HSS path (default 1e-12)  */
  int32_t hss_leaf;          /* HSS leaf block size (default 512)                       */
  int32_t hss_rp;            /* random samples r + p (default 128)                      */
  int64_t k_threshold;       /* AUTO: HSS only for merges with K >= this (default 8192) */
  int32_t ozaki_slices;      /* bf16 slices per operand (default 6, range 5..7; 7 gives */
                             /* FP64-level accuracy for 34 instead of 26 slice products)  */
  int32_t max_secular_iter;  /* iteration cap per secular root (default 64)             */
  int32_t tile_cfg;          /* FP64 product tile shape: -1 = autotuned (else a size    */
                             /* rule), 0..11 = 128x128, 128x64, 64x64, 64x32, 32x32,   */
                             /* 128x32, 64x16, 128x16, 16x16, 16x32, 16x64, 32x16       */
  int32_t secular_lanes;     /* lanes per secular root: 0 = chosen per tree level from  */
                             /* the level's root count (default), or 1, 2, 4, 8, 16, 32 */
  int32_t eigvec;            /* how the eigenvectors of D + rho z z^T keep orthogonal    */
                             /* (Section 1): TDC_EIGVEC_LOWNER (default) or             */
                             /* TDC_EIGVEC_EXTENDED                                       */
  int32_t hss_grow;          /* HSS: times r + p may be doubled when an ID rank reaches  */
                             /* the sample count (adaptive sampling), 0..4 (default 1);  */
                             /* a merge still saturated after that takes the dense       */
                             /* FP64 product                                              */
} tdc_opts;

/* tdc_opts.eigvec: the Loewner-theorem z of Remark 1 (Gu and Eisenstat), or Sorensen and
 * Tang's extended precision: each root is refined to double-double (tau + tau_lo, one
 * Newton step on the secular function evaluated in double-double arithmetic), the
 * original z is kept, and every difference d_j - lambda_i of the eigenvector
 * (D - lambda_i)^{-1} z is formed in double-double before it is rounded. */
enum tdc_eigvec { TDC_EIGVEC_LOWNER = 0, TDC_EIGVEC_EXTENDED = 1 };

/* Fills *opts with the defaults listed above. */
void tdc_default_opts(tdc_opts* opts);

/* Bytes of device workspace tdc_syev_tridiag needs for order n. */
size_t tdc_workspace_bytes(int64_t n, const tdc_opts* opts);

/*
 * tdc_syev_tridiag -- all eigenvalues and eigenvectors of tridiag(e, d, e).
 * (Eq. 1; the DC tree splits a node of size m at floor(m/2), Eq. 2.)
 *   n        order (>= 1)
 *   d        n diagonal entries (read only)
 *   e        n-1 off-diagonal entries (read only; may be NULL when n == 1)
 *   lambda   n outputs, ascending
 *   Q        n x n output, column j is the eigenvector of lambda[j]
 *   ldq      leading dimension of Q (>= n)
 *   opts     NULL for defaults
 *   ws       device workspace of at least tdc_workspace_bytes(n, opts) bytes,
 *            256-byte aligned
 * Scale: the entries are used as given (no internal rescaling).  The Loewner products
 * multiply differences of eigenvalues four at a time and the secular solver's FP32
 * phase holds d in FP32, so max |T| should lie in [2^-120, 2^120]; outside it, scale
 * d and e by a power of two first (exact: the eigenvalues scale by it, the
 * eigenvectors are unchanged).
 */
int tdc_syev_tridiag(int64_t n, const double* d, const double* e, double* lambda,
                     double* Q, int64_t ldq, const tdc_opts* opts, void* ws,
                     size_t ws_bytes, int* dev_status, void* stream);

/*
 * tdc_syev_tridiag_host -- the same solve from and to HOST memory: copies d, e in,
 * solves, copies lambda and Q (ld = ldq) out, and synchronizes the stream.  Uses
 * only the caller's device buffer dev_buf of tdc_host_buffer_bytes(n, opts) bytes.
 * Host buffers should be page-locked for full copy bandwidth.  Returns the launch
 * status, or the device status bits (positive) if the solve reported any.
 */
size_t tdc_host_buffer_bytes(int64_t n, const tdc_opts* opts);
int tdc_syev_tridiag_host(int64_t n, const double* d_host, const double* e_host,
                          double* lambda_host, double* Q_host, int64_t ldq,
                          const tdc_opts* opts, void* dev_buf, size_t dev_buf_bytes,
                          void* stream);

/*
 * tdc_syev_tridiag_host_async -- tdc_syev_tridiag_host without the wait: enqueues on
 * `stream` the copy of d, e in, the solve, and the copies of lambda, Q and the device
 * status word (to *status_host) out, and returns.  The outputs and *status_host are
 * valid once the stream has reached that point (synchronize it, or an event recorded
 * after the call).  Host buffers, status_host included, must be page-locked for the
 * copies to be asynchronous.  Calls on different streams with different dev_buf run
 * concurrently, so the copy-out of one problem overlaps the solve of the next.
 * Returns 0, -i for a bad argument i (-10: status_host NULL), 3 (buffer too small)
 * or 4 (launch error); the solve's own status arrives in *status_host.
 */
int tdc_syev_tridiag_host_async(int64_t n, const double* d_host, const double* e_host,
                                double* lambda_host, double* Q_host, int64_t ldq,
                                const tdc_opts* opts, void* dev_buf, size_t dev_buf_bytes,
                                int* status_host, void* stream);

/*
 * tdc_merge -- one rank-one merge (Eqs. 3-6).  Computes the eigendecomposition of
 *     diag(Q1 D1 Q1^T, Q2 D2 Q2^T) + |beta| v v^T,  v = e_{n1} + sign(beta) e_{n1+1},
 * i.e. D + rho z z^T in the basis Q = diag(Q1, Q2) with rho = 2|beta| and
 * z = Q^T v / sqrt(2) (last row of Q1, sign(beta) times the first row of Q2).
 *   n1, n2   sizes of the two halves (>= 1 each)
 *   D        n1 + n2 eigenvalues, each half ascending (read only)
 *   Q        (n1+n2) x (n1+n2) block-diagonal input, ld = ldq (read only; only the
 *            two diagonal blocks are read)
 *   beta     the coupling entry b_k of Eq. (2)
 *   lambda   n1+n2 outputs, ascending;  Q_out: output eigenvectors, ld = ldqo
 *   K_out    device int64: number of non-deflated entries K (may be NULL)
 *   Q_out must not overlap Q.  The eigenvector signs are those of Eq. (6) (no sign
 *   normalisation).  Workspace: tdc_merge_workspace_bytes(n1 + n2, opts).
 */
size_t tdc_merge_workspace_bytes(int64_t n, const tdc_opts* opts);
int tdc_merge(int64_t n1, int64_t n2, const double* D, const double* Q, int64_t ldq,
              double beta, double* lambda, double* Q_out, int64_t ldqo, int64_t* K_out,
              const tdc_opts* opts, void* ws, size_t ws_bytes, int* dev_status,
              void* stream);

/*
 * tdc_merge_inspect -- tdc_merge, plus a copy of the merge's intermediate values into
 * caller-provided device arrays, so that each step of the merge can be checked on its
 * own: the sort of D (the merge of the two ascending halves), deflation (Eq. 5: the
 * type-1 test on rho |z_j|, the type-2 plane rotations G on nearly equal d_j, and the
 * permutation P of the deflated entries), the secular roots (Section 1, stored as
 * (origin, tau) with lambda_i = dbar_origin + tau), the Loewner z of Remark 1 and
 * the normalisation of the columns of Qhat.  Arguments 1-15 are those of tdc_merge;
 * `trace` (host struct) holds device pointers, each of which may be NULL (not
 * copied).  Every array has room for n = n1 + n2 entries; only the prefix that the
 * counts give is defined.  Indices are 0-based.
 *   counts[8]  (int64): K, deflated count, plane rotations, Gu groups c1 (columns
 *              touching rows of T1 only) and c3 (both halves), type-1 deflations,
 *              then two zeros
 *   perm[n]    sorted position p -> input index j (ties: the T1 entry first)
 *   d_sorted, z_sorted [n]: the sorted d and z after the rotations (z scaled by
 *              1/sqrt(2), rotated entries' d and z updated as Eq. 5's G gives them)
 *   kept[K], deflated[nd]: sorted positions of the non-deflated and deflated entries,
 *              ascending
 *   rot_j, rot_k [nrot], rot_c, rot_s [nrot]: the rotations in the order applied;
 *              columns (j, k) become (c q_j + s q_k, -s q_j + c q_k)
 *   dbar, zbar [K]: the non-deflated values
 *   origin [K] (int32, index into dbar), tau [K]: the roots
 *   zhat [K]: the Loewner z (the original z with TDC_EIGVEC_EXTENDED);
 *   sinv [K]: 1 / ||(D - lambda_i)^{-1} zhat||
 *   tau_lo [K]: with TDC_EIGVEC_EXTENDED, the low parts of the roots (tau + tau_lo);
 *              not written otherwise
 * Returns as tdc_merge.
 */
typedef struct tdc_merge_trace {
  int64_t* counts;
  int32_t* perm;
  double* d_sorted;
  double* z_sorted;
  int32_t* kept;
  int32_t* deflated;
  int32_t* rot_j;
  int32_t* rot_k;
  double* rot_c;
  double* rot_s;
  double* dbar;
  double* zbar;
  int32_t* origin;
  double* tau;
  double* zhat;
  double* sinv;
  double* tau_lo;
} tdc_merge_trace;
int tdc_merge_inspect(int64_t n1, int64_t n2, const double* D, const double* Q, int64_t ldq,
                      double beta, double* lambda, double* Q_out, int64_t ldqo, int64_t* K_out,
                      const tdc_opts* opts, void* ws, size_t ws_bytes, int* dev_status,
                      void* stream, const tdc_merge_trace* trace);

/*
 * tdc_syev_tridiag_batched -- `batch` independent problems of orders n_host[p]
 * (host array), solved together level by level (one launch per phase per tree level
 * for the whole batch).
 *   off_de[p]  (host) element offset of problem p in d_cat, e_cat and lambda_cat;
 *              must be the dense packing off_de[p] = n_0 + ... + n_{p-1};
 *              e_cat[off_de[p] + i] is the i-th off-diagonal entry (i < n_p - 1)
 *   off_q[p]   (host) element offset of problem p's n_p x n_p block in Q_cat
 *              (ld = n_p)
 *   dev_status_per_problem: device int[batch] (may be NULL), same bits as above.
 *   Workspace: tdc_batched_workspace_bytes(batch, n_host, opts).
 */
size_t tdc_batched_workspace_bytes(int32_t batch, const int64_t* n_host, const tdc_opts* opts);
int tdc_syev_tridiag_batched(int32_t batch, const int64_t* n_host, const int64_t* off_de,
                             const int64_t* off_q, const double* d_cat, const double* e_cat,
                             double* lambda_cat, double* Q_cat, const tdc_opts* opts,
                             void* ws, size_t ws_bytes, int* dev_status_per_problem,
                             void* stream);

/*
 * tdc_syev_tridiag_backward -- gradient of a scalar loss L(lambda, Q) with respect to
 * (d, e), given lambda_bar = dL/dlambda and Qbar = dL/dQ at the forward output:
 *     Tbar = Q (diag(lambda_bar) + F o (Q^T Qbar)) Q^T,  F_ic = 1/(lambda_c - lambda_i), F_ii = 0,
 *     g_d[a] = Tbar_aa,   g_e[a] = Tbar_{a,a+1} + Tbar_{a+1,a}   (first-order perturbation
 *     theory of the symmetric eigenproblem; distinct eigenvalues assumed).
 * Only the band of Tbar is formed; the columns of Qbar that are entirely zero are
 * skipped (the call synchronizes the stream once to count them).
 *   lambda, Q (ld = ldq): the forward output;  g_lambda, g_Q (ld = ldg): may be NULL;
 *   g_d (n), g_e (n - 1): outputs.  Workspace: tdc_backward_workspace_bytes(n, opts).
 * The two products with Q (Q^T Qbar_S and Q M_S) run in FP64, or on the split-precision
 * tensor-core path when opts->path is TDC_PATH_DENSE_OZAKI (7 bf16 slices whatever
 * opts->ozaki_slices says, since the eigenvector term multiplies the products' error by
 * up to 1 / min |lambda_c - lambda_i|).  dev_status (may be NULL) gets bit 8 if a
 * tensor-core wait timed out.
 */
size_t tdc_backward_workspace_bytes(int64_t n, const tdc_opts* opts);
int tdc_syev_tridiag_backward(int64_t n, const double* lambda, const double* Q, int64_t ldq,
                              const double* g_lambda, const double* g_Q, int64_t ldg, double* g_d,
                              double* g_e, const tdc_opts* opts, void* ws, size_t ws_bytes,
                              int* dev_status, void* stream);

/*
 * tdc_syev_tridiag_backward_batched -- the gradient of tdc_syev_tridiag_backward for
 * `batch` problems at once (the batched forward's dense packing): problem p has order
 * n_host[p] (host array), its lambda, g_lambda, g_d and g_e at the prefix sum
 * n_0 + ... + n_{p-1} of the *_cat vectors (g_e holds n_p - 1 entries there; its
 * last slot is not written), and its n_p x n_p blocks of Q and Qbar (ld = n_p) at the
 * prefix sum of n^2 in Q_cat and g_Q_cat.  g_lambda_cat and g_Q_cat may be NULL.  The
 * nonzero columns of each problem's Qbar are found on the device and counted with one
 * synchronization of the stream; the products with Q are one batched launch each.
 * Workspace: tdc_backward_batched_workspace_bytes(batch, n_host, max_cols, opts),
 * max_cols = the most nonzero columns of any problem's Qbar (-1: any number).
 * Returns 0, -i for a bad argument i, 3 (workspace too small for the columns
 * found) or 4 (launch error).
 */
size_t tdc_backward_batched_workspace_bytes(int32_t batch, const int64_t* n_host, int64_t max_cols,
                                            const tdc_opts* opts);
int tdc_syev_tridiag_backward_batched(int32_t batch, const int64_t* n_host, const double* lambda_cat,
                                      const double* Q_cat, const double* g_lambda_cat,
                                      const double* g_Q_cat, double* g_d_cat, double* g_e_cat,
                                      const tdc_opts* opts, void* ws, size_t ws_bytes,
                                      int* dev_status, void* stream);

/*
 * Per-phase device timing.  Between tdc_profile_begin() and tdc_profile_end(), every
 * solve records a pair of CUDA events on its own stream around each phase of each
 * tree level, and synchronizes its stream once at its end to read back the
 * per-merge counts (K and the Gu groups) from which the algorithmic work of the
 * eigenvector product is counted.  Phases: 0 tear + leaves, 1 deflation + rotations,
 * 2 secular roots, 3 Loewner z + column norms, 4 eigenvalue placement,
 * 5 eigenvector product on the FP64 or HSS form (Eq. 6), 6 deflated-column copy,
 * 7 sign normalisation, 8 split-precision product (the tcgen05 GEMM alone),
 * 9 operand split of the split-precision product (digit slices of Q_sel and Qhat),
 * and inside phase 5 for HSS merges: 10 sampling (Omega, Y = Qhat Omega1,
 * Z = Qhat^T Omega2, the leaves' Phi and Theta), 11 compression (IDs, couplings B,
 * the rank check; repeated when the sample grows), 12 HSS multiply (up-sweep,
 * couplings, down-sweep, leaf blocks).
 * Not thread-safe; meant for benchmarks.
 */
#define TDC_NPHASE 13
#define TDC_PROFILE_LEVELS 32
typedef struct tdc_profile {
  double ms[TDC_NPHASE];           /* summed event time per phase                     */
  int64_t launches[TDC_NPHASE];    /* kernel launches per phase                       */
  double product_flops;            /* algorithmic flops of the Eq. (6) products:
                                      sum over merges of 2 K (n1 (c1 + c3) + n2 (c3 + c2)) */
  double product_min_bytes;        /* 8 bytes x (Q_sel read + U written) over merges   */
  int64_t merges;                  /* merges executed                                 */
  int64_t K_total;                 /* sum of K over merges                            */
  int64_t calls;                   /* solves recorded                                 */
  double fp64_product_flops;       /* product_flops of the merges on the FP64 product */
  double split_product_flops;      /* product_flops of the merges on the split product */
  double split_tensor_flops;       /* bf16 tensor flops those run: slice pairs x 2 m K K */
  double defl_copy_bytes;          /* top merges: 8 bytes x rows x deflated columns
                                      written plus 8 bytes x their live rows read         */
  double secular_flops;            /* 10 K x (FP64 secular-function evaluations) per
                                      merge: K terms of one division, four FMA and one
                                      multiplication each                                */
  int64_t hss_fallbacks;           /* HSS merges whose ID ranks reached the sample count
                                      (r + p) even after the adaptive growths and that
                                      took the dense product instead                      */
  int64_t hss_regrowths;           /* HSS compressions repeated with a doubled sample  */
  double hss_sampling_flops;       /* 4 K^2 (r + p) per HSS compression: Y and Z       */
  double level_fp64_min_bytes[TDC_PROFILE_LEVELS];   /* per tree level (leaves up): the
                                      product_min_bytes of its merges on the FP64 product */
  double level_fp64_flops[TDC_PROFILE_LEVELS];       /* the same for fp64_product_flops  */
  double level_fp64_product_ms[TDC_PROFILE_LEVELS];  /* event time of each level's FP64
                                                        product (tile count + GEMM)        */
  int64_t secular_evals;           /* FP64 secular-function evaluations, summed over the
                                      roots (the FP32 evaluations are not counted)        */
  double sg_gemm_ms;               /* event time of the dense split GEMM kernel's launches
                                      (the HSS products; the backward's split products)   */
  double sg_tensor_flops;          /* their bf16 tensor flops: slice pairs x 2 M N K per
                                      product, M, N, K the launch-time sizes               */
} tdc_profile;
void tdc_profile_begin(void);
int tdc_profile_end(tdc_profile* out);

/*
 * tdc_syev_tridiag_noalloc -- tdc_syev_tridiag with default options for orders
 * n <= TDC_NOALLOC_MAX_N, for callers that cannot allocate device memory: code
 * running under an allocator that forbids new device allocations, plug-ins handed
 * only the input and output buffers by their host application, or paths where an
 * allocation would synchronize the device.  The paper has no counterpart; this is an
 * interface convenience.
 *   The workspace is a fixed array of TDC_NOALLOC_SCRATCH_BYTES inside the library,
 *   held on every GPU that loads it until the process exits.  The caller passes
 *   inputs and outputs only (device pointers, as for tdc_syev_tridiag).  The first
 *   call on each device looks up the array's device address (cudaGetSymbolAddress)
 *   with that device current.  Calls share the array: calls whose work overlaps on the GPU (different streams,
 *   or the same array used from two host threads without ordering) race.  The call
 *   clears what must start at zero (the status word when dev_status is NULL) and
 *   calls no cudaMalloc, cudaFree or other allocating routine.
 *   Returns -1 if n < 1 or n > TDC_NOALLOC_MAX_N, otherwise as tdc_syev_tridiag.
 */
#define TDC_NOALLOC_MAX_N 512
#define TDC_NOALLOC_SCRATCH_BYTES (8u << 20)
int tdc_syev_tridiag_noalloc(int64_t n, const double* d, const double* e, double* lambda,
                             double* Q, int64_t ldq, int* dev_status, void* stream);

/*
 * Batched plans for repeated solves of the same ragged shape: the DC trees, the
 * per-level launch tables and the product path are built and uploaded once into
 * the workspace (create synchronizes its stream); execute then only launches
 * kernels and a status memset, so it can be captured in a CUDA graph and replayed.
 * The problem layout is the dense packing of tdc_syev_tridiag_batched (off_de =
 * prefix sums of n, Q blocks n_p x n_p packed back to back).  Dense product paths
 * only (the HSS path reads sizes back to the host).  The workspace passed to create
 * must stay alive and untouched by other calls until destroy.
 */
typedef struct tdc_batched_plan tdc_batched_plan;
int tdc_batched_plan_create(int32_t batch, const int64_t* n_host, const tdc_opts* opts, void* ws,
                            size_t ws_bytes, void* stream, tdc_batched_plan** out);
int tdc_batched_plan_execute(const tdc_batched_plan* plan, const double* d_cat, const double* e_cat,
                             double* lambda_cat, double* Q_cat, int* dev_status_per_problem,
                             void* stream);
void tdc_batched_plan_destroy(tdc_batched_plan* plan);

/*
 * tdc_batched_plan_execute_persistent -- the same solve as tdc_batched_plan_execute in ONE
 * kernel launch (after four status / counter memsets): every CTA of a grid of
 * (SMs x resident CTAs) takes whole problems from a work queue, largest first, and runs
 * all their phases -- tear (Eq. 2), leaves, and each merge bottom-up (Eqs. 3-6) -- with
 * block barriers only; no CTA waits on another.  Same layout, outputs and status words as
 * tdc_batched_plan_execute; capturable in a CUDA graph.  The FP64 product only (64 x 16
 * tiles; the lanes per secular root follow each merge's K, so results agree with the
 * level-by-level execute to rounding, not bit for bit).  Returns 0, -i for a bad argument
 * i (-1 also for a plan on another product path), or 4 for a launch error.
 */
int tdc_batched_plan_execute_persistent(const tdc_batched_plan* plan, const double* d_cat, const double* e_cat,
                                        double* lambda_cat, double* Q_cat, int* dev_status_per_problem,
                                        void* stream);

/*
 * tdc_batched_plan_execute_host -- one execute of the plan between host buffers,
 * without waiting: enqueues on `stream` the copies of d_host, e_host (the plan's dense
 * packing, sum(n) doubles each, e padded by one zero per problem) into the caller's
 * device arrays d_dev, e_dev, the execute (into lambda_dev, Q_dev and dev_status, one
 * int per problem), and the copies of lambda, Q (sum(n^2) doubles) and the status
 * words out to lambda_host, Q_host, status_host.  The outputs are valid once the
 * stream has reached that point.  Host buffers must be page-locked.  The plan was
 * uploaded at creation, so no pageable copy runs here, and executes of two plans on
 * two streams overlap the copy-out of one with the solve of the other (a plan and its
 * device arrays serve one execute at a time).  Returns 0, -i for a bad argument i, or
 * 4 for a launch error; the solves' status arrives in status_host.
 */
int tdc_batched_plan_execute_host(const tdc_batched_plan* plan, const double* d_host,
                                  const double* e_host, double* lambda_host, double* Q_host,
                                  int* status_host, double* d_dev, double* e_dev,
                                  double* lambda_dev, double* Q_dev, int* dev_status,
                                  void* stream);

/*
 * Autotuning of the FP64 product's tile shape per DC tree level (the twelve shapes of
 * tdc_opts.tile_cfg).  Every FP64 product sums each output element over k in the
 * same order whatever the shape, so the shape changes speed, never results.
 *
 * tdc_autotune -- runs the full solve of this input once per shape, twice over,
 * times each level's product with CUDA events on `stream`, and records the fastest
 * shape per level in a process-wide table keyed by the tree's level structure;
 * later calls on trees of that structure with tile_cfg == -1 use it.  Arguments as
 * for tdc_syev_tridiag (lambda and Q receive a valid solve).  shape_per_level
 * (nullable, max_levels entries) receives the chosen shapes, leaves to root,
 * and *n_levels (nullable) the number of levels.  Synchronizes `stream`.
 * Returns 0, -i for a bad argument i, 3 (workspace) or 4 (device error).
 *
 * tdc_batched_plan_autotune -- the same for a batched plan: the plan's own shapes are
 * replaced by the tuned ones (so tune before capturing execute in a graph).
 */
int tdc_autotune(int64_t n, const double* d, const double* e, double* lambda, double* Q, int64_t ldq,
                 const tdc_opts* opts, void* ws, size_t ws_bytes, int32_t* shape_per_level,
                 int32_t max_levels, int32_t* n_levels, int* dev_status, void* stream);
int tdc_batched_plan_autotune(tdc_batched_plan* plan, const double* d_cat, const double* e_cat,
                              double* lambda_cat, double* Q_cat, int32_t* shape_per_level,
                              int32_t max_levels, int32_t* n_levels, void* stream);

/* Reads a device status word on `stream` (synchronizes it).  Returns the bits. */
int tdc_read_status(const int* dev_status, void* stream);

/* Library version string. */
const char* tdc_version(void);

/* sizeof of the ABI's structs, for bindings to check their layouts: which = 0 tdc_opts,
 * 1 tdc_profile, 2 tdc_merge_trace; 0 for any other value. */
size_t tdc_struct_bytes(int which);

/*
 * tdc_diag_reciprocal -- diagnostic: r[i] = the reciprocal of x[i] as the secular
 * sums compute it (Section 1's secular function, one reciprocal per term): Newton-
 * Raphson on the hardware approximation, within about one unit in the last place of
 * 1/x for nonzero finite x with |x| <= 2^1022 (larger |x| gives 0).  x, r: n device
 * doubles.  Asynchronous on `stream`.  Returns 0, -i for a bad argument i, or 4 for a
 * launch error.
 */
int tdc_diag_reciprocal(const double* x, double* r, int64_t n, void* stream);

/*
 * tdc_diag_rsqrt -- diagnostic: r[i] = 1/sqrt(x[i]) as the leaf QL's plane rotations
 * compute it (Newton on the hardware approximation), for x in [2^-1020, 2^1020),
 * within a few units in the last place.  Arguments and returns as tdc_diag_reciprocal.
 */
int tdc_diag_rsqrt(const double* x, double* r, int64_t n, void* stream);

/*
 * tdc_diag_split_combine -- diagnostic: r[i] = (acc[i] + tsum[i] 2^-8) 2^e2[i] as the
 * split-precision product's epilogue forms each output from its exact integer levels
 * (acc, in level-5 units) and its FP32 tail levels (tsum, in level-6 units) (Eq. (6)'s
 * product, split form): acc and tsum 2^-8 converted to doubles exactly (acc rounded to
 * nearest when |acc| > 2^53), one FP64 addition, then the power-of-two scaling, exact
 * when the result is a normal double.  acc: n device int64, tsum: n device floats,
 * e2: n device int32, r: n device doubles.  Asynchronous on `stream`.  Returns 0, -i
 * for a bad argument i, or 4 for a launch error.
 */
int tdc_diag_split_combine(const int64_t* acc, const float* tsum, const int32_t* e2, double* r, int64_t n,
                           void* stream);

/*
 * tdc_diag_wait_timeout -- diagnostic of the bounded device waits: runs the split-
 * precision product's mbarrier wait (the one its producer, MMA and epilogue roles use)
 * on a barrier that nothing arrives on, with a limit of limit_ns nanoseconds.  The
 * wait gives up after the limit, ORs bit 3 (8, a timed-out wait) into *dev_status and
 * writes 0 to *dev_out (1 if the wait had completed); the kernel then returns and the
 * context stays usable.  limit_ns in [1000, 2e9] (the product's own limit is 2 s).
 * dev_status, dev_out: device ints.  Asynchronous on `stream`.  Returns 0, -i for a
 * bad argument i, or 4 for a launch error.
 */
int tdc_diag_wait_timeout(int64_t limit_ns, int* dev_status, int* dev_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TDC_H_ */
