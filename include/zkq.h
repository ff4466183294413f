/*
 * zkq: accurate batched Hermitian eigensolves for matrix-product-state (MPS) circuit simulation on
 * GB300 (sm_103a).  C ABI: plain pointers and sizes only.
 *
 * The computation follows arXiv:2402.11868 (SaiToh, "Recent Extensions of the ZKCM Library for
 * Parallel and Accurate MPS Simulation of Quantum Circuits"):
 *   - Section 2.1: Hermitian matrix diagonalisation is the dominant cost of the MPS simulation;
 *   - Section 2, ZKCM_CUS paragraph: a double-precision eigensolve followed by Rayleigh quotient
 *     iteration that recovers the precision;
 *   - Section 1 and its footnote: the working precision must be exponentially small in the number of
 *     qubits, because Schmidt coefficients as small as ~2^{-(n-1)/2} occur and must be kept.
 *
 * Conventions shared by every entry point
 *   Multi-word numbers: a real value is an unevaluated sum of w doubles, highest first, non-overlapping
 *     (w = 1: double; 2: double-double, ~106 bits; 4: quad-double, ~212 bits).
 *   Complex element layout: re words then im words: double[2][w] per element.
 *   Matrices: column-major, element (i, j) at index i + j*n.  A batch packs problem b's n_b x n_b
 *     matrix at element offset a_off[b] (elements, not doubles).
 *   Eigenvalues of problem b occupy positions w_off[b] .. w_off[b] + n_b - 1 of the eigenvalue array,
 *     with w_off[b] = n_0 + ... + n_{b-1}; they are sorted descending (ties keep the original order).
 *   Eigenvector c of problem b is column c of the n_b x n_b matrix at element offset a_off[b]; its first
 *     component of largest modulus is real and positive.
 *   Ownership: the caller owns every array passed in (device or host as stated per argument); the
 *     library never frees them.  A context owns its workspace.
 *   Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous on that
 *     stream; argument and launch errors return synchronously; per-problem convergence is reported in
 *     device `info` arrays, readable after the stream synchronises.  No call aborts or traps, and no C++
 *     exception leaves the library: a host allocation failure inside a call returns ZKQ_ENOMEM.
 */
#ifndef ZKQ_H
#define ZKQ_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ZKQ_OK = 0,
  ZKQ_EINVAL = 1,    /* invalid argument (sizes, word counts, null pointers, method) */
  ZKQ_ENOMEM = 2,    /* device workspace or host memory could not be allocated */
  ZKQ_ENOCONV = 3,   /* reserved: a problem did not converge (per-problem detail is in info[]) */
  ZKQ_ETIMEOUT = 4,  /* a bounded device-side wait expired */
  ZKQ_ECUDA = 5,     /* a CUDA runtime call failed; see zkq_last_cuda_error() */
  ZKQ_EADMIT = 6,    /* reserved: request refused by admission control */
  ZKQ_ETOOBIG = 7    /* the request needs more than the fixed scratch of zkq_eigh_batched_noalloc */
} zkq_status;

typedef enum { ZKQ_FP64 = 1, ZKQ_DD = 2, ZKQ_QD = 4 } zkq_prec;   /* value = words per real */

typedef enum {
  ZKQ_PLAIN_RQI = 0,  /* per-eigenpair Rayleigh quotient iteration in the target precision */
  ZKQ_OA_OZAKI = 1,   /* block Ogita-Aishima refinement with tensor-core split (Ozaki) products */
  ZKQ_OA_FP64 = 2,    /* the same refinement with its products in multi-word arithmetic on the FP64 pipe */
  ZKQ_SVD_OA = 3      /* gate updates only: FP64 SVD of M (zkq_svd_batched) in place of the FP64 eigensolve of
                         rho, its singular vectors refined as eigenvectors of rho as by ZKQ_OA_OZAKI */
} zkq_method;

typedef struct zkq_ctx zkq_ctx;

typedef struct {
  int device;             /* CUDA device ordinal */
  int max_sweeps;         /* Jacobi sweep limit (0: default 40) */
  int rqi_max_iter;       /* RQI steps per eigenpair (0: default 5) */
  int oa_max_iter;        /* Ogita-Aishima iterations (0: default 40) */
  int jacobi_cluster;     /* CTAs per large Jacobi problem (0: the context's autotune table when
                             zkq_autotune_jacobi has filled it, else 2 / 4 / 8 by the largest order) */
} zkq_config;

/* Human-readable name of a status code.  Never NULL. */
const char* zkq_status_string(zkq_status s);
/* Last CUDA error code recorded by the library in this process (0 if none). */
int zkq_last_cuda_error(void);

/* Create a context on cfg->device (cfg may be NULL: device 0, defaults).  *ctx receives the handle.
 * Errors: ZKQ_EINVAL (ctx NULL), ZKQ_ECUDA. */
zkq_status zkq_ctx_create(zkq_ctx** ctx, const zkq_config* cfg);
/* Free the context and its workspace (synchronises its device first).  NULL is accepted. */
zkq_status zkq_ctx_destroy(zkq_ctx* ctx);

/*
 * zkq_eigh_batched: double-precision eigen-decomposition of a batch of Hermitian matrices
 * (the FP64 stage of Section 2, ZKCM_CUS paragraph) by a two-sided complex Jacobi method.
 *   batch          number of problems (>= 0)
 *   n (host)       n[b] >= 1, matrix orders
 *   a_off (host)   element offsets of each matrix in A and V
 *   A (device)     input matrices, a_words words per real (1, 2 or 4); only the leading word is used;
 *                  the matrix must be Hermitian (the strictly lower triangle's conjugate is assumed)
 *   W (device)     out: double[sum n], eigenvalues per problem, descending
 *   V (device)     out: complex FP64 eigenvectors (double[2] per element) at a_off[b]
 *   info (device)  out: int32[batch]; 0 converged, > 0 sweep limit reached
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA.
 */
zkq_status zkq_eigh_batched(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                            const double* A, int a_words, double* W, double* V, int32_t* info, void* stream);

/*
 * zkq_eigh_batched_noalloc: zkq_eigh_batched for callers that cannot allocate device memory.  The paper
 * has no counterpart; it exists for callers such as code running while another part of the process
 * captures a CUDA graph, hosts that give the library a fixed memory budget, or latency-critical loops
 * where an allocation could stall on a device-wide synchronisation.
 * Arguments, layouts and errors are those of zkq_eigh_batched on the current device, with default settings
 * (40 sweeps); no context is needed.  Every problem above order 80 runs on a thread-block cluster of the
 * built-in width (2, 4 or 8 CTAs for a largest order <= 128, <= 256 or above); the cooperative-grid class
 * and a context's autotuned widths are never used, so the results agree with zkq_eigh_batched within the
 * FP64-stage tolerance (8 n 2^-53 ||A||), exactly where both take the same kernel and width.
 * The call allocates nothing: its scratch (batch metadata and the global-memory copies of A and V for
 * orders above 80, 32 n^2 bytes each) lives in one file-scope device array of ZKQ_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads the library holds until the process exits.
 *   - A batch whose scratch would exceed ZKQ_NOALLOC_SCRATCH_BYTES is rejected with ZKQ_ETOOBIG (e.g. one
 *     problem of order 1024 needs 32 MiB; orders <= 80 need no scratch beyond a few hundred bytes of metadata).
 *   - The call itself must not be captured into a CUDA graph: it uploads its metadata from host memory
 *     that is freed when it returns, and returns ZKQ_EINVAL when `stream` is capturing.  Other streams of
 *     the process may be capturing meanwhile.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current, and keeps it for the life of the process; do not use the entry point after a
 *     cudaDeviceReset of that device.
 *   - Every call uses the same array and leaves its last contents there: calls that overlap on the GPU
 *     (different streams, or different host threads, on the same device) race.
 */
#define ZKQ_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
zkq_status zkq_eigh_batched_noalloc(int batch, const int32_t* n, const int64_t* a_off, const double* A,
                                    int a_words, double* W, double* V, int32_t* info, void* stream);

/*
 * zkq_svd_batched: FP64 singular value decomposition of a batch of complex matrices by one-sided (Hestenes)
 * Jacobi -- the SVD that ZKCM_CUS offers beside the Hermitian diagonalisation (Section 2, ZKCM_CUS
 * paragraph).  Orthogonalising the columns of A (or of A^H when A is wide) does not square the
 * conditioning as the Gram matrix A A^H does, so on matrices with graded rows or columns (an MPS bond's M
 * carries its neighbours' Schmidt weights) the small singular values keep high relative accuracy.
 *   m, n (host)      int32[batch], 1 <= m, n <= 4096; k = min(m, n)
 *   a_off (host)     element offsets of A_b (m x n, column-major, complex, a_words words per real; only the
 *                    leading word of each real is read)
 *   S (device)       out: double[sum k_b], singular values of each problem, descending
 *   U (device)       out: complex FP64 (double[2] per element), m_b x k_b column-major at element offset
 *                    u_off[b] (host int64): left singular vectors, first largest-modulus component real > 0
 *   V (device)       out: n_b x k_b at element offset v_off[b]: right singular vectors (A = U diag(S) V^H)
 *   info (device)    out: int32[batch]; 0 converged, > 0 sweep limit (zkq_config.max_sweeps) reached
 * For a zero singular value the vector computed from A's columns (U's when m >= n, V's when m < n) is zero.
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA.
 */
zkq_status zkq_svd_batched(zkq_ctx* ctx, int batch, const int32_t* m, const int32_t* n, const int64_t* a_off,
                           const double* A, int a_words, double* S, double* U, const int64_t* u_off, double* V,
                           const int64_t* v_off, int32_t* info, void* stream);

/*
 * zkq_rqi_refine: recover the eigenpairs to the target precision from the FP64 ones
 * (Section 2, ZKCM_CUS paragraph: Rayleigh quotient iteration recovers the precision after the
 * double-precision eigensolve).
 *   A (device)        input matrices with a_words words per real (1, 2, 4), offsets a_off (host)
 *   W, V (device)     FP64 eigenpairs from zkq_eigh_batched (same layout)
 *   target_words      2 (double-double) or 4 (quad-double)
 *   method            ZKQ_PLAIN_RQI, ZKQ_OA_OZAKI or ZKQ_OA_FP64 (the refinement methods need n[b] <= 2048)
 *   W_out (device)    out: double[sum n][target_words], refined eigenvalues (descending)
 *   V_out (device)    out: eigenvectors, target_words words per real, element offsets a_off
 *   err_est (device)  out: double[sum n], ||A v - lambda v||_2 / max|lambda| per eigenpair (FP64 estimate)
 *   info (device)     out: int32[batch]; 0 ok; > 0 iteration limit reached on some eigenpair
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA.
 */
zkq_status zkq_rqi_refine(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                          const double* A, int a_words, const double* W, const double* V,
                          int target_words, int method, double* W_out, double* V_out, double* err_est,
                          int32_t* info, void* stream);

/*
 * zkq_workspace_size: device bytes that a context's workspace grows to when a batch is diagonalised
 * (zkq_eigh_batched) and then, if target_words is not 0, refined (zkq_rqi_refine) -- the memory the batched
 * diagonalisation of Section 2.1 holds beside the caller's arrays, for admission decisions before a call.
 * Host-side: it launches nothing and allocates nothing (it makes the context's device current).
 *   n (host)       n[b] >= 1, matrix orders (<= 4096; <= 2048 for the refinement methods)
 *   a_words        1, 2 or 4: words per real of A
 *   target_words   0 (eigensolve only), 2 or 4
 *   method         ZKQ_PLAIN_RQI, ZKQ_OA_OZAKI or ZKQ_OA_FP64 (ignored when target_words is 0)
 *   bytes (host)   out: the figure, for a context that held no workspace before.  The caller's arrays (A,
 *                  W, V, the outputs) are not included.
 * Exact for the eigensolve and plain RQI.  For the refinement methods the refinement state is exact and
 * the split-product scratch is an upper bound over the products formed for every problem (A X, then
 * X^H (A X) with I - X^H X, then X + X E).  Cluster separation steps, which run only when eigenvalues of a
 * problem lie within its cluster threshold, form further products over the clustered columns and may grow
 * the scratch beyond this figure; zkq_ctx_workspace_bytes reports what a context holds.
 * Errors: ZKQ_EINVAL, ZKQ_ECUDA.
 */
zkq_status zkq_workspace_size(zkq_ctx* ctx, int batch, const int32_t* n, int a_words, int target_words, int method,
                              size_t* bytes);
/* Device bytes of workspace the context holds now (eigensolve, refinement, split-product and MPS gate-update
 * buffers).  Errors: ZKQ_EINVAL. */
zkq_status zkq_ctx_workspace_bytes(const zkq_ctx* ctx, size_t* bytes);

/*
 * zkq_autotune_jacobi: measure the cluster width (CTAs per problem: 2, 4, 8 or 16) of the batched FP64
 * Jacobi for each order in sizes[0..nsizes) (81 .. 2048) and keep the fastest in the context's table; from
 * then on the context's eigensolves (zkq_eigh_batched, the refinement's cluster blocks, plans created
 * afterwards) take the width of the first table order >= their largest order (else the last entry), unless
 * zkq_config.jacobi_cluster fixes one.  The results do not depend on the width.  Each order is timed on a
 * synthetic batch of one Hermitian problem per SM (a_words words per real), reps timed runs after one
 * warm-up per width; the call allocates that batch and synchronises the device.
 *   best (host)   out: int32[nsizes], the chosen widths
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA (the table is unchanged then).
 */
zkq_status zkq_autotune_jacobi(zkq_ctx* ctx, int nsizes, const int32_t* sizes, int a_words, int reps, int32_t* best);

/*
 * zkq_autotune_gemm: measure the tile width of the tcgen05 split-product GEMM (256 or 128 output columns per
 * CTA tile) for each order in sizes[0..nsizes) (16..512: the Chinese-remainder form, K' = 2n <= 1024) and keep
 * the faster in a process-wide table (by K') that every later split product consults -- the batched products
 * of the refinement (Section 2, ZKCM_CUS paragraph: recovering the precision), tuned like the Jacobi width.
 * Each order is timed on a synthetic batch of n x n x n complex products in `words` words per real (enough
 * 128-column tiles to fill the GPU about four times), reps timed runs after one warm-up per width; the call
 * allocates that batch, uses the context's split-product workspace and synchronises its stream.  Both widths
 * form the same exact integer slice products: results do not change.  Needs the tcgen05 kernel selected
 * (zkq_set_gemm_kernel(1), the default).
 *   best (host)   out: int32[nsizes], 256 or 128
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA (the table is unchanged then).
 */
zkq_status zkq_autotune_gemm(zkq_ctx* ctx, int nsizes, const int32_t* sizes, int words, int reps, int32_t* best);

/*
 * Plans: a fixed-shape batch of the FP64 eigensolve (zkq_eigh_batched) followed, optionally, by plain RQI
 * refinement (zkq_rqi_refine with ZKQ_PLAIN_RQI) -- the batched diagonalisation of Section 2.1 repeated on
 * batches of one shape.  zkq_plan_create lays the batch out, allocates the plan's own device metadata and
 * workspace and uploads the metadata once (it synchronises the context's device); zkq_plan_execute then
 * only enqueues kernels and stream-ordered memsets (no allocation, no host copy, no synchronisation), so it
 * can be captured into a CUDA graph; zkq_plan_execute_graph does that capture at its first call for the
 * given buffers and replays the graph afterwards (a call with other buffers captures again).
 *   n, a_off (host)   as for zkq_eigh_batched; copied
 *   a_words           1, 2 or 4
 *   target_words      0 (eigensolve only), 2 or 4 (plain RQI to that precision)
 * Execute arguments have the layouts of zkq_eigh_batched (A, W, V, info) and zkq_rqi_refine (W_out, V_out,
 * err_est, rinfo); the refinement ones are ignored (may be NULL) when target_words is 0.  The caller owns
 * every buffer; a plan is used by one host thread at a time; calls that overlap on the GPU race on the
 * plan's workspace.  zkq_plan_execute_graph needs a stream other than the legacy default stream and
 * profiling (zkq_profile_enable) off.
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA.
 */
typedef struct zkq_plan zkq_plan;
zkq_status zkq_plan_create(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off, int a_words,
                           int target_words, zkq_plan** out);
zkq_status zkq_plan_execute(zkq_plan* plan, const double* A, double* W, double* V, int32_t* info, double* W_out,
                            double* V_out, double* err_est, int32_t* rinfo, void* stream);
zkq_status zkq_plan_execute_graph(zkq_plan* plan, const double* A, double* W, double* V, int32_t* info,
                                  double* W_out, double* V_out, double* err_est, int32_t* rinfo, void* stream);
/* Frees the plan (synchronises its device first).  NULL is accepted. */
zkq_status zkq_plan_destroy(zkq_plan* plan);

/*
 * Matrix-product state (Vidal form) resident on the device, and its gate updates (Section 1: an MPS is a
 * nested Schmidt decomposition evolved without leaving that form, cost O(n g r_max^3); Section 2.1:
 * diagonalisation at each gate dominates; footnote: Schmidt coefficients ~2^{-(n-1)/2} must survive).
 * Layout used by download/upload (host arrays): Gamma[l] is row-major (s, alpha, beta) with s in {0,1},
 * alpha < chi[l-1] (1 for l = 0), beta < chi[l] (1 for l = n-1), complex, `words` words per real,
 * concatenated over l = 0..n-1; lambda[l] (chi[l] reals of `words` words) concatenated over l = 0..n-2.
 * Site 0 is the most significant qubit of a basis index.  A two-qubit gate is 4x4 row-major complex in
 * (i j) x (k m), i the bit of `site`; a one-qubit gate is 2x2.  Gates are host arrays.
 */
typedef struct zkq_mps zkq_mps;
/* |0...0> on n_qubits sites (2 <= n <= 4096) on the context's device, bond dimensions capped at r_max
 * (<= 2048), words 2 or 4.  Gate updates need a context on the same device (else ZKQ_EINVAL).
 * Allocates per-site capacity min(2^min(l+1, n-l-1), r_max) from the device's stream-ordered memory pool
 * (cudaMallocAsync on a private stream; the pool keeps freed memory cached for later simulations), so
 * neither create nor destroy synchronises the whole device.  Errors: ZKQ_EINVAL, ZKQ_ENOMEM. */
zkq_status zkq_mps_create(zkq_ctx* ctx, int n_qubits, int r_max, int words, zkq_mps** out);
/* zkq_mps_footprint: device bytes for admitting a simulation before it exists (the many concurrent gate
 * updates of Section 2.1 held resident): *state_bytes, what zkq_mps_create(n_qubits, r_max, words) allocates;
 * *gate_bytes, what a context's workspace grows to for the widest gate update of that MPS with `method`
 * (gate scratch plus the eigensolve and refinement of zkq_workspace_size at the largest reduced matrix).
 * Host-side; allocates nothing.  Errors: ZKQ_EINVAL, ZKQ_ECUDA. */
zkq_status zkq_mps_footprint(zkq_ctx* ctx, int n_qubits, int r_max, int words, int method, size_t* state_bytes,
                             size_t* gate_bytes);
/* Frees the MPS's buffers in stream order after its last asynchronous call (apply1q); every other MPS call
 * has synchronised its stream before returning.  NULL is accepted. */
zkq_status zkq_mps_destroy(zkq_mps* mps);
/* current bond dimensions chi[0..n-2] (host) */
zkq_status zkq_mps_bond_dims(const zkq_mps* mps, int32_t* chi);
/* copy the state to / from host arrays in the layout above (synchronises the stream) */
zkq_status zkq_mps_download(const zkq_mps* mps, double* gammas, double* lambdas, void* stream);
zkq_status zkq_mps_upload(zkq_mps* mps, const int32_t* chi, const double* gammas, const double* lambdas, void* stream);
/* one-qubit gate U (2x2, host) on `site`: Gamma[site]^i <- sum_k U_ik Gamma[site]^k */
zkq_status zkq_mps_apply1q(zkq_ctx* ctx, zkq_mps* mps, int site, const double* U, void* stream);
/*
 * Two-qubit gate G (4x4, host) on (site, site+1): theta contraction (split products), the Hermitian Gram
 * matrix of the smaller side (rho = M M^H, ties left), its eigen-decomposition (FP64 Jacobi + refinement
 * `method`: ZKQ_PLAIN_RQI, ZKQ_OA_OZAKI or ZKQ_OA_FP64, to the state's words; or ZKQ_SVD_OA: the FP64 SVD of
 * M itself, whose singular vectors on that side start the same refinement), truncation to the Schmidt
 * values with sigma^2 > trunc_tau * sum sigma^2 (at most r_max), renormalisation sum lambda'^2 = 1, and the
 * split back into Gamma'[site], lambda'[site], Gamma'[site+1].  Synchronises the stream (the new bond
 * dimension is decided on the host).
 *   new_bond (host, may be NULL)          kept Schmidt rank
 *   discarded_weight (host, may be NULL)  dropped sum sigma^2 over total sum sigma^2 (FP64 estimate)
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA; ZKQ_ENOCONV if the eigensolve did not converge (the state is
 * still updated with the last iterate).
 */
zkq_status zkq_mps_apply2q(zkq_ctx* ctx, zkq_mps* mps, int site, const double* G, double trunc_tau, int method,
                           int32_t* new_bond, double* discarded_weight, void* stream);

/*
 * Measurements on the MPS in its working precision (Section 1: a Vidal MPS is a nested Schmidt
 * decomposition; in canonical form the parts of the chain away from a site reduce to the squared Schmidt
 * weights).  Both read the state as the last gate update left it; both synchronise the stream.  A state is
 * assumed normalised and canonical (every state the gate updates produce is, up to truncation).
 *
 * zkq_mps_expect1: one-qubit expectation values <O_k> at sites[k], k < count, from site k's tensor and its
 * two weight vectors: sum over alpha, beta, s, s' of lam_{l-1,alpha}^2 lam_{l,beta}^2
 * conj(Gamma[l]^s_{alpha beta}) O_{s s'} Gamma[l]^{s'}_{alpha beta}.
 *   sites (host)   int32[count], 0 <= site < n
 *   O (host)       count operators, each 2x2 row-major complex with the state's words per real
 *                  (double[count][4][2][words])
 *   out (host)     double[count][2][words]: re words then im words of each value
 * zkq_mps_sample: `shots` bit strings drawn from the Born distribution by the chain rule: site k of a shot
 * takes bit 1 when its uniform number u >= the conditional probability of bit 0 given the bits drawn so far
 * (inverse CDF, computed in the state's words), else 0.
 *   u (host)       double[shots][n], each in [0, 1) (the caller's random numbers; else ZKQ_EINVAL)
 *   bits (host)    out: int32[shots][n], site 0 first
 *   prob (host)    out: double[shots][words], the probability of each string (underflows to 0 below
 *                  about 2^-1000)
 * The context supplies the workspace (shots in chunks of 4 per SM, 3 prefix vectors of max chi each).
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA.
 */
zkq_status zkq_mps_expect1(zkq_ctx* ctx, const zkq_mps* mps, int count, const int32_t* sites, const double* O,
                           double* out, void* stream);
zkq_status zkq_mps_sample(zkq_ctx* ctx, const zkq_mps* mps, int shots, const double* u, int32_t* bits, double* prob,
                          void* stream);

/*
 * zkq_mw_gemm: batched multi-word complex products C_i = op(A_i) B_i, the dense products of the refinement
 * step (A X, X^H X, X^H (A X), X E) that recover the precision of the FP64 eigenpairs (Section 2, ZKCM_CUS
 * paragraph).  Rows of op(A) and columns of B are scaled by powers of two and truncated to integers.
 * Method 1 (Chinese-remainder form, Ozaki-Uchino-Imamura): each scaled integer is split in two halves,
 * the halves are reduced modulo r pairwise coprime moduli <= 256 (r is 17-18 for double-double and 32-33
 * for quad-double accuracy), three exact fp16 tensor-core products are formed per modulus (high x high,
 * high x low, low x high; fp32 accumulation is exact below 2^24), and the CRT reconstructs the exact
 * integer results; k > 512 takes the digit form instead.  Method 2 (digit form, Ozaki-Ogita-Oishi-Rump
 * 2012): 8-bit (7-bit when k > 512) balanced digits, one exact product per kept digit pair, exact
 * recombination.  Method 0 computes the same products directly in multi-word arithmetic on the FP64 pipe.
 *   count (>= 0)   number of products; m, n, k, opA (host, int32[count])
 *   opA[i]         0: A_i is m x k (column-major, ld m);  1: A_i is stored k x m (ld k), op(A) = A^H
 *   A, B, C        device arrays; product i uses element offsets a_off[i], b_off[i], c_off[i] (host int64)
 *   wa, wb, wc     words per real of A, B, C (1, 2 or 4); B_i is k x n (ld k), C_i is m x n (ld m)
 *   p_bits         requested accuracy of methods 1 and 2: |C - op(A) B| <= k 2^-p_bits 2^(e_row + f_col) per
 *                  element, where 2^e_row <= 8 max|row of op(A)| and 2^f_col <= 8 max|column of B| are the
 *                  power-of-two scales of the split; method 0 rounds in wc-word arithmetic instead.
 *                  1 <= p_bits <= 252
 * Constraints: k <= 2048.  C must not overlap A or B.
 * Errors: ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ECUDA.
 */
zkq_status zkq_mw_gemm(zkq_ctx* ctx, int count, const int32_t* m, const int32_t* n, const int32_t* k,
                       const int32_t* opA, const double* A, const int64_t* a_off, int wa, const double* B,
                       const int64_t* b_off, int wb, double* C, const int64_t* c_off, int wc, int p_bits, int method,
                       void* stream);

/*
 * Slice-GEMM kernel selection for the split products (process-wide): 1 = tcgen05 kernel (5th-generation
 * tensor cores, accumulators in tensor memory; default), 0 = warp-level mma.sync kernel.  Both compute
 * identical exact integer slice products.
 * zkq_check_device_waits: ZKQ_ETIMEOUT if a bounded device-side wait of the tcgen05 kernel expired since
 * the last check (synchronises the device), else ZKQ_OK.
 */
zkq_status zkq_set_gemm_kernel(int which);
int zkq_get_gemm_kernel(void);
zkq_status zkq_check_device_waits(void);
/* Tile width of the tcgen05 slice GEMM (process-wide): 256 or 128 output columns per tile for every batch, or
 * 0 to restore the default (256 where it fits, or the table zkq_autotune_gemm filled is cleared).  Both widths
 * give identical results.  Errors: ZKQ_EINVAL. */
zkq_status zkq_set_gemm_tile_width(int width);

/*
 * zkq_test_grid_barrier_hook: test hook of the bounded grid barrier of the cooperative-grid Jacobi class
 * (zkq_eigh_batched with a few problems of order above 80), so that a test can drive the barrier's expiry
 * path without faulting or hanging the GPU.  It sets, on the current device and for every later launch,
 * `extra_arrivals` (0 or 1) arrivals that the barrier waits for but that never come -- the waiting blocks
 * then poll a generation flag that nothing advances -- and the poll limit 2^log2_poll_limit (4..22; a poll
 * sleeps about 64 ns).  On expiry the barrier raises the problem's abort flag, no later barrier of that
 * problem waits, every block finishes its bounded loops, and the problem's info entry is -1; the context and
 * device stay usable.  (0, 22) restores the defaults.  The paper has no counterpart (its ZKCM_CUS relies on
 * cuSOLVER).  Errors: ZKQ_EINVAL, ZKQ_ECUDA.
 */
zkq_status zkq_test_grid_barrier_hook(int extra_arrivals, int log2_poll_limit);

/*
 * zkq_mw_op: element-wise multi-word arithmetic, the building block of every refinement step
 * (the paper's multiple-precision numbers, Section 1; here double-double / quad-double made of FP64
 * error-free transformations).  Diagnostic entry point used to check the arithmetic.
 *   op        0 add, 1 sub, 2 mul, 3 div, 4 sqrt(a), 5 complex mul, 6 complex div
 *   words     1, 2 or 4
 *   count     number of operands (real ops: count values; complex ops: count complex values)
 *   a, b, out arrays of count x words (real) or count x 2 x words (complex) doubles
 *   on_device 0: host arrays, computed on the CPU with the same header; 1: device arrays, one GPU thread
 *             per element on `stream`
 * Errors: ZKQ_EINVAL, ZKQ_ECUDA.
 */
zkq_status zkq_mw_op(int op, int words, int64_t count, const double* a, const double* b, double* out,
                     int on_device, void* stream);

/*
 * Launch profiler (tracing): when enabled, every kernel launch of the library is bracketed by CUDA events
 * on its launching stream and device time is accumulated per kernel class (jacobi, rqi, ozaki_scale,
 * ozaki_slice, ozaki_gemm, ozaki_combine, oa_elementwise, mps, other, jacobi_cluster: the refinement's
 * cluster eigensolves).  The paper reports only wall
 * times; this breaks them down for the roofline of each kernel.  Process-wide.
 *   zkq_profile_classes()        number of classes
 *   zkq_profile_class_name(c)    name of class c (never NULL)
 *   zkq_profile_enable(on)       start (1) / stop (0) recording
 *   zkq_profile_read(ms, n, w, k) waits for the recorded launches, writes per-class milliseconds, launch
 *                                counts and algorithmic work for the first k classes, then clears the
 *                                record.  Work: ozaki_gemm counts 2 m (2n) (2k) flops per exact slice
 *                                product (at launch); jacobi and jacobi_cluster count 32 n flops per
 *                                applied rotation, the scaled (fast-rotation) update of A and V (on the
 *                                device); 0 where not counted
 * Errors: ZKQ_EINVAL (null arrays, k < 1), ZKQ_ECUDA.
 */
int zkq_profile_classes(void);
const char* zkq_profile_class_name(int cls);
zkq_status zkq_profile_enable(int on);
zkq_status zkq_profile_read(double* ms, int64_t* launches, double* work, int nclasses);

#ifdef __cplusplus
}
#endif
#endif
