/*
 * sdpgb.h -- C ABI of libsdpgb, a GB300 (sm_103a) implementation of the
 * preconditioned-CG Hessian solve inside the modified interior-point method of
 * Zhang & Lavaei, "Modified Interior-Point Method for Large-and-Sparse Low-Rank
 * Semidefinite Programs" (arXiv 1703.10973).
 *
 * Problem (eq. SDP / SDD):  min C.X  s.t.  A_i.X = b_i (i < m), X psd;
 *                           max b^T y s.t.  sum_i y_i A_i + S = C, S psd.
 *
 * Conventions shared by every call
 *  - Symmetric matrices are passed as triplets (i, j, v) with i <= j meaning
 *    M[i][j] = M[j][i] = v; repeated positions add.  Indices are 0-based int32.
 *  - Dense n x n matrices are row-major double (equal to column-major for the
 *    symmetric ones).
 *  - Host arrays are copied during the call; the caller keeps ownership.
 *  - "_dev" pointers are device pointers owned by the caller; they must be
 *    valid on the handle's stream and must not alias each other.
 *  - The handle owns all other device memory and frees it in sdp_destroy.
 *    Handles and batches allocate from one stream-ordered memory pool per device
 *    (allocation waits for the handle's stream; a free is ordered on it), which
 *    keeps up to 32 GiB of freed memory for the next handle instead of returning
 *    it to the driver.  Destroy a handle only when no batch still has work in
 *    flight on it (sdp_batch_remove it first, or let the batch call return).
 *  - Every call returns an sdp_status; nothing is thrown across the ABI.  After
 *    any status the handle may still be destroyed; sdp_last_error() gives text.
 *  - One handle is used by one host thread at a time.  All work is issued on the
 *    stream given to sdp_setup (NULL = the legacy default stream).
 *  - Precision argument `prec`: SDP_FP64 computes in double.  With SDP_FP32 or
 *    SDP_BF16 the Hessian matvec rounds the part W_s of the split W = W_l + W_s
 *    (W_l = the top-k eigenpairs of the last preconditioner build, else W itself)
 *    to float or bfloat16 and accumulates in float, adding the low-rank terms in
 *    double.  sdp_precond_apply with SDP_FP32 or SDP_BF16 reads a float copy of
 *    the Hhat core's dense Schur-factor inverse and accumulates that product in
 *    float; inside PCG (sdp_pcg_solve, sdp_ipm_step, batches) the core is applied
 *    in double at every precision, because near the optimum the core has
 *    kappa ~ 1/mu.  The Algorithm 1 apply always runs in double; with a
 *    reduced-precision params.prec its core is formed on the tensor cores in TF32
 *    (sdp_mixed_gemm).  Vectors crossing the ABI stay double.
 */
#ifndef SDPGB_H
#define SDPGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdp_problem sdp_problem;

typedef enum {
  SDP_OK = 0,
  SDP_ERR_ARG = 1,          /* invalid argument (sizes, null pointers, indices)   */
  SDP_ERR_OOM = 2,          /* device or host allocation failed                  */
  SDP_ERR_NOT_PD = 3,       /* Cholesky met a non-positive pivot                  */
  SDP_ERR_MAXIT = 4,        /* iteration cap reached; best iterate is kept        */
  SDP_ERR_UNSUPPORTED = 5,  /* A^T A is not diagonal (Assumption 2 not met here)  */
  SDP_ERR_NUMERIC = 6,      /* NaN or Inf detected                                 */
  SDP_ERR_TIMEOUT = 7,      /* a bounded device-side wait expired                 */
  SDP_ERR_CUDA = 8          /* a CUDA runtime call failed                          */
} sdp_status;

typedef enum { SDP_FP64 = 0, SDP_FP32 = 1, SDP_BF16 = 2 } sdp_prec;

typedef enum {
  SDP_PRECOND_DIAG = 0,     /* tau^2 A^T A only (U = 0)                            */
  SDP_PRECOND_WOODBURY = 1, /* Ht = tau^2 A^T A + UU UU^T, eq. (AtIUUtAt)/(SMW2),    */
                            /* Algorithm 1 (Section III)                           */
  SDP_PRECOND_HAT = 2       /* Hhat = A^T (tau^2 I + 2 tau U U^T kron I) A,        */
                            /* eq. (sparse_prec) of Section V: the Algorithm 1     */
                            /* construction with Z = sqrt(2 tau) I, whose core is  */
                            /* conditioned like 1/mu instead of 1/mu^2; this is    */
                            /* the preconditioner of the paper's experiments       */
} sdp_precond_kind;

typedef struct {
  double gap_tol;      /* relative duality gap |C.X-b^Ty|/(1+|C.X|+|b^Ty|); 1e-6 */
  double infeas_tol;   /* ||b-A X||/(1+||b||) and ||C-S-A^T y||_F/(1+||C||_F);  1e-6 */
  double pcg_rtol;     /* PCG stop: ||H dy - r|| <= pcg_rtol ||r||;  1e-8          */
  int ipm_maxit;       /* 100 */
  int pcg_maxit;       /* 1000 */
  int refine_maxit;    /* max restarts of PCG on the true FP64 residual; 64         */
  int k;               /* rank k of the W split (eq. Wsplit2); 0 = value of sdp_setup */
  double step_frac;    /* fraction of the step to the boundary; 0.9                */
  int prec;            /* sdp_prec used inside PCG by sdp_ipm_step / sdp_solve     */
  int precond;         /* sdp_precond_kind; SDP_PRECOND_HAT                        */
  double inner_rtol;   /* PCG tolerance of one restart (sweep); 1e-9                */
  int verbose;         /* 1 = one line per IPM iteration on stderr; 2 = also one   */
                       /* line per PCG restart (sweep)                           */
  int pcg_graph;       /* 1 = the PCG loop runs on the device as a CUDA graph with */
                       /* a conditional while node (default); 0 = host-driven     */
                       /* loop launching the same kernels (for profilers that do  */
                       /* not support conditional graph nodes); a batch follows   */
                       /* the setting of its first problem                        */
  double inner_rtol_lp; /* PCG tolerance of one sweep whose matvec runs in FP32 or */
                        /* BF16 (the FP64 true residual refines it); 1e-4         */
  long long wait_cycles; /* bound of every device-side spin wait (the grid barriers */
                        /* of the cooperative tridiagonalisation, n > 1024), in SM */
                        /* clock cycles; a wait that runs out makes the call return */
                        /* SDP_ERR_TIMEOUT and leaves the handle usable; 0 = 4e9   */
                        /* (about 2 s)                                             */
  int k_max;            /* adaptive split rank (Section V implementation notes):   */
                        /* with eta > 0 every preconditioner build uses            */
                        /* k~ = max{i <= k_max : lambda_i(W) >= eta lambda_{i+1}(W)} */
                        /* (eigenvalues decreasing, lambda_0 = +inf, k~ >= 1);     */
                        /* 0 = k of sdp_setup.  At most SDP_K_MAX                  */
  double eta;           /* eigenvalue-gap ratio of that rule; 0 = fixed rank k     */
} sdp_params;

/* Largest split rank (k of sdp_setup, params.k, params.k_max). */
#define SDP_K_MAX 64

typedef struct {
  int iter;                 /* IPM iteration index that produced this record      */
  double mu;                /* X.S / n                                             */
  double obj_p, obj_d;      /* C.X and b^T y                                       */
  double relgap, pinf, dinf;
  double alpha_p, alpha_d, sigma;
  double tau;               /* lambda_min(W) of the split                          */
  int pcg_iters_pred, pcg_iters_corr;
  double pcg_relres_pred, pcg_relres_corr;   /* true FP64 residuals              */
  int converged;            /* 1 when the stopping test held at entry              */
  int nt_fallback;          /* 1 when W came from the Denman-Beavers iteration     */
  int k_split;              /* split rank of this iteration's preconditioner        */
} sdp_ipm_info;

typedef struct {
  double obj_p, obj_d, relgap, pinf, dinf;
  int iters;                /* IPM iterations taken                                */
  int pcg_iters_total;
  int converged;
  double seconds;           /* host wall time of the solve                         */
} sdp_result;

/* Fill *prm with the defaults listed above. */
void sdp_default_params(sdp_params* prm);

/*
 * sdp_setup -- eq. (SDP): copy C, the A_i and b to the device and build the
 * sparse constraint operator: the CSR pattern of V = sum_i v_i A_i (union of all
 * supports, both triangles), the gather map slot -> (constraint, coefficient),
 * the per-constraint entry list used by the Hessian gather, and
 * (A^T A)^{-1} = diag(1/||A_i||_F^2).  Assumption 2 is required in the form
 * "A^T A diagonal": SDP_ERR_UNSUPPORTED if two constraints have a nonzero inner
 * product.  Sets the start point X = S = xi I, y = 0.
 *   n >= 1, m >= 1, 1 <= k <= min(n, SDP_K_MAX); params k_max in [0, SDP_K_MAX],
 *   eta >= 0 (SDP_ERR_ARG otherwise).  C triplets: nnzC >= 0 (Ci, Cj, Cv may be
 *   NULL when nnzC == 0).  A triplets: (Ak[t], Ai[t], Aj[t], Av[t]) adds Av[t]
 *   at (Ai,Aj) and (Aj,Ai) of A_{Ak[t]}.  b has m entries.  prm may be NULL
 *   (defaults).  cuda_stream is a cudaStream_t or NULL.  On success *out owns
 *   the problem; on failure *out is NULL.
 */
sdp_status sdp_setup(int n, int m,
                     int64_t nnzC, const int32_t* Ci, const int32_t* Cj, const double* Cv,
                     int64_t nnzA, const int32_t* Ak, const int32_t* Ai, const int32_t* Aj,
                     const double* Av, const double* b, int k, const sdp_params* prm,
                     void* cuda_stream, sdp_problem** out);

/*
 * sdp_hessian_matvec -- eq. (hesseqn2): Hv_dev[i] = A_i . (W (sum_j v_dev[j] A_j) W)
 * for the handle's current scaling matrix W (set by sdp_ipm_step or sdp_set_W).
 * Matrix-free: V = sum v_j A_j on the CSR pattern, T = W V (sparse gather
 * SpMM), then one dot W[p,:] . T[q,:] per stored constraint entry.
 * v_dev, Hv_dev: device double[m].  prec: sdp_prec.
 */
sdp_status sdp_hessian_matvec(sdp_problem* h, const double* v_dev, double* Hv_dev, int prec);

/*
 * sdp_precond_build -- Algorithm 1 steps 1-2 for the current W:
 * tau = lambda_min(W), U = V_l (Lambda_l - tau I)^{1/2} from the k largest
 * eigenpairs (eq. Wsplit2), Z = chol(2 W0 + U U^T) (eq. hessExp2), the core
 * S = tau^2 I + UU^T (A^T A)^{-1} UU with UU = A^T (U kron Z) (eq. SMW2, using
 * tau^2), its Cholesky factor L and L^{-1}.  With params.precond =
 * SDP_PRECOND_HAT, Z = sqrt(2 tau) I (eq. sparse_prec, Section V): the core is
 * then tau^2 I + 2 tau K with K_(l,l') = sum_i (A_i u_l)(A_i u_l')^T / ||A_i||^2,
 * a sparse matrix scattered into the dense core.  SDP_ERR_NOT_PD if a factor fails.
 */
sdp_status sdp_precond_build(sdp_problem* h);

/*
 * sdp_precond_apply -- eq. (SMW2): z = (tau^2 G)^{-1} (r - UU S^{-1} UU^T G^{-1} r)
 * with G = A^T A, UU^T y = Z^T (sum y_i A_i) U and (UU X)_i = A_i . (Z X U^T)
 * (eq. Umv); Z = sqrt(2 tau) I for SDP_PRECOND_HAT, so neither product needs Z.
 * r_dev, z_dev: device double[m].  Needs sdp_precond_build first.
 */
sdp_status sdp_precond_apply(sdp_problem* h, const double* r_dev, double* z_dev, int prec);

/*
 * sdp_pcg_solve -- Algorithm 1 step 3: PCG for H y = r from y = 0 with the
 * built preconditioner, stopping when ||r - H y|| <= rtol ||r|| (recursive
 * residual) or after maxit iterations (SDP_ERR_MAXIT, y = last iterate).
 * prec selects the matvec/preconditioner precision; for prec != FP64 the solve
 * is an FP64 iterative refinement whose true residual is recomputed in FP64.
 * r_dev, y_dev: device double[m].  iters, relres (true FP64 relative residual)
 * may be NULL.
 */
sdp_status sdp_pcg_solve(sdp_problem* h, const double* r_dev, double* y_dev, double rtol,
                         int maxit, int prec, int* iters, double* relres);

/*
 * sdp_ipm_step -- one iteration of the infeasible NT predictor-corrector:
 * residuals; NT scaling W = L Q Lambda^{-1/2} Q^T L^T (X = L L^T, L^T S L = Q Lambda Q^T);
 * sdp_precond_build; predictor (sigma = 0) and corrector (sigma = (mu_aff/mu)^3)
 * Newton directions, each from H dy = Rp - A(Rc) + A(W Rd W) solved by PCG;
 * step to step_frac of the boundary; update.  info may be NULL.  Returns
 * SDP_OK also when the point already satisfies the stopping test
 * (info->converged = 1, nothing changed).  With the graph loop (pcg_graph = 1)
 * and a batchable configuration (SDP_PRECOND_HAT, 1 <= k <= 8, any prec) the
 * two Newton systems run through a one-problem batch of this
 * handle (its PCG graph is captured once); the iterates are the same.
 */
sdp_status sdp_ipm_step(sdp_problem* h, sdp_ipm_info* info);

/* sdp_solve -- repeat sdp_ipm_step until converged or ipm_maxit.  res may be NULL. */
sdp_status sdp_solve(sdp_problem* h, sdp_result* res);

/* Replace the scaling matrix W by W_dev (device double[n*n], symmetric positive definite). */
sdp_status sdp_set_W(sdp_problem* h, const double* W_dev);

/* Copy the current W to device memory W_dev (double[n*n]). */
sdp_status sdp_get_W(sdp_problem* h, double* W_dev);

/* Copy the current iterate to host arrays (each may be NULL): X, S n*n; y m. */
sdp_status sdp_get_solution(sdp_problem* h, double* X_host, double* y_host, double* S_host);

/* Replace the current iterate by host arrays X, S (n*n) and y (m); iter sets the counter. */
sdp_status sdp_set_state(sdp_problem* h, const double* X_host, const double* y_host,
                         const double* S_host, int iter);

/* Checkpoint: copy the current iterate to host arrays X, S (n*n) and y (m) and the
 * IPM iteration counter to *iter (each may be NULL).  sdp_set_state of these values
 * on a handle of the same problem resumes the solve with the same iterates. */
sdp_status sdp_get_state(sdp_problem* h, double* X_host, double* y_host, double* S_host, int* iter);

/* tau and the split rank used by the last sdp_precond_build. */
sdp_status sdp_precond_info(sdp_problem* h, double* tau, int* k);

/* Problem sizes: n, m, k, nnz of the V pattern. */
sdp_status sdp_sizes(const sdp_problem* h, int* n, int* m, int* k, int64_t* nnzV);

/* Reset the iterate to the start point X = S = xi I, y = 0 on the device (no host
 * transfer); the preconditioner and W are invalidated. */
sdp_status sdp_reset(sdp_problem* h);

/*
 * Per-kernel-class timing for measurement.  sdp_timing_enable(h, cls) records a
 * pair of CUDA events on the handle's stream around every later launch of the
 * kernel class `cls` ("gemm_f64", "sytrd", "matvec", "potrf", "trsm", "stein",
 * "ormtr", "precond_apply"); NULL turns recording off.  sdp_timing_read
 * synchronises the stream and returns the accumulated device milliseconds,
 * launch count, and algorithmic flops and bytes of the recorded launches, then
 * clears the accumulators.  Any pointer may be NULL.
 */
sdp_status sdp_timing_enable(sdp_problem* h, const char* cls);
sdp_status sdp_timing_read(sdp_problem* h, double* ms, int64_t* launches, double* flops, double* bytes);
/* cls "*" records every class (regions may nest: phases such as "nt_scaling",
 * "precond_build", "pcg", "max_step" contain kernel classes).  sdp_timing_report
 * synchronises the stream, writes one line "class ms launches flops bytes" per
 * recorded class into buf (NUL-terminated, truncated to len), clears the
 * accumulators and returns the length the full report needs. */
int64_t sdp_timing_report(sdp_problem* h, char* buf, int64_t len);

/* Device memory held by the handle (bytes of its allocations; buffers are
 * allocated on first use, so this grows during the first IPM iteration).
 * Serving admission compares estimates against it. */
int64_t sdp_device_bytes(const sdp_problem* h);

/* Number of kernel launches issued by this handle since setup (for accounting). */
int64_t sdp_launch_count(const sdp_problem* h);

/*
 * Batched solves (many uneven problems advanced together).  sdp_batch_create groups count set-up problems (each keeps its own
 * stream, data and state; all must use SDP_PRECOND_HAT with 1 <= k <= 8, and
 * the SDP_FP64, SDP_FP32 or SDP_BF16 (split) matvec; SDP_ERR_UNSUPPORTED otherwise).
 * sdp_batch_solve runs their interior-point iterations in lockstep: the dense
 * per-problem phases on each problem's stream (one host thread per problem),
 * and every PCG iteration of all their Newton systems as one sequence of
 * batched launches on cuda_stream (during those solves the problems' own work
 * also runs on cuda_stream; give it a high priority), captured once as a CUDA graph that loops on
 * the device while any problem's PCG is running.  A problem's iterates are the
 * same in a batch as alone.  results: count entries (NULL allowed); the
 * seconds field of each is the host wall time from the start of the call to
 * the end of that problem's last iteration.  Returns
 * SDP_OK when every problem converged, SDP_ERR_MAXIT when some hit an
 * iteration limit, else the first error (sdp_batch_last_error).  Problems
 * start from their current iterate (sdp_reset for the start point).  The batch
 * does not own the problems; destroy the batch before them.
 */
typedef struct sdp_batch sdp_batch;
sdp_status sdp_batch_create(sdp_problem* const* problems, int count, void* cuda_stream, sdp_batch** out);
sdp_status sdp_batch_solve(sdp_batch* b, sdp_result* results);
const char* sdp_batch_last_error(const sdp_batch* b);
void sdp_batch_destroy(sdp_batch* b);
/* Lockstep groups of a batch (default 0 = pairs: ceil(count / 2) groups).
 * sdp_batch_solve deals the problems, largest first, into the groups in a
 * snake order (0..G-1, G-1..0, ...) and solves every group as its own lockstep batch on its own stream
 * and host thread, so that one group's dense phases overlap another group's
 * batched PCG.  1 = all problems in one lockstep.  Results do not depend on
 * the grouping (each problem's iterates are the same as alone).
 * SDP_ERR_ARG for a NULL batch or groups < 0. */
sdp_status sdp_batch_set_groups(sdp_batch* b, int groups);
/* Host wall-clock seconds the last sdp_batch_solve spent in each stage, summed
 * over its iterations: out[0] residuals + NT scaling + preconditioner (all
 * problems), out[1] predictor PCG (batched), out[2] predictor step lengths and
 * corrector right-hand side, out[3] corrector PCG (batched), out[4] step
 * lengths and the checked update; out[5] the part of out[1] + out[3] spent in
 * the batched graph launches, out[6] the number of those launches (PCG sweeps
 * of the batch), out[7] the batched PCG iterations they ran (per launch, the
 * most any problem ran).  With groups, out[0..5] are the slowest group's and
 * out[6..7] the sum over groups.  out: 8 doubles.  SDP_ERR_ARG for NULL. */
sdp_status sdp_batch_stage_seconds(const sdp_batch* b, double* out);
/* Autotuner of the batched PCG matvec: the first batched Newton solve times the
 * SpMM tile (rows of W per CTA, R = 1, 2, 4, 8 within shared memory) on the
 * batch's own data and keeps the fastest (every R gives the same results).
 * *spmm_rows = the chosen R (0 before the first solve); ms[0..3] = least
 * milliseconds per launch of each candidate over five rounds (0 = not run).  With lockstep
 * groups, the first group's choice.  Either pointer may be NULL. */
sdp_status sdp_batch_tuning(const sdp_batch* b, int* spmm_rows, double* ms);

/*
 * Continuous batching (serving): members join and leave a batch between
 * interior-point iterations, and every PCG iteration of the members' Newton
 * systems shares the batched launches.  A batch made by sdp_batch_create with
 * count = 0 (problems NULL) starts empty.
 *   sdp_batch_add     -- the set-up problem h joins, from its current iterate, at
 *                        the next sdp_batch_step (SDP_ERR_UNSUPPORTED for a
 *                        configuration the batch cannot run, as sdp_batch_create;
 *                        SDP_ERR_ARG for a member already present or a batch with
 *                        lockstep groups from sdp_batch_solve).
 *   sdp_batch_step    -- one interior-point iteration of every running member in
 *                        lockstep; *running (may be NULL) = members still running.
 *                        A member stops running when its iterate meets the
 *                        tolerances, its ipm_maxit is reached or one of its calls
 *                        fails; the others carry on.  Returns the first batch-wide
 *                        failure (a member's own failure is reported by
 *                        sdp_batch_member).
 *   sdp_batch_member  -- result of member h (seconds = time since it joined) and
 *                        its state: 0 running, 1 converged, 2 iteration limit,
 *                        3 failed (the call then returns that member's status).
 *   sdp_batch_remove  -- h leaves the batch (finished, or cancelled while running:
 *                        its iterate stays where the last step left it).
 * Launch structures and the captured PCG loop are rebuilt at the next step after
 * a change of membership.  A member's iterates are the same as alone.
 */
sdp_status sdp_batch_add(sdp_batch* b, sdp_problem* h);
sdp_status sdp_batch_step(sdp_batch* b, int* running);
sdp_status sdp_batch_member(const sdp_batch* b, const sdp_problem* h, sdp_result* r, int* state);
sdp_status sdp_batch_remove(sdp_batch* b, sdp_problem* h);

/*
 * sdp_hessian_matvec_static -- handle-free, allocation-free variant of
 * sdp_hessian_matvec.  The paper has no counterpart: this call exists for
 * callers that cannot allocate device memory (code running inside a CUDA graph
 * that is being captured, a host callback, or an embedding runtime that owns
 * every device allocation itself), so it keeps no handle and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * Computes the same FP64 product as sdp_hessian_matvec, Hv_dev[k] = A_k . (W V W)
 * with V = sum_j v_dev[j] A_j, directly from the constraint triplets (same
 * convention as sdp_setup: (k, i, j, v) sets (A_k)_ij = (A_k)_ji = v,
 * duplicates add), all in device memory:
 *   Ak_dev, Ai_dev, Aj_dev: int32[nnzA];  Av_dev: double[nnzA];
 *   W_dev: double[n*n], symmetric, row-major;  v_dev: double[m];
 *   Hv_dev: double[m], overwritten (cleared first).  Hv_dev must not overlap
 *   v_dev or W_dev (SDP_ERR_ARG): it is cleared before they are read.
 * Scratch: two n x n FP64 matrices in a static __device__ array of this
 * library (SDP_STATIC_MAX_N^2 * 16 bytes = 4 MiB per device that loads it,
 * held until the process exits); nothing is allocated.
 * n > SDP_STATIC_MAX_N returns SDP_ERR_ARG before any launch.  Triplets with
 * an index out of range are skipped by the kernels, counted, and make the call
 * return SDP_ERR_ARG.  The call synchronises cuda_stream once, to read that
 * count.  The first call on each device looks up the scratch address
 * (cudaGetSymbolAddress), which can load the module: make that first call
 * before capturing any stream.  The products are accumulated with FP64
 * atomic adds, so the last bits of a result can differ between runs (the
 * handle matvec is deterministic).  Calls whose executions overlap (several
 * streams or host threads) share the scratch and race: serialise them.
 * Error text for this call: sdp_last_error(NULL), per host thread.
 */
#define SDP_STATIC_MAX_N 512
sdp_status sdp_hessian_matvec_static(int n, int m, int64_t nnzA, const int32_t* Ak_dev, const int32_t* Ai_dev,
                                     const int32_t* Aj_dev, const double* Av_dev, const double* W_dev,
                                     const double* v_dev, double* Hv_dev, void* cuda_stream);

/*
 * sdp_mixed_gemm -- the reduced-precision dense product of the Woodbury core
 * formation (Algorithm 1 step 2: the blocks Z^T (K_ll' Z)), on the tensor cores:
 *   C_dev (M x N, FP64, row stride ldc) = op(A) op(B),
 * op(A) = A (M x K) or A^T when transA (A then K x M), op(B) = B (K x N) or B^T
 * when transB; all row-major FP64 device arrays.  The operands are rounded to
 * BF16 (prec = SDP_BF16) or TF32 (prec = SDP_FP32) and the products accumulate
 * in FP32 (tcgen05.mma), so |C - op(A) op(B)| <= (2u + u^2 + K 2^-24) |op(A)| |op(B)|
 * entrywise with u = 2^-8 + 2^-24 (BF16) or 2^-11 + 2^-24 (TF32, rounded to
 * nearest from the FP32 copy).  work_dev: caller-owned device
 * scratch of at least sdp_mixed_gemm_work_bytes(M, N, K) bytes, 256-byte
 * aligned.  err_dev: one device int, set to 1 if a bounded wait inside the
 * kernel ran out (the product is then incomplete).  Issued on cuda_stream,
 * asynchronous.  SDP_ERR_ARG for bad sizes or pointers, SDP_ERR_UNSUPPORTED
 * when the driver offers no tensor-map encoder.  A handle whose params.prec is
 * SDP_FP32 or SDP_BF16 forms its Algorithm 1 core with this product in TF32
 * (BF16 operands left that core unusable as a preconditioner).
 */
int64_t sdp_mixed_gemm_work_bytes(int M, int N, int K);
sdp_status sdp_mixed_gemm(int prec, int M, int N, int K, const double* A_dev, int lda, int transA,
                          const double* B_dev, int ldb, int transB, double* C_dev, int ldc,
                          void* work_dev, int64_t work_bytes, int* err_dev, void* cuda_stream);

void sdp_destroy(sdp_problem* h);
const char* sdp_status_str(sdp_status s);
const char* sdp_last_error(const sdp_problem* h);   /* NULL: the last handle-free call */

#ifdef __cplusplus
}
#endif
#endif /* SDPGB_H */
