/*
 * qst.h -- C ABI of the GB300 (sm_103a) pooled-chain pCN sampler for Bayesian
 * quantum state tomography (Nguyen, Law, Lukens, arXiv:2501.17334).
 *
 * The library runs R independent, non-communicating preconditioned
 * Crank-Nicolson Metropolis-Hastings chains per tomography problem (Sec. I and
 * Algorithm 2), each over the Bures parameterisation rho(x) of Algorithm 1, with
 * the multinomial likelihood of Eq. likelihood, and pools every chain's kept
 * states into the posterior mean of Eq. BME2 plus the autocorrelation
 * diagnostics of Eq. ACFrho and Eq. IACT.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a qst_status; no C++ exception crosses the ABI.
 *     qst_last_error() gives a human-readable message for the last failure
 *     on the calling thread.
 *   - "host" pointers are CPU memory owned by the caller; "device" pointers are
 *     CUDA global memory on the handle's device, owned by the caller.
 *   - Work is enqueued on the caller's CUDA stream given at creation; calls that
 *     return host data synchronise that stream first.
 *   - Device-side trouble (a non-finite initial log-likelihood, an exhausted
 *     wait, a failed bounds check) sets bits of a device status word; the next
 *     synchronising call reports it as QST_ERR_NUMERIC or QST_ERR_TIMEOUT.
 *   - Latent vectors x in R^{4 D^2} are stored [Re G | Im G | Re H | Im H] with
 *     each D x D block column-major (Algorithm 1 steps 2-3).
 *   - The packed density matrix vec_h(rho) in R^{D^2} has, at row-major
 *     position (i, j): Re rho_ii on the diagonal, Re rho_ij above it (i < j),
 *     Im rho_ij below it (i > j).
 */
#ifndef QST_H
#define QST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QST_OK = 0,
    QST_ERR_INVALID_ARG = 1, /* rejected input; nothing was allocated or enqueued */
    QST_ERR_CUDA = 2,        /* a CUDA runtime/driver call failed */
    QST_ERR_OOM = 3,         /* workspace too small or allocation failed */
    QST_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    QST_ERR_NUMERIC = 5,     /* non-finite values where finite ones were required */
    QST_ERR_STATE = 6,       /* call not valid in the handle's current state */
    QST_ERR_UNSUPPORTED = 7  /* valid request this build does not implement */
} qst_status;

/* Arithmetic of the projector contraction p = vec_h(rho) . P (Sec. II, p_kl = Tr Lambda_kl rho). */
typedef enum {
    QST_PREC_FP32 = 0,   /* plain FP32 SIMT contraction */
    QST_PREC_BF16X3 = 1, /* tcgen05 tensor cores: rho split into three bf16 terms against the
                            exactly-representable Pauli projector matrix, FP32 accumulation
                            (hi products and mid + lo products in two accumulators); 1..5 qubits */
    QST_PREC_TF32 = 2,   /* tcgen05 kind::tf32: rho rounded once to TF32 (11 significant bits),
                            FP32 accumulation; 1..4 qubits.  Its log L error is O(1) at 4 qubits:
                            a comparison form, not an accurate one */
    QST_PREC_TF32X2 = 3, /* tcgen05 kind::tf32: rho = hi + lo, both TF32 (22 significant bits),
                            hi and lo products in two accumulators; 1..3 qubits */
    QST_PREC_PAULI = 4,  /* structured FP32 form for the Pauli POVMs only (NULL POVM arrays or
                            arrays equal to qst_pauli_povms): no projector matrix; the 6^Q
                            probabilities come from rho by one split per qubit, each a few FP32
                            adds of the parent block's entries (about 3.5 * 6^Q adds per chain
                            against 2 * 24^Q FLOPs dense), every setting renormalised by its own
                            sum; 1..6 qubits (6 only with NULL POVM arrays) */
    QST_PREC_AUTO = 5    /* per problem, the faster of the forms that apply to it: BF16X3 where its
                            packed projectors are exact in bf16 (1..5 qubits), PAULI where its POVMs
                            are the Pauli set (1..6 qubits), FP32 if neither; qst_create times the
                            candidates (with autotune; else PAULI from five qubits on, BF16X3 below)
                            and qst_diagnostics reports the form in use */
} qst_precision;

/* Prior of rho, i.e. the map from the latent Gaussian vector x to rho (Algorithm 1 is the
 * Bures one; the method leaves the prior open). */
typedef enum {
    QST_PRIOR_BURES = 0, /* Algorithm 1: W = (U + I) G with U the unitary QR factor of H (positive
                            real diagonal of R), rho = W W^dag / Tr */
    QST_PRIOR_HS = 1     /* Hilbert-Schmidt (Ginibre) prior: W = G, rho = G G^dag / Tr; the QR of H
                            is skipped (H's entries are still drawn and carried, unused) */
} qst_prior;

/* The likelihood of a problem's counts.  The method changes only its likelihood step for another
 * one (Sec. III); the Poisson form covers counts whose number of trials per setting is known but
 * whose detected outcomes do not exhaust the trials (lossy detectors: the elements of a setting
 * then sum to less than the identity). */
typedef enum {
    QST_LIKELIHOOD_MULTINOMIAL = 0, /* Eq. likelihood: log L = sum_kl c_kl log p_kl; every setting's
                                       elements must sum to the identity */
    QST_LIKELIHOOD_POISSON = 1      /* independent Poisson counts of mean mu_k p_kl:
                                       log L = sum_kl [c_kl log(mu_k p_kl) - mu_k p_kl] (the data-only
                                       - log c_kl! left out); mu_k = trials[k] > 0, exact in FP32 (an
                                       integer below 2^24, for instance).  A setting's
                                       elements must be Hermitian with diagonals in [0, 1] summing to at
                                       most 1 (the checks a sub-normalised POVM passes; the caller
                                       supplies positive semidefinite elements summing to at most I) */
} qst_likelihood;

/* One tomography problem (Sec. III Steps 1-4).  All pointers are host memory,
 * read during qst_create only. */
typedef struct {
    int32_t num_qubits;     /* Q, 1..5 (D = 2^Q); 6 with QST_PREC_PAULI and the built-in POVMs (NULL) */
    int32_t num_povms;      /* K, the number of measurement settings (3^Q for Pauli) */
    const int32_t *counts;  /* [K*D] outcome counts c_kl >= 0, setting-major */
    const double *povm_re;  /* [K*D][D][D] row-major real parts of Lambda_kl; NULL together with
                               povm_im selects the built-in Pauli POVMs (qst_pauli_povms; K must
                               then be 3^Q) */
    const double *povm_im;  /* [K*D][D][D] imaginary parts */
    int64_t num_chains;     /* R >= 1 */
    int64_t chain_offset;   /* global id of chain 0 (disjoint ranges shard one run) */
    uint64_t seed;          /* Philox4x32-10 key */
    double beta0;           /* this problem's initial beta (Algorithm 2, initialisation); 0 = the config's beta0 */
    int32_t likelihood;     /* qst_likelihood: QST_LIKELIHOOD_MULTINOMIAL (0, the default) or _POISSON */
    const double *trials;   /* [K] expected trials mu_k per setting (QST_LIKELIHOOD_POISSON; NULL otherwise) */
} qst_problem_desc;

/* Sampler settings (Algorithm 2 and Sec. IV); qst_default_config fills the paper's values. */
typedef struct {
    double beta0;           /* initial pCN step beta (Algorithm 2 initialises it to 0.1) */
    int32_t adapt_interval; /* M_A (Sec. III: 500); 0 keeps beta fixed */
    double acc_lo, acc_hi;  /* acceptance window [0.2, 0.6] (Algorithm 2, adaptation tests) */
    double adapt_factor;    /* 1.1 (Algorithm 2, adaptation) */
    double beta_max;        /* 1.0: clamp keeping sqrt(1 - beta^2) real (the paper is silent) */
    int32_t thin;           /* T: keep every T-th state (Algorithm 2, thinning) */
    int32_t burn_in;        /* pool only steps j > burn_in (the paper uses none: 0) */
    int32_t diag_chains;    /* chains per problem whose kept states are stored for the ACF */
    int32_t traj_capacity;  /* kept states stored per diagnostic chain (Sec. IV: N = 2^10) */
    int32_t acf_lmax;       /* l_max of Eq. ACFrho / Eq. IACT (Fig. 2: 200) */
    int32_t trace_steps;    /* record the accept flag and log L(y') of the first trace_steps steps */
    int32_t precision;      /* qst_precision */
    int32_t qr_passes;      /* how U of Algorithm 1 (QR and phase fix) is computed: 1, one FP32 modified
                               Gram-Schmidt pass (U off by about cond(H) 2^-24); 2, that pass plus a
                               first-order FP32 re-orthogonalisation (orthogonal to ~2^-24, still off
                               by cond(H) 2^-24); 3 (default), the pass plus a first-order refinement
                               to the exact QR factor from Q1^dag H and Q1^dag Q1 formed without
                               rounding error (U within ~2^-24 of the exact factor).  Five and six
                               qubits take 2 when 3 is asked for; 4, as 3 and five qubits refined
                               too (their proposal kernel then takes about 2.3 times as long; six
                               qubits still take 2) */
    int32_t use_graph;      /* 1 (default): qst_run_chains replays one step captured as a CUDA graph
                               (the step counter lives on the device); 0: plain launches. Kernel
                               timing (qst_set_profiling) always uses plain launches */
    int32_t autotune;       /* 1 (default): qst_create times, for every problem, the projection with
                               each candidate number of column groups (the split of its N tiles
                               over CTAs) and, at 1-4 qubits with fewer chains than fill the GPU
                               twice, the proposal kernel with 128-, 64- and 32-thread CTAs, and
                               keeps the fastest of each (reported by qst_diagnostics); 0: fixed
                               rules */
    int32_t prior;          /* qst_prior: QST_PRIOR_BURES (0, the default) or QST_PRIOR_HS */
    int32_t propose_threads;/* 0 (default): the proposal kernel's CTA size at 1-4 qubits is 128 threads,
                               or the autotuner's pick; 32, 64 or 128: that size, untimed (the chains
                               are the same bits for every size) */
} qst_sampler_cfg;

/* Diagnostics of one problem (Sec. IV). */
typedef struct {
    int64_t steps_done;      /* steps j taken so far */
    int64_t num_pooled;      /* N R: samples in the pooled mean */
    int64_t num_kept;        /* N: kept states per chain */
    double accept_rate;      /* accepted / proposed, over all chains and steps */
    double beta_min, beta_mean, beta_max;
    int64_t num_nonfinite;   /* chains whose current log L is not finite */
    int32_t diag_chains;     /* chains whose tau was computed (0 if N <= l_max) */
    int32_t acf_lmax;
    double tau_mean;         /* mean over diagnostic chains of tau (Eq. IACT) */
    double tau_max;
    double n_eff;            /* N R / tau_mean (Sec. IV) */
    uint32_t device_status;  /* raw status bits */
    uint32_t column_groups;  /* column groups of the projection schedule in use (autotuned or fixed) */
    uint32_t propose_chains_per_cta;  /* chains per CTA of the proposal kernel (autotuned at 1-4 qubits) */
    uint32_t accept_chains_per_cta;   /* chains per CTA of the accept kernel (one pooled-sum slot each) */
    int32_t projection_form;          /* qst_precision of the projection in use (QST_PREC_AUTO picks one) */
    int32_t qr_passes;                /* the QR form this problem's proposal runs (qst_sampler_cfg.qr_passes
                                         resolved for its size: 3 = refined, 2 = first-order, 0 = none) */
} qst_diag;

typedef struct qst_handle qst_handle;

/* Kernel kinds for the profiling counters. */
typedef enum {
    QST_KERNEL_PROPOSE = 0,  /* Philox, pCN proposal, Algorithm 1, packing */
    QST_KERNEL_PROJECT = 1,  /* projector contraction + log-likelihood epilogue */
    QST_KERNEL_ACCEPT = 2,   /* accept test, adaptation, write-back, pooling, trajectories */
    QST_KERNEL_DIAG = 3,     /* ACF / IACT and pooled-mean reductions */
    QST_KERNEL_KINDS = 4
} qst_kernel_kind;

/* ---- status and configuration -------------------------------------------------------- */

const char *qst_status_string(qst_status status);
/* Message of the last failing call on this thread ("" if none). */
const char *qst_last_error(void);
/* Fills cfg with the paper's settings: beta0 0.1, M_A 500, window [0.2, 0.6], factor 1.1,
 * beta_max 1, T 1, no burn-in, 256 diagnostic chains, capacity 1024, l_max 200, FP32,
 * qr_passes 3 (one Gram-Schmidt pass and the refinement), graphs and the autotuner on. */
void qst_default_config(qst_sampler_cfg *cfg);

/* ---- lifecycle ---------------------------------------------------------------------- */

/* Device bytes qst_create needs for these problems and settings.
 * Errors: QST_ERR_INVALID_ARG for an invalid problem or setting (see qst_create). */
qst_status qst_workspace_size(const qst_problem_desc *problems, int32_t num_problems,
                              const qst_sampler_cfg *cfg, size_t *bytes);

/* Validates the problems (Sec. III Step 1: counts >= 0; each Lambda_kl Hermitian and
 * sum_l Lambda_kl = I to 1e-12; Q in 1..5, or 6 for QST_PREC_PAULI with NULL POVM arrays; R >= 1;
 * T >= 1; 0 < beta0 <= beta_max <= 1 for the
 * config's and every problem's own beta0 (0 meaning the config's);
 * for the tensor-core precisions every packed projector entry exactly representable in
 * bf16 (QST_PREC_BF16X3) or TF32 (QST_PREC_TF32, QST_PREC_TF32X2), and Q within the
 * precision's range; for QST_PREC_PAULI the 3^Q Pauli settings of qst_pauli_povms:
 * QST_ERR_INVALID_ARG otherwise),
 * packs the projectors, uploads everything into the workspace and enqueues the chains'
 * initial states y^0 ~ N(0, I) with rho(y^0) and log L(y^0) (Algorithm 2, initialisation).
 * d_workspace: device memory of at least qst_workspace_size bytes, 256-byte aligned,
 * owned by the caller and kept alive until qst_destroy; NULL makes the library
 * allocate (and later free) it itself.  cuda_stream: a cudaStream_t (NULL = default).
 * The problem descriptions are copied; the caller may free them on return. */
qst_status qst_create(const qst_problem_desc *problems, int32_t num_problems, const qst_sampler_cfg *cfg,
                      void *d_workspace, size_t workspace_bytes, void *cuda_stream, qst_handle **out);

/* Enqueues num_steps steps j -> j+1 of Algorithm 2 for every chain of every problem
 * (proposal, Algorithm 1, likelihood, accept, adaptation, thinning and pooling).
 * Asynchronous on the handle's stream; resumable (step numbering continues).
 * A step is one small kernel that advances the device-side step counter, then the
 * proposal, projection and accept kernels of every problem.  With use_graph the first
 * call captures that sequence once (on private streams, the problems of a handle on up
 * to eight parallel branches, since they are independent) and every step launches the
 * graph; the results are bit-identical to plain launches.
 * Errors: QST_ERR_INVALID_ARG if num_steps < 0. */
qst_status qst_run_chains(qst_handle *h, int64_t num_steps);

/* Pooled posterior mean rho^{N,R} of Eq. BME2 / Step 6 for one problem, as row-major
 * host arrays rho_re[D*D], rho_im[D*D] (caller-owned), and the sample count N R.
 * Synchronises the stream.  Errors: QST_ERR_STATE if nothing has been pooled yet. */
qst_status qst_posterior_mean(qst_handle *h, int32_t problem, double *rho_re, double *rho_im,
                              int64_t *num_pooled);

/* The sum behind that mean, unnormalised: the FP64 sum over every kept state of one problem of
 * its packed vec_h(rho) (Eq. BME2's numerator), sum_packed host [D*D] doubles in the packed
 * layout of the header comment (caller-owned), and the count N R.  Sums from runs over
 * disjoint chain ranges add to the sum of one run over all of them (each state is summed in
 * FP64 once), which is how replicas on several GPUs are merged.  Synchronises the stream.
 * Errors as qst_posterior_mean. */
qst_status qst_posterior_sum(qst_handle *h, int32_t problem, double *sum_packed, int64_t *num_pooled);

/* Diagnostics of one problem (Sec. IV): acceptance, beta statistics, the chain-averaged
 * ACF c[0..l_max] of Eq. ACFrho into acf (host, l_max+1 doubles, may be NULL) and the
 * per-chain IACT tau of Eq. IACT into tau (host, diag_chains doubles, may be NULL).
 * Synchronises the stream. */
qst_status qst_diagnostics(qst_handle *h, int32_t problem, qst_diag *out, double *acf, double *tau);

/* Waits for the handle's work and reports device status bits. */
qst_status qst_synchronize(qst_handle *h);

/* Releases the handle (and the workspace if the library allocated it). */
void qst_destroy(qst_handle *h);

/* ---- state access, checkpoint, restore ----------------------------------------------- */

/* Copies the current chain states of one problem to host arrays (each may be NULL):
 * y [R][4 D^2] float, logl [R] double, beta [R] double, accepts [R] int64 (accepted
 * proposals so far).  Synchronises. */
qst_status qst_get_state(qst_handle *h, int32_t problem, float *y, double *logl, double *beta,
                         int64_t *accepts);

/* Accept flags [trace_steps][R] (uint8) and log L(y') [trace_steps][R] of the first
 * cfg.trace_steps steps (host, each may be NULL).  Synchronises. */
qst_status qst_get_trace(qst_handle *h, int32_t problem, uint8_t *accept, double *logl_prop);

/* Size of, writing of and reading of a host checkpoint of every chain state, pooled sum,
 * trajectory and step counter.  Philox streams are counter-based, so a restored handle
 * continues bit-identically.  qst_restore needs a handle created with the same problems
 * and settings.  Both synchronise. */
qst_status qst_checkpoint_size(qst_handle *h, size_t *bytes);
qst_status qst_checkpoint(qst_handle *h, void *buffer, size_t bytes);
qst_status qst_restore(qst_handle *h, const void *buffer, size_t bytes);

/* ---- stateless evaluation ---------------------------------------------------------------- */

/* For n latent vectors x (device, [n][4 D^2] float), computes rho(x) of Algorithm 1 as
 * packed vec_h (device [n][D^2] float, may be NULL), the outcome probabilities
 * p_kl = Tr Lambda_kl rho (device [n][K D] float, may be NULL) and log L(x) of
 * Eq. likelihood (device [n] double, may be NULL), with the handle's precision.
 * Uses the problem's proposal buffers as scratch: call it between qst_run_chains calls,
 * not concurrently with them.  Errors: QST_ERR_INVALID_ARG if n < 0 or n > R. */
qst_status qst_evaluate(qst_handle *h, int32_t problem, const float *x, int64_t n, float *rho, float *p,
                        double *logl);

/* ---- profiling ---------------------------------------------------------------------------- */

/* Enables (1) or disables (0) CUDA-event timing of every kernel launch on the stream. */
qst_status qst_set_profiling(qst_handle *h, int32_t enabled);
/* Total device milliseconds and launch count of one kernel kind since the last reset
 * (synchronises); reset != 0 zeroes the counters afterwards. */
qst_status qst_kernel_time(qst_handle *h, int32_t kind, int32_t reset, double *total_ms, int64_t *launches);
/* Kernel launches the handle has enqueued since creation. */
int64_t qst_launch_count(const qst_handle *h);

/* ---- test hooks ---------------------------------------------------------------------------- */

/* Raw Philox4x32-10 words: for chains chain0..chain0+nchains-1 and blocks
 * block0..block0+nblocks-1 of the stream (seed, step, tag), writes
 * out[((c - chain0) * nblocks + (b - block0)) * 4 + w] (device uint32).
 * Counter = (block, step, chain, tag), key = (seed low, seed high). */
qst_status qst_philox_blocks(uint64_t seed, uint32_t step, uint32_t tag, uint32_t chain0, int64_t nchains,
                             uint32_t block0, int32_t nblocks, uint32_t *out, void *cuda_stream);

/* The built-in Pauli POVMs of Q qubits (1..5; at 6 the arrays would take 3 GB), written to host arrays povm_re, povm_im of
 * [3^Q 2^Q][2^Q][2^Q] doubles (caller-owned): setting k = sum_q s_q 3^(Q-1-q) with s = 0, 1, 2
 * for X, Y, Z; outcome l = sum_q b_q 2^(Q-1-q) with b = 0 for the +1 eigenvalue; qubit 0 is the
 * most significant Kronecker factor (Sec. IV: all 3^Q Pauli settings).  Host-only.
 * QST_ERR_INVALID_ARG for Q outside 1..5 or a NULL array. */
qst_status qst_pauli_povms(int32_t num_qubits, double *povm_re, double *povm_im);

/* Packs the POVM elements into the real [D^2][K D] matrix P with p = vec_h(rho) . P:
 * P[(i,i), kl] = Re Lambda_ii, P[(i,j), kl] = 2 Re Lambda_ij (i < j), 2 Im Lambda_ij (i > j).
 * Host-only.  P_out: host [D^2][K D] float. */
qst_status qst_pack_projectors(int32_t num_qubits, int32_t num_povms, const double *povm_re,
                               const double *povm_im, float *P_out);

/* Fault injection: sets the current latent state of one chain to NaN, so every later
 * proposal has a non-finite log-likelihood and is rejected; the chain keeps (and keeps
 * pooling) its last valid rho.  Device-side only, asynchronous. */
qst_status qst_inject_nan(qst_handle *h, int32_t problem, int64_t chain);

/* Failure-path probe (test hook): runs, on the handle's stream, one warp that waits through
 * the kernels' own bounded mbarrier wait on a barrier nothing ever completes, with a limit of
 * wait_ms milliseconds (1..2000) instead of the kernels' 1 s.  The wait gives up, sets the
 * device status word's time-out bit and the kernel returns, so the context stays usable.
 * Synchronises; returns what the next synchronising call would report, QST_ERR_TIMEOUT, then
 * clears the bit it set.  If the status word already holds a failure, that failure is
 * returned and nothing is cleared.  QST_ERR_INVALID_ARG for a NULL handle or wait_ms out of
 * range. */
qst_status qst_probe_wait_timeout(qst_handle *h, int32_t wait_ms);

/* ---- evaluation without device allocation ---------------------------------------------------- */

/* The paper has no counterpart to this entry point: it serves callers that must not
 * allocate device memory on their call path -- a library or plugin whose host application
 * owns the device memory through its own allocator, or an asynchronous pipeline that
 * cannot afford cudaMalloc/cudaFree, which may synchronise the whole device.
 *
 * qst_loglik_noalloc returns, for n latent vectors x, the same log-likelihood that
 * qst_evaluate returns with QST_PREC_FP32 and the default configuration (the same
 * density-matrix assembly, FP32 projector contraction and FP64 reduction), but needs
 * no handle and no workspace: its intermediates live in one device array of
 * QST_NOALLOC_SCRATCH_BYTES (about 5.8 MiB) defined in the library, which every GPU that
 * loads the library holds until the process exits.
 *   num_qubits  Q, 1..4
 *   num_povms   K, with K * 2^Q <= 1408 (all 81 Pauli settings of 4 qubits fit)
 *   P           device [D^2][K D] float: the packed projector matrix, as qst_pack_projectors
 *               produces it; caller-owned, read by the enqueued work
 *   counts      host [K D] int32 outcome counts c_kl >= 0; read before the call returns
 *   x           device [n][4 D^2] float latent vectors (layout as in the header comment)
 *   n           0 <= n <= QST_NOALLOC_MAX_ROWS rows per call (larger batches: call again)
 *   logl        device [n] double, written
 *   cuda_stream cudaStream_t the work is enqueued on (NULL = default stream)
 * Returns QST_ERR_INVALID_ARG for a size beyond these limits, a NULL pointer or a negative
 * count, before anything is enqueued; QST_ERR_CUDA for a CUDA failure (message in
 * qst_last_error()).  It calls no cudaMalloc, cudaFree or other allocating routine and does
 * not wait for the device: the weights formed from the counts travel as kernel launch
 * parameters, so no host buffer is read after the call returns.  The first call on a device
 * (with that device current) looks up the scratch array's device address once; make that
 * first call before any stream capture.  All calls share the one scratch array, which keeps
 * the previous call's contents (each call rewrites what it reads): calls that can overlap on
 * the GPU -- on different streams without ordering between them -- race and must be
 * serialised by the caller. */
#define QST_NOALLOC_MAX_ROWS 4096
#define QST_NOALLOC_SCRATCH_BYTES 6043392
qst_status qst_loglik_noalloc(int32_t num_qubits, int32_t num_povms, const float *P, const int32_t *counts,
                              const float *x, int64_t n, double *logl, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* QST_H */
