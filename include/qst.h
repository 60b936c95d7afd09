/*
 * qst.h — C ABI of the B300 (sm_103a) forward/adjoint library for
 * rank-adaptive matrix-free atomic quantum state tomography with local Pauli
 * measurements.
 *
 * Model (Sec. II): rho = Psi diag(w) Psi^*  (Eq. atomic-density) with K atoms
 * psi_k in C^D, D = 2^n, and weights w on the simplex.  Measurements (Sec. IV):
 * M settings, each a Pauli string b_s in {X,Y,Z}^n, with
 * E_{s,u} = (1/B) V_s^* |u><u| V_s, V_s = V_{b_1} (x) ... (x) V_{b_n}.
 *
 * Conventions shared by every entry point:
 *   - Basis codes: 0 = Z, 1 = X, 2 = Y.  V_X = (1/sqrt2)[[1,1],[1,-1]],
 *     V_Y = (1/sqrt2)[[1,-i],[1,i]] (outcome bit 0 <-> eigenvalue +1).
 *   - Qubit 1 (basis[s][0]) is the most significant bit of the outcome index.
 *   - Complex numbers are interleaved (re, im) float32 pairs ("complex64").
 *   - Counts are CSR: row_ptr[M+1] (int64, row_ptr[0] = 0, non-decreasing,
 *     row_ptr[M] = nnz), outcome[nnz] (uint32, < D, STRICTLY INCREASING inside
 *     each row), count[nnz] (uint32), shots[M] (uint32, N_s, > 0 for every
 *     non-empty row).
 *   - pi = p / B and pihat = N_{s,u} / (B N_s), where B is
 *     qst_params.norm_settings (0 means B = M).
 *   - Every pointer argument of a compute call is caller-owned DEVICE memory
 *     unless the entry point says "host".  The library never takes ownership.
 *   - Compute calls are asynchronous on the given stream (a cudaStream_t passed
 *     as void*; NULL = legacy default stream).  Host-side argument errors return
 *     immediately; errors found on the device (bad data, non-finite results)
 *     are OR-ed into the plan's device status word, read with qst_plan_status.
 *   - A plan is not thread-safe: calls on one plan must be serialised by the
 *     caller (they share the plan's workspace).
 */
#ifndef QST_H
#define QST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qst_status {
    QST_OK = 0,
    QST_ERR_INVALID_ARG = 1, /* bad size, NULL where required, misaligned pointer */
    QST_ERR_UNSUPPORTED = 2, /* size outside what this build handles (see qst_plan_create) */
    QST_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    QST_ERR_NO_MEMORY = 4,   /* workspace allocation failed */
    QST_ERR_DEVICE = 5,      /* qst_plan_status found device-side error bits */
    QST_ERR_SCRATCH_TOO_SMALL = 6 /* qst_adjoint_noalloc: problem needs more than its scratch */
} qst_status;

/* Bits of the device status word. */
#define QST_DEV_BAD_BASIS    1  /* a basis code > 2 (treated as Z) */
#define QST_DEV_BAD_CSR      2  /* row_ptr / outcome malformed (range, order) */
#define QST_DEV_BAD_SHOTS    4  /* shots[s] == 0 for a non-empty row */
#define QST_DEV_NONFINITE    8  /* the loss is NaN or Inf */
#define QST_DEV_TIMEOUT     16  /* a kernel's bounded wait on its own bulk copies or MMAs ran out (the
                                   tensor-core kernels, the n = 20 single-setting kernels); the kernel
                                   stopped issuing work and returned, results are invalid */

typedef struct qst_params {
    double eps;           /* epsilon of Eq. qst-loss (default 1e-8) */
    int norm_settings;    /* B; 0 = M (default 0) */
    int chunk_qubits;     /* low qubits transformed on-chip per work unit; 0 = auto (min(n, 12) for
                             n <= 16, n - 8 for n = 17..20).  n = 17..20 also takes 16: 16-qubit chunks
                             on clusters of 8 CTAs (distributed shared memory between them), settings
                             binned by the n - 16 high qubits (see fixed_rounds = 4) */
    int max_bin_settings; /* cap on settings per work bin; 0 = auto */
    int validate;         /* 1 = check basis and CSR on the device (default 1) */
    int reg_bits;         /* amplitudes per thread per round = 2^reg_bits: 4 or 5; 0 = auto */
    int fixed_rounds;     /* chunk kernels.  12-qubit chunks: 2 = two rounds of six qubits, 64
                             amplitudes per thread, two atoms per CTA (one shared-memory exchange per
                             setting in the forward, two in the adjoint; n <= 16 only, n = 17..20
                             runs 1); 1 = three rounds of four qubits on fixed qubit groups, 16
                             amplitudes per thread (compile-time shared-memory offsets, warp-local
                             middle exchange).  Whole states of 10, 11 qubits: 2 = the same two
                             rounds with 2^(n-6) threads per atom (2^(13-n) atoms per CTA).
                             States of 5..9 qubits held in one chunk: 3 = one
                             warp per (bin, atom), 2^(n-5) amplitudes per lane, the low five bits'
                             butterflies by lane shuffles (QST_ERR_UNSUPPORTED for other plans).
                             0 = rounds chosen per setting (one CTA per (bin, atom)).  16-qubit
                             chunks (n = 17..20): 4 = a cluster of 8 CTAs per (bin, high pattern,
                             atom), each CTA two 12-qubit rows in two rounds of six qubits, then a
                             round of the top four chunk qubits over the cluster (asking for 4
                             selects these chunks; they take no other value).  -1 = automatic: 3
                             for whole states of 5..9 qubits, 4 for 16-qubit chunks, 2 for whole
                             states of 10, 11 qubits, for 12-qubit chunks 2 when a work bin may
                             hold >= 32 settings, else 1.  Other
                             values: QST_ERR_INVALID_ARG.  Default -1. */
    int phi_cache;        /* qst_evaluate's transform cache: the forward stores the transform of every
                             atom at every observed outcome (K x nnz complex64, owned by the plan) and
                             the adjoint then runs its inverse rounds only (on the n = 20 path it also
                             skips the high-bit pass before them).  Two-round plans, the n = 20
                             path (12-qubit chunks) and 16-qubit chunks.  1 = on
                             (QST_ERR_UNSUPPORTED for other plans), 0 = off, -1 = automatic: on for
                             two-round plans when K x nnz x 8 bytes <= 16 GiB (for whole states of
                             10, 11 qubits only when nnz <= M 2^n / 4: with denser outcomes the
                             cache costs more than recomputing) and for 16-qubit chunks, off on the
                             n = 20 path (whose adjoint recomputes the rotated amplitudes unless
                             asked).  qst_forward and qst_adjoint never use it
                             (16-qubit chunks: their adjoint kernel reads transforms, and
                             qst_adjoint first recomputes them with the forward kernel into the
                             plan's buffer, which those plans always hold).  Default -1. */
    int precision;        /* arithmetic of the 12-qubit chunk transforms of two-round plans (n = 12..16
                             with fixed_rounds resolving to 2).  0 = FP32 butterflies on the SIMT
                             pipes (default).  1, 2, 3 = the transform as two dense products over
                             groups of q = 6 qubits on the tensor cores (tcgen05.mma kind::f16):
                             operators exact in BF16 (entries 0, +-1 before the 2^-m/2 scale), the
                             data split into `precision` BF16 terms, FP32 accumulation in tensor
                             memory.  Per amplitude and step the data error is <= 2^-8 precision
                             times the amplitude (precision = 3 carries all 24 bits of FP32).
                             precision > 0 on other plans: QST_ERR_UNSUPPORTED; outside 0..3:
                             QST_ERR_INVALID_ARG.  The plan then also holds the 729 group operators
                             (24 MB) and a K x nnz complex64 transform buffer: without the
                             transform cache the adjoint first recomputes the transforms with the
                             tensor-core forward. */
} qst_params;

typedef struct qst_plan_s *qst_plan;

/* Fill *p with the defaults above. */
void qst_params_default(qst_params *p);

/* Human-readable name of a status code (static string). */
const char *qst_status_string(qst_status s);

/*
 * Create a plan for one problem shape: n qubits (1 <= n <= 20 in this build;
 * n <= 16 bins settings by their high-bit pattern, n = 17..20 applies the 8
 * high-bit factors by butterfly passes per setting group, or with 16-qubit
 * chunks on CTA clusters bins settings by their n - 16 high bits),
 * M >= 1 settings, K >= 1 atoms, nnz >= 0 observed (setting, outcome) pairs.
 * Allocates the device workspace (owned by the plan, freed by
 * qst_plan_destroy) on the current CUDA device.  params may be NULL.
 */
qst_status qst_plan_create(qst_plan *plan, int n, int M, int K, int64_t nnz,
                           const qst_params *params);
qst_status qst_plan_destroy(qst_plan plan);

/* Bytes of device workspace the plan holds. */
qst_status qst_plan_workspace_bytes(qst_plan plan, int64_t *bytes);

/* The plan's chunk geometry: qubits transformed on-chip per work unit, high
 * qubits applied outside the chunk (by setting bins, or by butterfly passes
 * on the n = 17..20 wide path), and which chunk kernels run: 4 = 16-qubit
 * chunks on CTA clusters, 3 = a warp per (bin, atom), 2 = two 6-qubit rounds,
 * 1 = three fixed 4-qubit rounds, 0 = rounds chosen per setting.  Any output
 * pointer may be NULL.  Host only. */
qst_status qst_plan_geometry(qst_plan plan, int *chunk_qubits, int *high_qubits, int *fixed_rounds);

/*
 * Forward pass (Eqs. atom-response, atomic-born-map, qst-loss,
 * likelihood-ratio-vector):
 *   p_{s,u} = sum_k w_k |(V_s psi_k)_u|^2,   pi = p / B,
 *   c_{s,u} = pihat_{s,u} / (pi_{s,u} + eps) at observed outcomes,
 *   L = - sum_{observed} pihat log(pi + eps).
 * Inputs:  psi [K][D] complex64, w [K] float32, basis [M][n] uint8, CSR counts.
 * Outputs (each may be NULL): p_obs [nnz] float32 (p at observed outcomes),
 *   c_obs [nnz] float32, loss [1] float64, p_dense [M][D] float32 (every
 *   outcome; for tests and small problems).
 * Pointers must be 16-byte aligned for psi and 4-byte aligned otherwise.
 */
qst_status qst_forward(qst_plan plan, const float *psi, const float *w,
                       const uint8_t *basis, const int64_t *row_ptr,
                       const uint32_t *outcome, const uint32_t *count,
                       const uint32_t *shots, float *p_obs, float *c_obs,
                       double *loss, float *p_dense, void *stream);

/*
 * Adjoint pass (Eqs. negative-gradient-product, atom-wirtinger-gradient,
 * weight-gradient):
 *   (G psi_k) = (1/B) sum_s V_s^* (c_s .* (V_s psi_k)),
 *   grad_psi_k = dJ/dpsi_k^* = -w_k G psi_k,
 *   grad_w_k   = dJ/dw_k     = -h_k,  h_k = (1/B) sum_{s,u} c_{s,u} |(V_s psi_k)_u|^2.
 * c_obs [nnz] is the likelihood ratio at observed outcomes (as written by
 * qst_forward); c is zero at every other outcome.  The rotated amplitudes are
 * recomputed, not stored.  Outputs: grad_psi [K][D] complex64 (required),
 * grad_w [K] float32 (may be NULL).  With w_k = -1 for every k, grad_psi is
 * G psi_k itself (the G v product used by spectral steps).
 */
qst_status qst_adjoint(qst_plan plan, const float *psi, const float *w,
                       const uint8_t *basis, const int64_t *row_ptr,
                       const uint32_t *outcome, const float *c_obs,
                       float *grad_psi, float *grad_w, void *stream);

/*
 * Forward and adjoint of one evaluation in one call (Eqs. atomic-born-map,
 * qst-loss, likelihood-ratio-vector, then negative-gradient-product,
 * atom-wirtinger-gradient, weight-gradient): the outputs of qst_forward
 * (p_obs and loss may be NULL; c_obs is required and receives c) followed by
 * those of qst_adjoint with that c, all device pointers, asynchronous on
 * `stream`.  With the plan's transform cache (qst_params.phi_cache) the
 * forward stores the rotated amplitudes at the observed outcomes and the
 * adjoint applies only the inverse rotations to c .* (V_s psi_k) instead of
 * recomputing V_s psi_k (the paper's optional response storage, Sec. III-B,
 * kept for the observed outcomes only); the results agree with separate
 * qst_forward / qst_adjoint calls within rounding.  Without the cache it is
 * exactly those two calls.  Same errors as qst_forward and qst_adjoint.
 */
qst_status qst_evaluate(qst_plan plan, const float *psi, const float *w, const uint8_t *basis,
                        const int64_t *row_ptr, const uint32_t *outcome, const uint32_t *count,
                        const uint32_t *shots, float *p_obs, float *c_obs, double *loss,
                        float *grad_psi, float *grad_w, void *stream);

/*
 * Forward then adjoint from HOST buffers: copies the inputs to plan-owned
 * device buffers, runs qst_evaluate on the stream, copies
 * loss [1], grad_psi [K][D] complex64 and grad_w [K] back to the host buffers,
 * and synchronises the stream.  Every pointer here is host memory (pinned
 * memory gives asynchronous copies).  c_obs_out [nnz] may be NULL.
 */
qst_status qst_evaluate_host(qst_plan plan, const float *psi, const float *w,
                             const uint8_t *basis, const int64_t *row_ptr,
                             const uint32_t *outcome, const uint32_t *count,
                             const uint32_t *shots, double *loss_out,
                             float *grad_psi_out, float *grad_w_out,
                             float *c_obs_out, void *stream);

/*
 * Projected descent direction of every atom (Sec. III-A, Eq.
 * atom-projected-descent-direction): d_k = w_k (I - psi_k psi_k^*) G psi_k,
 * formed from qst_adjoint's outputs as d_k = -grad_k + w_k grad_w_k psi_k
 * (grad_k = -w_k G psi_k, grad_w_k = -h_k with h_k = <psi_k|G psi_k>
 * accumulated in FP64 by the adjoint).  For a unit-norm psi_k, d_k is
 * orthogonal to psi_k.
 *   psi, grad_psi [K][2^n] complex64, w, grad_w [K] float32 (device, read)
 *   d [K][2^n] complex64 (device, written; may alias grad_psi)
 * One elementwise kernel on the stream (memory-bound).
 */
qst_status qst_tangent(qst_plan plan, const float *psi, const float *w, const float *grad_psi,
                       const float *grad_w, float *d, void *stream);

/* Synchronise the device and read (then clear) the plan's device status word.
 * Returns QST_ERR_DEVICE if any bit was set (bits in *device_status). */
qst_status qst_plan_status(qst_plan plan, int *device_status);

/* Kernel launch accounting.  Every launch the plan issues is counted.  With
 * timing enabled, each launch is bracketed by CUDA events on its stream;
 * qst_plan_kernel_stats synchronises on them and returns, per kernel kind,
 * the number of timed launches and their summed device time in ms. */
enum {
    QST_KERNEL_PACK = 0,
    QST_KERNEL_VALIDATE = 1,
    QST_KERNEL_FORWARD = 2,
    QST_KERNEL_LOSS = 3,
    QST_KERNEL_ADJOINT = 4,
    QST_KERNEL_REDUCE = 5,
    QST_KERNEL_HSUM = 6,
    QST_KERNEL_EPILOGUE = 7,
    QST_KERNEL_REFACTOR = 8,
    QST_KERNEL_STEP = 9,
    QST_KERNEL_HIGH = 10,
    QST_KERNEL_TANGENT = 11,
    QST_KERNEL_KINDS = 12
};
qst_status qst_plan_set_timing(qst_plan plan, int enable);
qst_status qst_plan_kernel_stats(qst_plan plan, int64_t *launches, double *ms,
                                 int kinds);
qst_status qst_plan_reset_stats(qst_plan plan);
/* Total kernel launches issued by this plan since creation / last reset. */
qst_status qst_plan_launch_count(qst_plan plan, int64_t *count);

/*
 * Euclidean projection onto the probability simplex followed by the
 * truncation map P_tau (Eq. coefficient-update's proj_Delta; Eq.
 * truncation-map): beta = max(v - theta, 0) with theta chosen so that
 * sum beta = 1 (sort-based exact method), then entries with beta_r <= tau are
 * dropped and the rest renormalised; if none survives, the largest is kept.
 *   v [K] double (device, read), 1 <= K <= 1024
 *   beta [K] double (device, written): renormalised kept weights, 0 elsewhere
 *   keep [K] int (device, written): kept indices in ascending order, first *K_out valid
 *   K_out [1] int (device, written)
 * FP64 throughout; one CTA.  Needs no plan and no workspace.
 */
qst_status qst_simplex_project(const double *v, int K, double tau, double *beta,
                               int *keep, int *K_out, void *stream);

/*
 * Exact spectral refactorisation of rho = Psi diag(w) Psi^*: the paper's
 * spectral step (Sec. III-C, Eqs. ritz-pairs, spectral-candidates) with
 * eta_rho = 0, where its Ritz pairs are exact eigenpairs of rho_t.  Through the
 * K x K Gram matrix H = diag(sqrt w) Psi^* Psi diag(sqrt w) = V Lambda V^* (FP64,
 * cyclic Jacobi on the GPU), the new atoms are
 * phi_j = Psi diag(sqrt w) v_j / sqrt(lambda_j) (orthonormal, FP32 combination)
 * with weights lambda_j / sum(lambda), sorted descending, then P_tau (as in
 * qst_simplex_project).  In place: psi [K][2^n] complex64 and w [K] float32
 * (device) receive the K' kept atoms/weights in their first K' slots; the
 * remaining slots get zero atoms and zero weights (a zero weight removes an
 * atom from the forward and adjoint).  K_out [1] int (device) receives K'.
 * The plan's K must be <= 32.
 */
qst_status qst_refactor(qst_plan plan, float *psi, float *w, double tau,
                        int *K_out, void *stream);

/*
 * One slot of the master loop of Algorithm 1 (Sec. III-C) on the state
 * (psi [K][2^n] complex64, w [K] float32; device, updated in place when the
 * proposal is accepted).  Atoms with w_r = 0 are inactive (not part of the
 * state); R counts the atoms with w_r > 0.
 *   slot 0 (T_psi): atom r; direction g = w_r (I - psi_r psi_r^*) G psi_r
 *          (Eq. atom-direction), trial (psi_r + eta g) / ||psi_r + eta g||
 *          (Eq. atom-trial).
 *   slot 1 (T_alpha): beta = proj_Delta(w + eta h) over the active atoms with
 *          h = A^T c (Eqs. h_t, coefficient-update), then P_tau.
 *   slot 2 (T_rho): the exact spectral refactorisation of rho_t (qst_refactor;
 *          the spectral step with eta_rho = 0), then P_tau; one proposal.
 *   slot 3 (T_rho): the spectral step of Sec. III-C with eta_rho from the step
 *          grid: Ritz pairs of S_t = rho_t + eta G_t (Eqs. density-proposal,
 *          density-product, ritz-pairs) from a block Krylov space started at
 *          the atoms (blocks of K vectors, one adjoint per block, full
 *          reorthogonalisation, at most n_krylov vectors), then the candidates
 *          P_tau(proj_Delta(lambda_1..s), Phi_s), s = 1..min(K, m), scored by
 *          Q_t (Eq. proximal-surrogate, evaluated through the Ritz values) and
 *          the best one proposed (Eq. spectral-selection).  Needs K <= 16 and
 *          n <= 16.
 * Step sizes (slots 0, 1, 3): eta = eta0 * eta_ratio^j, j = 0 .. n_eta-1, tried
 * from largest to smallest; the first proposal with
 * J(X~) <= J_t - tau_acc (Eq. state-acceptance-rule) is kept, where
 * J = L_eps + mu R (Eq. fixed-rank-objective).  Defaults (Table I): mu = 1e-3,
 * tau = 1e-3, tau_acc = 1e-10, grid {2^-j}, j = 0..10.
 * Host outputs: *J_out (J of the resulting state), *accepted (0/1),
 * *eta_used.  The call synchronises the stream (it reads each trial's loss).
 * Data arguments as in qst_forward.
 */
typedef struct qst_step_params {
    double mu, tau, tau_acc, eta0, eta_ratio;
    int n_eta;
    int n_krylov;  /* Krylov vectors of the spectral step (Table I: at most 30; default 30) */
    int rank_fix;  /* spectral step: 0 = the candidate with the least Q_t (default); R > 0 = only the
                      candidate with min(R, L_t) Ritz pairs (the known-rank variant of Sec. IV's
                      ablation), which P_tau may still prune */
} qst_step_params;
void qst_step_params_default(qst_step_params *sp);
qst_status qst_step(qst_plan plan, int slot, int r, float *psi, float *w,
                    const uint8_t *basis, const int64_t *row_ptr,
                    const uint32_t *outcome, const uint32_t *count,
                    const uint32_t *shots, const qst_step_params *params,
                    double *J_out, int *accepted, double *eta_used, void *stream);

/*
 * T iterations t = t0 .. t0 + T - 1 of Algorithm 1 (Sec. III-D) on the state
 * (psi, w), with every decision taken on the device and no host
 * synchronisation inside.  Iteration t is a refactor slot when T_ref > 0 and
 * (t + 1) mod T_ref == 0, else a coefficient slot when (t + 1) mod
 * T_alpha == 0, else an atom slot on r_t = the (s mod R_t)-th atom with
 * w > 0, s counting the atom slots since t = 0 (the cyclic choice; a run with
 * t0 > 0 continues the count of the previous run on this plan).  Each slot
 * does what qst_step does for that slot (same kernels, same step grid, first
 * accepted trial kept), so a run equals the matching sequence of qst_step
 * calls exactly.
 *   J_hist [T] double (device, written): J = L_eps + mu R after each iteration
 *   accepted_hist [T] int (device, written, may be NULL): 1 if the iteration moved
 * The whole launch sequence (packing, the starting J, then per iteration
 * adjoint, trials, forwards, acceptance, commit) is captured into a CUDA graph
 * on the first call with given pointers, T, t0 schedule and parameters, and
 * replayed on the stream afterwards.  Settings and counts must not change
 * between replays without new pointers.  n <= 16 (binned path); refactor
 * slots need K <= 32.
 */
typedef struct qst_iter_params {
    qst_step_params step;  /* mu, tau, tau_acc, step grid (qst_step_params_default) */
    int T_alpha;           /* coefficient slots: (t + 1) mod T_alpha == 0 (default 5) */
    int T_ref;             /* refactor slots: (t + 1) mod T_ref == 0 (default 50; 0 = never) */
    int delta_window;      /* stopping rule (Table I, delta_20): after accepted update i, stop when
                              (J_{i-w} - J_i) / |J_{i-w}| < delta_tol over the last w accepted updates
                              (default 20; 0 = off; at most 63) */
    double delta_tol;      /* default 1e-4 */
    long long max_oracle_calls; /* stopping rule N_oracle: stop once the serial-equivalent oracle calls
                              reach this count (default 1e5; 0 = off).  One call is one primitive of
                              Sec. III-B over all outcomes for one atom (a response, G v) or one loss /
                              A^T c evaluation, as Algorithm 1 issues them: the starting state costs
                              R + 1; an atom slot 1 + 2 per trial; a coefficient slot 1 + 1 per trial;
                              a refactor slot (new atoms) + 1; a spectral slot, per trial, K per Krylov
                              block (G on the block), the new atoms + 1.  A trial count is the accepted
                              trial's index + 1, or the whole grid when none is accepted. */
    int spectral;          /* T_rho slots: 0 = the exact refactor (qst_refactor, eta_rho = 0) inside the
                              graph (default); 1 = the spectral step of Sec. III-C (qst_step slot 3): the
                              iterations between T_rho slots run as graph segments (one graph replayed
                              for every segment with the same slots) and each T_rho slot runs qst_step
                              slot 3 on the stream, its J, acceptance and oracle calls entering the same
                              history and stopping rules; the host synchronises at those slots (the
                              Krylov block sizes are read there).  Needs what qst_step slot 3 needs
                              (K <= 16, n <= 16); a run stopped by a rule skips the step. */
} qst_iter_params;
void qst_iter_params_default(qst_iter_params *ip);
qst_status qst_iterate(qst_plan plan, int T, int t0, float *psi, float *w,
                       const uint8_t *basis, const int64_t *row_ptr,
                       const uint32_t *outcome, const uint32_t *count,
                       const uint32_t *shots, const qst_iter_params *params,
                       double *J_hist, int *accepted_hist, void *stream);

/*
 * State of the plan's device iteration after the last qst_iterate (waits for
 * the device): whether a stopping rule has fired (iterations after it leave
 * the state unchanged, their J_hist entries repeat J and their accepted_hist
 * entries are 0), the serial-equivalent oracle calls and accepted updates
 * since the run started at t0 = 0, and the current J.  Any pointer may be NULL.
 */
qst_status qst_iterate_state(qst_plan plan, int *stopped, long long *oracle_calls,
                             int *accepted_updates, double *J);

/*
 * Batched evaluation of many independent instances of uneven shape
 * (instances with different n, M, K and shots, e.g. 64 instances with n from
 * 6 to 14).  qst_batch_create makes one plan per instance (params shared;
 * unless params fixes max_bin_settings, plans of n = 10..16 bin up to 32
 * settings, because the instances fill the GPU together: their 12-qubit
 * chunks then run the two-round kernels).  qst_batch_evaluate runs every instance's qst_evaluate
 * (forward, then the adjoint with the instance plan's transform cache where
 * it has one); arguments are HOST arrays of `count` DEVICE pointers, one per
 * instance, with the per-instance layouts of qst_forward / qst_adjoint
 * (loss[i] -> double[1], c_obs[i] -> float[nnz_i], grad_psi[i] ->
 * complex64[K_i][2^n_i], grad_w[i] -> float[K_i]).  Each phase (packing,
 * validation, forward chunk kernels, epilogue, loss, adjoint chunk kernels,
 * reduction, h) is one launch over all instances per kernel family: the
 * CTAs of every instance's grid in one grid, each CTA finding its instance
 * from a table of CTA offsets; the families of a phase run on forked
 * streams.  Batches with an instance on the wide path (n > 16) or on the
 * tensor cores run every instance's qst_evaluate on forked streams instead.
 * The first call with a given set of pointers captures the launches into
 * one CUDA graph (on a batch-owned stream in thread-local mode); later calls
 * with the same pointers replay it as a single graph launch on `stream`.
 * qst_batch_plan returns instance i's plan (for qst_plan_status etc.).
 */
typedef struct qst_batch_s *qst_batch;
qst_status qst_batch_create(qst_batch *batch, int count, const int *n, const int *M,
                            const int *K, const int64_t *nnz, const qst_params *params);
/* The same with one params record per instance (params[0..count-1], taken as
 * given: no batch-wide bin rule), e.g. the layouts an autotuner chose per
 * size class.  params == NULL: QST_ERR_INVALID_ARG. */
qst_status qst_batch_create_each(qst_batch *batch, int count, const int *n, const int *M,
                                 const int *K, const int64_t *nnz, const qst_params *params);
qst_status qst_batch_destroy(qst_batch batch);
qst_status qst_batch_plan(qst_batch batch, int i, qst_plan *plan);
qst_status qst_batch_evaluate(qst_batch batch, const float *const *psi, const float *const *w,
                              const uint8_t *const *basis, const int64_t *const *row_ptr,
                              const uint32_t *const *outcome, const uint32_t *const *count,
                              const uint32_t *const *shots, double *const *loss,
                              float *const *c_obs, float *const *grad_psi,
                              float *const *grad_w, void *stream);

/*
 * Algorithm 1 on every instance of the batch (qst_iterate per instance, in
 * place on each instance's psi and w): each instance's iteration sequence,
 * with its conditional trial nodes and its device stopping rules, is captured
 * on its own forked stream into one CUDA graph on the first call with a given
 * set of pointers, T, start (t0 == 0 or not), slots and parameters, and
 * replayed afterwards.  Arguments are HOST arrays of `count` DEVICE pointers
 * (J_hist[i] -> double[T], accepted_hist[i] -> int[T] or accepted_hist NULL);
 * params as for qst_iterate (spectral must be 0: QST_ERR_INVALID_ARG).
 * qst_iterate_state on qst_batch_plan(i) reports instance i's state.
 */
qst_status qst_batch_iterate(qst_batch batch, int T, int t0, float *const *psi, float *const *w,
                             const uint8_t *const *basis, const int64_t *const *row_ptr,
                             const uint32_t *const *outcome, const uint32_t *const *count,
                             const uint32_t *const *shots, const qst_iter_params *params,
                             double *const *J_hist, int *const *accepted_hist, void *stream);

/*
 * Adjoint without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc.  Examples are
 * code running under an allocator it does not own (a framework's caching
 * pool, a sandbox that forbids raw device allocation) and loops that must not
 * pay cudaMalloc's implicit device synchronisation.
 *
 * It computes exactly what qst_adjoint computes (same arguments and outputs;
 * psi, w, basis, CSR, c_obs, grad_psi, grad_w are caller-owned device memory).
 * The shape and params take the place of a plan, and device_status is a
 * caller-owned device int.  The call zeroes it, then device-side data checks
 * OR their QST_DEV_* bits into it.  All workspace comes from one file-scope
 * device array of QST_NOALLOC_SCRATCH_BYTES, which every GPU that loads the
 * library holds until the process exits.  The call uses the largest bins
 * (fewest z buffers) and returns QST_ERR_SCRATCH_TOO_SMALL, with a message
 * on stderr, when the problem needs more.  Roughly, the workspace is
 * (bins) x K x 2^n x 8 bytes plus a few bytes per setting.  For example,
 * n = 12, M = 2000, K = 8 fits, while n = 16, K = 16 does not.
 *
 * Limits beyond the scratch size: n <= 16 with at most 4 qubits above the
 * chunk (n = 17..20, or a chunk_qubits that leaves more, returns
 * QST_ERR_UNSUPPORTED), and the call always runs the per-setting-round chunk
 * kernels that a plan with fixed_rounds = 0 runs, never the two-round or
 * fixed-round kernels a plan may choose.  So params->fixed_rounds must be -1
 * or 0 (anything else returns QST_ERR_INVALID_ARG), and results agree with a
 * plan's within rounding, not bit for bit.
 *
 * The first call on each device looks up the array's device address and sets
 * kernel attributes, so make that first call before any stream capture.
 * Every call shares the one array, and it keeps the last call's contents.
 * Calls that overlap on the GPU (other streams, other host threads) race on
 * it, so serialise them.
 */
#define QST_NOALLOC_SCRATCH_BYTES (32u << 20)
qst_status qst_adjoint_noalloc(int n, int M, int K, int64_t nnz,
                               const qst_params *params, const float *psi,
                               const float *w, const uint8_t *basis,
                               const int64_t *row_ptr, const uint32_t *outcome,
                               const float *c_obs, float *grad_psi,
                               float *grad_w, int *device_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QST_H */
