// Device-side iterations of Algorithm 1 (included inside qst.cu's anonymous
// namespace).  Every decision of an iteration -- the atom of a T_psi slot,
// which trial of the step grid is accepted, whether the state changes -- is
// taken by these single-thread kernels from device data, so a whole run of
// iterations is one fixed launch sequence that a CUDA graph can hold.

constexpr int kIterRing = 64;  // accepted-update window of the delta stopping rule (<= kIterRing - 1)

struct IterState {
    double J;       // J = L_eps + mu R of the current state
    double eta;     // step of the trial accepted in the current iteration (0: none)
    int done;       // a trial of the current iteration was accepted: later trials skip
    int acc;        // index of that trial, -1 if none
    int r;          // atom of the current T_psi slot
    int psi_slots;  // T_psi slots so far: r cycles over the atoms with w > 0
    // stopping rules of Table I, evaluated after every iteration
    int stopped;            // a rule fired: every later iteration does nothing
    int live;               // the current iteration was not skipped by a stop
    int n_acc;              // accepted updates since the start
    int pad;
    long long oracle_calls; // serial-equivalent oracle calls since the start
    double J_ring[kIterRing];  // J after accepted update i at index i mod kIterRing (i = 0: the start)
};

__device__ __forceinline__ int iter_active(const float *w, int K) {
    int R = 0;
    for (int k = 0; k < K; ++k) R += w[k] > 0.f;
    return R;
}
// J = L + mu R, rounded as the host computes it (no contraction)
__device__ __forceinline__ double iter_J(double L, double mu, int R) { return __dadd_rn(L, __dmul_rn(mu, (double)R)); }

// J of the starting state (its loss was just computed); reset = a new run:
// restart the cyclic atom choice, the stopping rules' history and the
// oracle-call count (which starts with the starting state's forward: one
// response per active atom and the loss).
__global__ void k_iter_init(IterState *s, const double *loss, const float *w, int K, double mu, int reset) {
    if (threadIdx.x | blockIdx.x) return;
    const int R = iter_active(w, K);
    s->J = iter_J(*loss, mu, R);
    if (reset) {
        s->psi_slots = 0;
        s->stopped = 0;
        s->n_acc = 0;
        s->oracle_calls = (long long)R + 1;
        s->J_ring[0] = s->J;
    }
}

// Start of an iteration: no trial accepted yet; a T_psi slot picks atom
// r = (active atoms)[psi_slots mod R] (or skips every trial when R = 0).
__global__ void k_iter_begin(IterState *s, const float *w, int K, int slot) {
    if (threadIdx.x | blockIdx.x) return;
    s->done = 0;
    s->acc = -1;
    s->eta = 0.0;
    s->live = !s->stopped;
    if (s->stopped) {  // a stopping rule fired earlier: nothing runs
        s->done = 1;
        return;
    }
    if (slot != 0) return;
    const int R = iter_active(w, K);
    if (R == 0) {  // no atom to move: the slot does nothing
        s->done = 1;
        s->live = 0;
        return;
    }
    int want = s->psi_slots % R, r = 0;
    for (int k = 0; k < K; ++k)
        if (w[k] > 0.f && want-- == 0) {
            r = k;
            break;
        }
    s->r = r;
    s->psi_slots += 1;
}

// Acceptance of trial j (Sec. III-D): J~ = L~ + mu R~ <= J - tau_acc, where
// R~ counts the trial's atoms with w > 0.  The first accepted trial wins.
// Trial j + 1 sits in a conditional graph node whose condition defaults to 0
// at every graph launch; only a rejected trial j opens it (has_next = 0 for
// the last trial of a grid).  A trial that did not run opens nothing, so once
// a trial is accepted, or the slot has nothing to do, no later trial launches.
__global__ void k_iter_accept(IterState *s, const double *loss, const float *w_trial, int K, double mu,
                              double tau_acc, int j, double eta, int has_next, cudaGraphConditionalHandle next) {
    if (threadIdx.x | blockIdx.x) return;
    if (s->done) return;
    const double Jt = iter_J(*loss, mu, iter_active(w_trial, K));
    if (Jt <= __dsub_rn(s->J, tau_acc)) {
        s->done = 1;
        s->acc = j;
        s->J = Jt;
        s->eta = eta;
    } else if (has_next) {
        cudaGraphSetConditional(next, 1u);
    }
}

// The accepted trial becomes the state: atom r (slot 0), the weights (slot 1)
// or every atom and weight (slot 2), and its likelihood ratio becomes c.
__global__ void k_iter_commit(const IterState *s, int slot, const float2 *trial, const float *tw, float2 *psi,
                              float *w, int K, int64_t D, const float *trial_c, float *c, int64_t nnz) {
    if (s->acc < 0) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot == 0) {
        const int64_t base = (int64_t)s->r * D;
        for (int64_t x = t0; x < D; x += stride) psi[base + x] = trial[base + x];
    } else if (slot == 2) {
        for (int64_t x = t0; x < (int64_t)K * D; x += stride) psi[x] = trial[x];
    }
    if (slot != 0)
        for (int64_t k = t0; k < K; k += stride) w[k] = tw[k];
    for (int64_t i = t0; i < nnz; i += stride) c[i] = trial_c[i];
}

// End of an iteration: the history, then the stopping rules of Table I.
// Serial-equivalent oracle calls (one primitive of Sec. III-B over all
// outcomes for one atom, or one loss evaluation), as Algorithm 1 issues them:
//   atom slot:        G psi_r, then per trial the response of the trial atom and the loss;
//   coefficient slot: A^T c, then per trial the loss (the responses are kept);
//   refactor slot:    the responses of the new atoms and the loss.
// A trial count is the accepted trial's index + 1, or the whole grid.  After
// accepted update i the relative decrease over the last `window` accepted
// updates, (J_{i-window} - J_i) / |J_{i-window}|, below `tol` stops the run,
// and so does reaching max_calls oracle calls (0 disables either rule).
__global__ void k_iter_end(IterState *s, double *J_hist, int *acc_hist, int i, int slot, int n_eta,
                           const float *w_trial, int K, int window, double tol, long long max_calls) {
    if (threadIdx.x | blockIdx.x) return;
    J_hist[i] = s->J;
    if (acc_hist) acc_hist[i] = s->acc >= 0;
    if (!s->live) return;
    const int trials = s->acc >= 0 ? s->acc + 1 : n_eta;
    if (slot == 0) s->oracle_calls += 1 + 2LL * trials;
    else if (slot == 1) s->oracle_calls += 1 + (long long)trials;
    else s->oracle_calls += (long long)iter_active(w_trial, K) + 1;
    if (s->acc >= 0) {
        s->n_acc += 1;
        s->J_ring[s->n_acc % kIterRing] = s->J;
        if (window > 0 && s->n_acc >= window) {
            const double J0 = s->J_ring[(s->n_acc - window) % kIterRing];
            if ((J0 - s->J) / fabs(J0) < tol) s->stopped = 1;
        }
    }
    if (max_calls > 0 && s->oracle_calls >= max_calls) s->stopped = 1;
}

// An iteration run outside the graph (the spectral slot through qst_step,
// between graph segments): its J, acceptance and serial-equivalent oracle
// calls enter the same history and stopping rules as k_iter_end.  A run that
// a rule has stopped records the unchanged J and no acceptance.
__global__ void k_iter_external(IterState *s, double *J_hist, int *acc_hist, int i, double J, int accepted,
                                long long calls, int window, double tol, long long max_calls) {
    if (threadIdx.x | blockIdx.x) return;
    const bool live = !s->stopped;
    if (live && accepted) s->J = J;
    J_hist[i] = s->J;
    if (acc_hist) acc_hist[i] = live && accepted;
    if (!live) return;
    s->oracle_calls += calls;
    if (accepted) {
        s->n_acc += 1;
        s->J_ring[s->n_acc % kIterRing] = s->J;
        if (window > 0 && s->n_acc >= window) {
            const double J0 = s->J_ring[(s->n_acc - window) % kIterRing];
            if ((J0 - s->J) / fabs(J0) < tol) s->stopped = 1;
        }
    }
    if (max_calls > 0 && s->oracle_calls >= max_calls) s->stopped = 1;
}
