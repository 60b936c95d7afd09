// Device-side iterations of Algorithm 1 (included inside qst.cu's anonymous
// namespace).  Every decision of an iteration -- the atom of a T_psi slot,
// which trial of the step grid is accepted, whether the state changes -- is
// taken by these single-thread kernels from device data, so a whole run of
// iterations is one fixed launch sequence that a CUDA graph can hold.

struct IterState {
    double J;       // J = L_eps + mu R of the current state
    double eta;     // step of the trial accepted in the current iteration (0: none)
    int done;       // a trial of the current iteration was accepted: later trials skip
    int acc;        // index of that trial, -1 if none
    int r;          // atom of the current T_psi slot
    int psi_slots;  // T_psi slots so far: r cycles over the atoms with w > 0
};

__device__ __forceinline__ int iter_active(const float *w, int K) {
    int R = 0;
    for (int k = 0; k < K; ++k) R += w[k] > 0.f;
    return R;
}
// J = L + mu R, rounded as the host computes it (no contraction)
__device__ __forceinline__ double iter_J(double L, double mu, int R) { return __dadd_rn(L, __dmul_rn(mu, (double)R)); }

// J of the starting state (its loss was just computed); reset = restart the
// cyclic atom choice
__global__ void k_iter_init(IterState *s, const double *loss, const float *w, int K, double mu, int reset) {
    if (threadIdx.x | blockIdx.x) return;
    s->J = iter_J(*loss, mu, iter_active(w, K));
    if (reset) s->psi_slots = 0;
}

// Start of an iteration: no trial accepted yet; a T_psi slot picks atom
// r = (active atoms)[psi_slots mod R] (or skips every trial when R = 0).
__global__ void k_iter_begin(IterState *s, const float *w, int K, int slot) {
    if (threadIdx.x | blockIdx.x) return;
    s->done = 0;
    s->acc = -1;
    s->eta = 0.0;
    if (slot != 0) return;
    const int R = iter_active(w, K);
    if (R == 0) {
        s->done = 1;
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

__global__ void k_iter_end(const IterState *s, double *J_hist, int *acc_hist, int i) {
    if (threadIdx.x | blockIdx.x) return;
    J_hist[i] = s->J;
    if (acc_hist) acc_hist[i] = s->acc >= 0;
}
