// qst_update.cuh — device kernels of the update rules that ride on top of the
// forward/adjoint (paper Sec. III-C): simplex projection with the truncation
// map P_tau, and the exact spectral refactorisation of rho = Psi diag(w) Psi^*.
// Included by qst.cu inside its anonymous namespace (one translation unit);
// FP64 for the K x K linear algebra.
#pragma once


constexpr int kProjMax = 1024;   // simplex projection: entries per call (one CTA)
constexpr int kRefacMax = 32;    // refactorisation: atoms per plan (K x K FP64 matrices in shared memory)
constexpr int kJacobiSweeps = 60;

// Projection onto the simplex (sort-based: Held-Wolfe-Crowder 1974 /
// Duchi et al. 2008) followed by P_tau (Eq. truncation-map): keep beta_r > tau,
// renormalise; if nothing survives keep the largest.  Runs on one CTA of
// kProjMax threads: bitonic sort in shared memory, sequential prefix sum in
// thread 0 (fixed order).  v is read from shared or global memory by the
// caller-supplied values vin[t] (t < K).  Outputs: beta [K] (0 at pruned
// entries), keep [K] (kept indices ascending, first *kout of them), *kout.
struct SimplexSmem {
    double u[kProjMax];
    double b[kProjMax];
    double theta, norm;
    int amax;
};
__device__ void simplex_prune_block(double vt, int K, double tau, double *beta, int *keep, int *kout,
                                    SimplexSmem &sm) {
    const int t = threadIdx.x;
    int P = 1;
    while (P < K) P <<= 1;
    sm.u[t] = (t < K) ? vt : -INFINITY;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {  // bitonic sort, descending
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (t < P) {
                const int partner = t ^ stride;
                if (partner > t) {
                    const bool desc = ((t & size) == 0);
                    const double x = sm.u[t], y = sm.u[partner];
                    if (desc ? (x < y) : (x > y)) {
                        sm.u[t] = y;
                        sm.u[partner] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        double css = 0.0, th = 0.0;
        for (int j = 0; j < K; ++j) {
            css += sm.u[j];
            const double cand = (css - 1.0) / (double)(j + 1);
            if (sm.u[j] - cand > 0.0) th = cand;
        }
        sm.theta = th;
    }
    __syncthreads();
    if (t < K) sm.b[t] = fmax(vt - sm.theta, 0.0);
    __syncthreads();
    if (t == 0) {
        double s = 0.0, best = -1.0;
        int nk = 0, am = 0;
        for (int j = 0; j < K; ++j) {
            if (sm.b[j] > best) { best = sm.b[j]; am = j; }
            if (sm.b[j] > tau) { s += sm.b[j]; keep[nk++] = j; }
        }
        if (nk == 0) { keep[0] = am; nk = 1; s = sm.b[am]; }
        *kout = nk;
        sm.norm = s;
        sm.amax = (nk == 1 && !(sm.b[am] > tau)) ? am : -1;
    }
    __syncthreads();
    if (t < K) {
        const bool kept = (sm.b[t] > tau) || (t == sm.amax);
        beta[t] = kept ? sm.b[t] / sm.norm : 0.0;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kProjMax) k_simplex(const double *__restrict__ v, int K, double tau,
                                                      double *__restrict__ beta, int *__restrict__ keep,
                                                      int *__restrict__ kout) {
    __shared__ SimplexSmem sm;
    const int t = threadIdx.x;
    simplex_prune_block(t < K ? v[t] : 0.0, K, tau, beta, keep, kout, sm);
}

// Coefficient trial of a T_alpha slot (Eq. coefficient-update, then P_tau):
// over the active atoms (w_r > 0, in index order) beta = proj(w + eta h),
// h = -grad_w; inactive and pruned atoms get weight 0.  One CTA, K <= kProjMax.
__global__ void __launch_bounds__(kProjMax) k_coeff_trial(const float *__restrict__ w,
                                                          const float *__restrict__ grad_w, double eta,
                                                          double tau, int K, float *__restrict__ w_out,
                                                          const int *skip) {
    if (skip && *skip) return;  // a trial of this slot was already accepted
    __shared__ SimplexSmem sm;
    __shared__ int idx[kProjMax];
    __shared__ double beta[kProjMax];
    __shared__ int keep[kProjMax];
    __shared__ int na_sm, kout_sm;
    const int t = threadIdx.x;
    if (t == 0) {
        int na = 0;
        for (int k = 0; k < K; ++k)
            if (w[k] > 0.f) idx[na++] = k;
        na_sm = na;
    }
    __syncthreads();
    const int na = na_sm;
    const double vt = (t < na) ? (double)w[idx[t]] - eta * (double)grad_w[idx[t]] : 0.0;
    if (na > 0) simplex_prune_block(vt, na, tau, beta, keep, &kout_sm, sm);
    if (t < K) w_out[t] = 0.f;
    __syncthreads();
    if (t < na) w_out[idx[t]] = (float)beta[t];
}

// Atom trial of a T_psi slot (Eqs. atom-direction, atom-trial): with
// G psi_r given, g = w_r (G psi_r - psi_r <psi_r, G psi_r>) and
// out = (psi_r + eta g) / ||psi_r + eta g||.  One CTA; FP64 reductions in a
// fixed order.  The atom is r_dev[0] when r_dev is given (chosen on the
// device), else r_host; skip as in k_coeff_trial.
__global__ void __launch_bounds__(1024) k_atom_trial(const float2 *__restrict__ psi, const float2 *__restrict__ gpsi,
                                                     const float *__restrict__ w, const int *r_dev, int r_host,
                                                     double eta, int64_t D, float2 *__restrict__ out_all,
                                                     const int *skip) {
    if (skip && *skip) return;
    const int r = r_dev ? *r_dev : r_host;
    const float2 *__restrict__ psi_r = psi + (size_t)r * D;
    const float2 *__restrict__ gpsi_r = gpsi + (size_t)r * D;
    float2 *__restrict__ out = out_all + (size_t)r * D;
    const float wr = w[r];
    __shared__ double red[1024];
    __shared__ double inr_sm, ini_sm, nrm_sm;
    const int t = threadIdx.x;
    double ir = 0.0, ii = 0.0;
    for (int64_t x = t; x < D; x += blockDim.x) {
        const float2 a = psi_r[x], g = gpsi_r[x];
        ir += (double)a.x * g.x + (double)a.y * g.y;   // conj(a) g
        ii += (double)a.x * g.y - (double)a.y * g.x;
    }
    red[t] = ir;
    __syncthreads();
    if (t == 0) { double s = 0.0; for (int q = 0; q < (int)blockDim.x; ++q) s += red[q]; inr_sm = s; }
    __syncthreads();
    red[t] = ii;
    __syncthreads();
    if (t == 0) { double s = 0.0; for (int q = 0; q < (int)blockDim.x; ++q) s += red[q]; ini_sm = s; }
    __syncthreads();
    const double inr = inr_sm, ini = ini_sm;
    auto trial = [&](int64_t x) {
        const float2 a = psi_r[x], g = gpsi_r[x];
        const double dr = (double)g.x - ((double)a.x * inr - (double)a.y * ini);
        const double di = (double)g.y - ((double)a.x * ini + (double)a.y * inr);
        return make_double2((double)a.x + eta * wr * dr, (double)a.y + eta * wr * di);
    };
    double nn = 0.0;
    for (int64_t x = t; x < D; x += blockDim.x) {
        const double2 v = trial(x);
        nn += v.x * v.x + v.y * v.y;
    }
    red[t] = nn;
    __syncthreads();
    if (t == 0) { double s = 0.0; for (int q = 0; q < (int)blockDim.x; ++q) s += red[q]; nrm_sm = s; }
    __syncthreads();
    const double inv = nrm_sm > 0.0 ? 1.0 / sqrt(nrm_sm) : 0.0;
    for (int64_t x = t; x < D; x += blockDim.x) {
        const double2 v = trial(x);
        out[x] = make_float2((float)(v.x * inv), (float)(v.y * inv));
    }
}

// C_ij = sum_x conj(psi_i[x]) psi_j[x] (FP64, fixed order), one block per
// pair i <= j; the lower triangle is filled by conjugation in k_eig.
__global__ void __launch_bounds__(256) k_gram(const float2 *__restrict__ psi, int K, int64_t D,
                                              double2 *__restrict__ C) {
    __shared__ double2 red[256];
    int p = blockIdx.x, i = 0;
    while (p >= K - i) { p -= K - i; ++i; }
    const int j = i + p;
    const float2 *a = psi + (size_t)i * D, *b = psi + (size_t)j * D;
    double re = 0.0, im = 0.0;
    for (int64_t x = threadIdx.x; x < D; x += blockDim.x) {
        const float2 u = a[x], w = b[x];
        re += (double)u.x * w.x + (double)u.y * w.y;   // conj(u) * w
        im += (double)u.x * w.y - (double)u.y * w.x;
    }
    red[threadIdx.x] = make_double2(re, im);
    __syncthreads();
    if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) { sr += red[q].x; si += red[q].y; }
        C[(size_t)i * K + j] = make_double2(sr, si);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Cyclic Jacobi on the Hermitian K x K matrix H (shared, row stride kRefacMax + 1),
// accumulating the rotations into V (Golub & Van Loan, Sec. 8.5): each rotation
// first removes the phase of H_pq, then applies the real symmetric Jacobi
// rotation.  Bounded sweep count; called by all threads of one CTA (>= K).
__device__ void jacobi_hermitian(double2 (*H)[kRefacMax + 1], double2 (*V)[kRefacMax + 1], int K) {
    __shared__ double2 rot[4];  // (c, s e^{i phi}) pieces of the current rotation
    __shared__ int skip;
    const int t = threadIdx.x;
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        // off-diagonal norm vs diagonal: stop when negligible
        if (t == 0) {
            double off = 0.0, dia = 0.0;
            for (int p = 0; p < K; ++p)
                for (int q = 0; q < K; ++q) {
                    const double a2 = H[p][q].x * H[p][q].x + H[p][q].y * H[p][q].y;
                    if (p == q) dia += a2; else off += a2;
                }
            skip = (off <= 1e-30 * (dia > 0.0 ? dia : 1.0)) ? 1 : 0;
        }
        __syncthreads();
        if (skip) break;
        for (int p = 0; p < K - 1; ++p) {
            for (int q = p + 1; q < K; ++q) {
                if (t == 0) {
                    const double2 hpq = H[p][q];
                    const double mag = sqrt(hpq.x * hpq.x + hpq.y * hpq.y);
                    if (mag < 1e-300) {
                        rot[0] = make_double2(1.0, 0.0);
                        rot[1] = make_double2(0.0, 0.0);
                        rot[2] = make_double2(0.0, 0.0);
                        rot[3] = make_double2(1.0, 0.0);
                    } else {
                        const double2 ph = make_double2(hpq.x / mag, hpq.y / mag);  // e^{i phi}
                        const double tau_r = (H[q][q].x - H[p][p].x) / (2.0 * mag);
                        const double tt = (tau_r >= 0.0 ? 1.0 : -1.0) / (fabs(tau_r) + sqrt(1.0 + tau_r * tau_r));
                        const double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
                        // unitary J acting on columns p, q:  col_p' = c col_p - s conj(ph) col_q ... written as
                        // [J_pp J_pq; J_qp J_qq] = [c, s ph; -s conj(ph), c]
                        rot[0] = make_double2(c, 0.0);
                        rot[1] = make_double2(s * ph.x, s * ph.y);
                        rot[2] = make_double2(-s * ph.x, s * ph.y);
                        rot[3] = make_double2(c, 0.0);
                    }
                }
                __syncthreads();
                const double2 Jpp = rot[0], Jpq = rot[1], Jqp = rot[2], Jqq = rot[3];
                // H <- J^* H J : first columns (H J), then rows (J^* H)
                if (t < K) {
                    const double2 hp = H[t][p], hq = H[t][q];
                    H[t][p] = make_double2(cmul(hp, Jpp).x + cmul(hq, Jqp).x, cmul(hp, Jpp).y + cmul(hq, Jqp).y);
                    H[t][q] = make_double2(cmul(hp, Jpq).x + cmul(hq, Jqq).x, cmul(hp, Jpq).y + cmul(hq, Jqq).y);
                    const double2 vp = V[t][p], vq = V[t][q];
                    V[t][p] = make_double2(cmul(vp, Jpp).x + cmul(vq, Jqp).x, cmul(vp, Jpp).y + cmul(vq, Jqp).y);
                    V[t][q] = make_double2(cmul(vp, Jpq).x + cmul(vq, Jqq).x, cmul(vp, Jpq).y + cmul(vq, Jqq).y);
                }
                __syncthreads();
                if (t < K) {
                    const double2 hp = H[p][t], hq = H[q][t];
                    const double2 a = cconj(Jpp), b = cconj(Jqp), c2 = cconj(Jpq), d = cconj(Jqq);
                    H[p][t] = make_double2(cmul(a, hp).x + cmul(b, hq).x, cmul(a, hp).y + cmul(b, hq).y);
                    H[q][t] = make_double2(cmul(c2, hp).x + cmul(d, hq).x, cmul(c2, hp).y + cmul(d, hq).y);
                }
                __syncthreads();
            }
        }
    }
}

// Eigen-decomposition of H = diag(sqrt w) C diag(sqrt w) (complex Hermitian,
// FP64) by cyclic Jacobi (Golub & Van Loan, Sec. 8.5), one CTA, K <= kRefacMax.
// Each rotation first removes the phase of H_pq, then applies the real
// symmetric Jacobi rotation; bounded sweep count.  Then: eigenpairs sorted
// descending, weights lambda / sum(lambda), P_tau, and the combination matrix
// T = diag(sqrt w) V_kept diag(1/sqrt lambda) (K x K, zero columns beyond K').
__global__ void __launch_bounds__(kRefacMax) k_eig(const double2 *__restrict__ Cin, const float *__restrict__ w,
                                                   int K, double tau, double2 *__restrict__ T,
                                                   float *__restrict__ w_out, int *__restrict__ kout) {
    __shared__ double2 H[kRefacMax][kRefacMax + 1];
    __shared__ double2 V[kRefacMax][kRefacMax + 1];
    __shared__ double lam[kRefacMax], sw[kRefacMax], wt[kRefacMax];
    __shared__ int ord[kRefacMax], keepj[kRefacMax];
    __shared__ int nk_sm;
    const int t = threadIdx.x;
    if (t < K) sw[t] = sqrt(fmax((double)w[t], 0.0));
    __syncthreads();
    if (t < K) {
        for (int j = 0; j < K; ++j) {
            double2 c = (t <= j) ? Cin[(size_t)t * K + j] : cconj(Cin[(size_t)j * K + t]);
            H[t][j] = make_double2(c.x * sw[t] * sw[j], c.y * sw[t] * sw[j]);
            V[t][j] = make_double2(t == j ? 1.0 : 0.0, 0.0);
        }
    }
    __syncthreads();
    jacobi_hermitian(H, V, K);
    if (t == 0) {
        double tot = 0.0;
        for (int j = 0; j < K; ++j) {
            lam[j] = fmax(H[j][j].x, 0.0);
            ord[j] = j;
            tot += lam[j];
        }
        for (int a = 1; a < K; ++a) {  // insertion sort, descending (stable)
            const int o = ord[a];
            int b = a - 1;
            while (b >= 0 && lam[ord[b]] < lam[o]) { ord[b + 1] = ord[b]; --b; }
            ord[b + 1] = o;
        }
        int nk = 0;
        double s = 0.0;
        for (int j = 0; j < K; ++j) {
            const double wj = tot > 0.0 ? lam[ord[j]] / tot : 0.0;
            if (wj > tau) { keepj[nk++] = ord[j]; s += wj; }
        }
        if (nk == 0) { keepj[0] = ord[0]; nk = 1; s = tot > 0.0 ? lam[ord[0]] / tot : 1.0; }
        for (int j = 0; j < K; ++j) wt[j] = (j < nk && tot > 0.0) ? (lam[keepj[j]] / tot) / s : 0.0;
        nk_sm = nk;
        *kout = nk;
    }
    __syncthreads();
    const int nk = nk_sm;
    if (t < K) {
        w_out[t] = (float)wt[t];
        for (int j = 0; j < K; ++j) {
            double2 val = make_double2(0.0, 0.0);
            if (j < nk) {
                const int e = keepj[j];
                const double inv = lam[e] > 0.0 ? 1.0 / sqrt(lam[e]) : 0.0;
                val = make_double2(sw[t] * V[t][e].x * inv, sw[t] * V[t][e].y * inv);
            }
            T[(size_t)t * K + j] = val;  // psi'_j = sum_t psi_t T_tj
        }
    }
}

// psi'_j[x] = sum_k psi_k[x] T_kj for every x, in place (each thread reads all
// K inputs of its x before writing); atoms j >= K' become zero.
__global__ void __launch_bounds__(256) k_combine(float2 *__restrict__ psi, int K, int64_t D,
                                                 const double2 *__restrict__ T) {
    __shared__ float2 Ts[kRefacMax * kRefacMax];
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) Ts[e] = make_float2((float)T[e].x, (float)T[e].y);
    __syncthreads();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (int64_t)gridDim.x * blockDim.x) {
        float2 in[kRefacMax];
#pragma unroll 4
        for (int k = 0; k < K; ++k) in[k] = psi[(size_t)k * D + x];
        for (int j = 0; j < K; ++j) {
            float re = 0.f, im = 0.f;
            for (int k = 0; k < K; ++k) {
                const float2 a = in[k], b = Ts[k * K + j];
                re += a.x * b.x - a.y * b.y;
                im += a.x * b.y + a.y * b.x;
            }
            psi[(size_t)j * D + x] = make_float2(re, im);
        }
    }
}
