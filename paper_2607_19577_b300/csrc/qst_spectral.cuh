// Spectral step of Sec. III-C on the GPU (included inside qst.cu's anonymous
// namespace, after qst_update.cuh): block Krylov products with
// S = Psi diag(w) Psi^* + eta G (Eq. density-product; G through the adjoint
// kernels), full reorthogonalisation, Rayleigh-Ritz (Eq. ritz-pairs), and the
// candidate scoring and selection of Eqs. spectral-candidates,
// proximal-surrogate and spectral-selection.  Vectors are complex64 rows of
// length D; every inner product and small matrix is FP64 in a fixed order.

constexpr int kKrylovMax = kRefacMax;  // Krylov basis vectors (Table I: at most 30)

// C[i * ldc + j] = sum_x conj(A_i[x]) B_j[x], one block per (i, j).
__global__ void __launch_bounds__(256) k_xgram(const float2 *__restrict__ A, int na, const float2 *__restrict__ B,
                                               int nb, int64_t D, double2 *__restrict__ C, int ldc) {
    __shared__ double2 red[256];
    const int i = blockIdx.x / nb, j = blockIdx.x % nb;
    if (i >= na) return;
    const float2 *a = A + (size_t)i * D, *b = B + (size_t)j * D;
    double re = 0.0, im = 0.0;
    for (int64_t x = threadIdx.x; x < D; x += blockDim.x) {
        const float2 u = a[x], v = b[x];
        re += (double)u.x * v.x + (double)u.y * v.y;
        im += (double)u.x * v.y - (double)u.y * v.x;
    }
    red[threadIdx.x] = make_double2(re, im);
    __syncthreads();
    if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) {
            sr += red[q].x;
            si += red[q].y;
        }
        C[(size_t)i * ldc + j] = make_double2(sr, si);
    }
}

// out_j = beta out_j + sum_i in_i (scale_i coef[i * ldc + j]), j < nout, i < nin
// (scale: optional per-input factor, e.g. the weights w_i; sign: +1 or -1).
// Each element accumulates in FP64.  out must not alias in.
__global__ void __launch_bounds__(256) k_lincomb(float2 *__restrict__ out, int nout, double beta,
                                                 const float2 *__restrict__ in, int nin,
                                                 const double2 *__restrict__ coef, int ldc,
                                                 const float *__restrict__ scale, double sign, int64_t D) {
    __shared__ double2 cs[kKrylovMax + kRefacMax][kRefacMax];
    for (int e = threadIdx.x; e < nin * nout; e += blockDim.x) {
        const int i = e / nout, j = e % nout;
        const double f = sign * (scale ? (double)scale[i] : 1.0);
        const double2 c = coef[(size_t)i * ldc + j];
        cs[i][j] = make_double2(f * c.x, f * c.y);
    }
    __syncthreads();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < nout; ++j) {
            const float2 o = out[(size_t)j * D + x];
            double re = beta * (double)o.x, im = beta * (double)o.y;
            for (int i = 0; i < nin; ++i) {
                const float2 v = in[(size_t)i * D + x];
                const double2 c = cs[i][j];
                re += (double)v.x * c.x - (double)v.y * c.y;
                im += (double)v.x * c.y + (double)v.y * c.x;
            }
            out[(size_t)j * D + x] = make_float2((float)re, (float)im);
        }
    }
}

// Load the Hermitian part (C + C^*) / 2 of an n x n matrix into H, V = I.
__device__ void load_hermitian(const double2 *__restrict__ C, int ldc, int n, double2 (*H)[kRefacMax + 1],
                               double2 (*V)[kRefacMax + 1]) {
    const int t = threadIdx.x;
    if (t < n)
        for (int j = 0; j < n; ++j) {
            const double2 a = C[(size_t)t * ldc + j], b = C[(size_t)j * ldc + t];
            H[t][j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
            V[t][j] = make_double2(t == j ? 1.0 : 0.0, 0.0);
        }
    __syncthreads();
}

// Eigenvalues descending (stable order), one thread.
__device__ void sort_desc(const double2 (*H)[kRefacMax + 1], int n, double *lam, int *ord) {
    for (int j = 0; j < n; ++j) {
        lam[j] = H[j][j].x;
        ord[j] = j;
    }
    for (int a = 1; a < n; ++a) {
        const int o = ord[a];
        int b = a - 1;
        while (b >= 0 && lam[ord[b]] < lam[o]) {
            ord[b + 1] = ord[b];
            --b;
        }
        ord[b + 1] = o;
    }
}

// Orthonormalisation of a block of k vectors through its Gram matrix
// C = V Lambda V^*: Tm = V_kept diag(lambda^-1/2) for lambda > drop * trace(P),
// where P is the block's Gram matrix before any projection, eigenvalues sorted
// descending; columns beyond the kept count are zero.  One CTA.
__global__ void __launch_bounds__(kRefacMax) k_orth_coef(const double2 *__restrict__ C, const double2 *__restrict__ P,
                                                         int k, double drop, double2 *__restrict__ Tm,
                                                         int *__restrict__ kout) {
    __shared__ double2 H[kRefacMax][kRefacMax + 1];
    __shared__ double2 V[kRefacMax][kRefacMax + 1];
    __shared__ double lam[kRefacMax];
    __shared__ int ord[kRefacMax];
    __shared__ int nk_sm;
    __shared__ double thr_sm;
    const int t = threadIdx.x;
    load_hermitian(C, k, k, H, V);
    jacobi_hermitian(H, V, k);
    if (t == 0) {
        double tr = 0.0;
        for (int j = 0; j < k; ++j) tr += P[(size_t)j * k + j].x;
        thr_sm = drop * tr;
        sort_desc(H, k, lam, ord);
        int nk = 0;
        while (nk < k && lam[ord[nk]] > thr_sm) ++nk;
        nk_sm = nk;
        *kout = nk;
    }
    __syncthreads();
    if (t < k)
        for (int j = 0; j < k; ++j) {
            double2 v = make_double2(0.0, 0.0);
            if (j < nk_sm) {
                const int e = ord[j];
                const double inv = 1.0 / sqrt(lam[e]);
                v = make_double2(V[t][e].x * inv, V[t][e].y * inv);
            }
            Tm[(size_t)t * k + j] = v;  // new_j = sum_t old_t Tm_tj
        }
}

// Rayleigh-Ritz: eigenpairs of the Hermitian part of T (m x m), eigenvalues
// descending in lam, eigenvectors as the columns of Y (m x m).  One CTA.
__global__ void __launch_bounds__(kRefacMax) k_heig(const double2 *__restrict__ T, int m, double *__restrict__ lam_out,
                                                    double2 *__restrict__ Y) {
    __shared__ double2 H[kRefacMax][kRefacMax + 1];
    __shared__ double2 V[kRefacMax][kRefacMax + 1];
    __shared__ double lam[kRefacMax];
    __shared__ int ord[kRefacMax];
    const int t = threadIdx.x;
    load_hermitian(T, m, m, H, V);
    jacobi_hermitian(H, V, m);
    if (t == 0) sort_desc(H, m, lam, ord);
    __syncthreads();
    if (t < m) {
        lam_out[t] = lam[ord[t]];
        for (int j = 0; j < m; ++j) Y[(size_t)t * m + j] = V[t][ord[j]];
    }
}

// Candidates and selection (Eqs. spectral-candidates, proximal-surrogate,
// spectral-selection): for s = 1..L, beta = proj_Delta(lam_1..s) (sort-based;
// lam is already descending), P_tau (strict >, the largest kept if none), and
// Q_s = (||beta||^2 - 2 beta^T lam_I) / (2 eta) + mu |I| (the constant ||S||^2
// dropped).  The first minimum wins.  Writes the kept Ritz coefficients
// Tc (m x K: column j = Y column of the j-th kept pair), the weights w_out
// (K, zero beyond the kept count) and kout.  One thread.
// rank_fix > 0 considers only the candidate with min(rank_fix, L) Ritz pairs
// (the known-rank variant of the ablation of Sec. IV).
__global__ void k_spectral_select(const double *__restrict__ lam, const double2 *__restrict__ Y, int m, int L,
                                  double eta, double mu, double tau, int K, double2 *__restrict__ Tc,
                                  float *__restrict__ w_out, int *__restrict__ kout, int *__restrict__ s_out,
                                  int rank_fix) {
    if (threadIdx.x | blockIdx.x) return;
    double best = 0.0;
    int best_s = 1;
    int keep[kRefacMax], bkeep[kRefacMax];
    double b[kRefacMax], bb[kRefacMax];
    int nbest = 0;
    const int s_lo = rank_fix > 0 ? (rank_fix < L ? rank_fix : L) : 1;
    for (int s = s_lo; s <= L && (rank_fix <= 0 || s == s_lo); ++s) {
        // projection of lam_1..s onto the simplex
        double css = 0.0, theta = 0.0;
        for (int j = 0; j < s; ++j) {
            css += lam[j];
            const double th = (css - 1.0) / (double)(j + 1);
            if (lam[j] - th > 0.0) theta = th;
        }
        int nk = 0;
        double tot = 0.0;
        for (int j = 0; j < s; ++j) {
            const double beta = fmax(lam[j] - theta, 0.0);
            if (beta > tau) {
                keep[nk] = j;
                b[nk++] = beta;
                tot += beta;
            }
        }
        if (nk == 0) {  // keep the largest (lowest index on ties)
            int a = 0;
            double ba = -1.0;
            for (int j = 0; j < s; ++j) {
                const double beta = fmax(lam[j] - theta, 0.0);
                if (beta > ba) {
                    ba = beta;
                    a = j;
                }
            }
            keep[0] = a;
            b[0] = ba;
            tot = ba;
            nk = 1;
        }
        double q2 = 0.0, ql = 0.0;
        for (int j = 0; j < nk; ++j) {
            b[j] /= tot;
            q2 += b[j] * b[j];
            ql += b[j] * lam[keep[j]];
        }
        const double q = (q2 - 2.0 * ql) / (2.0 * eta) + mu * (double)nk;
        if (s == s_lo || q < best) {
            best = q;
            best_s = s;
            nbest = nk;
            for (int j = 0; j < nk; ++j) {
                bkeep[j] = keep[j];
                bb[j] = b[j];
            }
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < K; ++j)
            Tc[(size_t)i * K + j] = (j < nbest) ? Y[(size_t)i * m + bkeep[j]] : make_double2(0.0, 0.0);
    for (int j = 0; j < K; ++j) w_out[j] = (j < nbest) ? (float)bb[j] : 0.f;
    *kout = nbest;
    if (s_out) *s_out = best_s;
}
