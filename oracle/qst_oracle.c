/*
 * qst_oracle.c — plain, slow, FP64 CPU oracle for the Pauli-measurement forward
 * and adjoint of rank-adaptive matrix-free atomic quantum state tomography.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * shares no code, header, table or helper with this file.
 *
 * Every routine follows the paper's definitions literally, one qubit and one
 * outcome at a time, with no blocking, fusion or reordering:
 *
 *   Pauli POVM (Sec. IV, "Numerical tests"): a setting s is a Pauli string
 *     b_s in {X,Y,Z}^n; V_b = V_{b_1} (x) ... (x) V_{b_n}, where V_X, V_Y, V_Z
 *     rotate the eigenbasis of the corresponding Pauli to the computational
 *     basis; E_{s,u} = (1/B) V_s^* |u><u| V_s with B the number of settings.
 *   Born probabilities per setting: P(u|s) = <u| V_s rho V_s^* |u>, and for the
 *     atomic model rho = Psi diag(w) Psi^* (Eq. atomic-density) this is
 *     p_{s,u} = sum_k w_k |(V_s psi_k)_u|^2, with pi = p / B (Eq. atomic-born-map).
 *   Empirical pmf: pihat_{s,u} = N_{s,u} / (B N_s).
 *   Loss (Eq. qst-loss): L = - sum_m pihat_m log(pi_m + eps).
 *   Likelihood ratio (Eq. likelihood-ratio-vector): c = pihat / (pi + eps).
 *   Weight gradient (Eq. weight-gradient): dJ/dw = -A^T c = -h,
 *     h_k = sum_m c_m a_m(psi_k),  a_m(psi) = <psi|E_m|psi>  (Eq. atom-response).
 *   G v (Eq. negative-gradient-product): G v = sum_m c_m E_m v
 *     = (1/B) sum_s V_s^* (c_s .* (V_s v)).
 *   Atom gradient (Eq. atom-wirtinger-gradient): d J / d psi_k^* = -w_k G psi_k.
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - V_X = (1/sqrt2)[[1,1],[1,-1]] and V_Y = (1/sqrt2)[[1,-i],[1,i]]: row u_j = 0
 *     is the +1 eigenvector (conjugated), so outcome bit 0 <-> eigenvalue +1.
 *   - Qubit 1 is the leftmost Kronecker factor, i.e. the most significant bit
 *     of the outcome index u (u = sum_j u_j 2^(n-j)).
 *   - Basis codes: 0 = Z, 1 = X, 2 = Y.
 *   - c is zero at outcomes never observed (pihat = 0 there).
 *   - N_s is given per setting (shots[s]); B is the normalising setting count,
 *     passed separately so a subset of settings (a shard) can be evaluated with
 *     the global normalisation of the full experiment.
 *
 * Complex vectors cross the ABI as interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* The single-qubit rotation V_b for basis code b (0 = Z, 1 = X, 2 = Y). */
static void rotation(int b, cplx V[2][2])
{
    const double h = 1.0 / sqrt(2.0);
    if (b == 0) {        /* V_Z = I */
        V[0][0] = 1.0; V[0][1] = 0.0;
        V[1][0] = 0.0; V[1][1] = 1.0;
    } else if (b == 1) { /* V_X: rows <+| and <-| */
        V[0][0] = h;   V[0][1] = h;
        V[1][0] = h;   V[1][1] = -h;
    } else {             /* V_Y: rows <+i| and <-i| */
        V[0][0] = h;   V[0][1] = -I * h;
        V[1][0] = h;   V[1][1] = I * h;
    }
}

static void dagger(cplx A[2][2], cplx Ad[2][2])
{
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            Ad[i][j] = conj(A[j][i]);
}

/* Apply the 2x2 matrix A on the tensor axis of qubit q (1-based; qubit 1 is
 * the most significant bit of the index). */
static void apply_one_qubit(cplx *v, int n, int q, cplx A[2][2])
{
    const int64_t D = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << (n - q);
    for (int64_t u = 0; u < D; ++u) {
        if (u & bit) continue;
        cplx a = v[u], b = v[u | bit];
        v[u] = A[0][0] * a + A[0][1] * b;
        v[u | bit] = A[1][0] * a + A[1][1] * b;
    }
}

/* v <- V_s v, V_s = V_{b_1} (x) ... (x) V_{b_n}: each factor acts on its own axis. */
static void apply_setting(cplx *v, int n, const uint8_t *b)
{
    for (int q = 1; q <= n; ++q) {
        cplx V[2][2];
        rotation(b[q - 1], V);
        apply_one_qubit(v, n, q, V);
    }
}

/* v <- V_s^* v (conjugate transpose of every factor). */
static void apply_setting_dagger(cplx *v, int n, const uint8_t *b)
{
    for (int q = 1; q <= n; ++q) {
        cplx V[2][2], Vd[2][2];
        rotation(b[q - 1], V);
        dagger(V, Vd);
        apply_one_qubit(v, n, q, Vd);
    }
}

static int check_basis(int n, int M, const uint8_t *basis)
{
    for (int64_t i = 0; i < (int64_t)M * n; ++i)
        if (basis[i] > 2) return -1;
    return 0;
}

static void load_vec(cplx *dst, const double *src_ri, int64_t D)
{
    for (int64_t u = 0; u < D; ++u) dst[u] = src_ri[2 * u] + I * src_ri[2 * u + 1];
}

/*
 * Forward pass: per-setting Born probabilities, the loss and the likelihood ratio.
 *
 *   n, M        qubits and number of settings passed in
 *   B           normalising setting count (B >= 1; the experiment's B)
 *   K           atoms
 *   basis       [M][n] basis codes
 *   psi         [K][2^n] complex atoms, interleaved (re, im)
 *   w           [K] mixture weights
 *   row_ptr     [M+1] CSR offsets into outcome/count
 *   outcome     [nnz] observed outcome indices u
 *   count       [nnz] counts N_{s,u}
 *   shots       [M] N_s
 *   eps         epsilon of Eq. qst-loss
 * outputs (any may be NULL):
 *   p_dense     [M][2^n] p_{s,u}
 *   p_obs       [nnz]    p_{s,u} at observed outcomes
 *   c_obs       [nnz]    c_{s,u} = pihat / (pi + eps) at observed outcomes
 *   loss        [1]      L_eps summed over the passed settings
 * Returns 0, or -1 on malformed input.
 */
int qst_oracle_forward(int n, int M, int B, int K, const uint8_t *basis,
                       const double *psi, const double *w,
                       const int64_t *row_ptr, const uint32_t *outcome,
                       const uint32_t *count, const uint32_t *shots, double eps,
                       double *p_dense, double *p_obs, double *c_obs, double *loss)
{
    if (n < 1 || n > 30 || M < 0 || B < 1 || K < 0) return -1;
    if (check_basis(n, M, basis)) return -1;
    const int64_t D = (int64_t)1 << n;
    cplx *phi = malloc(sizeof(cplx) * D);
    double *p = malloc(sizeof(double) * D);
    if (!phi || !p) { free(phi); free(p); return -1; }
    double L = 0.0;
    for (int s = 0; s < M; ++s) {
        const uint8_t *b = basis + (int64_t)s * n;
        for (int64_t u = 0; u < D; ++u) p[u] = 0.0;
        for (int k = 0; k < K; ++k) {
            load_vec(phi, psi + 2 * (int64_t)k * D, D);
            apply_setting(phi, n, b);
            for (int64_t u = 0; u < D; ++u) {
                double a = creal(phi[u]) * creal(phi[u]) + cimag(phi[u]) * cimag(phi[u]);
                p[u] += w[k] * a;
            }
        }
        if (p_dense) memcpy(p_dense + (int64_t)s * D, p, sizeof(double) * D);
        for (int64_t i = row_ptr[s]; i < row_ptr[s + 1]; ++i) {
            const uint32_t u = outcome[i];
            if ((int64_t)u >= D || shots[s] == 0) { free(phi); free(p); return -1; }
            const double pi = p[u] / B;
            const double pihat = (double)count[i] / ((double)B * shots[s]);
            if (p_obs) p_obs[i] = p[u];
            if (c_obs) c_obs[i] = pihat / (pi + eps);
            L -= pihat * log(pi + eps);
        }
    }
    if (loss) *loss = L;
    free(phi);
    free(p);
    return 0;
}

/*
 * Adjoint pass: atom gradients and the coefficient gradient.
 *
 *   c_obs       [nnz] likelihood ratio at observed outcomes (zero elsewhere)
 * outputs:
 *   G_psi       [K][2^n] complex, (G psi_k), interleaved; may be NULL
 *   grad_psi    [K][2^n] complex, dJ/dpsi_k^* = -w_k G psi_k; may be NULL
 *   h           [K] h_k = a(psi_k)^T c (so dJ/dw_k = -h_k); may be NULL
 * Returns 0, or -1 on malformed input.
 */
int qst_oracle_adjoint(int n, int M, int B, int K, const uint8_t *basis,
                       const double *psi, const double *w,
                       const int64_t *row_ptr, const uint32_t *outcome,
                       const double *c_obs, double *G_psi, double *grad_psi,
                       double *h)
{
    if (n < 1 || n > 30 || M < 0 || B < 1 || K < 0) return -1;
    if (check_basis(n, M, basis)) return -1;
    const int64_t D = (int64_t)1 << n;
    cplx *phi = malloc(sizeof(cplx) * D);
    cplx *y = malloc(sizeof(cplx) * D);
    cplx *acc = calloc((size_t)K * D, sizeof(cplx));
    double *hk = calloc((size_t)(K > 0 ? K : 1), sizeof(double));
    if (!phi || !y || !acc || !hk) { free(phi); free(y); free(acc); free(hk); return -1; }
    for (int s = 0; s < M; ++s) {
        const uint8_t *b = basis + (int64_t)s * n;
        for (int k = 0; k < K; ++k) {
            load_vec(phi, psi + 2 * (int64_t)k * D, D);
            apply_setting(phi, n, b);
            for (int64_t u = 0; u < D; ++u) y[u] = 0.0;
            for (int64_t i = row_ptr[s]; i < row_ptr[s + 1]; ++i) {
                const uint32_t u = outcome[i];
                if ((int64_t)u >= D) { free(phi); free(y); free(acc); free(hk); return -1; }
                y[u] = c_obs[i] * phi[u];
                hk[k] += c_obs[i] * (creal(phi[u]) * creal(phi[u]) + cimag(phi[u]) * cimag(phi[u]));
            }
            apply_setting_dagger(y, n, b);
            for (int64_t u = 0; u < D; ++u) acc[(int64_t)k * D + u] += y[u];
        }
    }
    for (int k = 0; k < K; ++k) {
        for (int64_t u = 0; u < D; ++u) {
            const cplx g = acc[(int64_t)k * D + u] / B;  /* (G psi_k)_u */
            if (G_psi) {
                G_psi[2 * ((int64_t)k * D + u)] = creal(g);
                G_psi[2 * ((int64_t)k * D + u) + 1] = cimag(g);
            }
            if (grad_psi) {
                grad_psi[2 * ((int64_t)k * D + u)] = -w[k] * creal(g);
                grad_psi[2 * ((int64_t)k * D + u) + 1] = -w[k] * cimag(g);
            }
        }
        if (h) h[k] = hk[k] / B;
    }
    free(phi);
    free(y);
    free(acc);
    free(hk);
    return 0;
}

/*
 * G v for arbitrary vectors (Eq. negative-gradient-product):
 *   out_j = (1/B) sum_s V_s^* (c_s .* (V_s v_j)),   j = 0..nv-1.
 * v, out: [nv][2^n] complex interleaved.  Returns 0, or -1 on malformed input.
 */
int qst_oracle_apply_G(int n, int M, int B, const uint8_t *basis,
                       const int64_t *row_ptr, const uint32_t *outcome,
                       const double *c_obs, int nv, const double *v, double *out)
{
    if (n < 1 || n > 30 || M < 0 || B < 1 || nv < 0) return -1;
    if (check_basis(n, M, basis)) return -1;
    const int64_t D = (int64_t)1 << n;
    cplx *phi = malloc(sizeof(cplx) * D);
    cplx *y = malloc(sizeof(cplx) * D);
    cplx *acc = malloc(sizeof(cplx) * D);
    if (!phi || !y || !acc) { free(phi); free(y); free(acc); return -1; }
    for (int j = 0; j < nv; ++j) {
        for (int64_t u = 0; u < D; ++u) acc[u] = 0.0;
        for (int s = 0; s < M; ++s) {
            const uint8_t *b = basis + (int64_t)s * n;
            load_vec(phi, v + 2 * (int64_t)j * D, D);
            apply_setting(phi, n, b);
            for (int64_t u = 0; u < D; ++u) y[u] = 0.0;
            for (int64_t i = row_ptr[s]; i < row_ptr[s + 1]; ++i) {
                const uint32_t u = outcome[i];
                if ((int64_t)u >= D) { free(phi); free(y); free(acc); return -1; }
                y[u] = c_obs[i] * phi[u];
            }
            apply_setting_dagger(y, n, b);
            for (int64_t u = 0; u < D; ++u) acc[u] += y[u];
        }
        for (int64_t u = 0; u < D; ++u) {
            out[2 * ((int64_t)j * D + u)] = creal(acc[u]) / B;
            out[2 * ((int64_t)j * D + u) + 1] = cimag(acc[u]) / B;
        }
    }
    free(phi);
    free(y);
    free(acc);
    return 0;
}

/* One rotated amplitude (V_s psi)_u by direct summation over all x:
 *   (V_s psi)_u = sum_x prod_j (V_{b_j})[u_j][x_j] psi_x.
 * Independent of the axis-by-axis application above; used for spot checks at
 * sizes where a full transform per setting is too slow.  out: (re, im). */
void qst_oracle_amplitude(int n, const uint8_t *b, const double *psi, uint32_t u,
                          double *out)
{
    const int64_t D = (int64_t)1 << n;
    cplx V[3][2][2];
    for (int t = 0; t < 3; ++t) rotation(t, V[t]);
    cplx acc = 0.0;
    for (int64_t x = 0; x < D; ++x) {
        cplx coef = 1.0;
        for (int q = 1; q <= n && coef != 0.0; ++q) {
            const int uq = (u >> (n - q)) & 1, xq = (int)((x >> (n - q)) & 1);
            coef *= V[b[q - 1]][uq][xq];
        }
        if (coef != 0.0) acc += coef * (psi[2 * x] + I * psi[2 * x + 1]);
    }
    out[0] = creal(acc);
    out[1] = cimag(acc);
}
