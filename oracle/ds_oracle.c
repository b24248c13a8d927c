/*
 * FP64 CPU oracle for the third-order directionally split exponential
 * Runge-Kutta integrator EXPRK3DS_REAL (Cassini, "Efficient third order
 * tensor-oriented directional splitting for exponential integrators",
 * arXiv 2310.07551).
 *
 * TEST INFRASTRUCTURE: this file is the plain, slow, independent reference
 * that the CUDA library is checked against.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it; the library
 * never does, and it shares no code, header or table with the CUDA sources.
 *
 * Conventions
 *   - Tensors are stored with mode 1 fastest (the paper's column-stacking
 *     vec, Section 2): element (i_1, ..., i_d) at i_1 + n_1 (i_2 + n_2 (...)).
 *   - Matrices are column-major: L[i + n j] is row i, column j.
 *   - Dimension arrays list n_1 first.  Everything is IEEE double, built
 *     without floating-point contraction so x86 and Arm hosts agree.
 *
 * Parity status: every function below is pinned by a test in tests/ against
 * an independent fact (order conditions, explicit Kronecker matrices, dense
 * expm of the assembled K, scalar closed forms, eigendecomposition,
 * observed order 3, steady-state invariance); none is "parity unpinned".
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 4

/* ------------------------------------------------------------------------ */
/* Split coefficients.                                                       */
/* d == 2: Table 1, real columns, "+" sign (Section 2.1 and 2.4).            */
/* d >= 3: Table 3, "+" sign in alpha_{1,mu}, eta_{2,d} scaled by 2^(d-3)    */
/*         (Section 2.3).                                                    */
/* Term i uses phi_{l_i}: l = (1, 2) for d == 2, (1, 2, 1) for d >= 3.       */
/* alpha is laid out alpha[i * 4 + mu] (mu 0-based).                        */
/* Returns the number of terms k, or -1 on bad input.                        */
/* ------------------------------------------------------------------------ */
int orc_coeffs(int d, int ell, int *ell_i, double *eta, double *alpha)
{
    if (d < 2 || d > ORC_MAXD || (ell != 1 && ell != 2)) return -1;
    memset(alpha, 0, sizeof(double) * 12);
    if (d == 2) {
        ell_i[0] = 1; ell_i[1] = 2;
        if (ell == 1) {
            double s = sqrt(10.0);
            eta[0] = -5.0 / 4.0;
            eta[1] = 9.0;
            alpha[0 * 4 + 0] = 4.0 * s / 15.0 + 4.0 / 3.0;
            alpha[0 * 4 + 1] = -4.0 * s / 15.0 + 4.0 / 3.0;
            alpha[1 * 4 + 0] = 2.0 * s / 9.0 + 16.0 / 9.0;
            alpha[1 * 4 + 1] = -2.0 * s / 9.0 + 16.0 / 9.0;
        } else {
            double s = sqrt(33.0);
            eta[0] = -4.0 / 3.0;
            eta[1] = 22.0 / 3.0;
            alpha[0 * 4 + 0] = s / 8.0 + 9.0 / 8.0;
            alpha[0 * 4 + 1] = -s / 8.0 + 9.0 / 8.0;
            alpha[1 * 4 + 0] = 3.0 * s / 22.0 + 3.0 / 2.0;
            alpha[1 * 4 + 1] = -3.0 * s / 22.0 + 3.0 / 2.0;
        }
        return 2;
    }
    ell_i[0] = 1; ell_i[1] = 2; ell_i[2] = 1;
    double scale = ldexp(1.0, d - 3);
    double a1, a2, a3;
    if (ell == 1) {
        double r = sqrt(2991111.0);
        eta[0] = 2243.0 / 1350.0 + 440521.0 / (675.0 * r);
        eta[1] = -12544.0 / 675.0 * scale;
        eta[2] = 2243.0 / 1350.0 - 440521.0 / (675.0 * r);
        a1 = 3.0 * (5161.0 + r) / 15869.0;
        a2 = 45.0 / 28.0;
        a3 = 3.0 * (5161.0 - r) / 15869.0;
    } else {
        double r = sqrt(2391.0);
        eta[0] = 19.0 / 27.0 + 151.0 / (27.0 * r);
        eta[1] = -196.0 / 27.0 * scale;
        eta[2] = 19.0 / 27.0 - 151.0 / (27.0 * r);
        a1 = 3.0 * (121.0 + r) / 490.0;
        a2 = 9.0 / 7.0;
        a3 = 3.0 * (121.0 - r) / 490.0;
    }
    for (int mu = 0; mu < d; ++mu) {
        alpha[0 * 4 + mu] = a1;
        alpha[1 * 4 + mu] = a2;
        alpha[2 * 4 + mu] = a3;
    }
    return 3;
}

/* ------------------------------------------------------------------------ */
/* Dense n x n helpers (column-major).                                       */
/* ------------------------------------------------------------------------ */
static void mat_mul(int n, const double *A, const double *B, double *C)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += A[i + (int64_t)n * q] * B[q + (int64_t)n * j];
            C[i + (int64_t)n * j] = s;
        }
    }
}

static double norm1(int n, const double *A)
{
    double best = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(A[i + (int64_t)n * j]);
        if (s > best) best = s;
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* phi_0 .. phi_lmax of a small dense matrix X (Section 1: the phi-functions */
/* are the power series sum_k X^k / (k + l)!).  Evaluated by scaling,        */
/* truncated Taylor series and the modified squaring of Skaflestad & Wright  */
/* (the paper's [SW09], Section 2.4):                                        */
/*   choose s >= 0 with ||2^-s X||_1 <= 1/2, Y = 2^-s X,                     */
/*   phi_k(Y) = sum_{j=0}^{q} Y^j / (j + k)!,  q = 16,                       */
/*   then s times: phi_0(2Y) = phi_0(Y)^2,                                   */
/*   phi_k(2Y) = 2^-k [phi_0(Y) phi_k(Y) + sum_{j=1}^{k} phi_j(Y)/(k-j)!].    */
/* out holds (lmax + 1) column-major n x n matrices.  Returns s, or -1.      */
/* ------------------------------------------------------------------------ */
int orc_phi(int n, const double *X, int lmax, double *out)
{
    if (n < 1 || lmax < 0 || lmax > 8) return -1;
    const int q = 16;
    int64_t nn = (int64_t)n * n;
    double nrm = norm1(n, X);
    int s = 0;
    while (ldexp(nrm, -s) > 0.5) ++s;
    double *Y = malloc(sizeof(double) * nn);
    double *Pw = malloc(sizeof(double) * nn);
    double *T = malloc(sizeof(double) * nn);
    double *old = malloc(sizeof(double) * nn * (lmax + 1));
    if (!Y || !Pw || !T || !old) { free(Y); free(Pw); free(T); free(old); return -1; }
    for (int64_t e = 0; e < nn; ++e) Y[e] = ldexp(X[e], -s);

    /* factorials 0! .. (q + lmax)! */
    double fact[32];
    fact[0] = 1.0;
    for (int j = 1; j < 32; ++j) fact[j] = fact[j - 1] * j;

    memset(out, 0, sizeof(double) * nn * (lmax + 1));
    /* Pw = Y^0 = I */
    memset(Pw, 0, sizeof(double) * nn);
    for (int i = 0; i < n; ++i) Pw[i + (int64_t)n * i] = 1.0;
    for (int j = 0; j <= q; ++j) {
        for (int k = 0; k <= lmax; ++k) {
            double c = 1.0 / fact[j + k];
            double *o = out + nn * k;
            for (int64_t e = 0; e < nn; ++e) o[e] += c * Pw[e];
        }
        if (j < q) {
            mat_mul(n, Pw, Y, T);
            memcpy(Pw, T, sizeof(double) * nn);
        }
    }
    for (int it = 0; it < s; ++it) {
        memcpy(old, out, sizeof(double) * nn * (lmax + 1));
        const double *p0 = old;
        /* phi_0(2Y) = phi_0(Y)^2 */
        mat_mul(n, p0, p0, out);
        for (int k = 1; k <= lmax; ++k) {
            double *o = out + nn * k;
            mat_mul(n, p0, old + nn * k, o);
            for (int j = 1; j <= k; ++j) {
                double c = 1.0 / fact[k - j];
                const double *pj = old + nn * j;
                for (int64_t e = 0; e < nn; ++e) o[e] += c * pj[e];
            }
            double w = ldexp(1.0, -k);
            for (int64_t e = 0; e < nn; ++e) o[e] *= w;
        }
    }
    free(Y); free(Pw); free(T); free(old);
    return s;
}

/* ------------------------------------------------------------------------ */
/* mu-mode product S = T x_mu L (Section 2):                                 */
/*   s_{i_1..i_d} = sum_j t_{i_1..j..i_d} l_{i_mu j}.                        */
/* mu is 0-based here (mode mu + 1 in the paper).  Plain loops, FP64         */
/* accumulator, natural j order.                                             */
/* ------------------------------------------------------------------------ */
/* Summation order of the mode products: 0 = j ascending (the default), */
/* 1 = j descending.  Running a computation both ways measures its FP64     */
/* rounding floor.                                                           */
static int g_reverse_sum = 0;
void orc_set_sum_order(int reverse) { g_reverse_sum = reverse != 0; }

/* Number of OpenMP threads of later calls (no effect without OpenMP).      */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

void orc_mode_product(int d, const int64_t *n, const double *X, int mu,
                      const double *L, double *Y)
{
    int64_t I = 1, O = 1, m = n[mu];
    for (int q = 0; q < mu; ++q) I *= n[q];
    for (int q = mu + 1; q < d; ++q) O *= n[q];
    const int rev = g_reverse_sum;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int64_t o = 0; o < O; ++o) {
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t x = 0; x < I; ++x) {
                double s = 0.0;
                for (int64_t jj = 0; jj < m; ++jj) {
                    const int64_t j = rev ? m - 1 - jj : jj;
                    s += L[i + m * j] * X[x + I * (j + m * o)];
                }
                Y[x + I * (i + m * o)] = s;
            }
        }
    }
}

static int64_t numel(int d, const int64_t *n)
{
    int64_t N = 1;
    for (int q = 0; q < d; ++q) N *= n[q];
    return N;
}

/* Tucker operator Y = X x_1 L_1 x_2 ... x_d L_d (Section 2, eq. krontomu). */
/* L[mu] points to the column-major n_mu x n_mu matrix of mode mu + 1.       */
int orc_tucker(int d, const int64_t *n, const double *X, const double *const *L, double *Y)
{
    int64_t N = numel(d, n);
    double *a = malloc(sizeof(double) * N), *b = malloc(sizeof(double) * N);
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, X, sizeof(double) * N);
    for (int mu = 0; mu < d; ++mu) {
        orc_mode_product(d, n, a, mu, L[mu], b);
        double *t = a; a = b; b = t;
    }
    memcpy(Y, a, sizeof(double) * N);
    free(a); free(b);
    return 0;
}

/* Action of the Kronecker sum in tensor form (Section 2.4, eq. kronsumv):   */
/* Y = sum_mu X x_mu A_mu.  Dense mode products, no stencil.                 */
int orc_kronsum(int d, const int64_t *n, const double *X, const double *const *A, double *Y)
{
    int64_t N = numel(d, n);
    double *t = malloc(sizeof(double) * N);
    if (!t) return -1;
    memset(Y, 0, sizeof(double) * N);
    for (int mu = 0; mu < d; ++mu) {
        orc_mode_product(d, n, X, mu, A[mu], t);
        for (int64_t e = 0; e < N; ++e) Y[e] += t[e];
    }
    free(t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reaction terms (Section 3 models; parameters as the workloads fix them).  */
/*   model 0, Schnakenberg, p = (gamma, a, b):                               */
/*     g_u = gamma (a - u + u^2 v),  g_v = gamma (b - u^2 v)                 */
/*   model 1, FitzHugh-Nagumo, p = (eps, alpha1, alpha0):                    */
/*     g_u = u - u^3 - v,            g_v = eps (u - alpha1 v - alpha0)       */
/*   model 2, linear test problem: g_u = g_v = 0 (pure diffusion).           */
/* U and G hold the two components back to back, N points each.             */
/* ------------------------------------------------------------------------ */
int orc_g(int model, const double *p, int64_t N, const double *U, double *G)
{
    if (model < 0 || model > 2) return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < N; ++e) {
        double u = U[e], v = U[N + e];
        if (model == 0) {
            double u2v = u * u * v;
            G[e] = p[0] * (p[1] - u + u2v);
            G[N + e] = p[0] * (p[2] - u2v);
        } else if (model == 1) {
            G[e] = u - u * u * u - v;
            G[N + e] = p[0] * (u - p[1] * v - p[2]);
        } else {
            G[e] = 0.0;
            G[N + e] = 0.0;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* phi-matrix set of Algorithms 1 and 2 ("Needed phi-functions").            */
/* For component c, slot q, term i and direction mu:                         */
/*   slot 0: P_{i,2}^{(1)} = phi_{l_i}(tau/3   alpha_{i,mu}^{(1)} A_{c,mu})   */
/*   slot 1: P_{i,3}^{(1)} = phi_{l_i}(2tau/3  alpha_{i,mu}^{(1)} A_{c,mu})   */
/*   slot 2: P_{i,3}^{(2)} = phi_{l_i}(2tau/3  alpha_{i,mu}^{(2)} A_{c,mu})   */
/*   slot 3: P_{i,f}^{(1)} = phi_{l_i}(tau     alpha_{i,mu}^{(1)} A_{c,mu})   */
/*   slot 4: P_{i,f}^{(2)} = phi_{l_i}(tau     alpha_{i,mu}^{(2)} A_{c,mu})   */
/* A holds, for c = 0, 1 and mu = 0..d-1 in that order, the column-major     */
/* n_mu x n_mu matrices A_{c,mu}.  P is written in the order                 */
/* [c][slot][i][mu], each block n_mu x n_mu, i over k terms.                 */
/* ------------------------------------------------------------------------ */
static const double kSlotC[5] = {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 1.0, 1.0};
static const int kSlotEll[5] = {1, 1, 2, 1, 2};

int64_t orc_phi_set_size(int d, const int64_t *n)
{
    int k = (d == 2) ? 2 : 3;
    int64_t per = 0;
    for (int mu = 0; mu < d; ++mu) per += n[mu] * n[mu];
    return 2 * 5 * k * per;
}

int orc_phi_set(int d, const int64_t *n, const double *A, double tau, double *P)
{
    if (d < 2 || d > ORC_MAXD || !(tau > 0.0)) return -1;
    int ell_i[3]; double eta[3], alpha[2][12];
    int k = orc_coeffs(d, 1, ell_i, eta, alpha[0]);
    orc_coeffs(d, 2, ell_i, eta, alpha[1]);
    int64_t nmax = 0;
    for (int mu = 0; mu < d; ++mu) if (n[mu] > nmax) nmax = n[mu];
    double *X = malloc(sizeof(double) * nmax * nmax);
    double *tmp = malloc(sizeof(double) * nmax * nmax * 3);
    if (!X || !tmp) { free(X); free(tmp); return -1; }
    const double *Acur = A;
    const double *Ac[2][ORC_MAXD];
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    double *out = P;
    for (int c = 0; c < 2; ++c) {
        for (int q = 0; q < 5; ++q) {
            for (int i = 0; i < k; ++i) {
                for (int mu = 0; mu < d; ++mu) {
                    int64_t m = n[mu], mm = m * m;
                    double z = kSlotC[q] * tau * alpha[kSlotEll[q] - 1][i * 4 + mu];
                    for (int64_t e = 0; e < mm; ++e) X[e] = z * Ac[c][mu][e];
                    if (orc_phi((int)m, X, ell_i[i], tmp) < 0) { free(X); free(tmp); return -1; }
                    memcpy(out, tmp + mm * ell_i[i], sizeof(double) * mm);
                    out += mm;
                }
            }
        }
    }
    free(X); free(tmp);
    return 0;
}

/* Pointer into the phi-set for (c, slot, term i, mu). */
static const double *pset_at(int d, const int64_t *n, int k, const double *P,
                             int c, int q, int i, int mu)
{
    int64_t per = 0;
    for (int v = 0; v < d; ++v) per += n[v] * n[v];
    const double *b = P + ((int64_t)c * 5 + q) * k * per + (int64_t)i * per;
    for (int v = 0; v < mu; ++v) b += n[v] * n[v];
    return b;
}

/* acc += w * sum_i eta_i T(X, {P_{c,q,i,mu}}_mu) */
static int split_action(int d, const int64_t *n, int k, const double *P, int c, int q,
                        const double *eta, double w, const double *X, double *acc, double *tmp)
{
    int64_t N = numel(d, n);
    double *s = malloc(sizeof(double) * N);
    if (!s) return -1;
    memset(s, 0, sizeof(double) * N);
    for (int i = 0; i < k; ++i) {
        const double *L[ORC_MAXD];
        for (int mu = 0; mu < d; ++mu) L[mu] = pset_at(d, n, k, P, c, q, i, mu);
        if (orc_tucker(d, n, X, L, tmp) < 0) { free(s); return -1; }
        for (int64_t e = 0; e < N; ++e) s[e] += eta[i] * tmp[e];
    }
    for (int64_t e = 0; e < N; ++e) acc[e] += w * s[e];
    free(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* nsteps steps of EXPRK3DS_REAL (Algorithm 1 for d == 2 with the real       */
/* Table 1 coefficients, Algorithm 2 for d >= 3 with Table 3), applied to    */
/* the two-component block system of Section 3 (eq. twocompdisc):            */
/*   G = g(U), F = K(U) + G                                                  */
/*   U2 = U + tau/3  S_2^{(1)}(F)                                            */
/*   D2 = g(U2) - G                                                          */
/*   U3 = U + 2tau/3 S_3^{(1)}(F) + 4tau/3 S_3^{(2)}(D2)                     */
/*   D3 = g(U3) - G                                                          */
/*   U <- U + tau S_f^{(1)}(F) + 3tau/2 S_f^{(2)}(D3)                        */
/* with S_s^{(l)}(X) = sum_i eta_i^{(l)} T(X, P_{i,s}^{(l)}).  The time      */
/* argument of g is dropped: both models are autonomous.                     */
/* A as in orc_phi_set; P from orc_phi_set; U is [2][N] in/out.              */
/* ------------------------------------------------------------------------ */
int orc_step(int d, const int64_t *n, const double *A, const double *P,
             int model, const double *p, double tau, double *U, int nsteps)
{
    if (d < 2 || d > ORC_MAXD || nsteps < 0) return -1;
    int ell_i[3]; double eta1[3], eta2[3], alpha[12];
    int k = orc_coeffs(d, 1, ell_i, eta1, alpha);
    orc_coeffs(d, 2, ell_i, eta2, alpha);
    int64_t N = numel(d, n);
    const double *Ac[2][ORC_MAXD];
    const double *Acur = A;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    double *G = malloc(sizeof(double) * 2 * N), *F = malloc(sizeof(double) * 2 * N);
    double *U2 = malloc(sizeof(double) * 2 * N), *U3 = malloc(sizeof(double) * 2 * N);
    double *Dt = malloc(sizeof(double) * 2 * N), *Un = malloc(sizeof(double) * 2 * N);
    double *tmp = malloc(sizeof(double) * N);
    int rc = -1;
    if (!G || !F || !U2 || !U3 || !Dt || !Un || !tmp) goto done;
    for (int step = 0; step < nsteps; ++step) {
        orc_g(model, p, N, U, G);
        for (int c = 0; c < 2; ++c) {
            if (orc_kronsum(d, n, U + c * N, Ac[c], F + c * N) < 0) goto done;
            for (int64_t e = 0; e < N; ++e) F[c * N + e] += G[c * N + e];
        }
        /* stage U_{n2} */
        memcpy(U2, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c)
            if (split_action(d, n, k, P, c, 0, eta1, tau / 3.0, F + c * N, U2 + c * N, tmp) < 0) goto done;
        orc_g(model, p, N, U2, Dt);
        for (int64_t e = 0; e < 2 * N; ++e) Dt[e] -= G[e];
        /* stage U_{n3} */
        memcpy(U3, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c) {
            if (split_action(d, n, k, P, c, 1, eta1, 2.0 * tau / 3.0, F + c * N, U3 + c * N, tmp) < 0) goto done;
            if (split_action(d, n, k, P, c, 2, eta2, 4.0 * tau / 3.0, Dt + c * N, U3 + c * N, tmp) < 0) goto done;
        }
        orc_g(model, p, N, U3, Dt);
        for (int64_t e = 0; e < 2 * N; ++e) Dt[e] -= G[e];
        /* final approximation U_{n+1} */
        memcpy(Un, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c) {
            if (split_action(d, n, k, P, c, 3, eta1, tau, F + c * N, Un + c * N, tmp) < 0) goto done;
            if (split_action(d, n, k, P, c, 4, eta2, 1.5 * tau, Dt + c * N, Un + c * N, tmp) < 0) goto done;
        }
        memcpy(U, Un, sizeof(double) * 2 * N);
    }
    rc = 0;
done:
    free(G); free(F); free(U2); free(U3); free(Dt); free(Un); free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Unsplit EXPRK3 (Section 2.4, eq. exprk3): the tableau of orc_step with    */
/* every split action replaced by the dense phi_l(c tau K_c) applied to the  */
/* vector, K_c = A_{c,d} (+) ... (+) A_{c,1} assembled as an N x N matrix    */
/* (Section 1, eq. kronsum) and phi by orc_phi.  This is what the splits     */
/* approximate; dense N x N matrices, so small grids only.                   */
/* ------------------------------------------------------------------------ */
static void kron_sum_dense(int d, const int64_t *n, const double *const *Ac, double *K)
{
    int64_t N = numel(d, n);
    memset(K, 0, sizeof(double) * N * N);
    for (int64_t j = 0; j < N; ++j) {
        int64_t rest = j, stride = 1;
        for (int mu = 0; mu < d; ++mu) {
            const int64_t jm = rest % n[mu];
            rest /= n[mu];
            for (int64_t im = 0; im < n[mu]; ++im) {
                const int64_t i = j + (im - jm) * stride;
                K[i + N * j] += Ac[mu][im + n[mu] * jm];
            }
            stride *= n[mu];
        }
    }
}

/* out += w * (P x), P column-major N x N */
static void dense_apply(int64_t N, const double *P, double w, const double *x, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) s += P[i + N * j] * x[j];
        out[i] += w * s;
    }
}

int orc_step_dense(int d, const int64_t *n, const double *A, int model, const double *p, double tau,
                   double *U, int nsteps)
{
    if (d < 2 || d > ORC_MAXD || nsteps < 0 || !(tau > 0.0)) return -1;
    const int64_t N = numel(d, n), NN = N * N;
    const double *Ac[2][ORC_MAXD];
    const double *Acur = A;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    /* per component: phi_1(tau/3 K), phi_1(2tau/3 K), phi_2(2tau/3 K), phi_1(tau K), phi_2(tau K) */
    double *Pm = malloc(sizeof(double) * NN * 10), *K = malloc(sizeof(double) * NN);
    double *X = malloc(sizeof(double) * NN), *ph = malloc(sizeof(double) * NN * 3);
    double *G = malloc(sizeof(double) * 2 * N), *F = malloc(sizeof(double) * 2 * N);
    double *U2 = malloc(sizeof(double) * 2 * N), *U3 = malloc(sizeof(double) * 2 * N);
    double *Dt = malloc(sizeof(double) * 2 * N), *Un = malloc(sizeof(double) * 2 * N);
    int rc = -1;
    if (!Pm || !K || !X || !ph || !G || !F || !U2 || !U3 || !Dt || !Un) goto done;
    const double cq[3] = {1.0 / 3.0, 2.0 / 3.0, 1.0};
    for (int c = 0; c < 2; ++c) {
        kron_sum_dense(d, n, Ac[c], K);
        for (int q = 0; q < 3; ++q) {
            for (int64_t e = 0; e < NN; ++e) X[e] = cq[q] * tau * K[e];
            if (orc_phi((int)N, X, 2, ph) < 0) goto done;
            double *base = Pm + NN * 5 * c;
            if (q == 0) memcpy(base, ph + NN, sizeof(double) * NN);
            if (q == 1) { memcpy(base + NN, ph + NN, sizeof(double) * NN); memcpy(base + 2 * NN, ph + 2 * NN, sizeof(double) * NN); }
            if (q == 2) { memcpy(base + 3 * NN, ph + NN, sizeof(double) * NN); memcpy(base + 4 * NN, ph + 2 * NN, sizeof(double) * NN); }
        }
    }
    for (int step = 0; step < nsteps; ++step) {
        orc_g(model, p, N, U, G);
        for (int c = 0; c < 2; ++c) {
            kron_sum_dense(d, n, Ac[c], K);
            for (int64_t i = 0; i < N; ++i) {
                double s = 0.0;
                for (int64_t j = 0; j < N; ++j) s += K[i + N * j] * U[c * N + j];
                F[c * N + i] = s + G[c * N + i];
            }
        }
        memcpy(U2, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c) dense_apply(N, Pm + NN * (5 * c + 0), tau / 3.0, F + c * N, U2 + c * N);
        orc_g(model, p, N, U2, Dt);
        for (int64_t e = 0; e < 2 * N; ++e) Dt[e] -= G[e];
        memcpy(U3, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c) {
            dense_apply(N, Pm + NN * (5 * c + 1), 2.0 * tau / 3.0, F + c * N, U3 + c * N);
            dense_apply(N, Pm + NN * (5 * c + 2), 4.0 * tau / 3.0, Dt + c * N, U3 + c * N);
        }
        orc_g(model, p, N, U3, Dt);
        for (int64_t e = 0; e < 2 * N; ++e) Dt[e] -= G[e];
        memcpy(Un, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c) {
            dense_apply(N, Pm + NN * (5 * c + 3), tau, F + c * N, Un + c * N);
            dense_apply(N, Pm + NN * (5 * c + 4), 1.5 * tau, Dt + c * N, Un + c * N);
        }
        memcpy(U, Un, sizeof(double) * 2 * N);
    }
    rc = 0;
done:
    free(Pm); free(K); free(X); free(ph); free(G); free(F); free(U2); free(U3); free(Dt); free(Un);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of one EXPRK3DS_REAL step (reverse mode of orc_step; the paper    */
/* has no adjoint, this is the exact transpose of the step above).           */
/* Forward values are recomputed from U = U_n.  With lam = dL/dU_{n+1}:      */
/*   lam_F  = tau S_f^{(1)T}(lam),  lam_D3 = 3tau/2 S_f^{(2)T}(lam)            */
/*   lam_U3 = J_g(U3)^T lam_D3                                               */
/*   lam_F += 2tau/3 S_3^{(1)T}(lam_U3),  lam_D2 = 4tau/3 S_3^{(2)T}(lam_U3)   */
/*   lam_U2 = J_g(U2)^T lam_D2                                               */
/*   lam_F += tau/3 S_2^{(1)T}(lam_U2)                                        */
/*   lam_G  = lam_F - lam_D2 - lam_D3                                        */
/*   lam_n  = lam + lam_U3 + lam_U2 + K^T lam_F + J_g(U)^T lam_G             */
/* where S^T(X) = sum_i eta_i T(X, {P_{i,s}{mu}^T}).  dp[q] += dL/dp_q for   */
/* the three model parameters:                                               */
/*   (dg/dp)(U)^T lam_G + (dg/dp)(U2)^T lam_D2 + (dg/dp)(U3)^T lam_D3.        */
/* ------------------------------------------------------------------------ */
static void transpose_into(int64_t m, const double *L, double *T)
{
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = 0; i < m; ++i) T[j + m * i] = L[i + m * j];
}

/* acc += w * sum_i eta_i T(X, {P_{c,q,i,mu}^T}) */
static int split_action_T(int d, const int64_t *n, int k, const double *P, int c, int q,
                          const double *eta, double w, const double *X, double *acc, double *tmp)
{
    int64_t N = numel(d, n);
    double *s = malloc(sizeof(double) * N);
    double *Ts[ORC_MAXD] = {0};
    int rc = -1;
    if (!s) return -1;
    memset(s, 0, sizeof(double) * N);
    for (int mu = 0; mu < d; ++mu) {
        Ts[mu] = malloc(sizeof(double) * n[mu] * n[mu]);
        if (!Ts[mu]) goto out;
    }
    for (int i = 0; i < k; ++i) {
        const double *L[ORC_MAXD];
        for (int mu = 0; mu < d; ++mu) {
            transpose_into(n[mu], pset_at(d, n, k, P, c, q, i, mu), Ts[mu]);
            L[mu] = Ts[mu];
        }
        if (orc_tucker(d, n, X, L, tmp) < 0) goto out;
        for (int64_t e = 0; e < N; ++e) s[e] += eta[i] * tmp[e];
    }
    for (int64_t e = 0; e < N; ++e) acc[e] += w * s[e];
    rc = 0;
out:
    for (int mu = 0; mu < d; ++mu) free(Ts[mu]);
    free(s);
    return rc;
}

/* J_g(U)^T lam added into out; model as in orc_g */
static void jacT_add(int model, const double *p, int64_t N, const double *U, const double *lam,
                     double *out)
{
    for (int64_t e = 0; e < N; ++e) {
        double u = U[e], v = U[N + e], lu = lam[e], lv = lam[N + e];
        double juu, juv, jvu, jvv;
        if (model == 0) {
            juu = p[0] * (-1.0 + 2.0 * u * v);
            juv = p[0] * u * u;
            jvu = -2.0 * p[0] * u * v;
            jvv = -p[0] * u * u;
        } else if (model == 1) {
            juu = 1.0 - 3.0 * u * u;
            juv = -1.0;
            jvu = p[0];
            jvv = -p[0] * p[1];
        } else {
            juu = juv = jvu = jvv = 0.0;
        }
        out[e] += juu * lu + jvu * lv;
        out[N + e] += juv * lu + jvv * lv;
    }
}

/* dp += (dg/dp)(U)^T lam, the three model parameters */
static void dparam_add(int model, const double *p, int64_t N, const double *U, const double *lam,
                       double *dp)
{
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t e = 0; e < N; ++e) {
        double u = U[e], v = U[N + e], lu = lam[e], lv = lam[N + e];
        if (model == 0) {
            a0 += (p[1] - u + u * u * v) * lu + (p[2] - u * u * v) * lv;
            a1 += p[0] * lu;
            a2 += p[0] * lv;
        } else if (model == 1) {
            a0 += (u - p[1] * v - p[2]) * lv;
            a1 += -p[0] * v * lv;
            a2 += -p[0] * lv;
        }
    }
    dp[0] += a0;
    dp[1] += a1;
    dp[2] += a2;
}

/* dL/ds_c for A_{c,mu}(s) = s A_{c,mu} at s = 1, for one Tucker operator     */
/* family: sum_i sum_mu < Ybar_i, T(X, {P_i{nu}}, P_i{mu} -> dP_i{mu}) > with */
/* Ybar_i = w eta_i lam_s and dP = d/ds phi_l(s Z) = phi_{l-1}(Z) - l phi_l(Z), */
/* Z = c_q tau alpha_{i,mu} A_{c,mu} (Z phi_l'(Z), from the power series).      */
static int dscale_family(int d, const int64_t *n, int k, const double *P, const double *const *Ac,
                         int c, int q, double tau, const double *eta, double w, const double *X,
                         const double *lam_s, double *acc, double *tmp)
{
    int ell_i[3]; double e_[3], alpha[12];
    orc_coeffs(d, kSlotEll[q], ell_i, e_, alpha);
    int64_t N = numel(d, n), nmax = 0;
    for (int mu = 0; mu < d; ++mu) if (n[mu] > nmax) nmax = n[mu];
    double *Z = malloc(sizeof(double) * nmax * nmax), *ph = malloc(sizeof(double) * nmax * nmax * 3);
    double *dP = malloc(sizeof(double) * nmax * nmax);
    int rc = -1;
    if (!Z || !ph || !dP) goto out;
    for (int i = 0; i < k; ++i) {
        for (int mu = 0; mu < d; ++mu) {
            int64_t m = n[mu], mm = m * m;
            double z = kSlotC[q] * tau * alpha[i * 4 + mu];
            for (int64_t e = 0; e < mm; ++e) Z[e] = z * Ac[mu][e];
            int l = ell_i[i];
            if (orc_phi((int)m, Z, l, ph) < 0) goto out;
            for (int64_t e = 0; e < mm; ++e) dP[e] = ph[mm * (l - 1) + e] - l * ph[mm * l + e];
            const double *L[ORC_MAXD];
            for (int nu = 0; nu < d; ++nu) L[nu] = (nu == mu) ? dP : pset_at(d, n, k, P, c, q, i, nu);
            if (orc_tucker(d, n, X, L, tmp) < 0) goto out;
            double dot = 0.0;
            for (int64_t e = 0; e < N; ++e) dot += lam_s[e] * tmp[e];
            *acc += w * eta[i] * dot;
        }
    }
    rc = 0;
out:
    free(Z); free(ph); free(dP);
    return rc;
}

int orc_step_adjoint(int d, const int64_t *n, const double *A, const double *P, int model,
                     const double *p, double tau, const double *U, const double *lam,
                     double *lam_out, double *dp, double *dscale)
{
    if (d < 2 || d > ORC_MAXD) return -1;
    int ell_i[3]; double eta1[3], eta2[3], alpha[12];
    int k = orc_coeffs(d, 1, ell_i, eta1, alpha);
    orc_coeffs(d, 2, ell_i, eta2, alpha);
    int64_t N = numel(d, n);
    const double *Ac[2][ORC_MAXD];
    const double *Acur = A;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    int64_t nb = 2 * N;
    double *G = malloc(sizeof(double) * nb), *F = malloc(sizeof(double) * nb);
    double *U2 = malloc(sizeof(double) * nb), *U3 = malloc(sizeof(double) * nb);
    double *D2 = malloc(sizeof(double) * nb), *lF = malloc(sizeof(double) * nb);
    double *lD2 = malloc(sizeof(double) * nb), *lD3 = malloc(sizeof(double) * nb);
    double *lU2 = malloc(sizeof(double) * nb), *lU3 = malloc(sizeof(double) * nb);
    double *tmp = malloc(sizeof(double) * N), *At = NULL;
    int rc = -1;
    if (!G || !F || !U2 || !U3 || !D2 || !lF || !lD2 || !lD3 || !lU2 || !lU3 || !tmp) goto done;
    /* forward recomputation */
    orc_g(model, p, N, U, G);
    for (int c = 0; c < 2; ++c) {
        if (orc_kronsum(d, n, U + c * N, Ac[c], F + c * N) < 0) goto done;
        for (int64_t e = 0; e < N; ++e) F[c * N + e] += G[c * N + e];
    }
    memcpy(U2, U, sizeof(double) * nb);
    for (int c = 0; c < 2; ++c)
        if (split_action(d, n, k, P, c, 0, eta1, tau / 3.0, F + c * N, U2 + c * N, tmp) < 0) goto done;
    orc_g(model, p, N, U2, D2);
    for (int64_t e = 0; e < nb; ++e) D2[e] -= G[e];
    memcpy(U3, U, sizeof(double) * nb);
    for (int c = 0; c < 2; ++c) {
        if (split_action(d, n, k, P, c, 1, eta1, 2.0 * tau / 3.0, F + c * N, U3 + c * N, tmp) < 0) goto done;
        if (split_action(d, n, k, P, c, 2, eta2, 4.0 * tau / 3.0, D2 + c * N, U3 + c * N, tmp) < 0) goto done;
    }
    /* reverse sweep */
    memset(lF, 0, sizeof(double) * nb);
    memset(lD3, 0, sizeof(double) * nb);
    memset(lD2, 0, sizeof(double) * nb);
    memset(lU2, 0, sizeof(double) * nb);
    memset(lU3, 0, sizeof(double) * nb);
    for (int c = 0; c < 2; ++c) {
        if (split_action_T(d, n, k, P, c, 3, eta1, tau, lam + c * N, lF + c * N, tmp) < 0) goto done;
        if (split_action_T(d, n, k, P, c, 4, eta2, 1.5 * tau, lam + c * N, lD3 + c * N, tmp) < 0) goto done;
    }
    jacT_add(model, p, N, U3, lD3, lU3);
    for (int c = 0; c < 2; ++c) {
        if (split_action_T(d, n, k, P, c, 1, eta1, 2.0 * tau / 3.0, lU3 + c * N, lF + c * N, tmp) < 0) goto done;
        if (split_action_T(d, n, k, P, c, 2, eta2, 4.0 * tau / 3.0, lU3 + c * N, lD2 + c * N, tmp) < 0) goto done;
    }
    jacT_add(model, p, N, U2, lD2, lU2);
    for (int c = 0; c < 2; ++c)
        if (split_action_T(d, n, k, P, c, 0, eta1, tau / 3.0, lU2 + c * N, lF + c * N, tmp) < 0) goto done;
    /* lam_n = lam + lam_U3 + lam_U2 + K^T lam_F + J_g(U)^T (lam_F - lam_D2 - lam_D3) */
    for (int64_t e = 0; e < nb; ++e) lam_out[e] = lam[e] + lU3[e] + lU2[e];
    {
        int64_t nmax = 0;
        for (int mu = 0; mu < d; ++mu) if (n[mu] > nmax) nmax = n[mu];
        At = malloc(sizeof(double) * nmax * nmax * ORC_MAXD);
        if (!At) goto done;
        for (int c = 0; c < 2; ++c) {
            const double *AT[ORC_MAXD];
            for (int mu = 0; mu < d; ++mu) {
                transpose_into(n[mu], Ac[c][mu], At + nmax * nmax * mu);
                AT[mu] = At + nmax * nmax * mu;
            }
            if (orc_kronsum(d, n, lF + c * N, AT, tmp) < 0) goto done;
            for (int64_t e = 0; e < N; ++e) lam_out[c * N + e] += tmp[e];
        }
    }
    /* lG reuses lU2's storage after its last use: lG = lF - lD2 - lD3 */
    for (int64_t e = 0; e < nb; ++e) lU2[e] = lF[e] - lD2[e] - lD3[e];
    jacT_add(model, p, N, U, lU2, lam_out);
    if (dp) {
        /* D3's forward value is not needed: only U3 enters (dg/dp)(U3) */
        dparam_add(model, p, N, U, lU2, dp);
        dparam_add(model, p, N, U2, lD2, dp);
        dparam_add(model, p, N, U3, lD3, dp);
    }
    if (dscale) {
        /* lU2 now holds lam_G; recompute lam_U2 = J_g(U2)^T lam_D2 and D3 */
        double *lU2b = malloc(sizeof(double) * nb), *D3 = malloc(sizeof(double) * nb);
        if (!lU2b || !D3) { free(lU2b); free(D3); goto done; }
        memset(lU2b, 0, sizeof(double) * nb);
        jacT_add(model, p, N, U2, lD2, lU2b);
        orc_g(model, p, N, U3, D3);
        for (int64_t e = 0; e < nb; ++e) D3[e] -= G[e];
        int bad = 0;
        for (int c = 0; c < 2 && !bad; ++c) {
            double acc = 0.0;
            /* through K: F = s K U + G */
            for (int64_t e = 0; e < N; ++e) acc += lF[c * N + e] * (F[c * N + e] - G[c * N + e]);
            const double *Fc = F + c * N, *Dc2 = D2 + c * N, *Dc3 = D3 + c * N;
            bad |= dscale_family(d, n, k, P, Ac[c], c, 0, tau, eta1, tau / 3.0, Fc, lU2b + c * N, &acc, tmp) < 0;
            bad |= dscale_family(d, n, k, P, Ac[c], c, 1, tau, eta1, 2.0 * tau / 3.0, Fc, lU3 + c * N, &acc, tmp) < 0;
            bad |= dscale_family(d, n, k, P, Ac[c], c, 2, tau, eta2, 4.0 * tau / 3.0, Dc2, lU3 + c * N, &acc, tmp) < 0;
            bad |= dscale_family(d, n, k, P, Ac[c], c, 3, tau, eta1, tau, Fc, lam + c * N, &acc, tmp) < 0;
            bad |= dscale_family(d, n, k, P, Ac[c], c, 4, tau, eta2, 1.5 * tau, Dc3, lam + c * N, &acc, tmp) < 0;
            dscale[c] += acc;
        }
        free(lU2b); free(D3);
        if (bad) goto done;
    }
    rc = 0;
done:
    free(G); free(F); free(U2); free(U3); free(D2); free(lF); free(lD2); free(lD3);
    free(lU2); free(lU3); free(tmp); free(At);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* ETD2RKDS: the exponential Runge-Kutta scheme ETD2RK (Section 1,          */
/* eq. ETD2RK) with the second-order directional split of the phi-actions   */
/* (Section 2, eq. secondord):                                               */
/*   phi_l(tau K) v ~ l!^(d-1) T(V, {phi_l(tau A_mu)}).                      */
/* phi-set layout: [c][l - 1][mu], column-major n_mu x n_mu blocks.          */
/*   G = g(U), F = K U + G                                                   */
/*   U2 = U + tau T(F, {phi_1(tau A_{c,mu})})                                */
/*   U <- U2 + tau 2^(d-1) T(g(U2) - G, {phi_2(tau A_{c,mu})})               */
/* ------------------------------------------------------------------------ */
int64_t orc_phi_set2_size(int d, const int64_t *n)
{
    int64_t per = 0;
    for (int mu = 0; mu < d; ++mu) per += n[mu] * n[mu];
    return 2 * 2 * per;
}

int orc_phi_set2(int d, const int64_t *n, const double *A, double tau, double *P)
{
    if (d < 2 || d > ORC_MAXD || !(tau > 0.0)) return -1;
    int64_t nmax = 0;
    for (int mu = 0; mu < d; ++mu) if (n[mu] > nmax) nmax = n[mu];
    double *X = malloc(sizeof(double) * nmax * nmax), *ph = malloc(sizeof(double) * nmax * nmax * 3);
    if (!X || !ph) { free(X); free(ph); return -1; }
    const double *Acur = A;
    const double *Ac[2][ORC_MAXD];
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    double *out = P;
    for (int c = 0; c < 2; ++c)
        for (int l = 1; l <= 2; ++l)
            for (int mu = 0; mu < d; ++mu) {
                int64_t mm = n[mu] * n[mu];
                for (int64_t e = 0; e < mm; ++e) X[e] = tau * Ac[c][mu][e];
                if (orc_phi((int)n[mu], X, l, ph) < 0) { free(X); free(ph); return -1; }
                memcpy(out, ph + mm * l, sizeof(double) * mm);
                out += mm;
            }
    free(X); free(ph);
    return 0;
}

int orc_step2(int d, const int64_t *n, const double *A, const double *P, int model, const double *p,
              double tau, double *U, int nsteps)
{
    if (d < 2 || d > ORC_MAXD || nsteps < 0) return -1;
    int64_t N = numel(d, n), per = 0;
    for (int mu = 0; mu < d; ++mu) per += n[mu] * n[mu];
    const double *Ac[2][ORC_MAXD];
    const double *Acur = A;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    double *G = malloc(sizeof(double) * 2 * N), *F = malloc(sizeof(double) * 2 * N);
    double *U2 = malloc(sizeof(double) * 2 * N), *D = malloc(sizeof(double) * 2 * N);
    double *T = malloc(sizeof(double) * N);
    int rc = -1;
    if (!G || !F || !U2 || !D || !T) goto done;
    const double w2 = ldexp(1.0, d - 1);   /* 2!^(d-1) */
    for (int step = 0; step < nsteps; ++step) {
        orc_g(model, p, N, U, G);
        for (int c = 0; c < 2; ++c) {
            if (orc_kronsum(d, n, U + c * N, Ac[c], F + c * N) < 0) goto done;
            for (int64_t e = 0; e < N; ++e) F[c * N + e] += G[c * N + e];
        }
        for (int c = 0; c < 2; ++c) {
            const double *L[ORC_MAXD];
            const double *b = P + ((int64_t)c * 2 + 0) * per;
            for (int mu = 0; mu < d; ++mu) { L[mu] = b; b += n[mu] * n[mu]; }
            if (orc_tucker(d, n, F + c * N, L, T) < 0) goto done;
            for (int64_t e = 0; e < N; ++e) U2[c * N + e] = U[c * N + e] + tau * T[e];
        }
        orc_g(model, p, N, U2, D);
        for (int64_t e = 0; e < 2 * N; ++e) D[e] -= G[e];
        for (int c = 0; c < 2; ++c) {
            const double *L[ORC_MAXD];
            const double *b = P + ((int64_t)c * 2 + 1) * per;
            for (int mu = 0; mu < d; ++mu) { L[mu] = b; b += n[mu] * n[mu]; }
            if (orc_tucker(d, n, D + c * N, L, T) < 0) goto done;
            for (int64_t e = 0; e < N; ++e) U[c * N + e] = U2[c * N + e] + tau * w2 * T[e];
        }
    }
    rc = 0;
done:
    free(G); free(F); free(U2); free(D); free(T);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* EXPRK3DS_CPLX: Algorithm 1 with the complex two-term coefficients of     */
/* Table 2 (Section 2.2, eq. splitnd; l_1 = 1, l_2 = 2, upper signs,         */
/* eta_{2,d} with 2^(d-2)).  Each split action is complex; the increment is  */
/* its real part (the state is real).  Complex values are C99 double        */
/* complex, laid out as (re, im) pairs.                                      */
/* ------------------------------------------------------------------------ */
#include <complex.h>
typedef double complex cplx;

int orc_coeffs_cplx(int d, int ell, double *eta, double *alpha)
{
    /* eta[2*i], eta[2*i+1] = re, im of eta_i; alpha likewise (same for every mu) */
    if (d < 2 || d > ORC_MAXD || (ell != 1 && ell != 2)) return -1;
    double s = ldexp(1.0, d - 2);
    cplx e1, a1, e2, a2;
    if (ell == 1) {
        e1 = 7.0 / 4.0 + 3.0 * sqrt(2.0) / 2.0 * I;
        a1 = 12.0 / 11.0 - 4.0 * sqrt(2.0) / 11.0 * I;
        e2 = s * (-3.0 - 6.0 * sqrt(2.0) * I);
        a2 = 4.0 / 3.0 - 2.0 * sqrt(2.0) / 3.0 * I;
    } else {
        e1 = 2.0 / 3.0 + 2.0 * sqrt(3.0) / 3.0 * I;
        a1 = 3.0 / 4.0 - sqrt(3.0) / 4.0 * I;
        e2 = s * (-2.0 / 3.0 - 8.0 * sqrt(3.0) / 3.0 * I);
        a2 = 6.0 / 7.0 - 3.0 * sqrt(3.0) / 7.0 * I;
    }
    eta[0] = creal(e1); eta[1] = cimag(e1); eta[2] = creal(e2); eta[3] = cimag(e2);
    alpha[0] = creal(a1); alpha[1] = cimag(a1); alpha[2] = creal(a2); alpha[3] = cimag(a2);
    return 2;
}

static void cmat_mul(int n, const cplx *A, const cplx *B, cplx *C)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            cplx s = 0.0;
            for (int q = 0; q < n; ++q) s += A[i + (int64_t)n * q] * B[q + (int64_t)n * j];
            C[i + (int64_t)n * j] = s;
        }
}

/* phi_0..phi_lmax of a complex matrix: the scaling / Taylor / modified      */
/* squaring of orc_phi, in complex arithmetic.                               */
int orc_phi_cplx(int n, const double *Xd, int lmax, double *outd)
{
    const cplx *X = (const cplx *)Xd;
    cplx *out = (cplx *)outd;
    if (n < 1 || lmax < 0 || lmax > 8) return -1;
    const int q = 16;
    int64_t nn = (int64_t)n * n;
    double nrm = 0.0;
    for (int j = 0; j < n; ++j) {
        double sc = 0.0;
        for (int i = 0; i < n; ++i) sc += cabs(X[i + (int64_t)n * j]);
        if (sc > nrm) nrm = sc;
    }
    int s = 0;
    while (ldexp(nrm, -s) > 0.5) ++s;
    cplx *Y = malloc(sizeof(cplx) * nn), *Pw = malloc(sizeof(cplx) * nn), *T = malloc(sizeof(cplx) * nn);
    cplx *old = malloc(sizeof(cplx) * nn * (lmax + 1));
    if (!Y || !Pw || !T || !old) { free(Y); free(Pw); free(T); free(old); return -1; }
    for (int64_t e = 0; e < nn; ++e) Y[e] = ldexp(1.0, -s) * X[e];
    double fact[32];
    fact[0] = 1.0;
    for (int j = 1; j < 32; ++j) fact[j] = fact[j - 1] * j;
    for (int64_t e = 0; e < nn * (lmax + 1); ++e) out[e] = 0.0;
    for (int64_t e = 0; e < nn; ++e) Pw[e] = 0.0;
    for (int i = 0; i < n; ++i) Pw[i + (int64_t)n * i] = 1.0;
    for (int j = 0; j <= q; ++j) {
        for (int k = 0; k <= lmax; ++k) {
            double c = 1.0 / fact[j + k];
            cplx *o = out + nn * k;
            for (int64_t e = 0; e < nn; ++e) o[e] += c * Pw[e];
        }
        if (j < q) {
            cmat_mul(n, Pw, Y, T);
            memcpy(Pw, T, sizeof(cplx) * nn);
        }
    }
    for (int it = 0; it < s; ++it) {
        memcpy(old, out, sizeof(cplx) * nn * (lmax + 1));
        cmat_mul(n, old, old, out);
        for (int k = 1; k <= lmax; ++k) {
            cplx *o = out + nn * k;
            cmat_mul(n, old, old + nn * k, o);
            for (int j = 1; j <= k; ++j) {
                double c = 1.0 / fact[k - j];
                const cplx *pj = old + nn * j;
                for (int64_t e = 0; e < nn; ++e) o[e] += c * pj[e];
            }
            double w = ldexp(1.0, -k);
            for (int64_t e = 0; e < nn; ++e) o[e] *= w;
        }
    }
    free(Y); free(Pw); free(T); free(old);
    return s;
}

static void cmode_product(int d, const int64_t *n, const cplx *X, int mu, const cplx *L, cplx *Y)
{
    int64_t In = 1, On = 1, m = n[mu];
    for (int q = 0; q < mu; ++q) In *= n[q];
    for (int q = mu + 1; q < d; ++q) On *= n[q];
    #pragma omp parallel for collapse(2) schedule(static)
    for (int64_t o = 0; o < On; ++o)
        for (int64_t i = 0; i < m; ++i)
            for (int64_t x = 0; x < In; ++x) {
                cplx s = 0.0;
                for (int64_t j = 0; j < m; ++j) s += L[i + m * j] * X[x + In * (j + m * o)];
                Y[x + In * (i + m * o)] = s;
            }
}

/* phi-set of the complex scheme: [c][slot][i][mu] complex blocks, k = 2 */
int64_t orc_phi_set_cplx_size(int d, const int64_t *n)
{
    int64_t per = 0;
    for (int mu = 0; mu < d; ++mu) per += n[mu] * n[mu];
    return 2 * 2 * 5 * 2 * per;   /* doubles: 2 comps, 5 slots, 2 terms, (re, im) */
}

int orc_phi_set_cplx(int d, const int64_t *n, const double *A, double tau, double *Pd)
{
    cplx *P = (cplx *)Pd;
    if (d < 2 || d > ORC_MAXD || !(tau > 0.0)) return -1;
    double eta[2][4], alpha[2][4];
    orc_coeffs_cplx(d, 1, eta[0], alpha[0]);
    orc_coeffs_cplx(d, 2, eta[1], alpha[1]);
    int64_t nmax = 0;
    for (int mu = 0; mu < d; ++mu) if (n[mu] > nmax) nmax = n[mu];
    cplx *X = malloc(sizeof(cplx) * nmax * nmax), *ph = malloc(sizeof(cplx) * nmax * nmax * 3);
    if (!X || !ph) { free(X); free(ph); return -1; }
    const double *Ac[2][ORC_MAXD];
    const double *Acur = A;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    cplx *out = P;
    for (int c = 0; c < 2; ++c)
        for (int q = 0; q < 5; ++q) {
            const double *al = alpha[kSlotEll[q] - 1];
            for (int i = 0; i < 2; ++i)
                for (int mu = 0; mu < d; ++mu) {
                    int64_t mm = n[mu] * n[mu];
                    cplx z = kSlotC[q] * tau * (al[2 * i] + al[2 * i + 1] * I);
                    for (int64_t e = 0; e < mm; ++e) X[e] = z * Ac[c][mu][e];
                    int l = i + 1;   /* l_1 = 1, l_2 = 2 */
                    if (orc_phi_cplx((int)n[mu], (const double *)X, l, (double *)ph) < 0) { free(X); free(ph); return -1; }
                    memcpy(out, ph + mm * l, sizeof(cplx) * mm);
                    out += mm;
                }
        }
    free(X); free(ph);
    return 0;
}

/* acc += w Re(sum_i eta_i T(X, {P_{c,q,i,mu}})), X real */
static int split_action_cplx(int d, const int64_t *n, const cplx *P, int c, int q, const double *eta,
                             double w, const double *X, double *acc)
{
    int64_t N = numel(d, n), per = 0;
    for (int mu = 0; mu < d; ++mu) per += n[mu] * n[mu];
    cplx *a = malloc(sizeof(cplx) * N), *b = malloc(sizeof(cplx) * N);
    if (!a || !b) { free(a); free(b); return -1; }
    for (int i = 0; i < 2; ++i) {
        for (int64_t e = 0; e < N; ++e) a[e] = X[e];
        const cplx *blk = P + (((int64_t)c * 5 + q) * 2 + i) * per;
        for (int mu = 0; mu < d; ++mu) {
            cmode_product(d, n, a, mu, blk, b);
            cplx *t = a; a = b; b = t;
            blk += n[mu] * n[mu];
        }
        cplx et = eta[2 * i] + eta[2 * i + 1] * I;
        for (int64_t e = 0; e < N; ++e) acc[e] += w * creal(et * a[e]);
    }
    free(a); free(b);
    return 0;
}

int orc_step_cplx(int d, const int64_t *n, const double *A, const double *Pd, int model,
                  const double *p, double tau, double *U, int nsteps)
{
    const cplx *P = (const cplx *)Pd;
    if (d < 2 || d > ORC_MAXD || nsteps < 0) return -1;
    double eta1[4], eta2[4], al[4];
    orc_coeffs_cplx(d, 1, eta1, al);
    orc_coeffs_cplx(d, 2, eta2, al);
    int64_t N = numel(d, n);
    const double *Ac[2][ORC_MAXD];
    const double *Acur = A;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < d; ++mu) { Ac[c][mu] = Acur; Acur += n[mu] * n[mu]; }
    double *G = malloc(sizeof(double) * 2 * N), *F = malloc(sizeof(double) * 2 * N);
    double *U2 = malloc(sizeof(double) * 2 * N), *U3 = malloc(sizeof(double) * 2 * N);
    double *Dt = malloc(sizeof(double) * 2 * N), *Un = malloc(sizeof(double) * 2 * N);
    int rc = -1;
    if (!G || !F || !U2 || !U3 || !Dt || !Un) goto done;
    for (int step = 0; step < nsteps; ++step) {
        orc_g(model, p, N, U, G);
        for (int c = 0; c < 2; ++c) {
            if (orc_kronsum(d, n, U + c * N, Ac[c], F + c * N) < 0) goto done;
            for (int64_t e = 0; e < N; ++e) F[c * N + e] += G[c * N + e];
        }
        memcpy(U2, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c)
            if (split_action_cplx(d, n, P, c, 0, eta1, tau / 3.0, F + c * N, U2 + c * N) < 0) goto done;
        orc_g(model, p, N, U2, Dt);
        for (int64_t e = 0; e < 2 * N; ++e) Dt[e] -= G[e];
        memcpy(U3, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c) {
            if (split_action_cplx(d, n, P, c, 1, eta1, 2.0 * tau / 3.0, F + c * N, U3 + c * N) < 0) goto done;
            if (split_action_cplx(d, n, P, c, 2, eta2, 4.0 * tau / 3.0, Dt + c * N, U3 + c * N) < 0) goto done;
        }
        orc_g(model, p, N, U3, Dt);
        for (int64_t e = 0; e < 2 * N; ++e) Dt[e] -= G[e];
        memcpy(Un, U, sizeof(double) * 2 * N);
        for (int c = 0; c < 2; ++c) {
            if (split_action_cplx(d, n, P, c, 3, eta1, tau, F + c * N, Un + c * N) < 0) goto done;
            if (split_action_cplx(d, n, P, c, 4, eta2, 1.5 * tau, Dt + c * N, Un + c * N) < 0) goto done;
        }
        memcpy(U, Un, sizeof(double) * 2 * N);
    }
    rc = 0;
done:
    free(G); free(F); free(U2); free(U3); free(Dt); free(Un);
    return rc;
}
