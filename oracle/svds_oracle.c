/*
 * Plain FP64 CPU oracle of restarted Lanczos bidiagonalization with full
 * re-orthogonalization and augmented (thick) restart -- the truncated-SVD
 * method of the svds-C paper (arXiv 2405.18966): Alg. 1 (LBP), the full
 * re-orthogonalization of Sec. 2.1, Proposition 1 / Eq. (2)-(4) (residual
 * test), Eq. (5)-(7) and Alg. 2 (augmented restart).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously-correct checker of
 * the CUDA solver.  Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header or constant with
 * the CUDA path.
 *
 * Style: loops written out in the order the paper states them, FP64
 * throughout, no blocking or fusion beyond a row-blocked loop order that does
 * not change which terms are summed in which order.  Every loop that OpenMP
 * splits computes each output element in one thread in a fixed order, so the
 * results do not depend on the thread count.
 *
 * Readings of points where the paper is silent (each also listed in the design
 * notes): CGS2 (two projection passes) wherever Sec. 2.1 asks for
 * re-orthogonalization; u_{t+1} of LBP(A,t+1) is not formed (nothing uses
 * it); the maximum iteration count counts SVD-and-test rounds and the last
 * round never restarts; a Lanczos vector whose norm falls to 1e-13 * (largest
 * alpha/beta/sigma seen) is a breakdown, its T entry is set to zero and a fresh
 * random vector, orthogonalized against the basis, takes its place; the
 * residual denominator is max(sigma_j, eps*sigma_1).  Two options beyond the
 * paper's default: the k smallest triplets (the same restart keeping the k
 * smallest Ritz triplets, S ascending, m >= n) and partial
 * re-orthogonalization (orthogonality estimates from the Lanczos relations
 * decide which vectors get CGS2, threshold eps^(3/4)).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t kind;            /* 0: CSR 0-based 3-array, 1: dense column-major */
    int32_t pad;
    int64_t m, n;
    const int64_t *row_ptr;  /* CSR: m+1 */
    const int32_t *col_idx;  /* CSR: nnz */
    const double *val;       /* CSR: nnz */
    const double *a;         /* dense: column-major, leading dimension lda */
    int64_t lda;
} orc_mat;

void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- products */

/* y = A x  (Alg. 1). */
void orc_matvec(const orc_mat *A, const double *x, double *y)
{
    if (A->kind == 0) {
        #pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < A->m; r++) {
            double s = 0.0;
            for (int64_t e = A->row_ptr[r]; e < A->row_ptr[r + 1]; e++)
                s += A->val[e] * x[A->col_idx[e]];
            y[r] = s;
        }
    } else {
        /* each y[r] = sum over c = 0..n-1 of a(r,c) x(c), in column order */
        const int64_t blk = 512;
        #pragma omp parallel for schedule(static)
        for (int64_t r0 = 0; r0 < A->m; r0 += blk) {
            int64_t r1 = r0 + blk < A->m ? r0 + blk : A->m;
            for (int64_t r = r0; r < r1; r++) y[r] = 0.0;
            for (int64_t c = 0; c < A->n; c++) {
                const double *col = A->a + c * A->lda;
                double xc = x[c];
                for (int64_t r = r0; r < r1; r++) y[r] += col[r] * xc;
            }
        }
    }
}

/* y = A^T x  (Alg. 1). */
void orc_matvec_t(const orc_mat *A, const double *x, double *y)
{
    if (A->kind == 0) {
        for (int64_t c = 0; c < A->n; c++) y[c] = 0.0;
        for (int64_t r = 0; r < A->m; r++) {
            double xr = x[r];
            for (int64_t e = A->row_ptr[r]; e < A->row_ptr[r + 1]; e++)
                y[A->col_idx[e]] += A->val[e] * xr;
        }
    } else {
        #pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < A->n; c++) {
            const double *col = A->a + c * A->lda;
            double s = 0.0;
            for (int64_t r = 0; r < A->m; r++) s += col[r] * x[r];
            y[c] = s;
        }
    }
}

/* h = W^T w  (W: len x ncols, column-major, leading dimension ldw). */
void orc_gemv_t(int64_t len, int64_t ncols, const double *W, int64_t ldw,
                const double *w, double *h)
{
    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < ncols; c++) {
        const double *col = W + c * ldw;
        double s = 0.0;
        for (int64_t r = 0; r < len; r++) s += col[r] * w[r];
        h[c] = s;
    }
}

/* w = w - W h : each w[r] loses sum over c (in order) of W(r,c) h(c). */
void orc_gemv_n_sub(int64_t len, int64_t ncols, const double *W, int64_t ldw,
                    const double *h, double *w)
{
    const int64_t blk = 512;
    #pragma omp parallel for schedule(static)
    for (int64_t r0 = 0; r0 < len; r0 += blk) {
        double acc[512];
        int64_t r1 = r0 + blk < len ? r0 + blk : len;
        for (int64_t r = r0; r < r1; r++) acc[r - r0] = 0.0;
        for (int64_t c = 0; c < ncols; c++) {
            const double *col = W + c * ldw;
            double hc = h[c];
            for (int64_t r = r0; r < r1; r++) acc[r - r0] += col[r] * hc;
        }
        for (int64_t r = r0; r < r1; r++) w[r] -= acc[r - r0];
    }
}

/* Full re-orthogonalization w <- (I - W W^T) w of Sec. 2.1, applied twice
 * (classical Gram-Schmidt with one re-projection, "CGS2"). */
void orc_cgs2(int64_t len, int64_t ncols, const double *W, int64_t ldw, double *w,
              double *h_scratch)
{
    if (ncols <= 0) return;
    for (int pass = 0; pass < 2; pass++) {
        orc_gemv_t(len, ncols, W, ldw, w, h_scratch);
        orc_gemv_n_sub(len, ncols, W, ldw, h_scratch, w);
    }
}

double orc_norm2(int64_t len, const double *x)
{
    double s = 0.0;
    for (int64_t r = 0; r < len; r++) s += x[r] * x[r];
    return sqrt(s);
}

/* C (rows x kk, ldc) = W (rows x tt, ldw) * Q (tt x kk, ldq): the restart
 * update of Alg. 2 and its final product. */
void orc_gemm_nn(int64_t rows, int64_t tt, int64_t kk, const double *W, int64_t ldw,
                 const double *Q, int64_t ldq, double *C, int64_t ldc)
{
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < rows; r++) {
        for (int64_t j = 0; j < kk; j++) {
            double s = 0.0;
            for (int64_t c = 0; c < tt; c++) s += W[r + c * ldw] * Q[c + j * ldq];
            C[r + j * ldc] = s;
        }
    }
}

/* ------------------------------------------------------------- random draws
 * Counter-based normal generator: SplitMix64 (Steele, Lea & Flood, 2014) as
 * the mixing function, Box-Muller (1958) for the normal deviate.  Element j
 * of random vector number `draw` under `seed`:
 *   key  = mix(seed) ;  c = 2*(draw*2^32 + j)
 *   U1   = ((mix(key + c)     >> 11) + 0.5) * 2^-53
 *   U2   = ((mix(key + c + 1) >> 11) + 0.5) * 2^-53
 *   z    = sqrt(-2 ln U1) * cos(2 pi U2)
 * where mix(x) adds the golden-ratio increment 0x9E3779B97F4A7C15 and applies
 * the SplitMix64 finaliser. */
static uint64_t orc_mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t x) { return orc_mix64(x); }

double orc_rng_normal(uint64_t seed, uint64_t draw, uint64_t j)
{
    uint64_t key = orc_mix64(seed);
    uint64_t c = 2ULL * ((draw << 32) + j);
    double u1 = ((double)(orc_mix64(key + c) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = ((double)(orc_mix64(key + c + 1ULL) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

void orc_rng_vector(uint64_t seed, uint64_t draw, int64_t len, double *x)
{
    for (int64_t j = 0; j < len; j++) x[j] = orc_rng_normal(seed, draw, (uint64_t)j);
}

/* --------------------------------------------------------- dense Jacobi SVD
 * One-sided (Hestenes) Jacobi SVD of an m x n matrix, m >= n: columns of
 * B = A V are rotated pairwise until mutually orthogonal; then sigma_j is the
 * norm of column j of B, u_j = B(:,j)/sigma_j and v_j the accumulated
 * rotation.  Output sorted by descending sigma (stable in the column index).
 * U is m x n (thin), V is n x n.  Returns the number of sweeps used, or -1 if
 * max_sweeps was reached. */
int orc_jacobi_svd(int64_t m, int64_t n, const double *A, int64_t lda,
                   double *S, double *U, int64_t ldu, double *V, int64_t ldv,
                   int max_sweeps)
{
    double *B = (double *)malloc(sizeof(double) * (size_t)(m * n));
    double *W = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *sig = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t c = 0; c < n; c++)
        for (int64_t r = 0; r < m; r++) B[r + c * m] = A[r + c * lda];
    for (int64_t c = 0; c < n; c++)
        for (int64_t r = 0; r < n; r++) W[r + c * n] = (r == c) ? 1.0 : 0.0;

    const double tol = DBL_EPSILON * sqrt((double)m);
    int sweeps = 0, converged = 0;
    while (!converged && sweeps < max_sweeps) {
        converged = 1;
        sweeps++;
        for (int64_t p = 0; p < n - 1; p++) {
            for (int64_t q = p + 1; q < n; q++) {
                double *bp = B + p * m, *bq = B + q * m;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t r = 0; r < m; r++) {
                    alpha += bp[r] * bp[r];
                    beta += bq[r] * bq[r];
                    gamma += bp[r] * bq[r];
                }
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
                converged = 0;
                /* rotation that zeroes the (p,q) entry of B^T B */
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (int64_t r = 0; r < m; r++) {
                    double x = bp[r], y = bq[r];
                    bp[r] = c * x - s * y;
                    bq[r] = s * x + c * y;
                }
                double *wp = W + p * n, *wq = W + q * n;
                for (int64_t r = 0; r < n; r++) {
                    double x = wp[r], y = wq[r];
                    wp[r] = c * x - s * y;
                    wq[r] = s * x + c * y;
                }
            }
        }
    }
    for (int64_t c = 0; c < n; c++) {
        double s = 0.0;
        for (int64_t r = 0; r < m; r++) s += B[r + c * m] * B[r + c * m];
        sig[c] = sqrt(s);
        perm[c] = c;
    }
    /* stable insertion sort by descending sigma */
    for (int64_t i = 1; i < n; i++) {
        int64_t pi = perm[i];
        int64_t j = i - 1;
        while (j >= 0 && sig[perm[j]] < sig[pi]) { perm[j + 1] = perm[j]; j--; }
        perm[j + 1] = pi;
    }
    for (int64_t j = 0; j < n; j++) {
        int64_t src = perm[j];
        S[j] = sig[src];
        for (int64_t r = 0; r < n; r++) V[r + j * ldv] = W[r + src * n];
        if (sig[src] > 0.0) {
            for (int64_t r = 0; r < m; r++) U[r + j * ldu] = B[r + src * m] / sig[src];
        } else {
            for (int64_t r = 0; r < m; r++) U[r + j * ldu] = 0.0;
        }
    }
    /* columns with sigma == 0: complete U to an orthonormal set with the
     * first unit vectors that survive two Gram-Schmidt passes */
    int64_t next_e = 0;
    for (int64_t j = 0; j < n; j++) {
        if (S[j] > 0.0) continue;
        while (next_e < m) {
            double *u = U + j * ldu;
            for (int64_t r = 0; r < m; r++) u[r] = (r == next_e) ? 1.0 : 0.0;
            next_e++;
            for (int pass = 0; pass < 2; pass++) {
                for (int64_t i = 0; i < n; i++) {
                    if (i == j || (S[i] == 0.0 && i > j)) continue;
                    const double *ui = U + i * ldu;
                    double d = 0.0;
                    for (int64_t r = 0; r < m; r++) d += ui[r] * u[r];
                    for (int64_t r = 0; r < m; r++) u[r] -= d * ui[r];
                }
            }
            double nu = orc_norm2(m, u);
            if (nu > 0.5) {
                for (int64_t r = 0; r < m; r++) u[r] /= nu;
                break;
            }
        }
    }
    free(B); free(W); free(sig); free(perm);
    return converged ? sweeps : -1;
}

/* ------------------------------------------------------------ Alg. 1 and 2 */

typedef struct {
    int32_t converged;      /* 1 if every res_j < tol */
    int32_t nconv;          /* number of j <= k with res_j < tol */
    int32_t restarts;       /* augmented restarts performed */
    int32_t breakdowns;     /* Lanczos vectors replaced by random ones */
    int64_t n_matvec;       /* products with A or A^T */
    int64_t n_steps;        /* Lanczos vectors formed (u and v each count 1) */
    int32_t svd_sweeps_max; /* most Jacobi sweeps taken by a small SVD */
    int32_t stopped_early;  /* 1 if the step budget ran out */
    double anorm_est;       /* largest alpha, beta or sigma seen */
    double beta_t;          /* T(t,t+1) at exit */
    int64_t n_reorth;       /* Lanczos vectors re-orthogonalized (CGS2) */
} orc_info;

typedef struct {
    const orc_mat *A;
    int64_t m, n, t;
    double *U, *V, *T;      /* U: m x t, V: n x (t+1), T: (t+1) x (t+1), column-major */
    double *h, *wm, *wn;    /* scratch */
    uint64_t seed;
    uint64_t draws;         /* random vectors drawn so far */
    double anorm;
    int64_t step_budget;    /* <0: unlimited */
    orc_info *info;
    /* partial re-orthogonalization (reorth = 1): mu[l] estimates u_i^T u_l for
       the newest u_i, nu[l] estimates v_j^T v_l for the newest v_j */
    int reorth;
    double *mu, *nu;
    int force_u, force_v;
} orc_lanczos;

#define T_(L, i, j) ((L)->T[(i) + (j) * ((L)->t + 1)])

static int orc_budget_hit(orc_lanczos *L)
{
    if (L->step_budget >= 0 && L->info->n_steps >= L->step_budget) {
        L->info->stopped_early = 1;
        return 1;
    }
    return 0;
}

/* Normalise w (after it was orthogonalized against the first `ncols` columns
 * of W) and store it as column `ncols`; a breakdown draws a random vector. */
static double orc_finish_vector(orc_lanczos *L, double *w, int64_t len, double *W,
                                int64_t ncols)
{
    double nrm = orc_norm2(len, w);
    double thresh = 1e-13 * L->anorm;
    if (!(nrm > thresh) || !isfinite(nrm)) {
        /* breakdown: the Krylov space is (numerically) invariant */
        L->info->breakdowns++;
        double beta_or_alpha = 0.0;
        for (int attempt = 0; attempt < 8; attempt++) {
            orc_rng_vector(L->seed, L->draws++, len, w);
            orc_cgs2(len, ncols, W, len, w, L->h);
            double nr = orc_norm2(len, w);
            if (nr > 1e-8) {
                for (int64_t r = 0; r < len; r++) W[r + ncols * len] = w[r] / nr;
                return beta_or_alpha;
            }
        }
        for (int64_t r = 0; r < len; r++) W[r + ncols * len] = 0.0;
        return 0.0;
    }
    if (nrm > L->anorm) L->anorm = nrm;
    for (int64_t r = 0; r < len; r++) W[r + ncols * len] = w[r] / nrm;
    return nrm;
}

/* ------------------------------------------- partial re-orthogonalization
 *
 * Opt-in alternative to re-orthogonalizing every vector (the scheme of
 * lansvd, Table 1).  The Lanczos relations A v_l = sum_r T(r,l) u_r and
 * A^T u_l = sum_r T(l,r) v_r (both also hold after an augmented restart, where
 * T carries the spike column of Eq. 6-7) turn into recurrences for the inner
 * products of the newest vector with the earlier ones:
 *   beta_i (v_{i+1}^T v_l) = u_i^T A v_l - alpha_i v_i^T v_l
 *                          = sum_r T(r,l) (u_i^T u_r) - alpha_i (v_i^T v_l)
 *   alpha_{i+1} (u_{i+1}^T u_l) = v_{i+1}^T A^T u_l - beta_i u_i^T u_l
 *                          = sum_r T(l,r) (v_{i+1}^T v_r) - beta_i (u_i^T u_l)
 * Each estimate also grows by a rounding term eps ||A|| / (divisor), signed
 * like the estimate.  A vector is re-orthogonalized (CGS2 against all earlier
 * ones) when its largest estimate exceeds eps^(3/4), and so is the next
 * vector of the same kind; the estimates of a re-orthogonalized vector are
 * reset to eps.  beta_i / alpha_{i+1} here are the norms before any
 * re-orthogonalization.  The level eps^(3/4) (not the sqrt(eps) that
 * suffices for accurate singular values) keeps the components CGS2 removes,
 * which the bidiagonal T does not record, small enough that the true
 * residuals A v - sigma u stay at ~1e-12 ||A|| instead of ~sqrt(eps) ||A||.
 */
#define ORC_PR_EPS DBL_EPSILON
#define ORC_PR_DELTA 1.8189894035458565e-12  /* DBL_EPSILON^(3/4) = 2^-39 */

/* nu <- estimates of v_{i+1}^T v_l, l = 1..i (i 1-based); returns 1 when
 * v_{i+1} must be re-orthogonalized. */
/* One step of each recurrence on plain arrays (T column-major, leading
 * dimension ldt; mu, nu of length >= i + 2; anorm the ||A|| estimate).
 * Returns the largest new estimate, or -1 when the norm is unusable. */
double orc_pr_nu_step(int64_t i, const double *T, int64_t ldt, const double *mu, double *nu,
                      double beta, double anorm)
{
    if (!(beta > 0.0) || !isfinite(beta)) return -1.0;
    const double tau = ORC_PR_EPS * anorm / beta;
    const double alpha_i = T[(i - 1) + (i - 1) * ldt];
    double mx = 0.0;
    for (int64_t l = 1; l <= i; l++) {
        double s = 0.0;
        for (int64_t r = 1; r <= l; r++) s += T[(r - 1) + (l - 1) * ldt] * mu[r - 1];
        double x = (s - alpha_i * nu[l - 1]) / beta;
        x += (x >= 0.0) ? tau : -tau;
        nu[l - 1] = x;
        if (fabs(x) > mx) mx = fabs(x);
    }
    nu[i] = 1.0;
    return mx;
}

/* mu <- estimates of u_{i+1}^T u_l, l = 1..i, from nu (v_{i+1}^T v_r,
 * r = 1..i+1) and the previous mu (u_i^T u_l). */
double orc_pr_mu_step(int64_t i, const double *T, int64_t ldt, double *mu, const double *nu,
                      double alpha, double anorm)
{
    if (!(alpha > 0.0) || !isfinite(alpha)) return -1.0;
    const double tau = ORC_PR_EPS * anorm / alpha;
    const double beta_i = T[(i - 1) + i * ldt];
    double mx = 0.0;
    for (int64_t l = 1; l <= i; l++) {
        double s = 0.0;
        for (int64_t r = l; r <= i + 1; r++) s += T[(l - 1) + (r - 1) * ldt] * nu[r - 1];
        double x = (s - beta_i * mu[l - 1]) / alpha;
        x += (x >= 0.0) ? tau : -tau;
        mu[l - 1] = x;
        if (fabs(x) > mx) mx = fabs(x);
    }
    mu[i] = 1.0;
    return mx;
}

/* nu <- estimates of v_{i+1}^T v_l, l = 1..i (i 1-based); returns 1 when
 * v_{i+1} must be re-orthogonalized. */
static int orc_pr_nu(orc_lanczos *L, int64_t i, double beta)
{
    const double mx = orc_pr_nu_step(i, L->T, L->t + 1, L->mu, L->nu, beta, L->anorm);
    return (mx < 0.0) || (mx > ORC_PR_DELTA) || L->force_v;
}

/* mu <- estimates of u_{i+1}^T u_l; returns 1 when u_{i+1} must be
 * re-orthogonalized. */
static int orc_pr_mu(orc_lanczos *L, int64_t i, double alpha)
{
    const double mx = orc_pr_mu_step(i, L->T, L->t + 1, L->mu, L->nu, alpha, L->anorm);
    return (mx < 0.0) || (mx > ORC_PR_DELTA) || L->force_u;
}

/* Re-orthogonalizes w against the first `ncols` columns of W when `need`,
 * keeping the estimates and the force flag of its kind. */
static void orc_pr_apply(orc_lanczos *L, int need, int64_t len, int64_t ncols, const double *W,
                         double *w, double *est, int *force)
{
    if (need) {
        orc_cgs2(len, ncols, W, len, w, L->h);
        L->info->n_reorth++;
        for (int64_t l = 0; l < ncols; l++) est[l] = ORC_PR_EPS;
        *force = !*force;   /* a triggered re-orthogonalization also forces the next one */
    }
}

/* Alg. 1 loop body for i = s..t (1-based): given u_1..u_s, v_1..v_s and
 * alpha_s = T(s,s), form v_{s+1}, u_{s+1}, ..., v_{t+1}. */
static void orc_lbp_from(orc_lanczos *L, int64_t s)
{
    const int64_t m = L->m, n = L->n, t = L->t;
    for (int64_t i = s; i <= L->t; i++) {
        /* v_{i+1} = A^T u_i - alpha_i v_i ; re-orthogonalize against V^(i) */
        if (orc_budget_hit(L)) return;
        double alpha_i = T_(L, i - 1, i - 1);
        orc_matvec_t(L->A, L->U + (i - 1) * m, L->wn);
        L->info->n_matvec++;
        for (int64_t r = 0; r < n; r++) L->wn[r] -= alpha_i * L->V[r + (i - 1) * n];
        if (L->reorth) {
            const int need = orc_pr_nu(L, i, orc_norm2(n, L->wn));
            orc_pr_apply(L, need, n, i, L->V, L->wn, L->nu, &L->force_v);
        } else {
            orc_cgs2(n, i, L->V, n, L->wn, L->h);
            L->info->n_reorth++;
        }
        const int32_t bdv = L->info->breakdowns;
        double beta_i = orc_finish_vector(L, L->wn, n, L->V, i);
        if (L->reorth && L->info->breakdowns != bdv)  /* a fresh orthogonalized vector */
            for (int64_t l = 0; l < i; l++) L->nu[l] = ORC_PR_EPS;
        T_(L, i - 1, i) = beta_i;
        L->info->n_steps++;
        if (i == t) break;  /* u_{t+1} is never used */
        /* u_{i+1} = A v_{i+1} - beta_i u_i ; re-orthogonalize against U^(i) */
        if (orc_budget_hit(L)) return;
        orc_matvec(L->A, L->V + i * n, L->wm);
        L->info->n_matvec++;
        for (int64_t r = 0; r < m; r++) L->wm[r] -= beta_i * L->U[r + (i - 1) * m];
        if (L->reorth) {
            const int need = orc_pr_mu(L, i, orc_norm2(m, L->wm));
            orc_pr_apply(L, need, m, i, L->U, L->wm, L->mu, &L->force_u);
        } else {
            orc_cgs2(m, i, L->U, m, L->wm, L->h);
            L->info->n_reorth++;
        }
        const int32_t bdu = L->info->breakdowns;
        double alpha_next = orc_finish_vector(L, L->wm, m, L->U, i);
        if (L->reorth && L->info->breakdowns != bdu)
            for (int64_t l = 0; l < i; l++) L->mu[l] = ORC_PR_EPS;
        T_(L, i, i) = alpha_next;
        L->info->n_steps++;
    }
}

/* Sign rule for returned pairs: flip (u_j, v_j) so that the entry of v_j of
 * largest magnitude (lowest index on ties) is positive. */
void orc_sign_normalize(int64_t m, int64_t n, int64_t k, double *U, int64_t ldu,
                        double *V, int64_t ldv)
{
    for (int64_t j = 0; j < k; j++) {
        double *v = V + j * ldv;
        int64_t best = 0;
        for (int64_t r = 1; r < n; r++)
            if (fabs(v[r]) > fabs(v[best])) best = r;
        if (v[best] < 0.0) {
            for (int64_t r = 0; r < n; r++) v[r] = -v[r];
            double *u = U + j * ldu;
            for (int64_t r = 0; r < m; r++) u[r] = -u[r];
        }
    }
}

/*
 * Alg. 2: k largest singular triplets of A (which = 0), or the k smallest
 * (which = 1: the Ritz values of the projected matrix approximate both ends
 * of the spectrum, Sec. 2; the same restart keeps the k smallest Ritz
 * triplets instead of the k largest; needs m >= n so that the n singular
 * values of A are those of A^T A).
 *   t = k + p (p < 0: t = max(15, 3k) as in Alg. 2); requires
 *   1 <= k <= t, t + 1 <= min(m, n) ... t <= m and t + 1 <= n.
 *   maxit: number of small-SVD-and-residual-test rounds (>= 1).
 *   reorth: 0 re-orthogonalizes every Lanczos vector (CGS2, Sec. 2.1); 1 only
 *   where the partial re-orthogonalization estimates ask for it (see above).
 *   v0: start vector (length n) or NULL for the seeded random draw 0.
 *   Outputs: S (k), U (m x k, ldu), V (n x k, ldv), res (k).
 *   Optional (may be NULL): Ubasis (m x t), Vbasis (n x (t+1)),
 *   Tout ((t+1) x (t+1)) hold the final Lanczos basis and projected matrix;
 *   mu_out, nu_out (t+2 each) the last partial re-orthogonalization estimates
 *   (newest u against the earlier u's, newest v against the earlier v's).
 * Returns 0 on success (converged or not: see info), -1 on bad arguments,
 * -4 if memory ran out.
 */
int orc_svds(const orc_mat *A, int64_t k, int64_t p, double tol, int64_t maxit, int64_t which,
             int64_t reorth, uint64_t seed, const double *v0, int64_t step_budget,
             double *S, double *Uout, int64_t ldu, double *Vout, int64_t ldv,
             double *res, orc_info *info, double *Ubasis, double *Vbasis, double *Tout,
             double *mu_out, double *nu_out)
{
    memset(info, 0, sizeof(*info));
    const int64_t m = A->m, n = A->n;
    int64_t t = (p < 0) ? (3 * k > 15 ? 3 * k : 15) : k + p;
    if (k < 1 || t < k || t > m || t + 1 > n || !(tol > 0.0) || maxit < 1) return -1;
    if (which != 0 && (which != 1 || m < n)) return -1;
    if (reorth != 0 && reorth != 1) return -1;

    orc_lanczos L;
    memset(&L, 0, sizeof(L));
    L.A = A; L.m = m; L.n = n; L.t = t; L.seed = seed; L.info = info;
    L.step_budget = step_budget;
    L.reorth = (int)reorth;
    L.U = (double *)calloc((size_t)(m * t), sizeof(double));
    L.V = (double *)calloc((size_t)(n * (t + 1)), sizeof(double));
    L.T = (double *)calloc((size_t)((t + 1) * (t + 1)), sizeof(double));
    L.h = (double *)calloc((size_t)(t + 2), sizeof(double));
    L.wm = (double *)calloc((size_t)m, sizeof(double));
    L.wn = (double *)calloc((size_t)n, sizeof(double));
    L.mu = (double *)calloc((size_t)(t + 2), sizeof(double));
    L.nu = (double *)calloc((size_t)(t + 2), sizeof(double));
    double *Uh = (double *)calloc((size_t)(t * t), sizeof(double));
    double *Vh = (double *)calloc((size_t)(t * t), sizeof(double));
    double *Sh = (double *)calloc((size_t)t, sizeof(double));
    double *Tt = (double *)calloc((size_t)(t * t), sizeof(double));
    double *Uk = (double *)calloc((size_t)(m * k), sizeof(double));
    double *Vk = (double *)calloc((size_t)(n * k), sizeof(double));
    double *rho = (double *)calloc((size_t)k, sizeof(double));
    if (!L.U || !L.V || !L.T || !L.h || !L.wm || !L.wn || !L.mu || !L.nu || !Uh || !Vh || !Sh ||
        !Tt || !Uk || !Vk || !rho) {
        free(L.U); free(L.V); free(L.T); free(L.h); free(L.wm); free(L.wn); free(L.mu); free(L.nu);
        free(Uh); free(Vh); free(Sh); free(Tt); free(Uk); free(Vk); free(rho);
        return -4;
    }

    /* Alg. 1, start: v_1 = randn(n), normalised (or the caller's v0) */
    if (v0) memcpy(L.wn, v0, sizeof(double) * (size_t)n);
    else orc_rng_vector(seed, L.draws++, n, L.wn);
    if (v0) L.draws++;  /* draw 0 is reserved for the start vector either way */
    {
        double nv = orc_norm2(n, L.wn);
        if (!(nv > 0.0) || !isfinite(nv)) {  /* unusable v0: fall back to a draw */
            orc_rng_vector(seed, L.draws++, n, L.wn);
            nv = orc_norm2(n, L.wn);
        }
        for (int64_t r = 0; r < n; r++) L.V[r] = L.wn[r] / nv;
    }
    /* u_1 = A v_1, alpha_1 = ||u_1||, u_1 /= alpha_1 */
    orc_matvec(A, L.V, L.wm);
    info->n_matvec++;
    T_(&L, 0, 0) = orc_finish_vector(&L, L.wm, m, L.U, 0);
    info->n_steps++;
    L.nu[0] = 1.0;   /* v_1^T v_1 */
    L.mu[0] = 1.0;   /* u_1^T u_1 */
    /* Alg. 2: LBP(A, t+1) */
    orc_lbp_from(&L, 1);

    int64_t it;
    for (it = 1; it <= maxit; it++) {
        if (info->stopped_early) break;
        /* Alg. 2: SVD of T(1:t,1:t) */
        for (int64_t c = 0; c < t; c++)
            for (int64_t r = 0; r < t; r++) Tt[r + c * t] = T_(&L, r, c);
        int sw = orc_jacobi_svd(t, t, Tt, t, Sh, Uh, t, Vh, t, 200);
        if (sw > info->svd_sweeps_max) info->svd_sweeps_max = sw;
        const double smax = Sh[0];    /* descending order from the Jacobi SVD */
        if (smax > L.anorm) L.anorm = smax;
        if (which == 1) {
            /* smallest: reverse the order of the Ritz triplets so the wanted
               k (ascending) are the first k columns used below */
            for (int64_t j = 0; j < t / 2; j++) {
                const int64_t jj = t - 1 - j;
                double x = Sh[j]; Sh[j] = Sh[jj]; Sh[jj] = x;
                for (int64_t r = 0; r < t; r++) {
                    x = Uh[r + j * t]; Uh[r + j * t] = Uh[r + jj * t]; Uh[r + jj * t] = x;
                    x = Vh[r + j * t]; Vh[r + j * t] = Vh[r + jj * t]; Vh[r + jj * t] = x;
                }
            }
        }
        /* Eq. (4): res_j = |beta_t Uh(t,j)| / sigma_j */
        double beta_t = T_(&L, t - 1, t);
        info->beta_t = beta_t;
        int64_t nconv = 0;
        for (int64_t j = 0; j < k; j++) {
            double den = Sh[j] > DBL_EPSILON * smax ? Sh[j] : DBL_EPSILON * smax;
            double rj = (den > 0.0) ? fabs(beta_t * Uh[(t - 1) + j * t]) / den : 0.0;
            res[j] = rj;
            if (rj < tol) nconv++;
        }
        info->nconv = (int32_t)nconv;
        info->converged = (nconv == k);
        if (info->converged || it == maxit) break;

        /* augmented restart (Eq. 5-7) */
        orc_gemm_nn(m, t, k, L.U, m, Uh, t, Uk, m);          /* U~_k = U(:,1:t) Uh(:,1:k) */
        orc_gemm_nn(n, t, k, L.V, n, Vh, t, Vk, n);          /* V~_k = V(:,1:t) Vh(:,1:k) */
        if (L.reorth) {
            /* v_{k+1} = v_{t+1} against V~_k: |v~_j^T v_{t+1}| <= sum_l |Vh(l,j)| |nu_l| */
            for (int64_t j = 0; j < k; j++) {
                double acc = 0.0;
                for (int64_t l = 0; l < t; l++) acc += fabs(Vh[l + j * t]) * fabs(L.nu[l]);
                L.h[j] = acc + ORC_PR_EPS;
            }
            for (int64_t j = 0; j < k; j++) L.nu[j] = L.h[j];
            L.nu[k] = 1.0;
            L.force_u = L.force_v = 0;
        }
        for (int64_t j = 0; j < k; j++) rho[j] = beta_t * Uh[(t - 1) + j * t];
        memset(L.T, 0, sizeof(double) * (size_t)((t + 1) * (t + 1)));
        for (int64_t j = 0; j < k; j++) {
            T_(&L, j, j) = Sh[j];
            T_(&L, j, k) = rho[j];
        }
        /* v_{k+1} = v_{t+1} */
        memcpy(L.V + k * n, L.V + t * n, sizeof(double) * (size_t)n);
        memcpy(L.V, Vk, sizeof(double) * (size_t)(n * k));
        memcpy(L.U, Uk, sizeof(double) * (size_t)(m * k));
        /* u_{k+1} = A v_{k+1} - U~_k rho  (Eq. 7), re-orthogonalized against U~_k */
        if (orc_budget_hit(&L)) break;
        orc_matvec(A, L.V + k * n, L.wm);
        info->n_matvec++;
        orc_gemv_n_sub(m, k, L.U, m, rho, L.wm);
        orc_cgs2(m, k, L.U, m, L.wm, L.h);
        info->n_reorth++;
        T_(&L, k, k) = orc_finish_vector(&L, L.wm, m, L.U, k);
        for (int64_t j = 0; j < k; j++) L.mu[j] = ORC_PR_EPS;
        L.mu[k] = 1.0;
        info->n_steps++;
        info->restarts++;
        /* continue Alg. 1 from i = k+1 */
        orc_lbp_from(&L, k + 1);
    }
    if (!info->stopped_early) {
        /* outputs: S, U~ = U(:,1:t) Uh(:,1:k), V~ = V(:,1:t) Vh(:,1:k) */
        for (int64_t j = 0; j < k; j++) S[j] = Sh[j];
        orc_gemm_nn(m, t, k, L.U, m, Uh, t, Uout, ldu);
        orc_gemm_nn(n, t, k, L.V, n, Vh, t, Vout, ldv);
        orc_sign_normalize(m, n, k, Uout, ldu, Vout, ldv);
    }
    info->anorm_est = L.anorm;
    if (Ubasis) memcpy(Ubasis, L.U, sizeof(double) * (size_t)(m * t));
    if (Vbasis) memcpy(Vbasis, L.V, sizeof(double) * (size_t)(n * (t + 1)));
    if (Tout) memcpy(Tout, L.T, sizeof(double) * (size_t)((t + 1) * (t + 1)));
    if (mu_out) memcpy(mu_out, L.mu, sizeof(double) * (size_t)(t + 2));
    if (nu_out) memcpy(nu_out, L.nu, sizeof(double) * (size_t)(t + 2));

    free(L.U); free(L.V); free(L.T); free(L.h); free(L.wm); free(L.wn); free(L.mu); free(L.nu);
    free(Uh); free(Vh); free(Sh); free(Tt); free(Uk); free(Vk); free(rho);
    return 0;
}

/* ================================================================ block form
 *
 * Block Lanczos bidiagonalization (Golub, Luk & Overton 1981) with the full
 * re-orthogonalization of Sec. 2.1 and the augmented restart of Alg. 2,
 * carried over from single vectors to blocks of b columns.  With b = 1 every
 * step below is the single-vector step of orc_svds, in the same order.
 *
 * Blocks (column offsets c are multiples of b before the first restart and
 * k + multiples of b after it):
 *   V(:, 0:b)  = orthonormalized start block
 *   U(:, 0:b) R = A V(:, 0:b)                          R -> T(0:b, 0:b)
 *   repeat, with c = columns of U and V formed so far:
 *     Z = A^T U(:, c-b:c) - V(:, c-b:c) T(c-b:c, c-b:c)^T
 *     Z -> V(:, c:c+b) S      (S upper triangular)      S^T -> T(c-b:c, c:c+b)
 *     stop here when c = t (V(:, t:t+b) is the residual block)
 *     W = A V(:, c:c+b) - U(:, c-b:c) T(c-b:c, c:c+b)
 *     W -> U(:, c:c+b) R                               R -> T(c:c+b, c:c+b)
 * so that A V(:, 0:t) = U(:, 0:t) T(0:t, 0:t) and
 * A^T U(:, 0:t) = V(:, 0:t) T(0:t, 0:t)^T + V(:, t:t+b) F^T E^T, with
 * F = T(t-b:t, t:t+b) and E the last b columns of the identity: T is upper
 * triangular with bandwidth b.  Each "->" is: both CGS passes of every column
 * against the earlier blocks (coefficients discarded: they vanish in exact
 * arithmetic), then a QR of the block column by column, each column
 * projected twice against the block's earlier columns (coefficients summed
 * into the triangular factor) and normalised.  A column whose norm falls to
 * 1e-13 * (largest norm or sigma seen) has a zero diagonal entry and is
 * replaced by a random vector orthogonalized (CGS2) against every earlier
 * column of its basis, as a broken-down single vector is.
 *
 * Ritz triplets of T(0:t, 0:t) = Uh diag(sigma) Vh^T: the residual of Eq. (4)
 * becomes res_j = || F^T Uh(t-b:t, j) ||_2 / sigma_j.  Augmented restart
 * (Eq. 5-7 with a block): rho = Uh(t-b:t, 0:k)^T F (k x b);
 * T <- [diag(sigma_1..k), rho; 0, R'] where U(:, k:k+b) R' comes from
 * W = A V(:, k:k+b) - U~_k rho after V(:, k:k+b) := V(:, t:t+b).
 * Subspace sizes: t0 = b * ceil(t / b) columns in the first pass and
 * t1 = k + b * ceil((t - k) / b) after each restart (t = k + p); both equal
 * t when b = 1.  Draws 0..b-1 are the start block's columns.
 */
typedef struct {
    const orc_mat *A;
    int64_t m, n, b, ld_t;  /* ld_t: leading dimension of T */
    double *U, *V, *T;      /* U: m x tmax, V: n x (tmax + b), T: ld_t x ld_t */
    double *h, *wm, *wn;    /* scratch: h (ld_t), wm (m x b), wn (n x b) */
    uint64_t seed, draws;
    double anorm;
    orc_info *info;
} orc_block;

#define TB_(L, i, j) ((L)->T[(i) + (j) * (L)->ld_t])

/* Orthonormalizes the len x b block Wb into columns c..c+b-1 of Basis (ld
 * len): CGS2 of each column against Basis(:, 0:c), then the column-by-column
 * QR; the triangular factor goes to R (b x b, leading dimension ldr). */
static void orc_block_orth(orc_block *L, double *Wb, int64_t len, double *Basis, int64_t c,
                           double *R, int64_t ldr)
{
    const int64_t b = L->b;
    for (int64_t l = 0; l < b && c > 0; l++) {
        double *w = Wb + l * len;
        orc_cgs2(len, c, Basis, len, w, L->h);            /* against the earlier blocks */
        L->info->n_reorth++;
    }
    for (int64_t l = 0; l < b; l++) {
        double *w = Wb + l * len;
        double *Q = Basis + c * len;                      /* the block's finished columns */
        for (int64_t i = 0; i < b; i++) R[i + l * ldr] = 0.0;
        for (int pass = 0; pass < 2; pass++) {
            if (l == 0) break;
            orc_gemv_t(len, l, Q, len, w, L->h);
            orc_gemv_n_sub(len, l, Q, len, L->h, w);
            for (int64_t i = 0; i < l; i++) R[i + l * ldr] += L->h[i];
        }
        double nrm = orc_norm2(len, w);
        if (!(nrm > 1e-13 * L->anorm) || !isfinite(nrm)) {
            L->info->breakdowns++;
            R[l + l * ldr] = 0.0;
            double *dst = Basis + (c + l) * len;
            int ok = 0;
            for (int attempt = 0; attempt < 8 && !ok; attempt++) {
                orc_rng_vector(L->seed, L->draws++, len, w);
                orc_cgs2(len, c + l, Basis, len, w, L->h);
                double nr = orc_norm2(len, w);
                if (nr > 1e-8) {
                    for (int64_t r = 0; r < len; r++) dst[r] = w[r] / nr;
                    ok = 1;
                }
            }
            if (!ok)
                for (int64_t r = 0; r < len; r++) dst[r] = 0.0;
            continue;
        }
        if (nrm > L->anorm) L->anorm = nrm;
        R[l + l * ldr] = nrm;
        for (int64_t r = 0; r < len; r++) Basis[r + (c + l) * len] = w[r] / nrm;
    }
}

/* Block Lanczos steps from c columns (c >= b; U and V hold c columns, the
 * last U block's R in T) until V holds tc + b columns. */
static void orc_block_lbp_from(orc_block *L, int64_t c, int64_t tc)
{
    const int64_t m = L->m, n = L->n, b = L->b;
    for (;;) {
        /* Z = A^T U(:, c-b:c) - V(:, c-b:c) T(c-b:c, c-b:c)^T */
        for (int64_t l = 0; l < b; l++) {
            double *z = L->wn + l * n;
            orc_matvec_t(L->A, L->U + (c - b + l) * m, z);
            L->info->n_matvec++;
            /* column l of T(c-b:c, c-b:c)^T is row l of the block: T(c-b+l, c-b+i) */
            for (int64_t i = 0; i < b; i++) {
                const double coef = TB_(L, c - b + l, c - b + i);
                if (coef == 0.0) continue;
                const double *v = L->V + (c - b + i) * n;
                for (int64_t r = 0; r < n; r++) z[r] -= coef * v[r];
            }
        }
        double *S = L->h + L->ld_t;  /* b x b scratch after h */
        orc_block_orth(L, L->wn, n, L->V, c, S, b);
        for (int64_t i = 0; i < b; i++)           /* T(c-b:c, c:c+b) = S^T */
            for (int64_t l = 0; l < b; l++) TB_(L, c - b + i, c + l) = S[l + i * b];
        L->info->n_steps += b;
        if (c >= tc) break;
        /* W = A V(:, c:c+b) - U(:, c-b:c) T(c-b:c, c:c+b) */
        for (int64_t l = 0; l < b; l++) {
            double *w = L->wm + l * m;
            orc_matvec(L->A, L->V + (c + l) * n, w);
            L->info->n_matvec++;
            for (int64_t i = 0; i < b; i++) {
                const double coef = TB_(L, c - b + i, c + l);
                if (coef == 0.0) continue;
                const double *u = L->U + (c - b + i) * m;
                for (int64_t r = 0; r < m; r++) w[r] -= coef * u[r];
            }
        }
        orc_block_orth(L, L->wm, m, L->U, c, S, b);
        for (int64_t l = 0; l < b; l++)
            for (int64_t i = 0; i < b; i++) TB_(L, c + i, c + l) = S[i + l * b];
        L->info->n_steps += b;
        c += b;
    }
}

/*
 * Block form of Alg. 2 (k largest triplets, full re-orthogonalization).
 *   b >= 1 block size; t = k + p (p < 0: max(15, 3k) - k); subspace sizes
 *   t0 = b ceil(t / b) (first pass) and t1 = k + b ceil((t - k) / b) (after
 *   each restart); needs 1 <= k, k + b <= t1, max(t0, t1) <= m and
 *   max(t0, t1) + b <= n.
 *   V0: n x b start block (column-major) or NULL for draws 0..b-1.
 *   Outputs as orc_svds; Ubasis (m x tmax), Vbasis (n x (tmax + b)) and
 *   Tout ((tmax + b) x (tmax + b)) hold the final basis and projected
 *   matrix (tmax = max(t0, t1)); *t_last receives the size of the last
 *   projected matrix.
 * Returns 0 on success, -1 on bad arguments, -4 if memory ran out.
 */
int orc_svds_block(const orc_mat *A, int64_t k, int64_t p, int64_t b, double tol, int64_t maxit,
                   uint64_t seed, const double *V0, double *S, double *Uout, int64_t ldu,
                   double *Vout, int64_t ldv, double *res, orc_info *info, double *Ubasis,
                   double *Vbasis, double *Tout, int64_t *t_last)
{
    memset(info, 0, sizeof(*info));
    const int64_t m = A->m, n = A->n;
    const int64_t t = (p < 0) ? (3 * k > 15 ? 3 * k : 15) : k + p;
    if (b < 1 || k < 1 || t < k || !(tol > 0.0) || maxit < 1) return -1;
    const int64_t t0 = b * ((t + b - 1) / b);
    const int64_t t1 = k + b * ((t - k + b - 1) / b);
    const int64_t tmax = t0 > t1 ? t0 : t1;
    if (k + b > t1 || tmax > m || tmax + b > n) return -1;

    orc_block L;
    memset(&L, 0, sizeof(L));
    L.A = A; L.m = m; L.n = n; L.b = b; L.ld_t = tmax + b; L.seed = seed; L.info = info;
    L.U = (double *)calloc((size_t)(m * tmax), sizeof(double));
    L.V = (double *)calloc((size_t)(n * (tmax + b)), sizeof(double));
    L.T = (double *)calloc((size_t)(L.ld_t * L.ld_t), sizeof(double));
    L.h = (double *)calloc((size_t)(L.ld_t + b * b + 2), sizeof(double));
    L.wm = (double *)calloc((size_t)(m * b), sizeof(double));
    L.wn = (double *)calloc((size_t)(n * b), sizeof(double));
    double *Uh = (double *)calloc((size_t)(tmax * tmax), sizeof(double));
    double *Vh = (double *)calloc((size_t)(tmax * tmax), sizeof(double));
    double *Sh = (double *)calloc((size_t)tmax, sizeof(double));
    double *Tt = (double *)calloc((size_t)(tmax * tmax), sizeof(double));
    double *Uk = (double *)calloc((size_t)(m * k), sizeof(double));
    double *Vk = (double *)calloc((size_t)(n * k), sizeof(double));
    double *rho = (double *)calloc((size_t)(k * b), sizeof(double));
    double *F = (double *)calloc((size_t)(b * b), sizeof(double));
    if (!L.U || !L.V || !L.T || !L.h || !L.wm || !L.wn || !Uh || !Vh || !Sh || !Tt || !Uk || !Vk ||
        !rho || !F) {
        free(L.U); free(L.V); free(L.T); free(L.h); free(L.wm); free(L.wn);
        free(Uh); free(Vh); free(Sh); free(Tt); free(Uk); free(Vk); free(rho); free(F);
        return -4;
    }

    /* start block: V0 or draws 0..b-1, orthonormalized (no T entries) */
    for (int64_t l = 0; l < b; l++) {
        if (V0) memcpy(L.wn + l * n, V0 + l * n, sizeof(double) * (size_t)n);
        else orc_rng_vector(seed, (uint64_t)l, n, L.wn + l * n);
    }
    L.draws = (uint64_t)b;
    {
        double *Rs = L.h + L.ld_t;
        const double keep = L.anorm;
        L.anorm = 0.0;  /* any nonzero column counts as independent here */
        orc_block_orth(&L, L.wn, n, L.V, 0, Rs, b);
        L.anorm = keep;
        info->breakdowns = 0;
        info->n_reorth = 0;
    }
    /* U(:, 0:b) R = A V(:, 0:b) */
    for (int64_t l = 0; l < b; l++) {
        orc_matvec(A, L.V + l * n, L.wm + l * m);
        info->n_matvec++;
    }
    {
        double *R = L.h + L.ld_t;
        orc_block_orth(&L, L.wm, m, L.U, 0, R, b);
        for (int64_t l = 0; l < b; l++)
            for (int64_t i = 0; i < b; i++) TB_(&L, i, l) = R[i + l * b];
        info->n_steps += b;
    }
    orc_block_lbp_from(&L, b, t0);

    int64_t tc = t0;
    for (int64_t it = 1; it <= maxit; it++) {
        /* SVD of T(0:tc, 0:tc) */
        for (int64_t c = 0; c < tc; c++)
            for (int64_t r = 0; r < tc; r++) Tt[r + c * tc] = TB_(&L, r, c);
        int sw = orc_jacobi_svd(tc, tc, Tt, tc, Sh, Uh, tc, Vh, tc, 200);
        if (sw > info->svd_sweeps_max) info->svd_sweeps_max = sw;
        const double smax = Sh[0];
        if (smax > L.anorm) L.anorm = smax;
        /* F = T(tc-b:tc, tc:tc+b); res_j = || F^T Uh(tc-b:tc, j) || / sigma_j */
        for (int64_t l = 0; l < b; l++)
            for (int64_t i = 0; i < b; i++) F[i + l * b] = TB_(&L, tc - b + i, tc + l);
        int64_t nconv = 0;
        double fnorm = 0.0;
        for (int64_t j = 0; j < k; j++) {
            double r2 = 0.0;
            for (int64_t l = 0; l < b; l++) {
                double s = 0.0;  /* (F^T u)_l = sum_i F(i, l) u_i */
                for (int64_t i = 0; i < b; i++) s += F[i + l * b] * Uh[(tc - b + i) + j * tc];
                rho[j + l * k] = s;  /* rho = Uh(tc-b:tc, 0:k)^T F */
                r2 += s * s;
            }
            double den = Sh[j] > DBL_EPSILON * smax ? Sh[j] : DBL_EPSILON * smax;
            double rj = (den > 0.0) ? sqrt(r2) / den : 0.0;
            res[j] = rj;
            if (rj < tol) nconv++;
        }
        for (int64_t l = 0; l < b; l++)
            for (int64_t i = 0; i < b; i++) fnorm += F[i + l * b] * F[i + l * b];
        info->beta_t = sqrt(fnorm);
        info->nconv = (int32_t)nconv;
        info->converged = (nconv == k);
        if (info->converged || it == maxit) break;

        /* augmented restart */
        orc_gemm_nn(m, tc, k, L.U, m, Uh, tc, Uk, m);   /* U~_k = U(:, 0:tc) Uh(:, 0:k) */
        orc_gemm_nn(n, tc, k, L.V, n, Vh, tc, Vk, n);   /* V~_k = V(:, 0:tc) Vh(:, 0:k) */
        memset(L.T, 0, sizeof(double) * (size_t)(L.ld_t * L.ld_t));
        for (int64_t j = 0; j < k; j++) {
            TB_(&L, j, j) = Sh[j];
            for (int64_t l = 0; l < b; l++) TB_(&L, j, k + l) = rho[j + l * k];
        }
        /* V(:, k:k+b) = V(:, tc:tc+b) */
        memmove(L.V + k * n, L.V + tc * n, sizeof(double) * (size_t)(n * b));
        memcpy(L.V, Vk, sizeof(double) * (size_t)(n * k));
        memcpy(L.U, Uk, sizeof(double) * (size_t)(m * k));
        /* W = A V(:, k:k+b) - U~_k rho, orthonormalized against U~_k */
        for (int64_t l = 0; l < b; l++) {
            orc_matvec(A, L.V + (k + l) * n, L.wm + l * m);
            info->n_matvec++;
            orc_gemv_n_sub(m, k, L.U, m, rho + l * k, L.wm + l * m);
        }
        {
            double *R = L.h + L.ld_t;
            orc_block_orth(&L, L.wm, m, L.U, k, R, b);
            for (int64_t l = 0; l < b; l++)
                for (int64_t i = 0; i < b; i++) TB_(&L, k + i, k + l) = R[i + l * b];
            info->n_steps += b;
        }
        info->restarts++;
        tc = t1;
        orc_block_lbp_from(&L, k + b, t1);
    }
    for (int64_t j = 0; j < k; j++) S[j] = Sh[j];
    orc_gemm_nn(m, tc, k, L.U, m, Uh, tc, Uout, ldu);
    orc_gemm_nn(n, tc, k, L.V, n, Vh, tc, Vout, ldv);
    orc_sign_normalize(m, n, k, Uout, ldu, Vout, ldv);
    info->anorm_est = L.anorm;
    if (t_last) *t_last = tc;
    if (Ubasis) memcpy(Ubasis, L.U, sizeof(double) * (size_t)(m * tmax));
    if (Vbasis) memcpy(Vbasis, L.V, sizeof(double) * (size_t)(n * (tmax + b)));
    if (Tout) memcpy(Tout, L.T, sizeof(double) * (size_t)(L.ld_t * L.ld_t));

    free(L.U); free(L.V); free(L.T); free(L.h); free(L.wm); free(L.wn);
    free(Uh); free(Vh); free(Sh); free(Tt); free(Uk); free(Vk); free(rho); free(F);
    return 0;
}
