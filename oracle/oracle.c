/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct FP64 CPU oracle for the R factor (and the thin Q factor)
 * of A = QR of a tall-and-skinny matrix, written from J. Langou, "Computing the R of the QR factorization
 * of tall and skinny matrices using MPI_Reduce" (arXiv:1002.4250).
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * this file's library.  The GPU library never links, calls or includes it, and nothing here
 * includes or calls the GPU library: the two share no code.
 *
 * Conventions (all functions):
 *   - matrices are column-major with an explicit leading dimension (element (i,j) of A is
 *     A[i + j*lda]);
 *   - an R factor is n x n, upper triangular, with diag(R) >= 0 and an explicit zero strict
 *     lower triangle (Section 2: the R factor is unique up to the sign of each row; fixing
 *     the diagonal's sign makes it unique);
 *   - a Householder reflector is H = I - tau * u * u^T with u = [1; v]; it maps [alpha; x]
 *     to [beta; 0] with beta = -sign(alpha) * ||[alpha; x]||_2, sign(+-0) = +1 (the
 *     reflector the paper's operator builds with LAPACK's dlarfg, Section 3 and Table 3).
 *
 * Every function is pinned by the CPU tests against something other than itself
 * (hand-derived closed forms, a planted R0, a long-double and a multiprecision Cholesky,
 * LAPACK's QR, invariants); no function here is parity unpinned.
 */
#define _POSIX_C_SOURCE 200809L
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(M, ld, i, j) ((M)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)])

/* ------------------------------------------------------------------------------------- */
/* Euclidean norm of len entries x[0], x[inc], ... by the two-pass scaled method:           */
/* s = max |x_i|, ||x|| = s * sqrt(sum (x_i / s)^2).  Immune to overflow and underflow of   */
/* the squares.                                                                           */
/* ------------------------------------------------------------------------------------- */
static double norm2_scaled(int64_t len, const double *x, int64_t inc) {
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) {
        double a = fabs(x[i * inc]);
        if (a > s) s = a;
    }
    if (s == 0.0) return 0.0;
    double q = 0.0;
    for (int64_t i = 0; i < len; ++i) {
        double t = x[i * inc] / s;
        q = fma(t, t, q);
    }
    return s * sqrt(q);
}

/* ------------------------------------------------------------------------------------- */
/* Householder reflector (the dlarfg step of the operator in Table 3, Section 2).           */
/*                                                                                         */
/* len   : number of entries of [alpha; x] (x holds len-1 entries, stride incx);           */
/* alpha : in: first entry; out: beta;                                                     */
/* x     : in: the rest; out: v, the reflector's tail (u = [1; v]);                        */
/* tau   : out: the reflector's scalar.                                                    */
/* If x is zero (or len <= 1) the reflector is the identity: tau = 0, alpha unchanged.     */
/* Otherwise beta = -sign(alpha) ||[alpha; x]||, tau = (beta - alpha)/beta,                */
/* v = x / (alpha - beta).                                                                 */
/* ------------------------------------------------------------------------------------- */
void oracle_reflector(int64_t len, double *alpha, double *x, int64_t incx, double *tau) {
    *tau = 0.0;
    if (len <= 1) return;
    double xnorm = norm2_scaled(len - 1, x, incx);
    if (xnorm == 0.0) return;
    double a = *alpha;
    double r = hypot(a, xnorm);
    double beta = (a >= 0.0) ? -r : r;
    *tau = (beta - a) / beta;
    double d = a - beta;
    for (int64_t i = 0; i < len - 1; ++i) x[i * incx] = x[i * incx] / d;
    *alpha = beta;
}

/* Apply H = I - tau [1; v][1; v]^T (v = W(j+1:m-1, j)) to column k of W, rows j..m-1.     */
static void apply_reflector_column(double *W, int64_t m, int64_t ldw, int64_t j, int64_t k,
                                   double tau) {
    const double *v = &AT(W, ldw, 0, j);
    double *y = &AT(W, ldw, 0, k);
    double w = y[j];
    for (int64_t i = j + 1; i < m; ++i) w = fma(v[i], y[i], w);
    double tw = tau * w;
    y[j] = y[j] - tw;
    for (int64_t i = j + 1; i < m; ++i) y[i] = fma(-tw, v[i], y[i]);
}

/* Row signs so that diag(R) >= 0, and an explicit zero strict lower triangle (Section 2,   */
/* the remark on uniqueness of R under a positive diagonal).                               */
void oracle_sign_fix(int64_t n, double *R, int64_t ldr) {
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t i = k + 1; i < n; ++i) AT(R, ldr, i, k) = 0.0;
        if (AT(R, ldr, k, k) < 0.0)
            for (int64_t c = k; c < n; ++c) AT(R, ldr, k, c) = -AT(R, ldr, k, c);
    }
}

/* ------------------------------------------------------------------------------------- */
/* Unblocked Householder QR of all of A, R only (the local factorization of Section 3,     */
/* Table 1, applied to the whole matrix; step 1 of Section 2).                             */
/*                                                                                         */
/* Column j is reduced by one reflector; every trailing column k > j is then updated by    */
/* it.  With nthreads > 1 the trailing columns are split cyclically over threads; each     */
/* column's arithmetic is the same sequence whatever the thread count, so the result is    */
/* bitwise independent of nthreads.                                                        */
/* ------------------------------------------------------------------------------------- */
typedef struct {
    double *W;
    int64_t m, n, ldw;
    int nthreads, tid;
    double *tau;
    pthread_barrier_t *bar;
} hh_team_t;

static void *hh_worker(void *p) {
    hh_team_t *a = (hh_team_t *)p;
    int64_t steps = a->m < a->n ? a->m : a->n;
    for (int64_t j = 0; j < steps; ++j) {
        if (j % a->nthreads == a->tid)
            oracle_reflector(a->m - j, &AT(a->W, a->ldw, j, j), &AT(a->W, a->ldw, j + 1, j), 1,
                             &a->tau[j]);
        if (a->nthreads > 1) pthread_barrier_wait(a->bar);
        double t = a->tau[j];
        if (t != 0.0)
            for (int64_t k = j + 1; k < a->n; ++k)
                if (k % a->nthreads == a->tid) apply_reflector_column(a->W, a->m, a->ldw, j, k, t);
        /* The owner of column j+1 both updates it here and builds reflector j+1 next, so the
         * next step needs no second barrier. */
    }
    return NULL;
}

int oracle_householder_r(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                         int64_t ldr, int nthreads) {
    if (n < 0 || m < 0 || ldr < n || (m > 0 && lda < m)) return 1;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) AT(R, ldr, i, k) = 0.0;
    if (m == 0 || n == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = (int)n;
    double *W = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double *tau = (double *)calloc((size_t)n, sizeof(double));
    if (!W || !tau) {
        free(W);
        free(tau);
        return 2;
    }
    for (int64_t k = 0; k < n; ++k) memcpy(&AT(W, m, 0, k), &AT(A, lda, 0, k), sizeof(double) * m);

    pthread_barrier_t bar;
    hh_team_t *team = (hh_team_t *)malloc(sizeof(hh_team_t) * nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    if (nthreads > 1) pthread_barrier_init(&bar, NULL, (unsigned)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        team[t] = (hh_team_t){W, m, n, m, nthreads, t, tau, &bar};
        if (t > 0) pthread_create(&th[t], NULL, hh_worker, &team[t]);
    }
    hh_worker(&team[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (nthreads > 1) pthread_barrier_destroy(&bar);

    int64_t rows = m < n ? m : n;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i <= k && i < rows; ++i) AT(R, ldr, i, k) = AT(W, m, i, k);
    oracle_sign_fix(n, R, ldr);
    free(team);
    free(th);
    free(W);
    free(tau);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Thin QR of all of A (m >= n): Q (m x n, orthonormal columns) and R (n x n, diag >= 0)    */
/* with A = Q R.  The factorization is the one of oracle_householder_r; Q is then formed by */
/* applying its reflectors to the first n columns of the identity, Q = H_0 H_1 ... H_{n-1}   */
/* [I_n; 0] (Section 3: the Q factor is obtained by applying the stored Householder        */
/* transformations to the identity).  Column k of [I_n; 0] is e_k, which H_j leaves alone   */
/* for j > k (it is zero on rows j..m-1), so column k receives H_k, H_{k-1}, ..., H_0 in    */
/* that order.  Columns are independent: with nthreads > 1 they are split cyclically and    */
/* the result is bitwise independent of nthreads.  The sign convention diag(R) >= 0 negates */
/* row k of R and column k of Q together, which leaves Q R unchanged.                       */
/* ------------------------------------------------------------------------------------- */
typedef struct {
    const double *W;
    double *Q;
    int64_t m, n, ldw, ldq;
    const double *tau;
    int nthreads, tid;
} q_team_t;

static void *q_worker(void *p) {
    q_team_t *a = (q_team_t *)p;
    for (int64_t k = a->tid; k < a->n; k += a->nthreads) {
        double *q = &AT(a->Q, a->ldq, 0, k);
        for (int64_t i = 0; i < a->m; ++i) q[i] = (i == k) ? 1.0 : 0.0;
        for (int64_t j = k; j >= 0; --j) {
            const double t = a->tau[j];
            if (t == 0.0) continue;
            const double *u = &AT(a->W, a->ldw, 0, j);
            double s = q[j];
            for (int64_t i = j + 1; i < a->m; ++i) s = fma(u[i], q[i], s);
            const double ts = t * s;
            q[j] -= ts;
            for (int64_t i = j + 1; i < a->m; ++i) q[i] = fma(-ts, u[i], q[i]);
        }
    }
    return NULL;
}

int oracle_householder_qr(const double *A, int64_t m, int64_t n, int64_t lda, double *Q,
                          int64_t ldq, double *R, int64_t ldr, int nthreads) {
    if (n < 0 || m < n || ldr < n || (m > 0 && (lda < m || ldq < m))) return 1;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) AT(R, ldr, i, k) = 0.0;
    if (n == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = (int)n;
    double *W = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double *tau = (double *)calloc((size_t)n, sizeof(double));
    hh_team_t *team = (hh_team_t *)malloc(sizeof(hh_team_t) * nthreads);
    q_team_t *qteam = (q_team_t *)malloc(sizeof(q_team_t) * nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    if (!W || !tau || !team || !qteam || !th) {
        free(W);
        free(tau);
        free(team);
        free(qteam);
        free(th);
        return 2;
    }
    for (int64_t k = 0; k < n; ++k) memcpy(&AT(W, m, 0, k), &AT(A, lda, 0, k), sizeof(double) * m);

    /* the factorization: reflector j's tail is W(j+1:m-1, j), its scalar tau[j] */
    pthread_barrier_t bar;
    if (nthreads > 1) pthread_barrier_init(&bar, NULL, (unsigned)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        team[t] = (hh_team_t){W, m, n, m, nthreads, t, tau, &bar};
        if (t > 0) pthread_create(&th[t], NULL, hh_worker, &team[t]);
    }
    hh_worker(&team[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (nthreads > 1) pthread_barrier_destroy(&bar);

    /* Q = H_0 ... H_{n-1} [I_n; 0], column by column */
    for (int t = 0; t < nthreads; ++t) {
        qteam[t] = (q_team_t){W, Q, m, n, m, ldq, tau, nthreads, t};
        if (t > 0) pthread_create(&th[t], NULL, q_worker, &qteam[t]);
    }
    q_worker(&qteam[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);

    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i <= k; ++i) AT(R, ldr, i, k) = AT(W, m, i, k);
    for (int64_t k = 0; k < n; ++k) {
        const double dkk = AT(R, ldr, k, k);  /* before the sign fix below negates row k */
        if (dkk < 0.0)
            for (int64_t i = 0; i < m; ++i) AT(Q, ldq, i, k) = -AT(Q, ldq, i, k);
    }
    oracle_sign_fix(n, R, ldr);
    free(team);
    free(qteam);
    free(th);
    free(W);
    free(tau);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* The reduction operator qr(R1, R2) of Section 2 (Table 3): the QR factorization of the   */
/* 2n x n matrix [R1; R2] of two upper triangles, with no arithmetic on known zeros.       */
/*                                                                                         */
/* For column j the reflector's support is R1(j,j) and R2(0:j, j) (j+2 entries).  When it  */
/* is not the identity and j < n-1, every trailing column k > j is updated:                */
/*   w_k = R1(j,k) + sum_{i=0..j} R2(i,j) R2(i,k)                                          */
/*   R1(j,k) -= tau w_k,   R2(i,k) -= tau R2(i,j) w_k  (i = 0..j).                         */
/* On return R1 holds R (diagonal signs as the reflectors leave them, not fixed) and R2    */
/* holds the reflector tails (the operator's V), tau the scalars.  If flops is non-NULL,   */
/* every floating-point multiply, add, divide and square root done on the operator's data  */
/* is counted there (reflector norm scaling counted as one division and one fma per entry). */
/* ------------------------------------------------------------------------------------- */
void oracle_qr_uppers(int64_t n, double *R1, int64_t ld1, double *R2, int64_t ld2, double *tau,
                      int64_t *flops) {
    int64_t f = 0;
    for (int64_t j = 0; j < n; ++j) {
        oracle_reflector(j + 2, &AT(R1, ld1, j, j), &AT(R2, ld2, 0, j), 1, &tau[j]);
        /* norm: (j+1) divisions + (j+1) fmas; hypot, sign, tau, divisor, scaling */
        f += 2 * (j + 1) * 2 + 1 + 2 + 1 + (j + 1);
        if (j < n - 1 && tau[j] != 0.0) {
            for (int64_t k = j + 1; k < n; ++k) {
                double w = AT(R1, ld1, j, k);
                for (int64_t i = 0; i <= j; ++i) w = fma(AT(R2, ld2, i, j), AT(R2, ld2, i, k), w);
                double tw = tau[j] * w;
                AT(R1, ld1, j, k) -= tw;
                for (int64_t i = 0; i <= j; ++i)
                    AT(R2, ld2, i, k) = fma(-tw, AT(R2, ld2, i, j), AT(R2, ld2, i, k));
                f += 2 * (j + 1) + 1 + 1 + 2 * (j + 1);
            }
        }
    }
    if (flops) *flops = f;
}

/* ------------------------------------------------------------------------------------- */
/* TSQR on the CPU (Section 2 with the trees of Section 1): every row tile of height b gets */
/* its own Householder QR (step 1), then the tile R factors are reduced with qr(R_i, R_j)  */
/* (step 2) along                                                                          */
/*   tree = 0 : a binary tree -- level by level, nodes (2t, 2t+1) combined with the lower   */
/*              index on top, an odd last node promoted unchanged (Fig. 1 for 4 tiles);    */
/*   tree = 1 : a flat tree -- R <- qr(R, R_t) for t = 1, 2, ... in tile order;             */
/*   tree = 2 : hybrid -- flat within consecutive groups of `group` tiles, binary across    */
/*              the groups' results.                                                        */
/* Diagonal signs are fixed once, at the root.  A tile shorter than n rows is zero-padded   */
/* to n rows, which leaves its R unchanged.                                                */
/* ------------------------------------------------------------------------------------- */
static int tile_r(const double *A, int64_t m, int64_t n, int64_t lda, int64_t r0, int64_t rows,
                  double *Rt) {
    /* R of rows r0..r0+rows-1 of A without the final sign fix: Householder as above. */
    int64_t h = rows < n ? n : rows;
    double *W = (double *)calloc((size_t)h * (size_t)n, sizeof(double));
    if (!W) return 2;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < rows; ++i) AT(W, h, i, k) = AT(A, lda, r0 + i, k);
    (void)m;
    for (int64_t j = 0; j < n; ++j) {
        double t;
        oracle_reflector(h - j, &AT(W, h, j, j), &AT(W, h, j + 1, j), 1, &t);
        if (t != 0.0)
            for (int64_t k = j + 1; k < n; ++k) apply_reflector_column(W, h, h, j, k, t);
    }
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) AT(Rt, n, i, k) = (i <= k) ? AT(W, h, i, k) : 0.0;
    free(W);
    return 0;
}

static void combine_into(int64_t n, double *Rl, const double *Rr, double *scratch, double *tau) {
    memcpy(scratch, Rr, sizeof(double) * n * n);
    oracle_qr_uppers(n, Rl, n, scratch, n, tau, NULL);
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = k + 1; i < n; ++i) AT(Rl, n, i, k) = 0.0;
}

int oracle_tsqr_r(const double *A, int64_t m, int64_t n, int64_t lda, int64_t b, int tree,
                  int64_t group, double *R, int64_t ldr) {
    if (n < 0 || m < 0 || b < 1 || ldr < n || (m > 0 && lda < m) || tree < 0 || tree > 2) return 1;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) AT(R, ldr, i, k) = 0.0;
    if (m == 0 || n == 0) return 0;
    int64_t T = (m + b - 1) / b;
    double *Rs = (double *)malloc(sizeof(double) * (size_t)T * n * n);
    double *scratch = (double *)malloc(sizeof(double) * n * n);
    double *tau = (double *)malloc(sizeof(double) * n);
    if (!Rs || !scratch || !tau) {
        free(Rs);
        free(scratch);
        free(tau);
        return 2;
    }
    for (int64_t t = 0; t < T; ++t) {
        int64_t r0 = t * b, rows = (r0 + b <= m) ? b : m - r0;
        if (tile_r(A, m, n, lda, r0, rows, Rs + t * n * n)) {
            free(Rs);
            free(scratch);
            free(tau);
            return 2;
        }
    }
    if (tree == 1 || (tree == 2 && group <= 1)) {
        for (int64_t t = 1; t < T; ++t) combine_into(n, Rs, Rs + t * n * n, scratch, tau);
    } else {
        int64_t g = (tree == 2) ? group : 1;
        int64_t cnt = 0;
        /* flat within groups (g == 1: nothing to do), results compacted to the front */
        for (int64_t s = 0; s < T; s += g) {
            double *dst = Rs + cnt * n * n;
            if (dst != Rs + s * n * n) memcpy(dst, Rs + s * n * n, sizeof(double) * n * n);
            for (int64_t t = s + 1; t < s + g && t < T; ++t)
                combine_into(n, dst, Rs + t * n * n, scratch, tau);
            ++cnt;
        }
        /* binary across what is left */
        while (cnt > 1) {
            int64_t nxt = 0;
            for (int64_t t = 0; t < cnt; t += 2) {
                double *dst = Rs + nxt * n * n;
                if (dst != Rs + t * n * n) memcpy(dst, Rs + t * n * n, sizeof(double) * n * n);
                if (t + 1 < cnt) combine_into(n, dst, Rs + (t + 1) * n * n, scratch, tau);
                ++nxt;
            }
            cnt = nxt;
        }
    }
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) AT(R, ldr, i, k) = AT(Rs, n, i, k);
    oracle_sign_fix(n, R, ldr);
    free(Rs);
    free(scratch);
    free(tau);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Closed form for full-rank A: R = the upper Cholesky factor of A^T A (R^T R = A^T A with  */
/* diag(R) > 0 is unique).  Gram matrix and factorization in long double.  Brute force for  */
/* tiny inputs only.  Returns 3 if A^T A is not numerically positive definite.             */
/* ------------------------------------------------------------------------------------- */
int oracle_cholesky_r_ld(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                         int64_t ldr) {
    if (n < 1 || m < 1 || lda < m || ldr < n) return 1;
    long double *G = (long double *)calloc((size_t)n * n, sizeof(long double));
    if (!G) return 2;
    for (int64_t k = 0; k < n; ++k)
        for (int64_t l = k; l < n; ++l) {
            long double s = 0.0L;
            for (int64_t i = 0; i < m; ++i)
                s += (long double)AT(A, lda, i, k) * (long double)AT(A, lda, i, l);
            G[k + l * n] = s;
        }
    int rc = 0;
    /* G = U^T U, U upper, row by row: U(k,k) = sqrt(G(k,k) - sum_{i<k} U(i,k)^2),
     * U(k,l) = (G(k,l) - sum_{i<k} U(i,k) U(i,l)) / U(k,k). U overwrites G's upper half. */
    for (int64_t k = 0; k < n && !rc; ++k) {
        long double d = G[k + k * n];
        for (int64_t i = 0; i < k; ++i) d -= G[i + k * n] * G[i + k * n];
        if (!(d > 0.0L)) {
            rc = 3;
            break;
        }
        long double ukk = sqrtl(d);
        G[k + k * n] = ukk;
        for (int64_t l = k + 1; l < n; ++l) {
            long double s = G[k + l * n];
            for (int64_t i = 0; i < k; ++i) s -= G[i + k * n] * G[i + l * n];
            G[k + l * n] = s / ukk;
        }
    }
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) AT(R, ldr, i, k) = (i <= k && !rc) ? (double)G[i + k * n] : 0.0;
    free(G);
    return rc;
}

/* ------------------------------------------------------------------------------------- */
/* Checker: compensated Gram matrix G = A^T A (upper triangle and its mirror), each entry   */
/* by the Dot2 algorithm of Ogita, Rump and Oishi (2005): TwoProduct by fma, TwoSum by      */
/* Knuth's six-operation sum, errors accumulated in a second double.  The result is as     */
/* accurate as if computed in twice the working precision, then rounded.                   */
/* ------------------------------------------------------------------------------------- */
static double dot2(int64_t len, const double *x, int64_t incx, const double *y, int64_t incy) {
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < len; ++i) {
        double p = x[i * incx] * y[i * incy];
        double pe = fma(x[i * incx], y[i * incy], -p);
        double t = s + p;
        double z = t - s;
        double se = (s - (t - z)) + (p - z);
        s = t;
        c += pe + se;
    }
    return s + c;
}

typedef struct {
    const double *A;
    int64_t m, n, lda;
    double *G;
    int64_t ldg;
    int nthreads, tid;
} gram_job_t;

static void *gram_worker(void *p) {
    gram_job_t *a = (gram_job_t *)p;
    int64_t idx = 0;
    for (int64_t k = 0; k < a->n; ++k)
        for (int64_t l = k; l < a->n; ++l, ++idx)
            if (idx % a->nthreads == a->tid) {
                double v = dot2(a->m, &AT(a->A, a->lda, 0, k), 1, &AT(a->A, a->lda, 0, l), 1);
                AT(a->G, a->ldg, k, l) = v;
                AT(a->G, a->ldg, l, k) = v;
            }
    return NULL;
}

int oracle_gram_dot2(const double *A, int64_t m, int64_t n, int64_t lda, double *G, int64_t ldg,
                     int nthreads) {
    if (n < 0 || m < 0 || ldg < n || (m > 0 && lda < m)) return 1;
    if (nthreads < 1) nthreads = 1;
    gram_job_t *jobs = (gram_job_t *)malloc(sizeof(gram_job_t) * nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (gram_job_t){A, m, n, lda, G, ldg, nthreads, t};
        if (t > 0) pthread_create(&th[t], NULL, gram_worker, &jobs[t]);
    }
    gram_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return 0;
}

/* ||R^T R - G||_F / trace(G), with R^T R by Dot2 (R upper triangular, n x n) and G = A^T A. */
double oracle_gram_residual(int64_t n, const double *G, int64_t ldg, const double *R, int64_t ldr) {
    double tr = 0.0, ss = 0.0;
    for (int64_t k = 0; k < n; ++k) tr += AT(G, ldg, k, k);
    for (int64_t k = 0; k < n; ++k)
        for (int64_t l = 0; l < n; ++l) {
            int64_t len = (k < l ? k : l) + 1; /* rows 0..min(k,l) of R are the nonzero overlap */
            double rr = dot2(len, &AT(R, ldr, 0, k), 1, &AT(R, ldr, 0, l), 1);
            double d = rr - AT(G, ldg, k, l);
            ss = fma(d, d, ss);
        }
    return tr > 0.0 ? sqrt(ss) / tr : sqrt(ss);
}
