/*
 * qmc_oracle.c -- plain, slow, fp64 CPU oracle for the delayed Slater-determinant
 * update (McDaniel, D'Azevedo, Li, Wong, Kent, "Delayed Slater determinant update
 * algorithms for high efficiency quantum Monte Carlo").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Convention: the paper's. The Slater matrix M has one COLUMN per electron,
 * M[i][k] = phi_i(r_k) (Sec. I). A move of electron k replaces column k; the
 * change is the column vector u = (new column) - (old column), so
 * M_new = M + u e_k' (Sec. I). The caller's matrices use the transposed layout
 * (one row per electron, A = M'), so every entry point transposes on the way in
 * and out; an inverse is returned as Minv stored row-major, which is exactly
 * A^{-1} stored column-major.
 *
 * Implementations of one sweep, each a different reading of the paper:
 *   O1 brute force: ratio det(M_new)/det(M) from two LU determinants.
 *   O2 Sherman-Morrison: ratio by the matrix determinant lemma (Eq. 1), inverse
 *      by the rank-1 Sherman-Morrison formula (Eq. 2).
 *   O3 delayed: ratios by look-ahead -- the explicit determinant of
 *      I_k + V' M^{-1} U (Eq. 3) divided by the previous one -- and the queued
 *      accepted moves applied en bloc by Sherman-Morrison-Woodbury (Eq. 4) when k
 *      reaches K or the sweep ends (Sec. II). Rejected moves change nothing.
 *   O3' delayed, fixed slots: Sec. II's other treatment of a rejected move --
 *      it takes a queue slot like an accepted one, with its column left
 *      unchanged (a zero change) -- so that the queue holds every proposal
 *      and is flushed every K proposals and at the end of the sweep.
 *
 * Metropolis rule: accept iff u < min(1, r^2) (the acceptance probability is
 * the squared determinant ratio, Sec. I). A per-move override (-1 decide, 0
 * reject, 1 accept) replays decisions; |min(1, r^2) - u| < 1e-10 counts as a
 * near tie.
 *
 * Threads: loops whose iterations write disjoint output elements (the rows of
 * an elimination step, the columns of an inverse, the rows of a rank-k update,
 * the entries of a look-ahead border) may run on several OpenMP threads. Every
 * element is still computed by the same sequence of operations as on one
 * thread, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SINGULAR 3
#define OR_ERR_OOM 4

#define METHOD_BRUTE 0
#define METHOD_SM 1
#define METHOD_DELAYED 2
#define METHOD_DELAYED_SLOT 3
#define IS_DELAYED(m) ((m) == METHOD_DELAYED || (m) == METHOD_DELAYED_SLOT)

static const double NEAR_TIE = 1e-10;

/* Wall time of the last oracle_sweeps call after its setup (the LU
 * determinant and inverse of the starting matrix): the update work alone,
 * for the benchmark's CPU baseline. */
static double last_update_seconds = 0.0;

double oracle_last_update_seconds(void) { return last_update_seconds; }

static double wall_seconds(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Below this many multiply-adds a loop stays on one thread. */
#define PAR_WORK 65536L

/* Threads for the parallel loops (n <= 0: every processor). Returns the
 * count in effect, 1 without OpenMP. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (textbook Doolittle, row interchanges).      */
/* a: n x n row-major, overwritten by L (unit, strictly below) and U.          */
/* perm[c]: row exchanged with row c at step c. Pivot = largest |a_ic|, first  */
/* index on ties. Returns 1 if an exactly zero pivot appears.                  */
/* ------------------------------------------------------------------------ */
static int lu_factor(int n, double *a, int *perm, int *nswaps)
{
    int singular = 0;
    *nswaps = 0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        double best = fabs(a[(size_t)c * n + c]);
        for (int i = c + 1; i < n; ++i) {
            double v = fabs(a[(size_t)i * n + c]);
            if (v > best) { best = v; p = i; }
        }
        perm[c] = p;
        if (p != c) {
            for (int j = 0; j < n; ++j) {
                double t = a[(size_t)c * n + j];
                a[(size_t)c * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
            ++*nswaps;
        }
        double piv = a[(size_t)c * n + c];
        if (piv == 0.0) { singular = 1; continue; }
        #pragma omp parallel for schedule(static) if ((long)(n - c) * (n - c) > PAR_WORK)
        for (int i = c + 1; i < n; ++i) {
            double l = a[(size_t)i * n + c] / piv;
            a[(size_t)i * n + c] = l;
            for (int j = c + 1; j < n; ++j)
                a[(size_t)i * n + j] -= l * a[(size_t)c * n + j];
        }
    }
    return singular;
}

/* log|det a| and sign(det a) of an n x n row-major matrix (a is not modified). */
int oracle_slogdet(int n, const double *a, double *logabs, int *sign)
{
    if (n < 0) return OR_ERR_ARG;
    if (n == 0) { *logabs = 0.0; *sign = 1; return OR_OK; }
    double *lu = malloc(sizeof(double) * (size_t)n * n);
    int *perm = malloc(sizeof(int) * (size_t)n);
    if (!lu || !perm) { free(lu); free(perm); return OR_ERR_OOM; }
    memcpy(lu, a, sizeof(double) * (size_t)n * n);
    int nswaps;
    int singular = lu_factor(n, lu, perm, &nswaps);
    double s = (nswaps % 2) ? -1.0 : 1.0, la = 0.0;
    for (int c = 0; c < n; ++c) {
        double d = lu[(size_t)c * n + c];
        if (d < 0) s = -s;
        la += log(fabs(d));
    }
    free(lu); free(perm);
    if (singular) { *logabs = -INFINITY; *sign = 0; return OR_ERR_SINGULAR; }
    *logabs = la;
    *sign = (int)s;
    return OR_OK;
}

/* inv = a^{-1} (both n x n row-major) by LU and two triangular solves per
 * column of the identity. */
int oracle_inverse(int n, const double *a, double *inv)
{
    if (n < 0) return OR_ERR_ARG;
    if (n == 0) return OR_OK;
    double *lu = malloc(sizeof(double) * (size_t)n * n);
    int *perm = malloc(sizeof(int) * (size_t)n);
    double *x = malloc(sizeof(double) * (size_t)n);
    if (!lu || !perm || !x) { free(lu); free(perm); free(x); return OR_ERR_OOM; }
    memcpy(lu, a, sizeof(double) * (size_t)n * n);
    int nswaps;
    if (lu_factor(n, lu, perm, &nswaps)) { free(lu); free(perm); free(x); return OR_ERR_SINGULAR; }
    int oom = 0;
    #pragma omp parallel if ((long)n * n > PAR_WORK)
    {
        double *xt = x;                      /* thread 0 reuses x, the others their own */
#ifdef _OPENMP
        if (omp_get_thread_num() != 0) xt = malloc(sizeof(double) * (size_t)n);
#endif
        if (!xt) {
            #pragma omp atomic write
            oom = 1;
        }
        #pragma omp for schedule(static)
        for (int col = 0; col < n; ++col) {
            if (!xt) continue;
            for (int i = 0; i < n; ++i) xt[i] = (i == col) ? 1.0 : 0.0;
            for (int c = 0; c < n; ++c) {          /* apply the row interchanges */
                int p = perm[c];
                if (p != c) { double t = xt[c]; xt[c] = xt[p]; xt[p] = t; }
            }
            for (int i = 0; i < n; ++i)             /* L y = P e_col */
                for (int j = 0; j < i; ++j) xt[i] -= lu[(size_t)i * n + j] * xt[j];
            for (int i = n - 1; i >= 0; --i) {      /* U x = y */
                for (int j = i + 1; j < n; ++j) xt[i] -= lu[(size_t)i * n + j] * xt[j];
                xt[i] /= lu[(size_t)i * n + i];
            }
            for (int i = 0; i < n; ++i) inv[(size_t)i * n + col] = xt[i];
        }
        if (xt != x) free(xt);
    }
    if (oom) { free(lu); free(perm); free(x); return OR_ERR_OOM; }
    free(lu); free(perm); free(x);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Walker state in the paper's convention.                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, K, method;
    double *M;      /* current Slater matrix, column k = electron k           */
    double *Minv;   /* SM/brute: inverse of M. Delayed: inverse at last flush */
    double logabs;  /* running log|det M|                                     */
    double sign;    /* running sign of det M                                  */
    /* delayed (O3) queue */
    int k;          /* queued accepted moves                                  */
    int *elec;      /* electron of queued move m (columns of V are e_elec[m]) */
    double *U;      /* n x K, column m = change of column elec[m] (stride K)  */
    double *S;      /* (K+1) x (K+1): I + V' Minv U for the queue + proposal  */
    double blk_logabs, blk_sign; /* det of the k x k block (product of ratios) */
    /* pending proposal */
    int prop_j;
    double *prop_col;  /* proposed new column                                 */
    double *u;         /* change u = prop_col - M[:, j]                        */
    double prop_logabs, prop_sign; /* look-ahead: det of the (k+1) block      */
    double ratio;
    double terms;   /* 1 + sum_i |row j of the inverse in use| |u_i|: the size of */
                    /* Eq. 1's terms, which bounds the rounding of its dot product */
} walker;

static void walker_free(walker *w)
{
    free(w->M); free(w->Minv); free(w->elec); free(w->U); free(w->S);
    free(w->prop_col); free(w->u);
}

/* init_alt = 1: the starting inverse from the LU of the caller's matrix A
 * (rows = electrons), transposed, instead of the LU of M = A' -- another fp64
 * computation of the same inverse, whose difference from the usual one shows
 * how much the starting inverse alone moves a walk. */
static int walker_init_alt(walker *w, int n, int K, int method, const double *A_rows, int init_alt);

static int walker_init(walker *w, int n, int K, int method, const double *A_rows)
{
    return walker_init_alt(w, n, K, method, A_rows, 0);
}

static int walker_init_alt(walker *w, int n, int K, int method, const double *A_rows, int init_alt)
{
    memset(w, 0, sizeof(*w));
    w->n = n; w->K = K > 0 ? K : 1; w->method = method;
    size_t nn = (size_t)n * n;
    w->M = malloc(sizeof(double) * (nn ? nn : 1));
    w->Minv = malloc(sizeof(double) * (nn ? nn : 1));
    w->elec = malloc(sizeof(int) * (size_t)w->K);
    w->U = malloc(sizeof(double) * ((size_t)n * w->K + 1));
    w->S = malloc(sizeof(double) * (size_t)(w->K + 1) * (w->K + 1));
    w->prop_col = malloc(sizeof(double) * ((size_t)n + 1));
    w->u = malloc(sizeof(double) * ((size_t)n + 1));
    if (!w->M || !w->Minv || !w->elec || !w->U || !w->S || !w->prop_col || !w->u) {
        walker_free(w); return OR_ERR_OOM;
    }
    for (int i = 0; i < n; ++i)          /* M = A': column k = row k of A */
        for (int k = 0; k < n; ++k) w->M[(size_t)i * n + k] = A_rows[(size_t)k * n + i];
    int sg;
    int st = oracle_slogdet(n, w->M, &w->logabs, &sg);
    if (st) { walker_free(w); return st; }
    w->sign = sg;
    if (init_alt) {
        st = oracle_inverse(n, A_rows, w->Minv);     /* A^{-1}, row-major */
        if (st) { walker_free(w); return st; }
        for (int i = 0; i < n; ++i)                   /* Minv = (A^{-1})' */
            for (int k = i + 1; k < n; ++k) {
                double t = w->Minv[(size_t)i * n + k];
                w->Minv[(size_t)i * n + k] = w->Minv[(size_t)k * n + i];
                w->Minv[(size_t)k * n + i] = t;
            }
    } else {
        st = oracle_inverse(n, w->M, w->Minv);
        if (st) { walker_free(w); return st; }
    }
    w->k = 0;
    w->blk_logabs = 0.0; w->blk_sign = 1.0;
    return OR_OK;
}

/* Determinant of the leading m x m block of the (K+1)-stride matrix S. */
static void small_slogdet(const double *S, int stride, int m, double *logabs, double *sign)
{
    double *t = malloc(sizeof(double) * (size_t)(m > 0 ? m * m : 1));
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) t[i * m + j] = S[i * stride + j];
    int sg;
    if (oracle_slogdet(m, t, logabs, &sg) != OR_OK) { *logabs = -INFINITY; *sign = 0.0; }
    else *sign = sg;
    free(t);
}

/* Ratio det(M_new)/det(M) for electron j moving to new column `col`. */
static double walker_propose(walker *w, int j, const double *col)
{
    int n = w->n;
    w->prop_j = j;
    memcpy(w->prop_col, col, sizeof(double) * n);
    for (int i = 0; i < n; ++i) w->u[i] = col[i] - w->M[(size_t)i * n + j];

    if (w->method == METHOD_BRUTE) {
        /* Direct calculation: det of the moved matrix over det of M. */
        double *Mn = malloc(sizeof(double) * (size_t)n * n);
        memcpy(Mn, w->M, sizeof(double) * (size_t)n * n);
        for (int i = 0; i < n; ++i) Mn[(size_t)i * n + j] = col[i];
        double la_new, la_old; int s_new, s_old;
        oracle_slogdet(n, Mn, &la_new, &s_new);
        oracle_slogdet(n, w->M, &la_old, &s_old);
        free(Mn);
        w->ratio = (s_new == 0) ? 0.0 : (double)(s_new * s_old) * exp(la_new - la_old);
        double ta = 1.0;
        for (int i = 0; i < n; ++i) ta += fabs(w->Minv[(size_t)j * n + i] * w->u[i]);
        w->terms = ta;
    } else if (w->method == METHOD_SM) {
        /* Eq. 1: det(M + u e_j')/det(M) = 1 + e_j' Minv u. */
        double t = 1.0;
        double ta = 1.0;
        for (int i = 0; i < n; ++i) {
            t += w->Minv[(size_t)j * n + i] * w->u[i];
            ta += fabs(w->Minv[(size_t)j * n + i] * w->u[i]);
        }
        w->ratio = t;
        w->terms = ta;
    } else {
        /* Eq. 3 look-ahead. The queue gives U (changes) and V (unit columns
         * e_elec[m]); the proposal appends u and e_j. Entry (a, b) of
         * I + V' Minv U is delta_ab + row elec[a] of Minv dotted with column b
         * of U. Rows/columns 0..k-1 were filled when the queue grew; fill the
         * new border and take the explicit determinant of the (k+1) block. */
        int k = w->k, st = w->K + 1;
        const double *urow_j = w->Minv + (size_t)j * n;     /* e_j' Minv */
        #pragma omp parallel for schedule(static) if ((long)n * k > PAR_WORK)
        for (int b = 0; b < k; ++b) {                         /* new row k */
            double t = 0.0;
            for (int i = 0; i < n; ++i) t += urow_j[i] * w->U[(size_t)i * w->K + b];
            w->S[k * st + b] = t;
        }
        #pragma omp parallel for schedule(static) if ((long)n * k > PAR_WORK)
        for (int a = 0; a < k; ++a) {                         /* new column k */
            const double *row = w->Minv + (size_t)w->elec[a] * n;
            double t = 0.0;
            for (int i = 0; i < n; ++i) t += row[i] * w->u[i];
            w->S[a * st + k] = t;
        }
        double t = 1.0;
        double ta = 1.0;
        for (int i = 0; i < n; ++i) {
            t += urow_j[i] * w->u[i];
            ta += fabs(urow_j[i] * w->u[i]);
        }
        w->terms = ta;
        w->S[k * st + k] = t;
        small_slogdet(w->S, st, k + 1, &w->prop_logabs, &w->prop_sign);
        if (w->prop_sign == 0.0) w->ratio = 0.0;
        else w->ratio = w->prop_sign * w->blk_sign * exp(w->prop_logabs - w->blk_logabs);
    }
    return w->ratio;
}

/* Apply the queued moves to Minv by Sherman-Morrison-Woodbury (Eq. 4):
 * Minv <- Minv - (Minv U) (I_k + V' Minv U)^{-1} (V' Minv). */
static int walker_flush(walker *w)
{
    if (!IS_DELAYED(w->method) || w->k == 0) return OR_OK;
    int n = w->n, k = w->k, st = w->K + 1, KK = w->K;
    double *S = malloc(sizeof(double) * (size_t)k * k);
    double *Sinv = malloc(sizeof(double) * (size_t)k * k);
    double *MU = malloc(sizeof(double) * (size_t)n * k);     /* Minv U, n x k */
    double *VM = malloc(sizeof(double) * (size_t)k * n);     /* V' Minv, k x n */
    double *X = malloc(sizeof(double) * (size_t)n * k);      /* (Minv U) Sinv */
    if (!S || !Sinv || !MU || !VM || !X) {
        free(S); free(Sinv); free(MU); free(VM); free(X); return OR_ERR_OOM;
    }
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) S[a * k + b] = w->S[a * st + b];
    int status = oracle_inverse(k, S, Sinv);
    if (status == OR_OK) {
        #pragma omp parallel for schedule(static) if ((long)n * n * k > PAR_WORK)
        for (int i = 0; i < n; ++i)
            for (int b = 0; b < k; ++b) {
                double t = 0.0;
                for (int l = 0; l < n; ++l) t += w->Minv[(size_t)i * n + l] * w->U[(size_t)l * KK + b];
                MU[(size_t)i * k + b] = t;
            }
        for (int a = 0; a < k; ++a)
            memcpy(VM + (size_t)a * n, w->Minv + (size_t)w->elec[a] * n, sizeof(double) * n);
        #pragma omp parallel for schedule(static) if ((long)n * k * k > PAR_WORK)
        for (int i = 0; i < n; ++i)
            for (int b = 0; b < k; ++b) {
                double t = 0.0;
                for (int a = 0; a < k; ++a) t += MU[(size_t)i * k + a] * Sinv[a * k + b];
                X[(size_t)i * k + b] = t;
            }
        #pragma omp parallel for schedule(static) if ((long)n * n * k > PAR_WORK)
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < n; ++l) {
                double t = 0.0;
                for (int b = 0; b < k; ++b) t += X[(size_t)i * k + b] * VM[(size_t)b * n + l];
                w->Minv[(size_t)i * n + l] -= t;
            }
        w->k = 0;
        w->blk_logabs = 0.0; w->blk_sign = 1.0;
    }
    free(S); free(Sinv); free(MU); free(VM); free(X);
    return status;
}

/* Accept the pending proposal. */
static int walker_accept(walker *w)
{
    int n = w->n, j = w->prop_j;
    double r = w->ratio;
    if (!(r != 0.0) || !isfinite(r)) return OR_ERR_SINGULAR;
    if (w->method == METHOD_SM) {
        /* Eq. 2: Minv <- Minv - (Minv u)(1 + e_j' Minv u)^{-1}(e_j' Minv). */
        double *x = malloc(sizeof(double) * n), *y = malloc(sizeof(double) * n);
        #pragma omp parallel for schedule(static) if ((long)n * n > PAR_WORK)
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int l = 0; l < n; ++l) t += w->Minv[(size_t)i * n + l] * w->u[l];
            x[i] = t;
        }
        memcpy(y, w->Minv + (size_t)j * n, sizeof(double) * n);
        #pragma omp parallel for schedule(static) if ((long)n * n > PAR_WORK)
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < n; ++l) w->Minv[(size_t)i * n + l] -= x[i] * y[l] / r;
        free(x); free(y);
    } else if (IS_DELAYED(w->method)) {
        int k = w->k;
        for (int i = 0; i < n; ++i) w->U[(size_t)i * w->K + k] = w->u[i];
        w->elec[k] = j;
        w->blk_logabs = w->prop_logabs;
        w->blk_sign = w->prop_sign;
        w->k = k + 1;
    }
    for (int i = 0; i < n; ++i) w->M[(size_t)i * n + j] = w->prop_col[i];
    w->logabs += log(fabs(r));
    if (r < 0) w->sign = -w->sign;
    if (w->method == METHOD_BRUTE) {
        int st = oracle_inverse(n, w->M, w->Minv);
        if (st) return st;
    }
    if (IS_DELAYED(w->method) && w->k == w->K) return walker_flush(w);
    return OR_OK;
}

/* Fixed slots (Sec. II): the rejected proposal still takes slot k, with the
 * unchanged column of electron j, i.e. a zero change. The new column of
 * I + V' Minv U is then e_k (row elec[a] of Minv times a zero column), its new
 * row the one filled at the proposal, so the block determinant is unchanged;
 * A, the running log|det| and sign stay as they are. */
static int walker_reject_slot(walker *w)
{
    int n = w->n, k = w->k, st = w->K + 1;
    for (int i = 0; i < n; ++i) w->U[(size_t)i * w->K + k] = 0.0;
    for (int a = 0; a < k; ++a) w->S[a * st + k] = 0.0;
    w->S[k * st + k] = 1.0;
    w->elec[k] = w->prop_j;
    w->k = k + 1;
    if (w->k == w->K) return walker_flush(w);
    return OR_OK;
}

static int in_queue(const walker *w, int j)
{
    for (int m = 0; m < w->k; ++m) if (w->elec[m] == j) return 1;
    return 0;
}

static void walker_export(const walker *w, double *A_rows, double *Ainv_cm,
                          double *logabs, int *sign)
{
    int n = w->n;
    if (A_rows)
        for (int k = 0; k < n; ++k)
            for (int i = 0; i < n; ++i) A_rows[(size_t)k * n + i] = w->M[(size_t)i * n + k];
    if (Ainv_cm) memcpy(Ainv_cm, w->Minv, sizeof(double) * (size_t)n * n);
    if (logabs) *logabs = w->logabs;
    if (sign) *sign = (int)w->sign;
}

static int decide(double r, double u, int override, long long *near_ties)
{
    double p = r * r;
    if (p > 1.0) p = 1.0;
    if (fabs(p - u) < NEAR_TIE) ++*near_ties;
    if (override == 0) return 0;
    if (override == 1) return 1;
    return u < p;
}

/*
 * One or more Metropolis sweeps. Electron j = 0..n-1 in order; the proposed
 * row is v = a_j + sigma * g with a_j the CURRENT row j and g = G[s][j][:].
 *   A0       n x n, row j = electron j (input)
 *   G        nsweeps x n x n Gaussians, U nsweeps x n uniforms
 *   override nsweeps x n (-1 decide, 0 reject, 1 accept) or NULL
 * Outputs: ratios, accepted (nsweeps x n), final A rows, final inverse in the
 * column-major layout of A^{-1}, running log|det| and sign, near-tie count;
 * terms (nsweeps x n, may be NULL): 1 + sum_i |(row j of the inverse) u_i| of
 * each proposal (for the delayed readings with the inverse of the last flush).
 * method + 16: the same reading started from the alternative inverse (see
 * walker_init_alt).
 * The delayed method flushes when k reaches K and at the end of every sweep.
 * max_moves >= 0 stops after that many proposals (a bounded sample; the queue
 * is flushed); -1 runs every sweep in full.
 */
int oracle_sweeps(int method, int n, int K, int nsweeps, double sigma,
                  const double *A0, const double *G, const double *U,
                  const signed char *override,
                  double *ratios, double *terms, unsigned char *accepted,
                  double *A_out, double *Ainv_out, double *logabs, int *sign,
                  long long *near_ties, long long max_moves)
{
    const int init_alt = (method & 16) != 0;
    method &= 15;
    if (n < 1 || nsweeps < 0 || method < METHOD_BRUTE || method > METHOD_DELAYED_SLOT ||
        (IS_DELAYED(method) && K < 1))
        return OR_ERR_ARG;
    walker w;
    int st = walker_init_alt(&w, n, K, method, A0, init_alt);
    if (st) return st;
    const double t_start = wall_seconds();
    double *col = malloc(sizeof(double) * n);
    *near_ties = 0;
    long long done = 0;
    for (int s = 0; s < nsweeps && st == OR_OK; ++s) {
        for (int j = 0; j < n && st == OR_OK; ++j) {
            if (max_moves >= 0 && done >= max_moves) break;
            ++done;
            const double *g = G + ((size_t)s * n + j) * n;
            for (int i = 0; i < n; ++i) col[i] = w.M[(size_t)i * n + j] + sigma * g[i];
            double r = walker_propose(&w, j, col);
            size_t at = (size_t)s * n + j;
            ratios[at] = r;
            if (terms) terms[at] = w.terms;
            int ov = override ? override[at] : -1;
            int acc = decide(r, U[at], ov, near_ties);
            accepted[at] = (unsigned char)acc;
            if (acc) st = walker_accept(&w);
            else if (method == METHOD_DELAYED_SLOT) st = walker_reject_slot(&w);
        }
        if (st == OR_OK) st = walker_flush(&w);
    }
    last_update_seconds = wall_seconds() - t_start;
    if (st == OR_OK) walker_export(&w, A_out, Ainv_out, logabs, sign);
    free(col);
    walker_free(&w);
    return st;
}

/*
 * Explicit moves: move m proposes new row vrows[m] for electron elec[m]; the
 * decision is given (decisions[m]: 1 accept, 0 reject). The delayed method
 * flushes when k reaches K, before proposing an electron already queued, when
 * flush_after[m] is set (may be NULL), and at the end.
 */
int oracle_moves(int method, int n, int K, int nmoves, const double *A0,
                 const int *elec, const double *vrows,
                 const unsigned char *decisions, const unsigned char *flush_after,
                 double *ratios, double *terms, double *A_out, double *Ainv_out,
                 double *logabs, int *sign)
{
    const int init_alt = (method & 16) != 0;
    method &= 15;
    if (n < 1 || nmoves < 0 || method < METHOD_BRUTE || method > METHOD_DELAYED_SLOT ||
        (IS_DELAYED(method) && K < 1))
        return OR_ERR_ARG;
    walker w;
    int st = walker_init_alt(&w, n, K, method, A0, init_alt);
    if (st) return st;
    for (int m = 0; m < nmoves && st == OR_OK; ++m) {
        int j = elec[m];
        if (j < 0 || j >= n) { st = OR_ERR_ARG; break; }
        if (IS_DELAYED(method) && in_queue(&w, j)) st = walker_flush(&w);
        if (st) break;
        ratios[m] = walker_propose(&w, j, vrows + (size_t)m * n);
        if (terms) terms[m] = w.terms;
        if (decisions[m]) st = walker_accept(&w);
        else if (method == METHOD_DELAYED_SLOT) st = walker_reject_slot(&w);
        if (st == OR_OK && flush_after && flush_after[m]) st = walker_flush(&w);
    }
    if (st == OR_OK) st = walker_flush(&w);
    if (st == OR_OK) walker_export(&w, A_out, Ainv_out, logabs, sign);
    walker_free(&w);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Multideterminant wavefunctions (the expansion Sec. II says the delayed     */
/* scheme combines with: Clark et al.'s table method).                        */
/*                                                                            */
/* Row convention throughout this part: A[e][o] = phi_o(r_e) (electron rows,  */
/* occupied orbital columns), B[e][a] = psi_a(r_e) (nv virtual orbitals).     */
/* Determinant I replaces occupied columns o_p by virtual columns a_p,        */
/* p = 1, 2 (exc[4 I + 2(p-1)] = o_p, exc[4 I + 2(p-1) + 1] = a_p, -1 when   */
/* unused: I with no pair is the reference); Psi = sum_I coef_I det(A_I).    */
/* ------------------------------------------------------------------------ */

/* log|Psi| and sign(Psi) from every det(A_I) by LU (the definition). */
static int md_psi_direct(int n, int nv, const double *A, const double *B, int ndet, const int *exc,
                         const double *coef, double *logabs, double *sign)
{
    double *AI = malloc(sizeof(double) * (size_t)n * n);
    double *la = malloc(sizeof(double) * (size_t)(ndet > 0 ? ndet : 1));
    int *sg = malloc(sizeof(int) * (size_t)(ndet > 0 ? ndet : 1));
    if (!AI || !la || !sg) { free(AI); free(la); free(sg); return OR_ERR_OOM; }
    double lmax = -INFINITY;
    for (int I = 0; I < ndet; ++I) {
        memcpy(AI, A, sizeof(double) * (size_t)n * n);
        for (int p = 0; p < 2; ++p) {
            int o = exc[4 * I + 2 * p], a = exc[4 * I + 2 * p + 1];
            if (o < 0 || a < 0) continue;
            for (int e = 0; e < n; ++e) AI[(size_t)e * n + o] = B[(size_t)e * nv + a];
        }
        if (oracle_slogdet(n, AI, &la[I], &sg[I]) != OR_OK) { la[I] = -INFINITY; sg[I] = 0; }
        if (sg[I] != 0 && la[I] > lmax) lmax = la[I];
    }
    double s = 0.0;
    for (int I = 0; I < ndet; ++I)
        if (sg[I] != 0) s += coef[I] * sg[I] * exp(la[I] - lmax);
    free(AI); free(la); free(sg);
    if (!(s != 0.0) || !isfinite(lmax)) { *logabs = -INFINITY; *sign = 0.0; return OR_ERR_SINGULAR; }
    *logabs = lmax + log(fabs(s));
    *sign = s < 0 ? -1.0 : 1.0;
    return OR_OK;
}

/* r Psi(new) / det(A_new) after a move with reference ratio r: each
 * determinant's table block T_I (rows o_p, columns a_p) changes by the rank-1
 * term x_I d_I' / r, and the matrix determinant lemma gives
 * r det(T_I + x_I d_I' / r) = r det(T_I) + d_I' adj(T_I) x_I (reference: r;
 * one pair: r T_oa + x_o d_a; two pairs: the 2 x 2 adjugate), with no
 * division by r. */
/* Eq. 4 for the multideterminant walker's delayed reading: Ainv (rows =
 * orbitals, columns = electrons, Ainv[o][e] = (A^{-1})_{oe}) <- Ainv -
 * P Kinv (U Ainv), P = the columns idx_m of Ainv, U = the kq queued changes
 * as rows. */
static void md_flush(int n, double *Ainv, int kq, const int *qidx, const double *Uq, const double *Ki,
                     double *Pq, double *Yq)
{
    if (kq == 0) return;
    for (int o = 0; o < n; ++o)
        for (int m = 0; m < kq; ++m) Pq[(size_t)o * kq + m] = Ainv[(size_t)o * n + qidx[m]];
    for (int m = 0; m < kq; ++m)                 /* Y = U Ainv */
        for (int e = 0; e < n; ++e) {
            double t = 0.0;
            for (int o = 0; o < n; ++o) t += Uq[(size_t)m * n + o] * Ainv[(size_t)o * n + e];
            Yq[(size_t)m * n + e] = t;
        }
    for (int o = 0; o < n; ++o) {                /* Ainv -= (P Kinv) Y */
        double pk[256];
        for (int l = 0; l < kq; ++l) {
            double t = 0.0;
            for (int m = 0; m < kq; ++m) t += Pq[(size_t)o * kq + m] * Ki[(size_t)m * kq + l];
            pk[l] = t;
        }
        for (int e = 0; e < n; ++e) {
            double t = 0.0;
            for (int l = 0; l < kq; ++l) t += pk[l] * Yq[(size_t)l * n + e];
            Ainv[(size_t)o * n + e] -= t;
        }
    }
}

/* Kinv = (I + U P)^{-1} of the kq queued moves (P = the columns idx_m of the
 * last flush's Ainv): the k x k matrix of Eq. 3. */
static int md_queue_inverse(int n, const double *Ainv, int kq, const int *qidx, const double *Uq, double *Km,
                            double *Ki)
{
    for (int m = 0; m < kq; ++m)
        for (int l = 0; l < kq; ++l) {
            double t = m == l ? 1.0 : 0.0;
            for (int o = 0; o < n; ++o) t += Uq[(size_t)m * n + o] * Ainv[(size_t)o * n + qidx[l]];
            Km[(size_t)m * kq + l] = t;
        }
    return oracle_inverse(kq, Km, Ki);
}

static double md_table_num(int nv, const double *T, const double *x, const double *d, double r,
                           int ndet, const int *exc, const double *coef)
{
    double s = 0.0;
    for (int I = 0; I < ndet; ++I) {
        int o1 = exc[4 * I], a1 = exc[4 * I + 1], o2 = exc[4 * I + 2], a2 = exc[4 * I + 3];
        double t;
        if (o1 < 0 || a1 < 0) {
            t = r;
        } else if (o2 < 0 || a2 < 0) {
            t = r * T[(size_t)o1 * nv + a1] + x[o1] * d[a1];
        } else {
            double t11 = T[(size_t)o1 * nv + a1], t12 = T[(size_t)o1 * nv + a2];
            double t21 = T[(size_t)o2 * nv + a1], t22 = T[(size_t)o2 * nv + a2];
            t = r * (t11 * t22 - t12 * t21) + d[a1] * (t22 * x[o1] - t12 * x[o2]) +
                d[a2] * (t11 * x[o2] - t21 * x[o1]);
        }
        s += coef[I] * t;
    }
    return s;
}

/* sum_I coef_I det(T_I) with T_I the rows o_p, columns a_p of the table (the
 * reference: 1): Psi / det(A) by the table method (Cramer's rule). */
static double md_table_sum(int nv, const double *T, int ndet, const int *exc, const double *coef)
{
    double s = 0.0;
    for (int I = 0; I < ndet; ++I) {
        int o1 = exc[4 * I], a1 = exc[4 * I + 1], o2 = exc[4 * I + 2], a2 = exc[4 * I + 3];
        double d;
        if (o1 < 0 || a1 < 0) d = 1.0;
        else if (o2 < 0 || a2 < 0) d = T[(size_t)o1 * nv + a1];
        else d = T[(size_t)o1 * nv + a1] * T[(size_t)o2 * nv + a2] - T[(size_t)o1 * nv + a2] * T[(size_t)o2 * nv + a1];
        s += coef[I] * d;
    }
    return s;
}

#define MD_BRUTE 0
#define MD_TABLE 1
#define MD_TABLE_DELAYED 2

/*
 * Metropolis sweeps of a multideterminant walker. Electron j = 0..n-1 in
 * order; the proposed rows are v = a_j + sigma g (occupied orbitals) and
 * w = b_j + sigma h (virtual orbitals), g = G[s][j][:], h = H[s][j][:]; the
 * move is accepted iff u < min(1, R^2) with R = Psi(new) / Psi(old).
 *   MD_BRUTE  R from Psi by md_psi_direct before and after (the definition)
 *   MD_TABLE  R = r S' / S with r the reference ratio (Eq. 1), S = sum_I
 *             coef_I det(T_I) over the table T = A^{-1} B (orbitals x
 *             virtuals) and T' = T + x d' / r, d = w - b_j - T'u, x = A^{-1} e_j
 *             (the table after the move, Sherman-Morrison), r S' formed
 *             without dividing by r (md_table_num); on accept A^{-1} by
 *             Eq. 2, T <- T' and S <- S'. The table is relative to the
 *             reference determinant: accepting a move that makes it singular
 *             (r = 0) returns OR_ERR_SINGULAR.
 *   MD_TABLE_DELAYED  the table method with the reference determinant's
 *             inverse under the delayed update (Sec. II): A^{-1} stays that
 *             of the last flush, the accepted changes u_m of electrons idx_m
 *             wait in a queue of at most K, the current column
 *             x = A_c^{-1} e_j is the Woodbury form of Eq. 3-4 applied to one
 *             column, x = a_j - P (I + U P)^{-1} U a_j (a_j = A^{-1} e_j,
 *             P = A^{-1}[:, idx], U the queued changes as rows), r = 1 + u'x,
 *             and Eq. 4 flushes the queue when it holds K moves or before an
 *             electron already in it moves again (and at the end).
 * exc: ndet x 4 ints as above; coef: ndet. Outputs: ratios R (nsweeps x n),
 * accepted, final A and B rows, log|Psi| and its sign.
 */
int oracle_md_sweeps(int method, int K, int n, int nv, int nsweeps, double sigma,
                     const double *A0, const double *B0, const double *G, const double *H,
                     const double *U, int ndet, const int *exc, const double *coef,
                     const signed char *override, double *ratios, unsigned char *accepted,
                     double *A_out, double *B_out, double *logabs, int *sign)
{
    if (n < 1 || nv < 1 || nsweeps < 0 || ndet < 1 ||
        (method != MD_BRUTE && method != MD_TABLE && method != MD_TABLE_DELAYED) ||
        (method == MD_TABLE_DELAYED && (K < 1 || K > n || K > 256)))
        return OR_ERR_ARG;
    if (method != MD_TABLE_DELAYED) K = 1;
    for (int I = 0; I < ndet; ++I)
        for (int p = 0; p < 2; ++p) {
            int o = exc[4 * I + 2 * p], a = exc[4 * I + 2 * p + 1];
            if ((o >= 0) != (a >= 0) || o >= n || a >= nv) return OR_ERR_ARG;
        }
    size_t nn = (size_t)n * n, nb = (size_t)n * nv;
    double *A = malloc(sizeof(double) * nn), *B = malloc(sizeof(double) * nb);
    double *An = malloc(sizeof(double) * nn), *Bn = malloc(sizeof(double) * nb);
    double *Ainv = malloc(sizeof(double) * nn), *T = malloc(sizeof(double) * nb);
    double *Tn = malloc(sizeof(double) * nb), *u = malloc(sizeof(double) * n);
    double *x = malloc(sizeof(double) * n), *dl = malloc(sizeof(double) * nv), *y = malloc(sizeof(double) * n);
    /* the delayed reading's queue: electrons, changes (rows), the k x k
     * matrix I + U P and its inverse, scratch for Eq. 4 */
    int *qidx = malloc(sizeof(int) * K);
    double *Uq = malloc(sizeof(double) * (size_t)K * n), *Pq = malloc(sizeof(double) * (size_t)n * K);
    double *Km = malloc(sizeof(double) * (size_t)K * K), *Ki = malloc(sizeof(double) * (size_t)K * K);
    double *cq = malloc(sizeof(double) * K), *tq = malloc(sizeof(double) * K);
    double *Yq = malloc(sizeof(double) * (size_t)K * n);
    int kq = 0;
    int st = OR_OK;
    if (!A || !B || !An || !Bn || !Ainv || !T || !Tn || !u || !x || !dl || !y || !qidx || !Uq || !Pq || !Km ||
        !Ki || !cq || !tq || !Yq) { st = OR_ERR_OOM; goto done; }
    memcpy(A, A0, sizeof(double) * nn);
    memcpy(B, B0, sizeof(double) * nb);
    double lpsi, spsi;
    st = md_psi_direct(n, nv, A, B, ndet, exc, coef, &lpsi, &spsi);
    if (st) goto done;
    double S = 1.0;
    if (method != MD_BRUTE) {
        st = oracle_inverse(n, A, Ainv);     /* Ainv[o][e]: (A^{-1})_{oe} */
        if (st) goto done;
        for (int o = 0; o < n; ++o)          /* T = A^{-1} B */
            for (int a = 0; a < nv; ++a) {
                double t = 0.0;
                for (int e = 0; e < n; ++e) t += Ainv[(size_t)o * n + e] * B[(size_t)e * nv + a];
                T[(size_t)o * nv + a] = t;
            }
        S = md_table_sum(nv, T, ndet, exc, coef);
    }
    for (int s = 0; s < nsweeps && st == OR_OK; ++s) {
        for (int j = 0; j < n && st == OR_OK; ++j) {
            const double *g = G + ((size_t)s * n + j) * n, *h = H + ((size_t)s * n + j) * nv;
            double R, lnew = 0.0, snew = 0.0, Sn = 0.0, r = 0.0;
            if (method == MD_BRUTE) {
                memcpy(An, A, sizeof(double) * nn);
                memcpy(Bn, B, sizeof(double) * nb);
                for (int o = 0; o < n; ++o) An[(size_t)j * n + o] = A[(size_t)j * n + o] + sigma * g[o];
                for (int a = 0; a < nv; ++a) Bn[(size_t)j * nv + a] = B[(size_t)j * nv + a] + sigma * h[a];
                if (md_psi_direct(n, nv, An, Bn, ndet, exc, coef, &lnew, &snew) != OR_OK) R = 0.0;
                else R = snew * spsi * exp(lnew - lpsi);
            } else {
                if (method == MD_TABLE_DELAYED) {
                    int queued = 0;
                    for (int m = 0; m < kq; ++m) queued |= qidx[m] == j;
                    if (queued) {
                        md_flush(n, Ainv, kq, qidx, Uq, Ki, Pq, Yq);
                        kq = 0;
                    }
                }
                for (int o = 0; o < n; ++o) {
                    double v = A[(size_t)j * n + o] + sigma * g[o];
                    u[o] = v - A[(size_t)j * n + o];
                    x[o] = Ainv[(size_t)o * n + j];
                }
                if (method == MD_TABLE_DELAYED && kq > 0) {
                    /* x = a_j - P Kinv (U a_j): column j of the current inverse */
                    for (int m = 0; m < kq; ++m) {
                        double t = 0.0;
                        for (int o = 0; o < n; ++o) t += Uq[(size_t)m * n + o] * x[o];
                        cq[m] = t;
                    }
                    for (int m = 0; m < kq; ++m) {
                        double t = 0.0;
                        for (int l = 0; l < kq; ++l) t += Ki[(size_t)m * kq + l] * cq[l];
                        tq[m] = t;
                    }
                    for (int o = 0; o < n; ++o) {
                        double t = 0.0;
                        for (int m = 0; m < kq; ++m) t += Ainv[(size_t)o * n + qidx[m]] * tq[m];
                        x[o] -= t;
                    }
                }
                r = 1.0;                                     /* Eq. 1 */
                for (int o = 0; o < n; ++o) r += u[o] * x[o];
                for (int a = 0; a < nv; ++a) {               /* w - b_j - T'u */
                    double wb = (B[(size_t)j * nv + a] + sigma * h[a]) - B[(size_t)j * nv + a];
                    double t = 0.0;
                    for (int o = 0; o < n; ++o) t += u[o] * T[(size_t)o * nv + a];
                    dl[a] = wb - t;
                }
                const double num = md_table_num(nv, T, x, dl, r, ndet, exc, coef);
                R = num / S;
                if (r != 0.0) Sn = num / r;
            }
            size_t at = (size_t)s * n + j;
            ratios[at] = R;
            int ov = override ? override[at] : -1;
            double p = R * R;
            if (p > 1.0) p = 1.0;
            int acc = ov == 0 ? 0 : (ov == 1 ? 1 : (U[at] < p));
            if (acc && (!(R != 0.0) || !isfinite(R))) { st = OR_ERR_SINGULAR; break; }
            accepted[at] = (unsigned char)acc;
            if (!acc) continue;
            if (method == MD_BRUTE) {
                memcpy(A, An, sizeof(double) * nn);
                memcpy(B, Bn, sizeof(double) * nb);
                lpsi = lnew; spsi = snew;
            } else {
                if (!(r != 0.0)) { st = OR_ERR_SINGULAR; break; }
                for (int o = 0; o < n; ++o)          /* T <- T + x d' / r */
                    for (int a = 0; a < nv; ++a)
                        Tn[(size_t)o * nv + a] = T[(size_t)o * nv + a] + x[o] * dl[a] / r;
                if (method == MD_TABLE) {
                    /* Eq. 2 on A^{-1} (row form): A^{-1} -= x (u' A^{-1}) / r */
                    for (int e = 0; e < n; ++e) {
                        double t = 0.0;
                        for (int o = 0; o < n; ++o) t += u[o] * Ainv[(size_t)o * n + e];
                        y[e] = t;
                    }
                    for (int o = 0; o < n; ++o)
                        for (int e = 0; e < n; ++e) Ainv[(size_t)o * n + e] -= x[o] * y[e] / r;
                } else {
                    /* queue the change; Eq. 4 once K moves wait */
                    qidx[kq] = j;
                    memcpy(Uq + (size_t)kq * n, u, sizeof(double) * n);
                    ++kq;
                    st = md_queue_inverse(n, Ainv, kq, qidx, Uq, Km, Ki);
                    if (st) break;
                    if (kq == K) {
                        md_flush(n, Ainv, kq, qidx, Uq, Ki, Pq, Yq);
                        kq = 0;
                    }
                }
                memcpy(T, Tn, sizeof(double) * nb);
                for (int o = 0; o < n; ++o) A[(size_t)j * n + o] = A[(size_t)j * n + o] + sigma * g[o];
                for (int a = 0; a < nv; ++a) B[(size_t)j * nv + a] = B[(size_t)j * nv + a] + sigma * h[a];
                lpsi += log(fabs(R));
                if (R < 0) spsi = -spsi;
                S = Sn;
            }
        }
    }
    if (st == OR_OK) {
        if (A_out) memcpy(A_out, A, sizeof(double) * nn);
        if (B_out) memcpy(B_out, B, sizeof(double) * nb);
        *logabs = lpsi;
        *sign = (int)spsi;
    }
done:
    free(A); free(B); free(An); free(Bn); free(Ainv); free(T); free(Tn); free(u); free(x); free(dl); free(y);
    free(qidx); free(Uq); free(Pq); free(Km); free(Ki); free(cq); free(tq); free(Yq);
    return st;
}
