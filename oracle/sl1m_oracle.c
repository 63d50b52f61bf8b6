/*
 * sl1m_oracle.c -- plain, slow, FP64 CPU oracle for the SL1M hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) links, imports or calls this file.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark use it.
 *
 * What it computes (Hardy 2013, "Direct deconvolution of radio synthesis
 * images using L1 minimisation"):
 *   - the operator entry A_kj for Dirac pixels (Eq. deltam), paraxial
 *     Gaussian pixels (Eq. samlm4) and wide-field Gaussian pixels (Eq. samlm5),
 *     times an optional per-pixel, per-antenna complex gain product;
 *   - the forward product  Vhat_k = sum_j A_kj x_j           (Eq. sme);
 *   - the adjoint          g_j    = sum_k Re(conj(A_kj) r_k);
 *   - the step constant L, the largest eigenvalue of Re(A^H W A), by power
 *     iteration (Sect. 3.1 names such a routine but not its method);
 *   - FISTA with the positive soft threshold (Sect. 3, the algorithm box and
 *     Eq. threshp), with the relative-change-of-E stopping rule;
 *   - MFISTA, the monotone variant Sect. 3 names (Beck & Teboulle 2009b).
 *
 * Index convention: pixel j (n_pix of them), visibility k (n_vis of them).
 * The paper's M_jk (j = visibility, k = pixel) is A_kj here.
 *
 * Readings of the paper taken here (each is pinned by a test):
 *   R1  Eq. samlm4/samlm5 print a factor 1/sigma^2 in front.  Integrating
 *       Eq. samlm3 with the unit-integral pixel of Eq. gaus gives the closed
 *       form WITHOUT it (and the sigma->0 limit the paper states only exists
 *       without it), so it is dropped: A = (g/n) q exp(q c).
 *   R2  Eq. samlmexp/samlm5 print the residual wide-field phase as
 *       w (n - 1 - r^2/2).  Its own Taylor expansion (Eq. taylorexp) and the
 *       sigma->0 limit only hold for w (n - 1 + r^2/2), which is used here.
 *   R3  The image is real and M complex: the gradient is Re(A^H (A y - V)).
 *   R4  The box's fixed point minimises  1/2 sum W|A I - V|^2 + lambda sum I
 *       over I >= 0; E reported by the solver is that objective (the paper's
 *       Eq. cme without the 1/2 is reported beside it).
 *   R5  n - 1 is evaluated as -(l^2+m^2)/(1+n) to avoid cancellation.
 *   R6  Gains: g_jk = G[j][a_k] * conj(G[j][b_k]).  Weights W_k >= 0 multiply
 *       the squared residual (W = 1 is the paper's case).
 *   R7  Threshold ties (x == d) map to 0, as Eq. threshp states.
 *   R8  MFISTA keeps the proximal point z_k when F(z_k) == F(x_{k-1}), and
 *       stops when the step proposed a relative change of F below tol.
 *
 * Summation order: forward sums pixels in index order j = 0..n_pix-1, adjoint
 * sums visibilities in index order k = 0..n_vis-1, with plain FP64 "+=".
 * A pixel with x_j == 0 contributes an exact zero and is skipped; that leaves
 * every partial sum unchanged.
 *
 * Threads: single-threaded unless the problem's n_threads is above 1.  Then
 * the outer loop of a forward (its rows) or an adjoint (its columns) is cut
 * into contiguous ranges, one per thread; every output element is still one
 * sum, in the order above, by one thread, so the results are bit for bit
 * those of the single-threaded run.  Nothing else is threaded.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_DIRAC 0
#define ORC_GAUSS_PARAXIAL 1
#define ORC_GAUSS_WIDE 2

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2

static const double ORC_PI = 3.14159265358979323846264338327950288;

typedef struct {
    long n_vis;
    const double *uvw;      /* [n_vis][3], wavelengths                       */
    const double *weights;  /* [n_vis] or NULL (= 1)                          */
    const int *ant_pair;    /* [n_vis][2] or NULL (needed only with gains)   */
    long n_pix;
    const double *lm;       /* [n_pix][2], direction cosines                 */
    const double *sigma;    /* [n_pix] or NULL (= 0)                          */
    const int *kind;        /* [n_pix] or NULL (= Dirac)                      */
    int n_ant;
    const double *gains;    /* [n_pix][n_ant][2] or NULL (= unit gains)      */
    int n_threads;          /* threads for the outer loops; <= 1: one        */
} orc_problem;

typedef struct {
    int iters;          /* number of FISTA steps taken (I_1 .. I_iters)        */
    int converged;      /* 1 when the relative change of E met the tolerance    */
    double E;           /* 1/2 sum W|A I - V|^2 + lambda sum I   (reading R4)   */
    double E_paper;     /* sum W|A I - V|^2 + lambda sum I       (Eq. cme)      */
    double resid2;      /* sum W|A I - V|^2                                     */
    double l1;          /* sum I                                                */
    long nnz;           /* number of I_j > 0                                    */
    double t_final;     /* t_{iters+1} of the momentum sequence                 */
} orc_stats;

/* Operator entry without gain, Eq. deltam (Dirac), Eq. samlm4 (paraxial
 * Gaussian, reading R1) and Eq. samlm5 (wide-field Gaussian, readings R1,R2). */
static double complex entry(int kind, double l, double m, double sigma,
                            double u, double v, double w)
{
    const double complex i = _Complex_I;
    double r2 = l * l + m * m;
    double n = sqrt(1.0 - r2);
    double nm1 = -r2 / (1.0 + n);                       /* R5 */
    if (kind == ORC_DIRAC) {
        /* Eq. deltam: (1/n) exp(-2 pi i (u l + v m + w (n - 1))) */
        return cexp(-2.0 * ORC_PI * i * (u * l + v * m + w * nm1)) / n;
    }
    /* Eq. samlm4: q = 1/(1 - i w sigma^2),
     *   exponent = q * ( -2 pi i (l u + m v) + i pi w (l^2+m^2)
     *                    - pi sigma^2 (u^2+v^2) ) */
    double s2 = sigma * sigma;
    double complex q = 1.0 / (1.0 - i * w * s2);
    double complex c = -2.0 * ORC_PI * i * (l * u + m * v)
                       + i * ORC_PI * w * r2
                       - ORC_PI * s2 * (u * u + v * v);
    double complex a = q * cexp(q * c) / n;
    if (kind == ORC_GAUSS_WIDE) {
        /* Eq. samlm5: keep the non-quadratic phase at the pixel centre (R2) */
        a *= cexp(-2.0 * ORC_PI * i * w * (nm1 + 0.5 * r2));
    }
    return a;
}

/* Full entry A_kj including the gain product of reading R6. */
static double complex entry_kj(const orc_problem *P, long k, long j)
{
    const double *uvw = P->uvw + 3 * k;
    int kind = P->kind ? P->kind[j] : ORC_DIRAC;
    double sg = P->sigma ? P->sigma[j] : 0.0;
    double complex a = entry(kind, P->lm[2 * j], P->lm[2 * j + 1], sg,
                             uvw[0], uvw[1], uvw[2]);
    if (P->gains) {
        int aa = P->ant_pair[2 * k], bb = P->ant_pair[2 * k + 1];
        const double *ga = P->gains + 2 * ((size_t)j * P->n_ant + aa);
        const double *gb = P->gains + 2 * ((size_t)j * P->n_ant + bb);
        double complex g = (ga[0] + _Complex_I * ga[1]) * conj(gb[0] + _Complex_I * gb[1]);
        a *= g;
    }
    return a;
}

static int check_problem(const orc_problem *P)
{
    if (!P || P->n_vis < 0 || P->n_pix < 0) return ORC_ERR_ARG;
    if ((P->n_vis > 0 && !P->uvw) || (P->n_pix > 0 && !P->lm)) return ORC_ERR_ARG;
    if (P->gains && (!P->ant_pair || P->n_ant <= 0)) return ORC_ERR_ARG;
    for (long j = 0; j < P->n_pix; ++j) {
        double l = P->lm[2 * j], m = P->lm[2 * j + 1];
        if (!(l * l + m * m < 1.0)) return ORC_ERR_ARG;
    }
    if (P->gains) {
        for (long k = 0; k < P->n_vis; ++k) {
            int aa = P->ant_pair[2 * k], bb = P->ant_pair[2 * k + 1];
            if (aa < 0 || bb < 0 || aa >= P->n_ant || bb >= P->n_ant) return ORC_ERR_ARG;
        }
    }
    return ORC_OK;
}

/* ---- exported entry points ------------------------------------------------ */

int orc_entry(int kind, double l, double m, double sigma,
              double u, double v, double w, double *out /* [2] */)
{
    if (!(l * l + m * m < 1.0) || !out) return ORC_ERR_ARG;
    double complex a = entry(kind, l, m, sigma, u, v, w);
    out[0] = creal(a);
    out[1] = cimag(a);
    return ORC_OK;
}

int orc_entry_kj(const orc_problem *P, long k, long j, double *out)
{
    if (check_problem(P) || k < 0 || k >= P->n_vis || j < 0 || j >= P->n_pix) return ORC_ERR_ARG;
    double complex a = entry_kj(P, k, j);
    out[0] = creal(a);
    out[1] = cimag(a);
    return ORC_OK;
}

/* One row of the forward product, Eq. sme: sum_j A_kj x_j in pixel order. */
static void forward_row(const orc_problem *P, const double *x, long k, double *out)
{
    double complex acc = 0.0;
    for (long j = 0; j < P->n_pix; ++j) {
        if (x[j] == 0.0) continue;
        acc += entry_kj(P, k, j) * x[j];
    }
    out[0] = creal(acc);
    out[1] = cimag(acc);
}

/* One column of the adjoint: sum_k Re(conj(A_kj) r_k) in visibility order. */
static void adjoint_col(const orc_problem *P, const double *r, long j, double *out)
{
    double acc = 0.0;
    for (long k = 0; k < P->n_vis; ++k) {
        double complex rk = r[2 * k] + _Complex_I * r[2 * k + 1];
        acc += creal(conj(entry_kj(P, k, j)) * rk);
    }
    *out = acc;
}

/* A contiguous range [t0, t1) of the outputs of a forward (rows) or an
 * adjoint (columns); idx == NULL: output t is row / column t. */
typedef struct {
    const orc_problem *P;
    const double *in;
    const long *idx;
    long t0, t1;
    double *out;
    int adjoint;
} orc_range;

static void *run_range(void *arg)
{
    const orc_range *R = (const orc_range *)arg;
    for (long t = R->t0; t < R->t1; ++t) {
        long e = R->idx ? R->idx[t] : t;
        if (R->adjoint) adjoint_col(R->P, R->in, e, R->out + t);
        else forward_row(R->P, R->in, e, R->out + 2 * t);
    }
    return NULL;
}

/* All n outputs: in one thread, or cut into P->n_threads contiguous ranges. */
static int run_outputs(const orc_problem *P, const double *in, long n, const long *idx,
                       double *out, int adjoint)
{
    long nt = P->n_threads > 1 ? P->n_threads : 1;
    if (nt > n) nt = n;
    if (nt <= 1) {
        orc_range R = {P, in, idx, 0, n, out, adjoint};
        run_range(&R);
        return ORC_OK;
    }
    orc_range *R = malloc(sizeof(orc_range) * nt);
    pthread_t *th = malloc(sizeof(pthread_t) * nt);
    if (!R || !th) { free(R); free(th); return ORC_ERR_OOM; }
    for (long q = 0; q < nt; ++q) {
        orc_range r = {P, in, idx, n * q / nt, n * (q + 1) / nt, out, adjoint};
        R[q] = r;
    }
    long started = 1;
    while (started < nt && pthread_create(&th[started], NULL, run_range, &R[started]) == 0) ++started;
    run_range(&R[0]);
    for (long q = 1; q < started; ++q) pthread_join(th[q], NULL);
    for (long q = started; q < nt; ++q) run_range(&R[q]);   /* threads that could not start */
    free(R);
    free(th);
    return ORC_OK;
}

/* Forward product, Eq. sme: out_k = sum_j A_kj x_j, for the visibilities
 * listed in rows[0..n_rows) (rows == NULL: all, in order).  out is
 * [n_rows][2]. */
int orc_forward_rows(const orc_problem *P, const double *x, long n_rows,
                     const long *rows, double *out)
{
    if (check_problem(P) || (!x && P->n_pix) || !out) return ORC_ERR_ARG;
    long nr = rows ? n_rows : P->n_vis;
    for (long t = 0; rows && t < nr; ++t)
        if (rows[t] < 0 || rows[t] >= P->n_vis) return ORC_ERR_ARG;
    return run_outputs(P, x, nr, rows, out, 0);
}

int orc_forward(const orc_problem *P, const double *x, double *out)
{
    return orc_forward_rows(P, x, 0, NULL, out);
}

/* Adjoint: out_j = sum_k Re(conj(A_kj) r_k) for the pixels listed in
 * cols[0..n_cols) (cols == NULL: all, in order).  r is [n_vis][2]. */
int orc_adjoint_cols(const orc_problem *P, const double *r, long n_cols,
                     const long *cols, double *out)
{
    if (check_problem(P) || (!r && P->n_vis) || !out) return ORC_ERR_ARG;
    long nc = cols ? n_cols : P->n_pix;
    for (long t = 0; cols && t < nc; ++t)
        if (cols[t] < 0 || cols[t] >= P->n_pix) return ORC_ERR_ARG;
    return run_outputs(P, r, nc, cols, out, 1);
}

int orc_adjoint(const orc_problem *P, const double *r, double *out)
{
    return orc_adjoint_cols(P, r, 0, NULL, out);
}

/* z = Re(A^H W A x); work is [n_vis][2]. */
static int normal_op(const orc_problem *P, const double *x, double *work, double *z)
{
    int st = orc_forward(P, x, work);
    if (st) return st;
    if (P->weights) {
        for (long k = 0; k < P->n_vis; ++k) {
            work[2 * k] *= P->weights[k];
            work[2 * k + 1] *= P->weights[k];
        }
    }
    return orc_adjoint(P, work, z);
}

static double norm2(const double *x, long n)
{
    double s = 0.0;
    for (long j = 0; j < n; ++j) s += x[j] * x[j];
    return sqrt(s);
}

/* Step constant L: largest eigenvalue of B = Re(A^H W A) by power iteration.
 * Start x = (1,...,1)/sqrt(n_pix); each step z = B x, mu = ||z||, x = z/mu.
 * Stop when |mu_i - mu_{i-1}| <= tol * mu_i or after max_iter steps.
 * L = the last mu (for a unit x, ||B x|| <= lambda_max). */
int orc_power(const orc_problem *P, int max_iter, double tol,
              double *L_out, int *iters_out)
{
    if (check_problem(P) || P->n_pix <= 0 || P->n_vis <= 0 || max_iter <= 0 || !L_out)
        return ORC_ERR_ARG;
    long np = P->n_pix;
    double *x = malloc(sizeof(double) * np);
    double *z = malloc(sizeof(double) * np);
    double *work = malloc(sizeof(double) * 2 * P->n_vis);
    if (!x || !z || !work) { free(x); free(z); free(work); return ORC_ERR_OOM; }
    for (long j = 0; j < np; ++j) x[j] = 1.0 / sqrt((double)np);
    double mu = 0.0, mu_prev = 0.0;
    int it = 0, st = ORC_OK;
    for (it = 1; it <= max_iter; ++it) {
        st = normal_op(P, x, work, z);
        if (st) break;
        mu = norm2(z, np);
        if (mu == 0.0) break;
        for (long j = 0; j < np; ++j) x[j] = z[j] / mu;
        if (it > 1 && fabs(mu - mu_prev) <= tol * mu) break;
        mu_prev = mu;
    }
    if (it > max_iter) it = max_iter;
    free(x); free(z); free(work);
    if (st) return st;
    *L_out = mu;
    if (iters_out) *iters_out = it;
    return mu > 0.0 ? ORC_OK : ORC_ERR_ARG;
}

/* Eq. threshp: T^d(x) = x - d when x > d, else 0 (reading R7). */
static double thresh_pos(double x, double d)
{
    return x > d ? x - d : 0.0;
}

/* sum W |A x - V|^2; work is [n_vis][2]. */
static int resid2_of(const orc_problem *P, const double *x, const double *vis,
                     double *work, double *out)
{
    int st = orc_forward(P, x, work);
    if (st) return st;
    double s = 0.0;
    for (long k = 0; k < P->n_vis; ++k) {
        double dr = work[2 * k] - vis[2 * k];
        double di = work[2 * k + 1] - vis[2 * k + 1];
        double wk = P->weights ? P->weights[k] : 1.0;
        s += wk * (dr * dr + di * di);
    }
    *out = s;
    return ORC_OK;
}

/* FISTA, Sect. 3 algorithm box, with the positive threshold of Eq. threshp.
 *   Step 0:  y_1 = I_0 = x0 (zero when x0 is NULL), t_1 = 1
 *   Step k:  I_k = T^{lambda/L}( y_k - (1/L) Re A^H W (A y_k - V) )
 *            t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
 *            y_{k+1} = I_k + ((t_k - 1)/t_{k+1}) (I_k - I_{k-1})
 * Stopping (Sect. 3): when tol > 0, stop after step k once
 *   |E_k - E_{k-1}| <= tol * E_{k-1}, E_k = E(I_k) of reading R4.
 * At most max_iter steps.  img_out receives the last I_k. */
int orc_fista(const orc_problem *P, const double *vis, double lambda, double L,
              int max_iter, double tol, const double *x0, double *img_out,
              orc_stats *stats)
{
    if (check_problem(P) || !vis || !img_out || !(L > 0.0) || !(lambda >= 0.0) || max_iter < 0)
        return ORC_ERR_ARG;
    long np = P->n_pix, nv = P->n_vis;
    double *Ik = calloc(np, sizeof(double));
    double *Iprev = calloc(np, sizeof(double));
    double *y = calloc(np, sizeof(double));
    double *g = calloc(np, sizeof(double));
    double *res = calloc(2 * nv + 2, sizeof(double));
    if (!Ik || !Iprev || !y || !g || !res) {
        free(Ik); free(Iprev); free(y); free(g); free(res);
        return ORC_ERR_OOM;
    }
    if (x0) {
        memcpy(Iprev, x0, sizeof(double) * np);
        memcpy(y, x0, sizeof(double) * np);
        memcpy(Ik, x0, sizeof(double) * np);
    }
    double t = 1.0;
    double E_prev = 0.0;
    int st = ORC_OK, k = 0, converged = 0;
    if (tol > 0.0) {
        double r2;
        st = resid2_of(P, Iprev, vis, res, &r2);
        double l1 = 0.0;
        for (long j = 0; j < np; ++j) l1 += Iprev[j];
        E_prev = 0.5 * r2 + lambda * l1;
    }
    for (k = 1; k <= max_iter && st == ORC_OK; ++k) {
        /* gradient Re A^H W (A y_k - V) */
        st = orc_forward(P, y, res);
        if (st) break;
        for (long q = 0; q < nv; ++q) {
            double wk = P->weights ? P->weights[q] : 1.0;
            res[2 * q] = wk * (res[2 * q] - vis[2 * q]);
            res[2 * q + 1] = wk * (res[2 * q + 1] - vis[2 * q + 1]);
        }
        st = orc_adjoint(P, res, g);
        if (st) break;
        for (long j = 0; j < np; ++j)
            Ik[j] = thresh_pos(y[j] - g[j] / L, lambda / L);
        double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double beta = (t - 1.0) / t_next;
        for (long j = 0; j < np; ++j)
            y[j] = Ik[j] + beta * (Ik[j] - Iprev[j]);
        memcpy(Iprev, Ik, sizeof(double) * np);
        t = t_next;
        if (tol > 0.0) {
            double r2;
            st = resid2_of(P, Ik, vis, res, &r2);
            if (st) break;
            double l1 = 0.0;
            for (long j = 0; j < np; ++j) l1 += Ik[j];
            double E = 0.5 * r2 + lambda * l1;
            if (fabs(E - E_prev) <= tol * E_prev) { converged = 1; break; }
            E_prev = E;
        }
    }
    int iters = (k > max_iter) ? max_iter : k;
    if (st == ORC_OK) {
        memcpy(img_out, Ik, sizeof(double) * np);
        if (stats) {
            double r2 = 0.0;
            st = resid2_of(P, Ik, vis, res, &r2);
            double l1 = 0.0;
            long nnz = 0;
            for (long j = 0; j < np; ++j) { l1 += Ik[j]; nnz += Ik[j] > 0.0; }
            stats->iters = iters;
            stats->converged = converged;
            stats->resid2 = r2;
            stats->l1 = l1;
            stats->nnz = nnz;
            stats->E = 0.5 * r2 + lambda * l1;
            stats->E_paper = r2 + lambda * l1;
            stats->t_final = t;
        }
    }
    free(Ik); free(Iprev); free(y); free(g); free(res);
    return st;
}

/* MFISTA, the monotone FISTA of Beck & Teboulle (2009b), which Sect. 3 names
 * as the alternative to FISTA that keeps the objective from rising.  With
 * F(x) = 1/2 sum W|A x - V|^2 + lambda sum x over x >= 0 (reading R4) and the
 * same proximal step as the FISTA box:
 *   Step 0:  x_0 = y_1 = x0 (zero when x0 is NULL), t_1 = 1
 *   Step k:  z_k = T^{lambda/L}( y_k - (1/L) Re A^H W (A y_k - V) )
 *            t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
 *            x_k = z_k if F(z_k) <= F(x_{k-1}), else x_{k-1}
 *            y_{k+1} = x_k + (t_k/t_{k+1}) (z_k - x_k)
 *                          + ((t_k - 1)/t_{k+1}) (x_k - x_{k-1})
 * (ties keep the new point z_k).  Stopping: when tol > 0, stop after step k
 * once |F(z_k) - F(x_{k-1})| <= tol * F(x_{k-1}), i.e. the step proposed a
 * relative change of the objective below tol (on an accepted step this is
 * the FISTA rule on E(x_k)).  img_out receives the last x_k.
 * trace (may be NULL) receives, for each step k = 1..iters, the row
 *   [ y_k (n_pix) | z_k (n_pix) | x_k (n_pix) | t_k | F(z_k) | F(x_k) ]
 * of 3 n_pix + 3 doubles; it must hold max_iter rows. */
static int objective_of(const orc_problem *P, const double *x, const double *vis, double lambda,
                        double *work, double *out)
{
    double r2;
    int st = resid2_of(P, x, vis, work, &r2);
    if (st) return st;
    double l1 = 0.0;
    for (long j = 0; j < P->n_pix; ++j) l1 += x[j];
    *out = 0.5 * r2 + lambda * l1;
    return ORC_OK;
}

int orc_mfista(const orc_problem *P, const double *vis, double lambda, double L,
               int max_iter, double tol, const double *x0, double *img_out,
               orc_stats *stats, double *trace)
{
    if (check_problem(P) || !vis || !img_out || !(L > 0.0) || !(lambda >= 0.0) || max_iter < 0)
        return ORC_ERR_ARG;
    long np = P->n_pix, nv = P->n_vis;
    double *x = calloc(np, sizeof(double));      /* x_{k-1}, then x_k */
    double *z = calloc(np, sizeof(double));
    double *y = calloc(np, sizeof(double));
    double *g = calloc(np, sizeof(double));
    double *res = calloc(2 * nv + 2, sizeof(double));
    if (!x || !z || !y || !g || !res) {
        free(x); free(z); free(y); free(g); free(res);
        return ORC_ERR_OOM;
    }
    if (x0) {
        memcpy(x, x0, sizeof(double) * np);
        memcpy(y, x0, sizeof(double) * np);
    }
    double t = 1.0, Fx = 0.0;
    int st = objective_of(P, x, vis, lambda, res, &Fx);
    int k = 0, converged = 0;
    const long row = 3 * np + 3;
    for (k = 1; k <= max_iter && st == ORC_OK; ++k) {
        double *tr = trace ? trace + (long)(k - 1) * row : NULL;
        if (tr) memcpy(tr, y, sizeof(double) * np);
        /* z_k: the proximal gradient step at y_k */
        st = orc_forward(P, y, res);
        if (st) break;
        for (long q = 0; q < nv; ++q) {
            double wk = P->weights ? P->weights[q] : 1.0;
            res[2 * q] = wk * (res[2 * q] - vis[2 * q]);
            res[2 * q + 1] = wk * (res[2 * q + 1] - vis[2 * q + 1]);
        }
        st = orc_adjoint(P, res, g);
        if (st) break;
        for (long j = 0; j < np; ++j)
            z[j] = thresh_pos(y[j] - g[j] / L, lambda / L);
        double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        /* x_k: the better of z_k and x_{k-1} */
        double Fz;
        st = objective_of(P, z, vis, lambda, res, &Fz);
        if (st) break;
        const double Fx_prev = Fx;
        const int take = Fz <= Fx;
        /* y_{k+1}; x_k - x_{k-1} is z_k - x_{k-1} when z_k is taken, else 0 */
        for (long j = 0; j < np; ++j) {
            double xk = take ? z[j] : x[j];
            y[j] = xk + (t / t_next) * (z[j] - xk) + ((t - 1.0) / t_next) * (xk - x[j]);
            x[j] = xk;
        }
        if (take) Fx = Fz;
        if (tr) {
            memcpy(tr + np, z, sizeof(double) * np);
            memcpy(tr + 2 * np, x, sizeof(double) * np);
            tr[3 * np] = t;
            tr[3 * np + 1] = Fz;
            tr[3 * np + 2] = Fx;
        }
        t = t_next;
        if (tol > 0.0 && fabs(Fz - Fx_prev) <= tol * Fx_prev) { converged = 1; break; }
    }
    int iters = (k > max_iter) ? max_iter : k;
    if (st == ORC_OK) {
        memcpy(img_out, x, sizeof(double) * np);
        if (stats) {
            double r2 = 0.0;
            st = resid2_of(P, x, vis, res, &r2);
            double l1 = 0.0;
            long nnz = 0;
            for (long j = 0; j < np; ++j) { l1 += x[j]; nnz += x[j] > 0.0; }
            stats->iters = iters;
            stats->converged = converged;
            stats->resid2 = r2;
            stats->l1 = l1;
            stats->nnz = nnz;
            stats->E = 0.5 * r2 + lambda * l1;
            stats->E_paper = r2 + lambda * l1;
            stats->t_final = t;
        }
    }
    free(x); free(z); free(y); free(g); free(res);
    return st;
}
