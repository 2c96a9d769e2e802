/*
 * Plain FP64 CPU oracle for Sinkhorn and Acc-Sinkhorn (entropy-regularised OT).
 *
 * TEST INFRASTRUCTURE ONLY. It is the slow, obviously correct statement of what
 * the GPU solver computes. Only the test suite, the smoke check and the CPU
 * baseline / reference legs of the benchmark may load it; the product path
 * never does. It shares no code, header, table or helper with the CUDA library.
 *
 * Paper: "Accelerating Sinkhorn for Entropy-Regularized Optimal Transport"
 * (Xu & Chen). Citations below name the paper's sections, equations and
 * algorithms.
 *
 * Conventions
 *   - The cost is divided by eps (Sec. 2, "Dual Formulation": the minimiser is
 *     unchanged, so the analysis takes eps = 1). Inside this file Chat = C/eps.
 *   - x is the paper's outer (column) variable v, called x_k in Sec. 4; u is
 *     the inner (row) variable. Both are dimensionless. Outputs are in cost
 *     units: f = eps*u, g = eps*x.
 *   - All arithmetic is IEEE double with libm exp/log/expm1; no blocking,
 *     fusion or reordering beyond the definitions.
 *   - The OpenMP pragmas only split independent rows/columns over threads;
 *     every per-row and per-column sum runs in plain index order.
 *
 * Every function is pinned by the "not gpu" tests (closed forms, brute force,
 * invariants, library routines); see tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Cost access (Sec. 5: dense C; squared Euclidean for colour transfer;       */
/* cosine 1 - <x,y> for word alignment).                                       */
/* ------------------------------------------------------------------------- */

enum { ORC_DENSE = 0, ORC_SQEUCLID = 1, ORC_COSINE = 2, ORC_DENSE64 = 3 };

typedef struct {
    int kind;         /* ORC_DENSE, ORC_SQEUCLID, ORC_COSINE, ORC_DENSE64     */
    long n, m, d;     /* rows, columns, point dimension (point clouds only)   */
    long ldc;         /* row stride of C in elements (dense only)             */
    const float *C;   /* n x m row-major FP32 cost (dense)                    */
    const float *X;   /* n x d row-major FP32 points                          */
    const float *Y;   /* m x d row-major FP32 points                          */
    double scale;     /* multiply every entry by this (1/max C, or 1)         */
    const double *C64; /* n x m row-major FP64 cost (ORC_DENSE64): a cost     */
                       /* already formed once, e.g. by orc_cost_matrix        */
} orc_cost;

/* One entry of the cost, formed in double from the FP32 inputs. */
double orc_cost_entry(const orc_cost *c, long i, long j)
{
    double v = 0.0;
    if (c->kind == ORC_DENSE) {
        v = (double)c->C[i * c->ldc + j];
    } else if (c->kind == ORC_DENSE64) {
        v = c->C64[i * c->ldc + j];
    } else if (c->kind == ORC_SQEUCLID) {
        /* C_ij = ||x_i - y_j||^2 (Sec. 5, colour transfer) */
        for (long k = 0; k < c->d; ++k) {
            double t = (double)c->X[i * c->d + k] - (double)c->Y[j * c->d + k];
            v += t * t;
        }
    } else {
        /* C_ij = 1 - <x_i, y_j> (Sec. 5, word alignment) */
        double dot = 0.0;
        for (long k = 0; k < c->d; ++k)
            dot += (double)c->X[i * c->d + k] * (double)c->Y[j * c->d + k];
        v = 1.0 - dot;
    }
    return v * c->scale;
}

/* max_ij C_ij by brute force (used for "normalised by its maximum entry",
 * Sec. 5 colour transfer). Returns the maximum of the unscaled entries. */
double orc_cost_max(const orc_cost *c)
{
    orc_cost u = *c;
    u.scale = 1.0;
    double mx = -INFINITY;
    /* a maximum does not depend on the order it is taken in */
#pragma omp parallel for schedule(static) reduction(max : mx)
    for (long i = 0; i < c->n; ++i)
        for (long j = 0; j < c->m; ++j) {
            double v = orc_cost_entry(&u, i, j);
            if (v > mx) mx = v;
        }
    return mx;
}

/* Materialise the (scaled) cost as an n x m double matrix. */
void orc_cost_matrix(const orc_cost *c, double *out)
{
    for (long i = 0; i < c->n; ++i)
        for (long j = 0; j < c->m; ++j)
            out[i * c->m + j] = orc_cost_entry(c, i, j);
}

/* ------------------------------------------------------------------------- */
/* The two exact block minimisations (Sec. 2, "Sinkhorn as Exact Coordinate   */
/* Minimization"), written in the log domain (Sec. 5 runs both solvers in the */
/* log domain).                                                               */
/* ------------------------------------------------------------------------- */

/* Row pass, the u-update of Sec. 2:
 *   u_i = log a_i - log( sum_j exp(x_j - Chat_ij) ),
 * with the log-sum-exp taken about its maximum term. */
void orc_row_pass(const orc_cost *c, double eps, const double *loga,
                  const double *x, double *u)
{
    const long n = c->n, m = c->m;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double mx = -INFINITY;
        for (long j = 0; j < m; ++j) {
            double z = x[j] - orc_cost_entry(c, i, j) / eps;
            if (z > mx) mx = z;
        }
        double s = 0.0;
        for (long j = 0; j < m; ++j)
            s += exp(x[j] - orc_cost_entry(c, i, j) / eps - mx);
        u[i] = loga[i] - (mx + log(s));
    }
}

/* Column log-sum-exp that the v-update of Sec. 2 needs:
 *   ell_j = log( sum_i exp(u_i - Chat_ij) ),
 * so that the column sums of P(u, x) are c_j = exp(x_j + ell_j) and the
 * v-update is x_j <- x_j + log(b_j / c_j) = log b_j - ell_j. */
void orc_col_lse(const orc_cost *c, double eps, const double *u, double *ell)
{
    const long n = c->n, m = c->m;
#pragma omp parallel for schedule(static)
    for (long j = 0; j < m; ++j) {
        double mx = -INFINITY;
        for (long i = 0; i < n; ++i) {
            double z = u[i] - orc_cost_entry(c, i, j) / eps;
            if (z > mx) mx = z;
        }
        double s = 0.0;
        for (long i = 0; i < n; ++i)
            s += exp(u[i] - orc_cost_entry(c, i, j) / eps - mx);
        ell[j] = mx + log(s);
    }
}

/* ------------------------------------------------------------------------- */
/* Normalised Sinkhorn map (Sec. 3, eq. normalized-sinkhorn):                 */
/*   S(x) = x - P_Nperp grad phi*( P_Nperp grad f(x) ),                       */
/* with grad f(x) = c_P - b (eq. grad-f), grad phi*(xi) = log(1 + xi./b)      */
/* (Sec. 3). When 1'a = 1'b = 1 the residual c_P - b already sums to zero, so */
/* the inner projection is the identity and S(x) is the plain v-update with   */
/* its mean removed.                                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    const orc_cost *cost;
    double eps;
    const double *a, *b;       /* marginals, each summing to 1 */
    const double *loga, *logb;
} orc_problem;

/* Evaluates S(x). Writes u = u(x) (row pass), c = column sums of P(u(x), x),
 * s = S(x). Returns the column marginal L1 error sum_j |c_j - b_j|, which is
 * the whole of the l1tol test of Sec. 5 because the row pass makes the row
 * marginal exact. */
double orc_sinkhorn_map(const orc_problem *p, const double *x, double *u,
                        double *c, double *s)
{
    const long m = p->cost->m;
    double *ell = (double *)malloc(sizeof(double) * (size_t)m);
    orc_row_pass(p->cost, p->eps, p->loga, x, u);
    orc_col_lse(p->cost, p->eps, u, ell);
    double err = 0.0, mean = 0.0;
    for (long j = 0; j < m; ++j) {
        c[j] = exp(x[j] + ell[j]);
        err += fabs(c[j] - p->b[j]);
        s[j] = p->logb[j] - ell[j];      /* v-update, eq. v-update */
        mean += s[j];
    }
    mean /= (double)m;
    for (long j = 0; j < m; ++j) s[j] -= mean; /* P_Nperp */
    free(ell);
    return err;
}

/* Dual objective in cost units, D = <f,a> + <g,b> - eps * sum_ij P_ij
 * (eq. dual-obj with the sign flipped and eps restored). After an exact row
 * pass sum_ij P_ij = 1'a = 1 (proof of the coercivity lemma, App. A), so
 * D = eps * (<u,a> + <x,b> - 1). */
double orc_dual_after_row_pass(const orc_problem *p, const double *u,
                               const double *x)
{
    double ua = 0.0, xb = 0.0;
    for (long i = 0; i < p->cost->n; ++i) ua += u[i] * p->a[i];
    for (long j = 0; j < p->cost->m; ++j) xb += x[j] * p->b[j];
    return p->eps * (ua + xb - 1.0);
}

/* ------------------------------------------------------------------------- */
/* Stability conditions (Theorem 4, App. B), evaluated literally with the     */
/* step alpha in use:                                                         */
/*   Cond 1: ||grad f(x_k)||^2_{D_k^-1 D_{k+1} D_k^-1}                        */
/*             <= (4 - alpha^2 - 2 alpha^(1/2)) / (2 alpha (1+alpha)^2)       */
/*                * D_phi*(0, grad f(x_k))                                    */
/*   Cond 2: ||v_k||^2_{D_{k+1} - D_k} <= alpha^(3/2) ||v_{k+1}||^2_{D_{k+1}} */
/* with v_k = y_k - x_k, y_k = w_k / alpha (Sec. 4), D_k = D(p_k),             */
/* p_k = grad phi*(grad f(x_k)) = log(c_k ./ b) and                            */
/* D(z) = diag(b .* (exp(z) - 1) ./ z) (eq. D, continuous at z = 0).           */
/* Because D_k p_k = grad f(x_k) (eq. D: D(z) z = grad phi(z)), the Cond 1     */
/* left side equals sum_j p_kj^2 D_{k+1,j}. D_phi*(0, xi) = sum b(e^p - 1 - p)  */
/* follows from phi*(xi) = sum (b+xi) log(1 + xi/b) - xi (Sec. 3).             */
/* Cond 2 is compared in squared form, where the left side may be negative.   */
/* ------------------------------------------------------------------------- */

/* Diagonal of D(z) for one coordinate. */
double orc_metric_D(double bj, double z)
{
    if (z == 0.0) return bj;               /* D(0) = grad^2 phi(0) = diag(b) */
    return bj * expm1(z) / z;
}

/* out[0] = Cond1 lhs, out[1] = Cond1 rhs, out[2] = Cond2 lhs,
 * out[3] = Cond2 rhs, out[4] = Cond1 holds (1/0), out[5] = Cond2 holds. */
void orc_stability_terms(long m, const double *b, const double *c_k,
                         const double *c_k1, const double *x_k,
                         const double *w_k, const double *x_k1,
                         const double *w_k1, double alpha, double *out)
{
    double l1 = 0.0, kl = 0.0, l2 = 0.0, r2 = 0.0;
    for (long j = 0; j < m; ++j) {
        double p0 = log(c_k[j] / b[j]);
        double p1 = log(c_k1[j] / b[j]);
        double D0 = orc_metric_D(b[j], p0);
        double D1 = orc_metric_D(b[j], p1);
        l1 += p0 * p0 * D1;
        kl += b[j] * (expm1(p0) - p0);
        double v0 = w_k[j] / alpha - x_k[j];
        double v1 = w_k1[j] / alpha - x_k1[j];
        l2 += v0 * v0 * (D1 - D0);
        r2 += v1 * v1 * D1;
    }
    double kappa1 = (4.0 - alpha * alpha - 2.0 * sqrt(alpha)) /
                    (2.0 * alpha * (1.0 + alpha) * (1.0 + alpha));
    out[0] = l1;
    out[1] = kappa1 * kl;
    out[2] = l2;
    out[3] = pow(alpha, 1.5) * r2;
    out[4] = (out[0] <= out[1]) ? 1.0 : 0.0;
    out[5] = (out[2] <= out[3]) ? 1.0 : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Solvers.                                                                   */
/* ------------------------------------------------------------------------- */

enum { ORC_PLAIN = 0, ORC_ACC = 1 };
enum { ORC_STAB_OFF = 0, ORC_STAB_REPORT = 1, ORC_STAB_GATE = 2, ORC_STAB_BACKTRACK = 3 };
enum { ORC_CONVERGED = 0, ORC_MAXITER = 7, ORC_BADARG = 1 };

typedef struct {
    int status;              /* ORC_CONVERGED or ORC_MAXITER                  */
    int sinkhorn_steps;      /* number of S(x) evaluations                     */
    int outer_stages;        /* completed homotopy stages (Algorithm 2)        */
    int stability_failures;  /* iterations where Cond 1 or Cond 2 failed      */
    double marginal_l1;      /* column L1 error at the returned iterate        */
    double dual;             /* dual objective D at the returned iterate       */
} orc_result;

/* History written per S evaluation (index = evaluation number), when the
 * caller passes room for it (hist_cap > 0):
 *   err_hist[e], dual_hist[e], mu_hist[e] (mu used to form that iterate, or 0
 *   for x_0 / plain), stab_hist[e] (bit0 = Cond1 failed, bit1 = Cond2 failed,
 *   for the step that produced iterate e), x_hist[e*m .. e*m+m-1] = iterate,
 *   cond[4e .. 4e+3] = Theorem 4's Cond 1 lhs, Cond 1 rhs, Cond 2 lhs and
 *   Cond 2 rhs of that step (zeros where no test ran: x_0, plain, OFF). */
typedef struct {
    long cap;
    double *err, *dual, *mu;
    int *stab;
    double *x;      /* may be NULL */
    double *cond;   /* may be NULL */
} orc_history;

static void record(orc_history *h, long e, long m, double err, double dual,
                   double mu, int stab, const double *x, const double *cond)
{
    if (!h || e >= h->cap) return;
    if (h->err) h->err[e] = err;
    if (h->dual) h->dual[e] = dual;
    if (h->mu) h->mu[e] = mu;
    if (h->stab) h->stab[e] = stab;
    if (h->x) memcpy(h->x + e * m, x, sizeof(double) * (size_t)m);
    if (h->cond)
        for (int q = 0; q < 4; ++q) h->cond[4 * e + q] = cond ? cond[q] : 0.0;
}

/*
 * Solve. method = ORC_PLAIN: x_{k+1} = S(x_k) (Sec. 3, normalised Sinkhorn).
 * method = ORC_ACC: Algorithm 1 inside the homotopy of Algorithm 2:
 *   alpha = sqrt(2 mu);
 *   x_{k+1} = (w_k + S(x_k)) / (1 + alpha);
 *   w_{k+1} = (w_k + (alpha^2 - 2) x_{k+1} + 2 S(x_{k+1})) / (1 + alpha);
 * S(x_{k+1}) is reused by the next x-update (remark after Algorithm 1); after
 * m_stage inner steps mu <- mu/2 and m_stage <- floor(sqrt(2) m_stage) + 1.
 * Both start from x_0 = w_0 = 0 (Sec. 5 starts from the zero dual variable).
 * Stopping (eq. l1tol): after each S evaluation, stop when the marginal L1
 * error of P(u(x), x) is below tol. The stability gate (mode GATE) restarts
 * the momentum, w_{k+1} <- alpha x_{k+1}, when a condition fails; mode
 * BACKTRACK instead backtracks on alpha: the current homotopy stage ends at
 * once, so the next step uses alpha = sqrt(2 mu / 2) (our reading of the
 * backtracking the paper mentions for Theorem 4's conditions).
 * Between homotopy stages Algorithm 2 hands (x, w) to the next stage as is
 * (carry_y = 0). With carry_y = 1 the stage hand-over keeps y = w / alpha
 * instead, w <- w * alpha_new / alpha_old, which is the state (x_k, y_k) that
 * Theorem 1 follows from stage to stage.
 * a and b must be positive and sum to one. f_out (n) and g_out (m) receive
 * eps*u and eps*x at the returned iterate.
 *
 * orc_solve_from starts the same iteration from a given point instead of
 * zero: x0 and w0 (m each; NULL means zero) and the homotopy position
 * (mu_start, m_stage_start, j_start inner steps taken, stages_start stages
 * completed). The loop is unchanged: its first S evaluation is at x0. When
 * x_out / w_out / stage_out are given they receive the loop's state at the
 * return, (x, w) and {mu, m_stage, j, stages}: the point the loop would
 * continue from, so a second call started there repeats S(x) once and then
 * takes exactly the steps an uninterrupted run would have taken.
 */
int orc_solve_from(const orc_problem *p, double tol, int method, double mu0,
                   int m0, int max_steps, int stab_mode, int carry_y,
                   const double *x0, const double *w0, double mu_start,
                   long m_stage_start, long j_start, int stages_start,
                   double *f_out, double *g_out, orc_result *res,
                   orc_history *hist, double *x_out, double *w_out,
                   double *stage_out)
{
    const long n = p->cost->n, m = p->cost->m;
    if (n < 1 || m < 1 || !(p->eps > 0) || !(tol > 0) || max_steps < 1)
        return ORC_BADARG;
    if (method == ORC_ACC && !(mu0 > 0 && mu0 < 1 && m0 >= 1)) return ORC_BADARG;
    if (method == ORC_ACC &&
        !(mu_start > 0 && m_stage_start >= 1 && j_start >= 0 && j_start < m_stage_start &&
          stages_start >= 0))
        return ORC_BADARG;

    double *x = calloc((size_t)m, sizeof(double));
    double *w = calloc((size_t)m, sizeof(double));
    if (x0) memcpy(x, x0, sizeof(double) * (size_t)m);
    if (w0) memcpy(w, w0, sizeof(double) * (size_t)m);
    double *s = malloc(sizeof(double) * (size_t)m);
    double *c = malloc(sizeof(double) * (size_t)m);
    double *u = malloc(sizeof(double) * (size_t)n);
    double *x1 = malloc(sizeof(double) * (size_t)m);
    double *w1 = malloc(sizeof(double) * (size_t)m);
    double *s1 = malloc(sizeof(double) * (size_t)m);
    double *c1 = malloc(sizeof(double) * (size_t)m);
    double *u1 = malloc(sizeof(double) * (size_t)n);

    memset(res, 0, sizeof(*res));
    res->outer_stages = stages_start;
    int steps = 0, status = ORC_MAXITER;
    double err = orc_sinkhorn_map(p, x, u, c, s);
    steps = 1;
    double dual = orc_dual_after_row_pass(p, u, x);
    record(hist, 0, m, err, dual, 0.0, 0, x, NULL);

    if (method == ORC_PLAIN) {
        for (;;) {
            if (err < tol) { status = ORC_CONVERGED; break; }
            if (steps >= max_steps) break;
            memcpy(x, s, sizeof(double) * (size_t)m);      /* x_{k+1} = S(x_k) */
            err = orc_sinkhorn_map(p, x, u, c, s);
            dual = orc_dual_after_row_pass(p, u, x);
            record(hist, steps, m, err, dual, 0.0, 0, x, NULL);
            ++steps;
        }
    } else {
        double mu = mu_start;
        long m_stage = m_stage_start, j = j_start;
        for (;;) {
            if (err < tol) { status = ORC_CONVERGED; break; }
            if (steps >= max_steps) break;
            double alpha = sqrt(2.0 * mu);
            for (long q = 0; q < m; ++q) x1[q] = (w[q] + s[q]) / (1.0 + alpha);
            double err1 = orc_sinkhorn_map(p, x1, u1, c1, s1);
            for (long q = 0; q < m; ++q)
                w1[q] = (w[q] + (alpha * alpha - 2.0) * x1[q] + 2.0 * s1[q]) /
                        (1.0 + alpha);
            int stab = 0;
            double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (stab_mode != ORC_STAB_OFF) {
                orc_stability_terms(m, p->b, c, c1, x, w, x1, w1, alpha, t);
                stab = (t[4] == 0.0 ? 1 : 0) | (t[5] == 0.0 ? 2 : 0);
                if (stab) {
                    res->stability_failures++;
                    if (stab_mode == ORC_STAB_GATE)
                        for (long q = 0; q < m; ++q) w1[q] = alpha * x1[q];
                }
            }
            double dual1 = orc_dual_after_row_pass(p, u1, x1);
            record(hist, steps, m, err1, dual1, mu, stab, x1, t);
            ++steps;
            double *tp;
            tp = x; x = x1; x1 = tp;
            tp = w; w = w1; w1 = tp;
            tp = s; s = s1; s1 = tp;
            tp = c; c = c1; c1 = tp;
            tp = u; u = u1; u1 = tp;
            err = err1;
            dual = dual1;
            const int back = (stab_mode == ORC_STAB_BACKTRACK) && stab;
            if (++j == m_stage || back) {                 /* Algorithm 2 */
                if (carry_y) {
                    double ratio = sqrt(2.0 * (mu / 2.0)) / alpha;
                    for (long q = 0; q < m; ++q) w[q] *= ratio;
                }
                mu = mu / 2.0;
                m_stage = (long)floor(sqrt(2.0) * (double)m_stage) + 1;
                j = 0;
                res->outer_stages++;
            }
        }
        if (stage_out) {
            stage_out[0] = mu;
            stage_out[1] = (double)m_stage;
            stage_out[2] = (double)j;
            stage_out[3] = (double)res->outer_stages;
        }
    }
    if (x_out) memcpy(x_out, x, sizeof(double) * (size_t)m);
    if (w_out) memcpy(w_out, w, sizeof(double) * (size_t)m);

    for (long i = 0; i < n; ++i) f_out[i] = p->eps * u[i];
    for (long q = 0; q < m; ++q) g_out[q] = p->eps * x[q];
    res->status = status;
    res->sinkhorn_steps = steps;
    res->marginal_l1 = err;
    res->dual = dual;

    free(x); free(w); free(s); free(c); free(u);
    free(x1); free(w1); free(s1); free(c1); free(u1);
    return status;
}

int orc_solve(const orc_problem *p, double tol, int method, double mu0,
              int m0, int max_steps, int stab_mode, int carry_y,
              double *f_out, double *g_out, orc_result *res,
              orc_history *hist)
{
    return orc_solve_from(p, tol, method, mu0, m0, max_steps, stab_mode, carry_y, NULL, NULL,
                          mu0, m0, 0, 0, f_out, g_out, res, hist, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------- */
/* Evaluation of given potentials (cost units) in FP64:                        */
/*   P_ij = exp((f_i + g_j - C_ij) / eps)            (eq. P-from-dual)        */
/* out[0] = ||P 1 - a||_1, out[1] = ||P' 1 - b||_1 (eq. l1tol),               */
/* out[2] = <C, P>, out[3] = dual <f,a> + <g,b> - eps sum P,                   */
/* out[4] = primal <C,P> + eps sum P (log P - 1) (eq. EOT), out[5] = sum P.    */
/* ------------------------------------------------------------------------- */
void orc_evaluate(const orc_cost *c, double eps, const double *a,
                  const double *b, const double *f, const double *g,
                  double *out)
{
    const long n = c->n, m = c->m;
    double *col = calloc((size_t)m, sizeof(double));
    double row_l1 = 0.0, cost = 0.0, mass = 0.0, ent = 0.0;
    for (long i = 0; i < n; ++i) {
        double r = 0.0;
        for (long j = 0; j < m; ++j) {
            double cij = orc_cost_entry(c, i, j);
            double z = (f[i] + g[j] - cij) / eps;
            double pij = exp(z);
            r += pij;
            col[j] += pij;
            cost += cij * pij;
            ent += pij * (z - 1.0);
        }
        row_l1 += fabs(r - a[i]);
        mass += r;
    }
    double col_l1 = 0.0;
    for (long j = 0; j < m; ++j) col_l1 += fabs(col[j] - b[j]);
    double fa = 0.0, gb = 0.0;
    for (long i = 0; i < n; ++i) fa += f[i] * a[i];
    for (long j = 0; j < m; ++j) gb += g[j] * b[j];
    out[0] = row_l1;
    out[1] = col_l1;
    out[2] = cost;
    out[3] = fa + gb - eps * mass;
    out[4] = cost + eps * ent;
    out[5] = mass;
    free(col);
}

/* Both marginal errors of P(f, g) (eq. l1tol) for large problems:
 *   out[0] = ||P 1 - a||_1,  out[1] = ||P' 1 - b||_1,
 * with P_ij = exp((f_i + g_j - C_ij) / eps) (eq. P-from-dual) in FP64, the
 * same quantities as out[0..1] of orc_evaluate. Rows are split over the
 * threads; each thread sums its rows' entries into its own column array and
 * the column arrays are added in thread order. */
void orc_marginal_l1(const orc_cost *c, double eps, const double *a,
                     const double *b, const double *f, const double *g,
                     double *out)
{
    const long n = c->n, m = c->m;
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double *cols = calloc((size_t)nt * (size_t)m, sizeof(double));
    double *rowl1 = calloc((size_t)nt, sizeof(double));
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *col = cols + (size_t)t * (size_t)m;
        double rl = 0.0;
#pragma omp for schedule(static)
        for (long i = 0; i < n; ++i) {
            double r = 0.0;
            for (long j = 0; j < m; ++j) {
                double pij = exp((f[i] + g[j] - orc_cost_entry(c, i, j)) / eps);
                r += pij;
                col[j] += pij;
            }
            rl += fabs(r - a[i]);
        }
        rowl1[t] = rl;
    }
    double row_l1 = 0.0, col_l1 = 0.0;
    for (int t = 0; t < nt; ++t) row_l1 += rowl1[t];
    for (long j = 0; j < m; ++j) {
        double cj = 0.0;
        for (int t = 0; t < nt; ++t) cj += cols[(size_t)t * (size_t)m + j];
        col_l1 += fabs(cj - b[j]);
    }
    out[0] = row_l1;
    out[1] = col_l1;
    free(cols);
    free(rowl1);
}

/* The transport plan P_ij = exp((f_i + g_j - C_ij) / eps) (eq. P-from-dual)
 * of given potentials, n x m row-major. */
void orc_plan(const orc_cost *c, double eps, const double *f, const double *g,
              double *P)
{
    const long n = c->n, m = c->m;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < m; ++j)
            P[i * m + j] = exp((f[i] + g[j] - orc_cost_entry(c, i, j)) / eps);
}

/* Barycentric projection of a feature matrix Z (m x dz, row-major) through the
 * plan: out_i = sum_j P_ij Z_j / sum_j P_ij (Sec. 5, colour transfer maps each
 * source pixel to the plan-weighted mean of the target colours). */
void orc_barycentric(const orc_cost *c, double eps, const double *f,
                     const double *g, const float *Z, long dz, double *out)
{
    const long n = c->n, m = c->m;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double mass = 0.0;
        for (long k = 0; k < dz; ++k) out[i * dz + k] = 0.0;
        for (long j = 0; j < m; ++j) {
            double pij = exp((f[i] + g[j] - orc_cost_entry(c, i, j)) / eps);
            mass += pij;
            for (long k = 0; k < dz; ++k) out[i * dz + k] += pij * (double)Z[j * dz + k];
        }
        for (long k = 0; k < dz; ++k) out[i * dz + k] /= mass;
    }
}

/* Row sums r_i and transport-cost contributions sum_j C_ij P_ij for a list of
 * rows only (for spot checks of large problems). */
void orc_rows_sample(const orc_cost *c, double eps, const double *f,
                     const double *g, const long *rows, long k, double *r_out,
                     double *cost_out)
{
#pragma omp parallel for schedule(static)
    for (long t = 0; t < k; ++t) {
        long i = rows[t];
        double r = 0.0, cs = 0.0;
        for (long j = 0; j < c->m; ++j) {
            double cij = orc_cost_entry(c, i, j);
            double pij = exp((f[i] + g[j] - cij) / eps);
            r += pij;
            cs += cij * pij;
        }
        r_out[t] = r;
        cost_out[t] = cs;
    }
}

/* Column sums c_j for a list of columns only. */
void orc_cols_sample(const orc_cost *c, double eps, const double *f,
                     const double *g, const long *cols, long k, double *c_out)
{
#pragma omp parallel for schedule(static)
    for (long t = 0; t < k; ++t) {
        long j = cols[t];
        double s = 0.0;
        for (long i = 0; i < c->n; ++i)
            s += exp((f[i] + g[j] - orc_cost_entry(c, i, j)) / eps);
        c_out[t] = s;
    }
}

/* Row pass for a list of rows only: u_i for i in rows (for spot checks of a
 * single full-size pass). Same definition as orc_row_pass. */
void orc_row_pass_sample(const orc_cost *c, double eps, const double *loga,
                         const double *x, const long *rows, long k,
                         double *u_out)
{
#pragma omp parallel for schedule(static)
    for (long t = 0; t < k; ++t) {
        long i = rows[t];
        double mx = -INFINITY;
        for (long j = 0; j < c->m; ++j) {
            double z = x[j] - orc_cost_entry(c, i, j) / eps;
            if (z > mx) mx = z;
        }
        double s = 0.0;
        for (long j = 0; j < c->m; ++j)
            s += exp(x[j] - orc_cost_entry(c, i, j) / eps - mx);
        u_out[t] = loga[i] - (mx + log(s));
    }
}

/* Column log-sum-exp for a list of columns only. */
void orc_col_lse_sample(const orc_cost *c, double eps, const double *u,
                        const long *cols, long k, double *ell_out)
{
#pragma omp parallel for schedule(static)
    for (long t = 0; t < k; ++t) {
        long j = cols[t];
        double mx = -INFINITY;
        for (long i = 0; i < c->n; ++i) {
            double z = u[i] - orc_cost_entry(c, i, j) / eps;
            if (z > mx) mx = z;
        }
        double s = 0.0;
        for (long i = 0; i < c->n; ++i)
            s += exp(u[i] - orc_cost_entry(c, i, j) / eps - mx);
        ell_out[t] = mx + log(s);
    }
}

int orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}
