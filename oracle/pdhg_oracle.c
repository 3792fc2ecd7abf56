/*
 * FP64 single-threaded CPU oracle of restarted PDHG for linear programming.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark call this code.  It shares nothing with the CUDA
 * solver: no headers, helpers, tables or kernels.  It is deliberately plain and
 * slow: explicit loops over the CSR matrix, no blocking, no fusion, no
 * reordering beyond what the paper's formulas state.
 *
 * Problem (Section 2.2):  min c^T x  s.t.  G x >= h,  A x = b,  l <= x <= u.
 * K = (G; A) is given row-wise in CSR with a per-row sense flag
 * (sense[i] = 1: row of G, K_i x >= q_i;  sense[i] = 0: row of A, K_i x = q_i),
 * q = (h; b).  Bounds may be +-INFINITY.
 *
 * Function map (paper sections, algorithms, equations):
 *   orc_spmv / orc_spmv_t     products K x and K^T y
 *   orc_ruiz                  Algorithm 3 (Ruiz), Section 2.4.1 change of variables,
 *                             optional Pock-Chambolle pass (parameter alpha)
 *   orc_pc_tune               choice of alpha by trial runs (a reading; not in the paper)
 *   orc_power_norm            Algorithm 2 (spectral norm estimate)
 *   orc_proj_lambda           projection onto Lambda (Section 2.2 dual)
 *   orc_kkt                   termination quantities, Eqs. (term1)-(term3) of
 *                             Section 2.3.2, and the KKT_omega error of Section 2.4.2
 *   orc_pdhg_step             one PDHG step, Algorithm 1 with theta = 1 in the sign
 *                             form of Appendix D (c - K^T y, q - K xbar)
 *   orc_primal_weight         Algorithm 4 (primal weight update, Section 2.4.3)
 *   orc_step_rule             Algorithm 5 (adaptive step size: eta_bar, eta', accept)
 *   orc_solve                 Algorithm 1 + restarts (Section 2.4.2), primal weight
 *                             (Section 2.4.3, Algorithm 4), adaptive step
 *                             (Algorithm 5), termination (Section 2.3.2)
 *   orc_infeasibility         Algorithm 6 (infeasibility detection, Section 2.4.5)
 *   orc_pnorm2 /
 *   orc_halpern_step /
 *   orc_solve_halpern         restarted (reflected) Halpern PDHG, the variant the
 *                             Conclusion names as future work (Lu and Yang, 2024)
 *   orc_fishnet               Algorithm 7 (fishnet casting, Section 2.5)
 *   orc_unrolled_forward /
 *   orc_unrolled_adjoint      K fixed-step iterations and their exact reverse-mode
 *                             derivative (the paper names autodiff only; the reverse
 *                             equations follow from Appendix D's step by the chain rule)
 *
 * Readings where the paper is silent or garbled are marked "reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t m, n;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const double* vals;
    const uint8_t* sense;
    const double* c;
    const double* q;
    const double* l;
    const double* u;
} orc_lp;

typedef struct {
    double tol;               /* epsilon of Section 2.3.2 */
    int64_t max_iters;        /* accepted PDHG iterations */
    int32_t check_every;      /* reading: the paper's "a set number" of iterations */
    int32_t ruiz_iters;       /* N_iter of Algorithm 3 (0 = no scaling) */
    double ruiz_tol;          /* "converged to 1 within tolerance" */
    int32_t pock_chambolle;   /* reading: 1 = one Pock-Chambolle pass (pc_alpha) after Ruiz;
                                 2 = pick alpha from {0, 1/2, 1, 2} by trial runs (orc_pc_tune) */
    int32_t power_iters;      /* N_iter of Algorithm 2 */
    int32_t adaptive_step;    /* Algorithm 5 on/off */
    int32_t primal_weight_update; /* Algorithm 4 on/off */
    int32_t restarts;         /* Section 2.4.2 on/off */
    double eta_scale;         /* eta = eta_scale / ||K||_2 (0.9, Section 3.2) */
    double beta_sufficient, beta_necessary, beta_artificial;
    double eps_zero;          /* 1e-6 */
    const double* x0;         /* optional warm start, unscaled (NULL: x = proj_X(0)) */
    const double* y0;         /* optional warm start, unscaled (NULL: y = 0) */
    double omega0;            /* > 0: use instead of InitializePrimalWeight */
    double eta0;              /* > 0: use instead of eta_scale / ||K||_2 */
    int32_t infeas_detect;    /* Algorithm 6 at every check */
    int32_t pad;
    double infeas_tol;        /* tol of Algorithm 6 */
    int32_t halpern;          /* 1: the restarted Halpern variant (orc_solve_halpern) */
    int32_t pad2;
    double reflect;           /* rho in [0, 1] of the Halpern variant */
    double pc_alpha;          /* alpha of the Pock-Chambolle pass (pock_chambolle = 1) */
    int32_t pc_trial_iters;   /* pock_chambolle = 2: iterations of each trial (0: 2 check_every) */
    int32_t pad3;
    /* replay (test use): the attempt records of another run (ORC_ATTEMPT_FIELDS
     * doubles each); attempt a of this run takes its step size ([1]) and its
     * accept / reject outcome ([4]) from record a, while eta_bar and eta' are
     * still computed here and logged.  NULL: off. */
    const double* replay;
    int64_t replay_len;
    /* replay of checks (test use): record c (2 doubles) gives check c's restart
     * decision ([0]) and candidate choice ([1], 1 = the average) as another run
     * took them; this run follows them and logs its own (orc_trace).  NULL: off. */
    const double* replay_checks;
    int64_t replay_checks_len;
} orc_opts;

typedef struct {
    int32_t status;           /* 1 optimal, 2 primal infeasible, 3 dual infeasible, 4 iteration limit */
    int32_t pad;
    int64_t iters;            /* accepted iterations */
    int64_t attempts;         /* step attempts (accepted + rejected) */
    int64_t restarts;
    double pobj, dobj, rel_gap, rel_pres, rel_dres;
    double omega, eta, norm_K;
    double pc_alpha;          /* alpha of the Pock-Chambolle pass used (NaN: no pass) */
} orc_info;

#define ORC_ATTEMPT_FIELDS 9

/* One record per termination / restart check.  fpr and fpr0: the Halpern
 * variant's fixed-point residual of the last iteration and of its epoch's first
 * iteration (0 for restarted PDHG). */
typedef struct {
    double k, attempts, restart, cand_is_avg, omega, eta;
    double kkt_cur, kkt_avg, rel_gap, rel_pres, rel_dres, kkt_cand;
    double fpr, fpr0;
    /* this run's own restart decision and candidate choice (they differ from
     * restart / cand_is_avg only under a replay of checks), and the two KKT
     * values the restart criteria compared the candidate with: the last
     * restart's candidate and the previous check's (+inf after a restart; NaN
     * for the Halpern variant, whose criteria use fpr and fpr0) */
    double own_restart, own_cand_is_avg, kkt_anchor, kkt_prev;
} orc_trace;

/* ------------------------------------------------------------------ */
/* basic linear algebra                                                */
/* ------------------------------------------------------------------ */

/* out = K x  (row-wise CSR product) */
void orc_spmv(const orc_lp* lp, const double* vals, const double* x, double* out)
{
    for (int64_t i = 0; i < lp->m; ++i) {
        double s = 0.0;
        for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
            s += vals[p] * x[lp->col_idx[p]];
        out[i] = s;
    }
}

/* out = K^T y  (scatter over the rows of K; no transposed copy) */
void orc_spmv_t(const orc_lp* lp, const double* vals, const double* y, double* out)
{
    for (int64_t j = 0; j < lp->n; ++j) out[j] = 0.0;
    for (int64_t i = 0; i < lp->m; ++i)
        for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
            out[lp->col_idx[p]] += vals[p] * y[i];
}

static double dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

static double clamp(double v, double lo, double hi)
{
    if (v < lo) return lo;
    if (v > hi) return hi;
    return v;
}

/* ------------------------------------------------------------------ */
/* Algorithm 3: Ruiz scaling (+ optional Pock-Chambolle pass)          */
/* ------------------------------------------------------------------ */

/*
 * Produces the scaled matrix vals_s and the accumulated diagonal factors
 * R (length m) and C (length n) with  K~ = diag(R) K diag(C).
 * In the paper's notation D_r = diag(R)^-1 and D_c = diag(C)^-1, so that
 * K~ = D_r^-1 K D_c^-1, x~ = D_c x = x / C, c~ = D_c^-1 c = C c, q~ = R q
 * (Section 2.4.1); bounds follow x: l~ = l / C, u~ = u / C.
 *
 * Each pass takes both factor sets from the current K~ (row and column
 * infinity norms), then rescales.  reading: the loop stops before a pass when
 * every non-empty row's and column's infinity norm is within ruiz_tol of 1
 * (the same set of passes as testing after each update); an empty row or
 * column keeps factor 1.  Returns the number of passes applied.
 */
/* |a|^e of a stored value for the Pock-Chambolle sums; |a|^0 is 1 for a
 * nonzero a and 0 for a stored zero (the sums run over the nonzeros of K). */
static double pc_pow(double a, double e)
{
    a = fabs(a);
    if (e == 0.0) return a != 0.0 ? 1.0 : 0.0;
    return pow(a, e);
}

int orc_ruiz(const orc_lp* lp, int32_t iters, double tol, int32_t pock_chambolle,
             double pc_alpha, double* vals_s, double* R, double* C)
{
    const int64_t m = lp->m, n = lp->n, nnz = lp->row_ptr[m];
    double* rn = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* cn = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(vals_s, lp->vals, sizeof(double) * (size_t)nnz);
    for (int64_t i = 0; i < m; ++i) R[i] = 1.0;
    for (int64_t j = 0; j < n; ++j) C[j] = 1.0;
    int passes = 0;
    for (int32_t it = 0; it < iters; ++it) {
        for (int64_t i = 0; i < m; ++i) rn[i] = 0.0;
        for (int64_t j = 0; j < n; ++j) cn[j] = 0.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p) {
                double a = fabs(vals_s[p]);
                if (a > rn[i]) rn[i] = a;
                if (a > cn[lp->col_idx[p]]) cn[lp->col_idx[p]] = a;
            }
        double dev = 0.0;
        for (int64_t i = 0; i < m; ++i)
            if (rn[i] > 0.0 && fabs(1.0 - rn[i]) > dev) dev = fabs(1.0 - rn[i]);
        for (int64_t j = 0; j < n; ++j)
            if (cn[j] > 0.0 && fabs(1.0 - cn[j]) > dev) dev = fabs(1.0 - cn[j]);
        if (dev <= tol) break;
        for (int64_t i = 0; i < m; ++i) rn[i] = rn[i] > 0.0 ? 1.0 / sqrt(rn[i]) : 1.0;
        for (int64_t j = 0; j < n; ++j) cn[j] = cn[j] > 0.0 ? 1.0 / sqrt(cn[j]) : 1.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
                vals_s[p] = vals_s[p] * rn[i] * cn[lp->col_idx[p]];
        for (int64_t i = 0; i < m; ++i) R[i] *= rn[i];
        for (int64_t j = 0; j < n; ++j) C[j] *= cn[j];
        ++passes;
    }
    if (pock_chambolle) {
        /* reading (the pass is not in the paper; Pock and Chambolle, 2011):
         * rows by 1 / sqrt(sum_j |K~_ij|^(2 - alpha)), columns by
         * 1 / sqrt(sum_i |K~_ij|^alpha), from the Ruiz-scaled K~ */
        for (int64_t i = 0; i < m; ++i) rn[i] = 0.0;
        for (int64_t j = 0; j < n; ++j) cn[j] = 0.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p) {
                rn[i] += pc_pow(vals_s[p], 2.0 - pc_alpha);
                cn[lp->col_idx[p]] += pc_pow(vals_s[p], pc_alpha);
            }
        for (int64_t i = 0; i < m; ++i) rn[i] = rn[i] > 0.0 ? 1.0 / sqrt(rn[i]) : 1.0;
        for (int64_t j = 0; j < n; ++j) cn[j] = cn[j] > 0.0 ? 1.0 / sqrt(cn[j]) : 1.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
                vals_s[p] = vals_s[p] * rn[i] * cn[lp->col_idx[p]];
        for (int64_t i = 0; i < m; ++i) R[i] *= rn[i];
        for (int64_t j = 0; j < n; ++j) C[j] *= cn[j];
    }
    free(rn);
    free(cn);
    return passes;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2: spectral norm by power iteration                       */
/* ------------------------------------------------------------------ */

double orc_power_norm(const orc_lp* lp, const double* vals, int32_t iters)
{
    const int64_t m = lp->m, n = lp->n;
    double* b = (double*)malloc(sizeof(double) * (size_t)n);
    double* t = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < n; ++j) b[j] = 1.0;
    for (int32_t it = 0; it < iters; ++it) {
        orc_spmv(lp, vals, b, t);
        orc_spmv_t(lp, vals, t, b);
        double nb = nrm2(n, b);
        if (nb == 0.0) break;
        for (int64_t j = 0; j < n; ++j) b[j] /= nb;
    }
    orc_spmv(lp, vals, b, t);
    double r = nrm2(m, t);
    free(b);
    free(t);
    return r;
}

/* ------------------------------------------------------------------ */
/* dual multipliers and the KKT quantities (Sections 2.2, 2.3.2, 2.4.2) */
/* ------------------------------------------------------------------ */

/* lambda = proj_Lambda(v): Lambda_i = {0} (free), R^- (only u finite),
 * R^+ (only l finite), R (both finite). */
void orc_proj_lambda(int64_t n, const double* l, const double* u, const double* v,
                     double* lam)
{
    for (int64_t j = 0; j < n; ++j) {
        int lf = isfinite(l[j]), uf = isfinite(u[j]);
        if (!lf && !uf) lam[j] = 0.0;
        else if (!lf) lam[j] = v[j] < 0.0 ? v[j] : 0.0;
        else if (!uf) lam[j] = v[j] > 0.0 ? v[j] : 0.0;
        else lam[j] = v[j];
    }
}

/*
 * KKT quantities of (x, y) for the LP with matrix values ``vals`` and vectors
 * c, q, l, u (scaled or not, whichever the caller passes).
 * out[0] pobj = c^T x
 * out[1] dobj = q^T y + l^T lambda^+ + u^T lambda^-   (a term is 0 when its
 *        lambda part is 0: reading of 0 * inf for infinite bounds)
 * out[2] ||(Ax - b, [h - Gx]^+)||_2   primal residual norm
 * out[3] ||c - K^T y - lambda||_2     dual residual norm
 * out[4] rel_gap   (term1)  |dobj - pobj| / (1 + |dobj| + |pobj|)
 * out[5] rel_pres  (term2)  out[2] / (1 + ||q||_2)
 * out[6] rel_dres  (term3)  out[3] / (1 + ||c||_2)
 * out[7] KKT_omega (Section 2.4.2) = sqrt(w^2 out[2]^2 + out[3]^2 / w^2 + (dobj - pobj)^2)
 */
void orc_kkt(const orc_lp* lp, const double* vals, const double* c, const double* q,
             const double* l, const double* u, const double* x, const double* y,
             double omega, double* out)
{
    const int64_t m = lp->m, n = lp->n;
    double* Kx = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    double* lam = (double*)malloc(sizeof(double) * (size_t)n);
    orc_spmv(lp, vals, x, Kx);
    double pres2 = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double r = q[i] - Kx[i];             /* h - Gx or b - Ax */
        if (lp->sense[i]) r = r > 0.0 ? r : 0.0;  /* [h - Gx]^+ */
        pres2 += r * r;
    }
    orc_spmv_t(lp, vals, y, v);
    for (int64_t j = 0; j < n; ++j) v[j] = c[j] - v[j];   /* c - K^T y */
    orc_proj_lambda(n, l, u, v, lam);
    double dres2 = 0.0, lterm = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double r = v[j] - lam[j];
        dres2 += r * r;
        if (lam[j] > 0.0) lterm += l[j] * lam[j];
        if (lam[j] < 0.0) lterm += u[j] * lam[j];
    }
    double pobj = dot(n, c, x);
    double dobj = dot(m, q, y) + lterm;
    double gap = dobj - pobj;
    out[0] = pobj;
    out[1] = dobj;
    out[2] = sqrt(pres2);
    out[3] = sqrt(dres2);
    out[4] = fabs(gap) / (1.0 + fabs(dobj) + fabs(pobj));
    out[5] = out[2] / (1.0 + nrm2(m, q));
    out[6] = out[3] / (1.0 + nrm2(n, c));
    out[7] = sqrt(omega * omega * pres2 + dres2 / (omega * omega) + gap * gap);
    free(Kx);
    free(v);
    free(lam);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (theta = 1), sign form of Appendix D                    */
/* ------------------------------------------------------------------ */

/*
 * x' = proj_X(x - tau (c - K^T y))
 * y' = proj_Y(y + sigma (q - K (2 x' - x)))
 * proj_X clamps to [l, u]; proj_Y clamps inequality rows at 0 (Appendix C).
 */
void orc_pdhg_step(const orc_lp* lp, const double* vals, const double* c, const double* q,
                   const double* l, const double* u, const double* x, const double* y,
                   double tau, double sigma, double* xn, double* yn)
{
    const int64_t m = lp->m, n = lp->n;
    double* KTy = (double*)malloc(sizeof(double) * (size_t)n);
    double* xbar = (double*)malloc(sizeof(double) * (size_t)n);
    double* Kxb = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    orc_spmv_t(lp, vals, y, KTy);
    for (int64_t j = 0; j < n; ++j) {
        xn[j] = clamp(x[j] - tau * (c[j] - KTy[j]), l[j], u[j]);
        xbar[j] = 2.0 * xn[j] - x[j];
    }
    orc_spmv(lp, vals, xbar, Kxb);
    for (int64_t i = 0; i < m; ++i) {
        double v = y[i] + sigma * (q[i] - Kxb[i]);
        if (lp->sense[i] && v < 0.0) v = 0.0;
        yn[i] = v;
    }
    free(KTy);
    free(xbar);
    free(Kxb);
}

/* ------------------------------------------------------------------ */
/* Algorithm 6: infeasibility detection from iterate differences       */
/* ------------------------------------------------------------------ */

/*
 * dx, dy: differences of consecutive iterates (unscaled); dlam: difference of
 * lambda = proj_Lambda(c - K^T y) between the two dual iterates.  The tests are
 * applied to the directions dx / ||dx|| and (dy, dlam) / ||(dy, dlam)||
 * (reading: a certificate is a direction; with the listing's absolute tol the
 * short steps of a converging feasible problem pass the dual test).
 * Dual infeasibility (certificate dx, Section 2.4.5):
 *   ||A v|| <= tol, min(G v) >= -tol, c^T v <= -tol, v_i in V_i within tol
 *   (V_i = R free, R^- only u finite, R^+ only l finite, {0} both finite).
 * Primal infeasibility (certificate dy, with the paper's v_lambda = -dlam, since
 * lambda = c - K^T y up to the projection):
 *   ||K^T w + dl|| <= tol, min(w_ineq) >= -tol,
 *   psi = q^T w + l^T dl^+ + u^T dl^- > tol   (reading: the listing's
 *   "psi >= -tol" would hold at every converging iterate; the certificate of
 *   Section 2.4.5 needs psi > 0), (w, dl) the normalised (dy, dlam).
 * terms (8 doubles, may be NULL): ||A v||, min(G v), c^T v, max distance of v
 * to V, ||K^T w + dl||, min(w_ineq), psi, 0 (all of the normalised directions).
 * Returns 3 (dual infeasible), 2 (primal infeasible) or 0.
 */
int orc_infeasibility(const orc_lp* lp, const double* dx, const double* dy, const double* dlam,
                      double tol, double* terms)
{
    const int64_t m = lp->m, n = lp->n;
    double* Kdx = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double* KTdy = (double*)calloc((size_t)n, sizeof(double));
    orc_spmv(lp, lp->vals, dx, Kdx);
    orc_spmv_t(lp, lp->vals, dy, KTdy);
    double adx2 = 0.0, gmin = INFINITY, ymin = INFINITY, psi = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        if (lp->sense[i]) {
            if (Kdx[i] < gmin) gmin = Kdx[i];
            if (dy[i] < ymin) ymin = dy[i];
        } else {
            adx2 += Kdx[i] * Kdx[i];
        }
        psi += lp->q[i] * dy[i];
    }
    double cdx = 0.0, vviol = 0.0, r2 = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        cdx += lp->c[j] * dx[j];
        const int lf = isfinite(lp->l[j]), uf = isfinite(lp->u[j]);
        double v = 0.0;
        if (lf && uf) v = fabs(dx[j]);
        else if (lf) v = dx[j] < 0.0 ? -dx[j] : 0.0;
        else if (uf) v = dx[j] > 0.0 ? dx[j] : 0.0;
        if (v > vviol) vviol = v;
        const double r = KTdy[j] + dlam[j];
        r2 += r * r;
        if (dlam[j] > 0.0) psi += lp->l[j] * dlam[j];
        if (dlam[j] < 0.0) psi += lp->u[j] * dlam[j];
    }
    if (gmin == INFINITY) gmin = 0.0;
    if (ymin == INFINITY) ymin = 0.0;
    const double nx = sqrt(dot(n, dx, dx));
    const double ny = sqrt(dot(m, dy, dy) + dot(n, dlam, dlam));
    const double sx = nx > 0.0 ? 1.0 / nx : 0.0, sy = ny > 0.0 ? 1.0 / ny : 0.0;
    const double t[7] = {sqrt(adx2) * sx, gmin * sx, cdx * sx, vviol * sx,
                         sqrt(r2) * sy, ymin * sy, psi * sy};
    if (terms) {
        for (int q = 0; q < 7; ++q) terms[q] = t[q];
        terms[7] = 0.0;
    }
    free(Kdx);
    free(KTdy);
    if (nx > 0.0 && t[0] <= tol && t[1] >= -tol && t[2] <= -tol && t[3] <= tol) return 3;
    if (ny > 0.0 && t[4] <= tol && t[5] >= -tol && t[6] > tol) return 2;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Algorithm 4 and Algorithm 5 as functions of their scalar inputs     */
/* ------------------------------------------------------------------ */

/*
 * Algorithm 4 (primal weight update at a restart, Section 2.4.3).
 * dx = ||x_new_anchor - x_old_anchor||_2, dy = ||y_new_anchor - y_old_anchor||_2.
 * reading: the printed ratio log(dy / dy) is garbled; the update is the
 * log-space average (smoothing 1/2) of the old weight and dy / dx, and it is
 * skipped when either distance is at most eps_zero.
 */
double orc_primal_weight(double omega, double dx, double dy, double eps_zero)
{
    if (dx > eps_zero && dy > eps_zero)
        return exp(0.5 * log(dy / dx) + 0.5 * log(omega));
    return omega;
}

/*
 * Algorithm 5 (adaptive step size): one attempt taken with step eta and primal
 * weight omega moved the iterate by (dx, dy); dx2 = ||dx||^2, dy2 = ||dy||^2,
 * inter = dy^T K dx.
 *   eta_bar  = ||(dx, dy)||_omega^2 / (2 |inter|), ||(dx, dy)||_omega^2 = omega dx2 + dy2 / omega
 *              (+infinity when inter = 0)
 *   eta'     = min((1 - (k + 1)^-0.3) eta_bar, (1 + (k + 1)^-0.6) eta)
 *   accepted when eta <= eta_bar.
 * reading: the paper's k is the 1-based index of the iteration being taken, so
 * with `accepted` iterations done so far k = accepted + 1 and the base of the
 * two powers is accepted + 2 (with a 0-based k the first step would get
 * eta' = 0).  Returns 1 when the attempt is accepted; writes eta_bar and eta'.
 */
int orc_step_rule(double eta, double omega, double dx2, double dy2, double inter,
                  int64_t accepted, double* eta_bar_out, double* eta_next_out)
{
    const double movement = omega * dx2 + dy2 / omega;
    const double eta_bar = inter != 0.0 ? movement / (2.0 * fabs(inter)) : INFINITY;
    const double kp1 = (double)accepted + 2.0;
    const double e1 = (1.0 - pow(kp1, -0.3)) * eta_bar;
    const double e2 = (1.0 + pow(kp1, -0.6)) * eta;
    *eta_bar_out = eta_bar;
    *eta_next_out = e1 < e2 ? e1 : e2;
    return eta <= eta_bar;
}

/* ------------------------------------------------------------------ */
/* the restarted, adaptive solver                                      */
/* ------------------------------------------------------------------ */

static void* xalloc(int64_t count) { return calloc((size_t)(count > 0 ? count : 1), sizeof(double)); }

/*
 * Restarted PDHG.  Returns the status (1 optimal, 4 iteration limit) and
 * writes the unscaled candidate solution to x_out, y_out.
 *
 * Steps, in the paper's order:
 *  1. Ruiz (Algorithm 3) -> K~, c~, q~, l~, u~.
 *  2. ||K~||_2 by Algorithm 2; eta = 0.9 / ||K~||_2 (Section 3.2);
 *     reading: eta = 1 when K~ = 0.
 *  3. omega = ||c~|| / ||q~|| if both exceed eps_zero, else 1 (Section 2.4.3).
 *  4. Start (reading): x = proj_X(0), y = 0; the restart anchor is the start.
 *  5. Each iteration takes a step of Algorithm 1 (fixed eta), or of Algorithm 5
 *     (adaptive eta; reading: its k is the 1-based index of the iteration being
 *     taken, i.e. accepted iterations so far + 1).  Accepted iterates enter the
 *     eta-weighted averages (Section 2.4.2).
 *  6. At the start and every check_every accepted iterations (and at max_iters):
 *     (optionally) Algorithm 6 on the last step's differences;
 *     KKT_omega of the current point and of the average on the scaled problem
 *     (reading); candidate = current if strictly better, else average;
 *     termination (Section 2.3.2) on the unscaled candidate: all three
 *     relative errors <= tol; then the three restart criteria; at a restart the
 *     iterate becomes the candidate, omega is updated by Algorithm 4 (reading:
 *     ratio Delta_y / Delta_x, smoothing 1/2) and the averages are reset.
 */
int orc_solve_halpern(const orc_lp* lp, const orc_opts* o, double* x_out, double* y_out,
                      orc_info* info, orc_trace* trace, int64_t trace_cap, int64_t* trace_len);

/*
 * alog (optional, alog_cap records of ORC_ATTEMPT_FIELDS doubles): one record
 * per step attempt, [0] accepted iterations before the attempt, [1] eta tried,
 * [2] eta_bar, [3] eta', [4] accepted (1/0), [5] omega, [6] ||dx||^2,
 * [7] ||dy||^2, [8] dy^T K dx (NaN in [2], [6..8] for fixed steps); *alog_len
 * receives the number of attempts (may exceed alog_cap).  Scaled problem.
 */
int orc_solve_logged(const orc_lp* lp, const orc_opts* o, double* x_out, double* y_out,
                     orc_info* info, orc_trace* trace, int64_t trace_cap, int64_t* trace_len,
                     double* alog, int64_t alog_cap, int64_t* alog_len);

int orc_solve(const orc_lp* lp, const orc_opts* o, double* x_out, double* y_out,
              orc_info* info, orc_trace* trace, int64_t trace_cap, int64_t* trace_len)
{
    return orc_solve_logged(lp, o, x_out, y_out, info, trace, trace_cap, trace_len, NULL, 0, NULL);
}

/*
 * Choice of the Pock-Chambolle alpha (pock_chambolle = 2).  reading: the paper
 * has no such pass; the rule is ours.  For each alpha of the grid
 * {0, 1/2, 1, 2}, in that order, a trial solve with that pass (all other
 * options as given, infeasibility detection off, no tolerance) runs
 * pc_trial_iters accepted iterations (0: 2 check_every) from the start point;
 * its last check's relative KKT error, max(rel_gap, rel_pres, rel_dres) of
 * Section 2.3.2 on the unscaled problem, is errs[g].  The alpha with the
 * smallest error wins (ties and NaN: the earlier one).  All trials start from
 * the same unscaled point, so equal starting errors make the ends comparable.
 */
#define ORC_PC_GRID 4
static const double kPcGrid[ORC_PC_GRID] = {0.0, 0.5, 1.0, 2.0};

double orc_pc_tune(const orc_lp* lp, const orc_opts* o, double* errs)
{
    const int64_t trial = o->pc_trial_iters > 0 ? o->pc_trial_iters : 2 * (int64_t)o->check_every;
    double* x = (double*)malloc(sizeof(double) * (size_t)(lp->n > 0 ? lp->n : 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)(lp->m > 0 ? lp->m : 1));
    double best = kPcGrid[0], best_err = INFINITY;
    for (int g = 0; g < ORC_PC_GRID; ++g) {
        orc_opts t = *o;
        t.pock_chambolle = 1;
        t.pc_alpha = kPcGrid[g];
        t.max_iters = trial;
        t.tol = 0.0;
        t.infeas_detect = 0;
        orc_info inf;
        orc_solve_logged(lp, &t, x, y, &inf, NULL, 0, NULL, NULL, 0, NULL);
        double e = inf.rel_gap;
        if (inf.rel_pres > e) e = inf.rel_pres;
        if (inf.rel_dres > e) e = inf.rel_dres;
        if (errs) errs[g] = e;
        if (e < best_err) {
            best_err = e;
            best = kPcGrid[g];
        }
    }
    free(x);
    free(y);
    return best;
}

int orc_solve_logged(const orc_lp* lp, const orc_opts* o, double* x_out, double* y_out,
                     orc_info* info, orc_trace* trace, int64_t trace_cap, int64_t* trace_len,
                     double* alog, int64_t alog_cap, int64_t* alog_len)
{
    if (o->pock_chambolle == 2) {
        orc_opts t = *o;
        t.pock_chambolle = 1;
        t.pc_alpha = orc_pc_tune(lp, o, NULL);
        return orc_solve_logged(lp, &t, x_out, y_out, info, trace, trace_cap, trace_len, alog,
                                alog_cap, alog_len);
    }
    if (o->halpern) return orc_solve_halpern(lp, o, x_out, y_out, info, trace, trace_cap, trace_len);
    int64_t al = 0;   /* attempts logged */
    const int64_t m = lp->m, n = lp->n, nnz = lp->row_ptr[m];
    double* vs = (double*)xalloc(nnz);
    double* R = (double*)xalloc(m);
    double* C = (double*)xalloc(n);
    double *cs = (double*)xalloc(n), *qs = (double*)xalloc(m);
    double *ls = (double*)xalloc(n), *us = (double*)xalloc(n);
    double *x = (double*)xalloc(n), *y = (double*)xalloc(m);
    double *xn = (double*)xalloc(n), *yn = (double*)xalloc(m);
    double *xsum = (double*)xalloc(n), *ysum = (double*)xalloc(m);
    double *xa = (double*)xalloc(n), *ya = (double*)xalloc(m);
    double *xanc = (double*)xalloc(n), *yanc = (double*)xalloc(m);
    double *dx = (double*)xalloc(n), *Kdx = (double*)xalloc(m);
    double *xu = (double*)xalloc(n), *yu = (double*)xalloc(m);
    double *xp = (double*)xalloc(n), *yp = (double*)xalloc(m);     /* previous iterate */
    double *ddx = (double*)xalloc(n), *ddy = (double*)xalloc(m), *dlam = (double*)xalloc(n);
    double *lam1 = (double*)xalloc(n), *tmpn = (double*)xalloc(n);
    double kc[8], ka[8], kk[8];
    int64_t tl = 0;

    /* 1. preconditioning */
    orc_ruiz(lp, o->ruiz_iters, o->ruiz_tol, o->pock_chambolle, o->pc_alpha, vs, R, C);
    for (int64_t j = 0; j < n; ++j) {
        cs[j] = C[j] * lp->c[j];
        ls[j] = lp->l[j] / C[j];
        us[j] = lp->u[j] / C[j];
    }
    for (int64_t i = 0; i < m; ++i) qs[i] = R[i] * lp->q[i];

    /* 2. step size */
    double normK = orc_power_norm(lp, vs, o->power_iters);
    double eta = normK > 0.0 ? o->eta_scale / normK : 1.0;
    if (o->eta0 > 0.0) eta = o->eta0;

    /* 3. primal weight */
    double nc = nrm2(n, cs), nq = nrm2(m, qs);
    double omega = (nc > o->eps_zero && nq > o->eps_zero) ? nc / nq : 1.0;
    if (o->omega0 > 0.0) omega = o->omega0;

    /* 4. start */
    for (int64_t j = 0; j < n; ++j) {
        double x0 = o->x0 ? o->x0[j] / C[j] : 0.0;
        x[j] = clamp(x0, ls[j], us[j]);
    }
    for (int64_t i = 0; i < m; ++i) {
        double y0 = o->y0 ? o->y0[i] / R[i] : 0.0;
        if (lp->sense[i] && y0 < 0.0) y0 = 0.0;
        y[i] = y0;
    }
    memcpy(xanc, x, sizeof(double) * (size_t)n);
    memcpy(yanc, y, sizeof(double) * (size_t)m);
    double wsum = 0.0;
    double kkt_anchor = 0.0, kkt_prev = INFINITY;
    int64_t k = 0, attempts = 0, epoch_k = 0, nrestarts = 0;
    int status = 0;
    int first = 1;
    double rel[3] = {0, 0, 0}, pobj = 0, dobj = 0;

    for (;;) {
        int do_check = first || (k % o->check_every == 0) || (k >= o->max_iters);
        if (do_check) {
            /* 6. KKT of current and average on the scaled problem */
            orc_kkt(lp, vs, cs, qs, ls, us, x, y, omega, kc);
            double kkt_avg = INFINITY;
            if (wsum > 0.0) {
                for (int64_t j = 0; j < n; ++j) xa[j] = xsum[j] / wsum;
                for (int64_t i = 0; i < m; ++i) ya[i] = ysum[i] / wsum;
                orc_kkt(lp, vs, cs, qs, ls, us, xa, ya, omega, ka);
                kkt_avg = ka[7];
            }
            const int cand_own = !(kc[7] < kkt_avg);
            const double* rc = (o->replay_checks && tl < o->replay_checks_len)
                                   ? o->replay_checks + 2 * tl : NULL;
            int cand_avg = rc ? (rc[1] != 0.0 && wsum > 0.0) : cand_own;
            const double* xc = cand_avg ? xa : x;
            const double* yc = cand_avg ? ya : y;
            double kkt_c = cand_avg ? kkt_avg : kc[7];
            /* termination on the unscaled candidate (Section 2.3.2) */
            for (int64_t j = 0; j < n; ++j) xu[j] = C[j] * xc[j];
            for (int64_t i = 0; i < m; ++i) yu[i] = R[i] * yc[i];
            orc_kkt(lp, lp->vals, lp->c, lp->q, lp->l, lp->u, xu, yu, omega, kk);
            rel[0] = kk[4]; rel[1] = kk[5]; rel[2] = kk[6];
            pobj = kk[0]; dobj = kk[1];
            int converged = rel[0] <= o->tol && rel[1] <= o->tol && rel[2] <= o->tol;
            int infeasible = 0;
            if (!converged && !first && o->infeas_detect && k > 0) {
                /* Algorithm 6 on the last step's differences, unscaled:
                 * dx = C (x - x_prev), dy = R (y - y_prev), dlam from proj_Lambda(c - K^T y) */
                for (int64_t j = 0; j < n; ++j) ddx[j] = C[j] * (x[j] - xp[j]);
                for (int64_t i = 0; i < m; ++i) ddy[i] = R[i] * (y[i] - yp[i]);
                for (int64_t i = 0; i < m; ++i) yu[i] = R[i] * y[i];
                orc_spmv_t(lp, lp->vals, yu, tmpn);
                for (int64_t j = 0; j < n; ++j) tmpn[j] = lp->c[j] - tmpn[j];
                orc_proj_lambda(n, lp->l, lp->u, tmpn, lam1);
                for (int64_t i = 0; i < m; ++i) yu[i] = R[i] * yp[i];
                orc_spmv_t(lp, lp->vals, yu, tmpn);
                for (int64_t j = 0; j < n; ++j) tmpn[j] = lp->c[j] - tmpn[j];
                orc_proj_lambda(n, lp->l, lp->u, tmpn, dlam);
                for (int64_t j = 0; j < n; ++j) dlam[j] = lam1[j] - dlam[j];
                infeasible = orc_infeasibility(lp, ddx, ddy, dlam, o->infeas_tol, NULL);
                /* yu is rebuilt for the output below */
                for (int64_t i = 0; i < m; ++i) yu[i] = R[i] * yc[i];
            }
            int restart = 0;
            const double anchor_before = first ? kkt_c : kkt_anchor, prev_before = kkt_prev;
            if (first) {
                kkt_anchor = kkt_c;
            } else if (!converged && !infeasible && o->restarts) {
                int crit1 = kkt_c <= o->beta_sufficient * kkt_anchor;
                int crit2 = kkt_c <= o->beta_necessary * kkt_anchor && kkt_c > kkt_prev;
                int crit3 = (double)epoch_k > o->beta_artificial * (double)k;
                restart = crit1 || crit2 || crit3;
            }
            const int restart_own = restart;
            if (rc && !first) restart = rc[0] != 0.0;
            if (restart) {
                if (cand_avg) {
                    memcpy(x, xa, sizeof(double) * (size_t)n);
                    memcpy(y, ya, sizeof(double) * (size_t)m);
                }
                if (o->primal_weight_update) {
                    /* Algorithm 4 */
                    double ddx = 0.0, ddy = 0.0;
                    for (int64_t j = 0; j < n; ++j) ddx += (x[j] - xanc[j]) * (x[j] - xanc[j]);
                    for (int64_t i = 0; i < m; ++i) ddy += (y[i] - yanc[i]) * (y[i] - yanc[i]);
                    ddx = sqrt(ddx);
                    ddy = sqrt(ddy);
                    omega = orc_primal_weight(omega, ddx, ddy, o->eps_zero);
                }
                memcpy(xanc, x, sizeof(double) * (size_t)n);
                memcpy(yanc, y, sizeof(double) * (size_t)m);
                kkt_anchor = kkt_c;
                kkt_prev = INFINITY;
                epoch_k = 0;
                wsum = 0.0;
                memset(xsum, 0, sizeof(double) * (size_t)n);
                memset(ysum, 0, sizeof(double) * (size_t)m);
                ++nrestarts;
            } else if (!first) {
                kkt_prev = kkt_c;
            }
            if (trace && tl < trace_cap) {
                orc_trace* t = &trace[tl];
                t->k = (double)k; t->attempts = (double)attempts; t->restart = restart;
                t->cand_is_avg = cand_avg; t->omega = omega; t->eta = eta;
                t->kkt_cur = kc[7]; t->kkt_avg = kkt_avg;
                t->rel_gap = rel[0]; t->rel_pres = rel[1]; t->rel_dres = rel[2];
                t->kkt_cand = kkt_c;
                t->fpr = 0.0; t->fpr0 = 0.0;
                t->own_restart = restart_own; t->own_cand_is_avg = cand_own;
                t->kkt_anchor = anchor_before; t->kkt_prev = prev_before;
            }
            ++tl;
            if (converged || infeasible || k >= o->max_iters) {
                memcpy(x_out, xu, sizeof(double) * (size_t)n);
                memcpy(y_out, yu, sizeof(double) * (size_t)m);
                status = converged ? 1 : (infeasible ? infeasible : 4);
                break;
            }
            first = 0;
        }

        /* 5. one accepted iteration */
        double used = eta;   /* the eta the accepted step was taken with */
        for (;;) {
            const double* rec = (o->replay && attempts < o->replay_len)
                                    ? o->replay + ORC_ATTEMPT_FIELDS * attempts : NULL;
            if (rec) eta = rec[1];   /* replay: the step the other run tried */
            double tau = eta / omega, sigma = eta * omega;
            orc_pdhg_step(lp, vs, cs, qs, ls, us, x, y, tau, sigma, xn, yn);
            ++attempts;
            used = eta;
            if (!o->adaptive_step) {
                if (alog && al < alog_cap) {
                    double* r = alog + ORC_ATTEMPT_FIELDS * al;
                    r[0] = (double)k; r[1] = eta; r[2] = NAN; r[3] = eta; r[4] = 1.0;
                    r[5] = omega; r[6] = NAN; r[7] = NAN; r[8] = NAN;
                }
                ++al;
                break;
            }
            /* Algorithm 5 */
            double dx2 = 0.0, dy2 = 0.0;
            for (int64_t j = 0; j < n; ++j) { dx[j] = xn[j] - x[j]; dx2 += dx[j] * dx[j]; }
            orc_spmv(lp, vs, dx, Kdx);
            double inter = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double d = yn[i] - y[i];
                dy2 += d * d;
                inter += d * Kdx[i];
            }
            double eta_bar = 0.0, eta_next = 0.0;
            const int accept = orc_step_rule(eta, omega, dx2, dy2, inter, k, &eta_bar, &eta_next);
            if (alog && al < alog_cap) {
                double* r = alog + ORC_ATTEMPT_FIELDS * al;
                r[0] = (double)k; r[1] = eta; r[2] = eta_bar; r[3] = eta_next; r[4] = accept;
                r[5] = omega; r[6] = dx2; r[7] = dy2; r[8] = inter;
            }
            ++al;
            eta = eta_next;            /* eta' is used by the next attempt either way */
            if (rec ? rec[4] != 0.0 : accept) break;
        }
        /* eta-weighted averages of the accepted iterates (Section 2.4.2) */
        for (int64_t j = 0; j < n; ++j) xsum[j] += used * xn[j];
        for (int64_t i = 0; i < m; ++i) ysum[i] += used * yn[i];
        wsum += used;
        memcpy(xp, x, sizeof(double) * (size_t)n);
        memcpy(yp, y, sizeof(double) * (size_t)m);
        memcpy(x, xn, sizeof(double) * (size_t)n);
        memcpy(y, yn, sizeof(double) * (size_t)m);
        ++k;
        ++epoch_k;
    }

    if (info) {
        info->status = status;
        info->iters = k;
        info->attempts = attempts;
        info->restarts = nrestarts;
        info->pobj = pobj; info->dobj = dobj;
        info->rel_gap = rel[0]; info->rel_pres = rel[1]; info->rel_dres = rel[2];
        info->omega = omega; info->eta = eta; info->norm_K = normK;
        info->pc_alpha = o->pock_chambolle ? o->pc_alpha : NAN;
    }
    if (alog_len) *alog_len = al;
    if (trace_len) *trace_len = tl;
    free(vs); free(R); free(C); free(cs); free(qs); free(ls); free(us);
    free(x); free(y); free(xn); free(yn); free(xsum); free(ysum); free(xa); free(ya);
    free(xanc); free(yanc); free(dx); free(Kdx); free(xu); free(yu);
    free(xp); free(yp); free(ddx); free(ddy); free(dlam); free(lam1); free(tmpn);
    return status;
}

/* ------------------------------------------------------------------ */
/* restarted (reflected) Halpern PDHG                                  */
/* ------------------------------------------------------------------ */

/*
 * The Conclusion names restarted Halpern PDHG (Lu and Yang, 2024) as a way to
 * extend the solver; the paper prints no algorithm for it.  This is the
 * published method restated on the operator of Algorithm 1.
 *
 * T(z), z = (x, y): one fixed-step PDHG step (orc_pdhg_step, theta = 1).  With
 * F(z) = (c - K^T y + N_X(x), K x - q + N_Y(y)) the step satisfies
 * 0 in F(T z) + P (T z - z) for P = [[I / tau, K^T], [K, I / sigma]], so T is
 * firmly nonexpansive in the P-norm when tau sigma ||K||^2 < 1, and
 * ||(dx, dy)||_P^2 = ||dx||^2 / tau + ||dy||^2 / sigma + 2 dy^T K dx.
 */
double orc_pnorm2(const orc_lp* lp, const double* vals, const double* dx, const double* dy,
                  double tau, double sigma)
{
    const int64_t m = lp->m, n = lp->n;
    double* Kdx = (double*)xalloc(m);
    orc_spmv(lp, vals, dx, Kdx);
    const double v = dot(n, dx, dx) / tau + dot(m, dy, dy) / sigma + 2.0 * dot(m, dy, Kdx);
    free(Kdx);
    return v;
}

/*
 * One inner step from z = (x, y) with anchor z0 = (xanc, yanc), inner index
 * k (0 at the anchor) and reflection rho:
 *   (xh, yh) = T(z)
 *   z_next = (k + 1) / (k + 2) * ((1 + rho) T(z) - rho z) + 1 / (k + 2) * z0
 * rho = 0 is plain Halpern on T; rho = 1 is Halpern on the reflection 2T - I
 * (nonexpansive).  Returns the fixed-point residual ||z - T(z)||_P.
 */
double orc_halpern_step(const orc_lp* lp, const double* vals, const double* c, const double* q,
                        const double* l, const double* u, const double* x, const double* y,
                        const double* xanc, const double* yanc, double tau, double sigma,
                        int64_t k, double rho, double* xh, double* yh, double* xn, double* yn)
{
    const int64_t m = lp->m, n = lp->n;
    orc_pdhg_step(lp, vals, c, q, l, u, x, y, tau, sigma, xh, yh);
    const double lam = (double)(k + 1) / (double)(k + 2);
    for (int64_t j = 0; j < n; ++j)
        xn[j] = lam * ((1.0 + rho) * xh[j] - rho * x[j]) + (1.0 - lam) * xanc[j];
    for (int64_t i = 0; i < m; ++i)
        yn[i] = lam * ((1.0 + rho) * yh[i] - rho * y[i]) + (1.0 - lam) * yanc[i];
    double* dx = (double*)xalloc(n);
    double* dy = (double*)xalloc(m);
    for (int64_t j = 0; j < n; ++j) dx[j] = xh[j] - x[j];
    for (int64_t i = 0; i < m; ++i) dy[i] = yh[i] - y[i];
    const double r2 = orc_pnorm2(lp, vals, dx, dy, tau, sigma);
    free(dx);
    free(dy);
    return sqrt(r2 > 0.0 ? r2 : 0.0);
}

/*
 * Restarted Halpern PDHG on the scaled problem of orc_solve (same steps 1-4:
 * Ruiz, eta = eta_scale / ||K~||_2 kept fixed, omega, start point and anchor).
 * adaptive_step and infeas_detect are not used (Algorithm 5 changes T from step
 * to step; Algorithm 6 is defined on the differences of plain PDHG iterates).
 *  - Each iteration is one orc_halpern_step; k counts them, epoch_k counts those
 *    since the last restart (the inner index of the step).  r_0 is the residual
 *    ||z - T(z)||_P of the first step of an epoch (at its anchor).
 *  - The candidate of a check is T(z) of the step just taken (at the start check:
 *    the start point).  Checks: at the start, every check_every iterations and at
 *    max_iters; termination (Section 2.3.2) on the unscaled candidate.
 *  - Restart criteria on the residual r of the step just taken (Lu and Yang):
 *    r <= beta_s r_0, or r <= beta_n r_0 and r > r at the previous check of the
 *    epoch, or epoch_k > beta_a k (the paper's artificial criterion).  At a
 *    restart the iterate and the anchor become the candidate T(z) and omega is
 *    updated by Algorithm 4 from the candidate's distance to the old anchor.
 *  - Trace: kkt_cur is KKT_omega of the Halpern iterate z_next, kkt_avg and
 *    kkt_cand that of the candidate (cand_is_avg = 1).
 */
int orc_solve_halpern(const orc_lp* lp, const orc_opts* o, double* x_out, double* y_out,
                      orc_info* info, orc_trace* trace, int64_t trace_cap, int64_t* trace_len)
{
    const int64_t m = lp->m, n = lp->n, nnz = lp->row_ptr[m];
    double* vs = (double*)xalloc(nnz);
    double* R = (double*)xalloc(m);
    double* C = (double*)xalloc(n);
    double *cs = (double*)xalloc(n), *qs = (double*)xalloc(m);
    double *ls = (double*)xalloc(n), *us = (double*)xalloc(n);
    double *x = (double*)xalloc(n), *y = (double*)xalloc(m);
    double *xh = (double*)xalloc(n), *yh = (double*)xalloc(m);
    double *xn = (double*)xalloc(n), *yn = (double*)xalloc(m);
    double *xanc = (double*)xalloc(n), *yanc = (double*)xalloc(m);
    double *xu = (double*)xalloc(n), *yu = (double*)xalloc(m);
    double kc[8], ka[8], kk[8];
    int64_t tl = 0;

    orc_ruiz(lp, o->ruiz_iters, o->ruiz_tol, o->pock_chambolle, o->pc_alpha, vs, R, C);
    for (int64_t j = 0; j < n; ++j) {
        cs[j] = C[j] * lp->c[j];
        ls[j] = lp->l[j] / C[j];
        us[j] = lp->u[j] / C[j];
    }
    for (int64_t i = 0; i < m; ++i) qs[i] = R[i] * lp->q[i];
    const double normK = orc_power_norm(lp, vs, o->power_iters);
    double eta = normK > 0.0 ? o->eta_scale / normK : 1.0;
    if (o->eta0 > 0.0) eta = o->eta0;
    const double nc = nrm2(n, cs), nq = nrm2(m, qs);
    double omega = (nc > o->eps_zero && nq > o->eps_zero) ? nc / nq : 1.0;
    if (o->omega0 > 0.0) omega = o->omega0;
    for (int64_t j = 0; j < n; ++j) x[j] = clamp(o->x0 ? o->x0[j] / C[j] : 0.0, ls[j], us[j]);
    for (int64_t i = 0; i < m; ++i) {
        double y0 = o->y0 ? o->y0[i] / R[i] : 0.0;
        if (lp->sense[i] && y0 < 0.0) y0 = 0.0;
        y[i] = y0;
    }
    memcpy(xanc, x, sizeof(double) * (size_t)n);
    memcpy(yanc, y, sizeof(double) * (size_t)m);
    /* the start check's candidate is the start point */
    memcpy(xh, x, sizeof(double) * (size_t)n);
    memcpy(yh, y, sizeof(double) * (size_t)m);
    memcpy(xn, x, sizeof(double) * (size_t)n);
    memcpy(yn, y, sizeof(double) * (size_t)m);
    int64_t k = 0, epoch_k = 0, nrestarts = 0;
    double r = 0.0, r0 = 0.0, r_prev = INFINITY;
    int status = 0, first = 1;
    double rel[3] = {0, 0, 0}, pobj = 0, dobj = 0;

    for (;;) {
        if (!first) {
            const double tau = eta / omega, sigma = eta * omega;
            r = orc_halpern_step(lp, vs, cs, qs, ls, us, x, y, xanc, yanc, tau, sigma, epoch_k,
                                 o->reflect, xh, yh, xn, yn);
            if (epoch_k == 0) r0 = r;
            ++k;
            ++epoch_k;
        }
        const int do_check = first || (k % o->check_every == 0) || (k >= o->max_iters);
        int restart = 0;
        if (do_check) {
            orc_kkt(lp, vs, cs, qs, ls, us, xn, yn, omega, kc);
            orc_kkt(lp, vs, cs, qs, ls, us, xh, yh, omega, ka);
            for (int64_t j = 0; j < n; ++j) xu[j] = C[j] * xh[j];
            for (int64_t i = 0; i < m; ++i) yu[i] = R[i] * yh[i];
            orc_kkt(lp, lp->vals, lp->c, lp->q, lp->l, lp->u, xu, yu, omega, kk);
            rel[0] = kk[4]; rel[1] = kk[5]; rel[2] = kk[6];
            pobj = kk[0]; dobj = kk[1];
            const int converged = rel[0] <= o->tol && rel[1] <= o->tol && rel[2] <= o->tol;
            if (!first && !converged && o->restarts) {
                const int crit1 = r <= o->beta_sufficient * r0;
                const int crit2 = r <= o->beta_necessary * r0 && r > r_prev;
                const int crit3 = (double)epoch_k > o->beta_artificial * (double)k;
                restart = crit1 || crit2 || crit3;
            }
            if (restart) {
                if (o->primal_weight_update) {
                    /* Algorithm 4 on the candidate's distance to the anchor */
                    double ddx = 0.0, ddy = 0.0;
                    for (int64_t j = 0; j < n; ++j) ddx += (xh[j] - xanc[j]) * (xh[j] - xanc[j]);
                    for (int64_t i = 0; i < m; ++i) ddy += (yh[i] - yanc[i]) * (yh[i] - yanc[i]);
                    ddx = sqrt(ddx);
                    ddy = sqrt(ddy);
                    omega = orc_primal_weight(omega, ddx, ddy, o->eps_zero);
                }
                memcpy(xanc, xh, sizeof(double) * (size_t)n);
                memcpy(yanc, yh, sizeof(double) * (size_t)m);
                epoch_k = 0;
                r_prev = INFINITY;
                ++nrestarts;
            } else if (!first) {
                r_prev = r;
            }
            if (trace && tl < trace_cap) {
                orc_trace* t = &trace[tl];
                t->k = (double)k; t->attempts = (double)k; t->restart = restart;
                t->cand_is_avg = 1; t->omega = omega; t->eta = eta;
                t->kkt_cur = kc[7]; t->kkt_avg = ka[7];
                t->rel_gap = rel[0]; t->rel_pres = rel[1]; t->rel_dres = rel[2];
                t->kkt_cand = ka[7];
                t->fpr = r; t->fpr0 = r0;
                t->own_restart = restart; t->own_cand_is_avg = 1;
                t->kkt_anchor = NAN; t->kkt_prev = NAN;
            }
            ++tl;
            if (converged || k >= o->max_iters) {
                memcpy(x_out, xu, sizeof(double) * (size_t)n);
                memcpy(y_out, yu, sizeof(double) * (size_t)m);
                status = converged ? 1 : 4;
                break;
            }
            first = 0;
        }
        if (restart) {
            memcpy(x, xh, sizeof(double) * (size_t)n);
            memcpy(y, yh, sizeof(double) * (size_t)m);
        } else {
            memcpy(x, xn, sizeof(double) * (size_t)n);
            memcpy(y, yn, sizeof(double) * (size_t)m);
        }
    }

    if (info) {
        info->status = status;
        info->iters = k;
        info->attempts = k;
        info->restarts = nrestarts;
        info->pobj = pobj; info->dobj = dobj;
        info->rel_gap = rel[0]; info->rel_pres = rel[1]; info->rel_dres = rel[2];
        info->omega = omega; info->eta = eta; info->norm_K = normK;
        info->pc_alpha = o->pock_chambolle ? o->pc_alpha : NAN;
    }
    if (trace_len) *trace_len = tl;
    free(vs); free(R); free(C); free(cs); free(qs); free(ls); free(us);
    free(x); free(y); free(xh); free(yh); free(xn); free(yn); free(xanc); free(yanc);
    free(xu); free(yu);
    return status;
}

/* ------------------------------------------------------------------ */
/* unrolled fixed-step PDHG and its reverse-mode derivative            */
/* ------------------------------------------------------------------ */

/*
 * K_iters fixed-step iterations on the unscaled problem from (x0, y0):
 * xs[t*n ..], ys[t*m ..] hold iterate t = 0..K_iters (caller sizes them).
 */
void orc_unrolled_forward(const orc_lp* lp, double tau, double sigma, int32_t K_iters,
                          const double* x0, const double* y0, double* xs, double* ys)
{
    const int64_t m = lp->m, n = lp->n;
    memcpy(xs, x0, sizeof(double) * (size_t)n);
    memcpy(ys, y0, sizeof(double) * (size_t)m);
    for (int32_t t = 0; t < K_iters; ++t)
        orc_pdhg_step(lp, lp->vals, lp->c, lp->q, lp->l, lp->u,
                      xs + (int64_t)t * n, ys + (int64_t)t * m, tau, sigma,
                      xs + (int64_t)(t + 1) * n, ys + (int64_t)(t + 1) * m);
}

/*
 * Gradient of L(x_K) with respect to c, q and the nonzeros of K, given
 * gxK = dL/dx_K, with tau and sigma held constant.  For one step
 *   v_x = x - tau (c - K^T y),  x' = clamp(v_x, l, u),  xbar = 2 x' - x,
 *   v_y = y + sigma (q - K xbar), y' = proj_Y(v_y),
 * the chain rule gives, for incoming adjoints (gx', gy'):
 *   gv_y = M_y * gy'      M_y = 1 on equality rows or where v_y > 0
 *   gq  += sigma gv_y;    gxbar = -sigma K^T gv_y;   gK_ij += -sigma gv_y_i xbar_j
 *   gv_x = M_x * (gx' + 2 gxbar)   M_x = 1 where l < v_x < u (strict interior)
 *   gc  += -tau gv_x;     gK_ij += tau y_i gv_x_j
 *   gx   = gv_x - gxbar;  gy = gv_y + tau K gv_x
 * dc, dq, dvals are overwritten.
 */
void orc_unrolled_adjoint(const orc_lp* lp, double tau, double sigma, int32_t K_iters,
                          const double* x0, const double* y0, const double* gxK,
                          double* dc, double* dq, double* dvals)
{
    const int64_t m = lp->m, n = lp->n, nnz = lp->row_ptr[m];
    double* xs = (double*)xalloc((int64_t)(K_iters + 1) * n);
    double* ys = (double*)xalloc((int64_t)(K_iters + 1) * m);
    orc_unrolled_forward(lp, tau, sigma, K_iters, x0, y0, xs, ys);
    double *gx = (double*)xalloc(n), *gy = (double*)xalloc(m);
    double *KTy = (double*)xalloc(n), *vx = (double*)xalloc(n), *xbar = (double*)xalloc(n);
    double *Kxb = (double*)xalloc(m), *gvy = (double*)xalloc(m), *gxbar = (double*)xalloc(n);
    double *gvx = (double*)xalloc(n), *Kgvx = (double*)xalloc(m);
    memcpy(gx, gxK, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < m; ++i) gy[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) dc[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) dq[i] = 0.0;
    for (int64_t p = 0; p < nnz; ++p) dvals[p] = 0.0;
    for (int32_t t = K_iters - 1; t >= 0; --t) {
        const double* x = xs + (int64_t)t * n;
        const double* y = ys + (int64_t)t * m;
        const double* xn = xs + (int64_t)(t + 1) * n;
        /* recompute the step's intermediates */
        orc_spmv_t(lp, lp->vals, y, KTy);
        for (int64_t j = 0; j < n; ++j) {
            vx[j] = x[j] - tau * (lp->c[j] - KTy[j]);
            xbar[j] = 2.0 * xn[j] - x[j];
        }
        orc_spmv(lp, lp->vals, xbar, Kxb);
        /* dual half */
        for (int64_t i = 0; i < m; ++i) {
            double vy = y[i] + sigma * (lp->q[i] - Kxb[i]);
            int my = !lp->sense[i] || vy > 0.0;
            gvy[i] = my ? gy[i] : 0.0;
            dq[i] += sigma * gvy[i];
        }
        orc_spmv_t(lp, lp->vals, gvy, gxbar);
        for (int64_t j = 0; j < n; ++j) gxbar[j] *= -sigma;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
                dvals[p] += -sigma * gvy[i] * xbar[lp->col_idx[p]];
        /* primal half */
        for (int64_t j = 0; j < n; ++j) {
            int mx = lp->l[j] < vx[j] && vx[j] < lp->u[j];
            gvx[j] = mx ? gx[j] + 2.0 * gxbar[j] : 0.0;
            dc[j] += -tau * gvx[j];
        }
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = lp->row_ptr[i]; p < lp->row_ptr[i + 1]; ++p)
                dvals[p] += tau * y[i] * gvx[lp->col_idx[p]];
        orc_spmv(lp, lp->vals, gvx, Kgvx);
        for (int64_t j = 0; j < n; ++j) gx[j] = gvx[j] - gxbar[j];
        for (int64_t i = 0; i < m; ++i) gy[i] = gvy[i] + tau * Kgvx[i];
    }
    free(xs); free(ys); free(gx); free(gy); free(KTy); free(vx); free(xbar);
    free(Kxb); free(gvy); free(gxbar); free(gvx); free(Kgvx);
}

/* ------------------------------------------------------------------ */
/* Algorithm 7: fishnet casting                                        */
/* ------------------------------------------------------------------ */

/*
 * Multi-start warm start of Section 2.5, on the scaled problem of the solver
 * (Ruiz per o->ruiz_iters, eta = eta_scale / ||K~||_2 or o->eta0,
 * omega = ||c~|| / ||q~|| or o->omega0, exactly as orc_solve sets them up).
 *
 * P columns (a power of two, 1..64); G holds n x P standard-normal draws,
 * G[j * P + p] for coordinate j of point p; Z holds the normal draws of the
 * repopulations, consumed in order (nZ of them available).
 *
 * Readings:
 *  - spectral casting: r = ||K~||_2 (the Algorithm 2 estimate); point p is
 *    x~_p = (r / sqrt(n)) g_p, so that E||x~_p||^2 = r^2 ("a normal
 *    distribution around B_r");
 *  - Y^0 = K~ X^0 as printed; PDHG(.) is k_steps fixed-step iterations of
 *    Algorithm 1 (theta = 1, tau = eta / omega, sigma = eta * omega) per column;
 *  - j is the column count at the top of a round; cull_points keeps the j / 2
 *    columns of smallest |duality gap| |c~^T x - (q~^T y + l~^T lambda^+ +
 *    u~^T lambda^-)|, lambda = proj_Lambda(c~ - K~^T y) (ties: lower index
 *    first), in their old order;
 *  - repopulate (round index i odd and j > 2) appends one new column per kept
 *    column: new column t = sum_s w_ts * kept_s with w_ts = |z_ts| / sum_s |z_ts|
 *    (the text normalises normal draws to sum one and calls the result a convex
 *    combination; absolute values make it one; all-zero draws give equal
 *    weights); the same weights combine the dual columns;
 *  - the loop ends when one column is left; its unscaled (C x~, R y~) is the
 *    output.
 * gaps (may be NULL): per round, the |gap| of each of the j columns before the
 * cull, at gaps[round * P + column] (unused entries untouched).
 * rounds_out (may be NULL): number of rounds.  Returns 0, or -1 for an invalid P
 * or too few draws in Z.
 */
int orc_fishnet(const orc_lp* lp, const orc_opts* o, int32_t P, int32_t k_steps,
                const double* G, const double* Z, int64_t nZ, double* x_out, double* y_out,
                double* gaps, int32_t* rounds_out)
{
    if (P < 1 || P > 64 || (P & (P - 1)) != 0 || k_steps < 0) return -1;
    const int64_t m = lp->m, n = lp->n, nnz = lp->row_ptr[m];
    double* vs = (double*)xalloc(nnz);
    double* R = (double*)xalloc(m);
    double* C = (double*)xalloc(n);
    double *cs = (double*)xalloc(n), *qs = (double*)xalloc(m);
    double *ls = (double*)xalloc(n), *us = (double*)xalloc(n);
    orc_ruiz(lp, o->ruiz_iters, o->ruiz_tol, o->pock_chambolle, o->pc_alpha, vs, R, C);
    for (int64_t j = 0; j < n; ++j) {
        cs[j] = C[j] * lp->c[j];
        ls[j] = lp->l[j] / C[j];
        us[j] = lp->u[j] / C[j];
    }
    for (int64_t i = 0; i < m; ++i) qs[i] = R[i] * lp->q[i];
    const double normK = orc_power_norm(lp, vs, o->power_iters);
    double eta = normK > 0.0 ? o->eta_scale / normK : 1.0;
    if (o->eta0 > 0.0) eta = o->eta0;
    const double nc = nrm2(n, cs), nq = nrm2(m, qs);
    double omega = (nc > o->eps_zero && nq > o->eps_zero) ? nc / nq : 1.0;
    if (o->omega0 > 0.0) omega = o->omega0;
    const double tau = eta / omega, sigma = eta * omega;

    /* columns: X[p] (n), Y[p] (m) */
    double** X = (double**)calloc((size_t)P, sizeof(double*));
    double** Y = (double**)calloc((size_t)P, sizeof(double*));
    double** X2 = (double**)calloc((size_t)P, sizeof(double*));
    double** Y2 = (double**)calloc((size_t)P, sizeof(double*));
    for (int p = 0; p < P; ++p) {
        X[p] = (double*)xalloc(n);
        Y[p] = (double*)xalloc(m);
        X2[p] = (double*)xalloc(n);
        Y2[p] = (double*)xalloc(m);
    }
    double* xn = (double*)xalloc(n);
    double* yn = (double*)xalloc(m);
    double* gap = (double*)calloc((size_t)P, sizeof(double));
    int* order = (int*)calloc((size_t)P, sizeof(int));
    double* w = (double*)calloc((size_t)P, sizeof(double));
    double kk[8];

    /* spectral casting and Y^0 = K~ X^0 */
    const double rad = normK / sqrt((double)n);
    for (int p = 0; p < P; ++p) {
        for (int64_t j = 0; j < n; ++j) X[p][j] = rad * G[j * P + p];
        orc_spmv(lp, vs, X[p], Y[p]);
    }

    int status = 0, cols = P, round = 0;
    int64_t zpos = 0;
    while (cols > 1) {
        const int j_top = cols;
        for (int p = 0; p < cols; ++p) {
            for (int t = 0; t < k_steps; ++t) {
                orc_pdhg_step(lp, vs, cs, qs, ls, us, X[p], Y[p], tau, sigma, xn, yn);
                memcpy(X[p], xn, sizeof(double) * (size_t)n);
                memcpy(Y[p], yn, sizeof(double) * (size_t)m);
            }
            orc_kkt(lp, vs, cs, qs, ls, us, X[p], Y[p], omega, kk);
            gap[p] = fabs(kk[0] - kk[1]);
            if (gaps) gaps[(int64_t)round * P + p] = gap[p];
        }
        /* cull_points: rank by gap (insertion sort, stable), keep the best half */
        for (int p = 0; p < cols; ++p) order[p] = p;
        for (int a = 1; a < cols; ++a) {
            const int v = order[a];
            int b = a - 1;
            while (b >= 0 && gap[order[b]] > gap[v]) {
                order[b + 1] = order[b];
                --b;
            }
            order[b + 1] = v;
        }
        const int keep = cols / 2;
        /* survivors in their old order */
        int* kept = (int*)calloc((size_t)keep, sizeof(int));
        for (int a = 0; a < keep; ++a) kept[a] = order[a];
        for (int a = 1; a < keep; ++a) {
            const int v = kept[a];
            int b = a - 1;
            while (b >= 0 && kept[b] > v) {
                kept[b + 1] = kept[b];
                --b;
            }
            kept[b + 1] = v;
        }
        for (int a = 0; a < keep; ++a) {
            memcpy(X2[a], X[kept[a]], sizeof(double) * (size_t)n);
            memcpy(Y2[a], Y[kept[a]], sizeof(double) * (size_t)m);
        }
        free(kept);
        for (int a = 0; a < keep; ++a) {
            memcpy(X[a], X2[a], sizeof(double) * (size_t)n);
            memcpy(Y[a], Y2[a], sizeof(double) * (size_t)m);
        }
        cols = keep;
        /* repopulate */
        if ((round & 1) == 1 && j_top > 2) {
            if (zpos + (int64_t)keep * keep > nZ) {
                status = -1;
                break;
            }
            for (int t = 0; t < keep; ++t) {
                double sw = 0.0;
                for (int a = 0; a < keep; ++a) {
                    w[a] = fabs(Z[zpos + (int64_t)t * keep + a]);
                    sw += w[a];
                }
                for (int a = 0; a < keep; ++a) w[a] = sw > 0.0 ? w[a] / sw : 1.0 / keep;
                double* xt = X[keep + t];
                double* yt = Y[keep + t];
                for (int64_t j = 0; j < n; ++j) {
                    double v = 0.0;
                    for (int a = 0; a < keep; ++a) v += w[a] * X[a][j];
                    xt[j] = v;
                }
                for (int64_t i = 0; i < m; ++i) {
                    double v = 0.0;
                    for (int a = 0; a < keep; ++a) v += w[a] * Y[a][i];
                    yt[i] = v;
                }
            }
            zpos += (int64_t)keep * keep;
            cols = 2 * keep;
        }
        ++round;
    }
    if (status == 0) {
        for (int64_t j = 0; j < n; ++j) x_out[j] = C[j] * X[0][j];
        for (int64_t i = 0; i < m; ++i) y_out[i] = R[i] * Y[0][i];
    }
    if (rounds_out) *rounds_out = round;
    for (int p = 0; p < P; ++p) {
        free(X[p]);
        free(Y[p]);
        free(X2[p]);
        free(Y2[p]);
    }
    free(X); free(Y); free(X2); free(Y2);
    free(xn); free(yn); free(gap); free(order); free(w);
    free(vs); free(R); free(C); free(cs); free(qs); free(ls); free(us);
    return status;
}
