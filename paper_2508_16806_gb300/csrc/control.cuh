// Per-LP control decisions of the restarted PDHG loop, shared by the single
// and the batched solver: the Algorithm 5 step decision and the KKT check
// (candidate, termination, restart criteria, Algorithm 4).  Each runs in one
// thread and updates one control block.
#pragma once

#include "common.cuh"

namespace pdhg {

// lambda = proj_Lambda(v) (Section 2.3.1): Lambda_j = {0}, R^-, R^+ or R by
// which of l_j, u_j is finite.
template <typename T>
__device__ __forceinline__ T proj_lambda(T v, bool lf, bool uf)
{
    if (!lf && !uf) return T(0);
    if (!lf) return v < T(0) ? v : T(0);
    if (!uf) return v > T(0) ? v : T(0);
    return v;
}

// Row-side terms of a KKT check, accumulated per thread in the iterate
// precision T (GB300's FP64 pipe is narrow; FP32 sums of a few rows per thread
// keep 1e-7 relative accuracy, and every partial is reduced in FP64):
// [0] sum r_s^2  [1] sum (r_s / R)^2  [2] q~^T y  [3] ||y - y_anchor||^2  (current)
// [4..7] the same for the average; r = q~ - K~ x, clamped at 0 on >= rows.
// Algorithm 6 on the last step: [8] ||A dx||^2, [9] ||dy||^2, [10] q^T dy and
// the maxima mx[0] of -(G dx), mx[1] of -dy_ineq (both >= 0).  With K~ = R K C,
// y = R y~, x = C x~: (K dx)_i = (K~ dx~)_i / R_i, dy_i = R_i dy~_i and
// q_i dy_i = q~_i dy~_i.
template <typename T>
struct RowCheck {
    T v[kRowSums] = {};
    T mx[kRowMax] = {};
    __device__ __forceinline__ void add(T q, T kx, T y, T kxa, T ya, T yanc, T rinv, bool ge)
    {
        T r = q - kx;
        if (ge && r < T(0)) r = T(0);
        const T ru = r * rinv;
        v[0] += r * r;
        v[1] += ru * ru;
        v[2] += q * y;
        v[3] += (y - yanc) * (y - yanc);
        T ra = q - kxa;
        if (ge && ra < T(0)) ra = T(0);
        const T rau = ra * rinv;
        v[4] += ra * ra;
        v[5] += rau * rau;
        v[6] += q * ya;
        v[7] += (ya - yanc) * (ya - yanc);
    }
    __device__ __forceinline__ void add_infeas(T q, T kx, T kxp, T y, T yp, T R, T rinv, bool ge)
    {
        const T adx = (kx - kxp) * rinv;
        const T dys = y - yp;
        const T dy = R * dys;
        if (ge) {
            mx[0] = fmax(mx[0], -adx);
            mx[1] = fmax(mx[1], -dy);
        } else {
            v[8] += adx * adx;
        }
        v[9] += dy * dy;
        v[10] += q * dys;
    }
};

// Column-side terms, same conventions: [0] sum d_s^2  [1] sum (d_s / C)^2
// [2] c~^T x  [3] l~^T lambda^+ + u~^T lambda^-  [4] ||x - x_anchor||^2
// (current), [5..9] average; d = v - lambda, v = c~ - K~^T y, lambda = proj_Lambda(v).
// Algorithm 6: [10] ||dx||^2, [11] c^T dx, [12] ||K^T dy + dlambda||^2,
// [13] ||dlambda||^2, [14] l^T dlambda^+ + u^T dlambda^- and mx[0] the largest
// distance of dx_j to V_j; dx_j = C_j dx~_j, c_j dx_j = c~_j dx~_j,
// (K^T dy)_j = (K~^T dy~)_j / C_j, dlambda_j = dlambda~_j / C_j and
// l_j dlambda_j = l~_j dlambda~_j.
template <typename T>
struct ColCheck {
    T v[kColSums] = {};
    T mx[kColMax] = {};
    __device__ __forceinline__ void side(int s, T c, T kty, T x, T xanc, T l, T u, T cinv, bool lf,
                                         bool uf)
    {
        const T vj = c - kty;
        const T lam = proj_lambda(vj, lf, uf);
        const T d = vj - lam;
        const T du = d * cinv;
        T lt = T(0);
        if (lam > T(0)) lt = l * lam;
        if (lam < T(0)) lt = u * lam;
        v[5 * s + 0] += d * d;
        v[5 * s + 1] += du * du;
        v[5 * s + 2] += c * x;
        v[5 * s + 3] += lt;
        v[5 * s + 4] += (x - xanc) * (x - xanc);
    }
    __device__ __forceinline__ void add_infeas(T c, T x, T xp, T kty, T ktyp, T l, T u, T C,
                                               T cinv, bool lf, bool uf)
    {
        const T dxs = x - xp;
        const T dx = C * dxs;
        v[10] += dx * dx;
        v[11] += c * dxs;
        T dist = T(0);
        if (lf && uf) dist = fabs(dx);
        else if (lf) dist = dx < T(0) ? -dx : T(0);
        else if (uf) dist = dx > T(0) ? dx : T(0);
        mx[0] = fmax(mx[0], dist);
        const T dls = proj_lambda(c - kty, lf, uf) - proj_lambda(c - ktyp, lf, uf);
        const T dl = dls * cinv;
        const T r = (kty - ktyp) * cinv + dl;
        v[12] += r * r;
        v[13] += dl * dl;
        if (dls > T(0)) v[14] += l * dls;
        if (dls < T(0)) v[14] += u * dls;
    }
};

// Whether the check kernels evaluate Algorithm 6 for this control block.
__device__ __forceinline__ bool infeas_active(const Ctrl& c)
{
    return c.infeas && !c.first && c.k > 0;
}

// Algorithm 5 decision (or the plain swap of a fixed step), by one thread.
// The paper's k is read as the 1-based index of the iteration being taken.
// Halpern iterations (fixed step) also record the fixed-point residual.
__device__ __forceinline__ void step_decide(Ctrl* ctrl, int adapt, double dy2, double dx2, double inter,
                                            double* eta_bar_out = nullptr)
{
    const double eta = ctrl->eta, omega = ctrl->omega;
    bool accept = true;
    double eta_next = eta;
    if (adapt) {
        const double movement = omega * dx2 + dy2 / omega;
        const double eta_bar = inter != 0.0 ? movement / (2.0 * fabs(inter)) : INFINITY;
        if (eta_bar_out) *eta_bar_out = eta_bar;
        // (k + 1) of the paper with its k 1-based: accepted iterations + 2; the two
        // factors come from the period's table when the check filled one
        const long long ti = ctrl->k - ctrl->ftab_k0;
        double f3, f6;
        if (ctrl->ftab && ti >= 0 && ti < ctrl->ftab_len) {
            f3 = ctrl->ftab[ti];
            f6 = ctrl->ftab[ctrl->ftab_len + ti];
        } else {
            const double kp1 = (double)(ctrl->k + 1) + 1.0;
            f3 = 1.0 - pow(kp1, -0.3);
            f6 = 1.0 + pow(kp1, -0.6);
        }
        const double e1 = f3 * eta_bar;
        const double e2 = f6 * eta;
        eta_next = e1 < e2 ? e1 : e2;
        accept = eta <= eta_bar;
        if (!isfinite(movement) || isnan(inter)) {
            ctrl->status = LP_NUMERICAL_ERROR;
            ctrl->done = 1;
            ctrl->skip = 1;
            return;
        }
    }
    if (ctrl->halpern) {
        // fixed-point residual of this iteration in the PDHG metric:
        // ||(dx, dy)||_P^2 = ||dx||^2 / tau + ||dy||^2 / sigma + 2 dy^T K dx
        const double r2 = (omega * dx2 + dy2 / omega) / eta + 2.0 * inter;
        if (!isfinite(r2)) {
            ctrl->status = LP_NUMERICAL_ERROR;
            ctrl->done = 1;
            ctrl->skip = 1;
            return;
        }
        ctrl->fpr = sqrt(r2 > 0.0 ? r2 : 0.0);
        if (ctrl->epoch_k == 0) ctrl->fpr0 = ctrl->fpr;
    }
    ctrl->attempts += 1;
    if (accept) {
        ctrl->cur ^= 1;
        ctrl->k += 1;
        ctrl->epoch_k += 1;
        ctrl->pend_w = ctrl->halpern ? 0.0 : eta;
        ctrl->W += eta;
        ctrl->Winv = 1.0 / ctrl->W;
        ctrl->rejects = 0;
    } else {
        ctrl->pend_w = 0.0;
        ctrl->rejects += 1;
    }
    ctrl->eta = eta_next;
    refresh_scalars(*ctrl);
    // a check follows an accepted iteration that completes a check period (or
    // reaches max_iters); a rejected attempt never checks (the iterate did not move)
    if (accept && (ctrl->k % ctrl->check_every == 0 || ctrl->k >= ctrl->max_iters)) {
        ctrl->want_check = 1;
        ctrl->skip = 1;
    }
    // guards that end the device loop even if no check is reached: Algorithm 5
    // accepts once eta <= 1/||K||, so a long run of rejections means broken
    // arithmetic; the wall-clock limit is also enforced per attempt.
    if (ctrl->rejects > 1000 || !(eta_next > 0.0)) {
        ctrl->status = LP_NUMERICAL_ERROR;
        ctrl->done = 1;
        ctrl->skip = 1;
        ctrl->want_check = 0;
    } else if ((double)(global_ns() - (unsigned long long)ctrl->t0_ns) > ctrl->time_limit_ns) {
        ctrl->status = LP_TIME_LIMIT;
        ctrl->done = 1;
        ctrl->skip = 1;
        ctrl->want_check = 0;
    }
}

// KKT_omega (Section 2.4.2) of the current point and of the average, the
// restart candidate, the termination test on the unscaled problem (Section
// 2.3.2), the three restart criteria (Section 2.4.2) and Algorithm 4, by one
// thread.  r[kRowQ] and cc[kColQ] are the row- and column-side reductions of
// k_check_rows / k_check_cols.
__device__ __forceinline__ void check_decide(Ctrl* ctrl, const double* r, const double* cc,
                                             lp_trace_rec* trace)
{
    const double w = ctrl->omega;
    // current
    const double pobj_c = cc[2], dobj_c = r[2] + cc[3];
    const double gap_c = dobj_c - pobj_c;
    const double kkt_c = sqrt(w * w * r[0] + cc[0] / (w * w) + gap_c * gap_c);
    // average
    const double pobj_a = cc[7], dobj_a = r[6] + cc[8];
    const double gap_a = dobj_a - pobj_a;
    // (Halpern iterations: the "average" slot holds T(z) of the last iteration,
    // which is always the candidate)
    const int halp = ctrl->halpern;
    const double kkt_a = (halp || ctrl->W > 0.0)
                             ? sqrt(w * w * r[4] + cc[5] / (w * w) + gap_a * gap_a)
                             : INFINITY;
    const int cand_avg = halp ? 1 : !(kkt_c < kkt_a);
    const double kkt_cand = cand_avg ? kkt_a : kkt_c;
    const double pobj = cand_avg ? pobj_a : pobj_c;
    const double dobj = cand_avg ? dobj_a : dobj_c;
    const double pres_u = sqrt(cand_avg ? r[5] : r[1]);
    const double dres_u = sqrt(cand_avg ? cc[6] : cc[1]);
    const double rel_gap = fabs(dobj - pobj) / (1.0 + fabs(dobj) + fabs(pobj));
    const double rel_pres = pres_u / (1.0 + ctrl->qnorm);
    const double rel_dres = dres_u / (1.0 + ctrl->cnorm);
    const int converged = rel_gap <= ctrl->tol && rel_pres <= ctrl->tol && rel_dres <= ctrl->tol;
    const int first = ctrl->first;
    // Algorithm 6 on the last step's differences, as normalised directions:
    // row side r[8] ||A dx||^2, r[9] ||dy||^2, r[10] q^T dy, r[11] max(-G dx), r[12] max(-dy_ineq);
    // column side cc[10] ||dx||^2, cc[11] c^T dx, cc[12] ||K^T dy + dlam||^2, cc[13] ||dlam||^2,
    // cc[14] l^T dlam^+ + u^T dlam^-, cc[15] max distance of dx to V
    int infeasible = 0;
    if (!converged && infeas_active(*ctrl)) {
        const double t = ctrl->infeas_tol;
        const double nx = sqrt(cc[10]), ny = sqrt(r[9] + cc[13]);
        if (nx > 0.0 && sqrt(r[8]) / nx <= t && -r[11] / nx >= -t && cc[11] / nx <= -t &&
            cc[15] / nx <= t)
            infeasible = LP_DUAL_INFEASIBLE;
        else if (ny > 0.0 && sqrt(cc[12]) / ny <= t && -r[12] / ny >= -t &&
                 (r[10] + cc[14]) / ny > t)
            infeasible = LP_PRIMAL_INFEASIBLE;
    }
    int restart = 0;
    if (first) {
        ctrl->kkt_anchor = kkt_cand;
    } else if (!converged && !infeasible && ctrl->restarts_on) {
        const int c3 = (double)ctrl->epoch_k > ctrl->beta_a * (double)ctrl->k;
        if (halp) {
            // the same criteria on the fixed-point residual (restarted Halpern PDHG)
            const double fr = ctrl->fpr, f0 = ctrl->fpr0;
            const int c1 = fr <= ctrl->beta_s * f0;
            const int c2 = fr <= ctrl->beta_n * f0 && fr > ctrl->fpr_prev;
            restart = c1 || c2 || c3;
        } else {
            const int c1 = kkt_cand <= ctrl->beta_s * ctrl->kkt_anchor;
            const int c2 = kkt_cand <= ctrl->beta_n * ctrl->kkt_anchor && kkt_cand > ctrl->kkt_prev;
            restart = c1 || c2 || c3;
        }
    }
    double omega = w;
    if (restart) {
        if (ctrl->pwu) {
            const double ddx = sqrt(cand_avg ? cc[9] : cc[4]);
            const double ddy = sqrt(cand_avg ? r[7] : r[3]);
            if (ddx > ctrl->eps_zero && ddy > ctrl->eps_zero)
                omega = exp(0.5 * log(ddy / ddx) + 0.5 * log(w));
        }
        ctrl->kkt_anchor = kkt_cand;
        ctrl->kkt_prev = INFINITY;
        ctrl->fpr_prev = INFINITY;
        ctrl->epoch_k = 0;
        ctrl->W = 0.0;
        ctrl->Winv = 0.0;
        ctrl->restarts += 1;
    } else if (!first) {
        ctrl->kkt_prev = kkt_cand;
        ctrl->fpr_prev = ctrl->fpr;
    }
    ctrl->omega = omega;
    ctrl->restart = restart;
    ctrl->cand_avg = cand_avg;
    ctrl->kkt_cur = kkt_c;
    ctrl->kkt_avg = kkt_a;
    ctrl->kkt_cand = kkt_cand;
    ctrl->rel_gap = rel_gap;
    ctrl->rel_pres = rel_pres;
    ctrl->rel_dres = rel_dres;
    ctrl->pobj = pobj;
    ctrl->dobj = dobj;
    ctrl->pend_w = 0.0;
    refresh_scalars(*ctrl);
    ctrl->first = 0;
    if (trace && ctrl->trace_len < ctrl->trace_cap) {
        lp_trace_rec* t = trace + ctrl->trace_len;
        t->k = (double)ctrl->k;
        t->attempts = (double)ctrl->attempts;
        t->restart = restart;
        t->cand_is_avg = cand_avg;
        t->omega = omega;
        t->eta = ctrl->eta;
        t->kkt_cur = kkt_c;
        t->kkt_avg = kkt_a;
        t->rel_gap = rel_gap;
        t->rel_pres = rel_pres;
        t->rel_dres = rel_dres;
        t->kkt_cand = kkt_cand;
    }
    ctrl->trace_len += 1;
    const unsigned long long now = global_ns();
    const bool bad = !isfinite(kkt_c) || isnan(rel_gap) || isnan(rel_pres) || isnan(rel_dres);
    if (bad) {
        ctrl->status = LP_NUMERICAL_ERROR;
        ctrl->done = 1;
    } else if (converged) {
        ctrl->status = LP_OPTIMAL;
        ctrl->done = 1;
    } else if (infeasible) {
        ctrl->status = infeasible;
        ctrl->done = 1;
    } else if (ctrl->k >= ctrl->max_iters) {
        ctrl->status = LP_ITERATION_LIMIT;
        ctrl->done = 1;
    } else if ((double)(now - (unsigned long long)ctrl->t0_ns) > ctrl->time_limit_ns) {
        ctrl->status = LP_TIME_LIMIT;
        ctrl->done = 1;
    }
    if (ctrl->done) ctrl->t_done_ns = (long long)now;
}

}  // namespace pdhg
