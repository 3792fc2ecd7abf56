// Per-LP control decisions of the restarted PDHG loop, shared by the single
// and the batched solver: the Algorithm 5 step decision and the KKT check
// (candidate, termination, restart criteria, Algorithm 4).  Each runs in one
// thread and updates one control block.
#pragma once

#include "common.cuh"

namespace pdhg {

// Algorithm 5 decision (or the plain swap of a fixed step), by one thread.
// The paper's k is read as the 1-based index of the iteration being taken.
__device__ __forceinline__ void step_decide(Ctrl* ctrl, int adapt, double dy2, double dx2, double inter)
{
    const double eta = ctrl->eta, omega = ctrl->omega;
    bool accept = true;
    double eta_next = eta;
    if (adapt) {
        const double movement = omega * dx2 + dy2 / omega;
        const double eta_bar = inter != 0.0 ? movement / (2.0 * fabs(inter)) : INFINITY;
        const double kp1 = (double)(ctrl->k + 1) + 1.0;
        const double e1 = (1.0 - pow(kp1, -0.3)) * eta_bar;
        const double e2 = (1.0 + pow(kp1, -0.6)) * eta;
        eta_next = e1 < e2 ? e1 : e2;
        accept = eta <= eta_bar;
        if (!isfinite(movement) || isnan(inter)) {
            ctrl->status = LP_NUMERICAL_ERROR;
            ctrl->done = 1;
            ctrl->skip = 1;
            return;
        }
    }
    ctrl->attempts += 1;
    if (accept) {
        ctrl->cur ^= 1;
        ctrl->k += 1;
        ctrl->epoch_k += 1;
        ctrl->pend_w = eta;
        ctrl->W += eta;
        ctrl->rejects = 0;
    } else {
        ctrl->pend_w = 0.0;
        ctrl->rejects += 1;
    }
    ctrl->eta = eta_next;
    if (ctrl->k % ctrl->check_every == 0 || ctrl->k >= ctrl->max_iters) {
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
// thread.  r[8] and cc[10] are the row- and column-side sums of k_check_rows /
// k_check_cols.
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
    const double kkt_a = ctrl->W > 0.0 ? sqrt(w * w * r[4] + cc[5] / (w * w) + gap_a * gap_a)
                                       : INFINITY;
    const int cand_avg = !(kkt_c < kkt_a);
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
    int restart = 0;
    if (first) {
        ctrl->kkt_anchor = kkt_cand;
    } else if (!converged && ctrl->restarts_on) {
        const int c1 = kkt_cand <= ctrl->beta_s * ctrl->kkt_anchor;
        const int c2 = kkt_cand <= ctrl->beta_n * ctrl->kkt_anchor && kkt_cand > ctrl->kkt_prev;
        const int c3 = (double)ctrl->epoch_k > ctrl->beta_a * (double)ctrl->k;
        restart = c1 || c2 || c3;
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
        ctrl->epoch_k = 0;
        ctrl->W = 0.0;
        ctrl->restarts += 1;
    } else if (!first) {
        ctrl->kkt_prev = kkt_cand;
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
