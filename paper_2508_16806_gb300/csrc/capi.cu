// C ABI (include/lp.h): handle lifetime, solve orchestration (FP64 or FP32 +
// FP64 polish), batch, gradient and measurement entry points.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

using namespace pdhg;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

void free_all(Handle* h)
{
    for (auto* E : {&h->e64.exec, &h->e64.body_exec, &h->e32.exec, &h->e32.body_exec})
        if (*E) {
            cudaGraphExecDestroy(*E);
            *E = nullptr;
        }
    for (auto& b : h->allocs) cudaFree(b.p);
    h->allocs.clear();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
}

constexpr double kFp32MaxReflect = 0.5;

lp_status check_opts(const lp_opts* o)
{
    if (!o) return LP_INVALID_ARGUMENT;
    if (!(o->tol >= 0.0) || o->max_iters < 0 || o->check_every < 1 || o->ruiz_iters < 0 ||
        o->power_iters < 0 || !(o->eta_scale > 0.0) || !(o->time_limit_s > 0.0))
        return LP_INVALID_ARGUMENT;
    if (o->precision != LP_PREC_FP64 && o->precision != LP_PREC_MIXED) return LP_INVALID_ARGUMENT;
    if (o->loop_mode != 0 && o->loop_mode != 1) return LP_INVALID_ARGUMENT;
    if (o->infeas_detect != 0 && o->infeas_detect != 1) return LP_INVALID_ARGUMENT;
    if (o->infeas_detect && !(o->infeas_tol > 0.0)) return LP_INVALID_ARGUMENT;
    if (o->autotune != 0 && o->autotune != 1) return LP_INVALID_ARGUMENT;
    if (o->halpern != 0 && o->halpern != 1) return LP_INVALID_ARGUMENT;
    if (o->halpern && !(o->halpern_reflect >= 0.0 && o->halpern_reflect <= 1.0))
        return LP_INVALID_ARGUMENT;
    if (o->pock_chambolle < 0 || o->pock_chambolle > 2) return LP_INVALID_ARGUMENT;
    if (!(o->pc_alpha >= 0.0 && o->pc_alpha <= 2.0) || o->pc_trial_iters < 0)
        return LP_INVALID_ARGUMENT;
    if (o->attempt_cap < 0 || (o->attempt_cap > 0 && !o->attempt_log)) return LP_INVALID_ARGUMENT;
    return LP_OK;
}

// The grid of Pock-Chambolle parameters that pock_chambolle = 2 tries.
constexpr double kPcGrid[4] = {0.0, 0.5, 1.0, 2.0};

void fill_result(lp_result* r, const Ctrl& c)
{
    r->status = (lp_status)c.status;
    r->iters = c.k;
    r->attempts = c.attempts;
    r->restarts = c.restarts;
    r->pobj = c.pobj;
    r->dobj = c.dobj;
    r->rel_gap = c.rel_gap;
    r->rel_pres = c.rel_pres;
    r->rel_dres = c.rel_dres;
    r->omega = c.omega;
    r->eta = c.eta;
}

}  // namespace

extern "C" {

void lp_opts_default(lp_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-4;
    o->max_iters = 1000000;
    o->time_limit_s = 3600.0;
    o->precision = LP_PREC_FP64;
    o->check_every = 64;
    o->ruiz_iters = 10;
    o->pock_chambolle = 0;
    o->adaptive_step = 1;
    o->primal_weight_update = 1;
    o->restarts = 1;
    o->power_iters = 100;
    o->ruiz_tol = 1e-4;
    o->eta_scale = 0.9;
    o->beta_sufficient = 0.2;
    o->beta_necessary = 0.8;
    o->beta_artificial = 0.36;
    o->eps_zero = 1e-6;
    o->polish_switch_tol = 1e-5;
    o->x0 = nullptr;
    o->y0 = nullptr;
    o->omega0 = 0.0;
    o->eta0 = 0.0;
    o->warm_memory_space = LP_MEM_HOST;
    o->loop_mode = 0;
    o->infeas_detect = 1;
    o->infeas_tol = 1e-6;
    o->autotune = 0;
    o->halpern = 0;
    o->halpern_reflect = 1.0;
    o->pc_alpha = 1.0;
    o->pc_trial_iters = 0;
}

const char* lp_status_string(lp_status s)
{
    switch (s) {
    case LP_OK: return "LP_OK";
    case LP_OPTIMAL: return "LP_OPTIMAL";
    case LP_PRIMAL_INFEASIBLE: return "LP_PRIMAL_INFEASIBLE";
    case LP_DUAL_INFEASIBLE: return "LP_DUAL_INFEASIBLE";
    case LP_ITERATION_LIMIT: return "LP_ITERATION_LIMIT";
    case LP_TIME_LIMIT: return "LP_TIME_LIMIT";
    case LP_NUMERICAL_ERROR: return "LP_NUMERICAL_ERROR";
    case LP_INVALID_ARGUMENT: return "LP_INVALID_ARGUMENT";
    case LP_CUDA_ERROR: return "LP_CUDA_ERROR";
    case LP_OUT_OF_MEMORY: return "LP_OUT_OF_MEMORY";
    case LP_DEVICE_TIMEOUT: return "LP_DEVICE_TIMEOUT";
    case LP_NOT_SUPPORTED: return "LP_NOT_SUPPORTED";
    }
    return "LP_UNKNOWN_STATUS";
}

int32_t lp_abi_version(void) { return LP_ABI_VERSION; }

lp_status lp_create(const lp_desc* d, void* cuda_stream, lp_handle* out)
{
    if (!out) return LP_INVALID_ARGUMENT;
    *out = nullptr;
    if (!d || d->m < 1 || d->n < 1 || d->nnz < 0 || d->nnz >= ((int64_t)1 << 31) - 64 ||
        d->n >= ((int64_t)1 << 31) || d->m >= ((int64_t)1 << 31))
        return LP_INVALID_ARGUMENT;
    if (!d->row_ptr || (d->nnz > 0 && (!d->col_idx || !d->vals)) || !d->sense || !d->c || !d->q ||
        !d->l || !d->u)
        return LP_INVALID_ARGUMENT;
    if (d->memory_space != LP_MEM_HOST && d->memory_space != LP_MEM_DEVICE)
        return LP_INVALID_ARGUMENT;
    if (d->memory_space == LP_MEM_HOST) {
        // cheap host-side checks of the structure before any device work
        if (d->row_ptr[0] != 0 || d->row_ptr[d->m] != d->nnz) return LP_INVALID_ARGUMENT;
    }
    lp_problem_s* p = new (std::nothrow) lp_problem_s();
    if (!p) return LP_OUT_OF_MEMORY;
    Handle* h = &p->h;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete p;
        return LP_CUDA_ERROR;
    }
    if (cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            delete p;
            return LP_CUDA_ERROR;
        }
        h->own_stream = true;
    }
    lp_status s = setup_create(h, d);
    if (s != LP_OK) {
        cudaStreamSynchronize(h->stream);
        (void)cudaGetLastError();
        free_all(h);
        delete p;
        return s;
    }
    *out = p;
    return LP_OK;
}

void lp_destroy(lp_handle p)
{
    if (!p) return;
    cudaStreamSynchronize(p->h.stream);
    free_all(&p->h);
    delete p;
}

// FP64 engine, scaling (Algorithm 3), ||K~||_2 (Algorithm 2), the initial step
// size eta_scale / ||K~||_2 (Section 3.2) and primal weight ||c~|| / ||q~||
// (Section 2.4.3), or the caller's eta0 / omega0.
static lp_status prepare_fp64(Handle* h, const lp_opts* o, double* normK, double* eta0,
                              double* omega0)
{
    LP_TRY(setup_engine<double>(h, o));
    // the FP64 schedule is tuned before its first use (the power iteration), so
    // that every solve on this handle sums in the same order
    if (o->autotune) LP_TRY(tune_engine<double>(h));
    LP_TRY(setup_scale(h, o, normK));
    double cs2 = 0.0, qs2 = 0.0;
    LP_TRY(sum_of_squares(h, h->e64.c, h->n, &cs2));
    LP_TRY(sum_of_squares(h, h->e64.q, h->m, &qs2));
    const double cn = std::sqrt(cs2), qn = std::sqrt(qs2);
    *omega0 = (cn > o->eps_zero && qn > o->eps_zero) ? cn / qn : 1.0;
    if (o->omega0 > 0.0) *omega0 = o->omega0;
    *eta0 = *normK > 0.0 ? o->eta_scale / *normK : 1.0;
    if (o->eta0 > 0.0) *eta0 = o->eta0;
    return LP_OK;
}

static lp_status solve_core(Handle* h, const lp_opts* o, lp_result* r);

// lp_solve: with pock_chambolle = 2, one trial solve per alpha of kPcGrid (the
// caller's options with that pass, pc_trial_iters accepted iterations, no
// tolerance, no infeasibility detection, no outputs), then the solve with the
// alpha whose trial ended with the smallest max(rel_gap, rel_pres, rel_dres);
// ties and NaN go to the earlier alpha.  The trials' time is added to setup_s.
static lp_status solve_impl(Handle* h, const lp_opts* o, lp_result* r)
{
    LP_TRY(check_opts(o));
    if (!r) return LP_INVALID_ARGUMENT;
    if (o->pock_chambolle != 2) {
        lp_status s = solve_core(h, o, r);
        r->pc_alpha_used = o->pock_chambolle ? o->pc_alpha : NAN;
        return s;
    }
    const double t0 = now_s();
    const long long launches0 = h->launches;
    double best = kPcGrid[0], best_err = INFINITY;
    for (double a : kPcGrid) {
        lp_opts t = *o;
        t.pock_chambolle = 1;
        t.pc_alpha = a;
        t.max_iters = o->pc_trial_iters > 0 ? o->pc_trial_iters : 2 * (int64_t)o->check_every;
        t.tol = 0.0;
        t.infeas_detect = 0;
        t.attempt_log = nullptr;
        t.attempt_cap = 0;
        lp_result rt;
        std::memset(&rt, 0, sizeof(rt));
        rt.memory_space = LP_MEM_HOST;
        const lp_status st = solve_core(h, &t, &rt);
        if (st < 0) return st;
        const double e = std::max(rt.rel_gap, std::max(rt.rel_pres, rt.rel_dres));
        if (e < best_err) {
            best_err = e;
            best = a;
        }
    }
    const double t_trials = now_s() - t0;
    lp_opts t = *o;
    t.pock_chambolle = 1;
    t.pc_alpha = best;
    const lp_status s = solve_core(h, &t, r);
    r->setup_s += t_trials;
    r->kernel_launches = h->launches - launches0;
    r->pc_alpha_used = best;
    return s;
}

static lp_status solve_core(Handle* h, const lp_opts* o, lp_result* r)
{
    LP_TRY(check_opts(o));
    if (!r) return LP_INVALID_ARGUMENT;
    if (r->memory_space != LP_MEM_HOST && r->memory_space != LP_MEM_DEVICE)
        return LP_INVALID_ARGUMENT;
    if ((o->x0 || o->y0) && o->warm_memory_space != LP_MEM_HOST &&
        o->warm_memory_space != LP_MEM_DEVICE)
        return LP_INVALID_ARGUMENT;
    const double t0 = now_s();
    const long long launches0 = h->launches;
    double normK = 0.0, eta0 = 0.0, omega0 = 0.0;
    LP_TRY(prepare_fp64(h, o, &normK, &eta0, &omega0));
    if (o->precision == LP_PREC_MIXED) LP_TRY(setup_engine<float>(h, o));
    LP_CUDA_TRY(cudaStreamSynchronize(h->stream));
    const double t1 = now_s();
    r->setup_s = t1 - t0;
    r->norm_K = normK;

    Ctrl c;
    std::memset(&c, 0, sizeof(c));
    r->trace_len = 0;
    r->attempt_len = 0;
    // the attempt log runs through the phases of this solve (run_solve reads it)
    struct AlogScope {
        Handle* h;
        ~AlogScope() { h->alog_host = nullptr; h->alog_cap_host = 0; h->alog_off = 0; }
    } alog_scope{h};
    h->alog_host = o->attempt_cap > 0 ? o->attempt_log : nullptr;
    h->alog_cap_host = h->alog_host ? o->attempt_cap : 0;
    h->alog_off = 0;
    if (o->precision == LP_PREC_MIXED) {
        lp_opts o32 = *o;
        o32.tol = std::max(o->tol, o->polish_switch_tol);
        // FP32 Halpern iterations take rho <= 1/2: (1 + rho) T - rho I is then
        // averaged, so FP32 rounding does not accumulate over a long epoch (with
        // rho near 1 the FP32 iterates can stall above the hand-over tolerance)
        o32.halpern_reflect = std::min(o->halpern_reflect, kFp32MaxReflect);
        LP_TRY(run_solve<float>(h, &o32, eta0, omega0, nullptr, nullptr, o->x0, o->y0,
                                o->warm_memory_space, 0, 0, 0, r->trace, r->trace_cap, 0, &c));
        r->trace_len = c.trace_len;
        r->precision_used = LP_PREC_MIXED;
        r->fp64_iters = 0;
        // An FP32 phase that stopped optimal hands its candidate to the FP64 engine
        // in every case: the FP64 start check re-evaluates the three relative
        // errors of Section 2.3.2 with FP64 products and FP64 element terms (the
        // FP32 phase judged them on FP32 products), and LP_OPTIMAL is returned
        // only when they hold there.  When tol is below the hand-over tolerance, or
        // the FP32 judgement does not survive the FP64 one, FP64 iterations continue
        // from the candidate to tol (the FP64 polish).
        const bool polish = c.status == LP_OPTIMAL;
        if (!polish) {
            fill_result(r, c);
            LP_TRY(extract_solution<float>(h, r->x, r->y, r->memory_space));
        } else {
            if (!h->wbuf) LP_TRY(dev_alloc_n(h, &h->wbuf, (size_t)(h->n + h->m)));
            LP_TRY(extract_solution_ex<float>(h, nullptr, nullptr, LP_MEM_DEVICE, h->wbuf,
                                              h->wbuf + h->n));
            lp_opts o64 = *o;
            o64.time_limit_s = std::max(1e-3, o->time_limit_s - (now_s() - t1));
            const long long k32 = c.k;
            h->alog_off = std::min<long long>(c.alog_len, h->alog_cap_host);
            Ctrl c2;
            LP_TRY(run_solve<double>(h, &o64, c.eta, c.omega, h->wbuf, h->wbuf + h->n, nullptr,
                                     nullptr, LP_MEM_HOST, c.k, c.attempts, c.restarts, r->trace,
                                     r->trace_cap, std::min<long long>(c.trace_len, r->trace_cap),
                                     &c2));
            r->trace_len = c.trace_len + c2.trace_len;
            fill_result(r, c2);
            r->fp64_iters = c2.k - k32;
            // FP64 is the precision of the last phase only if FP64 iterations ran
            // (a confirmation by the FP64 check alone keeps the FP32 result)
            r->precision_used = r->fp64_iters > 0 ? LP_PREC_FP64 : LP_PREC_MIXED;
            LP_TRY(extract_solution<double>(h, r->x, r->y, r->memory_space));
        }
    } else {
        LP_TRY(run_solve<double>(h, o, eta0, omega0, nullptr, nullptr, o->x0, o->y0,
                                 o->warm_memory_space, 0, 0, 0, r->trace, r->trace_cap, 0, &c));
        r->trace_len = c.trace_len;
        fill_result(r, c);
        r->fp64_iters = c.k;
        r->precision_used = LP_PREC_FP64;
        LP_TRY(extract_solution<double>(h, r->x, r->y, r->memory_space));
    }
    r->solve_s = now_s() - t1;
    r->kernel_launches = h->launches - launches0;
    r->attempt_len = std::min<long long>(r->attempts, h->alog_cap_host);
    if (o->precision == LP_PREC_MIXED)
        r->split_rows = engine_of<float>(h).splitK.n + engine_of<float>(h).splitT.n;
    else
        r->split_rows = engine_of<double>(h).splitK.n + engine_of<double>(h).splitT.n;
    return r->status;
}

lp_status lp_solve(lp_handle p, const lp_opts* o, lp_result* r)
{
    if (!p) return LP_INVALID_ARGUMENT;
    lp_status s = solve_impl(&p->h, o, r);
    if (s < 0) {
        cudaStreamSynchronize(p->h.stream);
        (void)cudaGetLastError();
    }
    return s;
}

lp_status lp_solve_batch(const lp_handle* hs, int32_t count, const lp_opts* o, lp_result* rs)
{
    if (!hs || !rs || count < 1 || !o) return LP_INVALID_ARGUMENT;
    lp_batch b = nullptr;
    lp_status s = lp_batch_create(hs, count, hs[0] ? (void*)hs[0]->h.stream : nullptr, &b);
    if (s != LP_OK) return s;
    s = lp_batch_solve(b, o, rs);
    lp_batch_destroy(b);
    return s < 0 ? s : LP_OK;
}

int64_t lp_fishnet_draws(int32_t P)
{
    if (P < 1 || P > 64 || (P & (P - 1)) != 0) return -1;
    return fishnet_draws(P);
}

lp_status lp_fishnet(lp_handle p, const lp_opts* o, int32_t P, int32_t k_steps, const double* G,
                     const double* Z, int64_t nZ, double* x0, double* y0, double* gaps,
                     int32_t* rounds, int32_t memory_space)
{
    if (!p || !o || P < 1 || P > 64 || (P & (P - 1)) != 0 || k_steps < 0 || !G || nZ < 0 ||
        (nZ > 0 && !Z) || !x0 || !y0)
        return LP_INVALID_ARGUMENT;
    if (memory_space != LP_MEM_HOST && memory_space != LP_MEM_DEVICE) return LP_INVALID_ARGUMENT;
    if (check_opts(o) != LP_OK) return LP_INVALID_ARGUMENT;
    if (fishnet_draws(P) > nZ) return LP_INVALID_ARGUMENT;
    Handle* h = &p->h;
    lp_status s = LP_OK;
    try {
        double normK = 0.0, eta0 = 0.0, omega0 = 0.0;
        s = prepare_fp64(h, o, &normK, &eta0, &omega0);
        if (s == LP_OK && o->precision == LP_PREC_MIXED) s = setup_engine<float>(h, o);
        std::vector<double> zh((size_t)nZ);
        if (s == LP_OK && nZ > 0) {
            if (memory_space == LP_MEM_HOST) {
                std::memcpy(zh.data(), Z, sizeof(double) * (size_t)nZ);
            } else if (cudaMemcpy(zh.data(), Z, sizeof(double) * (size_t)nZ,
                                  cudaMemcpyDeviceToHost) != cudaSuccess) {
                s = LP_CUDA_ERROR;
            }
        }
        if (s == LP_OK)
            s = run_fishnet(h, o->precision, eta0, omega0, normK, P, k_steps, G, zh.data(), nZ,
                            x0, y0, gaps, rounds, memory_space);
    } catch (const std::bad_alloc&) {
        s = LP_OUT_OF_MEMORY;
    }
    if (s < 0) {
        cudaStreamSynchronize(h->stream);
        (void)cudaGetLastError();
    }
    return s;
}

lp_status lp_grad(lp_handle p, const lp_opts* o, int32_t K_iters, int32_t ckpt_every,
                  const double* dL_dxK, double* dc, double* dq, double* dvals, double* x_K,
                  int32_t memory_space, double* tau_sigma_out)
{
    if (!p || !o || K_iters < 0 || ckpt_every < 1 || !dL_dxK || !dc || !dq || !dvals)
        return LP_INVALID_ARGUMENT;
    if (memory_space != LP_MEM_HOST && memory_space != LP_MEM_DEVICE) return LP_INVALID_ARGUMENT;
    if (check_opts(o) != LP_OK) return LP_INVALID_ARGUMENT;
    lp_status s = run_grad(&p->h, o, K_iters, ckpt_every, dL_dxK, dc, dq, dvals, x_K,
                           memory_space, tau_sigma_out);
    if (s < 0) {
        cudaStreamSynchronize(p->h.stream);
        (void)cudaGetLastError();
    }
    return s;
}

lp_status lp_unroll(lp_handle p, const lp_opts* o, int32_t K_iters, double* x_K, double* y_K,
                    int32_t memory_space, double* tau_sigma_out)
{
    if (!p || !o || K_iters < 0 || (!x_K && !y_K)) return LP_INVALID_ARGUMENT;
    if (memory_space != LP_MEM_HOST && memory_space != LP_MEM_DEVICE) return LP_INVALID_ARGUMENT;
    lp_status s = check_opts(o);
    if (s != LP_OK) return s;
    s = run_unroll(&p->h, o, K_iters, x_K, y_K, memory_space, tau_sigma_out);
    if (s < 0) {
        cudaStreamSynchronize(p->h.stream);
        (void)cudaGetLastError();
    }
    return s;
}

lp_status lp_update_values(lp_handle p, const double* vals, const double* c, const double* q,
                           const double* l, const double* u, int32_t memory_space)
{
    if (!p) return LP_INVALID_ARGUMENT;
    if (memory_space != LP_MEM_HOST && memory_space != LP_MEM_DEVICE) return LP_INVALID_ARGUMENT;
    lp_status s = setup_update(&p->h, vals, c, q, l, u, memory_space);
    if (s < 0) {
        cudaStreamSynchronize(p->h.stream);
        (void)cudaGetLastError();
    }
    return s;
}

lp_status lp_profile_step(lp_handle p, int32_t precision, int32_t reps, double* ms_out,
                          double* bytes_out)
{
    if (!p || !ms_out || reps < 1) return LP_INVALID_ARGUMENT;
    if (precision == LP_PREC_FP64) return profile_step<double>(&p->h, reps, ms_out, bytes_out);
    if (precision == LP_PREC_MIXED) return profile_step<float>(&p->h, reps, ms_out, bytes_out);
    return LP_INVALID_ARGUMENT;
}

}  // extern "C"
