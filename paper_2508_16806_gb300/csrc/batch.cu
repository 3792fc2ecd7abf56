// Batched restarted PDHG: many independent LPs solved together.
//
// The LPs of a batch form one block-diagonal problem: their CSR matrices are
// stacked (rows and columns offset), so one launch of each kernel works on every
// LP at once and the SpMV load balance is over the whole batch's nonzeros.  What
// stays per LP is everything the paper's method keeps per problem: Ruiz passes
// stop per LP (Algorithm 3), the spectral norm, eta_0 and omega_0 are per LP
// (Algorithm 2, Section 2.4.3), and each LP has its own control block (step size,
// primal weight, restart state, counters, status).  SpMV warp tasks never span two
// LPs; every reduction that feeds a decision is summed per task and then per LP in
// a fixed order, so results are bitwise reproducible.  A task of an LP that is
// done (or waiting for its check) is skipped.  The loop graph has the single
// solver's shape (attempt slots, then the check) and runs while any LP is live.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "control.cuh"
#include "spmv.cuh"

namespace pdhg {

namespace {

constexpr int kBW = 8;   // LPs (warps) per block of the per-LP kernels

inline int grid_n(int64_t count, int nt = kEW, int cap = kEWGrid)
{
    int64_t g = (count + nt - 1) / nt;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

struct BatchMeta {
    int B = 0;
    std::vector<int64_t> row0, col0, nz0;   // host offsets (B + 1)
    int32_t* lp_row = nullptr;   // [m] LP of each row
    int32_t* lp_col = nullptr;   // [n] LP of each column
    double* qn = nullptr;        // [B] ||q_k|| unscaled
    double* cn = nullptr;        // [B] ||c_k|| unscaled
};

// Per-precision task schedule of the batch: LP-aligned warp tasks.
template <typename T>
struct BatchSched {
    bool ready = false;
    bool tuned = false;
    SchedParams pK, pT;                              // task shapes of the two schedules
    int ntK = 0, ntT = 0;
    int32_t *taskK = nullptr, *taskT = nullptr;      // task -> first row (K) / column (K^T)
    int64_t *nzK = nullptr, *nzT = nullptr;          // task -> first nonzero
    int32_t *lpK = nullptr, *lpT = nullptr;          // task -> LP
    int32_t *wbegK = nullptr, *permK = nullptr;      // per-warp task lists (K)
    int32_t *wbegT = nullptr, *permT = nullptr;      // per-warp task lists (K^T)
    // the lists without the tasks of finished LPs (rebuilt at each check) and
    // their ends: list w is permKl[wbegK[w], wendK[w])
    int32_t *permKl = nullptr, *permTl = nullptr, *wendK = nullptr, *wendT = nullptr;
    int wK = 0, wT = 0;                              // lists per schedule
    int32_t *t0K = nullptr, *t0T = nullptr;          // LP -> first task [B + 1]
    double *partK = nullptr, *partT = nullptr;       // per-task step partials [1 | 2][nt]
    double *partR = nullptr, *partC = nullptr;       // per-task check partials [kRowQ | kColQ][nt]
    int gK = 0, gT = 0;
};

}  // namespace

struct BatchHandle {
    Handle h;                    // the stacked problem
    BatchMeta meta;
    BatchSched<double> s64;
    BatchSched<float> s32;
    Ctrl* ctrl = nullptr;        // [B]
    double* lpd = nullptr;       // per-LP scratch [8][B]
    int* go = nullptr;           // per-LP power-iteration flags [B]
    cudaGraphExec_t exec = nullptr;
    int exec_prec = -1, exec_slots = -1, exec_check = -1;
};

namespace {

template <typename T> BatchSched<T>& sched_of(BatchHandle* b);
template <> BatchSched<double>& sched_of<double>(BatchHandle* b) { return b->s64; }
template <> BatchSched<float>& sched_of<float>(BatchHandle* b) { return b->s32; }

// ---------------------------------------------------------------- stacking

__global__ void k_shift_i64(const int64_t* src, int64_t* dst, int64_t count, int64_t add)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = src[t] + add;
}

__global__ void k_shift_i32(const int32_t* src, int32_t* dst, int64_t count, int32_t add)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = src[t] + add;
}

__global__ void k_fill_i32(int32_t* dst, int64_t count, int32_t v)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = v;
}

__global__ void k_fill_f64(double* dst, int64_t count, double v)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = v;
}

// one block per LP: FP64 sum of squares of v over [off[k], off[k+1]) -> out[k]
__global__ void k_lp_sumsq(const double* v, const int64_t* off, double* out)
{
    const int k = blockIdx.x;
    double s = 0.0;
    for (int64_t t = off[k] + threadIdx.x; t < off[k + 1]; t += blockDim.x) s += v[t] * v[t];
    const double a[1] = {s};
    __shared__ double sh[1][kEW / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double w = warp_sum(a[0]);
    if (lane == 0) sh[0][warp] = w;
    __syncthreads();
    if (warp == 0) {
        double t2 = lane < kEW / 32 ? sh[0][lane] : 0.0;
        t2 = warp_sum(t2);
        if (lane == 0) out[k] = t2;
    }
}

// ---------------------------------------------------------------- Ruiz per LP

// per-LP deviation max |1 - norm| (bit pattern max) of non-empty rows / columns
__global__ void k_ruiz_dev_lp(int64_t m, int64_t n, const double* rn, const double* cn,
                              const int32_t* lp_row, const int32_t* lp_col,
                              unsigned long long* dev)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m + n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double v = t < m ? rn[t] : cn[t - m];
        const int k = t < m ? lp_row[t] : lp_col[t - m];
        if (v > 0.0)
            atomicMax(dev + k, (unsigned long long)__double_as_longlong(fabs(1.0 - v)));
    }
}

// LPs whose deviation is within tol stop (sticky); returns the count still going
__global__ void k_ruiz_stop_lp(int B, const unsigned long long* dev, double tol, int* go,
                               int* live)
{
    for (int k = threadIdx.x; k < B; k += blockDim.x) {
        double d;
        const unsigned long long b = dev[k];
        memcpy(&d, &b, sizeof(d));
        if (go[k] && d <= tol) go[k] = 0;
        if (go[k]) atomicAdd(live, 1);
    }
}

// factor 1/sqrt(norm) for a going LP, 1 otherwise (and for empty rows / columns)
__global__ void k_ruiz_factors_lp(int64_t count, double* nrm, double* acc, const int32_t* lp,
                                  const int* go)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double f = (go[lp[t]] && nrm[t] > 0.0) ? 1.0 / sqrt(nrm[t]) : 1.0;
        nrm[t] = f;
        acc[t] *= f;
    }
}

// ---------------------------------------------------------------- per-task epilogues

// out[r] = v; per-task partial of sum out^2 (power iteration); gated per LP
template <typename T>
struct EpiBStore {
    const T* x;
    T* out;
    double* part;            // [ntasks] or nullptr
    const int32_t* task_lp;
    const int* go;           // per-LP gate or nullptr
    const Ctrl* ctrl;        // per-LP gate on want_check or nullptr
    struct Pre {};
    struct Acc { double s2 = 0.0; };
    __device__ bool begin() const { return true; }
    __device__ const T* xin() const { return x; }
    __device__ bool live(int t) const {
        const int k = task_lp[t];
        if (go && !go[k]) return false;
        if (ctrl && !ctrl[k].want_check) return false;
        return true;
    }
    __device__ void task_start(int) {}
    __device__ Pre load(int) const { return Pre{}; }
    __device__ void row(int r, T v, const Pre&, Acc& a) const {
        out[r] = v;
        a.s2 += (double)v * (double)v;
    }
    __device__ void task_done(int t, Acc& a) const {
        const double s = warp_sum(a.s2);
        if (part && (threadIdx.x & 31) == 0) part[t] = s;
        a.s2 = 0.0;
    }
    __device__ void finish(Acc&) const {}
};

// K x' + dual step, per-LP scalars, per-task ||dy||^2 partial
template <typename T>
struct EpiBDual {
    const Ctrl* ctrl;
    const int32_t* task_lp;
    const T* xs0; const T* xs1;
    T* y0; T* y1; T* kx0; T* kx1;
    T* ys;
    const T* q;
    const uint8_t* sense;
    double* part;
    int cur = 0; T sigma = 0; T pw = 0; int adapt = 0;
    struct Pre { T y = 0, kx = 0, q = 0, ys = 0; uint8_t ge = 0; };
    struct Acc { T dy2 = T(0); };   // per-lane sums in T, reduced in FP64
    __device__ bool begin() const { return true; }
    __device__ const T* xin() const { return cur ? xs0 : xs1; }   // x' of the task's LP
    __device__ bool live(int t) const { return !ctrl[task_lp[t]].skip; }
    __device__ void task_start(int t) {
        const Ctrl& c = ctrl[task_lp[t]];
        cur = c.cur;
        sigma = step_scalars<T>(c).sigma;
        pw = step_scalars<T>(c).pw;
        adapt = c.adaptive;
    }
    __device__ Pre load(int i) const {
        Pre p;
        p.y = (cur ? y1 : y0)[i];
        p.kx = (cur ? kx1 : kx0)[i];
        p.q = q[i];
        p.ge = sense[i];
        if (pw != T(0)) p.ys = ys[i];
        return p;
    }
    __device__ void row(int i, T kxn, const Pre& p, Acc& a) const {
        if (pw != T(0)) ys[i] = p.ys + pw * p.y;
        T v = p.y + sigma * (p.q - (T(2) * kxn - p.kx));
        if (p.ge && v < T(0)) v = T(0);
        (cur ? y0 : y1)[i] = v;
        (cur ? kx0 : kx1)[i] = kxn;
        const T d = v - p.y;
        a.dy2 += d * d;
    }
    __device__ void task_done(int t, Acc& a) const {
        const double s = warp_sum((double)a.dy2);
        if (adapt && (threadIdx.x & 31) == 0) part[t] = s;
        a.dy2 = T(0);
    }
    __device__ void finish(Acc&) const {}
};

// K^T y' + Algorithm 5 terms, per-task partials
template <typename T>
struct EpiBPrimalT {
    const Ctrl* ctrl;
    const int32_t* task_lp;
    const T* ys0; const T* ys1;
    const T* x0; const T* x1;
    T* kty0; T* kty1;
    double* part;            // [2][ntasks]
    int ntasks;
    int cur = 0; int adapt = 0;
    struct Pre { T x = 0, xn = 0, kt = 0; };
    struct Acc { T dx2 = T(0), inter = T(0); };   // per-lane sums in T, reduced in FP64
    __device__ bool begin() const { return true; }
    __device__ const T* xin() const { return cur ? ys0 : ys1; }   // y' of the task's LP
    __device__ bool live(int t) const { return !ctrl[task_lp[t]].skip; }
    __device__ void task_start(int t) {
        const Ctrl& c = ctrl[task_lp[t]];
        cur = c.cur;
        adapt = c.adaptive;
    }
    __device__ Pre load(int j) const {
        Pre p;
        if (adapt) {
            p.x = (cur ? x1 : x0)[j];
            p.xn = (cur ? x0 : x1)[j];
            p.kt = (cur ? kty1 : kty0)[j];
        }
        return p;
    }
    __device__ void row(int j, T ktyn, const Pre& p, Acc& a) const {
        (cur ? kty0 : kty1)[j] = ktyn;
        if (adapt) {
            const T dx = p.xn - p.x;
            a.dx2 += dx * dx;
            a.inter += dx * (ktyn - p.kt);
        }
    }
    __device__ void task_done(int t, Acc& a) const {
        const double s0 = warp_sum((double)a.dx2), s1 = warp_sum((double)a.inter);
        if (adapt && (threadIdx.x & 31) == 0) {
            part[t] = s0;
            part[(size_t)ntasks + t] = s1;
        }
        a.dx2 = a.inter = T(0);
    }
    __device__ void finish(Acc&) const {}
};

// ---------------------------------------------------------------- step kernels

template <typename T>
__global__ void __launch_bounds__(kEW)
kb_primal(const Ctrl* __restrict__ ctrl, const int32_t* __restrict__ lp_col, T* x0, T* x1,
          const T* kty0, const T* kty1, const T* c, const T* l, const T* u, T* xs, int64_t n)
{
    for (int64_t j = (int64_t)blockIdx.x * kEW + threadIdx.x; j < n; j += (int64_t)gridDim.x * kEW) {
        const Ctrl& C = ctrl[lp_col[j]];
        if (C.skip) continue;
        const int cur = C.cur;
        const StepScalars<T>& sc = step_scalars<T>(C);
        const T tau = sc.tau;
        const T pw = sc.pw;
        const T xj = (cur ? x1 : x0)[j];
        if (pw != T(0)) xs[j] += pw * xj;
        T v = xj - tau * (c[j] - (cur ? kty1 : kty0)[j]);
        if (v < l[j]) v = l[j];
        if (v > u[j]) v = u[j];
        (cur ? x0 : x1)[j] = v;
    }
}

// warp-level fixed-order sum of part[a, b)
__device__ __forceinline__ double warp_range_sum(const double* part, int a, int b)
{
    const int lane = threadIdx.x & 31;
    // four independent loads in flight per lane, fixed order
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = a + lane;
    for (; i + 3 * 32 < b; i += 4 * 32) {
        s0 += __ldcg(part + i);
        s1 += __ldcg(part + i + 32);
        s2 += __ldcg(part + i + 64);
        s3 += __ldcg(part + i + 96);
    }
    for (; i < b; i += 32) s0 += __ldcg(part + i);
    return warp_sum((s0 + s1) + (s2 + s3));   // lane 0
}

// maximum of part[a..b) (0 when empty) by one warp; the result is valid in lane 0
__device__ double warp_range_max(const double* part, int a, int b)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = a + lane; i < b; i += 32) s = fmax(s, __ldcg(part + i));
    return warp_max(s);   // lane 0
}

// one warp per LP: Algorithm 5 decision from the LP's task partials
__global__ void kb_step_ctrl(Ctrl* ctrl, int B, const int32_t* t0K, const int32_t* t0T,
                             const double* partK, const double* partT, int ntT)
{
    const int k = blockIdx.x * kBW + (threadIdx.x >> 5);
    if (k >= B) return;
    Ctrl* c = ctrl + k;
    if (c->skip) return;
    double dy2 = 0.0, dx2 = 0.0, inter = 0.0;
    if (c->adaptive) {
        dy2 = warp_range_sum(partK, t0K[k], t0K[k + 1]);
        dx2 = warp_range_sum(partT, t0T[k], t0T[k + 1]);
        inter = warp_range_sum(partT + ntT, t0T[k], t0T[k + 1]);
    }
    if ((threadIdx.x & 31) == 0) step_decide(c, c->adaptive, dy2, dx2, inter);
}

// ---------------------------------------------------------------- check kernels

template <typename T>
__global__ void __launch_bounds__(kEW)
kb_check_prep(const Ctrl* __restrict__ ctrl, const int32_t* lp_row, const int32_t* lp_col,
              const T* x0, const T* x1, const T* y0, const T* y1, T* xs, T* ys, T* xa, T* ya,
              const T* l, const T* u, const uint8_t* sense, int64_t n, int64_t m)
{
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * kEW) {
        if (t < n) {
            const Ctrl& C = ctrl[lp_col[t]];
            if (!C.want_check) continue;
            const T pw = step_scalars<T>(C).pw;
            T s = xs[t];
            if (pw != T(0)) { s += pw * (C.cur ? x1 : x0)[t]; xs[t] = s; }
            T a = s * step_scalars<T>(C).winv;
            if (a < l[t]) a = l[t];
            if (a > u[t]) a = u[t];
            xa[t] = a;
        } else {
            const int64_t i = t - n;
            const Ctrl& C = ctrl[lp_row[i]];
            if (!C.want_check) continue;
            const T pw = step_scalars<T>(C).pw;
            T s = ys[i];
            if (pw != T(0)) { s += pw * (C.cur ? y1 : y0)[i]; ys[i] = s; }
            T a = s * step_scalars<T>(C).winv;
            if (sense[i] && a < T(0)) a = T(0);
            ya[i] = a;
        }
    }
}

// one warp per K task: the row-side terms of RowCheck over the task's rows
template <typename T>
__global__ void kb_check_rows(const Ctrl* ctrl, const int32_t* taskK, const int32_t* lpK, int ntK,
                              const T* y0, const T* y1, const T* kx0, const T* kx1, const T* ya,
                              const T* kxa, const T* yanc, const T* q, const uint8_t* sense,
                              const T* R, const T* Rinv, double* part)
{
    const int t = blockIdx.x * (kEW / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= ntK) return;
    const Ctrl& C = ctrl[lpK[t]];
    if (!C.want_check) return;
    const bool inf = infeas_active(C);
    const T* y = C.cur ? y1 : y0;
    const T* kx = C.cur ? kx1 : kx0;
    const T* yp = C.cur ? y0 : y1;
    const T* kxp = C.cur ? kx0 : kx1;
    RowCheck<T> rc;
    for (int i = taskK[t] + lane; i < taskK[t + 1]; i += 32) {
        const T qi = q[i], ri = Rinv[i], kxi = kx[i], yi = y[i];
        const bool ge = sense[i] != 0;
        rc.add(qi, kxi, yi, kxa[i], ya[i], yanc[i], ri, ge);
        if (inf) rc.add_infeas(qi, kxi, kxp[i], yi, yp[i], R[i], ri, ge);
    }
#pragma unroll
    for (int qq = 0; qq < kRowQ; ++qq) {
        const double s = qq < kRowSums ? warp_sum((double)rc.v[qq])
                                       : warp_max((double)rc.mx[qq - kRowSums]);
        if (lane == 0) part[(size_t)qq * ntK + t] = s;
    }
}

// one warp per K^T task: the column-side terms of ColCheck
template <typename T>
__global__ void kb_check_cols(const Ctrl* ctrl, const int32_t* taskT, const int32_t* lpT, int ntT,
                              const T* x0, const T* x1, const T* kty0, const T* kty1, const T* xa,
                              const T* ktya, const T* xanc, const T* c, const T* l, const T* u,
                              const T* Cs, const T* Cinv, double* part)
{
    const int t = blockIdx.x * (kEW / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= ntT) return;
    const Ctrl& CC = ctrl[lpT[t]];
    if (!CC.want_check) return;
    const bool inf = infeas_active(CC);
    const T* x = CC.cur ? x1 : x0;
    const T* kty = CC.cur ? kty1 : kty0;
    const T* xp = CC.cur ? x0 : x1;
    const T* ktyp = CC.cur ? kty0 : kty1;
    ColCheck<T> cc;
    for (int j = taskT[t] + lane; j < taskT[t + 1]; j += 32) {
        const T cj = c[j], lj = l[j], uj = u[j], ci = Cinv[j], xj = x[j], kj = kty[j];
        const T xan = xanc[j];
        const bool lf = isfinite(lj), uf = isfinite(uj);
        cc.side(0, cj, kj, xj, xan, lj, uj, ci, lf, uf);
        cc.side(1, cj, ktya[j], xa[j], xan, lj, uj, ci, lf, uf);
        if (inf) cc.add_infeas(cj, xj, xp[j], kj, ktyp[j], lj, uj, Cs[j], ci, lf, uf);
    }
#pragma unroll
    for (int qq = 0; qq < kColQ; ++qq) {
        const double s = qq < kColSums ? warp_sum((double)cc.v[qq])
                                       : warp_max((double)cc.mx[qq - kColSums]);
        if (lane == 0) part[(size_t)qq * ntT + t] = s;
    }
}

// one warp per LP: the check decision from the LP's task partials
__global__ void kb_check_ctrl(Ctrl* ctrl, int B, const int32_t* t0K, const int32_t* t0T,
                              const double* partR, int ntK, const double* partC, int ntT)
{
    const int k = blockIdx.x * kBW + (threadIdx.x >> 5);
    if (k >= B) return;
    Ctrl* c = ctrl + k;
    if (!c->want_check) return;
    double r[kRowQ], cc[kColQ];
    for (int q = 0; q < kRowQ; ++q)
        r[q] = q < kRowSums ? warp_range_sum(partR + (size_t)q * ntK, t0K[k], t0K[k + 1])
                            : warp_range_max(partR + (size_t)q * ntK, t0K[k], t0K[k + 1]);
    for (int q = 0; q < kColQ; ++q)
        cc[q] = q < kColSums ? warp_range_sum(partC + (size_t)q * ntT, t0T[k], t0T[k + 1])
                             : warp_range_max(partC + (size_t)q * ntT, t0T[k], t0T[k + 1]);
    if ((threadIdx.x & 31) == 0) check_decide(c, r, cc, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(kEW)
kb_restart_apply(const Ctrl* __restrict__ ctrl, const int32_t* lp_row, const int32_t* lp_col,
                 T* x0, T* x1, T* y0, T* y1, T* kx0, T* kx1, T* kty0, T* kty1, const T* xa,
                 const T* ya, const T* kxa, const T* ktya, T* xanc, T* yanc, T* xs, T* ys,
                 int64_t n, int64_t m)
{
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * kEW) {
        const bool col = t < n;
        const int64_t i = col ? t : t - n;
        const Ctrl& C = ctrl[col ? lp_col[i] : lp_row[i]];
        if (!C.want_check || !C.restart) continue;
        const int cur = C.cur, avg = C.cand_avg;
        if (col) {
            T* x = cur ? x1 : x0;
            T v = x[i];
            if (avg) {
                v = xa[i];
                x[i] = v;
                (cur ? kty1 : kty0)[i] = ktya[i];
            }
            xanc[i] = v;
            xs[i] = T(0);
        } else {
            T* y = cur ? y1 : y0;
            T v = y[i];
            if (avg) {
                v = ya[i];
                y[i] = v;
                (cur ? kx1 : kx0)[i] = kxa[i];
            }
            yanc[i] = v;
            ys[i] = T(0);
        }
    }
}

__global__ void kb_set_cond(Ctrl* ctrl, int B, cudaGraphConditionalHandle handle, int use_handle,
                            int in_body, int* any_live)
{
    __shared__ int live;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < B; k += blockDim.x) {
        Ctrl* c = ctrl + k;
        if (in_body && !c->done) c->bodies += 1;
        c->want_check = 0;
        c->restart = 0;
        c->skip = c->done;
        if (!c->done) atomicAdd(&live, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (any_live) *any_live = live;
        if (use_handle) cudaGraphSetConditional(handle, live ? 1u : 0u);
    }
}

// ---------------------------------------------------------------- setup kernels

// per-LP step sizes and weights from the per-LP sums; control blocks initialised
// prev (nullptr, or the control blocks of an FP32 phase): an LP that phase
// declared optimal continues from its step size, primal weight and counters
// (its first check is the FP64 confirmation); any other LP keeps its outcome and
// takes no part (done; its result is the warm start, X[0] / Y[0]).
__global__ void kb_init_ctrl(Ctrl* ctrl, int B, const double* normK, const double* cs2,
                             const double* qs2, const double* qn, const double* cn, Ctrl tmpl,
                             double eta_scale, double eta0, double omega0, double eps_zero,
                             unsigned long long t0, const Ctrl* prev)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < B; k += gridDim.x * blockDim.x) {
        Ctrl c = tmpl;
        const double nk = normK[k];
        c.eta = eta0 > 0.0 ? eta0 : (nk > 0.0 ? eta_scale / nk : 1.0);
        const double a = sqrt(cs2[k]), b = sqrt(qs2[k]);
        c.omega = omega0 > 0.0 ? omega0 : ((a > eps_zero && b > eps_zero) ? a / b : 1.0);
        c.qnorm = qn[k];
        c.cnorm = cn[k];
        c.t0_ns = (long long)t0;
        if (prev) {
            const Ctrl& p = prev[k];
            if (p.status == LP_OPTIMAL) {
                c.eta = p.eta;
                c.omega = p.omega;
                c.k = p.k;
                c.attempts = p.attempts;
                c.restarts = p.restarts;
                c.t0_ns = p.t0_ns;
            } else {
                c = p;
                c.done = 1;
                c.skip = 1;
                c.want_check = 0;
                c.cur = 0;
                c.cand_avg = 0;
            }
        }
        refresh_scalars(c);
        ctrl[k] = c;
    }
}

// one warp per LP: b-norm from task partials; 1/||b|| into inv[k] (0 stops the LP)
__global__ void kb_pow_norm(int B, const int32_t* t0, const double* part, double* inv, int* go,
                            double* out_norm)
{
    const int k = blockIdx.x * kBW + (threadIdx.x >> 5);
    if (k >= B) return;
    const double s = warp_range_sum(part, t0[k], t0[k + 1]);
    if ((threadIdx.x & 31) == 0) {
        if (out_norm) {
            out_norm[k] = sqrt(s);
        } else if (go[k]) {
            const double nb = sqrt(s);
            if (nb == 0.0) go[k] = 0;
            inv[k] = nb;
        }
    }
}

__global__ void kb_pow_scale(double* b, const int32_t* lp_col, const double* nb, const int* go,
                             int64_t n)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int k = lp_col[j];
        if (go[k]) b[j] = b[j] / nb[k];
    }
}

// Start point x = proj_X(0), y = 0, or the unscaled warm start w (n + m
// values: x then y) moved to scaled space and projected.
template <typename T>
__global__ void kb_init_state(T* x, T* y, T* xanc, T* yanc, T* xs, T* ys, const T* l, const T* u,
                              int64_t n, int64_t m, const double* w, const double* R,
                              const double* C, const uint8_t* sense)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n) {
            T v = w ? (T)(w[t] / C[t]) : T(0);
            if (v < l[t]) v = l[t];
            if (v > u[t]) v = u[t];
            x[t] = v;
            xanc[t] = v;
            xs[t] = T(0);
        } else {
            const int64_t i = t - n;
            T v = w ? (T)(w[t] / R[i]) : T(0);
            if (w && sense[i] && v < T(0)) v = T(0);
            y[i] = v;
            yanc[i] = v;
            ys[i] = T(0);
        }
    }
}

template <typename T>
__global__ void kb_extract(const Ctrl* ctrl, const int32_t* lp_row, const int32_t* lp_col,
                           const T* x0, const T* x1, const T* y0, const T* y1, const T* xa,
                           const T* ya, const double* R, const double* C, double* xo, double* yo,
                           int64_t n, int64_t m)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n) {
            const Ctrl& c = ctrl[lp_col[t]];
            const T* x = c.cand_avg ? xa : (c.cur ? x1 : x0);
            xo[t] = C[t] * (double)x[t];
        } else {
            const int64_t i = t - n;
            const Ctrl& c = ctrl[lp_row[i]];
            const T* y = c.cand_avg ? ya : (c.cur ? y1 : y0);
            yo[i] = R[i] * (double)y[i];
        }
    }
}

__global__ void kb_read_clock(unsigned long long* t) { *t = global_ns(); }

// ---------------------------------------------------------------- host

// LP-aligned task boundaries over all rows (K: rows = true, K^T: columns)
std::vector<int32_t> batch_blocks(BatchHandle* bh, bool rows, SchedParams p)
{
    Handle* h = &bh->h;
    std::vector<int32_t> out;
    for (int k = 0; k < bh->meta.B; ++k) {
        const int64_t a = rows ? bh->meta.row0[k] : bh->meta.col0[k];
        const int64_t b = rows ? bh->meta.row0[k + 1] : bh->meta.col0[k + 1];
        const int64_t* rp = (rows ? h->h_rp.data() : h->h_trp.data()) + a;
        std::vector<int32_t> t = make_row_blocks(rp, b - a, p.cap, p.max_rows);
        for (size_t i = 0; i + 1 < t.size(); ++i) out.push_back((int32_t)(t[i] + a));
    }
    out.push_back((int32_t)(rows ? h->m : h->n));
    return out;
}

// Builds (or rebuilds with other task shapes) the LP-aligned schedules and the
// per-task partials of precision T.
template <typename T>
lp_status build_sched(BatchHandle* bh, SchedParams pK, SchedParams pT)
{
    BatchSched<T>& S = sched_of<T>(bh);
    if (S.ready && S.pK.cap == pK.cap && S.pK.max_rows == pK.max_rows && S.pT.cap == pT.cap &&
        S.pT.max_rows == pT.max_rows)
        return LP_OK;
    Handle* h = &bh->h;
    const int B = bh->meta.B;
    if (S.ready) {
        for (void* p : {(void*)S.taskK, (void*)S.taskT, (void*)S.lpK, (void*)S.lpT,
                        (void*)S.t0K, (void*)S.t0T, (void*)S.nzK, (void*)S.nzT, (void*)S.partK,
                        (void*)S.partT, (void*)S.partR, (void*)S.partC, (void*)S.wbegK,
                        (void*)S.permK, (void*)S.wbegT, (void*)S.permT, (void*)S.permKl,
                        (void*)S.permTl, (void*)S.wendK, (void*)S.wendT})
            dev_free(h, p);
    }
    std::vector<int32_t> tK, tT, lK, lT, k0(B + 1), c0(B + 1);
    std::vector<int64_t> nK, nT;
    for (int k = 0; k < B; ++k) {
        k0[k] = (int32_t)tK.size();
        c0[k] = (int32_t)tT.size();
        const int64_t r0 = bh->meta.row0[k], r1 = bh->meta.row0[k + 1];
        const int64_t q0 = bh->meta.col0[k], q1 = bh->meta.col0[k + 1];
        std::vector<int32_t> a =
            make_row_blocks(h->h_rp.data() + r0, r1 - r0, pK.cap, pK.max_rows);
        std::vector<int32_t> c =
            make_row_blocks(h->h_trp.data() + q0, q1 - q0, pT.cap, pT.max_rows);
        for (size_t i = 0; i + 1 < a.size(); ++i) {
            tK.push_back((int32_t)(a[i] + r0));
            lK.push_back(k);
        }
        for (size_t i = 0; i + 1 < c.size(); ++i) {
            tT.push_back((int32_t)(c[i] + q0));
            lT.push_back(k);
        }
    }
    k0[B] = (int32_t)tK.size();
    c0[B] = (int32_t)tT.size();
    tK.push_back((int32_t)h->m);
    tT.push_back((int32_t)h->n);
    for (int32_t r : tK) nK.push_back(h->h_rp[(size_t)r]);
    for (int32_t r : tT) nT.push_back(h->h_trp[(size_t)r]);
    S.ntK = (int)lK.size();
    S.ntT = (int)lT.size();
    int sms = 0;
    LP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    S.gK = spmv_grid<T>(S.ntK, sms);
    S.gT = spmv_grid<T>(S.ntT, sms);
    std::vector<int32_t> wk, pk, wt, pt;
    assign_tasks(nK, pK.cap, S.gK * kSpmvWorkers, wk, pk);
    assign_tasks(nT, pT.cap, S.gT * kSpmvWorkers, wt, pt);
    auto up32 = [&](int32_t** d, const std::vector<int32_t>& v) -> lp_status {
        LP_TRY(dev_alloc_n(h, d, v.size()));
        LP_CUDA_TRY(cudaMemcpyAsync(*d, v.data(), v.size() * 4, cudaMemcpyHostToDevice, h->stream));
        return LP_OK;
    };
    auto up64 = [&](int64_t** d, const std::vector<int64_t>& v) -> lp_status {
        LP_TRY(dev_alloc_n(h, d, v.size()));
        LP_CUDA_TRY(cudaMemcpyAsync(*d, v.data(), v.size() * 8, cudaMemcpyHostToDevice, h->stream));
        return LP_OK;
    };
    LP_TRY(up32(&S.taskK, tK));
    LP_TRY(up32(&S.taskT, tT));
    LP_TRY(up32(&S.lpK, lK));
    LP_TRY(up32(&S.lpT, lT));
    LP_TRY(up32(&S.t0K, k0));
    LP_TRY(up32(&S.t0T, c0));
    LP_TRY(up64(&S.nzK, nK));
    LP_TRY(up64(&S.nzT, nT));
    LP_TRY(up32(&S.wbegK, wk));
    LP_TRY(up32(&S.permK, pk));
    LP_TRY(up32(&S.wbegT, wt));
    LP_TRY(up32(&S.permT, pt));
    S.wK = (int)wk.size() - 1;
    S.wT = (int)wt.size() - 1;
    LP_TRY(dev_alloc_n(h, &S.permKl, pk.size() + 1));
    LP_TRY(dev_alloc_n(h, &S.permTl, pt.size() + 1));
    LP_TRY(dev_alloc_n(h, &S.wendK, (size_t)S.wK + 1));
    LP_TRY(dev_alloc_n(h, &S.wendT, (size_t)S.wT + 1));
    LP_TRY(dev_alloc_n(h, &S.partK, (size_t)S.ntK + 8));
    LP_TRY(dev_alloc_n(h, &S.partT, 2 * (size_t)S.ntT + 8));
    LP_TRY(dev_alloc_n(h, &S.partR, kRowQ * (size_t)S.ntK + 8));
    LP_TRY(dev_alloc_n(h, &S.partC, kColQ * (size_t)S.ntT + 8));
    LP_CUDA_TRY(cudaStreamSynchronize(h->stream));
    S.pK = pK;
    S.pT = pT;
    // vectors and scaled data of this precision
    Engine<T>& E = engine_of<T>(h);
    if (!E.ready) {
        const int64_t m = h->m, n = h->n, nnz = h->nnz;
        LP_TRY(dev_alloc_n(h, &E.val, pad8(nnz)));
        LP_TRY(dev_alloc_n(h, &E.tval, pad8(nnz)));
        LP_CUDA_TRY(cudaMemsetAsync(E.val, 0, pad8(nnz) * sizeof(T), h->stream));
        LP_CUDA_TRY(cudaMemsetAsync(E.tval, 0, pad8(nnz) * sizeof(T), h->stream));
        T** vn[] = {&E.c, &E.l, &E.u, &E.X[0], &E.X[1], &E.KTY[0], &E.KTY[1],
                    &E.XS, &E.XA, &E.KTYA, &E.XANC};
        for (T** p : vn) LP_TRY(dev_alloc_n(h, p, (size_t)n));
        T** vm[] = {&E.q, &E.Y[0], &E.Y[1], &E.KX[0], &E.KX[1], &E.YS, &E.YA, &E.KXA, &E.YANC};
        for (T** p : vm) LP_TRY(dev_alloc_n(h, p, (size_t)m));
        E.ready = true;
    }
    S.ready = true;
    return LP_OK;
}

template <typename T>
lp_status ensure_sched(BatchHandle* bh)
{
    if (sched_of<T>(bh).ready) return LP_OK;
    const SchedParams d{cap_w<T>(), kTaskRows};
    return build_sched<T>(bh, d, d);
}

// Autotuner of the batch schedules (once per precision): candidate task shapes
// are timed on the stacked matrix with this precision's values; a change
// rebuilds the schedules and drops the captured loop graph.
template <typename T>
lp_status tune_batch(BatchHandle* bh)
{
    BatchSched<T>& S = sched_of<T>(bh);
    if (S.tuned) return LP_OK;
    Handle* h = &bh->h;
    Engine<T>& E = engine_of<T>(h);
    int sms = 0;
    LP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    LP_CUDA_TRY(cudaMemsetAsync(E.XA, 0, sizeof(T) * (size_t)h->n, h->stream));
    LP_CUDA_TRY(cudaMemsetAsync(E.YA, 0, sizeof(T) * (size_t)h->m, h->stream));
    SchedParams pK, pT;
    float msK = 0.0f, msT = 0.0f;
    LP_TRY(tune_schedule<T>(
        sms, h->stream, [&](int cap, int rows) { return batch_blocks(bh, true, {cap, rows}); },
        h->h_rp.data(), h->rp, h->ci, E.val, E.XA, E.KXA, h->n, h->dev_err, &pK, &msK));
    LP_TRY(tune_schedule<T>(
        sms, h->stream, [&](int cap, int rows) { return batch_blocks(bh, false, {cap, rows}); },
        h->h_trp.data(), h->trp, h->tci, E.tval, E.YA, E.KTYA, h->m, h->dev_err, &pT, &msT));
    h->launches += 2 * 6 * 4;
    if (pK.cap != S.pK.cap || pK.max_rows != S.pK.max_rows || pT.cap != S.pT.cap ||
        pT.max_rows != S.pT.max_rows) {
        LP_TRY(build_sched<T>(bh, pK, pT));
        if (bh->exec) {
            cudaGraphExecDestroy(bh->exec);
            bh->exec = nullptr;
        }
    }
    S.tuned = true;
    return LP_OK;
}

template <typename T>
__global__ void kb_cast(const double* src, const int32_t* perm, T* dst, int64_t count)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (T)src[perm ? perm[t] : t];
}

// Ruiz per LP into e64 (values, vectors) and R, C; spectral norm per LP.
lp_status batch_scale(BatchHandle* bh, const lp_opts* o, double* normK_dev)
{
    Handle* h = &bh->h;
    const int B = bh->meta.B;
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    cudaStream_t st = h->stream;
    LP_TRY(ensure_sched<double>(bh));
    Engine<double>& E = h->e64;
    BatchSched<double>& S = bh->s64;
    LP_CUDA_TRY(cudaMemcpyAsync(E.val, h->val0, pad8(nnz) * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
    // tuned before the power iteration uses it (same order of sums in every solve)
    if (o->autotune) LP_TRY(tune_batch<double>(bh));
    k_fill_f64<<<grid_n(m, 256, 65535), 256, 0, st>>>(h->R, m, 1.0);
    k_fill_f64<<<grid_n(n, 256, 65535), 256, 0, st>>>(h->C, n, 1.0);
    double* rn = h->scratch;
    double* cn = h->scratch + m;
    unsigned long long* dev = reinterpret_cast<unsigned long long*>(bh->lpd);
    int* live = reinterpret_cast<int*>(bh->lpd + B);
    k_fill_i32<<<grid_n(B, 256, 4096), 256, 0, st>>>(reinterpret_cast<int32_t*>(bh->go), B, 1);
    for (int it = 0; it < o->ruiz_iters; ++it) {
        k_row_inf<<<grid_n(m * 32, 256, 65535 * 8), 256, 0, st>>>(m, h->rp, E.val, rn);
        LP_CUDA_TRY(cudaMemsetAsync(cn, 0, sizeof(double) * (size_t)n, st));
        k_col_inf<<<grid_n(nnz, 256, 8192), 256, 0, st>>>(
            nnz, h->ci, E.val, reinterpret_cast<unsigned long long*>(cn));
        LP_CUDA_TRY(cudaMemsetAsync(dev, 0, sizeof(unsigned long long) * B, st));
        k_ruiz_dev_lp<<<grid_n(m + n, 256, 4096), 256, 0, st>>>(m, n, rn, cn, bh->meta.lp_row,
                                                                bh->meta.lp_col, dev);
        LP_CUDA_TRY(cudaMemsetAsync(live, 0, sizeof(int), st));
        k_ruiz_stop_lp<<<1, 256, 0, st>>>(B, dev, o->ruiz_tol, bh->go, live);
        int hl = 0;
        LP_CUDA_TRY(cudaMemcpyAsync(&hl, live, sizeof(int), cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
        if (hl == 0) break;
        k_ruiz_factors_lp<<<grid_n(m, 256, 65535), 256, 0, st>>>(m, rn, h->R, bh->meta.lp_row,
                                                                 bh->go);
        k_ruiz_factors_lp<<<grid_n(n, 256, 65535), 256, 0, st>>>(n, cn, h->C, bh->meta.lp_col,
                                                                 bh->go);
        k_scale_vals<<<grid_n(nnz, 256, 8192), 256, 0, st>>>(nnz, h->krow, h->ci, rn, cn, E.val);
        h->launches += 7;
        LP_CUDA_TRY(cudaGetLastError());
    }
    if (o->pock_chambolle) {
        k_pc_sums<<<grid_n(m + n, 256, 65535), 256, 0, st>>>(m, n, h->rp, h->trp, h->tperm, E.val,
                                                             o->pc_alpha, rn, cn);
        k_ruiz_factors<<<grid_n(m, 256, 65535), 256, 0, st>>>(m, rn, h->R);
        k_ruiz_factors<<<grid_n(n, 256, 65535), 256, 0, st>>>(n, cn, h->C);
        k_scale_vals<<<grid_n(nnz, 256, 8192), 256, 0, st>>>(nnz, h->krow, h->ci, rn, cn, E.val);
        h->launches += 4;
    }
    k_scale_vectors<<<grid_n(m + n, 256, 65535), 256, 0, st>>>(m, n, h->R, h->C, h->c0, h->q0,
                                                               h->l0, h->u0, E.c, E.q, E.l, E.u);
    kb_cast<double><<<grid_n(nnz, 256, 8192), 256, 0, st>>>(E.val, h->tperm, E.tval, nnz);
    h->launches += 2;
    LP_CUDA_TRY(cudaGetLastError());
    // Algorithm 2 per LP
    LP_CUDA_TRY((spmv_prepare<double, EpiBStore<double>>()));
    double* b = E.XA;
    double* t = E.KXA;
    double* nb = bh->lpd + 2 * B;
    k_fill_f64<<<grid_n(n, 256, 65535), 256, 0, st>>>(b, n, 1.0);
    k_fill_i32<<<grid_n(B, 256, 4096), 256, 0, st>>>(reinterpret_cast<int32_t*>(bh->go), B, 1);
    for (int it = 0; it < o->power_iters; ++it) {
        EpiBStore<double> e1{b, t, nullptr, S.lpK, bh->go, nullptr};
        launch_spmv<double>(S.gK, st, S.taskK, S.nzK, S.ntK, S.wbegK, S.permK, h->rp, h->ci, E.val, h->dev_err, n, e1);
        EpiBStore<double> e2{t, b, S.partT, S.lpT, bh->go, nullptr};
        launch_spmv<double>(S.gT, st, S.taskT, S.nzT, S.ntT, S.wbegT, S.permT, h->trp, h->tci, E.tval, h->dev_err, m,
                            e2);
        kb_pow_norm<<<(B + kBW - 1) / kBW, kBW * 32, 0, st>>>(B, S.t0T, S.partT, nb, bh->go,
                                                              nullptr);
        kb_pow_scale<<<grid_n(n, 256, 65535), 256, 0, st>>>(b, bh->meta.lp_col, nb, bh->go, n);
        h->launches += 4;
    }
    EpiBStore<double> e3{b, t, S.partK, S.lpK, nullptr, nullptr};
    launch_spmv<double>(S.gK, st, S.taskK, S.nzK, S.ntK, S.wbegK, S.permK, h->rp, h->ci, E.val, h->dev_err, n, e3);
    kb_pow_norm<<<(B + kBW - 1) / kBW, kBW * 32, 0, st>>>(B, S.t0K, S.partK, nullptr, bh->go,
                                                          normK_dev);
    h->launches += 2;
    LP_CUDA_TRY(cudaGetLastError());
    return LP_OK;
}

// The task lists without the tasks of finished LPs: one warp per list keeps,
// in order, the entries of perm[wbeg[w], wbeg[w + 1]) whose LP is not done and
// writes them to perm_live from wbeg[w] on; wend[w] is where they end.  Late in
// a batched solve most LPs have finished, and the SpMV's lists would otherwise
// step over their tasks one by one at every launch.
__global__ void kb_compact_tasks(const int32_t* __restrict__ wbeg, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ task_lp, const Ctrl* __restrict__ ctrl,
                                 int workers, int32_t* __restrict__ perm_live,
                                 int32_t* __restrict__ wend)
{
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= workers) return;
    const int b = wbeg[w], e = wbeg[w + 1];
    int out = b;
    for (int p0 = b; p0 < e; p0 += 32) {
        const int p = p0 + lane;
        int t = 0;
        bool keep = false;
        if (p < e) {
            t = perm[p];
            keep = !ctrl[task_lp[t]].done;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (keep) perm_live[out + __popc(mask & ((1u << lane) - 1u))] = t;
        out += __popc(mask);
    }
    if (lane == 0) wend[w] = out;
}

template <typename T>
void b_compact(BatchHandle* bh, cudaStream_t st)
{
    BatchSched<T>& S = sched_of<T>(bh);
    kb_compact_tasks<<<(S.wK * 32 + 255) / 256, 256, 0, st>>>(S.wbegK, S.permK, S.lpK, bh->ctrl,
                                                             S.wK, S.permKl, S.wendK);
    kb_compact_tasks<<<(S.wT * 32 + 255) / 256, 256, 0, st>>>(S.wbegT, S.permT, S.lpT, bh->ctrl,
                                                             S.wT, S.permTl, S.wendT);
}

template <typename T>
void b_launch_attempt(BatchHandle* bh, cudaStream_t st)
{
    Handle* h = &bh->h;
    Engine<T>& E = engine_of<T>(h);
    BatchSched<T>& S = sched_of<T>(bh);
    kb_primal<T><<<grid_n(h->n), kEW, 0, st>>>(bh->ctrl, bh->meta.lp_col, E.X[0], E.X[1], E.KTY[0],
                                                E.KTY[1], E.c, E.l, E.u, E.XS, h->n);
    EpiBDual<T> ed{bh->ctrl, S.lpK, E.X[0], E.X[1], E.Y[0], E.Y[1], E.KX[0], E.KX[1], E.YS,
                   E.q, h->sense, S.partK};
    SplitRows lK, lT;
    lK.wend = S.wendK;
    lT.wend = S.wendT;
    launch_spmv<T>(S.gK, st, S.taskK, S.nzK, S.ntK, S.wbegK, S.permKl, h->rp, h->ci, E.val, h->dev_err,
                   h->n, ed, false, lK);
    EpiBPrimalT<T> et{bh->ctrl, S.lpT, E.Y[0], E.Y[1], E.X[0], E.X[1], E.KTY[0], E.KTY[1],
                      S.partT, S.ntT};
    launch_spmv<T>(S.gT, st, S.taskT, S.nzT, S.ntT, S.wbegT, S.permTl, h->trp, h->tci, E.tval,
                   h->dev_err, h->m, et, false, lT);
    kb_step_ctrl<<<(bh->meta.B + kBW - 1) / kBW, kBW * 32, 0, st>>>(
        bh->ctrl, bh->meta.B, S.t0K, S.t0T, S.partK, S.partT, S.ntT);
}

template <typename T>
void b_launch_check(BatchHandle* bh, cudaStream_t st, cudaGraphConditionalHandle hd, int use_handle,
                    int in_body)
{
    Handle* h = &bh->h;
    Engine<T>& E = engine_of<T>(h);
    BatchSched<T>& S = sched_of<T>(bh);
    const int64_t m = h->m, n = h->n;
    const int B = bh->meta.B;
    // drop the tasks of the LPs that finished at the previous check
    b_compact<T>(bh, st);
    kb_check_prep<T><<<grid_n(n + m), kEW, 0, st>>>(bh->ctrl, bh->meta.lp_row, bh->meta.lp_col,
                                                     E.X[0], E.X[1], E.Y[0], E.Y[1], E.XS, E.YS,
                                                     E.XA, E.YA, E.l, E.u, h->sense, n, m);
    SplitRows lK, lT;
    lK.wend = S.wendK;
    lT.wend = S.wendT;
    EpiBStore<T> e1{E.XA, E.KXA, nullptr, S.lpK, nullptr, bh->ctrl};
    launch_spmv<T>(S.gK, st, S.taskK, S.nzK, S.ntK, S.wbegK, S.permKl, h->rp, h->ci, E.val,
                   h->dev_err, n, e1, false, lK);
    EpiBStore<T> e2{E.YA, E.KTYA, nullptr, S.lpT, nullptr, bh->ctrl};
    launch_spmv<T>(S.gT, st, S.taskT, S.nzT, S.ntT, S.wbegT, S.permTl, h->trp, h->tci, E.tval,
                   h->dev_err, m, e2, false, lT);
    kb_check_rows<T><<<(S.ntK + 7) / 8, kEW, 0, st>>>(bh->ctrl, S.taskK, S.lpK, S.ntK, E.Y[0],
                                                       E.Y[1], E.KX[0], E.KX[1], E.YA, E.KXA,
                                                       E.YANC, E.q, h->sense, E.Rt, E.Rinv, S.partR);
    kb_check_cols<T><<<(S.ntT + 7) / 8, kEW, 0, st>>>(bh->ctrl, S.taskT, S.lpT, S.ntT, E.X[0],
                                                       E.X[1], E.KTY[0], E.KTY[1], E.XA, E.KTYA,
                                                       E.XANC, E.c, E.l, E.u, E.Ct, E.Cinv, S.partC);
    kb_check_ctrl<<<(B + kBW - 1) / kBW, kBW * 32, 0, st>>>(bh->ctrl, B, S.t0K, S.t0T, S.partR,
                                                            S.ntK, S.partC, S.ntT);
    kb_restart_apply<T><<<grid_n(n + m), kEW, 0, st>>>(
        bh->ctrl, bh->meta.lp_row, bh->meta.lp_col, E.X[0], E.X[1], E.Y[0], E.Y[1], E.KX[0],
        E.KX[1], E.KTY[0], E.KTY[1], E.XA, E.YA, E.KXA, E.KTYA, E.XANC, E.YANC, E.XS, E.YS, n, m);
    kb_set_cond<<<1, 1024, 0, st>>>(bh->ctrl, B, hd, use_handle, in_body, nullptr);
}

template <typename T>
lp_status b_build_graph(BatchHandle* bh, int check_every, int slots)
{
    const int prec = sizeof(T) == 8 ? 0 : 1;
    if (bh->exec && bh->exec_prec == prec && bh->exec_slots == slots &&
        bh->exec_check == check_every)
        return LP_OK;
    if (bh->exec) {
        cudaGraphExecDestroy(bh->exec);
        bh->exec = nullptr;
    }
    Handle* h = &bh->h;
    cudaStream_t st = h->stream;
    cudaGraph_t graph = nullptr;
    LP_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle hd{};
    LP_CUDA_TRY(cudaGraphConditionalHandleCreate(&hd, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    LP_CUDA_TRY(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    LP_CUDA_TRY(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < slots; ++s) b_launch_attempt<T>(bh, st);
    b_launch_check<T>(bh, st, hd, 1, 1);
    cudaGraph_t captured = nullptr;
    LP_CUDA_TRY(cudaStreamEndCapture(st, &captured));
    LP_CUDA_TRY(cudaGraphInstantiate(&bh->exec, graph, 0));
    cudaGraphDestroy(graph);
    bh->exec_prec = prec;
    bh->exec_slots = slots;
    bh->exec_check = check_every;
    return LP_OK;
}

template <typename T>
__global__ void kb_cast_vec(const double* src, T* dst, int64_t count)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (T)src[t];
}

// One batched solve in precision T.  prev / warm (both or neither): the control
// blocks and the unscaled candidates (n + m, device) of an FP32 phase, for the
// FP64 confirmation and polish of the LPs it declared optimal.  ctrl_out /
// xo_out (optional): this phase's control blocks and its unscaled candidates
// (the caller then owns xo_out, a dev_alloc of the handle).
template <typename T>
lp_status batch_solve_t(BatchHandle* bh, const lp_opts* o, lp_result* rs,
                        const std::vector<Ctrl>* prev = nullptr, const double* warm = nullptr,
                        std::vector<Ctrl>* ctrl_out = nullptr, double** xo_out = nullptr)
{
    Handle* h = &bh->h;
    const int B = bh->meta.B;
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    cudaStream_t st = h->stream;
    const long long launches0 = h->launches;
    auto t_start = std::chrono::steady_clock::now();
    // setup: per-LP Ruiz and norms in FP64, then this precision's copies
    double* normK = bh->lpd + 3 * B;
    LP_TRY(batch_scale(bh, o, normK));
    LP_TRY(ensure_sched<T>(bh));
    Engine<T>& E = engine_of<T>(h);
    if (sizeof(T) == 4) {
        const Engine<double>& D = h->e64;
        kb_cast<T><<<grid_n(nnz, 256, 8192), 256, 0, st>>>(D.val, nullptr, E.val, nnz);
        kb_cast<T><<<grid_n(nnz, 256, 8192), 256, 0, st>>>(D.val, h->tperm, E.tval, nnz);
        kb_cast_vec<T><<<grid_n(n, 256, 8192), 256, 0, st>>>(D.c, E.c, n);
        kb_cast_vec<T><<<grid_n(n, 256, 8192), 256, 0, st>>>(D.l, E.l, n);
        kb_cast_vec<T><<<grid_n(n, 256, 8192), 256, 0, st>>>(D.u, E.u, n);
        kb_cast_vec<T><<<grid_n(m, 256, 8192), 256, 0, st>>>(D.q, E.q, m);
        h->launches += 6;
    }
    LP_CUDA_TRY((spmv_prepare<T, EpiBStore<T>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiBDual<T>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiBPrimalT<T>>()));
    // per-LP ||c~||^2, ||q~||^2 (scaled, for omega_0)
    double* cs2 = bh->lpd + 4 * B;
    double* qs2 = bh->lpd + 5 * B;
    int64_t* offc = nullptr;
    int64_t* offr = nullptr;
    LP_TRY(dev_alloc_n(h, &offc, (size_t)B + 1));
    LP_TRY(dev_alloc_n(h, &offr, (size_t)B + 1));
    LP_CUDA_TRY(cudaMemcpyAsync(offc, bh->meta.col0.data(), sizeof(int64_t) * (B + 1),
                                cudaMemcpyHostToDevice, st));
    LP_CUDA_TRY(cudaMemcpyAsync(offr, bh->meta.row0.data(), sizeof(int64_t) * (B + 1),
                                cudaMemcpyHostToDevice, st));
    k_lp_sumsq<<<B, kEW, 0, st>>>(h->e64.c, offc, cs2);
    k_lp_sumsq<<<B, kEW, 0, st>>>(h->e64.q, offr, qs2);
    // control blocks
    Ctrl tmpl;
    std::memset(&tmpl, 0, sizeof(tmpl));
    tmpl.kkt_prev = INFINITY;
    tmpl.tol = o->tol;
    tmpl.beta_s = o->beta_sufficient;
    tmpl.beta_n = o->beta_necessary;
    tmpl.beta_a = o->beta_artificial;
    tmpl.eps_zero = o->eps_zero;
    tmpl.time_limit_ns = o->time_limit_s * 1e9;
    tmpl.max_iters = o->max_iters;
    tmpl.status = kRunning;
    tmpl.first = 1;
    tmpl.want_check = 1;
    tmpl.skip = 1;
    tmpl.adaptive = o->adaptive_step ? 1 : 0;
    tmpl.pwu = o->primal_weight_update ? 1 : 0;
    tmpl.restarts_on = o->restarts ? 1 : 0;
    tmpl.infeas = o->infeas_detect ? 1 : 0;
    tmpl.infeas_tol = o->infeas_tol;
    tmpl.check_every = o->check_every;
    unsigned long long* tns = reinterpret_cast<unsigned long long*>(bh->lpd + 6 * B);
    kb_read_clock<<<1, 1, 0, st>>>(tns);
    unsigned long long t0 = 0;
    LP_CUDA_TRY(cudaMemcpyAsync(&t0, tns, sizeof(t0), cudaMemcpyDeviceToHost, st));
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    Ctrl* dprev = nullptr;
    if (prev) {
        LP_TRY(dev_alloc_n(h, &dprev, (size_t)B));
        LP_CUDA_TRY(cudaMemcpyAsync(dprev, prev->data(), sizeof(Ctrl) * B, cudaMemcpyHostToDevice,
                                    st));
    }
    kb_init_ctrl<<<grid_n(B, 256, 4096), 256, 0, st>>>(bh->ctrl, B, normK, cs2, qs2, bh->meta.qn,
                                                       bh->meta.cn, tmpl, o->eta_scale, o->eta0,
                                                       o->omega0, o->eps_zero, t0, dprev);
    LP_TRY(engine_factors<T>(h));
    if (o->autotune) LP_TRY(tune_batch<T>(bh));
    // start point and its products
    kb_init_state<T><<<grid_n(n + m, 256, 8192), 256, 0, st>>>(E.X[0], E.Y[0], E.XANC, E.YANC,
                                                               E.XS, E.YS, E.l, E.u, n, m, warm,
                                                               h->R, h->C, h->sense);
    BatchSched<T>& S = sched_of<T>(bh);
    {
        EpiBStore<T> e1{E.X[0], E.KX[0], nullptr, S.lpK, nullptr, nullptr};
        launch_spmv<T>(S.gK, st, S.taskK, S.nzK, S.ntK, S.wbegK, S.permK, h->rp, h->ci, E.val, h->dev_err, n, e1);
        EpiBStore<T> e2{E.Y[0], E.KTY[0], nullptr, S.lpT, nullptr, nullptr};
        launch_spmv<T>(S.gT, st, S.taskT, S.nzT, S.ntT, S.wbegT, S.permT, h->trp, h->tci, E.tval, h->dev_err, m, e2);
    }
    b_launch_check<T>(bh, st, cudaGraphConditionalHandle{}, 0, 0);
    h->launches += 11 + 3 + 4;
    LP_CUDA_TRY(cudaGetLastError());
    auto t_setup = std::chrono::steady_clock::now();
    const int slots = o->check_every + (o->adaptive_step ? 4 : 0);
    LP_TRY(b_build_graph<T>(bh, o->check_every, slots));
    LP_CUDA_TRY(cudaGraphLaunch(bh->exec, st));
    std::vector<Ctrl> hc((size_t)B);
    LP_CUDA_TRY(cudaMemcpyAsync(hc.data(), bh->ctrl, sizeof(Ctrl) * B, cudaMemcpyDeviceToHost, st));
    int derr = 0;
    LP_CUDA_TRY(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    if (derr) return LP_DEVICE_TIMEOUT;
    long long bodies = 0;
    for (const Ctrl& c : hc) bodies = std::max(bodies, c.bodies);
    h->launches += bodies * (long long)(slots * 4 + 11);
    // solutions, unscaled, stacked; then into each caller's buffers
    double* xo = nullptr;
    LP_TRY(dev_alloc_n(h, &xo, (size_t)(n + m)));
    kb_extract<T><<<grid_n(n + m, 256, 8192), 256, 0, st>>>(bh->ctrl, bh->meta.lp_row,
                                                            bh->meta.lp_col, E.X[0], E.X[1],
                                                            E.Y[0], E.Y[1], E.XA, E.YA, h->R,
                                                            h->C, xo, xo + n, n, m);
    ++h->launches;
    auto t_end = std::chrono::steady_clock::now();
    const double setup_s = std::chrono::duration<double>(t_setup - t_start).count();
    const double solve_s = std::chrono::duration<double>(t_end - t_setup).count();
    std::vector<double> nk((size_t)B);
    LP_CUDA_TRY(cudaMemcpyAsync(nk.data(), normK, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    for (int k = 0; k < B; ++k) {
        lp_result* r = rs + k;
        const Ctrl& c = hc[(size_t)k];
        const int64_t mk = bh->meta.row0[k + 1] - bh->meta.row0[k];
        const int64_t nk_ = bh->meta.col0[k + 1] - bh->meta.col0[k];
        const cudaMemcpyKind kind = r->memory_space == LP_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                     : cudaMemcpyDeviceToHost;
        if (r->x)
            LP_CUDA_TRY(cudaMemcpyAsync(r->x, xo + bh->meta.col0[k], sizeof(double) * nk_, kind, st));
        if (r->y)
            LP_CUDA_TRY(cudaMemcpyAsync(r->y, xo + n + bh->meta.row0[k], sizeof(double) * mk, kind,
                                        st));
        r->status = (lp_status)c.status;
        r->precision_used = sizeof(T) == 8 ? LP_PREC_FP64 : LP_PREC_MIXED;
        r->iters = c.k;
        r->attempts = c.attempts;
        r->restarts = c.restarts;
        r->fp64_iters = sizeof(T) == 8 ? c.k : 0;
        if (prev) {
            // after an FP32 phase: FP64 iterations only where the FP64 check sent
            // the LP on (a confirmation alone keeps the FP32 result)
            r->fp64_iters = c.k - (*prev)[(size_t)k].k;
            r->precision_used = r->fp64_iters > 0 ? LP_PREC_FP64 : LP_PREC_MIXED;
        }
        r->pobj = c.pobj;
        r->dobj = c.dobj;
        r->rel_gap = c.rel_gap;
        r->rel_pres = c.rel_pres;
        r->rel_dres = c.rel_dres;
        r->omega = c.omega;
        r->eta = c.eta;
        r->setup_s = setup_s;
        // the LP's own time to its outcome, from the device clock
        r->solve_s = c.t_done_ns > c.t0_ns ? 1e-9 * (double)(c.t_done_ns - c.t0_ns) : solve_s;
        r->trace_len = 0;
    }
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < B; ++k) rs[k].norm_K = nk[(size_t)k];
    const long long lz = h->launches - launches0;
    for (int k = 0; k < B; ++k) rs[k].kernel_launches = k == 0 ? lz : 0;
    if (ctrl_out) *ctrl_out = hc;
    if (xo_out) *xo_out = xo;
    for (void* p : {(void*)(xo_out ? nullptr : xo), (void*)offc, (void*)offr, (void*)dprev}) {
        if (!p) continue;
        for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
            if (it->p == p) {
                cudaFree(p);
                h->allocs.erase(it);
                break;
            }
    }
    return LP_OK;
}

// LP_PREC_MIXED: the FP32 phase to max(tol, polish_switch_tol), then, for the
// LPs it declared optimal, an FP64 phase from their candidates: its first check
// re-evaluates the relative errors with FP64 products (the FP32 phase judged
// them on FP32 products) and LP_OPTIMAL stands only if they hold; otherwise, or
// below the hand-over tolerance, FP64 iterations continue to tol.
lp_status batch_solve_mixed(BatchHandle* bh, const lp_opts* o, lp_result* rs)
{
    lp_opts o32 = *o;
    o32.tol = std::max(o->tol, o->polish_switch_tol);
    std::vector<Ctrl> c32;
    double* xo = nullptr;
    lp_status s = batch_solve_t<float>(bh, &o32, rs, nullptr, nullptr, &c32, &xo);
    if (s != LP_OK) return s;
    bool any = false;
    for (const Ctrl& c : c32) any = any || c.status == LP_OPTIMAL;
    const long long launches32 = rs[0].kernel_launches;
    if (any) {
        const int B = bh->meta.B;
        std::vector<double> setup32((size_t)B);
        for (int k = 0; k < B; ++k) setup32[(size_t)k] = rs[k].setup_s;
        s = batch_solve_t<double>(bh, o, rs, &c32, xo, nullptr, nullptr);
        for (int k = 0; k < B; ++k) rs[k].setup_s += setup32[(size_t)k];
        rs[0].kernel_launches += launches32;
    }
    Handle* h = &bh->h;
    for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
        if (it->p == xo) {
            cudaFree(xo);
            h->allocs.erase(it);
            break;
        }
    return s;
}

}  // namespace

// Stacks the handles' device data into one block-diagonal problem.
static lp_status batch_build(BatchHandle* bh, const lp_handle* hs, int B)
{
    Handle* h = &bh->h;
    cudaStream_t st = h->stream;
    BatchMeta& M = bh->meta;
    M.B = B;
    M.row0.assign((size_t)B + 1, 0);
    M.col0.assign((size_t)B + 1, 0);
    M.nz0.assign((size_t)B + 1, 0);
    for (int k = 0; k < B; ++k) {
        if (!hs[k]) return LP_INVALID_ARGUMENT;
        const Handle& g = hs[k]->h;
        M.row0[k + 1] = M.row0[k] + g.m;
        M.col0[k + 1] = M.col0[k] + g.n;
        M.nz0[k + 1] = M.nz0[k] + g.nnz;
        if (g.stream != st) LP_CUDA_TRY(cudaStreamSynchronize(g.stream));
    }
    const int64_t m = M.row0[B], n = M.col0[B], nnz = M.nz0[B];
    if (nnz >= ((int64_t)1 << 31) - 64 || m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31))
        return LP_INVALID_ARGUMENT;
    // stacked arrays in temporary buffers, then the usual device setup
    std::vector<void*> tmp;
    auto talloc = [&](void** p, size_t bytes) -> lp_status {
        cudaError_t e = cudaMalloc(p, bytes + 64);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? LP_OUT_OF_MEMORY : LP_CUDA_ERROR;
        }
        tmp.push_back(*p);
        return LP_OK;
    };
    int64_t* rp = nullptr;
    int32_t* ci = nullptr;
    double *vv = nullptr, *c = nullptr, *q = nullptr, *l = nullptr, *u = nullptr;
    uint8_t* se = nullptr;
    lp_status s = LP_OK;
    if ((s = talloc((void**)&rp, 8 * (size_t)(m + 1))) == LP_OK &&
        (s = talloc((void**)&ci, 4 * (size_t)std::max<int64_t>(nnz, 1))) == LP_OK &&
        (s = talloc((void**)&vv, 8 * (size_t)std::max<int64_t>(nnz, 1))) == LP_OK &&
        (s = talloc((void**)&se, (size_t)m)) == LP_OK && (s = talloc((void**)&c, 8 * (size_t)n)) == LP_OK &&
        (s = talloc((void**)&q, 8 * (size_t)m)) == LP_OK && (s = talloc((void**)&l, 8 * (size_t)n)) == LP_OK &&
        (s = talloc((void**)&u, 8 * (size_t)n)) == LP_OK) {
        for (int k = 0; k < B && s == LP_OK; ++k) {
            const Handle& g = hs[k]->h;
            const int gm = grid_n(std::max<int64_t>(g.m, g.nnz), 256, 4096);
            k_shift_i64<<<gm, 256, 0, st>>>(g.rp, rp + M.row0[k], g.m, M.nz0[k]);
            if (g.nnz > 0)
                k_shift_i32<<<gm, 256, 0, st>>>(g.ci, ci + M.nz0[k], g.nnz, (int32_t)M.col0[k]);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess && g.nnz > 0)
                e = cudaMemcpyAsync(vv + M.nz0[k], g.val0, 8 * (size_t)g.nnz, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(se + M.row0[k], g.sense, (size_t)g.m, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c + M.col0[k], g.c0, 8 * (size_t)g.n, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(q + M.row0[k], g.q0, 8 * (size_t)g.m, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(l + M.col0[k], g.l0, 8 * (size_t)g.n, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(u + M.col0[k], g.u0, 8 * (size_t)g.n, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                s = LP_CUDA_ERROR;
            }
        }
        if (s == LP_OK &&
            cudaMemcpyAsync(rp + m, &nnz, 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
            s = LP_CUDA_ERROR;
        if (s == LP_OK && cudaStreamSynchronize(st) != cudaSuccess) s = LP_CUDA_ERROR;
        if (s == LP_OK) {
            lp_desc d{};
            d.m = m; d.n = n; d.nnz = nnz;
            d.row_ptr = rp; d.col_idx = ci; d.vals = vv; d.sense = se;
            d.c = c; d.q = q; d.l = l; d.u = u;
            d.memory_space = LP_MEM_DEVICE;
            s = setup_create(h, &d);
        }
    }
    cudaStreamSynchronize(st);
    for (void* p : tmp) cudaFree(p);
    if (s != LP_OK) return s;
    // LP of every row and column; per-LP unscaled norms; control blocks
    LP_TRY(dev_alloc_n(h, &M.lp_row, (size_t)m));
    LP_TRY(dev_alloc_n(h, &M.lp_col, (size_t)n));
    for (int k = 0; k < B; ++k) {
        const int64_t mk = M.row0[k + 1] - M.row0[k], nk = M.col0[k + 1] - M.col0[k];
        k_fill_i32<<<grid_n(mk, 256, 4096), 256, 0, st>>>(M.lp_row + M.row0[k], mk, k);
        k_fill_i32<<<grid_n(nk, 256, 4096), 256, 0, st>>>(M.lp_col + M.col0[k], nk, k);
    }
    std::vector<double> qn((size_t)B), cn((size_t)B);
    for (int k = 0; k < B; ++k) {
        qn[(size_t)k] = hs[k]->h.qnorm;
        cn[(size_t)k] = hs[k]->h.cnorm;
    }
    LP_TRY(dev_alloc_n(h, &M.qn, (size_t)B));
    LP_TRY(dev_alloc_n(h, &M.cn, (size_t)B));
    LP_CUDA_TRY(cudaMemcpyAsync(M.qn, qn.data(), 8 * (size_t)B, cudaMemcpyHostToDevice, st));
    LP_CUDA_TRY(cudaMemcpyAsync(M.cn, cn.data(), 8 * (size_t)B, cudaMemcpyHostToDevice, st));
    LP_TRY(dev_alloc_n(h, &bh->ctrl, (size_t)B));
    LP_TRY(dev_alloc_n(h, &bh->lpd, 8 * (size_t)B + 8));
    LP_TRY(dev_alloc_n(h, &bh->go, (size_t)B));
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    return LP_OK;
}

}  // namespace pdhg

struct lp_batch_s {
    pdhg::BatchHandle b;
};

extern "C" {

lp_status lp_batch_create(const lp_handle* hs, int32_t count, void* cuda_stream, lp_batch* out)
{
    if (!out) return LP_INVALID_ARGUMENT;
    *out = nullptr;
    if (!hs || count < 1) return LP_INVALID_ARGUMENT;
    lp_batch_s* p = new (std::nothrow) lp_batch_s();
    if (!p) return LP_OUT_OF_MEMORY;
    pdhg::Handle* h = &p->b.h;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete p;
        return LP_CUDA_ERROR;
    }
    if (cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        delete p;
        return LP_CUDA_ERROR;
    } else {
        h->own_stream = true;
    }
    lp_status s = pdhg::batch_build(&p->b, hs, count);
    if (s != LP_OK) {
        lp_batch_destroy(p);
        return s;
    }
    *out = p;
    return LP_OK;
}

lp_status lp_batch_solve(lp_batch b, const lp_opts* o, lp_result* rs)
{
    if (!b || !o || !rs) return LP_INVALID_ARGUMENT;
    if (!(o->tol >= 0.0) || o->max_iters < 0 || o->check_every < 1 || o->ruiz_iters < 0 ||
        o->power_iters < 0 || !(o->eta_scale > 0.0) || !(o->time_limit_s > 0.0))
        return LP_INVALID_ARGUMENT;
    if (o->halpern) return LP_NOT_SUPPORTED;   // the batched loop runs averaged PDHG restarts
    if (o->pock_chambolle == 2) return LP_NOT_SUPPORTED;   // alpha trials: lp_solve only
    if (o->pock_chambolle < 0 || o->pock_chambolle > 2 || !(o->pc_alpha >= 0.0 && o->pc_alpha <= 2.0))
        return LP_INVALID_ARGUMENT;
    for (int k = 0; k < b->b.meta.B; ++k)
        if (rs[k].memory_space != LP_MEM_HOST && rs[k].memory_space != LP_MEM_DEVICE)
            return LP_INVALID_ARGUMENT;
    lp_status s;
    if (o->precision == LP_PREC_FP64) s = pdhg::batch_solve_t<double>(&b->b, o, rs);
    else if (o->precision == LP_PREC_MIXED) s = pdhg::batch_solve_mixed(&b->b, o, rs);
    else return LP_INVALID_ARGUMENT;
    if (s < 0) {
        cudaStreamSynchronize(b->b.h.stream);
        (void)cudaGetLastError();
    }
    return s;
}

void lp_batch_destroy(lp_batch b)
{
    if (!b) return;
    pdhg::Handle* h = &b->b.h;
    cudaStreamSynchronize(h->stream);
    if (b->b.exec) cudaGraphExecDestroy(b->b.exec);
    for (auto& a : h->allocs) cudaFree(a.p);
    h->allocs.clear();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete b;
}

}  // extern "C"
