// The restarted PDHG iteration on the device.
//
// One step attempt (Algorithm 1 with theta = 1, step sizes tau = eta / omega,
// sigma = eta * omega, Section 2.3.1) is two launches; the candidate x' of the
// attempt was formed by the launch before:
//   k_spmv<Dual>        K x', then y' = proj_Y(y + sigma (q - (2 K x' - K x))) (K x kept),
//                       ||y' - y||^2 and (y' - y)^T K (x' - x); its last block adds
//                       ||x' - x||^2 (from the launch that formed x') and takes the
//                       Algorithm 5 accept / reject decision, swaps the double buffers
//                       and sets eta'
//   k_spmv<PrimalStep>  accepted: K^T y', then per column the next candidate
//                       x'' = clamp(x' - tau' (c - K^T y'), l, u) with its ||x'' - x'||^2
//                       partials and the eta-weighted sum of the accepted x'; rejected:
//                       no product, x'' = clamp(x - tau' (c - K^T y), l, u) from the kept
//                       K^T y
// After a check (which may restart and change omega) k_primal forms the first
// candidate of the next period.  Every check_every accepted iterations the check
// launches run: averages
// (Section 2.4.2), their products, FP64 KKT reductions, the candidate, the
// termination test on the unscaled problem (Section 2.3.2), the three restart
// criteria and the primal-weight update (Algorithm 4).  The whole loop is a CUDA
// graph whose body is (check_every + spare) attempt slots plus the check, inside
// a conditional WHILE node; k_set_cond writes the loop condition on the device.
//
// Restarted Halpern PDHG (the variant the Conclusion names as future work; Lu
// and Yang, 2024) runs in the same loop with its own two step kernels:
//   k_primal_halpern        x^ = clamp(x - tau (c - K^T y), l, u) -> XH (the K launch's input;
//                           also -> XA before a check), x+ = lam ((1 + rho) x^ - rho x)
//                           + (1 - lam) x_anchor
//   k_spmv<HalpernDual>     K x^, y^ = proj_Y(y + sigma (q - (2 K x^ - K x))),
//                           y+ and K x+ by the same combination (K x of the anchor kept),
//                           y^ -> YA on the iteration before a check
//   k_spmv<PrT>             K^T y+; the last block records ||z - T(z)||_P
// with lam = (k + 1) / (k + 2), k the iterations since the last restart.  The
// check then evaluates T(z) = (XA, YA) in the slot of the average.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "control.cuh"
#include "spmv.cuh"

namespace pdhg {

// ------------------------------------------------------------------ step kernels

// x' = clamp(x - tau (c - K^T y), l, u): the first candidate after a check
// (in the loop body's check, after the restart decision, and at the start),
// and, where the primal step is not fused into the K^T launch, the candidate of
// every next attempt; the accepted iterates reach the eta-weighted sums in the
// K^T launch.  Block partials of ||x' - x||^2 go to part[blockIdx.x]; the
// grid is the K^T launch's, so that the step decision always sums the same
// number of partials.  16-byte vector loads, scalar tail.
template <typename T>
__global__ void __launch_bounds__(kEW)
k_primal(const Ctrl* __restrict__ ctrl, T* x0, T* x1, const T* __restrict__ kty0,
         const T* __restrict__ kty1, const T* __restrict__ c, const T* __restrict__ l,
         const T* __restrict__ u, int64_t n, double* part, int after_step, int nsplit)
{
    // after_step = 0: after a check (and at the start); 1: after the K^T launch
    // of an attempt when the primal step is not fused into it (its mode 1 or 3)
    if (after_step) {
        const int mode = ctrl->t_mode;
        if (mode != 1 && mode != 3) return;
    } else if (!ctrl->want_check || ctrl->done) {
        return;
    }
    T dx2 = T(0);
    using VT = VecTraits<T>;
    constexpr int VEC = VT::N;
    const int cur = ctrl->cur;
    const T tau = step_scalars<T>(*ctrl).tau;
    const T* x = cur ? x1 : x0;
    T* xn = cur ? x0 : x1;
    const T* kty = cur ? kty1 : kty0;
    const int64_t nv = n / VEC;
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < nv; t += (int64_t)gridDim.x * kEW) {
        T xj[VEC], kj[VEC], cj[VEC], lj[VEC], uj[VEC], o[VEC];
        VT::unpack(*reinterpret_cast<const typename VT::V*>(x + t * VEC), xj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(kty + t * VEC)), kj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(c + t * VEC)), cj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(l + t * VEC)), lj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(u + t * VEC)), uj);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            T v = xj[k] - tau * (cj[k] - kj[k]);
            if (v < lj[k]) v = lj[k];
            if (v > uj[k]) v = uj[k];
            o[k] = v;
            dx2 += (v - xj[k]) * (v - xj[k]);
        }
        *reinterpret_cast<typename VT::V*>(xn + t * VEC) = VT::pack(o);
    }
    for (int64_t j = nv * VEC + (int64_t)blockIdx.x * kEW + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * kEW) {
        const T xj = x[j];
        T v = xj - tau * (c[j] - kty[j]);
        const T lo = l[j], hi = u[j];
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        xn[j] = v;
        dx2 += (v - xj) * (v - xj);
    }
    const double t[1] = {(double)dx2};
    block_partials<1, kEW>(t, part, gridDim.x);
    // the K^T launch's split-row slots follow the block partials; every column
    // is covered above, so they hold nothing of this step
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < nsplit; i += kEW) part[gridDim.x + i] = 0.0;
}

// Halpern iteration, primal half: x^ = clamp(x - tau (c - K^T y), l, u) (the
// primal part of T(z)) goes to xh, the input of the K x^ launch, and on the
// iteration before a check also to xa (the check's candidate, left untouched
// until the next check so that a loop stopped in between returns a matching
// pair); the next iterate x+ = a x^ - b x + g x_anchor goes to the other half of
// X, with a = lam (1 + rho), b = lam rho, g = 1 - lam, lam = (k + 1) / (k + 2), k
// the iterations since the last restart.  Block partials of ||x^ - x||^2 (the
// fixed-point residual) go to part[blockIdx.x].
template <typename T>
__global__ void __launch_bounds__(kEW)
k_primal_halpern(const Ctrl* __restrict__ ctrl, T* x0, T* x1, const T* __restrict__ kty0,
                 const T* __restrict__ kty1, const T* __restrict__ c, const T* __restrict__ l,
                 const T* __restrict__ u, const T* __restrict__ xanc, T* __restrict__ xh,
                 T* __restrict__ xa, int64_t n, double* part)
{
    if (ctrl->skip) return;
    const long long k1 = ctrl->k + 1;
    const bool hat = k1 % ctrl->check_every == 0 || k1 >= ctrl->max_iters;
    T dx2 = T(0);
    using VT = VecTraits<T>;
    constexpr int VEC = VT::N;
    const int cur = ctrl->cur;
    const StepScalars<T>& sc = step_scalars<T>(*ctrl);
    const T tau = sc.tau, a = sc.ha, b = sc.hb, g = sc.hg;
    const T* x = cur ? x1 : x0;
    T* xn = cur ? x0 : x1;
    const T* kty = cur ? kty1 : kty0;
    const int64_t nv = n / VEC;
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < nv; t += (int64_t)gridDim.x * kEW) {
        T xj[VEC], kj[VEC], cj[VEC], lj[VEC], uj[VEC], aj[VEC], h[VEC], o[VEC];
        VT::unpack(*reinterpret_cast<const typename VT::V*>(x + t * VEC), xj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(kty + t * VEC)), kj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(c + t * VEC)), cj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(l + t * VEC)), lj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(u + t * VEC)), uj);
        VT::unpack(__ldg(reinterpret_cast<const typename VT::V*>(xanc + t * VEC)), aj);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            T v = xj[k] - tau * (cj[k] - kj[k]);
            if (v < lj[k]) v = lj[k];
            if (v > uj[k]) v = uj[k];
            h[k] = v;
            o[k] = a * v - b * xj[k] + g * aj[k];
            dx2 += (v - xj[k]) * (v - xj[k]);
        }
        *reinterpret_cast<typename VT::V*>(xh + t * VEC) = VT::pack(h);
        if (hat) *reinterpret_cast<typename VT::V*>(xa + t * VEC) = VT::pack(h);
        *reinterpret_cast<typename VT::V*>(xn + t * VEC) = VT::pack(o);
    }
    for (int64_t j = nv * VEC + (int64_t)blockIdx.x * kEW + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * kEW) {
        const T xj = x[j];
        T v = xj - tau * (c[j] - kty[j]);
        const T lo = l[j], hi = u[j];
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        xh[j] = v;
        if (hat) xa[j] = v;
        xn[j] = a * v - b * xj + g * xanc[j];
        dx2 += (v - xj) * (v - xj);
    }
    const double t[1] = {(double)dx2};
    block_partials<1, kEW>(t, part, gridDim.x);
}

// Thread 0 of the deciding block: step_decide, then (fused PDHG attempts) the
// mode of the K^T launch that follows.  Kept out of line so that its FP64
// arithmetic does not add to the register pressure of the SpMV kernels that
// call it once per launch.
__device__ __noinline__ void decide_thread0(Ctrl* ctrl, bool sums, int adapt, double dy2,
                                            double dx2, double inter, bool fused)
{
    ctrl->tick = 0;
    const long long k0 = ctrl->k;
    const double eta = ctrl->eta, omega = ctrl->omega;
    double eta_bar = NAN;
    if (sums) step_decide(ctrl, adapt, dy2, dx2, inter, &eta_bar);
    else step_decide(ctrl, adapt, 0.0, 0.0, 0.0);
    if (ctrl->alog && ctrl->alog_len < ctrl->alog_cap) {
        double* r = ctrl->alog + kAttemptFields * ctrl->alog_len;
        r[0] = (double)k0; r[1] = eta; r[2] = eta_bar; r[3] = ctrl->eta;
        r[4] = ctrl->k != k0 ? 1.0 : 0.0; r[5] = omega;
        r[6] = sums ? dx2 : NAN; r[7] = sums ? dy2 : NAN; r[8] = sums ? inter : NAN;
    }
    ctrl->alog_len += 1;
    if (fused) {
        int mode = 0;
        if (!ctrl->done) {
            if (ctrl->k != k0) mode = ctrl->want_check ? 2 : 1;
            else mode = 3;
        }
        ctrl->t_mode = mode;
    }
}

// The step decision of an attempt, taken by the last block of the launch that
// completes the attempt's reductions (no block waits for another: the last
// block is the one whose ticket completes the count).  Warps 0..2 sum, in a
// fixed order, ||y' - y||^2 (partD[0, nD)), the interaction (partD[nD, 2 nD))
// and ||x' - x||^2 (partX[0, nX)); thread 0 runs step_decide.  With `fused`
// it also tells the K^T launch what to do next (Ctrl::t_mode).  Out of line:
// inlined into the K-side SpMV it raised that kernel's register spills from 10
// to 34 bytes per thread (FP32).
template <int NT>
__device__ __noinline__ void last_block_decide(Ctrl* ctrl, const double* partD, int nD,
                                                  const double* partX, int nX, bool sums,
                                                  int adapt, bool fused)
{
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctrl->tick, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (sums && warp < 3) {
        const double* src = warp == 0 ? partD : warp == 1 ? partD + nD : partX;
        const int cnt = warp == 2 ? nX : nD;
        // eight independent loads in flight per lane (a single running sum would
        // wait one L2 round trip per 32 partials: about 10 us on a 608-block
        // grid, on the critical path of every attempt); fixed order
        double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int i = lane;
        for (; i + 7 * 32 < cnt; i += 8 * 32) {
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] += __ldcg(src + i + 32 * u);
        }
        for (; i < cnt; i += 32) a[0] += __ldcg(src + i);
        double v = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        v = warp_sum(v);
        if (lane == 0) tot[warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) decide_thread0(ctrl, sums, adapt, tot[0], tot[2], tot[1], fused);
}

// K x' SpMV + dual step: y' = proj_Y(y + sigma (q - (2 K x' - K x))); the
// pending weight of the current y (the last accepted iterate) goes to the y sums
// on the way.  The last block takes the attempt's Algorithm 5 decision.
template <typename T>
struct EpiDual {
    PDHG_SINGLE_LP_TASK_HOOKS
    Ctrl* ctrl;
    const T* xs0; const T* xs1;     // X[0], X[1]
    T* y0; T* y1; T* kx0; T* kx1;
    T* ys;
    const T* q;
    const uint8_t* sense;
    double* part;                   // [2][gridDim.x + nsplit] partials of this launch
    int cur; T sigma; T pw; int adapt;
    int nsplit = 0;                 // split rows of the schedule (set by the kernel)
    struct Pre { T y = 0, kx = 0, q = 0, ys = 0; uint8_t ge = 0; };
    // per-lane sums in T, reduced in FP64: ||y' - y||^2 and the Algorithm 5
    // interaction (y' - y)^T K (x' - x) = sum_i dy_i ((K x')_i - (K x)_i)
    struct Acc { T dy2 = T(0), inter = T(0); };
    // after begin(), the *0 members point at the current half and the *1 members
    // at the other one (x' and the new y, K x' are written there)
    __device__ bool begin() {
        if (ctrl->skip) {
            // a slot after a pending check or the end: its K^T launch does nothing
            if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->t_mode = 0;
            return false;
        }
        cur = ctrl->cur;
        if (cur) {
            const T* t = xs0; xs0 = xs1; xs1 = t;
            T* u = y0; y0 = y1; y1 = u;
            u = kx0; kx0 = kx1; kx1 = u;
        }
        const StepScalars<T>& sc = step_scalars<T>(*ctrl);
        sigma = sc.sigma;
        pw = sc.pw;
        adapt = ctrl->adaptive;
        return true;
    }
    __device__ const T* xin() const { return xs1; }   // x' lives in the other half
    __device__ Pre load(int i) const {
        Pre p;
        p.y = y0[i];
        p.kx = kx0[i];
        p.q = q[i];
        p.ge = sense[i];
        if (pw != T(0)) p.ys = ys[i];
        return p;
    }
    __device__ void row(int i, T kxn, const Pre& p, Acc& a) const {
        if (pw != T(0)) ys[i] = p.ys + pw * p.y;
        T v = p.y + sigma * (p.q - (T(2) * kxn - p.kx));
        if (p.ge && v < T(0)) v = T(0);
        y1[i] = v;
        kx1[i] = kxn;
        const T d = v - p.y;
        a.dy2 += d * d;
        a.inter += d * (kxn - p.kx);
    }
    // a split row's terms: after the block partials of each quantity
    __device__ void split_acc(int s, const Acc& a) const {
        if (adapt) {
            const int np = (int)gridDim.x + nsplit;
            part[gridDim.x + s] = (double)a.dy2;
            part[np + gridDim.x + s] = (double)a.inter;
        }
    }
    __device__ void finish(Acc& a) const {
        const int np = (int)gridDim.x + nsplit;
        if (adapt) {
            const double t[2] = {(double)a.dy2, (double)a.inter};
            block_partials<2, kSpmvNT>(t, part, np);
        }
        // ||x' - x||^2 partials: Ctrl::px[0, npx) (kept in the control block, not in
        // this epilogue, whose members live in registers through the whole SpMV)
        last_block_decide<kSpmvNT>(ctrl, part, np, ctrl->px, ctrl->npx, adapt != 0, adapt, true);
    }
};

// K^T launch of a PDHG attempt, after the decision (Ctrl::t_mode).
//  1, 2 (accepted; cur already points at (x', y')): K^T y' -> KTY[cur]; per column
//       the accepted x'_j enters the eta-weighted sum (weight pw = the eta the step
//       was taken with); mode 1 also forms the next candidate
//       x''_j = clamp(x'_j - tau' (c_j - (K^T y')_j), l_j, u_j) -> X[cur ^ 1] with the
//       ||x'' - x'||^2 block partials (tau' from the new eta').
//  3 (rejected): no product; every block runs the elementwise retry
//       x'' = clamp(x - tau' (c - K^T y), l, u) from the kept K^T y, and returns.
//  Without F (the primal step not fused), modes 1 and 2 only store K^T y' and
//  add x' to the sums, mode 3 does nothing here, and k_primal follows.
template <typename T, bool F>
struct EpiPrimalStep {
    PDHG_SINGLE_LP_TASK_HOOKS
    const Ctrl* ctrl;
    T* xs0; T* xs1;                 // X[0], X[1]
    const T* ys0; const T* ys1;     // Y[0], Y[1]
    T* kty0; T* kty1;               // KTY[0], KTY[1]
    const T* c; const T* l; const T* u;
    T* xsum;
    double* part;                   // [gridDim.x + nsplit] ||x'' - x'||^2 partials
    int64_t n;
    int mode; T tau; T pw; int adapt;
    int nsplit = 0;                 // split rows of the schedule (set by the kernel)
    struct Pre { T x = 0, c = 0, l = 0, u = 0, s = 0; };
    struct Acc { T dx2 = T(0); };
    // after begin(): xs0 / ys0 / kty0 are the current half (x', y', K^T y'),
    // xs1 the other half (the next candidate goes there)
    __device__ bool begin() {
        mode = ctrl->t_mode;
        if (mode == 0) return false;
        if (ctrl->cur) {
            T* t = xs0; xs0 = xs1; xs1 = t;
            const T* v = ys0; ys0 = ys1; ys1 = v;
            t = kty0; kty0 = kty1; kty1 = t;
        }
        const StepScalars<T>& sc = step_scalars<T>(*ctrl);
        tau = sc.tau;
        pw = sc.pw;
        adapt = ctrl->adaptive;
        if (!F && mode == 1) mode = 2;
        if (mode != 3) return true;
        if (!F) return false;
        // rejected attempt: the retry's candidate from the kept K^T y
        T dx2 = T(0);
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x) {
            const T xj = xs0[j];
            T v = xj - tau * (c[j] - kty0[j]);
            const T lo = l[j], hi = u[j];
            if (v < lo) v = lo;
            if (v > hi) v = hi;
            xs1[j] = v;
            dx2 += (v - xj) * (v - xj);
        }
        const double t[1] = {(double)dx2};
        block_partials<1, kSpmvNT>(t, part, gridDim.x);
        // the split rows' slots hold nothing of this step: their columns are
        // covered by the loop above
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i < nsplit; i += blockDim.x) part[gridDim.x + i] = 0.0;
        return false;
    }
    __device__ const T* xin() const { return ys0; }   // y'
    __device__ Pre load(int j) const {
        Pre p;
        p.x = xs0[j];
        if (pw != T(0)) p.s = xsum[j];
        if (mode == 1) {
            p.c = c[j];
            p.l = l[j];
            p.u = u[j];
        }
        return p;
    }
    __device__ void row(int j, T ktyn, const Pre& p, Acc& a) const {
        kty0[j] = ktyn;
        if (pw != T(0)) xsum[j] = p.s + pw * p.x;
        if (mode == 1) {
            T v = p.x - tau * (p.c - ktyn);
            if (v < p.l) v = p.l;
            if (v > p.u) v = p.u;
            xs1[j] = v;
            a.dx2 += (v - p.x) * (v - p.x);
        }
    }
    __device__ void split_acc(int s, const Acc& a) const {
        if (mode == 1 && adapt) part[gridDim.x + s] = (double)a.dx2;
    }
    __device__ void finish(Acc& a) const {
        if (mode == 1 && adapt) {
            const double t[1] = {(double)a.dx2};
            block_partials<1, kSpmvNT>(t, part, gridDim.x);
        }
    }
};

// Halpern iteration, dual half: K x^ SpMV, then
// y^ = proj_Y(y + sigma (q - (2 K x^ - K x))), the next iterate
// y+ = a y^ - b y + g y_anchor and its product K x+ = a K x^ - b K x + g K x_anchor
// (linearity: no product of x+ is formed).  y^ is stored on the iteration that
// precedes a check (its candidate T(z)).  Partials: ||y^ - y||^2 and
// (y^ - y)^T K (x^ - x) = sum_i dy_i ((K x^)_i - (K x)_i).
template <typename T>
struct EpiHalpernDual {
    PDHG_SINGLE_LP_TASK_HOOKS
    const Ctrl* ctrl;
    const T* xh;                    // x^ (gathered)
    T* y0; T* y1; T* kx0; T* kx1;   // Y[0], Y[1], KX[0], KX[1]
    const T* yanc; const T* kxanc;
    T* yh;
    const T* q;
    const uint8_t* sense;
    double* part;                   // [2][gridDim.x + nsplit]
    T sigma, a, b, g; int hat;
    int nsplit = 0;                 // split rows of the schedule (set by the kernel)
    // the anchor terms are read in row(): a smaller Pre keeps the SpMV's two
    // prefetched rows per lane in registers
    struct Pre { T y = 0, kx = 0, q = 0; uint8_t ge = 0; };
    struct Acc { T dy2 = T(0), inter = T(0); };
    __device__ bool begin() {
        if (ctrl->skip) return false;
        if (ctrl->cur) {
            T* t = y0; y0 = y1; y1 = t;
            t = kx0; kx0 = kx1; kx1 = t;
        }
        const StepScalars<T>& sc = step_scalars<T>(*ctrl);
        sigma = sc.sigma;
        a = sc.ha;
        b = sc.hb;
        g = sc.hg;
        const long long k1 = ctrl->k + 1;
        hat = k1 % ctrl->check_every == 0 || k1 >= ctrl->max_iters;
        return true;
    }
    __device__ const T* xin() const { return xh; }
    __device__ Pre load(int i) const {
        Pre p;
        p.y = y0[i];
        p.kx = kx0[i];
        p.q = q[i];
        p.ge = sense[i];
        return p;
    }
    __device__ void row(int i, T kxh, const Pre& p, Acc& acc) const {
        T v = p.y + sigma * (p.q - (T(2) * kxh - p.kx));
        if (p.ge && v < T(0)) v = T(0);
        const T d = v - p.y;
        acc.dy2 += d * d;
        acc.inter += d * (kxh - p.kx);
        y1[i] = a * v - b * p.y + g * yanc[i];
        kx1[i] = a * kxh - b * p.kx + g * kxanc[i];
        if (hat) yh[i] = v;
    }
    __device__ void split_acc(int s, const Acc& acc) const {
        const int np = (int)gridDim.x + nsplit;
        part[gridDim.x + s] = (double)acc.dy2;
        part[np + gridDim.x + s] = (double)acc.inter;
    }
    __device__ void finish(Acc& acc) const {
        const double t[2] = {(double)acc.dy2, (double)acc.inter};
        block_partials<2, kSpmvNT>(t, part, (int)gridDim.x + nsplit);
    }
};

// K^T y+ SpMV of a Halpern iteration; the last block sums the iteration's
// partials (||x^ - x||^2 from k_primal_halpern, ||y^ - y||^2 and the interaction
// from the K x^ launch; fixed order), records the fixed-point residual and
// advances the iteration (step_decide), so the iteration needs no separate
// control launch.
template <typename T>
struct EpiPrimalT {
    PDHG_SINGLE_LP_TASK_HOOKS
    Ctrl* ctrl;
    const T* ys0; const T* ys1;     // Y[0], Y[1]
    T* kty0; T* kty1;
    const double* partP;            // ||x' - x||^2 partials of k_primal [nP]
    int nP;
    const double* partD;            // [2][nD] partials of the K x' launch
    int nD;
    int cur; int adapt; int halp;
    struct Pre {};
    struct Acc {};
    // after begin(), the *0 members point at the current half, the *1 members at
    // the other one (y' and the new K^T y')
    __device__ bool begin() {
        if (ctrl->skip) return false;
        cur = ctrl->cur;
        if (cur) {
            const T* t = ys0; ys0 = ys1; ys1 = t;
            T* u = kty0; kty0 = kty1; kty1 = u;
        }
        adapt = ctrl->adaptive;
        halp = ctrl->halpern;
        return true;
    }
    __device__ const T* xin() const { return ys1; }   // y'
    __device__ Pre load(int) const { return Pre{}; }
    __device__ void row(int j, T ktyn, const Pre&, Acc&) const { kty1[j] = ktyn; }
    __device__ void finish(Acc&) const {
        last_block_decide<kSpmvNT>(ctrl, partD, nD, partP, nP, adapt || halp, adapt, false);
    }
};

// ------------------------------------------------------------------ check kernels

// Adds the pending y of the last accepted iterate to the y sums (its x was
// added by the K^T launch of its attempt) and materialises the averages.  An
// average of points of X (resp. Y) lies in X (resp. Y); the projection applied
// here only removes the rounding of the running sums (it matters for FP32 sums).
// Halpern iterations have no averages: only the start check copies z to XA, YA.
template <typename T>
__global__ void __launch_bounds__(kEW)
k_check_prep(const Ctrl* __restrict__ ctrl, const T* x0, const T* x1, const T* y0, const T* y1,
             T* xs, T* ys, T* xa, T* ya, const T* l, const T* u, const uint8_t* sense, int64_t n,
             int64_t m)
{
    if (!ctrl->want_check) return;
    const int cur = ctrl->cur;
    const StepScalars<T>& sc = step_scalars<T>(*ctrl);
    const T pw = sc.pw;
    const T winv = sc.winv;
    const T* x = cur ? x1 : x0;
    const T* y = cur ? y1 : y0;
    if (ctrl->halpern) {
        // XA, YA hold T(z) of the iteration before this check; the start check
        // takes the start point
        if (!ctrl->first) return;
        for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < n + m;
             t += (int64_t)gridDim.x * kEW) {
            if (t < n) xa[t] = x[t];
            else ya[t - n] = y[t - n];
        }
        return;
    }
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * kEW) {
        if (t < n) {
            T a = xs[t] * winv;
            if (a < l[t]) a = l[t];
            if (a > u[t]) a = u[t];
            xa[t] = a;
        } else {
            const int64_t i = t - n;
            T s = ys[i];
            if (pw != T(0)) { s += pw * y[i]; ys[i] = s; }
            T a = s * winv;
            if (sense[i] && a < T(0)) a = T(0);
            ya[i] = a;
        }
    }
}

// Row side of a KKT check (terms of RowCheck), block partials in FP64:
// part[q * gridDim.x + block], sums q < kRowSums, then the maxima.
template <typename T>
__global__ void __launch_bounds__(kEW)
k_check_rows(const Ctrl* __restrict__ ctrl, const T* y0, const T* y1, const T* kx0,
             const T* kx1, const T* ya, const T* kxa, const T* yanc, const T* q,
             const uint8_t* sense, const T* R, const T* Rinv, int64_t m, double* part)
{
    if (!ctrl->want_check) return;
    const int cur = ctrl->cur;
    const bool inf = infeas_active(*ctrl);
    const T* y = cur ? y1 : y0;
    const T* kx = cur ? kx1 : kx0;
    const T* yp = cur ? y0 : y1;
    const T* kxp = cur ? kx0 : kx1;
    RowCheck<T> rc;
    for (int64_t i = (int64_t)blockIdx.x * kEW + threadIdx.x; i < m; i += (int64_t)gridDim.x * kEW) {
        const T qi = q[i], ri = Rinv[i], kxi = kx[i], yi = y[i];
        const bool ge = sense[i] != 0;
        rc.add(qi, kxi, yi, kxa[i], ya[i], yanc[i], ri, ge);
        if (inf) rc.add_infeas(qi, kxi, kxp[i], yi, yp[i], R[i], ri, ge);
    }
    double v[kRowSums], mx[kRowMax];
#pragma unroll
    for (int k = 0; k < kRowSums; ++k) v[k] = (double)rc.v[k];
#pragma unroll
    for (int k = 0; k < kRowMax; ++k) mx[k] = (double)rc.mx[k];
    block_partials<kRowSums, kEW>(v, part, gridDim.x);
    block_partials_max<kRowMax, kEW>(mx, part + (size_t)kRowSums * gridDim.x, gridDim.x);
}

// Column side (terms of ColCheck), same layout with kColSums / kColMax.
template <typename T>
__global__ void __launch_bounds__(kEW)
k_check_cols(const Ctrl* __restrict__ ctrl, const T* x0, const T* x1, const T* kty0,
             const T* kty1, const T* xa, const T* ktya, const T* xanc, const T* c,
             const T* l, const T* u, const T* C, const T* Cinv, int64_t n, double* part)
{
    if (!ctrl->want_check) return;
    const int cur = ctrl->cur;
    const bool inf = infeas_active(*ctrl);
    const T* x = cur ? x1 : x0;
    const T* kty = cur ? kty1 : kty0;
    const T* xp = cur ? x0 : x1;
    const T* ktyp = cur ? kty0 : kty1;
    ColCheck<T> cc;
    for (int64_t j = (int64_t)blockIdx.x * kEW + threadIdx.x; j < n; j += (int64_t)gridDim.x * kEW) {
        const T cj = c[j], lj = l[j], uj = u[j], ci = Cinv[j], xj = x[j], kj = kty[j];
        const T xan = xanc[j];
        const bool lf = isfinite(lj), uf = isfinite(uj);
        cc.side(0, cj, kj, xj, xan, lj, uj, ci, lf, uf);
        cc.side(1, cj, ktya[j], xa[j], xan, lj, uj, ci, lf, uf);
        if (inf) cc.add_infeas(cj, xj, xp[j], kj, ktyp[j], lj, uj, C[j], ci, lf, uf);
    }
    double v[kColSums], mx[kColMax];
#pragma unroll
    for (int k = 0; k < kColSums; ++k) v[k] = (double)cc.v[k];
#pragma unroll
    for (int k = 0; k < kColMax; ++k) mx[k] = (double)cc.mx[k];
    block_partials<kColSums, kEW>(v, part, gridDim.x);
    block_partials_max<kColMax, kEW>(mx, part + (size_t)kColSums * gridDim.x, gridDim.x);
}

// KKT_omega (Section 2.4.2), candidate, termination (Section 2.3.2, unscaled),
// restart criteria (Section 2.4.2) and Algorithm 4.
__global__ void __launch_bounds__(kCtlNT)
k_check_ctrl(Ctrl* ctrl, const double* partR, const double* partC, int nparts,
             lp_trace_rec* trace, double* ftab)
{
    if (!ctrl->want_check) return;
    // Algorithm 5's two factors for the attempts of the coming period (k does not
    // change in a check): computed here by all threads at once instead of by the
    // single deciding thread at the end of every K launch, where the two FP64
    // powers sat on each attempt's critical path
    if (ftab && ctrl->adaptive) {
        const int len = ctrl->ftab_len;
        const long long k0 = ctrl->k;
        for (int i = threadIdx.x; i < len; i += kCtlNT) {
            const double kp1 = (double)(k0 + i + 1) + 1.0;
            ftab[i] = 1.0 - pow(kp1, -0.3);
            ftab[len + i] = 1.0 + pow(kp1, -0.6);
        }
        if (threadIdx.x == 0) ctrl->ftab_k0 = k0;
    }
    // one warp per reduced quantity (fixed order: lane-strided sums, then the
    // warp's tree); the Algorithm 6 terms only when the check runs it
    __shared__ double red[kRowQ + kColQ];
    const bool inf = infeas_active(*ctrl);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < kRowQ + kColQ; q += kCtlNT / 32) {
        const bool row_side = q < kRowQ;
        const int k = row_side ? q : q - kRowQ;
        const bool is_max = row_side ? k >= kRowSums : k >= kColSums;
        const bool used = inf || (row_side ? k < 8 : k < 10);
        const double* part = (row_side ? partR : partC) + (size_t)k * nparts;
        double v = 0.0;
        if (used)
            for (int i = lane; i < nparts; i += 32)
                v = is_max ? fmax(v, __ldcg(part + i)) : v + __ldcg(part + i);
        v = is_max ? warp_max(v) : warp_sum(v);
        if (lane == 0) red[q] = v;
    }
    __syncthreads();
    double r[kRowQ], cc[kColQ];
    for (int q = 0; q < kRowQ; ++q) r[q] = red[q];
    for (int q = 0; q < kColQ; ++q) cc[q] = red[kRowQ + q];
    if (threadIdx.x != 0) return;
    check_decide(ctrl, r, cc, trace);
}

// At a restart the iterate becomes the candidate and the anchor (with its K x);
// sums reset.
template <typename T>
__global__ void __launch_bounds__(kEW)
k_restart_apply(const Ctrl* __restrict__ ctrl, T* x0, T* x1, T* y0, T* y1, T* kx0, T* kx1,
                T* kty0, T* kty1, const T* xa, const T* ya, const T* kxa, const T* ktya,
                T* xanc, T* yanc, T* kxanc, T* xs, T* ys, int64_t n, int64_t m)
{
    if (!ctrl->want_check || !ctrl->restart) return;
    const int cur = ctrl->cur, avg = ctrl->cand_avg;
    T* x = cur ? x1 : x0;
    T* y = cur ? y1 : y0;
    T* kx = cur ? kx1 : kx0;
    T* kty = cur ? kty1 : kty0;
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * kEW) {
        if (t < n) {
            T v = x[t];
            if (avg) {
                v = xa[t];
                x[t] = v;
                kty[t] = ktya[t];
            }
            xanc[t] = v;
            xs[t] = T(0);
        } else {
            const int64_t i = t - n;
            T v = y[i];
            T kv = kx[i];
            if (avg) {
                v = ya[i];
                y[i] = v;
                kv = kxa[i];
                kx[i] = kv;
            }
            yanc[i] = v;
            kxanc[i] = kv;
            ys[i] = T(0);
        }
    }
}

__global__ void k_set_cond(Ctrl* ctrl, cudaGraphConditionalHandle handle, int use_handle,
                           int in_body)
{
    if (in_body) ctrl->bodies += 1;
    ctrl->want_check = 0;
    ctrl->t_mode = 0;
    ctrl->restart = 0;
    ctrl->skip = ctrl->done;
    if (use_handle) cudaGraphSetConditional(handle, ctrl->done ? 0u : 1u);
}

// Start point (reading: x = proj_X(0), y = 0; or the warm start) in scaled space.
template <typename T>
__global__ void k_init_state(T* x, T* y, T* xanc, T* yanc, T* xs, T* ys, const T* l, const T* u,
                             const uint8_t* sense, const double* R, const double* C,
                             const double* wx_scaled, const double* wy_scaled,
                             const double* wx_user, const double* wy_user, int64_t n, int64_t m)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n) {
            double v = 0.0;
            if (wx_scaled) v = wx_scaled[t];
            else if (wx_user) v = wx_user[t] / C[t];
            T xv = (T)v;
            if (xv < l[t]) xv = l[t];
            if (xv > u[t]) xv = u[t];
            x[t] = xv;
            xanc[t] = xv;
            xs[t] = T(0);
        } else {
            const int64_t i = t - n;
            double v = 0.0;
            if (wy_scaled) v = wy_scaled[i];
            else if (wy_user) v = wy_user[i] / R[i];
            if (sense[i] && v < 0.0) v = 0.0;
            y[i] = (T)v;
            yanc[i] = (T)v;
            ys[i] = T(0);
        }
    }
}

// Unscaled candidate -> caller buffers (double).
template <typename T>
__global__ void k_extract(const Ctrl* ctrl, const T* x0, const T* x1, const T* y0, const T* y1,
                          const T* xa, const T* ya, const double* R, const double* C,
                          double* xo, double* yo, double* xs_scaled, double* ys_scaled,
                          int64_t n, int64_t m)
{
    const int cur = ctrl->cur, avg = ctrl->cand_avg;
    const T* x = avg ? xa : (cur ? x1 : x0);
    const T* y = avg ? ya : (cur ? y1 : y0);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n) {
            const double v = (double)x[t];
            if (xo) xo[t] = C[t] * v;
            if (xs_scaled) xs_scaled[t] = v;
        } else {
            const int64_t i = t - n;
            const double v = (double)y[i];
            if (yo) yo[i] = R[i] * v;
            if (ys_scaled) ys_scaled[i] = v;
        }
    }
}

// ------------------------------------------------------------------ host side

static inline int ew_grid(int64_t count)
{
    int64_t g = (count + kEW - 1) / kEW;
    if (g < 1) g = 1;
    if (g > kEWGrid) g = kEWGrid;
    return (int)g;
}

__global__ void k_read_clock(unsigned long long* t) { *t = global_ns(); }

#ifndef PDHG_PRIMAL_GRID
#define PDHG_PRIMAL_GRID 608   // 152 SMs x 4 blocks: one wave of the partial-reducing primal step
#endif
template <typename T>
static int primal_grid(int64_t n)
{
    const int g = ew_grid((n + VecTraits<T>::N - 1) / VecTraits<T>::N);
    return g < PDHG_PRIMAL_GRID ? g : PDHG_PRIMAL_GRID;
}

// Whether the primal step of a PDHG attempt runs in the K^T launch's epilogue.
// FP32: yes (on the 1M x 2M power-law LP the K^T launch with the fused step
// takes 109 us against 114 + 16 us for the product and a separate primal
// kernel).  FP64: no; with FP64's fused products the fused launch no longer
// spills but takes 212 us against 173 + 33 us for the product and k_primal
// after it (the elementwise step costs more inside the SpMV, where the FP64 pipe
// is already the limit, than as its own streaming pass).
#ifndef PDHG_FUSE_PRIMAL_F32
#define PDHG_FUSE_PRIMAL_F32 1
#endif
#ifndef PDHG_FUSE_PRIMAL_F64
#define PDHG_FUSE_PRIMAL_F64 0
#endif
template <typename T> struct FusePrimal { static constexpr bool value = PDHG_FUSE_PRIMAL_F32 != 0; };
template <> struct FusePrimal<double> { static constexpr bool value = PDHG_FUSE_PRIMAL_F64 != 0; };

// a candidate x' from X[cur], KTY[cur]: after a check (and at the start), or
// after an unfused K^T launch; the K^T launch's grid, so that the ||x' - x||^2
// partials always number E.gT
template <typename T>
static void launch_primal(Handle* h, Engine<T>& E, cudaStream_t st, int after_step = 0)
{
    k_primal<T><<<E.gT, kEW, 0, st>>>(E.ctrl, E.X[0], E.X[1], E.KTY[0], E.KTY[1], E.c, E.l, E.u,
                                      h->n, E.partT, after_step, E.splitT.n);
}

template <typename T>
static void launch_dual(Handle* h, Engine<T>& E, cudaStream_t st)
{
    EpiDual<T> ed{E.ctrl, E.X[0], E.X[1], E.Y[0], E.Y[1], E.KX[0], E.KX[1], E.YS, E.q, h->sense,
                  E.partD};
    launch_spmv<T>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err, h->n, ed,
                   true, E.splitK);
}

template <typename T>
static void launch_primal_step(Handle* h, Engine<T>& E, cudaStream_t st, bool with_primal = true)
{
    constexpr bool F = FusePrimal<T>::value;
    EpiPrimalStep<T, F> ep{E.ctrl, E.X[0], E.X[1], E.Y[0], E.Y[1], E.KTY[0], E.KTY[1], E.c, E.l,
                           E.u, E.XS, E.partT, h->n};
    launch_spmv<T>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval,
                   h->dev_err, h->m, ep, true, E.splitT);
    if (!F && with_primal) launch_primal<T>(h, E, st, 1);
}

// K^T launch of a Halpern iteration (its last block advances the iteration)
template <typename T>
static void launch_primal_t(Handle* h, Engine<T>& E, cudaStream_t st)
{
    EpiPrimalT<T> et{E.ctrl, E.Y[0], E.Y[1], E.KTY[0], E.KTY[1], E.partT, primal_grid<T>(h->n),
                     E.partD, E.npK};
    launch_spmv<T>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval, h->dev_err, h->m, et,
                   false, E.splitT);
}

template <typename T>
static void launch_primal_halpern(Handle* h, Engine<T>& E, cudaStream_t st)
{
    k_primal_halpern<T><<<primal_grid<T>(h->n), kEW, 0, st>>>(
        E.ctrl, E.X[0], E.X[1], E.KTY[0], E.KTY[1], E.c, E.l, E.u, E.XANC, E.XH, E.XA, h->n,
        E.partT);
}

template <typename T>
static void launch_dual_halpern(Handle* h, Engine<T>& E, cudaStream_t st)
{
    EpiHalpernDual<T> ed{E.ctrl, E.XH, E.Y[0], E.Y[1], E.KX[0], E.KX[1], E.YANC, E.KXANC, E.YA,
                         E.q, h->sense, E.partD};
    launch_spmv<T>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val,
                   h->dev_err, h->n, ed, false, E.splitK);
}

// one step attempt: 2 launches (PDHG) or 3 (a Halpern iteration)
template <typename T>
static void launch_attempt(Handle* h, Engine<T>& E, cudaStream_t st, bool halpern)
{
    if (halpern) {
        launch_primal_halpern<T>(h, E, st);
        launch_dual_halpern<T>(h, E, st);
        launch_primal_t<T>(h, E, st);
    } else {
        launch_dual<T>(h, E, st);
        launch_primal_step<T>(h, E, st);
    }
}

// launches of one attempt and of one check
template <typename T>
inline int attempt_launches(bool halpern) { return halpern ? 3 : (FusePrimal<T>::value ? 2 : 3); }
inline int check_launches(bool halpern) { return halpern ? 9 : 10; }

// The check (every kernel gated on Ctrl::want_check); PDHG loops end it with
// k_primal, the first candidate of the next period.
template <typename T>
static void launch_check(Handle* h, Engine<T>& E, cudaStream_t st, cudaGraphConditionalHandle hd,
                         int use_handle, int in_body, bool halpern)
{
    const int64_t m = h->m, n = h->n;
    k_check_prep<T><<<ew_grid(n + m), kEW, 0, st>>>(E.ctrl, E.X[0], E.X[1], E.Y[0], E.Y[1], E.XS,
                                                     E.YS, E.XA, E.YA, E.l, E.u, h->sense, n, m);
    const int* gate = &E.ctrl->want_check;
    EpiStore<T> e1{E.XA, E.KXA, nullptr, nullptr, gate};
    launch_spmv<T>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err, h->n, e1,
                   false, E.splitK);
    EpiStore<T> e2{E.YA, E.KTYA, nullptr, nullptr, gate};
    launch_spmv<T>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval, h->dev_err, h->m, e2,
                   false, E.splitT);
    k_check_rows<T><<<kEWGrid, kEW, 0, st>>>(E.ctrl, E.Y[0], E.Y[1], E.KX[0], E.KX[1], E.YA,
                                             E.KXA, E.YANC, E.q, h->sense, E.Rt, E.Rinv, m,
                                             E.partR);
    k_check_cols<T><<<kEWGrid, kEW, 0, st>>>(E.ctrl, E.X[0], E.X[1], E.KTY[0], E.KTY[1], E.XA,
                                             E.KTYA, E.XANC, E.c, E.l, E.u, E.Ct, E.Cinv, n,
                                             E.partC);
    k_check_ctrl<<<1, kCtlNT, 0, st>>>(E.ctrl, E.partR, E.partC, kEWGrid, E.trace, E.ftab);
    k_restart_apply<T><<<ew_grid(n + m), kEW, 0, st>>>(
        E.ctrl, E.X[0], E.X[1], E.Y[0], E.Y[1], E.KX[0], E.KX[1], E.KTY[0], E.KTY[1], E.XA, E.YA,
        E.KXA, E.KTYA, E.XANC, E.YANC, E.KXANC, E.XS, E.YS, n, m);
    if (!halpern) launch_primal<T>(h, E, st);
    k_set_cond<<<1, 1, 0, st>>>(E.ctrl, hd, use_handle, in_body);
}

template <typename T>
static lp_status build_graph(Handle* h, Engine<T>& E, int check_every, int slots, int host_loop,
                             int halpern)
{
    if ((E.exec || E.body_exec) && E.graph_check_every == check_every && E.graph_slots == slots &&
        E.graph_host_loop == host_loop && E.graph_halpern == halpern)
        return LP_OK;
    if (E.exec) {
        cudaGraphExecDestroy(E.exec);
        E.exec = nullptr;
    }
    if (E.body_exec) {
        cudaGraphExecDestroy(E.body_exec);
        E.body_exec = nullptr;
    }
    cudaStream_t st = h->stream;
    cudaGraph_t graph = nullptr;
    LP_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle hd{};
    bool conditional = false;
    if (!host_loop) {
        cudaError_t ce = cudaGraphConditionalHandleCreate(&hd, graph, 1, cudaGraphCondAssignDefault);
        conditional = ce == cudaSuccess;
    }
    cudaError_t ce = cudaSuccess;
    cudaGraph_t body = nullptr;
    if (conditional) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
        if (ce == cudaSuccess) body = cp.conditional.phGraph_out[0];
        else conditional = false;
    }
    (void)cudaGetLastError();
    if (conditional) {
        LP_CUDA_TRY(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
        for (int s = 0; s < slots; ++s) launch_attempt<T>(h, E, st, halpern != 0);
        launch_check<T>(h, E, st, hd, 1, 1, halpern != 0);
        cudaGraph_t captured = nullptr;
        LP_CUDA_TRY(cudaStreamEndCapture(st, &captured));
        LP_CUDA_TRY(cudaGraphInstantiate(&E.exec, graph, 0));
        cudaGraphDestroy(graph);
    } else {
        cudaGraphDestroy(graph);
        LP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int s = 0; s < slots; ++s) launch_attempt<T>(h, E, st, halpern != 0);
        launch_check<T>(h, E, st, hd, 0, 1, halpern != 0);
        cudaGraph_t g2 = nullptr;
        LP_CUDA_TRY(cudaStreamEndCapture(st, &g2));
        LP_CUDA_TRY(cudaGraphInstantiate(&E.body_exec, g2, 0));
        cudaGraphDestroy(g2);
    }
    E.graph_conditional = conditional;
    E.graph_check_every = check_every;
    E.graph_slots = slots;
    E.graph_host_loop = host_loop;
    E.graph_halpern = halpern;
    return LP_OK;
}

template <typename T>
lp_status run_solve(Handle* h, const lp_opts* o, double eta0, double omega0,
                    const double* wxs, const double* wys, const double* wxu, const double* wyu,
                    int warm_space, long long k0, long long attempts0, long long restarts0,
                    lp_trace_rec* trace_host, long long trace_cap_host, long long trace_off,
                    Ctrl* out)
{
    Engine<T>& E = engine_of<T>(h);
    const int64_t m = h->m, n = h->n;
    cudaStream_t st = h->stream;
    LP_CUDA_TRY((spmv_prepare<T, EpiStore<T>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiDual<T>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiPrimalT<T>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiPrimalStep<T, FusePrimal<T>::value>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiHalpernDual<T>>()));
    LP_TRY(engine_factors<T>(h));
    if (o->autotune) LP_TRY(tune_engine<T>(h));
    // warm start from the caller (unscaled) must be on the device
    const double* dwx = nullptr;
    const double* dwy = nullptr;
    double* tmp = nullptr;
    if (wxu || wyu) {
        if (warm_space == LP_MEM_DEVICE) {
            dwx = wxu;
            dwy = wyu;
        } else {
            LP_TRY(dev_alloc_n(h, &tmp, (size_t)(n + m)));
            if (wxu) LP_CUDA_TRY(cudaMemcpyAsync(tmp, wxu, sizeof(double) * n, cudaMemcpyHostToDevice, st));
            if (wyu) LP_CUDA_TRY(cudaMemcpyAsync(tmp + n, wyu, sizeof(double) * m, cudaMemcpyHostToDevice, st));
            dwx = wxu ? tmp : nullptr;
            dwy = wyu ? tmp + n : nullptr;
        }
    }
    k_init_state<T><<<ew_grid(n + m), kEW, 0, st>>>(E.X[0], E.Y[0], E.XANC, E.YANC, E.XS, E.YS,
                                                     E.l, E.u, h->sense, h->R, h->C, wxs, wys,
                                                     dwx, dwy, n, m);
    EpiStore<T> e1{E.X[0], E.KX[0], nullptr, nullptr, nullptr};
    launch_spmv<T>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err, h->n, e1,
                   false, E.splitK);
    EpiStore<T> e2{E.Y[0], E.KTY[0], nullptr, nullptr, nullptr};
    launch_spmv<T>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval, h->dev_err, h->m, e2,
                   false, E.splitT);
    LP_CUDA_TRY(cudaGetLastError());
    if (m > 0)
        LP_CUDA_TRY(cudaMemcpyAsync(E.KXANC, E.KX[0], sizeof(T) * m, cudaMemcpyDeviceToDevice, st));

    // device trace buffer
    long long cap = trace_host ? std::max<long long>(0, trace_cap_host - trace_off) : 0;
    if (cap > E.trace_cap) {
        LP_TRY(dev_alloc_n(h, &E.trace, (size_t)cap));
        E.trace_cap = cap;
    }

    // device attempt log (when the caller asked for one)
    long long acap = h->alog_host ? std::max<long long>(0, h->alog_cap_host - h->alog_off) : 0;
    if (acap > E.alog_cap) {
        LP_TRY(dev_alloc_n(h, &E.alog, (size_t)acap * kAttemptFields));
        E.alog_cap = acap;
    }

    if (o->check_every > E.ftab_cap) {
        if (E.ftab) dev_free(h, E.ftab);
        E.ftab = nullptr;
        LP_TRY(dev_alloc_n(h, &E.ftab, 2 * (size_t)o->check_every));
        E.ftab_cap = o->check_every;
    }

    Ctrl c;
    std::memset(&c, 0, sizeof(c));
    c.ftab = E.ftab;
    c.ftab_len = o->check_every;
    c.ftab_k0 = -((long long)1 << 62);   // no period filled yet
    c.alog = acap > 0 ? E.alog : nullptr;
    c.alog_cap = acap;
    c.eta = eta0;
    c.omega = omega0;
    c.kkt_prev = INFINITY;
    c.tol = o->tol;
    c.beta_s = o->beta_sufficient;
    c.beta_n = o->beta_necessary;
    c.beta_a = o->beta_artificial;
    c.eps_zero = o->eps_zero;
    c.qnorm = h->qnorm;
    c.cnorm = h->cnorm;
    c.time_limit_ns = o->time_limit_s * 1e9;
    c.k = k0;
    c.attempts = attempts0;
    c.restarts = restarts0;
    c.max_iters = o->max_iters;
    c.trace_len = 0;
    c.trace_cap = cap;
    c.status = kRunning;
    c.first = 1;
    c.want_check = 1;
    c.skip = 1;
    const int halpern = o->halpern ? 1 : 0;
    c.halpern = halpern;
    c.reflect = o->halpern_reflect;
    c.fpr_prev = INFINITY;
    c.adaptive = o->adaptive_step && !halpern ? 1 : 0;
    c.pwu = o->primal_weight_update ? 1 : 0;
    c.restarts_on = o->restarts ? 1 : 0;
    c.infeas = o->infeas_detect && !halpern ? 1 : 0;
    c.infeas_tol = o->infeas_tol;
    c.check_every = o->check_every;
    c.px = E.partT;
    c.npx = E.npT;
    refresh_scalars(c);
    {
        // the time origin is the device clock read now
        unsigned long long* tns = reinterpret_cast<unsigned long long*>(h->scratch);
        k_read_clock<<<1, 1, 0, st>>>(tns);
        unsigned long long t0 = 0;
        LP_CUDA_TRY(cudaMemcpyAsync(&t0, tns, sizeof(t0), cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
        c.t0_ns = (long long)t0;
    }
    LP_CUDA_TRY(cudaMemcpyAsync(E.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));

    // the start-point check (KKT of z^0, anchor)
    launch_check<T>(h, E, st, cudaGraphConditionalHandle{}, 0, 0, halpern != 0);
    LP_CUDA_TRY(cudaGetLastError());
    // start state, its two products, the clock read, the start check
    h->launches += 3 + 1 + check_launches(halpern != 0);

    const int slots = o->check_every + (c.adaptive ? 4 : 0);
    LP_TRY(build_graph<T>(h, E, o->check_every, slots, o->loop_mode == 1 ? 1 : 0, halpern));
    if (E.graph_conditional) {
        LP_CUDA_TRY(cudaGraphLaunch(E.exec, st));
        LP_CUDA_TRY(cudaMemcpyAsync(out, E.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        // fallback: host loop over body launches, reading the done flag each time
        for (;;) {
            LP_CUDA_TRY(cudaMemcpyAsync(out, E.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            LP_CUDA_TRY(cudaStreamSynchronize(st));
            if (out->done) break;
            LP_CUDA_TRY(cudaGraphLaunch(E.body_exec, st));
        }
    }
    // loop bodies ran on the device: each is `slots` attempts and one check
    h->launches += out->bodies * (long long)(slots * attempt_launches<T>(halpern != 0) +
                                             check_launches(halpern != 0));
    {
        int derr = 0;
        LP_CUDA_TRY(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
        if (derr) return LP_DEVICE_TIMEOUT;
    }
    if (acap > 0) {
        const long long got = std::min<long long>(out->alog_len, acap);
        if (got > 0)
            LP_CUDA_TRY(cudaMemcpyAsync(h->alog_host + kAttemptFields * h->alog_off, E.alog,
                                        sizeof(double) * kAttemptFields * got,
                                        cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (trace_host && cap > 0) {
        const long long got = std::min<long long>(out->trace_len, cap);
        if (got > 0)
            LP_CUDA_TRY(cudaMemcpyAsync(trace_host + trace_off, E.trace, sizeof(lp_trace_rec) * got,
                                        cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (tmp) {
        for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
            if (it->p == tmp) {
                cudaFree(tmp);
                h->allocs.erase(it);
                break;
            }
    }
    return LP_OK;
}

// Writes the unscaled candidate to x / y (space: host or device), or, when
// x_scaled_dev / y_scaled_dev are given, the scaled candidate in FP64.
template <typename T>
lp_status extract_solution_ex(Handle* h, double* x, double* y, int space, double* xs_dev,
                              double* ys_dev)
{
    Engine<T>& E = engine_of<T>(h);
    const int64_t m = h->m, n = h->n;
    cudaStream_t st = h->stream;
    double* dx = x;
    double* dy = y;
    double* tmp = nullptr;
    if (space == LP_MEM_HOST && (x || y)) {
        tmp = h->scratch;   // n + m doubles fit in scratch
        dx = x ? tmp : nullptr;
        dy = y ? tmp + n : nullptr;
    }
    k_extract<T><<<ew_grid(n + m), kEW, 0, st>>>(E.ctrl, E.X[0], E.X[1], E.Y[0], E.Y[1], E.XA, E.YA,
                                                  h->R, h->C, dx, dy, xs_dev, ys_dev, n, m);
    ++h->launches;
    LP_CUDA_TRY(cudaGetLastError());
    if (tmp) {
        if (x) LP_CUDA_TRY(cudaMemcpyAsync(x, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        if (y) LP_CUDA_TRY(cudaMemcpyAsync(y, tmp + n, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    }
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    return LP_OK;
}

template <typename T>
lp_status extract_solution(Handle* h, double* x, double* y, int space)
{
    return extract_solution_ex<T>(h, x, y, space, nullptr, nullptr);
}

template <typename T>
lp_status profile_step(Handle* h, int reps, double* ms, double* bytes)
{
    Engine<T>& E = engine_of<T>(h);
    if (!E.ready || reps <= 0) return LP_INVALID_ARGUMENT;
    cudaStream_t st = h->stream;
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    // free-running state: no check, no stop
    Ctrl c;
    LP_CUDA_TRY(cudaMemcpyAsync(&c, E.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    c.skip = 0;
    c.want_check = 0;
    c.done = 0;
    c.max_iters = (long long)1 << 60;
    c.check_every = 1 << 30;
    c.time_limit_ns = 1e18;
    c.tick = 0;
    c.alog = nullptr;
    LP_CUDA_TRY(cudaMemcpyAsync(E.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    cudaEvent_t ev[4];
    for (auto& e : ev) LP_CUDA_TRY(cudaEventCreate(&e));
    double acc[3] = {0, 0, 0};
    const bool halp = E.graph_halpern == 1;   // the loop of the last lp_solve
    if (!halp) {
        // the candidate x' of the first timed attempt (the check gate of k_primal)
        c.want_check = 1;
        LP_CUDA_TRY(cudaMemcpyAsync(E.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
        launch_primal<T>(h, E, st);
        c.want_check = 0;
        LP_CUDA_TRY(cudaMemcpyAsync(E.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
        h->launches += 1;
    }
    // ev[0..3] bracket three launches: Halpern: primal, K side, K^T side; PDHG:
    // K side (with the decision), K^T side, then the unfused primal step (if any)
    constexpr bool F = FusePrimal<T>::value;
    for (int r = 0; r < reps + 2; ++r) {
        cudaEventRecord(ev[0], st);
        if (halp) launch_primal_halpern<T>(h, E, st);
        else launch_dual<T>(h, E, st);
        cudaEventRecord(ev[1], st);
        if (halp) launch_dual_halpern<T>(h, E, st);
        else launch_primal_step<T>(h, E, st, false);
        cudaEventRecord(ev[2], st);
        if (halp) launch_primal_t<T>(h, E, st);
        else if (!F) launch_primal<T>(h, E, st, 1);
        cudaEventRecord(ev[3], st);
        h->launches += halp ? 3 : attempt_launches<T>(false);
        LP_CUDA_TRY(cudaGetLastError());
        LP_CUDA_TRY(cudaEventSynchronize(ev[3]));
        if (r >= 2) {
            for (int k = 0; k < 3; ++k) {
                float t = 0.f;
                cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
                acc[k] += t;
            }
        }
    }
    if (!halp) {
        // order as for Halpern: [0] primal, [1] K side, [2] K^T side
        const double a0 = acc[0], a1 = acc[1], a2 = acc[2];
        acc[0] = a2;
        acc[1] = a0;
        acc[2] = a1;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int k = 0; k < 3; ++k) ms[k] = acc[k] / reps;
    ms[3] = 0.0;
    const bool fused = !halp && F;
    if (bytes) {
        const double s = sizeof(T);
        // Halpern primal: read x, c, l, u, K^T y, x-anchor; write x^, x+; the
        // unfused PDHG primal step: read x, K^T y, c, l, u; write x'
        bytes[0] = halp ? (double)n * 8 * s : (fused ? 0.0 : (double)n * 6 * s);
        // K x' + dual: values + indices + row pointers (int64) + x' (each element
        // gathered at least once) + y, q, K x, y-sum, sense read; y', K x', y-sum written
        // (Halpern: y, q, K x, y-anchor, K x-anchor, sense read; y+, K x+ written)
        bytes[1] = (double)nnz * (s + 4) + (double)(m + 1) * 8 + (double)n * s +
                   (double)m * (7 * s + 1);
        // K^T y' (values + indices + row pointers + y' gathered; K^T y' written);
        // PDHG adds the fused primal step: x', c, l, u, x-sum read; x'', x-sum written
        // (unfused: x', x-sum read and x-sum written)
        bytes[2] = (double)nnz * (s + 4) + (double)(n + 1) * 8 + (double)m * s + (double)n * s +
                   (halp ? 0.0 : (fused ? (double)n * 7 * s : (double)n * 3 * s));
        bytes[3] = 0.0;
    }
    return LP_OK;
}

template lp_status run_solve<double>(Handle*, const lp_opts*, double, double, const double*,
                                     const double*, const double*, const double*, int, long long,
                                     long long, long long, lp_trace_rec*, long long, long long,
                                     Ctrl*);
template lp_status run_solve<float>(Handle*, const lp_opts*, double, double, const double*,
                                    const double*, const double*, const double*, int, long long,
                                    long long, long long, lp_trace_rec*, long long, long long,
                                    Ctrl*);
template lp_status extract_solution<double>(Handle*, double*, double*, int);
template lp_status extract_solution<float>(Handle*, double*, double*, int);
template lp_status extract_solution_ex<double>(Handle*, double*, double*, int, double*, double*);
template lp_status extract_solution_ex<float>(Handle*, double*, double*, int, double*, double*);
template lp_status profile_step<double>(Handle*, int, double*, double*);
template lp_status profile_step<float>(Handle*, int, double*, double*);

}  // namespace pdhg
