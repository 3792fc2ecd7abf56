// Unrolled fixed-step PDHG and its reverse-mode derivative.
//
// Forward (Algorithm 1, theta = 1, unscaled problem): x' = clamp(x - tau (c - K^T y), l, u),
// y' = proj_Y(y + sigma (q - K (2 x' - x))) for K_iters steps from x = proj_X(0), y = 0.
// Reverse: for one step with v_x = x - tau (c - K^T y), v_y = y + sigma (q - K xbar),
// xbar = 2 x' - x, masks M_x = [l < v_x < u], M_y = [equality row or v_y > 0], and
// incoming adjoints (gx', gy'):
//   gv_y = M_y gy';   gq += sigma gv_y;   gxbar = -sigma K^T gv_y
//   gv_x = M_x (gx' + 2 gxbar);   gc += -tau gv_x
//   gx = gv_x - gxbar;   gy = gv_y + tau K gv_x
//   gK_ij += -sigma gv_y_i xbar_j + tau y_i gv_x_j
// tau and sigma are held constant.  Iterates are checkpointed every ckpt steps;
// the reverse pass recomputes one segment at a time into a ring (x, y and the
// two projection masks of every step of the segment).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "spmv.cuh"

namespace pdhg {

namespace {

inline int ew_grid_g(int64_t count)
{
    int64_t g = (count + kEW - 1) / kEW;
    if (g < 1) g = 1;
    if (g > kEWGrid) g = kEWGrid;
    return (int)g;
}

// x' = clamp(x - tau (c - K^T y), l, u); mask of the strict interior
template <typename T>
__global__ void k_g_primal(const T* x, const T* kty, const T* c, const T* l, const T* u,
                           const double* coef, T* xn, uint8_t* mx, int64_t n)
{
    const T tau = (T)coef[0];
    for (int64_t j = (int64_t)blockIdx.x * kEW + threadIdx.x; j < n; j += (int64_t)gridDim.x * kEW) {
        const T v = x[j] - tau * (c[j] - kty[j]);
        T o = v;
        if (o < l[j]) o = l[j];
        if (o > u[j]) o = u[j];
        xn[j] = o;
        if (mx) mx[j] = (l[j] < v && v < u[j]) ? 1 : 0;
    }
}

// K x' + dual step of the unrolled forward, with the dual mask
template <typename T>
struct EpiGDual {
    PDHG_SINGLE_LP_TASK_HOOKS
    const T* x;          // x' (being multiplied)
    const T* y;          // y
    const T* kx;         // K x
    const T* q;
    const uint8_t* sense;
    const double* coef;  // [1] = sigma
    T* yn;
    T* kxn;
    uint8_t* my;
    struct Pre { T y = 0, kx = 0, q = 0; uint8_t ge = 0; };
    struct Acc {};
    __device__ bool begin() const { return true; }
    __device__ const T* xin() const { return x; }
    __device__ Pre load(int i) const { return Pre{y[i], kx[i], q[i], sense[i]}; }
    __device__ void row(int i, T v, const Pre& p, Acc&) const {
        const T sigma = (T)coef[1];
        const T w = p.y + sigma * (p.q - (T(2) * v - p.kx));
        T o = w;
        if (p.ge && o < T(0)) o = T(0);
        yn[i] = o;
        kxn[i] = v;
        if (my) my[i] = (!p.ge || w > T(0)) ? 1 : 0;
    }
    __device__ void finish(Acc&) const {}
};

// reverse: gv_y = M_y gy; dq += sigma gv_y
template <typename T>
__global__ void k_g_gvy(const uint8_t* my, const T* gy, const double* coef, T* gvy, double* dq,
                        int64_t m)
{
    const double sigma = coef[1];
    for (int64_t i = (int64_t)blockIdx.x * kEW + threadIdx.x; i < m; i += (int64_t)gridDim.x * kEW) {
        const T g = my[i] ? gy[i] : T(0);
        gvy[i] = g;
        dq[i] += sigma * (double)g;
    }
}

// reverse: gv_x = M_x (gx + 2 gxbar); dc += -tau gv_x; gx <- gv_x - gxbar
template <typename T>
__global__ void k_g_gvx(const uint8_t* mx, T* gx, const T* gxbar, const double* coef, T* gvx,
                        double* dc, int64_t n)
{
    const double tau = coef[0];
    for (int64_t j = (int64_t)blockIdx.x * kEW + threadIdx.x; j < n; j += (int64_t)gridDim.x * kEW) {
        const T gb = gxbar[j];
        const T g = mx[j] ? gx[j] + T(2) * gb : T(0);
        gvx[j] = g;
        dc[j] += -tau * (double)g;
        gx[j] = g - gb;
    }
}

// reverse: gy <- gv_y + tau K gv_x (epilogue of the K gv_x product)
template <typename T>
struct EpiGy {
    PDHG_SINGLE_LP_TASK_HOOKS
    const T* gvx;        // being multiplied
    const T* gvy;
    const double* coef;  // [0] = tau
    T* gy;
    struct Pre { T g = 0; };
    struct Acc {};
    __device__ bool begin() const { return true; }
    __device__ const T* xin() const { return gvx; }
    __device__ Pre load(int i) const { return Pre{gvy[i]}; }
    __device__ void row(int i, T v, const Pre& p, Acc&) const { gy[i] = p.g + (T)coef[0] * v; }
    __device__ void finish(Acc&) const {}
};

// reverse: dA_p += -sigma gv_y_i xbar_j + tau y_i gv_x_j for every nonzero p = (i, j)
template <typename T>
__global__ void k_g_sddmm(const int32_t* krow, const int32_t* ci, const T* gvy, const T* gvx,
                          const T* x, const T* xn, const T* y, const double* coef, double* dvals,
                          int64_t nnz)
{
    const double tau = coef[0], sigma = coef[1];
    for (int64_t p = (int64_t)blockIdx.x * kEW + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * kEW) {
        const int32_t i = krow[p], j = ci[p];
        const double xbar = 2.0 * (double)xn[j] - (double)x[j];
        dvals[p] += -sigma * (double)gvy[i] * xbar + tau * (double)y[i] * (double)gvx[j];
    }
}

template <typename T>
__global__ void k_g_init(const T* l, const T* u, T* x, T* y, int64_t n, int64_t m)
{
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < n + m;
         t += (int64_t)gridDim.x * kEW) {
        if (t < n) {
            T v = T(0);
            if (v < l[t]) v = l[t];
            if (v > u[t]) v = u[t];
            x[t] = v;
        } else {
            y[t - n] = T(0);
        }
    }
}

template <typename T>
__global__ void k_g_from_double(const double* src, T* dst, int64_t count)
{
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * kEW)
        dst[t] = (T)src[t];
}

template <typename T>
__global__ void k_g_to_double(const T* src, double* dst, int64_t count)
{
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * kEW)
        dst[t] = (double)src[t];
}

// Everything one unrolled run needs, allocated per call and released at its end.
template <typename T>
struct GradBufs {
    Handle* h = nullptr;
    std::vector<void*> mem;
    lp_status alloc(void** p, size_t bytes)
    {
        cudaError_t e = cudaMalloc(p, bytes + 64);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? LP_OUT_OF_MEMORY : LP_CUDA_ERROR;
        }
        mem.push_back(*p);
        return LP_OK;
    }
    ~GradBufs()
    {
        if (h) cudaStreamSynchronize(h->stream);
        for (void* p : mem) cudaFree(p);
    }
};

// Unscaled data for the unrolled iterations: no Ruiz scaling, so the engine's
// "scaled" copies are the problem itself; step sizes from Algorithm 2 on K.
template <typename T>
lp_status grad_prepare(Handle* h, const lp_opts* o, double* tau, double* sigma)
{
    lp_opts o2 = *o;
    o2.ruiz_iters = 0;
    o2.pock_chambolle = 0;
    LP_TRY(setup_engine<double>(h, &o2));
    double normK = 0.0;
    LP_TRY(setup_scale(h, &o2, &normK));
    if (std::is_same<T, float>::value) LP_TRY(setup_engine<float>(h, &o2));
    double eta = normK > 0.0 ? o->eta_scale / normK : 1.0;
    if (o->eta0 > 0.0) eta = o->eta0;
    double omega = (h->cnorm > o->eps_zero && h->qnorm > o->eps_zero) ? h->cnorm / h->qnorm : 1.0;
    if (o->omega0 > 0.0) omega = o->omega0;
    *tau = eta / omega;
    *sigma = eta * omega;
    LP_CUDA_TRY((spmv_prepare<T, EpiGDual<T>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiStore<T>>()));
    LP_CUDA_TRY((spmv_prepare<T, EpiGy<T>>()));
    return LP_OK;
}

// One forward step from (x, y, kx, kty) into (xn, yn, kxn, ktyn), with masks.
template <typename T>
void forward_step(Handle* h, Engine<T>& E, const double* coef, const T* x, const T* y, const T* kx,
                  const T* kty, T* xn, T* yn, T* kxn, T* ktyn, uint8_t* mx, uint8_t* my)
{
    cudaStream_t st = h->stream;
    k_g_primal<T><<<ew_grid_g(h->n), kEW, 0, st>>>(x, kty, E.c, E.l, E.u, coef, xn, mx, h->n);
    EpiGDual<T> ed{xn, y, kx, E.q, h->sense, coef, yn, kxn, my};
    launch_spmv<T>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err, h->n, ed,
                   false, E.splitK);
    EpiStore<T> et{yn, ktyn, nullptr, nullptr, nullptr};
    launch_spmv<T>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval, h->dev_err, h->m, et,
                   false, E.splitT);
    h->launches += 3;
}

template <typename T>
lp_status products(Handle* h, Engine<T>& E, const T* x, const T* y, T* kx, T* kty)
{
    cudaStream_t st = h->stream;
    EpiStore<T> e1{x, kx, nullptr, nullptr, nullptr};
    launch_spmv<T>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err, h->n, e1,
                   false, E.splitK);
    EpiStore<T> e2{y, kty, nullptr, nullptr, nullptr};
    launch_spmv<T>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval, h->dev_err, h->m, e2,
                   false, E.splitT);
    h->launches += 2;
    LP_CUDA_TRY(cudaGetLastError());
    return LP_OK;
}

lp_status copy_out(Handle* h, double* dst, const double* src_dev, int64_t count, int space)
{
    LP_CUDA_TRY(cudaMemcpyAsync(dst, src_dev, sizeof(double) * (size_t)count,
                                space == LP_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyDeviceToHost,
                                h->stream));
    return LP_OK;
}

template <typename T>
lp_status grad_impl(Handle* h, const lp_opts* o, int K, int ckpt, const double* gxK, double* dc,
                    double* dq, double* dvals, double* xK, double* yK, int space,
                    double* tau_sigma, bool backward)
{
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    cudaStream_t st = h->stream;
    double tau = 0, sigma = 0;
    LP_TRY(grad_prepare<T>(h, o, &tau, &sigma));
    if (tau_sigma) {
        tau_sigma[0] = tau;
        tau_sigma[1] = sigma;
    }
    Engine<T>& E = engine_of<T>(h);
    GradBufs<T> B;
    B.h = h;
    double* coef = nullptr;   // [tau, sigma, -sigma]
    LP_TRY(B.alloc((void**)&coef, 4 * sizeof(double)));
    const double hc[4] = {tau, sigma, -sigma, 0.0};
    LP_CUDA_TRY(cudaMemcpyAsync(coef, hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    const int nseg = ckpt > 0 ? (K + ckpt - 1) / ckpt : 0;
    // checkpoints: (x, y) at t = 0, ckpt, 2 ckpt, ... (< K)
    T *CX = nullptr, *CY = nullptr;
    LP_TRY(B.alloc((void**)&CX, sizeof(T) * (size_t)std::max(1, nseg) * n));
    LP_TRY(B.alloc((void**)&CY, sizeof(T) * (size_t)std::max(1, nseg) * m));
    // forward with checkpointing
    T* x = E.X[0];
    T* y = E.Y[0];
    k_g_init<T><<<ew_grid_g(n + m), kEW, 0, st>>>(E.l, E.u, x, y, n, m);
    ++h->launches;
    LP_TRY(products<T>(h, E, x, y, E.KX[0], E.KTY[0]));
    int cur = 0;
    for (int t = 0; t < K; ++t) {
        if (backward && t % ckpt == 0) {
            const int c = t / ckpt;
            LP_CUDA_TRY(cudaMemcpyAsync(CX + (size_t)c * n, E.X[cur], sizeof(T) * n,
                                        cudaMemcpyDeviceToDevice, st));
            LP_CUDA_TRY(cudaMemcpyAsync(CY + (size_t)c * m, E.Y[cur], sizeof(T) * m,
                                        cudaMemcpyDeviceToDevice, st));
        }
        forward_step<T>(h, E, coef, E.X[cur], E.Y[cur], E.KX[cur], E.KTY[cur], E.X[cur ^ 1],
                        E.Y[cur ^ 1], E.KX[cur ^ 1], E.KTY[cur ^ 1], nullptr, nullptr);
        cur ^= 1;
    }
    LP_CUDA_TRY(cudaGetLastError());
    double* dtmp = nullptr;   // FP64 staging of outputs [max(n, m, nnz)]
    LP_TRY(B.alloc((void**)&dtmp, sizeof(double) * (size_t)std::max({n, m, nnz})));
    if (xK) {
        k_g_to_double<T><<<ew_grid_g(n), kEW, 0, st>>>(E.X[cur], dtmp, n);
        LP_TRY(copy_out(h, xK, dtmp, n, space));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (yK) {
        k_g_to_double<T><<<ew_grid_g(m), kEW, 0, st>>>(E.Y[cur], dtmp, m);
        LP_TRY(copy_out(h, yK, dtmp, m, space));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (!backward) {
        int derr = 0;
        LP_CUDA_TRY(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
        return derr ? LP_DEVICE_TIMEOUT : LP_OK;
    }

    // reverse pass
    T *RX = nullptr, *RY = nullptr, *gx = nullptr, *gy = nullptr, *gvx = nullptr, *gvy = nullptr,
      *gxbar = nullptr;
    uint8_t *RMX = nullptr, *RMY = nullptr;
    double *ddc = nullptr, *ddq = nullptr, *ddv = nullptr;
    LP_TRY(B.alloc((void**)&RX, sizeof(T) * (size_t)(ckpt + 1) * n));
    LP_TRY(B.alloc((void**)&RY, sizeof(T) * (size_t)(ckpt + 1) * m));
    LP_TRY(B.alloc((void**)&RMX, (size_t)ckpt * n));
    LP_TRY(B.alloc((void**)&RMY, (size_t)ckpt * m));
    LP_TRY(B.alloc((void**)&gx, sizeof(T) * n));
    LP_TRY(B.alloc((void**)&gy, sizeof(T) * m));
    LP_TRY(B.alloc((void**)&gvx, sizeof(T) * n));
    LP_TRY(B.alloc((void**)&gvy, sizeof(T) * m));
    LP_TRY(B.alloc((void**)&gxbar, sizeof(T) * n));
    LP_TRY(B.alloc((void**)&ddc, sizeof(double) * n));
    LP_TRY(B.alloc((void**)&ddq, sizeof(double) * m));
    LP_TRY(B.alloc((void**)&ddv, sizeof(double) * (size_t)std::max<int64_t>(nnz, 1)));
    LP_CUDA_TRY(cudaMemsetAsync(ddc, 0, sizeof(double) * n, st));
    LP_CUDA_TRY(cudaMemsetAsync(ddq, 0, sizeof(double) * m, st));
    LP_CUDA_TRY(cudaMemsetAsync(ddv, 0, sizeof(double) * (size_t)std::max<int64_t>(nnz, 1), st));
    LP_CUDA_TRY(cudaMemsetAsync(gy, 0, sizeof(T) * m, st));
    // incoming adjoint of x_K
    {
        double* g64 = dtmp;
        LP_CUDA_TRY(cudaMemcpyAsync(g64, gxK, sizeof(double) * n,
                                    space == LP_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyHostToDevice,
                                    st));
        k_g_from_double<T><<<ew_grid_g(n), kEW, 0, st>>>(g64, gx, n);
        ++h->launches;
    }
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int t0 = sgi * ckpt;
        const int len = std::min(ckpt, K - t0);
        // recompute the segment: ring slot s holds iterate t0 + s, masks of step t0 + s
        LP_CUDA_TRY(cudaMemcpyAsync(RX, CX + (size_t)sgi * n, sizeof(T) * n,
                                    cudaMemcpyDeviceToDevice, st));
        LP_CUDA_TRY(cudaMemcpyAsync(RY, CY + (size_t)sgi * m, sizeof(T) * m,
                                    cudaMemcpyDeviceToDevice, st));
        LP_TRY(products<T>(h, E, RX, RY, E.KX[0], E.KTY[0]));
        int c = 0;
        for (int s = 0; s < len; ++s) {
            forward_step<T>(h, E, coef, RX + (size_t)s * n, RY + (size_t)s * m, E.KX[c], E.KTY[c],
                            RX + (size_t)(s + 1) * n, RY + (size_t)(s + 1) * m, E.KX[c ^ 1],
                            E.KTY[c ^ 1], RMX + (size_t)s * n, RMY + (size_t)s * m);
            c ^= 1;
        }
        // reverse through the segment
        for (int s = len - 1; s >= 0; --s) {
            const T* xs = RX + (size_t)s * n;
            const T* xs1 = RX + (size_t)(s + 1) * n;
            const T* ys = RY + (size_t)s * m;
            k_g_gvy<T><<<ew_grid_g(m), kEW, 0, st>>>(RMY + (size_t)s * m, gy, coef, gvy, ddq, m);
            EpiStore<T> eg{gvy, gxbar, coef + 2, nullptr, nullptr};
            launch_spmv<T>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval, h->dev_err,
                           h->m, eg, false, E.splitT);
            k_g_gvx<T><<<ew_grid_g(n), kEW, 0, st>>>(RMX + (size_t)s * n, gx, gxbar, coef, gvx, ddc,
                                                    n);
            EpiGy<T> ey{gvx, gvy, coef, gy};
            launch_spmv<T>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err,
                           h->n, ey, false, E.splitK);
            if (nnz > 0)
                k_g_sddmm<T><<<ew_grid_g(nnz), kEW, 0, st>>>(h->krow, h->ci, gvy, gvx, xs, xs1, ys,
                                                             coef, ddv, nnz);
            h->launches += 5;
        }
        LP_CUDA_TRY(cudaGetLastError());
    }
    LP_TRY(copy_out(h, dc, ddc, n, space));
    LP_TRY(copy_out(h, dq, ddq, m, space));
    if (nnz > 0) LP_TRY(copy_out(h, dvals, ddv, nnz, space));
    int derr = 0;
    LP_CUDA_TRY(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    return derr ? LP_DEVICE_TIMEOUT : LP_OK;
}

}  // namespace

lp_status run_grad(Handle* h, const lp_opts* o, int K_iters, int ckpt, const double* gxK,
                   double* dc, double* dq, double* dvals, double* xK, int space, double* tau_sigma)
{
    if (o->precision == LP_PREC_MIXED)
        return grad_impl<float>(h, o, K_iters, ckpt, gxK, dc, dq, dvals, xK, nullptr, space,
                                tau_sigma, true);
    return grad_impl<double>(h, o, K_iters, ckpt, gxK, dc, dq, dvals, xK, nullptr, space,
                             tau_sigma, true);
}

lp_status run_unroll(Handle* h, const lp_opts* o, int K_iters, double* xK, double* yK, int space,
                     double* tau_sigma)
{
    if (o->precision == LP_PREC_MIXED)
        return grad_impl<float>(h, o, K_iters, 1, nullptr, nullptr, nullptr, nullptr, xK, yK, space,
                                tau_sigma, false);
    return grad_impl<double>(h, o, K_iters, 1, nullptr, nullptr, nullptr, nullptr, xK, yK, space,
                             tau_sigma, false);
}

}  // namespace pdhg
