// Algorithm 7 (fishnet casting, Section 2.5) on the GPU: P candidate points
// advanced together by fixed-step PDHG, so each product with K or K^T is a
// sparse-times-dense product over a row-major n x P (m x P) point block instead
// of P separate SpMVs; cull by duality gap and convex repopulation between
// rounds.  T = double keeps the point blocks and products in FP64 (the cull
// compares gaps, so its decisions are then taken as in the FP64 oracle);
// T = float keeps them in FP32 (GB300's FP64 pipe makes the FP64 block products
// arithmetic-bound: P fused multiply-adds per nonzero), with FP64 gap
// reductions.
//
// Readings shared with the oracle: points x~_p = (||K~||_2 / sqrt(n)) g_p on the
// scaled problem, Y^0 = K~ X^0, k fixed steps of Algorithm 1 per round with the
// solver's initial eta and omega, cull to the half with the smallest |gap|
// (stable by index, survivors in their old order), repopulation at odd rounds
// while more than two columns entered the round, with weights |z| / sum |z|.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "control.cuh"

namespace pdhg {
namespace {

constexpr int kFW = 8;             // warps per block of the block-SpMM kernels
constexpr int kFGrid = 152 * 16;   // grid cap of the block-SpMM kernels (persistent rows loop)

// out[r, p] = sum_k val_k X[col_k, p] for the rows r of a CSR matrix; X is row
// major with P columns (a power of two, 1..64).  One warp per row: lane l serves
// column l % P (and l + 32 when P = 64); for P < 32 the 32 / P lane groups take
// every (32 / P)-th nonzero of each batch of 32 and are added by a fixed
// butterfly.  Each gathered row of X is P contiguous values (coalesced).
// Rows with more nonzeros than this go to k_spmm_long (a block per row), so that
// no single warp walks a power-law row of thousands of nonzeros alone.
constexpr int64_t kLongRow = 32 * kFW;

// Accumulates the batches b0, b0 + stride, ... (32 nonzeros each) of row [s, e)
// into a0 (and a1 for P = 64); every lane of the warp calls it.
template <typename T>
__device__ __forceinline__ void spmm_row_part(const int32_t* __restrict__ ci,
                                              const T* __restrict__ val, int64_t b0, int64_t e,
                                              int64_t stride, int P, const T* __restrict__ X,
                                              int lane, int G, int g, int p, bool two, T& a0,
                                              T& a1)
{
    const unsigned full = 0xffffffffu;
    for (int64_t b = b0; b < e; b += stride) {
        const int64_t k = b + lane;
        const int c = k < e ? ci[k] : 0;
        const T v = k < e ? val[k] : T(0);
        const int cnt = e - b < 32 ? (int)(e - b) : 32;
#pragma unroll 8
        for (int t0 = 0; t0 < cnt; t0 += G) {
            const int t = t0 + g;   // <= 31; lanes past the row's end hold v = 0
            const int ct = __shfl_sync(full, c, t);
            const T vt = __shfl_sync(full, v, t);
            const T* xr = X + (int64_t)ct * P;
            a0 += vt * xr[p];
            if (two) a1 += vt * xr[p + 32];
        }
    }
}

template <typename T, class Epi>
__global__ void __launch_bounds__(kFW * 32)
k_spmm(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
       const T* __restrict__ val, int64_t rows, int P, const T* __restrict__ X, Epi epi)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int Pl = P < 32 ? P : 32;
    const int G = 32 / Pl;
    const int g = lane / Pl, p = lane % Pl;
    const bool two = P == 64;
    for (int64_t r = (int64_t)blockIdx.x * kFW + (threadIdx.x >> 5); r < rows;
         r += (int64_t)gridDim.x * kFW) {
        const int64_t s = rp[r], e = rp[r + 1];
        if (e - s > kLongRow) continue;
        T a0 = 0, a1 = 0;
        spmm_row_part(ci, val, s, e, 32, P, X, lane, G, g, p, two, a0, a1);
        for (int o = Pl; o < 32; o <<= 1) a0 += __shfl_xor_sync(full, a0, o);
        if (g == 0) {
            epi.row(r, p, a0);
            if (two) epi.row(r, p + 32, a1);
        }
    }
}

// The rows longer than kLongRow (listed in `rows`): one block per row, warp w
// takes the row's batches w, w + kFW, ...; the warps' sums are added in warp
// order (fixed) before the epilogue.
template <typename T, class Epi>
__global__ void __launch_bounds__(kFW * 32)
k_spmm_long(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
            const T* __restrict__ val, const int32_t* __restrict__ rows, int count, int P,
            const T* __restrict__ X, Epi epi)
{
    __shared__ T sh[kFW][64];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Pl = P < 32 ? P : 32;
    const int G = 32 / Pl;
    const int g = lane / Pl, p = lane % Pl;
    const bool two = P == 64;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int64_t r = rows[i];
        const int64_t s = rp[r], e = rp[r + 1];
        T a0 = 0, a1 = 0;
        spmm_row_part(ci, val, s + 32 * (int64_t)warp, e, 32 * (int64_t)kFW, P, X, lane, G, g,
                      p, two, a0, a1);
        for (int o = Pl; o < 32; o <<= 1) a0 += __shfl_xor_sync(full, a0, o);
        if (g == 0) {
            sh[warp][p] = a0;
            if (two) sh[warp][p + 32] = a1;
        }
        __syncthreads();
        if (warp == 0 && g == 0) {
            T t0 = 0, t1 = 0;
            for (int w = 0; w < kFW; ++w) {
                t0 += sh[w][p];
                if (two) t1 += sh[w][p + 32];
            }
            epi.row(r, p, t0);
            if (two) epi.row(r, p + 32, t1);
        }
        __syncthreads();
    }
}

template <typename T>
struct FStore {
    T* out;
    int P;
    __device__ void row(int64_t r, int p, T v) const { out[r * P + p] = v; }
};

// x' = proj_X(x - tau (c - K^T y)) per column (Algorithm 1, theta = 1)
template <typename T>
struct FPrimal {
    const T* X;
    T* Xn;
    const T *c, *l, *u;
    T tau;
    int P;
    __device__ void row(int64_t j, int p, T kty) const
    {
        const int64_t t = j * P + p;
        T v = X[t] - tau * (c[j] - kty);
        if (v < l[j]) v = l[j];
        if (v > u[j]) v = u[j];
        Xn[t] = v;
    }
};

// y' = proj_Y(y + sigma (q - (2 K x' - K x))); K x' replaces K x
template <typename T>
struct FDual {
    const T* Y;
    T* Yn;
    T* KX;
    const T* q;
    const uint8_t* sense;
    T sigma;
    int P;
    __device__ void row(int64_t i, int p, T kxn) const
    {
        const int64_t t = i * P + p;
        T v = Y[t] + sigma * (q[i] - (T(2) * kxn - KX[t]));
        if (sense[i] && v < T(0)) v = T(0);
        Yn[t] = v;
        KX[t] = kxn;
    }
};

template <typename T>
__global__ void k_cast(int64_t n, int P, double rad, const double* G, T* X)
{
    const int64_t total = n * P;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        X[t] = (T)(rad * G[t]);
}

// Per-column sums over the rows of a point block, fixed order: thread t of a
// block serves column t % P and rows blockIdx.x * (256 / P) + t / P, ... .
// part[q * P * gridDim.x + p * gridDim.x + block] for the NQ sums.
constexpr int kGapNT = 256;

template <int NQ>
__device__ void column_partials(const double (&v)[NQ], int P, double* part)
{
    __shared__ double sh[NQ][kGapNT];
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    if ((int)threadIdx.x < P) {
        const int per = kGapNT / P;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
            for (int k = 0; k < per; ++k) s += sh[q][k * P + threadIdx.x];
            part[((size_t)q * P + threadIdx.x) * gridDim.x + blockIdx.x] = s;
        }
    }
}

// c~^T x_p and l~^T lambda_p^+ + u~^T lambda_p^-, lambda_p = proj_Lambda(c~ - K~^T y_p)
template <typename T>
__global__ void __launch_bounds__(kGapNT)
k_gap_cols(int64_t n, int P, const T* X, const T* KTY, const T* c, const T* l, const T* u,
           double* part)
{
    const int p = threadIdx.x % P, per = kGapNT / P;
    T a[2] = {T(0), T(0)};
    for (int64_t j = (int64_t)blockIdx.x * per + threadIdx.x / P; j < n;
         j += (int64_t)gridDim.x * per) {
        const int64_t t = j * P + p;
        const T cj = c[j], lj = l[j], uj = u[j];
        a[0] += cj * X[t];
        const T lam = proj_lambda(cj - KTY[t], isfinite(lj), isfinite(uj));
        if (lam > T(0)) a[1] += lj * lam;
        if (lam < T(0)) a[1] += uj * lam;
    }
    const double v[2] = {(double)a[0], (double)a[1]};
    column_partials<2>(v, P, part);
}

// q~^T y_p
template <typename T>
__global__ void __launch_bounds__(kGapNT)
k_gap_rows(int64_t m, int P, const T* Y, const T* q, double* part)
{
    const int p = threadIdx.x % P, per = kGapNT / P;
    T a = T(0);
    for (int64_t i = (int64_t)blockIdx.x * per + threadIdx.x / P; i < m;
         i += (int64_t)gridDim.x * per)
        a += q[i] * Y[i * P + p];
    const double v[1] = {(double)a};
    column_partials<1>(v, P, part);
}

// |pobj_p - dobj_p| per column
__global__ void k_gap_final(int P, const double* partC, int nbC, const double* partR, int nbR,
                            double* gap)
{
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        double pobj = 0.0, lt = 0.0, qy = 0.0;
        for (int b = 0; b < nbC; ++b) pobj += partC[(size_t)p * nbC + b];
        for (int b = 0; b < nbC; ++b) lt += partC[((size_t)P + p) * nbC + b];
        for (int b = 0; b < nbR; ++b) qy += partR[(size_t)p * nbR + b];
        gap[p] = fabs(pobj - (qy + lt));
    }
}

// dst (rows x Pn) from src (rows x Po): columns t < keep copy src column
// kept[t]; column t >= keep is sum_a W[(t - keep) * keep + a] * src column kept[a].
template <typename T>
__global__ void k_combine(int64_t rows, int Po, int Pn, int keep, const int* kept,
                          const double* W, const T* src, T* dst)
{
    const int64_t total = rows * Pn;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Pn;
        const int t = (int)(e - r * Pn);
        const T* s = src + r * Po;
        if (t < keep) {
            dst[e] = s[kept[t]];
        } else {
            const double* w = W + (size_t)(t - keep) * keep;
            T v = T(0);
            for (int a = 0; a < keep; ++a) v += (T)w[a] * s[kept[a]];
            dst[e] = v;
        }
    }
}

template <typename T>
__global__ void k_unscale(int64_t count, const T* v, const double* f, double* out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        out[t] = f[t] * (double)v[t];
}

int ew_blocks(int64_t count)
{
    int64_t g = (count + 255) / 256;
    if (g < 1) g = 1;
    if (g > kEWGrid * 4) g = kEWGrid * 4;
    return (int)g;
}

int spmm_blocks(int64_t rows)
{
    int64_t g = (rows + kFW - 1) / kFW;
    if (g < 1) g = 1;
    if (g > kFGrid) g = kFGrid;
    return (int)g;
}

// Rows of a CSR orientation with more than kLongRow nonzeros (host).
std::vector<int32_t> long_rows(const std::vector<int64_t>& rp)
{
    std::vector<int32_t> out;
    for (size_t r = 0; r + 1 < rp.size(); ++r)
        if (rp[r + 1] - rp[r] > kLongRow) out.push_back((int32_t)r);
    return out;
}

// One block product: the short rows (a warp each), then the long ones (a block each).
template <typename T, class Epi>
void spmm(Handle* h, const int64_t* rp, const int32_t* ci, const T* val, int64_t rows, int P,
          const T* X, const int32_t* lrows, int nlong, const Epi& epi)
{
    k_spmm<T, Epi><<<spmm_blocks(rows), kFW * 32, 0, h->stream>>>(rp, ci, val, rows, P, X, epi);
    ++h->launches;
    if (nlong > 0) {
        k_spmm_long<T, Epi><<<std::min(nlong, kFGrid), kFW * 32, 0, h->stream>>>(
            rp, ci, val, lrows, nlong, P, X, epi);
        ++h->launches;
    }
}

// device buffers owned by one fishnet call
struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    lp_status get(T** p, size_t count)
    {
        *p = nullptr;
        cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *p = nullptr;
            return e == cudaErrorMemoryAllocation ? LP_OUT_OF_MEMORY : LP_CUDA_ERROR;
        }
        ptrs.push_back(*p);
        return LP_OK;
    }
};

}  // namespace

int64_t fishnet_draws(int P)
{
    int64_t total = 0;
    int cols = P, i = 0;
    while (cols > 1) {
        const int keep = cols / 2;
        if ((i & 1) == 1 && cols > 2) {
            total += (int64_t)keep * keep;
            cols = 2 * keep;
        } else {
            cols = keep;
        }
        ++i;
    }
    return total;
}

namespace {

template <typename T>
lp_status fishnet_t(Handle* h, double eta, double omega, double normK, int P, int k_steps,
                    const double* G, const double* Z_host, int64_t nZ, double* x0, double* y0,
                    double* gaps_host, int32_t* rounds_out, int space)
{
    const int64_t m = h->m, n = h->n;
    const Engine<T>& E = engine_of<T>(h);
    cudaStream_t st = h->stream;
    if (fishnet_draws(P) > nZ) return LP_INVALID_ARGUMENT;
    Scratch S;
    T *X, *Xn, *KTY, *Y, *Yn, *KX, *KX2;
    double *Gd = nullptr, *gap, *W, *partC, *partR;
    int* kept_d;
    LP_TRY(S.get(&X, (size_t)n * P));
    LP_TRY(S.get(&Xn, (size_t)n * P));
    LP_TRY(S.get(&KTY, (size_t)n * P));
    LP_TRY(S.get(&Y, (size_t)m * P));
    LP_TRY(S.get(&Yn, (size_t)m * P));
    LP_TRY(S.get(&KX, (size_t)m * P));
    LP_TRY(S.get(&KX2, (size_t)m * P));
    LP_TRY(S.get(&gap, (size_t)P));
    LP_TRY(S.get(&W, (size_t)P * P));
    LP_TRY(S.get(&kept_d, (size_t)P));
    const int nbC = ew_blocks(n), nbR = ew_blocks(m);
    LP_TRY(S.get(&partC, (size_t)2 * P * nbC));
    LP_TRY(S.get(&partR, (size_t)P * nbR));
    if (space == LP_MEM_HOST) {
        LP_TRY(S.get(&Gd, (size_t)n * P));
        LP_CUDA_TRY(cudaMemcpyAsync(Gd, G, sizeof(double) * (size_t)n * P,
                                    cudaMemcpyHostToDevice, st));
        G = Gd;
    }
    const std::vector<int32_t> lk = long_rows(h->h_rp), lt = long_rows(h->h_trp);
    int32_t *lk_d = nullptr, *lt_d = nullptr;
    LP_TRY(S.get(&lk_d, lk.size()));
    LP_TRY(S.get(&lt_d, lt.size()));
    if (!lk.empty())
        LP_CUDA_TRY(cudaMemcpyAsync(lk_d, lk.data(), lk.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, st));
    if (!lt.empty())
        LP_CUDA_TRY(cudaMemcpyAsync(lt_d, lt.data(), lt.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, st));
    const int nlk = (int)lk.size(), nlt = (int)lt.size();
    const T tau = (T)(eta / omega), sigma = (T)(eta * omega);
    // spectral casting, Y^0 = K~ X^0 (also the first K x)
    k_cast<T><<<ew_blocks(n * P), 256, 0, st>>>(n, P, normK / std::sqrt((double)n), G, X);
    ++h->launches;
    spmm<T>(h, h->rp, h->ci, E.val, m, P, X, lk_d, nlk, FStore<T>{Y, P});
    LP_CUDA_TRY(cudaMemcpyAsync(KX, Y, sizeof(T) * (size_t)m * P, cudaMemcpyDeviceToDevice, st));
    LP_CUDA_TRY(cudaGetLastError());

    std::vector<double> gh(P), wh((size_t)P * P);
    std::vector<int> order(P), kept(P);
    int cols = P, round = 0;
    int64_t zpos = 0;
    while (cols > 1) {
        const int j_top = cols;
        for (int t = 0; t < k_steps; ++t) {
            spmm<T>(h, h->trp, h->tci, E.tval, n, cols, Y, lt_d, nlt,
                    FPrimal<T>{X, Xn, E.c, E.l, E.u, tau, cols});
            spmm<T>(h, h->rp, h->ci, E.val, m, cols, Xn, lk_d, nlk,
                    FDual<T>{Y, Yn, KX, E.q, h->sense, sigma, cols});
            std::swap(X, Xn);
            std::swap(Y, Yn);
        }
        // |duality gap| of every column
        spmm<T>(h, h->trp, h->tci, E.tval, n, cols, Y, lt_d, nlt, FStore<T>{KTY, cols});
        k_gap_cols<T><<<nbC, kGapNT, 0, st>>>(n, cols, X, KTY, E.c, E.l, E.u, partC);
        k_gap_rows<T><<<nbR, kGapNT, 0, st>>>(m, cols, Y, E.q, partR);
        k_gap_final<<<1, 64, 0, st>>>(cols, partC, nbC, partR, nbR, gap);
        h->launches += 3;
        LP_CUDA_TRY(cudaGetLastError());
        LP_CUDA_TRY(cudaMemcpyAsync(gh.data(), gap, sizeof(double) * cols,
                                    cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
        if (gaps_host)
            for (int p = 0; p < cols; ++p) gaps_host[(int64_t)round * P + p] = gh[p];
        // cull_points: the half with the smallest gaps, in their old order
        std::iota(order.begin(), order.begin() + cols, 0);
        std::stable_sort(order.begin(), order.begin() + cols,
                         [&](int a, int b) { return gh[a] < gh[b]; });
        const int keep = cols / 2;
        std::copy(order.begin(), order.begin() + keep, kept.begin());
        std::sort(kept.begin(), kept.begin() + keep);
        int ncols = keep;
        // repopulate: one convex combination of the survivors per survivor
        if ((round & 1) == 1 && j_top > 2) {
            for (int t = 0; t < keep; ++t) {
                double sw = 0.0;
                for (int a = 0; a < keep; ++a) {
                    wh[(size_t)t * keep + a] = std::fabs(Z_host[zpos + (int64_t)t * keep + a]);
                    sw += wh[(size_t)t * keep + a];
                }
                for (int a = 0; a < keep; ++a)
                    wh[(size_t)t * keep + a] =
                        sw > 0.0 ? wh[(size_t)t * keep + a] / sw : 1.0 / keep;
            }
            zpos += (int64_t)keep * keep;
            ncols = 2 * keep;
            LP_CUDA_TRY(cudaMemcpyAsync(W, wh.data(), sizeof(double) * (size_t)keep * keep,
                                        cudaMemcpyHostToDevice, st));
        }
        LP_CUDA_TRY(cudaMemcpyAsync(kept_d, kept.data(), sizeof(int) * keep,
                                    cudaMemcpyHostToDevice, st));
        k_combine<T><<<ew_blocks(n * ncols), 256, 0, st>>>(n, cols, ncols, keep, kept_d, W, X, Xn);
        k_combine<T><<<ew_blocks(m * ncols), 256, 0, st>>>(m, cols, ncols, keep, kept_d, W, Y, Yn);
        k_combine<T><<<ew_blocks(m * ncols), 256, 0, st>>>(m, cols, ncols, keep, kept_d, W, KX,
                                                           KX2);
        h->launches += 3;
        LP_CUDA_TRY(cudaGetLastError());
        std::swap(X, Xn);
        std::swap(Y, Yn);
        std::swap(KX, KX2);
        // the host vectors above are reused next round: wait for the copies
        LP_CUDA_TRY(cudaStreamSynchronize(st));
        cols = ncols;
        ++round;
    }
    // the survivor, unscaled (x = C x~, y = R y~)
    double *xo = x0, *yo = y0, *xd = nullptr, *yd = nullptr;
    if (space == LP_MEM_HOST) {
        LP_TRY(S.get(&xd, (size_t)n));
        LP_TRY(S.get(&yd, (size_t)m));
        xo = xd;
        yo = yd;
    }
    k_unscale<T><<<ew_blocks(n), 256, 0, st>>>(n, X, h->C, xo);
    k_unscale<T><<<ew_blocks(m), 256, 0, st>>>(m, Y, h->R, yo);
    h->launches += 2;
    LP_CUDA_TRY(cudaGetLastError());
    if (space == LP_MEM_HOST) {
        LP_CUDA_TRY(cudaMemcpyAsync(x0, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaMemcpyAsync(y0, yd, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    }
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    if (rounds_out) *rounds_out = round;
    return LP_OK;
}

}  // namespace

lp_status run_fishnet(Handle* h, int precision, double eta, double omega, double normK, int P,
                      int k_steps, const double* G, const double* Z_host, int64_t nZ, double* x0,
                      double* y0, double* gaps_host, int32_t* rounds_out, int space)
{
    if (precision == LP_PREC_MIXED)
        return fishnet_t<float>(h, eta, omega, normK, P, k_steps, G, Z_host, nZ, x0, y0,
                                gaps_host, rounds_out, space);
    return fishnet_t<double>(h, eta, omega, normK, P, k_steps, G, Z_host, nZ, x0, y0, gaps_host,
                             rounds_out, space);
}

}  // namespace pdhg
