// lp_kkt_noalloc: the termination quantities of a primal-dual pair, computed
// without allocating any device memory.
//
// Who needs this: code that cannot call cudaMalloc at the moment it wants to
// check a candidate solution.  Examples are a host that forbids device
// allocation after start-up because an allocation can block or synchronise the
// whole device (real-time control loops, serving processes with strict latency
// budgets), and a plugin that runs inside an application that has already handed
// all device memory to its own pool.
//
// How: all scratch lives in one fixed array in the library's device image
// (g_na_scratch below, LP_KKT_NOALLOC_MAX_DOUBLES doubles = 8 MiB).  Every GPU
// that loads the library holds that array until the process exits.  The caller
// still passes the problem and the point in device memory and receives eight
// doubles on the host.  Every call uses the same array and leaves its contents
// behind; the accumulators that must start at zero are cleared by each call.
// Two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on the array and give wrong results: serialise them.
// The call waits for its stream before it returns (it copies eight doubles to
// the host), so it refuses a stream that is being captured.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace {

constexpr int kNaGrid = 256;   // fixed grid of the reduction kernels
constexpr int kNaNT = 256;
constexpr int kNaQ = 7;        // reduced quantities
constexpr long long kNaMax = LP_KKT_NOALLOC_MAX_DOUBLES;

static __device__ __align__(256) double g_na_scratch[LP_KKT_NOALLOC_MAX_DOUBLES];

// Device address of g_na_scratch on the current device.  In host code the
// symbol itself is only a host-side stand-in, not a device address, so it is
// looked up with the device current, on every call: the lookup is cheap once
// the module is loaded, and a cached address could outlive its context (after
// cudaDeviceReset or a re-created primary context the module, and the array,
// are loaded anew).
lp_status scratch_for_current_device(double** out)
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return LP_CUDA_ERROR;
    }
    *out = static_cast<double*>(p);
    return LP_OK;
}

__global__ void k_na_zero(double* v, int64_t count)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        v[t] = 0.0;
}

// one warp per row: (K x)_i by a warp sum; (K^T y)_j accumulated by atomics.
// The caller's structure is not validated beforehand, so every index is checked
// here: an out-of-range row pointer or column index is skipped and recorded in
// *bad, which turns the call into LP_INVALID_ARGUMENT.
__global__ void k_na_products(int64_t m, int64_t n, int64_t nnz, const int64_t* rp,
                              const int32_t* ci, const double* v, const double* x,
                              const double* y, double* kx, double* kty, unsigned int* bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nw) {
        const double yi = y[i];
        int64_t p0 = rp[i], p1 = rp[i + 1];
        if (p0 < 0 || p1 > nnz || p1 < p0) {
            if (lane == 0) atomicOr(bad, 1u);
            p0 = p1 = 0;
        }
        double a = 0.0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int32_t j = ci[p];
            if (j < 0 || j >= n) {
                atomicOr(bad, 2u);
                continue;
            }
            a += v[p] * x[j];
            if (yi != 0.0) atomicAdd(kty + j, v[p] * yi);
        }
        a = pdhg::warp_sum(a);
        if (lane == 0) kx[i] = a;
    }
}

// partial sums: [0] ||primal residual||^2 [1] q^T y [2] ||dual residual||^2
// [3] c^T x [4] l^T lambda^+ + u^T lambda^- [5] ||q||^2 [6] ||c||^2
__global__ void __launch_bounds__(kNaNT)
k_na_terms(int64_t m, int64_t n, const uint8_t* sense, const double* c, const double* q,
           const double* l, const double* u, const double* x, const double* y,
           const double* kx, const double* kty, double* part)
{
    double s[kNaQ] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t t = (int64_t)blockIdx.x * kNaNT + threadIdx.x; t < m + n;
         t += (int64_t)gridDim.x * kNaNT) {
        if (t < m) {
            double r = q[t] - kx[t];
            if (sense[t] && r < 0.0) r = 0.0;
            s[0] += r * r;
            s[1] += q[t] * y[t];
            s[5] += q[t] * q[t];
        } else {
            const int64_t j = t - m;
            const double vj = c[j] - kty[j];
            const bool lf = isfinite(l[j]), uf = isfinite(u[j]);
            double lam;
            if (!lf && !uf) lam = 0.0;
            else if (!lf) lam = vj < 0.0 ? vj : 0.0;
            else if (!uf) lam = vj > 0.0 ? vj : 0.0;
            else lam = vj;
            const double d = vj - lam;
            s[2] += d * d;
            s[3] += c[j] * x[j];
            if (lam > 0.0) s[4] += l[j] * lam;
            if (lam < 0.0) s[4] += u[j] * lam;
            s[6] += c[j] * c[j];
        }
    }
    pdhg::block_partials<kNaQ, kNaNT>(s, part, gridDim.x);
}

__global__ void k_na_final(const double* part, double* sums)
{
    for (int q = 0; q < kNaQ; ++q) {
        const double v = pdhg::block_sum_array<kNaNT>(part + (size_t)q * kNaGrid, kNaGrid);
        if (threadIdx.x == 0) sums[q] = v;
    }
}

}  // namespace

extern "C" lp_status lp_kkt_noalloc(const lp_desc* d, const double* x, const double* y,
                                    double omega, double* out, void* cuda_stream)
{
    if (!d || !x || !y || !out || d->memory_space != LP_MEM_DEVICE) return LP_INVALID_ARGUMENT;
    if (d->m < 1 || d->n < 1 || d->nnz < 0 || !d->row_ptr || !d->sense || !d->c || !d->q ||
        !d->l || !d->u || (d->nnz > 0 && (!d->col_idx || !d->vals)) || !(omega > 0.0))
        return LP_INVALID_ARGUMENT;
    // layout: K x [m] | K^T y [n] | partials [kNaQ * kNaGrid] | sums [kNaQ] | flag [1]
    const long long need = d->m + d->n + (long long)kNaQ * kNaGrid + kNaQ + 1;
    if (need > kNaMax) return LP_INVALID_ARGUMENT;   // the problem exceeds the fixed scratch
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the call ends with a copy to the host and a stream synchronisation, which
    // would invalidate a capture in progress: refuse before touching the stream
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        return LP_NOT_SUPPORTED;
    }
    if (cap != cudaStreamCaptureStatusNone) return LP_NOT_SUPPORTED;
    // an error left pending by earlier, unrelated work is the caller's: report it
    // without clearing it, before this call launches anything
    if (cudaPeekAtLastError() != cudaSuccess) return LP_CUDA_ERROR;
    double* base = nullptr;
    lp_status s = scratch_for_current_device(&base);
    if (s != LP_OK) return s;
    double* kx = base;
    double* kty = base + d->m;
    double* part = kty + d->n;
    double* sums = part + (size_t)kNaQ * kNaGrid;
    unsigned int* bad = reinterpret_cast<unsigned int*>(sums + kNaQ);
    const int64_t m = d->m, n = d->n;
    // K^T y accumulates with atomics and the flag with atomicOr: both start at 0.
    // Each launch is checked right after it, so only this call's failures map to
    // LP_CUDA_ERROR.
    bool launched = true;
    k_na_zero<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(kty, n);
    launched = launched && cudaGetLastError() == cudaSuccess;
    k_na_zero<<<1, 32, 0, st>>>(sums + kNaQ, 1);
    launched = launched && cudaGetLastError() == cudaSuccess;
    k_na_products<<<(int)std::min<int64_t>((m * 32 + 255) / 256, 65535), 256, 0, st>>>(
        m, n, d->nnz, d->row_ptr, d->col_idx, d->vals, x, y, kx, kty, bad);
    launched = launched && cudaGetLastError() == cudaSuccess;
    k_na_terms<<<kNaGrid, kNaNT, 0, st>>>(m, n, d->sense, d->c, d->q, d->l, d->u, x, y, kx, kty,
                                          part);
    launched = launched && cudaGetLastError() == cudaSuccess;
    k_na_final<<<1, kNaNT, 0, st>>>(part, sums);
    launched = launched && cudaGetLastError() == cudaSuccess;
    double h[kNaQ + 1];
    if (!launched ||
        cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return LP_CUDA_ERROR;
    }
    unsigned int hbad = 0;
    std::memcpy(&hbad, &h[kNaQ], sizeof(hbad));
    if (hbad) return LP_INVALID_ARGUMENT;
    const double pobj = h[3], dobj = h[1] + h[4];
    const double gap = dobj - pobj;
    out[0] = pobj;
    out[1] = dobj;
    out[2] = std::sqrt(h[0]);
    out[3] = std::sqrt(h[2]);
    out[4] = std::fabs(gap) / (1.0 + std::fabs(dobj) + std::fabs(pobj));
    out[5] = out[2] / (1.0 + std::sqrt(h[5]));
    out[6] = out[3] / (1.0 + std::sqrt(h[6]));
    out[7] = std::sqrt(omega * omega * h[0] + h[2] / (omega * omega) + gap * gap);
    return LP_OK;
}
