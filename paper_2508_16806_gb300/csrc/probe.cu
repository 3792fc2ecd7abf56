// lp_profile_gather: the gather ceiling of the SpMV kernels, measured on the
// handle's own scaled matrices.
//
// The two products of Algorithm 1 gather one element of an L2-resident vector
// per nonzero (x for K x', y for K^T y').  With random column indices each
// gather is its own 32-byte sector request from the SM, and the SpMV kernels are
// bound by how many such requests the SMs can issue, not by HBM bandwidth.  The
// kernel here is the smallest loop with the same request stream: every thread
// walks a contiguous share of the nonzeros with 16-byte loads of values and
// column indices (coalesced, evict-first), gathers the vector entry of each and
// multiply-adds into one running sum (written once at the end so that nothing is
// optimised away).  No row structure, no epilogue: its time is the floor of a
// CSR product over the same stream of nonzeros.
#include <algorithm>

#include "common.cuh"
#include "spmv.cuh"

namespace pdhg {
namespace {

constexpr int kProbeNT = 256;
constexpr int kProbeU = 2;   // 16-byte vectors per thread and iteration (8 FP32 gathers in flight)

template <typename T, bool L1>
__global__ void __launch_bounds__(kProbeNT)
k_gather_probe(const T* __restrict__ val, const int32_t* __restrict__ ci, int64_t nnz,
               const T* __restrict__ x, T* __restrict__ sink)
{
    using VT = VecTraits<T>;
    constexpr int VEC = VT::N;
    const int64_t nvec = nnz / VEC;
    const int64_t stride = (int64_t)gridDim.x * kProbeNT;
    T acc = T(0);
    int64_t t = (int64_t)blockIdx.x * kProbeNT + threadIdx.x;
    for (; t + (kProbeU - 1) * stride < nvec; t += kProbeU * stride) {
        T v[kProbeU][VEC];
        int c[kProbeU][VEC];
#pragma unroll
        for (int k = 0; k < kProbeU; ++k) {
            const int64_t e = (t + k * stride) * VEC;
            VT::unpack(__ldcs(reinterpret_cast<const typename VT::V*>(val + e)), v[k]);
            VT::unpacki(__ldcs(reinterpret_cast<const typename VT::I*>(ci + e)), c[k]);
        }
#pragma unroll
        for (int k = 0; k < kProbeU; ++k)
#pragma unroll
            for (int q = 0; q < VEC; ++q)
                acc += v[k][q] * (L1 ? __ldg(x + c[k][q]) : ld_gather(x + c[k][q]));
    }
    for (; t < nvec; t += stride) {
        T v[VEC];
        int c[VEC];
        VT::unpack(__ldcs(reinterpret_cast<const typename VT::V*>(val + t * VEC)), v);
        VT::unpacki(__ldcs(reinterpret_cast<const typename VT::I*>(ci + t * VEC)), c);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc += v[q] * (L1 ? __ldg(x + c[q]) : ld_gather(x + c[q]));
    }
    for (int64_t e = nvec * VEC + (int64_t)blockIdx.x * kProbeNT + threadIdx.x; e < nnz;
         e += stride)
        acc += val[e] * x[ci[e]];
    sink[(int64_t)blockIdx.x * kProbeNT + threadIdx.x] = acc;
}

template <typename T>
lp_status probe(Handle* h, int reps, int blocks_per_sm, double* out)
{
    Engine<T>& E = engine_of<T>(h);
    if (!E.ready) return LP_INVALID_ARGUMENT;
    cudaStream_t st = h->stream;
    int dev = 0, sms = 0;
    LP_CUDA_TRY(cudaGetDevice(&dev));
    LP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * blocks_per_sm;
    // the sink: one value per thread, in the handle's scratch when it fits
    T* sink = reinterpret_cast<T*>(h->scratch);
    if ((size_t)grid * kProbeNT * sizeof(T) > h->scratch_bytes) return LP_INVALID_ARGUMENT;
    cudaEvent_t e0, e1;
    LP_CUDA_TRY(cudaEventCreate(&e0));
    LP_CUDA_TRY(cudaEventCreate(&e1));
    // [0] K side (gathers x, n entries), [1] K^T side (gathers y, m entries);
    // through L1 when the vector is at most kL1GatherBytes, else without L1
    // allocation (the SpMV kernels' choice)
    const T* vals[2] = {E.val, E.tval};
    const int32_t* cis[2] = {h->ci, h->tci};
    const T* vec[2] = {E.X[0], E.Y[0]};
    const int64_t len[2] = {h->n, h->m};
    for (int side = 0; side < 2; ++side) {
        const bool l1 = len[side] * (int64_t)sizeof(T) <= kL1GatherBytes;
        for (int r = 0; r < reps + 1; ++r) {
            if (r == 1) cudaEventRecord(e0, st);
            if (l1)
                k_gather_probe<T, true><<<grid, kProbeNT, 0, st>>>(vals[side], cis[side], h->nnz,
                                                                   vec[side], sink);
            else
                k_gather_probe<T, false><<<grid, kProbeNT, 0, st>>>(vals[side], cis[side],
                                                                    h->nnz, vec[side], sink);
        }
        cudaEventRecord(e1, st);
        h->launches += reps + 1;
        LP_CUDA_TRY(cudaGetLastError());
        LP_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        out[side] = ms / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return LP_OK;
}

}  // namespace
}  // namespace pdhg

using namespace pdhg;

extern "C" lp_status lp_profile_gather(lp_handle p, int32_t precision, int32_t reps,
                                       int32_t blocks_per_sm, double* ms_out)
{
    if (!p || !ms_out || reps < 1 || blocks_per_sm < 1 || blocks_per_sm > 8)
        return LP_INVALID_ARGUMENT;
    lp_status s = LP_INVALID_ARGUMENT;
    if (precision == LP_PREC_FP64) s = probe<double>(&p->h, reps, blocks_per_sm, ms_out);
    else if (precision == LP_PREC_MIXED) s = probe<float>(&p->h, reps, blocks_per_sm, ms_out);
    if (s < 0) {
        cudaStreamSynchronize(p->h.stream);
        (void)cudaGetLastError();
    }
    return s;
}
