// Warp-task schedule autotuner: for each orientation (K, K^T) and precision,
// times the SpMV over a few candidate task shapes on the device and keeps the
// fastest.  The row-length distribution decides: long-row matrices favour the
// largest tasks, many short rows can favour fewer rows per task (shorter
// per-row reduction loops) or smaller tasks (more warps in flight).
#include <algorithm>
#include <cfloat>
#include <vector>

#include "common.cuh"
#include "spmv.cuh"

namespace pdhg {

template <typename T>
lp_status tune_schedule(int sms, cudaStream_t st, const RowBlockBuilder& build,
                        const int64_t* h_rp, const int64_t* rp, const int32_t* ci, const T* val,
                        const T* x, T* out, int64_t x_len, int* err, SchedParams* best,
                        float* best_ms)
{
    constexpr int CAPW = cap_w<T>();
    constexpr int VEC = VecTraits<T>::N;
    const int caps[2] = {CAPW, (CAPW / 2) / VEC * VEC};
    const int rows[3] = {kTaskRows, 32, 16};
    LP_CUDA_TRY((spmv_prepare<T, EpiStore<T>>()));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LP_CUDA_TRY(cudaEventCreate(&e0));
    LP_CUDA_TRY(cudaEventCreate(&e1));
    *best = SchedParams{CAPW, kTaskRows};
    *best_ms = FLT_MAX;
    lp_status status = LP_OK;
    for (int ci_ = 0; ci_ < 2 && status == LP_OK; ++ci_) {
        for (int ri = 0; ri < 3 && status == LP_OK; ++ri) {
            if (rows[ri] > kTaskRows || (ri > 0 && rows[ri] == rows[ri - 1])) continue;
            const std::vector<int32_t> b = build(caps[ci_], rows[ri]);
            const int nt = (int)b.size() - 1;
            std::vector<int64_t> nz(b.size());
            for (size_t t = 0; t < b.size(); ++t) nz[t] = h_rp[(size_t)b[t]];
            const int grid = spmv_grid<T>(nt, sms);
            std::vector<int32_t> wb, pm;
            assign_tasks(nz, caps[ci_], grid * kSpmvWorkers, wb, pm);
            int32_t *tb = nullptr, *wbd = nullptr, *pmd = nullptr;
            int64_t* tn = nullptr;
            if (cudaMalloc(&tb, b.size() * sizeof(int32_t)) != cudaSuccess ||
                cudaMalloc(&tn, nz.size() * sizeof(int64_t)) != cudaSuccess ||
                cudaMalloc(&wbd, wb.size() * sizeof(int32_t)) != cudaSuccess ||
                cudaMalloc(&pmd, std::max<size_t>(pm.size(), 1) * sizeof(int32_t)) !=
                    cudaSuccess) {
                (void)cudaGetLastError();
                cudaFree(tb);
                cudaFree(tn);
                cudaFree(wbd);
                status = LP_OUT_OF_MEMORY;
                break;
            }
            cudaMemcpyAsync(tb, b.data(), b.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(tn, nz.data(), nz.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                            st);
            cudaMemcpyAsync(wbd, wb.data(), wb.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            st);
            if (!pm.empty())
                cudaMemcpyAsync(pmd, pm.data(), pm.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, st);
            EpiStore<T> ep{x, out, nullptr, nullptr, nullptr};
            launch_spmv<T>(grid, st, tb, tn, nt, wbd, pmd, rp, ci, val, err, x_len, ep);
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3; ++r)
                launch_spmv<T>(grid, st, tb, tn, nt, wbd, pmd, rp, ci, val, err, x_len, ep);
            cudaEventRecord(e1, st);
            cudaError_t ce = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            cudaFree(tb);
            cudaFree(tn);
            cudaFree(wbd);
            cudaFree(pmd);
            if (ce != cudaSuccess) {
                (void)cudaGetLastError();
                status = LP_CUDA_ERROR;
                break;
            }
            ms /= 3.0f;
            // the first candidate (the compiled default) is kept unless another is
            // faster by more than 3 %, so that timing noise does not flip schedules
            if (*best_ms == FLT_MAX || ms < 0.97f * *best_ms) {
                *best_ms = ms;
                *best = SchedParams{caps[ci_], rows[ri]};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}

template lp_status tune_schedule<double>(int, cudaStream_t, const RowBlockBuilder&,
                                         const int64_t*, const int64_t*, const int32_t*,
                                         const double*, const double*, double*, int64_t, int*,
                                         SchedParams*, float*);
template lp_status tune_schedule<float>(int, cudaStream_t, const RowBlockBuilder&,
                                        const int64_t*, const int64_t*, const int32_t*,
                                        const float*, const float*, float*, int64_t, int*,
                                        SchedParams*, float*);

template <typename T>
lp_status tune_engine(Handle* h)
{
    Engine<T>& E = engine_of<T>(h);
    if (E.tuned) return LP_OK;
    const int64_t m = h->m, n = h->n;
    int sms = 0;
    LP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    // inputs: zeroed averages (scratch until the next check); outputs: their products
    LP_CUDA_TRY(cudaMemsetAsync(E.XA, 0, sizeof(T) * (size_t)n, h->stream));
    LP_CUDA_TRY(cudaMemsetAsync(E.YA, 0, sizeof(T) * (size_t)m, h->stream));
    SchedParams sK, sT;
    float msK = 0.0f, msT = 0.0f;
    const int64_t* hrp = h->h_rp.data();
    const int64_t* htrp = h->h_trp.data();
    LP_TRY(tune_schedule<T>(
        sms, h->stream, [&](int cap, int rows) { return make_row_blocks(hrp, m, cap, rows); },
        hrp, h->rp, h->ci, E.val, E.XA, E.KXA, n, h->dev_err, &sK, &msK));
    LP_TRY(tune_schedule<T>(
        sms, h->stream, [&](int cap, int rows) { return make_row_blocks(htrp, n, cap, rows); },
        htrp, h->trp, h->tci, E.tval, E.YA, E.KTYA, m, h->dev_err, &sT, &msT));
    h->launches += 2 * 6 * 4;
    const bool changed = sK.cap != E.schedK.cap || sK.max_rows != E.schedK.max_rows ||
                         sT.cap != E.schedT.cap || sT.max_rows != E.schedT.max_rows;
    if (changed) {
        LP_TRY(engine_schedule<T>(h, sK, sT));
        for (cudaGraphExec_t* g : {&E.exec, &E.body_exec})
            if (*g) {
                cudaGraphExecDestroy(*g);
                *g = nullptr;
            }
        E.graph_check_every = -1;
    }
    E.tuned = true;
    return LP_OK;
}

template lp_status tune_engine<double>(Handle*);
template lp_status tune_engine<float>(Handle*);

}  // namespace pdhg
