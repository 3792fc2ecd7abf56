// Problem setup on the device: copy + validation, the transposed CSR K^T,
// Ruiz / Pock-Chambolle scaling (Algorithm 3, Section 2.4.1), the spectral
// norm estimate (Algorithm 2) and the per-precision scaled copies.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <utility>
#include <type_traits>

#include "common.cuh"
#include "spmv.cuh"

namespace pdhg {

lp_status dev_alloc(Handle* h, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 64;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? LP_OUT_OF_MEMORY : LP_CUDA_ERROR;
    }
    h->allocs.push_back(DevBuf{*p, bytes});
    return LP_OK;
}

void dev_free(Handle* h, void* p)
{
    if (!p) return;
    for (size_t i = 0; i < h->allocs.size(); ++i)
        if (h->allocs[i].p == p) {
            cudaFree(p);
            h->allocs.erase(h->allocs.begin() + (std::ptrdiff_t)i);
            return;
        }
}

std::vector<int32_t> make_row_blocks(const int64_t* rp, int64_t rows, int cap, int max_rows)
{
    std::vector<int32_t> b;
    b.reserve((size_t)(rows / 16 + 2));
    b.push_back(0);
    int64_t nnz_acc = 0, rows_acc = 0;
    for (int64_t r = 0; r < rows; ++r) {
        const int64_t len = rp[r + 1] - rp[r];
        if (len > cap) {
            if (rows_acc > 0) b.push_back((int32_t)r);
            b.push_back((int32_t)(r + 1));
            nnz_acc = rows_acc = 0;
            continue;
        }
        if (rows_acc > 0 && (nnz_acc + len > cap || rows_acc == max_rows)) {
            b.push_back((int32_t)r);
            nnz_acc = rows_acc = 0;
        }
        nnz_acc += len;
        ++rows_acc;
    }
    if (rows_acc > 0) b.push_back((int32_t)rows);
    return b;
}

#ifndef PDHG_TASK_ASSIGN
#define PDHG_TASK_ASSIGN 1
#endif

void assign_tasks(const std::vector<int64_t>& task_nz, int cap, int warps,
                  std::vector<int32_t>& wbeg, std::vector<int32_t>& perm)
{
    const int nt = (int)task_nz.size() - 1;
    if (PDHG_TASK_ASSIGN == 0) {   // round robin: warp w takes tasks w, w + warps, ...
        wbeg.assign((size_t)warps + 1, 0);
        perm.clear();
        for (int w = 0; w < warps; ++w) {
            for (int t = w; t < nt; t += warps) perm.push_back(t);
            wbeg[(size_t)w + 1] = (int32_t)perm.size();
        }
        return;
    }
    std::vector<int64_t> cost((size_t)std::max(nt, 0));
    for (int t = 0; t < nt; ++t) {
        const int64_t len = task_nz[(size_t)t + 1] - task_nz[(size_t)t];
        cost[(size_t)t] = std::max<int64_t>(1, (len + cap - 1) / cap);
    }
    std::vector<int32_t> order((size_t)std::max(nt, 0));
    for (int t = 0; t < nt; ++t) order[(size_t)t] = t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return cost[(size_t)a] > cost[(size_t)b]; });
    using Slot = std::pair<int64_t, int32_t>;   // (load, warp)
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> pq;
    for (int w = 0; w < warps; ++w) pq.push(Slot{0, w});
    std::vector<int32_t> owner((size_t)std::max(nt, 0));
    for (int32_t t : order) {
        const Slot sl = pq.top();
        pq.pop();
        owner[(size_t)t] = sl.second;
        pq.push(Slot{sl.first + cost[(size_t)t], sl.second});
    }
    wbeg.assign((size_t)warps + 1, 0);
    for (int t = 0; t < nt; ++t) ++wbeg[(size_t)owner[(size_t)t] + 1];
    for (int w = 0; w < warps; ++w) wbeg[(size_t)w + 1] += wbeg[(size_t)w];
    std::vector<int32_t> cur(wbeg.begin(), wbeg.end() - 1);
    perm.assign((size_t)std::max(nt, 0), 0);
    for (int t = 0; t < nt; ++t) perm[(size_t)cur[(size_t)owner[(size_t)t]]++] = t;
}

// Busiest-lane steps above which a short task's rows are summed by equal lane
// shares (seg_row_sums) rather than by one group of lanes per row.
#ifndef PDHG_SEG_STEPS_F32
#define PDHG_SEG_STEPS_F32 (1 << 30)   // FP32: lane groups only (equal shares measured no faster)
#endif
#ifndef PDHG_SEG_STEPS_F64
#define PDHG_SEG_STEPS_F64 8
#endif

// Longest worker list (in chunks) of the longest-first assignment of
// assign_tasks, without building the lists.
static int64_t lpt_makespan(const std::vector<int64_t>& cost, int workers)
{
    std::vector<int64_t> c(cost);
    std::sort(c.begin(), c.end(), std::greater<int64_t>());
    using Slot = std::pair<int64_t, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> pq;
    for (int w = 0; w < workers; ++w) pq.push(Slot{0, w});
    int64_t mx = 0;
    for (int64_t x : c) {
        Slot sl = pq.top();
        pq.pop();
        sl.first += x;
        mx = std::max(mx, sl.first);
        pq.push(sl);
    }
    return mx;
}

SplitPlan split_long_rows(std::vector<int32_t>& rows, std::vector<int64_t>& nz, int cap,
                          int workers)
{
    SplitPlan plan;
    const int nt = (int)rows.size() - 1;
    if (!kSpmvWs || nt <= 0 || workers <= 0) return plan;
    std::vector<int64_t> cost((size_t)nt);
    int64_t total = 0;
    for (int t = 0; t < nt; ++t) {
        const int64_t len = nz[(size_t)t + 1] - nz[(size_t)t];
        cost[(size_t)t] = std::max<int64_t>(1, (len + cap - 1) / cap);
        total += cost[(size_t)t];
    }
    const double mean = (double)total / workers;
    if ((double)lpt_makespan(cost, workers) <= 1.15 * std::max(mean, 1.0)) return plan;
    // pieces of about an eighth of a list (at least two chunks)
    const int64_t tp = std::max<int64_t>(2, (int64_t)std::ceil(mean / 8.0));
    std::vector<int32_t> r2;
    std::vector<int64_t> n2;
    r2.reserve(rows.size());
    n2.reserve(nz.size());
    for (int t = 0; t < nt; ++t) {
        const int64_t a = nz[(size_t)t], b = nz[(size_t)t + 1];
        const int64_t c = cost[(size_t)t];
        const bool one_row = rows[(size_t)t + 1] - rows[(size_t)t] == 1;
        if (!one_row || b - a <= cap || c < 2 * tp) {
            r2.push_back(rows[(size_t)t]);
            n2.push_back(a);
            plan.task_piece.push_back(-1);
            continue;
        }
        const int64_t np = (c + tp - 1) / tp;
        const int64_t per = (c + np - 1) / np;   // chunks per piece
        const int s = (int)plan.info.size() / 2;
        plan.info.push_back(plan.npieces);
        int cnt = 0;
        for (int64_t p0 = a; p0 < b; p0 += per * cap) {
            r2.push_back(rows[(size_t)t]);
            n2.push_back(p0);
            plan.task_piece.push_back(plan.npieces + cnt);
            plan.pspl.push_back(s);
            ++cnt;
        }
        plan.info.push_back(cnt);
        plan.npieces += cnt;
    }
    r2.push_back(rows.back());
    n2.push_back(nz.back());
    plan.n = (int)plan.info.size() / 2;
    if (plan.n == 0) return SplitPlan{};
    rows.swap(r2);
    nz.swap(n2);
    return plan;
}

int64_t lane_group_steps(const int64_t* rp, int r0, int nr)
{
    int64_t steps = 0;
    if (nr <= 32) {
        int G = 32;
        while (G > 1 && G * nr > 32) G >>= 1;
        for (int j = 0; j < nr; ++j)
            steps = std::max<int64_t>(steps, (rp[r0 + j + 1] - rp[r0 + j] + G - 1) / G);
    } else {
        for (int j = 0; j < 32; ++j) {
            int64_t t = rp[r0 + j + 1] - rp[r0 + j];
            if (j + 32 < nr) t += rp[r0 + j + 33] - rp[r0 + j + 32];
            steps = std::max(steps, t);
        }
    }
    return steps;
}

std::vector<char> seg_tasks(const int64_t* rp, const std::vector<int32_t>& rows,
                            const std::vector<int64_t>& nz, int cap, int max_steps)
{
    std::vector<char> seg(rows.size() > 0 ? rows.size() - 1 : 0, 0);
    for (size_t t = 0; t + 1 < rows.size(); ++t) {
        const int64_t len = nz[t + 1] - nz[t];
        const int nr = rows[t + 1] - rows[t];
        if (len <= 0 || len > cap || nr <= 0) continue;   // long rows and pieces: no lane groups
        seg[t] = lane_group_steps(rp, rows[t], nr) > max_steps ? 1 : 0;
    }
    return seg;
}

// ------------------------------------------------------------------ kernels

__global__ void k_validate(int64_t m, int64_t n, int64_t nnz, const int64_t* rp,
                           const int32_t* ci, const double* val, const uint8_t* sense,
                           const double* c, const double* q, const double* l,
                           const double* u, int* flags)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    if (t0 == 0 && (rp[0] != 0 || rp[m] != nnz)) f |= 1;
    for (int64_t i = t0; i < m; i += stride) {
        if (rp[i + 1] < rp[i]) f |= 1;
        if (sense[i] > 1) f |= 16;
        if (isnan(q[i]) || isinf(q[i])) f |= 4;
    }
    for (int64_t p = t0; p < nnz; p += stride) {
        if (ci[p] < 0 || ci[p] >= n) f |= 2;
        if (!isfinite(val[p])) f |= 4;
    }
    for (int64_t j = t0; j < n; j += stride) {
        if (isnan(c[j]) || isinf(c[j])) f |= 4;
        if (isnan(l[j]) || isnan(u[j]) || l[j] > u[j] || l[j] == INFINITY || u[j] == -INFINITY)
            f |= 8;
    }
    if (f) atomicOr(flags, f);
}

// one warp per row: krow[p] = i for every nonzero of row i
__global__ void k_row_of_nnz(int64_t m, const int64_t* rp, int32_t* krow)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < m; w += nw)
        for (int64_t p = rp[w] + lane; p < rp[w + 1]; p += 32) krow[p] = (int32_t)w;
}

__global__ void k_col_count(int64_t nnz, const int32_t* ci, int64_t* cnt)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(cnt + ci[p]), 1ull);
}

__global__ void k_scatter_t(int64_t nnz, const int32_t* ci, unsigned long long* cursor,
                            int32_t* tperm)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long pos = atomicAdd(cursor + ci[p], 1ull);
        tperm[pos] = (int32_t)p;
    }
}

// Segments of <= 32 entries: one thread, insertion sort (ascending nonzero index).
__global__ void k_sort_short(int64_t n, const int64_t* trp, int32_t* tperm)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = trp[j], e = trp[j + 1];
        if (e - s > 32) continue;
        for (int64_t a = s + 1; a < e; ++a) {
            const int32_t key = tperm[a];
            int64_t b = a - 1;
            while (b >= s && tperm[b] > key) {
                tperm[b + 1] = tperm[b];
                --b;
            }
            tperm[b + 1] = key;
        }
    }
}

// Longer segments: one block per listed segment, bitonic sort over a
// power-of-two buffer padded with INT32_MAX; the buffer is shared memory when
// it fits (len2 <= smem_cap) and global scratch otherwise.
__global__ void k_sort_long(const int32_t* segs, const int64_t* trp, int32_t* tperm,
                            int32_t* gscratch, int smem_cap)
{
    extern __shared__ int32_t sbuf[];
    const int64_t j = segs[blockIdx.x];
    const int64_t s = trp[j], e = trp[j + 1];
    const int64_t len = e - s;
    int64_t len2 = 1;
    while (len2 < len) len2 <<= 1;
    int32_t* buf = len2 <= smem_cap ? sbuf : gscratch + 2 * s;
    for (int64_t i = threadIdx.x; i < len2; i += blockDim.x)
        buf[i] = i < len ? tperm[s + i] : INT32_MAX;
    __syncthreads();
    for (int64_t k = 2; k <= len2; k <<= 1) {
        for (int64_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (int64_t i = threadIdx.x; i < len2; i += blockDim.x) {
                const int64_t ixj = i ^ jj;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const int32_t a = buf[i], b = buf[ixj];
                    if ((a > b) == up) {
                        buf[i] = b;
                        buf[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) tperm[s + i] = buf[i];
}

__global__ void k_fill_tci(int64_t nnz, const int32_t* tperm, const int32_t* krow, int32_t* tci)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz;
         t += (int64_t)gridDim.x * blockDim.x)
        tci[t] = krow[tperm[t]];
}

template <typename T>
__global__ void k_fill(T* p, int64_t count, T v)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        p[t] = v;
}

// Ruiz: row infinity norms (one warp per row, exact max)
__global__ void k_row_inf(int64_t m, const int64_t* rp, const double* v, double* rn)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the trip count is uniform per warp (w steps by whole warps)
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < m; w += nw) {
        double a = 0.0;
        for (int64_t p = rp[w] + lane; p < rp[w + 1]; p += 32) a = fmax(a, fabs(v[p]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
        if (lane == 0) rn[w] = a;
    }
}

// Ruiz: column infinity norms by an integer max on the bit pattern
// (non-negative IEEE doubles order like their bits).
__global__ void k_col_inf(int64_t nnz, const int32_t* ci, const double* v, unsigned long long* cn)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs(v[p]);
        atomicMax(cn + ci[p], (unsigned long long)__double_as_longlong(a));
    }
}

// deviation max |1 - norm| over non-empty rows and columns -> dev (bit pattern max)
__global__ void k_ruiz_dev(int64_t m, int64_t n, const double* rn, const double* cn,
                           unsigned long long* dev)
{
    double d = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m + n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double v = t < m ? rn[t] : cn[t - m];
        if (v > 0.0) d = fmax(d, fabs(1.0 - v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dev, (unsigned long long)__double_as_longlong(d));
}

// norm -> factor 1/sqrt(norm) (1 for an empty row/column); accumulate
__global__ void k_ruiz_factors(int64_t count, double* nrm, double* acc)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double f = nrm[t] > 0.0 ? 1.0 / sqrt(nrm[t]) : 1.0;
        nrm[t] = f;
        acc[t] *= f;
    }
}

__global__ void k_scale_vals(int64_t nnz, const int32_t* krow, const int32_t* ci,
                             const double* r, const double* s, double* v)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        v[p] = v[p] * r[krow[p]] * s[ci[p]];
}

// |a|^e for the Pock-Chambolle sums: |a|^0 = 1 for a stored nonzero (0 for a
// stored zero); the exponents of alpha in {0, 1/2, 1, 2} by products and square
// roots, others by pow.
__device__ __forceinline__ double pc_pow(double a, double e)
{
    a = fabs(a);
    if (e == 0.0) return a != 0.0 ? 1.0 : 0.0;
    if (e == 1.0) return a;
    if (e == 2.0) return a * a;
    if (e == 0.5) return sqrt(a);
    if (e == 1.5) return a * sqrt(a);
    return pow(a, e);
}

// Pock-Chambolle pass (parameter alpha): sequential per-row sums of
// |v|^(2 - alpha) and per-column sums of |v|^alpha in row order (rows: CSR
// order; columns: K^T order, ascending rows).
__global__ void k_pc_sums(int64_t m, int64_t n, const int64_t* rp, const int64_t* trp,
                          const int32_t* tperm, const double* v, double alpha, double* rs,
                          double* cs)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m + n;
         t += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0;
        if (t < m) {
            const double e = 2.0 - alpha;
            for (int64_t p = rp[t]; p < rp[t + 1]; ++p) a += pc_pow(v[p], e);
            rs[t] = a;
        } else {
            const int64_t j = t - m;
            for (int64_t p = trp[j]; p < trp[j + 1]; ++p) a += pc_pow(v[tperm[p]], alpha);
            cs[j] = a;
        }
    }
}

__global__ void k_scale_vectors(int64_t m, int64_t n, const double* R, const double* C,
                                const double* c0, const double* q0, const double* l0,
                                const double* u0, double* c, double* q, double* l, double* u)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m + n;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n) {
            c[t] = C[t] * c0[t];
            l[t] = l0[t] / C[t];
            u[t] = u0[t] / C[t];
        } else {
            const int64_t i = t - n;
            q[i] = R[i] * q0[i];
        }
    }
}

template <typename T>
__global__ void k_gather_cast(int64_t count, const int32_t* perm, const double* src, T* dst)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (T)src[perm ? perm[t] : t];
}

// FP64 sum of squares: fixed grid, partials then one block
__global__ void k_sumsq_part(int64_t count, const double* v, double* part)
{
    double s = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * kEW + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * kEW)
        s += v[t] * v[t];
    const double a[1] = {s};
    block_partials<1, kEW>(a, part, gridDim.x);
}

__global__ void k_sum_final(const double* part, int count, double* out)
{
    const double s = block_sum_array<kCtlNT>(part, count);
    if (threadIdx.x == 0) *out = s;
}

// power iteration step: inv = 1 / ||b|| (the next K product is scaled by it,
// which is the product with b / ||b||), or stop when ||b|| = 0
__global__ void k_pow_inv_norm(const double* part, int nparts, double* inv, int* go)
{
    if (*go == 0) return;
    const double s = block_sum_array<kCtlNT>(part, nparts);
    if (threadIdx.x == 0) {
        if (s > 0.0) *inv = 1.0 / sqrt(s);
        else *go = 0;
    }
}

// ------------------------------------------------------------------ host

static inline int grid_for(int64_t count, int nt = 256, int cap = 65535 * 8)
{
    int64_t g = (count + nt - 1) / nt;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

static lp_status copy_in(Handle* h, void* dst, const void* src, size_t bytes, int space)
{
    if (bytes == 0) return LP_OK;
    LP_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                                space == LP_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice,
                                h->stream));
    return LP_OK;
}

lp_status sum_of_squares(Handle* h, const double* v, int64_t count, double* out_host)
{
    double* part = h->scratch;   // [kEWGrid] partials, then the total
    const int g = grid_for(count, kEW, kEWGrid);
    k_sumsq_part<<<g, kEW, 0, h->stream>>>(count, v, part);
    k_sum_final<<<1, kCtlNT, 0, h->stream>>>(part, g, part + kEWGrid);
    h->launches += 2;
    LP_CUDA_TRY(cudaGetLastError());
    LP_CUDA_TRY(cudaMemcpyAsync(out_host, part + kEWGrid, sizeof(double),
                                cudaMemcpyDeviceToHost, h->stream));
    LP_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

lp_status setup_create(Handle* h, const lp_desc* d)
{
    const int64_t m = d->m, n = d->n, nnz = d->nnz;
    h->m = m;
    h->n = n;
    h->nnz = nnz;
    LP_TRY(dev_alloc_n(h, &h->rp, (size_t)m + 1));
    LP_TRY(dev_alloc_n(h, &h->ci, pad8(nnz)));
    LP_TRY(dev_alloc_n(h, &h->val0, pad8(nnz)));
    LP_TRY(dev_alloc_n(h, &h->sense, (size_t)m));
    LP_TRY(dev_alloc_n(h, &h->c0, (size_t)n));
    LP_TRY(dev_alloc_n(h, &h->q0, (size_t)m));
    LP_TRY(dev_alloc_n(h, &h->l0, (size_t)n));
    LP_TRY(dev_alloc_n(h, &h->u0, (size_t)n));
    LP_TRY(dev_alloc_n(h, &h->krow, pad8(nnz)));
    LP_TRY(dev_alloc_n(h, &h->trp, (size_t)n + 1));
    LP_TRY(dev_alloc_n(h, &h->tci, pad8(nnz)));
    LP_TRY(dev_alloc_n(h, &h->tperm, pad8(nnz)));
    LP_TRY(dev_alloc_n(h, &h->R, (size_t)m));
    LP_TRY(dev_alloc_n(h, &h->C, (size_t)n));
    h->scratch_bytes = std::max<size_t>((size_t)(2 * pad8(nnz) + 64) * sizeof(int32_t),
                                        (size_t)(std::max(m, n) + 2 * kEWGrid + 64) * sizeof(double));
    h->scratch_bytes = std::max<size_t>(h->scratch_bytes, (size_t)(m + n + 64) * 8 * 2);
    LP_TRY(dev_alloc(h, (void**)&h->scratch, h->scratch_bytes));
    LP_TRY(dev_alloc_n(h, &h->dev_err, 1));
    LP_CUDA_TRY(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));

    LP_CUDA_TRY(cudaMemsetAsync(h->ci, 0, pad8(nnz) * sizeof(int32_t), h->stream));
    LP_CUDA_TRY(cudaMemsetAsync(h->val0, 0, pad8(nnz) * sizeof(double), h->stream));
    const int sp = d->memory_space;
    LP_TRY(copy_in(h, h->rp, d->row_ptr, sizeof(int64_t) * (size_t)(m + 1), sp));
    LP_TRY(copy_in(h, h->ci, d->col_idx, sizeof(int32_t) * (size_t)nnz, sp));
    LP_TRY(copy_in(h, h->val0, d->vals, sizeof(double) * (size_t)nnz, sp));
    LP_TRY(copy_in(h, h->sense, d->sense, (size_t)m, sp));
    LP_TRY(copy_in(h, h->c0, d->c, sizeof(double) * (size_t)n, sp));
    LP_TRY(copy_in(h, h->q0, d->q, sizeof(double) * (size_t)m, sp));
    LP_TRY(copy_in(h, h->l0, d->l, sizeof(double) * (size_t)n, sp));
    LP_TRY(copy_in(h, h->u0, d->u, sizeof(double) * (size_t)n, sp));

    // validation on the device
    int* flags = reinterpret_cast<int*>(h->scratch);
    LP_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), h->stream));
    k_validate<<<grid_for(std::max({m, n, nnz}), 256, 4096), 256, 0, h->stream>>>(
        m, n, nnz, h->rp, h->ci, h->val0, h->sense, h->c0, h->q0, h->l0, h->u0, flags);
    LP_CUDA_TRY(cudaGetLastError());
    int hflags = 0;
    LP_CUDA_TRY(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LP_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (hflags) return LP_INVALID_ARGUMENT;

    // host copy of row_ptr for the row-block scheduler
    h->h_rp.resize((size_t)m + 1);
    LP_CUDA_TRY(cudaMemcpyAsync(h->h_rp.data(), h->rp, sizeof(int64_t) * (size_t)(m + 1),
                                cudaMemcpyDeviceToHost, h->stream));

    // transpose: histogram, host scan, atomic scatter, per-segment sort
    const int gm = grid_for(m * 32, 256);
    k_row_of_nnz<<<gm, 256, 0, h->stream>>>(m, h->rp, h->krow);
    int64_t* cnt = reinterpret_cast<int64_t*>(h->scratch);
    LP_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)n, h->stream));
    k_col_count<<<grid_for(nnz, 256, 8192), 256, 0, h->stream>>>(nnz, h->ci, cnt);
    LP_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> hc((size_t)n);
    LP_CUDA_TRY(cudaMemcpyAsync(hc.data(), cnt, sizeof(int64_t) * (size_t)n,
                                cudaMemcpyDeviceToHost, h->stream));
    LP_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->h_trp.assign((size_t)n + 1, 0);
    std::vector<int32_t> long_segs;
    int64_t max_long = 0;
    for (int64_t j = 0; j < n; ++j) {
        h->h_trp[(size_t)j + 1] = h->h_trp[(size_t)j] + hc[(size_t)j];
        if (hc[(size_t)j] > 32) {
            long_segs.push_back((int32_t)j);
            max_long = std::max(max_long, hc[(size_t)j]);
        }
    }
    LP_CUDA_TRY(cudaMemcpyAsync(h->trp, h->h_trp.data(), sizeof(int64_t) * (size_t)(n + 1),
                                cudaMemcpyHostToDevice, h->stream));
    unsigned long long* cursor = reinterpret_cast<unsigned long long*>(h->scratch);
    LP_CUDA_TRY(cudaMemcpyAsync(cursor, h->trp, sizeof(int64_t) * (size_t)n,
                                cudaMemcpyDeviceToDevice, h->stream));
    k_scatter_t<<<grid_for(nnz, 256, 8192), 256, 0, h->stream>>>(nnz, h->ci, cursor, h->tperm);
    k_sort_short<<<grid_for(n, 256), 256, 0, h->stream>>>(n, h->trp, h->tperm);
    LP_CUDA_TRY(cudaGetLastError());
    if (!long_segs.empty()) {
        int32_t* segs = nullptr;
        int32_t* gscr = nullptr;
        // segment list after the global scratch area (2 * nnz ints)
        LP_TRY(dev_alloc_n(h, &segs, long_segs.size()));
        LP_TRY(dev_alloc_n(h, &gscr, 2 * pad8(nnz)));
        LP_CUDA_TRY(cudaMemcpyAsync(segs, long_segs.data(), sizeof(int32_t) * long_segs.size(),
                                    cudaMemcpyHostToDevice, h->stream));
        const int smem_cap = 8192;
        LP_CUDA_TRY(cudaFuncSetAttribute(k_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_cap * (int)sizeof(int32_t)));
        k_sort_long<<<(int)long_segs.size(), 512, smem_cap * sizeof(int32_t), h->stream>>>(
            segs, h->trp, h->tperm, gscr, smem_cap);
        LP_CUDA_TRY(cudaGetLastError());
        LP_CUDA_TRY(cudaStreamSynchronize(h->stream));
        // the scratch lists are not needed after the sort
        for (auto it = h->allocs.begin(); it != h->allocs.end();) {
            if (it->p == segs || it->p == gscr) {
                cudaFree(it->p);
                it = h->allocs.erase(it);
            } else {
                ++it;
            }
        }
    }
    LP_CUDA_TRY(cudaMemsetAsync(h->tci, 0, pad8(nnz) * sizeof(int32_t), h->stream));
    k_fill_tci<<<grid_for(nnz, 256, 8192), 256, 0, h->stream>>>(nnz, h->tperm, h->krow, h->tci);
    LP_CUDA_TRY(cudaGetLastError());

    // unscaled norms for the relative termination criteria (Section 2.3.2)
    double s = 0.0;
    LP_TRY(sum_of_squares(h, h->q0, m, &s));
    h->qnorm = std::sqrt(s);
    LP_TRY(sum_of_squares(h, h->c0, n, &s));
    h->cnorm = std::sqrt(s);
    return LP_OK;
}

// New values on the same sparsity pattern (any pointer may be NULL = keep).
lp_status setup_update(Handle* h, const double* vals, const double* c, const double* q,
                       const double* l, const double* u, int space)
{
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    if (vals) LP_TRY(copy_in(h, h->val0, vals, sizeof(double) * (size_t)nnz, space));
    if (c) LP_TRY(copy_in(h, h->c0, c, sizeof(double) * (size_t)n, space));
    if (q) LP_TRY(copy_in(h, h->q0, q, sizeof(double) * (size_t)m, space));
    if (l) LP_TRY(copy_in(h, h->l0, l, sizeof(double) * (size_t)n, space));
    if (u) LP_TRY(copy_in(h, h->u0, u, sizeof(double) * (size_t)n, space));
    int* flags = reinterpret_cast<int*>(h->scratch);
    LP_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), h->stream));
    k_validate<<<grid_for(std::max({m, n, nnz}), 256, 4096), 256, 0, h->stream>>>(
        m, n, nnz, h->rp, h->ci, h->val0, h->sense, h->c0, h->q0, h->l0, h->u0, flags);
    LP_CUDA_TRY(cudaGetLastError());
    int hflags = 0;
    LP_CUDA_TRY(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LP_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (hflags) return LP_INVALID_ARGUMENT;
    double s = 0.0;
    LP_TRY(sum_of_squares(h, h->q0, m, &s));
    h->qnorm = std::sqrt(s);
    LP_TRY(sum_of_squares(h, h->c0, n, &s));
    h->cnorm = std::sqrt(s);
    return LP_OK;
}

// Algorithm 3 (+ optional Pock-Chambolle) into e64.val and R, C, the scaled
// vectors e64.c/q/l/u and the scaled transpose e64.tval; then Algorithm 2.
lp_status setup_scale(Handle* h, const lp_opts* o, double* normK)
{
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    Engine<double>& E = h->e64;
    cudaStream_t st = h->stream;
    LP_CUDA_TRY(cudaMemcpyAsync(E.val, h->val0, pad8(nnz) * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
    k_fill<double><<<grid_for(m), 256, 0, st>>>(h->R, m, 1.0);
    ++h->launches;
    k_fill<double><<<grid_for(n), 256, 0, st>>>(h->C, n, 1.0);
    ++h->launches;
    double* rn = h->scratch;
    double* cn = h->scratch + m;
    unsigned long long* dev = reinterpret_cast<unsigned long long*>(h->scratch + m + n);
    for (int it = 0; it < o->ruiz_iters; ++it) {
        k_row_inf<<<grid_for(m * 32), 256, 0, st>>>(m, h->rp, E.val, rn);
        ++h->launches;
        LP_CUDA_TRY(cudaMemsetAsync(cn, 0, sizeof(double) * (size_t)n, st));
        k_col_inf<<<grid_for(nnz, 256, 8192), 256, 0, st>>>(
            nnz, h->ci, E.val, reinterpret_cast<unsigned long long*>(cn));
        ++h->launches;
        LP_CUDA_TRY(cudaMemsetAsync(dev, 0, sizeof(unsigned long long), st));
        k_ruiz_dev<<<grid_for(m + n, 256, 4096), 256, 0, st>>>(m, n, rn, cn, dev);
        ++h->launches;
        LP_CUDA_TRY(cudaGetLastError());
        unsigned long long hdev = 0;
        LP_CUDA_TRY(cudaMemcpyAsync(&hdev, dev, sizeof(hdev), cudaMemcpyDeviceToHost, st));
        LP_CUDA_TRY(cudaStreamSynchronize(st));
        double dv;
        std::memcpy(&dv, &hdev, sizeof(dv));
        if (dv <= o->ruiz_tol) break;
        k_ruiz_factors<<<grid_for(m), 256, 0, st>>>(m, rn, h->R);
        ++h->launches;
        k_ruiz_factors<<<grid_for(n), 256, 0, st>>>(n, cn, h->C);
        ++h->launches;
        k_scale_vals<<<grid_for(nnz, 256, 8192), 256, 0, st>>>(nnz, h->krow, h->ci, rn, cn, E.val);
        ++h->launches;
        LP_CUDA_TRY(cudaGetLastError());
    }
    if (o->pock_chambolle) {
        k_pc_sums<<<grid_for(m + n), 256, 0, st>>>(m, n, h->rp, h->trp, h->tperm, E.val,
                                                   o->pc_alpha, rn, cn);
        ++h->launches;
        k_ruiz_factors<<<grid_for(m), 256, 0, st>>>(m, rn, h->R);
        ++h->launches;
        k_ruiz_factors<<<grid_for(n), 256, 0, st>>>(n, cn, h->C);
        ++h->launches;
        k_scale_vals<<<grid_for(nnz, 256, 8192), 256, 0, st>>>(nnz, h->krow, h->ci, rn, cn, E.val);
        ++h->launches;
        LP_CUDA_TRY(cudaGetLastError());
    }
    k_scale_vectors<<<grid_for(m + n), 256, 0, st>>>(m, n, h->R, h->C, h->c0, h->q0, h->l0, h->u0,
                                                     E.c, E.q, E.l, E.u);
    ++h->launches;
    LP_CUDA_TRY(cudaMemsetAsync(E.tval, 0, pad8(nnz) * sizeof(double), st));
    k_gather_cast<double><<<grid_for(nnz, 256, 8192), 256, 0, st>>>(nnz, h->tperm, E.val, E.tval);
    ++h->launches;
    LP_CUDA_TRY(cudaGetLastError());

    // Algorithm 2 on K~: b = 1; repeat b <- K~^T (K~ b), b <- b / ||b||; ||K~ b||.
    // The normalisation is carried as a scale of the next K~ product
    // (K~ (b / ||b||) = (K~ b) / ||b||), so b is never rewritten.
    double* b = E.XA;          // n
    double* t = E.KXA;         // m
    double* part = h->scratch;  // partials of ||b||^2 (npT) / ||t||^2 (npK)
    int* go = reinterpret_cast<int*>(h->scratch + std::max(E.npK, E.npT) + 8);
    double* inv = h->scratch + std::max(E.npK, E.npT) + 16;   // 1 / ||b||
    LP_CUDA_TRY((spmv_prepare<double, EpiStore<double>>()));
    k_fill<double><<<grid_for(n), 256, 0, st>>>(b, n, 1.0);
    ++h->launches;
    k_fill<double><<<1, 32, 0, st>>>(inv, 1, 1.0);
    ++h->launches;
    LP_CUDA_TRY(cudaMemsetAsync(go, 0, sizeof(int), st));
    k_fill<int><<<1, 32, 0, st>>>(go, 1, 1);
    ++h->launches;
    for (int it = 0; it < o->power_iters; ++it) {
        EpiStore<double> e1{b, t, inv, nullptr, go};
        launch_spmv<double>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err, h->n, e1,
                            false, E.splitK);
        ++h->launches;
        EpiStore<double> e2{t, b, nullptr, part, go};
        launch_spmv<double>(E.gT, st, E.bcol, E.bnzT, E.ntblk, E.wbegT, E.permT, h->trp, h->tci, E.tval, h->dev_err, h->m,
                            e2, false, E.splitT);
        ++h->launches;
        k_pow_inv_norm<<<1, kCtlNT, 0, st>>>(part, E.npT, inv, go);
        ++h->launches;
        LP_CUDA_TRY(cudaGetLastError());
    }
    EpiStore<double> e3{b, t, inv, part, nullptr};
    launch_spmv<double>(E.gK, st, E.brow, E.bnzK, E.nblk, E.wbegK, E.permK, h->rp, h->ci, E.val, h->dev_err, h->n, e3,
                        false, E.splitK);
    ++h->launches;
    k_sum_final<<<1, kCtlNT, 0, st>>>(part, E.npK, part + E.npK + 4);
    ++h->launches;
    LP_CUDA_TRY(cudaGetLastError());
    double s2 = 0.0;
    int derr = 0;
    LP_CUDA_TRY(cudaMemcpyAsync(&s2, part + E.npK + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    LP_CUDA_TRY(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LP_CUDA_TRY(cudaStreamSynchronize(st));
    if (derr) return LP_DEVICE_TIMEOUT;
    *normK = std::sqrt(s2);
    return LP_OK;
}

// Device copy of a split plan (the previous one of the engine is freed); the
// tickets start at zero.
template <typename T>
static lp_status upload_split(Handle* h, const SplitPlan& plan, SplitRows& sp)
{
    dev_free(h, (void*)sp.pspl);
    dev_free(h, (void*)sp.info);
    dev_free(h, sp.cnt);
    dev_free(h, sp.slots);
    sp = SplitRows{};
    if (plan.n == 0) return LP_OK;
    int32_t *pspl = nullptr, *info = nullptr;
    T* slots = nullptr;
    LP_TRY(dev_alloc_n(h, &pspl, (size_t)plan.npieces));
    LP_TRY(dev_alloc_n(h, &info, plan.info.size()));
    LP_TRY(dev_alloc_n(h, &sp.cnt, (size_t)plan.n));
    LP_TRY(dev_alloc_n(h, &slots, (size_t)plan.npieces));
    LP_CUDA_TRY(cudaMemcpyAsync(pspl, plan.pspl.data(), plan.pspl.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaMemcpyAsync(info, plan.info.data(), plan.info.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaMemsetAsync(sp.cnt, 0, (size_t)plan.n * sizeof(int), h->stream));
    sp.pspl = pspl;
    sp.info = info;
    sp.slots = slots;
    sp.n = plan.n;
    return LP_OK;
}

// Allocation, schedules and (for T = float) the FP32 casts of the scaled data.
template <typename T>
lp_status engine_schedule(Handle* h, SchedParams sK, SchedParams sT)
{
    Engine<T>& E = engine_of<T>(h);
    std::vector<int32_t> bk = make_row_blocks(h->h_rp.data(), h->m, sK.cap, sK.max_rows);
    std::vector<int32_t> bt = make_row_blocks(h->h_trp.data(), h->n, sT.cap, sT.max_rows);
    std::vector<int64_t> nk(bk.size()), nt(bt.size());
    for (size_t t = 0; t < bk.size(); ++t) nk[t] = h->h_rp[(size_t)bk[t]];
    for (size_t t = 0; t < bt.size(); ++t) nt[t] = h->h_trp[(size_t)bt[t]];
    int sms = 0;
    LP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int gK = spmv_grid<T>((int)bk.size() - 1, sms), gT = spmv_grid<T>((int)bt.size() - 1, sms);
    // long rows cut into pieces where the lists would be unbalanced (the grids
    // stay those of the uncut schedules)
    const SplitPlan spK = split_long_rows(bk, nk, sK.cap, gK * kSpmvWorkers);
    const SplitPlan spT = split_long_rows(bt, nt, sT.cap, gT * kSpmvWorkers);
    std::vector<int32_t> wk, pk, wt, pt;
    assign_tasks(nk, sK.cap, gK * kSpmvWorkers, wk, pk);
    assign_tasks(nt, sT.cap, gT * kSpmvWorkers, wt, pt);
    for (void* p : {(void*)E.brow, (void*)E.bcol, (void*)E.bnzK, (void*)E.bnzT, (void*)E.wbegK,
                    (void*)E.permK, (void*)E.wbegT, (void*)E.permT})
        dev_free(h, p);
    E.brow = E.bcol = E.wbegK = E.permK = E.wbegT = E.permT = nullptr;
    E.bnzK = E.bnzT = nullptr;
    LP_TRY(upload_split<T>(h, spK, E.splitK));
    LP_TRY(upload_split<T>(h, spT, E.splitT));
    // Row sums of each short task: one group of lanes per row where that is
    // balanced, equal lane shares (seg_row_sums, with its fixed cost of a
    // search and a five-round scan) where the busiest lane would take more than
    // PDHG_SEG_STEPS_* steps.  FP64 only: GB300's FP64 pipe takes a whole warp
    // instruction however few lanes are active (on the 1M x 2M power-law LP it
    // was 81 % busy on the K side, where the busiest lane of a task does 6.1
    // times an equal share; above 8 steps: K side 284 -> 249 us, K^T side
    // 202 -> 193 us).  In FP32 no threshold (16 to 48) was faster than none.
    const int seg_steps = sizeof(T) == 8 ? PDHG_SEG_STEPS_F64 : PDHG_SEG_STEPS_F32;
    const std::vector<char> segK = seg_tasks(h->h_rp.data(), bk, nk, sK.cap, seg_steps);
    const std::vector<char> segT = seg_tasks(h->h_trp.data(), bt, nt, sT.cap, seg_steps);
    for (size_t t = 0; t < segK.size(); ++t)
        if (segK[t]) nk[t] |= kSegBit;
    for (size_t t = 0; t < segT.size(); ++t)
        if (segT[t]) nt[t] |= kSegBit;
    // a piece carries its slot + 1 in the high 32 bits of its first nonzero
    for (size_t t = 0; t < spK.task_piece.size(); ++t)
        if (spK.task_piece[t] >= 0) nk[t] |= (int64_t)(spK.task_piece[t] + 1) << 32;
    for (size_t t = 0; t < spT.task_piece.size(); ++t)
        if (spT.task_piece[t] >= 0) nt[t] |= (int64_t)(spT.task_piece[t] + 1) << 32;
    // step partials: one per block, then one per split row
    const size_t npK = (size_t)gK + (size_t)spK.n, npT = (size_t)gT + (size_t)spT.n;
    const size_t needD = 2 * npK + 8, needT = std::max<size_t>(npT, (size_t)kEWGrid) + 8;
    if (needD > E.partD_cap) {
        dev_free(h, E.partD);
        E.partD = nullptr;
        LP_TRY(dev_alloc_n(h, &E.partD, needD));
        E.partD_cap = needD;
    }
    if (needT > E.partT_cap) {
        dev_free(h, E.partT);
        E.partT = nullptr;
        LP_TRY(dev_alloc_n(h, &E.partT, needT));
        E.partT_cap = needT;
    }
    E.npK = (int)npK;
    E.npT = (int)npT;
    LP_TRY(dev_alloc_n(h, &E.brow, bk.size()));
    LP_TRY(dev_alloc_n(h, &E.bcol, bt.size()));
    LP_TRY(dev_alloc_n(h, &E.bnzK, nk.size()));
    LP_TRY(dev_alloc_n(h, &E.bnzT, nt.size()));
    LP_TRY(dev_alloc_n(h, &E.wbegK, wk.size()));
    LP_TRY(dev_alloc_n(h, &E.permK, pk.size()));
    LP_TRY(dev_alloc_n(h, &E.wbegT, wt.size()));
    LP_TRY(dev_alloc_n(h, &E.permT, pt.size()));
    LP_CUDA_TRY(cudaMemcpyAsync(E.wbegK, wk.data(), wk.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, h->stream));
    if (!pk.empty())
        LP_CUDA_TRY(cudaMemcpyAsync(E.permK, pk.data(), pk.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaMemcpyAsync(E.wbegT, wt.data(), wt.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, h->stream));
    if (!pt.empty())
        LP_CUDA_TRY(cudaMemcpyAsync(E.permT, pt.data(), pt.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaMemcpyAsync(E.brow, bk.data(), bk.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaMemcpyAsync(E.bcol, bt.data(), bt.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaMemcpyAsync(E.bnzK, nk.data(), nk.size() * sizeof(int64_t),
                                cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaMemcpyAsync(E.bnzT, nt.data(), nt.size() * sizeof(int64_t),
                                cudaMemcpyHostToDevice, h->stream));
    LP_CUDA_TRY(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
    E.nblk = (int)bk.size() - 1;
    E.ntblk = (int)bt.size() - 1;
    E.gK = gK;
    E.gT = gT;
    E.schedK = sK;
    E.schedT = sT;
    return LP_OK;
}

template lp_status engine_schedule<double>(Handle*, SchedParams, SchedParams);
template lp_status engine_schedule<float>(Handle*, SchedParams, SchedParams);

template <typename T>
lp_status setup_engine(Handle* h, const lp_opts* o)
{
    (void)o;
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    Engine<T>& E = engine_of<T>(h);
    if (!E.ready) {
        // the K side gathers x (n entries), the K^T side y (m entries)
        LP_TRY(engine_schedule<T>(h, SchedParams{spmv_cap<T>(n), kTaskRows},
                                  SchedParams{spmv_cap<T>(m), kTaskRows}));
        LP_TRY(dev_alloc_n(h, &E.val, pad8(nnz)));
        LP_TRY(dev_alloc_n(h, &E.tval, pad8(nnz)));
        LP_CUDA_TRY(cudaMemsetAsync(E.val, 0, pad8(nnz) * sizeof(T), h->stream));
        LP_CUDA_TRY(cudaMemsetAsync(E.tval, 0, pad8(nnz) * sizeof(T), h->stream));
        T** vn[] = {&E.c, &E.l, &E.u, &E.X[0], &E.X[1], &E.KTY[0], &E.KTY[1],
                    &E.XS, &E.XA, &E.KTYA, &E.XANC, &E.XH};
        for (T** p : vn) LP_TRY(dev_alloc_n(h, p, (size_t)n));
        T** vm[] = {&E.q,  &E.Y[0], &E.Y[1], &E.KX[0], &E.KX[1],
                    &E.YS, &E.YA,   &E.KXA,  &E.YANC,  &E.KXANC};
        for (T** p : vm) LP_TRY(dev_alloc_n(h, p, (size_t)m));
        LP_TRY(dev_alloc_n(h, &E.partR, kRowQ * (size_t)kEWGrid));
        LP_TRY(dev_alloc_n(h, &E.partC, kColQ * (size_t)kEWGrid));
        LP_TRY(dev_alloc_n(h, &E.ctrl, 1));
        E.ready = true;
    }
    if (std::is_same<T, float>::value) {
        const Engine<double>& D = h->e64;
        cudaStream_t st = h->stream;
        k_gather_cast<T><<<grid_for(nnz, 256, 8192), 256, 0, st>>>(nnz, nullptr, D.val, E.val);
        ++h->launches;
        k_gather_cast<T><<<grid_for(nnz, 256, 8192), 256, 0, st>>>(nnz, h->tperm, D.val, E.tval);
        ++h->launches;
        k_gather_cast<T><<<grid_for(n), 256, 0, st>>>(n, nullptr, D.c, E.c);
        ++h->launches;
        k_gather_cast<T><<<grid_for(n), 256, 0, st>>>(n, nullptr, D.l, E.l);
        ++h->launches;
        k_gather_cast<T><<<grid_for(n), 256, 0, st>>>(n, nullptr, D.u, E.u);
        ++h->launches;
        k_gather_cast<T><<<grid_for(m), 256, 0, st>>>(m, nullptr, D.q, E.q);
        ++h->launches;
        LP_CUDA_TRY(cudaGetLastError());
    }
    return LP_OK;
}

template lp_status setup_engine<double>(Handle*, const lp_opts*);
template lp_status setup_engine<float>(Handle*, const lp_opts*);

template <typename T>
__global__ void k_factors(int64_t m, int64_t n, const double* R, const double* C, T* Rt, T* Ct,
                          T* Rinv, T* Cinv)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m + n;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n) {
            Ct[t] = (T)C[t];
            Cinv[t] = (T)(1.0 / C[t]);
        } else {
            const int64_t i = t - n;
            Rt[i] = (T)R[i];
            Rinv[i] = (T)(1.0 / R[i]);
        }
    }
}

template <typename T>
lp_status engine_factors(Handle* h)
{
    Engine<T>& E = engine_of<T>(h);
    const int64_t m = h->m, n = h->n;
    if (!E.Rt) {
        LP_TRY(dev_alloc_n(h, &E.Rt, (size_t)m));
        LP_TRY(dev_alloc_n(h, &E.Rinv, (size_t)m));
        LP_TRY(dev_alloc_n(h, &E.Ct, (size_t)n));
        LP_TRY(dev_alloc_n(h, &E.Cinv, (size_t)n));
    }
    k_factors<T><<<grid_for(m + n), 256, 0, h->stream>>>(m, n, h->R, h->C, E.Rt, E.Ct, E.Rinv,
                                                         E.Cinv);
    ++h->launches;
    LP_CUDA_TRY(cudaGetLastError());
    return LP_OK;
}

template lp_status engine_factors<double>(Handle*);
template lp_status engine_factors<float>(Handle*);

}  // namespace pdhg
