// Warp-task CSR SpMV with fused epilogues (the products K x and K^T y of
// Algorithm 1, plus whatever elementwise update consumes each row result).
//
// Layout: the rows of a CSR matrix are cut on the host into warp tasks
// (task_row[t] .. task_row[t+1]) of at most CapW<T> nonzeros and at most 64 rows;
// a row longer than CapW<T> forms a task by itself.  Each warp owns one task and
// never waits for the other warps of its block:
//   1. it issues, before anything else, the loads of the task's row pointers
//      and of the epilogue operands of its rows (so their latency overlaps the
//      stream), then U 16-byte vector loads of values and column indices per
//      lane (evict-first, so the gathered vector keeps its place in L2), then all
//      the gathers of x;
//   2. products go to the warp's own slice of shared memory; after __syncwarp
//      each row is summed by a group of G lanes (G = largest power of two with
//      G * rows <= 32) with a shuffle tree, and lane j receives row j's sum;
//   3. lane j applies the epilogue to row j with the operands it prefetched.
// A long row is streamed by the whole warp with the same vector loads and a
// fixed shuffle tree.  All sums have a fixed order: results are bitwise
// reproducible from run to run.  The block's only barrier is in the epilogue's
// block-level partial sums at the end, after each warp has worked through its
// fixed share of the tasks.
//
// Epilogue interface (Epi):
//   bool begin()                        uniform per launch; false = return at once
//   const T* xin()                      the vector being multiplied
//   bool live(int task)                 false: skip the task (a finished LP of a batch)
//   void task_start(int task)           per-task state, before its rows' operands load
//   struct Pre; Pre load(int r)         operands of row r, loaded before the stream
//   struct Acc; void row(int r, T v, const Pre&, Acc&)   once per row, one lane
//   void task_done(int task, Acc&)      after a task's last row (all lanes)
//   void finish(Acc&)                   block-level work at the end (all threads)
// PDHG_SINGLE_LP_TASK_HOOKS supplies the no-op task hooks of a single LP.
#pragma once

#include <functional>
#include <type_traits>

#include "common.cuh"

namespace pdhg {

template <typename T> struct VecTraits;
template <> struct VecTraits<float> {
    using V = float4;
    using I = int4;
    static constexpr int N = 4;
    __device__ static __forceinline__ void unpack(const V& v, float (&o)[4]) {
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static __forceinline__ void unpacki(const I& v, int (&o)[4]) {
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static __forceinline__ V pack(const float (&o)[4]) {
        return make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct VecTraits<double> {
    using V = double2;
    using I = int2;
    static constexpr int N = 2;
    __device__ static __forceinline__ void unpack(const V& v, double (&o)[2]) {
        o[0] = v.x; o[1] = v.y;
    }
    __device__ static __forceinline__ void unpacki(const I& v, int (&o)[2]) {
        o[0] = v.x; o[1] = v.y;
    }
    __device__ static __forceinline__ V pack(const double (&o)[2]) {
        return make_double2(o[0], o[1]);
    }
};

constexpr int kTaskWarps = 8;        // warps per block of the SpMV kernel
#ifndef PDHG_TASK_ROWS
#define PDHG_TASK_ROWS 64
#endif
constexpr int kTaskRows = PDHG_TASK_ROWS;   // rows per warp task at most (32 or 64)
constexpr int kSpmvNT = kTaskWarps * 32;
#ifndef PDHG_SPMV_MIN_BLOCKS
#define PDHG_SPMV_MIN_BLOCKS 4
#endif
constexpr int kSpmvMinBlocks = PDHG_SPMV_MIN_BLOCKS;   // resident blocks per SM the registers allow
#ifndef PDHG_SPMV_MIN_BLOCKS_F64
#define PDHG_SPMV_MIN_BLOCKS_F64 PDHG_SPMV_MIN_BLOCKS
#endif
template <typename T> struct MinBlocks { static constexpr int value = PDHG_SPMV_MIN_BLOCKS; };
template <> struct MinBlocks<double> { static constexpr int value = PDHG_SPMV_MIN_BLOCKS_F64; };
#ifndef PDHG_SPMV_CARVEOUT
#define PDHG_SPMV_CARVEOUT -1
#endif
// Preferred shared-memory carveout of the SpMV kernels in percent of the
// unified L1/shared capacity (-1: the driver's choice).
constexpr int kSpmvCarveout = PDHG_SPMV_CARVEOUT;
#ifndef PDHG_SPMV_UNROLL
#define PDHG_SPMV_UNROLL 2
#endif
// 16-byte loads of values (and of column indices) per lane and task
#ifndef PDHG_SPMV_UNROLL_F64
#define PDHG_SPMV_UNROLL_F64 PDHG_SPMV_UNROLL
#endif
template <typename T> struct Unroll { static constexpr int value = PDHG_SPMV_UNROLL; };
template <> struct Unroll<double> { static constexpr int value = PDHG_SPMV_UNROLL_F64; };
// nonzeros per warp task: one pass of U vector loads per lane covers the task's
// aligned range, whose start may sit up to VEC - 1 elements before the first nonzero
// (PDHG_SPMV_CAP > 0 lowers it, trading nonzeros per stage for a smaller
// shared-memory footprint and so a larger L1 for the gathers)
#ifndef PDHG_SPMV_CAP
#define PDHG_SPMV_CAP 0
#endif
template <typename T>
__host__ __device__ constexpr int cap_w()
{
    return (PDHG_SPMV_CAP > 0 &&
            PDHG_SPMV_CAP < 32 * VecTraits<T>::N * Unroll<T>::value - VecTraits<T>::N)
               ? PDHG_SPMV_CAP
               : 32 * VecTraits<T>::N * Unroll<T>::value - VecTraits<T>::N;
}

// The warp-specialised SpMV's chunk when its gathers hit L1 (a vector of at most
// kL1GatherBytes): a gather costs little there and the chunk's fixed cost
// (copy, hand-overs, row starts) dominates, so chunks take PDHG_SPMV_UNROLL_L1
// 16-byte loads per lane (the 615,001 x 5,000 dispatch LP's K side, x 20 KB:
// 160 -> 132 us with 3).  Schedules of such a side use this capacity.
#ifndef PDHG_SPMV_UNROLL_L1
#define PDHG_SPMV_UNROLL_L1 3
#endif
template <typename T, bool L1G>
__host__ __device__ constexpr int cap_ws()
{
    return L1G && PDHG_SPMV_CAP <= 0 ? 32 * VecTraits<T>::N * PDHG_SPMV_UNROLL_L1 - VecTraits<T>::N
                                      : cap_w<T>();
}

// v[p] x[p] + v[p + step] x[p + step] + ... over [p, pe) by fused multiply-adds
// (one chain).
template <typename T>
__device__ __forceinline__ T strided_dot(const T* v, const T* x, int p, int pe, int step)
{
    T a = 0;
    for (; p < pe; p += step) a = fma(v[p], x[p], a);
    return a;
}

// v[p] + v[p + step] + ... over [p, pe).  In FP32 two partial sums keep two
// shared-memory loads in flight (measured: K side 112 -> 106 us on the 1M x 2M
// LP); in FP64 the single chain is faster (more registers per value).
template <typename T>
__device__ __forceinline__ T strided_sum(const T* v, int p, int pe, int step)
{
    if constexpr (sizeof(T) == 4) {
        T a0 = 0, a1 = 0;
        for (; p + step < pe; p += 2 * step) {
            a0 += v[p];
            a1 += v[p + step];
        }
        if (p < pe) a0 += v[p];
        return a0 + a1;
    } else {
        T a = 0;
        for (; p < pe; p += step) a += v[p];
        return a;
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum_T(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;   // valid in lane 0
}

// Row sums of a short task's products vs[0, len) (rows j < nrows start at
// rps[j], rps[nrows] = len) into rsum[0, nrows), by the whole warp with every
// lane on an equal share: lane l adds the E = ceil(len / 32) consecutive
// products from l E, cutting at row starts.  A row that lies inside one lane's
// share is stored by that lane; the pieces of a row that crosses lanes are
// combined by a segmented inclusive scan over the lanes (Hillis-Steele with the
// row of each lane's last piece as the key; the keys do not decrease from lane
// to lane, so a match over a distance covers every lane between), and the lane
// holding the row's last product stores it.  Rows with no products get 0.  The
// additions have a fixed order, so the sums are bitwise reproducible; the work
// per lane no longer depends on how the row lengths are mixed (with one group
// of lanes per row, a task with one long and many short rows waits for the long
// one).  Leaves the warp synchronised.
// With xs, the terms are the products vs[p] xs[p], taken by fused multiply-adds.
template <typename T>
__device__ __forceinline__ void seg_row_sums(const T* vs, const int* rps, int nrows, int len,
                                             int lane, T* rsum, const T* xs = nullptr)
{
    for (int j = lane; j < nrows; j += 32) rsum[j] = T(0);
    __syncwarp();
    const int E = (len + 31) >> 5;
    const int b = lane * E;
    const int e = b + E < len ? b + E : len;
    int key = -1;        // row of this lane's last piece (-1: no products)
    int rend = 0;        // its end
    int hrow = -1;       // row of the first piece when it continues from earlier lanes and ends here
    T h = T(0), t = T(0);
    if (b < len) {
        // the row holding product b: the last row whose start is <= b (it has products)
        int lo = 0, hi = nrows - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rps[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        int r = lo;
        rend = rps[r + 1];
        const bool cont = rps[r] < b;
        bool first = true;
        T a = T(0);
        for (int p = b; p < e; ++p) {
            if (p >= rend) {
                if (first && cont) {
                    hrow = r;
                    h = a;
                } else {
                    rsum[r] = a;   // a row inside this lane's share
                }
                first = false;
                a = T(0);
                do {
                    ++r;
                    rend = rps[r + 1];
                } while (p >= rend);
            }
            a = xs ? fma(vs[p], xs[p], a) : a + vs[p];
        }
        key = r;
        t = a;
    }
    T S = t;
    int K = key;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T Su = __shfl_up_sync(0xffffffffu, S, d);
        const int Ku = __shfl_up_sync(0xffffffffu, K, d);
        if (lane >= d && Ku == K) S += Su;
    }
    const T Sp = __shfl_up_sync(0xffffffffu, S, 1);
    const int Kp = __shfl_up_sync(0xffffffffu, K, 1);
    // the first piece of a row that began in earlier lanes: their pieces are the
    // previous lane's scan value
    if (hrow >= 0) rsum[hrow] = h + ((lane > 0 && Kp == hrow) ? Sp : T(0));
    // the last piece, where the row ends inside this share
    if (key >= 0 && rend <= e) rsum[key] = S;
    __syncwarp();
}

// ------------------------------------------------------------ async copies

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16),
// completing on the mbarrier, with an L2 eviction-priority hint
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// read-only gather that does not allocate in L1 (random gathers have no reuse there)
__device__ __forceinline__ float ld_gather(const float* p)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_gather(const double* p)
{
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for one phase of the mbarrier, giving up after `limit_ns` of device
// time; returns false on time-out.  Every lane of the warp calls it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// ------------------------------------------------------------ per-warp stages

// Shared memory of one warp: two stages of (values, column indices) of a short
// task, two mbarriers and the task's row pointers.  Stage sizes keep every stage
// 16-byte aligned and leave room for the rounding of the copied range.
template <typename T>
struct alignas(16) WarpStage {
    static constexpr int CAPW = cap_w<T>();
    static constexpr int VA = 16 / (int)sizeof(T);   // values per 16 bytes
    // a copied range is the task rounded out to 16 bytes at both ends
    static constexpr int VPAD = (CAPW + 2 * (VA - 1) + VA - 1) / VA * VA;
    static constexpr int IPAD = (CAPW + 6 + 3) / 4 * 4;
    T v[2][VPAD];
    int i[2][IPAD];
    uint64_t bar[2];
    int rps[kTaskRows + 1];   // row starts of a short task, relative to its first nonzero
};

static_assert(sizeof(WarpStage<float>) % 16 == 0 && sizeof(WarpStage<double>) % 16 == 0,
              "stages must stay 16-byte aligned");

// ------------------------------------------------ warp-specialised variant
// The warps of a block form producer / consumer pairs (warp 2p produces, warp
// 2p + 1 consumes) that work through one task list per pair.  The producer
// streams the chunks through a ring of kWsStages shared-memory stages (bulk
// copies, issued kWsStages - 1 chunks ahead), gathers the vector and writes the
// products back into the stage; the consumer sums the rows of a stage and runs
// the epilogue, then releases the stage.  Gathers thus stay in flight while rows
// are summed and epilogues run (the request stream of a plain gather loop),
// instead of pausing for them as in the one-warp form.  Long rows are summed as
// in the one-warp form; short tasks by seg_row_sums (the one-warp form's lane
// groups per row with PDHG_WS_SEGSUM=0).  Every order is fixed.
#ifndef PDHG_SPMV_WS
#define PDHG_SPMV_WS 1
#endif
constexpr bool kSpmvWs = PDHG_SPMV_WS != 0;
constexpr int kWsPairs = kTaskWarps / 2;
#ifndef PDHG_WS_STAGES
#define PDHG_WS_STAGES 3
#endif
constexpr int kWsStages = PDHG_WS_STAGES;
static_assert(kWsStages >= 3, "the consumer reads the descriptor one chunk ahead");
// Short tasks' row sums by the segmented form (seg_row_sums: equal shares per
// lane) instead of one group of lanes per row, for every task (otherwise only
// for the tasks the host marks with kSegBit).
#ifndef PDHG_WS_SEGSUM
#define PDHG_WS_SEGSUM 0
#endif
constexpr bool kWsSegSum = PDHG_WS_SEGSUM != 0;
// task lists (workers) per block of an SpMV launch
constexpr int kSpmvWorkers = kSpmvWs ? kWsPairs : kTaskWarps;

// Whether an epilogue's load() of one task may run before another task's rows
// are finished (no per-task state set by task_start).
template <class E, class = void>
struct StatelessTasks : std::false_type {};
template <class E>
struct StatelessTasks<E, std::void_t<decltype(E::kStatelessTasks)>>
    : std::integral_constant<bool, E::kStatelessTasks> {};

// A chunk of a stage: its task, nonzero range [cs, ce), flags (bit 0 the
// task's first chunk, bit 1 its last, bit 2 the task is one long row or a piece
// of one), the task's rows [r0, r0 + nrows) and, for a piece of a split row,
// its slot (else -1); task < 0 ends the pair's sequence.
struct WsDesc {
    int task, cs, ce, flags, r0, nrows, piece;
};
constexpr int kWsFirst = 1, kWsLast = 2, kWsLong = 4, kWsSeg = 8;

// Epilogues whose reductions take split rows: they provide
// split_acc(int s, const Acc&) and a member nsplit (the kernel sets it to
// SplitRows::n), and lay their partials out with a stride of gridDim.x + nsplit.
template <class E, class = void>
struct HasSplitAcc : std::false_type {};
template <class E>
struct HasSplitAcc<E, std::void_t<decltype(&E::split_acc)>> : std::true_type {};

// FP64: a short task's products are not formed by the producer; it stores the
// gathered entries beside the values and the consumer adds v x by fused
// multiply-adds (one FP64 instruction per nonzero instead of a multiply and an
// add: GB300's FP64 pipe bounds the FP64 SpMVs).
template <typename T> struct WsFmaSum { static constexpr bool value = sizeof(T) == 8; };

template <typename T, bool L1G>
struct alignas(16) PairStage {
    static constexpr int CAPW = cap_ws<T, L1G>();
    static constexpr int VA = 16 / (int)sizeof(T);
    static constexpr int VPAD = (CAPW + 2 * (VA - 1) + VA - 1) / VA * VA;
    static constexpr int IPAD = (CAPW + 6 + 3) / 4 * 4;
    T v[kWsStages][VPAD];          // values, then products (long row: lane sums)
    int i[kWsStages][IPAD];        // column indices
    uint64_t tma[kWsStages];       // bulk copy of the stage complete
    uint64_t full[kWsStages];      // products written (32 producer arrivals)
    uint64_t empty[kWsStages];     // stage read (32 consumer arrivals)
    WsDesc desc[kWsStages];
    int rps[kTaskRows + 1];        // row starts of the consumer's short task
    T rsum[kTaskRows];             // its row sums (segmented form)
    // the gathered vector entries of a short task's chunk (kWsFmaSum: the
    // consumer forms the products by fused multiply-adds into its row sums)
    T xg[WsFmaSum<T>::value ? kWsStages : 1][WsFmaSum<T>::value ? VPAD : 16 / sizeof(T)];
};
static_assert(sizeof(PairStage<float, false>) % 16 == 0 && sizeof(PairStage<double, false>) % 16 == 0 &&
                  sizeof(PairStage<float, true>) % 16 == 0 && sizeof(PairStage<double, true>) % 16 == 0,
              "stages must stay 16-byte aligned");

template <typename T, bool L1G = false>
constexpr size_t spmv_smem_bytes()
{
    return kSpmvWs ? sizeof(PairStage<T, L1G>) * kWsPairs : sizeof(WarpStage<T>) * kTaskWarps;
}

// Nonzeros per chunk (and the largest short task) of an SpMV whose gathered
// vector has x_len entries.
template <typename T>
inline int spmv_cap(int64_t x_len);

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Issues the bulk copies of a short task's values [s, e) and column indices
// into stage `st` (lane 0 only).  Each copy covers the 16-byte aligned range
// around [s, e); the arrays are padded so the rounded range stays inside them.
template <typename T>
__device__ __forceinline__ void stage_task(WarpStage<T>& W, int st, int64_t s, int64_t e,
                                           const T* val, const int32_t* ci, uint64_t pol)
{
    constexpr int VA = 16 / (int)sizeof(T);
    const int64_t v0 = s & ~(int64_t)(VA - 1), v1 = (e + VA - 1) & ~(int64_t)(VA - 1);
    const int64_t i0 = s & ~(int64_t)3, i1 = (e + 3) & ~(int64_t)3;
    const uint32_t vb = (uint32_t)((v1 - v0) * (int64_t)sizeof(T));
    const uint32_t ib = (uint32_t)((i1 - i0) * 4);
    fence_proxy_async_smem();
    mbar_expect_tx(&W.bar[st], vb + ib);
    bulk_g2s(W.v[st], val + v0, vb, &W.bar[st], pol);
    bulk_g2s(W.i[st], ci + i0, ib, &W.bar[st], pol);
}

// Each warp takes the tasks warp_id, warp_id + W, warp_id + 2W, ... (W = all warps
// of the launch): a fixed assignment, so every partial sum keeps a fixed order.
// A task is streamed through the warp's two shared-memory stages in chunks of at
// most CAPW nonzeros (one chunk for a short task; a long row is cut into
// consecutive chunks whose products accumulate per lane).  While the warp works
// on one chunk, the bulk copy of its next chunk is in flight into the other
// stage.  task_nz[t] = rp[task_row[t]].  A stage wait that exceeds 50 ms sets
// *err and abandons the launch's remaining work after a second bounded wait for
// the copy in flight.
template <typename T, class Epi, bool L1G>
__global__ void __launch_bounds__(kSpmvNT, MinBlocks<T>::value)
k_spmv(const int32_t* __restrict__ task_row, const int64_t* __restrict__ task_nz, int ntasks,
       const int32_t* __restrict__ wbeg, const int32_t* __restrict__ perm,
       const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ val,
       int* err, Epi epi)
{
    constexpr int CAPW = cap_w<T>();
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr unsigned long long kWaitNs = 50ull * 1000 * 1000;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // Programmatic dependent launch: a launch made with launch_spmv(..., pdl =
    // true) may start while the previous kernel of the stream finishes; it
    // waits here, before reading anything that kernel wrote.  Both
    // instructions are no-ops for ordinary launches.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    if (!epi.begin()) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStage<T>& W = reinterpret_cast<WarpStage<T>*>(smem_raw)[warp];
    typename Epi::Acc acc;
    const T* __restrict__ xv = epi.xin();   // re-read per task: a batch's LPs differ
    if (lane == 0) {
        mbar_init(&W.bar[0], 1);
        mbar_init(&W.bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const uint64_t pol = evict_first_policy();
    // the warp's tasks are perm[wbeg[w] .. wbeg[w + 1]) (assigned on the host by
    // their chunk counts); tasks the epilogue declares dead (a finished LP of a
    // batch) are passed over.  `ntasks` marks "no task".
    const int gw = blockIdx.x * kTaskWarps + warp;
    const int pend = wbeg[gw + 1];
    auto next_live = [&](int p) {
        while (p < pend && !epi.live(perm[p])) ++p;
        return p;
    };
    auto task_at = [&](int p) { return p < pend ? perm[p] : ntasks; };
    int npos = next_live(wbeg[gw]);   // position of the current task, then of the next
    int task = task_at(npos);
    int nt = ntasks;    // the next live task after `task`
    // current task [s, e), current chunk [cs, ce); next task bounds [ns, ne)
    // (32-bit: the library accepts fewer than 2^31 - 64 nonzeros)
    int s = 0, e = 0, ns = 0, ne = 0, cs = 0, ce = 0;
    if (task < ntasks) {
        s = (int)task_nz[task];
        e = (int)task_nz[task + 1];
        cs = s;
        ce = e - s > CAPW ? s + CAPW : e;
        if (lane == 0 && ce > cs) stage_task<T>(W, 0, cs, ce, val, ci, pol);
        npos = next_live(npos + 1);
        nt = task_at(npos);
        if (nt < ntasks) {
            ns = (int)task_nz[nt];
            ne = (int)task_nz[nt + 1];
        }
    }
    uint32_t par = 0;   // bit st: parity of the next wait on stage st
    int st = 0;
    int r0 = 0, nrows = 0;
    typename Epi::Pre pre0, pre1;
    T along = 0;        // per-lane sum of a long row over its chunks
#pragma unroll 1
    while (task < ntasks) {
        const bool first = cs == s;
        const bool last = ce == e;
        const bool is_long = e - s > CAPW;
        // the next chunk: the rest of this long row, or the first chunk of the next task
        int xs = 0, xe = 0;
        bool have_next = false;
        if (!last) {
            xs = ce;
            xe = e - ce > CAPW ? ce + CAPW : e;
            have_next = true;
        } else if (nt < ntasks) {
            xs = ns;
            xe = ne - ns > CAPW ? ns + CAPW : ne;
            have_next = true;
        }
        // an empty chunk (a task of empty rows) is neither copied nor waited for
        const bool next_staged = have_next && xe > xs;
        if (next_staged && lane == 0) stage_task<T>(W, st ^ 1, xs, xe, val, ci, pol);
        // row starts of a short task: loaded now (low 32 bits: fewer than 2^31
        // nonzeros), written to shared memory after the gathers are in flight, so
        // that their latency hides behind the stage wait and the gathers
        int rpl0 = 0, rpl1 = 0;
        if (first) {
            epi.task_start(task);
            xv = epi.xin();
            r0 = task_row[task];
            nrows = task_row[task + 1] - r0;
            if (lane < nrows) pre0 = epi.load(r0 + lane);
            if (kTaskRows > 32 && lane + 32 < nrows) pre1 = epi.load(r0 + 32 + lane);
            if (!is_long) {
                const int* rp32 = reinterpret_cast<const int*>(rp);
                if (lane < nrows) rpl0 = rp32[2 * ((int64_t)r0 + lane)];
                if (kTaskRows > 32 && lane + 32 < nrows) rpl1 = rp32[2 * ((int64_t)r0 + 32 + lane)];
            }
            along = 0;
        }
        if (ce > cs) {
            // every lane waits (acquiring the copied bytes); the outcome is made
            // warp-uniform before anyone acts on it
            const bool got = mbar_wait_bounded(&W.bar[st], (par >> st) & 1u, kWaitNs);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) atomicOr(err, 1);
                if (next_staged)
                    (void)mbar_wait_bounded(&W.bar[st ^ 1], (par >> (st ^ 1)) & 1u, kWaitNs);
                break;
            }
            par ^= 1u << st;
        }
        __syncwarp();
        // gathers for the chunk [cs, ce): lane l owns the 16-byte groups
        // l, l + 32, l + 64, ... of the staged values; it reads each group's values and
        // column indices with one vector load apiece, gathers x, and writes the
        // products back in place (or adds them to its long-row sum)
        const int v0 = cs & ~(VA - 1);
        const int d = v0 - (cs & ~3);   // index-buffer offset of v0
        const int vo = cs - v0;
        const int lim = vo + (ce - cs);
        T* vbuf = W.v[st];
        const int* ibuf = W.i[st] + d;
        using VT = VecTraits<T>;
        constexpr int VEC = VT::N;
        // groups per lane: a chunk spans at most VA - 1 + CAPW staged elements
        constexpr int UG = (VA - 1 + CAPW + 32 * VEC - 1) / (32 * VEC);
        T vv[UG][VEC];
        int ii[UG][VEC];
#pragma unroll
        for (int k = 0; k < UG; ++k) {
            const int off = (k * 32 + lane) * VEC;
            if (off < lim) {
                VT::unpack(*reinterpret_cast<const typename VT::V*>(vbuf + off), vv[k]);
                VT::unpacki(*reinterpret_cast<const typename VT::I*>(ibuf + off), ii[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < UG; ++k) {
            const int off = (k * 32 + lane) * VEC;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int p = off + v;
                if (p >= vo && p < lim) {
                    if constexpr (L1G) vv[k][v] *= __ldg(xv + ii[k][v]);
                    else vv[k][v] *= ld_gather(xv + ii[k][v]);
                } else {
                    vv[k][v] = T(0);
                }
            }
        }
        if (first && !is_long) {
            if (lane < nrows) W.rps[lane] = rpl0 - s;
            if (kTaskRows > 32 && lane + 32 < nrows) W.rps[lane + 32] = rpl1 - s;
            if (lane == 0) W.rps[nrows] = e - s;
        }
        if (is_long) {
#pragma unroll
            for (int k = 0; k < UG; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) along += vv[k][v];
            if (last) {
                const T a = warp_sum_T(along);
                if (lane == 0) epi.row(r0, a, pre0, acc);
            }
        } else {
#pragma unroll
            for (int k = 0; k < UG; ++k) {
                const int off = (k * 32 + lane) * VEC;
                if (off < lim) *reinterpret_cast<typename VT::V*>(vbuf + off) = VT::pack(vv[k]);
            }
            T* vs = vbuf + vo;
            __syncwarp();
            const int* rps = W.rps;
            if (nrows <= 32) {
                int G = 32;
                while (G > 1 && G * nrows > 32) G >>= 1;
                const int j = lane / G, g = lane % G;
                T a = 0;
                if (j < nrows) {
                    const int pb = rps[j], pe = rps[j + 1];
                    a = strided_sum(vs, pb + g, pe, G);
                }
                for (int o = G >> 1; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o, G);
                const T v = __shfl_sync(0xffffffffu, a, (lane * G) & 31);
                if (lane < nrows) epi.row(r0 + lane, v, pre0, acc);
            } else if (kTaskRows > 32) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int j = lane + 32 * half;
                    if (j < nrows) {
                        const int pb = rps[j], pe = rps[j + 1];
                        epi.row(r0 + j, strided_sum(vs, pb, pe, 1), half ? pre1 : pre0, acc);
                    }
                }
            }
        }
        __syncwarp();   // the stage is rewritten by the copy issued in two chunks' time
        st ^= 1;
        if (!last) {
            cs = xs;
            ce = xe;
        } else {
            epi.task_done(task, acc);
            task = nt;
            s = ns;
            e = ne;
            cs = xs;
            ce = xe;
            if (task < ntasks) {
                npos = next_live(npos + 1);
                nt = task_at(npos);
                if (nt < ntasks) {
                    ns = (int)task_nz[nt];
                    ne = (int)task_nz[nt + 1];
                }
            }
        }
    }
    epi.finish(acc);
}

// Bulk copy of the values [s, e) and column indices of one chunk into a stage
// (one lane); as stage_task, for the warp-specialised stages.
template <typename T>
__device__ __forceinline__ void stage_chunk(T* vdst, int* idst, uint64_t* bar, int64_t s,
                                            int64_t e, const T* val, const int32_t* ci,
                                            uint64_t pol)
{
    constexpr int VA = 16 / (int)sizeof(T);
    const int64_t v0 = s & ~(int64_t)(VA - 1), v1 = (e + VA - 1) & ~(int64_t)(VA - 1);
    const int64_t i0 = s & ~(int64_t)3, i1 = (e + 3) & ~(int64_t)3;
    const uint32_t vb = (uint32_t)((v1 - v0) * (int64_t)sizeof(T));
    const uint32_t ib = (uint32_t)((i1 - i0) * 4);
    fence_proxy_async_smem();
    mbar_expect_tx(bar, vb + ib);
    bulk_g2s(vdst, val + v0, vb, bar, pol);
    bulk_g2s(idst, ci + i0, ib, bar, pol);
}

// The warp-specialised SpMV (see PairStage).  Same arguments, task lists (one per
// pair: wbeg has gridDim.x * kWsPairs + 1 entries), epilogue interface, bounded
// waits and summation order as k_spmv.
template <typename T, class Epi, bool L1G>
__global__ void __launch_bounds__(kSpmvNT, MinBlocks<T>::value)
k_spmv_ws(const int32_t* __restrict__ task_row, const int64_t* __restrict__ task_nz, int ntasks,
          const int32_t* __restrict__ wbeg, const int32_t* __restrict__ perm,
          const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
          const T* __restrict__ val, int* err, SplitRows sp, Epi epi)
{
    constexpr int CAPW = cap_ws<T, L1G>();
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr int NS = kWsStages;
    constexpr unsigned long long kWaitNs = 50ull * 1000 * 1000;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    if constexpr (HasSplitAcc<Epi>::value) epi.nsplit = sp.n;
    if (!epi.begin()) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = warp >> 1;
    const bool producer = (warp & 1) == 0;
    PairStage<T, L1G>& P = reinterpret_cast<PairStage<T, L1G>*>(smem_raw)[pair];
    if (producer && lane == 0) {
        for (int q = 0; q < NS; ++q) {
            mbar_init(&P.tma[q], 1);
            mbar_init(&P.full[q], 32);
            mbar_init(&P.empty[q], 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    typename Epi::Acc acc;
    const int gw = blockIdx.x * kWsPairs + pair;
    const int pbeg = wbeg[gw], pend = sp.wend ? sp.wend[gw] : wbeg[gw + 1];
    if (producer) {
        // ---------------------------------------------------------- producer
        const uint64_t pol = evict_first_policy();
        auto next_live = [&](int p) {
            while (p < pend && !epi.live(perm[p])) ++p;
            return p;
        };
        // the issue cursor: task itask at position ipos, its nonzeros [is, ie) and
        // rows [ir0, ir0 + inr), next chunk at ics; the task after it (ntask at
        // npos) is read one task ahead, so that moving on never waits for the
        // task list and the task's bounds together
        auto task_at = [&](int p) { return p < pend ? perm[p] : ntasks; };
        int ipos = next_live(pbeg);
        int itask = task_at(ipos);
        int is = 0, ie = 0, ics = 0, ir0 = 0, inr = 0, ipc = -1, iseg = 0;
        // bounds, rows, piece slot and row-sum form of task itask (a piece has
        // no rows of its own)
        auto load_task = [&]() {
            const int64_t tz = task_nz[itask];
            is = (int)(uint32_t)tz;
            ipc = (int)((tz >> 32) & kPieceMask) - 1;
            iseg = (tz & kSegBit) ? kWsSeg : 0;
            ie = (int)(uint32_t)task_nz[itask + 1];
            ir0 = task_row[itask];
            inr = ipc < 0 ? task_row[itask + 1] - ir0 : 0;
            ics = is;
        };
        if (itask < ntasks) load_task();
        int npos = itask < ntasks ? next_live(ipos + 1) : pend;
        int ntask = task_at(npos);
        bool ended = false;       // the terminator has been issued
        bool failed = false;
        uint32_t tpar = 0;        // bit q: parity of the next wait on tma[q]
        uint32_t inflight = 0;    // bit q: a copy into stage q not yet waited for
        // issue(q): after the consumer released stage q % NS from its previous
        // chunk, describe chunk q there and start its copy
        auto issue = [&](int q) {
            if (ended || failed) return;
            const int st = q % NS, n = q / NS;
            if (n >= 1) {
                const bool got = mbar_wait_bounded(&P.empty[st], (uint32_t)((n - 1) & 1), kWaitNs);
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) atomicOr(err, 1);
                    failed = true;
                    return;
                }
            }
            WsDesc d{-1, 0, 0, 0, 0, 0, -1};
            if (itask < ntasks) {
                const int cs = ics, ce = ie - ics > CAPW ? ics + CAPW : ie;
                d.task = itask;
                d.cs = cs;
                d.ce = ce;
                d.flags = (cs == is ? kWsFirst : 0) | (ce == ie ? kWsLast : 0) |
                          (ie - is > CAPW || ipc >= 0 ? kWsLong : 0) | iseg;
                d.r0 = ir0;
                d.nrows = inr;
                d.piece = ipc;
                if (ce != ie) {
                    ics = ce;
                } else {
                    ipos = npos;
                    itask = ntask;
                    if (itask < ntasks) {
                        load_task();
                        npos = next_live(ipos + 1);
                        ntask = task_at(npos);
                    }
                }
                if (ce > cs) {
                    if (lane == 0) stage_chunk<T>(P.v[st], P.i[st], &P.tma[st], cs, ce, val, ci, pol);
                    inflight |= 1u << st;
                }
            } else {
                ended = true;
            }
            if (lane == 0) P.desc[st] = d;
            __syncwarp();
        };
        for (int q = 0; q < NS - 1; ++q) issue(q);
        const T* __restrict__ xv = epi.xin();
        T along = 0;
        using VT = VecTraits<T>;
        constexpr int VEC = VT::N;
        constexpr int UG = (VA - 1 + CAPW + 32 * VEC - 1) / (32 * VEC);
#pragma unroll 1
        for (int q = 0; !failed; ++q) {
            const int st = q % NS;
            const WsDesc d = P.desc[st];
            if (d.task < 0) {
                mbar_arrive(&P.full[st]);   // the consumer sees the end
                break;
            }
            if (d.flags & kWsFirst) {
                epi.task_start(d.task);
                xv = epi.xin();
                along = 0;
            }
            const int cs = d.cs, ce = d.ce;
            if (ce > cs) {
                const bool got = mbar_wait_bounded(&P.tma[st], (tpar >> st) & 1u, kWaitNs);
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) atomicOr(err, 1);
                    failed = true;
                    break;
                }
                tpar ^= 1u << st;
                inflight &= ~(1u << st);
                const int v0 = cs & ~(VA - 1);
                const int dd = v0 - (cs & ~3);
                const int vo = cs - v0;
                const int lim = vo + (ce - cs);
                T* vbuf = P.v[st];
                const int* ibuf = P.i[st] + dd;
                T vv[UG][VEC];
                int ii[UG][VEC];
#pragma unroll
                for (int k = 0; k < UG; ++k) {
                    const int off = (k * 32 + lane) * VEC;
                    if (off < lim) {
                        VT::unpack(*reinterpret_cast<const typename VT::V*>(vbuf + off), vv[k]);
                        VT::unpacki(*reinterpret_cast<const typename VT::I*>(ibuf + off), ii[k]);
                    }
                }
                if (d.flags & kWsLong) {
                    // a long row's lane sums take the products by fused multiply-adds
                    // (one FP64 instruction per nonzero instead of two)
#pragma unroll
                    for (int k = 0; k < UG; ++k) {
                        const int off = (k * 32 + lane) * VEC;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const int p = off + v;
                            if (p >= vo && p < lim) {
                                T g;
                                if constexpr (L1G) g = __ldg(xv + ii[k][v]);
                                else g = ld_gather(xv + ii[k][v]);
                                along = fma(vv[k][v], g, along);
                            }
                        }
                    }
                    if (d.flags & kWsLast) {
                        __syncwarp();   // every lane has read its values
                        vbuf[lane] = along;
                    }
                } else if constexpr (WsFmaSum<T>::value) {
                    // the gathered entries go beside the values (see WsFmaSum)
                    T* xbuf = P.xg[st];
#pragma unroll
                    for (int k = 0; k < UG; ++k) {
                        const int off = (k * 32 + lane) * VEC;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const int p = off + v;
                            if (p >= vo && p < lim) {
                                if constexpr (L1G) vv[k][v] = __ldg(xv + ii[k][v]);
                                else vv[k][v] = ld_gather(xv + ii[k][v]);
                            } else {
                                vv[k][v] = T(0);
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < UG; ++k) {
                        const int off = (k * 32 + lane) * VEC;
                        if (off < lim)
                            *reinterpret_cast<typename VT::V*>(xbuf + off) = VT::pack(vv[k]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < UG; ++k) {
                        const int off = (k * 32 + lane) * VEC;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const int p = off + v;
                            if (p >= vo && p < lim) {
                                if constexpr (L1G) vv[k][v] *= __ldg(xv + ii[k][v]);
                                else vv[k][v] *= ld_gather(xv + ii[k][v]);
                            } else {
                                vv[k][v] = T(0);
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < UG; ++k) {
                        const int off = (k * 32 + lane) * VEC;
                        if (off < lim)
                            *reinterpret_cast<typename VT::V*>(vbuf + off) = VT::pack(vv[k]);
                    }
                }
            }
            mbar_arrive(&P.full[st]);   // each lane releases its own writes
            issue(q + NS - 1);
        }
        if (failed) {
            // copies still in flight must land before the block's shared memory goes
            for (int q = 0; q < NS; ++q)
                if ((inflight >> q) & 1u)
                    (void)mbar_wait_bounded(&P.tma[q], (tpar >> q) & 1u, kWaitNs);
        }
    } else {
        // ---------------------------------------------------------- consumer
        typename Epi::Pre pre0, pre1;
        int r0 = 0, nrows = 0;
        // With stateless tasks the consumer loads the row operands and row starts
        // of the next task while it finishes the current one: the producer
        // describes chunk q + 1 before it releases chunk q, so once chunk q is
        // acquired its successor's descriptor (rows included) can be read.
        // (FP32 only: the FP64 operands of a second task spill registers.)
#ifndef PDHG_WS_PREFETCH_F64
#define PDHG_WS_PREFETCH_F64 0
#endif
        constexpr bool PF = StatelessTasks<Epi>::value && (sizeof(T) == 4 || PDHG_WS_PREFETCH_F64);
        typename Epi::Pre npre0, npre1;
        int nrpl0 = 0, nrpl1 = 0;
        bool have_next = false;   // npre / nrpl hold the next task's operands
        auto prefetch = [&](const WsDesc& dn) {
            const int nr0 = dn.r0, nn = dn.nrows;
            if (lane < nn) npre0 = epi.load(nr0 + lane);
            if (kTaskRows > 32 && lane + 32 < nn) npre1 = epi.load(nr0 + 32 + lane);
            if (!(dn.flags & kWsLong)) {
                const int* rp32 = reinterpret_cast<const int*>(rp);
                if (lane < nn) nrpl0 = rp32[2 * ((int64_t)nr0 + lane)];
                if (kTaskRows > 32 && lane + 32 < nn) nrpl1 = rp32[2 * ((int64_t)nr0 + 32 + lane)];
            }
        };
#pragma unroll 1
        for (int q = 0;; ++q) {
            const int st = q % NS, n = q / NS;
            const bool got = mbar_wait_bounded(&P.full[st], (uint32_t)(n & 1), kWaitNs);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) atomicOr(err, 1);
                break;
            }
            const WsDesc d = P.desc[st];
            if (d.task < 0) break;
            const bool lng = d.flags & kWsLong;
            if (d.flags & kWsFirst) {
                epi.task_start(d.task);
                r0 = d.r0;
                nrows = d.nrows;
                int rpl0 = 0, rpl1 = 0;
                if (PF && have_next) {
                    pre0 = npre0;
                    pre1 = npre1;
                    rpl0 = nrpl0;
                    rpl1 = nrpl1;
                } else {
                    const int* rp32 = reinterpret_cast<const int*>(rp);
                    if (lane < nrows) pre0 = epi.load(r0 + lane);
                    if (kTaskRows > 32 && lane + 32 < nrows) pre1 = epi.load(r0 + 32 + lane);
                    if (!lng) {
                        if (lane < nrows) rpl0 = rp32[2 * ((int64_t)r0 + lane)];
                        if (kTaskRows > 32 && lane + 32 < nrows)
                            rpl1 = rp32[2 * ((int64_t)r0 + 32 + lane)];
                    }
                }
                if (!lng) {
                    // row starts relative to the task's first nonzero (a short task
                    // is one chunk: [d.cs, d.ce))
                    if (lane < nrows) P.rps[lane] = rpl0 - d.cs;
                    if (kTaskRows > 32 && lane + 32 < nrows) P.rps[lane + 32] = rpl1 - d.cs;
                    if (lane == 0) P.rps[nrows] = d.ce - d.cs;
                }
            }
            if constexpr (PF) {
                have_next = false;
                const WsDesc dn = P.desc[(q + 1) % NS];
                if (dn.task >= 0 && (dn.flags & kWsFirst)) {
                    prefetch(dn);
                    have_next = true;
                }
            }
            __syncwarp();
            if (lng) {
                if (d.flags & kWsLast) {
                    const T a = warp_sum_T(P.v[st][lane]);
                    if (lane == 0) {
                        if (d.piece < 0) {
                            epi.row(r0, a, pre0, acc);
                        } else if (sp.slots == nullptr) {
                            atomicOr(err, 2);   // a schedule with pieces launched without them
                        } else {
                            // a piece of a split row (see SplitRows)
                            T* slots = static_cast<T*>(sp.slots);
                            slots[d.piece] = a;
                            __threadfence();
                            const int sr = sp.pspl[d.piece];
                            const int g0 = sp.info[2 * sr], np = sp.info[2 * sr + 1];
                            if (atomicAdd(&sp.cnt[sr], 1) == np - 1) {
                                __threadfence();
                                T v = T(0);
                                for (int p = 0; p < np; ++p) v += __ldcg(slots + g0 + p);
                                sp.cnt[sr] = 0;
                                const typename Epi::Pre pr = epi.load(r0);
                                typename Epi::Acc sa{};
                                epi.row(r0, v, pr, sa);
                                if constexpr (HasSplitAcc<Epi>::value)
                                    epi.split_acc(sr, sa);
                                else if constexpr (!std::is_empty<typename Epi::Acc>::value)
                                    atomicOr(err, 2);   // reductions without a split slot
                            }
                        }
                    }
                }
            } else {
                const int v0 = d.cs & ~(VA - 1);
                const T* vs = P.v[st] + (d.cs - v0);
                // FP64: the gathered entries, multiplied in here (WsFmaSum)
                const T* xs = WsFmaSum<T>::value ? P.xg[st] + (d.cs - v0) : nullptr;
                const int* rps = P.rps;
                if (kWsSegSum || (d.flags & kWsSeg)) {
                    seg_row_sums<T>(vs, rps, nrows, d.ce - d.cs, lane, P.rsum, xs);
                    if (lane < nrows) epi.row(r0 + lane, P.rsum[lane], pre0, acc);
                    if (kTaskRows > 32 && lane + 32 < nrows)
                        epi.row(r0 + 32 + lane, P.rsum[lane + 32], pre1, acc);
                } else if (nrows <= 32) {
                    int G = 32;
                    while (G > 1 && G * nrows > 32) G >>= 1;
                    const int j = lane / G, g = lane % G;
                    T a = 0;
                    if (j < nrows) {
                        const int pb = rps[j], pe = rps[j + 1];
                        if constexpr (WsFmaSum<T>::value) a = strided_dot(vs, xs, pb + g, pe, G);
                        else a = strided_sum(vs, pb + g, pe, G);
                    }
                    for (int o = G >> 1; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o, G);
                    const T v = __shfl_sync(0xffffffffu, a, (lane * G) & 31);
                    if (lane < nrows) epi.row(r0 + lane, v, pre0, acc);
                } else if (kTaskRows > 32) {
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int j = lane + 32 * half;
                        if (j < nrows) {
                            const int pb = rps[j], pe = rps[j + 1];
                            T v;
                            if constexpr (WsFmaSum<T>::value) v = strided_dot(vs, xs, pb, pe, 1);
                            else v = strided_sum(vs, pb, pe, 1);
                            epi.row(r0 + j, v, half ? pre1 : pre0, acc);
                        }
                    }
                }
            }
            if (d.flags & kWsLast) epi.task_done(d.task, acc);
            __syncwarp();
            mbar_arrive(&P.empty[st]);
        }
    }
    epi.finish(acc);
}

// Dynamic shared-memory limit (and the optional carveout preference) of one
// SpMV instantiation; spmv_prepare sets both gather variants of an epilogue.
// Call before any launch or graph capture of that epilogue.
template <typename T, bool L1G = false>
inline cudaError_t spmv_set_attrs(const void* f)
{
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)spmv_smem_bytes<T, L1G>());
    if (e != cudaSuccess || kSpmvCarveout < 0) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, kSpmvCarveout);
}

template <typename T, class Epi>
inline cudaError_t spmv_prepare()
{
    if constexpr (kSpmvWs) {
        cudaError_t e = spmv_set_attrs<T, true>((const void*)k_spmv_ws<T, Epi, true>);
        if (e != cudaSuccess) return e;
        return spmv_set_attrs<T, false>((const void*)k_spmv_ws<T, Epi, false>);
    } else {
        cudaError_t e = spmv_set_attrs<T>((const void*)k_spmv<T, Epi, true>);
        if (e != cudaSuccess) return e;
        return spmv_set_attrs<T>((const void*)k_spmv<T, Epi, false>);
    }
}

// Gathers from a vector of at most this many bytes go through L1 (it stays
// resident there); larger vectors are gathered without L1 allocation.
constexpr int64_t kL1GatherBytes = 96 * 1024;

template <typename T>
inline int spmv_cap(int64_t x_len)
{
    if (!kSpmvWs) return cap_w<T>();
    return x_len * (int64_t)sizeof(T) <= kL1GatherBytes ? cap_ws<T, true>() : cap_ws<T, false>();
}

// pdl: launch with programmatic stream serialisation (the kernel may start
// before the previous kernel of the stream has finished; it waits for it at its
// top), so that its launch and block start-up overlap the previous kernel's tail.
#ifndef PDHG_PDL
#define PDHG_PDL 0
#endif
// sp: the split rows of the schedule (none by default; a schedule with pieces
// must be launched with its SplitRows).
template <typename T, class Epi>
inline void launch_spmv(int grid, cudaStream_t st, const int32_t* task_row,
                        const int64_t* task_nz, int ntasks, const int32_t* wbeg,
                        const int32_t* perm, const int64_t* rp, const int32_t* ci, const T* val,
                        int* err, int64_t x_len, const Epi& epi, bool pdl = false,
                        const SplitRows& sp = SplitRows{})
{
    const bool l1 = x_len * (int64_t)sizeof(T) <= kL1GatherBytes;
    const size_t sm = !kSpmvWs ? spmv_smem_bytes<T>()
                      : l1     ? spmv_smem_bytes<T, true>()
                               : spmv_smem_bytes<T, false>();
    if constexpr (kSpmvWs) {
        if (pdl && PDHG_PDL) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3(kSpmvNT);
            cfg.dynamicSmemBytes = sm;
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            auto kern = l1 ? k_spmv_ws<T, Epi, true> : k_spmv_ws<T, Epi, false>;
            (void)cudaLaunchKernelEx(&cfg, kern, task_row, task_nz, ntasks, wbeg, perm, rp, ci,
                                     val, err, sp, epi);
            return;
        }
        if (l1)
            k_spmv_ws<T, Epi, true><<<grid, kSpmvNT, sm, st>>>(task_row, task_nz, ntasks, wbeg,
                                                               perm, rp, ci, val, err, sp, epi);
        else
            k_spmv_ws<T, Epi, false><<<grid, kSpmvNT, sm, st>>>(task_row, task_nz, ntasks, wbeg,
                                                                perm, rp, ci, val, err, sp, epi);
        return;
    }
    if (pdl && PDHG_PDL) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(kSpmvNT);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        auto kern = l1 ? k_spmv<T, Epi, true> : k_spmv<T, Epi, false>;
        (void)cudaLaunchKernelEx(&cfg, kern, task_row, task_nz, ntasks, wbeg, perm, rp, ci, val,
                                 err, epi);
        return;
    }
    if (l1)
        k_spmv<T, Epi, true><<<grid, kSpmvNT, sm, st>>>(task_row, task_nz, ntasks, wbeg, perm, rp,
                                                        ci, val, err, epi);
    else
        k_spmv<T, Epi, false><<<grid, kSpmvNT, sm, st>>>(task_row, task_nz, ntasks, wbeg, perm,
                                                         rp, ci, val, err, epi);
}

// The task hooks of an epilogue that serves a single LP: every task is live,
// no per-task state (so the operands of a task's rows can be loaded while an
// earlier task is still being finished).
#define PDHG_SINGLE_LP_TASK_HOOKS                                   \
    static constexpr bool kStatelessTasks = true;                   \
    __device__ bool live(int) const { return true; }               \
    __device__ void task_start(int) {}                              \
    template <class A>                                              \
    __device__ void task_done(int, A&) const {}

// Plain epilogue: out[r] = scale * v, with the optional FP64 partial
// sum of out[r]^2 (power iteration) and a gate read from a Ctrl field.
template <typename T>
struct EpiStore {
    PDHG_SINGLE_LP_TASK_HOOKS
    const T* x;
    T* out;
    const double* scale;     // nullptr = 1
    double* part;            // nullptr = no partials
    const int* gate;         // nullptr = always run; else run when *gate != 0
    int nsplit = 0;          // split rows of the schedule (set by the kernel)
    struct Pre {};
    struct Acc { double s2 = 0.0; };
    __device__ bool begin() const { return gate == nullptr || *gate != 0; }
    __device__ const T* xin() const { return x; }
    __device__ Pre load(int) const { return Pre{}; }
    __device__ void row(int r, T v, const Pre&, Acc& a) const {
        if (scale) v = (T)((double)v * *scale);
        out[r] = v;
        if (part) a.s2 += (double)v * (double)v;
    }
    // partials: part[0, gridDim.x + nsplit)
    __device__ void split_acc(int s, const Acc& a) const {
        if (part) part[gridDim.x + s] = a.s2;
    }
    __device__ void finish(Acc& a) const {
        if (part) {
            const double t[1] = {a.s2};
            block_partials<1, kSpmvNT>(t, part, gridDim.x);
        }
    }
};

// Blocks of an SpMV launch: one resident wave (SMs x resident blocks per SM),
// fewer when there are fewer tasks than warps.
#ifndef PDHG_SPMV_WAVES
#define PDHG_SPMV_WAVES 1
#endif
template <typename T>
inline int spmv_grid(int ntasks, int num_sms)
{
    const int full = (ntasks + kSpmvWorkers - 1) / kSpmvWorkers;
    if (PDHG_SPMV_WAVES <= 0) return full > 0 ? full : 1;
    const int wave = num_sms * MinBlocks<T>::value * PDHG_SPMV_WAVES;
    return full < wave ? (full > 0 ? full : 1) : wave;
}

// Greedy task partition (host): rows are added to the current task while it
// holds <= cap nonzeros and <= max_rows rows; a row longer than cap gets a task
// of its own.  Returns the task boundaries (ntasks + 1 entries).
std::vector<int32_t> make_row_blocks(const int64_t* rp, int64_t rows, int cap, int max_rows);

// Assigns tasks to the `warps` warps of a launch (host): a task costs its number
// of chunks of at most `cap` nonzeros (task_nz: ntasks + 1 nonzero bounds);
// longest first, each to the least-loaded warp (ties: lower warp), so one warp
// does not collect several long rows.  wbeg[warps + 1] indexes perm, which lists
// each warp's tasks in ascending order.
void assign_tasks(const std::vector<int64_t>& task_nz, int cap, int warps,
                  std::vector<int32_t>& wbeg, std::vector<int32_t>& perm);

// Split rows of a schedule (host side of SplitRows).  task_piece[t]: the piece
// slot of task t, or -1; pspl[g]: the split row of piece slot g; info[2 s],
// info[2 s + 1]: first piece slot and number of pieces of split row s.
struct SplitPlan {
    std::vector<int32_t> task_piece, pspl, info;
    int n = 0, npieces = 0;
};

// Cuts the one-row tasks of a schedule (rows: task row bounds, nz: task
// nonzero bounds, both ntasks + 1 entries) into pieces when the longest-first
// assignment to `workers` lists would leave the longest list more than 15 %
// above the mean (in chunks of `cap` nonzeros): each one-row task of at least
// two pieces' worth of chunks becomes pieces of about an eighth of a list (at
// least two chunks), whole chunks from the row's start.  rows / nz are
// rewritten in place (a piece repeats its row; the entry after the last piece
// is the next row); returns the plan (n = 0: nothing cut, rows / nz untouched).
// Only the warp-specialised SpMV takes pieces: without it nothing is cut.
SplitPlan split_long_rows(std::vector<int32_t>& rows, std::vector<int64_t>& nz, int cap,
                          int workers);

// Steps of the busiest lane when a short task's rows [r0, r0 + nr) are summed
// by one group of lanes per row: a row of length L summed by G lanes takes
// ceil(L / G) steps (G the largest power of two with G nr <= 32); above 32 rows
// a lane sums two rows.  rp: host row pointers.
int64_t lane_group_steps(const int64_t* rp, int r0, int nr);

// The short tasks of a schedule (rows, nz: task bounds; tasks of at most cap
// nonzeros with rows of their own) whose busiest lane would take more than
// max_steps steps: their rows are summed by equal lane shares instead
// (seg_row_sums).  Returns one flag per task.
std::vector<char> seg_tasks(const int64_t* rp, const std::vector<int32_t>& rows,
                            const std::vector<int64_t>& nz, int cap, int max_steps);

// Schedule autotuner (tune.cu).  Candidates: cap in {CAPW, CAPW / 2} nonzeros
// and max_rows in {kTaskRows, 32, 16} rows per task.  build(cap, max_rows)
// returns the task boundaries over all rows of one orientation (h_rp: its host
// row pointers).  Each candidate's SpMV (store epilogue, x -> out) is launched
// once to warm up and timed over three launches with CUDA events on `st`; the
// fastest is returned in *best (and its mean milliseconds in *best_ms).
using RowBlockBuilder = std::function<std::vector<int32_t>(int cap, int max_rows)>;
template <typename T>
lp_status tune_schedule(int sms, cudaStream_t st, const RowBlockBuilder& build,
                        const int64_t* h_rp, const int64_t* rp, const int32_t* ci, const T* val,
                        const T* x, T* out, int64_t x_len, int* err, SchedParams* best,
                        float* best_ms);

}  // namespace pdhg
