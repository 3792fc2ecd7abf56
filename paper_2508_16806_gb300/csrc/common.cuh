// Shared declarations of the CUDA solver: device control block, handle layout,
// error plumbing and small device reductions.  Everything here is the solver's
// own; nothing is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>

#include "../../include/lp.h"

namespace pdhg {

// ----------------------------------------------------------------- constants

constexpr int kNT = 256;          // threads of an SpMV row-block
constexpr int kEW = 256;          // threads of an elementwise block
constexpr int kEWGrid = 1216;     // elementwise grid cap: 152 SMs x 8 resident blocks
constexpr int kCtlNT = 512;       // threads of a control (single-block) kernel
// KKT-check reductions: row side 11 sums + 2 maxima, column side 15 sums + 1 maximum
constexpr int kRowSums = 11, kRowMax = 2, kRowQ = kRowSums + kRowMax;
constexpr int kColSums = 15, kColMax = 1, kColQ = kColSums + kColMax;
constexpr int kAttemptFields = 9;   // doubles per record of the attempt log

// status codes shared with the ABI
constexpr int kRunning = -100;

// --------------------------------------------------------------- control block
// One per handle and precision, in device memory.  Written only by
// single-thread sections of control kernels, read by all kernels of a step.
// Step scalars of one control block in one precision: tau = eta / omega,
// sigma = eta * omega, the pending averaging weight, 1 / W and the Halpern
// weights lam (1 + rho), lam rho, 1 - lam with lam = (k + 1) / (k + 2).
template <typename T>
struct StepScalars {
    T tau, sigma, pw, winv, ha, hb, hg;
};

struct Ctrl {
    // step state
    double eta, omega;
    double pend_w;       // eta of the last accepted iterate not yet added to the averages
    double W;            // sum of eta over the iterates in the averages
    double Winv;         // 1 / W (0 while W = 0)
    // restart state (Section 2.4.2)
    double kkt_anchor, kkt_prev;
    // last check
    double kkt_cur, kkt_avg, kkt_cand, rel_gap, rel_pres, rel_dres, pobj, dobj;
    // options
    double tol, beta_s, beta_n, beta_a, eps_zero;
    double qnorm, cnorm;         // ||q||_2, ||c||_2 of the unscaled problem
    double time_limit_ns;
    double infeas_tol;   // Algorithm 6 tolerance (normalised directions)
    // restarted Halpern variant: reflection rho, the fixed-point residual
    // ||z - T(z)||_P of the last iteration, of the first iteration of the epoch,
    // and of the last iteration before the previous check of the epoch
    double reflect, fpr, fpr0, fpr_prev;
    // counters
    long long k, attempts, epoch_k, restarts, max_iters, t0_ns, trace_len, trace_cap;
    int cur;             // which half of each double buffer holds the current iterate
    int skip;            // step kernels return at once (check pending or done)
    int want_check;      // the check kernels run
    int done;            // loop finished; status holds the outcome
    int status;
    int first;           // the next check is the start-point check
    int cand_avg;        // candidate of the last check is the average
    int restart;         // the last check restarted
    int adaptive, pwu, restarts_on, check_every;
    int infeas;          // Algorithm 6 at every check
    int halpern;         // restarted Halpern iterations instead of averaged PDHG restarts
    int rejects;         // consecutive rejected attempts (a guard against a stuck loop)
    // what the K^T launch of a fused PDHG attempt does after the decision taken
    // at the end of the K launch: 0 nothing, 1 K^T y' and the next x' (accepted),
    // 2 K^T y' only (accepted, a check or the end follows), 3 the next x' from the
    // kept K^T y (rejected: no product)
    int t_mode;
    int npx;             // number of ||x' - x||^2 partials at px (the K^T launch grid)
    const double* px;    // those partials (written by k_primal or the K^T launch)
    // optional log of every step attempt (kAttemptFields doubles per record;
    // nullptr: off): accepted iterations before it, eta tried, eta_bar, eta',
    // accepted, omega, ||dx||^2, ||dy||^2, dy^T K dx (scaled problem)
    double* alog;
    long long alog_cap, alog_len;
    // the Algorithm 5 factors 1 - (k + 2)^-0.3 and 1 + (k + 2)^-0.6 for
    // k = ftab_k0 .. ftab_k0 + ftab_len - 1 (ftab[i], ftab[ftab_len + i]), filled by
    // each check for the period that follows (nullptr: computed in place)
    const double* ftab;
    long long ftab_k0;
    int ftab_len;
    unsigned int tick;   // finished blocks of the launch that takes the step decision (its last block does)
    long long bodies;    // loop-body executions (for the launch count)
    long long t_done_ns; // device clock when the loop finished for this LP
    // the step scalars, formed in FP64 once per change of eta, omega, pend_w, W or
    // epoch_k (refresh_scalars) and read by every thread of the step and check
    // kernels: GB300's FP64 pipe is narrow, and an FP64 division in every thread
    // (or for every element of a batch) costs microseconds per launch
    StepScalars<float> s32;
    StepScalars<double> s64;
};

__host__ __device__ inline void refresh_scalars(Ctrl& c)
{
    const double tau = c.eta / c.omega, sigma = c.eta * c.omega;
    const double lam = (double)(c.epoch_k + 1) / (double)(c.epoch_k + 2);
    const double ha = lam * (1.0 + c.reflect), hb = lam * c.reflect, hg = 1.0 - lam;
    c.s64 = StepScalars<double>{tau, sigma, c.pend_w, c.Winv, ha, hb, hg};
    c.s32 = StepScalars<float>{(float)tau, (float)sigma, (float)c.pend_w, (float)c.Winv,
                               (float)ha, (float)hb, (float)hg};
}

template <typename T>
__device__ __forceinline__ const StepScalars<T>& step_scalars(const Ctrl& c);
template <>
__device__ __forceinline__ const StepScalars<float>& step_scalars<float>(const Ctrl& c)
{
    return c.s32;
}
template <>
__device__ __forceinline__ const StepScalars<double>& step_scalars<double>(const Ctrl& c)
{
    return c.s64;
}

// ------------------------------------------------------------- device buffers

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Warp-task schedule parameters: nonzeros (cap) and rows (max_rows) per task.
struct SchedParams {
    int cap = 0;
    int max_rows = 0;
};

// Rows cut into pieces across task lists (warp-specialised form only).  A row
// of a schedule whose lists would otherwise be unbalanced (few, long rows, as
// the columns of K in a dispatch-shaped LP) is cut on the host into pieces of
// whole chunks; each piece is a task of its own, marked by its slot g + 1 in
// bits 32-61 of its task_nz entry (nonzero offsets fit in the low 31; bit 62
// marks a short task whose rows are summed by equal lane shares, kSegBit).
// The warp that finishes a piece stores its sum in slots[g] and takes a ticket
// on the row's counter; the warp that takes the last ticket adds the row's
// slots in piece order, so the result does not depend on which warp that is,
// resets the counter for the next launch and applies the epilogue to the row.
// The epilogue's reductions of that row go to a fixed place too: Epi::split_acc
// stores them in the split's own partial slot (after the block partials),
// which the consumer of the partials sums with them in a fixed order.
constexpr int64_t kSegBit = (int64_t)1 << 62;
constexpr int64_t kPieceMask = ((int64_t)1 << 30) - 1;   // of task_nz >> 32

struct SplitRows {
    const int32_t* pspl = nullptr;   // [npieces] split of each piece slot
    const int32_t* info = nullptr;   // [n][2] first piece slot, number of pieces
    int* cnt = nullptr;              // [n] tickets taken in the current launch (0 between launches)
    void* slots = nullptr;           // [npieces] piece sums (the launch's T)
    int n = 0;                       // split rows
    // Compacted task lists (batched solves): list w is perm[wbeg[w], wend[w])
    // instead of perm[wbeg[w], wbeg[w + 1]).  nullptr: the full lists.
    const int32_t* wend = nullptr;
};

// State and scaled data of one precision T (double or float).
template <typename T>
struct Engine {
    bool ready = false;
    // scaled matrix in both orientations (values only; structure is shared)
    T* val = nullptr;      // K~, CSR order of K   (padded to a multiple of 8)
    T* tval = nullptr;     // K~^T, CSR order of K^T
    T *c = nullptr, *q = nullptr, *l = nullptr, *u = nullptr;   // scaled vectors
    // iterate double buffers
    T* X[2] = {nullptr, nullptr};
    T* Y[2] = {nullptr, nullptr};
    T* KX[2] = {nullptr, nullptr};
    T* KTY[2] = {nullptr, nullptr};
    T *XS = nullptr, *YS = nullptr;      // eta-weighted sums
    T *XA = nullptr, *YA = nullptr;      // averages
    T *KXA = nullptr, *KTYA = nullptr;   // their products
    T *XANC = nullptr, *YANC = nullptr;  // restart anchor
    T* KXANC = nullptr;                  // K x of the anchor (Halpern iterations)
    T* XH = nullptr;                     // x^ of the last Halpern iteration (K launch input)
    // warp-task schedules for this precision's task capacity
    int32_t* brow = nullptr;   int nblk = 0;    // K rows: task boundaries, task count
    int32_t* bcol = nullptr;   int ntblk = 0;   // K^T rows
    int64_t* bnzK = nullptr;   int64_t* bnzT = nullptr;   // first nonzero of each task
    int32_t* wbegK = nullptr;  int32_t* permK = nullptr;  // per-warp task lists (K)
    int32_t* wbegT = nullptr;  int32_t* permT = nullptr;  // per-warp task lists (K^T)
    int gK = 0, gT = 0;                         // blocks of the K and K^T SpMV launches
    SplitRows splitK, splitT;                   // rows cut into pieces (n = 0: none)
    int npK = 0, npT = 0;                       // partials of the two launches: grid + split rows
    SchedParams schedK, schedT;                 // parameters of the two schedules
    bool tuned = false;                         // schedules chosen by the autotuner
    // Ruiz factors R, C and their reciprocals in this precision (KKT checks)
    T* Rt = nullptr; T* Ct = nullptr; T* Rinv = nullptr; T* Cinv = nullptr;
    // reduction partials
    double* partD = nullptr;   // [2][npK] Algorithm 5 partials of the K x' launch
    double* partT = nullptr;   // [max(npT, kEWGrid)] ||x' - x||^2 partials (k_primal, or the
                               // K^T launch's fused primal step): one per block of the K^T
                               // launch grid, then one per split row of its schedule
    size_t partD_cap = 0, partT_cap = 0;        // allocated entries
    double* partR = nullptr;   // [kRowQ][kEWGrid]
    double* partC = nullptr;   // [kColQ][kEWGrid]
    Ctrl* ctrl = nullptr;
    lp_trace_rec* trace = nullptr;  // device trace ring
    long long trace_cap = 0;
    double* alog = nullptr;         // device attempt log (kAttemptFields per record)
    long long alog_cap = 0;
    double* ftab = nullptr;         // Algorithm 5 factors of a check period [2][ftab_cap]
    int ftab_cap = 0;
    // loop graph
    cudaGraphExec_t exec = nullptr;
    int graph_check_every = -1;
    int graph_slots = -1;
    bool graph_conditional = false;
    int graph_host_loop = -1;
    int graph_halpern = -1;
    cudaGraphExec_t body_exec = nullptr;   // host-loop fallback
};

struct Handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t m = 0, n = 0, nnz = 0;
    // original (unscaled) problem, FP64
    int64_t* rp = nullptr;       // [m+1]
    int32_t* ci = nullptr;       // [nnz] padded
    double* val0 = nullptr;      // [nnz] padded
    uint8_t* sense = nullptr;    // [m]
    double *c0 = nullptr, *q0 = nullptr, *l0 = nullptr, *u0 = nullptr;
    int32_t* krow = nullptr;     // row of each nonzero of K
    // transpose
    int64_t* trp = nullptr;      // [n+1]
    int32_t* tci = nullptr;      // [nnz] padded: row index i of each K^T entry
    int32_t* tperm = nullptr;    // [nnz]: K^T entry -> nonzero index of K
    // scaling
    double *R = nullptr, *C = nullptr;
    double qnorm = 0, cnorm = 0;
    // host copies of the structure (for the schedulers)
    std::vector<int64_t> h_rp, h_trp;
    // scratch
    double* scratch = nullptr;   size_t scratch_bytes = 0;
    double* wbuf = nullptr;      // [n + m] scaled FP64 hand-off state (mixed precision polish)
    int* dev_err = nullptr;      // device flag: a bounded wait of a kernel gave up
    std::vector<DevBuf> allocs;
    Engine<double> e64;
    Engine<float> e32;
    long long launches = 0;      // kernels launched by the host (graph bodies counted apart)
    // attempt log of the current lp_solve (host buffer of the caller, records
    // already written by an earlier phase)
    double* alog_host = nullptr;
    long long alog_cap_host = 0, alog_off = 0;
    int built_precision_mask = 0;
};

}  // namespace pdhg

// The opaque handle of the C ABI.
struct lp_problem_s {
    pdhg::Handle h;
};

namespace pdhg {

template <typename T> Engine<T>& engine_of(Handle* h);
template <> inline Engine<double>& engine_of<double>(Handle* h) { return h->e64; }
template <> inline Engine<float>& engine_of<float>(Handle* h) { return h->e32; }

// ------------------------------------------------------------ error plumbing

#define LP_CUDA_TRY(expr)                                                        \
    do {                                                                         \
        cudaError_t _e = (expr);                                                 \
        if (_e != cudaSuccess) {                                                 \
            (void)cudaGetLastError();                                            \
            return _e == cudaErrorMemoryAllocation ? LP_OUT_OF_MEMORY : LP_CUDA_ERROR; \
        }                                                                        \
    } while (0)

#define LP_TRY(expr)                                                             \
    do {                                                                         \
        lp_status _s = (expr);                                                   \
        if (_s != LP_OK) return _s;                                              \
    } while (0)

lp_status dev_alloc(Handle* h, void** p, size_t bytes);
template <typename T>
inline lp_status dev_alloc_n(Handle* h, T** p, size_t count)
{
    void* q = nullptr;
    lp_status s = dev_alloc(h, &q, count * sizeof(T) + 64);
    *p = static_cast<T*>(q);
    return s;
}
inline size_t pad8(int64_t n) { return (size_t)((n + 7) & ~(int64_t)7); }

// ------------------------------------------------------- device reductions

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sums NQ per-thread values over the block (fixed order) and stores the block
// totals at part[q * stride + blockIdx.x].
template <int NQ, int NT>
__device__ __forceinline__ void block_partials(const double (&v)[NQ], double* part, int stride)
{
    __shared__ double sh[NQ][NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double t = warp_sum(v[q]);
        if (lane == 0) sh[q][warp] = t;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = lane < NT / 32 ? sh[q][lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) part[(size_t)q * stride + blockIdx.x] = t;
        }
    }
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block maxima of NQ per-thread values into part[q * stride + blockIdx.x].
template <int NQ, int NT>
__device__ __forceinline__ void block_partials_max(const double (&v)[NQ], double* part, int stride)
{
    __shared__ double sh[NQ][NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double t = warp_max(v[q]);
        if (lane == 0) sh[q][warp] = t;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = lane < NT / 32 ? sh[q][lane] : -INFINITY;
            t = warp_max(t);
            if (lane == 0) part[(size_t)q * stride + blockIdx.x] = t;
        }
    }
}

// Maximum of part[0..count) by a whole block (valid in every thread).
template <int NT>
__device__ double block_max_array(const double* part, int count)
{
    __shared__ double sh[NT / 32];
    __shared__ double total;
    double s = -INFINITY;
    for (int i = threadIdx.x; i < count; i += NT) s = fmax(s, __ldcg(part + i));
    s = warp_max(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    if (warp == 0) {
        double t = lane < NT / 32 ? sh[lane] : -INFINITY;
        t = warp_max(t);
        if (lane == 0) total = t;
    }
    __syncthreads();
    double r = total;
    __syncthreads();
    return r;
}

// Fixed-order sum of part[0..count) by a whole block of NT threads; the
// result is valid in every thread.  Loads go through L2 (ld.global.cg), so
// values written by other blocks of the same launch are seen after a fence.
template <int NT>
__device__ double block_sum_array(const double* part, int count)
{
    __shared__ double sh[NT / 32];
    __shared__ double total;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * NT < count; i += 4 * NT) {
        s0 += __ldcg(part + i);
        s1 += __ldcg(part + i + NT);
        s2 += __ldcg(part + i + 2 * NT);
        s3 += __ldcg(part + i + 3 * NT);
    }
    for (; i < count; i += NT) s0 += __ldcg(part + i);
    double s = (s0 + s1) + (s2 + s3);
    s = warp_sum(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    if (warp == 0) {
        double t = lane < NT / 32 ? sh[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) total = t;
    }
    __syncthreads();
    double r = total;
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------ setup kernels
// (defined in setup.cu; the batched solver launches them too)
__global__ void k_row_inf(int64_t m, const int64_t* rp, const double* v, double* rn);
__global__ void k_col_inf(int64_t nnz, const int32_t* ci, const double* v, unsigned long long* cn);
__global__ void k_ruiz_factors(int64_t count, double* nrm, double* acc);
__global__ void k_scale_vals(int64_t nnz, const int32_t* krow, const int32_t* ci, const double* r,
                             const double* s, double* v);
__global__ void k_pc_sums(int64_t m, int64_t n, const int64_t* rp, const int64_t* trp,
                          const int32_t* tperm, const double* v, double alpha, double* rs,
                          double* cs);
__global__ void k_scale_vectors(int64_t m, int64_t n, const double* R, const double* C,
                                const double* c0, const double* q0, const double* l0,
                                const double* u0, double* c, double* q, double* l, double* u);

// ------------------------------------------------------------ entry points
// setup.cu
lp_status setup_create(Handle* h, const lp_desc* d);
lp_status setup_scale(Handle* h, const lp_opts* o, double* normK);
template <typename T> lp_status setup_engine(Handle* h, const lp_opts* o);
// Engine<T>::Rt, Ct, Rinv, Cinv from the current FP64 Ruiz factors (allocated once).
template <typename T> lp_status engine_factors(Handle* h);
// (Re)builds the engine's warp-task schedules of K and K^T with the given
// parameters (frees the previous ones).
template <typename T> lp_status engine_schedule(Handle* h, SchedParams sK, SchedParams sT);
// Times the candidate warp-task schedules of K and K^T on the engine's scaled
// values and keeps the fastest of each (once per engine; drops a captured loop
// graph when a schedule changes).
template <typename T> lp_status tune_engine(Handle* h);
// Frees one allocation made by dev_alloc / dev_alloc_n.
void dev_free(Handle* h, void* p);
// solver.cu
template <typename T>
lp_status run_solve(Handle* h, const lp_opts* o, double eta0, double omega0,
                    const double* warm_x_scaled_dev, const double* warm_y_scaled_dev,
                    const double* warm_x_user, const double* warm_y_user, int warm_space,
                    long long k0, long long attempts0, long long restarts0,
                    lp_trace_rec* trace_host, long long trace_cap_host, long long trace_off,
                    Ctrl* out_ctrl);
template <typename T>
lp_status extract_solution(Handle* h, double* x, double* y, int space);
template <typename T>
lp_status extract_solution_ex(Handle* h, double* x, double* y, int space, double* xs_dev,
                              double* ys_dev);
lp_status sum_of_squares(Handle* h, const double* v, int64_t count, double* out_host);
template <typename T>
lp_status profile_step(Handle* h, int reps, double* ms, double* bytes);
// grad.cu
lp_status run_grad(Handle* h, const lp_opts* o, int K_iters, int ckpt, const double* gxK,
                   double* dc, double* dq, double* dvals, double* xK, int space,
                   double* tau_sigma);
// Algorithm 7 (fishnet.cu): repopulation draws of P columns, and the run on
// the prepared FP64 engine.
int64_t fishnet_draws(int P);
lp_status run_fishnet(Handle* h, int precision, double eta, double omega, double normK, int P,
                      int k_steps, const double* G, const double* Z_host, int64_t nZ, double* x0,
                      double* y0, double* gaps_host, int32_t* rounds_out, int space);
lp_status run_unroll(Handle* h, const lp_opts* o, int K_iters, double* xK, double* yK, int space,
                     double* tau_sigma);
// setup.cu
lp_status setup_update(Handle* h, const double* vals, const double* c, const double* q,
                       const double* l, const double* u, int space);

}  // namespace pdhg
