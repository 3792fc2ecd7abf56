// Row-block CSR SpMV with fused epilogues (the products K x and K^T y of
// Algorithm 1, plus whatever elementwise update consumes each row result).
//
// Layout: the rows of a CSR matrix are cut on the host into row-blocks
// (brow[b] .. brow[b+1]) holding at most Cap<T> nonzeros and at most kNT rows,
// except that a row longer than Cap<T> forms a block by itself.  A short-row
// block streams its contiguous nonzero range with 16-byte vector loads of
// values and column indices (evict-first, so the gathered vector stays in L2),
// multiplies by the gathered x and stages the products in shared memory; each
// row is then summed by a group of G lanes (G = the largest power of two with
// G * rows <= kNT, at most 32) with a shuffle tree.  A long-row block loops over
// its row with the whole block and reduces in a fixed tree.  Every sum has a
// fixed order, so results are bitwise reproducible run to run.
//
// Epilogue interface (Epi):
//   bool begin()                       uniform per launch; false = return at once
//   const T* xin()                     the vector being multiplied
//   struct Acc; void row(int r, T v, Acc&)   called once per row by one thread
//   void finish(Acc&)                  block-level partial reductions (all threads)
#pragma once

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
};

template <typename T, int NT>
__device__ __forceinline__ T block_reduce_T(T v)
{
    __shared__ T sh[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    T r = 0;
    if (warp == 0) {
        r = lane < NT / 32 ? sh[lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;   // valid in thread 0
}

template <typename T, class Epi>
__global__ void __launch_bounds__(kNT)
k_spmv(const int32_t* __restrict__ brow, const int64_t* __restrict__ rp,
       const int32_t* __restrict__ ci, const T* __restrict__ val, Epi epi)
{
    constexpr int CAP = Cap<T>::value;
    using VT = VecTraits<T>;
    constexpr int VEC = VT::N;
    __shared__ T prod[CAP];
    if (!epi.begin()) return;
    const T* __restrict__ xv = epi.xin();
    const int tid = threadIdx.x;
    const int r0 = brow[blockIdx.x], r1 = brow[blockIdx.x + 1];
    const int64_t s = rp[r0], e = rp[r1];
    typename Epi::Acc acc;
    if (e - s > CAP) {
        T a = 0;
        for (int64_t p = s + tid; p < e; p += kNT) a += __ldcs(val + p) * __ldg(xv + __ldcs(ci + p));
        a = block_reduce_T<T, kNT>(a);
        if (tid == 0) epi.row(r0, a, acc);
    } else {
        const int64_t a0 = s & ~(int64_t)(VEC - 1);
        for (int64_t c = a0 + (int64_t)tid * VEC; c < e; c += (int64_t)kNT * VEC) {
            T vv[VEC];
            int ii[VEC];
            VT::unpack(__ldcs(reinterpret_cast<const typename VT::V*>(val + c)), vv);
            VT::unpacki(__ldcs(reinterpret_cast<const typename VT::I*>(ci + c)), ii);
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                const int64_t p = c + k;
                if (p >= s && p < e) prod[p - s] = vv[k] * __ldg(xv + ii[k]);
            }
        }
        __syncthreads();
        const int nrows = r1 - r0;
        int G = 32;
        while (G > 1 && G * nrows > kNT) G >>= 1;
        const int grp = tid / G, lane = tid % G, ngrp = kNT / G;
        for (int base = 0; base < nrows; base += ngrp) {
            const int r = r0 + base + grp;
            T a = 0;
            if (r < r1) {
                const int64_t pe = rp[r + 1];
                for (int64_t p = rp[r] + lane; p < pe; p += G) a += prod[p - s];
            }
            for (int o = G >> 1; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o, G);
            if (r < r1 && lane == 0) epi.row(r, a, acc);
        }
    }
    epi.finish(acc);
}

// Plain epilogue: out[r] = scale * v, with the optional FP64 partial
// sum of out[r]^2 (power iteration) and a skip flag read from a Ctrl field.
template <typename T>
struct EpiStore {
    const T* x;
    T* out;
    const double* scale;     // nullptr = 1
    double* part;            // nullptr = no partials
    const int* gate;         // nullptr = always run; else run when *gate != 0
    struct Acc { double s2 = 0.0; };
    __device__ bool begin() const { return gate == nullptr || *gate != 0; }
    __device__ const T* xin() const { return x; }
    __device__ void row(int r, T v, Acc& a) const {
        if (scale) v = (T)((double)v * *scale);
        out[r] = v;
        a.s2 += (double)v * (double)v;
    }
    __device__ void finish(Acc& a) const {
        if (part) {
            const double t[1] = {a.s2};
            block_partials<1, kNT>(t, part, gridDim.x);
        }
    }
};

// Greedy row-block partition (host): rows are added to the current block
// while it holds <= cap nonzeros and <= max_rows rows; a row longer than cap
// gets a block of its own.  Returns the block boundaries (nblk + 1 entries).
std::vector<int32_t> make_row_blocks(const int64_t* rp, int64_t rows, int cap, int max_rows);

}  // namespace pdhg
