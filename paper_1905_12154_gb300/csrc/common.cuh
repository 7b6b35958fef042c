// common.cuh -- shared device/host helpers of the BFM CUDA library (sm_103a).
//
// Line-tile addressing: every hot kernel of the method works on whole grid
// lines along one axis (the separable c-transform of Section 4.1 and the
// DCT-based Poisson solve of Section 4.3).  A CTA takes a tile of W lines
// into shared memory with coalesced loads:
//   axis 0 ("contiguous"): W consecutive rows, each n0 contiguous elements;
//   axis >= 1 ("interleaved"): W lines that are neighbours along axis 0, so
//   one element position of the W lines is W consecutive floats in memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/bfm.h"

namespace bfm {

constexpr int kMaxN = 8192;          // largest line length
constexpr int kMaxStages = 16;       // FFT stages (radix 2/3/4)
constexpr int kPartialSlots = 8;     // FP64 partial-sum slots in a workspace
constexpr int kMaxPartials = 8192;   // partials per slot (CTAs of one launch)

// ---------------------------------------------------------------------------
// host-side error capture
// ---------------------------------------------------------------------------
void set_last_error(const char* msg);
bfm_status cuda_status(cudaError_t e, const char* where);

#define BFM_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::bfm::cuda_status(e_, #call);     \
    } while (0)

#define BFM_LAUNCH_CHECK(where)                                          \
    do {                                                                 \
        cudaError_t e_ = cudaGetLastError();                             \
        if (e_ != cudaSuccess) return ::bfm::cuda_status(e_, where);     \
    } while (0)

// ---------------------------------------------------------------------------
// grid description
// ---------------------------------------------------------------------------
struct Grid {
    int ndim;
    int n[3];
    long long N;
    long long stride[3];
};

bool make_grid(const bfm_grid* g, Grid* out);

// Lines along one axis, grouped into tiles of W lines.
struct LineTiles {
    int n;                    // line length
    long long es;             // element stride along the line
    int contig;               // axis 0: lines are rows
    int W;                    // lines per tile
    long long nlines;         // total lines
    long long ntiles;
    // interleaved axes: line (outer, i) with i in [0, nfast)
    int nfast;                // n0
    long long os;             // stride of `outer`
    int tiles_per_outer;      // ceil(nfast / W)
    int axis;
};

LineTiles make_tiles(const Grid& g, int axis, int W);

struct Tile {
    int wact;                 // lines present in this tile (<= W)
    long long base0;          // address of line 0, element 0
    long long lstride;        // address step between lines of the tile
    long long outer;          // interleaved: the outer index (else row0)
    int i0;                   // interleaved: first axis-0 index of the tile
};

__host__ __device__ inline Tile tile_at(const LineTiles& lt, long long t)
{
    Tile r;
    if (lt.contig) {
        long long row0 = t * lt.W;
        long long rem = lt.nlines - row0;
        r.wact = (int)(rem < lt.W ? rem : lt.W);
        r.base0 = row0 * lt.n;
        r.lstride = lt.n;
        r.outer = row0;
        r.i0 = 0;
    } else {
        long long outer = t / lt.tiles_per_outer;
        int i0 = (int)(t % lt.tiles_per_outer) * lt.W;
        int rem = lt.nfast - i0;
        r.wact = rem < lt.W ? rem : lt.W;
        r.base0 = outer * lt.os + i0;
        r.lstride = 1;
        r.outer = outer;
        r.i0 = i0;
    }
    return r;
}

// Element e of a tile's load/store sweep -> (line w, position p) so that
// consecutive e touch consecutive addresses.
__device__ inline void sweep_index(const LineTiles& lt, const Tile& tl, int e, int& w, int& p)
{
    if (lt.contig) { w = e / lt.n; p = e - w * lt.n; }
    else           { p = e / tl.wact; w = e - p * tl.wact; }
}

__device__ inline long long addr_of(const LineTiles& lt, const Tile& tl, int w, int p)
{
    return tl.base0 + (long long)w * tl.lstride + (long long)p * lt.es;
}

// ---------------------------------------------------------------------------
// FP64 block reduction (deterministic for a fixed launch shape)
// ---------------------------------------------------------------------------
__device__ inline double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// All threads must call; returns the block total on thread 0.
__device__ inline double block_sum(double v, double* scratch32)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch32[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? scratch32[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    return v;
}

__device__ inline double block_max(double v, double* scratch32)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) scratch32[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? scratch32[threadIdx.x] : -1.0e300;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Per-thread dot-product / sum accumulator.  FP64 arithmetic runs at a small
// fraction of the FP32 rate, so FP32 terms are accumulated in FP32 with
// error-free transformations (the exact product a*b = p + e via one FMA, and a
// compensated sum of the p's), which keeps about twice FP32 precision; the
// partial is widened to FP64 once per tile and every reduction beyond the
// thread is FP64.  FP64 terms are summed in FP64.
// ---------------------------------------------------------------------------
template <typename T> struct Acc;

template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    // explicitly rounded operations: the compiler must not fuse or reorder them
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);                     // a*b - p exactly
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ void add(float a)
    {
        const float t = __fadd_rn(s, a);
        const float z = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(a, z)));
        s = t;
    }
    __device__ __forceinline__ double take()
    {
        const double v = (double)s + (double)c;
        s = 0.f; c = 0.f;
        return v;
    }
};

template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add(double a) { s += a; }
    __device__ __forceinline__ double take() { const double v = s; s = 0.0; return v; }
};

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename T> struct Cx;
template <> struct Cx<float>  { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }

int num_sms();

}  // namespace bfm
