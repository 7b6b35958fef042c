// ctpower.cu -- the grid c-transform for separable power costs (Section 5,
// eq. p_costs): c(x, y) = sum_a |y_a - x_a|^{p_a} / p_a, p_a > 1.
//
// The cost is separable, so the c-transform splits into 1-D passes along the
// axes exactly as for the quadratic cost (Section 4.1, dimension splitting).
// A 1-D pass on a line of n cells computes
//     u(i) = min_j  H(|i - j|) + f(j),     H(k) = (k h)^p / p,
// and the cost is strictly convex, so the leftmost minimiser J(i) is
// non-decreasing in i (Section 4.1): the minimiser of a cell is trapped
// between those of two cells on either side.  The pass therefore fixes J(0) by
// a full scan and then the cells at stride s = 2^k, ..., 2, 1 in turn: cell
// i = s(2q + 1) searches only [J(i - s), J(i + s)] (the divide-and-conquer of
// Section 4.1, O(n log n) per line).  One warp owns one line: levels with many
// cells give each lane its own cell, levels with few cells split each search
// over the lanes and reduce with shuffles.  H is tabulated once per CTA.
#include "common.cuh"
#include "kernels.h"

namespace bfm {

template <typename T>
struct CtPowArgs {
    const T* in;
    T* out;
    const T* w_in;        // optional: partial sums of in * w_in
    const T* w_out;       // optional: partial sums of out * w_out
    double* part_in;
    double* part_out;
    const int* done;
    LineTiles lt;
    int LD;               // shared leading dimension of a line (elements)
    double p;             // exponent of this axis
    double h;             // cell size on this axis
    int negate;           // the pass reads -in
    int lw;               // log2(W) for interleaved tiles
};

// lexicographic (value, index) minimum over the warp; every lane gets it
template <typename T>
__device__ __forceinline__ void warp_argmin(T& v, int& j)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int oj = __shfl_xor_sync(0xffffffffu, j, off);
        if (ov < v || (ov == v && oj < j)) { v = ov; j = oj; }
    }
}

template <typename T>
__device__ __forceinline__ T pow_t(T x, T p);
template <> __device__ __forceinline__ float pow_t<float>(float x, float p) { return powf(x, p); }
template <> __device__ __forceinline__ double pow_t<double>(double x, double p) { return pow(x, p); }

template <typename T, bool CONTIG>
__global__ void __launch_bounds__(256) ct_power_kernel(CtPowArgs<T> a)
{
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LineTiles& lt = a.lt;
    const int n = lt.n;
    const int W = lt.W;                        // lines per tile = warps per CTA
    T* H = reinterpret_cast<T*>(smem_raw);                     // n
    T* fs = H + a.LD;                                          // W x LD values
    T* us = fs + (size_t)W * a.LD;                             // W x LD outputs
    int* js = reinterpret_cast<int*>(us + (size_t)W * a.LD);   // W x LD minimisers
    __shared__ double red[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const T pe = (T)a.p, hh = (T)a.h;
    for (int k = tid; k < n; k += blockDim.x) H[k] = pow_t<T>((T)k * hh, pe) / pe;
    T* f = fs + (size_t)w * a.LD;
    T* u = us + (size_t)w * a.LD;
    int* J = js + (size_t)w * a.LD;
    Acc<T> acc_t_in, acc_t_out;
    double acc_in = 0.0, acc_out = 0.0;
    int S = 1;
    while (2 * S <= n - 1) S *= 2;             // largest power of two <= n - 1

    for (long long tile = blockIdx.x; tile < lt.ntiles; tile += gridDim.x) {
        const Tile tl = tile_at(lt, tile);
        // ---- load the tile's lines (rows, or W neighbouring columns) ----------
        if (CONTIG) {
            for (int ww = 0; ww < tl.wact; ++ww) {
                const long long rb = tl.base0 + (long long)ww * n;
                for (int q = tid; q < n; q += blockDim.x) {
                    const T v = a.in[rb + q];
                    if (a.w_in) acc_t_in.add_prod(v, a.w_in[rb + q]);
                    fs[(size_t)ww * a.LD + q] = a.negate ? -v : v;
                }
            }
        } else {
            const int total = n << a.lw;
            for (int e = tid; e < total; e += blockDim.x) {
                const int q = e >> a.lw, ww = e & (W - 1);
                if (ww < tl.wact) {
                    const long long ad = tl.base0 + ww + (long long)q * lt.es;
                    const T v = a.in[ad];
                    if (a.w_in) acc_t_in.add_prod(v, a.w_in[ad]);
                    fs[(size_t)ww * a.LD + q] = a.negate ? -v : v;
                }
            }
        }
        __syncthreads();
        if (w < tl.wact) {
            // cell 0: the full line
            T bv = (T)INFINITY;
            int bj = n;
            for (int j = lane; j < n; j += 32) {
                const T v = H[j] + f[j];
                if (v < bv) { bv = v; bj = j; }
            }
            warp_argmin(bv, bj);
            if (lane == 0) { J[0] = bj; u[0] = bv; }
            __syncwarp();
            for (int s = S; s >= 1; s >>= 1) {
                const int nq = (n - 1 - s) / (2 * s) + 1;       // cells s, 3s, 5s, ... < n
                if (nq >= 16) {
                    for (int q = lane; q < nq; q += 32) {
                        const int i = s * (2 * q + 1);
                        const int lo = J[i - s];
                        int hi = (i + s < n) ? J[i + s] : n - 1;
                        if (hi < lo) hi = lo;          // brackets are ordered; never empty
                        T v0 = (T)INFINITY;
                        int j0 = lo;
                        for (int j = lo; j <= hi; ++j) {
                            const T v = H[i > j ? i - j : j - i] + f[j];
                            if (v < v0) { v0 = v; j0 = j; }
                        }
                        J[i] = j0;
                        u[i] = v0;
                    }
                } else {
                    for (int q = 0; q < nq; ++q) {
                        const int i = s * (2 * q + 1);
                        const int lo = J[i - s];
                        int hi = (i + s < n) ? J[i + s] : n - 1;
                        if (hi < lo) hi = lo;
                        T v0 = (T)INFINITY;
                        int j0 = n;
                        for (int j = lo + lane; j <= hi; j += 32) {
                            const T v = H[i > j ? i - j : j - i] + f[j];
                            if (v < v0) { v0 = v; j0 = j; }
                        }
                        warp_argmin(v0, j0);
                        if (lane == 0) { J[i] = j0; u[i] = v0; }
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // ---- store ---------------------------------------------------------------
        if (CONTIG) {
            for (int ww = 0; ww < tl.wact; ++ww) {
                const long long rb = tl.base0 + (long long)ww * n;
                for (int q = tid; q < n; q += blockDim.x) {
                    const T v = us[(size_t)ww * a.LD + q];
                    a.out[rb + q] = v;
                    if (a.w_out) acc_t_out.add_prod(v, a.w_out[rb + q]);
                }
            }
        } else {
            const int total = n << a.lw;
            for (int e = tid; e < total; e += blockDim.x) {
                const int q = e >> a.lw, ww = e & (W - 1);
                if (ww < tl.wact) {
                    const long long ad = tl.base0 + ww + (long long)q * lt.es;
                    const T v = us[(size_t)ww * a.LD + q];
                    a.out[ad] = v;
                    if (a.w_out) acc_t_out.add_prod(v, a.w_out[ad]);
                }
            }
        }
        acc_in += acc_t_in.take();
        acc_out += acc_t_out.take();
        __syncthreads();
    }
    if (a.part_in) {
        const double s = block_sum(acc_in, red);
        if (threadIdx.x == 0) a.part_in[blockIdx.x] = s;
    }
    if (a.part_out) {
        const double s = block_sum(acc_out, red);
        if (threadIdx.x == 0) a.part_out[blockIdx.x] = s;
    }
}

// Lines per CTA: up to 8 warps, as many as fit about 100 KB of shared memory
// (a power of two for interleaved tiles).
static int power_lines_per_cta(const Grid& g, int axis, int eb, int* LD, size_t* smem)
{
    const int n = g.n[axis];
    *LD = n + (n & 1);
    const size_t line = (size_t)(*LD) * (2 * eb + 4);
    int W = 8;
    while (W > 1 && (size_t)(*LD) * eb + (size_t)W * line > 100 * 1024) W >>= 1;
    if (axis != 0 && W > g.n[0]) {
        int p2 = 1;
        while (p2 * 2 <= g.n[0]) p2 *= 2;
        W = p2;
    }
    *smem = (size_t)(*LD) * eb + (size_t)W * line;
    return W;
}

template <typename T>
bfm_status launch_ct_power_pass(const Grid& g, int axis, double p, const T* in, T* out, bool negate,
                                const T* w_in, double* part_in, const T* w_out, double* part_out,
                                const int* done, int max_blocks, cudaStream_t st, int* blocks_used)
{
    int LD;
    size_t smem;
    const int W = power_lines_per_cta(g, axis, (int)sizeof(T), &LD, &smem);
    if (smem > 220 * 1024) {
        set_last_error("power-cost c-transform: line too long for shared memory");
        return BFM_ERR_UNSUPPORTED;
    }
    CtPowArgs<T> a;
    a.in = in; a.out = out; a.w_in = w_in; a.w_out = w_out;
    a.part_in = part_in; a.part_out = part_out; a.done = done;
    a.lt = make_tiles(g, axis, W);
    a.LD = LD;
    a.p = p;
    a.h = 1.0 / g.n[axis];
    a.negate = negate ? 1 : 0;
    a.lw = 0;
    while ((1 << a.lw) < W) ++a.lw;
    void* k = (axis == 0) ? (void*)ct_power_kernel<T, true> : (void*)ct_power_kernel<T, false>;
    BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    long long blocks = a.lt.ntiles;
    const long long cap = (long long)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    void* args[] = {&a};
    BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(32 * W), args, smem, st));
    if (blocks_used) *blocks_used = (int)blocks;
    return BFM_OK;
}

template bfm_status launch_ct_power_pass<float>(const Grid&, int, double, const float*, float*, bool,
                                                const float*, double*, const float*, double*,
                                                const int*, int, cudaStream_t, int*);
template bfm_status launch_ct_power_pass<double>(const Grid&, int, double, const double*, double*,
                                                 bool, const double*, double*, const double*,
                                                 double*, const int*, int, cudaStream_t, int*);

}  // namespace bfm
