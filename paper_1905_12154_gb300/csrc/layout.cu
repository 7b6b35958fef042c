// layout.cu -- transposition of a 2-D field between the passes of a separable
// operation.
//
// The c-transform (Section 4.1, dimension splitting) and the DCT-based Poisson
// solve (Section 4.3) each sweep whole lines along every axis.  Lines along
// axis 0 are rows, read and written with full 128-byte sectors.  A tile of
// lines along axis 1 holds only a few neighbouring columns when the lines are
// long (two columns of 4096 FP32 cells fill a CTA's shared memory), so every
// row of such a tile moves 8 useful bytes per 32-byte sector.  On 2-D grids
// with such long columns the library instead transposes the field, runs the
// axis-1 sweep as a row sweep and transposes back.  A transpose moves square
// blocks through shared memory so that both its reads and its writes are
// whole rows: 64 x 64 FP32 blocks as float4 when the sides are multiples of
// 4 (a resident wave of CTAs, each prefetching its next block), else 32 x 32
// blocks of single elements.
#include "common.cuh"
#include "kernels.h"

namespace bfm {

constexpr int kTile = 32;
constexpr int kRowsPerPass = 8;            // 32 x 8 threads, four rows each

// out[c][r] = in[r][c] for an R x C input (R rows of C elements).  With w,
// each CTA also writes the FP64 partial sum of out * w (w laid out like out).
template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                        int R, int C, const T* __restrict__ w,
                                                        double* part, const int* done)
{
    if (done && *done) return;
    __shared__ T tile[kTile][kTile + 1];
    __shared__ double red[32];
    const int tx = threadIdx.x & (kTile - 1), ty = threadIdx.x / kTile;
    const int tilesC = (C + kTile - 1) / kTile;
    const long long ntiles = (long long)tilesC * ((R + kTile - 1) / kTile);
    Acc<T> acc;
    double total = 0.0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = (int)(t / tilesC) * kTile, c0 = (int)(t % tilesC) * kTile;
        T v[kTile / kRowsPerPass];
#pragma unroll
        for (int k = 0; k < kTile / kRowsPerPass; ++k) {
            const int r = r0 + ty + kRowsPerPass * k, c = c0 + tx;
            v[k] = (r < R && c < C) ? in[(long long)r * C + c] : (T)0;
        }
#pragma unroll
        for (int k = 0; k < kTile / kRowsPerPass; ++k) tile[ty + kRowsPerPass * k][tx] = v[k];
        __syncthreads();
        T u[kTile / kRowsPerPass];
        if (w) {
#pragma unroll
            for (int k = 0; k < kTile / kRowsPerPass; ++k) {
                const int c = c0 + ty + kRowsPerPass * k, r = r0 + tx;
                u[k] = (c < C && r < R) ? w[(long long)c * R + r] : (T)0;
            }
        }
#pragma unroll
        for (int k = 0; k < kTile / kRowsPerPass; ++k) {
            const int c = c0 + ty + kRowsPerPass * k, r = r0 + tx;
            if (c < C && r < R) {
                const T x = tile[tx][ty + kRowsPerPass * k];
                out[(long long)c * R + r] = x;
                if (w) acc.add_prod(x, u[k]);
            }
        }
        total += acc.take();
        __syncthreads();
    }
    if (part) {
        const double s = block_sum(total, red);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// FP32 fields whose sides are multiples of 4 (16-byte aligned): 64 x 64
// blocks moved as float4 on both sides (four loads in flight per thread).
// The shared block keeps an odd row length (65), so the column reads of the
// store side hit at most two threads per bank.
constexpr int kTileV = 64;

// A resident wave of CTAs (four per SM, every CTA the same number of blocks)
// loops over the blocks, software-pipelined: a CTA issues the loads of its
// next block right after its current block is in shared memory, so they are
// in flight while the current block is read out transposed and stored
// (against one block per CTA: 0.289 -> 0.262 ms per 4096^2 iteration).
__global__ void __launch_bounds__(256, 4) transpose4p_kernel(const float* __restrict__ in,
                                                          float* __restrict__ out, int R, int C,
                                                          const float* __restrict__ w, double* part,
                                                          const int* done)
{
    if (done && *done) return;
    __shared__ float tile[kTileV][kTileV + 1];
    __shared__ double red[32];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;      // 16 x 16 threads
    const int tilesC = (C + kTileV - 1) / kTileV;
    const long long ntiles = (long long)tilesC * ((R + kTileV - 1) / kTileV);
    Acc<float> acc;
    double total = 0.0;
    float4 v[4];
    auto load = [&](long long t) {
        const int r0 = (int)(t / tilesC) * kTileV, c0 = (int)(t % tilesC) * kTileV;
        const int c = c0 + 4 * tx;                    // C % 4 == 0: c < C covers c + 3
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = r0 + ty + 16 * k;
            v[k] = (r < R && c < C) ? *reinterpret_cast<const float4*>(in + (long long)r * C + c)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    long long t = blockIdx.x;
    if (t < ntiles) load(t);
    for (; t < ntiles; t += gridDim.x) {
        const int r0 = (int)(t / tilesC) * kTileV, c0 = (int)(t % tilesC) * kTileV;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float* row = tile[ty + 16 * k] + 4 * tx;
            row[0] = v[k].x; row[1] = v[k].y; row[2] = v[k].z; row[3] = v[k].w;
        }
        __syncthreads();
        if (t + gridDim.x < ntiles) load(t + gridDim.x);
        const int r = r0 + 4 * tx;                    // R % 4 == 0: r < R covers r + 3
        float4 u[4];
        if (w) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int oc = c0 + ty + 16 * k;
                u[k] = (oc < C && r < R) ? *reinterpret_cast<const float4*>(w + (long long)oc * R + r)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int cc = ty + 16 * k, oc = c0 + cc;
            if (oc < C && r < R) {
                const float4 o = make_float4(tile[4 * tx][cc], tile[4 * tx + 1][cc],
                                             tile[4 * tx + 2][cc], tile[4 * tx + 3][cc]);
                *reinterpret_cast<float4*>(out + (long long)oc * R + r) = o;
                if (w) {
                    acc.add_prod(o.x, u[k].x); acc.add_prod(o.y, u[k].y);
                    acc.add_prod(o.z, u[k].z); acc.add_prod(o.w, u[k].w);
                }
            }
        }
        total += acc.take();
        __syncthreads();
    }
    if (part) {
        const double s = block_sum(total, red);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

static bool aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T>
bfm_status launch_transpose(const T* in, T* out, int R, int C, const T* w, double* part,
                            const int* done, cudaStream_t st, int* blocks_used)
{
    if (R < 1 || C < 1 || in == out) {
        set_last_error("internal: bad transpose arguments");
        return BFM_ERR_INVALID_ARG;
    }
    if (sizeof(T) == 4 && R % 4 == 0 && C % 4 == 0 && aligned16(in) && aligned16(out) && aligned16(w)) {
        const long long tiles = (long long)((R + kTileV - 1) / kTileV) * ((C + kTileV - 1) / kTileV);
        const long long cap = (long long)num_sms() * 4;
        const long long per = (tiles + cap - 1) / cap;
        long long blocks = (tiles + per - 1) / per;
        if (blocks > kMaxPartials) blocks = kMaxPartials;
        transpose4p_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const float*>(in),
                                                             reinterpret_cast<float*>(out), R, C,
                                                             reinterpret_cast<const float*>(w), part,
                                                             done);
        BFM_LAUNCH_CHECK("transpose4p_kernel");
        if (blocks_used) *blocks_used = (int)blocks;
        return BFM_OK;
    }
    const long long tiles = (long long)((R + kTile - 1) / kTile) * ((C + kTile - 1) / kTile);
    long long blocks = (long long)num_sms() * 8;        // eight 256-thread CTAs per SM
    if (blocks > tiles) blocks = tiles;
    if (blocks > kMaxPartials) blocks = kMaxPartials;
    transpose_kernel<T><<<(unsigned)blocks, kTile * kRowsPerPass, 0, st>>>(in, out, R, C, w, part, done);
    BFM_LAUNCH_CHECK("transpose_kernel");
    if (blocks_used) *blocks_used = (int)blocks;
    return BFM_OK;
}

bool transposed_axis1(const Grid& g, int elem_bytes)
{
    // a column tile narrower than 8 lines moves less than one 32-byte sector
    // of FP32 per row
    return g.ndim == 2 && plan_ct_pass_default(g, 1, elem_bytes).W < 8;
}

Grid transposed_grid(const Grid& g)
{
    bfm_grid t;
    t.ndim = 2;
    t.n[0] = g.n[1];
    t.n[1] = g.n[0];
    t.n[2] = 1;
    Grid out;
    make_grid(&t, &out);
    return out;
}

template bfm_status launch_transpose<float>(const float*, float*, int, int, const float*, double*,
                                            const int*, cudaStream_t, int*);
template bfm_status launch_transpose<double>(const double*, double*, int, int, const double*,
                                             double*, const int*, cudaStream_t, int*);

}  // namespace bfm
