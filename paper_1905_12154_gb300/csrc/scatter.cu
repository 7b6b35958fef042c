// scatter.cu -- the map T(x) = x - grad psi(x) and the pushforward T # mu.
//
// Lemma 2.2(ii): the minimiser of the c-transform is T(x) = x -
// (grad h)^{-1}(grad phi^c(x)): x - grad phi^c(x) for the quadratic cost, and
// per axis x_a - sign(w_a)|w_a|^{1/(p_a - 1)} (w = grad phi^c) for the
// separable power cost of Section 5.  Lemma 3.1: the first variation of J is
// nu - T # mu.  The pushforward (Section 2.1) is discretised by sending the
// mass of every source cell to the 2^d cell centres around T(x) with
// multilinear weights; T is clamped to the box of cell centres so mass is
// conserved.  grad psi uses central differences, one-sided at the first and
// last cell of a line.  Positions are kept in cell-index units,
//   pos_a = i_a - (d psi / d x_a) * n_a,
// which keeps FP32 exact to the rounding of the difference itself.
#include "common.cuh"
#include "kernels.h"

namespace bfm {

struct GridDev {
    int n[3];
    long long s[3];
    long long N;
    int power;            // separable power cost: (h_a')^{-1}(w) = sign(w)|w|^{q_a}
    double q[3];          // q_a = 1 / (p_a - 1)
};

// p: the exponents of a separable power cost (axis 0 first), NULL for the
// quadratic cost
static GridDev dev_grid(const Grid& g, const double* p = nullptr)
{
    GridDev d;
    for (int a = 0; a < 3; ++a) {
        d.n[a] = g.n[a];
        d.s[a] = g.stride[a];
        d.q[a] = (p && a < g.ndim) ? 1.0 / (p[a] - 1.0) : 1.0;
    }
    d.N = g.N;
    d.power = p ? 1 : 0;
    return d;
}

template <typename T> __device__ __forceinline__ T pow_s(T x, T y);
template <> __device__ __forceinline__ float pow_s<float>(float x, float y) { return powf(x, y); }
template <> __device__ __forceinline__ double pow_s<double>(double x, double y) { return pow(x, y); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

static int grid_blocks(long long N, int threads)
{
    long long b = (N + threads - 1) / threads;
    const long long cap = (long long)num_sms() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// position of T(x) along one axis, in cell-index units, clamped to [0, n-1],
// from psi at the cell (pc) and its neighbours before (pm) and after (pp)
template <typename T>
__device__ __forceinline__ T axis_pos(T pm, T pc, T pp, int i, int n, int power, double q)
{
    T dpsi;                                   // psi difference per cell
    if (i == 0)          dpsi = pp - pc;
    else if (i == n - 1) dpsi = pc - pm;
    else                 dpsi = (pp - pm) * (T)0.5;
    T dpos;
    if (!power) {
        dpos = dpsi * ((T)n * (T)n);          // grad psi in cell units, divided by h
    } else {
        const T w = dpsi * (T)n;              // d psi / d x_a
        dpos = copysign(pow_s<T>(fabs(w), (T)q), w) * (T)n;
    }
    T pos = (T)i - dpos;
    pos = fmin(fmax(pos, (T)0), (T)(n - 1));
    return pos;
}

template <typename T>
__device__ __forceinline__ T map_pos(const T* psi, long long idx, int i, int n, long long s,
                                     int power, double q)
{
    const T pm = i > 0 ? psi[idx - s] : (T)0;
    const T pp = i < n - 1 ? psi[idx + s] : (T)0;
    return axis_pos(pm, psi[idx], pp, i, n, power, q);
}

template <typename T, int NDIM>
__device__ __forceinline__ void deposit(T* rho, const GridDev& g, const T* pos, T m)
{
    int i0[3];
    T w1[3];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        int c = (int)floor(pos[a]);
        if (c > g.n[a] - 2) c = g.n[a] - 2;
        if (c < 0) c = 0;
        i0[a] = c;
        w1[a] = pos[a] - (T)c;
    }
#pragma unroll
    for (int c = 0; c < (1 << NDIM); ++c) {
        T w = m;
        long long q = 0;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const int up = (c >> a) & 1;
            w *= up ? w1[a] : ((T)1 - w1[a]);
            q += (long long)(i0[a] + up) * g.s[a];
        }
        if (w != (T)0) atomicAdd(rho + q, w);
    }
}

template <typename T, int NDIM>
__global__ void pushforward_kernel(const T* __restrict__ psi, const T* __restrict__ mu,
                                   T* __restrict__ rho, GridDev g, const int* done)
{
    if (done && *done) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        const T m = mu[idx];
        if (m == (T)0) continue;
        long long r = idx;
        T pos[3];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const int i = (int)(r % g.n[a]);
            r /= g.n[a];
            pos[a] = map_pos(psi, idx, i, g.n[a], g.s[a], g.power, g.q[a]);
        }
        deposit<T, NDIM>(rho, g, pos, m);
    }
}

// The pushforward along rows: one 16-byte vector of cells per thread (4 FP32
// or 2 FP64 cells), a CTA segment of 256 vectors of one line along axis 0 per
// step, so the row and column indices cost one division per segment instead
// of per cell.  FP32 deposits go out as vector reductions: the two cells
// (c, c + 1) of a line that a bilinear deposit touches are one 8-byte red
// when c is even, one 16-byte red with zero ends when c = 1 mod 4, else two
// scalar reds.  Needs n0 % 4 == 0 and 16-byte aligned fields.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int V = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int V = 2; };

template <typename T>
__device__ __forceinline__ void unpack(const typename Vec16<T>::type& v, T* o);
template <> __device__ __forceinline__ void unpack<float>(const float4& v, float* o)
{ o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
template <> __device__ __forceinline__ void unpack<double>(const double2& v, double* o)
{ o[0] = v.x; o[1] = v.y; }

// rho[q] += a, rho[q + 1] += b
__device__ __forceinline__ void red_pair(float* rho, long long q, float a, float b)
{
    const int r = (int)(q & 3);
    if ((r & 1) == 0) {
        atomicAdd(reinterpret_cast<float2*>(rho + q), make_float2(a, b));
    } else if (r == 1) {
        atomicAdd(reinterpret_cast<float4*>(rho + q - 1), make_float4(0.f, a, b, 0.f));
    } else {
        atomicAdd(rho + q, a);
        atomicAdd(rho + q + 1, b);
    }
}

__device__ __forceinline__ void red_pair(double* rho, long long q, double a, double b)
{
    if (a != 0.0) atomicAdd(rho + q, a);
    if (b != 0.0) atomicAdd(rho + q + 1, b);
}

// Deposits of a thread's consecutive cells: cells whose multilinear stencils
// coincide (a map that contracts along the row) are summed in registers and
// sent as one set of reductions.
template <typename T, int NDIM>
struct StencilAcc {
    static constexpr int C = 1 << (NDIM - 1);     // lines of the stencil across axes 1..
    long long q0 = -1;                            // offset of the stencil's first cell
    T a[C], b[C];                                 // weights at q_c and q_c + 1
    __device__ __forceinline__ void flush(T* rho, const GridDev& g)
    {
        if (q0 < 0) return;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            long long q = q0;
#pragma unroll
            for (int ax = 1; ax < NDIM; ++ax) q += ((c >> (ax - 1)) & 1) * g.s[ax];
            red_pair(rho, q, a[c], b[c]);
        }
    }
    __device__ __forceinline__ void add(T* rho, const GridDev& g, const T* pos, T m)
    {
        int i0[3];
        T w1[3];
#pragma unroll
        for (int ax = 0; ax < NDIM; ++ax) {
            int c = (int)floor(pos[ax]);
            if (c > g.n[ax] - 2) c = g.n[ax] - 2;
            if (c < 0) c = 0;
            i0[ax] = c;
            w1[ax] = pos[ax] - (T)c;
        }
        long long q = i0[0];
#pragma unroll
        for (int ax = 1; ax < NDIM; ++ax) q += (long long)i0[ax] * g.s[ax];
        if (q != q0) {
            flush(rho, g);
            q0 = q;
#pragma unroll
            for (int c = 0; c < C; ++c) a[c] = b[c] = (T)0;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            T w = m;
#pragma unroll
            for (int ax = 1; ax < NDIM; ++ax) {
                const int up = (c >> (ax - 1)) & 1;
                w *= up ? w1[ax] : ((T)1 - w1[ax]);
            }
            a[c] += w * ((T)1 - w1[0]);
            b[c] += w * w1[0];
        }
    }
};

// 16-byte vectors per thread: two on 2-D grids, one on 3-D grids (whose six
// neighbour rows already hold a thread's registers)
template <int NDIM> __host__ __device__ constexpr int push_vecs() { return NDIM == 2 ? 2 : 1; }

// SWAP (2-D): psi and mu come in the transposed layout of rho's grid `go`
// (g is that transposed grid); each target position is swapped to go's axes
// before it is deposited, so rho comes out in go's layout with no transpose.
// part (optional): per-CTA FP64 partial sums of psi * mu (the second term of
// the dual value, eq. defJ / defI), taken from the loads the map needs: each
// item's few cells summed in the field precision, the items in FP64.
template <typename T, int NDIM, bool SWAP>
__device__ __forceinline__ void pushforward_rows_body(const T* __restrict__ psi,
                                                      const T* __restrict__ mu,
                                                      T* __restrict__ rho, const GridDev& g,
                                                      int per_row, const int* done,
                                                      const GridDev& go, double* part)
{
    if (done && *done) return;
    using VT = typename Vec16<T>::type;
    constexpr int V = Vec16<T>::V;
    constexpr int NV = push_vecs<NDIM>(), CW = NV * V;   // cells per thread
    const int n0 = g.n[0];
    const long long rows = g.N / n0;
    const unsigned items = (unsigned)(rows * per_row);     // < 2^31 (checked by the launcher)
    const unsigned stride = gridDim.x * blockDim.x;
    // the source density of the thread's next item is loaded while the current
    // one is processed (its psi loads wait for it otherwise)
    VT mv[NV];
    auto load_mu = [&](unsigned it) {
        const unsigned row = it / (unsigned)per_row;
        const int x0 = (int)(it - row * (unsigned)per_row) * CW;
        const long long base = (long long)row * n0 + x0;
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j == 0 || x0 + j * V < n0) mv[j] = *reinterpret_cast<const VT*>(mu + base + j * V);
    };
    unsigned it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it < items) load_mu(it);
    double dsum = 0.0;
    for (; it < items; it += stride) {
        const unsigned row = it / (unsigned)per_row;
        const int x0 = (int)(it - row * (unsigned)per_row) * CW;
        const long long base = (long long)row * n0 + x0;
        T m[CW];
        bool any = false;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            if (j == 0 || x0 + j * V < n0) unpack<T>(mv[j], m + j * V);
            else
#pragma unroll
                for (int k = 0; k < V; ++k) m[j * V + k] = (T)0;
        }
        if (it + stride < items) load_mu(it + stride);
#pragma unroll
        for (int k = 0; k < CW; ++k) any |= (m[k] != (T)0);
        if (!any) continue;
        T c[CW + 2];                                  // psi at x0 - 1 .. x0 + CW along the row
        T lo[NDIM - 1][CW], hi[NDIM - 1][CW];         // neighbours along axes 1.. (unused at a face)
        int ia[3] = {0, 0, 0};
        {
            long long r = row;
#pragma unroll
            for (int a = 1; a < NDIM; ++a) {
                ia[a] = (int)(r % g.n[a]);
                r /= g.n[a];
            }
        }
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            if (j > 0 && x0 + j * V >= n0) {
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    c[1 + j * V + k] = (T)0;
#pragma unroll
                    for (int a = 0; a < NDIM - 1; ++a) lo[a][j * V + k] = hi[a][j * V + k] = (T)0;
                }
                continue;
            }
            const long long bj = base + j * V;
            unpack<T>(*reinterpret_cast<const VT*>(psi + bj), c + 1 + j * V);
#pragma unroll
            for (int a = 1; a < NDIM; ++a) {
                const long long sl = ia[a] > 0 ? g.s[a] : 0, sh = ia[a] < g.n[a] - 1 ? g.s[a] : 0;
                unpack<T>(*reinterpret_cast<const VT*>(psi + bj - sl), lo[a - 1] + j * V);
                unpack<T>(*reinterpret_cast<const VT*>(psi + bj + sh), hi[a - 1] + j * V);
            }
        }
        c[0] = x0 > 0 ? psi[base - 1] : (T)0;
        c[CW + 1] = x0 + CW < n0 ? psi[base + CW] : (T)0;
        StencilAcc<T, NDIM> sa;
        T dot8 = (T)0;                                // this item's cells, then FP64
#pragma unroll
        for (int k = 0; k < CW; ++k) {
            if (m[k] == (T)0) continue;
            dot8 = fma(c[k + 1], m[k], dot8);
            T pos[3];
            pos[0] = axis_pos(c[k], c[k + 1], c[k + 2], x0 + k, n0, g.power, g.q[0]);
#pragma unroll
            for (int a = 1; a < NDIM; ++a)
                pos[a] = axis_pos(lo[a - 1][k], c[k + 1], hi[a - 1][k], ia[a], g.n[a], g.power, g.q[a]);
            if (SWAP) {
                const T p0 = pos[0];
                pos[0] = pos[1];
                pos[1] = p0;
                sa.add(rho, go, pos, m[k]);
            } else {
                sa.add(rho, g, pos, m[k]);
            }
        }
        sa.flush(rho, SWAP ? go : g);
        dsum += (double)dot8;
    }
    if (part) {
        __shared__ double red[32];
        const double sb = block_sum(dsum, red);
        if (threadIdx.x == 0) part[blockIdx.x] = sb;
    }
}

template <typename T, int NDIM>
__global__ void __launch_bounds__(256) pushforward_rows_kernel(const T* __restrict__ psi,
                                                               const T* __restrict__ mu,
                                                               T* __restrict__ rho, GridDev g,
                                                               int per_row, const int* done)
{
    pushforward_rows_body<T, NDIM, false>(psi, mu, rho, g, per_row, done, g, nullptr);
}

// the transposed form (three CTAs per SM in FP32: 80 registers, no spills)
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
pushforward_rows_t_kernel(const T* __restrict__ psi, const T* __restrict__ mu, T* __restrict__ rho,
                          GridDev g, int per_row, const int* done, GridDev go, double* part)
{
    pushforward_rows_body<T, 2, true>(psi, mu, rho, g, per_row, done, go, part);
}

// Batched pushforward: blockIdx.y selects the problem.
template <typename T>
struct PushArgs {
    const T* psi;
    const T* mu;
    T* rho;
    const int* done;
    GridDev g;
};

template <typename T>
__global__ void zero_batched_kernel(const PushArgs<T>* batch)
{
    const PushArgs<T>& a = batch[blockIdx.y];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.g.N; i += stride)
        a.rho[i] = (T)0;
}

template <typename T, int NDIM>
__global__ void pushforward_batched_kernel(const PushArgs<T>* batch)
{
    const PushArgs<T>& a = batch[blockIdx.y];
    if (a.done && *a.done) return;
    const GridDev& g = a.g;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        const T m = a.mu[idx];
        if (m == (T)0) continue;
        long long r = idx;
        T pos[3];
#pragma unroll
        for (int ax = 0; ax < NDIM; ++ax) {
            const int i = (int)(r % g.n[ax]);
            r /= g.n[ax];
            pos[ax] = map_pos(a.psi, idx, i, g.n[ax], g.s[ax], g.power, g.q[ax]);
        }
        deposit<T, NDIM>(a.rho, g, pos, m);
    }
}

size_t push_args_bytes(int elem_bytes) { return elem_bytes == 8 ? sizeof(PushArgs<double>) : sizeof(PushArgs<float>); }

template <typename T>
void fill_push_batch_args(const Grid& g, const T* psi, const T* mu, T* rho, const int* done, void* host_slot)
{
    PushArgs<T>* a = reinterpret_cast<PushArgs<T>*>(host_slot);
    a->psi = psi; a->mu = mu; a->rho = rho; a->done = done; a->g = dev_grid(g);
}

template <typename T>
bfm_status launch_pushforward_batched(int ndim, long long max_cells, int nprob, const void* dev_args,
                                      cudaStream_t st)
{
    const int th = 256, bl = grid_blocks(max_cells, th);
    const PushArgs<T>* b = reinterpret_cast<const PushArgs<T>*>(dev_args);
    zero_batched_kernel<T><<<dim3(bl, nprob), th, 0, st>>>(b);
    BFM_LAUNCH_CHECK("zero_batched_kernel");
    if (ndim == 2) pushforward_batched_kernel<T, 2><<<dim3(bl, nprob), th, 0, st>>>(b);
    else           pushforward_batched_kernel<T, 3><<<dim3(bl, nprob), th, 0, st>>>(b);
    BFM_LAUNCH_CHECK("pushforward_batched_kernel");
    return BFM_OK;
}

template void fill_push_batch_args<float>(const Grid&, const float*, const float*, float*, const int*, void*);
template void fill_push_batch_args<double>(const Grid&, const double*, const double*, double*, const int*, void*);
template bfm_status launch_pushforward_batched<float>(int, long long, int, const void*, cudaStream_t);
template bfm_status launch_pushforward_batched<double>(int, long long, int, const void*, cudaStream_t);

template <typename T, int NDIM>
__global__ void map_kernel(const T* __restrict__ psi, T* __restrict__ out, GridDev g)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        long long r = idx;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const int i = (int)(r % g.n[a]);
            r /= g.n[a];
            const T pos = map_pos(psi, idx, i, g.n[a], g.s[a], g.power, g.q[a]);
            out[a * g.N + idx] = (pos + (T)0.5) / (T)g.n[a];
        }
    }
}

template <typename T, int NDIM>
__global__ void interpolate_kernel(const T* __restrict__ map, const T* __restrict__ mu, T tt,
                                   T* __restrict__ rho, GridDev g)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        const T m = mu[idx];
        if (m == (T)0) continue;
        long long r = idx;
        T pos[3];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const int i = (int)(r % g.n[a]);
            r /= g.n[a];
            const T tpos = map[a * g.N + idx] * (T)g.n[a] - (T)0.5;   // T(x) in index units
            T p = (T)i + tt * (tpos - (T)i);
            p = fmin(fmax(p, (T)0), (T)(g.n[a] - 1));
            pos[a] = p;
        }
        deposit<T, NDIM>(rho, g, pos, m);
    }
}

template <typename T>
bfm_status launch_pushforward(const Grid& g, const T* psi, const T* mu, T* rho, const int* done,
                              cudaStream_t st, const double* p)
{
    BFM_CUDA(cudaMemsetAsync(rho, 0, sizeof(T) * g.N, st));
    const GridDev d = dev_grid(g, p);
    const int th = 256, bl = grid_blocks(g.N, th);
    const int CW = Vec16<T>::V * (g.ndim == 2 ? push_vecs<2>() : push_vecs<3>());
    const int per_row = (g.n[0] + CW - 1) / CW;                          // threads per row
    const long long items = (g.N / g.n[0]) * per_row;
    const bool rows = g.n[0] % 4 == 0 && aligned16(psi) && aligned16(mu) && aligned16(rho) &&
                      items < (1ll << 31);
    if (rows) {
        long long blr = (items + th - 1) / th;
        const long long cap = (long long)num_sms() * 8;
        if (blr > cap) blr = cap;
        if (g.ndim == 2) pushforward_rows_kernel<T, 2><<<(int)blr, th, 0, st>>>(psi, mu, rho, d, per_row, done);
        else             pushforward_rows_kernel<T, 3><<<(int)blr, th, 0, st>>>(psi, mu, rho, d, per_row, done);
        BFM_LAUNCH_CHECK("pushforward_rows_kernel");
        return BFM_OK;
    }
    if (g.ndim == 2) pushforward_kernel<T, 2><<<bl, th, 0, st>>>(psi, mu, rho, d, done);
    else             pushforward_kernel<T, 3><<<bl, th, 0, st>>>(psi, mu, rho, d, done);
    BFM_LAUNCH_CHECK("pushforward_kernel");
    return BFM_OK;
}

// The pushforward of a 2-D quadratic-cost step whose psi~ and mu are held
// in the transposed layout (gt = transposed_grid(g)): rho comes out in g's
// layout, and (part) the FP64 partials of <psi~, mu> per CTA, their number in
// *blocks_used.  Needs the row form's conditions (n % 4, 16-byte alignment).
template <typename T>
bfm_status launch_pushforward_t(const Grid& gt, const T* psi_t, const T* mu_t, T* rho,
                                const Grid& g, const int* done, cudaStream_t st, double* part,
                                int* blocks_used)
{
    const int th = 256;
    const int CW = Vec16<T>::V * push_vecs<2>();
    const int per_row = (gt.n[0] + CW - 1) / CW;
    const long long items = (gt.N / gt.n[0]) * per_row;
    if (gt.ndim != 2 || g.ndim != 2 || gt.n[0] != g.n[1] || gt.n[1] != g.n[0] || gt.n[0] % 4 != 0 ||
        !aligned16(psi_t) || !aligned16(mu_t) || !aligned16(rho) || items >= (1ll << 31)) {
        set_last_error("internal: transposed pushforward needs a 2-D grid, n % 4 == 0 and aligned fields");
        return BFM_ERR_INVALID_ARG;
    }
    BFM_CUDA(cudaMemsetAsync(rho, 0, sizeof(T) * g.N, st));
    const GridDev dt = dev_grid(gt), dg = dev_grid(g);
    long long blr = (items + th - 1) / th;
    const long long cap = (long long)num_sms() * 8;
    if (blr > cap) blr = cap;
    if (blr > kMaxPartials) blr = kMaxPartials;
    if (blr < 1) blr = 1;
    pushforward_rows_t_kernel<T><<<(int)blr, th, 0, st>>>(psi_t, mu_t, rho, dt, per_row, done, dg, part);
    BFM_LAUNCH_CHECK("pushforward_rows_t_kernel");
    if (blocks_used) *blocks_used = (int)blr;
    return BFM_OK;
}

template <typename T>
bfm_status launch_map(const Grid& g, const T* psi, T* map, cudaStream_t st, const double* p)
{
    const GridDev d = dev_grid(g, p);
    const int th = 256, bl = grid_blocks(g.N, th);
    if (g.ndim == 2) map_kernel<T, 2><<<bl, th, 0, st>>>(psi, map, d);
    else             map_kernel<T, 3><<<bl, th, 0, st>>>(psi, map, d);
    BFM_LAUNCH_CHECK("map_kernel");
    return BFM_OK;
}

template <typename T>
bfm_status launch_interpolate(const Grid& g, const T* map, const T* mu, double t, T* rho,
                              cudaStream_t st)
{
    BFM_CUDA(cudaMemsetAsync(rho, 0, sizeof(T) * g.N, st));
    const GridDev d = dev_grid(g);
    const int th = 256, bl = grid_blocks(g.N, th);
    if (g.ndim == 2) interpolate_kernel<T, 2><<<bl, th, 0, st>>>(map, mu, (T)t, rho, d);
    else             interpolate_kernel<T, 3><<<bl, th, 0, st>>>(map, mu, (T)t, rho, d);
    BFM_LAUNCH_CHECK("interpolate_kernel");
    return BFM_OK;
}

template bfm_status launch_pushforward<float>(const Grid&, const float*, const float*, float*,
                                              const int*, cudaStream_t, const double*);
template bfm_status launch_pushforward<double>(const Grid&, const double*, const double*, double*,
                                               const int*, cudaStream_t, const double*);
template bfm_status launch_pushforward_t<float>(const Grid&, const float*, const float*, float*,
                                                const Grid&, const int*, cudaStream_t, double*, int*);
template bfm_status launch_pushforward_t<double>(const Grid&, const double*, const double*, double*,
                                                 const Grid&, const int*, cudaStream_t, double*, int*);
template bfm_status launch_map<float>(const Grid&, const float*, float*, cudaStream_t, const double*);
template bfm_status launch_map<double>(const Grid&, const double*, double*, cudaStream_t, const double*);
template bfm_status launch_interpolate<float>(const Grid&, const float*, const float*, double,
                                              float*, cudaStream_t);
template bfm_status launch_interpolate<double>(const Grid&, const double*, const double*, double,
                                               double*, cudaStream_t);

}  // namespace bfm
