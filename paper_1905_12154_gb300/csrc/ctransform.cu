// ctransform.cu -- the grid c-transform for the quadratic cost (Section 4.1).
//
// phi^c(x) = min_y |x-y|^2/2 - phi(y) splits into 1-D passes along each axis
// (Section 4.1, dimension splitting): pass 1 takes f = -phi, later passes take
// the previous output.  A 1-D pass on a line of n cells computes
//     u(i) = min_j  hh (i - j)^2 + f(j),     hh = h^2 / 2,
// i.e. the lower envelope of n parabolas of equal curvature.  The paper
// evaluates it through the Legendre transform and a convex-hull sweep; here
// the same envelope is built in parallel inside one CTA per line tile:
//   A. each thread builds the envelope of its own K consecutive parabolas
//      with a stack (a parabola b between a and c is hidden when the a/b
//      crossing lies right of the b/c crossing);
//   B. neighbouring envelopes are merged pairwise in log2(G) rounds: two
//      envelopes whose parabolas are separated meet at one crossover, so the
//      merge keeps a prefix of the left one and a suffix of the right one,
//      found by popping hidden ends (the lower common tangent walk);
//   C. the surviving parabolas are compacted with a prefix sum;
//   D. each thread finds the parabola owning its first output cell by binary
//      search and sweeps its K outputs monotonically.
// The division-free hidden test compares second differences:
//   b hidden by (a, c)  <=>  (f_b-f_a)(c-b) - (f_c-f_b)(b-a) >= hh (c-a)(b-a)(c-b).
// Optional FP64 dot products of the input and of the output with weight
// fields (the two terms of the dual value J, eq. (defJ)) are fused into the
// load and store sweeps and written as one partial sum per CTA.
#include "common.cuh"
#include "kernels.h"

namespace bfm {

template <typename T>
struct CtArgs {
    const T* in;
    T* out;
    const T* w_in;        // optional: partial sums of in * w_in
    const T* w_out;       // optional: partial sums of out * w_out
    double* part_in;      // [gridDim.x]
    double* part_out;     // [gridDim.x]
    const int* done;      // optional: skip when *done != 0
    LineTiles lt;
    int G;                // threads per line (power of two)
    int LD;               // shared leading dimension of f (elements)
    int LDI;              // shared leading dimension of the index arrays
    T hh;                 // h^2 / 2 on this axis
    int negate;           // the pass reads -in
};

template <typename T>
__device__ __forceinline__ bool hidden(const T* f, int a, int b, int c, T hh)
{
    const T fa = f[a], fb = f[b], fc = f[c];
    const T lhs = (fb - fa) * (T)(c - b) - (fc - fb) * (T)(b - a);
    const T rhs = hh * (T)(c - a) * (T)(b - a) * (T)(c - b);
    return lhs >= rhs;
}

template <typename T>
__device__ __forceinline__ T parab(T hh, int x, int j, T fj)
{
    const int d = x - j;
    return fma(hh, (T)(d * d), fj);
}

// Phase B: merge the envelopes of thread groups [t, t+s) and [t+s, t+2s).
template <typename T>
__device__ void merge_pair(const T* f, const short* stk, short* beg, short* end,
                           int t, int s, int n, T hh)
{
    const int tl = t, tr = t + 2 * s;
    int lt = t + s - 1;
    while (lt >= tl && beg[lt] == end[lt]) --lt;
    int rt = t + s;
    while (rt < tr && beg[rt] == end[rt]) ++rt;
    if (lt < tl || rt >= tr) return;
    for (int guard = 0; guard <= n + 2; ++guard) {
        const int b = stk[end[lt] - 1];
        const int c = stk[beg[rt]];
        int a = -1;
        if (end[lt] - beg[lt] >= 2) {
            a = stk[end[lt] - 2];
        } else {
            int la = lt - 1;
            while (la >= tl && beg[la] == end[la]) --la;
            if (la >= tl) a = stk[end[la] - 1];
        }
        if (a >= 0 && hidden(f, a, b, c, hh)) {
            end[lt] = (short)(end[lt] - 1);
            while (lt >= tl && beg[lt] == end[lt]) --lt;
            if (lt < tl) return;
            continue;
        }
        int d = -1;
        if (end[rt] - beg[rt] >= 2) {
            d = stk[beg[rt] + 1];
        } else {
            int ra = rt + 1;
            while (ra < tr && beg[ra] == end[ra]) ++ra;
            if (ra < tr) d = stk[beg[ra]];
        }
        if (d >= 0 && hidden(f, b, c, d, hh)) {
            beg[rt] = (short)(beg[rt] + 1);
            while (rt < tr && beg[rt] == end[rt]) ++rt;
            if (rt >= tr) return;
            continue;
        }
        return;
    }
}

template <typename T, int K, bool CONTIG>
__global__ void __launch_bounds__(1024, 1) ct_pass_kernel(CtArgs<T> a)
{
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LineTiles& lt = a.lt;
    const int n = lt.n;
    const int G = a.G;
    const int W = lt.W;
    T* fs = reinterpret_cast<T*>(smem_raw);
    short* stk_all = reinterpret_cast<short*>(fs + (size_t)W * a.LD);
    short* hull_all = stk_all + (size_t)W * a.LDI;
    short* beg_all = hull_all + (size_t)W * a.LDI;
    short* end_all = beg_all + (size_t)W * G;
    int* wsum_all = reinterpret_cast<int*>(end_all + (size_t)W * G);   // 4-byte aligned
    const int nwl = (G + 31) / 32;                 // warps per line
    int* htot = wsum_all + W * nwl;
    __shared__ double red[32];

    const int tid = threadIdx.x;
    const int w = tid / G, t = tid - w * G;
    const int lane = tid & 31;
    T* f = fs + (size_t)w * a.LD;
    short* stk = stk_all + (size_t)w * a.LDI;
    short* hull = hull_all + (size_t)w * a.LDI;
    short* beg = beg_all + w * G;
    short* end = end_all + w * G;
    const T hh = a.hh;
    const int lo = t * K;
    const int hi = min(lo + K, n);

    double acc_in = 0.0, acc_out = 0.0;

    for (long long tile = blockIdx.x; tile < lt.ntiles; tile += gridDim.x) {
        const Tile tl = tile_at(lt, tile);
        const int total = tl.wact * n;
        // ---- load ----------------------------------------------------------
        for (int e = tid; e < total; e += blockDim.x) {
            int ww, p;
            if (CONTIG) { ww = e / n; p = e - ww * n; }
            else        { p = e / tl.wact; ww = e - p * tl.wact; }
            const long long ad = addr_of(lt, tl, ww, p);
            const T v = a.in[ad];
            fs[(size_t)ww * a.LD + p] = a.negate ? -v : v;
            if (a.w_in) acc_in += (double)v * (double)a.w_in[ad];
        }
        __syncthreads();
        const bool active = (w < tl.wact);
        // ---- A: envelope of this thread's chunk ------------------------------
        if (active) {
            if (lo < n) {
                int top = lo - 1;
                for (int q = lo; q < hi; ++q) {
                    while (top >= lo + 1 && hidden(f, (int)stk[top - 1], (int)stk[top], q, hh)) --top;
                    stk[++top] = (short)q;
                }
                beg[t] = (short)lo;
                end[t] = (short)(top + 1);
            } else {
                beg[t] = 0;
                end[t] = 0;
            }
        }
        __syncthreads();
        // ---- B: pairwise merges ------------------------------------------------
        for (int s = 1; s < G; s <<= 1) {
            if (active && (t & (2 * s - 1)) == 0 && t + s < G) merge_pair(f, stk, beg, end, t, s, n, hh);
            __syncthreads();
        }
        // ---- C: compaction -------------------------------------------------------
        const int cnt = active ? (end[t] - beg[t]) : 0;
        int incl = cnt;
        const int width = G < 32 ? G : 32;
        for (int d = 1; d < width; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d, width);
            if ((lane % width) >= d) incl += y;
        }
        if (G > 32) {
            if (active && (t & 31) == 31) wsum_all[w * nwl + (t >> 5)] = incl;
            __syncthreads();
            int add = 0;
            if (active)
                for (int i = 0; i < (t >> 5); ++i) add += wsum_all[w * nwl + i];
            incl += add;
        }
        if (active && t == G - 1) htot[w] = incl;
        if (active) {
            const int b0 = beg[t];
            const int excl = incl - cnt;
            for (int i = 0; i < cnt; ++i) hull[excl + i] = stk[b0 + i];
        }
        __syncthreads();
        // ---- D: evaluate this thread's outputs -----------------------------------
        T outv[K];
        if (active && lo < n) {
            const int H = htot[w];
            int kl = 0, kh = H - 1;
            while (kl < kh) {
                const int mid = (kl + kh) >> 1;
                const int j0 = hull[mid], j1 = hull[mid + 1];
                if (parab(hh, lo, j1, f[j1]) < parab(hh, lo, j0, f[j0])) kl = mid + 1;
                else kh = mid;
            }
            int k = kl;
            int jc = hull[k];
            T fc = f[jc];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int x = lo + q;
                if (x < hi) {
                    T vc = parab(hh, x, jc, fc);
                    while (k + 1 < H) {
                        const int jn = hull[k + 1];
                        const T fn = f[jn];
                        const T vn = parab(hh, x, jn, fn);
                        if (vn <= vc) { ++k; jc = jn; fc = fn; vc = vn; }
                        else break;
                    }
                    outv[q] = vc;
                }
            }
        }
        __syncthreads();
        if (active && lo < n) {
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (lo + q < hi) f[lo + q] = outv[q];
        }
        __syncthreads();
        // ---- store ---------------------------------------------------------------
        for (int e = tid; e < total; e += blockDim.x) {
            int ww, p;
            if (CONTIG) { ww = e / n; p = e - ww * n; }
            else        { p = e / tl.wact; ww = e - p * tl.wact; }
            const long long ad = addr_of(lt, tl, ww, p);
            const T v = fs[(size_t)ww * a.LD + p];
            a.out[ad] = v;
            if (a.w_out) acc_out += (double)v * (double)a.w_out[ad];
        }
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

int pick_K(int n)
{
    if (n <= 32) return 1;
    if (n <= 64) return 2;
    if (n <= 128) return 4;
    if (n <= 256) return 8;
    return 16;
}

// worst-case number of words one bank serves for a warp writing the W lines
// of consecutive positions (lane -> line lane % W, position lane / W)
int bank_conflicts(int LD, int W, int words)
{
    int cnt[32] = {0};
    for (int lane = 0; lane < 32; ++lane) {
        const int w = lane % W, p = lane / W;
        const long base = ((long)w * LD + p) * words;
        for (int k = 0; k < words; ++k) cnt[(base + k) % 32]++;
    }
    int m = 0;
    for (int b = 0; b < 32; ++b) m = cnt[b] > m ? cnt[b] : m;
    return m;
}

int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <typename T, int K>
void* kernel_for(bool contig)
{
    return contig ? (void*)ct_pass_kernel<T, K, true> : (void*)ct_pass_kernel<T, K, false>;
}

template <typename T>
void* select_kernel(int K, bool contig)
{
    switch (K) {
        case 1: return kernel_for<T, 1>(contig);
        case 2: return kernel_for<T, 2>(contig);
        case 4: return kernel_for<T, 4>(contig);
        case 8: return kernel_for<T, 8>(contig);
        default: return kernel_for<T, 16>(contig);
    }
}

}  // namespace

CtPlan plan_ct_pass(const Grid& g, int axis, int elem_bytes)
{
    CtPlan p;
    const int n = g.n[axis];
    p.K = pick_K(n);
    p.G = next_pow2((n + p.K - 1) / p.K);
    const bool contig = (axis == 0);
    const int LDI = n + (n & 1) + 8;
    // lines per CTA: at most 1024 threads, at most 32 lines, a shared-memory budget
    const size_t line_bytes = (size_t)(n + 32) * elem_bytes + 2 * (size_t)LDI * 2 + 2 * (size_t)p.G * 2 + 64;
    int W = 1024 / p.G;
    if (W < 1) W = 1;
    if (W > 32) W = 32;
    const size_t budget = 200 * 1024;
    while (W > 1 && (size_t)W * line_bytes > budget) --W;
    if (!contig && W > g.n[0]) W = g.n[0];
    // leading dimension: for interleaved loads consecutive lanes hit the W lines
    // of one position; pick the stride with the fewest shared-memory bank conflicts
    int LD = n;
    if (!contig) {
        int best = 1 << 30;
        for (int cand = n; cand <= n + 32; ++cand) {
            const int c = bank_conflicts(cand, W, elem_bytes / 4);
            if (c < best) { best = c; LD = cand; }
        }
    }
    p.W = W;
    p.LD = LD;
    p.LDI = LDI;
    const int nwl = (p.G + 31) / 32;
    p.smem = (size_t)W * LD * elem_bytes + 2 * (size_t)W * LDI * 2 + 2 * (size_t)W * p.G * 2 +
             (size_t)W * nwl * 4 + (size_t)W * 4 + 16;
    p.threads = ((W * p.G + 31) / 32) * 32;
    p.tiles = make_tiles(g, axis, W);
    return p;
}

template <typename T>
bfm_status launch_ct_pass(const Grid& g, int axis, const T* in, T* out, bool negate,
                          const T* w_in, double* part_in, const T* w_out, double* part_out,
                          const int* done, int max_blocks, cudaStream_t st, int* blocks_used)
{
    CtPlan p = plan_ct_pass(g, axis, (int)sizeof(T));
    CtArgs<T> a;
    a.in = in; a.out = out; a.w_in = w_in; a.w_out = w_out;
    a.part_in = part_in; a.part_out = part_out; a.done = done;
    a.lt = p.tiles; a.G = p.G; a.LD = p.LD; a.LDI = p.LDI;
    const double h = 1.0 / g.n[axis];
    a.hh = (T)(0.5 * h * h);
    a.negate = negate ? 1 : 0;
    void* k = select_kernel<T>(p.K, axis == 0);
    BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    long long blocks = p.tiles.ntiles;
    const long long cap = (long long)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    void* args[] = {&a};
    BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(p.threads), args, p.smem, st));
    if (blocks_used) *blocks_used = (int)blocks;
    return BFM_OK;
}

template bfm_status launch_ct_pass<float>(const Grid&, int, const float*, float*, bool, const float*,
                                          double*, const float*, double*, const int*, int,
                                          cudaStream_t, int*);
template bfm_status launch_ct_pass<double>(const Grid&, int, const double*, double*, bool,
                                           const double*, double*, const double*, double*,
                                           const int*, int, cudaStream_t, int*);

}  // namespace bfm
