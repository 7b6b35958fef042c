// autotune.cu -- launch shapes of the line c-transform chosen by timing.
//
// The c-transform of Section 4.1 is computed line by line; how many cells a
// thread takes (K) and how many lines share a CTA (W) trade the sequential
// stack work of a thread against the parallel join of the chunks and the
// occupancy of an SM, and the best trade depends on the line length.  The
// tuner times every candidate shape of one kernel kind and line length on a
// synthetic field (CUDA events, median of five launches after two untimed
// ones) and stores the fastest in the library's shape table, which every
// later plan of that kind and length reads (ctransform.cu).  Selection keeps
// the hand-picked default unless a candidate beats it by a margin, so noise
// does not flip shapes between runs.
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace bfm {

// The timing field: phi(x) = 0.45 (x - c)^2 + a sin(2 pi (4 x + 0.37 l)) along
// line l, x the cell centre along the line.  The pass works on -phi, whose
// lifted points hh j^2 - phi_j have curvature 0.1 plus the sine's, so each
// line is convex on part of its length and loses points to the envelope
// elsewhere, as the potentials of a solve do.  As in a solve, an axis-0 pass
// negates on load and passes along other axes do not: those get -phi stored.
template <typename T>
__global__ void tune_field_kernel(T* f, int n, long long nlines, int axis_stride_is_one,
                                  long long n0, double sign)
{
    const long long N = (long long)n * nlines;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        long long k, l;                    // position along the line, line index
        if (axis_stride_is_one) { k = i % n; l = i / n; }
        else { k = (i / n0) % n; l = i % n0 + n0 * (i / (n0 * n)); }
        const double x = (k + 0.5) / n;
        const double v = 0.45 * (x - 0.4) * (x - 0.4) +
                         1e-3 * sinpi(2.0 * (4.0 * x + 0.37 * (double)l));
        f[i] = (T)(sign * v);
    }
}

// The timing grid: lines of n cells along the kernel kind's axis, about 8 M
// cells in all (at least two lines), split over a third axis where one axis
// would exceed the longest supported line.
static bool tune_grid(int kind, int n, int elem_bytes, Grid* g, int* axis)
{
    const long long L = std::max<long long>(2, (8LL << 20) / n);
    bfm_grid bg;
    if (kind == CT_KIND_TILE_COLS || kind == CT_KIND_ROW_COLS) {
        const long long a = std::min<long long>(L, 2048), b = L / a;
        bg.n[0] = (int)a; bg.n[1] = n; bg.n[2] = (int)b;
        *axis = 1;
    } else {
        const long long a = std::min<long long>(L, 8192), b = L / a;
        bg.n[0] = n; bg.n[1] = (int)a; bg.n[2] = (int)b;
        *axis = 0;
    }
    bg.ndim = bg.n[2] >= 2 ? 3 : 2;
    if (!make_grid(&bg, g)) return false;
    return ct_kind(*g, *axis, elem_bytes) == kind;
}

}  // namespace bfm

using namespace bfm;

extern "C" int bfm_tune_candidates(int kind, int n, bfm_precision prec, int* K, int* W, int cap)
{
    if (kind < CT_KIND_TILE_ROWS || kind > CT_KIND_ROW_COLS || n < 2 || cap < 0) return -1;
    std::vector<CtShape> c(64);
    const int m = ct_shape_candidates(kind, n, prec == BFM_FP64 ? 8 : 4, c.data(), 64);
    for (int i = 0; i < m && i < cap; ++i) {
        if (K) K[i] = c[i].K;
        if (W) W[i] = c[i].W;
    }
    return m;
}

extern "C" int bfm_tune_default(int kind, int n, bfm_precision prec, int* K, int* W)
{
    if (kind < CT_KIND_TILE_ROWS || kind > CT_KIND_ROW_COLS || n < 2) return -1;
    const CtShape s = ct_default_shape(kind, n, prec == BFM_FP64 ? 8 : 4);
    if (K) *K = s.K;
    if (W) *W = s.W;
    return 0;
}

extern "C" bfm_status bfm_tune_set(int kind, int n, bfm_precision prec, int K, int W)
{
    const int eb = prec == BFM_FP64 ? 8 : 4;
    if (kind < CT_KIND_TILE_ROWS || kind > CT_KIND_ROW_COLS || !ct_shape_valid(kind, n, eb, CtShape{K, W})) {
        set_last_error("bfm_tune_set: not a candidate shape of this kernel kind and line length");
        return BFM_ERR_INVALID_ARG;
    }
    ct_set_tuned_shape(kind, n, eb, CtShape{K, W});
    return BFM_OK;
}

extern "C" int bfm_tune_get(int kind, int n, bfm_precision prec, int* K, int* W)
{
    const int eb = prec == BFM_FP64 ? 8 : 4;
    CtShape s;
    const bool tuned = ct_tuned_shape(kind, n, eb, &s);
    if (!tuned) s = ct_default_shape(kind, n, eb);
    if (K) *K = s.K;
    if (W) *W = s.W;
    return tuned ? 1 : 0;
}

extern "C" void bfm_tune_clear(void) { ct_clear_tuned_shapes(); }

extern "C" int bfm_tune_pick(const double* ms, int ncand, int default_index, double margin)
{
    if (!ms || ncand <= 0) return -1;
    int best = -1;
    for (int i = 0; i < ncand; ++i)
        if (ms[i] > 0.0 && (best < 0 || ms[i] < ms[best])) best = i;
    if (best < 0) return default_index;
    if (default_index >= 0 && default_index < ncand && ms[default_index] > 0.0 &&
        ms[best] * (1.0 + margin) >= ms[default_index])
        return default_index;
    return best;
}

extern "C" size_t bfm_autotune_scratch_bytes(int kind, int n, bfm_precision prec)
{
    Grid g;
    int axis = 0;
    const int eb = prec == BFM_FP64 ? 8 : 4;
    if (kind < CT_KIND_TILE_ROWS || kind > CT_KIND_ROW_COLS || n < 2 || !tune_grid(kind, n, eb, &g, &axis))
        return 0;
    return 2 * (size_t)g.N * (size_t)eb + 256;
}

template <typename T>
static bfm_status autotune_impl(int kind, int n, void* scratch, size_t bytes, cudaStream_t st,
                                int* K_out, int* W_out, double* ms_out, int ms_cap)
{
    Grid g;
    int axis = 0;
    if (!tune_grid(kind, n, (int)sizeof(T), &g, &axis)) {
        set_last_error("bfm_autotune: this line length does not take this kernel kind");
        return BFM_ERR_INVALID_ARG;
    }
    const int eb = (int)sizeof(T);
    if (bytes < 2 * (size_t)g.N * sizeof(T) || !scratch ||
        (reinterpret_cast<uintptr_t>(scratch) & 255u)) {
        set_last_error("bfm_autotune: scratch smaller than bfm_autotune_scratch_bytes or not 256-byte aligned");
        return BFM_ERR_WORKSPACE;
    }
    T* in = reinterpret_cast<T*>(scratch);
    T* out = in + g.N;
    tune_field_kernel<T><<<num_sms() * 4, 256, 0, st>>>(in, n, g.N / n, axis == 0 ? 1 : 0, g.n[0],
                                                         axis == 0 ? 1.0 : -1.0);
    BFM_LAUNCH_CHECK("tune_field_kernel");
    // as in a solve: the first pass (axis 0) reads -phi, later passes the
    // previous pass's output
    const bool negate = axis == 0;
    std::vector<CtShape> cand(64);
    const int m = std::min(ct_shape_candidates(kind, n, eb, cand.data(), 64), 64);
    const CtShape def = ct_default_shape(kind, n, eb);
    CtShape prev;
    const bool had = ct_tuned_shape(kind, n, eb, &prev);
    int def_idx = -1;
    std::vector<double> ms(m, -1.0);
    cudaEvent_t ev[2];
    for (cudaEvent_t& e : ev) BFM_CUDA(cudaEventCreate(&e));
    bfm_status s = BFM_OK;
    for (int c = 0; c < m && s == BFM_OK; ++c) {
        if (cand[c].K == def.K && cand[c].W == def.W) def_idx = c;
        ct_set_tuned_shape(kind, n, eb, cand[c]);
        for (int r = 0; r < 2 && s == BFM_OK; ++r)
            s = launch_ct_pass<T>(g, axis, in, out, negate, nullptr, nullptr, nullptr, nullptr,
                                  nullptr, 0, st, nullptr);
        double t[5];
        for (int r = 0; r < 5 && s == BFM_OK; ++r) {
            cudaEventRecord(ev[0], st);
            s = launch_ct_pass<T>(g, axis, in, out, negate, nullptr, nullptr, nullptr, nullptr,
                                  nullptr, 0, st, nullptr);
            cudaEventRecord(ev[1], st);
            cudaError_t e = cudaEventSynchronize(ev[1]);
            float f = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&f, ev[0], ev[1]);
            if (e != cudaSuccess && s == BFM_OK) s = cuda_status(e, "bfm_autotune timing");
            t[r] = f;
        }
        if (s == BFM_OK) {
            std::sort(t, t + 5);
            ms[c] = t[2];
        }
    }
    for (cudaEvent_t& e : ev) cudaEventDestroy(e);
    if (s != BFM_OK) {
        if (had) ct_set_tuned_shape(kind, n, eb, prev);
        else ct_erase_tuned_shape(kind, n, eb);
        return s;
    }
    const int pick = bfm_tune_pick(ms.data(), m, def_idx, 0.02);
    const CtShape win = pick >= 0 ? cand[pick] : def;
    ct_set_tuned_shape(kind, n, eb, win);
    if (K_out) *K_out = win.K;
    if (W_out) *W_out = win.W;
    if (ms_out)
        for (int c = 0; c < m && c < ms_cap; ++c) ms_out[c] = ms[c];
    return BFM_OK;
}

extern "C" bfm_status bfm_autotune(int kind, int n, bfm_precision prec, void* scratch,
                                   size_t scratch_bytes, void* stream, int* K_out, int* W_out,
                                   double* ms_out, int ms_cap)
{
    if (kind < CT_KIND_TILE_ROWS || kind > CT_KIND_ROW_COLS || n < 2) {
        set_last_error("bfm_autotune: unknown kernel kind or line length below 2");
        return BFM_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return prec == BFM_FP64
        ? autotune_impl<double>(kind, n, scratch, scratch_bytes, st, K_out, W_out, ms_out, ms_cap)
        : autotune_impl<float>(kind, n, scratch, scratch_bytes, st, K_out, W_out, ms_out, ms_cap);
}

extern "C" int bfm_tune_passes(const bfm_grid* grid, bfm_precision prec, int batched, int* kinds,
                               int* ns, int cap)
{
    Grid g;
    if (!make_grid(grid, &g)) return -1;
    const int eb = prec == BFM_FP64 ? 8 : 4;
    int kk[6], nn[6], m = 0;
    auto add = [&](int kind, int n) {
        for (int i = 0; i < m; ++i)
            if (kk[i] == kind && nn[i] == n) return;
        kk[m] = kind; nn[m] = n; ++m;
    };
    if (!batched && g.ndim == 2 && transposed_axis1(g, eb)) {
        // long columns: both axes are swept as rows (of the grid or of its transposed copy)
        add(ct_kind(g, 0, eb), g.n[0]);
        const Grid gt = transposed_grid(g);
        add(ct_kind(gt, 0, eb), gt.n[0]);
    } else {
        for (int a = 0; a < g.ndim; ++a) add(ct_kind(g, a, eb), g.n[a]);
    }
    for (int i = 0; i < m && i < cap; ++i) {
        if (kinds) kinds[i] = kk[i];
        if (ns) ns[i] = nn[i];
    }
    return m;
}
