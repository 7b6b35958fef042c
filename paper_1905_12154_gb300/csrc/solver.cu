// solver.cu -- Algorithm 1 (the back-and-forth method) on one GPU, and the
// library's C ABI.
//
// Per iteration n (Algorithm 1; 4 c-transforms and 2 Poisson solves, the
// operation count of Section 4.3):
//   phi-half: psi~ = phi^c and J(phi) = <phi,nu> + <psi~,mu> (eq. (defJ));
//             rho = T#mu with T = x - grad psi~ (Lemma 2.2(ii), Lemma 3.1);
//             g = (-Delta)^{-1}(nu - rho) and G = ||g||^2 (eq. (gradients_J_I));
//             residual r_n = sqrt(G / ||nu - 1||^2_{H^-1}); stop if r_n < tol;
//             phi += sigma g; psi = phi^c; step rule on J(phi_{n+1/2}) - J(phi_n).
//   psi-half: the same with mu <-> nu, phi <-> psi and I (eq. (defI)).
// The step rule (Section 4.2, no backtracking): gain < beta1 sigma G shrinks
// sigma by alpha2 (not below sigma_min), gain > beta2 sigma G grows it by
// alpha1.  One sigma is shared by both half steps.
//
// Every scalar decision (dual values, residual, step rule, convergence) is
// taken on the device by one-block FP64 kernels, so the host only enqueues
// launches and reads the `done` flag every few iterations.  Fields are FP32
// or FP64; all reductions are FP64 and deterministic for a fixed grid.
#include <string.h>
#include <math.h>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "kernels.h"
#include "state.cuh"

namespace bfm {

// ---------------------------------------------------------------------------
// small FP64 kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void stats_kernel(const T* __restrict__ x, long long N, double* psum, double* pmax,
                             double* pmin, double* pbad)
{
    __shared__ double red[32];
    double s = 0.0, mx = -1.0e300, mn = 1.0e300, bad = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double v = (double)x[i];
        if (!isfinite(v)) bad += 1.0;
        else { s += v; mx = fmax(mx, v); mn = fmin(mn, v); }
    }
    const double ts = block_sum(s, red);
    const double tb = block_sum(bad, red);
    const double tmx = block_max(mx, red);
    const double tmn = -block_max(-mn, red);
    if (threadIdx.x == 0) {
        psum[blockIdx.x] = ts; pmax[blockIdx.x] = tmx; pmin[blockIdx.x] = tmn; pbad[blockIdx.x] = tb;
    }
}

__global__ void stats_finalize_kernel(SolverState* st, const double* psum, const double* pmax,
                                      const double* pmin, const double* pbad, int nb, double hd,
                                      int which)
{
    __shared__ double red[32];
    const double s = block_sum_parts(psum, nb, red);
    const double b = block_sum_parts(pbad, nb, red);
    double mx = -1.0e300, mn = 1.0e300;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) { mx = fmax(mx, pmax[i]); mn = fmin(mn, pmin[i]); }
    mx = block_max(mx, red);
    mn = -block_max(-mn, red);
    if (threadIdx.x == 0) {
        const double mass = s * hd;
        if (which == 0) { st->mass_mu = mass; st->max_mu = mx; st->min_mu = mn; st->bad_mu = b > 0; }
        else            { st->mass_nu = mass; st->max_nu = mx; st->min_nu = mn; st->bad_nu = b > 0; }
    }
}

template <typename T>
__global__ void scale_kernel(const T* __restrict__ in, T* __restrict__ out, long long N,
                             const SolverState* st, int which)
{
    const double m = which == 0 ? st->mass_mu : st->mass_nu;
    const T inv = (T)(1.0 / m);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = in[i] * inv;
}

__global__ void init_state_kernel(SolverState* st, double sigma0, double tol, int max_iter,
                                  double b1, double b2, double a1, double a2, double smin,
                                  int power, double p0, double p1, double p2)
{
    if (threadIdx.x != 0) return;
    st->power = power;
    st->cost_p[0] = p0; st->cost_p[1] = p1; st->cost_p[2] = p2;
    const double mxm = st->max_mu / st->mass_mu, mxn = st->max_nu / st->mass_nu;
    st->max_mu = mxm;
    st->max_nu = mxn;
    st->sigma = sigma0 > 0.0 ? sigma0 : 8.0 * fmin(1.0 / mxm, 1.0 / mxn);
    st->tol = tol;
    st->max_iter = max_iter;
    st->beta1 = b1; st->beta2 = b2; st->alpha1 = a1; st->alpha2 = a2; st->sigma_min = smin;
    st->iter = 0;
    st->done = 0;
    st->row_ctr[0] = 0;
    st->row_ctr[1] = 0;
    st->converged = 0;
    st->nonfinite = 0;
    st->pend = 0;
    st->J_old = 0.0;
    st->G = 0.0;
    st->last_resid = 0.0;
}

__global__ void finalize_dual_kernel(SolverState* st, const double* pin, int nin,
                                     const double* pout, int nout, double hd, int mode, Logs logs)
{
    if (st->done) return;
    __shared__ double red[32];
    const double a = block_sum_parts(pin, nin, red);
    const double b = block_sum_parts(pout, nout, red);
    if (threadIdx.x == 0) finalize_dual_body(st, hd * (a + b), mode, logs);
}

// Flipped layout (half_step_flipped): the c-transform that ends a half step
// leaves its output's dot out, because the next half step's first sweep
// reads that field with the same weight.  At the start of a half step the
// sums of that sweep (pin) complete the previous half step's dual value
// (with pprev, the dot of that half step's updated potential), whose step
// rule runs first (mode 1 or 3), then the measurement of this one (pin + pout,
// mode 0 or 2).  The first half step of a solve has nothing pending.
__global__ void finalize_dual_pend_kernel(SolverState* st, const double* pprev, int nprev,
                                          const double* pin, int nin, const double* pout, int nout,
                                          double hd, int mode, Logs logs)
{
    if (st->done) return;
    __shared__ double red[96];
    double a = thread_sum_parts(pin, nin);
    double b = thread_sum_parts(pout, nout);
    double c = st->pend ? thread_sum_parts(pprev, nprev) : 0.0;
    block_sum3(a, b, c, red);
    if (threadIdx.x == 0) {
        if (st->pend) finalize_dual_body(st, hd * (c + a), mode == 0 ? 3 : 1, logs);
        if (!st->done) finalize_dual_body(st, hd * (a + b), mode, logs);
        st->pend = 1;
    }
}

__global__ void finalize_G_kernel(SolverState* st, const double* part, int np, int mode, Logs logs)
{
    if (mode != 2 && st->done) return;
    __shared__ double red[32];
    const double G = block_sum_parts(part, np, red);
    if (threadIdx.x == 0) finalize_G_body(st, G, mode, logs);
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

size_t tables_bytes(const Grid& g, int eb)
{
    size_t b = 0;
    for (int a = 0; a < g.ndim; ++a) b += axis_table_bytes(g.n[a], eb);
    return b;
}

size_t poisson_bytes(const Grid& g, int eb)
{
    return up256(sizeof(SolverState)) + up256(sizeof(double) * kPartialSlots * kMaxPartials) +
           tables_bytes(g, eb);
}

size_t solve_bytes(const Grid& g, int eb, int max_iter)
{
    return poisson_bytes(g, eb) + up256(sizeof(double) * 3 * ((size_t)max_iter + 1)) +
           (transposed_axis1(g, eb) ? 7 : 4) * up256((size_t)eb * g.N);
}

void carve(const Grid& g, int eb, int max_iter, unsigned char* base, Workspace* w, bool fields)
{
    unsigned char* p = base;
    w->state = reinterpret_cast<SolverState*>(p); p += up256(sizeof(SolverState));
    w->parts = reinterpret_cast<double*>(p); p += up256(sizeof(double) * kPartialSlots * kMaxPartials);
    w->tables = p;
    for (int a = 0; a < g.ndim; ++a) {
        // every view of the workspace rebuilds the same table pointers; sizes
        // were validated (2^p 3^q) before any workspace is carved
        if (!layout_axis_tables(g.n[a], eb, p, &w->tabs[a])) memset(&w->tabs[a], 0, sizeof(AxisTables));
        p += axis_table_bytes(g.n[a], eb);
    }
    if (fields) {
        w->logs = reinterpret_cast<double*>(p); p += up256(sizeof(double) * 3 * ((size_t)max_iter + 1));
        w->mu_n = p; p += up256((size_t)eb * g.N);
        w->nu_n = p; p += up256((size_t)eb * g.N);
        w->tmp = p;  p += up256((size_t)eb * g.N);
        w->rho = p;  p += up256((size_t)eb * g.N);
        w->xt = w->mu_t = w->nu_t = nullptr;
        if (transposed_axis1(g, eb)) {
            w->xt = p;   p += up256((size_t)eb * g.N);
            w->mu_t = p; p += up256((size_t)eb * g.N);
            w->nu_t = p; p += up256((size_t)eb * g.N);
        }
    } else {
        w->logs = nullptr;
        w->mu_n = w->nu_n = w->tmp = w->rho = w->xt = w->mu_t = w->nu_t = nullptr;
    }
    w->bytes = (size_t)(p - base);
}

template <typename T>
bfm_status fill_tables(const Grid& g, Workspace* w, cudaStream_t st)
{
    for (int a = 0; a < g.ndim; ++a) {
        // axes of equal length still get their own copy: simple and tiny
        bfm_status s = fill_axis_tables<T>(g.n[a], &w->tabs[a],
                                           reinterpret_cast<unsigned char*>(w->tabs[a].tw), st);
        if (s != BFM_OK) return s;
    }
    return BFM_OK;
}

bool fft_sizes_ok(const Grid& g)
{
    FftRadices rs;
    for (int a = 0; a < g.ndim; ++a)
        if (!fft_radices(g.n[a], &rs)) return false;
    return true;
}

double* slot(Workspace* w, int s) { return w->parts + (size_t)s * kMaxPartials; }

// ---------------------------------------------------------------------------
// optional per-launch timing (bfm_profile_begin / bfm_profile_end)
// ---------------------------------------------------------------------------
enum {
    PK_CT0 = 0, PK_CT1, PK_CT2, PK_DCT_FWD, PK_DCT_MID, PK_DCT_INV, PK_PUSH, PK_SMALL,
    PK_TRANSPOSE, PK_COUNT
};
static const char* kProfNames[PK_COUNT] = {
    "ct_pass_axis0", "ct_pass_axis1", "ct_pass_axis2", "dct_fwd", "dct_mid", "dct_inv",
    "pushforward", "reduce_step", "transpose"};

struct ProfRec { int kind; int launches; cudaEvent_t a, b; };
struct Profiler {
    bool on = false;
    int cap = 0, used = 0, dropped = 0;
    ProfRec* rec = nullptr;
};
static thread_local Profiler g_prof;

// Each kernel group also opens an NVTX range named like its profiler kind (a
// no-op unless a tool is attached; inside a stream capture the range marks
// the enqueue, not the replay).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct ProfScope {
    ProfRec* r = nullptr;
    cudaStream_t st;
    NvtxRange nv;
    ProfScope(int kind, int launches, cudaStream_t s) : st(s), nv(kProfNames[kind])
    {
        if (!g_prof.on) return;
        if (g_prof.used >= g_prof.cap) { g_prof.dropped++; return; }
        r = &g_prof.rec[g_prof.used++];
        r->kind = kind;
        r->launches = launches;
        cudaEventRecord(r->a, st);
    }
    ~ProfScope() { if (r) cudaEventRecord(r->b, st); }
};

// ---------------------------------------------------------------------------
// the pieces of one half step
// ---------------------------------------------------------------------------
template <typename T>
static bfm_status transpose(const Grid& g, bool forward, const T* in, T* out, const T* w,
                            double* part, int* n_part, const int* done, cudaStream_t st)
{
    ProfScope ps(PK_TRANSPOSE, 1, st);
    // forward: the n1 rows of n0 cells become n0 rows of n1 cells
    const int R = forward ? g.n[1] : g.n[0], C = forward ? g.n[0] : g.n[1];
    return launch_transpose<T>(in, out, R, C, w, part, done, st, n_part);
}

// c-transform out = src^c with the two dot products of the dual value.  With
// xt (2-D, long columns) the axis-1 sweep runs along the rows of a transposed
// copy and the dot product of the output is taken on the way back.
template <typename T>
static bfm_status ct_with_dots(const Grid& g, const T* src, T* out, const T* w_src, const T* w_out,
                               double* p_in, int* n_in, double* p_out, int* n_out, const int* done,
                               cudaStream_t st, T* xt, const double* pc, int* row_ctr)
{
    if (pc) {
        // separable power cost: every axis by the divide-and-conquer pass (columns
        // as interleaved tiles; a tile is read whole before it is written)
        for (int a = 0; a < g.ndim; ++a) {
            const bool first = (a == 0), last = (a == g.ndim - 1);
            int used = 0;
            ProfScope ps(PK_CT0 + a, 1, st);
            bfm_status s = launch_ct_power_pass<T>(g, a, pc[a], first ? src : out, out, first,
                                                   first ? w_src : nullptr, first ? p_in : nullptr,
                                                   last ? w_out : nullptr, last ? p_out : nullptr,
                                                   done, kMaxPartials, st, &used);
            if (s != BFM_OK) return s;
            if (first) *n_in = used;
            if (last) *n_out = used;
        }
        return BFM_OK;
    }
    if (xt) {
        bfm_status s;
        {
            ProfScope ps(PK_CT0, 1, st);
            s = launch_ct_pass<T>(g, 0, src, out, true, w_src, p_in, nullptr, nullptr, done,
                                  kMaxPartials, st, n_in, row_ctr);
            if (s != BFM_OK) return s;
        }
        s = transpose<T>(g, true, out, xt, nullptr, nullptr, nullptr, done, st);
        if (s != BFM_OK) return s;
        {
            ProfScope ps(PK_CT1, 1, st);
            s = launch_ct_pass<T>(transposed_grid(g), 0, xt, xt, false, nullptr, nullptr, nullptr,
                                  nullptr, done, kMaxPartials, st, nullptr, row_ctr);
            if (s != BFM_OK) return s;
        }
        return transpose<T>(g, false, xt, out, w_out, p_out, n_out, done, st);
    }
    for (int a = 0; a < g.ndim; ++a) {
        const bool first = (a == 0), last = (a == g.ndim - 1);
        int used = 0;
        ProfScope ps(PK_CT0 + a, 1, st);
        bfm_status s = launch_ct_pass<T>(g, a, first ? src : out, out, first,
                                         first ? w_src : nullptr, first ? p_in : nullptr,
                                         last ? w_out : nullptr, last ? p_out : nullptr, done,
                                         kMaxPartials, st, &used, row_ctr);
        if (s != BFM_OK) return s;
        if (first) *n_in = used;
        if (last) *n_out = used;
    }
    return BFM_OK;
}

// c-transform out = src^c that leaves its output transposed: the sweep along
// the rows of src (with the dot of src and w_src on load), one transpose,
// then the sweep along the rows of the transposed field in place.  2-D
// quadratic cost only; one transpose instead of the two of ct_with_dots.  The
// dot of the output is taken by the kernel that reads it next (a sweep, or
// the pushforward).
template <typename T>
static bfm_status ct_flip(const Grid& g, const T* src, T* out, const T* w_src, double* p_in,
                          int* n_in, const int* done, cudaStream_t st, T* scratch, int* row_ctr)
{
    bfm_status s;
    {
        ProfScope ps(PK_CT0, 1, st);
        s = launch_ct_pass<T>(g, 0, src, scratch, true, w_src, p_in, nullptr, nullptr, done,
                              kMaxPartials, st, n_in, row_ctr);
        if (s != BFM_OK) return s;
    }
    s = transpose<T>(g, true, scratch, out, nullptr, nullptr, nullptr, done, st);
    if (s != BFM_OK) return s;
    ProfScope ps(PK_CT1, 1, st);
    return launch_ct_pass<T>(transposed_grid(g), 0, out, out, false, nullptr, nullptr, nullptr,
                             nullptr, done, kMaxPartials, st, nullptr, row_ctr);
}

// Forward transforms of f = base - in up to (and including) the middle pass;
// the spectrum of g stays in `buf`.  G partials go to p_g.
// With xt (2-D, long columns) the middle pass runs along the rows of a
// transposed copy.
template <typename T>
static bfm_status poisson_forward(const Grid& g, const AxisTables* tabs, const T* in,
                                  const T* base, T* buf, double* p_g, int* n_g, const int* done,
                                  cudaStream_t st, T* xt)
{
    if (xt) {
        bfm_status s;
        {
            ProfScope ps(PK_DCT_FWD, 1, st);
            s = launch_dct_pass<T>(g, 0, PASS_FWD, tabs, in, base, buf, nullptr, nullptr, nullptr,
                                   done, st, nullptr);
            if (s != BFM_OK) return s;
        }
        s = transpose<T>(g, true, buf, xt, nullptr, nullptr, nullptr, done, st);
        if (s != BFM_OK) return s;
        {
            ProfScope ps(PK_DCT_MID, 1, st);
            const AxisTables swapped[3] = {tabs[1], tabs[0], tabs[2]};
            s = launch_dct_pass<T>(transposed_grid(g), 0, PASS_MID, swapped, xt, nullptr, xt,
                                   nullptr, nullptr, p_g, done, st, n_g);
            if (s != BFM_OK) return s;
        }
        return transpose<T>(g, false, xt, buf, nullptr, nullptr, nullptr, done, st);
    }
    const int last = g.ndim - 1;
    for (int a = 0; a < last; ++a) {
        ProfScope ps(PK_DCT_FWD, 1, st);
        bfm_status s = launch_dct_pass<T>(g, a, PASS_FWD, tabs, a == 0 ? in : buf,
                                          a == 0 ? base : nullptr, buf, nullptr, nullptr, nullptr,
                                          done, st, nullptr);
        if (s != BFM_OK) return s;
    }
    ProfScope ps(PK_DCT_MID, 1, st);
    return launch_dct_pass<T>(g, last, PASS_MID, tabs, buf, nullptr, buf, nullptr, nullptr, p_g,
                              done, st, n_g);
}

// Inverse transforms of the remaining axes; the last one writes
// out = upd + sigma * g (or out = g when upd is NULL).
template <typename T>
static bfm_status poisson_inverse(const Grid& g, const AxisTables* tabs, T* buf, T* out,
                                  const T* upd, const double* sigma, const int* done,
                                  cudaStream_t st)
{
    for (int a = g.ndim - 2; a >= 0; --a) {
        const bool final_ = (a == 0);
        ProfScope ps(PK_DCT_INV, 1, st);
        bfm_status s = launch_dct_pass<T>(g, a, PASS_INV, tabs, buf, nullptr, final_ ? out : buf,
                                          final_ ? upd : nullptr, sigma, nullptr, done, st, nullptr);
        if (s != BFM_OK) return s;
    }
    return BFM_OK;
}

// one CTA sums the FP64 partials of a half step's reductions (up to a few
// thousand: one per CTA of the launch that produced them)
constexpr int kFinThreads = 256;

// The half step on 2-D grids with long columns (quadratic cost): phi is kept
// in the grid's layout and psi in the transposed one, so the c-transforms
// phi -> psi and psi -> phi each leave their output transposed (ct_flip, one
// transpose) and the psi-half runs on the transposed grid with the
// transposed copies of mu and nu.  The c-transform psi~ before the Poisson
// solve leaves its output transposed too, where the pushforward reads it and
// deposits rho in the potential's layout (the layout the Poisson solve and
// the update share); rows that are not a multiple of 4 cells take the
// transpose back and the plain pushforward instead.  The dual value after the
// update (J(phi_{n+1/2}) or I(psi_{n+1})) shares its second term with the
// measurement that starts the next half step (<psi_{n+1/2}, mu> or
// <phi_{n+1}, nu>), so its step rule runs there (finalize_dual_pend_kernel),
// before the measurement and before the next update uses sigma.  Same steps
// and step rule as half_step.
template <typename T>
static bfm_status half_step_flipped(const Grid& g0, Workspace* w, bool phi_half, T* phi, T* psi,
                                    Logs logs, cudaStream_t st)
{
    const double hd = 1.0 / (double)g0.N;
    const int* done = &w->state->done;
    const Grid gt = transposed_grid(g0);
    const Grid& g = phi_half ? g0 : gt;                  // layout of this half's potential
    const AxisTables swapped[3] = {w->tabs[1], w->tabs[0], w->tabs[2]};
    const AxisTables* tabs = phi_half ? w->tabs : swapped;
    T* mu = (T*)(phi_half ? w->mu_n : w->mu_t);          // mu and nu in the layout of g
    T* nu = (T*)(phi_half ? w->nu_n : w->nu_t);
    T* tmp = (T*)w->tmp;
    T* rho = (T*)w->rho;
    T* xt = (T*)w->xt;
    T* xg = transposed_axis1(g, (int)sizeof(T)) ? xt : nullptr;
    T* src = phi_half ? phi : psi;
    T* dst = phi_half ? psi : phi;
    const T* w_src = phi_half ? nu : mu;
    const T* w_dst = phi_half ? mu : nu;
    const T* source = phi_half ? mu : nu;
    const T* target = phi_half ? nu : mu;
    int ni = 0, no = 0, ng = 0;
    bfm_status s;
    // psi~ = src^c is left in the transposed layout (in xt), where the
    // pushforward reads it together with the transposed copy of the source
    // density and deposits rho in g's layout: no transpose back (where the
    // transposed rows allow the pushforward's row form, else the transpose)
    const Grid& gtt = phi_half ? gt : g0;                // the transposed layout of g
    T* source_t = (T*)(phi_half ? w->mu_t : w->nu_n);
    // (the pushforward also takes the dot <psi~, mu> from its loads)
    const bool tpush = xg && gtt.n[0] % 4 == 0;
    if (tpush) {
        s = ct_flip<T>(g, src, xt, w_src, slot(w, 0), &ni, done, st, tmp, w->state->row_ctr);
        if (s != BFM_OK) return s;
        ProfScope ps(PK_PUSH, 1, st);
        s = launch_pushforward_t<T>(gtt, xt, source_t, rho, g, done, st, slot(w, 1), &no);
    } else {
        s = ct_with_dots<T>(g, src, tmp, w_src, w_dst, slot(w, 0), &ni, slot(w, 1), &no, done, st,
                            xg, nullptr, w->state->row_ctr);
    }
    if (s != BFM_OK) return s;
    {
        // the previous half step's flip swept the other layout's rows first
        const int nprev = ct_pass_blocks(phi_half ? gt : g0, 0, (int)sizeof(T), kMaxPartials);
        ProfScope ps(PK_SMALL, 1, st);
        finalize_dual_pend_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 3), nprev, slot(w, 0),
                                                             ni, slot(w, 1), no, hd,
                                                             phi_half ? 0 : 2, logs);
        BFM_LAUNCH_CHECK("finalize_dual_pend_kernel");
    }
    if (!tpush) {
        ProfScope ps(PK_PUSH, 1, st);
        s = launch_pushforward<T>(g, tmp, source, rho, done, st, nullptr);
        if (s != BFM_OK) return s;
    }
    s = poisson_forward<T>(g, tabs, rho, target, rho, slot(w, 2), &ng, done, st, xg);
    if (s != BFM_OK) return s;
    {
        ProfScope ps(PK_SMALL, 1, st);
        finalize_G_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 2), ng, phi_half ? 0 : 1, logs);
        BFM_LAUNCH_CHECK("finalize_G_kernel");
    }
    s = poisson_inverse<T>(g, tabs, rho, src, src, &w->state->sigma, done, st);
    if (s != BFM_OK) return s;
    return ct_flip<T>(g, src, dst, w_src, slot(w, 3), &ni, done, st, xt, w->state->row_ctr);
}

template <typename T>
bfm_status half_step(const Grid& g, Workspace* w, bool phi_half, T* phi, T* psi,
                            Logs logs, cudaStream_t st, const double* pc)
{
    NvtxRange nv(phi_half ? "bfm_phi_half_step" : "bfm_psi_half_step");
    const double hd = 1.0 / (double)g.N;
    const int* done = &w->state->done;
    T* mu = (T*)w->mu_n;
    T* nu = (T*)w->nu_n;
    T* tmp = (T*)w->tmp;
    T* rho = (T*)w->rho;
    // phi-half: src = phi (weight nu), transform weight mu, source measure mu, target nu
    T* src = phi_half ? phi : psi;
    T* dst = phi_half ? psi : phi;
    const T* w_src = phi_half ? nu : mu;
    const T* w_dst = phi_half ? mu : nu;
    const T* source = phi_half ? mu : nu;
    const T* target = phi_half ? nu : mu;
    int ni = 0, no = 0, ng = 0;
    bfm_status s;
    T* xt = (T*)w->xt;
    if (w->mu_t && !pc) return half_step_flipped<T>(g, w, phi_half, phi, psi, logs, st);
    s = ct_with_dots<T>(g, src, tmp, w_src, w_dst, slot(w, 0), &ni, slot(w, 1), &no, done, st, xt, pc, w->state->row_ctr);
    if (s != BFM_OK) return s;
    {
        ProfScope ps(PK_SMALL, 1, st);
        finalize_dual_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 0), ni, slot(w, 1), no, hd,
                                                phi_half ? 0 : 2, logs);
        BFM_LAUNCH_CHECK("finalize_dual_kernel");
    }
    {
        ProfScope ps(PK_PUSH, 1, st);
        s = launch_pushforward<T>(g, tmp, source, rho, done, st, pc);
        if (s != BFM_OK) return s;
    }
    s = poisson_forward<T>(g, w->tabs, rho, target, rho, slot(w, 2), &ng, done, st, xt);
    if (s != BFM_OK) return s;
    {
        ProfScope ps(PK_SMALL, 1, st);
        finalize_G_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 2), ng, phi_half ? 0 : 1, logs);
        BFM_LAUNCH_CHECK("finalize_G_kernel");
    }
    s = poisson_inverse<T>(g, w->tabs, rho, src, src, &w->state->sigma, done, st);
    if (s != BFM_OK) return s;
    s = ct_with_dots<T>(g, src, dst, w_src, w_dst, slot(w, 0), &ni, slot(w, 1), &no, done, st, xt, pc, w->state->row_ctr);
    if (s != BFM_OK) return s;
    {
        ProfScope ps(PK_SMALL, 1, st);
        finalize_dual_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 0), ni, slot(w, 1), no, hd,
                                                phi_half ? 1 : 3, logs);
        BFM_LAUNCH_CHECK("finalize_dual_kernel");
    }
    return BFM_OK;
}

// One iteration of the H1-dot gradient ascent on J compared with the method in
// Section 5: on entry tmp holds psi_n = phi_n^c and J(phi_n) is logged;
//   rho = (x - grad psi_n) # mu, g = (-Delta)^{-1}(nu - rho) (residual, stop),
//   phi_{n+1/2} = phi_n + sigma g, psi_{n+1} = phi_{n+1/2}^c (step rule on
//   J(phi_{n+1/2}) - J(phi_n)), phi_{n+1} = psi_{n+1}^c, J(phi_{n+1}) =
//   <phi_{n+1}, nu> + <psi_{n+1}, mu> logged (psi_{n+1}^{cc} = psi_{n+1}).
template <typename T>
static bfm_status ascent_step(const Grid& g, Workspace* w, T* phi, Logs logs, cudaStream_t st,
                              const double* pc)
{
    const double hd = 1.0 / (double)g.N;
    const int* done = &w->state->done;
    T* mu = (T*)w->mu_n;
    T* nu = (T*)w->nu_n;
    T* tmp = (T*)w->tmp;
    T* rho = (T*)w->rho;
    T* xt = (T*)w->xt;
    int ni = 0, no = 0, ng = 0;
    bfm_status s;
    {
        ProfScope ps(PK_PUSH, 1, st);
        s = launch_pushforward<T>(g, tmp, mu, rho, done, st, pc);
        if (s != BFM_OK) return s;
    }
    s = poisson_forward<T>(g, w->tabs, rho, nu, rho, slot(w, 2), &ng, done, st, xt);
    if (s != BFM_OK) return s;
    {
        ProfScope ps(PK_SMALL, 1, st);
        finalize_G_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 2), ng, 0, logs);
        BFM_LAUNCH_CHECK("finalize_G_kernel");
    }
    s = poisson_inverse<T>(g, w->tabs, rho, phi, phi, &w->state->sigma, done, st);
    if (s != BFM_OK) return s;
    s = ct_with_dots<T>(g, phi, tmp, nu, mu, slot(w, 0), &ni, slot(w, 1), &no, done, st, xt, pc, w->state->row_ctr);
    if (s != BFM_OK) return s;
    {
        ProfScope ps(PK_SMALL, 1, st);
        finalize_dual_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 0), ni, slot(w, 1), no, hd,
                                                        3, logs);
        BFM_LAUNCH_CHECK("finalize_dual_kernel");
    }
    s = ct_with_dots<T>(g, tmp, phi, mu, nu, slot(w, 0), &ni, slot(w, 1), &no, done, st, xt, pc, w->state->row_ctr);
    if (s != BFM_OK) return s;
    {
        ProfScope ps(PK_SMALL, 1, st);
        finalize_dual_kernel<<<1, kFinThreads, 0, st>>>(w->state, slot(w, 0), ni, slot(w, 1), no, hd,
                                                        0, logs);
        BFM_LAUNCH_CHECK("finalize_dual_kernel");
    }
    return BFM_OK;
}

template <typename T>
static bfm_status measure_density(const Grid& g, const T* x, Workspace* w, int which, cudaStream_t st)
{
    const int th = 256;
    long long nb = (g.N + th - 1) / th;
    if (nb > 1024) nb = 1024;
    stats_kernel<T><<<(int)nb, th, 0, st>>>(x, g.N, slot(w, 4), slot(w, 5), slot(w, 6), slot(w, 7));
    BFM_LAUNCH_CHECK("stats_kernel");
    stats_finalize_kernel<<<1, 256, 0, st>>>(w->state, slot(w, 4), slot(w, 5), slot(w, 6),
                                             slot(w, 7), (int)nb, 1.0 / (double)g.N, which);
    BFM_LAUNCH_CHECK("stats_finalize_kernel");
    return BFM_OK;
}

int elem_bytes(bfm_precision p) { return p == BFM_FP64 ? 8 : 4; }

Logs logs_of(Workspace* w, int max_iter)
{
    Logs logs;
    const int L = max_iter + 1;
    logs.dual = w->logs;
    logs.resid = w->logs + L;
    logs.sigma = w->logs + 2 * L;
    return logs;
}

__global__ void stop_now_kernel(SolverState* st)
{
    if (threadIdx.x == 0 && !st->done) st->max_iter = st->iter;
}

// Setup: validate and normalise the densities, fill the tables, measure
// ||nu - 1||^2_{H^-1}, set phi_0 (= 0 unless warm-started) and the state.
template <typename T>
bfm_status init_impl(const T* mu, const T* nu, const Grid& g, double tol, int max_iter,
                            const bfm_options& o, unsigned char* wsp, cudaStream_t st, T* phi,
                            T* psi)
{
    Workspace w;
    carve(g, sizeof(T), max_iter, wsp, &w, true);
    bfm_status s;
    s = measure_density<T>(g, mu, &w, 0, st); if (s != BFM_OK) return s;
    s = measure_density<T>(g, nu, &w, 1, st); if (s != BFM_OK) return s;
    SolverState hs;
    BFM_CUDA(cudaMemcpyAsync(&hs, w.state, sizeof(hs), cudaMemcpyDeviceToHost, st));
    BFM_CUDA(cudaStreamSynchronize(st));
    if (hs.bad_mu || hs.bad_nu || hs.min_mu < 0.0 || hs.min_nu < 0.0 || !(hs.mass_mu > 0.0) ||
        !(hs.mass_nu > 0.0)) {
        set_last_error("densities must be finite, non-negative and of positive mass");
        return BFM_ERR_INVALID_ARG;
    }
    const int th = 256;
    int nb = (int)((g.N + th - 1) / th);
    if (nb > num_sms() * 16) nb = num_sms() * 16;
    scale_kernel<T><<<nb, th, 0, st>>>(mu, (T*)w.mu_n, g.N, w.state, 0);
    scale_kernel<T><<<nb, th, 0, st>>>(nu, (T*)w.nu_n, g.N, w.state, 1);
    BFM_LAUNCH_CHECK("scale_kernel");
    if (w.mu_t) {
        s = transpose<T>(g, true, (const T*)w.mu_n, (T*)w.mu_t, nullptr, nullptr, nullptr, nullptr, st);
        if (s != BFM_OK) return s;
        s = transpose<T>(g, true, (const T*)w.nu_n, (T*)w.nu_t, nullptr, nullptr, nullptr, nullptr, st);
        if (s != BFM_OK) return s;
    }
    const double* pc = cost_exponents(&o);
    init_state_kernel<<<1, 1, 0, st>>>(w.state, o.sigma0, tol, max_iter, o.beta1, o.beta2,
                                       o.alpha1, o.alpha2, o.sigma_min, pc ? 1 : 0,
                                       o.cost_p[0], o.cost_p[1], o.cost_p[2]);
    BFM_LAUNCH_CHECK("init_state_kernel");
    s = fill_tables<T>(g, &w, st); if (s != BFM_OK) return s;
    // ||nu - 1||^2_{H^-1}: the mean of nu/mass is 1 and the zero mode is dropped
    int ng = 0;
    s = poisson_forward<T>(g, w.tabs, (const T*)w.nu_n, nullptr, (T*)w.rho, slot(&w, 2), &ng,
                           nullptr, st, (T*)w.xt);
    if (s != BFM_OK) return s;
    Logs logs = logs_of(&w, max_iter);
    finalize_G_kernel<<<1, 256, 0, st>>>(w.state, slot(&w, 2), ng, 2, logs);
    BFM_LAUNCH_CHECK("finalize_G_kernel");
    if (!o.warm_start) BFM_CUDA(cudaMemsetAsync(phi, 0, sizeof(T) * g.N, st));
    BFM_CUDA(cudaMemsetAsync(psi, 0, sizeof(T) * g.N, st));
    BFM_CUDA(cudaMemsetAsync(w.logs, 0, sizeof(double) * 3 * (max_iter + 1), st));
    if (o.method == BFM_GRADIENT_ASCENT) {
        // the ascent keeps psi_n = phi_n^c in tmp; measure J(phi_0)
        int ni = 0, no = 0;
        s = ct_with_dots<T>(g, phi, (T*)w.tmp, (const T*)w.nu_n, (const T*)w.mu_n, slot(&w, 0), &ni,
                            slot(&w, 1), &no, &w.state->done, st, (T*)w.xt, pc, w.state->row_ctr);
        if (s != BFM_OK) return s;
        finalize_dual_kernel<<<1, kFinThreads, 0, st>>>(w.state, slot(&w, 0), ni, slot(&w, 1), no,
                                                        1.0 / (double)g.N, 0, logs);
        BFM_LAUNCH_CHECK("finalize_dual_kernel");
    }
    return BFM_OK;
}

// Enqueue `iters` back-and-forth iterations; no host synchronisation.
template <typename T>
static bfm_status iterate_impl(const Grid& g, int max_iter, int iters, int method,
                               const double* pc, unsigned char* wsp, cudaStream_t st, T* phi,
                               T* psi)
{
    Workspace w;
    carve(g, sizeof(T), max_iter, wsp, &w, true);
    Logs logs = logs_of(&w, max_iter);
    if (method == BFM_GRADIENT_ASCENT) {
        for (int c = 0; c < iters; ++c) {
            bfm_status s = ascent_step<T>(g, &w, phi, logs, st, pc);
            if (s != BFM_OK) return s;
        }
        return BFM_OK;
    }
    for (int c = 0; c < iters; ++c) {
        bfm_status s = half_step<T>(g, &w, true, phi, psi, logs, st, pc); if (s != BFM_OK) return s;
        s = half_step<T>(g, &w, false, phi, psi, logs, st, pc); if (s != BFM_OK) return s;
    }
    return BFM_OK;
}

// A chunk of iterations captured once as a CUDA graph and replayed on a
// private non-blocking stream, which events order after the caller's stream
// on entry and the caller's stream after it on exit (nothing blocks).  The
// graph lives for one C-ABI call: the host keeps nothing between calls.
// Replays skip the per-kernel launch work of the host and the gaps it leaves.
struct ChunkGraph {
    cudaStream_t ps = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~ChunkGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);    // freed when in-flight replays finish
        if (graph) cudaGraphDestroy(graph);
        if (ev) cudaEventDestroy(ev);
        if (ps) cudaStreamDestroy(ps);
    }
    bfm_status begin(cudaStream_t user)
    {
        BFM_CUDA(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
        BFM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        BFM_CUDA(cudaEventRecord(ev, user));
        BFM_CUDA(cudaStreamWaitEvent(ps, ev, 0));
        return BFM_OK;
    }
    template <typename F>
    bfm_status capture(F enqueue)
    {
        BFM_CUDA(cudaStreamBeginCapture(ps, cudaStreamCaptureModeRelaxed));
        const bfm_status s = enqueue(ps);
        const cudaError_t e = cudaStreamEndCapture(ps, &graph);     // always ends the capture
        if (s != BFM_OK) return s;
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
        BFM_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        return BFM_OK;
    }
    bfm_status launch() { BFM_CUDA(cudaGraphLaunch(exec, ps)); return BFM_OK; }
    bfm_status end(cudaStream_t user)
    {
        BFM_CUDA(cudaEventRecord(ev, ps));
        BFM_CUDA(cudaStreamWaitEvent(user, ev, 0));
        return BFM_OK;
    }
};

constexpr int kGraphChunk = 4;       // iterations per captured graph

// `iters` iterations: replays of a captured chunk when there are enough of
// them and the per-launch profiler is off (its events must be recorded per
// launch), else plain launches on `user`.
template <typename T>
static bfm_status iterate_chunked(const Grid& g, int max_iter, int iters, int method,
                                  const double* pc, unsigned char* wsp, cudaStream_t user, T* phi,
                                  T* psi)
{
    if (g_prof.on || iters < 2 * kGraphChunk)
        return iterate_impl<T>(g, max_iter, iters, method, pc, wsp, user, phi, psi);
    ChunkGraph cg;
    bfm_status s = cg.begin(user);
    if (s != BFM_OK) return s;
    s = cg.capture([&](cudaStream_t st) {
        return iterate_impl<T>(g, max_iter, kGraphChunk, method, pc, wsp, st, phi, psi);
    });
    if (s != BFM_OK) return s;
    for (int r = 0; r < iters / kGraphChunk; ++r) {
        s = cg.launch();
        if (s != BFM_OK) return s;
    }
    s = iterate_impl<T>(g, max_iter, iters % kGraphChunk, method, pc, wsp, cg.ps, phi, psi);
    if (s != BFM_OK) return s;
    return cg.end(user);
}

static bfm_status read_done(const Grid& g, int eb, int max_iter, unsigned char* wsp,
                            cudaStream_t st, int* done)
{
    Workspace w;
    carve(g, eb, max_iter, wsp, &w, true);
    BFM_CUDA(cudaMemcpyAsync(done, &w.state->done, sizeof(int), cudaMemcpyDeviceToHost, st));
    BFM_CUDA(cudaStreamSynchronize(st));
    return BFM_OK;
}

// Outputs: if the loop has not stopped, one more measurement (the first part
// of a phi-half step) gives phi_n^c and J(phi_n); then psi = phi_n^c, the map
// T = x - grad psi, W2^2 = 2 J(phi_n) and the logs.
template <typename T>
bfm_status finish_impl(const Grid& g, int max_iter, unsigned char* wsp, cudaStream_t st,
                              bfm_result* out)
{
    Workspace w;
    carve(g, sizeof(T), max_iter, wsp, &w, true);
    Logs logs = logs_of(&w, max_iter);
    T* phi = (T*)out->phi;
    T* psi = (T*)out->psi;
    // the cost the solve was started with (finish synchronises anyway)
    SolverState hs0;
    BFM_CUDA(cudaMemcpyAsync(&hs0, w.state, sizeof(hs0), cudaMemcpyDeviceToHost, st));
    BFM_CUDA(cudaStreamSynchronize(st));
    const double* pc = hs0.power ? hs0.cost_p : nullptr;
    stop_now_kernel<<<1, 32, 0, st>>>(w.state);
    BFM_LAUNCH_CHECK("stop_now_kernel");
    bfm_status s = half_step<T>(g, &w, true, phi, psi, logs, st, pc);
    if (s != BFM_OK) return s;
    SolverState hs;
    BFM_CUDA(cudaMemcpyAsync(&hs, w.state, sizeof(hs), cudaMemcpyDeviceToHost, st));
    BFM_CUDA(cudaStreamSynchronize(st));
    if (hs.nonfinite) {
        set_last_error("a reduction produced a non-finite value");
        return BFM_ERR_NONFINITE;
    }
    // psi = phi_n^c formed afresh from the final phi (no done flag: it runs
    // even when the loop stopped inside a half step)
    int nd0 = 0, nd1 = 0;
    s = ct_with_dots<T>(g, phi, psi, nullptr, nullptr, nullptr, &nd0, nullptr, &nd1, nullptr, st,
                        (T*)w.xt, pc, w.state->row_ctr);
    if (s != BFM_OK) return s;
    if (out->map) { s = launch_map<T>(g, psi, (T*)out->map, st, pc); if (s != BFM_OK) return s; }
    const int nlog = hs.iter + 1;
    if (out->dual) BFM_CUDA(cudaMemcpyAsync(out->dual, logs.dual, sizeof(double) * nlog, cudaMemcpyDeviceToHost, st));
    if (out->resid) BFM_CUDA(cudaMemcpyAsync(out->resid, logs.resid, sizeof(double) * nlog, cudaMemcpyDeviceToHost, st));
    if (out->sigma) BFM_CUDA(cudaMemcpyAsync(out->sigma, logs.sigma, sizeof(double) * nlog, cudaMemcpyDeviceToHost, st));
    BFM_CUDA(cudaStreamSynchronize(st));
    out->w2sq = 2.0 * hs.J_old;
    out->mass_mu = hs.mass_mu;
    out->mass_nu = hs.mass_nu;
    out->max_mu = hs.max_mu;
    out->max_nu = hs.max_nu;
    out->sigma_final = hs.sigma;
    out->iters = hs.iter;
    out->converged = hs.converged;
    return hs.converged ? BFM_OK : BFM_NOT_CONVERGED;
}

template bfm_status init_impl<float>(const float*, const float*, const Grid&, double, int,
                                     const bfm_options&, unsigned char*, cudaStream_t, float*, float*);
template bfm_status init_impl<double>(const double*, const double*, const Grid&, double, int,
                                      const bfm_options&, unsigned char*, cudaStream_t, double*, double*);
template bfm_status finish_impl<float>(const Grid&, int, unsigned char*, cudaStream_t, bfm_result*);
template bfm_status finish_impl<double>(const Grid&, int, unsigned char*, cudaStream_t, bfm_result*);

}  // namespace bfm

// ===========================================================================
// C ABI
// ===========================================================================
using namespace bfm;

static bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

extern "C" size_t bfm_workspace_bytes(const bfm_grid* grid, bfm_precision prec, int max_iter)
{
    Grid g;
    if (!make_grid(grid, &g) || max_iter < 0) return 0;
    return solve_bytes(g, elem_bytes(prec), max_iter);
}

extern "C" size_t bfm_workspace_bytes_host(const bfm_grid* grid, bfm_precision prec, int max_iter)
{
    Grid g;
    if (!make_grid(grid, &g) || max_iter < 0) return 0;
    const size_t f = up256((size_t)elem_bytes(prec) * g.N);
    return solve_bytes(g, elem_bytes(prec), max_iter) + 4 * f + up256((size_t)elem_bytes(prec) * g.N * g.ndim);
}

extern "C" size_t bfm_poisson_workspace_bytes(const bfm_grid* grid, bfm_precision prec)
{
    Grid g;
    if (!make_grid(grid, &g)) return 0;
    return poisson_bytes(g, elem_bytes(prec));
}

const double* bfm::cost_exponents(const bfm_options* o)
{
    return (o && o->cost_p[0] > 0.0) ? o->cost_p : nullptr;
}

static bool exponents_ok(const double* p, int ndim)
{
    for (int a = 0; a < ndim; ++a)
        if (!(p[a] > 1.0 && p[a] <= 16.0)) return false;
    return true;
}

// BFM_COST_QUADRATIC takes cost_p all zero; BFM_COST_POWER takes 1 < p_a <= 16
static bfm_status check_cost(bfm_cost cost, const bfm_options& o, const Grid& g)
{
    if (cost == BFM_COST_QUADRATIC) {
        if (o.cost_p[0] != 0.0 || o.cost_p[1] != 0.0 || o.cost_p[2] != 0.0) {
            set_last_error("cost_p must be zero for the quadratic cost");
            return BFM_ERR_INVALID_ARG;
        }
        return BFM_OK;
    }
    if (!exponents_ok(o.cost_p, g.ndim)) {
        set_last_error("the power cost needs 1 < cost_p[a] <= 16 on every axis");
        return BFM_ERR_INVALID_ARG;
    }
    return BFM_OK;
}

static bfm_status check_common(const bfm_grid* grid, bfm_precision prec, Grid* g)
{
    if (prec != BFM_FP32 && prec != BFM_FP64) return BFM_ERR_INVALID_ARG;
    if (!make_grid(grid, g)) {
        set_last_error("grid must have ndim 2 or 3 and 2 <= n <= 8192 per axis");
        return BFM_ERR_INVALID_ARG;
    }
    return BFM_OK;
}

static bfm_status check_solver_args(const bfm_grid* grid, bfm_precision prec, int max_iter,
                                    void* workspace, size_t workspace_bytes, Grid* g)
{
    bfm_status s = check_common(grid, prec, g);
    if (s != BFM_OK) return s;
    if (!fft_sizes_ok(*g)) { set_last_error("every n[a] must be 2^p 3^q"); return BFM_ERR_UNSUPPORTED; }
    if (max_iter < 0 || max_iter > 10000000) { set_last_error("bad max_iter"); return BFM_ERR_INVALID_ARG; }
    if (!workspace || !aligned256(workspace) ||
        workspace_bytes < solve_bytes(*g, elem_bytes(prec), max_iter)) {
        set_last_error("workspace NULL, not 256-byte aligned or smaller than bfm_workspace_bytes()");
        return BFM_ERR_WORKSPACE;
    }
    return BFM_OK;
}

extern "C" bfm_status bfm_solver_init(const void* mu, const void* nu, const bfm_grid* grid,
                                      bfm_cost cost, bfm_precision prec, double tol, int max_iter,
                                      const bfm_options* opt, void* workspace,
                                      size_t workspace_bytes, void* stream, void* phi, void* psi)
{
    Grid g;
    bfm_status s = check_solver_args(grid, prec, max_iter, workspace, workspace_bytes, &g);
    if (s != BFM_OK) return s;
    if (cost != BFM_COST_QUADRATIC && cost != BFM_COST_POWER) {
        set_last_error("unknown cost");
        return BFM_ERR_UNSUPPORTED;
    }
    if (!mu || !nu || !phi || !psi || !(tol >= 0.0)) {
        set_last_error("null pointer or negative tolerance");
        return BFM_ERR_INVALID_ARG;
    }
    bfm_options o;
    bfm_default_options(&o);
    if (opt) o = *opt;
    if (!(o.beta1 > 0 && o.beta1 < o.beta2 && o.beta2 < 1 && o.alpha1 > 1 && o.alpha2 > 0 &&
          o.alpha2 < 1 && o.sigma_min >= 0)) {
        set_last_error("step rule needs 0 < beta1 < beta2 < 1, alpha1 > 1, 0 < alpha2 < 1");
        return BFM_ERR_INVALID_ARG;
    }
    if (o.method != BFM_BACK_AND_FORTH && o.method != BFM_GRADIENT_ASCENT) {
        set_last_error("unknown method");
        return BFM_ERR_INVALID_ARG;
    }
    s = check_cost(cost, o, g);
    if (s != BFM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* wsp = (unsigned char*)workspace;
    if (prec == BFM_FP32)
        return init_impl<float>((const float*)mu, (const float*)nu, g, tol, max_iter, o, wsp, st,
                                (float*)phi, (float*)psi);
    return init_impl<double>((const double*)mu, (const double*)nu, g, tol, max_iter, o, wsp, st,
                             (double*)phi, (double*)psi);
}

extern "C" bfm_status bfm_solver_iterate(const bfm_grid* grid, bfm_precision prec, int max_iter,
                                         int iterations, const bfm_options* opt, void* workspace,
                                         size_t workspace_bytes, void* stream, void* phi, void* psi)
{
    Grid g;
    bfm_status s = check_solver_args(grid, prec, max_iter, workspace, workspace_bytes, &g);
    if (s != BFM_OK) return s;
    if (!phi || !psi || iterations < 0) return BFM_ERR_INVALID_ARG;
    const int method = opt ? opt->method : BFM_BACK_AND_FORTH;
    if (method != BFM_BACK_AND_FORTH && method != BFM_GRADIENT_ASCENT) {
        set_last_error("unknown method");
        return BFM_ERR_INVALID_ARG;
    }
    const double* pc = cost_exponents(opt);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* wsp = (unsigned char*)workspace;
    if (prec == BFM_FP32)
        return iterate_chunked<float>(g, max_iter, iterations, method, pc, wsp, st, (float*)phi,
                                      (float*)psi);
    return iterate_chunked<double>(g, max_iter, iterations, method, pc, wsp, st, (double*)phi,
                                   (double*)psi);
}

extern "C" bfm_status bfm_solver_finish(const bfm_grid* grid, bfm_precision prec, int max_iter,
                                        void* workspace, size_t workspace_bytes, void* stream,
                                        bfm_result* out)
{
    Grid g;
    bfm_status s = check_solver_args(grid, prec, max_iter, workspace, workspace_bytes, &g);
    if (s != BFM_OK) return s;
    if (!out || !out->phi || !out->psi) return BFM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* wsp = (unsigned char*)workspace;
    if (prec == BFM_FP32) return finish_impl<float>(g, max_iter, wsp, st, out);
    return finish_impl<double>(g, max_iter, wsp, st, out);
}

extern "C" bfm_status bfm_solve(const void* mu, const void* nu, const bfm_grid* grid, bfm_cost cost,
                                bfm_precision prec, double tol, int max_iter, const bfm_options* opt,
                                void* workspace, size_t workspace_bytes, void* stream,
                                bfm_result* out)
{
    if (!out) return BFM_ERR_INVALID_ARG;
    NvtxRange nv("bfm_solve");
    bfm_status s = bfm_solver_init(mu, nu, grid, cost, prec, tol, max_iter, opt, workspace,
                                   workspace_bytes, stream, out->phi, out->psi);
    if (s != BFM_OK) return s;
    Grid g;
    make_grid(grid, &g);
    const int poll = (opt && opt->poll_every > 0) ? opt->poll_every : 4;
    if (!g_prof.on) {
        // one captured chunk of `poll` iterations, replayed between polls
        const int method = opt ? opt->method : BFM_BACK_AND_FORTH;
        const double* pc = cost_exponents(opt);
        unsigned char* wsp = (unsigned char*)workspace;
        cudaStream_t user = (cudaStream_t)stream;
        ChunkGraph cg;
        s = cg.begin(user);
        if (s != BFM_OK) return s;
        s = cg.capture([&](cudaStream_t st) {
            if (prec == BFM_FP32)
                return iterate_impl<float>(g, max_iter, poll, method, pc, wsp, st,
                                           (float*)out->phi, (float*)out->psi);
            return iterate_impl<double>(g, max_iter, poll, method, pc, wsp, st,
                                        (double*)out->phi, (double*)out->psi);
        });
        if (s != BFM_OK) return s;
        for (int enq = 0; enq <= max_iter; enq += poll) {
            s = cg.launch();
            if (s != BFM_OK) return s;
            int done = 0;
            s = read_done(g, elem_bytes(prec), max_iter, wsp, cg.ps, &done);
            if (s != BFM_OK) return s;
            if (done) break;
        }
        s = cg.end(user);
        if (s != BFM_OK) return s;
        return bfm_solver_finish(grid, prec, max_iter, workspace, workspace_bytes, stream, out);
    }
    int enq = 0;
    while (enq <= max_iter) {
        const int chunk = (max_iter + 1 - enq) < poll ? (max_iter + 1 - enq) : poll;
        s = bfm_solver_iterate(grid, prec, max_iter, chunk, opt, workspace, workspace_bytes, stream,
                               out->phi, out->psi);
        if (s != BFM_OK) return s;
        enq += chunk;
        int done = 0;
        s = read_done(g, elem_bytes(prec), max_iter, (unsigned char*)workspace,
                      (cudaStream_t)stream, &done);
        if (s != BFM_OK) return s;
        if (done) break;
    }
    return bfm_solver_finish(grid, prec, max_iter, workspace, workspace_bytes, stream, out);
}

extern "C" int bfm_profile_kinds(void) { return PK_COUNT; }

extern "C" const char* bfm_profile_kind_name(int kind)
{
    return (kind >= 0 && kind < PK_COUNT) ? kProfNames[kind] : "";
}

extern "C" bfm_status bfm_profile_begin(int max_records)
{
    if (max_records <= 0) return BFM_ERR_INVALID_ARG;
    if (g_prof.on) return BFM_ERR_INVALID_ARG;
    g_prof.rec = new ProfRec[max_records];
    for (int i = 0; i < max_records; ++i) {
        BFM_CUDA(cudaEventCreate(&g_prof.rec[i].a));
        BFM_CUDA(cudaEventCreate(&g_prof.rec[i].b));
    }
    g_prof.cap = max_records;
    g_prof.used = 0;
    g_prof.dropped = 0;
    g_prof.on = true;
    return BFM_OK;
}

extern "C" bfm_status bfm_profile_end(double* ms_by_kind, int* launches_by_kind, int nkinds,
                                      int* dropped)
{
    if (!g_prof.on) return BFM_ERR_INVALID_ARG;
    g_prof.on = false;
    bfm_status s = BFM_OK;
    for (int k = 0; k < nkinds; ++k) {
        if (ms_by_kind) ms_by_kind[k] = 0.0;
        if (launches_by_kind) launches_by_kind[k] = 0;
    }
    for (int i = 0; i < g_prof.used; ++i) {
        ProfRec& r = g_prof.rec[i];
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) { s = cuda_status(e, "bfm_profile_end"); continue; }
        if (r.kind < nkinds) {
            if (ms_by_kind) ms_by_kind[r.kind] += ms;
            if (launches_by_kind) launches_by_kind[r.kind] += r.launches;
        }
    }
    for (int i = 0; i < g_prof.cap; ++i) {
        cudaEventDestroy(g_prof.rec[i].a);
        cudaEventDestroy(g_prof.rec[i].b);
    }
    delete[] g_prof.rec;
    g_prof.rec = nullptr;
    if (dropped) *dropped = g_prof.dropped;
    g_prof.cap = g_prof.used = 0;
    return s;
}

extern "C" bfm_status bfm_solve_host(const void* mu, const void* nu, const bfm_grid* grid,
                                     bfm_cost cost, bfm_precision prec, double tol, int max_iter,
                                     const bfm_options* opt, void* workspace, size_t workspace_bytes,
                                     void* stream, bfm_result* out)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!mu || !nu || !out || !out->phi || !out->psi || max_iter < 0) return BFM_ERR_INVALID_ARG;
    const size_t need = bfm_workspace_bytes_host(grid, prec, max_iter);
    if (!workspace || !aligned256(workspace) || workspace_bytes < need) return BFM_ERR_WORKSPACE;
    const int eb = elem_bytes(prec);
    const size_t fb = (size_t)eb * g.N;
    const size_t f = up256(fb);
    unsigned char* p = (unsigned char*)workspace + solve_bytes(g, eb, max_iter);
    void* dmu = p; void* dnu = p + f; void* dphi = p + 2 * f; void* dpsi = p + 3 * f;
    void* dmap = p + 4 * f;
    cudaStream_t st = (cudaStream_t)stream;
    BFM_CUDA(cudaMemcpyAsync(dmu, mu, fb, cudaMemcpyHostToDevice, st));
    BFM_CUDA(cudaMemcpyAsync(dnu, nu, fb, cudaMemcpyHostToDevice, st));
    bfm_result r = *out;
    r.phi = dphi; r.psi = dpsi; r.map = out->map ? dmap : nullptr;
    if (opt && opt->warm_start) BFM_CUDA(cudaMemcpyAsync(dphi, out->phi, fb, cudaMemcpyHostToDevice, st));
    s = bfm_solve(dmu, dnu, grid, cost, prec, tol, max_iter, opt, workspace,
                  solve_bytes(g, eb, max_iter), stream, &r);
    if (s < 0) return s;
    BFM_CUDA(cudaMemcpyAsync(out->phi, dphi, fb, cudaMemcpyDeviceToHost, st));
    BFM_CUDA(cudaMemcpyAsync(out->psi, dpsi, fb, cudaMemcpyDeviceToHost, st));
    if (out->map) BFM_CUDA(cudaMemcpyAsync(out->map, dmap, fb * g.ndim, cudaMemcpyDeviceToHost, st));
    BFM_CUDA(cudaStreamSynchronize(st));
    void* keep_phi = out->phi; void* keep_psi = out->psi; void* keep_map = out->map;
    *out = r;
    out->phi = keep_phi; out->psi = keep_psi; out->map = keep_map;
    return s;
}

extern "C" bfm_status bfm_ctransform(const void* phi, void* out, const bfm_grid* grid,
                                     bfm_precision prec, void* stream)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!phi || !out) return BFM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (int a = 0; a < g.ndim; ++a) {
        if (prec == BFM_FP32)
            s = launch_ct_pass<float>(g, a, a == 0 ? (const float*)phi : (const float*)out, (float*)out,
                                      a == 0, nullptr, nullptr, nullptr, nullptr, nullptr, 0, st, nullptr);
        else
            s = launch_ct_pass<double>(g, a, a == 0 ? (const double*)phi : (const double*)out,
                                       (double*)out, a == 0, nullptr, nullptr, nullptr, nullptr,
                                       nullptr, 0, st, nullptr);
        if (s != BFM_OK) return s;
    }
    BFM_LAUNCH_CHECK("ct_pass_kernel");
    return BFM_OK;
}

extern "C" bfm_status bfm_ctransform_power(const void* phi, void* out, const bfm_grid* grid,
                                           bfm_precision prec, const double* p, void* stream)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!phi || !out || !p || !exponents_ok(p, g.ndim)) {
        set_last_error("null pointer or exponent outside (1, 16]");
        return BFM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int a = 0; a < g.ndim; ++a) {
        if (prec == BFM_FP32)
            s = launch_ct_power_pass<float>(g, a, p[a], a == 0 ? (const float*)phi : (const float*)out,
                                            (float*)out, a == 0, nullptr, nullptr, nullptr, nullptr,
                                            nullptr, 0, st, nullptr);
        else
            s = launch_ct_power_pass<double>(g, a, p[a], a == 0 ? (const double*)phi : (const double*)out,
                                             (double*)out, a == 0, nullptr, nullptr, nullptr, nullptr,
                                             nullptr, 0, st, nullptr);
        if (s != BFM_OK) return s;
    }
    BFM_LAUNCH_CHECK("ct_power_kernel");
    return BFM_OK;
}

extern "C" bfm_status bfm_map_power(const void* psi, void* map, const bfm_grid* grid,
                                    bfm_precision prec, const double* p, void* stream)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!psi || !map || !p || !exponents_ok(p, g.ndim)) {
        set_last_error("null pointer or exponent outside (1, 16]");
        return BFM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == BFM_FP32) return launch_map<float>(g, (const float*)psi, (float*)map, st, p);
    return launch_map<double>(g, (const double*)psi, (double*)map, st, p);
}

template <typename T>
static bfm_status poisson_impl(const T* f, T* gout, const Grid& g, double* G_out,
                               unsigned char* wsp, cudaStream_t st)
{
    Workspace w;
    carve(g, sizeof(T), 0, wsp, &w, false);
    bfm_status s = fill_tables<T>(g, &w, st);
    if (s != BFM_OK) return s;
    int ng = 0;
    s = poisson_forward<T>(g, w.tabs, f, nullptr, gout, slot(&w, 2), &ng, nullptr, st, (T*)nullptr);
    if (s != BFM_OK) return s;
    s = poisson_inverse<T>(g, w.tabs, gout, gout, nullptr, nullptr, nullptr, st);
    if (s != BFM_OK) return s;
    if (G_out) {
        Logs none = {nullptr, nullptr, nullptr};
        finalize_G_kernel<<<1, 256, 0, st>>>(w.state, slot(&w, 2), ng, 2, none);
        BFM_LAUNCH_CHECK("finalize_G_kernel");
        BFM_CUDA(cudaMemcpyAsync(G_out, &w.state->Gref, sizeof(double), cudaMemcpyDeviceToHost, st));
        BFM_CUDA(cudaStreamSynchronize(st));
    }
    return BFM_OK;
}

namespace bfm {
// The Poisson solve of bfm_poisson run on a caller-chosen scratch block (used
// by the allocation-free entry point of noalloc.cu).
size_t poisson_scratch_bytes(const Grid& g, int eb) { return poisson_bytes(g, eb); }

bfm_status poisson_on_scratch(const void* f, void* g_out, const Grid& g, bfm_precision prec,
                              double* G_out, unsigned char* scratch, cudaStream_t st)
{
    if (prec == BFM_FP32)
        return poisson_impl<float>((const float*)f, (float*)g_out, g, G_out, scratch, st);
    return poisson_impl<double>((const double*)f, (double*)g_out, g, G_out, scratch, st);
}
}  // namespace bfm

extern "C" bfm_status bfm_poisson(const void* f, void* g_out, const bfm_grid* grid,
                                  bfm_precision prec, double* G_out, void* workspace,
                                  size_t workspace_bytes, void* stream)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!fft_sizes_ok(g)) { set_last_error("every n[a] must be 2^p 3^q"); return BFM_ERR_UNSUPPORTED; }
    if (!f || !g_out) return BFM_ERR_INVALID_ARG;
    if (!workspace || !aligned256(workspace) || workspace_bytes < poisson_bytes(g, elem_bytes(prec)))
        return BFM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == BFM_FP32)
        return poisson_impl<float>((const float*)f, (float*)g_out, g, G_out, (unsigned char*)workspace, st);
    return poisson_impl<double>((const double*)f, (double*)g_out, g, G_out, (unsigned char*)workspace, st);
}

extern "C" bfm_status bfm_map(const void* psi, void* map, const bfm_grid* grid, bfm_precision prec,
                              void* stream)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!psi || !map) return BFM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == BFM_FP32) return launch_map<float>(g, (const float*)psi, (float*)map, st);
    return launch_map<double>(g, (const double*)psi, (double*)map, st);
}

extern "C" bfm_status bfm_pushforward(const void* psi, const void* mu, void* rho,
                                      const bfm_grid* grid, bfm_precision prec, void* stream)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!psi || !mu || !rho) return BFM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == BFM_FP32)
        return launch_pushforward<float>(g, (const float*)psi, (const float*)mu, (float*)rho, nullptr, st);
    return launch_pushforward<double>(g, (const double*)psi, (const double*)mu, (double*)rho, nullptr, st);
}

extern "C" bfm_status bfm_interpolate(const void* map, const void* mu, double t, void* rho,
                                      const bfm_grid* grid, bfm_precision prec, void* stream)
{
    Grid g;
    bfm_status s = check_common(grid, prec, &g);
    if (s != BFM_OK) return s;
    if (!map || !mu || !rho || !(t >= 0.0 && t <= 1.0)) return BFM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == BFM_FP32)
        return launch_interpolate<float>(g, (const float*)map, (const float*)mu, t, (float*)rho, st);
    return launch_interpolate<double>(g, (const double*)map, (const double*)mu, t, (double*)rho, st);
}
