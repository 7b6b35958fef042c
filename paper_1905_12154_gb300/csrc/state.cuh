// state.cuh -- solver state, per-half-step scalar logic and workspace layout,
// shared by the single-problem solver (solver.cu) and the batched solver
// (batched.cu).
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace bfm {

struct SolverState {
    double sigma;
    double J_old;
    double G;
    double Gref;
    double tol;
    double beta1, beta2, alpha1, alpha2, sigma_min;
    double mass_mu, mass_nu, max_mu, max_nu, min_mu, min_nu;
    double last_resid;
    int bad_mu, bad_nu;
    int iter;
    int max_iter;
    int done;
    int converged;
    int nonfinite;
    int pend;                 // the previous half step's step rule awaits its dual
                              // value (flipped layout: see finalize_dual_pend_kernel)
    int power;                // separable power cost with exponents cost_p
    double cost_p[3];
    int row_ctr[2];           // row c-transform: next row to take, groups done (0 between launches)
};

struct Logs {
    double* dual;
    double* resid;
    double* sigma;
};

inline size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Workspace {
    SolverState* state;
    double* parts;            // kPartialSlots * kMaxPartials
    double* logs;             // 3 * (max_iter + 1)
    unsigned char* tables;    // per-axis tables
    AxisTables tabs[3];
    void* mu_n;
    void* nu_n;
    void* tmp;
    void* rho;
    void* xt;                 // transposed copy for axis-1 sweeps of 2-D grids with
                              // long columns (transposed_axis1), else NULL
    void* mu_t;               // with xt: mu_n and nu_n transposed (the psi-half of a
    void* nu_t;               // step runs on the transposed grid), else NULL
    size_t bytes;
};

size_t tables_bytes(const Grid& g, int eb);
size_t poisson_bytes(const Grid& g, int eb);
size_t solve_bytes(const Grid& g, int eb, int max_iter);
void carve(const Grid& g, int eb, int max_iter, unsigned char* base, Workspace* w, bool fields);
bool fft_sizes_ok(const Grid& g);
double* slot(Workspace* w, int s);
Logs logs_of(Workspace* w, int max_iter);
int elem_bytes(bfm_precision p);
template <typename T> bfm_status fill_tables(const Grid& g, Workspace* w, cudaStream_t st);
template <typename T>
bfm_status init_impl(const T* mu, const T* nu, const Grid& g, double tol, int max_iter,
                     const bfm_options& o, unsigned char* wsp, cudaStream_t st, T* phi, T* psi);
template <typename T>
bfm_status finish_impl(const Grid& g, int max_iter, unsigned char* wsp, cudaStream_t st,
                       bfm_result* out);
// exponents of the solve's cost from its options: NULL for the quadratic cost
const double* cost_exponents(const bfm_options* o);

// ---------------------------------------------------------------------------
// device-side scalar logic of one half step (run by one thread)
// ---------------------------------------------------------------------------
// this thread's share of the n partials, four loads in flight
__device__ __forceinline__ double thread_sum_parts(const double* p, int n)
{
    const int bd = (int)blockDim.x;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int i = (int)threadIdx.x;
    for (; i + 3 * bd < n; i += 4 * bd) {
        v0 += p[i];
        v1 += p[i + bd];
        v2 += p[i + 2 * bd];
        v3 += p[i + 3 * bd];
    }
    for (; i < n; i += bd) v0 += p[i];
    return (v0 + v1) + (v2 + v3);
}

__device__ __forceinline__ double block_sum_parts(const double* p, int n, double* red)
{
    return block_sum(thread_sum_parts(p, n), red);
}

// three block sums with one pair of barriers (all threads call; the totals
// are valid on thread 0); red holds 96 doubles
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    __syncthreads();
    if (lane == 0) { red[wid] = a; red[32 + wid] = b; red[64 + wid] = c; }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    a = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    b = (threadIdx.x < nw) ? red[32 + threadIdx.x] : 0.0;
    c = (threadIdx.x < nw) ? red[64 + threadIdx.x] : 0.0;
    if (wid == 0) { a = warp_sum(a); b = warp_sum(b); c = warp_sum(c); }
}

__device__ __forceinline__ double step_rule(const SolverState* st, double sigma, double gain, double G)
{
    if (gain < st->beta1 * sigma * G) {
        const double s = st->alpha2 * sigma;
        const double fl = fmin(st->sigma_min, sigma);
        return fmax(s, fl);
    }
    if (gain > st->beta2 * sigma * G) return st->alpha1 * sigma;
    return sigma;
}

// mode 0: J(phi_n) at the start of the phi-half (logged); 1: J(phi_{n+1/2});
// mode 2: I(psi_{n+1/2}) at the start of the psi-half; 3: I(psi_{n+1}).
__device__ __forceinline__ void finalize_dual_body(SolverState* st, double J, int mode, Logs logs)
{
    if (!isfinite(J)) { st->nonfinite = 1; st->done = 1; return; }
    if (mode == 0) {
        st->J_old = J;
        if (logs.dual) logs.dual[st->iter] = J;
        if (logs.sigma) logs.sigma[st->iter] = st->sigma;
    } else if (mode == 2) {
        st->J_old = J;
    } else {
        st->sigma = step_rule(st, st->sigma, J - st->J_old, st->G);
        if (mode == 3) st->iter += 1;
    }
}

// mode 0: phi-half G -> residual, convergence; 1: psi-half G; 2: Gref.
__device__ __forceinline__ void finalize_G_body(SolverState* st, double G, int mode, Logs logs)
{
    if (!isfinite(G)) { st->nonfinite = 1; st->done = 1; return; }
    if (mode == 2) { st->Gref = G; return; }
    st->G = G;
    if (mode == 0) {
        const double r = st->Gref > 0.0 ? sqrt(fmax(G, 0.0) / st->Gref) : sqrt(fmax(G, 0.0));
        st->last_resid = r;
        if (logs.resid) logs.resid[st->iter] = r;
        if (r < st->tol) { st->converged = 1; st->done = 1; }
        else if (st->iter >= st->max_iter) st->done = 1;
    }
}

}  // namespace bfm
