// batched.cu -- many independent back-and-forth solves of uneven sizes at
// once, and the backward pass of the W2^2 loss.
//
// Batched solve: every problem runs Algorithm 1 with its own state, step size
// and convergence flag (the per-problem mask: a converged problem's kernels
// return at once).  Problems are grouped into classes of equal grid shape;
// every kernel step of a half step is one launch per class whose blockIdx.y
// picks the problem, with per-problem arguments read from device arrays built
// once at set-up.  A chunk of iterations is captured into a CUDA graph and
// replayed until every problem has stopped.
//
// Backward: by the envelope theorem on eq. (symmetric_dual) at the optimum,
// dC/dnu = phi and dC/dmu = psi (the potentials, integrated with weight hd),
// so with W2^2 = 2C and the inputs rescaled to unit mass, the derivative of
// W2^2 along mass-preserving perturbations of the density values is
//     dW2^2/dmu = 2 hd (psi - mean psi) / mass_mu,
//     dW2^2/dnu = 2 hd (phi - mean phi) / mass_nu,
// times the upstream gradient.
#include <string.h>
#include <map>
#include <vector>

#include "state.cuh"

namespace bfm {

// ---------------------------------------------------------------------------
// per-problem scalar kernels (one block per problem)
// ---------------------------------------------------------------------------
struct FinArgs {
    SolverState* st;
    const double* p_in;
    const double* p_out;
    const double* p_g;
    Logs logs;
    double hd;
};

__global__ void finalize_dual_batched(const FinArgs* fa, int nin, int nout, int mode)
{
    const FinArgs& a = fa[blockIdx.x];
    if (a.st->done) return;
    __shared__ double red[32];
    const double x = block_sum_parts(a.p_in, nin, red);
    const double y = block_sum_parts(a.p_out, nout, red);
    if (threadIdx.x == 0) finalize_dual_body(a.st, a.hd * (x + y), mode, a.logs);
}

__global__ void finalize_G_batched(const FinArgs* fa, int ng, int mode)
{
    const FinArgs& a = fa[blockIdx.x];
    if (a.st->done) return;
    __shared__ double red[32];
    const double G = block_sum_parts(a.p_g, ng, red);
    if (threadIdx.x == 0) finalize_G_body(a.st, G, mode, a.logs);
}

// number of problems that have not stopped, into *out (one block)
__global__ void count_running_kernel(const FinArgs* fa, int n, int* out)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (!fa[i].st->done) atomicAdd(&cnt, 1);
    __syncthreads();
    if (threadIdx.x == 0) *out = cnt;
}

// ---------------------------------------------------------------------------
// plan: classes of equal grid shape, workspace regions, argument arrays
// ---------------------------------------------------------------------------
struct ClassPlan {
    Grid g;
    std::vector<int> probs;
    size_t fin;                 // FinArgs[n] of this class (all problems of the batch in order)
    size_t ct[2][2][3];         // [half][before/after the step][axis]
    size_t fwd[2][3];           // [half][axis]
    size_t mid[2];
    size_t inv[2][3];
    size_t push[2];
    int nin, nout, ng;
    bool rows16 = false;        // every problem's phi and psi 16-byte aligned (workspace fields are)
};

struct BatchPlan {
    std::vector<Grid> grids;
    std::vector<size_t> region;     // byte offset of each problem's workspace
    std::vector<ClassPlan> classes;
    size_t args_off;                // start of the argument arrays
    size_t counter_off;             // one int for count_running_kernel
    size_t total;
};

static bool plan_batch(int nprob, const bfm_grid* grids, int eb, int max_iter, BatchPlan* bp)
{
    bp->grids.resize(nprob);
    bp->region.resize(nprob);
    size_t off = 0;
    std::map<std::vector<int>, int> cls;
    for (int p = 0; p < nprob; ++p) {
        Grid g;
        if (!make_grid(&grids[p], &g) || !fft_sizes_ok(g)) return false;
        bp->grids[p] = g;
        bp->region[p] = off;
        off += up256(solve_bytes(g, eb, max_iter));
        std::vector<int> key = {g.ndim, g.n[0], g.n[1], g.n[2]};
        auto it = cls.find(key);
        if (it == cls.end()) {
            ClassPlan c;
            c.g = g;
            cls[key] = (int)bp->classes.size();
            bp->classes.push_back(c);
            it = cls.find(key);
        }
        bp->classes[it->second].probs.push_back(p);
    }
    bp->args_off = off;
    const size_t ctb = ct_args_bytes(eb), dcb = dct_args_bytes(eb), pub = push_args_bytes(eb);
    for (ClassPlan& c : bp->classes) {
        const size_t n = c.probs.size();
        const int d = c.g.ndim;
        c.fin = off; off += up256(n * sizeof(FinArgs));
        for (int h = 0; h < 2; ++h) {
            for (int k = 0; k < 2; ++k)
                for (int a = 0; a < 3; ++a) {
                    c.ct[h][k][a] = off;
                    if (a < d) off += up256(n * ctb);
                }
            for (int a = 0; a < 3; ++a) { c.fwd[h][a] = off; if (a < d - 1) off += up256(n * dcb); }
            c.mid[h] = off; off += up256(n * dcb);
            for (int a = 0; a < 3; ++a) { c.inv[h][a] = off; if (a < d - 1) off += up256(n * dcb); }
            c.push[h] = off; off += up256(n * pub);
        }
    }
    bp->counter_off = off;
    off += 256;
    bp->total = off;
    return true;
}

template <typename T>
static bfm_status build_args(const BatchPlan& bp, unsigned char* wsp, bfm_result* outs,
                             int max_iter, std::vector<unsigned char>& host)
{
    host.assign(bp.total - bp.args_off, 0);
    auto at = [&](size_t off) { return host.data() + (off - bp.args_off); };
    const size_t ctb = ct_args_bytes(sizeof(T)), dcb = dct_args_bytes(sizeof(T)), pub = push_args_bytes(sizeof(T));
    for (const ClassPlan& c : bp.classes) {
        const Grid& g = c.g;
        const int d = g.ndim;
        for (size_t i = 0; i < c.probs.size(); ++i) {
            const int p = c.probs[i];
            Workspace w;
            carve(g, sizeof(T), max_iter, wsp + bp.region[p], &w, true);
            FinArgs* fa = reinterpret_cast<FinArgs*>(at(c.fin)) + i;
            fa->st = w.state;
            fa->p_in = slot(&w, 0);
            fa->p_out = slot(&w, 1);
            fa->p_g = slot(&w, 2);
            fa->logs = logs_of(&w, max_iter);
            fa->hd = 1.0 / (double)g.N;
            const int* done = &w.state->done;
            T* mu = (T*)w.mu_n;
            T* nu = (T*)w.nu_n;
            T* tmp = (T*)w.tmp;
            T* rho = (T*)w.rho;
            T* phi = (T*)outs[p].phi;
            T* psi = (T*)outs[p].psi;
            for (int h = 0; h < 2; ++h) {
                const bool ph = (h == 0);
                T* src = ph ? phi : psi;
                T* dst = ph ? psi : phi;
                const T* w_src = ph ? nu : mu;
                const T* w_dst = ph ? mu : nu;
                const T* source = ph ? mu : nu;
                const T* target = ph ? nu : mu;
                for (int a = 0; a < d; ++a) {
                    const bool first = (a == 0), last = (a == d - 1);
                    fill_ct_batch_args<T>(g, a, first ? src : tmp, tmp, first, first ? w_src : nullptr,
                                          first ? slot(&w, 0) : nullptr, last ? w_dst : nullptr,
                                          last ? slot(&w, 1) : nullptr, done,
                                          at(c.ct[h][0][a]) + i * ctb);
                    fill_ct_batch_args<T>(g, a, first ? src : dst, dst, first, first ? w_src : nullptr,
                                          first ? slot(&w, 0) : nullptr, last ? w_dst : nullptr,
                                          last ? slot(&w, 1) : nullptr, done,
                                          at(c.ct[h][1][a]) + i * ctb);
                }
                fill_push_batch_args<T>(g, tmp, source, rho, done, at(c.push[h]) + i * pub);
                bfm_status s;
                for (int a = 0; a < d - 1; ++a) {
                    s = fill_dct_batch_args<T>(g, a, w.tabs, rho, a == 0 ? target : nullptr, rho,
                                               nullptr, nullptr, nullptr, done,
                                               at(c.fwd[h][a]) + i * dcb);
                    if (s != BFM_OK) return s;
                }
                s = fill_dct_batch_args<T>(g, d - 1, w.tabs, rho, nullptr, rho, nullptr, nullptr,
                                           slot(&w, 2), done, at(c.mid[h]) + i * dcb);
                if (s != BFM_OK) return s;
                for (int a = d - 2; a >= 0; --a) {
                    const bool final_ = (a == 0);
                    s = fill_dct_batch_args<T>(g, a, w.tabs, rho, nullptr, final_ ? src : rho,
                                               final_ ? src : nullptr, &w.state->sigma, nullptr,
                                               done, at(c.inv[h][a]) + i * dcb);
                    if (s != BFM_OK) return s;
                }
            }
        }
    }
    return BFM_OK;
}

template <typename T>
static bfm_status enqueue_half(const ClassPlan& c, unsigned char* wsp, int h, cudaStream_t st)
{
    const Grid& g = c.g;
    const int d = g.ndim;
    const int n = (int)c.probs.size();
    const FinArgs* fin = reinterpret_cast<const FinArgs*>(wsp + c.fin);
    bfm_status s;
    for (int a = 0; a < d; ++a) {
        s = launch_ct_pass_batched<T>(g, a, n, wsp + c.ct[h][0][a], st);
        if (s != BFM_OK) return s;
    }
    finalize_dual_batched<<<n, 256, 0, st>>>(fin, c.nin, c.nout, h ? 2 : 0);
    BFM_LAUNCH_CHECK("finalize_dual_batched");
    s = launch_pushforward_batched<T>(d, g.N, n, wsp + c.push[h], st);
    if (s != BFM_OK) return s;
    for (int a = 0; a < d - 1; ++a) {
        s = launch_dct_pass_batched<T>(g, a, PASS_FWD, n, wsp + c.fwd[h][a], st, c.rows16);
        if (s != BFM_OK) return s;
    }
    s = launch_dct_pass_batched<T>(g, d - 1, PASS_MID, n, wsp + c.mid[h], st, c.rows16);
    if (s != BFM_OK) return s;
    finalize_G_batched<<<n, 256, 0, st>>>(fin, c.ng, h ? 1 : 0);
    BFM_LAUNCH_CHECK("finalize_G_batched");
    for (int a = d - 2; a >= 0; --a) {
        s = launch_dct_pass_batched<T>(g, a, PASS_INV, n, wsp + c.inv[h][a], st, c.rows16);
        if (s != BFM_OK) return s;
    }
    for (int a = 0; a < d; ++a) {
        s = launch_ct_pass_batched<T>(g, a, n, wsp + c.ct[h][1][a], st);
        if (s != BFM_OK) return s;
    }
    finalize_dual_batched<<<n, 256, 0, st>>>(fin, c.nin, c.nout, h ? 3 : 1);
    BFM_LAUNCH_CHECK("finalize_dual_batched");
    return BFM_OK;
}

struct BatchStreams;
template <typename T>
static bfm_status solve_batched_body(int nprob, const void* const* mu, const void* const* nu,
                                     BatchPlan& bp, double tol, int max_iter, const bfm_options& o,
                                     unsigned char* wsp, BatchStreams& bs, bfm_result* outs);

// The caller's stream may be the legacy default stream, which cannot be
// captured into a graph: the solve runs on a private stream once the caller's
// earlier work (the inputs) is complete, and is complete itself on return.
// Private streams of one batched solve: the main one and one per class of
// grid shape (the classes' chains are independent and run as parallel
// branches of the captured graph).
struct BatchStreams {
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> cls;
    std::vector<cudaEvent_t> ev;              // [0]: fork, [1 + c]: join of class c
    ~BatchStreams()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaStream_t c : cls) cudaStreamDestroy(c);
        if (main) cudaStreamDestroy(main);
    }
    bfm_status create(size_t nclass)
    {
        BFM_CUDA(cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking));
        cls.assign(nclass, nullptr);
        ev.assign(nclass + 1, nullptr);
        for (size_t c = 0; c < nclass; ++c) BFM_CUDA(cudaStreamCreateWithFlags(&cls[c], cudaStreamNonBlocking));
        for (size_t i = 0; i <= nclass; ++i) BFM_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
        return BFM_OK;
    }
};

template <typename T>
static bfm_status solve_batched_impl(int nprob, const void* const* mu, const void* const* nu,
                                     BatchPlan& bp, double tol, int max_iter, const bfm_options& o,
                                     unsigned char* wsp, cudaStream_t user, bfm_result* outs)
{
    BFM_CUDA(cudaStreamSynchronize(user));
    bfm_status s;
    cudaError_t e;
    {
        BatchStreams bs;
        s = bs.create(bp.classes.size());
        if (s != BFM_OK) return s;
        s = solve_batched_body<T>(nprob, mu, nu, bp, tol, max_iter, o, wsp, bs, outs);
        e = cudaStreamSynchronize(bs.main);
    }
    if (s == BFM_OK && e != cudaSuccess) return cuda_status(e, "batched solve");
    return s;
}

template <typename T>
static bfm_status solve_batched_body(int nprob, const void* const* mu, const void* const* nu,
                                     BatchPlan& bp, double tol, int max_iter, const bfm_options& o,
                                     unsigned char* wsp, BatchStreams& bs, bfm_result* outs)
{
    cudaStream_t st = bs.main;
    bfm_status s;
    for (int p = 0; p < nprob; ++p) {
        s = init_impl<T>((const T*)mu[p], (const T*)nu[p], bp.grids[p], tol, max_iter, o,
                         wsp + bp.region[p], st, (T*)outs[p].phi, (T*)outs[p].psi);
        if (s != BFM_OK) return s;
    }
    for (ClassPlan& c : bp.classes) {
        c.nin = ct_batch_blocks<T>(c.g, 0);
        c.nout = ct_batch_blocks<T>(c.g, c.g.ndim - 1);
        c.ng = dct_batch_blocks<T>(c.g, c.g.ndim - 1);
        c.rows16 = true;
        for (int p : c.probs)
            if ((reinterpret_cast<uintptr_t>(outs[p].phi) | reinterpret_cast<uintptr_t>(outs[p].psi)) & 15u)
                c.rows16 = false;
    }
    std::vector<unsigned char> host;
    s = build_args<T>(bp, wsp, outs, max_iter, host);
    if (s != BFM_OK) return s;
    BFM_CUDA(cudaMemcpyAsync(wsp + bp.args_off, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    BFM_CUDA(cudaStreamSynchronize(st));          // `host` is released when this function returns
    // all problems' FinArgs for the stop test: the classes' arrays are contiguous
    // per class, so count class by class
    int* counter = reinterpret_cast<int*>(wsp + bp.counter_off);
    const int chunk = o.poll_every > 0 ? o.poll_every : 4;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // one captured chunk: each class's iterations on its own stream, forked
    // from and joined back to the main stream (parallel graph branches)
    BFM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    bfm_status cap = BFM_OK;
    cudaError_t ce = cudaEventRecord(bs.ev[0], st);
    for (size_t ci = 0; ci < bp.classes.size() && cap == BFM_OK && ce == cudaSuccess; ++ci) {
        cudaStream_t cs = bs.cls[ci];
        ce = cudaStreamWaitEvent(cs, bs.ev[0], 0);
        for (int it = 0; it < chunk && cap == BFM_OK && ce == cudaSuccess; ++it)
            for (int h = 0; h < 2 && cap == BFM_OK; ++h) cap = enqueue_half<T>(bp.classes[ci], wsp, h, cs);
        if (ce == cudaSuccess) ce = cudaEventRecord(bs.ev[1 + ci], cs);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, bs.ev[1 + ci], 0);
    }
    if (cap == BFM_OK && ce != cudaSuccess) cap = cuda_status(ce, "batched capture fork/join");
    cudaError_t e = cudaStreamEndCapture(st, &graph);      // always ends the capture
    if (cap != BFM_OK) { if (graph) cudaGraphDestroy(graph); return cap; }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_status(e, "cudaGraphInstantiate"); }
    bfm_status result = BFM_OK;
    for (int launched = 0; launched <= max_iter; launched += chunk) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) { result = cuda_status(e, "cudaGraphLaunch"); break; }
        int running = 0;
        for (const ClassPlan& c : bp.classes) {
            count_running_kernel<<<1, 256, 0, st>>>(reinterpret_cast<const FinArgs*>(wsp + c.fin),
                                                    (int)c.probs.size(), counter);
            int r = 0;
            e = cudaMemcpyAsync(&r, counter, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) break;
            running += r;
        }
        if (e != cudaSuccess) { result = cuda_status(e, "batched poll"); break; }
        if (running == 0) break;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (result != BFM_OK) return result;
    bool all_converged = true;
    for (int p = 0; p < nprob; ++p) {
        s = finish_impl<T>(bp.grids[p], max_iter, wsp + bp.region[p], st, &outs[p]);
        if (s < 0) return s;
        if (s != BFM_OK) all_converged = false;
    }
    return all_converged ? BFM_OK : BFM_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// backward of the W2^2 loss
// ---------------------------------------------------------------------------
constexpr int kBwdBlocks = 128;

template <typename T>
struct BwdArgs {
    const T* phi;
    const T* psi;
    T* gmu;
    T* gnu;
    long long N;
    double mass_mu, mass_nu;
    double* part;          // 2 * kBwdBlocks: sums of psi and phi per block
};

template <typename T>
__global__ void bwd_sum_kernel(const BwdArgs<T>* batch)
{
    const BwdArgs<T>& a = batch[blockIdx.y];
    __shared__ double red[32];
    Acc<T> sp, sq;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.N;
         i += (long long)gridDim.x * blockDim.x) {
        sp.add(a.psi[i]);
        sq.add(a.phi[i]);
    }
    const double tp = block_sum(sp.take(), red);
    const double tq = block_sum(sq.take(), red);
    if (threadIdx.x == 0) {
        a.part[blockIdx.x] = tp;
        a.part[kBwdBlocks + blockIdx.x] = tq;
    }
}

template <typename T>
__global__ void bwd_apply_kernel(const BwdArgs<T>* batch, const T* grad_out)
{
    const BwdArgs<T>& a = batch[blockIdx.y];
    __shared__ double red[32];
    __shared__ double means[2];
    const double sp = block_sum_parts(a.part, kBwdBlocks, red);
    const double sq = block_sum_parts(a.part + kBwdBlocks, kBwdBlocks, red);
    if (threadIdx.x == 0) { means[0] = sp / (double)a.N; means[1] = sq / (double)a.N; }
    __syncthreads();
    const double g = (double)grad_out[blockIdx.y];
    const double hd = 1.0 / (double)a.N;
    const T fmu = (T)(2.0 * hd * g / a.mass_mu), fnu = (T)(2.0 * hd * g / a.mass_nu);
    const T mpsi = (T)means[0], mphi = (T)means[1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.N;
         i += (long long)gridDim.x * blockDim.x) {
        if (a.gmu) a.gmu[i] = fmu * (a.psi[i] - mpsi);
        if (a.gnu) a.gnu[i] = fnu * (a.phi[i] - mphi);
    }
}

static size_t bwd_bytes(int nprob)
{
    return up256((size_t)nprob * sizeof(BwdArgs<double>)) + up256((size_t)nprob * 2 * kBwdBlocks * sizeof(double));
}

template <typename T>
static bfm_status backward_impl(int nprob, const Grid* gs, const void* const* phi, const void* const* psi,
                                const double* mass_mu, const double* mass_nu, const void* grad_out,
                                void* const* grad_mu, void* const* grad_nu, unsigned char* wsp,
                                cudaStream_t st)
{
    std::vector<BwdArgs<T>> h(nprob);
    double* parts = reinterpret_cast<double*>(wsp + up256((size_t)nprob * sizeof(BwdArgs<double>)));
    for (int p = 0; p < nprob; ++p) {
        h[p].phi = (const T*)phi[p];
        h[p].psi = (const T*)psi[p];
        h[p].gmu = grad_mu ? (T*)grad_mu[p] : nullptr;
        h[p].gnu = grad_nu ? (T*)grad_nu[p] : nullptr;
        h[p].N = gs[p].N;
        h[p].mass_mu = mass_mu[p];
        h[p].mass_nu = mass_nu[p];
        h[p].part = parts + (size_t)p * 2 * kBwdBlocks;
    }
    BwdArgs<T>* d = reinterpret_cast<BwdArgs<T>*>(wsp);
    BFM_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(BwdArgs<T>) * nprob, cudaMemcpyHostToDevice, st));
    bwd_sum_kernel<T><<<dim3(kBwdBlocks, nprob), 256, 0, st>>>(d);
    BFM_LAUNCH_CHECK("bwd_sum_kernel");
    bwd_apply_kernel<T><<<dim3(kBwdBlocks, nprob), 256, 0, st>>>(d, (const T*)grad_out);
    BFM_LAUNCH_CHECK("bwd_apply_kernel");
    // the argument array is host memory read by the copy: wait before returning
    BFM_CUDA(cudaStreamSynchronize(st));
    return BFM_OK;
}

}  // namespace bfm

// ===========================================================================
// C ABI
// ===========================================================================
using namespace bfm;

extern "C" size_t bfm_workspace_bytes_batched(int nprob, const bfm_grid* grids, bfm_precision prec,
                                              int max_iter)
{
    if (nprob <= 0 || !grids || max_iter < 0) return 0;
    BatchPlan bp;
    if (!plan_batch(nprob, grids, elem_bytes(prec), max_iter, &bp)) return 0;
    return bp.total;
}

extern "C" bfm_status bfm_solve_batched(int nprob, const void* const* mu, const void* const* nu,
                                        const bfm_grid* grids, bfm_cost cost, bfm_precision prec,
                                        double tol, int max_iter, const bfm_options* opt,
                                        void* workspace, size_t workspace_bytes, void* stream,
                                        bfm_result* outs)
{
    if (prec != BFM_FP32 && prec != BFM_FP64) return BFM_ERR_INVALID_ARG;
    if (cost != BFM_COST_QUADRATIC) { set_last_error("only the quadratic cost is implemented"); return BFM_ERR_UNSUPPORTED; }
    if (nprob <= 0 || !mu || !nu || !grids || !outs || !(tol >= 0.0) || max_iter < 0 ||
        max_iter > 10000000 || nprob > 65535) {
        set_last_error("bad batch arguments");
        return BFM_ERR_INVALID_ARG;
    }
    for (int p = 0; p < nprob; ++p) {
        Grid g;
        if (!make_grid(&grids[p], &g)) { set_last_error("bad grid in batch"); return BFM_ERR_INVALID_ARG; }
        if (!fft_sizes_ok(g)) { set_last_error("every n[a] must be 2^p 3^q"); return BFM_ERR_UNSUPPORTED; }
        if (!mu[p] || !nu[p] || !outs[p].phi || !outs[p].psi) return BFM_ERR_INVALID_ARG;
    }
    BatchPlan bp;
    plan_batch(nprob, grids, elem_bytes(prec), max_iter, &bp);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < bp.total) {
        set_last_error("workspace NULL, not 256-byte aligned or smaller than bfm_workspace_bytes_batched()");
        return BFM_ERR_WORKSPACE;
    }
    bfm_options o;
    bfm_default_options(&o);
    if (opt) o = *opt;
    if (o.warm_start) { set_last_error("warm start is not supported in batched solves"); return BFM_ERR_UNSUPPORTED; }
    if (o.method != BFM_BACK_AND_FORTH) {
        set_last_error("batched solves run the back-and-forth iteration only");
        return BFM_ERR_UNSUPPORTED;
    }
    if (o.cost_p[0] != 0.0 || o.cost_p[1] != 0.0 || o.cost_p[2] != 0.0) {
        set_last_error("batched solves use the quadratic cost only");
        return BFM_ERR_UNSUPPORTED;
    }
    if (!(o.beta1 > 0 && o.beta1 < o.beta2 && o.beta2 < 1 && o.alpha1 > 1 && o.alpha2 > 0 &&
          o.alpha2 < 1 && o.sigma_min >= 0))
        return BFM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* wsp = (unsigned char*)workspace;
    if (prec == BFM_FP32)
        return solve_batched_impl<float>(nprob, mu, nu, bp, tol, max_iter, o, wsp, st, outs);
    return solve_batched_impl<double>(nprob, mu, nu, bp, tol, max_iter, o, wsp, st, outs);
}

extern "C" size_t bfm_w2_backward_workspace_bytes(int nprob)
{
    return nprob > 0 ? bwd_bytes(nprob) : 0;
}

extern "C" bfm_status bfm_w2_backward(int nprob, const bfm_grid* grids, bfm_precision prec,
                                      const void* const* phi, const void* const* psi,
                                      const double* mass_mu, const double* mass_nu,
                                      const void* grad_out, void* const* grad_mu,
                                      void* const* grad_nu, void* workspace,
                                      size_t workspace_bytes, void* stream)
{
    if (prec != BFM_FP32 && prec != BFM_FP64) return BFM_ERR_INVALID_ARG;
    if (nprob <= 0 || nprob > 65535 || !grids || !phi || !psi || !mass_mu || !mass_nu || !grad_out ||
        (!grad_mu && !grad_nu))
        return BFM_ERR_INVALID_ARG;
    std::vector<Grid> gs(nprob);
    for (int p = 0; p < nprob; ++p) {
        if (!make_grid(&grids[p], &gs[p]) || !phi[p] || !psi[p] || !(mass_mu[p] > 0) ||
            !(mass_nu[p] > 0))
            return BFM_ERR_INVALID_ARG;
    }
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < bwd_bytes(nprob))
        return BFM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == BFM_FP32)
        return backward_impl<float>(nprob, gs.data(), phi, psi, mass_mu, mass_nu, grad_out, grad_mu,
                                    grad_nu, (unsigned char*)workspace, st);
    return backward_impl<double>(nprob, gs.data(), phi, psi, mass_mu, mass_nu, grad_out, grad_mu,
                                 grad_nu, (unsigned char*)workspace, st);
}
