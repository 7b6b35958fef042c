// common.cu -- host helpers: status strings, CUDA error capture, grid and
// line-tile bookkeeping.
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"

namespace bfm {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* msg)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

bfm_status cuda_status(cudaError_t e, const char* where)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
    set_last_error(buf);
    return BFM_ERR_CUDA;
}

bool make_grid(const bfm_grid* g, Grid* out)
{
    if (!g || (g->ndim != 2 && g->ndim != 3)) return false;
    out->ndim = g->ndim;
    out->N = 1;
    for (int a = 0; a < 3; ++a) {
        const int na = (a < g->ndim) ? g->n[a] : 1;
        if (a < g->ndim && (na < 2 || na > kMaxN)) return false;
        out->n[a] = na;
        out->stride[a] = out->N;
        out->N *= na;
    }
    return true;
}

LineTiles make_tiles(const Grid& g, int axis, int W)
{
    LineTiles lt;
    lt.axis = axis;
    lt.n = g.n[axis];
    lt.es = g.stride[axis];
    lt.contig = (axis == 0);
    lt.W = W;
    lt.nlines = g.N / g.n[axis];
    lt.nfast = g.n[0];
    if (lt.contig) {
        lt.os = 0;
        lt.tiles_per_outer = 0;
        lt.ntiles = (lt.nlines + W - 1) / W;
    } else {
        // the outer index runs over the axis that is neither 0 nor `axis`
        lt.os = (axis == 1) ? (long long)g.n[0] * g.n[1] : (long long)g.n[0];
        lt.tiles_per_outer = (g.n[0] + W - 1) / W;
        const long long outers = lt.nlines / g.n[0];
        lt.ntiles = outers * lt.tiles_per_outer;
    }
    return lt;
}

int num_sms()
{
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

}  // namespace bfm

extern "C" const char* bfm_status_string(bfm_status s)
{
    switch (s) {
        case BFM_OK: return "BFM_OK";
        case BFM_NOT_CONVERGED: return "BFM_NOT_CONVERGED";
        case BFM_ERR_INVALID_ARG: return "BFM_ERR_INVALID_ARG";
        case BFM_ERR_NONFINITE: return "BFM_ERR_NONFINITE";
        case BFM_ERR_CUDA: return "BFM_ERR_CUDA";
        case BFM_ERR_TIMEOUT: return "BFM_ERR_TIMEOUT";
        case BFM_ERR_UNSUPPORTED: return "BFM_ERR_UNSUPPORTED";
        case BFM_ERR_WORKSPACE: return "BFM_ERR_WORKSPACE";
    }
    return "BFM_UNKNOWN_STATUS";
}

extern "C" const char* bfm_last_error(void)
{
    return bfm::g_last_error;
}

extern "C" void bfm_default_options(bfm_options* o)
{
    if (!o) return;
    o->beta1 = 0.25;
    o->beta2 = 0.75;
    o->alpha1 = 1.25;
    o->alpha2 = 0.8;
    o->sigma0 = 0.0;
    o->sigma_min = 0.01;
    o->poll_every = 4;
    o->warm_start = 0;
    o->method = BFM_BACK_AND_FORTH;
    o->cost_p[0] = o->cost_p[1] = o->cost_p[2] = 0.0;
}
