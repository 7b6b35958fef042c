// kernels.h -- internal launch interface between the library's .cu files.
#pragma once

#include "common.cuh"

namespace bfm {

struct CtPlan {
    int K, G, W, LD, LDI, LDH, threads;
    int ioff = 0;             // row kernel: byte offset of the int scratch
    int soff = 0;             // row kernel on interleaved tiles: byte offset of the output tile
    size_t smem;
    LineTiles tiles;
};

struct FftRadices {
    int nst;
    int r[kMaxStages];
};

struct AxisTables {
    int n;
    FftRadices rs;
    void* tw;                 // complex, n
    void* dtw;                // complex, n
    unsigned short* drev;     // n
    void* lam;                // n, element type of the call
    void* ptw;                // FP32 power-of-two lines: per-pass twiddles of the
                              // register FFT (n - 1 complex floats), else NULL
};

struct DctPlan {
    int G, W, LDZ, threads;
    int fast;                 // FP32 power-of-two line: register Stockham kernel
    size_t smem;
    LineTiles tiles;
};

// c-transform launch shapes: K cells per thread, W lines per CTA (0: as many
// as the thread and shared-memory limits allow), per kernel kind
enum { CT_KIND_TILE_ROWS = 0, CT_KIND_TILE_COLS = 1, CT_KIND_ROW = 2, CT_KIND_ROW_COLS = 3 };
struct CtShape { int K, W; };
int ct_kind(const Grid& g, int axis, int elem_bytes);
CtShape ct_default_shape(int kind, int n, int elem_bytes);
int ct_shape_candidates(int kind, int n, int elem_bytes, CtShape* out, int cap);
bool ct_shape_valid(int kind, int n, int elem_bytes, CtShape s);
bool ct_tuned_shape(int kind, int n, int elem_bytes, CtShape* s);
void ct_set_tuned_shape(int kind, int n, int elem_bytes, CtShape s);
void ct_erase_tuned_shape(int kind, int n, int elem_bytes);
void ct_clear_tuned_shapes();

CtPlan plan_ct_pass(const Grid& g, int axis, int elem_bytes);          // tuned shape, else default
CtPlan plan_ct_pass_default(const Grid& g, int axis, int elem_bytes);  // hand-picked shape
DctPlan plan_dct_pass(const Grid& g, int axis, int elem_bytes);

// number of CTAs (= partial sums) launch_ct_pass uses for this pass.  row_ctr
// (optional, device, two ints that are 0 between launches): rows of the row
// kernel are handed out by an atomic counter instead of a fixed stride
int ct_pass_blocks(const Grid& g, int axis, int elem_bytes, int max_blocks);
template <typename T>
bfm_status launch_ct_pass(const Grid& g, int axis, const T* in, T* out, bool negate,
                          const T* w_in, double* part_in, const T* w_out, double* part_out,
                          const int* done, int max_blocks, cudaStream_t st, int* blocks_used,
                          int* row_ctr = nullptr);

bool fft_radices(int n, FftRadices* rs);
size_t axis_table_bytes(int n, int elem_bytes);
// Pointers and radices of one axis's tables inside `ws` (deterministic, so any
// view of a workspace can rebuild them without touching the device).
bool layout_axis_tables(int n, int elem_bytes, unsigned char* ws, AxisTables* t);

template <typename T>
bfm_status fill_axis_tables(int n, AxisTables* t, unsigned char* ws, cudaStream_t st);

enum { PASS_FWD = 0, PASS_MID = 1, PASS_INV = 2 };

template <typename T>
bfm_status launch_dct_pass(const Grid& g, int axis, int mode, const AxisTables* tabs,
                           const T* in, const T* base, T* out, const T* upd,
                           const double* sigma, double* part, const int* done,
                           cudaStream_t st, int* blocks_used);

// scatter.cu (p: exponents of a separable power cost, NULL for the quadratic cost)
template <typename T>
bfm_status launch_pushforward(const Grid& g, const T* psi, const T* mu, T* rho,
                              const int* done, cudaStream_t st, const double* p = nullptr);
// 2-D: psi~ and mu in the transposed layout (gt), rho out in g's layout;
// part: per-CTA FP64 partials of <psi~, mu> (their number in *blocks_used)
template <typename T>
bfm_status launch_pushforward_t(const Grid& gt, const T* psi_t, const T* mu_t, T* rho,
                                const Grid& g, const int* done, cudaStream_t st, double* part,
                                int* blocks_used);
template <typename T>
bfm_status launch_map(const Grid& g, const T* psi, T* map, cudaStream_t st,
                      const double* p = nullptr);

// ctpower.cu: one 1-D c-transform pass of the separable power cost along
// `axis` with exponent p (same arguments as launch_ct_pass)
template <typename T>
bfm_status launch_ct_power_pass(const Grid& g, int axis, double p, const T* in, T* out, bool negate,
                                const T* w_in, double* part_in, const T* w_out, double* part_out,
                                const int* done, int max_blocks, cudaStream_t st, int* blocks_used);
template <typename T>
bfm_status launch_interpolate(const Grid& g, const T* map, const T* mu, double t, T* rho,
                              cudaStream_t st);

// batched forms: one launch per kernel step for a class of problems sharing a
// grid shape; per-problem arguments live in a device array (blockIdx.y)
template <typename T> int ct_batch_blocks(const Grid& g, int axis);
size_t ct_args_bytes(int elem_bytes);
template <typename T>
void fill_ct_batch_args(const Grid& g, int axis, const T* in, T* out, bool negate, const T* w_in,
                        double* part_in, const T* w_out, double* part_out, const int* done,
                        void* host_slot);
template <typename T>
bfm_status launch_ct_pass_batched(const Grid& g, int axis, int nprob, const void* dev_args,
                                  cudaStream_t st);
template <typename T> int dct_batch_blocks(const Grid& g, int axis);
size_t dct_args_bytes(int elem_bytes);
template <typename T>
bfm_status fill_dct_batch_args(const Grid& g, int axis, const AxisTables* tabs, const T* in,
                               const T* base, T* out, const T* upd, const double* sigma,
                               double* part, const int* done, void* host_slot);
// rows16: every problem's fields are 16-byte aligned (rows may move as float4)
template <typename T>
bfm_status launch_dct_pass_batched(const Grid& g, int axis, int mode, int nprob,
                                   const void* dev_args, cudaStream_t st, bool rows16);
size_t push_args_bytes(int elem_bytes);
template <typename T>
void fill_push_batch_args(const Grid& g, const T* psi, const T* mu, T* rho, const int* done,
                          void* host_slot);
template <typename T>
bfm_status launch_pushforward_batched(int ndim, long long max_cells, int nprob,
                                      const void* dev_args, cudaStream_t st);

// layout.cu: out (C rows of R elements) = transpose of in (R rows of C
// elements); with w (laid out like out), one FP64 partial sum of out * w per CTA
template <typename T>
bfm_status launch_transpose(const T* in, T* out, int R, int C, const T* w, double* part,
                            const int* done, cudaStream_t st, int* blocks_used);
// true when axis-1 sweeps of this 2-D grid run as row sweeps of a transposed copy
bool transposed_axis1(const Grid& g, int elem_bytes);
Grid transposed_grid(const Grid& g);

// solver.cu: the Poisson solve on an explicit scratch block
size_t poisson_scratch_bytes(const Grid& g, int eb);
bfm_status poisson_on_scratch(const void* f, void* g_out, const Grid& g, bfm_precision prec,
                              double* G_out, unsigned char* scratch, cudaStream_t st);

}  // namespace bfm
