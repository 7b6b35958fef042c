// ctransform.cu -- the grid c-transform for the quadratic cost (Section 4.1).
//
// phi^c(x) = min_y |x-y|^2/2 - phi(y) splits into 1-D passes along each axis
// (Section 4.1, dimension splitting): pass 1 takes f = -phi, later passes take
// the previous output.  A 1-D pass on a line of n cells computes
//     u(i) = min_j  hh (i - j)^2 + f(j),     hh = h^2 / 2,
// i.e. the lower envelope of n parabolas of equal curvature.  The paper
// evaluates it through the Legendre transform and a convex-hull sweep; here
// the same envelope is built in parallel by a thread group per line (a CTA
// holds several lines: whole rows, or interleaved tiles of neighbouring
// columns; in a solve, rows and column tiles are handed out by a counter):
//   A. each thread builds the envelope of its own K consecutive parabolas
//      with a stack kept in place over its cells (a parabola b between a and
//      c is hidden when the a/b crossing lies right of the b/c crossing);
//   B. the chunk envelopes are joined by rounds: a parabola is on the line's
//      envelope iff its lifted point is on the lower convex hull, and in the
//      concatenation of the chunk stacks only stack ends can be reflex, so in
//      a round every thread drops the first entries that lie on or above the
//      chord from the left neighbour's last entry and the last entries on or
//      above the chord to the right neighbour's first (each boundary by one
//      direct test and a binary search); rounds repeat until none drops, a
//      line still changing after a fixed number of rounds finishes with
//      pairwise merges of neighbouring stacks;
//   C. the non-empty stacks are listed in order (the tile kernel compacts
//      the surviving parabolas into one list);
//   D. FP32: every envelope parabola computes the first cell it owns from its
//      predecessor; the row kernel finds each cell's owner by the rank of the
//      owners' start cells, the tile kernel by marks at the start cells; FP64
//      lines, and lines whose start cells decrease under rounding, find the
//      owner of a thread's first cell by binary search and sweep its outputs.
// The division-free hidden test compares second differences:
//   b hidden by (a, c)  <=>  (f_b-f_a)(c-b) - (f_c-f_b)(b-a) >= hh (c-a)(b-a)(c-b).
// Optional FP64 dot products of the input and of the output with weight
// fields (the two terms of the dual value J, eq. (defJ)) are fused into the
// load and store sweeps and written as one partial sum per CTA.
#include <string.h>

#include <map>
#include <mutex>

#include <type_traits>

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
    int LDI;              // shared leading dimension of the index stacks
    int LDH;              // shared leading dimension of the compacted envelope
    T hh;                 // h^2 / 2 on this axis
    int negate;           // the pass reads -in
    int vec4;             // rows may be moved as float4 (n % 4 == 0, 16-byte aligned)
    int lw;               // log2(W); interleaved tiles have W a power of two
    int ioff;             // row kernel: byte offset of the int scratch in shared memory
    int soff;             // row kernel on interleaved tiles: byte offset of the output tile
    int* ctr;             // row kernel on rows: [0] next row to take, [1] groups finished
};

// Shared-memory layout of a line: thread t owns cells [tK, tK+K).  Stored
// plainly, the threads of a warp would touch cells K apart, a K-way bank
// conflict; one pad word per chunk for the values (two shorts for the index
// stacks) makes the per-thread stride odd, so the threads of a warp hit
// distinct banks.
template <int K> struct Skew {
    static constexpr int lg = (K >= 32) ? 5 : (K >= 16) ? 4 : (K >= 8) ? 3 : (K >= 4) ? 2 : (K >= 2) ? 1 : 0;
    __device__ __forceinline__ static int f(int p) { return p + (p >> lg); }
    __device__ __forceinline__ static int s(int p) { return p + 2 * (p >> lg); }
};

// The four products of a pair of float4 summed in FP32 (one FMA chain): the
// dual dots add one such sum per vector to their compensated accumulators.
__device__ __forceinline__ float dot4(const float4 a, const float4 b)
{
    float s = a.x * b.x;
    s = fmaf(a.y, b.y, s);
    s = fmaf(a.z, b.z, s);
    return fmaf(a.w, b.w, s);
}

template <int K, typename T>
__device__ __forceinline__ bool hidden(const T* f, int a, int b, int c, T hh)
{
    const T fa = f[Skew<K>::f(a)], fb = f[Skew<K>::f(b)], fc = f[Skew<K>::f(c)];
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

template <typename T>
__device__ __forceinline__ bool hidden_v(int a, T fa, int b, T fb, int c, T fc, T hh)
{
    const T lhs = (fb - fa) * (T)(c - b) - (fc - fb) * (T)(b - a);
    const T rhs = hh * (T)(c - a) * (T)(b - a) * (T)(c - b);
    return lhs >= rhs;
}

// Phase B: merge the envelopes of thread groups [t, t+s) and [t+s, t+2s).
// beg/end hold chunk-space positions into the stacks; the parabola at stack
// position p has its index in stk and its value in f at that position (the
// stacks are built in place over the line values).  The left chain's last
// two parabolas (a, b) and the right chain's first two (c, d) stay in
// registers, so a pop costs one pair of independent loads.
template <int K, typename T>
__device__ void merge_pair(const T* f, const short* stk, short* beg, short* end,
                           int t, int s, int n, T hh)
{
    using SK = Skew<K>;
    const int tl = t, tm = t + s, tr = t + 2 * s;
    int lt = tm - 1;
    while (lt >= tl && beg[lt] == end[lt]) --lt;
    int rt = tm;
    while (rt < tr && beg[rt] == end[rt]) ++rt;
    if (lt < tl || rt >= tr) return;
    // left: b at (lt, pb), a at (la, pa)
    int pb = end[lt] - 1;
    int la = lt, pa = pb - 1, begla = beg[lt];
    if (pa < begla) {
        la = lt - 1;
        while (la >= tl && beg[la] == end[la]) --la;
        if (la >= tl) { pa = end[la] - 1; begla = beg[la]; } else pa = -1;
    }
    // right: c at (rt, pc), d at (rd, pd)
    int pc = beg[rt];
    int rd = rt, pd = pc + 1, endrd = end[rt];
    if (pd >= endrd) {
        rd = rt + 1;
        while (rd < tr && beg[rd] == end[rd]) ++rd;
        if (rd < tr) { pd = beg[rd]; endrd = end[rd]; } else pd = -1;
    }
    int ib = stk[SK::s(pb)], ic = stk[SK::s(pc)];
    T fb = f[SK::f(pb)], fc = f[SK::f(pc)];
    int ia = -1, id = -1;
    T fa = (T)0, fd = (T)0;
    if (pa >= 0) { ia = stk[SK::s(pa)]; fa = f[SK::f(pa)]; }
    if (pd >= 0) { id = stk[SK::s(pd)]; fd = f[SK::f(pd)]; }
    for (int guard = 0; guard <= n + 2; ++guard) {
        if (ia >= 0 && hidden_v(ia, fa, ib, fb, ic, fc, hh)) {
            // pop b; if it was the last parabola of thread lt, that segment empties
            if (la != lt) { end[lt] = beg[lt]; lt = la; }
            pb = pa; ib = ia; fb = fa;
            pa = pa - 1;
            if (pa < begla) {
                la = la - 1;
                while (la >= tl && beg[la] == end[la]) --la;
                if (la >= tl) { pa = end[la] - 1; begla = beg[la]; } else pa = -1;
            }
            if (pa >= 0) { ia = stk[SK::s(pa)]; fa = f[SK::f(pa)]; } else ia = -1;
            continue;
        }
        if (id >= 0 && hidden_v(ib, fb, ic, fc, id, fd, hh)) {
            // pop c; if it was the last parabola of thread rt, that segment empties
            if (rd != rt) { beg[rt] = end[rt]; rt = rd; }
            pc = pd; ic = id; fc = fd;
            pd = pd + 1;
            if (pd >= endrd) {
                rd = rd + 1;
                while (rd < tr && beg[rd] == end[rd]) ++rd;
                if (rd < tr) { pd = beg[rd]; endrd = end[rd]; } else pd = -1;
            }
            if (pd >= 0) { id = stk[SK::s(pd)]; fd = f[SK::f(pd)]; } else id = -1;
            continue;
        }
        break;
    }
    end[lt] = (short)(pb + 1);
    beg[rt] = (short)pc;
}

// Barrier over the G threads of one line: a line of 32 or fewer threads lies
// in one warp; larger lines (whole warps, at most 8 per CTA) use named
// barrier 1 + w so the lines of a CTA do not wait for one another.
__device__ __forceinline__ void line_sync(int w, int G)
{
    if (G <= 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" :: "r"(1 + w), "r"(G) : "memory");
}

constexpr int kU = 4;      // column-tile loads each thread keeps in flight

// OR of a predicate over the line group of G threads, which also synchronises
// it (lines of at most 32 threads: the whole warp, all of whose lines run the
// same rounds)
__device__ __forceinline__ bool group_or(bool v, int w, int G)
{
    if (G <= 32) return __any_sync(0xffffffffu, v);
    unsigned r;
    asm volatile("{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\t"
                 "bar.red.or.pred po, %2, %3, pi;\n\tselp.u32 %0, 1, 0, po;\n\t}"
                 : "=r"(r) : "r"(v ? 1u : 0u), "r"(1 + w), "r"(G) : "memory");
    return r != 0;
}

constexpr int kFixRounds = 6;          // tile lines: fix-up rounds before the merges take over
constexpr int kFixRoundsRow = 16;      // row groups: the same

// Parabola indices held in T: differences of indices below 2^24 are exact in
// FP32, so these give the same values as the integer forms above while
// avoiding integer-to-float conversions (a fraction of the FP32 rate).
template <typename T>
__device__ __forceinline__ bool hidden_t(T a, T fa, T b, T fb, T c, T fc, T hh)
{
    const T lhs = (fb - fa) * (c - b) - (fc - fb) * (b - a);
    const T rhs = hh * (c - a) * (b - a) * (c - b);
    return lhs >= rhs;
}

template <typename T>
__device__ __forceinline__ T parab_t(T hh, T x, T j, T fj)
{
    const T d = x - j;
    return fma(hh, d * d, fj);
}

// First grid cell owned by parabola b, the successor of a on the envelope
// (FP32): the two meet at s = (f_b - f_a) / (2 hh (j_b - j_a)) + (j_a + j_b)/2
// and b is the lower one right of s, so the cell is ceil(s), clamped to
// [0, n].  For neighbours j_b - j_a < 16 apart an error of the rounded s
// moves at most values within a fraction of an ulp; for wider gaps, where
// the two parabolas separate faster, the cell is confirmed by comparing the
// evaluated parabolas at it and at the cell before (the comparison the
// sequential sweep makes), which the rounded s misses by at most one cell.
__device__ __forceinline__ int start_cell(float ja, float fa, float jb, float fb, float hh, int n)
{
    const float d = jb - ja;
    const float q = __fdividef(fb - fa, (2.f * hh) * d);
    const float s = fmaf(0.5f, ja + jb, q);
    int c = (int)fminf(fmaxf(ceilf(s), 0.f), (float)n);
    if (d >= 16.f && c > 0) {
        const float x = (float)c;
        if (c < n && !(parab_t(hh, x, jb, fb) <= parab_t(hh, x, ja, fa))) ++c;
        else if (parab_t(hh, x - 1.f, jb, fb) <= parab_t(hh, x - 1.f, ja, fa)) --c;
    }
    return c;
}

// Phase B as rounds of a parallel fix-up.  A parabola is on the envelope iff
// its lifted point (j, f_j + hh j^2) is on the lower convex hull of the line's
// points, and a point that lies on or above a chord between two other points
// of the line (one on each side) is not.  Each chunk stack is a convex chain,
// so in their concatenation only the stacks' ends can be reflex: in a round
// every thread reads the ends of the neighbouring non-empty stacks, then drops
// its own first entries while they lie on or above the chord from the left
// neighbour's last entry a to the entry after them, and its last entries
// while they lie on or above the chord from the entry before them to the
// right neighbour's first entry c.  The rounds end when no thread of the line
// dropped anything: the stacks then form the hull.
//
// Along a convex chain b_0, b_1, ... the slope from a to b_{k+1} is a
// weighted mean of the slope from a to b_k and the chain's slope from b_k to
// b_{k+1}; so the first test ("b_k on or above the chord a b_{k+1}", i.e. the
// slope a->b_k is at least the chain's slope at b_k) holds for a prefix of
// the chain and fails from the first k where it fails (the tangent from a).
// Mirrored, the second test holds for a suffix.  Each boundary is therefore
// found by one direct test and, only when that one drops, a binary search:
// at most 1 + log2(K) tests instead of up to K dependent ones.  The test of
// the stack's last entry against c (after all others dropped) is not part of
// the chain and is made last, as the sequential scan makes it.
template <int K, typename T>
__device__ __forceinline__ void drop_ends(const T* f, const short* stk, int& b0, int& e1,
                                          int pa, int pc, T hh)
{
    using SK = Skew<K>;
    auto J = [&](int p) { return (T)stk[SK::s(p)]; };
    auto V = [&](int p) { return f[SK::f(p)]; };
    T jc = (T)0, fc = (T)0;
    if (pc >= 0) { jc = J(pc); fc = V(pc); }
    if (pa >= 0) {
        const T ja = J(pa), fa = V(pa);
        // entry p (p + 1 < e1) on or above the chord from a to entry p + 1
        auto front = [&](int p) { return hidden_t(ja, fa, J(p), V(p), J(p + 1), V(p + 1), hh); };
        int p = b0;
        if (e1 - b0 >= 2 && front(b0)) {
            int lo = b0 + 1, hi = e1 - 1;          // first failing test in [b0 + 1, e1 - 2], else e1 - 1
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (front(mid)) lo = mid + 1;
                else hi = mid;
            }
            p = lo;
        }
        if (p == e1 - 1 && pc >= 0 && hidden_t(ja, fa, J(p), V(p), jc, fc, hh)) p = e1;
        b0 = p;
    }
    if (pc >= 0 && e1 - 1 > b0) {
        // entry p (p > b0) on or above the chord from entry p - 1 to c
        auto back = [&](int p) { return hidden_t(J(p - 1), V(p - 1), J(p), V(p), jc, fc, hh); };
        if (back(e1 - 1)) {
            int lo = b0 + 1, hi = e1 - 1;          // first holding test in [b0 + 1, e1 - 1]
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (back(mid)) hi = mid;
                else lo = mid + 1;
            }
            e1 = lo;
        }
    }
}

// One round for lines of a tile (G threads per line, possibly several lines
// per warp); the neighbouring non-empty stacks are found by scanning.
// Returns whether any thread of the line group dropped anything.
template <int K, typename T>
__device__ __forceinline__ bool fix_round(const T* f, const short* stk, short* beg, short* end,
                                          int t, int G, int w, T hh, bool active)
{
    int b0 = 0, e1 = 0, pa = -1, pc = -1;          // own range, neighbours' end entries
    if (active) {
        b0 = beg[t];
        e1 = end[t];
        if (e1 > b0) {
            int pv = t - 1;
            while (pv >= 0 && beg[pv] == end[pv]) --pv;
            int nx = t + 1;
            while (nx < G && beg[nx] == end[nx]) ++nx;
            if (pv >= 0) pa = end[pv] - 1;
            if (nx < G) pc = beg[nx];
        }
    }
    if (G <= 32) __syncwarp();                     // every read before any update
    else asm volatile("bar.sync %0, %1;" :: "r"(1 + w), "r"(G) : "memory");
    bool dropped = false;
    if (e1 > b0) {
        const int ob = b0, oe = e1;
        drop_ends<K>(f, stk, b0, e1, pa, pc, hh);
        dropped = (b0 != ob) || (e1 != oe);
        if (dropped) { beg[t] = (short)b0; end[t] = (short)e1; }
    }
    return group_or(dropped, w, G);                // also publishes the updates
}

// BATCHED: blockIdx.y selects the problem, whose arguments come from `batch`.
template <typename T, int K, bool CONTIG, bool BATCHED>
__global__ void __launch_bounds__(512, 2) ct_pass_kernel(CtArgs<T> a0, const CtArgs<T>* batch)
{
    const CtArgs<T>& a = BATCHED ? batch[blockIdx.y] : a0;
    if (BATCHED && blockIdx.x >= a.lt.ntiles) return;
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SK = Skew<K>;
    const LineTiles& lt = a.lt;
    const int n = lt.n;
    const int G = a.G;
    const int W = lt.W;
    T* fs = reinterpret_cast<T*>(smem_raw);
    T* hval_all = fs + (size_t)W * a.LD;
    short* stk_all = reinterpret_cast<short*>(hval_all + (size_t)W * a.LDH);
    short* hidx_all = stk_all + (size_t)W * a.LDI;
    short* beg_all = hidx_all + (size_t)W * a.LDH;
    short* end_all = beg_all + (size_t)W * G;
    int* wsum_all = reinterpret_cast<int*>(end_all + (size_t)W * G);   // 4-byte aligned
    const int nwl = (G + 31) / 32;                 // warps per line
    int* htot = wsum_all + W * nwl;
    __shared__ double red[32];

    const int tid = threadIdx.x;
    const int w = tid / G, t = tid - w * G;
    const int lane = tid & 31;
    T* f = fs + (size_t)w * a.LD;
    T* hval = hval_all + (size_t)w * a.LDH;
    short* stk = stk_all + (size_t)w * a.LDI;
    short* hidx = hidx_all + (size_t)w * a.LDH;
    short* beg = beg_all + w * G;
    short* end = end_all + w * G;
    const T hh = a.hh;
    const int lo = t * K;
    const int hi = min(lo + K, n);

    double acc_in = 0.0, acc_out = 0.0;
    Acc<T> acc_t_in, acc_t_out;

    for (long long tile = blockIdx.x; tile < lt.ntiles; tile += gridDim.x) {
        const Tile tl = tile_at(lt, tile);
        // ---- load ----------------------------------------------------------
        if (CONTIG) {
            for (int ww = 0; ww < tl.wact; ++ww) {
                const long long rb = tl.base0 + (long long)ww * n;
                T* frow = fs + (size_t)ww * a.LD;
                if (sizeof(T) == 4 && a.vec4) {
                    const float4* src = reinterpret_cast<const float4*>(a.in + rb);
                    const float4* wsrc = reinterpret_cast<const float4*>(a.w_in + rb);
                    for (int q = tid; q < (n >> 2); q += blockDim.x) {
                        float4 v = src[q];
                        if (a.w_in) acc_t_in.add(dot4(v, wsrc[q]));
                        if (a.negate) { v.x = -v.x; v.y = -v.y; v.z = -v.z; v.w = -v.w; }
                        frow[SK::f(4 * q)] = v.x;     frow[SK::f(4 * q + 1)] = v.y;
                        frow[SK::f(4 * q + 2)] = v.z; frow[SK::f(4 * q + 3)] = v.w;
                    }
                } else {
                    for (int p = tid; p < n; p += blockDim.x) {
                        const T v = a.in[rb + p];
                        if (a.w_in) acc_t_in.add_prod(v, a.w_in[rb + p]);
                        frow[SK::f(p)] = a.negate ? -v : v;
                    }
                }
            }
        } else {
            // a column tile reads W neighbouring floats per row, so every
            // thread keeps kU loads in flight before storing any of them
            const int total = n << a.lw;
            const int nt = blockDim.x;
            for (int e0 = tid; e0 < total; e0 += kU * nt) {
                T v[kU], u[kU];
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int e = e0 + k * nt;
                    const int p = e >> a.lw, ww = e & (W - 1);
                    const bool ok = e < total && ww < tl.wact;
                    const long long ad = tl.base0 + ww + (long long)p * lt.es;
                    v[k] = ok ? a.in[ad] : (T)0;
                    u[k] = (ok && a.w_in) ? a.w_in[ad] : (T)0;
                }
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int e = e0 + k * nt;
                    const int p = e >> a.lw, ww = e & (W - 1);
                    if (e < total && ww < tl.wact) {
                        if (a.w_in) acc_t_in.add_prod(v[k], u[k]);
                        fs[(size_t)ww * a.LD + SK::f(p)] = a.negate ? -v[k] : v[k];
                    }
                }
            }
        }
        __syncthreads();
        const bool active = (w < tl.wact);
        // ---- A: envelope of this thread's chunk ------------------------------
        // The stack lives in place: position p of the chunk holds the index
        // (stk) and value (f) of the p-th stacked parabola; a push writes at
        // the new top, which is never beyond the cell being read.
        if (active) {
            if (lo < n) {
                int top = lo;
                int s1 = lo, s0 = -1;
                T v1 = f[SK::f(lo)], v0 = (T)0;
                stk[SK::s(lo)] = (short)lo;
                for (int q = lo + 1; q < hi; ++q) {
                    const T vq = f[SK::f(q)];
                    while (s0 >= 0 && hidden_v(s0, v0, s1, v1, q, vq, hh)) {
                        --top;
                        s1 = s0; v1 = v0;
                        if (top > lo) { s0 = stk[SK::s(top - 1)]; v0 = f[SK::f(top - 1)]; }
                        else s0 = -1;
                    }
                    ++top;
                    stk[SK::s(top)] = (short)q;
                    f[SK::f(top)] = vq;
                    s0 = s1; v0 = v1;
                    s1 = q; v1 = vq;
                }
                beg[t] = (short)lo;
                end[t] = (short)(top + 1);
            } else {
                beg[t] = 0;
                end[t] = 0;
            }
        }
        line_sync(w, G);
        // ---- B: envelope of the whole line ------------------------------------
        // Rounds that drop reflex stack ends (see fix_round), then pairwise
        // merges for lines still changing after kFixRounds rounds.
        bool moved = true;
        for (int round = 0; round < kFixRounds && moved; ++round)
            moved = fix_round<K>(f, stk, beg, end, t, G, w, hh, active);
        if (moved) {
            for (int s = 1; s < G; s <<= 1) {
                if (active && (t & (2 * s - 1)) == 0 && t + s < G) merge_pair<K>(f, stk, beg, end, t, s, n, hh);
                // the next level merges groups of 4s threads: inside one warp a warp
                // barrier publishes this level's segment updates, else the line barrier
                if (4 * s <= 32) __syncwarp();
                else line_sync(w, G);
            }
            line_sync(w, G);
        }
        // ---- C: compaction of (index, value) pairs ---------------------------------
        const int cnt = active ? (end[t] - beg[t]) : 0;
        int incl = cnt;
        const int width = G < 32 ? G : 32;
        for (int d = 1; d < width; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d, width);
            if ((lane % width) >= d) incl += y;
        }
        if (G > 32) {
            if (active && (t & 31) == 31) wsum_all[w * nwl + (t >> 5)] = incl;
            line_sync(w, G);
            int add = 0;
            if (active)
                for (int i = 0; i < (t >> 5); ++i) add += wsum_all[w * nwl + i];
            incl += add;
        }
        if (active && t == G - 1) htot[w] = incl;
        if (active) {
            const int b0 = beg[t];
            const int excl = incl - cnt;
            for (int i = 0; i < cnt; ++i) {
                hidx[excl + i] = stk[SK::s(b0 + i)];
                hval[excl + i] = f[SK::f(b0 + i)];
            }
        }
        line_sync(w, G);
        bool walk = sizeof(T) != 4;
        if constexpr (sizeof(T) == 4) {
            // ---- D (FP32): owners by marks, no sweep ---------------------------------
            // The value array is free: each thread clears its cells to -1, then
            // every envelope parabola k computes the first cell it owns from its
            // predecessor (start_cell); a parabola owns cells iff the next one
            // starts later, and then writes k at its start cell.  The owner of
            // cell x is the last mark at or before x (marks grow with x).  A
            // start that decreases (rounding between nearly collinear parabolas)
            // sends the tile's lines to the sweep below.
            int* mk = reinterpret_cast<int*>(f);
            if (active)
                for (int x = lo; x < hi; ++x) mk[SK::f(x)] = -1;
            line_sync(w, G);
            bool bad = false;
            if (active && cnt > 0) {
                const int H = htot[w];
                const int k0 = incl - cnt;
                float jc = (float)hidx[k0], fc = (float)hval[k0];
                int cc = 0;
                if (k0 > 0) cc = start_cell((float)hidx[k0 - 1], (float)hval[k0 - 1], jc, fc, (float)hh, n);
                for (int k = k0; k < k0 + cnt; ++k) {
                    int cn = n;
                    float jn = 0.f, fn = 0.f;
                    if (k + 1 < H) {
                        jn = (float)hidx[k + 1]; fn = (float)hval[k + 1];
                        cn = start_cell(jc, fc, jn, fn, (float)hh, n);
                    }
                    bad |= cn < cc;
                    if (cn > cc) mk[SK::f(cc)] = k;
                    jc = jn; fc = fn; cc = cn;
                }
            }
            walk = group_or(bad, w, G);            // also publishes the marks
            if (!walk) {
                // the last mark in this thread's cells, then the last one before them
                int last = -1;
                if (active)
                    for (int x = hi - 1; x >= lo && last < 0; --x) last = mk[SK::f(x)];
                int inc = last;
                for (int d = 1; d < width; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, d, width);
                    if ((lane % width) >= d) inc = max(inc, y);
                }
                if (G > 32) {
                    if ((t & 31) == 31) wsum_all[w * nwl + (t >> 5)] = inc;
                    line_sync(w, G);
                    for (int i = 0; i < (t >> 5); ++i) inc = max(inc, wsum_all[w * nwl + i]);
                }
                // exclusive: the last mark of the threads before this one
                int prev = __shfl_up_sync(0xffffffffu, inc, 1, width);
                if ((lane % width) == 0) prev = -1;
                if (G > 32 && (lane % width) == 0)
                    for (int i = 0; i < (t >> 5); ++i) prev = max(prev, wsum_all[w * nwl + i]);
                if (active && lo < n) {
                    int kc = prev;
                    float jc = 0.f, fc = 0.f;
                    if (kc >= 0) { jc = (float)hidx[kc]; fc = (float)hval[kc]; }
                    for (int x = lo; x < hi; ++x) {
                        const int m = mk[SK::f(x)];
                        if (m >= 0) { kc = m; jc = (float)hidx[m]; fc = (float)hval[m]; }
                        f[SK::f(x)] = (T)parab_t((float)hh, (float)x, jc, fc);
                    }
                }
            }
        }
        if (walk) {
        // ---- D: evaluate this thread's outputs by a sweep into the (now free) value array
        // ---- D: evaluate this thread's outputs into the (now free) value array -----
        if (active && lo < n) {
            const int H = htot[w];
            int kl = 0, kh = H - 1;
            while (kl < kh) {
                const int mid = (kl + kh) >> 1;
                const int j0 = hidx[mid], j1 = hidx[mid + 1];
                const T g0 = hval[mid], g1 = hval[mid + 1];
                if (parab(hh, lo, j1, g1) < parab(hh, lo, j0, g0)) kl = mid + 1;
                else kh = mid;
            }
            int k = kl;
            int jc = hidx[k];
            T fc = hval[k];
            int jn = -1;
            T fn = (T)0;
            if (k + 1 < H) { jn = hidx[k + 1]; fn = hval[k + 1]; }
            for (int x = lo; x < hi; ++x) {
                T vc = parab(hh, x, jc, fc);
                while (jn >= 0) {
                    const T vn = parab(hh, x, jn, fn);
                    if (vn <= vc) {
                        ++k; jc = jn; fc = fn; vc = vn;
                        if (k + 1 < H) { jn = hidx[k + 1]; fn = hval[k + 1]; } else jn = -1;
                    } else break;
                }
                f[SK::f(x)] = vc;
            }
        }
        }
        __syncthreads();
        // ---- store ---------------------------------------------------------------
        if (CONTIG) {
            for (int ww = 0; ww < tl.wact; ++ww) {
                const long long rb = tl.base0 + (long long)ww * n;
                const T* frow = fs + (size_t)ww * a.LD;
                if (sizeof(T) == 4 && a.vec4) {
                    float4* dst = reinterpret_cast<float4*>(a.out + rb);
                    const float4* wsrc = reinterpret_cast<const float4*>(a.w_out + rb);
                    for (int q = tid; q < (n >> 2); q += blockDim.x) {
                        const float4 v = make_float4(frow[SK::f(4 * q)], frow[SK::f(4 * q + 1)],
                                                     frow[SK::f(4 * q + 2)], frow[SK::f(4 * q + 3)]);
                        dst[q] = v;
                        if (a.w_out) acc_t_out.add(dot4(v, wsrc[q]));
                    }
                } else {
                    for (int p = tid; p < n; p += blockDim.x) {
                        const T v = frow[SK::f(p)];
                        a.out[rb + p] = v;
                        if (a.w_out) acc_t_out.add_prod(v, a.w_out[rb + p]);
                    }
                }
            }
        } else {
            const int total = n << a.lw;
            const int nt = blockDim.x;
            for (int e0 = tid; e0 < total; e0 += kU * nt) {
                T u[kU];
                if (a.w_out) {
#pragma unroll
                    for (int k = 0; k < kU; ++k) {
                        const int e = e0 + k * nt;
                        const int p = e >> a.lw, ww = e & (W - 1);
                        const long long ad = tl.base0 + ww + (long long)p * lt.es;
                        u[k] = (e < total && ww < tl.wact) ? a.w_out[ad] : (T)0;
                    }
                }
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int e = e0 + k * nt;
                    const int p = e >> a.lw, ww = e & (W - 1);
                    if (e < total && ww < tl.wact) {
                        const long long ad = tl.base0 + ww + (long long)p * lt.es;
                        const T v = fs[(size_t)ww * a.LD + SK::f(p)];
                        a.out[ad] = v;
                        if (a.w_out) acc_t_out.add_prod(v, u[k]);
                    }
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


// merge_pair with the cached end parabolas' indices held in T
template <int K, typename T>
__device__ void merge_pair_t(const T* f, const short* stk, short* beg, short* end,
                             int t, int s, int n, T hh)
{
    using SK = Skew<K>;
    const int tl = t, tm = t + s, tr = t + 2 * s;
    int lt = tm - 1;
    while (lt >= tl && beg[lt] == end[lt]) --lt;
    int rt = tm;
    while (rt < tr && beg[rt] == end[rt]) ++rt;
    if (lt < tl || rt >= tr) return;
    int pb = end[lt] - 1;
    int la = lt, pa = pb - 1, begla = beg[lt];
    if (pa < begla) {
        la = lt - 1;
        while (la >= tl && beg[la] == end[la]) --la;
        if (la >= tl) { pa = end[la] - 1; begla = beg[la]; } else pa = -1;
    }
    int pc = beg[rt];
    int rd = rt, pd = pc + 1, endrd = end[rt];
    if (pd >= endrd) {
        rd = rt + 1;
        while (rd < tr && beg[rd] == end[rd]) ++rd;
        if (rd < tr) { pd = beg[rd]; endrd = end[rd]; } else pd = -1;
    }
    T ib = (T)stk[SK::s(pb)], ic = (T)stk[SK::s(pc)];
    T fb = f[SK::f(pb)], fc = f[SK::f(pc)];
    T ia = (T)0, id = (T)0, fa = (T)0, fd = (T)0;
    if (pa >= 0) { ia = (T)stk[SK::s(pa)]; fa = f[SK::f(pa)]; }
    if (pd >= 0) { id = (T)stk[SK::s(pd)]; fd = f[SK::f(pd)]; }
    for (int guard = 0; guard <= n + 2; ++guard) {
        if (pa >= 0 && hidden_t(ia, fa, ib, fb, ic, fc, hh)) {
            if (la != lt) { end[lt] = beg[lt]; lt = la; }
            pb = pa; ib = ia; fb = fa;
            pa = pa - 1;
            if (pa < begla) {
                la = la - 1;
                while (la >= tl && beg[la] == end[la]) --la;
                if (la >= tl) { pa = end[la] - 1; begla = beg[la]; } else pa = -1;
            }
            if (pa >= 0) { ia = (T)stk[SK::s(pa)]; fa = f[SK::f(pa)]; }
            continue;
        }
        if (pd >= 0 && hidden_t(ib, fb, ic, fc, id, fd, hh)) {
            if (rd != rt) { beg[rt] = end[rt]; rt = rd; }
            pc = pd; ic = id; fc = fd;
            pd = pd + 1;
            if (pd >= endrd) {
                rd = rd + 1;
                while (rd < tr && beg[rd] == end[rd]) ++rd;
                if (rd < tr) { pd = beg[rd]; endrd = end[rd]; } else pd = -1;
            }
            if (pd >= 0) { id = (T)stk[SK::s(pd)]; fd = f[SK::f(pd)]; }
            continue;
        }
        break;
    }
    end[lt] = (short)(pb + 1);
    beg[rt] = (short)pc;
}

// ---------------------------------------------------------------------------
// Row sweeps of long lines (axis 0, n > kRowMinN): one group of G threads
// per line, K = 32 cells per thread from 1024 cells, else 16 (G >= 32 either
// way).  Compared with the tile kernel above:
//   * lines are independent: each group takes rows g, g + groups, ... and
//     synchronises only its own G threads, so no line waits for another;
//   * shared memory holds only the line values (the stacks in place) and the
//     stack indices, about 6.2 bytes per cell, so 8 lines of 4096 FP32 cells
//     fit on an SM at 1024 threads;
//   * the merged envelope is not compacted cell by cell: the owner of a
//     thread's first output is found by binary search over the list of
//     non-empty segments (each thread's surviving stack range), then inside
//     one segment, and the sweep steps from segment to segment;
//   * the outputs go from registers straight to global memory, four at a
//     time (a thread's 32 outputs are one 128-byte line), fused with the dual
//     dot product.
// COLS: the same phases on lines along an axis > 0 (columns of 2-D grids,
// axes 1 and 2 of 3-D grids), W neighbouring lines per CTA as one
// interleaved tile: the CTA loads the tile cooperatively (each element
// position is W consecutive words of global memory), each group builds its
// line's envelope as above and writes its outputs into a shared copy of the
// tile, and the CTA stores the tile cooperatively, fused with the dual dot.
// Two CTA barriers per tile replace the per-row independence of the rows.
// The value arrays are double-buffered: while the groups work on one tile,
// the next tile is on its way into the other buffer (cp.async), so the CTA
// does not sit out the load latency of every tile (passes that negate or
// take a dot on load copy synchronously).
// ---------------------------------------------------------------------------
constexpr int kRowMinN = 256;          // rows longer than this take the row kernel
constexpr int kRowLongN = 1024;        // from here 32 cells per thread, else 16


static int row_cells_per_thread(int n) { return n >= kRowLongN ? 32 : 16; }

// Asynchronous global -> shared copies of one element (cp.async, 4 or 8
// bytes, cached in L1), grouped and waited for by the issuing thread.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" :: "r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" :: "r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Barrier of one line group (G >= 32 threads, whole warps): a single warp
// uses the warp barrier, larger groups named barrier 1 + w.
__device__ __forceinline__ void group_sync(int w, int G)
{
    if (G == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" :: "r"(1 + w), "r"(G) : "memory");
}

// One round for a row group (G >= 32 threads, whole warps).  The nearest
// non-empty stacks come from the row's mask of non-empty chunks (one bit per
// thread, nem[G / 32]), so runs of emptied chunks cost a few word reads
// instead of a walk; each round's ballot refreshes the mask.
template <int K, typename T>
__device__ __forceinline__ bool fix_round_row(const T* f, const short* stk, short* beg, short* end,
                                              unsigned* nem, int t, int G, int w, T hh)
{
    const int nwl = G >> 5;
    int b0 = beg[t], e1 = end[t], pa = -1, pc = -1;
    if (e1 > b0) {
        int wi = t >> 5;
        unsigned m = nem[wi] & ((1u << (t & 31)) - 1u);
        while (m == 0u && wi > 0) m = nem[--wi];
        if (m) pa = end[(wi << 5) + 31 - __clz(m)] - 1;
        wi = t >> 5;
        m = nem[wi] & (0xfffffffeu << (t & 31));
        while (m == 0u && wi + 1 < nwl) m = nem[++wi];
        if (m) pc = beg[(wi << 5) + __ffs(m) - 1];
    }
    group_sync(w, G);                              // every read before any update
    bool dropped = false;
    if (e1 > b0) {
        const int ob = b0, oe = e1;
        drop_ends<K>(f, stk, b0, e1, pa, pc, hh);
        dropped = (b0 != ob) || (e1 != oe);
        if (dropped) { beg[t] = (short)b0; end[t] = (short)e1; }
    }
    const unsigned ne = __ballot_sync(0xffffffffu, e1 > b0);
    if ((t & 31) == 0) nem[t >> 5] = ne;
    return group_or(dropped, w, G);                // also publishes the updates and the mask
}

// BATCHED: blockIdx.y selects the problem, whose arguments come from `batch`.
template <typename T, int K, bool BATCHED, bool COLS>
__global__ void __launch_bounds__(512, 2) ct_row_kernel(CtArgs<T> a0, const CtArgs<T>* batch)
{
    const CtArgs<T>& a = BATCHED ? batch[blockIdx.y] : a0;
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SK = Skew<K>;
    const int n = a.lt.n;
    const int G = a.G;
    const int W = a.lt.W;                          // line groups per CTA
    const long long nrows = a.lt.nlines;
    T* fs = reinterpret_cast<T*>(smem_raw);
    short* stk_all = reinterpret_cast<short*>(fs + (size_t)W * a.LD);
    short* seg_all = stk_all + (size_t)W * a.LDI;  // per group: beg[G], end[G], nzs[G]
    const int nwl = (G + 31) / 32;
    const int nsw = (n + 31) >> 5;                 // words of one cell bit mask
    // int scratch: per group 2 nwl scan words, 2 counts, then (FP32) the
    // cell bit mask of owner starts and the list of writer masks
    int* wsum_all = reinterpret_cast<int*>(smem_raw + a.ioff);
    int* cnt_all = wsum_all + W * 2 * nwl;
    unsigned* sw_all = reinterpret_cast<unsigned*>(cnt_all + 2 * W);
    unsigned* wbm_all = sw_all + (size_t)W * nsw;
    __shared__ double red[32];

    const int tid = threadIdx.x;
    const int w = tid / G, t = tid - w * G;
    const int lane = tid & 31;
    T* f = fs + (size_t)w * a.LD;
    short* stk = stk_all + (size_t)w * a.LDI;
    // COLS: the second value buffer follows the output tile
    T* fs_next = reinterpret_cast<T*>(smem_raw + a.soff) + (size_t)W * a.LD;
    short* beg = seg_all + (size_t)w * 3 * G;
    short* end = beg + G;
    short* nzs = end + G;
    int* wsum = wsum_all + w * 2 * nwl;
    unsigned* nem = reinterpret_cast<unsigned*>(wsum);   // phase B: mask of non-empty chunks
    int* cnt = cnt_all + 2 * w;
    unsigned* sw = sw_all + (size_t)w * nsw;
    unsigned* wbm = wbm_all + (size_t)w * G;
    const T hh = a.hh;
    const int lo = t * K;
    const int hi = min(lo + K, n);
    Acc<T> acc_t_in, acc_t_out;
    double acc_in = 0.0, acc_out = 0.0;
    const long long groups = (long long)gridDim.x * W;
    // COLS: the output tile in shared memory, laid out like the value arrays
    T* stg_all = reinterpret_cast<T*>(smem_raw + a.soff);
    const long long nitems = COLS ? a.lt.ntiles : nrows;
    const long long item0 = COLS ? (long long)blockIdx.x : (long long)blockIdx.x * W + w;
    const long long istep = COLS ? (long long)gridDim.x : groups;
    const bool prefetch = COLS && !a.negate && !a.w_in;
    // copies of tile `it` into the value buffers at `dst` (one element per
    // position and line, position-major like the global layout)
    auto issue_tile = [&](long long it, T* dst) {
        const Tile tn = tile_at(a.lt, it);
        const int lw = a.lw, total = n << lw, nth = (int)blockDim.x;
        for (int e = tid; e < total; e += nth) {
            const int ww = e & (W - 1), pp = e >> lw;
            if (ww < tn.wact)
                cp_async_elem(dst + (size_t)ww * a.LD + SK::f(pp),
                              a.in + tn.base0 + ww + (long long)pp * a.lt.es);
        }
        cp_async_commit();
    };
    // With a counter (solver launches), lines are handed out as they are
    // needed: each row group takes its next row when done with the last (rows),
    // each CTA its next tile one tile ahead, for the prefetch (COLS), so the
    // groups or CTAs that drew cheap lines take more and no SM idles while
    // others finish a fixed share.  The last group or CTA to finish resets
    // the counter for the next launch.
    const bool dyn = !COLS && !BATCHED && a.ctr != nullptr;
    const bool dync = COLS && !BATCHED && a.ctr != nullptr && prefetch;
    __shared__ int row_take[16];                   // one per group (W <= 16)
    auto take_row = [&]() -> long long {
        if (t == 0) row_take[w] = atomicAdd(a.ctr, 1);
        group_sync(w, G);
        return row_take[w];
    };
    long long first = item0, nxt_item = 0;
    if (dync) {
        if (tid == 0) row_take[0] = atomicAdd(a.ctr, 1);
        __syncthreads();
        first = row_take[0];
    }
    if (COLS && prefetch && first < nitems) issue_tile(first, fs);

    for (long long item = dyn ? take_row() : first; item < nitems;
         item = dyn ? take_row() : (dync ? nxt_item : item + istep)) {
        const long long rb = COLS ? 0 : item * n;
        Tile tl;
        bool active = true;
        if constexpr (COLS) {
            // ---- load: the CTA reads the tile, position-major (W consecutive
            // words per position), kU elements in flight per thread ----------
            tl = tile_at(a.lt, item);
            active = w < tl.wact;
            f = fs + (size_t)w * a.LD;
            if (prefetch) {
                if (dync && tid == 0) row_take[1] = atomicAdd(a.ctr, 1);   // the tile after this one
                cp_async_wait_all();
                __syncthreads();
                // the other buffer held the tile before this one, whose
                // groups all passed the barrier before its store
                nxt_item = dync ? (long long)row_take[1] : item + istep;
                if (nxt_item < nitems) issue_tile(nxt_item, fs_next);
            } else {
            const int lw = a.lw, total = n << lw, nth = (int)blockDim.x;
            for (int e0 = tid; e0 < total; e0 += kU * nth) {
                T v[kU], u[kU];
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int e = e0 + k * nth, ww = e & (W - 1), pp = e >> lw;
                    const bool ok = e < total && ww < tl.wact;
                    const long long ad = tl.base0 + ww + (long long)pp * a.lt.es;
                    v[k] = ok ? a.in[ad] : (T)0;
                    u[k] = (ok && a.w_in) ? a.w_in[ad] : (T)0;
                }
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int e = e0 + k * nth, ww = e & (W - 1), pp = e >> lw;
                    if (e < total && ww < tl.wact) {
                        if (a.w_in) acc_t_in.add_prod(v[k], u[k]);
                        fs[(size_t)ww * a.LD + SK::f(pp)] = a.negate ? -v[k] : v[k];
                    }
                }
            }
            __syncthreads();
            }
        } else {
        // ---- load: the group reads its row with coalesced loads, kU at a time ----
        if (sizeof(T) == 4 && a.vec4) {
            const float4* src = reinterpret_cast<const float4*>(a.in + rb);
            const float4* wsrc = reinterpret_cast<const float4*>(a.w_in + rb);
            const int nq = n >> 2;
            // float4 loads in flight per thread: U of the row, and as many of
            // the weight when the dual dot is taken on load (registers bound U)
            auto load_row = [&](auto Uc, auto dotc) {
                constexpr int U = decltype(Uc)::value;
                constexpr bool DOT = decltype(dotc)::value;
                for (int q0 = t; q0 < nq; q0 += U * G) {
                    float4 v[U], u[U];
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        const int q = q0 + k * G;
                        v[k] = q < nq ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                        if (DOT) u[k] = q < nq ? wsrc[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        const int q = q0 + k * G;
                        if (q < nq) {
                            float4 x = v[k];
                            if (DOT) acc_t_in.add(dot4(x, u[k]));
                            if (a.negate) { x.x = -x.x; x.y = -x.y; x.z = -x.z; x.w = -x.w; }
                            f[SK::f(4 * q)] = x.x;     f[SK::f(4 * q + 1)] = x.y;
                            f[SK::f(4 * q + 2)] = x.z; f[SK::f(4 * q + 3)] = x.w;
                        }
                    }
                }
            };
            if (a.w_in) load_row(std::integral_constant<int, 2>(), std::true_type());
            else        load_row(std::integral_constant<int, 4>(), std::false_type());
        } else {
            for (int p0 = t; p0 < n; p0 += kU * G) {
                T v[kU], u[kU];
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int p = p0 + k * G;
                    v[k] = p < n ? a.in[rb + p] : (T)0;
                    u[k] = (p < n && a.w_in) ? a.w_in[rb + p] : (T)0;
                }
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int p = p0 + k * G;
                    if (p < n) {
                        if (a.w_in) acc_t_in.add_prod(v[k], u[k]);
                        f[SK::f(p)] = a.negate ? -v[k] : v[k];
                    }
                }
            }
        }
        group_sync(w, G);
        }
        if (active) {
        // ---- A: envelope of this thread's chunk (stack in place) -------------
        // A chunk of K = 2^lg cells lies inside one skew block, so its cells
        // are consecutive from fl / sl.
        if (lo < n) {
            T* fl = f + SK::f(lo);
            short* sl = stk + SK::s(lo);
            const int cnt = hi - lo;
            int top = 0;
            bool has0 = false;
            T s1 = (T)lo, v1 = fl[0], s0 = (T)0, v0 = (T)0;
            T xq = (T)lo;
            sl[0] = (short)lo;
            for (int k = 1; k < cnt; ++k) {
                xq += (T)1;
                const T vq = fl[k];
                while (has0 && hidden_t(s0, v0, s1, v1, xq, vq, hh)) {
                    --top;
                    s1 = s0; v1 = v0;
                    if (top > 0) { s0 = (T)sl[top - 1]; v0 = fl[top - 1]; }
                    else has0 = false;
                }
                ++top;
                sl[top] = (short)(lo + k);
                fl[top] = vq;
                s0 = s1; v0 = v1; has0 = true;
                s1 = xq; v1 = vq;
            }
            beg[t] = (short)lo;
            end[t] = (short)(lo + top + 1);
        } else {
            beg[t] = 0;
            end[t] = 0;
        }
        {
            const unsigned ne = __ballot_sync(0xffffffffu, lo < n);
            if (lane == 0) nem[t >> 5] = ne;
        }
        group_sync(w, G);
        // ---- B: envelope of the whole line ------------------------------------
        // Rounds that drop reflex stack ends (see fix_round_row), then
        // pairwise merges for rows still changing after kFixRoundsRow rounds.
        bool moved = true;
        for (int round = 0; round < kFixRoundsRow && moved; ++round)
            moved = fix_round_row<K>(f, stk, beg, end, nem, t, G, w, hh);
        if (moved) {
            for (int s = 1; s < G; s <<= 1) {
                if ((t & (2 * s - 1)) == 0 && t + s < G) merge_pair_t<K>(f, stk, beg, end, t, s, n, hh);
                if (4 * s <= 32) __syncwarp();
                else group_sync(w, G);
            }
            group_sync(w, G);
        }
        // ---- C: list of non-empty segments, in order ---------------------------
        const bool ne = end[t] > beg[t];
        int pos;
        {
            // groups are whole warps (G >= 32)
            const unsigned mine = __ballot_sync(0xffffffffu, ne);
            pos = __popc(mine & ((1u << lane) - 1u));
            if (sizeof(T) == 4)
                for (int i = t; i < nsw; i += G) sw[i] = 0u;
            if (G > 32) {
                if (lane == 0) wsum[t >> 5] = __popc(mine);
                group_sync(w, G);
                for (int i = 0; i < (t >> 5); ++i) pos += wsum[i];
            }
            if (ne) nzs[pos] = (short)t;
            if (t == G - 1) cnt[0] = pos + (ne ? 1 : 0);
        }
        group_sync(w, G);
        // stores four outputs of this thread (float4 where the row allows) and
        // adds them to the dual dot; COLS: into the shared output tile
        T* dst = a.out + rb;
        const T* wo = a.w_out ? a.w_out + rb : nullptr;
        T* stg = stg_all + (size_t)w * a.LD;
        auto store4 = [&](int x0, const T* o) {
            if constexpr (COLS) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (x0 + k < hi) stg[SK::f(x0 + k)] = o[k];
            } else if (sizeof(T) == 4 && a.vec4 && x0 + 4 <= hi) {
                float4 v4 = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
                *reinterpret_cast<float4*>(dst + x0) = v4;
                if (wo) acc_t_out.add(dot4(v4, *reinterpret_cast<const float4*>(wo + x0)));
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (x0 + k < hi) {
                        dst[x0 + k] = o[k];
                        if (wo) acc_t_out.add_prod(o[k], wo[x0 + k]);
                    }
                }
            }
        };
        bool walk = true;
        if constexpr (sizeof(T) == 4) {
            // ---- D (FP32): owners by rank, no sweep -------------------------------
            // D1. every envelope parabola computes the first cell it owns from
            // its predecessor (start_cell); along the envelope these cells do
            // not decrease, and a parabola owns cells iff the next one starts
            // later ("writer").  Writers set the bit of their start cell in the
            // row's cell mask and their own bit in the thread's mask of stack
            // positions.  A start that decreases (rounding between nearly
            // collinear parabolas) sends the row to the sweep below.
            bool bad = false;
            unsigned bmask = 0u;
            if (ne) {
                const int M = cnt[0];
                const int b0 = beg[t], e1 = end[t];
                float jc = (float)stk[SK::s(b0)], fc = (float)f[SK::f(b0)];
                int cc = 0;
                if (pos > 0) {
                    const int pp = end[nzs[pos - 1]] - 1;
                    cc = start_cell((float)stk[SK::s(pp)], (float)f[SK::f(pp)], jc, fc, (float)hh, n);
                }
#pragma unroll 4
                for (int p = b0 + 1; p < e1; ++p) {
                    const float jn = (float)stk[SK::s(p)], fn = (float)f[SK::f(p)];
                    const int cn = start_cell(jc, fc, jn, fn, (float)hh, n);
                    bad |= cn < cc;
                    if (cn > cc) {
                        bmask |= 1u << (p - 1 - lo);
                        atomicOr(&sw[cc >> 5], 1u << (cc & 31));
                    }
                    jc = jn; fc = fn; cc = cn;
                }
                int cn = n;
                if (pos + 1 < M) {
                    const int ps = beg[nzs[pos + 1]];
                    cn = start_cell(jc, fc, (float)stk[SK::s(ps)], (float)f[SK::f(ps)], (float)hh, n);
                }
                bad |= cn < cc;
                if (cn > cc) {
                    bmask |= 1u << (e1 - 1 - lo);
                    atomicOr(&sw[cc >> 5], 1u << (cc & 31));
                }
            }
            walk = group_or(bad, w, G);            // also publishes the masks
            if (!walk) {
                // D2. the owner of cell x is the writer whose rank is the
                // number of start bits at cells <= x, minus one.  One scan
                // gives each thread the writers and starts before it (packed
                // as two 16-bit counts); threads with writers are listed in
                // order with their masks (nzs: thread, beg: writers before it).
                const int nb = __popc(bmask);
                unsigned sword = 0u;
                if (lo < n) {
                    sword = sw[lo >> 5];
                    if (K < 32) sword = (sword >> (lo & 31)) & ((1u << (K & 31)) - 1u);
                }
                const int v = (nb << 16) | __popc(sword);
                int incl = v;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += y;
                }
                const unsigned nzb = __ballot_sync(0xffffffffu, nb > 0);
                int zpos = __popc(nzb & ((1u << lane) - 1u));
                if (G > 32) {
                    if (lane == 31) wsum[t >> 5] = incl;
                    if (lane == 0) wsum[nwl + (t >> 5)] = __popc(nzb);
                    group_sync(w, G);
                    for (int i = 0; i < (t >> 5); ++i) { incl += wsum[i]; zpos += wsum[nwl + i]; }
                }
                const int excl = incl - v;
                if (nb > 0) {
                    nzs[zpos] = (short)t;
                    beg[zpos] = (short)(excl >> 16);
                    wbm[zpos] = bmask;
                }
                if (t == G - 1) cnt[1] = zpos + (nb > 0 ? 1 : 0);
                group_sync(w, G);
                if (lo < n) {
                    const int Mw = cnt[1];
                    const int R = (excl & 0xFFFF) + (int)(sword & 1u) - 1;
                    int ml = 0, mh = Mw - 1;
                    while (ml < mh) {
                        const int mid = (ml + mh + 1) >> 1;
                        if (beg[mid] <= R) ml = mid;
                        else mh = mid - 1;
                    }
                    int m = ml;
                    unsigned rem = wbm[m];
                    for (int i = R - beg[m]; i > 0; --i) rem &= rem - 1u;
                    int u = nzs[m];
                    int pc = K * u + __ffs(rem) - 1;
                    rem &= rem - 1u;
                    float jc = (float)stk[SK::s(pc)], fc = (float)f[SK::f(pc)];
                    // the next writer, loaded ahead of its start bit
                    float jn = jc, fn = fc;
                    auto load_next = [&]() {
                        if (rem == 0u && m + 1 < Mw) {
                            ++m;
                            rem = wbm[m];
                            u = nzs[m];
                        }
                        if (rem != 0u) {
                            const int pn = K * u + __ffs(rem) - 1;
                            rem &= rem - 1u;
                            jn = (float)stk[SK::s(pn)];
                            fn = (float)f[SK::f(pn)];
                        }
                    };
                    load_next();
                    float xf = (float)lo;
                    for (int x0 = lo; x0 < hi; x0 += 4) {
                        T o[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int xi = x0 + k - lo;
                            if (xi > 0 && ((sword >> xi) & 1u)) {
                                jc = jn; fc = fn;
                                load_next();
                            }
                            o[k] = (T)parab_t((float)hh, xf, jc, fc);
                            xf += 1.f;
                        }
                        store4(x0, o);
                    }
                }
            }
        }
        if (walk) {
        // ---- D: evaluate this thread's outputs by a sweep, store, dual dot -------
        if (lo < n) {
            const int M = cnt[0];
            const T xlo = (T)lo;
            int ml = 0, mh = M - 1;
            while (ml < mh) {
                const int mid = (ml + mh + 1) >> 1;
                const int pu = beg[nzs[mid]], pv = end[nzs[mid - 1]] - 1;
                if (parab_t(hh, xlo, (T)stk[SK::s(pu)], f[SK::f(pu)]) <
                    parab_t(hh, xlo, (T)stk[SK::s(pv)], f[SK::f(pv)])) ml = mid;
                else mh = mid - 1;
            }
            const int m = ml;
            const int pe = end[nzs[m]];
            int pl = beg[nzs[m]], ph = pe - 1;
            while (pl < ph) {
                const int mid = (pl + ph + 1) >> 1;
                if (parab_t(hh, xlo, (T)stk[SK::s(mid)], f[SK::f(mid)]) <
                    parab_t(hh, xlo, (T)stk[SK::s(mid - 1)], f[SK::f(mid - 1)])) pl = mid;
                else ph = mid - 1;
            }
            T jc = (T)stk[SK::s(pl)];
            T fc = f[SK::f(pl)];
            // the parabola after the current one on the envelope: the next
            // position of its segment, else the first of the next non-empty
            // segment; (mn, pen) are the list index and end of pn's segment
            int pn = pl + 1, mn = m, pen = pe;
            if (pn >= pe) {
                mn = m + 1;
                if (mn < M) { pn = beg[nzs[mn]]; pen = end[nzs[mn]]; } else pn = -1;
            }
            bool has_n = pn >= 0;
            T jn = (T)0, fn = (T)0;
            if (has_n) { jn = (T)stk[SK::s(pn)]; fn = f[SK::f(pn)]; }
            T xf = xlo;
            for (int x0 = lo; x0 < hi; x0 += 4) {
                T o[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    T vc = parab_t(hh, xf, jc, fc);
                    while (has_n) {
                        const T vn = parab_t(hh, xf, jn, fn);
                        if (!(vn <= vc)) break;
                        jc = jn; fc = fn; vc = vn;           // advance to pn
                        if (pn + 1 < pen) ++pn;
                        else {
                            ++mn;
                            if (mn < M) { pn = beg[nzs[mn]]; pen = end[nzs[mn]]; } else has_n = false;
                        }
                        if (has_n) { jn = (T)stk[SK::s(pn)]; fn = f[SK::f(pn)]; }
                    }
                    o[k] = vc;
                    xf += (T)1;
                }
                store4(x0, o);
            }
        }
        }
        }
        if constexpr (COLS) {
            // ---- store: the CTA writes the tile back, position-major, with
            // the dual dot; the next tile's load writes only the value arrays
            __syncthreads();
            const int lw = a.lw, total = n << lw, nth = (int)blockDim.x;
            for (int e = tid; e < total; e += nth) {
                const int ww = e & (W - 1), pp = e >> lw;
                if (ww < tl.wact) {
                    const T o = stg_all[(size_t)ww * a.LD + SK::f(pp)];
                    const long long ad = tl.base0 + ww + (long long)pp * a.lt.es;
                    a.out[ad] = o;
                    if (a.w_out) acc_t_out.add_prod(o, a.w_out[ad]);
                }
            }
        }
        acc_in += acc_t_in.take();
        acc_out += acc_t_out.take();
        if constexpr (!COLS) group_sync(w, G);   // the next row overwrites this group's arrays
        if (prefetch) { T* tb = fs; fs = fs_next; fs_next = tb; }
    }
    if ((dyn && t == 0) || (dync && tid == 0)) {
        __threadfence();                           // this group's (CTA's) takes precede its count
        const int takers = dyn ? (int)(gridDim.x * W) : (int)gridDim.x;
        if (atomicAdd(a.ctr + 1, 1) == takers - 1) {
            a.ctr[0] = 0;
            a.ctr[1] = 0;
            __threadfence();
        }
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
    if (n == 384) return 24;      // 16 chunks (a half warp per line, no idle lane)
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
void* kernel_for(bool contig, bool batched)
{
    if (batched)
        return contig ? (void*)ct_pass_kernel<T, K, true, true> : (void*)ct_pass_kernel<T, K, false, true>;
    return contig ? (void*)ct_pass_kernel<T, K, true, false> : (void*)ct_pass_kernel<T, K, false, false>;
}

template <typename T>
void* select_kernel(int K, bool contig, bool batched)
{
    switch (K) {
        case 1: return kernel_for<T, 1>(contig, batched);
        case 2: return kernel_for<T, 2>(contig, batched);
        case 4: return kernel_for<T, 4>(contig, batched);
        case 8: return kernel_for<T, 8>(contig, batched);
        case 12: return kernel_for<T, 12>(contig, batched);
        case 24: return kernel_for<T, 24>(contig, batched);
        case 32: return kernel_for<T, 32>(contig, batched);
        default: return kernel_for<T, 16>(contig, batched);
    }
}

}  // namespace

// Tile plan with K cells per thread and (Wreq > 0) at most Wreq lines per
// CTA; Wreq <= 0 takes as many lines as the thread and memory limits allow.
static CtPlan plan_ct_tile(const Grid& g, int axis, int elem_bytes, int K, int Wreq)
{
    CtPlan p;
    const int n = g.n[axis];
    p.K = K;
    p.G = next_pow2((n + p.K - 1) / p.K);
    const bool contig = (axis == 0);
    // pad words of the skewed layout: one per 2^lg cells (Skew<K>: lg = log2 of
    // the largest power of two <= K), plus one
    int lg = 0;
    while ((2 << lg) <= p.K && lg < 5) ++lg;
    const int chunks = (n >> lg) + 2;
    int LDI = n + 2 * chunks + 8;                         // skewed index stack (two shorts per chunk)
    LDI += LDI & 1;
    const int nf = n + chunks + 1;                        // skewed values (one word per chunk)
    const int LDH = n + (n & 1);                          // compacted envelope
    const int nwl = (p.G + 31) / 32;
    const size_t line_bytes = (size_t)(nf + 32) * elem_bytes + (size_t)LDH * elem_bytes +
                              (size_t)LDI * 2 + (size_t)LDH * 2 + 4 * (size_t)p.G + 4 * nwl + 64;
    // up to 512 threads per CTA so that two CTAs share an SM; lines of more
    // than one warp use named barriers 1..8, so at most 8 such lines
    int W = 512 / p.G;
    if (W < 1) W = 1;
    if (W > 32) W = 32;
    const size_t budget = 110 * 1024;
    while (W > 1 && (size_t)W * line_bytes > budget) --W;
    if (Wreq > 0 && W > Wreq) W = Wreq;
    if (!contig) {
        // interleaved tiles: W a power of two (division-free index math)
        int p2 = 1;
        while (p2 * 2 <= W) p2 *= 2;
        W = p2;
    }
    // leading dimension: for interleaved loads consecutive lanes hit the W lines
    // of one position; pick the stride with the fewest shared-memory bank conflicts
    int LD = nf;
    if (!contig) {
        int best = 1 << 30;
        for (int cand = nf; cand <= nf + 32; ++cand) {
            const int c = bank_conflicts(cand, W, elem_bytes / 4);
            if (c < best) { best = c; LD = cand; }
        }
    }
    LD += LD & 1;
    p.W = W;
    p.LD = LD;
    p.LDI = LDI;
    p.LDH = LDH;
    p.smem = (size_t)W * LD * elem_bytes + (size_t)W * LDH * elem_bytes + (size_t)W * LDI * 2 +
             (size_t)W * LDH * 2 + 2 * (size_t)W * p.G * 2 + (size_t)W * nwl * 4 + (size_t)W * 4 + 16;
    p.threads = ((W * p.G + 31) / 32) * 32;
    p.tiles = make_tiles(g, axis, W);
    return p;
}

// Row kernel plan: K = 32 or 16 cells per thread, G = the next power of two
// of n / K (at least 32 for n > 256, so every group is whole warps), as many
// groups per CTA as fit 512 threads and about 110 KB (two CTAs per SM).
// Lines along axis > 0 (COLS) come as interleaved tiles of W neighbouring
// lines, W a power of two, with a second value-sized array per line for the
// output tile and a leading dimension chosen against bank conflicts of the
// position-major tile loads and stores.
static CtPlan plan_ct_row_shape(const Grid& g, int elem_bytes, int K, int Wreq, int axis = 0)
{
    CtPlan p;
    const int n = g.n[axis];
    const bool cols = axis > 0;
    p.K = K;
    p.G = next_pow2((n + p.K - 1) / p.K);
    const int chunks = (n + p.K - 1) / p.K + 1;
    p.LD = n + chunks + 2;
    p.LD += p.LD & 1;
    p.LDI = n + 2 * chunks + 8;
    p.LDI += p.LDI & 1;
    const int nwl = (p.G + 31) / 32;
    // int scratch per group: 2 nwl scan words and 2 counts; FP32 rows add the
    // cell mask of owner starts (one bit per cell) and G writer masks
    const size_t ints = 2 * (size_t)nwl + 2 + (elem_bytes == 4 ? (size_t)((n + 31) >> 5) + p.G : 0);
    // COLS: value arrays twice (double-buffered loads) and the output tile
    const size_t line_bytes = (size_t)p.LD * elem_bytes * (cols ? 3 : 1) + (size_t)p.LDI * 2 +
                              3 * (size_t)p.G * 2 + 4 * ints;
    // (COLS: with room for the leading dimension's padding below)
    const size_t budget_line = line_bytes + (cols ? 3 * 32 * (size_t)elem_bytes : 0);
    int W = 512 / p.G;
    if (W < 1) W = 1;
    while (W > 1 && (size_t)W * budget_line > 110 * 1024) --W;
    if (Wreq > 0 && W > Wreq) W = Wreq;
    if (cols) {
        int p2 = 1;
        while (p2 * 2 <= W) p2 *= 2;
        W = p2;
        int best = 1 << 30, LD = p.LD;
        for (int cand = p.LD; cand <= p.LD + 32; cand += 2) {
            const int c = bank_conflicts(cand, W, elem_bytes / 4);
            if (c < best) { best = c; LD = cand; }
        }
        p.LD = LD;
    }
    p.W = W;
    size_t off = (size_t)W * p.LD * elem_bytes + (size_t)W * p.LDI * 2 + (size_t)W * 3 * p.G * 2;
    off = (off + 15) & ~(size_t)15;
    p.ioff = (int)off;
    p.LDH = 0;
    size_t end = off + (size_t)W * ints * 4;
    end = (end + 15) & ~(size_t)15;
    p.soff = (int)end;
    p.smem = end + (cols ? 2 * (size_t)W * p.LD * elem_bytes : 0) + 16;
    p.threads = W * p.G;
    p.tiles = make_tiles(g, axis, W);
    return p;
}

// Lines of more than 256 cells take the row kernel: rows always, lines along
// the other axes when a tile of the default shape spans at least 32 bytes per
// element position (one DRAM sector), else the tile kernel.
static bool use_row_kernel(const Grid& g, int axis, int elem_bytes)
{
    const int n = g.n[axis];
    if (n <= kRowMinN) return false;
    if (axis == 0) return true;
    return plan_ct_row_shape(g, elem_bytes, row_cells_per_thread(n), 0, axis).W * elem_bytes >= 32;
}

// ---------------------------------------------------------------------------
// launch shapes and the tuning table
// ---------------------------------------------------------------------------
// A pass's shape is (K cells per thread, W lines per CTA) of its kernel kind:
// tile rows (axis 0, lines of at most 256 cells), tile columns (axes > 0:
// W neighbouring lines interleaved) or the row kernel (axis 0, rows of more
// than 256 cells).  The default shapes are the hand-picked ones; the
// autotuner (bfm_autotune) times the candidates of a line length and stores
// the fastest here, and every later plan of that kind and length takes it.
// Any candidate gives the same envelope (the same exact-discrete transform),
// so a tuned shape changes timing, not results beyond rounding order.
int ct_kind(const Grid& g, int axis, int elem_bytes)
{
    if (use_row_kernel(g, axis, elem_bytes)) return axis == 0 ? CT_KIND_ROW : CT_KIND_ROW_COLS;
    return axis == 0 ? CT_KIND_TILE_ROWS : CT_KIND_TILE_COLS;
}

static bool row_kind(int kind) { return kind == CT_KIND_ROW || kind == CT_KIND_ROW_COLS; }

CtShape ct_default_shape(int kind, int n, int elem_bytes)
{
    if (row_kind(kind)) return CtShape{row_cells_per_thread(n), 0};
    const CtShape s{pick_K(n), 0};
    // 24 cells per thread where its lines fill whole warps, else 12
    if (s.K == 24 && !ct_shape_valid(kind, n, elem_bytes, s)) return CtShape{12, 0};
    return s;
}

static bool tile_K_ok(int n, int K)
{
    if (K != 1 && K != 2 && K != 4 && K != 8 && K != 12 && K != 16 && K != 24 && K != 32) return false;
    if (K > n) return false;
    if ((K == 12 || K == 24) && n % K != 0) return false;
    return next_pow2((n + K - 1) / K) <= 512;
}

static bool row_K_ok(int n, int K)
{
    if (n <= kRowMinN || (K != 16 && K != 32)) return false;
    const int G = next_pow2((n + K - 1) / K);
    return G >= 32 && G <= 512;
}

// the lines per CTA a plan with this K takes when unrestricted
static int max_lines(int kind, int n, int elem_bytes, int K)
{
    int dims[3] = {n, 64, 1};
    const bool cols = kind == CT_KIND_TILE_COLS || kind == CT_KIND_ROW_COLS;
    if (cols) { dims[0] = 64; dims[1] = n; }
    bfm_grid bg{2, {dims[0], dims[1], 1}};
    Grid g;
    make_grid(&bg, &g);
    if (row_kind(kind)) return plan_ct_row_shape(g, elem_bytes, K, 0, cols ? 1 : 0).W;
    return plan_ct_tile(g, kind == CT_KIND_TILE_COLS ? 1 : 0, elem_bytes, K, 0).W;
}

int ct_shape_candidates(int kind, int n, int elem_bytes, CtShape* out, int cap)
{
    static const int tileK[] = {1, 2, 4, 8, 12, 16, 24, 32};
    static const int rowK[] = {16, 32};
    const int* Ks = row_kind(kind) ? rowK : tileK;
    const int nK = row_kind(kind) ? 2 : 8;
    int cnt = 0;
    for (int i = 0; i < nK; ++i) {
        const int K = Ks[i];
        if (row_kind(kind) ? !row_K_ok(n, K) : !tile_K_ok(n, K)) continue;
        const int Wm = max_lines(kind, n, elem_bytes, K);
        const int G = next_pow2((n + K - 1) / K);
        // the unrestricted W and up to two halvings of it, keeping CTAs of
        // whole warps (lines shorter than a warp fill it)
        for (int W = Wm, k = 0; W >= 1 && k < 3; W = (W > 1 ? W / 2 : 0), ++k) {
            if (W * G < 32 || (G < 32 && (W * G) % 32 != 0)) break;
            if (cnt < cap && out) out[cnt] = CtShape{K, W == Wm ? 0 : W};
            ++cnt;
            if (W == 1) break;
        }
    }
    return cnt;
}

bool ct_shape_valid(int kind, int n, int elem_bytes, CtShape s)
{
    CtShape c[64];
    const int m = ct_shape_candidates(kind, n, elem_bytes, c, 64);
    for (int i = 0; i < m && i < 64; ++i)
        if (c[i].K == s.K && c[i].W == s.W) return true;
    return false;
}

namespace {
struct TuneKey {
    int kind, n, elem;
    bool operator<(const TuneKey& o) const
    {
        if (kind != o.kind) return kind < o.kind;
        if (n != o.n) return n < o.n;
        return elem < o.elem;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, CtShape> g_tune;
}  // namespace

bool ct_tuned_shape(int kind, int n, int elem_bytes, CtShape* s)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(TuneKey{kind, n, elem_bytes});
    if (it == g_tune.end()) return false;
    *s = it->second;
    return true;
}

void ct_set_tuned_shape(int kind, int n, int elem_bytes, CtShape s)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{kind, n, elem_bytes}] = s;
}

void ct_erase_tuned_shape(int kind, int n, int elem_bytes)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.erase(TuneKey{kind, n, elem_bytes});
}

void ct_clear_tuned_shapes()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

static CtShape shape_for(int kind, int n, int elem_bytes)
{
    CtShape s;
    if (ct_tuned_shape(kind, n, elem_bytes, &s)) return s;
    return ct_default_shape(kind, n, elem_bytes);
}

CtPlan plan_ct_pass(const Grid& g, int axis, int elem_bytes)
{
    const CtShape s = shape_for(axis == 0 ? CT_KIND_TILE_ROWS : CT_KIND_TILE_COLS, g.n[axis], elem_bytes);
    return plan_ct_tile(g, axis, elem_bytes, s.K, s.W);
}

CtPlan plan_ct_pass_default(const Grid& g, int axis, int elem_bytes)
{
    const CtShape s = ct_default_shape(axis == 0 ? CT_KIND_TILE_ROWS : CT_KIND_TILE_COLS, g.n[axis],
                                       elem_bytes);
    return plan_ct_tile(g, axis, elem_bytes, s.K, s.W);
}

static CtPlan plan_ct_row(const Grid& g, int axis, int elem_bytes)
{
    const CtShape s = shape_for(axis == 0 ? CT_KIND_ROW : CT_KIND_ROW_COLS, g.n[axis], elem_bytes);
    return plan_ct_row_shape(g, elem_bytes, s.K, s.W, axis);
}

// the row kernel for K cells per thread, batched or not, rows or interleaved tiles
template <typename T>
static void* row_kernel_for(int K, bool batched, bool cols)
{
    if (cols) {
        if (batched) return K == 32 ? (void*)ct_row_kernel<T, 32, true, true> : (void*)ct_row_kernel<T, 16, true, true>;
        return K == 32 ? (void*)ct_row_kernel<T, 32, false, true> : (void*)ct_row_kernel<T, 16, false, true>;
    }
    if (batched) return K == 32 ? (void*)ct_row_kernel<T, 32, true, false> : (void*)ct_row_kernel<T, 16, true, false>;
    return K == 32 ? (void*)ct_row_kernel<T, 32, false, false> : (void*)ct_row_kernel<T, 16, false, false>;
}

template <typename T>
static CtArgs<T> make_ct_args(const Grid& g, int axis, const CtPlan& p, const T* in, T* out,
                              bool negate, const T* w_in, double* part_in, const T* w_out,
                              double* part_out, const int* done)
{
    CtArgs<T> a;
    a.in = in; a.out = out; a.w_in = w_in; a.w_out = w_out;
    a.part_in = part_in; a.part_out = part_out; a.done = done;
    a.lt = p.tiles; a.G = p.G; a.LD = p.LD; a.LDI = p.LDI; a.LDH = p.LDH;
    const double h = 1.0 / g.n[axis];
    a.hh = (T)(0.5 * h * h);
    a.negate = negate ? 1 : 0;
    auto al16 = [](const void* q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    a.vec4 = (axis == 0 && g.n[0] % 4 == 0 && al16(in) && al16(out) && al16(w_in) && al16(w_out)) ? 1 : 0;
    a.lw = 0;
    while ((1 << a.lw) < p.W) ++a.lw;
    a.ioff = p.ioff;
    a.soff = p.soff;
    a.ctr = nullptr;
    return a;
}

static int ct_blocks(const CtPlan& p, int max_blocks)
{
    long long blocks = p.tiles.ntiles;
    const long long cap = (long long)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

int ct_pass_blocks(const Grid& g, int axis, int elem_bytes, int max_blocks)
{
    if (use_row_kernel(g, axis, elem_bytes)) {
        const CtPlan p = plan_ct_row(g, axis, elem_bytes);
        long long blocks = p.tiles.ntiles;
        // one resident wave: 1024 threads per SM at 64 registers each
        // (launch bounds 512, 2), fewer where shared memory runs out
        int per_sm = 1024 / p.threads;
        const int by_smem = (int)((227 * 1024) / (p.smem + 1024));
        if (per_sm > by_smem) per_sm = by_smem;
        if (per_sm < 1) per_sm = 1;
        const long long cap = (long long)num_sms() * per_sm;
        if (blocks > cap) blocks = cap;
        if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
        if (blocks < 1) blocks = 1;
        return (int)blocks;
    }
    return ct_blocks(plan_ct_pass(g, axis, elem_bytes), max_blocks);
}

template <typename T>
bfm_status launch_ct_pass(const Grid& g, int axis, const T* in, T* out, bool negate,
                          const T* w_in, double* part_in, const T* w_out, double* part_out,
                          const int* done, int max_blocks, cudaStream_t st, int* blocks_used, int* row_ctr)
{
    if (use_row_kernel(g, axis, (int)sizeof(T))) {
        CtPlan p = plan_ct_row(g, axis, (int)sizeof(T));
        CtArgs<T> a = make_ct_args<T>(g, axis, p, in, out, negate, w_in, part_in, w_out, part_out,
                                      done);
        a.ctr = row_ctr;
        void* k = row_kernel_for<T>(p.K, false, axis > 0);
        BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
        const int blocks = ct_pass_blocks(g, axis, (int)sizeof(T), max_blocks);
        const CtArgs<T>* none = nullptr;
        void* args[] = {&a, &none};
        BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(p.threads), args, p.smem, st));
        if (blocks_used) *blocks_used = (int)blocks;
        return BFM_OK;
    }
    CtPlan p = plan_ct_pass(g, axis, (int)sizeof(T));
    CtArgs<T> a = make_ct_args<T>(g, axis, p, in, out, negate, w_in, part_in, w_out, part_out, done);
    void* k = select_kernel<T>(p.K, axis == 0, false);
    BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int blocks = ct_pass_blocks(g, axis, (int)sizeof(T), max_blocks);
    const CtArgs<T>* none = nullptr;
    void* args[] = {&a, &none};
    BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(p.threads), args, p.smem, st));
    if (blocks_used) *blocks_used = blocks;
    return BFM_OK;
}

// Batched form: problems that share one grid shape; `dev_args` (device) is
// filled with one CtArgs per problem by fill_ct_batch_args.
template <typename T>
int ct_batch_blocks(const Grid& g, int axis)
{
    return ct_pass_blocks(g, axis, (int)sizeof(T), kMaxPartials);
}

template <typename T>
void fill_ct_batch_args(const Grid& g, int axis, const T* in, T* out, bool negate, const T* w_in,
                        double* part_in, const T* w_out, double* part_out, const int* done,
                        void* host_slot)
{
    CtPlan p = use_row_kernel(g, axis, (int)sizeof(T)) ? plan_ct_row(g, axis, (int)sizeof(T))
                                                       : plan_ct_pass(g, axis, (int)sizeof(T));
    *reinterpret_cast<CtArgs<T>*>(host_slot) =
        make_ct_args<T>(g, axis, p, in, out, negate, w_in, part_in, w_out, part_out, done);
}

size_t ct_args_bytes(int elem_bytes) { return elem_bytes == 8 ? sizeof(CtArgs<double>) : sizeof(CtArgs<float>); }

template <typename T>
bfm_status launch_ct_pass_batched(const Grid& g, int axis, int nprob, const void* dev_args,
                                  cudaStream_t st)
{
    if (use_row_kernel(g, axis, (int)sizeof(T))) {
        // long lines: the row kernel (rows or interleaved tiles), per problem
        const CtPlan p = plan_ct_row(g, axis, (int)sizeof(T));
        void* k = row_kernel_for<T>(p.K, true, axis > 0);
        BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
        const int blocks = ct_pass_blocks(g, axis, (int)sizeof(T), kMaxPartials);
        CtArgs<T> dummy;
        memset(&dummy, 0, sizeof(dummy));
        const CtArgs<T>* batch = reinterpret_cast<const CtArgs<T>*>(dev_args);
        void* args[] = {&dummy, &batch};
        BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks, (unsigned)nprob), dim3(p.threads), args,
                                  p.smem, st));
        return BFM_OK;
    }
    CtPlan p = plan_ct_pass(g, axis, (int)sizeof(T));
    void* k = select_kernel<T>(p.K, axis == 0, true);
    BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int blocks = ct_blocks(p, kMaxPartials);
    CtArgs<T> dummy;
    memset(&dummy, 0, sizeof(dummy));
    const CtArgs<T>* batch = reinterpret_cast<const CtArgs<T>*>(dev_args);
    void* args[] = {&dummy, &batch};
    BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks, (unsigned)nprob), dim3(p.threads), args,
                              p.smem, st));
    return BFM_OK;
}

template int ct_batch_blocks<float>(const Grid&, int);
template int ct_batch_blocks<double>(const Grid&, int);
template void fill_ct_batch_args<float>(const Grid&, int, const float*, float*, bool, const float*,
                                        double*, const float*, double*, const int*, void*);
template void fill_ct_batch_args<double>(const Grid&, int, const double*, double*, bool,
                                         const double*, double*, const double*, double*,
                                         const int*, void*);
template bfm_status launch_ct_pass_batched<float>(const Grid&, int, int, const void*, cudaStream_t);
template bfm_status launch_ct_pass_batched<double>(const Grid&, int, int, const void*, cudaStream_t);
template bfm_status launch_ct_pass<float>(const Grid&, int, const float*, float*, bool, const float*,
                                          double*, const float*, double*, const int*, int,
                                          cudaStream_t, int*, int*);
template bfm_status launch_ct_pass<double>(const Grid&, int, const double*, double*, bool,
                                           const double*, double*, const double*, double*,
                                           const int*, int, cudaStream_t, int*, int*);

}  // namespace bfm
