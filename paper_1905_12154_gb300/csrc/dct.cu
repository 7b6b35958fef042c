// dct.cu -- DCT-II / DCT-III along grid lines and the Neumann Poisson solve.
//
// The H1-dot gradient of Lemma 2.3 is g = (-Delta)^{-1}(f - mean f) with zero
// Neumann conditions; the paper inverts the Laplacian with FFTs (Section 4.3).
// On the cell-centred grid the Laplacian with reflected ghost cells is
// diagonalised by the DCT-II along every axis, with eigenvalues
//     lambda_k = sum_a 4 n_a^2 sin^2(pi k_a / (2 n_a)).
// Each line transform runs in shared memory: two real lines of a tile are
// packed into the real and imaginary parts of one complex sequence; the
// DCT-II is a length-n complex FFT of the even/odd reordering
// v = (x0, x2, x4, ..., x5, x3, x1) followed by the twiddle e^{-i pi k/(2n)}
// (Makhoul's construction); the inverse undoes both steps.  The forward FFT
// is an in-place mixed-radix (2/3/4) decimation-in-time network with a
// digit-reversed load, the inverse a decimation-in-frequency network whose
// digit-reversed output is gathered on store.
//
// Pass kinds (one launch each):
//   FWD  f -> DCT-II along the axis (optionally f = base - in on load);
//   MID  on the last axis: DCT-II, divide by lambda (zero mode -> 0),
//        accumulate G = ||g||^2_{H1-dot} in FP64, inverse DCT;
//   INV  inverse DCT along the axis (optionally out = upd + sigma * g).
#include <stdint.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"

namespace bfm {

enum { DCT_FWD = 0, DCT_MID = 1, DCT_INV = 2 };

template <typename T>
struct DctArgs {
    const T* in;
    const T* base;            // FWD: value = base - in (optional)
    T* out;
    const T* upd;             // INV: out = upd + sigma * value (optional)
    const double* sigma;      // device scalar used with upd
    double* part;             // MID: per-CTA partial sums of G
    const int* done;          // optional skip flag
    const cx_t<T>* tw;        // e^{-2 pi i j/n}
    const float2* ptw;        // register FFT: pass twiddles, pass of stride Ns at
                              // Ns - 1, entry (r - 1) Ns + k = e^{-2 pi i k r/(Ns R)}
    const cx_t<T>* dtw;       // e^{-i pi k/(2n)}
    const unsigned short* drev;   // digit reversal of the stage radices
    const T* lam_axis;        // MID: eigenvalues along this axis
    const T* lam_a0;          // MID: eigenvalues along axis 0 (index of the line)
    const T* lam_a1;          // MID (3D): eigenvalues along axis 1 (outer index)
    LineTiles lt;
    int G;                    // threads per line pair
    int LDZ;                  // shared leading dimension (complex elements)
    int nst;
    int rad[kMaxStages];
    int Ls[kMaxStages];       // sub-transform length entering stage s (product of earlier radices)
    unsigned mag[kMaxStages]; // ceil(2^32 / Ls[s]): b / Ls[s] = umulhi(b, mag[s]) for b < n
    int lnp;                  // log2(pairs per tile) for interleaved tiles
    double gscale;            // MID: 1 / N^2
    int fnst;                 // register Stockham path: number of passes
    int frad[8];              // and their radices (16, ..., 16, last in {2,4,8,16})
};

__device__ __forceinline__ int div_by(int b, int L, unsigned mag)
{
    return L == 1 ? b : (int)__umulhi((unsigned)b, mag);
}

// r-point DFT, SIGN = -1 forward, +1 inverse
template <int SIGN, typename C>
__device__ __forceinline__ void dft_small(int r, C* u)
{
    using T = decltype(u[0].x);
    if (r == 2) {
        const C a = u[0], b = u[1];
        u[0] = cadd(a, b);
        u[1] = csub(a, b);
    } else if (r == 4) {
        const C a0 = cadd(u[0], u[2]), a1 = csub(u[0], u[2]);
        const C b0 = cadd(u[1], u[3]), b1 = csub(u[1], u[3]);
        C ib1;                      // SIGN * i * b1
        if (SIGN < 0) { ib1.x = b1.y; ib1.y = -b1.x; }
        else          { ib1.x = -b1.y; ib1.y = b1.x; }
        u[0] = cadd(a0, b0);
        u[2] = csub(a0, b0);
        u[1] = cadd(a1, ib1);
        u[3] = csub(a1, ib1);
    } else {  // r == 3
        const T s = (T)(SIGN * 0.86602540378443864676);   // sin(2 pi / 3) with sign
        const C t1 = cadd(u[1], u[2]), t2 = csub(u[1], u[2]);
        C m; m.x = u[0].x - (T)0.5 * t1.x; m.y = u[0].y - (T)0.5 * t1.y;
        C it2; it2.x = -s * t2.y; it2.y = s * t2.x;          // s * i * t2
        u[0] = cadd(u[0], t1);
        u[1] = cadd(m, it2);
        u[2] = csub(m, it2);
    }
}

// One radix-R stage of the forward decimation-in-time network: butterfly b
// (sub-transform B = b / L, offset k1 = b mod L) combines z[B Lp + k1 + q L],
// q < R, twiddled by e^{-2 pi i q k1 tstep / n}.  R is a compile-time
// constant so the butterfly's values stay in registers.
template <int R, typename C>
__device__ __forceinline__ void dit_stage(C* z, const C* tw, int t, int G, int nb, int L, int Lp,
                                          int tstep, unsigned mg)
{
    for (int b = t; b < nb; b += G) {
        const int B = div_by(b, L, mg), k1 = b - B * L;
        const int base = B * Lp + k1;
        C u[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            C v = z[base + q * L];
            if (q) v = cmul(v, tw[q * k1 * tstep]);
            u[q] = v;
        }
        dft_small<-1>(R, u);
#pragma unroll
        for (int q = 0; q < R; ++q) z[base + q * L] = u[q];
    }
}

// The matching stage of the inverse decimation-in-frequency network.
template <int R, typename C>
__device__ __forceinline__ void dif_stage(C* z, const C* tw, int t, int G, int nb, int L, int Lp,
                                          int tstep, unsigned mg)
{
    for (int b = t; b < nb; b += G) {
        const int B = div_by(b, L, mg), k1 = b - B * L;
        const int base = B * Lp + k1;
        C u[R];
#pragma unroll
        for (int q = 0; q < R; ++q) u[q] = z[base + q * L];
        dft_small<+1>(R, u);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            C v = u[q];
            if (q) v = cmul(v, cconj(tw[q * k1 * tstep]));
            z[base + q * L] = v;
        }
    }
}

// BATCHED: blockIdx.y selects the problem, whose arguments come from `batch`.
template <typename T, int MODE, bool CONTIG, bool BATCHED>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024, 1)
dct_pass_kernel(DctArgs<T> a0, const DctArgs<T>* batch)
{
    using C = cx_t<T>;
    const DctArgs<T>& a = BATCHED ? batch[blockIdx.y] : a0;
    if (BATCHED && blockIdx.x >= a.lt.ntiles) return;
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* zs = reinterpret_cast<C*>(smem_raw);
    __shared__ double red[32];
    const LineTiles& lt = a.lt;
    const int n = lt.n;
    const int G = a.G;
    const int tid = threadIdx.x;
    const int pp = tid / G, t = tid - pp * G;
    const int npair_max = (lt.W + 1) / 2;
    C* z = zs + (size_t)pp * a.LDZ;
    const T inv_n = (T)1 / (T)n;
    T sig = (T)0;
    if (MODE == DCT_INV && a.upd) sig = (T)(*a.sigma);
    double acc = 0.0;
    Acc<T> gsum;

    for (long long tile = blockIdx.x; tile < lt.ntiles; tile += gridDim.x) {
        const Tile tl = tile_at(lt, tile);
        const int np = (tl.wact + 1) / 2;
        // ---- load ------------------------------------------------------------
        {
            // CONTIG: one row pair after another; interleaved: pairs fastest.
            // Each thread issues U loads (and their base loads) before storing
            // any, so a tile's loads overlap instead of forming a chain.
            constexpr int U = 4;
            const int np_pow = CONTIG ? 1 : (1 << a.lnp);
            const int per = CONTIG ? n : np_pow * n;
            const int reps = CONTIG ? np : 1;
            const int bd = blockDim.x;
            for (int q0 = 0; q0 < reps; ++q0)
            for (int e0 = tid; e0 < per; e0 += U * bd) {
                T xa[U], xb[U], ba[U], bb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * bd;
                    int q, j;
                    if (CONTIG) { q = q0; j = e; }
                    else        { q = e & (np_pow - 1); j = e >> a.lnp; }
                    xa[u] = xb[u] = ba[u] = bb[u] = (T)0;
                    if (e < per && q < np) {
                        const bool hb = 2 * q + 1 < tl.wact;
                        const long long ada = tl.base0 + (long long)(2 * q) * tl.lstride + (long long)j * lt.es;
                        xa[u] = a.in[ada];
                        if (hb) xb[u] = a.in[ada + tl.lstride];
                        if (MODE == DCT_FWD && a.base) {
                            ba[u] = a.base[ada];
                            if (hb) bb[u] = a.base[ada + tl.lstride];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * bd;
                    int q, j;
                    if (CONTIG) { q = q0; j = e; }
                    else        { q = e & (np_pow - 1); j = e >> a.lnp; }
                    if (e >= per || q >= np) continue;
                    C v;
                    if (MODE == DCT_FWD && a.base) { v.x = ba[u] - xa[u]; v.y = bb[u] - xb[u]; }
                    else { v.x = xa[u]; v.y = xb[u]; }
                    if (MODE == DCT_INV) {
                        zs[(size_t)q * a.LDZ + j] = v;                       // natural order
                    } else {
                        const int m = (j & 1) ? (n - 1 - (j >> 1)) : (j >> 1);
                        zs[(size_t)q * a.LDZ + a.drev[m]] = v;               // DIT input order
                    }
                }
            }
        }
        __syncthreads();
        const bool active = (pp < np);
        if (MODE != DCT_INV) {
            // ---- forward DIT FFT ---------------------------------------------
            for (int s = 0; s < a.nst; ++s) {
                const int r = a.rad[s];
                const int L = a.Ls[s];
                const int Lp = L * r;
                const int tstep = (s + 1 < a.nst) ? n / Lp : 1;
                const unsigned mg = a.mag[s];
                const int nb = (r == 4) ? (n >> 2) : (r == 2 ? (n >> 1) : n / 3);
                if (active) {
                    if (r == 4) dit_stage<4>(z, a.tw, t, G, nb, L, Lp, tstep, mg);
                    else if (r == 2) dit_stage<2>(z, a.tw, t, G, nb, L, Lp, tstep, mg);
                    else dit_stage<3>(z, a.tw, t, G, nb, L, Lp, tstep, mg);
                }
                __syncthreads();
            }
            // ---- separate the two lines, apply e^{-i pi k/2n} -------------------
            if (active) {
                for (int k = t; k <= n / 2; k += G) {
                    const int km = (n - k) % n;
                    const C Zk = z[k], Zm = z[km];
                    // A_k = (Z_k + conj Z_m)/2, B_k = -i (Z_k - conj Z_m)/2
                    C A, B;
                    A.x = (T)0.5 * (Zk.x + Zm.x); A.y = (T)0.5 * (Zk.y - Zm.y);
                    B.x = (T)0.5 * (Zk.y + Zm.y); B.y = (T)0.5 * (Zm.x - Zk.x);
                    const C dk = a.dtw[k];
                    C outk; outk.x = dk.x * A.x - dk.y * A.y; outk.y = dk.x * B.x - dk.y * B.y;
                    if (km != k) {
                        C Am, Bm;
                        Am.x = (T)0.5 * (Zm.x + Zk.x); Am.y = (T)0.5 * (Zm.y - Zk.y);
                        Bm.x = (T)0.5 * (Zm.y + Zk.y); Bm.y = (T)0.5 * (Zk.x - Zm.x);
                        const C dm = a.dtw[km];
                        C outm; outm.x = dm.x * Am.x - dm.y * Am.y; outm.y = dm.x * Bm.x - dm.y * Bm.y;
                        z[km] = outm;
                    }
                    z[k] = outk;
                }
            }
            __syncthreads();
        }
        if (MODE == DCT_MID) {
            // ---- divide by the eigenvalues; G = (1/N^2) sum w X^2 / lambda ------------
            if (active) {
                // index of the line along the other axis: the row of a row tile,
                // else the axis-0 position of an interleaved tile
                const int ia = (CONTIG ? (int)tl.outer : tl.i0) + 2 * pp, ib = ia + 1;
                const bool has_b = (2 * pp + 1 < tl.wact);
                T La = a.lam_a0[ia], Lb = has_b ? a.lam_a0[ib] : (T)0;
                T wa = (ia == 0) ? (T)1 : (T)2, wb = (ib == 0) ? (T)1 : (T)2;
                if (a.lam_a1) {
                    const int jo = (int)tl.outer;
                    La += a.lam_a1[jo]; Lb += a.lam_a1[jo];
                    const T wo = (jo == 0) ? (T)1 : (T)2;
                    wa *= wo; wb *= wo;
                }
                for (int k = t; k < n; k += G) {
                    const T lk = a.lam_axis[k];
                    const T wk = (k == 0) ? (T)1 : (T)2;
                    C v = z[k];
                    const T la = La + lk, lb = Lb + lk;
                    T ga = (T)0, gb = (T)0;
                    if (la > (T)0) { ga = v.x / la; gsum.add_prod(wa * wk * v.x, ga); }
                    if (has_b && lb > (T)0) { gb = v.y / lb; gsum.add_prod(wb * wk * v.y, gb); }
                    v.x = ga; v.y = gb;
                    z[k] = v;
                }
            }
            acc += gsum.take();
            __syncthreads();
        }
        if (MODE != DCT_FWD) {
            // ---- combine the two real spectra into one complex sequence -----------
            if (active) {
                for (int k = t; k <= n / 2; k += G) {
                    const int km = (n - k) % n;
                    const C Xk = z[k], Xm = z[km];
                    // V_k = e^{i pi k/2n} (X_k - i X_{n-k}), X_n = 0; Z = Va + i Vb
                    const T xam = (k == 0) ? (T)0 : Xm.x, xbm = (k == 0) ? (T)0 : Xm.y;
                    const C dk = cconj(a.dtw[k]);
                    C Va, Vb;
                    Va.x = dk.x * Xk.x + dk.y * xam; Va.y = dk.y * Xk.x - dk.x * xam;
                    Vb.x = dk.x * Xk.y + dk.y * xbm; Vb.y = dk.y * Xk.y - dk.x * xbm;
                    C Zk; Zk.x = Va.x - Vb.y; Zk.y = Va.y + Vb.x;
                    if (km != k) {
                        const C dm = cconj(a.dtw[km]);
                        C Wa, Wb;
                        Wa.x = dm.x * Xm.x + dm.y * Xk.x; Wa.y = dm.y * Xm.x - dm.x * Xk.x;
                        Wb.x = dm.x * Xm.y + dm.y * Xk.y; Wb.y = dm.y * Xm.y - dm.x * Xk.y;
                        C Zm; Zm.x = Wa.x - Wb.y; Zm.y = Wa.y + Wb.x;
                        z[km] = Zm;
                    }
                    z[k] = Zk;
                }
            }
            __syncthreads();
            // ---- inverse DIF FFT -----------------------------------------------------
            for (int s = a.nst - 1; s >= 0; --s) {
                const int r = a.rad[s];
                const int L = a.Ls[s];
                const int Lp = L * r;
                const int tstep = (s + 1 < a.nst) ? n / Lp : 1;
                const unsigned mg = a.mag[s];
                const int nb = (r == 4) ? (n >> 2) : (r == 2 ? (n >> 1) : n / 3);
                if (active) {
                    if (r == 4) dif_stage<4>(z, a.tw, t, G, nb, L, Lp, tstep, mg);
                    else if (r == 2) dif_stage<2>(z, a.tw, t, G, nb, L, Lp, tstep, mg);
                    else dif_stage<3>(z, a.tw, t, G, nb, L, Lp, tstep, mg);
                }
                __syncthreads();
            }
        }
        // ---- store ------------------------------------------------------------------
        {
            // the potential update reads its U values before any store
            constexpr int U = 4;
            const int np_pow = CONTIG ? 1 : (1 << a.lnp);
            const int per = CONTIG ? n : np_pow * n;
            const int reps = CONTIG ? np : 1;
            const int bd = blockDim.x;
            for (int q0 = 0; q0 < reps; ++q0)
            for (int e0 = tid; e0 < per; e0 += U * bd) {
                T ua[U], ub[U];
                if (MODE == DCT_INV && a.upd) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e = e0 + u * bd;
                        int q, j;
                        if (CONTIG) { q = q0; j = e; }
                        else        { q = e & (np_pow - 1); j = e >> a.lnp; }
                        ua[u] = ub[u] = (T)0;
                        if (e < per && q < np) {
                            const long long ada = tl.base0 + (long long)(2 * q) * tl.lstride + (long long)j * lt.es;
                            ua[u] = a.upd[ada];
                            if (2 * q + 1 < tl.wact) ub[u] = a.upd[ada + tl.lstride];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * bd;
                    int q, j;
                    if (CONTIG) { q = q0; j = e; }
                    else        { q = e & (np_pow - 1); j = e >> a.lnp; }
                    if (e >= per || q >= np) continue;
                    const int lb = 2 * q + 1;
                    const long long ada = tl.base0 + (long long)(2 * q) * tl.lstride + (long long)j * lt.es;
                    C v;
                    if (MODE == DCT_FWD) {
                        v = zs[(size_t)q * a.LDZ + j];
                    } else {
                        const int m = (j & 1) ? (n - 1 - (j >> 1)) : (j >> 1);
                        v = zs[(size_t)q * a.LDZ + a.drev[m]];
                        v.x *= inv_n;
                        v.y *= inv_n;
                    }
                    if (MODE == DCT_INV && a.upd) {
                        a.out[ada] = ua[u] + sig * v.x;
                        if (lb < tl.wact) a.out[ada + tl.lstride] = ub[u] + sig * v.y;
                    } else {
                        a.out[ada] = v.x;
                        if (lb < tl.wact) a.out[ada + tl.lstride] = v.y;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (MODE == DCT_MID && a.part) {
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) a.part[blockIdx.x] = s * a.gscale;
    }
    (void)npair_max;
}

// ---------------------------------------------------------------------------
// FP32 lines of power-of-two length: register Stockham FFT
// ---------------------------------------------------------------------------
// Each of the T = n/16 threads of a line pair holds 16 complex values per
// pass and applies radix-R butterflies (R = 16, the last pass 2, 4, 8 or 16)
// in registers.  A Stockham pass reads element j + r n/R, twiddles by
// e^{-+2 pi i (j mod Ns) r / (Ns R)}, transforms over r and writes
// ((j - j mod Ns) R + j mod Ns) + r Ns, so input and output are both in
// natural order and no digit reversal is needed.  Shared memory holds the
// pair with one pad element per 16, which keeps every pass's reads and writes
// free of bank conflicts.  Reads complete (barrier) before writes: in place.
__device__ __forceinline__ int padix(int i) { return i + (i >> 4); }

template <int SIGN>
__device__ __forceinline__ float2 cmul_sgn(float2 a, float2 w)
{
    // a * w (SIGN < 0) or a * conj(w) (SIGN > 0)
    float2 r;
    if (SIGN < 0) { r.x = a.x * w.x - a.y * w.y; r.y = a.x * w.y + a.y * w.x; }
    else          { r.x = a.x * w.x + a.y * w.y; r.y = a.y * w.x - a.x * w.y; }
    return r;
}

// radix-4 in place on v[o], v[o+s], v[o+2s], v[o+3s]
template <int SIGN, typename A>
__device__ __forceinline__ void r4(A& v, int o, int s)
{
    const float2 a0 = cadd(v[o], v[o + 2 * s]), a1 = csub(v[o], v[o + 2 * s]);
    const float2 b0 = cadd(v[o + s], v[o + 3 * s]), b1 = csub(v[o + s], v[o + 3 * s]);
    float2 ib1;
    if (SIGN < 0) { ib1.x = b1.y; ib1.y = -b1.x; } else { ib1.x = -b1.y; ib1.y = b1.x; }
    v[o] = cadd(a0, b0);
    v[o + 2 * s] = csub(a0, b0);
    v[o + s] = cadd(a1, ib1);
    v[o + 3 * s] = csub(a1, ib1);
}

// X[k] = sum_m v[O+m] e^{SIGN 2 pi i m k / R}, in place on v[O..O+R); X[k] is
// left in slot O + out_slot<R>(k) (radix 8 and 16 leave their outputs transposed)
template <int R>
__host__ __device__ constexpr int out_slot(int k)
{
    return R == 16 ? 4 * (k % 4) + k / 4 : R == 8 ? 2 * (k % 4) + k / 4 : k;
}

template <int R, int SIGN, int O>
__device__ __forceinline__ void dft_reg(float2 (&v)[16])
{
    if (R == 2) {
        const float2 a = v[O], b = v[O + 1];
        v[O] = cadd(a, b); v[O + 1] = csub(a, b);
    } else if (R == 4) {
        r4<SIGN>(v, O, 1);
    } else if (R == 8) {
        // m = 2 m1 + m2: radix-4 over m1, twiddle W8^(m2 k1), radix-2 over m2
        r4<SIGN>(v, O, 2);
        r4<SIGN>(v, O + 1, 2);
        const float c = 0.70710678118654752440f;
        float2 t;
        t = v[O + 3]; v[O + 3].x = c * (t.x - SIGN * t.y); v[O + 3].y = c * (t.y + SIGN * t.x);
        t = v[O + 5]; v[O + 5].x = -SIGN * t.y;           v[O + 5].y = SIGN * t.x;   // times SIGN i
        t = v[O + 7]; v[O + 7].x = c * (-t.x - SIGN * t.y); v[O + 7].y = c * (-t.y + SIGN * t.x);
        // X[k1 + 4 k2] is left at v[O + 2 k1 + k2] (see out_slot)
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const float2 a = v[O + 2 * k1], b = v[O + 2 * k1 + 1];
            v[O + 2 * k1] = cadd(a, b);
            v[O + 2 * k1 + 1] = csub(a, b);
        }
    } else {  // R == 16: m = 4 m1 + m2: radix-4 over m1, twiddle W16^(m2 k1), radix-4 over m2
#pragma unroll
        for (int m2 = 0; m2 < 4; ++m2) r4<SIGN>(v, O + m2, 4);        // v[O + m2 + 4 k1]
        const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
        const float c2 = 0.70710678118654752440f;
#pragma unroll
        for (int m2 = 1; m2 < 4; ++m2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) {
                const int m = m2 * k1;                       // W16^m, m in {1,2,3,4,6,9}
                const float wc = (m == 1) ? c1 : (m == 2) ? c2 : (m == 3) ? s1 : (m == 4) ? 0.f
                               : (m == 6) ? -c2 : -c1;
                const float ws = (m == 1) ? s1 : (m == 2) ? c2 : (m == 3) ? c1 : (m == 4) ? 1.f
                               : (m == 6) ? c2 : -s1;
                // W16^m = cos(2 pi m/16) + SIGN i sin(2 pi m/16)
                const float2 a = v[O + m2 + 4 * k1];
                float2 b;
                b.x = a.x * wc - SIGN * a.y * ws;
                b.y = a.y * wc + SIGN * a.x * ws;
                v[O + m2 + 4 * k1] = b;
            }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) r4<SIGN>(v, O + 4 * k1, 1);   // X[k1 + 4 k2] left at v[O + 4 k1 + k2]
    }
}

// Twiddles of a pass of stride Ns come from its own block of the pass table,
// laid out [r][k], so the lanes of a warp (consecutive k) read consecutive
// entries; the first pass (Ns = 1) has none.
template <int R, int SIGN, int Bi>
__device__ __forceinline__ void read_bfly(const float2* z, int n, int Ns, int t, int T,
                                          const float2* ptw, float2 (&v)[16])
{
    const int j = t + Bi * T;
    const int k = j & (Ns - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) v[Bi * R + r] = z[padix(j + r * (n / R))];
    if (Ns > 1) {
        const float2* pw = ptw + (Ns - 1) + k;
#pragma unroll
        for (int r = 1; r < R; ++r) v[Bi * R + r] = cmul_sgn<SIGN>(v[Bi * R + r], pw[(r - 1) * Ns]);
    }
    dft_reg<R, SIGN, Bi * R>(v);
}

template <int R, int SIGN>
__device__ __forceinline__ void pass_read(const float2* z, int n, int Ns, int t, int T,
                                          const float2* ptw, float2 (&v)[16])
{
    read_bfly<R, SIGN, 0>(z, n, Ns, t, T, ptw, v);
    if (16 / R > 1) read_bfly<R, SIGN, (16 / R > 1 ? 1 : 0)>(z, n, Ns, t, T, ptw, v);
    if (16 / R > 2) {
        read_bfly<R, SIGN, (16 / R > 2 ? 2 : 0)>(z, n, Ns, t, T, ptw, v);
        read_bfly<R, SIGN, (16 / R > 2 ? 3 : 0)>(z, n, Ns, t, T, ptw, v);
    }
    if (16 / R > 4) {
#pragma unroll
        for (int b = 4; b < 8; ++b) {
            const int j = t + b * T;
            const int k = j & (Ns - 1);
            float2 x0 = z[padix(j)], x1 = z[padix(j + n / R)];
            if (Ns > 1) x1 = cmul_sgn<SIGN>(x1, ptw[(Ns - 1) + k]);
            v[2 * b] = cadd(x0, x1);
            v[2 * b + 1] = csub(x0, x1);
        }
    }
}

template <int R>
__device__ __forceinline__ void pass_write(float2* z, int Ns, int t, int T, const float2 (&v)[16])
{
    constexpr int B = 16 / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * T;
        const int k = j & (Ns - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) z[padix(base + r * Ns)] = v[b * R + out_slot<R>(r)];
    }
}

// One FFT of every pair held by the CTA (all threads take part: barriers).
template <int SIGN>
__device__ __forceinline__ void stockham_fft(float2* z, int n, int t, int T, bool active, const float2* ptw,
                             int nst, const int* rad)
{
    float2 v[16];
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
        const int R = rad[s];
        if (active) {
            if (R == 16) pass_read<16, SIGN>(z, n, Ns, t, T, ptw, v);
            else if (R == 8) pass_read<8, SIGN>(z, n, Ns, t, T, ptw, v);
            else if (R == 4) pass_read<4, SIGN>(z, n, Ns, t, T, ptw, v);
            else pass_read<2, SIGN>(z, n, Ns, t, T, ptw, v);
        }
        __syncthreads();
        if (active) {
            if (R == 16) pass_write<16>(z, Ns, t, T, v);
            else if (R == 8) pass_write<8>(z, Ns, t, T, v);
            else if (R == 4) pass_write<4>(z, Ns, t, T, v);
            else pass_write<2>(z, Ns, t, T, v);
        }
        __syncthreads();
        Ns *= R;
    }
}

// The MID pass runs a forward and an inverse FFT in one kernel; inlined
// together they exceed 128 registers and spill, so there each FFT is a call
// with its own register allocation.
template <int SIGN>
__device__ __noinline__ void stockham_fft_call(float2* z, int n, int t, int T, bool active,
                                               const float2* ptw, int nst, const int* rad)
{
    stockham_fft<SIGN>(z, n, t, T, active, ptw, nst, rad);
}

template <int MODE, bool CONTIG, bool BATCHED>
__global__ void __launch_bounds__(256, MODE == DCT_MID ? 2 : 3) dct_fast_kernel(DctArgs<float> a0, const DctArgs<float>* batch)
{
    using C = float2;
    using T = float;
    const DctArgs<float>& a = BATCHED ? batch[blockIdx.y] : a0;
    if (BATCHED && blockIdx.x >= a.lt.ntiles) return;
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* zs = reinterpret_cast<C*>(smem_raw);
    __shared__ double red[32];
    const LineTiles& lt = a.lt;
    const int n = lt.n;
    const int G = a.G;                      // threads per pair = n / 16
    const int tid = threadIdx.x;
    const int pp = tid / G, t = tid - pp * G;
    C* z = zs + (size_t)pp * a.LDZ;
    const T inv_n = (T)1 / (T)n;
    T sig = (T)0;
    if (MODE == DCT_INV && a.upd) sig = (T)(*a.sigma);
    double acc = 0.0;
    Acc<T> gsum;

    for (long long tile = blockIdx.x; tile < lt.ntiles; tile += gridDim.x) {
        const Tile tl = tile_at(lt, tile);
        const int np = (tl.wact + 1) / 2;
        const bool active = (pp < np);
        // ---- load: natural order of the reordered sequence (FWD/MID) or spectrum (INV).
        // Each thread issues U independent loads before storing any, so a tile's
        // loads overlap instead of forming a chain of memory latencies.
        {
            constexpr int U = 4;
            const int np_pow = CONTIG ? 1 : (1 << a.lnp);
            const int per = CONTIG ? n : np_pow * n;
            const int reps = CONTIG ? np : 1;
            const int bd = blockDim.x;
            for (int q0 = 0; q0 < reps; ++q0)
            for (int e0 = tid; e0 < per; e0 += U * bd) {
                T xa[U], xb[U], ba[U], bb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * bd;
                    xa[u] = xb[u] = ba[u] = bb[u] = (T)0;
                    int q, j;
                    if (CONTIG) { q = q0; j = e; } else { q = e & (np_pow - 1); j = e >> a.lnp; }
                    if (e < per && q < np) {
                        const long long ada = tl.base0 + (long long)(2 * q) * tl.lstride + (long long)j * lt.es;
                        const bool hb = (2 * q + 1 < tl.wact);
                        xa[u] = a.in[ada];
                        if (hb) xb[u] = a.in[ada + tl.lstride];
                        if (MODE == DCT_FWD && a.base) {
                            ba[u] = a.base[ada];
                            if (hb) bb[u] = a.base[ada + tl.lstride];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * bd;
                    int q, j;
                    if (CONTIG) { q = q0; j = e; } else { q = e & (np_pow - 1); j = e >> a.lnp; }
                    if (e < per && q < np) {
                        C v;
                        if (MODE == DCT_FWD && a.base) { v.x = ba[u] - xa[u]; v.y = bb[u] - xb[u]; }
                        else { v.x = xa[u]; v.y = xb[u]; }
                        const int m = (MODE == DCT_INV) ? j : ((j & 1) ? (n - 1 - (j >> 1)) : (j >> 1));
                        zs[(size_t)q * a.LDZ + padix(m)] = v;
                    }
                }
            }
        }
        __syncthreads();
        if (MODE != DCT_INV) {
            if (MODE == DCT_MID) stockham_fft_call<-1>(z, n, t, G, active, a.ptw, a.fnst, a.frad);
            else stockham_fft<-1>(z, n, t, G, active, a.ptw, a.fnst, a.frad);
            if (active) {
                for (int k = t; k <= n / 2; k += G) {
                    const int km = (n - k) % n;
                    const C Zk = z[padix(k)], Zm = z[padix(km)];
                    C A, Bq;
                    A.x = (T)0.5 * (Zk.x + Zm.x); A.y = (T)0.5 * (Zk.y - Zm.y);
                    Bq.x = (T)0.5 * (Zk.y + Zm.y); Bq.y = (T)0.5 * (Zm.x - Zk.x);
                    const C dk = a.dtw[k];
                    C outk; outk.x = dk.x * A.x - dk.y * A.y; outk.y = dk.x * Bq.x - dk.y * Bq.y;
                    if (km != k) {
                        C Am, Bm;
                        Am.x = (T)0.5 * (Zm.x + Zk.x); Am.y = (T)0.5 * (Zm.y - Zk.y);
                        Bm.x = (T)0.5 * (Zm.y + Zk.y); Bm.y = (T)0.5 * (Zk.x - Zm.x);
                        const C dm = a.dtw[km];
                        C outm; outm.x = dm.x * Am.x - dm.y * Am.y; outm.y = dm.x * Bm.x - dm.y * Bm.y;
                        z[padix(km)] = outm;
                    }
                    z[padix(k)] = outk;
                }
            }
            __syncthreads();
        }
        if (MODE == DCT_MID) {
            if (active) {
                // index of the line along the other axis: the row of a row tile,
                // else the axis-0 position of an interleaved tile
                const int ia = (CONTIG ? (int)tl.outer : tl.i0) + 2 * pp, ib = ia + 1;
                const bool has_b = (2 * pp + 1 < tl.wact);
                T La = a.lam_a0[ia], Lb = has_b ? a.lam_a0[ib] : (T)0;
                T wa = (ia == 0) ? (T)1 : (T)2, wb = (ib == 0) ? (T)1 : (T)2;
                if (a.lam_a1) {
                    const int jo = (int)tl.outer;
                    La += a.lam_a1[jo]; Lb += a.lam_a1[jo];
                    const T wo = (jo == 0) ? (T)1 : (T)2;
                    wa *= wo; wb *= wo;
                }
                for (int k = t; k < n; k += G) {
                    const T lk = a.lam_axis[k];
                    const T wk = (k == 0) ? (T)1 : (T)2;
                    C v = z[padix(k)];
                    const T la = La + lk, lb = Lb + lk;
                    T ga = (T)0, gb = (T)0;
                    if (la > (T)0) { ga = v.x / la; gsum.add_prod(wa * wk * v.x, ga); }
                    if (has_b && lb > (T)0) { gb = v.y / lb; gsum.add_prod(wb * wk * v.y, gb); }
                    v.x = ga; v.y = gb;
                    z[padix(k)] = v;
                }
            }
            acc += gsum.take();
            __syncthreads();
        }
        if (MODE != DCT_FWD) {
            if (active) {
                for (int k = t; k <= n / 2; k += G) {
                    const int km = (n - k) % n;
                    const C Xk = z[padix(k)], Xm = z[padix(km)];
                    const T xam = (k == 0) ? (T)0 : Xm.x, xbm = (k == 0) ? (T)0 : Xm.y;
                    const C dk = cconj(a.dtw[k]);
                    C Va, Vb;
                    Va.x = dk.x * Xk.x + dk.y * xam; Va.y = dk.y * Xk.x - dk.x * xam;
                    Vb.x = dk.x * Xk.y + dk.y * xbm; Vb.y = dk.y * Xk.y - dk.x * xbm;
                    C Zk; Zk.x = Va.x - Vb.y; Zk.y = Va.y + Vb.x;
                    if (km != k) {
                        const C dm = cconj(a.dtw[km]);
                        C Wa, Wb;
                        Wa.x = dm.x * Xm.x + dm.y * Xk.x; Wa.y = dm.y * Xm.x - dm.x * Xk.x;
                        Wb.x = dm.x * Xm.y + dm.y * Xk.y; Wb.y = dm.y * Xm.y - dm.x * Xk.y;
                        C Zm; Zm.x = Wa.x - Wb.y; Zm.y = Wa.y + Wb.x;
                        z[padix(km)] = Zm;
                    }
                    z[padix(k)] = Zk;
                }
            }
            __syncthreads();
            if (MODE == DCT_MID) stockham_fft_call<+1>(z, n, t, G, active, a.ptw, a.fnst, a.frad);
            else stockham_fft<+1>(z, n, t, G, active, a.ptw, a.fnst, a.frad);
        }
        // ---- store (the potential update reads its U values first) ------------------
        {
            constexpr int U = 4;
            const int np_pow = CONTIG ? 1 : (1 << a.lnp);
            const int per = CONTIG ? n : np_pow * n;
            const int reps = CONTIG ? np : 1;
            const int bd = blockDim.x;
            for (int q0 = 0; q0 < reps; ++q0)
            for (int e0 = tid; e0 < per; e0 += U * bd) {
                T ua[U], ub[U];
                if (MODE == DCT_INV && a.upd) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e = e0 + u * bd;
                        ua[u] = ub[u] = (T)0;
                        int q, j;
                        if (CONTIG) { q = q0; j = e; } else { q = e & (np_pow - 1); j = e >> a.lnp; }
                        if (e < per && q < np) {
                            const long long ada = tl.base0 + (long long)(2 * q) * tl.lstride + (long long)j * lt.es;
                            ua[u] = a.upd[ada];
                            if (2 * q + 1 < tl.wact) ub[u] = a.upd[ada + tl.lstride];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * bd;
                    int q, j;
                    if (CONTIG) { q = q0; j = e; } else { q = e & (np_pow - 1); j = e >> a.lnp; }
                    if (e >= per || q >= np) continue;
                    const int lb = 2 * q + 1;
                    const long long ada = tl.base0 + (long long)(2 * q) * tl.lstride + (long long)j * lt.es;
                    C v;
                    if (MODE == DCT_FWD) {
                        v = zs[(size_t)q * a.LDZ + padix(j)];
                    } else {
                        const int m = (j & 1) ? (n - 1 - (j >> 1)) : (j >> 1);
                        v = zs[(size_t)q * a.LDZ + padix(m)];
                        v.x *= inv_n;
                        v.y *= inv_n;
                    }
                    if (MODE == DCT_INV && a.upd) {
                        a.out[ada] = ua[u] + sig * v.x;
                        if (lb < tl.wact) a.out[ada + tl.lstride] = ub[u] + sig * v.y;
                    } else {
                        a.out[ada] = v.x;
                        if (lb < tl.wact) a.out[ada + tl.lstride] = v.y;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (MODE == DCT_MID && a.part) {
        const double sacc = block_sum(acc, red);
        if (threadIdx.x == 0) a.part[blockIdx.x] = sacc * a.gscale;
    }
}

// ---------------------------------------------------------------------------
// Rows of 1024, 2048 or 4096 FP32 cells (the axis-0 passes and the middle
// pass on a transposed copy of 2-D grids): the same line-pair transform as
// dct_fast_kernel with the length fixed at compile time, so the pass
// structure, strides and twiddle offsets are constants, and each row moves as
// float4 vectors, every load of a pair issued before any is used.  One line
// pair per CTA of n/16 threads; a resident wave of CTAs loops over the pairs.
// ---------------------------------------------------------------------------
template <int SIGN, int LOGN>
__device__ __forceinline__ void fft_fixed(float2* z, int t, const float2* ptw)
{
    constexpr int n = 1 << LOGN, T = n / 16, NP = LOGN / 4;
    float2 v[16];
#pragma unroll
    for (int s = 0; s < NP; ++s) {
        const int Ns = 1 << (4 * s);
        pass_read<16, SIGN>(z, n, Ns, t, T, ptw, v);
        __syncthreads();
        pass_write<16>(z, Ns, t, T, v);
        __syncthreads();
    }
    if (LOGN % 4) {
        constexpr int R = 1 << (LOGN % 4), Ns = 1 << (4 * NP);
        pass_read<R, SIGN>(z, n, Ns, t, T, ptw, v);
        __syncthreads();
        pass_write<R>(z, Ns, t, T, v);
        __syncthreads();
    }
}

template <int SIGN, int LOGN>
__device__ __noinline__ void fft_fixed_call(float2* z, int t, const float2* ptw)
{
    fft_fixed<SIGN, LOGN>(z, t, ptw);
}

// position of element j of a line in the even/odd reordering
// (x0, x2, x4, ..., x5, x3, x1): m(j) = j/2 for even j, n - 1 - (j-1)/2 for odd j
template <int N>
__device__ __forceinline__ int reorder_pos(int j) { return (j & 1) ? (N - 1 - (j >> 1)) : (j >> 1); }

// resident CTAs per SM of 256 threads (rows of 4096; shorter rows scale up):
// the register budget per thread is 65536 / (256 x this)
constexpr int dct_row_ctas(int mode, int logn)
{
    return mode == DCT_FWD ? 3 : mode == DCT_INV ? 3 : (logn == 12 ? 4 : 2);
}

// BATCHED: blockIdx.y selects the problem, whose arguments come from `batch`.
template <int MODE, int LOGN, bool BATCHED>
__global__ void __launch_bounds__((1 << LOGN) / 16, dct_row_ctas(MODE, LOGN) * (4096 >> LOGN))
dct_row_kernel(DctArgs<float> a0, const DctArgs<float>* batch)
{
    using C = float2;
    constexpr int n = 1 << LOGN, T = n / 16, NQ = n / 4, QPT = NQ / T;   // QPT = 4 float4 per row
    const DctArgs<float>& a = BATCHED ? batch[blockIdx.y] : a0;
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* z = reinterpret_cast<C*>(smem_raw);
    __shared__ double red[32];
    const int t = threadIdx.x;
    const long long nrows = a.lt.nlines;
    const long long npairs = (nrows + 1) >> 1;
    constexpr float inv_n = 1.0f / (float)n;
    float sig = 0.f;
    if (MODE == DCT_INV && a.upd) sig = (float)(*a.sigma);
    double acc = 0.0;
    Acc<float> gsum;

    for (long long pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const long long ra = 2 * pr;
        const bool hb = ra + 1 < nrows;
        const long long off = ra * n;
        // ---- load: both rows (and the base rows of FWD) as float4, all in flight at once
        {
            const float4* ina = reinterpret_cast<const float4*>(a.in + off);
            const float4* inb = ina + NQ;
            const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 xa[QPT], xb[QPT], ba[QPT], bb[QPT];
#pragma unroll
            for (int u = 0; u < QPT; ++u) {
                const int q = t + u * T;
                xa[u] = ina[q];
                xb[u] = hb ? inb[q] : zero4;
            }
            if (MODE == DCT_FWD && a.base) {
                const float4* bsa = reinterpret_cast<const float4*>(a.base + off);
                const float4* bsb = bsa + NQ;
#pragma unroll
                for (int u = 0; u < QPT; ++u) {
                    const int q = t + u * T;
                    ba[u] = bsa[q];
                    bb[u] = hb ? bsb[q] : zero4;
                }
#pragma unroll
                for (int u = 0; u < QPT; ++u) {
                    xa[u].x = ba[u].x - xa[u].x; xa[u].y = ba[u].y - xa[u].y;
                    xa[u].z = ba[u].z - xa[u].z; xa[u].w = ba[u].w - xa[u].w;
                    xb[u].x = bb[u].x - xb[u].x; xb[u].y = bb[u].y - xb[u].y;
                    xb[u].z = bb[u].z - xb[u].z; xb[u].w = bb[u].w - xb[u].w;
                }
            }
#pragma unroll
            for (int u = 0; u < QPT; ++u) {
                const int j = 4 * (t + u * T);
                const C c0 = make_float2(xa[u].x, xb[u].x), c1 = make_float2(xa[u].y, xb[u].y);
                const C c2 = make_float2(xa[u].z, xb[u].z), c3 = make_float2(xa[u].w, xb[u].w);
                if (MODE == DCT_INV) {
                    z[padix(j)] = c0; z[padix(j + 1)] = c1; z[padix(j + 2)] = c2; z[padix(j + 3)] = c3;
                } else {
                    z[padix(reorder_pos<n>(j))] = c0;     z[padix(reorder_pos<n>(j + 1))] = c1;
                    z[padix(reorder_pos<n>(j + 2))] = c2; z[padix(reorder_pos<n>(j + 3))] = c3;
                }
            }
        }
        __syncthreads();
        if (MODE == DCT_MID) {
            fft_fixed_call<-1, LOGN>(z, t, a.ptw);
            // One pass over the pairs (k, n - k): the DCT-II of both lines from
            // the pair's FFT (Makhoul), the division by lambda(row) + lambda(k)
            // with G = sum w |f^|^2 / lambda (Parseval weights 1, 2; zero mode
            // -> 0), and the inverse twiddle and recombination that feed the
            // inverse FFT -- the arithmetic of the three separate loops of the
            // other passes, without their shared-memory round trips.
            const long long ia = ra, ib = ra + 1;
            const float La = a.lam_a0[ia], Lb = hb ? a.lam_a0[ib] : 0.f;
            const float wa = (ia == 0) ? 1.f : 2.f, wb = 2.f;
            // G's terms are all positive: the (up to four) terms of one pair
            // (k, n - k) are summed in FP32, that sum into the compensated one
            float gp = 0.f;
            auto divide = [&](int kk, C v) {
                const float lk = a.lam_axis[kk];
                const float wk = (kk == 0) ? 1.f : 2.f;
                const float la = La + lk, lb = Lb + lk;
                float ga = 0.f, gb = 0.f;
                if (la > 0.f) { ga = __fdividef(v.x, la); gp = fmaf(wa * wk * v.x, ga, gp); }
                if (hb && lb > 0.f) { gb = __fdividef(v.y, lb); gp = fmaf(wb * wk * v.y, gb, gp); }
                v.x = ga; v.y = gb;
                return v;
            };
            for (int k = t; k <= n / 2; k += T) {
                gp = 0.f;
                const int km = (n - k) & (n - 1);
                const C Zk = z[padix(k)], Zm = z[padix(km)];
                C A, Bq;
                A.x = 0.5f * (Zk.x + Zm.x); A.y = 0.5f * (Zk.y - Zm.y);
                Bq.x = 0.5f * (Zk.y + Zm.y); Bq.y = 0.5f * (Zm.x - Zk.x);
                const C dk = a.dtw[k];
                C outk; outk.x = dk.x * A.x - dk.y * A.y; outk.y = dk.x * Bq.x - dk.y * Bq.y;
                const C Xk = divide(k, outk);
                C Xm = Xk;
                const C dm = a.dtw[km];
                if (km != k) {
                    C Am, Bm;
                    Am.x = 0.5f * (Zm.x + Zk.x); Am.y = 0.5f * (Zm.y - Zk.y);
                    Bm.x = 0.5f * (Zm.y + Zk.y); Bm.y = 0.5f * (Zk.x - Zm.x);
                    C outm; outm.x = dm.x * Am.x - dm.y * Am.y; outm.y = dm.x * Bm.x - dm.y * Bm.y;
                    Xm = divide(km, outm);
                }
                const float xam = (k == 0) ? 0.f : Xm.x, xbm = (k == 0) ? 0.f : Xm.y;
                const C dki = cconj(dk);
                C Va, Vb;
                Va.x = dki.x * Xk.x + dki.y * xam; Va.y = dki.y * Xk.x - dki.x * xam;
                Vb.x = dki.x * Xk.y + dki.y * xbm; Vb.y = dki.y * Xk.y - dki.x * xbm;
                C Zk2; Zk2.x = Va.x - Vb.y; Zk2.y = Va.y + Vb.x;
                if (km != k) {
                    const C dmi = cconj(dm);
                    C Wa, Wb;
                    Wa.x = dmi.x * Xm.x + dmi.y * Xk.x; Wa.y = dmi.y * Xm.x - dmi.x * Xk.x;
                    Wb.x = dmi.x * Xm.y + dmi.y * Xk.y; Wb.y = dmi.y * Xm.y - dmi.x * Xk.y;
                    C Zm2; Zm2.x = Wa.x - Wb.y; Zm2.y = Wa.y + Wb.x;
                    z[padix(km)] = Zm2;
                }
                z[padix(k)] = Zk2;
                gsum.add(gp);
            }
            acc += gsum.take();
            __syncthreads();
            fft_fixed_call<+1, LOGN>(z, t, a.ptw);
        } else {
        // FWD: forward FFT and the DCT-II split; INV: inverse twiddle and FFT
        if (MODE != DCT_INV) {
                fft_fixed<-1, LOGN>(z, t, a.ptw);
                // DCT-II from the FFT of the pair (Makhoul): split the two real
                // lines' spectra, then twiddle by e^{-i pi k/(2n)}
                for (int k = t; k <= n / 2; k += T) {
                    const int km = (n - k) & (n - 1);
                    const C Zk = z[padix(k)], Zm = z[padix(km)];
                    C A, Bq;
                    A.x = 0.5f * (Zk.x + Zm.x); A.y = 0.5f * (Zk.y - Zm.y);
                    Bq.x = 0.5f * (Zk.y + Zm.y); Bq.y = 0.5f * (Zm.x - Zk.x);
                    const C dk = a.dtw[k];
                    C outk; outk.x = dk.x * A.x - dk.y * A.y; outk.y = dk.x * Bq.x - dk.y * Bq.y;
                    if (km != k) {
                        C Am, Bm;
                        Am.x = 0.5f * (Zm.x + Zk.x); Am.y = 0.5f * (Zm.y - Zk.y);
                        Bm.x = 0.5f * (Zm.y + Zk.y); Bm.y = 0.5f * (Zk.x - Zm.x);
                        const C dm = a.dtw[km];
                        C outm; outm.x = dm.x * Am.x - dm.y * Am.y; outm.y = dm.x * Bm.x - dm.y * Bm.y;
                        z[padix(km)] = outm;
                    }
                    z[padix(k)] = outk;
                }
                __syncthreads();
            }
            if (MODE != DCT_FWD) {
                // undo the DCT-II twiddle and recombine the pair's spectra
                for (int k = t; k <= n / 2; k += T) {
                    const int km = (n - k) & (n - 1);
                    const C Xk = z[padix(k)], Xm = z[padix(km)];
                    const float xam = (k == 0) ? 0.f : Xm.x, xbm = (k == 0) ? 0.f : Xm.y;
                    const C dk = cconj(a.dtw[k]);
                    C Va, Vb;
                    Va.x = dk.x * Xk.x + dk.y * xam; Va.y = dk.y * Xk.x - dk.x * xam;
                    Vb.x = dk.x * Xk.y + dk.y * xbm; Vb.y = dk.y * Xk.y - dk.x * xbm;
                    C Zk; Zk.x = Va.x - Vb.y; Zk.y = Va.y + Vb.x;
                    if (km != k) {
                        const C dm = cconj(a.dtw[km]);
                        C Wa, Wb;
                        Wa.x = dm.x * Xm.x + dm.y * Xk.x; Wa.y = dm.y * Xm.x - dm.x * Xk.x;
                        Wb.x = dm.x * Xm.y + dm.y * Xk.y; Wb.y = dm.y * Xm.y - dm.x * Xk.y;
                        C Zm; Zm.x = Wa.x - Wb.y; Zm.y = Wa.y + Wb.x;
                        z[padix(km)] = Zm;
                    }
                    z[padix(k)] = Zk;
                }
                __syncthreads();
                fft_fixed_call<+1, LOGN>(z, t, a.ptw);
            }
        }
        // ---- store: float4 per row (INV with an update reads its rows first) --------
        {
            float4* oa = reinterpret_cast<float4*>(a.out + off);
            float4* ob = oa + NQ;
            float4 ua[QPT], ub[QPT];
            if (MODE == DCT_INV && a.upd) {
                const float4* pa = reinterpret_cast<const float4*>(a.upd + off);
                const float4* pb = pa + NQ;
#pragma unroll
                for (int u = 0; u < QPT; ++u) {
                    const int q = t + u * T;
                    ua[u] = pa[q];
                    ub[u] = hb ? pb[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < QPT; ++u) {
                const int q = t + u * T, j = 4 * q;
                C c[4];
                if (MODE == DCT_FWD) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) c[e] = z[padix(j + e)];
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        c[e] = z[padix(reorder_pos<n>(j + e))];
                        c[e].x *= inv_n;
                        c[e].y *= inv_n;
                    }
                }
                float4 va = make_float4(c[0].x, c[1].x, c[2].x, c[3].x);
                float4 vb = make_float4(c[0].y, c[1].y, c[2].y, c[3].y);
                if (MODE == DCT_INV && a.upd) {
                    va.x = ua[u].x + sig * va.x; va.y = ua[u].y + sig * va.y;
                    va.z = ua[u].z + sig * va.z; va.w = ua[u].w + sig * va.w;
                    vb.x = ub[u].x + sig * vb.x; vb.y = ub[u].y + sig * vb.y;
                    vb.z = ub[u].z + sig * vb.z; vb.w = ub[u].w + sig * vb.w;
                }
                oa[q] = va;
                if (hb) ob[q] = vb;
            }
        }
        __syncthreads();
    }
    if (MODE == DCT_MID && a.part) {
        const double sacc = block_sum(acc, red);
        if (threadIdx.x == 0) a.part[blockIdx.x] = sacc * a.gscale;
    }
}

// ---------------------------------------------------------------------------
// Lines of 384 FP32 cells (the 3-D workload's axes): one warp per line pair,
// 12 complex values per lane, a register Stockham FFT with radices
// 4 x 4 x 4 x 6 whose passes synchronise only the warp.  A CTA holds 32 lines
// (16 pairs): 32 neighbouring rows, or 32 neighbouring lines of an axis > 0
// whose element j is a run of 32 consecutive floats; both move as float4.
// ---------------------------------------------------------------------------
template <int SIGN>
__device__ __forceinline__ void dft6(float2* u)
{
    // m = 2 m1 + m2: three-point transforms over m1, twiddle w6^(m2 k1), two-point over m2
    const float s3 = (float)SIGN * 0.86602540378443864676f;   // sin(2 pi/3) with sign
    float2 y[2][3];
#pragma unroll
    for (int m2 = 0; m2 < 2; ++m2) {
        const float2 u0 = u[m2], u1 = u[2 + m2], u2 = u[4 + m2];
        const float2 t1 = cadd(u1, u2), t2 = csub(u1, u2);
        const float2 m = make_float2(u0.x - 0.5f * t1.x, u0.y - 0.5f * t1.y);
        const float2 it2 = make_float2(-s3 * t2.y, s3 * t2.x);
        y[m2][0] = cadd(u0, t1);
        y[m2][1] = cadd(m, it2);
        y[m2][2] = csub(m, it2);
    }
    // w6 = e^{SIGN i pi/3} = (1/2, SIGN sqrt3/2), w6^2 = (-1/2, SIGN sqrt3/2)
    const float2 a1 = y[1][1], a2 = y[1][2];
    y[1][1] = make_float2(0.5f * a1.x - s3 * a1.y, 0.5f * a1.y + s3 * a1.x);
    y[1][2] = make_float2(-0.5f * a2.x - s3 * a2.y, -0.5f * a2.y + s3 * a2.x);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        u[k1] = cadd(y[0][k1], y[1][k1]);
        u[k1 + 3] = csub(y[0][k1], y[1][k1]);
    }
}

// One Stockham pass of radix R and stride Ns over a line of N held by the
// T = N / V lanes of a warp, V values per lane (V / R butterflies each).
template <int N, int V, int R, int Ns, int SIGN>
__device__ __forceinline__ void passv(float2* z, int t, const float2* ptw)
{
    constexpr int T = N / V, B = V / R;
    float2 v[V];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * T;
        const int k = j % Ns;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = z[padix(j + r * (N / R))];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[b * R + r] = cmul_sgn<SIGN>(v[b * R + r], ptw[(Ns - 1) + (r - 1) * Ns + k]);
        }
        if (R == 4) r4<SIGN>(v, b * R, 1);
        else dft6<SIGN>(v + b * R);
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * T;
        const int k = j % Ns;
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) z[padix(base + r * Ns)] = v[b * R + r];
    }
    __syncwarp();
}

template <int SIGN>
__device__ __forceinline__ void fft384(float2* z, int t, const float2* ptw)
{
    passv<384, 12, 4, 1, SIGN>(z, t, ptw);
    passv<384, 12, 4, 4, SIGN>(z, t, ptw);
    passv<384, 12, 4, 16, SIGN>(z, t, ptw);
    passv<384, 12, 6, 64, SIGN>(z, t, ptw);
}

template <int MODE, bool CONTIG>
__global__ void __launch_bounds__(512, 2) dct384_kernel(DctArgs<float> a)
{
    using C = float2;
    constexpr int N = 384, LDZ = N + N / 16 + 1;
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* zs = reinterpret_cast<C*>(smem_raw);
    __shared__ double red[32];
    const LineTiles& lt = a.lt;
    const int tid = threadIdx.x, lane = tid & 31, pw = tid >> 5;     // warp = line pair
    C* z = zs + pw * LDZ;
    constexpr float inv_n = 1.0f / (float)N;
    float sig = 0.f;
    if (MODE == DCT_INV && a.upd) sig = (float)(*a.sigma);
    double acc = 0.0;
    Acc<float> gsum;

    for (long long tile = blockIdx.x; tile < lt.ntiles; tile += gridDim.x) {
        const Tile tl = tile_at(lt, tile);               // every tile holds W lines
        // ---- load: 32 lines x 384 = 3072 float4, six per thread ----------------------
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 x[3], b[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int e = tid + 512 * (3 * h + u);
                long long ad;
                if (CONTIG) ad = tl.base0 + (long long)(tid >> 4) * N + 4 * ((tid & 15) + 16 * (3 * h + u));
                else ad = tl.base0 + 4 * (e & 7) + (long long)(e >> 3) * lt.es;
                x[u] = *reinterpret_cast<const float4*>(a.in + ad);
                if (MODE == DCT_FWD && a.base) b[u] = *reinterpret_cast<const float4*>(a.base + ad);
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int e = tid + 512 * (3 * h + u);
                float4 v = x[u];
                if (MODE == DCT_FWD && a.base) {
                    v.x = b[u].x - v.x; v.y = b[u].y - v.y; v.z = b[u].z - v.z; v.w = b[u].w - v.w;
                }
                if (CONTIG) {
                    // row r = tid / 16 (16 threads per row), elements j .. j+3:
                    // component r & 1 of pair r / 2
                    const int r = tid >> 4, j = 4 * ((tid & 15) + 16 * (3 * h + u));
                    float* zr = reinterpret_cast<float*>(zs + (r >> 1) * LDZ) + (r & 1);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int m = (MODE == DCT_INV) ? j + c : reorder_pos<N>(j + c);
                        zr[2 * padix(m)] = vv[c];
                    }
                } else {
                    // element j of lines 4q .. 4q+3: pairs 2q and 2q + 1
                    const int q = e & 7, j = e >> 3;
                    const int m = (MODE == DCT_INV) ? j : reorder_pos<N>(j);
                    zs[(2 * q) * LDZ + padix(m)] = make_float2(v.x, v.y);
                    zs[(2 * q + 1) * LDZ + padix(m)] = make_float2(v.z, v.w);
                }
            }
        }
        __syncthreads();
        if (MODE != DCT_INV) {
            fft384<-1>(z, lane, a.ptw);
            for (int k = lane; k <= N / 2; k += 32) {
                const int km = (k == 0) ? 0 : N - k;
                const C Zk = z[padix(k)], Zm = z[padix(km)];
                C A, Bq;
                A.x = 0.5f * (Zk.x + Zm.x); A.y = 0.5f * (Zk.y - Zm.y);
                Bq.x = 0.5f * (Zk.y + Zm.y); Bq.y = 0.5f * (Zm.x - Zk.x);
                const C dk = a.dtw[k];
                C outk; outk.x = dk.x * A.x - dk.y * A.y; outk.y = dk.x * Bq.x - dk.y * Bq.y;
                if (km != k) {
                    C Am, Bm;
                    Am.x = 0.5f * (Zm.x + Zk.x); Am.y = 0.5f * (Zm.y - Zk.y);
                    Bm.x = 0.5f * (Zm.y + Zk.y); Bm.y = 0.5f * (Zk.x - Zm.x);
                    const C dm = a.dtw[km];
                    C outm; outm.x = dm.x * Am.x - dm.y * Am.y; outm.y = dm.x * Bm.x - dm.y * Bm.y;
                    z[padix(km)] = outm;
                }
                z[padix(k)] = outk;
            }
            __syncwarp();
        }
        if (MODE == DCT_MID) {
            // eigenvalue of the pair's lines along the other axes (Parseval weights 1 or 2)
            const int ia = (CONTIG ? (int)tl.outer : tl.i0) + 2 * pw, ib = ia + 1;
            float La = a.lam_a0[ia], Lb = a.lam_a0[ib];
            float wa = (ia == 0) ? 1.f : 2.f, wb = 2.f;
            if (a.lam_a1) {
                const int jo = (int)tl.outer;
                La += a.lam_a1[jo]; Lb += a.lam_a1[jo];
                const float wo = (jo == 0) ? 1.f : 2.f;
                wa *= wo; wb *= wo;
            }
            for (int k = lane; k < N; k += 32) {
                const float lk = a.lam_axis[k];
                const float wk = (k == 0) ? 1.f : 2.f;
                C v = z[padix(k)];
                const float la = La + lk, lb = Lb + lk;
                float ga = 0.f, gb = 0.f, gp = 0.f;      // G's two (positive) terms in FP32
                if (la > 0.f) { ga = __fdividef(v.x, la); gp = (wa * wk * v.x) * ga; }
                if (lb > 0.f) { gb = __fdividef(v.y, lb); gp = fmaf(wb * wk * v.y, gb, gp); }
                gsum.add(gp);
                v.x = ga; v.y = gb;
                z[padix(k)] = v;
            }
            acc += gsum.take();
            __syncwarp();
        }
        if (MODE != DCT_FWD) {
            for (int k = lane; k <= N / 2; k += 32) {
                const int km = (k == 0) ? 0 : N - k;
                const C Xk = z[padix(k)], Xm = z[padix(km)];
                const float xam = (k == 0) ? 0.f : Xm.x, xbm = (k == 0) ? 0.f : Xm.y;
                const C dk = cconj(a.dtw[k]);
                C Va, Vb;
                Va.x = dk.x * Xk.x + dk.y * xam; Va.y = dk.y * Xk.x - dk.x * xam;
                Vb.x = dk.x * Xk.y + dk.y * xbm; Vb.y = dk.y * Xk.y - dk.x * xbm;
                C Zk; Zk.x = Va.x - Vb.y; Zk.y = Va.y + Vb.x;
                if (km != k) {
                    const C dm = cconj(a.dtw[km]);
                    C Wa, Wb;
                    Wa.x = dm.x * Xm.x + dm.y * Xk.x; Wa.y = dm.y * Xm.x - dm.x * Xk.x;
                    Wb.x = dm.x * Xm.y + dm.y * Xk.y; Wb.y = dm.y * Xm.y - dm.x * Xk.y;
                    C Zm; Zm.x = Wa.x - Wb.y; Zm.y = Wa.y + Wb.x;
                    z[padix(km)] = Zm;
                }
                z[padix(k)] = Zk;
            }
            __syncwarp();
            fft384<+1>(z, lane, a.ptw);
        }
        __syncthreads();
        // ---- store (the potential update reads its values first) ---------------------
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 up[3];
            if (MODE == DCT_INV && a.upd) {
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int e = tid + 512 * (3 * h + u);
                    long long ad;
                    if (CONTIG) ad = tl.base0 + (long long)(tid >> 4) * N + 4 * ((tid & 15) + 16 * (3 * h + u));
                    else ad = tl.base0 + 4 * (e & 7) + (long long)(e >> 3) * lt.es;
                    up[u] = *reinterpret_cast<const float4*>(a.upd + ad);
                }
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int e = tid + 512 * (3 * h + u);
                long long ad;
                float4 v;
                if (CONTIG) {
                    const int r = tid >> 4, j = 4 * ((tid & 15) + 16 * (3 * h + u));
                    ad = tl.base0 + (long long)r * N + j;
                    const float* zr = reinterpret_cast<const float*>(zs + (r >> 1) * LDZ) + (r & 1);
                    float vv[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int m = (MODE == DCT_FWD) ? j + c : reorder_pos<N>(j + c);
                        vv[c] = zr[2 * padix(m)];
                    }
                    v = make_float4(vv[0], vv[1], vv[2], vv[3]);
                } else {
                    const int q = e & 7, j = e >> 3;
                    ad = tl.base0 + 4 * q + (long long)j * lt.es;
                    const int m = (MODE == DCT_FWD) ? j : reorder_pos<N>(j);
                    const C p0 = zs[(2 * q) * LDZ + padix(m)], p1 = zs[(2 * q + 1) * LDZ + padix(m)];
                    v = make_float4(p0.x, p0.y, p1.x, p1.y);
                }
                if (MODE != DCT_FWD) { v.x *= inv_n; v.y *= inv_n; v.z *= inv_n; v.w *= inv_n; }
                if (MODE == DCT_INV && a.upd) {
                    v.x = up[u].x + sig * v.x; v.y = up[u].y + sig * v.y;
                    v.z = up[u].z + sig * v.z; v.w = up[u].w + sig * v.w;
                }
                *reinterpret_cast<float4*>(a.out + ad) = v;
            }
        }
        __syncthreads();
    }
    if (MODE == DCT_MID && a.part) {
        const double sacc = block_sum(acc, red);
        if (threadIdx.x == 0) a.part[blockIdx.x] = sacc * a.gscale;
    }
}

// ---------------------------------------------------------------------------
// tables: twiddles, digit reversal and eigenvalues (computed on the device in FP64)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fill_tables_kernel(int n, cx_t<T>* tw, cx_t<T>* dtw, unsigned short* drev,
                                   T* lam, int nst, FftRadices rs)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s, c;
    sincospi(-2.0 * (double)j / (double)n, &s, &c);
    tw[j].x = (T)c; tw[j].y = (T)s;
    sincospi(-(double)j / (2.0 * (double)n), &s, &c);
    dtw[j].x = (T)c; dtw[j].y = (T)s;
    const double sh = sinpi((double)j / (2.0 * (double)n));
    lam[j] = (T)(4.0 * (double)n * (double)n * sh * sh);
    // digit reversal: element m -> position p (DIT with radices rs.r[0..nst))
    int m = j, p = 0, Lw[kMaxStages];
    int L = 1;
    for (int l = 0; l < nst; ++l) { Lw[l] = L; L *= rs.r[l]; }
    for (int l = nst - 1; l >= 0; --l) {
        const int q = m % rs.r[l];
        m /= rs.r[l];
        p += q * Lw[l];
    }
    drev[j] = (unsigned short)p;
}

bool fft_radices(int n, FftRadices* rs)
{
    int m = n, k = 0;
    int twos = 0, fours = 0, threes = 0;
    while (m % 4 == 0) { ++fours; m /= 4; }
    while (m % 2 == 0) { ++twos; m /= 2; }
    while (m % 3 == 0) { ++threes; m /= 3; }
    if (m != 1) return false;
    if (twos + fours + threes > kMaxStages) return false;
    for (int i = 0; i < twos; ++i) rs->r[k++] = 2;
    for (int i = 0; i < threes; ++i) rs->r[k++] = 3;
    for (int i = 0; i < fours; ++i) rs->r[k++] = 4;
    rs->nst = k;
    return true;
}

static bool fast_radices(int n, int* nst, int* rad);

// Radices of the 384-point register FFT (dct384_kernel): 4 x 4 x 4 x 6
static bool radices_384(int n, int* nst, int* rad)
{
    if (n != 384) return false;
    rad[0] = rad[1] = rad[2] = 4;
    rad[3] = 6;
    *nst = 4;
    return true;
}

// FP32 power-of-two lines from 32 cells and FP32 lines of 384 run a register
// FFT and carry its pass twiddle table
static bool has_pass_table(int n, int elem_bytes)
{
    int nst, rad[8];
    return elem_bytes == 4 && (fast_radices(n, &nst, rad) || radices_384(n, &nst, rad));
}

size_t axis_table_bytes(int n, int elem_bytes)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up((size_t)n * 2 * elem_bytes) * 2 + up((size_t)n * 2) + up((size_t)n * 8) +
           (has_pass_table(n, elem_bytes) ? up((size_t)n * 8) : 0);
}

bool layout_axis_tables(int n, int elem_bytes, unsigned char* ws, AxisTables* t)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    FftRadices rs;
    if (!fft_radices(n, &rs)) return false;
    const size_t cb = up((size_t)n * 2 * elem_bytes);
    t->n = n;
    t->rs = rs;
    t->tw = ws;
    t->dtw = ws + cb;
    t->drev = reinterpret_cast<unsigned short*>(ws + 2 * cb);
    t->lam = ws + 2 * cb + up((size_t)n * 2);
    t->ptw = has_pass_table(n, elem_bytes) ? ws + 2 * cb + up((size_t)n * 2) + up((size_t)n * 8)
                                           : nullptr;
    return true;
}

// Pass twiddles of the register FFT: the pass of radix R and stride Ns (the
// product of the earlier radices) takes e^{-2 pi i k r/(Ns R)} for k < Ns,
// 0 < r < R; its block starts at Ns - 1 (the blocks before it hold
// sum (R' - 1) Ns' = Ns - 1 entries), so all passes fill n - 1 entries.
struct PassRadices { int nst; int rad[8]; };

__global__ void fill_pass_table_kernel(int n, float2* ptw, PassRadices pr)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n - 1) return;
    int Ns = 1, R = pr.rad[0];
    for (int s = 0; s < pr.nst; ++s) {
        R = pr.rad[s];
        if (j < Ns * R - 1) break;                 // j in [Ns - 1, Ns R - 1)
        Ns *= R;
    }
    const int local = j - (Ns - 1);
    const int r = local / Ns + 1, k = local % Ns;
    double s, c;
    sincospi(-2.0 * (double)k * (double)r / ((double)Ns * (double)R), &s, &c);
    ptw[j].x = (float)c;
    ptw[j].y = (float)s;
}

template <typename T>
bfm_status fill_axis_tables(int n, AxisTables* t, unsigned char* ws, cudaStream_t st)
{
    if (!layout_axis_tables(n, (int)sizeof(T), ws, t)) return BFM_ERR_UNSUPPORTED;
    fill_tables_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(
        n, reinterpret_cast<cx_t<T>*>(t->tw), reinterpret_cast<cx_t<T>*>(t->dtw), t->drev,
        reinterpret_cast<T*>(t->lam), t->rs.nst, t->rs);
    BFM_LAUNCH_CHECK("fill_tables_kernel");
    if (t->ptw) {
        PassRadices pr;
        if (!fast_radices(n, &pr.nst, pr.rad)) radices_384(n, &pr.nst, pr.rad);
        fill_pass_table_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, reinterpret_cast<float2*>(t->ptw), pr);
        BFM_LAUNCH_CHECK("fill_pass_table_kernel");
    }
    return BFM_OK;
}

template bfm_status fill_axis_tables<float>(int, AxisTables*, unsigned char*, cudaStream_t);
template bfm_status fill_axis_tables<double>(int, AxisTables*, unsigned char*, cudaStream_t);

// ---------------------------------------------------------------------------
// launch planning
// ---------------------------------------------------------------------------
static bool fast_radices(int n, int* nst, int* rad)
{
    if (n < 32 || (n & (n - 1))) return false;
    int k = 0;
    while ((1 << k) < n) ++k;
    int c = 0;
    for (int i = 0; i < k / 4; ++i) rad[c++] = 16;
    if (k % 4) rad[c++] = 1 << (k % 4);
    *nst = c;
    return c <= 8;
}

DctPlan plan_dct_pass(const Grid& g, int axis, int elem_bytes)
{
    DctPlan p;
    const int n = g.n[axis];
    const bool contig = (axis == 0);
    int fr[8], fn = 0;
    p.fast = (elem_bytes == 4 && fast_radices(n, &fn, fr)) ? 1 : 0;
    int G, max_threads;
    if (p.fast) {
        G = n / 16;                                   // 16 complex values per thread per pass
        // up to 128 registers per thread: one line pair per CTA and two CTAs
        // per SM, so one CTA's loads and stores overlap the other's FFT
        max_threads = 256;
        p.LDZ = n + n / 16 + 1;                       // one pad element per 16
    } else {
        G = n / 8;
        if (G < 8) G = 8;
        if (G > 256) G = 256;
        G = (G + 7) & ~7;
        max_threads = elem_bytes == 8 ? 512 : 1024;   // FP64 gets 128 registers
        p.LDZ = n + 1;
    }
    p.G = G;
    const size_t pair_bytes = (size_t)p.LDZ * 2 * elem_bytes;
    const size_t budget = 200 * 1024;
    int W = 2 * (max_threads / G);
    while (W > 2 && (size_t)(W / 2) * pair_bytes > budget) W -= 2;
    if (W > 32) W = 32;
    if (!contig) {
        if (W > g.n[0]) W = g.n[0];
        int p2 = 1;                       // power of two: division-free index math
        while (p2 * 2 <= W) p2 *= 2;
        W = p2;
    }
    if (W < 1) W = 1;
    p.W = W;
    const int npairs = (W + 1) / 2;
    p.threads = ((npairs * G + 31) / 32) * 32;      // whole warps; extra threads idle
    p.smem = (size_t)npairs * pair_bytes;
    p.tiles = make_tiles(g, axis, W);
    return p;
}

template <typename T, int MODE>
static void* dct_kernel(bool contig, bool batched)
{
    if (batched)
        return contig ? (void*)dct_pass_kernel<T, MODE, true, true> : (void*)dct_pass_kernel<T, MODE, false, true>;
    return contig ? (void*)dct_pass_kernel<T, MODE, true, false> : (void*)dct_pass_kernel<T, MODE, false, false>;
}

template <typename T>
static bfm_status make_dct_args(const Grid& g, int axis, const DctPlan& p, const AxisTables* tabs,
                                const T* in, const T* base, T* out, const T* upd,
                                const double* sigma, double* part, const int* done, DctArgs<T>* a)
{
    const AxisTables& tb = tabs[axis];
    // host-side guard: never launch with tables that do not describe this axis
    // a MID pass along rows (2-D, axis 0) takes the line eigenvalues of axis 1
    const int line_axis = (axis == 0) ? 1 : 0;
    if (tb.n != g.n[axis] || !tb.tw || !tb.dtw || !tb.drev || !tb.lam || tb.rs.nst < 1 ||
        (g.ndim == 2 && !tabs[line_axis].lam) || (g.ndim == 3 && (!tabs[0].lam || !tabs[1].lam))) {
        set_last_error("internal: DCT tables do not match the grid");
        return BFM_ERR_INVALID_ARG;
    }
    a->in = in; a->base = base; a->out = out; a->upd = upd; a->sigma = sigma; a->part = part;
    a->done = done;
    a->tw = reinterpret_cast<const cx_t<T>*>(tb.tw);
    a->ptw = reinterpret_cast<const float2*>(tb.ptw);
    if (p.fast && !tb.ptw) {
        set_last_error("internal: DCT pass twiddle table missing");
        return BFM_ERR_INVALID_ARG;
    }
    a->dtw = reinterpret_cast<const cx_t<T>*>(tb.dtw);
    a->drev = tb.drev;
    a->lam_axis = reinterpret_cast<const T*>(tb.lam);
    a->lam_a0 = reinterpret_cast<const T*>(g.ndim == 2 ? tabs[line_axis].lam : tabs[0].lam);
    a->lam_a1 = (g.ndim == 3) ? reinterpret_cast<const T*>(tabs[1].lam) : nullptr;
    a->lt = p.tiles;
    a->G = p.G;
    a->LDZ = p.LDZ;
    a->nst = tb.rs.nst;
    int L = 1;
    for (int i = 0; i < kMaxStages; ++i) {
        a->rad[i] = (i < tb.rs.nst) ? tb.rs.r[i] : 0;
        a->Ls[i] = L;
        a->mag[i] = (L > 1) ? (unsigned)((((unsigned long long)1 << 32) + L - 1) / L) : 0u;
        if (i < tb.rs.nst) L *= tb.rs.r[i];
    }
    const int npt = (p.W + 1) / 2;
    a->lnp = 0;
    while ((1 << a->lnp) < npt) ++a->lnp;
    a->gscale = 1.0 / ((double)g.N * (double)g.N);
    a->fnst = 0;
    for (int i = 0; i < 8; ++i) a->frad[i] = 0;
    if (p.fast) fast_radices(g.n[axis], &a->fnst, a->frad);
    return BFM_OK;
}

template <int MODE>
static void* dct_fast(bool contig, bool batched)
{
    if (batched)
        return contig ? (void*)dct_fast_kernel<MODE, true, true> : (void*)dct_fast_kernel<MODE, false, true>;
    return contig ? (void*)dct_fast_kernel<MODE, true, false> : (void*)dct_fast_kernel<MODE, false, false>;
}

static void* select_dct(int mode, int elem_bytes, bool contig, bool batched, bool fast)
{
    if (fast) {
        if (mode == DCT_FWD) return dct_fast<DCT_FWD>(contig, batched);
        if (mode == DCT_MID) return dct_fast<DCT_MID>(contig, batched);
        return dct_fast<DCT_INV>(contig, batched);
    }
    if (elem_bytes == 4) {
        if (mode == DCT_FWD) return dct_kernel<float, DCT_FWD>(contig, batched);
        if (mode == DCT_MID) return dct_kernel<float, DCT_MID>(contig, batched);
        return dct_kernel<float, DCT_INV>(contig, batched);
    }
    if (mode == DCT_FWD) return dct_kernel<double, DCT_FWD>(contig, batched);
    if (mode == DCT_MID) return dct_kernel<double, DCT_MID>(contig, batched);
    return dct_kernel<double, DCT_INV>(contig, batched);
}

template <int LOGN, bool BATCHED>
static void* dct_row_of(int mode)
{
    return mode == DCT_FWD ? (void*)dct_row_kernel<DCT_FWD, LOGN, BATCHED>
         : mode == DCT_MID ? (void*)dct_row_kernel<DCT_MID, LOGN, BATCHED>
                           : (void*)dct_row_kernel<DCT_INV, LOGN, BATCHED>;
}

// The compile-time row kernel for FP32 rows of 512-4096 cells whose fields
// are 16-byte aligned (float4 rows); the middle pass only on 2-D grids (its
// eigenvalue of the line comes from the one other axis).  NULL: the general
// kernel handles the pass.
static void* select_dct_row(int mode, int n, int ndim, bool batched)
{
    if (mode == DCT_MID && ndim != 2) return nullptr;
    if (n == 4096) return batched ? dct_row_of<12, true>(mode) : dct_row_of<12, false>(mode);
    if (n == 2048) return batched ? dct_row_of<11, true>(mode) : dct_row_of<11, false>(mode);
    if (n == 1024) return batched ? dct_row_of<10, true>(mode) : dct_row_of<10, false>(mode);
    if (n == 512) return batched ? dct_row_of<9, true>(mode) : dct_row_of<9, false>(mode);
    return nullptr;
}

static bool rows_aligned16(const void* in, const void* base, const void* out, const void* upd)
{
    auto al = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    return al(in) && al(base) && al(out) && al(upd);
}

static int dct_blocks(const DctPlan& p)
{
    long long blocks = p.tiles.ntiles;
    const long long cap = (long long)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    if (blocks > kMaxPartials) blocks = kMaxPartials;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <typename T>
bfm_status launch_dct_pass(const Grid& g, int axis, int mode, const AxisTables* tabs,
                           const T* in, const T* base, T* out, const T* upd,
                           const double* sigma, double* part, const int* done,
                           cudaStream_t st, int* blocks_used)
{
    DctPlan p = plan_dct_pass(g, axis, (int)sizeof(T));
    DctArgs<T> a;
    bfm_status s = make_dct_args<T>(g, axis, p, tabs, in, base, out, upd, sigma, part, done, &a);
    if (s != BFM_OK) return s;
    if (sizeof(T) == 4 && g.n[axis] == 384 && tabs[axis].ptw) {
        // tiles of 32 whole lines, float4 on both sides
        auto al = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
        const bool full = axis == 0 ? (g.N / 384) % 32 == 0 : g.n[0] % 32 == 0;
        if (full && al(in) && al(base) && al(out) && al(upd)) {
            a.lt = make_tiles(g, axis, 32);
            void* k384 = axis == 0
                ? (mode == DCT_FWD ? (void*)dct384_kernel<DCT_FWD, true>
                   : mode == DCT_MID ? (void*)dct384_kernel<DCT_MID, true> : (void*)dct384_kernel<DCT_INV, true>)
                : (mode == DCT_FWD ? (void*)dct384_kernel<DCT_FWD, false>
                   : mode == DCT_MID ? (void*)dct384_kernel<DCT_MID, false> : (void*)dct384_kernel<DCT_INV, false>);
            const size_t smem = (size_t)16 * (384 + 384 / 16 + 1) * sizeof(float2);
            BFM_CUDA(cudaFuncSetAttribute(k384, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int per_sm = 0;
            BFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k384, 512, smem));
            long long blocks = a.lt.ntiles;
            const long long cap = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
            if (blocks > cap) blocks = cap;
            if (blocks > kMaxPartials) blocks = kMaxPartials;
            if (blocks < 1) blocks = 1;
            void* args[] = {&a};
            BFM_CUDA(cudaLaunchKernel(k384, dim3((unsigned)blocks), dim3(512), args, smem, st));
            if (blocks_used) *blocks_used = (int)blocks;
            return BFM_OK;
        }
    }
    if (sizeof(T) == 4 && axis == 0 && p.fast && rows_aligned16(in, base, out, upd)) {
        void* rk = select_dct_row(mode, g.n[0], g.ndim, false);
        if (rk) {
            // one line pair per CTA of n/16 threads, one resident wave
            const int threads = g.n[0] / 16;
            const size_t smem = (size_t)p.LDZ * sizeof(float2);
            BFM_CUDA(cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int per_sm = 0;
            BFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rk, threads, smem));
            long long blocks = (p.tiles.nlines + 1) / 2;
            const long long cap = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
            if (blocks > cap) blocks = cap;
            if (blocks > kMaxPartials) blocks = kMaxPartials;
            if (blocks < 1) blocks = 1;
            const DctArgs<T>* none = nullptr;
            void* args[] = {&a, &none};
            BFM_CUDA(cudaLaunchKernel(rk, dim3((unsigned)blocks), dim3(threads), args, smem, st));
            if (blocks_used) *blocks_used = (int)blocks;
            return BFM_OK;
        }
    }
    void* k = select_dct(mode, (int)sizeof(T), axis == 0, false, p.fast != 0);
    BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    int blocks = dct_blocks(p);
    // one wave of resident CTAs, each looping over tiles: a second wave would
    // start only when first-wave CTAs finish all their tiles
    int per_sm = 0;
    BFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, p.threads, p.smem));
    if (per_sm > 0 && blocks > num_sms() * per_sm) blocks = num_sms() * per_sm;
    const DctArgs<T>* none = nullptr;
    void* args[] = {&a, &none};
    BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(p.threads), args, p.smem, st));
    if (blocks_used) *blocks_used = blocks;
    return BFM_OK;
}

template <typename T>
int dct_batch_blocks(const Grid& g, int axis) { return dct_blocks(plan_dct_pass(g, axis, (int)sizeof(T))); }

size_t dct_args_bytes(int elem_bytes) { return elem_bytes == 8 ? sizeof(DctArgs<double>) : sizeof(DctArgs<float>); }

template <typename T>
bfm_status fill_dct_batch_args(const Grid& g, int axis, const AxisTables* tabs, const T* in,
                               const T* base, T* out, const T* upd, const double* sigma,
                               double* part, const int* done, void* host_slot)
{
    DctPlan p = plan_dct_pass(g, axis, (int)sizeof(T));
    return make_dct_args<T>(g, axis, p, tabs, in, base, out, upd, sigma, part, done,
                            reinterpret_cast<DctArgs<T>*>(host_slot));
}

template <typename T>
bfm_status launch_dct_pass_batched(const Grid& g, int axis, int mode, int nprob,
                                   const void* dev_args, cudaStream_t st, bool rows16)
{
    DctPlan p = plan_dct_pass(g, axis, (int)sizeof(T));
    if (sizeof(T) == 4 && axis == 0 && p.fast && rows16) {
        void* rk = select_dct_row(mode, g.n[0], g.ndim, true);
        if (rk) {
            const int threads = g.n[0] / 16;
            const size_t smem = (size_t)p.LDZ * sizeof(float2);
            BFM_CUDA(cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int per_sm = 0;
            BFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rk, threads, smem));
            long long blocks = (p.tiles.nlines + 1) / 2;
            const long long cap = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
            if (blocks > cap) blocks = cap;
            if (blocks < 1) blocks = 1;
            DctArgs<float> dummy;
            memset(&dummy, 0, sizeof(dummy));
            const DctArgs<float>* batch = reinterpret_cast<const DctArgs<float>*>(dev_args);
            void* args[] = {&dummy, &batch};
            BFM_CUDA(cudaLaunchKernel(rk, dim3((unsigned)blocks, (unsigned)nprob), dim3(threads), args,
                                      smem, st));
            return BFM_OK;
        }
    }
    void* k = select_dct(mode, (int)sizeof(T), axis == 0, true, p.fast != 0);
    BFM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int blocks = dct_blocks(p);
    DctArgs<T> dummy;
    memset(&dummy, 0, sizeof(dummy));
    const DctArgs<T>* batch = reinterpret_cast<const DctArgs<T>*>(dev_args);
    void* args[] = {&dummy, &batch};
    BFM_CUDA(cudaLaunchKernel(k, dim3((unsigned)blocks, (unsigned)nprob), dim3(p.threads), args,
                              p.smem, st));
    return BFM_OK;
}

template int dct_batch_blocks<float>(const Grid&, int);
template int dct_batch_blocks<double>(const Grid&, int);
template bfm_status fill_dct_batch_args<float>(const Grid&, int, const AxisTables*, const float*,
                                               const float*, float*, const float*, const double*,
                                               double*, const int*, void*);
template bfm_status fill_dct_batch_args<double>(const Grid&, int, const AxisTables*, const double*,
                                                const double*, double*, const double*,
                                                const double*, double*, const int*, void*);
template bfm_status launch_dct_pass_batched<float>(const Grid&, int, int, int, const void*, cudaStream_t,
                                                   bool);
template bfm_status launch_dct_pass_batched<double>(const Grid&, int, int, int, const void*, cudaStream_t,
                                                    bool);
template bfm_status launch_dct_pass<float>(const Grid&, int, int, const AxisTables*, const float*,
                                           const float*, float*, const float*, const double*,
                                           double*, const int*, cudaStream_t, int*);
template bfm_status launch_dct_pass<double>(const Grid&, int, int, const AxisTables*,
                                            const double*, const double*, double*,
                                            const double*, const double*, double*, const int*,
                                            cudaStream_t, int*);

}  // namespace bfm
