/*
 * bfm_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, FP64 CPU restatement of the back-and-forth method (BFM) of
 * Jacobs & Leger, "A fast approach to optimal transport: the back-and-forth
 * method" (arXiv 1905.12154), used only to check the CUDA library.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline / reference arm
 * load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Each function cites the passage of the paper it follows.  Where the paper
 * is silent the reading taken is stated at the function:
 *   - Omega = [0,1]^d (Section 4.3), discretised by a cell-centred grid with
 *     n_a cells on axis a, spacing h_a = 1/n_a, centres x = (i + 1/2) h_a.
 *     Axis 0 varies fastest in memory: idx = (k*n1 + j)*n0 + i.
 *   - densities are stored as values with unit integral: hd * sum(mu) = 1,
 *     hd = prod_a h_a, so the uniform density is 1.
 *   - cost c(x,y) = |x-y|^2/2 (Section 4.3, quadratic cost); the transport
 *     cost C(mu,nu) is half the squared Wasserstein distance: W2^2 = 2 C.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared.  Floating point
 * contraction is off so every product and sum rounds as written.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int ndim;
    int n[3];     /* cells per axis, axis 0 fastest */
    long N;       /* total cells */
    long stride[3];
    double h[3];  /* spacing per axis */
    double hd;    /* cell volume */
} grid_t;

static int make_grid(int ndim, const int *n, grid_t *g)
{
    if (ndim < 1 || ndim > 3) return -1;
    g->ndim = ndim;
    g->N = 1;
    g->hd = 1.0;
    for (int a = 0; a < 3; a++) {
        g->n[a] = (a < ndim) ? n[a] : 1;
        if (g->n[a] < 1) return -1;
        g->stride[a] = g->N;
        g->N *= g->n[a];
        g->h[a] = 1.0 / g->n[a];
        if (a < ndim) g->hd *= g->h[a];
    }
    return 0;
}

/* number of lines along axis a, and the base index of line L */
static long n_lines(const grid_t *g, int a) { return g->N / g->n[a]; }

static long line_base(const grid_t *g, int a, long L)
{
    /* enumerate the other axes in memory order */
    long base = 0, rem = L;
    for (int b = 0; b < 3; b++) {
        if (b == a) continue;
        long c = rem % g->n[b];
        rem /= g->n[b];
        base += c * g->stride[b];
    }
    return base;
}

int bfm_oracle_omp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* c-transform (Definition 2.1; Section 4.1)                                 */
/* ------------------------------------------------------------------------ */

/*
 * One 1-D pass by brute force (Definition 2.1 restricted to a grid line):
 *     u(x_i) = min_j  (x_i - y_j)^2 / 2 + f(y_j)
 * over the grid points y_j of the line (reading: the discrete c-transform is
 * a minimum over grid points only).  O(n^2) per line.
 */
static void line_brute(const double *f, double *u, int n, double h)
{
    for (int i = 0; i < n; i++) {
        double x = (i + 0.5) * h;
        double best = INFINITY;
        for (int j = 0; j < n; j++) {
            double y = (j + 0.5) * h;
            double d = x - y;
            double v = 0.5 * d * d + f[j];
            if (v < best) best = v;
        }
        u[i] = best;
    }
}

/*
 * One 1-D pass through the Legendre transform (Section 4.1, eq. (legendre)):
 *     u(x) = x^2/2 - vp*(x),   vp(y) = y^2/2 + f(y),
 *     vp*(x) = sup_y x*y - vp(y).
 * vp* equals the transform of the lower convex hull of the points
 * (y_j, vp(y_j)); the hull is built in one left-to-right pass and the
 * maximiser for increasing x is found by one monotone sweep over the hull's
 * increasing slopes (Lucet's linear-time Legendre transform, as described
 * in Section 4.1).  O(n) per line.
 */
static void line_llt(const double *f, double *u, int n, double h, int *hull, double *vp)
{
    for (int j = 0; j < n; j++) {
        double y = (j + 0.5) * h;
        vp[j] = 0.5 * y * y + f[j];
    }
    /* lower convex hull of (y_j, vp_j), points already sorted by y */
    int H = 0;
    for (int j = 0; j < n; j++) {
        while (H >= 2) {
            int a = hull[H - 2], b = hull[H - 1];
            double ya = (a + 0.5) * h, yb = (b + 0.5) * h, yj = (j + 0.5) * h;
            /* b is kept only if it lies strictly below the chord a -> j */
            double cross = (yb - ya) * (vp[j] - vp[a]) - (yj - ya) * (vp[b] - vp[a]);
            if (cross <= 0.0) H--; else break;
        }
        hull[H++] = j;
    }
    /* sweep: slopes of consecutive hull edges increase */
    int k = 0;
    for (int i = 0; i < n; i++) {
        double x = (i + 0.5) * h;
        while (k + 1 < H) {
            int a = hull[k], b = hull[k + 1];
            double slope = (vp[b] - vp[a]) / (((b + 0.5) * h) - ((a + 0.5) * h));
            if (slope < x) k++; else break;
        }
        double yk = (hull[k] + 0.5) * h;
        double conj = x * yk - vp[hull[k]];
        u[i] = 0.5 * x * x - conj;
    }
}

/*
 * phi^c on the whole grid by dimension splitting (Section 4.1):
 *   phi^c(x) = min_{y_d} ... min_{y_1} sum_a (x_a-y_a)^2/2 - phi(y),
 * i.e. a 1-D pass along axis 0 applied to f = -phi, then 1-D passes along the
 * remaining axes applied to the previous pass's output.
 * mode 0: brute-force lines, mode 1: linear-time Legendre lines.
 */
int bfm_oracle_ctransform(const double *phi, double *out, int ndim, const int *n, int mode)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    double *cur = (double *)malloc(sizeof(double) * g.N);
    if (!cur) return -2;
    for (long i = 0; i < g.N; i++) cur[i] = -phi[i];
    for (int a = 0; a < ndim; a++) {
        int na = g.n[a];
        long L = n_lines(&g, a);
        long s = g.stride[a];
        #pragma omp parallel
        {
            double *fin = (double *)malloc(sizeof(double) * na);
            double *fo = (double *)malloc(sizeof(double) * na);
            double *vp = (double *)malloc(sizeof(double) * na);
            int *hull = (int *)malloc(sizeof(int) * na);
            #pragma omp for schedule(static)
            for (long l = 0; l < L; l++) {
                long b = line_base(&g, a, l);
                for (int i = 0; i < na; i++) fin[i] = cur[b + i * s];
                if (mode == 0) line_brute(fin, fo, na, g.h[a]);
                else line_llt(fin, fo, na, g.h[a], hull, vp);
                for (int i = 0; i < na; i++) cur[b + i * s] = fo[i];
            }
            free(fin); free(fo); free(vp); free(hull);
        }
    }
    memcpy(out, cur, sizeof(double) * g.N);
    free(cur);
    return 0;
}

/*
 * Separable power costs (Section 5, eq. p_costs): c(x,y) = sum_a h_a(y_a - x_a)
 * with h_a(z) = |z|^{p_a} / p_a, p_a > 1.  The c-transform splits along the
 * axes exactly as for the quadratic cost (Section 4.1, dimension splitting);
 * each 1-D pass is the minimum over the grid points of the line, O(n^2).
 */
static double hpow(double z, double p) { return pow(fabs(z), p) / p; }

static void line_brute_p(const double *f, double *u, int n, double h, double p)
{
    for (int i = 0; i < n; i++) {
        double x = (i + 0.5) * h;
        double best = INFINITY;
        for (int j = 0; j < n; j++) {
            double v = hpow((j + 0.5) * h - x, p) + f[j];
            if (v < best) best = v;
        }
        u[i] = best;
    }
}

int bfm_oracle_ctransform_p(const double *phi, double *out, int ndim, const int *n, const double *p)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    double *cur = (double *)malloc(sizeof(double) * g.N);
    if (!cur) return -2;
    for (long i = 0; i < g.N; i++) cur[i] = -phi[i];
    for (int a = 0; a < ndim; a++) {
        int na = g.n[a];
        long L = n_lines(&g, a);
        long s = g.stride[a];
        #pragma omp parallel
        {
            double *fin = (double *)malloc(sizeof(double) * na);
            double *fo = (double *)malloc(sizeof(double) * na);
            #pragma omp for schedule(static)
            for (long l = 0; l < L; l++) {
                long b = line_base(&g, a, l);
                for (int i = 0; i < na; i++) fin[i] = cur[b + i * s];
                line_brute_p(fin, fo, na, g.h[a], p[a]);
                for (int i = 0; i < na; i++) cur[b + i * s] = fo[i];
            }
            free(fin); free(fo);
        }
    }
    memcpy(out, cur, sizeof(double) * g.N);
    free(cur);
    return 0;
}

/*
 * phi^c by the definition with no splitting (Definition 2.1): the minimum
 * over every grid point y of |x-y|^2/2 - phi(y).  O(N^2); tiny grids only.
 */
int bfm_oracle_ctransform_full(const double *phi, double *out, int ndim, const int *n)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    #pragma omp parallel for schedule(static)
    for (long p = 0; p < g.N; p++) {
        double x[3];
        long r = p;
        for (int a = 0; a < 3; a++) { x[a] = ((r % g.n[a]) + 0.5) * g.h[a]; r /= g.n[a]; }
        double best = INFINITY;
        for (long q = 0; q < g.N; q++) {
            long s = q;
            double c = 0.0;
            for (int a = 0; a < g.ndim; a++) {
                double y = ((s % g.n[a]) + 0.5) * g.h[a];
                s /= g.n[a];
                double d = x[a] - y;
                c += 0.5 * d * d;
            }
            double v = c - phi[q];
            if (v < best) best = v;
        }
        out[p] = best;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* DCT and the Neumann Poisson solve (Lemma 2.3; Section 4.3)                */
/* ------------------------------------------------------------------------ */

/* DCT-II by its definition: X_k = sum_j x_j cos(pi k (j+1/2) / n). */
static void dct2_def(const double *x, double *X, int n)
{
    for (int k = 0; k < n; k++) {
        double s = 0.0;
        for (int j = 0; j < n; j++) s += x[j] * cos(M_PI * k * (j + 0.5) / n);
        X[k] = s;
    }
}

/* Inverse of DCT-II by its definition:
 * x_j = (1/n) [ X_0 + 2 sum_{k>=1} X_k cos(pi k (j+1/2) / n) ]. */
static void dct3_def(const double *X, double *x, int n)
{
    for (int j = 0; j < n; j++) {
        double s = X[0];
        for (int k = 1; k < n; k++) s += 2.0 * X[k] * cos(M_PI * k * (j + 0.5) / n);
        x[j] = s / n;
    }
}

/* Plain recursive discrete Fourier transform, X_k = sum_m x_m e^{-2 pi i sign m k / n}
 * (sign = +1 forward, -1 backward, unnormalised): splits on the smallest prime
 * factor p of n (Cooley-Tukey); a prime length is done by the definition. */
static void dft_rec(const cplx *x, cplx *X, int n, long xs, int sign)
{
    if (n == 1) { X[0] = x[0]; return; }
    int p = 0;
    for (int c = 2; c * c <= n; c++) if (n % c == 0) { p = c; break; }
    if (p == 0) {
        for (int k = 0; k < n; k++) {
            cplx s = 0;
            for (int m = 0; m < n; m++) {
                double ang = -2.0 * M_PI * sign * (double)((long)m * k % n) / n;
                s += x[m * xs] * (cos(ang) + I * sin(ang));
            }
            X[k] = s;
        }
        return;
    }
    int M = n / p;
    cplx *sub = (cplx *)malloc(sizeof(cplx) * n);
    for (int r = 0; r < p; r++) dft_rec(x + r * xs, sub + r * M, M, xs * p, sign);
    for (int k = 0; k < n; k++) {
        cplx s = 0;
        for (int r = 0; r < p; r++) {
            double ang = -2.0 * M_PI * sign * (double)((long)r * k % n) / n;
            s += (cos(ang) + I * sin(ang)) * sub[r * M + (k % M)];
        }
        X[k] = s;
    }
    free(sub);
}

/* DCT-II through one length-n complex FFT (Makhoul's reordering):
 * v = (x_0, x_2, x_4, ..., x_5, x_3, x_1),  X_k = Re(e^{-i pi k/(2n)} V_k). */
static void dct2_fft(const double *x, double *X, int n, cplx *buf, cplx *spec)
{
    int ne = (n + 1) / 2;
    for (int q = 0; q < ne; q++) buf[q] = x[2 * q];
    for (int q = 0; 2 * q + 1 < n; q++) buf[n - 1 - q] = x[2 * q + 1];
    dft_rec(buf, spec, n, 1, +1);
    for (int k = 0; k < n; k++) {
        double ang = -M_PI * k / (2.0 * n);
        X[k] = creal((cos(ang) + I * sin(ang)) * spec[k]);
    }
}

/* Inverse of dct2_fft: W_k = X_k - i X_{n-k} (X_n = 0), V_k = e^{i pi k/(2n)} W_k,
 * v = IDFT(V), then undo the reordering. */
static void dct3_fft(const double *X, double *x, int n, cplx *buf, cplx *spec)
{
    for (int k = 0; k < n; k++) {
        double xr = X[k];
        double xi = (k == 0) ? 0.0 : -X[n - k];
        double ang = M_PI * k / (2.0 * n);
        buf[k] = (cos(ang) + I * sin(ang)) * (xr + I * xi);
    }
    dft_rec(buf, spec, n, 1, -1);
    int ne = (n + 1) / 2;
    for (int q = 0; q < ne; q++) x[2 * q] = creal(spec[q]) / n;
    for (int q = 0; 2 * q + 1 < n; q++) x[2 * q + 1] = creal(spec[n - 1 - q]) / n;
}

/* Apply a 1-D transform along axis a of the field (in place).
 * kind 0: DCT-II, kind 1: inverse DCT-II.  mode 0: definition, 1: FFT. */
int bfm_oracle_dct_axis(double *field, int ndim, const int *n, int axis, int kind, int mode)
{
    grid_t g;
    if (make_grid(ndim, n, &g) || axis < 0 || axis >= ndim) return -1;
    int na = g.n[axis];
    long L = n_lines(&g, axis);
    long s = g.stride[axis];
    #pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * na);
        double *b = (double *)malloc(sizeof(double) * na);
        cplx *c1 = (cplx *)malloc(sizeof(cplx) * na);
        cplx *c2 = (cplx *)malloc(sizeof(cplx) * na);
        #pragma omp for schedule(static)
        for (long l = 0; l < L; l++) {
            long base = line_base(&g, axis, l);
            for (int i = 0; i < na; i++) a[i] = field[base + i * s];
            if (kind == 0) { if (mode == 0) dct2_def(a, b, na); else dct2_fft(a, b, na, c1, c2); }
            else           { if (mode == 0) dct3_def(a, b, na); else dct3_fft(a, b, na, c1, c2); }
            for (int i = 0; i < na; i++) field[base + i * s] = b[i];
        }
        free(a); free(b); free(c1); free(c2);
    }
    return 0;
}

/*
 * Neumann Poisson solve (Lemma 2.3; eq. (gradients_J_I)):
 *     g = (-Delta)^{-1} (f - mean f),  zero Neumann boundary conditions.
 * Reading (the paper says only "using the FFT", Section 4.3): the discrete
 * Laplacian is the 3/5/7-point stencil with reflected ghost cells, whose
 * eigenvectors are the DCT-II cosines with eigenvalues
 *     lambda_k = sum_a 4 n_a^2 sin^2(pi k_a / (2 n_a)),
 * and the zero mode is set to zero (the solution in the mean-zero space H1-dot).
 * Returns G = hd * sum g (f - mean f) = ||g||^2_{H1-dot} = ||f - mean f||^2_{H^-1}
 * (eq. (defHm1dot)), computed in physical space.
 */
int bfm_oracle_poisson(const double *f, double *gout, int ndim, const int *n, int mode, double *G)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    double mean = 0.0;
    for (long i = 0; i < g.N; i++) mean += f[i];
    mean /= (double)g.N;
    double *w = (double *)malloc(sizeof(double) * g.N);
    for (long i = 0; i < g.N; i++) w[i] = f[i] - mean;
    for (int a = 0; a < ndim; a++) bfm_oracle_dct_axis(w, ndim, n, a, 0, mode);
    for (long p = 0; p < g.N; p++) {
        long r = p;
        double lam = 0.0;
        for (int a = 0; a < ndim; a++) {
            long k = r % g.n[a];
            r /= g.n[a];
            double s = sin(M_PI * k / (2.0 * g.n[a]));
            lam += 4.0 * g.n[a] * (double)g.n[a] * s * s;
        }
        w[p] = (p == 0) ? 0.0 : w[p] / lam;
    }
    for (int a = 0; a < ndim; a++) bfm_oracle_dct_axis(w, ndim, n, a, 1, mode);
    double acc = 0.0;
    for (long i = 0; i < g.N; i++) acc += w[i] * (f[i] - mean);
    if (G) *G = g.hd * acc;
    memcpy(gout, w, sizeof(double) * g.N);
    free(w);
    return 0;
}

/* Neumann Laplacian with reflected ghost cells: out = -Delta_h u.
 * Used only to check the Poisson solve. */
int bfm_oracle_neg_laplacian(const double *u, double *out, int ndim, const int *n)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    for (long p = 0; p < g.N; p++) {
        double acc = 0.0;
        long r = p;
        for (int a = 0; a < ndim; a++) {
            long i = r % g.n[a];
            r /= g.n[a];
            long s = g.stride[a];
            double um = (i > 0) ? u[p - s] : u[p];
            double up = (i < g.n[a] - 1) ? u[p + s] : u[p];
            acc += (2.0 * u[p] - um - up) * (double)g.n[a] * g.n[a];
        }
        out[p] = acc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* map and pushforward (Lemma 2.2(ii); Lemma 3.1; pushforward, Section 2.1)  */
/* ------------------------------------------------------------------------ */

/*
 * The map T(x) = x - grad psi(x) of Lemma 2.2(ii) for the quadratic cost
 * ((grad h)^{-1} is the identity), with psi = phi^c.
 * Reading: grad psi by central differences, one-sided at the first and last
 * cell of a line; T is clamped to the box of cell centres [h/2, 1-h/2]^d so
 * that no mass leaves the grid.  out[a*N + p] = T_a(x_p).
 */
int bfm_oracle_map_p(const double *psi, double *out, int ndim, const int *n, const double *pw);

int bfm_oracle_map(const double *psi, double *out, int ndim, const int *n)
{
    return bfm_oracle_map_p(psi, out, ndim, n, NULL);
}

/*
 * The same map for the separable power cost (Lemma 2.2(ii)):
 * T_a(x) = x_a - (h_a')^{-1}(d psi / d x_a) with (h_a')^{-1}(w) =
 * sign(w) |w|^{1/(p_a - 1)} (pw holds the exponents p_a).  pw == NULL: the
 * quadratic cost.
 */
int bfm_oracle_map_p(const double *psi, double *out, int ndim, const int *n, const double *pw)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    for (long p = 0; p < g.N; p++) {
        long r = p;
        for (int a = 0; a < ndim; a++) {
            long i = r % g.n[a];
            r /= g.n[a];
            long s = g.stride[a];
            int na = g.n[a];
            double h = g.h[a];
            double grad;
            if (na == 1) grad = 0.0;
            else if (i == 0) grad = (psi[p + s] - psi[p]) / h;
            else if (i == na - 1) grad = (psi[p] - psi[p - s]) / h;
            else grad = (psi[p + s] - psi[p - s]) / (2.0 * h);
            double x = (i + 0.5) * h;
            double disp = grad;
            if (pw) disp = (grad < 0 ? -1.0 : 1.0) * pow(fabs(grad), 1.0 / (pw[a] - 1.0));
            double t = x - disp;
            if (t < 0.5 * h) t = 0.5 * h;
            if (t > 1.0 - 0.5 * h) t = 1.0 - 0.5 * h;
            out[a * g.N + p] = t;
        }
    }
    return 0;
}

/*
 * rho = T#mu (pushforward definition, Section 2.1), discretised by a
 * bilinear / trilinear deposit (reading): every cell x_p with mu_p != 0 sends
 * its mass mu_p * hd to the 2^d cell centres around T(x_p), weighted by the
 * multilinear interpolation weights; rho is the received mass divided by hd.
 * Because T is clamped to the box of cell centres the mass is conserved.
 */
int bfm_oracle_pushforward_p(const double *psi, const double *mu, double *rho, int ndim,
                             const int *n, const double *pw);

int bfm_oracle_pushforward(const double *psi, const double *mu, double *rho, int ndim, const int *n)
{
    return bfm_oracle_pushforward_p(psi, mu, rho, ndim, n, NULL);
}

/* The same deposit with the map of the separable power cost (pw == NULL: quadratic). */
int bfm_oracle_pushforward_p(const double *psi, const double *mu, double *rho, int ndim,
                             const int *n, const double *pw)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    double *T = (double *)malloc(sizeof(double) * g.N * ndim);
    bfm_oracle_map_p(psi, T, ndim, n, pw);
    for (long p = 0; p < g.N; p++) rho[p] = 0.0;
    for (long p = 0; p < g.N; p++) {
        if (mu[p] == 0.0) continue;
        int i0[3] = {0, 0, 0};
        double w1[3] = {0, 0, 0};
        for (int a = 0; a < ndim; a++) {
            double pos = T[a * g.N + p] / g.h[a] - 0.5;   /* in cell-index units */
            int i = (int)floor(pos);
            if (i > g.n[a] - 2) i = g.n[a] - 2;
            if (i < 0) i = 0;
            i0[a] = i;
            w1[a] = pos - i;
            if (g.n[a] == 1) { i0[a] = 0; w1[a] = 0.0; }
        }
        int corners = 1 << ndim;
        for (int c = 0; c < corners; c++) {
            double w = 1.0;
            long q = 0;
            for (int a = 0; a < ndim; a++) {
                int up = (c >> a) & 1;
                w *= up ? w1[a] : (1.0 - w1[a]);
                q += (long)(i0[a] + up) * g.stride[a];
            }
            if (w != 0.0) rho[q] += mu[p] * w;
        }
    }
    free(T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* the back-and-forth method (Algorithm 1; step sizes Section 4.2)           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double beta1, beta2, alpha1, alpha2;  /* Section 4.2: 1/4, 3/4, 5/4, 4/5 */
    double sigma0;                        /* <= 0: 8 min(1/|mu|inf, 1/|nu|inf) */
    double sigma_min;                     /* 0.01 */
    int ct_mode;                          /* 0 brute, 1 Legendre/linear */
    int dct_mode;                         /* 0 definition, 1 FFT */
    int method;                           /* 0 back-and-forth, 1 gradient ascent on J */
    int power;                            /* 1: separable power cost with exponents p */
    double p[3];
} oracle_opts;

/* c-transform, pushforward and map of the cost in use */
static void ct_cost(const double *in, double *out, int ndim, const int *n, const oracle_opts *o)
{
    if (o->power) bfm_oracle_ctransform_p(in, out, ndim, n, o->p);
    else bfm_oracle_ctransform(in, out, ndim, n, o->ct_mode);
}

typedef struct {
    int iters;        /* completed back-and-forth iterations */
    int converged;
    double w2sq;      /* 2 J(phi_final) */
    double mass_mu, mass_nu;
    double sigma_final;
} oracle_info;

static double dot_hd(const grid_t *g, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < g->N; i++) s += a[i] * b[i];
    return g->hd * s;
}

/*
 * Step-size rule of Section 4.2 (no backtracking).  The accepted-gain window
 * is beta1 sigma G <= gain <= beta2 sigma G where gain = J(new) - J(old) and
 * G = ||grad||^2_{H1-dot}.  Too little gain: sigma *= alpha2 (never below
 * sigma_min, and never raised by a decrease); too much gain: sigma *= alpha1.
 */
static double step_rule(double sigma, double gain, double G, const oracle_opts *o)
{
    if (gain < o->beta1 * sigma * G) {
        double s = o->alpha2 * sigma;
        double floor_ = (o->sigma_min < sigma) ? o->sigma_min : sigma;
        return (s > floor_) ? s : floor_;
    }
    if (gain > o->beta2 * sigma * G) return o->alpha1 * sigma;
    return sigma;
}

/*
 * Algorithm 1 with the step rule of Section 4.2.  Per iteration n:
 *   phi-half:  psi~ = phi^c; J_old = J(phi); rho = T_phi#mu (T = x - grad psi~);
 *              g = (-Delta)^{-1}(nu - rho); r_n = sqrt(G / ||nu - 1||^2_{H^-1});
 *              stop here if r_n < tol (outputs phi, psi~);
 *              phi += sigma g; psi = phi^c; J_new = J(phi); update sigma.
 *   psi-half:  phi~ = psi^c; I_old = I(psi); rho = T_psi#nu (T = y - grad phi~);
 *              g = (-Delta)^{-1}(mu - rho); psi += sigma g; phi = psi^c;
 *              I_new = I(psi); update sigma.
 * Reading: one shared sigma updated after every half step; the residual is
 * the H^-1 norm of nu - T#mu relative to that of nu - 1 (mu and nu have unit
 * mass so their mean is 1); it is measured at the start of each iteration;
 * when nu is uniform (||nu - 1|| = 0) the absolute residual sqrt(G) is used.
 * Logs (length max_iter+1, may be NULL): dual[n] = J(phi_n), resid[n] = r_n,
 * sig[n] = sigma at the start of iteration n; half (length 3*max_iter) holds
 * half[3n..3n+2] = (J(phi_{n+1/2}), I(psi_{n+1/2}), I(psi_{n+1})); J(phi_{n+1})
 * is dual[n+1].
 * mu and nu are rescaled to unit mass first.  phi_out, psi_out: N each;
 * map_out: ndim*N (may be NULL).
 */
int bfm_oracle_solve(const double *mu_in, const double *nu_in, int ndim, const int *n,
                     double tol, int max_iter, const double *opt_in,
                     double *phi_out, double *psi_out, double *map_out,
                     double *dual, double *resid, double *sig, double *half,
                     double *info_out)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    oracle_opts o = {0.25, 0.75, 1.25, 0.8, 0.0, 0.01, 1, 1, 0, 0, {2.0, 2.0, 2.0}};
    if (opt_in) {
        o.beta1 = opt_in[0]; o.beta2 = opt_in[1]; o.alpha1 = opt_in[2]; o.alpha2 = opt_in[3];
        o.sigma0 = opt_in[4]; o.sigma_min = opt_in[5];
        o.ct_mode = (int)opt_in[6]; o.dct_mode = (int)opt_in[7]; o.method = (int)opt_in[8];
        /* opt_in[9..11] > 0: exponents of the separable power cost */
        if (opt_in[9] > 0) {
            o.power = 1;
            for (int a = 0; a < 3; a++) o.p[a] = opt_in[9 + a];
        }
    }
    const double *pc = o.power ? o.p : NULL;
    long N = g.N;
    double *mu = malloc(sizeof(double) * N), *nu = malloc(sizeof(double) * N);
    double *phi = calloc(N, sizeof(double)), *psi = calloc(N, sizeof(double));
    double *tmp = malloc(sizeof(double) * N), *rho = malloc(sizeof(double) * N);
    double *f = malloc(sizeof(double) * N), *gr = malloc(sizeof(double) * N);
    double mass_mu = 0, mass_nu = 0, mx_mu = 0, mx_nu = 0;
    for (long i = 0; i < N; i++) { mass_mu += mu_in[i]; mass_nu += nu_in[i]; }
    mass_mu *= g.hd; mass_nu *= g.hd;
    if (!(mass_mu > 0) || !(mass_nu > 0)) return -3;
    for (long i = 0; i < N; i++) {
        mu[i] = mu_in[i] / mass_mu; nu[i] = nu_in[i] / mass_nu;
        if (mu[i] > mx_mu) mx_mu = mu[i];
        if (nu[i] > mx_nu) mx_nu = nu[i];
    }
    double sigma = o.sigma0 > 0 ? o.sigma0 : 8.0 * fmin(1.0 / mx_mu, 1.0 / mx_nu);
    double Gref;
    for (long i = 0; i < N; i++) f[i] = nu[i] - 1.0;
    bfm_oracle_poisson(f, gr, ndim, n, o.dct_mode, &Gref);
    int it = 0, conv = 0;
    double Jold = 0.0;
    /*
     * The comparison method of Section 5 (Tables 5 and 6): H1-dot gradient
     * ascent on J alone, phi_{n+1/2} = phi_n + sigma grad J(phi_n),
     * phi_{n+1} = (phi_{n+1/2})^{cc}.  Reading: the step rule of Section 4.2
     * compares J(phi_{n+1/2}) with J(phi_n); residual, logs and outputs as for
     * Algorithm 1 (half[3n] = J(phi_{n+1/2})).
     */
    if (o.method == 1) for (it = 0; it <= max_iter; it++) {
        ct_cost(phi, tmp, ndim, n, &o);          /* phi_n^c */
        Jold = dot_hd(&g, phi, nu) + dot_hd(&g, tmp, mu);
        bfm_oracle_pushforward_p(tmp, mu, rho, ndim, n, pc);
        for (long i = 0; i < N; i++) f[i] = nu[i] - rho[i];
        double G;
        bfm_oracle_poisson(f, gr, ndim, n, o.dct_mode, &G);
        double r = (Gref > 0) ? sqrt(fmax(G, 0.0) / Gref) : sqrt(fmax(G, 0.0));
        if (dual) dual[it] = Jold;
        if (resid) resid[it] = r;
        if (sig) sig[it] = sigma;
        if (r < tol) { conv = 1; break; }
        if (it == max_iter) break;
        for (long i = 0; i < N; i++) phi[i] += sigma * gr[i];        /* phi_{n+1/2} */
        ct_cost(phi, psi, ndim, n, &o);          /* phi_{n+1/2}^c */
        double Jnew = dot_hd(&g, phi, nu) + dot_hd(&g, psi, mu);
        sigma = step_rule(sigma, Jnew - Jold, G, &o);
        ct_cost(psi, phi, ndim, n, &o);          /* phi_{n+1} */
        if (half) { half[3 * it + 0] = Jnew; half[3 * it + 1] = 0.0; half[3 * it + 2] = 0.0; }
    }
    if (o.method == 0) for (it = 0; it <= max_iter; it++) {
        /* phi-half step */
        ct_cost(phi, tmp, ndim, n, &o);          /* psi~ = phi^c */
        Jold = dot_hd(&g, phi, nu) + dot_hd(&g, tmp, mu);
        bfm_oracle_pushforward_p(tmp, mu, rho, ndim, n, pc);
        for (long i = 0; i < N; i++) f[i] = nu[i] - rho[i];
        double G;
        bfm_oracle_poisson(f, gr, ndim, n, o.dct_mode, &G);
        double r = (Gref > 0) ? sqrt(fmax(G, 0.0) / Gref) : sqrt(fmax(G, 0.0));
        if (dual) dual[it] = Jold;
        if (resid) resid[it] = r;
        if (sig) sig[it] = sigma;
        if (r < tol) { conv = 1; break; }
        if (it == max_iter) break;
        for (long i = 0; i < N; i++) phi[i] += sigma * gr[i];
        ct_cost(phi, psi, ndim, n, &o);          /* psi_{n+1/2} */
        double Jnew = dot_hd(&g, phi, nu) + dot_hd(&g, psi, mu);
        sigma = step_rule(sigma, Jnew - Jold, G, &o);
        /* psi-half step */
        ct_cost(psi, tmp, ndim, n, &o);          /* phi~ = psi^c */
        double Iold = dot_hd(&g, tmp, nu) + dot_hd(&g, psi, mu);
        bfm_oracle_pushforward_p(tmp, nu, rho, ndim, n, pc);
        for (long i = 0; i < N; i++) f[i] = mu[i] - rho[i];
        double G2;
        bfm_oracle_poisson(f, gr, ndim, n, o.dct_mode, &G2);
        for (long i = 0; i < N; i++) psi[i] += sigma * gr[i];
        ct_cost(psi, phi, ndim, n, &o);          /* phi_{n+1} */
        double Inew = dot_hd(&g, phi, nu) + dot_hd(&g, psi, mu);
        sigma = step_rule(sigma, Inew - Iold, G2, &o);
        if (half) {
            half[3 * it + 0] = Jnew; half[3 * it + 1] = Iold; half[3 * it + 2] = Inew;
        }
    }
    /* outputs: phi_n and its c-transform, the map T = x - grad phi_n^c */
    memcpy(phi_out, phi, sizeof(double) * N);
    memcpy(psi_out, tmp, sizeof(double) * N);
    if (map_out) bfm_oracle_map_p(tmp, map_out, ndim, n, pc);
    if (info_out) {
        info_out[0] = it;
        info_out[1] = conv;
        info_out[2] = 2.0 * Jold;
        info_out[3] = mass_mu;
        info_out[4] = mass_nu;
        info_out[5] = sigma;
    }
    free(mu); free(nu); free(phi); free(psi); free(tmp); free(rho); free(f); free(gr);
    return conv ? 0 : 1;
}

/*
 * Displacement interpolation (Section 4.3, images): rho_t = (S_t)#mu with
 * S_t(x) = t T(x) + (1-t) x, deposited exactly as in the pushforward above.
 * T is given as map[a*N + p] (clamped cell-centre coordinates).
 */
int bfm_oracle_interpolate(const double *map, const double *mu, double t, double *rho,
                           int ndim, const int *n)
{
    grid_t g;
    if (make_grid(ndim, n, &g)) return -1;
    for (long p = 0; p < g.N; p++) rho[p] = 0.0;
    for (long p = 0; p < g.N; p++) {
        if (mu[p] == 0.0) continue;
        long r = p;
        int i0[3] = {0, 0, 0};
        double w1[3] = {0, 0, 0};
        for (int a = 0; a < ndim; a++) {
            long i = r % g.n[a];
            r /= g.n[a];
            double x = (i + 0.5) * g.h[a];
            double s = t * map[a * g.N + p] + (1.0 - t) * x;
            double pos = s / g.h[a] - 0.5;
            int c = (int)floor(pos);
            if (c > g.n[a] - 2) c = g.n[a] - 2;
            if (c < 0) c = 0;
            i0[a] = c;
            w1[a] = pos - c;
        }
        for (int c = 0; c < (1 << ndim); c++) {
            double w = 1.0;
            long q = 0;
            for (int a = 0; a < ndim; a++) {
                int up = (c >> a) & 1;
                w *= up ? w1[a] : (1.0 - w1[a]);
                q += (long)(i0[a] + up) * g.stride[a];
            }
            if (w != 0.0) rho[q] += mu[p] * w;
        }
    }
    return 0;
}
