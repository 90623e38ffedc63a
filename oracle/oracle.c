/*
 * Plain FP64 CPU oracle for the fibre-bundle linear solve of Gjerden,
 * "Making the case of GPUs in courses on computational physics"
 * (arXiv:1305.3625).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into oracle/liboracle.so and
 * is loaded by tests/, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg -- nowhere else.  It shares no code, header, table or constant
 * generator with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes (every function cites the passage it follows):
 *   Eq. 1a-1c define, per fibre i on an L x L grid, f_i = -k_i (u_i - D) and
 *   u_i = sum_j G_ij f_j with the elastic Green's function G_ij of Eq. 1c.
 *   Multiplying Eq. 2, (I + K G) f = K D, by K^-1 gives the symmetric system
 *   (S + C) x = b with S = diag(s_i), s_i = 1/k_i, C = G and b = D.  The
 *   solution is unique because C + S is symmetric positive definite
 *   (Section 3, first paragraph).
 *
 *   G(r) = 1/(pi r) for r > 0 (Eq. 1c with a = 1 and (1 - nu^2)/E = 1, cell
 *   integral replaced by its point value) and G(0) = 4 ln(1 + sqrt 2)/pi, the
 *   exact cell integral of 1/r over the unit square.  The cell integral of
 *   Eq. 1c for every offset is available too (orc_G_cell, selected by
 *   orc_set_green).
 *
 *   Readings of the paper the oracle takes (the paper is silent or garbled):
 *     - Eq. 1b prints f_i inside the sum over j; it is read as f_j.
 *     - Eq. 3 is garbled; it is read as G x = F^-1 diag(F g) F x on a
 *       zero-padded grid (Section 3, Fourier acceleration), i.e. a linear
 *       (non-periodic) convolution evaluated by circular convolution on an
 *       M x M grid, M the smallest power of two >= 2L, with the input at
 *       [0, L)^2 and the output cropped to [0, L)^2.
 *     - Forward transform exp(-2 pi i jk/n), unnormalised inverse; the
 *       1/M^2 factor (Listing 3's optional normalisation) is applied once.
 *     - Convergence: ||b - A x||_2 <= rtol ||b||_2 with b the masked
 *       right-hand side; the test is certified on a recomputed residual.
 *     - A removed fibre leaves the system: A_m = P (C + S) P on the active
 *       set, x = 0 off it.  The next fibre to break is argmax |x_i|/t_i over
 *       active sites, ties to the lowest flat index.
 *
 * Layout: fields are row-major, flat index i = iy*L + ix (iy, ix in [0, L)).
 *
 * Every function returns 0 on success and a negative value on bad arguments or
 * allocation failure.  All floating point is double precision.
 */
#include <math.h>
#include <quadmath.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------- Eq. 1c -- */

/* Green's function between two grid sites a lattice vector (dx, dy) apart.
 * Eq. 1c with a = 1 and (1 - nu^2)/E = 1.  For r > 0 the point value of the
 * integrand, 1/(pi r); for r = 0 the exact cell integral
 * (1/pi) * int_{[-1/2,1/2]^2} dA / r = 4 ln(1 + sqrt 2) / pi. */
double orc_G(long dx, long dy)
{
    if (dx == 0 && dy == 0)
        return 4.0 * log(1.0 + sqrt(2.0)) / ORC_PI;
    double r = sqrt((double)dx * (double)dx + (double)dy * (double)dy);
    return 1.0 / (ORC_PI * r);
}

/* The cell integral of Eq. 1c itself, for every offset: (1/pi) times the
 * integral of 1/r over the unit cell centred at (dx, dy).  Written out with
 * the antiderivative of 1/sqrt(x^2 + y^2) in x and y,
 *   F(x, y) = x asinh(y/|x|) + y asinh(x/|y|)     (F = 0 on the axes),
 * as F(x+, y+) - F(x-, y+) - F(x+, y-) + F(x-, y-) over the cell's corners
 * x+- = dx +- 1/2, y+- = dy +- 1/2 (terms of one variable cancel in this
 * sum).  The four terms grow like r ln r while the result falls like 1/r, so
 * they are evaluated in quad precision (113-bit significand): the relative
 * rounding error is below 1e-30 r^2 ln r, far under double precision for
 * every offset of a 4096 x 4096 grid.  At (0, 0) the sum is 4 asinh(1),
 * the closed form of the self term above. */
static __float128 cell_F(__float128 x, __float128 y)
{
    __float128 v = 0;
    if (x != 0 && y != 0)
        v = x * asinhq(y / fabsq(x)) + y * asinhq(x / fabsq(y));
    return v;
}

double orc_G_cell(long dx, long dy)
{
    const __float128 h = 0.5Q, X = (__float128)dx, Y = (__float128)dy;
    __float128 I = cell_F(X + h, Y + h) - cell_F(X - h, Y + h) - cell_F(X + h, Y - h) + cell_F(X - h, Y - h);
    return (double)(I / M_PIq);
}

/* Which Green's function the functions below use: ORC_GREEN_POINT (orc_G, the
 * default) or ORC_GREEN_CELL (orc_G_cell, tabulated once for offsets below
 * lmax in each coordinate by orc_set_green).  Not thread-safe: a test sets it
 * before a call and resets it afterwards. */
#define ORC_GREEN_POINT 0
#define ORC_GREEN_CELL 1
static int g_kind = ORC_GREEN_POINT;
static double *g_cell = NULL;
static long g_cell_n = 0;

int orc_set_green(int kind, long lmax)
{
    if (kind == ORC_GREEN_POINT) {
        g_kind = kind;
        return 0;
    }
    if (kind != ORC_GREEN_CELL || lmax < 1 || lmax > 8192)
        return -1;
    if (lmax > g_cell_n) {
        double *t = malloc(sizeof(double) * (size_t)lmax * lmax);
        if (!t)
            return -1;
#pragma omp parallel for schedule(dynamic)
        for (long dy = 0; dy < lmax; ++dy)
            for (long dx = 0; dx <= dy; ++dx) {
                double g = orc_G_cell(dx, dy);
                t[dy * lmax + dx] = g;
                t[dx * lmax + dy] = g;
            }
        free(g_cell);
        g_cell = t;
        g_cell_n = lmax;
    }
    g_kind = kind;
    return 0;
}

/* The Green's function in use between sites (dx, dy) apart. */
static double Gk(long dx, long dy)
{
    if (g_kind == ORC_GREEN_POINT)
        return orc_G(dx, dy);
    long ax = labs(dx), ay = labs(dy);
    if (ax < g_cell_n && ay < g_cell_n)
        return g_cell[ay * g_cell_n + ax];
    return orc_G_cell(dx, dy);
}

/* Side of the padded grid: smallest power of two >= 2L (linear convolution of
 * two length-L sequences needs a period of at least 2L - 1). */
int orc_padded_side(int L)
{
    if (L < 1 || L > (1 << 14))
        return -1;
    int m = 2;
    while (m < 2 * L)
        m *= 2;
    return m;
}

/* Signed lattice offset stored at padded index j, or a flag that index j holds
 * no offset reachable between two sites of the L x L grid. */
static int wrap_offset(int j, int L, int M, long *d)
{
    if (j < L) {
        *d = j;
        return 1;
    }
    if (j > M - L) {
        *d = (long)j - M;
        return 1;
    }
    return 0;
}

/* Circulant embedding of G on the M x M grid (Section 3, Fourier
 * acceleration): k[jy*M + jx] = G(dx, dy) where (dx, dy) are the wrapped
 * offsets of (jx, jy); entries that no pair of sites can reach are 0. */
int orc_kernel_table(int L, double *k)
{
    int M = orc_padded_side(L);
    if (M < 0 || !k)
        return -1;
    for (int jy = 0; jy < M; ++jy)
        for (int jx = 0; jx < M; ++jx) {
            long dx, dy;
            int okx = wrap_offset(jx, L, M, &dx);
            int oky = wrap_offset(jy, L, M, &dy);
            k[(size_t)jy * M + jx] = (okx && oky) ? Gk(dx, dy) : 0.0;
        }
    return 0;
}

/* ------------------------------------------------- direct convolution ---- */

/* One output of the coupling term of Eq. 1b: y_i = sum_j G(r_i - r_j) x_j over
 * the open (non-periodic) L x L grid.  O(L^2) work. */
double orc_conv_direct_at(int L, const double *x, int iy, int ix)
{
    double acc = 0.0;
    for (int jy = 0; jy < L; ++jy)
        for (int jx = 0; jx < L; ++jx)
            acc += Gk((long)ix - jx, (long)iy - jy) * x[(size_t)jy * L + jx];
    return acc;
}

/* Whole coupling term y = C x by the definition (Eq. 1b), O(L^4). */
int orc_conv_direct(int L, const double *x, double *y)
{
    if (L < 1 || !x || !y)
        return -1;
#pragma omp parallel for schedule(dynamic)
    for (int iy = 0; iy < L; ++iy)
        for (int ix = 0; ix < L; ++ix)
            y[(size_t)iy * L + ix] = orc_conv_direct_at(L, x, iy, ix);
    return 0;
}

/* Dense operator A = C + diag(s) as an N x N row-major matrix, N = L^2
 * (Eq. 2 in its symmetric form).  s may be NULL for C alone. */
int orc_dense_operator(int L, const double *s, double *A)
{
    if (L < 1 || L > 128 || !A)
        return -1;
    long N = (long)L * L;
#pragma omp parallel for
    for (long i = 0; i < N; ++i) {
        long iy = i / L, ix = i % L;
        for (long j = 0; j < N; ++j) {
            long jy = j / L, jx = j % L;
            A[i * N + j] = Gk(ix - jx, iy - jy);
        }
        if (s)
            A[i * N + i] += s[i];
    }
    return 0;
}

/* ------------------------------------------------------------------ FFT -- */

/* In-place iterative radix-2 Cooley-Tukey transform of length n (a power of
 * two): X[k] = sum_j x[j] exp(sign * 2 pi i jk / n), sign = -1 forward,
 * +1 inverse, no normalisation.  Bit-reversal permutation, then log2(n)
 * butterfly levels; each twiddle is evaluated directly with cos/sin. */
int orc_fft(int n, double *re, double *im, int sign)
{
    if (n < 1 || (n & (n - 1)) || !re || !im || (sign != 1 && sign != -1))
        return -1;
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1)
            j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i];
            re[i] = re[j];
            re[j] = t;
            t = im[i];
            im[i] = im[j];
            im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double ang = sign * 2.0 * ORC_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int start = 0; start < n; start += len) {
                int a = start + k, b = a + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr;
                im[b] = im[a] - ti;
                re[a] += tr;
                im[a] += ti;
            }
        }
    }
    return 0;
}

/* 2D transform of an M x M row-major array: 1D transforms of every row, then
 * of every column. */
int orc_fft2(int M, double *re, double *im, int sign)
{
    if (M < 1 || (M & (M - 1)) || !re || !im)
        return -1;
    int bad = 0;
#pragma omp parallel for reduction(| : bad)
    for (int r = 0; r < M; ++r)
        bad |= orc_fft(M, re + (size_t)r * M, im + (size_t)r * M, sign) != 0;
#pragma omp parallel reduction(| : bad)
    {
        double *cr = malloc(sizeof(double) * M), *ci = malloc(sizeof(double) * M);
        if (!cr || !ci)
            bad |= 1;
#pragma omp for
        for (int c = 0; c < M; ++c) {
            if (!cr || !ci)
                continue;
            for (int r = 0; r < M; ++r) {
                cr[r] = re[(size_t)r * M + c];
                ci[r] = im[(size_t)r * M + c];
            }
            bad |= orc_fft(M, cr, ci, sign) != 0;
            for (int r = 0; r < M; ++r) {
                re[(size_t)r * M + c] = cr[r];
                im[(size_t)r * M + c] = ci[r];
            }
        }
        free(cr);
        free(ci);
    }
    return bad ? -1 : 0;
}

/* Kernel spectrum FFT2(k) / M^2 (Listing 3's normalisation folded in once; the
 * transform of G is computed at set-up, Listing 4 comment).  re and im are
 * M x M. */
int orc_spectrum(int L, double *re, double *im)
{
    int M = orc_padded_side(L);
    if (M < 0 || !re || !im)
        return -1;
    if (orc_kernel_table(L, re))
        return -1;
    memset(im, 0, sizeof(double) * (size_t)M * M);
    if (orc_fft2(M, re, im, -1))
        return -1;
    double scale = 1.0 / ((double)M * (double)M);
    for (size_t i = 0; i < (size_t)M * M; ++i) {
        re[i] *= scale;
        im[i] *= scale;
    }
    return 0;
}

/* ------------------------------------------------- FFT convolution ------ */

typedef struct {
    int L, M;
    double *kre, *kim; /* spectrum FFT2(k)/M^2 */
    double *wre, *wim; /* work grid */
} orc_conv;

static void conv_free(orc_conv *c)
{
    free(c->kre);
    free(c->kim);
    free(c->wre);
    free(c->wim);
}

static int conv_init(orc_conv *c, int L)
{
    memset(c, 0, sizeof(*c));
    c->L = L;
    c->M = orc_padded_side(L);
    if (c->M < 0)
        return -1;
    size_t mm = (size_t)c->M * c->M;
    c->kre = malloc(sizeof(double) * mm);
    c->kim = malloc(sizeof(double) * mm);
    c->wre = malloc(sizeof(double) * mm);
    c->wim = malloc(sizeof(double) * mm);
    if (!c->kre || !c->kim || !c->wre || !c->wim || orc_spectrum(L, c->kre, c->kim)) {
        conv_free(c);
        return -1;
    }
    return 0;
}

/* y = C x through the Fourier route of Listing 4: copy x into a zero complex
 * grid, forward 2D transform, multiply by the kernel spectrum, inverse 2D
 * transform, keep the real part of the [0, L)^2 corner. */
static int conv_apply(orc_conv *c, const double *x, double *y)
{
    int L = c->L, M = c->M;
    size_t mm = (size_t)M * M;
    memset(c->wre, 0, sizeof(double) * mm);
    memset(c->wim, 0, sizeof(double) * mm);
    for (int iy = 0; iy < L; ++iy)
        for (int ix = 0; ix < L; ++ix)
            c->wre[(size_t)iy * M + ix] = x[(size_t)iy * L + ix];
    if (orc_fft2(M, c->wre, c->wim, -1))
        return -1;
    for (size_t i = 0; i < mm; ++i) {
        double ar = c->kre[i], ai = c->kim[i], br = c->wre[i], bi = c->wim[i];
        c->wre[i] = ar * br - ai * bi;
        c->wim[i] = ar * bi + ai * br;
    }
    if (orc_fft2(M, c->wre, c->wim, +1))
        return -1;
    for (int iy = 0; iy < L; ++iy)
        for (int ix = 0; ix < L; ++ix)
            y[(size_t)iy * L + ix] = c->wre[(size_t)iy * M + ix];
    return 0;
}

int orc_conv_fft(int L, const double *x, double *y)
{
    orc_conv c;
    if (!x || !y || conv_init(&c, L))
        return -1;
    int rc = conv_apply(&c, x, y);
    conv_free(&c);
    return rc;
}

/* ----------------------------------------------------- CG (Listing 2) ---- */

static double dot(long n, const double *a, const double *b)
{
    double acc = 0.0;
    for (long i = 0; i < n; ++i)
        acc += a[i] * b[i];
    return acc;
}

/* q = P (C + S) P v with P the projection on active sites. */
static int apply_A(orc_conv *c, const double *s, const unsigned char *mask, const double *v,
                   double *tmp, double *q)
{
    long N = (long)c->L * c->L;
    for (long i = 0; i < N; ++i)
        tmp[i] = (!mask || mask[i]) ? v[i] : 0.0;
    if (conv_apply(c, tmp, q))
        return -1;
    for (long i = 0; i < N; ++i)
        q[i] = (!mask || mask[i]) ? q[i] + s[i] * tmp[i] : 0.0;
    return 0;
}

/* Unpreconditioned conjugate gradients (Listing 2; Section 3 names CG and the
 * paper drops the preconditioner) on (P (C + S) P) x = P b, from the initial
 * x given (warm start), Hestenes-Stiefel form:
 *   q = A p; alpha = rr / (p.q); x += alpha p; r -= alpha q;
 *   rr' = r.r; stop if sqrt(rr') <= rtol ||Pb||; p = r + (rr'/rr) p.
 * On the recursive-residual stop the residual b - A x is recomputed; if it is
 * still above rtol the iteration restarts from it.  x is zeroed off the active
 * set.  Returns 0 when converged, 1 when maxit was reached, <0 on error.
 * iters receives the number of matrix-vector products spent in the loop and
 * relres the final recomputed ||b - A x|| / ||b||. */
int orc_cg(int L, const double *s, const double *b, double *x, const unsigned char *mask,
           double rtol, int maxit, int *iters, double *relres)
{
    if (L < 1 || !s || !b || !x)
        return -1;
    orc_conv c;
    if (conv_init(&c, L))
        return -1;
    long N = (long)L * L;
    double *r = malloc(sizeof(double) * N), *p = malloc(sizeof(double) * N);
    double *q = malloc(sizeof(double) * N), *tmp = malloc(sizeof(double) * N);
    double *bm = malloc(sizeof(double) * N);
    int rc = 0, it = 0;
    if (!r || !p || !q || !tmp || !bm) {
        rc = -2;
        goto out;
    }
    for (long i = 0; i < N; ++i) {
        bm[i] = (!mask || mask[i]) ? b[i] : 0.0;
        if (mask && !mask[i])
            x[i] = 0.0;
    }
    double bnorm = sqrt(dot(N, bm, bm));
    double relres_now = 0.0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * N);
        goto done;
    }
    for (;;) {
        /* r = b - A x (recomputed residual), p = r */
        if (apply_A(&c, s, mask, x, tmp, q)) {
            rc = -3;
            goto out;
        }
        for (long i = 0; i < N; ++i) {
            r[i] = bm[i] - q[i];
            p[i] = r[i];
        }
        double rr = dot(N, r, r);
        relres_now = sqrt(rr) / bnorm;
        if (relres_now <= rtol)
            break;
        if (it >= maxit) {
            rc = 1;
            break;
        }
        while (it < maxit) {
            if (apply_A(&c, s, mask, p, tmp, q)) {
                rc = -3;
                goto out;
            }
            ++it;
            double alpha = rr / dot(N, p, q);
            for (long i = 0; i < N; ++i) {
                x[i] += alpha * p[i];
                r[i] -= alpha * q[i];
            }
            double rr_new = dot(N, r, r);
            if (sqrt(rr_new) <= rtol * bnorm)
                break;
            double beta = rr_new / rr;
            for (long i = 0; i < N; ++i)
                p[i] = r[i] + beta * p[i];
            rr = rr_new;
        }
    }
done:
    if (iters)
        *iters = it;
    if (relres)
        *relres = relres_now;
out:
    free(r);
    free(p);
    free(q);
    free(tmp);
    free(bm);
    conv_free(&c);
    return rc;
}

/* (C + S) x (+ masking) for the caller: q = P (C + S) P x. */
int orc_apply_A(int L, const double *s, const unsigned char *mask, const double *x, double *q)
{
    orc_conv c;
    if (L < 1 || !s || !x || !q || conv_init(&c, L))
        return -1;
    double *tmp = malloc(sizeof(double) * (size_t)L * L);
    int rc = tmp ? apply_A(&c, s, mask, x, tmp, q) : -2;
    free(tmp);
    conv_free(&c);
    return rc;
}

/* ------------------------------------------------------- dense solve ---- */

/* Solve A x = b for a symmetric positive definite n x n matrix by the textbook
 * Cholesky factorisation A = R^T R followed by two triangular solves.  A is
 * not modified.  Returns -4 if A is not positive definite. */
int orc_cholesky_solve(int n, const double *A, const double *b, double *x)
{
    if (n < 1 || !A || !b || !x)
        return -1;
    double *R = calloc((size_t)n * n, sizeof(double));
    double *y = malloc(sizeof(double) * n);
    if (!R || !y) {
        free(R);
        free(y);
        return -2;
    }
    int rc = 0;
    for (int j = 0; j < n && !rc; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k)
            d -= R[(size_t)k * n + j] * R[(size_t)k * n + j];
        if (!(d > 0.0)) {
            rc = -4;
            break;
        }
        double rjj = sqrt(d);
        R[(size_t)j * n + j] = rjj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)j * n + i];
            for (int k = 0; k < j; ++k)
                v -= R[(size_t)k * n + j] * R[(size_t)k * n + i];
            R[(size_t)j * n + i] = v / rjj;
        }
    }
    if (!rc) {
        for (int i = 0; i < n; ++i) { /* R^T y = b */
            double v = b[i];
            for (int k = 0; k < i; ++k)
                v -= R[(size_t)k * n + i] * y[k];
            y[i] = v / R[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) { /* R x = y */
            double v = y[i];
            for (int k = i + 1; k < n; ++k)
                v -= R[(size_t)i * n + k] * x[k];
            x[i] = v / R[(size_t)i * n + i];
        }
    }
    free(R);
    free(y);
    return rc;
}

/* ----------------------------------------------- quasi-static breaking -- */

/* Next fibre to break (Section 2: bonds break when the local strain is
 * large; the load is linear in D, so the first fibre to reach its threshold
 * as D grows is the one with the largest |x_i| / t_i).  Active sites only;
 * ties go to the lowest flat index.  Returns the index or -1 if none. */
long orc_argmax_ratio(long N, const double *x, const double *t, const unsigned char *mask,
                      double *ratio)
{
    long best = -1;
    double bv = 0.0;
    for (long i = 0; i < N; ++i) {
        if (mask && !mask[i])
            continue;
        double v = fabs(x[i]) / t[i];
        if (best < 0 || v > bv) {
            best = i;
            bv = v;
        }
    }
    if (ratio)
        *ratio = bv;
    return best;
}

/* Quasi-static removal loop (Section 2, one solve per simulation step): for
 * each step, solve P(C+S)P x = P b warm-started from x, pick
 * i* = argmax |x_i|/t_i, record it, set mask[i*] = 0 and x[i*] = 0.
 * picks, ratios and iters receive one entry per step.  mask and x are
 * updated in place. */
/* Front of a breaking run (Section 2: the front separates wholly broken from
 * wholly intact material).  Per column ix: first_intact = smallest iy with
 * mask 1 (L if none), damage_end = 1 + largest iy with mask 0 (0 if none). */
int orc_front(int L, const unsigned char *mask, int *first_intact, int *damage_end)
{
    if (L < 1 || !mask || !first_intact || !damage_end)
        return -1;
    for (int ix = 0; ix < L; ++ix) {
        int fi = L, de = 0;
        for (int iy = 0; iy < L; ++iy) {
            if (mask[(size_t)iy * L + ix]) {
                if (fi == L)
                    fi = iy;
            } else {
                de = iy + 1;
            }
        }
        first_intact[ix] = fi;
        damage_end[ix] = de;
    }
    return 0;
}

int orc_masked_loop(int L, const double *s, const double *b, const double *t, unsigned char *mask,
                    double *x, int steps, double rtol, int maxit, long *picks, double *ratios,
                    int *iters)
{
    if (L < 1 || !s || !b || !t || !mask || !x || steps < 0)
        return -1;
    long N = (long)L * L;
    for (int st = 0; st < steps; ++st) {
        int it = 0;
        double rel = 0.0;
        int rc = orc_cg(L, s, b, x, mask, rtol, maxit, &it, &rel);
        if (rc < 0)
            return rc;
        double ratio = 0.0;
        long k = orc_argmax_ratio(N, x, t, mask, &ratio);
        if (picks)
            picks[st] = k;
        if (ratios)
            ratios[st] = ratio;
        if (iters)
            iters[st] = it;
        if (k < 0)
            break;
        mask[k] = 0;
        x[k] = 0.0;
    }
    return 0;
}
