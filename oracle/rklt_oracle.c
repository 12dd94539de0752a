/*
 * rklt_oracle.c -- plain, slow, FP64 CPU oracle of the rounded-KLT (RKLT) image
 * compression path of "Low-complexity Rounded KLT Approximation for Image
 * Compression" (Radunz, Bayer, Cintra; arXiv 2111.14239).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library: only the test-suite, the smoke entry point and the benchmark's CPU
 * baseline may build, load or call it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Everything is written as the plain definition, in double precision, with
 * straight loops and no blocking or reordering:
 *   - Markov-1 autocorrelation R[i][j] = rho^|i-j|             (Sec. 2.1, Sec. 3.1)
 *   - exact KLT by two routes: the closed form with the omega roots found by
 *     bisection (Sec. 2.1), and a cyclic Jacobi eigen-solver of R (Sec. 3)
 *   - T = round(alpha*K), round(x) = floor(x + 1/2)               (Sec. 2.3, Eq. 2)
 *   - S from Eq. 1; That = S*T                                    (Sec. 2.2)
 *   - per N x N block: B = That*A*That^T, zig-zag order, keep the first r,
 *     A' = That^{-1}*B'*That^{-T}                               (Sec. 4.1, Appendix)
 *   - SSE, MSE and PSNR with peak 255                            (Sec. 4.1, Table 3)
 *   - unified coding gain, transform efficiency, MSE to the KLT and total
 *     error energy                                                (Sec. 3.1)
 *   - the comparison transforms of the results (Sec. 4.1): the exact KLT (above)
 *     and the orthonormal DCT-II, both run through the same per-block path with
 *     That replaced by the transform matrix
 *   - JPEG-like quantisation with S absorbed into Q (Appendix)
 *   - the MSSIM quality measure of the results (Sec. 4.1)
 *
 * Readings taken where the paper is garbled or silent (each one is tested):
 *   - the closed form's sine argument is omega_i*(j - (N-1)/2) + (i+1)*pi/2
 *     (row i = eigen-index, column j = sample); the printed form swaps i and j
 *     inside the bracket and is not orthogonal;
 *   - omega_i is the root of the Sec. 2.1 equation in (i*pi/N, (i+1)*pi/N);
 *   - eigenvector signs make K[i][0] > 0;
 *   - the 2-D forward transform is That*A*That^T for every T and the inverse is
 *     That^{-1}*B'*That^{-T} (Appendix, with the transpose kept for the right
 *     factor so that r = N*N reconstructs A exactly);
 *   - no level shift; zig-zag is the JPEG walk generalised to any N;
 *   - PSNR uses the unrounded reconstruction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_SINGULAR 2
#define ORC_ERR_NOCONV 3

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Signal model (Sec. 2.1)                                                  */
/* ------------------------------------------------------------------------ */

/* R[i][j] = rho^|i-j|: autocorrelation of a unit-variance first-order Markov
 * signal (Sec. 3.1, used by the coding gain and transform efficiency). */
void orc_markov_autocorr(int n, double rho, double *R)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            R[i * n + j] = pow(rho, (double)abs(i - j));
}

/* The omega equation of Sec. 2.1, tan(N w) = -(1-rho^2) sin w / ((1+rho^2) cos w - 2 rho),
 * multiplied through by cos(N w) so that it has no poles:
 *   g(w) = sin(N w) ((1+rho^2) cos w - 2 rho) + (1-rho^2) sin w cos(N w). */
static double orc_omega_eq(int n, double rho, double w)
{
    return sin(n * w) * ((1.0 + rho * rho) * cos(w) - 2.0 * rho)
         + (1.0 - rho * rho) * sin(w) * cos(n * w);
}

/* The i-th root lies in (i*pi/N, (i+1)*pi/N).  At the interval ends g takes the
 * signs +1 (as w -> 0+) and (-1)^k at w = k*pi/N for 1 <= k <= N-1, and
 * (-1)^N (as w -> pi-); bisection keeps the sign of the left end. */
static double orc_omega_root(int n, double rho, int i)
{
    double a = i * ORC_PI / n, b = (i + 1) * ORC_PI / n;
    double sa = (i == 0) ? 1.0 : ((i % 2) ? -1.0 : 1.0);
    for (int it = 0; it < 200; it++) {
        double m = 0.5 * (a + b);
        double gm = orc_omega_eq(n, rho, m);
        if ((gm > 0.0 && sa > 0.0) || (gm < 0.0 && sa < 0.0)) a = m; else b = m;
        if (gm == 0.0) { a = b = m; break; }
    }
    return 0.5 * (a + b);
}

/* Closed-form KLT of the Markov-1 process (Sec. 2.1), with the index reading
 * described at the top of this file.  K is row-major, row i = i-th basis
 * vector; lambda[i] are the eigenvalues, in decreasing order. */
int orc_klt_closed_form(int n, double rho, double *K, double *lambda)
{
    if (n < 2 || !(rho > 0.0 && rho < 1.0)) return ORC_ERR_ARG;
    for (int i = 0; i < n; i++) {
        double w = orc_omega_root(n, rho, i);
        double lam = (1.0 - rho * rho) / (1.0 + rho * rho - 2.0 * rho * cos(w));
        lambda[i] = lam;
        double amp = sqrt(2.0 / (n + lam));
        for (int j = 0; j < n; j++)
            K[i * n + j] = amp * sin(w * (j - (n - 1) / 2.0) + (i + 1) * ORC_PI / 2.0);
    }
    return ORC_OK;
}

/* Exact KLT by eigendecomposition of R (the paper obtains its exact KLT
 * matrices numerically, Sec. 3): cyclic Jacobi rotations until the
 * off-diagonal mass vanishes, rows sorted by decreasing eigenvalue, each row's
 * sign fixed so that K[i][0] > 0. */
int orc_klt_jacobi(int n, double rho, double *K, double *lambda)
{
    if (n < 2 || !(rho > 0.0 && rho < 1.0)) return ORC_ERR_ARG;
    double *a = (double *)malloc(sizeof(double) * n * n);
    double *v = (double *)malloc(sizeof(double) * n * n);
    orc_markov_autocorr(n, rho, a);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) v[i * n + j] = (i == j) ? 1.0 : 0.0;

    int converged = 0;
    for (int sweep = 0; sweep < 100 && !converged; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off += a[p * n + q] * a[p * n + q];
        if (off < 1e-30) { converged = 1; break; }
        for (int p = 0; p < n; p++) {
            for (int q = p + 1; q < n; q++) {
                double apq = a[p * n + q];
                if (apq == 0.0) continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < n; k++) {
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = v[k * n + p], vkq = v[k * n + q];
                    v[k * n + p] = c * vkp - s * vkq;
                    v[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    if (!converged) { free(a); free(v); return ORC_ERR_NOCONV; }

    /* columns of v are eigenvectors; order by decreasing eigenvalue */
    int *idx = (int *)malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++) idx[i] = i;
    for (int i = 0; i < n; i++)          /* selection sort, descending */
        for (int j = i + 1; j < n; j++)
            if (a[idx[j] * n + idx[j]] > a[idx[i] * n + idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < n; i++) {
        int c = idx[i];
        lambda[i] = a[c * n + c];
        double sg = (v[0 * n + c] < 0.0) ? -1.0 : 1.0;
        for (int j = 0; j < n; j++) K[i * n + j] = sg * v[j * n + c];
    }
    free(idx); free(a); free(v);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Approximation design (Sec. 2.2, 2.3)                                    */
/* ------------------------------------------------------------------------ */

/* T = round(alpha*K) with round(x) = floor(x + 1/2), elementwise (Eq. 2).
 * *tie_margin receives min |alpha*k - (m + 1/2)| over all entries and integers
 * m: how far the rounding is from a tie.  Returns ORC_ERR_ARG if an entry falls
 * outside {0, +1, -1} (the restriction of Sec. 2.3). */
int orc_round_alpha(int n, double alpha, const double *K, int *T, double *tie_margin)
{
    double margin = 1e300;
    int ok = 1;
    for (int i = 0; i < n * n; i++) {
        double x = alpha * K[i];
        double t = floor(x + 0.5);
        T[i] = (int)t;
        double d = fabs(x - (floor(x) + 0.5));
        if (d < margin) margin = d;
        if (t < -1.0 || t > 1.0) ok = 0;
    }
    if (tie_margin) *tie_margin = margin;
    return ok ? ORC_OK : ORC_ERR_ARG;
}

/* Eq. 1: S = sqrt((T T^T)^{-1}) when T T^T is diagonal ("orthogonal" rows),
 * else S = sqrt(diag(T T^T)^{-1}).  Both are diagonal; s[i] = 1/sqrt((T T^T)_ii).
 * *orthogonal = 1 when every off-diagonal entry of T T^T is zero.
 * Returns ORC_ERR_SINGULAR for an all-zero row. */
int orc_normalisation(int n, const int *T, double *s, int *orthogonal)
{
    int orth = 1;
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            long acc = 0;
            for (int k = 0; k < n; k++) acc += (long)T[i * n + k] * T[j * n + k];
            if (i == j) {
                if (acc == 0) return ORC_ERR_SINGULAR;
                s[i] = 1.0 / sqrt((double)acc);
            } else if (acc != 0) {
                orth = 0;
            }
        }
    }
    if (orthogonal) *orthogonal = orth;
    return ORC_OK;
}

/* That = S * T  (Sec. 2.2) */
void orc_that(int n, const int *T, const double *s, double *That)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) That[i * n + j] = s[i] * (double)T[i * n + j];
}

/* Matrix inverse by Gauss-Jordan elimination with partial pivoting, FP64. */
int orc_invert(int n, const double *M, double *Minv)
{
    double *a = (double *)malloc(sizeof(double) * n * 2 * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            a[i * 2 * n + j] = (j < n) ? M[i * n + j] : ((j - n == i) ? 1.0 : 0.0);
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int i = col + 1; i < n; i++)
            if (fabs(a[i * 2 * n + col]) > fabs(a[piv * 2 * n + col])) piv = i;
        if (fabs(a[piv * 2 * n + col]) < 1e-12) { free(a); return ORC_ERR_SINGULAR; }
        if (piv != col)
            for (int j = 0; j < 2 * n; j++) {
                double t = a[col * 2 * n + j]; a[col * 2 * n + j] = a[piv * 2 * n + j]; a[piv * 2 * n + j] = t;
            }
        double p = a[col * 2 * n + col];
        for (int j = 0; j < 2 * n; j++) a[col * 2 * n + j] /= p;
        for (int i = 0; i < n; i++) {
            if (i == col) continue;
            double f = a[i * 2 * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; j++) a[i * 2 * n + j] -= f * a[col * 2 * n + j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Minv[i * n + j] = a[i * 2 * n + n + j];
    free(a);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Zig-zag order (Sec. 4.1)                                                 */
/* ------------------------------------------------------------------------ */

/* Position k of the zig-zag walk is (row[k], col[k]) of the coefficient block,
 * row = vertical frequency.  The walk visits the anti-diagonals d = i + j in
 * increasing order; on odd d it moves down-left (row increasing), on even d
 * up-right (row decreasing); so it starts (0,0), (0,1), (1,0), (2,0), (1,1)... */
/* Orthonormal DCT-II (the DCT the results compare against, Sec. 4.1):
 * M[k][j] = c_k cos(pi (2j + 1) k / (2n)), c_0 = sqrt(1/n), c_k = sqrt(2/n). */
void orc_dct2(int n, double *M)
{
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; k++) {
        double c = sqrt((k == 0 ? 1.0 : 2.0) / n);
        for (int j = 0; j < n; j++)
            M[k * n + j] = c * cos(pi * (2 * j + 1) * k / (2.0 * n));
    }
}

void orc_zigzag(int n, int *row, int *col)
{
    int k = 0;
    for (int d = 0; d <= 2 * n - 2; d++) {
        int lo = (d - (n - 1) > 0) ? d - (n - 1) : 0;
        int hi = (d < n - 1) ? d : n - 1;
        if (d % 2 == 1) {
            for (int i = lo; i <= hi; i++) { row[k] = i; col[k] = d - i; k++; }
        } else {
            for (int i = hi; i >= lo; i--) { row[k] = i; col[k] = d - i; k++; }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Blockwise 2-D transforms (Sec. 4.1, Appendix)                            */
/* ------------------------------------------------------------------------ */

static int orc_shape_ok(int n, int H, int W, long ld)
{
    return n >= 2 && H >= 0 && W >= 0 && H % n == 0 && W % n == 0 && ld >= W;
}

/* Integer stage: C = T * A * T^T for every block, exactly, in int64.  Output
 * C[blk][i][j] (raster order inside the block); blocks ordered row-major over
 * the (H/n) x (W/n) block grid. */
int orc_int_stage(int n, const int *T, const uint8_t *img, int H, int W, long ld, int64_t *C)
{
    if (!orc_shape_ok(n, H, W, ld)) return ORC_ERR_ARG;
    int bw = W / n, bh = H / n;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * n * n);
    for (int by = 0; by < bh; by++)
        for (int bx = 0; bx < bw; bx++) {
            const uint8_t *a = img + (long)by * n * ld + (long)bx * n;
            /* tmp = T * A */
            for (int i = 0; i < n; i++)
                for (int l = 0; l < n; l++) {
                    int64_t acc = 0;
                    for (int k = 0; k < n; k++) acc += (int64_t)T[i * n + k] * a[(long)k * ld + l];
                    tmp[i * n + l] = acc;
                }
            /* C = tmp * T^T */
            int64_t *c = C + ((long)by * bw + bx) * n * n;
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) {
                    int64_t acc = 0;
                    for (int l = 0; l < n; l++) acc += tmp[i * n + l] * (int64_t)T[j * n + l];
                    c[i * n + j] = acc;
                }
        }
    free(tmp);
    return ORC_OK;
}

/* One block: B = M * A * M^T, FP64, A given as doubles (stride n). */
static void orc_block_forward(int n, const double *M, const double *A, double *tmp, double *B)
{
    for (int i = 0; i < n; i++)
        for (int l = 0; l < n; l++) {
            double acc = 0.0;
            for (int k = 0; k < n; k++) acc += M[i * n + k] * A[k * n + l];
            tmp[i * n + l] = acc;
        }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double acc = 0.0;
            for (int l = 0; l < n; l++) acc += tmp[i * n + l] * M[j * n + l];
            B[i * n + j] = acc;
        }
}

/* One block: A' = Minv * B * Minv^T, FP64. */
static void orc_block_inverse(int n, const double *Minv, const double *B, double *tmp, double *A)
{
    for (int i = 0; i < n; i++)
        for (int l = 0; l < n; l++) {
            double acc = 0.0;
            for (int k = 0; k < n; k++) acc += Minv[i * n + k] * B[k * n + l];
            tmp[i * n + l] = acc;
        }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double acc = 0.0;
            for (int l = 0; l < n; l++) acc += tmp[i * n + l] * Minv[j * n + l];
            A[i * n + j] = acc;
        }
}

/* Forward 2-D transform of every block with a real N x N matrix M (That for
 * the RKLT): B = M A M^T, written in zig-zag order: out[blk][k] = B[row[k]][col[k]]. */
int orc_forward(int n, const double *M, const uint8_t *img, int H, int W, long ld, double *out)
{
    if (!orc_shape_ok(n, H, W, ld)) return ORC_ERR_ARG;
    int bw = W / n, bh = H / n;
    int *zr = (int *)malloc(sizeof(int) * n * n), *zc = (int *)malloc(sizeof(int) * n * n);
    orc_zigzag(n, zr, zc);
    double *A = (double *)malloc(sizeof(double) * n * n), *tmp = (double *)malloc(sizeof(double) * n * n);
    double *B = (double *)malloc(sizeof(double) * n * n);
    for (int by = 0; by < bh; by++)
        for (int bx = 0; bx < bw; bx++) {
            for (int k = 0; k < n; k++)
                for (int l = 0; l < n; l++)
                    A[k * n + l] = img[((long)by * n + k) * ld + (long)bx * n + l];
            orc_block_forward(n, M, A, tmp, B);
            double *o = out + ((long)by * bw + bx) * n * n;
            for (int k = 0; k < n * n; k++) o[k] = B[zr[k] * n + zc[k]];
        }
    free(zr); free(zc); free(A); free(tmp); free(B);
    return ORC_OK;
}

/* Zonal retention (Sec. 4.1): keep the first r zig-zag coefficients of every
 * block.  Compact output out[blk][0..r-1]. */
int orc_zonal(int n, const double *coef, long nblk, int r, double *out)
{
    if (r < 0 || r > n * n) return ORC_ERR_ARG;
    for (long b = 0; b < nblk; b++)
        for (int k = 0; k < r; k++) out[b * r + k] = coef[b * n * n + k];
    return ORC_OK;
}

/* Inverse 2-D transform from the first r zig-zag coefficients of each block
 * (zero elsewhere): A' = Minv B' Minv^T with Minv = M^{-1} computed here by
 * Gauss-Jordan.  recon is (H x W) doubles with row stride ldr. */
int orc_inverse(int n, const double *M, const double *zcoef, int r, int H, int W,
                double *recon, long ldr)
{
    if (!orc_shape_ok(n, H, W, ldr) || r < 0 || r > n * n) return ORC_ERR_ARG;
    double *Minv = (double *)malloc(sizeof(double) * n * n);
    if (orc_invert(n, M, Minv) != ORC_OK) { free(Minv); return ORC_ERR_SINGULAR; }
    int bw = W / n, bh = H / n;
    int *zr = (int *)malloc(sizeof(int) * n * n), *zc = (int *)malloc(sizeof(int) * n * n);
    orc_zigzag(n, zr, zc);
    double *B = (double *)malloc(sizeof(double) * n * n), *tmp = (double *)malloc(sizeof(double) * n * n);
    double *A = (double *)malloc(sizeof(double) * n * n);
    for (int by = 0; by < bh; by++)
        for (int bx = 0; bx < bw; bx++) {
            const double *z = zcoef + ((long)by * bw + bx) * r;
            for (int k = 0; k < n * n; k++) B[k] = 0.0;
            for (int k = 0; k < r; k++) B[zr[k] * n + zc[k]] = z[k];
            orc_block_inverse(n, Minv, B, tmp, A);
            for (int k = 0; k < n; k++)
                for (int l = 0; l < n; l++)
                    recon[((long)by * n + k) * ldr + (long)bx * n + l] = A[k * n + l];
        }
    free(Minv); free(zr); free(zc); free(B); free(tmp); free(A);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Quality (Sec. 4.1, Table 3)                                              */
/* ------------------------------------------------------------------------ */

/* Sum of squared errors between the original bytes and a real-valued
 * reconstruction. */
double orc_sse(const uint8_t *img, long ld, const double *recon, long ldr, int H, int W)
{
    double sse = 0.0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double e = (double)img[(long)y * ld + x] - recon[(long)y * ldr + x];
            sse += e * e;
        }
    return sse;
}

/* PSNR = 10 log10(255^2 / MSE), MSE = SSE / (H W); +inf when SSE = 0. */
double orc_psnr(double sse, int H, int W)
{
    double mse = sse / ((double)H * (double)W);
    if (mse == 0.0) return INFINITY;
    return 10.0 * log10(255.0 * 255.0 / mse);
}

/* Rounded, clipped 8-bit reconstruction: clip(floor(x + 1/2), 0, 255). */
void orc_recon_u8(const double *recon, long ldr, int H, int W, uint8_t *out, long ldo)
{
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double v = floor(recon[(long)y * ldr + x] + 0.5);
            if (v < 0.0) v = 0.0;
            if (v > 255.0) v = 255.0;
            out[(long)y * ldo + x] = (uint8_t)v;
        }
}

/* Whole path for one image, block by block: forward with M, zonal r, inverse,
 * SSE.  Optional outputs (NULL to skip): compact coefficients [nblk][r] and the
 * real-valued reconstruction (H x W, stride W).  Blocks are split over OpenMP
 * threads; each block's arithmetic is the same as orc_forward/orc_inverse and
 * the per-block squared errors are summed in block order, so the result does
 * not depend on the thread count.  Returns the SSE (negative on error). */
double orc_pipeline(int n, const double *M, const uint8_t *img, int H, int W, long ld, int r,
                    double *zcoef_out, double *recon_out, int nthreads)
{
    if (!orc_shape_ok(n, H, W, ld) || r < 0 || r > n * n) return -1.0;
    double *Minv = (double *)malloc(sizeof(double) * n * n);
    if (orc_invert(n, M, Minv) != ORC_OK) { free(Minv); return -2.0; }
    int bw = W / n, bh = H / n;
    long nblk = (long)bw * bh;
    int *zr = (int *)malloc(sizeof(int) * n * n), *zc = (int *)malloc(sizeof(int) * n * n);
    orc_zigzag(n, zr, zc);
    double *blk_sse = (double *)malloc(sizeof(double) * (nblk > 0 ? nblk : 1));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *A = (double *)malloc(sizeof(double) * n * n);
        double *B = (double *)malloc(sizeof(double) * n * n);
        double *Bz = (double *)malloc(sizeof(double) * n * n);
        double *tmp = (double *)malloc(sizeof(double) * n * n);
        double *Ar = (double *)malloc(sizeof(double) * n * n);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (long b = 0; b < nblk; b++) {
            int by = (int)(b / bw), bx = (int)(b % bw);
            for (int k = 0; k < n; k++)
                for (int l = 0; l < n; l++)
                    A[k * n + l] = img[((long)by * n + k) * ld + (long)bx * n + l];
            orc_block_forward(n, M, A, tmp, B);
            for (int k = 0; k < n * n; k++) Bz[k] = 0.0;
            for (int k = 0; k < r; k++) {
                Bz[zr[k] * n + zc[k]] = B[zr[k] * n + zc[k]];
                if (zcoef_out) zcoef_out[b * r + k] = B[zr[k] * n + zc[k]];
            }
            orc_block_inverse(n, Minv, Bz, tmp, Ar);
            double s = 0.0;
            for (int k = 0; k < n; k++)
                for (int l = 0; l < n; l++) {
                    double e = A[k * n + l] - Ar[k * n + l];
                    s += e * e;
                    if (recon_out) recon_out[((long)by * n + k) * W + (long)bx * n + l] = Ar[k * n + l];
                }
            blk_sse[b] = s;
        }
        free(A); free(B); free(Bz); free(tmp); free(Ar);
    }
    double sse = 0.0;
    for (long b = 0; b < nblk; b++) sse += blk_sse[b];
    free(blk_sse); free(Minv); free(zr); free(zc);
    return sse;
}

/* JPEG-like quantisation with S absorbed (Appendix, Eq. bbar and the identity
 * below it): Bbar = round(B / Q) = round(C / Qtilde) with C = T A T^T (exact
 * integers), B = R o C, R = s s^T, Qtilde = Q / R.  round(x) = floor(x + 1/2)
 * (the paper's rounding, Eq. 2).  The decoder dequantises B' = Bbar o Q, keeps
 * the first r zig-zag positions, and reconstructs A' = That^{-1} B' That^{-T}.
 *
 * Floating point decides the integer Bbar, so this function takes that decision
 * in binary32 exactly as specified for the kernel: w_ij = fl32(s_i s_j / Q_ij)
 * (the FP64 quotient rounded once), q = fl32(fl32(C_ij) * w_ij), Bbar =
 * floor(q + 1/2) (exact for |q| < 2^22).  Everything after Bbar is FP64.
 * Outputs: qcoef_out [nblk][r] int32 (zig-zag order), recon_out H x W FP64
 * (either may be NULL).  Returns the SSE of the FP64 reconstruction, < 0 on
 * bad arguments. */
double orc_quant_pipeline(int n, const int *T, const double *s, const double *Q, const uint8_t *img, int H,
                          int W, long ld, int r, int32_t *qcoef_out, double *recon_out)
{
    if (!orc_shape_ok(n, H, W, ld) || r < 0 || r > n * n) return -1.0;
    for (int k = 0; k < n * n; k++)
        if (!(Q[k] > 0.0)) return -1.0;
    double *That = (double *)malloc(sizeof(double) * n * n);
    double *Tinv = (double *)malloc(sizeof(double) * n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) That[i * n + j] = s[i] * T[i * n + j];
    if (orc_invert(n, That, Tinv) != ORC_OK) { free(That); free(Tinv); return -2.0; }
    float *w = (float *)malloc(sizeof(float) * n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) w[i * n + j] = (float)(s[i] * s[j] / Q[i * n + j]);
    int *zr = (int *)malloc(sizeof(int) * n * n), *zc = (int *)malloc(sizeof(int) * n * n);
    orc_zigzag(n, zr, zc);
    int bw = W / n, bh = H / n;
    long nblk = (long)bw * bh;
    int64_t *C = (int64_t *)malloc(sizeof(int64_t) * (nblk > 0 ? nblk : 1) * n * n);
    orc_int_stage(n, T, img, H, W, ld, C);
    double *Bp = (double *)malloc(sizeof(double) * n * n);
    double *tmp = (double *)malloc(sizeof(double) * n * n);
    double *Ar = (double *)malloc(sizeof(double) * n * n);
    double sse = 0.0;
    for (long b = 0; b < nblk; b++) {
        int by = (int)(b / bw), bx = (int)(b % bw);
        const int64_t *c = C + b * n * n;
        for (int k = 0; k < n * n; k++) Bp[k] = 0.0;
        for (int k = 0; k < r; k++) {
            int i = zr[k], j = zc[k];
            float q = (float)c[i * n + j] * w[i * n + j];
            int32_t qb = (int32_t)floorf(q + 0.5f);
            if (qcoef_out) qcoef_out[b * r + k] = qb;
            Bp[i * n + j] = (double)qb * Q[i * n + j];
        }
        orc_block_inverse(n, Tinv, Bp, tmp, Ar);
        for (int k = 0; k < n; k++)
            for (int l = 0; l < n; l++) {
                double e = (double)img[((long)by * n + k) * ld + (long)bx * n + l] - Ar[k * n + l];
                sse += e * e;
                if (recon_out) recon_out[((long)by * n + k) * W + (long)bx * n + l] = Ar[k * n + l];
            }
    }
    free(That); free(Tinv); free(w); free(zr); free(zc); free(C); free(Bp); free(tmp); free(Ar);
    return sse;
}

/* Mean structural similarity (MSSIM), the quality measure of Sec. 4.1 (Wang et
 * al. 2004): for every position where an 11 x 11 window fits, with Gaussian
 * weights w (sigma = 1.5, normalised to sum 1) over the window,
 *   mu_x = sum w x,  sigma_x^2 = sum w (x - mu_x)^2,  sigma_xy = sum w (x - mu_x)(y - mu_y)
 *   SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2))
 * with C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2; MSSIM = the mean over the
 * (H - 10) x (W - 10) positions.  Written as the direct definition (each window
 * summed explicitly, deviations from the window mean), FP64.  Returns NaN when the
 * image is smaller than the window.  map_out: (H - 10) x (W - 10) or NULL. */
double orc_mssim(const uint8_t *x, long ldx, const uint8_t *y, long ldy, int H, int W, double *map_out)
{
    const int R = 5, S = 11;
    if (H < S || W < S) return NAN;
    double w[11][11], tot = 0.0;
    for (int i = 0; i < S; i++)
        for (int j = 0; j < S; j++) {
            double di = i - R, dj = j - R;
            w[i][j] = exp(-(di * di + dj * dj) / (2.0 * 1.5 * 1.5));
            tot += w[i][j];
        }
    for (int i = 0; i < S; i++)
        for (int j = 0; j < S; j++) w[i][j] /= tot;
    const double C1 = (0.01 * 255.0) * (0.01 * 255.0), C2 = (0.03 * 255.0) * (0.03 * 255.0);
    const int OH = H - S + 1, OW = W - S + 1;
    double sum = 0.0;
    for (int r = 0; r < OH; r++)
        for (int c = 0; c < OW; c++) {
            double mx = 0.0, my = 0.0;
            for (int i = 0; i < S; i++)
                for (int j = 0; j < S; j++) {
                    mx += w[i][j] * x[(long)(r + i) * ldx + c + j];
                    my += w[i][j] * y[(long)(r + i) * ldy + c + j];
                }
            double vx = 0.0, vy = 0.0, cxy = 0.0;
            for (int i = 0; i < S; i++)
                for (int j = 0; j < S; j++) {
                    double dx = x[(long)(r + i) * ldx + c + j] - mx, dy = y[(long)(r + i) * ldy + c + j] - my;
                    vx += w[i][j] * dx * dx;
                    vy += w[i][j] * dy * dy;
                    cxy += w[i][j] * dx * dy;
                }
            double v = (2.0 * mx * my + C1) * (2.0 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2));
            if (map_out) map_out[(long)r * OW + c] = v;
            sum += v;
        }
    return sum / ((double)OH * OW);
}

/* Number of OpenMP threads a parallel region uses (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Figures of merit (Sec. 3.1)                                              */
/* ------------------------------------------------------------------------ */

/* Unified coding gain: Cg = 10 log10 prod_k (A_k B_k)^(-1/N), with
 * A_k = su((h_k^T h_k) o R), h_k the k-th row of That, and B_k = ||g_k||^2,
 * g_k the k-th row of That^{-1} (as printed). */
int orc_coding_gain(int n, double rho, const double *That, double *cg)
{
    double *R = (double *)malloc(sizeof(double) * n * n);
    double *Ti = (double *)malloc(sizeof(double) * n * n);
    orc_markov_autocorr(n, rho, R);
    if (orc_invert(n, That, Ti) != ORC_OK) { free(R); free(Ti); return ORC_ERR_SINGULAR; }
    double logsum = 0.0;
    for (int k = 0; k < n; k++) {
        double Ak = 0.0, Bk = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) Ak += That[k * n + i] * That[k * n + j] * R[i * n + j];
        for (int j = 0; j < n; j++) Bk += Ti[k * n + j] * Ti[k * n + j];
        logsum += log10(1.0 / pow(Ak * Bk, 1.0 / n));
    }
    *cg = 10.0 * logsum;
    free(R); free(Ti);
    return ORC_OK;
}

/* Transform efficiency: eta = 100 sum_i |r_ii| / sum_ij |r_ij|, r = That R That^T. */
void orc_transform_efficiency(int n, double rho, const double *That, double *eta)
{
    double *R = (double *)malloc(sizeof(double) * n * n);
    double *t = (double *)malloc(sizeof(double) * n * n);
    orc_markov_autocorr(n, rho, R);
    double diag = 0.0, all = 0.0;
    for (int i = 0; i < n; i++)
        for (int l = 0; l < n; l++) {
            double acc = 0.0;
            for (int k = 0; k < n; k++) acc += That[i * n + k] * R[k * n + l];
            t[i * n + l] = acc;
        }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double acc = 0.0;
            for (int l = 0; l < n; l++) acc += t[i * n + l] * That[j * n + l];
            all += fabs(acc);
            if (i == j) diag += fabs(acc);
        }
    *eta = 100.0 * diag / all;
    free(R); free(t);
}

/* MSE to the exact KLT: (1/N) tr{(K - That) R (K - That)^T}. */
void orc_mse_to_klt(int n, double rho, const double *K, const double *That, double *mse)
{
    double *R = (double *)malloc(sizeof(double) * n * n);
    double *D = (double *)malloc(sizeof(double) * n * n);
    orc_markov_autocorr(n, rho, R);
    for (int i = 0; i < n * n; i++) D[i] = K[i] - That[i];
    double tr = 0.0;
    for (int i = 0; i < n; i++)
        for (int k = 0; k < n; k++)
            for (int l = 0; l < n; l++) tr += D[i * n + k] * R[k * n + l] * D[i * n + l];
    *mse = tr / n;
    free(R); free(D);
}

/* Total error energy: eps = pi ||K - That||_F^2. */
void orc_total_error_energy(int n, const double *K, const double *That, double *eps)
{
    double acc = 0.0;
    for (int i = 0; i < n * n; i++) acc += (K[i] - That[i]) * (K[i] - That[i]);
    *eps = ORC_PI * acc;
}
