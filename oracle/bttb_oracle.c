/*
 * CPU oracle for the two-level block-Toeplitz MoM matrix (test
 * infrastructure only: the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it; the solver library never links or calls it).
 *
 * Everything here is the plain definition, in IEEE binary64, with no FFT,
 * no blocking and no reordering of the sums beyond the definition itself.
 *
 * Matrix definition (paper Sec. II-A, Eq. (Tblock) with L = 2):
 *   the top level (rows of the array, N[2] = ny) is block Toeplitz with
 *   blocks R_{m-n}; each R is itself block Toeplitz over the cells of a row
 *   (N[1] = nx) with unstructured b x b blocks (N[0] = b).  Hence
 *     Z[(m*b + p), (n*b + q)] = T[ix_m - ix_n, iy_m - iy_n][p][q],
 *   where cell m = iy_m*nx + ix_m.  The generator table is
 *     gen[((j + ny - 1)*(2nx - 1) + (i + nx - 1))*b*b + p*b + q] = T[i,j][p][q].
 * Complex numbers are stored interleaved (re, im).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

static inline cplx gen_at(const cplx *gen, int nx, int ny, int b, int i, int j, int p, int q)
{
    long blk = (long)(j + ny - 1) * (2 * nx - 1) + (i + nx - 1);
    return gen[blk * b * b + (long)p * b + q];
}

/* Dense assembly of Z (row-major, N x N), Eq. (Tblock) for L = 2. */
void oracle_assemble(int nx, int ny, int b, const double *gen_d, double *z_d)
{
    const cplx *gen = (const cplx *)gen_d;
    cplx *z = (cplx *)z_d;
    long n = (long)nx * ny * b;
    for (int iym = 0; iym < ny; ++iym)
        for (int ixm = 0; ixm < nx; ++ixm)
            for (int p = 0; p < b; ++p) {
                long row = ((long)iym * nx + ixm) * b + p;
                for (int iyn = 0; iyn < ny; ++iyn)
                    for (int ixn = 0; ixn < nx; ++ixn)
                        for (int q = 0; q < b; ++q) {
                            long col = ((long)iyn * nx + ixn) * b + q;
                            z[row * n + col] = gen_at(gen, nx, ny, b, ixm - ixn, iym - iyn, p, q);
                        }
            }
}

/* One output row of the product y = Z x, summed in the definition's order. */
static cplx row_product(const cplx *gen, int nx, int ny, int b, long row, const cplx *x)
{
    int p = (int)(row % b);
    long m = row / b;
    int ixm = (int)(m % nx), iym = (int)(m / nx);
    cplx acc = 0.0;
    for (int iyn = 0; iyn < ny; ++iyn)
        for (int ixn = 0; ixn < nx; ++ixn) {
            long base = ((long)iyn * nx + ixn) * b;
            for (int q = 0; q < b; ++q)
                acc += gen_at(gen, nx, ny, b, ixm - ixn, iym - iyn, p, q) * x[base + q];
        }
    return acc;
}

/*
 * Brute-force O(N^2) product streamed from the generator table:
 *   y[:, c] = Z x[:, c] for c < nrhs, column c of x at x + c*ldx.
 * Rows are independent, so they are shared out over OpenMP threads; each
 * row's sum keeps the definition's order.
 */
void oracle_matvec(int nx, int ny, int b, const double *gen_d,
                   const double *x_d, long ldx, double *y_d, long ldy, int nrhs)
{
    const cplx *gen = (const cplx *)gen_d;
    long n = (long)nx * ny * b;
    for (int c = 0; c < nrhs; ++c) {
        const cplx *x = (const cplx *)x_d + (long)c * ldx;
        cplx *y = (cplx *)y_d + (long)c * ldy;
#pragma omp parallel for schedule(static)
        for (long row = 0; row < n; ++row)
            y[row] = row_product(gen, nx, ny, b, row, x);
    }
}

/* Selected rows of Z x (for sampled checks at sizes where a full product is slow). */
void oracle_matvec_rows(int nx, int ny, int b, const double *gen_d, const double *x_d,
                        const long *rows, int nrows, double *out_d)
{
    const cplx *gen = (const cplx *)gen_d;
    const cplx *x = (const cplx *)x_d;
    cplx *out = (cplx *)out_d;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nrows; ++k)
        out[k] = row_product(gen, nx, ny, b, rows[k], x);
}

/*
 * Dense complex LU with partial pivoting, in place on the row-major n x n
 * matrix a, then forward/back substitution on the n x nrhs right-hand side
 * rhs (row-major, overwritten by the solution).  Returns 0, or k+1 if the
 * k-th pivot is exactly zero.  Textbook Doolittle elimination (the "mld"
 * direct reference of the paper's comparisons).
 */
int oracle_lu_solve(int n, double *a_d, double *rhs_d, int nrhs)
{
    cplx *a = (cplx *)a_d;
    cplx *r = (cplx *)rhs_d;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = cabs(a[(long)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = cabs(a[(long)i * n + k]);
            if (v > best) { best = v; piv = i; }
        }
        if (best == 0.0) return k + 1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                cplx t = a[(long)k * n + j]; a[(long)k * n + j] = a[(long)piv * n + j]; a[(long)piv * n + j] = t;
            }
            for (int j = 0; j < nrhs; ++j) {
                cplx t = r[(long)k * nrhs + j]; r[(long)k * nrhs + j] = r[(long)piv * nrhs + j]; r[(long)piv * nrhs + j] = t;
            }
        }
        cplx d = a[(long)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            cplx l = a[(long)i * n + k] / d;
            a[(long)i * n + k] = l;
            for (int j = k + 1; j < n; ++j) a[(long)i * n + j] -= l * a[(long)k * n + j];
            for (int j = 0; j < nrhs; ++j) r[(long)i * nrhs + j] -= l * r[(long)k * nrhs + j];
        }
    }
    for (int k = n - 1; k >= 0; --k)
        for (int j = 0; j < nrhs; ++j) {
            cplx s = r[(long)k * nrhs + j];
            for (int i = k + 1; i < n; ++i) s -= a[(long)k * n + i] * r[(long)i * nrhs + j];
            r[(long)k * nrhs + j] = s / a[(long)k * n + k];
        }
    return 0;
}

/*
 * Naive DFT of length n, X[k] = sum_t x[t] exp(sign * 2 pi i k t / n),
 * accumulated in long double with the angle reduced exactly as (k*t mod n).
 * sign = -1 is the forward transform the paper uses (MATLAB fft).
 */
void oracle_dft(int n, const double *x_d, double *out_d, int sign)
{
    const cplx *x = (const cplx *)x_d;
    cplx *out = (cplx *)out_d;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int k = 0; k < n; ++k) {
        long double re = 0.0L, im = 0.0L;
        for (int t = 0; t < n; ++t) {
            long kt = ((long)k * t) % n;
            long double ang = (long double)sign * two_pi * (long double)kt / (long double)n;
            long double c = cosl(ang), s = sinl(ang);
            long double xr = creal(x[t]), xi = cimag(x[t]);
            re += xr * c - xi * s;
            im += xr * s + xi * c;
        }
        out[k] = (double)re + I * (double)im;
    }
}
