/*
 * Oracle (test infrastructure only): complex FP64 banded LU with partial pivoting
 * and the banded solve with several right-hand sides. Plain unblocked C.
 *
 * The contour method factors T(z_j) at every quadrature point (the "matrix
 * factorizations" whose cost dominates the solvers of Sec. 4, cf. Table 2); the
 * banded LU is the textbook Gaussian elimination restricted to the band.
 *
 * Storage (LAPACK gbtrf convention, column-major, 0-based):
 *   A(i, j) lives at ab[(kl + ku + i - j) + j * ldab], ldab >= 2 kl + ku + 1.
 *   Rows 0 .. kl-1 of the band array are workspace for the fill-in that row
 *   interchanges create (U gets bandwidth kl + ku).
 * Pivot rule: in column j, the row r in [j, min(n-1, j+kl)] maximising
 *   |Re a(r,j)| + |Im a(r,j)|, first index on ties. ipiv[j] = r (0-based).
 * Return: 0, or 1 + (first column with an exactly zero pivot); elimination
 *   continues past a zero pivot (that column is skipped), like gbtrf's info > 0.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>

typedef double _Complex zc;

#define AB(i, j) ab[(size_t)(kv + (i) - (j)) + (size_t)(j) * (size_t)ldab]

int oracle_gbtrf(int n, int kl, int ku, zc *ab, int ldab, int *ipiv) {
    const int kv = kl + ku;
    int info = 0;
    /* the fill-in rows start out as zero */
    for (int j = 0; j < n; ++j)
        for (int r = 0; r < kl; ++r) ab[(size_t)r + (size_t)j * ldab] = 0.0;
    for (int j = 0; j < n; ++j) {
        int last_row = j + kl < n - 1 ? j + kl : n - 1;
        int last_col = j + kv < n - 1 ? j + kv : n - 1;
        int p = j;
        double best = -1.0;
        for (int r = j; r <= last_row; ++r) {
            zc v = AB(r, j);
            double m = fabs(creal(v)) + fabs(cimag(v));
            if (m > best) { best = m; p = r; }
        }
        ipiv[j] = p;
        if (AB(p, j) == 0.0) {
            if (info == 0) info = j + 1;
            continue;
        }
        if (p != j) {
            for (int c = j; c <= last_col; ++c) {
                zc t = AB(j, c);
                AB(j, c) = AB(p, c);
                AB(p, c) = t;
            }
        }
        zc piv = AB(j, j);
        for (int r = j + 1; r <= last_row; ++r) AB(r, j) = AB(r, j) / piv;
        for (int c = j + 1; c <= last_col; ++c) {
            zc u = AB(j, c);
            if (u == 0.0) continue;
            for (int r = j + 1; r <= last_row; ++r) AB(r, c) -= AB(r, j) * u;
        }
    }
    return info;
}

/*
 * Solve A X = B with the factors of oracle_gbtrf. B is n x nrhs column-major with
 * leading dimension ldb, overwritten by X. Forward: row interchanges and unit-lower
 * L column by column; backward: U (bandwidth kl + ku) from the last column up.
 */
void oracle_gbtrs(int n, int kl, int ku, int nrhs, const zc *ab, int ldab, const int *ipiv,
                  zc *b, int ldb) {
    const int kv = kl + ku;
    for (int k = 0; k < nrhs; ++k) {
        zc *x = b + (size_t)k * ldb;
        for (int j = 0; j < n; ++j) {
            int p = ipiv[j];
            if (p != j) { zc t = x[j]; x[j] = x[p]; x[p] = t; }
            int last_row = j + kl < n - 1 ? j + kl : n - 1;
            zc xj = x[j];
            for (int r = j + 1; r <= last_row; ++r) x[r] -= AB(r, j) * xj;
        }
        for (int j = n - 1; j >= 0; --j) {
            x[j] = x[j] / AB(j, j);
            zc xj = x[j];
            int first_row = j - kv > 0 ? j - kv : 0;
            for (int r = first_row; r < j; ++r) x[r] -= AB(r, j) * xj;
        }
    }
}
