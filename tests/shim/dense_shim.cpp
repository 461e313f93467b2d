// Test-only C shim over the engine's host linear algebra (paper_0707_0131_gb300/csrc/dense.cpp),
// compiled with g++ by tests/test_host_dense.py so that it can be checked without a GPU.
#include <complex>

#include "dense.h"

using eig::dense::cd;

extern "C" {
void shim_herm_eig_lowest(int n, const cd *A, int k, double *w, cd *Y) { eig::dense::herm_eig_lowest(n, A, k, w, Y); }
void shim_window_lowest(int m, const cd *T, int kh, int n, int k, double *w, cd *Y) {
    eig::dense::window_lowest(m, T, kh, n, k, w, Y);
}
int shim_restart_coefficients(int m, const cd *T, int kh, int nev, double drop, cd *QZ, double *M) {
    return eig::dense::restart_coefficients(m, T, kh, nev, drop, QZ, M);
}
int shim_cholesky_solve(int n, cd *H, cd *B, int nrhs) {
    if (!eig::dense::cholesky(n, H)) return 0;
    eig::dense::chol_solve(n, H, B, nrhs);
    return 1;
}
int shim_lu_solve(int n, cd *A, cd *B, int nrhs) { return eig::dense::lu_solve(n, A, B, nrhs) ? 1 : 0; }
int shim_orth_columns(int n, int c, cd *X, double drop, int *keep) { return eig::dense::orth_columns(n, c, X, drop, keep); }
void shim_tridiag_eig(int n, const double *d, const double *e, int lo, int hi, double *w, double *Z) {
    eig::dense::tridiag_eig(n, d, e, lo, hi, w, Z);
}
}
