// Host FP64 linear algebra for the small matrices of eigCG and the deflation basis:
// the m x m window projection T (Fig. 1 steps 11.3-11.6), H = U^H A U (Sec. 4 box),
// and the Gram matrices of re-orthogonalisation.  Sizes are at most a few hundred,
// so everything runs on the host CPU between kernel launches.
#pragma once
#include <complex>
#include <vector>

namespace eig {
namespace dense {

using cd = std::complex<double>;

// Householder reduction of Hermitian A (n x n, row-major, overwritten) to a real
// symmetric tridiagonal T = Q^H A Q (diagonal d[n], off-diagonal e[n-1]).  Q is
// returned row-major (n x n); its first column is e_0.
void herm_tridiag(int n, cd *A, double *d, double *e, cd *Q);

// Eigenpairs lo..hi-1 (ascending order) of the real symmetric tridiagonal (d, e):
// eigenvalues by bisection on Sturm counts, eigenvectors by inverse iteration with
// re-orthogonalisation inside clusters.  Z: n x (hi-lo), column-major.
void tridiag_eig(int n, const double *d, const double *e, int lo, int hi, double *w, double *Z);

// k lowest eigenpairs of Hermitian A (n x n row-major): w[k] ascending, Y n x k column-major.
void herm_eig_lowest(int n, const cd *A, int k, double *w, cd *Y);

// The eigCG window projection T (m x m, row-major, Hermitian) whose entries at
// rows/columns >= kh + 1 are tridiagonal and whose first kh rows/columns are a
// diagonal block coupled only to index kh.  Returns the k lowest eigenpairs of the
// leading n x n block (n <= m, n >= kh + 1 or the block is tiny) without a dense
// reduction of the tridiagonal part.  Y: n x k column-major.
void window_lowest(int m, const cd *T, int kh, int n, int k, double *w, cd *Y);

// Fig. 1 steps 11.3-11.6 on the host: Y = nev lowest eigenvectors of T_m, Ybar =
// those of T_{m-1} padded with a zero row, Q = orth([Y Ybar]) (modified Gram-
// Schmidt twice, dropping columns whose remainder is below drop_tol), H = Q^H T Q,
// H Z = Z M.  Outputs QZ (m x r column-major), M[r] ascending; returns r.
int restart_coefficients(int m, const cd *T, int kh, int nev, double drop_tol, cd *QZ, double *M);

// Cholesky H = L L^H in place (lower triangle of row-major H).  false if not HPD.
bool cholesky(int n, cd *L);
// Solves L L^H X = B for nrhs columns (B column-major n x nrhs, overwritten).
void chol_solve(int n, const cd *L, cd *B, int nrhs);

// Solves A X = B by Gaussian elimination with partial pivoting (A n x n row-major,
// overwritten; B column-major n x nrhs, overwritten).  false if A is singular.
bool lu_solve(int n, cd *A, cd *B, int nrhs);

// Orthonormalises the columns of X (n x c column-major) by modified Gram-Schmidt
// applied twice; a column whose norm after projection is below drop_tol times its
// original norm is dropped.  Kept columns are compacted to the front; returns
// their count and writes their original indices to keep (if non-null).
int orth_columns(int n, int c, cd *X, double drop_tol, int *keep);

}  // namespace dense
}  // namespace eig
