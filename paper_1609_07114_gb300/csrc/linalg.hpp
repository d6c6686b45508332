// Dense FP64 host linear algebra for the one-time reduced-model build.
//
// Only what the build needs: row-major matrices, products, Householder QR,
// one-sided Jacobi SVD, cyclic Jacobi symmetric eigensolver, LU with partial
// pivoting, and a banded Cholesky factorisation.  Everything is plain C++17
// so that it builds and behaves identically on x86-64 and AArch64.
#pragma once

#include <cmath>
#include <cstddef>
#include <vector>

namespace la {

struct Mat {
  int r = 0, c = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(int rows, int cols) : r(rows), c(cols), a((size_t)rows * cols, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)i * c + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * c + j]; }
  double* row(int i) { return a.data() + (size_t)i * c; }
  const double* row(int i) const { return a.data() + (size_t)i * c; }
};

Mat eye(int n);
Mat transpose(const Mat& A);
Mat matmul(const Mat& A, const Mat& B);          // A B
Mat matmul_tn(const Mat& A, const Mat& B);       // A^T B
Mat matmul_nt(const Mat& A, const Mat& B);       // A B^T
Mat cols(const Mat& A, int c0, int c1);          // A[:, c0:c1]
Mat rows(const Mat& A, int r0, int r1);          // A[r0:r1, :]
double norm_fro(const Mat& A);

// Thin Householder QR of A (m x n, m >= n): A = Q R, Q m x n orthonormal.
void qr_thin(const Mat& A, Mat& Q, Mat& R);

// Thin SVD A = U diag(s) V^T (m x n, any shape), s in decreasing order,
// U m x k, V n x k with k = min(m, n).  Tall inputs go through QR first.
void svd(const Mat& A, Mat& U, std::vector<double>& s, Mat& V);

// Symmetric eigendecomposition A = Q diag(w) Q^T, w increasing.
void eig_sym(const Mat& A, std::vector<double>& w, Mat& Q);

// A^p for symmetric positive definite A.
Mat sym_pow(const Mat& A, double p);

// LU with partial pivoting, in place.  Returns false if a pivot is exactly 0.
bool lu_factor(Mat& A, std::vector<int>& piv);
void lu_solve(const Mat& LU, const std::vector<int>& piv, Mat& B);  // B <- A^{-1} B

// Cholesky of an SPD matrix; returns false if not positive definite.
bool chol_ok(const Mat& A);

// Symmetric positive definite band matrix, lower storage: entry (i, i-d),
// d = 0..bw, stored at a[i*(bw+1) + d].
struct Band {
  int n = 0, bw = 0;
  std::vector<double> a;
  Band(int n_, int bw_) : n(n_), bw(bw_), a((size_t)n_ * (bw_ + 1), 0.0) {}
  double& at(int i, int j) { return a[(size_t)i * (bw + 1) + (i - j)]; }  // i >= j
  bool cholesky();                 // in place: L with A = L L^T
  void solve(double* x) const;     // x <- A^{-1} x using the factor
};

}  // namespace la
