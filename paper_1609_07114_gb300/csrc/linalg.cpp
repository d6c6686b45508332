// Dense FP64 host linear algebra (see linalg.hpp).
#include "linalg.hpp"

#include <algorithm>
#include <numeric>

namespace la {

Mat eye(int n) {
  Mat I(n, n);
  for (int i = 0; i < n; ++i) I(i, i) = 1.0;
  return I;
}

Mat transpose(const Mat& A) {
  Mat T(A.c, A.r);
  for (int i = 0; i < A.r; ++i)
    for (int j = 0; j < A.c; ++j) T(j, i) = A(i, j);
  return T;
}

Mat matmul(const Mat& A, const Mat& B) {
  Mat C(A.r, B.c);
  for (int i = 0; i < A.r; ++i) {
    double* ci = C.row(i);
    const double* ai = A.row(i);
    for (int k = 0; k < A.c; ++k) {
      const double aik = ai[k];
      if (aik == 0.0) continue;
      const double* bk = B.row(k);
      for (int j = 0; j < B.c; ++j) ci[j] += aik * bk[j];
    }
  }
  return C;
}

Mat matmul_tn(const Mat& A, const Mat& B) {
  Mat C(A.c, B.c);
  for (int k = 0; k < A.r; ++k) {
    const double* ak = A.row(k);
    const double* bk = B.row(k);
    for (int i = 0; i < A.c; ++i) {
      const double aki = ak[i];
      if (aki == 0.0) continue;
      double* ci = C.row(i);
      for (int j = 0; j < B.c; ++j) ci[j] += aki * bk[j];
    }
  }
  return C;
}

Mat matmul_nt(const Mat& A, const Mat& B) {
  Mat C(A.r, B.r);
  for (int i = 0; i < A.r; ++i) {
    const double* ai = A.row(i);
    for (int j = 0; j < B.r; ++j) {
      const double* bj = B.row(j);
      double s = 0.0;
      for (int k = 0; k < A.c; ++k) s += ai[k] * bj[k];
      C(i, j) = s;
    }
  }
  return C;
}

Mat cols(const Mat& A, int c0, int c1) {
  Mat B(A.r, c1 - c0);
  for (int i = 0; i < A.r; ++i)
    for (int j = c0; j < c1; ++j) B(i, j - c0) = A(i, j);
  return B;
}

Mat rows(const Mat& A, int r0, int r1) {
  Mat B(r1 - r0, A.c);
  std::copy(A.a.begin() + (size_t)r0 * A.c, A.a.begin() + (size_t)r1 * A.c, B.a.begin());
  return B;
}

double norm_fro(const Mat& A) {
  double s = 0.0;
  for (double v : A.a) s += v * v;
  return std::sqrt(s);
}

// Householder QR on a column-major copy.
void qr_thin(const Mat& A, Mat& Q, Mat& R) {
  const int m = A.r, n = A.c;
  std::vector<double> W((size_t)m * n);  // column-major
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) W[(size_t)j * m + i] = A(i, j);
  std::vector<double> beta(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double* x = &W[(size_t)k * m];
    double sig = 0.0;
    for (int i = k + 1; i < m; ++i) sig += x[i] * x[i];
    const double x0 = x[k];
    if (sig == 0.0) {  // already upper triangular in this column
      beta[k] = 0.0;
      continue;
    }
    const double mu = std::sqrt(x0 * x0 + sig);
    const double v0 = (x0 <= 0.0) ? x0 - mu : -sig / (x0 + mu);
    beta[k] = 2.0 * v0 * v0 / (sig + v0 * v0);
    for (int i = k + 1; i < m; ++i) x[i] /= v0;  // v = [1; x[k+1:]]
    x[k] = mu;                                   // H x = mu e_k
    for (int j = k + 1; j < n; ++j) {
      double* y = &W[(size_t)j * m];
      double s = y[k];
      for (int i = k + 1; i < m; ++i) s += x[i] * y[i];
      s *= beta[k];
      y[k] -= s;
      for (int i = k + 1; i < m; ++i) y[i] -= s * x[i];
    }
  }
  R = Mat(n, n);
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) R(i, j) = W[(size_t)j * m + i];
  // Q = H_0 H_1 ... H_{n-1} [I_n; 0], accumulated backwards (column-major).
  std::vector<double> Qc((size_t)m * n, 0.0);
  for (int j = 0; j < n; ++j) Qc[(size_t)j * m + j] = 1.0;
  for (int k = n - 1; k >= 0; --k) {
    if (beta[k] == 0.0) continue;
    const double* x = &W[(size_t)k * m];
    for (int j = k; j < n; ++j) {
      double* y = &Qc[(size_t)j * m];
      double s = y[k];
      for (int i = k + 1; i < m; ++i) s += x[i] * y[i];
      s *= beta[k];
      y[k] -= s;
      for (int i = k + 1; i < m; ++i) y[i] -= s * x[i];
    }
  }
  Q = Mat(m, n);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) Q(i, j) = Qc[(size_t)j * m + i];
}

// One-sided Jacobi on a square or tall matrix with few columns (Hestenes).
static void svd_jacobi(const Mat& A, Mat& U, std::vector<double>& s, Mat& V) {
  const int m = A.r, n = A.c;
  std::vector<double> W((size_t)m * n), Vc((size_t)n * n, 0.0);  // column-major
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) W[(size_t)j * m + i] = A(i, j);
  for (int j = 0; j < n; ++j) Vc[(size_t)j * n + j] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double* wp = &W[(size_t)p * m];
        double* wq = &W[(size_t)q * m];
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < m; ++i) {
          alpha += wp[i] * wp[i];
          beta += wq[i] * wq[i];
          gamma += wp[i] * wq[i];
        }
        if (gamma == 0.0) continue;
        const double rel = std::fabs(gamma) / std::sqrt(alpha * beta);
        off = std::max(off, rel);
        if (rel < 1e-15) continue;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          const double a = wp[i], b = wq[i];
          wp[i] = cs * a - sn * b;
          wq[i] = sn * a + cs * b;
        }
        double* vp = &Vc[(size_t)p * n];
        double* vq = &Vc[(size_t)q * n];
        for (int i = 0; i < n; ++i) {
          const double a = vp[i], b = vq[i];
          vp[i] = cs * a - sn * b;
          vq[i] = sn * a + cs * b;
        }
      }
    }
    if (off < 1e-15) break;
  }
  std::vector<double> nrm(n);
  for (int j = 0; j < n; ++j) {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += W[(size_t)j * m + i] * W[(size_t)j * m + i];
    nrm[j] = std::sqrt(t);
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  U = Mat(m, n);
  V = Mat(n, n);
  s.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    const int j = ord[k];
    s[k] = nrm[j];
    const double inv = nrm[j] > 0.0 ? 1.0 / nrm[j] : 0.0;
    for (int i = 0; i < m; ++i) U(i, k) = W[(size_t)j * m + i] * inv;
    for (int i = 0; i < n; ++i) V(i, k) = Vc[(size_t)j * n + i];
  }
}

void svd(const Mat& A, Mat& U, std::vector<double>& s, Mat& V) {
  if (A.r < A.c) {
    Mat Ut, Vt;
    svd(transpose(A), Ut, s, Vt);
    U = Vt;
    V = Ut;
    return;
  }
  if (A.r > A.c) {
    Mat Q, R, Ur;
    qr_thin(A, Q, R);
    svd_jacobi(R, Ur, s, V);
    U = matmul(Q, Ur);
    return;
  }
  svd_jacobi(A, U, s, V);
}

void eig_sym(const Mat& A0, std::vector<double>& w, Mat& Q) {
  const int n = A0.r;
  Mat A = A0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) A(i, j) = A(j, i) = 0.5 * (A0(i, j) + A0(j, i));
  Q = eye(n);
  double scale = 0.0;
  for (double v : A.a) scale = std::max(scale, std::fabs(v));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) off = std::max(off, std::fabs(A(p, q)));
    if (off <= 1e-16 * scale || scale == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A(p, q);
        if (std::fabs(apq) <= 1e-18 * scale) continue;
        const double theta = (A(q, q) - A(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(1.0 + theta * theta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A(k, p), akq = A(k, q);
          A(k, p) = c * akp - s * akq;
          A(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A(p, k), aqk = A(q, k);
          A(p, k) = c * apk - s * aqk;
          A(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q(k, p), qkq = Q(k, q);
          Q(k, p) = c * qkp - s * qkq;
          Q(k, q) = s * qkp + c * qkq;
        }
      }
    }
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return A(x, x) < A(y, y); });
  Mat Qs(n, n);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    w[k] = A(ord[k], ord[k]);
    for (int i = 0; i < n; ++i) Qs(i, k) = Q(i, ord[k]);
  }
  Q = Qs;
}

Mat sym_pow(const Mat& A, double p) {
  std::vector<double> w;
  Mat Q;
  eig_sym(A, w, Q);
  const int n = A.r;
  Mat QW(n, n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) QW(i, k) = Q(i, k) * std::pow(w[k], p);
  return matmul_nt(QW, Q);
}

bool lu_factor(Mat& A, std::vector<int>& piv) {
  const int n = A.r;
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A(k, k));
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A(i, k)) > best) best = std::fabs(A(i, k)), p = i;
    piv[k] = p;
    if (best == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
    const double inv = 1.0 / A(k, k);
    for (int i = k + 1; i < n; ++i) {
      const double l = (A(i, k) *= inv);
      if (l == 0.0) continue;
      double* ai = A.row(i);
      const double* ak = A.row(k);
      for (int j = k + 1; j < n; ++j) ai[j] -= l * ak[j];
    }
  }
  return true;
}

void lu_solve(const Mat& LU, const std::vector<int>& piv, Mat& B) {
  const int n = LU.r, m = B.c;
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int j = 0; j < m; ++j) std::swap(B(k, j), B(piv[k], j));
  for (int i = 0; i < n; ++i) {
    double* bi = B.row(i);
    for (int k = 0; k < i; ++k) {
      const double l = LU(i, k);
      if (l == 0.0) continue;
      const double* bk = B.row(k);
      for (int j = 0; j < m; ++j) bi[j] -= l * bk[j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double* bi = B.row(i);
    for (int k = i + 1; k < n; ++k) {
      const double u = LU(i, k);
      if (u == 0.0) continue;
      const double* bk = B.row(k);
      for (int j = 0; j < m; ++j) bi[j] -= u * bk[j];
    }
    const double inv = 1.0 / LU(i, i);
    for (int j = 0; j < m; ++j) bi[j] *= inv;
  }
}

bool chol_ok(const Mat& A) {
  const int n = A.r;
  Mat L(n, n);
  for (int j = 0; j < n; ++j) {
    double d = 0.5 * (A(j, j) + A(j, j));
    for (int k = 0; k < j; ++k) d -= L(j, k) * L(j, k);
    if (!(d > 0.0)) return false;
    L(j, j) = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = 0.5 * (A(i, j) + A(j, i));
      for (int k = 0; k < j; ++k) s -= L(i, k) * L(j, k);
      L(i, j) = s / L(j, j);
    }
  }
  return true;
}

bool Band::cholesky() {
  for (int i = 0; i < n; ++i) {
    const int j0 = std::max(0, i - bw);
    for (int j = j0; j <= i; ++j) {
      double s = at(i, j);
      const int k0 = std::max(j0, j - bw);
      for (int k = k0; k < j; ++k) s -= at(i, k) * at(j, k);
      if (i == j) {
        if (!(s > 0.0)) return false;
        at(i, i) = std::sqrt(s);
      } else {
        at(i, j) = s / at(j, j);
      }
    }
  }
  return true;
}

void Band::solve(double* x) const {
  auto L = [&](int i, int j) { return a[(size_t)i * (bw + 1) + (i - j)]; };
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int k = std::max(0, i - bw); k < i; ++k) s -= L(i, k) * x[k];
    x[i] = s / L(i, i);
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k <= std::min(n - 1, i + bw); ++k) s -= L(k, i) * x[k];
    x[i] = s / L(i, i);
  }
}

}  // namespace la
