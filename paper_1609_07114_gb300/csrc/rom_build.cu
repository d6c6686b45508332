// Reduced-model construction on the host, FP64 (runs once per region).
//
// Sec. II: the fine-region equations (Eqs. (3)-(5)) as the descriptor system
//   (R + F) x^{n+1} = (R - F) x^n + B u^{n+1/2},  y^n = L^T x^n   (Eq. (6))
// with x = [E; H], R = [[D_eps/dt, -K/2], [-K^T/2, D_mu/dt]],
// F = [[D_sigma/2, -K/2], [K^T/2, 0]], boundary E edges on half cells
// (Eq. (4)), B = L S_hat with S_hat = diag(-dx, +dx, +dy, -dy) over the
// South, North, West, East ports (Eq. (25)).
// Sec. III: SPRIM -- a block-Krylov basis of ((psi0 R + F)^{-1} R,
// (psi0 R + F)^{-1} B B_in) split into E rows (V1) and H rows (V2), each
// orthonormalised; the reduced blocks follow by congruence (Eq. (12)).
// Block Arnoldi keeps, per block, the left singular vectors above a relative
// deflation tolerance, in decreasing order; a block truncated to fit the
// order q/2 is cut at a singular-value gap so that the subspace is unique.
// Sec. V-E: if a singular value s_k of R11^{-1/2} K~ R22^{-1/2} exceeds
// gamma * 2/dt (Eq. (27)) it is clamped there and K~ is rebuilt.
//
// The Krylov operator is applied by eliminating E (a diagonal block) and
// solving the remaining 5-point system on Hz,
//   S_H = psi0 D_mu/dt + (1 - psi0^2)/4 K^T A11^{-1} K,  A11 = psi0 D_eps/dt + D_sigma/2,
// with a banded Cholesky factorisation (bandwidth = fine cells per row).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>

#include <nvtx3/nvToolsExt.h>

#include "internal.hpp"

namespace {

using la::Mat;

struct FineSys {
  int nxf = 0, nyf = 0, nEx = 0, nEy = 0, nE = 0, nH = 0, nu = 0;
  double dxf = 0, dyf = 0;
  std::vector<double> d_eps, d_sig, d_mu;
  // K (nE x nH): every E row holds at most two entries.
  std::vector<int> k_h[2];
  std::vector<double> k_v[2];
  // K^T: every H column holds exactly four entries (e index, value).
  std::vector<int> kt_e[4];
  std::vector<double> kt_v[4];
  std::vector<int> port_row;     // E index of port p
  std::vector<double> S_hat;     // Eq. (25)
};

FineSys assemble(int nxf, int nyf, double dxf, double dyf, const double* eps_r,
                 const double* sigma) {
  using fdtdrom::kEps0;
  using fdtdrom::kMu0;
  FineSys f;
  f.nxf = nxf, f.nyf = nyf, f.dxf = dxf, f.dyf = dyf;
  f.nEx = nxf * (nyf + 1);
  f.nEy = (nxf + 1) * nyf;
  f.nE = f.nEx + f.nEy;
  f.nH = nxf * nyf;
  f.nu = 2 * (nxf + nyf);
  f.d_eps.assign(f.nE, 0.0);
  f.d_sig.assign(f.nE, 0.0);
  f.d_mu.assign(f.nH, dxf * dyf * kMu0);
  for (int s = 0; s < 2; ++s) {
    f.k_h[s].assign(f.nE, -1);
    f.k_v[s].assign(f.nE, 0.0);
  }
  for (int s = 0; s < 4; ++s) {
    f.kt_e[s].assign(f.nH, 0);
    f.kt_v[s].assign(f.nH, 0.0);
  }
  auto cell = [&](const double* a, int ih, int jh) { return a[(size_t)jh * nxf + ih]; };
  const double area = dxf * dyf;
  // Ex(ih, jh): Eq. (3) inside, half cell on the South/North boundary (Eq. (4)).
  for (int jh = 0; jh <= nyf; ++jh) {
    for (int ih = 0; ih < nxf; ++ih) {
      const int e = jh * nxf + ih;
      double ep, sg, ar;
      if (jh == 0) {
        ep = cell(eps_r, ih, 0), sg = cell(sigma, ih, 0), ar = area / 2;
      } else if (jh == nyf) {
        ep = cell(eps_r, ih, nyf - 1), sg = cell(sigma, ih, nyf - 1), ar = area / 2;
      } else {
        ep = 0.5 * (cell(eps_r, ih, jh - 1) + cell(eps_r, ih, jh));
        sg = 0.5 * (cell(sigma, ih, jh - 1) + cell(sigma, ih, jh));
        ar = area;
      }
      f.d_eps[e] = ar * kEps0 * ep;
      f.d_sig[e] = ar * sg;
      if (jh < nyf) { f.k_h[0][e] = jh * nxf + ih; f.k_v[0][e] = +dxf; }        // Hz above
      if (jh > 0) { f.k_h[1][e] = (jh - 1) * nxf + ih; f.k_v[1][e] = -dxf; }   // Hz below
    }
  }
  // Ey(ih, jh): half cell on the West/East boundary.
  for (int jh = 0; jh < nyf; ++jh) {
    for (int ih = 0; ih <= nxf; ++ih) {
      const int e = f.nEx + jh * (nxf + 1) + ih;
      double ep, sg, ar;
      if (ih == 0) {
        ep = cell(eps_r, 0, jh), sg = cell(sigma, 0, jh), ar = area / 2;
      } else if (ih == nxf) {
        ep = cell(eps_r, nxf - 1, jh), sg = cell(sigma, nxf - 1, jh), ar = area / 2;
      } else {
        ep = 0.5 * (cell(eps_r, ih - 1, jh) + cell(eps_r, ih, jh));
        sg = 0.5 * (cell(sigma, ih - 1, jh) + cell(sigma, ih, jh));
        ar = area;
      }
      f.d_eps[e] = ar * kEps0 * ep;
      f.d_sig[e] = ar * sg;
      if (ih < nxf) { f.k_h[0][e] = jh * nxf + ih; f.k_v[0][e] = -dyf; }        // Hz right
      if (ih > 0) { f.k_h[1][e] = jh * nxf + ih - 1; f.k_v[1][e] = +dyf; }      // Hz left
    }
  }
  // K^T columns: Hz(ih, jh) touches Ex below/above and Ey left/right.
  for (int jh = 0; jh < nyf; ++jh) {
    for (int ih = 0; ih < nxf; ++ih) {
      const int h = jh * nxf + ih;
      f.kt_e[0][h] = jh * nxf + ih;              f.kt_v[0][h] = +dxf;  // Ex below: +dx Hz above it
      f.kt_e[1][h] = (jh + 1) * nxf + ih;        f.kt_v[1][h] = -dxf;  // Ex above
      f.kt_e[2][h] = f.nEx + jh * (nxf + 1) + ih;     f.kt_v[2][h] = -dyf;  // Ey left
      f.kt_e[3][h] = f.nEx + jh * (nxf + 1) + ih + 1; f.kt_v[3][h] = +dyf;  // Ey right
    }
  }
  // Ports in the order S, N, W, E (Eq. (8)); B = L S_hat (Eq. (24c)).
  f.port_row.resize(f.nu);
  f.S_hat.resize(f.nu);
  int p = 0;
  for (int ih = 0; ih < nxf; ++ih, ++p) f.port_row[p] = ih, f.S_hat[p] = -dxf;
  for (int ih = 0; ih < nxf; ++ih, ++p) f.port_row[p] = nyf * nxf + ih, f.S_hat[p] = +dxf;
  for (int jh = 0; jh < nyf; ++jh, ++p) f.port_row[p] = f.nEx + jh * (nxf + 1), f.S_hat[p] = +dyf;
  for (int jh = 0; jh < nyf; ++jh, ++p) f.port_row[p] = f.nEx + jh * (nxf + 1) + nxf, f.S_hat[p] = -dyf;
  return f;
}

// K h for one vector.
void k_apply(const FineSys& f, const double* h, double* out) {
  for (int e = 0; e < f.nE; ++e) {
    double s = 0.0;
    for (int t = 0; t < 2; ++t)
      if (f.k_h[t][e] >= 0) s += f.k_v[t][e] * h[f.k_h[t][e]];
    out[e] = s;
  }
}

// K^T e for one vector.
void kt_apply(const FineSys& f, const double* e, double* out) {
  for (int h = 0; h < f.nH; ++h) {
    double s = 0.0;
    for (int t = 0; t < 4; ++t) s += f.kt_v[t][h] * e[f.kt_e[t][h]];
    out[h] = s;
  }
}

// Solver for (psi0 R + F) x = b by elimination of E (module header).
struct PencilSolver {
  const FineSys& f;
  double psi0, dt;
  std::vector<double> a11;   // psi0 D_eps/dt + D_sig/2
  la::Band S;
  PencilSolver(const FineSys& fs, double psi, double dtb)
      : f(fs), psi0(psi), dt(dtb), a11(fs.nE), S(fs.nH, fs.nxf) {
    for (int e = 0; e < f.nE; ++e) a11[e] = psi0 * f.d_eps[e] / dt + f.d_sig[e] / 2;
    const double c1 = (1.0 - psi0 * psi0) / 4.0;
    for (int h = 0; h < f.nH; ++h) S.at(h, h) += psi0 * f.d_mu[h] / dt;
    for (int e = 0; e < f.nE; ++e) {
      for (int s = 0; s < 2; ++s) {
        const int hs = f.k_h[s][e];
        if (hs < 0) continue;
        for (int t = 0; t < 2; ++t) {
          const int ht = f.k_h[t][e];
          if (ht < 0 || ht > hs) continue;
          S.at(hs, ht) += c1 * f.k_v[s][e] * f.k_v[t][e] / a11[e];
        }
      }
    }
  }
  bool factor() { return S.cholesky(); }
  // x = [e; h] <- (psi0 R + F)^{-1} [f; g], in place on one column of length nE + nH.
  void solve(double* x) const {
    std::vector<double> t(f.nE), w(f.nH), kh(f.nE);
    for (int e = 0; e < f.nE; ++e) t[e] = x[e] / a11[e];
    kt_apply(f, t.data(), w.data());
    double* h = x + f.nE;
    for (int i = 0; i < f.nH; ++i) h[i] -= 0.5 * (1.0 - psi0) * w[i];
    S.solve(h);
    k_apply(f, h, kh.data());
    for (int e = 0; e < f.nE; ++e) x[e] = t[e] + 0.5 * (psi0 + 1.0) * kh[e] / a11[e];
  }
};

// R x for one column (R at time step dt).
void r_apply(const FineSys& f, double dt, const double* x, double* out) {
  std::vector<double> kh(f.nE), kte(f.nH);
  k_apply(f, x + f.nE, kh.data());
  kt_apply(f, x, kte.data());
  for (int e = 0; e < f.nE; ++e) out[e] = f.d_eps[e] / dt * x[e] - 0.5 * kh[e];
  for (int h = 0; h < f.nH; ++h) out[f.nE + h] = -0.5 * kte[h] + f.d_mu[h] / dt * x[f.nE + h];
}

// Applies op column by column: Y = op(X); X, Y are N x m row-major.
template <class Op>
Mat apply_cols(const Mat& X, Op op) {
  const int N = X.r, m = X.c;
  Mat Y(N, m);
  std::vector<double> col(N), out(N);
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < N; ++i) col[i] = X(i, j);
    op(col.data(), out.data());
    for (int i = 0; i < N; ++i) Y(i, j) = out[i];
  }
  return Y;
}

double spectral_norm(const Mat& W) {
  if (W.r == 0 || W.c == 0) return 0.0;
  Mat U, V;
  std::vector<double> s;
  la::svd(W, U, s, V);
  return s.empty() ? 0.0 : s[0];
}

// Orthonormal columns spanning range(X) above tol * s_max (decreasing s).
Mat orth(const Mat& X, double tol) {
  Mat U, V;
  std::vector<double> s;
  la::svd(X, U, s, V);
  int keep = 0;
  if (!s.empty() && s[0] > 0.0)
    while (keep < (int)s.size() && s[keep] > tol * s[0]) ++keep;
  return la::cols(U, 0, keep);
}

Mat diag_congruence(const Mat& V, const std::vector<double>& d) {  // V^T diag(d) V
  Mat DV = V;
  for (int i = 0; i < V.r; ++i)
    for (int j = 0; j < V.c; ++j) DV(i, j) *= d[i];
  return la::matmul_tn(V, DV);
}

bool is_diagonal(const Mat& A) {
  for (int i = 0; i < A.r; ++i)
    for (int j = 0; j < A.c; ++j)
      if (i != j && A(i, j) != 0.0) return false;
  return true;
}

Mat spd_pow(const Mat& A, double p) {
  if (is_diagonal(A)) {
    Mat B(A.r, A.c);
    for (int i = 0; i < A.r; ++i) B(i, i) = std::pow(A(i, i), p);
    return B;
  }
  return la::sym_pow(A, p);
}

// The part of a build after the congruences (m->R11, Sig, R22, Kt set):
// port blocks, Eq. (27) and the report.
rom_build_report finish_model(rom_model* m, const FineSys& f, const rom_desc* d, int n_inputs) {
  const Mat& V1 = m->V1;
  m->LE = Mat(m->qE, f.nu);
  m->BE = Mat(m->qE, f.nu);
  for (int p = 0; p < f.nu; ++p)
    for (int i = 0; i < m->qE; ++i) {
      m->LE(i, p) = V1(f.port_row[p], i);
      m->BE(i, p) = V1(f.port_row[p], i) * f.S_hat[p];
    }
  // Sec. V-E: singular values of R11^{-1/2} K~ R22^{-1/2} (Eq. (27)).
  const Mat r11m = spd_pow(m->R11, -0.5), r22m = spd_pow(m->R22, -0.5);
  const Mat M = la::matmul(la::matmul(r11m, m->Kt), r22m);
  Mat U, Wt;
  std::vector<double> s;
  la::svd(M, U, s, Wt);
  const double lim = 2.0 / d->dt;
  rom_build_report r{};
  r.qE = m->qE, r.qH = m->qH, r.n_inputs = n_inputs;
  r.smax_before = s.empty() ? 0.0 : s[0] / lim;
  r.smax_after = r.smax_before;
  if (d->gamma > 0 && !s.empty() && s[0] > d->gamma * lim) {
    std::vector<double> sc = s;
    for (auto& v : sc)
      if (v > d->gamma * lim) v = d->gamma * lim, ++r.n_clamped;
    Mat US = U;
    for (int i = 0; i < US.r; ++i)
      for (int j = 0; j < US.c; ++j) US(i, j) *= sc[j];
    const Mat Mc = la::matmul_nt(US, Wt);
    m->Kt = la::matmul(la::matmul(spd_pow(m->R11, 0.5), Mc), spd_pow(m->R22, 0.5));
    r.smax_after = sc[0] / lim;
  }
  // Eq. (26a) at the run dt, Eq. (26c).
  {
    const int q = m->qE + m->qH;
    Mat R(q, q);
    for (int i = 0; i < m->qE; ++i)
      for (int j = 0; j < m->qE; ++j) R(i, j) = m->R11(i, j) / d->dt;
    for (int i = 0; i < m->qH; ++i)
      for (int j = 0; j < m->qH; ++j) R(m->qE + i, m->qE + j) = m->R22(i, j) / d->dt;
    for (int i = 0; i < m->qE; ++i)
      for (int j = 0; j < m->qH; ++j) R(i, m->qE + j) = R(m->qE + j, i) = -0.5 * m->Kt(i, j);
    if (q <= 1200) {
      std::vector<double> w;
      Mat Qe;
      la::eig_sym(R, w, Qe);
      r.min_eig_R = w.empty() ? 0.0 : w[0] / std::fabs(w.back());
    } else {
      r.min_eig_R = la::chol_ok(R) ? 1.0 : -1.0;  // sign only for very large models
    }
    double num = 0.0, den = 0.0;
    for (int i = 0; i < m->qE; ++i)
      for (int p = 0; p < f.nu; ++p) {
        const double dv = m->BE(i, p) - m->LE(i, p) * f.S_hat[p];
        num += dv * dv;
        den += m->BE(i, p) * m->BE(i, p);
      }
    r.cond3_residual = den > 0 ? std::sqrt(num / den) : 0.0;
  }
  return r;
}


#include "rom_build_gpu.cuh"

}  // namespace

namespace {

// gpu: the Krylov basis and the Eq. (12) blocks on the device (stream st).
int rom_build_impl(const rom_desc* d, rom_model** out, rom_build_report* rep, bool gpu, cudaStream_t st) {
  using fdtdrom::set_global_error;
  if (!d || !out) return set_global_error(FDTD_EINVAL, "rom_build: null argument");
  if (d->a < 1 || d->b < 1 || d->r < 1 || !(d->dx > 0) || !(d->dy > 0) || !(d->dt > 0) ||
      !d->eps_r || !d->sigma || d->q < 0 || (d->q % 2) != 0 ||
      (d->rule != FDTD_RULE_DUAL && d->rule != FDTD_RULE_PAPER))
    return set_global_error(FDTD_EINVAL, "rom_build: malformed descriptor (q must be even)");
  const int nxf = d->r * d->a, nyf = d->r * d->b;
  for (int k = 0; k < nxf * nyf; ++k)
    if (!(d->eps_r[k] > 0.0) || !(d->sigma[k] >= 0.0))
      return set_global_error(FDTD_EINVAL, "rom_build: eps_r must be > 0 and sigma >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  rom_model* m = new (std::nothrow) rom_model();
  if (!m) return set_global_error(FDTD_ENOMEM, "rom_build: out of host memory");
  static std::atomic<long long> next_id{1};
  m->id = next_id++;
  try {
    const double dxf = d->dx / d->r, dyf = d->dy / d->r;
    FineSys f = assemble(nxf, nyf, dxf, dyf, d->eps_r, d->sigma);
    m->a = d->a, m->b = d->b, m->r = d->r, m->dx = d->dx, m->dy = d->dy, m->dt = d->dt;
    m->rule = d->rule, m->nxf = nxf, m->nyf = nyf, m->nE = f.nE, m->nH = f.nH, m->nu = f.nu;
    m->S_hat = f.S_hat;
    const double tol = d->defl_tol > 0 ? d->defl_tol : 1e-12;
    const int N = f.nE + f.nH;
    Mat V1, V2;
    int n_inputs = 0;
    if (d->q == 0) {
      if (N > 6000) {
        delete m;
        return set_global_error(FDTD_EINVAL, "rom_build: full order (q = 0) limited to 6000 unknowns");
      }
      V1 = la::eye(f.nE);
      V2 = la::eye(f.nH);
    } else {
      // Krylov operator at dt_b = min(dt, 0.99 * Eq. (1) limit of the fine mesh).
      const double c0 = 1.0 / std::sqrt(fdtdrom::kEps0 * fdtdrom::kMu0);
      const double dt_fine = 1.0 / (c0 * std::sqrt(1.0 / (dxf * dxf) + 1.0 / (dyf * dyf)));
      const double dt_b = std::fmin(d->dt, 0.99 * dt_fine);
      const double psi0 = std::tan(M_PI * d->f0 * dt_b);
      if (!(psi0 > 0.0) || !(psi0 < 1.0)) {
        delete m;
        return set_global_error(FDTD_EINVAL, "rom_build: f0 must give 0 < tan(pi f0 dt) < 1");
      }
      PencilSolver ps(f, psi0, dt_b);
      if (!ps.factor()) {
        delete m;
        return set_global_error(FDTD_ENOTPASSIVE, "rom_build: Krylov pencil not positive definite");
      }
      // Start block (psi0 R + F)^{-1} B B_in: B_in = I (paper) or T (dual).
      const bool dual = d->rule == FDTD_RULE_DUAL;
      n_inputs = dual ? 2 * (d->a + d->b) : f.nu;
      Mat W(N, n_inputs);
      for (int p = 0; p < f.nu; ++p) {
        int col = p;
        if (dual) {
          if (p < nxf) col = p / d->r;
          else if (p < 2 * nxf) col = d->a + (p - nxf) / d->r;
          else if (p < 2 * nxf + nyf) col = 2 * d->a + (p - 2 * nxf) / d->r;
          else col = 2 * d->a + d->b + (p - 2 * nxf - nyf) / d->r;
        }
        W(f.port_row[p], col) += f.S_hat[p];
      }
      if (gpu) {
        gpu_blocks(f, ps, psi0, dt_b, W, d->q / 2, tol, st, m);
        rom_build_report r = finish_model(m, f, d, n_inputs);
        r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        m->rep = r;
        if (rep) *rep = r;
        *out = m;
        return FDTD_OK;
      }
      auto pencil_inv = [&](const double* x, double* y) {
        std::memcpy(y, x, sizeof(double) * N);
        ps.solve(y);
      };
      W = apply_cols(W, pencil_inv);
      auto krylov_op = [&](const double* x, double* y) {
        r_apply(f, dt_b, x, y);
        ps.solve(y);
      };
      // Block Arnoldi with SVD deflation (Sec. III).
      const int k = d->q / 2;
      Mat Q(N, 0);
      while (Q.c < k) {
        const double ref = spectral_norm(W);
        if (!(ref > 0.0)) break;
        for (int pass = 0; pass < 2 && Q.c > 0; ++pass) {
          Mat C = la::matmul_tn(Q, W);
          Mat QC = la::matmul(Q, C);
          for (size_t t = 0; t < W.a.size(); ++t) W.a[t] -= QC.a[t];
        }
        Mat U, Vs;
        std::vector<double> s;
        la::svd(W, U, s, Vs);
        int keep = 0;
        while (keep < (int)s.size() && s[keep] > tol * ref) ++keep;
        if (keep == 0) break;
        int take = std::min(keep, k - Q.c);
        // A truncated block is cut at a singular-value gap (relative 1e-8) so
        // that the kept subspace is unique even for symmetric regions.
        const bool truncated = take < keep;
        if (truncated) {
          while (take > 0 && s[take - 1] - s[take] <= 1e-8 * s[take - 1]) --take;
          if (take == 0) break;
        }
        Mat Ub = la::cols(U, 0, take);
        Mat Qn(N, Q.c + take);
        for (int i = 0; i < N; ++i) {
          for (int j = 0; j < Q.c; ++j) Qn(i, j) = Q(i, j);
          for (int j = 0; j < take; ++j) Qn(i, Q.c + j) = Ub(i, j);
        }
        Q = Qn;
        if (truncated) break;
        if (Q.c < k) W = apply_cols(Ub, krylov_op);
      }
      V1 = orth(la::rows(Q, 0, f.nE), tol);
      V2 = orth(la::rows(Q, f.nE, N), tol);
    }
    m->qE = V1.c;
    m->qH = V2.c;
    // Congruence, Eq. (12).
    m->R11 = diag_congruence(V1, f.d_eps);
    m->Sig = diag_congruence(V1, f.d_sig);
    m->R22 = diag_congruence(V2, f.d_mu);
    {
      Mat KV2(f.nE, V2.c);
      std::vector<double> col(f.nH), kc(f.nE);
      for (int j = 0; j < V2.c; ++j) {
        for (int i = 0; i < f.nH; ++i) col[i] = V2(i, j);
        k_apply(f, col.data(), kc.data());
        for (int i = 0; i < f.nE; ++i) KV2(i, j) = kc[i];
      }
      m->Kt = la::matmul_tn(V1, KV2);
    }
    m->V1 = V1;
    m->V2 = V2;
    rom_build_report r = finish_model(m, f, d, n_inputs);
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    m->rep = r;
    if (rep) *rep = r;
  } catch (const std::bad_alloc&) {
    delete m;
    return set_global_error(FDTD_ENOMEM, "rom_build: out of host or device memory");
  } catch (const std::runtime_error& e) {
    delete m;
    return set_global_error(FDTD_ECUDA, e.what());
  }
  *out = m;
  return FDTD_OK;
}

}  // namespace

extern "C" int rom_build(const rom_desc* d, rom_model** out, rom_build_report* rep) {
  nvtxRangePushA("rom_build");
  const int rc = rom_build_impl(d, out, rep, false, nullptr);
  nvtxRangePop();
  return rc;
}

extern "C" int rom_build_gpu(const rom_desc* d, void* cuda_stream, rom_model** out, rom_build_report* rep) {
  nvtxRangePushA("rom_build_gpu");
  const int rc = rom_build_impl(d, out, rep, true, static_cast<cudaStream_t>(cuda_stream));
  nvtxRangePop();
  return rc;
}

extern "C" void rom_free(rom_model* m) { delete m; }

extern "C" int rom_get_info(const rom_model* m, int* qE, int* qH, int* nu) {
  if (!m) return fdtdrom::set_global_error(FDTD_EINVAL, "rom_get_info: null model");
  if (qE) *qE = m->qE;
  if (qH) *qH = m->qH;
  if (nu) *nu = m->nu;
  return FDTD_OK;
}

extern "C" int rom_get_blocks(const rom_model* m, double* R11, double* R22, double* Kt,
                              double* Sig, double* LE) {
  if (!m) return fdtdrom::set_global_error(FDTD_EINVAL, "rom_get_blocks: null model");
  auto put = [](const la::Mat& A, double* dst) {
    if (dst) std::memcpy(dst, A.a.data(), sizeof(double) * A.a.size());
  };
  put(m->R11, R11);
  put(m->R22, R22);
  put(m->Kt, Kt);
  put(m->Sig, Sig);
  put(m->LE, LE);
  return FDTD_OK;
}

extern "C" int rom_get_basis(const rom_model* m, int* nE, int* nH, double* V1, double* V2) {
  if (!m) return fdtdrom::set_global_error(FDTD_EINVAL, "rom_get_basis: null model");
  if (nE) *nE = m->V1.r;
  if (nH) *nH = m->V2.r;
  if (V1) std::memcpy(V1, m->V1.a.data(), sizeof(double) * m->V1.a.size());
  if (V2) std::memcpy(V2, m->V2.a.data(), sizeof(double) * m->V2.a.size());
  return FDTD_OK;
}
