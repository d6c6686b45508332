// Coupling of a reduced model to the coarse grid (host, FP64).
//
// Sec. IV, Eqs. (13)-(23).  For every coarse interface edge k (ordered S, N,
// W, E like the ports of Eq. (8)) the coarse half-cell update of Eq. (14) is
//   dplus_k y_k^{n+1} = dminus_k y_k^n + g_k h_k^{n+1/2} - g_k U_k^{n+1/2},
// dplus/dminus = Dl Dl' (Deps_b/dt +- Dsig_b/2) with the material of the
// coarse cell just outside, g = Dl G^T with the local curl sign per side
// (S -1, N +1, W +1, E -1), so that Dl G^T = T^T S_hat T and the interface
// is lossless.  The reduced model (Eq. (11)) is
//   G x~^{n+1} = (R~ - F~) x~^n + B~ u_hat,   G = R~ + F~.
// Eliminating the hanging variables gives the explicit map of Eq. (23):
//   [y; x~]^{n+1} = P [y; x~]^n + Q h^{n+1/2}.
//
// Paper rule (Eqs. (15)-(16)): T y^{n+1} = L~^T x~^{n+1}, U = (1/r) T^T u_hat.
//   With a = 1/dplus:  y+ = a(dminus y + g h) - a g (1/r) T^T u_hat,
//   x~+ = M x~ + Nb u_hat  (M = G^{-1}(R~-F~), Nb = G^{-1} B~), and
//   [T diag(a g / r) T^T + L~^T Nb] u_hat = T a (dminus y + g h) - L~^T M x~.
//   The n_u x n_u matrix may be singular (reduced order below the port
//   count); it is solved with an SVD-based generalised inverse, and the
//   consistency of the solution is checked.  If the interface cannot carry
//   any field (y rows of P and Q vanish) the embedding is rejected.
// Dual rule: y = (1/r) T^T L~^T x~, u_hat = T U.
//   U solves [diag(a g) + C Nd] U = a dminus y + a g h - C M x~,
//   C = (1/r) T^T L~^T, Nd = G^{-1} B~ T  (n_y x n_y, nonsingular).
#include <algorithm>
#include <cmath>

#include "internal.hpp"

namespace fdtdrom {

using la::Mat;

InterfaceDesc make_interface(int i0, int j0, int a, int b, double dx, double dy, double dt,
                             const double* eps_r, const double* sigma, int nx) {
  InterfaceDesc d;
  auto add = [&](int comp, int ei, int ej, int hi, int hj, double sign, double len,
                 double half) {
    const double e = kEps0 * eps_r[(size_t)hj * nx + hi];
    const double s = sigma[(size_t)hj * nx + hi];
    d.comp.push_back(comp), d.ei.push_back(ei), d.ej.push_back(ej);
    d.hi.push_back(hi), d.hj.push_back(hj);
    d.dplus.push_back(len * half * (e / dt + s / 2));
    d.dminus.push_back(len * half * (e / dt - s / 2));
    d.dlg.push_back(sign * len);
  };
  for (int i = i0; i < i0 + a; ++i) add(0, i, j0, i, j0 - 1, -1.0, dx, dy / 2);      // S
  for (int i = i0; i < i0 + a; ++i) add(0, i, j0 + b, i, j0 + b, +1.0, dx, dy / 2);  // N
  for (int j = j0; j < j0 + b; ++j) add(1, i0, j, i0 - 1, j, +1.0, dy, dx / 2);      // W
  for (int j = j0; j < j0 + b; ++j) add(1, i0 + a, j, i0 + a, j, -1.0, dy, dx / 2);  // E
  d.ny = (int)d.comp.size();
  return d;
}

namespace {

// Coarse interface edge of fine port p (the T of Eq. (15)).
int port_edge(const rom_model& m, int p) {
  const int nxf = m.nxf, nyf = m.nyf, r = m.r, a = m.a, b = m.b;
  if (p < nxf) return p / r;
  if (p < 2 * nxf) return a + (p - nxf) / r;
  if (p < 2 * nxf + nyf) return 2 * a + (p - 2 * nxf) / r;
  return 2 * a + b + (p - 2 * nxf - nyf) / r;
}

}  // namespace

int couple(const rom_model& m, const InterfaceDesc& itf, double dt, Mat& P, Mat& Q,
           std::string& msg) {
  const int qE = m.qE, qH = m.qH, q = qE + qH, ny = itf.ny, nu = m.nu;
  // G = R~ + F~ and R~ - F~ (Eq. (12) with F~ = [[Sig/2, -Kt/2], [Kt^T/2, 0]]).
  Mat G(q, q), RmF(q, q);
  for (int i = 0; i < qE; ++i)
    for (int j = 0; j < qE; ++j) {
      G(i, j) = m.R11(i, j) / dt + m.Sig(i, j) / 2;
      RmF(i, j) = m.R11(i, j) / dt - m.Sig(i, j) / 2;
    }
  for (int i = 0; i < qH; ++i)
    for (int j = 0; j < qH; ++j) G(qE + i, qE + j) = RmF(qE + i, qE + j) = m.R22(i, j) / dt;
  for (int i = 0; i < qE; ++i)
    for (int j = 0; j < qH; ++j) {
      G(i, qE + j) = -m.Kt(i, j);
      RmF(qE + j, i) = -m.Kt(i, j);
    }
  // Eq. (26a) at this dt.
  {
    Mat R(q, q);
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) R(i, j) = 0.5 * (G(i, j) + RmF(i, j));
    for (int i = 0; i < qE; ++i)
      for (int j = 0; j < qH; ++j) R(i, qE + j) = R(qE + j, i) = -0.5 * m.Kt(i, j);
    if (!la::chol_ok(R)) {
      msg = "reduced model is not passive at this time step (R~ not positive definite)";
      return FDTD_ENOTPASSIVE;
    }
  }
  std::vector<int> piv;
  Mat Glu = G;
  if (!la::lu_factor(Glu, piv)) {
    msg = "R~ + F~ is singular";
    return FDTD_ESINGULAR;
  }
  Mat M = RmF;
  la::lu_solve(Glu, piv, M);  // M = G^{-1}(R~ - F~)
  std::vector<double> a(ny), ag(ny), ad(ny);
  for (int k = 0; k < ny; ++k) {
    a[k] = 1.0 / itf.dplus[k];
    ag[k] = a[k] * itf.dlg[k];
    ad[k] = a[k] * itf.dminus[k];
  }
  const int n = ny + q;
  P = Mat(n, n);
  Q = Mat(n, ny);
  if (m.rule == FDTD_RULE_DUAL) {
    Mat BT(q, ny);  // B~ T
    for (int p = 0; p < nu; ++p) {
      const int k = port_edge(m, p);
      for (int i = 0; i < qE; ++i) BT(i, k) += m.BE(i, p);
    }
    Mat Nd = BT;
    la::lu_solve(Glu, piv, Nd);  // G^{-1} B~ T  (q x ny)
    Mat C(ny, q);                // (1/r) T^T L~^T
    for (int p = 0; p < nu; ++p) {
      const int k = port_edge(m, p);
      for (int i = 0; i < qE; ++i) C(k, i) += m.LE(i, p) / m.r;
    }
    Mat S = la::matmul(C, Nd);
    for (int k = 0; k < ny; ++k) S(k, k) += ag[k];
    // U = S^{-1} [diag(ad) y + diag(ag) h - C M x~]
    Mat rhs(ny, ny + ny + q);
    for (int k = 0; k < ny; ++k) {
      rhs(k, k) = ad[k];
      rhs(k, ny + k) = ag[k];
    }
    const Mat CM = la::matmul(C, M);
    for (int k = 0; k < ny; ++k)
      for (int j = 0; j < q; ++j) rhs(k, 2 * ny + j) = -CM(k, j);
    std::vector<int> pv;
    Mat Slu = S;
    if (!la::lu_factor(Slu, pv)) {
      msg = "dual-rule interface system is singular";
      return FDTD_ESINGULAR;
    }
    Mat Uop = rhs;
    la::lu_solve(Slu, pv, Uop);  // U = Uop [y; h; x~]
    // y+ = ad y + ag h - ag U ;  x~+ = M x~ + Nd U
    const Mat NU = la::matmul(Nd, Uop);
    for (int k = 0; k < ny; ++k) {
      for (int j = 0; j < ny; ++j) {
        P(k, j) = (k == j ? ad[k] : 0.0) - ag[k] * Uop(k, j);
        Q(k, j) = (k == j ? ag[k] : 0.0) - ag[k] * Uop(k, ny + j);
      }
      for (int j = 0; j < q; ++j) P(k, ny + j) = -ag[k] * Uop(k, 2 * ny + j);
    }
    for (int i = 0; i < q; ++i) {
      for (int j = 0; j < ny; ++j) {
        P(ny + i, j) = NU(i, j);
        Q(ny + i, j) = NU(i, ny + j);
      }
      for (int j = 0; j < q; ++j) P(ny + i, ny + j) = M(i, j) + NU(i, 2 * ny + j);
    }
    return FDTD_OK;
  }
  // Paper rule.
  Mat Bf(q, nu);
  for (int i = 0; i < qE; ++i)
    for (int p = 0; p < nu; ++p) Bf(i, p) = m.BE(i, p);
  Mat Nb = Bf;
  la::lu_solve(Glu, piv, Nb);  // G^{-1} B~  (q x nu)
  Mat Sp(nu, nu);              // T diag(a g / r) T^T + L~^T Nb
  for (int p = 0; p < nu; ++p)
    for (int s = 0; s < nu; ++s) {
      double v = 0.0;
      if (port_edge(m, p) == port_edge(m, s)) v += ag[port_edge(m, p)] / m.r;
      for (int i = 0; i < qE; ++i) v += m.LE(i, p) * Nb(i, s);
      Sp(p, s) = v;
    }
  Mat rhs(nu, ny + ny + q);  // columns act on [y; h; x~]
  const Mat LM = [&] {       // L~^T M (nu x q)
    Mat R(nu, q);
    for (int p = 0; p < nu; ++p)
      for (int j = 0; j < q; ++j) {
        double v = 0.0;
        for (int i = 0; i < qE; ++i) v += m.LE(i, p) * M(i, j);
        R(p, j) = v;
      }
    return R;
  }();
  for (int p = 0; p < nu; ++p) {
    const int k = port_edge(m, p);
    rhs(p, k) = ad[k];
    rhs(p, ny + k) = ag[k];
    for (int j = 0; j < q; ++j) rhs(p, 2 * ny + j) = -LM(p, j);
  }
  Mat U, V;
  std::vector<double> s;
  la::svd(Sp, U, s, V);
  const double thr = (s.empty() ? 0.0 : s[0]) * 1e-12;
  const Mat UtR = la::matmul_tn(U, rhs);
  Mat Y(nu, rhs.c);  // u_hat operator = V diag(1/s) U^T rhs
  for (int t = 0; t < (int)s.size(); ++t) {
    if (!(s[t] > thr)) continue;
    const double inv = 1.0 / s[t];
    for (int p = 0; p < nu; ++p) {
      const double vp = V(p, t) * inv;
      if (vp == 0.0) continue;
      for (int j = 0; j < rhs.c; ++j) Y(p, j) += vp * UtR(t, j);
    }
  }
  {  // consistency of the generalised solve
    const Mat SY = la::matmul(Sp, Y);
    double num = 0.0, den = 0.0;
    for (size_t t = 0; t < SY.a.size(); ++t) {
      num += (SY.a[t] - rhs.a[t]) * (SY.a[t] - rhs.a[t]);
      den += rhs.a[t] * rhs.a[t];
    }
    if (!(std::sqrt(num) <= 1e-9 * std::sqrt(den))) {
      msg = "paper-rule coupling system of Eq. (19) is inconsistent";
      return FDTD_ESINGULAR;
    }
  }
  // TtY = (1/r) T^T u_hat operator (ny x cols)
  Mat TtY(ny, rhs.c);
  for (int p = 0; p < nu; ++p) {
    const int k = port_edge(m, p);
    for (int j = 0; j < rhs.c; ++j) TtY(k, j) += Y(p, j) / m.r;
  }
  const Mat NbY = la::matmul(Nb, Y);
  for (int k = 0; k < ny; ++k) {
    for (int j = 0; j < ny; ++j) {
      P(k, j) = (k == j ? ad[k] : 0.0) - ag[k] * TtY(k, j);
      Q(k, j) = (k == j ? ag[k] : 0.0) - ag[k] * TtY(k, ny + j);
    }
    for (int j = 0; j < q; ++j) P(k, ny + j) = -ag[k] * TtY(k, 2 * ny + j);
  }
  for (int i = 0; i < q; ++i) {
    for (int j = 0; j < ny; ++j) {
      P(ny + i, j) = NbY(i, j);
      Q(ny + i, j) = NbY(i, ny + j);
    }
    for (int j = 0; j < q; ++j) P(ny + i, ny + j) = M(i, j) + NbY(i, 2 * ny + j);
  }
  double qmax = 0.0;
  for (int k = 0; k < ny; ++k)
    for (int j = 0; j < ny; ++j) qmax = std::fmax(qmax, std::fabs(Q(k, j)));
  double amax = 0.0;
  for (int k = 0; k < ny; ++k) amax = std::fmax(amax, std::fabs(ag[k]));
  if (qmax < 1e-9 * amax) {
    msg = "paper-rule interface is degenerate: the reduced model cannot match any coarse "
          "interface field (order below the port count); use FDTD_RULE_DUAL";
    return FDTD_ESINGULAR;
  }
  return FDTD_OK;
}

}  // namespace fdtdrom

extern "C" int rom_couple(const rom_model* m, const double* ring_eps_r, const double* ring_sigma,
                          double* P, double* Q) {
  using namespace fdtdrom;
  if (!m || !ring_eps_r || !ring_sigma || !P || !Q)
    return set_global_error(FDTD_EINVAL, "rom_couple: null argument");
  // A (a+2) x (b+2) coarse patch whose ring cells carry the given materials.
  const int a = m->a, b = m->b, nx = a + 2, ny = b + 2;
  std::vector<double> eps((size_t)nx * ny, 1.0), sig((size_t)nx * ny, 0.0);
  InterfaceDesc probe = make_interface(1, 1, a, b, m->dx, m->dy, m->dt, eps.data(), sig.data(), nx);
  for (int k = 0; k < probe.ny; ++k) {
    if (!(ring_eps_r[k] > 0) || !(ring_sigma[k] >= 0))
      return set_global_error(FDTD_EINVAL, "rom_couple: eps_r must be > 0 and sigma >= 0");
    eps[(size_t)probe.hj[k] * nx + probe.hi[k]] = ring_eps_r[k];
    sig[(size_t)probe.hj[k] * nx + probe.hi[k]] = ring_sigma[k];
  }
  InterfaceDesc itf = make_interface(1, 1, a, b, m->dx, m->dy, m->dt, eps.data(), sig.data(), nx);
  la::Mat Pm, Qm;
  std::string msg;
  const int rc = couple(*m, itf, m->dt, Pm, Qm, msg);
  if (rc) return set_global_error(rc, "rom_couple: " + msg);
  std::copy(Pm.a.begin(), Pm.a.end(), P);
  std::copy(Qm.a.begin(), Qm.a.end(), Q);
  return FDTD_OK;
}
