// Internal host-side structures shared by the library's translation units.
#pragma once

#include <string>
#include <vector>

#include "../../include/fdtd.h"
#include "linalg.hpp"

namespace fdtdrom {

constexpr double kEps0 = 8.8541878128e-12;   // CODATA 2018
constexpr double kMu0 = 1.25663706212e-6;

// Records a message for fdtd_last_error(NULL) and returns code.
int set_global_error(int code, const std::string& msg);

}  // namespace fdtdrom

// A reduced model of one fine region (Sec. III, Eqs. (11)-(12)), FP64.
struct rom_model {
  long long id = 0;                    // unique per build (keys shared couplings)
  int a = 0, b = 0, r = 0;
  double dx = 0, dy = 0, dt = 0;
  int rule = FDTD_RULE_DUAL;
  int nxf = 0, nyf = 0, nE = 0, nH = 0, nu = 0;
  int qE = 0, qH = 0;
  la::Mat R11, R22, Kt, Sig, BE, LE;   // BE, LE: qE x nu
  la::Mat V1, V2;                      // projection bases: nE x qE, nH x qH (Sec. III)
  std::vector<double> S_hat;           // nu, Eq. (25)
  rom_build_report rep{};
};

namespace fdtdrom {

// One side of an embedding (Sec. IV-A, Eq. (14)), ordered S, N, W, E.
struct InterfaceDesc {
  int ny = 0;                      // number of coarse interface edges
  std::vector<int> comp, ei, ej;   // E edge holding y_k
  std::vector<int> hi, hj;         // coarse cell whose Hz is h_k
  std::vector<double> dplus, dminus, dlg;  // Eq. (14) diagonals
};

InterfaceDesc make_interface(int i0, int j0, int a, int b, double dx, double dy, double dt,
                             const double* eps_r, const double* sigma, int nx);

// Run-time map of Eq. (23): [y; x~]^{n+1} = P [y; x~]^n + Q h^{n+1/2}.
// Returns FDTD_OK or FDTD_ESINGULAR / FDTD_ENOTPASSIVE with msg set.
int couple(const rom_model& m, const InterfaceDesc& itf, double dt, la::Mat& P, la::Mat& Q,
           std::string& msg);

}  // namespace fdtdrom
