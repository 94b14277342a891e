// Lanczos (Gauss) quadrature from CG coefficients, on the host.
//
// Preconditioned CG started from x = 0 on B~ x = L v (M = L L') is Lanczos on
// C = L^-1 B~ L^-T started from v / ||v||; its coefficients give the Lanczos tridiagonal
//   T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},   T_{j,j+1} = sqrt(beta_j)/alpha_j,
// and v' f(C) v is approximated by ||v||^2 sum_i tau_i^2 f(theta_i) over the eigenpairs
// (theta_i, first eigenvector component tau_i) of T (Golub & Meurant; the stochastic Lanczos
// quadrature of Ubaru, Chen & Saad for log det). The eigenpairs come from implicit symmetric
// QR sweeps with Wilkinson shifts (Golub & Van Loan, Matrix Computations, Section 8.3),
// tracking only the first row of the accumulated rotations.
#include <cmath>
#include <vector>

#include "../../include/bfmri.h"

namespace bfmri {

// a (diagonal, m), b (off-diagonal, m-1) are overwritten; q receives the first row of Q.
bool tridiag_eig_first_row(int m, std::vector<double>& a, std::vector<double>& b, std::vector<double>& q) {
  q.assign(m, 0.0);
  if (m <= 0) return true;
  q[0] = 1.0;
  const double eps = 2.220446049250313e-16;
  int hi = m - 1;
  long guard = 0;
  while (hi > 0) {
    if (++guard > 100L * m + 100) return false;
    if (std::fabs(b[hi - 1]) <= eps * (std::fabs(a[hi - 1]) + std::fabs(a[hi]))) {
      b[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(b[lo - 1]) > eps * (std::fabs(a[lo - 1]) + std::fabs(a[lo]))) --lo;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block closer to its last entry
    const double d = 0.5 * (a[hi - 1] - a[hi]);
    const double e = b[hi - 1];
    const double den = d + std::copysign(std::hypot(d, e), d == 0.0 ? 1.0 : d);
    const double mu = a[hi] - e * e / den;
    double x = a[lo] - mu, z = b[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      const double c = r == 0.0 ? 1.0 : x / r;
      const double s = r == 0.0 ? 0.0 : z / r;
      if (k > lo) b[k - 1] = r;
      const double ak = a[k], ak1 = a[k + 1], bk = b[k];
      a[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
      a[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
      b[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
      if (k + 1 < hi) {
        z = s * b[k + 1];       // bulge at (k, k+2)
        b[k + 1] = c * b[k + 1];
        x = b[k];
      }
      const double qk = q[k], qk1 = q[k + 1];
      q[k] = c * qk + s * qk1;
      q[k + 1] = -s * qk + c * qk1;
    }
  }
  return true;
}

}  // namespace bfmri

extern "C" bfmri_status bfmri_lanczos_log_quadrature(int m, const double* cg_alpha,
                                                      const double* cg_beta, double* value) {
  if (m < 1 || !cg_alpha || !value || (m > 1 && !cg_beta)) return BFMRI_ERR_INVALID_ARG;
  std::vector<double> a(m), b(m > 1 ? m - 1 : 1, 0.0), q;
  for (int j = 0; j < m; ++j) {
    if (!(cg_alpha[j] > 0.0)) return BFMRI_ERR_INVALID_ARG;
    a[j] = 1.0 / cg_alpha[j] + (j > 0 ? cg_beta[j - 1] / cg_alpha[j - 1] : 0.0);
    if (j + 1 < m) {
      if (!(cg_beta[j] >= 0.0)) return BFMRI_ERR_INVALID_ARG;
      b[j] = std::sqrt(cg_beta[j]) / cg_alpha[j];
    }
  }
  if (!bfmri::tridiag_eig_first_row(m, a, b, q)) return BFMRI_ERR_NOT_CONVERGED;
  double s = 0.0;
  for (int i = 0; i < m; ++i) {
    if (!(a[i] > 0.0)) return BFMRI_ERR_NOT_SPD;
    s += q[i] * q[i] * std::log(a[i]);
  }
  *value = s;
  return BFMRI_OK;
}
