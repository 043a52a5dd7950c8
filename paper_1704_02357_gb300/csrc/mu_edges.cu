// Transverse (mu = 0) systematics, Sec. 3.1: the leakage response R(mu) of a mu = 0 spike
// reconstructed from the even multipoles up to l_max (eq. response), and the non-uniform mu
// edges that confine it to the first wedge (eq. nonuniform-bins). Host code, FP64.
#include <cmath>
#include <vector>
#include "pspec.h"

namespace {

// Power-basis coefficients of the Legendre polynomial L_n (c[k] multiplies t^k).
std::vector<double> legendre_coeffs(int n) {
  std::vector<double> p0(n + 2, 0.0), p1(n + 2, 0.0), p2(n + 2, 0.0);
  p0[0] = 1.0;
  if (n == 0) return p0;
  p1[1] = 1.0;
  for (int m = 1; m < n; m++) {  // L_{m+1} = ((2m+1) t L_m - m L_{m-1}) / (m+1)
    for (int k = 0; k <= n + 1; k++) {
      const double tl = k > 0 ? p1[k - 1] : 0.0;
      p2[k] = ((2.0 * m + 1.0) * tl - m * p0[k]) / (m + 1.0);
    }
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

double legendre(int n, double x) {
  if (n == 0) return 1.0;
  double a = 1.0, b = x;
  for (int m = 1; m < n; m++) {
    const double c = ((2.0 * m + 1.0) * x * b - m * a) / (m + 1.0);
    a = b;
    b = c;
  }
  return b;
}

// G(mu) = int_0^mu L_m(t)/t dt for odd m (L_m(t)/t is a polynomial): sum_k c_k mu^k / k.
double g_integral(const std::vector<double>& c, double mu) {
  double s = 0.0;
  for (int k = (int)c.size() - 1; k >= 1; k--) s = s * mu + c[k] / k;
  return s * mu;
}

bool valid_lmax(int ell_max) { return ell_max >= 2 && ell_max <= PSPEC_MAX_ELL && !(ell_max & 1); }

}  // namespace

extern "C" pspec_status pspec_mu_edges_nonuniform(int32_t ell_max, double* mu_edges) {
  if (!mu_edges || !valid_lmax(ell_max)) return PSPEC_EINVAL;
  const std::vector<double> c = legendre_coeffs(ell_max + 1);
  const double g1 = g_integral(c, 1.0);
  auto h = [&](double mu) { return g_integral(c, mu) - g1; };
  // the interior roots of G(mu) = G(1): scan a fine grid for sign changes, then bisect
  const int ngrid = 1 << 16;
  std::vector<double> roots;
  double x0 = 1e-12, h0 = h(x0);
  for (int i = 1; i < ngrid; i++) {
    const double x1 = (double)i / ngrid, h1 = h(x1);
    if (h0 == 0.0) {
      roots.push_back(x0);
    } else if ((h0 < 0.0) != (h1 < 0.0) && h1 != 0.0) {
      double a = x0, b = x1, ha = h0;
      for (int it = 0; it < 200 && b - a > 1e-16; it++) {
        const double m = 0.5 * (a + b), hm = h(m);
        if ((hm < 0.0) == (ha < 0.0)) {
          a = m;
          ha = hm;
        } else {
          b = m;
        }
      }
      roots.push_back(0.5 * (a + b));
    }
    x0 = x1;
    h0 = h1;
  }
  if ((int)roots.size() != ell_max / 2) return PSPEC_EUNSUPPORTED;  // not expected for l_max <= 16
  mu_edges[0] = 0.0;
  for (int i = 0; i < ell_max / 2; i++) mu_edges[i + 1] = roots[i];
  mu_edges[ell_max / 2 + 1] = 1.0;
  return PSPEC_OK;
}

extern "C" pspec_status pspec_transverse_response(int32_t ell_max, const double* mu, int32_t n, double* R) {
  if (!valid_lmax(ell_max) || n < 0 || (n > 0 && (!mu || !R))) return PSPEC_EINVAL;
  const double lmax0 = legendre(ell_max, 0.0);
  const std::vector<double> c = legendre_coeffs(ell_max + 1);
  for (int i = 0; i < n; i++) {
    const double m = mu[i];
    if (!(m >= -1.0 && m <= 1.0)) return PSPEC_EINVAL;
    // L_{l_max+1}(mu)/mu, its limit c_1 at mu = 0
    const double q = m == 0.0 ? c[1] : legendre(ell_max + 1, m) / m;
    R[i] = -0.5 * (ell_max + 1) * lmax0 * q;
  }
  return PSPEC_OK;
}
