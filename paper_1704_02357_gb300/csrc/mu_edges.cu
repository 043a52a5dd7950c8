// Wedge statistics, host code in FP64. Sec. 3.1: the leakage response R(mu) of a mu = 0 spike
// reconstructed from the even multipoles up to l_max (eq. response), and the non-uniform mu
// edges that confine it to the first wedge (eq. nonuniform-bins). Sec. 4.1: the mean Legendre
// matrix of the wedges (eq. Lbar) and the Kaiser-model wedge covariance gamma_mn (eq. gamma).
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

namespace {

// n-point Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on L_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; i++) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int m = 1; m < n; m++) {
        const double p2 = ((2.0 * m + 1.0) * z * p1 - m * p0) / (m + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);  // L_n'(z)
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

double lbar(int l, double a, double b) {
  if (l == 0) return 1.0;
  return ((legendre(l + 1, b) - legendre(l - 1, b)) - (legendre(l + 1, a) - legendre(l - 1, a))) /
         ((2.0 * l + 1.0) * (b - a));
}

bool edges_ok(const double* e, int n_mu) {
  if (!e || n_mu < 1 || n_mu > PSPEC_MAX_MU) return false;
  for (int w = 0; w <= n_mu; w++) {
    if (!(e[w] >= 0.0 && e[w] <= 1.0)) return false;
    if (w && !(e[w] > e[w - 1])) return false;
  }
  return true;
}

}  // namespace

extern "C" pspec_status pspec_wedge_lbar(const int32_t* ells, int32_t n_ells, const double* mu_edges, int32_t n_mu,
                                         double* out) {
  if (!ells || !out || n_ells < 1 || !edges_ok(mu_edges, n_mu)) return PSPEC_EINVAL;
  for (int i = 0; i < n_ells; i++)
    if (ells[i] < 0 || ells[i] > PSPEC_MAX_ELL) return PSPEC_EINVAL;
  for (int w = 0; w < n_mu; w++)
    for (int i = 0; i < n_ells; i++) out[w * n_ells + i] = lbar(ells[i], mu_edges[w], mu_edges[w + 1]);
  return PSPEC_OK;
}

extern "C" pspec_status pspec_wedge_gamma_kaiser(int32_t ell_max, const double* mu_edges, int32_t n_mu, double beta,
                                                 double* gamma) {
  if (!gamma || !valid_lmax(ell_max) || !edges_ok(mu_edges, n_mu) || !std::isfinite(beta)) return PSPEC_EINVAL;
  const int nl = ell_max / 2 + 1;  // the even multipoles the wedges are built from
  // I_ll' = int dmu/2 L_l L_l' (1 + beta mu^2)^4: a polynomial of degree <= 2 l_max + 8
  std::vector<double> x, w;
  gauss_legendre(ell_max + 8, x, w);
  std::vector<double> I((size_t)nl * nl, 0.0);
  for (size_t q = 0; q < x.size(); q++) {
    const double k = 1.0 + beta * x[q] * x[q], k4 = k * k * k * k;
    for (int a = 0; a < nl; a++)
      for (int b = 0; b < nl; b++) I[a * nl + b] += 0.5 * w[q] * legendre(2 * a, x[q]) * legendre(2 * b, x[q]) * k4;
  }
  for (int m = 0; m < n_mu; m++)
    for (int n = 0; n < n_mu; n++) {
      double s = 0.0;
      for (int a = 0; a < nl; a++)
        for (int b = 0; b < nl; b++)
          s += (4.0 * a + 1.0) * (4.0 * b + 1.0) * lbar(2 * a, mu_edges[m], mu_edges[m + 1]) *
               lbar(2 * b, mu_edges[n], mu_edges[n + 1]) * I[a * nl + b];
      gamma[m * n_mu + n] = s;
    }
  return PSPEC_OK;
}
