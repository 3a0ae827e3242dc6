// Host-side monomial tables of the Zernike basis (fp64).
//
// Methods ("Computational Scaling"): each Zernike polynomial is evaluated per
// pixel as a sum of monomials, Z_d(x, y) = sum a_nm^(d) x^n y^m, from global
// coefficient tables. The tables are derived here from
//   Z_n^m = R_n^|m|(rho) * {cos, sin}(|m| theta)
//         = sum_k c_k (x^2 + y^2)^(s-k) * {Re, Im}((x + i y)^|m|),
// with s = (n - |m|)/2 and c_k the radial-polynomial coefficients
//   c_k = (-1)^k (n-k)! / (k! ((n+|m|)/2-k)! ((n-|m|)/2-k)!),
// expanding both factors binomially.
#include "basis_host.h"

#include <cmath>
#include <vector>

namespace ash {

static double factorial(int n) {
  double f = 1.0;
  for (int q = 2; q <= n; ++q) f *= (double)q;
  return f;
}

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double b = 1.0;
  for (int q = 1; q <= k; ++q) b = b * (double)(n - k + q) / (double)q;
  return std::round(b);
}

bool noll_to_nm(int j, int* n_out, int* m_out) {
  if (j < 1 || j > 100000) return false;
  // radial order: number of complete rows before j
  int n = (int)std::floor((std::sqrt(8.0 * (double)j - 7.0) - 1.0) / 2.0);
  while (n > 0 && n * (n + 1) / 2 >= j) --n;
  while ((n + 1) * (n + 2) / 2 < j) ++n;
  const int k = j - n * (n + 1) / 2 - 1;   // 0-based position in row n
  const int par = n % 2;
  const int am = par + 2 * ((k + 1 - par) / 2);
  *n_out = n;
  *m_out = (am == 0) ? 0 : ((j % 2 == 0) ? am : -am);
  return true;
}

bool zernike_monomials(int n, int m, std::vector<MonoTerm>* out) {
  const int a = m < 0 ? -m : m;
  if (a > n || ((n - a) & 1)) return false;
  const int s = (n - a) / 2;
  // dense coefficient grid c[px][py], px + py <= n
  std::vector<double> grid((size_t)(n + 1) * (n + 1), 0.0);
  for (int k = 0; k <= s; ++k) {
    const double ck = ((k & 1) ? -1.0 : 1.0) * factorial(n - k) /
                      (factorial(k) * factorial((n + a) / 2 - k) * factorial((n - a) / 2 - k));
    const int q = s - k;   // power of (x^2 + y^2)
    for (int u = 0; u <= q; ++u) {
      const double bq = binom(q, u);
      for (int v = 0; v <= a; ++v) {
        // (i y)^v: real part for even v, imaginary part for odd v
        const bool real_part = (v % 2) == 0;
        if (real_part != (m >= 0)) continue;
        const double sign = ((v / 2) % 2) ? -1.0 : 1.0;
        const int px = 2 * u + (a - v);
        const int py = 2 * (q - u) + v;
        grid[(size_t)px * (n + 1) + py] += ck * bq * binom(a, v) * sign;
      }
    }
  }
  for (int px = 0; px <= n; ++px)
    for (int py = 0; py + px <= n; ++py) {
      const double c = grid[(size_t)px * (n + 1) + py];
      if (c != 0.0) out->push_back(MonoTerm{c, px, py});
    }
  return true;
}

}  // namespace ash
