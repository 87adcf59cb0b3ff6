// fit.cu -- least-squares polynomial fit of a nonlinearity (Sec. 3, Eq. 3):
// the host utility behind polynomials such as Table 2's, which replace a
// loss gradient that CKKS arithmetic cannot evaluate by additions and
// multiplications only.  Given samples (x_i, y_i = f(x_i)), it returns the
// coefficients c_0 .. c_d minimising sum_i (y_i - sum_k c_k x_i^k)^2.
//
// Host code only.  The abscissas are scaled to t = x / s, s = max |x_i|, so
// that the normal equations sum_i t_i^(j+k) b_k = sum_i t_i^j y_i are well
// conditioned for the low degrees used here; they are accumulated and solved
// (Gaussian elimination with partial pivoting) in long double, and c_k =
// b_k / s^k.
#include <math.h>

#include <vector>

#include "he_internal.h"

using namespace he;

extern "C" int he_fit_poly(const double* x, const double* y, size_t n, uint32_t degree, double* coeffs) {
  if (!x || !y || !coeffs) return fail(HE_EINVAL, "he_fit_poly: null argument");
  if (degree > 16) return fail(HE_EINVAL, "he_fit_poly: degree above 16");
  const size_t m = (size_t)degree + 1;
  if (n < m) return fail(HE_EINVAL, "he_fit_poly: fewer samples than coefficients");
  long double s = 0;
  for (size_t i = 0; i < n; ++i) {
    if (!isfinite(x[i]) || !isfinite(y[i])) return fail(HE_EINVAL, "he_fit_poly: non-finite sample");
    s = fmaxl(s, fabsl((long double)x[i]));
  }
  if (s == 0) s = 1;
  // G[j][k] = sum t^(j+k) (from the power sums), r[j] = sum t^j y
  std::vector<long double> pw(2 * m - 1, 0.0L), r(m, 0.0L);
  for (size_t i = 0; i < n; ++i) {
    const long double t = (long double)x[i] / s;
    long double p = 1;
    for (size_t k = 0; k < 2 * m - 1; ++k) {
      pw[k] += p;
      if (k < m) r[k] += p * (long double)y[i];
      p *= t;
    }
  }
  std::vector<long double> G(m * (m + 1));  // augmented [G | r]
  for (size_t j = 0; j < m; ++j) {
    for (size_t k = 0; k < m; ++k) G[j * (m + 1) + k] = pw[j + k];
    G[j * (m + 1) + m] = r[j];
  }
  for (size_t col = 0; col < m; ++col) {
    size_t piv = col;
    for (size_t row = col + 1; row < m; ++row)
      if (fabsl(G[row * (m + 1) + col]) > fabsl(G[piv * (m + 1) + col])) piv = row;
    if (G[piv * (m + 1) + col] == 0) return fail(HE_EINVAL, "he_fit_poly: samples do not determine the polynomial");
    if (piv != col)
      for (size_t k = 0; k <= m; ++k) std::swap(G[piv * (m + 1) + k], G[col * (m + 1) + k]);
    for (size_t row = col + 1; row < m; ++row) {
      const long double f = G[row * (m + 1) + col] / G[col * (m + 1) + col];
      for (size_t k = col; k <= m; ++k) G[row * (m + 1) + k] -= f * G[col * (m + 1) + k];
    }
  }
  std::vector<long double> b(m);
  for (size_t j = m; j-- > 0;) {
    long double v = G[j * (m + 1) + m];
    for (size_t k = j + 1; k < m; ++k) v -= G[j * (m + 1) + k] * b[k];
    b[j] = v / G[j * (m + 1) + j];
  }
  long double sk = 1;
  for (size_t k = 0; k < m; ++k) {
    coeffs[k] = (double)(b[k] / sk);
    sk *= s;
  }
  return HE_OK;
}
