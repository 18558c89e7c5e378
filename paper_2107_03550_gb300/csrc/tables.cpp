// Host FP64 builder of the convolution kernels C^T_II and C^N_II (Sec. 2.3,
// Sec. 2.4) as piecewise Chebyshev tables, plus FFT twiddles.
//
// Route (independent of any quadrature):
//   W(x) = int_x^inf J1(t)/t dt  (App. A).  Since int_0^x J0 = 2 sum_{k>=0}
//   J_{2k+1}(x) and W = 1 - int_0^x J0 + J1 (Sec. 2.3 with App. A), W follows
//   from the odd-order Bessel functions, which Miller's backward recurrence
//   (normalised by J0 + 2 sum J_{2k} = 1) gives for x <= 12; for
//   12 < x <= 40, W(x) = W(40) + int_x^40 J1(t)/t dt by Gauss-Legendre,
//   anchored on the asymptotic value at 40.
//   For x > 40 the Struve-Bessel difference K_nu = H_nu - Y_nu has the
//   asymptotic series of DLMF 11.6.1; with the Wronskian J1 Y0 - J0 Y1 =
//   2/(pi x) the psi of Sec. 2.3 becomes 1 + x (J1 A0 - J0 A1), A = (pi/2) K,
//   and the leading cancellation of the kernels is removed analytically:
//     X(x) = x^2 W(x) - x J0(x)
//          = J0(x) sum_{k>=2} a_k x^{3-2k} + J1(x) (1 - sum_{k>=1} b_k x^{2-2k}),
//   a_k = (-1)^k ((2k-1)!!)^2 / (1 - 2k),  b_k = (-1)^k ((2k-1)!!)^2,
//   truncated at the smallest term.  The kernels are then
//     C^T = r^2 W(s/r) + r^2 X(s/r) - W(s) - X(s) - r^2 J1(s/r) + J1(s)/2
//     C^N = (A - r^2) W(s/r) - r^2 X(s/r) + (1 - 1/(2r^2)) W(s) + X(s)
//           + (r^2 - A) J1(s/r) + (1/(2r^2) - 1) J1(s),
//   with s = c_s k t, r = c_s/c_p, A = (1/r^2 - 2)^2 r^2 / 2 (Eq. Ct and the
//   C^N expression of Sec. 2.4 regrouped so that no two large terms cancel).
//   J0, J1 are the C library's j0/j1.
#include <cmath>
#include <vector>

#include "internal.h"
#include "sbiem.h"

namespace sbiem {

namespace {

// Miller backward recurrence: J_0..J_{nmax}(x), x > 0, normalised by
// J0 + 2 sum_{k>=1} J_{2k} = 1.
void bessel_j_all(double x, int nmax, std::vector<double>& J) {
  int nstart = nmax + 30 + static_cast<int>(x);
  if (nstart % 2) ++nstart;
  J.assign(nstart + 2, 0.0);
  double jp1 = 0.0, j = 1e-300;
  J[nstart] = j;
  for (int n = nstart; n >= 1; --n) {
    const double jm1 = (2.0 * n / x) * j - jp1;
    jp1 = j;
    j = jm1;
    J[n - 1] = j;
    if (std::fabs(j) > 1e250) {
      for (int m = n - 1; m <= nstart; ++m) J[m] *= 1e-250;
      jp1 *= 1e-250;
      j *= 1e-250;
    }
  }
  double norm = J[0];
  for (int k = 2; k <= nstart; k += 2) norm += 2.0 * J[k];
  for (int m = 0; m <= nstart; ++m) J[m] /= norm;
  J.resize(nmax + 1);
}

constexpr double kSwitch = 40.0;   // asymptotic series above
constexpr double kMiller = 12.0;   // Miller recurrence below

// Gauss-Legendre nodes/weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double>& xs, std::vector<double>& ws) {
  xs.assign(n, 0.0);
  ws.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-16) break;
    }
    xs[i] = -z;
    xs[n - 1 - i] = z;
    ws[i] = ws[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

// int_a^b J1(t)/t dt, composite 20-point Gauss-Legendre on panels <= 1.
double j1_over_t_integral(double a, double b) {
  static const struct GL {
    std::vector<double> x, w;
    GL() { gauss_legendre(20, x, w); }
  } gl;
  const int panels = static_cast<int>(std::ceil((b - a) / 1.0));
  double sum = 0.0;
  for (int p = panels - 1; p >= 0; --p) {  // small-magnitude end first
    const double lo = a + (b - a) * p / panels, hi = a + (b - a) * (p + 1) / panels;
    const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    double ps = 0.0;
    for (size_t i = 0; i < gl.x.size(); ++i) {
      const double t = mid + half * gl.x[i];
      ps += gl.w[i] * ::j1(t) / t;
    }
    sum += half * ps;
  }
  return sum;
}

void w_and_x_asymptotic(double x, double* W, double* X);

// W(x) and X(x) = x^2 W - x J0 for x >= 0.
void w_and_x(double x, double* W, double* X) {
  if (x == 0.0) {
    *W = 1.0;
    *X = 0.0;
    return;
  }
  if (x > kMiller && x <= kSwitch) {
    // W(x) = W(40) + int_x^40 J1(t)/t dt: anchored on the asymptotic value so
    // that no "1 - (sum close to 1)" cancellation enters x^2 W
    double W40, X40;
    w_and_x_asymptotic(kSwitch, &W40, &X40);
    const double w = W40 + j1_over_t_integral(x, kSwitch);
    *W = w;
    *X = x * x * w - x * ::j0(x);
    return;
  }
  if (x <= kMiller) {
    static thread_local std::vector<double> J;
    const int nmax = static_cast<int>(x) + 40;
    bessel_j_all(x, nmax, J);
    double odd = 0.0;  // J3 + J5 + ...
    for (int n = static_cast<int>(J.size()) - 1; n >= 3; --n)
      if (n % 2 == 1) odd += J[n];
    const double w = 1.0 - J[1] - 2.0 * odd;
    *W = w;
    *X = x * x * w - x * ::j0(x);
    return;
  }
  w_and_x_asymptotic(x, W, X);
}

// x >= 40: DLMF 11.6.1 series, truncated at the smallest term.
void w_and_x_asymptotic(double x, double* W, double* X) {
  const double j0 = ::j0(x), j1 = ::j1(x);
  const double ix2 = 1.0 / (x * x);
  // running ((2k-1)!!)^2 x^{-2k}
  double t = 1.0;  // k = 0
  double sa = 0.0, sb = 0.0;  // sum_{k>=2} a_k x^{-2k}, sum_{k>=1} b_k x^{-2k}
  double sa1 = 0.0;            // sum_{k>=1} a_k x^{-2k} for W
  double prev = 1e300;
  for (int k = 1; k < 200; ++k) {
    const double dk = 2.0 * k - 1.0;
    t *= dk * dk * ix2;  // ((2k-1)!!)^2 / x^{2k}
    if (t > prev) break;  // asymptotic series: stop at the smallest term
    prev = t;
    const double sgn = (k % 2) ? -1.0 : 1.0;
    const double ak = sgn * t / (1.0 - 2.0 * k);
    const double bk = sgn * t;
    sa1 += ak;
    if (k >= 2) sa += ak;
    sb += bk;
    if (t < 1e-22) break;
  }
  // W = x J0 (A1 - 1) + J1 (1 - x A0) = x J0 sa1 + J1 (-sb)
  *W = x * j0 * sa1 - j1 * sb;
  // X = x J0 [x^2 (A1 - 1) - 1] + x^2 J1 (1 - x A0) = J0 x^3 sa + J1 x^2 (-sb)
  *X = j0 * x * x * x * sa - j1 * x * x * sb;
}

}  // namespace

void kernel_values(double s, double r, double* cT, double* cN) {
  double Ws, Xs, Wp, Xp;
  w_and_x(s, &Ws, &Xs);
  w_and_x(s / r, &Wp, &Xp);
  const double J1s = ::j1(s), J1p = ::j1(s / r);
  const double r2 = r * r;
  const double A = (1.0 / r2 - 2.0) * (1.0 / r2 - 2.0) * r2 / 2.0;
  *cT = r2 * Wp + r2 * Xp - Ws - Xs - r2 * J1p + 0.5 * J1s;
  *cN = (A - r2) * Wp - r2 * Xp + (1.0 - 1.0 / (2.0 * r2)) * Ws + Xs + (r2 - A) * J1p +
        (1.0 / (2.0 * r2) - 1.0) * J1s;
}

// Piecewise Chebyshev interpolants of C^T and C^N on [0, smax]: pieces of
// width h, degree deg, coefficients from the values at the Chebyshev nodes.
void build_cheb(double r, double smax, ChebTable* tab) {
  const double h = 0.5;
  const int deg = 16;
  const int npieces = static_cast<int>(std::ceil(smax / h)) + 1;
  tab->h = h;
  tab->deg = deg;
  tab->npieces = npieces;
  tab->coef.assign(static_cast<size_t>(npieces) * (deg + 1) * 2, 0.0);
  const int n = deg + 1;
  std::vector<double> vT(n), vN(n);
  for (int p = 0; p < npieces; ++p) {
    const double a = p * h, b = (p + 1) * h;
    for (int i = 0; i < n; ++i) {
      const double xi = std::cos(M_PI * (i + 0.5) / n);
      kernel_values(0.5 * (a + b) + 0.5 * (b - a) * xi, r, &vT[i], &vN[i]);
    }
    for (int k = 0; k < n; ++k) {
      double sT = 0.0, sN = 0.0;
      for (int i = 0; i < n; ++i) {
        const double c = std::cos(M_PI * k * (i + 0.5) / n);
        sT += vT[i] * c;
        sN += vN[i] * c;
      }
      const double f = (k == 0 ? 1.0 : 2.0) / n;
      double* out = &tab->coef[(static_cast<size_t>(p) * n + k) * 2];
      out[0] = f * sT;
      out[1] = f * sN;
    }
  }
}

// FP32 table of the midpoint weights dt C(s) for the history sweep to evaluate
// on chip (the weights depend on the mode only through s = c_s k_n (j + 1/2)
// dt_min).  Piece q starts at s = q kGenH and its polynomial of degree
// kGenDeg holds on [q kGenH, q kGenH + kGenSpan kGenH] (a span longer than
// the piece, so a run of consecutive lags that starts in piece q stays on its
// polynomial), in t = (s - q kGenH) / (kGenSpan kGenH / 2) - 1 in [-1, 1];
// it interpolates C^T and C^N at the Chebyshev nodes of that span (monomial
// coefficients from the nodal values by Gaussian elimination in FP64, then
// scaled by dt and rounded to FP32).  Layout per piece: coefficient pairs
// (T, N) for k = 0..kGenDeg, kGenDeg + 1 pairs.  *max_err: the largest
// |table - dt C| over 16 points per span, evaluated in FP64 from the rounded
// coefficients, over dt max|C|.
void build_gen_table(double r, double dt, double smax, std::vector<float>& tab, int* npieces, double* max_err) {
  const int n = kGenDeg + 1;
  const int P = static_cast<int>(std::ceil(smax / kGenH)) + 1;
  *npieces = P;
  tab.assign(static_cast<size_t>(P) * n * 2, 0.0f);
  std::vector<double> xi(n), vT(n), vN(n), A(n * n), bT(n), bN(n);
  for (int i = 0; i < n; ++i) xi[i] = std::cos(M_PI * (i + 0.5) / n);
  double err = 0.0, cmax = 0.0;
  for (int p = 0; p < P; ++p) {
    const double a = p * kGenH, half = 0.5 * kGenSpan * kGenH;
    for (int i = 0; i < n; ++i) kernel_values(a + half * (xi[i] + 1.0), r, &vT[i], &vN[i]);
    // Vandermonde system V c = v, V[i][k] = xi_i^k, by elimination with partial pivoting
    for (int i = 0; i < n; ++i) {
      double x = 1.0;
      for (int k = 0; k < n; ++k) {
        A[i * n + k] = x;
        x *= xi[i];
      }
      bT[i] = vT[i];
      bN[i] = vN[i];
    }
    for (int c = 0; c < n; ++c) {
      int piv = c;
      for (int i = c + 1; i < n; ++i)
        if (std::fabs(A[i * n + c]) > std::fabs(A[piv * n + c])) piv = i;
      if (piv != c) {
        for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
        std::swap(bT[c], bT[piv]);
        std::swap(bN[c], bN[piv]);
      }
      for (int i = c + 1; i < n; ++i) {
        const double f = A[i * n + c] / A[c * n + c];
        for (int k = c; k < n; ++k) A[i * n + k] -= f * A[c * n + k];
        bT[i] -= f * bT[c];
        bN[i] -= f * bN[c];
      }
    }
    for (int c = n - 1; c >= 0; --c) {
      for (int k = c + 1; k < n; ++k) {
        bT[c] -= A[c * n + k] * bT[k];
        bN[c] -= A[c * n + k] * bN[k];
      }
      bT[c] /= A[c * n + c];
      bN[c] /= A[c * n + c];
    }
    float* out = &tab[static_cast<size_t>(p) * n * 2];
    for (int k = 0; k < n; ++k) {
      out[2 * k] = static_cast<float>(dt * bT[k]);
      out[2 * k + 1] = static_cast<float>(dt * bN[k]);
    }
    for (int q = 0; q < 16; ++q) {
      const double t = -1.0 + (q + 0.5) / 8.0;
      double eT = out[2 * kGenDeg], eN = out[2 * kGenDeg + 1];
      for (int k = kGenDeg - 1; k >= 0; --k) {
        eT = eT * t + out[2 * k];
        eN = eN * t + out[2 * k + 1];
      }
      double cT, cN;
      kernel_values(a + half * (t + 1.0), r, &cT, &cN);
      err = std::max(err, std::max(std::fabs(eT - dt * cT), std::fabs(eN - dt * cN)));
      cmax = std::max(cmax, std::max(std::fabs(cT), std::fabs(cN)));
    }
  }
  *max_err = cmax > 0.0 ? err / (dt * cmax) : 0.0;
}

// exp(-2 pi i j / N), j = 0..N-1, via octant symmetry so that every value is
// a sin/cos of an angle in [0, pi/4].
void build_twiddles(int64_t N, std::vector<double>& tw) {
  tw.assign(static_cast<size_t>(2 * N), 0.0);
  for (int64_t j = 0; j < N; ++j) {
    // angle = 2 pi j / N = (pi/4) * (8 j / N); reduce 8j mod 8N
    const int64_t e = 8 * j;              // in units of (pi/4)/N
    const int64_t oct = e / N;            // octant 0..7
    const int64_t rem = e - oct * N;      // 0..N-1
    double c, s;
    const double ang_rem = (M_PI / 4.0) * static_cast<double>(rem) / static_cast<double>(N);
    const double ang_co = (M_PI / 4.0) * static_cast<double>(N - rem) / static_cast<double>(N);
    // cos/sin of theta = oct*pi/4 + ang_rem
    switch (oct) {
      case 0: c = std::cos(ang_rem); s = std::sin(ang_rem); break;
      case 1: c = std::sin(ang_co); s = std::cos(ang_co); break;
      case 2: c = -std::sin(ang_rem); s = std::cos(ang_rem); break;
      case 3: c = -std::cos(ang_co); s = std::sin(ang_co); break;
      case 4: c = -std::cos(ang_rem); s = -std::sin(ang_rem); break;
      case 5: c = -std::sin(ang_co); s = -std::cos(ang_co); break;
      case 6: c = std::sin(ang_rem); s = -std::cos(ang_rem); break;
      default: c = std::cos(ang_co); s = -std::sin(ang_co); break;
    }
    tw[2 * j] = c;       // cos(2 pi j/N)
    tw[2 * j + 1] = -s;  // -sin(2 pi j/N): forward transform sign
  }
}

}  // namespace sbiem

extern "C" int sbiem_kernel_values(const double* s, int64_t n, double r, double* cT, double* cN) {
  if (!s || !cT || !cN || n < 0 || !(r > 0.0) || !(r < 1.0)) return SBIEM_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (!(s[i] >= 0.0)) return SBIEM_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i) sbiem::kernel_values(s[i], r, &cT[i], &cN[i]);
  return SBIEM_OK;
}
