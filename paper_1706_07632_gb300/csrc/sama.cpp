// Two-grid convergence factor predicted by mode analysis (Section 5, Table 2): sine modes in space,
// the time matrix treated exactly.  Host code.
//
// The two-grid operator (nu1 + nu2 red-black zebra-in-time sweeps, full weighting, (bi)linear
// interpolation, exact coarse solve) maps a group of sine modes -- a mode k and its partner N+1-k in
// 1D, the four combinations in 2D -- into itself, and on a group every time block is a rational
// function of the lower-triangular time matrix.  Its eigenvalues are therefore those of the small
// group matrices evaluated at the diagonal entries R_mm, and the predicted factor is the largest
// spectral radius over groups and time levels.  Per group, with c = cos(k pi / (N+1)):
//   smoother (one red-black sweep): values on the point classes are linear in the amplitudes;
//     a red point takes (neighbour sum) / (h^2 (R_mm + s)), s = 2/h^2 or 4/h^2, then the black ones;
//   coarse correction: I - P (R_mm + lam_c)^-1 W (R_mm + diag(lam)), W the full-weighting row of the
//     group (1D: ((1+c)/2, -(1-c)/2)), P = W^T the interpolation, lam the groups' eigenvalues of A_h.
#include <cmath>
#include <complex>
#include <vector>

namespace fhmg {

namespace {

template <int n>
struct Mat {
  double a[n][n];
};

template <int n>
Mat<n> mul(const Mat<n>& x, const Mat<n>& y) {
  Mat<n> z{};
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += x.a[i][k] * y.a[k][j];
      z.a[i][j] = s;
    }
  return z;
}

template <int n>
Mat<n> eye() {
  Mat<n> z{};
  for (int i = 0; i < n; ++i) z.a[i][i] = 1.0;
  return z;
}

template <int n>
Mat<n> power(const Mat<n>& x, int p) {
  Mat<n> z = eye<n>();
  for (int i = 0; i < p; ++i) z = mul(z, x);
  return z;
}

double radius2(const Mat<2>& T) {
  const double tr = T.a[0][0] + T.a[1][1], det = T.a[0][0] * T.a[1][1] - T.a[0][1] * T.a[1][0];
  const double disc = 0.25 * tr * tr - det;
  if (disc >= 0.0) {
    const double r = std::sqrt(disc);
    return std::max(std::fabs(0.5 * tr + r), std::fabs(0.5 * tr - r));
  }
  return std::sqrt(det);
}

// spectral radius of a 4x4 matrix: characteristic polynomial by the Faddeev-LeVerrier recursion,
// its roots by the Durand-Kerner (Weierstrass) iteration
double radius4(const Mat<4>& A) {
  double c[5];  // lambda^4 + c[1] lambda^3 + c[2] lambda^2 + c[3] lambda + c[4]
  c[0] = 1.0;
  Mat<4> Mk = eye<4>();
  for (int k = 1; k <= 4; ++k) {
    const Mat<4> AM = mul(A, Mk);
    double tr = 0.0;
    for (int i = 0; i < 4; ++i) tr += AM.a[i][i];
    c[k] = -tr / k;
    Mk = AM;
    for (int i = 0; i < 4; ++i) Mk.a[i][i] += c[k];
  }
  double bound = 0.0;
  for (int k = 1; k <= 4; ++k) bound = std::max(bound, std::pow(std::fabs(c[k]), 1.0 / k));
  bound = 2.0 * bound + 1e-300;
  using cd = std::complex<double>;
  cd z[4];
  const cd seed(0.4, 0.9);
  for (int k = 0; k < 4; ++k) z[k] = bound * std::pow(seed, k);
  auto poly = [&](cd x) { return (((x + c[1]) * x + c[2]) * x + c[3]) * x + c[4]; };
  for (int it = 0; it < 500; ++it) {
    double move = 0.0;
    for (int k = 0; k < 4; ++k) {
      cd den(1.0, 0.0);
      for (int j = 0; j < 4; ++j)
        if (j != k) den *= z[k] - z[j];
      if (std::abs(den) == 0.0) den = cd(1e-300, 0.0);
      const cd step = poly(z[k]) / den;
      z[k] -= step;
      move = std::max(move, std::abs(step));
    }
    if (move <= 1e-15 * bound) break;
  }
  double r = 0.0;
  for (int k = 0; k < 4; ++k) r = std::max(r, std::abs(z[k]));
  return r;
}

double group1d(double mu, double c, double h, int nu1, int nu2) {
  const double ih2 = 1.0 / (h * h);
  const double G = 2.0 * c * ih2 / (mu + 2.0 * ih2);
  // amplitudes (a, b) of modes k and N+1-k; odd points hold a+b, even ones a-b; odd points first:
  // p' = G q, q' = G p'  ->  in (a, b): S = C^-1 [[0, G], [0, G^2]] C, C = [[1, 1], [1, -1]]
  Mat<2> S{};
  const double g1 = G, g2 = G * G;
  S.a[0][0] = 0.5 * (g1 + g2);
  S.a[0][1] = -0.5 * (g1 + g2);
  S.a[1][0] = 0.5 * (g1 - g2);
  S.a[1][1] = -0.5 * (g1 - g2);
  const double lk = 2.0 * ih2 * (1.0 - c), lkp = 2.0 * ih2 * (1.0 + c), lc = (1.0 - c * c) * ih2;
  const double w[2] = {0.5 * (1.0 + c), -0.5 * (1.0 - c)};
  const double d[2] = {mu + lk, mu + lkp};
  Mat<2> K = eye<2>();
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) K.a[i][j] -= w[i] * w[j] * d[j] / (mu + lc);
  return radius2(mul(mul(power(S, nu2), K), power(S, nu1)));
}

double group2d(double mu, double cx, double cy, double h, int nu1, int nu2) {
  const double ih2 = 1.0 / (h * h);
  const double g = ih2 / (mu + 4.0 * ih2);
  // amplitudes of (k,l), (k',l'), (k',l), (k,l'); point classes (i odd/even, j odd/even) oo, ee, oe,
  // eo hold v = C a with the Hadamard C below (C^-1 = C / 4)
  static const double C[4][4] = {{1, 1, 1, 1}, {1, 1, -1, -1}, {1, -1, 1, -1}, {1, -1, -1, 1}};
  Mat<4> red = eye<4>(), black = eye<4>();
  // red points (i + j even: oo, ee) from their neighbours (x-neighbours of oo are eo, y-neighbours oe)
  red.a[0][0] = red.a[1][1] = 0.0;
  red.a[0][2] = 2 * cy * g;
  red.a[0][3] = 2 * cx * g;
  red.a[1][2] = 2 * cx * g;
  red.a[1][3] = 2 * cy * g;
  black.a[2][2] = black.a[3][3] = 0.0;
  black.a[2][0] = 2 * cy * g;
  black.a[2][1] = 2 * cx * g;
  black.a[3][0] = 2 * cx * g;
  black.a[3][1] = 2 * cy * g;
  const Mat<4> Sv = mul(black, red);
  Mat<4> S{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) s += 0.25 * C[i][p] * Sv.a[p][q] * C[q][j];
      S.a[i][j] = s;
    }
  auto l1 = [&](double c) { return 2.0 * ih2 * (1.0 - c); };
  const double lam[4] = {l1(cx) + l1(cy), l1(-cx) + l1(-cy), l1(-cx) + l1(cy), l1(cx) + l1(-cy)};
  const double lc = (1.0 - cx * cx) * ih2 + (1.0 - cy * cy) * ih2;
  const double w[4] = {0.25 * (1 + cx) * (1 + cy), 0.25 * (1 - cx) * (1 - cy), -0.25 * (1 - cx) * (1 + cy),
                       -0.25 * (1 + cx) * (1 - cy)};
  Mat<4> K = eye<4>();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) K.a[i][j] -= w[i] * w[j] * (mu + lam[j]) / (mu + lc);
  return radius4(mul(mul(power(S, nu2), K), power(S, nu1)));
}

}  // namespace

double sama_two_grid(const std::vector<double>& rdiag, int dim, int N, double h, int nu1, int nu2) {
  const double pi = std::acos(-1.0);
  double best = 0.0;
  for (int k = 1; k <= (N - 1) / 2; ++k) {
    const double cx = std::cos(k * pi / (N + 1));
    if (dim == 1) {
      for (double mu : rdiag) best = std::max(best, group1d(mu, cx, h, nu1, nu2));
    } else {
      for (int l = 1; l <= (N - 1) / 2; ++l) {
        const double cy = std::cos(l * pi / (N + 1));
        for (double mu : rdiag) best = std::max(best, group2d(mu, cx, cy, h, nu1, nu2));
      }
    }
  }
  return best;
}

}  // namespace fhmg
