// Host construction of the H-matrix approximation of the L1 matrix R (Sections 2 and 3).
// See hbuild.h for the data layout handed to the kernels.
#include "hbuild.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <numeric>

namespace fhmg {
namespace {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Quad {
  std::vector<double> x, w;
  Quad() { gauss_legendre(20, x, w); }
};
const Quad& quad() {
  static Quad q;
  return q;
}

// (b + d)^p - b^p for b >= 0, d > 0 without cancellation.
double pow_step(double b, double d, double p) {
  if (b > 0.0) return std::pow(b, p) * std::expm1(p * std::log1p(d / b));
  return std::pow(d, p);
}

// D(m, i) = [(t_m - t_{i-1})^{1-a} - (t_m - t_i)^{1-a}] / ((t_i - t_{i-1}) Gamma(2-a)):
// the rising-half integral of phi_i' against the kernel (the paper's d_{m, m-i+1}).
double Dfun(const std::vector<double>& t, double a, int m, int i) {
  double tau = t[i] - t[i - 1];
  return pow_step(t[m] - t[i], tau, 1.0 - a) / (tau * std::tgamma(2.0 - a));
}

}  // namespace

double l1_entry(const std::vector<double>& t, double a, int m, int j) {
  if (j == m) return std::pow(t[m] - t[m - 1], -a) / std::tgamma(2.0 - a);
  if (j >= m - 2) return Dfun(t, a, m, j) - Dfun(t, a, m, j + 1);
  // Integration by parts: R_{m,j} = -a/Gamma(1-a) int (t_m - s)^{-1-a} phi_j(s) ds, the
  // support [t_{j-1}, t_{j+1}] ending at least two steps before t_m.
  const Quad& q = quad();
  double tl = t[j] - t[j - 1], tr = t[j + 1] - t[j];
  double dl0 = t[m] - t[j - 1], dr0 = t[m] - t[j];
  double sl = 0.0, sr = 0.0;
  for (size_t k = 0; k < q.x.size(); ++k) {
    double up = 0.5 * (1.0 + q.x[k]);
    sl += q.w[k] * up * std::pow(dl0 - tl * up, -1.0 - a);
    sr += q.w[k] * (1.0 - up) * std::pow(dr0 - tr * up, -1.0 - a);
  }
  return -a / std::tgamma(1.0 - a) * (0.5 * tl * sl + 0.5 * tr * sr);
}

namespace {

struct Rec {
  const std::vector<double>& t;
  int M, L;
  bool dense_mode;
  std::vector<std::array<int, 4>> rk, dense;
};

bool admissible(const std::vector<double>& t, int M, int r0, int r1, int c0, int c1) {
  double a = t[r0 + 1], b = t[r1];
  double d = t[std::min(c1 + 1, M)];
  return d < a && (b - a) <= (a - d);
}

void recurse(Rec& R, int r0, int r1, int c0, int c1) {
  if (c0 >= r1) return;  // zero block above the diagonal
  if (!R.dense_mode && admissible(R.t, R.M, r0, r1, c0, c1)) {
    R.rk.push_back({r0, r1, c0, c1});
    return;
  }
  if (r1 - r0 <= R.L) {
    R.dense.push_back({r0, r1, c0, c1});
    return;
  }
  int rm = (r0 + r1) / 2, cm = (c0 + c1) / 2;
  recurse(R, r0, rm, c0, cm);
  recurse(R, r0, rm, cm, c1);
  recurse(R, rm, r1, c0, cm);
  recurse(R, rm, r1, cm, c1);
}

// Scaled Taylor factors of one admissible block: A (nr x k), B (nc x k), block ~ A B^T.
void taylor_factors(const std::vector<double>& t, double a, int r0, int r1, int c0, int c1, int k,
                    std::vector<double>& A, std::vector<double>& B) {
  double ta = t[r0 + 1], tb = t[r1];
  double tc = 0.5 * (ta + tb), rho = 0.5 * (tb - ta);
  if (rho == 0.0) rho = 1.0;
  int nr = r1 - r0, nc = c1 - c0;
  double ig = 1.0 / std::tgamma(1.0 - a);
  A.assign((size_t)nr * k, 0.0);
  for (int r = 0; r < nr; ++r) {
    double x = (t[r0 + 1 + r] - tc) / rho, p = ig;
    for (int nu = 0; nu < k; ++nu) {
      A[(size_t)r * k + nu] = p;
      p *= x;
    }
  }
  std::vector<double> cnu(k);
  cnu[0] = 1.0;
  for (int nu = 1; nu < k; ++nu) cnu[nu] = cnu[nu - 1] * (1.0 - a - nu) / nu;
  const Quad& q = quad();
  B.assign((size_t)nc * k, 0.0);
  std::vector<double> acc(k);
  for (int c = 0; c < nc; ++c) {
    int j = c0 + 1 + c;
    double tl = t[j] - t[j - 1], tr = t[j + 1] - t[j];
    std::fill(acc.begin(), acc.end(), 0.0);
    for (size_t n = 0; n < q.x.size(); ++n) {
      double up = 0.5 * (1.0 + q.x[n]);
      double s1 = t[j - 1] + tl * up, s2 = t[j] + tr * up;
      double b1 = 0.5 * tl * q.w[n] * up * std::pow(tc - s1, -1.0 - a), r1v = rho / (tc - s1);
      double b2 = 0.5 * tr * q.w[n] * (1.0 - up) * std::pow(tc - s2, -1.0 - a), r2v = rho / (tc - s2);
      for (int nu = 0; nu < k; ++nu) {
        acc[nu] += b1 + b2;
        b1 *= r1v;
        b2 *= r2v;
      }
    }
    for (int nu = 0; nu < k; ++nu) B[(size_t)c * k + nu] = -cnu[nu] * (a + nu) * acc[nu];
  }
}

// Thin Householder QR of X (n x k, row-major): Q (n x r), R (r x k), r = min(n, k).
void householder_qr(const std::vector<double>& X, int n, int k, std::vector<double>& Q,
                    std::vector<double>& Rm, int& r) {
  r = std::min(n, k);
  std::vector<double> W(X);  // working copy, n x k
  std::vector<std::vector<double>> vs(r);
  for (int c = 0; c < r; ++c) {
    double nrm = 0.0;
    for (int i = c; i < n; ++i) nrm += W[(size_t)i * k + c] * W[(size_t)i * k + c];
    nrm = std::sqrt(nrm);
    std::vector<double> v(n - c, 0.0);
    if (nrm > 0.0) {
      double x0 = W[(size_t)c * k + c];
      double alpha = x0 >= 0 ? -nrm : nrm;
      for (int i = c; i < n; ++i) v[i - c] = W[(size_t)i * k + c];
      v[0] -= alpha;
      double vn = 0.0;
      for (double e : v) vn += e * e;
      if (vn > 0.0) {
        for (int cc = c; cc < k; ++cc) {
          double s = 0.0;
          for (int i = c; i < n; ++i) s += v[i - c] * W[(size_t)i * k + cc];
          s *= 2.0 / vn;
          for (int i = c; i < n; ++i) W[(size_t)i * k + cc] -= s * v[i - c];
        }
        double sc = 1.0 / std::sqrt(vn);
        for (double& e : v) e *= sc;
      } else {
        std::fill(v.begin(), v.end(), 0.0);
      }
    }
    vs[c] = v;
  }
  Rm.assign((size_t)r * k, 0.0);
  for (int i = 0; i < r; ++i)
    for (int c = i; c < k; ++c) Rm[(size_t)i * k + c] = W[(size_t)i * k + c];
  // Q = H_0 H_1 ... H_{r-1} applied to the first r columns of the identity
  Q.assign((size_t)n * r, 0.0);
  for (int i = 0; i < r; ++i) Q[(size_t)i * r + i] = 1.0;
  for (int c = r - 1; c >= 0; --c) {
    const std::vector<double>& v = vs[c];
    for (int cc = 0; cc < r; ++cc) {
      double s = 0.0;
      for (int i = c; i < n; ++i) s += v[i - c] * Q[(size_t)i * r + cc];
      s *= 2.0;
      if (s != 0.0)
        for (int i = c; i < n; ++i) Q[(size_t)i * r + cc] -= s * v[i - c];
    }
  }
}

// One-sided Jacobi SVD of S (p x q, row-major): S = U diag(sig) V^T with U's columns stored
// unnormalised in S (column j = sig_j u_j) and V (q x q, row-major).
void jacobi_svd(std::vector<double>& S, int p, int q, std::vector<double>& V) {
  V.assign((size_t)q * q, 0.0);
  for (int i = 0; i < q; ++i) V[(size_t)i * q + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int i = 0; i < q - 1; ++i)
      for (int j = i + 1; j < q; ++j) {
        double al = 0, be = 0, ga = 0;
        for (int r = 0; r < p; ++r) {
          double x = S[(size_t)r * q + i], y = S[(size_t)r * q + j];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
        rotated = true;
        double zeta = (be - al) / (2.0 * ga);
        double tt = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + tt * tt), s = c * tt;
        for (int r = 0; r < p; ++r) {
          double x = S[(size_t)r * q + i], y = S[(size_t)r * q + j];
          S[(size_t)r * q + i] = c * x - s * y;
          S[(size_t)r * q + j] = s * x + c * y;
        }
        for (int r = 0; r < q; ++r) {
          double x = V[(size_t)r * q + i], y = V[(size_t)r * q + j];
          V[(size_t)r * q + i] = c * x - s * y;
          V[(size_t)r * q + j] = s * x + c * y;
        }
      }
    if (!rotated) break;
  }
}

// Recompress A B^T (A: nr x k, B: nc x k) to the smallest rank with sigma_i > tol sigma_1.
void recompress(const std::vector<double>& A, const std::vector<double>& B, int nr, int nc, int k,
                double tol, RkBlock& out) {
  std::vector<double> Qa, Ra, Qb, Rb;
  int ra, rb;
  householder_qr(A, nr, k, Qa, Ra, ra);
  householder_qr(B, nc, k, Qb, Rb, rb);
  // S = Ra Rb^T (ra x rb)
  std::vector<double> S((size_t)ra * rb, 0.0);
  for (int i = 0; i < ra; ++i)
    for (int j = 0; j < rb; ++j) {
      double s = 0.0;
      for (int c = 0; c < k; ++c) s += Ra[(size_t)i * k + c] * Rb[(size_t)j * k + c];
      S[(size_t)i * rb + j] = s;
    }
  std::vector<double> V;
  jacobi_svd(S, ra, rb, V);
  std::vector<double> sig(rb);
  for (int j = 0; j < rb; ++j) {
    double s = 0.0;
    for (int r = 0; r < ra; ++r) s += S[(size_t)r * rb + j] * S[(size_t)r * rb + j];
    sig[j] = std::sqrt(s);
  }
  std::vector<int> order(rb);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return sig[x] > sig[y]; });
  double smax = rb ? sig[order[0]] : 0.0;
  int kk = 0;
  while (kk < rb && sig[order[kk]] > tol * smax) ++kk;
  if (kk == 0) kk = 1;
  out.k = kk;
  out.U.assign((size_t)nr * kk, 0.0);
  out.V.assign((size_t)nc * kk, 0.0);
  for (int c = 0; c < kk; ++c) {
    int j = order[c];
    // U column = Qa * (sigma_j u_j), stored unnormalised in S's column j
    for (int r = 0; r < nr; ++r) {
      double s = 0.0;
      for (int i = 0; i < ra; ++i) s += Qa[(size_t)r * ra + i] * S[(size_t)i * rb + j];
      out.U[(size_t)r * kk + c] = s;
    }
    for (int r = 0; r < nc; ++r) {
      double s = 0.0;
      for (int i = 0; i < rb; ++i) s += Qb[(size_t)r * rb + i] * V[(size_t)i * rb + j];
      out.V[(size_t)r * kk + c] = s;
    }
  }
}

// Adaptive cross approximation with partial pivoting (Bebendorf): A B^T of the block of R with rows
// r0..r1-1 and columns c0..c1-1 from single accurate entries, no kernel expansion.  Step k takes the
// residual row at the pivot row i, its largest entry's column j, and the residual column j (scaled
// by the pivot), and stops when |u_k| |v_k| <= eps |sum_l u_l v_l^T|_F (the norm updated
// incrementally); the next pivot row is the largest unused entry of u_k.
void aca_factors(const std::vector<double>& t, double alpha, int r0, int r1, int c0, int c1, double eps, int kmax,
                 std::vector<double>& A, std::vector<double>& B, int& k) {
  const int nr = r1 - r0, nc = c1 - c0;
  std::vector<std::vector<double>> us, vs;
  std::vector<char> row_used(nr, 0), col_used(nc, 0);
  auto entry = [&](int r, int c) { return l1_entry(t, alpha, r0 + r + 1, c0 + c + 1); };
  double norm2 = 0.0;
  int i = 0;
  for (int step = 0; step < kmax; ++step) {
    std::vector<double> v(nc);
    for (int c = 0; c < nc; ++c) {
      double x = entry(i, c);
      for (size_t l = 0; l < us.size(); ++l) x -= us[l][i] * vs[l][c];
      v[c] = x;
    }
    row_used[i] = 1;
    int j = -1;
    double vmax = 0.0;
    for (int c = 0; c < nc; ++c)
      if (!col_used[c] && std::fabs(v[c]) > vmax) {
        vmax = std::fabs(v[c]);
        j = c;
      }
    if (j < 0 || vmax == 0.0) {  // this residual row vanishes: try the next unused row
      int next = -1;
      for (int r = 0; r < nr && next < 0; ++r)
        if (!row_used[r]) next = r;
      if (next < 0) break;
      i = next;
      continue;
    }
    col_used[j] = 1;
    const double piv = v[j];
    for (double& x : v) x /= piv;
    std::vector<double> u(nr);
    for (int r = 0; r < nr; ++r) {
      double x = entry(r, j);
      for (size_t l = 0; l < us.size(); ++l) x -= vs[l][j] * us[l][r];
      u[r] = x;
    }
    double uu = 0.0, vv = 0.0;
    for (double x : u) uu += x * x;
    for (double x : v) vv += x * x;
    for (size_t l = 0; l < us.size(); ++l) {
      double uul = 0.0, vvl = 0.0;
      for (int r = 0; r < nr; ++r) uul += u[r] * us[l][r];
      for (int c = 0; c < nc; ++c) vvl += v[c] * vs[l][c];
      norm2 += 2.0 * uul * vvl;
    }
    norm2 += uu * vv;
    us.push_back(u);
    vs.push_back(v);
    if (std::sqrt(uu * vv) <= eps * std::sqrt(std::max(norm2, 0.0))) break;
    int inext = -1;
    double umax = -1.0;
    for (int r = 0; r < nr; ++r)
      if (!row_used[r] && std::fabs(u[r]) > umax) {
        umax = std::fabs(u[r]);
        inext = r;
      }
    if (inext < 0) break;
    i = inext;
  }
  k = (int)us.size();
  if (k == 0) {  // an all-zero block: one zero term
    us.assign(1, std::vector<double>(nr, 0.0));
    vs.assign(1, std::vector<double>(nc, 0.0));
    k = 1;
  }
  A.assign((size_t)nr * k, 0.0);
  B.assign((size_t)nc * k, 0.0);
  for (int l = 0; l < k; ++l) {
    for (int r = 0; r < nr; ++r) A[(size_t)r * k + l] = us[l][r];
    for (int c = 0; c < nc; ++c) B[(size_t)c * k + l] = vs[l][c];
  }
}

}  // namespace

int build_hmatrix(double alpha, double gamma, double T, int M, int leaf, int rank, double tol,
                  HostH& h, int lowrank) {
  if (!(alpha > 0.0 && alpha < 1.0) || !(gamma >= 1.0) || !(T > 0.0) || M < 1 || leaf < 1 ||
      rank < 0 || !(tol >= 0.0) || rank > 64 || (lowrank == 1 && !(rank == 0 && tol > 0.0)))
    return -1;
  int L = std::min(leaf, M);
  if (M % L) return -1;
  int nb = M / L;
  if (nb & (nb - 1)) return -1;  // index bisection down to the leaf needs M / L = 2^p
  if (L > 128) return -1;
  h = HostH();
  h.alpha = alpha;
  h.gamma = gamma;
  h.T = T;
  h.M = M;
  h.L = L;
  h.nb = nb;
  h.rank = rank;
  h.tol = tol;
  h.dense_mode = (rank == 0 && tol == 0.0);
  h.t.resize(M + 1);
  for (int m = 0; m <= M; ++m) h.t[m] = T * std::pow((double)m / M, gamma);
  h.t[M] = T;
  h.dmm.resize(M);
  for (int m = 1; m <= M; ++m) h.dmm[m - 1] = Dfun(h.t, alpha, m, 1);

  Rec rec{h.t, M, L, h.dense_mode, {}, {}};
  recurse(rec, 0, M, 0, M);

  // dense leaves (exact entries)
  h.diag.assign(nb, -1);
  for (auto& b : rec.dense) {
    DenseBlock db;
    db.bi = b[0] / L;
    db.bj = b[2] / L;
    db.D.assign((size_t)L * L, 0.0);
    for (int r = 0; r < L; ++r)
      for (int c = 0; c < L; ++c) {
        int m = b[0] + r + 1, j = b[2] + c + 1;
        if (j <= m) db.D[(size_t)r * L + c] = l1_entry(h.t, alpha, m, j);
      }
    if (db.bi == db.bj) h.diag[db.bi] = (int)h.dense.size();
    h.dense.push_back(std::move(db));
  }
  // low-rank blocks
  int kt = rank;
  if (rank == 0 && tol > 0.0) {
    kt = 1;
    while (kt < 48 && std::pow(3.0, -kt) * (1.5 * (alpha + kt) + 0.75) > 0.01 * tol) ++kt;
  }
  h.taylor_terms = kt;
  for (auto& b : rec.rk) {
    RkBlock rb;
    rb.r0 = b[0];
    rb.r1 = b[1];
    rb.c0 = b[2];
    rb.c1 = b[3];
    std::vector<double> A, B;
    if (lowrank == 1) {
      int ka = 0;
      aca_factors(h.t, alpha, b[0], b[1], b[2], b[3], 0.01 * tol, std::min(64, std::min(b[1] - b[0], b[3] - b[2])), A,
                  B, ka);
      recompress(A, B, b[1] - b[0], b[3] - b[2], ka, tol, rb);
      h.max_rank = std::max(h.max_rank, rb.k);
      h.rk.push_back(std::move(rb));
      continue;
    }
    taylor_factors(h.t, alpha, b[0], b[1], b[2], b[3], kt, A, B);
    if (rank > 0) {
      rb.k = kt;
      rb.U = std::move(A);
      rb.V = std::move(B);
    } else {
      recompress(A, B, b[1] - b[0], b[3] - b[2], kt, tol, rb);
    }
    h.max_rank = std::max(h.max_rank, rb.k);
    h.rk.push_back(std::move(rb));
  }
  return 0;
}

void flatten(const HostH& h, FlatH& f) {
  const int L = h.L, nb = h.nb;
  f = FlatH();
  f.M = h.M;
  f.L = L;
  f.nb = nb;
  // dense
  f.dense_data.reserve(h.dense.size() * (size_t)L * L);
  for (auto& d : h.dense) f.dense_data.insert(f.dense_data.end(), d.D.begin(), d.D.end());
  std::vector<std::vector<std::pair<int, int>>> rows(nb);
  for (int b = 0; b < (int)h.dense.size(); ++b)
    if (h.dense[b].bj < h.dense[b].bi) rows[h.dense[b].bi].push_back({h.dense[b].bj, b});
  f.dptr.assign(nb + 1, 0);
  for (int i = 0; i < nb; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    for (auto& p : rows[i]) {
      f.dlist_col.push_back(p.first);
      f.dlist_blk.push_back(p.second);
    }
    f.dptr[i + 1] = (int)f.dlist_col.size();
  }
  f.diag_blk = h.diag;
  // z-pool: live range of block b is [c0/L, r1/L - 1]; rows may be reused by a block that
  // starts at the leaf where another one is last read (reads precede writes in a leaf step).
  int nrk = (int)h.rk.size();
  std::vector<int> order(nrk), zbase(nrk, 0);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return h.rk[x].c0 < h.rk[y].c0; });
  std::vector<int> row_end;  // per pool row: last leaf at which it is read (-1 = free)
  for (int b : order) {
    int s = h.rk[b].c0 / L, e = h.rk[b].r1 / L - 1, k = h.rk[b].k;
    int base = -1;
    for (int r0 = 0; r0 + k <= (int)row_end.size() && base < 0; ++r0) {
      bool ok = true;
      for (int r = r0; r < r0 + k && ok; ++r) ok = row_end[r] <= s;
      if (ok) base = r0;
    }
    if (base < 0) {
      // extend: reuse a free tail if any
      int tail = (int)row_end.size();
      while (tail > 0 && row_end[tail - 1] <= s) --tail;
      base = tail;
      if ((int)row_end.size() < base + k) row_end.resize(base + k, -1);
    }
    for (int r = base; r < base + k; ++r) row_end[r] = e;
    zbase[b] = base;
  }
  f.pool_rows = (int)row_end.size();
  // U panels
  f.uptr.assign(nb + 1, 0);
  f.uoff.assign(nb, 0);
  f.vptr.assign(nb + 1, 0);
  f.voff.assign(nb, 0);
  for (int i = 0; i < nb; ++i) {
    std::vector<int> cov;
    for (int b = 0; b < nrk; ++b)
      if (h.rk[b].r0 <= i * L && i * L < h.rk[b].r1) cov.push_back(b);
    int K = 0;
    for (int b : cov) K += h.rk[b].k;
    f.uoff[i] = (long long)f.udata.size();
    f.udata.resize(f.udata.size() + (size_t)L * K, 0.0);
    int col = 0;
    for (int b : cov) {
      const RkBlock& B = h.rk[b];
      for (int nu = 0; nu < B.k; ++nu, ++col) {
        f.uz.push_back(zbase[b] + nu);
        for (int r = 0; r < L; ++r)
          f.udata[f.uoff[i] + (size_t)r * K + col] = B.U[(size_t)(i * L - B.r0 + r) * B.k + nu];
      }
    }
    f.uptr[i + 1] = (int)f.uz.size();
    // V panels
    std::vector<int> vc;
    for (int b = 0; b < nrk; ++b)
      if (h.rk[b].c0 <= i * L && i * L < h.rk[b].c1) vc.push_back(b);
    f.voff[i] = (long long)f.vdata.size();
    for (int b : vc) {
      const RkBlock& B = h.rk[b];
      for (int nu = 0; nu < B.k; ++nu) {
        f.vz.push_back(zbase[b] + nu);
        f.vinit.push_back(B.c0 == i * L ? 1 : 0);
        for (int c = 0; c < L; ++c) f.vdata.push_back(B.V[(size_t)(i * L - B.c0 + c) * B.k + nu]);
      }
    }
    f.vptr[i + 1] = (int)f.vz.size();
  }
  long long fl = 0;
  for (int i = 0; i < nb; ++i)
    fl += (long long)(f.dptr[i + 1] - f.dptr[i]) * L * L + (long long)L * (L + 1) / 2 +
          (long long)(f.uptr[i + 1] - f.uptr[i]) * L + (long long)(f.vptr[i + 1] - f.vptr[i]) * L;
  f.flops_per_col_matvec = 2 * fl;
  f.flops_per_col_solve = 2 * fl;
}

void diag_inverses(const HostH& h, const FlatH& f, double shift, std::vector<double>& out) {
  const int L = f.L;
  out.assign((size_t)f.nb * L * L, 0.0);
  for (int i = 0; i < f.nb; ++i) {
    const std::vector<double>& D = h.dense[f.diag_blk[i]].D;
    double* X = &out[(size_t)i * L * L];
    for (int c = 0; c < L; ++c) {
      // solve (D + shift I) x = e_c; x_r = 0 for r < c
      X[(size_t)c * L + c] = 1.0 / (D[(size_t)c * L + c] + shift);
      for (int r = c + 1; r < L; ++r) {
        double s = 0.0;
        for (int k = c; k < r; ++k) s += D[(size_t)r * L + k] * X[(size_t)k * L + c];
        X[(size_t)r * L + c] = -s / (D[(size_t)r * L + r] + shift);
      }
    }
  }
}

}  // namespace fhmg

namespace fhmg {
namespace {

void put_value(std::vector<unsigned char>& b, size_t off, double v, int elem_bytes) {
  if (elem_bytes == 8) {
    std::memcpy(&b[off], &v, 8);
  } else {
    float x = (float)v;
    std::memcpy(&b[off], &x, 4);
  }
}

size_t pad16(size_t n) { return (n + 15) & ~(size_t)15; }

}  // namespace

void build_panel(const HostH& h, const FlatH& f, int eb, PanelHost& out) {
  const int L = f.L, nb = f.nb;
  const int VE = 16 / eb;  // elements per 16-byte vector
  out = PanelHost();
  out.cptr.assign(nb + 1, 0);
  int maxdist = 0;
  for (int i = 0; i < nb; ++i)
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) maxdist = std::max(maxdist, i - f.dlist_col[d]);
  out.W = std::min(8, maxdist + 1);
  auto add_chunk = [&](int type, int count, int aux, size_t bytes) -> size_t {
    size_t off = out.pkg.size();
    size_t nbytes = pad16(bytes);
    out.pkg.resize(off + nbytes, 0);
    out.chunks.push_back(type | (count << 4));
    out.chunks.push_back(aux);
    out.chunks.push_back((int)nbytes);
    out.chunks.push_back((int)(off / 16));
    out.slot_bytes = std::max(out.slot_bytes, (int)nbytes);
    return off;
  };
  // entry (k, r) of a chunk matrix with R rows, k the reduction index
  auto at = [&](size_t off, int k, int r, int R) { return off + (((size_t)(k / VE) * R + r) * VE + k % VE) * eb; };
  auto put_square = [&](const double* D, size_t off, bool zero_diag) {
    for (int k = 0; k < L; ++k)
      for (int r = 0; r < L; ++r)
        put_value(out.pkg, at(off, k, r, L), (zero_diag && k == r) ? 0.0 : D[(size_t)r * L + k], eb);
  };
  for (int i = 0; i < nb; ++i) {
    // near-field blocks
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) {
      size_t off = add_chunk(CH_DENSE, L, f.dlist_col[d], (size_t)L * L * eb);
      put_square(&f.dense_data[(size_t)f.dlist_blk[d] * L * L], off, false);
    }
    // U panel (row-major L x K in FlatH) in slabs of up to L columns, padded with zero columns to
    // whole vectors (their z index repeats the slab's first one)
    const int K = f.uptr[i + 1] - f.uptr[i];
    for (int k0 = 0; k0 < K; k0 += L) {
      const int kc = std::min(L, K - k0);
      const int kp = (kc + VE - 1) / VE * VE;
      size_t off = add_chunk(CH_UPART, kp, k0, (size_t)kp * L * eb + (size_t)kp * 4);
      for (int kk = 0; kk < kc; ++kk)
        for (int r = 0; r < L; ++r)
          put_value(out.pkg, at(off, kk, r, L), f.udata[f.uoff[i] + (size_t)r * K + k0 + kk], eb);
      for (int kk = 0; kk < kp; ++kk) {
        int z = f.uz[f.uptr[i] + k0 + (kk < kc ? kk : 0)];
        std::memcpy(&out.pkg[off + (size_t)kp * L * eb + (size_t)kk * 4], &z, 4);
      }
    }
    // diagonal block (FP32 streams carry it without its diagonal, which the kernels apply in
    // the grid functions' precision)
    {
      size_t off = add_chunk(CH_DIAG, L, i, (size_t)L * L * eb);
      put_square(&f.dense_data[(size_t)f.diag_blk[i] * L * L], off, eb == 4);
    }
    // V panel (row-major K' x L in FlatH) in slabs of up to L rows; the slab's rows are the
    // outputs, its columns the reduction index
    const int Kv = f.vptr[i + 1] - f.vptr[i];
    for (int k0 = 0; k0 < Kv; k0 += L) {
      const int kc = std::min(L, Kv - k0);
      size_t off = add_chunk(CH_VPART, kc, k0, (size_t)kc * L * eb + (size_t)kc * 4);
      for (int kk = 0; kk < kc; ++kk)
        for (int c = 0; c < L; ++c)
          put_value(out.pkg, at(off, c, kk, kc), f.vdata[f.voff[i] + (size_t)(k0 + kk) * L + c], eb);
      for (int kk = 0; kk < kc; ++kk) {
        int code = 2 * f.vz[f.vptr[i] + k0 + kk] + f.vinit[f.vptr[i] + k0 + kk];
        std::memcpy(&out.pkg[off + (size_t)kc * L * eb + (size_t)kk * 4], &code, 4);
      }
    }
    out.chunks[out.chunks.size() - 4] |= 1 << 12;  // the leaf row's last chunk
    out.cptr[i + 1] = (int)(out.chunks.size() / 4);
  }
}

namespace {

// round to the nearest TF32 value (10 explicit mantissa bits), ties away from zero
float tf32_round(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7f800000u) != 0x7f800000u) b = (b + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// float index of part hl of entry (r, k) in the fragment layout of an R x K chunk matrix
size_t mma_index(int r, int k, int nkb, int hl) {
  const int rt = r / 16, half = (r % 16) / 8, g = r % 8;
  const int kb = k / 16, t = (k % 16) / 4, e = k % 4;
  const int lane = g * 4 + t;
  return (((((size_t)rt * nkb + kb) * 2 + hl) * 2 + half) * 32 + lane) * 4 + e;
}

void put_mma(std::vector<unsigned char>& pkg, size_t off, int r, int k, int nkb, double v) {
  const float hi = tf32_round((float)v);
  const float lo = tf32_round((float)(v - (double)hi));
  std::memcpy(&pkg[off + mma_index(r, k, nkb, 0) * 4], &hi, 4);
  std::memcpy(&pkg[off + mma_index(r, k, nkb, 1) * 4], &lo, 4);
}

}  // namespace

void build_panel_mma(const HostH& h, const FlatH& f, PanelHost& out) {
  const int L = f.L, nb = f.nb;
  const int nkbL = (L + 15) / 16;
  out = PanelHost();
  out.cptr.assign(nb + 1, 0);
  int maxdist = 0;
  for (int i = 0; i < nb; ++i)
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) maxdist = std::max(maxdist, i - f.dlist_col[d]);
  out.W = std::min(8, maxdist + 1);
  out.far = maxdist + 1 > out.W;
  auto add_chunk = [&](int type, int count, int aux, size_t bytes) -> size_t {
    size_t off = out.pkg.size();
    size_t nbytes = pad16(bytes);
    out.pkg.resize(off + nbytes, 0);
    out.chunks.push_back(type | (count << 4));
    out.chunks.push_back(aux);
    out.chunks.push_back((int)nbytes);
    out.chunks.push_back((int)(off / 16));
    out.slot_bytes = std::max(out.slot_bytes, (int)nbytes);
    return off;
  };
  const size_t sq = (size_t)nkbL * 16 * nkbL * 16 * 2 * 4;  // padded L x L, hi + lo
  auto put_square = [&](const double* D, size_t off, bool zero_diag) {
    for (int r = 0; r < L; ++r)
      for (int k = 0; k < L; ++k) put_mma(out.pkg, off, r, k, nkbL, (zero_diag && k == r) ? 0.0 : D[(size_t)r * L + k]);
  };
  for (int i = 0; i < nb; ++i) {
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) {
      size_t off = add_chunk(CH_DENSE, L, f.dlist_col[d], sq);
      put_square(&f.dense_data[(size_t)f.dlist_blk[d] * L * L], off, false);
    }
    const int K = f.uptr[i + 1] - f.uptr[i];
    for (int k0 = 0; k0 < K; k0 += L) {
      const int kc = std::min(L, K - k0);
      const int kp = (kc + 15) / 16 * 16;
      const size_t mat = (size_t)nkbL * 16 * kp * 2 * 4;
      size_t off = add_chunk(CH_UPART, kp, k0, mat + (size_t)kp * 4);
      for (int r = 0; r < L; ++r)
        for (int kk = 0; kk < kc; ++kk) put_mma(out.pkg, off, r, kk, kp / 16, f.udata[f.uoff[i] + (size_t)r * K + k0 + kk]);
      for (int kk = 0; kk < kp; ++kk) {
        int z = f.uz[f.uptr[i] + k0 + (kk < kc ? kk : 0)];
        std::memcpy(&out.pkg[off + mat + (size_t)kk * 4], &z, 4);
      }
    }
    {
      size_t off = add_chunk(CH_DIAG, L, i, sq);
      put_square(&f.dense_data[(size_t)f.diag_blk[i] * L * L], off, true);
    }
    const int Kv = f.vptr[i + 1] - f.vptr[i];
    for (int k0 = 0; k0 < Kv; k0 += L) {
      const int kc = std::min(L, Kv - k0);
      const int rp = (kc + 15) / 16 * 16;
      const size_t mat = (size_t)rp * nkbL * 16 * 2 * 4;
      size_t off = add_chunk(CH_VPART, kc, k0, mat + (size_t)kc * 4);
      for (int kk = 0; kk < kc; ++kk)
        for (int c = 0; c < L; ++c) put_mma(out.pkg, off, kk, c, nkbL, f.vdata[f.voff[i] + (size_t)(k0 + kk) * L + c]);
      for (int kk = 0; kk < kc; ++kk) {
        int code = 2 * f.vz[f.vptr[i] + k0 + kk] + f.vinit[f.vptr[i] + k0 + kk];
        std::memcpy(&out.pkg[off + mat + (size_t)kk * 4], &code, 4);
      }
    }
    out.chunks[out.chunks.size() - 4] |= 1 << 12;
    out.cptr[i + 1] = (int)(out.chunks.size() / 4);
  }
}

void build_panel_df(const HostH& h, const FlatH& f, PanelHost& out) {
  const int L = f.L, nb = f.nb;
  out = PanelHost();
  out.cptr.assign(nb + 1, 0);
  int maxdist = 0;
  for (int i = 0; i < nb; ++i)
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) maxdist = std::max(maxdist, i - f.dlist_col[d]);
  out.W = std::min(8, maxdist + 1);
  out.far = maxdist + 1 > out.W;
  auto add_chunk = [&](int type, int count, int aux, size_t bytes) -> size_t {
    size_t off = out.pkg.size();
    size_t nbytes = pad16(bytes);
    out.pkg.resize(off + nbytes, 0);
    out.chunks.push_back(type | (count << 4));
    out.chunks.push_back(aux);
    out.chunks.push_back((int)nbytes);
    out.chunks.push_back((int)(off / 16));
    out.slot_bytes = std::max(out.slot_bytes, (int)nbytes);
    return off;
  };
  // entry (k, r) of an R x K chunk matrix: hi at float index ((k/4) R + r) 4 + k%4 of the hi block,
  // lo at the same index of the lo block that follows it (R K floats later)
  auto put = [&](size_t off, int k, int r, int R, int K, double v) {
    const float hi = (float)v;
    const float lo = (float)(v - (double)hi);
    const size_t idx = ((size_t)(k / 4) * R + r) * 4 + k % 4;
    std::memcpy(&out.pkg[off + idx * 4], &hi, 4);
    std::memcpy(&out.pkg[off + ((size_t)R * K + idx) * 4], &lo, 4);
  };
  for (int i = 0; i < nb; ++i) {
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) {
      const double* D = &f.dense_data[(size_t)f.dlist_blk[d] * L * L];
      size_t off = add_chunk(CH_DENSE, L, f.dlist_col[d], (size_t)L * L * 8);
      for (int k = 0; k < L; ++k)
        for (int r = 0; r < L; ++r) put(off, k, r, L, L, D[(size_t)r * L + k]);
    }
    const int K = f.uptr[i + 1] - f.uptr[i];
    for (int k0 = 0; k0 < K; k0 += L) {
      const int kc = std::min(L, K - k0);
      const int kp = (kc + 3) / 4 * 4;
      size_t off = add_chunk(CH_UPART, kp, k0, (size_t)kp * L * 8 + (size_t)kp * 4);
      for (int kk = 0; kk < kc; ++kk)
        for (int r = 0; r < L; ++r) put(off, kk, r, L, kp, f.udata[f.uoff[i] + (size_t)r * K + k0 + kk]);
      for (int kk = 0; kk < kp; ++kk) {
        int z = f.uz[f.uptr[i] + k0 + (kk < kc ? kk : 0)];
        std::memcpy(&out.pkg[off + (size_t)kp * L * 8 + (size_t)kk * 4], &z, 4);
      }
    }
    {
      const double* D = &f.dense_data[(size_t)f.diag_blk[i] * L * L];
      size_t off = add_chunk(CH_DIAG, L, i, (size_t)L * L * 8);
      for (int k = 0; k < L; ++k)
        for (int r = 0; r < L; ++r) put(off, k, r, L, L, D[(size_t)r * L + k]);
    }
    const int Kv = f.vptr[i + 1] - f.vptr[i];
    for (int k0 = 0; k0 < Kv; k0 += L) {
      const int kc = std::min(L, Kv - k0);
      size_t off = add_chunk(CH_VPART, kc, k0, (size_t)kc * L * 8 + (size_t)kc * 4);
      for (int kk = 0; kk < kc; ++kk)
        for (int c = 0; c < L; ++c) put(off, c, kk, kc, L, f.vdata[f.voff[i] + (size_t)(k0 + kk) * L + c]);
      for (int kk = 0; kk < kc; ++kk) {
        int code = 2 * f.vz[f.vptr[i] + k0 + kk] + f.vinit[f.vptr[i] + k0 + kk];
        std::memcpy(&out.pkg[off + (size_t)kc * L * 8 + (size_t)kk * 4], &code, 4);
      }
    }
    out.chunks[out.chunks.size() - 4] |= 1 << 12;
    out.cptr[i + 1] = (int)(out.chunks.size() / 4);
  }
}

namespace {

// BF16 bits of v, round to nearest even (finite values)
uint16_t bf16_bits(double v) {
  const float x = (float)v;
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7f800000u) != 0x7f800000u) b += 0x7fffu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}

}  // namespace

size_t umma_offset(int r, int k, int K) {
  return ((size_t)(r / 8) * (K / 8) + k / 8) * 128 + (size_t)(r % 8) * 16 + (size_t)(k % 8) * 2;
}

void build_panel_umma(const HostH& h, const FlatH& f, PanelHost& out) {
  const int L = f.L, nb = f.nb;
  out = PanelHost();
  out.cptr.assign(nb + 1, 0);
  int maxdist = 0;
  for (int i = 0; i < nb; ++i)
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) maxdist = std::max(maxdist, i - f.dlist_col[d]);
  out.W = std::min(8, maxdist + 1);
  out.far = maxdist + 1 > out.W;
  auto add_chunk = [&](int type, int count, int aux, size_t bytes) -> size_t {
    size_t off = out.pkg.size();
    size_t nbytes = pad16(bytes);
    out.pkg.resize(off + nbytes, 0);
    out.chunks.push_back(type | (count << 4));
    out.chunks.push_back(aux);
    out.chunks.push_back((int)nbytes);
    out.chunks.push_back((int)(off / 16));
    out.slot_bytes = std::max(out.slot_bytes, (int)nbytes);
    return off;
  };
  auto put = [&](size_t off, int r, int k, int K, double v) {
    const uint16_t b = bf16_bits(v);
    std::memcpy(&out.pkg[off + umma_offset(r, k, K)], &b, 2);
  };
  for (int i = 0; i < nb; ++i) {
    for (int d = f.dptr[i]; d < f.dptr[i + 1]; ++d) {
      const double* D = &f.dense_data[(size_t)f.dlist_blk[d] * L * L];
      size_t off = add_chunk(CH_DENSE, L, f.dlist_col[d], (size_t)L * L * 2);
      for (int r = 0; r < L; ++r)
        for (int k = 0; k < L; ++k) put(off, r, k, L, D[(size_t)r * L + k]);
    }
    const int K = f.uptr[i + 1] - f.uptr[i];
    for (int k0 = 0; k0 < K; k0 += L) {
      const int kc = std::min(L, K - k0);
      const int kp = (kc + 15) / 16 * 16;
      const size_t mat = (size_t)L * kp * 2;
      size_t off = add_chunk(CH_UPART, kp, k0, mat + (size_t)kp * 4);
      for (int r = 0; r < L; ++r)
        for (int kk = 0; kk < kc; ++kk) put(off, r, kk, kp, f.udata[f.uoff[i] + (size_t)r * K + k0 + kk]);
      for (int kk = 0; kk < kp; ++kk) {
        int z = f.uz[f.uptr[i] + k0 + (kk < kc ? kk : 0)];
        std::memcpy(&out.pkg[off + mat + (size_t)kk * 4], &z, 4);
      }
    }
    {
      const double* D = &f.dense_data[(size_t)f.diag_blk[i] * L * L];
      size_t off = add_chunk(CH_DIAG, L, i, (size_t)L * L * 2);
      for (int r = 0; r < L; ++r)
        for (int k = 0; k < L; ++k) put(off, r, k, L, k == r ? 0.0 : D[(size_t)r * L + k]);
    }
    const int Kv = f.vptr[i + 1] - f.vptr[i];
    for (int k0 = 0; k0 < Kv; k0 += L) {
      const int kc = std::min(L, Kv - k0);
      const int rp = (kc + 15) / 16 * 16;
      const size_t mat = (size_t)rp * L * 2;
      size_t off = add_chunk(CH_VPART, kc, k0, mat + (size_t)kc * 4);
      for (int kk = 0; kk < kc; ++kk)
        for (int c = 0; c < L; ++c) put(off, kk, c, L, f.vdata[f.voff[i] + (size_t)(k0 + kk) * L + c]);
      for (int kk = 0; kk < kc; ++kk) {
        int code = 2 * f.vz[f.vptr[i] + k0 + kk] + f.vinit[f.vptr[i] + k0 + kk];
        std::memcpy(&out.pkg[off + mat + (size_t)kk * 4], &code, 4);
      }
    }
    out.chunks[out.chunks.size() - 4] |= 1 << 12;
    out.cptr[i + 1] = (int)(out.chunks.size() / 4);
  }
}

void to_umma_layout(const double* A, int L, bool zero_diag, uint16_t* out) {
  for (int r = 0; r < L; ++r)
    for (int k = 0; k < L; ++k) out[umma_offset(r, k, L) / 2] = bf16_bits((zero_diag && k == r) ? 0.0 : A[(size_t)r * L + k]);
}

void build_split(const std::vector<double>& R, int M, SplitHost& out) {
  constexpr int G = 7, TR = 128, TK = 64;
  const int nI = M / TR;
  out.tiles.clear();
  out.pairs.clear();
  out.rexp.assign(M, 0);
  // digits of every entry, row-major per digit
  std::vector<int> dig((size_t)G * M * M, 0);
  for (int m = 0; m < M; ++m) {
    double mx = 0.0;
    for (int k = 0; k <= m; ++k) mx = std::max(mx, std::fabs(R[(size_t)m * M + k]));
    int E = 0;
    if (mx > 0.0) std::frexp(mx, &E);
    out.rexp[m] = E;
    for (int k = 0; k <= m; ++k) {
      long long X = std::llrint(std::ldexp(R[(size_t)m * M + k], 49 - E));
      for (int a = G - 1; a >= 1; --a) {
        const long long d = ((X + 64) & 127) - 64;
        dig[((size_t)a * M + m) * M + k] = (int)d;
        X = (X - d) / 128;
      }
      dig[(size_t)m * M + k] = (int)X;
    }
  }
  const size_t tile_elems = (size_t)TR * TK;
  for (int I = 0; I < nI; ++I)
    for (int J = 0; J <= 2 * I + 1; ++J) {
      int mask = 0;
      const int first = (int)(out.tiles.size() / tile_elems);
      for (int a = 0; a < G; ++a) {
        bool any = false;
        for (int r = 0; r < TR && !any; ++r)
          for (int kk = 0; kk < TK; ++kk)
            if (dig[((size_t)a * M + I * TR + r) * M + J * TK + kk] != 0) {
              any = true;
              break;
            }
        if (!any) continue;
        mask |= 1 << a;
        const size_t base = out.tiles.size();
        out.tiles.resize(base + tile_elems, 0);
        for (int r = 0; r < TR; ++r)
          for (int kk = 0; kk < TK; ++kk) {
            const int d = dig[((size_t)a * M + I * TR + r) * M + J * TK + kk];
            // K-major, 128-byte swizzle: 16-byte chunk c of row r at chunk position c ^ (r % 8)
            const size_t off = (size_t)(r / 8) * 1024 + (r % 8) * 128 + (size_t)(((kk / 8) ^ (r % 8)) & 7) * 16 + (kk % 8) * 2;
            out.tiles[base + off / 2] = bf16_bits((double)d);
          }
      }
      out.pairs.insert(out.pairs.end(), {mask, first, 0, 0});
    }
}

void to_mma_layout(const double* A, int L, bool zero_diag, float* out) {
  const int nkb = (L + 15) / 16;
  std::vector<unsigned char> buf((size_t)nkb * 16 * nkb * 16 * 2 * 4, 0);
  for (int r = 0; r < L; ++r)
    for (int k = 0; k < L; ++k) put_mma(buf, 0, r, k, nkb, (zero_diag && k == r) ? 0.0 : A[(size_t)r * L + k]);
  std::memcpy(out, buf.data(), buf.size());
}

void to_panel_layout(const double* A, int L, int eb, bool zero_diag, double* out) {
  const int VE = 16 / eb;
  for (int k = 0; k < L; ++k)
    for (int r = 0; r < L; ++r)
      out[((size_t)(k / VE) * L + r) * VE + k % VE] = (zero_diag && k == r) ? 0.0 : A[(size_t)r * L + k];
}

}  // namespace fhmg
