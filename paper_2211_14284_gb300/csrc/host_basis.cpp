// 1D FDM bases (Sec. 2.2-2.3): GLL nodes by Newton iteration, barycentric
// Lagrange interpolation, the generalised eigenproblem of Eq. eigs solved by
// a Cholesky reduction and cyclic Jacobi rotations, the interface functions
// from the duality condition (Eq. unisolvence), and the differentiation
// matrix D_ij = (r_i, s_j') in closed form from A-hat and lambda.
#include "host_basis.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace rm {

namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double &P, double &dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  // derivative from (x^2 - 1) P_n' = n (x P_n - P_{n-1})
  if (std::fabs(x) < 1.0)
    dP = n * (x * p1 - p0) / (x * x - 1.0);
  else
    dP = (x > 0 ? 1.0 : ((n % 2) ? 1.0 : -1.0)) * 0.5 * n * (n + 1.0);
}

// Barycentric weights of the nodes.
std::vector<double> bary_weights(const std::vector<double> &nodes) {
  int n = (int)nodes.size();
  std::vector<double> w(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) w[j] /= (nodes[j] - nodes[m]);
  return w;
}

// Values and derivatives of all Lagrange polynomials at one point.
void lagrange_at(const std::vector<double> &nodes, const std::vector<double> &bw,
                 double x, double *L, double *dL) {
  int n = (int)nodes.size();
  int hit = -1;
  for (int j = 0; j < n; ++j)
    if (x == nodes[j]) hit = j;
  if (hit >= 0) {
    // at a node: l_j = delta, l_j'(x_i) from the differentiation matrix
    for (int j = 0; j < n; ++j) L[j] = (j == hit) ? 1.0 : 0.0;
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == hit) continue;
      dL[j] = (bw[j] / bw[hit]) / (nodes[hit] - nodes[j]);
      diag -= dL[j];
    }
    dL[hit] = diag;
    return;
  }
  double den = 0.0;
  for (int j = 0; j < n; ++j) den += bw[j] / (x - nodes[j]);
  for (int j = 0; j < n; ++j) {
    L[j] = (bw[j] / (x - nodes[j])) / den;
    double s = 0.0;
    for (int m = 0; m < n; ++m)
      if (m != j) s += 1.0 / (x - nodes[m]);
    dL[j] = L[j] * s;
  }
}

// In-place Cholesky of a dense SPD n x n (row-major), lower factor.
void chol(std::vector<double> &A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (d <= 0) throw std::runtime_error("basis: mass matrix not SPD");
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
    for (int i = 0; i < j; ++i) A[i * n + j] = 0.0;
  }
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix: C = W diag W^T.
void jacobi_eig(std::vector<double> C, int n, std::vector<double> &ev,
                std::vector<double> &W) {
  W.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) W[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += C[i * n + j] * C[i * n + j];
        if (i != j) off += C[i * n + j] * C[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b) {
        double cab = C[a * n + b];
        if (std::fabs(cab) < 1e-300) continue;
        double theta = (C[b * n + b] - C[a * n + a]) / (2.0 * cab);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns a, b
          double ka = C[k * n + a], kb = C[k * n + b];
          C[k * n + a] = c * ka - s * kb;
          C[k * n + b] = s * ka + c * kb;
        }
        for (int k = 0; k < n; ++k) {  // rows a, b
          double ak = C[a * n + k], bk = C[b * n + k];
          C[a * n + k] = c * ak - s * bk;
          C[b * n + k] = s * ak + c * bk;
        }
        for (int k = 0; k < n; ++k) {
          double ka = W[k * n + a], kb = W[k * n + b];
          W[k * n + a] = c * ka - s * kb;
          W[k * n + b] = s * ka + c * kb;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = C[i * n + i];
}

}  // namespace

std::vector<double> gll_nodes(int p) {
  if (p < 1) throw std::runtime_error("gll_nodes: p >= 1");
  std::vector<double> x(p + 1);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double t = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, t, P, dP);
      // P'' from the Legendre equation
      double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[j] = t;
  }
  std::sort(x.begin(), x.end());
  return x;
}

void gll_rule(int q, std::vector<double> &x, std::vector<double> &w) {
  x = gll_nodes(q - 1);
  w.resize(q);
  for (int j = 0; j < q; ++j) {
    double P, dP;
    legendre(q - 1, x[j], P, dP);
    w[j] = 2.0 / (q * (q - 1.0) * P * P);
  }
}

void gauss_rule(int m, std::vector<double> &x, std::vector<double> &w) {
  x.resize(m);
  w.resize(m);
  for (int j = 0; j < m; ++j) {
    double t = -std::cos(M_PI * (j + 0.75) / (m + 0.5));
    double P = 0, dP = 1;
    for (int it = 0; it < 100; ++it) {
      legendre(m, t, P, dP);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    legendre(m, t, P, dP);
    x[j] = t;
    w[j] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
  std::vector<int> ord(m);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(m), ws(m);
  for (int j = 0; j < m; ++j) { xs[j] = x[ord[j]]; ws[j] = w[ord[j]]; }
  x = xs;
  w = ws;
}

Basis1D::Basis1D(int p_) : p(p_) {
  if (p < 1 || p > 30) throw std::runtime_error("Basis1D: 1 <= p <= 30");
  const int n = p + 1;
  xi = gll_nodes(p);
  std::vector<double> bw = bary_weights(xi);
  std::vector<double> xg, wg;
  gauss_rule(p + 1, xg, wg);
  std::vector<double> L(n), dL(n);
  std::vector<double> Bg(n * n, 0.0), Ag(n * n, 0.0);
  for (int g = 0; g < (int)xg.size(); ++g) {
    lagrange_at(xi, bw, xg[g], L.data(), dL.data());
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        Bg[i * n + j] += wg[g] * L[i] * L[j];
        Ag[i * n + j] += wg[g] * dL[i] * dL[j];
      }
  }
  S.assign(n * n, 0.0);
  S[0] = 1.0;
  S[p * n + p] = 1.0;
  lam.assign(p, 2.0);
  const int m = p - 1;  // interior size
  if (m > 0) {
    // Eq. eigs: A_II v = lam B_II v; B_II = L L^T, C = L^-1 A_II L^-T
    std::vector<double> Bi(m * m), Ai(m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        Bi[i * m + j] = Bg[(i + 1) * n + (j + 1)];
        Ai[i * m + j] = Ag[(i + 1) * n + (j + 1)];
      }
    std::vector<double> Lc = Bi;
    chol(Lc, m);
    // Y = L^-1 A  (forward substitution on columns)
    std::vector<double> Y(m * m), C(m * m);
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < m; ++i) {
        double s = Ai[i * m + c];
        for (int k = 0; k < i; ++k) s -= Lc[i * m + k] * Y[k * m + c];
        Y[i * m + c] = s / Lc[i * m + i];
      }
    // C = Y L^-T: C^T = L^-1 Y^T
    for (int r = 0; r < m; ++r)
      for (int i = 0; i < m; ++i) {
        double s = Y[r * m + i];
        for (int k = 0; k < i; ++k) s -= Lc[i * m + k] * C[r * m + k];
        C[r * m + i] = s / Lc[i * m + i];
      }
    for (int i = 0; i < m; ++i)  // symmetrise
      for (int j = i + 1; j < m; ++j) {
        double a = 0.5 * (C[i * m + j] + C[j * m + i]);
        C[i * m + j] = C[j * m + i] = a;
      }
    std::vector<double> ev, W;
    jacobi_eig(C, m, ev, W);
    // V = L^-T W (back substitution)
    std::vector<double> V(m * m);
    for (int c = 0; c < m; ++c)
      for (int i = m - 1; i >= 0; --i) {
        double s = W[i * m + c];
        for (int k = i + 1; k < m; ++k) s -= Lc[k * m + i] * V[k * m + c];
        V[i * m + c] = s / Lc[i * m + i];
      }
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    // sign rule: s_j'(-1) > 0
    lagrange_at(xi, bw, -1.0, L.data(), dL.data());
    for (int jj = 0; jj < m; ++jj) {
      int c = ord[jj];
      double slope = 0.0;
      for (int i = 0; i < m; ++i) slope += dL[i + 1] * V[i * m + c];
      double sg = slope >= 0 ? 1.0 : -1.0;
      for (int i = 0; i < m; ++i) S[(i + 1) * n + (jj + 1)] = sg * V[i * m + c];
      lam[jj + 1] = ev[c];
    }
    // interface columns: S_IG = -S_II S_II^T B_IG
    for (int gcol : {0, p}) {
      std::vector<double> t(m, 0.0);
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) t[j] += S[(i + 1) * n + (j + 1)] * Bg[(i + 1) * n + gcol];
      for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += S[(i + 1) * n + (j + 1)] * t[j];
        S[(i + 1) * n + gcol] = -s;
      }
    }
  }
  // B-hat = S^T Bgll S, A-hat = S^T Agll S
  Bhat.assign(n * n, 0.0);
  Ahat.assign(n * n, 0.0);
  std::vector<double> tb(n * n, 0.0), ta(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        tb[i * n + j] += Bg[i * n + k] * S[k * n + j];
        ta[i * n + j] += Ag[i * n + k] * S[k * n + j];
      }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        Bhat[i * n + j] += S[k * n + i] * tb[k * n + j];
        Ahat[i * n + j] += S[k * n + i] * ta[k * n + j];
      }
  // D_ij = (r_i, s_j'): row 0 = 2^-1/2 (s_j(1) - s_j(-1)); row i >= 1 =
  // lam_i^-1/2 A-hat_ij, which is lam_i^1/2 delta_ij on interior columns.
  D.assign(p * n, 0.0);
  D[0 * n + 0] = -1.0 / std::sqrt(2.0);
  D[0 * n + p] = 1.0 / std::sqrt(2.0);
  for (int i = 1; i < p; ++i) {
    double s = 1.0 / std::sqrt(lam[i]);
    D[i * n + 0] = s * Ahat[i * n + 0];
    D[i * n + p] = s * Ahat[i * n + p];
    D[i * n + i] = std::sqrt(lam[i]);
  }
  // p = 1 hats in this basis: nodal values c solve S c = hat(xi)
  Js.assign(n * 2, 0.0);
  for (int c = 0; c < 2; ++c) {
    std::vector<double> nod(n);
    for (int i = 0; i < n; ++i) nod[i] = c == 0 ? 0.5 * (1.0 - xi[i]) : 0.5 * (1.0 + xi[i]);
    // S = [[1,0,0],[S_I0, S_II, S_Ip],[0,0,1]]: c_0 = nod_0, c_p = nod_p,
    // S_II c_I = nod_I - S_I0 c_0 - S_Ip c_p; S_II^-1 = S_II^T B_II
    double c0 = nod[0], cp = nod[p];
    std::vector<double> rhs(m);
    for (int i = 0; i < m; ++i)
      rhs[i] = nod[i + 1] - S[(i + 1) * n + 0] * c0 - S[(i + 1) * n + p] * cp;
    std::vector<double> tmp(m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < m; ++k) tmp[i] += Bg[(i + 1) * n + (k + 1)] * rhs[k];
    Js[0 * 2 + c] = c0;
    Js[p * 2 + c] = cp;
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += S[(i + 1) * n + (j + 1)] * tmp[i];
      Js[(j + 1) * 2 + c] = s;
    }
  }
}

void Basis1D::tab_s(const double *x, int nx, double *out) const {
  const int n = p + 1;
  std::vector<double> bw = bary_weights(xi), L(n), dL(n);
  for (int k = 0; k < nx; ++k) {
    lagrange_at(xi, bw, x[k], L.data(), dL.data());
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += L[i] * S[i * n + j];
      out[k * n + j] = s;
    }
  }
}

void Basis1D::tab_ds(const double *x, int nx, double *out) const {
  const int n = p + 1;
  std::vector<double> bw = bary_weights(xi), L(n), dL(n);
  for (int k = 0; k < nx; ++k) {
    lagrange_at(xi, bw, x[k], L.data(), dL.data());
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += dL[i] * S[i * n + j];
      out[k * n + j] = s;
    }
  }
}

void Basis1D::tab_r(const double *x, int nx, double *out) const {
  const int n = p + 1;
  std::vector<double> ds(nx * n);
  tab_ds(x, nx, ds.data());
  for (int k = 0; k < nx; ++k) {
    out[k * p + 0] = 1.0 / std::sqrt(2.0);
    for (int i = 1; i < p; ++i) out[k * p + i] = ds[k * n + i] / std::sqrt(lam[i]);
  }
}

}  // namespace rm
