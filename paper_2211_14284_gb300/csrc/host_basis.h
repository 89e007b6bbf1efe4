// 1D FDM bases on [-1, 1] (Sec. 2.2-2.3), host FP64.
#pragma once
#include <vector>

namespace rm {

// Gauss-Lobatto-Legendre nodes (p+1 points, p >= 1), Newton on P_p'.
std::vector<double> gll_nodes(int p);
// q-point GLL rule.
void gll_rule(int q, std::vector<double> &x, std::vector<double> &w);
// m-point Gauss-Legendre rule, Newton on P_m.
void gauss_rule(int m, std::vector<double> &x, std::vector<double> &w);

struct Basis1D {
  int p = 0;
  std::vector<double> xi;     // GLL nodes, p+1
  std::vector<double> S;      // (p+1)x(p+1) row-major, S[i*(p+1)+j] = s_j(xi_i)
  std::vector<double> lam;    // lam[0] = 2, lam[j] = (s_j', s_j')
  std::vector<double> Bhat;   // (p+1)^2, (s_i, s_j)
  std::vector<double> Ahat;   // (p+1)^2, (s_i', s_j')
  std::vector<double> D;      // p x (p+1) row-major, (r_i, s_j')
  std::vector<double> Js;     // (p+1) x 2: coefficients of the p=1 hats (1-x)/2, (1+x)/2

  explicit Basis1D(int p);
  // tabulations at n points x: out[k*(p+1)+j] = s_j(x_k) (resp. s_j'), r: out[k*p+i] = r_i(x_k)
  void tab_s(const double *x, int n, double *out) const;
  void tab_ds(const double *x, int n, double *out) const;
  void tab_r(const double *x, int n, double *out) const;
};

}  // namespace rm
