// Host-side FP64 reference-element tables of libhopu (quadrature, Dubiner basis,
// facet traces, the BDM_k degree-of-freedom matrix and its inverse).
#pragma once
#include <string>
#include <vector>

namespace hopu {

inline int binom(int n, int r) {
  if (r < 0 || n < r) return 0;
  long long v = 1;
  for (int i = 1; i <= r; ++i) v = v * (n - r + i) / i;
  return (int)v;
}
inline int nbasis(int dim, int k) { return k < 0 ? 0 : binom(k + dim, dim); }
// points per collapsed direction of a rule exact to degree deg
inline int rule_m(int deg) { return deg < 1 ? 1 : (deg + 2) / 2; }

struct RefTables {
  int dim = 0, k = 0, nb = 0, nf = 0, nint = 0, nloc = 0, nq = 0, nqf = 0;
  std::vector<double> xq, wq;    // [nq][dim], [nq]   volume rule, exact to degree 3k-1
  std::vector<double> sq, wf;    // [nqf][dim-1], [nqf] facet rule, exact to degree 3k
  std::vector<double> phi;       // [nq][nb]          phi_i(xq)
  std::vector<double> dphi;      // [nq][nb][dim]     reference gradients
  std::vector<double> phif;      // [dim+1][nqf][nb]  phi_i(xhat_f(sq))
  std::vector<double> psi;       // [nqf][nf]         facet basis at facet points
  std::vector<double> trm;       // [dim+1][nf][nb]   modal trace <phi_i o xhat_f, psi_m>
  std::vector<double> z;         // [nint][nq][dim]   interior moment functions
  std::vector<double> D, Dinv;   // [nloc][nloc]      functionals x (component-major basis)
  // the volume kernels' rule (exact to degree 3k-1; compact where one is tabulated, else
  // the rule above) and the basis there
  int nqk = 0;
  std::vector<double> xk, wk;    // [nqk][dim], [nqk]
  std::vector<double> phik;      // [nqk][nb]
};

// Gauss-Jacobi nodes t in (0,1) and weights for int_0^1 f(t) (1-t)^alpha dt.
void gauss_jacobi01(int m, int alpha, std::vector<double>& t, std::vector<double>& w);
// Collapsed Gauss-Jacobi rule on the unit simplex of dimension dim (1..3).
void simplex_rule(int dim, int degree, std::vector<double>& x, std::vector<double>& w);
// Orthonormal Dubiner basis of P^k on the unit simplex at one point x[dim].
// vals[nb], grads[nb*dim] (grads may be null).
void dubiner(int dim, int k, const double* x, double* vals, double* grads);

bool build_ref_tables(int dim, int k, RefTables& out, std::string& err);

// Host self-check: max errors of the rules on monomials, of basis orthonormality and
// of D * Dinv - I.  Returns false on a failed construction.
bool selftest_ref_tables(int dim, int k, double report[4], std::string& err);

}  // namespace hopu
