// Host-side FP64 reference tables of libhopu.
//
// * Gauss-Jacobi rules: Newton iteration with deflation on the Jacobi polynomial
//   P_m^{(alpha,0)} (three-term recurrence), weights from the closed form
//   w_i = 2^{alpha+1} / ((1 - x_i^2) P_m'(x_i)^2) for beta = 0; collapsed (Stroud
//   conical) products on the simplex.  The paper asks for exact integration of every
//   form (Section 2.2); the volume rule is exact to degree 3k-1, the facet rule to 3k.
// * Dubiner basis: products of homogenised Jacobi polynomials
//   Q_n^{(a)}(x, s) = s^n P_n^{(a,0)}(2x/s - 1), evaluated by their own recurrence (no
//   division by the collapsed coordinate), orthonormal on the unit simplex.
// * BDM_k degrees of freedom: facet normal moments against the orthonormal facet basis
//   and interior moments against the Nedelec-first-kind space of index k-1.
#include "reftables.h"

#include "hopu_internal.h"
#include "volume_rules.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace hopu {

namespace {

// Q_n^{(a)}(x, s), n = 0..N, with partial derivatives in x and s.
void scaled_jacobi(int N, double a, double x, double s, double* Q, double* Qx, double* Qs) {
  Q[0] = 1.0;
  Qx[0] = 0.0;
  Qs[0] = 0.0;
  if (N >= 1) {
    Q[1] = (a + 2.0) * x - s;
    Qx[1] = a + 2.0;
    Qs[1] = -1.0;
  }
  for (int n = 2; n <= N; ++n) {
    const double A = (2 * n + a - 1) * (2 * n + a) * (2 * n + a - 2);
    const double B = (2 * n + a - 1) * a * a;
    const double C = 2.0 * (n + a - 1) * (n - 1) * (2 * n + a);
    const double K = 2.0 * n * (n + a) * (2 * n + a - 2);
    const double L = A * (2 * x - s) + B * s;
    Q[n] = (L * Q[n - 1] - C * s * s * Q[n - 2]) / K;
    Qx[n] = (2 * A * Q[n - 1] + L * Qx[n - 1] - C * s * s * Qx[n - 2]) / K;
    Qs[n] = ((B - A) * Q[n - 1] + L * Qs[n - 1] - 2 * C * s * Q[n - 2] - C * s * s * Qs[n - 2]) / K;
  }
}

// P_m^{(alpha,0)}(x) and its derivative on [-1, 1].
void jacobi_pd(int m, double alpha, double x, double* p, double* dp) {
  std::vector<double> Q(m + 1), Qx(m + 1), Qs(m + 1);
  scaled_jacobi(m, alpha, 0.5 * (x + 1.0), 1.0, Q.data(), Qx.data(), Qs.data());
  *p = Q[m];
  *dp = 0.5 * Qx[m];
}

struct Idx3 { int p, q, r; };

std::vector<Idx3> dubiner_indices(int dim, int k) {
  std::vector<Idx3> out;
  for (int n = 0; n <= k; ++n) {
    if (dim == 1) {
      out.push_back({n, 0, 0});
    } else if (dim == 2) {
      for (int p = 0; p <= n; ++p) out.push_back({p, n - p, 0});
    } else {
      for (int p = 0; p <= n; ++p)
        for (int q = 0; q <= n - p; ++q) out.push_back({p, q, n - p - q});
    }
  }
  return out;
}

bool invert(int n, const std::vector<double>& A, std::vector<double>& Ainv) {
  std::vector<long double> M((size_t)n * 2 * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      M[(size_t)i * 2 * n + j] = A[(size_t)i * n + j];
      M[(size_t)i * 2 * n + n + j] = (i == j) ? 1.0L : 0.0L;
    }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs((double)M[(size_t)r * 2 * n + c]) > std::fabs((double)M[(size_t)piv * 2 * n + c])) piv = r;
    if (M[(size_t)piv * 2 * n + c] == 0.0L) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(M[(size_t)c * 2 * n + j], M[(size_t)piv * 2 * n + j]);
    const long double d = M[(size_t)c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[(size_t)c * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const long double f = M[(size_t)r * 2 * n + c];
      if (f == 0.0L) continue;
      for (int j = 0; j < 2 * n; ++j) M[(size_t)r * 2 * n + j] -= f * M[(size_t)c * 2 * n + j];
    }
  }
  Ainv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[(size_t)i * n + j] = (double)M[(size_t)i * 2 * n + n + j];
  return true;
}

}  // namespace

void gauss_jacobi01(int m, int alpha, std::vector<double>& t, std::vector<double>& w) {
  std::vector<double> x(m);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < m; ++i) {
    double r = -std::cos((2.0 * i + 1.0) * pi / (2.0 * m));
    if (i > 0) r = 0.5 * (r + x[i - 1]);
    for (int it = 0; it < 200; ++it) {
      double p, dp;
      jacobi_pd(m, alpha, r, &p, &dp);
      double s = 0.0;
      for (int j = 0; j < i; ++j) s += 1.0 / (r - x[j]);
      const double delta = -p / (dp - s * p);
      r += delta;
      if (std::fabs(delta) < 1e-17) break;
    }
    x[i] = r;
  }
  std::sort(x.begin(), x.end());
  t.resize(m);
  w.resize(m);
  for (int i = 0; i < m; ++i) {
    double p, dp;
    jacobi_pd(m, alpha, x[i], &p, &dp);
    // int_{-1}^{1} (1-x)^alpha f dx weights, then mapped to [0, 1]: divide by 2^{alpha+1}
    t[i] = 0.5 * (1.0 + x[i]);
    w[i] = 1.0 / ((1.0 - x[i] * x[i]) * dp * dp);
  }
}

void simplex_rule(int dim, int degree, std::vector<double>& x, std::vector<double>& w) {
  const int m = rule_m(degree);
  std::vector<double> t0, w0, t1, w1, t2, w2;
  gauss_jacobi01(m, 0, t0, w0);
  x.clear();
  w.clear();
  if (dim == 1) {
    x = t0;
    w = w0;
    return;
  }
  gauss_jacobi01(m, 1, t1, w1);
  if (dim == 2) {
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        x.push_back(t0[i] * (1.0 - t1[j]));
        x.push_back(t1[j]);
        w.push_back(w0[i] * w1[j]);
      }
    return;
  }
  gauss_jacobi01(m, 2, t2, w2);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      for (int l = 0; l < m; ++l) {
        x.push_back(t0[i] * (1.0 - t1[j]) * (1.0 - t2[l]));
        x.push_back(t1[j] * (1.0 - t2[l]));
        x.push_back(t2[l]);
        w.push_back(w0[i] * w1[j] * w2[l]);
      }
}

void dubiner(int dim, int k, const double* x, double* vals, double* grads) {
  const std::vector<Idx3> idx = dubiner_indices(dim, k);
  const int K1 = k + 1;
  std::vector<double> Q1(K1), Q1x(K1), Q1s(K1), Q2(K1), Q2x(K1), Q2s(K1), Q3(K1), Q3x(K1), Q3s(K1);
  for (size_t j = 0; j < idx.size(); ++j) {
    const int p = idx[j].p, q = idx[j].q, r = idx[j].r;
    if (dim == 1) {
      scaled_jacobi(p, 0.0, x[0], 1.0, Q1.data(), Q1x.data(), Q1s.data());
      const double c = std::sqrt(2.0 * p + 1.0);
      vals[j] = c * Q1[p];
      if (grads) grads[j] = c * Q1x[p];
    } else if (dim == 2) {
      const double s = 1.0 - x[1];
      scaled_jacobi(p, 0.0, x[0], s, Q1.data(), Q1x.data(), Q1s.data());
      scaled_jacobi(q, 2.0 * p + 1.0, x[1], 1.0, Q2.data(), Q2x.data(), Q2s.data());
      const double c = std::sqrt((2.0 * p + 1.0) * (2.0 * p + 2.0 * q + 2.0));
      vals[j] = c * Q1[p] * Q2[q];
      if (grads) {
        grads[j * 2 + 0] = c * Q1x[p] * Q2[q];
        grads[j * 2 + 1] = c * (-Q1s[p] * Q2[q] + Q1[p] * Q2x[q]);
      }
    } else {
      const double s1 = 1.0 - x[1] - x[2], s2 = 1.0 - x[2];
      scaled_jacobi(p, 0.0, x[0], s1, Q1.data(), Q1x.data(), Q1s.data());
      scaled_jacobi(q, 2.0 * p + 1.0, x[1], s2, Q2.data(), Q2x.data(), Q2s.data());
      scaled_jacobi(r, 2.0 * p + 2.0 * q + 2.0, x[2], 1.0, Q3.data(), Q3x.data(), Q3s.data());
      const double c = std::sqrt((2.0 * p + 1.0) * (2.0 * p + 2.0 * q + 2.0) *
                                 (2.0 * p + 2.0 * q + 2.0 * r + 3.0));
      const double A = Q1[p], B = Q2[q], C = Q3[r];
      vals[j] = c * A * B * C;
      if (grads) {
        grads[j * 3 + 0] = c * Q1x[p] * B * C;
        grads[j * 3 + 1] = c * (-Q1s[p] * B + A * Q2x[q]) * C;
        grads[j * 3 + 2] = c * (-Q1s[p] * B * C - A * Q2s[q] * C + A * B * Q3x[r]);
      }
    }
  }
}

namespace {

// Reference facet f: the vertices other than f, in ascending local order.
void facet_vertices(int dim, int f, double P[3][3]) {
  int row = 0;
  for (int v = 0; v <= dim; ++v) {
    if (v == f) continue;
    for (int c = 0; c < dim; ++c) P[row][c] = (v > 0 && c == v - 1) ? 1.0 : 0.0;
    ++row;
  }
}

void facet_point(int dim, int f, const double* s, double* x) {
  double P[3][3];
  facet_vertices(dim, f, P);
  for (int c = 0; c < dim; ++c) {
    x[c] = P[0][c];
    for (int j = 0; j < dim - 1; ++j) x[c] += s[j] * (P[j + 1][c] - P[0][c]);
  }
}

// -grad(lambda_f): outward normal of reference facet f scaled by |facet| / |param|.
void scaled_normal(int dim, int f, double* n) {
  for (int c = 0; c < dim; ++c) n[c] = (f == 0) ? 1.0 : ((c == f - 1) ? -1.0 : 0.0);
}

// Interior moment functions (BDM_k interior space, Nedelec first kind of index k-1)
// at one point: part A = phi_j e_m (Dubiner P^{k-2}); part B = x~ x (q e_m) in 3D with
// q in the degree-(k-2) Dubiner block (3D basis for m = 0, 1; 2D basis of (x1, x2) for
// m = 2), or x~^perp q in 2D; x~ = (dim+1) (x - centroid).
void interior_functions(int dim, int k, const double* x, std::vector<double>& out /*[nint][dim]*/) {
  out.clear();
  if (k < 2) return;
  const int nbm2 = nbasis(dim, k - 2), nbm3 = nbasis(dim, k - 3);
  std::vector<double> phi(nbm2);
  dubiner(dim, k - 2, x, phi.data(), nullptr);
  for (int m = 0; m < dim; ++m)
    for (int j = 0; j < nbm2; ++j)
      for (int c = 0; c < dim; ++c) out.push_back(c == m ? phi[j] : 0.0);
  double xt[3];
  for (int c = 0; c < dim; ++c) xt[c] = (dim + 1) * (x[c] - 1.0 / (dim + 1));
  if (dim == 2) {
    for (int j = nbm3; j < nbm2; ++j) {
      out.push_back(-xt[1] * phi[j]);
      out.push_back(xt[0] * phi[j]);
    }
    return;
  }
  const int n2m2 = nbasis(2, k - 2), n2m3 = nbasis(2, k - 3);
  std::vector<double> chi(n2m2);
  dubiner(2, k - 2, x, chi.data(), nullptr);
  for (int m = 0; m < 3; ++m) {
    double cr[3];  // x~ cross e_m
    if (m == 0) { cr[0] = 0.0; cr[1] = xt[2]; cr[2] = -xt[1]; }
    if (m == 1) { cr[0] = -xt[2]; cr[1] = 0.0; cr[2] = xt[0]; }
    if (m == 2) { cr[0] = xt[1]; cr[1] = -xt[0]; cr[2] = 0.0; }
    const int lo = (m < 2) ? nbm3 : n2m3, hi = (m < 2) ? nbm2 : n2m2;
    for (int j = lo; j < hi; ++j) {
      const double qv = (m < 2) ? phi[j] : chi[j];
      for (int c = 0; c < 3; ++c) out.push_back(cr[c] * qv);
    }
  }
}

}  // namespace

bool build_ref_tables(int dim, int k, RefTables& T, std::string& err) {
  if (dim < 2 || dim > 3 || k < 1 || k > 5) {
    err = "reference tables: dim must be 2 or 3 and k in 1..5";
    return false;
  }
  T.dim = dim;
  T.k = k;
  T.nb = nbasis(dim, k);
  T.nf = nbasis(dim - 1, k);
  T.nloc = dim * T.nb;
  T.nint = T.nloc - (dim + 1) * T.nf;
  simplex_rule(dim, 3 * k - 1, T.xq, T.wq);
  simplex_rule(dim - 1, 3 * k, T.sq, T.wf);
  T.nq = (int)T.wq.size();
  T.nqf = (int)T.wf.size();
  const int nb = T.nb, nf = T.nf, nq = T.nq, nqf = T.nqf, nloc = T.nloc;

  T.phi.assign((size_t)nq * nb, 0.0);
  T.dphi.assign((size_t)nq * nb * dim, 0.0);
  for (int q = 0; q < nq; ++q)
    dubiner(dim, k, &T.xq[(size_t)q * dim], &T.phi[(size_t)q * nb], &T.dphi[(size_t)q * nb * dim]);

  // the volume kernels' rule
  const double* tab = nullptr;
  int ntab = 0;
  if (dim == 3 && k == 3) tab = kTetRule3, ntab = kTetRule3N;
  if (dim == 3 && k == 4) tab = kTetRule4, ntab = kTetRule4N;
  if (dim == 3 && k == 5) tab = kTetRule5, ntab = kTetRule5N;
  if (ntab != compact_volume_points(dim, k)) {
    err = "reference tables: compact volume rule size mismatch";
    return false;
  }
  if (tab) {
    T.nqk = ntab;
    T.xk.resize((size_t)ntab * 3);
    T.wk.resize(ntab);
    for (int q = 0; q < ntab; ++q) {
      for (int c = 0; c < 3; ++c) T.xk[(size_t)q * 3 + c] = tab[q * 4 + c];
      T.wk[q] = tab[q * 4 + 3];
    }
  } else {
    T.nqk = nq;
    T.xk = T.xq;
    T.wk = T.wq;
  }
  T.phik.assign((size_t)T.nqk * nb, 0.0);
  for (int q = 0; q < T.nqk; ++q) dubiner(dim, k, &T.xk[(size_t)q * dim], &T.phik[(size_t)q * nb], nullptr);

  T.psi.assign((size_t)nqf * nf, 0.0);
  for (int q = 0; q < nqf; ++q) dubiner(dim - 1, k, &T.sq[(size_t)q * (dim - 1)], &T.psi[(size_t)q * nf], nullptr);

  T.phif.assign((size_t)(dim + 1) * nqf * nb, 0.0);
  for (int f = 0; f <= dim; ++f)
    for (int q = 0; q < nqf; ++q) {
      double xf[3];
      facet_point(dim, f, &T.sq[(size_t)q * (dim - 1)], xf);
      dubiner(dim, k, xf, &T.phif[((size_t)f * nqf + q) * nb], nullptr);
    }

  T.trm.assign((size_t)(dim + 1) * nf * nb, 0.0);
  for (int f = 0; f <= dim; ++f)
    for (int m = 0; m < nf; ++m)
      for (int i = 0; i < nb; ++i) {
        double acc = 0.0;
        for (int q = 0; q < nqf; ++q)
          acc += T.wf[q] * T.psi[(size_t)q * nf + m] * T.phif[((size_t)f * nqf + q) * nb + i];
        T.trm[((size_t)f * nf + m) * nb + i] = acc;
      }

  T.z.assign((size_t)T.nint * nq * dim, 0.0);
  std::vector<double> zq;
  for (int q = 0; q < nq; ++q) {
    interior_functions(dim, k, &T.xq[(size_t)q * dim], zq);
    if ((int)zq.size() != T.nint * dim) {
      err = "reference tables: interior moment space has the wrong dimension";
      return false;
    }
    for (int j = 0; j < T.nint; ++j)
      for (int c = 0; c < dim; ++c) T.z[((size_t)j * nq + q) * dim + c] = zq[(size_t)j * dim + c];
  }

  // D[row][b*nb + i]: facet rows (f, m) then interior rows j.
  T.D.assign((size_t)nloc * nloc, 0.0);
  for (int f = 0; f <= dim; ++f) {
    double N[3];
    scaled_normal(dim, f, N);
    for (int m = 0; m < nf; ++m)
      for (int b = 0; b < dim; ++b)
        for (int i = 0; i < nb; ++i)
          T.D[(size_t)(f * nf + m) * nloc + b * nb + i] = N[b] * T.trm[((size_t)f * nf + m) * nb + i];
  }
  for (int j = 0; j < T.nint; ++j)
    for (int b = 0; b < dim; ++b)
      for (int i = 0; i < nb; ++i) {
        double acc = 0.0;
        for (int q = 0; q < nq; ++q)
          acc += T.wq[q] * T.phi[(size_t)q * nb + i] * T.z[((size_t)j * nq + q) * dim + b];
        T.D[(size_t)((dim + 1) * nf + j) * nloc + b * nb + i] = acc;
      }
  if (!invert(nloc, T.D, T.Dinv)) {
    err = "reference tables: the BDM degree-of-freedom matrix is singular";
    return false;
  }
  return true;
}

bool selftest_ref_tables(int dim, int k, double report[4], std::string& err) {
  RefTables T;
  if (!build_ref_tables(dim, k, T, err)) return false;
  auto fact = [](int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; };
  // (0) both volume rules (collapsed, kernels') on monomials up to 3k-1 and (1) the facet
  // rule up to 3k
  double e0 = 0.0, e1 = 0.0;
  for (int pass = 0; pass < 3; ++pass) {  // 0: collapsed volume, 1: facet, 2: kernel volume
    const int d = pass == 1 ? dim - 1 : dim;
    const int deg = pass == 1 ? 3 * k : 3 * k - 1;
    const std::vector<double>& X = pass == 0 ? T.xq : pass == 1 ? T.sq : T.xk;
    const std::vector<double>& Wt = pass == 0 ? T.wq : pass == 1 ? T.wf : T.wk;
    const int n = (int)Wt.size();
    for (int a = 0; a <= deg; ++a)
      for (int b = 0; b <= (d >= 2 ? deg - a : 0); ++b)
        for (int c = 0; c <= (d >= 3 ? deg - a - b : 0); ++c) {
          double val = 0.0;
          for (int q = 0; q < n; ++q) {
            double mono = std::pow(X[(size_t)q * d], a);
            if (d >= 2) mono *= std::pow(X[(size_t)q * d + 1], b);
            if (d >= 3) mono *= std::pow(X[(size_t)q * d + 2], c);
            val += Wt[q] * mono;
          }
          const double ex = fact(a) * fact(b) * fact(c) / fact(a + b + c + d);
          const double e = std::fabs(val - ex) / ex;
          if (pass == 1) e1 = std::max(e1, e); else e0 = std::max(e0, e);
        }
  }
  // (2) orthonormality of the basis under both volume rules (exact to 3k-1 >= 2k for k>=1)
  double e2 = 0.0;
  for (int i = 0; i < T.nb; ++i)
    for (int j = 0; j < T.nb; ++j) {
      double acc = 0.0, acck = 0.0;
      for (int q = 0; q < T.nq; ++q) acc += T.wq[q] * T.phi[(size_t)q * T.nb + i] * T.phi[(size_t)q * T.nb + j];
      for (int q = 0; q < T.nqk; ++q) acck += T.wk[q] * T.phik[(size_t)q * T.nb + i] * T.phik[(size_t)q * T.nb + j];
      e2 = std::max(e2, std::max(std::fabs(acc - (i == j ? 1.0 : 0.0)), std::fabs(acck - (i == j ? 1.0 : 0.0))));
    }
  // (3) D * Dinv = I
  double e3 = 0.0;
  for (int i = 0; i < T.nloc; ++i)
    for (int j = 0; j < T.nloc; ++j) {
      double acc = 0.0;
      for (int l = 0; l < T.nloc; ++l) acc += T.D[(size_t)i * T.nloc + l] * T.Dinv[(size_t)l * T.nloc + j];
      e3 = std::max(e3, std::fabs(acc - (i == j ? 1.0 : 0.0)));
    }
  report[0] = e0;
  report[1] = e1;
  report[2] = e2;
  report[3] = e3;
  return true;
}

}  // namespace hopu
