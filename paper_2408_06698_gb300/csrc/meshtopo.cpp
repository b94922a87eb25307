// Host-side mesh topology and FP64 affine geometry of libhopu.
//
// Element vertices are reordered by ascending periodic-representative id, so the two
// elements sharing a facet see its vertices in the same order and parametrise it the
// same way (the jump/average notation of Section 2.1 needs both traces at the same
// physical points).  Facets are found by sorting the representative tuples.
#include "meshtopo.h"

#include <algorithm>
#include <cmath>
#include <numeric>

#include "../../include/hopu.h"

namespace hopu {

namespace {

double det_inv(int d, const double* J, double* Ji) {
  if (d == 2) {
    const double det = J[0] * J[3] - J[1] * J[2];
    if (det == 0.0) return 0.0;
    Ji[0] = J[3] / det;
    Ji[1] = -J[1] / det;
    Ji[2] = -J[2] / det;
    Ji[3] = J[0] / det;
    return det;
  }
  const double c00 = J[4] * J[8] - J[5] * J[7];
  const double c01 = J[5] * J[6] - J[3] * J[8];
  const double c02 = J[3] * J[7] - J[4] * J[6];
  const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  if (det == 0.0) return 0.0;
  Ji[0] = c00 / det;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = c01 / det;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = c02 / det;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  return det;
}

// canonical (unnormalised) normal of facet f of element e from its physical vertices
void facet_cross(const MeshTopo& m, int64_t e, int f, double* cr) {
  const int d = m.dim;
  const double* X = &m.X[(size_t)e * (d + 1) * d];
  int loc[3], c = 0;
  for (int v = 0; v <= d; ++v)
    if (v != f) loc[c++] = v;
  if (d == 3) {
    double a[3], b[3];
    for (int i = 0; i < 3; ++i) {
      a[i] = X[loc[1] * 3 + i] - X[loc[0] * 3 + i];
      b[i] = X[loc[2] * 3 + i] - X[loc[0] * 3 + i];
    }
    cr[0] = a[1] * b[2] - a[2] * b[1];
    cr[1] = a[2] * b[0] - a[0] * b[2];
    cr[2] = a[0] * b[1] - a[1] * b[0];
  } else {
    const double tx = X[loc[1] * 2 + 0] - X[loc[0] * 2 + 0];
    const double ty = X[loc[1] * 2 + 1] - X[loc[0] * 2 + 1];
    cr[0] = ty;
    cr[1] = -tx;
  }
}

}  // namespace

int build_mesh_topo(int d, int64_t nv, const double* coords, int64_t ne, const int64_t* ev,
                    const int64_t* rep, MeshTopo& m, std::string& err) {
  if (d != 2 && d != 3) { err = "mesh: dim must be 2 or 3"; return HOPU_EINVAL; }
  if (nv <= 0 || ne <= 0 || !coords || !ev) { err = "mesh: empty or NULL arrays"; return HOPU_EINVAL; }
  if (ne > (int64_t(1) << 28)) { err = "mesh: more than 2^28 elements"; return HOPU_ENOTSUP; }
  const int nvl = d + 1;
  m.dim = d;
  m.n_elems = ne;
  m.X.assign((size_t)ne * nvl * d, 0.0);
  const int G = geo_stride(d);
  m.geo.assign((size_t)ne * G, 0.0);
  std::vector<int64_t> rsorted((size_t)ne * nvl);
  for (int64_t e = 0; e < ne; ++e) {
    int64_t v[4], r[4];
    for (int j = 0; j < nvl; ++j) {
      v[j] = ev[e * nvl + j];
      if (v[j] < 0 || v[j] >= nv) { err = "mesh: vertex id out of range"; return HOPU_EMESH; }
      r[j] = rep ? rep[v[j]] : v[j];
      if (r[j] < 0) { err = "mesh: negative representative id"; return HOPU_EMESH; }
    }
    int ord[4] = {0, 1, 2, 3};
    std::sort(ord, ord + nvl, [&](int a, int b) { return r[a] < r[b]; });
    for (int j = 0; j + 1 < nvl; ++j)
      if (r[ord[j]] == r[ord[j + 1]]) { err = "mesh: element with two identified vertices"; return HOPU_EMESH; }
    for (int j = 0; j < nvl; ++j) {
      rsorted[(size_t)e * nvl + j] = r[ord[j]];
      for (int c = 0; c < d; ++c) m.X[((size_t)e * nvl + j) * d + c] = coords[v[ord[j]] * d + c];
    }
    double* g = &m.geo[(size_t)e * G];
    const double* X = &m.X[(size_t)e * nvl * d];
    double scale = 0.0;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        g[a * d + b] = X[(b + 1) * d + a] - X[a];
        scale = std::max(scale, std::fabs(g[a * d + b]));
      }
    const double det = det_inv(d, g, g + d * d);
    if (!(std::fabs(det) > 1e-13 * std::pow(scale, d))) { err = "mesh: degenerate element"; return HOPU_EMESH; }
    g[2 * d * d] = det;
    g[2 * d * d + 1] = std::fabs(det);
  }

  // facets: sort (element, local facet) by the representative tuple of the facet
  const int64_t nef = ne * nvl;
  auto key = [&](int64_t id, int64_t* k) {
    const int64_t e = id / nvl;
    const int f = (int)(id % nvl);
    int c = 0;
    for (int v = 0; v < nvl; ++v)
      if (v != f) k[c++] = rsorted[(size_t)e * nvl + v];
  };
  std::vector<int64_t> order((size_t)nef);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    int64_t ka[3], kb[3];
    key(a, ka);
    key(b, kb);
    for (int i = 0; i < d; ++i)
      if (ka[i] != kb[i]) return ka[i] < kb[i];
    return a < b;
  });
  m.efc.assign((size_t)nef, 0);
  m.fa.clear();
  m.fb.clear();
  m.boundary.clear();
  m.fgeo.clear();
  int64_t i = 0;
  while (i < nef) {
    int64_t j = i + 1;
    int64_t ki[3], kj[3];
    key(order[i], ki);
    while (j < nef) {
      key(order[j], kj);
      bool same = true;
      for (int c = 0; c < d; ++c) same = same && (ki[c] == kj[c]);
      if (!same) break;
      ++j;
    }
    const int64_t cnt = j - i;
    if (cnt > 2) { err = "mesh: non-manifold facet (more than two neighbours)"; return HOPU_EMESH; }
    const bool bnd = (cnt == 1);  // boundary facet: its single element is side A
    const int64_t F = (int64_t)m.fa.size();
    int side_a = -1;
    double nA[3] = {0, 0, 0}, aA = 0.0;
    for (int64_t t = i; t < j; ++t) {
      const int64_t id = order[t];
      const int64_t e = id / nvl;
      const int f = (int)(id % nvl);
      double cr[3];
      facet_cross(m, e, f, cr);
      double area = 0.0;
      for (int c = 0; c < d; ++c) area += cr[c] * cr[c];
      area = std::sqrt(area);
      // outward direction J^{-T} Nhat_f, Nhat_0 = (1,..,1), Nhat_f = -e_{f-1}
      const double* Ji = &m.geo[(size_t)e * G + d * d];
      double dot = 0.0;
      for (int b = 0; b < d; ++b) {
        double o = 0.0;
        for (int c = 0; c < d; ++c) {
          const double N = (f == 0) ? 1.0 : (c == f - 1 ? -1.0 : 0.0);
          o += Ji[c * d + b] * N;
        }
        dot += o * cr[b];
      }
      // a boundary facet whose element points against the canonical normal is flipped
      const bool flip = bnd && !(dot > 0.0);
      if (flip) {
        for (int c = 0; c < d; ++c) cr[c] = -cr[c];
        dot = -dot;
      }
      const bool is_a = dot > 0.0;
      const double det = m.geo[(size_t)e * G + 2 * d * d];
      const bool sigma_neg = ((dot > 0.0) != (det > 0.0));
      m.efc[(size_t)id] = (int32_t)(F * 4 + (sigma_neg ? 2 : 0) + (is_a ? 0 : 1));
      if (is_a) {
        if (side_a >= 0) { err = "mesh: both neighbours of a facet lie on the same side"; return HOPU_EMESH; }
        side_a = (int)(t - i);
        m.fa.push_back((int32_t)(e * 4 + f));
        for (int c = 0; c < d; ++c) nA[c] = cr[c] / area;
        aA = area;
      }
    }
    if (side_a < 0) { err = "mesh: both neighbours of a facet lie on the same side"; return HOPU_EMESH; }
    if (bnd) {
      m.fb.push_back(m.fa.back());  // side B = side A: the wall / outlet rule (no jump)
      m.boundary.push_back(F);
    } else {
      const int64_t idb = order[i + (side_a == 0 ? 1 : 0)];
      m.fb.push_back((int32_t)((idb / nvl) * 4 + (idb % nvl)));
    }
    for (int c = 0; c < d; ++c) m.fgeo.push_back(nA[c]);
    m.fgeo.push_back(aA);
    i = j;
  }
  m.n_facets = (int64_t)m.fa.size();
  return HOPU_OK;
}

void facet_points(const MeshTopo& m, const std::vector<double>& sq, int nqf, double* out) {
  const int d = m.dim;
  for (int64_t F = 0; F < m.n_facets; ++F) {
    const int64_t e = m.fa[F] >> 2;
    const int f = m.fa[F] & 3;
    const double* X = &m.X[(size_t)e * (d + 1) * d];
    int loc[3], c = 0;
    for (int v = 0; v <= d; ++v)
      if (v != f) loc[c++] = v;
    for (int q = 0; q < nqf; ++q)
      for (int a = 0; a < d; ++a) {
        double x = X[loc[0] * d + a];
        for (int jj = 0; jj < d - 1; ++jj) x += sq[(size_t)q * (d - 1) + jj] * (X[loc[jj + 1] * d + a] - X[loc[0] * d + a]);
        out[((size_t)F * nqf + q) * d + a] = x;
      }
  }
}

void volume_points(const MeshTopo& m, const std::vector<double>& xq, int nq, double* out) {
  const int d = m.dim;
  const int G = geo_stride(d);
  for (int64_t e = 0; e < m.n_elems; ++e) {
    const double* X = &m.X[(size_t)e * (d + 1) * d];
    const double* J = &m.geo[(size_t)e * G];
    for (int q = 0; q < nq; ++q)
      for (int a = 0; a < d; ++a) {
        double x = X[a];
        for (int b = 0; b < d; ++b) x += J[a * d + b] * xq[(size_t)q * d + b];
        out[((size_t)e * nq + q) * d + a] = x;
      }
  }
}

}  // namespace hopu
