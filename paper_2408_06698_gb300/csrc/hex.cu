// C ABI of the hexahedral path (include/hopu_hex.h): box geometry and 1D tables on the
// host in FP64, the sum-factorised kernels of kernels_hex.cuh on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hopu_hex.h"
#include "kernels_hex.cuh"
#include "reftables.h"

using namespace hopu::hex;

struct hopu_hex {
  int n[3] = {0, 0, 0};
  int k = 0, prec = 0, bmask = 0;
  int64_t E = 0;
  cudaStream_t stream = nullptr;
  double* d_geo = nullptr;   // G [E][9] | invabs [E] | nF [3E][3] | aF [3E]
  void* d_tab = nullptr;     // B | Dd | w1 | e0 | e1 | e0lo | e1lo in the working precision
  void* d_gam = nullptr;     // facet moments [3E][2][3][(k+1)^2] (side A, side B)
  void* d_u1 = nullptr;      // two stage vectors
  void* d_u2 = nullptr;
  int grid[4] = {0, 0, 0, 0};  // facet, volume, volume (w = u), facet (eta): set at the first launch
  const int8_t* facet_l = nullptr;  // per-facet orders (hopu_hex_set_facet_l), caller-owned
  void* d_inlet[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};  // inlet modes
  bool inlet_on[3][2] = {{false, false}, {false, false}, {false, false}};
  double* d_part = nullptr;  // FP64 partial sums of the reductions
  int64_t n_part = 0;
  std::string err;
};

namespace {

std::string g_create_err;

int fail(hopu_hex* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(hopu_hex* h, cudaError_t e, const char* where) {
  return fail(h, HOPU_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Orthonormal Legendre polynomials on [0,1] up to degree k at x: the three-term recurrence
// (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1} of P_n on [-1,1] at t = 2x - 1, and its
// t-derivative; values v[k+1] and x-derivatives dv[k+1] of sqrt(2n+1) P_n(2x - 1).
void legendre01(int k, double x, double* v, double* dv) {
  const double t = 2.0 * x - 1.0;
  double pm = 0.0, p = 1.0, dpm = 0.0, dp = 0.0;
  for (int n = 0; n <= k; ++n) {
    const double s = std::sqrt(2.0 * n + 1.0);
    v[n] = s * p;
    dv[n] = 2.0 * s * dp;
    const double pn = ((2 * n + 1) * t * p - n * pm) / (n + 1);
    const double dpn = ((2 * n + 1) * (p + t * dp) - n * dpm) / (n + 1);
    pm = p;
    p = pn;
    dpm = dp;
    dp = dpn;
  }
}

template <typename T>
std::vector<T> tables(int k) {
  const int K1 = k + 1, M = (3 * k + 2) / 2;
  std::vector<double> x, w;
  hopu::gauss_jacobi01(M, 0, x, w);
  std::vector<T> out(2 * M * K1 + M + 4 * K1);
  std::vector<double> v(K1), dv(K1);
  for (int q = 0; q < M; ++q) {
    legendre01(k, x[q], v.data(), dv.data());
    for (int i = 0; i < K1; ++i) {
      out[q * K1 + i] = T(v[i]);
      out[M * K1 + q * K1 + i] = T(dv[i]);
    }
    out[2 * M * K1 + q] = T(w[q]);
  }
  // end values and the part of each that T drops (zero for double)
  for (int side = 0; side < 2; ++side) {
    legendre01(k, side ? 1.0 : 0.0, v.data(), dv.data());
    for (int i = 0; i < K1; ++i) {
      const T hi = T(v[i]);
      out[2 * M * K1 + M + side * K1 + i] = hi;
      out[2 * M * K1 + M + (2 + side) * K1 + i] = T(v[i] - double(hi));
    }
  }
  return out;
}

double det3(const double* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
}

// inverse of a 3x3 row-major matrix
void inv3(const double* a, double* o) {
  const double d = det3(a);
  o[0] = (a[4] * a[8] - a[5] * a[7]) / d;
  o[1] = (a[2] * a[7] - a[1] * a[8]) / d;
  o[2] = (a[1] * a[5] - a[2] * a[4]) / d;
  o[3] = (a[5] * a[6] - a[3] * a[8]) / d;
  o[4] = (a[0] * a[8] - a[2] * a[6]) / d;
  o[5] = (a[2] * a[3] - a[0] * a[5]) / d;
  o[6] = (a[3] * a[7] - a[4] * a[6]) / d;
  o[7] = (a[1] * a[6] - a[0] * a[7]) / d;
  o[8] = (a[0] * a[4] - a[1] * a[3]) / d;
}

MeshDev mesh_dev(const hopu_hex* h) {
  MeshDev m;
  m.n0 = h->n[0];
  m.n1 = h->n[1];
  m.n2 = h->n[2];
  m.bmask = h->bmask;
  m.E = h->E;
  m.G = h->d_geo;
  m.invabs = h->d_geo + 9 * h->E;
  m.nF = m.invabs + h->E;
  m.aF = m.nF + 9 * h->E;
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 2; ++e) m.inlet[d][e] = h->inlet_on[d][e] ? h->d_inlet[d][e] : nullptr;
  m.facet_l = h->facet_l;
  return m;
}

template <typename T, int K>
Tabs<T> tabs_dev(const hopu_hex* h) {
  constexpr int K1 = K + 1, M = Shape<K>::M;
  const T* t = static_cast<const T*>(h->d_tab);
  Tabs<T> tb;
  tb.B = t;
  tb.Dd = t + M * K1;
  tb.w1 = t + 2 * M * K1;
  tb.e0 = tb.w1 + M;
  tb.e1 = tb.e0 + K1;
  tb.e0lo = tb.e1 + K1;
  tb.e1lo = tb.e0lo + K1;
  return tb;
}

// grid of a persistent launch (resident CTAs x SMs, at most one CTA per items_per_block
// items); computed once per context and kernel (the dynamic shared memory attribute is set
// on that first call)
template <typename Kern>
cudaError_t grid_for(Kern kern, int threads, size_t smem, int64_t items_per_block, int64_t items, int* grid) {
  if (*grid > 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (items + items_per_block - 1) / items_per_block;
  const int64_t full = (int64_t)sms * per_sm;
  *grid = (int)(need < full ? need : full);
  if (*grid < 1) *grid = 1;
  return cudaSuccess;
}

// one apply: facet moments, then volume + lift + inverse mass + out = c0 u0 + c1 us + c2 y
template <typename T, int K>
int stage(hopu_hex* h, const T* w, const T* us, int l, const T* u0, T c0, T c1, T c2, T* out,
          double* diss = nullptr) {
  const MeshDev m = mesh_dev(h);
  const Tabs<T> tb = tabs_dev<T, K>(h);
  T* gam = static_cast<T*>(h->d_gam);
  int& gf = h->grid[0];
  using CF = Fac<T, K>;
  // a fully periodic box runs the facet kernel without the boundary-facet code
  auto kf = h->bmask ? k_hex_facet<T, K, true> : k_hex_facet<T, K, false>;
  cudaError_t ga = grid_for(kf, 32 * CF::WARPS, CF::SMEM, CF::WARPS, 3 * h->E, &gf);
  if (ga != cudaSuccess) return cuda_fail(h, ga, "hopu_hex: k_hex_facet attributes");
  kf<<<gf, 32 * CF::WARPS, CF::SMEM, h->stream>>>(m, tb, w, us, l, gam, diss, EtaArgs{});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "k_hex_facet launch");
  if (w == us) {  // the wind is the convected field: each component interpolated once
    int& gv = h->grid[2];
    auto kv = k_hex_volume_same<T, K>;
    using CV = VolS<T, K>;
    if ((ga = grid_for(kv, 32 * CV::WARPS, CV::SMEM, CV::WARPS, h->E, &gv)) != cudaSuccess)
      return cuda_fail(h, ga, "hopu_hex: k_hex_volume_same attributes");
    kv<<<gv, 32 * CV::WARPS, CV::SMEM, h->stream>>>(m, tb, us, gam, u0, c0, c1, c2, out);
  } else {
    int& gv = h->grid[1];
    auto kv = k_hex_volume<T, K>;
    using CV = Vol<T, K>;
    if ((ga = grid_for(kv, 32 * CV::WARPS, CV::SMEM, CV::WARPS, h->E, &gv)) != cudaSuccess)
      return cuda_fail(h, ga, "hopu_hex: k_hex_volume attributes");
    kv<<<gv, 32 * CV::WARPS, CV::SMEM, h->stream>>>(m, tb, w, us, gam, u0, c0, c1, c2, out);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "k_hex_volume launch");
  return HOPU_OK;
}

template <typename T, int K>
int substeps(hopu_hex* h, T* u, double dt, int n, int l) {
  T* u1 = static_cast<T*>(h->d_u1);
  T* u2 = static_cast<T*>(h->d_u2);
  const T z = T(0), one = T(1);
  for (int s = 0; s < n; ++s) {
    int st;
    if ((st = stage<T, K>(h, u, u, l, u, z, one, T(-dt), u1)) != HOPU_OK) return st;
    if ((st = stage<T, K>(h, u1, u1, l, u, T(0.75), T(0.25), T(-0.25 * dt), u2)) != HOPU_OK) return st;
    if ((st = stage<T, K>(h, u2, u2, l, u, T(1.0 / 3.0), T(2.0 / 3.0), T(-2.0 / 3.0 * dt), u)) != HOPU_OK)
      return st;
  }
  return HOPU_OK;
}

template <typename T>
int dispatch_apply(hopu_hex* h, const T* w, const T* u, int l, T* y, double* diss = nullptr) {
  switch (h->k) {
    case 2: return stage<T, 2>(h, w, u, l, u, T(0), T(0), T(1), y, diss);
    case 3: return stage<T, 3>(h, w, u, l, u, T(0), T(0), T(1), y, diss);
    case 4: return stage<T, 4>(h, w, u, l, u, T(0), T(0), T(1), y, diss);
    case 5: return stage<T, 5>(h, w, u, l, u, T(0), T(0), T(1), y, diss);
  }
  return fail(h, HOPU_ENOTSUP, "hopu_hex: order");
}

// the adaptive step (see hopu_hex_adapt_l)
template <typename T, int K>
int adapt(hopu_hex* h, const T* u, const double* thr, int8_t* facet_l, double* eta_out) {
  MeshDev m = mesh_dev(h);
  m.facet_l = facet_l;
  EtaArgs ea{};
  for (int i = 0; i <= K; ++i) ea.thr[i] = thr[i];
  ea.l_out = facet_l;
  ea.eta_out = eta_out;
  using CF = Fac<T, K>;
  auto kf = k_hex_facet<T, K, false, true>;
  cudaError_t ga = grid_for(kf, 32 * CF::WARPS, CF::SMEM, CF::WARPS, 3 * h->E, &h->grid[3]);
  if (ga != cudaSuccess) return cuda_fail(h, ga, "hopu_hex: k_hex_facet (eta) attributes");
  kf<<<h->grid[3], 32 * CF::WARPS, CF::SMEM, h->stream>>>(m, tabs_dev<T, K>(h), u, u, -1,
                                                          static_cast<T*>(h->d_gam), nullptr, ea);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "k_hex_facet (eta) launch");
  return HOPU_OK;
}

template <typename T>
int dispatch_adapt(hopu_hex* h, const T* u, const double* thr, int8_t* facet_l, double* eta_out) {
  switch (h->k) {
    case 2: return adapt<T, 2>(h, u, thr, facet_l, eta_out);
    case 3: return adapt<T, 3>(h, u, thr, facet_l, eta_out);
    case 4: return adapt<T, 4>(h, u, thr, facet_l, eta_out);
    case 5: return adapt<T, 5>(h, u, thr, facet_l, eta_out);
  }
  return fail(h, HOPU_ENOTSUP, "hopu_hex: order");
}

// kinetic energy, c(w; u, u) and the facet dissipation in FP64 (see hopu_hex_energy)
template <typename T>
int energy(hopu_hex* h, const T* w, const T* u, int l, double* out) {
  const int64_t K1 = h->k + 1, nl = h->E * 3 * K1 * K1 * K1;
  int dev = 0, sms = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "hopu_hex_energy: device");
  const int ge = (int)std::min<int64_t>((nl + 255) / 256, 4LL * sms);
  const int64_t nfac = (int64_t)sms * 32 * 4;  // facet partials: at most 32 CTAs of 4 warps per SM
  if (!h->d_part) {
    h->n_part = nfac + 2 * ge;
    if ((ce = cudaMalloc(&h->d_part, h->n_part * sizeof(double))) != cudaSuccess)
      return cuda_fail(h, ce, "hopu_hex_energy: partial sums");
  }
  T* y = static_cast<T*>(h->d_u1);
  int st;
  if (w) {
    if ((ce = cudaMemsetAsync(h->d_part, 0, nfac * sizeof(double), h->stream)) != cudaSuccess)
      return cuda_fail(h, ce, "hopu_hex_energy: memset");
    if ((st = dispatch_apply<T>(h, w, u, l, y, h->d_part)) != HOPU_OK) return st;
  }
  k_hex_energy<T><<<ge, 256, 0, h->stream>>>(mesh_dev(h), nl, u, w ? y : nullptr, h->d_part + nfac);
  if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, ce, "k_hex_energy launch");
  std::vector<double> part(h->n_part);
  if ((ce = cudaMemcpyAsync(part.data(), h->d_part, h->n_part * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream)) != cudaSuccess ||
      (ce = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    return cuda_fail(h, ce, "hopu_hex_energy: read back");
  double e0 = 0.0, e1 = 0.0, d = 0.0;
  for (int b = 0; b < ge; ++b) {
    e0 += part[nfac + 2 * b];
    e1 += part[nfac + 2 * b + 1];
  }
  if (w)
    for (int64_t j = 0; j < nfac; ++j) d += part[j];
  out[0] = 0.5 * e0;
  out[1] = w ? e1 : 0.0;
  out[2] = w ? d : 0.0;
  return HOPU_OK;
}

template <typename T>
int dispatch_substeps(hopu_hex* h, T* u, double dt, int n, int l) {
  switch (h->k) {
    case 2: return substeps<T, 2>(h, u, dt, n, l);
    case 3: return substeps<T, 3>(h, u, dt, n, l);
    case 4: return substeps<T, 4>(h, u, dt, n, l);
    case 5: return substeps<T, 5>(h, u, dt, n, l);
  }
  return fail(h, HOPU_ENOTSUP, "hopu_hex: order");
}

void release(hopu_hex* h) {
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 2; ++e) cudaFree(h->d_inlet[d][e]);
  cudaFree(h->d_part);
  cudaFree(h->d_geo);
  cudaFree(h->d_tab);
  cudaFree(h->d_gam);
  cudaFree(h->d_u1);
  cudaFree(h->d_u2);
}

}  // namespace

extern "C" {

int hopu_hex_create(int n0, int n1, int n2, const double* lines, const double* A, int periodic, int k, int prec,
                    void* stream, hopu_hex** out) {
  if (!out || !lines || !A) return fail(nullptr, HOPU_EINVAL, "hopu_hex_create: NULL argument");
  *out = nullptr;
  if (n0 < 3 || n1 < 3 || n2 < 3) return fail(nullptr, HOPU_EINVAL, "hopu_hex_create: fewer than 3 cells in a direction");
  if (prec != HOPU_FP64 && prec != HOPU_FP32)
    return fail(nullptr, HOPU_EINVAL, "hopu_hex_create: precision must be HOPU_FP64 or HOPU_FP32");
  if (k < 2 || k > 5) return fail(nullptr, HOPU_ENOTSUP, "hopu_hex_create: order k outside 2..5");
  if (periodic < 0 || periodic > 7) return fail(nullptr, HOPU_EINVAL, "hopu_hex_create: periodic is a 3-bit mask");
  const int n[3] = {n0, n1, n2};
  const double* ln[3] = {lines, lines + n0 + 1, lines + n0 + 1 + n1 + 1};
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < n[a]; ++i)
      if (!(ln[a][i + 1] > ln[a][i])) return fail(nullptr, HOPU_EMESH, "hopu_hex_create: grid lines not increasing");
  const double detA = det3(A);
  if (!(detA > 0.0)) return fail(nullptr, HOPU_EMESH, "hopu_hex_create: det A <= 0");
  const int64_t E = (int64_t)n0 * n1 * n2;

  // geometry (FP64): J = A diag(h), |det J| J^-1 = |det J| diag(1/h) A^-1; facet normals
  // and area factors from side A (the lower cell): n dA = det J J^-T e_d
  double Ai[9];
  inv3(A, Ai);
  std::vector<double> geo(9 * E + E + 9 * E + 3 * E);
  double* G = geo.data();
  double* invabs = G + 9 * E;
  double* nF = invabs + E;
  double* aF = nF + 9 * E;
  for (int64_t e = 0; e < E; ++e) {
    const int c[3] = {int(e % n0), int((e / n0) % n1), int(e / ((int64_t)n0 * n1))};
    double h[3];
    for (int a = 0; a < 3; ++a) h[a] = ln[a][c[a] + 1] - ln[a][c[a]];
    const double detJ = detA * h[0] * h[1] * h[2];
    for (int r = 0; r < 3; ++r)
      for (int b = 0; b < 3; ++b) G[e * 9 + r * 3 + b] = detJ * Ai[r * 3 + b] / h[r];
    invabs[e] = 1.0 / detJ;
  }
  for (int d = 0; d < 3; ++d)
    for (int64_t e = 0; e < E; ++e) {
      int c[3] = {int(e % n0), int((e / n0) % n1), int(e / ((int64_t)n0 * n1))};
      c[d] = (c[d] - 1 + n[d]) % n[d];  // side A: the cell below
      const int64_t eA = c[0] + (int64_t)n0 * (c[1] + (int64_t)n1 * c[2]);
      double v[3];
      for (int b = 0; b < 3; ++b) v[b] = G[eA * 9 + d * 3 + b];  // row d of det J J^-1
      const double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      const int64_t F = d * E + e;
      for (int b = 0; b < 3; ++b) nF[F * 3 + b] = v[b] / nv;
      aF[F] = nv;
    }

  hopu_hex* h = new (std::nothrow) hopu_hex;
  if (!h) return fail(nullptr, HOPU_ENOMEM, "hopu_hex_create: host allocation");
  h->n[0] = n0;
  h->n[1] = n1;
  h->n[2] = n2;
  h->k = k;
  h->prec = prec;
  h->bmask = (~periodic) & 7;
  h->E = E;
  h->stream = static_cast<cudaStream_t>(stream);
  const size_t ts = prec == HOPU_FP64 ? 8 : 4;
  const int K1 = k + 1;
  const size_t nl2 = (size_t)E * 3 * K1 * K1 * K1;
  cudaError_t ce;
  if ((ce = cudaMalloc(&h->d_geo, geo.size() * 8)) != cudaSuccess ||
      (ce = cudaMalloc(&h->d_gam, (size_t)3 * E * 6 * K1 * K1 * ts)) != cudaSuccess ||
      (ce = cudaMalloc(&h->d_u1, nl2 * ts)) != cudaSuccess || (ce = cudaMalloc(&h->d_u2, nl2 * ts)) != cudaSuccess) {
    const int st = cuda_fail(nullptr, ce, "hopu_hex_create: device allocation");
    release(h);
    delete h;
    return ce == cudaErrorMemoryAllocation ? HOPU_ENOMEM : st;
  }
  if ((ce = cudaMemcpy(h->d_geo, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess) {
    release(h);
    delete h;
    return cuda_fail(nullptr, ce, "hopu_hex_create: upload");
  }
  if (prec == HOPU_FP64) {
    const std::vector<double> t = tables<double>(k);
    ce = cudaMalloc(&h->d_tab, t.size() * 8);
    if (ce == cudaSuccess) ce = cudaMemcpy(h->d_tab, t.data(), t.size() * 8, cudaMemcpyHostToDevice);
  } else {
    const std::vector<float> t = tables<float>(k);
    ce = cudaMalloc(&h->d_tab, t.size() * 4);
    if (ce == cudaSuccess) ce = cudaMemcpy(h->d_tab, t.data(), t.size() * 4, cudaMemcpyHostToDevice);
  }
  if (ce != cudaSuccess) {
    release(h);
    delete h;
    return cuda_fail(nullptr, ce, "hopu_hex_create: tables");
  }
  *out = h;
  return HOPU_OK;
}

int hopu_hex_destroy(hopu_hex* h) {
  if (!h) return HOPU_EINVAL;
  release(h);
  delete h;
  return HOPU_OK;
}

int hopu_hex_sizes(const hopu_hex* h, int64_t* n_cells, int64_t* n_l2) {
  if (!h) return HOPU_EINVAL;
  const int64_t K1 = h->k + 1;
  if (n_cells) *n_cells = h->E;
  if (n_l2) *n_l2 = h->E * 3 * K1 * K1 * K1;
  return HOPU_OK;
}

int hopu_hex_apply(hopu_hex* h, const void* wL, const void* uL, int l, void* yL) {
  if (!h) return HOPU_EINVAL;
  if (!wL || !uL || !yL) return fail(h, HOPU_EINVAL, "hopu_hex_apply: NULL vector");
  if (yL == wL || yL == uL) return fail(h, HOPU_EINVAL, "hopu_hex_apply: yL aliases an input");
  if (h->prec == HOPU_FP64)
    return dispatch_apply<double>(h, static_cast<const double*>(wL), static_cast<const double*>(uL), l,
                                  static_cast<double*>(yL));
  return dispatch_apply<float>(h, static_cast<const float*>(wL), static_cast<const float*>(uL), l,
                               static_cast<float*>(yL));
}

int hopu_hex_rk_substeps(hopu_hex* h, void* uL, double dt, int n, int l) {
  if (!h) return HOPU_EINVAL;
  if (!uL || n < 0 || !std::isfinite(dt)) return fail(h, HOPU_EINVAL, "hopu_hex_rk_substeps: bad argument");
  if (h->prec == HOPU_FP64) return dispatch_substeps<double>(h, static_cast<double*>(uL), dt, n, l);
  return dispatch_substeps<float>(h, static_cast<float*>(uL), dt, n, l);
}

int hopu_hex_set_inlet(hopu_hex* h, int dir, int end, const void* modes) {
  if (!h) return HOPU_EINVAL;
  if (dir < 0 || dir > 2 || end < 0 || end > 1) return fail(h, HOPU_EINVAL, "hopu_hex_set_inlet: dir / end");
  if (!((h->bmask >> dir) & 1)) return fail(h, HOPU_EINVAL, "hopu_hex_set_inlet: direction is periodic");
  if (!modes) {
    h->inlet_on[dir][end] = false;
    return HOPU_OK;
  }
  const int64_t K1 = h->k + 1;
  const int64_t nface = (int64_t)h->n[0] * h->n[1] * h->n[2] / h->n[dir];
  const size_t bytes = (size_t)(nface * 3 * K1 * K1) * (h->prec == HOPU_FP64 ? 8 : 4);
  cudaError_t ce;
  if (!h->d_inlet[dir][end] && (ce = cudaMalloc(&h->d_inlet[dir][end], bytes)) != cudaSuccess)
    return cuda_fail(h, ce, "hopu_hex_set_inlet: allocation");
  if ((ce = cudaMemcpyAsync(h->d_inlet[dir][end], modes, bytes, cudaMemcpyDeviceToDevice, h->stream)) != cudaSuccess)
    return cuda_fail(h, ce, "hopu_hex_set_inlet: copy");
  h->inlet_on[dir][end] = true;
  return HOPU_OK;
}

int hopu_hex_set_facet_l(hopu_hex* h, const int8_t* facet_l) {
  if (!h) return HOPU_EINVAL;
  h->facet_l = facet_l;
  return HOPU_OK;
}

int hopu_hex_adapt_l(hopu_hex* h, const void* uL, const double* thresholds, int8_t* facet_l, double* eta_out) {
  if (!h) return HOPU_EINVAL;
  if (!uL || !thresholds || !facet_l) return fail(h, HOPU_EINVAL, "hopu_hex_adapt_l: NULL argument");
  if (h->bmask) return fail(h, HOPU_ENOTSUP, "hopu_hex_adapt_l: the box has boundary facets");
  for (int i = 0; i <= h->k; ++i)
    if (!(thresholds[i] > 0.0 && thresholds[i] < 1.0) || (i > 0 && !(thresholds[i] > thresholds[i - 1])))
      return fail(h, HOPU_EINVAL, "hopu_hex_adapt_l: thresholds must be k+1 increasing values in (0, 1)");
  if (h->prec == HOPU_FP64)
    return dispatch_adapt<double>(h, static_cast<const double*>(uL), thresholds, facet_l, eta_out);
  return dispatch_adapt<float>(h, static_cast<const float*>(uL), thresholds, facet_l, eta_out);
}

int hopu_hex_energy(hopu_hex* h, const void* wL, const void* uL, int l, double* host_out) {
  if (!h) return HOPU_EINVAL;
  if (!uL || !host_out) return fail(h, HOPU_EINVAL, "hopu_hex_energy: NULL argument");
  if (h->prec == HOPU_FP64)
    return energy<double>(h, static_cast<const double*>(wL), static_cast<const double*>(uL), l, host_out);
  return energy<float>(h, static_cast<const float*>(wL), static_cast<const float*>(uL), l, host_out);
}

const char* hopu_hex_last_error(const hopu_hex* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
