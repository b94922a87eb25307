// C ABI of libhopu (declared in include/hopu.h): context management, the explicit
// SSP-RK3 substep driver with CUDA-graph replay, FP64 reductions and the host-side
// interpolation / point queries.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/hopu.h"
#include "hopu_internal.h"
#include "meshtopo.h"
#include "reftables.h"

namespace hopu {
Ops* make_ops_2_1(bool, int);
Ops* make_ops_2_2(bool, int);
Ops* make_ops_2_3(bool, int);
Ops* make_ops_2_4(bool, int);
Ops* make_ops_3_1(bool, int);
Ops* make_ops_3_2(bool, int);
Ops* make_ops_3_3(bool, int);
Ops* make_ops_3_4(bool, int);
Ops* make_ops_3_5(bool, int);

Ops* make_ops(int dim, int k, bool fp64, int tc) {
  if (dim == 2) {
    switch (k) {
      case 1: return make_ops_2_1(fp64, tc);
      case 2: return make_ops_2_2(fp64, tc);
      case 3: return make_ops_2_3(fp64, tc);
      case 4: return make_ops_2_4(fp64, tc);
      default: return nullptr;
    }
  }
  if (dim == 3) {
    switch (k) {
      case 1: return make_ops_3_1(fp64, tc);
      case 2: return make_ops_3_2(fp64, tc);
      case 3: return make_ops_3_3(fp64, tc);
      case 4: return make_ops_3_4(fp64, tc);
      case 5: return make_ops_3_5(fp64, tc);
      default: return nullptr;
    }
  }
  return nullptr;
}

// ---------------------------------------------------------------- FP64 reductions
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kRedThreads];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  return red[0];
}

// partial[b] = sum over this block's strided entries of |det J_e| a_t b_t
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_weighted_dot(int64_t E, int NL, int G, const double* geo,
                                                              const T* a, const T* b, double* partial) {
  double s = 0.0;
  const int64_t n = E * NL;
  if (n < (int64_t(1) << 31)) {  // 32-bit index arithmetic (a 64-bit division per entry is slow)
    const int n32 = (int)n, stride = (int)gridDim.x * kRedThreads;
    for (int t = (int)blockIdx.x * kRedThreads + (int)threadIdx.x; t < n32; t += stride)
      s += geo[(int64_t)(t / NL) * G + G - 1] * (double(a[t]) * double(b[t]));
  } else {
    for (int64_t t = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; t < n; t += (int64_t)gridDim.x * kRedThreads)
      s += geo[(t / NL) * G + G - 1] * (double(a[t]) * double(b[t]));
  }
  const double tot = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// sum_t u_t^2 over one element's NL entries.  FP32: every square split exactly into
// p + e (p = fl(u*u), e = fma(u, u, -p)) and the p summed with TwoSum (Knuth), so the pair
// hi + lo carries the element sum to about NL * 2^-48 relative; FP64: fused multiply-adds.
// GB300 issues FP64 at a small fraction of its FP32 rate: this keeps FP64 arithmetic to a
// few operations per element.  Up to 16 float4 loads are issued before the first is used.
__device__ __forceinline__ void two_sum_sq(float x, float& hi, float& lo) {
  const float p = __fmul_rn(x, x), e = __fmaf_rn(x, x, -p);
  const float s = __fadd_rn(hi, p), bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  lo = __fadd_rn(lo, __fadd_rn(err, e));
  hi = s;
}
__device__ __forceinline__ double elem_sq(const float* u, int NL) {
  float hi = 0.f, lo = 0.f;
  if ((NL & 3) == 0 && (reinterpret_cast<uintptr_t>(u) & 15) == 0) {
    const float4* v = reinterpret_cast<const float4*>(u);
    const int n4 = NL / 4;
    for (int i = 0; i < n4; i += 16) {
      float4 q[16];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (i + j < n4) q[j] = __ldg(v + i + j);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (i + j < n4)
          two_sum_sq(q[j].x, hi, lo), two_sum_sq(q[j].y, hi, lo), two_sum_sq(q[j].z, hi, lo), two_sum_sq(q[j].w, hi, lo);
    }
  } else {
#pragma unroll 4
    for (int i = 0; i < NL; ++i) two_sum_sq(__ldg(u + i), hi, lo);
  }
  return double(hi) + double(lo);
}
__device__ __forceinline__ double elem_sq(const double* u, int NL) {
  double s = 0.0;
#pragma unroll 8
  for (int i = 0; i < NL; ++i) s = fma(__ldg(u + i), __ldg(u + i), s);
  return s;
}

// butterfly sum over the warp (the same order, and result, in every lane)
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Kinetic energy of the state into the device log in one kernel: one thread per element
// (strided), |det J_e| sum_t u_t^2 accumulated in FP64; every block writes its partial to
// partial[block]; the block that arrives last (ticket) sums the partials in block order
// (deterministic), writes 1/2 * total to log[*pos % cap], advances *pos and resets the
// ticket, so replayed graphs log every substep.  Small blocks spread the elements over
// every SM.  Launched as a programmatic dependent of the projection before it.
constexpr int kElogThreads = 64;
template <typename T>
__global__ void __launch_bounds__(kElogThreads) k_energy_log(int64_t E, int NL, int G, const double* geo,
                                                             const T* u, double* partial, unsigned* ticket,
                                                             double* log, int64_t cap, int64_t* pos) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  constexpr int NW = kElogThreads / 32;
  __shared__ double ws[NW];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * kElogThreads + threadIdx.x; e < E; e += (int64_t)gridDim.x * kElogThreads)
    s = fma(__ldg(geo + e * G + G - 1), elem_sq(u + e * NL, NL), s);
  s = warp_sum(s);
  if (lane == 0) ws[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < NW; ++w) tot += ws[w];
    partial[blockIdx.x] = tot;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s2 = 0.0;
  for (int t0 = threadIdx.x; t0 < (int)gridDim.x; t0 += 8 * kElogThreads) {  // 8 loads in flight
    double q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) q[j] = (t0 + j * kElogThreads < (int)gridDim.x) ? __ldcg(partial + t0 + j * kElogThreads) : 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s2 += q[j];
  }
  s2 = warp_sum(s2);
  if (lane == 0) ws[warp] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int w = 0; w < NW; ++w) total += ws[w];
    const int64_t p = *pos;
    log[p % cap] = 0.5 * total;
    *pos = p + 1;
    *ticket = 0u;
  }
}

// blocks of the energy-log kernel: one thread per element, at most 8 blocks per SM
int64_t elog_blocks(int64_t n_elems, int nsm) {
  const int64_t need = (n_elems + kElogThreads - 1) / kElogThreads;
  return std::max<int64_t>(1, std::min<int64_t>(need, 8 * (int64_t)nsm));
}

// x = a x + b y (n entries)
template <typename T>
__global__ void __launch_bounds__(256) k_axpby(int64_t n, Combine w, T* x, const T* y) {
  for (int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256)
    if constexpr (sizeof(T) == 8) x[t] = fma(T(w.a0), x[t], T(w.a2) * y[t]);  // w = {a, x, 0, null, b}
    else x[t] = fmaf(w.h2, y[t], fmaf(w.h0, x[t], fmaf(w.l2, y[t], w.l0 * x[t])));
}

// Copy element blocks of nl values: pack (dst[j] = src[ids[j]]) or unpack (dst[ids[j]] =
// src[j]), j < n.  An id outside [0, E) is skipped and flagged in the error word (bit 2).
template <typename T, bool PACK>
__global__ void __launch_bounds__(256) k_copy_blocks(int64_t E, int nl, const int32_t* __restrict__ ids, int64_t n,
                                                     const T* __restrict__ src, T* __restrict__ dst, int* err) {
  const int64_t total = n * nl;
  for (int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x; t < total; t += (int64_t)gridDim.x * 256) {
    const int64_t j = t / nl;
    const int off = (int)(t - j * nl);
    const int32_t id = ids[j];
    if (id < 0 || id >= E) {
      atomicOr(err, 4);
      continue;
    }
    if (PACK) dst[t] = src[(int64_t)id * nl + off];
    else dst[(int64_t)id * nl + off] = src[t];
  }
}

// y = M x for an L2 field (M = |det J| I per element): the gradient of 1/2 int |x|^2
template <typename T>
__global__ void __launch_bounds__(256) k_mass(int64_t E, int NL, int G, const double* geo, const T* x, T* y) {
  const int64_t n = E * NL;
  for (int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256)
    y[t] = T(geo[(t / NL) * G + G - 1]) * x[t];
}

__global__ void __launch_bounds__(kRedThreads) k_sum(const double* in, int64_t n, double* out) {
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += kRedThreads) s += in[t];
  const double tot = block_sum(s);
  if (threadIdx.x == 0) *out = tot;
}

}  // namespace hopu

using namespace hopu;

#include "context.h"


namespace {

hopu_status fail(hopu_ctx* c, int code, const std::string& msg) {
  if (c && c->status == HOPU_OK) {
    c->status = code;
    c->err = msg;
  }
  return (hopu_status)code;
}

hopu_status cuda_fail(hopu_ctx* c, cudaError_t e, const char* where) {
  return fail(c, HOPU_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define HOPU_CUDA(ctx, call)                                 \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

#define HOPU_PRECHECK(ctx)                           \
  do {                                               \
    if (!(ctx)) return HOPU_EINVAL;                  \
    if ((ctx)->status != HOPU_OK) return (hopu_status)(ctx)->status; \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

hopu_status check_launch(hopu_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return HOPU_OK;
}

// Read the device error word (the stream must have been synchronised): ETIMEOUT when a
// tensor-core kernel gave up waiting for its MMAs (bit 0: k_v2l_tc, bit 1: k_volume_tc,
// bit 3: k_l2v_tc); EINVAL for bit 2 (pack / unpack ids); the word is cleared once read.
hopu_status device_status(hopu_ctx* c) {
  int e = 0;
  HOPU_CUDA(c, cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e & 4) {
    HOPU_CUDA(c, cudaMemset(c->d_err, 0, sizeof(int)));
    return fail(c, HOPU_EINVAL, "pack / unpack: an element id was outside the mesh (those blocks were skipped)");
  }
  if (e & 11) {
    HOPU_CUDA(c, cudaMemset(c->d_err, 0, sizeof(int)));
    std::string who = (e & 1) ? "k_v2l_tc / k_v2l_tcr (V_h -> L2 projection)" : "";
    if (e & 2) who += std::string(who.empty() ? "" : " and ") + "k_volume_tc (volume term)";
    if (e & 8) who += std::string(who.empty() ? "" : " and ") + "k_l2v_tc (back-projection)";
    return fail(c, HOPU_ETIMEOUT, "a tensor-core MMA completion wait gave up in " + who +
                                      "; the outputs of that launch are incomplete");
  }
  return HOPU_OK;
}

void free_all(hopu_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  void* ptrs[] = {c->d_elog_pos, c->d_mesh, c->d_geoT, c->d_tabs, c->d_gam, c->d_lf, c->d_uL, c->d_yL, c->d_wL,
                  c->d_wfz, c->d_s1, c->d_s2, c->d_diss, c->d_red, c->d_gamW, c->d_adj, c->d_err, c->d_tcvol,
                  c->d_inlet, c->d_inlet_modes, c->d_csr, c->d_tcl2v, c->d_tcv2l, c->d_csr_tc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c->ops;
}

size_t align16(size_t n) { return (n + 15) / 16 * 16; }

template <typename T>
void convert(const std::vector<double>& src, std::vector<unsigned char>& dst, size_t off) {
  T* p = reinterpret_cast<T*>(dst.data() + off);
  for (size_t i = 0; i < src.size(); ++i) p[i] = (T)src[i];
}

// Reorder the host FP64 tables into the kernel layouts (see hopu_internal.h).
constexpr int kNumTables = 14;

// Row stride of the point-major tables: an odd multiple of 16 bytes (matches
// row_stride<T> in kernels.cuh).
int point_row_stride(int n, bool fp64) {
  if (!fp64) return (n + 3) / 4 * 4 + (((n + 3) / 4) % 2 == 0 ? 4 : 0);
  return (n + 1) / 2 * 2 + (((n + 1) / 2) % 2 == 0 ? 2 : 0);
}

void kernel_tables(const RefTables& R, bool fp64, std::vector<std::vector<double>>& out) {
  const int d = R.dim, nb = R.nb, nf = R.nf, nq = R.nq, nqk = R.nqk, nqf = R.nqf, nl = R.nloc;
  const int nbq = point_row_stride(nb, fp64);
  const int nb1 = nbasis(d, R.k - 1);
  out.assign(kNumTables, {});
  auto& Bt = out[0];
  auto& Wq = out[1];
  auto& Dm = out[2];
  auto& TrM = out[3];
  auto& TrP = out[4];
  auto& Psi = out[5];
  auto& WPsi = out[6];
  auto& Wf = out[7];
  auto& DinvT = out[8];
  auto& DT = out[9];
  auto& Dinv = out[10];
  auto& Drow = out[11];
  auto& Dn = out[12];
  Bt.assign((size_t)nqk * nbq, 0.0);  // point-major [q][nbq], the volume kernels' rule
  for (int q = 0; q < nqk; ++q)
    for (int i = 0; i < nb; ++i) Bt[(size_t)q * nbq + i] = R.phik[(size_t)q * nb + i];
  Wq = R.wk;
  // modal differentiation: d phi_i / d xhat_c = sum_{j < nb(k-1)} Dm[c][j][i] phi_j, with
  // Dm[c][j][i] = int (d phi_i / d xhat_c) phi_j (exact: degree 2k-2 <= 3k-1)
  Dm.assign((size_t)d * nb1 * nb, 0.0);
  for (int c = 0; c < d; ++c)
    for (int j = 0; j < nb1; ++j)
      for (int i = 0; i < nb; ++i) {
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) acc += R.wq[q] * R.dphi[((size_t)q * nb + i) * d + c] * R.phi[(size_t)q * nb + j];
        Dm[((size_t)c * nb1 + j) * nb + i] = acc;
      }
  // reference gradients at the kernels' volume points: d phi_i / d xhat_c = sum_j Dm[c][j][i] phi_j
  auto& dBt = out[13];
  dBt.assign((size_t)d * nqk * nbq, 0.0);
  for (int c = 0; c < d; ++c)
    for (int q = 0; q < nqk; ++q)
      for (int i = 0; i < nb; ++i) {
        double acc = 0.0;
        for (int j = 0; j < nb1; ++j) acc += Dm[((size_t)c * nb1 + j) * nb + i] * R.phik[(size_t)q * nb + j];
        dBt[((size_t)c * nqk + q) * nbq + i] = acc;
      }
  TrM = R.trm;
  TrP.assign((size_t)(d + 1) * nqf * nbq, 0.0);  // point-major [f][q][nbq]
  for (int f = 0; f <= d; ++f)
    for (int q = 0; q < nqf; ++q)
      for (int i = 0; i < nb; ++i) TrP[((size_t)f * nqf + q) * nbq + i] = R.phif[((size_t)f * nqf + q) * nb + i];
  Psi.resize((size_t)nf * nqf);
  WPsi.resize((size_t)nf * nqf);
  for (int m = 0; m < nf; ++m)
    for (int q = 0; q < nqf; ++q) {
      Psi[(size_t)m * nqf + q] = R.psi[(size_t)q * nf + m];
      WPsi[(size_t)m * nqf + q] = R.wf[q] * R.psi[(size_t)q * nf + m];
    }
  Wf = R.wf;
  // n_loc x n_loc tables for the projection GEMMs, [s][r] with rows padded to nlp
  const int nlp = (nl + 3) / 4 * 4;
  DinvT.assign((size_t)nl * nlp, 0.0);
  DT.assign((size_t)nl * nlp, 0.0);
  Dinv.assign((size_t)nl * nlp, 0.0);
  for (int r = 0; r < nl; ++r)
    for (int s = 0; s < nl; ++s) {
      DinvT[(size_t)s * nlp + r] = R.Dinv[(size_t)r * nl + s];
      DT[(size_t)s * nlp + r] = R.D[(size_t)r * nl + s];
      Dinv[(size_t)s * nlp + r] = R.Dinv[(size_t)s * nl + r];
    }
  Dn.assign((size_t)nl * nlp, 0.0);  // Dn[s][r] = D[s][r] (transposed back-projection)
  for (int r = 0; r < nl; ++r)
    for (int s = 0; s < nl; ++s) Dn[(size_t)s * nlp + r] = R.D[(size_t)s * nl + r];
  // row-major D with an odd-multiple-of-16-byte row stride (fused back-projection)
  const int nlr = point_row_stride(nl, fp64);
  Drow.assign((size_t)nl * nlr, 0.0);
  for (int r = 0; r < nl; ++r)
    for (int s = 0; s < nl; ++s) Drow[(size_t)r * nlr + s] = R.D[(size_t)r * nl + s];
}

// The nonzeros of the dof matrix D (row s = functional, column r = basis function b*nb + i)
// for the residual of the refined FP32 projection: nloc row headers {s, first entry, count,
// grouped} (int32 bits) sorted by count, largest first, then one entry {r (int32 bits), hi, lo, 0}
// per nonzero with hi = float(D[s][r]), lo = float(D[s][r] - hi).  Entries below 1e-13 of
// max |D| are the exact zeros of the orthogonality relations, rounded by the quadrature.
std::vector<std::vector<std::pair<int, double>>> dof_matrix_rows(const RefTables& R) {
  const int nl = R.nloc;
  double mx = 0.0;
  for (double v : R.D) mx = std::max(mx, std::fabs(v));
  std::vector<std::vector<std::pair<int, double>>> rows(nl);
  for (int s = 0; s < nl; ++s)
    for (int r = 0; r < nl; ++r) {
      const double v = R.D[(size_t)s * nl + r];
      if (std::fabs(v) > 1e-13 * mx) rows[s].push_back({r, v});
    }
  return rows;
}

// Rows whose dim component blocks are equal entry by entry (the facet whose reference
// normal has equal components: D[s][b nb + i] = T[s][i] for every b) are grouped: only
// block 0's nonzeros are kept (column i < nb) and D Y for the row is sum_i T[s][i] S_i with
// S_i = sum_b Y[b nb + i].  Used by the refined tensor-core projection only.
std::vector<bool> grouped_rows(const RefTables& R) {
  const int nl = R.nloc, nb = R.nb, d = R.dim;
  std::vector<bool> g(nl, false);
  for (int s = 0; s < nl; ++s) {
    bool eq = true;
    for (int i = 0; i < nb && eq; ++i)
      for (int b = 1; b < d; ++b)
        if (R.D[(size_t)s * nl + b * nb + i] != R.D[(size_t)s * nl + i]) eq = false;
    g[s] = eq;
  }
  return g;
}

// The order of the CSR rows: by number of stored nonzeros, largest first (stable).
std::vector<int> csr_row_order(const RefTables& R, bool grouped) {
  auto rows = dof_matrix_rows(R);
  const std::vector<bool> g = grouped ? grouped_rows(R) : std::vector<bool>(R.nloc, false);
  std::vector<size_t> cnt(R.nloc);
  for (int s = 0; s < R.nloc; ++s) {
    size_t c = 0;
    for (const auto& e : rows[s]) c += (!g[s] || e.first < R.nb);
    cnt[s] = c;
  }
  std::vector<int> order(R.nloc);
  for (int s = 0; s < R.nloc; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] > cnt[b]; });
  return order;
}

// grouped: rows with equal component blocks keep block 0 only and carry the flag 1 in the
// fourth header word.
void dof_matrix_csr(const RefTables& R, std::vector<float>& out, bool grouped = false) {
  const int nl = R.nloc;
  auto rows = dof_matrix_rows(R);
  const std::vector<int> order = csr_row_order(R, grouped);
  const std::vector<bool> g = grouped ? grouped_rows(R) : std::vector<bool>(nl, false);
  for (int s = 0; s < nl; ++s)
    if (g[s]) {
      std::vector<std::pair<int, double>> keep;
      for (const auto& e : rows[s])
        if (e.first < R.nb) keep.push_back(e);
      rows[s] = keep;
    }
  size_t nnz = 0;
  for (const auto& r : rows) nnz += r.size();
  out.assign(4 * (nl + nnz), 0.0f);
  auto put_int = [&](size_t i, int v) { std::memcpy(&out[i], &v, 4); };
  int next = nl;
  for (int h = 0; h < nl; ++h) {
    const int s = order[h];
    put_int(4 * h, s);
    put_int(4 * h + 1, next);
    put_int(4 * h + 2, (int)rows[s].size());
    put_int(4 * h + 3, g[s] ? 1 : 0);
    for (const auto& e : rows[s]) {
      const float hi = (float)e.second;
      put_int(4 * (size_t)next, e.first);
      out[4 * (size_t)next + 1] = hi;
      out[4 * (size_t)next + 2] = (float)(e.second - (double)hi);
      ++next;
    }
  }
}

// Round an FP32 value to TF32 (10 mantissa bits), to nearest with ties away from zero.
float tf32_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Tables of the tensor-core volume kernel, FP32, in the blocked K-major operand layout of
// the tensor cores (core matrices of 8 rows x 4 values, 128 bytes each):
//   phiA[q][i] = phi_i(x_q)  (128 x KP1, KP1 = nb rounded up to 8)   hi part, then lo part
//   phiB[i][q] = phi_i(x_q)  (N2 x 128, N2 = nb rounded up to 16)     hi part, then lo part
// hi = tf32(phi), lo = tf32(phi - hi); zero outside the points and the basis.
void tensor_core_volume_table(const RefTables& R, std::vector<float>& out) {
  const int nb = R.nb, nq = R.nqk, KP1 = (nb + 7) / 8 * 8, N2 = (nb + 15) / 16 * 16, K2 = 128;
  const size_t PA = (size_t)128 * KP1, PB = (size_t)N2 * K2;
  out.assign(2 * PA + 2 * PB, 0.0f);
  auto off = [](int row, int col, int kp) {
    return (size_t)(((row >> 3) * (kp >> 2) + (col >> 2)) * 32 + (row & 7) * 4 + (col & 3));
  };
  for (int q = 0; q < nq && q < 128; ++q)
    for (int i = 0; i < nb; ++i) {
      const float v = (float)R.phik[(size_t)q * nb + i];
      const float h = tf32_round(v), l = tf32_round(v - h);
      out[off(q, i, KP1)] = h;
      out[PA + off(q, i, KP1)] = l;
      out[2 * PA + off(i, q, K2)] = h;
      out[2 * PA + PB + off(i, q, K2)] = l;
    }
}

// B operand of the tensor-core back-projection: B[r][kappa(b, i)] = D[r][b nb + i] (r the
// local functional, b the component, i the basis index, kappa the K column of l2v_tc_gw),
// N = nloc padded to 16 rows; hi = tf32(D), lo = tf32(D - hi), the hi parts then the lo
// parts, in the blocked K-major layout of tensor_core_volume_table.
void tensor_core_l2v_table(const RefTables& R, std::vector<float>& out) {
  const int d = R.dim, nb = R.nb, nl = R.nloc;
  const int IPG = l2v_tc_ipg(nb), GW = l2v_tc_gw(d, nb), KP = l2v_tc_kp(d, nb), NP = l2v_tc_np(nl);
  const size_t P = (size_t)NP * KP;
  out.assign(2 * P, 0.0f);
  auto off = [&](int row, int col) {
    return (size_t)(((row >> 3) * (KP >> 2) + (col >> 2)) * 32 + (row & 7) * 4 + (col & 3));
  };
  for (int r = 0; r < nl; ++r)
    for (int s2 = 0; s2 < nl; ++s2) {
      const double v = R.D[(size_t)r * nl + s2];
      const float h = tf32_round((float)v), l = tf32_round((float)(v - (double)h));
      const int b = s2 / nb, i = s2 % nb, g = i / IPG;
      const int col = g * GW + b * IPG + (i - g * IPG);
      out[off(r, col)] = h;
      out[P + off(r, col)] = l;
    }
}

// B operand of the refined tensor-core projection: B[r][kappa(h)] = Dinv[r][s_h] (r the basis
// index, s_h the local functional of CSR row h, kappa(h) = (h % 4) GW + h / 4 the K column
// of v2l_tc_gw), N = nloc padded to 16 rows; hi / lo TF32 parts, the hi parts then the lo
// parts, blocked K-major as above.
void tensor_core_v2l_table(const RefTables& R, std::vector<float>& out) {
  const int nl = R.nloc, GW = v2l_tc_gw(nl), KP = v2l_tc_kp(nl), NP = (nl + 15) / 16 * 16;
  const std::vector<int> order = csr_row_order(R, true);
  const size_t P = (size_t)NP * KP;
  out.assign(2 * P, 0.0f);
  auto off = [&](int row, int col) {
    return (size_t)(((row >> 3) * (KP >> 2) + (col >> 2)) * 32 + (row & 7) * 4 + (col & 3));
  };
  for (int r = 0; r < nl; ++r)
    for (int h = 0; h < nl; ++h) {
      const double v = R.Dinv[(size_t)r * nl + order[h]];
      const float hi = tf32_round((float)v), lo = tf32_round((float)(v - (double)hi));
      const int col = (h % 4) * GW + h / 4;
      out[off(r, col)] = hi;
      out[P + off(r, col)] = lo;
    }
}

void enqueue_v2l(hopu_ctx* c, const void* uV, void* uL) {
  timed(c, HOPU_K_V2L, [&] { c->ops->v2l(c->dm, c->dt, uV, uL, c->stream); });
}

void enqueue_l2v(hopu_ctx* c, const void* yL, bool dual, Combine cmb, void* outV) {
  timed(c, HOPU_K_L2V_ELEM, [&] { c->ops->l2v_elem(c->dm, c->dt, yL, dual, c->d_lf, cmb, outV, c->stream); });
  timed(c, HOPU_K_L2V_FACET, [&] { c->ops->l2v_facet(c->dm, c->d_lf, dual, cmb, outV, c->stream); });
}

hopu_status enqueue_stage_apply(hopu_ctx* c, const void* uL, const void* wL, int l, const int8_t* facet_l,
                                double* diss, Combine cmb, void* out) {
  timed(c, HOPU_K_FACET, [&] { c->ops->facet(c->dm, c->dt, uL, wL, l, facet_l, c->d_gam, diss, c->stream); });
  timed(c, HOPU_K_VOLUME, [&] { c->ops->volume(c->dm, c->dt, uL, wL, c->d_gam, cmb, out, c->stream); });
  return check_launch(c, "apply kernels");
}

// STAGE wind, after u_L = E u_V: facet flux, volume term with the element part of the
// back-projection fused in (when the kernel family has it), facet averaging R.
hopu_status enqueue_stage_fused(hopu_ctx* c, Combine cmb, void* outV) {
  timed(c, HOPU_K_FACET, [&] { c->ops->facet(c->dm, c->dt, c->d_uL, c->d_uL, c->l, c->facet_l, c->d_gam, nullptr, c->stream); });
  if (c->ops->has_fused()) {
    timed(c, HOPU_K_VOLUME, [&] { c->ops->volume_l2v(c->dm, c->dt, c->d_uL, c->d_gam, c->d_lf, cmb, outV, c->stream); });
  } else {
    Combine plain;
    timed(c, HOPU_K_VOLUME, [&] { c->ops->volume(c->dm, c->dt, c->d_uL, c->d_uL, c->d_gam, plain, c->d_yL, c->stream); });
    timed(c, HOPU_K_L2V_ELEM, [&] { c->ops->l2v_elem(c->dm, c->dt, c->d_yL, false, c->d_lf, cmb, outV, c->stream); });
  }
  timed(c, HOPU_K_L2V_FACET, [&] { c->ops->l2v_facet(c->dm, c->d_lf, false, cmb, outV, c->stream); });
  return check_launch(c, "stage kernels");
}

hopu_status energy_log(hopu_ctx* c, const void* uL) {
  const int G = geo_stride(c->dim);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)elog_blocks(c->topo.n_elems, c->nsm));
  cfg.blockDim = dim3(kElogThreads);
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  unsigned* ticket = reinterpret_cast<unsigned*>(c->d_elog_pos + 1);
  double* partial = reinterpret_cast<double*>(c->d_elog_pos + 2);
  if (c->fp64)
    cudaLaunchKernelEx(&cfg, k_energy_log<double>, (int64_t)c->topo.n_elems, (int)c->ref.nloc, G, c->dm.geo,
                       (const double*)uL, partial, ticket, c->elog, c->elog_cap, c->d_elog_pos);
  else
    cudaLaunchKernelEx(&cfg, k_energy_log<float>, (int64_t)c->topo.n_elems, (int)c->ref.nloc, G, c->dm.geo,
                       (const float*)uL, partial, ticket, c->elog, c->elog_cap, c->d_elog_pos);
  return check_launch(c, "energy log kernel");
}

// One SSP-RK3 (Shu-Osher) substep on the context stream.
hopu_status enqueue_substep(hopu_ctx* c, void* state, double dt) {
  const Combine st[3] = {
      {1.0, state, 0.0, nullptr, -dt},
      {0.75, state, 0.25, c->d_s1, -0.25 * dt},
      {1.0 / 3.0, state, 2.0 / 3.0, c->d_s2, -2.0 / 3.0 * dt},
  };
  const void* in[3] = {state, c->d_s1, c->d_s2};
  void* out[3] = {c->d_s1, c->d_s2, state};
  for (int s = 0; s < 3; ++s) {
    if (s == 0 && c->elog) {  // a8: kinetic energy of the state at the start of the substep
      if (c->wind == HOPU_WIND_STAGE) enqueue_v2l(c, in[0], c->d_uL);
      const void* uL0 = (c->wind == HOPU_WIND_STAGE) ? c->d_uL : in[0];
      hopu_status r = energy_log(c, uL0);
      if (r != HOPU_OK) return r;
      if (c->wind == HOPU_WIND_STAGE) {
        r = enqueue_stage_fused(c, st[s], out[s]);
        if (r != HOPU_OK) return r;
        continue;
      }
    }
    if (c->wind == HOPU_WIND_STAGE) {
      enqueue_v2l(c, in[s], c->d_uL);
      hopu_status r = enqueue_stage_fused(c, st[s], out[s]);
      if (r != HOPU_OK) return r;
    } else {
      hopu_status r = enqueue_stage_apply(c, in[s], c->d_wfz, c->l, c->facet_l, nullptr, st[s], out[s]);
      if (r != HOPU_OK) return r;
    }
  }
  return check_launch(c, "substep kernels");
}

// ---------------------------------------------------------------- derivatives
// facet-moment scratch of the wind cotangent (the apply's own d_gam holds the other set)
hopu_status ensure_gamW(hopu_ctx* c) {
  if (c->d_gamW) return HOPU_OK;
  const size_t n = (size_t)c->topo.n_elems * (c->dim + 1) * c->ref.nf * c->dim;
  HOPU_CUDA(c, cudaMalloc(&c->d_gamW, n * c->tsize));
  return HOPU_OK;
}

// VJP of the apply y = M^{-1} c(w; u, .) for the L2 wind wL: facet moments, then volume
// part + lift.  wL == uL means w = u (ubar then receives ubar + wbar, wbarL unused).
void enqueue_apply_vjp(hopu_ctx* c, const void* uL, const void* wL, const void* ybar, void* ubar, void* wbarL) {
  timed(c, HOPU_K_FACET_ADJ, [&] {
    c->ops->facet_adj(c->dm, c->dt, uL, wL, ybar, c->l, c->facet_l, c->d_gam, c->d_gamW, c->stream);
  });
  timed(c, HOPU_K_VOLUME_ADJ, [&] {
    c->ops->volume_adj(c->dm, c->dt, uL, wL, ybar, c->d_gam, c->d_gamW, ubar, wbarL, c->stream);
  });
}

// out = cmb(J_F(u)^T vbar) with F(u) = R E^{-1} y(Eu, Eu), the STAGE right-hand side:
// J_F^T vbar = E^T J_y^T(Eu) (R E^{-1})^T vbar.
hopu_status enqueue_rhs_vjp(hopu_ctx* c, const void* uV, const void* vbar, Combine cmb, void* out) {
  enqueue_v2l(c, uV, c->d_uL);
  timed(c, HOPU_K_V2L, [&] { c->ops->v2l_pt(c->dm, c->dt, vbar, c->d_yL, c->stream); });
  enqueue_apply_vjp(c, c->d_uL, c->d_uL, c->d_yL, c->d_wL, nullptr);
  enqueue_l2v(c, c->d_wL, true, cmb, out);
  return check_launch(c, "rhs vjp kernels");
}

void enqueue_axpby(hopu_ctx* c, int64_t n, double a, void* x, double b, const void* y) {
  const int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->nsm * 8);
  const Combine w{a, x, 0.0, nullptr, b};
  if (c->fp64) k_axpby<double><<<g, 256, 0, c->stream>>>(n, w, (double*)x, (const double*)y);
  else k_axpby<float><<<g, 256, 0, c->stream>>>(n, w, (float*)x, (const float*)y);
}

void enqueue_mass(hopu_ctx* c, const void* x, void* y) {
  const int64_t n = c->n_l2;
  const int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->nsm * 8);
  const int G = geo_stride(c->dim);
  if (c->fp64) k_mass<double><<<g, 256, 0, c->stream>>>(c->topo.n_elems, c->ref.nloc, G, c->dm.geo, (const double*)x, (double*)y);
  else k_mass<float><<<g, 256, 0, c->stream>>>(c->topo.n_elems, c->ref.nloc, G, c->dm.geo, (const float*)x, (float*)y);
}

// cnt STAGE substeps of `work` in place, keeping the substep states (u, u1, u2) of
// substep j in seg[3j], seg[3j+1], seg[3j+2] (each `slot` bytes apart).
hopu_status stored_substeps(hopu_ctx* c, void* work, double dt, int cnt, unsigned char* seg, size_t slot) {
  void* s1 = c->d_s1;
  void* s2 = c->d_s2;
  hopu_status r = HOPU_OK;
  for (int j = 0; j < cnt && r == HOPU_OK; ++j) {
    unsigned char* b = seg + 3 * (size_t)j * slot;
    cudaError_t e = cudaMemcpyAsync(b, work, c->n_hdiv * c->tsize, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) {
      r = cuda_fail(c, e, "vjp_rollout: checkpoint copy");
      break;
    }
    c->d_s1 = b + slot;
    c->d_s2 = b + 2 * slot;
    r = enqueue_substep(c, work, dt);
  }
  c->d_s1 = s1;
  c->d_s2 = s2;
  return r;
}

hopu_status weighted_dot(hopu_ctx* c, const void* a, const void* b, int slot) {
  const int G = geo_stride(c->dim);
  if (c->fp64)
    k_weighted_dot<double><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
        c->topo.n_elems, c->ref.nloc, G, c->dm.geo, (const double*)a, (const double*)b, c->d_red);
  else
    k_weighted_dot<float><<<c->red_blocks, kRedThreads, 0, c->stream>>>(
        c->topo.n_elems, c->ref.nloc, G, c->dm.geo, (const float*)a, (const float*)b, c->d_red);
  k_sum<<<1, kRedThreads, 0, c->stream>>>(c->d_red, c->red_blocks, c->d_red + c->red_blocks + slot);
  return check_launch(c, "reduction kernels");
}

}  // namespace

namespace {
thread_local std::string g_create_error;

// Autotuner of the kernel variants, run at create on this context's own mesh
// (zero-filled scratch; one warm-up launch, then three launches between CUDA events on
// the context stream, the faster variant kept):
//  * the element part of a STAGE stage (volume term, lift, inverse mass and the element
//    back-projection): the register-resident kernel with the back-projection fused or as a
//    separate launch, the warp-per-element fused kernel, the tensor-core kernel - whichever
//    this (dim, k, precision) has;
//  * the V_h -> L2 projection in HOPU_TF32: FMA or tensor cores;
//  * the element back-projection in the tensor-core modes: FMA or tensor cores (timed
//    first, so that the volume variants with a separate back-projection use the choice).
// tile_hint 1 keeps to the FMA kernels, 2 to the tensor-core kernels where they exist.
// hopu_tuning / hopu_tuning_volume / hopu_tuning_l2v report the choice and the times.
hopu_status autotune(hopu_ctx* c, int hint) {
  Ops* o = c->ops;
  std::vector<int> cand;
  for (int v = 0; v < kVolVariants; ++v) {
    if (!o->volume_variant_ok(v)) continue;
    if (hint == 1 && v == kVolTensor) continue;
    if (hint == 2 && o->volume_variant_ok(kVolTensor) && v != kVolTensor) continue;
    cand.push_back(v);
  }
  const bool tc_v2l = o->tensor_cores();
  int v2l = (tc_v2l && hint == 2) ? 1 : 0;
  o->select(v2l, 0);
  const bool tc_l2v = o->tensor_core_l2v();
  o->select_l2v(tc_l2v && hint == 2);
  if (cand.size() <= 1 && !(tc_v2l && hint == 0) && !(tc_l2v && hint == 0)) {
    if (cand.size() == 1) o->select_volume_variant(cand[0]);
    return HOPU_OK;
  }
  const int64_t nstate = std::max(c->n_hdiv, c->n_l2);
  HOPU_CUDA(c, cudaMemsetAsync(c->d_s1, 0, c->tsize * nstate, c->stream));
  HOPU_CUDA(c, cudaMemsetAsync(c->d_uL, 0, c->tsize * c->n_l2, c->stream));
  HOPU_CUDA(c, cudaMemsetAsync(c->d_gam, 0, c->tsize * c->topo.n_elems * (c->dim + 1) * c->ref.nf * c->dim,
                               c->stream));
  cudaEvent_t a = nullptr, b = nullptr;
  HOPU_CUDA(c, cudaEventCreate(&a));
  HOPU_CUDA(c, cudaEventCreate(&b));
  auto timed_ms = [&](auto&& launch) -> float {
    launch();
    cudaEventRecord(a, c->stream);
    for (int i = 0; i < 3; ++i) launch();
    cudaEventRecord(b, c->stream);
    float ms = 1e30f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) ms = 1e30f;
    return ms;
  };
  if (tc_v2l && hint == 0) {
    o->select(0, 0);
    const float t0 = timed_ms([&] { o->v2l(c->dm, c->dt, c->d_s1, c->d_uL, c->stream); });
    o->select(1, 0);
    const float t1 = timed_ms([&] { o->v2l(c->dm, c->dt, c->d_s1, c->d_uL, c->stream); });
    v2l = t1 < t0;
    o->select(v2l, 0);
  }
  Combine plain;
  if (tc_l2v && hint == 0) {
    auto l2v = [&] { o->l2v_elem(c->dm, c->dt, c->d_uL, false, c->d_lf, plain, c->d_s2, c->stream); };
    o->select_l2v(0);
    const float t0 = timed_ms(l2v);
    o->select_l2v(1);
    const float t1 = timed_ms(l2v);
    c->l2v_ms[0] = t0 / 3.0;
    c->l2v_ms[1] = t1 / 3.0;
    o->select_l2v(t1 < t0);
  }
  auto stage_volume = [&]() {
    if (!o->volume_l2v(c->dm, c->dt, c->d_uL, c->d_gam, c->d_lf, plain, c->d_s2, c->stream)) {
      o->volume(c->dm, c->dt, c->d_uL, c->d_uL, c->d_gam, plain, c->d_yL, c->stream);
      o->l2v_elem(c->dm, c->dt, c->d_yL, false, c->d_lf, plain, c->d_s2, c->stream);
    }
  };
  int best = cand.empty() ? -1 : cand[0];
  if (cand.size() > 1) {
    float tbest = 1e30f;
    for (int v : cand) {
      o->select_volume_variant(v);
      const float t = timed_ms(stage_volume);
      c->vol_ms[v] = t / 3.0;
      if (t < tbest) {
        tbest = t;
        best = v;
      }
    }
  }
  if (best >= 0) o->select_volume_variant(best);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  HOPU_CUDA(c, cudaStreamSynchronize(c->stream));
  return device_status(c);
}

hopu_status create_impl(const hopu_mesh_desc* mesh, const hopu_options* opts, void* cuda_stream, hopu_ctx** out) {
  if (!mesh || !opts) return HOPU_EINVAL;
  if (opts->prec != HOPU_FP64 && opts->prec != HOPU_FP32 && opts->prec != HOPU_FP32_TC && opts->prec != HOPU_TF32)
    return HOPU_EINVAL;
  if (opts->wind_mode != HOPU_WIND_STAGE && opts->wind_mode != HOPU_WIND_FROZEN) return HOPU_EINVAL;
  if (mesh->dim != 2 && mesh->dim != 3) return HOPU_EINVAL;
  if (opts->k < 1 || opts->k > (mesh->dim == 2 ? 4 : 5)) return HOPU_ENOTSUP;
  if (opts->l < -1 || opts->l > opts->k) return HOPU_EINVAL;
  if (opts->tile_hint < 0 || opts->tile_hint > 2) return HOPU_EINVAL;
  hopu_ctx* c = new (std::nothrow) hopu_ctx();
  if (!c) return HOPU_ENOMEM;
  c->dim = mesh->dim;
  c->k = opts->k;
  c->l = opts->l;
  c->prec = opts->prec;
  c->wind = opts->wind_mode;
  c->fp64 = opts->prec == HOPU_FP64;
  c->tsize = c->fp64 ? 8 : 4;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = c;
  std::string err;
  int rc = build_mesh_topo(mesh->dim, mesh->n_vertices, mesh->coords, mesh->n_elems, mesh->elem_vertices,
                           mesh->vertex_rep, c->topo, err);
  if (rc != HOPU_OK) return fail(c, rc, err);
  if (!build_ref_tables(c->dim, c->k, c->ref, err)) return fail(c, HOPU_EINVAL, err);
  const RefTables& R = c->ref;
  const int64_t E = c->topo.n_elems, NF = c->topo.n_facets;
  c->n_l2 = E * R.nloc;
  c->n_hdiv = NF * R.nf + E * R.nint;
  c->ops = make_ops(c->dim, c->k, c->fp64, c->prec == HOPU_FP32_TC ? 3 : (c->prec == HOPU_TF32 ? 1 : 0));
  if (!c->ops) return fail(c, HOPU_ENOTSUP, "no kernel family for this (dim, k)");
  cudaError_t ce = c->ops->prepare();
  if (ce != cudaSuccess) return cuda_fail(c, ce, "kernel setup");
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
  c->red_blocks = 2 * c->nsm;

  // mesh upload
  const int G = geo_stride(c->dim);
  const size_t s_geo = align16(sizeof(double) * E * G), s_efc = align16(sizeof(int32_t) * E * (c->dim + 1));
  const size_t s_f = align16(sizeof(int32_t) * NF), s_fgeo = align16(sizeof(double) * NF * (c->dim + 1));
  std::vector<unsigned char> hm(s_geo + s_efc + 2 * s_f + s_fgeo, 0);
  std::memcpy(hm.data(), c->topo.geo.data(), sizeof(double) * E * G);
  std::memcpy(hm.data() + s_geo, c->topo.efc.data(), sizeof(int32_t) * E * (c->dim + 1));
  std::memcpy(hm.data() + s_geo + s_efc, c->topo.fa.data(), sizeof(int32_t) * NF);
  std::memcpy(hm.data() + s_geo + s_efc + s_f, c->topo.fb.data(), sizeof(int32_t) * NF);
  std::memcpy(hm.data() + s_geo + s_efc + 2 * s_f, c->topo.fgeo.data(), sizeof(double) * NF * (c->dim + 1));
  HOPU_CUDA(c, cudaMalloc(&c->d_mesh, hm.size()));
  HOPU_CUDA(c, cudaMemcpy(c->d_mesh, hm.data(), hm.size(), cudaMemcpyHostToDevice));
  unsigned char* base = static_cast<unsigned char*>(c->d_mesh);
  c->dm.E = E;
  c->dm.NF = NF;
  c->dm.geo = reinterpret_cast<const double*>(base);
  c->dm.efc = reinterpret_cast<const int32_t*>(base + s_geo);
  c->dm.fa = reinterpret_cast<const int32_t*>(base + s_geo + s_efc);
  c->dm.fb = reinterpret_cast<const int32_t*>(base + s_geo + s_efc + s_f);
  c->dm.fgeo = reinterpret_cast<const double*>(base + s_geo + s_efc + 2 * s_f);

  // geometry factors, computed and kept in FP64 (the FP32 kernels round them at load)
  {
    const int d = c->dim, GT = geoT_stride(d);
    std::vector<double> gt((size_t)E * GT, 0.0);
    for (int64_t e = 0; e < E; ++e) {
      const double* g = &c->topo.geo[(size_t)e * G];
      const double det = g[2 * d * d], ad = g[2 * d * d + 1];
      double* o = &gt[(size_t)e * GT];
      for (int i = 0; i < d * d; ++i) {
        o[i] = g[i] / det;                  // Pf = J / det J
        o[d * d + i] = det * g[d * d + i];  // Pi = det J * Jinv
        o[2 * d * d + i] = ad * g[d * d + i];  // M = |det J| * Jinv
      }
      o[3 * d * d] = 1.0 / ad;
    }
    HOPU_CUDA(c, cudaMalloc(&c->d_geoT, sizeof(double) * gt.size()));
    HOPU_CUDA(c, cudaMemcpy(c->d_geoT, gt.data(), sizeof(double) * gt.size(), cudaMemcpyHostToDevice));
    c->dm.geoT = static_cast<const double*>(c->d_geoT);
  }

  // tables upload, converted to the working precision
  std::vector<std::vector<double>> tabs;
  kernel_tables(R, c->fp64, tabs);
  std::vector<size_t> offs;
  size_t total = 0;
  for (auto& t : tabs) {
    offs.push_back(total);
    total += align16(c->tsize * t.size());
  }
  std::vector<unsigned char> ht(total, 0);
  for (size_t i = 0; i < tabs.size(); ++i) {
    if (c->fp64) convert<double>(tabs[i], ht, offs[i]);
    else convert<float>(tabs[i], ht, offs[i]);
  }
  HOPU_CUDA(c, cudaMalloc(&c->d_tabs, total));
  HOPU_CUDA(c, cudaMemcpy(c->d_tabs, ht.data(), total, cudaMemcpyHostToDevice));
  unsigned char* tb = static_cast<unsigned char*>(c->d_tabs);
  const void** slots[kNumTables] = {&c->dt.Bt,   &c->dt.Wq,  &c->dt.Dm,    &c->dt.TrM,
                                    &c->dt.TrP,  &c->dt.Psi, &c->dt.WPsi,  &c->dt.Wf,
                                    &c->dt.DinvT, &c->dt.DT, &c->dt.Dinv, &c->dt.Drow, &c->dt.Dn,
                                    &c->dt.dBt};
  for (int i = 0; i < kNumTables; ++i) *slots[i] = tb + offs[i];
  if (!c->fp64) {
    std::vector<float> csr;
    dof_matrix_csr(R, csr);
    HOPU_CUDA(c, cudaMalloc(&c->d_csr, csr.size() * sizeof(float)));
    HOPU_CUDA(c, cudaMemcpy(c->d_csr, csr.data(), csr.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->dt.Dcsr = c->d_csr;
    c->dt.csr_n = (int)(csr.size() / 4);
  }
  if (c->ops->tensor_core_volume()) {
    std::vector<float> tv;
    tensor_core_volume_table(R, tv);
    HOPU_CUDA(c, cudaMalloc(&c->d_tcvol, tv.size() * sizeof(float)));
    HOPU_CUDA(c, cudaMemcpy(c->d_tcvol, tv.data(), tv.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->dt.tcvol = c->d_tcvol;
  }
  if (c->ops->tensor_cores() && c->prec == HOPU_FP32_TC) {
    std::vector<float> csr;
    dof_matrix_csr(R, csr, true);
    HOPU_CUDA(c, cudaMalloc(&c->d_csr_tc, csr.size() * sizeof(float)));
    HOPU_CUDA(c, cudaMemcpy(c->d_csr_tc, csr.data(), csr.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->dt.Dcsr_tc = c->d_csr_tc;
    c->dt.csr_tc_n = (int)(csr.size() / 4);
    std::vector<float> tv;
    tensor_core_v2l_table(R, tv);
    HOPU_CUDA(c, cudaMalloc(&c->d_tcv2l, tv.size() * sizeof(float)));
    HOPU_CUDA(c, cudaMemcpy(c->d_tcv2l, tv.data(), tv.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->dt.tcv2l = c->d_tcv2l;
  }
  if (c->ops->tensor_core_l2v()) {
    std::vector<float> tv;
    tensor_core_l2v_table(R, tv);
    HOPU_CUDA(c, cudaMalloc(&c->d_tcl2v, tv.size() * sizeof(float)));
    HOPU_CUDA(c, cudaMemcpy(c->d_tcl2v, tv.data(), tv.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->dt.tcl2v = c->d_tcl2v;
  }

  // scratch
  const size_t ts = c->tsize;
  const int64_t nstate = std::max(c->n_hdiv, c->n_l2);
  HOPU_CUDA(c, cudaMalloc(&c->d_gam, ts * E * (c->dim + 1) * R.nf * c->dim));
  HOPU_CUDA(c, cudaMalloc(&c->d_lf, ts * E * (c->dim + 1) * R.nf));
  HOPU_CUDA(c, cudaMalloc(&c->d_uL, ts * c->n_l2));
  HOPU_CUDA(c, cudaMalloc(&c->d_yL, ts * c->n_l2));
  HOPU_CUDA(c, cudaMalloc(&c->d_wL, ts * c->n_l2));
  HOPU_CUDA(c, cudaMalloc(&c->d_wfz, ts * c->n_l2));
  HOPU_CUDA(c, cudaMalloc(&c->d_s1, ts * nstate));
  HOPU_CUDA(c, cudaMalloc(&c->d_s2, ts * nstate));
  HOPU_CUDA(c, cudaMalloc((void**)&c->d_diss, sizeof(double) * NF));
  HOPU_CUDA(c, cudaMalloc((void**)&c->d_red, sizeof(double) * (c->red_blocks + 8)));
  HOPU_CUDA(c, cudaMalloc((void**)&c->d_err, sizeof(int)));
  HOPU_CUDA(c, cudaMemset(c->d_err, 0, sizeof(int)));
  c->dm.err = c->d_err;
  // position, ticket, then the per-block partials of the energy-log kernel
  const size_t elog_bytes = sizeof(int64_t) * (2 + elog_blocks(c->topo.n_elems, c->nsm));
  HOPU_CUDA(c, cudaMalloc((void**)&c->d_elog_pos, elog_bytes));
  HOPU_CUDA(c, cudaMemset(c->d_elog_pos, 0, elog_bytes));
  ce = c->ops->configure(c->dt);
  if (ce != cudaSuccess) return cuda_fail(c, ce, "kernel configuration");
  return autotune(c, opts->tile_hint);
}
}  // namespace

extern "C" {

hopu_status hopu_create(const hopu_mesh_desc* mesh, const hopu_options* opts, void* cuda_stream, hopu_ctx** out) {
  if (!out) return HOPU_EINVAL;
  *out = nullptr;
  hopu_ctx* c = nullptr;
  hopu_status r = create_impl(mesh, opts, cuda_stream, &c);
  if (r != HOPU_OK) {
    g_create_error = c ? c->err : std::string("invalid arguments");
    if (c) hopu_destroy(c);
    return r;
  }
  g_create_error.clear();
  *out = c;
  return HOPU_OK;
}

hopu_status hopu_destroy(hopu_ctx* c) {
  if (!c) return HOPU_OK;
  free_all(c);
  delete c;
  return HOPU_OK;
}

hopu_status hopu_set_stream(hopu_ctx* c, void* cuda_stream) {
  HOPU_PRECHECK(c);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return HOPU_OK;
}

hopu_status hopu_tuning(const hopu_ctx* c, int* out2) {
  if (!c || !out2) return HOPU_EINVAL;
  out2[0] = c->ops ? c->ops->selected_v2l() : 0;
  out2[1] = c->ops ? c->ops->selected_volume() : 0;
  return HOPU_OK;
}

hopu_status hopu_set_volume_variant(hopu_ctx* c, int variant) {
  HOPU_PRECHECK(c);
  if (variant < 0 || variant >= kVolVariants || !c->ops->volume_variant_ok(variant))
    return fail(c, HOPU_EINVAL, "set_volume_variant: not available for this order and precision");
  c->ops->select_volume_variant(variant);
  if (c->gexec) {  // the captured substep uses the previous variant
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return HOPU_OK;
}

hopu_status hopu_tuning_l2v(const hopu_ctx* c, int* tc, double* ms2) {
  if (!c || !tc) return HOPU_EINVAL;
  *tc = c->ops ? c->ops->selected_l2v() : 0;
  if (ms2) {
    ms2[0] = c->l2v_ms[0];
    ms2[1] = c->l2v_ms[1];
  }
  return HOPU_OK;
}

hopu_status hopu_set_l2v_variant(hopu_ctx* c, int tc) {
  HOPU_PRECHECK(c);
  if (tc != 0 && tc != 1) return fail(c, HOPU_EINVAL, "set_l2v_variant: 0 (FMA) or 1 (tensor cores)");
  if (tc == 1 && !c->ops->tensor_core_l2v())
    return fail(c, HOPU_EINVAL, "set_l2v_variant: no tensor-core back-projection for this order and precision");
  c->ops->select_l2v(tc);
  if (c->gexec) {  // the captured substep uses the previous variant
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return HOPU_OK;
}

hopu_status hopu_tuning_volume(const hopu_ctx* c, int* variant, double* ms6) {
  if (!c || !variant) return HOPU_EINVAL;
  *variant = c->ops ? c->ops->volume_variant() : -1;
  if (ms6)
    for (int v = 0; v < kVolVariants; ++v) ms6[v] = c->vol_ms[v];
  return HOPU_OK;
}

hopu_status hopu_sync(hopu_ctx* c) {
  HOPU_PRECHECK(c);
  HOPU_CUDA(c, cudaStreamSynchronize(c->stream));
  return device_status(c);
}

hopu_status hopu_set_wait_limit(hopu_ctx* c, int64_t polls) {
  HOPU_PRECHECK(c);
  if (polls > (int64_t)UINT32_MAX) return fail(c, HOPU_EINVAL, "set_wait_limit: more than 2^32 - 1 polls");
  c->dm.tc_wait_limit = polls < 0 ? (1u << 22) : (uint32_t)polls;
  if (c->gexec) {  // the captured substep holds the old limit in its kernel parameters
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return HOPU_OK;
}

hopu_status hopu_sizes(const hopu_ctx* c, int64_t* n_hdiv, int64_t* n_l2, int64_t* n_facets) {
  if (!c) return HOPU_EINVAL;
  if (n_hdiv) *n_hdiv = c->n_hdiv;
  if (n_l2) *n_l2 = c->n_l2;
  if (n_facets) *n_facets = c->topo.n_facets;
  return HOPU_OK;
}

hopu_status hopu_project(hopu_ctx* c, int dir, const void* in, void* out) {
  HOPU_PRECHECK(c);
  if (!in || !out || in == out) return fail(c, HOPU_EINVAL, "project: NULL or aliased vectors");
  if (!aligned16(in) || !aligned16(out)) return fail(c, HOPU_EINVAL, "project: vectors must be 16-byte aligned");
  if (dir == HOPU_HDIV_TO_L2) {
    enqueue_v2l(c, in, out);
  } else if (dir == HOPU_L2_TO_HDIV || dir == HOPU_L2_TO_HDIV_DUAL) {
    Combine plain;
    enqueue_l2v(c, in, dir == HOPU_L2_TO_HDIV_DUAL, plain, out);
  } else {
    return fail(c, HOPU_EINVAL, "project: unknown direction");
  }
  return check_launch(c, "project kernels");
}

hopu_status hopu_apply_convection(hopu_ctx* c, const void* w_hdiv, const void* u_l2, void* y_l2,
                                  const int8_t* facet_l) {
  HOPU_PRECHECK(c);
  if (!w_hdiv || !u_l2 || !y_l2 || y_l2 == u_l2) return fail(c, HOPU_EINVAL, "apply_convection: NULL or aliased vectors");
  if (!aligned16(w_hdiv) || !aligned16(u_l2) || !aligned16(y_l2))
    return fail(c, HOPU_EINVAL, "apply_convection: vectors must be 16-byte aligned");
  enqueue_v2l(c, w_hdiv, c->d_wL);
  Combine plain;
  return enqueue_stage_apply(c, u_l2, c->d_wL, c->l, facet_l ? facet_l : c->facet_l, nullptr, plain, y_l2);
}

hopu_status hopu_apply_convection_l2(hopu_ctx* c, const void* w_l2, const void* u_l2, void* y_l2,
                                     const int8_t* facet_l) {
  HOPU_PRECHECK(c);
  if (!w_l2 || !u_l2 || !y_l2 || y_l2 == u_l2 || y_l2 == w_l2)
    return fail(c, HOPU_EINVAL, "apply_convection_l2: NULL or aliased vectors");
  if (!aligned16(w_l2) || !aligned16(u_l2) || !aligned16(y_l2))
    return fail(c, HOPU_EINVAL, "apply_convection_l2: vectors must be 16-byte aligned");
  Combine plain;
  return enqueue_stage_apply(c, u_l2, w_l2, c->l, facet_l ? facet_l : c->facet_l, nullptr, plain, y_l2);
}

hopu_status hopu_pack_elements(hopu_ctx* c, const int32_t* ids, int64_t n, const void* l2, void* buf) {
  HOPU_PRECHECK(c);
  if (n < 0 || (n > 0 && (!ids || !l2 || !buf))) return fail(c, HOPU_EINVAL, "pack_elements: bad arguments");
  if (n == 0) return HOPU_OK;
  const int g = (int)std::min<int64_t>((n * c->ref.nloc + 255) / 256, (int64_t)c->nsm * 8);
  if (c->fp64)
    k_copy_blocks<double, true><<<g, 256, 0, c->stream>>>(c->topo.n_elems, c->ref.nloc, ids, n, (const double*)l2,
                                                          (double*)buf, c->d_err);
  else
    k_copy_blocks<float, true><<<g, 256, 0, c->stream>>>(c->topo.n_elems, c->ref.nloc, ids, n, (const float*)l2,
                                                         (float*)buf, c->d_err);
  return check_launch(c, "pack_elements");
}

hopu_status hopu_unpack_elements(hopu_ctx* c, const int32_t* ids, int64_t n, const void* buf, void* l2) {
  HOPU_PRECHECK(c);
  if (n < 0 || (n > 0 && (!ids || !l2 || !buf))) return fail(c, HOPU_EINVAL, "unpack_elements: bad arguments");
  if (n == 0) return HOPU_OK;
  const int g = (int)std::min<int64_t>((n * c->ref.nloc + 255) / 256, (int64_t)c->nsm * 8);
  if (c->fp64)
    k_copy_blocks<double, false><<<g, 256, 0, c->stream>>>(c->topo.n_elems, c->ref.nloc, ids, n, (const double*)buf,
                                                           (double*)l2, c->d_err);
  else
    k_copy_blocks<float, false><<<g, 256, 0, c->stream>>>(c->topo.n_elems, c->ref.nloc, ids, n, (const float*)buf,
                                                          (float*)l2, c->d_err);
  return check_launch(c, "unpack_elements");
}

hopu_status hopu_set_frozen_wind(hopu_ctx* c, const void* w_hdiv) {
  HOPU_PRECHECK(c);
  if (!w_hdiv || !aligned16(w_hdiv)) return fail(c, HOPU_EINVAL, "set_frozen_wind: NULL or unaligned wind");
  enqueue_v2l(c, w_hdiv, c->d_wfz);
  c->have_frozen = true;
  return check_launch(c, "set_frozen_wind");
}

hopu_status hopu_rk_substep(hopu_ctx* c, void* state, double dt, int n_substeps) {
  HOPU_PRECHECK(c);
  if (!state || n_substeps < 0 || !std::isfinite(dt)) return fail(c, HOPU_EINVAL, "rk_substep: bad arguments");
  if (!aligned16(state)) return fail(c, HOPU_EINVAL, "rk_substep: state must be 16-byte aligned");
  if (c->wind == HOPU_WIND_FROZEN && !c->have_frozen) return fail(c, HOPU_EINVAL, "rk_substep: FROZEN wind not set");
  if (n_substeps == 0) return HOPU_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HOPU_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
  const bool can_graph = (c->stream != nullptr) && cs == cudaStreamCaptureStatusNone;
  if (!can_graph) {
    for (int s = 0; s < n_substeps; ++s) {
      hopu_status r = enqueue_substep(c, state, dt);
      if (r != HOPU_OK) return r;
    }
    return HOPU_OK;
  }
  if (!c->gexec || c->g_state != state || c->g_dt != dt || c->g_wind != c->wind) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    HOPU_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->prof_graph.clear();
    hopu_status r = enqueue_substep(c, state, dt);
    c->capturing = false;
    cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
    if (r != HOPU_OK) return r;
    if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      c->gexec = nullptr;
      return cuda_fail(c, ie, "cudaGraphInstantiate");
    }
    c->g_state = state;
    c->g_dt = dt;
    c->g_wind = c->wind;
  }
  for (int s = 0; s < n_substeps; ++s) HOPU_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
  c->graph_replayed = true;
  return HOPU_OK;
}

hopu_status hopu_energy(hopu_ctx* c, const void* w_hdiv, const void* u_l2, double* host_out) {
  HOPU_PRECHECK(c);
  if (!u_l2 || !host_out) return fail(c, HOPU_EINVAL, "energy: NULL pointer");
  if (!aligned16(u_l2) || (w_hdiv && !aligned16(w_hdiv))) return fail(c, HOPU_EINVAL, "energy: vectors must be 16-byte aligned");
  hopu_status r = weighted_dot(c, u_l2, u_l2, 0);
  if (r != HOPU_OK) return r;
  double vals[3] = {0.0, 0.0, 0.0};
  if (w_hdiv) {
    enqueue_v2l(c, w_hdiv, c->d_wL);
    Combine plain;
    r = enqueue_stage_apply(c, u_l2, c->d_wL, c->l, c->facet_l, c->d_diss, plain, c->d_yL);
    if (r != HOPU_OK) return r;
    // c(w;u,u) = sum_T |det J| u . y  (y = M^{-1} r, M = |det J| I)
    r = weighted_dot(c, u_l2, c->d_yL, 1);
    if (r != HOPU_OK) return r;
    k_sum<<<1, kRedThreads, 0, c->stream>>>(c->d_diss, c->topo.n_facets, c->d_red + c->red_blocks + 2);
    r = check_launch(c, "dissipation sum");
    if (r != HOPU_OK) return r;
  }
  HOPU_CUDA(c, cudaMemcpyAsync(vals, c->d_red + c->red_blocks, sizeof(double) * (w_hdiv ? 3 : 1),
                               cudaMemcpyDeviceToHost, c->stream));
  HOPU_CUDA(c, cudaStreamSynchronize(c->stream));
  r = device_status(c);
  if (r != HOPU_OK) return r;
  host_out[0] = 0.5 * vals[0];
  host_out[1] = w_hdiv ? vals[1] : 0.0;
  host_out[2] = w_hdiv ? vals[2] : 0.0;
  return HOPU_OK;
}

hopu_status hopu_vjp_apply(hopu_ctx* c, const void* w_hdiv, const void* u_l2, const void* ybar_l2, void* wbar_hdiv,
                           void* ubar_l2) {
  HOPU_PRECHECK(c);
  if (!w_hdiv || !u_l2 || !ybar_l2 || (!wbar_hdiv && !ubar_l2))
    return fail(c, HOPU_EINVAL, "vjp_apply: NULL input or no output");
  const void* ins[3] = {w_hdiv, u_l2, ybar_l2};
  for (const void* p : ins)
    if (p == wbar_hdiv || p == ubar_l2) return fail(c, HOPU_EINVAL, "vjp_apply: an output aliases an input");
  if (wbar_hdiv && wbar_hdiv == ubar_l2) return fail(c, HOPU_EINVAL, "vjp_apply: aliased outputs");
  if (!aligned16(w_hdiv) || !aligned16(u_l2) || !aligned16(ybar_l2) || (wbar_hdiv && !aligned16(wbar_hdiv)) ||
      (ubar_l2 && !aligned16(ubar_l2)))
    return fail(c, HOPU_EINVAL, "vjp_apply: vectors must be 16-byte aligned");
  if (!c->topo.boundary.empty()) return fail(c, HOPU_ENOTSUP, "vjp_apply: meshes with boundary facets");
  hopu_status r = ensure_gamW(c);
  if (r != HOPU_OK) return r;
  enqueue_v2l(c, w_hdiv, c->d_wL);
  enqueue_apply_vjp(c, u_l2, c->d_wL, ybar_l2, ubar_l2 ? ubar_l2 : c->d_uL, c->d_yL);
  if (wbar_hdiv) {
    Combine plain;
    enqueue_l2v(c, c->d_yL, true, plain, wbar_hdiv);
  }
  return check_launch(c, "vjp_apply kernels");
}

hopu_status hopu_vjp_rollout(hopu_ctx* c, const void* u0_hdiv, double dt, int n_substeps, int ckpt_every,
                             void* u0bar_hdiv, double* loss) {
  HOPU_PRECHECK(c);
  if (!u0_hdiv || !u0bar_hdiv || u0_hdiv == u0bar_hdiv || n_substeps < 0 || ckpt_every < 1 || !std::isfinite(dt))
    return fail(c, HOPU_EINVAL, "vjp_rollout: bad arguments");
  if (!aligned16(u0_hdiv) || !aligned16(u0bar_hdiv))
    return fail(c, HOPU_EINVAL, "vjp_rollout: vectors must be 16-byte aligned");
  if (c->wind != HOPU_WIND_STAGE) return fail(c, HOPU_ENOTSUP, "vjp_rollout: only the STAGE wind rule");
  if (!c->topo.boundary.empty()) return fail(c, HOPU_ENOTSUP, "vjp_rollout: meshes with boundary facets");
  hopu_status r = ensure_gamW(c);
  if (r != HOPU_OK) return r;
  const int n = n_substeps;
  const int C = n > 0 ? std::min(ckpt_every, n) : 1;
  const int nseg = n > 0 ? (n + C - 1) / C : 0;
  // one slot per V_h vector, 256-byte aligned: checkpoints, 3C stage states, work, b2, b1
  const size_t slot = (c->n_hdiv * c->tsize + 255) / 256 * 256;
  const size_t need = slot * ((size_t)std::max(nseg - 1, 0) + 3 * (size_t)C + 3);
  if (need > c->adj_bytes) {
    if (c->d_adj) {
      HOPU_CUDA(c, cudaStreamSynchronize(c->stream));
      cudaFree(c->d_adj);
      c->d_adj = nullptr;
      c->adj_bytes = 0;
    }
    HOPU_CUDA(c, cudaMalloc(&c->d_adj, need));
    c->adj_bytes = need;
  }
  unsigned char* base = static_cast<unsigned char*>(c->d_adj);
  void* work = base;
  void* b2 = base + slot;
  void* b1 = base + 2 * slot;
  unsigned char* seg = base + 3 * slot;
  unsigned char* ckpt = seg + 3 * (size_t)C * slot;
  const size_t vbytes = c->n_hdiv * c->tsize;
  double* elog = c->elog;  // no energy logging inside the rollout
  c->elog = nullptr;
  auto body = [&]() -> hopu_status {
    HOPU_CUDA(c, cudaMemcpyAsync(work, u0_hdiv, vbytes, cudaMemcpyDeviceToDevice, c->stream));
    // forward: checkpoints at segment starts, stage states of the last segment
    for (int g = 0; g < nseg; ++g) {
      const int cnt = std::min(C, n - g * C);
      if (g < nseg - 1) {
        HOPU_CUDA(c, cudaMemcpyAsync(ckpt + (size_t)g * slot, work, vbytes, cudaMemcpyDeviceToDevice, c->stream));
        for (int j = 0; j < cnt; ++j) {
          hopu_status q = enqueue_substep(c, work, dt);
          if (q != HOPU_OK) return q;
        }
      } else {
        hopu_status q = stored_substeps(c, work, dt, cnt, seg, slot);
        if (q != HOPU_OK) return q;
      }
    }
    // seed: the cotangent of u_N, or the gradient E^T M E u_N of 1/2 int |E u_N|^2
    if (loss) {
      enqueue_v2l(c, work, c->d_uL);
      hopu_status q = weighted_dot(c, c->d_uL, c->d_uL, 3);
      if (q != HOPU_OK) return q;
      enqueue_mass(c, c->d_uL, c->d_yL);
      Combine plain;
      enqueue_l2v(c, c->d_yL, true, plain, u0bar_hdiv);
    }
    // backward over the segments, recomputing the stage states from the checkpoints
    for (int g = nseg - 1; g >= 0; --g) {
      const int cnt = std::min(C, n - g * C);
      if (g < nseg - 1) {
        HOPU_CUDA(c, cudaMemcpyAsync(work, ckpt + (size_t)g * slot, vbytes, cudaMemcpyDeviceToDevice, c->stream));
        hopu_status q = stored_substeps(c, work, dt, cnt, seg, slot);
        if (q != HOPU_OK) return q;
      }
      for (int j = cnt - 1; j >= 0; --j) {
        const unsigned char* st = seg + 3 * (size_t)j * slot;
        void* ub = u0bar_hdiv;
        // b2 = 2/3 (ub - dt J(u2)^T ub); b1 = 1/4 (b2 - dt J(u1)^T b2);
        // ub = 1/3 ub + 3/4 b2 + b1 - dt J(u)^T b1
        hopu_status q = enqueue_rhs_vjp(c, st + 2 * slot, ub, Combine{2.0 / 3.0, ub, 0.0, nullptr, -2.0 / 3.0 * dt}, b2);
        if (q == HOPU_OK) q = enqueue_rhs_vjp(c, st + slot, b2, Combine{0.25, b2, 0.0, nullptr, -0.25 * dt}, b1);
        if (q != HOPU_OK) return q;
        enqueue_axpby(c, c->n_hdiv, 1.0 / 3.0, ub, 0.75, b2);
        q = enqueue_rhs_vjp(c, st, b1, Combine{1.0, ub, 1.0, b1, -dt}, ub);
        if (q != HOPU_OK) return q;
      }
    }
    if (loss) {
      double v = 0.0;
      HOPU_CUDA(c, cudaMemcpyAsync(&v, c->d_red + c->red_blocks + 3, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      HOPU_CUDA(c, cudaStreamSynchronize(c->stream));
      *loss = 0.5 * v;
    }
    return check_launch(c, "vjp_rollout kernels");
  };
  r = body();
  c->elog = elog;
  return r;
}

hopu_status hopu_boundary_facets(const hopu_ctx* c, int64_t* out, int64_t* count) {
  if (!c) return HOPU_EINVAL;
  if (count) *count = (int64_t)c->topo.boundary.size();
  if (out) std::copy(c->topo.boundary.begin(), c->topo.boundary.end(), out);
  return HOPU_OK;
}

hopu_status hopu_set_inlet(hopu_ctx* c, const int64_t* facets, int64_t n, const double* values) {
  HOPU_PRECHECK(c);
  if (n < 0 || (n > 0 && (!facets || !values))) return fail(c, HOPU_EINVAL, "set_inlet: bad arguments");
  const RefTables& R = c->ref;
  const int d = c->dim, nf = R.nf, nqf = R.nqf;
  const int64_t NF = c->topo.n_facets;
  std::vector<int32_t> row((size_t)NF, -1);
  std::vector<double> modes((size_t)n * nf * d, 0.0);
  for (int64_t r = 0; r < n; ++r) {
    const int64_t F = facets[r];
    if (F < 0 || F >= NF || !std::binary_search(c->topo.boundary.begin(), c->topo.boundary.end(), F))
      return fail(c, HOPU_EINVAL, "set_inlet: facet " + std::to_string(F) + " is not a boundary facet");
    if (row[(size_t)F] >= 0) return fail(c, HOPU_EINVAL, "set_inlet: facet listed twice");
    row[(size_t)F] = (int32_t)r;
    // modal exterior trace: the facet-rule moments against the orthonormal facet basis
    for (int m = 0; m < nf; ++m)
      for (int a = 0; a < d; ++a) {
        double acc = 0.0;
        for (int q = 0; q < nqf; ++q)
          acc += R.wf[q] * R.psi[(size_t)q * nf + m] * values[((size_t)r * nqf + q) * d + a];
        modes[((size_t)r * nf + m) * d + a] = acc;
      }
  }
  HOPU_CUDA(c, cudaStreamSynchronize(c->stream));  // kernels in flight may read the old data
  if (c->d_inlet) cudaFree(c->d_inlet);
  if (c->d_inlet_modes) cudaFree(c->d_inlet_modes);
  c->d_inlet = nullptr;
  c->d_inlet_modes = nullptr;
  c->dm.inlet = nullptr;
  c->dm.inlet_modes = nullptr;
  c->n_inlet = n;
  if (c->gexec) {  // the cached substep graph holds the old mesh view
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  if (n == 0) return HOPU_OK;
  std::vector<unsigned char> hm(c->tsize * modes.size());
  if (c->fp64) convert<double>(modes, hm, 0);
  else convert<float>(modes, hm, 0);
  HOPU_CUDA(c, cudaMalloc((void**)&c->d_inlet, sizeof(int32_t) * NF));
  HOPU_CUDA(c, cudaMemcpy(c->d_inlet, row.data(), sizeof(int32_t) * NF, cudaMemcpyHostToDevice));
  HOPU_CUDA(c, cudaMalloc(&c->d_inlet_modes, hm.size()));
  HOPU_CUDA(c, cudaMemcpy(c->d_inlet_modes, hm.data(), hm.size(), cudaMemcpyHostToDevice));
  c->dm.inlet = c->d_inlet;
  c->dm.inlet_modes = c->d_inlet_modes;
  return HOPU_OK;
}

hopu_status hopu_set_facet_l(hopu_ctx* c, const int8_t* facet_l) {
  HOPU_PRECHECK(c);
  if (c->facet_l != facet_l && c->gexec) {  // the cached substep graph holds the old pointer
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->facet_l = facet_l;
  return HOPU_OK;
}

hopu_status hopu_adapt_l(hopu_ctx* c, const void* u_l2, const double* thresholds, int8_t* facet_l,
                         double* eta_out) {
  HOPU_PRECHECK(c);
  if (!u_l2 || !thresholds || !facet_l) return fail(c, HOPU_EINVAL, "adapt_l: NULL pointer");
  if (!aligned16(u_l2)) return fail(c, HOPU_EINVAL, "adapt_l: u must be 16-byte aligned");
  hopu::EtaThresholds th{};
  for (int i = 0; i <= c->k; ++i) {
    th.t[i] = thresholds[i];
    if (!(thresholds[i] > (i ? thresholds[i - 1] : 0.0)) || !(thresholds[i] < 1.0))
      return fail(c, HOPU_EINVAL, "adapt_l: need k+1 increasing thresholds in (0, 1)");
  }
  c->ops->eta(c->dm, c->dt, u_l2, c->l, facet_l, th, eta_out, c->stream);
  return check_launch(c, "adapt_l kernel");
}

hopu_status hopu_points(hopu_ctx* c, int which, double* host_out, int64_t* count_out) {
  HOPU_PRECHECK(c);
  if (which != 0 && which != 1) return fail(c, HOPU_EINVAL, "points: which must be 0 or 1");
  const int64_t cnt = which == 0 ? c->topo.n_facets * c->ref.nqf : c->topo.n_elems * c->ref.nq;
  if (count_out) *count_out = cnt;
  if (!host_out) return HOPU_OK;
  if (which == 0) facet_points(c->topo, c->ref.sq, c->ref.nqf, host_out);
  else volume_points(c->topo, c->ref.xq, c->ref.nq, host_out);
  return HOPU_OK;
}

hopu_status hopu_interpolate(hopu_ctx* c, const double* fvals, const double* vvals, void* u_hdiv) {
  HOPU_PRECHECK(c);
  if (!fvals || !vvals || !u_hdiv) return fail(c, HOPU_EINVAL, "interpolate: NULL pointer");
  if (!aligned16(u_hdiv)) return fail(c, HOPU_EINVAL, "interpolate: output must be 16-byte aligned");
  const RefTables& R = c->ref;
  const int d = c->dim, G = geo_stride(d);
  const int64_t NF = c->topo.n_facets, E = c->topo.n_elems;
  std::vector<double> h((size_t)c->n_hdiv, 0.0);
  for (int64_t F = 0; F < NF; ++F) {
    const double* n = &c->topo.fgeo[(size_t)F * (d + 1)];
    const double aF = n[d];
    for (int m = 0; m < R.nf; ++m) {
      double acc = 0.0;
      for (int q = 0; q < R.nqf; ++q) {
        double un = 0.0;
        for (int a = 0; a < d; ++a) un += fvals[((size_t)F * R.nqf + q) * d + a] * n[a];
        acc += R.wf[q] * un * R.psi[(size_t)q * R.nf + m];
      }
      h[(size_t)F * R.nf + m] = aF * acc;
    }
  }
  std::vector<double> uhat((size_t)R.nq * d);
  for (int64_t e = 0; e < E; ++e) {
    const double* g = &c->topo.geo[(size_t)e * G];
    const double det = g[2 * d * d];
    for (int q = 0; q < R.nq; ++q)
      for (int b = 0; b < d; ++b) {
        double acc = 0.0;
        for (int a = 0; a < d; ++a) acc += g[d * d + b * d + a] * vvals[((size_t)e * R.nq + q) * d + a];
        uhat[(size_t)q * d + b] = det * acc;
      }
    for (int j = 0; j < R.nint; ++j) {
      double acc = 0.0;
      for (int q = 0; q < R.nq; ++q)
        for (int b = 0; b < d; ++b) acc += R.wq[q] * uhat[(size_t)q * d + b] * R.z[((size_t)j * R.nq + q) * d + b];
      h[(size_t)NF * R.nf + (size_t)e * R.nint + j] = acc;
    }
  }
  std::vector<unsigned char> buf(c->tsize * h.size());
  if (c->fp64) convert<double>(h, buf, 0);
  else convert<float>(h, buf, 0);
  HOPU_CUDA(c, cudaMemcpyAsync(u_hdiv, buf.data(), buf.size(), cudaMemcpyHostToDevice, c->stream));
  HOPU_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOPU_OK;
}

hopu_status hopu_set_energy_log(hopu_ctx* c, double* dev_log, int64_t capacity) {
  HOPU_PRECHECK(c);
  if ((dev_log == nullptr) != (capacity == 0) || capacity < 0)
    return fail(c, HOPU_EINVAL, "set_energy_log: log and capacity must be both set or both empty");
  if (c->gexec) {  // the captured substep changes
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->elog = dev_log;
  c->elog_cap = capacity;
  HOPU_CUDA(c, cudaMemsetAsync(c->d_elog_pos, 0, sizeof(int64_t), c->stream));
  return HOPU_OK;
}

hopu_status hopu_profile(hopu_ctx* c, int enable) {
  HOPU_PRECHECK(c);
  if (enable && c->ev.empty()) {
    c->ev.resize(4 * kProfPairs, nullptr);
    for (auto& e : c->ev) HOPU_CUDA(c, cudaEventCreate(&e));
  }
  if ((enable != 0) != c->prof_on && c->gexec) {  // the cached graph must be re-captured
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->prof_on = enable != 0;
  c->prof_graph.clear();
  c->prof_direct.clear();
  c->graph_replayed = false;
  return HOPU_OK;
}

hopu_status hopu_profile_read(hopu_ctx* c, double* ms, int64_t* launches) {
  HOPU_PRECHECK(c);
  if (!ms || !launches) return fail(c, HOPU_EINVAL, "profile_read: NULL pointer");
  if (!c->prof_on) return HOPU_OK;
  HOPU_CUDA(c, cudaStreamSynchronize(c->stream));
  auto add = [&](const std::vector<std::pair<int, int>>& lst) -> hopu_status {
    for (const auto& pf : lst) {
      float t = 0.f;
      HOPU_CUDA(c, cudaEventElapsedTime(&t, c->ev[2 * pf.first], c->ev[2 * pf.first + 1]));
      ms[pf.second] += t;
      launches[pf.second] += 1;
    }
    return HOPU_OK;
  };
  if (c->graph_replayed) {
    hopu_status r = add(c->prof_graph);
    if (r != HOPU_OK) return r;
  }
  hopu_status r = add(c->prof_direct);
  if (r != HOPU_OK) return r;
  c->prof_direct.clear();
  c->graph_replayed = false;
  return HOPU_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches
struct hopu_batch {
  int dim = 0;
  cudaStream_t stream = nullptr;
  std::vector<hopu_ctx*> cls;          // one merged context per order class
  std::vector<int> cls_k;
  std::vector<std::array<int64_t, 7>> layout;  // per mesh
  cudaGraphExec_t gexec = nullptr;
  std::vector<void*> g_states;
  double g_dt = 0.0;
  std::string err;
};

namespace {
hopu_status batch_fail(hopu_batch* b, int code, const std::string& msg) {
  if (b && b->err.empty()) b->err = msg;
  return (hopu_status)code;
}
}  // namespace

extern "C" {

hopu_status hopu_batch_destroy(hopu_batch* b) {
  if (!b) return HOPU_OK;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (hopu_ctx* c : b->cls) hopu_destroy(c);
  delete b;
  return HOPU_OK;
}

hopu_status hopu_batch_create(const hopu_mesh_desc* meshes, const int* k, int n, const hopu_options* opts,
                              void* cuda_stream, hopu_batch** out) {
  if (!out) return HOPU_EINVAL;
  *out = nullptr;
  if (!meshes || !k || n <= 0 || !opts) return HOPU_EINVAL;
  const int dim = meshes[0].dim;
  for (int i = 0; i < n; ++i) {
    if (meshes[i].dim != dim || !meshes[i].coords || !meshes[i].elem_vertices) return HOPU_EINVAL;
    if (k[i] < 1 || k[i] > (dim == 2 ? 4 : 5)) return HOPU_ENOTSUP;
  }
  hopu_batch* b = new (std::nothrow) hopu_batch();
  if (!b) return HOPU_ENOMEM;
  b->dim = dim;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->layout.assign(n, {0, 0, 0, 0, 0, 0, 0});
  std::vector<int> ks(k, k + n);
  std::sort(ks.begin(), ks.end());
  ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
  for (int kk : ks) {
    // disjoint union of the meshes of order kk: vertex and representative ids offset
    std::vector<int> members;
    for (int i = 0; i < n; ++i)
      if (k[i] == kk) members.push_back(i);
    int64_t nv = 0, ne = 0;
    for (int i : members) {
      nv += meshes[i].n_vertices;
      ne += meshes[i].n_elems;
    }
    std::vector<double> coords((size_t)nv * dim);
    std::vector<int64_t> ev((size_t)ne * (dim + 1)), rep((size_t)nv);
    int64_t vo = 0, eo = 0;
    std::vector<int64_t> elem_start;
    for (int i : members) {
      const hopu_mesh_desc& m = meshes[i];
      std::memcpy(&coords[(size_t)vo * dim], m.coords, sizeof(double) * m.n_vertices * dim);
      for (int64_t v = 0; v < m.n_vertices; ++v) rep[vo + v] = vo + (m.vertex_rep ? m.vertex_rep[v] : v);
      for (int64_t t = 0; t < m.n_elems * (dim + 1); ++t) ev[(size_t)eo * (dim + 1) + t] = vo + m.elem_vertices[t];
      elem_start.push_back(eo);
      vo += m.n_vertices;
      eo += m.n_elems;
    }
    elem_start.push_back(eo);
    hopu_mesh_desc md{dim, nv, coords.data(), ne, ev.data(), rep.data()};
    hopu_options o = *opts;
    o.k = kk;
    o.l = opts->l < -1 ? std::max(-1, kk + 1 + opts->l) : std::min(opts->l, kk);
    hopu_ctx* c = nullptr;
    hopu_status r = hopu_create(&md, &o, cuda_stream, &c);
    if (r != HOPU_OK) {
      const std::string msg = std::string("batch class k=") + std::to_string(kk) + ": " + g_create_error;
      hopu_batch_destroy(b);
      g_create_error = msg;
      return r;
    }
    const int cidx = (int)b->cls.size();
    b->cls.push_back(c);
    b->cls_k.push_back(kk);
    // per-mesh ranges: facets of a mesh are contiguous (sorted by offset representative ids)
    const int64_t NF = c->topo.n_facets;
    std::vector<int64_t> fcount(members.size(), 0);
    std::vector<int64_t> fmin(members.size(), INT64_MAX);
    for (int64_t F = 0; F < NF; ++F) {
      const int64_t e = c->topo.fa[F] >> 2;
      const size_t mi = std::upper_bound(elem_start.begin(), elem_start.end(), e) - elem_start.begin() - 1;
      fcount[mi] += 1;
      fmin[mi] = std::min(fmin[mi], F);
    }
    for (size_t j = 0; j < members.size(); ++j) {
      const int64_t e0 = elem_start[j], e1 = elem_start[j + 1];
      b->layout[members[j]] = {cidx, fmin[j] * c->ref.nf, fcount[j] * c->ref.nf,
                               NF * c->ref.nf + e0 * c->ref.nint, (e1 - e0) * c->ref.nint,
                               e0 * c->ref.nloc, (e1 - e0) * c->ref.nloc};
    }
  }
  *out = b;
  return HOPU_OK;
}

hopu_status hopu_batch_classes(const hopu_batch* b, int* n_classes, int* class_k, int64_t* class_n_hdiv,
                               int64_t* class_n_l2) {
  if (!b) return HOPU_EINVAL;
  if (n_classes) *n_classes = (int)b->cls.size();
  for (size_t c = 0; c < b->cls.size(); ++c) {
    if (class_k) class_k[c] = b->cls_k[c];
    if (class_n_hdiv) class_n_hdiv[c] = b->cls[c]->n_hdiv;
    if (class_n_l2) class_n_l2[c] = b->cls[c]->n_l2;
  }
  return HOPU_OK;
}

hopu_status hopu_batch_context(hopu_batch* b, int c, hopu_ctx** ctx) {
  if (!b || !ctx || c < 0 || c >= (int)b->cls.size()) return HOPU_EINVAL;
  *ctx = b->cls[c];
  return HOPU_OK;
}

hopu_status hopu_batch_layout(const hopu_batch* b, int mesh, int64_t* out7) {
  if (!b || !out7 || mesh < 0 || mesh >= (int)b->layout.size()) return HOPU_EINVAL;
  for (int i = 0; i < 7; ++i) out7[i] = b->layout[mesh][i];
  return HOPU_OK;
}

hopu_status hopu_batch_rk_substep(hopu_batch* b, void* const* states, double dt, int n_substeps) {
  if (!b || !states || n_substeps < 0 || !std::isfinite(dt)) return HOPU_EINVAL;
  for (size_t c = 0; c < b->cls.size(); ++c) {
    if (!states[c] || !aligned16(states[c])) return batch_fail(b, HOPU_EINVAL, "batch_rk_substep: bad state pointer");
    if (b->cls[c]->status != HOPU_OK) return (hopu_status)b->cls[c]->status;
    b->cls[c]->stream = b->stream;
  }
  if (n_substeps == 0) return HOPU_OK;
  if (b->stream == nullptr) {  // legacy default stream cannot be captured
    for (int s = 0; s < n_substeps; ++s)
      for (size_t c = 0; c < b->cls.size(); ++c) {
        hopu_status r = enqueue_substep(b->cls[c], states[c], dt);
        if (r != HOPU_OK) return r;
      }
    return HOPU_OK;
  }
  std::vector<void*> key(states, states + b->cls.size());
  if (!b->gexec || b->g_states != key || b->g_dt != dt) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, HOPU_ECUDA, cudaGetErrorString(e));
    hopu_status r = HOPU_OK;
    for (size_t c = 0; c < b->cls.size() && r == HOPU_OK; ++c) r = enqueue_substep(b->cls[c], states[c], dt);
    e = cudaStreamEndCapture(b->stream, &graph);
    if (r != HOPU_OK) return r;
    if (e != cudaSuccess) return batch_fail(b, HOPU_ECUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->gexec = nullptr;
      return batch_fail(b, HOPU_ECUDA, cudaGetErrorString(e));
    }
    b->g_states = key;
    b->g_dt = dt;
  }
  for (int s = 0; s < n_substeps; ++s) {
    cudaError_t e = cudaGraphLaunch(b->gexec, b->stream);
    if (e != cudaSuccess) return batch_fail(b, HOPU_ECUDA, cudaGetErrorString(e));
  }
  return HOPU_OK;
}

const char* hopu_batch_last_error(const hopu_batch* b) {
  if (!b) return g_create_error.c_str();
  if (!b->err.empty()) return b->err.c_str();
  for (const hopu_ctx* c : b->cls)
    if (c->status != HOPU_OK) return c->err.c_str();
  return "";
}

const char* hopu_last_error(const hopu_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

hopu_status hopu_clear_error(hopu_ctx* c) {
  if (!c) return HOPU_EINVAL;
  c->status = HOPU_OK;
  c->err.clear();
  return HOPU_OK;
}

hopu_status hopu_selftest(int dim, int k, double* report) {
  if (!report) return HOPU_EINVAL;
  std::string err;
  if (!selftest_ref_tables(dim, k, report, err)) return HOPU_EINVAL;
  return HOPU_OK;
}

}  // extern "C"
