// CUDA kernels of the HOPU convection hot path for sm_103a, templated on the
// dimension D, the polynomial order K and the working precision T.
//
// Work decomposition: one warp per element (projections, volume term) or per facet
// (facet flux).  Reference tables are staged once per CTA in shared memory and the
// grids are persistent (a multiple of the SM count), so every CTA loads them once.
// Geometry is stored in FP64 and rounded to T at use.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "hopu_internal.h"

namespace hopu {

__host__ __device__ constexpr int cbinom(int n, int r) {
  int v = 1;
  for (int i = 1; i <= r; ++i) v = v * (n - r + i) / i;
  return (r < 0 || n < r) ? 0 : v;
}
__host__ __device__ constexpr int cnbasis(int dim, int k) { return k < 0 ? 0 : cbinom(k + dim, dim); }
__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

template <int D, int K>
struct Shape {
  static constexpr int nb = cnbasis(D, K);          // dim P^K(T)
  static constexpr int nf = cnbasis(D - 1, K);      // dim P^K(F)
  static constexpr int nloc = D * nb;               // local L2 / V_h block
  static constexpr int nint = nloc - (D + 1) * nf;  // interior V_h dofs
  static constexpr int mv = (3 * K - 1 + 2) / 2;    // points per direction, degree 3K-1
  static constexpr int mf = (3 * K + 2) / 2;        // points per direction, degree 3K
  static constexpr int nq = cpow(mv, D);
  static constexpr int nqf = cpow(mf, D - 1);
  static constexpr int geo = 2 * D * D + 2;
  static constexpr int nvp = ((nloc + 31) / 32) * 32;  // accumulators, padded to the warp
};

constexpr int kWarps = 4;  // warps per CTA of the warp-per-item kernels
constexpr unsigned kFull = 0xffffffffu;

// Butterfly reduce-scatter of N (multiple of 32) per-lane values: afterwards lane L holds
// the warp totals of indices [L*N/32, (L+1)*N/32) in v[0 .. N/32).
template <int O, int S, int N, typename T>
__device__ __forceinline__ void rs_level(T (&v)[N], int lane) {
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int j = 0; j < S / 2; ++j) {
    const T lo = v[j], hi = v[j + S / 2];
    const T send = up ? lo : hi;
    const T keep = up ? hi : lo;
    v[j] = keep + __shfl_xor_sync(kFull, send, O);
  }
}
template <int N, typename T>
__device__ __forceinline__ void reduce_scatter(T (&v)[N], int lane) {
  static_assert(N % 32 == 0, "reduce_scatter needs a multiple of 32 values");
  rs_level<16, N, N>(v, lane);
  rs_level<8, N / 2, N>(v, lane);
  rs_level<4, N / 4, N>(v, lane);
  rs_level<2, N / 8, N>(v, lane);
  rs_level<1, N / 16, N>(v, lane);
}

// Every lane ends with the warp totals of all N values.
template <int N, typename T>
__device__ __forceinline__ void allreduce(T (&v)[N]) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] += __shfl_xor_sync(kFull, v[j], o);
  }
}

template <typename T>
__device__ __forceinline__ T combine_at(const Combine& c, T v, int64_t idx) {
  T o = T(c.a2) * v;
  if (c.x0) o += T(c.a0) * static_cast<const T*>(c.x0)[idx];
  if (c.x1) o += T(c.a1) * static_cast<const T*>(c.x1)[idx];
  return o;
}

// ------------------------------------------------------------------------------------
// a1: V_h -> L2.  Per element: gather the (d+1) facet blocks with the sign sigma and the
// interior block, reference change of basis Dinv, contravariant Piola map J / det J.
template <int D, int K, typename T, bool STAB>
__global__ void __launch_bounds__(32 * kWarps) k_v2l(DevMesh m, const T* __restrict__ tab,
                                                     const T* __restrict__ uV, T* __restrict__ uL) {
  using S = Shape<D, K>;
  constexpr int NL = S::nloc, NF = S::nf, NB = S::nb, NINT = S::nint;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbase = reinterpret_cast<T*>(smem_raw);
  const T* E = tab;
  T* sw = sbase;
  if (STAB) {
    for (int t = threadIdx.x; t < NL * NL; t += blockDim.x) sbase[t] = tab[t];
    E = sbase;
    sw = sbase + NL * NL;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* l = sw + warp * 2 * NL;
  T* ch = l + NL;
  for (int64_t e = (int64_t)blockIdx.x * kWarps + warp; e < m.E; e += (int64_t)gridDim.x * kWarps) {
    for (int s = lane; s < NL; s += 32) {
      T v;
      if (s < (D + 1) * NF) {
        const int f = s / NF, mm = s - f * NF;
        const int code = m.efc[e * (D + 1) + f];
        v = uV[(int64_t)(code >> 2) * NF + mm];
        if (code & 2) v = -v;
      } else {
        v = uV[m.NF * NF + e * NINT + (s - (D + 1) * NF)];
      }
      l[s] = v;
    }
    __syncwarp();
    for (int r = lane; r < NL; r += 32) {
      T acc = T(0);
#pragma unroll 4
      for (int s = 0; s < NL; ++s) acc = fma(E[s * NL + r], l[s], acc);
      ch[r] = acc;
    }
    __syncwarp();
    const double* g = m.geo + e * S::geo;
    T J[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) J[a][b] = T(g[a * D + b]);
    const T invdet = T(1.0 / g[2 * D * D]);
    for (int idx = lane; idx < NL; idx += 32) {
      const int a = idx / NB, i = idx - a * NB;
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < D; ++b) acc = fma(J[a][b], ch[b * NB + i], acc);
      uL[e * NL + idx] = acc * invdet;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// a4: facet term.  One warp per facet, lanes own facet quadrature points.  Computes at
// every point w.n (from the average of both sides), the jump [[u]] = u^A - u^B and the
// average, then g = (w.n)<u> + (I-Pi^l)[1/2|w.n|(I-Pi^l)[[u]]] with Pi^l the tangential
// P^l projection (Section 3.2), and writes the facet moments
// gam[F][m][a] = a_F sum_q w_q psi_m(s_q) g_a(s_q) for side A (side B: -gam).
template <int D, int K, typename T, int QP, int NF>
__device__ __forceinline__ void complement_projection(T (&V)[QP][D], const T (&wq)[QP], const T* Psi,
                                                      const int (&qc)[QP], const T (&n)[D], int nl) {
  constexpr int NQF = Shape<D, K>::nqf;
  T eta[NF * D];
#pragma unroll
  for (int mm = 0; mm < NF; ++mm)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      T s = T(0);
#pragma unroll
      for (int qq = 0; qq < QP; ++qq) s += wq[qq] * Psi[mm * NQF + qc[qq]] * V[qq][a];
      eta[mm * D + a] = (mm < nl) ? s : T(0);
    }
  allreduce<NF * D>(eta);
#pragma unroll
  for (int qq = 0; qq < QP; ++qq) {
    T pis[D];
#pragma unroll
    for (int a = 0; a < D; ++a) pis[a] = T(0);
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      const T p = Psi[mm * NQF + qc[qq]];
#pragma unroll
      for (int a = 0; a < D; ++a) pis[a] = fma(p, eta[mm * D + a], pis[a]);
    }
    T dn = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) dn += pis[a] * n[a];
#pragma unroll
    for (int a = 0; a < D; ++a) V[qq][a] -= pis[a] - dn * n[a];
  }
}

template <int D, int K, typename T, bool WSEP, bool STAB>
__global__ void __launch_bounds__(32 * kWarps) k_facet(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                       const T* __restrict__ wL, int lconst,
                                                       const int8_t* __restrict__ facet_l,
                                                       T* __restrict__ gam, double* __restrict__ diss) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NF = S::nf, NL = S::nloc, NQF = S::nqf, QP = (NQF + 31) / 32;
  constexpr int TRP = (D + 1) * NB * NQF, PSI = NF * NQF;
  constexpr int TABN = ((TRP + PSI + NQF + 3) / 4) * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbase = reinterpret_cast<T*>(smem_raw);
  const T* TrP = static_cast<const T*>(tb.TrP);
  const T* Psi = static_cast<const T*>(tb.Psi);
  const T* Wf = static_cast<const T*>(tb.Wf);
  T* sw = sbase;
  if (STAB) {
    for (int t = threadIdx.x; t < TRP; t += blockDim.x) sbase[t] = TrP[t];
    for (int t = threadIdx.x; t < PSI; t += blockDim.x) sbase[TRP + t] = Psi[t];
    for (int t = threadIdx.x; t < NQF; t += blockDim.x) sbase[TRP + PSI + t] = Wf[t];
    TrP = sbase;
    Psi = sbase + TRP;
    Wf = sbase + TRP + PSI;
    sw = sbase + TABN;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int PER_WARP = WSEP ? 4 * NL : 2 * NL;
  T* cA = sw + warp * PER_WARP;
  T* cB = cA + NL;
  T* wA = WSEP ? cB + NL : cA;
  T* wB = WSEP ? wA + NL : cB;
  for (int64_t F = (int64_t)blockIdx.x * kWarps + warp; F < m.NF; F += (int64_t)gridDim.x * kWarps) {
    const int pa = m.fa[F], pb = m.fb[F];
    const int64_t eA = pa >> 2, eB = pb >> 2;
    const int fa = pa & 3, fb = pb & 3;
    const double* fg = m.fgeo + F * (D + 1);
    T n[D];
#pragma unroll
    for (int c = 0; c < D; ++c) n[c] = T(fg[c]);
    const T aF = T(fg[D]);
    const int l = facet_l ? int(facet_l[F]) : lconst;
    for (int s = lane; s < NL; s += 32) {
      cA[s] = uL[eA * NL + s];
      cB[s] = uL[eB * NL + s];
      if (WSEP) {
        wA[s] = wL[eA * NL + s];
        wB[s] = wL[eB * NL + s];
      }
    }
    __syncwarp();
    T wn[QP], J[QP][D], avg[QP][D], wq[QP];
    int qc[QP];
#pragma unroll
    for (int qq = 0; qq < QP; ++qq) {
      const int q = lane + 32 * qq;
      const bool ok = q < NQF;
      qc[qq] = ok ? q : 0;
      T ua[D], ub[D], wa[D], wb[D];
#pragma unroll
      for (int a = 0; a < D; ++a) ua[a] = ub[a] = wa[a] = wb[a] = T(0);
#pragma unroll 4
      for (int i = 0; i < NB; ++i) {
        const T ta = TrP[(fa * NB + i) * NQF + qc[qq]];
        const T tbv = TrP[(fb * NB + i) * NQF + qc[qq]];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          ua[a] = fma(ta, cA[a * NB + i], ua[a]);
          ub[a] = fma(tbv, cB[a * NB + i], ub[a]);
          if (WSEP) {
            wa[a] = fma(ta, wA[a * NB + i], wa[a]);
            wb[a] = fma(tbv, wB[a * NB + i], wb[a]);
          }
        }
      }
      T s = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) s += (WSEP ? (wa[a] + wb[a]) : (ua[a] + ub[a])) * n[a];
      wn[qq] = T(0.5) * s;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        J[qq][a] = ua[a] - ub[a];
        avg[qq][a] = T(0.5) * (ua[a] + ub[a]);
      }
      wq[qq] = ok ? Wf[qc[qq]] : T(0);
    }
    const int nl = (l < 0) ? 0 : cnbasis(D - 1, l);
    if (l >= 0) complement_projection<D, K, T, QP, NF>(J, wq, Psi, qc, n, nl);  // J <- (I-Pi)[[u]]
    T dsum = T(0);
#pragma unroll
    for (int qq = 0; qq < QP; ++qq) {
      const T aw = T(0.5) * fabs(wn[qq]);
      T j2 = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        j2 += J[qq][a] * J[qq][a];
        J[qq][a] *= aw;  // h = 1/2 |w.n| (I-Pi)[[u]]
      }
      dsum += wq[qq] * aw * j2;
    }
    if (l >= 0) complement_projection<D, K, T, QP, NF>(J, wq, Psi, qc, n, nl);  // (I-Pi) h
    T part[NF * D];
#pragma unroll
    for (int mm = 0; mm < NF; ++mm)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        T s = T(0);
#pragma unroll
        for (int qq = 0; qq < QP; ++qq)
          s += wq[qq] * Psi[mm * NQF + qc[qq]] * (wn[qq] * avg[qq][a] + J[qq][a]);
        part[mm * D + a] = s;
      }
    allreduce<NF * D>(part);
#pragma unroll
    for (int v = 0; v < NF * D; ++v)
      if ((v & 31) == lane) gam[F * NF * D + v] = aF * part[v];
    if (diss) {
      T dv[1] = {dsum};
      allreduce<1>(dv);
      if (lane == 0) diss[F] = double(aF) * double(dv[0]);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// a3 + a5: volume term, facet lift and inverse mass.  One warp per element; lanes own
// volume quadrature points:
//   r[a][i] = - sum_q w_q u_a(q) grad^ phi_i(q) . (|det J| J^{-1} w(q))
//           + sum_f side_f sum_m TrM_f[m][i] gam_F(f)[m][a],
//   y = r / |det J|      (orthonormal basis: M_T = |det J| I),
// then out = a0*x0 + a1*x1 + a2*y.  On an affine element the Piola factors of the
// volume term cancel except |det J| J^{-1}, applied to w.
template <int D, int K, typename T, bool WSEP, bool STAB>
__global__ void __launch_bounds__(32 * kWarps) k_volume(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                        const T* __restrict__ wL, const T* __restrict__ gam,
                                                        T* out, Combine cmb) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NF = S::nf, NL = S::nloc, NQ = S::nq, NVP = S::nvp, CPL = NVP / 32;
  constexpr int BT = NB * NQ, GT = NB * D * NQ, TRM = (D + 1) * NF * NB;
  constexpr int TABN = ((BT + GT + TRM + 3) / 4) * 4;
  constexpr int NG = (D + 1) * NF * D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbase = reinterpret_cast<T*>(smem_raw);
  const T* Bt = static_cast<const T*>(tb.Bt);
  const T* Gt = static_cast<const T*>(tb.Gt);
  const T* TrM = static_cast<const T*>(tb.TrM);
  T* sw = sbase;
  if (STAB) {
    for (int t = threadIdx.x; t < BT; t += blockDim.x) sbase[t] = Bt[t];
    for (int t = threadIdx.x; t < GT; t += blockDim.x) sbase[BT + t] = Gt[t];
    for (int t = threadIdx.x; t < TRM; t += blockDim.x) sbase[BT + GT + t] = TrM[t];
    Bt = sbase;
    Gt = sbase + BT;
    TrM = sbase + BT + GT;
    sw = sbase + TABN;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int PER_WARP = (WSEP ? 2 * NL : NL) + NG;
  T* c = sw + warp * PER_WARP;
  T* wt = c + NL;                    // |det J| J^{-1} w coefficients (WSEP only)
  T* gl = c + (WSEP ? 2 * NL : NL);  // signed facet moments of the element's facets
  for (int64_t e = (int64_t)blockIdx.x * kWarps + warp; e < m.E; e += (int64_t)gridDim.x * kWarps) {
    const double* g = m.geo + e * S::geo;
    T M[D][D];
    const double ad = g[2 * D * D + 1];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) M[a][b] = T(ad * g[D * D + a * D + b]);
    const T invabs = T(1.0 / ad);
    for (int s = lane; s < NL; s += 32) c[s] = uL[e * NL + s];
    if (WSEP) {
      for (int s = lane; s < NL; s += 32) {
        const int cc = s / NB, i = s - cc * NB;
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fma(M[cc][b], wL[e * NL + b * NB + i], acc);
        wt[s] = acc;
      }
    }
    for (int idx = lane; idx < NG; idx += 32) {
      const int f = idx / (NF * D), rest = idx - f * (NF * D);
      const int code = m.efc[e * (D + 1) + f];
      const T v = gam[(int64_t)(code >> 2) * NF * D + rest];
      gl[idx] = (code & 1) ? -v : v;
    }
    __syncwarp();
    T acc[NVP];
#pragma unroll
    for (int j = 0; j < NVP; ++j) acc[j] = T(0);
    for (int q = lane; q < NQ; q += 32) {
      T u[D], W[D];
#pragma unroll
      for (int a = 0; a < D; ++a) u[a] = W[a] = T(0);
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const T b = Bt[i * NQ + q];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          u[a] = fma(b, c[a * NB + i], u[a]);
          if (WSEP) W[a] = fma(b, wt[a * NB + i], W[a]);
        }
      }
      if (!WSEP) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          T s = T(0);
#pragma unroll
          for (int b = 0; b < D; ++b) s = fma(M[a][b], u[b], s);
          W[a] = s;
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        T gi = T(0);
#pragma unroll
        for (int cc = 0; cc < D; ++cc) gi = fma(Gt[(i * D + cc) * NQ + q], W[cc], gi);
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a * NB + i] = fma(u[a], gi, acc[a * NB + i]);
      }
    }
    reduce_scatter<NVP>(acc, lane);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int idx = lane * CPL + j;
      if (idx < NL) {
        const int a = idx / NB, i = idx - a * NB;
        T r = -acc[j];
#pragma unroll 4
        for (int fm = 0; fm < (D + 1) * NF; ++fm) r = fma(TrM[fm * NB + i], gl[fm * D + a], r);
        out[e * NL + idx] = combine_at<T>(cmb, r * invabs, e * NL + idx);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// a7: L2 -> V_h.  Element part: local functionals ell = D (det J J^{-1} y) (or, for the
// transpose map, ell = Dinv^T (J^T y / det J)); interior rows are final, facet rows go to
// lf[e][f][m] with the sign sigma.  Facet part (R): average (or, transposed, sum) the two
// copies of every facet functional.
template <int D, int K, typename T, bool DUAL, bool STAB>
__global__ void __launch_bounds__(32 * kWarps) k_l2v_elem(DevMesh m, const T* __restrict__ tab,
                                                          const T* __restrict__ yL, T* __restrict__ lf,
                                                          T* outV, Combine cmb) {
  using S = Shape<D, K>;
  constexpr int NL = S::nloc, NF = S::nf, NB = S::nb, NINT = S::nint;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbase = reinterpret_cast<T*>(smem_raw);
  const T* Tb = tab;
  T* sw = sbase;
  if (STAB) {
    for (int t = threadIdx.x; t < NL * NL; t += blockDim.x) sbase[t] = tab[t];
    Tb = sbase;
    sw = sbase + NL * NL;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* ch = sw + warp * NL;
  for (int64_t e = (int64_t)blockIdx.x * kWarps + warp; e < m.E; e += (int64_t)gridDim.x * kWarps) {
    const double* g = m.geo + e * S::geo;
    T A[D][D];
    if (!DUAL) {  // det J * Jinv
      const double det = g[2 * D * D];
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int a = 0; a < D; ++a) A[b][a] = T(det * g[D * D + b * D + a]);
    } else {      // J^T / det J
      const double inv = 1.0 / g[2 * D * D];
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int a = 0; a < D; ++a) A[b][a] = T(g[a * D + b] * inv);
    }
    for (int idx = lane; idx < NL; idx += 32) {
      const int b = idx / NB, i = idx - b * NB;
      T acc = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) acc = fma(A[b][a], yL[e * NL + a * NB + i], acc);
      ch[idx] = acc;
    }
    __syncwarp();
    for (int r = lane; r < NL; r += 32) {
      T v = T(0);
#pragma unroll 4
      for (int s = 0; s < NL; ++s) v = fma(Tb[s * NL + r], ch[s], v);
      if (r < (D + 1) * NF) {
        const int f = r / NF, mm = r - f * NF;
        const int code = m.efc[e * (D + 1) + f];
        lf[(e * (D + 1) + f) * NF + mm] = (code & 2) ? -v : v;
      } else {
        const int64_t idx = m.NF * NF + e * NINT + (r - (D + 1) * NF);
        outV[idx] = combine_at<T>(cmb, v, idx);
      }
    }
    __syncwarp();
  }
}

template <int D, int K, typename T, bool DUAL>
__global__ void __launch_bounds__(256) k_l2v_facet(DevMesh m, const T* __restrict__ lf, T* outV, Combine cmb) {
  constexpr int NF = Shape<D, K>::nf;
  const int64_t total = m.NF * NF;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t F = t / NF;
    const int mm = (int)(t - F * NF);
    const int pa = m.fa[F], pb = m.fb[F];
    T v = lf[((int64_t)(pa >> 2) * (D + 1) + (pa & 3)) * NF + mm] + lf[((int64_t)(pb >> 2) * (D + 1) + (pb & 3)) * NF + mm];
    if (!DUAL) v *= T(0.5);
    outV[t] = combine_at<T>(cmb, v, t);
  }
}

}  // namespace hopu
