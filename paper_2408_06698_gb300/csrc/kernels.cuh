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
__host__ __device__ constexpr int r4i(int n) { return ((n + 3) / 4) * 4; }

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
// Projections: each warp handles kEPW elements at once so that every table entry read
// from shared memory feeds kEPW FMAs (the per-element operands are stored interleaved,
// [s][kEPW], and read with one vector load).
constexpr int kEPW = 4;

template <typename T>
__device__ __forceinline__ void load_epw(const T* p, T (&v)[kEPW]);
template <>
__device__ __forceinline__ void load_epw<float>(const float* p, float (&v)[kEPW]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <>
__device__ __forceinline__ void load_epw<double>(const double* p, double (&v)[kEPW]) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  const double2 y = *reinterpret_cast<const double2*>(p + 2);
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// out[k][r] = sum_s tab[s][r] * in[s][k] for kEPW elements (in interleaved, out [k][NL]).
template <int NL, typename T>
__device__ __forceinline__ void epw_gemv(const T* tab, const T* in, T* out, int lane) {
  for (int r0 = lane; r0 < NL; r0 += 64) {
    const int r1 = r0 + 32;
    const bool has1 = r1 < NL;
    const int r1c = has1 ? r1 : r0;
    T a0[kEPW], a1[kEPW];
#pragma unroll
    for (int k = 0; k < kEPW; ++k) a0[k] = a1[k] = T(0);
#pragma unroll 4
    for (int s2 = 0; s2 < NL; ++s2) {
      T v[kEPW];
      load_epw<T>(in + s2 * kEPW, v);
      const T t0 = tab[s2 * NL + r0], t1 = tab[s2 * NL + r1c];
#pragma unroll
      for (int k = 0; k < kEPW; ++k) {
        a0[k] = fma(t0, v[k], a0[k]);
        a1[k] = fma(t1, v[k], a1[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kEPW; ++k) {
      out[k * NL + r0] = a0[k];
      if (has1) out[k * NL + r1] = a1[k];
    }
  }
}

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
    sw = sbase + r4i(NL * NL);  // keeps the per-warp buffers 16-byte aligned
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* l = sw + warp * 2 * kEPW * NL;  // [NL][kEPW] gathered local dofs
  T* ch = l + kEPW * NL;             // [kEPW][NL] reference coefficients
  for (int64_t e0 = ((int64_t)blockIdx.x * kWarps + warp) * kEPW; e0 < m.E;
       e0 += (int64_t)gridDim.x * kWarps * kEPW) {
    for (int t = lane; t < kEPW * NL; t += 32) {
      const int k = t / NL, s2 = t - k * NL;
      const int64_t e = e0 + k;
      T v = T(0);
      if (e < m.E) {
        if (s2 < (D + 1) * NF) {
          const int f = s2 / NF, mm = s2 - f * NF;
          const int code = m.efc[e * (D + 1) + f];
          v = uV[(int64_t)(code >> 2) * NF + mm];
          if (code & 2) v = -v;
        } else {
          v = uV[m.NF * NF + e * NINT + (s2 - (D + 1) * NF)];
        }
      }
      l[s2 * kEPW + k] = v;
    }
    __syncwarp();
    epw_gemv<NL, T>(E, l, ch, lane);
    __syncwarp();
    for (int t = lane; t < kEPW * NL; t += 32) {
      const int k = t / NL, idx = t - k * NL;
      const int64_t e = e0 + k;
      if (e >= m.E) continue;
      const double* g = m.geo + e * S::geo;
      const int a = idx / NB, i = idx - a * NB;
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < D; ++b) acc = fma(T(g[a * D + b]), ch[k * NL + b * NB + i], acc);
      uL[e * NL + idx] = acc * T(1.0 / g[2 * D * D]);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// Vectorised dot product of a register array with a 16-byte aligned shared-memory row
// (the row is padded to a multiple of 4 entries; padding entries are never used).
template <typename T> struct Pack;
template <> struct Pack<float> {
  static constexpr int W = 4;
  using V = float4;
  __device__ __forceinline__ static void unpack(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};
template <> struct Pack<double> {
  static constexpr int W = 2;
  using V = double2;
  __device__ __forceinline__ static void unpack(const V& v, double* o) { o[0] = v.x; o[1] = v.y; }
};

template <int N, typename T>
__device__ __forceinline__ T dot_row(const T* x, const T* s) {
  constexpr int W = Pack<T>::W;
  T acc = T(0);
#pragma unroll
  for (int i = 0; i < N; i += W) {
    const typename Pack<T>::V v = *reinterpret_cast<const typename Pack<T>::V*>(s + i);
    T o[W];
    Pack<T>::unpack(v, o);
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (i + w < N) acc = fma(x[i + w], o[w], acc);
  }
  return acc;
}

__host__ __device__ constexpr int gcd_pow2(int bytes) { return (bytes % 16 == 0) ? 16 : (bytes % 8 == 0) ? 8 : 4; }

// Asynchronous global -> shared copies (cp.async, completion tracked per thread by
// commit/wait groups).  CH is the chunk size in bytes (4, 8 or 16); both addresses must
// be CH-aligned.
template <int CH>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (CH == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  } else if constexpr (CH == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// A warp copies one contiguous record of NBYTES bytes (record offsets are multiples of
// NBYTES and base pointers are 16-byte aligned, so gcd_pow2(NBYTES) alignment holds).
template <int NBYTES>
__device__ __forceinline__ void warp_copy_async(void* sdst, const void* gsrc, int lane) {
  constexpr int CH = gcd_pow2(NBYTES);
  constexpr int N = NBYTES / CH;
  for (int i = lane; i < N; i += 32)
    cp_async<CH>(static_cast<char*>(sdst) + i * CH, static_cast<const char*>(gsrc) + i * CH);
}

// ------------------------------------------------------------------------------------
// a4: facet term.  One warp per facet, lanes own facet quadrature points.  At every
// point: w.n from the average of both sides' w (equal to w.n for normal-continuous w),
// the jump J = u^A - u^B, (I - Pi^l) J with Pi^l the tangential P^l projection of
// Section 3.2, h = 1/2 |w.n| (I - Pi^l) J.  Writes two sets of facet moments
//   gam[F][0][m][a] = a_F sum_q w_q psi_m(q) (-1/2 (w.n) J_a(q))            ("alpha")
//   gam[F][1][m][a] = a_F sum_q w_q psi_m(q) ((I - Pi^l) h)_a(q)              ("beta")
// Side A of the facet receives alpha + beta, side B alpha - beta.  Together with the
// volume kernel this is the conservative form of the convection operator rewritten by
// the element-wise integration by parts, which is exact for the rules used (volume
// degree 3k-1, facet degree 3k): every term is O(|u| |grad u|) or O(jump), so FP32
// does not lose digits to the O(1/h) cancellation between volume and facet terms.
// The projection of h needs no second reduction: with an orthonormal facet basis the
// moments of (I - Pi^l) h are those of h with the tangential part of the first
// C(l+d-1, d-1) moments removed.
template <int D, int K, typename T, bool WSEP, bool STAB>
__global__ void __launch_bounds__(32 * kWarps) k_facet(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                       const T* __restrict__ wL, int lconst,
                                                       const int8_t* __restrict__ facet_l,
                                                       T* __restrict__ gam, double* __restrict__ diss) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NF = S::nf, NL = S::nloc, NQF = S::nqf, QP = (NQF + 31) / 32;
  constexpr int TRP = (D + 1) * NB * NQF, PSI = NF * NQF;
  constexpr int TABN = r4i(TRP + 2 * PSI + NQF);
  constexpr int NBP = r4i(NB);
  constexpr int CW = D * NBP;
  constexpr int SV = NQF * 4;
  constexpr int PER_WARP = (WSEP ? 4 : 2) * CW + 2 * SV + NF * 4 + 2 * NF * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbase = reinterpret_cast<T*>(smem_raw);
  const T* TrP = static_cast<const T*>(tb.TrP);
  const T* Psi = static_cast<const T*>(tb.Psi);
  const T* WPsi = static_cast<const T*>(tb.WPsi);
  const T* Wf = static_cast<const T*>(tb.Wf);
  T* sw = sbase;
  if (STAB) {
    for (int t = threadIdx.x; t < TRP; t += blockDim.x) sbase[t] = TrP[t];
    for (int t = threadIdx.x; t < PSI; t += blockDim.x) {
      sbase[TRP + t] = Psi[t];
      sbase[TRP + PSI + t] = WPsi[t];
    }
    for (int t = threadIdx.x; t < NQF; t += blockDim.x) sbase[TRP + 2 * PSI + t] = Wf[t];
    TrP = sbase;
    Psi = sbase + TRP;
    WPsi = sbase + TRP + PSI;
    Wf = sbase + TRP + 2 * PSI;
    sw = sbase + TABN;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* cA = sw + warp * PER_WARP;
  T* cB = cA + CW;
  T* wA = WSEP ? cB + CW : cA;
  T* wB = WSEP ? wA + CW : cB;
  T* sH = cA + (WSEP ? 4 : 2) * CW;  // [NQF][4]  h, or the jump while projecting
  T* sC = sH + SV;                   // [NQF][4]  -1/2 (w.n) J
  T* sEta = sC + SV;                 // [NF][4]   P^l moments of the jump
  T* sOut = sEta + NF * 4;           // [2][NF][4] alpha, beta
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
    const int nl = (l < 0) ? 0 : cnbasis(D - 1, l);
    for (int s = lane; s < NL; s += 32) {
      const int a = s / NB, i = s - a * NB;
      cA[a * NBP + i] = uL[eA * NL + s];
      cB[a * NBP + i] = uL[eB * NL + s];
      if (WSEP) {
        wA[a * NBP + i] = wL[eA * NL + s];
        wB[a * NBP + i] = wL[eB * NL + s];
      }
    }
    __syncwarp();
    T wn[QP], J[QP][D], P[QP][D], wq[QP];
    int qc[QP];
#pragma unroll
    for (int qq = 0; qq < QP; ++qq) {
      const int q = lane + 32 * qq;
      const bool ok = q < NQF;
      qc[qq] = ok ? q : 0;
      T ta[NB], tbv[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        ta[i] = TrP[(fa * NB + i) * NQF + qc[qq]];
        tbv[i] = TrP[(fb * NB + i) * NQF + qc[qq]];
      }
      T s = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const T ua = dot_row<NB>(ta, cA + a * NBP);
        const T ub = dot_row<NB>(tbv, cB + a * NBP);
        const T wa = WSEP ? dot_row<NB>(ta, wA + a * NBP) : ua;
        const T wb = WSEP ? dot_row<NB>(tbv, wB + a * NBP) : ub;
        s += (wa + wb) * n[a];
        J[qq][a] = ua - ub;
        P[qq][a] = J[qq][a];
      }
      wn[qq] = T(0.5) * s;
      wq[qq] = ok ? Wf[qc[qq]] : T(0);
    }
    if (nl > 0) {  // (I - Pi^l) J: one reduction for the P^l moments of the jump
#pragma unroll
      for (int qq = 0; qq < QP; ++qq) {
        const int q = lane + 32 * qq;
        if (q < NQF)
#pragma unroll
          for (int a = 0; a < D; ++a) sH[q * 4 + a] = J[qq][a];
      }
      __syncwarp();
      for (int v = lane; v < nl * D; v += 32) {
        const int mm = v / D, a = v - mm * D;
        T acc = T(0);
        for (int q = 0; q < NQF; ++q) acc = fma(WPsi[mm * NQF + q], sH[q * 4 + a], acc);
        sEta[mm * 4 + a] = acc;
      }
      __syncwarp();
#pragma unroll
      for (int qq = 0; qq < QP; ++qq) {
        T pis[D];
#pragma unroll
        for (int a = 0; a < D; ++a) pis[a] = T(0);
        for (int mm = 0; mm < nl; ++mm) {
          const T p = Psi[mm * NQF + qc[qq]];
#pragma unroll
          for (int a = 0; a < D; ++a) pis[a] = fma(p, sEta[mm * 4 + a], pis[a]);
        }
        T dn = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) dn += pis[a] * n[a];
#pragma unroll
        for (int a = 0; a < D; ++a) P[qq][a] -= pis[a] - dn * n[a];
      }
      __syncwarp();  // sH is overwritten below
    }
    T dsum = T(0);
#pragma unroll
    for (int qq = 0; qq < QP; ++qq) {
      const int q = lane + 32 * qq;
      const T aw = T(0.5) * fabs(wn[qq]);
      T p2 = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) p2 += P[qq][a] * P[qq][a];
      dsum += wq[qq] * aw * p2;
      if (q < NQF) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          sH[q * 4 + a] = aw * P[qq][a];
          sC[q * 4 + a] = T(-0.5) * wn[qq] * J[qq][a];
        }
      }
    }
    __syncwarp();
    for (int v = lane; v < 2 * NF; v += 32) {
      const int which = v / NF, mm = v - which * NF;  // 0: alpha (central), 1: beta (upwind part)
      const T* src = which ? sH : sC;
      T acc[D];
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = T(0);
      for (int q = 0; q < NQF; ++q) {
        const T wp = WPsi[mm * NQF + q];
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] = fma(wp, src[q * 4 + a], acc[a]);
      }
      if (which && mm < nl) {  // (I - Pi^l) h: keep only the normal part of the low moments
        T dn = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) dn += acc[a] * n[a];
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] = dn * n[a];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) sOut[(which * NF + mm) * 4 + a] = aF * acc[a];
    }
    __syncwarp();
    // element-major output: side A's slot gets alpha + beta, side B's alpha - beta
    for (int v = lane; v < 2 * NF * D; v += 32) {
      const int side = v / (NF * D), rest = v - side * (NF * D);
      const int mm = rest / D, a = rest - mm * D;
      const T al = sOut[mm * 4 + a], be = sOut[(NF + mm) * 4 + a];
      const int64_t slot = side ? (eB * (D + 1) + fb) : (eA * (D + 1) + fa);
      gam[slot * NF * D + rest] = side ? al - be : al + be;
    }
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
// volume quadrature points.  With W = |det J| J^{-1} w (so that |det J| (w.grad) u =
// W . grad^ u and |det J| div w = div^ W on an affine element):
//   r[a][i] = sum_q w_q phi_i(q) [ W(q) . grad^ u_a(q) + div^ W(q) u_a(q) ]
//           + sum_f sum_m TrM_f[m][i] (alpha_F(f) +- beta_F(f))[m][a],
//   y = r / |det J|      (orthonormal basis: M_T = |det J| I),
// then out = a0*x0 + a1*x1 + a2*y.  The reference gradients come from the modal
// differentiation matrices Dm (grad^ u_a = sum_j (Dm u_a)_j phi_j, j < dim P^{k-1}), so
// the only per-point table is phi_i(q).  Every per-element input (coefficients, the
// element's signed facet moments, geometry) is one contiguous record; a warp prefetches
// the next element's records with cp.async while it computes the current one.
template <int D, int K, typename T, bool WSEP, bool STAB>
__global__ void __launch_bounds__(32 * kWarps, 2) k_volume(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                           const T* __restrict__ wL, const T* __restrict__ gam,
                                                           T* out, Combine cmb) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NB1 = cnbasis(D, K - 1), NF = S::nf, NL = S::nloc, NQ = S::nq;
  constexpr int NVP = S::nvp, CPL = NVP / 32, GEO = S::geo;
  constexpr int NBP = r4i(NB), NB1P = r4i(NB1);
  constexpr int BT = NB * NQ, DM = D * NB1 * NB, TRM = (D + 1) * NF * NB;
  constexpr int TABN = r4i(BT + NQ + DM + TRM);
  constexpr int NG = (D + 1) * NF * D;
  // per-warp layout: two staging buffers (u record, w record, facet moments, geometry),
  // then the working arrays
  constexpr int STU = r4i(NL), STG = r4i(NG), STGEO = 2 * r4i(GEO);  // geometry in T units
  constexpr int STAGE = STU + (WSEP ? STU : 0) + STG + STGEO;
  constexpr int PER_WARP = 2 * STAGE + D * NBP + D * D * NB1P + (WSEP ? D * NBP + NB1P : 0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbase = reinterpret_cast<T*>(smem_raw);
  const T* Bt = static_cast<const T*>(tb.Bt);
  const T* Wq = static_cast<const T*>(tb.Wq);
  const T* Dm = static_cast<const T*>(tb.Dm);
  const T* TrM = static_cast<const T*>(tb.TrM);
  T* sw = sbase;
  if (STAB) {
    for (int t = threadIdx.x; t < BT; t += blockDim.x) sbase[t] = Bt[t];
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) sbase[BT + t] = Wq[t];
    for (int t = threadIdx.x; t < DM; t += blockDim.x) sbase[BT + NQ + t] = Dm[t];
    for (int t = threadIdx.x; t < TRM; t += blockDim.x) sbase[BT + NQ + DM + t] = TrM[t];
    Bt = sbase;
    Wq = sbase + BT;
    Dm = sbase + BT + NQ;
    TrM = sbase + BT + NQ + DM;
    sw = sbase + TABN;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* wbase = sw + warp * PER_WARP;
  T* sC = wbase + 2 * STAGE;                // [D][NBP]       u coefficients
  T* sG = sC + D * NBP;                     // [D][D][NB1P]   modal reference gradients of u
  T* sW = sG + D * D * NB1P;                // [D][NBP]       W coefficients (WSEP)
  T* sDv = sW + (WSEP ? D * NBP : 0);       // [NB1P]         modal div^ W (WSEP)
  auto st_u = [&](int b) { return wbase + b * STAGE; };
  auto st_w = [&](int b) { return wbase + b * STAGE + STU; };
  auto st_g = [&](int b) { return wbase + b * STAGE + STU + (WSEP ? STU : 0); };
  auto st_geo = [&](int b) { return reinterpret_cast<double*>(st_g(b) + STG); };
  auto issue = [&](int64_t e, int b) {
    warp_copy_async<NL * (int)sizeof(T)>(st_u(b), uL + e * NL, lane);
    if (WSEP) warp_copy_async<NL * (int)sizeof(T)>(st_w(b), wL + e * NL, lane);
    warp_copy_async<NG * (int)sizeof(T)>(st_g(b), gam + e * NG, lane);
    warp_copy_async<GEO * 8>(st_geo(b), m.geo + e * GEO, lane);
  };
  const int64_t stride = (int64_t)gridDim.x * kWarps;
  int64_t e = (int64_t)blockIdx.x * kWarps + warp;
  if (e < m.E) issue(e, 0);
  cp_commit();
  int b = 0;
  for (; e < m.E; e += stride, b ^= 1) {
    if (e + stride < m.E) issue(e + stride, b ^ 1);  // prefetch the next element
    cp_commit();
    cp_wait<1>();                                    // this element's copies are done
    __syncwarp();
    const double* g = st_geo(b);
    const T* gl = st_g(b);                           // signed facet moments of the element
    T M[D][D];
    const double ad = g[2 * D * D + 1];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) M[a][c] = T(ad * g[D * D + a * D + c]);
    const T invabs = T(1.0 / ad);
    for (int s2 = lane; s2 < NL; s2 += 32) {
      const int a = s2 / NB, i = s2 - a * NB;
      sC[a * NBP + i] = st_u(b)[s2];
      if (WSEP) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) acc = fma(M[a][c], st_w(b)[c * NB + i], acc);
        sW[a * NBP + i] = acc;
      }
    }
    __syncwarp();
    for (int v = lane; v < D * D * NB1; v += 32) {
      const int a = v / (D * NB1), c = (v / NB1) % D, j = v % NB1;
      T acc = T(0);
#pragma unroll 4
      for (int i = 0; i < NB; ++i) acc = fma(Dm[(c * NB1 + j) * NB + i], sC[a * NBP + i], acc);
      sG[(a * D + c) * NB1P + j] = acc;
    }
    if (WSEP) {
      for (int j = lane; j < NB1; j += 32) {
        T acc = T(0);
        for (int c = 0; c < D; ++c)
#pragma unroll 4
          for (int i = 0; i < NB; ++i) acc = fma(Dm[(c * NB1 + j) * NB + i], sW[c * NBP + i], acc);
        sDv[j] = acc;
      }
    }
    __syncwarp();
    T acc[NVP];
#pragma unroll
    for (int j = 0; j < NVP; ++j) acc[j] = T(0);
    for (int q = lane; q < NQ; q += 32) {
      T ph[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) ph[i] = Bt[i * NQ + q];
      T u[D], G[D][D], W[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        u[a] = dot_row<NB>(ph, sC + a * NBP);
#pragma unroll
        for (int c = 0; c < D; ++c) G[a][c] = dot_row<NB1>(ph, sG + (a * D + c) * NB1P);
      }
      T dv = T(0);
      if (WSEP) {
#pragma unroll
        for (int c = 0; c < D; ++c) W[c] = dot_row<NB>(ph, sW + c * NBP);
        dv = dot_row<NB1>(ph, sDv);
      } else {
#pragma unroll
        for (int c = 0; c < D; ++c) {
          T sacc = T(0);
#pragma unroll
          for (int bb = 0; bb < D; ++bb) {
            sacc = fma(M[c][bb], u[bb], sacc);
            dv = fma(M[c][bb], G[bb][c], dv);
          }
          W[c] = sacc;
        }
      }
      const T wq = Wq[q];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        T f = dv * u[a];
#pragma unroll
        for (int c = 0; c < D; ++c) f = fma(W[c], G[a][c], f);
        f *= wq;
#pragma unroll
        for (int i = 0; i < NB; ++i) acc[a * NB + i] = fma(f, ph[i], acc[a * NB + i]);
      }
    }
    reduce_scatter<NVP>(acc, lane);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int idx = lane * CPL + j;
      if (idx < NL) {
        const int a = idx / NB, i = idx - a * NB;
        T r = acc[j];
#pragma unroll 4
        for (int fm = 0; fm < (D + 1) * NF; ++fm) r = fma(TrM[fm * NB + i], gl[fm * D + a], r);
        out[e * NL + idx] = combine_at<T>(cmb, r * invabs, e * NL + idx);
      }
    }
    __syncwarp();
  }
  cp_wait<0>();
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
    sw = sbase + r4i(NL * NL);  // keeps the per-warp buffers 16-byte aligned
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* ch = sw + warp * 2 * kEPW * NL;  // [NL][kEPW] reference coefficients (interleaved)
  T* ell = ch + kEPW * NL;            // [kEPW][NL] local functionals
  for (int64_t e0 = ((int64_t)blockIdx.x * kWarps + warp) * kEPW; e0 < m.E;
       e0 += (int64_t)gridDim.x * kWarps * kEPW) {
    for (int t = lane; t < kEPW * NL; t += 32) {
      const int k = t / NL, idx = t - k * NL;
      const int64_t e = e0 + k;
      T acc = T(0);
      if (e < m.E) {
        const double* g = m.geo + e * S::geo;
        const int b = idx / NB, i = idx - b * NB;
        if (!DUAL) {  // det J * Jinv * y
          const double det = g[2 * D * D];
#pragma unroll
          for (int a = 0; a < D; ++a) acc = fma(T(det * g[D * D + b * D + a]), yL[e * NL + a * NB + i], acc);
        } else {      // J^T y / det J
          const double inv = 1.0 / g[2 * D * D];
#pragma unroll
          for (int a = 0; a < D; ++a) acc = fma(T(g[a * D + b] * inv), yL[e * NL + a * NB + i], acc);
        }
      }
      ch[idx * kEPW + k] = acc;
    }
    __syncwarp();
    epw_gemv<NL, T>(Tb, ch, ell, lane);
    __syncwarp();
    for (int t = lane; t < kEPW * NL; t += 32) {
      const int k = t / NL, r = t - k * NL;
      const int64_t e = e0 + k;
      if (e >= m.E) continue;
      const T v = ell[k * NL + r];
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
