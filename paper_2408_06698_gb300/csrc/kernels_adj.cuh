// Adjoint (VJP) kernels of the convection apply y = M^{-1} c(w; u, .) (conservative form
// of Section 3.2, eq. "hopudefinition").  With z = M^{-1} ybar:
//
//   ubar = c(w; phi_j, z)          the transposed form (u slot = basis function):
//          volume  -int ((w . grad) z) . phi_j
//          facets  side A: ( 1/2 (w.n)[[z]] + (I-Pi)(1/2|w.n|(I-Pi)[[z]]) ) . phi_j
//                  side B: ( 1/2 (w.n)[[z]] - (I-Pi)(1/2|w.n|(I-Pi)[[z]]) ) . phi_j
//   wbar = d/dw c(w; u, z) tested with phi_j:
//          volume  -sum_a u_a d_b z_a
//          facets  both sides: n [ 1/2 <u>.[[z]] + 1/4 sign(w.n) (I-Pi)[[u]].(I-Pi)[[z]] ]
//
// (w.n = <w>.n on facets; sign(0) = 0 at the kink of |w.n|).  The facet kernel writes two
// element-major moment sets (for ubar and for wbar); the volume kernel adds the volume
// parts, lifts the moments and writes ubar, wbar (or their sum when w = u).
#pragma once
#include "kernels.cuh"

namespace hopu {

template <int D, int K, typename T, bool WSEP>
__global__ void __launch_bounds__(32 * kWarps) k_facet_adj(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                           const T* __restrict__ wL, const T* __restrict__ ybar,
                                                           int lconst, const int8_t* __restrict__ facet_l,
                                                           T* __restrict__ gamU, T* __restrict__ gamW) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NF = S::nf, NL = S::nloc, NQF = S::nqf, QP = (NQF + 31) / 32;
  constexpr int NBP = r4i(NB);
  constexpr int TRM = (D + 1) * NF * NBP, PSI = NF * NQF;
  constexpr int TABN = r4i(TRM + 2 * PSI + NQF);
  constexpr int CW = D * NBP, SV = NQF * 4, GT = S::gt;
  constexpr int PER_WARP = (WSEP ? 6 : 4) * CW + 3 * SV + 4 * NF * 4 + 3 * NF * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  T* sbase = reinterpret_cast<T*>(smem_raw);
  {
    const T* TrMg = static_cast<const T*>(tb.TrM);
    for (int t = threadIdx.x; t < TRM; t += blockDim.x) {
      const int row = t / NBP, i = t - row * NBP;
      sbase[t] = (i < NB) ? TrMg[row * NB + i] : T(0);
    }
    for (int t = threadIdx.x; t < PSI; t += blockDim.x) {
      sbase[TRM + t] = static_cast<const T*>(tb.Psi)[t];
      sbase[TRM + PSI + t] = static_cast<const T*>(tb.WPsi)[t];
    }
    for (int t = threadIdx.x; t < NQF; t += blockDim.x) sbase[TRM + 2 * PSI + t] = static_cast<const T*>(tb.Wf)[t];
  }
  const T* TrM = sbase;
  const T* Psi = sbase + TRM;
  const T* WPsi = sbase + TRM + PSI;
  const double* geoT = m.geoT;
  pdl_wait();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* cuA = sbase + TABN + warp * PER_WARP;
  T* cuB = cuA + CW;
  T* czA = cuB + CW;
  T* czB = czA + CW;
  T* cwA = WSEP ? czB + CW : cuA;
  T* cwB = WSEP ? cwA + CW : cuB;
  T* sC1 = cuA + (WSEP ? 6 : 4) * CW;  // [NQF][4] 1/2 (w.n) [[z]]
  T* sH1 = sC1 + SV;                   // [NQF][4] 1/2 |w.n| (I-Pi)[[z]]
  T* sSn = sH1 + SV;                   // [NQF][4] s n (wind derivative density)
  T* sJu = sSn + SV;                   // [NF][4] modal jump of u
  T* sAu = sJu + NF * 4;               // [NF][4] modal average of u
  T* sJz = sAu + NF * 4;               // [NF][4] modal jump of z
  T* sWv = sJz + NF * 4;               // [NF][4] modal average wind
  T* sOut = sWv + NF * 4;              // [3][NF][4] alpha, beta, gamma
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
    const T iA = T(geoT[eA * GT + 3 * D * D]), iB = T(geoT[eB * GT + 3 * D * D]);  // 1/|det J|
    for (int s2 = lane; s2 < NL; s2 += 32) {
      const int a = s2 / NB, i = s2 - a * NB;
      cuA[a * NBP + i] = uL[eA * NL + s2];
      cuB[a * NBP + i] = uL[eB * NL + s2];
      czA[a * NBP + i] = ybar[eA * NL + s2] * iA;
      czB[a * NBP + i] = ybar[eB * NL + s2] * iB;
      if (WSEP) {
        cwA[a * NBP + i] = wL[eA * NL + s2];
        cwB[a * NBP + i] = wL[eB * NL + s2];
      }
    }
    __syncwarp();
    for (int v = lane; v < NF * D; v += 32) {
      const int mm = v / D, a = v - mm * D;
      const T* ra = TrM + (fa * NF + mm) * NBP;
      const T* rb = TrM + (fb * NF + mm) * NBP;
      const T ua = dot_ss<NB>(ra, cuA + a * NBP), ub = dot_ss<NB>(rb, cuB + a * NBP);
      const T za = dot_ss<NB>(ra, czA + a * NBP), zb = dot_ss<NB>(rb, czB + a * NBP);
      const T wa = WSEP ? dot_ss<NB>(ra, cwA + a * NBP) : ua;
      const T wb = WSEP ? dot_ss<NB>(rb, cwB + a * NBP) : ub;
      sJu[mm * 4 + a] = ua - ub;
      sAu[mm * 4 + a] = T(0.5) * (ua + ub);
      sJz[mm * 4 + a] = za - zb;
      sWv[mm * 4 + a] = T(0.5) * (wa + wb);
    }
    __syncwarp();
#pragma unroll
    for (int qq = 0; qq < QP; ++qq) {
      const int q = lane + 32 * qq;
      const bool ok = q < NQF;
      const int qc = ok ? q : 0;
      T PJu[D], Au[D], Jz[D], PJz[D], wn = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) PJu[a] = Au[a] = Jz[a] = PJz[a] = T(0);
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) {
        const T p = Psi[mm * NQF + qc];
        T ju[4], au[4], jz[4], wv[4];
        lds4(sJu + mm * 4, ju);
        lds4(sAu + mm * 4, au);
        lds4(sJz + mm * 4, jz);
        lds4(sWv + mm * 4, wv);
        T jun = T(0), jzn = T(0), wvn = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          jun = fma(ju[a], n[a], jun);
          jzn = fma(jz[a], n[a], jzn);
          wvn = fma(wv[a], n[a], wvn);
        }
        wn = fma(p, wvn, wn);
        const bool low = mm < nl;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          PJu[a] = fma(p, low ? jun * n[a] : ju[a], PJu[a]);
          PJz[a] = fma(p, low ? jzn * n[a] : jz[a], PJz[a]);
          Au[a] = fma(p, au[a], Au[a]);
          Jz[a] = fma(p, jz[a], Jz[a]);
        }
      }
      const T aw = T(0.5) * fabs(wn);
      const T sg = (wn > T(0)) ? T(1) : ((wn < T(0)) ? T(-1) : T(0));
      T s = T(0), pp = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        s = fma(Au[a], Jz[a], s);
        pp = fma(PJu[a], PJz[a], pp);
      }
      s = T(0.5) * s + T(0.25) * sg * pp;
      if (ok) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          sC1[q * 4 + a] = T(0.5) * wn * Jz[a];
          sH1[q * 4 + a] = aw * PJz[a];
          sSn[q * 4 + a] = s * n[a];
        }
      }
    }
    __syncwarp();
    for (int v = lane; v < 3 * NF; v += 32) {
      const int which = v / NF, mm = v - which * NF;  // 0: alpha, 1: beta, 2: wind moments
      const T* src = which == 0 ? sC1 : (which == 1 ? sH1 : sSn);
      T acc[D];
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = T(0);
      for (int q = 0; q < NQF; ++q) {
        const T wp = WPsi[mm * NQF + q];
        T x[4];
        lds4(src + q * 4, x);
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] = fma(wp, x[a], acc[a]);
      }
      if (which == 1 && mm < nl) {
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
    for (int v = lane; v < 2 * NF * D; v += 32) {
      const int side = v / (NF * D), rest = v - side * (NF * D);
      const int mm = rest / D, a = rest - mm * D;
      const T al = sOut[mm * 4 + a], be = sOut[(NF + mm) * 4 + a], ga = sOut[(2 * NF + mm) * 4 + a];
      const int64_t slot = side ? (eB * (D + 1) + fb) : (eA * (D + 1) + fa);
      gamU[slot * NF * D + rest] = side ? al - be : al + be;
      gamW[slot * NF * D + rest] = ga;
    }
    __syncwarp();
  }
}

// Volume part of the adjoint plus the lift of the facet moments.  WSEP: separate wind
// (outputs ubar and wbar); otherwise w = u and the two cotangents are summed into ubar.
template <int D, int K, typename T, bool WSEP>
__global__ void __launch_bounds__(32 * kWarps) k_volume_adj(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                            const T* __restrict__ wL, const T* __restrict__ ybar,
                                                            const T* __restrict__ gamU, const T* __restrict__ gamW,
                                                            T* __restrict__ ubar, T* __restrict__ wbar) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NB1 = cnbasis(D, K - 1), NF = S::nf, NL = S::nloc, NQ = S::nq;
  constexpr int NVP = S::nvp, CPL = NVP / 32, GT = S::gt;
  constexpr int NBP = r4i(NB), NB1P = r4i(NB1), NBQ = row_stride<T>(NB);
  constexpr int NG = (D + 1) * NF * D;
  constexpr int PER_WARP = 2 * D * NBP + D * D * NB1P + (WSEP ? D * NBP : 0) + 2 * r4i(NG);
  const T* Bt = static_cast<const T*>(tb.Bt);   // global: read through L1
  const T* Wq = static_cast<const T*>(tb.Wq);
  const T* Dm = static_cast<const T*>(tb.Dm);
  const T* TrM = static_cast<const T*>(tb.TrM);
  const double* geoT = m.geoT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  pdl_wait();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* sC = reinterpret_cast<T*>(smem_raw) + warp * PER_WARP;  // [D][NBP] u
  T* sZ = sC + D * NBP;                                     // [D][NBP] z = ybar / |det J|
  T* sGz = sZ + D * NBP;                                    // [D][D][NB1P] modal grad z
  T* sW = sGz + D * D * NB1P;                               // [D][NBP] W = M w (WSEP)
  T* sGU = sW + (WSEP ? D * NBP : 0);                       // [NG] facet moments for ubar
  T* sGW = sGU + r4i(NG);                                   // [NG] facet moments for wbar
  for (int64_t e = (int64_t)blockIdx.x * kWarps + warp; e < m.E; e += (int64_t)gridDim.x * kWarps) {
    const double* g = geoT + e * GT;
    T M[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) M[a][c] = T(g[2 * D * D + a * D + c]);
    const T invabs = T(g[3 * D * D]);
    for (int s2 = lane; s2 < NL; s2 += 32) {
      const int a = s2 / NB, i = s2 - a * NB;
      sC[a * NBP + i] = uL[e * NL + s2];
      sZ[a * NBP + i] = ybar[e * NL + s2] * invabs;
      if (WSEP) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) acc = fma(M[a][c], wL[e * NL + c * NB + i], acc);
        sW[a * NBP + i] = acc;
      }
    }
    for (int idx = lane; idx < NG; idx += 32) {
      sGU[idx] = gamU[e * NG + idx];
      sGW[idx] = gamW[e * NG + idx];
    }
    __syncwarp();
    for (int v = lane; v < D * D * NB1; v += 32) {
      const int a = v / (D * NB1), c = (v / NB1) % D, j = v % NB1;
      T acc = T(0);
      for (int i = 0; i < NB; ++i) acc = fma(Dm[(c * NB1 + j) * NB + i], sZ[a * NBP + i], acc);
      sGz[(a * D + c) * NB1P + j] = acc;
    }
    __syncwarp();
    T accU[NVP], accW[WSEP ? NVP : 1];
#pragma unroll
    for (int j = 0; j < NVP; ++j) accU[j] = T(0);
#pragma unroll
    for (int j = 0; j < (WSEP ? NVP : 1); ++j) accW[j] = T(0);
    for (int q = lane; q < NQ; q += 32) {
      T ph[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) ph[i] = Bt[q * NBQ + i];
      T u[D], Gz[D][D], W[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        u[a] = dot_row<NB>(ph, sC + a * NBP);
#pragma unroll
        for (int c = 0; c < D; ++c) Gz[a][c] = dot_row<NB1>(ph, sGz + (a * D + c) * NB1P);
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (WSEP) {
          W[c] = dot_row<NB>(ph, sW + c * NBP);
        } else {
          T s = T(0);
#pragma unroll
          for (int b = 0; b < D; ++b) s = fma(M[c][b], u[b], s);
          W[c] = s;
        }
      }
      const T wq = Wq[q];
      T f1[D], g2[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {  // -(W . grad^) z_a
        T s = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) s = fma(W[c], Gz[a][c], s);
        f1[a] = -wq * s;
      }
      T ug[D];  // sum_a u_a d^_c z_a
#pragma unroll
      for (int c = 0; c < D; ++c) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) s = fma(u[a], Gz[a][c], s);
        ug[c] = s;
      }
#pragma unroll
      for (int b = 0; b < D; ++b) {  // -sum_c M[c][b] ug_c
        T s = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) s = fma(M[c][b], ug[c], s);
        g2[b] = -wq * s;
      }
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (WSEP) {
            accU[a * NB + i] = fma(f1[a], ph[i], accU[a * NB + i]);
            accW[(WSEP ? a * NB + i : 0)] = fma(g2[a], ph[i], accW[(WSEP ? a * NB + i : 0)]);
          } else {
            accU[a * NB + i] = fma(f1[a] + g2[a], ph[i], accU[a * NB + i]);
          }
        }
    }
    reduce_scatter<NVP>(accU, lane);
    if constexpr (WSEP) reduce_scatter<NVP>(accW, lane);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int idx = lane * CPL + j;
      if (idx < NL) {
        const int a = idx / NB, i = idx - a * NB;
        T ru = accU[j], rw = T(0);
        for (int fm = 0; fm < (D + 1) * NF; ++fm) {
          const T t = TrM[fm * NB + i];
          ru = fma(t, sGU[fm * D + a], ru);
          rw = fma(t, sGW[fm * D + a], rw);
        }
        if constexpr (WSEP) {
          ubar[e * NL + idx] = ru;
          wbar[e * NL + idx] = accW[j] + rw;
        } else {
          ubar[e * NL + idx] = ru + rw;
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace hopu
