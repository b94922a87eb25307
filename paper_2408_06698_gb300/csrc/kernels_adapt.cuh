// Adaptive HOPU (Section 3.2): the facet jump indicator
//   eta_F = int_F |(I - Pi^l)[[u]]| ds / int_F |<u>| ds
// with the facet's current order l, and the order rule eta_i < eta <= eta_{i+1} -> l = i
// (eta_{-1} = 0, eta_{k+1} = 1; below eta_0 standard upwinding l = -1; eta > 1 -> l = k;
// an empty average with a non-zero jump counts as eta = +inf).  One warp per facet,
// the traces through the modal trace matrices as in the facet kernels; the sums and the
// decision are in FP64.
#pragma once
#include "kernels.cuh"

namespace hopu {

template <int D, int K, typename T>
__global__ void __launch_bounds__(32 * kWarps) k_eta(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                     int lconst, int8_t* facet_l, EtaThresholds th,
                                                     double* __restrict__ eta_out) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NF = S::nf, NL = S::nloc, NQF = S::nqf, QP = (NQF + 31) / 32;
  constexpr int NBP = r4i(NB);
  constexpr int TRM = (D + 1) * NF * NBP, PSI = NF * NQF;
  constexpr int TABN = r4i(TRM + PSI + NQF);
  constexpr int CW = D * NBP;
  constexpr int PER_WARP = 2 * CW + 2 * NF * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  T* sbase = reinterpret_cast<T*>(smem_raw);
  {
    const T* TrMg = static_cast<const T*>(tb.TrM);
    for (int t = threadIdx.x; t < TRM; t += blockDim.x) {
      const int row = t / NBP, i = t - row * NBP;
      sbase[t] = (i < NB) ? TrMg[row * NB + i] : T(0);
    }
    for (int t = threadIdx.x; t < PSI; t += blockDim.x) sbase[TRM + t] = static_cast<const T*>(tb.Psi)[t];
    for (int t = threadIdx.x; t < NQF; t += blockDim.x) sbase[TRM + PSI + t] = static_cast<const T*>(tb.Wf)[t];
  }
  const T* TrM = sbase;
  const T* Psi = sbase + TRM;
  const T* Wf = sbase + TRM + PSI;
  pdl_wait();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* cuA = sbase + TABN + warp * PER_WARP;
  T* cuB = cuA + CW;
  T* sJu = cuB + CW;      // [NF][4] modal jump
  T* sAu = sJu + NF * 4;  // [NF][4] modal average
  for (int64_t F = (int64_t)blockIdx.x * kWarps + warp; F < m.NF; F += (int64_t)gridDim.x * kWarps) {
    const int pa = m.fa[F], pb = m.fb[F];
    const int64_t eA = pa >> 2, eB = pb >> 2;
    const int fa = pa & 3, fb = pb & 3;
    const double* fg = m.fgeo + F * (D + 1);
    T n[D];
#pragma unroll
    for (int c = 0; c < D; ++c) n[c] = T(fg[c]);
    const int l = facet_l ? int(facet_l[F]) : lconst;
    const int nl = (l < 0) ? 0 : cnbasis(D - 1, l);
    for (int s2 = lane; s2 < NL; s2 += 32) {
      const int a = s2 / NB, i = s2 - a * NB;
      cuA[a * NBP + i] = uL[eA * NL + s2];
      cuB[a * NBP + i] = uL[eB * NL + s2];
    }
    __syncwarp();
    for (int v = lane; v < NF * D; v += 32) {
      const int mm = v / D, a = v - mm * D;
      const T ua = dot_ss<NB>(TrM + (fa * NF + mm) * NBP, cuA + a * NBP);
      const T ub = dot_ss<NB>(TrM + (fb * NF + mm) * NBP, cuB + a * NBP);
      sJu[mm * 4 + a] = ua - ub;
      sAu[mm * 4 + a] = T(0.5) * (ua + ub);
    }
    __syncwarp();
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int qq = 0; qq < QP; ++qq) {
      const int q = lane + 32 * qq;
      if (q < NQF) {
        T PJ[D], Au[D];
#pragma unroll
        for (int a = 0; a < D; ++a) PJ[a] = Au[a] = T(0);
#pragma unroll
        for (int mm = 0; mm < NF; ++mm) {
          const T p = Psi[mm * NQF + q];
          T ju[4], au[4];
          lds4(sJu + mm * 4, ju);
          lds4(sAu + mm * 4, au);
          T jn = T(0);
#pragma unroll
          for (int a = 0; a < D; ++a) jn = fma(ju[a], n[a], jn);
          const bool low = mm < nl;  // (I - Pi^l) keeps only the normal part of the low modes
#pragma unroll
          for (int a = 0; a < D; ++a) {
            PJ[a] = fma(p, low ? jn * n[a] : ju[a], PJ[a]);
            Au[a] = fma(p, au[a], Au[a]);
          }
        }
        double pj2 = 0.0, au2 = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          pj2 += double(PJ[a]) * double(PJ[a]);
          au2 += double(Au[a]) * double(Au[a]);
        }
        const double w = double(Wf[q]);
        num += w * sqrt(pj2);
        den += w * sqrt(au2);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(kFull, num, o);
      den += __shfl_xor_sync(kFull, den, o);
    }
    if (lane == 0) {
      const double eta = den > 0.0 ? num / den : (num > 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : 0.0);
      if (eta_out) eta_out[F] = eta;
      int lnew = -1;
#pragma unroll
      for (int i = 0; i <= K; ++i)
        if (eta > th.t[i]) lnew = i;
      if (facet_l) facet_l[F] = (int8_t)lnew;
    }
    __syncwarp();
  }
}

}  // namespace hopu
