// The facet part of the adjoint (VJP) of the STAGE apply (w = u), FP32, with the facet's
// data in registers: the layout of k_facet_r applied to the transposed form of
// k_facet_adj (same moments, same arithmetic per point).
//
// A lane owns one (facet, component a) pair.  From the coefficients of both sides it forms
// the modal traces of u_a and of z_a = ybar_a / |det J| (each side with its own inverse
// mass): the jumps [[u]]_m, [[z]]_m and the average <u>_m (= the averaged wind, w = u); the
// facet's lanes sum the normal parts by shuffles, giving (I - Pi^l)[[u]] and (I - Pi^l)[[z]]
// in modal form.  The facet points are walked in the same order by every lane (broadcast
// rows of psi and w_q psi): w.n, the point values, s = 1/2 <u>.[[z]] + 1/4 sign(w.n)
// (I - Pi)[[u]].(I - Pi)[[z]] (summed over the lanes), and the moments
//   alpha_m += w_q psi_m 1/2 (w.n) [[z]]_a,  beta_m += w_q psi_m 1/2 |w.n| (I - Pi)[[z]]_a,
//   gamma_m += w_q psi_m s n_a
// in registers; beta's low modes keep their normal part; alpha +- beta (sides A / B) go to
// the ubar moments, gamma to the wbar moments, scaled by a_F, element-major.
#pragma once
#include "kernels.cuh"
#include "kernels_fr.cuh"

namespace hopu {

template <int D, int K>
struct FacAR {
  using F = FacR<D, K>;
  static constexpr int NB = F::NB, NF = F::NF, NL = F::NL, NQF = F::NQF, FPW = F::FPW, WARPS = 4;
  static constexpr int NB4 = F::NB4, NF4 = F::NF4;
  static constexpr size_t SMEM = F::SMEM;        // the tables of k_facet_r
  static constexpr int REGS = 2 * NB + 8 * NF;   // coefficients of one field, modal vectors, moments
  static constexpr bool OK = REGS <= 200;
  static constexpr int MINB = REGS <= 110 ? 3 : 2;
};

template <int D, int K>
__global__ void __launch_bounds__(32 * FacAR<D, K>::WARPS, FacAR<D, K>::MINB)
    k_facet_adj_r(DevMesh m, DevTabs tb, const float* __restrict__ uL, const float* __restrict__ ybar, int lconst,
                  const int8_t* __restrict__ facet_l, float* __restrict__ gamU, float* __restrict__ gamW) {
  using C = FacAR<D, K>;
  using FR = FacR<D, K>;
  constexpr int NB = C::NB, NF = C::NF, NL = C::NL, NQF = C::NQF, NB4 = C::NB4, NF4 = C::NF4, FPW = C::FPW;
  constexpr int GT = Shape<D, K>::gt;
  extern __shared__ __align__(16) float sm[];
  pdl_trigger();
  {
    const float* TrMg = static_cast<const float*>(tb.TrM);
    const float* Psig = static_cast<const float*>(tb.Psi);    // [NF][NQF]
    const float* WPsig = static_cast<const float*>(tb.WPsi);  // [NF][NQF]
    const float* Wfg = static_cast<const float*>(tb.Wf);
    for (int t = threadIdx.x; t < (D + 1) * NF * NB4; t += blockDim.x) {
      const int row = t / NB4, i = t - row * NB4;
      sm[FR::O_TRM + t] = i < NB ? TrMg[row * NB + i] : 0.0f;
    }
    for (int t = threadIdx.x; t < NQF * NF4; t += blockDim.x) {
      const int q = t / NF4, mm = t - q * NF4;
      sm[FR::O_PSI + t] = mm < NF ? Psig[mm * NQF + q] : 0.0f;
      sm[FR::O_WPSI + t] = mm < NF ? WPsig[mm * NQF + q] : 0.0f;
    }
    for (int t = threadIdx.x; t < NQF; t += blockDim.x) sm[FR::O_WF + t] = Wfg[t];
  }
  const float* sTrM = sm + FR::O_TRM;
  const float* sPsi = sm + FR::O_PSI;
  const float* sWPsi = sm + FR::O_WPSI;
  pdl_wait();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool lane_on = lane < D * FPW;
  const int fl = lane_on ? lane / D : 0;
  const int a = lane_on ? lane - fl * D : 0;
  const int p1 = lane_on ? fl * D + (a + 1) % D : lane;
  const int p2 = lane_on ? fl * D + (a + 2) % D : lane;
  auto lanes_sum = [&](float v) {
    float s = v + __shfl_sync(kFull, v, p1);
    if (D == 3) s += __shfl_sync(kFull, v, p2);
    return s;
  };
  // modal traces of one field of both sides: tA_m = sum_i TrM_fA[m][i] cA_i (same for B)
  auto traces = [&](const float* src, int64_t eA, int64_t eB, int fA, int fB, float sA, float sB, float* tA,
                    float* tB) {
    float cA[NB], cB[NB];
    const float* pa = src + eA * NL + a * NB;
    const float* pb = src + eB * NL + a * NB;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      cA[i] = __ldg(pa + i) * sA;
      cB[i] = __ldg(pb + i) * sB;
    }
    const float* trA = sTrM + fA * NF * NB4;
    const float* trB = sTrM + fB * NF * NB4;
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      float s0 = 0.0f, s1 = 0.0f, t0 = 0.0f, t1 = 0.0f;
#pragma unroll
      for (int i = 0; i < NB; i += 4) {
        float ta[4], tbv[4];
        lds_v(trA + mm * NB4 + i, ta);
        lds_v(trB + mm * NB4 + i, tbv);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (i + w < NB) {
            if (w & 1) {
              s1 = fmaf(ta[w], cA[i + w], s1);
              t1 = fmaf(tbv[w], cB[i + w], t1);
            } else {
              s0 = fmaf(ta[w], cA[i + w], s0);
              t0 = fmaf(tbv[w], cB[i + w], t0);
            }
          }
      }
      tA[mm] = s0 + s1;
      tB[mm] = t0 + t1;
    }
  };
  const int64_t ngroups = (m.NF + FPW - 1) / FPW;
  for (int64_t grp = (int64_t)warp * gridDim.x + blockIdx.x; grp < ngroups; grp += (int64_t)gridDim.x * C::WARPS) {
    const int64_t F0 = grp * FPW;
    const bool act = lane_on && F0 + fl < m.NF;
    const int64_t F = act ? F0 + fl : F0;  // inactive lanes compute the group's first facet
    const int pa = m.fa[F], pb = m.fb[F];
    const int64_t eA = pa >> 2, eB = pb >> 2;
    const int fA = pa & 3, fB = pb & 3;
    const double* fg = m.fgeo + F * (D + 1);
    float n[D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) n[cc] = float(fg[cc]);
    const float aF = float(fg[D]);
    const float na = (a == 0) ? n[0] : (a == 1 ? n[1] : n[D - 1]);
    const int l = facet_l ? int(facet_l[F]) : lconst;
    const int nl = (l < 0) ? 0 : cnbasis(D - 1, l);
    const float iA = float(m.geoT[eA * GT + 3 * D * D]), iB = float(m.geoT[eB * GT + 3 * D * D]);
    // modal jumps and averages, component a
    float Ju[NF], Au[NF], Jz[NF];
    {
      float tA[NF], tB[NF];
      traces(uL, eA, eB, fA, fB, 1.0f, 1.0f, tA, tB);
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) {
        Ju[mm] = tA[mm] - tB[mm];
        Au[mm] = 0.5f * (tA[mm] + tB[mm]);
      }
      traces(ybar, eA, eB, fA, fB, iA, iB, tA, tB);
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) Jz[mm] = tA[mm] - tB[mm];
    }
    // normal parts over the facet's lanes: <w>_m . n (w = u), and (I - Pi^l) in modal form
    float Wn[NF], PJu[NF], PJz[NF];
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      Wn[mm] = lanes_sum(Au[mm] * na);
      const float jun = lanes_sum(Ju[mm] * na);
      const float jzn = lanes_sum(Jz[mm] * na);
      PJu[mm] = (mm < nl) ? jun * na : Ju[mm];
      PJz[mm] = (mm < nl) ? jzn * na : Jz[mm];
    }
    float al[NF], be[NF], ga[NF];
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) al[mm] = be[mm] = ga[mm] = 0.0f;
#pragma unroll 1
    for (int q = 0; q < NQF; ++q) {
      const float* ps = sPsi + q * NF4;
      float wn = 0.0f, pu = 0.0f, pz = 0.0f, au = 0.0f, jz = 0.0f;
#pragma unroll
      for (int mm = 0; mm < NF; mm += 4) {
        float pv[4];
        lds_v(ps + mm, pv);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (mm + w < NF) {
            wn = fmaf(pv[w], Wn[mm + w], wn);
            pu = fmaf(pv[w], PJu[mm + w], pu);
            pz = fmaf(pv[w], PJz[mm + w], pz);
            au = fmaf(pv[w], Au[mm + w], au);
            jz = fmaf(pv[w], Jz[mm + w], jz);
          }
      }
      const float aw = 0.5f * fabsf(wn);
      const float sg = (wn > 0.0f) ? 1.0f : ((wn < 0.0f) ? -1.0f : 0.0f);
      const float s = 0.5f * lanes_sum(au * jz) + 0.25f * sg * lanes_sum(pu * pz);
      const float c1 = 0.5f * wn * jz, h1 = aw * pz, sn = s * na;
      const float* wp = sWPsi + q * NF4;
#pragma unroll
      for (int mm = 0; mm < NF; mm += 4) {
        float wv[4];
        lds_v(wp + mm, wv);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (mm + w < NF) {
            al[mm + w] = fmaf(wv[w], c1, al[mm + w]);
            be[mm + w] = fmaf(wv[w], h1, be[mm + w]);
            ga[mm + w] = fmaf(wv[w], sn, ga[mm + w]);
          }
      }
    }
    // (I - Pi^l) beta: the low modes keep their normal part; scale by a_F; write
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      const float bn = lanes_sum(be[mm] * na);
      if (mm < nl) be[mm] = bn * na;
    }
    if (act) {
      const int64_t sA = (eA * (D + 1) + fA) * NF * D + a;
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) {
        gamU[sA + mm * D] = aF * (al[mm] + be[mm]);
        gamW[sA + mm * D] = aF * ga[mm];
      }
      if (pb != pa) {
        const int64_t sB = (eB * (D + 1) + fB) * NF * D + a;
#pragma unroll
        for (int mm = 0; mm < NF; ++mm) {
          gamU[sB + mm * D] = aF * (al[mm] - be[mm]);
          gamW[sB + mm * D] = aF * ga[mm];
        }
      }
    }
  }
}

}  // namespace hopu
