// a4 with the facet's data in registers (FP32): the facet flux moments of the HOPU form.
//
// A warp takes FPW = 32 / D facets and a lane owns one (facet, component a) pair.  Per facet
// mode m (the orthonormal facet basis psi_m) the lane forms its component of both sides'
// modal traces tau^X_m = sum_i TrM_{f_X}[m][i] c^X_a[i] from the coefficients it holds in
// registers (the degree <= 1 terms compensated, as in k_facet), the jump J_m = tau^A - tau^B
// and the averaged wind <w>_m; the facet's lanes sum J_m . n and <w>_m . n by shuffles, which
// gives (I - Pi^l) J in modal form (modes below dim P^l(F) keep only (J_m . n) n).  The facet
// quadrature points are then walked in the same order by every lane (broadcast rows of psi
// and of w_q psi), with w.n, J and (I - Pi^l) J at the point, h = 1/2 |w.n| (I - Pi^l) J and
// -1/2 (w.n) J accumulated into the moments alpha_m and beta_m in registers; beta's low modes
// keep their normal part ((I - Pi^l) h), both are scaled by a_F and written element-major as
// in k_facet (alpha + beta for side A, alpha - beta for side B).  Boundary facets (fb == fa)
// write side A only; inlet facets take side B's trace of u from the given data and keep the
// wind's own trace.  Compared with a warp per facet (phases exchanged through shared memory)
// this keeps the modal vectors and the moments in registers.
#pragma once
#include "kernels.cuh"

namespace hopu {

template <int D, int K>
struct FacR {
  using S = Shape<D, K>;
  static constexpr int NB = S::nb, NF = S::nf, NL = S::nloc, NQF = S::nqf;
  static constexpr int FPW = 32 / D;     // facets per warp
  static constexpr int WARPS = 4;
  static constexpr int NB4 = r4i(NB), NF4 = r4i(NF);
  static constexpr int O_TRM = 0;                                // [(D+1) NF][NB4]
  static constexpr int O_PSI = O_TRM + (D + 1) * NF * NB4;       // [NQF][NF4]   psi_m(s_q)
  static constexpr int O_WPSI = O_PSI + NQF * NF4;               // [NQF][NF4]   w_q psi_m(s_q)
  static constexpr int O_WF = O_WPSI + NQF * NF4;                // [NQF]
  static constexpr size_t SMEM = size_t(O_WF + r4i(NQF)) * 4;
  static constexpr int REGS = 2 * NB + 5 * NF;                   // coefficients, then the modal vectors
  static constexpr bool OK = REGS <= 230;
  static constexpr bool OK_WSEP = REGS <= 110;  // with a separate wind the w coefficients add 2 nb registers
  static constexpr int MINB = REGS <= 110 ? 3 : 2;
};

template <int D, int K, bool WSEP>
__global__ void __launch_bounds__(32 * FacR<D, K>::WARPS, FacR<D, K>::MINB)
    k_facet_r(DevMesh m, DevTabs tb, const float* __restrict__ uL, const float* __restrict__ wL, int lconst,
              const int8_t* __restrict__ facet_l, float* __restrict__ gam, double* __restrict__ diss) {
  using C = FacR<D, K>;
  constexpr int NB = C::NB, NF = C::NF, NL = C::NL, NQF = C::NQF, NB4 = C::NB4, NF4 = C::NF4, FPW = C::FPW;
  extern __shared__ __align__(16) float sm[];
  pdl_trigger();
  {
    const float* TrMg = static_cast<const float*>(tb.TrM);
    const float* Psig = static_cast<const float*>(tb.Psi);    // [NF][NQF]
    const float* WPsig = static_cast<const float*>(tb.WPsi);  // [NF][NQF]
    const float* Wfg = static_cast<const float*>(tb.Wf);
    for (int t = threadIdx.x; t < (D + 1) * NF * NB4; t += blockDim.x) {
      const int row = t / NB4, i = t - row * NB4;
      sm[C::O_TRM + t] = i < NB ? TrMg[row * NB + i] : 0.0f;
    }
    for (int t = threadIdx.x; t < NQF * NF4; t += blockDim.x) {
      const int q = t / NF4, mm = t - q * NF4;
      sm[C::O_PSI + t] = mm < NF ? Psig[mm * NQF + q] : 0.0f;
      sm[C::O_WPSI + t] = mm < NF ? WPsig[mm * NQF + q] : 0.0f;
    }
    for (int t = threadIdx.x; t < NQF; t += blockDim.x) sm[C::O_WF + t] = Wfg[t];
  }
  const float* sTrM = sm + C::O_TRM;
  const float* sPsi = sm + C::O_PSI;
  const float* sWPsi = sm + C::O_WPSI;
  const float* sWf = sm + C::O_WF;
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
    const float na = (a == 0) ? n[0] : (a == 1 ? n[1] : n[D - 1]);  // this lane's component of n
    const int l = facet_l ? int(facet_l[F]) : lconst;
    const int nl = (l < 0) ? 0 : cnbasis(D - 1, l);
    const int inl = m.inlet ? m.inlet[F] : -1;
    const float* ext = inl >= 0 ? static_cast<const float*>(m.inlet_modes) + (int64_t)inl * NF * D : nullptr;
    // modal traces of component a: jump J and averaged wind Wv
    // modes in groups of MG (a rolled loop: the unrolled trace phase of every mode did not
    // fit the instruction cache beside the point loop); J and Wv stay in registers, moving
    // down by MG after every group and taking the new group at their end
    constexpr int MG = 5, NGRP = (NF + MG - 1) / MG, NFP = NGRP * MG;
    float J[NFP], Wv[NFP];
#pragma unroll
    for (int t = 0; t < NFP; ++t) J[t] = Wv[t] = 0.0f;
    {
      float cA[NB], cB[NB];
      const float* ua = uL + eA * NL + a * NB;
      const float* ub = uL + eB * NL + a * NB;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        cA[i] = __ldg(ua + i);
        cB[i] = __ldg(ub + i);
      }
      const float* trA = sTrM + fA * NF * NB4;
      const float* trB = sTrM + fB * NF * NB4;
#pragma unroll 1
      for (int g5 = 0; g5 < NGRP; ++g5) {
        float J5[MG], W5[MG];
#pragma unroll
        for (int t = 0; t < MG; ++t) {
          const int mm = g5 * MG + t;
          const int mr = mm < NF ? mm : NF - 1;
          float sa = 0.0f, ca = 0.0f, pa_ = 0.0f, sb = 0.0f, cb = 0.0f, pb_ = 0.0f;
#pragma unroll
          for (int i = 0; i < NB; i += 4) {
            float ta[4], tbv[4];
            lds_v(trA + mr * NB4 + i, ta);
            lds_v(trB + mr * NB4 + i, tbv);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const int idx = i + w;
              if (idx < D + 1) {
                dot2_step(sa, ca, ta[w], cA[idx]);
                dot2_step(sb, cb, tbv[w], cB[idx]);
              } else if (idx < NB) {
                pa_ = fmaf(ta[w], cA[idx], pa_);
                pb_ = fmaf(tbv[w], cB[idx], pb_);
              }
            }
          }
          ca = __fadd_rn(ca, pa_);
          cb = __fadd_rn(cb, pb_);
          if (ext) {
            sb = ext[mr * D + a];
            cb = 0.0f;
          }
          const float ta_ = __fadd_rn(sa, ca), tb_ = __fadd_rn(sb, cb);
          J5[t] = mm < NF ? __fadd_rn(__fsub_rn(sa, sb), __fsub_rn(ca, cb)) : 0.0f;
          W5[t] = mm < NF ? (ext ? ta_ : 0.5f * (ta_ + tb_)) : 0.0f;  // an inlet keeps the wind's own trace
        }
#pragma unroll
        for (int t = 0; t + MG < NFP; ++t) {
          J[t] = J[t + MG];
          Wv[t] = Wv[t + MG];
        }
#pragma unroll
        for (int t = 0; t < MG; ++t) {
          J[NFP - MG + t] = J5[t];
          Wv[NFP - MG + t] = W5[t];
        }
      }
    }
    if (WSEP) {  // the wind's traces from its own coefficients
      float wA[NB], wB[NB];
      const float* wa = wL + eA * NL + a * NB;
      const float* wb = wL + eB * NL + a * NB;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        wA[i] = __ldg(wa + i);
        wB[i] = __ldg(wb + i);
      }
      const float* trA = sTrM + fA * NF * NB4;
      const float* trB = sTrM + fB * NF * NB4;
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int i = 0; i < NB; i += 4) {
          float ta[4], tbv[4];
          lds_v(trA + mm * NB4 + i, ta);
          lds_v(trB + mm * NB4 + i, tbv);
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (i + w < NB) {
              s0 = fmaf(ta[w], wA[i + w], s0);
              s1 = fmaf(tbv[w], wB[i + w], s1);
            }
        }
        Wv[mm] = ext ? s0 : 0.5f * (s0 + s1);
      }
    }
    // normal components over the facet's lanes: wvn_m = <w>_m . n, and (I - Pi^l) J in modal
    // form (Pj: modes below nl keep only (J_m . n) n)
    float Pj[NF];
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      const float jn = lanes_sum(J[mm] * na);
      Wv[mm] = lanes_sum(Wv[mm] * na);  // now <w>_m . n
      Pj[mm] = (mm < nl) ? jn * na : J[mm];
    }
    // facet quadrature points: moments alpha (central) and beta (upwind part)
    float al[NF], be[NF];
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) al[mm] = be[mm] = 0.0f;
    float dsum = 0.0f;
#pragma unroll 1
    for (int q = 0; q < NQF; ++q) {
      const float* ps = sPsi + q * NF4;
      float jq = 0.0f, pq = 0.0f, wn = 0.0f;
#pragma unroll
      for (int mm = 0; mm < NF; mm += 4) {
        float pv[4];
        lds_v(ps + mm, pv);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (mm + w < NF) {
            jq = fmaf(pv[w], J[mm + w], jq);
            pq = fmaf(pv[w], Pj[mm + w], pq);
            wn = fmaf(pv[w], Wv[mm + w], wn);
          }
      }
      const float aw = 0.5f * fabsf(wn);
      const float h = aw * pq, cq = -0.5f * wn * jq;
      dsum = fmaf(sWf[q] * aw, pq * pq, dsum);
      const float* wp = sWPsi + q * NF4;
#pragma unroll
      for (int mm = 0; mm < NF; mm += 4) {
        float wv[4];
        lds_v(wp + mm, wv);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (mm + w < NF) {
            al[mm + w] = fmaf(wv[w], cq, al[mm + w]);
            be[mm + w] = fmaf(wv[w], h, be[mm + w]);
          }
      }
    }
    // (I - Pi^l) h: the low modes of beta keep their normal part; scale by a_F; write
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      const float bn = lanes_sum(be[mm] * na);
      if (mm < nl) be[mm] = bn * na;
    }
    if (act) {
      float* gA = gam + (eA * (D + 1) + fA) * NF * D + a;
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) gA[mm * D] = aF * (al[mm] + be[mm]);
      if (pb != pa) {
        float* gB = gam + (eB * (D + 1) + fB) * NF * D + a;
#pragma unroll
        for (int mm = 0; mm < NF; ++mm) gB[mm * D] = aF * (al[mm] - be[mm]);
      }
    }
    if (diss) {
      const float tot = lanes_sum(dsum);
      if (act && a == 0) diss[F] = double(aF) * double(tot);
    }
  }
}

}  // namespace hopu
