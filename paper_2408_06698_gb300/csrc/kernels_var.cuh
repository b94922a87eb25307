// The volume part of the adjoint (VJP) of the STAGE apply (w = u), FP32, with the element's
// data in registers: the layout of k_volume_r applied to the transposed form.
//
// For the cotangent ybar of y = M^-1 c(u; u, .) the volume part of ubar is, with
// z = ybar / |det J| (the inverse mass moved onto the cotangent) and W = M u
// (M = |det J| J^-1),
//   ubar_a[i] = - sum_q w_q ( W . grad^ z_a + sum_c M[c][a] sum_b u_b d^_c z_b ) phi_i(x_q),
// the first term the derivative through the convected field, the second through the wind
// (both summed into ubar when w = u); the lift of the facet moments of the adjoint facet
// kernel, sum_fm TrM[fm][i] (gamU + gamW)[e][fm][a], follows.  A lane owns one (element,
// component a) pair: the coefficients c of u_a, the modal gradients G_c = Dm_c z_a of its
// cotangent and the test accumulators r in registers; the quadrature points are walked in
// the same order by every lane (broadcast basis rows), W_c and sum_b u_b d^_c z_b are summed
// over the element's lanes by shuffles.  Same arithmetic as k_volume_adj, whose lanes sit on
// quadrature points and whose element vectors are read from shared memory per point.
#pragma once
#include "kernels.cuh"
#include "kernels_vr.cuh"

namespace hopu {

template <int D, int K>
struct VolAR {
  using V = VolR<D, K>;
  static constexpr int NB = V::NB, NB1 = V::NB1, NF = V::NF, NL = V::NL, NQ = V::NQ;
  static constexpr int ELW = V::ELW, WARPS = 4, NBQ = V::NBQ, NB4 = V::NB4, NG = V::NG;
  static constexpr int O_WQ = NQ * NBQ;
  static constexpr int O_DM = r4i(O_WQ + NQ);
  static constexpr int O_TRM = O_DM + D * NB1 * NB4;
  static constexpr int O_W = O_TRM + (D + 1) * NF * NB4;
  static constexpr int PER_WARP = r4i(ELW * NL);   // output staging
  static constexpr int GW = r4i(ELW * NG);         // one moment array of the warp's elements
  static constexpr int O_G = O_W + WARPS * PER_WARP;  // gamU, then gamW, per warp
  static constexpr size_t SMEM = size_t(O_G + WARPS * 2 * GW) * 4;
  static constexpr int MINB = V::MINB;
  static constexpr bool OK = V::OK && SMEM <= 200 * 1024;
};

template <int D, int K>
__global__ void __launch_bounds__(32 * VolAR<D, K>::WARPS, VolAR<D, K>::MINB)
    k_volume_adj_r(DevMesh m, DevTabs tb, const float* __restrict__ uL, const float* __restrict__ ybar,
                   const float* __restrict__ gamU, const float* __restrict__ gamW, float* __restrict__ ubar) {
  using C = VolAR<D, K>;
  constexpr int NB = C::NB, NB1 = C::NB1, NF = C::NF, NL = C::NL, NQ = C::NQ, GT = Shape<D, K>::gt;
  constexpr int NBQ = C::NBQ, NB4 = C::NB4, NG = C::NG, ELW = C::ELW;
  extern __shared__ __align__(16) float sm[];
  pdl_trigger();
  {
    const float* Btg = static_cast<const float*>(tb.Bt);
    const float* Wqg = static_cast<const float*>(tb.Wq);
    const float* Dmg = static_cast<const float*>(tb.Dm);
    const float* TrMg = static_cast<const float*>(tb.TrM);
    for (int t = threadIdx.x; t < NQ * NBQ; t += blockDim.x) sm[t] = Btg[t];
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) sm[C::O_WQ + t] = Wqg[t];
    for (int t = threadIdx.x; t < D * NB1 * NB4; t += blockDim.x) {
      const int row = t / NB4, i = t - row * NB4;
      sm[C::O_DM + t] = i < NB ? Dmg[row * NB + i] : 0.0f;
    }
    for (int t = threadIdx.x; t < (D + 1) * NF * NB4; t += blockDim.x) {
      const int row = t / NB4, i = t - row * NB4;
      sm[C::O_TRM + t] = i < NB ? TrMg[row * NB + i] : 0.0f;
    }
  }
  const float* sBt = sm;
  const float* sWq = sm + C::O_WQ;
  const float* sDm = sm + C::O_DM;
  const float* sTrM = sm + C::O_TRM;
  pdl_wait();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool lane_on = lane < D * ELW;
  const int el = lane_on ? lane / D : 0;
  const int a = lane_on ? lane - el * D : 0;
  const int p1 = lane_on ? el * D + (a + 1) % D : lane;
  const int p2 = lane_on ? el * D + (a + 2) % D : lane;
  float* sY = sm + C::O_W + warp * C::PER_WARP;
  float* sGU = sm + C::O_G + warp * 2 * C::GW;
  float* sGW = sGU + C::GW;
  const int64_t ngroups = (m.E + ELW - 1) / ELW;
  for (int64_t grp = (int64_t)warp * gridDim.x + blockIdx.x; grp < ngroups; grp += (int64_t)gridDim.x * C::WARPS) {
    const int64_t e0 = grp * ELW;
    const int ne = (m.E - e0 < ELW) ? (int)(m.E - e0) : ELW;
    const bool act = lane_on && el < ne;
    const int64_t e = act ? e0 + el : e0;  // inactive lanes read the group's first element
    // the group's adjoint facet moments arrive while the points are walked
    for (int k2 = 0; k2 < ne; ++k2) {
      warp_copy_async<NG * 4>(sGU + k2 * NG, gamU + (e0 + k2) * NG, lane);
      warp_copy_async<NG * 4>(sGW + k2 * NG, gamW + (e0 + k2) * NG, lane);
    }
    cp_commit();
    const double* gp = m.geoT + e * GT;
    float Mcol[D];  // column a of M = |det J| J^-1
#pragma unroll
    for (int cc = 0; cc < D; ++cc) Mcol[cc] = float(__ldg(gp + 2 * D * D + cc * D + a));
    const float invabs = float(__ldg(gp + 3 * D * D));
    float c[NB];
    {
      const float* up = uL + e * NL + a * NB;
#pragma unroll
      for (int i = 0; i < NB; ++i) c[i] = __ldg(up + i);
    }
    // modal reference gradients of z_a = ybar_a / |det J|: G[cc][j] = sum_i Dm[cc][j][i] z_i
    float G[D][NB1];
    {
      float z[NB];
      const float* yp = ybar + e * NL + a * NB;
#pragma unroll
      for (int i = 0; i < NB; ++i) z[i] = __ldg(yp + i) * invabs;
#pragma unroll
      for (int cc = 0; cc < D; ++cc)
#pragma unroll
        for (int j = 0; j < NB1; ++j) {
          const float* drow = sDm + (cc * NB1 + j) * NB4;
          float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
          for (int i = 0; i < NB; i += 4) {
            float dv[4];
            lds_v(drow + i, dv);
#pragma unroll
            for (int w = 0; w < 4; ++w)
              if (i + w < NB) {
                if (w & 1) s1 = fmaf(dv[w], z[i + w], s1);
                else s0 = fmaf(dv[w], z[i + w], s0);
              }
          }
          G[cc][j] = s0 + s1;
        }
    }
    float r[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) r[i] = 0.0f;
    // u_a and the reference gradient of z_a at point q
    auto point_values = [&](int q, float& u, float (&gz)[D]) {
      const float* ph = sBt + q * NBQ;
      float u0 = 0.0f, u1 = 0.0f;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) gz[cc] = 0.0f;
#pragma unroll
      for (int i = 0; i < NB; i += 4) {
        float pv[4];
        lds_v(ph + i, pv);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int idx = i + w;
          if (idx < NB) {
            if (w & 1) u1 = fmaf(pv[w], c[idx], u1);
            else u0 = fmaf(pv[w], c[idx], u0);
          }
          if (idx < NB1) {
#pragma unroll
            for (int cc = 0; cc < D; ++cc) gz[cc] = fmaf(pv[w], G[cc][idx < NB1 ? idx : 0], gz[cc]);
          }
        }
      }
      u = u0 + u1;
    };
    auto lanes_sum = [&](float v) {
      float s = v + __shfl_sync(kFull, v, p1);
      if (D == 3) s += __shfl_sync(kFull, v, p2);
      return s;
    };
    // two points per pass (an odd last point is paired with itself at weight 0)
#pragma unroll 1
    for (int q = 0; q < NQ; q += 2) {
      const bool two = q + 1 < NQ;
      const int qb = two ? q + 1 : q;
      float ua, ub, ga[D], gb[D];
      point_values(q, ua, ga);
      point_values(qb, ub, gb);
      // W_c = sum_b M[c][b] u_b and ug_c = sum_b u_b d^_c z_b over the element's lanes
      float Wa[D], Wb[D], Ua[D], Ub[D];
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        Wa[cc] = lanes_sum(Mcol[cc] * ua);
        Wb[cc] = lanes_sum(Mcol[cc] * ub);
        Ua[cc] = lanes_sum(ua * ga[cc]);
        Ub[cc] = lanes_sum(ub * gb[cc]);
      }
      float fa = 0.0f, fb = 0.0f;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        fa = fmaf(Wa[cc], ga[cc], fmaf(Mcol[cc], Ua[cc], fa));
        fb = fmaf(Wb[cc], gb[cc], fmaf(Mcol[cc], Ub[cc], fb));
      }
      fa *= -sWq[q];
      fb *= two ? -sWq[qb] : 0.0f;
      const float* pha = sBt + q * NBQ;
      const float* phb = sBt + qb * NBQ;
#pragma unroll
      for (int i = 0; i < NB; i += 4) {
        float va[4], vb[4];
        lds_v(pha + i, va);
        lds_v(phb + i, vb);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (i + w < NB) r[i + w] = fmaf(fb, vb[w], fmaf(fa, va[w], r[i + w]));
      }
    }
    // lift of the adjoint facet moments of component a (both cotangents, w = u)
    cp_wait<0>();
    __syncwarp();
    {
      const float* gu = sGU + el * NG + a;
      const float* gw = sGW + el * NG + a;
#pragma unroll 4
      for (int fm = 0; fm < (D + 1) * NF; ++fm) {
        const float gv = gu[fm * D] + gw[fm * D];
        const float* trow = sTrM + fm * NB4;
#pragma unroll
        for (int i = 0; i < NB; i += 4) {
          float tv[4];
          lds_v(trow + i, tv);
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (i + w < NB) r[i + w] = fmaf(tv[w], gv, r[i + w]);
        }
      }
    }
    if (act) {
#pragma unroll
      for (int i = 0; i < NB; ++i) sY[(el * D + a) * NB + i] = r[i];
    }
    __syncwarp();
    for (int t = lane; t < ne * NL; t += 32) ubar[e0 * NL + t] = sY[t];
    __syncwarp();
  }
}

}  // namespace hopu
