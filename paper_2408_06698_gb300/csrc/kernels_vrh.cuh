// a3 + a5 with the element's data in registers, the basis split over two lanes (FP32,
// STAGE wind w = u): volume term, facet lift and inverse mass.
//
// The structure of k_volume_r (a lane per (element, component a), the quadrature points
// walked in the same order by every lane, broadcast basis rows, W and div^ W summed over
// the element's lanes by shuffles, f_a = w_q (div^W u_a + W . grad^ u_a) tested against
// phi_i), with each (element, component) pair on two lanes: half h owns the basis indices
// i = 2 t + h (coefficients c_i, test accumulators r_i) and the modal gradient entries
// G_c[j], j = 2 t + h < dim P^{k-1}.  Per point a lane forms its half's partial sums of u_a
// and d^_c u_a, and one shuffle with the other half completes them; both halves then hold
// the same f_a and accumulate their own r_i.  The tables are staged with their basis columns
// permuted so that each half reads one contiguous block of a row (half h at column offset
// h HP).  Half the registers per lane of k_volume_r: twice the resident warps at k = 4, and
// a register kernel at all at k = 5 (where a whole basis does not fit in one lane).
#pragma once
#include "kernels.cuh"

namespace hopu {

template <int D, int K>
struct VolRH {
  using S = Shape<D, K>;
  static constexpr int NB = S::nb, NB1 = cnbasis(D, K - 1), NF = S::nf, NL = S::nloc, NQ = S::nq, GT = S::gt;
  static constexpr int LPE = 2 * D;               // lanes per element: (component, half)
  static constexpr int ELW = 32 / LPE;            // elements per warp
  static constexpr int WARPS = 8;
  static constexpr int NH = (NB + 1) / 2;         // basis indices of half 0 (half 1: NB - NH)
  static constexpr int NH1 = (NB1 + 1) / 2;       // modal-gradient indices of half 0
  static constexpr int HP = r4i(NH);              // one half's block of a permuted row
  static constexpr int RW = 2 * HP;               // permuted row width
  static constexpr int NBQ = (RW / 4) % 2 == 0 ? RW + 4 : RW;  // Bt row stride: an odd multiple of 16 bytes
  static constexpr int NG = (D + 1) * NF * D;
  static constexpr int O_WQ = NQ * NBQ;           // Bt [NQ][NBQ], permuted columns
  static constexpr int O_DM = r4i(O_WQ + NQ);     // Dm [D][NB1][RW], permuted columns
  static constexpr int O_TRM = O_DM + D * NB1 * RW;   // TrM [(D+1) NF][RW], permuted columns
  static constexpr int O_W = O_TRM + (D + 1) * NF * RW;
  static constexpr int PER_WARP = r4i(ELW * NL);  // output staging of the warp's elements
  static constexpr int GW = r4i(ELW * NG);        // the warp's facet moments, staged by cp.async
  static constexpr int O_G = O_W + WARPS * PER_WARP;
  static constexpr size_t SMEM = size_t(O_G + WARPS * GW) * 4;
  static constexpr int REGS = 2 * NH + D * NH1;   // c, r and G of a lane
  static constexpr int MINB = 2 * SMEM <= 200 * 1024 ? 2 : 1;
  static constexpr bool OK = REGS <= 128 && SMEM <= 200 * 1024 && NB >= 2;
  // permuted column of basis index i
  static constexpr __host__ __device__ int col(int i) { return (i & 1) * HP + (i >> 1); }
};

template <int D, int K>
__global__ void __launch_bounds__(32 * VolRH<D, K>::WARPS, VolRH<D, K>::MINB)
    k_volume_rh(DevMesh m, DevTabs tb, const float* __restrict__ uL, const float* __restrict__ gam, float* out,
                Combine cmb) {
  using C = VolRH<D, K>;
  constexpr int NB = C::NB, NB1 = C::NB1, NF = C::NF, NL = C::NL, NQ = C::NQ, GT = C::GT;
  constexpr int NBQ = C::NBQ, HP = C::HP, RW = C::RW, NG = C::NG, ELW = C::ELW, LPE = C::LPE;
  constexpr int NH = C::NH, NH1 = C::NH1;
  extern __shared__ __align__(16) float sm[];
  pdl_trigger();
  {  // tables with permuted basis columns (zero padding)
    const float* Btg = static_cast<const float*>(tb.Bt);
    const float* Wqg = static_cast<const float*>(tb.Wq);
    const float* Dmg = static_cast<const float*>(tb.Dm);
    const float* TrMg = static_cast<const float*>(tb.TrM);
    constexpr int NBQG = row_stride<float>(NB);  // Bt rows in global memory
    for (int t = threadIdx.x; t < NQ * NBQ; t += blockDim.x) {
      const int q = t / NBQ, p = t - q * NBQ, h = p / HP, i = 2 * (p - h * HP) + h;
      sm[t] = (p < RW && i < NB) ? Btg[q * NBQG + i] : 0.0f;
    }
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) sm[C::O_WQ + t] = Wqg[t];
    for (int t = threadIdx.x; t < D * NB1 * RW; t += blockDim.x) {
      const int row = t / RW, p = t - row * RW, h = p / HP, i = 2 * (p - h * HP) + h;
      sm[C::O_DM + t] = i < NB ? Dmg[row * NB + i] : 0.0f;
    }
    for (int t = threadIdx.x; t < (D + 1) * NF * RW; t += blockDim.x) {
      const int row = t / RW, p = t - row * RW, h = p / HP, i = 2 * (p - h * HP) + h;
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
  const bool lane_on = lane < LPE * ELW;
  const int el = lane_on ? lane / LPE : 0;
  const int rr = lane_on ? lane - el * LPE : 0;
  const int a = rr >> 1, h = rr & 1;
  const int nh = h ? NB - NH : NH;          // this half's basis indices
  const int nh1 = h ? NB1 - NH1 : NH1;      // and modal-gradient indices
  const int pt = lane ^ 1;                  // the other half of this (element, component)
  // the other components' lanes of the same half (idle lanes talk to themselves)
  const int p1 = lane_on ? el * LPE + ((a + 1) % D) * 2 + h : lane;
  const int p2 = lane_on ? el * LPE + ((a + 2) % D) * 2 + h : lane;
  float* sY = sm + C::O_W + warp * C::PER_WARP;
  float* sG = sm + C::O_G + warp * C::GW;
  const int64_t ngroups = (m.E + ELW - 1) / ELW;
  for (int64_t grp = (int64_t)warp * gridDim.x + blockIdx.x; grp < ngroups; grp += (int64_t)gridDim.x * C::WARPS) {
    const int64_t e0 = grp * ELW;
    const int ne = (m.E - e0 < ELW) ? (int)(m.E - e0) : ELW;
    const bool act = lane_on && el < ne;
    const int64_t e = act ? e0 + el : e0;  // inactive lanes read the group's first element
    // the group's facet moments arrive in shared memory while the points are walked
    for (int k2 = 0; k2 < ne; ++k2) warp_copy_async<NG * 4>(sG + k2 * NG, gam + (e0 + k2) * NG, lane);
    cp_commit();
    // this half's coefficients c[t] = c_a[2 t + h] (zero beyond the half)
    float c[NH];
    {
      const float* up = uL + e * NL + a * NB + h;
#pragma unroll
      for (int t = 0; t < NH; ++t) c[t] = (t < nh) ? __ldg(up + 2 * t) : 0.0f;
    }
    const double* gp = m.geoT + e * GT;
    float Mcol[D];  // column a of M = |det J| J^-1
#pragma unroll
    for (int cc = 0; cc < D; ++cc) Mcol[cc] = float(__ldg(gp + 2 * D * D + cc * D + a));
    const float invabs = float(__ldg(gp + 3 * D * D));
    // this half's modal gradient entries G[cc][t1] = sum_i Dm[cc][2 t1 + h][i] c_i, with the
    // other half's coefficients taken once from the partner lane
    float G[D][NH1];
    {
      float co[NH];
#pragma unroll
      for (int t = 0; t < NH; ++t) co[t] = __shfl_sync(kFull, c[t], pt);
#pragma unroll
      for (int cc = 0; cc < D; ++cc)
#pragma unroll
        for (int t1 = 0; t1 < NH1; ++t1) {
          const int j = 2 * t1 + h;
          const float* drow = sDm + (cc * NB1 + (j < NB1 ? j : 0)) * RW;
          const float* mine = drow + h * HP;
          const float* other = drow + (1 - h) * HP;
          float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
          for (int t = 0; t < NH; t += 4) {
            float dv[4], ov[4];
            lds_v(mine + t, dv);
            lds_v(other + t, ov);
#pragma unroll
            for (int w = 0; w < 4; ++w)
              if (t + w < NH) {
                s0 = fmaf(dv[w], c[t + w], s0);
                s1 = fmaf(ov[w], co[t + w], s1);
              }
          }
          G[cc][t1] = (t1 < nh1) ? s0 + s1 : 0.0f;
        }
    }
    float r[NH];
#pragma unroll
    for (int t = 0; t < NH; ++t) r[t] = 0.0f;
    // u_a and the reference gradient of u_a at point q: this half's partial sums, completed
    // by one shuffle each with the other half
    auto point_values = [&](int q, float& u, float (&gd)[D]) {
      const float* ph = sBt + q * NBQ + h * HP;
      float u0 = 0.0f, u1 = 0.0f;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) gd[cc] = 0.0f;
#pragma unroll
      for (int t = 0; t < NH; t += 4) {
        float pv[4];
        lds_v(ph + t, pv);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int idx = t + w;
          if (idx < NH) {
            if (w & 1) u1 = fmaf(pv[w], c[idx], u1);
            else u0 = fmaf(pv[w], c[idx], u0);
          }
          if (idx < NH1) {
#pragma unroll
            for (int cc = 0; cc < D; ++cc) gd[cc] = fmaf(pv[w], G[cc][idx < NH1 ? idx : 0], gd[cc]);
          }
        }
      }
      const float up = u0 + u1;
      u = up + __shfl_sync(kFull, up, pt);
#pragma unroll
      for (int cc = 0; cc < D; ++cc) gd[cc] += __shfl_sync(kFull, gd[cc], pt);
    };
    // two points per pass (an odd last point is paired with itself at weight 0)
#pragma unroll 1
    for (int q = 0; q < NQ; q += 2) {
      const bool two = q + 1 < NQ;
      const int qb = two ? q + 1 : q;
      float ua, ub, ga[D], gb[D];
      point_values(q, ua, ga);
      point_values(qb, ub, gb);
      float pda = 0.0f, pdb = 0.0f, pwa[D], pwb[D];
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        pda = fmaf(Mcol[cc], ga[cc], pda);
        pdb = fmaf(Mcol[cc], gb[cc], pdb);
        pwa[cc] = Mcol[cc] * ua;
        pwb[cc] = Mcol[cc] * ub;
      }
      // sums over the element's components (lanes of the same half): W_c and div^ W
      float Wa[D], Wb[D];
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        Wa[cc] = pwa[cc] + __shfl_sync(kFull, pwa[cc], p1);
        Wb[cc] = pwb[cc] + __shfl_sync(kFull, pwb[cc], p1);
        if (D == 3) {
          Wa[cc] += __shfl_sync(kFull, pwa[cc], p2);
          Wb[cc] += __shfl_sync(kFull, pwb[cc], p2);
        }
      }
      float dva = pda + __shfl_sync(kFull, pda, p1), dvb = pdb + __shfl_sync(kFull, pdb, p1);
      if (D == 3) {
        dva += __shfl_sync(kFull, pda, p2);
        dvb += __shfl_sync(kFull, pdb, p2);
      }
      float fa = dva * ua, fb = dvb * ub;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        fa = fmaf(Wa[cc], ga[cc], fa);
        fb = fmaf(Wb[cc], gb[cc], fb);
      }
      fa *= sWq[q];
      fb *= two ? sWq[qb] : 0.0f;
      const float* pha = sBt + q * NBQ + h * HP;
      const float* phb = sBt + qb * NBQ + h * HP;
#pragma unroll
      for (int t = 0; t < NH; t += 4) {
        float va[4], vb[4];
        lds_v(pha + t, va);
        lds_v(phb + t, vb);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (t + w < NH) r[t + w] = fmaf(fb, vb[w], fmaf(fa, va[w], r[t + w]));
      }
    }
    // facet lift of component a, this half: r_t += sum_fm TrM[fm][2 t + h] gam[e][fm][a]
    cp_wait<0>();
    __syncwarp();
    {
      const float* gl = sG + el * NG + a;
#pragma unroll 4
      for (int fm = 0; fm < (D + 1) * NF; ++fm) {
        const float gv = gl[fm * D];
        const float* trow = sTrM + fm * RW + h * HP;
#pragma unroll
        for (int t = 0; t < NH; t += 4) {
          float tv[4];
          lds_v(trow + t, tv);
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (t + w < NH) r[t + w] = fmaf(tv[w], gv, r[t + w]);
        }
      }
    }
    // inverse mass, then coalesced stores of the warp's element records
    if (act) {
#pragma unroll
      for (int t = 0; t < NH; ++t)
        if (t < nh) sY[(el * D + a) * NB + 2 * t + h] = r[t] * invabs;
    }
    __syncwarp();
    for (int t = lane; t < ne * NL; t += 32) {
      const int64_t idx = e0 * NL + t;
      out[idx] = combine_at<float>(cmb, sY[t], idx);
    }
    __syncwarp();
  }
}

}  // namespace hopu
