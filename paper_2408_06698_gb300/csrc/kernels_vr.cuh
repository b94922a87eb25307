// a3 + a5 with the element's data in registers (FP32, STAGE wind w = u): volume term, facet
// lift and inverse mass.
//
// A warp takes ELW = 32 / D elements and a lane owns one (element, component a) pair: the
// coefficients c of u_a, its modal reference gradients G_c = Dm_c c (c < D, dim P^{k-1}
// entries each) and the accumulators r of its test integrals stay in registers for the whole
// element.  The quadrature points are walked in the same order by every lane, so the basis
// row phi(x_q) is one broadcast shared-memory load for the whole warp; per point a lane forms
//   u_a = sum_i phi_i c_i,   d^_c u_a = sum_j phi_j G_c[j],
// its shares M[c][a] u_a of W_c = sum_b M[c][b] u_b (M = |det J| J^-1, so W = |det J| J^-1 u)
// and sum_c M[c][a] d^_c u_a of div^ W, sums them over the D lanes of its element with
// shuffles, and adds f_a = w_q (div^W u_a + W . grad^ u_a) phi_i to r_i (the element-wise
// integration by parts of the conservative form, as the other volume kernels).  The facet
// lift sum_fm TrM[fm][i] gam[e][fm][a] and 1/|det J| follow; the outputs leave through a
// per-warp staging buffer with coalesced stores.  Compared with one warp per element (lanes
// on quadrature points, coefficient rows read from shared memory per point) this moves the
// contractions from the shared-memory pipe into registers.
//
// GTAB: the reference gradients at the points come from staged tables of d phi_i / d xhat_c
// instead of the modal gradients G held in registers (d n_{b,k-1} fewer registers, more
// resident warps, d n_b instead of d n_{b,k-1} FMAs per point); 6-warp CTAs amortise the
// tables.  The autotuner picks between the two.
//
// FUSE: the element part of the back-projection R E^-1 (a7) follows in the same kernel:
// chat = det J J^-1 y (lane b mixes the element's components from the staging buffer and
// keeps component b in registers), ell = D chat (every lane forms its component's share of
// each row, D staged per CTA, the shares summed by shuffles); interior rows are combined
// into the V_h output, facet rows go to lf with the sign sigma.
#pragma once
#include "kernels.cuh"

namespace hopu {

template <int D, int K, bool GTAB = false>
struct VolR {
  using S = Shape<D, K>;
  static constexpr int NB = S::nb, NB1 = cnbasis(D, K - 1), NF = S::nf, NL = S::nloc, NQ = S::nq, GT = S::gt;
  static constexpr int ELW = 32 / D;                 // elements per warp
  static constexpr int WARPS = GTAB ? 6 : 4;
  static constexpr int NBQ = row_stride<float>(NB);  // Bt rows (point-major, as in global memory)
  static constexpr int NB4 = r4i(NB);                // Dm / TrM rows padded for 16-byte loads
  static constexpr int NG = (D + 1) * NF * D;
  static constexpr int O_DBT = NQ * NBQ;             // GTAB: [D][NQ][NBQ] reference gradients
  static constexpr int O_WQ = O_DBT + (GTAB ? D * NQ * NBQ : 0);
  static constexpr int O_DM = r4i(O_WQ + NQ);
  static constexpr int O_TRM = O_DM + (GTAB ? 0 : D * NB1 * NB4);
  static constexpr int O_W = O_TRM + (D + 1) * NF * NB4;
  static constexpr int PER_WARP = r4i(ELW * NL);     // output staging of the warp's elements
  static constexpr int GW = r4i(ELW * NG);           // the warp's facet moments, staged by cp.async
  static constexpr int O_G = O_W + WARPS * PER_WARP;
  static constexpr size_t SMEM = size_t(O_G + WARPS * GW) * 4;
  static constexpr int NLR = row_stride<float>(NL);  // rows of the row-major D in global memory
  static constexpr int NDP = D * NB4;                // fused back-projection: D [NL][D blocks of NB4]
  static constexpr int O_D = O_G + WARPS * GW;
  static constexpr size_t SMEM_FUSE = size_t(O_D + NL * NDP) * 4;
  static constexpr int REGS = 2 * NB + (GTAB ? 0 : D * NB1);  // c, r (and G) of a lane
  static constexpr int MINB = GTAB ? 2 : (REGS <= 100 ? 3 : 2);  // resident CTAs asked of the register allocator
  static constexpr bool OK = REGS <= 140 && SMEM <= 200 * 1024;
  static constexpr bool FUSE_OK = OK && SMEM_FUSE <= 200 * 1024;
};

template <int D, int K, bool FUSE, bool GTAB>
__global__ void __launch_bounds__(32 * VolR<D, K, GTAB>::WARPS, VolR<D, K, GTAB>::MINB)
    k_volume_r(DevMesh m, DevTabs tb, const float* __restrict__ uL, const float* __restrict__ gam, float* out,
               Combine cmb, float* __restrict__ lf) {
  using C = VolR<D, K, GTAB>;
  using S = Shape<D, K>;
  constexpr int NB = C::NB, NB1 = C::NB1, NF = C::NF, NL = C::NL, NQ = C::NQ, GT = C::GT;
  constexpr int NBQ = C::NBQ, NB4 = C::NB4, NG = C::NG, ELW = C::ELW;
  extern __shared__ __align__(16) float sm[];
  pdl_trigger();
  {
    const float* Btg = static_cast<const float*>(tb.Bt);
    const float* Wqg = static_cast<const float*>(tb.Wq);
    const float* Dmg = static_cast<const float*>(tb.Dm);
    const float* TrMg = static_cast<const float*>(tb.TrM);
    for (int t = threadIdx.x; t < NQ * NBQ; t += blockDim.x) sm[t] = Btg[t];
    if (GTAB) {
      const float* dBtg = static_cast<const float*>(tb.dBt);
      for (int t = threadIdx.x; t < D * NQ * NBQ; t += blockDim.x) sm[C::O_DBT + t] = dBtg[t];
    }
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) sm[C::O_WQ + t] = Wqg[t];
    for (int t = threadIdx.x; t < (GTAB ? 0 : D * NB1 * NB4); t += blockDim.x) {
      const int row = t / NB4, i = t - row * NB4;
      sm[C::O_DM + t] = i < NB ? Dmg[row * NB + i] : 0.0f;
    }
    for (int t = threadIdx.x; t < (D + 1) * NF * NB4; t += blockDim.x) {
      const int row = t / NB4, i = t - row * NB4;
      sm[C::O_TRM + t] = i < NB ? TrMg[row * NB + i] : 0.0f;
    }
    if (FUSE) {  // row rr, component block b: D[rr][b*nb + i] at rr*NDP + b*NB4 + i (16-byte rows)
      const float* Dg = static_cast<const float*>(tb.Drow);
      for (int t = threadIdx.x; t < NL * C::NDP; t += blockDim.x) {
        const int rr = t / C::NDP, col = t - rr * C::NDP, b = col / NB4, i = col - b * NB4;
        sm[C::O_D + t] = i < NB ? Dg[rr * C::NLR + b * NB + i] : 0.0f;
      }
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
  // the other lanes of the element (idle lanes talk to themselves)
  const int p1 = lane_on ? el * D + (a + 1) % D : lane;
  const int p2 = lane_on ? el * D + (a + 2) % D : lane;
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
    float c[NB];
    {
      const float* up = uL + e * NL + a * NB;
#pragma unroll
      for (int i = 0; i < NB; ++i) c[i] = __ldg(up + i);
    }
    const double* gp = m.geoT + e * GT;
    float Mcol[D];  // column a of M = |det J| J^-1
#pragma unroll
    for (int cc = 0; cc < D; ++cc) Mcol[cc] = float(__ldg(gp + 2 * D * D + cc * D + a));
    const float invabs = float(__ldg(gp + 3 * D * D));
    // modal reference gradients of u_a: G[cc][j] = sum_i Dm[cc][j][i] c_i (not with GTAB)
    constexpr int NG1 = GTAB ? 1 : NB1;
    float G[D][NG1];
    if constexpr (!GTAB) {
#pragma unroll
      for (int cc = 0; cc < D; ++cc)
#pragma unroll
        for (int j = 0; j < NG1; ++j) {
          const float* drow = sDm + (cc * NB1 + j) * NB4;
          float p0 = 0.0f, p1s = 0.0f;
#pragma unroll
          for (int i = 0; i < NB; i += 4) {
            float dv[4];
            lds_v(drow + i, dv);
#pragma unroll
            for (int w = 0; w < 4; ++w)
              if (i + w < NB) {
                if (w & 1) p1s = fmaf(dv[w], c[i + w], p1s);
                else p0 = fmaf(dv[w], c[i + w], p0);
              }
          }
          G[cc][j] = p0 + p1s;
        }
    }
    float r[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) r[i] = 0.0f;
    // u_a and the reference gradient of u_a at point q
    auto point_values = [&](int q, float& u, float (&gd)[D]) {
      const float* ph = sBt + q * NBQ;
      float u0 = 0.0f, u1 = 0.0f;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) gd[cc] = 0.0f;
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
          if constexpr (!GTAB) {
            if (idx < NB1) {
#pragma unroll
              for (int cc = 0; cc < D; ++cc) gd[cc] = fmaf(pv[w], G[cc][idx < NG1 ? idx : 0], gd[cc]);
            }
          }
        }
      }
      if constexpr (GTAB) {  // d^_c u_a = sum_i (d phi_i / d xhat_c)(x_q) c_i
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
          const float* dph = sm + C::O_DBT + (cc * NQ + q) * NBQ;
          float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
          for (int i = 0; i < NB; i += 4) {
            float pv[4];
            lds_v(dph + i, pv);
#pragma unroll
            for (int w = 0; w < 4; ++w)
              if (i + w < NB) {
                if (w & 1) s1 = fmaf(pv[w], c[i + w], s1);
                else s0 = fmaf(pv[w], c[i + w], s0);
              }
          }
          gd[cc] = s0 + s1;
        }
      }
      u = u0 + u1;
    };
    // two points per pass: the loads and shuffles of one overlap the arithmetic of the other
    // (an odd last point is paired with itself at weight 0)
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
      // sums over the element's D lanes: W_c = sum_b M[c][b] u_b, div^ W = sum_b sum_c M[c][b] d^_c u_b
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
    // facet lift of component a: r_i += sum_fm TrM[fm][i] gam[e][fm][a]
    cp_wait<0>();
    __syncwarp();
    {
      const float* gl = sG + el * NG + a;
#pragma unroll 4
      for (int fm = 0; fm < (D + 1) * NF; ++fm) {
        const float gv = gl[fm * D];
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
    // inverse mass, then coalesced stores of the warp's element records
    if (act) {
#pragma unroll
      for (int i = 0; i < NB; ++i) sY[(el * D + a) * NB + i] = r[i] * invabs;
    }
    __syncwarp();
    if constexpr (!FUSE) {
      for (int t = lane; t < ne * NL; t += 32) {
        const int64_t idx = e0 * NL + t;
        out[idx] = combine_at<float>(cmb, sY[t], idx);
      }
    } else {
      // chat[b][i] = sum_c Pi[b][c] y[c][i], Pi = det J J^-1 (lane b of the element), kept in
      // registers; row rr of ell = D chat is the sum over the element's lanes of
      // sum_i D[rr][b*nb + i] chat[b][i], reduced by shuffles and written by lane rr / nb
      float Pi[D];
#pragma unroll
      for (int cc = 0; cc < D; ++cc) Pi[cc] = float(__ldg(gp + D * D + a * D + cc));
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int cc = 0; cc < D; ++cc) acc = fmaf(Pi[cc], sY[el * NL + cc * NB + i], acc);
        r[i] = acc;
      }
      const float* sD = sm + C::O_D + a * NB4;
      const int* codes = m.efc + e * (D + 1);
#pragma unroll 1
      for (int rr = 0; rr < NL; ++rr) {
        const float* drow = sD + rr * C::NDP;
        float p0 = 0.0f, p1s = 0.0f;
#pragma unroll
        for (int i = 0; i < NB; i += 4) {
          float dv[4];
          lds_v(drow + i, dv);
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (i + w < NB) {
              if (w & 1) p1s = fmaf(dv[w], r[i + w], p1s);
              else p0 = fmaf(dv[w], r[i + w], p0);
            }
        }
        const float part = p0 + p1s;
        float v = part + __shfl_sync(kFull, part, p1);
        if (D == 3) v += __shfl_sync(kFull, part, p2);
        if (act && rr / NB == a) {
          if (rr < (D + 1) * NF) {
            lf[e * (D + 1) * NF + rr] = (__ldg(codes + rr / NF) & 2) ? -v : v;
          } else {
            const int64_t idx = m.NF * NF + e * S::nint + (rr - (D + 1) * NF);
            out[idx] = combine_at<float>(cmb, v, idx);
          }
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace hopu
