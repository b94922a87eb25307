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
// FUSE: the element part of the back-projection R E^-1 (a7) follows in the same kernel:
// chat = det J J^-1 y (lane b mixes the element's components from the staging buffer and
// keeps component b in registers), ell = D chat (every lane forms its component's share of
// each row, D staged per CTA, the shares summed by shuffles); interior rows are combined
// into the V_h output, facet rows go to lf with the sign sigma.
#pragma once
#include "kernels.cuh"

namespace hopu {

template <int D, int K>
struct VolR {
  using S = Shape<D, K>;
  static constexpr int NB = S::nb, NB1 = cnbasis(D, K - 1), NF = S::nf, NL = S::nloc, NQ = S::nq, GT = S::gt;
  static constexpr int ELW = 32 / D;                 // elements per warp
  static constexpr int WARPS = 4;
  static constexpr int NBQ = row_stride<float>(NB);  // Bt rows (point-major, as in global memory)
  static constexpr int NB4 = r4i(NB);                // Dm / TrM rows padded for 16-byte loads
  static constexpr int NG = (D + 1) * NF * D;
  static constexpr int O_WQ = NQ * NBQ;
  static constexpr int O_DM = r4i(O_WQ + NQ);
  static constexpr int O_TRM = O_DM + D * NB1 * NB4;
  static constexpr int O_W = O_TRM + (D + 1) * NF * NB4;
  static constexpr int PER_WARP = r4i(ELW * NL);     // output staging of the warp's elements
  static constexpr size_t SMEM = size_t(O_W + WARPS * PER_WARP) * 4;
  static constexpr int NLR = row_stride<float>(NL);  // rows of the row-major D in global memory
  static constexpr int NDP = D * NB4;                // fused back-projection: D [NL][D blocks of NB4]
  static constexpr int O_D = O_W + WARPS * PER_WARP;
  static constexpr size_t SMEM_FUSE = size_t(O_D + NL * NDP) * 4;
  static constexpr int REGS = 2 * NB + D * NB1;      // c, r and G of a lane
  static constexpr int MINB = REGS <= 100 ? 3 : 2;   // resident CTAs asked of the register allocator
  static constexpr bool OK = REGS <= 140 && SMEM <= 200 * 1024;
  static constexpr bool FUSE_OK = OK && SMEM_FUSE <= 200 * 1024;
};

template <int D, int K, bool FUSE>
__global__ void __launch_bounds__(32 * VolR<D, K>::WARPS, VolR<D, K>::MINB)
    k_volume_r(DevMesh m, DevTabs tb, const float* __restrict__ uL, const float* __restrict__ gam, float* out,
               Combine cmb, float* __restrict__ lf) {
  using C = VolR<D, K>;
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
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) sm[C::O_WQ + t] = Wqg[t];
    for (int t = threadIdx.x; t < D * NB1 * NB4; t += blockDim.x) {
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
  const int64_t ngroups = (m.E + ELW - 1) / ELW;
  for (int64_t grp = (int64_t)warp * gridDim.x + blockIdx.x; grp < ngroups; grp += (int64_t)gridDim.x * C::WARPS) {
    const int64_t e0 = grp * ELW;
    const int ne = (m.E - e0 < ELW) ? (int)(m.E - e0) : ELW;
    const bool act = lane_on && el < ne;
    const int64_t e = act ? e0 + el : e0;  // inactive lanes read the group's first element
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
    // modal reference gradients of u_a: G[cc][j] = sum_i Dm[cc][j][i] c_i
    float G[D][NB1];
#pragma unroll
    for (int cc = 0; cc < D; ++cc)
#pragma unroll
      for (int j = 0; j < NB1; ++j) {
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
    float r[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) r[i] = 0.0f;
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      const float* ph = sBt + q * NBQ;
      float u0 = 0.0f, u1 = 0.0f, gd[D];
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
          if (idx < NB1) {
#pragma unroll
            for (int cc = 0; cc < D; ++cc) gd[cc] = fmaf(pv[w], G[cc][idx], gd[cc]);
          }
        }
      }
      const float u = u0 + u1;
      float W[D], pd = 0.0f;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) pd = fmaf(Mcol[cc], gd[cc], pd);
      // sums over the element's D lanes: W_c = sum_b M[c][b] u_b, div^ W = sum_b sum_c M[c][b] d^_c u_b
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        const float pw = Mcol[cc] * u;
        float s = pw + __shfl_sync(kFull, pw, p1);
        if (D == 3) s += __shfl_sync(kFull, pw, p2);
        W[cc] = s;
      }
      float dv = pd + __shfl_sync(kFull, pd, p1);
      if (D == 3) dv += __shfl_sync(kFull, pd, p2);
      float f = dv * u;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) f = fmaf(W[cc], gd[cc], f);
      f *= sWq[q];
#pragma unroll
      for (int i = 0; i < NB; i += 4) {
        float pv[4];
        lds_v(ph + i, pv);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (i + w < NB) r[i + w] = fmaf(f, pv[w], r[i + w]);
      }
    }
    // facet lift of component a: r_i += sum_fm TrM[fm][i] gam[e][fm][a]
    {
      const float* gl = gam + e * NG + a;
#pragma unroll 2
      for (int fm = 0; fm < (D + 1) * NF; ++fm) {
        const float gv = __ldg(gl + fm * D);
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
