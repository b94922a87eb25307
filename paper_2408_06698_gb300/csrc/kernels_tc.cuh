// Tensor-core (tcgen05, kind::tf32) kernels of the FP32 tensor-core precision modes.
//
// a1 (E: V_h -> L2) as a batched GEMM: 128 elements per tile are the M = 128 rows, the
// gathered local functionals l[e][s] (facet blocks with the sign sigma, interior block)
// the K-major A operand, the reference change of basis B[r][s] = Dinv[r][s] (N = n_loc
// padded to 16, K = n_loc padded to 8) the K-major B operand; chat = l Dinv^T lands in
// TMEM (lane = element, column = r), each thread reads its element's row, applies the
// contravariant Piola map J / det J and the tile is written back through shared memory
// with coalesced stores.  3xTF32 (three MMAs per K step) or 1xTF32.
#pragma once
#include "kernels.cuh"
#include "tc.cuh"

namespace hopu {

template <int D, int K>
struct V2lTc {
  using S = Shape<D, K>;
  static constexpr int NL = S::nloc;
  static constexpr int KP = (NL + 7) / 8 * 8;    // K padded to the MMA step (8 tf32)
  static constexpr int NP = (NL + 15) / 16 * 16; // N padded (M = 128 needs N % 16 == 0)
  static constexpr int TM = 128;                 // elements per tile = MMA M = TMEM lanes
  static constexpr int THREADS = 256;            // 8 warps: all gather, warp w reads lane quarter w % 4
  static constexpr int SST = NL + 1;             // staging row stride (odd: conflict-free)
  static constexpr size_t A_BYTES = size_t(TM) * KP * 4;
  static constexpr size_t B_BYTES = size_t(NP) * KP * 4;
  static constexpr size_t CODE_BYTES = size_t(TM) * (D + 1) * 4;
  static constexpr uint32_t TCOLS = NP <= 32 ? 32 : NP <= 64 ? 64 : NP <= 128 ? 128 : 256;
  static constexpr size_t SMEM = 2 * A_BYTES + 2 * B_BYTES + CODE_BYTES + 16;
  static constexpr bool OK = SMEM <= 227 * 1024 && NP <= 256 && size_t(TM) * SST * 4 <= A_BYTES;
};

// Error word bit set by tensor-core kernels when a completion wait gave up.
constexpr int kErrTcTimeoutV2l = 1;  // bits of the device error word (DevMesh::err)
constexpr int kErrTcTimeoutVol = 2;

template <int D, int K, bool THREE>
__global__ void __launch_bounds__(256) k_v2l_tc(DevMesh m, const float* __restrict__ dinv, int nlp,
                                                const float* __restrict__ uV, float* __restrict__ uL) {
  using C = V2lTc<D, K>;
  using S = Shape<D, K>;
  constexpr int NL = C::NL, KP = C::KP, NP = C::NP, NF = S::nf, NB = S::nb, NINT = S::nint, GT = S::gt;
  constexpr int TM = C::TM, NT = C::THREADS, NW = NT / 32;
  constexpr uint32_t LBO = 128, SBO = (KP / 4) * 128;
  constexpr int NCH = (NL + 3) / 4;           // column chunks holding data
  constexpr int NCM = (TM / 8) * NCH;         // core matrices of the A tile holding data
  constexpr int GB = 15;                      // core matrices gathered per batch (independent loads)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sAh = smem_raw;
  unsigned char* sAl = smem_raw + C::A_BYTES;
  unsigned char* sBh = smem_raw + 2 * C::A_BYTES;
  unsigned char* sBl = sBh + C::B_BYTES;
  int* sCode = reinterpret_cast<int*>(sBl + C::B_BYTES);        // [TM][D+1]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sCode + TM * (D + 1));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* geoT = m.geoT;
  pdl_trigger();

  // B operand (once per CTA) and the zero padding columns of A
  for (int t = tid; t < NP * KP; t += NT) {
    const int r = t / KP, s = t - r * KP;
    const float v = (r < NL && s < NL) ? dinv[r * nlp + s] : 0.0f;
    float h, l;
    tc::split_tf32(v, h, l, THREE);
    *reinterpret_cast<float*>(sBh + tc::blk_off(r, s, KP)) = h;
    *reinterpret_cast<float*>(sBl + tc::blk_off(r, s, KP)) = l;
  }
  if constexpr (KP > 4 * NCH) {
    for (int t = tid; t < TM * (KP - 4 * NCH); t += NT) {
      const int row = t / (KP - 4 * NCH), s = 4 * NCH + (t - row * (KP - 4 * NCH));
      *reinterpret_cast<float*>(sAh + tc::blk_off(row, s, KP)) = 0.0f;
      *reinterpret_cast<float*>(sAl + tc::blk_off(row, s, KP)) = 0.0f;
    }
  }
  if (warp == 0) tc::tmem_alloc(tslot, C::TCOLS);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  uint32_t phase = 0;
  bool ok = true;
  const int64_t ntiles = (m.E + TM - 1) / TM;
  pdl_wait();
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * TM;
    for (int t = tid; t < TM * (D + 1); t += NT)
      sCode[t] = (e0 + t / (D + 1) < m.E) ? m.efc[e0 * (D + 1) + t] : 0;
    __syncthreads();
    // gather: a warp fills whole core matrices (8 elements x 4 local functionals), lane
    // (r, j) = (lane / 4, lane % 4) -> one conflict-free 128-byte shared-memory store
    const int rr = lane >> 2, jj = lane & 3;
    for (int cm0 = warp * GB; cm0 < NCM; cm0 += NW * GB) {
      float v[GB];
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int cm = cm0 + u;
        v[u] = 0.0f;
        if (cm < NCM) {
          const int g = cm / NCH, c = cm - g * NCH;
          const int row = g * 8 + rr, s = c * 4 + jj;
          const int64_t e = e0 + row;
          if (e < m.E && s < NL) {
            if (s < (D + 1) * NF) {
              const int f = s / NF, mm = s - f * NF;
              const int code = sCode[row * (D + 1) + f];
              const float x = __ldg(uV + (int64_t)(code >> 2) * NF + mm);
              v[u] = (code & 2) ? -x : x;
            } else {
              v[u] = __ldg(uV + m.NF * NF + e * NINT + (s - (D + 1) * NF));
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int cm = cm0 + u;
        if (cm < NCM) {
          const int g = cm / NCH, c = cm - g * NCH;
          const uint32_t off = (uint32_t)((g * (KP / 4) + c) * 128 + lane * 4);
          float h, l;
          tc::split_tf32(v[u], h, l, THREE);
          *reinterpret_cast<float*>(sAh + off) = h;
          if (THREE) *reinterpret_cast<float*>(sAl + off) = l;
        }
      }
    }
    tc::fence_smem_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t aH = tc::smem_u32(sAh), aL = tc::smem_u32(sAl);
      const uint32_t bH = tc::smem_u32(sBh), bL = tc::smem_u32(sBl);
#pragma unroll 1
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint32_t off = ks * 256;
        tc::mma_tf32(tbase, tc::sdesc(aH + off, LBO, SBO), tc::sdesc(bH + off, LBO, SBO), idesc, ks > 0);
        if (THREE) {
          tc::mma_tf32(tbase, tc::sdesc(aH + off, LBO, SBO), tc::sdesc(bL + off, LBO, SBO), idesc, 1);
          tc::mma_tf32(tbase, tc::sdesc(aL + off, LBO, SBO), tc::sdesc(bH + off, LBO, SBO), idesc, 1);
        }
      }
      tc::commit(mbar);
    }
    ok = __syncthreads_and(tc::mbar_wait(mbar, phase, m.tc_wait_limit)) != 0;
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) break;
    // epilogue: warps w and w + 4 share TMEM lane quarter w % 4 (elements 32(w%4)..+31)
    // and split the n_loc outputs of the Piola map; staged with an odd row stride
    {
      const int row = (warp & 3) * 32 + lane;
      float chat[NP];
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16)
        tc::ld16(tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, chat + c0);
      tc::fence_before_sync();
      float* stage = reinterpret_cast<float*>(sAh);  // [TM][SST]; the MMAs reading A are done
      const int64_t e = e0 + row;
      if (e < m.E) {
        const double* gp = geoT + e * GT;  // Pf = J / det J
        float P[D][D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) P[a][b] = float(__ldg(gp + a * D + b));
        constexpr int HALF = (NL + 1) / 2;
        const int lo = (warp >> 2) * HALF, hi = lo + HALF < NL ? lo + HALF : NL;
#pragma unroll
        for (int idx = 0; idx < NL; ++idx) {
          if (idx < lo || idx >= hi) continue;
          const int a = idx / NB, i = idx - a * NB;
          float acc = 0.0f;
#pragma unroll
          for (int b = 0; b < D; ++b) acc = fmaf(P[a][b], chat[b * NB + i], acc);
          stage[row * C::SST + idx] = acc;
        }
      }
    }
    __syncthreads();
    const int64_t nrow = (m.E - e0 < TM) ? (m.E - e0) : TM;
    for (int64_t t = tid; t < nrow * NL; t += NT) {
      const int row = (int)(t / NL), idx = (int)(t - (int64_t)row * NL);
      uL[e0 * NL + t] = reinterpret_cast<const float*>(sAh)[row * C::SST + idx];
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicOr(m.err, kErrTcTimeoutV2l);
    tc::mbar_wait(mbar, phase ^ 1u);  // bounded (full limit): the MMAs in flight drain before TMEM is freed
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, C::TCOLS);
  }
}

// ------------------------------------------------------------------------------------
// a3 + a5 + fused a7 (element part), STAGE wind (w = u), on the tensor cores.
//
// Per CTA, super-chunks of EB = 40 elements, processed in chunks of EC = 8:
//   X (B operand, 96 rows = 8 elements x 12 quantities, K = basis index padded to 24):
//     the coefficients of u_a (3 rows) and of the modal reference gradients
//     d^_c u_a = sum_j (Dm_c u_a)_j phi_j (9 rows, j < dim P^{k-1});
//   GEMM1: D1[q][n] = sum_i phi_i(x_q) X[n][i]   (M = 128 quadrature points, N = 96)
//     -> every thread (one quadrature point) reads u, grad^ u of 4 elements from TMEM,
//        forms W = |det J| J^-1 u, div^ W and f_a = w_q (div^W u_a + W . grad^ u_a);
//   F (A operand, rows (element, a) of the super-chunk, K = quadrature point);
//   GEMM2: D2[(e,a)][i] = sum_q F[(e,a)][q] phi_i(x_q)   (M = 128 rows, 120 used, N = 32);
//   epilogue: facet lift sum_fm TrM[fm][i] gam[e][fm][a], inverse mass 1/|det J|, the
//     contravariant pull-back det J J^-1 and the local functionals D (back-projection),
//     interior rows combined into the V_h output, facet rows to lf with the sign sigma.
// Tables (phi in both operand layouts, hi and lo TF32 parts) arrive by one bulk copy.
template <int D, int K>
struct VolTc {
  using S = Shape<D, K>;
  static constexpr int NB = S::nb, NB1 = cnbasis(D, K - 1), NQ = S::nq, NL = S::nloc;
  static constexpr int KP1 = (NB + 7) / 8 * 8;          // GEMM1 K (basis index)
  static constexpr int QTY = D + D * D;                 // u_a and d^_c u_a
  static constexpr int EC = 8;                          // elements per GEMM1
  static constexpr int N1 = QTY * EC;                   // GEMM1 N
  static constexpr int NCH = 5;                         // chunks per super-chunk
  static constexpr int EB = EC * NCH;                   // elements per GEMM2
  static constexpr int K2 = 128;                        // GEMM2 K (quadrature points)
  static constexpr int N2 = (NB + 15) / 16 * 16;        // GEMM2 N (basis index)
  static constexpr int THREADS = 512;                   // 16 warps: lane quarter w % 4, element group w / 4
  static constexpr int GT = S::gt;
  // bytes
  static constexpr size_t PA = size_t(128) * KP1 * 4;   // phi, GEMM1 A operand (one part)
  static constexpr size_t PB = size_t(N2) * K2 * 4;     // phi, GEMM2 B operand (one part)
  static constexpr size_t TAB = 2 * PA + 2 * PB;        // the bulk-copied table
  static constexpr size_t FB = size_t(128) * K2 * 4;    // F (one part)
  static constexpr size_t XB = size_t(N1) * KP1 * 4;    // X (one part)
  static constexpr size_t O_F = TAB, O_X = O_F + 2 * FB, O_U = O_X + 2 * XB;
  static constexpr size_t O_GEO = O_U + size_t(EC) * NL * 4;
  static constexpr size_t O_WQ = O_GEO + size_t(EB) * GT * 4;
  static constexpr size_t O_DM = O_WQ + 128 * 4;
  static constexpr size_t O_TRM = O_DM + size_t(D) * NB1 * NB * 4;
  static constexpr size_t O_BAR = (O_TRM + size_t(D + 1) * S::nf * NB * 4 + 15) / 16 * 16;
  static constexpr size_t SMEM = O_BAR + 32;
  // the epilogue keeps y in the X region and the pulled-back coefficients in the lo part
  // of F ahead of its last row group (rows 120..127, which must stay zero)
  static constexpr int ZR = D * EB;                      // F rows from ZR on stay zero
  static constexpr bool OK = (NQ <= 128) && N1 <= 256 && ZR <= 120 && ZR % 8 == 0 && SMEM <= 227 * 1024 &&
                             size_t(EB) * NL * 4 <= 2 * XB && size_t(EB) * NL * 4 <= size_t(ZR / 8) * (K2 / 4) * 128;
  static constexpr uint32_t TCOLS = 256;                // D1 at column 0, D2 at column 128
};

template <int D, int K>
__global__ void __launch_bounds__(512, 1) k_volume_tc(DevMesh m, const float* __restrict__ tctab,
                                                      const float* __restrict__ Dm_g, const float* __restrict__ Wq_g,
                                                      const float* __restrict__ TrM_g, const float* __restrict__ Drow_g,
                                                      int nlr, const float* __restrict__ uL,
                                                      const float* __restrict__ gam, float* out, Combine cmb,
                                                      float* __restrict__ lf) {
  using C = VolTc<D, K>;
  using S = Shape<D, K>;
  constexpr int NB = C::NB, NB1 = C::NB1, NL = C::NL, NF = S::nf, NINT = S::nint, GT = C::GT;
  constexpr int KP1 = C::KP1, QTY = C::QTY, EC = C::EC, N1 = C::N1, EB = C::EB, K2 = C::K2, N2 = C::N2;
  constexpr int NT = C::THREADS, NG = (D + 1) * NF * D;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sPAh = smem_raw;
  unsigned char* sPAl = smem_raw + C::PA;
  unsigned char* sPBh = smem_raw + 2 * C::PA;
  unsigned char* sPBl = sPBh + C::PB;
  unsigned char* sFh = smem_raw + C::O_F;
  unsigned char* sFl = sFh + C::FB;
  unsigned char* sXh = smem_raw + C::O_X;
  unsigned char* sXl = sXh + C::XB;
  float* sU = reinterpret_cast<float*>(smem_raw + C::O_U);     // [EC][NL]
  float* sGeo = reinterpret_cast<float*>(smem_raw + C::O_GEO); // [EB][GT]
  float* sWq = reinterpret_cast<float*>(smem_raw + C::O_WQ);   // [128]
  float* sDm = reinterpret_cast<float*>(smem_raw + C::O_DM);   // [D][NB1][NB]
  float* sTrM = reinterpret_cast<float*>(smem_raw + C::O_TRM); // [(D+1) NF][NB]
  uint64_t* mb_tab = reinterpret_cast<uint64_t*>(smem_raw + C::O_BAR);
  uint64_t* mb_mma = mb_tab + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mb_tab + 2);
  float* sY = reinterpret_cast<float*>(sXh);                   // [EB][NL] (epilogue, X is free)
  float* sCh = reinterpret_cast<float*>(sFl);                  // [EB][NL] (epilogue, F is free)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* geoT = m.geoT;
  pdl_trigger();

  if (warp == 0) tc::tmem_alloc(tslot, C::TCOLS);
  if (tid == 0) {
    tc::mbar_init(mb_tab, 1);
    tc::mbar_init(mb_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    tc::mbar_expect_tx(mb_tab, (uint32_t)C::TAB);
    tc::bulk_g2s(smem_raw, tctab, (uint32_t)C::TAB, mb_tab);
  }
  for (int t = tid; t < 128; t += NT) sWq[t] = t < S::nq ? Wq_g[t] : 0.0f;
  for (int t = tid; t < D * NB1 * NB; t += NT) sDm[t] = Dm_g[t];
  for (int t = tid; t < (D + 1) * NF * NB; t += NT) sTrM[t] = TrM_g[t];
  // rows ZR .. 127 of F stay zero
  for (int t = tid; t < (128 - C::ZR) * K2; t += NT) {
    const int row = C::ZR + t / K2, q = t % K2;
    *reinterpret_cast<float*>(sFh + tc::blk_off(row, q, K2)) = 0.0f;
    *reinterpret_cast<float*>(sFl + tc::blk_off(row, q, K2)) = 0.0f;
  }
  bool ok = __syncthreads_and(tc::mbar_wait(mb_tab, 0)) != 0;
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t id1 = tc::idesc_tf32(128, N1), id2 = tc::idesc_tf32(128, N2);
  uint32_t phase = 0;
  const int64_t nsc = (m.E + EB - 1) / EB;
  const int qrow = (warp & 3) * 32 + lane;              // TMEM lane of this thread
  const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;
  pdl_wait();
  for (int64_t sc = blockIdx.x; ok && sc < nsc; sc += gridDim.x) {
    const int64_t e0 = sc * EB;
    for (int t = tid; t < EB * GT; t += NT) {
      const int64_t e = e0 + t / GT;
      sGeo[t] = e < m.E ? float(geoT[e0 * GT + t]) : 0.0f;
    }
#pragma unroll 1
    for (int c = 0; c < C::NCH && ok; ++c) {
      const int64_t ec = e0 + c * EC;
      for (int t = tid; t < EC * NL; t += NT) sU[t] = (ec + t / NL < m.E) ? uL[ec * NL + t] : 0.0f;
      __syncthreads();
      // X rows (element el, quantity qq): qq < D -> u_a, else grad^ of u_a in direction cc
      for (int t = tid; t < N1 * KP1; t += NT) {
        const int n = t / KP1, j = t - n * KP1;
        const int el = n / QTY, qq = n - el * QTY;
        float v = 0.0f;
        if (qq < D) {
          if (j < NB) v = sU[el * NL + qq * NB + j];
        } else if (j < NB1) {
          const int a = (qq - D) / D, cc = (qq - D) - a * D;
          const float* dm = sDm + (cc * NB1 + j) * NB;
          const float* uu = sU + el * NL + a * NB;
          float p[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
          for (int i = 0; i < NB; ++i) p[i & 3] = fmaf(dm[i], uu[i], p[i & 3]);
          v = (p[0] + p[1]) + (p[2] + p[3]);
        }
        float h, l;
        tc::split_tf32(v, h, l, true);
        *reinterpret_cast<float*>(sXh + tc::blk_off(n, j, KP1)) = h;
        *reinterpret_cast<float*>(sXl + tc::blk_off(n, j, KP1)) = l;
      }
      tc::fence_smem_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t SBA = (KP1 / 4) * 128;
        const uint32_t aH = tc::smem_u32(sPAh), aL = tc::smem_u32(sPAl);
        const uint32_t bH = tc::smem_u32(sXh), bL = tc::smem_u32(sXl);
#pragma unroll 1
        for (int ks = 0; ks < KP1 / 8; ++ks) {
          const uint32_t off = ks * 256;
          tc::mma_tf32(tbase, tc::sdesc(aH + off, 128, SBA), tc::sdesc(bH + off, 128, SBA), id1, ks > 0);
          tc::mma_tf32(tbase, tc::sdesc(aH + off, 128, SBA), tc::sdesc(bL + off, 128, SBA), id1, 1);
          tc::mma_tf32(tbase, tc::sdesc(aL + off, 128, SBA), tc::sdesc(bH + off, 128, SBA), id1, 1);
        }
        tc::commit(mb_mma);
      }
      ok = __syncthreads_and(tc::mbar_wait(mb_mma, phase, m.tc_wait_limit)) != 0;
      phase ^= 1u;
      tc::fence_after_sync();
      if (!ok) break;
      // pointwise: quadrature point qrow, elements 4 (warp / 4) .. +3 of the chunk
      const float wq = sWq[qrow];
#pragma unroll 1
      for (int el = (warp >> 2) * (EC / 4); el < (warp >> 2) * (EC / 4) + EC / 4; ++el) {
        float v[16];
        tc::ld16(tbase + tlane + (uint32_t)(el * QTY), v);
        const float* g = sGeo + (c * EC + el) * GT;
        float u[D], G[D][D], W[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          u[a] = v[a];
#pragma unroll
          for (int cc = 0; cc < D; ++cc) G[a][cc] = v[D + a * D + cc];
        }
        float dv = 0.0f;
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
          float s = 0.0f;
#pragma unroll
          for (int b = 0; b < D; ++b) {
            const float Mcb = g[2 * D * D + cc * D + b];
            s = fmaf(Mcb, u[b], s);
            dv = fmaf(Mcb, G[b][cc], dv);
          }
          W[cc] = s;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float f = dv * u[a];
#pragma unroll
          for (int cc = 0; cc < D; ++cc) f = fmaf(W[cc], G[a][cc], f);
          f *= wq;
          float h, l;
          tc::split_tf32(f, h, l, true);
          const int row = (c * EC + el) * D + a;
          *reinterpret_cast<float*>(sFh + tc::blk_off(row, qrow, K2)) = h;
          *reinterpret_cast<float*>(sFl + tc::blk_off(row, qrow, K2)) = l;
        }
      }
      tc::fence_before_sync();
      __syncthreads();
    }
    if (!ok) break;
    // GEMM2: D2[(e,a)][i] = sum_q F[(e,a)][q] phi_i(x_q)
    tc::fence_smem_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      constexpr uint32_t SB2 = (K2 / 4) * 128;
      const uint32_t aH = tc::smem_u32(sFh), aL = tc::smem_u32(sFl);
      const uint32_t bH = tc::smem_u32(sPBh), bL = tc::smem_u32(sPBl);
#pragma unroll 1
      for (int ks = 0; ks < K2 / 8; ++ks) {
        const uint32_t off = ks * 256;
        tc::mma_tf32(tbase + 128, tc::sdesc(aH + off, 128, SB2), tc::sdesc(bH + off, 128, SB2), id2, ks > 0);
        tc::mma_tf32(tbase + 128, tc::sdesc(aH + off, 128, SB2), tc::sdesc(bL + off, 128, SB2), id2, 1);
        tc::mma_tf32(tbase + 128, tc::sdesc(aL + off, 128, SB2), tc::sdesc(bH + off, 128, SB2), id2, 1);
      }
      tc::commit(mb_mma);
    }
    ok = __syncthreads_and(tc::mbar_wait(mb_mma, phase, m.tc_wait_limit)) != 0;
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) break;
    // epilogue 1: row (e, a) = qrow; warps w and w + 4 split the basis index range
    {
      float r[N2];
#pragma unroll
      for (int c0 = 0; c0 < N2; c0 += 16) tc::ld16(tbase + tlane + 128u + (uint32_t)c0, r + c0);
      tc::fence_before_sync();
      const int el = qrow / D, a = qrow - el * D;
      const int64_t e = e0 + el;
      if (qrow < D * EB && e < m.E) {
        constexpr int PART = (NB + 3) / 4;
        const int i0 = (warp >> 2) * PART, i1 = i0 + PART < NB ? i0 + PART : NB;
        const float invabs = sGeo[el * GT + 3 * D * D];
        const float* gl = gam + e * NG;
        float gv[(D + 1) * NF];
#pragma unroll
        for (int fm = 0; fm < (D + 1) * NF; ++fm) gv[fm] = __ldg(gl + fm * D + a);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i < i0 || i >= i1) continue;
          float p[4] = {r[i], 0.0f, 0.0f, 0.0f};
#pragma unroll
          for (int fm = 0; fm < (D + 1) * NF; ++fm) p[fm & 3] = fmaf(sTrM[fm * NB + i], gv[fm], p[fm & 3]);
          sY[el * NL + a * NB + i] = ((p[0] + p[1]) + (p[2] + p[3])) * invabs;
        }
      }
    }
    __syncthreads();
    // epilogue 2: chat = det J Jinv y, then ell = D chat, combined into the outputs
    for (int t = tid; t < EB * NL; t += NT) {
      const int el = t / NL, s2 = t - el * NL;
      const int b = s2 / NB, i = s2 - b * NB;
      const float* g = sGeo + el * GT;
      float acc = 0.0f;
#pragma unroll
      for (int a = 0; a < D; ++a) acc = fmaf(g[D * D + b * D + a], sY[el * NL + a * NB + i], acc);
      sCh[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < EB * NL; t += NT) {
      const int el = t / NL, rr = t - el * NL;
      const int64_t e = e0 + el;
      if (e >= m.E) continue;
      const float* drow = Drow_g + rr * nlr;
      const float* ch = sCh + el * NL;
      float p[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int s2 = 0; s2 < NL; ++s2) p[s2 & 3] = fmaf(__ldg(drow + s2), ch[s2], p[s2 & 3]);
      const float v = (p[0] + p[1]) + (p[2] + p[3]);
      if (rr < (D + 1) * NF) {
        const int code = m.efc[e * (D + 1) + rr / NF];
        lf[e * (D + 1) * NF + rr] = (code & 2) ? -v : v;
      } else {
        const int64_t idx = m.NF * NF + e * NINT + (rr - (D + 1) * NF);
        out[idx] = combine_at<float>(cmb, v, idx);
      }
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicOr(m.err, kErrTcTimeoutVol);
    tc::mbar_wait(mb_tab, 0);          // bounded (full limit): the table copy and the MMAs in flight drain
    tc::mbar_wait(mb_mma, phase ^ 1u);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, C::TCOLS);
  }
}

}  // namespace hopu

namespace hopu {

// ------------------------------------------------------------------------------------
// a7 (element part, not dual) on the tensor cores: ell = D (det J Jinv y) per element.
//
// 128 elements per tile are the M = 128 rows and the 128 TMEM lanes.  The tile's L2 blocks
// (contiguous in memory) arrive in shared memory by one bulk copy, issued as soon as the
// previous tile's blocks have been read, so that it lands while that tile's MMAs and
// stores run.  Thread (lane quarter q, warp group g) owns element 32 q + lane and the
// basis indices i = g IPG .. g IPG + IPG - 1: it forms X[(b, i)] = sum_a (det J Jinv)[b][a]
// y[a][i] for every component b from its element's row (odd row stride: conflict-free)
// and its element's geometry (loaded into registers one tile ahead), splits them into
// TF32 parts and writes them into its own TMEM lane, columns g GW + b IPG + t: the A
// operand of the MMA is read from TMEM.  B = D[r][kappa] (N = n_loc padded to 16), hi /
// lo TF32 parts from the host, resident in shared memory.  ell lands in TMEM (lane =
// element, column = functional r) and leaves through a shared staging buffer to coalesced
// stores: facet rows to lf with the sign sigma, interior rows combined into the V_h output
// (the combination inputs of a batch of rows are loaded before any is used).  3xTF32 or
// 1xTF32.
template <int D, int K>
struct L2vTc {
  using S = Shape<D, K>;
  static constexpr int NB = S::nb, NL = S::nloc;
  static constexpr int IPG = l2v_tc_ipg(NB);       // basis indices per warp group
  static constexpr int GW = l2v_tc_gw(D, NB);      // A columns per warp group
  static constexpr int KP = l2v_tc_kp(D, NB);      // K
  static constexpr int NP = l2v_tc_np(NL);         // N
  static constexpr int TM = 128, THREADS = 512;    // 4 warp groups x 4 lane quarters
  static constexpr int SST = NL | 1;               // staging row stride (odd: conflict-free)
  // TMEM columns: accumulator [0, NP), A hi [AH, AH + KP), A lo [AL, AL + KP)
  static constexpr uint32_t AH = (NP + 31) / 32 * 32, AL = AH + (KP + 31) / 32 * 32;
  static constexpr uint32_t TCOLS = AL + KP <= 32 ? 32 : AL + KP <= 64 ? 64 : AL + KP <= 128 ? 128
                                  : AL + KP <= 256 ? 256 : 512;
  static constexpr size_t B_BYTES = size_t(NP) * KP * 4;
  static constexpr size_t Y_BYTES = size_t(TM) * NL * 4;  // one tile of L2 blocks
  static constexpr size_t O_Y = 2 * B_BYTES;
  static constexpr size_t O_ST = O_Y + (Y_BYTES + 15) / 16 * 16;
  static constexpr size_t O_CODE = O_ST + (size_t(TM) * SST * 4 + 15) / 16 * 16;
  static constexpr size_t O_BAR = O_CODE + size_t(TM) * (D + 1) * 4;
  static constexpr size_t SMEM = O_BAR + 32;
  static constexpr bool OK = SMEM <= 227 * 1024 && NP <= 256 && AL + KP <= 512 && (2 * B_BYTES) % 16 == 0 &&
                             Y_BYTES % 16 == 0 && TM * (D + 1) <= THREADS && GW % 4 == 0;
  static constexpr size_t TABLE_FLOATS = 2 * size_t(NP) * KP;  // hi parts, then lo parts
};

constexpr int kErrTcTimeoutL2v = 8;  // device error word bit of k_l2v_tc

template <int D, int K, bool THREE>
__global__ void __launch_bounds__(512, 1) k_l2v_tc(DevMesh m, const float* __restrict__ tab,
                                                   const float* __restrict__ yL, float* __restrict__ lf,
                                                   float* outV, Combine cmb) {
  using C = L2vTc<D, K>;
  using S = Shape<D, K>;
  constexpr int NB = C::NB, NL = C::NL, NF = S::nf, NINT = S::nint, GT = S::gt, DD = D * D;
  constexpr int KP = C::KP, NP = C::NP, IPG = C::IPG, GW = C::GW, TM = C::TM, NT = C::THREADS;
  constexpr int NFL = (D + 1) * NF, SST = C::SST;
  constexpr uint32_t LBO = 128, SBO = (KP / 4) * 128;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sB = smem_raw;                                         // hi parts, then lo parts
  float* sY = reinterpret_cast<float*>(smem_raw + C::O_Y);              // [TM][NL]  this tile's y
  float* stage = reinterpret_cast<float*>(smem_raw + C::O_ST);          // [TM][SST] ell
  int* sCode = reinterpret_cast<int*>(smem_raw + C::O_CODE);            // [TM][D+1]
  uint64_t* mb = reinterpret_cast<uint64_t*>(smem_raw + C::O_BAR);      // table, MMAs, y copy
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mb + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, grp = warp >> 2;  // lane quarter, warp group
  const int el = q * 32 + lane;             // this thread's element (TMEM lane)
  pdl_trigger();

  if (warp == 0) tc::tmem_alloc(tslot, C::TCOLS);
  if (tid == 0) {
    tc::mbar_init(mb, 1);
    tc::mbar_init(mb + 1, 1);
    tc::mbar_init(mb + 2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {  // the constant B operand (written at context creation)
    tc::mbar_expect_tx(mb, (uint32_t)(2 * C::B_BYTES));
    tc::bulk_g2s(sB, tab, (uint32_t)(2 * C::B_BYTES), mb);
  }
  const uint32_t tbase = *tslot;
  const uint32_t tquad = tbase + ((uint32_t)(q * 32) << 16);
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  const int64_t ntiles = (m.E + TM - 1) / TM;
  const double* geoT = m.geoT;
  double pg[DD];  // (det J Jinv)[b][a] of this thread's element, one tile ahead
  int code = 0;   // facet code tid of the tile, one tile ahead
  auto load_regs = [&](int64_t tile) {
    const int64_t e = tile * TM + el;
#pragma unroll
    for (int t = 0; t < DD; ++t) pg[t] = e < m.E ? __ldg(geoT + e * GT + DD + t) : 0.0;
    if (tid < TM * (D + 1))
      code = (tile * TM + tid / (D + 1) < m.E) ? __ldg(m.efc + tile * TM * (D + 1) + tid) : 0;
  };
  bool ypend = false;  // a bulk copy of y is in flight
  uint32_t yph = 0, phase = 0;
  // bring tile's y into sY: one bulk copy for a full tile, plain loads for the ragged tail
  // (the caller synchronises before sY is read)
  auto fetch_y = [&](int64_t tile) {
    const int64_t e0 = tile * TM;
    if (e0 + TM <= m.E) {
      if (tid == 0) {
        tc::mbar_expect_tx(mb + 2, (uint32_t)C::Y_BYTES);
        tc::bulk_g2s(sY, yL + e0 * NL, (uint32_t)C::Y_BYTES, mb + 2);
      }
      ypend = true;
    } else {
      for (int64_t t = tid; t < (m.E - e0) * NL; t += NT) sY[t] = yL[e0 * NL + t];
    }
  };
  bool ok = __syncthreads_and(tc::mbar_wait(mb, 0)) != 0;
  pdl_wait();
  int64_t tile = blockIdx.x;
  if (tile < ntiles) {
    load_regs(tile);
    fetch_y(tile);
    __syncthreads();
  }
  for (; ok && tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * TM;
    const int nrow = (m.E - e0 < TM) ? (int)(m.E - e0) : TM;
    if (ypend) {  // this tile's bulk copy
      ok = __syncthreads_and(tc::mbar_wait(mb + 2, yph)) != 0;
      yph ^= 1u;
      ypend = false;
      if (!ok) break;
    }
    // A: X for this thread's element and basis indices, TF32 parts into its TMEM lane
    {
      float xh[GW], xl[GW];
      const float* y = sY + el * NL;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        float P[D];
#pragma unroll
        for (int a = 0; a < D; ++a) P[a] = float(pg[b * D + a]);
#pragma unroll
        for (int t = 0; t < IPG; ++t) {
          const int i = grp * IPG + t;
          float x = 0.0f;
          if (el < nrow && i < NB) {
#pragma unroll
            for (int a = 0; a < D; ++a) x = fmaf(P[a], y[a * NB + i], x);
          }
          tc::split_tf32(x, xh[b * IPG + t], xl[b * IPG + t], THREE);
        }
      }
#pragma unroll
      for (int t = D * IPG; t < GW; ++t) xh[t] = xl[t] = 0.0f;
      tc::tmem_st_cols<GW>(tquad + C::AH + (uint32_t)(grp * GW), xh);
      if (THREE) tc::tmem_st_cols<GW>(tquad + C::AL + (uint32_t)(grp * GW), xl);
      tc::tmem_st_wait();
    }
    if (tid < TM * (D + 1)) sCode[tid] = code;
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t bH = tc::smem_u32(sB), bL = bH + (uint32_t)C::B_BYTES;
#pragma unroll 1
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint32_t off = ks * 256;
        const uint32_t aH = tbase + C::AH + 8 * ks, aL = tbase + C::AL + 8 * ks;
        tc::mma_tf32_ts(tbase, aH, tc::sdesc(bH + off, LBO, SBO), idesc, ks > 0);
        if (THREE) {
          tc::mma_tf32_ts(tbase, aH, tc::sdesc(bL + off, LBO, SBO), idesc, 1);
          tc::mma_tf32_ts(tbase, aL, tc::sdesc(bH + off, LBO, SBO), idesc, 1);
        }
      }
      tc::commit(mb + 1);
    }
    // the next tile's y (sY has been read) and registers, in flight while the MMAs run
    const int64_t nxt = tile + gridDim.x;
    if (nxt < ntiles) {
      load_regs(nxt);
      fetch_y(nxt);
    }
    ok = __syncthreads_and(tc::mbar_wait(mb + 1, phase, m.tc_wait_limit)) != 0;
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) break;
    // TMEM -> staging: warp (q, g) reads lane quarter q, column groups g, g + 4, ...
#pragma unroll 1
    for (int c0 = grp * 16; c0 < NP; c0 += 64) {
      float v[16];
      tc::ld16(tquad + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < NL) stage[el * SST + c0 + j] = v[j];
    }
    tc::fence_before_sync();
    __syncthreads();
    for (int t = tid; t < nrow * NFL; t += NT) {
      const int r = t / NFL, f = t - r * NFL;
      const float v = stage[r * SST + f];
      lf[e0 * NFL + t] = (sCode[r * (D + 1) + f / NF] & 2) ? -v : v;
    }
    if constexpr (NINT > 0) {
      constexpr int NB8 = 6;  // rows per thread and batch
      const float* x0 = static_cast<const float*>(cmb.x0);
      const float* x1 = static_cast<const float*>(cmb.x1);
      const int64_t base = (int64_t)m.NF * NF + e0 * NINT;
      for (int t0 = tid; t0 < nrow * NINT; t0 += NB8 * NT) {
        float xa[NB8], xb[NB8];
#pragma unroll
        for (int u = 0; u < NB8; ++u) {
          const int t = t0 + u * NT;
          const bool in = t < nrow * NINT;
          xa[u] = (in && x0) ? x0[base + t] : 0.0f;
          xb[u] = (in && x1) ? x1[base + t] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < NB8; ++u) {
          const int t = t0 + u * NT;
          if (t < nrow * NINT) {
            const int r = t / NINT, ii = t - r * NINT;
            outV[base + t] = combine_f32(cmb, stage[r * SST + NFL + ii], xa[u], xb[u]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicOr(m.err, kErrTcTimeoutL2v);
    tc::mbar_wait(mb, 0);                 // bounded (full limit): the table copy lands before exit,
    if (ypend) tc::mbar_wait(mb + 2, yph);  // so does a y copy in flight,
    tc::mbar_wait(mb + 1, phase ^ 1u);    // and the MMAs in flight drain before TMEM is freed
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, C::TCOLS);
  }
}

}  // namespace hopu
