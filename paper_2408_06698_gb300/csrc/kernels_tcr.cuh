// a1 (E: V_h -> L2) in HOPU_FP32_TC: the refined FP32 projection of k_v2l with its two
// dense products on the tensor cores (tcgen05, kind::tf32).
//
// Per tile of 128 elements (the MMA rows, one TMEM lane each), thread (lane quarter q,
// warp group g) owns element 32 q + lane and the rows h = g + 4 j of the dof matrix D in
// the sorted CSR order (every group gets every fourth row of a list sorted by length:
// balanced residual work):
//   X  = its element's local functionals l[s_h] (facet blocks with the sign sigma, interior
//        block), gathered into registers one tile ahead (the loads fly during the previous
//        tile's residual) and kept exactly for the residual; their TF32 parts go to the
//        thread's TMEM lane, columns g GW + j: the A operand read from TMEM;
//   Y0 = X Dinv^T in TMEM (3xTF32; B = Dinv with its K columns in the same order, hi / lo
//        parts from the host, resident in shared memory);
//   R  = X - D Y0 on the CUDA cores in compensated FP32 (Dot2; the reference change of
//        basis is ill-conditioned on the high-degree modes, which a plain FP32 or 3xTF32
//        product loses): Y0 staged in shared memory (odd row stride), the CSR rows of D in
//        shared memory (every lane of a warp reads the same entry), the sum D Y0 formed
//        from zero and X entering last by TwoSum; rows whose component blocks are equal
//        (the facet with the normal of equal components) are stored once and contracted
//        with S_i = sum_b Y0[b nb + i], formed per element as an exact pair by TwoSum;
//   Y  = Y0 + R Dinv^T: a second 3xTF32 MMA with R in TMEM in X's columns into a second
//        accumulator, added to the staged Y0 in FP32 (one rounding: accumulating the small
//        correction onto Y0 inside the tensor core would round Y at every MMA);
//   uL = the contravariant Piola map J / det J of Y, through shared memory to coalesced
//        stores.
// The result has the accuracy of k_v2l's refined projection (the residual decides it).
#pragma once
#include "kernels.cuh"
#include "kernels_tc.cuh"
#include "tc.cuh"

namespace hopu {

template <int D, int K>
struct V2lTcr {
  using S = Shape<D, K>;
  static constexpr int NL = S::nloc;
  static constexpr int RPG = v2l_tc_rpg(NL);          // CSR rows per warp group
  static constexpr int GW = v2l_tc_gw(NL);            // A columns per warp group
  static constexpr int KP = v2l_tc_kp(NL);            // K
  static constexpr int NP = (NL + 15) / 16 * 16;      // N (basis index; M = 128 needs N % 16 == 0)
  static constexpr int TM = 128, THREADS = 512;
  static constexpr int SST = NL | 1;                  // staging row stride (odd: conflict-free)
  static constexpr int GPT = (TM * D * D + THREADS - 1) / THREADS;  // geometry values per thread
  // TMEM columns: Y0 [0, NP), A hi [AH, AH + KP), A lo [AL, AL + KP), correction [DC, DC + NP)
  static constexpr uint32_t AH = (NP + 31) / 32 * 32, AL = AH + (KP + 31) / 32 * 32;
  static constexpr uint32_t DC = AL + (KP + 31) / 32 * 32, TEND = DC + NP;
  static constexpr uint32_t TCOLS = TEND <= 32 ? 32 : TEND <= 64 ? 64 : TEND <= 128 ? 128 : TEND <= 256 ? 256 : 512;
  static constexpr size_t B_BYTES = size_t(NP) * KP * 4;
  static constexpr size_t O_ST = 2 * B_BYTES;
  static constexpr size_t O_CODE = O_ST + (size_t(TM) * SST * 4 + 15) / 16 * 16;
  static constexpr size_t O_GEO = O_CODE + size_t(TM) * (D + 1) * 4;
  static constexpr int NB = S::nb;
  static constexpr int SS = 2 * NB + 1;               // S pairs row stride (odd: conflict-free)
  static constexpr int IPG = (NB + 3) / 4;            // S entries formed per thread
  static constexpr size_t O_S = O_GEO + (size_t(TM) * D * D * 4 + 15) / 16 * 16;
  static constexpr size_t O_BAR = O_S + (size_t(TM) * SS * 4 + 15) / 16 * 16;
  static constexpr size_t O_CSR = O_BAR + 32;         // the CSR of D (csr_n 16-byte entries) last
  static constexpr size_t smem(int csr_n) { return O_CSR + size_t(csr_n) * 16; }
  static constexpr bool OK = smem(NL) <= 227 * 1024 && NP <= 256 && TEND <= 512 && (2 * B_BYTES) % 16 == 0 &&
                             TM * (D + 1) <= THREADS && GW % 4 == 0;
  static constexpr size_t TABLE_FLOATS = 2 * size_t(NP) * KP;  // hi parts, then lo parts
};

template <int D, int K>
__global__ void __launch_bounds__(512, 1) k_v2l_tcr(DevMesh m, const float* __restrict__ tab,
                                                    const float4* __restrict__ csr, int csr_n,
                                                    const float* __restrict__ uV, float* __restrict__ uL) {
  using C = V2lTcr<D, K>;
  using S = Shape<D, K>;
  constexpr int NL = C::NL, KP = C::KP, NP = C::NP, NF = S::nf, NB = S::nb, NINT = S::nint, GT = S::gt;
  constexpr int TM = C::TM, NT = C::THREADS, DD = D * D, NFL = (D + 1) * NF, SST = C::SST;
  constexpr int RPG = C::RPG, GW = C::GW, GPT = C::GPT;
  constexpr uint32_t LBO = 128, SBO = (KP / 4) * 128;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sB = smem_raw;                                       // hi parts, then lo parts
  float* stage = reinterpret_cast<float*>(smem_raw + C::O_ST);        // [TM][SST]  Y0, then Y
  int* sCode = reinterpret_cast<int*>(smem_raw + C::O_CODE);          // [TM][D+1]  next tile's codes
  float* sGeo = reinterpret_cast<float*>(smem_raw + C::O_GEO);        // [TM][D*D]  Pf = J / det J
  float* sS = reinterpret_cast<float*>(smem_raw + C::O_S);            // [TM][SS]   S_i (hi, lo)
  uint64_t* mb = reinterpret_cast<uint64_t*>(smem_raw + C::O_BAR);    // [0] tables, [1] MMAs
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mb + 2);
  float4* sCsr = reinterpret_cast<float4*>(smem_raw + C::O_CSR);
  const int4* hdr = reinterpret_cast<const int4*>(sCsr);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, grp = warp >> 2;
  const int el = q * 32 + lane;  // this thread's element (TMEM lane)
  pdl_trigger();

  if (warp == 0) tc::tmem_alloc(tslot, C::TCOLS);
  if (tid == 0) {
    tc::mbar_init(mb, 1);
    tc::mbar_init(mb + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {  // the constant tables (written at context creation): B, then the CSR of D
    tc::mbar_expect_tx(mb, (uint32_t)(2 * C::B_BYTES + size_t(csr_n) * 16));
    tc::bulk_g2s(sB, tab, (uint32_t)(2 * C::B_BYTES), mb);
    tc::bulk_g2s(sCsr, csr, (uint32_t)(size_t(csr_n) * 16), mb);
  }
  const uint32_t tbase = *tslot;
  const uint32_t tquad = tbase + ((uint32_t)(q * 32) << 16);
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  const int64_t ntiles = (m.E + TM - 1) / TM;
  const double* geoT = m.geoT;
  bool ok = __syncthreads_and(tc::mbar_wait(mb, 0)) != 0;
  uint32_t phase = 0;

  // this thread's functionals l[s_h] of a tile (codes of that tile in sCode), as the raw
  // V_h values and the orientation signs (bit j of *neg): nothing waits for the loads here
  auto gather = [&](int64_t tile, float* x, uint32_t* neg) {
    const int64_t e = tile * TM + el;
    const bool in = e < m.E;
    uint32_t sg = 0;
#pragma unroll
    for (int j = 0; j < RPG; ++j) {
      const int h = grp + 4 * j;
      float v = 0.0f;
      if (in && h < NL) {
        const int s = hdr[h].x;
        if (s < NFL) {
          const int f = s / NF, mm = s - f * NF;
          const int code = sCode[el * (D + 1) + f];
          v = __ldg(uV + (int64_t)(code >> 2) * NF + mm);
          sg |= (uint32_t)((code >> 1) & 1) << j;
        } else {
          v = __ldg(uV + m.NF * NF + e * NINT + (s - NFL));
        }
      }
      x[j] = v;
    }
    *neg = sg;
  };
  static_assert(RPG <= 32, "one sign bit per row");
  auto load_code = [&](int64_t tile) -> int {
    return (tid < TM * (D + 1) && tile * TM + tid / (D + 1) < m.E) ? __ldg(m.efc + tile * TM * (D + 1) + tid) : 0;
  };
  auto load_geo = [&](int64_t tile, double* g) {
#pragma unroll
    for (int u = 0; u < GPT; ++u) {
      const int t = tid + u * NT, r = t / DD, ab = t - r * DD;
      g[u] = (t < TM * DD && tile * TM + r < m.E) ? __ldg(geoT + (tile * TM + r) * GT + ab) : 0.0;
    }
  };
  // accumulator columns [col, col + NP) -> staging rows (add: onto the staged values):
  // warp (q, g) reads lane quarter q, column groups g, g + 4, ...
  auto tmem_to_stage = [&](uint32_t col, bool add) {
#pragma unroll 1
    for (int c0 = grp * 16; c0 < NP; c0 += 64) {
      float v[16];
      tc::ld16(tquad + col + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < NL) stage[el * SST + c0 + j] = add ? __fadd_rn(stage[el * SST + c0 + j], v[j]) : v[j];
    }
  };
  auto mma_3x = [&](uint32_t dcol) {  // D = A(TMEM) B^T in 3xTF32, K steps of 8
    const uint32_t bH = tc::smem_u32(sB), bL = bH + (uint32_t)C::B_BYTES;
#pragma unroll 1
    for (int ks = 0; ks < KP / 8; ++ks) {
      const uint32_t off = ks * 256;
      const uint32_t aH = tbase + C::AH + 8 * ks, aL = tbase + C::AL + 8 * ks;
      tc::mma_tf32_ts(tbase + dcol, aH, tc::sdesc(bH + off, LBO, SBO), idesc, ks > 0 ? 1u : 0u);
      tc::mma_tf32_ts(tbase + dcol, aH, tc::sdesc(bL + off, LBO, SBO), idesc, 1);
      tc::mma_tf32_ts(tbase + dcol, aL, tc::sdesc(bH + off, LBO, SBO), idesc, 1);
    }
    tc::commit(mb + 1);
  };

  float xr[RPG];    // this tile's functionals (exact; raw V_h values until the tile starts)
  uint32_t xneg = 0;  // their orientation signs
  double gr[GPT];   // this tile's geometry, staged into sGeo at the tile start
  pdl_wait();
  int64_t tile = blockIdx.x;
  if (ok && tile < ntiles) {
    const int cd = load_code(tile);
    if (tid < TM * (D + 1)) sCode[tid] = cd;
    load_geo(tile, gr);
    __syncthreads();
    gather(tile, xr, &xneg);
  }
  for (; ok && tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * TM;
    const int nrow = (m.E - e0 < TM) ? (int)(m.E - e0) : TM;
#pragma unroll
    for (int j = 0; j < RPG; ++j)
      if ((xneg >> j) & 1u) xr[j] = -xr[j];
#pragma unroll
    for (int u = 0; u < GPT; ++u)
      if (tid + u * NT < TM * DD) sGeo[tid + u * NT] = float(gr[u]);
    // A = X: TF32 parts of this thread's GW columns
#pragma unroll
    for (int c0 = 0; c0 < GW; c0 += 4) {
      float h4[4], l4[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const float x = (c0 + jj < RPG) ? xr[c0 + jj] : 0.0f;
        tc::split_tf32(x, h4[jj], l4[jj], true);
      }
      tc::tmem_st<4>(tquad + C::AH + (uint32_t)(grp * GW + c0), h4);
      tc::tmem_st<4>(tquad + C::AL + (uint32_t)(grp * GW + c0), l4);
    }
    tc::tmem_st_wait();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {  // Y0 = X Dinv^T
      tc::fence_after_sync();
      mma_3x(0);
    }
    const int64_t nxt = tile + gridDim.x;
    const int cdn = (nxt < ntiles) ? load_code(nxt) : 0;
    if (nxt < ntiles) load_geo(nxt, gr);
    ok = __syncthreads_and(tc::mbar_wait(mb + 1, phase, m.tc_wait_limit)) != 0;
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) break;
    tmem_to_stage(0, false);  // Y0
    if (tid < TM * (D + 1)) sCode[tid] = cdn;
    tc::fence_before_sync();
    __syncthreads();
    // S_i = sum_b Y0[b nb + i] as an exact pair (hi, lo) for the grouped rows: thread (q, g)
    // forms the entries i = g IPG .. of its element
    {
      const float* y = stage + el * SST;
#pragma unroll
      for (int t2 = 0; t2 < C::IPG; ++t2) {
        const int i = grp * C::IPG + t2;
        if (i < NB) {
          float hi = y[i], lo = 0.0f;
#pragma unroll
          for (int b = 1; b < D; ++b) {
            const float v = y[b * NB + i];
            const float t = __fadd_rn(hi, v);
            const float z = __fsub_rn(t, hi);
            lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(v, z)));
            hi = t;
          }
          sS[el * C::SS + 2 * i] = hi;
          sS[el * C::SS + 2 * i + 1] = lo;
        }
      }
    }
    __syncthreads();
    // the next tile's functionals, in flight during the residual
    float xn[RPG];
    uint32_t xnneg = 0;
    if (nxt < ntiles) {
      gather(nxt, xn, &xnneg);
    } else {
#pragma unroll
      for (int j = 0; j < RPG; ++j) xn[j] = 0.0f;
    }
    // R = X - D Y0 (Dot2), TF32 parts into X's TMEM columns, four rows at a time.  Only the
    // four rows of a group are unrolled (the row bodies hold data-dependent loops: unrolling
    // all of them overflows the instruction cache); the group's X values are the first four
    // of the register array, which moves down by four after every group.
    {
      const float* y0 = stage + el * SST;
      const bool in = el < nrow;
#pragma unroll 1
      for (int c0 = 0; c0 < GW; c0 += 4) {
        float h4[4], l4[4], x4[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) x4[jj] = (jj < RPG) ? xr[jj < RPG ? jj : 0] : 0.0f;
#pragma unroll
        for (int j2 = 0; j2 + 4 < RPG; ++j2) xr[j2] = xr[j2 + 4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int j = c0 + jj, h = grp + 4 * j;
          float r = 0.0f;
          if (j < RPG && h < NL) {
            const int4 hd = hdr[h];
            // two interleaved Dot2 chains (even / odd entries) for instruction-level
            // parallelism, joined by TwoSum
            float a = 0.0f, c = 0.0f, a1 = 0.0f, c1 = 0.0f;
            const int kend = hd.y + hd.z;
            int k = hd.y;
            if (hd.w) {  // grouped row: entries (i, T) against the pairs S_i
              const float* sp = sS + el * C::SS;
#pragma unroll 2
              for (; k + 1 < kend; k += 2) {
                const float4 e0 = sCsr[k], e1 = sCsr[k + 1];
                const int i0 = 2 * __float_as_int(e0.x), i1 = 2 * __float_as_int(e1.x);
                const float v0 = sp[i0], w0 = sp[i0 + 1], v1 = sp[i1], w1 = sp[i1 + 1];
                dot2_step(a, c, e0.y, v0);
                dot2_step(a1, c1, e1.y, v1);
                c = __fmaf_rn(e0.y, w0, __fmaf_rn(e0.z, v0, c));
                c1 = __fmaf_rn(e1.y, w1, __fmaf_rn(e1.z, v1, c1));
              }
              if (k < kend) {
                const float4 e0 = sCsr[k];
                const int i0 = 2 * __float_as_int(e0.x);
                const float v0 = sp[i0], w0 = sp[i0 + 1];
                dot2_step(a, c, e0.y, v0);
                c = __fmaf_rn(e0.y, w0, __fmaf_rn(e0.z, v0, c));
              }
            } else {
#pragma unroll 2
              for (; k + 1 < kend; k += 2) {
                const float4 e0 = sCsr[k], e1 = sCsr[k + 1];
                const float v0 = y0[__float_as_int(e0.x)], v1 = y0[__float_as_int(e1.x)];
                dot2_step(a, c, e0.y, v0);
                dot2_step(a1, c1, e1.y, v1);
                c = __fmaf_rn(e0.z, v0, c);
                c1 = __fmaf_rn(e1.z, v1, c1);
              }
              if (k < kend) {
                const float4 e0 = sCsr[k];
                const float v0 = y0[__float_as_int(e0.x)];
                dot2_step(a, c, e0.y, v0);
                c = __fmaf_rn(e0.z, v0, c);
              }
            }
            {
              const float t = __fadd_rn(a, a1);
              const float z = __fsub_rn(t, a);
              const float te = __fadd_rn(__fsub_rn(a, __fsub_rn(t, z)), __fsub_rn(a1, z));
              a = t;
              c = __fadd_rn(c, __fadd_rn(c1, te));
            }
            // r = x - (a + c): t + te = x - a exactly (TwoSum), then the small parts
            const float x = x4[jj];
            const float t = __fsub_rn(x, a);
            const float z = __fsub_rn(t, x);
            const float te = __fadd_rn(__fsub_rn(x, __fsub_rn(t, z)), __fsub_rn(-a, z));
            r = in ? __fadd_rn(t, __fsub_rn(te, c)) : 0.0f;
          }
          tc::split_tf32(r, h4[jj], l4[jj], true);
        }
        tc::tmem_st<4>(tquad + C::AH + (uint32_t)(grp * GW + c0), h4);
        tc::tmem_st<4>(tquad + C::AL + (uint32_t)(grp * GW + c0), l4);
      }
      tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {  // the correction R Dinv^T
      tc::fence_after_sync();
      mma_3x(C::DC);
    }
    ok = __syncthreads_and(tc::mbar_wait(mb + 1, phase, m.tc_wait_limit)) != 0;
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) break;
    tmem_to_stage(C::DC, true);  // Y = Y0 + R Dinv^T
    tc::fence_before_sync();
    __syncthreads();
    // uL[a][i] = sum_b Pf[a][b] Y[b nb + i], coalesced
    for (int t = tid; t < nrow * NL; t += NT) {
      const int r = t / NL, idx = t - r * NL;
      const int a = idx / NB, i = idx - a * NB;
      const float* P = sGeo + r * DD + a * D;
      const float* y = stage + r * SST + i;
      float acc = 0.0f;
#pragma unroll
      for (int b = 0; b < D; ++b) acc = fmaf(P[b], y[b * NB], acc);
      uL[e0 * NL + t] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RPG; ++j) xr[j] = xn[j];
    xneg = xnneg;
  }
  if (!ok) {
    if (tid == 0) atomicOr(m.err, kErrTcTimeoutV2l);
    tc::mbar_wait(mb, 0);               // bounded (full limit): the table copies land before exit
    tc::mbar_wait(mb + 1, phase ^ 1u);  // and the MMAs in flight drain before TMEM is freed
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, C::TCOLS);
  }
}

}  // namespace hopu
