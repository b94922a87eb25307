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
constexpr int kErrTcTimeout = 1;

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
  const float* geoT = static_cast<const float*>(m.geoT);

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
    ok = __syncthreads_and(tc::mbar_wait(mbar, phase)) != 0;
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
        const float* gp = geoT + e * GT;  // Pf = J / det J
        float P[D][D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) P[a][b] = __ldg(gp + a * D + b);
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
    if (tid == 0) atomicOr(m.err, kErrTcTimeout);
    tc::mbar_wait(mbar, phase ^ 1u);  // bounded: let the MMAs in flight drain before freeing TMEM
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, C::TCOLS);
  }
}

}  // namespace hopu
