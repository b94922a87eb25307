// CUDA kernels of the HOPU convection hot path for sm_103a, templated on the
// dimension D, the polynomial order K and the working precision T.
//
// Work decomposition: one warp per element (projections, volume term) or per facet
// (facet flux).  Reference tables are staged once per CTA in shared memory and the
// grids are persistent (a multiple of the SM count), so every CTA loads them once.
// Geometry is stored in FP64 (every precision mode) and rounded to T at use.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>

#include <cstdint>

#include "hopu_internal.h"

namespace hopu {

__host__ __device__ constexpr int cbinom(int n, int r) {
  int v = 1;
  for (int i = 1; i <= r; ++i) v = v * (n - r + i) / i;
  return (r < 0 || n < r) ? 0 : v;
}
__host__ __device__ constexpr int cnbasis(int dim, int k) { return k < 0 ? 0 : cbinom(k + dim, dim); }
__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }
__host__ __device__ constexpr int r4i(int n) { return ((n + 3) / 4) * 4; }

template <int D, int K>
struct Shape {
  static constexpr int nb = cnbasis(D, K);          // dim P^K(T)
  static constexpr int nf = cnbasis(D - 1, K);      // dim P^K(F)
  static constexpr int nloc = D * nb;               // local L2 / V_h block
  static constexpr int nint = nloc - (D + 1) * nf;  // interior V_h dofs
  static constexpr int mv = (3 * K - 1 + 2) / 2;    // points per direction, degree 3K-1
  static constexpr int mf = (3 * K + 2) / 2;        // points per direction, degree 3K
  static constexpr int nq = compact_volume_points(D, K) ? compact_volume_points(D, K) : cpow(mv, D);  // kernel rule
  static constexpr int nqf = cpow(mf, D - 1);
  static constexpr int geo = 2 * D * D + 2;
  static constexpr int gt = geoT_stride(D);  // Pf [0, d^2), Pi [d^2, 2d^2), M [2d^2, 3d^2), 1/|det J|
  static constexpr int nvp = ((nloc + 31) / 32) * 32;  // accumulators, padded to the warp
};

constexpr int kWarps = 4;  // warps per CTA of the warp-per-item kernels
constexpr unsigned kFull = 0xffffffffu;

// Programmatic dependent launch: every kernel lets the next kernel of the stream be
// scheduled as soon as all of its own CTAs have started (pdl_trigger), and waits for the
// previous kernel to complete, with its memory visible (pdl_wait), only after its
// prologue, which reads nothing but constant tables and mesh data and writes only shared
// memory.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Butterfly reduce-scatter of N (multiple of 32) per-lane values: afterwards lane L holds
// the warp totals of indices [L*N/32, (L+1)*N/32) in v[0 .. N/32).
template <int O, int S, int N, typename T>
__device__ __forceinline__ void rs_level(T (&v)[N], int lane) {
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int j = 0; j < S / 2; ++j) {
    const T lo = v[j], hi = v[j + S / 2];
    const T send = up ? lo : hi;
    const T keep = up ? hi : lo;
    v[j] = keep + __shfl_xor_sync(kFull, send, O);
  }
}
template <int N, typename T>
__device__ __forceinline__ void reduce_scatter(T (&v)[N], int lane) {
  static_assert(N % 32 == 0, "reduce_scatter needs a multiple of 32 values");
  rs_level<16, N, N>(v, lane);
  rs_level<8, N / 2, N>(v, lane);
  rs_level<4, N / 4, N>(v, lane);
  rs_level<2, N / 8, N>(v, lane);
  rs_level<1, N / 16, N>(v, lane);
}

// Every lane ends with the warp totals of all N values.
template <int N, typename T>
__device__ __forceinline__ void allreduce(T (&v)[N]) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] += __shfl_xor_sync(kFull, v[j], o);
  }
}

// FP32 combination a0 x0 + a1 x1 + a2 v with x0, x1 already loaded (0 where absent); the
// arithmetic of combine_at.
__device__ __forceinline__ float combine_f32(const Combine& c, float v, float x0, float x1) {
  float o = fmaf(c.l2, v, fmaf(c.l0, x0, c.l1 * x1));  // the small parts first
  o = fmaf(c.h1, x1, o);
  o = fmaf(c.h0, x0, o);
  return fmaf(c.h2, v, o);
}

template <typename T>
__device__ __forceinline__ T combine_at(const Combine& c, T v, int64_t idx) {
  if constexpr (sizeof(T) == 8) {
    T o = T(c.a2) * v;
    if (c.x0) o = fma(T(c.a0), static_cast<const T*>(c.x0)[idx], o);
    if (c.x1) o = fma(T(c.a1), static_cast<const T*>(c.x1)[idx], o);
    return o;
  } else {
    const float x0 = c.x0 ? static_cast<const float*>(c.x0)[idx] : 0.0f;
    const float x1 = c.x1 ? static_cast<const float*>(c.x1)[idx] : 0.0f;
    return combine_f32(c, v, x0, x1);
  }
}

// Error-free transformations of FP32 arithmetic (compensated dot products, Ogita, Rump
// and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2): the
// product a*x splits exactly into p + pe (pe by one FMA) and the running sum s + p into
// t + se (Knuth's TwoSum); the rounding errors collect in c, so that s + c carries the dot
// product as if it had been computed in twice the working precision and rounded once.
// The intrinsics keep the compiler from contracting or reordering the steps.
__device__ __forceinline__ void dot2_step(float& s, float& c, float a, float x) {
  const float p = __fmul_rn(a, x);
  const float pe = __fmaf_rn(a, x, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(se, pe));
}

// Vector views of shared memory: 16-byte loads of 4 floats or 2 doubles.
template <typename T> struct Pack;
template <> struct Pack<float> {
  static constexpr int W = 4;
  using V = float4;
  __device__ __forceinline__ static void unpack(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};
template <> struct Pack<double> {
  static constexpr int W = 2;
  using V = double2;
  __device__ __forceinline__ static void unpack(const V& v, double* o) { o[0] = v.x; o[1] = v.y; }
};

// ------------------------------------------------------------------------------------
// Projections (a1, a7) as products of the n_loc x n_loc reference matrix with the local
// vectors of tiles of elements.  The matrix is staged once per CTA ([s][NLP], so that four
// rows are one 16-byte load) when it fits in shared memory; the tiles are per warp (below).
template <int D, int K, typename T>
struct ProjCfg {
  using S = Shape<D, K>;
  static constexpr int NL = S::nloc;
  static constexpr int RG = (NL + 3) / 4;   // row groups of four
  static constexpr int NLP = RG * 4;        // padded table row
  static constexpr int NLQ = (NL % 2) ? NL : NL + 1;  // odd stride of the element rows
  static constexpr size_t TAB = size_t(NL) * NLP * sizeof(T);
  static constexpr bool STAB = TAB <= 120 * 1024;
  static constexpr size_t TABS = STAB ? ((TAB + 15) / 16) * 16 : 0;
};

template <int D, int K, typename T>
__device__ __forceinline__ const T* proj_setup(unsigned char* smem, const T* tab) {
  using C = ProjCfg<D, K, T>;
  if (!C::STAB) return tab;
  T* sT = reinterpret_cast<T*>(smem);
  for (int t = threadIdx.x; t < C::NL * C::NLP; t += blockDim.x) sT[t] = tab[t];
  return sT;
}

// a1: V_h -> L2 in warp tiles.  A warp takes EW = 8 elements at a time and needs no
// block-wide barrier, so the warps of an SM overlap one another's gathers and products.
// Per tile: one connectivity code per lane ((d+1) x 8 <= 32; code = facet << 2 | sign),
// the gather of the (d+1) facet blocks with the sign sigma and the interior block into
// X[s][k] (lane-consecutive addresses), the reference change of basis Dinv as a
// register-blocked product (four rows x four elements per lane; both operands one 16-byte
// load), and the contravariant Piola map J / det J on the way out (coalesced stores).
// tab = Dinv^T with rows padded to NLP: tab[s][r] = Dinv[r][s].
// PT = true computes instead the transpose of the back-projection R E_T^{-1}: each facet
// value goes to both copies with the averaging weight 1/2 and the sign sigma, interior
// values are copied, then (D Piola^{-1})^T: tab[s][r] = D[s][r], Piola^{-1}^T = Pi^T.
template <int D, int K, typename T>
struct ProjWCfg {
  using S = Shape<D, K>;
  using C = ProjCfg<D, K, T>;
  static constexpr int EW = 8;  // elements per warp tile
  static constexpr int NL = S::nloc, RG = C::RG, NLP = C::NLP, NLQ = C::NLQ, DD = D * D;
  static constexpr int NTASK = RG * (EW / 4);  // four rows x four elements per task
  static constexpr int NPASS = (NTASK + 31) / 32;
  static constexpr int XW = ((NL * EW > EW * NLQ ? NL * EW : EW * NLQ) + 3) / 4 * 4;  // X, then Y
  static constexpr int PER_WARP = XW + (EW * DD + 3) / 4 * 4;
  static constexpr int WARPS = 8;
  static constexpr size_t SMEM = C::TABS + size_t(WARPS) * PER_WARP * sizeof(T);
  static_assert((D + 1) * EW <= 32, "one connectivity code per lane");
  static_assert(SMEM <= 227 * 1024, "projection tile exceeds shared memory");
};

// The refined FP32 V_h -> L2 projection (k_v2l, FP32): per warp tile X [NL][EW] (the
// gathered local dofs, then the residual) and Y [EW][NLQ] (the coefficients) side by
// side; the sparse rows of D (csr, 16-byte entries) and, when it fits, Dinv^T are staged
// per CTA.  More warps per CTA where the per-CTA tables are large.
template <int D, int K>
struct ProjRCfg {
  using W = ProjWCfg<D, K, float>;
  using C = ProjCfg<D, K, float>;
  static constexpr int NL = W::NL, EW = W::EW, NLQ = W::NLQ, DD = W::DD;
  static constexpr int XS = (NL * EW + 3) / 4 * 4, YS = (EW * NLQ + 3) / 4 * 4, PS = (EW * DD + 3) / 4 * 4;
  static constexpr int PER_WARP = XS + YS + PS;
  static constexpr size_t CSR_MAX = size_t(NL + NL * NL) * 16;  // headers + every entry (upper bound)
  static constexpr size_t TILE = size_t(PER_WARP) * 4;
  static constexpr size_t TAB = C::TAB;                          // Dinv^T, FP32
  static constexpr int fit_warps(size_t fixed) {
    return fixed + 16 * TILE <= 220 * 1024 ? 16 : fixed + 12 * TILE <= 220 * 1024 ? 12 : fixed + 8 * TILE <= 220 * 1024 ? 8 : 4;
  }
};

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* o) {  // 4 consecutive values, 16-byte aligned
  Pack<T>::unpack(*reinterpret_cast<const typename Pack<T>::V*>(p), o);
  if constexpr (Pack<T>::W == 2) Pack<T>::unpack(*reinterpret_cast<const typename Pack<T>::V*>(p + 2), o + 2);
}

// The product of a warp tile: X[s][k] (s < NL, k < EW, in sX) is replaced by
// Y[k][r] = sum_s tab[s][r] X[s][k] (at sX[k * NLQ + r]).  Lanes own four rows x four
// elements; the tile stays in registers until every lane has read X.
template <int D, int K, typename T>
__device__ __forceinline__ void warp_tile_gemm(const T* Tb, T* sX, int lane) {
  using W = ProjWCfg<D, K, T>;
  constexpr int NL = W::NL, NLP = W::NLP, NLQ = W::NLQ, EW = W::EW;
  T keep[W::NPASS][4][4];
#pragma unroll
  for (int p = 0; p < W::NPASS; ++p) {
    const int task = lane + 32 * p, rg = task / (EW / 4), eg = task - rg * (EW / 4);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) keep[p][i][j] = T(0);
    if (task < W::NTASK) {
#pragma unroll 4
      for (int s2 = 0; s2 < NL; ++s2) {
        T tv[4], xv[4];
        ld4(Tb + s2 * NLP + rg * 4, tv);
        ld4(sX + s2 * EW + eg * 4, xv);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) keep[p][i][j] = fma(tv[i], xv[j], keep[p][i][j]);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int p = 0; p < W::NPASS; ++p) {
    const int task = lane + 32 * p, rg = task / (EW / 4), eg = task - rg * (EW / 4);
    if (task < W::NTASK) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (rg * 4 + i < NL)
#pragma unroll
          for (int j = 0; j < 4; ++j) sX[(eg * 4 + j) * NLQ + rg * 4 + i] = keep[p][i][j];
    }
  }
  __syncwarp();
}

// The product of a warp tile into a separate buffer: Y[k][r] (=|+=) sum_s tab[s][r] X[s][k]
// (X [s][EW] in sX, Y [EW][NLQ] in sY).
template <int D, int K, bool ADD>
__device__ __forceinline__ void warp_tile_gemm_to(const float* Tb, const float* sX, float* sY, int lane) {
  using W = ProjWCfg<D, K, float>;
  constexpr int NL = W::NL, NLP = W::NLP, NLQ = W::NLQ, EW = W::EW;
  float keep[W::NPASS][4][4];
#pragma unroll
  for (int p = 0; p < W::NPASS; ++p) {
    const int task = lane + 32 * p, rg = task / (EW / 4), eg = task - rg * (EW / 4);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) keep[p][i][j] = 0.0f;
    if (task < W::NTASK) {
#pragma unroll 4
      for (int s2 = 0; s2 < NL; ++s2) {
        float tv[4], xv[4];
        ld4(Tb + s2 * NLP + rg * 4, tv);
        ld4(sX + s2 * EW + eg * 4, xv);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) keep[p][i][j] = fmaf(tv[i], xv[j], keep[p][i][j]);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < W::NPASS; ++p) {
    const int task = lane + 32 * p, rg = task / (EW / 4), eg = task - rg * (EW / 4);
    if (task < W::NTASK) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (rg * 4 + i < NL)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float* y = sY + (eg * 4 + j) * NLQ + rg * 4 + i;
            *y = ADD ? __fadd_rn(*y, keep[p][i][j]) : keep[p][i][j];
          }
    }
  }
  __syncwarp();
}

// Residual of the reference change of basis, in place: X[s][k] <- X[s][k] - sum_r D[s][r] Y[k][r]
// in compensated FP32 (Dot2), so that it is accurate to the rounding of its own (small)
// size.  csr: NL row headers {s, first entry, count, 0} sorted by count (the rows a warp
// instruction serves have similar lengths), then entries {r, D_hi, D_lo, 0} with
// D_hi = float(D[s][r]) and D_lo = float(D[s][r] - D_hi) (the nonzeros of D only).  A lane
// takes one row for two of the tile's eight elements (eight rows per warp instruction: the
// row lengths of D are skewed, and more rows per instruction would leave more lanes idle).
template <int D, int K>
__device__ __forceinline__ void warp_tile_residual(const float4* csr, float* sX, const float* sY, int lane) {
  using W = ProjWCfg<D, K, float>;
  constexpr int NL = W::NL, EW = W::EW, NLQ = W::NLQ;
  static_assert(EW == 8, "four pairs of elements per row");
  const int4* hdr = reinterpret_cast<const int4*>(csr);
  for (int t = lane; t < NL * 4; t += 32) {
    const int h = t >> 2, q = t & 3;  // row header h, elements q and q + 4
    const int4 hd = hdr[h];
    float a0 = sX[hd.x * EW + q], a1 = sX[hd.x * EW + q + 4], c0 = 0.0f, c1 = 0.0f;
    const float* y0 = sY + q * NLQ;
    const float* y1 = y0 + 4 * NLQ;
    for (int j = hd.y; j < hd.y + hd.z; ++j) {
      const float4 ent = csr[j];
      const int r = __float_as_int(ent.x);
      const float v0 = y0[r], v1 = y1[r];
      dot2_step(a0, c0, -ent.y, v0);
      dot2_step(a1, c1, -ent.y, v1);
      c0 = __fmaf_rn(-ent.z, v0, c0);
      c1 = __fmaf_rn(-ent.z, v1, c1);
    }
    sX[hd.x * EW + q] = __fadd_rn(a0, c0);
    sX[hd.x * EW + q + 4] = __fadd_rn(a1, c1);
  }
  __syncwarp();
}

// FP32 (PT = false): the reference change of basis Dinv X is refined once, Y = Dinv X,
// then Y += Dinv (X - D Y) with the residual in compensated FP32 (csr: the sparse rows of
// D, see warp_tile_residual).  Reason: on smooth fields the reference coefficients of
// degree >= 2 are small differences of O(|u|) local dofs, so the plain FP32 product loses
// ~cond(D) ulps of |u| in them, and the convection operator, a first derivative,
// amplifies that by ~k^2/h (3e-6 of max |y| on a 16^3, k = 3 Taylor-Green field); after
// the refinement the projection is accurate to the rounding of its output.  nw: warps of
// the CTA (blockDim.x / 32); tab_staged: stage tab in shared memory.
template <int D, int K, typename T, bool PT>
__global__ void __launch_bounds__((!PT && sizeof(T) == 4) ? 512 : 32 * ProjWCfg<D, K, T>::WARPS) k_v2l(DevMesh m, const T* __restrict__ tab, const float4* __restrict__ csr,
                                             int csr_n, int tab_staged, const T* __restrict__ uV,
                                             T* __restrict__ uL) {
  using S = Shape<D, K>;
  using W = ProjWCfg<D, K, T>;
  constexpr int NL = S::nloc, NF = S::nf, NB = S::nb, NINT = S::nint, GEO = S::gt;
  constexpr int NLP = W::NLP, NLQ = W::NLQ, EW = W::EW, DD = W::DD, NC = (D + 1) * EW;
  constexpr int NIT = (NL * EW + 31) / 32;
  constexpr bool REF = !PT && sizeof(T) == 4;
  using R = ProjRCfg<D, K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  const T* Tb = tab;
  const float4* sCsr = csr;
  T* sX;
  T* sY;
  T* sP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if constexpr (REF) {
    // [csr (csr_n float4)][Dinv^T if staged][per-warp X | Y | P]
    float4* c4 = reinterpret_cast<float4*>(smem_raw);
    for (int t = threadIdx.x; t < csr_n; t += blockDim.x) c4[t] = csr[t];
    sCsr = c4;
    size_t off = size_t(csr_n) * 16;
    if (tab_staged) {
      T* sT = reinterpret_cast<T*>(smem_raw + off);
      for (int t = threadIdx.x; t < NL * NLP; t += blockDim.x) sT[t] = tab[t];
      Tb = sT;
      off += (R::TAB + 15) / 16 * 16;
    }
    sX = reinterpret_cast<T*>(smem_raw + off) + warp * R::PER_WARP;
    sY = sX + R::XS;
    sP = sY + R::YS;
  } else {
    Tb = proj_setup<D, K, T>(smem_raw, tab);
    sX = reinterpret_cast<T*>(smem_raw + ProjCfg<D, K, T>::TABS) + warp * W::PER_WARP;  // X [NL][EW], Y [EW][NLQ]
    sY = sX;
    sP = sX + W::XW;                                                                   // [EW][D*D]
  }
  const double* geoT = m.geoT;
  pdl_wait();
  __syncthreads();
  // tiles interleaved over the CTAs (tile = warp * gridDim.x + block), so that every SM of
  // the persistent grid gets the same number of tiles
  const int64_t ngroups = (m.E + EW - 1) / EW;
  for (int64_t grp = (int64_t)warp * gridDim.x + blockIdx.x; grp < ngroups; grp += (int64_t)gridDim.x * nwarps) {
    const int64_t e0 = grp * EW;
    const int ne = (m.E - e0 < EW) ? (int)(m.E - e0) : EW;
    const int code = (lane < NC && lane / (D + 1) < ne) ? m.efc[e0 * (D + 1) + lane] : 0;
    for (int t = lane; t < EW * DD; t += 32) {  // Pf = J / det J   (PT: Pi^T, Pi = det J Jinv)
      const int k = t / DD, r = t - k * DD, a = r / D, b = r - a * D;
      sP[t] = (k < ne) ? T(geoT[(e0 + k) * GEO + (PT ? DD + b * D + a : a * D + b)]) : T(0);
    }
#pragma unroll 5
    for (int it = 0; it < NIT; ++it) {
      const int t = lane + 32 * it;
      const int k = t % EW, s2 = t / EW;
      const int f = min(s2 / NF, D);
      const int c = __shfl_sync(kFull, code, k * (D + 1) + f);
      T v = T(0);
      if (t < NL * EW && k < ne) {
        if (s2 < (D + 1) * NF) {
          v = uV[(int64_t)(c >> 2) * NF + (s2 - f * NF)];
          if (c & 2) v = -v;
          if (PT) v *= T(0.5);
        } else {
          v = uV[(int64_t)m.NF * NF + (e0 + k) * NINT + (s2 - (D + 1) * NF)];
        }
      }
      if (t < NL * EW) sX[t] = v;  // t = s2 * EW + k
    }
    __syncwarp();
    if constexpr (REF) {
      const float* Tf = reinterpret_cast<const float*>(Tb);
      float* fX = reinterpret_cast<float*>(sX);
      float* fY = reinterpret_cast<float*>(sY);
      warp_tile_gemm_to<D, K, false>(Tf, fX, fY, lane);  // Y = Dinv X
      warp_tile_residual<D, K>(sCsr, fX, fY, lane);       // X <- X - D Y (compensated)
      warp_tile_gemm_to<D, K, true>(Tf, fX, fY, lane);   // Y += Dinv X
    } else {
      warp_tile_gemm<D, K, T>(Tb, sX, lane);
    }
    for (int t = lane; t < ne * NL; t += 32) {
      const int k = t / NL, idx = t - k * NL;
      const int a = idx / NB, i = idx - a * NB;
      T acc1 = T(0);
#pragma unroll
      for (int b = 0; b < D; ++b) acc1 = fma(sP[k * DD + a * D + b], sY[k * NLQ + b * NB + i], acc1);
      uL[e0 * NL + t] = acc1;
    }
    __syncwarp();
  }
}

// a7 (element part): local functionals of an L2 field, in the warp tiles of k_v2l.
// Not dual: ell = D (det J Jinv y); dual (the transpose E^T): ell = Dinv^T (J^T y / det J).
// Interior rows are combined into the V_h output; facet rows go to lf[e][f][m] with the
// sign sigma.  tab[s][r] (rows padded to NLP) = D[r][s] (not dual) or Dinv[s][r] (dual).
template <int D, int K, typename T, bool DUAL>
__global__ void __launch_bounds__(32 * ProjWCfg<D, K, T>::WARPS) k_l2v_elem(DevMesh m, const T* __restrict__ tab,
                                                                            const T* __restrict__ yL, T* __restrict__ lf,
                                                                            T* outV, Combine cmb) {
  using S = Shape<D, K>;
  using W = ProjWCfg<D, K, T>;
  constexpr int NL = S::nloc, NF = S::nf, NB = S::nb, NINT = S::nint, GEO = S::gt;
  constexpr int NLQ = W::NLQ, EW = W::EW, DD = W::DD, NC = (D + 1) * EW;
  constexpr int NIT = (NL * EW + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  const T* Tb = proj_setup<D, K, T>(smem_raw, tab);
  const double* geoT = m.geoT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* sX = reinterpret_cast<T*>(smem_raw + ProjCfg<D, K, T>::TABS) + warp * W::PER_WARP;  // X [NL][EW], Y [EW][NLQ]
  T* sP = sX + W::XW;                                                                   // [EW][D*D]
  pdl_wait();
  __syncthreads();
  const int64_t ngroups = (m.E + EW - 1) / EW;  // tiles interleaved over the CTAs (see k_v2l)
  for (int64_t grp = (int64_t)warp * gridDim.x + blockIdx.x; grp < ngroups; grp += (int64_t)gridDim.x * W::WARPS) {
    const int64_t e0 = grp * EW;
    const int ne = (m.E - e0 < EW) ? (int)(m.E - e0) : EW;
    const int code = (lane < NC && lane / (D + 1) < ne) ? m.efc[e0 * (D + 1) + lane] : 0;
    for (int t = lane; t < EW * DD; t += 32) {  // F[b][a]: Pi[b][a] = (det J Jinv)[b][a], or Pf^T[b][a]
      const int k = t / DD, r = t - k * DD, b = r / D, a = r - b * D;
      sP[t] = (k < ne) ? T(geoT[(e0 + k) * GEO + (DUAL ? a * D + b : DD + b * D + a)]) : T(0);
    }
    __syncwarp();
    for (int t = lane; t < NL * EW; t += 32) {  // X[s][k] = sum_a F_k[b][a] y_k[a][i],  s = b NB + i
      const int k = t % EW, s2 = t / EW;
      T acc1 = T(0);
      if (k < ne) {
        const int b = s2 / NB, i = s2 - b * NB;
        const T* y = yL + (e0 + k) * NL + i;
#pragma unroll
        for (int a = 0; a < D; ++a) acc1 = fma(sP[k * DD + b * D + a], y[a * NB], acc1);
      }
      sX[t] = acc1;
    }
    __syncwarp();
    warp_tile_gemm<D, K, T>(Tb, sX, lane);
#pragma unroll 5
    for (int it = 0; it < NIT; ++it) {
      const int t = lane + 32 * it;
      const int k = t / NL, r = t - k * NL;
      const int c = __shfl_sync(kFull, code, min(k, EW - 1) * (D + 1) + min(r / NF, D));
      if (t < ne * NL) {
        const int64_t e = e0 + k;
        const T v = sX[k * NLQ + r];
        if (r < (D + 1) * NF) {
          lf[e * (D + 1) * NF + r] = (c & 2) ? -v : v;
        } else {
          const int64_t idx = (int64_t)m.NF * NF + e * NINT + (r - (D + 1) * NF);
          outV[idx] = combine_at<T>(cmb, v, idx);
        }
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// Vectorised dot product of a register array with a 16-byte aligned shared-memory row
// (the row is padded to a multiple of 4 entries; padding entries are never used).
// Row stride (in elements) of point-major tables: a multiple of 16 bytes that is an odd
// multiple of 16 bytes, so that 8 consecutive lanes reading 16-byte chunks of 8
// consecutive rows hit 8 distinct bank groups.
template <typename T>
__host__ __device__ constexpr int row_stride(int n) {
  return sizeof(T) == 4 ? ((n + 3) / 4 * 4 + (((n + 3) / 4) % 2 == 0 ? 4 : 0))
                        : ((n + 1) / 2 * 2 + (((n + 1) / 2) % 2 == 0 ? 2 : 0));
}

// 16-byte shared-memory load that the compiler may not hoist out of a loop (keeps the
// loop-invariant coefficient rows in shared memory instead of in registers).
__device__ __forceinline__ void lds_v(const float* p, float* o) {
  asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];\n"
               : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
               : "r"((unsigned)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void lds_v(const double* p, double* o) {
  asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];\n"
               : "=d"(o[0]), "=d"(o[1])
               : "r"((unsigned)__cvta_generic_to_shared(p)));
}

// x[0..N) = s[0..N) with 16-byte loads (s 16-byte aligned)
template <int N, typename T>
__device__ __forceinline__ void load_row(const T* s, T* x) {
  constexpr int W = Pack<T>::W;
#pragma unroll
  for (int i = 0; i < N; i += W) {
    T o[W];
    Pack<T>::unpack(*reinterpret_cast<const typename Pack<T>::V*>(s + i), o);
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (i + w < N) x[i + w] = o[w];
  }
}

// sum_i x[i] s[i] with volatile 16-byte shared loads
template <int N, typename T>
__device__ __forceinline__ T dot_row_v(const T* x, const T* s) {
  constexpr int W = Pack<T>::W;
  T acc = T(0);
#pragma unroll
  for (int i = 0; i < N; i += W) {
    T o[W];
    lds_v(s + i, o);
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (i + w < N) acc = fma(x[i + w], o[w], acc);
  }
  return acc;
}

// the same row against two point vectors: every 16-byte shared load feeds both sums
template <int N, typename T>
__device__ __forceinline__ void dot2_row_v(const T* x0, const T* x1, const T* s, T& a0, T& a1) {
  constexpr int W = Pack<T>::W;
  a0 = T(0);
  a1 = T(0);
#pragma unroll
  for (int i = 0; i < N; i += W) {
    T o[W];
    lds_v(s + i, o);
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (i + w < N) {
        a0 = fma(x0[i + w], o[w], a0);
        a1 = fma(x1[i + w], o[w], a1);
      }
  }
}

template <int N, typename T>
__device__ __forceinline__ T dot_row(const T* x, const T* s) {
  constexpr int W = Pack<T>::W;
  T acc = T(0);
#pragma unroll
  for (int i = 0; i < N; i += W) {
    const typename Pack<T>::V v = *reinterpret_cast<const typename Pack<T>::V*>(s + i);
    T o[W];
    Pack<T>::unpack(v, o);
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (i + w < N) acc = fma(x[i + w], o[w], acc);
  }
  return acc;
}

__host__ __device__ constexpr int gcd_pow2(int bytes) { return (bytes % 16 == 0) ? 16 : (bytes % 8 == 0) ? 8 : 4; }

// Asynchronous global -> shared copies (cp.async, completion tracked per thread by
// commit/wait groups).  CH is the chunk size in bytes (4, 8 or 16); both addresses must
// be CH-aligned.
template <int CH>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (CH == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  } else if constexpr (CH == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// A warp copies one contiguous record of NBYTES bytes (record offsets are multiples of
// NBYTES and base pointers are 16-byte aligned, so gcd_pow2(NBYTES) alignment holds).
template <int NBYTES>
__device__ __forceinline__ void warp_copy_async(void* sdst, const void* gsrc, int lane) {
  constexpr int CH = gcd_pow2(NBYTES);
  constexpr int N = NBYTES / CH;
  for (int i = lane; i < N; i += 32)
    cp_async<CH>(static_cast<char*>(sdst) + i * CH, static_cast<const char*>(gsrc) + i * CH);
}

// ------------------------------------------------------------------------------------
// a4: facet term.  One warp per facet.  The traces of both sides are taken in modal
// form: tau^X_m = sum_i TrM_{f_X}[m][i] c^X_i (TrM = <phi_i o xhat_f, psi_m>, exact since
// phi_i restricted to a facet lies in P^k(F)), so the jump J and its complement
// (I - Pi^l) J are exact modal vectors: Pi^l (Section 3.2) keeps the tangential part of
// the first C(l+d-1, d-1) modes (hierarchical orthonormal facet basis), i.e. modes below
// that count keep only (J_m . n) n.  Lanes then own facet quadrature points and evaluate
// w.n (from the average of both sides' w, equal to w.n for normal-continuous w), J and
// (I - Pi^l) J there, and form h = 1/2 |w.n| (I - Pi^l) J and -1/2 (w.n) J.  Moments:
//   alpha[m][a] = a_F sum_q w_q psi_m(q) (-1/2 (w.n) J_a(q)),
//   beta[m][a]  = a_F sum_q w_q psi_m(q) ((I - Pi^l) h)_a(q),
// where, with an orthonormal facet basis, the moments of (I - Pi^l) h are those of h
// with the tangential part of the first modes removed.  They are written element-major:
// gam[e][f][m][a] for the element e that sees the facet as its local facet f,
// alpha + beta for side A and alpha - beta for side B.  Together with the volume kernel
// this is the conservative form of the convection operator rewritten by the
// element-wise integration by parts, which is exact for the rules used (volume degree
// 3k-1, facet degree 3k): every term is O(|u| |grad u|) or O(jump), so FP32 does not
// lose digits to the O(1/h) cancellation between volume and facet terms.
template <int N, typename T>
__device__ __forceinline__ T dot_ss(const T* p, const T* q) {
  constexpr int W = Pack<T>::W;
  T acc = T(0);
#pragma unroll
  for (int i = 0; i < N; i += W) {
    T a[W], b[W];
    Pack<T>::unpack(*reinterpret_cast<const typename Pack<T>::V*>(p + i), a);
    Pack<T>::unpack(*reinterpret_cast<const typename Pack<T>::V*>(q + i), b);
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (i + w < N) acc = fma(a[w], b[w], acc);
  }
  return acc;
}

// sum_i p[i] q[i] as the pair s + c, the first NC terms compensated (Dot2) and the rest
// summed plainly into c (both rows 16-byte aligned).  For a modal trace the first D + 1
// terms are the basis functions of degree <= 1: on smooth fields they carry the O(|u|)
// parts that cancel in the jump of two traces; the higher terms are O(h |grad u|) and
// smaller, so their plain FP32 sum leaves the jump accurate to ~1e-8 of |u| (a CPU
// emulation: 1.1e-8 with NC = 4, 6.6e-9 with every term compensated, 3.6e-7 with none).
template <int N, int NC>
__device__ __forceinline__ void dot2_ss(const float* p, const float* q, float& s, float& c) {
  s = 0.0f;
  c = 0.0f;
  float plain = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i += 4) {
    const float4 a = *reinterpret_cast<const float4*>(p + i);
    const float4 b = *reinterpret_cast<const float4*>(q + i);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (i + w < NC) dot2_step(s, c, av[w], bv[w]);
      else if (i + w < N) plain = fmaf(av[w], bv[w], plain);
    }
  }
  c = __fadd_rn(c, plain);
}

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T* o) {  // 4 consecutive values, 16-byte aligned
  Pack<T>::unpack(*reinterpret_cast<const typename Pack<T>::V*>(p), o);
  if constexpr (Pack<T>::W == 2) Pack<T>::unpack(*reinterpret_cast<const typename Pack<T>::V*>(p + 2), o + 2);
}

template <int D, int K, typename T, bool WSEP, bool STAB>
__global__ void __launch_bounds__(32 * kWarps) k_facet(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                       const T* __restrict__ wL, int lconst,
                                                       const int8_t* __restrict__ facet_l,
                                                       T* __restrict__ gam, double* __restrict__ diss) {
  static_assert(STAB, "facet tables always fit in shared memory");
  static_assert(Shape<D, K>::nf <= 32, "one lane per facet mode");
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NF = S::nf, NL = S::nloc, NQF = S::nqf, QP = (NQF + 31) / 32;
  constexpr int NBP = r4i(NB);
  constexpr int TRM = (D + 1) * NF * NBP, PSI = NF * NQF;
  constexpr int TABN = r4i(TRM + 2 * PSI + NQF);
  constexpr int CW = D * NBP;
  constexpr int SV = NQF * 4;
  constexpr int PER_WARP = (WSEP ? 4 : 2) * CW + 2 * SV + 2 * NF * 4 + 2 * NF * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  T* sbase = reinterpret_cast<T*>(smem_raw);
  {
    const T* TrMg = static_cast<const T*>(tb.TrM);
    const T* Psig = static_cast<const T*>(tb.Psi);
    const T* WPsig = static_cast<const T*>(tb.WPsi);
    const T* Wfg = static_cast<const T*>(tb.Wf);
    for (int t = threadIdx.x; t < TRM; t += blockDim.x) {
      const int row = t / NBP, i = t - row * NBP;
      sbase[t] = (i < NB) ? TrMg[row * NB + i] : T(0);
    }
    for (int t = threadIdx.x; t < PSI; t += blockDim.x) {
      sbase[TRM + t] = Psig[t];
      sbase[TRM + PSI + t] = WPsig[t];
    }
    for (int t = threadIdx.x; t < NQF; t += blockDim.x) sbase[TRM + 2 * PSI + t] = Wfg[t];
  }
  const T* TrM = sbase;
  const T* Psi = sbase + TRM;
  const T* WPsi = sbase + TRM + PSI;
  const T* Wf = sbase + TRM + 2 * PSI;
  T* sw = sbase + TABN;
  pdl_wait();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* cA = sw + warp * PER_WARP;
  T* cB = cA + CW;
  T* wA = WSEP ? cB + CW : cA;
  T* wB = WSEP ? wA + CW : cB;
  T* sH = cA + (WSEP ? 4 : 2) * CW;  // [NQF][4]   1/2 |w.n| (I - Pi^l) J
  T* sC = sH + SV;                   // [NQF][4]   -1/2 (w.n) J
  T* sJ = sC + SV;                   // [NF][4]    modal jump
  T* sWv = sJ + NF * 4;              // [NF][4]    modal average wind
  T* sOut = sWv + NF * 4;            // [2][NF][4] alpha, beta
  for (int64_t F = (int64_t)blockIdx.x * kWarps + warp; F < m.NF; F += (int64_t)gridDim.x * kWarps) {
    const int pa = m.fa[F], pb = m.fb[F];
    const int64_t eA = pa >> 2, eB = pb >> 2;
    const int fa = pa & 3, fb = pb & 3;
    const double* fg = m.fgeo + F * (D + 1);
    T n[D];
#pragma unroll
    for (int c = 0; c < D; ++c) n[c] = T(fg[c]);
    const T aF = T(fg[D]);
    const int l = facet_l ? int(facet_l[F]) : lconst;
    const int nl = (l < 0) ? 0 : cnbasis(D - 1, l);
    if constexpr (NBP == NB && (NL * sizeof(T)) % 16 == 0) {  // unpadded rows: 16-byte chunks
      constexpr int NCH = NL * (int)sizeof(T) / 16, CH = 16 / (int)sizeof(T);
      for (int c = lane; c < (WSEP ? 4 : 2) * NCH; c += 32) {
        const int which = c / NCH, cc = c - which * NCH;  // cA, cB, wA, wB (contiguous blocks of CW = NL)
        const T* src = (which < 2 ? uL : wL) + ((which & 1) ? eB : eA) * NL + cc * CH;
        *reinterpret_cast<uint4*>(cA + which * CW + cc * CH) = __ldg(reinterpret_cast<const uint4*>(src));
      }
    } else {
      for (int s2 = lane; s2 < NL; s2 += 32) {
        const int a = s2 / NB, i = s2 - a * NB;
        cA[a * NBP + i] = uL[eA * NL + s2];
        cB[a * NBP + i] = uL[eB * NL + s2];
        if (WSEP) {
          wA[a * NBP + i] = wL[eA * NL + s2];
          wB[a * NBP + i] = wL[eB * NL + s2];
        }
      }
    }
    __syncwarp();
    // modal traces: jump and average wind (an inlet facet's side B of u is its given data)
    const int inl = m.inlet ? m.inlet[F] : -1;
    const T* ext = inl >= 0 ? static_cast<const T*>(m.inlet_modes) + (int64_t)inl * NF * D : nullptr;
    for (int v = lane; v < NF * D; v += 32) {
      const int mm = v / D, a = v - mm * D;
      const T* ra = TrM + (fa * NF + mm) * NBP;
      const T* rb = TrM + (fb * NF + mm) * NBP;
      T ta, tbv, jump;
      if constexpr (sizeof(T) == 4) {
        // FP32: both traces as pairs with their degree <= 1 terms compensated, so that the
        // jump of a smooth field (a small difference of O(|u|) traces whose plain FP32 sums
        // carry errors of several ulps of the largest partial sum) stays accurate
        float sa, ca, sb = 0.0f, cb = 0.0f;
        dot2_ss<NB, D + 1>(ra, cA + a * NBP, sa, ca);
        if (ext) sb = ext[mm * D + a];
        else dot2_ss<NB, D + 1>(rb, cB + a * NBP, sb, cb);
        ta = __fadd_rn(sa, ca);
        tbv = __fadd_rn(sb, cb);
        jump = __fadd_rn(__fsub_rn(sa, sb), __fsub_rn(ca, cb));
      } else {
        ta = dot_ss<NB>(ra, cA + a * NBP);
        tbv = ext ? ext[mm * D + a] : dot_ss<NB>(rb, cB + a * NBP);
        jump = ta - tbv;
      }
      const T wa = WSEP ? dot_ss<NB>(ra, wA + a * NBP) : ta;
      const T wb = ext ? wa : (WSEP ? dot_ss<NB>(rb, wB + a * NBP) : tbv);  // an inlet keeps the wind's own w.n
      sJ[mm * 4 + a] = jump;
      sWv[mm * 4 + a] = T(0.5) * (wa + wb);
    }
    __syncwarp();
    // per mode: the normal component of the averaged wind (slot 3 of sJ) and the source of
    // the Pi^l complement (modes below nl keep only (J_m . n) n)
    T* sPj = sOut;  // [NF][4], free until the moments are written
    if (lane < NF) {
      T jm[4], wv[4];
      lds4(sJ + lane * 4, jm);
      lds4(sWv + lane * 4, wv);
      T jn = T(0), wvn = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        jn = fma(jm[a], n[a], jn);
        wvn = fma(wv[a], n[a], wvn);
      }
      const bool low = lane < nl;
#pragma unroll
      for (int a = 0; a < D; ++a) sPj[lane * 4 + a] = low ? jn * n[a] : jm[a];
      sJ[lane * 4 + 3] = wvn;
    }
    __syncwarp();
    T dsum = T(0);
#pragma unroll
    for (int qq = 0; qq < QP; ++qq) {
      const int q = lane + 32 * qq;
      const bool ok = q < NQF;
      const int qc = ok ? q : 0;
      T J[D], P[D], wn = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) J[a] = P[a] = T(0);
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) {
        const T p = Psi[mm * NQF + qc];
        T jm[4], pm[4];
        lds4(sJ + mm * 4, jm);   // J_m, (w.n)_m
        lds4(sPj + mm * 4, pm);  // J_m or (J_m . n) n
        wn = fma(p, jm[3], wn);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          J[a] = fma(p, jm[a], J[a]);
          P[a] = fma(p, pm[a], P[a]);
        }
      }
      const T aw = T(0.5) * fabs(wn);
      T p2 = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) p2 = fma(P[a], P[a], p2);
      if (ok) {
        dsum += Wf[q] * aw * p2;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          sH[q * 4 + a] = aw * P[a];
          sC[q * 4 + a] = T(-0.5) * wn * J[a];
        }
      }
    }
    __syncwarp();
    for (int v = lane; v < 2 * NF; v += 32) {
      const int which = v / NF, mm = v - which * NF;  // 0: alpha (central), 1: beta (upwind part)
      const T* src = which ? sH : sC;
      T acc[D];
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = T(0);
      for (int q = 0; q < NQF; ++q) {
        const T wp = WPsi[mm * NQF + q];
        T x[4];
        lds4(src + q * 4, x);
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] = fma(wp, x[a], acc[a]);
      }
      if (which && mm < nl) {  // (I - Pi^l) h: keep only the normal part of the low moments
        T dn = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) dn += acc[a] * n[a];
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] = dn * n[a];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) sOut[(which * NF + mm) * 4 + a] = aF * acc[a];
    }
    __syncwarp();
    // element-major output: side A's slot gets alpha + beta, side B's alpha - beta (a
    // boundary facet has no side B: fb == fa)
    for (int v = lane; v < (pb == pa ? 1 : 2) * NF * D; v += 32) {
      const int side = v / (NF * D), rest = v - side * (NF * D);
      const int mm = rest / D, a = rest - mm * D;
      const T al = sOut[mm * 4 + a], be = sOut[(NF + mm) * 4 + a];
      const int64_t slot = side ? (eB * (D + 1) + fb) : (eA * (D + 1) + fa);
      gam[slot * NF * D + rest] = side ? al - be : al + be;
    }
    if (diss) {
      T dv[1] = {dsum};
      allreduce<1>(dv);
      if (lane == 0) diss[F] = double(aF) * double(dv[0]);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// a3 + a5: volume term, facet lift and inverse mass.  One warp per element; lanes own
// volume quadrature points.  With W = |det J| J^{-1} w (so that |det J| (w.grad) u =
// W . grad^ u and |det J| div w = div^ W on an affine element):
//   r[a][i] = sum_q w_q phi_i(q) [ W(q) . grad^ u_a(q) + div^ W(q) u_a(q) ]
//           + sum_f sum_m TrM_f[m][i] (alpha_F(f) +- beta_F(f))[m][a],
//   y = r / |det J|      (orthonormal basis: M_T = |det J| I),
// then out = a0*x0 + a1*x1 + a2*y.  The reference gradients come from the modal
// differentiation matrices Dm (grad^ u_a = sum_j (Dm u_a)_j phi_j, j < dim P^{k-1}), so
// the only per-point table is phi_i(q).  Every per-element input (coefficients, the
// element's signed facet moments, geometry) is one contiguous record; a warp prefetches
// the next element's records with cp.async while it computes the current one.
template <int D, int K, typename T>
struct FuseCfg {  // row-major D table (local functionals) staged for the fused back-projection
  using S = Shape<D, K>;
  static constexpr int NLR = row_stride<T>(S::nloc);
  static constexpr int TAB = S::nloc * NLR;
  static constexpr bool OK = size_t(TAB) * sizeof(T) <= 40 * 1024;
};

template <int D, int K, typename T, bool WSEP, bool STAB, bool FUSE>
__global__ void __launch_bounds__(32 * kWarps, sizeof(T) == 4 ? 3 : 2) k_volume(DevMesh m, DevTabs tb, const T* __restrict__ uL,
                                                           const T* __restrict__ wL, const T* __restrict__ gam,
                                                           T* out, Combine cmb, T* __restrict__ lf) {
  using S = Shape<D, K>;
  constexpr int NB = S::nb, NB1 = cnbasis(D, K - 1), NF = S::nf, NL = S::nloc, NQ = S::nq;
  constexpr int NVP = S::nvp, CPL = NVP / 32, GEO = S::gt;
  constexpr int NBP = r4i(NB), NB1P = r4i(NB1);
  constexpr int NBQ = row_stride<T>(NB);
  constexpr int BT = NQ * NBQ, DM = D * NB1 * NB, TRM = (D + 1) * NF * NB;
  constexpr int FT = FUSE ? FuseCfg<D, K, T>::TAB : 0, NLR = FuseCfg<D, K, T>::NLR;
  constexpr int ODM = r4i(BT + NQ);          // staged Dm rows padded to NBP, 16-byte aligned
  constexpr int OTRM = r4i(ODM + D * NB1 * NBP);  // TrM 16-byte aligned (paired loads in the lift)
  constexpr int TABN = r4i(OTRM + TRM) + r4i(FT);
  constexpr int NG = (D + 1) * NF * D;
  constexpr int QB = (sizeof(T) == 4 && NQ > 32) ? 2 : 1;  // quadrature points per lane and pass
  static_assert(!FUSE || (STAB && FuseCfg<D, K, T>::OK), "fused back-projection needs staged tables");
  // per-warp layout: two staging buffers (u record, w record, facet moments, geometry),
  // then the working arrays
  constexpr int STU = r4i(NL), STG = r4i(NG), STGEO = r4i(GEO * 8 / (int)sizeof(T));  // FP64 record
  constexpr int STAGE = STU + (WSEP ? STU : 0) + STG + STGEO;
  constexpr int PER_WARP = 2 * STAGE + D * NBP + D * D * NB1P + (WSEP ? D * NBP + NB1P : 0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_trigger();
  T* sbase = reinterpret_cast<T*>(smem_raw);
  const T* Bt = static_cast<const T*>(tb.Bt);
  const T* Wq = static_cast<const T*>(tb.Wq);
  const T* Dm = static_cast<const T*>(tb.Dm);
  const T* TrM = static_cast<const T*>(tb.TrM);
  T* sw = sbase;
  if (STAB) {
    for (int t = threadIdx.x; t < BT; t += blockDim.x) sbase[t] = Bt[t];
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) sbase[BT + t] = Wq[t];
    for (int t = threadIdx.x; t < D * NB1 * NBP; t += blockDim.x) {
      const int row = t / NBP, i = t - row * NBP;
      sbase[ODM + t] = i < NB ? Dm[row * NB + i] : T(0);
    }
    for (int t = threadIdx.x; t < TRM; t += blockDim.x) sbase[OTRM + t] = TrM[t];
    Bt = sbase;
    Wq = sbase + BT;
    Dm = sbase + ODM;
    TrM = sbase + OTRM;
    sw = sbase + TABN;
  }
  T* Drow = sbase + r4i(OTRM + TRM);  // [NL][NLR] row-major D (FUSE)
  if (FUSE) {
    const T* Dg = static_cast<const T*>(tb.Drow);
    for (int t = threadIdx.x; t < FT; t += blockDim.x) Drow[t] = Dg[t];
  }
  pdl_wait();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* wbase = sw + warp * PER_WARP;
  T* sCpad = wbase + 2 * STAGE;             // [D][NBP]       u coefficients (padded rows)
  T* sG = sCpad + D * NBP;                  // [D][D][NB1P]   modal reference gradients of u
  T* sW = sG + D * D * NB1P;                // [D][NBP]       W coefficients (WSEP)
  T* sDv = sW + (WSEP ? D * NBP : 0);       // [NB1P]         modal div^ W (WSEP)
  auto st_u = [&](int b) { return wbase + b * STAGE; };
  auto st_w = [&](int b) { return wbase + b * STAGE + STU; };
  auto st_g = [&](int b) { return wbase + b * STAGE + STU + (WSEP ? STU : 0); };
  auto st_geo = [&](int b) { return st_g(b) + STG; };
  auto issue = [&](int64_t e, int b) {
    warp_copy_async<NL * (int)sizeof(T)>(st_u(b), uL + e * NL, lane);
    if (WSEP) warp_copy_async<NL * (int)sizeof(T)>(st_w(b), wL + e * NL, lane);
    warp_copy_async<NG * (int)sizeof(T)>(st_g(b), gam + e * NG, lane);
    warp_copy_async<GEO * 8>(st_geo(b), m.geoT + e * GEO, lane);
  };
  // facet lift of this lane's outputs: acc[j] += sum_fm TrM[fm][i] gl[fm][a]; with two
  // outputs per lane of one component and consecutive basis indices (NB even) every
  // paired TrM load and every moment load feed two FMAs
  auto lift = [&](T* accv, const T* gl) {
    if constexpr (CPL == 2 && NB % 2 == 0) {
      const int idx = lane * 2;
      if (idx < NL) {
        const int a = idx / NB, i = idx - a * NB;
#pragma unroll 4
        for (int fm = 0; fm < (D + 1) * NF; ++fm) {
          using P2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
          const T gv = gl[fm * D + a];
          const P2 tp = *reinterpret_cast<const P2*>(TrM + fm * NB + i);  // i even: aligned pair
          accv[0] = fma(tp.x, gv, accv[0]);
          accv[1] = fma(tp.y, gv, accv[1]);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int idx = lane * CPL + j;
        if (idx < NL) {
          const int a = idx / NB, i = idx - a * NB;
#pragma unroll 4
          for (int fm = 0; fm < (D + 1) * NF; ++fm) accv[j] = fma(TrM[fm * NB + i], gl[fm * D + a], accv[j]);
        }
      }
    }
  };
  if constexpr (NBP != NB)  // the padding of the u rows meets zero Dm columns: keep it finite
    for (int t = lane; t < D * NBP; t += 32) sCpad[t] = T(0);
  const int64_t stride = (int64_t)gridDim.x * kWarps;
  int64_t e = (int64_t)blockIdx.x * kWarps + warp;
  if (e < m.E) issue(e, 0);
  cp_commit();
  int b = 0;
  for (; e < m.E; e += stride, b ^= 1) {
    if (e + stride < m.E) issue(e + stride, b ^ 1);  // prefetch the next element
    cp_commit();
    cp_wait<1>();                                    // this element's copies are done
    __syncwarp();
    const double* g = reinterpret_cast<const double*>(st_geo(b));  // Pf, Pi, M = |det J| Jinv, 1/|det J|
    const T* gl = st_g(b);                           // signed facet moments of the element
    T M[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) M[a][c] = T(g[2 * D * D + a * D + c]);
    const T invabs = T(g[3 * D * D]);
    // u coefficients [D][NBP]: the staged record itself when its rows need no padding
    T* sC = (NBP == NB) ? st_u(b) : sCpad;
    for (int s2 = lane; s2 < NL; s2 += 32) {
      const int a = s2 / NB, i = s2 - a * NB;
      if (NBP != NB) sC[a * NBP + i] = st_u(b)[s2];
      if (WSEP) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) acc = fma(M[a][c], st_w(b)[c * NB + i], acc);
        sW[a * NBP + i] = acc;
      }
    }
    __syncwarp();
    if constexpr (STAB) {  // lane (c, j): (Dm_c u_a)_j for every a; padded rows, 16-byte loads
      for (int v = lane; v < D * NB1; v += 32) {
        const int c = v / NB1, j = v - c * NB1;
        const T* drow = Dm + (c * NB1 + j) * NBP;
        T acc[D];
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] = T(0);
#pragma unroll
        for (int i = 0; i < NBP; i += 4) {
          T dv[4];
          lds4(drow + i, dv);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            T cv[4];
            lds4(sC + a * NBP + i, cv);
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[a] = fma(dv[t], cv[t], acc[a]);
          }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) sG[(a * D + c) * NB1P + j] = acc[a];
      }
    } else {
      for (int v = lane; v < D * D * NB1; v += 32) {
        const int a = v / (D * NB1), c = (v / NB1) % D, j = v % NB1;
        T acc = T(0);
#pragma unroll 4
        for (int i = 0; i < NB; ++i) acc = fma(Dm[(c * NB1 + j) * NB + i], sC[a * NBP + i], acc);
        sG[(a * D + c) * NB1P + j] = acc;
      }
    }
    if (WSEP) {
      for (int j = lane; j < NB1; j += 32) {
        T acc = T(0);
        for (int c = 0; c < D; ++c)
#pragma unroll 4
          for (int i = 0; i < NB; ++i) acc = fma(Dm[(c * NB1 + j) * (STAB ? NBP : NB) + i], sW[c * NBP + i], acc);
        sDv[j] = acc;
      }
    }
    __syncwarp();
    T acc[NVP];
#pragma unroll
    for (int j = 0; j < NVP; ++j) acc[j] = T(0);
    if constexpr (QB == 2) {
      // two points per lane (q and q + 32): every coefficient row loaded from shared
      // memory feeds both points
      for (int q = lane; q < NQ; q += 64) {
        const int q1 = q + 32;
        const bool v1 = q1 < NQ;
        T ph0[NB], ph1[NB];
        load_row<NB>(Bt + q * NBQ, ph0);
        load_row<NB>(Bt + (v1 ? q1 : q) * NBQ, ph1);
        T u0[D], u1[D], G0[D][D], G1[D][D], W0[D], W1[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          dot2_row_v<NB>(ph0, ph1, sC + a * NBP, u0[a], u1[a]);
#pragma unroll
          for (int c = 0; c < D; ++c) dot2_row_v<NB1>(ph0, ph1, sG + (a * D + c) * NB1P, G0[a][c], G1[a][c]);
        }
        T dv0 = T(0), dv1 = T(0);
        if (WSEP) {
#pragma unroll
          for (int c = 0; c < D; ++c) dot2_row_v<NB>(ph0, ph1, sW + c * NBP, W0[c], W1[c]);
          dot2_row_v<NB1>(ph0, ph1, sDv, dv0, dv1);
        } else {
#pragma unroll
          for (int c = 0; c < D; ++c) {
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int bb = 0; bb < D; ++bb) {
              s0 = fma(M[c][bb], u0[bb], s0);
              s1 = fma(M[c][bb], u1[bb], s1);
              dv0 = fma(M[c][bb], G0[bb][c], dv0);
              dv1 = fma(M[c][bb], G1[bb][c], dv1);
            }
            W0[c] = s0;
            W1[c] = s1;
          }
        }
        const T wq0 = Wq[q], wq1 = v1 ? Wq[q1] : T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          T f0 = dv0 * u0[a], f1 = dv1 * u1[a];
#pragma unroll
          for (int c = 0; c < D; ++c) {
            f0 = fma(W0[c], G0[a][c], f0);
            f1 = fma(W1[c], G1[a][c], f1);
          }
          f0 *= wq0;
          f1 *= wq1;
#pragma unroll
          for (int i = 0; i < NB; ++i) acc[a * NB + i] = fma(f1, ph1[i], fma(f0, ph0[i], acc[a * NB + i]));
        }
      }
    } else
    for (int q = lane; q < NQ; q += 32) {
      T ph[NB];
      load_row<NB>(Bt + q * NBQ, ph);
      T u[D], G[D][D], W[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        u[a] = dot_row_v<NB>(ph, sC + a * NBP);
#pragma unroll
        for (int c = 0; c < D; ++c) G[a][c] = dot_row_v<NB1>(ph, sG + (a * D + c) * NB1P);
      }
      T dv = T(0);
      if (WSEP) {
#pragma unroll
        for (int c = 0; c < D; ++c) W[c] = dot_row_v<NB>(ph, sW + c * NBP);
        dv = dot_row_v<NB1>(ph, sDv);
      } else {
#pragma unroll
        for (int c = 0; c < D; ++c) {
          T sacc = T(0);
#pragma unroll
          for (int bb = 0; bb < D; ++bb) {
            sacc = fma(M[c][bb], u[bb], sacc);
            dv = fma(M[c][bb], G[bb][c], dv);
          }
          W[c] = sacc;
        }
      }
      const T wq = Wq[q];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        T f = dv * u[a];
#pragma unroll
        for (int c = 0; c < D; ++c) f = fma(W[c], G[a][c], f);
        f *= wq;
#pragma unroll
        for (int i = 0; i < NB; ++i) acc[a * NB + i] = fma(f, ph[i], acc[a * NB + i]);
      }
    }
    reduce_scatter<NVP>(acc, lane);
    if (!FUSE) {
      lift(acc, gl);
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int idx = lane * CPL + j;
        if (idx < NL) out[e * NL + idx] = combine_at<T>(cmb, acc[j] * invabs, e * NL + idx);
      }
    } else {
      // fused a7 (element part): y -> chat = det J Jinv y -> ell = D chat; interior rows
      // combined into the V_h output, facet rows to lf with the sign sigma
      T* sY = sC;  // [D][NBP], u coefficients are no longer needed
      T* sCh = sG; // [NL (padded to 4)]
      lift(acc, gl);
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int idx = lane * CPL + j;
        if (idx < NL) {
          const int a = idx / NB, i = idx - a * NB;
          sY[a * NBP + i] = acc[j] * invabs;
        }
      }
      __syncwarp();
      for (int idx = lane; idx < NL; idx += 32) {
        const int bb = idx / NB, i = idx - bb * NB;
        T c2 = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) c2 = fma(T(g[D * D + bb * D + a]), sY[a * NBP + i], c2);
        sCh[idx] = c2;
      }
      if (lane < r4i(NL) - NL) sCh[NL + lane] = T(0);
      __syncwarp();
      for (int r = lane; r < NL; r += 32) {
        const T v = dot_ss<r4i(NL)>(Drow + r * NLR, sCh);
        if (r < (D + 1) * NF) {
          const int code = m.efc[e * (D + 1) + r / NF];
          lf[e * (D + 1) * NF + r] = (code & 2) ? -v : v;
        } else {
          const int64_t idx = m.NF * NF + e * S::nint + (r - (D + 1) * NF);
          out[idx] = combine_at<T>(cmb, v, idx);
        }
      }
    }
    __syncwarp();
  }
  cp_wait<0>();
}

// ------------------------------------------------------------------------------------
// a7: L2 -> V_h.  Element part: local functionals ell = D (det J J^{-1} y) (or, for the
// transpose map, ell = Dinv^T (J^T y / det J)); interior rows are final, facet rows go to
// lf[e][f][m] with the sign sigma.  Facet part (R): average (or, transposed, sum) the two
// copies of every facet functional.
template <int D, int K, typename T, bool DUAL>
__global__ void __launch_bounds__(256) k_l2v_facet(DevMesh m, const T* __restrict__ lf, T* outV, Combine cmb) {
  constexpr int NF = Shape<D, K>::nf;
  pdl_trigger();
  pdl_wait();
  const int64_t total = m.NF * NF;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t F = t / NF;
    const int mm = (int)(t - F * NF);
    const int pa = m.fa[F], pb = m.fb[F];
    T v = lf[((int64_t)(pa >> 2) * (D + 1) + (pa & 3)) * NF + mm];
    if (pb != pa) {  // an interior facet: average (R) or sum (transpose) of the two copies
      v += lf[((int64_t)(pb >> 2) * (D + 1) + (pb & 3)) * NF + mm];
      if (!DUAL) v *= T(0.5);
    }
    outV[t] = combine_at<T>(cmb, v, t);
  }
}

}  // namespace hopu
