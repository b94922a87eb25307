// Hexahedral cells: the HOPU convection apply (Section 3.2, eq. "hopudefinition", in the
// conservative reading) on a structured periodic box of parallelepipeds (Section 2.1: the
// paper's meshes are hexahedral), with sum-factorised tensor-product contractions.
//
// Space: per velocity component, Q^k on the reference cube [0,1]^3 with the orthonormal
// tensor Legendre basis phi_i = L_i1(x1) L_i2(x2) L_i3(x3), i = i1 + K1 (i2 + K1 i3),
// K1 = k + 1; element blocks [E][3][K1^3].  Rules: M = ceil((3k+1)/2) Gauss points per
// direction, exact to degree 3k per direction (volume and facets).  Affine cells:
// M_T = |det J| I, so the inverse mass is 1/|det J| per cell.
//
// One warp per cell (k_hex_volume) or per facet (k_hex_facet); the contractions run as
// one-dimensional passes through the warp's shared-memory buffers (lanes over the outputs
// of a pass).  Cell e = i0 + n0 (i1 + n1 i2); facet F = d E + e is the low facet of cell e
// in direction d: side A the cell below (periodic), local facet x_d = 1; side B = e,
// x_d = 0.  The facet coordinates (s, t) are the two other axes in increasing order.
//
// Evaluation: the conservative form is rewritten cell by cell with the divergence theorem
// (exact under these rules: u w v has degree <= 3k per direction),
//   c(w; u, v) = sum_T int_T ((grad u) w + (div w) u) . v
//              + sum_F int_F [ -1/2 (w.n) [[u]] - 1/2 [[w.n]] u^A + Ph ] . v^A
//                          + [ -1/2 (w.n) [[u]] - 1/2 [[w.n]] u^B - Ph ] . v^B,
// Ph = (I - Pi^l)[1/2 |w.n| (I - Pi^l)[[u]]], w.n = <w>.n.  The same operator, but every term
// is of the size of the result for smooth fields; the conservative terms are k^2/h larger
// and cancel, which in FP32 costs about an order of magnitude of accuracy.
//
// Facets: traces of Q^k at x_d = 0 / 1 are the modal sums sum_{i_d} L_{i_d}(0 or 1) c_i,
// giving the facet's Q^k modes in the orthonormal facet basis L_s L_t.  (I - Pi^l) acts on
// modes: a mode (s, t) with max(s, t) <= l keeps only its normal part (Pi^l projects the
// tangential part onto Q^l, the reading of Section 3.2's P^l on quadrilateral facets).  The
// point values are taken back to moments by the facet rule; the moments (times the area
// factor) are lifted into the two cells by the trace's transpose,
// r_i += L_{i_d}(1) gA_(i_s,i_t) on side A and r_i += L_{i_d}(0) gB_(i_s,i_t) on side B,
// inside the volume kernel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hopu {
namespace hex {

template <int K>
struct Shape {
  static constexpr int K1 = K + 1;
  static constexpr int M = (3 * K + 2) / 2;
  static constexpr int NB = K1 * K1 * K1;
  static constexpr int NQ = M * M * M;
  static constexpr int NFM = K1 * K1;  // facet modes
  static constexpr int NQF = M * M;
};

struct MeshDev {
  int n0, n1, n2;
  int64_t E;
  const double* G;       // [E][3][3]  |det J| J^-1
  const double* invabs;  // [E]        1 / |det J|
  const double* nF;      // [3E][3]    unit normal of facet F (side A outward)
  const double* aF;      // [3E]       |F| / |F^| (= |det J| |J^-T e_d| of either side)
};

// 1D tables of one order in the working precision: B[q][i] = L_i(x_q), Dd[q][i] = L_i'(x_q),
// w1[q] (Gauss weights on [0,1]), e0[i] = L_i(0), e1[i] = L_i(1), and the parts of e0, e1 that
// the working precision drops (e0lo = L_i(0) - e0 rounded; zero in FP64).
template <typename T>
struct Tabs {
  const T* B;
  const T* Dd;
  const T* w1;
  const T* e0;
  const T* e1;
  const T* e0lo;
  const T* e1lo;
};

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// rounded operations the compiler may not contract into FMAs (the compensated sums need
// every product and sum rounded on its own)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }


template <typename T, int K>
struct Vol {
  using S = Shape<K>;
  static constexpr int K1 = S::K1, M = S::M, NB = S::NB, NQ = S::NQ, NFM = S::NFM;
  static constexpr int WARPS = sizeof(T) == 8 ? 2 : 4;
  // one field's coefficients | x-pass (B, D) | y-pass (BB, BD, DB) | wind at the points
  // (G w, |det J| div w) | the three integrands
  static constexpr int O_C = 0;
  static constexpr int O_X = O_C + NB;
  static constexpr int O_Y = O_X + 2 * K1 * K1 * M;
  static constexpr int O_W = O_Y + 3 * K1 * M * M;
  static constexpr int O_F = O_W + 4 * NQ;
  static constexpr int PER_WARP = O_F + 3 * NQ;
  static constexpr int TAB = 2 * M * K1 + M + 4 * K1;
  static constexpr size_t SMEM = size_t(TAB + WARPS * PER_WARP) * sizeof(T);
};

template <typename T, int K>
struct Fac {
  using S = Shape<K>;
  static constexpr int K1 = S::K1, M = S::M, NB = S::NB, NFM = S::NFM, NQF = S::NQF;
  static constexpr int WARPS = 4;
  static constexpr int NV = 11;  // point fields: w.n, [[w.n]], [[u]] (3), <u> (3), (I-Pi)[[u]] (3)
  static constexpr int NM = 9;   // moment fields: S (3), T (3), h (3)
  static constexpr int O_TR = 0;                 // traces: u^A, w^A, u^B, w^B (3 each)
  static constexpr int O_TL = O_TR + 12 * NFM;   // their low parts (compensated sums)
  static constexpr int O_V = O_TL + 12 * NFM;    // modal point fields
  static constexpr int O_T = O_V + NV * NFM;     // x-pass
  static constexpr int O_P = O_T + NV * K1 * M;  // point values
  static constexpr int O_Q = O_P + NV * NQF;     // weighted integrands
  static constexpr int O_U = O_Q + NM * NQF;     // transposed x-pass
  static constexpr int O_MO = O_U + NM * M * K1; // moments
  static constexpr int PER_WARP = O_MO + NM * NFM;
  static constexpr int TAB = 2 * M * K1 + M + 4 * K1;
  static constexpr size_t SMEM = size_t(TAB + WARPS * PER_WARP) * sizeof(T);
};

template <typename T, int K>
__device__ __forceinline__ void stage_tabs(const Tabs<T>& tb, T* s) {
  constexpr int K1 = K + 1, M = Shape<K>::M;
  for (int t = threadIdx.x; t < M * K1; t += blockDim.x) {
    s[t] = tb.B[t];
    s[M * K1 + t] = tb.Dd[t];
  }
  for (int t = threadIdx.x; t < M; t += blockDim.x) s[2 * M * K1 + t] = tb.w1[t];
  for (int t = threadIdx.x; t < K1; t += blockDim.x) {
    s[2 * M * K1 + M + t] = tb.e0[t];
    s[2 * M * K1 + M + K1 + t] = tb.e1[t];
    s[2 * M * K1 + M + 2 * K1 + t] = tb.e0lo[t];
    s[2 * M * K1 + M + 3 * K1 + t] = tb.e1lo[t];
  }
}

// basis index of the mode with index a_d on axis d and (s, t) on the other two axes
template <int K1>
__device__ __forceinline__ int mode_index(int d, int ad, int s, int t) {
  return d == 0 ? ad + K1 * (s + K1 * t) : (d == 1 ? s + K1 * (ad + K1 * t) : s + K1 * (t + K1 * ad));
}

__device__ __forceinline__ int64_t cell_shift(const MeshDev& m, int64_t e, int d, int by) {
  int i0 = int(e % m.n0), i1 = int((e / m.n0) % m.n1), i2 = int(e / ((int64_t)m.n0 * m.n1));
  if (d == 0) i0 = (i0 + by + m.n0) % m.n0;
  else if (d == 1) i1 = (i1 + by + m.n1) % m.n1;
  else i2 = (i2 + by + m.n2) % m.n2;
  return i0 + (int64_t)m.n0 * (i1 + (int64_t)m.n1 * i2);
}

// Facet kernel: gam[F][0][a][m] = a_F (moments of gA_a), gam[F][1][a][m] = a_F (moments of gB_a),
//   gA = S + T + Ph, gB = S - T - Ph,  S = -1/2 (w.n) [[u]] - 1/2 [[w.n]] <u>,  T = -1/4 [[w.n]] [[u]]
// (S + T = -1/2 (w.n)[[u]] - 1/2 [[w.n]] u^A, S - T the same with u^B).
template <typename T, int K>
__global__ void __launch_bounds__(32 * Fac<T, K>::WARPS)
    k_hex_facet(MeshDev m, Tabs<T> tb, const T* __restrict__ wL, const T* __restrict__ uL, int l,
                T* __restrict__ gam) {
  using C = Fac<T, K>;
  constexpr int K1 = C::K1, M = C::M, NB = C::NB, NFM = C::NFM, NQF = C::NQF, NV = C::NV, NM = C::NM;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  stage_tabs<T, K>(tb, sm);
  __syncthreads();
  const T* sB = sm;
  const T* sW = sm + 2 * M * K1;
  const T* sE0 = sW + M;
  const T* sE1 = sE0 + K1;
  const T* sE0l = sE1 + K1;
  const T* sE1l = sE0l + K1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* buf = sm + C::TAB + warp * C::PER_WARP;
  const int64_t NF = 3 * m.E;
  for (int64_t F = (int64_t)blockIdx.x * C::WARPS + warp; F < NF; F += (int64_t)gridDim.x * C::WARPS) {
    const int d = int(F / m.E);
    const int64_t eB = F - d * m.E;
    const int64_t eA = cell_shift(m, eB, d, -1);
    const T n0 = T(m.nF[F * 3 + 0]), n1 = T(m.nF[F * 3 + 1]), n2 = T(m.nF[F * 3 + 2]);
    const T aF = T(m.aF[F]);
    // 1. traces: fields 0-2 u^A, 3-5 w^A, 6-8 u^B, 9-11 w^B, each a compensated sum
    //    (hi + lo: error-free products by FMA, Knuth's TwoSum, L(0 or 1) as hi + lo), so that
    //    the jumps of nearly equal traces keep their relative accuracy in FP32
    for (int t = lane; t < 12 * NFM; t += 32) {
      const int f = t / NFM, mm = t - f * NFM;
      const int s = mm % K1, tt = mm / K1;
      const bool sideA = f < 6;
      const int comp = (f % 6) % 3;
      const T* src = ((f % 6) < 3 ? uL : wL) + ((sideA ? eA : eB) * 3 + comp) * NB;
      const T* en = sideA ? sE1 : sE0;
      const T* el = sideA ? sE1l : sE0l;
      T hi = T(0), lo = T(0);
#pragma unroll
      for (int ad = 0; ad < K1; ++ad) {
        const T c = src[mode_index<K1>(d, ad, s, tt)];
        const T p = mul_rn(en[ad], c);
        const T pe = fma(en[ad], c, -p);
        const T sum = add_rn(hi, p);
        const T bb = sub_rn(sum, hi);
        lo += add_rn(sub_rn(hi, sub_rn(sum, bb)), sub_rn(p, bb)) + fma(el[ad], c, pe);
        hi = sum;
      }
      buf[C::O_TR + t] = hi;
      buf[C::O_TL + t] = lo;
    }
    __syncwarp();
    // 2. modal point fields; the jumps from the pairs (hi_A - hi_B is exact for close traces)
    for (int mm = lane; mm < NFM; mm += 32) {
      const T* tr = buf + C::O_TR;
      const T* tl = buf + C::O_TL;
      T* v = buf + C::O_V + mm;
      T ja[3], wa = T(0), wj = T(0);
      const T nv[3] = {n0, n1, n2};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T uA = tr[a * NFM + mm], uB = tr[(6 + a) * NFM + mm];
        const T wA = tr[(3 + a) * NFM + mm], wB = tr[(9 + a) * NFM + mm];
        const T djw = (wA - wB) + (tl[(3 + a) * NFM + mm] - tl[(9 + a) * NFM + mm]);
        wa += T(0.5) * (wA + wB) * nv[a];
        wj += djw * nv[a];
        ja[a] = (uA - uB) + (tl[a * NFM + mm] - tl[(6 + a) * NFM + mm]);
        v[(2 + a) * NFM] = ja[a];
        v[(5 + a) * NFM] = T(0.5) * (uA + uB);
      }
      v[0] = wa;
      v[NFM] = wj;
      const int s = mm % K1, tt = mm / K1;
      const bool low = (s > tt ? s : tt) <= l;
      const T jn = ja[0] * n0 + ja[1] * n1 + ja[2] * n2;
      v[8 * NFM] = low ? jn * n0 : ja[0];
      v[9 * NFM] = low ? jn * n1 : ja[1];
      v[10 * NFM] = low ? jn * n2 : ja[2];
    }
    __syncwarp();
    // 3. to the points: x-pass over s, then y-pass over t
    for (int t = lane; t < NV * K1 * M; t += 32) {
      const int f = t / (K1 * M), r = t - f * K1 * M, tt = r / M, p1 = r - tt * M;
      const T* v = buf + C::O_V + f * NFM + tt * K1;
      T acc = T(0);
#pragma unroll
      for (int s = 0; s < K1; ++s) acc += sB[p1 * K1 + s] * v[s];
      buf[C::O_T + t] = acc;
    }
    __syncwarp();
    for (int t = lane; t < NV * NQF; t += 32) {
      const int f = t / NQF, p = t - f * NQF, p2 = p / M, p1 = p - p2 * M;
      const T* v = buf + C::O_T + f * K1 * M + p1;
      T acc = T(0);
#pragma unroll
      for (int tt = 0; tt < K1; ++tt) acc += sB[p2 * K1 + tt] * v[tt * M];
      buf[C::O_P + t] = acc;
    }
    __syncwarp();
    // 4. weighted integrands at the points: 0-2 S, 3-5 T, 6-8 h = 1/2|w.n| (I-Pi)[[u]]
    for (int p = lane; p < NQF; p += 32) {
      const int p2 = p / M, p1 = p - p2 * M;
      const T wgt = sW[p1] * sW[p2];
      const T* P = buf + C::O_P + p;
      const T wn = P[0], wj = P[NQF];
      const T hw = T(0.5) * fabs(wn) * wgt;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T ju = P[(2 + a) * NQF], au = P[(5 + a) * NQF], pj = P[(8 + a) * NQF];
        buf[C::O_Q + a * NQF + p] = T(-0.5) * wgt * (wn * ju + wj * au);
        buf[C::O_Q + (3 + a) * NQF + p] = T(-0.25) * wgt * wj * ju;
        buf[C::O_Q + (6 + a) * NQF + p] = hw * pj;
      }
    }
    __syncwarp();
    // 5. moments: transposed x-pass over p1, then y-pass over p2
    for (int t = lane; t < NM * M * K1; t += 32) {
      const int f = t / (M * K1), r = t - f * M * K1, p2 = r / K1, s = r - p2 * K1;
      const T* q = buf + C::O_Q + f * NQF + p2 * M;
      T acc = T(0);
#pragma unroll
      for (int p1 = 0; p1 < M; ++p1) acc += sB[p1 * K1 + s] * q[p1];
      buf[C::O_U + t] = acc;
    }
    __syncwarp();
    for (int t = lane; t < NM * NFM; t += 32) {
      const int f = t / NFM, mm = t - f * NFM, tt = mm / K1, s = mm - tt * K1;
      const T* u = buf + C::O_U + f * M * K1 + s;
      T acc = T(0);
#pragma unroll
      for (int p2 = 0; p2 < M; ++p2) acc += sB[p2 * K1 + tt] * u[p2 * K1];
      buf[C::O_MO + t] = acc;
    }
    __syncwarp();
    // 6. Ph = (I - Pi^l) h on the moments; gA = S + T + Ph, gB = S - T - Ph; times a_F
    for (int mm = lane; mm < NFM; mm += 32) {
      const T* mo = buf + C::O_MO + mm;
      const int s = mm % K1, tt = mm / K1;
      const bool low = (s > tt ? s : tt) <= l;
      const T h0 = mo[6 * NFM], h1 = mo[7 * NFM], h2 = mo[8 * NFM];
      const T hn = h0 * n0 + h1 * n1 + h2 * n2;
      const T ph[3] = {low ? hn * n0 : h0, low ? hn * n1 : h1, low ? hn * n2 : h2};
      T* out = gam + F * 6 * NFM + mm;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T sv = mo[a * NFM], tv = mo[(3 + a) * NFM];
        out[a * NFM] = aF * (sv + tv + ph[a]);
        out[(3 + a) * NFM] = aF * (sv - tv - ph[a]);
      }
    }
    __syncwarp();
  }
}

// Volume kernel + lift of the six facets' moments + inverse mass + the stage combination:
//   y = (1/|det J|) (r_vol + r_fac),
//   r_vol[a][i] = sum_q w_q ( sum_c (G w)_c d^_c u_a + |det J| div w  u_a ) phi_i,  G = |det J| J^-1,
//   |det J| div w = sum_{c,b} G[c][b] d^_c w_b,
//   out = c0 u0 + c1 us + c2 y   (out may alias u0: each warp reads and writes its own cell).
// Each of the six fields (w_0..2, then u_0..2) goes through one x-pass (B and D tables), one
// y-pass (BB, BD, DB) and a z-pass fused with its use at the points: the value and the three
// reference derivatives are BBB, DBB, BDB, BBD.
template <typename T, int K>
__global__ void __launch_bounds__(32 * Vol<T, K>::WARPS)
    k_hex_volume(MeshDev m, Tabs<T> tb, const T* __restrict__ wL, const T* us, const T* __restrict__ gam,
                 const T* u0, T c0, T c1, T c2, T* out) {
  using C = Vol<T, K>;
  constexpr int K1 = C::K1, M = C::M, NB = C::NB, NQ = C::NQ, NFM = C::NFM;
  constexpr int XS = K1 * K1 * M, YS = K1 * M * M, MM = M * M;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  stage_tabs<T, K>(tb, sm);
  __syncthreads();
  const T* sB = sm;
  const T* sD = sm + M * K1;
  const T* sW = sm + 2 * M * K1;
  const T* sE0 = sW + M;
  const T* sE1 = sE0 + K1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* base = sm + C::TAB + warp * C::PER_WARP;
  T* Cf = base + C::O_C;
  T* X = base + C::O_X;
  T* Y = base + C::O_Y;
  T* Wp = base + C::O_W;  // [4][NQ]: (G w)_0..2, |det J| div w
  T* Fp = base + C::O_F;  // [3][NQ]
  for (int64_t e = (int64_t)blockIdx.x * C::WARPS + warp; e < m.E; e += (int64_t)gridDim.x * C::WARPS) {
    T G[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) G[j] = T(m.G[e * 9 + j]);
    for (int f = 0; f < 6; ++f) {
      const bool wind = f < 3;
      const int comp = wind ? f : f - 3;
      const T* src = (wind ? wL : us) + (e * 3 + comp) * NB;
      for (int t = lane; t < NB; t += 32) Cf[t] = src[t];
      __syncwarp();
      // x-pass: X[0] = B over i1, X[1] = D over i1
      for (int t = lane; t < 2 * XS; t += 32) {
        const int v = t / XS, r = t - v * XS, i32 = r / M, q1 = r - i32 * M;
        const T* tab = v ? sD : sB;
        const T* c = Cf + i32 * K1;
        T acc = T(0);
#pragma unroll
        for (int i1 = 0; i1 < K1; ++i1) acc += tab[q1 * K1 + i1] * c[i1];
        X[t] = acc;
      }
      __syncwarp();
      // y-pass: Y[0] = BB, Y[1] = BD (D over i2), Y[2] = DB (from the x-derivative)
      for (int t = lane; t < 3 * YS; t += 32) {
        const int o = t / YS, r = t - o * YS, i3 = r / MM, r2 = r - i3 * MM, q2 = r2 / M, q1 = r2 - q2 * M;
        const T* tab = (o == 1) ? sD : sB;
        const T* c = X + (o == 2 ? XS : 0) + i3 * K1 * M + q1;
        T acc = T(0);
#pragma unroll
        for (int i2 = 0; i2 < K1; ++i2) acc += tab[q2 * K1 + i2] * c[i2 * M];
        Y[t] = acc;
      }
      __syncwarp();
      // z-pass fused with the use at the points; column comp of G (selects, not an indexed load)
      const T gc0 = comp == 0 ? G[0] : (comp == 1 ? G[1] : G[2]);
      const T gc1 = comp == 0 ? G[3] : (comp == 1 ? G[4] : G[5]);
      const T gc2 = comp == 0 ? G[6] : (comp == 1 ? G[7] : G[8]);
      for (int q = lane; q < NQ; q += 32) {
        const int q3 = q / MM, r2 = q - q3 * MM;
        T v = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
        for (int i3 = 0; i3 < K1; ++i3) {
          const T b = sB[q3 * K1 + i3], dz = sD[q3 * K1 + i3];
          const T bb = Y[i3 * MM + r2];
          v += b * bb;
          d3 += dz * bb;
          d2 += b * Y[YS + i3 * MM + r2];
          d1 += b * Y[2 * YS + i3 * MM + r2];
        }
        if (wind) {
          const T W0 = gc0 * v, W1 = gc1 * v, W2 = gc2 * v;
          const T dv = gc0 * d1 + gc1 * d2 + gc2 * d3;
          if (comp == 0) {
            Wp[q] = W0;
            Wp[NQ + q] = W1;
            Wp[2 * NQ + q] = W2;
            Wp[3 * NQ + q] = dv;
          } else {
            Wp[q] += W0;
            Wp[NQ + q] += W1;
            Wp[2 * NQ + q] += W2;
            Wp[3 * NQ + q] += dv;
          }
        } else {
          const int q2 = r2 / M, q1 = r2 - q2 * M;
          const T wq = sW[q1] * sW[q2] * sW[q3];
          Fp[comp * NQ + q] = wq * (Wp[q] * d1 + Wp[NQ + q] * d2 + Wp[2 * NQ + q] * d3 + Wp[3 * NQ + q] * v);
        }
      }
      __syncwarp();
    }
    const T ia = T(m.invabs[e]);
    int64_t fA[3], fB[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      fB[d] = d * m.E + e;
      fA[d] = d * m.E + cell_shift(m, e, d, 1);
    }
    for (int a = 0; a < 3; ++a) {
      // test with phi_i: passes over q3, q2, q1 (B tables)
      for (int t = lane; t < YS; t += 32) {
        const int i3 = t / MM, r2 = t - i3 * MM;
        const T* f = Fp + a * NQ + r2;
        T acc = T(0);
#pragma unroll
        for (int q3 = 0; q3 < M; ++q3) acc += sB[q3 * K1 + i3] * f[q3 * MM];
        Y[t] = acc;
      }
      __syncwarp();
      for (int t = lane; t < XS; t += 32) {
        const int i3 = t / (K1 * M), r = t - i3 * K1 * M, i2 = r / M, q1 = r - i2 * M;
        const T* g = Y + i3 * MM + q1;
        T acc = T(0);
#pragma unroll
        for (int q2 = 0; q2 < M; ++q2) acc += sB[q2 * K1 + i2] * g[q2 * M];
        X[t] = acc;
      }
      __syncwarp();
      for (int i = lane; i < NB; i += 32) {
        const int i3 = i / (K1 * K1), i2 = (i / K1) % K1, i1 = i % K1;
        const T* h = X + (i3 * K1 + i2) * M;
        T r = T(0);
#pragma unroll
        for (int q1 = 0; q1 < M; ++q1) r += sB[q1 * K1 + i1] * h[q1];
        // facets: direction 0 -> (s, t) = (i2, i3), 1 -> (i1, i3), 2 -> (i1, i2)
        const int md0 = i2 + K1 * i3, md1 = i1 + K1 * i3, md2 = i1 + K1 * i2;
        r += sE1[i1] * gam[(fA[0] * 6 + a) * NFM + md0] + sE0[i1] * gam[(fB[0] * 6 + 3 + a) * NFM + md0];
        r += sE1[i2] * gam[(fA[1] * 6 + a) * NFM + md1] + sE0[i2] * gam[(fB[1] * 6 + 3 + a) * NFM + md1];
        r += sE1[i3] * gam[(fA[2] * 6 + a) * NFM + md2] + sE0[i3] * gam[(fB[2] * 6 + 3 + a) * NFM + md2];
        const int64_t o = (e * 3 + a) * NB + i;
        T v = c2 * (r * ia);
        if (c1 != T(0)) v += c1 * us[o];
        if (c0 != T(0)) v += c0 * u0[o];
        out[o] = v;
      }
      __syncwarp();
    }
  }
}

}  // namespace hex
}  // namespace hopu
