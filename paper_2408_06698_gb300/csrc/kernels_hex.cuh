// Hexahedral cells: the HOPU convection apply (Section 3.2, eq. "hopudefinition", in the
// conservative reading) on a structured box of parallelepipeds, periodic or ending in walls,
// outlets or inlets per direction (Section 2.1: the paper's meshes are hexahedral), with
// sum-factorised tensor-product contractions.
//
// Space: per velocity component, Q^k on the reference cube [0,1]^3 with the orthonormal
// tensor Legendre basis phi_i = L_i1(x1) L_i2(x2) L_i3(x3), i = i1 + K1 (i2 + K1 i3),
// K1 = k + 1; element blocks [E][3][K1^3].  Rules: M = ceil((3k+1)/2) Gauss points per
// direction, exact to degree 3k per direction (volume and facets).  Affine cells:
// M_T = |det J| I, so the inverse mass is 1/|det J| per cell.
//
// One warp per cell (k_hex_volume, k_hex_volume_same) or per facet (k_hex_facet); the
// contractions run as one-dimensional passes through the warp's shared-memory buffers, a
// lane owning one line of the tensor with its inputs and (FP32) the 1D tables in registers.
// Cell e = i0 + n0 (i1 + n1 i2); facet F = d E + e is the low facet of cell e in direction
// d: side A the cell below (periodic wrap), local facet x_d = 1; side B = e, x_d = 0.  The
// facet coordinates (s, t) are the two other axes in increasing order.  At the ends of a
// non-periodic direction the slot F of the first cell holds two boundary facets (see
// k_hex_facet).
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
  int bmask;  // bit d set: direction d is not periodic (walls / outlets at its two ends)
  int64_t E;
  // inlet data of the two ends of a non-periodic direction (NULL: wall / outlet): the
  // exterior velocity's facet modes [cell (s, t) of the end][3][(k+1)^2] in the working
  // precision, s, t the cell indices of the two other directions (lower axis fastest)
  const void* inlet[3][2];
  // per-facet HOPU orders [3E] (-1..k; NULL: the launch's l); a boundary slot's two facets
  // share the slot's order
  const int8_t* facet_l;
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


// The 1D tables B[q][i], D[q][i] of one order, in registers (FP32) or read from shared
// memory (FP64, where the FP64 FMA rate, not the loads, bounds the passes).
template <typename T, int K, bool REG>
struct Tab1 {
  static constexpr int K1 = K + 1, M = Shape<K>::M;
  T b_[REG ? M * K1 : 1], d_[REG ? M * K1 : 1];
  const T* sb;
  const T* sd;
  __device__ __forceinline__ void load(const T* sB, const T* sD) {
    sb = sB;
    sd = sD;
    if constexpr (REG) {
#pragma unroll
      for (int j = 0; j < M * K1; ++j) {
        b_[j] = sB[j];
        d_[j] = sD[j];
      }
    }
  }
  __device__ __forceinline__ T b(int q, int i) const {
    if constexpr (REG) return b_[q * K1 + i];
    else return sb[q * K1 + i];
  }
  __device__ __forceinline__ T d(int q, int i) const {
    if constexpr (REG) return d_[q * K1 + i];
    else return sd[q * K1 + i];
  }
};

template <typename T, int K>
struct Fac {
  using S = Shape<K>;
  static constexpr int K1 = S::K1, M = S::M, NB = S::NB, NFM = S::NFM, NQF = S::NQF;
  static constexpr int K1o = K1 | 1, Mo = M | 1;  // odd line strides
  static constexpr int WARPS = 4;
  static constexpr bool REG = sizeof(T) == 4;
  static constexpr int MINB = sizeof(T) == 4 && K <= 4 ? 5 : 1;  // resident CTAs per SM the registers allow
  static constexpr int NV = 11;  // point fields: w.n, [[w.n]], [[u]] (3), <u> (3), (I-Pi)[[u]] (3)
  static constexpr int NM = 9;   // moment fields: S (3), T (3), h (3)
  static constexpr int O_TR = 0;                     // traces: u^A, w^A, u^B, w^B (3 each)
  static constexpr int O_TL = O_TR + 12 * NFM;       // their low parts (compensated sums)
  static constexpr int O_V = O_TL + 12 * NFM;        // modal point fields [f][t][s]
  static constexpr int O_T = O_V + NV * K1 * K1o;    // x-pass [f][p1][t]
  static constexpr int O_P = O_T + NV * M * K1o;     // point values [f][p2][p1]
  static constexpr int O_Q = O_P + NV * NQF;         // weighted integrands [f][p2][p1]
  static constexpr int O_U = O_Q + NM * M * Mo;      // transposed x-pass [f][s][p2]
  static constexpr int O_MO = O_U + NM * K1 * Mo;    // moments [f][t][s]
  static constexpr int PER_WARP = O_MO + NM * NFM;
  static constexpr int TAB = 2 * M * K1 + M + 4 * K1;
  static constexpr size_t SMEM = size_t(TAB + WARPS * PER_WARP) * sizeof(T);
  static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
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

// The adaptive step of k_hex_facet in its ETA instantiation: thresholds eta_0 < ... < eta_k,
// the new orders written to l_out[F] (may be the array the orders are read from: each facet
// reads its own entry first), eta to eta_out[F] when given.
struct EtaArgs {
  double thr[6];
  int8_t* l_out;
  double* eta_out;
};

// Facet kernel (BND: the box has non-periodic directions, whose end facets are walls,
// outlets or inlets): gam[F][0][a][m] = a_F (moments of gA_a), gam[F][1][a][m] = a_F (moments of gB_a),
//   gA = S + T + Ph, gB = S - T - Ph,  S = -1/2 (w.n) [[u]] - 1/2 [[w.n]] <u>,  T = -1/4 [[w.n]] [[u]]
// (S + T = -1/2 (w.n)[[u]] - 1/2 [[w.n]] u^A, S - T the same with u^B).
// ETA: instead of the moments, the jump indicator of adaptive HOPU (Section 3.2, after eq.
// "hopudefinition") eta = int |(I - Pi^l)[[u]]| / int |<u>| with the facet's current order,
// summed in FP64 over the facet points, and the new order (-1 for eta <= eta_0, i for
// eta_i < eta <= eta_{i+1}, k above eta_k; a zero average with a non-zero jump: +inf).
template <typename T, int K, bool BND, bool ETA = false>
__global__ void __launch_bounds__(32 * Fac<T, K>::WARPS, Fac<T, K>::MINB)
    k_hex_facet(MeshDev m, Tabs<T> tb, const T* __restrict__ wL, const T* __restrict__ uL, int l0,
                T* __restrict__ gam, double* __restrict__ diss_part, EtaArgs ea) {
  using C = Fac<T, K>;
  constexpr int K1 = C::K1, M = C::M, NB = C::NB, NFM = C::NFM, NQF = C::NQF, NV = C::NV, NM = C::NM;
  constexpr int K1o = C::K1o, Mo = C::Mo;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  stage_tabs<T, K>(tb, sm);
  __syncthreads();
  Tab1<T, K, C::REG> t1;
  t1.load(sm, sm + M * K1);
  const T* sW = sm + 2 * M * K1;
  const T* sE0 = sW + M;
  const T* sE1 = sE0 + K1;
  const T* sE0l = sE1 + K1;
  const T* sE1l = sE0l + K1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* buf = sm + C::TAB + warp * C::PER_WARP;
  const int64_t NF = 3 * m.E;
  const bool same = wL == uL;
  double dacc = 0.0;  // facet dissipation of this lane's points (when diss_part is given)
  // work item wi -> the facet of direction wi % 3 below cell wi / 3: the three facets of a
  // cell are taken together, so that its coefficients are read from DRAM once
  for (int64_t wi = (int64_t)blockIdx.x * C::WARPS + warp; wi < NF; wi += (int64_t)gridDim.x * C::WARPS) {
    const int d = int(wi % 3);
    const int64_t eB = wi / 3;
    const int64_t F = d * m.E + eB;
    const T aF = T(m.aF[F]);
    const int l = m.facet_l ? int(m.facet_l[F]) : l0;
    // The slot of the first cell of a non-periodic direction holds two boundary facets: the
    // top one of the last cell (its moments in the slot's side-A part) and the bottom one of
    // the first (side-B part).  Walls and outlets add nothing in the evaluated form (the
    // cell-wise integration by parts cancels the conservative form's own-trace flux): zero
    // moments.  An inlet runs the facet's steps below with the cell as side A (its own
    // normal), the inlet data as side B's velocity and the cell's own wind on both sides.
    bool bslot = false;
    int jend = 0;
    if (BND && ((m.bmask >> d) & 1)) {
      const int c0i = int(eB % m.n0), c1i = int((eB / m.n0) % m.n1), c2i = int(eB / ((int64_t)m.n0 * m.n1));
      bslot = (d == 0 ? c0i : (d == 1 ? c1i : c2i)) == 0;
      jend = d == 0 ? c1i + m.n1 * c2i : (d == 1 ? c0i + m.n0 * c2i : c0i + m.n0 * c1i);
    }
    const int64_t eBelow = cell_shift(m, eB, d, -1);
#pragma unroll 1
    for (int sub = 0; sub < (BND && bslot ? 2 : 1); ++sub) {
      // sub-facet: side A cell and its end (x_d = 1 or 0), side B cell or inlet data, normal sign
      int64_t eA = eBelow;
      bool endA1 = true;
      T sgn = T(1);
      const T* ext = nullptr;
      T* outA = gam + F * 6 * NFM;           // side-A part of the slot
      T* outB = outA + 3 * NFM;              // side-B part
      if (BND && bslot) {
        const void* in = m.inlet[d][sub == 0 ? 1 : 0];
        T* part = sub == 0 ? outA : outB;
        if (!in) {
          for (int t = lane; t < 3 * NFM; t += 32) part[t] = T(0);
          continue;
        }
        ext = static_cast<const T*>(in) + (int64_t)jend * 3 * NFM;
        if (sub == 1) {
          eA = eB;
          endA1 = false;
          sgn = T(-1);
        }
        outA = part;
        outB = nullptr;
      }
      const bool extB = BND && ext != nullptr;
      const bool samew = same && !extB;  // w^A, w^B read from the velocity traces
      const T n0 = sgn * T(m.nF[F * 3 + 0]), n1 = sgn * T(m.nF[F * 3 + 1]), n2 = sgn * T(m.nF[F * 3 + 2]);
      // 1. traces: fields 0-2 u^A, 3-5 w^A, 6-8 u^B, 9-11 w^B, each a compensated sum
      //    (hi + lo: error-free products by FMA, Knuth's TwoSum, L(0 or 1) as hi + lo), so
      //    that the jumps of nearly equal traces keep their relative accuracy in FP32.  A lane
      //    owns one line (field, t) of the facet and forms its K1 traces (s = 0..K1-1), all
      //    its loads issued first; the coefficient of mode (a_d, s, t) sits at
      //    a_d sd + s ss + t st.  When the wind is the convected field (w = u, a STAGE
      //    substep) only the velocity traces are formed, and read for both.
      const int sd = d == 0 ? 1 : (d == 1 ? K1 : K1 * K1);
      const int ss = d == 0 ? K1 : 1;
      const int st = d == 2 ? K1 : K1 * K1;
      // lines: w = u: u^A, u^B; else u^A, w^A, u^B, w^B; an inlet: u^A (and w^A unless w = u)
      const int nlines = (extB ? (same ? 3 : 6) : (same ? 6 : 12)) * K1;
      for (int L = lane; L < nlines; L += 32) {
        const int f0 = L / K1, tt = L - f0 * K1;
        const int f = same && f0 >= 3 ? f0 + 3 : f0;
        const bool sideA = f < 6;
        const int comp = (f % 6) % 3;
        const T* src = ((f % 6) < 3 ? uL : wL) + ((sideA ? eA : eB) * 3 + comp) * NB + tt * st;
        const bool e1 = sideA ? endA1 : false;
        const T* en = e1 ? sE1 : sE0;
        const T* el = e1 ? sE1l : sE0l;
        T cv[K1][K1];
#pragma unroll
        for (int s2 = 0; s2 < K1; ++s2)
#pragma unroll
          for (int ad = 0; ad < K1; ++ad) cv[s2][ad] = __ldg(src + ad * sd + s2 * ss);
#pragma unroll
        for (int s2 = 0; s2 < K1; ++s2) {
          T hi = T(0), lo = T(0);
#pragma unroll
          for (int ad = 0; ad < K1; ++ad) {
            const T c = cv[s2][ad];
            const T p = mul_rn(en[ad], c);
            const T pe = fma(en[ad], c, -p);
            const T sum = add_rn(hi, p);
            const T bb = sub_rn(sum, hi);
            lo += add_rn(sub_rn(hi, sub_rn(sum, bb)), sub_rn(p, bb)) + fma(el[ad], c, pe);
            hi = sum;
          }
          buf[C::O_TR + f * NFM + s2 + K1 * tt] = hi;
          buf[C::O_TL + f * NFM + s2 + K1 * tt] = lo;
        }
      }
      if (extB) {  // side B's velocity: the inlet modes (exact, no low part)
        for (int t = lane; t < 3 * NFM; t += 32) {
          buf[C::O_TR + 6 * NFM + t] = ext[t];
          buf[C::O_TL + 6 * NFM + t] = T(0);
        }
      }
      __syncwarp();
      // 2. modal point fields [f][t][s]; the jumps from the pairs (hi_A - hi_B is exact for
      //    close traces)
      for (int mm = lane; mm < NFM; mm += 32) {
        const T* tr = buf + C::O_TR;
        const T* tl = buf + C::O_TL;
        const int s = mm % K1, tt = mm / K1;
        T* v = buf + C::O_V + tt * K1o + s;
        constexpr int FS = K1 * K1o;  // one field
        T ja[3], wa = T(0), wj = T(0);
        const T nv[3] = {n0, n1, n2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T uA = tr[a * NFM + mm], uB = tr[(6 + a) * NFM + mm];
          const int iwA = same ? a : 3 + a, iwB = extB ? iwA : (samew ? 6 + a : 9 + a);
          const T wA = tr[iwA * NFM + mm], wB = tr[iwB * NFM + mm];
          const T djw = (wA - wB) + (tl[iwA * NFM + mm] - tl[iwB * NFM + mm]);
          wa += T(0.5) * (wA + wB) * nv[a];
          wj += djw * nv[a];
          ja[a] = (uA - uB) + (tl[a * NFM + mm] - tl[(6 + a) * NFM + mm]);
          v[(2 + a) * FS] = ja[a];
          v[(5 + a) * FS] = T(0.5) * (uA + uB);
        }
        v[0] = wa;
        v[FS] = wj;
        const bool low = (s > tt ? s : tt) <= l;
        const T jn = ja[0] * n0 + ja[1] * n1 + ja[2] * n2;
        v[8 * FS] = low ? jn * n0 : ja[0];
        v[9 * FS] = low ? jn * n1 : ja[1];
        v[10 * FS] = low ? jn * n2 : ja[2];
      }
      __syncwarp();
      // 3. to the points, lanes owning lines: over s (lines (f, t)), then over t (lines (f, p1))
      for (int L = lane; L < NV * K1; L += 32) {
        const int f = L / K1, tt = L - f * K1;
        T c[K1];
#pragma unroll
        for (int s = 0; s < K1; ++s) c[s] = buf[C::O_V + L * K1o + s];
#pragma unroll
        for (int p1 = 0; p1 < M; ++p1) {
          T acc = T(0);
#pragma unroll
          for (int s = 0; s < K1; ++s) acc = fma(t1.b(p1, s), c[s], acc);
          buf[C::O_T + (f * M + p1) * K1o + tt] = acc;
        }
      }
      __syncwarp();
      for (int L = lane; L < NV * M; L += 32) {
        const int f = L / M, p1 = L - f * M;
        T c[K1];
#pragma unroll
        for (int tt = 0; tt < K1; ++tt) c[tt] = buf[C::O_T + L * K1o + tt];
#pragma unroll
        for (int p2 = 0; p2 < M; ++p2) {
          T acc = T(0);
#pragma unroll
          for (int tt = 0; tt < K1; ++tt) acc = fma(t1.b(p2, tt), c[tt], acc);
          buf[C::O_P + f * NQF + p2 * M + p1] = acc;
        }
      }
      __syncwarp();
      if constexpr (ETA) {
        double sn = 0.0, sdn = 0.0;
        for (int p = lane; p < NQF; p += 32) {
          const int p2 = p / M, p1 = p - p2 * M;
          const double wgt = double(sW[p1]) * double(sW[p2]);
          const T* P = buf + C::O_P + p;
          const double j0 = P[8 * NQF], j1 = P[9 * NQF], j2 = P[10 * NQF];
          const double a0 = P[5 * NQF], a1 = P[6 * NQF], a2 = P[7 * NQF];
          sn += wgt * sqrt(j0 * j0 + j1 * j1 + j2 * j2);
          sdn += wgt * sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sn += __shfl_xor_sync(0xffffffffu, sn, o);
          sdn += __shfl_xor_sync(0xffffffffu, sdn, o);
        }
        if (lane == 0) {
          const double eta = sdn > 0.0 ? sn / sdn : (sn > 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : 0.0);
          int lnew = -1;
#pragma unroll
          for (int i = 0; i <= K; ++i)
            if (eta > ea.thr[i]) lnew = i;
          if (ea.eta_out) ea.eta_out[F] = eta;
          ea.l_out[F] = int8_t(lnew);
        }
        __syncwarp();
      } else {
        // 4. weighted integrands at the points: 0-2 S, 3-5 T, 6-8 h = 1/2|w.n| (I-Pi)[[u]]
        for (int p = lane; p < NQF; p += 32) {
          const int p2 = p / M, p1 = p - p2 * M;
          const T wgt = sW[p1] * sW[p2];
          const T* P = buf + C::O_P + p;
          const T wn = P[0], wj = P[NQF];
          const T hw = T(0.5) * fabs(wn) * wgt;
          if (diss_part) {
            const double p0 = P[8 * NQF], p1 = P[9 * NQF], p2v = P[10 * NQF];
            dacc += double(aF) * double(hw) * (p0 * p0 + p1 * p1 + p2v * p2v);
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const T ju = P[(2 + a) * NQF], au = P[(5 + a) * NQF], pj = P[(8 + a) * NQF];
            const int qo = p2 * Mo + p1;
            buf[C::O_Q + a * M * Mo + qo] = T(-0.5) * wgt * (wn * ju + wj * au);
            buf[C::O_Q + (3 + a) * M * Mo + qo] = T(-0.25) * wgt * wj * ju;
            buf[C::O_Q + (6 + a) * M * Mo + qo] = hw * pj;
          }
        }
        __syncwarp();
        // 5. moments: over p1 (lines (f, p2)), then over p2 (lines (f, s))
        for (int L = lane; L < NM * M; L += 32) {
          const int f = L / M, p2 = L - f * M;
          T q[M];
#pragma unroll
          for (int p1 = 0; p1 < M; ++p1) q[p1] = buf[C::O_Q + L * Mo + p1];
#pragma unroll
          for (int s = 0; s < K1; ++s) {
            T acc = T(0);
#pragma unroll
            for (int p1 = 0; p1 < M; ++p1) acc = fma(t1.b(p1, s), q[p1], acc);
            buf[C::O_U + (f * K1 + s) * Mo + p2] = acc;
          }
        }
        __syncwarp();
        for (int L = lane; L < NM * K1; L += 32) {
          const int f = L / K1, s = L - f * K1;
          T u[M];
#pragma unroll
          for (int p2 = 0; p2 < M; ++p2) u[p2] = buf[C::O_U + L * Mo + p2];
#pragma unroll
          for (int tt = 0; tt < K1; ++tt) {
            T acc = T(0);
#pragma unroll
            for (int p2 = 0; p2 < M; ++p2) acc = fma(t1.b(p2, tt), u[p2], acc);
            buf[C::O_MO + f * NFM + s + K1 * tt] = acc;
          }
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
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const T sv = mo[a * NFM], tv = mo[(3 + a) * NFM];
            outA[a * NFM + mm] = aF * (sv + tv + ph[a]);
            if (outB) outB[a * NFM + mm] = aF * (sv - tv - ph[a]);
          }
        }
        __syncwarp();
      }  // ETA
    }  // sub-facets
  }
  if (diss_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
    if (lane == 0) diss_part[(int64_t)blockIdx.x * C::WARPS + warp] = dacc;
  }
}

template <typename T, int K>
struct Vol {
  using S = Shape<K>;
  static constexpr int K1 = S::K1, M = S::M, NB = S::NB, NQ = S::NQ, NFM = S::NFM;
  static constexpr int K1o = K1 | 1, Mo = M | 1;  // odd line strides: no bank conflicts
  static constexpr int WARPS = 4;
  static constexpr bool REG = sizeof(T) == 4;
  // one field's coefficients [line (i2,i3)][i1] | x-pass B, D [line (q1,i3)][i2] | y-pass BB,
  // BD, DB [line (q1,q2)][i3] | wind at the points [4][NQ] | test pass over q3 of one
  // component [line (q1,i3)][q2]; the test pass over q2 reuses the x region
  static constexpr int XS = K1 * M * K1o;
  static constexpr int YS = M * M * K1o;
  static constexpr int O_C = 0;
  static constexpr int O_X = O_C + K1 * K1 * K1o;
  static constexpr int O_Y = O_X + 2 * XS;
  static constexpr int O_W = O_Y + 3 * YS;
  static constexpr int O_G = O_W + 4 * NQ;
  static constexpr int PER_WARP = O_G + K1 * M * Mo;
  static constexpr int TAB = 2 * M * K1 + M + 4 * K1;
  static constexpr size_t SMEM = size_t(TAB + WARPS * PER_WARP) * sizeof(T);
  static_assert(K1 * K1 * Mo <= 2 * XS, "test pass over q2 in the x region");
  static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
};

// x- and y-pass of one field (its coefficients in C): B and D over i1, then BB, BD (from B)
// and DB (from D) over i2.  Lanes own lines of the tensor.
template <typename T, int K, bool REG>
__device__ __forceinline__ void interp_xy(const Tab1<T, K, REG>& tb, T* base, int lane) {
  using C = Vol<T, K>;
  constexpr int K1 = C::K1, M = C::M, K1o = C::K1o;
  const T* Cf = base + C::O_C;
  T* XB = base + C::O_X;
  T* XD = XB + C::XS;
  for (int line = lane; line < K1 * K1; line += 32) {
    const int i2 = line % K1, i3 = line / K1;
    T c[K1];
#pragma unroll
    for (int i1 = 0; i1 < K1; ++i1) c[i1] = Cf[line * K1o + i1];
    T* xb = XB + i3 * M * K1o + i2;
    T* xd = XD + i3 * M * K1o + i2;
#pragma unroll
    for (int q1 = 0; q1 < M; ++q1) {
      T sb = T(0), sd = T(0);
#pragma unroll
      for (int i1 = 0; i1 < K1; ++i1) {
        sb = fma(tb.b(q1, i1), c[i1], sb);
        sd = fma(tb.d(q1, i1), c[i1], sd);
      }
      xb[q1 * K1o] = sb;
      xd[q1 * K1o] = sd;
    }
  }
  __syncwarp();
  T* YBB = base + C::O_Y;
  T* YBD = YBB + C::YS;
  T* YDB = YBD + C::YS;
  for (int line = lane; line < K1 * M; line += 32) {
    const int q1 = line % M, i3 = line / M;
    T xb[K1], xd[K1];
#pragma unroll
    for (int i2 = 0; i2 < K1; ++i2) {
      xb[i2] = XB[line * K1o + i2];
      xd[i2] = XD[line * K1o + i2];
    }
    const int o = q1 * K1o + i3;
#pragma unroll
    for (int q2 = 0; q2 < M; ++q2) {
      T bb = T(0), bd = T(0), db = T(0);
#pragma unroll
      for (int i2 = 0; i2 < K1; ++i2) {
        bb = fma(tb.b(q2, i2), xb[i2], bb);
        bd = fma(tb.d(q2, i2), xb[i2], bd);
        db = fma(tb.b(q2, i2), xd[i2], db);
      }
      YBB[o + q2 * M * K1o] = bb;
      YBD[o + q2 * M * K1o] = bd;
      YDB[o + q2 * M * K1o] = db;
    }
  }
  __syncwarp();
}

// z-pass at one line (q1, q2): value v and reference derivatives d1, d2, d3 at every q3
template <typename T, int K, bool REG>
__device__ __forceinline__ void interp_z(const Tab1<T, K, REG>& tb, const T* base, int line, T (&v)[Shape<K>::M],
                                         T (&d1)[Shape<K>::M], T (&d2)[Shape<K>::M], T (&d3)[Shape<K>::M]) {
  using C = Vol<T, K>;
  constexpr int K1 = C::K1, M = C::M, K1o = C::K1o;
  const T* YBB = base + C::O_Y + line * K1o;
  const T* YBD = YBB + C::YS;
  const T* YDB = YBD + C::YS;
  T bb[K1], bd[K1], db[K1];
#pragma unroll
  for (int i3 = 0; i3 < K1; ++i3) {
    bb[i3] = YBB[i3];
    bd[i3] = YBD[i3];
    db[i3] = YDB[i3];
  }
#pragma unroll
  for (int q3 = 0; q3 < M; ++q3) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
    for (int i3 = 0; i3 < K1; ++i3) {
      const T b = tb.b(q3, i3);
      a0 = fma(b, bb[i3], a0);
      a3 = fma(tb.d(q3, i3), bb[i3], a3);
      a2 = fma(b, bd[i3], a2);
      a1 = fma(b, db[i3], a1);
    }
    v[q3] = a0;
    d1[q3] = a1;
    d2[q3] = a2;
    d3[q3] = a3;
  }
}

// Volume kernel + lift of the six facets' moments + inverse mass + the stage combination:
//   y = (1/|det J|) (r_vol + r_fac),
//   r_vol[a][i] = sum_q w_q ( sum_c (G w)_c d^_c u_a + |det J| div w  u_a ) phi_i,  G = |det J| J^-1,
//   |det J| div w = sum_{c,b} G[c][b] d^_c w_b,
//   out = c0 u0 + c1 us + c2 y   (out may alias u0: each warp reads and writes its own cell).
// One warp per cell, one field at a time (w_0..2, then u_0..2); each pass is a set of
// one-dimensional contractions, a lane owning one line of the tensor (its inputs in
// registers, the 1D tables in registers in FP32).  The wind's z-pass accumulates G w and
// |det J| div w at the points; a velocity component's z-pass forms its integrand along the
// line and contracts it with phi over q3 at once, then the passes over q2 and q1 finish its
// test.  The values and reference derivatives are BBB, DBB, BDB, BBD.
template <typename T, int K>
__global__ void __launch_bounds__(32 * Vol<T, K>::WARPS)
    k_hex_volume(MeshDev m, Tabs<T> tb, const T* __restrict__ wL, const T* us, const T* __restrict__ gam,
                 const T* u0, T c0, T c1, T c2, T* out) {
  using C = Vol<T, K>;
  constexpr int K1 = C::K1, M = C::M, NB = C::NB, NQ = C::NQ, NFM = C::NFM, K1o = C::K1o, Mo = C::Mo;
  constexpr int MM = M * M;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  stage_tabs<T, K>(tb, sm);
  __syncthreads();
  Tab1<T, K, C::REG> t1;
  t1.load(sm, sm + M * K1);
  const T* sW = sm + 2 * M * K1;
  const T* sE0 = sW + M;
  const T* sE1 = sE0 + K1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* base = sm + C::TAB + warp * C::PER_WARP;
  T* Cf = base + C::O_C;
  T* Wp = base + C::O_W;  // [4][NQ]: (G w)_0..2, |det J| div w
  T* Gz = base + C::O_G;  // [line (q1, i3)][q2]
  T* Hx = base + C::O_X;  // [line (i2, i3)][q1]
  // the next field's coefficients are loaded into registers while the current one is
  // processed (the first field of the warp's next cell after the last one)
  constexpr int NPRE = (NB + 31) / 32;
  const int64_t estep = (int64_t)gridDim.x * C::WARPS;
  T pre[NPRE];
  auto prefetch = [&](int64_t ee, int ff) {
    if (ee >= m.E) return;
    const T* src = (ff < 3 ? wL : us) + (ee * 3 + (ff < 3 ? ff : ff - 3)) * NB;
#pragma unroll
    for (int j = 0; j < NPRE; ++j) {
      const int i = lane + 32 * j;
      if (i < NB) pre[j] = src[i];
    }
  };
  prefetch((int64_t)blockIdx.x * C::WARPS + warp, 0);
  for (int64_t e = (int64_t)blockIdx.x * C::WARPS + warp; e < m.E; e += estep) {
    T G[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) G[j] = T(m.G[e * 9 + j]);
    const T ia = T(m.invabs[e]);
    int64_t fA[3], fB[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      fB[d] = d * m.E + e;
      fA[d] = d * m.E + cell_shift(m, e, d, 1);
    }
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      const bool wind = f < 3;
      const int comp = wind ? f : f - 3;
#pragma unroll
      for (int j = 0; j < NPRE; ++j) {
        const int i = lane + 32 * j;
        if (i < NB) Cf[(i / K1) * K1o + i % K1] = pre[j];
      }
      __syncwarp();
      if (f < 5) prefetch(e, f + 1);
      else prefetch(e + estep, 0);
      interp_xy<T, K, C::REG>(t1, base, lane);
      // column comp of G (selects, not an indexed load)
      const T gc0 = comp == 0 ? G[0] : (comp == 1 ? G[1] : G[2]);
      const T gc1 = comp == 0 ? G[3] : (comp == 1 ? G[4] : G[5]);
      const T gc2 = comp == 0 ? G[6] : (comp == 1 ? G[7] : G[8]);
      for (int line = lane; line < MM; line += 32) {
        T v[M], d1[M], d2[M], d3[M];
        interp_z<T, K, C::REG>(t1, base, line, v, d1, d2, d3);
        if (wind) {
#pragma unroll
          for (int q3 = 0; q3 < M; ++q3) {
            const int q = line + q3 * MM;
            const T W0 = gc0 * v[q3], W1 = gc1 * v[q3], W2 = gc2 * v[q3];
            const T dv = fma(gc0, d1[q3], fma(gc1, d2[q3], gc2 * d3[q3]));
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
          }
        } else {
          const int q1 = line % M, q2 = line / M;
          const T w12 = sW[q1] * sW[q2];
          T fz[M];
#pragma unroll
          for (int q3 = 0; q3 < M; ++q3) {
            const int q = line + q3 * MM;
            const T s = Wp[q] * d1[q3] + Wp[NQ + q] * d2[q3] + Wp[2 * NQ + q] * d3[q3] + Wp[3 * NQ + q] * v[q3];
            fz[q3] = (w12 * sW[q3]) * s;
          }
          // test over q3
#pragma unroll
          for (int i3 = 0; i3 < K1; ++i3) {
            T acc = T(0);
#pragma unroll
            for (int q3 = 0; q3 < M; ++q3) acc = fma(t1.b(q3, i3), fz[q3], acc);
            Gz[(q1 + M * i3) * Mo + q2] = acc;
          }
        }
      }
      __syncwarp();
      if (wind) continue;
      // test over q2 (lines (q1, i3)), then over q1 (lines (i2, i3)) + lift + epilogue
      for (int line = lane; line < K1 * M; line += 32) {
        const int q1 = line % M, i3 = line / M;
        T g[M];
#pragma unroll
        for (int q2 = 0; q2 < M; ++q2) g[q2] = Gz[line * Mo + q2];
#pragma unroll
        for (int i2 = 0; i2 < K1; ++i2) {
          T acc = T(0);
#pragma unroll
          for (int q2 = 0; q2 < M; ++q2) acc = fma(t1.b(q2, i2), g[q2], acc);
          Hx[(i2 + K1 * i3) * Mo + q1] = acc;
        }
      }
      __syncwarp();
      const int a = comp;
      for (int line = lane; line < K1 * K1; line += 32) {
        const int i2 = line % K1, i3 = line / K1;
        T h[M];
#pragma unroll
        for (int q1 = 0; q1 < M; ++q1) h[q1] = Hx[line * Mo + q1];
        // facet moments: direction 0 -> mode (i2, i3), 1 -> (i1, i3), 2 -> (i1, i2)
        const T f0A = gam[(fA[0] * 6 + a) * NFM + i2 + K1 * i3];
        const T f0B = gam[(fB[0] * 6 + 3 + a) * NFM + i2 + K1 * i3];
        const T* gA1 = gam + (fA[1] * 6 + a) * NFM + K1 * i3;
        const T* gB1 = gam + (fB[1] * 6 + 3 + a) * NFM + K1 * i3;
        const T* gA2 = gam + (fA[2] * 6 + a) * NFM + K1 * i2;
        const T* gB2 = gam + (fB[2] * 6 + 3 + a) * NFM + K1 * i2;
        const T l1 = sE1[i2], l0 = sE0[i2], m1 = sE1[i3], m0 = sE0[i3];
#pragma unroll
        for (int i1 = 0; i1 < K1; ++i1) {
          T r = T(0);
#pragma unroll
          for (int q1 = 0; q1 < M; ++q1) r = fma(t1.b(q1, i1), h[q1], r);
          r += sE1[i1] * f0A + sE0[i1] * f0B;
          r += l1 * gA1[i1] + l0 * gB1[i1];
          r += m1 * gA2[i1] + m0 * gB2[i1];
          const int64_t o = (e * 3 + a) * NB + i1 + K1 * line;
          T v = c2 * (r * ia);
          if (c1 != T(0)) v += c1 * us[o];
          if (c0 != T(0)) v += c0 * u0[o];
          out[o] = v;
        }
      }
      __syncwarp();
    }
  }
}

// The volume kernel when the wind is the convected field (w = u, a STAGE substep): the three
// components pass through x and y once (batched), and one z-pass per line of points forms,
// point by point, the values and reference derivatives of all three, G u, |det J| div u, the
// three integrands and their test over q3; the passes over q2 and q1, the lift, the inverse
// mass and the stage combination follow as in k_hex_volume.  Half the interpolation work.
template <typename T, int K>
struct VolS {
  using S = Shape<K>;
  static constexpr int K1 = S::K1, M = S::M, NB = S::NB, NQ = S::NQ, NFM = S::NFM;
  static constexpr int K1o = K1 | 1, Mo = M | 1;
  static constexpr int WARPS = sizeof(T) == 8 ? 2 : 4;
  static constexpr bool REG = sizeof(T) == 4;
  static constexpr int CS = K1 * K1 * K1o;  // one field's coefficients [line (i2,i3)][i1]
  static constexpr int XS = K1 * M * K1o;   // one x-pass output [line (q1,i3)][i2]
  static constexpr int YS = M * M * K1o;    // one y-pass output [line (q1,q2)][i3]
  static constexpr int GS = K1 * M * Mo;    // one test pass over q3 [line (q1,i3)][q2]
  // buffers by lifetime: the x region holds the x-pass outputs, then the test pass over q3;
  // the y region the cell's coefficients, then the y-pass outputs, then the test pass over q2
  static constexpr int O_X = 0;                 // [f][B|D], then [a] test over q3
  static constexpr int O_Y = O_X + 6 * XS;      // coefficients, then [f][BB|BD|DB], then [a] test over q2
  static constexpr int O_C = O_Y;
  static constexpr int O_G = O_X;
  static constexpr int PER_WARP = O_Y + 9 * YS;
  static constexpr int TAB = 2 * M * K1 + M + 4 * K1;
  static constexpr size_t SMEM = size_t(TAB + WARPS * PER_WARP) * sizeof(T);
  static_assert(3 * CS <= 9 * YS, "coefficients in the y region");
  static_assert(3 * GS <= 6 * XS, "test pass over q3 in the x region");
  static_assert(3 * K1 * K1 * Mo <= 9 * YS, "test pass over q2 in the y region");
  static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
};

template <typename T, int K>
__global__ void __launch_bounds__(32 * VolS<T, K>::WARPS)
    k_hex_volume_same(MeshDev m, Tabs<T> tb, const T* us, const T* __restrict__ gam, const T* u0, T c0, T c1,
                      T c2, T* out) {
  using C = VolS<T, K>;
  constexpr int K1 = C::K1, M = C::M, NB = C::NB, NFM = C::NFM, K1o = C::K1o, Mo = C::Mo;
  constexpr int MM = M * M, XS = C::XS, YS = C::YS, GS = C::GS, CS = C::CS;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  stage_tabs<T, K>(tb, sm);
  __syncthreads();
  Tab1<T, K, C::REG> t1;
  t1.load(sm, sm + M * K1);
  const T* sW = sm + 2 * M * K1;
  const T* sE0 = sW + M;
  const T* sE1 = sE0 + K1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* base = sm + C::TAB + warp * C::PER_WARP;
  T* Cf = base + C::O_C;
  T* X = base + C::O_X;
  T* Y = base + C::O_Y;
  T* Gz = base + C::O_G;
  T* Hx = Y;  // [a][line (i2, i3)][q1]
  constexpr int NPRE = (3 * NB + 31) / 32;
  const int64_t estep = (int64_t)gridDim.x * C::WARPS;
  T pre[NPRE];
  auto prefetch = [&](int64_t ee) {
    if (ee >= m.E) return;
#pragma unroll
    for (int j = 0; j < NPRE; ++j) {
      const int t = lane + 32 * j;
      if (t < 3 * NB) pre[j] = us[ee * 3 * NB + t];
    }
  };
  prefetch((int64_t)blockIdx.x * C::WARPS + warp);
  for (int64_t e = (int64_t)blockIdx.x * C::WARPS + warp; e < m.E; e += estep) {
    T G[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) G[j] = T(m.G[e * 9 + j]);
    const T ia = T(m.invabs[e]);
    int64_t fA[3], fB[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      fB[d] = d * m.E + e;
      fA[d] = d * m.E + cell_shift(m, e, d, 1);
    }
#pragma unroll
    for (int j = 0; j < NPRE; ++j) {
      const int t = lane + 32 * j;
      if (t < 3 * NB) {
        const int f = t / NB, i = t - f * NB;
        Cf[f * CS + (i / K1) * K1o + i % K1] = pre[j];
      }
    }
    __syncwarp();
    prefetch(e + estep);
    // x-pass (lines (f, i2, i3)): B and D over i1
    for (int L = lane; L < 3 * K1 * K1; L += 32) {
      const int f = L / (K1 * K1), line = L - f * K1 * K1, i2 = line % K1, i3 = line / K1;
      T c[K1];
#pragma unroll
      for (int i1 = 0; i1 < K1; ++i1) c[i1] = Cf[f * CS + line * K1o + i1];
      T* xb = X + 2 * f * XS + i3 * M * K1o + i2;
#pragma unroll
      for (int q1 = 0; q1 < M; ++q1) {
        T sb = T(0), sd = T(0);
#pragma unroll
        for (int i1 = 0; i1 < K1; ++i1) {
          sb = fma(t1.b(q1, i1), c[i1], sb);
          sd = fma(t1.d(q1, i1), c[i1], sd);
        }
        xb[q1 * K1o] = sb;
        xb[XS + q1 * K1o] = sd;
      }
    }
    __syncwarp();
    // y-pass (lines (f, q1, i3)): BB, BD, DB over i2
    for (int L = lane; L < 3 * K1 * M; L += 32) {
      const int f = L / (K1 * M), line = L - f * K1 * M, q1 = line % M, i3 = line / M;
      T xb[K1], xd[K1];
#pragma unroll
      for (int i2 = 0; i2 < K1; ++i2) {
        xb[i2] = X[2 * f * XS + line * K1o + i2];
        xd[i2] = X[(2 * f + 1) * XS + line * K1o + i2];
      }
      T* y = Y + 3 * f * YS + q1 * K1o + i3;
#pragma unroll
      for (int q2 = 0; q2 < M; ++q2) {
        T bb = T(0), bd = T(0), db = T(0);
#pragma unroll
        for (int i2 = 0; i2 < K1; ++i2) {
          bb = fma(t1.b(q2, i2), xb[i2], bb);
          bd = fma(t1.d(q2, i2), xb[i2], bd);
          db = fma(t1.b(q2, i2), xd[i2], db);
        }
        y[q2 * M * K1o] = bb;
        y[YS + q2 * M * K1o] = bd;
        y[2 * YS + q2 * M * K1o] = db;
      }
    }
    __syncwarp();
    // z-pass (lines (q1, q2)), point by point: values and derivatives of the three
    // components, G u, |det J| div u, the integrands and their test over q3
    for (int line = lane; line < MM; line += 32) {
      const int q1 = line % M, q2 = line / M;
      const T w12 = sW[q1] * sW[q2];
      T in[3][3][K1];  // [component][BB, BD, DB][i3]
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
          for (int i3 = 0; i3 < K1; ++i3) in[f][o][i3] = Y[(3 * f + o) * YS + line * K1o + i3];
      T acc[3][K1];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i3 = 0; i3 < K1; ++i3) acc[a][i3] = T(0);
#pragma unroll
      for (int q3 = 0; q3 < M; ++q3) {
        T v[3], d1[3], d2[3], d3[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
          for (int i3 = 0; i3 < K1; ++i3) {
            const T b = t1.b(q3, i3);
            a0 = fma(b, in[f][0][i3], a0);
            a3 = fma(t1.d(q3, i3), in[f][0][i3], a3);
            a2 = fma(b, in[f][1][i3], a2);
            a1 = fma(b, in[f][2][i3], a1);
          }
          v[f] = a0;
          d1[f] = a1;
          d2[f] = a2;
          d3[f] = a3;
        }
        const T W0 = G[0] * v[0] + G[1] * v[1] + G[2] * v[2];
        const T W1 = G[3] * v[0] + G[4] * v[1] + G[5] * v[2];
        const T W2 = G[6] * v[0] + G[7] * v[1] + G[8] * v[2];
        T dv = T(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) dv += G[b] * d1[b] + G[3 + b] * d2[b] + G[6 + b] * d3[b];
        const T wq = w12 * sW[q3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T fz = wq * (W0 * d1[a] + W1 * d2[a] + W2 * d3[a] + dv * v[a]);
#pragma unroll
          for (int i3 = 0; i3 < K1; ++i3) acc[a][i3] = fma(t1.b(q3, i3), fz, acc[a][i3]);
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i3 = 0; i3 < K1; ++i3) Gz[a * GS + (q1 + M * i3) * Mo + q2] = acc[a][i3];
    }
    __syncwarp();
    // test over q2 (lines (a, q1, i3))
    for (int L = lane; L < 3 * K1 * M; L += 32) {
      const int a = L / (K1 * M), line = L - a * K1 * M, q1 = line % M, i3 = line / M;
      T g[M];
#pragma unroll
      for (int q2 = 0; q2 < M; ++q2) g[q2] = Gz[a * GS + line * Mo + q2];
#pragma unroll
      for (int i2 = 0; i2 < K1; ++i2) {
        T s = T(0);
#pragma unroll
        for (int q2 = 0; q2 < M; ++q2) s = fma(t1.b(q2, i2), g[q2], s);
        Hx[(a * K1 * K1 + i2 + K1 * i3) * Mo + q1] = s;
      }
    }
    __syncwarp();
    // test over q1 (lines (a, i2, i3)) + lift + inverse mass + stage combination
    for (int L = lane; L < 3 * K1 * K1; L += 32) {
      const int a = L / (K1 * K1), line = L - a * K1 * K1, i2 = line % K1, i3 = line / K1;
      T h[M];
#pragma unroll
      for (int q1 = 0; q1 < M; ++q1) h[q1] = Hx[(a * K1 * K1 + line) * Mo + q1];
      const T f0A = gam[(fA[0] * 6 + a) * NFM + i2 + K1 * i3];
      const T f0B = gam[(fB[0] * 6 + 3 + a) * NFM + i2 + K1 * i3];
      const T* gA1 = gam + (fA[1] * 6 + a) * NFM + K1 * i3;
      const T* gB1 = gam + (fB[1] * 6 + 3 + a) * NFM + K1 * i3;
      const T* gA2 = gam + (fA[2] * 6 + a) * NFM + K1 * i2;
      const T* gB2 = gam + (fB[2] * 6 + 3 + a) * NFM + K1 * i2;
      const T l1 = sE1[i2], l0 = sE0[i2], m1 = sE1[i3], m0 = sE0[i3];
#pragma unroll
      for (int i1 = 0; i1 < K1; ++i1) {
        T r = T(0);
#pragma unroll
        for (int q1 = 0; q1 < M; ++q1) r = fma(t1.b(q1, i1), h[q1], r);
        r += sE1[i1] * f0A + sE0[i1] * f0B;
        r += l1 * gA1[i1] + l0 * gB1[i1];
        r += m1 * gA2[i1] + m0 * gB2[i1];
        const int64_t o = (e * 3 + a) * NB + i1 + K1 * line;
        T v = c2 * (r * ia);
        if (c1 != T(0)) v += c1 * us[o];
        if (c0 != T(0)) v += c0 * u0[o];
        out[o] = v;
      }
    }
    __syncwarp();
  }
}

// FP64 reductions over the cells (row a8): part[2 block + 0] = sum |det J| |u|^2 and
// part[2 block + 1] = sum |det J| u . y over the block's cells (y = M^-1 c(w; u, .), so the
// latter is c(w; u, u)); the host adds the per-block partials in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_hex_energy(MeshDev m, int64_t nl, const T* __restrict__ u,
                                                   const T* __restrict__ y, double* __restrict__ part) {
  __shared__ double s0[8], s1[8];
  double a0 = 0.0, a1 = 0.0;
  const int64_t per = nl / m.E;  // 3 (k+1)^3 coefficients per cell
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += (int64_t)gridDim.x * blockDim.x) {
    const double ad = 1.0 / m.invabs[t / per];
    const double uv = u[t];
    a0 += ad * uv * uv;
    if (y) a1 += ad * uv * double(y[t]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s0[warp] = a0;
    s1[warp] = a1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = 0.0, b1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      b0 += s0[w];
      b1 += s1[w];
    }
    part[2 * blockIdx.x] = b0;
    part[2 * blockIdx.x + 1] = b1;
  }
}

}  // namespace hex
}  // namespace hopu
