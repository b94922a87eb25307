// Internal interface between the C ABI (capi.cu) and the per-(dim, k, precision)
// kernel families (ops_*.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hopu {

// Device view of the mesh (FP64 geometry, int32 connectivity).
struct DevMesh {
  int64_t E = 0, NF = 0;
  const double* geo = nullptr;   // [E][2d^2+2]: J (row-major), Jinv, det J, |det J| (FP64)
  const double* geoT = nullptr;  // [E][geoT_stride(d)] FP64 in every precision mode (the FP32 kernels
                                 // round each factor when they load it):
                                 //   Pf = J / det J, Pi = det J * Jinv, M = |det J| * Jinv, 1/|det J|
  const int32_t* efc = nullptr;  // [E][d+1]: F*4 + (sigma<0)*2 + (element is side B)
  const int32_t* fa = nullptr;   // [NF]: element*4 + local facet of side A
  const int32_t* fb = nullptr;   // [NF]: same for side B
  const double* fgeo = nullptr;  // [NF][d+1]: canonical unit normal n_F, a_F = |F|/|param|
  int* err = nullptr;            // device error word (bits 0 / 1 / 3: a completion wait of the
                                 // tensor-core projection / volume / back-projection kernel gave
                                 // up; bit 2: element ids out of range in pack / unpack)
  uint32_t tc_wait_limit = 1u << 22;  // polls of the tensor-core MMA completion waits (hopu_set_wait_limit)
  // boundary facets have fb[F] == fa[F] (wall / outlet rule: the exterior trace is the
  // interior one); inlet facets also have inlet[F] >= 0, the row of their exterior data
  const int32_t* inlet = nullptr;  // [NF] or NULL (no inlets)
  const void* inlet_modes = nullptr;  // [n_inlet][nf][d] modal exterior trace, working precision
};

// Device reference tables in working precision (all element-type T, 16-byte aligned).
struct DevTabs {
  const void* Bt = nullptr;     // [nq][nbq]       phi_i(x_q), point-major, rows padded to nbq
  const void* dBt = nullptr;    // [d][nq][nbq]    d phi_i / d xhat_c (x_q), same layout as Bt
                                //                 (an odd multiple of 16 bytes)
  const void* Wq = nullptr;     // [nq]            volume weights
  const void* Dm = nullptr;     // [d][nb(k-1)][nb] d phi_i / d xhat_c = sum_j Dm[c][j][i] phi_j
  const void* TrM = nullptr;    // [d+1][nf][nb]   <phi_i o xhat_f, psi_m>_facet
  const void* TrP = nullptr;    // [d+1][nqf][nbq] phi_i(xhat_f(s_q)), point-major
  const void* Psi = nullptr;    // [nf][nqf]       psi_m(s_q)
  const void* WPsi = nullptr;   // [nf][nqf]       w_q psi_m(s_q)
  const void* Wf = nullptr;     // [nqf]           facet weights
  const void* DinvT = nullptr;  // [nloc][nlp]     DinvT[s][r] = Dinv[r][s]  (nlp = nloc rounded up to 4)
  const void* Dcsr = nullptr;   // FP32: the nonzeros of D by rows, 16-byte entries (layout in
                                //   k_v2l / warp_tile_residual); csr_n entries in all
  int csr_n = 0;
  const void* Dcsr_tc = nullptr;  // FP32_TC: the same with grouped rows (rows whose component blocks are
  int csr_tc_n = 0;               //   equal keep block 0 only, flag 1 in the header's fourth word)
  const void* DT = nullptr;     // [nloc][nlp]     DT[s][r]    = D[r][s]
  const void* Dinv = nullptr;   // [nloc][nlp]     Dinv[s][r]
  const void* Dn = nullptr;     // [nloc][nlp]     Dn[s][r] = D[s][r]
  const void* tcvol = nullptr;  // FP32 tensor-core volume tables (phi in the two operand layouts,
                                //   TF32 hi and lo parts), or NULL
  const void* Drow = nullptr;   // [nloc][nlr]     D[r][s] row-major, rows padded to nlr (an odd
                                //                 multiple of 16 bytes), zero padding
  const void* tcv2l = nullptr;  // FP32 3xTF32 refined projection table (Dinv as the B operand,
                                //   TF32 hi and lo parts, layout of V2lTcr), or NULL
  const void* tcl2v = nullptr;  // FP32 tensor-core back-projection table (D as the B operand,
                                //   TF32 hi and lo parts, layout of L2vTc), or NULL
};

// out = a0*x0 + a1*x1 + a2*v  (x0 / x1 may be null; out may alias x0 or x1).
// In FP32 every coefficient is applied as the sum of two floats (hi = float(a),
// lo = float(a - hi)), so the combination weights keep FP64 accuracy: with plain
// float weights the SSP-RK3 weights float(1/3) + float(2/3) = 1 + 3e-8 would scale the
// state by that factor in every substep.
struct Combine {
  double a0 = 0.0;
  const void* x0 = nullptr;
  double a1 = 0.0;
  const void* x1 = nullptr;
  double a2 = 1.0;
  float h0 = float(a0), l0 = float(a0 - double(float(a0)));
  float h1 = float(a1), l1 = float(a1 - double(float(a1)));
  float h2 = float(a2), l2 = float(a2 - double(float(a2)));
};

// thresholds eta_0 < ... < eta_k of the adaptive HOPU order rule (k + 1 <= 6 values)
struct EtaThresholds {
  double t[6];
};

// K layout of the tensor-core back-projection (k_l2v_tc and its host table): the basis
// indices are split into 4 groups of IPG (one warp group each); group g owns the GW
// consecutive K columns g GW + b IPG + t for component b and basis index i = g IPG + t,
// zero-padded to a multiple of 4; K = 4 GW; N = nloc padded to 16.
inline constexpr int l2v_tc_ipg(int nb) { return (nb + 3) / 4; }
inline constexpr int l2v_tc_gw(int d, int nb) { return (d * l2v_tc_ipg(nb) + 3) / 4 * 4; }
inline constexpr int l2v_tc_kp(int d, int nb) { return 4 * l2v_tc_gw(d, nb); }
inline constexpr int l2v_tc_np(int nloc) { return (nloc + 15) / 16 * 16; }

// K layout of the refined tensor-core projection (k_v2l_tcr and its host table): the rows h
// of the sorted dof-matrix CSR (csr_row_order) are dealt to 4 warp groups, h = g + 4 j;
// group g owns the RPG rows j and the K columns g GW + j (zero-padded to GW, a multiple
// of 4); K = 4 GW; N = nloc padded to 16.
inline constexpr int v2l_tc_rpg(int nloc) { return (nloc + 3) / 4; }
inline constexpr int v2l_tc_gw(int nloc) { return (v2l_tc_rpg(nloc) + 3) / 4 * 4; }
inline constexpr int v2l_tc_kp(int nloc) { return 4 * v2l_tc_gw(nloc); }

// layout of the working-precision geometry record (offsets in elements)
inline constexpr int geoT_stride(int d) { return ((3 * d * d + 1 + 3) / 4) * 4; }

// Points of the compact volume rule the volume kernels use (exact to degree 3k - 1; the
// tables are in volume_rules.h), or 0 where they use the collapsed Gauss-Jacobi rule.
inline constexpr int compact_volume_points(int d, int k) {
  return d != 3 ? 0 : k == 3 ? 46 : k == 4 ? 100 : k == 5 ? 190 : 0;
}

enum VolumeVariant {
  kVolRegFused = 0,   // register kernel, back-projection fused
  kVolRegSplit = 1,   // register kernel + separate back-projection
  kVolWarpFused = 2,  // warp-per-element kernel, back-projection fused
  kVolTensor = 3,     // tensor-core kernel
  kVolRegTab = 4,     // register kernel with reference-gradient tables + separate back-projection
  kVolRegHalf = 5,    // register kernel, basis split over two lanes + separate back-projection
  kVolVariants = 6
};

// One family of kernels for a fixed (dim, k, precision).  Every call enqueues on the
// given stream and returns the number of kernels it launched.
class Ops {
 public:
  virtual ~Ops() {}
  virtual cudaError_t prepare() = 0;
  // launch configuration that depends on the uploaded tables (after prepare)
  virtual cudaError_t configure(const DevTabs&) = 0;
  // E: V_h -> L2
  virtual int v2l(const DevMesh&, const DevTabs&, const void* uV, void* uL, cudaStream_t) = 0;
  // facet flux moments, element-major: gam[e][f][nf][d] for the element e that sees the
  // facet as its local facet f (alpha + beta on side A, alpha - beta on side B) and, if
  // diss is not null, the facet dissipation per facet.  wL == uL means w = u.
  virtual int facet(const DevMesh&, const DevTabs&, const void* uL, const void* wL, int l,
                    const int8_t* facet_l, void* gam, double* diss, cudaStream_t) = 0;
  // volume term + facet lift + inverse mass, combined into out.  wL == uL means w = u.
  virtual int volume(const DevMesh&, const DevTabs&, const void* uL, const void* wL,
                     const void* gam, Combine c, void* out, cudaStream_t) = 0;
  // volume kernel with the element part of R E^{-1} fused into its epilogue (w = u
  // only): writes the combined interior V_h dofs into outV and the local facet
  // functionals into lf.  Returns 0 (nothing launched) when this family has no fused
  // variant; the caller then runs volume + l2v_elem.
  virtual int volume_l2v(const DevMesh&, const DevTabs&, const void* uL, const void* gam, void* lf,
                         Combine c, void* outV, cudaStream_t) = 0;
  virtual bool has_fused() const = 0;
  virtual bool tensor_cores() const = 0;  // the V_h -> L2 projection runs on tensor cores
  virtual bool tensor_core_volume() const = 0;  // a tensor-core fused STAGE volume kernel exists
  // variant choice per kernel family (autotuner): 0 = FP32 FMA kernel, 1 = tensor-core kernel
  virtual void select(int v2l_tc, int volume_tc) = 0;
  virtual int selected_v2l() const = 0;
  virtual int selected_volume() const = 0;
  // kernel variants of the element part of a STAGE stage (volume term, lift, inverse mass,
  // element back-projection), VolumeVariant; the autotuner times the available ones and
  // selects one
  virtual bool volume_variant_ok(int v) const = 0;
  virtual void select_volume_variant(int v) = 0;
  virtual int volume_variant() const = 0;
  // adjoint kernels: (R E_T^{-1})^T, the facet and the volume parts of the VJP of the
  // apply (ybar = cotangent of y; wL == uL means w = u and the cotangents are summed
  // into ubar, wbar unused); gamU / gamW are element-major facet-moment scratch.
  // adaptive HOPU: eta per facet with the current orders, new orders written in place
  virtual int eta(const DevMesh&, const DevTabs&, const void* uL, int l, int8_t* facet_l,
                  const EtaThresholds& th, double* eta_out, cudaStream_t) = 0;
  virtual int v2l_pt(const DevMesh&, const DevTabs&, const void* vV, void* yL, cudaStream_t) = 0;
  virtual int facet_adj(const DevMesh&, const DevTabs&, const void* uL, const void* wL, const void* ybar,
                        int l, const int8_t* facet_l, void* gamU, void* gamW, cudaStream_t) = 0;
  virtual int volume_adj(const DevMesh&, const DevTabs&, const void* uL, const void* wL, const void* ybar,
                         const void* gamU, const void* gamW, void* ubar, void* wbar, cudaStream_t) = 0;
  // R E^{-1} (dual = false) or E^T (dual = true), combined into outV, in two launches:
  // the element part writes interior dofs and the local facet functionals lf
  // [E][d+1][nf]; the facet part averages (or sums) the two copies into the facet dofs.
  virtual int l2v_elem(const DevMesh&, const DevTabs&, const void* yL, bool dual, void* lf,
                       Combine c, void* outV, cudaStream_t) = 0;
  virtual int l2v_facet(const DevMesh&, const void* lf, bool dual, Combine c, void* outV,
                        cudaStream_t) = 0;
  // the element part of R E^{-1} (not dual) on the tensor cores: available in the tensor-core
  // modes where the tiles fit; selected by the autotuner (1) or not (0)
  virtual bool tensor_core_l2v() const = 0;
  virtual void select_l2v(int tc) = 0;
  virtual int selected_l2v() const = 0;
};

Ops* make_ops(int dim, int k, bool fp64);

}  // namespace hopu
