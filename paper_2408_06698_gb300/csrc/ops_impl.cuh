// Launch wrappers of one kernel family (dimension D, order K, precision T).
#pragma once
#include <algorithm>
#include <type_traits>
#include <utility>

#include "kernels.cuh"
#include "kernels_adj.cuh"
#include "kernels_tc.cuh"
#include "kernels_tcr.cuh"
#include "kernels_adapt.cuh"
#include "kernels_vr.cuh"
#include "kernels_vrh.cuh"
#include "kernels_var.cuh"
#include "kernels_far.cuh"
#include "kernels_fr.cuh"

namespace hopu {

template <int D, int K, typename T>
class OpsImpl final : public Ops {
  using S = Shape<D, K>;
  static constexpr size_t kLimit = 200 * 1024;  // shared-memory budget per CTA
  static constexpr size_t sz = sizeof(T);
  static constexpr size_t r4(size_t n) { return ((n + 3) / 4) * 4; }

  using PW = ProjWCfg<D, K, T>;  // warp tiles of the projections
  // V_h -> L2 in FP32: the refined projection (its launch shape is set by configure())
  static constexpr bool kRef = std::is_same<T, float>::value;
  int ref_warps_ = 8, ref_staged_ = 0, csr_n_ = 0;
  size_t ref_smem_ = 0;

  // facet kernel: padded modal trace matrices, Psi, WPsi, Wf; per warp: coefficient
  // blocks, two [nqf][4] point buffers, modal jump / wind, moments (layout of k_facet)
  static constexpr size_t kNBQ = row_stride<T>(S::nb);
  static constexpr size_t kFacTab = r4(size_t(D + 1) * S::nf * r4(S::nb) + 2 * S::nf * S::nqf + S::nqf) * sz;
  static constexpr size_t facet_warp(bool wsep) {
    return (size_t(wsep ? 4 : 2) * D * r4(S::nb) + 2 * S::nqf * 4 + 2 * S::nf * 4 + 2 * S::nf * 4) * sz;
  }
  static constexpr bool kFacetTab = true;
  static constexpr size_t facet_smem(bool wsep) { return kFacTab + kWarps * facet_warp(wsep); }

  // volume kernel: Bt, Wq, Dm, TrM; per warp: coefficients, modal gradients, (W and its
  // divergence), signed facet moments (layout of k_volume)
  static constexpr int kNB1 = cnbasis(D, K - 1);
  static constexpr size_t kVolTab =  // Dm rows padded, Dm and TrM 16-byte aligned (layout of k_volume)
      r4(r4(r4(size_t(S::nq) * kNBQ + S::nq) + size_t(D) * kNB1 * r4(S::nb)) + size_t(D + 1) * S::nf * S::nb) * sz;
  static constexpr size_t volume_stage(bool wsep) {
    return r4(S::nloc) * (wsep ? 2 : 1) + r4(size_t(D + 1) * S::nf * D) + r4(S::gt * 8 / sz);  // FP64 geometry
  }
  static constexpr size_t volume_warp(bool wsep) {
    return (2 * volume_stage(wsep) + size_t(D) * r4(S::nb) + size_t(D) * D * r4(kNB1) +
            (wsep ? size_t(D) * r4(S::nb) + r4(kNB1) : 0)) * sz;
  }
  static constexpr bool kVolumeTab = kVolTab + kWarps * volume_warp(true) <= kLimit;
  static constexpr size_t volume_smem(bool wsep) { return (kVolumeTab ? kVolTab : 0) + kWarps * volume_warp(wsep); }
  using FC = FuseCfg<D, K, T>;
  static constexpr size_t kFuseTab = r4(size_t(FC::TAB)) * sz;
  static constexpr bool kFuse = kVolumeTab && FC::OK && kVolTab + kFuseTab + kWarps * volume_warp(false) <= kLimit;
  static constexpr size_t kFuseSmem = kVolTab + kFuseTab + kWarps * volume_warp(false);
  int g_fuse_ = 1;

  // adjoint kernels (layouts of k_facet_adj / k_volume_adj)
  static constexpr size_t facet_adj_warp(bool wsep) {
    return (size_t(wsep ? 6 : 4) * D * r4(S::nb) + 3 * S::nqf * 4 + 7 * S::nf * 4) * sz;
  }
  static constexpr size_t facet_adj_smem(bool wsep) { return kFacTab + kWarps * facet_adj_warp(wsep); }
  static constexpr size_t volume_adj_smem(bool wsep) {
    return kWarps * (2 * size_t(D) * r4(S::nb) + size_t(D) * D * r4(kNB1) + (wsep ? size_t(D) * r4(S::nb) : 0) +
                     2 * r4(size_t(D + 1) * S::nf * D)) * sz;
  }
  int g_fadj_ = 1, g_vadj_ = 1, g_eta_ = 1;
  static constexpr size_t eta_smem() {
    return (r4(size_t(D + 1) * S::nf * r4(S::nb) + S::nf * S::nqf + S::nqf) +
            kWarps * (2 * size_t(D) * r4(S::nb) + 2 * S::nf * 4)) * sz;
  }
  int nsm_ = 1;
  int tc_ = 0;  // FP32 only: 0 = FMA, 3 = 3xTF32 tensor cores, 1 = 1xTF32 tensor cores
  int g_v2l_tc_ = 1;
  static constexpr bool kTcV2l = std::is_same<T, float>::value && V2lTc<D, K>::OK;
  static constexpr bool kTcV2lR = std::is_same<T, float>::value && V2lTcr<D, K>::OK;
  int g_v2l_tcr_ = 1;
  bool tcr_fits_ = true;  // the CSR of D fits beside the refined tensor-core projection's tiles
  static constexpr bool kTcVol = std::is_same<T, float>::value && VolTc<D, K>::OK;
  int g_vol_tc_ = 1;
  static constexpr bool kTcL2v = std::is_same<T, float>::value && L2vTc<D, K>::OK;
  int g_l2v_tc_ = 1;
  bool use_tc_l2v_ = false;  // autotuner choice of the element back-projection
  bool use_tc_v2l_ = true;  // autotuner choice of the projection (TF32 mode)
  int vvar_ = -1;           // STAGE volume variant (VolumeVariant), -1: unfused warp-per-element
  // register-resident FP32 volume kernel (STAGE wind) where the lane's registers suffice
  static constexpr bool kVolR = std::is_same<T, float>::value && VolR<D, K>::OK;
  static constexpr bool kVolRF = std::is_same<T, float>::value && VolR<D, K>::FUSE_OK;
  static constexpr bool kVolRT = std::is_same<T, float>::value && VolR<D, K, true>::OK;
  int g_volrt_ = 1;
  // register kernel with the basis split over two lanes
  static constexpr bool kVolRH = std::is_same<T, float>::value && VolRH<D, K>::OK;
  int g_volrh_ = 1;
  // register-resident adjoint volume kernel (w = u)
  static constexpr bool kVolAR = std::is_same<T, float>::value && VolAR<D, K>::OK;
  int g_volar_ = 1;
  // register-resident adjoint facet kernel (w = u)
  static constexpr bool kFacAR = std::is_same<T, float>::value && FacAR<D, K>::OK;
  int g_facar_ = 1;
  int g_volr_ = 1, g_volrf_ = 1;
  // register-resident FP32 facet kernel
  static constexpr bool kFacR = std::is_same<T, float>::value && FacR<D, K>::OK;
  static constexpr bool kFacRW = std::is_same<T, float>::value && FacR<D, K>::OK_WSEP;
  int g_facr_[2] = {1, 1};
  int g_v2l_ = 1, g_v2lpt_ = 1, g_fac_[2] = {1, 1}, g_vol_[2] = {1, 1}, g_elem_[2] = {1, 1}, g_fsum_ = 1;

  template <typename Kern>
  cudaError_t setup(Kern kern, size_t smem, int threads, int* grid, bool max_carveout = false) {
    cudaError_t err = cudaSuccess;
    if (smem > 48 * 1024) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
    }
    if (max_carveout) {  // the largest shared-memory carveout, so that it does not cut occupancy
      err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      if (err != cudaSuccess) return err;
    }
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (err != cudaSuccess) return err;
    if (max_carveout) {  // resident blocks by shared memory, threads and registers
      int dev = 0, sm_smem = 0, reserved = 0;
      cudaFuncAttributes fa{};
      if (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
          cudaFuncGetAttributes(&fa, kern) == cudaSuccess) {
        const int by_smem = sm_smem / (int)(smem + fa.sharedSizeBytes + reserved);
        const int by_threads = 2048 / threads;
        const int by_regs = fa.numRegs > 0 ? 65536 / (fa.numRegs * threads) : by_threads;
        occ = std::max(occ, std::min(by_smem, std::min(by_threads, by_regs)));
      }
    }
    *grid = nsm_ * std::max(occ, 1);
    return cudaSuccess;
  }

  // Every launch of the family carries the programmatic-stream-serialization attribute
  // (the kernels wait for their predecessor after their prologue, see pdl_wait).
  template <typename... KArgs, typename... Args>
  static void launch(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  }

  static int clamp_grid(int g, int64_t items, int per_block) {
    const int64_t need = (items + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, need));
  }

 public:
  explicit OpsImpl(int tc = 0) : tc_(std::is_same<T, float>::value ? tc : 0) { vvar_ = default_volume_variant(); }
  // The V_h -> L2 change of basis on the tensor cores: one TF32 product in TF32 mode
  // (k_v2l_tc); in 3xTF32 mode the refined projection (k_v2l_tcr), whose two dense products
  // run on the tensor cores and whose compensated residual keeps the small high-degree
  // coefficients of smooth fields that a plain FP32 or 3xTF32 product loses.
  bool tensor_cores() const override { return (tc_ == 1 && kTcV2l) || (tc_ == 3 && kTcV2lR && tcr_fits_); }
  bool tensor_core_volume() const override { return tc_ != 0 && kTcVol; }
  void select(int v2l_tc, int volume_tc) override {
    use_tc_v2l_ = v2l_tc != 0 && tensor_cores();
    if (volume_tc != 0 && tensor_core_volume()) vvar_ = kVolTensor;
    else if (vvar_ == kVolTensor || vvar_ < 0) vvar_ = default_volume_variant();
  }
  int selected_v2l() const override { return (use_tc_v2l_ && tensor_cores()) ? 1 : 0; }
  int selected_volume() const override { return vvar_ == kVolTensor ? 1 : 0; }
  bool volume_variant_ok(int v) const override {
    switch (v) {
      case kVolRegFused: return kVolRF;
      case kVolRegSplit: return kVolR;
      case kVolWarpFused: return kFuse;
      case kVolTensor: return tensor_core_volume();
      case kVolRegTab: return kVolRT;
      case kVolRegHalf: return kVolRH;
      default: return false;
    }
  }
  void select_volume_variant(int v) override {
    if (volume_variant_ok(v)) vvar_ = v;
  }
  int volume_variant() const override { return vvar_; }
  int default_volume_variant() const {
    return kVolR ? kVolRegSplit : (kVolRH ? kVolRegHalf : (kFuse ? kVolWarpFused : -1));
  }

  cudaError_t prepare() override {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    const int th = 32 * kWarps;
    if constexpr (!kRef) {
      if ((err = setup(k_v2l<D, K, T, false>, PW::SMEM, 32 * PW::WARPS, &g_v2l_)) != cudaSuccess) return err;
    }
    if ((err = setup(k_v2l<D, K, T, true>, PW::SMEM, 32 * PW::WARPS, &g_v2lpt_)) != cudaSuccess) return err;
    if constexpr (kTcVol) {
      if (tc_ && (err = setup(k_volume_tc<D, K>, VolTc<D, K>::SMEM, VolTc<D, K>::THREADS, &g_vol_tc_, true)) !=
                     cudaSuccess)
        return err;
    }
    if constexpr (kTcV2l) {
      if (tc_ == 1) {
        err = setup(k_v2l_tc<D, K, false>, V2lTc<D, K>::SMEM, V2lTc<D, K>::THREADS, &g_v2l_tc_, true);
        if (err != cudaSuccess) return err;
      }
    }

    if constexpr (kTcL2v) {
      if (tc_) {
        err = tc_ == 3 ? setup(k_l2v_tc<D, K, true>, L2vTc<D, K>::SMEM, L2vTc<D, K>::THREADS, &g_l2v_tc_, true)
                       : setup(k_l2v_tc<D, K, false>, L2vTc<D, K>::SMEM, L2vTc<D, K>::THREADS, &g_l2v_tc_, true);
        if (err != cudaSuccess) return err;
      }
    }
    if ((err = setup(k_eta<D, K, T>, eta_smem(), th, &g_eta_)) != cudaSuccess) return err;
    if ((err = setup(k_facet_adj<D, K, T, false>, facet_adj_smem(false), th, &g_fadj_)) != cudaSuccess) return err;
    if ((err = setup(k_facet_adj<D, K, T, true>, facet_adj_smem(true), th, &g_fadj_)) != cudaSuccess) return err;
    if ((err = setup(k_volume_adj<D, K, T, false>, volume_adj_smem(false), th, &g_vadj_)) != cudaSuccess) return err;
    if ((err = setup(k_volume_adj<D, K, T, true>, volume_adj_smem(true), th, &g_vadj_)) != cudaSuccess) return err;
    if constexpr (kFacR) {
      using R = FacR<D, K>;
      if ((err = setup(k_facet_r<D, K, false>, R::SMEM, 32 * R::WARPS, &g_facr_[0])) != cudaSuccess) return err;
    }
    if constexpr (kFacRW) {
      using R = FacR<D, K>;
      if ((err = setup(k_facet_r<D, K, true>, R::SMEM, 32 * R::WARPS, &g_facr_[1])) != cudaSuccess) return err;
    }
    if ((err = setup(k_facet<D, K, T, false, kFacetTab>, facet_smem(false), th, &g_fac_[0])) != cudaSuccess) return err;
    if ((err = setup(k_facet<D, K, T, true, kFacetTab>, facet_smem(true), th, &g_fac_[1])) != cudaSuccess) return err;
    if ((err = setup(k_volume<D, K, T, false, kVolumeTab, false>, volume_smem(false), th, &g_vol_[0])) != cudaSuccess) return err;
    if ((err = setup(k_volume<D, K, T, true, kVolumeTab, false>, volume_smem(true), th, &g_vol_[1])) != cudaSuccess) return err;
    if constexpr (kVolR) {
      if ((err = setup(k_volume_r<D, K, false, false>, VolR<D, K>::SMEM, 32 * VolR<D, K>::WARPS, &g_volr_)) != cudaSuccess)
        return err;
    }
    if constexpr (kFacAR) {
      if ((err = setup(k_facet_adj_r<D, K>, FacAR<D, K>::SMEM, 32 * FacAR<D, K>::WARPS, &g_facar_)) != cudaSuccess)
        return err;
    }
    if constexpr (kVolAR) {
      if ((err = setup(k_volume_adj_r<D, K>, VolAR<D, K>::SMEM, 32 * VolAR<D, K>::WARPS, &g_volar_)) != cudaSuccess)
        return err;
    }
    if constexpr (kVolRH) {
      if ((err = setup(k_volume_rh<D, K>, VolRH<D, K>::SMEM, 32 * VolRH<D, K>::WARPS, &g_volrh_)) != cudaSuccess)
        return err;
    }
    if constexpr (kVolRT) {
      if ((err = setup(k_volume_r<D, K, false, true>, VolR<D, K, true>::SMEM, 32 * VolR<D, K, true>::WARPS,
                       &g_volrt_)) != cudaSuccess)
        return err;
    }
    if constexpr (kVolRF) {
      if ((err = setup(k_volume_r<D, K, true, false>, VolR<D, K>::SMEM_FUSE, 32 * VolR<D, K>::WARPS, &g_volrf_)) !=
          cudaSuccess)
        return err;
    }
    if constexpr (kFuse) {
      if ((err = setup(k_volume<D, K, T, false, true, true>, kFuseSmem, th, &g_fuse_)) != cudaSuccess) return err;
    }
    if ((err = setup(k_l2v_elem<D, K, T, false>, PW::SMEM, 32 * PW::WARPS, &g_elem_[0])) != cudaSuccess) return err;
    if ((err = setup(k_l2v_elem<D, K, T, true>, PW::SMEM, 32 * PW::WARPS, &g_elem_[1])) != cudaSuccess) return err;
    if ((err = setup(k_l2v_facet<D, K, T, false>, 0, 256, &g_fsum_)) != cudaSuccess) return err;
    return cudaSuccess;
  }

  // The refined FP32 projection stages the sparse rows of D and, when they fit, Dinv^T per
  // CTA; as many warps per CTA as fit in ~220 KB (16, 12, 8 or 4).
  cudaError_t configure(const DevTabs& t) override {
    if constexpr (kTcV2lR) {
      if (tc_ == 3) {
        const size_t sm = V2lTcr<D, K>::smem(t.csr_tc_n);
        tcr_fits_ = sm <= 227 * 1024;
        if (tcr_fits_) {
          cudaError_t err = setup(k_v2l_tcr<D, K>, sm, V2lTcr<D, K>::THREADS, &g_v2l_tcr_, true);
          if (err != cudaSuccess) return err;
        }
      }
    }
    if constexpr (kRef) {
      using R = ProjRCfg<D, K>;
      csr_n_ = t.csr_n;
      const size_t csr = size_t(csr_n_) * 16, tab = (R::TAB + 15) / 16 * 16;
      ref_staged_ = csr + tab + 8 * R::TILE <= 220 * 1024;
      const size_t fixed = csr + (ref_staged_ ? tab : 0);
      ref_warps_ = R::fit_warps(fixed);
      ref_smem_ = fixed + size_t(ref_warps_) * R::TILE;
      return setup(k_v2l<D, K, T, false>, ref_smem_, 32 * ref_warps_, &g_v2l_);
    }
    return cudaSuccess;
  }

  int v2l(const DevMesh& m, const DevTabs& t, const void* uV, void* uL, cudaStream_t st) override {
    if constexpr (kTcV2lR) {
      if (tc_ == 3 && tcr_fits_ && use_tc_v2l_ && t.tcv2l && t.Dcsr_tc) {
        const int g = clamp_grid(g_v2l_tcr_, m.E, V2lTcr<D, K>::TM);
        launch(k_v2l_tcr<D, K>, g, V2lTcr<D, K>::THREADS, V2lTcr<D, K>::smem(t.csr_tc_n), st, m,
               static_cast<const float*>(t.tcv2l), static_cast<const float4*>(t.Dcsr_tc), t.csr_tc_n,
               static_cast<const float*>(uV), static_cast<float*>(uL));
        return 1;
      }
    }
    if constexpr (kTcV2l) {
      if (tc_ == 1 && use_tc_v2l_) {
        const int g = clamp_grid(g_v2l_tc_, m.E, V2lTc<D, K>::TM);
        const int nlp = (S::nloc + 3) / 4 * 4;
        launch(k_v2l_tc<D, K, false>, g, V2lTc<D, K>::THREADS, V2lTc<D, K>::SMEM, st, m,
               static_cast<const float*>(t.Dinv), nlp, static_cast<const float*>(uV), static_cast<float*>(uL));
        return 1;
      }
    }
    if constexpr (kRef) {
      const int g = clamp_grid(g_v2l_, (m.E + PW::EW - 1) / PW::EW, 1);
      launch(k_v2l<D, K, T, false>, g, 32 * ref_warps_, ref_smem_, st, m, static_cast<const T*>(t.DinvT),
             static_cast<const float4*>(t.Dcsr), csr_n_, ref_staged_, static_cast<const T*>(uV),
             static_cast<T*>(uL));
    } else {
      const int g = clamp_grid(g_v2l_, (m.E + PW::EW - 1) / PW::EW, 1);
      launch(k_v2l<D, K, T, false>, g, 32 * PW::WARPS, PW::SMEM, st, m, static_cast<const T*>(t.DinvT),
             static_cast<const float4*>(nullptr), 0, 0, static_cast<const T*>(uV), static_cast<T*>(uL));
    }
    return 1;
  }

  int facet(const DevMesh& m, const DevTabs& t, const void* uL, const void* wL, int l,
            const int8_t* facet_l, void* gam, double* diss, cudaStream_t st) override {
    const bool wsep = (wL != nullptr && wL != uL);
    if constexpr (kFacRW) {
      if (wsep) {
        using R = FacR<D, K>;
        const int g = clamp_grid(g_facr_[1], (m.NF + R::FPW - 1) / R::FPW, 1);
        launch(k_facet_r<D, K, true>, g, 32 * R::WARPS, R::SMEM, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(wL), l, facet_l, static_cast<float*>(gam), diss);
        return 1;
      }
    }
    if constexpr (kFacR) {
      if (!wsep) {
        using R = FacR<D, K>;
        const int g = clamp_grid(g_facr_[0], (m.NF + R::FPW - 1) / R::FPW, 1);
        launch(k_facet_r<D, K, false>, g, 32 * R::WARPS, R::SMEM, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(uL), l, facet_l, static_cast<float*>(gam), diss);
        return 1;
      }
    }
    const int g = clamp_grid(g_fac_[wsep ? 1 : 0], m.NF, kWarps);
    if (wsep)
      launch(k_facet<D, K, T, true, kFacetTab>, g, 32 * kWarps, facet_smem(true), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(wL), l, facet_l, static_cast<T*>(gam), diss);
    else
      launch(k_facet<D, K, T, false, kFacetTab>, g, 32 * kWarps, facet_smem(false), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(uL), l, facet_l, static_cast<T*>(gam), diss);
    return 1;
  }

  int volume(const DevMesh& m, const DevTabs& t, const void* uL, const void* wL, const void* gam,
             Combine c, void* out, cudaStream_t st) override {
    const bool wsep = (wL != nullptr && wL != uL);
    if constexpr (kVolRH) {
      if (!wsep && (vvar_ == kVolRegHalf || !kVolR)) {
        using R = VolRH<D, K>;
        const int g = clamp_grid(g_volrh_, (m.E + R::ELW - 1) / R::ELW, 1);
        launch(k_volume_rh<D, K>, g, 32 * R::WARPS, R::SMEM, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(gam), static_cast<float*>(out), c);
        return 1;
      }
    }
    if constexpr (kVolRT) {
      if (!wsep && vvar_ == kVolRegTab) {
        using R = VolR<D, K, true>;
        const int g = clamp_grid(g_volrt_, (m.E + R::ELW - 1) / R::ELW, 1);
        launch(k_volume_r<D, K, false, true>, g, 32 * R::WARPS, R::SMEM, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(gam), static_cast<float*>(out), c, static_cast<float*>(nullptr));
        return 1;
      }
    }
    if constexpr (kVolR) {
      if (!wsep) {
        using R = VolR<D, K>;
        const int g = clamp_grid(g_volr_, (m.E + R::ELW - 1) / R::ELW, 1);
        launch(k_volume_r<D, K, false, false>, g, 32 * R::WARPS, R::SMEM, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(gam), static_cast<float*>(out), c, static_cast<float*>(nullptr));
        return 1;
      }
    }
    const int g = clamp_grid(g_vol_[wsep ? 1 : 0], m.E, kWarps);
    if (wsep)
      launch(k_volume<D, K, T, true, kVolumeTab, false>, g, 32 * kWarps, volume_smem(true), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(wL), static_cast<const T*>(gam),
          static_cast<T*>(out), c, nullptr);
    else
      launch(k_volume<D, K, T, false, kVolumeTab, false>, g, 32 * kWarps, volume_smem(false), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(uL), static_cast<const T*>(gam),
          static_cast<T*>(out), c, nullptr);
    return 1;
  }

  bool has_fused() const override {
    return vvar_ == kVolRegFused || vvar_ == kVolWarpFused || vvar_ == kVolTensor;
  }

  int eta(const DevMesh& m, const DevTabs& t, const void* uL, int l, int8_t* facet_l, const EtaThresholds& th,
          double* eta_out, cudaStream_t st) override {
    const int g = clamp_grid(g_eta_, m.NF, kWarps);
    launch(k_eta<D, K, T>, g, 32 * kWarps, eta_smem(), st, m, t, static_cast<const T*>(uL), l, facet_l, th, eta_out);
    return 1;
  }

  int v2l_pt(const DevMesh& m, const DevTabs& t, const void* vV, void* yL, cudaStream_t st) override {
    const int g = clamp_grid(g_v2lpt_, (m.E + PW::EW - 1) / PW::EW, 1);
    launch(k_v2l<D, K, T, true>, g, 32 * PW::WARPS, PW::SMEM, st, m, static_cast<const T*>(t.Dn),
           static_cast<const float4*>(nullptr), 0, 0, static_cast<const T*>(vV), static_cast<T*>(yL));
    return 1;
  }

  int facet_adj(const DevMesh& m, const DevTabs& t, const void* uL, const void* wL, const void* ybar, int l,
                const int8_t* facet_l, void* gamU, void* gamW, cudaStream_t st) override {
    const bool wsep = (wL != nullptr && wL != uL);
    if constexpr (kFacAR) {
      if (!wsep) {
        using R = FacAR<D, K>;
        const int g = clamp_grid(g_facar_, (m.NF + R::FPW - 1) / R::FPW, 1);
        launch(k_facet_adj_r<D, K>, g, 32 * R::WARPS, R::SMEM, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(ybar), l, facet_l, static_cast<float*>(gamU), static_cast<float*>(gamW));
        return 1;
      }
    }
    const int g = clamp_grid(g_fadj_, m.NF, kWarps);
    if (wsep)
      launch(k_facet_adj<D, K, T, true>, g, 32 * kWarps, facet_adj_smem(true), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(wL), static_cast<const T*>(ybar), l, facet_l,
          static_cast<T*>(gamU), static_cast<T*>(gamW));
    else
      launch(k_facet_adj<D, K, T, false>, g, 32 * kWarps, facet_adj_smem(false), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(uL), static_cast<const T*>(ybar), l, facet_l,
          static_cast<T*>(gamU), static_cast<T*>(gamW));
    return 1;
  }

  int volume_adj(const DevMesh& m, const DevTabs& t, const void* uL, const void* wL, const void* ybar,
                 const void* gamU, const void* gamW, void* ubar, void* wbar, cudaStream_t st) override {
    const bool wsep = (wL != nullptr && wL != uL);
    if constexpr (kVolAR) {
      if (!wsep) {
        using R = VolAR<D, K>;
        const int g = clamp_grid(g_volar_, (m.E + R::ELW - 1) / R::ELW, 1);
        launch(k_volume_adj_r<D, K>, g, 32 * R::WARPS, R::SMEM, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(ybar), static_cast<const float*>(gamU), static_cast<const float*>(gamW),
               static_cast<float*>(ubar));
        return 1;
      }
    }
    const int g = clamp_grid(g_vadj_, m.E, kWarps);
    if (wsep)
      launch(k_volume_adj<D, K, T, true>, g, 32 * kWarps, volume_adj_smem(true), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(wL), static_cast<const T*>(ybar),
          static_cast<const T*>(gamU), static_cast<const T*>(gamW), static_cast<T*>(ubar), static_cast<T*>(wbar));
    else
      launch(k_volume_adj<D, K, T, false>, g, 32 * kWarps, volume_adj_smem(false), st, 
          m, t, static_cast<const T*>(uL), static_cast<const T*>(uL), static_cast<const T*>(ybar),
          static_cast<const T*>(gamU), static_cast<const T*>(gamW), static_cast<T*>(ubar), nullptr);
    return 1;
  }

  int volume_l2v(const DevMesh& m, const DevTabs& t, const void* uL, const void* gam, void* lf, Combine c,
                 void* outV, cudaStream_t st) override {
    if constexpr (kTcVol) {
      if (vvar_ == kVolTensor && tensor_core_volume() && t.tcvol) {
        const int g = clamp_grid(g_vol_tc_, m.E, VolTc<D, K>::EB);
        const int nlr = row_stride<float>(S::nloc);
        launch(k_volume_tc<D, K>, g, VolTc<D, K>::THREADS, VolTc<D, K>::SMEM, st,
            m, static_cast<const float*>(t.tcvol), static_cast<const float*>(t.Dm), static_cast<const float*>(t.Wq),
            static_cast<const float*>(t.TrM), static_cast<const float*>(t.Drow), nlr, static_cast<const float*>(uL),
            static_cast<const float*>(gam), static_cast<float*>(outV), c, static_cast<float*>(lf));
        return 1;
      }
    }
    if constexpr (kVolRF) {
      if (vvar_ == kVolRegFused) {
        using R = VolR<D, K>;
        const int g = clamp_grid(g_volrf_, (m.E + R::ELW - 1) / R::ELW, 1);
        launch(k_volume_r<D, K, true, false>, g, 32 * R::WARPS, R::SMEM_FUSE, st, m, t, static_cast<const float*>(uL),
               static_cast<const float*>(gam), static_cast<float*>(outV), c, static_cast<float*>(lf));
        return 1;
      }
    }
    if constexpr (kFuse) {
      if (vvar_ == kVolWarpFused) {
        const int g = clamp_grid(g_fuse_, m.E, kWarps);
        launch(k_volume<D, K, T, false, true, true>, g, 32 * kWarps, kFuseSmem, st,
            m, t, static_cast<const T*>(uL), static_cast<const T*>(uL), static_cast<const T*>(gam),
            static_cast<T*>(outV), c, static_cast<T*>(lf));
        return 1;
      }
    }
    return 0;
  }

  bool tensor_core_l2v() const override { return kTcL2v && tc_ != 0; }
  void select_l2v(int tc) override { use_tc_l2v_ = tc != 0 && tensor_core_l2v(); }
  int selected_l2v() const override { return use_tc_l2v_ && tensor_core_l2v() ? 1 : 0; }

  int l2v_elem(const DevMesh& m, const DevTabs& t, const void* yL, bool dual, void* lf, Combine c,
               void* outV, cudaStream_t st) override {
    if constexpr (kTcL2v) {
      if (!dual && use_tc_l2v_ && tc_ && t.tcl2v) {
        using LC = L2vTc<D, K>;
        const int g = clamp_grid(g_l2v_tc_, m.E, LC::TM);
        if (tc_ == 3)
          launch(k_l2v_tc<D, K, true>, g, LC::THREADS, LC::SMEM, st, m, static_cast<const float*>(t.tcl2v),
                 static_cast<const float*>(yL), static_cast<float*>(lf), static_cast<float*>(outV), c);
        else
          launch(k_l2v_tc<D, K, false>, g, LC::THREADS, LC::SMEM, st, m, static_cast<const float*>(t.tcl2v),
                 static_cast<const float*>(yL), static_cast<float*>(lf), static_cast<float*>(outV), c);
        return 1;
      }
    }
    const int g = clamp_grid(g_elem_[dual ? 1 : 0], (m.E + PW::EW - 1) / PW::EW, 1);
    if (dual)
      launch(k_l2v_elem<D, K, T, true>, g, 32 * PW::WARPS, PW::SMEM, st, 
          m, static_cast<const T*>(t.Dinv), static_cast<const T*>(yL), static_cast<T*>(lf), static_cast<T*>(outV), c);
    else
      launch(k_l2v_elem<D, K, T, false>, g, 32 * PW::WARPS, PW::SMEM, st, 
          m, static_cast<const T*>(t.DT), static_cast<const T*>(yL), static_cast<T*>(lf), static_cast<T*>(outV), c);
    return 1;
  }

  int l2v_facet(const DevMesh& m, const void* lf, bool dual, Combine c, void* outV, cudaStream_t st) override {
    const int gf = clamp_grid(g_fsum_, m.NF * S::nf, 256);
    if (dual)
      launch(k_l2v_facet<D, K, T, true>, gf, 256, 0, st, m, static_cast<const T*>(lf), static_cast<T*>(outV), c);
    else
      launch(k_l2v_facet<D, K, T, false>, gf, 256, 0, st, m, static_cast<const T*>(lf), static_cast<T*>(outV), c);
    return 1;
  }
};

}  // namespace hopu

#define HOPU_DEFINE_OPS(D, K)                                               \
  namespace hopu {                                                          \
  Ops* make_ops_##D##_##K(bool fp64, int tc) {                              \
    if (fp64) return new OpsImpl<D, K, double>();                           \
    return new OpsImpl<D, K, float>(tc);                                    \
  }                                                                         \
  }
