// Definition of the opaque hopu_ctx (internal to libhopu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/hopu.h"
#include "hopu_internal.h"
#include "meshtopo.h"
#include "reftables.h"

struct hopu_ctx {
  using MeshTopo = hopu::MeshTopo;
  using RefTables = hopu::RefTables;
  using DevMesh = hopu::DevMesh;
  using DevTabs = hopu::DevTabs;
  using Ops = hopu::Ops;
  int dim = 0, k = 0, l = -1, prec = 0, wind = 0;
  bool fp64 = true;
  size_t tsize = 8;
  cudaStream_t stream = nullptr;
  MeshTopo topo;
  RefTables ref;
  int64_t n_hdiv = 0, n_l2 = 0;
  DevMesh dm;
  DevTabs dt;
  Ops* ops = nullptr;
  int nsm = 1, red_blocks = 1;
  double l2v_ms[2] = {-1.0, -1.0};  // autotuner: ms per launch of the FMA / tensor-core back-projection
  double vol_ms[6] = {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0};  // autotuner: ms per launch of each STAGE volume variant
  // device memory
  void* d_mesh = nullptr;   // geo, efc, fa, fb, fgeo
  void* d_geoT = nullptr;   // working-precision geometry factors
  void* d_tabs = nullptr;   // every reference table
  void* d_tcvol = nullptr;  // tensor-core volume tables (FP32 tensor-core modes)
  void* d_tcv2l = nullptr;  // tensor-core refined projection table (HOPU_FP32_TC)
  void* d_csr_tc = nullptr; // its CSR of D with grouped rows
  void* d_tcl2v = nullptr;  // tensor-core back-projection table (FP32 tensor-core modes)
  void* d_csr = nullptr;    // FP32: nonzeros of the dof matrix D (refined projection)
  void* d_gam = nullptr;    // [E][d+1][nf][d] signed facet flux moments, element-major
  void* d_lf = nullptr;     // [E][d+1][nf] local facet functionals
  void* d_uL = nullptr;     // L2 stage field
  void* d_yL = nullptr;     // L2 operator output
  void* d_wL = nullptr;     // L2 wind of apply_convection / energy
  void* d_wfz = nullptr;    // L2 frozen wind
  void* d_s1 = nullptr;     // RK stage vectors (max of V_h and L2 lengths)
  void* d_s2 = nullptr;
  void* d_gamW = nullptr;   // VJP: facet moments of the wind cotangent (first VJP call)
  void* d_adj = nullptr;    // VJP rollout: checkpoints, stage states, cotangent stages
  size_t adj_bytes = 0;
  double* d_diss = nullptr; // [NF]
  double* d_red = nullptr;  // partial sums + 4 scalars
  int* d_err = nullptr;     // device error word (DevMesh::err)
  bool have_frozen = false;
  const int8_t* facet_l = nullptr;  // per-facet HOPU orders (hopu_set_facet_l), or NULL
  int32_t* d_inlet = nullptr;       // [NF] inlet row or -1 (hopu_set_inlet)
  void* d_inlet_modes = nullptr;    // [n_inlet][nf][d] modal exterior traces
  int64_t n_inlet = 0;
  // per-substep kinetic-energy log (device ring buffer owned by the caller)
  double* elog = nullptr;
  int64_t elog_cap = 0;
  int64_t elog_next = 0;     // host-side counter of logged substeps
  int64_t* d_elog_pos = nullptr;  // device-side counter (graph replays advance it)
  // cached CUDA graph of one substep
  cudaGraphExec_t gexec = nullptr;
  void* g_state = nullptr;
  double g_dt = 0.0;
  int g_wind = -1;
  // profiling: CUDA events around every kernel launch (pairs 0..kProfPairs-1 belong to
  // the captured substep graph, the rest to direct launches)
  bool prof_on = false;
  bool capturing = false;
  bool graph_replayed = false;
  std::vector<cudaEvent_t> ev;
  std::vector<std::pair<int, int>> prof_graph, prof_direct;  // (pair index, kernel family)
  int prof_next_direct = 0;
  int status = HOPU_OK;
  std::string err;
};

namespace hopu {

constexpr int kProfPairs = 64;

// Run launch() on the context stream, bracketed by a pair of timing events when
// profiling is on (hopu_profile).  Inside a graph capture the event records become graph
// nodes, so every replay re-records them.
template <class F>
void timed(hopu_ctx* c, int family, F&& launch) {
  if (!c->prof_on || c->ev.empty()) {
    launch();
    return;
  }
  int p;
  if (c->capturing) {
    p = (int)c->prof_graph.size() % kProfPairs;
    c->prof_graph.push_back({p, family});
  } else {
    p = kProfPairs + c->prof_next_direct;
    c->prof_next_direct = (c->prof_next_direct + 1) % kProfPairs;
    if ((int)c->prof_direct.size() >= kProfPairs) c->prof_direct.erase(c->prof_direct.begin());
    c->prof_direct.push_back({p, family});
  }
  // inside a capture only the External flag turns the record into a graph node
  const unsigned flags = c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  cudaEventRecordWithFlags(c->ev[2 * p], c->stream, flags);
  launch();
  cudaEventRecordWithFlags(c->ev[2 * p + 1], c->stream, flags);
}

}  // namespace hopu
