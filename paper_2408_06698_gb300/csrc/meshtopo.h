// Host-side mesh topology and FP64 affine geometry of libhopu.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hopu {

struct MeshTopo {
  int dim = 0;
  int64_t n_elems = 0, n_facets = 0;
  // per element, vertices reordered by ascending representative id
  std::vector<double> X;        // [E][dim+1][dim] physical vertex coordinates
  std::vector<double> geo;      // [E][GEO]: J (row-major), Jinv, det J, |det J|
  // per (element, local facet): packed F*4 + (sigma<0)*2 + (element is side B)
  std::vector<int32_t> efc;     // [E][dim+1]
  // per facet
  std::vector<int32_t> fa, fb;  // packed element*4 + local facet of side A / side B
  std::vector<double> fgeo;     // [F][dim+1]: n_F (unit, canonical), a_F = |F| / |param|
  // boundary facets (one neighbour, side B = side A, n_F outward), ascending
  std::vector<int64_t> boundary;
};

inline int geo_stride(int dim) { return 2 * dim * dim + 2; }

// Build topology and geometry.  Returns 0 on success, otherwise a hopu_status code with
// a message in err (EMESH for invalid meshes).  Facets with one neighbour are boundary
// facets: that element is side A (n_F flipped outward if needed) and also side B.
int build_mesh_topo(int dim, int64_t nv, const double* coords, int64_t ne, const int64_t* ev,
                    const int64_t* rep, MeshTopo& out, std::string& err);

// Physical facet points [F][nqf][dim] (side A parametrisation) for parameters sq.
void facet_points(const MeshTopo& m, const std::vector<double>& sq, int nqf, double* out);
// Physical volume points [E][nq][dim] for reference points xq.
void volume_points(const MeshTopo& m, const std::vector<double>& xq, int nq, double* out);

}  // namespace hopu
