/*
 * hopu.h -- C ABI of libhopu, the GB300 (sm_103a) implementation of the explicit
 * convection part of the HOPU / MCS splitting scheme of
 *   Lederer, Mooslechner, Schoeberl, "High-order projection-based upwind method for
 *   simulation of transitional turbulent flows" (arXiv 2408.06698).
 *
 * The library applies, without assembling a matrix, the projection-based high-order
 * upwind (HOPU) convection operator of Section 3.2 (eq. "hopudefinition"; with l = -1
 * it is the upwind form of Section 2.2, eq. "upwind") to velocity fields on affine
 * simplicial meshes (triangles, tetrahedra), and advances such fields by explicit
 * SSP-RK3 substeps.  The implicit Stokes / pressure solves of Section 2.3 are not
 * part of this library.
 *
 * Spaces and coefficient layouts (fixed by this ABI):
 *
 *   Reference element.  Every element's vertices are reordered by ascending periodic
 *   representative id; the affine map x = x_0 + J xhat uses that order.  Local facet f
 *   is opposite local vertex f.  Facets are numbered by the lexicographic order of their
 *   sorted representative vertex tuples.  The canonical facet normal n_F is the unit
 *   right-hand normal of the sorted vertex tuple (3D: (P1-P0)x(P2-P0); 2D: (P1-P0)
 *   turned by -90 degrees); side A of a facet is the element whose outward normal is
 *   n_F, side B the other one.
 *
 *   L2 space [P^k(T)]^d (the discontinuous space the convection operator acts in):
 *   u|_T(x) = sum_{a,i} u[e][a][i] phi_i(xhat(x)) e_a, with phi_i the orthonormal
 *   Dubiner basis of the unit simplex (graded by total degree; in 3D the index runs
 *   over n = 0..k, p = 0..n, q = 0..n-p, r = n-p-q), e_a the Cartesian unit vectors.
 *   Element-major: index (e*d + a)*nb + i, nb = C(k+d, d).
 *
 *   Velocity space V_h (the normal-continuous [P^k]^d space of Section 2.2, eq.
 *   "disc_velspace", read as BDM_k so that Pi^l = I at l = k as Section 3.2 states):
 *     facet dofs   u[F*nf + m]            = int_F (u . n_F) q_m ds,
 *                  q_m(x(s)) the orthonormal Dubiner basis of the unit (d-1)-simplex in
 *                  the sorted-vertex facet parameter s, nf = C(k+d-1, d-1);
 *     interior dofs u[NF*nf + e*nint + j] = int_That uhat . z_j dxhat,
 *                  uhat the contravariant Piola pull-back (u = J uhat / det J), z_j the
 *                  interior moment functions of the BDM_k element (Nedelec first kind
 *                  of index k-1), nint = d*nb - (d+1)*nf, in this order:
 *                  (A) phi_j e_m for every Dubiner phi_j of P^{k-2}, m = 0..d-1 (m-major);
 *                  (B) with x~ = (d+1)(xhat - centroid): in 2D x~^perp phi_j,
 *                  x~^perp = (-x~_2, x~_1), phi_j over the degree-(k-2) block of the 2D
 *                  Dubiner basis; in 3D x~ x (phi_j e_m) for m = 0, 1 with phi_j over the
 *                  degree-(k-2) block of the 3D Dubiner basis, then x~ x (chi_j e_2) with
 *                  chi_j over the degree-(k-2) block of the 2D Dubiner basis of
 *                  (xhat_1, xhat_2).
 *
 *   Quadrature (Section 2.2 asks for exact integration of every form): facet rules are
 *   collapsed Gauss-Jacobi rules exact to degree 3k; volume integrals of the operator use
 *   rules exact to degree 3k-1 -- in 3D for k = 3, 4, 5 compact rules of 46, 100 and
 *   190 points (the project's own, checked on every monomial), otherwise the
 *   collapsed Gauss-Jacobi rule.  hopu_points / hopu_interpolate use the collapsed rules.
 *   Every exact rule gives the same operator up to rounding (the integrand is a
 *   polynomial of degree 3k-1 on an affine element).
 *
 * Conventions of every call:
 *   - Coefficient pointers are DEVICE pointers owned by the caller, in the working
 *     precision of the context (double for HOPU_FP64, float for HOPU_FP32), 16-byte
 *     aligned (EINVAL otherwise; the kernels copy per-element records with cp.async).
 *     The library never frees or keeps them beyond the call.
 *   - Mesh arrays and *host* pointers are host memory, copied or read during the call.
 *   - All device work is enqueued asynchronously on the context's stream (set at
 *     create time or by hopu_set_stream); calls that return host values synchronise
 *     that stream.
 *   - Every call returns a hopu_status.  The first error is sticky in the context
 *     (later calls return it unchanged until hopu_clear_error); hopu_last_error gives
 *     its text.  No call aborts or exits the process.
 */
#ifndef HOPU_H
#define HOPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hopu_ctx hopu_ctx; /* opaque; owns every device table and scratch buffer */

typedef enum {
  HOPU_OK = 0,
  HOPU_EINVAL = -1,   /* bad argument (NULL pointer, size, enum value)               */
  HOPU_ENOMEM = -2,   /* host or device allocation failed                            */
  HOPU_ECUDA = -3,    /* a CUDA runtime call failed (text in hopu_last_error)        */
  HOPU_EMESH = -4,    /* mesh is not a valid conforming simplicial mesh              */
  HOPU_ETIMEOUT = -5, /* a bounded device-side wait ran out                          */
  HOPU_ENOTSUP = -6   /* valid request this build does not support (e.g. the VJP on
                         a mesh with boundary facets)                                 */
} hopu_status;

typedef enum {
  HOPU_FP64 = 0,     /* FP64 coefficients and arithmetic                                     */
  HOPU_FP32 = 1,     /* FP32 coefficients, FP32 FMA arithmetic; the V_h -> L2 projection and
                        the facet traces of the jump as compensated FP32 dot products (as if
                        in twice the working precision), the geometry kept in FP64            */
  HOPU_FP32_TC = 2,  /* as HOPU_FP32, with dense contractions on the tensor cores in 3xTF32
                        (hi*hi + hi*lo + lo*hi, FP32 accumulation) where the autotuner finds
                        them faster: the two dense products of the refined V_h -> L2
                        projection (its residual stays compensated FP32 on the CUDA cores,
                        so the projection keeps the accuracy of HOPU_FP32), the element part
                        of the back-projection, and the STAGE volume contractions (3D k <= 3)
                                                                                            */
  HOPU_TF32 = 3      /* FP32 coefficients; the V_h -> L2 projection GEMM, the back-projection
                        and the STAGE volume contractions on the tensor cores with one TF32
                        product (about 1e-3 relative); FP32 FMA elsewhere                    */
} hopu_prec;

typedef enum {
  HOPU_HDIV_TO_L2 = 0,      /* E      : V_h -> L2 (gather, reference change of basis, Piola) */
  HOPU_L2_TO_HDIV = 1,      /* R E^-1 : L2 -> V_h, local functionals then averaging R        */
  HOPU_L2_TO_HDIV_DUAL = 2  /* E^T    : restrict an L2 residual to the V_h test functions    */
} hopu_dir;

typedef enum {
  HOPU_WIND_STAGE = 0, /* w = u at every RK stage; the state lives in V_h          */
  HOPU_WIND_FROZEN = 1 /* w fixed for all substeps; the state lives in L2          */
} hopu_wind;

/* Mesh description (all host memory, copied by hopu_create). */
typedef struct {
  int dim;                        /* 2 (triangles) or 3 (tetrahedra)                        */
  int64_t n_vertices;
  const double* coords;           /* [n_vertices][dim], unwrapped coordinates               */
  int64_t n_elems;
  const int64_t* elem_vertices;   /* [n_elems][dim+1] vertex ids                            */
  const int64_t* vertex_rep;      /* [n_vertices] periodic representative, or NULL = itself */
} hopu_mesh_desc;

typedef struct {
  int k;          /* polynomial order, 1..5                                               */
  int l;          /* HOPU projection order: -1 = standard upwind (ILES, Section 3.1),
                     0..k = Pi^l of Section 3.2 (l = k: central flux)                      */
  int prec;       /* hopu_prec                                                            */
  int wind_mode;  /* hopu_wind, used by hopu_rk_substep                                    */
  int tile_hint;  /* kernel variants in the tensor-core modes: 0 = autotune (time the FP32
                     FMA and the tensor-core kernel of each family on this mesh at create
                     and keep the faster), 1 = FMA kernels, 2 = tensor-core kernels      */
} hopu_options;

/* Build a context: validate and copy the mesh, compute FP64 geometry (Jacobians, Piola
 * maps, normals), facet pairing, reference tables, and allocate device scratch.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  On failure *out is NULL
 * and the status says why (EMESH: non-manifold facet, a facet whose two sides agree on
 * the normal, a degenerate element; ENOTSUP: k outside 1..5 in 3D or 1..4 in 2D).
 * Facets with one element are boundary facets (walls / outlets unless declared inlets,
 * see hopu_boundary_facets).  The geometry (Jacobians, Piola maps, inverse mass) is
 * computed and stored in FP64 in every precision mode.                                 */
hopu_status hopu_create(const hopu_mesh_desc* mesh, const hopu_options* opts,
                        void* cuda_stream, hopu_ctx** out);

/* Release every device and host resource of the context.  NULL is accepted. */
hopu_status hopu_destroy(hopu_ctx* ctx);

/* Replace the stream later calls enqueue on. */
hopu_status hopu_set_stream(hopu_ctx* ctx, void* cuda_stream);

/* Kernel variants in use: out2[0] for the V_h -> L2 projection (HOPU_TF32: one TF32
 * product, k_v2l_tc; HOPU_FP32_TC: the refined projection with its two dense products on
 * the tensor cores and the compensated residual on the CUDA cores, k_v2l_tcr, 3D k <= 4
 * and 2D), out2[1] for the fused STAGE volume kernel; 0 = FP32 FMA kernel, 1 =
 * tensor-core kernel.  No paper counterpart (launch tuning).                           */
hopu_status hopu_tuning(const hopu_ctx* ctx, int* out2);

/* The kernel variant of the element part of a STAGE stage (volume term, facet lift,
 * inverse mass, element part of the back-projection) that hopu_create's autotuner kept:
 *   0 = register-resident FP32 kernel (a lane per element component, modal gradients in
 *       registers) with the back-projection fused, 1 = the same kernel followed by the
 *       separate element back-projection, 2 = warp-per-element kernel with the
 *       back-projection fused, 3 = tensor-core kernel (HOPU_FP32_TC / HOPU_TF32),
 *   4 = register-resident kernel reading the reference gradients from tables (fewer
 *       registers, more resident warps) + the separate back-projection,
 *   5 = register-resident kernel with each (element, component)'s basis split over two
 *       lanes (half the registers per lane; FP32 k <= 5) + the separate back-projection,
 *  -1 = warp-per-element kernel and the separate back-projection (no other variant for
 *       this order and precision).
 * ms6 (host, 6 doubles, may be NULL): the autotuner's time per launch of each variant on
 * this mesh in ms, -1 for variants not timed (one variant only, or not available).  No
 * paper counterpart (launch tuning).                                                  */
hopu_status hopu_tuning_volume(const hopu_ctx* ctx, int* variant, double* ms6);

/* Override the autotuner's STAGE volume variant (the numbering of hopu_tuning_volume;
 * EINVAL for a variant this order and precision does not have).  Drops the cached substep
 * graph.  No paper counterpart (launch tuning).                                       */
hopu_status hopu_set_volume_variant(hopu_ctx* ctx, int variant);

/* The element part of the back-projection R E^{-1} (Section 2.3, the local functionals
 * D (det J Jinv y) of an L2 field y, not dual) that the autotuner kept: *tc = 1 for the
 * tensor-core kernel (k_l2v_tc: 128 elements per tile as the MMA rows, D as the B
 * operand; HOPU_FP32_TC runs it in 3xTF32, HOPU_TF32 in 1xTF32; 3D k <= 4 and 2D),
 * 0 for the FMA kernel.  ms2 (host, 2 doubles, may be NULL): the autotuner's time per
 * launch of the FMA and of the tensor-core kernel on this mesh in ms, -1 where not timed
 * (FP32 / FP64 modes, tile_hint 1 or 2, or no tensor-core kernel for this order).  No
 * paper counterpart (launch tuning).                                                  */
hopu_status hopu_tuning_l2v(const hopu_ctx* ctx, int* tc, double* ms2);

/* Override the autotuner's back-projection kernel: tc = 0 FMA, 1 tensor cores (EINVAL
 * where this order and precision have none).  Drops the cached substep graph.  No paper
 * counterpart (launch tuning).                                                        */
hopu_status hopu_set_l2v_variant(hopu_ctx* ctx, int tc);

/* Synchronise the context stream and report device-side failures: ETIMEOUT when a
 * tensor-core kernel (HOPU_FP32_TC / HOPU_TF32) gave up waiting for its MMAs (its
 * output is then incomplete).  hopu_energy performs the same check.  No paper
 * counterpart: error reporting of the asynchronous calls.                             */
hopu_status hopu_sync(hopu_ctx* ctx);

/* Poll limit of the tensor-core kernels' MMA completion waits (k_v2l_tc in HOPU_TF32,
 * k_volume_tc and k_l2v_tc in HOPU_FP32_TC / HOPU_TF32): polls >= 0 sets it (0 makes the first such
 * wait give up at once), polls < 0 restores the default of 2^22 polls (~0.3 s).  A wait
 * that gives up records ETIMEOUT in the device error word (hopu_sync / hopu_energy
 * report it and name the kernel); the kernel then stops issuing work, waits with the
 * default limit for its MMAs in flight, frees its tensor memory and returns, leaving
 * that launch's outputs incomplete.  No paper counterpart: failure detection of the
 * asynchronous calls, settable so that the time-out path can be exercised.  Drops the
 * cached substep graph.  EINVAL for polls above 2^32 - 1.                             */
hopu_status hopu_set_wait_limit(hopu_ctx* ctx, int64_t polls);

/* Sizes of the coefficient vectors: V_h length, L2 length (n_elems*dim*nb), facets. */
hopu_status hopu_sizes(const hopu_ctx* ctx, int64_t* n_hdiv, int64_t* n_l2, int64_t* n_facets);

/* Map coefficient vectors between V_h and L2 (Section 2.3: R is the averaging operator
 * of the element-wise BDDC preconditioner, reused here as the back-projection).
 * in/out: device vectors of the lengths hopu_sizes gives for the two spaces.
 * in and out must not overlap.                                                         */
hopu_status hopu_project(hopu_ctx* ctx, int dir, const void* in, void* out);

/* y_l2 = M_L^{-1} c(w; u, .), the HOPU convection operator of Section 3.2 in its
 * conservative form  c = sum_T -int (u (x) w) : grad v
 *                      + sum_F int [(w.n)<u> + (I-Pi^l)(1/2|w.n|(I-Pi^l)[[u]])] . [[v]],
 * equal to the paper's form for divergence-free normal-continuous w.  du/dt = -y.
 * w_hdiv: wind as a V_h vector; u_l2: field as an L2 vector; y_l2: output L2 vector
 * (must not overlap the inputs).  facet_l: optional per-facet projection order
 * (int8 device array of n_facets entries in -1..k), NULL = opts.l for every facet.     */
hopu_status hopu_apply_convection(hopu_ctx* ctx, const void* w_hdiv, const void* u_l2,
                                  void* y_l2, const int8_t* facet_l);
/* (facet_l NULL: the orders of hopu_set_facet_l when set, else the context's l.) */

/* The same operator with the wind given as an L2 vector w_l2 (element-major, the layout of
 * u_l2) instead of a V_h vector: y_l2 = M_L^{-1} c(w; u, .) with w.n on a facet taken from
 * the average of both sides' traces (equal to w.n for normal-continuous w).  Used by the
 * element-partitioned apply, whose partitions hold the wind of their halo elements in L2
 * (Section 3.2, eq. "hopudefinition", as hopu_apply_convection).  The vectors must not
 * alias y_l2.                                                                          */
hopu_status hopu_apply_convection_l2(hopu_ctx* ctx, const void* w_l2, const void* u_l2, void* y_l2,
                                     const int8_t* facet_l);

/* Halo exchange of an element partition (no paper counterpart: the data movement of a
 * partitioned apply).  ids: device int32 array of n element ids of this context's mesh.
 *   hopu_pack_elements:   buf[j] = l2 block of element ids[j]   (buf: n * dim * nb values)
 *   hopu_unpack_elements: l2 block of element ids[j] = buf[j]
 * Working precision, asynchronous on the stream.  An id outside the mesh is skipped and
 * reported as EINVAL by the next hopu_sync / hopu_energy.                              */
hopu_status hopu_pack_elements(hopu_ctx* ctx, const int32_t* ids, int64_t n, const void* l2, void* buf);
hopu_status hopu_unpack_elements(hopu_ctx* ctx, const int32_t* ids, int64_t n, const void* buf, void* l2);

/* n_substeps explicit SSP-RK3 substeps (Shu-Osher) of du/dt = -y(u) with step dt.
 * STAGE wind: state is a V_h vector, updated in place, w = u at every stage.
 * FROZEN wind: state is an L2 vector updated in place; the wind is the V_h vector last
 * given to hopu_set_frozen_wind.  On a non-default stream the substep is captured once
 * as a CUDA graph per (state pointer, dt) and replayed n_substeps times; on the legacy
 * default stream (NULL) the kernels are launched directly.                             */
hopu_status hopu_rk_substep(hopu_ctx* ctx, void* state, double dt, int n_substeps);

/* Per-substep kinetic energy (row a8 of the hot path), kept on the device: with a log
 * set, every later substep (also when replayed from its CUDA graph) writes
 * 1/2 int |u|^2 of the state at the start of that substep, in FP64, to
 * dev_log[i % capacity] for the i-th substep since this call (the L2 image of the state
 * is the one the first RK stage computes anyway).  dev_log: caller-owned device array of
 * capacity doubles; NULL with capacity 0 switches logging off.                         */
hopu_status hopu_set_energy_log(hopu_ctx* ctx, double* dev_log, int64_t capacity);

/* Set the wind used by FROZEN substeps (copied to an internal L2 buffer). */
hopu_status hopu_set_frozen_wind(hopu_ctx* ctx, const void* w_hdiv);

/* FP64 reductions (synchronises the stream):
 *   host_out[0] = 1/2 int |u|^2                             (kinetic energy)
 *   host_out[1] = c(w; u, u)                                (0 if w_hdiv is NULL)
 *   host_out[2] = sum_F int 1/2 |w.n| |(I-Pi^l)[[u]]|^2     (facet dissipation; 0 if NULL)
 * For divergence-free normal-continuous w, host_out[1] == host_out[2] >= 0.            */
hopu_status hopu_energy(hopu_ctx* ctx, const void* w_hdiv, const void* u_l2, double* host_out);

/* Boundary facets (meshes that are not closed; Section 2.1: F^I holds interior, periodic
 * and inlet facets, walls and outlets carry no convection term).  A facet with a single
 * element is a boundary facet: its normal n_F points out of the domain and by default it
 * is a wall / outlet facet, whose exterior trace is the element's own (no jump; the
 * conservative form keeps the flux (w.n) u.v that makes it equal to the paper's form).
 * hopu_boundary_facets lists their ids in ascending order (out may be NULL to query the
 * count).                                                                             */
hopu_status hopu_boundary_facets(const hopu_ctx* ctx, int64_t* out, int64_t* count);

/* Declare n boundary facets inlets (Section 2.2: jump and average of the convected
 * velocity use the inlet data u_I) and give u_I at their facet quadrature points (the
 * points of hopu_points, facet order of `facets`): values host FP64 [n][nqf][dim].  The
 * data enter through their L2 projection onto P^k of the facet (exact for polynomial
 * data of degree <= k); the wind keeps its own normal component there (w.n of a V_h
 * field is single-valued).  Replaces the previous inlet set; n = 0 makes every
 * boundary facet a wall / outlet again.  EINVAL for a facet that is not a boundary
 * facet or is listed twice.  Synchronises the stream; drops the cached substep graph. */
hopu_status hopu_set_inlet(hopu_ctx* ctx, const int64_t* facets, int64_t n, const double* values);

/* Per-facet HOPU orders (device int8 [n_facets], values -1..k, caller-owned, read at every
 * later launch) used by hopu_rk_substep, hopu_vjp_apply, hopu_vjp_rollout, hopu_energy
 * and by hopu_apply_convection* when their facet_l is NULL.  NULL restores the
 * context's uniform l.  Not itself asynchronous: the cached substep graph is dropped. */
hopu_status hopu_set_facet_l(hopu_ctx* ctx, const int8_t* facet_l);

/* Adaptive HOPU (Section 3.2): for every facet the average absolute jump
 *   eta = int_F |(I - Pi^l)[[u]]| ds / int_F |<u>| ds
 * of the L2 field u_l2, with l the facet's current order in facet_l (device int8
 * [n_facets], in/out); then the new order: l = i for eta_i < eta <= eta_{i+1}, -1 for
 * eta <= eta_0, k for eta > eta_k (eta_{k+1} = 1 and eta > 1 both give k; a zero
 * average with a non-zero jump counts as eta = +inf), written back to facet_l.
 * thresholds: host, k+1 increasing values in (0, 1) (EINVAL otherwise).  eta_out:
 * device FP64 [n_facets] or NULL.  Sums and the decision in FP64.  The paper repeats
 * this every 10th time step (the caller's loop; see the Python binding).           */
hopu_status hopu_adapt_l(hopu_ctx* ctx, const void* u_l2, const double* thresholds, int8_t* facet_l,
                         double* eta_out);

/* Reverse-mode derivative (vector-Jacobian product) of y = hopu_apply_convection(w, u)
 * with the context's l.  The apply is linear in u and, on facets, depends on w through
 * w.n and |w.n| (Section 3.2, eq. "hopudefinition", conservative form); with
 * z = M^{-1} ybar:
 *   ubar_l2   = c(w; phi_j, z) for every L2 basis function phi_j (the transposed form);
 *   wbar_hdiv = E^T of d/dw c(w; u, z) tested with phi_j (E: V_h -> L2 of HOPU_HDIV_TO_L2),
 *               with d|s|/ds taken as 0 at s = w.n = 0.
 * Either output may be NULL (not both); outputs may not alias inputs or each other.
 * Layouts and working precision as hopu_apply_convection; asynchronous on the stream.  */
hopu_status hopu_vjp_apply(hopu_ctx* ctx, const void* w_hdiv, const void* u_l2, const void* ybar_l2,
                           void* wbar_hdiv, void* ubar_l2);
/* (hopu_vjp_apply and hopu_vjp_rollout: ENOTSUP on meshes with boundary facets.)       */

/* Gradient through n_substeps STAGE SSP-RK3 substeps (hopu_rk_substep) started at u0_hdiv
 * (not modified), by the discrete adjoint of the Shu-Osher stages:
 *   b2 = 2/3 (ubar - dt J(u2)^T ubar),  b1 = 1/4 (b2 - dt J(u1)^T b2),
 *   ubar <- 1/3 ubar + 3/4 b2 + b1 - dt J(u)^T b1,
 * where J is the Jacobian of the STAGE right-hand side u -> R E^{-1} y(Eu, Eu).
 * loss != NULL: the seed is the gradient of loss = 1/2 int |E u_N|^2 (FP64, written to
 * *loss, the call then synchronises the stream) and u0bar_hdiv receives d loss / d u0.
 * loss == NULL: u0bar_hdiv holds on entry the cotangent of u_N and on return that of u0.
 * States are checkpointed every ckpt_every substeps (>= 1) and each segment is recomputed
 * once, so device memory of (n_substeps/ckpt_every + 3 ckpt_every + 3) V_h vectors is
 * allocated by the call and kept by the context.  STAGE wind only (ENOTSUP otherwise);
 * not capturable into a CUDA graph; no energy-log entries are written.               */
hopu_status hopu_vjp_rollout(hopu_ctx* ctx, const void* u0_hdiv, double dt, int n_substeps,
                             int ckpt_every, void* u0bar_hdiv, double* loss);

/* Physical quadrature points (host output, FP64):
 *   which = 0: facet points [n_facets][nqf][dim], taken from side A;
 *   which = 1: volume points [n_elems][nq][dim].
 * count_out (may be NULL) receives the number of points.  host_out may be NULL to
 * query the count only.                                                                */
hopu_status hopu_points(hopu_ctx* ctx, int which, double* host_out, int64_t* count_out);

/* Canonical V_h interpolant (the moments above, by the library's quadrature) of a
 * field given at the points of hopu_points: fvals [n_facets][nqf][dim] and
 * vvals [n_elems][nq][dim] (host, FP64).  u_hdiv: device output in working precision. */
hopu_status hopu_interpolate(hopu_ctx* ctx, const double* fvals, const double* vvals,
                             void* u_hdiv);

/* ------------------------------------------------------------------ batches of meshes
 * Many independent meshes of uneven size and order k advanced together.  The meshes of
 * one order are merged into one context (their disjoint union: no facet is shared
 * across meshes), so each kernel family runs once per order class and a substep of the
 * whole batch is one CUDA-graph replay.  Inside a class vector every mesh owns
 * contiguous ranges: its facet dofs, its interior dofs (V_h) and its element blocks
 * (L2); hopu_batch_layout gives the offsets, so per-mesh views need no copies.        */
typedef struct hopu_batch hopu_batch;

/* meshes[i] with order k[i] (1..5 in 3D, 1..4 in 2D; one dimension for the whole
 * batch).  opts->k is ignored; opts->l >= -1 is used as min(l, k_i); opts->l < -1 means
 * l = k_i + 1 + opts->l per mesh (-2: k_i - 1).  prec and wind_mode apply to all.      */
hopu_status hopu_batch_create(const hopu_mesh_desc* meshes, const int* k, int n_meshes,
                              const hopu_options* opts, void* cuda_stream, hopu_batch** out);
hopu_status hopu_batch_destroy(hopu_batch* batch);

/* Number of order classes; per class (arrays of n_classes entries, each may be NULL)
 * its order, V_h length and L2 length.                                                */
hopu_status hopu_batch_classes(const hopu_batch* batch, int* n_classes, int* class_k,
                               int64_t* class_n_hdiv, int64_t* class_n_l2);

/* The context of class c (owned by the batch: do not destroy it); hopu_points,
 * hopu_interpolate, hopu_project, hopu_energy, ... act on the merged class mesh.       */
hopu_status hopu_batch_context(hopu_batch* batch, int c, hopu_ctx** ctx);

/* Where mesh i lives: its class, and offset/length of its facet dofs, interior dofs
 * (both inside the class V_h vector) and L2 coefficients (inside the class L2 vector).
 * out7 = {class, facet_off, facet_len, interior_off, interior_len, l2_off, l2_len}.   */
hopu_status hopu_batch_layout(const hopu_batch* batch, int mesh, int64_t* out7);

/* n_substeps SSP-RK3 substeps of every mesh: class_states[c] is the state vector of
 * class c (V_h for STAGE wind, L2 for FROZEN; FROZEN winds are set per class context
 * with hopu_set_frozen_wind).  The substeps of all classes are captured once per
 * (states, dt) as one CUDA graph and replayed (direct launches on the legacy default
 * stream).                                                                            */
hopu_status hopu_batch_rk_substep(hopu_batch* batch, void* const* class_states, double dt,
                                  int n_substeps);

/* Text of the batch's first error, else of the first failing class context ("" when
 * none).  With batch == NULL: the last failed hopu_batch_create on this thread.        */
const char* hopu_batch_last_error(const hopu_batch* batch);

/* Text of the sticky error ("" when none).  Valid until the next call on ctx.
 * With ctx == NULL: the text of the last failed hopu_create on this thread.          */
const char* hopu_last_error(const hopu_ctx* ctx);

/* Clear the sticky error. */
hopu_status hopu_clear_error(hopu_ctx* ctx);

/* Kernel families timed by the profiling hook. */
typedef enum {
  HOPU_K_V2L = 0,        /* V_h -> L2 projection                                       */
  HOPU_K_FACET = 1,      /* facet flux (traces, upwind, HOPU projections)              */
  HOPU_K_VOLUME = 2,     /* volume term + facet lift + inverse mass (+ RK combination) */
  HOPU_K_L2V_ELEM = 3,   /* L2 -> V_h, element-local functionals                       */
  HOPU_K_L2V_FACET = 4,  /* L2 -> V_h, averaging R of the facet functionals            */
  HOPU_K_FACET_ADJ = 5,  /* VJP: facet moments of the two cotangents                   */
  HOPU_K_VOLUME_ADJ = 6, /* VJP: volume part + lift of the facet moments               */
  HOPU_K_COUNT = 7
} hopu_kernel_family;

/* Measured fused multiply-add throughput of the current CUDA device (no context needed):
 * fp64 = 0 for FP32, 1 for FP64; iters = timed loop trips (each thread 128 FMA per trip;
 * about 2000 for FP32 and 50 for FP64 give a launch of a few milliseconds on GB300).  One
 * warm-up launch, then one launch timed with CUDA events on a private stream; writes the
 * rate in TFLOP/s (2 flop per FMA) to *tflops.  Synchronises that stream.
 * Errors: EINVAL (NULL tflops, iters <= 0), ECUDA (launch or event failure).            */
hopu_status hopu_measure_alu_peak(int fp64, int iters, double* tflops);

/* Profiling: with enable != 0 every later kernel launch of the context is bracketed by
 * CUDA timing events on the context stream (also inside captured substep graphs; the
 * cached graph is re-captured when profiling is switched).                            */
hopu_status hopu_profile(hopu_ctx* ctx, int enable);

/* Synchronise the stream and ADD the device time (ms) and launch count of every
 * profiled launch since the previous read to ms[HOPU_K_COUNT] / launches[HOPU_K_COUNT]
 * (host arrays the caller initialises).  A replayed substep graph is read once per
 * call: read after every hopu_rk_substep(..., n_substeps = 1) for exact totals.       */
hopu_status hopu_profile_read(hopu_ctx* ctx, double* ms, int64_t* launches);

/* The convection apply of hopu_apply_convection, for callers that cannot allocate
 * device memory (no counterpart in the paper: it is a deployment aid).  Code that runs
 * inside a caller-owned memory pool or budget, or in a process that reserves all device
 * memory up front, may not let a library call cudaMalloc; this entry point allocates
 * nothing and does not use the scratch hopu_create set aside.  Its two scratch arrays
 * (the wind projected to L2 and the facet moments) live in a static device buffer of
 * 32 MiB that is part of the library image, so every GPU that loads libhopu holds it
 * until the process exits.  Meshes that need more scratch than that (n_l2 plus
 * n_elems*(dim+1)*nf*dim values in the working precision) are rejected with EINVAL.
 * Every call made outside a stream capture looks up the buffer's device address on the
 * current device (so a device reset or a new primary context is picked up); a call made
 * while the stream is being captured reuses the address of the last earlier call on that
 * device, so make one call on each device before capturing (EINVAL otherwise), and do
 * not capture across a device reset.  Every call shares the buffer, which keeps the last
 * call's contents (nothing in it needs to start at zero); calls that overlap on the GPU
 * (other streams, threads or contexts on the same device) race on it.  Profiling
 * (hopu_profile) times its kernels like those of hopu_apply_convection.  Arguments,
 * result and errors as hopu_apply_convection.                                         */
hopu_status hopu_apply_convection_noalloc(hopu_ctx* ctx, const void* w_hdiv, const void* u_l2,
                                          void* y_l2, const int8_t* facet_l);

/* Host-only self check of the reference tables of (dim, k), no GPU needed:
 * report[0] = max relative error of the volume rules (the collapsed Gauss-Jacobi rule of
 *             hopu_points / hopu_interpolate and the compact rule of the volume kernels)
 *             on monomials up to degree 3k-1,
 * report[1] = same for the facet rule up to degree 3k (closed form a!b!c!/(a+b+c+d)!),
 * report[2] = max |M - I| of the basis mass matrix under both volume rules,
 * report[3] = max |D Dinv - I| of the degree-of-freedom matrix.                        */
hopu_status hopu_selftest(int dim, int k, double* report);

#ifdef __cplusplus
}
#endif

#endif /* HOPU_H */
