/* libhopu, hexahedral cells: the HOPU convection apply and explicit SSP-RK3 substeps on a
 * structured periodic box of parallelepipeds (the paper's meshes are hexahedral, Section
 * 2.1; the operator is Section 3.2, eq. "hopudefinition", in its conservative form).
 *
 * Space and layout.  Per velocity component the discontinuous space Q^k of the reference
 * cube [0,1]^3 (degree <= k in each coordinate), orthonormal tensor Legendre basis
 * phi_i(x) = L_i1(x1) L_i2(x2) L_i3(x3), L_n(x) = sqrt(2n+1) P_n(2x-1), basis index
 * i = i1 + (k+1)(i2 + (k+1) i3).  An L2 vector is [E][3][(k+1)^3] in the context's precision
 * (double for HOPU_FP64, float for HOPU_FP32), cells numbered e = c0 + n0 (c1 + n1 c2)
 * (axis 0 fastest), Cartesian velocity components.  Geometry stays FP64 on the device.
 *
 * Box.  Grid lines lines[a][0..n_a] (increasing, n_a >= 3) and a 3x3 matrix A (row-major,
 * det A > 0): cell (c0, c1, c2) is A applied to [lines0[c0], lines0[c0+1]] x ... ; in a
 * periodic direction a the box is periodic with period A (L_a e_a), L_a = lines_a[n_a] -
 * lines_a[0]; the two ends of another direction are walls or outlets (Section 2.1: facets
 * of F^W and F^N, which carry no term in the paper's form; the cell's own trace is the
 * exterior one), or inlets with data (hopu_hex_set_inlet).
 *
 * Facets.  The facet between a cell and the next one in direction a is one facet with
 * side A the lower cell; [[u]] = u^A - u^B, n its unit normal out of side A; w.n is
 * <w>.n.  (I - Pi^l) removes the tangential Q^l modes of a facet field (Section 3.2's
 * V_h^proj with P^l read as Q^l on quadrilaterals, so that l = k leaves only the normal
 * part of the jump); l < 0 is plain upwinding (Pi = 0).
 *
 * Quadrature: ceil((3k+1)/2) Gauss-Legendre points per direction in the volume and on the
 * facets (exact to degree 3k per direction; |w.n| is integrated by the same rule).
 *
 * Calls run on the stream given at creation (NULL: the legacy default stream) and return
 * at once; pointers to coefficient vectors are device pointers, 16-byte aligned.
 * Status values are those of hopu.h (HOPU_OK, HOPU_EINVAL, ...).
 */
#ifndef HOPU_HEX_H
#define HOPU_HEX_H

#include <stdint.h>

#include "hopu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hopu_hex hopu_hex; /* opaque; owns its device tables and scratch */

/* Creates a context for the box (n0, n1, n2, lines = the n0+1, n1+1, n2+1 grid-line positions
 * of the three directions one after the other, A, periodic = bit mask of the periodic
 * directions, 7 for a fully periodic box) at order k (2..5) and precision prec (HOPU_FP64 or
 * HOPU_FP32).  Copies what it needs (the caller keeps ownership of lines and A).  EINVAL:
 * NULL pointer, n_a < 3, periodic outside 0..7, prec not one of the two; ENOTSUP: k outside
 * 2..5; EMESH: lines not increasing or det A <= 0; ENOMEM / ECUDA: allocation or CUDA
 * failure (text in hopu_hex_last_error(NULL)). */
int hopu_hex_create(int n0, int n1, int n2, const double* lines, const double* A, int periodic, int k,
                    int prec, void* stream, hopu_hex** out);
int hopu_hex_destroy(hopu_hex* h);

/* Number of cells and length of an L2 vector (E * 3 * (k+1)^3 elements). */
int hopu_hex_sizes(const hopu_hex* h, int64_t* n_cells, int64_t* n_l2);

/* y = M^-1 c(w; u, .) with the wind w given in L2 (Section 3.2, eq. "hopudefinition";
 * M the block-diagonal mass, |det J| I on a parallelepiped).  wL, uL, yL: device L2
 * vectors; yL must not alias wL or uL.  l: the HOPU order of every facet (l < 0: upwind). */
int hopu_hex_apply(hopu_hex* h, const void* wL, const void* uL, int l, void* yL);

/* n SSP-RK3 substeps (Shu-Osher form) of du/dt = -M^-1 c(u; u, .) in place on the device
 * L2 vector uL (the wind is the stage's own field). */
int hopu_hex_rk_substeps(hopu_hex* h, void* uL, double dt, int n, int l);

/* Makes the low (end 0) or high (end 1) end of the non-periodic direction dir an inlet
 * (Section 2.2: the exterior velocity u_I enters the jump and the average; the wind keeps
 * its own normal component): modes = device array [n_s * n_t][3][(k+1)^2] in the working
 * precision, the L2 projection of u_I onto Q^k of each end facet in the facet's orthonormal
 * basis L_ms(s) L_mt(t), mode m = ms + (k+1) mt, (s, t) the two other reference
 * coordinates in increasing axis order; facet j = c_s + n_s c_t by the cell's two other
 * indices.  Copied (stream-ordered); NULL turns the end back into a wall / outlet.
 * EINVAL: dir / end out of range or dir periodic. */
int hopu_hex_set_inlet(hopu_hex* h, int dir, int end, const void* modes);

/* Per-facet HOPU orders (device int8 [3E], values -1..k, caller-owned, read at every later
 * apply, substep and hopu_hex_energy; entry F = d E + e is the facet of direction d below
 * cell e, and on a box with boundary facets the two boundary facets of such a slot share
 * its order).  NULL restores the l of each call. */
int hopu_hex_set_facet_l(hopu_hex* h, const int8_t* facet_l);

/* Adaptive HOPU (Section 3.2, after eq. "hopudefinition"): per facet the jump indicator
 *   eta = int_F |(I - Pi^l)[[u]]| ds / int_F |<u>| ds
 * of the L2 field uL with l the facet's current order in facet_l (device int8 [3E],
 * in/out), then the new order: -1 for eta <= eta_0, i for eta_i < eta <= eta_{i+1}, k for
 * eta > eta_k (a zero average with a non-zero jump counts as eta = +inf), written back to
 * facet_l.  thresholds: host, k+1 increasing values in (0, 1) (EINVAL otherwise);
 * eta_out: device FP64 [3E] or NULL.  Sums and the decision in FP64.  ENOTSUP on a box
 * with boundary facets. */
int hopu_hex_adapt_l(hopu_hex* h, const void* uL, const double* thresholds, int8_t* facet_l, double* eta_out);

/* FP64 reductions (row a8 of the hot path; synchronises the stream):
 *   host_out[0] = 1/2 int |u|^2                             (kinetic energy)
 *   host_out[1] = c(w; u, u)                                (0 if wL is NULL)
 *   host_out[2] = sum_F int 1/2 |w.n| |(I-Pi^l)[[u]]|^2     (facet dissipation; 0 if NULL)
 * The point values are those of the working precision, summed in FP64.  Uses the
 * context's stage scratch (not to be called while substeps are in flight on another
 * stream).  For a divergence-free w with a continuous normal component,
 * host_out[1] == host_out[2] >= 0. */
int hopu_hex_energy(hopu_hex* h, const void* wL, const void* uL, int l, double* host_out);

/* Text of the last failure of h (NULL: of the last failed hopu_hex_create); never NULL. */
const char* hopu_hex_last_error(const hopu_hex* h);

#ifdef __cplusplus
}
#endif
#endif
