/*
 * vsie_bem.h -- C ABI of the nested PMCHWT boundary element solver in libvsie: the
 * comparison method of the paper for piecewise-constant media (Sec. 2.4 "Boundary Element
 * Method"; benchmark 2 of Table "benchmarks"), a P1 Galerkin discretisation on triangulated
 * interfaces solved by GMRES with mass-matrix preconditioning (Sec. 3.1).
 *
 * Geometry and unknowns.  n_interfaces (1 or 2) closed, nested triangulated surfaces,
 * outermost first, triangles oriented with the right-hand normal pointing outward.
 * Layer l (l = 1, 2) lies inside interface l-1 and outside interface l, with density
 * rho[l-1] and sound speed c[l-1]; the exterior has (rho0, c0) and wavenumber k0, layer
 * l the wavenumber k0 c0 / c[l-1].  On every interface the unknowns are the nodal values
 * (P1, one per vertex) of u = p and v = (1/rho) dp/dn, both continuous across it
 * (Eqs. transmission_pressure, transmission_velocity).  Unknown order:
 * [u_1 | v_1 | u_2 | v_2], each block in the interface's vertex order; complex128.
 *
 * System (PMCHWT).  With the single-layer V, double-layer K, adjoint double-layer K' and
 * hypersingular W boundary operators of wavenumber k_j between interfaces (G of Eq.
 * greens_function) and sigma_jm = +1 where the interface normal points out of layer j,
 * -1 where it points into it:
 *     sum_j sigma_jm sigma_jl [[-K_j, rho_j V_j], [W_j/rho_j, K'_j]]_{m <- l} (u_l, v_l)
 *        = (p_inc, (1/rho0) dp_inc/dn) on interface 1, 0 on interface 2,
 * the sum of the Calderon identities of the layers adjacent to both interfaces (their
 * identity parts cancel).  Galerkin with P1 test functions; W through surface curls
 * (<phi_a, W phi_b> = int int G [curl phi_a . curl phi_b - k^2 n_x.n_y phi_a phi_b]).
 * Every row is divided by its vertex's lumped mass (row sum of the P1 mass matrix):
 * vsie_bem_apply and vsie_bem_rhs return the preconditioned operator and right-hand side.
 *
 * Quadrature.  All triangle pairs: a collapsed Gauss rule with far_order^2 points on each
 * triangle (point pairs at zero distance contribute nothing).  Pairs sharing a vertex, or
 * with centroid distance^2 < near_factor^2 max(diameter^2) (any two interfaces bounding a
 * common layer), are replaced by a near_order^2 rule on the test triangle with the static
 * part 1/(4 pi r) of the kernel integrated in closed form over the trial triangle (linear
 * densities: edge integrals and the solid angle) and the smooth remainder on a
 * near_order^2 rule; a near pair's V block is the mean of its two test/trial orders.  The
 * far-rule sums run on the device as N-body sums over quadrature points; the near pairs'
 * corrections (near rule minus far rule, all layers combined) are built once at creation.
 *
 * Conventions as in vsie.h: d_* device pointers, h_* host pointers, caller-owned;
 * ``stream`` a cudaStream_t as void*; every call returns a vsie_status and sets
 * vsie_last_error() on failure.
 */
#ifndef VSIE_BEM_H
#define VSIE_BEM_H

#include <stdint.h>

#include "vsie.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vsie_bem vsie_bem;

typedef struct {
  int32_t n_interfaces;      /* 1 or 2 */
  const double* h_vert[2];   /* (n_vert[m], 3) row-major vertex coordinates of interface m */
  const int32_t* h_tri[2];   /* (n_tri[m], 3) vertex indices, right-hand normal outward */
  int64_t n_vert[2];
  int64_t n_tri[2];
  double k0, rho0, c0;       /* exterior wavenumber, density, sound speed */
  double rho[2], c[2];       /* layers inside interface 1 (and 2) */
  int32_t far_order;         /* Gauss points per direction of the far rule, 1..8 (0: 3) */
  int32_t near_order;        /* the same for the near rule, 1..8 (0: 4) */
  double near_factor;        /* near-pair radius in triangle diameters, >= 0 (0: 2.0) */
} vsie_bem_desc;

/* Builds the boundary element operator on the current device: quadrature points, near-pair
 * lists (a device search over all triangle pairs) and their correction blocks.  Blocking.
 * Errors: VSIE_ERR_ARG (null pointer, n_interfaces not 1 or 2, fewer than 4 vertices or
 * triangles, a non-positive k0, density or sound speed, an order outside 1..8, a negative
 * near_factor), VSIE_ERR_MESH (a vertex index out of range, a zero-area triangle),
 * VSIE_ERR_OOM, VSIE_ERR_CUDA.  *out is NULL on error. */
vsie_status vsie_bem_create(const vsie_bem_desc* desc, vsie_bem** out);
void vsie_bem_destroy(vsie_bem* b);

/* Unknowns (2 x total vertices), far-rule quadrature points, near triangle pairs. */
vsie_status vsie_bem_sizes(const vsie_bem* b, int64_t* n_unknowns, int64_t* n_points, int64_t* n_near_pairs);

/* d_y = P A d_x (P: the lumped-mass row scaling); d_x, d_y complex128 of n_unknowns,
 * distinct.  precision 32: the far-rule N-body sums in FP32 (per-tile partial sums folded
 * into FP64); 48: in double-float arithmetic on the FP32 pipe (FP64-class accuracy); 64: in
 * FP64; the near corrections and the P1 gathers in FP64 in every case.  Asynchronous.
 * Errors: VSIE_ERR_ARG (null, aliasing, precision), VSIE_ERR_CUDA. */
vsie_status vsie_bem_apply(vsie_bem* b, const void* d_x, void* d_y, int32_t precision, void* stream);

/* d_b = P (int phi_a p_inc, int phi_a (1/rho0) dp_inc/dn) on interface 1 (zero on interface
 * 2) for p_inc = exp(i k0 x.d) (Eq. planewave), far rule; h_direction: 3 doubles (need not
 * be normalised).  Asynchronous.  Errors: VSIE_ERR_ARG (null, zero direction). */
vsie_status vsie_bem_rhs(vsie_bem* b, const double* h_direction, void* d_b, void* stream);

/* GMRES on P A x = P b with the options and report of vsie_solve: mode 64 FP64 GMRES,
 * mode 32 FP64 iterative refinement around FP32-apply inner cycles (residuals with the
 * double-float apply, precision 48); adjoint and initial_guess must be 0.  Blocking;
 * allocates the Krylov basis.  Errors: as vsie_solve. */
vsie_status vsie_bem_solve(vsie_bem* b, const void* d_b, void* d_x, const vsie_solve_opts* opts,
                           vsie_solve_info* info, void* stream);

/* Far-field pattern (p_s ~ e^{i k0 R}/R p_inf(xhat)) from the exterior representation on
 * interface 1: p_inf(xhat) = (1/4 pi) int e^{-i k0 xhat.y} [-i k0 (xhat.n_y) u(y) - rho0 v(y)]
 * dy, far rule.  d_x: solution (complex128, n_unknowns); h_dirs: 3 x ndir unit vectors;
 * d_out: complex128 ndir.  FP64; blocking (the directions go through a stream-ordered
 * device buffer that is freed before returning).  Errors: VSIE_ERR_ARG, VSIE_ERR_CUDA. */
vsie_status vsie_bem_far_field(vsie_bem* b, const void* d_x, const double* h_dirs, int32_t ndir, void* d_out,
                               void* stream);

#ifdef __cplusplus
}
#endif

#endif /* VSIE_BEM_H */
