/*
 * iga_multipatch.h -- gluing of conforming B-spline patches (arXiv 2102.11536,
 * Sec. 5.1: the global space V_h, Assumption ass:conformity, the numbering G^(r),
 * def:mp_basis, def:n_l, def:N_patch) for the additive Schwarz mass preconditioner
 * of Sec. 5.4 (def:asp). Host-only: no device memory is touched and no CUDA call is
 * made, so it runs without a GPU. Status codes and iga_last_error as in iga_galpha.h.
 */
#ifndef IGA_MULTIPATCH_H
#define IGA_MULTIPATCH_H

#include "iga_galpha.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * iga_mp_layout -- interfaces, global numbering and local index boxes of patches that
 * are glued face to face.
 *   npatch   number of patches, >= 1.
 *   dim      2 or 3, the same for every patch.
 *   degree   host [npatch][dim], degrees 1..6.
 *   nknots   host [npatch][dim], knot-vector lengths; m = nknots - degree - 1 >= 2.
 *   knots    host [npatch * dim] pointers: patch r, direction a at knots[r * dim + a];
 *            open, non-decreasing knot vectors.
 *   ctrl     host [npatch] pointers to full control nets laid out as in iga_create
 *            (prod_a m_a points, direction 0 fastest, dim coordinates per point).
 *   tol      two control points coincide when every coordinate differs by at most
 *            tol * max(1, largest absolute coordinate of all nets); 0 => 1e-10.
 *   lo, hi   out, host [npatch][dim]: the box of each patch's local functions, full
 *            indices, inclusive: 1 .. m-2, widened to 0 (to m-1) where the face
 *            i_a = 0 (i_a = m-1) is an interface.
 *   nglob    out: number of global functions (degrees of freedom).
 *   n_adj    out: the largest number of patches sharing one global function (def:N_patch).
 *   gid      out, host, or NULL: for patch 0, 1, ... in turn and every index of its box
 *            (direction 0 fastest), the global id of that function, or -1 where the box
 *            holds a copy of a function that lies on the Dirichlet boundary (only next to
 *            a re-entrant corner). Ids run from 0 in order of first appearance in that
 *            walk.
 *   gid_len  length of gid, which must equal sum_r prod_a (hi - lo + 1); call once with
 *            gid = NULL to obtain lo and hi.
 * Rules. A face of one patch and a face of another form an interface when, under one
 * orientation (a permutation of the face's directions and a reversal of each), their
 * control points coincide one by one; the two faces must then have the same degrees and
 * knots along the matched directions (Assumption ass:conformity). Every other face
 * carries homogeneous Dirichlet conditions: a global function -- one set of identified
 * copies, def:mp_basis -- is dropped when any copy lies on such a face.
 * Errors: IGA_EINVAL (message by iga_last_error(NULL)) for bad sizes, knots or
 * pointers, non-finite control points, a face that coincides with two other faces, two
 * faces that cover the same region (equal bounding boxes) without matching control points,
 * an interface whose faces differ in degree or knots, or a wrong gid_len. The caller owns
 * every buffer; nothing is retained.
 */
int iga_mp_layout(int npatch, int dim, const int* degree, const int* nknots, const double* const* knots,
                  const double* const* ctrl, double tol, int* lo, int* hi, long long* nglob, int* n_adj,
                  long long* gid, long long gid_len);

/*
 * iga_mp_create -- a system of conforming patches glued as iga_mp_layout describes (same
 * arguments npatch .. tol), for the explicit generalized-alpha steps on V_h with the
 * additive Schwarz mass preconditioner of Sec. 5.4.
 *   opt   options as for iga_create (NULL => defaults), shared by every patch: op_form and
 *         precond are the patches' forms (each local preconditioner P^(r) of def:loc_forms2
 *         in that arithmetic); the learned guess is refused (IGA_EINVAL).
 *   out   receives a handle that the iga_galpha.h entry points accept: vectors have length
 *         nglob (iga_ndof) in the global numbering of iga_mp_layout, and
 *           M = sum_r R^(r)T M^(r) R^(r),  K likewise,
 *           P_ad^{-1} = sum_r R^(r)T P^(r)^{-1} R^(r)  (def:asp),
 *         where M^(r), K^(r) are patch r's integrals over its box and R^(r) gathers the
 *         box's global functions (zero at box entries that are not degrees of freedom;
 *         their results are dropped). iga_apply_M / _K / _Pinv, iga_solve_M (PCG with
 *         P_ad: plain for the FP64 local forms, flexible otherwise), iga_state_init,
 *         iga_step, iga_step_host, iga_cfl, iga_set_damping / _forcing / _time /
 *         _tol / _guess / _op_form / _precond / _band_config, iga_assemble, iga_ndof,
 *         iga_last_error and iga_destroy work on it; the steps run the host-driven loop
 *         unless iga_set_graphs(h, 1) asks for the captured step (one graph launch per
 *         step, the PCG loop on the device). iga_profile selects the kernel class in every
 *         patch and iga_profile_read returns the sums over the patches (launches, time,
 *         algorithmic work); iga_autotune tunes every patch's band product for its own
 *         size (the outputs are the last patch's choice). The iga_ws_*
 *         calls, iga_apply_Pinv_noalloc and iga_batch_create refuse it (IGA_EINVAL).
 * Each patch gets a handle over its index box (the interior functions widened to the
 * interface faces), with its own geometry factors, diag(M^(r)) and Kronecker factors.
 * Errors: those of iga_mp_layout and iga_create (the message of iga_last_error(NULL)
 * names the patch); IGA_EINVAL if no function is a degree of freedom.
 */
int iga_mp_create(int npatch, int dim, const int* degree, const int* nknots, const double* const* knots,
                  const double* const* ctrl, double tol, const iga_options* opt, iga_handle** out);

/*
 * iga_mp_set_concurrent -- on != 0: in the host-driven loop every operator of the system
 * runs its patches on streams of their own, forked from and joined back into the system's
 * stream by events; 0: one after another on the system's stream (default). A captured
 * step (iga_set_graphs) always runs them one after another on its capture stream: streams
 * joined to the step's capture cannot also join the capture of its PCG loop body. Results
 * are the same either way. IGA_EINVAL for a single-patch handle.
 */
int iga_mp_set_concurrent(iga_handle* h, int on);

/*
 * iga_mp_patch -- the handle of patch r of a multi-patch system (borrowed: it lives until
 * iga_destroy of the system and must not be destroyed; it works on the system's stream).
 * Its vectors are the patch's box (iga_ndof of it gives the box size, direction 0 fastest),
 * so iga_gauss_points, iga_evaluate and iga_integrate give per-patch points, fields and
 * integrals (a box entry that is not a degree of freedom is a function of the patch like
 * the others). IGA_EINVAL for a bad r or a single-patch handle. Host only.
 */
int iga_mp_patch(iga_handle* h, int r, iga_handle** patch);

/*
 * iga_mp_patch_io -- between the global vectors (device [nvec][N]) and patch r's box
 * (device [nvec][box size]): add = 0 gathers, out = R^(r) in (zero at box entries that are
 * no degree of freedom); add = 1 adds, out += R^(r)T in (each global function of the patch
 * receives its copy). Sum the add = 1 calls over the patches for sum_r R^(r)T b^(r), e.g.
 * a global load vector from per-patch integrals. Asynchronous on the system's stream.
 */
int iga_mp_patch_io(iga_handle* h, int r, int nvec, int add, const double* in, double* out);

/* iga_mp_info -- number of patches, N_adj and the summed box sizes of a multi-patch
 * handle (any pointer may be NULL). IGA_EINVAL for a single-patch handle. Host only. */
int iga_mp_info(const iga_handle* h, int* npatch, int* n_adj, long long* nloc);

#ifdef __cplusplus
}
#endif

#endif /* IGA_MULTIPATCH_H */
