/*
 * sgn_amr.h -- C ABI of the refined hierarchy: block-structured adaptive
 * refinement (Berger-Oliger-Colella) of the explicit step, as the paper runs
 * the method in GeoClaw (Sec. 4: patches with refinement ratio r and
 * subcycling in time; refinement along the advancing front, Sec. 6.3).
 *
 * Every patch of a level is laid out in one padded "atlas" grid of that level
 * (runs of patches with the same rows that abut in x share one frame of ghost
 * cells: three layers in mixed precision, two in FP64), so that every stage of
 * the step runs as ONE launch over all patches of the level, whatever their
 * number and sizes: in mixed precision a level step is one launch of the
 * one-pass kernel of the uniform grid (on every level large enough to fill
 * the GPU), after one ghost-fill launch; a level-0 step with all finer
 * substeps is replayed as one CUDA graph.
 *
 * Definitions the paper leaves to GeoClaw (they are the library's readings):
 *  - level 0 is one patch covering the grid; level l >= 1 holds disjoint boxes
 *    (i0, j0, nx, ny) in level-l cell indices (spacing dx / r^l), aligned to
 *    whole parent cells, each inside one level-(l-1) patch and at least two
 *    parent cells from its edges except along the domain boundary;
 *  - bathymetry of a coarser level is the mean of the r x r children of the
 *    next finer level (the finest level's bathymetry is given);
 *  - ghost cells: boundary condition (outside the domain), copy from another
 *    patch of the level, or limited interpolation of surface and primitives
 *    from the parent at the substep's time weight (a dry parent cell gives a
 *    ghost at the still level; a conserved ghost value never exceeds the
 *    parent cell's own in magnitude);
 *  - positivity factors of ghost cells copied from a patch are the patch's
 *    own (copied, or computed in the three-layer frame, to the same value);
 *  - mass is refluxed at coarse faces between covered and uncovered cells (a
 *    correction that would leave a negative depth is clipped to zero depth and
 *    the water added is reported); covered coarse cells hold the mean of their
 *    children; dt_0 = min over levels of CFL r^l / (max cell speed of level l).
 *
 * Errors as in sgn.h (negative SGN_E* codes).  Periodic boundaries and dx != dy
 * are rejected (SGN_EINVAL).
 */
#ifndef SGN_AMR_H
#define SGN_AMR_H
#include "sgn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgn_amr sgn_amr;

/* grid0: level-0 grid (nx, ny, dx = dy, boundary conditions wall or
 * extrapolation).  b_finest: bathymetry of the finest level, (ny r^(L-1)) x
 * (nx r^(L-1)) doubles, row-major (copied).  nlevels L in 1..8, ratio r in
 * 2..8.  nboxes[l-1] boxes on level l = 1..L-1; boxes: 4 ints (i0, j0, nx, ny)
 * per box, level by level.  model, params, allocator and stream as for
 * sgn_create.  Errors: EINVAL (arguments, box rules), ENOMEM, ECUDA. */
int sgn_amr_create(const sgn_grid* grid0, const double* b_finest, int nlevels, int ratio, const int* nboxes,
                   const int* boxes, int model, const sgn_params* params, const sgn_allocator* allocator,
                   void* cuda_stream, sgn_amr** out);
void sgn_amr_destroy(sgn_amr* a);

/* Number of patches of a level (level 0: 1), or EINVAL. */
int sgn_amr_npatches(const sgn_amr* a, int level);

/* State of one patch's interior: nvar x ny x nx doubles (field order of
 * sgn.h), host memory.  set applies the SWE / dry switch; the first step after
 * a set recomputes the time step from the new states and resets the time, the
 * status and the clipped water.  Errors: EINVAL. */
int sgn_amr_set_patch(sgn_amr* a, int level, int patch, const double* q);
int sgn_amr_get_patch(sgn_amr* a, int level, int patch, double* q);
/* Fields 0 .. nfields-1 (field order as in sgn.h) of every patch of `level`,
 * interior cells only, into out_dev: caller-owned device memory, FP64
 * [nfields][NY][NX] over the level's full grid (NX = level-0 nx * ratio^level,
 * likewise NY), row-major, x fastest.  Cells no patch of the level covers are
 * left unchanged.  For level 0 this is the whole coarse state.  One launch over
 * all patches (at most 65535; more: SGN_ERANGE); synchronises the hierarchy's
 * stream.  SGN_EINVAL for a bad level, nfields outside 1 .. nvar or a NULL
 * pointer. */
int sgn_amr_get_level_device(sgn_amr* a, int level, int nfields, double* out_dev);

/* n level-0 steps with the CFL step of all levels (subcycling below), or one
 * level-0 step of the given dt0.  Return the status of the batch as an error
 * code; *t_out (may be NULL) receives the level-0 time. */
int sgn_amr_step(sgn_amr* a, int n, double* t_out);
int sgn_amr_step_dt(sgn_amr* a, double dt0);
/* The level-0 step the next sgn_amr_step will take. */
int sgn_amr_next_dt(sgn_amr* a, double* dt0);

/* Mass sum(h) dx^2 over the uncovered interior cells of every level (FP64,
 * fixed order), and the water added by clipped reflux corrections since the
 * last set (either pointer may be NULL).  Synchronises the stream. */
int sgn_amr_mass(sgn_amr* a, double* mass, double* clipped);
/* OR of the status words of all levels (bits of sgn.h). */
int sgn_amr_status(sgn_amr* a, unsigned* flags);
/* Per level (L entries each, either pointer may be NULL): interior cells of all
 * patches and cells of the level's atlas grid (padding and frames included). */
int sgn_amr_info(const sgn_amr* a, long long* cells, long long* atlas_cells);
/* Kernel launches in one level-0 step (all levels); 0 before the first step. */
int sgn_amr_launches_per_step(const sgn_amr* a);

/* Regridding: replace the patches of levels 1..L-1 by a new box list (same
 * rules and layout as sgn_amr_create) and carry the state over, so that the
 * refined region can follow the flow (the paper's patches track the advancing
 * front, Sec. 6.3; GeoClaw regrids every few steps).  b_finest must be the
 * bathymetry given to sgn_amr_create (it is not kept by the library).  The
 * new state: level 0 unchanged; coarse to fine, each interior cell of a new
 * patch takes the old patch's value of the same cell where an old patch of
 * its level covered it, else the limited interpolation of the ghost cells
 * (surface and primitives, A4 of the header's definitions) from its new parent
 * at the current time; then every covered coarse cell becomes the mean of its
 * children (average-down, finest level first).  The time and the clipped water
 * carry over; the next step is recomputed from the new states; the status
 * starts clear; the launch shapes of levels >= 1 return to their defaults
 * (tune again with sgn_amr_autotune; level 0 keeps its solver, tuning and
 * state, which the new hierarchy takes over).  The new hierarchy is built
 * before the old one is released (both are held on the device for the
 * duration of the call).  On an error other than ECUDA the old hierarchy is
 * left as it was (level 0 handed back).  Synchronises the stream.
 * Errors: EINVAL (arguments, box rules), ENOMEM, ECUDA. */
int sgn_amr_regrid(sgn_amr* a, const double* b_finest, const int* nboxes, const int* boxes);

/* Flag-driven regridding, so that the patches follow the flow between calls
 * (Sec. 6.3: cells are flagged where the surface jump to a neighbouring cell
 * exceeds a threshold).  Level by level from the coarsest: a wet cell of
 * level l (h > dry_tol) is flagged where |eta - eta_n| > tol for a wet
 * neighbour n in the same patch (a dry cell's eta is its bathymetry, not a
 * surface; where level l has no patch, the cell takes its parent cell's flag); the
 * flags are widened by `buffer` cells of that level; the part of each new
 * level-l box that may hold finer patches (two cells inside its edges, except
 * along the domain boundary) is cut into tile x tile squares of level-l cells
 * (tile >= 2; the last ones clipped, a one-cell remainder joined to the square
 * before it), and every square holding a widened flag becomes a level-(l+1)
 * box.  Then as sgn_amr_regrid with those boxes.  nboxes (L - 1
 * ints, may be NULL) receives the number of boxes per level >= 1.  Errors as
 * sgn_amr_regrid; EINVAL also for L = 1, tol <= 0, tile < 2 or buffer < 0. */
int sgn_amr_regrid_flagged(sgn_amr* a, const double* b_finest, double tol, int tile, int buffer, int* nboxes);

/* Boxes of a level (4 ints i0, j0, nx, ny each, in that level's cells) into
 * boxes (capacity cap boxes; NULL to query); returns the number of boxes, or
 * EINVAL / ERANGE. */
int sgn_amr_get_boxes(const sgn_amr* a, int level, int* boxes, int cap);

/* Autotuner of every level (sgn_autotune of sgn.h on each level's atlas grid,
 * which differ in size and shape): choice (L * SGN_TUNE_N ints, may be NULL)
 * receives level l's tuning at choice[l * SGN_TUNE_N]; ms (may be NULL) L *
 * SGN_TUNE_N * SGN_TUNE_OPTS times laid out per level as in sgn_autotune.  The
 * hierarchy's state, time and next step are unchanged; its graphs are
 * re-captured by the next step.  sgn_amr_set_tuning installs one tuning per
 * level.  Errors: EINVAL, ECUDA. */
int sgn_amr_autotune(sgn_amr* a, int reps, int* choice, double* ms);
int sgn_amr_set_tuning(sgn_amr* a, const int* choice);

/* Retaking of level-0 steps that break the CFL limit.  The level-0 step is
 * fixed for all substeps of a level-0 step (Sec. 4: CFL step from the global
 * maximum wave speeds, subcycling in time across levels), but the speeds can
 * grow within it, most of all on fine levels; the paper's step-size
 * controller (Sec. 7) then takes a smaller step.  With max_retakes > 0 every
 * level-0 step of sgn_amr_step and sgn_amr_step_dt whose largest face Courant
 * number on any level exceeded 1 is undone (the states of all levels, the
 * time, the clipped water and the status words as before it) and taken again
 * with dt0 * CFL / (that Courant number), up to max_retakes times; a step still
 * over the limit stays taken and the call returns SGN_ECFL as without
 * retaking.  sgn_amr_step_dt may so advance by less than dt0 (the time
 * returned by sgn_amr_step tells by how much).  Each level-0 step then
 * synchronises the stream once, and the states of levels >= 1 are copied
 * once per step into buffers held by the hierarchy (allocated at the first
 * call with max_retakes > 0).  max_retakes in 0 (off, the default) .. 16; the
 * setting carries over regrids.  Errors: EINVAL, ENOMEM.
 * sgn_amr_retakes: the number of level-0 steps retaken since creation. */
int sgn_amr_set_retake(sgn_amr* a, int max_retakes);
int sgn_amr_retakes(const sgn_amr* a, long long* count);

#ifdef __cplusplus
}
#endif
#endif
