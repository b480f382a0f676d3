/*
 * mg.h -- C ABI of the GB300 octree geometric multigrid library
 * (libmg_gb300.so).  The method is the cell-centred geometric multigrid for
 * quadtree/octree AMR grids of Teunissen & Keppens, arXiv:1901.11370.
 *
 * Problem (Sec. 1, Sec. 2.2):  div(eps grad phi) - lambda phi = f  on a 2D/3D
 * Cartesian or 2D cylindrical (r, z) domain, discretised with the 5/7-point
 * second-order stencil on a 2:1 balanced quadtree/octree of blocks of N^D
 * cells (Sec. 2.5).
 *
 * Conventions for every entry point:
 *  - Every call returns an int status: MG_OK (0) or a negative MG_ERR_*; the
 *    message of the last failure on the calling thread is mg_last_error().
 *    Nothing throws across this boundary.
 *  - "dev_" pointers are CUDA device pointers (global memory of the device
 *    the tree was finalised on); "host_" pointers are host memory.  Pointers
 *    are borrowed for the duration of the call only; the library copies what
 *    it keeps.  Outputs go to caller-allocated buffers.
 *  - Work is enqueued on the stream given to mg_tree_finalize.  Calls that
 *    return numbers to the host (norms, mg_solve) synchronise that stream;
 *    the others are asynchronous.
 *  - Leaf data (one value per leaf cell) are ordered by leaf block -- depth
 *    ascending, then the Morton code of the block coordinates (bit b of
 *    i, j, k at bits 3b, 3b+1, 3b+2) -- and inside a block by cell with x
 *    fastest.  mg_tree_leaf_blocks lists the blocks in that order.
 *  - Faces are numbered 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z; in the cylindrical
 *    form x = r and y = z.
 */
#ifndef MG_GB300_H
#define MG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_tree mg_tree;   /* opaque: mesh, level tables, device fields */
typedef struct mg_batch mg_batch; /* opaque: many independent trees solved together */

enum {
    MG_OK = 0,
    MG_ERR_ARG = -1,            /* invalid argument or call order */
    MG_ERR_BALANCE = -2,        /* mesh not 2:1 balanced across faces */
    MG_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    MG_ERR_NOT_CONVERGED = -4,  /* mg_solve hit max_cycles */
    MG_ERR_NAN = -5,            /* a residual norm is not finite */
    MG_ERR_TIMEOUT = -6,        /* a bounded wait inside a kernel expired */
    MG_ERR_INCOMPATIBLE_RHS = -7, /* singular problem whose residual mean cannot vanish */
    MG_ERR_STATE = -8,          /* call out of order (before finalize, refine after build, ...) */
    MG_ERR_UNSUPPORTED = -9     /* valid request outside what is built */
};
enum { MG_CART = 0, MG_CYL = 1 };
enum { MG_BC_DIRICHLET = 0, MG_BC_NEUMANN = 1, MG_BC_PERIODIC = 2, MG_BC_AXIS = 3 };
enum { MG_FP64 = 0, MG_FP32_DC = 1 };

/* Boundary condition per face (Sec. 2.6): Dirichlet phi = value at the face,
 * Neumann d(phi)/dx_d = value, periodic (both faces of a dimension), or the
 * symmetry axis r = 0 of the cylindrical form (zero flux). */
typedef struct {
    int type[6];
    double value[6];
} mg_bc;

/* Smoothers: red-black Gauss-Seidel (Sec. 2.2, the default) or weighted
 * Jacobi (the smoother of the paper's scaling runs, Sec. 3.3): every cell of
 * a level takes x + omega (x_GS - x), x_GS its local solution from the values
 * before the step, then the ghosts are refreshed. */
enum { MG_SMOOTH_RBGS = 0, MG_SMOOTH_JACOBI = 1 };

/* Cycle parameters (Sec. 2.4): n_down / n_up smoothing steps per level
 * (paper default 2 / 2; one red-black sweep or one Jacobi step each).
 * precision MG_FP32_DC runs the cycles in FP32 inside an FP64
 * defect-correction loop (mg_solve only); inner_cycles is the number of FP32
 * V-cycles per outer FP64 residual.  smoother MG_SMOOTH_RBGS or
 * MG_SMOOTH_JACOBI; omega the Jacobi weight (<= 0: 4/5 in 2D, 6/7 in 3D;
 * at most 1).  coarse_mode MG_COARSE_EXACT solves the coarsest level
 * exactly (a dense FP64 inverse; in a batch, the block-tridiagonal form
 * described at mg_batch_create, FP32 inside FP32 cycles); MG_COARSE_SMOOTH
 * is the paper's coarse-grid
 * solve: red-black Gauss-Seidel sweeps of the coarsest level (FP64) until
 * max |r| there is at most coarse_abs_tol or at most coarse_rel_tol times its
 * value before the first sweep, or coarse_max_it sweeps (values <= 0 take the
 * paper's defaults 1e-8, 1e-8, 1000); it needs the coarsest level of each
 * tree to fit one CTA's shared memory (MG_ERR_UNSUPPORTED otherwise).  A
 * NULL mg_params means 2 / 2, FP64, one inner cycle, red-black Gauss-Seidel,
 * exact coarsest solve. */
enum { MG_COARSE_EXACT = 0, MG_COARSE_SMOOTH = 1 };
typedef struct {
    int n_down, n_up;
    int precision;
    int inner_cycles;
    int smoother;
    double omega;
    int coarse_mode;
    int coarse_max_it;
    double coarse_abs_tol, coarse_rel_tol;
} mg_params;

/*
 * mg_tree_create -- start a mesh (Sec. 2.5, "the user indicates the block
 * size and the size of the unrefined domain").  dim 2 or 3; block_size N
 * (even, >= 2) cells per block edge; geometry MG_CART or MG_CYL (dim 2);
 * base_cells[d] the unrefined grid (multiples of N; base_cells[2] ignored in
 * 2D); lo/hi the domain corners; coarse_max_cells: below the base the block
 * count is halved while every count is even, then the block size is halved
 * while a level holds more than this many cells; the last level is solved
 * exactly (mg_params.coarse_mode).  helmholtz: lambda >= 0.  *out receives
 * the handle.
 */
int mg_tree_create(int dim, int block_size, int geometry, const mg_bc *bc,
                   const int base_cells[3], const double lo[3], const double hi[3],
                   int coarse_max_cells, double helmholtz, mg_tree **out);

/*
 * mg_tree_refine -- cover existing blocks by 2^D children (Sec. 2.5,
 * "Copying the application's grid refinement").  host_entries holds n
 * records (depth, i, j, k): depth 0 is the base grid.  Parents must exist
 * (list shallower depths first or in any order; all are applied at build).
 * 2:1 balance across faces is checked at build (MG_ERR_BALANCE).
 */
int mg_tree_refine(mg_tree *t, int n, const int32_t *host_entries);

/*
 * Mesh construction (Sec. 2.5): the block tables (levels, Morton order with
 * covered blocks first, offsets, parents, face neighbours) are built at the
 * first query or at finalize, on the current CUDA device when there is one
 * (kernels and one radix sort per level; the block table stays on the
 * device for finalize), else on the host.  Both give identical tables.
 * mg_tree_build_on -- before the build: where = 0 device when present,
 *   1 host, 2 device (MG_ERR_UNSUPPORTED without a device); MG_ERR_STATE
 *   once built.
 * mg_tree_built_on -- builds if needed; *where = 1 host, 2 device.
 * mg_tree_block_table -- builds if needed; *nblocks = blocks of all levels;
 *   host_out (NULL: count only) receives 24 int64 per block in global id
 *   order: cell offset, ghost offset, N, level, flags (bit 0: covered),
 *   parent id (-1 on level 0), block coordinates [3], offset inside the
 *   parent in parent cells [3], face neighbours [6] (>= 0 same-level id,
 *   -1 physical face, <= -2 the coarser block -2 - v), ghost push slots [6]
 *   (first ghost value of the neighbour's opposite face, -1 if none).
 *   A refine entry naming no block gives MG_ERR_ARG; a mesh that is not 2:1
 *   balanced across faces, MG_ERR_BALANCE.
 *
 * Mesh queries (build the tables if not built yet).
 * level_info: info[0..8] = N_l, depth, blocks, blocks per dim[3], cells per
 * dim[3]; h[3] cell size.  Level 0 is the coarsest. */
int mg_tree_build_on(mg_tree *t, int where);
int mg_tree_built_on(mg_tree *t, int *where);
int mg_tree_block_table(mg_tree *t, int64_t *nblocks, int64_t *host_out);
int mg_tree_num_levels(mg_tree *t, int *nlev);
int mg_tree_level_info(mg_tree *t, int level, int32_t info[9], double h[3]);
int mg_tree_num_leaf_cells(mg_tree *t, int64_t *n);
int mg_tree_leaf_blocks(mg_tree *t, int32_t *host_out /* 4 per leaf block */);

/*
 * mg_set_bc_plane -- boundary values (Dirichlet a or Neumann b) at the face
 * centres of one face of one level, replacing the constant of mg_bc there.
 * host_vals has cells_t1 * cells_t2 entries, t1 < t2 the tangential
 * dimensions, t1 fastest (2D: cells_t1 entries).  Call before finalize or
 * after it (a later mg_set_phi or cycle picks it up).
 */
int mg_set_bc_plane(mg_tree *t, int face, int level, const double *host_vals);

/* mg_tree_finalize -- build tables, allocate device fields (phi = 0, eps = 1,
 * f = 0) and bind cuda_stream (a cudaStream_t, NULL = legacy default). */
int mg_tree_finalize(mg_tree *t, void *cuda_stream);

/*
 * mg_tree_adapt -- a new mesh from a finalized tree t (Sec. 2.5, "Adapting
 * the grid structure": the application reports the blocks it added and
 * removed).  add holds n_add records (depth, i, j, k) of leaf blocks of t to
 * cover by 2^D children; remove holds n_remove records of refined blocks of
 * t whose children are all leaves, whose refinement is undone.  The base
 * grid, boundary conditions, Helmholtz term and coarse-level rule of t are
 * kept, and so are the boundary planes of every level depth both meshes
 * have.  The new tree is finalized on t's stream and phi is carried over on
 * the device: a leaf block that is also a block of t takes its values (the
 * mean of its former children where a refinement was removed), a new child
 * takes the prolongation of Sec. 2.3 of its parent's values, parent ghosts
 * included.  Right-hand side and eps start at 0 and 1: set them for the
 * new mesh.  The sweep kernel of each level is the one t uses at the same
 * depth (the default kernel at a new depth): no second autotuning.
 * t is not changed (its covered cells and ghosts are refreshed);
 * *out receives the new handle, which the caller destroys.  Errors:
 * MG_ERR_ARG (a record names no such leaf or refinement, a removed
 * refinement has refined children, t is a batch), MG_ERR_BALANCE (the new
 * mesh breaks 2:1 balance), MG_ERR_CUDA; on error *out is NULL.
 */
int mg_tree_adapt(mg_tree *t, int n_add, const int32_t *add, int n_remove, const int32_t *remove,
                  mg_tree **out);

/*
 * mg_tree_build_times -- wall seconds of this tree's construction: out4[0]
 * the mesh tables (levels, neighbours, offsets; on the device or the host,
 * mg_tree_built_on), out4[1] device setup
 * (allocation, uploads, coarsest-level inverse), out4[2] FP64 sweep
 * autotuning at finalize (0 for a tree made by mg_tree_adapt, which takes
 * over the old tree's choices), out4[3] the phi transfer of mg_tree_adapt
 * (0 for a tree not made by it).  Host pointer; entries not reached yet
 * are 0.
 */
int mg_tree_build_times(mg_tree *t, double *out4);

/* Leaf fields, device pointers, leaf order (see above). mg_set_phi also
 * restricts the covered cells and refills every ghost layer. */
int mg_set_rhs(mg_tree *t, const double *dev_f);
int mg_set_eps(mg_tree *t, const double *dev_eps); /* eps > 0; coarse eps = mean of children */
int mg_set_phi(mg_tree *t, const double *dev_phi);
int mg_get_phi(mg_tree *t, double *dev_phi);

/* mg_vcycle -- n_cycles FAS V-cycles on the whole tree (Sec. 2.4, eqs. for
 * the coarse right-hand side and the coarse-grid correction), FP64. */
int mg_vcycle(mg_tree *t, int n_cycles, const mg_params *p);

/* mg_fmg -- one FMG cycle (Sec. 2.4 and the figure of the cycles), FP64. */
int mg_fmg(mg_tree *t, const mg_params *p);

/*
 * mg_residual_norm -- composite residual r = f - L phi on the leaf cells
 * after resetting every covered cell to the mean of its children:
 * *l2 = sqrt(sum V r^2 / sum V) (the norm of Sec. 4.2), *linf = max |r|.
 * dev_r (may be NULL) receives r in leaf order.  Synchronises the stream.
 */
int mg_residual_norm(mg_tree *t, double *l2, double *linf, double *dev_r);

/*
 * mg_solve -- from the current phi, cycle until the composite residual L2
 * norm is at most rel_tol times its value at the starting phi, or
 * max_cycles.  On a singular problem (no Dirichlet face, lambda = 0) the
 * volume-weighted mean of the residual cannot change; when it exceeds
 * rel_tol times the starting residual norm the call returns
 * MG_ERR_INCOMPATIBLE_RHS before cycling (project f first).
 * MG_FP64: one FMG cycle if fmg_first, then V-cycles.  MG_FP32_DC: each
 * outer step computes r = f - A phi in FP64, runs p->inner_cycles FP32
 * V-cycles on A e = r (homogeneous boundary values, coarsest solve in FP64)
 * and adds e to phi in FP64.  *cycles_done counts outer steps, *rel_out the
 * final relative residual.  On a singular problem phi is returned with zero
 * volume-weighted mean.  Returns MG_ERR_NOT_CONVERGED at max_cycles.
 */
int mg_solve(mg_tree *t, double rel_tol, int max_cycles, int fmg_first,
             const mg_params *p, int *cycles_done, double *rel_out);

/*
 * mg_adjoint -- for a loss L(phi) at the current (converged) phi:
 * dev_dLdf = lambda = A^-T dev_dLdphi, and dev_dLdeps[c] = dL/d eps_c
 * through the harmonic face coefficients (Sec. 2.2), the eps ghosts and the
 * coarse-level means of eps.  A is the composite operator with its boundary
 * values held fixed.  At refinement faces A is not symmetric (the
 * refinement ghosts of Sec. 2.6), so A^T is applied as the exact transpose
 * of the forward steps.  lambda comes from defect correction with A's own
 * V-cycle on the volume-weighted form (W the cell volumes):
 * mu_0 = FMG(W^-1 g), lambda_0 = W mu_0, then n_cycles times
 * lambda += W M W^-1 (g - A^T lambda), homogeneous boundary values.  On a
 * problem without Dirichlet faces (lambda_helmholtz = 0) the forward map
 * includes the zero-mean projection of f and of phi: g is made compatible
 * (sum g = 0) and lambda is returned without its component along W.  Such a
 * problem with variable eps and refinement faces returns MG_ERR_UNSUPPORTED
 * (fluxes are not conserved there).  dev_dLdeps may be NULL.  phi is left
 * unchanged; n_cycles >= 0.  p->precision = MG_FP32_DC makes M an FP32
 * V-cycle on the FP32 copy of W^-1 (g - A^T lambda) (the tree's FP32 fields,
 * allocated on first use), the transpose, residual and update staying FP64
 * (the split of the forward solve's defect correction): the same fixed point,
 * reached in about as many iterations at the cost of FP32 cycles.  The
 * FMG start is FP64 in both forms.
 */
int mg_adjoint(mg_tree *t, const double *dev_dLdphi, double *dev_dLdf, double *dev_dLdeps,
               const mg_params *p, int n_cycles);

/*
 * mg_adjoint_solve -- mg_adjoint iterated until the volume-weighted norm of
 * W^-1 (g - A^T lambda) is at most rel_tol times that of W^-1 g (after the
 * compatibility projection), or max_cycles iterations.  *cycles_done and
 * *rel_out (optional) receive the count and the final ratio.  Returns
 * MG_ERR_NOT_CONVERGED when max_cycles is reached first (the outputs are
 * still written), MG_ERR_ARG for rel_tol <= 0.
 */
int mg_adjoint_solve(mg_tree *t, const double *dev_dLdphi, double *dev_dLdf, double *dev_dLdeps,
                     const mg_params *p, double rel_tol, int max_cycles, int *cycles_done, double *rel_out);

/*
 * mg_apply_transpose -- dev_out = A^T dev_y on the leaf cells (leaf order),
 * A the composite operator with homogeneous boundary values (the linear
 * part of L phi).  The adjoint of every step of the forward operator
 * (stencil, refinement-face ghosts of Sec. 2.6, the mean restriction of
 * covered cells of Sec. 2.3), applied in reverse.
 */
int mg_apply_transpose(mg_tree *t, const double *dev_y, double *dev_out);

/*
 * Divergence cleaning (Sec. 4.1, eqs. for the projection method and the
 * central-difference divergence), Cartesian meshes:
 * mg_divergence: dev_divB = sum_d (B_d(c+e_d) - B_d(c-e_d)) / (2 h_d) on the
 *   leaf cells.  dev_B holds dim leaf arrays (x, y[, z]) back to back; each
 *   component is restricted to covered cells and ghost-filled with the rules
 *   of Sec. 2.6 (physical faces copy the interior value).
 * mg_divergence_order: order 2 as mg_divergence; order 4 the fourth-order
 *   difference (-B(c+2e) + 8 B(c+e) - 8 B(c-e) + B(c-2e)) / (12 h_d) along
 *   each dimension where both cells two away are same-level cells (this
 *   block or a same-level neighbour, periodic wrap included), the
 *   second-order difference beside physical and refinement faces (the grid
 *   has one ghost layer).  MG_ERR_ARG for another order.
 * mg_project: dev_Bnew = dev_B - grad phi with second-order central
 *   differences of the current phi (dim leaf arrays back to back).
 * A cleaning step is mg_divergence, mg_set_rhs (projected to zero mean when
 * no face is Dirichlet), mg_solve and mg_project.
 */
int mg_divergence(mg_tree *t, const double *dev_B, double *dev_divB);
int mg_divergence_order(mg_tree *t, const double *dev_B, double *dev_divB, int order);
int mg_project(mg_tree *t, const double *dev_B, double *dev_Bnew);

/*
 * mg_clean -- one whole cleaning step on the device: f = div B
 * (mg_divergence_order), minus its volume-weighted mean when no face is
 * Dirichlet (the compatibility condition of the periodic/Neumann problem),
 * phi = 0, mg_solve(rel_tol, max_cycles, FMG first, p) for Lap phi = f, then
 * dev_Bnew = dev_B - grad phi.  dev_divB (optional, n_leaf values) receives
 * the right-hand side f.  Returns as mg_solve (MG_ERR_NOT_CONVERGED still
 * writes dev_Bnew).
 */
int mg_clean(mg_tree *t, const double *dev_B, double *dev_Bnew, double *dev_divB, int order, double rel_tol,
             int max_cycles, const mg_params *p, int *cycles_done, double *rel_out);

/*
 * mg_clean_adjoint -- vector-Jacobian product of the cleaning map
 * B -> B_new = B - grad phi, phi the solution of Lap phi = div B (second
 * order, Sec. 4.1; zero-mean projections when no face is Dirichlet):
 * dev_gB = dev_gBnew - D^T P^T A^-T Q^T G^T dev_gBnew, with D, G the
 * central divergence and gradient on the mesh (refinement ghosts
 * included) and the adjoint solve of mg_adjoint_solve (rel_tol,
 * max_cycles).  dev_gBnew and dev_gB hold dim leaf arrays back to back and
 * must not alias.  Cartesian meshes; the map is linear, so the result does
 * not depend on the tree's phi.  Returns as mg_adjoint_solve.
 */
int mg_clean_adjoint(mg_tree *t, const double *dev_gBnew, double *dev_gB, const mg_params *p, double rel_tol,
                     int max_cycles, int *cycles_done, double *rel_out);

/*
 * mg_set_schedule -- N_down / N_up of Sec. 2.4 chosen per level: down[l],
 * up[l] smoothing steps on level l = 0..n-1 (level 0 the coarsest, solved
 * exactly, so its entries are not used; 0..16, or -1 to keep the n_down /
 * n_up of the call's mg_params).  n = 0 clears the schedule.  Host arrays.
 * Applies to every later cycle of the tree (mg_vcycle, mg_fmg, mg_solve,
 * the adjoint).  mg_get_schedule writes the current per-level values (-1
 * where none is set) for levels 0..n-1.
 */
int mg_set_schedule(mg_tree *t, int n, const int *host_down, const int *host_up);
int mg_get_schedule(mg_tree *t, int n, int *host_down, int *host_up);

/*
 * mg_tune_schedule -- autotuner of the sweeps per level: times full solves
 * of the tree's current problem (phi = 0, FMG first, mg_solve to rel_tol in
 * `precision`) for candidate schedules -- (n_down, n_up) in {1, 2, 3} set
 * separately for the levels holding leaves and for the coarser levels, and
 * for MG_FP32_DC one to four inner cycles per outer step -- each run three
 * times (the first captures the graphs), and keeps the fastest candidate
 * that converges (mg_set_schedule).  A batch pool gives MG_ERR_ARG (use
 * mg_batch_tune_schedule).  *inner_cycles_out receives its inner
 * cycle count (pass it in mg_params.inner_cycles), *ms_out its solve time.
 * phi is restored afterwards.  MG_ERR_NOT_CONVERGED when no candidate
 * reaches rel_tol within max_cycles.  The paper has no counterpart (it
 * fixes N_down = N_up = 2).
 */
int mg_tune_schedule(mg_tree *t, double rel_tol, int max_cycles, int precision, int *inner_cycles_out,
                     double *ms_out);

/*
 * Instrumentation (the paper has no counterpart; used by the benchmark).
 * mg_launch_count: number of CUDA kernels this tree has launched so far.
 * mg_time_sweeps: runs n_sweeps red-black sweeps on `level` of the FP64
 * (precision MG_FP64) or FP32 (MG_FP32_DC) fields -- a real smoothing step,
 * the field changes -- each colour as one fused sweep launch followed by a
 * full ghost-fill launch, with CUDA events around every kernel on the
 * tree's stream.  out[0] = mean ms of one sweep launch (one colour, ghost
 * pushes included), out[1] = mean ms of one full ghost-fill launch,
 * out[2] = algorithmic bytes of one sweep launch (read x, f, eps and the
 * face ghosts once, write x once), out[3] = algorithmic bytes of one ghost
 * fill (read the source cells, write the ghosts once).  Synchronises.
 */
int mg_launch_count(mg_tree *t, int64_t *n);
/* mg_set_wait_limit: polls of every bounded wait in this tree's staged
 * kernels before the wait gives up (polls < 0: the default, 2^20, a few
 * milliseconds).  A kernel whose wait gives up sets the tree's status word,
 * lets its own copies in flight land (under the default bound) and returns;
 * the call that launched it returns MG_ERR_TIMEOUT and clears the word.
 * polls = 0 makes every staged kernel give up at once, which exercises that
 * path: no solve is meaningful until the limit is restored. */
int mg_set_wait_limit(mg_tree *t, int64_t polls);
/* mg_sweep_variant: the sweep kernel variant in use for a level and
 * precision (MG_FP64 / MG_FP32_DC): 0 persistent CTA-per-block TMA,
 * 1 CTA-per-block plain loads, 2 / 3 warp-per-block TMA (8 / 4 warps),
 * 4 / 5 row-wise warp TMA (8 warps x 2 stages / 4 warps x 3 stages),
 * 6 one thread per colour cell (blocks of at most 16 cells without
 * refinement faces), 7 / 8 / 9 row-wise warp TMA with the right-hand side
 * loaded into registers (FP32; 8 x 3, 4 x 4, 8 x 2), 10 variant 0 with
 * half-width CTAs (two colour cells per thread).  Variants 2-5 and 7-9
 * need 8^D blocks (4, 5, 7-9: 3D, constant coefficient, Cartesian).
 *
 * mg_set_sweep_variant: override the autotuner -- use `variant` on `level`
 * (level -1: on every level where it applies; variant -1: back to the
 * automatic choice).  MG_ERR_ARG when a single level is named and the
 * variant does not apply there.  Every variant computes the same red-black
 * half-sweep; this call exists to test and time them one by one. */
int mg_sweep_variant(mg_tree *t, int precision, int level, int *variant);
int mg_set_sweep_variant(mg_tree *t, int precision, int level, int variant);
/* mg_set_tail: an option for the small levels at the bottom of a V-cycle
 * (Sec. 2.4) -- groups of at most max_cells cells, from the coarsest up,
 * whose segments have no refinement faces: they run as one cooperative
 * launch per cycle leg (the downward steps, then after the coarsest solve
 * the upward steps), with a grid barrier between consecutive steps instead
 * of a kernel launch each.  max_cells <= 0 turns it off, the default: on
 * GB300, inside the solve's CUDA graphs, a barrier and a one-thread-per-item
 * step cost more than the launch they replace.  The result equals the
 * launch-by-launch cycle up to rounding order.  The damped-Jacobi smoother
 * always runs launch by launch.  MG_ERR_ARG on a null tree. */
int mg_set_tail(mg_tree *t, int64_t max_cells);
int mg_time_sweeps(mg_tree *t, int level, int n_sweeps, int precision, double out[4]);

/*
 * mg_residual_norm_noalloc -- the same composite residual norms as
 * mg_residual_norm (without the optional residual vector), for callers
 * whose device memory belongs to their own allocator (a pool reserved up
 * front) and who therefore may not call cudaMalloc or have memory allocated
 * on their behalf when they ask for a norm.  This call allocates nothing: its
 * reduction scratch is a fixed static device array of 16384 partial sums
 * (3 doubles each, 384 KiB) that every GPU loading this library holds until
 * the process exits.  A mesh whose residual launches need more partial sums
 * than that (for instance very many small leaf blocks) is rejected with
 * MG_ERR_ARG.  The first call on a device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture.  The address is cached per device for the life of the process,
 * so a reset of the device's primary context (cudaDeviceReset) while the
 * library stays loaded leaves it stale.  The tree's device must be current.
 * All calls share the array: calls that overlap on the GPU (from two
 * threads or two streams) race on it.  Synchronises the tree's stream.
 * Errors: MG_ERR_ARG (null tree or output, mesh beyond the scratch, another
 * device current), MG_ERR_STATE (tree not finalized), MG_ERR_CUDA,
 * MG_ERR_TIMEOUT, MG_ERR_NAN.  The paper has no counterpart.
 */
int mg_residual_norm_noalloc(mg_tree *t, double *l2, double *linf);

/* mg_tree_destroy -- free device and host memory (synchronises the stream). */
int mg_tree_destroy(mg_tree *t);

/* ------------------------------------------------------------- batch ----
 * Many independent trees solved together: every smoothing, transfer and
 * residual step is one launch over the blocks of all trees (the trees'
 * cycles are those of Sec. 2.4, run side by side), each tree keeps its own
 * exact coarsest-level solve, and a whole cycle plus its per-tree residual
 * norms is replayed as one CUDA graph.  In a batch of two or more trees a
 * tree whose coarsest level has a Dirichlet face and a non-periodic
 * dimension of at least 4 cells, across which a plane holds at most 64
 * cells, is solved by a block-tridiagonal factorisation over those planes
 * (2 nc P values read and FMAs per solve, P cells per plane) instead of
 * the dense inverse (nc^2).  Both are direct solves: in FP64 for FP64
 * cycles; inside the FP32 cycles of MG_FP32_DC the block form uses its
 * factors rounded to FP32 (the cycle is FP32 throughout and the outer FP64
 * defect correction removes its error).  Flat segments (blocks of at most
 * 16 cells) of a group share one launch per step.
 *
 * mg_batch_create -- merge n trees into a batch with its own device
 *   storage on `stream`.  The trees are read (mesh, refinement, boundary
 *   planes set with mg_set_bc_plane) and may be finalized or not; the batch
 *   keeps no reference to them, so they may be destroyed afterwards.  All
 *   trees must share dim, geometry, boundary types and values, lambda and
 *   lo; block size, base grid, hi and refinement may differ.
 *   MG_ERR_ARG on a mismatch, MG_ERR_BALANCE / MG_ERR_UNSUPPORTED as for
 *   mg_tree_finalize, MG_ERR_CUDA on allocation failure.
 *
 * Leaf data of a batch are the trees' leaf arrays (each in its tree's leaf
 * order) concatenated in tree order; mg_batch_leaf_offsets gives the n + 1
 * offsets (host_off[i] = first value of tree i, host_off[n] = total). */
int mg_batch_create(int n, mg_tree *const *trees, void *stream, mg_batch **out);
int mg_batch_leaf_offsets(mg_batch *b, int64_t *host_off);

/* Field I/O (FP64 device arrays of host_off[n] values), as mg_set_rhs,
 * mg_set_eps, mg_set_phi and mg_get_phi for every tree at once. */
int mg_batch_set_rhs(mg_batch *b, const double *dev_f);
int mg_batch_set_eps(mg_batch *b, const double *dev_eps);
int mg_batch_set_phi(mg_batch *b, const double *dev_phi);
int mg_batch_get_phi(mg_batch *b, double *dev_phi);

/* mg_batch_vcycle / mg_batch_fmg -- n V-cycles / one FMG cycle of every
 * tree (FP64), as mg_vcycle / mg_fmg. */
int mg_batch_vcycle(mg_batch *b, int n_cycles, const mg_params *p);
int mg_batch_fmg(mg_batch *b, const mg_params *p);

/* mg_batch_residual_norms -- composite residual norms of every tree, as
 * mg_residual_norm: host_l2[i], host_linf[i] for tree i (n values each).
 * Synchronises the stream. */
int mg_batch_residual_norms(mg_batch *b, double *host_l2, double *host_linf);

/* mg_batch_solve -- as mg_solve, cycling all trees together until every
 * tree's residual is at most rel_tol times its initial residual (a tree
 * that has converged keeps cycling with the others).  host_rel (optional,
 * n values) receives each tree's final relative residual; *cycles_done the
 * number of cycles.  MG_ERR_NOT_CONVERGED when some tree is above rel_tol
 * after max_cycles. */
int mg_batch_solve(mg_batch *b, double rel_tol, int max_cycles, int fmg_first, const mg_params *p,
                   int *cycles_done, double *host_rel);

/* Introspection: kernels launched so far; the segments (launch units) of
 * the batch -- per segment host_info = {block size, group, blocks, covered
 * blocks, coarsest flag, parent has the same block size}; and sweep timing
 * on one segment, as mg_time_sweeps. */
int mg_batch_launch_count(mg_batch *b, int64_t *n);
int mg_batch_num_segments(mg_batch *b, int *nseg, int *ngroups);
int mg_batch_segment_info(mg_batch *b, int seg, int32_t host_info[6]);
int mg_batch_time_sweeps(mg_batch *b, int segment, int n_sweeps, int precision, double host_out[4]);
/* mg_batch_set_tail -- mg_set_tail for the batch's pool (the bound applies
 * to the cells of a whole group, all trees together). */
int mg_batch_set_tail(mg_batch *b, int64_t max_cells);
/* mg_batch_tune_schedule -- mg_tune_schedule for a batch: the candidates
 * are timed as mg_batch_solve runs (every tree to rel_tol) and the chosen
 * schedule applies to the batch's segments (leaf segments and those above
 * the lowest one take the leaf sweeps). */
int mg_batch_tune_schedule(mg_batch *b, double rel_tol, int max_cycles, int precision, int *inner_cycles_out,
                           double *ms_out);
/* mg_batch_coarse_info -- the coarsest-level solves: host_out = {trees
 * solved by a dense inverse, trees solved in block-tridiagonal form, bytes
 * of the dense inverses, bytes of the block-tridiagonal plane records}. */
int mg_batch_coarse_info(mg_batch *b, int64_t host_out[4]);

/* mg_batch_destroy -- free the batch (synchronises its stream). */
int mg_batch_destroy(mg_batch *b);

/* Message of the last failed call on this thread ("" if none). */
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
