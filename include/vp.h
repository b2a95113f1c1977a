/*
 * vp.h -- C ABI of the GB300 volume-potential library (libvp.so).
 *
 * The library evaluates the free-space volume potential of a source sampled on
 * the leaves of a level-restricted quadtree (af Klinteberg, Askham & Kropinski,
 * "A fast integral equation method for the two-dimensional Navier-Stokes
 * equations", Sec. 2.1, Eq. vol_pot, in its scalar form):
 *
 *     u(x) = sum over leaves L of int_L G(x - y) f_L(y) dy,   and grad u(x),
 *
 * at every leaf node x, where f_L is the tensor Lagrange interpolant of the
 * nodal values of the leaf and G is one of
 *
 *     VP_KERNEL_MHELMHOLTZ   G1(r) = K0(alpha r) / (2 pi)
 *                            (free-space Green's function of alpha^2 - Laplacian,
 *                            the elliptic operator each implicit time step of
 *                            Sec. 2 reduces to);
 *     VP_KERNEL_MBIHARMONIC  G2(r) = (K0(alpha r) + log r) / (2 pi alpha^2)
 *                            = Q0(r) / (2 pi alpha^2) with Q0 of Sec. 3.2.1 (Eq. Q0);
 *                            minus the modified-biharmonic Green's function of
 *                            Sec. 2 (Eq. modbiharm), i.e. Laplacian(alpha^2 -
 *                            Laplacian) G2 = delta.
 *
 * Method: adjacent leaves interact through precomputed per-level leaf-to-leaf
 * tables (one dense matrix per relative position); well-separated interactions
 * go through a fast multipole method with expansions in K_n / I_n (and, for
 * G2, the log / r^n Laplace part), following the separation-of-variables
 * representations of Sec. 3.2.1 (Eqs. mpole, loc) on the level-restricted tree
 * of Sec. 3.2.1 ("Tree structure").
 *
 * Conventions shared by every entry point:
 *  - Root box: centre (cx, cy), side `root_side`. A leaf is (level, ix, iy):
 *    side h = root_side / 2^level, lower-left corner
 *    (cx - root_side/2 + ix*h, cy - root_side/2 + iy*h), 0 <= ix, iy < 2^level.
 *  - Each leaf carries p x p Gauss-Legendre nodes (tensor product of the
 *    p-point Gauss-Legendre rule mapped to the leaf); node (i, j), i the x
 *    index, has index j*p + i within its leaf; leaves are stored in the order
 *    given to vp_tree_upload. N = n_leaves * p * p.
 *  - Device pointers are plain CUDA device addresses owned by the caller
 *    (for example torch tensors' data_ptr()); handles are owned by the library.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Every call
 *    that takes a stream is asynchronous on it unless stated otherwise.
 *  - Every function returns VP_OK (0) or a negative VP_ERR_* code; nothing
 *    throws across the ABI. vp_strerror() names a code.
 */
#ifndef VP_H_
#define VP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vp_tables_s* vp_tables;
typedef struct vp_tree_s* vp_tree;

enum { VP_KERNEL_MHELMHOLTZ = 0, VP_KERNEL_MBIHARMONIC = 1 };
enum { VP_PREC_FP64 = 0, VP_PREC_SPLIT = 1 };

enum {
  VP_OK = 0,
  VP_ERR_ARG = -1,             /* an argument is out of range or NULL */
  VP_ERR_TREE_UNBALANCED = -2, /* adjacent leaves differ by more than one level */
  VP_ERR_LEVELS = -3,          /* a leaf is deeper than the tables were built for */
  VP_ERR_OOM = -4,             /* a device or host allocation failed */
  VP_ERR_CUDA = -5,            /* a CUDA runtime call failed */
  VP_ERR_TREE = -6,            /* leaves overlap, leave gaps, or lie outside the root */
  VP_ERR_TIMEOUT = -7          /* a bounded device wait ran out */
};

/*
 * vp_tables_build -- precompute every per-level operator for one kernel.
 *
 * Builds, on the device, for levels 0..levels (leaf side root_side/2^level):
 *  - the leaf-to-leaf near tables: for each of the 33 relative positions of
 *    an adjacent leaf (self, 8 same-level neighbours, 12 coarser and 12
 *    finer adjacent leaves) a dense [3 p^2 x p^2] matrix mapping the source
 *    leaf's nodal values to u, du/dx, du/dy at the target leaf's nodes
 *    (integrals of the kernel against the Lagrange basis, Eq. vol_pot);
 *  - the expansion operators of order `order` (the truncation P of Eqs.
 *    mpole/loc; 2P+1 real coefficients per channel): source-to-multipole,
 *    multipole-to-multipole, multipole-to-local (40 offsets), local-to-local,
 *    local-to-target (values and gradients), multipole-to-target and
 *    source-to-local for the adaptive W and X lists.
 *  kernel     VP_KERNEL_MHELMHOLTZ or VP_KERNEL_MBIHARMONIC.
 *  alpha      > 0.
 *  p          nodes per leaf side, 2 <= p <= 16.
 *  levels     deepest leaf level the tables serve, 0 <= levels <= 20.
 *  root_side  side of the root box (> 0); the tables depend on absolute leaf
 *             sizes because K0(alpha r) is not scale invariant.
 *  order      expansion order P, 4 <= P <= 60 (40 gives about 12 digits, as in
 *             Sec. 3.2.1).
 *  precision  VP_PREC_FP64 (all contractions in FP64) or VP_PREC_SPLIT (every
 *             contraction -- near tables, source-to-multipole, multipole-to-
 *             multipole, multipole-to-local, source-to-local, local-to-local,
 *             local-to-target, multipole-to-target -- on the tensor cores from
 *             exact 8-bit bf16 slices of the FP64 operands, folded in
 *             double-float; the kernel values and the level scaling of the
 *             operators are computed in FP64).
 *  stream     stream for the build kernels; the call synchronises it before
 *             returning.
 *  out        receives the handle; free with vp_tables_free.
 * Errors: VP_ERR_ARG, VP_ERR_OOM, VP_ERR_CUDA.
 */
int vp_tables_build(int kernel, double alpha, int p, int levels, double root_side, int order,
                    int precision, void* stream, vp_tables* out);

/*
 * vp_tree_upload -- validate a leaf list and build its interaction lists.
 *
 * Checks that the leaves tile the root box exactly (no overlap, no gap) and
 * that adjacent leaves differ by at most one level (the level restriction of
 * Sec. 3.2.1), builds the adaptive FMM lists (U: adjacent leaves; V: same-level
 * well-separated boxes; W/X: the mixed-level lists), groups every interaction
 * by operator, and uploads the work descriptors to the device.
 *  tables   built by vp_tables_build; must outlive the tree.
 *  cx, cy   root box centre (its side is the tables' root_side).
 *  level, ix, iy  HOST arrays of n_leaves entries (n_leaves >= 1).
 *  stream   stream for the uploads; the call synchronises it before returning.
 * Errors: VP_ERR_ARG, VP_ERR_TREE, VP_ERR_TREE_UNBALANCED, VP_ERR_LEVELS,
 * VP_ERR_OOM, VP_ERR_CUDA.
 */
int vp_tree_upload(vp_tables tables, double cx, double cy, int n_leaves, const int32_t* level,
                   const int32_t* ix, const int32_t* iy, void* stream, vp_tree* out);

/* Number of leaves and nodes (N = n_leaves * p^2) of a tree. */
int vp_tree_size(vp_tree tree, int64_t* n_leaves, int64_t* n_nodes);

/*
 * vp_tree_nodes -- node coordinates of the tree, computed on the device.
 *  xy  device array [2][N]: xy[0..N) = x, xy[N..2N) = y, in node order.
 */
int vp_tree_nodes(vp_tree tree, double* xy, void* stream);

/*
 * vp_tree_interp -- evaluate nodal fields off the grid through each leaf's tensor Lagrange
 * interpolant on its p x p Gauss-Legendre nodes (the same leaf polynomial that represents f in
 * Eq. vol_pot, Sec. 3.1). Used to carry a volume potential to boundary nodes (Sec. 2.2: the
 * boundary data of the homogeneous problem is the boundary condition minus the particular solution).
 *  fields  device [n_fields][N] nodal values in node order (e.g. gradu of vp_eval, n_fields = 2).
 *  xy      device [2][M] points; out device [n_fields][M].
 * A point on a leaf edge takes either adjacent leaf. Points outside the root box get NaN.
 * The first call on a tree allocates and fills a cell-to-leaf map of 4^L ints (L = deepest leaf
 * level; not inside graph capture). Errors: VP_ERR_ARG, VP_ERR_LEVELS (L > 13), VP_ERR_OOM,
 * VP_ERR_CUDA.
 */
int vp_tree_interp(vp_tree tree, int n_fields, const double* fields, int n_points, const double* xy, double* out,
                   void* stream);

/*
 * vp_eval -- the volume potential and its gradient at every node.
 *  f      device [N] nodal source values (read only).
 *  u      device [N] output.
 *  gradu  device [2][N] output: du/dx then du/dy.
 * Outputs are overwritten. The tree's work buffers are reused, so calls on
 * one tree must not overlap on the GPU (issue them on one stream).
 * Inside one call the near-field contraction runs on `stream` while the
 * far-field chain runs on a high-priority stream owned by the tree, forked
 * from and joined back to `stream` with events, so the call stays ordered on
 * `stream` as a whole (also under stream capture).
 * Errors: VP_ERR_ARG, VP_ERR_CUDA (launch failures are reported; asynchronous
 * faults surface at the next synchronising call).
 */
int vp_eval(vp_tree tree, const double* f, double* u, double* gradu, void* stream);

/*
 * vp_eval_host -- vp_eval from and to HOST memory.
 *  f (host [N]) in, u (host [N]) and gradu (host [2][N]) out; the call
 *  synchronises `stream` before returning. Page-locked buffers (cudaHostAlloc,
 *  cudaHostRegister) are used in place: the output reduction writes u and
 *  gradu straight into them, and trees on VP_PREC_SPLIT tables read f from
 *  them (f is read once, by the slicing kernel). Other buffers go through
 *  device staging copies owned by the tree (allocated on first use).
 */
int vp_eval_host(vp_tree tree, const double* f, double* u, double* gradu, void* stream);

/*
 * vp_special -- the device special functions the tables and expansion operators are built from,
 * evaluated at `count` arguments z (device array) for checks against reference values:
 *  which 0: out [2][count] = e^z K0(z), e^z K1(z) (small-argument series of App. C for z <= 2,
 *           the integral representation by the trapezoidal rule for 2 < z <= 25, the Hankel
 *           expansion beyond);
 *  which 1: out [nmax+1][count] = e^z Khat_n(z), Khat_n = K_n(z) (z/2)^n 2/(n-1)! (n >= 1),
 *           Khat_0 = K0 -- the normalised multipole basis of Sec. 3.2.1 (Eq. mpole);
 *  which 2: out [nmax+1][count] = Ihat_n(z) = I_n(z) n!/(z/2)^n -- the normalised local basis
 *           (Eq. loc); meant for the arguments the expansions use (z up to about 50).
 * 1 <= nmax <= 64 for which 1 and 2. Errors: VP_ERR_ARG, VP_ERR_CUDA.
 */
int vp_special(int which, int nmax, int count, const double* z, double* out, void* stream);

/* Stages of one evaluation, for vp_eval_timed and vp_tree_stats. */
enum {
  VP_STAGE_UPWARD = 0,   /* clear, source-to-multipole, multipole-to-multipole */
  VP_STAGE_M2L = 1,      /* multipole-to-local (V lists), source-to-local (X lists) */
  VP_STAGE_DOWNWARD = 2, /* local reduction, local-to-local */
  VP_STAGE_TARGETS = 3,  /* local-to-target, multipole-to-target (W lists) */
  VP_STAGE_NEAR = 4,     /* near tables (U lists) */
  VP_STAGE_OUTPUT = 5,   /* reduction into u and grad u */
  VP_NSTAGES = 6
};

/*
 * vp_eval_timed -- vp_eval with every stage issued in order on `stream` (no
 * overlap) and a CUDA event recorded between stages; waits for the last event
 * and writes the milliseconds of each stage to stage_ms[VP_NSTAGES] (host
 * array). Same arguments and errors as vp_eval.
 */
int vp_eval_timed(vp_tree tree, const double* f, double* u, double* gradu, void* stream, float* stage_ms);

/*
 * vp_tree_stats -- static work of one evaluation of `tree`:
 *  launches     number of kernel launches (and memsets) one vp_eval issues;
 *  stage_flops  host array [VP_NSTAGES]: algorithmic floating-point operations
 *               per stage (2*M*K per column of each contraction, one add per
 *               reduced element). Either pointer may be NULL.
 */
int vp_tree_stats(vp_tree tree, int64_t* launches, double* stage_flops);

/*
 * vp_tree_bytes -- algorithmic device-memory bytes of one evaluation per stage (host array
 * [VP_NSTAGES]): every operator matrix and every distinct source vector a launch reads counted
 * once, every output element counted once (twice when the launch accumulates into it), in the
 * representation the tree's precision uses (FP64, or S bf16 slices plus an exponent per row or
 * vector). The denominator of each stage's achieved bandwidth.
 */
int vp_tree_bytes(vp_tree tree, double* stage_bytes);

/*
 * vp_eval_steps -- vp_eval with every launch issued in order on `stream` and a CUDA event
 * recorded before each and after the last; waits for the last event. With cap = 0 only
 * *n_steps (the number of launches, including memsets) is returned. Otherwise cap >= *n_steps and
 * the host arrays receive, per launch k: ms[k] (milliseconds), info[4k..4k+3] = (kind: 0 FP64
 * contraction, 1 FP64 reduction, 2 memset, 3 slicing, 4 split contraction, 5 double-float
 * reduction; stage VP_STAGE_*; operator table id or -1; split engine or -1), flops[k] and
 * bytes[k] (algorithmic, as vp_tree_stats and vp_tree_bytes count them). Same device arguments
 * as vp_eval. Errors: VP_ERR_ARG, VP_ERR_CUDA.
 */
int vp_eval_steps(vp_tree tree, const double* f, double* u, double* gradu, void* stream, int cap, int* n_steps,
                  float* ms, int* info, double* flops, double* bytes);

/*
 * vp_plan_pairs -- host-only planning diagnostic (no GPU needed): validates a
 * leaf list like vp_tree_upload and returns, for every interaction the lists
 * generate, the covered (target leaf, source leaf) pairs with the mechanism
 * (0 near table, 1 multipole-to-local, 2 multipole-to-target, 3
 * source-to-local). Call with tgt = src = mech = NULL to get the count in
 * *n_out, then with arrays of that size. Errors as vp_tree_upload.
 */
int vp_plan_pairs(int n_leaves, const int32_t* level, const int32_t* ix, const int32_t* iy, int64_t* n_out,
                  int32_t* tgt, int32_t* src, int32_t* mech);

/*
 * Layer potential at the nodes of a tree (Sec. 2.2, Eqs. uH_dbl, dbl_lyr_pot: the homogeneous part
 * u^H = D[mu] of the velocity, as the boundary quadrature of Eq. dbl_lyr_quad; Sec. 3.2.1 for its
 * fast evaluation): for a density mu given at boundary points y_j with unit normals n_j (pointing
 * into the fluid domain, as for the boundary integral equation of bie.h) and quadrature weights w_j,
 *
 *     u_a(x) = sum_j D_ab(x, y_j) mu_b(y_j) w_j,   D_ab(x, y) = -T_bak(x - y) n_k(y),
 *
 * T the modified Stokes stresslet (App. B), at every node x of the tree (both velocity components).
 * The far field goes through the tree's expansions: multipole coefficients of the sources of each
 * leaf and local coefficients for the X lists come from sampling the kernel (split into its K0 and
 * log r derived parts, the two channels of Eqs. mpole and loc) on a circle, and the tree's
 * translation, multipole-to-local and target operators then apply as for the volume potential
 * (split precision when the tables are VP_PREC_SPLIT); sources in leaves adjacent to a target leaf
 * (and in the leaf itself) are summed directly in FP64 from matrices built at creation. Boxes
 * without sources below them are left out of the upward pass. The values at nodes close to the
 * boundary carry the error of the plain quadrature there, like the direct sum (Sec. 4 treats that).
 *
 * vp_layer_create -- bin the points into the tree's leaves and build the operators.
 *  tree    a tree on VP_KERNEL_MBIHARMONIC tables (the two-channel bases; VP_ERR_ARG otherwise);
 *          the layer uses the tree's tables (which must outlive it) but not its work buffers.
 *  n_src   number of boundary points (>= 1).
 *  src     HOST array [5][n_src]: x, y, n_x, n_y, w. Points must lie in the root box (VP_ERR_ARG).
 *  stream  stream for the set-up; synchronised before returning.
 * vp_layer_eval -- u (device [2][N]: u_x then u_y, node order as vp_eval) from mu (device
 *  [n_src][2]: (mu_x, mu_y) per point, in the order given to vp_layer_create). Calls on one layer
 *  must not overlap on the GPU; like vp_eval, the near part runs on `stream` while the far-field
 *  chain runs on a side stream joined back before the output.
 * vp_layer_steps -- vp_layer_eval with every launch timed in order, as vp_eval_steps.
 * vp_layer_near_star -- accurate values at the nodes close to the boundary (Sec. 4.2 and 4.4: the
 *  plain panel rule loses accuracy within about a panel length), for a layer whose points are the panel
 *  nodes of the star r(t) = R + A cos(k t + phase), t in [0, 2 pi) counter-clockwise, in n_panels equal
 *  parameter panels of 16 Gauss-Legendre nodes, panel after panel (as bie_nodes lists them; VP_ERR_ARG
 *  otherwise). Every (node, panel) pair closer than `dist` panel lengths (0 < dist <= 8; the paper tests
 *  1.2) gets the panel's contribution with the density interpolated by the panel's Lagrange basis,
 *  integrated on the exact curve by 20-point Gauss-Legendre on pieces graded dyadically toward the
 *  closest point, in place of the plain rule. The weight differences are built here on the device
 *  (FP64) and vp_layer_eval adds them after the tree sum. *n_pairs (may be NULL) receives the number of
 *  pairs. At most once per layer; synchronises `stream`.
 * Errors: VP_ERR_ARG, VP_ERR_OOM, VP_ERR_CUDA.
 */
typedef struct vp_layer_s* vp_layer;
int vp_layer_create(vp_tree tree, int n_src, const double* src, void* stream, vp_layer* out);
int vp_layer_eval(vp_layer layer, const double* mu, double* u, void* stream);
int vp_layer_steps(vp_layer layer, const double* mu, double* u, void* stream, int cap, int* n_steps, float* ms,
                   int* info, double* flops, double* bytes);
int vp_layer_near_star(vp_layer layer, double R, double A, int k, double phase, int n_panels, double dist,
                       void* stream, int64_t* n_pairs);
void vp_layer_free(vp_layer layer);

/*
 * Periodic particular solution by FFT (Sec. 2.1, Eqs. uhat, periodic_stokeslet, uP_Fourier,
 * uP_Fourier_deriv; Sec. 3.1.2): for a force F sampled on the uniform n x n grid of a periodic box of
 * side L (points x0 + i L/n, y0 + j L/n), the velocity of (alpha^2 - Laplacian) u + grad p = F,
 * div u = 0 with Fourier multiplier S_hat(k) = (I - k k^T/|k|^2) / (alpha^2 + |k|^2) (S_hat(0) = I /
 * alpha^2) and its gradient by Fourier differentiation (the Nyquist mode differentiates to zero).
 * The paper feeds it the PUX extension of the force; here the caller supplies a periodic force.
 * vp_periodic_create -- plan for alpha > 0, n a power of two in 32..4096, side L > 0 (work arrays of
 *  4 n^2 complex doubles on the device; synchronises `stream`).
 * vp_periodic_eval -- F device [2][n][n] (component, row j, column i), u device [2][n][n], gradu
 *  device [2][2][n][n] with gradu[a][m] = d u_a / d x_m. Calls on one plan must not overlap.
 * Errors: VP_ERR_ARG, VP_ERR_OOM, VP_ERR_CUDA.
 */
typedef struct vp_periodic_s* vp_periodic;
int vp_periodic_create(double alpha, int n, double side, void* stream, vp_periodic* out);
int vp_periodic_eval(vp_periodic plan, const double* F, double* u, double* gradu, void* stream);
void vp_periodic_free(vp_periodic plan);

/*
 * Semi-implicit spectral deferred correction time stepping (Sec. 3.3; Eqs. sisdc_initial,
 * sisdc_formula, rhs_initial, rhs_correction, rhs_correction_integral) of the Navier-Stokes equations
 * u_t + (u . grad) u = Laplacian u / Re - grad p, div u = 0 on a periodic box of side L, every implicit
 * substep solved by the periodic modified Stokes solution above with alpha^2 = Re / dt. Order K in
 * 1..4: K >= 2 takes K - 1 equal substeps of dt = Delta t / (K - 1) and K - 1 correction passes (K^2 - K
 * solves per step; global order K); K = 1 is one IMEX Euler step (one solve). The nonlinear term
 * (u . grad) u is formed pointwise on the grid from u and its Fourier gradient; the implicit term of a
 * substep is recovered from its own equation (Laplacian u - Re grad p = alpha^2 u - F).
 * vp_sdc_create -- Re > 0, Delta t > 0, order 1..4, n and L as vp_periodic_create (device memory:
 *  about (2 K^2 + 12) n^2 doubles; synchronises `stream`).
 * vp_sdc_set -- the state at the first time: u0 device [2][n][n], its gradient gradu0 [2][2][n][n]
 *  (gradu0[a][m] = d u_a / d x_m) and its Laplacian lap0 [2][n][n] (the paper supplies Laplacian u at the
 *  initial time, Sec. 3.3). Must precede vp_sdc_step and vp_sdc_get (VP_ERR_ARG otherwise).
 * vp_sdc_step -- advances n_steps steps of Delta t, all on `stream` without host synchronisation.
 * vp_sdc_get -- copies the current u [2][n][n] and its gradient [2][2][n][n] (device).
 * Calls on one stepper must not overlap on the GPU.
 * Errors: VP_ERR_ARG, VP_ERR_OOM, VP_ERR_CUDA.
 */
typedef struct vp_sdc_s* vp_sdc;
int vp_sdc_create(double re, double dt, int order, int n, double side, void* stream, vp_sdc* out);
int vp_sdc_set(vp_sdc sdc, const double* u0, const double* gradu0, const double* lap0, void* stream);
int vp_sdc_step(vp_sdc sdc, int n_steps, void* stream);
int vp_sdc_get(vp_sdc sdc, double* u, double* gradu, void* stream);
void vp_sdc_free(vp_sdc sdc);

/*
 * vp_eval_static -- vp_eval that allocates nothing.
 *
 * For callers that cannot call cudaMalloc (or any allocating routine) at the
 * time they evaluate -- a fixed memory budget handed out before the work
 * starts, an allocator that must not be touched while other work holds it.
 * The tree and tables are still created beforehand with vp_tables_build and
 * vp_tree_upload; this call then keeps every work buffer of the evaluation
 * (multipole/local coefficients and per-interaction contribution slots) in a
 * file-scope device array of VP_STATIC_SCRATCH_BYTES that every GPU loading
 * the library reserves until the process exits. The paper has no counterpart;
 * it is an interface convenience.
 *  tree, f, u, gradu, stream  as vp_eval (caller-owned device inputs and outputs).
 *  The first call on a device looks up the array's device address (once per
 *  device, with that device current); make that first call before any stream
 *  capture.
 *  All calls share the one array and it keeps the last call's contents (the
 *  parts that must start at zero are cleared by each call); calls that overlap
 *  on the GPU race, so issue them on one stream.
 * Errors: VP_ERR_ARG if the tree needs more than VP_STATIC_SCRATCH_BYTES of
 * work space (2*boxes*coefficients + contribution slots, in doubles) or was
 * built on VP_PREC_SPLIT tables; VP_ERR_CUDA.
 */
#define VP_STATIC_SCRATCH_BYTES (64u << 20)
int vp_eval_static(vp_tree tree, const double* f, double* u, double* gradu, void* stream);

/*
 * Engines of the split-precision contractions (trees on VP_PREC_SPLIT tables):
 *  0  warp-level mma.sync m16n8k16 (bf16 slices in, four fp32 accumulators in registers), tiles of
 *     128 rows x 64 columns;
 *  1  tcgen05.mma kind::f16 (bf16 slices) issued by one thread of a persistent CTA per SM, four fp32
 *     accumulators in tensor memory, tiles of 128 x 128; operator slices staged by one bulk copy per
 *     K step, gathered source columns by cp.async, a 4-stage ring handed over through mbarriers;
 *     every wait bounded;
 *  2  mma.sync as engine 0 on tiles of 64 x 32 (four times the blocks: for small launches whose
 *     time is the latency of a few tiles);
 *  3  tcgen05 as engine 1 on tiles of 128 x 64, with two sets of four accumulators in tensor
 *     memory, so that the epilogue of one tile overlaps the MMAs of the next (for short K, where
 *     draining the accumulators takes longer than filling them);
 *  4  tcgen05 on transposed tiles: the tile's 128 columns are the MMA's rows and the operator's rows
 *     its N (rounded up to 96 or 128), so operators of at most 128 rows (the 81-row multipole and
 *     local operators) fill every tensor-memory lane; launches with taller operators run on engine 1.
 * All compute the same exact slice sums. vp_tree_set_engine sets one engine for every launch of
 * the tree (VP_ERR_ARG for other values). vp_autotune times each split-precision launch of one
 * evaluation of `f` with every engine (tile shape) on `stream`, keeps the fastest per launch shape,
 * evaluates once more into u, gradu with the choice, and, if *n_tcgen05 is given, reports how many
 * launches use a tcgen05 engine (1, 3 or 4).
 * With cache_path (may be NULL) the choices are read from / appended to a text file keyed by
 * (p, P, channels, operator, rows, padded K, tiles). Trees on FP64 tables are left unchanged.
 * vp_device_status reads and clears the device flag a bounded wait sets when it gives up:
 * VP_ERR_TIMEOUT if it was set, VP_OK otherwise (synchronising).
 */
int vp_tree_set_engine(vp_tree tree, int engine);
int vp_autotune(vp_tree tree, const double* f, double* u, double* gradu, const char* cache_path, void* stream,
                int* n_tcgen05);
int vp_device_status(void);

/*
 * vp_selftest_timeout -- exercises the give-up path of the bounded device waits: a one-thread
 * kernel waits on an mbarrier that nothing arrives at, gives up after about two million clocks
 * (about a millisecond), raises the device flag and returns; the call synchronises `stream` and
 * returns what vp_device_status then reports: VP_ERR_TIMEOUT when the path works (the flag is
 * cleared again). The device stays usable afterwards.
 */
int vp_selftest_timeout(void* stream);

/*
 * Batches -- many independent trees (each with its own tables: kernel, alpha, p and depth may all
 * differ) evaluated together.
 *
 * vp_batch_create records one CUDA graph that evaluates tree t from f[t] into u[t], gradu[t] for
 * every t (device pointers, layouts as vp_eval). Each tree's evaluation becomes one branch of the
 * graph, captured on one of n_streams forked streams (1..128), so the GPU overlaps the trees.
 * The graph keeps the pointers it was recorded with: the caller keeps those buffers (and the trees)
 * alive and in place for the batch's lifetime and writes new sources into the same f[t] buffers.
 * A tree may appear in only one batch that runs at a time (its work buffers are reused).
 * `stream` is used for the capture (it must not be capturing already).
 * vp_batch_run replays the graph on `stream` (asynchronous).
 * vp_batch_stats: total nodes of the batch and kernel launches per replay.
 * vp_eval_batched: one-shot form; use_graph != 0 creates, runs (synchronising `stream`) and frees a
 * batch with 16 streams; use_graph == 0 issues the trees one after another on `stream`.
 * Errors: VP_ERR_ARG, VP_ERR_OOM, VP_ERR_CUDA. (Overlapping trees through a graph is not in the
 * paper; it is how this library fills one GPU with many small problems.)
 */
typedef struct vp_batch_s* vp_batch;
int vp_batch_create(int n_trees, const vp_tree* trees, const double* const* f, double* const* u,
                    double* const* gradu, int n_streams, void* stream, vp_batch* out);
int vp_batch_run(vp_batch batch, void* stream);
int vp_batch_stats(vp_batch batch, int64_t* nodes, int64_t* launches);
void vp_batch_free(vp_batch batch);
int vp_eval_batched(int n_trees, const vp_tree* trees, const double* const* f, double* const* u,
                    double* const* gradu, int use_graph, void* stream);

/* Free a tree (after work on it has finished) / tables (after their trees). */
void vp_tree_free(vp_tree tree);
void vp_tables_free(vp_tables tables);

/* Static description of an error code. */
const char* vp_strerror(int code);

/* Name of the last CUDA runtime error the library saw in this thread (diagnostics for VP_ERR_CUDA). */
const char* vp_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VP_H_ */
