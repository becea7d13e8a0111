/*
 * eb.h -- C ABI of the GB300 (sm_103a) embedded-boundary Laplacian library.
 *
 * The method: Peng, Appelo & Liu, "Universal AMG accelerated embedded boundary
 * method without small cell stiffness" (arXiv 2204.06083).  Dirichlet problems
 * on a domain Omega embedded in a uniform Cartesian grid are discretised by
 * central differences (eq. 3, beta = 1) at the computational points (CPs,
 * Sec. 2); the values at the interior boundary points (BPs) are eliminated by
 * the line-by-line interpolant of Sec. 2.1 (eqs. 4-6), which changes only the
 * diagonal of the matrix.  The resulting A = -L is symmetric and diagonally
 * dominant; it is solved by CG with an AMG preconditioner (Algorithm 1 step 4)
 * and marched in time by the theta-scheme of Sec. 3.5 (theta = 0: leapfrog)
 * and by the theta-method for the heat equation (Sec. 3.4).
 *
 * Conventions shared by every call
 *   - Every call returns an eb_status; EB_OK is 0.  eb_last_error() gives a
 *     thread-local message for the last failing call on this host thread.
 *     No C++ exception crosses this boundary.
 *   - Vectors are caller-owned DEVICE pointers in the full-grid layout: one
 *     entry per grid node, node (i, j, k) at i + n0 (j + n1 k) (x fastest),
 *     n0*n1*n2 entries.  The entries at nodes that are not CPs are ignored on
 *     input.  On output every node of the "active tiles" (the tiles of the
 *     grid that contain at least one CP, see eb_info) is written, with 0 at
 *     the non-CP nodes; nodes outside the active tiles are never written, so
 *     callers that read the whole grid should zero-initialise outputs once.
 *   - Geometry and option structs are HOST pointers read during the call.
 *   - Calls that take a cudaStream_t are asynchronous on that stream unless
 *     noted "synchronous" (those read a result back to the host).
 *   - Handles own all their device memory and are released by *_destroy.
 *     A handle built on another (an AMG hierarchy on its grid, a geometry
 *     borrowed from a batch) must not be used after the one it was built on
 *     is destroyed; destroying it is allowed in either order.
 */
#ifndef EB_H_
#define EB_H_

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EB_OK = 0,
  EB_ERR_INVALID = 1,        /* bad argument, size or handle */
  EB_ERR_GEOMETRY = 2,       /* Omega touches the outermost node ring, or no CP */
  EB_ERR_CUDA = 3,           /* a CUDA runtime call failed (message has details) */
  EB_ERR_NONFINITE = 4,      /* NaN / Inf in an input or a reduction */
  EB_ERR_NO_CONVERGENCE = 5, /* maxit reached; statistics are still filled */
  EB_ERR_BREAKDOWN = 6,      /* p^T A p <= 0 or r^T z <= 0 in CG */
  EB_ERR_TIMEOUT = 7,        /* a device-wide barrier gave up waiting */
  EB_ERR_OOM = 8,            /* device allocation failed or a capacity was exceeded */
  EB_ERR_NOT_IMPLEMENTED = 9
} eb_status;

/* EB_DF64 (pcg_opts.outer_prec only): double-float, a value held as the
 * unevaluated sum of two FP32 numbers (about 48 significant bits) and computed
 * with error-free FP32 transformations */
typedef enum { EB_F64 = 0, EB_F32 = 1, EB_BF16 = 2, EB_DF64 = 3 } eb_prec;

/* Uniform grid: n[a] nodes on axis a at lo[a] + i h, i = 0..n[a]-1 (Sec. 2).
 * dim is 2 or 3; for dim 2, n[2] must be 1.  n[0] must be a multiple of 2. */
typedef struct {
  int dim;
  int n[3];
  double lo[3];
  double h;
} eb_grid;

/* Level set psi, psi < 0 strictly inside Omega (Sec. 2, mask m_ij).
 *  EB_LS_QUADRIC: psi = sum_a (y_a/semi[a])^2 - 1, y = Q^T (x - center),
 *                 Q = rot (row-major 3x3; only the leading dim x dim block is
 *                 used in 2D).  Circle, sphere and rotated ellipsoid.
 *                 Grid-line roots are found in closed form.
 *  EB_LS_STAR2D:  psi = |x - c| - r(phi), r(phi) = r0 + sum_k a[k] sin(k[k]
 *                 phi + p[k]), phi = atan2(y - c_y, x - c_x); 2D only.  Grid-
 *                 line roots by the Illinois (safeguarded secant) iteration,
 *                 the secant root finder named in Sec. 2.1.
 *  EB_LS_SAMPLED: psi known only at the grid nodes: psi points to a caller-
 *                 owned DEVICE array of n0 n1 n2 doubles in the full-grid
 *                 layout, read during eb_build only (not kept).  The crossing
 *                 beyond a BP is the linear-ratio distance of Sec. 3.3 between
 *                 the last inside node (psi_in < 0, m nodes beyond the BP) and
 *                 the next node (psi_out >= 0): delta = m h + psi_in /
 *                 (psi_in - psi_out) h.  Second-order accurate for a smooth
 *                 psi; 2D and 3D.  The other fields are ignored. */
typedef enum { EB_LS_QUADRIC = 0, EB_LS_STAR2D = 1, EB_LS_SAMPLED = 2 } eb_ls_kind;

#define EB_STAR_MAX_TERMS 16
typedef struct {
  int kind;
  double center[3];
  double semi[3];
  double rot[9];
  double r0;
  int nk;
  int k[EB_STAR_MAX_TERMS];
  double a[EB_STAR_MAX_TERMS];
  double p[EB_STAR_MAX_TERMS];
  const double* psi;     /* EB_LS_SAMPLED only: psi at the nodes (device); NULL otherwise */
} eb_levelset;

typedef struct eb_handle eb_handle;
typedef struct amg_handle amg_handle;

typedef struct {
  int64_t num_nodes;     /* n0 n1 n2 */
  int64_t num_cp;        /* N_C, the number of unknowns (Algorithm 1 step 1) */
  int64_t num_bp;        /* interior boundary points */
  int64_t num_cut;       /* (CP, direction) pairs with a BP neighbour */
  int64_t num_far;       /* cuts whose boundary crossing lies beyond the BP's next node (delta > h) */
  int64_t num_tiles;     /* active tiles (tiles holding >= 1 CP) */
  int tile[3];           /* tile extents in nodes */
  double max_delta_over_h;
  double min_abs_psi;    /* smallest |psi| over all nodes: the classification margin */
  double min_dominance_margin;  /* smallest D_k - sum_j |h^2 a_kj| over the rows with a cut, i.e. the
                                   smallest sum of c_s over the BP directions of a CP (h^2 units): > 0
                                   means strict diagonal dominance of every cut row (Sec. 2.1); interior
                                   rows have margin 0 (RBF cuts may make it negative, Sec. 2.4) */
  int64_t num_rbf;       /* cuts closed by RBF interpolation (mixed / RBF-based closures) */
  int64_t num_rbf_rotated;  /* of those, with G2 from Algorithm 2's rotated line */
} eb_info_t;

/* Closure of the boundary points (Sec. 2.3).
 *  EB_CLOSURE_LINE:  line-by-line interpolation everywhere (Sec. 2.1); when the
 *                    node past the BP is inside, the crossing is the first one
 *                    walking outward along the grid line (delta may exceed h).
 *  EB_CLOSURE_MIXED: line-by-line where the node past the BP is outside, the
 *                    RBF interpolation of Sec. 2.2 elsewhere (the paper's
 *                    "mixed" method, Algorithm 1 step 3).
 *  EB_CLOSURE_RBF:   RBF interpolation at every cut ("RBF-based").
 * RBF cuts: u_BP = w_ij u_ij + w_1 u_G1 + w_2 u_G2 from the cubic polyharmonic
 * RBF with linear augmentation (eqs. 7-9) through the CP and two boundary
 * points chosen by Algorithm 2 (G1 nearest to x_BP; G2 nearest to the CP if
 * more than rbf_eps h from G1, else the crossing of the line x_BP -> G1 turned
 * counterclockwise by pi/4).  The cut's diagonal term becomes 1 - w_ij, its
 * crossing point G1; its second value u_G2 is an extra boundary sample.  The
 * RBF forms need a 2D quadric or star level set (EB_ERR_NOT_IMPLEMENTED
 * otherwise); their nearest points are found on the descriptor's curve by 256
 * parameter samples and Newton's method (Sec. 3.3). */
typedef enum { EB_CLOSURE_LINE = 0, EB_CLOSURE_MIXED = 1, EB_CLOSURE_RBF = 2 } eb_closure;
typedef struct {
  int closure;           /* eb_closure, default EB_CLOSURE_LINE */
  double rbf_eps;        /* Algorithm 2's epsilon, default 0.025 */
} eb_build_opts;

/* Algorithm 1 steps 1-3 on the device: classifies every node (mask, BP, CP),
 * numbers the CPs lexicographically, finds for every CP and axis direction
 * whose neighbour is a BP the first crossing of Gamma walking outward from the
 * BP along the grid line (delta = distance BP -> Gamma), and forms the
 * diagonal D_k = sum_s c_s with c_s = 1 towards a CP and c_s = h/(h+delta)
 * towards a BP (Sec. 2.1: g_Gamma of eq. 6 evaluated at the BP).
 * Synchronous (reads N_C back).  EB_ERR_GEOMETRY when an inside node lies on
 * the outermost ring of the grid or when there is no CP; EB_ERR_INVALID for
 * an EB_LS_SAMPLED level set without psi. */
int eb_build(const eb_grid* grid, const eb_levelset* ls, eb_handle** out, cudaStream_t stream);
/* eb_build with a closure (opts may be NULL: EB_CLOSURE_LINE).  With RBF cuts
 * the right-hand side takes num_cut + num_rbf boundary values (eb_rhs). */
int eb_build_ex(const eb_grid* grid, const eb_levelset* ls, const eb_build_opts* opts, eb_handle** out,
                cudaStream_t stream);
/* The RBF cuts (device buffers of num_rbf entries, any may be NULL): the cut
 * index of each (ascending), its second boundary point G2 (num_rbf x 2), its
 * weights (w_ij, w_1, w_2) (num_rbf x 3) and whether G2 came from the rotated
 * line (1) or is the point nearest to the CP (0). */
int eb_rbf_cuts(const eb_handle* eb, int32_t* cut_index_dev, double* xg2_dev, double* weights_dev,
                int32_t* rotated_dev, cudaStream_t stream);
void eb_destroy(eb_handle* eb);
int eb_info(const eb_handle* eb, eb_info_t* out);

/* Variable coefficient of eq. 3: div(beta grad u) = f.  beta_a_dev (a = x, y
 * and, in 3D, z) are caller-owned DEVICE arrays of n0 n1 n2 doubles in the
 * full-grid layout holding beta at the half point node + h/2 e_a of every
 * node (the beta_{i+1/2} of eq. 3 on axis a); they are copied (FP64 and FP32)
 * and may be freed on return.  Every operator of the handle then uses the
 * beta-weighted stencil: the coupling of neighbours k, j is -beta/h^2 with the
 * beta of their half point, and the closure of Sec. 2.1 leaves beta_s c_s on
 * the diagonal and beta_s c_s u_Gamma / h^2 in eb_rhs, so D_k = sum_s beta_s
 * c_s (eb_cp_data).  beta must be positive and finite at every half point a
 * CP uses (EB_ERR_INVALID otherwise; for a negative constant beta solve the
 * negated equation); beta_z_dev is ignored in 2D.  Call once, before
 * amg_setup (hierarchies built earlier describe beta = 1 and must not be used
 * with the handle afterwards).  EB_ERR_NOT_IMPLEMENTED for a geometry
 * borrowed from a batch; the learned stage rejects such grids.  Synchronous. */
int eb_set_beta(eb_handle* eb, const double* beta_x_dev, const double* beta_y_dev, const double* beta_z_dev,
                cudaStream_t stream);

/* Node classes as one byte per node (full grid), written to a device buffer
 * of num_nodes bytes: 0 outside, 0x40 BP, 0x80|m CP where bit s of m (s = 2
 * axis + (0 for -, 1 for +)) marks a BP neighbour in direction s. */
int eb_classes(const eb_handle* eb, uint8_t* code_dev, cudaStream_t stream);
/* Per-CP data, device buffers of num_cp entries: the node index of CP k and
 * its diagonal D_k in units of 1/h^2. */
int eb_cp_data(const eb_handle* eb, int32_t* cp_node_dev, double* diag_dev, cudaStream_t stream);
/* Per-cut data, device buffers of num_cut entries, ordered by (CP, direction):
 * CP index, direction s, delta, and the crossing point (num_cut x dim, row-major).
 * Any pointer may be NULL. */
int eb_cuts(const eb_handle* eb, int32_t* cut_cp_dev, int32_t* cut_dir_dev, double* delta_dev,
            double* xg_dev, cudaStream_t stream);

/* Right-hand side of A u = b for div(grad u) = f with u = u_Gamma on Gamma:
 * b_k = -f_k + sum_s c_s u_Gamma,s / h^2 (the g_Gamma u_Gamma term of
 * Sec. 2.1).  f: full grid; ugamma: one value per cut (eb_cuts order, at the
 * cut's crossing point), followed, with RBF cuts, by one value per RBF cut at
 * its G2 (eb_rbf_cuts order): num_cut + num_rbf values; an RBF cut adds
 * (w_1 u_G1 + w_2 u_G2) / h^2.  b: full grid output. */
int eb_rhs(const eb_handle* eb, const double* f_dev, const double* ugamma_dev, double* b_dev,
           cudaStream_t stream);

/* y = A x, A = -L of eq. 3 with the line-by-line diagonal (Sec. 2.1), matrix
 * free.  x and y have the element type of prec (double, float, bf16).  y is
 * written at the CPs and, with 0, at the other node of every x-pair (2j,
 * 2j + 1) that holds a CP; its other nodes keep their values (pass a zeroed y
 * for a full-grid result).  x's entries off the CPs do not affect y. */
int eb_apply(const eb_handle* eb, int prec, const void* x_dev, void* y_dev, cudaStream_t stream);

/* --------------------------------------------------------------- tile shapes
 * The grid kernels walk the "active tiles" of a grid: blocks of 256 nodes,
 * tile[0] x tile[1] x tile[2] with power-of-two extents, x fastest (eb_info
 * reports the shape in use; eb_build starts from 32 x 8 in 2D and 16 x 4 x 4
 * in 3D).  The shape changes how the work is cut into CTAs, never a result.
 * The paper has no counterpart: this is how the library is fitted to a GPU. */
typedef struct {
  int count;         /* candidate shapes timed */
  int tile[16][3];   /* the candidates */
  double us[16];     /* mean duration of the timed operation with each (microseconds) */
  int best;          /* index of the shape in use on return */
} eb_tune_t;

/* Rebuilds the active-tile list of eb for the given shape (powers of two,
 * product 256, 2 <= tile[0] <= 128, tile[1], tile[2] <= 128, tile[2] = 1 in
 * 2D; EB_ERR_INVALID otherwise).  Hierarchies and captured iterations built on
 * eb stay valid (their next solve captures again).  Do not call while work on
 * eb is in flight on another stream.  Synchronous. */
int eb_retile(eb_handle* eb, const int tile[3], cudaStream_t stream);
/* Operations the grid autotuner can time. */
typedef enum { EB_TUNE_APPLY = 0, EB_TUNE_LEAPFROG = 1 } eb_tune_op;
/* Autotuner: for each candidate shape, times `reps` calls of the operation
 * (EB_TUNE_APPLY: one eb_apply launch; EB_TUNE_LEAPFROG: one wave_step of 16
 * steps) in precision prec (EB_F64, EB_F32; EB_BF16 for apply) with CUDA
 * events on stream, and keeps the fastest shape.  out (may be NULL) receives
 * the timings.  Synchronous. */
int eb_autotune(eb_handle* eb, int op, int prec, int reps, eb_tune_t* out, cudaStream_t stream);

/* ---------------------------------------------------------------- AMG + PCG */
/* EB_PC_AMG_NN (V-cycle followed by the learned stage) is selected by
 * pcg_solve_nn only; pcg_solve rejects it. */
typedef enum { EB_PC_AMG = 0, EB_PC_JACOBI = 1, EB_PC_NONE = 2, EB_PC_AMG_NN = 3 } eb_pc_kind;

/* Coarsening of amg_setup: smoothed aggregation (the default) or the classical
 * Ruge-Stueben method the paper uses (Sec. 3): strength -a_ij >= 0.25
 * max_k(-a_ik), the independent-set (PMIS) form of its C/F splitting with
 * measure |S_i^T| and lowbias32 tie-break, direct interpolation. */
typedef enum { EB_AMG_SA = 0, EB_AMG_RS = 1 } eb_amg_coarsening;

typedef struct {
  int max_levels;        /* default 25 */
  int coarse_max;        /* coarsen until n <= coarse_max (default 1024) */
  double strength;       /* theta of |a_ij| >= theta sqrt(a_ii a_jj), default 0.02 */
  int cheb_degree;       /* Chebyshev smoother degree, default 2 */
  int vcycle_prec;       /* storage of level vectors/matrices: EB_F64 (default), EB_F32, or EB_BF16
                            (bfloat16 storage, FP32 sums; the level-0 diagonal stays FP32); the
                            reduced precisions make pcg_solve use the flexible (Polak-Ribiere) beta */
  int coarsening;        /* eb_amg_coarsening, default EB_AMG_SA (strength then ignored for EB_AMG_RS) */
  int cycle;             /* 1 (default): V-cycle; 2: W-cycle (every coarse-grid correction is two cycles
                            of the coarser level, the second from the first one's result; Sec. 3) */
} amg_opts;

typedef struct {
  int num_levels;
  int64_t rows[32];
  int64_t nnz[32];
  double operator_complexity;
  double setup_ms;
} amg_info_t;

/* Smoothed-aggregation AMG hierarchy for sigma I + A (sigma = shift >= 0;
 * sigma = 1/dt for the implicit heat step).  The paper uses a library AMG
 * (Sec. 3, first paragraph); this hierarchy is deterministic: strength
 * |a_ij| >= theta sqrt(a_ii a_jj); distance-2 maximal independent set with
 * priorities (lowbias32 hash of the index, index); aggregates grown from its
 * nodes; P = (I - 4/(3 rho) D^-1 A) P_hat; Galerkin A_c = P^T A P; on the
 * coarsest level an explicit dense inverse formed by Gauss-Jordan elimination
 * without pivoting (the coarsest matrix is SPD), applied as a dense
 * matrix-vector product.  opts may be NULL for the defaults.
 * Synchronous. */
int amg_setup(const eb_handle* eb, double shift, const amg_opts* opts, amg_handle** out, cudaStream_t stream);
void amg_destroy(amg_handle* amg);
int amg_info(const amg_handle* amg, amg_info_t* out);
/* Copies of one level for inspection: CSR of A_l (which = 0) or P_l (which =
 * 1) into caller device buffers sized from amg_info (rows + 1, nnz), and the
 * aggregate id of each row of level l (which = 2, into col_dev). */
int amg_level_copy(const amg_handle* amg, int level, int which, int32_t* rowptr_dev, int32_t* col_dev,
                   double* val_dev, cudaStream_t stream);
/* z = M^-1 r: one symmetric V-cycle (Chebyshev pre/post smoothing). */
int amg_vcycle(const amg_handle* amg, const double* r_dev, double* z_dev, cudaStream_t stream);
/* Tile-shape autotuner for a solve: retiles the hierarchy's grid with each
 * candidate shape, times `reps` V-cycles, keeps the fastest (see eb_autotune).
 * Synchronous. */
int amg_autotune(amg_handle* amg, int reps, eb_tune_t* out, cudaStream_t stream);
/* Tunes the row groups of the V-cycle's CSR kernels (coarse levels, level-0
 * restriction and prolongation): a group of G <= 32 lanes owns one row, G the
 * largest power of two with G x (entries per lane) <= the mean row length.
 * Times `reps` V-cycles with 1, 2, 4 and 8 entries per lane, keeps the
 * fastest.  us_out (4 doubles, may be NULL) receives the timings, best_out
 * (may be NULL) the entries per lane chosen.  Results do not change (the sums
 * are grouped differently: FP rounding only).  Synchronous. */
int amg_tune_csr(amg_handle* amg, int reps, double* us_out, int* best_out, cudaStream_t stream);
/* Sets the entries per lane of the CSR kernels' row groups (1, 2, 4 or 8; see
 * amg_tune_csr) without timing, e.g. to a value a previous tuning found.  The
 * paper has no counterpart.  EB_ERR_INVALID for other values. */
int amg_set_csr_epl(amg_handle* amg, int epl);
/* Times one V-cycle kernel on its own (instrumentation; the paper has no
 * counterpart).  kernel EB_TK_SMOOTH_STEP: one Chebyshev smoothing step of
 * level `level` (level 0: the stencil kernel of Sec. 2 over the active tiles;
 * coarser levels: the CSR kernel with the tuned row groups), in its V-cycle
 * launch configuration, on the hierarchy's own matrices and level vectors.
 * `launches` (1..10000) back-to-back launches are captured in one CUDA graph
 * and timed by events around the graph, so no per-launch event enters the
 * figure.  clear_bytes > 0: each launch is preceded by a read of a buffer of
 * that many bytes (choose more than the L2 size), so that the kernel finds
 * none of its data in L2 and no dirty lines to write back, as after a cache
 * flush; the time of the reads alone, measured the same way, is subtracted.
 * The buffer is allocated for the call.
 * level must have a coarser level below it.  Overwrites the level's smoother
 * vectors: call between solves.  us_out: microseconds per launch.
 * Synchronous. */
enum { EB_TK_SMOOTH_STEP = 0 };
/* The size-matched reference of amg_time_kernel (instrumentation; the paper
 * has no counterpart): a plain streaming copy that reads bytes/2 and writes
 * bytes/2 (16-byte accesses, grid-stride), timed the same way -- `launches`
 * back-to-back launches in one graph, each preceded by a read of clear_bytes
 * when > 0, whose time is subtracted -- so that a kernel moving the same bytes
 * can be compared with the best a single launch of that size achieves.  The
 * buffers are allocated for the call.  Synchronous. */
int eb_time_copy(int64_t bytes, int launches, int64_t clear_bytes, double* us_out, cudaStream_t stream);
/* eb_apply timed like amg_time_kernel (instrumentation; the paper has no
 * counterpart): `launches` (1..10000) back-to-back eb_apply launches of
 * precision prec on x_dev -> y_dev, captured in one CUDA graph and timed by
 * events around it; clear_bytes > 0 puts a read of a buffer of that many
 * bytes before each launch (its own time subtracted), so that every launch
 * finds its data in DRAM.  us_out: microseconds per launch.  y_dev is written
 * as by eb_apply.  The clear buffer is allocated for the call.  Synchronous. */
int eb_time_apply(const eb_handle* eb, int prec, const void* x_dev, void* y_dev, int launches, int64_t clear_bytes,
                  double* us_out, cudaStream_t stream);
int amg_time_kernel(const amg_handle* amg, int kernel, int level, int launches, int64_t clear_bytes, double* us_out,
                    cudaStream_t stream);

/* Measured FP64 arithmetic peak of the current GPU (instrumentation; the paper
 * has no counterpart): a kernel of independent fused multiply-add chains with
 * no memory traffic, `reps` launches (1..10000) timed by CUDA events on
 * stream; *tflops_out = FP64 TFLOP/s (an FMA counts 2).  The roof of the FP64
 * kernels whose time is spent in the FP64 pipe.  Synchronous. */
int eb_fp64_peak(int reps, double* tflops_out, cudaStream_t stream);

typedef struct {
  int precond;           /* eb_pc_kind, default EB_PC_AMG */
  int check_every;       /* host convergence check period in iterations (default 1) */
  int use_graph;         /* 1 (default): the whole iteration loop runs on the device in one graph launch (a
                            conditional WHILE node around one captured iteration; no host round trip per
                            iteration); with profile set, or 2: captured chunks of check_every iterations
                            with a host convergence check between them; 0: direct launches */
  int profile;           /* 1: time every level-0 smoother launch with CUDA events; 2 (pcg_solve_nn):
                            time the learned stage's 32 -> 32 convolution launches instead; 3: time the
                            level-1 (first coarse level, CSR) Chebyshev-step launches; 4: the PCG's
                            p update + operator apply launches; 5: its x/r update launches (with an AMG
                            V-cycle, fused with the first level-0 smoothing step) */
  int outer_prec;        /* arithmetic of the outer iteration's vectors x, r, p, q: EB_F64 (default) or
                            EB_DF64 -- double-float pairs in the same 8 bytes per entry, updated on the FP32
                            pipe (GB300 issues FP64 and float <-> double conversions at under 2 lanes per
                            clock per SM, FP32 at about 116); z is then the V-cycle's FP32 output, the
                            reductions are summed in DF and rounded to FP64 once per CTA, the scalars are
                            FP64, and b and x cross to DF scaled by a power of two (the scaled b has a
                            unit root mean square).  The exit test is the FP64 true residual, as for
                            EB_F64.  EB_DF64 needs EB_PC_AMG with an FP32 or BF16 V-cycle of two or more
                            levels (EB_ERR_NOT_IMPLEMENTED otherwise); a variable beta (eb_set_beta) enters
                            through DF copies of beta at the half points and of D_k */
} pcg_opts;

typedef struct {
  int iterations;
  double rel_residual;       /* ||r_k|| / ||b|| of the recurrence at exit */
  double true_rel_residual;  /* ||b - A x|| / ||b|| recomputed at exit */
  double solve_ms;
  int converged;
  double prof_kernel_ms;     /* with opts.profile: summed duration of the timed launches */
  int prof_launches;         /* with opts.profile: their number */
  int64_t launches;          /* kernel launches this solve issued */
} pcg_stats;

/* The outer precision (pcg_opts.outer_prec) of the solves that take no
 * options of their own: heat_step, wave_theta_step and pcg_solve with NULL
 * opts.  EB_F64 (the default) or EB_DF64: double-float where that iteration
 * applies (an FP32 or BF16 V-cycle of two or more levels), FP64 for the
 * others (e.g. a hierarchy that a large shift leaves at one level).
 * EB_ERR_INVALID for other values or a NULL handle. */
int amg_set_outer_prec(amg_handle* amg, int prec);

/* Solves (sigma I + A) x = b by PCG (Algorithm 1 step 4) with the
 * preconditioner of opts, stopping when ||r_k||_2 / ||b||_2 <= rtol; at exit
 * the true residual is recomputed and the iteration continues if it misses
 * rtol.  x holds the initial guess on entry.  Synchronous (fills stats).
 * Returns EB_ERR_NO_CONVERGENCE after maxit iterations. */
int pcg_solve(const amg_handle* amg, const double* b_dev, double* x_dev, double rtol, int maxit,
              const pcg_opts* opts, pcg_stats* stats, cudaStream_t stream);

/* Solves (sigma I + A) x = b for any real sigma by preconditioned MINRES:
 * the Helmholtz problem omega^2 u + Lap u = f of Sec. 3.3.2 is sigma =
 * -omega^2 with b from eb_rhs (indefinite; the paper solves it by MINRES).
 * precond: EB_PC_AMG (amg's V-cycle, built for amg's own shift, which must be
 * positive definite -- e.g. shift 0: the Laplacian), EB_PC_JACOBI or
 * EB_PC_NONE.  Stops when the preconditioned residual norm (the M^-1 norm
 * MINRES minimises) falls to rtol times its initial value; stats report the
 * iterations, that ratio (rel_residual) and the true ||b - (sigma I + A) x|| /
 * ||b|| (true_rel_residual).  x holds the initial guess on entry.  Allocates
 * its work vectors for the call.  EB_ERR_BREAKDOWN if the preconditioner is
 * not positive definite, EB_ERR_NO_CONVERGENCE after maxit.  Synchronous. */
int minres_solve(const amg_handle* amg, double sigma, int precond, const double* b_dev, double* x_dev, double rtol,
                 int maxit, pcg_stats* stats, cudaStream_t stream);

/* One theta-method step of u_t = L u + F (Sec. 3.4 uses theta = 1/2; theta = 1
 * is backward Euler): (I/dt + theta A) u1 = (I/dt - (1-theta) A) u0 + theta
 * b1 + (1-theta) b0, where b = eb_rhs(-F, u_Gamma) at the two times.  amg
 * must have been set up with shift = 1/(theta dt).  u is overwritten with u1
 * (warm start from u0).  b0 may be NULL when theta = 1. */
int heat_step(const amg_handle* amg, double dt, double theta, const double* b1_dev, const double* b0_dev,
              double* u_dev, double rtol, int maxit, pcg_stats* stats, cudaStream_t stream);

/* nsteps of the implicit theta-scheme of Sec. 3.5 for u_tt = div(beta grad u)
 * with homogeneous Dirichlet data, theta > 0 (theta = 1/2, 1/4: second-order
 * unconditionally stable; theta = 1/12: fourth order in time), the printed
 * scheme read with the Laplacian on its (1 - 2 theta) term:
 *   (I + theta dt^2 A) u^{n+1} = 2 u^n - (1 - 2 theta) dt^2 A u^n - u^{n-1}
 *                                - theta dt^2 A u^{n-1}.
 * Each step solves (sigma I + A) u^{n+1} = sigma (2 u^n - u^{n-1}) - ((1 -
 * 2 theta)/theta) A u^n - A u^{n-1} by PCG with amg's preconditioner from the
 * guess 2 u^n - u^{n-1}; amg must have been set up with shift sigma = 1 /
 * (theta dt^2).  On entry (u_prev, u_cur) = (u^{n-1}, u^n) (FP64 device
 * fields), on exit (u^{n+nsteps-1}, u^{n+nsteps}).  stats (may be NULL):
 * iterations summed over the steps, the largest residuals, converged = all
 * steps converged.  Returns the first failing step's status (the fields then
 * hold a partial run).  Synchronous. */
int wave_theta_step(const amg_handle* amg, double dt, double theta, double* u_prev_dev, double* u_cur_dev,
                    int nsteps, double rtol, int maxit, pcg_stats* stats, cudaStream_t stream);

/* nsteps of the explicit leapfrog scheme (the theta-scheme of Sec. 3.5 with
 * theta = 0): u^{n+1} = 2 u^n - u^{n-1} - dt^2 A u^n (homogeneous Dirichlet
 * data).  On entry (u_prev, u_cur) = (u^{n-1}, u^n); on exit they hold
 * (u^{n+nsteps-1}, u^{n+nsteps}).  One kernel launch per step; whole chunks of
 * 32 steps run as one launch of a CUDA graph that the handle caches for these
 * fields, prec, dt and tile list (built on first use, which allocates).
 * prec: EB_F64 or EB_F32 element type of both fields.  Asynchronous on
 * stream; the fields must not be touched by other work until it completes. */
int wave_step(const eb_handle* eb, int prec, double dt, void* u_prev_dev, void* u_cur_dev, int nsteps,
              cudaStream_t stream);

/* ---------------------------------------------------------------- batches
 * Many 2D geometries of uneven size advanced together: one launch per PCG
 * phase over the active tiles of all of them, per-geometry CG recurrences and
 * convergence, one AMG hierarchy on the block-diagonal operator.  Used for
 * batches of implicit heat steps (Sec. 3.4) on different domains.
 *
 * Batch layout of every batch vector: geometry g's full grid (n0_g x n1_g
 * nodes, x fastest) at node offset node_off[g], rows of common stride S
 * (batch_info.stride): node (i, j) of g is node_off[g] + j S + i.  Cut values
 * (u_Gamma) are concatenated geometry by geometry (cut_off[g]), each in the
 * eb_cuts order of that geometry.  Entries outside the CPs are ignored on
 * input; outputs follow the active-tile rule of the single-grid calls. */
typedef struct batch_handle batch_handle;

typedef struct {
  int count;
  int64_t stride;        /* S, the common row stride */
  int64_t num_nodes;     /* total nodes of the batch layout */
  int64_t num_cp;
  int64_t num_cut;
  int64_t num_tiles;
} batch_info_t;

/* Builds every geometry (eb_build semantics, 2D only) and the batch layout.
 * grids / lss: host arrays of count entries.  Synchronous. */
int batch_build(const eb_grid* grids, const eb_levelset* lss, int count, batch_handle** out, cudaStream_t stream);
void batch_destroy(batch_handle* b);
int batch_info(const batch_handle* b, batch_info_t* out);
/* Host arrays of count + 1 entries each (any may be NULL): node, cut and CP
 * offsets of the geometries in the batch layout. */
int batch_offsets(const batch_handle* b, int64_t* node_off, int64_t* cut_off, int64_t* cp_off);
/* The batch's own handle of geometry g (owned by the batch; valid until
 * batch_destroy), for eb_cuts / eb_classes / eb_apply on that grid alone. */
const eb_handle* batch_geometry(const batch_handle* b, int g);
/* eb_rhs for every geometry, in the batch layout. */
int batch_rhs(const batch_handle* b, const double* f_all, const double* ug_all, double* b_all, cudaStream_t stream);
/* Fixes the time steps dt[g] (host array) and theta of the theta-method and
 * builds the AMG hierarchy of the batch.  dt[g] = +INFINITY (with theta = 1)
 * drops the time derivative: batch_heat_step then solves the steady problem
 * A u = b1 of every such geometry (a batch of Poisson solves, e.g. a sweep of
 * a geometry parameter as in Sec. 3.6).  Synchronous. */
int batch_heat_setup(batch_handle* b, const double* dt, double theta, const amg_opts* opts, cudaStream_t stream);
/* Tile-shape autotuner for a batch (after batch_heat_setup): retiles every
 * geometry and the batch with each candidate 2D shape, times `reps` V-cycles
 * of the batch hierarchy, keeps the fastest.  Synchronous. */
int batch_autotune(batch_handle* b, int reps, eb_tune_t* out, cudaStream_t stream);
/* Quantities of interest of a batch (Sec. 3.6): out_dev[g] = sum over the
 * nodes of geometry g of w u (w_all, u_all: batch vectors; out_dev: count
 * doubles on the device), each sum in a fixed order (deterministic).  With w
 * the interpolation weights of a point, this is u at that point; with h^2 on
 * the nodes of a region, the integral of u over it.  Synchronous. */
int batch_weighted_sum(const batch_handle* b, const double* w_all, const double* u_all, double* out_dev,
                       cudaStream_t stream);
/* on != 0: later batch_heat_step calls time every level-0 smoother launch of
 * their captured PCG iterations with CUDA events and report the summed
 * duration and the launch count in prof_kernel_ms / prof_launches of every
 * geometry's stats (batch totals). */
int batch_set_profile(batch_handle* b, int on);
/* prec EB_DF64: later batch_heat_step calls run the outer PCG of every
 * geometry in double-float (pcg_opts.outer_prec semantics: x, r, p, q as FP32
 * pairs, the FP32 V-cycle output z, DF per-tile partials, FP64 scalars; each
 * geometry's b and x cross into DF scaled by its own power of two; the exit
 * test stays the FP64 true residual).  Needs a batch_heat_setup with an FP32
 * or BF16 V-cycle of two or more levels (EB_ERR_NOT_IMPLEMENTED from the step
 * otherwise).  EB_F64 (the default) restores the FP64 iteration.
 * EB_ERR_INVALID for other values. */
int batch_set_outer_prec(batch_handle* b, int prec);
/* on != 0 (the default): the level-0 Chebyshev steps of the batched V-cycle
 * (FP32 storage, tiles 16 to 128 nodes wide, batch row stride a multiple of 16
 * nodes) stage each tile's x box with its halo, b, d and codes in shared
 * memory through tensor copies (cp.async.bulk.tensor, a 4-stage ring) instead
 * of loading them per thread; the results are the same bit for bit.  on = 0
 * keeps the per-thread kernel (instrumentation: the paper has no
 * counterpart).  A step whose bounded waits give up makes the next
 * batch_heat_step return EB_ERR_TIMEOUT. */
int batch_set_level0_tma(batch_handle* b, int on);
/* One theta-method step of every geometry (heat_step semantics, warm start
 * from u), u overwritten.  stats: host array of count entries (may be NULL).
 * Returns EB_ERR_NO_CONVERGENCE if any geometry missed rtol.  Synchronous. */
int batch_heat_step(batch_handle* b, const double* b1_all, const double* b0_all, double* u_all, double rtol,
                    int maxit, pcg_stats* stats, cudaStream_t stream);

/* ------------------------------------------------------------ learned stage
 * A small convolutional network N on the 2D Cartesian grid used as an extra
 * stage of the preconditioner.  The paper has no learned component: this is
 * an extension of its AMG-PCG (Algorithm 1 step 4).
 *
 * N(s_hat, m): six zero-padded 3x3 cross-correlations, 2 -> 32 -> 32 -> 32 ->
 * 32 -> 32 -> 1 channels, ReLU after the first five; the output is multiplied
 * by the mask channel m (1 at the CPs, 0 elsewhere).  Tap d = 3 (dy+1) +
 * (dx+1) reads the pixel (row + dy, column + dx); x is the column.
 * Parameters: one float vector of nn_num_params() = 37889 entries,
 *   W1 [32][9][2], b1 [32], 4 x (W [32][9][32], b [32]), W6 [9][32], b6 [1]
 * (W[co][d][ci]).  Hidden activations are stored in bfloat16 (NHWC, 64 bytes
 * per pixel) and the four 32 -> 32 layers run on the tensor cores (tcgen05,
 * accumulators in tensor memory) with bf16 weights; every sum is accumulated
 * in float.
 *
 * Images: "images" images of height x width pixels, stored one after the
 * other, row-major (x fastest); each image is zero-padded separately.
 *
 * Training pairs (nn_pairs) come from the solver itself: for a right-hand side
 * b with solution x*, x_0 = 0, x_k = x_{k-1} + V(b - A x_{k-1}) (V: the
 * handle's V-cycle), e_k = x* - x_k, t_k = h^2 A e_k, rho_k = rms of t_k over
 * the CPs, s_hat_k = t_k / rho_k, e_hat_k = e_k / rho_k, c_k = e_hat_k' s_hat_k.
 * Loss of an output o on pair k: (o'A~o - 2 o's_hat_k + c_k) / c_k =
 * ||o - e_hat_k||^2 / ||e_hat_k||^2 in the energy norm of A~ = h^2 A.
 * Stage in the flexible PCG: z1 = V(r), s = r - A z1,
 * z = z1 + h^2 rms(s) N(s / rms(s), m).
 */
typedef struct nn_handle nn_handle;

/* A network with all parameters 0 (set them with nn_set_params).  Synchronous. */
int nn_create(nn_handle** out, cudaStream_t stream);
void nn_destroy(nn_handle* nn);
int nn_num_params(void);
/* The 32 -> 32 layers run on the tensor cores (tcgen05); a wait for them that
 * gives up (bounded) marks the handle.  nn_status reads and clears the mark:
 * EB_ERR_TIMEOUT if any convolution since the last check gave up (its
 * results are invalid), else EB_OK.  nn_get_params and pcg_solve_nn check it
 * themselves.  Synchronous. */
int nn_status(nn_handle* nn, cudaStream_t stream);
/* on != 0: later nn_forward / nn_backward / nn_train_step calls time every
 * 32 -> 32 convolution launch of their forward passes with CUDA events;
 * nn_profile returns (synchronously) the summed milliseconds and the number
 * of timed launches since, and restarts the count. */
int nn_set_profile(nn_handle* nn, int on);
int nn_profile(nn_handle* nn, double* ms, int* launches, cudaStream_t stream);
/* Forward path of nn_forward and of the learned stage in pcg_solve_nn /
 * nn_precondition.  on != 0 (the default): one launch computes all six layers
 * with the hidden activations kept in shared memory and tensor memory (strips
 * of 116 columns walked down the rows); on = 0: one launch per layer through
 * activation buffers in device memory, the path nn_backward and nn_train_step
 * always take.  Both give bit-identical outputs.  With profiling on, the fused
 * launch is the one timed launch of a forward.  Set it before a solve: a
 * solver's captured iteration keeps the path it was captured with. */
int nn_set_fused(nn_handle* nn, int on);
/* Copies nn_num_params() floats from HOST memory into the network and resets
 * the Adam state (moments and step count).  Synchronous. */
int nn_set_params(nn_handle* nn, const float* params_host, cudaStream_t stream);
/* Copies the parameters and / or the gradient of the last nn_backward or
 * nn_train_step to HOST memory (either pointer may be NULL).  Synchronous. */
int nn_get_params(const nn_handle* nn, float* params_host, float* grad_host, cudaStream_t stream);
/* out = N(in): in is [images][height][width][2] floats (s_hat, m), out is
 * [images][height][width] floats, both device buffers (in 8-byte aligned).
 * width, height >= 1.  Activation memory (layer-by-layer path only, see
 * nn_set_fused) is held by the handle and grows to the largest images x
 * height x width seen (64 bytes x 7 per pixel). */
int nn_forward(nn_handle* nn, int width, int height, int images, const float* in_dev, float* out_dev,
               cudaStream_t stream);
/* Gradient of sum(dout * N(in)) in the parameters (kept in the handle, read
 * with nn_get_params).  Runs the forward pass itself; dout has the layout of
 * nn_forward's out. */
int nn_backward(nn_handle* nn, int width, int height, int images, const float* in_dev, const float* dout_dev,
                cudaStream_t stream);
/* The first `count` training pairs of the V-cycle iteration of amg (above)
 * for b and x* (full-grid device vectors): s_hat into s_hat_dev[count][num_nodes]
 * (float), c_k into c_dev[count] (double), e_hat into e_hat_dev[count][num_nodes]
 * (double; may be NULL).  Entries off the CPs are 0. */
int nn_pairs(const amg_handle* amg, const double* b_dev, const double* xstar_dev, int count, float* s_hat_dev,
             double* c_dev, double* e_hat_dev, cudaStream_t stream);
/* The geometry a training image needs: the eb_classes byte of every node and
 * the diagonal D_k as float (0 off the CPs), into num_nodes-entry buffers. */
int nn_geometry(const eb_handle* eb, uint8_t* code_dev, float* diag_dev, cudaStream_t stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the mean
 * loss of `batch` pairs.  Pair j of the batch is pair pick[j] of a store:
 * s_hat[pick[j]] (float, height x width), c[pick[j]] (double), on the
 * geometry geo_of[pick[j]] of code[][height x width] / diag[][height x width]
 * (nn_geometry).  pick and geo_of are device int32 arrays; the caller keeps
 * every index in range.  loss_dev (may be NULL): device floats, batch + 1
 * entries, the loss of every pair before the step and their mean last. */
int nn_train_step(nn_handle* nn, int width, int height, int batch, const float* s_hat_dev, const double* c_dev,
                  const int32_t* geo_of_dev, const uint8_t* code_dev, const float* diag_dev, const int32_t* pick_dev,
                  float lr, float* loss_dev, cudaStream_t stream);
/* Step length of the stage: EB_NN_PLAIN uses z1 + h^2 rms(s) N (as above);
 * EB_NN_ENERGY multiplies the correction by omega = (o's_hat) / (o'A~o),
 * o = N(s_hat, m), A~ = h^2 (shift I + A): the step along o that minimises the
 * energy norm of the error left after z1, so that the stage never increases
 * it (omega = 1 for a network returning A~^-1 s_hat exactly; omega = 0 when
 * o'A~o <= 0). */
typedef enum { EB_NN_PLAIN = 0, EB_NN_ENERGY = 1 } eb_nn_mode;
/* One application of the preconditioner with the stage: z = V(r) followed by
 * the stage of the given mode (full-grid device vectors, r != z). */
int nn_precondition(const amg_handle* amg, nn_handle* nn, int mode, const double* r_dev, double* z_dev,
                    cudaStream_t stream);
/* pcg_solve with the preconditioner V-cycle + learned stage (above), flexible
 * (Polak-Ribiere) beta.  2D grids; amg must hold a hierarchy.  opts->precond
 * is ignored. */
int pcg_solve_nn(const amg_handle* amg, nn_handle* nn, int mode, const double* b_dev, double* x_dev, double rtol,
                 int maxit, const pcg_opts* opts, pcg_stats* stats, cudaStream_t stream);

/* The leapfrog steps of wave_step for callers that must not allocate during
 * the call.  The paper has no counterpart: this is a service of this library.
 * wave_step builds and caches a CUDA graph on its first call for a set of
 * fields, which allocates; loops with a fixed memory budget that must not
 * touch the allocator after start-up, programs whose device memory is held by
 * another framework's pool, and time-critical loops that cannot afford the
 * device synchronisation of cudaMalloc / cudaFree cannot allow that.  This
 * entry point runs all nsteps in one persistent cooperative launch and keeps
 * the scratch of its grid-wide barrier in a fixed device array of the library
 * (one flag per cooperative CTA, at most 2048 CTAs -- larger grids are capped
 * at 2048, which limits parallelism, not the result -- about 8 KB, held by
 * every GPU that loads the library until the process exits); it calls no cudaMalloc,
 * cudaFree or allocating library routine.  Same arguments, arithmetic and
 * results as wave_step; the handle and the fields are created by the caller
 * beforehand.  The first call on each device looks up the array's device
 * address (no allocation); make that first call before any stream capture.
 * All calls share the array and each clears the part it uses before its
 * launch, so two calls whose kernels overlap on the GPU race and must not be
 * issued.  A barrier wait that gives up returns EB_ERR_TIMEOUT.
 * Synchronous. */
int wave_step_noalloc(const eb_handle* eb, int prec, double dt, void* u_prev_dev, void* u_cur_dev, int nsteps,
                      cudaStream_t stream);

const char* eb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EB_H_ */
