/* fhmg -- multigrid waveform relaxation with an H-matrix time operator for the
 * time-fractional heat equation, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Hu, Rodrigo & Gaspar, "Using hierarchical matrices in the solution of the
 * time-fractional heat equation by multigrid waveform relaxation" (arXiv 1706.07632).
 *
 * The discrete problem (Section 2, Eqs. discrete_model_IVP_1-3) couples M time levels
 * t_m = T (m/M)^gamma (m = 1..M) and N^dim interior spatial points (dim = 1 or 2, grid size
 * h = Lx/(N+1), homogeneous Dirichlet boundaries):
 *
 *     sum_{j<=m} R_{m,j} u_{.,j} + A_h u_{.,m} = f_{.,m} + d_{m,m} g,
 *
 * R the Petrov-Galerkin L1 matrix of the Caputo derivative of order alpha (Eq.
 * elements_matrix_R), A_h the 3-point / 5-point negative Laplacian, g the initial data.
 *
 * Conventions shared by every entry point:
 *  - Grid functions (u, f, residuals, corrections) are caller-owned DEVICE arrays of doubles,
 *    time-major with space contiguous: element (m, p) at m * N^dim + p, m = 0..M-1 for t_1..t_M,
 *    p = n - 1 (1D) or p = iy * N + ix (2D).  g is a device array of N^dim doubles or NULL (= 0).
 *  - Every call is ordered on the problem's stream and returns before the GPU work ends unless
 *    it returns a host value (norms, cycle counts), in which case it synchronises the stream.
 *  - Every function returns an fhmg_status and never aborts; arguments are validated on the
 *    host.  Outputs are written only on FHMG_OK, except u after a solve that did not reach
 *    rtol, which holds the last iterate.  The library never frees caller memory.
 *  - fhmg_last_error() returns a message for the last failure of the calling thread.
 *  - A problem lives on the CUDA device that was current when it was created; every call on it
 *    makes that device current for its duration and restores the caller's device afterwards.
 *  - Every device-side wait of the walk kernels is bounded.  A walk whose wait gives up leaves
 *    early and sets the problem's error word; the next call that returns a host value (a norm, a
 *    solve) reports it as FHMG_ETIMEOUT and clears it, so the problem stays usable.
 */
#ifndef FHMG_H_
#define FHMG_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fhmg_hmatrix_s* fhmg_hmatrix; /* opaque; host-side H-matrix, library-owned */
typedef struct fhmg_problem_s* fhmg_problem; /* opaque; device data + workspaces, library-owned */

enum fhmg_status {
  FHMG_OK = 0,
  FHMG_EINVAL = -1,   /* invalid argument (message in fhmg_last_error) */
  FHMG_ECUDA = -2,    /* a CUDA call failed */
  FHMG_ENOMEM = -3,   /* device or host allocation failed */
  FHMG_ENOTCONV = -4, /* solve stopped at max_cycles above rtol (u holds the last iterate) */
  FHMG_ENAN = -5,     /* a residual norm was NaN or Inf */
  FHMG_ETIMEOUT = -6  /* a bounded device wait gave up */
};

enum fhmg_prec {
  FHMG_FP64 = 0,       /* every product in FP64 */
  FHMG_MIXED_FP32 = 1, /* defect correction: FP64 residual, FP32 inner V-cycles */
  FHMG_MIXED_BF16 = 2  /* as FHMG_MIXED_FP32, but the inner cycles' FP32-storage walks over panels wide
                          enough for a 128-column tile per SM run BF16 H-matrix products with FP32
                          accumulation on the tcgen05 tensor cores (leaf 64; narrower walks and the
                          FP64-storage levels keep the FP32 products) */
};

const char* fhmg_last_error(void);

/* Builds the time operator (host, one-time).  Section 2: mesh t_m = T (m/M)^gamma and the
 * L1 matrix R; Section 3: its H-matrix form (index bisection, Definition 3.1 admissibility,
 * Taylor degenerate kernel Eqs. A_elements / B_elements).
 *   alpha in (0,1): fractional order (the paper's delta); gamma >= 1: grading exponent (the
 *   paper's r); T > 0: final time; M: time steps, M = leaf * 2^p; leaf in {16, 32, 64}
 *   (leaf > M means one leaf of size M);
 *   rank > 0: k Taylor terms per admissible block, no recompression (the paper's form);
 *   rank == 0 and tol > 0: Taylor terms from the Theorem 3.1 bound, then each block
 *     recompressed (QR + SVD) to singular values > tol * (largest of the block);
 *   rank == 0 and tol == 0: dense lower-triangular R (no low-rank blocks).
 * On success *out owns host memory released by fhmg_hmatrix_destroy. */
int fhmg_build_hmatrix(double alpha, double gamma, double T, int M, int leaf, int rank, double tol,
                       fhmg_hmatrix* out);
/* The same H-matrix with its low-rank blocks built algebraically (the construction Section 6 names
 * for kernels without a separable expansion): each admissible block by adaptive cross approximation
 * with partial pivoting from single accurate entries R_{m,j} (pivot row -> its largest residual
 * entry's column -> the next pivot row at the column's largest unused residual entry), stopped at
 * |u_k| |v_k| <= 0.01 tol |sum u_l v_l^T|_F, then recompressed (QR + SVD) to singular values
 * > tol * (largest of the block) like the Taylor form.  tol > 0; the other arguments as above. */
int fhmg_build_hmatrix_aca(double alpha, double gamma, double T, int M, int leaf, double tol, fhmg_hmatrix* out);
/* Block counts, largest rank and bytes of the FP64 device representation. Any pointer may be NULL. */
int fhmg_hmatrix_info(fhmg_hmatrix h, int* n_dense, int* n_lowrank, int* max_rank, size_t* bytes);
/* Copies the mesh t_0..t_M (M+1 host doubles) and the initial-data weights d_{m,m} (M host
 * doubles); either pointer may be NULL. */
int fhmg_hmatrix_mesh(fhmg_hmatrix h, double* t_out, double* dmm_out);
/* Writes the approximated matrix R~ densely (M*M host doubles, row-major, upper part zero). */
int fhmg_hmatrix_dense(fhmg_hmatrix h, double* R_out);
/* Algorithmic FP64 flops of one H-matvec (Algorithm 3) or line solve (Algorithm 4) per column. */
int fhmg_hmatrix_flops(fhmg_hmatrix h, double* flops_per_column);
/* Host only: the digit tiles of R~ that the outer defect of defect arithmetic 2 multiplies
 * (fhmg_problem_set_defect_arith), for inspection and tests.  Needs M a multiple of 128 and
 * M <= 512 (else EINVAL).  Row m of the dense R~ (fhmg_hmatrix_dense) is rounded to the integers
 * X_mk = round(R~_mk 2^{49 - E_m}), E_m the binary exponent of max_k |R~_mk| (frexp: 2^{E_m - 1} <=
 * max < 2^{E_m}; 0 for a zero row), and written as X_mk = sum_{a=0..6} d_a 2^{7 (6 - a)} with
 * balanced digits: d_1..d_6 in [-64, 63], |d_0| <= 129.  Blocks (I, J) of 128 time rows x 64 time
 * levels, I = 0..M/128-1, J = 0..2I+1 (the blocks that meet the lower triangle), in I-major order;
 * for each the digit tiles with a nonzero entry, in digit order, each 128 x 64 BF16 values (8192
 * uint16 bit patterns, exact small integers) in the tensor cores' K-major 128-byte-swizzled
 * layout: entry (r, k) at uint16 index (r/8)*512 + (r%8)*64 + (((k/8) ^ (r%8)) & 7)*8 + k%8.
 * tiles: NULL to query the tile count into *n_tiles; otherwise a host buffer of *n_tiles * 8192
 * values (*n_tiles on entry is its capacity in tiles, EINVAL if too small; on return the count
 * written).  pairs: 4 ints per block {digit mask, index of its first tile, 0, 0}, M/128 (M/128 + 1)
 * blocks (may be NULL); rexp: the M exponents E_m (may be NULL).  Caller-owned host memory. */
int fhmg_hmatrix_split_digits(fhmg_hmatrix h, unsigned short* tiles, long long* n_tiles, int* pairs, int* rexp);
int fhmg_hmatrix_destroy(fhmg_hmatrix h);
/* Two-grid convergence factor predicted by mode analysis (Section 5, the SAMA column of Table 2):
 * sine modes in space (a mode and its partner N+1-k per dimension: 2x2 groups in 1D, 4x4 in 2D),
 * the time matrix exactly -- on each group every time block is a rational function of the
 * lower-triangular time matrix, so the two-grid operator's eigenvalues are those of the group
 * matrices at the diagonal entries R_mm.  Two-grid cycle with nu1 pre- and nu2 post-smoothing
 * red-black sweeps (nu1 + nu2 >= 1), full weighting, (bi)linear interpolation, exact coarse solve, on
 * the dim-D grid of N = 2^k - 1 >= 3 points per dimension of (0, Lx).  Host computation; *rho_out
 * receives the largest spectral radius over the paired modes k (and l) = 1..(N-1)/2 and all m. */
int fhmg_sama_two_grid(fhmg_hmatrix h, int dim, int N, double Lx, int nu1, int nu2, double* rho_out);

/* Creates a problem on the current CUDA device: dim in {1,2}; N = 2^levels - 1 interior points
 * per dimension (levels >= 1); Lx > 0 domain length; prec an fhmg_prec; stream a cudaStream_t
 * (NULL = legacy default stream).  Uploads the H-matrix, builds the per-level inverted diagonal
 * leaves (D_ii + s_l I)^{-1}, s_l = 2/h_l^2 (1D) or 4/h_l^2 (2D), and allocates workspaces.
 * The problem keeps a reference to h; destroy the problem before h. */
int fhmg_problem_create(fhmg_hmatrix h, int dim, int N, double Lx, int prec, void* stream,
                        fhmg_problem* out);
int fhmg_problem_destroy(fhmg_problem p);
/* Chooses the column tile of each kernel by timing (autotuner); optional. */
int fhmg_problem_autotune(fhmg_problem p);
/* Mixed path: V-cycles run on the correction equation between two FP64 defect evaluations
 * (>= 1; 0 restores the default: 2 with FP32 storage, 4 with FP64 storage).  After the first round
 * a round runs fewer cycles where the previous round's contraction per cycle predicts that fewer
 * reach rtol with a factor 2 to spare (so the last round runs no cycle the target does not need). */
int fhmg_problem_set_inner(fhmg_problem p, int inner_cycles);
/* Mixed path, storage of the inner cycles: 0 automatic, per level: FP32 on every level whose
 * stencil conditioning allows it (6e-8 * 4 (N+1)^2 / pi^2 <= 0.05, i.e. N <= 1023), FP64 grid
 * functions / stencil / diagonal with FP32 H-matrix products on the finer ones (a coarse-grid
 * correction below them then runs in FP32 storage); 1 FP64 storage with FP32 products on every
 * level; 2 FP32 throughout.  The outer defect and the update of u are FP64 in every mode. */
int fhmg_problem_set_mixed_storage(fhmg_problem p, int mode);
/* Resets the counters below and, if enable != 0, records CUDA events on the problem's stream
 * around every smoother launch on the finest grid and every FP64 defect product on the finest
 * grid (the stopping test's and the mixed path's outer defects). */
int fhmg_problem_profile(fhmg_problem p, int enable);
/* Synchronises the stream and reports, since the last fhmg_problem_profile: the number of
 * kernel launches issued, the number of finest-grid smoother launches timed and their summed
 * device time in milliseconds.  Any pointer may be NULL. */
int fhmg_problem_counters(fhmg_problem p, long long* launches, long long* smooth_launches, double* smooth_ms);
/* Synchronises the stream and reports, since the last fhmg_problem_profile: the number of
 * finest-grid FP64 defect products timed, their summed device time in milliseconds, and the
 * finest grid's point count (a full defect walks that many columns; the stopping test of the
 * FP64 path walks the first colour only).  Any pointer may be NULL. */
int fhmg_problem_defect_timing(fhmg_problem p, long long* defect_launches, double* defect_ms, long long* columns);

/* --- the hot-path steps, exposed one by one (each is one or more kernel launches) --- */

/* Algorithm 4 over many columns: X = (R~ + s_level I)^{-1} B; X, B device [M][ncols]
 * (time-major, column-contiguous); level 0..levels-1 selects the shift (level levels-1 is the
 * finest grid).  X may alias B. */
int fhmg_line_solve(fhmg_problem p, int level, double* X, const double* B, long long ncols);
/* Algorithm 3 over many columns: Y = R~ X; device [M][ncols]; Y must not alias X. */
int fhmg_hmatvec(fhmg_problem p, double* Y, const double* X, long long ncols);
/* The same two steps with the mixed path's FP32 products (mixed-precision problems only; EINVAL
 * otherwise): H-matrix entries and x tiles in FP32, accumulation in FP32 per leaf, the diagonal
 * of the diagonal leaves (and of the level inverses) applied in FP64, FP64 arrays in and out.
 * tile: 0 automatic, else the column tile (1, 2, 4, ..., 32); with leaf 64 and tensor cores
 * enabled (fhmg_problem_set_tensor_cores) tiles 16 and 32 run on the tensor cores. */
int fhmg_line_solve_f32(fhmg_problem p, int level, double* X, const double* B, long long ncols, int tile);
int fhmg_hmatvec_f32(fhmg_problem p, double* Y, const double* X, long long ncols, int tile);
/* The FP32-storage walks of the mixed path's inner cycles on FP32 device arrays [M][ncols]
 * (mixed-precision problems only): X = (R~ + s_level I)^{-1} B (Algorithm 4; X may alias B) and
 * Y = R~ X (Algorithm 3; Y must not alias X).  FHMG_MIXED_BF16 problems run them on the tcgen05 walk
 * when ncols >= 128 x the SM count: BF16 products (H-matrix entries, x, y and z operands rounded to
 * BF16) with FP32 accumulation; the diagonal of the diagonal leaves (and of the level inverses) is
 * applied in FP32.  Otherwise FP32 products (3xTF32 tensor cores or SIMT). */
int fhmg_line_solve_s(fhmg_problem p, int level, float* X, const float* B, long long ncols);
int fhmg_hmatvec_s(fhmg_problem p, float* Y, const float* X, long long ncols);
/* Y = R~ X with the double-float products of fhmg_problem_set_defect_arith (mixed-precision
 * problems only; EINVAL otherwise); device [M][ncols] FP64; tile 0 (automatic), 4, 8 or 16. */
int fhmg_hmatvec_df(fhmg_problem p, double* Y, const double* X, long long ncols, int tile);
/* nsweeps red-black zebra-in-time sweeps (Section 4) on the finest grid: u updated in place,
 * F the full right-hand side (f + d_{m,m} g). */
int fhmg_smooth(fhmg_problem p, double* u, const double* F, int nsweeps);
/* Defect r = f + d_{m,m} g - (R~ (x) I) u - (I (x) A_h) u on the finest grid, all points. */
int fhmg_residual(fhmg_problem p, const double* u, const double* f, const double* g, double* r_out);
/* Full-weighting restriction of the defect to the next coarser grid (Algorithm 2), computed as
 * FW(F - A_h u) - R~ FW(u); rc_out is device [M][Nc^dim], Nc = (N-1)/2. */
int fhmg_restrict_residual(fhmg_problem p, const double* u, const double* F, double* rc_out);
/* u += I_{2h}^h e (linear / bilinear interpolation in space, Algorithm 2); e is [M][Nc^dim]. */
int fhmg_prolong_correct(fhmg_problem p, double* u, const double* e);

/* One V(nu1, nu2) cycle of Algorithm 2 on u (in place). */
int fhmg_vcycle(fhmg_problem p, double* u, const double* f, const double* g, int nu1, int nu2);
/* ||f + d g - A_{h,tau} u||_inf into *out_max (host). */
int fhmg_residual_norm(fhmg_problem p, const double* u, const double* f, const double* g,
                       double* out_max);
/* The same max-norm for callers that cannot allocate device memory once their loop runs (a fixed
 * budget reserved up front, a real-time loop, a host framework that owns every allocation).  The
 * paper has no counterpart: this is a library service.  It allocates nothing: its scratch is a
 * fixed library-owned device array of 2^21 doubles (16 MiB, held on every GPU that loads the
 * library until the process exits), so M * N^dim must be <= 2^21 (else FHMG_EINVAL).  f is the
 * full right-hand side (fold any initial data into it: there is no g).  The products follow the
 * problem's defect arithmetic (fhmg_problem_set_defect_arith), as in fhmg_residual_norm.  The first
 * call for a problem on a given device looks the array's address up on that device -- make it
 * before any stream capture; after cudaDeviceReset on that device the address is stale and the
 * entry point must not be used there again in the process.  All calls share the array: calls whose
 * GPU work overlaps race and must be serialised by the caller. */
int fhmg_residual_norm_noalloc(fhmg_problem p, const double* u, const double* f, double* out_max);
/* V(nu1, nu2) cycles from the initial guess in u until ||r_k||_inf <= rtol ||r_0||_inf or
 * max_cycles.  cycles_out / relres_out (host, may be NULL) receive the cycle count and
 * ||r_k||/||r_0||.  With prec FHMG_MIXED_FP32 the cycles run in FP32 on the correction
 * equation and the defect is recomputed in FP64 after each inner stage (defect correction);
 * *cycles_out then counts inner cycles. */
int fhmg_solve(fhmg_problem p, double* u, const double* f, const double* g, int nu1, int nu2,
               double rtol, int max_cycles, int* cycles_out, double* relres_out);
/* Solves n independent problems together (1 <= n <= 4096; each with its own H-matrix, alpha,
 * gamma, M, N; all FHMG_FP64 or all FHMG_MIXED_FP32).  Their V-cycles advance in lockstep by
 * depth below each finest grid: every smoother colour, every coarse-grid product and every
 * defect of all instances is ONE persistent panel-kernel launch (one per leaf size present);
 * one cycle of all active instances is captured into a CUDA graph and replayed.  Mixed: defect
 * correction with FP32 H-matrix products (FP64 grid functions) and FP64 defects.  u[i], f[i]
 * device arrays of problem i; cycles_out / relres_out (n host entries each, may be NULL).
 * Runs on an internal stream ordered after, and before, every problem's stream. */
int fhmg_solve_batched(int n, fhmg_problem* probs, double** u, const double** f, int nu1, int nu2,
                       double rtol, int max_cycles, int* cycles_out, double* relres_out);
/* Autotuner for the leaf size: builds the H-matrix with leaf 16, 32 and 64 (those <= M), autotunes
 * the column tiles of each, times one V-cycle, and returns the fastest leaf (and its cycle time in
 * ms).  (The tensor-core walks need leaf 64; smaller leaves trade them for fewer near-field entries.) */
int fhmg_autotune_leaf(double alpha, double gamma, double T, int M, double tol, int dim, int N, double Lx,
                       int prec, void* stream, int* best_leaf, double* best_ms);
/* Host only: the H-matrix form for (alpha, gamma, T, M, leaf) with the fewest H-matvec flops per
 * column (Algorithm 3; the FP64 walks run FP64-pipe-bound, so their time follows these flops) whose
 * row-relative error max_m max_j |R~_mj - R_mj| / max_j |R_mj| against the exact R (every entry,
 * Section 2) is at most err_target.  Candidates: the paper's Taylor factors with k = 4, 6, 8, 10,
 * 12, 16, 20 terms (Section 3), Taylor factors recompressed to tol = 1e-6 .. 1e-14, and R itself
 * (rank 0, tol 0: always admissible).  Writes the choice as the (rank, tol) arguments of
 * fhmg_build_hmatrix, and its error and flops per column (either of those two may be NULL).
 * EINVAL for invalid arguments or err_target < 0.  Builds every candidate on the host (seconds at
 * M = 4096). */
int fhmg_autotune_hmatrix(double alpha, double gamma, double T, int M, int leaf, double err_target, int* best_rank,
                          double* best_tol, double* best_err, double* best_flops);
/* Stopping reference of fhmg_solve: 0 (default) ||r_k|| <= rtol ||r_0|| (the paper's test, §5);
 * 1 ||r_k|| <= rtol max|F| -- the same absolute target whatever the initial guess, used to compare
 * a warm start with the zero initial guess fairly. */
int fhmg_problem_set_rtol_reference(fhmg_problem p, int ref);

/* Arithmetic of the mixed path's FP64-accurate steps -- the outer defect (the residual that decides
 * convergence) and the mode solves of the exactly solved coarse level
 * (fhmg_problem_set_coarse_direct).  0: FP64 (DFMA) products.  1: double-float -- pairs of floats
 * with error-free transformations on the FP32 pipe (entries and x split as a = hi + lo,
 * |a - hi - lo| <= 2^-48 |a|; each dot product accurate to a few 2^-48 of sum |a_k x_k|), which on
 * GB300 outruns the 1/64-rate FP64 pipe; the stencil part and r = F - ... in FP64.  2 (the default
 * where available: mixed problems with M a multiple of 128 and M <= 512): the outer defect on the
 * tcgen05 tensor cores by error-free digit splitting (Ozaki et al. 2012) -- R~ (dense) and u are split
 * per time row / per grid point into 7 base-2^7 digits of 49 bits (fhmg_hmatrix_split_digits), the
 * digit products are summed exactly in FP32 tensor memory per digit-sum group and the groups are
 * combined in double-float; the stencil part B = F - A_h u is formed by a pre-pass in FP64 (every
 * third time level exactly, in 64-bit fixed point).  For time row m = 0..M-1 and grid point c,
 * |r - r_exact| <= (m+2) 2^{E_m + F_c - 46} + 2^-45 (|R~| |u|)_{m,c} + 2^-50 ((|A_h| |u|)_{m,c} + |F_{m,c}|)
 * (2^E_m > max_k |R~_mk|, 2^F_c > max_k |u_kc|).  The mode solves use double-float in modes 1 and 2.
 * EINVAL for mode 2 where it is not available. */
int fhmg_problem_set_defect_arith(fhmg_problem p, int mode);
/* BF16 tensor-core flops that one defect of defect arithmetic 2 executes per grid point (the
 * digit-tile products of the split factors, all-zero R~ digit tiles left out); EINVAL where the
 * problem has no such defect. */
int fhmg_problem_split_flops(fhmg_problem p, double* per_point);

/* FP32 products of the mixed path on the tensor cores (enable != 0, the default): with leaf 64,
 * walks with column tiles of 16 or 32 run as mma.sync m16n8k8 TF32 products split in three
 * (hi*hi + hi*lo + lo*hi, hi = tf32(a), lo = tf32(a - hi): FP32 accuracy, FP32 accumulation);
 * enable = 0 keeps every walk on the FP32 SIMT kernel.  Clears the autotuned tiles. */
int fhmg_problem_set_tensor_cores(fhmg_problem p, int enable);

/* Coarse-grid solver of fhmg_vcycle / fhmg_solve.  n <= 1 (default): the paper's recursion to one
 * interior point (Algorithm 2; the one-point system is solved by the line solve).  n = 2^k - 1 < N:
 * the coarse-grid correction on the level with n points per dimension is solved exactly in FP64
 * instead of recursing further -- a choice the paper leaves open.  A_h's sine eigenvectors
 * (eigenvalues (4/h^2) sin^2(p pi / (2(n+1))), sums of two in 2D) decouple the level into one
 * lower-triangular time system (R~ + lam_p I) w_p = RC^_p per spatial mode: an orthonormal DST-I in
 * space, one H-matrix walk per mode (Algorithm 4 with the mode's shift; the per-mode diagonal
 * inverses are built here on the device, n^dim * nb * L^2 doubles), the inverse transform.
 * Synchronises the problem's stream.  EINVAL if n is not a coarse grid size or the level has more
 * than 65535 points.  fhmg_solve_batched keeps the full recursion. */
int fhmg_problem_set_coarse_direct(fhmg_problem p, int n);

/* Cycle index of the cycles run by fhmg_vcycle / fhmg_solve (Algorithm 2's number of coarse-grid
 * cycles per level, the paper's gamma -- not the grading exponent): 1 (default) V-cycle, 2 W-cycle,
 * up to 4.  The one-point coarsest level and an exactly solved level (fhmg_problem_set_coarse_direct)
 * are solved once whatever the index.  fhmg_solve_batched always runs V-cycles. */
int fhmg_problem_set_cycle_index(fhmg_problem p, int cycle_index);

/* Test hook for the bounded device waits (the paper has no counterpart).  Arms the problem's next
 * walk launch so that every CTA's producer withholds the second chunk of its stream and the
 * consumer warps' waits give up after consumer_spin polls (1 .. 2^24) instead of 2^24: that launch
 * then leaves early without touching memory it has not been given, every copy it issued lands
 * before its CTAs retire, and the call that reads the error word returns FHMG_ETIMEOUT.  One-shot:
 * later launches run normally. */
int fhmg_problem_inject_timeout(fhmg_problem p, long long consumer_spin);

/* --- learned warm start (an addition to the method; the paper has none) ------------------------
 * For a source constant in time and a finite sine series, each spatial eigenmode s_k of A_h
 * (eigenvalue lam_k) evolves independently: u = sum_k c_k w_k(t) s_k with (R + lam_k I) w_k = 1.
 * A small network (6 features of (lam, alpha, t) -> hidden x layers, SiLU -> 1) predicts
 * lam_k w_k(t_m); the warm start projects f onto the K (1D) or K x K (2D) leading modes and
 * synthesises u0.  Training and inference run in the library's own CUDA kernels (FP32 training
 * with Adam, FP32 or BF16 tensor-core inference).  Parameters: one FP32 array, layer by layer
 * (W_l row-major n_{l+1} x n_l, then b_l). */
typedef struct fhmg_wsnet_s* fhmg_wsnet;
int fhmg_wsnet_create(int hidden, int layers, unsigned long long seed, fhmg_wsnet* out);
int fhmg_wsnet_destroy(fhmg_wsnet net);
int fhmg_wsnet_num_params(fhmg_wsnet net, long long* n);
int fhmg_wsnet_get_params(fhmg_wsnet net, float* host);
int fhmg_wsnet_set_params(fhmg_wsnet net, const float* host);
/* Y (n device floats) = network(X) for X (n x 6 device floats); bf16 != 0: BF16 tensor cores. */
int fhmg_wsnet_forward(fhmg_wsnet net, const float* X, int n, int bf16, float* Y, void* stream);
/* Mean-squared loss against targets Y and its gradient (host outputs, either may be NULL). */
int fhmg_wsnet_loss_grad(fhmg_wsnet net, const float* X, const float* Y, int n, float* loss_host,
                         float* grad_host, void* stream);
/* steps Adam steps on mini-batches of `batch` consecutive rows at random offsets of the
 * (pre-shuffled) device samples X (nsamples x 6), Y (nsamples); last mini-batch loss to *last_loss. */
int fhmg_wsnet_train(fhmg_wsnet net, const float* X, const float* Y, long long nsamples, int batch, int steps,
                     float lr, unsigned long long seed, float* last_loss, void* stream);
/* Training pairs from a solution u of the problem for a source f constant in time: features and
 * targets lam_k uhat_k(t_m) / c_k of the modes with |c_k| >= rel_thr max|c| (device outputs with room
 * for K^dim * M rows; *nrows receives the count). */
int fhmg_ws_dataset(fhmg_problem prob, const double* u, const double* f, double alpha, int K, float rel_thr,
                    float* X_out, float* Y_out, long long* nrows);
/* u0 (device, M x N^dim) = warm start for source f (constant in time) and order alpha. */
int fhmg_ws_predict(fhmg_wsnet net, fhmg_problem prob, const double* f, double alpha, int K, int bf16, double* u0);
/* Kernel launches issued so far by the network and warm-start kernels (training, inference,
 * projection, synthesis) of the whole process. */
int fhmg_wsnet_launches(long long* n);
/* The warm-started solve from HOST buffers: copies f (M x N^dim doubles, constant in time) to the
 * device, predicts u0 with the network (fhmg_ws_predict, K modes per dimension, bf16 != 0: BF16
 * inference), runs fhmg_solve from u0 and copies the solution into u_host.  Returns like fhmg_solve
 * (u_host is written also after FHMG_ENOTCONV). */
int fhmg_ws_solve_host(fhmg_wsnet net, fhmg_problem p, double* u_host, const double* f_host, double alpha, int K,
                       int bf16, int nu1, int nu2, double rtol, int max_cycles, int* cycles_out, double* relres_out);

/* fhmg_solve with HOST arrays (u in/out, f, g or NULL): copies in, solves, copies u back. */
int fhmg_solve_host(fhmg_problem p, double* u_host, const double* f_host, const double* g_host,
                    int nu1, int nu2, double rtol, int max_cycles, int* cycles_out,
                    double* relres_out);

#ifdef __cplusplus
}
#endif
#endif /* FHMG_H_ */
