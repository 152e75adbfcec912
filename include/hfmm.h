/*
 * hfmm.h - C ABI of the GB300 FMM-accelerated Helmholtz boundary-integral library.
 *
 * The operator follows the problem statement of "Extreme Scale FMM-Accelerated
 * Boundary Integral Equation Solver for Wave Scattering" (arXiv:1803.09948):
 *
 *   Green's function        G(x,y) = exp(i k R) / (4 pi R), R = |x - y|      (Eq. 6)
 *   sound-soft scattering   int_S G(r,r') q(r') dS' = p_inc(r) on S          (Eq. 7)
 *   Nystrom discretisation  Z I = V_inc, [V_inc]_i = p_inc(x_i)              (Eq. 9, 10)
 *
 * Discretisation used by every call (flat triangles, three points each):
 *   point 3n+a (a = 0,1,2) of triangle n sits at barycentric (2/3,1/6,1/6)
 *   rotated to vertex a; its weight is area_n/3 and its basis function the
 *   linear Lagrange function L_(n,a) = 2 lambda_a - 1/3 (1 at the point, 0 at
 *   the other two).  For target x_i the singular set S(i) holds its own
 *   triangle and every triangle with a point within near_factor * (mean edge
 *   length) of x_i; those triangles are integrated exactly (Sec. 2.2, the
 *   self- and near-singularity treatment of Listing 1 and Sec. 6.4), every
 *   other source point enters with the point rule w_j G(x_i, x_j):
 *
 *     (Z s)_i = sum_{n not in S(i)} sum_a w_(n,a) G(x_i, x_(n,a)) s_(n,a)
 *             + sum_{n in S(i)}     sum_a s_(n,a) int_{T_n} G(x_i,y) L_(n,a)(y) dS_y
 *
 * The point part is evaluated by the FMM (Sec. 2.3, Eq. 11-14: P2M, M2M, M2L,
 * L2L, L2P on a uniform octree, P2P between neighbouring leaves) and the
 * exact-minus-point correction on S(i) is a sparse matrix built once per plan.
 *
 * Conventions
 *   - Status: 0 success, negative error (HFMM_E_*), HFMM_NOT_CONVERGED (+1)
 *     from hfmm_solve when max_iter is reached.  No C++ exception crosses the ABI.
 *   - Vectors ("density", "potential", "rhs", "x") are DEVICE pointers to
 *     complex64 (interleaved float re, im) of length N = 3 * n_tri in user
 *     point order (point 3n+a as above), nrhs of them stored one after another
 *     (column-major N x nrhs).  The caller owns them; the library never frees
 *     or keeps them beyond the call.
 *   - Mesh arrays passed to hfmm_plan_create are HOST pointers; they are
 *     copied and need not outlive the call.
 *   - Streams are cudaStream_t passed as void* (NULL: the legacy default
 *     stream).  hfmm_matvec and hfmm_direct are stream-ordered and return
 *     before the work completes; hfmm_solve returns after the solve completes.
 *   - A plan is not thread-safe: calls on one plan must not overlap in time or
 *     on the device (it owns one set of scratch buffers).
 *   - Only real wavenumbers are supported (k_im must be 0).
 */
#ifndef HFMM_H
#define HFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HFMM_OK 0
#define HFMM_NOT_CONVERGED 1
#define HFMM_E_INVALID (-1)   /* bad argument (null pointer, size, value out of range) */
#define HFMM_E_MESH (-2)      /* degenerate mesh: zero-area triangle, non-finite vertex, bad index */
#define HFMM_E_NOMEM (-3)     /* device allocation failed or over the configured memory budget */
#define HFMM_E_CUDA (-4)      /* a CUDA runtime call failed */
#define HFMM_E_TIMEOUT (-5)   /* reserved: a bounded device wait gave up */
#define HFMM_E_OVERFLOW (-6)  /* a fixed-capacity table overflowed (e.g. near set too large) */

typedef struct hfmm_plan hfmm_plan; /* opaque; owns all device state of one mesh and wavenumber */

typedef struct {
    int leaf_max;       /* max points per leaf; the octree depth is the smallest meeting it (64) */
    int depth;          /* >0: force this octree depth instead (0: automatic) */
    int p_fixed;        /* >0: expansion order on every level; 0: per-level formula below */
    int p_min;          /* floor for the formula p_l = ceil(k a_l + 6 log10(k a_l + pi)),
                           a_l = circumradius of a level-l box */
    double near_factor; /* near radius = near_factor * mean edge length (1.0) */
    int quad_order;     /* Gauss-Legendre points per direction of the Duffy-type
                           self/near quadrature (10) */
    int restart;        /* GMRES restart length m (30) */
    int max_iter;       /* GMRES iteration cap (1000) */
    double tol;         /* GMRES relative residual ||b - Z x|| / ||b|| target (1e-4) */
    double mem_budget_bytes; /* refuse a plan whose device footprint exceeds this (0: no limit) */
    int m2l_tensor;     /* 1: M2L of levels with (p+1)^2 <= 64 on the tensor cores (BF16 split in
                           three products, FP32 accumulation); 0: FP32 SIMT everywhere (1) */
    int adaptive;       /* 1: adaptive octree: a box is split only while it holds more than
                           leaf_max points, so leaves sit at several depths (depth > 0 caps them);
                           leaves interact directly when their ancestors at the coarser leaf's
                           level touch, every other pair through M2L between same-level boxes
                           (the interaction lists of Sec. 2.3 read for unequal leaves).  Batched
                           right-hand sides then run one at a time.  0: uniform depth (0) */
    int autotune;       /* 1: at plan creation, time each tunable choice below that is left at -1
                           (or 0 for tc_group) on the plan's own data with CUDA events and keep the
                           fastest (the GPU counterpart of the paper's search for task size and
                           leaf size, Sec. 3.2 / 6.2); hfmm_plan_tuning reports the result.
                           0: use the defaults (0) */
    int p2p_kernel;     /* near-field kernel: 0 staged (four lanes per target), 1 packed FP32x2
                           (two targets per lane, two sources per instruction), 2 the packed
                           arithmetic in persistent blocks that load the next leaf's sources
                           (cp.async) while evaluating the current one; -1 default/tuned (-1) */
    int m2l_kernel;     /* tensor-core M2L: 0 source-stationary work items (one offset's operator
                           applied to gathered multipoles, bulk reductions into the locals);
                           1 target-stationary tiles (a block keeps 128 targets' locals on chip and
                           applies the 56 canonical operators of the offsets' reflection classes,
                           writing each local once); -1 default/tuned (-1) */
    int tc_group;       /* work items per tensor-core block: 8, 16 or 32; 0 default/tuned (0) */
    int overlap;        /* single right-hand-side matvec on a uniform tree, captured once as a
                           CUDA graph and replayed: 1 near field and correction on a second branch
                           beside the far field; 0 one stage after another; -1 default/tuned (-1) */
    int precision;      /* 1: the plan also keeps an FP64 near field and correction: FP64 positions
                           and weights, correction integrals with FP64 quadrature nodes kept in
                           FP64, used by hfmm_matvec_df and by the outer residual of
                           hfmm_solve_refined (the far field stays FP32); 0: FP32 only (0) */
} hfmm_config;

/* Fills *cfg with the defaults shown in parentheses above (p_min = 7). */
void hfmm_default_config(hfmm_config* cfg);

/*
 * Builds a plan for the surface (vertices: n_vert x 3 doubles, tris: n_tri x 3
 * vertex indices, counter-clockwise) and wavenumber k = k_re + i k_im (Eq. 3,
 * 6).  Computes quadrature points and weights, the octree and interaction
 * lists, the translation operators and the sparse near/self correction
 * (Sec. 2.2-2.3).  Work is issued on `stream` and the call returns after it
 * completes.  On failure *out is NULL and nothing is leaked.
 */
int hfmm_plan_create(const hfmm_config* cfg, const double* vertices, int64_t n_vert,
                     const int32_t* tris, int64_t n_tri, double k_re, double k_im,
                     void* stream, hfmm_plan** out);

/* Releases the plan's device memory.  The caller must have completed (or synchronised) the work
 * it issued with this plan on its own streams; the plan's internal streams are synchronised
 * here, not the whole device.  NULL is a no-op. */
void hfmm_plan_destroy(hfmm_plan* plan);

int64_t hfmm_num_points(const hfmm_plan* plan); /* N = 3 * n_tri, or -1 for NULL */

/*
 * Copies the quadrature points (xyz: N x 3), weights (w: N) and triangle ids
 * (tri: N) to HOST arrays in user order; any of the three may be NULL.
 */
int hfmm_points(const hfmm_plan* plan, double* xyz, double* w, int32_t* tri);

/*
 * Plan facts for reporting: depth (octree leaf level), order per level
 * (orders[l] for l = 0..depth; levels 0 and 1 carry no expansions and report 0,
 * orders must hold 32 ints), number of leaves, near/self correction nonzeros,
 * M2L translations, and device bytes held by the plan.  Any pointer may be NULL.
 */
int hfmm_plan_info(const hfmm_plan* plan, int* depth, int* orders, int64_t* n_leaves,
                   int64_t* corr_nnz, int64_t* m2l_translations, int64_t* device_bytes);

/*
 * potential = Z density (Eq. 9-10) with the FMM for the point part, nrhs
 * right-hand sides.  density and potential are device complex64 vectors,
 * N x nrhs, user point order; they may not overlap.  Stream-ordered.
 */
int hfmm_matvec(hfmm_plan* plan, const void* density, void* potential, int nrhs, void* stream);

/*
 * hfmm_matvec with HOST buffers: density and potential are host complex64
 * vectors, N x nrhs, user point order (page-locked memory gives the fastest
 * copies; pageable memory works).  Each chunk of up to 64 right-hand sides is
 * copied to plan-owned device staging (allocated on the first call, 2 x 8 x N x
 * min(nrhs, 64) bytes, kept and counted in the plan's device bytes), multiplied,
 * and copied back, all on `stream`; the call returns after the last copy has
 * landed.  The caller owns both buffers.
 */
int hfmm_matvec_host(hfmm_plan* plan, const void* density, void* potential, int nrhs, void* stream);

/*
 * Like hfmm_matvec but evaluates only part of the operator (for tests and
 * breakdowns): parts bit 0 = near field (P2P between neighbouring leaves),
 * bit 1 = far field (P2M..L2P), bit 2 = near/self correction.  parts = 7 is
 * hfmm_matvec.
 */
int hfmm_matvec_parts(hfmm_plan* plan, const void* density, void* potential, int nrhs,
                      int parts, void* stream);

/*
 * potential = Z density by direct O(N^2) summation of the point part plus the
 * same correction (a reference for tests and small problems).  Same argument
 * conventions as hfmm_matvec.
 */
int hfmm_direct(hfmm_plan* plan, const void* density, void* potential, int nrhs, void* stream);

/*
 * rhs_out (device complex64, N x nrhs) = incident plane waves
 * p_inc(x) = exp(i k d.x) at the quadrature points (Eq. 9's V_inc);
 * dirs: HOST array of nrhs unit vectors (3 doubles each).  Stream-ordered.
 */
int hfmm_rhs_planewave(hfmm_plan* plan, const double* dirs, int nrhs, void* rhs_out, void* stream);

/*
 * Solves Z x = rhs by restarted GMRES(m) (the paper's solver, Sec. 5.1 and
 * 6.4) with the FP32 FMM matvec.  The Krylov basis and the element-wise
 * Arnoldi arithmetic (Gram-Schmidt, two classical passes; norms; updates) are
 * FP64-class double-float (hi + lo FP32 pairs, 48-bit significand, error-free
 * transformations); partial sums, the Hessenberg matrix, Givens rotations,
 * the least-squares solve and the residual tests are FP64.  x0 = 0.  Stops when
 * the relative residual reaches cfg->tol (checked on the true residual at
 * exit).  rhs, x_out: device complex64, N x nrhs (right-hand sides solved one
 * after another).  iters_out / relres_out (HOST, nrhs entries each, may be
 * NULL) receive the iteration count and final true relative residual.
 * Returns HFMM_NOT_CONVERGED if any right-hand side hit max_iter (x_out then
 * holds the last iterate).  Returns after completion.
 */
int hfmm_solve(hfmm_plan* plan, const void* rhs, void* x_out, int nrhs, int* iters_out,
               double* relres_out, void* stream);

/*
 * Whether the plan's last single right-hand-side solve ran each GMRES cycle as one graph
 * launch: a CUDA graph whose while node repeats one Arnoldi step (matvec, Gram-Schmidt,
 * rotations, residual estimate) until a kernel of the step sets its condition to zero, with no
 * host round trip per iteration (*cycle_graph = 1), or with the host driving the same steps
 * (0: adaptive trees, or a graph that could not be built).  HOST output.
 */
int hfmm_solver_info(const hfmm_plan* plan, int* cycle_graph);

/*
 * Solves G independent problems Z_g x_g = rhs_g together (the paper's GMRES solve, Sec. 5.1 and
 * 6.4, for several scattering requests at once): one right-hand side per plan, G distinct plans
 * of possibly different meshes and wavenumbers, each with its own restart, tolerance and
 * iteration limit.  The solves advance in lockstep over restart cycles; each cycle of every
 * unfinished solve runs inside ONE shared graph launch (one while node per solve, a finished
 * solve's loop closed by a gate), so the requests' steps share the launch and run side by side
 * on the device; the cycle ends (update, true residual) run per solve.  Results equal
 * hfmm_solve's on each plan.  plans, rhs, x_out: HOST arrays of G entries (rhs / x_out are
 * device complex64 [N_g]); iters_out / relres_out: HOST arrays of G (may be NULL).  Returns
 * after completion; HFMM_NOT_CONVERGED if any solve hit its iteration limit; HFMM_E_INVALID for
 * G outside 1..HFMM_GROUP_MAX, NULL entries or a plan given twice.
 */
#define HFMM_GROUP_MAX 64
int hfmm_solve_group(hfmm_plan* const* plans, int G, const void* const* rhs, void* const* x_out, int* iters_out,
                     double* relres_out, void* stream);

/*
 * Off-surface evaluation (the paper's scattered field at observation points,
 * Sec. 6.4): field[t] = sum_j w_j exp(i k |t - x_j|) / (4 pi |t - x_j|) density_j,
 * the single-layer potential of the density at n_targets points t away from the
 * surface (the point rule: accurate for targets farther than about one mean edge
 * length from the surface).  density: device complex64 [N], user order;
 * targets: HOST doubles [n_targets][3]; field_out: device complex64
 * [n_targets].  Direct summation on the device (all pairs, FP32 arithmetic on
 * positions split into FP32 hi + lo).  For the sound-soft scattering problem the
 * scattered field is -field of the solved density.  Stream-ordered.
 */
int hfmm_field(hfmm_plan* plan, const void* density, const double* targets, int64_t n_targets, void* field_out,
               void* stream);

/*
 * Mixed-precision iterative refinement for one right-hand side (the paper's
 * GMRES solve taken to a tighter residual; configuration "refinement to
 * 1e-6"): x_0 = 0; repeat  r = b - A_outer x  (formed in double-float, FP64-class;
 * on an outer plan created with precision = 1 its near field and correction are evaluated
 * in FP64 on the whole double-float iterate, as in hfmm_matvec_df),
 * stop when |r| <= tol_outer |b|, solve A_inner d = r by GMRES on the inner plan
 * (its own restart and tolerance), x += d (double-float).  `inner` and `outer`
 * are plans of the same mesh and wavenumber (same N, user point order); the
 * outer plan should be the more accurate operator (higher order, FP32 SIMT M2L).
 * rhs, x_out: device complex64 [N].  outer_iters / inner_iters / relres_out
 * (HOST, may be NULL): refinement steps, GMRES iterations summed over the inner
 * solves, final |r| / |b| with the outer operator.  Returns HFMM_NOT_CONVERGED
 * if max_outer steps do not reach tol_outer, HFMM_E_INVALID on mismatched plans.
 */
int hfmm_solve_refined(hfmm_plan* inner, hfmm_plan* outer, const void* rhs, void* x_out, double tol_outer,
                       int max_outer, int* outer_iters, int* inner_iters, double* relres_out, void* stream);

/*
 * Double-float matvec for one right-hand side: density_df and potential_df are device arrays
 * of N float4 (re_hi, im_hi, re_lo, im_lo), user order, the value being hi + lo.  On a plan
 * created with precision = 1, the near field (the point sum over each leaf's own and
 * neighbouring leaves, Eq. 7) and the near/self correction (Sec. 2.2) are evaluated in FP64 on
 * the full hi + lo density; the far field (Sec. 2.3's FMM) in FP32 on the high part.  parts:
 * bit 0 near field, 1 far field, 2 correction (7: the whole operator).  Stream-ordered.
 * HFMM_E_INVALID on a precision-0 plan or bad arguments.
 */
int hfmm_matvec_df(hfmm_plan* plan, const void* density_df, void* potential_df, int parts, void* stream);

/*
 * hfmm_matvec for one right-hand side with CUDA events recorded on `stream`
 * between the stages; returns after completion.  stage_ms (HOST,
 * HFMM_NUM_STAGES floats) receives the device time of: 0 density prep, 1 near
 * field (P2P), 2 P2M, 3 M2M, 4 M2L on the FP32 SIMT kernel (levels above the
 * tensor-core order limit, or every level when m2l_tensor = 0), 5 M2L on the
 * tensor cores, 6 L2L, 7 L2P, 8 correction, 9 output permutation.
 */
#define HFMM_NUM_STAGES 10
int hfmm_matvec_timed(hfmm_plan* plan, const void* density, void* potential, float* stage_ms,
                      void* stream);

/*
 * Algorithmic work of one matvec (HOST, HFMM_NUM_COSTS doubles): 0 near-field
 * source-target pairs (j != i), 1 M2L complex multiply-adds (sum over
 * translations of P_l^2), 2 M2M + L2L complex multiply-adds, 3 correction
 * nonzeros, 4 points N, 5 expansion coefficients (all levels, multipoles +
 * locals, padded), 6 the part of 1 done on the tensor cores, 7 the number of
 * M2L translations done on the tensor cores, 8 complex coefficients of the
 * leaves' expansions (sum over leaves of P_leaf-level), 9 complex multipole
 * coefficients of level 2, 10 complex multipole coefficients of levels 2..L,
 * 11 complex multipole coefficients of level L.
 */
#define HFMM_NUM_COSTS 12
int hfmm_plan_costs(const hfmm_plan* plan, double* costs);

/*
 * Reads and clears the plan's device error flag, set by a kernel whose bounded
 * wait gave up (it then skips its remaining work).  Synchronises `stream`.
 * Returns HFMM_OK or HFMM_E_TIMEOUT.
 */
int hfmm_device_status(hfmm_plan* plan, void* stream);

/*
 * The plan's kernel choices (HOST, HFMM_NUM_TUNABLES ints): 0 near-field kernel
 * (p2p_kernel), 1 tensor-core M2L kernel (m2l_kernel), 2 work items per tensor-core
 * block (tc_group), 3 two-branch captured matvec (overlap) -- the configured value,
 * or when that was left open the default or, with autotune = 1, the fastest measured.
 * tuned_ms (HOST, HFMM_NUM_TUNABLES x HFMM_TUNE_CANDIDATES floats, may be NULL): the
 * device time of one matvec with each candidate of each tunable, in the order of the
 * candidates (near field: 0, 1; M2L kernel: 0, 1; tc_group: 8, 16, 32; overlap: 0, 1),
 * -1 where not measured.
 */
#define HFMM_NUM_TUNABLES 4
#define HFMM_TUNE_CANDIDATES 4
int hfmm_plan_tuning(const hfmm_plan* plan, int* choices, float* tuned_ms);

/*
 * The plan-time tuner's rule, on its own (host only, no device work): given the measured
 * time ms[c] of candidate c of `tunable` (n candidates in the order above; a negative or
 * non-finite entry means not measured), *value = the fastest measured candidate's value,
 * except that the default stays unless the fastest is at least 2 % faster.  Returns
 * HFMM_E_INVALID for a bad tunable or count, or when nothing was measured.
 */
int hfmm_tune_choose(int tunable, const float* ms, int n, int* value);

/* Number of kernels this plan has launched on the device since it was created. */
int64_t hfmm_launch_count(const hfmm_plan* plan);

/*
 * Scratch-free point sum (the paper has no counterpart; it is a service for
 * callers that cannot allocate device memory, e.g. code running inside
 * another framework's memory pool or arena, or a process whose device
 * footprint must stay fixed after start-up, where cudaMalloc is forbidden or
 * unavailable).
 *
 *   potential_i = sum_{j != i, R_ij > 0} w_j exp(i k R_ij) / (4 pi R_ij) density_j
 *
 * i.e. the point part of the operator, the same result as hfmm_matvec_parts
 * with parts = 1 on a plan whose single leaf holds every point.  No plan is
 * needed.  xyz (n x 3 doubles) and w (n doubles) are DEVICE arrays (for
 * example the output of hfmm_points copied to the device); density and
 * potential are DEVICE complex64 vectors of length n; the caller owns all of
 * them.  Stream-ordered, O(n^2) work.
 *
 * Working memory is a fixed file-scope device array of HFMM_NOALLOC_MAX_POINTS
 * entries (32 bytes each, 8 MiB), held by every device that loads the library
 * until the process exits; the call itself never calls cudaMalloc or cudaFree.
 * With CUDA's default lazy module loading the array (with the module holding
 * it) is brought onto a device by the first call there, which therefore grows
 * the device footprint by about 8 MiB once: a caller whose footprint must not
 * grow later makes one call (any n) at start-up, or runs with
 * CUDA_MODULE_LOADING=EAGER.  That first call on a device also looks up the
 * array's device address (with that device current); make it before any
 * stream capture.  `stream` must belong to the current device (else
 * HFMM_E_INVALID).  n > HFMM_NOALLOC_MAX_POINTS returns HFMM_E_OVERFLOW;
 * a null pointer, n <= 0, or k not finite and positive returns HFMM_E_INVALID
 * (see hfmm_last_error).  All calls on a device share the one array, so calls
 * that overlap on the GPU (on different streams, or from different threads)
 * race and must be serialised by the caller.  Each call overwrites the entries
 * it reads; nothing needs clearing between calls.  Positions are staged as
 * float32 hi + lo parts of k (x - x_0), so close pairs keep float32 relative
 * precision at any |k x|.
 */
#define HFMM_NOALLOC_MAX_POINTS 262144
int hfmm_point_sum_noalloc(const double* xyz, const double* w, int64_t n, double k,
                           const void* density, void* potential, void* stream);

/* Static description of a status code (never NULL). */
const char* hfmm_status_string(int status);

/* Detail of the last error raised on the calling thread ("" if none); the
   string is owned by the library and valid until the next call on the thread. */
const char* hfmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HFMM_H */
