/*
 * nf.h -- C ABI of the GB300 (sm_103a) library for the RBF neural-field method of
 * Shaw, Kilpatrick & Avitabile, "Radial Basis Function Techniques for Neural Field
 * Models on Surfaces".
 *
 * The problem (§2, Eq. (2.1)): du/dt = -u + g + int_D w(x, y) f(u(y)) dmu(y) on a
 * node set Xi with a triangulation {E_j}, discretised as the fully discrete
 * collocation scheme of §2.2, Eq. (2.9):
 *     alpha_i' = -alpha_i + sum_j w(x_i, x_j) mu_j f(alpha_j) + gamma_i(t),
 * whose weights mu_j come from RBF quadrature (§3.2 Eq. (3.5), §3.3 Eq. (3.6)).
 *
 * Conventions, for every entry point:
 *  - Return value: nf_status.  NF_OK on success; on failure a thread-local message is
 *    available from nf_last_error().  The library never aborts, traps or exits.
 *  - Array arguments are DEVICE pointers (e.g. torch CUDA tensor data pointers),
 *    contiguous, row-major, owned by the caller; outputs are allocated by the caller.
 *    Arguments documented as "host" are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *    work is ordered on that stream.  Calls return once the work is enqueued, except
 *    where a call documents that it synchronises the stream.
 *  - The library owns only what lives inside an nf_operator handle (packed node
 *    arrays, dense operator planes, partial-sum workspace, CUDA graphs) and frees it
 *    in nf_operator_destroy.  Temporary setup workspace is stream-ordered
 *    (cudaMallocAsync) and released before the call returns its work.
 *  - Asynchronous device faults surface as NF_ERR_CUDA at the next call.
 */
#ifndef NF_H
#define NF_H

#include <stdint.h>

#if defined(__GNUC__)
#define NF_API __attribute__((visibility("default")))
#else
#define NF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NF_OK = 0,
    NF_ERR_ARG = 1,          /* invalid argument (null pointer, size, alignment, rule of §3.1) */
    NF_ERR_SINGULAR = 2,     /* an element's interpolation system is singular (§3.1) */
    NF_ERR_NONFINITE = 3,    /* an RK4 step produced a non-finite state (see nf_operator_check) */
    NF_ERR_TIMEOUT = 4,      /* a bounded device wait gave up; the kernel returned early */
    NF_ERR_NOMEM = 5,        /* device allocation failed */
    NF_ERR_CUDA = 6,         /* CUDA runtime / launch error */
    NF_ERR_UNSUPPORTED = 7   /* valid request the library does not implement */
} nf_status;

/* Message describing the last failure on the calling thread ("" if none). */
NF_API const char *nf_last_error(void);

/* ABI version, (major << 16) | minor. */
NF_API int nf_version(void);

/* ------------------------------------------------------------------------------
 * §3.1 stencils.  For each element E_e (a triangle of the caller's triangulation),
 * S(E_e) = the k nodes nearest to the centre of E_e.  The centre is the centroid
 * ((a + b) + c) / 3; distance is Euclidean in R^dim (§4: "standard Euclidean
 * distance ... for stencil selection").  Ties are broken by node index, so the
 * result is unique: row e lists node indices in ascending (distance^2, index).
 *
 *   nodes     n x dim   FP64   node coordinates, dim in {2, 3}
 *   tris      m x 3     int32  element vertex indices (0-based, < n)
 *   k                          stencil size, 1 <= k <= min(n, 128)
 *   stencils  m x k     int32  output
 * Errors: NF_ERR_ARG (sizes, k), NF_ERR_CUDA.  Distances are evaluated in FP64
 * without contraction, so indices agree bit-for-bit with a plain FP64 evaluation.
 * ---------------------------------------------------------------------------- */
NF_API nf_status nf_build_stencils(const double *nodes, int64_t n, int dim,
                            const int32_t *tris, int64_t m, int k,
                            int32_t *stencils, void *stream);

/* The same selection around m caller-given centres (m x dim FP64 device array) instead of
 * triangle centroids: row e lists the k nodes nearest to centers[e], ascending (distance^2,
 * index).  Centres may lie anywhere (the search grid covers nodes and centres).
 * Errors: NF_ERR_ARG (sizes, k, non-finite coordinates), NF_ERR_CUDA. */
NF_API nf_status nf_build_stencils_at(const double *nodes, int64_t n, int dim, const double *centers, int64_t m,
                                      int k, int32_t *stencils, void *stream);

/* ------------------------------------------------------------------------------
 * §3.2 Eq. (3.5) (flat, dim = 2) and §3.3 Eq. (3.6) (closed surfaces, dim = 3):
 * RBF quadrature weights mu (written q here).  Per element: polyharmonic spline
 * r^3 (§3.1 Eq. (3.3), ell = 3) plus polynomials of total degree <= deg, the saddle
 * system of Eq. (3.4) with the analytic integrals of each basis function over the
 * element as right-hand side; node weight = sum of the element weights of every
 * stencil containing the node.  On surfaces the stencil is first mapped to the
 * element's plane by the central projection through the projection point p_E
 * (three cutting planes, §3.3) and each weight is multiplied by the Jacobian of
 * mu_E at the projected node (the area factor of Eq. (3.6)).
 *
 *   nodes     n x dim   FP64   node coordinates
 *   normals   n x 3     FP64   outward unit node normals (dim 3); NULL when dim = 2
 *   tris      m x 3     int32  triangulation (closed and edge-manifold when dim = 3)
 *   stencils  m x k     int32  from nf_build_stencils
 *   deg                        appended polynomial degree, 0..4, with
 *                              (deg+1)(deg+2)/2 <= k (unisolvency, §3.1)
 *   q         n         FP64   output weights
 *   bad_element  host int64*   set to the first singular element, or -1 (may be NULL)
 * Synchronises `stream` (it must report per-element failures).
 * Errors: NF_ERR_ARG, NF_ERR_SINGULAR (q undefined), NF_ERR_NOMEM, NF_ERR_CUDA.
 * ---------------------------------------------------------------------------- */
NF_API nf_status nf_quad_weights(const double *nodes, const double *normals, int64_t n, int dim,
                          const int32_t *tris, int64_t m, const int32_t *stencils, int k,
                          int deg, double *q, int64_t *bad_element, void *stream);

/* The same call with the options gathered in a struct: dim (2 flat, 3 surface), phs_order
 * (the polyharmonic spline r^phs_order of Eq. (3.3); 3 is what is implemented, others
 * return NF_ERR_UNSUPPORTED), poly_deg (0..4), curved (1: closed surface, normals required;
 * must agree with dim).  o is a host pointer.  Errors as nf_quad_weights. */
typedef struct {
    int dim;
    int phs_order;
    int poly_deg;
    int curved;
} nf_quad_opts;
NF_API nf_status nf_quad_weights_opts(const double *nodes, const double *normals, int64_t n, const int32_t *tris,
                                      int64_t m, const int32_t *stencils, int k, const nf_quad_opts *o, double *q,
                                      int64_t *bad_element, void *stream);

/* ------------------------------------------------------------------------------
 * Kernel and operator.
 * Lateral-inhibition ("Mexican hat") kernel, §5 Eq. (5.1) in unnormalised form:
 *     w(r) = A1 exp(-r^2 / s1^2) - A2 exp(-r^2 / s2^2),   r = |x_i - x_j| (Euclidean,
 * chord distance on surfaces).  Firing rate §4 Eq. (4.4):
 *     f(u) = 1 / (1 + exp(-beta (u - theta))), per-trajectory beta, theta.
 * period = L > 0 takes r as the doubly periodic distance of §4, Eq. (dist), on the flat
 * square of side L: the x and y differences are reduced to their nearest images
 * (|dx|, |dy| <= L/2), z differences are not.  Nodes may lie anywhere; the square's
 * flat-torus metric is the same for every cell.  period = 0: Euclidean.
 * ---------------------------------------------------------------------------- */
typedef struct {
    float A1, s1, A2, s2;
    float period;
} nf_kernel;

typedef enum {
    NF_MATRIX_FREE = 0,   /* pair sum evaluated on the fly every stage (FP32) */
    NF_DENSE_FP32 = 1,    /* W diag(q) precomputed once, FP32, streamed every stage */
    NF_DENSE_BF16X2 = 2,  /* W diag(q) / s_i stored as bf16 hi + bf16 lo, FP32 accumulate */
    NF_DENSE_SYM_FP32 = 4, /* the symmetric kernel matrix W (w is radial, §2.2) stored once as
                             its upper-triangle 1024 x 1024 blocks, FP32; q applied on the
                             vector side; each block serves a row and a column sum, half the
                             bytes of NF_DENSE_FP32 per stage */
    NF_DENSE_SYM_BF16X2 = 5 /* the same blocks in the precision form: W_ij = s_i s_j (hi + lo),
                             bf16 hi + bf16 lo (16 significant bits), s_i a power of two near
                             sqrt(max_j |W_ij|), FP32 accumulation; the vector is scaled by s
                             on the way in and each sum by its s_i on the way out */
} nf_path;

typedef struct nf_operator nf_operator;

/* Create the operator I = W diag(q) f(.) of Eq. (2.9) on n nodes.
 *   x   n x 3  FP32  node coordinates (z = 0 for flat domains)
 *   q   n      FP32  quadrature weights mu_j
 *   path             nf_path; dense paths allocate n x n (FP32: 4 n^2 bytes; BF16X2:
 *                    4 n^2 bytes + 4 n; the symmetric paths 2 n^2 + 2048 n bytes, plus 4 n
 *                    for SYM_BF16X2) inside the handle and build it on `stream`.
 *   op  host         receives the handle.
 * x and q are copied into the handle; the caller may free them afterwards.
 * Errors: NF_ERR_ARG, NF_ERR_NOMEM, NF_ERR_CUDA. */
NF_API nf_status nf_operator_create(const float *x, const float *q, int64_t n, nf_kernel kp,
                             int path, void *stream, nf_operator **op);

NF_API nf_status nf_operator_destroy(nf_operator *op);

/* Batched tensor-core operator over several node sets (the batching form of Eq. (2.9)):
 * ops[g] (count <= 8) are NF_DENSE_BF16X2 operators with n_g >= 64 nodes, advanced with
 * B_per_op[g] trajectories each.  Per RK4 stage one persistent tcgen05 GEMM computes, for
 * every group, D = Whi Fhi + Whi Flo + Wlo Fhi (bf16 inputs, FP32 tensor-memory
 * accumulation; F = f(U) split into bf16 hi + lo) and its epilogue performs the stage
 * update.  The GEMM works on sub-groups of at most 256 trajectories of one node set (its
 * MMA width); one launch holds at most 8 sub-groups, so sum_g ceil(B_g / 256) <= 8
 * (otherwise NF_ERR_UNSUPPORTED).  At creation the call times a small set of launch
 * configurations on the device (ring depth, whether members of 128 or more trajectories are
 * cut in two, the weight of the MMA term in the tile schedule) and keeps the fastest; see
 * nf_operator_group_tuning.  Results do not depend on that choice.  A grouped operator
 * takes, in nf_nonlocal_apply / nf_rk4_advance, B = the total number of trajectories and
 * u, I as the concatenation over g (in ops order) of the B_g x n_g blocks; beta, theta
 * likewise concatenated; forcing must be NONE; ckpt holds (nsteps / C + 1) copies of the
 * concatenated state.  The members must outlive the group, which does not own them
 * (nf_operator_destroy on the group frees only its own buffers).  Synchronises `stream`.
 * Errors: NF_ERR_ARG, NF_ERR_NOMEM, NF_ERR_CUDA, NF_ERR_UNSUPPORTED (more than 8 sub-groups;
 * no two-SM cluster of the kernel fits on the device), NF_ERR_TIMEOUT (a bounded wait gave
 * up during the timing launches). */
NF_API nf_status nf_operator_group(nf_operator *const *ops, const int *B_per_op, int count, void *stream,
                                   nf_operator **grouped);

/* Launch configuration the autotuner of nf_operator_group chose (no paper counterpart),
 * host outputs: ring depth (64 KB shared-memory slots in flight per CTA: 2 or 3), the
 * number of pieces a member of 128 or more trajectories was cut into (1 or 2), the weight of
 * the MMA term in the longest-processing-time tile costs, the sub-groups of one launch, and
 * the chosen configuration's time per nonlocal-sum launch (ms).  Errors: NF_ERR_ARG. */
NF_API nf_status nf_operator_group_tuning(nf_operator *op, int *ring_depth, int *traj_split, double *lpt_coef,
                                          int *subgroups, float *ms);

/* Set the launch configuration of a grouped operator instead of the autotuner's choice (no
 * paper counterpart; for reproducible measurements and for testing every candidate):
 * ring_depth 2 or 3, traj_split 1 or 2, lpt_coef > 0.  Synchronises `stream`, drops captured
 * RK4 steps (the next nf_rk4_advance captures again).  Results do not depend on the
 * configuration.  Errors: NF_ERR_ARG, NF_ERR_UNSUPPORTED (the split needs more than 8
 * sub-groups), NF_ERR_CUDA. */
NF_API nf_status nf_operator_group_configure(nf_operator *op, int ring_depth, int traj_split, double lpt_coef,
                                             void *stream);

/* Synchronise `stream` and report device-side failures recorded on the operator:
 * NF_ERR_TIMEOUT when a bounded wait in a kernel gave up; NF_ERR_NONFINITE when a step of
 * nf_rk4_advance on the matrix-free or a dense path left a non-finite value (NaN or
 * infinity, e.g. from a non-finite initial state) in the state.  The first failure stays
 * recorded: clears nothing. */
NF_API nf_status nf_operator_check(nf_operator *op, void *stream);

/* Measurement helpers (no paper counterpart).  With profiling enabled, the captured RK4
 * step records CUDA events immediately before and after each stage's nonlocal-sum
 * launches (the dominant kernels).
 *   nf_operator_profile: enable = 0 switches profiling off; enable = K >= 1 switches it on
 *     with a ring of K event sets: the K most recent steps of nf_rk4_advance keep their
 *     own timings (each graph replay records into the next set), so a caller can time
 *     steps back to back and read them afterwards.  Resets the count of profiled steps.
 *   nf_operator_kernel_ms: waits for the most recent profiled step and returns its four
 *     stage durations in milliseconds (host float[4]).
 *   nf_operator_kernel_ms_history: waits for the most recent profiled step and returns the
 *     stage durations of the last `steps` profiled steps, oldest first (host float[4 steps]);
 *     steps <= K and <= the steps launched since profiling was enabled.
 * Errors: NF_ERR_ARG (profiling off, steps out of range), NF_ERR_CUDA. */
NF_API nf_status nf_operator_profile(nf_operator *op, int enable);
NF_API nf_status nf_operator_kernel_ms(nf_operator *op, float *ms);
NF_API nf_status nf_operator_kernel_ms_history(nf_operator *op, int steps, float *ms);
/* Launch shape of the matrix-free pair kernel picked by the operator's autotuner (timed
 * once per node count at creation): rows per warp, columns per shared-memory tile and
 * column splits (host ints; -1 for other paths). */
NF_API nf_status nf_operator_launch_shape(nf_operator *op, int *rows_per_warp, int *tile_cols, int *splits);

/* Schedule of a matrix-free operator's sums for up to three trajectories (Eq. (2.9); from
 * four trajectories on the multi-trajectory kernels share each pair's exponentials):
 *   NF_MF_AUTO       the symmetric block-pair kernel (each unordered pair once, w radial)
 *                    when it has block pairs for 2/3 of the SMs and its partial sums
 *                    (4 n^2 / 1024 bytes per trajectory) fit an eighth of the device
 *                    memory, else the packed kernel (default; the switch is at about
 *                    13,300 nodes on 152 SMs, and again at about 3 million);
 *   NF_MF_SYMMETRIC  always the symmetric kernel;
 *   NF_MF_PACKED     always the packed row-block x column-split kernel (ordered pairs);
 *   NF_MF_SYMMETRIC_512, NF_MF_SYMMETRIC_1024   the symmetric kernel with that node-block
 *                    size (by default the operator's autotuner picks 1,024, or 512 where
 *                    that measured faster); a change of block size switches culling off.
 * Results agree to FP32 rounding (summation order differs).  Sums of four or more
 * trajectories and nf_adjoint are unaffected.  Errors: NF_ERR_ARG (not matrix-free, unknown
 * value). */
enum { NF_MF_AUTO = 0, NF_MF_SYMMETRIC = 1, NF_MF_PACKED = 2, NF_MF_SYMMETRIC_512 = 3, NF_MF_SYMMETRIC_1024 = 4 };
NF_API nf_status nf_operator_mf_schedule(nf_operator *op, int schedule);

/* Block-pair culling for the symmetric schedule (opt-in; off at creation).
 * A pair of node blocks whose bounding boxes lie so far apart that the wider Gaussian
 * has an exponent above 160 (base 2) for every node pair in it contributes exactly zero in
 * FP32 (the exponential flushes to 0 below 2^-126), so it is skipped: the kernel runs over
 * the remaining block pairs only, and each node adds its block's live partial sums in the
 * same order as the full sum.  Results are bit-identical to the unculled sum; narrow
 * kernels on large domains (the Gauss(1/40) kernel of §4.3-4.4 on the 2 pi square) skip
 * almost every pair.  The distance bound respects the kernel's period.
 *   enable       1 to build the live-pair lists (host work over all block pairs; copies
 *                the coordinates to the host and synchronises `stream`), 0 to switch off
 *   live_pairs, block_pairs   host int64 outputs (may be NULL): live and total block pairs
 * nf_adjoint culls its adjoint pass as well (lists built from both Gaussians, so that the
 * A2 and s2 gradients stay exact); gradients are bit-identical to the unculled ones.  Sums
 * of four or more trajectories and the packed schedule do not cull.
 * Errors: NF_ERR_ARG (not matrix-free), NF_ERR_NOMEM/NF_ERR_CUDA. */
NF_API nf_status nf_operator_mf_cull(nf_operator *op, int enable, int64_t *live_pairs, int64_t *block_pairs,
                                     void *stream);

/* Failure-path self-test (no paper counterpart): launches a one-warp kernel whose
 * mbarrier wait can never complete, with a short poll limit.  The wait gives up, the
 * kernel records a timeout and returns; the call synchronises `stream` and returns
 * NF_ERR_TIMEOUT (anything else means the bounded-wait machinery is broken).  The CUDA
 * context stays usable afterwards. */
NF_API nf_status nf_selftest_timeout(void *stream);

/* Instruction-rate probe (no paper counterpart; it measures the denominators of the
 * pair kernels' roofline).  One CTA of 1,024 threads per SM runs independent chains of
 *   kind 0: fma.rn.f32        (1 FP32 FMA-pipe lane operation per instruction)
 *   kind 1: fma.rn.f32x2      (2 lane operations per instruction)
 *   kind 2: ex2.approx.ftz.f32 (1 SFU operation)
 *   kind 3: fma.rn.f32x2 as a 4 x 2 outer product (8 accumulators, a different pair of
 *           operand registers in every instruction, as in a register-tiled GEMM)
 * `iters` times 64 per thread, timed by each SM's cycle counter.  Host outputs: the median
 * over SMs of operations per clock per SM, the SM clock (MHz) implied by the slowest SM's
 * cycles over the launch's wall time, and that wall time in ms.  Synchronises `stream`;
 * allocates a few bytes stream-ordered.  Errors: NF_ERR_ARG, NF_ERR_CUDA. */
NF_API nf_status nf_probe_pipe(int kind, int64_t iters, double *ops_per_clk_sm, double *sm_mhz, float *ms,
                               void *stream);

/* Nonlocal sum of Eq. (2.9) for B trajectories:
 *     I[b, i] = sum_j w(|x_i - x_j|) q_j f_b(u[b, j]).
 *   u      B x n  FP32   states (trajectory-major)
 *   beta, theta   B FP32 device arrays
 *   I      B x n  FP32   output
 * Errors: NF_ERR_ARG, NF_ERR_CUDA. */
NF_API nf_status nf_nonlocal_apply(nf_operator *op, const float *u, int B, const float *beta,
                            const float *theta, float *I, void *stream);

/* Allocation-free nonlocal sum for one trajectory (the paper has no counterpart: this
 * is a deployment convenience).  For callers that cannot allocate device memory when
 * they need the sum -- e.g. inside a host framework that owns all allocations, or a
 * fixed-budget loop where a cudaMalloc would synchronise the device -- it computes
 *     I[i] = sum_j w(|x_i - x_j|) q_j f(u[j])
 * without an operator handle and without allocating.  It runs the row-block x column-
 * split pair kernel over ordered pairs with two exponentials per pair (not the
 * operator's symmetric or packed kernels, which need per-operator set-up), so it is
 * slower per pair than nf_nonlocal_apply on a matrix-free operator.  Its working memory
 * is a fixed file-scope device array of about 2.6 MB, held by every GPU that loads the
 * library until the process exits.
 *   x  n x 3 FP32, q n FP32, u n FP32, I n FP32 (output): caller-owned device memory.
 *   n  1 .. 32768 (larger n returns NF_ERR_ARG: the scratch size is fixed).  The pair
 *      kernel uses at most 16 column splits, which is what the array holds.
 * The first call on a device looks up the array's device address (with that device
 * current); make that first call before any stream capture.  All calls share the
 * array: each call rewrites what it reads, but calls whose work overlaps on the GPU
 * race and must be serialised by the caller.  Returns after enqueuing on `stream`.
 * A bounded device wait that gives up (NF_ERR_TIMEOUT, reported by nf_noalloc_status)
 * makes the call write NaN to every entry of I instead of an incomplete sum.
 * Errors: NF_ERR_ARG, NF_ERR_CUDA. */
NF_API nf_status nf_nonlocal_apply_noalloc(const float *x, const float *q, int64_t n, nf_kernel kp,
                                           const float *u, float beta, float theta, float *I, void *stream);

/* Status of the most recent nf_nonlocal_apply_noalloc on this device (no paper
 * counterpart): synchronises `stream`, then reads the scratch array's error flag.
 * NF_OK, or NF_ERR_TIMEOUT when a bounded wait in that call gave up (its I is NaN).
 * Allocates nothing. */
NF_API nf_status nf_noalloc_status(void *stream);

/* Limits of nf_nonlocal_apply_noalloc (no paper counterpart), host outputs: the largest
 * n it accepts, the most column splits its scratch holds, and the splits a call on n
 * nodes uses on the current device (always <= max_splits).  Errors: NF_ERR_ARG. */
NF_API nf_status nf_noalloc_limits(int64_t n, int64_t *max_n, int *max_splits, int *splits);

/* Failure-path self-test of the allocation-free call (no paper counterpart): records a
 * timeout in the scratch array's flag, as a pair-kernel block that gave up waiting
 * would, then runs the call's final reduction on n entries of I.  Afterwards every
 * entry of I is NaN and nf_noalloc_status returns NF_ERR_TIMEOUT; the next
 * nf_nonlocal_apply_noalloc clears the flag.  No kernel waits or faults.
 * Errors: NF_ERR_ARG, NF_ERR_CUDA. */
NF_API nf_status nf_selftest_noalloc_flag(int64_t n, float *I, void *stream);

/* Forcing gamma(t) of Eq. (2.9).
 *  NF_FORCE_NONE: gamma = 0.
 *  NF_FORCE_MMS_EIGEN: the manufactured-solution technique of §4 Eq. (4.5) with two
 *    eigenfunctions of the integral operator, W Y1 = lam1 Y1, W Y2 = lam2 Y2, W 1 = lam0:
 *      z = c + a(t) (Y1 + Y2),  a(t) = a0 cos t,  u* = theta + ln(z / (1 - z)) / beta,
 *      gamma = d(u*)/dt + u* - [lam0 c + a(t) (lam1 Y1 + lam2 Y2)],
 *    so that f(u*) = z solves the continuous problem exactly.  Y1, Y2: n FP32 device. */
/*  NF_FORCE_MMS_FLAT: the manufactured solution of the convergence study on the square,
 *    §4.3 (and, with scale = r, on the torus of §4.4 in its (phi, theta) coordinates), on
 *    the operator's periodic square (kernel period L > 0; nodes' x, y are the square's
 *    coordinates):
 *      z = G(x, x0(t); sigma) + c,  x0(t) = radius (cos t, sin t),
 *      G(x, y; s) = exp(-dist^2(x, y) / (2 s^2)) / (2 pi s^2),  u* = theta + ln(z / (1 - z)) / beta,
 *      gamma = d(u*)/dt + u* - scale * int_cell w(dist(x, y)) z(t, y) dy,
 *    the integral in closed form (w and G are products of one-dimensional Gaussians; each
 *    factor splits where the nearest image of x0 changes and integrates with erf).
 *    Fields used: c, radius, sigma, scale; Y1, Y2 unused. */
/*  NF_FORCE_MMS_SPHERE: the NF_FORCE_MMS_EIGEN form on the unit sphere with the library
 *    supplying what the caller would: Y1 = z/2 and Y2 = x y at the operator's nodes, and the
 *    eigenvalues lam0, lam1, lam2 of the operator's kernel (nf_mms_sphere_eigs).  Fields
 *    used: c, a0 (0 < c -+ 1.5 |a0| < 1, so that z stays in (0, 1)).  Euclidean (chord)
 *    distance only; nf_adjoint refuses it (the eigenvalues depend on the kernel). */
enum { NF_FORCE_NONE = 0, NF_FORCE_MMS_EIGEN = 1, NF_FORCE_MMS_FLAT = 2, NF_FORCE_MMS_SPHERE = 3 };
typedef struct {
    int kind;
    const float *Y1;
    const float *Y2;
    double c, a0, lam0, lam1, lam2;
    double radius, sigma, scale;
} nf_forcing;

/* Funk-Hecke eigenvalues lam_l, l = 0, 1, 2, of the kernel w on the unit sphere
 * (int_{S^2} w(|x - y|) Y_l(y) dS(y) = lam_l Y_l(x)), in closed form; host output
 * lam[3].  For the manufactured forcing on the sphere (Y1 = z/2, Y2 = x y). */
NF_API nf_status nf_mms_sphere_eigs(nf_kernel kp, double *lam);

/* Classical RK4 on Eq. (2.9), nsteps steps of size dt from t0, in place:
 *     k_s = -U_s + I(U_s) + gamma(t_s),   u <- u + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 *   u      B x n FP32  in/out
 *   beta, theta  B FP32 device
 *   g      host pointer to nf_forcing, or NULL
 *   ckpt   ((nsteps / C) + 1) x B x n FP32 device, or NULL: receives u at steps
 *          0, C, 2C, ... (checkpoints for nf_adjoint)
 * The step sequence is captured once in a CUDA graph and replayed.
 * Errors: NF_ERR_ARG, NF_ERR_CUDA; a non-finite state is recorded on the operator and
 * reported as NF_ERR_NONFINITE by nf_operator_check. */
NF_API nf_status nf_rk4_advance(nf_operator *op, float *u, int B, double t0, double dt, int nsteps,
                         const float *beta, const float *theta, const nf_forcing *g,
                         float *ckpt, int C, void *stream);

/* The models of §5, on any single operator path.
 *   kind NF_MODEL_FIELD:      du/dt = -u + sum_j w_ij mu_j f(u_j)          (Eq. (2.9), no forcing)
 *   kind NF_MODEL_DEPRESSION: du/dt = -u + sum_j w_ij mu_j s_j f(u_j),
 *                             tau ds/dt = 1 - s - beta_d s f(u)          (Eq. (nfsyndep); s is the
 *                             synaptic efficacy, 0 depleted .. 1 available)
 *   rate NF_RATE_SIGMOID:     f(u) = 1 / (1 + exp(-beta_b (u - theta_b)))  (per trajectory)
 *   rate NF_RATE_SMOOTHSTEP:  f = 0 below a, 1 from b on, between them the degree-9
 *                             polynomial that is C^4 at both ends (Eq. (smoothf); the
 *                             paper's labyrinth example uses a = 0.06, b = 0.54)
 * The paper's examples integrate with Adams-Bashforth 5. */
enum { NF_MODEL_FIELD = 0, NF_MODEL_DEPRESSION = 1 };
enum { NF_RATE_SIGMOID = 0, NF_RATE_SMOOTHSTEP = 1 };
enum { NF_INTEGRATOR_RK4 = 0, NF_INTEGRATOR_AB5 = 1 };
typedef struct {
    int kind, rate;
    float a, b;          /* smooth-step transition interval */
    float tau, beta_d;   /* depression time constant and strength */
} nf_model;

/* Advance a §5 model nsteps steps of dt, in place:
 *   model       host pointer to nf_model
 *   integrator  NF_INTEGRATOR_RK4 (classical tableau, 4 nonlocal sums per step) or
 *               NF_INTEGRATOR_AB5 (y += dt (1901 F_n - 2774 F_{n-1} + 2616 F_{n-2}
 *               - 1274 F_{n-3} + 251 F_{n-4}) / 720, one nonlocal sum per step; the paper
 *               does not say how to start it, and the first four steps are RK4 steps whose
 *               first-stage derivatives seed the history)
 *   u           B x n FP32 device, in/out
 *   s           B x n FP32 device, in/out, efficacy (NF_MODEL_DEPRESSION), else NULL
 *   beta, theta B FP32 device (used by the sigmoid rate)
 * The operator must be a single (not grouped) operator; its W (with mu) is reused
 * unchanged.  Allocates stage and history buffers on `stream` for the call.
 * Errors: NF_ERR_ARG, NF_ERR_NOMEM, NF_ERR_CUDA. */
NF_API nf_status nf_field_advance(nf_operator *op, const nf_model *model, int integrator, float *u, float *s, int B,
                                  double dt, int nsteps, const float *beta, const float *theta, void *stream);

/* Discrete adjoint of nf_rk4_advance for a terminal loss L(u_N):
 *   lambda_T  B x n FP32   dL/du_N
 *   ckpt      checkpoints written by nf_rk4_advance with the same arguments
 *   grad_u0   B x n FP32   output dL/du_0
 *   grad_kernel B x 4 FP32 output dL/d(A1, s1, A2, s2), per trajectory
 * Stages are recomputed segment by segment from the checkpoints, on an internal stream
 * forked from `stream` and joined back into it before the call returns (the work stays
 * ordered on `stream`; scratch memory is allocated stream-ordered on it and released at
 * the end, so the call is not for use inside a stream capture).  The transposed pair
 * sum uses the symmetry of the radial kernel (W^T = W).  A manufactured forcing on the
 * sphere enters as given (its eigenvalues are inputs, not functions of the kernel
 * parameters here).
 * Errors: NF_ERR_ARG, NF_ERR_UNSUPPORTED (dense operators; the flat manufactured forcing,
 * which depends on the kernel parameters), NF_ERR_CUDA. */
NF_API nf_status nf_adjoint(nf_operator *op, const float *ckpt, int C, int B, double t0, double dt,
                     int nsteps, const float *beta, const float *theta, const nf_forcing *g,
                     const float *lambda_T, float *grad_u0, float *grad_kernel, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NF_H */
