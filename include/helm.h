/*
 * helm.h -- C ABI of the GB300 finite-difference Poisson-iteration solver for the
 * Dirichlet-cavity Helmholtz problem.
 *
 * Problem (Section 2.2, the cavity problem Eq. (2.4) with damping p = 0 and a wall that
 * is Dirichlet everywhere; discretised as in Section 2.4):
 *
 *     (Delta_h + k^2) u = f on the n^D interior nodes of a cube of side (n+1) h,
 *     u = g on the wall nodes,
 *
 * with Delta_h the 5-point (D = 2) / 7-point (D = 3) second-order Laplacian.  The solver
 * runs the paper's recasting of Helmholtz as a sequence of Poisson problems (Eq. (1.4)
 * and the cavity iteration Eq. (2.6)-(2.8) with alpha = k^2): each outer step solves
 *
 *     Delta_h e_n = r_n := f - (Delta_h + k^2) u_n,   e_n = 0 on the wall,
 *     u_{n+1} = u_n + e_n,
 *
 * which is Delta_h u_{n+1} = f - k^2 u_n; with exact inner solves e_n = v_n + i w_n of the
 * paper and u_N is the N-th partial sum of its series.  The inner Poisson solve is
 * geometric multigrid (red-black Gauss-Seidel, full weighting, multilinear
 * prolongation, exact coarsest solve), run in complex64 (HELM_PREC_MIXED: FP32 V-cycles,
 * FP64 residual and solution, i.e. iterative refinement) or complex128 (HELM_PREC_FP64).
 * The iteration converges iff k^2 < lambda_min(-Delta_h) (Section 2.4: the iteration
 * matrix is G = -k^2 Delta_h^{-1}, the series converges iff its spectral radius is < 1).
 *
 * Memory layouts (all device pointers, the caller owns them):
 *   complex128 = interleaved {re, im} doubles (the layout of torch.complex128);
 *   complex64  = interleaved {re, im} floats  (torch.complex64);
 *   an "interior" array holds n^D values, a "padded" array (n+2)^D values; index order
 *   [z][y][x] with x fastest; padded node (i, j[, l]) sits at x = i h.
 * Every pointer must be 16-byte aligned and device memory of the plan's device.
 *
 * Errors: every entry point returns a helm_status; nothing throws, exits or traps.
 * Negative values are errors (the call had no effect on caller memory unless stated),
 * non-negative values are outcomes of a solve.
 *
 * Threading: a plan / batch may be used by one host thread at a time.  All work runs on
 * the CUDA stream given at creation.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HELM_API __attribute__((visibility("default")))
#else
#define HELM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HELM_CONVERGED = 0,      /* relres <= tol                                        */
    HELM_OK = 0,
    HELM_MAXITER = 1,        /* max_outer steps without convergence                 */
    HELM_DIVERGED = 2,       /* relres > 1e4, or >= 20 steps, 10 non-decreasing and
                                at least twice the smallest relres so far            */
    HELM_EINVAL = -1,        /* bad argument (null / misaligned pointer, bad size)  */
    HELM_ENOMEM = -2,        /* device allocation failed / batch memory cap reached */
    HELM_ECUDA = -3,         /* a CUDA runtime call failed                          */
    HELM_ENONFINITE = -4,    /* NaN or Inf met in the residual                      */
    HELM_ETIMEOUT = -5,      /* a bounded wait ran out                              */
    HELM_EUNSUPPORTED = -6   /* valid request this build does not handle            */
} helm_status;

typedef enum { HELM_BC_DIRICHLET = 0 } helm_bc;
typedef enum { HELM_PREC_FP64 = 0, HELM_PREC_MIXED = 1 } helm_prec;

typedef struct helm_plan helm_plan;
typedef struct helm_batch helm_batch;

/* Human-readable name of a status code (static string, never NULL). */
HELM_API const char* helm_status_str(int status);

/* Text of the last CUDA error this library met on the calling thread ("" if none). */
HELM_API const char* helm_last_error(void);

/* Number of CUDA kernel launches this library has issued from the calling process
 * (graph replays count every kernel node they run).  Used to report launch counts. */
HELM_API uint64_t helm_launch_count(void);

/* Diagnostic: compares, on `count` seeded random values, the integer-pipe binary64 ->
 * binary32 (round to nearest even) and binary32 -> binary64 conversions the complex64
 * residual path uses with the GPU's own conversions; *mismatches = disagreements outside
 * the binary32 subnormal range (which these conversions flush to zero).  Synchronous;
 * allocates 8 bytes of device memory for the count. */
HELM_API helm_status helm_selftest_conversions(int count, uint64_t seed, uint64_t* mismatches);

/* Diagnostic (no counterpart in the paper): the current device's FP64 FMA rate, the peak
 * the FP64 residual kernels are measured against.  Every SM runs 8 blocks of 256
 * threads, each thread 8 independent chains of 4096 fused multiply-adds; *tflops = flops
 * (2 per FMA) / the best of five timed launches (*ms, CUDA events on the legacy default
 * stream, after one warm-up launch).  Synchronous; allocates and frees a small buffer. */
HELM_API helm_status helm_measure_fp64_rate(double* tflops, double* ms);

/*
 * Plan: one cavity geometry (D, n, h), wave number k and precision, with its multigrid
 * hierarchy and workspace allocated on the current CUDA device.
 *   ndim      2 or 3.
 *   n         ndim entries, all equal to 2^m - 1 with 1 <= m <= 15 (2D) / 11 (3D);
 *             unequal entries -> HELM_EUNSUPPORTED.
 *   h         grid spacing > 0 (the unit cube has h = 1/(n+1)).
 *   k         wave number >= 0 (any value is accepted; k >= k_max diverges).
 *   bc        HELM_BC_DIRICHLET.
 *   prec      HELM_PREC_FP64 or HELM_PREC_MIXED.
 *   cuda_stream  cudaStream_t (NULL = the legacy default stream).
 * On success *out owns device memory until helm_plan_destroy.
 */
HELM_API helm_status helm_plan_create(helm_plan** out, int ndim, const int* n, double h, double k,
                             int bc, int prec, void* cuda_stream);
HELM_API helm_status helm_plan_destroy(helm_plan* plan);

/* Closed forms of the plan (Section 2.4, Dirichlet case): lambda_min of -Delta_h; the
 * spectral radius rho of the iteration matrix G = -(alpha + i p)(Delta_h - sigma)^{-1},
 * sigma = alpha - k^2: rho = sqrt(alpha^2 + p^2) / (lambda_min + sigma) (= k^2 / lambda_min
 * for the default alpha = k^2, p = 0); k_max = the supremum of the k with rho < 1 at the
 * plan's alpha and p: sqrt(lambda_min + alpha - sqrt(alpha^2 + p^2)), which is
 * sqrt(lambda_min) when p = 0 (0 when no k qualifies); and the workspace bytes owned.
 * Any output pointer may be NULL. */
HELM_API helm_status helm_plan_info(const helm_plan* plan, double* lambda_min, double* k_max,
                           double* rho_pred, size_t* workspace_bytes);

/* General cavity iteration (Section 2.2, Eq. (2.4)-(2.8), Dirichlet wall): solve
 * Delta u + (i p + k^2) u = f with the shift alpha >= k^2 and damping p >= 0, i.e. every
 * outer step solves (Delta_h - sigma) e = r_N, sigma = alpha - k^2, with
 * r_N = f - (Delta_h + k^2 + i p) u_N.  A new plan has alpha = k^2, p = 0.  Applies to
 * the plan's later helm_solve / poisson_vcycle / helm_batch_submit calls (the V-cycle
 * then solves (Delta_h - sigma) e = rhs).  HELM_EINVAL for a NULL plan, a non-finite
 * value, p < 0 or alpha < k^2. */
HELM_API helm_status helm_plan_set_cavity(helm_plan* plan, double alpha, double p);

/* Mean exit time and the sufficient bound of the cavity iteration (Section 2.2): E solves
 * Delta_h E = -1 with E = 0 on the wall (Eq. (2.10), discretised as in Section 2.4; the
 * plan's geometry and precision, solved by the outer iteration with k = 0 to
 * relres <= tol in at most max_outer steps); k_*^C = sqrt(1 / max E - p) (Eq. (2.9), p the
 * plan's damping; 0 when 1 / max E <= p).  No alpha >= k^2 satisfies the convergence
 * condition of Section 2.2 above k_*^C.
 *   E_out   padded (n+2)^D complex128 (device, 16-byte aligned) or NULL: receives E
 *           (imaginary part 0, wall ring 0).
 *   e_max, k_star   (host, may be NULL).
 * Allocates a k = 0 plan and three (n+2)^D-sized buffers for the call; synchronous.
 * Returns the solve's status (HELM_CONVERGED when tol was reached) or an error. */
HELM_API helm_status helm_exit_time(helm_plan* plan, double tol, int max_outer, void* E_out,
                                    double* e_max, double* k_star);

/* Spectral radius of the iteration matrix G = -(alpha + i p)(Delta_h - sigma)^{-1}
 * (Section 2.4: the partial sums converge iff rho(G) < 1), measured by power iteration on
 * the GPU: v <- M^{-1} v / ||M^{-1} v|| with M = Delta_h - sigma (zero walls) applied as
 * `cycles` multigrid cycles of the plan's schedule from zero, in the plan's inner
 * precision, starting from the constant vector; rho = |alpha + i p| ||M^{-1} v||.
 * Stops when successive estimates agree to tol (relative) or after max_iters.
 *   rho, iters_done   (host, may be NULL).
 * Returns HELM_OK when converged, HELM_MAXITER otherwise, or an error.  Synchronous;
 * allocates a small reduction buffer.  (For this Dirichlet cavity rho has the closed form
 * of helm_plan_info; the measurement checks the operator the solver actually applies.) */
HELM_API helm_status helm_spectral_radius(helm_plan* plan, int max_iters, double tol, int cycles,
                                          double* rho, int* iters_done);

/* Shape of the plan's multigrid hierarchy (this project's inner solver; the paper leaves
 * the Poisson solver open, Section 3): *tail_n = the grid size from which one CTA per
 * instance runs every coarser level in shared memory; *exact_n = the size of the level
 * that is solved exactly in the sine basis instead of being cycled (complex64: 31 in 2D,
 * 15 in 3D; FP64: 15 in 2D; 0: every level down to n = 1 is cycled).  Either pointer may
 * be NULL; HELM_EINVAL on a NULL plan. */
HELM_API helm_status helm_plan_coarse(const helm_plan* plan, int* tail_n, int* exact_n);

/* Inner-solve schedule: V(nu1, nu2) cycles, `cycles` V-cycles per outer step.
 * Defaults: 2D (2, 2, 1), 3D (2, 2, 1).  nu1, nu2 in [0, 8] with nu1 + nu2 >= 1,
 * cycles in [1, 16]. */
HELM_API helm_status helm_plan_set_cycle(helm_plan* plan, int nu1, int nu2, int cycles);

/* Autotuner: solves the given problem (f, g, starting iterate u, tol, max_outer as in
 * helm_solve) with each candidate inner schedule -- V(1,0), V(0,1), V(0,2), V(0,3),
 * V(1,1), V(2,1), V(1,2), V(2,2), V(3,3) with one cycle per outer step, V(1,1) with
 * two -- times each converged solve on the plan's stream (best of two after a warm-up
 * run), keeps the fastest in the plan and reports it (outputs may be NULL).  Every
 * tuning solve starts from the given u, so a u that already solves the problem makes
 * the timings meaningless: pass the starting iterate of the solves to be tuned (zeros
 * for the paper's start).  u is restored to the starting iterate.  2D plans then time the
 * three tile-shape policies (helm_plan_set_tiles) with the chosen schedule and keep the
 * fastest, and 2D complex64 plans then the three coarse-level policies
 * (helm_plan_set_coarse_mode).  HELM_DIVERGED if no candidate converged (schedule unchanged).  Allocates one
 * temporary copy of u. */
HELM_API helm_status helm_plan_autotune(helm_plan* plan, const void* f, const void* g, void* u,
                                        double tol, int max_outer, int* nu1, int* nu2,
                                        int* cycles, double* best_ms);

/* Tile shape of the 2D fused multigrid level kernels (this project's tuning, no paper
 * counterpart): HELM_TILES_AUTO = 64 x 32 tiles, or 32 x 16 on levels up to 511 where
 * the large tiles would give fewer than two per SM; HELM_TILES_LARGE = 64 x 32 everywhere;
 * HELM_TILES_SMALL = 32 x 16 on every level up to 511.  The solutions agree to the
 * inner precision's rounding (each shape is its own kernel instantiation, whose FP32
 * arithmetic may round differently in the last bit).  helm_plan_autotune tries the three policies
 * with its chosen schedule (2D plans) and keeps the fastest; helm_plan_tiles reports it,
 * helm_batch_set_tiles applies a policy to every solve of a batch.  HELM_EINVAL for an
 * unknown policy; 3D plans ignore it. */
#define HELM_TILES_AUTO 0
#define HELM_TILES_LARGE 1
#define HELM_TILES_SMALL 2
HELM_API helm_status helm_plan_set_tiles(helm_plan* plan, int policy);
HELM_API helm_status helm_plan_tiles(const helm_plan* plan, int* policy);

/* Where the coarse levels of 2D complex64 V-cycles run (this project's scheduling, no paper
 * counterpart; the cycle's operations are the same either way).  HELM_COARSE_CTA: the
 * levels above 63 in the fused tile kernels, levels 63 and below (31 solved exactly) in one
 * CTA per solve.  HELM_COARSE_CLUSTER: for cycles without pre-smoothing (nu1 = 0, nu2 = 1
 * or 2) of solves with n >= 511, levels 255, 127, 63 and the exact level 31 in one launch of
 * an 8-CTA thread-block cluster per solve (row bands per CTA, rhs halos exchanged through
 * distributed shared memory), replacing four fused level launches and the one-CTA tail;
 * other schedules and sizes keep the CTA form; with it, level 1's ascent (prolongation and
 * sweeps) is formed inside the fused finest-level kernel of same-size solves instead of its
 * own launch (the lowest latency for a solve running alone; more work per outer step, which
 * costs throughput when several solves share the GPU).  HELM_COARSE_AUTO (default): the
 * cluster where it applies to every solve of the launch and all their clusters can be
 * resident at once (15 on a GB300); else the CTA form; also the CTA form when the device
 * cannot hold one cluster.  Level 1's ascent is fused as with HELM_COARSE_CLUSTER where the
 * launch is a critical path: a plan's own solve, or, in a batch step, the lane with the
 * longest predicted solve when it holds that solve alone; the other lanes keep its own
 * launch.
 * The results agree to the inner precision's rounding.  helm_plan_coarse_mode reports the
 * policy and, if cluster_used is not NULL, whether the plan's last built outer step used the
 * cluster (0 before its first solve).  helm_batch_set_coarse_mode applies a policy to every
 * solve of a batch.  HELM_EINVAL for an unknown mode. */
#define HELM_COARSE_AUTO 0
#define HELM_COARSE_CTA 1
#define HELM_COARSE_CLUSTER 2
HELM_API helm_status helm_plan_set_coarse_mode(helm_plan* plan, int mode);
HELM_API helm_status helm_plan_coarse_mode(const helm_plan* plan, int* mode, int* cluster_used);

/*
 * Solve (Delta_h + k^2) u = f, u = g on the wall, by the outer Poisson iteration
 * (with helm_plan_set_cavity: (Delta_h + k^2 + i p) u = f, inner operator Delta_h - sigma).
 *   f         interior complex128, n^D (device).
 *   g         padded complex128, (n+2)^D (device); only its wall ring is read.
 *   u         padded complex128, (n+2)^D (device).  In: the interior is the starting
 *             iterate u_0 (zeros = the paper's start).  Out: the last iterate u_iters,
 *             its wall ring overwritten with g.
 *   tol       stop when relres_N = ||r_N||_2 / ||b||_2 <= tol (interior 2-norms), where
 *             r_N = f - (Delta_h + k^2) u_N and b = f minus the wall values' share of the
 *             stencil (the right-hand side with the Dirichlet nodes eliminated, Section
 *             2.4).  With a zero starting interior r_0 = b and relres_0 = 1; a starting
 *             iterate from an earlier solve (resume) starts at its own, smaller relres.
 *             If b = 0 the denominator is ||r_0||.
 *   max_outer >= 0 outer steps at most.
 *   iters     (host, may be NULL) number of outer steps performed.
 *   res_hist  (host, may be NULL) relres_0 .. relres_iters (iters + 1 doubles; the
 *             caller provides max_outer + 1).
 * Returns HELM_CONVERGED / HELM_MAXITER / HELM_DIVERGED / HELM_ENONFINITE, or an error.
 * Synchronous: returns after the stream has finished the solve.
 */
HELM_API helm_status helm_solve(helm_plan* plan, const void* f, const void* g, void* u, double tol,
                       int max_outer, int* iters, double* res_hist);

/* As helm_solve, and also returns the increment sup-norms ||e_N||_inf, N = 0..iters-1
 * (Section 3 proposes truncating on the size of successive iterates).  einf_hist may
 * be NULL. */
HELM_API helm_status helm_solve_ex(helm_plan* plan, const void* f, const void* g, void* u, double tol,
                          int max_outer, int* iters, double* res_hist, double* einf_hist);

/*
 * One multigrid V(nu1, nu2)-cycle for Delta_h e = rhs with e = 0 on the wall, in the
 * plan's inner precision (complex64 for HELM_PREC_MIXED, complex128 for HELM_PREC_FP64).
 *   rhs  interior n^D (device), read.
 *   e    interior n^D (device), in: initial guess, out: after one cycle.
 * The inner solver of each outer step, exposed for standalone use.  Synchronous.
 */
HELM_API helm_status poisson_vcycle(helm_plan* plan, const void* rhs, void* e, int nu1, int nu2);

/*
 * poisson_vcycle without a plan and without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc -- code
 * running under another framework's memory manager that has reserved the device memory,
 * or a latency-critical loop that cannot take the implicit device synchronisation of
 * cudaMalloc / cudaFree.  It runs the same kernels as poisson_vcycle (same cycle, same
 * results) on one statically sized device array of 16 MiB that the library keeps on every
 * device that loads it, until the process exits (enough for 2D n <= 511 in complex64,
 * 2D n <= 255 in complex128, 3D n <= 63 in either precision).
 *   ndim, n, h, prec   as helm_plan_create (prec picks complex64 or complex128 arrays).
 *   rhs, e             as poisson_vcycle (interior n^D, 16-byte aligned, memory of the
 *                      current device or managed memory; HELM_EINVAL otherwise).
 *   cuda_stream        stream the work is enqueued on (NULL = legacy default stream).
 * Returns HELM_EUNSUPPORTED, doing nothing, when the grid's multigrid arrays would not fit
 * the 16 MiB array.  Asynchronous: the call copies nothing from host memory (its
 * descriptors travel as kernel arguments), so it returns once the work is enqueued, and
 * the result is in e once the stream reaches it.
 * The first call on a device (with that device current) looks up the array's device
 * address and raises the kernels' shared-memory limits; make that first call before any
 * stream capture.  Every call reuses the same array (it clears what it uses), so calls
 * that overlap on the GPU -- from two streams or two host threads -- race.
 */
HELM_API helm_status poisson_vcycle_noalloc(int ndim, int n, double h, int prec, const void* rhs,
                                            void* e, int nu1, int nu2, void* cuda_stream);

/*
 * Batch / serving: many independent solves of uneven size, dimension and k advanced
 * together, each outer step of all active instances in one launch per kernel.
 *   hbm_cap_bytes  device-memory cap for the instances' workspace (0 = no cap).
 * helm_batch_submit copies the plan's parameters (the plan may be destroyed after) and
 * reserves workspace; HELM_ENOMEM when the cap would be exceeded (retry after others
 * finish).  f, g, u follow helm_solve and must stay valid until the solve is polled done.
 * helm_batch_step runs up to `max_steps` outer steps (0 = until every active solve has
 * finished, as one CUDA-graph launch; a bounded chunk right after admissions or
 * retirements runs as direct launches, so admitting between chunks costs no re-capture).  helm_batch_poll reports a solve; once it returns done = 1 the result is in
 * u (synchronised), the histories are copied (res_hist may be NULL), and the instance's
 * workspace is released.
 */
HELM_API helm_status helm_batch_create(helm_batch** out, size_t hbm_cap_bytes, void* cuda_stream);
HELM_API helm_status helm_batch_destroy(helm_batch* batch);
HELM_API helm_status helm_batch_submit(helm_batch* batch, const helm_plan* plan, const void* f,
                              const void* g, void* u, double tol, int max_outer,
                              uint64_t* ticket);
/* As helm_batch_submit, with the geometry, k and precision given directly (no plan, so
 * no plan workspace is allocated): for a serving loop admitting many requests. */
HELM_API helm_status helm_batch_submit_geom(helm_batch* batch, int ndim, int n, double h, double k,
                                            int prec, const void* f, const void* g, void* u,
                                            double tol, int max_outer, uint64_t* ticket);
HELM_API helm_status helm_batch_step(helm_batch* batch, int max_steps);
/* Many submissions in one call (no paper counterpart: a serving loop admitting a burst of
 * requests): solve i is helm_batch_submit_geom(batch, ndim[i], n[i], h[i], k[i], prec,
 * f[i], g[i], u[i], tol, max_outer, &tickets[i]), in order.  Stops at the first solve the
 * memory cap refuses (HELM_ENOMEM) or an invalid one (its error); *admitted = the solves
 * submitted before it. */
HELM_API helm_status helm_batch_submit_many(helm_batch* batch, int count, const int* ndim, const int* n,
                                            const double* h, const double* k, int prec,
                                            const void* const* f, const void* const* g, void* const* u,
                                            double tol, int max_outer, uint64_t* tickets, int* admitted);
/* As helm_batch_poll for `count` tickets without the histories: done[i], and for the
 * finished ones status[i] and iters[i] (either array may be NULL).  release = 1: each
 * finished solve's record is released as by helm_batch_poll (its history discarded);
 * release = 0: nothing is released (helm_batch_poll then returns the history and releases
 * it).  HELM_EINVAL for an unknown ticket. */
HELM_API helm_status helm_batch_poll_many(helm_batch* batch, int count, const uint64_t* tickets, int release,
                                          int* done, int* status, int* iters);
/* Inner schedule (as helm_plan_set_cycle) used by every solve of the batch from the next
 * step on (the batch's solves share their launches, hence one schedule). */
HELM_API helm_status helm_batch_set_cycle(helm_batch* batch, int nu1, int nu2, int cycles);
/* As helm_batch_set_cycle for the solves of one kernel class only (dimension ndim and
 * precision prec): a batch mixing 2D and 3D solves can run each class with its own tuned
 * schedule (their launches are separate anyway).  helm_batch_set_cycle resets every class
 * to the batch-wide schedule.  No paper counterpart (scheduling). */
HELM_API helm_status helm_batch_set_cycle_class(helm_batch* batch, int ndim, int prec, int nu1, int nu2,
                                                int cycles);
HELM_API helm_status helm_batch_set_tiles(helm_batch* batch, int policy);
HELM_API helm_status helm_batch_set_coarse_mode(helm_batch* batch, int mode);
/* Solves of one kernel class (dimension, precision) and grid size share engines of their
 * own (every launch of an engine covers one size, so the size-specific fused kernels apply)
 * and are spread over `lanes` (1 .. HELM_MAX_LANES, default 4) of them, each with its own
 * launch stream: each submission joins the lane of its class and size with the least
 * predicted work (outer steps from the closed-form contraction and the
 * tolerance, times n^D), and helm_batch_step runs the lanes' step graphs concurrently on
 * streams of decreasing priority, the lane holding the longest predicted solve first, so
 * one lane's FP64 residual overlaps another lane's coarse multigrid levels and the critical
 * solve is scheduled ahead.  Applies to later submissions; results do not depend on the
 * lane.  HELM_EINVAL outside the range.
 * (The lane split is a scheduling choice of this library; the paper has no counterpart.) */
#define HELM_MAX_LANES 4
HELM_API helm_status helm_batch_set_lanes(helm_batch* batch, int lanes);
/* Also copy a submitted solve's result to host memory: host_u receives the padded u
 * ((n+2)^D complex128, the layout of the device u) once the solve has finished, before
 * helm_batch_poll reports it done.  When a helm_batch_step runs its lanes to completion
 * (max_steps = 0) the copy is queued on the solve's lane right behind its last step, so it
 * overlaps the lanes still running; otherwise, and always for pageable host memory (whose
 * copy would hold the other lanes' launches), it is made when the solve retires.  host_u
 * must stay valid until then.  HELM_EINVAL for an unknown or finished ticket, or a device
 * pointer. */
HELM_API helm_status helm_batch_set_host_result(helm_batch* batch, uint64_t ticket, void* host_u);

/* Submit a solve whose data are in host memory (the end-to-end entry point: a caller with
 * host arrays needs no device memory of its own).  f_host (n^D complex128) and g_host
 * ((n+2)^D complex128, the wall data on the ring) are read; u_host ((n+2)^D complex128)
 * receives the padded solution when the solve ends (as helm_batch_set_host_result).  The
 * batch allocates the solve's device copies with its workspace (counted against the memory
 * cap), uploads f and g on its own upload stream in submission order and starts the solve
 * from zero (the paper's start) once they are on the device, so a solve submitted first
 * runs while the later ones upload.  With page-locked host memory the copies are
 * asynchronous and the result goes to the host right behind the solve's last step; with
 * pageable memory each upload returns once its data are copied and the result is copied
 * when the solve retires.  The host arrays must stay valid until the solve is polled.
 * HELM_EINVAL for device or managed pointers, overlapping f / g with u, or the conditions of
 * helm_batch_submit; HELM_ENOMEM over the cap (nothing queued).  No paper counterpart. */
HELM_API helm_status helm_batch_submit_host(helm_batch* batch, const helm_plan* plan, const void* f_host,
                                            const void* g_host, void* u_host, double tol, int max_outer,
                                            uint64_t* ticket);
HELM_API helm_status helm_batch_poll(helm_batch* batch, uint64_t ticket, int* done, int* status,
                            int* iters, double* res_hist);
/*
 * Diagnostic twin of helm_batch_step: the same outer steps, each kernel launched on its
 * own (no graph) between CUDA events on the batch's stream, accumulating per kernel
 * kind k (0 smoothing half-sweep, 1 residual + restriction, 2 prolongation + correction,
 * 3 zeroing, 4 coarse-level tail, 5 Helmholtz residual + update + norm, 6 convergence
 * check, 7 fused 2D smoothing + residual + restriction, 8 fused 2D prolongation +
 * correction + smoothing, 9 the finest level's prolongation + correction + smoothing fused
 * with the Helmholtz residual + update + norm (2D complex64 batches of one size), 10 the
 * cluster tail (levels 255 ... 31 of 2D complex64 cycles in one 8-CTA cluster per solve),
 * 11 two descent steps (rhs restrictions) in one launch, 12 kind 9 with level 1's ascent
 * formed inside it too): launches[k], device milliseconds ms[k] and algorithmic bytes
 * bytes[k] (each datum a launch must read or write, counted once).  nkinds >= 13.
 */
HELM_API helm_status helm_batch_profile(helm_batch* batch, int max_steps, uint64_t* launches,
                                        double* ms, double* bytes, int nkinds);

/* Active (submitted, not yet polled done) solves and the workspace bytes they hold. */
HELM_API helm_status helm_batch_info(const helm_batch* batch, int* active, size_t* bytes_in_use);

/*
 * Annular problem (Section 2.3; the FD discussion of Section 2.4): the square
 * [-side/2, side/2]^2 with a square hole |x|, |y| <= hole, Dirichlet data g on the hole,
 * the Robin condition du/dn - i k u = q on the outer edge, Delta u + k^2 u = f inside.
 *
 * Grid: n intervals per axis (n a power of two, 16 <= n <= 16384), h = side / n, node
 * (i, j) at (-side/2 + i h, -side/2 + j h) stored at i (n + 1) + j.  Hole nodes: the closed
 * hole (their values are the data g); outer-edge nodes (i or j in {0, n}): the row is the
 * outward normal derivative as a one-sided difference towards the inward neighbour (the
 * mean of the two at a corner); other nodes: the 5-point Laplacian.  Solved by the
 * iteration of Section 2.3 (shift alpha >= k^2, default k^2) in residual form: FP64
 * residual and solution, inner solves by multigrid cycles in the plan's precision.
 * The hole must contain a node and stay clear of the outer edge and its first layer at
 * every multigrid level down to n = 8; otherwise create returns HELM_EINVAL.
 */
typedef struct helm_annulus helm_annulus;
HELM_API helm_status helm_annulus_create(helm_annulus** out, int n, double side, double hole, double k,
                                         int prec);
HELM_API helm_status helm_annulus_destroy(helm_annulus* plan);
/* Shift alpha >= k^2 of Section 2.3's iteration (HELM_EINVAL below k^2 or not finite). */
HELM_API helm_status helm_annulus_set_shift(helm_annulus* plan, double alpha);
/* Multigrid cycle per outer step, as helm_plan_set_cycle (default V(2,2), 1 cycle). */
HELM_API helm_status helm_annulus_set_cycle(helm_annulus* plan, int nu1, int nu2, int cycles);
/*
 * data: (n+1)^2 complex128 (device): f on the PDE nodes, q on the outer-edge nodes, g on the
 * hole nodes.  u: (n+1)^2 complex128 (device, output only): the solution, g on the hole.
 * The iteration starts from zero (with the hole data); res_hist (host, max_outer + 1
 * doubles, may be NULL) receives relres_N = ||r_N|| / ||r_0||; *iters the steps made.
 * Returns HELM_CONVERGED / HELM_MAXITER / HELM_DIVERGED / HELM_ENONFINITE (the cavity's
 * status rule), or an error.  Synchronous, on a stream of the plan that is ordered after
 * prior work on the legacy default stream; data and u must not overlap.
 */
HELM_API helm_status helm_annulus_solve(helm_annulus* plan, const void* data, void* u, double tol,
                                        int max_outer, int* iters, double* res_hist);
/*
 * Mean exit time E (Delta E = -c_tau, dE/dn = 0 on the outer edge) and expected local time
 * L (Delta L = 0, dL/dn = 1 on the outer edge), both zero on the hole (Section 2.3's
 * remarks), into E_out and L_out ((n+1)^2 doubles, device), each solved to relres tol; and
 * k_*^A = min over the PDE nodes of (-L + sqrt(L^2 + 4 E)) / (2 E) (host, may be NULL).
 * c_tau = 1 is Eq. (2.10)'s normalisation, 2 Section 3's.  Allocates a k = 0 plan of the
 * same geometry for the duration of the call.
 */
HELM_API helm_status helm_annulus_exit_times(helm_annulus* plan, double c_tau, double tol, int max_outer,
                                             void* E_out, void* L_out, double* kstar);
/*
 * Spectrum of the iteration matrix G = A_sigma^{-1} M of Section 2.4 (M = -alpha on the
 * PDE rows, +i k on the outer-edge rows; the partial sums converge iff rho(G) < 1), the
 * quantities of Section 2.4's figure, measured on the GPU with the plan's multigrid as
 * A_sigma^{-1} (`cycles` cycles of the plan's V(nu1, nu2) from zero per application, in the
 * plan's inner precision; 1 <= cycles <= 64).
 * helm_annulus_spectral_radius: power iteration x <- G x / ||G x|| from a seeded start;
 *   rho = ||G x|| for the unit x, lambda = x^H G x (the dominant eigenvalue, when it is
 *   unique in modulus).  Stops when two successive estimates of rho agree to tol
 *   (relative) twice in a row, or after max_iters.
 * helm_annulus_condition: the 2-norm condition number of G, cond = sigma_max / sigma_min.
 *   sigma_max by power iteration on G^H G: the adjoint solve uses that W A_sigma, W = 1 on
 *   PDE rows and -1/h on outer-edge rows, is symmetric apart from the corner rows (which no
 *   other row references), so A^{-T} = corners h, elsewhere W A^{-1} W^{-1} after moving
 *   the corners' couplings to the right-hand side.  sigma_min = 1 / sqrt(lambda_max(A^T D
 *   A)), D = |M|^{-2}, by Lanczos (stencil applications only, FP64).  Needs k > 0.
 *   iters_done: the larger of the two loops' counts.
 * Outputs (host) may be NULL.  Returns HELM_OK when converged, HELM_MAXITER when the
 * estimates still moved after max_iters (they are returned all the same), or an error.
 * Synchronous; allocates small reduction buffers (and four FP64 grids for the Lanczos
 * vectors) for the call.
 */
HELM_API helm_status helm_annulus_spectral_radius(helm_annulus* plan, int max_iters, double tol, int cycles,
                                                  double* rho, double* lambda_re, double* lambda_im,
                                                  int* iters_done);
HELM_API helm_status helm_annulus_condition(helm_annulus* plan, int max_iters, double tol, int cycles,
                                            double* sigma_max, double* sigma_min, double* cond,
                                            int* iters_done);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
