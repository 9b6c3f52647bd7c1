/*
 * stokesreg.h -- C ABI of libstokesreg: regularized Stokes single- and
 * double-layer sums on an overlapping-patch capsule surface, GB300 (sm_103a).
 *
 * Method: arXiv 2310.13908 (Agarwal & Biros), Sec. 3.3-3.4. For every target
 * x with regularization parameter delta_x, the library evaluates the
 * trapezoid-rule discretization (Eq. smoothint) of the regularized layer
 * potentials over the N quadrature nodes y of the surface:
 *
 *   single layer (Eq. regstokes):
 *     u(x) = 1/(8 pi mu) sum_y w_y [ f_y s1(r/delta)/r + (f_y . d) d s2(r/delta)/r^3 ]
 *   double layer (the regularized stresslet the paper cites in Sec. 1,
 *   Limitations (ii); the paper prints no formula):
 *     D(x) = 1/(8 pi) sum_y w_y (-6) (d . q_y)(d . n_y) d s3(r/delta)/r^5
 *
 *   d = x - y, r = |d|; s1, s2 as printed in Sec. 3.4;
 *   s3(p) = erf p - (2/9) p (8p^6 - 36p^4 + 6p^2 + 9) e^{-p^2}/sqrt(pi).
 *   At r = 0 the single layer takes the limit of Sec. 3.4,
 *   s1/r -> 16/(3 delta sqrt(pi)); the double layer's self term is zero.
 *
 * Conventions for every function below:
 *   - Arrays are row-major FP64: points and vector densities are [n][3].
 *   - All caller buffers stay owned by the caller and are not retained after
 *     the call returns -- except for asynchronous calls (non-NULL stream),
 *     whose buffers must stay valid until that stream has completed.
 *   - Functions return a status (SK_OK = 0 on success) and never throw; the
 *     message of the last failure is sk_last_error(ctx).
 *   - A context is not thread-safe: one host thread at a time.
 *   - Calls on one context share its device workspace and its cached
 *     operators' scratch, so its asynchronous calls must not overlap on the
 *     GPU: enqueue them on one stream (or order their streams with events).
 *     Growing the workspace synchronizes the device first.
 */
#ifndef STOKESREG_H
#define STOKESREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define SK_OK        0
#define SK_EINVAL    1  /* invalid argument (NULL pointer, negative size, delta <= 0, ...) */
#define SK_ENOMEM    2  /* device or pinned memory exhausted, or a fixed workspace too small */
#define SK_ECUDA     3  /* a CUDA runtime call failed */
#define SK_EBUSY     4  /* serving queue full; retry later */
#define SK_EAGAIN    5  /* result not ready yet */
#define SK_ETIMEOUT  6  /* a bounded device-side wait or a host poll ran out of time */
#define SK_ENOTIMPL  7  /* feature not available in this build */

/* ---- precision and memory-space selectors -------------------------------- */
#define SK_FP64   0  /* every pair in FP64 */
#define SK_FP32C  1  /* FP32 pairs, compensated (two-sum) accumulation per target,
                        FP64 series for pairs with r/delta < rho_T, FP64 final sum */
#define SK_HOST   0  /* all array arguments are host pointers */
#define SK_DEVICE 1  /* all array arguments are device pointers on the context's device */

/* ---- context (library infrastructure: the paper defines no API) --------- */
typedef struct sk_ctx sk_ctx;

/* Create a context on CUDA device `device`. workspace_bytes = 0 lets the
 * context grow its device workspace on demand; > 0 preallocates exactly
 * that much and never grows it (calls needing more return SK_ENOMEM).
 * The context owns two CUDA streams and its workspace: an evaluation runs
 * part of its preparation (the target sort) on the second stream, forked
 * from and joined back into the evaluation's stream by events, so the
 * caller's stream still orders all of the call's work. *out is set to NULL
 * on failure. The environment variable SK_SMALL_SORT_POINTS (an integer
 * 0..2^24, read here) sets the largest point set that is ordered by the
 * single-block sort (default 3072; 0: always the multi-block sort); results
 * do not depend on it. */
int sk_create(sk_ctx** out, int device, size_t workspace_bytes);

/* Release the context, its streams and workspace. NULL is ignored. */
void sk_destroy(sk_ctx* ctx);

/* Message of the most recent failure on ctx ("" if none). Valid until the
 * next call on ctx. ctx may be NULL (returns a creation-failure message). */
const char* sk_last_error(const sk_ctx* ctx);

/* Library version, e.g. 100 for 0.1.0. */
int sk_version(void);

/* Tuning knobs of the SK_FP32C path (defaults: rho_T = 0.5, rho_c = 5.0).
 *   rho_T: pairs with r/delta below it are evaluated in FP64 by power series
 *          (Sec. 3.4: s1/r and s2/r^3 are smooth at r = 0). 0 < rho_T <= 2.
 *   rho_c: pairs with r/delta at or above it use s1 = s2 = s3 = 1, the plain
 *          Stokeslet/stresslet. The omitted fraction of a pair's value is
 *          largest at r/delta = rho_c: at rho_c = 5 it is 1.2e-9 (s1) and
 *          5.6e-8 (s2) for the single layer, and 8.9e-7 (s3) for the double
 *          layer; at rho_c = 5.5 it is 4.9e-10 (s2) and 9.5e-9 (s3).
 *          rho_T < rho_c <= 8.
 * Returns SK_EINVAL outside those ranges. */
int sk_set_fp32c_thresholds(sk_ctx* ctx, double rho_T, double rho_c);

/* Counters of the most recent *_eval on ctx. Waits for that evaluation's
 * stream to complete before reading them. */
typedef struct {
  int64_t n_src_active;      /* sources with w != 0 (the N_s of the interaction count) */
  int64_t n_tgt;             /* targets */
  int64_t near_pairs;        /* pairs evaluated in FP64 by series (SK_FP32C) */
  int64_t overflow_targets;  /* targets rescanned because their group's near-pair list
                                overflowed (a group: the 64 or 128 targets of one warp) */
  int64_t kernel_launches;   /* CUDA kernels the evaluation launched */
  int32_t n_chunks;          /* source chunks per target block (split of the source sum) */
  int32_t precision;         /* SK_FP64 or SK_FP32C */
  double pair_ms;            /* device time of the pair kernel (profiling on), else -1; when
                                finish_fused, it includes the FP64 finish of the target blocks */
  double eval_ms;            /* device time of the whole evaluation (profiling on), else -1 */
  int32_t finish_fused;      /* SK_FP32C: 1 if the pair kernel finished the target blocks
                                itself (grids of >= 2 target blocks per SM), 0 if separate
                                finish kernels followed */
} sk_eval_stats;
int sk_last_eval_stats(const sk_ctx* ctx, sk_eval_stats* out);

/* Throughput ceilings measured on the context's device by three
 * microbenchmarks with fixed trip counts (about 0.1 s in all):
 *   ffma2_tflops     packed FP32 FMA (FFMA2) over full occupancy, 4 flops per
 *                    instruction and lane;
 *   dfma_tflops      FP64 FMA, 2 flops per FMA;
 *   far_pairs_per_s  the single-layer far-field pair (Sec. 3.4 kernel with
 *                    s1 = s2 = 1) as the FP32C pair kernel runs it for large
 *                    problems (two f32x2 target pairs per lane, two CTAs per
 *                    SM), with sources in shared memory: the ceiling of the
 *                    pair loop without global traffic, near/far tests or
 *                    compensated merges.
 * Blocks until done; runs on the context's stream. SK_EINVAL for NULL
 * arguments, SK_ECUDA if a launch fails. */
typedef struct {
  double ffma2_tflops;
  double dfma_tflops;
  double far_pairs_per_s;
  int32_t sm_count;
} sk_peaks;
int sk_probe_peaks(sk_ctx* ctx, sk_peaks* out);

/* Profiling: enable = 1 records CUDA events on the evaluation's stream around
 * the pair kernel and around the whole evaluation (see sk_eval_stats). */
int sk_set_profiling(sk_ctx* ctx, int enable);

/* Regularized single layer (Sec. 3.4, Eq. regstokes; Sec. 3.3, Eq. smoothint).
 *   n_src    number of quadrature nodes N (>= 0; at most 2^30, and at most 2^25
 *            in SK_FP32C, whose near-pair lists hold source indices in 25 bits)
 *   src_xyz  [n_src][3] node positions y
 *   src_w    [n_src]    quadrature weights w = psi W h^2 (zero weights allowed)
 *   f        [n_src][3] density (traction) f at the nodes
 *   n_tgt    number of targets M (>= 0; 0 is a no-op)
 *   tgt_xyz  [n_tgt][3] targets x (nodes themselves and/or off-surface points)
 *   delta    [n_delta]  regularization parameter per target (n_delta = n_tgt)
 *                       or one global value (n_delta = 1); every delta > 0
 *   mu       viscosity > 0
 *   u_out    [n_tgt][3] result, FP64 in both precisions
 *   cuda_stream  NULL: the call is synchronous (returns after u_out is written);
 *                otherwise a cudaStream_t on the context's device: the work is
 *                enqueued on it and the call returns without waiting.
 * Targets may coincide with nodes; r = 0 takes the limit above. With n_src = 0
 * or all weights zero, u_out is zero. Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA,
 * SK_ETIMEOUT (a bounded device wait expired; u_out is then unspecified). */
int stokes_sl_eval(sk_ctx* ctx, int precision, int mem,
                   int64_t n_src, const double* src_xyz, const double* src_w, const double* f,
                   int64_t n_tgt, const double* tgt_xyz,
                   const double* delta, int64_t n_delta,
                   double mu, double* u_out, void* cuda_stream);

/* Regularized double layer (stresslet), same conventions as stokes_sl_eval:
 * the sum D(x) of the file header, the regularized stresslet that the paper
 * cites in Sec. 1, Limitations (ii), with the smoothing factor s3.
 *   src_n  [n_src][3] unit normals n at the nodes (orientation sets the sign)
 *   q      [n_src][3] double-layer density q
 * No viscosity argument: the stresslet is viscosity-free. For a constant q on
 * a closed surface with outward normals the result is q inside, 0 outside and
 * q/2 on the surface. */
int stokes_dl_eval(sk_ctx* ctx, int precision, int mem,
                   int64_t n_src, const double* src_xyz, const double* src_w,
                   const double* src_n, const double* q,
                   int64_t n_tgt, const double* tgt_xyz,
                   const double* delta, int64_t n_delta,
                   double* u_out, void* cuda_stream);

/* ---- capsule time stepping ----------------------------------------------
 *
 * A capsule keeps the N = 6 (m-1)^2 surface nodes of an m-th order grid
 * resident on the device and advances them with explicit Euler steps of
 * dx/dt = u_inf(x) + S[f](x) (Sec. 3.6, Eq. bi_combined): every step
 * evaluates the regularized single layer at all nodes (targets = sources)
 * and adds the background flow. Nodes are ordered patch-major, then by the
 * u index j, then by the v index k (Sec. 3.2, Eq. grid). Without a
 * membrane the quadrature weights w = psi W h^2 stay those given at creation;
 * after capsule_set_membrane every step recomputes them from the current
 * tangents (overset finite differences, Sec. 3.5) and f = NULL selects the
 * Skalak membrane force. One step is captured once into a CUDA graph and
 * replayed. */
typedef struct sk_capsule sk_capsule;

#define SK_FLOW_NONE       0  /* u_inf = 0 */
#define SK_FLOW_SHEAR      1  /* u_inf = (rate y, 0, 0)                  (Eq. shear_flow) */
#define SK_FLOW_POISEUILLE 2  /* u_inf = (alpha (R0^2 - y^2 - z^2), 0, 0) (Eq. poiseuille_flow) */

typedef struct {
  int32_t kind;
  double rate;   /* shear rate */
  double alpha;  /* Poiseuille curvature */
  double R0;     /* Poiseuille radius */
} sk_flow;

/* Create a capsule on ctx from host arrays (copied).
 *   m      grid order (>= 3); X is [6 (m-1)^2][3], w is [6 (m-1)^2]
 *   delta  NULL: delta = delta* recomputed on the device before every step
 *          (largest distance from a node to its grid neighbours on its patch,
 *          per patch, Eq. regparam with C = 1); otherwise [n_delta] fixed
 *          values, n_delta in {1, N}
 *   mu     viscosity > 0; precision SK_FP64 or SK_FP32C (at most 2^30
 *          nodes, SK_FP32C at most 2^25, as for stokes_sl_eval).
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int capsule_create(sk_ctx* ctx, sk_capsule** out, int m, const double* X, const double* w,
                   const double* delta, int64_t n_delta, double mu, int precision);

/* Advance n_steps >= 0 Euler steps of size dt > 0 in the background flow
 * (flow NULL: none) with the interfacial force density f [N][3] (host, held
 * fixed over these steps). f = NULL: the Skalak membrane force
 * f = div_gamma Lambda of the current shape, recomputed every step (Sec. 2.1,
 * Eqs. tensor and intf); needs capsule_set_membrane, else SK_ENOTIMPL.
 * Synchronous. Errors: SK_EINVAL, SK_ENOTIMPL, SK_ENOMEM, SK_ECUDA, SK_ETIMEOUT. */
int capsule_step(sk_capsule* c, int n_steps, double dt, const sk_flow* flow, const double* f);

/* Adaptive Runge-Kutta-Fehlberg 4(5) integration (Sec. 3.6) of
 * dx/dt = u_inf(x) + S[f](x) from now over a time t_end > 0. Every stage
 * recomputes what capsule_step does per step (membrane force and weights
 * when a membrane is set and f is NULL, delta* when created with
 * delta = NULL). The fourth-order solution is propagated; a step is accepted
 * when max |x5 - x4| / max |x4| <= tol, and the next trial step is
 * dt min(5, max(0.2, 0.9 (tol / err)^(1/5))); the last step lands on t_end.
 *   dt_inout   first trial step in (> 0), the suggested next step out
 *   f          as for capsule_step (host [N][3], or NULL for the membrane)
 *   max_steps  bound on accepted + rejected steps (SK_EAGAIN if t_end is
 *              not reached; the nodes hold the last accepted state)
 *   stats_out  NULL or [2]: accepted, rejected steps
 * Synchronous (one device-to-host read of two numbers per step).
 * Errors: SK_EINVAL (also for a non-finite step), SK_ENOTIMPL, SK_EAGAIN,
 * SK_ENOMEM, SK_ECUDA, SK_ETIMEOUT. */
int capsule_integrate_rkf45(sk_capsule* c, double t_end, double* dt_inout, double tol,
                            const sk_flow* flow, const double* f, int64_t max_steps,
                            int64_t* stats_out);

/* Give the capsule a Skalak membrane (Sec. 2.1, Eq. tensor): stress-free
 * reference nodes X_ref [N][3] (host, same grid order as X; copied), shear
 * modulus Es >= 0 and dilatation modulus ED >= 0. Reference tangents come
 * from the derivative scheme of Sec. 3.5. From now on every step updates the
 * quadrature weights, and capsule_step(f = NULL) uses the membrane force.
 * Needs m >= 6. Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int capsule_set_membrane(sk_capsule* c, const double* X_ref, double Es, double ED);

/* Evaluate the single layer of every step on the four-times upsampled grid
 * (Sec. 3.4, "Upsampling"; factor 4, as stokes_sl_eval_upsampled; W from the derivative scheme at
 * the current nodes; delta_u per patch replaces delta) or on the nodes
 * themselves (factor 1, the default). Needs m >= 6 for factor 4, and at
 * most 2^30 fine nodes (6 (4m - 1)^2), in SK_FP32C at most 2^25.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int capsule_set_upsampling(sk_capsule* c, int factor);

/* Area A = sum psi W h^2 and enclosed volume V = sum psi W h^2 x n_x (the
 * divergence-theorem form of Sec. 4.1) of the current nodes, with W and n
 * from the derivative scheme of Sec. 3.5. Needs m >= 6. Synchronous.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int capsule_area_volume(sk_capsule* c, double* area, double* volume);

/* Shape moments of the current nodes (Sec. 4.2, Table convg_full): out[14]
 * = area A, volume V, centroid c (3), moment of inertia tensor about the
 * centroid J = int_V (|x - c|^2 I - (x - c)(x - c)^T) (3 x 3, row-major).
 * Volume integrals by the divergence theorem (int_V x_i = 1/4 int x_i x.n,
 * int_V x_i x_j = 1/5 int x_i x_j x.n) with W and n from the derivative
 * scheme and the POU quadrature. Needs m >= 6. Synchronous.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int capsule_shape_moments(sk_capsule* c, double* out);

/* Copy the current node positions [N][3] to host memory, in the node order of
 * capsule_create (patch, then u index, then v index; Sec. 3.2, Eq. grid). */
int capsule_get(sk_capsule* c, double* X_out);

/* Release the capsule. NULL is ignored. */
void capsule_destroy(sk_capsule* c);

/* ---- surface derivatives and the membrane force ------------------------
 *
 * The overset finite-difference scheme of Sec. 3.5 on the six-patch grid of
 * order m (6 <= m <= 4097; N = 6 (m-1)^2 nodes in the capsule's order): patch
 * extension to three ghost layers (Eq. ext) with tensor-product not-a-knot
 * cubic splines, 7-point central differences (Eq. fdm) and blending with the
 * transition-map Jacobians (Eqs. blendu / blendv). FP64 throughout. The
 * operator depends only on m and is built on first use and kept in ctx.
 * mem selects host or device pointers; stream as for stokes_sl_eval (device
 * memory with a stream: asynchronous, buffers must stay valid until it
 * completes). The spline slope solves stage their grid lines in shared memory
 * when they fit (m <= 342); SK_SLOPE_STAGING=0 in the environment when the
 * operator is built keeps them in global memory (same arithmetic, same
 * results). */

/* u- and v-derivatives of n_fields functions g [N][n_fields] on the surface
 * (values at the nodes; each node's derivatives are in its own patch's (u, v))
 * into g_u, g_v [N][n_fields]. Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int surface_derivatives(sk_ctx* ctx, int m, int mem, int64_t n_fields, const double* g,
                        double* g_u, double* g_v, void* cuda_stream);

/* Skalak membrane force f = div_gamma Lambda (Sec. 2.1, Eqs. tensor and
 * intf; formulas of the Appendix) at nodes X [N][3] with stress-free
 * reference X_ref [N][3], shear modulus Es >= 0, dilatation modulus ED >= 0,
 * into f_out [N][3]; w_out [N] (may be NULL) receives the quadrature weights
 * psi W h^2 of X (Sec. 3.3, Eq. smoothint). Errors: SK_EINVAL, SK_ENOMEM,
 * SK_ECUDA. */
int membrane_force(sk_ctx* ctx, int m, int mem, const double* X, const double* X_ref, double Es,
                   double ED, double* f_out, double* w_out, void* cuda_stream);

/* Single layer on the four-times upsampled grid (Sec. 3.4, "Upsampling"):
 * node positions X [N][3], area elements W [N] (e.g. from the derivative
 * scheme) and densities f [N][3] of the m-th order grid are interpolated by
 * each patch's tensor-product not-a-knot cubic spline to the 4m-th order
 * grid (6 (4m-1)^2 nodes); the fine weights are psi_u W_u h_u^2 (h_u =
 * pi / (4m)) and delta is Eq. regparam (C = 1) on the fine grid, per patch.
 * The regularized sum (Eq. regstokes, viscosity mu) over the fine nodes is
 * evaluated at the m-th order nodes, which are fine nodes, so downsampling
 * there is the identity. u_out [N][3]. 6 <= m <= 4097. Errors as for
 * stokes_sl_eval. */
int stokes_sl_eval_upsampled(sk_ctx* ctx, int precision, int mem, int m, const double* X,
                             const double* W, const double* f, double mu, double* u_out,
                             void* cuda_stream);

/* Single layer by the single-level kernel-independent FMM of Sec. 5.
 * precision: SK_FP64, or SK_FP32C (the neighbouring clusters through the
 * FP32-compensated pair sums of stokes_sl_eval, with FP64 near lists; the
 * equivalent sources in FP32; check potentials FP32, equivalent densities
 * FP64). Arguments otherwise as for stokes_sl_eval (sources with zero weight
 * are dropped), plus:
 *   k           clusters (1..65536), centers0 [k][3] their initial centres
 *               (host or device per mem), lloyd_iters >= 0 k-means steps
 *   p           equivalent/check points per cube edge (3..10; 6 p^2 - 12 p + 8
 *               points per cube)
 * Clusters get a cube (half width a), equivalent sources on the 1.05 a cube
 * and check points on the 2.95 a cube. Box against box (Sec. 5, step 3):
 * each target joins the box of its nearest final centre; a target box takes
 * a cluster's equivalent sources when it lies wholly outside the cluster's
 * check cube and at least 7 delta (its largest) from the cluster cube, else
 * the direct regularized sum over the cluster's points. Deterministic. The
 * SK_FP32C path synchronizes the stream once, to plan its work items on the
 * host, and returns after the result is complete.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA, SK_ETIMEOUT. */
int stokes_sl_eval_fmm(sk_ctx* ctx, int precision, int mem, int64_t n_src,
                       const double* src_xyz, const double* src_w, const double* f,
                       int64_t n_tgt, const double* tgt_xyz, const double* delta,
                       int64_t n_delta, double mu, int k, const double* centers0,
                       int lloyd_iters, int p, double* u_out, void* cuda_stream);

/* ---- serving: continuous batching of single-layer requests -------------
 *
 * A server keeps up to max_slots requests resident on the device and runs
 * one persistent kernel that takes work items (request, block of targets,
 * chunk of sources) from all resident requests. A request that arrives while
 * others run is admitted as soon as a slot and enough of the server's HBM
 * arena are free; its items then interleave with the running ones. Each
 * request is the SK_FP32C single layer of stokes_sl_eval (Sec. 3.4, Eq.
 * regstokes) with the context's thresholds, and for up to 131,072 targets
 * its result is bit-identical to stokes_sl_eval(ctx, SK_FP32C, ...) on the
 * same inputs, whatever else is in flight. Work item order inside a request
 * is fixed, so the mix cannot change a result.
 *
 * The server owns a host scheduler thread, four CUDA streams, an HBM arena,
 * a slot table and a mapped host page; it uses the context's device and
 * thresholds. One server per context at a time. serve_submit and serve_poll
 * may be called from any host thread. The server's arena is separate from the
 * context workspace; a standalone call on the same context that has to grow
 * the workspace synchronizes the device, and so waits until the persistent
 * kernel has run out of work and exited. */
typedef struct sk_server sk_server;

typedef struct {
  int32_t max_slots;         /* resident requests (1..256; default 32) */
  int32_t queue_capacity;    /* submitted, not yet admitted requests (default 4096) */
  size_t hbm_budget_bytes;   /* arena for resident requests (0: a quarter of free memory,
                                at most 16 GiB) */
  int64_t idle_exit_us;      /* the persistent kernel exits after this long without work
                                and is relaunched on demand (default 20000) */
  size_t host_staging_bytes; /* pinned host pool holding submitted inputs and results
                                (0: 512 MiB); a full pool makes serve_submit return
                                SK_EBUSY until results are polled */
} sk_serve_cfg;

typedef struct {
  int64_t n_src;             /* as in stokes_sl_eval (SK_FP32C: at most 2^25); host pointers,
                                copied by serve_submit */
  const double* src_xyz;
  const double* src_w;
  const double* f;
  int64_t n_tgt;
  const double* tgt_xyz;
  const double* delta;
  int64_t n_delta;
  double mu;
  /* A capsule request when capsule != NULL (the fields above are then
   * ignored): the server advances this resident capsule (capsule_create on
   * the server's context, SK_FP32C, not upsampled) by n_steps explicit Euler
   * steps of dt (Sec. 3.6, Eq. bi_combined) under the background flow (kind
   * SK_FLOW_NONE for none). Each step takes the Skalak force and weights at
   * the current nodes when the capsule has a membrane (capsule_set_membrane),
   * else its current f, and delta* when the capsule's delta is automatic, as
   * capsule_step does; each step's sum is served beside the other requests.
   * The capsule's state stays in device memory across requests; the result
   * (serve_poll's u_out) is its nodes [N][3] after the last step. One request
   * per capsule at a time (SK_EBUSY otherwise); do not step or destroy the
   * capsule while its request is pending. */
  sk_capsule* capsule;
  int32_t n_steps;
  double dt;
  sk_flow flow;
} sk_request;

typedef struct {
  double submit_us;          /* host clock, microseconds since serve_create */
  double admit_us;           /* slot and memory granted, preparation enqueued */
  double publish_us;         /* work items visible to the persistent kernel */
  double done_us;            /* last item finished (seen by the host) */
  double ready_us;           /* result copied back, serve_poll can return it */
  int64_t interactions;      /* n_tgt x sources with w != 0 */
  int32_t n_chunks;
  int32_t status;            /* SK_OK, SK_ETIMEOUT, ... */
} sk_req_stats;

/* Create a server on ctx. cfg may be NULL (defaults). Errors: SK_EINVAL,
 * SK_ENOMEM (arena), SK_ECUDA, SK_EBUSY (ctx already serves). */
int serve_create(sk_ctx* ctx, const sk_serve_cfg* cfg, sk_server** out);

/* Queue one request; its arrays are copied before the call returns, so the
 * caller may free them at once. *ticket identifies it for serve_poll.
 * Errors: SK_EINVAL (bad request), SK_EBUSY (queue full: retry later),
 * SK_ENOMEM (the request can never fit in the arena). */
int serve_submit(sk_server* srv, const sk_request* req, uint64_t* ticket);

/* Wait up to timeout_us (0: do not wait, < 0: wait forever) for a ticket.
 * SK_OK: u_out [n_tgt][3] (host) and *st (may be NULL) are filled and the
 * ticket is released. SK_EAGAIN: not ready yet. SK_EINVAL: unknown ticket.
 * A request that failed on the device returns its error code (e.g.
 * SK_ETIMEOUT) and releases the ticket. */
int serve_poll(sk_server* srv, uint64_t ticket, double* u_out, sk_req_stats* st,
               int64_t timeout_us);

/* Finish every queued and resident request, stop the persistent kernel and
 * free the server. Results that were never polled are discarded. */
void serve_destroy(sk_server* srv);

/* The single layer of stokes_sl_eval without any memory allocation. Library
 * infrastructure: the paper has no counterpart of this call; it is a service
 * for callers that cannot allocate.
 *
 * Who needs it: code that runs under a fixed device-memory budget owned by
 * a framework allocator, where a library's own cudaMalloc could fail or
 * fragment the pool; latency-critical loops, where cudaMalloc/cudaFree
 * would stall the device; and callers that cannot keep an sk_ctx. This
 * call creates no context or stream and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * It computes what stokes_sl_eval(ctx, SK_FP32C, SK_DEVICE, ...) computes,
 * with the default thresholds rho_T = 0.5, rho_c = 5, on the calling
 * thread's current CUDA device: bit for bit while the scratch holds the
 * context call's split of the source sum; otherwise the sum is split into
 * fewer chunks and the chunk merge may differ in the last bits (~1e-16).
 * All arrays are device pointers on that device, with the layout of
 * stokes_sl_eval; the caller owns them.
 *
 * Scratch: one static device array of 32 MiB inside the library, shared by
 * every call on a device. A GPU that loads the library's code holds it until
 * the process exits. Problems whose scratch does not fit -- roughly beyond
 * 40,000 targets with 40,000 nodes -- are rejected with SK_EINVAL before any
 * work is enqueued. The array keeps the last call's contents; each call
 * clears what has to start at zero. Calls that overlap on the GPU (on
 * different streams, or from different host threads) race on the array and
 * corrupt each other's results: serialize them.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for the life of the process; make
 * that first call before any stream capture on that device. A
 * cudaDeviceReset of that device reloads the library's device code and
 * leaves the cached address stale: do not call this function on a device
 * after resetting it.
 *
 * cuda_stream NULL: the call runs on the legacy default stream, waits for
 * completion and reports a device-side failure (SK_ETIMEOUT, SK_EINVAL for a
 * non-positive delta). Otherwise it is enqueued on that stream and returns
 * at once; device-side failures are then not reported.
 * Errors: SK_EINVAL (bad argument or too large), SK_ECUDA, SK_ETIMEOUT. */
int stokes_sl_eval_noalloc(int64_t n_src, const double* src_xyz, const double* src_w,
                           const double* f, int64_t n_tgt, const double* tgt_xyz,
                           const double* delta, int64_t n_delta, double mu, double* u_out,
                           void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* STOKESREG_H */
