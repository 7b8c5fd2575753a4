/*
 * sssp.h — C ABI of the GB300 spectral split-step Pade (SSSP) range marcher.
 *
 * The library advances the complex depth field u(r, z) of the wide-angle parabolic
 * equation  d_r u = i sqrt(d_z^2 + k^2) u  (Section 2, Eq. PDPE) range step by range
 * step with the [p/p] Pade propagator
 *     u(r + dr) = e^{i k0 dr} prod_j (1 + a_j X)(1 + b_j X)^{-1} u,
 *     X = (d_z^2 + k^2 - k0^2)/k0^2 = d_z^2/k0^2 + V(z),  V = n^2 - 1,
 * (Section 2; the product form equals the paper's sum form d0 + sum_j d_j/(1 + b_j X)).
 * Each (1 + b_j X)^{-1} is applied spectrally (Section 3): a DST-I (homogeneous
 * Dirichlet boundaries at z = 0 and z = H, Section 3.1) diagonalises d_z^2 with
 * eigenvalues lambda_m = -(pi m/(k0 H))^2, and a depth-dependent V is handled by the
 * Neumann series of Eq. (Neumann), one forward and one inverse DST-I per term.
 * Algorithm 1 is the per-step loop that pe_march runs on the GPU.
 *
 * Conventions
 *  - Grid: N interior points z_n = n H/(N+1), n = 1..N.  N + 1 must be a power of two
 *    in [8, 65536] for this build (up to 4096 the whole march runs in one CTA's shared
 *    memory; larger grids use a per-plan workspace of 4 (N+1) complex values in HBM).  Fields are N complex64 values stored as interleaved
 *    float pairs (re, im), index n-1 for z_n.
 *  - Every function returns a pe_status; PE_OK is 0.  On failure the plan (if any) keeps
 *    a message readable with pe_last_error().  No C++ exception crosses this boundary.
 *  - The library owns all device memory it allocates (in pe_plan_create and when
 *    profile / TL storage grows); pe_plan_destroy frees it.  Caller buffers are only
 *    read or written during the call (device copies are ordered on the plan's stream
 *    and complete before functions that return data to the host return).
 *  - A plan is not thread-safe.  All device work of a plan is ordered on its CUDA
 *    stream (the stream given at creation, NULL = legacy default stream).
 */
#ifndef SSSP_H_
#define SSSP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pe_plan pe_plan;

typedef enum {
  PE_OK = 0,
  PE_ERR_ARG = 1,               /* invalid argument or unsupported size                  */
  PE_ERR_CUDA = 2,              /* a CUDA runtime call failed (message holds the error)   */
  PE_ERR_OOM = 3,               /* device allocation failed                              */
  PE_ERR_NEUMANN_DIVERGED = 4,  /* a Neumann term grew to 1e4 x the first correction term */
  PE_ERR_TIMEOUT = 5,           /* a bounded device wait expired                         */
  PE_ERR_STATE = 6,             /* call out of order (e.g. march before set_field)        */
  PE_ERR_NUMERIC = 7            /* a non-finite value appeared in the march               */
} pe_status;

/* ABI revision; bumped when a signature changes. */
int pe_abi_version(void);

/*
 * Create a plan.  Section 2 (Pade [p/p] of exp(i sigma (sqrt(1+X) - 1)), sigma = k0 dr,
 * coefficients by Baker's linear system in FP64 on the host) and Section 3 (tables of
 * the isovelocity inverse 1/(1 + b_j lambda_m)).
 *   N             interior depth points; N + 1 a power of two in [8, 65536]
 *   H             depth of the guide [m], > 0
 *   k0            reference wavenumber omega/c0 [1/m], > 0
 *   dr            range step [m], > 0
 *   pade_order    p in [1, 8]
 *   neumann_terms maximum number of Neumann terms including m = 0 (0 or 1: V is ignored,
 *                 the isovelocity step of Section 3); at most 64
 *   neumann_tol   per-term stop: after term m >= 1 once ||t_m|| <= tol ||w_j||; >= 0
 *   cuda_stream   cudaStream_t to order all work on (NULL = legacy default stream)
 * Errors: PE_ERR_ARG (sizes/values), PE_ERR_OOM, PE_ERR_CUDA.  *out is NULL on error.
 */
pe_status pe_plan_create(pe_plan** out, int N, double H, double k0, double dr, int pade_order,
                         int neumann_terms, double neumann_tol, void* cuda_stream);

/*
 * Boundary conditions of Section 3.1: homogeneous Dirichlet (the DST-I, pe_plan_create's
 * default); periodic (the DFT; N grid points z_n = n H/N, n = 0..N-1, N a power of two in
 * [8, 4096]; eigenvalues -(2 pi l/(k0 H))^2 for the signed frequency l); homogeneous Neumann
 * (the DCT-I; N points z_n = n H/(N-1), n = 0..N-1 including both boundaries, N - 1 a power of
 * two in [4, 2048]; eigenvalues -(pi m/(k0 H))^2).  A Neumann plan marches the periodic
 * problem on [0, 2H] of the even extension of the field (an exact equivalence: d_z^2 + V
 * commutes with the reflection) and returns the N points of [0, H].  For a periodic plan
 * every "DST-I" of this header is the DFT; for a Neumann plan it is the DCT-I
 * C_m = x_0/2 + (-1)^m x_{N-1}/2 + sum_{n=1..N-2} x_n cos(pi n m/(N-1)); N values in and out.
 * pe_dst1_batch and the GEMM batch take Dirichlet plans only.
 */
enum { PE_BC_DIRICHLET = 0, PE_BC_PERIODIC = 1, PE_BC_NEUMANN = 2 };
pe_status pe_plan_create_bc(pe_plan** out, int N, double H, double k0, double dr, int pade_order, int neumann_terms,
                            double neumann_tol, int bc, void* cuda_stream);

/* Release every device and host resource of the plan (NULL is ignored). */
void pe_plan_destroy(pe_plan* plan);

/* Last error message of the plan ("" if none).  Valid until the next call on the plan. */
const char* pe_last_error(const pe_plan* plan);

/* Message of the last failed pe_plan_create in this process (it has no plan to hold it). */
const char* pe_create_error(void);

/*
 * Transmission-loss output (TL = -20 log10|u| + 10 log10(r / 1 m), dB).  During pe_march
 * a TL row of N floats is recorded after every global step number s (counted from the
 * last pe_set_field, 1-based) with s % tl_every == 0.  tl_every = 0 disables recording
 * (the default).  Clears the recorded rows.  Errors: PE_ERR_ARG if tl_every < 0.
 */
pe_status pe_set_output(pe_plan* plan, int tl_every);

/*
 * Set the field u(r, z_n), n = 1..N, at range r [m] (the starter, Section 3.2).
 *   u          N interleaved complex64 values (2N floats)
 *   on_device  0: u is host memory (copied before return); 1: u is device memory
 * Resets the step counter and the recorded TL rows.  Errors: PE_ERR_ARG (NULL u),
 * PE_ERR_CUDA.
 */
pe_status pe_set_field(pe_plan* plan, const float* u, int on_device, double r);

/*
 * Append a profile node: n^2(z_n), n = 1..N, in force from range `range` on.  A range
 * step [r, r + dr] uses V = n^2 - 1 of the last node whose range is <= r + dr/2, or the
 * first node if there is none (the step-midpoint reading of Section 4.2's range
 * dependence).  Node ranges must be non-decreasing.
 *   n2         N doubles (is_complex = 0), or N interleaved (re, im) pairs (is_complex = 1:
 *              the complex absorbing potential of Section 3.1; Im n^2 > 0 absorbs).
 *              n^2 is taken in FP64 because n^2 ~ 1: rounded to FP32 it would carry an
 *              absolute error ~6e-8, a fixed perturbation of the medium whose phase error
 *              grows with range; V = n^2 - 1 is formed in FP64 and only then rounded.
 *   on_device  0: host memory, 1: device memory
 * Real and complex nodes may be mixed (real nodes have Im n^2 = 0).
 * Errors: PE_ERR_ARG (NULL, decreasing range, non-finite values), PE_ERR_OOM, PE_ERR_CUDA.
 */
pe_status pe_set_profile(pe_plan* plan, const double* n2, int is_complex, double range, int on_device);

/*
 * Append `count` profile nodes at once: n2 holds count rows of N doubles (row-major),
 * ranges the count node ranges (host memory, non-decreasing).  Same rules as
 * pe_set_profile with is_complex = 0.
 */
pe_status pe_set_profiles(pe_plan* plan, const double* n2, const double* ranges, int count, int on_device);

/* Remove all profile nodes. */
pe_status pe_clear_profiles(pe_plan* plan);

/*
 * Enqueue `steps` range steps of Algorithm 1 on the plan's stream (asynchronous: errors
 * raised on the device are reported by the next pe_read_* / pe_sync).  steps >= 0.
 * Errors: PE_ERR_STATE (no field set; no profile set while neumann_terms > 1),
 * PE_ERR_ARG, PE_ERR_CUDA, PE_ERR_OOM (TL storage growth).
 */
pe_status pe_march(pe_plan* plan, int steps);

/*
 * Enqueue `steps` range steps for `count` plans at once: one kernel launch per distinct
 * grid size N + 1 (plans of equal size share one launch; each CTA marches one plan).
 * Every plan must satisfy pe_march's preconditions; the plans' own streams are ignored
 * and the work is ordered on the stream of plans[0].
 */
pe_status pe_march_batch(pe_plan** plans, int count, int steps);

/*
 * As pe_march_batch, but plan i advances steps[i] >= 0 steps (0: left untouched).  Plans of
 * equal size still share one launch; each CTA marches its own count.
 */
pe_status pe_march_batch_steps(pe_plan** plans, const int* steps, int count);

/*
 * Device bytes a plan of this size will hold (tables, state, `nodes` profile rows, `tl_rows`
 * TL rows, workspace for N + 1 > 4096): the unit of the serving loop's memory budget.
 * Host-only; no GPU needed.
 */
size_t pe_plan_bytes_estimate(int N, int pade_order, int nodes, long long tl_rows);

/* Wait for the plan's stream; returns a device-side error raised by an earlier march. */
pe_status pe_sync(pe_plan* plan);

/*
 * Read the field after the last march: N interleaved complex64 values including the
 * carrier e^{i k0 (r - r_set)} (Section 2, applied once in FP64 phase arithmetic).
 *   to_device 0: `out` is host memory; 1: device memory.  Synchronises the stream.
 */
pe_status pe_read_field(pe_plan* plan, float* out, int to_device);

/*
 * Copy the recorded TL rows (row i: N floats, row-major) into `out` (host memory,
 * capacity `cap` floats) and their ranges into `ranges` (may be NULL; capacity
 * cap / N doubles).  *n_rows receives the number of rows recorded.  With out = NULL only
 * *n_rows is set (size query).  Synchronises.
 * Errors: PE_ERR_ARG if cap is smaller than rows * N.
 */
pe_status pe_read_TL(pe_plan* plan, float* out, size_t cap, double* ranges, size_t* n_rows);

/*
 * Number of DST-I transforms of length N the plan's marches have executed so far (every
 * Neumann term costs one forward and, unless it is the last, one inverse transform;
 * Section 3 counts m + 1 transform pairs for the m-th term).  Synchronises the stream.
 */
pe_status pe_get_transform_count(pe_plan* plan, unsigned long long* count);

/*
 * One unnormalised DST-I of length N on the GPU (Section 3.1's transform, the kernel the
 * marcher uses for every transform): out_m = sum_{n=1..N} in_n sin(pi n m/(N+1)), m = 1..N.
 * in/out: N interleaved complex64 values, host (on_device = 0) or device memory
 * (on_device = 1).  Uses the plan's size and stream; synchronises when on_device = 0.
 */
pe_status pe_dst1(pe_plan* plan, const float* in, float* out, int on_device);

/*
 * `count` DST-I of length N at once (one CTA per field), in and out device memory holding
 * count x N interleaved complex64 values (row b = field b).  Asynchronous on the plan's
 * stream.  Section 3.1's transform, batched.
 */
pe_status pe_dst1_batch(pe_plan* plan, const float* in, float* out, int count);

/*
 * pe_dst1 for callers that cannot allocate device memory.  (The paper has no counterpart:
 * this is a deployment variant of the transform, not a step of the method.)
 *
 * Same result as pe_dst1 (unnormalised DST-I of N complex64 values, in and out in device
 * memory, ordered on `cuda_stream`, NULL = legacy default stream) but no plan and no
 * allocation: the staged input and the length-(N+1) result live in a fixed scratch array
 * compiled into the library.  It is meant for applications that reserve all GPU memory up
 * front and forbid later cudaMalloc calls, or that run inside a framework whose allocator
 * owns every device buffer.
 *   N  interior points; N + 1 a power of two in [8, 4096] (larger sizes: PE_ERR_ARG).
 * The first call on a device performs that device's set-up (array addresses, tables);
 * make it before any stream capture.  All calls share the scratch array, which keeps the
 * last call's contents: calls that overlap on the GPU race and must be ordered by the
 * caller.  Errors: PE_ERR_ARG (NULL pointers, unsupported N), PE_ERR_CUDA.
 */
pe_status pe_dst1_noalloc(const float* in, float* out, int N, void* cuda_stream);

/*
 * Which kernel marches a plan (no counterpart in the paper, which gives no implementation).
 *   PE_KERNEL_CTA      one CTA per solve, the field in that SM's shared memory (N + 1 <= 4096) or
 *                      in a per-plan global workspace (larger grids);
 *   PE_KERNEL_CLUSTER  one solve over a thread-block cluster of 8 or 16 CTAs (the cluster shape below),
 *                      every length-(N + 1) array in the cluster's distributed shared memory and
 *                      each DST-I of Section 3.1 as local FFTs plus one all-to-all exchange;
 *                      Dirichlet grids with N + 1 in [4096, 32768];
 *   PE_KERNEL_AUTO     (default) the cluster kernel for Dirichlet grids with N + 1 in
 *                      [4096, 32768] when the device holds such a cluster, else one CTA; for
 *                      N + 1 = 4096 in a batched march only while that size's solves fit on
 *                      the device as clusters at once (beyond that one CTA per solve gives
 *                      more throughput).
 * Both compute the same step; results agree to FP32 rounding, not bit for bit.
 * pe_plan_set_kernel fails with PE_ERR_ARG for a choice the plan or device cannot take.
 * pe_plan_get_kernel reports the kernel a march of the plan uses (PE_KERNEL_CTA or _CLUSTER).
 * pe_dst1 on a plan set to PE_KERNEL_CLUSTER runs the cluster transform.
 */
enum { PE_KERNEL_AUTO = 0, PE_KERNEL_CTA = 1, PE_KERNEL_CLUSTER = 2 };
pe_status pe_plan_set_kernel(pe_plan* plan, int kernel);
pe_status pe_plan_get_kernel(const pe_plan* plan, int* kernel);

/*
 * Shape of the cluster kernel (no counterpart in the paper): ncta CTAs per cluster — 8
 * (N + 1 = 4096 .. 16384) or 16 (N + 1 = 8192 .. 32768), 0 for the size's default — and how each
 * transform's all-to-all exchange moves the values between the CTAs: push = 1 by remote stores
 * before the cluster barrier, 0 by remote loads after it, -1 the size's default.  The defaults
 * are the shapes measured fastest for batches of 1 to 38 solves: 8 CTAs at N + 1 = 4096 and
 * 8192, 16 CTAs at 16384 and 32768, the exchange pulled.  The exchange mode does not
 * change the arithmetic (the results are bitwise the same); the cluster size changes how each
 * transform is split, so the results agree to FP32 rounding.  The shape applies whenever a march
 * of the plan runs the cluster kernel; batched marches group solves by it.  PE_ERR_ARG for a shape
 * the plan (Dirichlet grids with N + 1 in [4096, 32768]) or the device cannot take.
 * pe_plan_get_cluster_shape reports the shape a cluster march of the plan takes (ncta 0 and
 * push -1 for plans the cluster kernel does not take).
 */
pe_status pe_plan_set_cluster_shape(pe_plan* plan, int ncta, int push);
pe_status pe_plan_get_cluster_shape(const pe_plan* plan, int* ncta, int* push);

/*
 * Depth operator of a plan.  PE_OP_SPECTRAL (default): the paper's DST-I diagonalisation with the
 * continuous eigenvalues and the Neumann series for V (Section 3).  PE_OP_FD3: FD-SSP, the
 * comparison of Section 4.3 and the FD-SSP remark of Section 2 — the same product-form Pade
 * propagator with the standard 3-point finite difference for d_z^2 (our choice of stencil),
 * X = D2/k0^2 + V, each (1 + b_j X) w_j = y solved directly (tridiagonal; FP64 Thomas factors per
 * profile node on the host, the sweeps on the GPU); neumann_terms and neumann_tol are not used,
 * V is always applied and a profile is required.  FD-SSP takes Dirichlet grids with N + 1 in
 * [8, 4096] and real n^2.  Set the operator before the profile and the field (PE_ERR_STATE
 * otherwise).  pe_read_field / pe_read_TL / checkpoints work as for spectral plans.
 */
enum { PE_OP_SPECTRAL = 0, PE_OP_FD3 = 1 };
pe_status pe_plan_set_operator(pe_plan* plan, int op);

/*
 * Shape of the one-CTA shared-memory kernel (no counterpart in the paper): points per thread
 * P = 4, 8 (default; 0 means 8) or 16, i.e. L/P threads per solve, each transform a Stockham FFT
 * of radix-P passes.  4 and 16 take Dirichlet grids with N + 1 in [256, 4096]; PE_ERR_ARG
 * otherwise.  All shapes compute the same step (results agree to FP32 rounding).
 * pe_plan_get_shape reports the P a march of the plan runs (0 when it runs the cluster or the
 * large-grid kernel).
 */
pe_status pe_plan_set_shape(pe_plan* plan, int points_per_thread);
pe_status pe_plan_get_shape(const pe_plan* plan, int* points_per_thread);

/*
 * Shape autotuners (no counterpart in the paper).  pe_march_batch_autotune times `steps` range
 * steps of the batched march of `plans` (pe_march_batch) with each shape the plans can take —
 * one CTA per solve at 4, 8 and 16 points per thread, and one thread-block cluster per solve in
 * each cluster shape (pe_plan_set_cluster_shape) —
 * a warm-up run then a timed run each, restores every plan's state and TL bookkeeping after each
 * run, and sets the fastest shape on every plan that can take it; it then measures every plan's
 * DST-I count per step on that shape (one more run, restored), and later batched marches launch
 * each group's solves in descending cost (heavy and light solves share SMs; the results do not
 * depend on the order).  ms: PE_AUTOTUNE_SHAPES floats, the timed milliseconds of (CTA P=4,
 * CTA P=8, CTA P=16, 8-CTA cluster pulling, 8-CTA cluster pushing, 16-CTA cluster pulling, 16-CTA
 * cluster pushing), -1 where no plan can take the shape, or NULL; kernel / points_per_thread: the
 * shape chosen (pe_plan_get_cluster_shape gives the cluster shape set),
 * or NULL.  pe_plan_autotune_shapes is the
 * same for one plan.  Plans need a field (and a profile when Neumann terms are asked for);
 * synchronises.
 */
enum { PE_AUTOTUNE_SHAPES = 7 };
pe_status pe_march_batch_autotune(pe_plan** plans, int count, int steps, float* ms, int* kernel,
                                  int* points_per_thread);
pe_status pe_plan_autotune_shapes(pe_plan* plan, int steps, float* ms, int* kernel, int* points_per_thread);

/*
 * Autotuner (no counterpart in the paper): times `steps` range steps of the plan's own march on
 * each kernel it can take (one CTA; the cluster where supported), a warm-up run then a timed
 * run each, restores the marcher's state and TL bookkeeping after every run (pe_save_state /
 * pe_load_state), and sets the faster kernel on the plan.  ms: 2 floats, the timed milliseconds
 * of PE_KERNEL_CTA and PE_KERNEL_CLUSTER (-1 where not a candidate), or NULL; chosen: the kernel
 * set, or NULL.  Needs a field (and a profile when Neumann terms are asked for); synchronises.
 */
pe_status pe_plan_autotune(pe_plan* plan, int steps, float* ms, int* chosen);

/*
 * Checkpoint / resume of a march (bit-exact).  The state is the marcher's own variables: the
 * unnormalised transform coefficients of the envelope and its depth-domain copy, L complex
 * values each (L = N + 1 Dirichlet, N periodic, 2 (N - 1) Neumann), interleaved re/im, 4 L
 * floats in all (pe_state_size gives the count), plus the range of the starter and the steps
 * marched since.  Loading it into a plan of the same parameters (pe_load_state makes no check
 * that they agree) and marching on gives the same bits as never stopping.  Host memory; both
 * calls synchronise.  TL rows are not part of the state: a loaded plan records from its
 * next step.
 */
size_t pe_state_size(const pe_plan* plan);
pe_status pe_save_state(pe_plan* plan, float* state, double* r_set, long long* steps);
pe_status pe_load_state(pe_plan* plan, const float* state, double r_set, long long steps);

/*
 * Host FP64 bound on the Neumann series of Eq. (Neumann) for profile node `node`:
 * rho_j = max|V| max_m |b_j / (1 + b_j lambda_m)| for every Pade term j (the 2-norm of
 * b_j L_j^{-1} V, since the transform is orthogonal).  rho < 1 guarantees convergence; the
 * operator is not normal, so a bound above 1 is a warning, not a divergence (the march reports
 * PE_ERR_NEUMANN_DIVERGED only on an actual blow-up).  rho: pade_order doubles.
 */
pe_status pe_neumann_bound(pe_plan* plan, int node, double* rho);

/*
 * Fault injection for tests of the error path (no GPU fault is involved): writes `status`
 * (e.g. 4 = diverged, 7 = non-finite) into the plan's device status word with a copy, as a
 * failing march would; the next pe_sync / pe_read_* reports it.
 */
pe_status pe_inject_status(pe_plan* plan, int status);

/* Current range of the field and number of steps marched since pe_set_field. */
pe_status pe_get_range(const pe_plan* plan, double* r, long long* steps);

/*
 * Host-only: the [p/p] Pade data the plan uses for sigma = k0 dr (Section 2), in FP64:
 * b[2p] and a[2p] interleaved complex (Q = prod (1 + b_j X), P = prod (1 + a_j X)),
 * d[2p + 2] = (d0, d_1..d_p) of the sum form.  Runs without a GPU.
 */
pe_status pe_pade_coefficients(double sigma, int p, double* b, double* a, double* d);

/* ------------------------------------------------------------------------------------
 * Tensor-core GEMM-DST (a precision variant for batches of one small grid size).  Every
 * transform of the march (Section 3's DST-I, applied to all fields of the batch at once) is
 * the dense product S X with S[m][n] = sin(pi n m/(N+1)), computed by a library GEMM in the
 * given precision with FP32 accumulation; the rest of the step is the FFT marcher's arithmetic.
 * All plans must share N, Pade order, neumann_terms (>= 2; a fixed count of terms is taken)
 * and dr, have a field set and exactly one profile node.  The batch copies the plans' spectral
 * states at creation and marches its own copy (the plans are not advanced).
 * ------------------------------------------------------------------------------------ */
enum { PE_GEMM_FP32 = 0, PE_GEMM_TF32 = 1, PE_GEMM_3XTF32 = 2, PE_GEMM_BF16X3 = 3 };
typedef struct pe_gemm_batch pe_gemm_batch;
pe_status pe_gemm_batch_create(pe_gemm_batch** out, pe_plan** plans, int count, int mode);
/* Enqueue `steps` range steps (one captured CUDA graph per step) on plans[0]'s stream. */
pe_status pe_gemm_batch_march(pe_gemm_batch* batch, int steps);
/* Field of member `index` (N interleaved complex64, host; carrier included).  Synchronises. */
pe_status pe_gemm_batch_read_field(pe_gemm_batch* batch, int index, float* out);
const char* pe_gemm_batch_error(const pe_gemm_batch* batch);
void pe_gemm_batch_destroy(pe_gemm_batch* batch);

/* ------------------------------------------------------------------------------------
 * Serving loop (continuous batching).  The paper marches one solve at a time; this is the
 * deployment form: many independent marches share the GPU.  Requests queue in arrival order;
 * each pe_server_step admits queued requests while a slot is free and their device bytes
 * (pe_plan_bytes_estimate) fit in the remaining budget, advances every live solve in one
 * batched march, and retires finished ones (field and TL rows copied to host memory, plan
 * freed).  Pacing: the costliest kind of live request (transforms per step x the work of a
 * transform, (1 + p (terms - 1)) (N + 1) log2(N + 1)) marches up to `chunk_steps` range steps per
 * pe_server_step and a cheaper one up to w times as many, w = the largest live cost over its own
 * cost rounded down, at most max_weight (64 by default; pe_server_set_pacing, 1 = every request
 * `chunk_steps`), so that small grids do not march at the pace of the largest.  A solve's result
 * is bit-identical to marching it alone.  The server is not thread-safe.
 * ------------------------------------------------------------------------------------ */
typedef struct pe_server pe_server;

typedef struct {
  int N;                 /* interior depth points (as pe_plan_create) */
  double H, k0, dr;
  int pade_order, neumann_terms;
  double neumann_tol;
  long long steps;       /* range steps to march */
  int tl_every;          /* TL row every tl_every steps (0: none) */
  const float* u0;       /* starter, N interleaved complex64, host; copied at submit */
  const double* n2;      /* nodes x N FP64 n^2 rows, host (NULL when neumann_terms <= 1) */
  const double* node_r;  /* node ranges, non-decreasing */
  int nodes;
  double r0;             /* range of the starter */
  int flags;             /* PE_ADMIT_* bits (0: march the request as given) */
} pe_request;

/*
 * Admission adaptations (no counterpart in the paper).  PE_ADMIT_MINIMAX_C0: the reference
 * sound speed c0 is chosen to minimise max|V| over the request's profile nodes (n^2 -> s n^2,
 * k0 -> k0/sqrt(s), s = 2/(min n^2 + max n^2); k0^2 n^2 is unchanged).  PE_ADMIT_CONVERGENT_ORDER:
 * the Pade order is chosen from the contraction rate rho_j of the Neumann operator
 * -b_j L_j^{-1} V of Eq. (Neumann) (the FP64 bound max|V| max_m |b_j/(1 + b_j lambda_m)|, else an
 * FP64 power-iteration estimate, for the node with the largest max|V|): for sigma = k0 dr < 10
 * the highest order with every rho_j <= 0.3 (there orders 7 and 8 leave a cut 12-term series
 * whose march grows without bound even with rho_j < 1), otherwise the highest order with every
 * rho_j < 0.98.  A request that diverges at every order fails at admission (state 3); a march
 * whose device status reports a failure after a chunk (non-finite value, diverging series) is
 * restarted from its starter one order lower (at most 8 times).  The starter is kept as given.
 */
enum { PE_ADMIT_MINIMAX_C0 = 1, PE_ADMIT_CONVERGENT_ORDER = 2 };

/*
 * Host-only (no GPU): the admission's FP64 power-iteration estimate of the spectral radius of
 * the Neumann operator -b L^{-1} V of Eq. (Neumann), L^{-1} = IDST diag(1/(1 + b lambda_m)) DST,
 * lambda_m = -(pi m/(k0 H))^2, for V at the N interior points (N + 1 a power of two) and one
 * Pade coefficient b = b_re + i b_im: the geometric mean growth of ||M^k x|| over k = 16..48 from
 * a fixed start vector.  PE_ERR_ARG on bad sizes.
 */
pe_status pe_neumann_radius_estimate(const double* V, int N, double H, double k0, double b_re, double b_im,
                                     double* rho);

/* hbm_budget_bytes > 0, max_live >= 1 concurrent solves, chunk_steps >= 1 steps per launch. */
pe_status pe_server_create(pe_server** out, size_t hbm_budget_bytes, int max_live, int chunk_steps, void* cuda_stream);
/* Pacing limit (see above): max_weight in [1, 4096]; PE_ERR_ARG otherwise. */
pe_status pe_server_set_pacing(pe_server* server, int max_weight);
void pe_server_destroy(pe_server* server);
const char* pe_server_error(const pe_server* server);
/* Queue a request (inputs copied); *id identifies it.  PE_ERR_OOM if it can never fit. */
pe_status pe_server_submit(pe_server* server, const pe_request* request, unsigned long long* id);
/* Admit, march every live solve one chunk, retire.  Outputs may be NULL.  Synchronises. */
pe_status pe_server_step(pe_server* server, int* live, int* queued, int* completed);
/* state: 0 queued, 1 running, 2 done, 3 failed. */
pe_status pe_server_state(pe_server* server, unsigned long long id, int* state);
/* Copy a finished request's field (2N floats) and TL rows (rows x N floats, capacity tl_cap)
 * and release it; with field = tl = NULL only *rows is set. */
pe_status pe_server_take(pe_server* server, unsigned long long id, float* field, float* tl, size_t tl_cap,
                         size_t* rows);
pe_status pe_server_stats(pe_server* server, size_t* bytes_in_use, size_t* peak_bytes, int* peak_live);
/* The values an admitted request marches with: k0, the factor s its n^2 rows were scaled by,
 * and its Pade order (each pointer may be NULL).  PE_ERR_STATE while it is still queued. */
pe_status pe_server_request_params(pe_server* server, unsigned long long id, double* k0, double* n2_scale,
                                   int* pade_order);
/* Withdraw a queued or running request (its plan is freed at once; state becomes 3, failed,
 * with the message "cancelled").  PE_ERR_STATE if it already finished. */
pe_status pe_server_cancel(pe_server* server, unsigned long long id);

#ifdef __cplusplus
}
#endif
#endif /* SSSP_H_ */
