/*
 * cpct.h -- C ABI of the GB300-native compressive phase-contrast tomography
 * library: the Fourier-slice Radon transform by gridding (non-uniform FFT),
 * its adjoint, the cubic ring-artifact filter and the SPGL1 basis-pursuit
 * solver that calls them.
 *
 * Paper: Maia et al., "Compressive Phase Contrast Tomography" (arXiv 1009.1380).
 *  - Section "fast radon transform": Radon{x} = 2D FFT of x on a regular grid,
 *    gridding interpolation onto a polar grid, 1D inverse FFT along each
 *    radial line; the adjoint runs the steps in reverse (gridding).
 *  - Section "Introduction", the L1 problem: min ||x||_1 subject to
 *    ||filter(Radon{x} - data)||_2 < eps, solved by SPGL1, which needs the
 *    operator y = Radon{x} and its adjoint.
 *
 * Conventions shared by every entry point (the paper fixes none of them):
 *  - image x: N x N float32, row-major, x[p*N + q]; row p is the y axis,
 *    column q the x axis; pixel centre at (p, q) = (N/2, N/2);
 *  - sinogram y: M x Ns float32, row-major, y[j*Ns + s]; angle theta_j,
 *    detector bin s with the rotation axis at s = Ns/2, pitch = pixel pitch;
 *  - default angles theta_j = pi j / M (from +x towards +y);
 *  - the real operator is R x = Re(A x) with A the complex Fourier-slice
 *    transform (unnormalised 2D DFT, centred ray inverse DFT scaled by 1/Ns);
 *    radon_adj computes R^T w = Re(A^H w), the exact adjoint up to rounding;
 *  - Kaiser-Bessel kernel, width 6, grid oversampling 2 (G = 2N).
 *
 * Ownership: every pointer argument named d_* is DEVICE memory owned by the
 * caller (CUDA runtime allocations, e.g. from PyTorch); h_* arguments are host
 * memory owned by the caller.  A plan owns its own device workspaces (the
 * oversampled spectrum, tables and bin lists) and frees them in
 * cpct_plan_destroy.  Device pointers to float data must be 16-byte aligned.
 *
 * Streams: every call is stream-ordered on the given stream (NULL = legacy
 * default stream) and asynchronous unless stated otherwise.  A plan holds
 * per-call workspaces and must not be used by two streams concurrently.
 *
 * Errors: every function returns CPCT_OK (0) or a negative cpct_status; an
 * argument error is detected on the host before anything is enqueued.
 * Asynchronous device-side failures (a bounded wait that expired) are
 * recorded in the plan and returned by the next cpct_plan_sync().
 */
#ifndef CPCT_H_
#define CPCT_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cpct_status {
  CPCT_OK = 0,
  CPCT_EINVAL = -1,       /* null pointer, bad size, unsupported geometry      */
  CPCT_ENOMEM = -2,       /* a device or host allocation failed                */
  CPCT_ECUDA = -3,        /* a CUDA runtime/driver call failed                 */
  CPCT_ETIMEOUT = -4,     /* a bounded device wait expired (kernel returned)   */
  CPCT_ENONFINITE = -5,   /* the solver met a NaN/Inf                          */
  CPCT_ENOTCONV = -6,     /* the solver hit its iteration cap                  */
  CPCT_EUNSUPPORTED = -7  /* feature not available (e.g. no sm_103a device)    */
} cpct_status;

/* Geometry of one slice.  Section "fast radon transform".
 *   n        image side N; power of two, 32 <= N <= 2048
 *   n_det    detector bins Ns; power of two, N <= Ns <= 4096
 *   n_views  number of projection angles M, 1 <= M <= 32768
 *   angles   host array of M angles in [0, pi) radians, or NULL for pi j / M
 *   kb_width kernel width W; only 6 is supported (0 selects 6)
 *   oversamp grid oversampling sigma; only 2.0 is supported (0 selects 2)
 *   flags    CPCT_PLAN_* bits                                               */
typedef struct cpct_geom {
  int n;
  int n_det;
  int n_views;
  const double* angles;
  int kb_width;
  double oversamp;
  int flags;
} cpct_geom;

/* plan flags */
#define CPCT_PLAN_FAIL_ALLOC 0x1000 /* testing: make the first device allocation fail */

typedef struct cpct_plan cpct_plan;

/* Create a plan: builds, on the device and in FP64, the Kaiser-Bessel kernel
 * approximation and deapodization vector and the FFT twiddle tables; builds
 * the tile bin lists of the polar samples (gridding, section "fast radon
 * transform": the sample plane is divided into bins with one thread block per
 * bin) and uploads them.  Synchronous on `stream`.  *out is NULL on failure. */
int cpct_plan_create(cpct_plan** out, const cpct_geom* g, cudaStream_t stream);

/* Free a plan and every workspace it owns.  NULL is accepted. */
int cpct_plan_destroy(cpct_plan* plan);

/* Wait for the plan's work on `stream` and report the first asynchronous
 * device-side error recorded since the previous call (CPCT_ETIMEOUT ...). */
int cpct_plan_sync(cpct_plan* plan, cudaStream_t stream);

/* Query plan sizes: image side, detector bins, views, oversampled grid G,
 * bytes of plan-owned device memory. Any output pointer may be NULL. */
int cpct_plan_info(const cpct_plan* plan, int* n, int* n_det, int* n_views,
                   int* grid, size_t* device_bytes);

/* Forward operator  y = Re(A x).  Section "fast radon transform": deapodize
 * and zero-pad, oversampled 2D FFT, Kaiser-Bessel interpolation onto the
 * polar grid, inverse FFT along each ray.
 *   d_img   device, N*N float32 (read)
 *   d_sino  device, M*Ns float32 (written)                                  */
int radon_fwd(cpct_plan* plan, const float* d_img, float* d_sino, cudaStream_t stream);

/* Adjoint operator  x = Re(A^H w) (the transpose of radon_fwd): FFT along each
 * ray, gridding (polar -> Cartesian convolution) as a deterministic
 * tile-binned gather, inverse 2D FFT, crop and deapodize.
 *   d_sino  device, M*Ns float32 (read)
 *   d_img   device, N*N float32 (written)                                   */
int radon_adj(cpct_plan* plan, const float* d_sino, float* d_img, cudaStream_t stream);

/* Complex operator pair.  Section "fast radon transform" builds the
 * projections from the polar samples of the image's Fourier transform; the
 * inverse FFT along each ray gives a complex sinogram y = A x, whose real
 * part is what radon_fwd returns.  For a real image the polar spectrum is
 * Hermitian in k, so y is real except for the Nyquist frequency k = -Ns/2,
 * which has no partner: Im y[j, s] = (1/Ns) Im(P[j, -Ns/2]) (-1)^(s - Ns/2).
 *   radon_fwd_c: y = A x,  d_img N*N float32 (read), d_sino_c M*Ns complex64
 *                (interleaved re, im; written);
 *   radon_adj_c: x = Re(A^H w),  d_sino_c M*Ns complex64 (read), d_img N*N
 *                float32 (written): the exact adjoint of radon_fwd_c for the
 *                real inner product Re<u, v> on complex sinograms (the image
 *                is real).  Re(w) takes radon_adj's path; Im(w) only reaches
 *                the Nyquist samples.
 * A complex image x = a + i b maps to A a + i A b (two radon_fwd_c calls),
 * and A^H w = Re(A^H w) + i Re(A^H (-i w)) (two radon_adj_c calls).  Same
 * alignment, stream and error rules as radon_fwd / radon_adj. */
int radon_fwd_c(cpct_plan* plan, const float* d_img, void* d_sino_c, cudaStream_t stream);
int radon_adj_c(cpct_plan* plan, const void* d_sino_c, float* d_img, cudaStream_t stream);

/* Filtered back-projection x = R^T(h * y): the ray spectra of the sinogram
 * are weighted by the ramp h[k] = (pi / M) |k| / Ns (the DC bin by (pi / M)
 * 0.25 / Ns, the mean of |k| over its width) before the adjoint, which
 * discretises the polar Fourier inversion integral with d(theta) = pi / M
 * (uniform angles over [0, pi)).  The paper's baseline reconstruction
 * ("using a filter", Fig. 3); here also the input of the learned warm
 * start.  Same arguments, layout and errors as radon_adj. */
int radon_fbp(cpct_plan* plan, const float* d_sino, float* d_img, cudaStream_t stream);

/* The finite-difference synthesis operator of the analysis-l1 variant.  The
 * paper puts the l1 norm on the phase-contrast image itself (a Laplacian of
 * the object, section "Introduction"); its Conclusions point to total
 * variation instead, i.e. l1 of the object's gradient.  The variant
 * puts it on the horizontal differences z of a piecewise-constant image u
 * through u = C z (prefix sums along every row: C inverts z[p, 0] = u[p, 0],
 * z[p, q] = u[p, q] - u[p, q - 1]).
 *   adjoint = 0: d_out = C d_in     (u[p, q] = sum_{q' <= q} z[p, q'])
 *   adjoint = 1: d_out = C^T d_in   (sum_{q' >= q} of every row)
 * d_in, d_out: device, n x n float32 row-major (row = y); in place allowed;
 * FP32 sums.  n <= 4096.  Stream-ordered, asynchronous.  CPCT_EINVAL for
 * null pointers, n out of range or adjoint not 0 / 1. */
int cpct_synth_dh(const float* d_in, float* d_out, int n, int adjoint, cudaStream_t stream);

/* Host-buffer variants: copy h_in (pinned or pageable host memory) to a
 * plan-owned device staging buffer, run the operator, copy the result back
 * to h_out and synchronize `stream`.  For end-to-end timing and for callers
 * without device memory. */
int radon_fwd_host(cpct_plan* plan, const float* h_img, float* h_sino, cudaStream_t stream);
int radon_adj_host(cpct_plan* plan, const float* h_sino, float* h_img, cudaStream_t stream);

/* The operator pair over `count` slices in host memory, pipelined (the
 * forward operator and its adjoint of section "fast radon transform",
 * applied slice by slice):
 *   h_sinos[i] = R h_imgs[i]   (radon_fwd: N x N in, M x Ns out)
 *   h_outs[i]  = R^H h_sinos[i] (radon_adj of the device-resident sinogram)
 * Two device buffer sets alternate: slice i + 1's image is copied in and
 * slice i - 1's results are copied out (on two copy streams) while slice
 * i's operators run; the sets' operators run on `stream` with `plan` and on
 * a second compute stream with a clone of `plan` (the same tables, its own
 * workspaces; if the clone cannot be made, both sets use `plan` on
 * `stream`).  The buffer sets (2 x (2 N^2 + M Ns) floats), the clone, the
 * streams and their events are made by the first call and kept in the plan
 * for later calls.  They are freed with the plan, or before a call that
 * changes the plan's configuration (cpct_plan_set_caps, _auto_caps,
 * _set_bins, _set_rounds, _tune).  The clone follows the plan's graph mode.
 * Host buffers are the
 * caller's; with pinned memory the copies overlap the kernels (pageable
 * memory works, without overlap).  Output buffers of different slices may
 * coincide (the copies into them are ordered).  Synchronous: returns once
 * every result is in host memory.  Calls on one plan must not overlap (they
 * share the kept buffers).  CPCT_EINVAL for null arguments or count < 1,
 * CPCT_ENOMEM if the two buffer sets cannot be allocated. */
int radon_pair_host_stream(cpct_plan* plan, const float* const* h_imgs, float* const* h_sinos,
                           float* const* h_outs, int count, cudaStream_t stream);

/* Preprocessing front end (section "Introduction", Fig. 1): the radiographs
 * taken with the detector near the sample and 1 m downstream are background
 * normalized, n = (I - D) / (F - D) (flat-field correction; 0 where the
 * reference F - D <= 0, a dead or saturated pixel), and subtracted; the
 * difference is the propagation-based phase-contrast image, and its rows
 * over all angles are the sinograms, one per detector row:
 *   sino_z[j, s] = n_near[j, z, s] - n_far[j, z, s].
 *   d_near, d_far            device, n_views x n_rows x n_det uint16 camera
 *                            frames (angle j, detector row z, column s)
 *   d_flat_near, d_flat_far  device, n_rows x n_det float32 open-beam frames
 *   d_dark                   device, n_rows x n_det float32 dark frame
 *   d_sinos                  device, n_rows x n_views x n_det float32 (slice
 *                            z's M x Ns sinogram at d_sinos + z M Ns), written
 * FP32 arithmetic (the reciprocal of each reference is formed once).
 * Stream-ordered, asynchronous (a small stream-ordered workspace of 2
 * n_rows n_det floats).  CPCT_EINVAL for null pointers or sizes < 1. */
int cpct_preprocess_pc(const uint16_t* d_near, const uint16_t* d_far, const float* d_flat_near,
                       const float* d_flat_far, const float* d_dark, int n_views, int n_rows, int n_det,
                       float* d_sinos, cudaStream_t stream);

/* ---- many slices: clones, autotuner, batches ----------------------------- */

/* A new plan for the same geometry as `src` that shares src's read-only
 * tables and bin lists (freed with the last plan using them) but owns its own
 * workspaces, so that it can run concurrently with src on another slice.
 * Synchronous on `stream`.  Cheap: no bin building. */
int cpct_plan_clone(const cpct_plan* src, cpct_plan** out, cudaStream_t stream);

/* Install the work items of a plan with the given caps: fwd_cap samples per
 * forward gather item, adj_cap conflict-free rounds per adjoint spread item
 * (0 keeps the current cap).  A new plan's caps are chosen from its
 * geometry and the GPU: about the work of one resident CTA per item when
 * the work is spread evenly (gather 256..4096 samples, spread 8..64
 * rounds), since a launch lasts at least as long as its longest item; a
 * new bin plan or round width takes its own automatic cap unless a cap was
 * fixed here.  The plan must not have clones yet.  Allocates the new item
 * lists; synchronous. */
int cpct_plan_set_caps(cpct_plan* plan, int fwd_cap, int adj_cap, cudaStream_t stream);

/* Install the automatic caps for `concurrent` slices applying the operator
 * at the same time (the batched solver's or a batch's slices): each slice
 * gets 1 / concurrent of the resident CTAs, so the items grow with the
 * concurrency (one slice alone is cut finest: its launch is bound by its
 * longest item; many at once are bound by their total work, which small
 * items raise by their partial tiles).  Clones made afterwards share the
 * items.  CPCT_EINVAL for concurrent < 1 or a plan with clones;
 * synchronous. */
int cpct_plan_auto_caps(cpct_plan* plan, int concurrent, cudaStream_t stream);

/* Bin plans (section "fast radon transform": the sample plane is divided
 * into bins, one thread block per bin, chosen by a quadtree that repeatedly
 * divides the bin of largest samples x grid points into four).  A bin is a
 * square of T x T points of the oversampled half spectrum, T = 16, 32 or 64;
 * a plan is a uniform tiling with one T (kind CPCT_BINS_UNIFORM, `tile` = T)
 * or that quadtree (kind CPCT_BINS_QUADTREE, leaves of 16..64 points; a bin
 * is split while its cost exceeds twice the mean cost of the non-empty
 * leaves).  which = 0: the forward gather (a sample belongs to the bin of
 * its footprint's first point), 1: the adjoint spread (a sample belongs to
 * every bin its 6x6 footprint touches).  cpct_plan_set_bins installs a plan
 * for one operator (keeping a cap fixed by cpct_plan_set_caps, else taking
 * the automatic cap of the new bins); the plan must not have clones;
 * synchronous.  The default is uniform 32 for both.  Results do not depend
 * on the bin plan beyond FP32 rounding (each bin sums its samples in its
 * own order); for a given plan they are bitwise reproducible.
 * Changing the bins of a plan that a captured batch (cpct_batch_create)
 * uses leaves that batch's graph with freed bin lists: install bin plans
 * (and caps) before building batches.
 * cpct_plan_bins reports the installed plans (kind, tile, 0 for a quadtree)
 * and, per operator, the number of bins of each size (16, 32, 64; host
 * arrays of 3, may be NULL). */
#define CPCT_BINS_UNIFORM 0
#define CPCT_BINS_QUADTREE 1
int cpct_plan_set_bins(cpct_plan* plan, int which, int kind, int tile, cudaStream_t stream);

/* Width of the adjoint spread's conflict-free rounds (default 32): every
 * half-warp holds at most one sample per 64-bit shared-memory bank class, so
 * each of its accumulator accesses is served in one pass.  16 uses the lower
 * half-warp only; 32 one warp (two samples per class); 64 two warps of one
 * work item (four per class; rounds of the larger tiles have room for 64
 * disjoint footprints).  CPCT_ROUNDS_COLUMNS selects column groups instead:
 * five samples per warp, six lanes per sample, one per footprint column,
 * each applying its column's six taps row after row; the five samples'
 * first cells follow a fixed bank pattern, so every half-warp access is
 * served in one pass, and each entry carries the sample's fractions and
 * accumulator coordinates (16 bytes per entry instead of 4).
 * cpct_plan_set_rounds re-packs the installed adjoint bins (with the
 * automatic cap unless cpct_plan_set_caps fixed one; the plan must not have
 * clones; synchronous);
 * cpct_plan_rounds returns the width (or CPCT_EINVAL for a NULL plan). */
#define CPCT_ROUNDS_COLUMNS 5
int cpct_plan_set_rounds(cpct_plan* plan, int lanes, cudaStream_t stream);
int cpct_plan_rounds(const cpct_plan* plan);

/* Graph replay of the operators.  The paper has no counterpart: this is a
 * launch mechanism of this library.  With enable = 1, radon_fwd, radon_adj,
 * their host-buffer variants and radon_pair_host_stream capture the kernels
 * of one application into a CUDA graph the first time they see a given
 * (operator, input address, output address, profiling mask) and replay that
 * graph on the caller's stream on later calls with the same addresses: the
 * same kernels with the same arguments, so the results are bit for bit those
 * of direct launches, without the per-kernel launch cost of the host.  At
 * most 8 graphs are kept per plan (least recently used dropped); changing the
 * bin plans, caps or round width drops them all.  A call made while the
 * caller's stream is being captured launches directly (into the caller's
 * graph).  The first call with new addresses captures and instantiates a
 * graph (host work of the order of 100 us); callers that pass new buffers on
 * every call should leave graph mode off (the default).  enable = 0 turns the
 * mode off and frees the graphs.  Returns CPCT_EINVAL for a NULL plan or an
 * enable other than 0 or 1.
 * cpct_plan_graphs returns the number of graphs held (CPCT_EINVAL for NULL). */
int cpct_plan_set_graphs(cpct_plan* plan, int enable);
int cpct_plan_graphs(const cpct_plan* plan);
int cpct_plan_bins(const cpct_plan* plan, int* fwd_kind, int* fwd_tile, int* adj_kind, int* adj_tile,
                   int* fwd_class_bins, int* adj_class_bins);

/* Work items of a plan: forward gather items, adjoint spread items, heavy
 * bins split over several spread items, and their partial-tile space in
 * units of 32 x 32 tiles (slots).  Host only; any output pointer may be
 * NULL. */
int cpct_plan_work(const cpct_plan* plan, int* n_fwd_items, int* n_adj_items, int* n_split, int* n_slots);

/* Autotuner of the bin plans and work-item sizes: for each operator times
 * the bin plans uniform 16, 32, 64 and the quadtree at the automatic cap,
 * keeps the fastest (for the adjoint then the fastest round width, 16, 32
 * or 64), then times its caps (the automatic one, 256..4096 samples per
 * gather item, 8..128 rounds per spread item) and keeps the fastest (median of `reps`
 * launches each, CUDA events on `stream`); reports the chosen caps
 * (cpct_plan_bins reports the bin plans).  The plan must not have clones
 * yet.  Allocates temporary buffers; synchronous. */
int cpct_plan_tune(cpct_plan* plan, int reps, int* fwd_cap, int* adj_cap, cudaStream_t stream);

/* A batch: the operator applied to `batch` slices, each with its own plan
 * (clones of one plan per distinct geometry; uneven view counts are fine),
 * captured once as a CUDA graph whose `branches` concurrent branches (0: 16)
 * take the slices longest first, round robin.  d_in/d_out are host arrays of
 * `batch` device pointers bound into the graph (they must stay valid and keep
 * their addresses).  mode: CPCT_BATCH_FWD (image -> sinogram),
 * CPCT_BATCH_ADJ (sinogram -> image), CPCT_BATCH_PAIR (image -> radon_adj of
 * radon_fwd, the sinogram kept in a plan-owned buffer).  Creation runs the
 * batch once eagerly and synchronizes `stream`. */
typedef struct cpct_batch cpct_batch;
#define CPCT_BATCH_FWD 0
#define CPCT_BATCH_ADJ 1
#define CPCT_BATCH_PAIR 2
int cpct_batch_create(cpct_batch** out, cpct_plan* const* plans, int batch, const float* const* d_in,
                      float* const* d_out, int mode, int branches, cudaStream_t stream);
/* Run the whole batch: one graph launch on `stream` (asynchronous). */
int cpct_batch_run(cpct_batch* batch, cudaStream_t stream);
/* Slices, polar samples per operator application over all slices, branches. */
int cpct_batch_info(const cpct_batch* batch, int* n_slices, long long* samples, int* branches);
int cpct_batch_destroy(cpct_batch* batch);

/* ---- ring filter and SPGL1 (section "Introduction", the L1 problem) ---- */

/* Ring-artifact filter ("polynomial subtraction" with a 3rd-order fit), read
 * as the orthogonal projector  F y = y - 1_M (m - Pi_3 m),  m[s] the mean of
 * detector column s over the M views, Pi_3 the least-squares cubic fit over
 * s (FP64 column means and fit).  Per-detector-column offsets (rings) that a
 * cubic does not explain are removed.
 *   d_in, d_out  device, M*Ns float32 (may alias).  Allocates a small
 *   workspace (Ns x 6 doubles) and synchronizes `stream`. */
int cpct_ring_filter(cpct_plan* plan, const float* d_in, float* d_out, cudaStream_t stream);

/* SPGL1 options (0 selects the default shown). */
typedef struct spgl1_opts {
  int max_iter;       /* iteration cap, 300                                     */
  int memory;         /* non-monotone line-search memory, 3 (<= 8)            */
  int max_line;       /* halvings per line search, 10 (at most 11 arc trials   */
                      /* and 10 feasible-direction trials per iteration)        */
  int flags;          /* CPCT_SPGL1_* bits                                      */
  double opt_tol;     /* relative duality gap / root tolerance, 1e-4            */
  double bp_tol;      /* basis-pursuit tolerance, 1e-6                          */
  double gamma;       /* sufficient decrease, 1e-4                              */
  double step_min;    /* Barzilai-Borwein step clamp, 1e-16                     */
  double step_max;    /* 1e5                                                    */
  double tau0;        /* initial l1 radius (CPCT_SPGL1_TAU0), or the fixed      */
                      /* radius of a LASSO solve (CPCT_SPGL1_LASSO)             */
  double ls_tol;      /* least-squares exit ||A^T r||_inf <= ls_tol ||r||, 1e-6 */
  double dec_tol;     /* relative objective decrease that counts as stagnation  */
                      /* far from the root, 1e-4                                */
  int max_line_errors;/* failed searches (each divides step_max by 10), 10      */
  int pad_;
} spgl1_opts;

#define CPCT_SPGL1_TAU0 0x1       /* start from opts->tau0 instead of ||x0||_1  */
#define CPCT_SPGL1_NO_FILTER 0x2  /* solve with A = R (no ring filter)          */
#define CPCT_SPGL1_SYNTH_DH 0x4   /* analysis-l1 variant: x is z, the operator  */
                                  /* acts on u = C z (cpct_synth_dh), so the    */
                                  /* solve is min ||z||_1 s.t.                  */
                                  /* ||F(R C z) - F b|| <= sigma; u = C x after */
#define CPCT_SPGL1_LASSO 0x8      /* the LASSO problem alone: min ||F(R x) -    */
                                  /* F b||_2 s.t. ||x||_1 <= opts->tau0, tau    */
                                  /* fixed, sigma ignored (may be NULL)         */

/* Result record of one solve.  status:
 *   1 root found: | ||r|| - sigma | <= opt_tol max(1, ||F b||) at a point
 *     whose LASSO problem is nearly optimal (duality gap) or at that root
 *     error directly, as in the published method's exit test;
 *   2 basis-pursuit solution (||r|| <= bp_tol ||F b||);
 *   3 iteration cap;  4 line-search failure (max_line_errors exhausted);
 *   5 non-finite values;
 *   6 least-squares solution (||A^T r||_inf <= ls_tol ||r||);
 *   7 suboptimal BP: ||r|| <= sigma at a nearly optimal LASSO point short
 *     of the root error;
 *   8 LASSO optimal (CPCT_SPGL1_LASSO): relative duality gap <= opt_tol. */
typedef struct spgl1_info {
  int status;
  int iterations;     /* SPGL1 iterations (spectral projected-gradient steps)  */
  int ticks;          /* device ticks (line-search trials + bookkeeping)        */
  int trials;         /* line-search trials                                     */
  double tau;         /* final l1 radius                                        */
  double rnorm;       /* ||F(R x) - F b||_2                                     */
  double xnorm1;      /* ||x||_1                                                */
  double rel_gap;     /* relative duality gap of the last LASSO subproblem      */
  int newton;         /* Newton updates of tau                                  */
  int line_errors;    /* failed line searches                                   */
  int safeguards;     /* flat-arc rescalings of the arc search                  */
  int stationary;     /* iterations whose first trial did not move x            */
  double gstep;       /* final Barzilai-Borwein step                            */
} spgl1_info;

/* Basis-pursuit denoising  min ||x||_1  s.t.  ||F(R x - b)||_2 <= sigma by
 * SPGL1 (van den Berg & Friedlander 2008; the L1 problem of section
 * "Introduction"): Newton root-finding on the Pareto curve tau -> ||r_tau||
 * (tau updated when the objective of the current LASSO problem stagnates),
 * each LASSO problem solved by spectral projected gradient with a
 * non-monotone search along the projection arc (with the published flat-arc
 * rescaling), a feasible-direction fallback search and step-max damping
 * after failed searches; FP32 per-element work, partial sums combined in
 * FP64, exact l1-ball projection (cpct_project_l1), and the controller
 * (Newton step, Armijo tests, Barzilai-Borwein step, duality gap) in FP64 on
 * the device, one CUDA graph per iteration tick.
 *   d_b     device, M*Ns float32 data (read)
 *   sigma   misfit bound eps >= 0 (0: basis pursuit); ignored with
 *           CPCT_SPGL1_LASSO
 *   d_x     device, N*N float32: in = warm start (zeros for a cold start),
 *           out = solution; tau starts at ||x0||_1 unless CPCT_SPGL1_TAU0
 *   opts    NULL for defaults;  info  host record, may be NULL
 * Returns CPCT_OK (status 1, 2, 6, 7, 8), CPCT_ENOTCONV (iteration cap or
 * line-search failure; d_x holds the last iterate), CPCT_ENONFINITE (NaN or
 * Inf in the data, the warm start or a trial), CPCT_EINVAL, CPCT_ENOMEM,
 * CPCT_ECUDA.  Allocates its workspace (6 N^2 + 4 M Ns floats) for the
 * duration of the call and synchronizes `stream`.  Kernel event profiling
 * of the plan is switched off by this call. */
int spgl1_solve(cpct_plan* plan, const float* d_b, double sigma, float* d_x, const spgl1_opts* opts,
                spgl1_info* info, cudaStream_t stream);

/* The same for `batch` independent slices solved together (one graph whose
 * branches run the slices concurrently).  Each slice needs its own plan (a
 * plan holds per-call workspaces); arrays are host arrays of `batch` entries
 * (sigma may be NULL with CPCT_SPGL1_LASSO); info is an array of `batch`
 * records. */
int spgl1_solve_batched(cpct_plan* const* plans, int batch, const float* const* d_b, const double* sigma,
                        float* const* d_x, const spgl1_opts* opts, spgl1_info* info, cudaStream_t stream);

/* Euclidean projection onto the l1 ball {x : ||x||_1 <= tau}, the
 * projection step of SPGL1's spectral projected gradient (van den Berg &
 * Friedlander 2008; the L1 problem of section "Introduction"):
 *   out_i = sign(v_i) max(|v_i| - theta, 0),  theta >= 0 the root of
 *   sum_i max(|v_i| - theta, 0) = tau;  out = v and theta = 0 when
 *   ||v||_1 <= tau;  out = 0 (theta reported as 0) when tau <= 0.
 * theta is exact for the FP32 input: the set of |v_i| above it is found by a
 * radix selection on the float bit patterns with exact integer bin sums, and
 * theta = (sum of that set - tau) / its size is evaluated in FP64; out is
 * rounded to FP32.  Deterministic, sort-free, three histogram passes.
 *   d_v     device, n float32 (read; finite values)
 *   n       1 <= n <= 2^30
 *   tau     radius (finite)
 *   d_out   device, n float32 (may alias d_v)
 *   theta   host, may be NULL: the threshold (FP64)
 * Returns CPCT_OK, CPCT_EINVAL (null pointer, n or tau out of range),
 * CPCT_ENOMEM, CPCT_ECUDA.  Allocates a small workspace (about 30 KB) for
 * the call and synchronizes `stream`. */
int cpct_project_l1(const float* d_v, long long n, double tau, float* d_out, double* theta, cudaStream_t stream);

/* The same for `batch` vectors of n values each (host arrays of device
 * pointers d_v / d_out, radii tau, thresholds theta (may be NULL)), one
 * workspace and one synchronization for all of them. */
int cpct_project_l1_batched(const float* const* d_v, int batch, long long n, const double* tau,
                            float* const* d_out, double* theta, cudaStream_t stream);

/* ---- learned warm start: convolutional denoiser (no counterpart in the
 * paper; the network maps a filtered back-projection to a starting point of
 * spgl1_solve) ------------------------------------------------------------ */

/* U-Net on single-channel H x W images, `levels` resolution levels, c_l =
 * base * 2^l channels at level l:
 *   encoder l = 0..L-1:  h = relu(conv_b(relu(conv_a(x)))), skip_l = h,
 *                        x = 2x2 average pool of h below the last level;
 *   decoder l = L-2..0:  u = relu(conv_up(nearest 2x upsample of h)),
 *                        h = relu(conv_b(relu(conv_a([skip_l, u]))));
 *   output:              out = x_in + bias + sum_c w_c h_c  (1x1 head).
 * 3x3 convolutions are cross-correlations with zero padding 1 and a bias.
 * Loss of a batch: L = sum (out - target)^2 / (2 P) over its P pixels.
 * Precision: activations and gradients FP32, convolution weights rounded to
 * BF16 and activations rounded to BF16 inside each tensor-core contraction,
 * FP32 accumulation; FP32 master weights and Adam state.
 * Parameter vector (host, float32): layers in the order enc0.a, enc0.b, ...,
 * enc(L-1).b, then for l = L-2..0: dec_l.up, dec_l.a, dec_l.b, then head;
 * per layer W as (Cout, k, k, Cin) row-major, then b (Cout).  Cin of enc0.a
 * is 1, of dec_l.a 2 c_l (skip channels first). */
typedef struct cpct_unet cpct_unet;

/* Number of parameters of the vector above; -1 for an unsupported shape
 * (levels 1..6, base a positive multiple of 32).  Host only. */
long long cpct_unet_param_count(int levels, int base);

/* Network with device activations for up to max_batch images of height x
 * width (both divisible by 2^(levels-1)), parameters zero.  CPCT_EINVAL for
 * unsupported shapes (also base * 2^(levels-1) > 1024), CPCT_ENOMEM. */
int cpct_unet_create(cpct_unet** out, int levels, int base, int max_batch, int height, int width,
                     cudaStream_t stream);
int cpct_unet_destroy(cpct_unet* net);

/* Host copies of the parameters / of the gradients of the last
 * cpct_unet_backward (layout above).  set_params resets the Adam state.
 * Synchronous. */
int cpct_unet_set_params(cpct_unet* net, const float* h_params, cudaStream_t stream);
int cpct_unet_get_params(cpct_unet* net, float* h_params, cudaStream_t stream);
int cpct_unet_get_grads(cpct_unet* net, float* h_grads, cudaStream_t stream);

/* out = net(in) for `batch` images; d_in, d_out device float32 batch x H x W
 * (16-byte aligned).  Stream-ordered, asynchronous.  The 3x3 convolutions
 * of the forward pass run on the tensor-memory (tcgen05) kernel, whose
 * waits are bounded: an expired wait sets the net's device error flag
 * (reported by cpct_unet_sync) and leaves that layer's output undefined. */
int cpct_unet_forward(cpct_unet* net, const float* d_in, float* d_out, int batch, cudaStream_t stream);

/* Synchronizes `stream` and reads and clears the net's device error flag:
 * CPCT_OK, or CPCT_ETIMEOUT if a bounded device wait of a forward pass
 * (cpct_unet_forward or cpct_unet_backward) expired since the last call. */
int cpct_unet_sync(cpct_unet* net, cudaStream_t stream);

/* Forward pass, loss against d_target and the gradients of every parameter
 * (kept on the device for cpct_unet_adam_step / cpct_unet_get_grads);
 * *loss (host, may be NULL) receives the loss and then the call synchronizes
 * `stream`. */
int cpct_unet_backward(cpct_unet* net, const float* d_in, const float* d_target, int batch, double* loss,
                       cudaStream_t stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the
 * gradients of the last backward pass, scaled by min(1, max_grad_norm /
 * ||g||_2) when max_grad_norm > 0 (no clipping when 0); refreshes the BF16
 * weights.  grad_norm (host, may be NULL) receives ||g||_2 before clipping,
 * and then the call synchronizes `stream`. */
int cpct_unet_adam_step(cpct_unet* net, float lr, float max_grad_norm, double* grad_norm, cudaStream_t stream);

/* One denoiser operation on caller tensors, for tests (B images, channels
 * fastest, device float32; H x W is the size of a for ops 0, 1, 2, 5 and
 * the size of y for ops 3, 4):
 *   op 0: y = relu(conv3x3([a | b]) + bias), a: C1 channels, b: C2 (or NULL
 *         with C2 = 0), y: Cout; h_w host float32: weights (Cout, 3, 3,
 *         C1 + C2) then Cout biases; operands rounded as in the network
 *   op 1: y = 2x2 average pool of a (C1 channels)
 *   op 2: y = nearest 2x upsampling of a
 *   op 3: y = adjoint of the pooling of an H x W image applied to the
 *         half-size gradient a, plus b (H x W, may be NULL)
 *   op 4: y = adjoint of the upsampling of an H x W image applied to the
 *         double-size gradient a
 *   op 5: y = data gradient of op 0's convolution at output gradient a
 *         (Cout channels) with ReLU mask taken from b (Cout channels, the
 *         op's output); y has C1 + C2 channels
 *   op 6: weight and bias gradients of op 0's convolution at input a (C1
 *         channels, C2 = 0) and output gradient b (Cout channels, used as
 *         is): y = (Cout, 3, 3, C1) weights then Cout biases (flat)
 *   op 7: op 0 computed by the mma.sync kernel that reads BF16 copies of its
 *         inputs; equals op 0
 *   op 8: op 0 computed by the tensor-memory (tcgen05) kernel that reads
 *         BF16 copies of its inputs, as in the network's forward pass (Cout
 *         in {32, 64, 128} or a multiple of 256; other Cout: CPCT_EINVAL):
 *         operand tiles loaded by TMA where the image tiles into 128-pixel
 *         boxes (W a multiple of 128, or a power of two below 128 dividing
 *         H x W into 128-pixel blocks), else by cp.async gathers; the same
 *         BF16 operands as op 0.  CPCT_ETIMEOUT if a bounded wait of the
 *         kernel expired.
 *   op 9: op 8 with the cp.async gathers whatever the shape.
 *   op 12: op 6 computed by the weight-gradient kernel that reads BF16 copies
 *         of a and b (the network's backward pass).
 *   op 11: op 5 computed by the tensor-memory kernel on a BF16 copy of the
 *         masked gradient (the network's backward pass; C2 = 0, C1 in {32,
 *         64, 128} or a multiple of 256).
 *   op 10: the network's first layer, y = relu(conv3x3(a) + bias) for a
 *         single-channel a (B x H x W, C1 = 1, C2 = 0), w = [Cout][3][3][1]
 *         then the Cout biases, Cout a multiple of 8 up to 1024: the direct
 *         kernel (BF16 operands, FP32 accumulation in tap order).
 * C1, C2 multiples of 32 (C1 > 0), Cout a multiple of 32 for ops 0, 5-9, 11, 12.
 * Synchronous; allocates a workspace for ops 0 and 5-12. */
int cpct_unet_debug_op(int op, const float* d_a, const float* d_b, float* d_y, const float* h_w, int B, int H, int W,
                       int C1, int C2, int Cout, cudaStream_t stream);

/* Per-slice statistics and scaling of the learned warm start (no
 * counterpart in the paper).  A batch is `batch` (1..65535) slices of n >= 1
 * contiguous float32 values each (device, caller-owned); h_* arrays are host
 * arrays of `batch` entries.  Reductions are deterministic (fixed grids,
 * FP64 sums in a fixed order).  Each call allocates a small stream-ordered
 * workspace and synchronizes `stream`; CPCT_EINVAL for null pointers, sizes
 * out of range or non-finite per-slice parameters.
 *   cpct_slice_moments: mean and sample standard deviation (divisor n - 1;
 *                       0 for n = 1) of every slice, two passes (the second
 *                       about the mean); either output may be NULL;
 *   cpct_slice_soft_l1: h_out[i] = sum_j max(|x_ij| - h_thresh[i], 0), the
 *                       l1 norm of the soft-thresholded slice (thresholds
 *                       finite, >= 0);
 *   cpct_slice_scale:   d_out slice i = h_factor[i] * d_in slice i (FP32
 *                       product; d_out may alias d_in). */
int cpct_slice_moments(const float* d_x, int batch, long long n, double* h_mean, double* h_std, cudaStream_t stream);
int cpct_slice_soft_l1(const float* d_x, int batch, long long n, const double* h_thresh, double* h_out,
                       cudaStream_t stream);
int cpct_slice_scale(const float* d_in, float* d_out, int batch, long long n, const double* h_factor,
                     cudaStream_t stream);

/* Test introspection of the tensor-core (tcgen05) path: D = A * B^T with one
 * CTA and the accumulator in tensor memory.  A: 128 x k, B: n x k (bfloat16,
 * row-major, device, 16-byte aligned), D: 128 x n (float32, device); k a
 * multiple of 32, n in {32, 64, 128}.  Synchronous; CPCT_ETIMEOUT if a
 * bounded wait for the MMA gave up. */
int cpct_debug_tc_gemm(const void* d_a, const void* d_b, float* d_d, int n, int k, cudaStream_t stream);

/* Allocation-free adjoint.  Some callers cannot allocate device memory at
 * the point where they apply the operator: code running under an allocator
 * that has reserved the whole device pool (a framework's caching allocator),
 * real-time acquisition loops that must not pay for or risk an allocation,
 * or code that must not allocate while its stream work is being recorded.
 * radon_adj_noalloc computes exactly what radon_adj computes (same kernels,
 * same summation order), but the only scratch of its gridding step -- the
 * partial tiles of the few heavy tiles that are split over several work
 * items -- lives in a fixed device array inside this library instead of plan
 * memory: CPCT_NOALLOC_MAX_SLOTS tiles of 32 x 32 complex64 (8 KB each, 16
 * MB in all), held by every GPU that loads the library until the process
 * exits.
 * The paper has no counterpart of this entry point.
 *   plan    an existing plan (created earlier; this call allocates nothing:
 *           no cudaMalloc, cudaFree or allocating library routine)
 *   d_sino  device, M*Ns float32 (read);  d_img  device, N*N float32 (written)
 * Returns CPCT_EINVAL for bad arguments or if the plan's geometry needs more
 * partial tiles than the array holds, CPCT_ECUDA if the array's device
 * address cannot be obtained.  The first call on each device looks that
 * address up (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  Every call shares the one array and it
 * keeps the last call's contents (each call overwrites every tile it reads,
 * so nothing needs clearing); calls that overlap on the GPU -- on different
 * streams, or from different plans -- race on it and must be serialised. */
#define CPCT_NOALLOC_MAX_SLOTS 2048
int radon_adj_noalloc(cpct_plan* plan, const float* d_sino, float* d_img, cudaStream_t stream);

/* Human-readable name of a cpct_status (static string). */
const char* cpct_strerror(int status);

/* ---- introspection for tests (host-only unless stated) ------------------ */

/* Bin lists of a geometry, built on the host exactly as cpct_plan_create
 * builds them (no GPU needed).  which = 0: forward bins (each polar sample
 * k = 0..Ns/2 in the 32x32 tile of its footprint's first grid point);
 * which = 1: adjoint bins (every tile of the extended half spectrum that the
 * 6x6 footprint touches).  Reports the tile count, the entry count and
 * checksum = sum_i id_i * (i mod 1000003 + 1). */
int cpct_debug_bins(const cpct_geom* g, int which, int* n_tiles, int* n_entries, int64_t* checksum);

/* Copy the sample ids (j << 16 | k) of one tile's bin into ids (capacity
 * cap).  Returns the bin length (may exceed cap) or a negative status. */
int cpct_debug_bin_tile(const cpct_geom* g, int which, int tile, uint32_t* ids, int cap);

/* Round packing of the adjoint bins (host only): the samples of every tile
 * are packed into rounds of <= 32 samples with pairwise disjoint footprints,
 * one lane each, lanes chosen so that their shared-memory accesses are
 * bank-conflict free.  Reports the round count, the packed sample count and
 * valid = 1 if every invariant holds (each bin entry exactly once, no two
 * footprints of a round overlap, lane = bank class). */
int cpct_debug_rounds(const cpct_geom* g, int* n_rounds, int* n_packed, int* valid);

/* The adjoint work items that a plan of geometry g gets with its default
 * bin plan and `cap` rounds per spread item (0: the automatic cap of
 * cpct_plan_create, for the current GPU, or for a GB300 when there is
 * none), built on the host exactly as cpct_plan_create / cpct_plan_set_caps
 * build them: items, split heavy bins, partial-tile slots of 32 x 32.  No
 * GPU needed. */
int cpct_debug_adj_items(const cpct_geom* g, int cap, int* n_items, int* n_split, int* n_slots);

/* A bin plan of a geometry built on the host exactly as cpct_plan_set_bins
 * builds it (kind, tile as there; adjoint rounds of `lanes` samples, 16, 32
 * or 64, CPCT_ROUNDS_COLUMNS for column groups, 0 for the default): forward
 * and adjoint bin counts, the adjoint bins of each size (16, 32, 64; host
 * array of 3, may be NULL), the adjoint rounds (or groups), and valid = 1 if
 * every invariant holds (disjoint aligned bins; forward lists partition the
 * samples by first point; adjoint lists hold exactly the samples whose
 * footprint touches the bin; rounds hold each entry once, footprints
 * disjoint, lane = bank class mod 16, or for groups the slots' classes in
 * the conflict-free pattern and each entry's payload that of its sample).  No GPU
 * needed; CPCT_EINVAL for another width. */
int cpct_debug_binplan(const cpct_geom* g, int kind, int tile, int lanes, int* n_fwd_bins, int* n_adj_bins,
                       int* adj_class_bins, int* n_rounds, int* valid);

/* The split of a sample coordinate u = k (hi + lo) into floor and fraction,
 * with the same float32 operations as the kernels. */
int cpct_debug_split(float k, float hi, float lo, int* fl, float* z);

/* Copy a plan's FP64 kernel-approximation coefficients (6 taps x 10
 * monomial coefficients in s = 2 frac(u) - 1) and its float32 deapodization
 * vector (N) to host buffers; either pointer may be NULL.  Synchronous. */
int cpct_debug_tables(cpct_plan* plan, double* h_poly64, float* h_deapod);

/* ---- profiling ---------------------------------------------------------- */

/* Kernel ids: 0 k_fwd_col, 1 k_fwd_row, 2 k_fwd_interp, 3 k_fwd_ray,
 * 4 k_adj_ray, 5 k_adj_spread, 6 k_adj_reduce, 7 k_adj_row, 8 k_adj_col. */
#define CPCT_NUM_KERNELS 9

/* Bracket every later launch of the kernels whose bit (1 << id) is set in
 * `mask` with a CUDA event pair on its launch stream (0 disables). */
int cpct_profile_enable(cpct_plan* plan, unsigned mask);

/* Synchronize on the recorded events and return, per kernel id, the summed
 * device milliseconds and the launch count since the previous read
 * (arrays of CPCT_NUM_KERNELS entries). */
int cpct_profile_read(cpct_plan* plan, double* total_ms, long long* launches);

/* Name of kernel id `kid` (static string). */
const char* cpct_kernel_name(int kid);

/* Number of kernels the plan's operators have launched (optionally reset). */
long long cpct_launch_count(cpct_plan* plan, int reset);

#ifdef __cplusplus
}
#endif
#endif /* CPCT_H_ */
