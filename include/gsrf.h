/*
 * gsrf.h -- C ABI of the GB300 (sm_103a) GSRF render library, libgsrf.so.
 *
 * GSRF (arXiv 2502.01826) renders the RF signal received at a receiver from a scene
 * of complex-valued 3D Gaussians: orthographic splatting of the Gaussians onto the
 * receiver's azimuth x elevation ray grid (Sec. 4.3), a Fourier-Legendre radiance per
 * ray (Sec. 4.2, Eq. 9), and complex front-to-back accumulation along every ray
 * (Sec. 4.4, Eq. 14; App. A), reduced to the received spectrum, RSSI or CSI.  The
 * calls below follow the paper's statement of the problem (Sec. 4.1): given the
 * transmitter position t, receiver positions r_i and the scene parameters theta,
 * synthesise S_i.  They run as CUDA kernels on the caller's stream; nothing here
 * falls back to the CPU.
 *
 * Conventions (all calls):
 *   - Pointers marked [dev] are device pointers, [host] host pointers.  The caller
 *     owns every buffer: inputs, outputs and one workspace.  The library allocates no
 *     device memory and never synchronises the stream, except gsrf_read_status.
 *   - Arrays are C-contiguous FP32 unless stated; complex values are interleaved
 *     (re, im) pairs.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Argument errors return synchronously (nothing is launched).  Conditions met on
 *     the device (pair capacity exceeded, non-finite parameters, a bounded wait that
 *     ran out) set the status word in the workspace; gsrf_read_status reads it.  No
 *     call aborts, traps or throws.
 *   - The workspace carries state from gsrf_project to gsrf_bin to gsrf_render_fwd /
 *     gsrf_render_bwd: call them in that order with the same plan and workspace.
 *
 * Readings of the paper built into the arithmetic (each also listed in the
 * repository's design notes): alpha_k = min(sigmoid(opacity_k) * exp(-m2_rep/2),
 * alpha_max); the complex transmittance of a Gaussian is (1 - alpha_k)
 * exp(-j 2 pi f b_k dt_k / c); every Gaussian re-radiates with the path phase
 * exp(-j 2 pi f (|t - mu_k| + |mu_k - r|) / c); 3-sigma = Mahalanobis^2 9; the
 * Fourier-Legendre basis is evaluated at each ray's (azimuth, sin elevation) without
 * the Condon-Shortley phase; depth order is ascending FP32 |mu_k - r|, ties by index;
 * a ray hits iff m2 < 9 and t_out >= r_rx, with t_in clipped to r_rx; c = 3e8 m/s.
 */
#ifndef GSRF_H
#define GSRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSRF_OK = 0,
    GSRF_ERR_INVALID_ARG = 1,  /* a size, pointer or grid field is out of range */
    GSRF_ERR_CUDA = 2,         /* a CUDA launch or copy failed */
    GSRF_ERR_CAPACITY = 3,     /* more (tile, Gaussian) pairs than plan.pair_capacity */
    GSRF_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out */
    GSRF_ERR_NONFINITE = 5,    /* a Gaussian parameter is NaN or infinite */
    GSRF_ERR_UNSUPPORTED = 6,  /* a configuration this build does not implement */
    GSRF_ERR_TOO_LARGE = 7     /* the problem does not fit gsrf_render_static's fixed array */
} gsrf_status;

/* The receiver's ray grid (Sec. 4.3, Eqs. 10-12): ray (u, v) points at azimuth
 * az0 + (u + 1/2) daz and elevation el0 + (v + 1/2) del (degrees), i.e. at the
 * centre of the one-bin cell that Eq. 12 maps it to. */
typedef struct {
    int32_t n_az, n_el;        /* rays along azimuth / elevation, >= 1 */
    float az0_deg, daz_deg;    /* azimuth of the grid origin (|az0| <= 360), bin width > 0 */
    float el0_deg, del_deg;    /* elevation of the grid origin, bin height > 0 */
    float r_rx;                /* radius of the ray-emitting sphere (App. E table: 1.0 m) */
    float eps_T;               /* stop a ray once prod(1 - alpha) < eps_T; 0 = never */
    float alpha_max;           /* clamp on alpha, in (0, 1) (0.99 keeps 1/(1-alpha) finite) */
    int32_t tile_w, tile_h;    /* rays per tile (App. E: 16 x 16): tile_w 8, 16 or 32, tile_h 4, 8, 16
                                * or 32, each a multiple of the plan's ray block; at most 64 tiles
                                * along azimuth and 1024 in all */
} gsrf_grid;

/* Scene parameters theta, [dev], structure-of-arrays, n Gaussians (Sec. 4.2). */
typedef struct {
    int64_t n;                 /* number of Gaussians, 0 <= n < 2^31 */
    const float *means;        /* [n,3] mu_k, metres */
    const float *log_scales;   /* [n,3] log of the diagonal of S_k */
    const float *quats;        /* [n,4] rotation R_k as a quaternion (w,x,y,z), any non-zero norm */
    const float *opacity_logit;/* [n]   opacity before the sigmoid */
    const float *coeffs;       /* [n,(L+1)^2,2] Fourier-Legendre coefficients c_{l,m}, index l*l+l+m
                                * (L = plan.fle_degree, 3 by default: [n,16,2]) */
    const float *phase_b;      /* [n] excess-phase coefficient b_k of the transmittance, or NULL (= 0) */
} gsrf_gaussians;

/* One render problem: n_rx receivers of one scene against one transmitter, at the
 * n_f frequencies f0 + i*df (i < n_f). */
typedef struct {
    int64_t n_gauss;           /* Gaussians in the scene */
    int32_t n_rx;              /* receivers, >= 1 */
    int32_t n_f;               /* frequencies, 1 <= n_f <= 64 */
    double f0_hz, df_hz;       /* first frequency and spacing (Hz), f0 > 0 */
    gsrf_grid grid;
    int64_t pair_capacity;     /* room for (tile, Gaussian) instances over all receivers */
    int32_t ray_block_w;       /* rays a warp renders along azimuth: 4, 8, 16 or 32, the block
                                * being 32 / ray_block_w high; 0 = 8 (8 x 4) */
    int32_t stage;             /* candidates a warp stages in shared memory per batch: 16 or 32;
                                * 0 = 32.  Tile shape, ray block and stage change speed only,
                                * never results; gsrf_autotune picks them by measurement */
    int32_t ckpt_every;        /* transmittance checkpoints for the backward: 0 = none, else K, a
                                * multiple of 32 -- the forward keeps every ray's transmittance
                                * in front of tile-list positions K, 2K, ... (ckpt_slots of them)
                                * and the backward re-anchors its recomputed transmittance there */
    int32_t ckpt_slots;        /* checkpoints kept per ray, 1..64 when ckpt_every > 0 */
    int32_t variant;           /* other readings of the paper (bit mask, 0 = the
                                * default): GSRF_VARIANT_RADIANCE_AT_MEAN takes Gaussian k's
                                * Fourier-Legendre radiance at the direction of mu_k seen from
                                * the receiver (Sec. 4.3's v_k) for all its rays instead of at
                                * each ray's direction; GSRF_VARIANT_NORMALISED_WEIGHT weights by
                                * the normalised density (App. A.3), g / ((2 pi)^1.5 |Sigma|^0.5);
                                * GSRF_VARIANT_PAPER_CULLING lets ray (u, v) meet Gaussian k only
                                * inside its splatting circle (Sec. 4.3): centre (u_k, v_k) = the
                                * bin of mu_k's direction, radius 3 sqrt(lambda_max(J Sigma J^T))
                                * in bins, decided in FP32 with correctly rounded operations; the
                                * exact test still decides the hit inside it;
                                * GSRF_VARIANT_PATH_AT_REP gives each (ray, Gaussian) pair the
                                * path through its representative point, |t - x_rep| +
                                * |x_rep - r|, instead of through mu (one frequency, L = 3, not
                                * in the batched render); GSRF_VARIANT_ORDER_T_MID composites a
                                * ray's hits in ascending t_mid (closest approach along the ray,
                                * ties by list position) instead of in the list's |mu - r|
                                * order: one frequency, L = 3, without bit 8, not batched; a ray
                                * keeps its 512 nearest hits and must terminate on them (else
                                * GSRF_ERR_UNSUPPORTED in the status word).  The backward has
                                * bits 2 and 4 (and none); bits 1, 8 and 16 are forward-only.
                                * 0..31 */
    int32_t fle_degree;        /* degree L of the Fourier-Legendre radiance (Sec. 4.2), 1..5;
                                * 0 = 3, the paper's choice.  The Gaussians then carry (L + 1)^2
                                * complex coefficients each.  L != 3 is single-frequency:
                                * GSRF_ERR_UNSUPPORTED for n_f > 1, for the batched render and
                                * for variant GSRF_VARIANT_RADIANCE_AT_MEAN; the forward and the
                                * backward run at every degree */
} gsrf_plan;
#define GSRF_VARIANT_RADIANCE_AT_MEAN 1
#define GSRF_VARIANT_NORMALISED_WEIGHT 2
#define GSRF_VARIANT_PAPER_CULLING 4
#define GSRF_VARIANT_PATH_AT_REP 8
#define GSRF_VARIANT_ORDER_T_MID 16

/* Bytes of workspace a plan needs (256-byte aligned base required). [host] out. */
gsrf_status gsrf_workspace_size(const gsrf_plan *plan, size_t *bytes);

/* Byte offsets inside the workspace of the arrays tests and tools may inspect after
 * gsrf_project (view) and gsrf_bin (the rest): the sorted pairs' Gaussian ids [uint32]
 * over all receivers back to back; per receiver the first pair (int64, [n_rx + 1]); per
 * receiver and tile the list start relative to the receiver's first pair (uint32,
 * [n_rx][n_tiles + 1]); and the sorted 64-bit splat keys (tile << 32 | FP32 depth bits)
 * [uint64] parallel to the ids, which gsrf_pair_keys fills on request (gsrf_bin does not:
 * the render needs only the ids and the tile ranges). */
typedef struct {
    size_t pair_keys, pair_ids, rx_pair_base, tile_start;
    size_t status;
    int32_t n_tiles_u, n_tiles_v;
    size_t view;               /* per (receiver, Gaussian) 48-byte records after gsrf_project,
                                * receiver-major: floats 0-2 mu - r, 3 D cos(theta) of the
                                * cone of directions that can reach the Gaussian (culling),
                                * 4-6 whitened receiver offset, 7-8 e^{-j 2 pi f0 d / c}
                                * (cos, -sin) with the phase reduced in FP64, 9 the
                                * per-subcarrier step 2 pi df d / c, 10-11 the radiance at
                                * the direction of mu (GSRF_VARIANT_RADIANCE_AT_MEAN), else 0;
                                * for a Gaussian that covers no tile of that receiver only
                                * floats 0-2 and a NaN in float 3 (the rest is not written) */
} gsrf_layout;
gsrf_status gsrf_workspace_layout(const gsrf_plan *plan, gsrf_layout *out);

/* Step 1 -- Alg. 1's splatting step, Sec. 4.3: per Gaussian the
 * whitening matrix diag(1/s) R^T and opacity; per (receiver, Gaussian) the whitened
 * receiver offset, the FP32 depth |mu - r| (sort key), the set of tiles the Gaussian
 * may touch (conservative: every ray that can hit it lies in one of them) and the
 * path phase exp(-j 2 pi f0 d / c), d = |t - mu| + |mu - r|, range-reduced in FP64.
 *   rx_pos [dev] [n_rx,3]; tx_pos [dev] [3].
 * Clears the status word.  Non-finite parameters set GSRF_ERR_NONFINITE. */
gsrf_status gsrf_project(const gsrf_plan *plan, const gsrf_gaussians *g, const float *rx_pos,
                         const float *tx_pos, void *workspace, size_t ws_bytes, void *stream);

/* Step 2 -- the key sort of Alg. 1 and App. E: one 64-bit key per (tile, Gaussian) pair,
 * high 32 bits the tile index (tv * n_tiles_u + tu), low 32 bits the FP32 depth;
 * all pairs of a receiver sorted by key, ties by Gaussian index (a stable radix sort
 * written for this library), and each tile's [start, end) range.  If the pairs of all
 * receivers exceed plan.pair_capacity the status word gets GSRF_ERR_CAPACITY and the
 * required count; later steps then write zeros. */
gsrf_status gsrf_bin(const gsrf_plan *plan, void *workspace, size_t ws_bytes, void *stream);

/* Inspection after gsrf_bin -- App. E, the splat keys of Alg. 1: writes the sorted
 * 64-bit key (tile << 32 | FP32 depth bits) of every pair into the workspace array that
 * gsrf_workspace_layout's pair_keys names, parallel to the pair ids.  The depth bits are
 * those the depth sort used (|mu - r| in deterministic FP32).  Same arguments and errors as
 * gsrf_bin; the workspace must hold a completed gsrf_bin of this plan. */
gsrf_status gsrf_pair_keys(const gsrf_plan *plan, void *workspace, size_t ws_bytes, void *stream);

/* Step 3 -- the blend loop of Alg. 1, Eq. 14: every ray walks its tile's list front to back,
 * intersects the 3-sigma ellipsoid (App. D.3), weights by the Gaussian at the midpoint
 * of the chord beyond r_rx (App. A.2), evaluates the Fourier-Legendre radiance and
 * accumulates S += alpha psi e^{-j phi} T, T *= (1 - alpha) e^{-j theta}.
 *   out_rays  [dev] [n_rx][n_f][n_el][n_az][2]  per-ray received signal S.
 *   ray_state [dev] NULL, or gsrf_ray_state_bytes(plan) bytes (16-byte aligned) that the
 *             backward needs: 32 per ray, plus 16 per ray and checkpoint slot when
 *             plan.ckpt_every > 0. */
gsrf_status gsrf_render_fwd(const gsrf_plan *plan, const gsrf_gaussians *g, void *workspace,
                            size_t ws_bytes, float *out_rays, void *ray_state, void *stream);
size_t gsrf_ray_state_bytes(const gsrf_plan *plan);

/* Step 4 -- the backward (adjoint) render of App. D, after gsrf_render_fwd with a ray
 * state and the same plan and workspace.  Each ray is walked back to front from its last
 * composited Gaussian, recomputing the transmittance T_k = T_{k+1} / ((1 - alpha_k)
 * e^{-j theta_k}) instead of storing it; with the suffix R_k of later contributions,
 * dS/dalpha_k = psi_k E_k T_k - R_k / (1 - alpha_k), dS/dtheta_k = -j R_k,
 * dS/dphi_k = -j z_k, dS/dpsi_k = alpha_k E_k T_k (App. D.1-D.2), carried through the
 * midpoint weight and the ray-ellipsoid quadratic (App. D.3) to the raw parameters.
 *   ray_state [dev] from gsrf_render_fwd; grad_rays [dev] [n_rx][n_f][n_el][n_az][2] holds
 *   dL/dRe S and dL/dIm S.  Gradients [dev], same shapes as the parameters, are ADDED to
 *   (+=); any may be NULL.  The gradient of the opacity is taken through its sigmoid, of
 *   the rotation through the quaternion's normalisation, of the scales through exp.
 *   Hit decisions that sit on the integer steps of the method (splatting, the 3-sigma
 *   boundary, the early stop, the paper's splatting circle) carry no gradient.  Readings:
 *   the default, GSRF_VARIANT_NORMALISED_WEIGHT (the normalisation adds a log-scale term)
 *   and GSRF_VARIANT_PAPER_CULLING; GSRF_ERR_UNSUPPORTED for the other variant bits.  Any
 *   Fourier-Legendre degree (one frequency when L != 3).  With plan.ckpt_every = K > 0 the
 *   recomputed transmittance is replaced by the forward's own at every checkpoint the
 *   walk crosses, so division by (1 - alpha) never runs over more than K list positions
 *   (the per-tile checkpointing of deep scenes).  With n_f > 1 every subcarrier
 *   f0 + s df contributes with its own suffix sum and its own 2 pi f_s / c in the path and
 *   transmittance phases; the ray state then also carries sum(b dt) of each ray. */
gsrf_status gsrf_render_bwd(const gsrf_plan *plan, const gsrf_gaussians *g, void *workspace,
                            size_t ws_bytes, const void *ray_state, const float *grad_rays,
                            float *g_means, float *g_log_scales, float *g_quats,
                            float *g_opacity_logit, float *g_coeffs, float *g_phase_b, void *stream);

/* Batched persistent render (reading of Alg. 1's blend loop for many
 * problems at once; the paper renders one query at a time).  n_jobs problems -- each a
 * plan (n_f == 1) with its own workspace that gsrf_project and gsrf_bin have filled,
 * e.g. different scenes, receiver groups, transmitters and carriers -- are rendered by
 * ONE persistent kernel: the (job, receiver, tile, ray block) work items of all jobs are
 * ordered heaviest first (longest tile list) by a counting sort and taken by the warps
 * of a single resident wave from an atomic counter.  The jobs' descriptions are copied
 * into batch_ws on the stream, so the host arrays may be reused once the call returns.
 * Results are the same as gsrf_render_fwd's for each job (same per-ray arithmetic).
 *   plans, workspaces, ws_bytes, outs: [host] arrays of n_jobs (1..GSRF_MAX_BATCH_JOBS);
 *   outs[j] [dev] as gsrf_render_fwd's out_rays; batch_ws [dev] of
 *   gsrf_batch_workspace_size bytes (256-byte aligned).
 *   job_done_ns [dev] NULL, or n_jobs + 1 uint64 (8-byte aligned) that get the GPU's
 *   global timer (ns): [j] when the last work item of job j finished, [n_jobs] when the
 *   first warp of the launch started, so that [j] - [n_jobs] is job j's completion time
 *   inside the launch (a per-request latency when all jobs arrive together).
 *   flags: 0, or GSRF_BATCH_JOB_ORDER: the queue takes the jobs in the given order
 *   (heaviest first inside each job) instead of heaviest first over all jobs, so that a
 *   caller who orders its jobs (e.g. by deadline, or by size for shortest-first) gets
 *   them completed roughly in that order; results are the same either way.
 * GSRF_ERR_UNSUPPORTED when the jobs hold 2^32 work items or more. */
#define GSRF_MAX_BATCH_JOBS 4096
#define GSRF_BATCH_JOB_ORDER 1
gsrf_status gsrf_batch_workspace_size(int32_t n_jobs, const gsrf_plan *plans, size_t *bytes);
gsrf_status gsrf_render_batch(int32_t n_jobs, const gsrf_plan *plans, void *const *workspaces,
                              const size_t *ws_bytes, float *const *outs, void *batch_ws,
                              size_t batch_ws_bytes, uint64_t *job_done_ns, int32_t flags, void *stream);

/* Convenience: gsrf_project + gsrf_bin + gsrf_render_fwd in one call. */
gsrf_status gsrf_render(const gsrf_plan *plan, const gsrf_gaussians *g, const float *rx_pos,
                        const float *tx_pos, void *workspace, size_t ws_bytes, float *out_rays,
                        void *ray_state, void *stream);

/* Received signal from per-ray signals (Sec. 4.4, loss paragraph):
 *   GSRF_SIG_COMPLEX_SUM  out [n_rx][n_f][2]  S_hat = sum over rays of S_{u,v}
 *   GSRF_SIG_RSSI_DB      out [n_rx][n_f]     20 log10 |S_hat| (dB re unit amplitude)
 *   GSRF_SIG_POWER_SUM    out [n_rx][n_f]     sum over rays of |S_{u,v}|^2
 *   GSRF_SIG_SPECTRUM_MAG out [n_rx][n_f][n_el][n_az]  |S_{u,v}|, the spatial spectrum
 * rays [dev] [n_rx][n_f][n_el][n_az][2]; out [dev].  Sums run in a fixed order with
 * FP64 accumulation, so results are reproducible bit for bit. */
typedef enum {
    GSRF_SIG_COMPLEX_SUM = 0,
    GSRF_SIG_RSSI_DB = 1,
    GSRF_SIG_POWER_SUM = 2,
    GSRF_SIG_SPECTRUM_MAG = 3
} gsrf_sig_mode;
gsrf_status gsrf_received_signal(const float *rays, int32_t n_rx, int32_t n_f, int32_t n_el,
                                 int32_t n_az, int32_t mode, float *out, void *stream);

/* Device-side status after the calls above (synchronises `stream`). */
typedef struct {
    int32_t code;              /* gsrf_status */
    int32_t first_bad;         /* first offending Gaussian for GSRF_ERR_NONFINITE, else -1 */
    int64_t required_pairs;    /* pairs the last gsrf_bin needed */
    int64_t stats[4];          /* [0] candidate tests, [1] composited pairs (last render) */
} gsrf_run_status;
gsrf_status gsrf_read_status(const void *workspace, size_t ws_bytes, gsrf_run_status *out,
                             void *stream);

/* Stage timers.  The paper reports the render's cost as training time and inference
 * latency per spectrum (Sec. 5.1, "Training & Inference Efficiency"; App. F); this call
 * splits that latency over the stages.  Every gsrf_project, gsrf_bin, gsrf_render_fwd and
 * gsrf_render_bwd call records a CUDA event before and after its launches on its own
 * stream, keyed by its workspace (gsrf_render_batch: by its batch_ws).  Recording never
 * synchronises; a call on a stream that is capturing records nothing.  Only the last call
 * of each stage per workspace is kept.
 *   workspace [dev] a workspace (or batch_ws) passed to those calls; ms [host] float[8] gets
 *   the milliseconds of the last call of GSRF_STAGE_PROJECT, _BIN, _RENDER_FWD, _RENDER_BWD
 *   and _BATCH (slots 5..7 reserved), -1 for a stage not recorded.
 * Synchronises on the recorded end events.  GSRF_ERR_INVALID_ARG for a workspace with no
 * recorded call.  Host state only: events of up to 1024 workspaces are kept, the oldest
 * forgotten first; nothing is allocated on the device. */
#define GSRF_STAGE_PROJECT 0
#define GSRF_STAGE_BIN 1
#define GSRF_STAGE_RENDER_FWD 2
#define GSRF_STAGE_RENDER_BWD 3
#define GSRF_STAGE_BATCH 4
gsrf_status gsrf_stage_times(const void *workspace, float ms[8]);

/* Autotuner of the work split (tile shape, rays per warp block, candidates per
 * shared-memory stage), which changes speed, never results.  The paper fixes 16 x 16
 * tiles (App. E) and has no tuner; this is a property of this library.  For the
 * caller's own problem, on the caller's stream, it tries the tile shapes 16x16, 32x8,
 * 16x8, 8x16, 32x16, 16x32, 32x32 and 8x8 (each timed over gsrf_project + gsrf_bin).
 * Within each tile shape it tries every ray block width 4, 8, 16 or 32 that tiles it and
 * stages of 16 and 32 candidates (each timed over gsrf_render_fwd).  Every time is the
 * median of `reps` event-timed runs after one untimed run.  best gets the split with the
 * smallest sum of the two times; results (up to max_results, may be NULL when
 * max_results is 0) get every measurement, and n_results their number.
 *   plan, g, rx_pos, tx_pos as for gsrf_render; workspace [dev] of at least
 *   gsrf_autotune_workspace_size bytes; out_rays [dev] as for gsrf_render_fwd (holds the
 *   last candidate's rays); backward NULL to tune the forward, else the buffers below
 *   to tune forward + backward (the split that renders fastest need not be the one
 *   that trains fastest: larger tiles shorten binning but lengthen the backward's walk).  Tile shapes whose tiles exceed the grid limits or whose
 *   pairs exceed plan.pair_capacity are skipped; GSRF_ERR_CAPACITY if all are.  The call
 *   synchronises the stream and must not be captured into a graph.  To use the choice,
 *   copy best into plan.grid.tile_w / tile_h, plan.ray_block_w and plan.stage. */
typedef struct {
    int32_t tile_w, tile_h, ray_block_w, stage;
    float project_bin_ms;      /* gsrf_project + gsrf_bin with this tile shape */
    float render_ms;           /* gsrf_render_fwd (+ gsrf_render_bwd when tuning for training) */
} gsrf_tune_result;
/* Buffers that make the tuner time the training step's render: gsrf_render_fwd with
 * a ray state, then gsrf_render_bwd.  All [dev]; ray_state of gsrf_ray_state_bytes(plan)
 * bytes, grad_rays shaped like out_rays; the gradient buffers are scratch (their
 * contents are overwritten with meaningless sums) and any may be NULL. */
typedef struct {
    void *ray_state;
    const float *grad_rays;
    float *g_means, *g_log_scales, *g_quats, *g_opacity_logit, *g_coeffs, *g_phase_b;
} gsrf_tune_backward;
gsrf_status gsrf_autotune_workspace_size(const gsrf_plan *plan, size_t *bytes);
gsrf_status gsrf_autotune(const gsrf_plan *plan, const gsrf_gaussians *g, const float *rx_pos,
                          const float *tx_pos, void *workspace, size_t ws_bytes, float *out_rays,
                          const gsrf_tune_backward *backward, int32_t reps,
                          gsrf_tune_result *results, int32_t max_results, int32_t *n_results,
                          gsrf_tune_result *best, void *stream);

/* gsrf_render without a caller-supplied workspace, for callers that cannot allocate
 * device memory: hosts that forbid allocation once running (real-time or embedded
 * loops), plugins inside an application whose allocator owns all device memory, code
 * held to a fixed memory budget.  The paper has no counterpart; this is a deployment
 * convenience of this library.
 *   Inputs and outputs as for gsrf_render (out_rays [dev]); the workspace is a device
 *   array of GSRF_STATIC_SCRATCH_BYTES compiled into the library, which every device
 *   that loads the library holds until the process exits.
 *   A plan whose gsrf_workspace_size exceeds GSRF_STATIC_SCRATCH_BYTES is rejected with
 *   GSRF_ERR_TOO_LARGE before anything is launched (32 MiB holds, for one receiver on a
 *   360 x 90 grid, about 50,000 Gaussians with 300,000 tile pairs).
 *   status [host] NULL, or filled with the device status after the call (this
 *   synchronises `stream`).
 *   Every call made outside a stream capture looks up the array's device address
 *   afresh (so a cudaDeviceReset, after which the array may move, leaves no stale
 *   address); make the first call on a device before any stream capture.  All calls share the array and it keeps the last
 *   call's contents (every call initialises what it reads); calls that overlap on the
 *   GPU -- other streams, other host threads -- race on it.  Nothing is allocated. */
#define GSRF_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
gsrf_status gsrf_render_static(const gsrf_plan *plan, const gsrf_gaussians *g, const float *rx_pos,
                               const float *tx_pos, float *out_rays, gsrf_run_status *status,
                               void *stream);

/* Library version string. */
const char *gsrf_version(void);

#ifdef __cplusplus
}
#endif
#endif
