/*
 * slingbag.h -- C ABI of the GB300 (sm_103a) SlingBAG Pro hot path.
 *
 * The library renders a point cloud of spherical sources ("balls") onto an
 * arbitrary array of oriented sensors (the differentiable radiator that
 * Section 4.1 of the paper calls Simulate; Section 4.2, equation for y_sim;
 * Section 4.3, equation for y_sim^(k)), gathers a trace-space gradient back
 * onto every ball parameter (the backpropagation step of Algorithm 1), and
 * filters and grows the cloud (zero-gradient filtering, Section 4.2 and
 * Algorithm 1; destroy / split / duplicate, Section 4.1 and Algorithm 1).
 *
 * Conventions that hold for every entry point:
 *  - Units: positions and radii in mm, time in microseconds, speed of sound
 *    in mm/us, sampling frequency in MHz.
 *  - A ball is (x, y, z, R, p0): centre, radius and initial pressure. A
 *    point cloud is passed as five caller-owned device arrays of float32
 *    (structure of arrays), each at least `n_cap` long.
 *  - The current number of balls lives in DEVICE memory (`n_dev`, int32), so
 *    that growth can change it without a host round trip; every kernel reads
 *    it and the grid is sized from `n_cap`. Passing n_dev = NULL means
 *    "n = n_cap". Balls at and past the live count are ignored, and per-ball
 *    outputs (gradients, Adam moments) are written for the live balls only:
 *    entries past the live count are left as they were.
 *  - Traces are float32 row-major [M][T_k] device arrays owned by the caller.
 *  - All work is enqueued on `stream` (a cudaStream_t passed as void*; NULL
 *    is the legacy default stream); calls do not synchronise unless stated.
 *  - Return value: SBP_OK or a negative sbp_status for argument or launch
 *    errors, detected on the host before anything is enqueued where
 *    possible. Device-side conditions (capacity overflow during growth) are
 *    latched in the array object and reported by sbp_sync_status.
 *  - No C++ exception crosses this boundary. sbp_last_error returns a
 *    thread-local message describing the last failure.
 */
#ifndef SLINGBAG_H
#define SLINGBAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbp_array_s* sbp_array; /* opaque; owned by the library */
typedef void* sbp_stream;              /* cudaStream_t */

typedef enum {
    SBP_OK = 0,
    SBP_ERR_ARG = -1,      /* invalid argument (null pointer, size, level) */
    SBP_ERR_CUDA = -2,     /* a CUDA call or kernel launch failed */
    SBP_ERR_CAPACITY = -3, /* growth would exceed n_cap (device-latched) */
    SBP_ERR_LEVEL = -4,    /* level index out of range */
    SBP_ERR_TIMEOUT = -5,  /* a bounded device wait gave up (sbp_cnn_status; the
                              radiator path has no device waits) */
    SBP_ERR_NUMERIC = -6   /* non-finite input detected */
} sbp_status;

/* Orientation weight w of a (sensor m, ball i) pair with unit normal n_m and
 * unit direction u = (c_i - s_m)/|c_i - s_m|. The paper asks the method to
 * handle "complex transducer orientations" (Section 1) and builds inward
 * normals of the array envelope (Section 4.2) but prints no weighting law;
 * this library reads it as the obliquity factor w = max(0, n.u). */
enum { SBP_W_CLAMP = 0, SBP_W_NONE = 1, SBP_W_COS = 2 };

/* Gradient components (bit mask). The coarse stage of Section 4.1 updates
 * p0 and R only; the fine stage updates all five. SBP_SOFTPLUS_R (only for
 * sbp_adam_step and stages) optimises R through R = softplus(a) with a free
 * variable a, the positivity-constrained refinement of Section 4.3. */
enum { SBP_MASK_P0 = 1, SBP_MASK_R = 2, SBP_MASK_XYZ = 4, SBP_MASK_ALL = 7, SBP_SOFTPLUS_R = 8 };

/* sbp_filter_grow modes. The three zero-gradient rules are the readings of
 * Section 4.2: Algorithm 1 keeps g < 0 (SBP_KEEP_NEG, default), the
 * equations of Section 4.2 keep g <= 0 (SBP_KEEP_NONPOS), and a literal
 * "drop exactly-zero gradients" keeps g != 0 (SBP_DROP_ZERO). SBP_GROW
 * applies the growth rules of sbp_grow_params. */
enum { SBP_KEEP_NEG = 0, SBP_KEEP_NONPOS = 1, SBP_DROP_ZERO = 2, SBP_GROW = 3 };

/* Forward flags. Every forward of this library accumulates traces in
 * fixed-point integers, so it is bitwise reproducible for any launch order;
 * SBP_DETERMINISTIC is accepted for clarity and changes nothing. */
enum { SBP_DETERMINISTIC = 1 };

typedef struct {
    float *x, *y, *z, *R, *p0;
} sbp_balls;

typedef struct {
    float *gx, *gy, *gz, *gR, *gp0;
} sbp_grads;

typedef struct {
    int weight_mode;      /* SBP_W_* (default SBP_W_CLAMP) */
    int reserved[7];
} sbp_params;

/* Growth rules (Section 4.1 / Algorithm 1 name the operations; the paper
 * gives no thresholds or geometry, so these are parameters). For ball i, in
 * this order of precedence:
 *   pruned      if prune_zero and every gradient component selected by
 *               grad_mask is exactly zero;
 *   destroyed   if destroy and (p0 < p_min or R < R_min);
 *   split       if split and R > R_max: two balls at c +- (R/2) v, radius
 *               R * 2^(-1/3), same p0, zero gradients and carried state;
 *   duplicated  if duplicate and gx^2+gy^2+gz^2 > g_dup^2 (evaluated in
 *               double): the ball is kept and followed by a clone at
 *               c + (R/2) v with zero gradients and carried state;
 *   kept        otherwise.
 * v is a unit vector drawn from SplitMix64: three 24-bit draws
 * u_r = mix(seed + (3i + r + 1) * 0x9E3779B97F4A7C15) >> 40, r = 0, 1, 2,
 * mapped to (2 u_r + 1 - 2^24) / 2^24 and normalised. Output order is stable;
 * children take their parent's place. */
typedef struct {
    float p_min, R_min, R_max, g_dup;
    uint64_t seed;
    int grad_mask;
    int prune_zero, destroy, split, duplicate;
} sbp_grow_params;

/* Adam (the paper names no optimizer; Section 2.1 only fixes that both
 * methods use the same learning rates). lr[] is per component in the order
 * x, y, z, R, p0. */
typedef struct {
    float lr[5];
    float beta1, beta2, eps;
} sbp_adam_params;

/* ---------------------------------------------------------------------- */

/* Create a sensor array and its sampling hierarchy (Section 4.3:
 * dt_k = f_k dt, T_k = T / f_k, rounded up when f_k does not divide T).
 *   pos_host, normal_host: host float32 [M][3]; normals need not be unit
 *                          length (they are normalised on the device copy).
 *   M >= 1, c_mm_per_us > 0, fs_mhz > 0, T >= 1.
 *   factors_host: host int32 [n_levels], each >= 1 (e.g. {4, 2, 1}).
 *   n_cap: largest point cloud any later call will pass (sizes scratch).
 *   params: may be NULL (defaults).
 * The library copies the sensors to the device, allocates its scratch for
 * the finest level and returns the handle in *out. The current level is 0. */
int sbp_create_array(const float* pos_host, const float* normal_host, int M,
                     double c_mm_per_us, double fs_mhz, int T, const int* factors_host,
                     int n_levels, int n_cap, const sbp_params* params, sbp_array* out);

int sbp_destroy_array(sbp_array arr);

/* Samples T_k and sampling interval dt_k (us) of level k. */
int sbp_level_info(sbp_array arr, int k, int* T_k, double* dt_k);

/* Select level k (Section 4.3). If y_full_dev is not NULL, also write
 * y_k = Downsample_{f_k}(y_full) into y_k_dev: block means of f_k samples,
 * the record zero-padded to T_k * f_k (reading of the unspecified
 * Downsample operator; under the cell-average sampling of sbp_forward it is
 * exact: the level-k traces are block means of the level-0 traces).
 *   y_full_dev: device float32 [M][T] (finest level), y_k_dev: [M][T_k]. */
int sbp_set_sampling_level(sbp_array arr, int k, const float* y_full_dev, float* y_k_dev,
                           sbp_stream stream);

/* Differentiable radiator at the current level (Section 4.2, y_sim; the
 * model of Section 4.1). Writes S_dev [M][T_k]:
 *   S[m][j] = sum_i p0_i w_mi (E(e_a)^2 - E(e_b)^2) / (4 d_mi c dt_k),
 *   e_a = d_mi - c j dt_k, e_b = e_a - c dt_k, E(e) = clamp(e, -R_i, R_i),
 * i.e. the average over sample cell [j dt_k, (j+1) dt_k) of the uniform-sphere
 * N-wave p0 w (d - c t)/(2 d) on |d - c t| < R. Pairs with d <= R contribute
 * nothing (counted, see sbp_get_inside_pairs); samples outside [0, T_k) are
 * dropped. A live ball with a non-finite x, y, z, R or p0 latches
 * SBP_ERR_NUMERIC (reported by sbp_sync_status; its traces are then not
 * meaningful). flags: 0 or SBP_DETERMINISTIC. */
int sbp_forward(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap, float* S_dev,
                unsigned flags, sbp_stream stream);

/* sbp_forward without any device allocation, for callers that cannot call
 * cudaMalloc: a host that borrows every buffer from a framework owning all
 * allocations (a serving runtime with its own pool), or one held to a fixed
 * device-memory budget. The
 * paper has no counterpart; this is a deployment variant of sbp_forward.
 * It takes no array object: the caller passes the sensors, the level and all
 * inputs and outputs; the scratch (trace accumulators and state words) is a
 * file-scope device array of 2^21 int64 cells plus 256 bytes (16 MiB) that
 * every GPU loading the library holds until the process exits.
 *   sensors_dev: device float32 [6][M]: x, y, z of every sensor, then the
 *                UNIT normals nx, ny, nz (not normalised here).
 *   dt_us = f_k / fs (sampling interval of the level), T_k samples;
 *   weight_mode: SBP_W_*; balls, n_dev, n_cap, S_dev as in sbp_forward.
 * Returns SBP_ERR_ARG when M * T_k exceeds 2^21 cells (use sbp_forward then).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress). Under lazy module loading that look-up loads the
 * library's module, which allocates the 16 MiB array and the module's code:
 * make that first call before any stream capture. The address is kept per
 * device and per context, and looked up again (with the same caveat) when
 * the calling thread's current context is not the one it was taken in, e.g.
 * after cudaDeviceReset.
 * Every call clears the part of the array it uses, and all calls share it:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * corrupt each other's traces; serialise them. */
int sbp_forward_static(const float* sensors_dev, int M, double c_mm_per_us, double dt_us,
                       int T_k, int weight_mode, sbp_balls balls, const int* n_dev, int n_cap,
                       float* S_dev, sbp_stream stream);

/* Residual of the per-level loss L = ||S - y_k||_2^2 (Section 4.2 and 4.3):
 * G = 2 (S - y_k) into G_dev [M][T_k]; if loss_dev is not NULL the loss is
 * written there as one double (a fixed-order reduction, reproducible).
 * S_dev may be NULL, meaning S = 0 (the all-zero-pressure forward of
 * zero-gradient filtering). */
int sbp_residual(sbp_array arr, const float* S_dev, const float* y_k_dev, float* G_dev,
                 double* loss_dev, sbp_stream stream);

/* Adjoint of sbp_forward at the current level: given G = dL/dS [M][T_k],
 * writes every ball's dL/dx, dL/dy, dL/dz, dL/dR, dL/dp0 into `out`
 * (overwritten, each written exactly once; components outside grad_mask are
 * written as zero). Gradients are derived from the forward's closed form
 * (the paper prints none). */
int sbp_adjoint(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                const float* G_dev, sbp_grads out, unsigned grad_mask, sbp_stream stream);

/* Stored windows: the alternative to sbp_adjoint's recomputation of every
 * pair's geometry in the backpropagation step of Algorithm 1 (kept to
 * measure the memory / time trade; sbp_adjoint is the path the loop uses).
 * sbp_store_windows writes, for every (sensor m, ball i) pair of the live
 * balls at the current level, a record into rec_dev: five planes of
 * [M][n_cap] 4-byte words (20 M n_cap bytes, caller-owned device memory,
 * 4-byte aligned): the offset of the first boundary inside the support
 * (float), the orientation weight (float), ~1/d (float), the first and the
 * last boundary inside the support (int; first = -1 when the pair adds
 * nothing, bit 31 of the last set when the weight's derivative is non-zero).
 * sbp_adjoint_stored then computes what sbp_adjoint computes (same
 * gradients up to float summation order, same masks, each live ball's
 * components written once) from those records, G_dev and the cloud, without
 * evaluating distances, windows or weights. The records must come from the
 * same cloud, level and array. SBP_ERR_ARG for null or misaligned pointers. */
int sbp_store_windows(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                      void* rec_dev, sbp_stream stream);
int sbp_adjoint_stored(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                       const void* rec_dev, const float* G_dev, sbp_grads out,
                       unsigned grad_mask, sbp_stream stream);

/* Tile choice of the single-cloud sbp_forward and sbp_adjoint at level k
 * (a launch parameter only: the forward is bitwise identical for every
 * choice, the adjoint differs by float summation order). fwd_chunk: balls
 * per forward CTA, 0 (default: 512, fewer for small clouds) or a power of
 * two in [32, 2048], optionally or'ed with SBP_TILE_WIDE (each CTA holds
 * 832 instead of 416 trace cells per sensor in shared memory and runs 32
 * warps, one CTA per SM: fewer impulses spill to the global accumulators
 * when a chunk spans many cells, at the finest sampling rates); adj_split:
 * adjoint CTAs sharing a ball chunk, each taking a share of the sensors,
 * 0 (default 8), 1, 2, 4 or 8. SBP_ERR_ARG for other values, SBP_ERR_LEVEL
 * for k out of range. */
enum { SBP_TILE_WIDE = 0x10000 };
int sbp_set_tiles(sbp_array arr, int k, int fwd_chunk, int adj_split);
int sbp_get_tiles(sbp_array arr, int k, int* fwd_chunk, int* adj_split);

/* Tile autotuner for the current level: times sbp_forward with the default
 * tile and with 128, 256, 512, 1024 and 2048 balls per CTA and 1024 and
 * 2048 with SBP_TILE_WIDE, and sbp_adjoint (all
 * components) with the default and with 1, 2, 4 and 8 CTAs per ball chunk, on
 * the given cloud; keeps for this level (as sbp_set_tiles would) the
 * fastest choice of each if it beats the default by more than 3%, else the
 * default (reported as 0), and reports them in the optional outputs. S_dev [M][T_k] is overwritten; G_dev [M][T_k] is read only (its
 * values change the timings little: pass a residual of the data). Allocates
 * 5 n_cap floats of scratch and synchronises. On a failed launch the level
 * keeps the defaults and the error is returned. */
int sbp_autotune(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap, float* S_dev,
                 const float* G_dev, int* fwd_chunk_out, int* adj_split_out);

/* Filter and grow the point cloud in place (stable compaction/expansion).
 * mode SBP_KEEP_NEG / SBP_KEEP_NONPOS / SBP_DROP_ZERO: zero-gradient
 * filtering on grads.gp0 (computed by sbp_adjoint with G = -2 y_k, i.e.
 * sbp_residual with S = NULL); p0 itself is untouched, which restores the
 * original pressures of the kept balls as Section 4.2 prescribes.
 * mode SBP_GROW: the rules of sbp_grow_params (gp must not be NULL).
 * Balls, grads and the n_extra carried arrays extra[e] (float32, n_cap each,
 * e.g. Adam moments) are permuted together; *n_dev is updated on the device.
 * If the result would exceed n_cap, nothing changes and SBP_ERR_CAPACITY is
 * latched (see sbp_sync_status). n_extra <= 16. */
int sbp_filter_grow(sbp_array arr, sbp_balls balls, sbp_grads grads, float* const* extra,
                    int n_extra, int* n_dev, int n_cap, const sbp_grow_params* gp, int mode,
                    sbp_stream stream);

/* One Adam step at step count t >= 1 on the components in mask; m and v
 * are the first and second moments, laid out like the balls. With
 * SBP_SOFTPLUS_R in mask (and SBP_MASK_R), the R component is updated in the
 * softplus parameterisation of Section 4.3: a = softplus^-1(R), its gradient
 * sigma(a) dL/dR = (1 - exp(-R)) dL/dR drives the moments, and R becomes
 * softplus(a - step), which is positive for every step. */
int sbp_adam_step(sbp_array arr, sbp_balls balls, sbp_grads grads, sbp_balls m, sbp_balls v,
                  const int* n_dev, int n_cap, int t, const sbp_adam_params* ap,
                  unsigned mask, sbp_stream stream);

/* One reconstruction stage: `iterations` iterations at sampling level
 * `level`, updating the components in grad_mask (coarse stage of Section
 * 4.1: p0 and R; fine stage: all five), followed in every iteration by
 * filter/grow when grow != 0 (duplication only when duplicate != 0, the fine
 * stage of Section 4.1). */
typedef struct {
    int level;
    int iterations;
    unsigned grad_mask; /* may include SBP_SOFTPLUS_R */
    int grow;
    int duplicate;
} sbp_stage;

#define SBP_MAX_STAGES 32

typedef struct {
    int zero_grad_mode;  /* -1: skip; else SBP_KEEP_NEG / SBP_KEEP_NONPOS / SBP_DROP_ZERO */
    int zero_grad_level; /* level whose downsampled data drives the filter */
    int n_stages;
    sbp_stage stages[SBP_MAX_STAGES];
    sbp_adam_params adam;
    sbp_grow_params grow; /* seed of iteration t is grow.seed + t */
    double* loss_log_dev; /* optional: L of every iteration (device doubles) */
    int* n_log_dev;       /* optional: ball count entering every iteration */
    int log_capacity;     /* entries available in the logs */
    int spatial_sort;     /* 1: put the live cloud in Morton order (sbp_sort_cloud) before
                             zero-gradient filtering; single-cloud sbp_reconstruct only
                             (sbp_reconstruct_frames returns SBP_ERR_ARG when it is set) */
} sbp_recon_params;

/* The point-cloud reconstruction loop of Algorithm 1 on the device.
 * A stage whose grad_mask holds SBP_SOFTPLUS_R is the positivity-constrained
 * refinement of Section 4.3: its R moments restart from zero when it begins
 * (the free variable is new), and it should run with grow = 0 (the paper
 * stops adaptive density changes in that phase). */
/* The point-cloud reconstruction loop of Algorithm 1 on the device:
 * zero-gradient filtering at zero_grad_level (Section 4.2), then for every
 * stage and iteration: forward, residual (L = ||S - y_k||^2), adjoint, one
 * Adam step, and filter/grow, with y_k = Downsample_{f_k}(y_full) refreshed at
 * every level change (Section 4.3). The ball count stays on the device
 * throughout; nothing synchronises. Adam moments start at zero and are
 * carried through filtering and growth. The library allocates its scratch
 * (traces, residual, gradients, moments for n_cap balls) on the first call.
 *   y_full_dev: device float32 [M][T]; balls/n_dev: in/out as in
 *   sbp_filter_grow. Convergence tests are left to the caller (the paper's
 *   "until converged" is read as a fixed iteration count per stage). */
int sbp_reconstruct(sbp_array arr, const float* y_full_dev, sbp_balls balls, int* n_dev,
                    int n_cap, const sbp_recon_params* rp, sbp_stream stream);

/* Spatial ordering (no counterpart in the paper; its random initialisation,
 * Section 4.1, leaves the cloud in random order): puts the n_dev live balls
 * in Morton (Z-curve) order of their centres, so that the forward's and the
 * adjoint's chunks of consecutive balls are compact. The key quantises each
 * axis to 10 bits over the live cloud's bounding cube: with lo the
 * componentwise minimum and span the largest extent, q = min(1023,
 * floor((c - lo) * (1024 / span))), each float32 operation rounded once
 * (no fused multiply-add), and the key interleaves the bits of (q_x, q_y,
 * q_z), x lowest. The order is stable (equal keys keep their index order).
 * The n_extra rows of carried state (device float arrays of n_cap, e.g. Adam
 * moments; n_extra <= 21) follow the same permutation. Allocates its key
 * scratch on the first call; nothing synchronises. */
int sbp_sort_cloud(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                   float* const* extra, int n_extra, sbp_stream stream);

/* ---------------------------------------------------------------------- */
/* Batched frames: many acquisitions (e.g. the frames of dynamic imaging) of
 * the same array, reconstructed together. Frame f's balls occupy the slice
 * [off[f], off[f+1]) of one packed cloud (five float32 arrays of the array's
 * n_cap), its live count is n_dev[f] (int32, device), and its traces are the
 * [M][T_k] block f of a [F][M][T_k] float32 array. Every step below runs all
 * frames in one launch per kernel, so an iteration over all frames is a fixed
 * sequence of launches with no host synchronisation (graph-capturable after
 * the first call). Results equal those of the single-cloud calls applied to
 * each frame (growth draws its split direction from the ball's index within
 * its frame). The paper reconstructs one acquisition at a time; batching is
 * a property of this library. */

/* Define the frame layout: frame f gets capacity frame_cap_host[f] rounded
 * up to a multiple of 1024; the padded capacities must fit n_cap. Writes
 * the n_frames + 1 offsets to frame_off_out (host, may be NULL). Allocates
 * per-frame scratch; synchronises the device. */
int sbp_set_frames(sbp_array arr, const int* frame_cap_host, int n_frames, int* frame_off_out);

/* Level select and downsampling of all frames' records ([F][M][T] -> [F][M][T_k]). */
int sbp_set_sampling_level_frames(sbp_array arr, int k, const float* y_full_dev, float* y_k_dev,
                                  sbp_stream stream);

int sbp_forward_frames(sbp_array arr, sbp_balls packed, const int* n_dev, float* S_dev,
                       sbp_stream stream);

/* G = 2 (S - y_k) for all frames; loss_dev (may be NULL) receives one double
 * per frame. S_dev may be NULL (S = 0). */
int sbp_residual_frames(sbp_array arr, const float* S_dev, const float* y_k_dev, float* G_dev,
                        double* loss_dev, sbp_stream stream);

int sbp_adjoint_frames(sbp_array arr, sbp_balls packed, const int* n_dev, const float* G_dev,
                       sbp_grads out, unsigned grad_mask, sbp_stream stream);

/* Filter/grow each frame inside its slice; a frame that would exceed its
 * capacity is left unchanged and SBP_ERR_CAPACITY is latched. */
int sbp_filter_grow_frames(sbp_array arr, sbp_balls packed, sbp_grads grads, float* const* extra,
                           int n_extra, int* n_dev, const sbp_grow_params* gp, int mode,
                           sbp_stream stream);

int sbp_adam_step_frames(sbp_array arr, sbp_balls packed, sbp_grads grads, sbp_balls m,
                         sbp_balls v, const int* n_dev, int t, const sbp_adam_params* ap,
                         unsigned mask, sbp_stream stream);

/* sbp_reconstruct for all frames in lockstep (same schedule). y_full_dev is
 * [F][M][T]; the logs hold F entries per iteration (loss_log_dev[t*F + f]). */
int sbp_reconstruct_frames(sbp_array arr, const float* y_full_dev, sbp_balls packed, int* n_dev,
                           const sbp_recon_params* rp, sbp_stream stream);

/* Tiles of the batched path (the values sbp_autotune_frames chooses, or the
 * caller's own): the forward's balls per CTA, 0 (default: 512) or a power of
 * two in [32, 1024] optionally or'ed with SBP_TILE_WIDE, and the adjoint's
 * CTAs per ball chunk, 0 (default 8), 1, 2, 4 or 8. Launch parameters only:
 * the forward's traces are the same bit for bit for every choice. SBP_ERR_ARG
 * for other values or an array without a frame layout. */
int sbp_set_frame_tiles(sbp_array arr, int fwd_chunk, int adj_split);
int sbp_get_frame_tiles(sbp_array arr, int* fwd_chunk, int* adj_split);

/* Tile autotuner for the batched path: times the forward with 256, 512 and
 * 1024 balls per CTA and 1024 with SBP_TILE_WIDE, and the adjoint with 1, 2, 4 and 8 CTAs per ball chunk on
 * the given cloud at the current level (S_dev, G_dev: [F][M][T_k] scratch of
 * the caller, overwritten), keeps the fastest of each for later batched
 * calls and reports them. Synchronises. */
int sbp_autotune_frames(sbp_array arr, sbp_balls packed, const int* n_dev, float* S_dev,
                        float* G_dev, int* fwd_chunk_out, int* adj_split_out);

/* ------------------------------------------------------------------------
 * Gaussian-profile radiator (Section 4.1: the balls as Gaussian spherical
 * sources of peak p0 and standard deviation a0). The cloud's R row holds
 * the standard deviation a. The initial pressure p0 exp(-r^2 / 2a^2)
 * radiates the outgoing wave p0 w (d - ct) exp(-(d - ct)^2 / 2a^2) / (2d)
 * (far field: pairs with d <= 6a are skipped and counted); sample j of the
 * current level is its cell average
 *     S_j = p0 w a^2 [g(b_{j+1}) - g(b_j)] / (2 d c dt_k),  g(b) = exp(-b^2 / 2a^2),
 * b_j = d - j c dt_k, with the boundaries |b| >= 6a left out. Accumulated in
 * fixed point like sbp_forward (bitwise independent of ball order).
 * ---------------------------------------------------------------------- */

/* Traces S (device [M][T_k], overwritten) of the live balls. Allocates its
 * accumulators on first use per level size (synchronising then). */
int sbp_forward_gauss(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap, float* S_dev,
                      sbp_stream stream);

/* Gradients (x, y, z, a, p0; overwritten, masked as in sbp_adjoint) of
 * sum_j G_j S_j for G_dev = dL/dS ([M][T_k]). */
int sbp_adjoint_gauss(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                      const float* G_dev, sbp_grads out, unsigned grad_mask, sbp_stream stream);

/* ------------------------------------------------------------------------
 * Envelope, initialisation and voxel grid: the steps of Algorithm 1 before
 * and after the iteration (Section 4.1; Algorithm 1, envelope mesh
 * generation, ray-casting initialisation, point cloud to voxel grid).
 * ---------------------------------------------------------------------- */

typedef struct sbp_envelope_s* sbp_envelope; /* opaque; owned by the library */

/* Envelope mesh from the array coordinates: the convex hull of the M sensor
 * positions (pos_host: HOST memory, [M][3] float32, mm), a closed triangle
 * mesh with outward orientation, built on the host in double precision.
 * The paper names no construction: the convex hull is this library's
 * reading. Copies the mesh to the current device. Returns SBP_ERR_ARG for
 * M < 4 or a flat array (a line or plane of sensors), SBP_ERR_NUMERIC for a
 * non-finite coordinate. */
int sbp_envelope_create(const float* pos_host, int M, sbp_envelope* out);
int sbp_envelope_destroy(sbp_envelope env); /* synchronises the device */

/* Face count, enclosed volume (mm^3) and the sensors' bounding box
 * (bbox6 = {xmin, ymin, zmin, xmax, ymax, zmax}); any pointer may be NULL. */
int sbp_envelope_info(sbp_envelope env, int* n_faces, double* volume, double* bbox6);

/* The triangles as sensor indices, [n_faces][3], into host memory. */
int sbp_envelope_faces(sbp_envelope env, int* tri_host);

/* Region test of n points (device SoA x, y, z): inside_dev[i] = 1 when the
 * point is inside the envelope (ray casting: odd number of crossings of a
 * fixed ray, double precision) and at least `inset` mm from its surface (the
 * reconstruction region pulled inward along the normals), else 0. */
int sbp_envelope_classify(sbp_envelope env, const float* x_dev, const float* y_dev,
                          const float* z_dev, long long n, double inset,
                          unsigned char* inside_dev, sbp_stream stream);

/* Random initialisation of the point cloud inside the region. Candidate k
 * takes x, y, z uniform over the sensors' bounding box and R, p0 uniform in
 * [R_lo, R_hi], [p_lo, p_hi], from SplitMix64 outputs 5k .. 5k+4 of the
 * stream seeded with `seed` (each a double lo + (hi - lo) u, u = top 53 bits
 * x 2^-53, rounded to float). Candidates first .. first + n_cand - 1 are
 * tested in order; the first n_want inside the region (see classify) are
 * written to out[0 .. ) and their number to *n_dev (device int). The
 * result depends only on the seed and the candidate range. Allocates its
 * scratch on first use (and when n_cand grows, synchronising then). */
int sbp_envelope_sample(sbp_envelope env, uint64_t seed, long long first, long long n_cand,
                        double inset, double R_lo, double R_hi, double p_lo, double p_hi,
                        sbp_balls out, int n_want, int* n_dev, sbp_stream stream);

/* Point cloud to voxel grid. Voxel (i, j, k) has centre origin + (index +
 * 1/2) spacing and takes the sum of value_dev[b] (NULL: the balls' p0) over
 * the live balls b with |centre - c_b| < R_b; the test is evaluated in
 * double as (dx^2 + dy^2) + dz^2 < R^2. The paper's voxel shader is not
 * specified: this is the uniform-sphere reading. Sums are accumulated in
 * fixed point (2^-F units, F = 40 - ceil(log2 max|value|)), so the grid is
 * independent of ball order. vol_dev: [nz][ny][nx] float32, overwritten.
 * scratch_dev: nx*ny*nz + 1 uint64 words of device memory that must be zero
 * before the first call; every call leaves them zero. n_dev may be NULL
 * (all n_cap balls). */
int sbp_voxelize(sbp_balls balls, const float* value_dev, const int* n_dev, int n_cap,
                 const double* origin3, double spacing, int nx, int ny, int nz,
                 unsigned long long* scratch_dev, float* vol_dev, sbp_stream stream);

/* ------------------------------------------------------------------------
 * Learned initial proposal: the small volume CNN (no counterpart in the
 * paper, which initialises at random and filters by zero gradients; the
 * learned proposal is this library's extension of that step).
 * ---------------------------------------------------------------------- */

/* 3x3x3 convolution with zero padding on a channels-last bf16 volume, on the
 * tensor cores (tcgen05, BF16 x BF16 -> FP32 in tensor memory).
 * in_dev:  bf16 [nz][ny][nx][cin] (device, 16-byte aligned);
 * w_dev:   bf16 [cout][kp], row n holding the weights of output channel n at
 *          k = tap * cin + c, tap = (dz+1)*9 + (dy+1)*3 + (dx+1), zero for
 *          27*cin <= k < kp; kp a multiple of 64;
 * bias_dev: float [cout] or NULL; relu: apply max(., 0) after the bias;
 * out_dev: [nz][ny][nx][cout], bf16 (out_f32 = 0) or float (out_f32 = 1).
 * Supported (cin, cout): (1,16) (16,16) (16,32) (32,32) (32,64) (64,64)
 * (64,32) (32,16). A bounded wait that gives up (a device fault elsewhere)
 * sets the status read by sbp_cnn_status. */
int sbp_conv3d_bf16(const void* in_dev, int nx, int ny, int nz, int cin, const void* w_dev,
                    int kp, const float* bias_dev, int cout, int relu, void* out_dev, int out_f32,
                    sbp_stream stream);

/* Delay-and-sum volume of measured traces (y_full_dev: [M][T] at the
 * array's full rate) on a voxel grid: voxel v (centre origin + (index +
 * 1/2) spacing, [nz][ny][nx]) takes sum_m w_m(v) y_m(|x_v - s_m| / c), the
 * trace interpolated linearly between cell centres (j + 1/2) dt and zero
 * outside the record, w the array's orientation weight (mode of
 * sbp_create_array). vol_dev: float [nz][ny][nx], overwritten. */
int sbp_das_volume(sbp_array arr, const float* y_full_dev, const double* origin3, double spacing,
                   int nx, int ny, int nz, float* vol_dev, sbp_stream stream);

/* The volume CNN of the learned proposal: a delay-and-sum volume scaled to
 * max |.| = 1 (bf16), three 3x3x3 convolutions with ReLU (1 -> 16 -> 32 ->
 * 64 channels, sbp_conv3d_bf16) and a 1x1x1 head with two outputs per voxel
 * (the logit of "a source lies here" and its pressure). Weights are FP32
 * masters (He-normal from `seed`, zero biases) with bf16 copies for the
 * tensor cores; Adam state; activation buffers for one nx x ny x nz volume
 * (allocated here). */
typedef struct sbp_cnn_s* sbp_cnn;
int sbp_cnn_create(int nx, int ny, int nz, uint64_t seed, sbp_cnn* out);
int sbp_cnn_destroy(sbp_cnn cnn); /* synchronises the device */
int sbp_cnn_num_params(void);
/* Copy the FP32 parameters to (set = 0) or from (set = 1) host memory
 * (sbp_cnn_num_params floats: w1, b1, w2, b2, w3, b3, head w, head b, each
 * weight [cout][27][cin] or [2][32]). Synchronises. */
int sbp_cnn_params(sbp_cnn cnn, float* host, int set);
/* Forward pass; out_dev (float [V][2]: logit, pressure) may be NULL. */
int sbp_cnn_forward(sbp_cnn cnn, const float* vol_dev, float* out_dev, sbp_stream stream);
/* One Adam step (lr, beta = 0.9 / 0.999) on the loss
 *   mean_v [ pos_weight t log(1 + e^-z) + (1 - t) log(1 + e^z) ]
 *     + mean_v [ t (q - p)^2 ]
 * for targets t = occ_dev (0/1) and p = p0_dev (float [V]); loss_dev
 * (double [2]: the two terms) may be NULL. The weight gradients are GEMMs
 * over voxels on the tensor cores, added in a fixed order: a step is
 * reproducible bit for bit. */
int sbp_cnn_train_step(sbp_cnn cnn, const float* vol_dev, const float* occ_dev, const float* p0_dev,
                       float pos_weight, float lr, double* loss_dev, sbp_stream stream);
/* The gradient of that loss with respect to every FP32 parameter, written to
 * grad_dev (device, sbp_cnn_num_params floats, the layout of
 * sbp_cnn_params), without changing the parameters; loss_dev as above (may
 * be NULL). Reproducible bit for bit. */
int sbp_cnn_grad(sbp_cnn cnn, const float* vol_dev, const float* occ_dev, const float* p0_dev,
                 float pos_weight, double* loss_dev, float* grad_dev, sbp_stream stream);
/* Proposal: forward pass, then per_voxel balls (1 .. 4096) in every voxel v
 * with sigmoid(z) > prob_threshold, in voxel order, ball j of voxel v at a
 * uniformly random point of the voxel (SplitMix64 of `seed`, outputs
 * 3 (v per_voxel + j) .. + 2), radius R, pressure q clamped to
 * [p_min, p_max]. Writes at most n_cap balls and their number to *n_dev
 * (device int). Allocates scratch on first use (synchronising then). */
int sbp_cnn_propose(sbp_cnn cnn, const float* vol_dev, float prob_threshold, uint64_t seed,
                    const double* origin3, double spacing, float R, float p_min, float p_max,
                    int per_voxel, sbp_balls out, int n_cap, int* n_dev, sbp_stream stream);

/* Synchronise `stream` and return (then clear) the convolution status:
 * 0 = fine, SBP_ERR_TIMEOUT = a bounded wait of the tensor-core
 * convolution gave up (the CTA freed its tensor memory and returned). */
int sbp_cnn_status(sbp_stream stream, int* status);

/* Number of CUDA kernels this library has launched in this process. */
long long sbp_launch_count(void);

/* Synchronise `stream`, then return SBP_OK or the first device-latched
 * status since the last call (which is cleared). */
int sbp_sync_status(sbp_array arr, sbp_stream stream);

/* Pairs with d <= R skipped so far (synchronises `stream`). */
int sbp_get_inside_pairs(sbp_array arr, sbp_stream stream, long long* count);

/* Thread-local description of the last error (never NULL). */
const char* sbp_last_error(void);

/* Library version string. */
const char* sbp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SLINGBAG_H */
