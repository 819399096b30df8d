/* air.h -- C ABI of the GB300 adaptive image ray-tracing (AIR) library.
 *
 * Method: E. R. Parkin (2010), "Adaptive image ray-tracing for astrophysical
 * simulations" (MNRAS Letters; arXiv:1010.5534).
 *
 * Conventions for every entry point
 *   - Plain C types only; no exceptions cross the ABI. Every call returns an
 *     air_status; on failure air_last_error() gives a message (thread-local,
 *     valid until the next call on the same thread).
 *   - Device work is ordered on the handle's CUDA stream (air_set_stream).
 *     Calls that return results to the caller synchronise that stream before
 *     returning; inputs are copied, the caller keeps ownership of its arrays.
 *   - Buffers of an air_image are host or device memory, as its `mem` field
 *     says; they are caller-owned and caller-sized (`capacity` entries). Host
 *     arrays are filled from device staging arrays by copies (page-locked
 *     arrays, from cudaHostAlloc or cudaHostRegister, take them at the copy
 *     engines' full rate). They are complete when the call returns.
 *   - Images are orthographic (the paper's observer is at 1 kpc from a box of
 *     1e18 cm, Section 3). Pixel (L, i, j) of an n0 x n0 base image has its
 *     centre at u = -H + (i + 1/2) 2H / (n0 2^L), v likewise with j, where the
 *     image basis is u = normalize(up x dir), v = dir x u and H = half_extent.
 *   - Cells are half-open [x_k, x_k+1): a ray lying exactly on a cell face
 *     samples the cell of higher index.
 */
#ifndef AIR_H
#define AIR_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define AIR_API __attribute__((visibility("default")))
#else
#define AIR_API
#endif

typedef enum {
  AIR_OK = 0,
  AIR_ERR_ARG = 1,      /* invalid argument or input field value */
  AIR_ERR_OOM = 2,      /* device or host allocation failed */
  AIR_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  AIR_ERR_CAPACITY = 4, /* output arrays too small: n_out holds the size needed */
  AIR_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
  AIR_ERR_NUMERIC = 6   /* non-finite result */
} air_status;

typedef enum { AIR_GRID_UNIFORM = 0, AIR_GRID_AMR = 1 } air_grid_kind;
typedef enum { AIR_F32 = 0, AIR_F64 = 1 } air_dtype;
typedef enum { AIR_HOST = 0, AIR_DEVICE = 1 } air_mem;

/* Simulation grid (Section 2 step i; Section 3: FLASH/PARAMESH block AMR).
 * Uniform: n[0] x n[1] x n[2] cells over the box [lo, hi]; fields laid out
 *   [n2][n1][n0], x fastest.
 * Block AMR: n[] base cells per axis, cut into cubic bricks of `brick` cells
 *   (a power of two dividing every n[a]); `max_level` refinement levels by a
 *   factor 2. Only LEAF bricks are given: brick b sits at level brick_level[b]
 *   with its lowest corner at brick_origin[3b..3b+2] in units of the finest
 *   cell (n[a] << max_level per axis); the leaf bricks must tile the box
 *   exactly. Fields are [n_bricks][brick][brick][brick], x fastest.
 * Emission (Section 1: column density and emergent intensity): per band b,
 *   emissivity j_b = rho^2 Lambda_b(T) (emis_mode 1) or rho^2 (emis_mode 0),
 *   absorption coefficient alpha_b = kappa[b] rho. Lambda_b is tabulated at
 *   n_tbins points uniform in log10 T over [logT_lo, logT_hi] and interpolated
 *   linearly in log10 T, clamped at both ends.
 * Fields must be finite, rho >= 0 and T > 0 (checked on the device). */
typedef struct {
  int32_t kind;          /* air_grid_kind */
  int32_t n[3];
  double lo[3], hi[3];
  int32_t brick, max_level, n_bricks;
  const int32_t *brick_level;   /* [n_bricks], host memory */
  const int32_t *brick_origin;  /* [n_bricks][3], host memory */
  int32_t field_dtype;          /* air_dtype of rho and temp */
  const void *rho;              /* host memory */
  const void *temp;             /* host memory; may be NULL when emis_mode == 0 */
  int32_t n_bands, emis_mode;
  const float *lambda_table;    /* [n_bands][n_tbins], host memory */
  int32_t n_tbins;
  double logT_lo, logT_hi;
  const double *kappa;          /* [n_bands], host memory */
} air_grid_desc;

typedef struct {
  double dir[3];      /* direction the rays travel (need not be normalised) */
  double up[3];       /* must not be parallel to dir */
  double center[3];   /* world point at the image centre */
  double half_extent; /* H > 0 */
} air_view;

/* Adaptive image parameters (Section 2 steps iii-v; Section 3 Eq. 1, Eq. 2). */
typedef struct {
  int32_t base_res;   /* n0: base image n0 x n0 (step i) */
  int32_t max_level;  /* maximum image refinement level, n0 << max_level <= 2^20 */
  double xi_crit;     /* refine a pixel when xi >= xi_crit (>= 0) */
  int32_t xi_norm;    /* Eq. 2 denominator: 0 = sum over the axis u only (reduces to
                         Eq. 1 in 1-D, bounded by 1), 1 = literal sum over u and v */
  int32_t refine_on;  /* parameter p: 0 = band-summed intensity, 1 = column density,
                         2 = refine when either parameter is flagged */
  int32_t fp64_level; /* AMR bricks at this level or deeper get FP64 entry/exit
                         parameters; negative = library default (3) */
  int32_t include_interior; /* 0: output the leaf pixels (the final image);
                               1: output every traced pixel, interior ones too */
} air_params;

/* Output image: one entry per pixel. Leaves (or all traced nodes) come in
 * creation order: the base image row-major, then, sweep by sweep, the four
 * children of each refined pixel (child c at (2i + (c & 1), 2j + (c >> 1))) in
 * the order of their parents. Optional arrays may be NULL. */
typedef struct {
  int32_t mem;         /* air_mem of every array below */
  int64_t capacity;    /* entries available in each per-pixel array */
  int64_t n_out;       /* out: entries written (or needed, on AIR_ERR_CAPACITY) */
  int64_t n_leaves;    /* out: leaf pixels of the final image */
  int64_t n_rays;      /* out: traced rays = all tree nodes (Table 1 "Pixels") */
  int64_t n_steps;     /* out: ray-cell segments marched, summed over all rays */
  int32_t n_sweeps;    /* out: refinement sweeps that refined something */
  int32_t *level;      /* [capacity] optional */
  int32_t *i, *j;      /* [capacity] optional */
  uint8_t *is_leaf;    /* [capacity] optional */
  float *coldens;      /* [capacity] column density, optional */
  float *intensity;    /* [n_bands][capacity] band-major, optional */
  float *p;            /* [capacity] band-summed intensity as used by the scan, optional */
  double *band_flux;   /* [n_bands] sum over leaves of I_b x pixel area, optional */
} air_image;

/* Launch configuration of a grid handle (air_autotune, air_set_tuning). Every
 * field only changes how work maps to GPU threads, never the results; 0 means
 * the library default. */
typedef struct {
  int32_t tile_w;                 /* fixed images: a warp traces tile_w x (32 / tile_w)
                                     pixels (1, 2, 4, 8, 16, 32; default 8) */
  int32_t bands_per_thread;       /* single-view renders: bands one thread carries
                                     along a ray (1, 2, 4, 8, 16; default: all of them up to 8 bands, else 8) */
  int32_t batch_bands_per_thread; /* batched renders (default 8 for more than 4 bands) */
  int32_t batch_blocks_per_sm;    /* persistent CTAs per SM of batched renders
                                     (default: as many as fit) */
  double best_ms[3];              /* out of air_autotune: fixed, adaptive, batched time */
  int32_t trials;                 /* out of air_autotune: configurations timed */
} air_tuning;

typedef struct air_grid air_grid;

/* Copy a grid to the device and build its brick lookup (Section 2 step i).
 * `stream` is a cudaStream_t (NULL = legacy default stream). On success *out
 * owns the device copy until air_free. */
AIR_API air_status air_load_grid(const air_grid_desc *desc, void *stream, air_grid **out);

/* Change the stream later calls on this handle are ordered on. */
AIR_API air_status air_set_stream(air_grid *g, void *stream);

/* Fixed-resolution image (the paper's comparison arm, Section 3 / Table 1):
 * one ray per pixel of a res x res image, output row-major (pixel (i, j) at
 * entry j * res + i, level 0). `fp64_level` as in air_params. */
AIR_API air_status air_render_fixed(air_grid *g, const air_view *view, int32_t res, int32_t fp64_level,
                            air_image *out);

/* Adaptive image (Section 2 steps i-vi): trace the base image, then repeat
 * {scan every leaf below max_level with Eq. 2, flag xi >= xi_crit, extend the
 * flags so adjacent pixels differ by at most one level, split every flagged
 * pixel into four and trace the new rays} until no pixel is flagged. */
AIR_API air_status air_render_adaptive(air_grid *g, const air_view *view, const air_params *params,
                               air_image *out);

/* Options of a batched render. Zero-initialise and set what you need, or pass
 * NULL for the defaults. */
typedef struct {
  int32_t bands_per_thread;   /* bands one thread carries along a ray: 1, 2, 4, 8 or 16;
                                 0 = library default (8 for more than 4 bands) */
  int32_t use_graph;          /* 1: launch through a CUDA graph captured on first use
                                 (re-captured when the configuration changes) */
  double wait_timeout_ms;     /* time limit of every device-side wait of the persistent
                                 kernel (grid barriers); <= 0 means 2000 ms. A wait that
                                 runs out makes the call return AIR_ERR_TIMEOUT. */
  int32_t test_stall_barrier; /* fault test: the first grid barrier waits for one block
                                 more than is launched, so it must run out (0 in use) */
} air_batch_opts;

/* Batched adaptive images (Section 2 steps i-vi for every view): n_views views
 * of one grid, each with all the grid's bands, each refined on its own image,
 * rendered by one cooperative persistent kernel that runs every sweep of every
 * view (a work queue of (ray, band chunk) items for the march; scan, balance
 * and a per-view prefix sum between grid barriers), launched through a CUDA
 * graph. outs[v] receives view v exactly as air_render_adaptive would (same
 * pixels, same order); band fluxes are summed with FP64 atomics (equal to the
 * single-view result up to FP64 summation order). The views share params
 * (and the image half-extent used for pixel areas is per view). At most 256
 * views; every view's node list shares the handle's workspace, grown (and the
 * render repeated) when a batch does not fit. */
AIR_API air_status air_render_batch(air_grid *g, const air_view *views, int32_t n_views,
                                    const air_params *params, const air_batch_opts *opts,
                                    air_image *outs);

/* ---- One image over several processes (Section 2, parallelisation) ---------
 * The paper distributes the pixels of each ray-tracing sweep over the
 * processors and gathers the traced values for the refinement check. Here
 * every process (rank) holds the grid and runs the refinement itself on the
 * gathered values, so all ranks build the same quadtree: the new rays of each
 * sweep, nodes [first, first + count) in creation order, are split into
 * `world` contiguous slices, rank r traces nodes
 * [first + count r / world, first + count (r + 1) / world), and `exchange` is
 * called to fill in the other ranks' slices.
 * exchange(user, first, count, n_bands, coldens, intensity, stride, p, steps):
 *   the arrays are device memory of the library's quadtree (node k at
 *   coldens[k], intensity[b * stride + k], p[k], steps[k]); on entry this
 *   rank's slice is complete (the handle's stream has been synchronised), on
 *   return every node of [first, first + count) must hold its traced values,
 *   written or queued on the handle's stream. Return 0, or nonzero to abort
 *   the render (AIR_ERR_ARG). It is called once per sweep, the base image
 *   included, on the calling thread. */
typedef int32_t (*air_exchange_fn)(void *user, int64_t first, int64_t count, int32_t n_bands,
                                   float *coldens, float *intensity, int64_t stride, float *p,
                                   uint32_t *steps);
typedef struct {
  int32_t rank, world;      /* 0 <= rank < world */
  air_exchange_fn exchange; /* required when world > 1 */
  void *user;
} air_shard;

/* air_render_adaptive with the rays of every sweep split over `world` ranks
 * (see air_shard). Every rank must make the same call (same grid contents,
 * view and params); each returns the whole image, bitwise equal to
 * air_render_adaptive's. Errors: as air_render_adaptive; AIR_ERR_ARG for a
 * bad rank / world, a missing exchange, or an exchange that failed. */
AIR_API air_status air_render_adaptive_sharded(air_grid *g, const air_view *view,
                                               const air_params *params, const air_shard *shard,
                                               air_image *out);

/* ---- Learned refinement-depth proposal (not in the paper) ------------------
 * A perceptron 16 -> 64 -> 64 -> 5 (ReLU) with BF16 weights and activations and
 * FP32 accumulation predicts, per base pixel, the depth (0..4) plain AIR will
 * refine it to. Parameters are FP32 master copies in one flat array:
 * W1[16][64], b1[64], W2[64][64], b2[64], W3[64][5], b3[5] (input index first).
 * Features are 16 BF16 values per sample (uint16 bit patterns). */
#define AIR_MLP_NIN 16
#define AIR_MLP_NHIDDEN 64
#define AIR_MLP_NOUT 5
#define AIR_MLP_NPARAMS (16 * 64 + 64 + 64 * 64 + 64 + 64 * 5 + 5)
typedef struct air_mlp air_mlp;

/* New network on `stream`; params (host, AIR_MLP_NPARAMS floats) or NULL for zeros. */
AIR_API air_status air_mlp_create(const float *params, void *stream, air_mlp **out);
AIR_API air_status air_mlp_set_stream(air_mlp *m, void *stream);
/* Copy the parameters out (get, host) and/or replace them (set, host; resets Adam). */
AIR_API air_status air_mlp_params(air_mlp *m, float *get, const float *set);
/* logits[n][5] (device) for features x[n][16] (device). */
AIR_API air_status air_mlp_forward(air_mlp *m, const uint16_t *x, int64_t n, float *logits);
/* Mean softmax cross-entropy over n samples with labels y (device, 0..4); its
 * gradient to grad (device, AIR_MLP_NPARAMS floats, may be NULL), the loss to
 * *loss (host, may be NULL). */
AIR_API air_status air_mlp_loss_grad(air_mlp *m, const uint16_t *x, const int32_t *y, int64_t n,
                                     float *grad, double *loss);
/* `epochs` passes of minibatch Adam (beta 0.9/0.999, eps 1e-8, learning rate lr)
 * over the n samples; loss_history[e] (host, may be NULL) = mean loss of epoch e. */
AIR_API air_status air_mlp_train(air_mlp *m, const uint16_t *x, const int32_t *y, int64_t n,
                                 int32_t batch, int32_t epochs, float lr, double *loss_history);
AIR_API void air_mlp_free(air_mlp *m);

/* Training samples of one view, four per base pixel: sample 4 b + q stands
 * for quadrant q (level-1 pixel (2 bi + (q & 1), 2 bj + (q >> 1))) of base
 * pixel b = bj * n0 + bi. x[4*n0*n0][16] (device, BF16 bits) receives the 16
 * features of every sample and, if y is not NULL, y[4*n0*n0] (device) the
 * deepest level plain AIR reaches below the sample's level-1 pixel (0 when
 * the base pixel is not refined, 1 when that level-1 pixel is a leaf), taken
 * from a plain render with `params`. */
AIR_API air_status air_learn_samples(air_grid *g, const air_view *view, const air_params *params,
                                     uint16_t *x, int32_t *y);

typedef struct {
  double quantile; /* propose the smallest depth whose predicted cumulative
                      probability reaches this (0 < q <= 1; 0 = default 0.8) */
} air_learned_opts;

typedef struct {
  int64_t proposed_rays;   /* traced in the proposal wave */
  int64_t used_rays;       /* of those, pixels plain AIR created */
  int64_t wasted_rays;     /* proposed but not part of the image's tree */
  int64_t fallback_rays;   /* pixels the proposal missed, traced afterwards */
  int32_t waves;           /* march launches: base + proposal + fallback waves */
  int32_t sweeps;          /* refinement sweeps (as plain AIR) */
  int64_t under_predicted; /* quadrant samples whose final depth exceeded the proposal */
  int64_t over_predicted;  /* quadrant samples proposed deeper than needed */
} air_learned_stats;

/* Adaptive image with the learned proposal: trace the base image, run the
 * network on the features of every base pixel's four quadrants, trace every
 * pixel of the proposed subtrees (each quadrant to its proposed depth) in one
 * wave, then run plain AIR (Section 2 steps iii-v) taking pixel values from
 * that wave, tracing only the pixels it missed. The image (pixels, order,
 * values) is identical to air_render_adaptive's; stats may be NULL. */
AIR_API air_status air_render_learned(air_grid *g, const air_view *view, const air_params *params,
                                      air_mlp *mlp, const air_learned_opts *opts, air_image *out,
                                      air_learned_stats *stats);

/* Batched adaptive images with the learned proposal: air_render_batch with
 * the proposal of air_render_learned for every view. The base images of all
 * views are traced by the persistent kernel; the network proposes a depth for
 * every quadrant of every base pixel of every view; a second persistent launch traces every
 * view's proposal wave from one work queue and then runs the sweeps of every
 * view, taking a new pixel's values from its view's wave where the wave
 * traced it and tracing the pixels the proposal missed. outs[v] is bitwise
 * the image air_render_batch (and air_render_adaptive) gives; stats (may be
 * NULL) sums over the views: proposed_rays, used_rays, wasted_rays,
 * fallback_rays, sweeps = the most of any view, waves = 2 launches. No CUDA
 * graph is used (opts->use_graph is ignored). Errors: as air_render_batch and
 * air_render_learned. */
AIR_API air_status air_render_batch_learned(air_grid *g, const air_view *views, int32_t n_views,
                                            const air_params *params, const air_batch_opts *opts,
                                            air_mlp *mlp, const air_learned_opts *lopts,
                                            air_image *outs, air_learned_stats *stats);

/* Autotuner (not in the paper): time candidate launch configurations on this
 * grid with this view and parameters (fixed image of up to 2048^2 pixels,
 * adaptive image, and, if n_views_batch > 0, a batch of that many copies of the
 * view), keep the fastest per knob in the handle and return it in *out (may be
 * NULL). Later renders on the handle use it. */
AIR_API air_status air_autotune(air_grid *g, const air_view *view, const air_params *params,
                                int32_t n_views_batch, air_tuning *out);
AIR_API air_status air_set_tuning(air_grid *g, const air_tuning *t);
AIR_API air_status air_get_tuning(air_grid *g, air_tuning *t);

/* Phase profiling: when enabled, every kernel launch group of a render is
 * bracketed by CUDA events on the handle's stream, and the elapsed device time
 * is added per phase when the render completes. Enabling resets the counters. */
enum {
  AIR_PHASE_MARCH = 0,   /* ray march (Section 2 step ii) */
  AIR_PHASE_SCAN = 1,    /* truncation-error scan, Eq. 2 (step iii) */
  AIR_PHASE_BALANCE = 2, /* 2:1 level balance (step iii) */
  AIR_PHASE_REFINE = 3,  /* prefix sum + child emission (step iv) */
  AIR_PHASE_OUTPUT = 4,  /* leaf compaction + band flux (step vi) */
  AIR_PHASE_BATCH = 5,   /* the batched persistent kernel (all sweeps, all views) */
  AIR_PHASE_LEARN = 6,   /* features, network, proposal layout, gathers */
  AIR_N_PHASES = 7
};
AIR_API air_status air_profile_enable(air_grid *g, int32_t on);
/* ms[p]: summed device milliseconds, launches[p]: kernel launches, for each
 * phase p < AIR_N_PHASES (either pointer may be NULL). */
AIR_API air_status air_profile_read(air_grid *g, double *ms, int64_t *launches);

/* Adaptive image whose per-node spectra go to host memory sweep by sweep
 * instead of staying on the device. Section 2 notes that an integrated
 * spectrum needs every pixel's spectrum kept until the calculation ends, and
 * that writing them out during the calculation bounds the memory this takes.
 * As air_render_adaptive, with params->include_interior = 1 required (the
 * spectra are indexed by node, and out lists every traced node in creation
 * order) and out->intensity NULL (not written). spectra: caller-owned
 * page-locked host memory (cudaHostAlloc or cudaHostRegister), spectra_cap
 * nodes x n_bands floats; node k's band b is spectra[b * spectra_cap + k].
 * On the device each sweep's spectra go to one of two staging buffers, and a
 * second stream copies them to `spectra` while the next sweep's scan and
 * refinement run; the quadtree keeps only the band-summed intensity and the
 * column density, so device memory no longer grows with n_bands x nodes.
 * band_flux is computed by a kernel that reads `spectra` from host memory.
 * The call returns after `spectra` and out are complete.
 * Errors: as air_render_adaptive; AIR_ERR_ARG if spectra is not page-locked
 * or include_interior != 1 or out->intensity is set; AIR_ERR_CAPACITY if
 * spectra_cap is smaller than the number of traced nodes (out->n_rays set;
 * the spectra are then incomplete) or out->capacity is too small. */
AIR_API air_status air_render_adaptive_spectra(air_grid *g, const air_view *view,
                                               const air_params *params, air_image *out,
                                               float *spectra, int64_t spectra_cap);

/* Finest-level raster of the most recent single-view adaptive image on this
 * handle (air_render_adaptive or air_render_learned; a batched render or
 * air_free ends it). Section 2 step vi allows the output image's edges to be
 * sharpened by interpolating between adjacent pixels of differing resolution
 * (a super-resolution step; the paper fixes no method). With base n0 and
 * max level Lm of that render, out holds (n0 2^Lm)^2 floats, row-major
 * [y][x], y along v:
 *   AIR_RASTER_NEAREST : each finest pixel takes the value of its leaf;
 *   AIR_RASTER_BILINEAR: with L the level of that leaf, the pixel centre is
 *     placed on the level-L pixel grid, u = (x + 1/2) 2^(L - Lm) - 1/2 (v
 *     likewise), and the value is the bilinear interpolation between the
 *     four level-L pixels floor(u) + {0,1} x floor(v) + {0,1}, indices
 *     clamped to the image; a level-L pixel's value is that of the deepest
 *     traced node at level <= L covering it (the refinement scan's neighbour
 *     rule). Finest-level leaves keep their values exactly.
 * quantity: AIR_RASTER_INTENSITY (band `band`), AIR_RASTER_SUM (band-summed
 * intensity), AIR_RASTER_COLDENS (column density). out: device or host
 * memory (detected), caller-owned, n_out floats. Computed in FP32 on the
 * handle's stream; the call returns after out is written.
 * Errors: AIR_ERR_ARG (NULL out, unknown quantity or mode, band out of range,
 * no image to rasterise), AIR_ERR_CAPACITY (n_out < (n0 2^Lm)^2; nothing is
 * written), AIR_ERR_CUDA. */
enum { AIR_RASTER_NEAREST = 0, AIR_RASTER_BILINEAR = 1 };
enum { AIR_RASTER_INTENSITY = 0, AIR_RASTER_SUM = 1, AIR_RASTER_COLDENS = 2 };
AIR_API air_status air_render_raster(air_grid *g, int32_t quantity, int32_t band, int32_t mode,
                                     float *out, int64_t n_out);

/* Band flux of an image already in device memory, computed without allocating
 * any memory. The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc when they need the flux -- a real-time or serving loop
 * that must not stall the device (cudaFree synchronises it), a plugin whose
 * host application owns all device memory through its own pool, or code that
 * runs where the CUDA runtime forbids allocation.
 *   band_flux[b] = sum over entries k < n with is_leaf[k] != 0 (every entry if
 *   is_leaf is NULL) of intensity[b * stride + k] * area0 / 4^level[k]
 *   (level 0 if level is NULL); area0 is the pixel area at level 0, e.g.
 *   (2H / base_res)^2. The result matches the band_flux of the render that
 *   produced the arrays up to FP64 summation order. Every counted level[k]
 *   must lie in [0, 20] (the levels a render can produce); a counted entry
 *   outside that range makes every band_flux entry NaN.
 * All arrays are device memory of the current device (checked; managed memory
 * is accepted); the work is queued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and band_flux is valid once the
 * stream reaches that point; the call does not synchronise.
 * Scratch: a fixed 512 KiB device array inside this library (1024 partial sums
 * x 64 bands), which every GPU that loads the library holds until the process
 * exits. Limits: 1 <= n_bands <= 64, 0 <= n <= 2^31 - 1, n <= stride, and
 * (n_bands - 1) * stride + n within int64; other requests fail with
 * AIR_ERR_ARG. The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. The address is kept until the process
 * exits, so do not call this across a cudaDeviceReset. Every call shares the array and
 * overwrites the partial sums it uses, so nothing needs clearing, but calls
 * whose work overlaps on the GPU (other streams, other threads) race on it. */
AIR_API air_status air_band_flux_static(const float *intensity, int64_t stride, int32_t n_bands,
                                        const int32_t *level, const uint8_t *is_leaf, int64_t n,
                                        double area0, double *band_flux, void *stream);

/* Release the device copy and every buffer the handle holds. NULL is a no-op. */
AIR_API void air_free(air_grid *g);

/* Message for the last failing call on this thread ("" if none). */
AIR_API const char *air_last_error(void);

/* Library version string. */
AIR_API const char *air_version(void);

#ifdef __cplusplus
}
#endif
#endif
