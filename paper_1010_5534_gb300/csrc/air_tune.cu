// air_tune.cu -- autotuner of the launch configuration (not in the paper).
// Times candidate configurations on the caller's own grid and view, with
// CUDA events on the handle's stream, and keeps the fastest per knob:
//   tile_w                 : fixed images, a warp traces tile_w x (32 / tile_w) pixels;
//   bands_per_thread       : single-view renders, bands one thread carries
//                            along a ray (fewer -> more threads per ray);
//   batch_bands_per_thread : the same for the batched persistent kernel;
//   batch_blocks_per_sm    : persistent CTAs per SM of the batched kernel.
// Every knob only changes how work maps to threads: results are bitwise the
// same under every configuration.
#include <cstring>
#include <vector>

#include "air_handle.cuh"

namespace air {

#define CU_TRY(x)                                    \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

// Time fn() twice on the handle's stream, return the faster (ms).
template <class Fn>
static air_status time_best(air_grid *g, Fn fn, double *ms) {
  cudaEvent_t a, b;
  CU_TRY(cudaEventCreate(&a));
  CU_TRY(cudaEventCreate(&b));
  double best = 1e300;
  for (int rep = 0; rep < 2; ++rep) {
    CU_TRY(cudaEventRecord(a, g->stream));
    air_status s = fn();
    if (s) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return s;
    }
    CU_TRY(cudaEventRecord(b, g->stream));
    CU_TRY(cudaEventSynchronize(b));
    float t = 0.f;
    CU_TRY(cudaEventElapsedTime(&t, a, b));
    if (t < best) best = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = best;
  return AIR_OK;
}

air_status autotune(air_grid *g, const air_view *view, const air_params *pr, int32_t n_views,
                    air_tuning *out) {
  if (!view || !pr) return set_error(AIR_ERR_ARG, "view and params must not be NULL");
  if (n_views < 0 || n_views > 256) return set_error(AIR_ERR_ARG, "n_views_batch must be in [0, 256]");
  const int nb = g->gv.n_bands;
  air_tuning best = g->tune;
  int trials = 0;
  air_status s;
  // fixed images: warp tile shape (at most 2048^2 pixels)
  {
    int64_t res = (int64_t)pr->base_res << pr->max_level;
    if (res > 2048) res = 2048;
    double tbest = 1e300;
    for (int tw : {4, 8, 16, 32}) {
      g->tune.tile_w = tw;
      air_image im{};
      im.mem = AIR_DEVICE;
      im.capacity = res * res;
      double ms;
      s = time_best(g, [&] { return render_fixed(g, view, (int32_t)res, pr->fp64_level, &im); }, &ms);
      if (s) return s;
      ++trials;
      if (ms < tbest) {
        tbest = ms;
        best.tile_w = tw;
      }
    }
    best.best_ms[0] = tbest;
    g->tune.tile_w = best.tile_w;
  }
  // single-view adaptive image: bands per thread
  {
    double tbest = 1e300;
    for (int bpt : {1, 2, 4, 8, 16}) {
      if (bpt > 1 && bpt / 2 >= nb) break;
      g->tune.bands_per_thread = bpt;
      air_image im{};
      im.mem = AIR_DEVICE;
      im.capacity = INT64_MAX / 4;  // no arrays: only counts and flux are produced
      double ms;
      s = time_best(g, [&] { return render_adaptive(g, view, pr, &im); }, &ms);
      if (s) return s;
      ++trials;
      if (ms < tbest) {
        tbest = ms;
        best.bands_per_thread = bpt;
      }
    }
    best.best_ms[1] = tbest;
    g->tune.bands_per_thread = best.bands_per_thread;
  }
  // batched images: bands per thread x persistent CTAs per SM
  if (n_views > 0) {
    std::vector<air_view> vs(n_views, *view);
    std::vector<air_image> ims(n_views);
    double tbest = 1e300;
    for (int bpt : {1, 2, 4, 8, 16}) {
      if (bpt > 1 && bpt / 2 >= nb) break;
      for (int per : {0, 1, 2}) {
        g->tune.batch_bands_per_thread = bpt;
        g->tune.batch_blocks_per_sm = per;
        for (auto &im : ims) {
          std::memset(&im, 0, sizeof(im));
          im.mem = AIR_DEVICE;
          im.capacity = INT64_MAX / 4;
        }
        air_batch_opts op{};
        op.use_graph = 1;
        op.wait_timeout_ms = 2000.0;
        double ms;
        s = time_best(g, [&] { return render_batch(g, vs.data(), n_views, pr, &op, ims.data()); }, &ms);
        if (s) return s;
        ++trials;
        if (ms < tbest) {
          tbest = ms;
          best.batch_bands_per_thread = bpt;
          best.batch_blocks_per_sm = per;
        }
      }
    }
    best.best_ms[2] = tbest;
  }
  best.trials = trials;
  g->tune = best;
  if (out) *out = best;
  return AIR_OK;
}

}  // namespace air

extern "C" {

air_status air_autotune(air_grid *g, const air_view *view, const air_params *params,
                        int32_t n_views_batch, air_tuning *out) {
  air::set_error(AIR_OK, "");
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  return air::autotune(g, view, params, n_views_batch, out);
}

air_status air_set_tuning(air_grid *g, const air_tuning *t) {
  air::set_error(AIR_OK, "");
  if (!g || !t) return air::set_error(AIR_ERR_ARG, "grid and tuning must not be NULL");
  const int tw = t->tile_w;
  if (tw != 0 && tw != 1 && tw != 2 && tw != 4 && tw != 8 && tw != 16 && tw != 32)
    return air::set_error(AIR_ERR_ARG, "tile_w must divide 32");
  for (int v : {t->bands_per_thread, t->batch_bands_per_thread})
    if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8 && v != 16)
      return air::set_error(AIR_ERR_ARG, "bands per thread must be 0, 1, 2, 4, 8 or 16");
  if (t->batch_blocks_per_sm < 0) return air::set_error(AIR_ERR_ARG, "batch_blocks_per_sm must be >= 0");
  g->tune = *t;
  return AIR_OK;
}

air_status air_get_tuning(air_grid *g, air_tuning *t) {
  air::set_error(AIR_OK, "");
  if (!g || !t) return air::set_error(AIR_ERR_ARG, "grid and tuning must not be NULL");
  *t = g->tune;
  return AIR_OK;
}

}  // extern "C"
