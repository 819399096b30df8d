// air_api.cu -- the C ABI (include/air.h): argument checks, device workspace,
// and the host side of the adaptive loop (Parkin 2010, Section 2 steps i-vi).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "air_handle.cuh"

namespace air {

static thread_local char g_err[512] = "";
void clear_error() { g_err[0] = 0; }

air_status set_error(air_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

air_status cuda_fail(cudaError_t e, const char *what) {
  const air_status s = (e == cudaErrorMemoryAllocation) ? AIR_ERR_OOM : AIR_ERR_CUDA;
  cudaGetLastError();  // clear a sticky launch error so the next call can run
  return set_error(s, "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t ensure(void **p, size_t *have, size_t bytes) {
  if (*have >= bytes && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (bytes == 0) return cudaSuccess;
  // headroom for the next, slightly larger request: a quarter, a sixteenth
  // above 4 GiB (buffers of many-band, many-view renders)
  const size_t grow = bytes + (bytes > ((size_t)4 << 30) ? bytes / 16 : bytes / 4);
  cudaError_t e = cudaMalloc(p, grow);
  if (e == cudaSuccess) *have = grow;
  return e;
}

#define CU_TRY(x)                                    \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

air_status init_scalars(Workspace &w) {
  if (!w.d_total) CU_TRY(cudaMalloc((void **)&w.d_total, 3 * sizeof(int64_t)));
  if (!w.d_err) CU_TRY(cudaMalloc((void **)&w.d_err, sizeof(uint32_t)));
  if (!w.d_flux) CU_TRY(cudaMalloc((void **)&w.d_flux, sizeof(double) * (kMaxBands + 1)));
  if (!w.h_total) CU_TRY(cudaMallocHost((void **)&w.h_total, 3 * sizeof(int64_t)));
  if (!w.h_err) CU_TRY(cudaMallocHost((void **)&w.h_err, sizeof(uint32_t)));
  if (!w.h_flux) CU_TRY(cudaMallocHost((void **)&w.h_flux, sizeof(double) * (kMaxBands + 1)));
  return AIR_OK;
}

cudaError_t prof_open(air_grid *g, int phase, int nlaunch) {
  Profiler &P = g->prof;
  if (!P.on) return cudaSuccess;
  if ((size_t)(2 * P.used + 2) > P.ev.size()) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      P.ev.push_back(e);
    }
    P.phase.push_back(0);
    P.nlaunch.push_back(0);
  }
  P.phase[P.used] = phase;
  P.nlaunch[P.used] = nlaunch;
  return cudaEventRecord(P.ev[2 * P.used], g->stream);
}

cudaError_t prof_close(air_grid *g) {
  Profiler &P = g->prof;
  if (!P.on) return cudaSuccess;
  cudaError_t r = cudaEventRecord(P.ev[2 * P.used + 1], g->stream);
  ++P.used;
  return r;
}

cudaError_t prof_resolve(air_grid *g) {
  Profiler &P = g->prof;
  if (!P.on) return cudaSuccess;
  for (int k = 0; k < P.used; ++k) {
    float ms = 0.f;
    cudaError_t r = cudaEventSynchronize(P.ev[2 * k + 1]);
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, P.ev[2 * k], P.ev[2 * k + 1]);
    if (r != cudaSuccess) return r;
    P.ms[P.phase[k]] += ms;
    P.launches[P.phase[k]] += P.nlaunch[k];
  }
  P.used = 0;
  return cudaSuccess;
}

// Grow the quadtree arrays to `cap` nodes, keeping the first `keep`.
template <typename T>
static cudaError_t regrow(T *&p, int64_t old_cap, int64_t cap, int64_t keep, int rows,
                          cudaStream_t st) {
  T *q = nullptr;
  cudaError_t e = cudaMalloc((void **)&q, sizeof(T) * (size_t)cap * rows);
  if (e != cudaSuccess) return e;
  if (p && keep > 0)
    for (int r = 0; r < rows; ++r) {
      e = cudaMemcpyAsync(q + (size_t)r * cap, p + (size_t)r * old_cap, sizeof(T) * keep,
                          cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) { cudaFree(q); return e; }
    }
  if (p) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(q); return e; }
    cudaFree(p);
  }
  p = q;
  return cudaSuccess;
}

air_status ensure_nodes(air_grid *g, int64_t need, int64_t keep, int64_t bound, bool with_I, bool exact) {
  Workspace &w = g->ws;
  const int nb = with_I ? g->gv.n_bands : -1;  // -1 tags arrays without intensities
  if (w.cap >= need && w.n_bands == nb) return AIR_OK;
  int64_t cap = exact ? need
                      : std::max<int64_t>(need, std::min<int64_t>(bound, std::max<int64_t>(2 * w.cap, need + need / 2)));
  if (cap < need) cap = need;
  if (w.n_bands != nb) {
    keep = 0;
    if (w.I) cudaFree(w.I);
    w.I = nullptr;
  }
  cudaStream_t st = g->stream;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = regrow(w.view, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess) e = regrow(w.lvl, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess) e = regrow(w.pi, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess) e = regrow(w.pj, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess) e = regrow(w.child, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess) e = regrow(w.N, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess && with_I) e = regrow(w.I, w.cap, cap, keep, nb, st);
  if (e == cudaSuccess) e = regrow(w.p, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess) e = regrow(w.steps, w.cap, cap, keep, 1, st);
  if (e == cudaSuccess) e = regrow(w.flag, w.cap, cap, keep, 1, st);
  if (e != cudaSuccess) return cuda_fail(e, "quadtree allocation");
  w.cap = cap;
  w.n_bands = nb;
  return AIR_OK;
}

static bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// Image basis: u = normalize(up x d), v = d x u, with d = normalize(dir).
air_status make_camera(const air_view *v, Camera &c) {
  if (!v) return set_error(AIR_ERR_ARG, "view is NULL");
  if (!finite3(v->dir) || !finite3(v->up) || !finite3(v->center) || !std::isfinite(v->half_extent) ||
      !(v->half_extent > 0.0))
    return set_error(AIR_ERR_ARG, "view needs finite dir, up, center and half_extent > 0");
  const double n = std::sqrt(v->dir[0] * v->dir[0] + v->dir[1] * v->dir[1] + v->dir[2] * v->dir[2]);
  if (!(n > 0.0)) return set_error(AIR_ERR_ARG, "view dir is zero");
  for (int a = 0; a < 3; ++a) c.d[a] = v->dir[a] / n;
  double ux = v->up[1] * c.d[2] - v->up[2] * c.d[1];
  double uy = v->up[2] * c.d[0] - v->up[0] * c.d[2];
  double uz = v->up[0] * c.d[1] - v->up[1] * c.d[0];
  const double un = std::sqrt(ux * ux + uy * uy + uz * uz);
  if (!(un > 0.0)) return set_error(AIR_ERR_ARG, "view up is parallel to dir");
  c.u[0] = ux / un; c.u[1] = uy / un; c.u[2] = uz / un;
  c.v[0] = c.d[1] * c.u[2] - c.d[2] * c.u[1];
  c.v[1] = c.d[2] * c.u[0] - c.d[0] * c.u[2];
  c.v[2] = c.d[0] * c.u[1] - c.d[1] * c.u[0];
  for (int a = 0; a < 3; ++a) c.c[a] = v->center[a];
  c.H = v->half_extent;
  return AIR_OK;
}

MarchTune march_tune(const air_grid *g, int fp64_level) {
  MarchTune t;
  t.block = 128;
  t.fp64_level = fp64_level < 0 ? 3 : fp64_level;
  t.nbt = g->tune.bands_per_thread;
  return t;
}

// Fixed image -> output arrays: level 0, (i, j) from the row-major index.
__global__ void k_fixed_out(int64_t n, int res, const float *N, const float *p, const float *I,
                            int n_bands, OutView o) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (o.level) o.level[k] = 0;
  if (o.i) o.i[k] = (int32_t)(k % res);
  if (o.j) o.j[k] = (int32_t)(k / res);
  if (o.is_leaf) o.is_leaf[k] = 1;
  if (o.N) o.N[k] = N[k];
  if (o.p) o.p[k] = p[k];
  if (o.I)
    for (int b = 0; b < n_bands; ++b) o.I[(int64_t)b * o.stride + k] = I[(int64_t)b * n + k];
}

// Device address of page-locked host memory (NULL if p is not page-locked):
// the streamed spectra's flux kernel reads the host array through it.
static void *host_locked(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Where the output kernels write: the caller's device arrays, or, for host
// arrays (page-locked or not), device staging arrays that finish_out copies
// back. The copies run on the copy engines, which move ~190 GB/s over the
// host link of a Grace-hosted GB300 where kernel stores through the link
// reach ~60 GB/s.
static air_status out_view(air_grid *g, const air_image *im, int64_t n, OutView &o) {
  Workspace &w = g->ws;
  const int nb = g->gv.n_bands;
  o.n_bands = nb;
  if (im->mem == AIR_DEVICE) {
    o.level = im->level; o.i = im->i; o.j = im->j; o.is_leaf = im->is_leaf;
    o.N = im->coldens; o.p = im->p; o.I = im->intensity;
    o.stride = im->capacity;
    return AIR_OK;
  }
  const size_t m = (size_t)std::max<int64_t>(n, 1);
  o.stride = (int64_t)m;
  o.level = o.i = o.j = nullptr; o.is_leaf = nullptr; o.N = o.p = o.I = nullptr;
  if (im->level) { CU_TRY(ensure((void **)&w.o_level, &w.o_level_b, 4 * m)); o.level = w.o_level; }
  if (im->i) { CU_TRY(ensure((void **)&w.o_i, &w.o_i_b, 4 * m)); o.i = w.o_i; }
  if (im->j) { CU_TRY(ensure((void **)&w.o_j, &w.o_j_b, 4 * m)); o.j = w.o_j; }
  if (im->is_leaf) { CU_TRY(ensure((void **)&w.o_leaf, &w.o_leaf_b, m)); o.is_leaf = w.o_leaf; }
  if (im->coldens) { CU_TRY(ensure((void **)&w.o_N, &w.o_N_b, 4 * m)); o.N = w.o_N; }
  if (im->p) { CU_TRY(ensure((void **)&w.o_p, &w.o_p_b, 4 * m)); o.p = w.o_p; }
  if (im->intensity) { CU_TRY(ensure((void **)&w.o_I, &w.o_I_b, 4 * m * nb)); o.I = w.o_I; }
  return AIR_OK;
}

// Staging -> host arrays (host-memory outputs), then band flux and step count.
static air_status finish_out(air_grid *g, air_image *im, const OutView &o, int64_t n) {
  cudaStream_t st = g->stream;
  const int nb = g->gv.n_bands;
  Workspace &w = g->ws;
  if (im->mem == AIR_HOST && n > 0) {
    if (im->level) CU_TRY(cudaMemcpyAsync(im->level, o.level, 4 * n, cudaMemcpyDeviceToHost, st));
    if (im->i) CU_TRY(cudaMemcpyAsync(im->i, o.i, 4 * n, cudaMemcpyDeviceToHost, st));
    if (im->j) CU_TRY(cudaMemcpyAsync(im->j, o.j, 4 * n, cudaMemcpyDeviceToHost, st));
    if (im->is_leaf) CU_TRY(cudaMemcpyAsync(im->is_leaf, o.is_leaf, n, cudaMemcpyDeviceToHost, st));
    if (im->coldens) CU_TRY(cudaMemcpyAsync(im->coldens, o.N, 4 * n, cudaMemcpyDeviceToHost, st));
    if (im->p) CU_TRY(cudaMemcpyAsync(im->p, o.p, 4 * n, cudaMemcpyDeviceToHost, st));
    if (im->intensity)
      for (int b = 0; b < nb; ++b)
        CU_TRY(cudaMemcpyAsync(im->intensity + (size_t)b * im->capacity, o.I + (size_t)b * o.stride,
                               4 * n, cudaMemcpyDeviceToHost, st));
  }
  CU_TRY(cudaMemcpyAsync(w.h_flux, w.d_flux, sizeof(double) * (nb + 1), cudaMemcpyDeviceToHost, st));
  if (im->band_flux && im->mem == AIR_DEVICE)
    CU_TRY(cudaMemcpyAsync(im->band_flux, w.d_flux, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
  CU_TRY(cudaStreamSynchronize(st));
  if (im->band_flux && im->mem == AIR_HOST) std::memcpy(im->band_flux, w.h_flux, sizeof(double) * nb);
  im->n_steps = (int64_t)w.h_flux[nb];
  return AIR_OK;
}

air_status check_image(const air_image *im) {
  if (!im) return set_error(AIR_ERR_ARG, "out is NULL");
  if (im->mem != AIR_HOST && im->mem != AIR_DEVICE) return set_error(AIR_ERR_ARG, "out->mem must be AIR_HOST or AIR_DEVICE");
  if (im->capacity < 0) return set_error(AIR_ERR_ARG, "out->capacity < 0");
  return AIR_OK;
}

air_status render_fixed(air_grid *g, const air_view *view, int32_t res, int32_t fp64_level,
                        air_image *im) {
  air_status s = check_image(im);
  if (s) return s;
  Camera cam;
  if ((s = make_camera(view, cam))) return s;
  if (res < 1 || res > (1 << 16)) return set_error(AIR_ERR_ARG, "res must be in [1, 65536]");
  const int64_t n = (int64_t)res * res;
  im->n_out = n; im->n_leaves = n; im->n_rays = n; im->n_sweeps = 0; im->n_steps = 0;
  if (im->capacity < n) return set_error(AIR_ERR_CAPACITY, "capacity %lld < %lld pixels", (long long)im->capacity, (long long)n);
  if ((s = init_scalars(g->ws))) return s;
  Workspace &w = g->ws;
  const int nb = g->gv.n_bands;
  CU_TRY(ensure((void **)&w.fN, &w.fN_b, 4 * n));
  CU_TRY(ensure((void **)&w.fI, &w.fI_b, 4 * n * nb));
  CU_TRY(ensure((void **)&w.fp, &w.fp_b, 4 * n));
  CU_TRY(ensure((void **)&w.fsteps, &w.fsteps_b, 4 * n));
  CU_TRY(ensure((void **)&w.partial, &w.partial_b, sizeof(double) * (nb + 1) * flux_blocks(n)));
  cudaStream_t st = g->stream;
  RaySource src{};
  src.mode = 1; src.n0 = res; src.first = 0; src.count = n;
  src.tile_w = g->tune.tile_w > 0 ? g->tune.tile_w : 8;
  {
    const air_status sa = axis_table(g, cam, res, 0, src);
    if (sa) return sa;
  }
  RayOut ro{w.fN, w.fI, n, w.fsteps, w.fp};
  g->prof.used = 0;
  CU_TRY(prof_open(g, AIR_PHASE_MARCH, nb > (g->tune.bands_per_thread > 0 ? g->tune.bands_per_thread : default_bands_per_thread(nb)) ? 2 : 1));
  CU_TRY(launch_march(g->gv, cam, src, ro, march_tune(g, fp64_level), st));
  CU_TRY(prof_close(g));
  FluxArgs fa{};
  fa.n = n; fa.child = nullptr; fa.lvl = nullptr; fa.I = w.fI; fa.stride = n; fa.steps = w.fsteps;
  fa.n_bands = nb; fa.area0 = (2.0 * cam.H / res) * (2.0 * cam.H / res); fa.partial = w.partial;
  OutView o;
  if ((s = out_view(g, im, n, o))) return s;
  CU_TRY(prof_open(g, AIR_PHASE_OUTPUT, 3));
  CU_TRY(launch_flux(fa, w.d_flux, w.d_flux + nb, st));
  k_fixed_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, res, w.fN, w.fp, w.fI, nb, o);
  CU_TRY(cudaGetLastError());
  CU_TRY(prof_close(g));
  s = finish_out(g, im, o, n);
  if (s) return s;
  CU_TRY(prof_resolve(g));
  return AIR_OK;
}

air_status axis_table(air_grid *g, const Camera &cam, int n0, int lmax, RaySource &src) {
  Workspace &w = g->ws;
  src.axtab = nullptr;
  src.axtab_slot = 0;
  src.axtab_byj = 0;
  const bool same = w.ax_n0 == n0 && w.ax_lmax == lmax && !std::memcmp(&w.ax_cam, &cam, sizeof(Camera));
  if (!same) {
    w.ax_ok = false;
    const int64_t slot = axis_table_slot(n0, lmax);
    CU_TRY(ensure((void **)&w.axtab, &w.axtab_b, sizeof(int32_t) * 2 * (size_t)slot));
    bool ok = false;
    CU_TRY(launch_axis_table(g->gv, cam, n0, lmax, w.axtab, &w.ax_byj, &w.ax_slot, &ok, g->stream));
    w.ax_ok = ok;
    w.ax_cam = cam;
    w.ax_n0 = n0;
    w.ax_lmax = lmax;
  }
  if (w.ax_ok) {
    src.axtab = w.axtab;
    src.axtab_slot = w.ax_slot;
    src.axtab_byj = w.ax_byj;
  }
  return AIR_OK;
}

air_status level_maps(air_grid *g, int n0, int Lm, int32_t **out) {
  Workspace &w = g->ws;
  *out = nullptr;
  const size_t map_bytes = sizeof(int32_t) * (size_t)level_map_offset(n0, Lm);
  if (map_bytes == 0) return AIR_OK;
  bool fits = w.lmap_b >= map_bytes;
  if (!fits) {
    size_t fr = 0, tot = 0;
    CU_TRY(cudaMemGetInfo(&fr, &tot));
    fits = (double)map_bytes <= 0.25 * (double)fr;
    if (fits) CU_TRY(ensure((void **)&w.lmap, &w.lmap_b, map_bytes));
  }
  if (fits) {
    CU_TRY(cudaMemsetAsync(w.lmap, 0xff, map_bytes, g->stream));
    *out = w.lmap;
  }
  return AIR_OK;
}

bool pyramid_fits(air_grid *g, int64_t bound) {
  Workspace &w = g->ws;
  const int nb = g->gv.n_bands;
  if (w.cap >= bound && w.n_bands == nb) return true;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const double need = ((double)bound - (double)w.cap) * (31.0 + 4.0 * nb);
  return need <= 0.5 * (double)fr;
}

air_status sweep_loop_device(air_grid *g, const Camera &cam, const air_params *pr, int64_t nbase,
                             int64_t m, int64_t bound, int64_t open_max, const MarchTune &tune,
                             int march_launches, int32_t *lmap, const Proposal *prop,
                             SweepState *fin) {
  Workspace &w = g->ws;
  cudaStream_t st = g->stream;
  TreeView t = w.tree(pr->base_res, pr->max_level);
  // Steps iii-v with every count on the device: each sweep's kernels read
  // the open-list length, the flag count and the node count from the
  // device state, so the host queues sweep after sweep without waiting.
  // It reads the state back two sweeps behind, only to learn that the
  // loop has ended; the (at most two) sweeps queued past the end find
  // `done` set and do nothing.
  if (!w.d_sweep) CU_TRY(cudaMalloc((void **)&w.d_sweep, sizeof(SweepState)));
  if (!w.h_sweep) CU_TRY(cudaMallocHost((void **)&w.h_sweep, 3 * sizeof(SweepState)));
  for (int k = 0; k < 2; ++k)
    if (!w.ev_sweep[k]) CU_TRY(cudaEventCreateWithFlags(&w.ev_sweep[k], cudaEventDisableTiming));
  SweepState &s0 = w.h_sweep[2];
  std::memset(&s0, 0, sizeof(SweepState));
  s0.n = nbase;
  s0.m = m;
  s0.done = m == 0;
  CU_TRY(cudaMemcpyAsync(w.d_sweep, &s0, sizeof(SweepState), cudaMemcpyHostToDevice, st));
  // the fused scan and balance only set flags: the base pixels' start at zero
  CU_TRY(cudaMemsetAsync(w.flag, 0, sizeof(uint32_t) * (size_t)nbase, st));
  int32_t *const open2[2] = {w.open[0], w.open[1]};
  const int64_t nb_cap = scan_blocks(open_max);
  RaySource ds{};
  ds.mode = 2; ds.n0 = pr->base_res; ds.lvl = t.lvl; ds.pi = t.pi; ds.pj = t.pj; ds.sweep = w.d_sweep;
  {
    const air_status sa = axis_table(g, cam, pr->base_res, pr->max_level, ds);
    if (sa) return sa;
  }
  if (prop) {
    ds.use_prop = 1;
    ds.prop = *prop;
  }
  RayOut ro{t.N, t.I, t.cap, t.steps, t.p};
  constexpr int kAhead = 2;
  // every sweep refines at least one pixel
  const int64_t max_sweeps = (bound - nbase) / 4 + kAhead + 1;
  int64_t q = 0;
  for (;; ++q) {
    if (q >= kAhead) {
      CU_TRY(cudaEventSynchronize(w.ev_sweep[q % kAhead]));
      if (w.h_sweep[q % kAhead].done) break;
    }
    if (q > max_sweeps) return set_error(AIR_ERR_NUMERIC, "sweep loop did not end");
    // step iii: scan and balance in one pass (counted as the scan phase)
    CU_TRY(prof_open(g, AIR_PHASE_SCAN, 1));
    CU_TRY(launch_sweep_scan_balance(t, open2, w.d_sweep, pr->xi_crit, pr->xi_norm, pr->refine_on,
                                     w.flag, w.d_err, st, lmap));
    CU_TRY(prof_close(g));
    CU_TRY(prof_open(g, AIR_PHASE_REFINE, 3));
    CU_TRY(launch_sweep_count(t, open2, w.d_sweep, w.flag, w.bcount, w.boff, nb_cap, st));
    CU_TRY(launch_sweep_emit(t, open2, w.d_sweep, w.flag, w.boff, nb_cap, st, lmap));
    CU_TRY(prof_close(g));
    // step ii on the new pixels (or their values from the proposal); the
    // march's last block (or the band sum after it) moves the state on
    CU_TRY(prof_open(g, AIR_PHASE_MARCH, march_launches));
    CU_TRY(launch_march(g->gv, cam, ds, ro, tune, st));
    CU_TRY(prof_close(g));
    CU_TRY(cudaMemcpyAsync(&w.h_sweep[q % kAhead], w.d_sweep, sizeof(SweepState),
                           cudaMemcpyDeviceToHost, st));
    CU_TRY(cudaEventRecord(w.ev_sweep[q % kAhead], st));
  }
  CU_TRY(cudaStreamSynchronize(st));
  *fin = w.h_sweep[(q - 1) % kAhead];
  return AIR_OK;
}

air_status render_adaptive(air_grid *g, const air_view *view, const air_params *pr, air_image *im,
                           float *spectra, int64_t spectra_cap, const air_shard *shard) {
  g->raster.ok = false;  // the workspace tree is about to change
  air_status s = check_image(im);
  if (s) return s;
  const bool streamed = spectra != nullptr;
  const bool sharded = shard != nullptr && shard->world > 1;
  if (shard) {
    if (shard->world < 1 || shard->rank < 0 || shard->rank >= shard->world)
      return set_error(AIR_ERR_ARG, "shard needs 0 <= rank < world");
    if (sharded && !shard->exchange) return set_error(AIR_ERR_ARG, "shard->exchange is NULL");
    if (sharded && streamed) return set_error(AIR_ERR_ARG, "sharded renders do not stream spectra");
  }
  const float *spectra_dev = nullptr;
  if (streamed) {
    if (!pr || pr->include_interior != 1)
      return set_error(AIR_ERR_ARG, "streamed spectra are indexed by node: include_interior must be 1");
    if (im->intensity) return set_error(AIR_ERR_ARG, "with streamed spectra out->intensity must be NULL");
    if (spectra_cap < 0) return set_error(AIR_ERR_ARG, "spectra_cap < 0");
    if (!(spectra_dev = (const float *)host_locked(spectra)))
      return set_error(AIR_ERR_ARG, "spectra must be page-locked host memory (cudaHostAlloc / cudaHostRegister)");
    g->last.valid = false;
  }
  Camera cam;
  if ((s = make_camera(view, cam))) return s;
  if (!pr) return set_error(AIR_ERR_ARG, "params is NULL");
  const int n0 = pr->base_res, Lm = pr->max_level;
  if (n0 < 1 || Lm < 0 || Lm >= kMaxLevels || ((int64_t)n0 << Lm) > (1 << 20))
    return set_error(AIR_ERR_ARG, "need base_res >= 1, 0 <= max_level < %d, base_res << max_level <= 2^20", kMaxLevels);
  if (!std::isfinite(pr->xi_crit) || pr->xi_crit < 0.0) return set_error(AIR_ERR_ARG, "xi_crit must be finite and >= 0");
  if (pr->xi_norm != 0 && pr->xi_norm != 1) return set_error(AIR_ERR_ARG, "xi_norm must be 0 or 1");
  if (pr->refine_on < 0 || pr->refine_on > 2) return set_error(AIR_ERR_ARG, "refine_on must be 0, 1 or 2");
  if (pr->include_interior != 0 && pr->include_interior != 1) return set_error(AIR_ERR_ARG, "include_interior must be 0 or 1");
  if ((s = init_scalars(g->ws))) return s;
  Workspace &w = g->ws;
  const int nb = g->gv.n_bands;
  cudaStream_t st = g->stream;
  int64_t bound = 0;
  for (int l = 0; l <= Lm; ++l) bound += ((int64_t)n0 << l) * ((int64_t)n0 << l);
  if (bound > INT32_MAX) return set_error(AIR_ERR_ARG, "image pyramid exceeds 2^31 nodes");
  // per-block scan offsets for any node count up to the bound (never resized mid-render)
  CU_TRY(ensure((void **)&w.bcount, &w.bcount_b, 3 * sizeof(int32_t) * scan_blocks(bound)));
  CU_TRY(ensure((void **)&w.boff, &w.boff_b, 3 * sizeof(int64_t) * scan_blocks(bound)));
  // open-leaf lists: at most every node below the top level
  const int64_t open_max = std::max<int64_t>(1, bound - ((int64_t)n0 << Lm) * ((int64_t)n0 << Lm));
  for (int k = 0; k < 2; ++k)
    CU_TRY(ensure((void **)&w.open[k], &w.open_b[k], sizeof(int32_t) * (size_t)open_max));

  air_params key = *pr;
  key.include_interior = 0;
  const bool cached = !streamed && g->last.valid && !std::memcmp(&g->last.view, view, sizeof(air_view)) &&
                      !std::memcmp(&g->last.params, &key, sizeof(air_params));
  SpectraWork &sp = g->spectra;
  bool stage_used[2] = {false, false}, overflow = false;
  int stage_k = 0;
  if (streamed) {
    if (!sp.copy) CU_TRY(cudaStreamCreateWithFlags(&sp.copy, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      if (!sp.marched[k]) CU_TRY(cudaEventCreateWithFlags(&sp.marched[k], cudaEventDisableTiming));
      if (!sp.copied[k]) CU_TRY(cudaEventCreateWithFlags(&sp.copied[k], cudaEventDisableTiming));
    }
  }
  // Step ii on nodes [first, first + count): with streamed spectra the march
  // writes them to staging buffer k, which the copy stream then moves to the
  // host array while the next sweep proceeds; buffer k is reused only after
  // its copy has finished.
  auto march_nodes = [&](const TreeView &tv, RaySource src, const MarchTune &tune, int launches) -> air_status {
    RayOut ro{tv.N, tv.I, tv.cap, tv.steps, tv.p};
    const int k = stage_k;
    if (streamed) {
      if (stage_used[k]) CU_TRY(cudaStreamWaitEvent(g->stream, sp.copied[k], 0));
      CU_TRY(ensure((void **)&sp.stage[k], &sp.stage_b[k], sizeof(float) * (size_t)nb * (size_t)src.count));
      ro.I = sp.stage[k];
      ro.stride = src.count;
      ro.ioff = src.first;
    }
    if (sharded) {
      // this rank's slice of the sweep's rays, then the other slices from
      // the other ranks (Section 2: trace distributed, gather for the scan)
      const int64_t first = src.first, count = src.count;
      const int64_t lo = count * shard->rank / shard->world;
      const int64_t hi = count * (shard->rank + 1) / shard->world;
      src.first = first + lo;
      src.count = hi - lo;
      if (src.count > 0) {
        CU_TRY(prof_open(g, AIR_PHASE_MARCH, launches));
        CU_TRY(launch_march(g->gv, cam, src, ro, tune, g->stream));
        CU_TRY(prof_close(g));
      }
      CU_TRY(cudaStreamSynchronize(g->stream));
      if (shard->exchange(shard->user, first, count, nb, tv.N, tv.I, tv.cap, tv.p, tv.steps) != 0)
        return set_error(AIR_ERR_ARG, "shard exchange failed (sweep rays %lld..%lld)", (long long)first,
                         (long long)(first + count));
      return AIR_OK;
    }
    CU_TRY(prof_open(g, AIR_PHASE_MARCH, launches));
    CU_TRY(launch_march(g->gv, cam, src, ro, tune, g->stream));
    CU_TRY(prof_close(g));
    if (streamed) {
      if (src.first + src.count <= spectra_cap) {
        CU_TRY(cudaEventRecord(sp.marched[k], g->stream));
        CU_TRY(cudaStreamWaitEvent(sp.copy, sp.marched[k], 0));
        CU_TRY(cudaMemcpy2DAsync(spectra + src.first, sizeof(float) * (size_t)spectra_cap, sp.stage[k],
                                 sizeof(float) * (size_t)src.count, sizeof(float) * (size_t)src.count,
                                 (size_t)nb, cudaMemcpyDeviceToHost, sp.copy));
        CU_TRY(cudaEventRecord(sp.copied[k], sp.copy));
        stage_used[k] = true;
      } else {
        overflow = true;  // finish the tree; the caller retries with a larger array
      }
      stage_k ^= 1;
    }
    return AIR_OK;
  };
  int64_t n = 0, n_refined = 0;
  int32_t sweeps = 0;
  TreeView t;
  if (cached) {
    n = g->last.n_nodes; n_refined = g->last.n_refined; sweeps = g->last.n_sweeps;
    t = w.tree(n0, Lm);
  } else {
    g->last.valid = false;
    const int64_t nbase = (int64_t)n0 * n0;
    // The sweep loop keeps its counts on the device when the node arrays can
    // be sized for the whole image pyramid at once (no growth mid-loop); a
    // render whose pyramid would take more than half of the free device
    // memory reads the counts back sweep by sweep and grows on demand.
    const bool dev_loop = !streamed && !sharded && pyramid_fits(g, bound);
    if ((s = ensure_nodes(g, dev_loop ? bound : std::min<int64_t>(bound, std::max<int64_t>(4 * nbase, w.cap)),
                          0, bound, !streamed))) return s;
    t = w.tree(n0, Lm);
    const MarchTune tune = march_tune(g, pr->fp64_level);
    g->prof.used = 0;
    const int nbt_eff = tune.nbt > 0 ? tune.nbt : default_bands_per_thread(nb);
    const int march_launches = nb > nbt_eff ? 2 : 1;  // march (+ band sum when bands are chunked)
    // step i + ii: base image
    CU_TRY(prof_open(g, AIR_PHASE_REFINE, 1));
    CU_TRY(launch_init_base(t, st));
    CU_TRY(prof_close(g));
    CU_TRY(cudaMemsetAsync(w.d_err, 0, sizeof(uint32_t), st));
    RaySource src{};
    src.mode = 0; src.n0 = n0; src.lvl = t.lvl; src.pi = t.pi; src.pj = t.pj; src.first = 0; src.count = nbase;
    if ((s = axis_table(g, cam, n0, Lm, src))) return s;
    if ((s = march_nodes(t, src, tune, march_launches))) return s;
    n = nbase;
    // open-leaf list: the base pixels, unless the base is the top level
    int cur = 0;
    int64_t m = Lm > 0 ? nbase : 0;
    CU_TRY(launch_list_init(w.open[0], m, st));
    int32_t *lmap = nullptr;
    if ((s = level_maps(g, n0, Lm, &lmap))) return s;
    if (dev_loop) {
      SweepState fin;
      if ((s = sweep_loop_device(g, cam, pr, nbase, m, bound, open_max, tune, march_launches, lmap,
                                 nullptr, &fin)))
        return s;
      n = fin.n;
      n_refined = fin.n_refined;
      sweeps = fin.sweeps;
      m = 0;
    }
    for (;;) {
      if (m == 0) break;  // no leaf below the top level: nothing can be flagged
      // step iii: scan, then balance; count the flags and the next list
      CU_TRY(prof_open(g, AIR_PHASE_SCAN, 1));
      CU_TRY(launch_list_scan(t, w.open[cur], m, pr->xi_crit, pr->xi_norm, pr->refine_on, w.flag, st, lmap));
      CU_TRY(prof_close(g));
      CU_TRY(prof_open(g, AIR_PHASE_BALANCE, 1));
      CU_TRY(launch_list_balance(t, w.open[cur], m, w.flag, w.d_err, st, lmap));
      CU_TRY(prof_close(g));
      CU_TRY(prof_open(g, AIR_PHASE_REFINE, 2));
      CU_TRY(launch_list_count(t, w.open[cur], m, w.flag, w.bcount, w.boff, w.d_total, st));
      CU_TRY(prof_close(g));
      CU_TRY(cudaMemcpyAsync(w.h_total, w.d_total, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      CU_TRY(cudaStreamSynchronize(st));
      const int64_t nflag = w.h_total[0];
      const int64_t m_next = w.h_total[1] + 4 * w.h_total[2];
      if (nflag == 0) break;
      const int64_t n_new = n + 4 * nflag;
      if (n_new > bound) return set_error(AIR_ERR_NUMERIC, "quadtree exceeds its bound (%lld > %lld)", (long long)n_new, (long long)bound);
      if (n_new > w.cap) {
        if ((s = ensure_nodes(g, n_new, n, bound, !streamed))) return s;
        t = w.tree(n0, Lm);
        // the per-block offsets were computed for n items; they stay valid
      }
      // step iv: refine (and the next open-leaf list), then step ii on the new pixels
      CU_TRY(prof_open(g, AIR_PHASE_REFINE, 1));
      CU_TRY(launch_list_emit(t, w.open[cur], m, w.flag, w.boff, w.d_total, n, w.open[cur ^ 1], st, lmap));
      CU_TRY(prof_close(g));
      src.lvl = t.lvl; src.pi = t.pi; src.pj = t.pj; src.first = n; src.count = 4 * nflag;
      if ((s = march_nodes(t, src, tune, march_launches))) return s;
      n = n_new;
      n_refined += nflag;
      ++sweeps;
      m = m_next;
      cur ^= 1;
    }
    CU_TRY(cudaMemcpyAsync(w.h_err, w.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CU_TRY(cudaStreamSynchronize(st));
    if (*w.h_err) return set_error(AIR_ERR_NUMERIC, "balance closure overflowed its stack");
    g->last.view = *view;
    g->last.params = key;
    g->last.n_nodes = n; g->last.n_refined = n_refined; g->last.n_sweeps = sweeps;
  }
  if (!streamed) return output_tree(g, cam, pr, im, n, n_refined, sweeps);
  // the copies of the last sweeps must land before the flux reads the host array
  for (int k = 0; k < 2; ++k)
    if (stage_used[k]) CU_TRY(cudaStreamWaitEvent(st, sp.copied[k], 0));
  if (overflow) {
    CU_TRY(cudaStreamSynchronize(st));
    im->n_out = n; im->n_leaves = (int64_t)n0 * n0 + 3 * n_refined; im->n_rays = n; im->n_sweeps = sweeps;
    g->last.valid = false;
    return set_error(AIR_ERR_CAPACITY, "spectra_cap %lld < %lld traced nodes", (long long)spectra_cap, (long long)n);
  }
  s = output_tree(g, cam, pr, im, n, n_refined, sweeps, spectra_dev, spectra_cap);
  g->last.valid = false;  // the tree holds no intensities: no reuse by another render
  return s;
}

air_status output_tree(air_grid *g, const Camera &cam, const air_params *pr, air_image *im,
                       int64_t n, int64_t n_refined, int32_t sweeps, const float *spectra_dev,
                       int64_t spectra_cap) {
  air_status s = AIR_OK;
  Workspace &w = g->ws;
  const int nb = g->gv.n_bands;
  cudaStream_t st = g->stream;
  const int n0 = pr->base_res;
  TreeView t = w.tree(n0, pr->max_level);
  // step vi: output
  const int all = pr->include_interior;
  const int64_t n_leaves = (int64_t)n0 * n0 + 3 * n_refined;
  const int64_t n_out = all ? n : n_leaves;
  im->n_out = n_out; im->n_leaves = n_leaves; im->n_rays = n; im->n_sweeps = sweeps; im->n_steps = 0;
  if (im->capacity < n_out) {
    // keep the finished tree so that a retry with larger arrays only copies it out
    g->last.valid = true;
    return set_error(AIR_ERR_CAPACITY, "capacity %lld < %lld pixels", (long long)im->capacity, (long long)n_out);
  }
  g->last.valid = false;
  g->raster.ok = true;
  g->raster.n0 = n0;
  g->raster.Lm = pr->max_level;
  CU_TRY(ensure((void **)&w.partial, &w.partial_b, sizeof(double) * (nb + 1) * flux_blocks(n)));
  FluxArgs fa{};
  fa.n = n; fa.child = t.child; fa.lvl = t.lvl; fa.steps = t.steps;
  fa.I = spectra_dev ? spectra_dev : t.I;
  fa.stride = spectra_dev ? spectra_cap : t.cap;
  fa.n_bands = nb; fa.area0 = (2.0 * cam.H / n0) * (2.0 * cam.H / n0); fa.partial = w.partial;
  OutView o;
  if ((s = out_view(g, im, n_out, o))) return s;
  CU_TRY(prof_open(g, AIR_PHASE_OUTPUT, 5));
  CU_TRY(launch_flux(fa, w.d_flux, w.d_flux + nb, st));
  CU_TRY(launch_count_leaves(t, all, n, w.bcount, w.boff, w.d_total, st));
  CU_TRY(launch_emit_out(t, o, all, n, w.boff, st));
  CU_TRY(prof_close(g));
  s = finish_out(g, im, o, n_out);
  if (s) return s;
  CU_TRY(prof_resolve(g));
  return AIR_OK;
}

}  // namespace air

// ---------------------------------------------------------------- C ABI

extern "C" {

air_status air_load_grid(const air_grid_desc *desc, void *stream, air_grid **out) {
  air::g_err[0] = 0;
  if (!desc || !out) return air::set_error(AIR_ERR_ARG, "desc and out must not be NULL");
  *out = nullptr;
  air_grid *g = new (std::nothrow) air_grid();
  if (!g) return air::set_error(AIR_ERR_OOM, "host allocation failed");
  g->stream = (cudaStream_t)stream;
  air_status s = air::load_grid_impl(desc, g);
  if (s != AIR_OK) {
    air::free_grid_impl(g);
    delete g;
    return s;
  }
  *out = g;
  return AIR_OK;
}

air_status air_set_stream(air_grid *g, void *stream) {
  air::g_err[0] = 0;
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  g->stream = (cudaStream_t)stream;
  return AIR_OK;
}

air_status air_render_fixed(air_grid *g, const air_view *view, int32_t res, int32_t fp64_level,
                            air_image *out) {
  air::g_err[0] = 0;
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  return air::render_fixed(g, view, res, fp64_level, out);
}

air_status air_render_adaptive(air_grid *g, const air_view *view, const air_params *params,
                               air_image *out) {
  air::g_err[0] = 0;
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  return air::render_adaptive(g, view, params, out);
}

air_status air_render_adaptive_sharded(air_grid *g, const air_view *view, const air_params *params,
                                       const air_shard *shard, air_image *out) {
  air::g_err[0] = 0;
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  if (!shard) return air::set_error(AIR_ERR_ARG, "shard is NULL");
  return air::render_adaptive(g, view, params, out, nullptr, 0, shard);
}

air_status air_render_adaptive_spectra(air_grid *g, const air_view *view, const air_params *params,
                                       air_image *out, float *spectra, int64_t spectra_cap) {
  air::g_err[0] = 0;
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  if (!spectra) return air::set_error(AIR_ERR_ARG, "spectra is NULL");
  return air::render_adaptive(g, view, params, out, spectra, spectra_cap);
}

air_status air_profile_enable(air_grid *g, int32_t on) {
  air::g_err[0] = 0;
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  g->prof.on = on != 0;
  g->prof.used = 0;
  for (int p = 0; p < AIR_N_PHASES; ++p) {
    g->prof.ms[p] = 0.0;
    g->prof.launches[p] = 0;
  }
  return AIR_OK;
}

air_status air_profile_read(air_grid *g, double *ms, int64_t *launches) {
  air::g_err[0] = 0;
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  for (int p = 0; p < AIR_N_PHASES; ++p) {
    if (ms) ms[p] = g->prof.ms[p];
    if (launches) launches[p] = g->prof.launches[p];
  }
  return AIR_OK;
}

void air_free(air_grid *g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  else cudaDeviceSynchronize();
  air::free_grid_impl(g);
  delete g;
}

const char *air_last_error(void) { return air::g_err; }

const char *air_version(void) { return "air-gb300 0.1 (sm_103a)"; }

}  // extern "C"
