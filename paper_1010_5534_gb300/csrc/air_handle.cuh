// air_handle.cuh -- the opaque air_grid handle and its device workspace.
#pragma once
#include <string>
#include <vector>

#include "air_refine.cuh"

namespace air {

air_status set_error(air_status s, const char *fmt, ...);
void clear_error();  // empties the calling thread's error text
air_status cuda_fail(cudaError_t e, const char *what);

// Grows a device buffer to at least `bytes` (contents are not kept).
cudaError_t ensure(void **p, size_t *have, size_t bytes);

struct Workspace {
  // image quadtree
  int64_t cap = 0;
  int n_bands = 0;
  int16_t *view = nullptr;  // view of each node (batched renders)
  int8_t *lvl = nullptr;
  int32_t *pi = nullptr, *pj = nullptr, *child = nullptr;
  float *N = nullptr, *I = nullptr, *p = nullptr;
  uint32_t *steps = nullptr, *flag = nullptr;
  // scans
  int32_t *bcount = nullptr;
  int64_t *boff = nullptr;
  size_t bcount_b = 0, boff_b = 0;
  int64_t *d_total = nullptr;  // [3]
  int32_t *open[2] = {nullptr, nullptr};  // open-leaf lists (ping-pong)
  int32_t *lmap = nullptr;                 // level maps of the single-view tree
  // column table of the last axis view (RayGeom::tab) and what it was built for
  int32_t *axtab = nullptr;
  size_t axtab_b = 0;
  Camera ax_cam{};
  int ax_n0 = -1, ax_lmax = -1, ax_byj = 0;
  int64_t ax_slot = 0;
  bool ax_ok = false;
  size_t lmap_b = 0;
  size_t open_b[2] = {0, 0};
  uint32_t *d_err = nullptr;
  double *partial = nullptr;
  size_t partial_b = 0;
  double *d_flux = nullptr;  // [kMaxBands + 1]: flux then steps
  // fixed image
  float *fN = nullptr, *fI = nullptr, *fp = nullptr;
  uint32_t *fsteps = nullptr;
  size_t fN_b = 0, fI_b = 0, fp_b = 0, fsteps_b = 0;
  // staging for host outputs
  int32_t *o_level = nullptr, *o_i = nullptr, *o_j = nullptr;
  uint8_t *o_leaf = nullptr;
  float *o_N = nullptr, *o_p = nullptr, *o_I = nullptr;
  size_t o_level_b = 0, o_i_b = 0, o_j_b = 0, o_leaf_b = 0, o_N_b = 0, o_p_b = 0, o_I_b = 0;
  // sweep loop with counts on the device: its state, pinned copies of it
  // (two in flight, one for the initial state) and the copies' events
  SweepState *d_sweep = nullptr;
  SweepState *h_sweep = nullptr;  // [3]
  cudaEvent_t ev_sweep[2] = {nullptr, nullptr};
  // pinned host scalars
  int64_t *h_total = nullptr;  // [3]
  uint32_t *h_err = nullptr;
  double *h_flux = nullptr;  // [kMaxBands + 1]

  TreeView tree(int n0, int Lm) const {
    TreeView t;
    t.n0 = n0; t.Lm = Lm; t.cap = cap;
    t.lvl = lvl; t.pi = pi; t.pj = pj; t.child = child;
    t.N = N; t.I = I; t.p = p; t.steps = steps;
    return t;
  }
};

// Event pairs around launch groups, resolved when a render completes.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pool, 2 per group
  std::vector<int> phase;       // phase of group g
  std::vector<int> nlaunch;     // kernel launches in group g
  int used = 0;                 // groups recorded in the current render
  double ms[AIR_N_PHASES] = {0};
  int64_t launches[AIR_N_PHASES] = {0};
};

struct RayGeom;

// Control block of the batched persistent kernel (device memory).
struct BatchCtl {
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned long long q_head;
  long long n_nodes;
  long long need;
  int sweeps;
  unsigned int err;
  unsigned long long fb_rays;  // learned mode: pixels the proposal missed, traced in sweeps
};

struct BatchArgs {
  GridView g;
  const RayGeom *geoms;  // [V]
  int V, chunks, fp64_level, xi_norm, refine_on, stall;
  double xi_crit;
  TreeView t;
  int16_t *view;
  uint32_t *flag;
  BatchCtl *ctl;
  int32_t *bcnt;         // [blocks][V]
  int64_t *refined;      // [V]
  int32_t *vsweeps;      // [V]
  long long timeout_ns;
  // learned proposal (air_render_batch_learned): mode 0 runs every step;
  // mode 1 traces the base images only (and the deepest brick level each
  // base ray crossed, for the features); mode 2 continues from the traced
  // base images: it traces every view's proposal wave, then runs the sweeps,
  // copying a new pixel's values from the wave where it traced the pixel
  int mode;
  uint8_t *maxlev;       // [V n0^2] (mode 1)
  const int8_t *pdepth;  // [V n0^2][4] proposed depth per quadrant of each base pixel (mode 2)
  const int64_t *poff;   // [V n0^2] first proposal ray of each base pixel
  const int8_t *plvl;    // [P] proposal rays: level, pixel, view
  const int32_t *ppi, *ppj;
  const int16_t *pview;
  int64_t P;
  float *pN, *pI, *pp;   // [P], [n_bands][P], [P] traced values of the wave
  uint32_t *psteps;      // [P]
};

// Buffers and the captured graph of batched renders.
struct BatchWork {
  RayGeom *geoms = nullptr;
  BatchCtl *ctl = nullptr;
  int32_t *bcnt = nullptr;
  int64_t *refined = nullptr, *boff = nullptr;
  int32_t *vsweeps = nullptr;
  unsigned long long *vsteps = nullptr;
  double *vflux = nullptr;
  OutView *outs = nullptr;
  size_t geoms_b = 0, ctl_b = 0, bcnt_b = 0, refined_b = 0, boff_b = 0, vsweeps_b = 0,
         vsteps_b = 0, vflux_b = 0, outs_b = 0;
  BatchCtl *h_ctl = nullptr;
  void *h_geoms = nullptr;  // pinned staging of the per-view ray geometry
  size_t h_geoms_b = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
  BatchArgs key{};
  int key_grid = 0, key_nbt = 0;
  size_t key_smem = 0;
};

// Buffers of the learned-proposal render (single view and batched).
struct LearnWork {
  float *tau0 = nullptr, *xi_p = nullptr, *xi_n = nullptr, *logits = nullptr;
  uint8_t *maxlev = nullptr;
  uint16_t *x = nullptr;
  int8_t *depth = nullptr, *plvl = nullptr;
  int64_t *off = nullptr;
  int32_t *label = nullptr, *ppi = nullptr, *ppj = nullptr, *list = nullptr;
  float *pN = nullptr, *pI = nullptr, *pp = nullptr;
  uint32_t *psteps = nullptr, *missing = nullptr;
  int16_t *pview = nullptr;  // batched: view of each proposal ray
  size_t pview_b = 0;
  unsigned long long *counters = nullptr;
  size_t tau0_b = 0, xi_p_b = 0, xi_n_b = 0, logits_b = 0, maxlev_b = 0, x_b = 0, depth_b = 0,
         plvl_b = 0, off_b = 0, label_b = 0, ppi_b = 0, ppj_b = 0, list_b = 0, pN_b = 0, pI_b = 0,
         pp_b = 0, psteps_b = 0, missing_b = 0, counters_b = 0;
};

// Streamed spectra (air_render_adaptive_spectra): two device staging buffers
// that take turns holding one sweep's spectra while a copy stream moves the
// other to the caller's page-locked host array.
struct SpectraWork {
  cudaStream_t copy = nullptr;
  cudaEvent_t marched[2] = {nullptr, nullptr};  // staging k written (compute stream)
  cudaEvent_t copied[2] = {nullptr, nullptr};   // staging k free again (copy stream)
  float *stage[2] = {nullptr, nullptr};
  size_t stage_b[2] = {0, 0};
};

// The single-view tree that air_render_raster reads (set by output_tree).
struct RasterSrc {
  bool ok = false;
  int n0 = 0, Lm = 0;
  float *scratch = nullptr;  // device staging for host outputs
  size_t scratch_b = 0;
};

struct LastRender {
  bool valid = false;
  air_view view;
  air_params params;
  int64_t n_nodes = 0, n_refined = 0;
  int32_t n_sweeps = 0;
};

}  // namespace air

struct air_grid {
  cudaStream_t stream = nullptr;
  air::GridView gv{};
  // owned device memory
  void *d_cells = nullptr;
  int32_t *d_base = nullptr, *d_oct = nullptr;
  int32_t *d_bmap = nullptr;
  float *d_table = nullptr, *d_kappa = nullptr, *d_invkappa = nullptr;
  int64_t n_cells = 0;
  air::Workspace ws;
  air::LastRender last;
  air::RasterSrc raster;
  air::SpectraWork spectra;
  air::Profiler prof;
  air::BatchWork batch;
  air::LearnWork learn;
  air_tuning tune{};  // launch configuration (air_autotune / air_set_tuning)
};

namespace air {
air_status load_grid_impl(const air_grid_desc *d, air_grid *g);
// Profiling: open a launch group of `phase` containing `nlaunch` kernels; close
// it after the launches; resolve all groups after the render's final sync.
cudaError_t prof_open(air_grid *g, int phase, int nlaunch);
cudaError_t prof_close(air_grid *g);
cudaError_t prof_resolve(air_grid *g);
void free_grid_impl(air_grid *g);
void free_batch(air_grid *g);
// Shared by the single-view and batched renders (air_api.cu).
air_status check_image(const air_image *im);
air_status make_camera(const air_view *v, Camera &c);
air_status init_scalars(Workspace &w);
// Node arrays for `need` nodes (the first `keep` preserved); with_I = false
// leaves out the per-band intensities (streamed spectra keep them elsewhere);
// exact: allocate `need` nodes, not the growth margin.
air_status ensure_nodes(air_grid *g, int64_t need, int64_t keep, int64_t bound, bool with_I = true,
                        bool exact = false);
// mlp set: the batched render with the learned proposal (lopts, stats may be NULL).
air_status render_batch(air_grid *g, const air_view *views, int32_t n_views,
                        const air_params *params, const air_batch_opts *opts, air_image *outs,
                        air_mlp *mlp = nullptr, const air_learned_opts *lopts = nullptr,
                        air_learned_stats *stats = nullptr);
// spectra (page-locked host, [n_bands][spectra_cap]) set: streamed spectra.
// shard set: the rays of every sweep split over ranks (air_render_adaptive_sharded).
air_status render_adaptive(air_grid *g, const air_view *view, const air_params *pr, air_image *im,
                           float *spectra = nullptr, int64_t spectra_cap = 0,
                           const air_shard *shard = nullptr);
// Step vi on the quadtree of nodes [0, n) in the workspace; with spectra_dev
// set, the band intensities are read from there (stride spectra_cap).
air_status output_tree(air_grid *g, const Camera &cam, const air_params *pr, air_image *im,
                       int64_t n, int64_t n_refined, int32_t sweeps,
                       const float *spectra_dev = nullptr, int64_t spectra_cap = 0);
air_status mlp_forward(air_mlp *m, const uint16_t *x, int64_t n, float *logits, cudaStream_t st);
// The learned proposal of the V base images traced in the workspace (nodes
// view-major), with the deepest brick level of each base ray in maxlev:
// features, the network, the proposed depths and the proposal rays
// (g->learn: depth, off, plvl, ppi, ppj, pview and room for the traced
// values). *P: number of proposal rays.
air_status batch_proposal(air_grid *g, int V, const air_params *pr, air_mlp *mlp, double q,
                          const uint8_t *maxlev, int64_t *P);
// Level maps of the single-view tree, reset (NULL if they do not fit).
air_status level_maps(air_grid *g, int n0, int Lm, int32_t **out);
// src's column table (RaySource::axtab) for a view with camera cam and pixels
// of levels 0 .. lmax of an n0 image: built once per view and kept until the
// view changes; left NULL when the view does not qualify.
air_status axis_table(air_grid *g, const Camera &cam, int n0, int lmax, RaySource &src);
// Whether the node arrays can be sized for a whole image pyramid of `bound`
// nodes (at most half the free device memory beyond what is held).
bool pyramid_fits(air_grid *g, int64_t bound);
// Steps iii-v of one view with every count on the device, over the tree in
// the workspace (nodes [0, nbase) traced, open[0] holding the first m
// leaves; node arrays sized for `bound`); prop: values of new pixels from a
// learned proposal wave where it traced them, or NULL. *fin: the final state.
air_status sweep_loop_device(air_grid *g, const Camera &cam, const air_params *pr, int64_t nbase,
                             int64_t m, int64_t bound, int64_t open_max, const MarchTune &tune,
                             int march_launches, int32_t *lmap, const Proposal *prop,
                             SweepState *fin);
// The march configuration of this handle's tuning.
MarchTune march_tune(const air_grid *g, int fp64_level);
air_status render_fixed(air_grid *g, const air_view *view, int32_t res, int32_t fp64_level,
                        air_image *im);
void free_learn(air_grid *g);
}  // namespace air
