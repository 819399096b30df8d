// air_learned.cu -- learned refinement-depth proposal (not in the paper).
//
// The base image is traced as in plain AIR (Section 2 steps i-ii). A small
// network (air_mlp.cu) reads 16 features of every quadrant of every base
// pixel (its four level-1 pixels) and proposes the depth plain AIR will refine
// that quadrant to; every pixel of the proposed subtrees is traced in ONE
// wave (layout: Proposal, air_internal.cuh). Then plain AIR runs exactly as before --
// scan (Eq. 2), balance, refine -- except that the values of a new pixel are
// gathered from the proposal wave instead of being traced; pixels the proposal
// missed are traced in a fallback wave. The paper's criterion, evaluated on
// every traced pixel, decides the image, so the output is identical to plain
// AIR's; the proposal only changes how many launches trace it and how many
// rays are wasted on over-predicted subtrees.
#include <cuda_bf16.h>

#include <cfloat>
#include <cmath>
#include <vector>

#include "air_handle.cuh"
#include "air_tree.cuh"

namespace air {

constexpr int kFeat = 16;

__device__ __forceinline__ uint16_t f2bf(float x) {
  __nv_bfloat16 v = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t *>(&v);
}

// Eq. 2 on the base image (values in row-major [n0][n0]), edges clamped.
__device__ __forceinline__ double base_xi(const float *v, int n0, int i, int j) {
  double s[9];
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const int ii = min(max(i + di, 0), n0 - 1), jj = min(max(j + dj, 0), n0 - 1);
      s[3 * (dj + 1) + (di + 1)] = (double)v[jj * n0 + ii];
    }
  return xi_eq2(s, 0);
}

// Pass 1: Eq. 2 of the base image on p and on N.
__global__ void k_base_xi(const float *p, const float *N, int n0, float *xi_p, float *xi_n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n0 * n0) return;
  const int i = k % n0, j = k / n0;
  xi_p[k] = (float)base_xi(p, n0, i, j);
  xi_n[k] = (float)base_xi(N, n0, i, j);
}

// Pass 2: the 16 features of every quadrant sample s = 4 b + q of base pixel
// b = (i, j) (row-major), quadrant q on the side (sx, sy) = (q & 1 ? 1 : -1,
// q & 2 ? 1 : -1); S = the three base neighbours on that side, (i + sx, j),
// (i, j + sy) and (i + sx, j + sy), and Q = S and the pixel itself (edges
// clamped; scale-free where possible):
//  0 xi(p)  1 xi(N)  2 [p > 0]  3 sx Sobel_u(p) / sum|p|  4 sy Sobel_v(p) / sum|p|
//    (3x3, the gradient towards the quadrant)
//  5 (max - min)/max of p over Q   6 same for N   7 min(tau_0, 10)/10
//  8 deepest brick level crossed / max level   9 emitting pixels of S / 3
// 10 log10(N)/10   11 log10(p)/20 (both clamped)   12 max xi(p) over S
// 13 max xi(N) over S   14 p / max of p over Q   15 1
__global__ void k_features(const float *p, const float *N, const float *tau0, const uint8_t *maxlev,
                           const float *xi_p, const float *xi_n, int n0, int grid_levels,
                           uint16_t *x, const float *kappa) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 4 * (int64_t)n0 * n0) return;
  const int k = (int)(s >> 2), qd = (int)(s & 3);
  const int i = k % n0, j = k / n0;
  const int sx = (qd & 1) ? 1 : -1, sy = (qd & 2) ? 1 : -1;
  float pv[9], nv[9];
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const int ii = min(max(i + di, 0), n0 - 1), jj = min(max(j + dj, 0), n0 - 1);
      const int m = 3 * (dj + 1) + (di + 1);
      pv[m] = p[jj * n0 + ii];
      nv[m] = N[jj * n0 + ii];
    }
  float sp = 0.f;
#pragma unroll
  for (int m = 0; m < 9; ++m) sp += fabsf(pv[m]);
  // the side set S (its entries of the 3x3 stencil and its pixels' indices)
  const int ms[3] = {4 + sx, 4 + 3 * sy, 4 + 3 * sy + sx};
  const int is[3] = {min(max(i + sx, 0), n0 - 1), i, min(max(i + sx, 0), n0 - 1)};
  const int js[3] = {j, min(max(j + sy, 0), n0 - 1), min(max(j + sy, 0), n0 - 1)};
  float pmax = pv[4], pmin = pv[4], nmax = nv[4], nmin = nv[4], xp = 0.f, xn = 0.f;
  int emit = 0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const float a = pv[ms[e]], c = nv[ms[e]];
    pmax = fmaxf(pmax, a);
    pmin = fminf(pmin, a);
    nmax = fmaxf(nmax, c);
    nmin = fminf(nmin, c);
    if (a > 0.f) ++emit;
    const int qn = js[e] * n0 + is[e];
    xp = fmaxf(xp, xi_p[qn]);
    xn = fmaxf(xn, xi_n[qn]);
  }
  const float gu = (pv[2] + 2.f * pv[5] + pv[8]) - (pv[0] + 2.f * pv[3] + pv[6]);
  const float gv = (pv[6] + 2.f * pv[7] + pv[8]) - (pv[0] + 2.f * pv[1] + pv[2]);
  const float tiny = 1e-30f;
  float f[kFeat];
  f[0] = xi_p[k];
  f[1] = xi_n[k];
  f[2] = pv[4] > 0.f ? 1.f : 0.f;
  f[3] = (float)sx * gu / (sp + tiny);
  f[4] = (float)sy * gv / (sp + tiny);
  f[5] = (pmax - pmin) / (pmax + tiny);
  f[6] = (nmax - nmin) / (nmax + tiny);
  // band-0 optical depth: the march's kappa_0 N, or formed here the same way
  f[7] = fminf(tau0 ? tau0[k] : (kappa ? kappa[0] * nv[4] : 0.f), 10.f) * 0.1f;
  f[8] = maxlev ? (float)maxlev[k] / (float)max(1, grid_levels) : 0.f;
  f[9] = (float)emit * (1.f / 3.f);
  f[10] = fminf(fmaxf(log10f(nv[4] + tiny) * 0.1f, -3.f), 3.f);
  f[11] = fminf(fmaxf(log10f(pv[4] + tiny) * 0.05f, -3.f), 3.f);
  f[12] = xp;
  f[13] = xn;
  f[14] = pv[4] / (pmax + tiny);
  f[15] = 1.f;
#pragma unroll
  for (int c = 0; c < kFeat; ++c) x[s * kFeat + c] = f2bf(f[c]);
}

// Depth label of every quadrant sample 4 b + q: the deepest node below
// base pixel b's level-1 pixel q (nodes [0, n)); 1 for every quadrant of a
// refined base pixel whose level-1 pixel is a leaf; the labels must be zeroed
// first.
__global__ void k_depth_labels(const int8_t *lvl, const int32_t *pi, const int32_t *pj, int64_t n,
                               int n0, int32_t *label) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  // labels start at zero (the base level); children come in groups of four
  // at n0^2 + 4 m, all of one level and one quadrant below level 1: the
  // first of each group stands for it
  const int64_t nbase = (int64_t)n0 * n0;
  if (k < nbase || ((k - nbase) & 3) != 0) return;
  const int L = lvl[k];
  const int64_t b = (int64_t)(pj[k] >> L) * n0 + (pi[k] >> L);
  if (L == 1) {
    for (int q = 0; q < 4; ++q) atomicMax(label + 4 * b + q, 1);
    return;
  }
  const int q = ((pi[k] >> (L - 1)) & 1) + 2 * ((pj[k] >> (L - 1)) & 1);
  atomicMax(label + 4 * b + q, L);
}

// Decision: the smallest depth d whose cumulative probability reaches q.
__global__ void k_decide(const float *logits, int n, int max_level, float q, int8_t *depth) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float l[5], m = -INFINITY;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    l[c] = logits[(int64_t)k * 5 + c];
    m = fmaxf(m, l[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    l[c] = expf(l[c] - m);
    s += l[c];
  }
  float acc = 0.f;
  int d = 4;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    acc += l[c] / s;
    if (acc >= q) {
      d = c;
      break;
    }
  }
  depth[k] = (int8_t)min(d, max_level);
}

// Per block of kScanItems base pixels: proposal rays (prop_rays of each
// pixel's four quadrant depths).
__global__ void __launch_bounds__(256) k_prop_count(const int8_t *depth, int64_t nb, int32_t *bcount) {
  __shared__ int64_t s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * kScanItems, s1 = min(nb, s0 + kScanItems);
  int64_t c = 0;
  for (int64_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) c += prop_rays(depth + 4 * k);
  atomicAdd((unsigned long long *)&s, (unsigned long long)c);
  __syncthreads();
  if (threadIdx.x == 0) bcount[blockIdx.x] = (int32_t)s;
}

// First proposal ray of every base pixel (sequential within the block by a
// shared-memory scan).
__global__ void __launch_bounds__(256) k_prop_offsets(const int8_t *depth, int64_t nb,
                                                      const int64_t *boff, int64_t *off) {
  __shared__ int64_t part[256];
  const int64_t s0 = (int64_t)blockIdx.x * kScanItems, s1 = min(nb, s0 + kScanItems);
  const int64_t per = (kScanItems + 255) / 256;
  const int64_t a = s0 + threadIdx.x * per, b = min(s1, a + per);
  int64_t c = 0;
  for (int64_t k = a; k < b; ++k) c += prop_rays(depth + 4 * k);
  part[threadIdx.x] = c;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int64_t u = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += u;
    __syncthreads();
  }
  int64_t run = boff[blockIdx.x] + part[threadIdx.x] - c;
  for (int64_t k = a; k < b; ++k) {
    off[k] = run;
    run += prop_rays(depth + 4 * k);
  }
}

// The proposal rays: one warp per base pixel, its lanes striding over the
// pixel's rays in the Proposal layout (the four level-1 pixels, then each
// quadrant's subtree level by level, row-major within a level), so the
// writes are coalesced and no thread carries a whole subtree.
// Base pixels of several views lie view-major (pixel k of view k / n0^2);
// pview (may be NULL) receives each proposal ray's view.
__global__ void __launch_bounds__(256) k_prop_fill(const int8_t *depth, int64_t nb, int n0,
                                                   const int64_t *off, int8_t *plvl, int32_t *ppi,
                                                   int32_t *ppj, int16_t *pview) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nb) return;
  const int8_t *d4 = depth + 4 * k;
  const int64_t base = off[k], size = prop_rays(d4);
  const int64_t nn0 = (int64_t)n0 * n0;
  const int64_t r0 = k % nn0;
  const int bi = (int)(r0 % n0), bj = (int)(r0 / n0);
  if (pview)
    for (int64_t r = lane; r < size; r += 32) pview[base + r] = (int16_t)(k / nn0);
  for (int64_t r = lane; r < size; r += 32) {
    int L, i, j;
    prop_ray(d4, r, bi, bj, L, i, j);
    plvl[base + r] = (int8_t)L;
    ppi[base + r] = i;
    ppj[base + r] = j;
  }
}

// New nodes [first, n): copy their values from the proposal wave when the
// proposal covers them; otherwise flag them for the fallback wave.
__global__ void k_gather(TreeView t, int64_t first, int64_t n, int n_bands, const int8_t *depth,
                         const int64_t *off, const float *pN, const float *pI, int64_t pstride,
                         const float *pp, const uint32_t *psteps, uint32_t *missing) {
  const int64_t k = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int L = t.lvl[k], i = t.pi[k], j = t.pj[k];
  const int64_t b = (int64_t)(j >> L) * t.n0 + (i >> L);
  const int64_t q = prop_index(depth + 4 * b, off[b], L, i, j);
  if (q < 0) {
    missing[k - first] = 1u;
    return;
  }
  missing[k - first] = 0u;
  t.N[k] = pN[q];
  t.p[k] = pp[q];
  t.steps[k] = psteps[q];
  for (int c = 0; c < n_bands; ++c) t.I[(int64_t)c * t.cap + k] = pI[(int64_t)c * pstride + q];
}

// Node indices of the flagged entries (in order).
__global__ void __launch_bounds__(256) k_list_missing(const uint32_t *missing, int64_t m,
                                                      const int64_t *boff, int64_t first,
                                                      int32_t *list) {
  __shared__ int32_t wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t start = (int64_t)blockIdx.x * kScanItems;
  int64_t run = boff[blockIdx.x];
  for (int rr = 0; rr < kScanRounds; ++rr) {
    const int64_t k = start + (int64_t)rr * kScanBlock + threadIdx.x;
    const bool p = k < m && missing[k];
    const uint32_t bal = __ballot_sync(0xffffffffu, p);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int32_t before = 0, tot = 0;
    for (int w = 0; w < 8; ++w) {
      before += w < warp ? wsum[w] : 0;
      tot += wsum[w];
    }
    if (p) list[run + before + __popc(bal & ((1u << lane) - 1u))] = (int32_t)(first + k);
    run += tot;
    __syncthreads();
  }
}

// Final depth per quadrant sample vs the proposal: under / over counts.
__global__ void k_pred_stats(const int32_t *label, const int8_t *depth, int nb,
                             unsigned long long *under, unsigned long long *over) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  if (label[k] > depth[k]) atomicAdd(under, 1ull);
  if (label[k] < depth[k]) atomicAdd(over, 1ull);
}

#define CU_TRY(x)                                    \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Base image of one view traced into the quadtree workspace (nodes [0, n0^2))
// with band-0 optical depth and deepest level, then the features of its
// 4 n0^2 quadrant samples -> x.
static air_status base_and_features(air_grid *g, const Camera &cam, const air_params *pr,
                                    uint16_t *x, cudaStream_t st) {
  Workspace &w = g->ws;
  LearnWork &lw = g->learn;
  const int n0 = pr->base_res;
  const int64_t nbase = (int64_t)n0 * n0;
  TreeView t = w.tree(n0, pr->max_level);
  CU_TRY(ensure((void **)&lw.tau0, &lw.tau0_b, sizeof(float) * nbase));
  CU_TRY(ensure((void **)&lw.maxlev, &lw.maxlev_b, nbase));
  CU_TRY(ensure((void **)&lw.xi_p, &lw.xi_p_b, sizeof(float) * nbase));
  CU_TRY(ensure((void **)&lw.xi_n, &lw.xi_n_b, sizeof(float) * nbase));
  CU_TRY(launch_init_base(t, st));
  RaySource src{};
  src.mode = 0; src.n0 = n0; src.lvl = t.lvl; src.pi = t.pi; src.pj = t.pj; src.first = 0; src.count = nbase;
  {
    const air_status sa = axis_table(g, cam, n0, pr->max_level, src);
    if (sa) return sa;
  }
  RayOut ro{t.N, t.I, t.cap, t.steps, t.p, lw.tau0, lw.maxlev};
  const MarchTune tune = march_tune(g, pr->fp64_level);
  CU_TRY(prof_open(g, AIR_PHASE_MARCH, g->gv.n_bands > (tune.nbt > 0 ? tune.nbt : default_bands_per_thread(g->gv.n_bands)) ? 2 : 1));
  CU_TRY(launch_march(g->gv, cam, src, ro, tune, st));
  CU_TRY(prof_close(g));
  CU_TRY(prof_open(g, AIR_PHASE_LEARN, 2));
  k_base_xi<<<nblk(nbase, 256), 256, 0, st>>>(t.p, t.N, n0, lw.xi_p, lw.xi_n);
  k_features<<<nblk(4 * nbase, 256), 256, 0, st>>>(t.p, t.N, lw.tau0, lw.maxlev, lw.xi_p, lw.xi_n, n0,
                                               g->gv.kind == AIR_GRID_AMR ? g->gv.Lm : 0, x, nullptr);
  CU_TRY(cudaGetLastError());
  CU_TRY(prof_close(g));
  return AIR_OK;
}

air_status batch_proposal(air_grid *g, int V, const air_params *pr, air_mlp *mlp, double q,
                          const uint8_t *maxlev, int64_t *P_out) {
  Workspace &w = g->ws;
  LearnWork &lw = g->learn;
  cudaStream_t st = g->stream;
  const int n0 = pr->base_res, Lm = pr->max_level;
  const int64_t nn0 = (int64_t)n0 * n0, nbase = (int64_t)V * nn0;
  const int nb = g->gv.n_bands;
  TreeView t = w.tree(n0, Lm);
  CU_TRY(ensure((void **)&lw.xi_p, &lw.xi_p_b, sizeof(float) * nbase));
  CU_TRY(ensure((void **)&lw.xi_n, &lw.xi_n_b, sizeof(float) * nbase));
  CU_TRY(ensure((void **)&lw.x, &lw.x_b, sizeof(uint16_t) * 4 * nbase * kFeat));
  CU_TRY(ensure((void **)&lw.logits, &lw.logits_b, sizeof(float) * 4 * nbase * 5));
  CU_TRY(ensure((void **)&lw.depth, &lw.depth_b, 4 * nbase));
  CU_TRY(ensure((void **)&lw.off, &lw.off_b, sizeof(int64_t) * nbase));
  CU_TRY(ensure((void **)&w.bcount, &w.bcount_b, sizeof(int32_t) * scan_blocks(nbase)));
  CU_TRY(ensure((void **)&w.boff, &w.boff_b, sizeof(int64_t) * scan_blocks(nbase)));
  // features of every view's base image (view v: nodes [v n0^2, (v + 1) n0^2))
  CU_TRY(prof_open(g, AIR_PHASE_LEARN, 2 * V + 5));
  for (int v = 0; v < V; ++v) {
    const int64_t o = (int64_t)v * nn0;
    k_base_xi<<<nblk(nn0, 256), 256, 0, st>>>(t.p + o, t.N + o, n0, lw.xi_p + o, lw.xi_n + o);
    k_features<<<nblk(4 * nn0, 256), 256, 0, st>>>(t.p + o, t.N + o, nullptr, maxlev + o, lw.xi_p + o,
                                                   lw.xi_n + o, n0, g->gv.kind == AIR_GRID_AMR ? g->gv.Lm : 0,
                                                   lw.x + 4 * o * kFeat, g->gv.kappa);
  }
  CU_TRY(cudaGetLastError());
  air_status s = mlp_forward(mlp, lw.x, 4 * nbase, lw.logits, st);
  if (s) return s;
  k_decide<<<nblk(4 * nbase, 256), 256, 0, st>>>(lw.logits, (int)(4 * nbase), Lm, (float)q, lw.depth);
  const int64_t nbb = scan_blocks(nbase);
  k_prop_count<<<(unsigned)nbb, 256, 0, st>>>(lw.depth, nbase, w.bcount);
  CU_TRY(cudaGetLastError());
  CU_TRY(launch_scan_offsets(w.bcount, nbb, w.boff, w.d_total, st));
  CU_TRY(cudaMemcpyAsync(w.h_total, w.d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaStreamSynchronize(st));
  const int64_t P = *w.h_total, P1 = std::max<int64_t>(P, 1);
  CU_TRY(ensure((void **)&lw.plvl, &lw.plvl_b, P1));
  CU_TRY(ensure((void **)&lw.ppi, &lw.ppi_b, sizeof(int32_t) * P1));
  CU_TRY(ensure((void **)&lw.ppj, &lw.ppj_b, sizeof(int32_t) * P1));
  CU_TRY(ensure((void **)&lw.pview, &lw.pview_b, sizeof(int16_t) * P1));
  CU_TRY(ensure((void **)&lw.pN, &lw.pN_b, sizeof(float) * P1));
  CU_TRY(ensure((void **)&lw.pI, &lw.pI_b, sizeof(float) * P1 * nb));
  CU_TRY(ensure((void **)&lw.pp, &lw.pp_b, sizeof(float) * P1));
  CU_TRY(ensure((void **)&lw.psteps, &lw.psteps_b, sizeof(uint32_t) * P1));
  k_prop_offsets<<<(unsigned)nbb, 256, 0, st>>>(lw.depth, nbase, w.boff, lw.off);
  k_prop_fill<<<nblk(nbase * 32, 256), 256, 0, st>>>(lw.depth, nbase, n0, lw.off, lw.plvl, lw.ppi, lw.ppj,
                                                     lw.pview);
  CU_TRY(cudaGetLastError());
  CU_TRY(prof_close(g));
  *P_out = P;
  return AIR_OK;
}

air_status learn_samples(air_grid *g, const air_view *view, const air_params *pr, uint16_t *x,
                         int32_t *y) {
  Camera cam;
  air_status s = make_camera(view, cam);
  if (s) return s;
  if (!x) return set_error(AIR_ERR_ARG, "x must not be NULL");
  const int n0 = pr->base_res;
  cudaStream_t st = g->stream;
  if (y) {
    // the plain render, then the depth reached under every base pixel
    air_image im{};
    im.mem = AIR_DEVICE;
    im.capacity = 0;
    s = render_adaptive(g, view, pr, &im);
    if (s != AIR_OK && s != AIR_ERR_CAPACITY) return s;
    set_error(AIR_OK, "");
    TreeView t = g->ws.tree(n0, pr->max_level);
    CU_TRY(cudaMemsetAsync(y, 0, sizeof(int32_t) * 4 * n0 * n0, st));
    k_depth_labels<<<nblk(g->last.n_nodes, 256), 256, 0, st>>>(t.lvl, t.pi, t.pj, g->last.n_nodes, n0, y);
    CU_TRY(cudaGetLastError());
    g->last.valid = false;
  }
  if ((s = init_scalars(g->ws))) return s;
  int64_t bound = 0;
  for (int l = 0; l <= pr->max_level; ++l) bound += ((int64_t)n0 << l) * ((int64_t)n0 << l);
  if ((s = ensure_nodes(g, std::max<int64_t>((int64_t)n0 * n0, g->ws.cap), 0, bound))) return s;
  g->prof.used = 0;
  s = base_and_features(g, cam, pr, x, st);
  if (s) return s;
  CU_TRY(cudaStreamSynchronize(st));
  CU_TRY(prof_resolve(g));
  return AIR_OK;
}

air_status render_learned(air_grid *g, const air_view *view, const air_params *pr, air_mlp *mlp,
                          const air_learned_opts *opts, air_image *im, air_learned_stats *stats) {
  g->raster.ok = false;  // the workspace tree is about to change
  air_status s = check_image(im);
  if (s) return s;
  Camera cam;
  if ((s = make_camera(view, cam))) return s;
  if (!pr || !mlp) return set_error(AIR_ERR_ARG, "params and mlp must not be NULL");
  const int n0 = pr->base_res, Lm = pr->max_level;
  if (n0 < 1 || Lm < 0 || Lm >= kMaxLevels || ((int64_t)n0 << Lm) > (1 << 20))
    return set_error(AIR_ERR_ARG, "need base_res >= 1, 0 <= max_level < %d, base_res << max_level <= 2^20", kMaxLevels);
  if (!std::isfinite(pr->xi_crit) || pr->xi_crit < 0.0) return set_error(AIR_ERR_ARG, "xi_crit must be finite and >= 0");
  if (pr->xi_norm != 0 && pr->xi_norm != 1) return set_error(AIR_ERR_ARG, "xi_norm must be 0 or 1");
  if (pr->refine_on < 0 || pr->refine_on > 2) return set_error(AIR_ERR_ARG, "refine_on must be 0, 1 or 2");
  if (pr->include_interior != 0 && pr->include_interior != 1) return set_error(AIR_ERR_ARG, "include_interior must be 0 or 1");
  const double q = (opts && opts->quantile > 0.0 && opts->quantile <= 1.0) ? opts->quantile : 0.8;
  if ((s = init_scalars(g->ws))) return s;
  Workspace &w = g->ws;
  LearnWork &lw = g->learn;
  const int nb = g->gv.n_bands;
  cudaStream_t st = g->stream;
  g->last.valid = false;
  const int64_t nbase = (int64_t)n0 * n0;
  int64_t bound = 0;
  for (int l = 0; l <= Lm; ++l) bound += ((int64_t)n0 << l) * ((int64_t)n0 << l);
  if (bound > INT32_MAX) return set_error(AIR_ERR_ARG, "image pyramid exceeds 2^31 nodes");
  CU_TRY(ensure((void **)&w.bcount, &w.bcount_b, sizeof(int32_t) * scan_blocks(bound)));
  CU_TRY(ensure((void **)&w.boff, &w.boff_b, sizeof(int64_t) * scan_blocks(bound)));
  // the replay runs with its counts on the device when the node arrays can
  // hold the whole pyramid (as the plain render's loop)
  const bool dev_loop = pyramid_fits(g, bound);
  if ((s = ensure_nodes(g, dev_loop ? bound : std::min<int64_t>(bound, std::max<int64_t>(4 * nbase, w.cap)),
                        0, bound))) return s;
  CU_TRY(ensure((void **)&lw.x, &lw.x_b, sizeof(uint16_t) * 4 * nbase * kFeat));
  CU_TRY(ensure((void **)&lw.logits, &lw.logits_b, sizeof(float) * 4 * nbase * 5));
  CU_TRY(ensure((void **)&lw.depth, &lw.depth_b, 4 * nbase));
  CU_TRY(ensure((void **)&lw.off, &lw.off_b, sizeof(int64_t) * nbase));
  CU_TRY(ensure((void **)&lw.label, &lw.label_b, sizeof(int32_t) * 4 * nbase));
  CU_TRY(ensure((void **)&lw.counters, &lw.counters_b, sizeof(unsigned long long) * 2));
  g->prof.used = 0;
  int waves = 0;
  // steps i-ii + features + the network's proposal
  if ((s = base_and_features(g, cam, pr, lw.x, st))) return s;
  ++waves;
  CU_TRY(prof_open(g, AIR_PHASE_LEARN, 1));
  if ((s = mlp_forward(mlp, lw.x, 4 * nbase, lw.logits, st))) return s;
  CU_TRY(prof_close(g));
  CU_TRY(prof_open(g, AIR_PHASE_LEARN, 5));
  k_decide<<<nblk(4 * nbase, 256), 256, 0, st>>>(lw.logits, (int)(4 * nbase), Lm, (float)q, lw.depth);
  CU_TRY(cudaGetLastError());
  const int64_t nbb = scan_blocks(nbase);
  k_prop_count<<<(unsigned)nbb, 256, 0, st>>>(lw.depth, nbase, w.bcount);
  CU_TRY(cudaGetLastError());
  CU_TRY(launch_scan_offsets(w.bcount, nbb, w.boff, w.d_total, st));
  CU_TRY(cudaMemcpyAsync(w.h_total, w.d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaStreamSynchronize(st));
  const int64_t P = *w.h_total;
  CU_TRY(ensure((void **)&lw.plvl, &lw.plvl_b, std::max<int64_t>(P, 1)));
  CU_TRY(ensure((void **)&lw.ppi, &lw.ppi_b, sizeof(int32_t) * std::max<int64_t>(P, 1)));
  CU_TRY(ensure((void **)&lw.ppj, &lw.ppj_b, sizeof(int32_t) * std::max<int64_t>(P, 1)));
  CU_TRY(ensure((void **)&lw.pN, &lw.pN_b, sizeof(float) * std::max<int64_t>(P, 1)));
  CU_TRY(ensure((void **)&lw.pI, &lw.pI_b, sizeof(float) * std::max<int64_t>(P, 1) * nb));
  CU_TRY(ensure((void **)&lw.pp, &lw.pp_b, sizeof(float) * std::max<int64_t>(P, 1)));
  CU_TRY(ensure((void **)&lw.psteps, &lw.psteps_b, sizeof(uint32_t) * std::max<int64_t>(P, 1)));
  k_prop_offsets<<<(unsigned)nbb, 256, 0, st>>>(lw.depth, nbase, w.boff, lw.off);
  k_prop_fill<<<nblk(nbase * 32, 256), 256, 0, st>>>(lw.depth, nbase, n0, lw.off, lw.plvl, lw.ppi, lw.ppj,
                                                     nullptr);
  CU_TRY(cudaGetLastError());
  CU_TRY(prof_close(g));
  const MarchTune tune = march_tune(g, pr->fp64_level);
  const int march_launches = nb > (tune.nbt > 0 ? tune.nbt : default_bands_per_thread(nb)) ? 2 : 1;
  if (P > 0) {
    // the proposal wave: every pixel of every proposed subtree
    RaySource ps{};
    ps.mode = 0; ps.n0 = n0; ps.lvl = lw.plvl; ps.pi = lw.ppi; ps.pj = lw.ppj; ps.first = 0; ps.count = P;
    if ((s = axis_table(g, cam, n0, Lm, ps))) return s;
    RayOut po{lw.pN, lw.pI, std::max<int64_t>(P, 1), lw.psteps, lw.pp};
    CU_TRY(prof_open(g, AIR_PHASE_MARCH, march_launches));
    CU_TRY(launch_march(g->gv, cam, ps, po, tune, st));
    CU_TRY(prof_close(g));
    ++waves;
  }
  // plain AIR over the traced values (steps iii-v)
  TreeView t = w.tree(n0, Lm);
  CU_TRY(cudaMemsetAsync(w.d_err, 0, sizeof(uint32_t), st));
  int64_t n = nbase, n_refined = 0, fallback = 0;
  int32_t sweeps = 0;
  // steps iii-iv over the open-leaf list, as in the plain loop
  const int64_t open_max = std::max<int64_t>(1, bound - ((int64_t)n0 << Lm) * ((int64_t)n0 << Lm));
  for (int k = 0; k < 2; ++k)
    CU_TRY(ensure((void **)&w.open[k], &w.open_b[k], sizeof(int32_t) * (size_t)open_max));
  CU_TRY(ensure((void **)&w.bcount, &w.bcount_b, 3 * sizeof(int32_t) * scan_blocks(bound)));
  CU_TRY(ensure((void **)&w.boff, &w.boff_b, 3 * sizeof(int64_t) * scan_blocks(bound)));
  int cur = 0;
  int64_t mo = Lm > 0 ? nbase : 0;
  CU_TRY(launch_list_init(w.open[0], mo, st));
  if (dev_loop) {
    // the device-count sweep loop; new pixels copy their values from the
    // proposal wave where it traced them, the march traces the rest
    int32_t *lmap = nullptr;
    if ((s = level_maps(g, n0, Lm, &lmap))) return s;
    const Proposal prop{lw.depth, lw.off, lw.pN, lw.pI, lw.pp, lw.psteps, std::max<int64_t>(P, 1)};
    SweepState fin;
    if ((s = sweep_loop_device(g, cam, pr, nbase, mo, bound, open_max, tune, march_launches, lmap, &prop,
                               &fin)))
      return s;
    n = fin.n;
    n_refined = fin.n_refined;
    sweeps = fin.sweeps;
    fallback = (int64_t)fin.fb_total;
    waves += fin.fb_waves;
    mo = 0;
  }
  for (;;) {
    if (mo == 0) break;
    CU_TRY(prof_open(g, AIR_PHASE_SCAN, 1));
    CU_TRY(launch_list_scan(t, w.open[cur], mo, pr->xi_crit, pr->xi_norm, pr->refine_on, w.flag, st));
    CU_TRY(prof_close(g));
    CU_TRY(prof_open(g, AIR_PHASE_BALANCE, 1));
    CU_TRY(launch_list_balance(t, w.open[cur], mo, w.flag, w.d_err, st));
    CU_TRY(prof_close(g));
    CU_TRY(prof_open(g, AIR_PHASE_REFINE, 2));
    CU_TRY(launch_list_count(t, w.open[cur], mo, w.flag, w.bcount, w.boff, w.d_total, st));
    CU_TRY(prof_close(g));
    CU_TRY(cudaMemcpyAsync(w.h_total, w.d_total, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CU_TRY(cudaStreamSynchronize(st));
    const int64_t nflag = w.h_total[0];
    const int64_t mo_next = w.h_total[1] + 4 * w.h_total[2];
    if (nflag == 0) break;
    const int64_t n_new = n + 4 * nflag;
    if (n_new > bound) return set_error(AIR_ERR_NUMERIC, "quadtree exceeds its bound");
    if (n_new > w.cap) {
      if ((s = ensure_nodes(g, n_new, n, bound))) return s;
      t = w.tree(n0, Lm);
    }
    CU_TRY(prof_open(g, AIR_PHASE_REFINE, 1));
    CU_TRY(launch_list_emit(t, w.open[cur], mo, w.flag, w.boff, w.d_total, n, w.open[cur ^ 1], st));
    CU_TRY(prof_close(g));
    // values of the new pixels: gathered from the proposal, or traced
    const int64_t m = 4 * nflag;
    CU_TRY(ensure((void **)&lw.missing, &lw.missing_b, sizeof(uint32_t) * m));
    CU_TRY(prof_open(g, AIR_PHASE_LEARN, 3));
    k_gather<<<nblk(m, 256), 256, 0, st>>>(t, n, n_new, nb, lw.depth, lw.off, lw.pN, lw.pI,
                                            std::max<int64_t>(P, 1), lw.pp, lw.psteps, lw.missing);
    CU_TRY(cudaGetLastError());
    CU_TRY(launch_count_flags(lw.missing, m, w.bcount, w.boff, w.d_total, st));
    CU_TRY(prof_close(g));
    CU_TRY(cudaMemcpyAsync(w.h_total, w.d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CU_TRY(cudaStreamSynchronize(st));
    const int64_t miss = *w.h_total;
    if (miss > 0) {
      CU_TRY(ensure((void **)&lw.list, &lw.list_b, sizeof(int32_t) * miss));
      CU_TRY(prof_open(g, AIR_PHASE_LEARN, 1));
      k_list_missing<<<(unsigned)scan_blocks(m), kScanBlock, 0, st>>>(lw.missing, m, w.boff, n, lw.list);
      CU_TRY(cudaGetLastError());
      CU_TRY(prof_close(g));
      RaySource fs{};
      fs.mode = 0; fs.n0 = n0; fs.lvl = t.lvl; fs.pi = t.pi; fs.pj = t.pj; fs.count = miss; fs.list = lw.list;
      if ((s = axis_table(g, cam, n0, Lm, fs))) return s;
      RayOut fo{t.N, t.I, t.cap, t.steps, t.p};
      CU_TRY(prof_open(g, AIR_PHASE_MARCH, march_launches));
      CU_TRY(launch_march(g->gv, cam, fs, fo, tune, st));
      CU_TRY(prof_close(g));
      fallback += miss;
      ++waves;
    }
    n = n_new;
    n_refined += nflag;
    ++sweeps;
    mo = mo_next;
    cur ^= 1;
  }
  CU_TRY(cudaMemcpyAsync(w.h_err, w.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaStreamSynchronize(st));
  if (*w.h_err) return set_error(AIR_ERR_NUMERIC, "balance closure overflowed its stack");
  // statistics of the proposal against the final tree
  CU_TRY(cudaMemsetAsync(lw.label, 0, sizeof(int32_t) * 4 * nbase, st));
  CU_TRY(cudaMemsetAsync(lw.counters, 0, sizeof(unsigned long long) * 2, st));
  k_depth_labels<<<nblk(n, 256), 256, 0, st>>>(t.lvl, t.pi, t.pj, n, n0, lw.label);
  k_pred_stats<<<nblk(4 * nbase, 256), 256, 0, st>>>(lw.label, lw.depth, (int)(4 * nbase), lw.counters,
                                                      lw.counters + 1);
  CU_TRY(cudaGetLastError());
  unsigned long long hc[2] = {0, 0};
  CU_TRY(cudaMemcpyAsync(hc, lw.counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
  // step vi: output, exactly as the plain render
  g->last.n_nodes = n;
  g->last.n_refined = n_refined;
  g->last.n_sweeps = sweeps;
  s = output_tree(g, cam, pr, im, n, n_refined, sweeps);
  if (s) return s;
  if (stats) {
    stats->proposed_rays = P;
    stats->used_rays = n - nbase - fallback;
    stats->wasted_rays = P - (n - nbase - fallback);
    stats->fallback_rays = fallback;
    stats->waves = waves;
    stats->sweeps = sweeps;
    stats->under_predicted = (int64_t)hc[0];
    stats->over_predicted = (int64_t)hc[1];
  }
  return AIR_OK;
}

void free_learn(air_grid *g) {
  LearnWork &l = g->learn;
  void *ps[] = {l.tau0, l.xi_p, l.xi_n, l.logits, l.maxlev, l.x, l.depth, l.plvl, l.off, l.label,
                l.ppi, l.ppj, l.list, l.pN, l.pI, l.pp, l.psteps, l.missing, l.counters, l.pview};
  for (void *p : ps)
    if (p) cudaFree(p);
  l = LearnWork{};
}

}  // namespace air

extern "C" {

air_status air_learn_samples(air_grid *g, const air_view *view, const air_params *params,
                             uint16_t *x, int32_t *y) {
  air::set_error(AIR_OK, "");
  if (!g || !view || !params) return air::set_error(AIR_ERR_ARG, "grid, view and params must not be NULL");
  if (params->base_res < 1) return air::set_error(AIR_ERR_ARG, "base_res must be >= 1");
  return air::learn_samples(g, view, params, x, y);
}

air_status air_render_learned(air_grid *g, const air_view *view, const air_params *params,
                              air_mlp *mlp, const air_learned_opts *opts, air_image *out,
                              air_learned_stats *stats) {
  air::set_error(AIR_OK, "");
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  return air::render_learned(g, view, params, mlp, opts, out, stats);
}

}  // extern "C"
