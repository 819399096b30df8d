// air_raster.cu -- Section 2 step vi: the output image as a finest-level
// raster, each finest pixel from the leaf that covers it, either that leaf's
// value or a bilinear interpolation on the leaf's own level between adjacent
// pixels of differing resolution (the super-resolution step the paper allows
// and leaves open).
#include "air_handle.cuh"
#include "air_tree.cuh"

namespace air {

// One thread per finest pixel (x, y) of an (n0 2^Lm)^2 raster. The covering
// leaf is the deepest node containing the pixel. For the bilinear form, with
// s = Lm - L, the pixel centre on the level-L grid is
// u = (x + 1/2) 2^-s - 1/2 = (2x + 1 - 2^s) / 2^(s+1): its floor is an
// arithmetic shift and its fraction an exact dyadic number, so the weights
// carry no rounding.
__global__ void k_raster(TreeView t, int Lm, int mode, const float *__restrict__ val,
                         float *__restrict__ out) {
  const int nf = t.n0 << Lm;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)nf * nf) return;
  const int x = (int)(k % nf), y = (int)(k / nf);
  const int leaf = descend(t, 0, Lm, x, y);
  if (mode == AIR_RASTER_NEAREST) {
    out[k] = val[leaf];
    return;
  }
  const int L = t.lvl[leaf];
  const int s = Lm - L;
  const int nl = t.n0 << L;
  const int nu = 2 * x + 1 - (1 << s), nv = 2 * y + 1 - (1 << s);
  const int i0 = nu >> (s + 1), j0 = nv >> (s + 1);
  const float sc = __int_as_float((127 - (s + 1)) << 23);  // 2^-(s+1)
  const float fu = (float)(nu - i0 * (2 << s)) * sc;
  const float fv = (float)(nv - j0 * (2 << s)) * sc;
  const int ia = min(max(i0, 0), nl - 1), ib = min(max(i0 + 1, 0), nl - 1);
  const int ja = min(max(j0, 0), nl - 1), jb = min(max(j0 + 1, 0), nl - 1);
  const float v00 = val[descend(t, 0, L, ia, ja)], v10 = val[descend(t, 0, L, ib, ja)];
  const float v01 = val[descend(t, 0, L, ia, jb)], v11 = val[descend(t, 0, L, ib, jb)];
  const float gu = 1.f - fu, gv = 1.f - fv;
  out[k] = (gu * gv) * v00 + (fu * gv) * v10 + (gu * fv) * v01 + (fu * fv) * v11;
}

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

air_status render_raster(air_grid *g, int32_t quantity, int32_t band, int32_t mode, float *out,
                         int64_t n_out) {
  if (!out) return set_error(AIR_ERR_ARG, "out must not be NULL");
  if (mode != AIR_RASTER_NEAREST && mode != AIR_RASTER_BILINEAR)
    return set_error(AIR_ERR_ARG, "unknown raster mode %d", mode);
  if (quantity != AIR_RASTER_INTENSITY && quantity != AIR_RASTER_SUM && quantity != AIR_RASTER_COLDENS)
    return set_error(AIR_ERR_ARG, "unknown raster quantity %d", quantity);
  if (!g->raster.ok) return set_error(AIR_ERR_ARG, "no single-view adaptive image to rasterise");
  if (quantity == AIR_RASTER_INTENSITY && (band < 0 || band >= g->gv.n_bands))
    return set_error(AIR_ERR_ARG, "band %d out of range", band);
  if (quantity == AIR_RASTER_INTENSITY && !g->ws.I)
    return set_error(AIR_ERR_ARG, "the image's band intensities were streamed to host memory");
  const int n0 = g->raster.n0, Lm = g->raster.Lm;
  const int64_t nf = (int64_t)n0 << Lm;
  if (nf > (1 << 30)) return set_error(AIR_ERR_ARG, "raster side %lld too large", (long long)nf);
  const int64_t n = nf * nf;
  if (n_out < n) return set_error(AIR_ERR_CAPACITY, "raster needs %lld floats, out holds %lld", (long long)n, (long long)n_out);
  Workspace &w = g->ws;
  const TreeView t = w.tree(n0, Lm);
  const float *val = quantity == AIR_RASTER_COLDENS ? t.N
                     : (quantity == AIR_RASTER_SUM ? t.p : t.I + (int64_t)band * t.cap);
  cudaStream_t st = g->stream;
  const bool dev = is_device_ptr(out);
  float *dst = out;
  if (!dev) {
    cudaError_t e = ensure((void **)&g->raster.scratch, &g->raster.scratch_b, sizeof(float) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e, "raster staging");
    dst = g->raster.scratch;
  }
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffff) return set_error(AIR_ERR_ARG, "raster too large");
  k_raster<<<(unsigned)blocks, 256, 0, st>>>(t, Lm, mode, val, dst);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(out, dst, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "air_render_raster");
  return AIR_OK;
}

}  // namespace air

extern "C" AIR_API air_status air_render_raster(air_grid *g, int32_t quantity, int32_t band,
                                                int32_t mode, float *out, int64_t n_out) {
  air::clear_error();
  if (!g) return air::set_error(AIR_ERR_ARG, "grid handle is NULL");
  return air::render_raster(g, quantity, band, mode, out, n_out);
}
