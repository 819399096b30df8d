// air_mlp.cu -- the refinement-depth network: a perceptron 16 -> 64 -> 64 -> 5
// (ReLU), BF16 weights and activations with FP32 accumulation, trained with
// softmax cross-entropy and Adam. Not in the paper: it proposes, per quadrant
// of every base pixel, the depth plain AIR will reach, so the finest rays can
// be traced in one wave; the paper's criterion still decides the image
// (air_learned.cu).
//
// Tensor cores: every layer of the forward pass and both data-gradient
// products of the backward pass are mma.sync m16n8k16 (BF16 in, FP32 out). A
// warp owns 32 samples (two 16-row tiles); the FP32 accumulator fragments of
// two adjacent 8-column tiles are exactly the BF16 A-operand fragment of the
// next 16-wide K slice, so layers chain in registers. The weight gradients
// dW = act^T d over the block's 128 samples are mma.sync products as well:
// the activations are staged in BF16 (as the forward used them) and read
// transposed by ldmatrix.trans; each d is staged as two BF16 parts, hi =
// bf16(d) and lo = bf16(d - hi), and both products are accumulated, so d
// keeps about 16 significant bits (error <= 2^-16 |d| per term, against the
// FP32 sums of the plain form's 2^-24). Bias gradients are column sums of
// hi + lo. Per-block sums are reduced over blocks in a fixed order
// (deterministic).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "air_handle.cuh"

namespace air {

constexpr int kIn = 16, kH = 64, kOut = 5, kOutP = 8;
constexpr int oW1 = 0, ob1 = oW1 + kIn * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kOut, kNP = ob3 + kOut;
static_assert(kNP == AIR_MLP_NPARAMS, "parameter count");
constexpr int kTile = 128;  // samples per block (4 warps x 32)

// BF16 copies of the weights in the layouts the fragments read, as 32-bit
// words (two BF16 along K per word):
//   W1T [64][16]  forward layer 1, B[k][n] = W1[k][n] stored n-major
//   W2T [64][64]  forward layer 2, n-major
//   W3T [8][64]   forward layer 3 (outputs 5..7 zero), n-major
//   W3P [64][8]   backward d3 W3^T: B[k=out][n=hidden] = W3[n][k], row-major W3 padded
//   W2R [64][64]  backward d2 W2^T: B[k][n] = W2[n][k], row-major W2
constexpr int kW1T = 0, kW2T = kW1T + kH * kIn / 2, kW3T = kW2T + kH * kH / 2,
              kW3P = kW3T + kOutP * kH / 2, kW2R = kW3P + kH * kOutP / 2, kWords = kW2R + kH * kH / 2;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ uint16_t bf16_bits(float x) {
  __nv_bfloat16 v = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t *>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ldmatrix: four (two) 8 x 8 BF16 blocks, transposed; lane l gives the
// address of row l & 7 of block l >> 3 (16-byte aligned) and receives
// elements (2 (l & 3), l >> 2) and (2 (l & 3) + 1, l >> 2) of each block.
__device__ __forceinline__ void ldsm_x4_trans(uint32_t r[4], const void *p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t r[2], const void *p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(s));
}

// Two values of d as BF16 parts: hi = bf16(v), lo = bf16(v - hi), two per
// word (v0 in the low half).
__device__ __forceinline__ void stage_hi_lo(uint32_t *h, uint32_t *l, int w, float v0, float v1) {
  const uint32_t hw = pack_bf16(v0, v1);
  h[w] = hw;
  l[w] = pack_bf16(v0 - bf16_lo(hw), v1 - bf16_hi(hw));
}

__global__ void k_pack_weights(const float *__restrict__ th, uint32_t *__restrict__ w) {
  uint16_t *h = reinterpret_cast<uint16_t *>(w);
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < kWords * 2; x += gridDim.x * blockDim.x) {
    float v = 0.f;
    if (x < kW2T * 2) {  // W1T[n][k]
      const int n = x / kIn, k = x % kIn;
      v = th[oW1 + k * kH + n];
    } else if (x < kW3T * 2) {  // W2T[n][k]
      const int y = x - kW2T * 2, n = y / kH, k = y % kH;
      v = th[oW2 + k * kH + n];
    } else if (x < kW3P * 2) {  // W3T[n][k], n < 8
      const int y = x - kW3T * 2, n = y / kH, k = y % kH;
      v = n < kOut ? th[oW3 + k * kOut + n] : 0.f;
    } else if (x < kW2R * 2) {  // W3P[n][k], k < 8
      const int y = x - kW3P * 2, n = y / kOutP, k = y % kOutP;
      v = k < kOut ? th[oW3 + n * kOut + k] : 0.f;
    } else {  // W2R[n][k] = W2[n][k]
      const int y = x - kW2R * 2;
      v = th[oW2 + y];
    }
    h[x] = bf16_bits(v);
  }
}

struct MlpArgs {
  const uint32_t *x;   // [n][8] words: 16 BF16 features per sample
  const int32_t *y;    // [n] labels (training)
  int64_t n;
  float inv_count;     // 1 / (samples in the mean)
  const uint32_t *w;   // packed weights
  const float *th;     // FP32 parameters (biases)
  float *logits;       // [n][5] (forward)
  float *partial;      // [blocks][kNP + 1] gradient partials + loss (training)
};

// Shared memory of a training block (bytes): weights + staged tile.
constexpr size_t kSmW = sizeof(uint32_t) * kWords;
constexpr size_t kSmTrain = kSmW + sizeof(uint32_t) * kTile * (kIn / 2 + kH / 2 + kH / 2) +
                            sizeof(float) * kTile * (kH + kH + kOutP) + sizeof(float) * 4;

template <bool TRAIN>
__global__ void __launch_bounds__(kTile) k_mlp(MlpArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t *sw = sm;
  for (int x = threadIdx.x; x < kWords; x += blockDim.x) sw[x] = a.w[x];
  uint32_t *xs = sm + kWords;                 // [128][8]
  uint32_t *h1s = xs + kTile * (kIn / 2);     // [128][32]
  uint32_t *h2s = h1s + kTile * (kH / 2);     // [128][32]
  // back-propagated errors, two BF16 parts each (hi, lo), two per word along
  // the output unit: d1 and d2 [128][64], d3 [128][8]
  uint32_t *d1h = h2s + kTile * (kH / 2), *d1l = d1h + kTile * (kH / 2);
  uint32_t *d2h = d1l + kTile * (kH / 2), *d2l = d2h + kTile * (kH / 2);
  uint32_t *d3h = d2l + kTile * (kH / 2), *d3l = d3h + kTile * (kOutP / 2);
  float *lsum = reinterpret_cast<float *>(d3l + kTile * (kOutP / 2));  // [4] per-warp loss
  __syncthreads();
  const uint32_t *W1T = sw + kW1T, *W2T = sw + kW2T, *W3T = sw + kW3T, *W3P = sw + kW3P, *W2R = sw + kW2R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  float wloss = 0.f;
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = warp * 32 + mt * 16;                 // row in the tile
    const int64_t gr0 = (int64_t)blockIdx.x * kTile + r0;  // global sample
    const int64_t ra = gr0 + g, rb = gr0 + g + 8;
    const bool va = ra < a.n, vb = rb < a.n;
    uint32_t ax[4];
    ax[0] = va ? a.x[ra * 8 + t] : 0u;
    ax[1] = vb ? a.x[rb * 8 + t] : 0u;
    ax[2] = va ? a.x[ra * 8 + t + 4] : 0u;
    ax[3] = vb ? a.x[rb * 8 + t + 4] : 0u;
    // layer 1
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float b0 = a.th[ob1 + nt * 8 + 2 * t], b1 = a.th[ob1 + nt * 8 + 2 * t + 1];
      acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
      const uint32_t *wr = W1T + (nt * 8 + g) * (kIn / 2);
      mma16816(acc[nt], ax, wr[t], wr[t + 4]);
    }
    uint32_t a2[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      a2[kt][0] = pack_bf16(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
      a2[kt][1] = pack_bf16(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
      a2[kt][2] = pack_bf16(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
      a2[kt][3] = pack_bf16(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
    }
    // layer 2
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float b0 = a.th[ob2 + nt * 8 + 2 * t], b1 = a.th[ob2 + nt * 8 + 2 * t + 1];
      acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
      const uint32_t *wr = W2T + (nt * 8 + g) * (kH / 2);
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) mma16816(acc[nt], a2[kt], wr[kt * 8 + t], wr[kt * 8 + t + 4]);
    }
    uint32_t a3[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      a3[kt][0] = pack_bf16(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
      a3[kt][1] = pack_bf16(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
      a3[kt][2] = pack_bf16(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
      a3[kt][3] = pack_bf16(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
    }
    // layer 3 (outputs 0..4 of 8)
    float lg[4];
    {
      const int c0 = 2 * t, c1 = 2 * t + 1;
      const float b0 = c0 < kOut ? a.th[ob3 + c0] : 0.f, b1 = c1 < kOut ? a.th[ob3 + c1] : 0.f;
      lg[0] = b0; lg[1] = b1; lg[2] = b0; lg[3] = b1;
      const uint32_t *wr = W3T + g * (kH / 2);
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) mma16816(lg, a3[kt], wr[kt * 8 + t], wr[kt * 8 + t + 4]);
    }
    if (!TRAIN) {
      if (a.logits) {
        const int c0 = 2 * t, c1 = 2 * t + 1;
        if (va) {
          if (c0 < kOut) a.logits[ra * kOut + c0] = lg[0];
          if (c1 < kOut) a.logits[ra * kOut + c1] = lg[1];
        }
        if (vb) {
          if (c0 < kOut) a.logits[rb * kOut + c0] = lg[2];
          if (c1 < kOut) a.logits[rb * kOut + c1] = lg[3];
        }
      }
      continue;
    }
    // ---- training: stage activations (BF16, as used in the products)
    const int la = r0 + g, lb = r0 + g + 8;
    xs[la * 8 + t] = ax[0];
    xs[lb * 8 + t] = ax[1];
    xs[la * 8 + t + 4] = ax[2];
    xs[lb * 8 + t + 4] = ax[3];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      h1s[la * 32 + kt * 8 + t] = a2[kt][0];
      h1s[lb * 32 + kt * 8 + t] = a2[kt][1];
      h1s[la * 32 + kt * 8 + 4 + t] = a2[kt][2];
      h1s[lb * 32 + kt * 8 + 4 + t] = a2[kt][3];
      h2s[la * 32 + kt * 8 + t] = a3[kt][0];
      h2s[lb * 32 + kt * 8 + t] = a3[kt][1];
      h2s[la * 32 + kt * 8 + 4 + t] = a3[kt][2];
      h2s[lb * 32 + kt * 8 + 4 + t] = a3[kt][3];
    }
    // softmax cross-entropy on rows g and g+8 (a quad holds one row's 8 columns)
    float d3[4];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const bool vr = half ? vb : va;
      const float l0 = lg[2 * half], l1 = lg[2 * half + 1];
      const bool v0 = 2 * t < kOut, v1 = 2 * t + 1 < kOut;
      float m = fmaxf(v0 ? l0 : -INFINITY, v1 ? l1 : -INFINITY);
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
      const float e0 = v0 ? expf(l0 - m) : 0.f, e1 = v1 ? expf(l1 - m) : 0.f;
      float s = e0 + e1;
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      const int yr = vr ? a.y[half ? rb : ra] : -1;
      const float p0 = e0 / s, p1 = e1 / s;
      d3[2 * half] = (vr && v0) ? (p0 - (yr == 2 * t ? 1.f : 0.f)) * a.inv_count : 0.f;
      d3[2 * half + 1] = (vr && v1) ? (p1 - (yr == 2 * t + 1 ? 1.f : 0.f)) * a.inv_count : 0.f;
      if (vr && yr == 2 * t) wloss -= logf(p0);
      if (vr && yr == 2 * t + 1) wloss -= logf(p1);
    }
    stage_hi_lo(d3h, d3l, la * (kOutP / 2) + t, d3[0], d3[1]);
    stage_hi_lo(d3h, d3l, lb * (kOutP / 2) + t, d3[2], d3[3]);
    // d2 = (d3 W3^T) * [z2 > 0]
    const uint32_t ad3[4] = {pack_bf16(d3[0], d3[1]), pack_bf16(d3[2], d3[3]), 0u, 0u};
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
      mma16816(acc[nt], ad3, W3P[(nt * 8 + g) * (kOutP / 2) + t], 0u);
      const uint32_t hg = a3[nt >> 1][(nt & 1) * 2], hg8 = a3[nt >> 1][(nt & 1) * 2 + 1];
      if (bf16_lo(hg) == 0.f) acc[nt][0] = 0.f;
      if (bf16_hi(hg) == 0.f) acc[nt][1] = 0.f;
      if (bf16_lo(hg8) == 0.f) acc[nt][2] = 0.f;
      if (bf16_hi(hg8) == 0.f) acc[nt][3] = 0.f;
      stage_hi_lo(d2h, d2l, la * (kH / 2) + nt * 4 + t, acc[nt][0], acc[nt][1]);
      stage_hi_lo(d2h, d2l, lb * (kH / 2) + nt * 4 + t, acc[nt][2], acc[nt][3]);
    }
    uint32_t ad2[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      ad2[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
      ad2[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
      ad2[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
      ad2[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
    }
    // d1 = (d2 W2^T) * [z1 > 0]
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
      const uint32_t *wr = W2R + (nt * 8 + g) * (kH / 2);
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) mma16816(acc[nt], ad2[kt], wr[kt * 8 + t], wr[kt * 8 + t + 4]);
      const uint32_t hg = a2[nt >> 1][(nt & 1) * 2], hg8 = a2[nt >> 1][(nt & 1) * 2 + 1];
      if (bf16_lo(hg) == 0.f) acc[nt][0] = 0.f;
      if (bf16_hi(hg) == 0.f) acc[nt][1] = 0.f;
      if (bf16_lo(hg8) == 0.f) acc[nt][2] = 0.f;
      if (bf16_hi(hg8) == 0.f) acc[nt][3] = 0.f;
      stage_hi_lo(d1h, d1l, la * (kH / 2) + nt * 4 + t, acc[nt][0], acc[nt][1]);
      stage_hi_lo(d1h, d1l, lb * (kH / 2) + nt * 4 + t, acc[nt][2], acc[nt][3]);
    }
  }
  if (!TRAIN) return;
  // per-warp loss
  for (int off = 16; off > 0; off >>= 1) wloss += __shfl_xor_sync(0xffffffffu, wloss, off);
  if (lane == 0) lsum[warp] = wloss;
  __syncthreads();
  // weight gradients: 44 output tiles of 16 x 8 (dW1: 1 x 8, dW2: 4 x 8,
  // dW3: 4 x 1), a warp taking every fourth; each sums the 128 samples in 8
  // K steps of 16, hi and lo parts of d in turn (fixed order)
  float *out = a.partial + (int64_t)blockIdx.x * (kNP + 1);
  for (int tile = warp; tile < 44; tile += 4) {
    const uint32_t *act, *dh, *dl;
    int lda, ldd, m0, n0, ow, ncols;
    if (tile < 8) {
      act = xs; lda = kIn; dh = d1h; dl = d1l; ldd = kH; m0 = 0; n0 = tile * 8; ow = oW1; ncols = kH;
    } else if (tile < 40) {
      const int u = tile - 8;
      act = h1s; lda = kH; dh = d2h; dl = d2l; ldd = kH; m0 = (u >> 3) * 16; n0 = (u & 7) * 8;
      ow = oW2; ncols = kH;
    } else {
      act = h2s; lda = kH; dh = d3h; dl = d3l; ldd = kOutP; m0 = (tile - 40) * 16; n0 = 0;
      ow = oW3; ncols = kOut;
    }
    const uint16_t *ah = reinterpret_cast<const uint16_t *>(act);
    const uint16_t *bh = reinterpret_cast<const uint16_t *>(dh);
    const uint16_t *bl = reinterpret_cast<const uint16_t *>(dl);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int mi = lane >> 3, j = lane & 7;
#pragma unroll 2
    for (int r0 = 0; r0 < kTile; r0 += 16) {
      // A = act^T: 8 x 8 blocks (samples r0 + 8 (mi >> 1) .., features m0 + 8 (mi & 1) ..)
      uint32_t fa[4], fb[2], fl[2];
      ldsm_x4_trans(fa, ah + (r0 + j + ((mi >> 1) << 3)) * lda + m0 + ((mi & 1) << 3));
      // B = d: 8 x 8 blocks (samples r0 + 8 (mi & 1) .., units n0 ..)
      const int br = r0 + j + ((mi & 1) << 3);
      ldsm_x2_trans(fb, bh + br * ldd + n0);
      ldsm_x2_trans(fl, bl + br * ldd + n0);
      mma16816(acc, fa, fb[0], fb[1]);
      mma16816(acc, fa, fl[0], fl[1]);
    }
    // D[m][n]: (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int m = m0 + g + ((e >> 1) << 3), n = n0 + 2 * t + (e & 1);
      if (n < ncols) out[ow + m * ncols + n] = acc[e];
    }
  }
  // bias gradients: column sums of hi + lo over the 128 samples (fixed order)
  for (int c = threadIdx.x; c < 2 * kH + kOut; c += blockDim.x) {
    const uint16_t *bh, *bl;
    int ldd, n, ob;
    if (c < kH) {
      bh = reinterpret_cast<const uint16_t *>(d1h); bl = reinterpret_cast<const uint16_t *>(d1l);
      ldd = kH; n = c; ob = ob1;
    } else if (c < 2 * kH) {
      bh = reinterpret_cast<const uint16_t *>(d2h); bl = reinterpret_cast<const uint16_t *>(d2l);
      ldd = kH; n = c - kH; ob = ob2;
    } else {
      bh = reinterpret_cast<const uint16_t *>(d3h); bl = reinterpret_cast<const uint16_t *>(d3l);
      ldd = kOutP; n = c - 2 * kH; ob = ob3;
    }
    float sum = 0.f;
    for (int r = 0; r < kTile; ++r)
      sum += __uint_as_float((uint32_t)bh[r * ldd + n] << 16) + __uint_as_float((uint32_t)bl[r * ldd + n] << 16);
    out[ob + n] = sum;
  }
  if (threadIdx.x == 0) out[kNP] = lsum[0] + lsum[1] + lsum[2] + lsum[3];
}

// grad[j] = sum over blocks of partial[b][j] (block order); loss likewise.
__global__ void k_reduce_partials(const float *__restrict__ partial, int64_t nblocks,
                                  float *__restrict__ grad, double *__restrict__ loss) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > kNP) return;
  double s = 0.0;
  for (int64_t b = 0; b < nblocks; ++b) s += (double)partial[b * (kNP + 1) + j];
  if (j < kNP) grad[j] = (float)s;
  else *loss = s;
}

__global__ void k_adam(float *__restrict__ th, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float c1, float c2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kNP) return;
  const float gj = g[j];
  const float mj = 0.9f * m[j] + 0.1f * gj;
  const float vj = 0.999f * v[j] + 0.001f * gj * gj;
  m[j] = mj;
  v[j] = vj;
  th[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + 1e-8f);
}

}  // namespace air

struct air_mlp {
  cudaStream_t stream = nullptr;
  float *th = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *partial = nullptr;
  uint32_t *w = nullptr;
  double *d_loss = nullptr, *h_loss = nullptr;
  size_t partial_b = 0;
  int64_t step = 0;
};

namespace air {

#define CU_TRY(x)                                    \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

static air_status mlp_pack(air_mlp *m) {
  k_pack_weights<<<16, 256, 0, m->stream>>>(m->th, m->w);
  CU_TRY(cudaGetLastError());
  return AIR_OK;
}

air_status mlp_forward(air_mlp *m, const uint16_t *x, int64_t n, float *logits, cudaStream_t st) {
  if (n <= 0) return AIR_OK;
  MlpArgs a{};
  a.x = reinterpret_cast<const uint32_t *>(x);
  a.n = n;
  a.w = m->w;
  a.th = m->th;
  a.logits = logits;
  const int64_t blocks = (n + kTile - 1) / kTile;
  k_mlp<false><<<(unsigned)blocks, kTile, kSmW, st>>>(a);
  CU_TRY(cudaGetLastError());
  return AIR_OK;
}

// Mean cross-entropy gradient over x[0..n) into m->grad (device), loss to m->d_loss.
static air_status mlp_grad(air_mlp *m, const uint16_t *x, const int32_t *y, int64_t n) {
  const int64_t blocks = (n + kTile - 1) / kTile;
  CU_TRY(ensure((void **)&m->partial, &m->partial_b, sizeof(float) * (size_t)blocks * (kNP + 1)));
  MlpArgs a{};
  a.x = reinterpret_cast<const uint32_t *>(x);
  a.y = y;
  a.n = n;
  a.inv_count = 1.0f / (float)n;
  a.w = m->w;
  a.th = m->th;
  a.partial = m->partial;
  static bool attr = false;
  if (!attr) {
    CU_TRY(cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmTrain));
    attr = true;
  }
  k_mlp<true><<<(unsigned)blocks, kTile, kSmTrain, m->stream>>>(a);
  CU_TRY(cudaGetLastError());
  k_reduce_partials<<<(kNP + 1 + 255) / 256, 256, 0, m->stream>>>(m->partial, blocks, m->grad, m->d_loss);
  CU_TRY(cudaGetLastError());
  return AIR_OK;
}

static air_status mlp_adam(air_mlp *m, float lr) {
  m->step += 1;
  const float c1 = 1.0f - powf(0.9f, (float)m->step), c2 = 1.0f - powf(0.999f, (float)m->step);
  k_adam<<<(kNP + 255) / 256, 256, 0, m->stream>>>(m->th, m->m, m->v, m->grad, lr, c1, c2);
  CU_TRY(cudaGetLastError());
  return mlp_pack(m);
}

}  // namespace air

extern "C" {

air_status air_mlp_create(const float *params, void *stream, air_mlp **out) {
  using namespace air;
  set_error(AIR_OK, "");
  if (!out) return set_error(AIR_ERR_ARG, "out is NULL");
  *out = nullptr;
  air_mlp *m = new (std::nothrow) air_mlp();
  if (!m) return set_error(AIR_ERR_OOM, "host allocation failed");
  m->stream = (cudaStream_t)stream;
  cudaError_t e = cudaMalloc((void **)&m->th, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMalloc((void **)&m->m, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMalloc((void **)&m->v, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMalloc((void **)&m->grad, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMalloc((void **)&m->w, sizeof(uint32_t) * kWords);
  if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&m->h_loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->th, 0, sizeof(float) * kNP, m->stream);
  if (e == cudaSuccess && params)
    e = cudaMemcpyAsync(m->th, params, sizeof(float) * kNP, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * kNP, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * kNP, m->stream);
  if (e != cudaSuccess) {
    air_mlp_free(m);
    return cuda_fail(e, "air_mlp_create");
  }
  air_status s = mlp_pack(m);
  if (s) {
    air_mlp_free(m);
    return s;
  }
  e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    air_mlp_free(m);
    return cuda_fail(e, "air_mlp_create");
  }
  *out = m;
  return AIR_OK;
}

air_status air_mlp_set_stream(air_mlp *m, void *stream) {
  air::set_error(AIR_OK, "");
  if (!m) return air::set_error(AIR_ERR_ARG, "mlp is NULL");
  m->stream = (cudaStream_t)stream;
  return AIR_OK;
}

air_status air_mlp_params(air_mlp *m, float *get, const float *set) {
  using namespace air;
  set_error(AIR_OK, "");
  if (!m) return set_error(AIR_ERR_ARG, "mlp is NULL");
  if (set) {
    CU_TRY(cudaMemcpyAsync(m->th, set, sizeof(float) * kNP, cudaMemcpyHostToDevice, m->stream));
    CU_TRY(cudaMemsetAsync(m->m, 0, sizeof(float) * kNP, m->stream));
    CU_TRY(cudaMemsetAsync(m->v, 0, sizeof(float) * kNP, m->stream));
    m->step = 0;
    air_status s = mlp_pack(m);
    if (s) return s;
  }
  if (get) CU_TRY(cudaMemcpyAsync(get, m->th, sizeof(float) * kNP, cudaMemcpyDeviceToHost, m->stream));
  CU_TRY(cudaStreamSynchronize(m->stream));
  return AIR_OK;
}

air_status air_mlp_forward(air_mlp *m, const uint16_t *x, int64_t n, float *logits) {
  using namespace air;
  set_error(AIR_OK, "");
  if (!m || !x || !logits || n < 0) return set_error(AIR_ERR_ARG, "bad arguments");
  air_status s = mlp_forward(m, x, n, logits, m->stream);
  if (s) return s;
  CU_TRY(cudaStreamSynchronize(m->stream));
  return AIR_OK;
}

air_status air_mlp_loss_grad(air_mlp *m, const uint16_t *x, const int32_t *y, int64_t n,
                             float *grad, double *loss) {
  using namespace air;
  set_error(AIR_OK, "");
  if (!m || !x || !y || n < 1) return set_error(AIR_ERR_ARG, "bad arguments");
  air_status s = mlp_grad(m, x, y, n);
  if (s) return s;
  if (grad) CU_TRY(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kNP, cudaMemcpyDeviceToDevice, m->stream));
  CU_TRY(cudaMemcpyAsync(m->h_loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CU_TRY(cudaStreamSynchronize(m->stream));
  if (loss) *loss = *m->h_loss / (double)n;
  return AIR_OK;
}

air_status air_mlp_train(air_mlp *m, const uint16_t *x, const int32_t *y, int64_t n, int32_t batch,
                         int32_t epochs, float lr, double *loss_history) {
  using namespace air;
  set_error(AIR_OK, "");
  if (!m || !x || !y || n < 1 || batch < 1 || epochs < 0 || !(lr > 0.f))
    return set_error(AIR_ERR_ARG, "bad arguments");
  const int64_t nb = (n + batch - 1) / batch;
  // visit the minibatches of an epoch in a strided order that changes per epoch
  int64_t stride = 1;
  for (int64_t c = (int64_t)(nb * 0.618) | 1; c < 2 * nb + 3; c += 2) {
    int64_t a = c, b = nb;
    while (b) { const int64_t r = a % b; a = b; b = r; }
    if (a == 1) { stride = c % (nb > 0 ? nb : 1); if (stride == 0) stride = 1; break; }
  }
  for (int e = 0; e < epochs; ++e) {
    double ep = 0.0;
    for (int64_t q = 0; q < nb; ++q) {
      const int64_t bi = (q * stride + (int64_t)e * 7) % nb;
      const int64_t s0 = bi * batch, cnt = std::min<int64_t>(batch, n - s0);
      air_status s = mlp_grad(m, x + s0 * kIn, y + s0, cnt);
      if (s) return s;
      s = mlp_adam(m, lr);
      if (s) return s;
      if (loss_history) {
        CU_TRY(cudaMemcpyAsync(m->h_loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        CU_TRY(cudaStreamSynchronize(m->stream));
        ep += *m->h_loss;
      }
    }
    if (loss_history) loss_history[e] = ep / (double)n;
  }
  CU_TRY(cudaStreamSynchronize(m->stream));
  return AIR_OK;
}

void air_mlp_free(air_mlp *m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  else cudaDeviceSynchronize();
  cudaFree(m->th); cudaFree(m->m); cudaFree(m->v); cudaFree(m->grad); cudaFree(m->partial);
  cudaFree(m->w); cudaFree(m->d_loss);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  delete m;
}

}  // extern "C"
