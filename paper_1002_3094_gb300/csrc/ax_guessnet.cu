// Initial-guess network: a small convolutional encoder-decoder that maps
// (log kappa, q, f / s) on an H x W lattice to u0 / s, trained on solutions
// that the solver itself produced.  The paper has no such component; it is
// the learned warm start of the production form: the CG solve always starts
// from it only if it lowers the initial residual, and always iterates to the
// same tolerance.
//
// Layout: activations [B][C][H][W] (NCHW), BF16 between layers, FP32 for
// gradients and the final output.  Conv weights [3][3][Cin][Cout]
// ([dy+1][dx+1][ci][co], "same" cross-correlation with zero padding), FP32
// master copy + BF16 compute copy; FP32 accumulation everywhere.
//
// Architecture (levels H, H/2, H/4, H/8; channels c1..c4):
//   e1a e1b | pool | e2a e2b | pool | e3a e3b | pool | b1 b2 | up |
//   d3a(+skip e3b) d3b | up | d2a(+skip e2b) d2b | up | d1a(+skip e1b) d1b | head(1x1)
// Every 3x3 conv is followed by ReLU; the "+skip" layers add the encoder
// activation of the same level after their ReLU.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ax_common.cuh"

namespace ax {
namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float ld_as_float(const float *p) { return *p; }
__device__ __forceinline__ float ld_as_float(const bf16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st_from_float(float *p, float v) { *p = v; }

constexpr int kTile = 32;   // output tile edge (pixels)
constexpr int kCib = 8;     // input channels per smem stage
constexpr int kCob = 16;    // output channels per CTA

// ---------------------------------------------------------------------------
// 3x3 convolution, forward (also used for the backward-data pass with
// flipped, transposed weights).  256 threads; each owns a 2x2 pixel block and
// 16 output channels.  out = act(conv(in) + bias) (+ skip, into out2).
// ---------------------------------------------------------------------------
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(256) conv3x3_kernel(const TIn *__restrict__ in, const bf16 *__restrict__ w,
                                                      const float *__restrict__ bias, TOut *__restrict__ out,
                                                      const bf16 *__restrict__ skip, bf16 *__restrict__ out2,
                                                      int Cin, int Cout, int H, int W, int relu) {
  __shared__ float s_in[kCib][kTile + 2][kTile + 2];
  __shared__ float s_w[kCib][9][kCob];
  const int tiles_x = (W + kTile - 1) / kTile;
  const int tx0 = (blockIdx.x % tiles_x) * kTile, ty0 = (blockIdx.x / tiles_x) * kTile;
  const int co0 = blockIdx.y * kCob;
  const int b = blockIdx.z;
  const int t = threadIdx.x;
  const int px = (t % 16) * 2, py = (t / 16) * 2;  // 2x2 block inside the tile
  const size_t plane = (size_t)H * W;
  const TIn *inb = in + (size_t)b * Cin * plane;
  float acc[4][kCob];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int c = 0; c < kCob; ++c) acc[p][c] = 0.f;

  for (int ci0 = 0; ci0 < Cin; ci0 += kCib) {
    __syncthreads();
    for (int e = t; e < kCib * (kTile + 2) * (kTile + 2); e += 256) {
      const int ci = e / ((kTile + 2) * (kTile + 2));
      const int rem = e - ci * (kTile + 2) * (kTile + 2);
      const int yy = rem / (kTile + 2), xx = rem - yy * (kTile + 2);
      const int gy = ty0 + yy - 1, gx = tx0 + xx - 1;
      float v = 0.f;
      if (ci0 + ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W)
        v = ld_as_float(inb + (size_t)(ci0 + ci) * plane + (size_t)gy * W + gx);
      s_in[ci][yy][xx] = v;
    }
    for (int e = t; e < kCib * 9 * kCob; e += 256) {
      const int ci = e / (9 * kCob);
      const int rem = e - ci * 9 * kCob;
      const int tap = rem / kCob, c = rem - tap * kCob;
      float v = 0.f;
      if (ci0 + ci < Cin && co0 + c < Cout) v = __bfloat162float(w[((size_t)tap * Cin + ci0 + ci) * Cout + co0 + c]);
      s_w[ci][tap][c] = v;
    }
    __syncthreads();
    const int cmax = min(kCib, Cin - ci0);
    for (int ci = 0; ci < cmax; ++ci) {
      float nb[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) nb[r][c] = s_in[ci][py + r][px + c];
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
        for (int c = 0; c < kCob; ++c) {
          const float wv = s_w[ci][tap][c];
          acc[0][c] = fmaf(nb[dy][dx], wv, acc[0][c]);
          acc[1][c] = fmaf(nb[dy][dx + 1], wv, acc[1][c]);
          acc[2][c] = fmaf(nb[dy + 1][dx], wv, acc[2][c]);
          acc[3][c] = fmaf(nb[dy + 1][dx + 1], wv, acc[3][c]);
        }
      }
    }
  }
  // epilogue
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int y = ty0 + py + (p >> 1), x = tx0 + px + (p & 1);
    if (y >= H || x >= W) continue;
#pragma unroll
    for (int c = 0; c < kCob; ++c) {
      const int co = co0 + c;
      if (co >= Cout) continue;
      float v = acc[p][c] + (bias ? bias[co] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      const size_t o = ((size_t)b * Cout + co) * plane + (size_t)y * W + x;
      st_from_float(out + o, v);
      if (skip) out2[o] = __float2bfloat16(v + __bfloat162float(skip[o]));
    }
  }
}

// ---------------------------------------------------------------------------
// 3x3 convolution, forward, on the tensor cores: implicit GEMM with
// mma.sync m16n8k16 (BF16 inputs, FP32 accumulation).  A CTA computes a
// 16 x 8 pixel patch (8 warps, one patch row of 16 pixels each) for 32 output
// channels; K runs over the 9 taps x input channels in chunks of 16.
// Shared memory holds the haloed input patch as [pixel][16 channels] and the
// weights as [tap][32 out][16 in], so each (k, k+1) pair of a fragment is one
// 32-bit word.
// ---------------------------------------------------------------------------
constexpr int kPx = 16, kPy = 8, kCo = 32;

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename TIn>
__global__ void __launch_bounds__(256) conv3x3_mma_kernel(const TIn *__restrict__ in, const bf16 *__restrict__ w,
                                                          const float *__restrict__ bias, bf16 *__restrict__ out,
                                                          const bf16 *__restrict__ skip, bf16 *__restrict__ out2,
                                                          int Cin, int Cout, int H, int W, int relu) {
  __shared__ __align__(16) bf16 s_in[(kPy + 2) * (kPx + 2)][16];
  __shared__ __align__(16) bf16 s_w[9][kCo][16];
  const int tiles_x = (W + kPx - 1) / kPx;
  const int x0 = (blockIdx.x % tiles_x) * kPx, y0 = (blockIdx.x / tiles_x) * kPy;
  const int co0 = blockIdx.y * kCo;
  const int b = blockIdx.z;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int g = lane >> 2, tq = lane & 3;
  const size_t plane = (size_t)H * W;
  const TIn *inb = in + (size_t)b * Cin * plane;
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[n][c] = 0.f;
  const unsigned *sin32 = reinterpret_cast<const unsigned *>(&s_in[0][0]);
  const unsigned *sw32 = reinterpret_cast<const unsigned *>(&s_w[0][0][0]);
  for (int ci0 = 0; ci0 < Cin; ci0 += 16) {
    __syncthreads();
    for (int e = t; e < (kPy + 2) * (kPx + 2) * 16; e += 256) {
      const int ci = e / ((kPy + 2) * (kPx + 2));
      const int pix = e - ci * (kPy + 2) * (kPx + 2);
      const int yy = pix / (kPx + 2), xx = pix - yy * (kPx + 2);
      const int gy = y0 + yy - 1, gx = x0 + xx - 1;
      float v = 0.f;
      if (ci0 + ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W)
        v = ld_as_float(inb + (size_t)(ci0 + ci) * plane + (size_t)gy * W + gx);
      s_in[pix][ci] = __float2bfloat16(v);
    }
    for (int e = t; e < 9 * kCo * 16; e += 256) {
      const int tap = e / (kCo * 16);
      const int rem = e - tap * kCo * 16;
      const int c = rem / 16, ci = rem - c * 16;
      bf16 v = __float2bfloat16(0.f);
      if (ci0 + ci < Cin && co0 + c < Cout) v = w[((size_t)tap * Cin + ci0 + ci) * Cout + co0 + c];
      s_w[tap][c][ci] = v;
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap % 3;
      // A rows: pixels x = g and x = g + 8 of patch row `warp`, shifted by the tap
      const int p0 = (warp + dy) * (kPx + 2) + g + dx;
      const int p1 = p0 + 8;
      unsigned a[4];
      a[0] = sin32[p0 * 8 + tq];
      a[1] = sin32[p1 * 8 + tq];
      a[2] = sin32[p0 * 8 + tq + 4];
      a[3] = sin32[p1 * 8 + tq + 4];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        const int c = n * 8 + g;
        unsigned bb[2];
        bb[0] = sw32[(tap * kCo + c) * 8 + tq];
        bb[1] = sw32[(tap * kCo + c) * 8 + tq + 4];
        mma_bf16_16816(acc[n], a, bb);
      }
    }
  }
  // epilogue: acc[n][0..1] pixel x = g, channels n*8 + 2tq + {0,1}; acc[n][2..3] pixel x = g + 8
  const int y = y0 + warp;
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int x = x0 + g + ((c >> 1) ? 8 : 0);
      const int co = co0 + n * 8 + 2 * tq + (c & 1);
      if (y >= H || x >= W || co >= Cout) continue;
      float v = acc[n][c] + bias[co];
      if (relu) v = fmaxf(v, 0.f);
      const size_t o = ((size_t)b * Cout + co) * plane + (size_t)y * W + x;
      out[o] = __float2bfloat16(v);
      if (skip) out2[o] = __float2bfloat16(v + __bfloat162float(skip[o]));
    }
}

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3 conv over one 32x32 tile of one sample:
//   partial[tile][tap][ci][co] = sum_{pixels} in[ci][y+dy-1][x+dx-1] gz[co][y][x]
// 144 threads: (tap, ci) x 2 halves of the 16 output channels.
// ---------------------------------------------------------------------------
template <typename TIn>
__global__ void __launch_bounds__(144) conv3x3_wgrad_kernel(const TIn *__restrict__ in, const float *__restrict__ gz,
                                                            float *__restrict__ partial, int Cin, int Cout, int H,
                                                            int W) {
  extern __shared__ __align__(16) float smem[];
  float *s_in = smem;                                           // [kCib][34][34]
  float *s_g = smem + kCib * (kTile + 2) * (kTile + 2);         // [1024][kCob]
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  const int tile = blockIdx.x;
  const int tx0 = (tile % tiles_x) * kTile, ty0 = (tile / tiles_x) * kTile;
  const int ci0 = blockIdx.y * kCib;
  const int nco = (Cout + kCob - 1) / kCob;
  const int co0 = (blockIdx.z % nco) * kCob;
  const int b = blockIdx.z / nco;
  const int t = threadIdx.x;
  const size_t plane = (size_t)H * W;
  for (int e = t; e < kCib * (kTile + 2) * (kTile + 2); e += blockDim.x) {
    const int ci = e / ((kTile + 2) * (kTile + 2));
    const int rem = e - ci * (kTile + 2) * (kTile + 2);
    const int yy = rem / (kTile + 2), xx = rem - yy * (kTile + 2);
    const int gy = ty0 + yy - 1, gx = tx0 + xx - 1;
    float v = 0.f;
    if (ci0 + ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W)
      v = ld_as_float(in + ((size_t)b * Cin + ci0 + ci) * plane + (size_t)gy * W + gx);
    s_in[e] = v;
  }
  for (int e = t; e < kTile * kTile * kCob; e += blockDim.x) {
    const int pix = e / kCob, c = e - pix * kCob;
    const int y = ty0 + pix / kTile, x = tx0 + pix % kTile;
    float v = 0.f;
    if (co0 + c < Cout && y < H && x < W) v = gz[((size_t)b * Cout + co0 + c) * plane + (size_t)y * W + x];
    s_g[e] = v;
  }
  __syncthreads();
  const int half = t % 2, pair = t / 2;   // pair = tap * kCib + ci
  const int tap = pair / kCib, ci = pair % kCib;
  const int dy = tap / 3, dx = tap % 3;
  float acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.f;
  for (int pix = 0; pix < kTile * kTile; ++pix) {
    const int y = pix / kTile, x = pix % kTile;
    const float xv = s_in[(ci * (kTile + 2) + y + dy) * (kTile + 2) + x + dx];
    const float4 g0 = *reinterpret_cast<const float4 *>(s_g + pix * kCob + half * 8);
    const float4 g1 = *reinterpret_cast<const float4 *>(s_g + pix * kCob + half * 8 + 4);
    acc[0] = fmaf(xv, g0.x, acc[0]); acc[1] = fmaf(xv, g0.y, acc[1]);
    acc[2] = fmaf(xv, g0.z, acc[2]); acc[3] = fmaf(xv, g0.w, acc[3]);
    acc[4] = fmaf(xv, g1.x, acc[4]); acc[5] = fmaf(xv, g1.y, acc[5]);
    acc[6] = fmaf(xv, g1.z, acc[6]); acc[7] = fmaf(xv, g1.w, acc[7]);
  }
  const size_t slot = (size_t)b * tiles_x * tiles_y + tile;
  float *pp = partial + slot * 9 * Cin * Cout;
  if (ci0 + ci < Cin) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int co = co0 + half * 8 + c;
      if (co < Cout) pp[((size_t)tap * Cin + ci0 + ci) * Cout + co] = acc[c];
    }
  }
}

// out[i] = sum_s partial[s][i], fixed order (deterministic).
__global__ void sum_partials(const float *__restrict__ partial, int slots, size_t n, float *__restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < slots; ++k) s += partial[(size_t)k * n + i];
    out[i] = s;
  }
}

// Per-(sample, channel) sums of gz over the plane -> partial[b][c]; the bias
// gradient is then the sum over b.
__global__ void channel_sums(const float *__restrict__ g, int C, size_t plane, float *__restrict__ partial) {
  __shared__ double red[8];
  const int c = blockIdx.x, b = blockIdx.y;
  const float *p = g + ((size_t)b * C + c) * plane;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < plane; i += blockDim.x) s += p[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[(size_t)b * C + c] = (float)s;
}

// gz = g * (a > 0) (ReLU derivative from the stored activation)
__global__ void relu_mask(const float *__restrict__ g, const bf16 *__restrict__ a, float *__restrict__ gz, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    gz[i] = (__bfloat162float(a[i]) > 0.f) ? g[i] : 0.f;
}

// 2x2 average pooling (bf16 -> bf16); backward (float -> float) adds into dst
// when `accumulate` (the pooled tensor is also a skip source).
__global__ void pool2_fwd(const bf16 *__restrict__ x, bf16 *__restrict__ y, int BC, int H, int W) {
  const int h = H / 2, w = W / 2;
  const size_t n = (size_t)BC * h * w;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int xx = i % w, yy = (i / w) % h;
    const size_t bc = i / ((size_t)h * w);
    const bf16 *s = x + bc * H * W + (size_t)(2 * yy) * W + 2 * xx;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[1]) + __bfloat162float(s[W]) +
                    __bfloat162float(s[W + 1]);
    y[i] = __float2bfloat16(0.25f * v);
  }
}
__global__ void pool2_bwd(const float *__restrict__ gy, const float *__restrict__ gskip, float *__restrict__ gx,
                          int BC, int H, int W) {
  const size_t n = (size_t)BC * H * W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int xx = i % W, yy = (i / W) % H;
    const size_t bc = i / ((size_t)H * W);
    float v = 0.25f * gy[bc * (H / 2) * (W / 2) + (size_t)(yy / 2) * (W / 2) + xx / 2];
    if (gskip) v += gskip[i];
    gx[i] = v;
  }
}
// nearest 2x upsampling (bf16) and its adjoint (2x2 sums, float)
__global__ void up2_fwd(const bf16 *__restrict__ x, bf16 *__restrict__ y, int BC, int h, int w) {
  const int H = 2 * h, W = 2 * w;
  const size_t n = (size_t)BC * H * W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int xx = i % W, yy = (i / W) % H;
    const size_t bc = i / ((size_t)H * W);
    y[i] = x[bc * h * w + (size_t)(yy / 2) * w + xx / 2];
  }
}
__global__ void up2_bwd(const float *__restrict__ gy, float *__restrict__ gx, int BC, int h, int w) {
  const int W = 2 * w;
  const size_t n = (size_t)BC * h * w;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int xx = i % w, yy = (i / w) % h;
    const size_t bc = i / ((size_t)h * w);
    const float *s = gy + bc * 4 * h * w + (size_t)(2 * yy) * W + 2 * xx;
    gx[i] = s[0] + s[1] + s[W] + s[W + 1];
  }
}

// 1x1 head (Cin -> 1): y = sum_c w[c] a[c] + b
__global__ void head_fwd(const bf16 *__restrict__ a, const float *__restrict__ w, const float *__restrict__ bias,
                         float *__restrict__ y, int B, int C, size_t plane) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * plane;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / plane, p = i - b * plane;
    float s = bias[0];
    for (int c = 0; c < C; ++c) s = fmaf(w[c], __bfloat162float(a[(b * C + c) * plane + p]), s);
    y[i] = s;
  }
}
// head backward: ga[c] = w[c] gy; partial[b][c] = sum_p a[c] gy (per CTA-row)
__global__ void head_bwd_data(const float *__restrict__ gy, const float *__restrict__ w, float *__restrict__ ga, int B,
                              int C, size_t plane) {
  const size_t n = (size_t)B * C * plane;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i % plane, bc = i / plane;
    const int c = bc % C;
    const size_t b = bc / C;
    ga[i] = w[c] * gy[b * plane + p];
  }
}
__global__ void head_bwd_weight(const bf16 *__restrict__ a, const float *__restrict__ gy, float *__restrict__ partial,
                                int C, size_t plane) {
  __shared__ double red[8];
  const int c = blockIdx.x, b = blockIdx.y;
  double s = 0.0;
  for (size_t p = threadIdx.x; p < plane; p += blockDim.x)
    s += (double)__bfloat162float(a[((size_t)b * C + c) * plane + p]) * gy[(size_t)b * plane + p];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[(size_t)b * C + c] = (float)s;
}

// Loss over n = B H W lattice values, d = y - t:
//   loss = (1/n) [ sum d^2 + lam sum_{lattice edges (p, q)} (d_p - d_q)^2 ]
// (lam = 0: mean squared error; the edge term is a discrete H1 seminorm, which
// weighs an error the way the operator's energy norm does: smooth errors
// little, pixel-scale noise much).  gy_p = (2/n) [d_p + lam sum_q (d_p - d_q)]
// over the lattice neighbours q of p.  Per-block partial sums of the loss.
__global__ void loss_kernel(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ gy,
                            int B, int H, int W, float lam, double *__restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  const size_t n = (size_t)B * H * W;
  const float sc = 2.0f / (float)n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    float g = d;
    double e = (double)d * d;
    if (lam != 0.f) {
      const int x = (int)(i % W), yy = (int)((i / W) % H);
      float lap = 0.f;
      if (x > 0) lap += d - (y[i - 1] - t[i - 1]);
      if (yy > 0) lap += d - (y[i - W] - t[i - W]);
      if (x + 1 < W) {
        const float dr = d - (y[i + 1] - t[i + 1]);
        lap += dr;
        e += (double)lam * dr * dr;
      }
      if (yy + 1 < H) {
        const float dd = d - (y[i + W] - t[i + W]);
        lap += dd;
        e += (double)lam * dd * dd;
      }
      g = fmaf(lam, lap, d);
    }
    gy[i] = sc * g;
    s += e;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Weight transform for the backward-data pass: wt[8 - tap][co][ci] = w[tap][ci][co]
__global__ void flip_transpose(const bf16 *__restrict__ w, bf16 *__restrict__ wt, int Cin, int Cout) {
  const size_t n = (size_t)9 * Cin * Cout;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int co = i % Cout;
    const int ci = (i / Cout) % Cin;
    const int tap = i / ((size_t)Cin * Cout);
    wt[((size_t)(8 - tap) * Cout + co) * Cin + ci] = w[i];
  }
}

// Adam (FP32 master weights) and refresh of the BF16 compute copy.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, bf16 *__restrict__ pb, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    const float pi = p[i] - upd;
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
  }
}

__global__ void to_bf16(const float *__restrict__ x, bf16 *__restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// ---------------------------------------------------------------------------
// Features and lift (solver side)
// ---------------------------------------------------------------------------
// s[m] = max |f_m| (one CTA per right-hand side)
__global__ void maxabs_kernel(const double *__restrict__ f, size_t n, double *__restrict__ s) {
  __shared__ double red[256];
  const double *p = f + (size_t)blockIdx.x * n;
  double v = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) v = fmax(v, fabs(p[i]));
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) s[blockIdx.x] = red[0] > 0.0 ? red[0] : 1.0;
}

// x[m][0] = mean log kappa, x[m][1] = mean q, x[m][2] = mean f / s over the
// grid cells that fall into each lattice cell (area average when the grid is
// an integer multiple of the lattice, nearest sample otherwise).
__global__ void features_kernel(const double *__restrict__ kappa, const double *__restrict__ q,
                                const double *__restrict__ f, const double *__restrict__ s, int nr, int nz, int hw,
                                float *__restrict__ x) {
  const int m = blockIdx.y;
  const size_t plane = (size_t)hw * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const int py = i / hw, px = i % hw;   // py along r, px along z
    const int fr = (nr % hw == 0) ? nr / hw : 1, fz = (nz % hw == 0) ? nz / hw : 1;
    const int r0 = (nr % hw == 0) ? py * fr : (int)(((long long)py * nr) / hw);
    const int z0 = (nz % hw == 0) ? px * fz : (int)(((long long)px * nz) / hw);
    double lk = 0.0, qq = 0.0, ff = 0.0;
    for (int a = 0; a < fr; ++a)
      for (int c = 0; c < fz; ++c) {
        const size_t e = (size_t)(r0 + a) * nz + z0 + c;
        lk += log(kappa[e]);
        qq += q[e];
        ff += f[(size_t)m * nr * nz + e];
      }
    const double inv = 1.0 / (fr * fz);
    x[((size_t)m * 3 + 0) * plane + i] = (float)(lk * inv);
    x[((size_t)m * 3 + 1) * plane + i] = (float)(qq * inv);
    x[((size_t)m * 3 + 2) * plane + i] = (float)(ff * inv / s[m]);
  }
}

// u[m][i][k] = s[m] * bilinear(y[m], at the lattice position of grid node (i, k)),
// lattice values sitting at cell centres ((p + 1/2) / hw).
// s[i] /= t for i < m (the feature scale of a lift whose training targets were
// u / s times t)
__global__ void div_scale_kernel(double *s, int m, double t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) s[i] /= t;
}

__global__ void lift_kernel(const float *__restrict__ y, const double *__restrict__ s, int hw, int nr, int nz,
                            double *__restrict__ u) {
  const int m = blockIdx.y;
  const size_t n = (size_t)nr * nz;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = e / nz, k = e % nz;
    const float gy = ((i + 0.5f) * hw) / nr - 0.5f, gx = ((k + 0.5f) * hw) / nz - 0.5f;
    const int y0 = max(0, min(hw - 1, (int)floorf(gy))), x0 = max(0, min(hw - 1, (int)floorf(gx)));
    const int y1 = min(hw - 1, y0 + 1), x1 = min(hw - 1, x0 + 1);
    const float wy = fminf(fmaxf(gy - y0, 0.f), 1.f), wx = fminf(fmaxf(gx - x0, 0.f), 1.f);
    const float *p = y + (size_t)m * hw * hw;
    const float v = (1 - wy) * ((1 - wx) * p[y0 * hw + x0] + wx * p[y0 * hw + x1]) +
                    wy * ((1 - wx) * p[y1 * hw + x0] + wx * p[y1 * hw + x1]);
    u[(size_t)m * n + e] = s[m] * (double)v;
  }
}

int grid1d(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

// ---------------------------------------------------------------------------
// Network object
// ---------------------------------------------------------------------------
struct NetLayer {
  char kind;     // 'c' conv+relu, 's' conv+relu+skip, 'p' pool, 'u' up, 'h' head
  int cin = 0, cout = 0, res = 0;  // res: spatial size of this layer's output
  size_t woff = 0, boff = 0;       // offsets into the flat parameter vector
  int out = -1, out2 = -1;         // activation buffers (out2: relu output + skip)
  int skip = -1;                   // buffer added after ReLU ('s')
};

struct GuessNet {
  int hw = 0, cap = 0;   // lattice size, batch capacity
  int ch[4] = {24, 48, 96, 192};
  std::vector<NetLayer> layers;
  size_t nparams = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grads, Adam moments
  bf16 *pb = nullptr;                                            // BF16 compute copy
  bf16 *wt = nullptr;                                            // flipped/transposed weights scratch
  std::vector<std::pair<int, int>> bufshape;                     // (channels, res) per activation buffer
  std::vector<bf16 *> act;                                       // activations [cap][C][res][res]
  float *y = nullptr;                                            // head output [cap][hw][hw]
  float *gA = nullptr, *gB = nullptr, *gZ = nullptr;             // gradient scratch (largest activation)
  std::vector<float *> gskip;                                    // skip gradients per level
  float *partial = nullptr;                                      // weight-gradient partials
  size_t partial_n = 0;
  double *lpart = nullptr;                                       // loss partials
  float h1 = 0.f;                                                // weight of the loss's edge term
  int step = 0;
};

size_t act_elems(const GuessNet *n, int buf) {
  return (size_t)n->cap * n->bufshape[buf].first * n->bufshape[buf].second * n->bufshape[buf].second;
}

void build_layers(GuessNet *n) {
  const int c1 = n->ch[0], c2 = n->ch[1], c3 = n->ch[2], c4 = n->ch[3];
  const int H = n->hw;
  auto buf = [&](int c, int r) {
    n->bufshape.push_back({c, r});
    return (int)n->bufshape.size() - 1;
  };
  size_t off = 0;
  auto conv = [&](char kind, int cin, int cout, int res, int skip) {
    NetLayer L;
    L.kind = kind;
    L.cin = cin;
    L.cout = cout;
    L.res = res;
    L.woff = off;
    off += (size_t)9 * cin * cout;
    L.boff = off;
    off += cout;
    L.out = buf(cout, res);
    if (kind == 's') {
      L.out2 = buf(cout, res);
      L.skip = skip;
    }
    n->layers.push_back(L);
    return (kind == 's') ? L.out2 : L.out;
  };
  auto pool = [&](int c, int res) {
    NetLayer L;
    L.kind = 'p';
    L.cin = L.cout = c;
    L.res = res;
    L.out = buf(c, res);
    n->layers.push_back(L);
    return L.out;
  };
  auto up = [&](int c, int res) {
    NetLayer L;
    L.kind = 'u';
    L.cin = L.cout = c;
    L.res = res;
    L.out = buf(c, res);
    n->layers.push_back(L);
    return L.out;
  };
  conv('c', 3, c1, H, -1);
  const int s1 = conv('c', c1, c1, H, -1);
  pool(c1, H / 2);
  conv('c', c1, c2, H / 2, -1);
  const int s2 = conv('c', c2, c2, H / 2, -1);
  pool(c2, H / 4);
  conv('c', c2, c3, H / 4, -1);
  const int s3 = conv('c', c3, c3, H / 4, -1);
  pool(c3, H / 8);
  conv('c', c3, c4, H / 8, -1);
  conv('c', c4, c4, H / 8, -1);
  up(c4, H / 4);
  conv('s', c4, c3, H / 4, s3);
  conv('c', c3, c3, H / 4, -1);
  up(c3, H / 2);
  conv('s', c3, c2, H / 2, s2);
  conv('c', c2, c2, H / 2, -1);
  up(c2, H);
  conv('s', c2, c1, H, s1);
  conv('c', c1, c1, H, -1);
  NetLayer hd;
  hd.kind = 'h';
  hd.cin = c1;
  hd.cout = 1;
  hd.res = H;
  hd.woff = off;
  off += c1;
  hd.boff = off;
  off += 1;
  n->layers.push_back(hd);
  n->nparams = off;
}

// deterministic host initialisation: He-normal weights (Box-Muller on a
// splitmix64 stream), zero biases
uint64_t splitmix64(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t &st) { return ((splitmix64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

void init_host_params(const GuessNet *n, uint64_t seed, std::vector<float> &h) {
  h.assign(n->nparams, 0.f);
  uint64_t st = seed;
  for (const NetLayer &L : n->layers) {
    if (L.kind == 'p' || L.kind == 'u') continue;
    const size_t nw = (L.kind == 'h') ? (size_t)L.cin : (size_t)9 * L.cin * L.cout;
    const double fan_in = (L.kind == 'h') ? L.cin : 9.0 * L.cin;
    const double sd = (L.kind == 'h') ? std::sqrt(1.0 / fan_in) : std::sqrt(2.0 / fan_in);
    for (size_t i = 0; i < nw; ++i) {
      const double u1 = uniform01(st), u2 = uniform01(st);
      h[L.woff + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
    }
  }
}

template <typename P>
cudaError_t zalloc(P **p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(P));
  // the fill runs on the legacy stream: finish it before any launch on a
  // non-blocking stream can touch the buffer
  if (e == cudaSuccess) e = cudaMemset(*p, 0, count * sizeof(P));
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  return e;
}

void net_free(GuessNet *n) {
  cudaFree(n->p); cudaFree(n->g); cudaFree(n->m); cudaFree(n->v); cudaFree(n->pb); cudaFree(n->wt);
  for (auto *a : n->act) cudaFree(a);
  for (auto *a : n->gskip) cudaFree(a);
  cudaFree(n->y); cudaFree(n->gA); cudaFree(n->gB); cudaFree(n->gZ); cudaFree(n->partial); cudaFree(n->lpart);
  delete n;
}

// ---------------------------------------------------------------------------
// passes
// ---------------------------------------------------------------------------
template <typename TIn, typename TOut>
void launch_conv(const TIn *in, const bf16 *w, const float *bias, TOut *out, const bf16 *skip, bf16 *out2, int B,
                 int Cin, int Cout, int res, bool relu, cudaStream_t s) {
  const int tiles = ((res + kTile - 1) / kTile) * ((res + kTile - 1) / kTile);
  dim3 grid(tiles, (Cout + kCob - 1) / kCob, B);
  note_launch();
  conv3x3_kernel<TIn, TOut><<<grid, 256, 0, s>>>(in, w, bias, out, skip, out2, Cin, Cout, res, res, relu ? 1 : 0);
}

template <typename TIn>
void launch_conv_mma(const TIn *in, const bf16 *w, const float *bias, bf16 *out, const bf16 *skip, bf16 *out2, int B,
                     int Cin, int Cout, int res, cudaStream_t s) {
  const int tiles = ((res + kPx - 1) / kPx) * ((res + kPy - 1) / kPy);
  dim3 grid(tiles, (Cout + kCo - 1) / kCo, B);
  note_launch();
  conv3x3_mma_kernel<TIn><<<grid, 256, 0, s>>>(in, w, bias, out, skip, out2, Cin, Cout, res, res, 1);
}

template <typename TIn>
void launch_wgrad(GuessNet *n, const TIn *in, const float *gz, float *gw, int B, int Cin, int Cout, int res,
                  cudaStream_t s) {
  const int tiles = ((res + kTile - 1) / kTile) * ((res + kTile - 1) / kTile);
  const int nco = (Cout + kCob - 1) / kCob;
  const size_t smem = sizeof(float) * (kCib * (kTile + 2) * (kTile + 2) + kTile * kTile * kCob);
  ensure_smem_attr((const void *)conv3x3_wgrad_kernel<TIn>, smem);
  dim3 grid(tiles, (Cin + kCib - 1) / kCib, nco * B);
  note_launch();
  conv3x3_wgrad_kernel<TIn><<<grid, 144, smem, s>>>(in, gz, n->partial, Cin, Cout, res, res);
  const size_t nw = (size_t)9 * Cin * Cout;
  note_launch();
  sum_partials<<<grid1d(nw), 256, 0, s>>>(n->partial, B * tiles, nw, gw);
}

void bias_grad(GuessNet *n, const float *gz, float *gb, int B, int C, int res, cudaStream_t s) {
  note_launch();
  channel_sums<<<dim3(C, B), 256, 0, s>>>(gz, C, (size_t)res * res, n->partial);
  note_launch();
  sum_partials<<<grid1d(C), 256, 0, s>>>(n->partial, B, (size_t)C, gb);
}

void forward_pass(GuessNet *n, const float *x, int B, cudaStream_t s) {
  const int H = n->hw;
  int cur = -1;  // current activation buffer (-1: the FP32 input x)
  for (const NetLayer &L : n->layers) {
    if (L.kind == 'c' || L.kind == 's') {
      const bf16 *w = n->pb + L.woff;
      const float *bias = n->p + L.boff;
      bf16 *out = n->act[L.out];
      const bf16 *skip = (L.kind == 's') ? n->act[L.skip] : nullptr;
      bf16 *out2 = (L.kind == 's') ? n->act[L.out2] : nullptr;
      if (cur < 0)
        launch_conv_mma<float>(x, w, bias, out, skip, out2, B, L.cin, L.cout, L.res, s);
      else
        launch_conv_mma<bf16>(n->act[cur], w, bias, out, skip, out2, B, L.cin, L.cout, L.res, s);
      cur = (L.kind == 's') ? L.out2 : L.out;
    } else if (L.kind == 'p') {
      note_launch();
      pool2_fwd<<<grid1d((size_t)B * L.cout * L.res * L.res), 256, 0, s>>>(n->act[cur], n->act[L.out], B * L.cout,
                                                                           2 * L.res, 2 * L.res);
      cur = L.out;
    } else if (L.kind == 'u') {
      note_launch();
      up2_fwd<<<grid1d((size_t)B * L.cout * L.res * L.res), 256, 0, s>>>(n->act[cur], n->act[L.out], B * L.cout,
                                                                         L.res / 2, L.res / 2);
      cur = L.out;
    } else {
      note_launch();
      head_fwd<<<grid1d((size_t)B * H * H), 256, 0, s>>>(n->act[cur], n->p + L.woff, n->p + L.boff, n->y, B, L.cin,
                                                         (size_t)H * H);
    }
  }
}

// input buffer of layer li during the forward pass (-1 = x)
int layer_input(const GuessNet *n, int li) {
  int cur = -1;
  for (int k = 0; k < li; ++k) {
    const NetLayer &L = n->layers[k];
    if (L.kind == 'h') continue;
    cur = (L.kind == 's') ? L.out2 : L.out;
  }
  return cur;
}

// Backward pass from gy (d loss / d y, FP32 [B][H][W]); fills n->g.
void backward_pass(GuessNet *n, const float *x, const float *gy, int B, cudaStream_t s) {
  const int H = n->hw;
  float *g = n->gA, *gnext = n->gB;
  int level_skip = 0;  // skip gradients pushed (level 1 first)
  std::vector<float *> skip_stack;
  for (int li = (int)n->layers.size() - 1; li >= 0; --li) {
    const NetLayer &L = n->layers[li];
    const int inbuf = layer_input(n, li);
    if (L.kind == 'h') {
      note_launch();
      head_bwd_weight<<<dim3(L.cin, B), 256, 0, s>>>(n->act[inbuf], gy, n->partial, L.cin, (size_t)H * H);
      note_launch();
      sum_partials<<<grid1d(L.cin), 256, 0, s>>>(n->partial, B, (size_t)L.cin, n->g + L.woff);
      // bias gradient: sum of gy over all samples and pixels
      note_launch();
      channel_sums<<<dim3(1, B), 256, 0, s>>>(gy, 1, (size_t)H * H, n->partial);
      note_launch();
      sum_partials<<<1, 256, 0, s>>>(n->partial, B, 1, n->g + L.boff);
      note_launch();
      head_bwd_data<<<grid1d((size_t)B * L.cin * H * H), 256, 0, s>>>(gy, n->p + L.woff, g, B, L.cin, (size_t)H * H);
    } else if (L.kind == 'c' || L.kind == 's') {
      const size_t ne = (size_t)B * L.cout * L.res * L.res;
      if (L.kind == 's') {
        // the skip source receives the incoming gradient unchanged
        float *sg = n->gskip[level_skip++];
        cudaMemcpyAsync(sg, g, ne * sizeof(float), cudaMemcpyDeviceToDevice, s);
        skip_stack.push_back(sg);
      }
      note_launch();
      relu_mask<<<grid1d(ne), 256, 0, s>>>(g, n->act[L.out], n->gZ, ne);
      if (inbuf < 0)
        launch_wgrad<float>(n, x, n->gZ, n->g + L.woff, B, L.cin, L.cout, L.res, s);
      else
        launch_wgrad<bf16>(n, n->act[inbuf], n->gZ, n->g + L.woff, B, L.cin, L.cout, L.res, s);
      bias_grad(n, n->gZ, n->g + L.boff, B, L.cout, L.res, s);
      if (li > 0) {
        note_launch();
        flip_transpose<<<grid1d((size_t)9 * L.cin * L.cout), 256, 0, s>>>(n->pb + L.woff, n->wt, L.cin, L.cout);
        launch_conv<float, float>(n->gZ, n->wt, nullptr, gnext, nullptr, nullptr, B, L.cout, L.cin, L.res, false, s);
        std::swap(g, gnext);
      }
    } else if (L.kind == 'u') {
      note_launch();
      up2_bwd<<<grid1d((size_t)B * L.cin * (L.res / 2) * (L.res / 2)), 256, 0, s>>>(g, gnext, B * L.cin, L.res / 2,
                                                                                      L.res / 2);
      std::swap(g, gnext);
    } else {  // pool: gradient of the pooled input plus its skip gradient
      float *sg = skip_stack.back();
      skip_stack.pop_back();
      note_launch();
      pool2_bwd<<<grid1d((size_t)B * L.cin * 4 * L.res * L.res), 256, 0, s>>>(g, sg, gnext, B * L.cin, 2 * L.res,
                                                                                2 * L.res);
      std::swap(g, gnext);
    }
  }
}

int loss_and_grad(GuessNet *n, const float *target, int B, cudaStream_t s, double *loss) {
  const size_t N = (size_t)B * n->hw * n->hw;
  const int blocks = std::min<int>(grid1d(N), 1024);
  note_launch();
  loss_kernel<<<blocks, 256, 0, s>>>(n->y, target, n->gZ, B, n->hw, n->hw, n->h1, n->lpart);
  std::vector<double> h(blocks);
  if (cudaMemcpyAsync(h.data(), n->lpart, blocks * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return AX_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return AX_ERR_CUDA;
  double sum = 0.0;
  for (double v : h) sum += v;
  if (loss) *loss = sum / N;
  return AX_OK;
}

}  // namespace
}  // namespace ax

using namespace ax;

extern "C" {

int ax_guessnet_create(int32_t hw, const int32_t *channels, int32_t batch_capacity, uint64_t seed, void **out) {
  if (!out) return AX_ERR_INVALID_ARG;
  *out = nullptr;
  if (hw < 8 || hw % 8 != 0 || hw > 4096 || batch_capacity < 1) return AX_ERR_INVALID_ARG;
  GuessNet *n = new GuessNet();
  n->hw = hw;
  n->cap = batch_capacity;
  if (channels)
    for (int i = 0; i < 4; ++i) {
      if (channels[i] < 1 || channels[i] > 1024) {
        delete n;
        return AX_ERR_INVALID_ARG;
      }
      n->ch[i] = channels[i];
    }
  build_layers(n);
  std::vector<float> h;
  init_host_params(n, seed, h);
  cudaError_t e = zalloc(&n->p, n->nparams);
  if (e == cudaSuccess) e = zalloc(&n->g, n->nparams);
  if (e == cudaSuccess) e = zalloc(&n->m, n->nparams);
  if (e == cudaSuccess) e = zalloc(&n->v, n->nparams);
  if (e == cudaSuccess) e = zalloc(&n->pb, n->nparams);
  size_t maxw = 0, maxact = 0;
  for (const NetLayer &L : n->layers) maxw = std::max(maxw, (size_t)9 * L.cin * L.cout);
  if (e == cudaSuccess) e = zalloc(&n->wt, maxw);
  for (size_t b = 0; b < n->bufshape.size() && e == cudaSuccess; ++b) {
    bf16 *a = nullptr;
    e = zalloc(&a, act_elems(n, (int)b));
    n->act.push_back(a);
    maxact = std::max(maxact, act_elems(n, (int)b));
  }
  maxact = std::max(maxact, (size_t)n->cap * 3 * hw * hw);
  if (e == cudaSuccess) e = zalloc(&n->y, (size_t)n->cap * hw * hw);
  if (e == cudaSuccess) e = zalloc(&n->gA, maxact);
  if (e == cudaSuccess) e = zalloc(&n->gB, maxact);
  if (e == cudaSuccess) e = zalloc(&n->gZ, maxact);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    float *sg = nullptr;
    e = zalloc(&sg, maxact);
    n->gskip.push_back(sg);
  }
  // weight-gradient partials: slots (B * tiles) x (9 Cin Cout), largest layer
  size_t pn = 0;
  for (const NetLayer &L : n->layers) {
    const size_t tiles = (size_t)((L.res + kTile - 1) / kTile) * ((L.res + kTile - 1) / kTile);
    pn = std::max(pn, (size_t)n->cap * tiles * 9 * std::max(L.cin, 1) * std::max(L.cout, 1));
    pn = std::max(pn, (size_t)n->cap * std::max(L.cout, L.cin));
  }
  n->partial_n = pn;
  if (e == cudaSuccess) e = zalloc(&n->partial, pn);
  if (e == cudaSuccess) e = zalloc(&n->lpart, 1024);
  if (e == cudaSuccess) e = cudaMemcpy(n->p, h.data(), n->nparams * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    to_bf16<<<grid1d(n->nparams), 256>>>(n->p, n->pb, n->nparams);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    net_free(n);
    return e == cudaErrorMemoryAllocation ? AX_ERR_OOM : AX_ERR_CUDA;
  }
  *out = n;
  return AX_OK;
}

int ax_guessnet_destroy(void *net) {
  if (net) net_free((GuessNet *)net);
  return AX_OK;
}

int64_t ax_guessnet_num_params(void *net) { return net ? (int64_t)((GuessNet *)net)->nparams : 0; }

int ax_guessnet_get_params(void *net, float *host, int64_t n) {
  GuessNet *g = (GuessNet *)net;
  if (!g || !host || n != (int64_t)g->nparams) return AX_ERR_INVALID_ARG;
  return cudaMemcpy(host, g->p, n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

int ax_guessnet_set_params(void *net, const float *host, int64_t n) {
  GuessNet *g = (GuessNet *)net;
  if (!g || !host || n != (int64_t)g->nparams) return AX_ERR_INVALID_ARG;
  if (cudaMemcpy(g->p, host, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return AX_ERR_CUDA;
  note_launch();
  to_bf16<<<grid1d(g->nparams), 256>>>(g->p, g->pb, g->nparams);
  cudaMemset(g->m, 0, n * sizeof(float));
  cudaMemset(g->v, 0, n * sizeof(float));
  g->step = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

int ax_guessnet_forward(void *net, const float *x, float *y, int32_t batch, void *stream) {
  GuessNet *n = (GuessNet *)net;
  if (!n || !x || !y || batch < 1 || batch > n->cap) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  forward_pass(n, x, batch, s);
  cudaMemcpyAsync(y, n->y, (size_t)batch * n->hw * n->hw * sizeof(float), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError() == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

int ax_guessnet_set_loss(void *net, double h1_weight) {
  GuessNet *g = (GuessNet *)net;
  if (!g || !(h1_weight >= 0.0) || h1_weight > 1e6) return AX_ERR_INVALID_ARG;
  g->h1 = (float)h1_weight;
  return AX_OK;
}

int ax_guessnet_gradients(void *net, const float *x, const float *target, int32_t batch, float *grad_host,
                          double *loss, void *stream) {
  GuessNet *n = (GuessNet *)net;
  if (!n || !x || !target || batch < 1 || batch > n->cap) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  forward_pass(n, x, batch, s);
  int rc = loss_and_grad(n, target, batch, s, loss);
  if (rc != AX_OK) return rc;
  // loss_and_grad left d loss / d y in gZ, which the backward pass reuses as
  // scratch; move it into the output buffer (no longer needed)
  float *gyc = n->y;
  cudaMemcpyAsync(gyc, n->gZ, (size_t)batch * n->hw * n->hw * sizeof(float), cudaMemcpyDeviceToDevice, s);
  backward_pass(n, x, gyc, batch, s);
  if (grad_host) {
    if (cudaMemcpyAsync(grad_host, n->g, n->nparams * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return AX_ERR_CUDA;
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

int ax_guessnet_train_step(void *net, const float *x, const float *target, int32_t batch, float lr, double *loss,
                           void *stream) {
  GuessNet *n = (GuessNet *)net;
  if (!n || !(lr > 0.f)) return AX_ERR_INVALID_ARG;
  int rc = ax_guessnet_gradients(net, x, target, batch, nullptr, loss, stream);
  if (rc != AX_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
  note_launch();
  adam_kernel<<<grid1d(n->nparams), 256, 0, s>>>(n->p, n->g, n->m, n->v, n->pb, n->nparams, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError() == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

int ax_guessnet_save(void *net, const char *path) {
  GuessNet *n = (GuessNet *)net;
  if (!n || !path) return AX_ERR_INVALID_ARG;
  std::vector<float> h(n->nparams);
  if (cudaMemcpy(h.data(), n->p, h.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return AX_ERR_CUDA;
  FILE *fp = fopen(path, "wb");
  if (!fp) return AX_ERR_INVALID_ARG;
  // header: magic, version, hw, channels[4], nparams; then FP32 little-endian
  // parameters and a 64-bit FNV-1a checksum of their bytes
  const int32_t hdr[8] = {0x4e475841 /* "AXGN" */, 1, n->hw, n->ch[0], n->ch[1], n->ch[2], n->ch[3],
                          (int32_t)n->nparams};
  uint64_t sum = 1469598103934665603ull;
  const unsigned char *bytes = reinterpret_cast<const unsigned char *>(h.data());
  for (size_t i = 0; i < h.size() * sizeof(float); ++i) sum = (sum ^ bytes[i]) * 1099511628211ull;
  const bool ok = fwrite(hdr, sizeof(hdr), 1, fp) == 1 && fwrite(h.data(), sizeof(float), h.size(), fp) == h.size() &&
                  fwrite(&sum, sizeof(sum), 1, fp) == 1;
  fclose(fp);
  return ok ? AX_OK : AX_ERR_INVALID_ARG;
}

int ax_guessnet_load(void *net, const char *path) {
  GuessNet *n = (GuessNet *)net;
  if (!n || !path) return AX_ERR_INVALID_ARG;
  FILE *fp = fopen(path, "rb");
  if (!fp) return AX_ERR_INVALID_ARG;
  int32_t hdr[8];
  std::vector<float> h(n->nparams);
  uint64_t sum = 0;
  bool ok = fread(hdr, sizeof(hdr), 1, fp) == 1 && hdr[0] == 0x4e475841 && hdr[1] == 1 && hdr[2] == n->hw &&
            hdr[3] == n->ch[0] && hdr[4] == n->ch[1] && hdr[5] == n->ch[2] && hdr[6] == n->ch[3] &&
            hdr[7] == (int32_t)n->nparams && fread(h.data(), sizeof(float), h.size(), fp) == h.size() &&
            fread(&sum, sizeof(sum), 1, fp) == 1;
  fclose(fp);
  if (!ok) return AX_ERR_INVALID_ARG;
  uint64_t chk = 1469598103934665603ull;
  const unsigned char *bytes = reinterpret_cast<const unsigned char *>(h.data());
  for (size_t i = 0; i < h.size() * sizeof(float); ++i) chk = (chk ^ bytes[i]) * 1099511628211ull;
  if (chk != sum) return AX_ERR_INVALID_ARG;
  return ax_guessnet_set_params(net, h.data(), (int64_t)h.size());
}

int ax_guessnet_features(const double *kappa, const double *q, const double *f, int32_t m, int32_t nr, int32_t nz,
                         int32_t hw, float *x, double *scale, void *stream) {
  if (!kappa || !q || !f || !x || !scale || m < 1 || nr < 1 || nz < 1 || hw < 1) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  note_launch();
  maxabs_kernel<<<m, 256, 0, s>>>(f, (size_t)nr * nz, scale);
  note_launch();
  features_kernel<<<dim3(grid1d((size_t)hw * hw), m), 256, 0, s>>>(kappa, q, f, scale, nr, nz, hw, x);
  return cudaGetLastError() == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

int ax_guessnet_lift(const float *y, int32_t m, int32_t hw, const double *scale, int32_t nr, int32_t nz, double *u,
                     void *stream) {
  if (!y || !scale || !u || m < 1 || nr < 1 || nz < 1 || hw < 1) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  note_launch();
  lift_kernel<<<dim3(grid1d((size_t)nr * nz), m), 256, 0, s>>>(y, scale, hw, nr, nz, u);
  return cudaGetLastError() == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

int ax_solve_learned(ax_operator *op, void *net, const double *kappa, const double *q, const double *f, double *u,
                     int32_t m, double tol, int32_t max_iter, int32_t method, int32_t flags, int32_t pre,
                     double target_scale, ax_solve_info *info, void *stream) {
  GuessNet *n = (GuessNet *)net;
  if (!op || !n || !kappa || !q || !f || !u || m < 1 || !(target_scale > 0.0) || !std::isfinite(target_scale))
    return AX_ERR_INVALID_ARG;
  if (flags & AX_FLAG_HOST_BUFFERS) return AX_ERR_UNSUPPORTED;
  const int32_t nr = op->nr, nz = op->nz;
  cudaStream_t s = (cudaStream_t)stream;
  const int hw = n->hw;
  float *x = nullptr, *y = nullptr;
  double *sc = nullptr;
  struct Free {
    float *x, *y;
    double *sc;
    ~Free() {
      if (x) cudaFree(x);
      if (y) cudaFree(y);
      if (sc) cudaFree(sc);
    }
  } hold{nullptr, nullptr, nullptr};
  if (cudaMalloc(&x, (size_t)m * 3 * hw * hw * sizeof(float)) != cudaSuccess) return AX_ERR_OOM;
  hold.x = x;
  if (cudaMalloc(&y, (size_t)m * hw * hw * sizeof(float)) != cudaSuccess) return AX_ERR_OOM;
  hold.y = y;
  if (cudaMalloc(&sc, (size_t)m * sizeof(double)) != cudaSuccess) return AX_ERR_OOM;
  hold.sc = sc;
  int rc = pre ? ax_guessnet_features_pre(op, kappa, q, f, m, hw, x, sc, stream)
               : ax_guessnet_features(kappa, q, f, m, nr, nz, hw, x, sc, stream);
  if (rc != AX_OK) return rc;
  for (int c = 0; c < m; c += n->cap) {  // the network's batches
    const int b = std::min(n->cap, m - c);
    if ((rc = ax_guessnet_forward(net, x + (size_t)c * 3 * hw * hw, y + (size_t)c * hw * hw, b, stream)) != AX_OK)
      return rc;
  }
  if (target_scale != 1.0) {
    note_launch();
    div_scale_kernel<<<(m + 255) / 256, 256, 0, s>>>(sc, m, target_scale);
  }
  if ((rc = ax_guessnet_lift(y, m, hw, sc, nr, nz, u, stream)) != AX_OK) return rc;
  return ax_solve(op, f, u, m, tol, max_iter, method, flags | AX_FLAG_USE_GUESS | AX_FLAG_CHECK_GUESS, info,
                  stream);
}

}  // extern "C"
