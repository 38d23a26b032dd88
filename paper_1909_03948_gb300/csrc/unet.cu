// unet.cu -- the learned warm start: a 4-level U-Net (16-32-64-128 channels,
// 3x3 convolutions, BF16 weights, FP32 accumulation) that maps (m, rhs, mask)
// on the padded nodal grid to an initial guess for the PCG solves, trained on
// the GPU by the kernels below.  Not part of the paper.
//
// Layers (same order and shapes as the CPU reference): enc1a 3->16, enc1b 16->16,
// enc2a 16->32, enc2b, enc3a 32->64, enc3b, bota 64->128, botb, dec3a 192->64,
// dec3b, dec2a 96->32, dec2b, dec1a 48->16, dec1b, out 1x1 16->1.  Pooling: 2x2
// mean.  Decoder inputs: [nearest-upsampled coarser features, skip] -- the
// upsampling and the concatenation are folded into the convolution's input read.
// Activations are stored after ReLU (ReLU'(z) = [a > 0]); all tensors NCHW FP32.
//
// Training loss: the relative residual of the guess y in its stiffness system,
// L = 1/(2N) sum_n |mask b - S y|^2 / |mask b|^2 with S = mask K mask, K the
// symmetric 5-point stencil (diag, cx = coupling to the right neighbour, cy = to
// the neighbour below) carried per sample in aux = (b, diag, cx, cy) and the mask
// in input channel 2.
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>
#include <mutex>
#include <numeric>
#include <random>
#include <vector>

#include "internal.h"
#include "tc.cuh"

namespace hp {

struct ULayer {
  int ci, co, k;
  long woff, boff;  // offsets in the packed parameter vector
};

static const int kUL = 15;
static const int kUDims[kUL][3] = {{3, 16, 3},   {16, 16, 3}, {16, 32, 3}, {32, 32, 3}, {32, 64, 3},
                                   {64, 64, 3},  {64, 128, 3}, {128, 128, 3}, {192, 64, 3}, {64, 64, 3},
                                   {96, 32, 3},  {32, 32, 3}, {48, 16, 3},  {16, 16, 3}, {16, 1, 1}};

}  // namespace hp

struct hp_unet {
  int H = 0, W = 0, cap = 0;
  hp::ULayer L[hp::kUL];
  long nparam = 0;
  float *p32 = nullptr;           // master parameters (FP32), packed
  __nv_bfloat16 *w16 = nullptr;   // BF16 copy used by the kernels (weights; biases stay FP32 in p32)
  float *g = nullptr;             // gradients (packed like p32)
  float *am = nullptr, *av = nullptr;  // Adam moments
  long step = 0;
  // activations for a batch of up to cap samples
  float *x = nullptr, *aux = nullptr;  // input (cap,3,H,W); loss data (cap,4,H,W) = (b, diag, cx, cy)
  float *a[hp::kUL] = {};         // layer outputs (post-ReLU; out: linear)
  float *pl[3] = {};              // pooled inputs of enc2a, enc3a, bota
  float *da = nullptr, *db = nullptr, *dc = nullptr;  // gradient scratch (largest activation)
  double *lossbuf = nullptr;      // [0, 64): per-sample loss weights; then block partials
  cudaStream_t st = nullptr;
  // 3x3 convolutions on the tensor cores (default) or on the FP32 pipes
  int tensor_cores = 1;
  __nv_bfloat16 *wtc = nullptr;   // BF16 weights packed for the tensor-core kernel (forward and data-backward)
  long tc_fo[hp::kUL] = {}, tc_bo[hp::kUL] = {};  // offsets of each layer's packs in wtc (-1: none)
};

namespace hp {

constexpr int TB = 16;   // output tile edge of the convolutions
constexpr int OCB = 8;   // output channels per block

// Input channel c of a convolution whose input is [up(in1) (c1 channels, half
// resolution), in2 (c2 channels)] (decoder) or just in1 (c2 = 0, no upsampling).
struct ConvIn {
  const float *in1;
  int c1, up1;  // up1: in1 is at half resolution, read nearest-upsampled
  const float *in2;
  int c2;
};

__device__ __forceinline__ float read_in(const ConvIn &I, int n, int c, int y, int x, int H, int W) {
  if (y < 0 || y >= H || x < 0 || x >= W) return 0.f;
  if (c < I.c1) {
    if (I.up1) {
      const int h2 = H >> 1, w2 = W >> 1;
      return I.in1[(((long)n * I.c1 + c) * h2 + (y >> 1)) * w2 + (x >> 1)];
    }
    return I.in1[(((long)n * I.c1 + c) * H + y) * W + x];
  }
  return I.in2[(((long)n * I.c2 + (c - I.c1)) * H + y) * W + x];
}

// out[n, co, y, x] = b[co] + sum_{ci, dy, dx} w[co, ci, dy, dx] in[n, ci, y+dy-1, x+dx-1]; relu optional
__global__ void __launch_bounds__(256) k_conv_fwd(ConvIn I, const __nv_bfloat16 *__restrict__ w,
                                                  const float *__restrict__ b, float *__restrict__ out, int co_n,
                                                  int H, int W, int K, int relu) {
  __shared__ float tile[TB + 2][TB + 2];
  __shared__ float ws[OCB][9];
  const int ci_n = I.c1 + I.c2;
  const int tx = threadIdx.x % TB, ty = threadIdx.x / TB;
  const int ntx = (W + TB - 1) / TB;
  const int x0 = (blockIdx.x % ntx) * TB, y0 = (blockIdx.x / ntx) * TB;
  const int cob = blockIdx.y * OCB, n = blockIdx.z;
  const int x = x0 + tx, y = y0 + ty;
  float acc[OCB];
#pragma unroll
  for (int q = 0; q < OCB; ++q) acc[q] = (cob + q < co_n) ? b[cob + q] : 0.f;
  const int hal = K == 3 ? 1 : 0;
  for (int ci = 0; ci < ci_n; ++ci) {
    __syncthreads();
    for (int t = threadIdx.x; t < (TB + 2) * (TB + 2); t += 256) {
      const int ly = t / (TB + 2), lx = t % (TB + 2);
      tile[ly][lx] = read_in(I, n, ci, y0 + ly - hal, x0 + lx - hal, H, W);
    }
    if (threadIdx.x < OCB * K * K) {
      const int q = threadIdx.x / (K * K), kk = threadIdx.x % (K * K);
      ws[q][kk] = (cob + q < co_n) ? __bfloat162float(w[((long)(cob + q) * ci_n + ci) * K * K + kk]) : 0.f;
    }
    __syncthreads();
    if (K == 3) {
      float v[9];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) v[dy * 3 + dx] = tile[ty + dy][tx + dx];
#pragma unroll
      for (int q = 0; q < OCB; ++q)
#pragma unroll
        for (int kk = 0; kk < 9; ++kk) acc[q] += ws[q][kk] * v[kk];
    } else {
      const float v = tile[ty][tx];
#pragma unroll
      for (int q = 0; q < OCB; ++q) acc[q] += ws[q][0] * v;
    }
  }
  if (x < W && y < H) {
#pragma unroll
    for (int q = 0; q < OCB; ++q) {
      if (cob + q >= co_n) break;
      float r = acc[q];
      if (relu) r = fmaxf(r, 0.f);
      out[(((long)n * co_n + cob + q) * H + y) * W + x] = r;
    }
  }
}

// ---------------------------------------------------------------------------
// 3x3 convolutions on the tensor cores, as implicit GEMMs:
//   D[pixel, o] = sum_{tap, c} A[pixel, (tap, c)] B[(tap, c), o],
//   A[pixel, (tap, c)] = in[c, pixel + tap offset],  B[(tap, c), o] = w[o, c, tap].
// A CTA of 128 threads computes a tile of TC_TR rows x 8 tx columns: tx MMAs of M = 128
// pixels (MMA row group j = tile row j, 8 pixels), N = the output channels, accumulating
// in tensor memory.  K runs over 16-channel slabs and the 9 taps.  Per slab the CTA
// stages in shared memory the input halo ((TC_TR + 2) x (8 tx + 2) pixels, 16 channels)
// and the slab's weights, both in the no-swizzle core-matrix layout:
//   halo:    [term][channel group of 8][halo row][halo column][8 channels] BF16,
//   weights: [tap][channel group of 8][o][8 channels] BF16.
// A tap is the same halo with the descriptor's start moved by (dy rows, dx columns):
// the 8 pixels of an MMA row group are consecutive halo columns, 16 bytes apart, and
// consecutive row groups are consecutive halo rows (SBO = the halo row's bytes).
// The FP32 inputs enter as three BF16 terms (hi + mid + lo, each the rounded remainder of
// the previous ones: the FP32 significand) multiplied by the same BF16 weights, so the
// products carry the FP32 inputs, as the FP32-pipe kernels do.  The accumulation is the
// tensor core's FP32, which aligns and truncates each MMA's sum: a relative error of order
// 1e-5 over a layer.  (Two terms, 16 significant bits, flip ReLU decisions near zero
// often enough to move the first layer's weight gradient by 2.5e-3; three do not.)  Two stages: the loads of slab s + 1 overlap the MMAs of slab s;
// a stage is refilled once the tcgen05.commit of the MMAs that read it has arrived on
// its mbarrier.
// ---------------------------------------------------------------------------
constexpr int TC_NT = 128;   // threads per CTA: one accumulator row (tensor-memory lane) each
constexpr int TC_TR = 16;    // tile rows
constexpr int TC_TERMS = 3;  // BF16 terms of an FP32 input

__host__ __device__ constexpr int tc_hx(int tx) { return 8 * tx + 2; }                // halo columns
__host__ __device__ constexpr int tc_rs(int tx) { return tc_hx(tx) * 16; }            // bytes per halo row
__host__ __device__ constexpr int tc_g(int tx) { return (TC_TR + 2) * tc_rs(tx); }    // bytes per 8-channel group
__host__ __device__ constexpr int tc_halo_bytes(int tx) { return TC_TERMS * 2 * tc_g(tx); }
__host__ __device__ constexpr int tc_w_bytes(int co) { return 9 * 2 * co * 16; }
__host__ __device__ constexpr int tc_stage_bytes(int tx, int co) { return tc_halo_bytes(tx) + tc_w_bytes(co); }
// the most dynamic shared memory a launch takes: two stages of 16-row x 8-column tiles with up
// to 256 output channels (two 16 x 16 strips take less for the <= 128 channels they serve)
constexpr int TC_MAX_SMEM = 2 * tc_stage_bytes(1, 256);
static_assert(2 * tc_stage_bytes(2, 128) <= TC_MAX_SMEM, "stage size");

// set by a tensor-core convolution whose MMAs did not complete within its wait limit
__device__ int g_tc_timeout;

struct TcArgs {
  ConvIn I;
  int cin;             // input channels (I.c1 + I.c2)
  const uint4 *w;      // packed weights, one slab after another
  const float *bias;   // co values, or null
  float *out;          // (N, co, H, W)
  int co, H, W, relu;
  int tx, ntx;         // MMAs per tile (8-column strips), tiles per image row
  int cs;              // tensor-memory columns between the strips' accumulators
  unsigned ncols;      // tensor-memory columns allocated
  // optional 1x1 head on the activated outputs: hout[n, 0, y, x] = hb + sum_o hw[o] out[n, o, y, x]
  const __nv_bfloat16 *hw;
  const float *hb;
  float *hout;
};

constexpr int TC_IPT = 6;  // halo items per thread: 2 x (TC_TR + 2) x (8 tx + 2) <= TC_IPT x TC_NT
static_assert(2 * (TC_TR + 2) * tc_hx(2) <= TC_IPT * TC_NT, "halo items");

__device__ __forceinline__ unsigned bf16_bits(float v) {
  return static_cast<unsigned>(__bfloat16_as_ushort(__float2bfloat16_rn(v)));
}

// v = hi + mid + lo (+ a remainder below 2^-24 |v|); the two subtractions are exact
__device__ __forceinline__ void split3(float v, unsigned &h, unsigned &m, unsigned &l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(v);
  const float r1 = __fsub_rn(v, __bfloat162float(bh));
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = bf16_bits(__fsub_rn(r1, __bfloat162float(bm)));
}

template <int TX>
__global__ void __launch_bounds__(TC_NT, 4) k_conv_tc(TcArgs a) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int bx = blockIdx.x % a.ntx, by = blockIdx.x / a.ntx, n = blockIdx.y;
  const int x0 = bx * 8 * TX, y0 = by * TC_TR;
  constexpr int HX = tc_hx(TX), RS = tc_rs(TX), G = tc_g(TX), hbytes = tc_halo_bytes(TX);
  const int stage = tc_stage_bytes(TX, a.co), wbytes = tc_w_bytes(a.co);
  const uint32_t sbase = tc::saddr(tc_smem);
  const uint32_t bar0 = tc::saddr(&bars[0]), bar1 = tc::saddr(&bars[1]);
  auto bar = [&](int i) { return i ? bar1 : bar0; };
  if (warp == 0) tc::tmem_alloc(tc::saddr(&tslot), a.ncols);
  if (tid == 0) {
    tc::mbar_init(bar0, 1);
    tc::mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const int nslab = (a.cin + 15) / 16;
  const uint32_t idesc = tc::idesc_bf16(128, a.co);
  constexpr int items = 2 * (TC_TR + 2) * HX;
  bool ok = true;
  int last = -1;  // the last slab whose MMAs were committed
  for (int s = 0; s < nslab; ++s) {
    const int b = s & 1;
    unsigned char *stg = tc_smem + b * stage;
    if (s >= 2 && !(ok = __syncthreads_and(tc::mbar_wait(bar(b), ((s - 2) >> 1) & 1)))) break;
    // the slab's 16 channels come from one input tensor (c1 is a multiple of 16 when c2 > 0)
    const bool first = 16 * s < a.I.c1;
    const int up = first && a.I.up1;
    const int Hs = up ? a.H >> 1 : a.H, Ws = up ? a.W >> 1 : a.W;
    const int nsrc = first ? a.I.c1 : a.I.c2, cb = first ? 16 * s : 16 * s - a.I.c1;
    const long plane = (long)Hs * Ws;
    const float *src = (first ? a.I.in1 : a.I.in2) + ((long)n * nsrc + cb) * plane;
    // every load of this thread's items is issued before any is converted
    float v[TC_IPT][8];
#pragma unroll
    for (int k = 0; k < TC_IPT; ++k) {
      const int it = tid + k * TC_NT;
      const int cg = it / ((TC_TR + 2) * HX), rem = it - cg * ((TC_TR + 2) * HX);
      const int hy = rem / HX, hx = rem - hy * HX;
      const int y = y0 - 1 + hy, x = x0 - 1 + hx;
      const bool inb = it < items && y >= 0 && y < a.H && x >= 0 && x < a.W;
      const float *p = src + 8 * cg * plane + (long)(up ? y >> 1 : y) * Ws + (up ? x >> 1 : x);
#pragma unroll
      for (int e = 0; e < 8; ++e) v[k][e] = (inb && cb + 8 * cg + e < nsrc) ? p[e * plane] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < TC_IPT; ++k) {
      const int it = tid + k * TC_NT;
      if (it >= items) break;
      const int cg = it / ((TC_TR + 2) * HX), rem = it - cg * ((TC_TR + 2) * HX);
      const int hy = rem / HX, hx = rem - hy * HX;
      unsigned h[8], m[8], l[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) split3(v[k][e], h[e], m[e], l[e]);
      const int off = cg * G + hy * RS + hx * 16;
      *reinterpret_cast<uint4 *>(stg + off) =
          make_uint4(h[0] | h[1] << 16, h[2] | h[3] << 16, h[4] | h[5] << 16, h[6] | h[7] << 16);
      *reinterpret_cast<uint4 *>(stg + 2 * G + off) =
          make_uint4(m[0] | m[1] << 16, m[2] | m[3] << 16, m[4] | m[5] << 16, m[6] | m[7] << 16);
      *reinterpret_cast<uint4 *>(stg + 4 * G + off) =
          make_uint4(l[0] | l[1] << 16, l[2] | l[3] << 16, l[4] | l[5] << 16, l[6] | l[7] << 16);
    }
    const uint4 *wsrc = a.w + (long)s * (wbytes / 16);
    uint4 *wdst = reinterpret_cast<uint4 *>(stg + hbytes);
    for (int i = tid; i < wbytes / 16; i += TC_NT) wdst[i] = wsrc[i];
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t hb = sbase + b * stage, wb = hb + hbytes;
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap - 3 * (tap / 3);
        const uint64_t bd = tc::sdesc(wb + tap * 2 * a.co * 16, a.co * 16, 128);
#pragma unroll
        for (int t = 0; t < TX; ++t)
#pragma unroll
          for (int q = 0; q < TC_TERMS; ++q)
            tc::mma_bf16(tmem + t * a.cs, tc::sdesc(hb + q * 2 * G + dy * RS + (8 * t + dx) * 16, G, RS), bd,
                         idesc, (s | tap | q) != 0);
      }
      tc::commit(bar(b));
    }
    last = s;
  }
  if (ok && last >= 0) ok = __syncthreads_and(tc::mbar_wait(bar(last & 1), (last >> 1) & 1));
  if (!ok) {
    // raise the flag; wait once more (bounded) for the MMAs already issued before the
    // tensor memory and the shared memory they use are released
    if (tid == 0) {
      atomicExch(&g_tc_timeout, 1);
      if (last >= 0) (void)tc::mbar_wait(bar(last & 1), (last >> 1) & 1);
    }
  } else {
    tc::fence_after_sync();
    const int j = tid >> 3, r = tid & 7;  // accumulator row tid = tile row j, pixel r of the strip
    const int y = y0 + j;
    const long HW = (long)a.H * a.W;
#pragma unroll
    for (int t = 0; t < TX; ++t) {
      const int x = x0 + 8 * t + r;
      const bool in = y < a.H && x < a.W;
      float *o = a.out + (long)n * a.co * HW + (long)y * a.W + x;
      float head = a.hout ? a.hb[0] : 0.f;
      for (int c0 = 0; c0 < a.co; c0 += 16) {
        float v[16];
        tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * a.cs + c0), v);
        if (in) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float z = v[i] + (a.bias ? a.bias[c0 + i] : 0.f);
            if (a.relu) z = fmaxf(z, 0.f);
            o[(long)(c0 + i) * HW] = z;
            if (a.hout) head = fmaf(__bfloat162float(a.hw[c0 + i]), z, head);
          }
        }
      }
      if (in && a.hout) a.hout[(long)n * HW + (long)y * a.W + x] = head;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, a.ncols);
  }
}

// Weight packs of the tensor-core kernel, from the BF16 weights w[o, c, 3, 3]:
//   forward (N = co, K over c):      [slab][tap][kq][o][8]  = w[o, 16 slab + 8 kq + e, tap]
//   data-backward (N = ci, K over o): [slab][tap][kq][c][8] = w[16 slab + 8 kq + e, c, 8 - tap]
// (the data-backward is the forward convolution of dz with the flipped, transposed
// filter); channels past the end of a slab are zero.
struct TcPackL {
  long woff, fo, bo;  // source offset, forward / backward pack offsets (-1: none)
  int ci, co;
};
struct TcPack {
  TcPackL L[kUL];
};

__global__ void k_pack_tc(const __nv_bfloat16 *__restrict__ w16, TcPack P, __nv_bfloat16 *__restrict__ dst) {
  const TcPackL L = P.L[blockIdx.y];
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  const long stride = (long)gridDim.x * blockDim.x;
  if (L.fo >= 0) {
    const long nf = (long)((L.ci + 15) / 16) * 16 * 9 * L.co;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nf; i += stride) {
      long t = i >> 3;
      const int e = (int)(i & 7), o = (int)(t % L.co);
      t /= L.co;
      const int kq = (int)(t & 1), tap = (int)((t >> 1) % 9), sl = (int)((t >> 1) / 9);
      const int c = 16 * sl + 8 * kq + e;
      dst[L.fo + i] = c < L.ci ? w16[L.woff + ((long)o * L.ci + c) * 9 + tap] : zero;
    }
  }
  if (L.bo >= 0) {
    const long nb = (long)((L.co + 15) / 16) * 16 * 9 * L.ci;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nb; i += stride) {
      long t = i >> 3;
      const int e = (int)(i & 7), c = (int)(t % L.ci);
      t /= L.ci;
      const int kq = (int)(t & 1), tap = (int)((t >> 1) % 9), sl = (int)((t >> 1) / 9);
      const int o = 16 * sl + 8 * kq + e;
      dst[L.bo + i] = o < L.co ? w16[L.woff + ((long)o * L.ci + c) * 9 + (8 - tap)] : zero;
    }
  }
}

// dz = da * [a > 0] (relu) or da (linear), in place on da
__global__ void k_relu_back(float *da, const float *__restrict__ a, long cnt) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x)
    if (a[i] <= 0.f) da[i] = 0.f;
}

// d_in[n, ci, y, x] = sum_{co, dy, dx} w[co, ci, dy, dx] dz[n, co, y-dy+1, x-dx+1]  (full-resolution input grad)
__global__ void __launch_bounds__(256) k_conv_bwd_data(const float *__restrict__ dz, const __nv_bfloat16 *__restrict__ w,
                                                       float *__restrict__ din, int ci_n, int co_n, int H, int W,
                                                       int K) {
  __shared__ float tile[TB + 2][TB + 2];
  __shared__ float ws[OCB][9];
  const int tx = threadIdx.x % TB, ty = threadIdx.x / TB;
  const int ntx = (W + TB - 1) / TB;
  const int x0 = (blockIdx.x % ntx) * TB, y0 = (blockIdx.x / ntx) * TB;
  const int cib = blockIdx.y * OCB, n = blockIdx.z;
  const int x = x0 + tx, y = y0 + ty;
  const int hal = K == 3 ? 1 : 0;
  float acc[OCB];
#pragma unroll
  for (int q = 0; q < OCB; ++q) acc[q] = 0.f;
  for (int co = 0; co < co_n; ++co) {
    __syncthreads();
    for (int t = threadIdx.x; t < (TB + 2) * (TB + 2); t += 256) {
      const int ly = t / (TB + 2), lx = t % (TB + 2);
      const int yy = y0 + ly - hal, xx = x0 + lx - hal;
      tile[ly][lx] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? dz[(((long)n * co_n + co) * H + yy) * W + xx] : 0.f;
    }
    if (threadIdx.x < OCB * K * K) {
      const int q = threadIdx.x / (K * K), kk = threadIdx.x % (K * K);
      ws[q][kk] = (cib + q < ci_n) ? __bfloat162float(w[((long)co * ci_n + cib + q) * K * K + kk]) : 0.f;
    }
    __syncthreads();
    if (K == 3) {
      // output pixel (y, x) gets w[dy][dx] * dz(y - dy + 1, x - dx + 1) = tile[ty + 2 - dy][tx + 2 - dx]
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const float v = tile[ty + 2 - dy][tx + 2 - dx];
#pragma unroll
          for (int q = 0; q < OCB; ++q) acc[q] += ws[q][dy * 3 + dx] * v;
        }
    } else {
      const float v = tile[ty][tx];
#pragma unroll
      for (int q = 0; q < OCB; ++q) acc[q] += ws[q][0] * v;
    }
  }
  if (x < W && y < H) {
#pragma unroll
    for (int q = 0; q < OCB; ++q) {
      if (cib + q >= ci_n) break;
      din[(((long)n * ci_n + cib + q) * H + y) * W + x] = acc[q];
    }
  }
}

// gw[co, ci, dy, dx] = sum_{n, y, x} dz[n, co, y, x] in[n, ci, y+dy-1, x+dx-1];  one block per (co, ci)
__global__ void __launch_bounds__(256) k_conv_bwd_weight(ConvIn I, const float *__restrict__ dz, float *__restrict__ gw,
                                                         int co_n, int N, int H, int W, int K) {
  const int ci_n = I.c1 + I.c2;
  const int co = blockIdx.x / ci_n, ci = blockIdx.x % ci_n;
  const int hal = K == 3 ? 1 : 0;
  float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const long HW = (long)H * W;
  for (long t = threadIdx.x; t < (long)N * HW; t += blockDim.x) {
    const int n = (int)(t / HW);
    const int y = (int)((t % HW) / W), x = (int)(t % W);
    const float g = dz[((long)n * co_n + co) * HW + (long)y * W + x];
    if (g == 0.f) continue;
    for (int dy = 0; dy < K; ++dy)
      for (int dx = 0; dx < K; ++dx) acc[dy * K + dx] += g * read_in(I, n, ci, y + dy - hal, x + dx - hal, H, W);
  }
  for (int kk = 0; kk < K * K; ++kk) {
    const double s = block_sum<256>((double)acc[kk]);
    if (threadIdx.x == 0) gw[((long)co * ci_n + ci) * K * K + kk] = (float)s;
  }
}

__global__ void __launch_bounds__(256) k_bias_grad(const float *__restrict__ dz, float *__restrict__ gb, int co_n, int N,
                                                   long HW) {
  const int co = blockIdx.x;
  double acc = 0.0;
  for (long t = threadIdx.x; t < (long)N * HW; t += blockDim.x) {
    const int n = (int)(t / HW);
    acc += dz[((long)n * co_n + co) * HW + t % HW];
  }
  acc = block_sum<256>(acc);
  if (threadIdx.x == 0) gb[co] = (float)acc;
}

__global__ void k_pool(const float *__restrict__ in, float *__restrict__ out, long NC, int H, int W) {
  const int h2 = H / 2, w2 = W / 2;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NC * h2 * w2; i += (long)gridDim.x * blockDim.x) {
    const long nc = i / ((long)h2 * w2);
    const int y = (int)((i / w2) % h2), x = (int)(i % w2);
    const float *p = in + nc * H * W + (long)(2 * y) * W + 2 * x;
    out[i] = 0.25f * (p[0] + p[1] + p[W] + p[W + 1]);
  }
}

// d_in_full += pool_backward(d_out): each fine pixel gets a quarter of its coarse gradient
__global__ void k_pool_back_add(const float *__restrict__ dpo, float *__restrict__ din, long NC, int H, int W) {
  const int h2 = H / 2, w2 = W / 2;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NC * H * W; i += (long)gridDim.x * blockDim.x) {
    const long nc = i / ((long)H * W);
    const int y = (int)((i / W) % H), x = (int)(i % W);
    din[i] += 0.25f * dpo[nc * h2 * w2 + (long)(y / 2) * w2 + x / 2];
  }
}

// split the gradient of a decoder input [up(coarse) (c1), skip (c2)]:
// d_coarse = up_backward(first c1 channels) ; d_skip += last c2 channels
__global__ void k_split_up_back(const float *__restrict__ dcat, float *__restrict__ dcoarse, float *__restrict__ dskip,
                                int N, int c1, int c2, int H, int W) {
  const int h2 = H / 2, w2 = W / 2;
  const long nc1 = (long)N * c1 * h2 * w2;
  const long nc2 = (long)N * c2 * H * W;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nc1 + nc2; i += (long)gridDim.x * blockDim.x) {
    if (i < nc1) {
      const int x = (int)(i % w2), y = (int)((i / w2) % h2);
      const long nc = i / ((long)h2 * w2);
      const int n = (int)(nc / c1), c = (int)(nc % c1);
      const float *p = dcat + (((long)n * (c1 + c2) + c) * H + 2 * y) * W + 2 * x;
      dcoarse[i] = p[0] + p[1] + p[W] + p[W + 1];
    } else {
      const long j = i - nc1;
      const long HW = (long)H * W;
      const int n = (int)(j / (c2 * HW)), c = (int)((j / HW) % c2);
      dskip[j] += dcat[((long)n * (c1 + c2) + c1 + c) * HW + j % HW];
    }
  }
}

// (S v)(r, c) = mask(r, c) [diag v + cx(r, c) v(r, c+1) + cx(r, c-1) v(r, c-1) + cy(r, c) v(r+1, c)
//                           + cy(r-1, c) v(r-1, c)] with v masked; aux = (b, diag, cx, cy), mask = x channel 2
__device__ __forceinline__ float stencil_at(const float *__restrict__ v, const float *__restrict__ aux,
                                            const float *__restrict__ mk, int r, int c, int H, int W) {
  const long HW = (long)H * W;
  const long i = (long)r * W + c;
  if (mk[i] == 0.f) return 0.f;
  const float *d = aux + HW, *cx = aux + 2 * HW, *cy = aux + 3 * HW;
  float acc = d[i] * v[i];
  if (c + 1 < W) acc += cx[i] * (mk[i + 1] * v[i + 1]);
  if (c > 0) acc += cx[i - 1] * (mk[i - 1] * v[i - 1]);
  if (r + 1 < H) acc += cy[i] * (mk[i + W] * v[i + W]);
  if (r > 0) acc += cy[i - W] * (mk[i - W] * v[i - W]);
  return acc;
}

// per-sample weights w_n = 1 / (N |mask_n b_n|^2), 0 for a zero right-hand side; one block per sample
__global__ void __launch_bounds__(256) k_sample_w(const float *__restrict__ x, const float *__restrict__ aux, long HW,
                                                  int N, double *__restrict__ w) {
  const int n = blockIdx.x;
  const float *b = aux + (long)n * 4 * HW, *mk = x + ((long)n * 3 + 2) * HW;
  double acc = 0.0;
  for (long i = threadIdx.x; i < HW; i += blockDim.x) {
    const double v = (double)b[i] * mk[i];
    acc += v * v;
  }
  acc = block_sum<256>(acc);
  if (threadIdx.x == 0) w[n] = acc > 0.0 ? 1.0 / (N * acc) : 0.0;
}

// wr = w_n (mask b - S y) and the loss partials 1/2 w_n |mask b - S y|^2
__global__ void __launch_bounds__(256) k_residual(const float *__restrict__ y, const float *__restrict__ x,
                                                  const float *__restrict__ aux, const double *__restrict__ w,
                                                  float *__restrict__ wr, int H, int W, long cnt,
                                                  double *__restrict__ part) {
  const long HW = (long)H * W;
  double acc = 0.0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < cnt; t += (long)gridDim.x * blockDim.x) {
    const long n = t / HW, i = t % HW;
    const float *an = aux + n * 4 * HW, *mk = x + (n * 3 + 2) * HW;
    const float r = an[i] * mk[i] - stencil_at(y + n * HW, an, mk, (int)(i / W), (int)(i % W), H, W);
    wr[t] = (float)(w[n] * r);
    acc += 0.5 * w[n] * (double)r * r;
  }
  acc = block_sum<256>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// dL/dy = -S (w r)   (S symmetric)
__global__ void __launch_bounds__(256) k_residual_grad(const float *__restrict__ wr, const float *__restrict__ x,
                                                       const float *__restrict__ aux, float *__restrict__ dy, int H,
                                                       int W, long cnt) {
  const long HW = (long)H * W;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < cnt; t += (long)gridDim.x * blockDim.x) {
    const long n = t / HW, i = t % HW;
    dy[t] = -stencil_at(wr + n * HW, aux + n * 4 * HW, x + (n * 3 + 2) * HW, (int)(i / W), (int)(i % W), H, W);
  }
}

__global__ void k_adam(float *p, __nv_bfloat16 *w16, const float *__restrict__ g, float *m, float *v, long cnt,
                       const unsigned char *__restrict__ is_w, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    if (is_w[i]) w16[i] = __float2bfloat16(pi);
  }
}

__global__ void k_to_bf16(const float *__restrict__ p, __nv_bfloat16 *w16, long cnt) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x)
    w16[i] = __float2bfloat16(p[i]);
}

static int gblocks(long cnt) { return (int)std::max<long>(1, std::min<long>((cnt + 255) / 256, 4096)); }

// ---------------------------------------------------------------------------
// forward / backward of a batch of N <= cap samples held in U->x (N,3,H,W)
// ---------------------------------------------------------------------------
// the tensor-core convolution of I (cin channels) with a weight pack into co output channels
static void conv_tc(hp_unet *U, const ConvIn &I, int cin, const __nv_bfloat16 *pack, const float *bias, float *out,
                    int co, int N, int H, int W, int relu, const __nv_bfloat16 *hw = nullptr,
                    const float *hb = nullptr, float *hout = nullptr) {
  // (a failure here surfaces as the launch's error, which the calling entry point returns)
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_MAX_SMEM);
    cudaFuncSetAttribute(k_conv_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_MAX_SMEM);
  });
  TcArgs a;
  a.I = I;
  a.cin = cin;
  a.w = reinterpret_cast<const uint4 *>(pack);
  a.bias = bias;
  a.out = out;
  a.co = co;
  a.H = H;
  a.W = W;
  a.relu = relu;
  a.tx = co <= 128 ? 2 : 1;
  a.ntx = (W + 8 * a.tx - 1) / (8 * a.tx);
  a.cs = (co + 31) / 32 * 32;
  unsigned nc = 32;
  while (nc < (unsigned)(a.tx * a.cs)) nc <<= 1;
  a.ncols = nc;
  a.hw = hw;
  a.hb = hb;
  a.hout = hout;
  const dim3 grid(a.ntx * ((H + TC_TR - 1) / TC_TR), N);
  const int stages = cin > 16 ? 2 : 1;  // one 16-channel slab needs no second stage
  if (a.tx == 2)
    k_conv_tc<2><<<grid, TC_NT, stages * tc_stage_bytes(2, co), U->st>>>(a);
  else
    k_conv_tc<1><<<grid, TC_NT, stages * tc_stage_bytes(1, co), U->st>>>(a);
  count_launch();
}

// whether layer li runs on the tensor cores (3x3, output channels a multiple of 16 up to 256)
static bool use_tc(const hp_unet *U, int li) { return U->tensor_cores && U->tc_fo[li] >= 0; }

// rebuilds the tensor-core weight packs from the BF16 weights (after every change of them)
static void tc_repack(hp_unet *U) {
  TcPack P;
  long most = 0;
  for (int l = 0; l < kUL; ++l) {
    const ULayer &L = U->L[l];
    P.L[l] = TcPackL{L.woff, U->tc_fo[l], U->tc_bo[l], L.ci, L.co};
    most = std::max(most, (long)(L.ci + 15) / 16 * 16 * 9 * L.co);
  }
  k_pack_tc<<<dim3((unsigned)std::min<long>((most + 255) / 256, 256), kUL), 256, 0, U->st>>>(U->w16, P, U->wtc);
  count_launch();
}

static void conv_fwd(hp_unet *U, int li, ConvIn I, float *out, int N, int H, int W, int relu) {
  const ULayer &L = U->L[li];
  if (use_tc(U, li) && (I.c2 == 0 || I.c1 % 16 == 0)) {  // a 16-channel slab reads one input tensor
    conv_tc(U, I, L.ci, U->wtc + U->tc_fo[li], U->p32 + L.boff, out, L.co, N, H, W, relu);
    return;
  }
  const int tiles = ((W + TB - 1) / TB) * ((H + TB - 1) / TB);
  dim3 grid(tiles, (L.co + OCB - 1) / OCB, N);
  k_conv_fwd<<<grid, 256, 0, U->st>>>(I, U->w16 + L.woff, U->p32 + L.boff, out, L.co, H, W, L.k, relu);
  count_launch();
}

static ConvIn cin(const float *a, int c, int up = 0, const float *b = nullptr, int cb = 0) {
  return ConvIn{a, c, up, b, cb};
}

static void unet_forward(hp_unet *U, int N) {
  const int H = U->H, W = U->W;
  const int h[4] = {H, H / 2, H / 4, H / 8}, w[4] = {W, W / 2, W / 4, W / 8};
  conv_fwd(U, 0, cin(U->x, 3), U->a[0], N, h[0], w[0], 1);
  conv_fwd(U, 1, cin(U->a[0], 16), U->a[1], N, h[0], w[0], 1);
  k_pool<<<gblocks((long)N * 16 * h[1] * w[1]), 256, 0, U->st>>>(U->a[1], U->pl[0], (long)N * 16, h[0], w[0]);
  conv_fwd(U, 2, cin(U->pl[0], 16), U->a[2], N, h[1], w[1], 1);
  conv_fwd(U, 3, cin(U->a[2], 32), U->a[3], N, h[1], w[1], 1);
  k_pool<<<gblocks((long)N * 32 * h[2] * w[2]), 256, 0, U->st>>>(U->a[3], U->pl[1], (long)N * 32, h[1], w[1]);
  conv_fwd(U, 4, cin(U->pl[1], 32), U->a[4], N, h[2], w[2], 1);
  conv_fwd(U, 5, cin(U->a[4], 64), U->a[5], N, h[2], w[2], 1);
  k_pool<<<gblocks((long)N * 64 * h[3] * w[3]), 256, 0, U->st>>>(U->a[5], U->pl[2], (long)N * 64, h[2], w[2]);
  conv_fwd(U, 6, cin(U->pl[2], 64), U->a[6], N, h[3], w[3], 1);
  conv_fwd(U, 7, cin(U->a[6], 128), U->a[7], N, h[3], w[3], 1);
  conv_fwd(U, 8, cin(U->a[7], 128, 1, U->a[5], 64), U->a[8], N, h[2], w[2], 1);
  conv_fwd(U, 9, cin(U->a[8], 64), U->a[9], N, h[2], w[2], 1);
  conv_fwd(U, 10, cin(U->a[9], 64, 1, U->a[3], 32), U->a[10], N, h[1], w[1], 1);
  conv_fwd(U, 11, cin(U->a[10], 32), U->a[11], N, h[1], w[1], 1);
  conv_fwd(U, 12, cin(U->a[11], 32, 1, U->a[1], 16), U->a[12], N, h[0], w[0], 1);
  if (use_tc(U, 13)) {
    // dec1b with the 1x1 output layer folded into its epilogue
    const ULayer &L = U->L[13], &O = U->L[14];
    conv_tc(U, cin(U->a[12], 16), L.ci, U->wtc + U->tc_fo[13], U->p32 + L.boff, U->a[13], L.co, N, h[0], w[0], 1,
            U->w16 + O.woff, U->p32 + O.boff, U->a[14]);
  } else {
    conv_fwd(U, 13, cin(U->a[12], 16), U->a[13], N, h[0], w[0], 1);
    conv_fwd(U, 14, cin(U->a[13], 16), U->a[14], N, h[0], w[0], 0);
  }
  count_launch(3);
}

// backward of conv layer li: dz (in place in `d`, N x co x H x W) -> weight / bias grads and input grad d_in
static void conv_bwd(hp_unet *U, int li, ConvIn I, float *d, const float *a_out, bool relu, float *d_in, int N, int H,
                     int W) {
  const ULayer &L = U->L[li];
  const long cnt = (long)N * L.co * H * W;
  if (relu) {
    k_relu_back<<<gblocks(cnt), 256, 0, U->st>>>(d, a_out, cnt);
    count_launch();
  }
  k_conv_bwd_weight<<<L.co * L.ci, 256, 0, U->st>>>(I, d, U->g + L.woff, L.co, N, H, W, L.k);
  k_bias_grad<<<L.co, 256, 0, U->st>>>(d, U->g + L.boff, L.co, N, (long)H * W);
  count_launch(2);
  if (d_in && use_tc(U, li) && U->tc_bo[li] >= 0) {
    conv_tc(U, ConvIn{d, L.co, 0, nullptr, 0}, L.co, U->wtc + U->tc_bo[li], nullptr, d_in, L.ci, N, H, W, 0);
  } else if (d_in) {
    const int tiles = ((W + TB - 1) / TB) * ((H + TB - 1) / TB);
    dim3 grid(tiles, (L.ci + OCB - 1) / OCB, N);
    k_conv_bwd_data<<<grid, 256, 0, U->st>>>(d, U->w16 + L.woff, d_in, L.ci, L.co, H, W, L.k);
    count_launch();
  }
}

// gradients of the loss with respect to all parameters, for dy already in U->da (N,1,H,W)
static void unet_backward(hp_unet *U, int N) {
  const int H = U->H, W = U->W;
  const int h[4] = {H, H / 2, H / 4, H / 8}, w[4] = {W, W / 2, W / 4, W / 8};
  float *A = U->da, *B = U->db, *Cs = U->dc;  // scratch (each >= largest activation)
  // skip gradients accumulate in dedicated regions of the pooled buffers? keep them explicit:
  // ds1 (N,16,H,W), ds2 (N,32,H/2), ds3 (N,64,H/4) live in the upper parts of Cs
  float *ds1 = Cs, *ds2 = Cs + (long)N * 16 * h[0] * w[0], *ds3 = ds2 + (long)N * 32 * h[1] * w[1];
  cudaMemsetAsync(ds1, 0, sizeof(float) * ((long)N * 16 * h[0] * w[0] + (long)N * 32 * h[1] * w[1] +
                                           (long)N * 64 * h[2] * w[2]), U->st);
  // out (linear): d(a13) into B
  conv_bwd(U, 14, cin(U->a[13], 16), A, nullptr, false, B, N, h[0], w[0]);
  conv_bwd(U, 13, cin(U->a[12], 16), B, U->a[13], true, A, N, h[0], w[0]);
  conv_bwd(U, 12, cin(U->a[11], 32, 1, U->a[1], 16), A, U->a[12], true, B, N, h[0], w[0]);  // B: d concat (48)
  k_split_up_back<<<gblocks((long)N * 48 * h[0] * w[0]), 256, 0, U->st>>>(B, A, ds1, N, 32, 16, h[0], w[0]);
  conv_bwd(U, 11, cin(U->a[10], 32), A, U->a[11], true, B, N, h[1], w[1]);
  conv_bwd(U, 10, cin(U->a[9], 64, 1, U->a[3], 32), B, U->a[10], true, A, N, h[1], w[1]);  // A: d concat (96)
  k_split_up_back<<<gblocks((long)N * 96 * h[1] * w[1]), 256, 0, U->st>>>(A, B, ds2, N, 64, 32, h[1], w[1]);
  conv_bwd(U, 9, cin(U->a[8], 64), B, U->a[9], true, A, N, h[2], w[2]);
  conv_bwd(U, 8, cin(U->a[7], 128, 1, U->a[5], 64), A, U->a[8], true, B, N, h[2], w[2]);  // B: d concat (192)
  k_split_up_back<<<gblocks((long)N * 192 * h[2] * w[2]), 256, 0, U->st>>>(B, A, ds3, N, 128, 64, h[2], w[2]);
  conv_bwd(U, 7, cin(U->a[6], 128), A, U->a[7], true, B, N, h[3], w[3]);
  conv_bwd(U, 6, cin(U->pl[2], 64), B, U->a[6], true, A, N, h[3], w[3]);  // A: d pooled (64, H/8)
  // d(a5) = pool_back(A) + ds3
  k_pool_back_add<<<gblocks((long)N * 64 * h[2] * w[2]), 256, 0, U->st>>>(A, ds3, (long)N * 64, h[2], w[2]);
  conv_bwd(U, 5, cin(U->a[4], 64), ds3, U->a[5], true, B, N, h[2], w[2]);
  conv_bwd(U, 4, cin(U->pl[1], 32), B, U->a[4], true, A, N, h[2], w[2]);
  k_pool_back_add<<<gblocks((long)N * 32 * h[1] * w[1]), 256, 0, U->st>>>(A, ds2, (long)N * 32, h[1], w[1]);
  conv_bwd(U, 3, cin(U->a[2], 32), ds2, U->a[3], true, B, N, h[1], w[1]);
  conv_bwd(U, 2, cin(U->pl[0], 16), B, U->a[2], true, A, N, h[1], w[1]);
  k_pool_back_add<<<gblocks((long)N * 16 * h[0] * w[0]), 256, 0, U->st>>>(A, ds1, (long)N * 16, h[0], w[0]);
  conv_bwd(U, 1, cin(U->a[0], 16), ds1, U->a[1], true, B, N, h[0], w[0]);
  conv_bwd(U, 0, cin(U->x, 3), B, U->a[0], true, nullptr, N, h[0], w[0]);
  count_launch(6);
}

float *unet_input(hp_unet *U) { return U->x; }
const float *unet_output(const hp_unet *U) { return U->a[14]; }
int unet_cap(const hp_unet *U) { return U->cap; }
void unet_dims(const hp_unet *U, int *H, int *W) {
  *H = U->H;
  *W = U->W;
}
// after the network's stream has synchronised: fails the call if a tensor-core convolution
// gave up waiting for its MMAs, and clears the flag
static int tc_status() {
  int f = 0;
  HP_CUDA(cudaMemcpyFromSymbol(&f, g_tc_timeout, sizeof(int)));
  if (!f) return HP_OK;
  const int zero = 0;
  HP_CUDA(cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int)));
  return set_error(HP_ERR_CUDA, "a tensor-core convolution timed out waiting for its MMAs");
}

void unet_run(hp_unet *U, int N, cudaStream_t st) {
  cudaStream_t own = U->st;
  U->st = st;
  unet_forward(U, N);
  U->st = own;
}

}  // namespace hp

using namespace hp;

extern "C" {

int hp_unet_create(int H, int W, int batch_cap, hp_unet **out) {
  if (!out || H < 8 || W < 8 || H % 8 || W % 8 || batch_cap < 1 || batch_cap > 64)
    return set_error(HP_ERR_INVALID, "hp_unet_create: H, W multiples of 8, 1 <= batch_cap <= 64");
  hp_unet *U = new hp_unet();
  U->H = H;
  U->W = W;
  U->cap = batch_cap;
  long off = 0;
  for (int l = 0; l < kUL; ++l) {
    U->L[l] = ULayer{kUDims[l][0], kUDims[l][1], kUDims[l][2], 0, 0};
    U->L[l].woff = off;
    off += (long)U->L[l].co * U->L[l].ci * U->L[l].k * U->L[l].k;
    U->L[l].boff = off;
    off += U->L[l].co;
  }
  U->nparam = off;
  // tensor-core weight packs: forward for every 3x3 layer, data-backward where the input
  // gradient is needed and the input channels are a multiple of 16 (not the first layer)
  long toff = 0;
  for (int l = 0; l < kUL; ++l) {
    const ULayer &L = U->L[l];
    U->tc_fo[l] = U->tc_bo[l] = -1;
    if (L.k != 3 || L.co % 16 || L.co > 256) continue;
    U->tc_fo[l] = toff;
    toff += (long)(L.ci + 15) / 16 * 16 * 9 * L.co;
    if (l > 0 && L.ci % 16 == 0 && L.ci <= 256) {
      U->tc_bo[l] = toff;
      toff += (long)(L.co + 15) / 16 * 16 * 9 * L.ci;
    }
  }
  auto fail = [&](const char *w) {
    hp_unet_destroy(U);
    return set_error(HP_ERR_NOMEM, w);
  };
  if (cudaMalloc(&U->wtc, sizeof(__nv_bfloat16) * toff)) return fail("hp_unet_create: tensor-core weights");
  if (cudaMalloc(&U->p32, sizeof(float) * off) || cudaMalloc(&U->w16, sizeof(__nv_bfloat16) * off) ||
      cudaMalloc(&U->g, sizeof(float) * off) || cudaMalloc(&U->am, sizeof(float) * off) ||
      cudaMalloc(&U->av, sizeof(float) * off))
    return fail("hp_unet_create: parameters");
  cudaMemset(U->am, 0, sizeof(float) * off);
  cudaMemset(U->av, 0, sizeof(float) * off);
  const long HW = (long)H * W, N = batch_cap;
  const int ch[kUL] = {16, 16, 32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16, 16, 1};
  const int lev[kUL] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0};
  for (int l = 0; l < kUL; ++l)
    if (cudaMalloc(&U->a[l], sizeof(float) * N * ch[l] * (HW >> (2 * lev[l])))) return fail("hp_unet_create: act");
  const int plc[3] = {16, 32, 64};
  for (int q = 0; q < 3; ++q)
    if (cudaMalloc(&U->pl[q], sizeof(float) * N * plc[q] * (HW >> (2 * (q + 1))))) return fail("hp_unet_create: pool");
  const long big = N * 192 * (HW >> 4) > N * 48 * HW ? N * 192 * (HW >> 4) : N * 48 * HW;
  const long skips = N * (16 * HW + 32 * (HW >> 2) + 64 * (HW >> 4));
  if (cudaMalloc(&U->x, sizeof(float) * N * 3 * HW) || cudaMalloc(&U->aux, sizeof(float) * N * 4 * HW) ||
      cudaMalloc(&U->da, sizeof(float) * big) ||
      cudaMalloc(&U->db, sizeof(float) * big) || cudaMalloc(&U->dc, sizeof(float) * std::max(big, skips)) ||
      cudaMalloc(&U->lossbuf, sizeof(double) * (64 + 4096)))
    return fail("hp_unet_create: buffers");
  *out = U;
  return HP_OK;
}

void hp_unet_destroy(hp_unet *U) {
  if (!U) return;
  cudaDeviceSynchronize();
  for (void *p : {(void *)U->p32, (void *)U->w16, (void *)U->wtc, (void *)U->g, (void *)U->am, (void *)U->av, (void *)U->x,
                  (void *)U->aux, (void *)U->da, (void *)U->db, (void *)U->dc, (void *)U->lossbuf})
    if (p) cudaFree(p);
  for (int l = 0; l < kUL; ++l)
    if (U->a[l]) cudaFree(U->a[l]);
  for (int q = 0; q < 3; ++q)
    if (U->pl[q]) cudaFree(U->pl[q]);
  delete U;
}

long hp_unet_num_params(const hp_unet *U) { return U ? U->nparam : 0; }

int hp_unet_set_tensor_cores(hp_unet *U, int on) {
  if (!U || (on != 0 && on != 1)) return set_error(HP_ERR_INVALID, "hp_unet_set_tensor_cores: on is 0 or 1");
  HP_CUDA(cudaStreamSynchronize(U->st));
  U->tensor_cores = on;
  return HP_OK;
}

int hp_unet_get_tensor_cores(const hp_unet *U) { return U ? U->tensor_cores : -1; }

int hp_unet_set_params(hp_unet *U, const float *params_host) {
  if (!U || !params_host) return set_error(HP_ERR_INVALID, "null");
  HP_CUDA(cudaMemcpy(U->p32, params_host, sizeof(float) * U->nparam, cudaMemcpyHostToDevice));
  k_to_bf16<<<gblocks(U->nparam), 256, 0, U->st>>>(U->p32, U->w16, U->nparam);
  count_launch();
  tc_repack(U);
  HP_CUDA(cudaMemset(U->am, 0, sizeof(float) * U->nparam));
  HP_CUDA(cudaMemset(U->av, 0, sizeof(float) * U->nparam));
  U->step = 0;
  HP_CUDA(cudaStreamSynchronize(U->st));
  return HP_OK;
}

int hp_unet_get_params(const hp_unet *U, float *params_host) {
  if (!U || !params_host) return set_error(HP_ERR_INVALID, "null");
  HP_CUDA(cudaMemcpy(params_host, U->p32, sizeof(float) * U->nparam, cudaMemcpyDeviceToHost));
  return HP_OK;
}

// y (N,1,H,W) = net(x (N,3,H,W)); device pointers, N <= cap
int hp_unet_forward(hp_unet *U, const float *x_dev, int N, float *y_dev) {
  if (!U || !x_dev || !y_dev || N < 1 || N > U->cap) return set_error(HP_ERR_INVALID, "hp_unet_forward: arguments");
  const long HW = (long)U->H * U->W;
  HP_CUDA(cudaMemcpyAsync(U->x, x_dev, sizeof(float) * N * 3 * HW, cudaMemcpyDeviceToDevice, U->st));
  unet_forward(U, N);
  HP_CUDA(cudaMemcpyAsync(y_dev, U->a[14], sizeof(float) * N * HW, cudaMemcpyDeviceToDevice, U->st));
  HP_CUDA(cudaStreamSynchronize(U->st));
  HP_CUDA(cudaGetLastError());
  return tc_status();
}

// loss and parameter gradients of one batch: x (N,3,H,W), aux (N,4,H,W)
static int unet_grad(hp_unet *U, const float *x, const float *aux, int N, double *loss) {
  const long HW = (long)U->H * U->W;
  HP_CUDA(cudaMemcpyAsync(U->x, x, sizeof(float) * N * 3 * HW, cudaMemcpyDeviceToDevice, U->st));
  HP_CUDA(cudaMemcpyAsync(U->aux, aux, sizeof(float) * N * 4 * HW, cudaMemcpyDeviceToDevice, U->st));
  unet_forward(U, N);
  const long cnt = (long)N * HW;
  const int nb = gblocks(cnt);
  double *wts = U->lossbuf, *part = U->lossbuf + 64;
  k_sample_w<<<N, 256, 0, U->st>>>(U->x, U->aux, HW, N, wts);
  k_residual<<<nb, 256, 0, U->st>>>(U->a[14], U->x, U->aux, wts, U->db, U->H, U->W, cnt, part);
  k_residual_grad<<<nb, 256, 0, U->st>>>(U->db, U->x, U->aux, U->da, U->H, U->W, cnt);
  count_launch(3);
  unet_backward(U, N);
  std::vector<double> hp(nb);
  HP_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, U->st));
  HP_CUDA(cudaStreamSynchronize(U->st));
  if (loss) *loss = std::accumulate(hp.begin(), hp.end(), 0.0);
  HP_TRY(tc_status());
  return cuda_check(cudaGetLastError(), "unet_grad");
}

int hp_unet_loss_grad(hp_unet *U, const float *x_dev, const float *aux_dev, int N, double *loss_host,
                      float *grad_host) {
  if (!U || !x_dev || !aux_dev || N < 1 || N > U->cap) return set_error(HP_ERR_INVALID, "hp_unet_loss_grad: arguments");
  HP_TRY(unet_grad(U, x_dev, aux_dev, N, loss_host));
  if (grad_host) HP_CUDA(cudaMemcpy(grad_host, U->g, sizeof(float) * U->nparam, cudaMemcpyDeviceToHost));
  return HP_OK;
}

// Adam training over nsamples stored contiguously (X: nsamples x 3 x H x W, A: nsamples x 4 x H x W)
int hp_unet_train(hp_unet *U, const float *X, const float *A, int nsamples, int epochs, int batch, double lr,
                  unsigned long long seed, double *loss_per_epoch) {
  if (!U || !X || !A || nsamples < 1 || epochs < 1 || batch < 1 || batch > U->cap)
    return set_error(HP_ERR_INVALID, "hp_unet_train: arguments");
  const long HW = (long)U->H * U->W;
  std::vector<int> order(nsamples);
  std::iota(order.begin(), order.end(), 0);
  std::mt19937_64 rng(seed);
  float *bx = nullptr, *ba = nullptr;
  unsigned char *isw = nullptr;
  HP_CUDA(cudaMalloc(&bx, sizeof(float) * batch * 3 * HW));
  HP_CUDA(cudaMalloc(&ba, sizeof(float) * batch * 4 * HW));
  HP_CUDA(cudaMalloc(&isw, U->nparam));
  {
    std::vector<unsigned char> h(U->nparam, 0);
    for (int l = 0; l < kUL; ++l)
      std::fill(h.begin() + U->L[l].woff, h.begin() + U->L[l].boff, 1);
    HP_CUDA(cudaMemcpy(isw, h.data(), U->nparam, cudaMemcpyHostToDevice));
  }
  int rc = 0;
  for (int ep = 0; ep < epochs && !rc; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    double ep_loss = 0.0;
    int nbat = 0;
    for (int b0 = 0; b0 + batch <= nsamples && !rc; b0 += batch) {
      for (int q = 0; q < batch; ++q) {
        const long src = order[b0 + q];
        cudaMemcpyAsync(bx + (long)q * 3 * HW, X + src * 3 * HW, sizeof(float) * 3 * HW, cudaMemcpyDeviceToDevice,
                        U->st);
        cudaMemcpyAsync(ba + (long)q * 4 * HW, A + src * 4 * HW, sizeof(float) * 4 * HW, cudaMemcpyDeviceToDevice,
                        U->st);
      }
      double l = 0.0;
      rc = unet_grad(U, bx, ba, batch, &l);
      if (rc) break;
      ++U->step;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.f / (1.f - std::pow(b1, (float)U->step)), c2 = 1.f / (1.f - std::pow(b2, (float)U->step));
      k_adam<<<gblocks(U->nparam), 256, 0, U->st>>>(U->p32, U->w16, U->g, U->am, U->av, U->nparam, isw, (float)lr, b1,
                                                   b2, 1e-8f, c1, c2);
      count_launch();
      tc_repack(U);
      ep_loss += l;
      ++nbat;
    }
    if (loss_per_epoch) loss_per_epoch[ep] = nbat ? ep_loss / nbat : 0.0;
  }
  cudaStreamSynchronize(U->st);
  cudaFree(bx);
  cudaFree(ba);
  cudaFree(isw);
  if (rc) return rc;
  return cuda_check(cudaGetLastError(), "hp_unet_train");
}

}  // extern "C"
