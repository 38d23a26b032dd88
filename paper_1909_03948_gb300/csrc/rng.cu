// rng.cu -- Philox4x32-10 normals for the Laplace sampler.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 4 x 32-bit counter, 2 x 32-bit
// key, 10 rounds of  (c0,c1,c2,c3) <- (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1,
// lo(M0 c0))  with the key bumped by the Weyl constants between rounds.
// Normal t of sample j: call g = t/4 with counter (g, g>>32, j, j>>32) and key
// (seed, seed>>32); words (x0,x1), (x2,x3) give two Box-Muller pairs with
// u = ((x >> 8) + 1/2) 2^-24, r = sqrt(-2 ln u_a), z = r cos(2 pi u_b), r sin(2 pi u_b)
// in FP32.  One thread per call: every normal is generated once.
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace hp {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ void box_muller(unsigned xa, unsigned xb, float *z0, float *z1) {
  const float ua = ((float)(xa >> 8) + 0.5f) * 5.9604644775390625e-08f;  // 2^-24
  const float ub = ((float)(xb >> 8) + 0.5f) * 5.9604644775390625e-08f;
  const float r = sqrtf(-2.0f * logf(ua));
  const float th = 6.2831853071795864769f * ub;
  *z0 = r * cosf(th);
  *z1 = r * sinf(th);
}

// out[ld * j + t] for t < nper, j < nsamples; raw != 0 writes the 32-bit words instead
__global__ void k_philox_normals(unsigned long long seed, long long first, int nper, double *out, long ld, int raw) {
  const int j = blockIdx.y;
  const unsigned long long smp = (unsigned long long)(first + j);
  const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
  const long ncalls = (nper + 3) / 4;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < ncalls; g += (long)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(
        make_uint4((unsigned)g, (unsigned)((unsigned long long)g >> 32), (unsigned)smp, (unsigned)(smp >> 32)), key);
    double v[4];
    if (raw) {
      v[0] = w.x;
      v[1] = w.y;
      v[2] = w.z;
      v[3] = w.w;
    } else {
      float z[4];
      box_muller(w.x, w.y, &z[0], &z[1]);
      box_muller(w.z, w.w, &z[2], &z[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = z[q];
    }
    const long t0 = 4 * g;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (t0 + q < nper) out[ld * j + t0 + q] = v[q];
  }
}

void launch_philox_normals(unsigned long long seed, long long first, int nsamples, int nper, double *out, long ld,
                           int raw, cudaStream_t st) {
  const long ncalls = (nper + 3) / 4;
  const int nb = (int)std::min<long>((ncalls + 255) / 256, std::max<long>(1, 4096 / std::max(nsamples, 1)));
  k_philox_normals<<<dim3(nb, nsamples), 256, 0, st>>>(seed, first, nper, out, ld, raw);
  count_launch();
}

}  // namespace hp

extern "C" int hp_philox_normals(unsigned long long seed, long long first_sample, int nsamples, int nper, double *out,
                                 int ld, int raw, void *stream) {
  using namespace hp;
  if (nsamples == 0 || nper == 0) return HP_OK;
  if (!out || nsamples < 0 || nper < 0 || ld < nper || first_sample < 0)
    return set_error(HP_ERR_INVALID, "hp_philox_normals: arguments");
  launch_philox_normals(seed, first_sample, nsamples, nper, out, ld, raw, static_cast<cudaStream_t>(stream));
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return HP_OK;
}
