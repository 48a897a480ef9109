// Device helpers: complex arithmetic on (re, im) pairs, block reductions, Philox-4x32-10.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace afq {

struct cplx { double re, im; };
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cinv(cplx a) {
  double d = 1.0 / fma(a.re, a.re, a.im * a.im);
  return {a.re * d, -a.im * d};
}

// Sum of up to 4 doubles over the block; result valid in thread 0.  `red` needs
// 4 * (blockDim.x / 32) doubles of shared memory.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) red[q * nw + wid] = v[q];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = 0;
      for (int i = 0; i < nw; ++i) s += red[q * nw + i];
      v[q] = s;
    }
}

// Sum over the block, broadcast to every thread.  `red` as above plus K doubles.
template <int K>
__device__ __forceinline__ void block_allsum(double (&v)[K], double* red) {
  const int nw = blockDim.x >> 5;
  block_sum<K>(v, red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) red[4 * nw + q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = red[4 * nw + q];
  __syncthreads();
}

// Philox-4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box network with
// multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Two standard normals from one Philox block: 53-bit uniforms u1 in (0,1], u2 in
// [0,1), then Box-Muller (cos branch first).
__device__ __forceinline__ void philox_normal2(uint4 r, double& z0, double& z1) {
  const uint64_t a = ((uint64_t)r.y << 32) | r.x;
  const uint64_t b = ((uint64_t)r.w << 32) | r.z;
  const double u1 = (double)((a >> 11) + 1ull) * 0x1p-53;
  const double u2 = (double)(b >> 11) * 0x1p-53;
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

}  // namespace afq
