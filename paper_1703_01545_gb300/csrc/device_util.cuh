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

// binary64 -> binary32 with round-to-nearest-even, on the integer pipes (IEEE 754 layouts:
// sign, 11 / 8 exponent bits biased by 1023 / 127, 52 / 23 fraction bits); the FP64 pipe, which
// also carries the conversion instructions, is thin on this part.  Results in the binary32
// normal range are formed here (a carry out of the fraction rounds up into the exponent, up
// to infinity); zero, subnormal, out-of-range and non-finite inputs take the conversion
// instruction.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;                 // binary32 biased exponent
  if (e < 1 || e > 254) return __double2float_rn(x);
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
  const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | ((((uint32_t)e << 23) | m) + up));
}

// binary32 -> binary64 (exact) on the integer pipes; zero keeps its sign, subnormal and
// non-finite inputs take the conversion instruction
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f), e = (b >> 23) & 0xffu;
  if (e == 0u || e == 255u) {
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)f;
  }
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

}  // namespace afq
