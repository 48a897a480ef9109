// Preliminary equilibration scheme (Sec. II.C): population control of the primary system by
// the comb, and the seeding of the secondary system's walkers from the primary's.
//
// Comb population control, in which heavy walkers are copied and light ones dropped
// (Sec. II.C): within a repeat, the running sum of the n weights (left to right, dead walkers
// counting 0; W its last value) is cut at the points (j + u_r) W / n, j = 0 .. n-1, and walker
// j of the repeat becomes a copy of the first walker whose running sum exceeds point j; every
// copy carries W / n.
// Seeding: walker k of B takes the first N_s^B columns of each spin block of walker k of A,
// and the weight w_A |R| max(0, cos arg R), R = <psi_T^B|phi_B> / <psi_T^A|phi_A>.
#include <cmath>

#include "internal.h"

namespace afq {
namespace {

// Walkers of repeat r: k in [ceil(r Nw / R), ceil((r + 1) Nw / R)), i.e. floor(k R / Nw) == r.
__host__ __device__ inline int64_t repeat_begin(int r, int Nw, int R) {
  return ((int64_t)r * Nw + R - 1) / R;
}

// One CTA per repeat.  Thread 0 forms the running sum in the order the oracle does; every
// thread then places its points by binary search.  share[r] = W / n, or NaN when the repeat
// has no weight (the caller then leaves the walkers untouched).
__global__ void __launch_bounds__(256) k_comb(const double* __restrict__ w,
                                              const int* __restrict__ alive,
                                              const double* __restrict__ u, double* __restrict__ cum,
                                              int* __restrict__ src, double* __restrict__ share,
                                              int Nw, int R) {
  const int r = blockIdx.x;
  const int64_t k0 = repeat_begin(r, Nw, R), k1 = repeat_begin(r + 1, Nw, R);
  const int n = (int)(k1 - k0);
  __shared__ double s_q;
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      acc += alive[k0 + i] ? w[k0 + i] : 0.0;
      cum[k0 + i] = acc;
    }
    s_q = (n > 0 && acc > 0.0) ? acc / (double)n : NAN;
    share[r] = s_q;
  }
  __syncthreads();
  const double q = s_q;
  if (!(q > 0.0)) return;
  const double ur = u[r];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double p = ((double)j + ur) * q;
    int lo = 0, hi = n;   // first i with cum[k0 + i] > p
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cum[k0 + mid] > p) hi = mid;
      else lo = mid + 1;
    }
    src[k0 + j] = (int)(k0 + (lo < n ? lo : n - 1));
  }
}

// out[k] = phi[src[k]] for both planes of the [2][Nw][N][M] layout (one CTA per walker).
__global__ void __launch_bounds__(256) k_gather_walkers(const double* __restrict__ phi,
                                                        double* __restrict__ out,
                                                        const int* __restrict__ src, int64_t NM,
                                                        int Nw) {
  const int64_t k = blockIdx.x, s = src[k], plane = (int64_t)Nw * NM;
  for (int64_t e = threadIdx.x; e < NM; e += blockDim.x) {
    out[k * NM + e] = phi[s * NM + e];
    out[plane + k * NM + e] = phi[plane + s * NM + e];
  }
}

__global__ void k_combed_weights(double* __restrict__ w, int* __restrict__ alive,
                                 const double* __restrict__ share, int Nw, int R) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nw) return;
  w[k] = share[(int)(((int64_t)k * R) / Nw)];
  w[Nw + k] = 0.0;
  alive[k] = 1;
}

// Column n of B's walker from column c(n) of A's: c = n in the spin-up block, n_up^A + (n -
// n_up^B) in the spin-down block ([2][Nw][N][M] layouts, one CTA per walker).
__global__ void __launch_bounds__(256) k_seed_columns(const double* __restrict__ phiA,
                                                      double* __restrict__ phiB, int M, int NA,
                                                      int nuA, int NB, int nuB, int Nw) {
  const int64_t k = blockIdx.x;
  const int64_t planeA = (int64_t)Nw * NA * M, planeB = (int64_t)Nw * NB * M;
  for (int e = threadIdx.x; e < NB * M; e += blockDim.x) {
    const int n = e / M, i = e - n * M;
    const int c = n < nuB ? n : nuA + (n - nuB);
    const int64_t a = (k * NA + c) * M + i, b = (k * NB + n) * M + i;
    phiB[b] = phiA[a];
    phiB[planeB + b] = phiA[planeA + a];
  }
}

// w_B = w_A |R| max(0, cos arg R) with log R = log O_B - log O_A; dead in A, singular in B
// (killed by the refresh) or cut by the projection: dead in B.
__global__ void k_seed_weights(const double* __restrict__ logOA, const double* __restrict__ wA,
                               const int* __restrict__ aliveA, const double* __restrict__ logOB,
                               double* __restrict__ wB, int* __restrict__ aliveB, int Nw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nw) return;
  const double lr = logOB[k] - logOA[k], li = logOB[Nw + k] - logOA[Nw + k];
  const double wn = wA[k] * exp(lr) * fmax(0.0, cos(li));
  const bool live = aliveA[k] != 0 && aliveB[k] != 0 && wn > 0.0;
  wB[k] = live ? wn : 0.0;
  wB[Nw + k] = 0.0;
  aliveB[k] = live ? 1 : 0;
}

}  // namespace

cudaError_t launch_comb(const Ctx& c, const double* u_dev, double* cum, int* src, double* share,
                        cudaStream_t s) {
  k_comb<<<c.R, 256, 0, s>>>(c.w, c.alive, u_dev, cum, src, share, c.Nw, c.R);
  return cudaGetLastError();
}

cudaError_t launch_apply_comb(const Ctx& c, const int* src, const double* share, double* scratch,
                              cudaStream_t s) {
  const int64_t NM = (int64_t)c.N * c.M;
  k_gather_walkers<<<c.Nw, 256, 0, s>>>(c.phi, scratch, src, NM, c.Nw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(c.phi, scratch, sizeof(double) * 2 * (size_t)c.Nw * NM,
                      cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  k_combed_weights<<<(c.Nw + 255) / 256, 256, 0, s>>>(c.w, c.alive, share, c.Nw, c.R);
  return cudaGetLastError();
}

cudaError_t launch_seed_columns(const Ctx& A, const Ctx& B, cudaStream_t s) {
  k_seed_columns<<<B.Nw, 256, 0, s>>>(A.phi, B.phi, B.M, A.N, A.n_up, B.N, B.n_up, B.Nw);
  return cudaGetLastError();
}

cudaError_t launch_seed_weights(const Ctx& A, const Ctx& B, cudaStream_t s) {
  k_seed_weights<<<(B.Nw + 255) / 256, 256, 0, s>>>(A.logO, A.w, A.alive, B.logO, B.w, B.alive,
                                                    B.Nw);
  return cudaGetLastError();
}

}  // namespace afq
