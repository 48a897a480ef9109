// Small element-wise kernels used once per afqmc_setup / afqmc_set_walkers.
#include "device_util.cuh"
#include "internal.h"

namespace afq {
namespace {

__global__ void k_transpose(const double* __restrict__ in, double* __restrict__ out, int rows, int cols) {
  __shared__ double tile[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  for (int k = 0; k < 32; k += 8) {
    const int r = blockIdx.y * 32 + threadIdx.y + k;
    if (r < rows && c < cols) tile[threadIdx.y + k][threadIdx.x] = in[(int64_t)r * cols + c];
  }
  __syncthreads();
  const int r2 = blockIdx.y * 32 + threadIdx.x;
  for (int k = 0; k < 32; k += 8) {
    const int c2 = blockIdx.x * 32 + threadIdx.y + k;
    if (r2 < rows && c2 < cols) out[(int64_t)c2 * rows + r2] = tile[threadIdx.x][threadIdx.y + k];
  }
}

// Lt[p(i,j)][g] = L[g][i][j] for i <= j, p(i,j) = i*M - i*(i-1)/2 + (j-i)
__global__ void k_pack_Lt(const double* __restrict__ L, double* __restrict__ Lt, int M, int X) {
  const int64_t total = (int64_t)X * M * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % M);
    const int64_t r = e / M;
    const int i = (int)(r % M);
    const int g = (int)(r / M);
    if (i > j) continue;
    const int64_t p = (int64_t)i * M - (int64_t)i * (i - 1) / 2 + (j - i);
    Lt[p * X + g] = L[e];
  }
}

// <rho_g>_T = sum_(n,i) Ltil[g][n][i] psi[n][i]
__global__ void k_rho_mf(const double* __restrict__ Ltil, const double* __restrict__ psi, double* rho,
                         int NM) {
  __shared__ double red[4 * 8 + 4];
  const int g = blockIdx.x;
  double v[1] = {0};
  for (int e = threadIdx.x; e < NM; e += blockDim.x) v[0] += Ltil[(int64_t)g * NM + e] * psi[e];
  block_sum<1>(v, red);
  if (threadIdx.x == 0) rho[g] = v[0];
}

// K = h1 - 1/2 Q + sum_g rho_g L_g, then scaled by `scale`
__global__ void k_build_K(const double* h1, const double* Q, const double* L, const double* rho,
                          double* K, int M, int X, double scale) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  double s = 0;
  for (int g = 0; g < X; ++g) s = fma(rho[g], L[(int64_t)g * M * M + e], s);
  K[e] = scale * (h1[e] - 0.5 * Q[e] + s);
}

__global__ void k_add_identity(double* A, int M, double a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) A[(int64_t)i * M + i] += a;
}

// max_j sum_i |A[i][j]|
__global__ void k_norm1(const double* A, int M, double* out) {
  __shared__ double red[4 * 8 + 4];
  double best = 0;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double s = 0;
    for (int i = 0; i < M; ++i) s += fabs(A[(int64_t)i * M + j]);
    best = fmax(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b = fmax(b, red[i]);
    *out = b;
  }
}

// Lp[i][g][k] = L[g][i][k]
__global__ void k_permute_L(const double* __restrict__ L, double* __restrict__ Lp, int M, int X) {
  const int64_t total = (int64_t)X * M * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % M);
    const int64_t r = e / M;
    const int g = (int)(r % X);
    const int i = (int)(r / X);
    Lp[e] = L[((int64_t)g * M + i) * M + k];
  }
}

// phi[p][w][:] = psi  (p = 0 real plane; imaginary plane zeroed)
__global__ void k_broadcast_walkers(const double* __restrict__ psi, double* __restrict__ phi, int Nw, int NM) {
  const int64_t total = (int64_t)Nw * NM;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    phi[e] = psi[e % NM];
    phi[total + e] = 0.0;
  }
}

__global__ void k_init_weights(double* w, int* alive, const double* w_in, int Nw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nw) return;
  const double re = w_in ? w_in[k] : 1.0, im = w_in ? w_in[Nw + k] : 0.0;
  w[k] = re;
  w[Nw + k] = im;
  alive[k] = (re != 0.0 || im != 0.0) ? 1 : 0;
}

// external [2][Nw][M][N] <-> internal [2][Nw][N][M]
__global__ void k_phi_layout(const double* __restrict__ in, double* __restrict__ out, int Nw, int M, int N,
                             int to_internal) {
  const int64_t per = (int64_t)M * N, total = 2 * (int64_t)Nw * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wk = e / per;
    const int64_t r = e % per;
    if (to_internal) {  // e indexes internal [n][i]
      const int n = (int)(r / M), i = (int)(r % M);
      out[e] = in[wk * per + (int64_t)i * N + n];
    } else {            // e indexes external [i][n]
      const int i = (int)(r / N), n = (int)(r % N);
      out[e] = in[wk * per + (int64_t)n * M + i];
    }
  }
}

int grid_for(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_transpose(const double* in, double* out, int rows, int cols, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, s>>>(in, out, rows, cols);
  return cudaGetLastError();
}
cudaError_t launch_pack_Lt(const double* L, double* Lt, int M, int X, cudaStream_t s) {
  k_pack_Lt<<<grid_for((int64_t)X * M * M, 256), 256, 0, s>>>(L, Lt, M, X);
  return cudaGetLastError();
}
cudaError_t launch_rho_mf(const double* Ltil, const double* psi, double* rho, int X, int NM,
                          cudaStream_t s) {
  k_rho_mf<<<X, 256, 0, s>>>(Ltil, psi, rho, NM);
  return cudaGetLastError();
}
cudaError_t launch_build_K(const double* h1, const double* Q, const double* L, const double* rho,
                           double* K, int M, int X, double scale, cudaStream_t s) {
  k_build_K<<<(M * M + 255) / 256, 256, 0, s>>>(h1, Q, L, rho, K, M, X, scale);
  return cudaGetLastError();
}
cudaError_t launch_add_identity(double* A, int M, double a, cudaStream_t s) {
  k_add_identity<<<(M + 255) / 256, 256, 0, s>>>(A, M, a);
  return cudaGetLastError();
}
cudaError_t launch_norm1(const double* A, int M, double* out, cudaStream_t s) {
  k_norm1<<<1, 256, 0, s>>>(A, M, out);
  return cudaGetLastError();
}
cudaError_t launch_permute_L(const double* L, double* Lp, int M, int X, cudaStream_t s) {
  k_permute_L<<<grid_for((int64_t)X * M * M, 256), 256, 0, s>>>(L, Lp, M, X);
  return cudaGetLastError();
}
cudaError_t launch_broadcast_walkers(const double* psi, double* phi, int Nw, int NM,
                                     cudaStream_t s) {
  k_broadcast_walkers<<<grid_for((int64_t)Nw * NM, 256), 256, 0, s>>>(psi, phi, Nw, NM);
  return cudaGetLastError();
}
cudaError_t launch_init_weights(double* w, int* alive, const double* w_in, int Nw,
                                cudaStream_t s) {
  k_init_weights<<<(Nw + 255) / 256, 256, 0, s>>>(w, alive, w_in, Nw);
  return cudaGetLastError();
}
cudaError_t launch_phi_layout(const double* in, double* out, int Nw, int M, int N, int to_internal,
                              cudaStream_t s) {
  k_phi_layout<<<grid_for(2 * (int64_t)Nw * M * N, 256), 256, 0, s>>>(in, out, Nw, M, N, to_internal);
  return cudaGetLastError();
}

}  // namespace afq
