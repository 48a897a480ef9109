// Local energies for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's
// memory pool or under a strict memory budget, an embedding that hands over only
// pre-allocated device buffers, or a process whose allocation path is unavailable
// at the point of the call.  afqmc_local_energy_static serves them: it needs no
// handle (afqmc_setup allocates) and allocates nothing.  Its intermediates (trial
// columns, half-rotated Cholesky tensor, walker Green's functions) live in the
// file-scope array below, which every GPU that loads this library holds until the
// process exits.  The kernels are the library's own overlap and local-energy kernels.
#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_energy_scratch[kStaticScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// The array's name is only a host-side stand-in: its device address must be
// looked up once per device, with that device current.
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Device memory of device `dev` (managed memory is reachable from every device).  A buffer
// on another GPU is refused: the kernels would read it over the peer link, or fault without
// peer access.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// caller layout phi[2][Nw][M][N] (walkers w0..w0+c) -> internal [2][c][N][M]
__global__ void k_chunk_to_internal(const double* __restrict__ phi, double* __restrict__ out,
                                    int Nw, int w0, int c, int M, int N) {
  const int64_t per = (int64_t)M * N, total = 2 * (int64_t)c * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pw = e / per, r = e % per;
    const int plane = (int)(pw / c), wk = (int)(pw % c);
    const int n = (int)(r / M), i = (int)(r % M);
    out[e] = phi[((int64_t)plane * Nw + w0 + wk) * per + (int64_t)i * N + n];
  }
}

// internal eloc[2][c] -> caller e_local[2][Nw] at walkers w0..w0+c; a walker the overlap
// refresh killed (singular or non-finite overlap: it has no Green's function) gets NaN
__global__ void k_chunk_energy_out(const double* __restrict__ el, const int* __restrict__ alive,
                                   double* __restrict__ out, int Nw, int w0, int c) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= c) return;
  const bool ok = alive[k] != 0;
  out[w0 + k] = ok ? el[k] : NAN;
  out[(int64_t)Nw + w0 + k] = ok ? el[c + k] : NAN;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" afqmc_status afqmc_local_energy_static(const double* h1, const double* L,
                                                  const double* trial, const double* phi,
                                                  int M, int X, int n_up, int n_dn,
                                                  int n_walkers, double* e_local,
                                                  cudaStream_t s) {
  const int N = n_up + n_dn;
  if (!h1 || !L || !trial || !phi || !e_local) return AFQMC_ERR_ARG;
  if (M < 1 || X < 1 || n_up < 0 || n_dn < 0 || N < 1 || n_up > M || n_dn > M || n_up > 32 ||
      n_dn > 32 || (int64_t)N * M > 4096 || n_walkers < 1)
    return AFQMC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AFQMC_ERR_CUDA;
  for (const void* p : {(const void*)h1, (const void*)L, (const void*)trial, (const void*)phi,
                        (const void*)e_local})
    if (!on_device(p, dev)) return AFQMC_ERR_ARG;
  // fixed part: psi [N][M], Ltil [X][N][M], htil [N][M], flags
  const size_t NM = (size_t)N * M;
  const size_t fixed = align256(NM * 8) + align256((size_t)X * NM * 8) + align256(NM * 8) + 256;
  // per walker: phi, theta [2][N][M]; logO, w, eloc [2]; aux [4]; alive.  The seven
  // per-walker buffers are each rounded up to 256 bytes, so 7 * 256 bytes of slack suffice.
  const size_t per_w = 4 * NM * 8 + 10 * 8 + 4, slack = 7 * 256;
  if (fixed + per_w + slack > kStaticScratchBytes) return AFQMC_ERR_ARG;
  const int chunk = (int)std::min<size_t>((size_t)n_walkers,
                                          (kStaticScratchBytes - fixed - slack) / per_w);
  void* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) return AFQMC_ERR_CUDA;
  unsigned char* p = static_cast<unsigned char*>(base);
  auto take = [&](size_t bytes) {
    unsigned char* q = p;
    p += align256(bytes);
    return q;
  };
  afq::Ctx c;
  c.M = M; c.X = X; c.n_up = n_up; c.n_dn = n_dn; c.N = N; c.Nw = chunk; c.R = 1;
  afqmc_default_options(&c.opt);
  c.opt.n_walkers = chunk;
  c.psi = (double*)take(NM * 8);
  c.Ltil = (double*)take((size_t)X * NM * 8);
  c.htil = (double*)take(NM * 8);
  c.d_flags = (int*)take(256);
  c.phi = (double*)take(2 * (size_t)chunk * NM * 8);
  c.theta = (double*)take(2 * (size_t)chunk * NM * 8);
  c.logO = (double*)take(2 * (size_t)chunk * 8);
  c.w = (double*)take(2 * (size_t)chunk * 8);
  c.eloc = (double*)take(2 * (size_t)chunk * 8);
  c.aux = (double*)take(4 * (size_t)chunk * 8);
  c.alive = (int*)take((size_t)chunk * 4);
  if ((size_t)(p - static_cast<unsigned char*>(base)) > kStaticScratchBytes) return AFQMC_ERR_ARG;

  cudaError_t e = afq::prepare_kernels(c);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.d_flags, 0, 256, s);
  if (e == cudaSuccess) e = afq::launch_transpose(trial, c.psi, M, N, s);
  if (e == cudaSuccess)
    e = afq::gemm_tn_f64(M, N, M, 1.0, L, M, (int64_t)M * M, c.psi, M, 0, 0.0, c.Ltil, M,
                         (int64_t)NM, X, s);
  if (e == cudaSuccess)
    e = afq::gemm_tn_f64(M, N, M, 1.0, h1, M, 0, c.psi, M, 0, 0.0, c.htil, M, 0, 1, s);
  for (int w0 = 0; w0 < n_walkers && e == cudaSuccess; w0 += chunk) {
    const int cw = std::min(chunk, n_walkers - w0);
    c.Nw = cw;  // the chunk's planes are packed back to back in the scratch
    const int64_t tot = 2 * (int64_t)cw * NM;
    const int grid = (int)std::min<int64_t>((tot + 255) / 256, 152 * 32);
    k_chunk_to_internal<<<grid, 256, 0, s>>>(phi, c.phi, n_walkers, w0, cw, M, N);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = afq::launch_init_weights(c.w, c.alive, nullptr, cw, s);
    if (e == cudaSuccess) e = afq::launch_overlap(c, nullptr, afq::OV_REFRESH, s);
    if (e == cudaSuccess) e = afq::launch_energy(c, s);
    if (e == cudaSuccess) {
      k_chunk_energy_out<<<(cw + 255) / 256, 256, 0, s>>>(c.eloc, c.alive, e_local, n_walkers,
                                                           w0, cw);
      e = cudaGetLastError();
    }
  }
  return e == cudaSuccess ? AFQMC_OK : AFQMC_ERR_CUDA;
}
