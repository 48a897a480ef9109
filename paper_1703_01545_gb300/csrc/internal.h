// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstdint>
#include <mutex>
#include <string>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include "../../include/afqmc.h"

namespace afq {

// Packed upper triangle (i <= j) of a symmetric M x M matrix, row-major:
// idx(i, j) = i*M - i*(i-1)/2 + (j - i).
inline int64_t packed_size(int M) { return (int64_t)M * (M + 1) / 2; }

// Dynamic shared-memory limits already raised on a group of kernels, kept per device (a
// function attribute belongs to the device's context) and guarded for setups on several
// threads.  raise(slot, bytes, set) calls set() when `bytes` is above what the slot allows on
// the current device; limits only grow, so handles set up earlier keep valid launches.
struct SmemLimits {
  static constexpr int kDevices = 64, kSlots = 8;
  std::mutex mu;
  size_t have[kDevices][kSlots] = {};
  template <class Set>
  cudaError_t raise(int slot, size_t bytes, Set set) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kDevices && slot >= 0 && slot < kSlots;
    std::lock_guard<std::mutex> lock(mu);
    if (cached && bytes <= have[dev][slot]) return cudaSuccess;
    e = set();
    if (e == cudaSuccess && cached) have[dev][slot] = bytes;
    return e;
  }
};

struct Workspace;
struct TcOperand;
// tensor-core local energy of the split-precision step (energy_tc.cu)
struct EnergyTc {
  TcOperand* A = nullptr;     // rows (g, n') of Psi^T L_g, spin blocks padded to NP / 2
  TcOperand* B = nullptr;     // rows (w, re/im, n') of Theta
  float* part = nullptr;      // [RT][2][NwP] partial two-body energies per row tile
  float* trs = nullptr;       // spin-blocked form: [2 spins][Nw][X] (re, im) traces tr T^s_g
  float* hh = nullptr;        // [N][M] Psi^T h1 as FP32 pairs hh + hl (the one-body term)
  float* hl = nullptr;
  int NP = 0, Kp = 0, RT = 0, NwP = 0;
};

struct Ctx {
  int M = 0, X = 0, n_up = 0, n_dn = 0, N = 0, Nw = 0, R = 1;
  int64_t P = 0;              // packed size of a symmetric M x M matrix
  afqmc_options opt{};
  double sqrt_dt = 0, c_mf = 0, e_trial = 0;
  uint64_t step = 0;          // host mirror of the device step counter
  int device = 0;
  // constants (device)
  double* h1 = nullptr;       // [M][M]
  double* L = nullptr;        // [X][M][M]
  double* Lt = nullptr;       // [P][X]  packed upper triangle of every L_g, g fastest
  double* Ltil = nullptr;     // [X][N][M]  rows of Psi_s^T L_g
  double* htil = nullptr;     // [N][M]     rows of Psi_s^T h1
  double* psi = nullptr;      // [N][M]     trial columns
  double* expK = nullptr;     // [M][M]     exp(-dt K / 2)
  double* rho_mf = nullptr;   // [X]        <rho_g>_T
  // walker state (device), planar complex
  double* phi = nullptr;      // [2][Nw][N][M]
  double* phi2 = nullptr;     // [2][Nw][N][M]  propagation scratch
  double* theta = nullptr;    // [2][Nw][N][M]  Theta = Phi O^{-1}, then scratch within a step
  double* logO = nullptr;     // [2][Nw]
  double* w = nullptr;        // [2][Nw]
  int* alive = nullptr;       // [Nw]
  // per-step scratch
  double* rhobar = nullptr;   // [2][Nw][X]
  double* U = nullptr;        // [2][Nw][X]   sqrt(dt)-scaled coefficients of A = sum_g (U_re + i U_im)_g L_g
  double* Avhs = nullptr;     // [2][Nw][P]   packed A of every walker
  double* aux = nullptr;      // [Nw][4]      log s (re, im), x.xbar - xbar.xbar/2 (re, im)
  double* eloc = nullptr;     // [2][Nw]
  double* esum = nullptr;     // [R][4]       sum w E_L (re, im), sum w (re, im)
  unsigned long long* d_step = nullptr;  // device step counter t of the field stream
  int* d_flags = nullptr;     // [4] error counters: [0] singular overlaps
  // split-precision (AFQMC_BF16X3) operands and FP32 work arrays; null in FP64 mode
  struct TcOperand* tc_L = nullptr;      // A of V_HS: rows ij (M^2), K = g
  struct TcOperand* tc_Ltri = nullptr;   // the same rows for the lower-triangle blocks only
  struct TcOperand* tc_Ltil = nullptr;   // A of the force bias: rows g, K = (n, i)
  struct TcOperand* tc_U = nullptr;      // B of V_HS: rows (p, w), K = g
  struct TcOperand* tc_Theta = nullptr;  // B of the force bias: rows (p, w), K = (n, i)
  float* Avhs32 = nullptr;    // [2][Nw][M*M]
  float* phi32 = nullptr;     // [2][Nw][N][M]
  float* expK32 = nullptr;    // [M][M]
  float* Ltil32 = nullptr;    // [X][N][M]
  float* theta32 = nullptr;   // [2][Nw][N][M]  Theta in FP32 (split-precision mode)
  float* LtT = nullptr;       // [X][M][NPT]    Psi_s^T L_g transposed, spin-padded (FP32)
  float *psi32h = nullptr, *psi32l = nullptr;   // [N][M]  psi = psi32h + psi32l (FP32 pair)
  double* ovdet = nullptr;    // [Nw][8]  per-walker determinant factors between the overlap kernels
  uint32_t* emI_pk = nullptr; // [64][64] e^{-dt K/2} - I as split-bf16 words (tensor-core propagator)
  // large-M tensor-core propagator (propagate_tcl.cu): V_HS as split bf16 [2][Nw][M][Mp] (written
  // by the V_HS contraction when that propagator runs), e^{-dt K/2} - I as split bf16 [M][Mp],
  // and their four tensor maps (A hi, A lo, E hi, E lo)
  __nv_bfloat16 *tcl_ahi = nullptr, *tcl_alo = nullptr, *tcl_ehi = nullptr, *tcl_elo = nullptr;
  CUtensorMap* tcl_maps = nullptr;
  float* rhobar32 = nullptr;  // [2][Nw][X]  force bias of the split-precision step (FP32 GEMM output)
  float* rho_mf32 = nullptr;  // [X]         <rho_g>_T in FP32
  int* d_tc_err = nullptr;    // set by a tensor-core kernel whose bounded wait expired
  EnergyTc* etc = nullptr;    // tensor-core local energy (null when the shape is unsupported)
  // autotuned variants (autotune.cpp); -1 = not tuned, use the default
  int tune_energy_wb = -1;    // local energy: 0 tensor cores, else walkers per CTA of the FP32 kernel (2, 4, 8)
  int tune_taylor_smem = -1;  // propagation: 2 fused kernel; Taylor kernel with A in shared memory (1) or L1 (0)
  int tune_mgs = -1;          // orthonormalisation: 1 Cholesky QR, 0 modified Gram-Schmidt kernels
  // tangent mode (tangent.cu): derivative along h1 -> h1 + lambda P, FP64 path only
  bool tangent_on = false;
  double* Bneg = nullptr;     // [M][M]  -dt K / 2 (kept from setup)
  double* dexpK = nullptr;    // [M][M]  Frechet derivative of exp(-dt K/2) along -dt P/2
  double* htilP = nullptr;    // [N][M]  rows of Psi_s^T P
  double de_trial = 0.0;      // dE_T/dlambda = sum_s tr(P Psi_s Psi_s^T)
  double *dphi = nullptr, *dphi2 = nullptr, *dtheta = nullptr;   // [2][Nw][N][M]
  double *drhobar = nullptr, *dU = nullptr;                      // [2][Nw][X]
  double* dAvhs = nullptr;    // [2][Nw][P]
  double *dlogO = nullptr, *dlogw = nullptr, *daux = nullptr, *deloc = nullptr, *desum = nullptr;
  // multi-determinant trial psi_T = sum_d c_d D_d (multidet.cu; FP64); n_det = 0: one determinant
  int n_det = 0;
  double* md_coef = nullptr;   // [Nd]        c_d
  double* md_psi = nullptr;    // [Nd][N][M]  columns of D_d
  double* md_Ltil = nullptr;   // [Nd][X][N][M] rows of D_d,s^T L_g
  double* md_htil = nullptr;   // [Nd][N][M]  rows of D_d,s^T h1
  double* md_logO = nullptr;   // [Nd][2][Nw] log O_d (-inf: O_d = 0)
  double* md_theta = nullptr;  // [Nd][2][Nw][N][M] Theta_d
  double* md_share = nullptr;  // [Nd][2][Nw] w_d = c_d O_d / <psi_T|phi>
  double* md_rhobar = nullptr; // [Nd][2][Nw][X] force bias of each determinant
  double* md_eloc = nullptr;   // [Nd][2][Nw] local energy of each determinant
  // pair-run graph cache (owned; see pair.cu)
  void* pair_cache = nullptr;
  int pair_loop = 1;          // pair run: 1 one graph launch looping over the blocks on the device,
                              // 0 one launch of the block graph per measurement block
  uint64_t uid = 0;           // unique per handle, so a cached graph never outlives its partner
  std::string err;
};
void destroy_pair_cache(Ctx* h);

// ---- kernel launchers (implemented in the .cu files) ----
// C[z][n*ldc + m] = alpha * sum_k A[z][m*lda + k] * B[z][n*ldb + k] + beta * C[...]
enum GemmUse { GEMM_GENERIC = 0, GEMM_FORCE_BIAS = 1, GEMM_VHS = 2, GEMM_ONEBODY = 3 };
cudaError_t gemm_tn_f64(int Md, int Nd, int Kd, double alpha, const double* A, int64_t lda,
                        int64_t sA, const double* B, int64_t ldb, int64_t sB, double beta,
                        double* C, int64_t ldc, int64_t sC, int batch, cudaStream_t s,
                        GemmUse use = GEMM_GENERIC);

// ---- split-BF16 tensor-core GEMM (gemm_tc.cu) ----
// A K-major operand split into bf16 hi/lo rows of Kp (multiple of 64) elements, with
// its two TMA descriptors (128-row boxes, 128-byte swizzle).
struct TcOperand {
  CUtensorMap map_hi, map_lo;
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;
  int rows = 0, Kp = 0;
};
cudaError_t tc_make_operand(TcOperand& op, __nv_bfloat16* hi, __nv_bfloat16* lo, int rows, int Kp,
                            int box_rows);
cudaError_t split_bf16(const double* in, int64_t ld_in, int rows, int K, int Kp, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, cudaStream_t s);
int tc_bn();
int tc_pad_rows(int rows);
// C[n*ldc + m] = alpha * sum_k A[m][k] B[n][k] with both operands split (3 MMAs per product)
cudaError_t gemm_bf16x3(const TcOperand& A, const TcOperand& B, int Md, int Nd, float alpha,
                        float* C, int64_t ldc, int* err, cudaStream_t s);
cudaError_t gemm_bf16x3(const TcOperand& A, const TcOperand& B, int Md, int Nd, float alpha,
                        double* C, int64_t ldc, int* err, cudaStream_t s);
// Split-BF16 output of the product C[n][m] with Md = M^2 rows m = i M + j: hi = bf16(C) and
// lo = bf16(C - hi) stored at n * ld + i * Mp + j (Mp >= M elements per orbital row, so that the
// rows of every matrix meet the 16-byte stride rule of a TMA descriptor); the padding entries
// j >= M are not written.
struct SplitOut {
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;
  int M = 0, Mp = 0;
  int64_t ld = 0;
  int tri = 0;   // 1: A's rows are the lower-triangle 16 x 16 (i, j) blocks (vhs_tri_rows)
};
// Rows of the V_HS operand that covers only the lower-triangle blocks of the symmetric
// matrices: block (a, b), a >= b, of 16 x 16 index pairs (i, j) is two 128-row tiles
// (i in 16 a + 8 h + [0, 8), j in 16 b + [0, 16), h = 0, 1); V_HS[j][i] = V_HS[i][j] gives
// the rest.
int vhs_tri_rows(int M);
bool tc_persistent_ok(int Md, int Nd, int b_rows);
cudaError_t split_bf16_tri(const double* in, int64_t ld_in, int M, int K, int Kp, __nv_bfloat16* hi,
                           __nv_bfloat16* lo, cudaStream_t s);
cudaError_t gemm_bf16x3_split_out(const TcOperand& A, const TcOperand& B, int Md, int Nd,
                                  float alpha, const SplitOut& so, int* err, cudaStream_t s);
cudaError_t prepare_tc_kernels();
cudaError_t gemm_bf16x3_wait_selftest(const TcOperand& A, const TcOperand& B, int Md, int Nd,
                                      float* C, int64_t ldc, int* err, uint64_t wait_ns,
                                      cudaStream_t s);
// FP32 kernels of the split-precision step (mixed_kernels.cu)
cudaError_t prepare_mixed_kernels(const Ctx& c);
cudaError_t gemm_f32_from_f64(int Md, int Nd, int Kd, float alpha, const float* A, int64_t lda,
                              const double* B, int64_t ldb, float* C, int64_t ldc, cudaStream_t s);
cudaError_t gemm_f32_to_f64(int Md, int Nd, int Kd, float alpha, const float* A, int64_t lda,
                            const float* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s);
cudaError_t launch_taylor_f32(const Ctx& c, float* phi32, const float* A32, cudaStream_t s);
cudaError_t launch_energy_f32(const Ctx& c, const float* Ltil32, cudaStream_t s, int n_walkers = -1);
cudaError_t to_float(const double* in, float* out, int64_t n, cudaStream_t s);
// hi = fl32(in), lo = fl32(in - hi)
cudaError_t split_f32(const double* in, float* hi, float* lo, int64_t n, cudaStream_t s);
cudaError_t prepare_mixed_kernels2(const Ctx& c);
cudaError_t build_LtT(const Ctx& c, float* LtT, cudaStream_t s);
int64_t LtT_size(const Ctx& c);
cudaError_t launch_energy_tiled(const Ctx& c, const float* theta32, const float* LtT,
                                cudaStream_t s, int n_walkers = -1, int wb = -1);
bool energy_variant_ok(const Ctx& c, int wb);
bool taylor_variant_ok(const Ctx& c, int use_smem);
cudaError_t launch_taylor_f32_variant(const Ctx& c, float* phi32, const float* A32, cudaStream_t s,
                                      int use_smem);
// fused FP32 propagator e^{-dt K/2} e^A e^{-dt K/2} of the split-precision step (propagate_f32.cu)
bool propagate_f32_ok(const Ctx& c);
cudaError_t prepare_propagate_f32();
cudaError_t launch_propagate_f32(const Ctx& c, double* out, float* out32, cudaStream_t s);
// tensor-core propagator (propagate_tc.cu), M <= 64 and N <= 16
bool propagate_tc_ok(const Ctx& c);
cudaError_t prepare_propagate_tc();
cudaError_t pack_propagate_tc(const Ctx& c, uint32_t* emI_pk, cudaStream_t s);
cudaError_t launch_propagate_tc(const Ctx& c, double* out, float* out32, cudaStream_t s);
// large-M tensor-core propagator (propagate_tcl.cu), M <= 256 and N <= 32: reads V_HS in the
// split form c.tcl_ahi / c.tcl_alo (rows of Mp = propagate_tcl_mp(M) elements)
bool propagate_tcl_ok(const Ctx& c);
int propagate_tcl_mp(int M);
cudaError_t prepare_propagate_tcl();
cudaError_t setup_propagate_tcl(Ctx& c, cudaStream_t s);
cudaError_t launch_propagate_tcl(const Ctx& c, double* out, float* out32, cudaStream_t s);
// Propagation variants of the split-precision step: 4 large-M tensor-core kernel, 3 tensor-core
// kernel (M <= 64, N <= 16), 2 fused FP32 kernel, 1 / 0 two FP32 GEMMs around a Taylor kernel
// with A in shared memory / through L1.  The effective variant is the tuned one, else the
// first the shape supports in the order 3, 4, 2, 1, 0.  Variant 4 reads V_HS in its split form,
// the others in FP32 (c.Avhs32): vhs_launch writes the form the variant reads.
int propagation_variant(const Ctx& c);
// V_HS of every walker from the split coefficients c.tc_U, in the form variant `pv` reads
cudaError_t vhs_launch(const Ctx& c, int pv, cudaStream_t s);
// Phi' of every walker from c.phi and V_HS into out (FP64); variants 2, 3 and 4 also write
// the FP32 copy out32 (may be null), variants 0 and 1 use c.phi32 as scratch
cudaError_t launch_propagation(const Ctx& c, int variant, double* out, float* out32, cudaStream_t s);
// tensor-core local energy (energy_tc.cu)
int energy_tc_np(const Ctx& c);   // padded orbitals per Cholesky vector (8, 16, 32) or 0
cudaError_t prepare_energy_tc_kernels();
void energy_tc_sizes(const Ctx& c, int NP, int* rows_A, int* rows_B, int* Kp, int* RT, int* NwP);
bool energy_tc_spin(const Ctx& c);   // M > 64: one product per spin block
cudaError_t energy_tc_init(const Ctx& c, EnergyTc& et, cudaStream_t s);
cudaError_t launch_energy_tc(const Ctx& c, cudaStream_t s, int n_walkers = -1);
// runtime autotuner (autotune.cpp): times the variants on the handle's buffers at setup
cudaError_t autotune_mixed(Ctx& c, const char* cache_path, cudaStream_t s);
cudaError_t launch_taylor_f32_best(const Ctx& c, float* phi32, const float* A32, cudaStream_t s);
// latency-oriented FP64 walker kernels of the split-precision step (walker_fast.cu)
bool fast_walker_kernels_ok(const Ctx& c);
cudaError_t prepare_fast_walker_kernels(const Ctx& c);
// with_weights = false launches the overlap kernel without the per-walker weight kernel
cudaError_t launch_overlap_fast(const Ctx& c, const double* src, int mode, cudaStream_t s,
                                const float* src32 = nullptr, bool with_weights = true);
// update_logO: subtract log det R (the column norms) from log O instead of recomputing it
cudaError_t launch_mgs_warp(const Ctx& c, cudaStream_t s, bool update_logO = false);
bool mgs_chol_ok(const Ctx& c);
cudaError_t launch_fields_mixed(const Ctx& c, const double* fields, cudaStream_t s);
// tangent mode (tangent.cu)
bool tangent_fits(const Ctx& c);
cudaError_t prepare_tangent_kernels(const Ctx& c);
cudaError_t launch_fields_tan(const Ctx& c, const double* fields, cudaStream_t s);
cudaError_t launch_taylor_tan(const Ctx& c, cudaStream_t s);
cudaError_t launch_overlap_tan(const Ctx& c, int mode, cudaStream_t s);
cudaError_t launch_mgs_tan(const Ctx& c, cudaStream_t s);
cudaError_t launch_energy_tan(const Ctx& c, cudaStream_t s);
cudaError_t launch_mixed_sum_tan(const Ctx& c, double* out, cudaStream_t s);
// reverse mode (adjoint_kernels.cu): see those kernels for the adjoint of each step piece
bool adjoint_fits(const Ctx& c);
cudaError_t prepare_adjoint_kernels(const Ctx& c);
cudaError_t adj_inv_overlap(const Ctx& c, const double* phi, double* Y, double* logO, double* theta,
                            const int* mask, cudaStream_t s);
cudaError_t adj_rbar(const Ctx& c, const double* logO_new, const double* logO_old, const int* still,
                     double* lwbar, double* rbar, cudaStream_t s);
cudaError_t adj_mask(const Ctx& c, double* pb, const int* still, cudaStream_t s);
cudaError_t adj_logdet(const Ctx& c, double* pb, const double* Y, const double* rbar, double sgn,
                       cudaStream_t s);
cudaError_t adj_taylor(const Ctx& c, const double* phi1, double* pbar, double* terms, double* Abar,
                       double* phi2, const int* mask, cudaStream_t s);
constexpr int kOuterSlices = 64;   // row slices of the Ebar outer product; part: [64][M][M]
cudaError_t adj_outer(const Ctx& c, const double* Xm, const double* Ym, const int* mask, double* part,
                      double* Ebar, cudaStream_t s);
cudaError_t adj_fields(const Ctx& c, const double* fields, const double* S, const double* rbar,
                       const double* lwbar, double* rbb, const int* mask, cudaStream_t s);
cudaError_t adj_overlap(const Ctx& c, const double* phi, const double* Y, const double* thb,
                        double* pb, const int* mask, cudaStream_t s);
cudaError_t adj_mgs(const Ctx& c, const double* Q, const double* phi3, double* pb, const int* alive,
                    cudaStream_t s);
cudaError_t adj_energy(const Ctx& c, const double* theta, const double* ebar, double* thb,
                       double* eloc, const int* mask, cudaStream_t s);
cudaError_t adj_meas_weights(const Ctx& c, double* ebar, double inv_meas, cudaStream_t s);
cudaError_t adj_meas_finish(const Ctx& c, const double* eloc, const double* ebar, double* lwbar,
                            double* e_acc, double n_meas, cudaStream_t s);
cudaError_t adj_theta_avg(const Ctx& c, const double* theta, const double* ebar, double* avg,
                          cudaStream_t s);
cudaError_t adj_h1bar(const Ctx& c, const double* Lx, double alpha, const double* avg, double* out,
                      cudaStream_t s);
cudaError_t place_block(double* Z, int ldz, int r0, int c0, const double* src, int M, double alpha,
                        cudaStream_t s);
cudaError_t take_block(const double* Z, int ldz, int r0, int c0, double* dst, int M, double alpha,
                       cudaStream_t s);
cudaError_t set_step(const Ctx& c, unsigned long long v, cudaStream_t s);
// preliminary equilibration scheme (pes.cu): comb per repeat into src / share (cum: Nw
// doubles of scratch), then gather the walkers through `scratch` ([2][Nw][N][M]) and set the
// combed weights; seeding of B's walkers and weights from A's
cudaError_t launch_comb(const Ctx& c, const double* u_dev, double* cum, int* src, double* share,
                        cudaStream_t s);
cudaError_t launch_apply_comb(const Ctx& c, const int* src, const double* share, double* scratch,
                              cudaStream_t s);
cudaError_t launch_seed_columns(const Ctx& A, const Ctx& B, cudaStream_t s);
cudaError_t launch_seed_weights(const Ctx& A, const Ctx& B, cudaStream_t s);
// out = L_exp(-dt K/2, scale * dir), the exponential's Frechet derivative (api.cu)
afqmc_status frechet_expm(Ctx* h, const double* dir, double scale, double* out, cudaStream_t s);
inline int pad64(int k) { return (k + 63) / 64 * 64; }

// OV_DET: overlap, log det and Theta of every determinant of a multi-determinant trial from
// src (or the current walkers when src is null), with no weight update and no walker killed
enum OverlapMode { OV_REFRESH = 0, OV_UPDATE = 1, OV_DET = 2 };
cudaError_t prepare_kernels(const Ctx& c);
cudaError_t launch_overlap(const Ctx& c, const double* src, int mode, cudaStream_t s,
                           int n_walkers = -1);
// multi-determinant trial (multidet.cu, FP64): log O_d and Theta_d of every determinant
// (walker_kernels.cu), the overlap update or refresh with the shares w_d, the force bias and
// the local energy as share-weighted sums over the determinants
cudaError_t launch_overlap_dets(const Ctx& c, const double* src, cudaStream_t s);
cudaError_t md_overlap(const Ctx& c, const double* src, int mode, cudaStream_t s);
cudaError_t md_force_bias(const Ctx& c, cudaStream_t s);
cudaError_t md_energy(const Ctx& c, cudaStream_t s);
cudaError_t launch_fields(const Ctx& c, const double* fields, cudaStream_t s);
cudaError_t launch_taylor(const Ctx& c, double* phi_io, cudaStream_t s);
cudaError_t launch_mgs(const Ctx& c, cudaStream_t s);
cudaError_t launch_energy(const Ctx& c, cudaStream_t s, int n_walkers = -1);
cudaError_t launch_mixed_sum(const Ctx& c, double* out, const int* slot, int slot_stride,
                             cudaStream_t s);
cudaError_t launch_step_advance(const Ctx& c, cudaStream_t s);

// setup helpers
cudaError_t launch_transpose(const double* in, double* out, int rows, int cols, cudaStream_t s);
cudaError_t launch_pack_Lt(const double* L, double* Lt, int M, int X, cudaStream_t s);
cudaError_t launch_rho_mf(const double* Ltil, const double* psi, double* rho, int X, int NM,
                          cudaStream_t s);
cudaError_t launch_build_K(const double* h1, const double* Q, const double* L, const double* rho,
                           double* K, int M, int X, double scale, cudaStream_t s);
cudaError_t launch_add_identity(double* A, int M, double a, cudaStream_t s);
cudaError_t launch_norm1(const double* A, int M, double* out, cudaStream_t s);
cudaError_t launch_permute_L(const double* L, double* Lp, int M, int X, cudaStream_t s);
cudaError_t launch_broadcast_walkers(const double* psi, double* phi, int Nw, int NM,
                                     cudaStream_t s);
cudaError_t launch_init_weights(double* w, int* alive, const double* w_in, int Nw,
                                cudaStream_t s);
cudaError_t launch_phi_layout(const double* in, double* out, int Nw, int M, int N, int to_internal,
                              cudaStream_t s);

}  // namespace afq
