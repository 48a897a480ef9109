// Reverse-mode derivative dE/dh1 of one run's mixed energy (FP64 phaseless path), with
// checkpointed recomputation.  The forward pass keeps the walker state (Phi, log O, w,
// alive) every K steps.  The reverse pass takes the segments last to first: it re-runs a
// segment from its checkpoint to tape the state before each of its steps, then walks the
// segment backwards, re-running each step once more from its taped state to recover that
// step's intermediates (force bias, A, Phi2, new overlaps) in the handle's own buffers
// before the adjoint kernels of adjoint_kernels.cu consume them.  All kernels are
// deterministic, so every recomputation reproduces the forward pass exactly.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

struct afqmc_ctx : afq::Ctx {};

namespace afq {
afqmc_status run_step(Ctx* h, const double* fields_t, cudaStream_t s);
afqmc_status pair_ortho(Ctx* h, cudaStream_t s);
}  // namespace afq

namespace {

using afq::Ctx;

// Device allocations of one call, released together after the stream has drained.
struct Arena {
  std::vector<void*> ptrs;
  bool ok = true;
  template <class T>
  T* get(size_t n) {
    if (!ok) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
};

struct State {
  double* phi = nullptr;   // [2][Nw][N][M]
  double* logO = nullptr;  // [2][Nw]
  double* w = nullptr;     // [2][Nw]
  int* alive = nullptr;    // [Nw]
};

State alloc_state(Arena& ar, const Ctx& c) {
  State st;
  st.phi = ar.get<double>(2 * (size_t)c.Nw * c.N * c.M);
  st.logO = ar.get<double>(2 * (size_t)c.Nw);
  st.w = ar.get<double>(2 * (size_t)c.Nw);
  st.alive = ar.get<int>((size_t)c.Nw);
  return st;
}

cudaError_t copy_state(const Ctx& c, State dst, State src, cudaStream_t s) {
  const size_t nphi = 2 * (size_t)c.Nw * c.N * c.M;
  cudaError_t e = cudaMemcpyAsync(dst.phi, src.phi, sizeof(double) * nphi, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst.logO, src.logO, sizeof(double) * 2 * c.Nw, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst.w, src.w, sizeof(double) * 2 * c.Nw, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst.alive, src.alive, sizeof(int) * c.Nw, cudaMemcpyDeviceToDevice, s);
  return e;
}

afqmc_status fail(Ctx* h, afqmc_status code, const std::string& msg) {
  h->err = msg;
  return code;
}

afqmc_status cfail(Ctx* h, const char* what, cudaError_t e) {
  return fail(h, AFQMC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define ADJ_CK(call)                                      \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cfail(h, #call, e_);    \
  } while (0)
#define ADJ_ST(call)                                      \
  do {                                                    \
    afqmc_status s_ = (call);                             \
    if (s_ != AFQMC_OK) return s_;                        \
  } while (0)

afqmc_status adjoint_body(Ctx* h, Arena& ar, int n_steps, const double* fields, int mgs_every,
                          int energy_every, int K, double* e_mixed, double* dE_dh1, cudaStream_t s) {
  const Ctx& c = *h;
  const int M = c.M, X = c.X, N = c.N, Nw = c.Nw, NM = N * M, MM = M * M;
  const int nu = c.n_up, nd = N - c.n_up, nn = nu * nu + nd * nd;
  const size_t nphi = 2 * (size_t)Nw * NM;
  const int64_t per = (int64_t)Nw * X;
  const int nseg = (n_steps + K - 1) / K;
  const int n_meas = n_steps / energy_every;
  const unsigned long long t0 = c.step;

  const double* fd = nullptr;
  if (fields) {
    if (on_device(fields)) {
      fd = fields;
    } else {
      double* staged = ar.get<double>((size_t)per * n_steps);
      if (!ar.ok) return fail(h, AFQMC_ERR_NOMEM, "cannot stage the fields");
      ADJ_CK(cudaMemcpyAsync(staged, fields, sizeof(double) * per * n_steps, cudaMemcpyHostToDevice, s));
      fd = staged;
    }
  }
  auto field_t = [&](int t) { return fd ? fd + per * t : nullptr; };
  auto mgs_at = [&](int t) { return mgs_every > 0 && (t + 1) % mgs_every == 0; };
  auto meas_at = [&](int t) { return (t + 1) % energy_every == 0; };

  std::vector<State> ck(nseg), tape(K);
  for (State& st : ck) st = alloc_state(ar, c);
  for (State& st : tape) st = alloc_state(ar, c);
  const State fin = alloc_state(ar, c);
  const State cur{h->phi, h->logO, h->w, h->alive};
  double* phibar = ar.get<double>(nphi);
  double* pbA = ar.get<double>(nphi);
  double* phi1 = ar.get<double>(nphi);
  double* phi3b = ar.get<double>(nphi);
  double* thb = ar.get<double>(nphi);
  double* terms = ar.get<double>(nphi * c.opt.taylor_order);
  double* Abar = ar.get<double>(2 * (size_t)Nw * MM);
  double* S = ar.get<double>(2 * (size_t)per);
  double* rbb = ar.get<double>(2 * (size_t)per);
  double* Y1 = ar.get<double>(2 * (size_t)Nw * nn);
  double* Y2 = ar.get<double>(2 * (size_t)Nw * nn);
  double* lwbar = ar.get<double>(Nw);
  double* rbar = ar.get<double>(2 * (size_t)Nw);
  int* still = ar.get<int>(Nw);
  double* logO_new = ar.get<double>(2 * (size_t)Nw);
  double* logO_tmp = ar.get<double>(2 * (size_t)Nw);
  double* ebar = ar.get<double>(Nw);
  double* eloc_r = ar.get<double>(Nw);
  double* e_acc = ar.get<double>(1);
  double* LtilT = ar.get<double>((size_t)NM * X);
  double* Ebar = ar.get<double>(MM);
  double* part = ar.get<double>((size_t)afq::kOuterSlices * MM);
  double* avg = ar.get<double>(NM);
  double* LE = ar.get<double>(MM);
  double* h1bar = ar.get<double>(MM);
  if (!ar.ok) return fail(h, AFQMC_ERR_NOMEM, "cannot allocate the adjoint's checkpoints and scratch");

  ADJ_CK(afq::prepare_adjoint_kernels(c));
  ADJ_CK(afq::launch_transpose(c.Ltil, LtilT, X, NM, s));   // [NM][X]
  ADJ_CK(cudaMemsetAsync(phibar, 0, sizeof(double) * nphi, s));
  ADJ_CK(cudaMemsetAsync(lwbar, 0, sizeof(double) * Nw, s));
  ADJ_CK(cudaMemsetAsync(Ebar, 0, sizeof(double) * MM, s));
  ADJ_CK(cudaMemsetAsync(avg, 0, sizeof(double) * NM, s));
  ADJ_CK(cudaMemsetAsync(e_acc, 0, sizeof(double), s));

  // ---- forward pass, checkpoint every K steps ----
  for (int t = 0; t < n_steps; ++t) {
    if (t % K == 0) ADJ_CK(copy_state(c, ck[t / K], cur, s));
    ADJ_ST(afq::run_step(h, field_t(t), s));
    if (mgs_at(t)) ADJ_ST(afq::pair_ortho(h, s));
  }
  ADJ_CK(copy_state(c, fin, cur, s));

  // ---- reverse pass ----
  const int cols = 2 * Nw * N;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int s0 = seg * K, s1 = std::min(n_steps, s0 + K);
    ADJ_CK(copy_state(c, cur, ck[seg], s));
    ADJ_CK(afq::set_step(c, t0 + s0, s));
    ADJ_CK(afq::launch_overlap(c, nullptr, afq::OV_REFRESH, s));
    for (int t = s0; t < s1; ++t) {
      ADJ_CK(copy_state(c, tape[t - s0], cur, s));
      ADJ_ST(afq::run_step(h, field_t(t), s));
      if (mgs_at(t)) ADJ_ST(afq::pair_ortho(h, s));
    }
    for (int t = s1 - 1; t >= s0; --t) {
      const State tp = tape[t - s0];
      // recompute step t: rhobar, U, A, aux, Phi2 (in phi2), Phi3, new log O, w, alive
      ADJ_CK(copy_state(c, cur, tp, s));
      ADJ_CK(afq::set_step(c, t0 + t, s));
      ADJ_CK(afq::launch_overlap(c, nullptr, afq::OV_REFRESH, s));
      ADJ_ST(afq::run_step(h, field_t(t), s));
      ADJ_CK(cudaMemcpyAsync(still, c.alive, sizeof(int) * Nw, cudaMemcpyDeviceToDevice, s));
      const double* phi3 = c.phi;
      if (mgs_at(t)) {
        ADJ_CK(cudaMemcpyAsync(phi3b, c.phi, sizeof(double) * nphi, cudaMemcpyDeviceToDevice, s));
        ADJ_ST(afq::pair_ortho(h, s));
        phi3 = phi3b;
      }
      // measurement after step t: E_m = sum w Re E_L / sum w on the (orthonormalised) walkers
      if (meas_at(t)) {
        ADJ_CK(afq::adj_meas_weights(c, ebar, 1.0 / n_meas, s));
        ADJ_CK(afq::adj_energy(c, c.theta, ebar, thb, eloc_r, c.alive, s));
        ADJ_CK(afq::adj_meas_finish(c, eloc_r, ebar, lwbar, e_acc, (double)n_meas, s));
        ADJ_CK(afq::adj_theta_avg(c, c.theta, ebar, avg, s));
        ADJ_CK(afq::adj_inv_overlap(c, c.phi, Y1, logO_tmp, nullptr, c.alive, s));
        ADJ_CK(afq::adj_overlap(c, c.phi, Y1, thb, phibar, c.alive, s));
      }
      if (mgs_at(t)) ADJ_CK(afq::adj_mgs(c, c.phi, phi3b, phibar, c.alive, s));
      // step t backwards
      ADJ_CK(afq::adj_mask(c, phibar, still, s));
      ADJ_CK(afq::adj_inv_overlap(c, phi3, Y1, logO_new, nullptr, still, s));
      ADJ_CK(afq::adj_rbar(c, logO_new, tp.logO, still, lwbar, rbar, s));
      ADJ_CK(afq::adj_logdet(c, phibar, Y1, rbar, 1.0, s));
      ADJ_CK(afq::adj_outer(c, phibar, c.phi2, still, part, Ebar, s));
      ADJ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, c.expK, M, 0, phibar, M, 0, 0.0, pbA, M, 0, 1, s,
                              afq::GEMM_ONEBODY));
      ADJ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, c.expK, M, 0, tp.phi, M, 0, 0.0, phi1, M, 0, 1, s,
                              afq::GEMM_ONEBODY));
      ADJ_CK(afq::adj_taylor(c, phi1, pbA, terms, Abar, c.phi2, still, s));
      ADJ_CK(afq::adj_outer(c, pbA, tp.phi, still, part, Ebar, s));
      ADJ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, c.expK, M, 0, pbA, M, 0, 0.0, phibar, M, 0, 1, s,
                              afq::GEMM_ONEBODY));
      // S[(p,w)][g] = sum_ij L_g,ij Abar[(p,w)][ij]
      ADJ_CK(afq::gemm_tn_f64(X, 2 * Nw, MM, 1.0, c.L, MM, 0, Abar, MM, 0, 0.0, S, X, 0, 1, s));
      ADJ_CK(afq::set_step(c, t0 + t, s));
      ADJ_CK(afq::adj_fields(c, field_t(t), S, rbar, lwbar, rbb, still, s));
      // Thetabar[(p,w)][(n,i)] = sum_g rhobarbar[(p,w)][g] Ltil[g][(n,i)]
      ADJ_CK(afq::gemm_tn_f64(NM, 2 * Nw, X, 1.0, LtilT, X, 0, rbb, X, 0, 0.0, thb, NM, 0, 1, s));
      ADJ_CK(afq::adj_inv_overlap(c, tp.phi, Y2, logO_tmp, nullptr, still, s));
      ADJ_CK(afq::adj_overlap(c, tp.phi, Y2, thb, phibar, still, s));
      ADJ_CK(afq::adj_logdet(c, phibar, Y2, rbar, -1.0, s));
    }
  }
  // the handle ends after the forward run
  ADJ_CK(copy_state(c, cur, fin, s));
  ADJ_CK(afq::set_step(c, t0 + n_steps, s));
  ADJ_CK(afq::launch_overlap(c, nullptr, afq::OV_REFRESH, s));
  h->step = t0 + n_steps;
  // h1bar = -dt/2 L_exp(B, Ebar) + sum_meas sum_k ebar_k Re G_k^T
  ADJ_ST(afq::frechet_expm(h, Ebar, 1.0, LE, s));
  ADJ_CK(afq::adj_h1bar(c, LE, -0.5 * c.opt.dt, avg, h1bar, s));
  double E = 0;
  ADJ_CK(cudaMemcpyAsync(&E, e_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (dE_dh1) ADJ_CK(cudaMemcpyAsync(dE_dh1, h1bar, sizeof(double) * MM, cudaMemcpyDefault, s));
  ADJ_CK(cudaStreamSynchronize(s));
  if (e_mixed) *e_mixed = E;
  if (!std::isfinite(E)) return fail(h, AFQMC_ERR_NUMERIC, "no live walker at a measurement");
  return AFQMC_OK;
}

}  // namespace

extern "C" afqmc_status afqmc_adjoint_run(afqmc_handle h, int n_steps, const double* fields,
                                          int mgs_every, int energy_every, int checkpoint,
                                          double* e_mixed, double* dE_dh1, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  if (h->tangent_on) return fail(h, AFQMC_ERR_STATE, "tangent mode is on");
  if (h->opt.precision != AFQMC_FP64 || h->opt.mode != AFQMC_PHASELESS)
    return fail(h, AFQMC_ERR_ARG, "the adjoint needs the FP64 phaseless path");
  if (h->R != 1) return fail(h, AFQMC_ERR_ARG, "the adjoint needs n_repeats == 1");
  if (h->n_det > 0) return fail(h, AFQMC_ERR_ARG, "the adjoint needs a single-determinant trial");
  if (n_steps < 1) return fail(h, AFQMC_ERR_ARG, "n_steps must be >= 1");
  if (energy_every < 1 || energy_every > n_steps)
    return fail(h, AFQMC_ERR_ARG, "energy_every must be in [1, n_steps]");
  if (mgs_every < 0) return fail(h, AFQMC_ERR_ARG, "mgs_every must be >= 0");
  if (checkpoint < 1) return fail(h, AFQMC_ERR_ARG, "checkpoint must be >= 1");
  if (!afq::adjoint_fits(*h)) return fail(h, AFQMC_ERR_ARG, "adjoint kernels exceed shared memory");
  const int K = std::min(checkpoint, n_steps);
  afqmc_status st;
  {
    Arena ar;
    st = adjoint_body(h, ar, n_steps, fields, mgs_every, energy_every, K, e_mixed, dE_dh1, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == AFQMC_OK && e != cudaSuccess) st = cfail(h, "afqmc_adjoint_run", e);
  }
  return st;
}
