// C-ABI entry points: argument checking, device memory, the setup sequence, the
// per-step kernel schedule, and the CUDA-graph driven correlated pair run.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

struct afqmc_ctx : afq::Ctx {};

namespace {

using afq::Ctx;

afqmc_status set_err(Ctx* h, afqmc_status code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

afqmc_status cuda_fail(Ctx* h, const char* what, cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return set_err(h, AFQMC_ERR_CUDA, buf);
}

#define AFQ_CK(call)                                  \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, #call, e_); \
  } while (0)

template <class T>
afqmc_status dalloc(Ctx* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(h, AFQMC_ERR_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  return AFQMC_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_ctx(Ctx* h) {
  afq::destroy_pair_cache(h);
  double* bufs[] = {h->h1, h->L, h->Lt, h->Ltil, h->htil, h->psi, h->expK, h->rho_mf, h->phi,
                    h->phi2, h->theta, h->logO, h->w, h->rhobar, h->U, h->Avhs, h->aux,
                    h->eloc, h->esum};
  for (double* b : bufs)
    if (b) cudaFree(b);
  if (h->alive) cudaFree(h->alive);
  if (h->d_step) cudaFree(h->d_step);
  if (h->d_flags) cudaFree(h->d_flags);
  for (afq::TcOperand* op : {h->tc_L, h->tc_Ltri, h->tc_Ltil, h->tc_U, h->tc_Theta})
    if (op) {
      if (op->hi) cudaFree(op->hi);
      if (op->lo) cudaFree(op->lo);
      delete op;
    }
  if (h->ovdet) cudaFree(h->ovdet);
  if (h->emI_pk) cudaFree(h->emI_pk);
  for (__nv_bfloat16* b : {h->tcl_ahi, h->tcl_alo, h->tcl_ehi, h->tcl_elo})
    if (b) cudaFree(b);
  delete[] h->tcl_maps;
  h->tcl_maps = nullptr;
  for (double* b : {h->Bneg, h->dexpK, h->htilP, h->dphi, h->dphi2, h->dtheta, h->drhobar, h->dU,
                    h->dAvhs, h->dlogO, h->dlogw, h->daux, h->deloc, h->desum})
    if (b) cudaFree(b);
  for (float* b : {h->Avhs32, h->phi32, h->expK32, h->Ltil32, h->theta32, h->LtT, h->psi32h, h->psi32l,
                   h->rhobar32, h->rho_mf32})
    if (b) cudaFree(b);
  if (h->d_tc_err) cudaFree(h->d_tc_err);
  for (double* b : {h->md_coef, h->md_psi, h->md_Ltil, h->md_htil, h->md_logO, h->md_theta,
                    h->md_share, h->md_rhobar, h->md_eloc})
    if (b) cudaFree(b);
  if (h->etc) {
    for (afq::TcOperand* op : {h->etc->A, h->etc->B})
      if (op) {
        if (op->hi) cudaFree(op->hi);
        if (op->lo) cudaFree(op->lo);
        delete op;
      }
    if (h->etc->part) cudaFree(h->etc->part);
    if (h->etc->trs) cudaFree(h->etc->trs);
    if (h->etc->hh) cudaFree(h->etc->hh);
    if (h->etc->hl) cudaFree(h->etc->hl);
    delete h->etc;
    h->etc = nullptr;
  }
}

afqmc_status overlap_launch(Ctx* h, const double* src, int mode, cudaStream_t s,
                            const float* src32 = nullptr);

// Allocate a split operand of `rows` logical rows (padded to whole TMA boxes, zero-filled)
// and K = Kp columns, and encode its tensor maps.
afqmc_status make_operand(Ctx* h, afq::TcOperand** out, int rows, int K, cudaStream_t s) {
  auto* op = new afq::TcOperand();
  *out = op;
  const int rp = afq::tc_pad_rows(rows), Kp = afq::pad64(K);
  const size_t bytes = 2 * (size_t)rp * Kp;
  if (dalloc(h, &op->hi, bytes / 2) != AFQMC_OK || dalloc(h, &op->lo, bytes / 2) != AFQMC_OK)
    return AFQMC_ERR_NOMEM;
  AFQ_CK(cudaMemsetAsync(op->hi, 0, bytes, s));
  AFQ_CK(cudaMemsetAsync(op->lo, 0, bytes, s));
  AFQ_CK(afq::tc_make_operand(*op, op->hi, op->lo, rp, Kp, 128));
  return AFQMC_OK;
}

// Split-precision operands and FP32 copies, built from the FP64 setup results.
afqmc_status setup_mixed(Ctx* h, cudaStream_t s) {
  const int M = h->M, X = h->X, N = h->N, Nw = h->Nw;
  const int64_t NM = (int64_t)N * M, MM = (int64_t)M * M;
  afqmc_status st;
  AFQ_CK(afq::prepare_tc_kernels());
  AFQ_CK(afq::prepare_mixed_kernels(*h));
  AFQ_CK(afq::prepare_mixed_kernels2(*h));
  AFQ_CK(afq::prepare_fast_walker_kernels(*h));
  AFQ_CK(afq::prepare_propagate_f32());
  AFQ_CK(afq::prepare_propagate_tc());
  AFQ_CK(afq::prepare_propagate_tcl());
  if ((st = make_operand(h, &h->tc_L, (int)MM, X, s)) != AFQMC_OK) return st;
  if ((st = make_operand(h, &h->tc_Ltil, X, (int)NM, s)) != AFQMC_OK) return st;
  if ((st = make_operand(h, &h->tc_U, 2 * Nw, X, s)) != AFQMC_OK) return st;
  if ((st = make_operand(h, &h->tc_Theta, 2 * Nw, (int)NM, s)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->Avhs32, 2 * (size_t)Nw * MM)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->phi32, 2 * (size_t)Nw * NM)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->expK32, (size_t)MM)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->Ltil32, (size_t)X * NM)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->d_tc_err, 1)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->theta32, 2 * (size_t)Nw * NM)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->LtT, (size_t)afq::LtT_size(*h))) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->psi32h, (size_t)NM)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->psi32l, (size_t)NM)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->ovdet, 8 * (size_t)Nw)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->rhobar32, 2 * (size_t)Nw * X)) != AFQMC_OK) return st;
  if ((st = dalloc(h, &h->rho_mf32, (size_t)X)) != AFQMC_OK) return st;
  AFQ_CK(cudaMemsetAsync(h->d_tc_err, 0, sizeof(int), s));
  // L as rows ij with g contiguous: transpose [X][M*M] -> [M*M][X] through phi2 (large enough
  // only when 2*Nw*N*M >= X*M*M; otherwise a temporary)
  double* tmp = nullptr;
  const bool own = 2 * (int64_t)Nw * NM < (int64_t)X * MM;
  if (own) {
    if ((st = dalloc(h, &tmp, (size_t)X * MM)) != AFQMC_OK) return st;
  } else {
    tmp = h->phi2;
  }
  cudaError_t e = afq::launch_transpose(h->L, tmp, X, (int)MM, s);
  if (e == cudaSuccess) e = afq::split_bf16(tmp, X, (int)MM, X, h->tc_L->Kp, h->tc_L->hi, h->tc_L->lo, s);
  if (e == cudaSuccess && afq::propagate_tcl_ok(*h) &&
      afq::tc_persistent_ok(afq::vhs_tri_rows(M), 2 * Nw, h->tc_U->rows)) {
    // the lower-triangle blocks of the V_HS rows, for the split output the large-M
    // tensor-core propagator reads (V_HS is symmetric: the kernel writes the mirror half)
    if ((st = make_operand(h, &h->tc_Ltri, afq::vhs_tri_rows(M), X, s)) != AFQMC_OK) {
      if (own) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
      }
      return st;
    }
    e = afq::split_bf16_tri(tmp, X, M, X, h->tc_Ltri->Kp, h->tc_Ltri->hi, h->tc_Ltri->lo, s);
  }
  if (e == cudaSuccess) e = afq::split_bf16(h->Ltil, NM, X, (int)NM, h->tc_Ltil->Kp, h->tc_Ltil->hi, h->tc_Ltil->lo, s);
  if (e == cudaSuccess) e = afq::to_float(h->expK, h->expK32, MM, s);
  if (e == cudaSuccess) e = afq::to_float(h->Ltil, h->Ltil32, (int64_t)X * NM, s);
  if (e == cudaSuccess) e = afq::build_LtT(*h, h->LtT, s);
  if (e == cudaSuccess) e = afq::split_f32(h->psi, h->psi32h, h->psi32l, NM, s);
  if (e == cudaSuccess) e = afq::to_float(h->rho_mf, h->rho_mf32, X, s);
  if (e == cudaSuccess && afq::propagate_tc_ok(*h)) {
    if (dalloc(h, &h->emI_pk, 64 * 64) != AFQMC_OK) return AFQMC_ERR_NOMEM;
    e = afq::pack_propagate_tc(*h, h->emI_pk, s);
  }
  if (e == cudaSuccess && afq::propagate_tcl_ok(*h)) {
    // V_HS in split form for the large-M tensor-core propagator (zero until the first step)
    const size_t na = 2 * (size_t)Nw * M * afq::propagate_tcl_mp(M), ne = (size_t)M * afq::propagate_tcl_mp(M);
    if (dalloc(h, &h->tcl_ahi, na) != AFQMC_OK || dalloc(h, &h->tcl_alo, na) != AFQMC_OK ||
        dalloc(h, &h->tcl_ehi, ne) != AFQMC_OK || dalloc(h, &h->tcl_elo, ne) != AFQMC_OK) {
      if (own) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
      }
      return AFQMC_ERR_NOMEM;
    }
    e = cudaMemsetAsync(h->tcl_ahi, 0, na * 2, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->tcl_alo, 0, na * 2, s);
    if (e == cudaSuccess) e = afq::setup_propagate_tcl(*h, s);
  }
  // Theta of the current walkers in FP32 and as the split force-bias operand
  if (e == cudaSuccess && overlap_launch(h, nullptr, afq::OV_REFRESH, s) != AFQMC_OK)
    e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Avhs32, 0, sizeof(float) * 2 * (size_t)Nw * MM, s);
  if (e == cudaSuccess && afq::energy_tc_np(*h) > 0) {
    // tensor-core local energy: operands in the padded (g, n') / (w, re/im, n') row layouts
    const int np = afq::energy_tc_np(*h);
    e = afq::prepare_energy_tc_kernels();
    if (e == cudaSuccess) {
      h->etc = new afq::EnergyTc();
      h->etc->NP = np;
      int ra = 0, rb = 0;
      afq::energy_tc_sizes(*h, np, &ra, &rb, &h->etc->Kp, &h->etc->RT, &h->etc->NwP);
      h->etc->A = new afq::TcOperand();
      h->etc->B = new afq::TcOperand();
      h->etc->A->rows = ra;
      h->etc->B->rows = rb;
      const size_t ka = (size_t)ra * h->etc->Kp, kb = (size_t)rb * h->etc->Kp;
      if (dalloc(h, &h->etc->A->hi, ka) != AFQMC_OK || dalloc(h, &h->etc->A->lo, ka) != AFQMC_OK ||
          dalloc(h, &h->etc->B->hi, kb) != AFQMC_OK || dalloc(h, &h->etc->B->lo, kb) != AFQMC_OK ||
          dalloc(h, &h->etc->part, 2 * (size_t)h->etc->RT * h->etc->NwP) != AFQMC_OK ||
          dalloc(h, &h->etc->hh, (size_t)NM) != AFQMC_OK || dalloc(h, &h->etc->hl, (size_t)NM) != AFQMC_OK ||
          (afq::energy_tc_spin(*h) &&
           dalloc(h, &h->etc->trs, 2 * 2 * (size_t)Nw * X) != AFQMC_OK)) {
        if (own) {
          cudaStreamSynchronize(s);
          cudaFree(tmp);
        }
        return AFQMC_ERR_NOMEM;
      }
      e = afq::energy_tc_init(*h, *h->etc, s);
    }
  }
  if (e == cudaSuccess && h->opt.autotune)
    e = afq::autotune_mixed(*h, h->opt.autotune_cache, s);
  if (own) {
    cudaStreamSynchronize(s);
    cudaFree(tmp);
  }
  AFQ_CK(e);
  return AFQMC_OK;
}

// One split-precision step: tensor-core contractions, FP32 propagator, FP64 overlaps.
afqmc_status step_launch_mixed(Ctx* h, const double* fields_t, cudaStream_t s) {
  const int X = h->X, Nw = h->Nw;
  if (h->opt.mode == AFQMC_PHASELESS) {
    // the Theta operand was written by the last overlap kernel
    AFQ_CK(afq::gemm_bf16x3(*h->tc_Ltil, *h->tc_Theta, X, 2 * Nw, 1.0f, h->rhobar32, X,
                            h->d_tc_err, s));
  }
  AFQ_CK(afq::launch_fields_mixed(*h, fields_t, s));
  const int pv = afq::propagation_variant(*h);
  AFQ_CK(afq::vhs_launch(*h, pv, s));
  // Phi' = e^{-dt K/2} e^A e^{-dt K/2} Phi into theta (FP64; the tensor-core propagators write
  // the live walkers in place) and, variants 2 to 4, into phi32 (FP32)
  double* pout = pv >= 3 ? h->phi : h->theta;
  AFQ_CK(afq::launch_propagation(*h, pv, pout, h->phi32, s));
  afqmc_status os = overlap_launch(h, pout, afq::OV_UPDATE, s, pv >= 2 ? h->phi32 : nullptr);
  if (os != AFQMC_OK) return os;
  AFQ_CK(afq::launch_step_advance(*h, s));
  return AFQMC_OK;
}

afqmc_status energy_launch(Ctx* h, cudaStream_t s) {
  if (h->opt.precision == AFQMC_BF16X3) {
    if (h->etc && h->tune_energy_wb <= 0) {
      AFQ_CK(afq::launch_energy_tc(*h, s));
    } else {
      AFQ_CK(afq::launch_energy_tiled(*h, h->theta32, h->LtT, s));
    }
  } else if (h->n_det > 0) {
    AFQ_CK(afq::md_energy(*h, s));
  } else {
    AFQ_CK(afq::launch_energy(*h, s));
  }
  return AFQMC_OK;
}

// After a synchronisation: report an expired tensor-core wait.
afqmc_status check_tc(Ctx* h) {
  if (!h->d_tc_err) return AFQMC_OK;
  int v = 0;
  AFQ_CK(cudaMemcpy(&v, h->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) return set_err(h, AFQMC_ERR_TIMEOUT, "a tensor-core kernel's bounded wait expired");
  return AFQMC_OK;
}

afqmc_status step_launch_mixed(Ctx* h, const double* fields_t, cudaStream_t s);

// One FP64 step of the walkers and their tangents along h1 -> h1 + lambda P.
afqmc_status step_launch_tangent(Ctx* h, const double* fields_t, cudaStream_t s) {
  const int M = h->M, X = h->X, N = h->N, Nw = h->Nw;
  const int64_t NM = (int64_t)N * M;
  AFQ_CK(afq::gemm_tn_f64(X, 2 * Nw, (int)NM, 1.0, h->Ltil, NM, 0, h->theta, NM, 0, 0.0,
                          h->rhobar, X, 0, 1, s, afq::GEMM_FORCE_BIAS));
  AFQ_CK(afq::gemm_tn_f64(X, 2 * Nw, (int)NM, 1.0, h->Ltil, NM, 0, h->dtheta, NM, 0, 0.0,
                          h->drhobar, X, 0, 1, s, afq::GEMM_FORCE_BIAS));
  AFQ_CK(afq::launch_fields_tan(*h, fields_t, s));
  AFQ_CK(afq::gemm_tn_f64((int)h->P, 2 * Nw, X, 1.0, h->Lt, X, 0, h->U, X, 0, 0.0, h->Avhs,
                          h->P, 0, 1, s, afq::GEMM_VHS));
  AFQ_CK(afq::gemm_tn_f64((int)h->P, 2 * Nw, X, 1.0, h->Lt, X, 0, h->dU, X, 0, 0.0, h->dAvhs,
                          h->P, 0, 1, s, afq::GEMM_VHS));
  const int cols = 2 * Nw * N;
  AFQ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, h->expK, M, 0, h->phi, M, 0, 0.0, h->phi2, M, 0, 1, s,
                          afq::GEMM_ONEBODY));
  AFQ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, h->dexpK, M, 0, h->phi, M, 0, 0.0, h->dphi2, M, 0, 1, s,
                          afq::GEMM_ONEBODY));
  AFQ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, h->expK, M, 0, h->dphi, M, 0, 1.0, h->dphi2, M, 0, 1, s,
                          afq::GEMM_ONEBODY));
  AFQ_CK(afq::launch_taylor_tan(*h, s));
  AFQ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, h->expK, M, 0, h->phi2, M, 0, 0.0, h->theta, M, 0, 1, s,
                          afq::GEMM_ONEBODY));
  AFQ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, h->dexpK, M, 0, h->phi2, M, 0, 0.0, h->dtheta, M, 0, 1, s,
                          afq::GEMM_ONEBODY));
  AFQ_CK(afq::gemm_tn_f64(M, cols, M, 1.0, h->expK, M, 0, h->dphi2, M, 0, 1.0, h->dtheta, M, 0, 1, s,
                          afq::GEMM_ONEBODY));
  AFQ_CK(afq::launch_overlap_tan(*h, afq::OV_UPDATE, s));
  AFQ_CK(afq::launch_step_advance(*h, s));
  return AFQMC_OK;
}

// One propagation step of every walker of system h (Eqs. 3-5, 8-9, 11, hybrid weight).
afqmc_status step_launch(Ctx* h, const double* fields_t, cudaStream_t s) {
  if (h->tangent_on) return step_launch_tangent(h, fields_t, s);
  if (h->opt.precision == AFQMC_BF16X3) return step_launch_mixed(h, fields_t, s);
  const int M = h->M, X = h->X, N = h->N, Nw = h->Nw;
  const int64_t NM = (int64_t)N * M;
  if (h->opt.mode == AFQMC_PHASELESS) {
    // rhobar[(p,w)][g] = sum_(n,i) Ltil[g][(n,i)] Theta[(p,w)][(n,i)]       (Eq. 9); a
    // multi-determinant trial sums the determinants' contractions with their shares
    if (h->n_det > 0) {
      AFQ_CK(afq::md_force_bias(*h, s));
    } else {
      AFQ_CK(afq::gemm_tn_f64(X, 2 * Nw, (int)NM, 1.0, h->Ltil, NM, 0, h->theta, NM, 0, 0.0,
                              h->rhobar, X, 0, 1, s, afq::GEMM_FORCE_BIAS));
    }
  }
  AFQ_CK(afq::launch_fields(*h, fields_t, s));
  // packed A[(p,w)][ij] = sum_g Lt[ij][g] U[(p,w)][g]                         (Eq. 11)
  AFQ_CK(afq::gemm_tn_f64((int)h->P, 2 * Nw, X, 1.0, h->Lt, X, 0, h->U, X, 0, 0.0, h->Avhs,
                          h->P, 0, 1, s, afq::GEMM_VHS));
  // e^{-dt K/2} on every column of every walker
  AFQ_CK(afq::gemm_tn_f64(M, 2 * Nw * N, M, 1.0, h->expK, M, 0, h->phi, M, 0, 0.0, h->phi2, M,
                          0, 1, s, afq::GEMM_ONEBODY));
  AFQ_CK(afq::launch_taylor(*h, h->phi2, s));
  AFQ_CK(afq::gemm_tn_f64(M, 2 * Nw * N, M, 1.0, h->expK, M, 0, h->phi2, M, 0, 0.0, h->theta,
                          M, 0, 1, s, afq::GEMM_ONEBODY));
  // new overlaps, Theta, ratio, phase, weight; live walkers take the new determinant
  afqmc_status os = overlap_launch(h, h->theta, afq::OV_UPDATE, s);
  if (os != AFQMC_OK) return os;
  AFQ_CK(afq::launch_step_advance(*h, s));
  return AFQMC_OK;
}

// Overlap / Theta / weight kernel: the warp-synchronous variant in split-precision mode.
afqmc_status overlap_launch(Ctx* h, const double* src, int mode, cudaStream_t s,
                            const float* src32) {
  if (h->n_det > 0) {
    AFQ_CK(afq::md_overlap(*h, src, mode, s));
    return AFQMC_OK;
  }
  if (h->theta32 && h->tc_Theta && afq::fast_walker_kernels_ok(*h)) {
    AFQ_CK(afq::launch_overlap_fast(*h, src, mode, s, src32));
  } else {
    AFQ_CK(afq::launch_overlap(*h, src, mode, s));
  }
  return AFQMC_OK;
}

afqmc_status ortho_launch(Ctx* h, cudaStream_t s) {
  if (h->tangent_on) {
    AFQ_CK(afq::launch_mgs_tan(*h, s));
    AFQ_CK(afq::launch_overlap_tan(*h, afq::OV_REFRESH, s));
    return AFQMC_OK;
  }
  if (h->theta32 && h->tc_Theta && afq::fast_walker_kernels_ok(*h)) {
    // Gram-Schmidt is Phi -> Phi R^{-1}: Theta is unchanged and log O drops by log det R, so the
    // kernel updates log O from its column norms and no overlap recomputation follows
    AFQ_CK(afq::launch_mgs_warp(*h, s, true));
    return AFQMC_OK;
  }
  if (h->theta32 && afq::fast_walker_kernels_ok(*h)) {
    AFQ_CK(afq::launch_mgs_warp(*h, s));
  } else {
    AFQ_CK(afq::launch_mgs(*h, s));
  }
  return overlap_launch(h, nullptr, afq::OV_REFRESH, s);
}

afqmc_status check_opts(const afqmc_options* o, std::string& why) {
  if (!o) { why = "options is NULL"; return AFQMC_ERR_ARG; }
  if (!(o->dt > 0.0) || !std::isfinite(o->dt)) { why = "dt must be > 0"; return AFQMC_ERR_ARG; }
  if (o->n_walkers < 1) { why = "n_walkers must be >= 1"; return AFQMC_ERR_ARG; }
  if (o->taylor_order < 1 || o->taylor_order > 64) { why = "taylor_order must be in [1, 64]"; return AFQMC_ERR_ARG; }
  if (o->precision != AFQMC_FP64 && o->precision != AFQMC_BF16X3) { why = "unsupported precision"; return AFQMC_ERR_ARG; }
  if (o->mode != AFQMC_PHASELESS && o->mode != AFQMC_FREE) { why = "unknown mode"; return AFQMC_ERR_ARG; }
  if (o->n_repeats < 1 || o->n_repeats > o->n_walkers) { why = "n_repeats must be in [1, n_walkers]"; return AFQMC_ERR_ARG; }
  if (!std::isfinite(o->fb_cap)) { why = "fb_cap must be finite"; return AFQMC_ERR_ARG; }
  if (o->walker_offset < 0 || o->walker_offset + (int64_t)o->n_walkers > ((int64_t)1 << 32)) {
    why = "walker_offset out of range";
    return AFQMC_ERR_ARG;
  }
  if (o->independent_fields != 0 && o->independent_fields != 1) {
    why = "independent_fields must be 0 or 1";
    return AFQMC_ERR_ARG;
  }
  return AFQMC_OK;
}

}  // namespace

namespace afq {
afqmc_status pair_step(Ctx* h, cudaStream_t s) { return step_launch(h, nullptr, s); }
afqmc_status run_step(Ctx* h, const double* fields_t, cudaStream_t s) { return step_launch(h, fields_t, s); }
afqmc_status pair_ortho(Ctx* h, cudaStream_t s) { return ortho_launch(h, s); }
afqmc_status pair_energy(Ctx* h, cudaStream_t s) { return energy_launch(h, s); }
afqmc_status pair_check(Ctx* h) { return check_tc(h); }
}  // namespace afq

extern "C" {

void afqmc_default_options(afqmc_options* o) {
  if (!o) return;
  o->dt = 0.01;
  o->n_walkers = 128;
  o->taylor_order = 6;
  o->precision = AFQMC_FP64;
  o->mode = AFQMC_PHASELESS;
  o->n_repeats = 1;
  o->seed = 1;
  o->fb_cap = 1.0;
  o->walker_offset = 0;
  o->autotune = 1;
  o->autotune_cache = nullptr;
  o->independent_fields = 0;
}

const char* afqmc_status_string(afqmc_status s) {
  switch (s) {
    case AFQMC_OK: return "ok";
    case AFQMC_ERR_ARG: return "invalid argument";
    case AFQMC_ERR_CUDA: return "CUDA error";
    case AFQMC_ERR_NUMERIC: return "numerical failure";
    case AFQMC_ERR_STATE: return "invalid state";
    case AFQMC_ERR_TIMEOUT: return "device wait timed out";
    case AFQMC_ERR_NOMEM: return "out of device memory";
  }
  return "unknown status";
}

const char* afqmc_last_error(afqmc_handle h) { return h ? h->err.c_str() : ""; }

afqmc_status afqmc_setup(afqmc_handle* out, const double* h1_in, const double* L_in,
                         const double* trial_in, int M, int X, int n_up, int n_dn,
                         const afqmc_options* opt, cudaStream_t s) {
  if (!out) return AFQMC_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (check_opts(opt, why) != AFQMC_OK) return AFQMC_ERR_ARG;
  if (!h1_in || !L_in || !trial_in) return AFQMC_ERR_ARG;
  const int N = n_up + n_dn;
  if (M < 1 || X < 1 || n_up < 0 || n_dn < 0 || N < 1 || n_up > M || n_dn > M || n_up > 32 ||
      n_dn > 32 || (int64_t)N * M > 4096)
    return AFQMC_ERR_ARG;
  if ((int64_t)opt->n_walkers * N * M * 2 > (int64_t)1 << 40) return AFQMC_ERR_ARG;

  afqmc_ctx* h = new afqmc_ctx();
  h->M = M; h->X = X; h->n_up = n_up; h->n_dn = n_dn; h->N = N;
  h->Nw = opt->n_walkers; h->R = opt->n_repeats; h->opt = *opt;
  h->opt.autotune_cache = nullptr;   // used only inside setup (below), never kept
  h->P = afq::packed_size(M);
  h->sqrt_dt = std::sqrt(opt->dt);
  cudaGetDevice(&h->device);
  {
    static std::atomic<uint64_t> next_uid{0};
    h->uid = ++next_uid;
  }
  const int64_t NM = (int64_t)N * M, Nw = h->Nw;
  afqmc_status st = AFQMC_OK;
#define AFQ_ALLOC(p, n) \
  if ((st = dalloc(h, &(p), (size_t)(n))) != AFQMC_OK) { free_ctx(h); delete h; return st; }
  AFQ_ALLOC(h->h1, (int64_t)M * M);
  AFQ_ALLOC(h->L, (int64_t)X * M * M);
  AFQ_ALLOC(h->Lt, h->P * X);
  AFQ_ALLOC(h->Ltil, (int64_t)X * NM);
  AFQ_ALLOC(h->htil, NM);
  AFQ_ALLOC(h->psi, NM);
  AFQ_ALLOC(h->expK, (int64_t)M * M);
  AFQ_ALLOC(h->Bneg, (int64_t)M * M);
  AFQ_ALLOC(h->rho_mf, X);
  AFQ_ALLOC(h->phi, 2 * Nw * NM);
  AFQ_ALLOC(h->phi2, 2 * Nw * NM);
  AFQ_ALLOC(h->theta, 2 * Nw * NM);
  AFQ_ALLOC(h->logO, 2 * Nw);
  AFQ_ALLOC(h->w, 2 * Nw);
  AFQ_ALLOC(h->alive, Nw);
  AFQ_ALLOC(h->rhobar, 2 * Nw * X);
  AFQ_ALLOC(h->U, 2 * Nw * X);
  AFQ_ALLOC(h->Avhs, 2 * Nw * h->P);
  AFQ_ALLOC(h->aux, 4 * Nw);
  AFQ_ALLOC(h->eloc, 2 * Nw);
  AFQ_ALLOC(h->esum, 4 * (int64_t)h->R);
  AFQ_ALLOC(h->d_step, 1);
  AFQ_ALLOC(h->d_flags, 4);
#undef AFQ_ALLOC
  // scratch for the setup only
  double *tmp = nullptr, *Q = nullptr, *Kb = nullptr, *E0 = nullptr, *E1 = nullptr, *dnorm = nullptr;
  auto cleanup_tmp = [&]() {
    for (double* p : {tmp, Q, Kb, E0, E1, dnorm})
      if (p) cudaFree(p);
  };
  auto bail = [&](afqmc_status code) {
    cleanup_tmp();
    std::string msg = h->err;
    free_ctx(h);
    delete h;
    return code;
  };
  if (dalloc(h, &tmp, std::max<int64_t>((int64_t)X * M * M, NM)) != AFQMC_OK ||
      dalloc(h, &Q, (int64_t)M * M) != AFQMC_OK || dalloc(h, &Kb, (int64_t)M * M) != AFQMC_OK ||
      dalloc(h, &E0, (int64_t)M * M) != AFQMC_OK || dalloc(h, &E1, (int64_t)M * M) != AFQMC_OK ||
      dalloc(h, &dnorm, 1) != AFQMC_OK)
    return bail(AFQMC_ERR_NOMEM);

#define AFQ_SCK(call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      cuda_fail(h, #call, e_);                     \
      return bail(AFQMC_ERR_CUDA);                 \
    }                                              \
  } while (0)

  AFQ_SCK(afq::prepare_kernels(*h));
  AFQ_SCK(cudaMemcpyAsync(h->h1, h1_in, sizeof(double) * M * M, cudaMemcpyDefault, s));
  AFQ_SCK(cudaMemcpyAsync(h->L, L_in, sizeof(double) * X * M * M, cudaMemcpyDefault, s));
  AFQ_SCK(cudaMemcpyAsync(tmp, trial_in, sizeof(double) * NM, cudaMemcpyDefault, s));
  AFQ_SCK(afq::launch_transpose(tmp, h->psi, M, N, s));   // [M][N] -> [N][M]
  // Ltil[g][n][i] = sum_j L_g[i][j] psi[n][j]  (rows of Psi_s^T L_g)
  AFQ_SCK(afq::gemm_tn_f64(M, N, M, 1.0, h->L, M, (int64_t)M * M, h->psi, M, 0, 0.0, h->Ltil, M,
                           NM, X, s));
  AFQ_SCK(afq::gemm_tn_f64(M, N, M, 1.0, h->h1, M, 0, h->psi, M, 0, 0.0, h->htil, M, 0, 1, s));
  AFQ_SCK(afq::launch_rho_mf(h->Ltil, h->psi, h->rho_mf, X, (int)NM, s));
  // Q = sum_g L_g L_g through the permuted tensor Lp[i][(g,k)] = L_g[i][k]
  AFQ_SCK(afq::launch_permute_L(h->L, tmp, M, X, s));
  AFQ_SCK(afq::gemm_tn_f64(M, M, X * M, 1.0, tmp, (int64_t)X * M, 0, tmp, (int64_t)X * M, 0, 0.0,
                           Q, M, 0, 1, s));
  // B = -(dt/2) K,  K = h1 - Q/2 + sum_g <rho_g>_T L_g
  AFQ_SCK(afq::launch_build_K(h->h1, Q, h->L, h->rho_mf, Kb, M, X, -0.5 * opt->dt, s));
  AFQ_SCK(afq::launch_pack_Lt(h->L, h->Lt, M, X, s));
  AFQ_SCK(afq::launch_norm1(Kb, M, dnorm, s));
  double nrm = 0;
  std::vector<double> rho(X);
  AFQ_SCK(cudaMemcpyAsync(&nrm, dnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
  AFQ_SCK(cudaMemcpyAsync(rho.data(), h->rho_mf, sizeof(double) * X, cudaMemcpyDeviceToHost, s));
  AFQ_SCK(cudaStreamSynchronize(s));
  if (!std::isfinite(nrm)) {
    set_err(h, AFQMC_ERR_ARG, "non-finite one-body matrix");
    return bail(AFQMC_ERR_ARG);
  }
  double cmf = 0;
  for (double r : rho) cmf += r * r;
  h->c_mf = -0.5 * cmf;
  // exp(B) by scaling and squaring around a degree-20 Taylor polynomial (Horner form):
  // ||B / 2^sq||_1 <= 1/2 makes the truncation error below 2^-75.
  int sq = 0;
  while (nrm / std::ldexp(1.0, sq) > 0.5) ++sq;
  const double sc = std::ldexp(1.0, -sq);
  const int deg = 20;
  AFQ_SCK(cudaMemsetAsync(E0, 0, sizeof(double) * M * M, s));
  AFQ_SCK(afq::launch_add_identity(E0, M, 1.0, s));
  for (int k = deg; k >= 1; --k) {
    // E1 = (sc/k) * B E0 + I   (B and E0 symmetric and commuting)
    AFQ_SCK(afq::gemm_tn_f64(M, M, M, sc / k, E0, M, 0, Kb, M, 0, 0.0, E1, M, 0, 1, s));
    AFQ_SCK(afq::launch_add_identity(E1, M, 1.0, s));
    std::swap(E0, E1);
  }
  for (int q = 0; q < sq; ++q) {
    AFQ_SCK(afq::gemm_tn_f64(M, M, M, 1.0, E0, M, 0, E0, M, 0, 0.0, E1, M, 0, 1, s));
    std::swap(E0, E1);
  }
  AFQ_SCK(cudaMemcpyAsync(h->expK, E0, sizeof(double) * M * M, cudaMemcpyDeviceToDevice, s));
  AFQ_SCK(cudaMemcpyAsync(h->Bneg, Kb, sizeof(double) * M * M, cudaMemcpyDeviceToDevice, s));
  // walkers = trial, w = 1; trial energy E_T = E_L(psi_T)
  AFQ_SCK(afq::launch_broadcast_walkers(h->psi, h->phi, (int)Nw, (int)NM, s));
  AFQ_SCK(afq::launch_init_weights(h->w, h->alive, nullptr, (int)Nw, s));
  AFQ_SCK(cudaMemsetAsync(h->d_step, 0, sizeof(unsigned long long), s));
  AFQ_SCK(cudaMemsetAsync(h->d_flags, 0, sizeof(int) * 4, s));
  AFQ_SCK(afq::launch_overlap(*h, nullptr, afq::OV_REFRESH, s));
  AFQ_SCK(afq::launch_energy(*h, s, 1));   // every walker is the trial: one is enough
  double et = 0;
  int flags = 0;
  AFQ_SCK(cudaMemcpyAsync(&et, h->eloc, sizeof(double), cudaMemcpyDeviceToHost, s));
  AFQ_SCK(cudaMemcpyAsync(&flags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  AFQ_SCK(cudaStreamSynchronize(s));
  if (flags != 0 || !std::isfinite(et)) {
    set_err(h, AFQMC_ERR_NUMERIC, "trial determinant has a singular overlap with itself");
    return bail(AFQMC_ERR_NUMERIC);
  }
  h->e_trial = et;
  if (opt->precision == AFQMC_BF16X3) {
    h->opt.autotune_cache = opt->autotune_cache;
    afqmc_status ms = setup_mixed(h, s);
    h->opt.autotune_cache = nullptr;
    if (ms != AFQMC_OK) return bail(ms);
    AFQ_SCK(cudaStreamSynchronize(s));
  }
  cleanup_tmp();
#undef AFQ_SCK
  *out = h;
  return AFQMC_OK;
}

afqmc_status afqmc_setup_multidet(afqmc_handle* out, const double* h1, const double* L,
                                  const double* dets, const double* coeffs, int n_det,
                                  const double* start, int M, int X, int n_up, int n_dn,
                                  const afqmc_options* opt, cudaStream_t s) {
  if (!out) return AFQMC_ERR_ARG;
  *out = nullptr;
  if (!dets || !coeffs || !opt || n_det < 1 || n_det > 4096) return AFQMC_ERR_ARG;
  if (opt->precision != AFQMC_FP64) return AFQMC_ERR_ARG;
  std::vector<double> c(n_det);
  if (cudaMemcpy(c.data(), coeffs, sizeof(double) * n_det, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return AFQMC_ERR_ARG;
  }
  bool any = false;
  for (double v : c) {
    if (!std::isfinite(v)) return AFQMC_ERR_ARG;
    any = any || v != 0.0;
  }
  if (!any) return AFQMC_ERR_ARG;
  // the first determinant plays the single-determinant trial's part: <rho_g>_T, K, E_T
  afqmc_handle h = nullptr;
  afqmc_status st = afqmc_setup(&h, h1, L, dets, M, X, n_up, n_dn, opt, s);
  if (st != AFQMC_OK) return st;
  const int N = h->N, Nw = h->Nw;
  const int64_t NM = (int64_t)N * M;
  auto fail_with = [&](afqmc_status code) {
    afqmc_destroy(h);
    return code;
  };
  double* tmp = nullptr;
  if (dalloc(h, &h->md_coef, n_det) != AFQMC_OK || dalloc(h, &h->md_psi, n_det * NM) != AFQMC_OK ||
      dalloc(h, &h->md_Ltil, (size_t)n_det * X * NM) != AFQMC_OK ||
      dalloc(h, &h->md_htil, n_det * NM) != AFQMC_OK ||
      dalloc(h, &h->md_logO, (size_t)n_det * 2 * Nw) != AFQMC_OK ||
      dalloc(h, &h->md_theta, (size_t)n_det * 2 * Nw * NM) != AFQMC_OK ||
      dalloc(h, &h->md_share, (size_t)n_det * 2 * Nw) != AFQMC_OK ||
      dalloc(h, &h->md_rhobar, (size_t)n_det * 2 * Nw * X) != AFQMC_OK ||
      dalloc(h, &h->md_eloc, (size_t)n_det * 2 * Nw) != AFQMC_OK ||
      dalloc(h, &tmp, (size_t)(n_det + 1) * NM) != AFQMC_OK)
    return fail_with(AFQMC_ERR_NOMEM);
  cudaError_t e = cudaMemcpyAsync(h->md_coef, c.data(), sizeof(double) * n_det,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tmp, dets, sizeof(double) * n_det * NM, cudaMemcpyDefault, s);
  for (int d = 0; d < n_det && e == cudaSuccess; ++d) {
    double* pd = h->md_psi + d * NM;
    e = afq::launch_transpose(tmp + d * NM, pd, M, N, s);          // [M][N] -> [N][M]
    if (e == cudaSuccess)
      e = afq::gemm_tn_f64(M, N, M, 1.0, h->L, M, (int64_t)M * M, pd, M, 0, 0.0,
                           h->md_Ltil + (int64_t)d * X * NM, M, NM, X, s);
    if (e == cudaSuccess)
      e = afq::gemm_tn_f64(M, N, M, 1.0, h->h1, M, 0, pd, M, 0, 0.0, h->md_htil + d * NM, M, 0,
                           1, s);
  }
  if (e == cudaSuccess && start) {
    double* st_t = tmp + n_det * NM;
    e = cudaMemcpyAsync(tmp, start, sizeof(double) * NM, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = afq::launch_transpose(tmp, st_t, M, N, s);
    if (e == cudaSuccess) e = afq::launch_broadcast_walkers(st_t, h->phi, Nw, (int)NM, s);
  }
  if (e == cudaSuccess) e = afq::launch_init_weights(h->w, h->alive, nullptr, Nw, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, sizeof(int) * 4, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) {
    cuda_fail(h, "afqmc_setup_multidet", e);
    return fail_with(AFQMC_ERR_CUDA);
  }
  h->n_det = n_det;
  if ((st = overlap_launch(h, nullptr, afq::OV_REFRESH, s)) != AFQMC_OK) return fail_with(st);
  int flags = 0;
  e = cudaMemcpyAsync(&flags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_with(AFQMC_ERR_CUDA);
  if (flags != 0) return fail_with(AFQMC_ERR_NUMERIC);
  *out = h;
  return AFQMC_OK;
}

afqmc_status afqmc_destroy(afqmc_handle h) {
  if (!h) return AFQMC_OK;
  free_ctx(h);
  delete h;
  return AFQMC_OK;
}

afqmc_status afqmc_set_walkers(afqmc_handle h, const double* phi, const double* w, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  if (!phi) return set_err(h, AFQMC_ERR_ARG, "phi is NULL");
  const int64_t n = 2 * (int64_t)h->Nw * h->N * h->M;
  // stage the external layout in theta, convert into phi
  AFQ_CK(cudaMemcpyAsync(h->theta, phi, sizeof(double) * n, cudaMemcpyDefault, s));
  AFQ_CK(afq::launch_phi_layout(h->theta, h->phi, h->Nw, h->M, h->N, 1, s));
  const double* wd = nullptr;
  if (w) {
    AFQ_CK(cudaMemcpyAsync(h->eloc, w, sizeof(double) * 2 * h->Nw, cudaMemcpyDefault, s));
    wd = h->eloc;
  }
  AFQ_CK(afq::launch_init_weights(h->w, h->alive, wd, h->Nw, s));
  AFQ_CK(cudaMemsetAsync(h->d_step, 0, sizeof(unsigned long long), s));
  afqmc_status rs = overlap_launch(h, nullptr, afq::OV_REFRESH, s);
  if (rs != AFQMC_OK) return rs;
  h->step = 0;
  return AFQMC_OK;
}

afqmc_status afqmc_set_step(afqmc_handle h, uint64_t step, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  AFQ_CK(afq::set_step(*h, (unsigned long long)step, s));
  h->step = step;
  return AFQMC_OK;
}

afqmc_status afqmc_population_control(afqmc_handle h, const double* u, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  if (!u) return set_err(h, AFQMC_ERR_ARG, "u is NULL");
  if (h->opt.mode != AFQMC_PHASELESS)
    return set_err(h, AFQMC_ERR_ARG, "population control needs real (phaseless) weights");
  if (h->tangent_on) return set_err(h, AFQMC_ERR_STATE, "tangent mode is on");
  const int R = h->R;
  // between steps phi2, aux and esum are free scratch: the running sums, the comb's picks and
  // (u, W / n) per repeat
  double* u_dev = h->esum;
  double* share = h->esum + R;
  int* src = reinterpret_cast<int*>(h->aux);
  AFQ_CK(cudaMemcpyAsync(u_dev, u, sizeof(double) * R, cudaMemcpyDefault, s));
  AFQ_CK(afq::launch_comb(*h, u_dev, h->phi2, src, share, s));
  std::vector<double> q(R);
  AFQ_CK(cudaMemcpyAsync(q.data(), share, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  AFQ_CK(cudaStreamSynchronize(s));
  for (double v : q)
    if (!(v > 0.0) || !std::isfinite(v))
      return set_err(h, AFQMC_ERR_NUMERIC, "a repeat has no live walker to comb");
  AFQ_CK(afq::launch_apply_comb(*h, src, share, h->theta, s));
  return overlap_launch(h, nullptr, afq::OV_REFRESH, s);
}

afqmc_status afqmc_seed_secondary(afqmc_handle B, afqmc_handle A, cudaStream_t s) {
  if (!A || !B || A == B) return AFQMC_ERR_ARG;
  if (B->M != A->M || B->Nw != A->Nw || B->R != A->R || B->n_up > A->n_up || B->n_dn > A->n_dn)
    return set_err(B, AFQMC_ERR_ARG,
                   "the secondary system needs the primary's basis size, walkers and repeats, "
                   "and no more electrons of either spin");
  if (A->opt.mode != AFQMC_PHASELESS || B->opt.mode != AFQMC_PHASELESS)
    return set_err(B, AFQMC_ERR_ARG, "seeding projects phases: phaseless handles only");
  if (A->tangent_on || B->tangent_on) return set_err(B, AFQMC_ERR_STATE, "tangent mode is on");
  afqmc_ctx* h = B;   // the error helpers below report on B
  AFQ_CK(afq::launch_seed_columns(*A, *B, s));
  AFQ_CK(afq::launch_init_weights(B->w, B->alive, nullptr, B->Nw, s));
  afqmc_status rs = overlap_launch(B, nullptr, afq::OV_REFRESH, s);
  if (rs != AFQMC_OK) return rs;
  AFQ_CK(afq::launch_seed_weights(*A, *B, s));
  AFQ_CK(afq::set_step(*B, (unsigned long long)A->step, s));
  B->step = A->step;
  return AFQMC_OK;
}

afqmc_status afqmc_get_state(afqmc_handle h, double* phi, double* logO, double* w, int* alive,
                             cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  if (phi) {
    const int64_t n = 2 * (int64_t)h->Nw * h->N * h->M;
    AFQ_CK(afq::launch_phi_layout(h->phi, h->phi2, h->Nw, h->M, h->N, 0, s));
    AFQ_CK(cudaMemcpyAsync(phi, h->phi2, sizeof(double) * n, cudaMemcpyDefault, s));
  }
  if (logO) AFQ_CK(cudaMemcpyAsync(logO, h->logO, sizeof(double) * 2 * h->Nw, cudaMemcpyDefault, s));
  if (w) AFQ_CK(cudaMemcpyAsync(w, h->w, sizeof(double) * 2 * h->Nw, cudaMemcpyDefault, s));
  if (alive) AFQ_CK(cudaMemcpyAsync(alive, h->alive, sizeof(int) * h->Nw, cudaMemcpyDefault, s));
  AFQ_CK(cudaStreamSynchronize(s));
  return check_tc(h);
}

afqmc_status afqmc_get_info(afqmc_handle h, afqmc_info* info, cudaStream_t s) {
  if (!h || !info) return AFQMC_ERR_ARG;
  info->M = h->M; info->X = h->X; info->n_up = h->n_up; info->n_dn = h->n_dn;
  info->n_walkers = h->Nw; info->n_repeats = h->R; info->step = h->step;
  info->e_trial = h->e_trial; info->c_mf = h->c_mf;
  info->tuned_energy_walkers_per_cta = h->tune_energy_wb;
  info->tuned_taylor_smem = h->tune_taylor_smem;
  info->tuned_orthonormalise = h->tune_mgs;
  info->n_det = h->n_det;
  std::vector<int> al(h->Nw);
  AFQ_CK(cudaMemcpyAsync(al.data(), h->alive, sizeof(int) * h->Nw, cudaMemcpyDeviceToHost, s));
  AFQ_CK(cudaStreamSynchronize(s));
  int n = 0;
  for (int a : al) n += a != 0;
  info->n_alive = n;
  return check_tc(h);
}

afqmc_status afqmc_propagate(afqmc_handle h, int n_steps, const double* fields, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  if (n_steps < 0) return set_err(h, AFQMC_ERR_ARG, "n_steps < 0");
  if (n_steps == 0) return AFQMC_OK;
  const int64_t per = (int64_t)h->Nw * h->X;
  const double* fd = nullptr;
  double* staged = nullptr;
  if (fields) {
    if (is_device_ptr(fields)) {
      fd = fields;
    } else {
      if (dalloc(h, &staged, (size_t)(per * n_steps)) != AFQMC_OK) return AFQMC_ERR_NOMEM;
      cudaError_t e = cudaMemcpyAsync(staged, fields, sizeof(double) * per * n_steps,
                                      cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) { cudaFree(staged); return cuda_fail(h, "staging fields", e); }
      fd = staged;
    }
  }
  afqmc_status st = AFQMC_OK;
  for (int t = 0; t < n_steps && st == AFQMC_OK; ++t) st = step_launch(h, fd ? fd + per * t : nullptr, s);
  if (staged) {
    cudaStreamSynchronize(s);
    cudaFree(staged);
  }
  if (st == AFQMC_OK) h->step += (uint64_t)n_steps;
  return st;
}

afqmc_status afqmc_orthonormalise(afqmc_handle h, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  return ortho_launch(h, s);
}

afqmc_status afqmc_energy(afqmc_handle h, double* e_local, double* e_mixed, double* w_sum,
                          cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  afqmc_status est = energy_launch(h, s);
  if (est != AFQMC_OK) return est;
  if (e_local) AFQ_CK(cudaMemcpyAsync(e_local, h->eloc, sizeof(double) * 2 * h->Nw, cudaMemcpyDefault, s));
  if (e_mixed || w_sum) {
    AFQ_CK(afq::launch_mixed_sum(*h, h->esum, nullptr, 0, s));
    std::vector<double> es(4 * (size_t)h->R);
    AFQ_CK(cudaMemcpyAsync(es.data(), h->esum, sizeof(double) * es.size(), cudaMemcpyDeviceToHost, s));
    AFQ_CK(cudaStreamSynchronize(s));
    std::vector<double> em(h->R), ws(h->R);
    for (int r = 0; r < h->R; ++r) {
      const double nr = es[4 * r], ni = es[4 * r + 1], dr = es[4 * r + 2], di = es[4 * r + 3];
      const double d2 = dr * dr + di * di;
      em[r] = d2 > 0 ? (nr * dr + ni * di) / d2 : NAN;
      ws[r] = dr;
    }
    if (e_mixed) AFQ_CK(cudaMemcpyAsync(e_mixed, em.data(), sizeof(double) * h->R, cudaMemcpyDefault, s));
    if (w_sum) AFQ_CK(cudaMemcpyAsync(w_sum, ws.data(), sizeof(double) * h->R, cudaMemcpyDefault, s));
    AFQ_CK(cudaStreamSynchronize(s));
    return check_tc(h);
  } else if (e_local && !is_device_ptr(e_local)) {
    AFQ_CK(cudaStreamSynchronize(s));
  }
  return AFQMC_OK;
}

afqmc_status afqmc_time_kernel(afqmc_handle h, int which, int reps, double* ms, cudaStream_t s) {
  if (!h || !ms || reps < 1 || which < 0 || which > 6) return AFQMC_ERR_ARG;
  if (which == AFQMC_K_MGS && h->tangent_on) {
    h->err = "AFQMC_K_MGS is not timed in tangent mode";
    return AFQMC_ERR_STATE;
  }
  const bool fast_ov = h->theta32 && h->tc_Theta && h->phi32 && afq::fast_walker_kernels_ok(*h);
  if (which == AFQMC_K_OVERLAP_UPDATE && !fast_ov) {
    h->err = "AFQMC_K_OVERLAP_UPDATE times the split-precision overlap kernel only";
    return AFQMC_ERR_ARG;
  }
  const int M = h->M, X = h->X, N = h->N, Nw = h->Nw;
  const int64_t NM = (int64_t)N * M;
  cudaEvent_t e0, e1;
  AFQ_CK(cudaEventCreate(&e0));
  AFQ_CK(cudaEventCreate(&e1));
  auto one = [&]() -> cudaError_t {
    switch (which) {
      case AFQMC_K_VHS:   // split precision: in the form the propagation variant reads
        if (h->tc_L) return afq::vhs_launch(*h, afq::propagation_variant(*h), s);
        return afq::gemm_tn_f64((int)h->P, 2 * Nw, X, 1.0, h->Lt, X, 0, h->U, X, 0, 0.0, h->Avhs,
                                h->P, 0, 1, s, afq::GEMM_VHS);
      case AFQMC_K_FORCE_BIAS:
        if (h->n_det > 0) return afq::md_force_bias(*h, s);
        if (h->tc_Ltil)
          return afq::gemm_bf16x3(*h->tc_Ltil, *h->tc_Theta, X, 2 * Nw, 1.0f, h->rhobar32, X,
                                  h->d_tc_err, s);
        return afq::gemm_tn_f64(X, 2 * Nw, (int)NM, 1.0, h->Ltil, NM, 0, h->theta, NM, 0, 0.0,
                                h->rhobar, X, 0, 1, s, afq::GEMM_FORCE_BIAS);
      case AFQMC_K_OVERLAP_UPDATE:   // Phi <- Phi (unchanged), Theta from the FP32 walkers
        return afq::launch_overlap_fast(*h, h->phi, afq::OV_UPDATE, s, h->phi32, false);
      case AFQMC_K_OVERLAP:
        if (h->n_det > 0) return afq::md_overlap(*h, nullptr, afq::OV_REFRESH, s);
        if (h->theta32 && h->tc_Theta && afq::fast_walker_kernels_ok(*h))
          return afq::launch_overlap_fast(*h, nullptr, afq::OV_REFRESH, s);
        return afq::launch_overlap(*h, nullptr, afq::OV_REFRESH, s);
      case AFQMC_K_MGS: {
        const afqmc_status st = ortho_launch(h, s);
        return st == AFQMC_OK ? cudaSuccess : cudaErrorUnknown;
      }
      case AFQMC_K_TAYLOR:   // split precision: the fused propagator times its two one-body products too
        if (h->phi32) return afq::launch_propagation(*h, afq::propagation_variant(*h), h->theta, nullptr, s);
        return afq::launch_taylor(*h, h->phi2, s);
      default:
        if (h->n_det > 0) return afq::md_energy(*h, s);
        if (h->etc && h->tune_energy_wb <= 0) return afq::launch_energy_tc(*h, s);
        if (h->LtT) return afq::launch_energy_tiled(*h, h->theta32, h->LtT, s);
        return afq::launch_energy(*h, s);
    }
  };
  cudaError_t e = one();  // warm
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = one();
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  // the update form took Theta from the FP32 walkers, which Gram-Schmidt leaves stale
  if (e == cudaSuccess && which == AFQMC_K_OVERLAP_UPDATE)
    e = afq::launch_overlap_fast(*h, nullptr, afq::OV_REFRESH, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(h, "afqmc_time_kernel", e);
  *ms = (double)t / reps;
  return AFQMC_OK;
}

// C = X Y for n x n row-major matrices through the TN kernel (Y transposed into Yt first).
afqmc_status gemm_nn(Ctx* h, int n, double alpha, const double* Xm, const double* Ym, double* Yt,
                     double* C, cudaStream_t s) {
  AFQ_CK(afq::launch_transpose(Ym, Yt, n, n, s));
  AFQ_CK(afq::gemm_tn_f64(n, n, n, alpha, Yt, n, 0, Xm, n, 0, 0.0, C, n, 0, 1, s));
  return AFQMC_OK;
}

}  // extern "C"

namespace afq {
// out = L_exp(B, scale * dir), B = -dt K / 2: the Frechet derivative of the matrix exponential
// at B along scale * dir, read off the upper-right block of exp([[B, D], [0, B]]) (Taylor
// series of order 20 with scaling and squaring, as at setup).  The direction is scaled down
// to the norm of B first and the result scaled back (the map is linear in D), so the block
// matrix needs no more squarings than B itself.  dir, out: device [M][M].
afqmc_status frechet_expm(Ctx* h, const double* dir, double scale, double* out, cudaStream_t s) {
  const int M = h->M, n2 = 2 * M;
  const size_t zz = (size_t)n2 * n2;
  double *Z = nullptr, *E0 = nullptr, *E1 = nullptr, *Yt = nullptr, *dn = nullptr;
  auto cleanup = [&]() {
    for (double* p : {Z, E0, E1, Yt, dn})
      if (p) cudaFree(p);
  };
  if (dalloc(h, &Z, zz) != AFQMC_OK || dalloc(h, &E0, zz) != AFQMC_OK || dalloc(h, &E1, zz) != AFQMC_OK ||
      dalloc(h, &Yt, zz) != AFQMC_OK || dalloc(h, &dn, 3) != AFQMC_OK) {
    cleanup();
    return AFQMC_ERR_NOMEM;
  }
  double nrm[3] = {0, 0, 0};
  cudaError_t e = launch_norm1(dir, M, dn, s);
  if (e == cudaSuccess) e = launch_norm1(h->Bneg, M, dn + 1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nrm, dn, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(h, "frechet_expm", e);
  }
  const double nd = std::fabs(scale) * nrm[0], nb = nrm[1];
  if (!std::isfinite(nd)) {
    cleanup();
    return set_err(h, AFQMC_ERR_NUMERIC, "non-finite direction for the exponential's derivative");
  }
  if (nd == 0.0) {
    e = cudaMemsetAsync(out, 0, sizeof(double) * M * M, s);
    cleanup();
    return e == cudaSuccess ? AFQMC_OK : cuda_fail(h, "frechet_expm", e);
  }
  const double eps = (nb > 0.0 && nd > nb) ? nb / nd : 1.0;
  e = cudaMemsetAsync(Z, 0, sizeof(double) * zz, s);
  if (e == cudaSuccess) e = place_block(Z, n2, 0, 0, h->Bneg, M, 1.0, s);
  if (e == cudaSuccess) e = place_block(Z, n2, M, M, h->Bneg, M, 1.0, s);
  if (e == cudaSuccess) e = place_block(Z, n2, 0, M, dir, M, scale * eps, s);
  if (e == cudaSuccess) e = launch_norm1(Z, n2, dn + 2, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nrm + 2, dn + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(h, "frechet_expm", e);
  }
  int sq = 0;
  while (nrm[2] / std::ldexp(1.0, sq) > 0.5) ++sq;
  const double sc = std::ldexp(1.0, -sq);
  e = cudaMemsetAsync(E0, 0, sizeof(double) * zz, s);
  if (e == cudaSuccess) e = launch_add_identity(E0, n2, 1.0, s);
  for (int k = 20; k >= 1 && e == cudaSuccess; --k) {
    if (gemm_nn(h, n2, sc / k, Z, E0, Yt, E1, s) != AFQMC_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = launch_add_identity(E1, n2, 1.0, s);
    std::swap(E0, E1);
  }
  for (int q = 0; q < sq && e == cudaSuccess; ++q) {
    if (gemm_nn(h, n2, 1.0, E0, E0, Yt, E1, s) != AFQMC_OK) e = cudaErrorUnknown;
    std::swap(E0, E1);
  }
  if (e == cudaSuccess) e = take_block(E0, n2, 0, M, out, M, 1.0 / eps, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  return e == cudaSuccess ? AFQMC_OK : cuda_fail(h, "frechet_expm", e);
}
}  // namespace afq

extern "C" {

afqmc_status afqmc_set_tangent(afqmc_handle h, const double* P, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  if (!P) {
    h->tangent_on = false;
    return AFQMC_OK;
  }
  if (h->opt.precision != AFQMC_FP64 || h->opt.mode != AFQMC_PHASELESS)
    return set_err(h, AFQMC_ERR_ARG, "tangent mode needs the FP64 phaseless path");
  if (h->n_det > 0) return set_err(h, AFQMC_ERR_ARG, "tangent mode needs a single-determinant trial");
  if (!afq::tangent_fits(*h)) return set_err(h, AFQMC_ERR_ARG, "tangent kernels exceed shared memory");
  const int M = h->M, X = h->X, N = h->N, Nw = h->Nw;
  const int64_t NM = (int64_t)N * M;
  afqmc_status st;
  if (!h->dphi) {
    if ((st = dalloc(h, &h->dexpK, (size_t)M * M)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->htilP, (size_t)NM)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->dphi, 2 * (size_t)Nw * NM)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->dphi2, 2 * (size_t)Nw * NM)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->dtheta, 2 * (size_t)Nw * NM)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->drhobar, 2 * (size_t)Nw * X)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->dU, 2 * (size_t)Nw * X)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->dAvhs, 2 * (size_t)Nw * h->P)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->dlogO, 2 * (size_t)Nw)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->dlogw, (size_t)Nw)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->daux, 4 * (size_t)Nw)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->deloc, 2 * (size_t)Nw)) != AFQMC_OK) return st;
    if ((st = dalloc(h, &h->desum, 4 * (size_t)h->R)) != AFQMC_OK) return st;
  }
  AFQ_CK(afq::prepare_tangent_kernels(*h));
  double *dP = nullptr, *dE = nullptr;
  if (dalloc(h, &dP, (size_t)M * M) != AFQMC_OK || dalloc(h, &dE, 1) != AFQMC_OK) {
    if (dP) cudaFree(dP);
    return AFQMC_ERR_NOMEM;
  }
  auto cleanup = [&]() {
    cudaFree(dP);
    cudaFree(dE);
  };
  cudaError_t e = cudaMemcpyAsync(dP, P, sizeof(double) * M * M, cudaMemcpyDefault, s);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(h, "afqmc_set_tangent", e);
  }
  // d exp(B) along dB = -dt P / 2
  afqmc_status fs = afq::frechet_expm(h, dP, -0.5 * h->opt.dt, h->dexpK, s);
  if (fs != AFQMC_OK) {
    cleanup();
    return fs;
  }
  // Psi^T P rows and dE_T = sum_s tr(P P_s)
  if (e == cudaSuccess) e = afq::gemm_tn_f64(M, N, M, 1.0, dP, M, 0, h->psi, M, 0, 0.0, h->htilP, M, 0, 1, s);
  if (e == cudaSuccess) e = afq::launch_rho_mf(h->htilP, h->psi, dE, 1, (int)NM, s);
  double det = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&det, dE, sizeof(double), cudaMemcpyDeviceToHost, s);
  for (double* b : {h->dphi, h->dtheta})
    if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, sizeof(double) * 2 * Nw * NM, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->dlogO, 0, sizeof(double) * 2 * Nw, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->dlogw, 0, sizeof(double) * Nw, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(h, "afqmc_set_tangent", e);
  h->de_trial = det;
  h->tangent_on = true;
  // consistent Theta / log O / tangents of the current walkers
  AFQ_CK(afq::launch_overlap_tan(*h, afq::OV_REFRESH, s));
  return AFQMC_OK;
}

afqmc_status afqmc_energy_tangent(afqmc_handle h, double* de_local, double* e_mixed,
                                  double* de_mixed, cudaStream_t s) {
  if (!h) return AFQMC_ERR_ARG;
  if (!h->tangent_on) return set_err(h, AFQMC_ERR_STATE, "tangent mode is not enabled");
  AFQ_CK(afq::launch_energy_tan(*h, s));
  if (de_local) AFQ_CK(cudaMemcpyAsync(de_local, h->deloc, sizeof(double) * 2 * h->Nw, cudaMemcpyDefault, s));
  AFQ_CK(afq::launch_mixed_sum_tan(*h, h->desum, s));
  std::vector<double> es(4 * (size_t)h->R);
  AFQ_CK(cudaMemcpyAsync(es.data(), h->desum, sizeof(double) * es.size(), cudaMemcpyDeviceToHost, s));
  AFQ_CK(cudaStreamSynchronize(s));
  std::vector<double> em(h->R), dm(h->R);
  for (int r = 0; r < h->R; ++r) {
    const double num = es[4 * r], den = es[4 * r + 1], dnum = es[4 * r + 2], dden = es[4 * r + 3];
    em[r] = den != 0 ? num / den : NAN;
    dm[r] = den != 0 ? (dnum - em[r] * dden) / den : NAN;
  }
  if (e_mixed) AFQ_CK(cudaMemcpy(e_mixed, em.data(), sizeof(double) * h->R, cudaMemcpyDefault));
  if (de_mixed) AFQ_CK(cudaMemcpy(de_mixed, dm.data(), sizeof(double) * h->R, cudaMemcpyDefault));
  return AFQMC_OK;
}

afqmc_status afqmc_get_tangent_state(afqmc_handle h, double* dlogw, cudaStream_t s) {
  if (!h || !dlogw) return AFQMC_ERR_ARG;
  if (!h->tangent_on) return set_err(h, AFQMC_ERR_STATE, "tangent mode is not enabled");
  AFQ_CK(cudaMemcpyAsync(dlogw, h->dlogw, sizeof(double) * h->Nw, cudaMemcpyDefault, s));
  AFQ_CK(cudaStreamSynchronize(s));
  return AFQMC_OK;
}

afqmc_status afqmc_select_kernel(afqmc_handle h, int which, int variant) {
  if (!h) return AFQMC_ERR_ARG;
  if (which == AFQMC_K_PAIR_LOOP) {
    if (variant != 0 && variant != 1) return set_err(h, AFQMC_ERR_ARG, "pair-run form is 0 or 1");
    h->pair_loop = variant;
    return AFQMC_OK;
  }
  if (h->opt.precision != AFQMC_BF16X3) return set_err(h, AFQMC_ERR_ARG, "FP64 handles have no variants");
  if (which == AFQMC_K_EXCHANGE) {
    const bool ok = variant == 0 ? h->etc != nullptr
                                 : (variant == 2 || variant == 4 || variant == 8) &&
                                       afq::energy_variant_ok(*h, variant);
    if (!ok) return set_err(h, AFQMC_ERR_ARG, "local-energy variant unsupported for this shape");
    h->tune_energy_wb = variant;
    return AFQMC_OK;
  }
  if (which == AFQMC_K_MGS) {
    if (variant != 0 && !(variant == 1 && afq::mgs_chol_ok(*h)))
      return set_err(h, AFQMC_ERR_ARG, "orthonormalisation variant unsupported for this shape");
    h->tune_mgs = variant;
    return AFQMC_OK;
  }
  if (which == AFQMC_K_TAYLOR) {
    if (variant < 0 || variant > 4 || !afq::taylor_variant_ok(*h, variant))
      return set_err(h, AFQMC_ERR_ARG, "Taylor variant unsupported for this shape");
    h->tune_taylor_smem = variant;
    return AFQMC_OK;
  }
  return set_err(h, AFQMC_ERR_ARG, "no variants for this kernel");
}

afqmc_status afqmc_test_gemm(int impl, int Md, int Nd, int K, const double* A, const double* B,
                             double alpha, double* C, cudaStream_t s) {
  if (Md < 1 || Nd < 1 || K < 1 || !A || !B || !C || impl < 0 || impl > 2) return AFQMC_ERR_ARG;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  float* fC = nullptr;
  __nv_bfloat16 *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  int* err = nullptr;
  const int Kp = afq::pad64(K);
  auto cleanup = [&]() {
    for (void* p : {(void*)dA, (void*)dB, (void*)dC, (void*)fC, (void*)ah, (void*)al, (void*)bh,
                    (void*)bl, (void*)err})
      if (p) cudaFree(p);
  };
  afqmc_status st = AFQMC_OK;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&dA, sizeof(double) * Md * (size_t)K)) != cudaSuccess) break;
    if ((e = cudaMalloc(&dB, sizeof(double) * Nd * (size_t)K)) != cudaSuccess) break;
    if ((e = cudaMalloc(&dC, sizeof(double) * Md * (size_t)Nd)) != cudaSuccess) break;
    if ((e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(dA, A, sizeof(double) * Md * (size_t)K, cudaMemcpyDefault, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(dB, B, sizeof(double) * Nd * (size_t)K, cudaMemcpyDefault, s)) != cudaSuccess) break;
    if (impl == 0) {
      if ((e = afq::gemm_tn_f64(Md, Nd, K, alpha, dA, K, 0, dB, K, 0, 0.0, dC, Md, 0, 1, s)) != cudaSuccess) break;
    } else {
      if ((e = afq::prepare_tc_kernels()) != cudaSuccess) break;
      const int Mp = afq::tc_pad_rows(Md), Np = afq::tc_pad_rows(Nd);
      if ((e = cudaMalloc(&fC, sizeof(float) * Md * (size_t)Nd)) != cudaSuccess) break;
      if ((e = cudaMalloc(&ah, 2 * (size_t)Mp * Kp)) != cudaSuccess) break;
      if ((e = cudaMalloc(&al, 2 * (size_t)Mp * Kp)) != cudaSuccess) break;
      if ((e = cudaMalloc(&bh, 2 * (size_t)Np * Kp)) != cudaSuccess) break;
      if ((e = cudaMalloc(&bl, 2 * (size_t)Np * Kp)) != cudaSuccess) break;
      for (void* p : {(void*)ah, (void*)al})
        if ((e = cudaMemsetAsync(p, 0, 2 * (size_t)Mp * Kp, s)) != cudaSuccess) break;
      for (void* p : {(void*)bh, (void*)bl})
        if ((e = cudaMemsetAsync(p, 0, 2 * (size_t)Np * Kp, s)) != cudaSuccess) break;
      if (e != cudaSuccess) break;
      if ((e = afq::split_bf16(dA, K, Md, K, Kp, ah, al, s)) != cudaSuccess) break;
      if ((e = afq::split_bf16(dB, K, Nd, K, Kp, bh, bl, s)) != cudaSuccess) break;
      afq::TcOperand oa, ob;
      if ((e = afq::tc_make_operand(oa, ah, al, Mp, Kp, 128)) != cudaSuccess) break;
      if ((e = afq::tc_make_operand(ob, bh, bl, Np, Kp, afq::tc_bn())) != cudaSuccess) break;
      if (impl == 2) {
        if ((e = afq::gemm_bf16x3_wait_selftest(oa, ob, Md, Nd, fC, Md, err, 20000000ull, s)) !=
            cudaSuccess)
          break;
      } else if ((e = afq::gemm_bf16x3(oa, ob, Md, Nd, (float)alpha, fC, Md, err, s)) != cudaSuccess) {
        break;
      }
      std::vector<float> hf((size_t)Md * Nd);
      if ((e = cudaMemcpyAsync(hf.data(), fC, sizeof(float) * hf.size(), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
      int herr = 0;
      if ((e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
      if (herr) { st = AFQMC_ERR_TIMEOUT; break; }
      std::vector<double> hd(hf.begin(), hf.end());
      if ((e = cudaMemcpy(C, hd.data(), sizeof(double) * hd.size(), cudaMemcpyDefault)) != cudaSuccess) break;
      break;
    }
    if ((e = cudaMemcpyAsync(C, dC, sizeof(double) * Md * (size_t)Nd, cudaMemcpyDefault, s)) != cudaSuccess) break;
    e = cudaStreamSynchronize(s);
  } while (0);
  cleanup();
  if (st != AFQMC_OK) return st;
  return e == cudaSuccess ? AFQMC_OK : AFQMC_ERR_CUDA;
}

}  // extern "C"
