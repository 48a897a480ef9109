// Correlated-sampling pair run (Sec. II.B): both systems advance in lockstep on the
// shared field stream.  One measurement block (energy_every steps of A and B on two
// forked capture streams, the orthonormalisation passes, both energies and their
// per-repeat sums) is captured once as a CUDA graph.  Default form: the block is the body
// of a device-side while loop, so the whole run of both systems is one graph launch; the
// block's last kernel counts the blocks and ends the loop.  Form 0 (afqmc_select_kernel
// AFQMC_K_PAIR_LOOP): the block graph is launched once per measurement block.  Either way
// the only host crossing is one copy of the energy series at the end.
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

struct afqmc_ctx : afq::Ctx {};

namespace afq {
afqmc_status pair_step(Ctx* h, cudaStream_t s);
afqmc_status pair_ortho(Ctx* h, cudaStream_t s);
afqmc_status pair_energy(Ctx* h, cudaStream_t s);
afqmc_status pair_check(Ctx* h);
cudaError_t launch_meas_advance(int* meas, cudaStream_t s);
}  // namespace afq

namespace {

// Captured pair run of one (A, B, energy_every, mgs_every, form) combination, kept in A.
struct Res {
  uint64_t partner_uid = 0;
  int ee = 0, me = 0, capacity = 0;
  int form = 0;   // 1: graph = while loop around the block; 0: graph = the block
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, ready = nullptr, done = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double* series = nullptr;
  int* meas = nullptr;   // [0] blocks done in this call, [1] blocks this call asks for
  int n_kernels = 0;     // kernel nodes of one captured block
  ~Res() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (series) cudaFree(series);
    if (meas) cudaFree(meas);
    for (cudaEvent_t e : {fork, join, ready, done})
      if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
    if (cs2) cudaStreamDestroy(cs2);
  }
};

afqmc_status fail(afqmc_ctx* A, afqmc_ctx* B, afqmc_status code, const std::string& msg) {
  if (A) A->err = msg;
  if (B) B->err = msg;
  return code;
}

// Loop form: the last kernel of every block counts it and clears the loop's condition once
// the call's blocks are done (meas[1]) or the series buffer is full (capacity), whichever
// comes first, so the loop ends after at most `capacity` blocks whatever meas[1] holds.
__global__ void k_meas_next(int* meas, int capacity, cudaGraphConditionalHandle loop) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int m = meas[0] + 1;
    meas[0] = m;
    if (m >= meas[1] || m >= capacity) cudaGraphSetConditional(loop, 0);
  }
}

__global__ void k_meas_start(int* meas, int n_meas) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    meas[0] = 0;
    meas[1] = n_meas;
  }
}

// Records one measurement block of A (on r->cs) and B (on r->cs2) into the capture running
// on r->cs; `last` adds the block's final kernel on r->cs after the two branches join.
template <class F>
afqmc_status record_block(afqmc_ctx* A, afqmc_ctx* B, Res* r, F last) {
  const int R = A->R, stride = 8 * R;
  afqmc_status st = AFQMC_OK;
  cudaError_t ce = cudaEventRecord(r->fork, r->cs);
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(r->cs2, r->fork, 0);
  for (int j = 0; j < r->ee && st == AFQMC_OK && ce == cudaSuccess; ++j) {
    st = afq::pair_step(A, r->cs);
    if (st == AFQMC_OK) st = afq::pair_step(B, r->cs2);
    if (st == AFQMC_OK && (j + 1) % r->me == 0) {
      st = afq::pair_ortho(A, r->cs);
      if (st == AFQMC_OK) st = afq::pair_ortho(B, r->cs2);
    }
  }
  if (st == AFQMC_OK && ce == cudaSuccess) st = afq::pair_energy(A, r->cs);
  if (st == AFQMC_OK && ce == cudaSuccess) st = afq::pair_energy(B, r->cs2);
  if (st == AFQMC_OK && ce == cudaSuccess) {
    ce = afq::launch_mixed_sum(*A, r->series, r->meas, stride, r->cs);
    if (ce == cudaSuccess) ce = afq::launch_mixed_sum(*B, r->series + 4 * R, r->meas, stride, r->cs2);
    if (ce == cudaSuccess) ce = cudaEventRecord(r->join, r->cs2);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(r->cs, r->join, 0);
    if (ce == cudaSuccess) ce = last();
  }
  if (st != AFQMC_OK) return st;
  if (ce != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  return AFQMC_OK;
}

afqmc_status count_kernels(afqmc_ctx* A, afqmc_ctx* B, cudaGraph_t g, int* n) {
  size_t n_nodes = 0;
  *n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n_nodes) != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, "cudaGraphGetNodes failed");
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  if (n_nodes && cudaGraphGetNodes(g, nodes.data(), &n_nodes) != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, "cudaGraphGetNodes failed");
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess)
      return fail(A, B, AFQMC_ERR_CUDA, "cudaGraphNodeGetType failed");
    if (ty == cudaGraphNodeTypeKernel) ++*n;
  }
  return AFQMC_OK;
}

// Form 0: the block alone, launched once per measurement block.
afqmc_status build_block_graph(afqmc_ctx* A, afqmc_ctx* B, Res* r) {
  cudaError_t ce = cudaStreamBeginCapture(r->cs, cudaStreamCaptureModeRelaxed);
  if (ce != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  afqmc_status st = record_block(A, B, r, [&]() { return afq::launch_meas_advance(r->meas, r->cs); });
  ce = cudaStreamEndCapture(r->cs, &r->graph);
  if (st != AFQMC_OK) return st;
  if (ce != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  if ((ce = cudaGraphInstantiate(&r->exec, r->graph, 0)) != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ce));
  return count_kernels(A, B, r->graph, &r->n_kernels);
}

// Form 1: a graph whose only node is a while loop with the block as its body; one launch
// runs every block of the call.
afqmc_status build_loop_graph(afqmc_ctx* A, afqmc_ctx* B, Res* r) {
  cudaGraphConditionalHandle cond;
  cudaError_t ce = cudaGraphCreate(&r->graph, 0);
  if (ce == cudaSuccess)
    ce = cudaGraphConditionalHandleCreate(&cond, r->graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, r->graph, nullptr, nullptr, 0, &p);
  if (ce != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("loop node: ") + cudaGetErrorString(ce));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  ce = cudaStreamBeginCaptureToGraph(r->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (ce != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  const int cap = r->capacity;
  int* meas = r->meas;
  cudaStream_t cs = r->cs;
  afqmc_status st = record_block(A, B, r, [&]() {
    k_meas_next<<<1, 32, 0, cs>>>(meas, cap, cond);
    return cudaGetLastError();
  });
  cudaGraph_t got = nullptr;
  ce = cudaStreamEndCapture(r->cs, &got);
  if (st != AFQMC_OK) return st;
  if (ce != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  if ((ce = cudaGraphInstantiate(&r->exec, r->graph, 0)) != cudaSuccess)
    return fail(A, B, AFQMC_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ce));
  return count_kernels(A, B, body, &r->n_kernels);
}

}  // namespace

namespace afq {
void destroy_pair_cache(Ctx* h) {
  if (h->pair_cache) {
    delete static_cast<Res*>(h->pair_cache);
    h->pair_cache = nullptr;
  }
}
}  // namespace afq

extern "C" afqmc_status afqmc_pair_delta_E(afqmc_handle A, afqmc_handle B, int n_steps,
                                           int energy_every, int mgs_every, double tau_eq,
                                           double* e_series, double* dE_mean, double* dE_sigma,
                                           double* tau_at_min, cudaStream_t s) {
  if (!A || !B || A == B) return fail(A, B, AFQMC_ERR_ARG, "need two distinct handles");
  if (A->Nw != B->Nw || A->R != B->R || A->opt.dt != B->opt.dt ||
      A->opt.mode != B->opt.mode || A->opt.walker_offset != B->opt.walker_offset ||
      A->opt.precision != B->opt.precision)
    return fail(A, B, AFQMC_ERR_ARG, "pair handles differ in walkers, repeats, dt, mode, precision or walker offset");
  // Correlated sampling shares one field stream (one key); the uncorrelated comparison
  // needs two keys, so equal seeds there would silently correlate the pair.
  if (A->opt.independent_fields != B->opt.independent_fields)
    return fail(A, B, AFQMC_ERR_ARG, "pair handles differ in independent_fields");
  if (!A->opt.independent_fields && A->opt.seed != B->opt.seed)
    return fail(A, B, AFQMC_ERR_ARG, "correlated pair handles need the same seed");
  if (A->opt.independent_fields && A->opt.seed == B->opt.seed)
    return fail(A, B, AFQMC_ERR_ARG, "independent_fields needs different seeds");
  if (A->step != B->step) return fail(A, B, AFQMC_ERR_STATE, "pair handles are at different steps");
  if (A->tangent_on || B->tangent_on)
    return fail(A, B, AFQMC_ERR_STATE, "tangent mode runs through afqmc_propagate, not the pair graph");
  if (energy_every < 1 || mgs_every < 1 || energy_every % mgs_every != 0 || n_steps < 0 ||
      n_steps % energy_every != 0)
    return fail(A, B, AFQMC_ERR_ARG, "need energy_every % mgs_every == 0 and n_steps % energy_every == 0");
  if (A->step % (uint64_t)energy_every != 0)
    return fail(A, B, AFQMC_ERR_STATE, "step counter is not a multiple of energy_every");
  const int n_meas = n_steps / energy_every, R = A->R;
  const int stride = 8 * R;  // per measurement: [A: R x 4][B: R x 4]
#define AFQ_PCK(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(A, B, AFQMC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  Res* r = static_cast<Res*>(A->pair_cache);
  const int form = A->pair_loop ? 1 : 0;
  if (n_meas > 0 && (!r || r->partner_uid != B->uid || r->ee != energy_every ||
                     r->me != mgs_every || r->capacity < n_meas || r->form != form)) {
    afq::destroy_pair_cache(A);
    r = new Res();
    A->pair_cache = r;
    r->partner_uid = B->uid;
    r->ee = energy_every;
    r->me = mgs_every;
    r->capacity = n_meas;
    r->form = form;
    AFQ_PCK(cudaMalloc(&r->series, sizeof(double) * (size_t)n_meas * stride));
    AFQ_PCK(cudaMalloc(&r->meas, 2 * sizeof(int)));
    AFQ_PCK(cudaStreamCreateWithFlags(&r->cs, cudaStreamNonBlocking));
    AFQ_PCK(cudaStreamCreateWithFlags(&r->cs2, cudaStreamNonBlocking));
    AFQ_PCK(cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming));
    AFQ_PCK(cudaEventCreateWithFlags(&r->join, cudaEventDisableTiming));
    AFQ_PCK(cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming));
    AFQ_PCK(cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming));
    const afqmc_status st = form ? build_loop_graph(A, B, r) : build_block_graph(A, B, r);
    if (st != AFQMC_OK) {
      afq::destroy_pair_cache(A);
      return st;
    }
  }
  cudaStream_t cs = s;
  if (n_meas > 0) {
    cs = r->cs;
    AFQ_PCK(cudaEventRecord(r->ready, s));
    AFQ_PCK(cudaStreamWaitEvent(r->cs, r->ready, 0));
    if (r->form) {
      k_meas_start<<<1, 32, 0, r->cs>>>(r->meas, n_meas);
      AFQ_PCK(cudaGetLastError());
      AFQ_PCK(cudaGraphLaunch(r->exec, r->cs));
    } else {
      AFQ_PCK(cudaMemsetAsync(r->meas, 0, sizeof(int), r->cs));
      for (int m = 0; m < n_meas; ++m) AFQ_PCK(cudaGraphLaunch(r->exec, r->cs));
    }
    A->step += (uint64_t)n_steps;
    B->step += (uint64_t)n_steps;
  }
  std::vector<double> ser((size_t)n_meas * stride);
  std::vector<int> alA(A->Nw), alB(B->Nw);
  if (n_meas > 0)
    AFQ_PCK(cudaMemcpyAsync(ser.data(), r->series, sizeof(double) * ser.size(), cudaMemcpyDeviceToHost, cs));
  AFQ_PCK(cudaMemcpyAsync(alA.data(), A->alive, sizeof(int) * A->Nw, cudaMemcpyDeviceToHost, cs));
  AFQ_PCK(cudaMemcpyAsync(alB.data(), B->alive, sizeof(int) * B->Nw, cudaMemcpyDeviceToHost, cs));
  if (n_meas > 0) {
    AFQ_PCK(cudaEventRecord(r->done, cs));
    AFQ_PCK(cudaStreamWaitEvent(s, r->done, 0));   // the caller's stream sees the whole run
  }
  AFQ_PCK(cudaStreamSynchronize(cs));
  // E_r = Re(sum w E_L / sum w) per system, measurement and repeat
  std::vector<double> E((size_t)n_meas * 2 * R), dE((size_t)n_meas * R), taus(n_meas);
  for (int m = 0; m < n_meas; ++m) {
    taus[m] = (double)(m + 1) * energy_every * A->opt.dt;
    for (int sy = 0; sy < 2; ++sy)
      for (int q = 0; q < R; ++q) {
        const double* v = ser.data() + (size_t)m * stride + sy * 4 * R + 4 * q;
        const double d2 = v[2] * v[2] + v[3] * v[3];
        E[((size_t)m * 2 + sy) * R + q] = d2 > 0 ? (v[0] * v[2] + v[1] * v[3]) / d2 : NAN;
      }
    for (int q = 0; q < R; ++q)
      dE[(size_t)m * R + q] = E[((size_t)m * 2 + 1) * R + q] - E[((size_t)m * 2) * R + q];
  }
  double est[3] = {NAN, NAN, NAN};
  if (n_meas > 0) afqmc_delta_E_stats(dE.data(), taus.data(), n_meas, R, tau_eq, nullptr, nullptr, est);
  if (e_series && n_meas > 0)
    AFQ_PCK(cudaMemcpy(e_series, E.data(), sizeof(double) * E.size(), cudaMemcpyDefault));
  if (dE_mean) AFQ_PCK(cudaMemcpy(dE_mean, &est[0], sizeof(double), cudaMemcpyDefault));
  if (dE_sigma) AFQ_PCK(cudaMemcpy(dE_sigma, &est[1], sizeof(double), cudaMemcpyDefault));
  if (tau_at_min) AFQ_PCK(cudaMemcpy(tau_at_min, &est[2], sizeof(double), cudaMemcpyDefault));
#undef AFQ_PCK
  afqmc_status tcs = afq::pair_check(A);
  if (tcs == AFQMC_OK) tcs = afq::pair_check(B);
  if (tcs != AFQMC_OK) return tcs;
  int na = 0, nb = 0;
  for (int a : alA) na += a != 0;
  for (int b : alB) nb += b != 0;
  if (na == 0 || nb == 0) return fail(A, B, AFQMC_ERR_NUMERIC, "every walker of a system is dead");
  return AFQMC_OK;
}

extern "C" afqmc_status afqmc_pair_graph_kernels(afqmc_handle A, int* n_kernels) {
  if (!A || !n_kernels) return AFQMC_ERR_ARG;
  const Res* r = static_cast<const Res*>(A->pair_cache);
  *n_kernels = r ? r->n_kernels : 0;
  return AFQMC_OK;
}

extern "C" afqmc_status afqmc_pair_run_form(afqmc_handle A, int* form) {
  if (!A || !form) return AFQMC_ERR_ARG;
  const Res* r = static_cast<const Res*>(A->pair_cache);
  *form = r ? r->form : -1;
  return AFQMC_OK;
}
