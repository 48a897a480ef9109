/*
 * afqmc.h -- C ABI of the GB300 (sm_103a) correlated-sampling phaseless AFQMC
 * walker-propagation library.
 *
 * Method: Shee, Zhang, Reichman, Friesner, "Chemical transformations approaching
 * chemical accuracy via correlated sampling in auxiliary-field quantum Monte
 * Carlo" (arXiv:1703.01545).  Section and equation numbers below refer to it.
 *
 * Conventions shared by every entry point
 *  - Every function returns an afqmc_status; nothing aborts, exits or prints.
 *    After a failure on a handle, afqmc_last_error(h) gives a one-line message.
 *  - Real matrices are row-major float64.  Complex arrays are planar: the real
 *    parts of all elements first, then the imaginary parts ("[2][...]").
 *  - Any pointer argument may be a host pointer or a device pointer of the
 *    current device (unified addressing decides; host memory may be pageable).
 *  - Work is issued on the caller's stream and is asynchronous unless stated.
 *    Outputs written to host memory are complete when the call returns.
 *  - Orbital index i, j < M; Cholesky index g < X (X = number of vectors);
 *    electron column n < N = N_up + N_dn, spin-up columns first.
 *  - Ownership: afqmc_setup copies every input into library-owned device
 *    memory; the caller may free its copies on return.  The library owns its
 *    device workspaces until afqmc_destroy.  Output buffers are caller-owned.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AFQMC_OK = 0,
  AFQMC_ERR_ARG = 1,      /* invalid argument (sizes, null pointers, mismatched pair)       */
  AFQMC_ERR_CUDA = 2,     /* a CUDA runtime call or kernel launch failed                     */
  AFQMC_ERR_NUMERIC = 3,  /* singular trial overlap at setup, every walker dead, or a repeat
                             with no live walker to comb                                    */
  AFQMC_ERR_STATE = 4,    /* call not valid in the handle's current state                    */
  AFQMC_ERR_TIMEOUT = 5,  /* a bounded device-side wait gave up                              */
  AFQMC_ERR_NOMEM = 6     /* device allocation failed                                        */
} afqmc_status;

/* Projection mode (Sec. II.A): phaseless (force bias + cos cut, real weights) or
 * free projection (no force bias, complex weights). */
enum { AFQMC_PHASELESS = 0, AFQMC_FREE = 1 };

/* Arithmetic of the step.  Overlap ratios, phases and weights are float64 in every mode.
 *   AFQMC_FP64:   every contraction, the determinants and MGS in float64.
 *   AFQMC_BF16X3: every product over the Cholesky index or the orbital basis runs on the
 *                 tensor cores with split operands x = hi + lo (two bf16), three MMAs per
 *                 product (hi*hi + hi*lo + lo*hi) accumulated in FP32: the force bias
 *                 (Eq. 9), V_HS (Eq. 11), the one-body half steps and the Taylor terms of
 *                 the propagator for M <= 256, N <= 32 (FP32 CUDA-core kernels otherwise)
 *                 and the two-body local energy (the FP32 kernel where the tensor-core one
 *                 does not apply).  Walkers are kept in float64 and float32; the
 *                 overlap-and-Theta kernel (overlap sums, LU, Theta solves) and the
 *                 orthonormalisation (Cholesky QR: Gram matrix and factor) work in FP32,
 *                 with the log-determinants formed and kept in float64 (or Gram-Schmidt in
 *                 float64; select_kernel K_MGS). */
enum { AFQMC_FP64 = 0, AFQMC_BF16X3 = 1 };

typedef struct afqmc_ctx* afqmc_handle;

typedef struct {
  double dt;          /* imaginary-time step in Ha^-1 (> 0)                                 */
  int n_walkers;      /* walkers of this system, Nw >= 1                                    */
  int taylor_order;   /* order n of the Taylor exponential T_n(A) = sum_{m<=n} A^m/m!, >= 1 */
  int precision;      /* AFQMC_FP64 or AFQMC_BF16X3                                        */
  int mode;           /* AFQMC_PHASELESS or AFQMC_FREE                                      */
  int n_repeats;      /* R >= 1 independent repeats; walker k belongs to repeat k*R/Nw      */
  uint64_t seed;      /* key of the counter-based field stream                              */
  double fb_cap;      /* |xbar_g| above fb_cap is scaled back to fb_cap; <= 0 disables      */
  int64_t walker_offset; /* global pair index of walker 0 (replicas on several GPUs take
                            disjoint ranges of k); 0 <= walker_offset, + Nw <= 2^32          */
  int autotune;       /* AFQMC_BF16X3 only: 1 = time the kernel variants at setup on this
                         handle's buffers and keep the fastest (default), 0 = defaults    */
  const char* autotune_cache; /* NULL, or a JSON file of tuned choices keyed by kernel and
                         shape; read at setup, rewritten when a new shape was timed        */
  int independent_fields; /* 0 (default): afqmc_pair_delta_E requires equal seeds, so walker
                         k of both systems draws the same fields (correlated sampling);
                         1 on both handles of a pair: the seeds must differ and each system
                         draws its own fields (the uncorrelated comparison of Sec. III)    */
} afqmc_options;

typedef struct {
  int M, X, n_up, n_dn, n_walkers, n_repeats;
  uint64_t step;      /* propagation steps taken since setup / afqmc_set_walkers            */
  double e_trial;     /* E_T = E_L(psi_T), the trial (HF) energy used as the energy shift   */
  double c_mf;        /* C = -1/2 sum_g <rho_g>_T^2, scalar of the one-body part H_1        */
  int n_alive;        /* live walkers (synchronises the stream)                             */
  int tuned_energy_walkers_per_cta; /* local-energy kernel of the split-precision step: 0 =
                                       tensor cores, 2/4/8 = FP32 kernel with that many walkers
                                       per CTA, -1 = not tuned (tensor cores where supported) */
  int tuned_taylor_smem;            /* propagation variant of the split-precision step: 4 =
                                       tensor cores with V_HS streamed (M <= 256), 3 = tensor
                                       cores (M <= 64), 2 = fused FP32 kernel, 1 / 0 = Taylor
                                       kernel with A in shared memory / through L1, -1 = not
                                       tuned */
  int tuned_orthonormalise;         /* orthonormalisation of the split-precision step: 1 =
                                       Cholesky QR, 0 = modified Gram-Schmidt kernels, -1 = not
                                       tuned (Gram-Schmidt)                                  */
  int n_det;                        /* determinants of a multi-determinant trial; 0 for a
                                       single-determinant trial                             */
} afqmc_info;

/* Fill *o with dt = 0.01, n_walkers = 128, taylor_order = 6, FP64, phaseless,
 * n_repeats = 1, seed = 1, fb_cap = 1.0, walker_offset = 0, autotune = 1,
 * autotune_cache = NULL, independent_fields = 0. */
void afqmc_default_options(afqmc_options* o);

const char* afqmc_status_string(afqmc_status s);

/* Message of the last failure on h (empty string if none).  Never NULL. */
const char* afqmc_last_error(afqmc_handle h);

/*
 * afqmc_setup -- Sec. II.A, Eqs. 1-2.  Creates a system from the Hamiltonian
 *   H = sum_ij h1_ij sum_s c+_is c_js + 1/2 sum_ijkl V_ijkl sum_st c+_is c+_jt c_lt c_ks,
 *   V_ijkl = sum_g L^g_ik L^g_jl,
 * and a single-determinant trial.  On the device it forms <rho_g>_T, the one-body
 * matrix K = h1 - 1/2 sum_g L_g L_g + sum_g <rho_g>_T L_g of H_1, exp(-dt K/2),
 * C, the half-rotated tensors Psi_s^T L_g and Psi_s^T h1, the packed transposed
 * Cholesky tensor, E_T, and initialises every walker to the trial with weight 1.
 *   h1    [M][M] symmetric.
 *   L     [X][M][M], each L_g symmetric.
 *   trial [M][N] = [Psi_up | Psi_dn], real, orthonormal columns within each spin.
 *   M >= 1, X >= 1, 1 <= N, 0 <= n_up, n_dn <= min(M, 32).
 * Synchronises the stream.  Errors: ARG (sizes, nulls, options), NUMERIC (trial has
 * zero overlap with itself), NOMEM, CUDA.  *out is NULL on failure.
 */
afqmc_status afqmc_setup(afqmc_handle* out, const double* h1, const double* L,
                         const double* trial, int M, int X, int n_up, int n_dn,
                         const afqmc_options* opt, cudaStream_t stream);

/*
 * afqmc_setup_multidet -- Sec. II.D and the truncated CASSCF trials of Sec. III: a system
 * whose trial is a multi-determinant expansion psi_T = sum_d c_d D_d.  The walkers are
 * propagated exactly as with one determinant; every mixed quantity is a sum over the
 * determinants weighted by their shares w_d = c_d O_d / <psi_T|phi>, O_d = <D_d|phi>:
 *   <psi_T|phi> = sum_d c_d O_d (importance function, overlap ratio and phase),
 *   force bias from G = sum_d w_d G_d (Eq. 9), local energy E_L = sum_d w_d E_L,d (Eq. 7).
 * <rho_g>_T, K, C and E_T are those of the first determinant D_0 (a constant background is
 * exact under the force-bias reweighting; E_T cancels in every mixed estimate).
 *   dets   [n_det][M][N], each [D_up | D_dn] real with orthonormal columns per spin; host
 *          or device memory, copied.
 *   coeffs [n_det] real CI coefficients (host or device), finite, not all zero.
 *   start  [M][N] initial determinant of every walker (host or device), or NULL for D_0.
 *          A determinant with O_d = 0 contributes nothing (its Green's function would need
 *          cofactor formulas), so start should overlap every D_d: a walker sitting on one
 *          determinant of an orthonormal expansion is orthogonal to all the others.
 *   1 <= n_det <= 4096; the other arguments as afqmc_setup.  FP64 only (ARG for
 *   AFQMC_BF16X3); afqmc_set_tangent and afqmc_adjoint_run refuse these handles (ARG).
 * Memory grows with n_det: Theta_d and the force bias of every determinant, n_det *
 * 2 Nw (N M + X) doubles.  Synchronises the stream.  Errors: ARG, NUMERIC (a walker's
 * start has zero overlap with psi_T), NOMEM, CUDA.  *out is NULL on failure.
 */
afqmc_status afqmc_setup_multidet(afqmc_handle* out, const double* h1, const double* L,
                                  const double* dets, const double* coeffs, int n_det,
                                  const double* start, int M, int X, int n_up, int n_dn,
                                  const afqmc_options* opt, cudaStream_t stream);

/* Release every device buffer of h.  h may be NULL. */
afqmc_status afqmc_destroy(afqmc_handle h);

/*
 * afqmc_set_walkers -- replace the population (e.g. to seed a secondary system
 * from another one's determinants).  phi [2][Nw][M][N] planar complex; w [2][Nw]
 * planar complex (imaginary part ignored in phaseless mode), or NULL for w = 1.
 * Walkers with w == 0 are dead.  Resets the step counter to 0 and recomputes
 * log <psi_T|phi>.  Errors: ARG, CUDA.
 */
afqmc_status afqmc_set_walkers(afqmc_handle h, const double* phi, const double* w,
                               cudaStream_t stream);

/*
 * afqmc_set_step -- checkpoint/resume, no counterpart in the paper.  Sets the step counter
 * t, the time index of the counter-based field stream x_{t,k,g} that the next propagation
 * step draws from.  With afqmc_get_state and
 * afqmc_set_walkers this resumes a run from a checkpoint: the state between steps is
 * (Phi, w, t) for a given seed and walker offset, so a handle restored at a step right after
 * an orthonormalisation continues along the same fields as the run that wrote it.  FP64
 * handles then continue bit for bit, because log O and Theta are recomputed from Phi in both.
 * Split-precision handles continue within rounding: they lower log O by log det R at
 * orthonormalisation instead.  Asynchronous on the stream.  Errors: ARG (h NULL), CUDA.
 */
afqmc_status afqmc_set_step(afqmc_handle h, uint64_t step, cudaStream_t stream);

/*
 * afqmc_population_control -- population control of the preliminary equilibration scheme
 * (Sec. II.C), applied to the primary system while it equilibrates alone.  It is the comb:
 * within each repeat r, the n walkers' weights are summed left to right (a dead walker counts
 * 0; W is the last running sum), and walker j of the repeat becomes a copy of the first walker
 * whose running sum exceeds (j + u[r]) W / n.  Every copy has weight W / n and is alive; the
 * copies' Theta and log O are recomputed from Phi.
 *   u [R] uniforms in [0, 1), host or device, drawn by the caller.
 * Phaseless handles only (ARG otherwise).  Synchronises the stream.  Errors: ARG, STATE
 * (tangent mode), NUMERIC (a repeat with no live walker; the walkers are left unchanged), CUDA.
 */
afqmc_status afqmc_population_control(afqmc_handle h, const double* u, cudaStream_t stream);

/*
 * afqmc_seed_secondary -- second stage of the preliminary equilibration scheme (Sec. II.C):
 * the secondary system B starts from the equilibrated walkers of the primary A.  Walker k of
 * B takes the first N_up^B columns of walker k's spin-up block and the first N_dn^B columns
 * of its spin-down block (an ion seeded from the neutral loses the last occupied trial
 * orbital of a spin).  Its weight is w_A |R| max(0, cos arg R), R = <psi_T^B|phi_B> /
 * <psi_T^A|phi_A>: the ratio rescales the importance sampling to B's trial, with the phase
 * projected as in the phaseless step.  B's step counter is set to A's, so
 * afqmc_pair_delta_E(A, B, ...) continues both on the shared fields.
 * Requirements: same M, walkers and repeats, N_s^B <= N_s^A, phaseless handles.
 * Asynchronous on the stream.  Errors: ARG, STATE (tangent mode), CUDA.
 */
afqmc_status afqmc_seed_secondary(afqmc_handle B, afqmc_handle A, cudaStream_t stream);

/*
 * afqmc_get_state -- copy the population out.  Any output may be NULL.
 *   phi  [2][Nw][M][N]  walker determinants
 *   logO [2][Nw]        log <psi_T|phi_k> (branch of the imaginary part unspecified)
 *   w    [2][Nw]        weights
 *   alive [Nw]          1 live, 0 dead
 * Synchronises the stream.
 */
afqmc_status afqmc_get_state(afqmc_handle h, double* phi, double* logO, double* w,
                             int* alive, cudaStream_t stream);

afqmc_status afqmc_get_info(afqmc_handle h, afqmc_info* info, cudaStream_t stream);

/*
 * afqmc_propagate -- Eqs. 3-5, 8-9, 11 and the hybrid weight of Sec. II.D; n_steps
 * steps of every walker.  Per step and walker k:
 *   xbar_g = -i sqrt(dt) (rhobar_g - <rho_g>_T)            (Eq. 9, capped by fb_cap)
 *   c_g = x_g - xbar_g,  A = i sqrt(dt) sum_g c_g L_g,  s = exp(-i sqrt(dt) sum_g c_g <rho_g>_T)
 *   phi' = e^{-dt K/2} T_n(A) e^{-dt K/2} phi
 *   R = s <psi_T|phi'>/<psi_T|phi>,  I = R exp(x.xbar - xbar.xbar/2) exp(-dt (C - E_T))
 *   phaseless: w <- w |I| max(0, cos arg R), w <= 0 kills the walker for good;
 *   free:      w <- w I (xbar = 0).
 * fields: NULL draws x_{t,k,g} ~ N(0,1) from Philox-4x32-10 with key (seed low, seed
 *   high 32 bits), counter (g/2, k, t, 0), k = walker_offset + walker, and Box-Muller
 *   (u1 = (top 53 bits of words 1:0, + 1) 2^-53, u2 = (top 53 bits of words 3:2) 2^-53,
 *   x_{2j} = sqrt(-2 ln u1) cos(2 pi u2), x_{2j+1} = sqrt(-2 ln u1) sin(2 pi u2));
 *   otherwise [n_steps][Nw][X] explicit fields.  Dead walkers are carried through the
 *   batched arithmetic but their determinants and weights no longer change.
 * Errors: ARG, CUDA.  In AFQMC_BF16X3 mode an expired bounded wait inside a tensor-core
 * kernel is reported as TIMEOUT by the next call that synchronises (energy with host
 * outputs, get_state, get_info, pair_delta_E).
 */
afqmc_status afqmc_propagate(afqmc_handle h, int n_steps, const double* fields,
                             cudaStream_t stream);

/* afqmc_orthonormalise -- Sec. II.D: modified Gram-Schmidt of each spin block of
 * every live walker (columns in order), Phi -> Phi R^{-1}; log <psi_T|phi> follows
 * (recomputed, or in AFQMC_BF16X3 mode lowered by log det R = sum_j log R_jj; Theta =
 * Phi (Psi_T^T Phi)^{-1} is unchanged by it).  The weights are unchanged.  Errors: CUDA. */
afqmc_status afqmc_orthonormalise(afqmc_handle h, cudaStream_t stream);

/*
 * afqmc_energy -- Eqs. 6-7 and 10.  Local energies
 *   E_L = sum_s tr(h1 G_s) + 1/2 sum_g [ (sum_s tr(L_g G_s))^2 - sum_s tr(L_g G_s L_g G_s) ]
 * with the mixed Green's function G_s; and per repeat r the mixed estimate
 *   E_r = sum_k w_k Re E_L,k / sum_k w_k       (phaseless)
 *   E_r = Re( sum_k w_k E_L,k / sum_k w_k )    (free projection).
 *   e_local [2][Nw] or NULL;  e_mixed [R] or NULL;  w_sum [R] (Re sum_k w_k) or NULL.
 * Synchronises the stream when any output is host memory.  Errors: ARG, CUDA.
 */
afqmc_status afqmc_energy(afqmc_handle h, double* e_local, double* e_mixed, double* w_sum,
                          cudaStream_t stream);

/*
 * afqmc_pair_delta_E -- Sec. II.B.  Correlated sampling of two systems: walker k
 * of A and walker k of B draw the same x_{t,k,g} for every g both have (systems
 * with different X share the first min(X_A, X_B) fields).  No population control;
 * each system keeps its own force bias and mean field.  Runs n_steps steps of both
 * systems; every mgs_every steps orthonormalises, every energy_every steps measures
 * (order: propagate, orthonormalise, measure).  One measurement block of both systems
 * (A and B on two concurrent branches) is captured once as a CUDA graph and cached on A.
 * By default that block is the body of a device-side while loop, so the whole run is one
 * graph launch: the block's last kernel counts the blocks and ends the loop after
 * n_steps / energy_every of them (afqmc_select_kernel AFQMC_K_PAIR_LOOP 0 launches the
 * block graph once per block instead; both give identical results).  Requirements: same seed, Nw, R, dt, mode and
 * step counter on both handles; the step counter a multiple of energy_every;
 * energy_every a multiple of mgs_every; n_steps a multiple of energy_every.  With
 * independent_fields = 1 on both handles the seeds must differ instead: each system then
 * draws its own fields and the same statistics measure uncorrelated sampling.
 * Outputs (host or device, any may be NULL):
 *   e_series [n_meas][2][R]   E_A,r and E_B,r at each measurement
 *   dE_mean, dE_sigma, tau_at_min: mean and standard error (over the R repeats) of
 *     the cumulative averages of dE = E_B - E_A over measurements with tau >= tau_eq,
 *     at the tau (relative to the start of this call) where the error is smallest,
 *     earliest on ties (Sec. II.B).  sigma is NaN when R == 1.
 * Synchronises the stream.  Errors: ARG, STATE, NUMERIC (all walkers of a system
 * dead), CUDA.
 */
afqmc_status afqmc_pair_delta_E(afqmc_handle A, afqmc_handle B, int n_steps,
                                int energy_every, int mgs_every, double tau_eq,
                                double* e_series, double* dE_mean, double* dE_sigma,
                                double* tau_at_min, cudaStream_t stream);

/*
 * afqmc_pair_graph_kernels -- instrumentation, no counterpart in the paper.  *n_kernels =
 * the kernel launches in one measurement block of the pair graph that afqmc_pair_delta_E
 * captured and cached on A (A as its first handle): energy_every steps of both systems,
 * their orthonormalisations and measurement.  0 when no graph is cached.  Host only; does
 * not synchronise.  Errors: ARG (null pointer), CUDA.
 */
afqmc_status afqmc_pair_graph_kernels(afqmc_handle A, int* n_kernels);

/*
 * afqmc_pair_run_form -- instrumentation, no counterpart in the paper.  *form = 1 when the
 * pair graph cached on A runs the whole call as one graph launch (device-side loop over the
 * measurement blocks), 0 when it is launched once per block, -1 when no graph is cached.
 * Host only.  Errors: ARG (null pointer).
 */
afqmc_status afqmc_pair_run_form(afqmc_handle A, int* form);

/*
 * afqmc_set_tangent -- tangent-mode (forward) derivative along a one-body perturbation
 * h1 -> h1 + lambda P of Eq. 1, with the fields and the trial held fixed: the paper has no
 * derivative; this gives d/dlambda of the mixed estimate of Eq. 7 (with Eq. 10) along one
 * field realisation.  P [M][M] symmetric, host or device; NULL switches tangent mode off.
 * FP64 phaseless handles only (ERR_ARG otherwise).  Resets dPhi = 0 and d log w = 0.
 * While on, afqmc_propagate and afqmc_orthonormalise also advance the tangents:
 *   e^{-dt K/2} -> its Frechet derivative along -dt P/2 (2M x 2M block exponential),
 *   Taylor terms by the product rule, d log O = tr(O^{-1} Psi^T dPhi),
 *   dTheta = (dPhi - Theta Psi^T dPhi) O^{-1}, the force bias through its cap,
 *   d log w += Re d log I - tan(arg R) Im d log R while cos(arg R) > 0 (0 once dead),
 *   Gram-Schmidt applies its column operations to dPhi.
 * afqmc_pair_delta_E refuses tangent handles (STATE).  Synchronises.
 * Errors: ARG, NOMEM, CUDA.
 */
afqmc_status afqmc_set_tangent(afqmc_handle h, const double* P, cudaStream_t stream);

/* afqmc_energy_tangent -- per repeat r: e_mixed[r] = sum w Re E_L / sum w and
 * de_mixed[r] = its d/dlambda; de_local [2][Nw] (or NULL): dE_L of every walker.
 * Synchronises.  Errors: STATE (tangent mode off), CUDA. */
afqmc_status afqmc_energy_tangent(afqmc_handle h, double* de_local, double* e_mixed,
                                  double* de_mixed, cudaStream_t stream);

/* afqmc_get_tangent_state -- d log w [Nw] of every walker.  Synchronises. */
afqmc_status afqmc_get_tangent_state(afqmc_handle h, double* dlogw, cudaStream_t stream);

/*
 * afqmc_adjoint_run -- reverse-mode (adjoint) derivative of one run's mixed energy with
 * respect to every entry of h1 (Eq. 1), with the fields and the trial held fixed: the paper
 * has no derivative.  Runs n_steps FP64 phaseless steps of the handle's walkers (Eqs. 3-5,
 * 8-9, 11 and the hybrid weight of Sec. II.D), orthonormalising after every step t with
 * (t + 1) % mgs_every == 0 (0: never) and measuring after every step with
 * (t + 1) % energy_every == 0, t counted from the first step of this call, and returns
 *   *e_mixed = mean over the measurements of sum_k w_k Re E_L,k / sum_k w_k  (Eqs. 7, 10),
 *   dE_dh1 [M][M] row-major (host or device) = dE/dh1_ij, the M^2 entries taken as
 *   independent (contracting with a symmetric P gives the tangent-mode derivative along P).
 * The forward pass keeps the walker state (Phi, log O, w, alive) every `checkpoint` steps;
 * the reverse pass recomputes one segment at a time from its checkpoint, so device memory
 * grows as (n_steps / checkpoint + checkpoint) walker states.  fields: as afqmc_propagate
 * ([n_steps][Nw][X], host or device) or NULL for the Philox stream from the handle's current
 * step.  The handle ends in the state after the n_steps steps (step counter advanced), as if
 * afqmc_propagate and afqmc_orthonormalise had run.  Walkers that die get no adjoint flow
 * past the step that killed them (the derivative of the branch that is taken).
 * Requires precision AFQMC_FP64, mode AFQMC_PHASELESS, n_repeats == 1, tangent mode off,
 * 1 <= energy_every <= n_steps, checkpoint >= 1.  Synchronises.
 * Errors: ARG, STATE (tangent mode on), NOMEM, NUMERIC (no live walker at a measurement),
 * CUDA.
 */
afqmc_status afqmc_adjoint_run(afqmc_handle h, int n_steps, const double* fields, int mgs_every,
                               int energy_every, int checkpoint, double* e_mixed,
                               double* dE_dh1, cudaStream_t stream);

/*
 * afqmc_delta_E_stats -- host-only statistics of Sec. II.B (no GPU needed).
 *   dE [n_meas][R] energy differences per measurement and repeat, taus [n_meas].
 *   mean_tau, se_tau [n_meas] (may be NULL): mean and standard error sd/sqrt(R) per tau.
 *   est [3]: mean, SE and tau of the cumulative averages (tau >= tau_eq) at the
 *   earliest minimum SE.  Errors: ARG.
 */
afqmc_status afqmc_delta_E_stats(const double* dE, const double* taus, int n_meas, int R,
                                 double tau_eq, double* mean_tau, double* se_tau,
                                 double* est);

/*
 * afqmc_time_kernel -- benchmarking aid (no counterpart in the paper).  Launches one
 * kernel of the propagation step `reps` times on `stream` with the handle's current
 * data, timed with CUDA events recorded on that stream, and stores the mean duration
 * of one launch in *ms.  which: AFQMC_K_VHS (V_HS contraction), AFQMC_K_FORCE_BIAS
 * (force-bias contraction), AFQMC_K_TAYLOR (Taylor exponential, on scratch memory),
 * AFQMC_K_EXCHANGE (local-energy kernel), AFQMC_K_OVERLAP (overlap / inverse / log det /
 * Theta kernel in its refresh form, which recomputes the same values from the current
 * walkers), AFQMC_K_OVERLAP_UPDATE (AFQMC_BF16X3 only, ERR_ARG otherwise: the same kernel in
 * the form each propagation step runs, FP32-pair overlap sums from the FP32 walkers, without
 * the weight update; one refresh afterwards restores Theta and log O), AFQMC_K_MGS (the
 * modified Gram-Schmidt pass in the form afqmc_orthonormalise runs it, with its overlap
 * update or refresh).  None of them changes the weights; none but AFQMC_K_MGS changes the
 * walkers, and AFQMC_K_MGS, applied to walkers that are already orthonormal (as after
 * afqmc_orthonormalise), changes them and log O only by rounding.
 * Synchronises the stream.  Errors: ARG, CUDA.
 */
enum { AFQMC_K_VHS = 0, AFQMC_K_FORCE_BIAS = 1, AFQMC_K_TAYLOR = 2, AFQMC_K_EXCHANGE = 3,
       AFQMC_K_OVERLAP = 4, AFQMC_K_OVERLAP_UPDATE = 5, AFQMC_K_MGS = 6,
       AFQMC_K_PAIR_LOOP = 7 /* afqmc_select_kernel only */ };
afqmc_status afqmc_time_kernel(afqmc_handle h, int which, int reps, double* ms,
                               cudaStream_t stream);

/*
 * afqmc_select_kernel -- testing and benchmarking aid (no counterpart in the paper): fixes
 * the variant of a tunable kernel of the split-precision step, overriding the autotuner.
 *   which AFQMC_K_EXCHANGE: variant 0 = tensor-core local energy, 2 / 4 / 8 = FP32 kernel
 *                           with that many walkers per CTA;
 *   which AFQMC_K_TAYLOR:   the propagation e^{-dt K/2} e^A e^{-dt K/2}: variant 4 = split-BF16
 *                           tensor-core kernel over V_HS streamed as split BF16 by TMA
 *                           (M <= 256, N <= 32), 3 = split-BF16 tensor-core kernel (M <= 64,
 *                           N <= 16), 2 = one fused FP32 kernel per walker, 0 / 1 = two FP32
 *                           GEMMs around a Taylor kernel reading A through L1 (0) or from
 *                           shared memory (1);
 *   which AFQMC_K_MGS:      the orthonormalisation: 1 = Cholesky QR (Gram matrix, R and Q
 *                           in FP32, log det R in FP64), 0 = modified Gram-Schmidt in FP64;
 *   which AFQMC_K_PAIR_LOOP (either precision; applies to runs with h as the first handle
 *                           of afqmc_pair_delta_E): 1 = the whole run as one graph launch
 *                           with a device-side loop over the measurement blocks (default),
 *                           0 = one launch of the block graph per measurement block.
 * The kernel choices show in afqmc_get_info.  Errors: ARG (FP64 handle for a kernel
 * variant, unknown kernel, or a variant this shape does not support).
 */
afqmc_status afqmc_select_kernel(afqmc_handle h, int which, int variant);

/*
 * afqmc_local_energy_static -- local energies E_L of the walkers phi, like
 * afqmc_energy's e_local, for callers that cannot allocate device memory (code
 * inside another framework's memory pool or under a fixed memory budget, or an
 * embedding that only hands over existing device buffers).  The paper has no
 * counterpart: this is a deployment variant of the energy evaluation.
 * It needs no handle and allocates nothing: its intermediates live in one 32 MiB
 * static device array that every GPU loading this library holds until the process
 * exits; walkers are processed in chunks that fit it.  All pointers must be device
 * memory of the current device (ERR_ARG otherwise):
 *   h1 [M][M], L [X][M][M], trial [M][N] as in afqmc_setup; phi [2][Nw][M][N];
 *   e_local [2][Nw] (real parts, then imaginary parts).
 * Problems whose fixed part (X*N*M + 2*N*M doubles plus one walker) exceeds the
 * array are rejected with ERR_ARG before anything is launched.
 * A walker whose overlap with the trial is singular (or not finite) has no local
 * energy: both of its e_local entries are set to NaN while the call still returns OK;
 * the other walkers are unaffected.
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.
 * Asynchronous on `stream`.  Every call shares the one array, so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race; serialise
 * them.  Errors: ARG, CUDA.
 */
afqmc_status afqmc_local_energy_static(const double* h1, const double* L, const double* trial,
                                       const double* phi, int M, int X, int n_up, int n_dn,
                                       int n_walkers, double* e_local, cudaStream_t stream);

/*
 * afqmc_test_gemm -- testing aid (no counterpart in the paper): one of the library's
 * contraction kernels on given operands, C[n][m] = alpha sum_k A[m][k] B[n][k] with
 * A [Md][K], B [Nd][K] (row-major float64, host or device) and C [Nd][Md].
 * impl 0: FP64 kernel; impl 1: split-BF16 tensor-core kernel (hi/lo operands, three MMAs
 * per product, FP32 accumulation; the persistent 128 x 256-tile form from 2 x 152 tiles on,
 * as for V_HS); impl 2: self-test of the tensor-core kernel's bounded
 * waits -- its TMA producer issues nothing, so the first wait expires after 20 ms and the
 * call must return TIMEOUT with the CUDA context still usable.  Allocates temporary
 * device memory; synchronises.
 * Errors: ARG, CUDA, TIMEOUT (a bounded wait inside the tensor-core kernel expired).
 */
afqmc_status afqmc_test_gemm(int impl, int Md, int Nd, int K, const double* A, const double* B,
                             double alpha, double* C, cudaStream_t stream);

/* Flyvbjerg-Petersen reblocking error of the mean of series[n] (host only): the
 * largest block-level estimate among levels with >= 16 blocks. */
double afqmc_reblock_error(const double* series, int n);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
