/*
 * lindtebd.h -- C ABI of the batched quantum-trajectory TEBD library (sm_103a).
 *
 * The library integrates many independent quantum trajectories of the Lindblad
 * equation (Sec. 4.1, Eqs. QJump1, QJump2, MasterEq, TransitionRate) for a
 * one-dimensional chain whose histories are matrix product states in
 * Vidal-Hastings form (Sec. 2.2-2.3).  The hot operation is the two-site TEBD
 * update of Sec. 2.3 (Eq. Theta): contract Lambda_{b-1} B_b B_{b+1} with the
 * two-site gate exp(-i h_b^eff tau) into theta, take a truncated SVD back to
 * chi_max and renormalise (Sec. 2.3, Eq. TruncationErr and the normalisation
 * that follows it).  The same update serves quantum state diffusion (Sec. 5.2,
 * method LT_QSD) and the vectorised density matrix (Sec. 3.1, method LT_MPDO):
 * |rho>> = sum_ij rho_ij |i> (x) |j> (Eq. Choi) as an MPS with the local index
 * m = 2n + n' of four values (Eq. MPDO), advanced by the two-site Liouvillian
 * gates exp(tau Lv_b) (Eq. Liouvillian).  An LT_MPDO context holds n_traj
 * independent chains (one density matrix each; they share the rates).
 *
 * Conventions shared by every entry point
 *  - Sites 0..L-1, bond b joins sites b and b+1, single-site basis |0> empty,
 *    |1> occupied, two-site index s_b * 2 + s_{b+1}.
 *  - Every pointer argument is caller-owned HOST memory unless stated; inputs
 *    are copied before the call returns.  The library owns all device memory
 *    of a context (allocated in lt_create, freed in lt_destroy).
 *  - Work is queued on the context's CUDA stream; lt_measure_*, lt_get_*,
 *    lt_set_state/lt_get_state and lt_save/lt_load synchronise that stream.
 *  - Every call returns an lt_status.  LT_ERR_NUMERICAL and LT_ERR_TIMEOUT
 *    poison the context: later calls return LT_ERR_STATE until lt_destroy.
 *    No call throws, exits or traps the GPU.  lt_last_error() describes the
 *    most recent failure of a context.
 *  - Contexts are independent; one context per stream.
 */
#ifndef LINDTEBD_H
#define LINDTEBD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lt_ctx_s* lt_ctx;

typedef enum {
  LT_OK = 0,
  LT_ERR_ARG = 1,         /* invalid argument or configuration            */
  LT_ERR_OOM = 2,         /* device allocation failed                     */
  LT_ERR_CUDA = 3,        /* a CUDA runtime call failed                   */
  LT_ERR_NUMERICAL = 4,   /* theta vanished, or jump probability >= 0.5   */
  LT_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out           */
  LT_ERR_STATE = 6,       /* context poisoned by an earlier error         */
  LT_ERR_UNSUPPORTED = 7  /* method or option not built                   */
} lt_status;

typedef enum { LT_TRAJ = 0, LT_QSD = 1, LT_MPDO = 2, LT_PURIFIED = 3 } lt_method;

/* LT_FP64: every step in double precision.  LT_MIXED: site tensors stored in
 * single precision; theta formed on the tensor cores from exact products of 8-bit
 * digits (pure states; the vectorised and purified forms in single precision) and
 * rounded once; the Jacobi rotations in single precision, the kept right singular
 * vectors re-orthonormalised with norms in double; singular values, the truncation
 * weight, the renormalisation, the Schmidt values Lambda and the jump
 * probabilities in double precision. */
typedef enum { LT_FP64 = 0, LT_MIXED = 1 } lt_precision;

typedef enum {
  LT_INIT_VACUUM = 0,       /* all sites empty (Sec. 2.1 initial state)      */
  LT_INIT_NEEL = 1,         /* site i occupied iff i is even                  */
  LT_INIT_DOMAIN_WALL = 2,  /* sites 0..L/2-1 occupied                        */
  LT_INIT_PRODUCT = 3       /* occupations from product_occ                   */
} lt_init;

typedef struct {
  int32_t L;                 /* chain length, 2 <= L <= 1024                       */
  int32_t chi_max;           /* bond-dimension cap, 1 <= chi_max <= 256 (<= 128 for*/
                             /* LT_MPDO and LT_PURIFIED, whose theta is 4 chi wide)*/
  int32_t n_traj;            /* trajectories held by this context, >= 1            */
  int32_t kraus_dim;         /* LT_PURIFIED: Kraus dimension, 2 (0 selects 2); set */
                             /* 0 for the other methods                            */
  int32_t method;            /* lt_method (all four are built)                     */
  int32_t precision;         /* lt_precision                                       */
  int32_t init;              /* lt_init                                            */
  int32_t trotter_order;     /* 1: A(dt) B(dt); 2: A(dt/2) B(dt) A(dt/2)           */
  const uint8_t* product_occ;/* [L] 0/1, read for LT_INIT_PRODUCT only; copied      */
  double J;                  /* hopping amplitude, H = -J sum (c+_{i+1} c_i + h.c.) */
  double dt;                 /* time step                                          */
  const double* gamma_loss;  /* [L] rates of L = c_i, NULL = all zero; copied       */
  const double* gamma_gain;  /* [L] rates of L = c_i^+, NULL = all zero; copied     */
  const double* gamma_deph;  /* [L] rates of L = n_i, NULL = all zero; copied       */
  int32_t fermionic_jumps;   /* 1: c_i carries the Jordan-Wigner string; 0: spin   */
  int32_t max_sweeps;        /* Jacobi sweep limit per SVD, 0 = default (40)       */
  double svd_cut;            /* keep singular values > svd_cut * largest           */
  uint64_t seed;             /* Philox4x32-10 key                                  */
  int64_t traj_offset;       /* global id of trajectory 0 (Philox counter word 0)  */
  double jacobi_tol;         /* rotate a row pair while |x.y^+| > tol |x| |y|;     */
                             /* 0 = default eps sqrt(n) of the working precision   */
  int32_t theta_path;        /* LT_MIXED, two values per site: 0 = the tuned        */
                             /* schedule's choice, 1 = tensor cores (exact 8-bit   */
                             /* digit products, error below the final rounding),   */
                             /* 2 = single-precision FMAs                          */
  int32_t env_ctas_per_sm;   /* CTAs per SM of the environment kernels (rates and  */
                             /* observables): 0 = tuned, 1..8                      */
} lt_config;

/* Schedules.  The fields theta_path and env_ctas_per_sm left at 0 take
 * the values of a table the library carries, written by the autotuner
 * (paper_2609_18841_b300/autotune.py) from timings on the device: for each number of
 * values per site (2 or 4), precision and chi_max (the smallest tabulated chi_max at
 * or above the context's), the candidate schedule with the shortest time step.
 * Without an entry: tensor cores, up to 8 CTAs per SM. */

/* Create a context: validate cfg, allocate the ensemble on the current device
 * and set every trajectory to the initial product state (Sec. 4.1: the
 * initial pure state is an eigenvector of rho(0), here a product state); an
 * LT_MPDO chain starts from rho = |n><n| of that product state (local index
 * 3 n_i on every site), an LT_PURIFIED chain from X = |n> with Kraus index 0
 * (s = 2 n_i).  LT_ERR_UNSUPPORTED: LT_MPDO or LT_PURIFIED with chi_max > 128,
 * LT_PURIFIED with kraus_dim other than 0 or 2, either with fermionic loss or
 * gain on a bulk site (on the chain
 * ends the Jordan-Wigner string acts as the total parity, which commutes with
 * every state reached from a product state, so c and c^+ act there as the
 * local sigma- and sigma+; in the bulk they would not be local).
 * stream: a cudaStream_t, or NULL for a stream the context creates and owns.
 * On success *out holds the context; on failure *out is NULL. */
lt_status lt_create(const lt_config* cfg, void* stream, lt_ctx* out);

/* Free every device buffer of the context (and its stream if it owns one). */
lt_status lt_destroy(lt_ctx ctx);

/* One Trotter layer (Sec. 2.3): apply G_b(tau) = exp(-i h_b^eff tau) by the
 * two-site update at every bond b with b % 2 == parity, for every trajectory
 * not marked as jumped by the last lt_apply_jumps (all trajectories before
 * the first call).  h_b^eff carries half of each bulk site's dissipator
 * -(i/2) sum_k gamma_k L_k^+ L_k and the whole of an end site's (Eq.
 * EffHamiltonian, split as in Eq. LindbladLocal).  Gates are built on the host
 * in double precision once per distinct tau.  In an LT_MPDO context the gate
 * is the 16 x 16 matrix exp(tau Lv_b) over (m_b, m_{b+1}) with
 * Lv_b = -i(h_b (x) 1 - 1 (x) h_b^T) + the same weighted site dissipators
 * sum_k gamma_k [L_k (x) conj(L_k) - 1/2 L_k^+L_k (x) 1 - 1/2 1 (x) (L_k^+L_k)^T]
 * (Eq. Liouvillian, with the conjugate and transpose that the vectorisation
 * gives), and the update renormalises the Hilbert-Schmidt norm of |rho>>, so
 * its scale is arbitrary and every observable is a ratio to Tr rho. */
lt_status lt_apply_layer(lt_ctx ctx, int32_t parity, double tau);

/* Jump-or-evolve decision of time step `step` (Sec. 4.1): for every
 * trajectory compute W_k = gamma_k <L_k^+ L_k> for the channels k = 3 * site
 * + kind (kind 0 loss, 1 gain, 2 dephasing; Eq. TransitionRate) with exact
 * environment contractions, draw r from Philox4x32-10 with counter
 * (traj_offset + traj, step, 0, step >> 32) and key seed, and jump iff
 * r < P = sum_k W_k dt, to the least channel whose cumulative W dt exceeds r.
 * A jump applies L_k (and the string for fermionic loss/gain), renormalises
 * and restores the canonical form; the trajectory then skips this step's
 * layers.  replay: [n_traj] forced channels (-1 none, -2 draw), or NULL to
 * draw for every trajectory.  out_channel: [n_traj] receives the channel
 * (-1 = no jump), or NULL.  Returns LT_ERR_NUMERICAL if some P >= 0.5. */
lt_status lt_apply_jumps(lt_ctx ctx, int64_t step, const int32_t* replay,
                         int32_t* out_channel);

/* Host only (no device work): the two-site gates a context of cfg would build for
 * time step tau, as lt_apply_layer applies them.  out receives (L-1) matrices of
 * D^2 x D^2 complex entries, interleaved (re, im) doubles, bond b at
 * b * 2 D^4, row-major over (s_b, s_{b+1}) x (t_b, t_{b+1}): D = 2 for LT_TRAJ and
 * LT_QSD (exp(-i h_b^eff tau)), D = 4 for LT_MPDO (exp(tau Lv_b), Eq. Liouvillian
 * on m = 2n + n') and LT_PURIFIED (exp(-i h_b^eff tau) (x) 1 over the Kraus
 * indices, s = 2n + k).  capacity: doubles available at out (at least
 * 2 D^4 (L-1)), else LT_ERR_ARG. */
lt_status lt_gates(const lt_config* cfg, double tau, double* out, int64_t capacity);

/* Quantum state diffusion noise of time step `step` (Sec. 5.2, LT_QSD
 * contexts; LT_ERR_UNSUPPORTED otherwise).  The scheme iterates
 * |psi> <- prod_k (1 + eta_k sqrt(gamma_k dt) L_k) exp(-i H_eff dt) |psi> on
 * unnormalised histories: in an LT_QSD context lt_apply_layer keeps the norm
 * change of its non-unitary gates in the state (B_b <- theta~ V_k, no division
 * by ||S_k||), and this call then applies on every site the real 2 x 2 matrix
 * prod over the site's channels (loss, then gain, then dephasing) of
 * 1 + eta_k sqrt(gamma_k dt) L_k, with eta_k standard normal: eta_{2j} and
 * eta_{2j+1} are the Box-Muller pair of the Philox4x32-10 draw with counter
 * (traj_offset + traj, step, 1 + j, step >> 32) and key seed, k = 3 site +
 * kind.  It then restores the exact canonical form of every history (one-site
 * SVDs right to left, then left to right) and adds ln <psi|psi>, found at bond
 * 0, to the history's log weight (lt_get_log_weights).  The left-to-right pass
 * (also the one after a jump) stores Lambda_b as the norms of the columns of
 * Lambda_{b-1} B_b as stored, accumulated in double: the normalised singular
 * values in exact arithmetic, and in single precision the norm the stored
 * tensors carry.  Only site-local L_k are
 * accepted: lt_create returns LT_ERR_UNSUPPORTED for an LT_QSD context with
 * fermionic loss or gain beyond site 0 (the string would make the factor a sum
 * of non-local products). */
lt_status lt_apply_noise(lt_ctx ctx, int64_t step);

/* The R step of the locally purified density matrix (Sec. 3.2, Eqs. MatrixR,
 * NewPurified; LT_PURIFIED contexts, LT_ERR_UNSUPPORTED otherwise).  rho = X X^+
 * with X an MPS over s = 2n + k (physical n, Kraus index k, kraus_dim = 2).  On
 * every site the Kraus vectors are enlarged to A~ = [A^{.,k} ; sqrt(gamma_c dt)
 * L_c A^{.,k}] over the site's channels (loss sigma-, gain sigma+, dephasing n),
 * which turns sum_k A A^+ into the tensor R of Eq. MatrixR (rho -> rho + dt
 * sum_c gamma_c L_c rho L_c^+ on that site), and replaced by A~ V with V the two
 * leading eigenvectors of the Lambda_{i-1}-weighted Gram matrix A~^+ W^2 A~ (at
 * most 8 x 8, W the left Schmidt values: the site's environment in this gauge);
 * W A~ V are then the leading eigenvectors of W R W scaled by sqrt(lambda), the
 * paper's R taken in that environment.  In an
 * LT_PURIFIED context lt_apply_layer applies exp(-i h_b^eff tau) (x) 1 over the
 * Kraus indices and keeps the norm change (B_b <- theta~ V_k), and lt_step runs
 * the layers, then this call. */
lt_status lt_apply_kraus(lt_ctx ctx);

/* ln <psi|psi> of every unnormalised QSD history, out: [n_traj] (0 for the
 * trajectory method and after lt_set_state). */
lt_status lt_get_log_weights(lt_ctx ctx, double* out);

/* n_steps full time steps with step counting on from the context's step
 * counter (starting at 0): for LT_TRAJ lt_apply_jumps(step, NULL, NULL) then
 * the layers of the configured Trotter order; for LT_QSD the layers then
 * lt_apply_noise(step); for LT_MPDO the layers only (lt_apply_jumps and
 * lt_apply_noise return LT_ERR_UNSUPPORTED there); for LT_PURIFIED the layers
 * then lt_apply_kraus. */
lt_status lt_step(lt_ctx ctx, int32_t n_steps);

/* The same n_steps time steps as lt_step, replayed from a CUDA graph: the first
 * call uploads the schedule's gates, captures one step's launches on the
 * context's stream (their Philox step is read from a device counter that the
 * captured step advances) and instantiates it; every call then replays it
 * n_steps times.  Results are bit-identical to lt_step, and the two can be
 * interleaved (the step counter is shared).  The graph saves the host launch
 * cost of the roughly 2L + 7 kernels of a step (trajectory method), which
 * matters for small ensembles.  LT_ERR_UNSUPPORTED if the stream cannot be
 * captured (the legacy default stream). */
lt_status lt_step_graph(lt_ctx ctx, int32_t n_steps);

/* Ensemble density <n_i> = <psi|n_i|psi>/<psi|psi> (exact environments).
 * mean: [L] average over trajectories; sem: [L] CLT error sqrt(var/n_traj)
 * (Eq. ErrorCLT), or NULL; per_traj: [n_traj * L] row-major, or NULL.  For
 * LT_QSD the ensemble quantities average w_t <n_i>_t with w_t = <psi_t|psi_t>
 * (the mean of |psi><psi| over unnormalised histories, Sec. 5.2), while
 * per_traj holds the normalised <n_i>_t.  For LT_MPDO per_traj holds each
 * chain's Re Tr(n_i rho) / Tr rho, the traces contracting |rho>> with the
 * vectors o[2n + n'] = O[n', n] of each site's operator, and mean/sem run over
 * the chains.  For LT_PURIFIED per_traj holds Tr(n_i X X^+) / Tr(X X^+) =
 * <X| n_i (x) 1 |X> / <X|X> by exact environments. */
lt_status lt_measure_density(lt_ctx ctx, double* mean, double* sem, double* per_traj);

/* Correlation matrix C_ij = <c_i^+ c_j> (Sec. 2.1) by transfer matrices with
 * the Jordan-Wigner string.  C_re/C_im: [L * L] row-major ensemble mean
 * (weighted as for the density in LT_QSD contexts); per_traj_re/per_traj_im:
 * [n_traj * L * L] normalised, or NULL.  For LT_MPDO C_ij = Tr(c_i^+ c_j rho) /
 * Tr rho for i < j, C_ji = conj(C_ij), C_ii = <n_i>. */
lt_status lt_measure_corr(lt_ctx ctx, double* C_re, double* C_im,
                          double* per_traj_re, double* per_traj_im);

/* trunc_weight: [n_traj] accumulated discarded weight sum_{a>k} S_a^2 / sum S^2
 * (Eq. HilbertSchmidtNorm), or NULL.  bond_dims: [n_traj * (L-1)] or NULL. */
lt_status lt_get_stats(lt_ctx ctx, double* trunc_weight, int32_t* bond_dims);

/* Replace / read trajectories traj0 .. traj0+n-1.  Layout per trajectory:
 * dims [L-1] int32; lam [(L-1) * chi_max] double, bond b at b * chi_max;
 * B [L * d * chi_max^2] complex128 as interleaved (re, im) doubles, site i at
 * i * d * chi_max^2, holding B_i[a][s][c] row-major over its actual shape
 * (chi_{i-1}, d, chi_i), d = 2 (d = 4 for LT_MPDO, s the local index
 * m = 2n + n', and for LT_PURIFIED, s = 2n + k).  Dimensions must satisfy
 * 1 <= chi_b <= chi_max.
 * lt_set_state also clears the truncation accumulators and the log weights of
 * those trajectories. */
lt_status lt_set_state(lt_ctx ctx, int32_t traj0, int32_t n, const int32_t* dims,
                       const double* lam, const double* B);
lt_status lt_get_state(lt_ctx ctx, int32_t traj0, int32_t n, int32_t* dims,
                       double* lam, double* B);

/* Checkpoint / resume: write or read the whole ensemble, the step counter, the
 * truncation accumulators and the log weights to or from a file (format
 * LTCKPT02; the method, precision and sizes must match the context).  Philox draws are keyed by
 * (trajectory, step), so a resumed run is bit-identical to an uninterrupted one. */
lt_status lt_save(lt_ctx ctx, const char* path);
lt_status lt_load(lt_ctx ctx, const char* path);

/* Diagnostics: sweep_hist [64] receives how many SVDs took s Jacobi sweeps
 * (index s, the last bin collects s >= 63) since the context was created or
 * the histogram was last cleared; clear != 0 resets it after reading. */
lt_status lt_get_sweep_histogram(lt_ctx ctx, int32_t* sweep_hist, int32_t clear);

/* Work counters of the two-site update since creation or the last clear:
 * out[0] two-site updates executed (all), out[1] Jacobi rotations applied,
 * out[2] Jacobi row-pair inner products, out[3] algorithmic real floating-point
 * operations of the updates in Trotter layers, out[4] the same for the
 * identity-gate updates that restore the canonical form after jumps,
 * out[5] two-site updates executed in Trotter layers.  The operation count of
 * one update with theta of m x n, middle dimension chi_M, r = min(m, n), k kept
 * values and s Jacobi sweeps on the r x r preconditioned factor is
 * 4 r^2 (s + 1) + 8 r P + 24 r Rot (P = s r (r - 1) / 2 inner products, Rot
 * applied rotations) + 16 sum_{j<r} [(m-j-1)(n-j) + (m-j)(r-j-1) + k (n-j)]
 * (the Householder LQ, the QR and the application of Q1) + 8 m n (chi_M + 4) +
 * 8 m k n (theta and theta~ V_k; the one-site steps count their own
 * contractions).  clear != 0 resets the counters after reading.  out: [6] or
 * NULL. */
lt_status lt_get_counters(lt_ctx ctx, uint64_t* out, int32_t clear);

/* ---- request server (continuous batching; the paper has no serving layer) ----
 * A request is one ensemble (an lt_config, any method) run for
 * n_steps time steps.  Each admitted request owns a context and its stream on
 * the current device, so the steps of all active requests are queued side by
 * side and the GPU interleaves their kernels; the ensemble stays resident from
 * admission to retirement.  lt_server_tick (1) admits queued requests in
 * arrival order while their device footprint fits the budget and fewer than
 * max_active run (a request whose footprint exceeds the budget finishes with
 * LT_ERR_OOM), (2) queues one time step for every active request (at most two
 * in flight each) and (3) retires requests whose last step has completed: the
 * ensemble density (lt_measure_density) is kept and the context freed.
 * Results are bit-identical to running the request alone.  Not thread-safe:
 * one host thread drives a server. */
typedef struct lt_server_s* lt_server;

/* Device bytes lt_create allocates for cfg on a GPU with num_sms SMs (the
 * occupancy-dependent scratch grids bounded above): the admission estimate. */
lt_status lt_context_bytes(const lt_config* cfg, int32_t num_sms, uint64_t* out);

/* Admission rule, host only: how many of the queue head (queued_bytes[0..n_queued))
 * fit in order under budget and max_active, given used bytes and n_active. */
lt_status lt_admit_plan(uint64_t budget, uint64_t used, int32_t max_active, int32_t n_active,
                        const uint64_t* queued_bytes, int32_t n_queued, int32_t* n_admit);

lt_status lt_server_create(uint64_t hbm_budget_bytes, int32_t max_active, lt_server* out);
lt_status lt_server_destroy(lt_server server);
/* Queue a request (cfg and its arrays are copied); *out_id identifies it. */
lt_status lt_server_submit(lt_server server, const lt_config* cfg, int32_t n_steps,
                           int64_t* out_id);
/* One scheduling round; the counts after it, each may be NULL. */
lt_status lt_server_tick(lt_server server, int32_t* n_queued, int32_t* n_active,
                         int32_t* n_finished);
/* Result of a finished request: mean and sem [L] as lt_measure_density (NULL
 * allowed), times [3] = submit, admission and completion in seconds since the
 * server was created.  LT_ERR_STATE while it runs; the request's own status if
 * it failed (times are still written). */
lt_status lt_server_result(lt_server server, int64_t id, double* mean, double* sem,
                           double* times);
/* Two-site updates a request executed (its context's work counter, lt_get_counters
 * out[0]): for a finished request as read at retirement (0 if it failed), for an
 * active one so far (this synchronises its stream), 0 while it is queued. */
lt_status lt_server_updates(lt_server server, int64_t id, uint64_t* updates);
/* Why a finished request failed (the failing call and the CUDA message), "" if
 * it succeeded or is unknown; valid until the server is destroyed. */
const char* lt_server_error(lt_server server, int64_t id);
/* Device bytes held by active requests, and the budget. */
lt_status lt_server_usage(lt_server server, uint64_t* used_bytes, uint64_t* budget_bytes);

/* Allocation-free variant of the per-trajectory density measurement, for
 * callers that cannot call cudaMalloc: processes whose device memory is owned
 * by another allocator (a framework's caching allocator, or a serving runtime
 * that reserves the GPU's memory up front), where an extra cudaMalloc either
 * fails or takes memory the owner has promised elsewhere, and callers that
 * cannot accept the device-wide synchronisation cudaMalloc/cudaFree may cause.
 * The paper has no counterpart; it is an interface convenience.
 *
 * Computes <n_i> = <psi|n_i|psi>/<psi|psi> (the densities lt_measure_density
 * returns per trajectory) for an MPS ensemble the caller holds on the current
 * device, in the library's layout: B [n_traj][L][2 chi_max^2] complex
 * (float2 for LT_MIXED, double2 for LT_FP64, site i holding B_i[a][s][c]
 * row-major over its actual shape), dims [n_traj][L-1] int32 with
 * 1 <= dims <= chi_max, density [n_traj][L] double (written; a trajectory
 * with a dimension outside [1, chi_max] is skipped and its row set to NaN, the
 * kernel checking the dimensions before it reads a site).  All three are
 * DEVICE pointers owned by the caller.  Work is queued on `stream` (a
 * cudaStream_t, NULL = the legacy default stream); the call does not
 * synchronise it and calls no cudaMalloc, cudaFree or allocating routine.
 *
 * Scratch: a 32 MiB array in the library's static device memory, present on
 * every GPU that loads the library until the process exits.  One trajectory
 * needs (L + 8) * chi_max^2 complex elements of it, so the call returns
 * LT_ERR_ARG when (L + 8) chi_max^2 * 8 bytes (LT_MIXED) or * 16 bytes (LT_FP64)
 * exceeds 32 MiB (e.g. LT_FP64 with L > 504 at chi_max = 64), and LT_ERR_ARG for
 * any other invalid size or NULL pointer.  Every call looks up the array's
 * address on the current device (cudaGetSymbolAddress, which allocates
 * nothing), so no address outlives a device reset; the first call on a device
 * may load the library's device code, so make it before any stream capture.
 * Every call shares the one
 * array and the kernel writes each scratch element before reading it, so
 * nothing needs clearing between calls; calls that overlap on the GPU (on
 * different streams, or from several threads) race on it and must be
 * serialised by the caller. */
lt_status lt_measure_density_noalloc(int32_t precision, int32_t L, int32_t chi_max,
                                     int32_t n_traj, const void* B, const int32_t* dims,
                                     double* density, void* stream);

/* Roofline denominators of the SIMT pipes on the current device (the paper has no
 * counterpart; the measurement reports each kernel's arithmetic rate against them).
 * A microbenchmark of independent fused multiply-add chains held in registers,
 * four CTAs of 256 threads per SM, each kernel launched twice on an internal
 * stream and the second launch timed with CUDA events (about 0.1 s in all).
 * out[0]: single-precision TFLOP/s of packed FMA pairs (__ffma2_rn, 4 flops per
 * instruction), out[1]: double-precision TFLOP/s of scalar FMAs, out[2]: the SM
 * clock the device reports (MHz), out[3]: the number of SMs.  out: [4] host doubles.
 * Synchronises the device's work on that stream only; allocates 2 KiB. */
lt_status lt_pipe_peaks(double* out);

/* Number of kernels this context has launched so far. */
int64_t lt_launch_count(lt_ctx ctx);

/* Number of those launches made as thread-block clusters: a single-precision Trotter
 * layer with few tasks whose theta can exceed 128 x 128 (a launch of n_traj x bonds
 * tasks when that many clusters of 2, 4 or 8 CTAs fit the device at once) gives each
 * task a cluster, whose CTAs share the task's Jacobi sweeps and, when theta is no
 * taller than wide, its preconditioning, V_k^+ and split; the results are those of the
 * one-CTA launch bit for bit. */
int64_t lt_cluster_launches(lt_ctx ctx);

/* The context's CUDA stream (a cudaStream_t). */
void* lt_stream(lt_ctx ctx);

/* Current step counter of the context. */
int64_t lt_get_step(lt_ctx ctx);

const char* lt_status_str(lt_status s);
const char* lt_last_error(lt_ctx ctx);

#ifdef __cplusplus
}
#endif
#endif /* LINDTEBD_H */
