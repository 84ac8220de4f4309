// Internal declarations of the lindtebd CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lindtebd.h"

#define LT_MAX_CHI 256
#define LT_MAX_DIM 512  // largest theta side: 2 chi_max for pure states, 4 chi_max (<= 128) otherwise
// the single-precision register paths of the two-site update (row-resident
// Householder steps, blocked Jacobi, V_k^+ assembly) cover theta sides up to
// LT_REG_DIM and up to LT_REG_CHI kept values; larger tasks take the
// shared/global-memory paths
#define LT_REG_DIM 128
#define LT_REG_CHI 64
#define LT_BLOCK 256
#define LT_NCOUNTERS 6

// device error bits (ctx->err_dev)
#define LT_EBIT_THETA_ZERO 1   // a theta matrix vanished
#define LT_EBIT_PROB 2         // jump probability per step >= 0.5
#define LT_EBIT_NOCONV 4       // Jacobi hit its sweep limit (recorded, not fatal)
#define LT_EBIT_BADARG 8       // replayed channel out of range
#define LT_EBIT_WORKSPACE 16   // a task did not fit its workspace (skipped)
#define LT_EBIT_TIMEOUT 32     // a bounded wait on the tensor cores ran out (kernel returned)

// ---- complex arithmetic on float2 / double2 ------------------------------------
template <typename R> struct CT;
template <> struct CT<float> { typedef float2 T; };
template <> struct CT<double> { typedef double2 T; };

template <typename T> __host__ __device__ __forceinline__ T cmk(double x, double y) {
  T r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T> __device__ __forceinline__ T czero() {
  T r;
  r.x = 0;
  r.y = 0;
  return r;
}
// acc += a * b
template <typename T> __device__ __forceinline__ void cfma(T& acc, const T a, const T b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += a * conj(b)
template <typename T> __device__ __forceinline__ void cfmac(T& acc, const T a, const T b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y);
  acc.y = fma(-a.x, b.y, acc.y);
}
template <typename T> __device__ __forceinline__ T cmul(const T a, const T b) {
  T r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T, typename R> __device__ __forceinline__ T cscale(const T a, R s) {
  T r;
  r.x = a.x * s;
  r.y = a.y * s;
  return r;
}

// ---- Philox4x32-10 (Salmon et al., SC'11) ---------------------------------------
__device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                             uint32_t& x3, uint32_t k0, uint32_t k1) {
  const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(m0, x0), lo0 = m0 * x0;
  uint32_t hi1 = __umulhi(m1, x2), lo1 = m1 * x2;
  uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
  x0 = y0;
  x1 = lo1;
  x2 = y2;
  x3 = lo0;
}
// the four output words for counter (c0, step, purpose, step >> 32) and key seed
__device__ __forceinline__ void philox4(uint64_t seed, uint32_t c0, uint64_t step, uint32_t purpose,
                                        uint32_t (&x)[4]) {
  uint32_t x0 = c0, x1 = (uint32_t)step, x2 = purpose, x3 = (uint32_t)(step >> 32);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(x0, x1, x2, x3, k0, k1);
  }
  x[0] = x0;
  x[1] = x1;
  x[2] = x2;
  x[3] = x3;
}
// uniform double in [0,1) from 27 bits of hi and 26 bits of lo
__device__ __forceinline__ double philox_words_uniform(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) * (1.0 / 9007199254740992.0);
}
// uniform double in [0,1) for counter (c0, step, purpose, step >> 32) and key seed
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint32_t c0, uint64_t step,
                                                 uint32_t purpose) {
  uint32_t x[4];
  philox4(seed, c0, step, purpose, x);
  return philox_words_uniform(x[0], x[1]);
}
// the j-th pair of standard normal numbers of (c0, step): Box-Muller (Box and
// Muller 1958) of the uniforms u1 (words 0, 1) and u2 (words 2, 3) of the draw
// with purpose 1 + j: r = sqrt(-2 ln(1 - u1)), (r cos 2 pi u2, r sin 2 pi u2)
__device__ __forceinline__ void philox_gaussian_pair(uint64_t seed, uint32_t c0, uint64_t step,
                                                     uint32_t j, double& g0, double& g1) {
  uint32_t x[4];
  philox4(seed, c0, step, 1u + j, x);
  const double u1 = philox_words_uniform(x[0], x[1]), u2 = philox_words_uniform(x[2], x[3]);
  const double r = sqrt(-2.0 * log1p(-u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  g0 = r * cs;
  g1 = r * sn;
}

// ---- launch descriptors -----------------------------------------------------------
// One launch of the two-site update over a list of trajectories and a set of
// bonds bond0, bond0 + 2, ..., bond0 + 2 (nb - 1).
template <typename R> struct BondArgs {
  typedef typename CT<R>::T Tc;
  Tc* B;            // [n_traj][L][slot]
  double* lam;      // [n_traj][L-1][chi]
  int* dims;        // [n_traj][L-1]
  double* trunc;    // [n_traj][L-1]
  const int* trajs; // trajectory list
  const int* n_trajs;
  int bond0, nb;
  const double2* gates;  // [L-1][16] or nullptr = identity
  int mode;              // 0 two-site gate update, 1 shift left, 2 restore bond
  long long ws_elems;    // largest workspace of a task, in complex elements
  int L, chi, slot;
  double cut;
  int* err;
  long long smem_elems;  // dynamic shared memory of the launch, in complex elements: a
                         // task whose workspace fits works there
  Tc* scratch;           // per-CTA global workspace of the tasks that do not fit, or nullptr
  long long scratch_stride;
  int use_tc;            // mode 0, single precision, D = 2: theta on the tensor cores
  int cluster;           // CTAs per thread-block cluster (1: no clusters); a cluster
                         // shares the Jacobi of each task that works in global scratch
  float* cl_state;       // per cluster: LT_CL_STATE floats (row norms, flags, rotations)
  int max_sweeps;
  double tol;            // Jacobi threshold, 0 = eps sqrt(n) of the working precision
  int* sweep_hist;       // [64] histogram of Jacobi sweep counts, or nullptr
  unsigned long long* counters;  // see lt_get_counters
  int keep_norm;         // mode 0: B_b keeps the factor ||S_k|| (quantum state diffusion)
  double* logw;          // mode 2 at bond 0: += ln ||S||^2 per trajectory, or nullptr
  double multiplet;      // > 0: k never splits singular values closer than this x sigma_0
};

struct EnvArgs {
  void* B;
  const double* lam;
  const int* dims;
  int L, chi, slot, n_traj;
  void* scratch;  // per-CTA environment workspace
  long long scratch_stride;
  double* density;      // [n_traj][L]
  double* rates;        // [n_traj][3L]
  const double* gl;     // [L]
  const double* gg;
  const double* gd;
  double dt;
  int decide;           // 1: draw/replay the jump decision
  const int* replay;    // [n_traj] or nullptr
  int* channel;         // [n_traj]
  int* evolve;          // [n_traj]
  uint64_t seed;
  long long traj_offset;
  long long step;
  const long long* step_dev;  // the step from device memory (captured steps), or nullptr
  int* err;
  double2* corr;        // [n_traj][L][L] for the correlation kernel
};

// traces of the vectorised density matrix (method LT_MPDO)
struct MpdoArgs {
  const void* B;
  const int* dims;
  int L, chi, slot, n_traj;
  double2* scratch;     // per-CTA [2][L + 1][chi] right and left vectors
  long long stride;     // scratch elements (double2) per CTA
  double* density;      // [n_traj][L]
  double2* corr;        // [n_traj][L][L] or nullptr
};

// ---- context -------------------------------------------------------------------------
struct lt_ctx_s {
  int L, chi, n_traj, prec, order, fermionic, max_sweeps, method;
  int d;            // values per site: 2 (pure states), 4 (vectorised rho; purified X, s = 2n + k)
  double J, dt, cut, jacobi_tol;
  uint64_t seed;
  long long traj_offset;
  std::vector<double> gl, gg, gd;
  std::vector<uint8_t> occ;
  std::vector<int> replay_host;
  int init;

  cudaStream_t stream;
  bool own_stream;
  int device, num_sms;

  int slot;         // complex elements per site tensor slot = d chi^2
  size_t celt;      // bytes per complex element (8 mixed, 16 fp64)
  void* B;          // site tensors
  double* lam;
  int* dims;
  double* trunc;
  int* evolve;
  int* channel;
  int* replay;
  int* active_list;
  int* jumped_list;
  int* counts;      // [0] = n_active, [1] = n_jumped
  double* density;
  double* logw;     // [n_traj] ln <psi|psi> of the unnormalised QSD histories
  double* rates;
  double* gam;      // [3][L]
  int* err_dev;
  int* sweep_hist;  // [64]
  unsigned long long* counters;  // [LT_NCOUNTERS]

  // gate cache: up to 8 distinct tau values
  std::vector<double> gate_taus;
  double2* gates;   // [8][L-1][d^4]

  void* bond_scratch;
  long long bond_scratch_stride;
  int bond_grid;
  int bond_ncl[9];  // clusters of 2, 4, 8 CTAs that can be resident at once (0: none)
  float* bond_cl_state;
  int theta_tc;     // single precision, D = 2: theta on the tensor cores (digit products)
  int env_occ;      // environment-kernel CTAs per SM (0: as many as fit, up to 8)
  size_t bond_smem;

  void* env_scratch;
  long long env_scratch_stride;
  int env_grid;

  double2* corr;    // [n_traj][L][L], allocated on first correlation measurement
  double* red;      // reduction output buffer

  long long step_counter;
  long long launches;
  long long cluster_launches;  // of them, bond launches as thread-block clusters
  // a captured time step (lt_step_graph): its launches read the step from step_dev
  long long* step_dev;
  bool use_step_dev;
  cudaGraphExec_t step_graph;
  long long graph_launches;   // kernels per captured step
  long long step_host;        // source of the counter upload (outlives the async copy)
  size_t dev_bytes;   // device memory this context allocated
  bool poisoned;
  std::string last_error;
};

// ---- kernel launchers (lt_kernels.cu) ----------------------------------------------
cudaError_t launch_bond(lt_ctx_s* c, const int* trajs, const int* n_trajs, int bond0, int nb,
                        const double2* gates, int mode);
cudaError_t launch_env(lt_ctx_s* c, int decide, long long step, const int* replay);
cudaError_t launch_jump_apply(lt_ctx_s* c);
cudaError_t launch_compact(lt_ctx_s* c);
cudaError_t launch_qsd_noise(lt_ctx_s* c, long long step);
cudaError_t launch_corr(lt_ctx_s* c);
cudaError_t launch_mpdo_trace(lt_ctx_s* c, bool corr);
size_t mpdo_scratch_bytes(int L, int chi);
cudaError_t launch_kraus(lt_ctx_s* c);
cudaError_t launch_step_advance(lt_ctx_s* c);
cudaError_t launch_purified_env(lt_ctx_s* c, bool corr);
size_t purified_scratch_bytes(int L, int chi);
cudaError_t launch_reduce_density(lt_ctx_s* c, double* out_mean, double* out_sem);
cudaError_t launch_reduce_corr(lt_ctx_s* c, double* out);
cudaError_t launch_convert_in(lt_ctx_s* c, const double* src, long long n, long long dst_off);
cudaError_t launch_convert_out(lt_ctx_s* c, double* dst, long long n, long long src_off);
cudaError_t launch_init_state(lt_ctx_s* c, const uint8_t* occ_dev);
size_t bond_smem_bytes(int chi, size_t celt, int d);
// Per-cluster state of the cluster-shared phases, in floats (global memory):
#define LT_CL_NRM 0                        // Jacobi row norms [LT_MAX_DIM]
#define LT_CL_FLG LT_MAX_DIM               // Jacobi flags and rotation count (8 ints)
#define LT_CL_B1 (LT_MAX_DIM + 8)          // betas of the LQ of theta [LT_MAX_DIM]
#define LT_CL_B2 (2 * LT_MAX_DIM + 8)      // betas of the LQ of L1^+, two in turn
#define LT_CL_E2 (2 * LT_MAX_DIM + 16)     // its reflectors, two of LT_MAX_DIM complex
#define LT_CL_PERM (6 * LT_MAX_DIM + 16)   // ranked rows [LT_MAX_DIM] (ints)
#define LT_CL_SIG (7 * LT_MAX_DIM + 16)    // squared singular values [LT_MAX_DIM] (doubles)
#define LT_CL_K (9 * LT_MAX_DIM + 16)      // kept values (int)
#define LT_CL_STATE (9 * LT_MAX_DIM + 32)
size_t env_scratch_elems(int L, int chi);
#define LT_ENV_SCRATCH_BYTES (4ull << 30)  // cap of the environment kernels' scratch
long long env_grid_cap(int L, int chi, size_t celt, int num_sms);
