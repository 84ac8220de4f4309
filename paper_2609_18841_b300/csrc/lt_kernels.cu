// Kernels of the batched quantum-trajectory TEBD path (sm_103a).
//
//  bond_update_kernel  the two-site update of Sec. 2.3 (Eq. Theta) in
//                      Vidal-Hastings form, one (trajectory, bond) task per CTA
//                      iteration: theta formation with the gate fused, a
//                      one-sided (Hestenes) Jacobi SVD on the rows of theta,
//                      truncation to chi_max (Sec. 2.2), renormalisation and the
//                      split B_b <- theta~ V_k / ||S_k||, B_{b+1} <- V_k^+.
//  env_kernel          exact <n_k> by left/right environments, jump rates
//                      W_k = gamma_k <L_k^+ L_k> (Eq. TransitionRate) and the
//                      Philox jump-or-evolve decision (Sec. 4.1).
//  jump_apply_kernel   L_k on site k and the Jordan-Wigner string on j < k.
//  corr_kernel         C_ij = <c_i^+ c_j> by transfer matrices.
#include <cfloat>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lt_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename R> struct Eps;
template <> struct Eps<float> { static constexpr float v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

__device__ __forceinline__ double block_sum_double(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

// ---- theta formation (Eq. Theta) -----------------------------------------------------
// X[(a,s'),(t',c)] = w_a sum_{s,t} G[s't',st] sum_mu Bl[a,s,mu] Br[mu,t,c]
template <typename R>
__device__ void form_theta(typename CT<R>::T* X, int ldx, const typename CT<R>::T* Bl,
                           const typename CT<R>::T* Br, int chiL, int chiM, int chiR,
                           const typename CT<R>::T* G, const double* lamL, bool weighted) {
  typedef typename CT<R>::T Tc;
  const int n2 = 2 * chiR;
  for (int idx = threadIdx.x; idx < chiL * chiR; idx += blockDim.x) {
    const int a = idx / chiR, c = idx - a * chiR;
    Tc p00 = czero<Tc>(), p01 = czero<Tc>(), p10 = czero<Tc>(), p11 = czero<Tc>();
    const Tc* l0 = Bl + (2 * a) * chiM;
    const Tc* l1 = l0 + chiM;
    for (int mu = 0; mu < chiM; ++mu) {
      const Tc x0 = l0[mu], x1 = l1[mu];
      const Tc y0 = Br[mu * n2 + c], y1 = Br[mu * n2 + chiR + c];
      cfma(p00, x0, y0);
      cfma(p01, x0, y1);
      cfma(p10, x1, y0);
      cfma(p11, x1, y1);
    }
    const R w = weighted ? (R)lamL[a] : (R)1;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
      for (int tp = 0; tp < 2; ++tp) {
        const Tc* g = G + (sp * 2 + tp) * 4;
        Tc v = czero<Tc>();
        cfma(v, g[0], p00);
        cfma(v, g[1], p01);
        cfma(v, g[2], p10);
        cfma(v, g[3], p11);
        X[(2 * a + sp) * ldx + tp * chiR + c] = cscale(v, w);
      }
    }
  }
}

// circle-method pairing of m (even) rows: m-1 rounds of m/2 disjoint pairs
__device__ __forceinline__ void rr_pair(int round, int i, int m, int& p, int& q) {
  if (i == 0) {
    p = round;
    q = m - 1;
  } else {
    p = (round + i) % (m - 1);
    q = (round - i + (m - 1)) % (m - 1);
  }
}

// One-sided Jacobi on the m rows of X (length n): unitary 2x2 rotations of row
// pairs until every pair is orthogonal to tol * |x| |y|.  Afterwards row r holds
// sigma_r v_r^+ for the right singular vectors v_r of the input.  Returns sweeps.
template <typename R>
__device__ int jacobi_rows(typename CT<R>::T* X, int ld, int m, int n, R* nrm, int* flag,
                           int* nrot, int max_sweeps, double tol_override) {
  typedef typename CT<R>::T Tc;
  int gs = 1;
  while (gs * 4 < n && gs < 32) gs <<= 1;
  const int ng = blockDim.x / gs, gid = threadIdx.x / gs, gl = threadIdx.x - gid * gs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int npairs = m / 2;
  const int iters = (npairs + ng - 1) / ng;
  const R tol = tol_override > 0.0 ? (R)tol_override : Eps<R>::v * sqrt((R)n);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    __syncthreads();
    if (threadIdx.x == 0) *flag = 0;
    for (int r = warp; r < m; r += nw) {
      R acc = 0;
      for (int c = lane; c < n; c += 32) {
        const Tc v = X[r * ld + c];
        acc = fma(v.x, v.x, fma(v.y, v.y, acc));
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (lane == 0) nrm[r] = acc;
    }
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      for (int it = 0; it < iters; ++it) {
        const int pi = it * ng + gid;
        const bool valid = pi < npairs;
        int p = 0, q = 0;
        if (valid) rr_pair(round, pi, m, p, q);
        Tc g = czero<Tc>();
        if (valid) {
          for (int c = gl; c < n; c += gs) cfmac(g, X[p * ld + c], X[q * ld + c]);
        }
        for (int o = gs >> 1; o; o >>= 1) {
          g.x += __shfl_xor_sync(FULL, g.x, o);
          g.y += __shfl_xor_sync(FULL, g.y, o);
        }
        if (valid) {
          const R alpha = nrm[p], beta = nrm[q];
          const R ga = sqrt(g.x * g.x + g.y * g.y);
          if (alpha > (R)0 && beta > (R)0 && ga > tol * sqrt(alpha) * sqrt(beta)) {
            const R zeta = (beta - alpha) / (2 * ga);
            const R az = fabs(zeta);
            const R root = az > (R)1 ? az * sqrt((R)1 + (R)1 / (zeta * zeta)) : sqrt((R)1 + zeta * zeta);
            const R t = (zeta >= (R)0 ? (R)1 : (R)-1) / (az + root);
            const R cs = (R)1 / sqrt((R)1 + t * t);
            const R sn = cs * t;
            const R ex = g.x / ga, ey = g.y / ga;  // e^{i phi} = gamma / |gamma|
            // x' = c x - s e^{i phi} y ; y' = s e^{-i phi} x + c y
            for (int c = gl; c < n; c += gs) {
              const Tc x = X[p * ld + c], y = X[q * ld + c];
              Tc xn, yn;
              xn.x = cs * x.x - sn * (ex * y.x - ey * y.y);
              xn.y = cs * x.y - sn * (ex * y.y + ey * y.x);
              yn.x = sn * (ex * x.x + ey * x.y) + cs * y.x;
              yn.y = sn * (ex * x.y - ey * x.x) + cs * y.y;
              X[p * ld + c] = xn;
              X[q * ld + c] = yn;
            }
            if (gl == 0) {
              nrm[p] = alpha - t * ga;
              nrm[q] = beta + t * ga;
              *flag = 1;
              atomicAdd(nrot, 1);
            }
          }
        }
      }
      __syncthreads();
    }
    const int rotated = *flag;
    __syncthreads();
    if (!rotated) break;
  }
  return sweep + 1;
}

// ---- the two-site update -----------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(LT_BLOCK) bond_update_kernel(BondArgs<R> a) {
  typedef typename CT<R>::T Tc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_sig[LT_MAX_DIM];
  __shared__ R s_nrm[LT_MAX_DIM];
  __shared__ int s_perm[LT_MAX_DIM];
  __shared__ Tc s_gate[16];
  __shared__ double s_lamL[LT_MAX_CHI];
  __shared__ int s_flag, s_k, s_nrot;
  __shared__ double s_norm, s_wdisc;

  Tc* X = a.use_smem ? reinterpret_cast<Tc*>(smem_raw) : a.scratch + (long long)blockIdx.x * a.scratch_stride;
  const int L = a.L, chi = a.chi, tid = threadIdx.x;
  const long long ntask = (long long)(*a.n_trajs) * a.nb;
  for (long long task = blockIdx.x; task < ntask; task += gridDim.x) {
    const int traj = a.trajs[task / a.nb];
    const int b = a.bond0 + 2 * (int)(task % a.nb);
    if (a.rl_filter) {
      const int site = a.channel[traj] / 3;
      if (!(b <= site - 1)) continue;
    }
    const int* dm = a.dims + (long long)traj * (L - 1);
    const int chiL = b == 0 ? 1 : dm[b - 1];
    const int chiM = dm[b];
    const int chiR = b == L - 2 ? 1 : dm[b + 1];
    const int m = 2 * chiL, n = 2 * chiR, ld = n + 1;
    Tc* Bl = a.B + ((long long)traj * L + b) * a.slot;
    Tc* Br = Bl + a.slot;
    Tc* Y = X + m * ld;
    if (tid < 16) {
      if (a.gates) {
        const double2 g = a.gates[b * 16 + tid];
        s_gate[tid] = cmk<Tc>(g.x, g.y);
      } else {
        s_gate[tid] = cmk<Tc>((tid % 5) == 0 ? 1.0 : 0.0, 0.0);
      }
    }
    for (int i = tid; i < chiL; i += blockDim.x)
      s_lamL[i] = b == 0 ? 1.0 : a.lam[((long long)traj * (L - 1) + b - 1) * chi + i];
    if (tid == 0) s_nrot = 0;
    __syncthreads();
    form_theta<R>(X, ld, Bl, Br, chiL, chiM, chiR, s_gate, s_lamL, true);
    const int sweeps = jacobi_rows<R>(X, ld, m, n, s_nrm, &s_flag, &s_nrot, a.max_sweeps, a.tol);
    // singular values squared, accumulated in double
    {
      const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
      for (int r = warp; r < m; r += nw) {
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) {
          const Tc v = X[r * ld + c];
          acc += (double)v.x * v.x + (double)v.y * v.y;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0) s_sig[r] = acc;
      }
    }
    __syncthreads();
    for (int r = tid; r < m; r += blockDim.x) {
      const double v = s_sig[r];
      int rank = 0;
      for (int j = 0; j < m; ++j) {
        const double u = s_sig[j];
        rank += (u > v) || (u == v && j < r);
      }
      s_perm[rank] = r;
    }
    __syncthreads();
    if (tid == 0) {
      double total = 0.0;
      for (int j = 0; j < m; ++j) total += s_sig[j];
      const double s0 = s_sig[s_perm[0]];
      int k = 0;
      if (s0 > 0.0) {
        const double thr = a.cut * sqrt(s0);
        while (k < m && k < n && k < chi && sqrt(s_sig[s_perm[k]]) > thr) ++k;
      } else {
        atomicOr(a.err, LT_EBIT_THETA_ZERO);
      }
      if (k < 1) k = 1;
      double kept = 0.0;
      for (int j = 0; j < k; ++j) kept += s_sig[s_perm[j]];
      s_k = k;
      s_norm = kept > 0.0 ? sqrt(kept) : 1.0;
      s_wdisc = total > 0.0 ? (total - kept) / total : 0.0;
      if (a.sweep_hist) atomicAdd(a.sweep_hist + (sweeps < 63 ? sweeps : 63), 1);
      if (a.counters) {
        // algorithmic real flops: theta (once) + Jacobi (row norms, one complex
        // dot per pair per sweep, 24n per applied rotation, final norms) + split
        const double dm_ = m, dn_ = n;
        const double pairs = 0.5 * dm_ * (dm_ - 1.0) * sweeps;
        const double fl = 8.0 * dm_ * dn_ * (chiM + 4) + 4.0 * dm_ * dn_ * (sweeps + 1) +
                          8.0 * dn_ * pairs + 24.0 * dn_ * s_nrot + 8.0 * dm_ * k * dn_;
        atomicAdd(a.counters + 0, 1ull);
        atomicAdd(a.counters + 1, (unsigned long long)s_nrot);
        atomicAdd(a.counters + 2, (unsigned long long)pairs);
        atomicAdd(a.counters + (a.gates ? 3 : 4), (unsigned long long)fl);
        if (a.gates) atomicAdd(a.counters + 5, 1ull);
      }
      if (sweeps > a.max_sweeps) atomicOr(a.err, LT_EBIT_NOCONV);
    }
    __syncthreads();
    const int k = s_k;
    // V_k^+ rows: Y[j] = X[perm j] / sigma_j
    for (int idx = tid; idx < k * n; idx += blockDim.x) {
      const int j = idx / n, c = idx - j * n;
      const int r = s_perm[j];
      const double sg = s_sig[r];
      const R inv = sg > 0.0 ? (R)(1.0 / sqrt(sg)) : (R)0;
      Y[j * ld + c] = cscale(X[r * ld + c], inv);
    }
    __syncthreads();
    // theta~ again (unweighted), then B_b' = theta~ V_k / ||S_k||
    form_theta<R>(X, ld, Bl, Br, chiL, chiM, chiR, s_gate, s_lamL, false);
    __syncthreads();
    {
      const R invn = (R)(1.0 / s_norm);
      for (int idx = tid; idx < m * k; idx += blockDim.x) {
        const int r = idx / k, j = idx - r * k;
        const Tc* xr = X + r * ld;
        const Tc* yj = Y + j * ld;
        Tc acc = czero<Tc>();
        for (int c = 0; c < n; ++c) cfmac(acc, xr[c], yj[c]);
        Bl[idx] = cscale(acc, invn);
      }
      for (int idx = tid; idx < k * n; idx += blockDim.x) {
        const int j = idx / n, c = idx - j * n;
        Br[idx] = Y[j * ld + c];
      }
      double* lb = a.lam + ((long long)traj * (L - 1) + b) * chi;
      for (int j = tid; j < k; j += blockDim.x) lb[j] = sqrt(s_sig[s_perm[j]]) / s_norm;
      if (tid == 0) {
        a.dims[(long long)traj * (L - 1) + b] = k;
        a.trunc[(long long)traj * (L - 1) + b] += s_wdisc;
      }
    }
    __syncthreads();
  }
}

// ---- block GEMM on generic pointers: C = (acc ? C : 0) + sgn * op(A) op(B) --------------
// op = identity, or the conjugate transpose when the h flag is set.
template <typename R>
__device__ void bgemm(int M, int N, int K, const typename CT<R>::T* A, int lda, int hA,
                      const typename CT<R>::T* B, int ldb, int hB, typename CT<R>::T* C, int ldc,
                      int acc, R sgn) {
  typedef typename CT<R>::T Tc;
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    Tc s = czero<Tc>();
    for (int k = 0; k < K; ++k) {
      Tc x = hA ? A[k * lda + i] : A[i * lda + k];
      Tc y = hB ? B[j * ldb + k] : B[k * ldb + j];
      if (hA) x.y = -x.y;
      if (hB) y.y = -y.y;
      cfma(s, x, y);
    }
    if (acc) {
      Tc o = C[i * ldc + j];
      o.x += sgn * s.x;
      o.y += sgn * s.y;
      C[i * ldc + j] = o;
    } else {
      C[i * ldc + j] = cscale(s, sgn);
    }
  }
}

// sum_{a,b} conj(P[a,b]) Q[a,b] (complex, double accumulation)
template <typename R>
__device__ double2 block_cdot(int M, int N, const typename CT<R>::T* P, int ldp,
                              const typename CT<R>::T* Q, int ldq, double* red) {
  double re = 0.0, im = 0.0;
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const typename CT<R>::T p = P[i * ldp + j], q = Q[i * ldq + j];
    re += (double)p.x * q.x + (double)p.y * q.y;
    im += (double)p.x * q.y - (double)p.y * q.x;
  }
  double2 r;
  r.x = block_sum_double(re, red);
  r.y = block_sum_double(im, red);
  return r;
}

// Right environments R_i = sum_s B_i^s R_{i+1} B_i^{s+}, R_L = 1, stored with
// leading dimension chi at Rl + i chi^2.  Returns <psi|psi> = R_0.
template <typename R>
__device__ double right_envs(const typename CT<R>::T* B, const int* dm, int L, int chi, int slot,
                             typename CT<R>::T* Rl, typename CT<R>::T* T) {
  typedef typename CT<R>::T Tc;
  const int chi2 = chi * chi;
  if (threadIdx.x == 0) Rl[(long long)L * chi2] = cmk<Tc>(1.0, 0.0);
  __syncthreads();
  for (int i = L - 1; i >= 0; --i) {
    const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
    const Tc* Bi = B + (long long)i * slot;
    const Tc* Rn = Rl + (long long)(i + 1) * chi2;
    Tc* Ri = Rl + (long long)i * chi2;
    for (int s = 0; s < 2; ++s) {
      bgemm<R>(cl, cr, cr, Bi + s * cr, 2 * cr, 0, Rn, chi, 0, T, chi, 0, (R)1);
      __syncthreads();
      bgemm<R>(cl, cl, cr, T, chi, 0, Bi + s * cr, 2 * cr, 1, Ri, chi, s, (R)1);
      __syncthreads();
    }
  }
  return (double)Rl[0].x;
}

// env_kernel: per trajectory, exact <n_k> for every site, rates and decision
// (kRates = false: densities only).
template <typename R, bool kRates = true>
__global__ void __launch_bounds__(LT_BLOCK) env_kernel(EnvArgs a) {
  typedef typename CT<R>::T Tc;
  __shared__ double red[32];
  const int L = a.L, chi = a.chi, chi2 = chi * chi;
  Tc* ws = reinterpret_cast<Tc*>(a.scratch) + (long long)blockIdx.x * a.scratch_stride;
  Tc* Rl = ws;                                  // (L+1) chi^2
  Tc* T = Rl + (long long)(L + 1) * chi2;       // chi^2
  Tc* Le = T + chi2;                            // chi^2
  Tc* Ln = Le + chi2;                           // chi^2
  Tc* M0 = Ln + chi2;
  Tc* M1 = M0 + chi2;
  Tc* N1 = M1 + chi2;
  for (int traj = blockIdx.x; traj < a.n_traj; traj += gridDim.x) {
    const Tc* B = reinterpret_cast<const Tc*>(a.B) + (long long)traj * L * a.slot;
    const int* dm = a.dims + (long long)traj * (L - 1);
    const double nrm2 = right_envs<R>(B, dm, L, chi, a.slot, Rl, T);
    if (threadIdx.x == 0) Le[0] = cmk<Tc>(1.0, 0.0);
    __syncthreads();
    for (int k = 0; k < L; ++k) {
      const int cl = k == 0 ? 1 : dm[k - 1], cr = k == L - 1 ? 1 : dm[k];
      const Tc* Bk = B + (long long)k * a.slot;
      bgemm<R>(cl, cr, cl, Le, chi, 0, Bk + cr, 2 * cr, 0, M1, chi, 0, (R)1);
      bgemm<R>(cl, cr, cl, Le, chi, 0, Bk, 2 * cr, 0, M0, chi, 0, (R)1);
      __syncthreads();
      bgemm<R>(cl, cr, cr, M1, chi, 0, Rl + (long long)(k + 1) * chi2, chi, 0, N1, chi, 0, (R)1);
      bgemm<R>(cr, cr, cl, Bk, 2 * cr, 1, M0, chi, 0, Ln, chi, 0, (R)1);
      __syncthreads();
      bgemm<R>(cr, cr, cl, Bk + cr, 2 * cr, 1, M1, chi, 0, Ln, chi, 1, (R)1);
      const double2 d = block_cdot<R>(cl, cr, Bk + cr, 2 * cr, N1, chi, red);
      if (threadIdx.x == 0) {
        const double nk = d.x / nrm2;
        a.density[(long long)traj * L + k] = nk;
        if (kRates) {
          double* rt = a.rates + (long long)traj * 3 * L + 3 * k;
          rt[0] = a.gl[k] * nk;
          rt[1] = a.gg[k] * (1.0 - nk);
          rt[2] = a.gd[k] * nk;
        }
      }
      __syncthreads();
      Tc* tmp = Le;
      Le = Ln;
      Ln = tmp;
    }
    if (kRates && a.decide && threadIdx.x == 0) {
      const double* rt = a.rates + (long long)traj * 3 * L;
      int ch = -1;
      const int rep = a.replay ? a.replay[traj] : -2;
      if (rep == -2) {
        double total = 0.0;
        for (int j = 0; j < 3 * L; ++j) total += rt[j] * a.dt;
        if (total >= 0.5) atomicOr(a.err, LT_EBIT_PROB);
        const double r = philox_uniform(a.seed, (uint32_t)(a.traj_offset + traj), (uint64_t)a.step, 0u);
        if (r < total) {
          double cs = 0.0;
          for (int j = 0; j < 3 * L; ++j) {
            cs += rt[j] * a.dt;
            if (cs > r) {
              ch = j;
              break;
            }
          }
        }
      } else if (rep >= 0) {
        if (rep < 3 * L) ch = rep;
        else atomicOr(a.err, LT_EBIT_BADARG);
      }
      a.channel[traj] = ch;
      a.evolve[traj] = ch < 0 ? 1 : 0;
    }
    __syncthreads();
  }
}

// corr_kernel: per trajectory, C_ij = <c_i^+ c_j> (double2 [L][L]).
template <typename R>
__global__ void __launch_bounds__(LT_BLOCK) corr_kernel(EnvArgs a) {
  typedef typename CT<R>::T Tc;
  __shared__ double red[32];
  const int L = a.L, chi = a.chi, chi2 = chi * chi;
  Tc* ws = reinterpret_cast<Tc*>(a.scratch) + (long long)blockIdx.x * a.scratch_stride;
  Tc* Rl = ws;
  Tc* T = Rl + (long long)(L + 1) * chi2;
  Tc* Le = T + chi2;
  Tc* Ln = Le + chi2;
  Tc* E = Ln + chi2;
  Tc* T1 = E + chi2;
  Tc* T0 = T1 + chi2;
  for (int traj = blockIdx.x; traj < a.n_traj; traj += gridDim.x) {
    const Tc* B = reinterpret_cast<const Tc*>(a.B) + (long long)traj * L * a.slot;
    const int* dm = a.dims + (long long)traj * (L - 1);
    double2* C = a.corr + (long long)traj * L * L;
    const double nrm2 = right_envs<R>(B, dm, L, chi, a.slot, Rl, T);
    if (threadIdx.x == 0) Le[0] = cmk<Tc>(1.0, 0.0);
    __syncthreads();
    for (int i = 0; i < L; ++i) {
      const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
      const Tc* Bi = B + (long long)i * a.slot;
      // diagonal: <n_i>
      bgemm<R>(cl, cr, cl, Le, chi, 0, Bi + cr, 2 * cr, 0, T1, chi, 0, (R)1);
      bgemm<R>(cl, cr, cl, Le, chi, 0, Bi, 2 * cr, 0, T0, chi, 0, (R)1);
      __syncthreads();
      bgemm<R>(cl, cr, cr, T1, chi, 0, Rl + (long long)(i + 1) * chi2, chi, 0, T, chi, 0, (R)1);
      // E = (B_i^1)^+ Le B_i^0   (s+ = |1><0|)
      bgemm<R>(cr, cr, cl, Bi + cr, 2 * cr, 1, T0, chi, 0, E, chi, 0, (R)1);
      // next left environment
      bgemm<R>(cr, cr, cl, Bi, 2 * cr, 1, T0, chi, 0, Ln, chi, 0, (R)1);
      __syncthreads();
      bgemm<R>(cr, cr, cl, Bi + cr, 2 * cr, 1, T1, chi, 0, Ln, chi, 1, (R)1);
      const double2 d = block_cdot<R>(cl, cr, Bi + cr, 2 * cr, T, chi, red);
      if (threadIdx.x == 0) C[i * L + i] = make_double2(d.x / nrm2, 0.0);
      __syncthreads();
      for (int j = i + 1; j < L; ++j) {
        const int cl2 = dm[j - 1], cr2 = j == L - 1 ? 1 : dm[j];
        const Tc* Bj = B + (long long)j * a.slot;
        bgemm<R>(cl2, cr2, cl2, E, chi, 0, Bj + cr2, 2 * cr2, 0, T1, chi, 0, (R)1);
        bgemm<R>(cl2, cr2, cl2, E, chi, 0, Bj, 2 * cr2, 0, T0, chi, 0, (R)1);
        __syncthreads();
        bgemm<R>(cl2, cr2, cr2, T1, chi, 0, Rl + (long long)(j + 1) * chi2, chi, 0, T, chi, 0, (R)1);
        // E <- (B^0)^+ E B^0 - (B^1)^+ E B^1  (string (-1)^n on site j)
        bgemm<R>(cr2, cr2, cl2, Bj, 2 * cr2, 1, T0, chi, 0, E, chi, 0, (R)1);
        __syncthreads();
        bgemm<R>(cr2, cr2, cl2, Bj + cr2, 2 * cr2, 1, T1, chi, 0, E, chi, 1, (R)-1);
        // close with s- = |0><1|: sum conj(B_j^0) (E B_j^1 R_{j+1})
        const double2 cij = block_cdot<R>(cl2, cr2, Bj, 2 * cr2, T, chi, red);
        if (threadIdx.x == 0) {
          C[i * L + j] = make_double2(cij.x / nrm2, cij.y / nrm2);
          C[j * L + i] = make_double2(cij.x / nrm2, -cij.y / nrm2);
        }
        __syncthreads();
      }
      Tc* tmp = Le;
      Le = Ln;
      Ln = tmp;
    }
  }
}

// jump_apply_kernel: one CTA per jumped trajectory.
template <typename R>
__global__ void jump_apply_kernel(typename CT<R>::T* Bdev, const int* dims, const int* jumped,
                                  const int* n_jumped, const int* channel, int L, int slot,
                                  int fermionic) {
  typedef typename CT<R>::T Tc;
  const int nj = *n_jumped;
  for (int ti = blockIdx.x; ti < nj; ti += gridDim.x) {
    const int traj = jumped[ti];
    const int ch = channel[traj];
    const int site = ch / 3, kind = ch - 3 * site;
    const int* dm = dims + (long long)traj * (L - 1);
    Tc* B = Bdev + (long long)traj * L * slot;
    const bool string = fermionic && kind != 2;
    if (string) {
      for (int j = 0; j < site; ++j) {
        const int cl = j == 0 ? 1 : dm[j - 1], cr = j == L - 1 ? 1 : dm[j];
        Tc* Bj = B + (long long)j * slot;
        for (int idx = threadIdx.x; idx < cl * cr; idx += blockDim.x) {
          const int aa = idx / cr, c = idx - aa * cr;
          Tc v = Bj[(2 * aa + 1) * cr + c];
          v.x = -v.x;
          v.y = -v.y;
          Bj[(2 * aa + 1) * cr + c] = v;
        }
      }
    }
    const int cl = site == 0 ? 1 : dm[site - 1], cr = site == L - 1 ? 1 : dm[site];
    Tc* Bk = B + (long long)site * slot;
    for (int idx = threadIdx.x; idx < cl * cr; idx += blockDim.x) {
      const int aa = idx / cr, c = idx - aa * cr;
      const Tc v0 = Bk[(2 * aa) * cr + c], v1 = Bk[(2 * aa + 1) * cr + c];
      Tc n0, n1;
      if (kind == 0) {        // s- = |0><1|
        n0 = v1;
        n1 = czero<Tc>();
      } else if (kind == 1) { // s+ = |1><0|
        n0 = czero<Tc>();
        n1 = v0;
      } else {                // n = |1><1|
        n0 = czero<Tc>();
        n1 = v1;
      }
      Bk[(2 * aa) * cr + c] = n0;
      Bk[(2 * aa + 1) * cr + c] = n1;
    }
    __syncthreads();
  }
}

// compact: active list (evolve = 1) and jumped list (channel >= 0), in order.
__global__ void compact_kernel(const int* evolve, const int* channel, int n, int* active,
                               int* jumped, int* counts) {
  __shared__ int s_w[2][32];
  __shared__ int s_base[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_base[0] = s_base[1] = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int fa = i < n && evolve[i] != 0;
    const int fj = i < n && channel[i] >= 0;
    const unsigned ba = __ballot_sync(FULL, fa), bj = __ballot_sync(FULL, fj);
    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0) {
      s_w[0][warp] = __popc(ba);
      s_w[1][warp] = __popc(bj);
    }
    __syncthreads();
    int oa = s_base[0], oj = s_base[1];
    for (int w = 0; w < warp; ++w) {
      oa += s_w[0][w];
      oj += s_w[1][w];
    }
    if (fa) active[oa + __popc(ba & lt)] = i;
    if (fj) jumped[oj + __popc(bj & lt)] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < nw; ++w) {
        s_base[0] += s_w[0][w];
        s_base[1] += s_w[1][w];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counts[0] = s_base[0];
    counts[1] = s_base[1];
  }
}

// ensemble mean and CLT error over trajectories: x [n][M] -> mean [M], sem [M]
__global__ void reduce_mean_sem_kernel(const double* x, int n, int M, double* mean, double* sem) {
  __shared__ double red[32];
  for (int col = blockIdx.x; col < M; col += gridDim.x) {
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) s += x[(long long)t * M + col];
    const double mu = block_sum_double(s, red) / n;
    double v = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double d = x[(long long)t * M + col] - mu;
      v += d * d;
    }
    const double var = block_sum_double(v, red) / n;
    if (threadIdx.x == 0) {
      mean[col] = mu;
      if (sem) sem[col] = n > 1 ? sqrt(var / n) : 0.0;
    }
  }
}

// ensemble mean of a double2 [n][M] array -> interleaved double [M][2]
__global__ void reduce_mean_c_kernel(const double2* x, int n, int M, double* out) {
  __shared__ double red[32];
  for (int col = blockIdx.x; col < M; col += gridDim.x) {
    double re = 0.0, im = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double2 v = x[(long long)t * M + col];
      re += v.x;
      im += v.y;
    }
    re = block_sum_double(re, red);
    im = block_sum_double(im, red);
    if (threadIdx.x == 0) {
      out[2 * col] = re / n;
      out[2 * col + 1] = im / n;
    }
  }
}

template <typename R>
__global__ void convert_in_kernel(typename CT<R>::T* dst, const double* src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = cmk<typename CT<R>::T>(src[2 * i], src[2 * i + 1]);
}

template <typename R>
__global__ void convert_out_kernel(double* dst, const typename CT<R>::T* src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const typename CT<R>::T v = src[i];
    dst[2 * i] = v.x;
    dst[2 * i + 1] = v.y;
  }
}

template <typename R>
__global__ void init_state_kernel(typename CT<R>::T* B, double* lam, int* dims, double* trunc,
                                  int* evolve, int* channel, const uint8_t* occ, int n_traj,
                                  int L, int chi, int slot) {
  const long long nt = (long long)n_traj * L;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nt;
       i += (long long)gridDim.x * blockDim.x) {
    const int traj = (int)(i / L), site = (int)(i - (long long)traj * L);
    typename CT<R>::T* s = B + i * slot;
    s[0] = cmk<typename CT<R>::T>(occ[site] ? 0.0 : 1.0, 0.0);
    s[1] = cmk<typename CT<R>::T>(occ[site] ? 1.0 : 0.0, 0.0);
    if (site < L - 1) {
      const long long bi = (long long)traj * (L - 1) + site;
      lam[bi * chi] = 1.0;
      dims[bi] = 1;
      trunc[bi] = 0.0;
    }
    if (site == 0) {
      evolve[traj] = 1;
      channel[traj] = -1;
    }
  }
}

inline int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 65535) g = 65535;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ---- launchers -------------------------------------------------------------------------------
size_t bond_smem_bytes(int chi, size_t celt) {
  const size_t m = 2 * (size_t)chi, n = 2 * (size_t)chi, k = chi;
  return (m + k) * (n + 1) * celt;
}

size_t env_scratch_elems(int L, int chi) { return ((size_t)L + 1 + 7) * (size_t)chi * chi; }

template <typename R>
static cudaError_t launch_bond_t(lt_ctx_s* c, const int* trajs, const int* n_trajs, int bond0,
                                 int nb, const double2* gates, int rl_filter) {
  BondArgs<R> a;
  a.B = reinterpret_cast<typename CT<R>::T*>(c->B);
  a.lam = c->lam;
  a.dims = c->dims;
  a.trunc = c->trunc;
  a.trajs = trajs;
  a.n_trajs = n_trajs;
  a.bond0 = bond0;
  a.nb = nb;
  a.gates = gates;
  a.channel = c->channel;
  a.rl_filter = rl_filter;
  a.L = c->L;
  a.chi = c->chi;
  a.slot = c->slot;
  a.cut = c->cut;
  a.err = c->err_dev;
  a.scratch = reinterpret_cast<typename CT<R>::T*>(c->bond_scratch);
  a.scratch_stride = c->bond_scratch_stride;
  a.use_smem = c->bond_use_smem;
  a.max_sweeps = c->max_sweeps;
  a.tol = c->jacobi_tol;
  a.sweep_hist = c->sweep_hist;
  a.counters = c->counters;
  bond_update_kernel<R><<<c->bond_grid, LT_BLOCK, c->bond_use_smem ? c->bond_smem : 0, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_bond(lt_ctx_s* c, const int* trajs, const int* n_trajs, int bond0, int nb,
                        const double2* gates, int rl_filter) {
  if (c->prec == LT_MIXED) return launch_bond_t<float>(c, trajs, n_trajs, bond0, nb, gates, rl_filter);
  return launch_bond_t<double>(c, trajs, n_trajs, bond0, nb, gates, rl_filter);
}

static EnvArgs env_args(lt_ctx_s* c) {
  EnvArgs a;
  a.B = c->B;
  a.lam = c->lam;
  a.dims = c->dims;
  a.L = c->L;
  a.chi = c->chi;
  a.slot = c->slot;
  a.n_traj = c->n_traj;
  a.scratch = c->env_scratch;
  a.scratch_stride = c->env_scratch_stride;
  a.density = c->density;
  a.rates = c->rates;
  a.gl = c->gam;
  a.gg = c->gam + c->L;
  a.gd = c->gam + 2 * c->L;
  a.dt = c->dt;
  a.decide = 0;
  a.replay = nullptr;
  a.channel = c->channel;
  a.evolve = c->evolve;
  a.seed = c->seed;
  a.traj_offset = c->traj_offset;
  a.step = 0;
  a.err = c->err_dev;
  a.corr = c->corr;
  return a;
}

cudaError_t launch_env(lt_ctx_s* c, int decide, long long step, const int* replay) {
  EnvArgs a = env_args(c);
  a.decide = decide;
  a.step = step;
  a.replay = replay;
  if (c->prec == LT_MIXED) env_kernel<float><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  else env_kernel<double><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_corr(lt_ctx_s* c) {
  EnvArgs a = env_args(c);
  if (c->prec == LT_MIXED) corr_kernel<float><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  else corr_kernel<double><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_jump_apply(lt_ctx_s* c) {
  const int grid = c->n_traj < 4 * c->num_sms ? c->n_traj : 4 * c->num_sms;
  if (c->prec == LT_MIXED)
    jump_apply_kernel<float><<<grid, LT_BLOCK, 0, c->stream>>>(
        reinterpret_cast<float2*>(c->B), c->dims, c->jumped_list, c->counts + 1, c->channel, c->L,
        c->slot, c->fermionic);
  else
    jump_apply_kernel<double><<<grid, LT_BLOCK, 0, c->stream>>>(
        reinterpret_cast<double2*>(c->B), c->dims, c->jumped_list, c->counts + 1, c->channel, c->L,
        c->slot, c->fermionic);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_compact(lt_ctx_s* c) {
  compact_kernel<<<1, 1024, 0, c->stream>>>(c->evolve, c->channel, c->n_traj, c->active_list,
                                            c->jumped_list, c->counts);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_reduce_density(lt_ctx_s* c, double* out_mean, double* out_sem) {
  reduce_mean_sem_kernel<<<c->L, LT_BLOCK, 0, c->stream>>>(c->density, c->n_traj, c->L, out_mean,
                                                           out_sem);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_reduce_corr(lt_ctx_s* c, double* out) {
  const int M = c->L * c->L;
  reduce_mean_c_kernel<<<M < 4096 ? M : 4096, LT_BLOCK, 0, c->stream>>>(c->corr, c->n_traj, M, out);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_convert_in(lt_ctx_s* c, const double* src, long long n, long long dst_off) {
  if (c->prec == LT_MIXED)
    convert_in_kernel<float><<<grid_for(n, 256), 256, 0, c->stream>>>(
        reinterpret_cast<float2*>(c->B) + dst_off, src, n);
  else
    convert_in_kernel<double><<<grid_for(n, 256), 256, 0, c->stream>>>(
        reinterpret_cast<double2*>(c->B) + dst_off, src, n);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_convert_out(lt_ctx_s* c, double* dst, long long n, long long src_off) {
  if (c->prec == LT_MIXED)
    convert_out_kernel<float><<<grid_for(n, 256), 256, 0, c->stream>>>(
        dst, reinterpret_cast<const float2*>(c->B) + src_off, n);
  else
    convert_out_kernel<double><<<grid_for(n, 256), 256, 0, c->stream>>>(
        dst, reinterpret_cast<const double2*>(c->B) + src_off, n);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_init_state(lt_ctx_s* c, const uint8_t* occ_dev) {
  const long long nt = (long long)c->n_traj * c->L;
  if (c->prec == LT_MIXED)
    init_state_kernel<float><<<grid_for(nt, 256), 256, 0, c->stream>>>(
        reinterpret_cast<float2*>(c->B), c->lam, c->dims, c->trunc, c->evolve, c->channel, occ_dev,
        c->n_traj, c->L, c->chi, c->slot);
  else
    init_state_kernel<double><<<grid_for(nt, 256), 256, 0, c->stream>>>(
        reinterpret_cast<double2*>(c->B), c->lam, c->dims, c->trunc, c->evolve, c->channel, occ_dev,
        c->n_traj, c->L, c->chi, c->slot);
  c->launches++;
  return cudaGetLastError();
}

// attribute setup and occupancy for the bond kernel (called once per context)
cudaError_t configure_bond(lt_ctx_s* c) {
  const size_t need = bond_smem_bytes(c->chi, c->celt);
  const size_t limit = 200 * 1024;
  c->bond_use_smem = need <= limit;
  c->bond_smem = c->bond_use_smem ? need : 0;
  cudaError_t e;
  int occ = 0;
  if (c->prec == LT_MIXED) {
    e = cudaFuncSetAttribute(bond_update_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)c->bond_smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bond_update_kernel<float>, LT_BLOCK,
                                                      c->bond_smem);
  } else {
    e = cudaFuncSetAttribute(bond_update_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)c->bond_smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bond_update_kernel<double>, LT_BLOCK,
                                                      c->bond_smem);
  }
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  c->bond_grid = occ * c->num_sms;
  c->bond_scratch_stride = c->bond_use_smem ? 0 : (long long)(need / c->celt);
  return cudaSuccess;
}

// ---- allocation-free density entry point -------------------------------------------------
// Scratch of lt_measure_density_noalloc: a file-scope device array, so that the
// call itself allocates nothing.  Every GPU that loads the library holds it until
// the process exits.
#define LT_NOALLOC_SCRATCH_BYTES (32ull << 20)
#define LT_NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) unsigned char lt_noalloc_scratch[LT_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[LT_NOALLOC_MAX_DEVICES];
}  // namespace

extern "C" lt_status lt_measure_density_noalloc(int32_t precision, int32_t L, int32_t chi_max,
                                                int32_t n_traj, const void* B,
                                                const int32_t* dims, double* density,
                                                void* stream) {
  if (L < 2 || L > 1024 || chi_max < 1 || chi_max > LT_MAX_CHI || n_traj < 1 ||
      (precision != LT_FP64 && precision != LT_MIXED) || !B || !dims || !density)
    return LT_ERR_ARG;
  const size_t celt = precision == LT_MIXED ? sizeof(float2) : sizeof(double2);
  const size_t stride = env_scratch_elems(L, chi_max);
  const size_t per_cta = stride * celt;
  if (per_cta > LT_NOALLOC_SCRATCH_BYTES) return LT_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LT_ERR_CUDA;
  if (dev < 0 || dev >= LT_NOALLOC_MAX_DEVICES) return LT_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  {
    // once per device, with that device current: the host-side name of the
    // array is only a stand-in, the kernel needs its device address
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, lt_noalloc_scratch) != cudaSuccess || !p) return LT_ERR_CUDA;
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LT_ERR_CUDA;
  long long grid = (long long)(LT_NOALLOC_SCRATCH_BYTES / per_cta);
  if (grid > 2LL * sms) grid = 2LL * sms;
  if (grid > n_traj) grid = n_traj;
  EnvArgs a;
  std::memset(&a, 0, sizeof(a));
  a.B = const_cast<void*>(B);
  a.dims = dims;
  a.L = L;
  a.chi = chi_max;
  a.slot = 2 * chi_max * chi_max;
  a.n_traj = n_traj;
  a.scratch = scratch;
  a.scratch_stride = (long long)stride;
  a.density = density;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == LT_MIXED) env_kernel<float, false><<<(int)grid, LT_BLOCK, 0, st>>>(a);
  else env_kernel<double, false><<<(int)grid, LT_BLOCK, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}
