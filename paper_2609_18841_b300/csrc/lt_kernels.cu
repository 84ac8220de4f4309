// Kernels of the batched quantum-trajectory TEBD path (sm_103a).
//
//  bond_update_kernel  the two-site update of Sec. 2.3 (Eq. Theta) in
//                      Vidal-Hastings form, one (trajectory, bond) task per CTA
//                      iteration: theta formation with the gate fused, a
//                      two-level Householder preconditioning and a one-sided
//                      (Hestenes) block Jacobi SVD, truncation to chi_max
//                      (Sec. 2.2), renormalisation and the split
//                      B_b <- theta~ V_k / ||S_k||, B_{b+1} <- V_k^+; modes 1 and
//                      2 are the one-site SVDs that restore the canonical form.
//  env_tiled_kernel    exact <n_k> by left/right environments (tiled complex
//                      GEMMs), jump rates W_k = gamma_k <L_k^+ L_k> (Eq.
//                      TransitionRate) and the Philox jump-or-evolve decision
//                      (Sec. 4.1).
//  jump_apply_kernel   L_k on site k and the Jordan-Wigner string on j < k.
//  qsd_noise_kernel    the quantum-state-diffusion noise factors (Sec. 5.2).
//  corr_kernel         C_ij = <c_i^+ c_j> by transfer matrices.
#include <cfloat>
#include <cstdio>
#include <cstring>

#include <cuda_bf16.h>

#include "lt_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename R> struct MinNormal;
template <> struct MinNormal<float> { static constexpr float v = FLT_MIN; };
template <> struct MinNormal<double> { static constexpr double v = DBL_MIN; };
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

// ---- packed pairs of reals ----------------------------------------------------------------
// Two adjacent elements of one plane (real or imaginary parts) as a float2 go
// through Blackwell's packed single-precision FMA (IEEE round-to-nearest per
// lane); double2 falls back to two scalar FMAs.
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 pmul(double2 a, double2 b) {
  return make_double2(a.x * b.x, a.y * b.y);
}
template <typename V, typename R> __device__ __forceinline__ V splat(R v) {
  V r;
  r.x = v;
  r.y = v;
  return r;
}

// ---- theta formation (Eq. Theta) -----------------------------------------------------
// theta[(a,s'),(t',c)] = w_a sum_{s,t} G[s't',st] sum_mu Bl[a,s,mu] Br[mu,t,c] with D
// physical values per site (D = 2 for pure states; D = 4 for the vectorised
// density matrix, m = 2n + n', Eq. MPDO), written planar (real parts in Xr,
// imaginary parts in Xi, row stride ldp).  Br is first staged in shared memory
// (Bs_in, chiM x D chiR) when a staging area is given.  For D = 2 each thread
// computes two values of a for one column c, so consecutive lanes read
// consecutive Bs words and share the broadcast Bl reads; for D = 4 a thread
// takes one (a, c) and its 16 products.  Columns n..npad-1 are set to zero (the
// Jacobi sweeps run over npad columns without tests), and so are the padding
// rows D chiL .. mp-1.  Glo (single precision, or nullptr) holds the rounding
// residual G - fl(G) of every gate entry: the gate is applied as fl(G) + Glo, so
// the same rounding of the gate does not recur in every layer of every step (a
// coherent error that the ensemble average would not remove), leaving only the
// independent rounding of each accumulation.
template <typename R, int D>
__device__ void form_theta(R* Xr, R* Xi, int ldp, int npad, int mp, const typename CT<R>::T* Bl,
                           const typename CT<R>::T* Br, const typename CT<R>::T* Bs_in, int chiL,
                           int chiM, int chiR, const typename CT<R>::T* G,
                           const typename CT<R>::T* Glo, const double* lamL, bool weighted) {
  typedef typename CT<R>::T Tc;
  const int n2 = D * chiR;
  if (npad > n2) {
    const int w = npad - n2;
    for (int i = threadIdx.x; i < D * chiL * w; i += blockDim.x) {
      const int r = i / w, c = n2 + (i - r * w);
      Xr[r * ldp + c] = (R)0;
      Xi[r * ldp + c] = (R)0;
    }
  }
  for (int i = threadIdx.x; i < (mp - D * chiL) * npad; i += blockDim.x) {
    const int r = D * chiL + i / npad, c = i - (i / npad) * npad;
    Xr[r * ldp + c] = (R)0;
    Xi[r * ldp + c] = (R)0;
  }
  const Tc* Bs = Bs_in;
  if (Bs_in) {
    Tc* st = const_cast<Tc*>(Bs_in);
    for (int i = threadIdx.x; i < chiM * n2; i += blockDim.x) st[i] = Br[i];
    __syncthreads();
  } else {
    Bs = Br;  // no room to stage: read B_{b+1} through L1
  }
  if constexpr (D != 2) {
    for (int idx = threadIdx.x; idx < chiL * chiR; idx += blockDim.x) {
      const int a = idx / chiR, c = idx - a * chiR;
      Tc p[D * D];
#pragma unroll
      for (int v = 0; v < D * D; ++v) p[v] = czero<Tc>();
      const Tc* la = Bl + (D * a) * chiM;
      for (int mu = 0; mu < chiM; ++mu) {
        Tc x[D], y[D];
#pragma unroll
        for (int s = 0; s < D; ++s) {
          x[s] = la[s * chiM + mu];
          y[s] = Bs[mu * n2 + s * chiR + c];
        }
#pragma unroll
        for (int s = 0; s < D; ++s)
#pragma unroll
          for (int t = 0; t < D; ++t) cfma(p[s * D + t], x[s], y[t]);
      }
      const R w = weighted ? (R)lamL[a] : (R)1;
      for (int sp = 0; sp < D; ++sp) {
        for (int tp = 0; tp < D; ++tp) {
          const Tc* g = G + (sp * D + tp) * (D * D);
          Tc v = czero<Tc>();
          if (Glo) {
            const Tc* gl = Glo + (sp * D + tp) * (D * D);
#pragma unroll
            for (int u = 0; u < D * D; ++u) cfma(v, gl[u], p[u]);
          }
#pragma unroll
          for (int u = 0; u < D * D; ++u) cfma(v, g[u], p[u]);
          const int o = (D * a + sp) * ldp + tp * chiR + c;
          Xr[o] = v.x * w;
          Xi[o] = v.y * w;
        }
      }
    }
    return;
  }
  const int ahalf = (chiL + 1) >> 1;
  for (int idx = threadIdx.x; idx < ahalf * chiR; idx += blockDim.x) {
    const int a0 = idx / chiR, c = idx - a0 * chiR;
    const int a1 = a0 + ahalf;
    const bool two = a1 < chiL;
    Tc p[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) p[u][v] = czero<Tc>();
    const Tc* l00 = Bl + (2 * a0) * chiM;
    const Tc* l10 = Bl + (2 * (two ? a1 : a0)) * chiM;
    for (int mu = 0; mu < chiM; ++mu) {
      const Tc y0 = Bs[mu * n2 + c], y1 = Bs[mu * n2 + chiR + c];
      const Tc x0 = l00[mu], x1 = l00[chiM + mu];
      const Tc z0 = l10[mu], z1 = l10[chiM + mu];
      cfma(p[0][0], x0, y0);
      cfma(p[0][1], x0, y1);
      cfma(p[0][2], x1, y0);
      cfma(p[0][3], x1, y1);
      cfma(p[1][0], z0, y0);
      cfma(p[1][1], z0, y1);
      cfma(p[1][2], z1, y0);
      cfma(p[1][3], z1, y1);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
      const int a = u ? a1 : a0;
      const R w = weighted ? (R)lamL[a] : (R)1;
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
        for (int tp = 0; tp < 2; ++tp) {
          const Tc* g = G + (sp * 2 + tp) * 4;
          Tc v = czero<Tc>();
          if (Glo) {
            const Tc* gl = Glo + (sp * 2 + tp) * 4;
            cfma(v, gl[0], p[u][0]);
            cfma(v, gl[1], p[u][1]);
            cfma(v, gl[2], p[u][2]);
            cfma(v, gl[3], p[u][3]);
          }
          cfma(v, g[0], p[u][0]);
          cfma(v, g[1], p[u][1]);
          cfma(v, g[2], p[u][2]);
          cfma(v, g[3], p[u][3]);
          const int o = (2 * a + sp) * ldp + tp * chiR + c;
          Xr[o] = v.x * w;
          Xi[o] = v.y * w;
        }
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

// One-sided Jacobi on the m rows of the planar matrix (Xr, Xi), length n:
// unitary 2x2 rotations of row pairs until every pair is orthogonal to
// tol * |x| |y|.  Afterwards row r holds sigma_r v_r^+ for the right singular
// vectors v_r of the input.  Returns the number of sweeps.
//
// A pair is handled by gs lanes; each lane holds EPP element pairs of both
// rows (real and imaginary planes) in registers, so every element is loaded
// once and, when the pair rotates, stored once.  Packed FMAs work on two
// elements at a time: the inner product is 2 and the rotation 6 instructions
// per element.  All m/2 pairs of a round run at once when the block has enough
// groups; with 8-lane groups the two groups of a half-warp take rows 8 apart,
// which with the row stride n + 2 puts their windows in disjoint banks.
// 1/sqrt(x): single precision refines the hardware estimate y by the residual
// form y + y (1 - x y^2) / 2 (within about one ulp, so the rotations stay
// unitary to working precision); double precision divides.
__device__ __forceinline__ float rsqrt_nr(float x) {
  const float y = rsqrtf(x);
  const float r = fmaf(-x * y, y, 1.0f);
  return fmaf(0.5f * y, r, y);
}
__device__ __forceinline__ double rsqrt_nr(double x) { return 1.0 / sqrt(x); }

// Parameters of the 2x2 unitary that orthogonalises rows x, y with squared
// norms alpha, beta and inner product g = x . y^+ (gx + i gy):
//   zeta = (beta - alpha) / (2|g|),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1/sqrt(1 + t^2),  s e^{i phi} = c t g/|g|;
// the squared norms become alpha - t|g| and beta + t|g|.  Returns false when the
// pair is already orthogonal to tol |x| |y| (or a row vanishes).  The reciprocal
// square roots are refined to about one ulp.
// t only selects the rotation angle: c and s follow from t through the refined
// reciprocal square root, so the rotation is unitary to working precision
// whatever rounding t carries.  Single precision therefore takes sqrt(1 + zeta^2)
// and the quotient from the hardware estimates (a few ulp); double divides.
__device__ __forceinline__ float tangent(float zeta, float az) {
  const float y = fmaf(zeta, zeta, 1.0f);
  const float root = az < 1e18f ? y * rsqrtf(y) : az;
  return __fdividef(zeta >= 0.f ? 1.0f : -1.0f, az + root);
}
__device__ __forceinline__ double tangent(double zeta, double az) {
  const double root = az < 1e18 ? sqrt(fma(zeta, zeta, 1.0)) : az;
  return (zeta >= 0.0 ? 1.0 : -1.0) / (az + root);
}

template <typename R>
__device__ __forceinline__ bool rot_params(R gx, R gy, R alpha, R beta, R tol, R& cs, R& sex,
                                           R& sey, R& tga) {
  const R g2 = gx * gx + gy * gy;
  // below the normal range |g|^2 carries too few bits for 1/|g| (the rotation
  // would not be unitary); such a pair is orthogonal to 1e-19 absolutely
  if (!(alpha > (R)0 && beta > (R)0 && g2 > tol * tol * alpha * beta && g2 >= MinNormal<R>::v))
    return false;
  const R inv = rsqrt_nr(g2);
  const R zeta = (beta - alpha) * (R)0.5 * inv;
  const R t = tangent(zeta, fabs(zeta));
  cs = rsqrt_nr(fma(t, t, (R)1));
  const R sn = cs * t;
  sex = sn * gx * inv;
  sey = sn * gy * inv;
  tga = t * (g2 * inv);
  return true;
}

template <typename R, int EPP>
__device__ __forceinline__ int jacobi_span(int n) {
  int gs = 1;
  while (gs * 2 * EPP < n && gs < 32) gs <<= 1;
  return gs;
}

template <typename R, int EPP, bool CHUNKED>
__device__ int jacobi_rows(R* Xr, R* Xi, int ldp, int m, int n, R* nrm, int* nrot, int max_sweeps,
                           double tol_override) {
  typedef typename CT<R>::T V;  // a pair of reals of one plane
  const int gs = jacobi_span<R, EPP>(n);
  const int ng = blockDim.x / gs, gid = threadIdx.x / gs, gl = threadIdx.x - gid * gs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int npairs = m / 2;
  const int iters = (npairs + ng - 1) / ng;
  // rows longer than one group's span (2 EPP 32 columns) are handled in chunks of it:
  // the inner product accumulates over the chunks, the rotation reloads them
  const int span = 2 * EPP * gs, nch = CHUNKED ? (n + span - 1) / span : 1;
  const bool remap = gs == 8 && ng == 64 && npairs == 64;
  const R tol = tol_override > 0.0 ? (R)tol_override : Eps<R>::v * sqrt((R)n);
  // partner rows of this group's pair in round 0; when every pair of a round
  // has its own group they advance by one (mod m-1) per round
  const int pi0 = remap ? (((gid >> 4) << 4) | ((gid & 1) << 3) | ((gid >> 1) & 7)) : gid;
  int p0 = 0, q0 = 0;
  if (gid < npairs) rr_pair(0, pi0, m, p0, q0);
  int my_rot = 0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    __syncthreads();
    for (int r = warp; r < m; r += nw) {
      R acc = 0;
      for (int c = lane; c < n; c += 32) {
        const R u = Xr[r * ldp + c], v = Xi[r * ldp + c];
        acc = fma(u, u, fma(v, v, acc));
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (lane == 0) nrm[r] = acc;
    }
    __syncthreads();
    int any = 0;
    int pr = p0, qr = q0;
    for (int round = 0; round < m - 1; ++round) {
      for (int it = 0; it < iters; ++it) {
        const int slot = it * ng + gid;
        const bool valid = slot < npairs;
        int p = pr, q = qr;
        if (iters > 1 && valid) rr_pair(round, slot, m, p, q);
        R gx = 0, gy = 0;
        V xr[EPP], xi[EPP], yr[EPP], yi[EPP];
        if (valid) {
          V A = splat<V>((R)0), B = A, C = A, D = A;
          for (int ch = 0; ch < nch; ++ch) {
            const int c0 = ch * span + 2 * gl;
            const R* px = Xr + p * ldp + c0;
            const R* pxi = Xi + p * ldp + c0;
            const R* py = Xr + q * ldp + c0;
            const R* pyi = Xi + q * ldp + c0;
#pragma unroll
            for (int e = 0; e < EPP; ++e) {
              xr[e] = *reinterpret_cast<const V*>(px + 2 * gs * e);
              xi[e] = *reinterpret_cast<const V*>(pxi + 2 * gs * e);
              yr[e] = *reinterpret_cast<const V*>(py + 2 * gs * e);
              yi[e] = *reinterpret_cast<const V*>(pyi + 2 * gs * e);
              // x . conj(y) = (xr yr + xi yi) + i (xi yr - xr yi)
              A = pfma(xr[e], yr[e], A);
              B = pfma(xi[e], yi[e], B);
              C = pfma(xi[e], yr[e], C);
              D = pfma(xr[e], yi[e], D);
            }
          }
          gx = (A.x + A.y) + (B.x + B.y);
          gy = (C.x + C.y) - (D.x + D.y);
        }
        for (int o = gs >> 1; o; o >>= 1) {
          gx += __shfl_xor_sync(FULL, gx, o);
          gy += __shfl_xor_sync(FULL, gy, o);
        }
        if (valid) {
          const R alpha = nrm[p], beta = nrm[q];
          R cs, sex, sey, tga;
          if (rot_params(gx, gy, alpha, beta, tol, cs, sex, sey, tga)) {
            const V CS = splat<V>(cs), SX = splat<V>(sex), SY = splat<V>(sey);
            const V NSX = splat<V>(-sex), NSY = splat<V>(-sey);
            // one chunk: still in registers; several: each reloaded
            for (int ch = nch - 1; ch >= 0; --ch) {
              const int c0 = ch * span + 2 * gl;
              R* px = Xr + p * ldp + c0;
              R* pxi = Xi + p * ldp + c0;
              R* py = Xr + q * ldp + c0;
              R* pyi = Xi + q * ldp + c0;
              if (CHUNKED) {
#pragma unroll
                for (int e = 0; e < EPP; ++e) {
                  xr[e] = *reinterpret_cast<const V*>(px + 2 * gs * e);
                  xi[e] = *reinterpret_cast<const V*>(pxi + 2 * gs * e);
                  yr[e] = *reinterpret_cast<const V*>(py + 2 * gs * e);
                  yi[e] = *reinterpret_cast<const V*>(pyi + 2 * gs * e);
                }
              }
              // x' = c x - se y ; y' = conj(se) x + c y
#pragma unroll
              for (int e = 0; e < EPP; ++e) {
                *reinterpret_cast<V*>(px + 2 * gs * e) = pfma(SY, yi[e], pfma(NSX, yr[e], pmul(CS, xr[e])));
                *reinterpret_cast<V*>(pxi + 2 * gs * e) = pfma(NSY, yr[e], pfma(NSX, yi[e], pmul(CS, xi[e])));
                *reinterpret_cast<V*>(py + 2 * gs * e) = pfma(SY, xi[e], pfma(SX, xr[e], pmul(CS, yr[e])));
                *reinterpret_cast<V*>(pyi + 2 * gs * e) = pfma(NSY, xr[e], pfma(SX, xi[e], pmul(CS, yi[e])));
              }
            }
            if (gl == 0) {
              nrm[p] = alpha - tga;
              nrm[q] = beta + tga;
              ++my_rot;
            }
            any = 1;
          }
        }
      }
      if (pi0 == 0) {
        pr = round + 1;
      } else {
        pr = pr + 1 == m - 1 ? 0 : pr + 1;
        qr = qr + 1 == m - 1 ? 0 : qr + 1;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(any)) break;
  }
  if (gl == 0 && my_rot) atomicAdd(nrot, my_rot);
  return sweep + 1;
}

// ---- block Jacobi with register-resident rows (single precision) -------------------------
// The rows are grouped in blocks of four.  In a block round each warp holds a
// pair of blocks (eight rows) in registers, lane l owning the element pairs at
// columns 2l + 64j of each row, and makes every cross pair of the two blocks
// orthogonal in four sub-rounds of four disjoint pairs (in the first block round
// of a sweep also the six pairs inside each block, in three sub-rounds).  The
// blocks meet in circle-method order, so a sweep still visits every row pair
// once; only the block rounds need block-wide barriers.  The four inner products
// of a sub-round are reduced across the warp together (a 9-shuffle
// reduce-scatter); lanes 8k..8k+7 then compute the rotation of pair k and
// broadcast it.
template <int CPL>
struct BJRows {
  float2 r[8][CPL];  // real parts, element pairs
  float2 i[8][CPL];  // imaginary parts
  float nrl;         // squared norm of row (lane & 7) of the eight
};

// Rows longer than a warp's 128 columns: GW warps hold one column slice each of the
// same eight rows, and the eight partial sums of a sub-round go through shared memory
// (two buffers used in turn, one named barrier per sub-round) and are added in warp
// order, so that every warp of the group derives the same rotations.
struct BJGroup {
  float* part;  // [2][GW][8]
  int bar;      // named barrier of the group
  int wg;       // this warp's slice
  int buf;      // buffer of the next sub-round
};

template <int CPL, int GW, int P0, int Q0, int P1, int Q1, int P2, int Q2, int P3, int Q3>
__device__ __forceinline__ void bj_subround(BJRows<CPL>& w, float tol, int& any, int& nrot,
                                            BJGroup& grp) {
  const int lane = threadIdx.x & 31;
  const float2 ONE2 = make_float2(1.f, 1.f), MONE2 = make_float2(-1.f, -1.f);
  float v[8];
#define LT_BJ_DOT(K, P, Q)                                                   \
  {                                                                         \
    float2 A = make_float2(0.f, 0.f), B = A, C = A, D = A;                  \
    _Pragma("unroll") for (int j = 0; j < CPL; ++j) {                       \
      A = pfma(w.r[P][j], w.r[Q][j], A);                                    \
      B = pfma(w.i[P][j], w.i[Q][j], B);                                    \
      C = pfma(w.i[P][j], w.r[Q][j], C);                                    \
      D = pfma(w.r[P][j], w.i[Q][j], D);                                    \
    }                                                                       \
    const float2 AB = pfma(B, ONE2, A), CD = pfma(D, MONE2, C);             \
    v[2 * K] = AB.x + AB.y;                                                 \
    v[2 * K + 1] = CD.x + CD.y;                                             \
  }
  LT_BJ_DOT(0, P0, Q0)
  LT_BJ_DOT(1, P1, Q1)
  LT_BJ_DOT(2, P2, Q2)
  LT_BJ_DOT(3, P3, Q3)
#undef LT_BJ_DOT
  // reduce-scatter: afterwards lane l holds value (l >> 2) summed over the warp
  {
    const bool hi = lane & 16;
    float k4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float send = hi ? v[t] : v[4 + t];
      const float keep = hi ? v[4 + t] : v[t];
      k4[t] = keep + __shfl_xor_sync(FULL, send, 16);
    }
    const bool h8 = lane & 8;
    float k2[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float send = h8 ? k4[t] : k4[2 + t];
      const float keep = h8 ? k4[2 + t] : k4[t];
      k2[t] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    const bool h4 = lane & 4;
    float k1 = (h4 ? k2[1] : k2[0]) + __shfl_xor_sync(FULL, h4 ? k2[0] : k2[1], 4);
    k1 += __shfl_xor_sync(FULL, k1, 2);
    k1 += __shfl_xor_sync(FULL, k1, 1);
    v[0] = k1;
  }
  if constexpr (GW > 1) {
    float* pb = grp.part + grp.buf * (GW * 8);
    if ((lane & 3) == 0) pb[grp.wg * 8 + (lane >> 2)] = v[0];
    asm volatile("bar.sync %0, %1;" ::"r"(grp.bar), "r"(GW * 32) : "memory");
    float sum = pb[lane >> 2];
#pragma unroll
    for (int t = 1; t < GW; ++t) sum += pb[t * 8 + (lane >> 2)];
    v[0] = sum;
    grp.buf ^= 1;
  }
  // lanes 8k..8k+3 hold gx of pair k, lanes 8k+4..8k+7 its gy
  const float other = __shfl_xor_sync(FULL, v[0], 4);
  const float gx = (lane & 4) ? other : v[0];
  const float gy = (lane & 4) ? v[0] : other;
  const int k = lane >> 3;
  const int sp = k == 0 ? P0 : k == 1 ? P1 : k == 2 ? P2 : P3;
  const int sq = k == 0 ? Q0 : k == 1 ? Q1 : k == 2 ? Q2 : Q3;
  const float alpha = __shfl_sync(FULL, w.nrl, sp);
  const float beta = __shfl_sync(FULL, w.nrl, sq);
  float cs = 1.f, sex = 0.f, sey = 0.f, tga = 0.f;
  const int rot = rot_params(gx, gy, alpha, beta, tol, cs, sex, sey, tga) ? 1 : 0;
  const unsigned rmask = __ballot_sync(FULL, rot);
#define LT_BJ_ROT(K, P, Q)                                                    \
  if (rmask & (1u << (8 * K))) {                                             \
    const float c_ = __shfl_sync(FULL, cs, 8 * K);                           \
    const float x_ = __shfl_sync(FULL, sex, 8 * K);                          \
    const float y_ = __shfl_sync(FULL, sey, 8 * K);                          \
    const float t_ = __shfl_sync(FULL, tga, 8 * K);                          \
    const float2 CS = make_float2(c_, c_), SX = make_float2(x_, x_);         \
    const float2 SY = make_float2(y_, y_), NSX = make_float2(-x_, -x_);      \
    const float2 NSY = make_float2(-y_, -y_);                                \
    _Pragma("unroll") for (int j = 0; j < CPL; ++j) {                        \
      const float2 xr = w.r[P][j], xi = w.i[P][j], yr = w.r[Q][j], yi = w.i[Q][j]; \
      w.r[P][j] = pfma(SY, yi, pfma(NSX, yr, pmul(CS, xr)));                 \
      w.i[P][j] = pfma(NSY, yr, pfma(NSX, yi, pmul(CS, xi)));                \
      w.r[Q][j] = pfma(SY, xi, pfma(SX, xr, pmul(CS, yr)));                  \
      w.i[Q][j] = pfma(NSY, xr, pfma(SX, xi, pmul(CS, yi)));                 \
    }                                                                        \
    {                                                                        \
      const int rl = threadIdx.x & 7;                                        \
      w.nrl += rl == Q ? t_ : (rl == P ? -t_ : 0.f);                         \
    }                                                                        \
    any = 1;                                                                 \
    ++nrot;                                                                  \
  }
  LT_BJ_ROT(0, P0, Q0)
  LT_BJ_ROT(1, P1, Q1)
  LT_BJ_ROT(2, P2, Q2)
  LT_BJ_ROT(3, P3, Q3)
#undef LT_BJ_ROT
}

// Sweeps over the mp (multiple of 8, rows m..mp-1 zero) rows of the planar
// matrix; returns the number of sweeps.  CPL element pairs per lane and row
// cover npad = 64 CPL columns (lanes beyond npad hold zeros).
template <int CPL>
__device__ int jacobi_blocked(float* Xr, float* Xi, int ldp, int mp, int n, int npad, float* nrm,
                              int* nrot_out, int max_sweeps, double tol_override) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int NB = mp >> 2;  // even
  const float tol = tol_override > 0.0 ? (float)tol_override : FLT_EPSILON * sqrtf((float)n);
  BJGroup grp{nullptr, 0, 0, 0};
  int nrot = 0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    __syncthreads();
    for (int r = warp; r < mp; r += nw) {
      float acc = 0.f;
      for (int c = lane; c < n; c += 32) {
        const float u = Xr[r * ldp + c], v = Xi[r * ldp + c];
        acc = fmaf(u, u, fmaf(v, v, acc));
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (lane == 0) nrm[r] = acc;
    }
    __syncthreads();
    int any = 0;
    for (int br = 0; br < NB - 1; ++br) {
      for (int bp = warp; bp < (NB >> 1); bp += nw) {
        int A, B;
        rr_pair(br, bp, NB, A, B);
        BJRows<CPL> w;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int row = t < 4 ? 4 * A + t : 4 * B + (t - 4);
          if (t == (lane & 7)) w.nrl = nrm[row];
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
            const int c = 2 * lane + 64 * j;
            if (c < npad) {
              w.r[t][j] = *reinterpret_cast<const float2*>(Xr + row * ldp + c);
              w.i[t][j] = *reinterpret_cast<const float2*>(Xi + row * ldp + c);
            } else {
              w.r[t][j] = make_float2(0.f, 0.f);
              w.i[t][j] = make_float2(0.f, 0.f);
            }
          }
        }
        if (br == 0) {
          // pairs inside each block: circle method on four rows
          bj_subround<CPL, 1, 0, 3, 1, 2, 4, 7, 5, 6>(w, tol, any, nrot, grp);
          bj_subround<CPL, 1, 1, 3, 2, 0, 5, 7, 6, 4>(w, tol, any, nrot, grp);
          bj_subround<CPL, 1, 2, 3, 0, 1, 6, 7, 4, 5>(w, tol, any, nrot, grp);
        }
        bj_subround<CPL, 1, 0, 4, 1, 5, 2, 6, 3, 7>(w, tol, any, nrot, grp);
        bj_subround<CPL, 1, 0, 5, 1, 6, 2, 7, 3, 4>(w, tol, any, nrot, grp);
        bj_subround<CPL, 1, 0, 6, 1, 7, 2, 4, 3, 5>(w, tol, any, nrot, grp);
        bj_subround<CPL, 1, 0, 7, 1, 4, 2, 5, 3, 6>(w, tol, any, nrot, grp);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int row = t < 4 ? 4 * A + t : 4 * B + (t - 4);
          if (lane == t) nrm[row] = w.nrl;
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
            const int c = 2 * lane + 64 * j;
            if (c < npad) {
              *reinterpret_cast<float2*>(Xr + row * ldp + c) = w.r[t][j];
              *reinterpret_cast<float2*>(Xi + row * ldp + c) = w.i[t][j];
            }
          }
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(any)) break;
  }
  if (lane == 0 && nrot) atomicAdd(nrot_out, nrot);
  return sweep + 1;
}

// ---- thread-block clusters ------------------------------------------------------------
__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return (int)r;
}
__device__ __forceinline__ int cluster_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return (int)r;
}
// every thread of every CTA of the cluster; writes before it are visible after it
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Block Jacobi for rows of 128 < n <= 512 columns (single precision, the same
// rotations and circle-method block order as jacobi_blocked): groups of G warps take
// a pair of 4-row blocks at a time, warp g of a group the columns [128 g, 128 g + 128)
// of its eight rows in registers, the inner products summed over the group (BJGroup).
// The rows stay in the workspace (global scratch for these sizes) between block rounds,
// so a sweep moves the matrix through the registers NB - 1 times instead of once per
// row pair.  npad = 128 G columns, mp (a multiple of 8) rows; the window beyond the
// r x r factor is zero.  part: [NT/32/G][2][G][8] floats of shared memory.
// With C > 1 the C CTAs of a thread-block cluster share the sweeps: the block pairs of
// a round are dealt over all their groups, a cluster barrier separates the rounds, the
// row norms live in global memory (nrm), the rows and norms are read past L1 (another
// SM may have written them), and cl[0..1] (zero on entry) carry the "any rotation" flag
// of alternate sweeps, cl[2] the rotation count.  Every CTA of the cluster takes the
// same number of barriers: the loop bounds and the convergence test are cluster-wide.
template <int G>
__device__ __noinline__ int jacobi_wide(float* Xr, float* Xi, int ldp, int mp, int n, float* nrm,
                                        float* part, int* nrot_out, int max_sweeps,
                                        double tol_override, int crank, int C, int* cl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ngr = nw / G, gid = warp / G, wg = warp - gid * G;
  const bool active = gid < ngr;
  const bool shared = C > 1;
  const int NB = mp >> 2;  // even
  const float tol = tol_override > 0.0 ? (float)tol_override : FLT_EPSILON * sqrtf((float)n);
  BJGroup grp{part + (active ? gid : 0) * 2 * G * 8, 1 + gid, wg, 0};
  auto ld = [&](const float* q) { return shared ? __ldcg(q) : *q; };
  auto ld2 = [&](const float* q) {
    return shared ? __ldcg(reinterpret_cast<const float2*>(q)) : *reinterpret_cast<const float2*>(q);
  };
  auto sync = [&]() {
    if (shared)
      cluster_sync();
    else
      __syncthreads();
  };
  int nrot = 0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    sync();
    for (int r = crank * nw + warp; r < mp; r += C * nw) {
      float acc = 0.f;
      for (int c = lane; c < n; c += 32) {
        const float u = ld(Xr + (long long)r * ldp + c), v = ld(Xi + (long long)r * ldp + c);
        acc = fmaf(u, u, fmaf(v, v, acc));
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (lane == 0) nrm[r] = acc;
    }
    sync();
    // the flag of the sweep before the last was read by every CTA before this barrier
    if (shared && sweep > 0 && crank == 0 && threadIdx.x == 0) cl[(sweep + 1) & 1] = 0;
    int any = 0;
    for (int br = 0; br < NB - 1; ++br) {
      if (active) {
        for (int bp = crank * ngr + gid; bp < (NB >> 1); bp += C * ngr) {
          int A, B;
          rr_pair(br, bp, NB, A, B);
          BJRows<2> w;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int row = t < 4 ? 4 * A + t : 4 * B + (t - 4);
            if (t == (lane & 7)) w.nrl = ld(nrm + row);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const long long o = (long long)row * ldp + 128 * wg + 2 * lane + 64 * j;
              w.r[t][j] = ld2(Xr + o);
              w.i[t][j] = ld2(Xi + o);
            }
          }
          if (br == 0) {
            bj_subround<2, G, 0, 3, 1, 2, 4, 7, 5, 6>(w, tol, any, nrot, grp);
            bj_subround<2, G, 1, 3, 2, 0, 5, 7, 6, 4>(w, tol, any, nrot, grp);
            bj_subround<2, G, 2, 3, 0, 1, 6, 7, 4, 5>(w, tol, any, nrot, grp);
          }
          bj_subround<2, G, 0, 4, 1, 5, 2, 6, 3, 7>(w, tol, any, nrot, grp);
          bj_subround<2, G, 0, 5, 1, 6, 2, 7, 3, 4>(w, tol, any, nrot, grp);
          bj_subround<2, G, 0, 6, 1, 7, 2, 4, 3, 5>(w, tol, any, nrot, grp);
          bj_subround<2, G, 0, 7, 1, 4, 2, 5, 3, 6>(w, tol, any, nrot, grp);
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int row = t < 4 ? 4 * A + t : 4 * B + (t - 4);
            if (wg == 0 && lane == t) nrm[row] = w.nrl;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const long long o = (long long)row * ldp + 128 * wg + 2 * lane + 64 * j;
              *reinterpret_cast<float2*>(Xr + o) = w.r[t][j];
              *reinterpret_cast<float2*>(Xi + o) = w.i[t][j];
            }
          }
        }
      }
      sync();
    }
    int more = __syncthreads_or(any);
    if (shared) {
      if (threadIdx.x == 0 && more) atomicOr(cl + (sweep & 1), 1);
      __threadfence();
      cluster_sync();
      more = __ldcg(cl + (sweep & 1));
    }
    if (!more) break;
  }
  if (lane == 0 && wg == 0 && nrot) atomicAdd(shared ? cl + 2 : nrot_out, nrot);
  return sweep + 1;
}

// The wide Jacobi of one task, by one CTA (C = 1) or shared by the C CTAs of a cluster
// (cl: the cluster's LT_CL_STATE floats in global memory: row norms, then the flags and
// the rotation count).  The cluster variant starts and ends with a cluster barrier, so
// that rank 0's preconditioned factor is visible to all before the sweeps and every row
// to rank 0 after them; rank 0 adds the cluster's rotations to *nrot.
__device__ __noinline__ int wide_jacobi(float* Xr, float* Xi, int ldp, int mp, int n, int npad,
                                        float* s_nrm, float* part, int* nrot, int max_sweeps,
                                        double tol, int C, int crank, float* cl_state) {
  float* nrm = s_nrm;
  int* cl = nullptr;
  if (C > 1) {
    nrm = cl_state;
    cl = reinterpret_cast<int*>(cl_state + LT_MAX_DIM);
    if (crank == 0 && threadIdx.x == 0) cl[0] = cl[1] = cl[2] = 0;
    __threadfence();
    cluster_sync();
  }
  int sweeps;
  if (npad == 256)
    sweeps = jacobi_wide<2>(Xr, Xi, ldp, mp, n, nrm, part, nrot, max_sweeps, tol, crank, C, cl);
  else if (npad == 384)
    sweeps = jacobi_wide<3>(Xr, Xi, ldp, mp, n, nrm, part, nrot, max_sweeps, tol, crank, C, cl);
  else
    sweeps = jacobi_wide<4>(Xr, Xi, ldp, mp, n, nrm, part, nrot, max_sweeps, tol, crank, C, cl);
  if (C > 1) {
    __threadfence();
    cluster_sync();
    __threadfence();
    if (crank == 0 && threadIdx.x == 0) *nrot += __ldcg(cl + 2);
  }
  return sweeps;
}

// threads per CTA of the bond kernel per precision (the row-pair Jacobi holds 4 element
// pairs of each row per lane; 8 measured slower in every configuration, spilling)
template <typename R> struct BondShape;
template <> struct BondShape<float> { static constexpr int NT = 512; };
template <> struct BondShape<double> { static constexpr int NT = 256; };

// ---- two-level Householder preconditioning of the row Jacobi ---------------------------
// The one-sided Jacobi on the rows of X converges slowly when the rows are
// strongly graded (theta's rows carry the weights Lambda_{b-1}).  With an LQ
// factorisation X = L1 Q1^+ (Householder reflectors from the rows) followed by a
// QR factorisation L1 = Q2 R2, the rows of R2 = Q2^+ X Q1 are nearly orthogonal
// and the sweeps converge in a few rounds (the two-sided preconditioning of
// Drmac and Veselic, without pivoting).  Q2 is not needed: if the Jacobi turns
// the rows of R2 into sigma_j w_j^+, the right singular vectors of X are
// v_j^+ = w_j^+ Q1^+ = w_j^+ H_{r-1} ... H_0.
// On entry X (planar, m x n, row stride ldp) holds the matrix; on exit
// X[0:r, 0:r] holds R2 (upper triangular), every other entry is zero, and Vst
// holds the reflectors of Q1 = H_0 ... H_{r-1}: for a row x, x H_j = x - beta_j
// (sum_c x_c conj(e_c)) e with e the stored vector of H_j (the tail of row j
// plus ph alpha in its first entry), acting on columns j..n-1 and packed at
// offset sum_{i<j} (n - i).
template <typename R>
__device__ __forceinline__ void warp_sum2(R& a, R& b) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(FULL, a, o);
    b += __shfl_xor_sync(FULL, b, o);
  }
}

#define LT_QR_CH 8  // entries staged in registers per chunk of a Householder update

template <typename R> struct TinyNorm;
template <> struct TinyNorm<float> { static constexpr float v = 1e-18f; };
template <> struct TinyNorm<double> { static constexpr double v = 1e-150; };

// Reflector from the n-j entries x_t = X[p(t)] (stride st from base b0):
// alpha = |x|, ph = x_0/|x_0|; e = x + ph alpha e_0 is stored at dst, the entries
// are replaced by (-ph alpha, 0, ...), and beta = 2/|e|^2 is returned (0 when
// alpha is below TinyNorm, in which case the entries are simply set to zero:
// they are below any precision of the result).  One warp.
// The unit phase x0 / |x0| and |x0| of a reflector's leading entry.  x0 is scaled by
// max(|Re x0|, |Im x0|) before it is squared: on a rank-deficient theta single
// precision meets leading entries near 1e-23, whose square is subnormal, and a
// phase taken from that rounded square is not of modulus one, which makes the
// reflector non-unitary.
template <typename R>
__device__ __forceinline__ void unit_phase(R xr, R xi, R& phr, R& phi, R& ax) {
  const R m = fmax(fabs(xr), fabs(xi));
  if (!(m > (R)0)) {
    phr = (R)1;
    phi = (R)0;
    ax = (R)0;
    return;
  }
  const R sr = xr / m, si = xi / m;
  const R nn = sqrt(sr * sr + si * si);
  phr = sr / nn;
  phi = si / nn;
  ax = m * nn;
}

template <typename R, bool CG = false>
__device__ __forceinline__ R make_reflector(R* Xr, R* Xi, int base, int st, int len,
                                            typename CT<R>::T* dst) {
  typedef typename CT<R>::T Tc;
  // CG: the entries may have been written by another CTA of the cluster; read past L1
  auto ld = [](const R* p) { return CG ? __ldcg(p) : *p; };
  const int lane = threadIdx.x & 31;
  R a2 = 0, dummy = 0;
  for (int t = lane; t < len; t += 32) {
    const R u = ld(Xr + base + t * st), w = ld(Xi + base + t * st);
    a2 = fma(u, u, fma(w, w, a2));
  }
  warp_sum2(a2, dummy);
  const R x0r = ld(Xr + base), x0i = ld(Xi + base);
  const R alpha = sqrt(a2);
  const bool tiny = !(alpha > TinyNorm<R>::v);
  R phr, phi, ax0;
  unit_phase(x0r, x0i, phr, phi, ax0);
  for (int t = lane; t < len; t += 32) {
    Tc e = cmk<Tc>(ld(Xr + base + t * st), ld(Xi + base + t * st));
    if (t == 0) {
      e.x += phr * alpha;
      e.y += phi * alpha;
    }
    dst[t] = tiny ? czero<Tc>() : e;
    Xr[base + t * st] = (t == 0 && !tiny) ? -phr * alpha : (R)0;
    Xi[base + t * st] = (t == 0 && !tiny) ? -phi * alpha : (R)0;
  }
  return tiny ? (R)0 : (R)2 / (2 * alpha * (alpha + ax0));
}

// One LQ step on rows j+1..m-1 of a wide matrix: a warp takes a row at a time, lane l
// the columns l + 32 u (coalesced), with the row and the reflector e (len <= 32 EPL
// entries) in registers; the inner product is summed over the warp.
template <typename R, int EPL>
__device__ __forceinline__ void lq_update_warp(R* Xr, R* Xi, int ldp, int m, int j, int len,
                                               const typename CT<R>::T* e, R bt) {
  typedef typename CT<R>::T Tc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (j + 1 + warp >= m) return;
  Tc ev[EPL];
#pragma unroll
  for (int u = 0; u < EPL; ++u) {
    const int c = lane + 32 * u;
    ev[u] = c < len ? e[c] : czero<Tc>();
  }
  for (int i = j + 1 + warp; i < m; i += nw) {
    R* __restrict__ xr = Xr + (long long)i * ldp + j;
    R* __restrict__ xi = Xi + (long long)i * ldp + j;
    R a[EPL], b[EPL];
    R dr = 0, di = 0;  // d = sum_c x_c conj(e_c)
#pragma unroll
    for (int u = 0; u < EPL; ++u) {
      const int c = lane + 32 * u;
      a[u] = c < len ? xr[c] : (R)0;
      b[u] = c < len ? xi[c] : (R)0;
      dr = fma(a[u], ev[u].x, fma(b[u], ev[u].y, dr));
      di = fma(b[u], ev[u].x, fma(-a[u], ev[u].y, di));
    }
    warp_sum2(dr, di);
    dr *= bt;
    di *= bt;
#pragma unroll
    for (int u = 0; u < EPL; ++u) {  // x -= beta d e
      const int c = lane + 32 * u;
      if (c < len) {
        xr[c] = a[u] - fma(dr, ev[u].x, -di * ev[u].y);
        xi[c] = b[u] - fma(dr, ev[u].y, di * ev[u].x);
      }
    }
  }
}

// In-place conjugate transpose of the leading m x m block of the planar matrix
// (barriers before and after); CG: read past L1 (other CTAs of a cluster wrote it).
template <typename R, bool CG = false>
__device__ void conj_transpose_square(R* Xr, R* Xi, int ldp, int m) {
  auto ld = [](const R* p) { return CG ? __ldcg(p) : *p; };
  __syncthreads();
  const int np = m * (m + 1) / 2;  // entries on and above the diagonal
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    // row i, column j >= i of the upper triangle, t enumerating rows of m - i entries
    int i = (int)((2.0 * m + 1.0 - sqrt((2.0 * m + 1.0) * (2.0 * m + 1.0) - 8.0 * t)) / 2.0);
    while (i > 0 && (long long)i * (2 * m - i + 1) / 2 > t) --i;
    while ((long long)(i + 1) * (2 * m - i) / 2 <= t) ++i;
    const int j = i + (t - i * (2 * m - i + 1) / 2);
    const long long a = (long long)i * ldp + j, b = (long long)j * ldp + i;
    const R ar = ld(Xr + a), ai = ld(Xi + a), br = ld(Xr + b), bi = ld(Xi + b);
    Xr[a] = br;
    Xi[a] = -bi;
    Xr[b] = ar;
    Xi[b] = -ai;
  }
  __syncthreads();
}

// An LQ (rows 0..m-1 of n columns, r reflectors) shared by the C CTAs of a cluster, the
// same arithmetic as qr_precondition's warp-per-row steps: row i belongs to warp
// i mod (C nw) of the cluster (warp w of rank c is number c nw + w), whose lanes hold its
// columns l + 32 u; the owner of row j builds reflector j into E (packed at the offset
// sum_{t<j} (n - t), or into two buffers in turn) and its beta into gb (gb[j], or the
// two in turn); one cluster barrier per step, and one at the end.  Rows and reflectors
// are read past L1: other CTAs write them.
template <int EPL>
__device__ void lq_cluster(float* Xr, float* Xi, int ldp, int m, int n, int r, float2* E,
                           bool packed, float* gb, int crank, int C) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int GW = C * nw, gw = crank * nw + warp;
  long long off = 0;
  for (int j = 0; j < r; ++j) {
    const int len = n - j;
    float2* e = packed ? E + off : E + (j & 1) * LT_MAX_DIM;
    float* bp = packed ? gb + j : gb + (j & 1);
    if (j % GW == gw) {
      const float bt = make_reflector<float, true>(Xr, Xi, j * ldp + j, 1, len, e);
      if (lane == 0) *bp = bt;
    }
    __threadfence();
    cluster_sync();
    const float bt = __ldcg(bp);
    // this warp's first row after j
    const int i0 = j + 1 + (((gw - (j + 1)) % GW) + GW) % GW;
    if (bt != 0.f && i0 < m) {
      float2 ev[EPL];
#pragma unroll
      for (int u = 0; u < EPL; ++u) {
        const int c = lane + 32 * u;
        ev[u] = c < len ? __ldcg(e + c) : make_float2(0.f, 0.f);
      }
      for (int i = i0; i < m; i += GW) {
        float* __restrict__ xr = Xr + (long long)i * ldp + j;
        float* __restrict__ xi = Xi + (long long)i * ldp + j;
        float a[EPL], b[EPL];
        float dr = 0.f, di = 0.f;  // d = sum_c x_c conj(e_c)
#pragma unroll
        for (int u = 0; u < EPL; ++u) {
          const int c = lane + 32 * u;
          a[u] = c < len ? __ldcg(xr + c) : 0.f;
          b[u] = c < len ? __ldcg(xi + c) : 0.f;
          dr = fmaf(a[u], ev[u].x, fmaf(b[u], ev[u].y, dr));
          di = fmaf(b[u], ev[u].x, fmaf(-a[u], ev[u].y, di));
        }
        warp_sum2(dr, di);
        dr *= bt;
        di *= bt;
#pragma unroll
        for (int u = 0; u < EPL; ++u) {  // x -= beta d e
          const int c = lane + 32 * u;
          if (c < len) {
            xr[c] = a[u] - fmaf(dr, ev[u].x, -di * ev[u].y);
            xi[c] = b[u] - fmaf(dr, ev[u].y, di * ev[u].x);
          }
        }
      }
    }
    off += len;
  }
  __threadfence();
  cluster_sync();
}

// The two-level preconditioning of a task with m <= n and m > 128, shared by the C CTAs
// of a cluster (the same factors as qr_precondition): the LQ of theta with its reflectors
// packed into Vst and its betas in the cluster state, then the QR of the square L1 as
// the LQ of L1^+ (rank 0 transposes before and after).  Starts with a cluster barrier
// (rank 0's theta visible); every CTA takes the same barriers.
__device__ __noinline__ void precondition_cluster(float* Xr, float* Xi, int ldp, int m, int n,
                                                  float2* Vst, float* cl_state, int crank,
                                                  int C) {
  __threadfence();
  cluster_sync();
  if (n > 256)
    lq_cluster<16>(Xr, Xi, ldp, m, n, m, Vst, true, cl_state + LT_CL_B1, crank, C);
  else
    lq_cluster<8>(Xr, Xi, ldp, m, n, m, Vst, true, cl_state + LT_CL_B1, crank, C);
  if (crank == 0) conj_transpose_square<float, true>(Xr, Xi, ldp, m);
  __threadfence();
  cluster_sync();
  float2* E2 = reinterpret_cast<float2*>(cl_state + LT_CL_E2);
  if (m > 256)
    lq_cluster<16>(Xr, Xi, ldp, m, m, m, E2, false, cl_state + LT_CL_B2, crank, C);
  else
    lq_cluster<8>(Xr, Xi, ldp, m, m, m, E2, false, cl_state + LT_CL_B2, crank, C);
  if (crank == 0) conj_transpose_square<float, true>(Xr, Xi, ldp, m);
}

template <typename R>
__device__ void qr_precondition(R* Xr, R* Xi, int ldp, int m, int n, int r,
                                typename CT<R>::T* Vst, R* beta, typename CT<R>::T* su) {
  typedef typename CT<R>::T Tc;
  const int warp = threadIdx.x >> 5;
  __syncthreads();
  // LQ: H_j from the tail of row j, applied from the right to the rows below.  Rows of
  // up to 128 columns: a thread owns a row (no reductions across threads); longer rows
  // (global scratch): a warp takes a row at a time, coalesced (lq_update_warp)
  int off = 0;
  for (int j = 0; j < r; ++j) {
    Tc* e = Vst + off;
    const int len = n - j;
    if (warp == 0) {
      const R bt = make_reflector<R>(Xr, Xi, j * ldp + j, 1, len, e);
      if ((threadIdx.x & 31) == 0) beta[j] = bt;
    }
    __syncthreads();
    const R bt = beta[j];
    if (bt != (R)0 && n > 256) {
      lq_update_warp<R, 16>(Xr, Xi, ldp, m, j, len, e, bt);
    } else if (bt != (R)0 && n > 128) {
      lq_update_warp<R, 8>(Xr, Xi, ldp, m, j, len, e, bt);
    } else if (bt != (R)0) {
      const Tc* __restrict__ ev = e;
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
        R* __restrict__ xr = Xr + i * ldp + j;
        R* __restrict__ xi = Xi + i * ldp + j;
        R dr = 0, di = 0;  // d = sum_c x_c conj(e_c), in chunks staged in registers
        for (int c0 = 0; c0 < len; c0 += LT_QR_CH) {
          R a[LT_QR_CH], b[LT_QR_CH];
          Tc w[LT_QR_CH];
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            const bool in = c0 + u < len;
            a[u] = in ? xr[c0 + u] : (R)0;
            b[u] = in ? xi[c0 + u] : (R)0;
            w[u] = in ? ev[c0 + u] : czero<Tc>();
          }
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            dr = fma(a[u], w[u].x, fma(b[u], w[u].y, dr));
            di = fma(b[u], w[u].x, fma(-a[u], w[u].y, di));
          }
        }
        dr *= bt;
        di *= bt;
        for (int c0 = 0; c0 < len; c0 += LT_QR_CH) {  // x -= beta d e
          R a[LT_QR_CH], b[LT_QR_CH];
          Tc w[LT_QR_CH];
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            const bool in = c0 + u < len;
            a[u] = in ? xr[c0 + u] : (R)0;
            b[u] = in ? xi[c0 + u] : (R)0;
            w[u] = in ? ev[c0 + u] : czero<Tc>();
          }
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            if (c0 + u < len) {
              xr[c0 + u] = a[u] - fma(dr, w[u].x, -di * w[u].y);
              xi[c0 + u] = b[u] - fma(dr, w[u].y, di * w[u].x);
            }
          }
        }
      }
    }
    __syncthreads();
    off += len;
  }
  if (r == m && m > 128) {
    // square L1 wider than 128: its QR as the LQ of L1^+ (if L1^+ = L' Q^+ then
    // L1 = Q L'^+, so R2 = L'^+ with the same diagonal phases), which takes the
    // coalesced warp-per-row steps; the reflectors go through su, Q is discarded
    conj_transpose_square(Xr, Xi, ldp, m);
    for (int j = 0; j < m; ++j) {
      const int len = m - j;
      if (warp == 0) {
        const R bt = make_reflector<R>(Xr, Xi, j * ldp + j, 1, len, su);
        if ((threadIdx.x & 31) == 0) beta[LT_MAX_DIM] = bt;
      }
      __syncthreads();
      const R bt = beta[LT_MAX_DIM];
      if (bt != (R)0) {
        if (m > 256)
          lq_update_warp<R, 16>(Xr, Xi, ldp, m, j, len, su, bt);
        else
          lq_update_warp<R, 8>(Xr, Xi, ldp, m, j, len, su, bt);
      }
      __syncthreads();
    }
    conj_transpose_square(Xr, Xi, ldp, m);
    return;
  }
  // QR of the lower-trapezoidal L1 (columns 0..r-1): reflectors from the columns,
  // applied from the left to the columns on their right, one thread per column;
  // Q2 is discarded
  for (int j = 0; j < r; ++j) {
    const int len = m - j;
    if (warp == 0) {
      const R bt = make_reflector<R>(Xr, Xi, j * ldp + j, ldp, len, su);
      if ((threadIdx.x & 31) == 0) beta[LT_MAX_DIM] = bt;
    }
    __syncthreads();
    const R bt = beta[LT_MAX_DIM];
    if (bt != (R)0) {
      const Tc* __restrict__ uv = su;
      for (int c = j + 1 + threadIdx.x; c < r; c += blockDim.x) {
        R* __restrict__ xr = Xr + j * ldp + c;
        R* __restrict__ xi = Xi + j * ldp + c;
        R dr = 0, di = 0;  // d = sum_i conj(u_i) x_i
        for (int t0 = 0; t0 < len; t0 += LT_QR_CH) {
          R a[LT_QR_CH], b[LT_QR_CH];
          Tc w[LT_QR_CH];
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            const bool in = t0 + u < len;
            a[u] = in ? xr[(t0 + u) * ldp] : (R)0;
            b[u] = in ? xi[(t0 + u) * ldp] : (R)0;
            w[u] = in ? uv[t0 + u] : czero<Tc>();
          }
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            dr = fma(w[u].x, a[u], fma(w[u].y, b[u], dr));
            di = fma(w[u].x, b[u], fma(-w[u].y, a[u], di));
          }
        }
        dr *= bt;
        di *= bt;
        for (int t0 = 0; t0 < len; t0 += LT_QR_CH) {  // x -= u d
          R a[LT_QR_CH], b[LT_QR_CH];
          Tc w[LT_QR_CH];
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            const bool in = t0 + u < len;
            a[u] = in ? xr[(t0 + u) * ldp] : (R)0;
            b[u] = in ? xi[(t0 + u) * ldp] : (R)0;
            w[u] = in ? uv[t0 + u] : czero<Tc>();
          }
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            if (t0 + u < len) {
              xr[(t0 + u) * ldp] = a[u] - fma(w[u].x, dr, -w[u].y * di);
              xi[(t0 + u) * ldp] = b[u] - fma(w[u].x, di, w[u].y * dr);
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

// ---- the same preconditioning in single precision, rows held in registers -------------
// Identical factorisation and reflector convention as qr_precondition, but each
// row stays in the registers of G lanes for the whole factorisation: thread t
// holds row t / G, lane q = t % G the columns c = G s + q (s < 128 / G), packed
// as float2 pairs h (column 2 G h + q in .x, 2 G h + G + q in .y).  A step only
// reads its reflector from shared memory, and the lanes of the next row build
// the next reflector into the other of two buffers, so each reflector costs one
// barrier.  The QR of L1 runs as the LQ of L1^+ (L1 is written
// conjugate-transposed to shared memory in between): if L1^+ = L' Q^+ then
// L1 = Q L'^+, so R2 = L'^+ with the same diagonal phases.
template <int G>
struct LQRow {
  static constexpr int NH = 64 / G;  // float2 pairs per lane (128 columns)
  float2 r[NH], i[NH];
};

// floats between the G lanes' parts of a reflector buffer (2 spare floats per
// part shift the banks, so the G broadcast reads of a step are conflict-free)
template <int G> struct LQBuf { static constexpr int PART = 128 / G + 2, SIZE = G * PART; };

__device__ __forceinline__ bool lq_block_live(int hb, int j0, int ncol) {
  return 16 * hb + 16 > j0 && 16 * hb < ncol;  // columns 16 hb .. 16 hb + 15
}

template <int G>
__device__ __forceinline__ void lq_load(LQRow<G>& x, const float* Xr, const float* Xi, int ld,
                                        int row, int nrow, int ncol, int q) {
#pragma unroll
  for (int h = 0; h < LQRow<G>::NH; ++h) {
    const int c0 = 2 * G * h + q, c1 = c0 + G;
    const bool ok = row < nrow;
    x.r[h] = make_float2(ok && c0 < ncol ? Xr[row * ld + c0] : 0.f,
                         ok && c1 < ncol ? Xr[row * ld + c1] : 0.f);
    x.i[h] = make_float2(ok && c0 < ncol ? Xi[row * ld + c0] : 0.f,
                         ok && c1 < ncol ? Xi[row * ld + c1] : 0.f);
  }
}

// x <- x - beta (sum_c x_c conj(e_c)) e over the live column blocks; er/ei is
// this lane's part of the reflector buffer
template <int G>
__device__ __forceinline__ void lq_apply(LQRow<G>& x, const float* er, const float* ei, float bt,
                                         int j0, int ncol) {
  constexpr int HPB = 8 / G;  // pairs per 16-column block
  float2 A = make_float2(0.f, 0.f), B = A, C = A, D = A;
#pragma unroll
  for (int hb = 0; hb < 8; ++hb) {
    if (lq_block_live(hb, j0, ncol)) {
#pragma unroll
      for (int u = 0; u < HPB; ++u) {
        const int h = HPB * hb + u;
        const float2 a = *reinterpret_cast<const float2*>(er + 2 * h);
        const float2 b = *reinterpret_cast<const float2*>(ei + 2 * h);
        A = pfma(x.r[h], a, A);
        B = pfma(x.i[h], b, B);
        C = pfma(x.i[h], a, C);
        D = pfma(x.r[h], b, D);
      }
    }
  }
  float dr = (A.x + A.y) + (B.x + B.y), di = (C.x + C.y) - (D.x + D.y);
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    dr += __shfl_xor_sync(FULL, dr, o);
    di += __shfl_xor_sync(FULL, di, o);
  }
  const float2 NDR = make_float2(-dr * bt, -dr * bt);
  const float2 DI = make_float2(di * bt, di * bt), NDI = make_float2(-di * bt, -di * bt);
#pragma unroll
  for (int hb = 0; hb < 8; ++hb) {
    if (lq_block_live(hb, j0, ncol)) {
#pragma unroll
      for (int u = 0; u < HPB; ++u) {
        const int h = HPB * hb + u;
        const float2 a = *reinterpret_cast<const float2*>(er + 2 * h);
        const float2 b = *reinterpret_cast<const float2*>(ei + 2 * h);
        x.r[h] = pfma(NDR, a, pfma(DI, b, x.r[h]));   // xr - dr ar + di ai
        x.i[h] = pfma(NDR, b, pfma(NDI, a, x.i[h]));  // xi - dr ai - di ar
      }
    }
  }
}

// Reflector from row jn (columns jn .. ncol-1), built by that row's G lanes
// into the buffer ebr/ebi (all parts): e = x + ph alpha e_jn, entries below jn
// zero; beta = 2 / |e|^2 (0 below TinyNorm) and the diagonal -ph alpha of L.
template <int G>
__device__ __forceinline__ void lq_build(const LQRow<G>& x, float* ebr, float* ebi, int jn,
                                         int ncol, int q, float* bt_out, float2* diag) {
  constexpr int HPB = 8 / G, PART = LQBuf<G>::PART;
  const unsigned pm = ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  float* er = ebr + q * PART;
  float* ei = ebi + q * PART;
  float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int hb = 0; hb < 8; ++hb) {
    if (lq_block_live(hb, jn, ncol)) {
#pragma unroll
      for (int u = 0; u < HPB; ++u) {
        const int h = HPB * hb + u, c0 = 2 * G * h + q;
        float2 vr = x.r[h], vi = x.i[h];
        if (c0 < jn) {
          vr.x = 0.f;
          vi.x = 0.f;
        }
        if (c0 + G < jn) {
          vr.y = 0.f;
          vi.y = 0.f;
        }
        n2 = pfma(vr, vr, pfma(vi, vi, n2));
        *reinterpret_cast<float2*>(er + 2 * h) = vr;
        *reinterpret_cast<float2*>(ei + 2 * h) = vi;
      }
    }
  }
  float a2 = n2.x + n2.y;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) a2 += __shfl_xor_sync(pm, a2, o);
  __syncwarp(pm);
  if (q == 0) {
    const int p = (jn % G) * PART + jn / G;
    const float x0r = ebr[p], x0i = ebi[p];
    // square roots from the refined reciprocal square root (about one ulp)
    const float alpha = a2 > 0.f ? a2 * rsqrt_nr(a2) : 0.f;
    const bool tiny = !(alpha > TinyNorm<float>::v);
    float phr, phi, ax0;
    unit_phase(x0r, x0i, phr, phi, ax0);
    ebr[p] = x0r + phr * alpha;
    ebi[p] = x0i + phi * alpha;
    *bt_out = tiny ? 0.f : __frcp_rn(alpha * (alpha + ax0));
    diag[jn] = tiny ? make_float2(0.f, 0.f) : make_float2(-phr * alpha, -phi * alpha);
  }
  __syncwarp(pm);
}

// LQ of the nrow x ncol (<= 128 x 128) matrix in the LQRow of every thread
// (rows >= nrow zero), r reflectors.  On return row i of L is x for columns
// below i, diag[i] at column i and zero beyond.  With Vst, reflector j is also
// stored packed there (ncol - j entries from column j), its beta in beta[j].
template <int G>
__device__ void lq_rows(LQRow<G>& x, int nrow, int ncol, int r, float2* Vst, float* beta,
                        float (*ebr)[LQBuf<G>::SIZE], float (*ebi)[LQBuf<G>::SIZE], float* bt2,
                        float2* diag) {
  constexpr int PART = LQBuf<G>::PART, RPW = 32 / G;  // rows per warp
  const int t = threadIdx.x, row = t / G, q = t % G;
  const int wrow0 = (t >> 5) * RPW;
  if (row == 0) lq_build<G>(x, ebr[0], ebi[0], 0, ncol, q, bt2, diag);
  __syncthreads();
  int off = 0;
  for (int j = 0; j < r; ++j) {
    const int b = j & 1;
    if (Vst) {
      for (int c = j + t; c < ncol; c += blockDim.x) {
        const int p = (c % G) * PART + c / G;
        Vst[off + c - j] = make_float2(ebr[b][p], ebi[b][p]);
      }
      if (t == 0) beta[j] = bt2[b];
      off += ncol - j;
    }
    const float bt = bt2[b];
    // rows <= j are finished (H_j only touches their columns >= j, which the
    // caller replaces by the diagonal and zeros), so warps holding only such
    // rows skip the step
    if (bt != 0.f && wrow0 + RPW - 1 > j && wrow0 < nrow)
      lq_apply<G>(x, ebr[b] + q * PART, ebi[b] + q * PART, bt, j, ncol);
    if (j + 1 < r && row == j + 1)
      lq_build<G>(x, ebr[b ^ 1], ebi[b ^ 1], j + 1, ncol, q, bt2 + (b ^ 1), diag);
    __syncthreads();
  }
}

// Row `row` of L from the LQRow (see lq_rows), entry of pair h, element u, conjugated
template <int G>
__device__ __forceinline__ float2 lq_entry_conj(const LQRow<G>& x, int h, int u, int q, int row,
                                                int nrow, const float2* diag) {
  const int c = 2 * G * h + G * u + q;
  float2 v = make_float2(0.f, 0.f);
  if (row < nrow) {
    if (c < row) v = make_float2(u ? x.r[h].y : x.r[h].x, u ? x.i[h].y : x.i[h].x);
    else if (c == row) v = diag[row];
  }
  return make_float2(v.x, -v.y);
}

// Single-precision qr_precondition (same contract; blockDim.x = 128 G, m, n <=
// 128; X[0:mp2, 0:npad2] is the window the Jacobi reads afterwards)
template <int G>
__device__ void qr_precondition_reg(float* Xr, float* Xi, int ldp, int m, int n, int r, int mp2,
                                    int npad2, float2* Vst, float* beta) {
  __shared__ __align__(16) float s_ebr[2][LQBuf<G>::SIZE];
  __shared__ __align__(16) float s_ebi[2][LQBuf<G>::SIZE];
  __shared__ float s_bt2[2];
  __shared__ float2 s_diag[LT_REG_DIM];
  const int t = threadIdx.x, row = t / G, q = t % G;
  LQRow<G> x;
  __syncthreads();
  lq_load<G>(x, Xr, Xi, ldp, row, m, n, q);
  // level 1: X = L1 Q1^+ (r reflectors kept for the right singular vectors)
  lq_rows<G>(x, m, n, r, Vst, beta, s_ebr, s_ebi, s_bt2, s_diag);
  // L1^+ (r x m) into X with row stride m: r m <= mcap ldp, and X is no longer read
#pragma unroll
  for (int h = 0; h < LQRow<G>::NH; ++h)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int c = 2 * G * h + G * u + q;
      if (row < m && c < r) {
        const float2 v = lq_entry_conj<G>(x, h, u, q, row, m, s_diag);
        Xr[c * m + row] = v.x;
        Xi[c * m + row] = v.y;
      }
    }
  __syncthreads();
  lq_load<G>(x, Xr, Xi, m, row, r, m, q);
  // level 2: L1^+ = L' Q^+ (the reflectors are not needed)
  lq_rows<G>(x, r, m, r, nullptr, nullptr, s_ebr, s_ebi, s_bt2, s_diag);
  // R2 = L'^+ into the Jacobi window (zero outside r x r)
  if (row < npad2) {
#pragma unroll
    for (int h = 0; h < LQRow<G>::NH; ++h)
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int a = 2 * G * h + G * u + q;
        if (a < mp2) {
          const float2 v = lq_entry_conj<G>(x, h, u, q, row, r, s_diag);
          Xr[a * ldp + row] = v.x;
          Xi[a * ldp + row] = v.y;
        }
      }
  }
  __syncthreads();
}

// Right singular vectors from the Jacobi rows: for j < k, row p = perm[j] holds
// sigma_j w_j^+ in its first r entries; scaled to w_j^+ and multiplied by
// Q1^+ = H_{r-1} ... H_0 it becomes v_j^+ (n entries), written to Y[j].  Four
// lanes per row, each taking every fourth entry.
template <typename R>
__device__ void apply_q1(R* Xr, R* Xi, int ldp, int n, int r, int k, const int* perm,
                         const double* sig, const typename CT<R>::T* Vst, const R* beta,
                         typename CT<R>::T* Y, int ldy) {
  typedef typename CT<R>::T Tc;
  __syncthreads();
  const int q = threadIdx.x & 3;
  const int rows_per_pass = blockDim.x >> 2;
  const int passes = (k + rows_per_pass - 1) / rows_per_pass;
  for (int pass = 0; pass < passes; ++pass) {
    const int j = pass * rows_per_pass + (threadIdx.x >> 2);
    const bool act = j < k;
    const int p = act ? perm[j] : 0;
    R* xr = Xr + p * ldp;
    R* xi = Xi + p * ldp;
    if (act) {
      const double sg = sig[p];
      const R inv = sg > 0.0 ? (R)(1.0 / sqrt(sg)) : (R)0;
      for (int c = q; c < n; c += 4) {
        xr[c] *= inv;
        xi[c] *= inv;
      }
    }
    int off = r * n - r * (r - 1) / 2;
    for (int l = r - 1; l >= 0; --l) {
      off -= n - l;
      const R bt = beta[l];
      if (bt == (R)0) continue;  // uniform across the block
      const Tc* e = Vst + off;
      const int len = n - l;
      const Tc* __restrict__ ev = e;
      R dr = 0, di = 0;  // d = sum_c x_c conj(e_c)
      if (act)
        for (int c0 = q; c0 < len; c0 += 4 * LT_QR_CH) {
          R a[LT_QR_CH], b[LT_QR_CH];
          Tc w[LT_QR_CH];
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            const int c = c0 + 4 * u;
            const bool in = c < len;
            a[u] = in ? xr[l + c] : (R)0;
            b[u] = in ? xi[l + c] : (R)0;
            w[u] = in ? ev[c] : czero<Tc>();
          }
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            dr = fma(a[u], w[u].x, fma(b[u], w[u].y, dr));
            di = fma(b[u], w[u].x, fma(-a[u], w[u].y, di));
          }
        }
      dr += __shfl_xor_sync(FULL, dr, 1);
      di += __shfl_xor_sync(FULL, di, 1);
      dr += __shfl_xor_sync(FULL, dr, 2);
      di += __shfl_xor_sync(FULL, di, 2);
      dr *= bt;
      di *= bt;
      if (act)
        for (int c0 = q; c0 < len; c0 += 4 * LT_QR_CH) {  // x -= beta d e
          R a[LT_QR_CH], b[LT_QR_CH];
          Tc w[LT_QR_CH];
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            const int c = c0 + 4 * u;
            const bool in = c < len;
            a[u] = in ? xr[l + c] : (R)0;
            b[u] = in ? xi[l + c] : (R)0;
            w[u] = in ? ev[c] : czero<Tc>();
          }
#pragma unroll
          for (int u = 0; u < LT_QR_CH; ++u) {
            const int c = c0 + 4 * u;
            if (c < len) {
              xr[l + c] = a[u] - fma(dr, w[u].x, -di * w[u].y);
              xi[l + c] = b[u] - fma(dr, w[u].y, di * w[u].x);
            }
          }
        }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < k * n; idx += blockDim.x) {
    const int j = idx / n, c = idx - j * n;
    const int p = perm[j];
    Y[j * ldy + c] = cmk<Tc>(Xr[p * ldp + c], Xi[p * ldp + c]);
  }
}

// Single-precision apply_q1 (same contract; columns >= r of the Jacobi rows are
// taken as zero): G lanes per row (rows j = t / G < k), lane q holding columns
// G s + q (s < 128 / G) as float2 pairs (2 G h + q, 2 G h + G + q); the
// reflectors are read from their packed store with no barrier between them, and
// Y (which overlays that store) is written after one barrier at the end.
// V_k^+ for rows longer than 128 columns (single precision): a warp takes one of the k
// kept rows at a time and keeps it in registers (lane l the columns l + 32 u) through all
// r reflectors, which it reads coalesced; each inner product is summed over the warp.
// The same result as apply_q1 up to the order of the sums.  Rows are written back in
// place; the caller copies them into V_k^+'s region (which holds the reflectors until
// every row is done).  The k rows are dealt over the warps of `parts` CTAs (a cluster's),
// this CTA taking share `part`.
template <int EPL, bool CG = false>
__device__ void apply_q1_wide(float* Xr, float* Xi, int ldp, int n, int r, int k, const int* perm,
                              const double* sig, const float2* Vst, const float* beta, int part,
                              int parts) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int total = r * n - r * (r - 1) / 2;
  auto ld = [](const float* q) { return CG ? __ldcg(q) : *q; };
  for (int j = part * nw + warp; j < k; j += parts * nw) {
    const int p = CG ? __ldcg(perm + j) : perm[j];
    const double sg = CG ? __ldcg(sig + p) : sig[p];
    const float inv = sg > 0.0 ? (float)(1.0 / sqrt(sg)) : 0.f;
    float* xr = Xr + (long long)p * ldp;
    float* xi = Xi + (long long)p * ldp;
    float ar[EPL], ai[EPL];
#pragma unroll
    for (int u = 0; u < EPL; ++u) {
      const int c = lane + 32 * u;
      ar[u] = c < n ? ld(xr + c) * inv : 0.f;
      ai[u] = c < n ? ld(xi + c) * inv : 0.f;
    }
    int off = total;
    for (int l = r - 1; l >= 0; --l) {
      off -= n - l;
      const float bt = ld(beta + l);
      if (bt == 0.f) continue;
      const float2* e = Vst + off - l;  // e[c] for columns c >= l
      float dr = 0.f, di = 0.f;       // d = sum_c x_c conj(e_c)
      float2 w[EPL];
#pragma unroll
      for (int u = 0; u < EPL; ++u) {
        const int c = lane + 32 * u;
        w[u] = c >= l && c < n ? (CG ? __ldcg(e + c) : e[c]) : make_float2(0.f, 0.f);
        dr = fmaf(ar[u], w[u].x, fmaf(ai[u], w[u].y, dr));
        di = fmaf(ai[u], w[u].x, fmaf(-ar[u], w[u].y, di));
      }
      warp_sum2(dr, di);
      dr *= bt;
      di *= bt;
#pragma unroll
      for (int u = 0; u < EPL; ++u) {  // x -= beta d e
        ar[u] -= fmaf(dr, w[u].x, -di * w[u].y);
        ai[u] -= fmaf(dr, w[u].y, di * w[u].x);
      }
    }
#pragma unroll
    for (int u = 0; u < EPL; ++u) {
      const int c = lane + 32 * u;
      if (c < n) {
        xr[c] = ar[u];
        xi[c] = ai[u];
      }
    }
  }
}

// The generic preconditioning and V_k^+ of the single-precision kernel, kept out of line
// so that they do not take registers from its register paths.
__device__ __noinline__ void qr_precondition_f(float* Xr, float* Xi, int ldp, int m, int n, int r,
                                               float2* Vst, float* beta, float2* su) {
  qr_precondition<float>(Xr, Xi, ldp, m, n, r, Vst, beta, su);
}
__device__ __noinline__ void apply_q1_f(float* Xr, float* Xi, int ldp, int n, int r, int k,
                                        const int* perm, const double* sig, const float2* Vst,
                                        const float* beta, float2* Y, int ldy) {
  apply_q1<float>(Xr, Xi, ldp, n, r, k, perm, sig, Vst, beta, Y, ldy);
}

// V_k^+ of a task with rows longer than 128 columns, by one CTA: the rows in place, then
// (every reflector read) copied into V_k^+'s region Y.
__device__ __noinline__ void wide_q1(float* Xr, float* Xi, int ldp, int n, int r, int k,
                                     const int* perm, const double* sig, float2* Y,
                                     const float* beta, int ldy) {
  __syncthreads();
  if (n > 256)
    apply_q1_wide<16>(Xr, Xi, ldp, n, r, k, perm, sig, Y, beta, 0, 1);
  else
    apply_q1_wide<8>(Xr, Xi, ldp, n, r, k, perm, sig, Y, beta, 0, 1);
  __syncthreads();
  for (int idx = threadIdx.x; idx < k * n; idx += blockDim.x) {
    const int j = idx / n, c = idx - j * n;
    const long long o = (long long)perm[j] * ldp + c;
    Y[j * ldy + c] = make_float2(Xr[o], Xi[o]);
  }
}

// Whether a cluster also shares the preconditioning and V_k^+ of a task whose Jacobi it
// shares: theta no taller than wide (m <= n), so that L1 is square, and wider than 128.
__device__ __forceinline__ bool cluster_shares_precondition(int m, int n) {
  return m <= n && m > LT_REG_DIM;
}

// V_k^+ shared by a cluster: rank 0 publishes k, the ranked rows and the squared singular
// values (cluster_q1_lead), every CTA transforms its share of the k rows in place
// (reflectors and betas from the cluster's LQ), and rank 0 copies them into V_k^+'s
// region once all are done.  Two cluster barriers, taken by every CTA.
__device__ void cluster_q1_rows(float* Xr, float* Xi, int ldp, int n, int r, const float2* Vst,
                                const float* cls, int crank, int C) {
  __threadfence();
  cluster_sync();  // k, ranks and singular values published
  const int k = __ldcg(reinterpret_cast<const int*>(cls + LT_CL_K));
  const int* perm = reinterpret_cast<const int*>(cls + LT_CL_PERM);
  const double* sig = reinterpret_cast<const double*>(cls + LT_CL_SIG);
  if (n > 256)
    apply_q1_wide<16, true>(Xr, Xi, ldp, n, r, k, perm, sig, Vst, cls + LT_CL_B1, crank, C);
  else
    apply_q1_wide<8, true>(Xr, Xi, ldp, n, r, k, perm, sig, Vst, cls + LT_CL_B1, crank, C);
  __threadfence();
  cluster_sync();  // every row transformed
}

__device__ __noinline__ void cluster_q1(float* Xr, float* Xi, int ldp, int n, int r,
                                        const float2* Vst, float* cls, int crank, int C) {
  cluster_q1_rows(Xr, Xi, ldp, n, r, Vst, cls, crank, C);
}

__device__ __noinline__ void cluster_q1_lead(float* Xr, float* Xi, int ldp, int n, int r, int k,
                                             const int* perm, const double* sig, float2* Y,
                                             int ldy, float* cls, int C) {
  int* gperm = reinterpret_cast<int*>(cls + LT_CL_PERM);
  double* gsig = reinterpret_cast<double*>(cls + LT_CL_SIG);
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    gperm[i] = perm[i];
    gsig[i] = sig[i];
  }
  if (threadIdx.x == 0) *reinterpret_cast<int*>(cls + LT_CL_K) = k;
  __syncthreads();
  cluster_q1_rows(Xr, Xi, ldp, n, r, Y, cls, 0, C);
  for (int idx = threadIdx.x; idx < k * n; idx += blockDim.x) {
    const int j = idx / n, c = idx - j * n;
    const long long o = (long long)perm[j] * ldp + c;
    Y[j * ldy + c] = make_float2(__ldcg(Xr + o), __ldcg(Xi + o));
  }
}

template <int G>
__device__ void apply_q1_reg(const float* Xr, const float* Xi, int ldp, int n, int r, int k,
                             const int* perm, const double* sig, const float2* Vst,
                             const float* beta, float2* Y, int ldy) {
  constexpr int NH = 64 / G, HPB = 8 / G > 0 ? 8 / G : 1, CPB = 2 * G * HPB;
  __syncthreads();
  const int q = threadIdx.x % G, j = threadIdx.x / G;
  const bool act = j < k;
  float2 xr[NH], xi[NH];
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    xr[h] = make_float2(0.f, 0.f);
    xi[h] = xr[h];
  }
  if ((threadIdx.x >> 5) * (32 / G) < k) {  // warp-uniform: the warp holds a live row
    const int p = act ? perm[j] : 0;
    const float inv = act && sig[p] > 0.0 ? (float)(1.0 / sqrt(sig[p])) : 0.f;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const int c0 = 2 * G * h + q, c1 = c0 + G;
      if (act && c0 < r) {
        xr[h].x = Xr[p * ldp + c0] * inv;
        xi[h].x = Xi[p * ldp + c0] * inv;
      }
      if (act && c1 < r) {
        xr[h].y = Xr[p * ldp + c1] * inv;
        xi[h].y = Xi[p * ldp + c1] * inv;
      }
    }
    int off = r * n - r * (r - 1) / 2;
    for (int l = r - 1; l >= 0; --l) {
      off -= n - l;
      const float bt = beta[l];
      if (bt == 0.f) continue;  // uniform across the block
      const float2* e = Vst + off - l;  // e[c], l <= c < n
      float dr0 = 0.f, di0 = 0.f, dr1 = 0.f, di1 = 0.f;
#pragma unroll
      for (int sb = 0; sb < NH / HPB; ++sb) {
        if (CPB * sb + CPB > l && CPB * sb < n) {
#pragma unroll
          for (int u = 0; u < HPB; ++u) {
            const int h = HPB * sb + u, c0 = 2 * G * h + q, c1 = c0 + G;
            const float2 e0 = (c0 >= l && c0 < n) ? e[c0] : make_float2(0.f, 0.f);
            const float2 e1 = (c1 >= l && c1 < n) ? e[c1] : make_float2(0.f, 0.f);
            dr0 = fmaf(xr[h].x, e0.x, fmaf(xi[h].x, e0.y, dr0));
            di0 = fmaf(xi[h].x, e0.x, fmaf(-xr[h].x, e0.y, di0));
            dr1 = fmaf(xr[h].y, e1.x, fmaf(xi[h].y, e1.y, dr1));
            di1 = fmaf(xi[h].y, e1.x, fmaf(-xr[h].y, e1.y, di1));
          }
        }
      }
      float dr = dr0 + dr1, di = di0 + di1;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        dr += __shfl_xor_sync(FULL, dr, o);
        di += __shfl_xor_sync(FULL, di, o);
      }
      dr *= bt;
      di *= bt;
#pragma unroll
      for (int sb = 0; sb < NH / HPB; ++sb) {
        if (CPB * sb + CPB > l && CPB * sb < n) {
#pragma unroll
          for (int u = 0; u < HPB; ++u) {
            const int h = HPB * sb + u, c0 = 2 * G * h + q, c1 = c0 + G;
            const float2 e0 = (c0 >= l && c0 < n) ? e[c0] : make_float2(0.f, 0.f);
            const float2 e1 = (c1 >= l && c1 < n) ? e[c1] : make_float2(0.f, 0.f);
            xr[h].x -= fmaf(dr, e0.x, -di * e0.y);
            xi[h].x -= fmaf(dr, e0.y, di * e0.x);
            xr[h].y -= fmaf(dr, e1.x, -di * e1.y);
            xi[h].y -= fmaf(dr, e1.y, di * e1.x);
          }
        }
      }
    }
  }
  __syncthreads();  // every reflector read before Y overwrites their store
  if (act) {
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const int c0 = 2 * G * h + q, c1 = c0 + G;
      if (c0 < n) Y[j * ldy + c0] = make_float2(xr[h].x, xi[h].x);
      if (c1 < n) Y[j * ldy + c1] = make_float2(xr[h].y, xi[h].y);
    }
  }
}



// ---- re-orthonormalisation of V_k^+ (single precision) -----------------------------------
// The one-sided Jacobi stops once every row pair is orthogonal to eps sqrt(r) |x| |y|,
// so the rows v_j^+ it yields are orthonormal only to about that threshold (1e-6 at
// r = 128), well above the rounding of the stored tensors; the split B_b = theta~ V_k,
// B_{b+1} = V_k^+ then carries that defect into the state.  One step of the polar
// (Lowdin) iteration removes it without changing the span of the kept rows: each row is
// scaled to unit length by its norm accumulated in double, E = V^+ V - I is formed (zero
// diagonal; the off-diagonal entries are of the order of the threshold, so their
// single-precision rounding lies orders of magnitude below it) and V^+ <- (I - E/2) V^+,
// which is orthonormal to O(|E|^2) plus the final rounding.  E is written to the
// scratch array Es (k x k complex); the product runs in column chunks held in registers.
template <int NT>
__device__ void reorthonormalise_rows(float2* Y, int ld, int k, int n, float2* Es) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < k; j += NW) {
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) {
      const float2 v = Y[j * ld + c];
      acc = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, acc));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    const float sc = acc > 0.0 ? (float)(1.0 / sqrt(acc)) : 0.f;
    for (int c = lane; c < n; c += 32) {
      float2 v = Y[j * ld + c];
      v.x *= sc;
      v.y *= sc;
      Y[j * ld + c] = v;
    }
  }
  __syncthreads();
  // E[i][j] = sum_c y_i conj(y_j) (i != j, E[j][i] its conjugate, zero diagonal): 2 x 2
  // tiles of the upper triangle, four complex products per four loads
  const int kb = (k + 1) >> 1, ntile = kb * (kb + 1) / 2;
  for (int t = tid; t < ntile; t += NT) {
    int I = 0, rem = t;
    while (rem >= kb - I) {  // row I of the triangle holds kb - I tiles
      rem -= kb - I;
      ++I;
    }
    const int J = I + rem;
    const int i0 = 2 * I, i1 = i0 + 1, j0 = 2 * J, j1 = j0 + 1;
    const bool vi1 = i1 < k, vj1 = j1 < k;
    const float2* y0 = Y + i0 * ld;
    const float2* y1 = Y + (vi1 ? i1 : i0) * ld;
    const float2* z0 = Y + j0 * ld;
    const float2* z1 = Y + (vj1 ? j1 : j0) * ld;
    float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
    for (int c = 0; c < n; ++c) {
      const float2 u0 = y0[c], u1 = y1[c], v0 = z0[c], v1 = z1[c];
      cfmac(a00, u0, v0);
      cfmac(a01, u0, v1);
      cfmac(a10, u1, v0);
      cfmac(a11, u1, v1);
    }
    const float2 zero = make_float2(0.f, 0.f);
    auto put = [&](int i, int j, float2 v) {
      Es[i * k + j] = i == j ? zero : v;
      if (i != j) Es[j * k + i] = make_float2(v.x, -v.y);
    };
    put(i0, j0, a00);
    if (vj1) put(i0, j1, a01);
    if (vi1 && I != J) put(i1, j0, a10);
    if (vi1 && vj1) put(i1, j1, a11);
  }
  __syncthreads();
  // Y <- Y - E Y / 2: an item is four rows of one column; each load of Y[j][c] feeds the
  // four rows, E is read as a broadcast within the warp
  constexpr int RG = 4, ITEMS = 4;
  const int kg = (k + RG - 1) / RG;
  const int cw = (NT * ITEMS) / kg < n ? ((NT * ITEMS) / kg > 0 ? (NT * ITEMS) / kg : 1) : n;
  for (int c0 = 0; c0 < n; c0 += cw) {
    const int w = n - c0 < cw ? n - c0 : cw;
    float2 acc[ITEMS][RG];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
#pragma unroll
      for (int r = 0; r < RG; ++r) acc[it][r] = make_float2(0.f, 0.f);
      const int item = tid + NT * it;
      if (item < kg * w) {
        const int g = item / w, c = c0 + item - g * w;
        const float2* e0 = Es + (RG * g) * k;
        for (int j = 0; j < k; ++j) {
          const float2 y = Y[j * ld + c];
#pragma unroll
          for (int r = 0; r < RG; ++r)
            if (RG * g + r < k) cfma(acc[it][r], e0[r * k + j], y);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int item = tid + NT * it;
      if (item < kg * w) {
        const int g = item / w, c = c0 + item - g * w;
#pragma unroll
        for (int r = 0; r < RG; ++r) {
          const int i = RG * g + r;
          if (i < k) {
            float2 v = Y[i * ld + c];
            v.x = fmaf(-0.5f, acc[it][r].x, v.x);
            v.y = fmaf(-0.5f, acc[it][r].y, v.y);
            Y[i * ld + c] = v;
          }
        }
      }
    }
    __syncthreads();
  }
}


// ---- theta on the tensor cores: exact products of 8-bit digits (single precision) --------
// P = Bl Br (rows (a, s) of Bl, columns (t, c) of Br, inner index mu) is formed on the
// 5th-generation tensor cores (tcgen05.mma, kind::f16 with bf16 operands, FP32
// accumulators in tensor memory) without rounding: every single-precision value x of a
// row of Bl (of a column of Br) is written as 2^e (d0 2^-7 + d1 2^-15 + d2 2^-23 + d3
// 2^-31) + r, |r| <= 2^(e-32), with 2^e above the row's (column's) largest |Re|, |Im|
// and signed integer digits |d| <= 128, which bf16 holds exactly.  A product of two
// digits is an integer below 2^14, so the sum over mu <= 64 and over the (at most four)
// digit pairs (i, j) of one order q = i + j, for Re = ArBr - AiBi and Im = ArBi + AiBr,
// stays an integer below 2^23: each FP32 accumulator S_q is exact whatever order or
// rounding mode the tensor core adds in.  The orders q = 0..3 are kept (the dropped
// ones lie 2^-32 below the row-column scale), and P = 2^(e_r + f_c) sum_q S_q 2^(-14-8q)
// is recombined as a pair of floats (two-sum of the two leading orders, the rest in the
// low part).  The gate is then applied to that pair (its single-precision value and
// residual, as in form_theta), so theta~ comes out rounded once.  Plain TF32 products
// are not used here: their accumulation in the tensor core rounds toward zero, which
// biases every contraction by a few 1e-7 in the same direction.
namespace tcg {

constexpr int TMEM_COLS = 512;   // 8 accumulators (S_0..S_3 of Re and Im) x 64 columns
constexpr int TILE_N = 64;       // columns (t, c) per pass

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x
// 16 bytes, `lbo` bytes between core matrices along K, `sbo` between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;
}
// D[tmem] (+)= A B for M = 128, N = 64, K = 16, bf16 operands, FP32 accumulate
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_addr(bar)));
}
// wait for the phase `parity` of the barrier, at most 2^24 polls
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity));
  return done != 0;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// 8 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
// byte offset of (row, k) in a digit plane of `rows` rows (K-major, no swizzle)
__device__ __forceinline__ int koff(int row, int k, int rows) {
  return (k >> 3) * (rows * 16) + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// the four digits of x 2^-e (|x| < 2^e)
__device__ __forceinline__ void digits(float x, int e, float* d) {
  float v = ldexpf(x, 7 - e);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    d[t] = rintf(v);
    v = (v - d[t]) * 256.f;
  }
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ int expo(float m) { return m > 0.f ? ilogbf(m) + 1 : -100; }
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// Bytes of shared memory the digit planes of one pass take for inner dimension <= kp
__host__ __device__ constexpr int smem_bytes(int kp) { return 8 * 128 * kp * 2 + 8 * TILE_N * kp * 2; }

}  // namespace tcg

template <typename R>
__device__ __forceinline__ void jacobi_layout(int mJ, int nJ, bool& blocked, bool& wide, int& npad,
                                              int& mp) {
  blocked = sizeof(R) == 4 && mJ >= 32 && nJ >= 64 && nJ <= LT_REG_DIM;
  wide = sizeof(R) == 4 && mJ >= 32 && nJ > LT_REG_DIM;
  const int span = 8 * jacobi_span<R, 4>(nJ);  // 4 element pairs per lane
  npad = blocked ? (nJ <= 64 ? 64 : 128)
                 : wide ? 128 * ((nJ + 127) / 128) : span * ((nJ + span - 1) / span);
  // the circle-method pairing needs an even count, the block pairing a multiple of 8
  mp = blocked || wide ? (mJ + 7) & ~7 : mJ + (mJ & 1);
}

// Workspace layout of one task (complex elements): the matrix the Jacobi sweeps act
// on is mJ rows of length nJ; after the two-level Householder preconditioning they act
// on the r x r triangular factor, whose window (mp2 x npad2) can have more rows than
// the mJ x nJ layout: a wide matrix (nJ > LT_REG_DIM, rows rounded to even) whose
// factor takes the blocked layout (rows rounded to 8).  The planes hold both, plus in
// mode 1 the D chi_{b-1} rows of theta~ formed afterwards; every row below mJ is zero
// from the formation on.  Behind them: V_k^+ rows,
// the LQ reflectors before it, and the staging of B_{b+1} (mode 0) or of the new site
// tensors (mode 2).
struct TaskLayout {
  int mJ, nJ, rr, npad, mpJ, npad2, mp2, mpad, mcap, ldp, ld, kmax;
  bool blocked, wide, blk2, wide2;
  long long need;
};

template <typename R, int D>
__device__ __forceinline__ TaskLayout task_layout(int mode, int chiL, int chiM, int chiR,
                                                  int chi) {
  TaskLayout t;
  t.mJ = mode == 1 ? chiM : D * chiL;
  t.nJ = mode == 2 ? chiM : D * chiR;
  jacobi_layout<R>(t.mJ, t.nJ, t.blocked, t.wide, t.npad, t.mpJ);
  t.rr = t.mJ < t.nJ ? t.mJ : t.nJ;
  jacobi_layout<R>(t.rr, t.rr, t.blk2, t.wide2, t.npad2, t.mp2);
  t.mpad = t.mpJ > t.mp2 ? t.mpJ : t.mp2;
  t.mcap = mode == 1 ? (t.mpad > D * chiL ? t.mpad : D * chiL) : t.mpad;
  t.ldp = t.npad + 2;
  t.ld = t.nJ + 1;
  t.kmax = t.rr < chi ? t.rr : chi;
  const long long vrows = (long long)t.kmax * t.ld;         // V_k^+
  const long long stage0 = (long long)chiM * D * chiR;      // B_{b+1} staged in V_k^+'s place
  const long long stage2 = (long long)t.kmax * (chiL > chiR ? D * chiL : D * chiR);
  // the r LQ reflectors (n - j entries each) occupy the same region until V_k^+
  // is assembled; with D = 2 they never exceed the V_k^+ rows, with D = 4 they do
  const long long r0 = t.rr;
  const long long refl = r0 * t.nJ - r0 * (r0 - 1) / 2;
  long long tail = mode == 0 ? (vrows > stage0 ? vrows : stage0)
                             : vrows + (mode == 2 ? stage2 : 0);
  if (refl > tail) tail = refl;
  t.need = (long long)t.mcap * t.ldp + tail;
  return t;
}

// Whether a mode-0 task of this shape takes the tensor-core theta: 2 chi_L and 2 chi_R
// at most 128, chi_M at most 64, its digit planes within the workspace, and (with two
// column passes) the first pass's theta~ within the slot of site b.
__device__ __forceinline__ bool theta_tc_fits(int chiL, int chiM, int chiR, long long slot,
                                              long long ws_bytes) {
  const int kp = (chiM + 15) & ~15;
  if (2 * chiL > 128 || 2 * chiR > 128 || chiM > 64) return false;
  if ((long long)tcg::smem_bytes(kp) > ws_bytes) return false;
  return 2 * chiR <= tcg::TILE_N || (long long)(2 * chiL) * tcg::TILE_N <= slot;
}

// theta~ = G (Bl Br) on the tensor cores, written over the site tensors of sites b and
// b+1 (Bl, and the slot after it): pass T (columns n' = 2c + t in [64 T, 64 T + 64)) is
// stored row-major with its own width at Bl + T slot, or, in one pass, across both
// slots.  W: shared workspace (digit planes); s_er, s_fc: [128] exponents; tmem, bar,
// phase: the CTA's tensor memory and barrier.  Returns false if a wait ran out.
__device__ bool theta_tc(unsigned char* W, float2* Bl, const float2* Br, int chiL, int chiM,
                         int chiR, long long slot, const float2* G, const float2* Glo,
                         int* s_er, int* s_fc, uint32_t tmem, uint64_t* bar, uint32_t& phase) {
  using namespace tcg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int m = 2 * chiL, n = 2 * chiR, kp = (chiM + 15) & ~15;
  const int aplane = 128 * kp * 2, bplane = TILE_N * kp * 2;
  unsigned char* A = W;
  unsigned char* B = W + 8 * aplane;
  // row exponents of Bl (rows (a, s)), column exponents of Br (columns n' = 2c + t)
  for (int r = warp; r < 128; r += nw) {
    float mx = 0.f;
    if (r < m)
      for (int k = lane; k < chiM; k += 32) {
        const float2 v = Bl[(long long)r * chiM + k];
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    if (lane == 0) s_er[r] = expo(mx);
  }
  for (int c2 = tid; c2 < n; c2 += blockDim.x) {
    const int c = c2 >> 1, t = c2 & 1;
    float mx = 0.f;
    for (int k = 0; k < chiM; ++k) {
      const float2 v = Br[(long long)k * n + t * chiR + c];
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    s_fc[c2] = expo(mx);
  }
  __syncthreads();
  // A digit planes (Re digits 0..3, Im digits 0..3), 128 rows x kp, two k per thread step
  for (int i = tid; i < 128 * (kp >> 1); i += blockDim.x) {
    const int r = i / (kp >> 1), k = 2 * (i - r * (kp >> 1));
    float2 v0 = make_float2(0.f, 0.f), v1 = v0;
    if (r < m) {
      if (k < chiM) v0 = Bl[(long long)r * chiM + k];
      if (k + 1 < chiM) v1 = Bl[(long long)r * chiM + k + 1];
    }
    float d0r[4], d1r[4], d0i[4], d1i[4];
    const int e = s_er[r];
    digits(v0.x, e, d0r);
    digits(v1.x, e, d1r);
    digits(v0.y, e, d0i);
    digits(v1.y, e, d1i);
    const int o = koff(r, k, 128);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      *reinterpret_cast<uint32_t*>(A + t * aplane + o) = pack2(d0r[t], d1r[t]);
      *reinterpret_cast<uint32_t*>(A + (4 + t) * aplane + o) = pack2(d0i[t], d1i[t]);
    }
  }
  const int passes = (n + TILE_N - 1) / TILE_N;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TILE_N >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  const uint32_t idesc_neg = idesc | (1u << 13);
  bool ok = true;
  for (int T = 0; T < passes && ok; ++T) {
    const int n0 = T * TILE_N, nt = n - n0 < TILE_N ? n - n0 : TILE_N;
    // B digit planes of this pass: row n' - n0 (column (t, c) of Br), inner index k
    for (int i = tid; i < TILE_N * (kp >> 1); i += blockDim.x) {
      const int nl = i % TILE_N, k = 2 * (i / TILE_N);
      const int c2 = n0 + nl, c = c2 >> 1, t = c2 & 1;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      int e = -100;
      if (nl < nt) {
        e = s_fc[c2];
        if (k < chiM) v0 = Br[(long long)k * n + t * chiR + c];
        if (k + 1 < chiM) v1 = Br[(long long)(k + 1) * n + t * chiR + c];
      }
      float d0r[4], d1r[4], d0i[4], d1i[4];
      digits(v0.x, e, d0r);
      digits(v1.x, e, d1r);
      digits(v0.y, e, d0i);
      digits(v1.y, e, d1i);
      const int o = koff(nl, k, TILE_N);
#pragma unroll
      for (int t4 = 0; t4 < 4; ++t4) {
        *reinterpret_cast<uint32_t*>(B + t4 * bplane + o) = pack2(d0r[t4], d1r[t4]);
        *reinterpret_cast<uint32_t*>(B + (4 + t4) * bplane + o) = pack2(d0i[t4], d1i[t4]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
      for (int ks = 0; ks < kp / 16; ++ks)
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j + i < 4; ++j) {
            const int q = i + j;
            const uint32_t acc = (ks > 0 || i > 0) ? 1u : 0u;  // (0, q) opens S_q
            const uint32_t dre = tmem + q * TILE_N, dim = tmem + (4 + q) * TILE_N;
            const uint64_t ar = sdesc(a0 + i * aplane + ks * 2 * 128 * 16, 128 * 16, 128);
            const uint64_t ai = sdesc(a0 + (4 + i) * aplane + ks * 2 * 128 * 16, 128 * 16, 128);
            const uint64_t br = sdesc(b0 + j * bplane + ks * 2 * TILE_N * 16, TILE_N * 16, 128);
            const uint64_t bi = sdesc(b0 + (4 + j) * bplane + ks * 2 * TILE_N * 16, TILE_N * 16, 128);
            mma(dre, ar, br, idesc, acc);
            mma(dre, ai, bi, idesc_neg, 1u);
            mma(dim, ar, bi, idesc, acc);
            mma(dim, ai, br, idesc, 1u);
          }
      commit(bar);
    }
    // block-uniform outcome: every thread takes the same path through the epilogue
    ok = __syncthreads_and(wait(bar, phase) ? 1 : 0) != 0;
    phase ^= 1u;
    fence_after();
    if (ok) {
      // epilogue: warp (quadrant, column group); lane = row (a, s) of the accumulators
      const int row = 32 * (warp & 3) + lane, cg = warp >> 2;
      const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
      const int width = passes == 1 ? n : nt;
      float2* out = Bl + (passes == 1 ? 0 : (long long)T * slot);
      for (int h = 0; h < (TILE_N / 8) / (nw / 4); ++h) {
        const int col0 = 8 * (cg + (nw / 4) * h);  // 8 columns n' - n0 = 4 values of c
        float S[8][8];
#pragma unroll
        for (int acc = 0; acc < 8; ++acc) ld8(tl + acc * TILE_N + col0, S[acc]);
        // P = 2^(e_r + f_c) sum_q S_q 2^(-14 - 8q) as hi + lo, Re and Im
        float ph[8][2], pl[8][2];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c2 = n0 + col0 + j;
          const int e = s_er[row] + (c2 < n ? s_fc[c2] : 0);
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            const float* q = &S[4 * part][0];
            float hi, lo;
            two_sum(ldexpf(q[0 * 8 + j], -14), ldexpf(q[1 * 8 + j], -22), hi, lo);
            lo += ldexpf(q[2 * 8 + j], -30) + ldexpf(q[3 * 8 + j], -38);
            ph[j][part] = ldexpf(hi, e);
            pl[j][part] = ldexpf(lo, e);
          }
        }
        // gate on (s, t): the partner row (a, 1 - s) is the neighbouring lane
        const int s = row & 1;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          float2 Ph[4], Pl[4];  // index u = 2 s2 + t2
#pragma unroll
          for (int t2 = 0; t2 < 2; ++t2) {
            const int j = 2 * cc + t2;
            const float oh0 = __shfl_xor_sync(FULL, ph[j][0], 1), oh1 = __shfl_xor_sync(FULL, ph[j][1], 1);
            const float ol0 = __shfl_xor_sync(FULL, pl[j][0], 1), ol1 = __shfl_xor_sync(FULL, pl[j][1], 1);
            Ph[2 * s + t2] = make_float2(ph[j][0], ph[j][1]);
            Pl[2 * s + t2] = make_float2(pl[j][0], pl[j][1]);
            Ph[2 * (1 - s) + t2] = make_float2(oh0, oh1);
            Pl[2 * (1 - s) + t2] = make_float2(ol0, ol1);
          }
          const int c = (n0 + col0) / 2 + cc;
          if (row < m && c < chiR) {
#pragma unroll
            for (int tp = 0; tp < 2; ++tp) {
              const float2* g = G + (s * 2 + tp) * 4;
              const float2* gl = Glo + (s * 2 + tp) * 4;
              float2 hi = make_float2(0.f, 0.f), lo = hi;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                cfma(hi, g[u], Ph[u]);
                cfma(lo, g[u], Pl[u]);
                cfma(lo, gl[u], Ph[u]);
              }
              out[(long long)row * width + (2 * c + tp - n0)] = make_float2(hi.x + lo.x, hi.y + lo.y);
            }
          }
        }
      }
    }
    fence_before();
    __syncthreads();
    fence_after();
  }
  return ok;
}

// theta~ (in the layout theta_tc wrote) into the planes, times w_a when weighted; zero
// padding to mp rows and npad columns as form_theta leaves it
__device__ void theta_tc_planes(float* Xr, float* Xi, int ldp, int npad, int mp, const float2* Bl,
                                int chiL, int chiR, long long slot, const double* lamL,
                                bool weighted) {
  const int m = 2 * chiL, n = 2 * chiR;
  const int passes = (n + tcg::TILE_N - 1) / tcg::TILE_N;
  for (int i = threadIdx.x; i < mp * npad; i += blockDim.x) {
    const int r = i / npad, col = i - r * npad;
    float2 v = make_float2(0.f, 0.f);
    if (r < m && col < n) {
      const int tp = col / chiR, c = col - tp * chiR, c2 = 2 * c + tp;
      const int T = passes == 1 ? 0 : c2 / tcg::TILE_N;
      const int width = passes == 1 ? n : (n - T * tcg::TILE_N < tcg::TILE_N ? n - T * tcg::TILE_N
                                                                               : tcg::TILE_N);
      v = Bl[(long long)T * slot + (long long)r * width + (c2 - T * tcg::TILE_N)];
      if (weighted) {
        const float w = (float)lamL[r >> 1];
        v.x *= w;
        v.y *= w;
      }
    }
    Xr[r * ldp + col] = v.x;
    Xi[r * ldp + col] = v.y;
  }
}


// Tensor-core pass of a Trotter layer (single precision, two values per site): for every
// (trajectory, bond) task of the layer whose shape fits (theta_tc_fits, the same test
// the bond kernel makes), theta~ = G (B_b B_{b+1}) replaces the two site tensors in the
// layout theta_tc describes; the bond kernel then reads it instead of forming theta.
// One CTA per SM (the digit planes take up to 192 KB of shared memory), each holding 512
// columns of tensor memory and one barrier for the whole launch.
__global__ void __launch_bounds__(512, 1) theta_tc_kernel(BondArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_er[128], s_fc[128];
  __shared__ float2 s_gate[16], s_glo[16];
  const int tid = threadIdx.x, L = a.L;
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tcg::smem_addr(&s_tmem)),
                 "r"(tcg::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tcg::smem_addr(&s_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  uint32_t phase = 0;
  bool ok = true;
  const long long ntask = (long long)(*a.n_trajs) * a.nb;
  const long long ws_bytes = a.smem_elems * (long long)sizeof(float2);
  for (long long task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
    const int traj = a.trajs[task / a.nb];
    const int b = a.bond0 + 2 * (int)(task % a.nb);
    const int* dm = a.dims + (long long)traj * (L - 1);
    const int chiL = b == 0 ? 1 : dm[b - 1];
    const int chiM = dm[b];
    const int chiR = b == L - 2 ? 1 : dm[b + 1];
    // the bond kernel takes theta~ from this pass exactly for these tasks
    if (task_layout<float, 2>(0, chiL, chiM, chiR, a.chi).need > a.smem_elems ||
        !theta_tc_fits(chiL, chiM, chiR, a.slot, ws_bytes))
      continue;
    if (tid < 16) {
      const double2 g = a.gates[b * 16 + tid];
      const float2 h = make_float2((float)g.x, (float)g.y);
      s_gate[tid] = h;
      s_glo[tid] = make_float2((float)(g.x - (double)h.x), (float)(g.y - (double)h.y));
    }
    __syncthreads();
    float2* Bl = a.B + ((long long)traj * L + b) * a.slot;
    ok = theta_tc(smem_raw, Bl, Bl + a.slot, chiL, chiM, chiR, a.slot, s_gate, s_glo, s_er, s_fc,
                  s_tmem, &s_bar, phase);
    if (!ok && tid == 0) atomicOr(a.err, LT_EBIT_TIMEOUT);
  }
  // after a wait that ran out, give the outstanding products one more bounded wait
  // before the tensor memory is released
  if (!ok) tcg::wait(&s_bar, phase ^ 1u);
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                 "r"(tcg::TMEM_COLS));
}

// ---- the two-site update and the one-site canonical-form steps -----------------------------
// mode 0: two-site update with the layer's gate (Eq. Theta): theta = Lambda_{b-1}
//         G (B_b B_{b+1}), SVD, keep k, Lambda_b = S_k/|S_k|, B_{b+1} = V_k^+,
//         B_b = theta~ V_k / |S_k|.
// mode 1: shift the orthogonality centre left across bond b (Eq. ShiftCenter by
//         a one-site SVD): B_{b+1} = U S V^+ (chi_b x 2chi_{b+1}), B_{b+1} = V_k^+,
//         B_b = B_b B_{b+1} V_k (= B_b U_k S_k), no renormalisation.
// mode 2: restore bond b: Lambda_{b-1} B_b = U S V^+ (2chi_{b-1} x chi_b),
//         B_b = B_b V_k / |S_k|, B_{b+1} = V_k^+ B_{b+1}, Lambda_b = the column
//         norms of Lambda_{b-1} B_b (= S_k/|S_k| in exact arithmetic).
// Workspace (shared memory, or per-CTA global scratch when it does not fit):
// the Jacobi matrix planar (2 mcap ldp reals; in mode 0/1 later theta~), then
// V_k^+ rows (k x (nJ+1) complex); in mode 0 the region after theta first
// stages B_{b+1}, in mode 2 the region after V_k^+ stages the new site tensors.
// sum_{j<r} (a - j)(b - j), or sum_{j<r} (a - j) when `linear`
__device__ __forceinline__ long long sum_prod(int a, int b, int r, bool linear = false) {
  const long long R = r, A = a, B = b;
  const long long s1 = R * (R - 1) / 2, s2 = (R - 1) * R * (2 * R - 1) / 6;
  if (linear) return R * A - s1;
  return R * A * B - (A + B) * s1 + s2;
}

// B_b = theta~ V_k (times invn) by a cluster, as the one-CTA split computes it: an item is
// four rows of B_b and two of its columns; the items are dealt over the cluster's threads
// (this CTA taking share `part` of `parts`), and every operand is read past L1.
__device__ void split_rows_cluster(const float* Xr, const float* Xi, int ldp, int m, int nJ,
                                   const float2* Y, int ld, int k, float invn, float2* Bl,
                                   int part, int parts) {
  const int rq = (m + 3) >> 2, kq = (k + 1) >> 1;
  for (int idx = part * blockDim.x + threadIdx.x; idx < rq * kq; idx += parts * blockDim.x) {
    const int g = idx / kq, r0 = g << 2, j0 = 2 * (idx - g * kq);
    const bool two = j0 + 1 < k;
    const float2* y0 = Y + j0 * ld;
    const float2* y1 = Y + (two ? j0 + 1 : j0) * ld;
    float2 acc[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = make_float2(0.f, 0.f);
    const int nr = m - r0 < 4 ? m - r0 : 4;
    for (int c = 0; c < nJ; ++c) {
      const float2 v0 = __ldcg(y0 + c), v1 = __ldcg(y1 + c);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < nr) {
          const long long o = (long long)(r0 + u) * ldp + c;
          const float2 x = make_float2(__ldcg(Xr + o), __ldcg(Xi + o));
          cfmac(acc[u][0], x, v0);
          cfmac(acc[u][1], x, v1);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (u < nr) {
        Bl[(r0 + u) * k + j0] = cscale(acc[u][0], invn);
        if (two) Bl[(r0 + u) * k + j0 + 1] = cscale(acc[u][1], invn);
      }
  }
}

// The split's part of a helper CTA: rank 0 has re-formed theta~, finished V_k^+ and
// published 1/|S_k|; every CTA computes its items of B_b; two cluster barriers.
__device__ __noinline__ void cluster_split(const float* Xr, const float* Xi, int ldp, int m,
                                           int nJ, const float2* Y, int ld, float2* Bl,
                                           const float* cls, int crank, int C) {
  __threadfence();
  cluster_sync();  // theta~, V_k^+ and 1/|S_k| published
  const int k = __ldcg(reinterpret_cast<const int*>(cls + LT_CL_K));
  const float invn = __ldcg(cls + LT_CL_K + 1);
  split_rows_cluster(Xr, Xi, ldp, m, nJ, Y, ld, k, invn, Bl, crank, C);
  __threadfence();
  cluster_sync();  // every item of B_b written
}

// The CTAs of rank > 0 of a cluster: they walk the tasks of their cluster like rank 0
// and join exactly the Jacobis that rank 0 shares (tasks in global scratch with rows
// of more than 128 columns); everything else of a task is rank 0's.
template <int D>
__device__ __noinline__ void cluster_helper(const BondArgs<float>& a, float* s_nrm, float* s_part,
                                           int* s_nrot) {
  const int C = a.cluster, crank = cluster_rank(), L = a.L;
  const long long cid = cluster_index(), ncid = cluster_count();
  const long long ntask = (long long)(*a.n_trajs) * a.nb;
  for (long long task = cid; task < ntask; task += ncid) {
    const int traj = a.trajs[task / a.nb];
    const int b = a.bond0 + 2 * (int)(task % a.nb);
    const int* dm = a.dims + (long long)traj * (L - 1);
    const int chiL = b == 0 ? 1 : dm[b - 1];
    const int chiM = dm[b];
    const int chiR = b == L - 2 ? 1 : dm[b + 1];
    const TaskLayout lay = task_layout<float, D>(a.mode, chiL, chiM, chiR, a.chi);
    const bool in_smem = lay.need <= a.smem_elems;
    if ((!in_smem && (a.scratch == nullptr || lay.need > a.ws_elems)) || lay.npad2 > lay.npad)
      continue;
    if (in_smem || !lay.wide2) continue;
    float* W = reinterpret_cast<float*>(a.scratch + cid * C * a.scratch_stride);
    float* Xr = W;
    float* Xi = W + (long long)lay.mcap * lay.ldp;
    float2* Y = reinterpret_cast<float2*>(W + 2ll * lay.mcap * lay.ldp);
    float* cls = a.cl_state + cid * LT_CL_STATE;
    const bool cl_pre = cluster_shares_precondition(lay.mJ, lay.nJ);
    if (cl_pre) precondition_cluster(Xr, Xi, lay.ldp, lay.mJ, lay.nJ, Y, cls, crank, C);
    wide_jacobi(Xr, Xi, lay.ldp, lay.mp2, lay.rr, lay.npad2, s_nrm, s_part, s_nrot, a.max_sweeps,
                a.tol, C, crank, cls);
    if (cl_pre) {
      cluster_q1(Xr, Xi, lay.ldp, lay.nJ, lay.rr, Y, cls, crank, C);
      float2* Bl = a.B + ((long long)traj * L + b) * a.slot;
      cluster_split(Xr, Xi, lay.ldp, D * chiL, lay.nJ, Y, lay.ld, Bl, cls, crank, C);
    }
  }
}

// D physical values per site: 2 for pure states (trajectories, QSD), 4 for the
// vectorised density matrix (Eq. MPDO; only mode 0 is launched with D = 4).  CL: the
// instance launched in thread-block clusters (single precision, a.cluster CTAs each).
template <typename R, int D, bool CL>
__global__ void __launch_bounds__(BondShape<R>::NT, 1) bond_update_kernel(BondArgs<R> a) {
  typedef typename CT<R>::T Tc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_sig[LT_MAX_DIM];
  __shared__ R s_nrm[LT_MAX_DIM];
  __shared__ int s_perm[LT_MAX_DIM];
  __shared__ Tc s_gate[D * D * D * D];
  __shared__ Tc s_glo[D * D * D * D];  // gate rounding residual (single precision)
  __shared__ double s_lamL[LT_MAX_CHI];
  __shared__ int s_k, s_nrot;
  __shared__ double s_norm, s_wdisc;
  __shared__ R s_beta[LT_MAX_DIM + 1];
  __shared__ Tc s_u[LT_MAX_DIM];
  __shared__ float s_part[256];  // group sums of the wide Jacobi

  const int L = a.L, chi = a.chi, tid = threadIdx.x, mode = a.mode;
  const long long ntask = (long long)(*a.n_trajs) * a.nb;
  // theta~ formed beforehand on the tensor cores (theta_tc_kernel) for the mode-0 tasks
  // that fit, left over the two site slots
  constexpr bool kTc = sizeof(R) == 4 && D == 2;
  const bool use_tc = kTc && a.use_tc;
  // thread-block clusters (single precision): every CTA of a cluster walks the same
  // tasks; rank 0 works a task alone, except that the whole cluster shares the Jacobi
  // of a task in global scratch
  constexpr bool kCl = CL && sizeof(R) == 4;
  const int C = kCl ? a.cluster : 1;
  if constexpr (kCl) {
    if (cluster_rank() != 0) {
      cluster_helper<D>(a, s_nrm, s_part, &s_nrot);
      return;
    }
  }
  const long long cid = kCl ? cluster_index() : blockIdx.x;
  const long long ncid = kCl ? cluster_count() : gridDim.x;
  for (long long task = cid; task < ntask; task += ncid) {
    const int traj = a.trajs[task / a.nb];
    const int b = a.bond0 + 2 * (int)(task % a.nb);
    const int* dm = a.dims + (long long)traj * (L - 1);
    const int chiL = b == 0 ? 1 : dm[b - 1];
    const int chiM = dm[b];
    const int chiR = b == L - 2 ? 1 : dm[b + 1];
    const TaskLayout lay = task_layout<R, D>(mode, chiL, chiM, chiR, chi);
    const int mJ = lay.mJ, nJ = lay.nJ, rr = lay.rr, npad = lay.npad, npad2 = lay.npad2;
    const int mp2 = lay.mp2, mpad = lay.mpad, mcap = lay.mcap, ldp = lay.ldp, ld = lay.ld;
    const int kmax = lay.kmax;
    const bool blk2 = lay.blk2;
    // the workspace: shared memory when the task fits it, else this CTA's global scratch;
    // a task that fits neither is skipped
    const bool in_smem = lay.need <= a.smem_elems;
    if ((!in_smem && (a.scratch == nullptr || lay.need > a.ws_elems)) || npad2 > npad) {
      if (tid == 0) atomicOr(a.err, LT_EBIT_WORKSPACE);
      continue;
    }
    // the cluster shares the Jacobi of a task in global scratch (the helper CTAs make
    // the same decision from the same dimensions in cluster_helper)
    const bool shared_jac = kCl && C > 1 && !in_smem && lay.wide2;
    const long long slot_cta = kCl ? cid * C : blockIdx.x;
    R* W = in_smem ? reinterpret_cast<R*>(smem_raw)
                   : reinterpret_cast<R*>(a.scratch + slot_cta * a.scratch_stride);
    Tc* Bl = a.B + ((long long)traj * L + b) * a.slot;
    Tc* Br = Bl + a.slot;
    R* Xr = W;
    R* Xi = W + mcap * ldp;
    Tc* Y = reinterpret_cast<Tc*>(W + 2 * mcap * ldp);
    constexpr int D4 = D * D * D * D;
    for (int i = tid; i < D4; i += blockDim.x) {
      const double2 g = a.gates ? a.gates[b * D4 + i]
                                : make_double2((i % (D * D + 1)) == 0 ? 1.0 : 0.0, 0.0);
      const Tc h = cmk<Tc>(g.x, g.y);
      s_gate[i] = h;
      s_glo[i] = cmk<Tc>(g.x - (double)h.x, g.y - (double)h.y);
    }
    for (int i = tid; i < chiL; i += blockDim.x)
      s_lamL[i] = b == 0 ? 1.0 : a.lam[((long long)traj * (L - 1) + b - 1) * chi + i];
    if (tid == 0) s_nrot = 0;
    __syncthreads();
    bool tc_task = false;
    if constexpr (kTc) {
      tc_task = use_tc && mode == 0 && in_smem &&
                theta_tc_fits(chiL, chiM, chiR, a.slot, a.smem_elems * (long long)sizeof(Tc));
    }
    // register paths for the sizes they hold (every task up to chi_max = 64)
    const bool reg = sizeof(R) == 4 && mJ <= LT_REG_DIM && nJ <= LT_REG_DIM && kmax <= LT_REG_CHI;
    if (tc_task) {
      if constexpr (kTc)
        theta_tc_planes(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, npad,
                        mpad, reinterpret_cast<const float2*>(Bl), chiL, chiR, a.slot, s_lamL,
                        true);
    } else if (mode == 0) {
      form_theta<R, D>(Xr, Xi, ldp, npad, mpad, Bl, Br, Y, chiL, chiM, chiR, s_gate,
                       sizeof(R) == 4 ? s_glo : nullptr, s_lamL, true);
    } else {
      // one-site matrix, zero-padded to mpad x npad
      for (int i = tid; i < mpad * npad; i += blockDim.x) {
        const int r = i / npad, c = i - r * npad;
        Tc v = czero<Tc>();
        if (r < mJ && c < nJ) {
          if (mode == 1) v = Br[r * nJ + c];
          else v = cscale(Bl[r * nJ + c], (R)s_lamL[D == 2 ? r >> 1 : r / D]);
        }
        Xr[r * ldp + c] = v.x;
        Xi[r * ldp + c] = v.y;
      }
    }
    if constexpr (sizeof(R) == 4) {
      if (reg)
        qr_precondition_reg<BondShape<R>::NT / LT_REG_DIM>(
            reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, mJ, nJ, rr, mp2, npad2,
            reinterpret_cast<float2*>(Y), reinterpret_cast<float*>(s_beta));
      else if (shared_jac && cluster_shares_precondition(mJ, nJ))
        precondition_cluster(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, mJ,
                             nJ, reinterpret_cast<float2*>(Y), a.cl_state + cid * LT_CL_STATE, 0,
                             C);
      else
        qr_precondition_f(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, mJ, nJ,
                          rr, reinterpret_cast<float2*>(Y), reinterpret_cast<float*>(s_beta),
                          reinterpret_cast<float2*>(s_u));
    } else {
      qr_precondition<R>(Xr, Xi, ldp, mJ, nJ, rr, Y, s_beta, s_u);
    }
    int sweeps = 0;
    if (blk2) {
      if (npad2 == 64)
        sweeps = jacobi_blocked<1>(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp,
                                   mp2, rr, npad2, reinterpret_cast<float*>(s_nrm), &s_nrot,
                                   a.max_sweeps, a.tol);
      else
        sweeps = jacobi_blocked<2>(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp,
                                   mp2, rr, npad2, reinterpret_cast<float*>(s_nrm), &s_nrot,
                                   a.max_sweeps, a.tol);
    } else if (lay.wide2) {
      if constexpr (sizeof(R) == 4) {
        sweeps = wide_jacobi(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, mp2,
                             rr, npad2, reinterpret_cast<float*>(s_nrm), s_part, &s_nrot,
                             a.max_sweeps, a.tol, shared_jac ? C : 1, 0,
                             shared_jac ? a.cl_state + cid * LT_CL_STATE : nullptr);
      }
    } else {
      if (rr > 2 * 4 * 32) {
        sweeps = jacobi_rows<R, 4, true>(Xr, Xi, ldp, mp2, rr, s_nrm, &s_nrot, a.max_sweeps, a.tol);
      } else {
        sweeps = jacobi_rows<R, 4, false>(Xr, Xi, ldp, mp2, rr, s_nrm, &s_nrot, a.max_sweeps, a.tol);
      }
    }
    // singular values squared, accumulated in double
    {
      const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
      for (int r = warp; r < rr; r += nw) {
        double acc = 0.0;
        for (int c = lane; c < rr; c += 32) {
          const double u = Xr[r * ldp + c], v = Xi[r * ldp + c];
          acc += u * u + v * v;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0) s_sig[r] = acc;
      }
    }
    __syncthreads();
    // descending order; non-negative doubles order like their bit patterns,
    // which keeps the comparisons off the double-precision pipe
    for (int r = tid; r < rr; r += blockDim.x) {
      const long long v = __double_as_longlong(s_sig[r]);
      int rank = 0;
      for (int j = 0; j < rr; ++j) {
        const long long u = __double_as_longlong(s_sig[j]);
        rank += (u > v) || (u == v && j < r);
      }
      s_perm[rank] = r;
    }
    __syncthreads();
    if (tid < 32) {
      // k = #{sigma_j > cut sigma_0} (capped at kmax, at least 1), compared
      // as sigma_j^2 > cut^2 sigma_0^2; kept and total weights by warp sums
      const int lane = tid;
      const double s0 = s_sig[s_perm[0]];
      const double thr2 = a.cut * a.cut * s0;
      double total = 0.0;
      int cnt = 0;
      for (int j = lane; j < rr; j += 32) {
        total += s_sig[j];
        cnt += (j < kmax && s_sig[s_perm[j]] > thr2) ? 1 : 0;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        total += __shfl_xor_sync(FULL, total, o);
        cnt += __shfl_xor_sync(FULL, cnt, o);
      }
      int k = s0 > 0.0 ? cnt : 0;
      if (k < 1) k = 1;
      // vectorised density matrix: never split a multiplet of equal singular
      // values (the spectrum of |rho>> pairs the coherences q and -q; keeping
      // one member of a pair would leave rho non-Hermitian and the kept vector
      // arbitrary).  Every lane walks the same values, so k stays warp-uniform.
      if (a.multiplet > 0.0 && s0 > 0.0) {
        const double tol = a.multiplet * sqrt(s0);
        while (k > 1 && k < rr && sqrt(s_sig[s_perm[k - 1]]) - sqrt(s_sig[s_perm[k]]) <= tol) --k;
      }
      double kept = 0.0;
      for (int j = lane; j < k; j += 32) kept += s_sig[s_perm[j]];
#pragma unroll
      for (int o = 16; o; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
      if (lane == 0) {
        if (!(s0 > 0.0)) atomicOr(a.err, LT_EBIT_THETA_ZERO);
        s_k = k;
        s_norm = kept > 0.0 ? sqrt(kept) : 1.0;
        s_wdisc = total > 0.0 ? (total - kept) / total : 0.0;
        if (a.sweep_hist) atomicAdd(a.sweep_hist + (sweeps < 63 ? sweeps : 63), 1);
        if (a.counters) {
          // algorithmic real flops: the Jacobi (row norms each sweep and at the end,
          // one complex inner product per pair per sweep, 24 nJ per applied
          // rotation), the Householder preconditioning (sum_j 16 (mJ-j-1)(nJ-j)
          // for the LQ, sum_j 16 (mJ-j)(r-j-1) for the QR, 16 k sum_l (nJ-l) to
          // apply Q1) and the contractions of the mode (theta formed once)
          const double dr_ = rr;
          const double pairs = 0.5 * dr_ * (dr_ - 1.0) * sweeps;
          double fl = 4.0 * dr_ * dr_ * (sweeps + 1) + 8.0 * dr_ * pairs + 24.0 * dr_ * s_nrot;
          fl += 16.0 * (double)(sum_prod(mJ - 1, nJ, rr) + sum_prod(mJ, rr - 1, rr) +
                                (long long)k * sum_prod(nJ, 1, rr, true));
          const double mL = (double)D * chiL, nR = (double)D * chiR;
          if (mode == 0) fl += 8.0 * mL * nR * (chiM + D * D) + 8.0 * mL * k * nR;
          else if (mode == 1) fl += 8.0 * mL * nR * chiM + 8.0 * mL * k * nR;
          else fl += 8.0 * mL * chiM * k + 8.0 * k * chiM * nR;
          atomicAdd(a.counters + 0, 1ull);
          atomicAdd(a.counters + 1, (unsigned long long)s_nrot);
          atomicAdd(a.counters + 2, (unsigned long long)pairs);
          atomicAdd(a.counters + (a.gates ? 3 : 4), (unsigned long long)fl);
          if (a.gates) atomicAdd(a.counters + 5, 1ull);
        }
        if (sweeps > a.max_sweeps) atomicOr(a.err, LT_EBIT_NOCONV);
      }
    }
    __syncthreads();
    const int k = s_k;
    // V_k^+ rows: row perm j holds sigma_j w_j^+; v_j^+ = w_j^+ Q1^+ goes to Y[j]
    if constexpr (sizeof(R) == 4) {
      if (reg)
        apply_q1_reg<BondShape<R>::NT / LT_REG_CHI>(
            reinterpret_cast<const float*>(Xr), reinterpret_cast<const float*>(Xi), ldp, nJ, rr, k,
            s_perm, s_sig, reinterpret_cast<const float2*>(Y), reinterpret_cast<const float*>(s_beta),
            reinterpret_cast<float2*>(Y), ld);
      else if (shared_jac && cluster_shares_precondition(mJ, nJ))
        cluster_q1_lead(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, nJ, rr, k,
                        s_perm, s_sig, reinterpret_cast<float2*>(Y), ld,
                        a.cl_state + cid * LT_CL_STATE, C);
      else if (nJ > LT_REG_DIM)
        wide_q1(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, nJ, rr, k, s_perm,
                s_sig, reinterpret_cast<float2*>(Y), reinterpret_cast<const float*>(s_beta), ld);
      else
        apply_q1_f(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, nJ, rr, k,
                   s_perm, s_sig, reinterpret_cast<const float2*>(Y),
                   reinterpret_cast<const float*>(s_beta), reinterpret_cast<float2*>(Y), ld);
    } else {
      apply_q1<R>(Xr, Xi, ldp, nJ, rr, k, s_perm, s_sig, Y, s_beta, Y, ld);
    }
    __syncthreads();
    // single precision: V_k^+ orthonormal to working precision (E in the free planes)
    if constexpr (sizeof(R) == 4)
      reorthonormalise_rows<BondShape<R>::NT>(reinterpret_cast<float2*>(Y), ld, k, nJ,
                                              reinterpret_cast<float2*>(Xr));
    if (mode != 2) {
      // theta~ = G (B_b B_{b+1}) (identity gate in mode 1), then
      // B_b <- theta~ V_k (/ |S_k| in mode 0), B_{b+1} <- V_k^+
      if (tc_task) {
        // theta~ as the tensor-core pass left it over the two site slots
        if constexpr (kTc)
          theta_tc_planes(reinterpret_cast<float*>(Xr), reinterpret_cast<float*>(Xi), ldp, nJ,
                          D * chiL, reinterpret_cast<const float2*>(Bl), chiL, chiR, a.slot,
                          s_lamL, false);
      } else {
        form_theta<R, D>(Xr, Xi, ldp, nJ, D * chiL, Bl, Br, nullptr, chiL, chiM, chiR, s_gate,
                         sizeof(R) == 4 ? s_glo : nullptr, s_lamL, false);
      }
      __syncthreads();
      const int m = D * chiL;
      const R invn = mode == 0 && !a.keep_norm ? (R)(1.0 / s_norm) : (R)1;
      // B_b[r][j] = sum_c theta~[r][c] conj(V_k^+[j][c]): a thread takes four rows and two
      // columns j, j + 1, so each load of theta~ feeds two products and each load of V_k^+
      // four
      const int rq = (m + 3) >> 2, kq = (k + 1) >> 1;
      if constexpr (kCl) {
        if (shared_jac && cluster_shares_precondition(mJ, nJ)) {
          // the cluster computes B_b's items (rank 0's share here, the rest in cluster_split)
          float* cls = a.cl_state + cid * LT_CL_STATE;
          if (tid == 0) cls[LT_CL_K + 1] = invn;
          __threadfence();
          cluster_sync();
          split_rows_cluster(reinterpret_cast<const float*>(Xr), reinterpret_cast<const float*>(Xi),
                             ldp, m, nJ, reinterpret_cast<const float2*>(Y), ld, k, invn,
                             reinterpret_cast<float2*>(Bl), 0, C);
          __threadfence();
          cluster_sync();
        }
      }
      const bool split_here = !(kCl && shared_jac && cluster_shares_precondition(mJ, nJ));
      for (int idx = tid; split_here && idx < rq * kq; idx += blockDim.x) {
        const int g = idx / kq, r0 = g << 2, j0 = 2 * (idx - g * kq);
        const bool two = j0 + 1 < k;
        const Tc* y0 = Y + j0 * ld;
        const Tc* y1 = Y + (two ? j0 + 1 : j0) * ld;
        Tc acc[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = czero<Tc>();
        const int nr = m - r0 < 4 ? m - r0 : 4;
        for (int c = 0; c < nJ; ++c) {
          const Tc v0 = y0[c], v1 = y1[c];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u < nr) {
              const int o = (r0 + u) * ldp + c;
              const Tc x = cmk<Tc>(Xr[o], Xi[o]);
              cfmac(acc[u][0], x, v0);
              cfmac(acc[u][1], x, v1);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < nr) {
            Bl[(r0 + u) * k + j0] = cscale(acc[u][0], invn);
            if (two) Bl[(r0 + u) * k + j0 + 1] = cscale(acc[u][1], invn);
          }
      }
      for (int idx = tid; idx < k * nJ; idx += blockDim.x) {
        const int j = idx / nJ, c = idx - j * nJ;
        Br[idx] = Y[j * ld + c];
      }
    } else {
      // B_b <- B_b V_k / |S_k| (2chi_{b-1} x k), staged, then written
      Tc* St = Y + k * ld;
      const int m = D * chiL, nR = D * chiR;
      const R invn = (R)(1.0 / s_norm);
      for (int idx = tid; idx < m * k; idx += blockDim.x) {
        const int r = idx / k, j = idx - r * k;
        const Tc* yj = Y + j * ld;
        const Tc* br = Bl + r * chiM;
        Tc acc = czero<Tc>();
        for (int c = 0; c < chiM; ++c) cfmac(acc, br[c], yj[c]);
        St[idx] = cscale(acc, invn);
      }
      __syncthreads();
      // Lambda_b as the norms of the columns of Lambda_{b-1} B_b that are stored
      // (accumulated in double): S_k/|S_k| in exact arithmetic, and in single
      // precision the norm the new tensors carry, which S_k from the rotated
      // columns misstates by a bias that the sweep would pass into <psi|psi>
      {
        double* lb = a.lam + ((long long)traj * (L - 1) + b) * chi;
        for (int j = tid; j < k; j += blockDim.x) {
          double s = 0.0;
          for (int r = 0; r < m; ++r) {
            const double w = s_lamL[D == 2 ? r >> 1 : r / D];
            const Tc x = St[r * k + j];
            s += w * w * ((double)x.x * (double)x.x + (double)x.y * (double)x.y);
          }
          lb[j] = sqrt(s);
        }
      }
      for (int idx = tid; idx < m * k; idx += blockDim.x) Bl[idx] = St[idx];
      __syncthreads();
      // B_{b+1} <- V_k^+ B_{b+1} (k x 2chi_{b+1}), staged, then written
      for (int idx = tid; idx < k * nR; idx += blockDim.x) {
        const int j = idx / nR, x = idx - j * nR;
        const Tc* yj = Y + j * ld;
        Tc acc = czero<Tc>();
        for (int c = 0; c < chiM; ++c) cfma(acc, yj[c], Br[c * nR + x]);
        St[idx] = acc;
      }
      __syncthreads();
      for (int idx = tid; idx < k * nR; idx += blockDim.x) Br[idx] = St[idx];
    }
    {
      double* lb = a.lam + ((long long)traj * (L - 1) + b) * chi;
      for (int j = tid; mode != 2 && j < k; j += blockDim.x) lb[j] = sqrt(s_sig[s_perm[j]]) / s_norm;
      if (tid == 0) {
        a.dims[(long long)traj * (L - 1) + b] = k;
        if (mode != 1) a.trunc[(long long)traj * (L - 1) + b] += s_wdisc;
        // after the right-to-left sweep everything right of bond 0 is
        // right-canonical, so ||S||^2 there is <psi|psi>, divided out here
        if (mode == 2 && b == 0 && a.logw) a.logw[traj] += 2.0 * log(s_norm);
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

// Jump-or-evolve decision of one trajectory (Sec. 4.1): P = sum_k W_k dt over
// the rates just written; draw r from Philox (counter traj_offset + traj, step,
// purpose 0); jump iff r < P, to the least channel whose cumulative W dt
// exceeds r.  Replayed channels bypass the draw.
__device__ void decide_channel(const EnvArgs& a, int traj) {
  const int L = a.L;
  const double* rt = a.rates + (long long)traj * 3 * L;
  int ch = -1;
  const int rep = a.replay ? a.replay[traj] : -2;
  if (rep == -2) {
    double total = 0.0;
    for (int j = 0; j < 3 * L; ++j) total += rt[j] * a.dt;
    if (total >= 0.5) atomicOr(a.err, LT_EBIT_PROB);
    const long long step = a.step_dev ? *a.step_dev : a.step;
    const double r = philox_uniform(a.seed, (uint32_t)(a.traj_offset + traj), (uint64_t)step, 0u);
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

// ---- shared-memory tiled complex GEMM (one CTA of 256 threads) -----------------------
// C (M x N) = (acc ? C : 0) + op(A) op(B), where op(A)(i,k) = A[i ar + k ac] and
// op(B)(k,j) = B[k br + j bc], each conjugated when its flag is set.  Output
// tiles of 64 x 64, each thread holding a 4 x 4 block; K in chunks of 16 staged
// in shared memory (pitch 65, odd, so 8-byte accesses are conflict-free), with
// the staging loop running along whichever operand stride is unit.
#define LT_TG_P 65
template <typename R>
__device__ void tile_gemm(int M, int N, int K, const typename CT<R>::T* A, int ar, int ac,
                          bool conjA, const typename CT<R>::T* B, int br, int bc, bool conjB,
                          typename CT<R>::T* C, int ldc, bool acc, typename CT<R>::T* sA,
                          typename CT<R>::T* sB) {
  typedef typename CT<R>::T Tc;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int i0 = 0; i0 < M; i0 += 64) {
    for (int j0 = 0; j0 < N; j0 += 64) {
      Tc c[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) c[u][v] = czero<Tc>();
      for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
          int ii, kk;
          if (ac == 1) {
            kk = e & 15;
            ii = e >> 4;
          } else {
            ii = e & 63;
            kk = e >> 6;
          }
          const int gi = i0 + ii, gk = k0 + kk;
          Tc v = czero<Tc>();
          if (gi < M && gk < K) {
            v = A[(long long)gi * ar + (long long)gk * ac];
            if (conjA) v.y = -v.y;
          }
          sA[kk * LT_TG_P + ii] = v;
          int jj, kb;
          if (bc == 1) {
            jj = e & 63;
            kb = e >> 6;
          } else {
            kb = e & 15;
            jj = e >> 4;
          }
          const int gj = j0 + jj, gkb = k0 + kb;
          Tc w = czero<Tc>();
          if (gkb < K && gj < N) {
            w = B[(long long)gkb * br + (long long)gj * bc];
            if (conjB) w.y = -w.y;
          }
          sB[kb * LT_TG_P + jj] = w;
        }
        __syncthreads();
        const int kn = K - k0 < 16 ? K - k0 : 16;
        for (int kk = 0; kk < kn; ++kk) {
          Tc av[4], bv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) av[u] = sA[kk * LT_TG_P + ty + 16 * u];
#pragma unroll
          for (int v = 0; v < 4; ++v) bv[v] = sB[kk * LT_TG_P + tx + 16 * v];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) cfma(c[u][v], av[u], bv[v]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int gi = i0 + ty + 16 * u;
        if (gi >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int gj = j0 + tx + 16 * v;
          if (gj >= N) continue;
          Tc o = c[u][v];
          if (acc) {
            const Tc p = C[(long long)gi * ldc + gj];
            o.x += p.x;
            o.y += p.y;
          }
          C[(long long)gi * ldc + gj] = o;
        }
      }
    }
  }
  __syncthreads();
}

// Right environments by tiled GEMMs: T'[(a,s)][b'] = sum_b B[(a,s)][b] R_{i+1}[b][b'],
// R_i[a][a'] = sum_{(s,b')} T'[a][(s,b')] conj(B[a'][(s,b')]).  Returns <psi|psi>.
template <typename R>
__device__ double right_envs_tiled(const typename CT<R>::T* B, const int* dm, int L, int chi,
                                   int slot, typename CT<R>::T* Rl, typename CT<R>::T* T,
                                   typename CT<R>::T* sA, typename CT<R>::T* sB) {
  typedef typename CT<R>::T Tc;
  const int chi2 = chi * chi;
  if (threadIdx.x == 0) Rl[(long long)L * chi2] = cmk<Tc>(1.0, 0.0);
  __syncthreads();
  for (int i = L - 1; i >= 0; --i) {
    const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
    const Tc* Bi = B + (long long)i * slot;
    const Tc* Rn = Rl + (long long)(i + 1) * chi2;
    Tc* Ri = Rl + (long long)i * chi2;
    tile_gemm<R>(2 * cl, cr, cr, Bi, cr, 1, false, Rn, chi, 1, false, T, cr, false, sA, sB);
    tile_gemm<R>(cl, cl, 2 * cr, T, 2 * cr, 1, false, Bi, 1, 2 * cr, true, Ri, chi, false, sA, sB);
  }
  return (double)Rl[0].x;
}

// env kernel with tiled contractions: per trajectory exact <n_k> for every
// site, then (kRates) rates and the Philox decision (decide_channel)
template <typename R, bool kRates = true>
__global__ void __launch_bounds__(LT_BLOCK) env_tiled_kernel(EnvArgs a) {
  typedef typename CT<R>::T Tc;
  __shared__ double red[32];
  __shared__ Tc sA[16 * LT_TG_P], sB[16 * LT_TG_P];
  const int L = a.L, chi = a.chi, chi2 = chi * chi;
  Tc* ws = reinterpret_cast<Tc*>(a.scratch) + (long long)blockIdx.x * a.scratch_stride;
  Tc* Rl = ws;                                  // (L+1) chi^2
  Tc* T = Rl + (long long)(L + 1) * chi2;       // 2 chi^2
  Tc* Le = T + 2 * chi2;                        // chi^2
  Tc* Ln = Le + chi2;                           // chi^2
  Tc* Mb = Ln + chi2;                           // 2 chi^2
  Tc* N1 = T;                                   // reuses T in the left sweep
  for (int traj = blockIdx.x; traj < a.n_traj; traj += gridDim.x) {
    const Tc* B = reinterpret_cast<const Tc*>(a.B) + (long long)traj * L * a.slot;
    const int* dm = a.dims + (long long)traj * (L - 1);
    // bond dimensions outside [1, chi] would take the contractions past the site
    // slots and the scratch: such a trajectory's densities become NaN, it draws
    // no jump, and it is skipped (its dimensions come from the caller in
    // lt_measure_density_noalloc)
    int bad = 0;
    for (int b = threadIdx.x; b < L - 1; b += blockDim.x) bad |= (dm[b] < 1 || dm[b] > chi);
    if (__syncthreads_or(bad)) {
      const double qnan = __longlong_as_double(0x7ff8000000000000LL);
      for (int k = threadIdx.x; k < L; k += blockDim.x) a.density[(long long)traj * L + k] = qnan;
      if (kRates) {
        for (int k = threadIdx.x; k < 3 * L; k += blockDim.x) a.rates[(long long)traj * 3 * L + k] = 0.0;
        if (threadIdx.x == 0) {
          a.channel[traj] = -1;
          a.evolve[traj] = 1;
          if (a.err) atomicOr(a.err, LT_EBIT_BADARG);
        }
      }
      __syncthreads();
      continue;
    }
    const double nrm2 = right_envs_tiled<R>(B, dm, L, chi, a.slot, Rl, T, sA, sB);
    if (threadIdx.x == 0) Le[0] = cmk<Tc>(1.0, 0.0);
    __syncthreads();
    for (int k = 0; k < L; ++k) {
      const int cl = k == 0 ? 1 : dm[k - 1], cr = k == L - 1 ? 1 : dm[k];
      const Tc* Bk = B + (long long)k * a.slot;
      const Tc* Rn = Rl + (long long)(k + 1) * chi2;
      // M[a][(s,b)] = sum_a' Le[a][a'] B[a'][(s,b)]
      tile_gemm<R>(cl, 2 * cr, cl, Le, chi, 1, false, Bk, 2 * cr, 1, false, Mb, 2 * cr, false, sA, sB);
      // N1[a][b'] = sum_b M[a][(1,b)] R_{k+1}[b][b']
      tile_gemm<R>(cl, cr, cr, Mb + cr, 2 * cr, 1, false, Rn, chi, 1, false, N1, cr, false, sA, sB);
      // Le'[b'][b] = sum_{(a,s)} conj(B[(a,s)][b']) M[(a,s)][b]
      tile_gemm<R>(cr, cr, 2 * cl, Bk, 1, cr, true, Mb, cr, 1, false, Ln, chi, false, sA, sB);
      // <n_k> |psi|^2 = sum_{a,b} conj(B[a][1][b]) N1[a][b]
      double re = 0.0;
      for (int idx = threadIdx.x; idx < cl * cr; idx += blockDim.x) {
        const int aa = idx / cr, bb = idx - aa * cr;
        const Tc p = Bk[aa * 2 * cr + cr + bb], q = N1[aa * cr + bb];
        re += (double)p.x * q.x + (double)p.y * q.y;
      }
      re = block_sum_double(re, red);
      if (threadIdx.x == 0) {
        const double nk = re / nrm2;
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
    if (kRates && a.decide && threadIdx.x == 0) decide_channel(a, traj);
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
// (with logw, of w_t x[t] with w_t = exp(logw[t]): the quantum-state-diffusion
// estimator mean_t(w_t <O>_t) of Sec. 5.2)
__global__ void reduce_mean_sem_kernel(const double* x, int n, int M, double* mean, double* sem,
                                       const double* logw) {
  __shared__ double red[32];
  for (int col = blockIdx.x; col < M; col += gridDim.x) {
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x)
      s += x[(long long)t * M + col] * (logw ? exp(logw[t]) : 1.0);
    const double mu = block_sum_double(s, red) / n;
    double v = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double d = x[(long long)t * M + col] * (logw ? exp(logw[t]) : 1.0) - mu;
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
__global__ void reduce_mean_c_kernel(const double2* x, int n, int M, double* out,
                                     const double* logw) {
  __shared__ double red[32];
  for (int col = blockIdx.x; col < M; col += gridDim.x) {
    double re = 0.0, im = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double2 v = x[(long long)t * M + col];
      const double w = logw ? exp(logw[t]) : 1.0;
      re += w * v.x;
      im += w * v.y;
    }
    re = block_sum_double(re, red);
    im = block_sum_double(im, red);
    if (threadIdx.x == 0) {
      out[2 * col] = re / n;
      out[2 * col + 1] = im / n;
    }
  }
}

// ---- quantum state diffusion noise (Sec. 5.2) ----------------------------------------
// B_i <- M_i B_i on the physical index of every site of every trajectory, with
// M_i = prod over the site's channels k = 3 i + kind (loss, then gain, then
// dephasing) of 1 + eta_k sqrt(gamma_k dt) L_k; eta_{2j}, eta_{2j+1} is the j-th
// Gaussian pair of (trajectory, step).  M_i is real; one CTA per (trajectory,
// site), thread 0 builds M_i.
template <typename R>
__global__ void __launch_bounds__(128) qsd_noise_kernel(typename CT<R>::T* B, const int* dims, int L,
                                                        int slot, int n_traj, long long traj_offset,
                                                        long long step_arg, const long long* step_dev,
                                                        uint64_t seed, const double* gam, double dt) {
  typedef typename CT<R>::T Tc;
  __shared__ double sM[4];
  const long long step = step_dev ? *step_dev : step_arg;
  const long long ntask = (long long)n_traj * L;
  for (long long task = blockIdx.x; task < ntask; task += gridDim.x) {
    const int traj = (int)(task / L), i = (int)(task - (long long)traj * L);
    if (threadIdx.x == 0) {
      double m00 = 1.0, m01 = 0.0, m10 = 0.0, m11 = 1.0;
      for (int kind = 0; kind < 3; ++kind) {
        const double g = gam[kind * L + i];
        if (!(g > 0.0)) continue;
        const int k = 3 * i + kind;
        double e0, e1;
        philox_gaussian_pair(seed, (uint32_t)(traj_offset + traj), (uint64_t)step, (uint32_t)(k >> 1),
                             e0, e1);
        const double a = ((k & 1) ? e1 : e0) * sqrt(g * dt);
        if (kind == 0) {         // loss |0><1|: row 0 += a row 1
          m00 += a * m10;
          m01 += a * m11;
        } else if (kind == 1) {  // gain |1><0|: row 1 += a row 0
          m10 += a * m00;
          m11 += a * m01;
        } else {                 // dephasing |1><1|: row 1 *= 1 + a
          m10 += a * m10;
          m11 += a * m11;
        }
      }
      sM[0] = m00;
      sM[1] = m01;
      sM[2] = m10;
      sM[3] = m11;
    }
    __syncthreads();
    const int* dm = dims + (long long)traj * (L - 1);
    const int chiL = i == 0 ? 1 : dm[i - 1], chiR = i == L - 1 ? 1 : dm[i];
    Tc* Bi = B + ((long long)traj * L + i) * slot;
    const R m00 = (R)sM[0], m01 = (R)sM[1], m10 = (R)sM[2], m11 = (R)sM[3];
    for (int idx = threadIdx.x; idx < chiL * chiR; idx += blockDim.x) {
      const int aa = idx / chiR, cc = idx - aa * chiR;
      Tc* p0 = Bi + aa * 2 * chiR + cc;
      Tc* p1 = p0 + chiR;
      const Tc v0 = *p0, v1 = *p1;
      *p0 = cmk<Tc>(m00 * v0.x + m01 * v1.x, m00 * v0.y + m01 * v1.y);
      *p1 = cmk<Tc>(m10 * v0.x + m11 * v1.x, m10 * v0.y + m11 * v1.y);
    }
    __syncthreads();
  }
}

// ---- traces of the vectorised density matrix (Sec. 3.1) -------------------------------
// Tr(O rho) of a product operator O contracts |rho>> with one vector per site,
// o[2n + n'] = O[n', n]: identity (1,0,0,1), n (0,0,0,1), sigma+ = |1><0| (0,1,0,0),
// sigma- = |0><1| (0,0,1,0), parity (1,0,0,-1).  With T_i(o) = sum_m o[m] B_i[:, m, :]
// a CTA per chain builds the right vectors R_i = T_i(id) R_{i+1} (R_L = 1) and the
// left vectors L_{i+1} = L_i T_i(id) (L_0 = 1) in its scratch, Tr rho = R_0, and
//   <n_i> = Re(L_i T_i(n) R_{i+1} / Tr rho),
//   C_ij  = L_i T_i(s+) [prod_{i<l<j} T_l(parity)] T_j(s-) R_{j+1} / Tr rho  (i < j),
// C_ji = conj(C_ij), C_ii = <n_i> (Jordan-Wigner string as for pure states).  The
// scale of |rho>> is arbitrary (each bond update fixes its Hilbert-Schmidt norm),
// so only these ratios are physical.  Every contraction accumulates in double
// precision in a fixed order, so results do not depend on the grid.
static_assert(LT_MAX_CHI <= LT_BLOCK, "one vector element per thread");

__device__ __forceinline__ double2 block_sum_c2(double2 v, double2* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    v.x += __shfl_xor_sync(FULL, v.x, o);
    v.y += __shfl_xor_sync(FULL, v.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    s.x += red[w].x;
    s.y += red[w].y;
  }
  __syncthreads();
  return s;
}

__device__ __forceinline__ void zfma(double2& acc, double2 x, double yr, double yi) {
  acc.x = fma(x.x, yr, fma(-x.y, yi, acc.x));
  acc.y = fma(x.x, yi, fma(x.y, yr, acc.y));
}

// Re(num / den)
__device__ __forceinline__ double re_ratio(double2 num, double2 den) {
  return (num.x * den.x + num.y * den.y) / (den.x * den.x + den.y * den.y);
}

template <typename R>
__global__ void __launch_bounds__(LT_BLOCK) mpdo_trace_kernel(MpdoArgs a) {
  typedef typename CT<R>::T Tc;
  __shared__ double2 s_v[LT_MAX_CHI];
  __shared__ double2 s_red[LT_BLOCK / 32];
  const int L = a.L, chi = a.chi, tid = threadIdx.x;
  double2* Rv = a.scratch + (long long)blockIdx.x * a.stride;  // [L + 1][chi]
  double2* Lv = Rv + (long long)(L + 1) * chi;                 // [L + 1][chi]
  for (int t = blockIdx.x; t < a.n_traj; t += gridDim.x) {
    const int* dm = a.dims + (long long)t * (L - 1);
    const Tc* Bt = reinterpret_cast<const Tc*>(a.B) + (long long)t * L * a.slot;
    if (tid == 0) {
      Rv[(long long)L * chi] = make_double2(1.0, 0.0);
      Lv[0] = make_double2(1.0, 0.0);
    }
    __syncthreads();
    for (int i = L - 1; i >= 0; --i) {
      const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
      const Tc* Bi = Bt + (long long)i * a.slot;
      if (tid < cl) {
        const Tc* row = Bi + (long long)tid * 4 * cr;  // B_i[x][m][c] at (4x + m) cr + c
        double2 acc = make_double2(0.0, 0.0);
        for (int c = 0; c < cr; ++c) {
          const Tc b0 = row[c], b3 = row[3 * cr + c];
          zfma(acc, Rv[(long long)(i + 1) * chi + c], (double)b0.x + (double)b3.x,
               (double)b0.y + (double)b3.y);
        }
        Rv[(long long)i * chi + tid] = acc;
      }
      __syncthreads();
    }
    const double2 tr = Rv[0];
    for (int i = 0; i < L; ++i) {
      const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
      const Tc* Bi = Bt + (long long)i * a.slot;
      double2 part = make_double2(0.0, 0.0);
      if (tid < cr) {
        double2 nxt = make_double2(0.0, 0.0), num = make_double2(0.0, 0.0);
        for (int x = 0; x < cl; ++x) {
          const double2 l = Lv[(long long)i * chi + x];
          const Tc b0 = Bi[(long long)(4 * x) * cr + tid], b3 = Bi[(long long)(4 * x + 3) * cr + tid];
          zfma(num, l, b3.x, b3.y);
          zfma(nxt, l, (double)b0.x + (double)b3.x, (double)b0.y + (double)b3.y);
        }
        Lv[(long long)(i + 1) * chi + tid] = nxt;
        const double2 r = Rv[(long long)(i + 1) * chi + tid];
        zfma(part, num, r.x, r.y);
      }
      const double2 tot = block_sum_c2(part, s_red);
      if (tid == 0) {
        const double n = re_ratio(tot, tr);
        a.density[(long long)t * L + i] = n;
        if (a.corr) a.corr[((long long)t * L + i) * L + i] = make_double2(n, 0.0);
      }
    }
    if (a.corr) {
      for (int i = 0; i + 1 < L; ++i) {
        const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
        const Tc* Bi = Bt + (long long)i * a.slot;
        if (tid < cr) {
          double2 v = make_double2(0.0, 0.0);
          for (int x = 0; x < cl; ++x) {
            const Tc b1 = Bi[(long long)(4 * x + 1) * cr + tid];
            zfma(v, Lv[(long long)i * chi + x], b1.x, b1.y);
          }
          s_v[tid] = v;
        }
        __syncthreads();
        for (int j = i + 1; j < L; ++j) {
          const int jl = dm[j - 1], jr = j == L - 1 ? 1 : dm[j];
          const Tc* Bj = Bt + (long long)j * a.slot;
          double2 part = make_double2(0.0, 0.0), nv = make_double2(0.0, 0.0);
          if (tid < jr) {
            double2 w = make_double2(0.0, 0.0);
            for (int x = 0; x < jl; ++x) {
              const double2 v = s_v[x];
              const Tc b0 = Bj[(long long)(4 * x) * jr + tid], b2 = Bj[(long long)(4 * x + 2) * jr + tid];
              const Tc b3 = Bj[(long long)(4 * x + 3) * jr + tid];
              zfma(w, v, b2.x, b2.y);
              zfma(nv, v, (double)b0.x - (double)b3.x, (double)b0.y - (double)b3.y);
            }
            const double2 r = Rv[(long long)(j + 1) * chi + tid];
            zfma(part, w, r.x, r.y);
          }
          const double2 tot = block_sum_c2(part, s_red);  // its barriers end every read of s_v
          if (tid < jr) s_v[tid] = nv;
          if (tid == 0) {
            const double den = tr.x * tr.x + tr.y * tr.y;
            const double2 cij = make_double2((tot.x * tr.x + tot.y * tr.y) / den,
                                             (tot.y * tr.x - tot.x * tr.y) / den);
            a.corr[((long long)t * L + i) * L + j] = cij;
            a.corr[((long long)t * L + j) * L + i] = make_double2(cij.x, -cij.y);
          }
          __syncthreads();
        }
      }
    }
    __syncthreads();
  }
}

// ---- locally purified density matrix (Sec. 3.2) ------------------------------------------
// rho = X X^+ with X an MPS over s = 2n + k (physical n, Kraus k, chi_k = 2).
__device__ __forceinline__ double2 d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 d2(double2 v) { return v; }

// C (+)= sgn op(A) op(B) with double accumulation; op = identity or, with the h
// flag, the conjugate transpose.  A and B are site-tensor slices (float2 or
// double2) or double2 environments.
template <typename TA, typename TB>
__device__ void zgemm(int M, int N, int K, const TA* A, int lda, bool hA, const TB* B, int ldb,
                      bool hB, double2* C, int ldc, bool acc, double sgn) {
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    double2 sacc = make_double2(0.0, 0.0);
    for (int k = 0; k < K; ++k) {
      double2 x = d2(hA ? A[(long long)k * lda + i] : A[(long long)i * lda + k]);
      double2 y = d2(hB ? B[(long long)j * ldb + k] : B[(long long)k * ldb + j]);
      if (hA) x.y = -x.y;
      if (hB) y.y = -y.y;
      sacc.x = fma(x.x, y.x, fma(-x.y, y.y, sacc.x));
      sacc.y = fma(x.x, y.y, fma(x.y, y.x, sacc.y));
    }
    double2 o = acc ? C[(long long)i * ldc + j] : make_double2(0.0, 0.0);
    o.x += sgn * sacc.x;
    o.y += sgn * sacc.y;
    C[(long long)i * ldc + j] = o;
  }
}

// sum_{a,c} conj(P[a][c]) Q[a][c] over a (M x N) block of double2 P and slice Q
template <typename TQ>
__device__ double2 zdot(int M, int N, const TQ* P, int ldp, const double2* Qd, int ldq, double2* red) {
  double2 part = make_double2(0.0, 0.0);
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const double2 x = d2(P[(long long)i * ldp + j]), y = Qd[(long long)i * ldq + j];
    part.x = fma(x.x, y.x, fma(x.y, y.y, part.x));
    part.y = fma(x.x, y.y, fma(-x.y, y.x, part.y));
  }
  return block_sum_c2(part, red);
}

// The R step of one site (Eqs. MatrixR, NewPurified): the enlarged Kraus set
// A~ = [A^{.,k} ; sqrt(gamma_c dt) L_c A^{.,k}] (identity first, then loss,
// gain, dephasing with gamma > 0; columns p 2 + k), its Lambda_{i-1}-weighted
// Gram matrix G = A~^+ W^2 A~ (at most 8 x 8), the two leading eigenvectors
// V of G, and A <- A~ V.  G comes from the 16 n-resolved sums
// g[m][m'][k][k'] = sum_{a,c} w_a^2 conj(B[a][2m+k][c]) B[a][2m'+k'][c]:
// G[(p,k),(q,k')] = sum_n sum_{m,m'} O_p[n][m] O_q[n][m'] g[m][m'][k][k'].
// One thread diagonalises G by cyclic complex Jacobi rotations in double.
struct KrausArgs {
  void* B;
  const double* lam;
  const int* dims;
  int L, chi, slot, n_traj;
  const double* gam;  // [3][L] loss, gain, dephasing
  double dt;
};

template <typename R>
__global__ void __launch_bounds__(LT_BLOCK) kraus_step_kernel(KrausArgs a) {
  typedef typename CT<R>::T Tc;
  __shared__ double s_part[LT_BLOCK / 32][32];
  __shared__ double s_g[32];
  __shared__ double2 s_V[8][2];
  __shared__ double s_op[4][4];  // op p: O_p[n][m] (real), row-major 2 x 2
  __shared__ int s_nops;
  const int L = a.L, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long ntask = (long long)a.n_traj * L;
  for (long long task = blockIdx.x; task < ntask; task += gridDim.x) {
    const int t = (int)(task / L), i = (int)(task - (long long)t * L);
    const int* dm = a.dims + (long long)t * (L - 1);
    const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
    Tc* Bi = reinterpret_cast<Tc*>(a.B) + ((long long)t * L + i) * a.slot;
    const double* lw = a.lam + ((long long)t * (L - 1) + (i > 0 ? i - 1 : 0)) * a.chi;
    if (tid == 0) {
      int p = 0;
      s_op[0][0] = 1.0; s_op[0][1] = 0.0; s_op[0][2] = 0.0; s_op[0][3] = 1.0;
      const double g[3] = {a.gam[i], a.gam[L + i], a.gam[2 * L + i]};
      for (int kind = 0; kind < 3; ++kind) {
        if (!(g[kind] > 0.0)) continue;
        const double r = sqrt(g[kind] * a.dt);
        ++p;
        for (int e = 0; e < 4; ++e) s_op[p][e] = 0.0;
        if (kind == 0) s_op[p][0 * 2 + 1] = r;       // sigma- = |0><1|
        else if (kind == 1) s_op[p][1 * 2 + 0] = r;  // sigma+ = |1><0|
        else s_op[p][1 * 2 + 1] = r;                 // n
      }
      s_nops = p + 1;
    }
    // the 16 weighted sums g[m][m'][k][k'] (complex: 32 doubles per thread)
    double acc[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) acc[e] = 0.0;
    for (int x = tid; x < cl * cr; x += blockDim.x) {
      const int aa = x / cr, c = x - aa * cr;
      const double w = i > 0 ? lw[aa] : 1.0, w2 = w * w;
      double2 v[4];
#pragma unroll
      for (int sidx = 0; sidx < 4; ++sidx) v[sidx] = d2(Bi[(long long)(aa * 4 + sidx) * cr + c]);
#pragma unroll
      for (int s1 = 0; s1 < 4; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) {
          // conj(v[s1]) v[s2], s = 2m + k: index ((m1 2 + m2) 2 + k1) 2 + k2
          const int m1 = s1 >> 1, k1 = s1 & 1, m2 = s2 >> 1, k2 = s2 & 1;
          const int e = (((m1 * 2 + m2) * 2 + k1) * 2 + k2) * 2;
          acc[e] = fma(w2, v[s1].x * v[s2].x + v[s1].y * v[s2].y, acc[e]);
          acc[e + 1] = fma(w2, v[s1].x * v[s2].y - v[s1].y * v[s2].x, acc[e + 1]);
        }
    }
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      double v = acc[e];
#pragma unroll
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
      if (lane == 0) s_part[warp][e] = v;
    }
    __syncthreads();
    if (tid < 32) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_part[w][tid];
      s_g[tid] = v;
    }
    __syncthreads();
    if (tid == 0) {
      const int np = s_nops, nc = 2 * np;
      double2 G[8][8], V[8][8];
      for (int P = 0; P < nc; ++P)
        for (int Q = 0; Q < nc; ++Q) {
          const int p = P >> 1, k1 = P & 1, q = Q >> 1, k2 = Q & 1;
          double2 z = make_double2(0.0, 0.0);
          for (int n = 0; n < 2; ++n)
            for (int m1 = 0; m1 < 2; ++m1)
              for (int m2 = 0; m2 < 2; ++m2) {
                const double o = s_op[p][n * 2 + m1] * s_op[q][n * 2 + m2];
                if (o == 0.0) continue;
                const int e = (((m1 * 2 + m2) * 2 + k1) * 2 + k2) * 2;
                z.x += o * s_g[e];
                z.y += o * s_g[e + 1];
              }
          G[P][Q] = z;
          V[P][Q] = make_double2(P == Q ? 1.0 : 0.0, 0.0);
        }
      // cyclic Jacobi for the Hermitian G: for the pair (p, q) with
      // G_pq = |b| e, the unitary U = D J (D = diag(1, conj e) on (p, q), J the
      // real rotation that diagonalises D^+ G D) gives U^+ G U with G_pq = 0
      double scale = 0.0;
      for (int P = 0; P < nc; ++P) scale = fmax(scale, fabs(G[P][P].x));
      for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0;
        for (int P = 0; P < nc; ++P)
          for (int Q = P + 1; Q < nc; ++Q) off = fmax(off, hypot(G[P][Q].x, G[P][Q].y));
        if (!(off > 1e-15 * scale)) break;
        for (int p = 0; p < nc; ++p)
          for (int q = p + 1; q < nc; ++q) {
            const double ab = hypot(G[p][q].x, G[p][q].y);
            if (!(ab > 1e-300)) continue;
            const double ex = G[p][q].x / ab, ey = G[p][q].y / ab;  // e
            const double tau = (G[q][q].x - G[p][p].x) / (2.0 * ab);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + tt * tt), sn = tt * c;
            // columns: new p = c col_p - s conj(e) col_q, new q = s col_p + c conj(e) col_q
            for (int r = 0; r < nc; ++r) {
              const double2 gp = G[r][p], gq = G[r][q];
              const double2 qe = make_double2(gq.x * ex + gq.y * ey, gq.y * ex - gq.x * ey);  // gq conj(e)
              G[r][p] = make_double2(c * gp.x - sn * qe.x, c * gp.y - sn * qe.y);
              G[r][q] = make_double2(sn * gp.x + c * qe.x, sn * gp.y + c * qe.y);
              const double2 vp = V[r][p], vq = V[r][q];
              const double2 ve = make_double2(vq.x * ex + vq.y * ey, vq.y * ex - vq.x * ey);
              V[r][p] = make_double2(c * vp.x - sn * ve.x, c * vp.y - sn * ve.y);
              V[r][q] = make_double2(sn * vp.x + c * ve.x, sn * vp.y + c * ve.y);
            }
            // rows: new p = c row_p - s e row_q, new q = s row_p + c e row_q
            for (int r = 0; r < nc; ++r) {
              const double2 gp = G[p][r], gq = G[q][r];
              const double2 qe = make_double2(gq.x * ex - gq.y * ey, gq.y * ex + gq.x * ey);  // e gq
              G[p][r] = make_double2(c * gp.x - sn * qe.x, c * gp.y - sn * qe.y);
              G[q][r] = make_double2(sn * gp.x + c * qe.x, sn * gp.y + c * qe.y);
            }
            G[p][q] = make_double2(0.0, 0.0);
            G[q][p] = make_double2(0.0, 0.0);
          }
      }
      // the two largest eigenvalues (ties to the lower index)
      int first = 0;
      for (int P = 1; P < nc; ++P)
        if (G[P][P].x > G[first][first].x) first = P;
      int second = first == 0 ? 1 : 0;
      for (int P = 0; P < nc; ++P)
        if (P != first && G[P][P].x > G[second][second].x) second = P;
      for (int P = 0; P < 8; ++P) {
        s_V[P][0] = P < nc ? V[P][first] : make_double2(0.0, 0.0);
        s_V[P][1] = P < nc ? V[P][second] : make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
    // A <- A~ V: new B[a][2n + k][c] = sum_{p,k0} (O_p B_{k0})[a][n][c] V[p 2 + k0][k]
    const int np = s_nops;
    for (int x = tid; x < cl * cr; x += blockDim.x) {
      const int aa = x / cr, c = x - aa * cr;
      double2 v[4];
#pragma unroll
      for (int sidx = 0; sidx < 4; ++sidx) v[sidx] = d2(Bi[(long long)(aa * 4 + sidx) * cr + c]);
      double2 o[4];
#pragma unroll
      for (int sidx = 0; sidx < 4; ++sidx) o[sidx] = make_double2(0.0, 0.0);
      for (int p = 0; p < np; ++p)
        for (int k0 = 0; k0 < 2; ++k0)
          for (int n = 0; n < 2; ++n) {
            double2 col = make_double2(0.0, 0.0);  // (O_p B_{k0})[a][n][c]
            for (int m = 0; m < 2; ++m) {
              const double op = s_op[p][n * 2 + m];
              col.x += op * v[m * 2 + k0].x;
              col.y += op * v[m * 2 + k0].y;
            }
            for (int k = 0; k < 2; ++k) {
              const double2 w = s_V[p * 2 + k0][k];
              o[n * 2 + k].x += col.x * w.x - col.y * w.y;
              o[n * 2 + k].y += col.x * w.y + col.y * w.x;
            }
          }
#pragma unroll
      for (int sidx = 0; sidx < 4; ++sidx)
        Bi[(long long)(aa * 4 + sidx) * cr + c] = cmk<Tc>(o[sidx].x, o[sidx].y);
    }
    __syncthreads();
  }
}

// <n_i> and C_ij of rho = X X^+: <X| O (x) 1 |X> / <X|X> with exact environments in
// double (one CTA per chain).  Lenv_{i+1} = sum_s B_s^+ Lenv_i B_s and
// Renv_i = sum_s B_s Renv_{i+1} B_s^+ over the four values s = 2n + k;
// <n_i> <X|X> = sum_{k} <B_{(1,k)}, Lenv_i B_{(1,k)} Renv_{i+1}>; for i < j
// C_ij <X|X> = sum_k <B_j(0,k), E B_j(1,k) Renv_{j+1}> with
// E = sum_k B_i(1,k)^+ Lenv_i B_i(0,k) carried through the sites between by
// sum_k [B(0,k)^+ E B(0,k) - B(1,k)^+ E B(1,k)] (the string).
struct PurEnvArgs {
  const void* B;
  const int* dims;
  int L, chi, slot, n_traj;
  double2* scratch;  // per CTA: Renv [L+1][chi^2], Lenv [L+1][chi^2], T, E, E2 [chi^2]
  long long stride;
  double* density;   // [n_traj][L]
  double2* corr;     // [n_traj][L][L] or nullptr
};

template <typename R>
__global__ void __launch_bounds__(LT_BLOCK) purified_env_kernel(PurEnvArgs a) {
  typedef typename CT<R>::T Tc;
  __shared__ double2 s_red[LT_BLOCK / 32];
  const int L = a.L, chi = a.chi, tid = threadIdx.x;
  const long long chi2 = (long long)chi * chi;
  double2* Renv = a.scratch + (long long)blockIdx.x * a.stride;
  double2* Lenv = Renv + (long long)(L + 1) * chi2;
  double2* T = Lenv + (long long)(L + 1) * chi2;
  double2* E = T + chi2;
  double2* E2 = E + chi2;
  for (int t = blockIdx.x; t < a.n_traj; t += gridDim.x) {
    const int* dm = a.dims + (long long)t * (L - 1);
    const Tc* Bt = reinterpret_cast<const Tc*>(a.B) + (long long)t * L * a.slot;
    if (tid == 0) {
      Renv[(long long)L * chi2] = make_double2(1.0, 0.0);
      Lenv[0] = make_double2(1.0, 0.0);
    }
    __syncthreads();
    for (int i = L - 1; i >= 0; --i) {
      const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
      const Tc* Bi = Bt + (long long)i * a.slot;
      for (int s = 0; s < 4; ++s) {
        zgemm(cl, cr, cr, Bi + s * cr, 4 * cr, false, Renv + (long long)(i + 1) * chi2, chi, false,
              T, chi, false, 1.0);
        __syncthreads();
        zgemm(cl, cl, cr, T, chi, false, Bi + s * cr, 4 * cr, true, Renv + (long long)i * chi2, chi,
              s > 0, 1.0);
        __syncthreads();
      }
    }
    const double nrm = Renv[0].x;
    for (int i = 0; i < L; ++i) {
      const int cl = i == 0 ? 1 : dm[i - 1], cr = i == L - 1 ? 1 : dm[i];
      const Tc* Bi = Bt + (long long)i * a.slot;
      double2 num = make_double2(0.0, 0.0);
      for (int k = 0; k < 2; ++k) {
        const Tc* B1 = Bi + (2 + k) * cr;
        zgemm(cl, cr, cl, Lenv + (long long)i * chi2, chi, false, B1, 4 * cr, false, T, chi, false, 1.0);
        __syncthreads();
        zgemm(cl, cr, cr, T, chi, false, Renv + (long long)(i + 1) * chi2, chi, false, E, chi, false, 1.0);
        __syncthreads();
        const double2 d = zdot(cl, cr, B1, 4 * cr, E, chi, s_red);
        num.x += d.x;
        num.y += d.y;
      }
      if (tid == 0) {
        a.density[(long long)t * L + i] = num.x / nrm;
        if (a.corr) a.corr[((long long)t * L + i) * L + i] = make_double2(num.x / nrm, 0.0);
      }
      for (int s = 0; s < 4; ++s) {
        zgemm(cl, cr, cl, Lenv + (long long)i * chi2, chi, false, Bi + s * cr, 4 * cr, false, T, chi,
              false, 1.0);
        __syncthreads();
        zgemm(cr, cr, cl, Bi + s * cr, 4 * cr, true, T, chi, false, Lenv + (long long)(i + 1) * chi2,
              chi, s > 0, 1.0);
        __syncthreads();
      }
    }
    if (a.corr) {
      for (int i = 0; i + 1 < L; ++i) {
        const int cl = i == 0 ? 1 : dm[i - 1], cr = dm[i];
        const Tc* Bi = Bt + (long long)i * a.slot;
        for (int k = 0; k < 2; ++k) {  // E = sum_k B(1,k)^+ Lenv_i B(0,k)
          zgemm(cl, cr, cl, Lenv + (long long)i * chi2, chi, false, Bi + k * cr, 4 * cr, false, T, chi,
                false, 1.0);
          __syncthreads();
          zgemm(cr, cr, cl, Bi + (2 + k) * cr, 4 * cr, true, T, chi, false, E, chi, k > 0, 1.0);
          __syncthreads();
        }
        for (int j = i + 1; j < L; ++j) {
          const int jl = dm[j - 1], jr = j == L - 1 ? 1 : dm[j];
          const Tc* Bj = Bt + (long long)j * a.slot;
          double2 num = make_double2(0.0, 0.0);
          for (int k = 0; k < 2; ++k) {
            zgemm(jl, jr, jl, E, chi, false, Bj + (2 + k) * jr, 4 * jr, false, T, chi, false, 1.0);
            __syncthreads();
            zgemm(jl, jr, jr, T, chi, false, Renv + (long long)(j + 1) * chi2, chi, false, E2, chi,
                  false, 1.0);
            __syncthreads();
            const double2 d = zdot(jl, jr, Bj + k * jr, 4 * jr, E2, chi, s_red);
            num.x += d.x;
            num.y += d.y;
          }
          if (tid == 0) {
            a.corr[((long long)t * L + i) * L + j] = make_double2(num.x / nrm, num.y / nrm);
            a.corr[((long long)t * L + j) * L + i] = make_double2(num.x / nrm, -num.y / nrm);
          }
          if (j + 1 < L) {  // E <- sum_k [B(0,k)^+ E B(0,k) - B(1,k)^+ E B(1,k)]
            for (int s = 0; s < 4; ++s) {
              zgemm(jl, jr, jl, E, chi, false, Bj + s * jr, 4 * jr, false, T, chi, false, 1.0);
              __syncthreads();
              zgemm(jr, jr, jl, Bj + s * jr, 4 * jr, true, T, chi, false, E2, chi, s > 0,
                    s < 2 ? 1.0 : -1.0);
              __syncthreads();
            }
            for (int x = tid; x < jr * jr; x += blockDim.x) {
              const int r = x / jr, c = x - r * jr;
              E[(long long)r * chi + c] = E2[(long long)r * chi + c];
            }
            __syncthreads();
          }
        }
      }
    }
    __syncthreads();
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

// Product state: |n_i> per site for pure states (d = 2); for the vectorised
// density matrix (d = 4) the site factor |n_i><n_i| has the one non-zero local
// index m = 2 n_i + n_i = 3 n_i (Eq. MPDO); for the purified density matrix
// X = |n> with Kraus index 0, s = 2 n_i.  occ_index is the index of n_i = 1.
template <typename R>
__global__ void init_state_kernel(typename CT<R>::T* B, double* lam, int* dims, double* trunc,
                                  int* evolve, int* channel, const uint8_t* occ, int n_traj,
                                  int L, int chi, int slot, int d, int occ_index) {
  const long long nt = (long long)n_traj * L;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nt;
       i += (long long)gridDim.x * blockDim.x) {
    const int traj = (int)(i / L), site = (int)(i - (long long)traj * L);
    typename CT<R>::T* s = B + i * slot;
    const int on = occ[site] ? occ_index : 0;
    for (int m = 0; m < d; ++m) s[m] = cmk<typename CT<R>::T>(m == on ? 1.0 : 0.0, 0.0);
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
size_t bond_smem_bytes(int chi, size_t celt, int d) {
  // Largest workspace of a task, in complex elements, over the three modes with
  // every dimension at chi and d physical values per site (mirrors the layout of
  // bond_update_kernel): the Jacobi matrix planar mcap x (npad + 2), V_k^+
  // k x (nJ + 1), plus the staging of B_{b+1} (mode 0) or of the new site
  // tensors (mode 2).
  const bool single = celt == sizeof(float2);
  const size_t epp = 4;  // element pairs per lane of the row-pair Jacobi
  auto npad_of = [&](size_t m, size_t n) {
    size_t gs = 1;
    while (gs * 2 * epp < n && gs < 32) gs <<= 1;
    const bool blk = single && m >= 32 && n >= 64 && n <= LT_REG_DIM;
    const bool wide = single && m >= 32 && n > LT_REG_DIM;
    const size_t span = 2 * epp * gs;
    return blk ? (n <= 64 ? (size_t)64 : (size_t)128)
               : wide ? 128 * ((n + 127) / 128) : span * ((n + span - 1) / span);
  };
  auto mp_of = [&](size_t m, size_t n) {
    return (single && m >= 32 && n >= 64) ? ((m + 7) & ~(size_t)7) : m + (m & 1);
  };
  const size_t c2 = (size_t)d * chi, c1 = chi;
  // the LQ reflectors of an m x n matrix (r = min(m, n) of n - j entries) share
  // the region of V^+ until V^+ is assembled
  auto refl = [](size_t r, size_t n) { return r * n - r * (r - 1) / 2; };
  auto mx = [](size_t a, size_t b) { return a > b ? a : b; };
  // mode 0: theta d chi x d chi, V^+ chi x (d chi+1), B_{b+1} staged in V^+'s region
  const size_t need0 = mp_of(c2, c2) * (npad_of(c2, c2) + 2) +
                       mx(mx(c1 * (c2 + 1), c1 * c2), refl(c2, c2));
  // mode 1: B_{b+1} chi x d chi, later theta~ d chi x d chi in the same planes
  const size_t mcap1 = mp_of(c1, c2) > c2 ? mp_of(c1, c2) : c2;
  const size_t need1 = mcap1 * (npad_of(c1, c2) + 2) + mx(c1 * (c2 + 1), refl(c1, c2));
  // mode 2: Lambda B_b d chi x chi, V^+ chi x (chi+1), staged tensors chi x d chi
  const size_t need2 =
      mp_of(c2, c1) * (npad_of(c2, c1) + 2) + mx(c1 * (c1 + 1) + c1 * c2, refl(c1, c1));
  size_t need = need0 > need1 ? need0 : need1;
  need = need > need2 ? need : need2;
  size_t bytes = need * celt;
  if (single && d == 2) {
    // digit planes of the tensor-core theta (inner dimension up to 64)
    const int kp = ((chi < 64 ? chi : 64) + 15) & ~15;
    const size_t tc = (size_t)tcg::smem_bytes(kp);
    if (tc > bytes) bytes = tc;
  }
  return bytes;
}

size_t env_scratch_elems(int L, int chi) { return ((size_t)L + 1 + 7) * (size_t)chi * chi; }

// CTAs of the environment kernels: each holds (L + 8) chi^2 elements of scratch,
// so their number is capped to keep it within LT_ENV_SCRATCH_BYTES (one CTA per SM
// at least)
long long env_grid_cap(int L, int chi, size_t celt, int num_sms) {
  const long long per = (long long)(env_scratch_elems(L, chi) * celt);
  const long long cap = (long long)LT_ENV_SCRATCH_BYTES / (per > 0 ? per : 1);
  return cap > num_sms ? cap : num_sms;
}

template <typename R, int D>
static cudaError_t launch_bond_t(lt_ctx_s* c, const int* trajs, const int* n_trajs, int bond0,
                                 int nb, const double2* gates, int mode) {
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
  a.mode = mode;
  a.ws_elems = (long long)(bond_smem_bytes(c->chi, c->celt, D) / c->celt);
  a.L = c->L;
  a.chi = c->chi;
  a.slot = c->slot;
  a.cut = c->cut;
  a.err = c->err_dev;
  a.smem_elems = (long long)(c->bond_smem / c->celt);
  a.scratch = reinterpret_cast<typename CT<R>::T*>(c->bond_scratch);
  a.scratch_stride = c->bond_scratch_stride;
  a.use_tc = sizeof(R) == 4 && D == 2 && mode == 0 && c->theta_tc;
  a.max_sweeps = c->max_sweeps;
  a.tol = c->jacobi_tol;
  a.sweep_hist = c->sweep_hist;
  a.counters = c->counters;
  a.keep_norm = (c->method == LT_QSD || c->method == LT_PURIFIED) && mode == 0;
  a.logw = c->method == LT_QSD && mode == 2 ? c->logw : nullptr;
  a.multiplet = c->method == LT_MPDO ? (c->prec == LT_MIXED ? 1e-5 : 1e-9) : 0.0;
  if constexpr (sizeof(R) == 4 && D == 2) {
    if (a.use_tc) {
      const int kp = ((c->chi < 64 ? c->chi : 64) + 15) & ~15;
      theta_tc_kernel<<<c->num_sms, 512, tcg::smem_bytes(kp), c->stream>>>(a);
      c->launches++;
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  // A launch of few tasks that may need global scratch (single precision, mode 0) gives
  // each task a cluster of C CTAs, which share its Jacobi: the largest C for which every
  // task's cluster can be resident at once.
  a.cluster = 1;
  a.cl_state = c->bond_cl_state;
  if constexpr (sizeof(R) == 4) {
    const long long ntask = (long long)c->n_traj * nb;
    int C = 1;
    if (mode == 0 && c->bond_scratch_stride > 0 && c->bond_cl_state)
      for (int cs = 8; cs >= 2 && C == 1; cs >>= 1)
        if (c->bond_ncl[cs] >= ntask) C = cs;
    if (C == 1) {
      bond_update_kernel<R, D, false><<<c->bond_grid, BondShape<R>::NT, c->bond_smem,
                                        c->stream>>>(a);
      c->launches++;
      return cudaGetLastError();
    }
    a.cluster = C;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * ntask));
    cfg.blockDim = dim3(BondShape<R>::NT);
    cfg.dynamicSmemBytes = c->bond_smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, bond_update_kernel<R, D, true>, a);
    c->launches++;
    c->cluster_launches++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  } else {
    bond_update_kernel<R, D, false><<<c->bond_grid, BondShape<R>::NT, c->bond_smem,
                                      c->stream>>>(a);
    c->launches++;
    return cudaGetLastError();
  }
}

cudaError_t launch_bond(lt_ctx_s* c, const int* trajs, const int* n_trajs, int bond0, int nb,
                        const double2* gates, int mode) {
  if (c->d == 4) {
    if (c->prec == LT_MIXED) return launch_bond_t<float, 4>(c, trajs, n_trajs, bond0, nb, gates, mode);
    return launch_bond_t<double, 4>(c, trajs, n_trajs, bond0, nb, gates, mode);
  }
  if (c->prec == LT_MIXED) return launch_bond_t<float, 2>(c, trajs, n_trajs, bond0, nb, gates, mode);
  return launch_bond_t<double, 2>(c, trajs, n_trajs, bond0, nb, gates, mode);
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
  a.step_dev = c->use_step_dev ? c->step_dev : nullptr;
  a.err = c->err_dev;
  a.corr = c->corr;
  return a;
}

cudaError_t launch_env(lt_ctx_s* c, int decide, long long step, const int* replay) {
  EnvArgs a = env_args(c);
  a.decide = decide;
  a.step = step;
  a.replay = replay;
  if (c->prec == LT_MIXED) env_tiled_kernel<float><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  else env_tiled_kernel<double><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
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

size_t mpdo_scratch_bytes(int L, int chi) { return 2 * ((size_t)L + 1) * (size_t)chi * sizeof(double2); }

cudaError_t launch_mpdo_trace(lt_ctx_s* c, bool corr) {
  MpdoArgs a;
  a.B = c->B;
  a.dims = c->dims;
  a.L = c->L;
  a.chi = c->chi;
  a.slot = c->slot;
  a.n_traj = c->n_traj;
  a.scratch = reinterpret_cast<double2*>(c->env_scratch);
  a.stride = (long long)(c->env_scratch_stride * c->celt / sizeof(double2));
  a.density = c->density;
  a.corr = corr ? c->corr : nullptr;
  if (c->prec == LT_MIXED) mpdo_trace_kernel<float><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  else mpdo_trace_kernel<double><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

size_t purified_scratch_bytes(int L, int chi) {
  return (2 * (size_t)L + 5) * (size_t)chi * chi * sizeof(double2);
}

cudaError_t launch_kraus(lt_ctx_s* c) {
  KrausArgs a;
  a.B = c->B;
  a.lam = c->lam;
  a.dims = c->dims;
  a.L = c->L;
  a.chi = c->chi;
  a.slot = c->slot;
  a.n_traj = c->n_traj;
  a.gam = c->gam;
  a.dt = c->dt;
  const long long ntask = (long long)c->n_traj * c->L;
  const int grid = (int)(ntask < 8LL * c->num_sms ? ntask : 8LL * c->num_sms);
  if (c->prec == LT_MIXED) kraus_step_kernel<float><<<grid, LT_BLOCK, 0, c->stream>>>(a);
  else kraus_step_kernel<double><<<grid, LT_BLOCK, 0, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_purified_env(lt_ctx_s* c, bool corr) {
  PurEnvArgs a;
  a.B = c->B;
  a.dims = c->dims;
  a.L = c->L;
  a.chi = c->chi;
  a.slot = c->slot;
  a.n_traj = c->n_traj;
  a.scratch = reinterpret_cast<double2*>(c->env_scratch);
  a.stride = (long long)(c->env_scratch_stride * c->celt / sizeof(double2));
  a.density = c->density;
  a.corr = corr ? c->corr : nullptr;
  if (c->prec == LT_MIXED) purified_env_kernel<float><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  else purified_env_kernel<double><<<c->env_grid, LT_BLOCK, 0, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

// the step counter of a captured time step advances on the device
__global__ void step_advance_kernel(long long* step_dev) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step_dev += 1;
}

cudaError_t launch_step_advance(lt_ctx_s* c) {
  step_advance_kernel<<<1, 32, 0, c->stream>>>(c->step_dev);
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
                                                           out_sem, c->method == LT_QSD ? c->logw : nullptr);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_reduce_corr(lt_ctx_s* c, double* out) {
  const int M = c->L * c->L;
  reduce_mean_c_kernel<<<M < 4096 ? M : 4096, LT_BLOCK, 0, c->stream>>>(
      c->corr, c->n_traj, M, out, c->method == LT_QSD ? c->logw : nullptr);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_qsd_noise(lt_ctx_s* c, long long step) {
  const long long ntask = (long long)c->n_traj * c->L;
  const int grid = (int)(ntask < (long long)c->num_sms * 16 ? ntask : (long long)c->num_sms * 16);
  if (c->prec == LT_MIXED)
    qsd_noise_kernel<float><<<grid, 128, 0, c->stream>>>(reinterpret_cast<float2*>(c->B), c->dims, c->L,
                                                          c->slot, c->n_traj, c->traj_offset, step,
                                                          c->use_step_dev ? c->step_dev : nullptr,
                                                          c->seed, c->gam, c->dt);
  else
    qsd_noise_kernel<double><<<grid, 128, 0, c->stream>>>(reinterpret_cast<double2*>(c->B), c->dims,
                                                           c->L, c->slot, c->n_traj, c->traj_offset,
                                                           step, c->use_step_dev ? c->step_dev : nullptr,
                                                           c->seed, c->gam, c->dt);
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
  const int occ_index = c->d == 2 ? 1 : (c->method == LT_MPDO ? 3 : 2);
  if (c->prec == LT_MIXED)
    init_state_kernel<float><<<grid_for(nt, 256), 256, 0, c->stream>>>(
        reinterpret_cast<float2*>(c->B), c->lam, c->dims, c->trunc, c->evolve, c->channel, occ_dev,
        c->n_traj, c->L, c->chi, c->slot, c->d, occ_index);
  else
    init_state_kernel<double><<<grid_for(nt, 256), 256, 0, c->stream>>>(
        reinterpret_cast<double2*>(c->B), c->lam, c->dims, c->trunc, c->evolve, c->channel, occ_dev,
        c->n_traj, c->L, c->chi, c->slot, c->d, occ_index);
  c->launches++;
  return cudaGetLastError();
}

// The dynamic shared-memory ceiling of the bond kernel: 200 KB, or less when the kernel's
// static shared memory leaves less of the per-block opt-in maximum
template <typename R, int D>
static cudaError_t bond_smem_limit(int device, size_t* limit) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, bond_update_kernel<R, D, false>);
  if (e != cudaSuccess) return e;
  size_t stat = fa.sharedSizeBytes;
  if constexpr (sizeof(R) == 4) {
    e = cudaFuncGetAttributes(&fa, bond_update_kernel<R, D, true>);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes > stat) stat = fa.sharedSizeBytes;
  }
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  const size_t room = (size_t)optin > stat ? (size_t)optin - stat : 0;
  *limit = room < (size_t)200 * 1024 ? room : (size_t)200 * 1024;
  return cudaSuccess;
}

template <typename R, int D>
static cudaError_t bond_attributes(size_t limit, size_t smem, int* occ) {
  cudaError_t e = cudaFuncSetAttribute(bond_update_kernel<R, D, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  if (e != cudaSuccess) return e;
  if constexpr (sizeof(R) == 4) {
    e = cudaFuncSetAttribute(bond_update_kernel<R, D, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, bond_update_kernel<R, D, false>,
                                                       BondShape<R>::NT, smem);
}

// How many clusters of 2, 4 and 8 CTAs of the cluster instance fit on the device at
// once with this context's shared memory (0 where none does, or the query fails).
template <int D>
static void bond_clusters(lt_ctx_s* c) {
  for (int cs = 2; cs <= 8; cs <<= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(cs * (c->num_sms / cs)));
    cfg.blockDim = dim3(BondShape<float>::NT);
    cfg.dynamicSmemBytes = c->bond_smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, bond_update_kernel<float, D, true>, &cfg) !=
        cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    c->bond_ncl[cs] = n;
  }
}

// attribute setup and occupancy for the bond kernel (called once per context)
cudaError_t configure_bond(lt_ctx_s* c) {
  const size_t need = bond_smem_bytes(c->chi, c->celt, c->d);
  size_t limit = 0;
  cudaError_t el;
  if (c->d == 4)
    el = c->prec == LT_MIXED ? bond_smem_limit<float, 4>(c->device, &limit)
                             : bond_smem_limit<double, 4>(c->device, &limit);
  else
    el = c->prec == LT_MIXED ? bond_smem_limit<float, 2>(c->device, &limit)
                             : bond_smem_limit<double, 2>(c->device, &limit);
  if (el != cudaSuccess) return el;
  // every launch gets shared memory for the tasks that fit it, and global scratch for the
  // larger ones when the largest task does not fit; except in double precision, whose
  // tasks at such sizes nearly all work in scratch and run faster with the whole L1
  c->bond_smem = need <= limit ? need : (c->prec == LT_MIXED ? limit : 0);
  cudaError_t e;
  int occ = 0;
  // The dynamic shared-memory ceiling is a property of the kernel, shared by
  // every context in the process: it is raised to the most any context may
  // request (limit), never lowered to one context's need, so contexts of
  // different chi_max can live side by side.
  if (c->d == 4)
    e = c->prec == LT_MIXED ? bond_attributes<float, 4>(limit, c->bond_smem, &occ)
                            : bond_attributes<double, 4>(limit, c->bond_smem, &occ);
  else
    e = c->prec == LT_MIXED ? bond_attributes<float, 2>(limit, c->bond_smem, &occ)
                            : bond_attributes<double, 2>(limit, c->bond_smem, &occ);
  if (e != cudaSuccess) return e;
  if (c->prec == LT_MIXED && c->d == 2) {
    e = cudaFuncSetAttribute(theta_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tcg::smem_bytes(64));
    if (e != cudaSuccess) return e;
  }
  if (occ < 1) occ = 1;
  c->bond_grid = occ * c->num_sms;
  c->bond_scratch_stride = need <= limit ? 0 : (long long)(need / c->celt);
  if (c->prec == LT_MIXED && c->bond_scratch_stride > 0) {
    if (c->d == 4)
      bond_clusters<4>(c);
    else
      bond_clusters<2>(c);
  }
  return cudaSuccess;
}

// ---- allocation-free density entry point -------------------------------------------------
// Scratch of lt_measure_density_noalloc: a file-scope device array, so that the
// call itself allocates nothing.  Every GPU that loads the library holds it until
// the process exits.
#define LT_NOALLOC_SCRATCH_BYTES (32ull << 20)
static __device__ __align__(256) unsigned char lt_noalloc_scratch[LT_NOALLOC_SCRATCH_BYTES];


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
  // the host-side name of the array is only a stand-in: the kernel needs the
  // device address on the current device, looked up on every call (no
  // allocation), so nothing cached outlives a device reset
  void* scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, lt_noalloc_scratch) != cudaSuccess || !scratch)
    return LT_ERR_CUDA;
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
  if (precision == LT_MIXED) env_tiled_kernel<float, false><<<(int)grid, LT_BLOCK, 0, st>>>(a);
  else env_tiled_kernel<double, false><<<(int)grid, LT_BLOCK, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}

// resident environment CTAs: as many as fit on the device (their workspace
// is global scratch), at most one per trajectory
int env_grid(lt_ctx_s* c) {
  int occ = 0;
  cudaError_t e = c->prec == LT_MIXED
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, env_tiled_kernel<float>, LT_BLOCK, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, env_tiled_kernel<double>, LT_BLOCK, 0);
  if (e != cudaSuccess || occ < 1) occ = 2;
  if (occ > 8) occ = 8;
  if (c->env_occ > 0 && c->env_occ < occ) occ = c->env_occ;  // the schedule's CTAs per SM
  long long g = (long long)occ * c->num_sms;
  const long long cap = env_grid_cap(c->L, c->chi, c->celt, c->num_sms);
  if (g > cap) g = cap;
  return (int)(g < c->n_traj ? g : c->n_traj);
}

