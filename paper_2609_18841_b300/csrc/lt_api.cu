// Host side of the lindtebd C ABI: configuration checks, context memory,
// two-site gate construction and the order of kernel launches of a time step.
#include <complex>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <new>

#include "lt_internal.cuh"
#include "lt_schedule_table.h"

// the tuned schedule of (values per site, precision, chi_max): the entry with the smallest
// tabulated chi_max at or above the context's
static void lt_schedule_lookup(int d, int precision, int chi, int* path, int* env) {
  const LtSchedule* best = nullptr;
  for (const LtSchedule& e : kLtSchedules) {
    if (e.d != d || e.precision != precision || e.chi_max < chi) continue;
    if (!best || e.chi_max < best->chi_max) best = &e;
  }
  if (!best) return;
  if (best->theta_path) *path = best->theta_path;
  if (best->env_ctas_per_sm) *env = best->env_ctas_per_sm;
}

cudaError_t configure_bond(lt_ctx_s* c);
int env_grid(lt_ctx_s* c);

namespace {

typedef std::complex<double> cd;

#define LT_CK(call)                                                               \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return fail(c, LT_ERR_CUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

lt_status fail(lt_ctx_s* c, lt_status s, const char* what, const char* why) {
  if (c) {
    c->last_error = std::string(what) + ": " + why;
    if (s == LT_ERR_NUMERICAL || s == LT_ERR_TIMEOUT || s == LT_ERR_CUDA) c->poisoned = true;
  }
  return s;
}

// 4x4 complex matrix helpers (row-major)
struct M4 {
  cd v[16];
};
M4 mmul(const M4& a, const M4& b) {
  M4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd s = 0;
      for (int k = 0; k < 4; ++k) s += a.v[i * 4 + k] * b.v[k * 4 + j];
      r.v[i * 4 + j] = s;
    }
  return r;
}

// exp(A) by scaling and squaring of a Taylor series (Sec. 2.3: the two-site
// exponential "by series expansion"): halve A until its 1-norm is below 1/2,
// sum the series until the terms drop below 1e-18, square back.
M4 expm4(M4 A) {
  double nrm = 0.0;
  for (int j = 0; j < 4; ++j) {
    double col = 0.0;
    for (int i = 0; i < 4; ++i) col += std::abs(A.v[i * 4 + j]);
    nrm = col > nrm ? col : nrm;
  }
  int s = 0;
  while (nrm > 0.5) {
    nrm *= 0.5;
    ++s;
  }
  const double scale = std::ldexp(1.0, -s);
  for (auto& x : A.v) x *= scale;
  M4 E, term;
  for (int i = 0; i < 16; ++i) E.v[i] = term.v[i] = (i % 5 == 0) ? 1.0 : 0.0;
  for (int n = 1; n < 40; ++n) {
    term = mmul(term, A);
    double mx = 0.0;
    for (auto& x : term.v) {
      x /= (double)n;
      mx = std::abs(x) > mx ? std::abs(x) : mx;
    }
    for (int i = 0; i < 16; ++i) E.v[i] += term.v[i];
    if (mx < 1e-18) break;
  }
  for (int k = 0; k < s; ++k) E = mmul(E, E);
  return E;
}

// G_b(tau) = exp(-i tau h_b^eff), h_b^eff = -J (s+ s- + s- s+)
//   - (i/2) (w_l K_b(s_b) + w_r K_{b+1}(s_{b+1})),  K(s) = loss s + gain (1-s) + deph s,
// w = 1 for a chain end, 1/2 in the bulk (Eq. EffHamiltonian split per bond).
void build_gates(const lt_ctx_s* c, double tau, std::vector<double2>& out) {
  const int L = c->L;
  out.assign((size_t)(L - 1) * 16, make_double2(0, 0));
  for (int b = 0; b < L - 1; ++b) {
    const double wl = b == 0 ? 1.0 : 0.5, wr = b + 1 == L - 1 ? 1.0 : 0.5;
    M4 h;
    for (auto& x : h.v) x = 0;
    h.v[2 * 4 + 1] = -c->J;  // |10><01|
    h.v[1 * 4 + 2] = -c->J;  // |01><10|
    for (int sb = 0; sb < 2; ++sb)
      for (int sc = 0; sc < 2; ++sc) {
        const double Kl = c->gl[b] * sb + c->gg[b] * (1 - sb) + c->gd[b] * sb;
        const double Kr = c->gl[b + 1] * sc + c->gg[b + 1] * (1 - sc) + c->gd[b + 1] * sc;
        h.v[(sb * 2 + sc) * 5] += cd(0.0, -0.5 * (wl * Kl + wr * Kr));
      }
    M4 A;
    for (int i = 0; i < 16; ++i) A.v[i] = cd(0.0, -tau) * h.v[i];
    const M4 G = expm4(A);
    for (int i = 0; i < 16; ++i) out[(size_t)b * 16 + i] = make_double2(G.v[i].real(), G.v[i].imag());
  }
}

// ---- Liouvillian gates of the vectorised density matrix (Sec. 3.1) -----------------------
// |rho>> = sum_ij rho_ij |i> (x) |j> (Eq. Choi) turns rho -> A rho B into a matrix;
// on one bond, over the local indices m = 2n + n' of its two sites (Eq. MPDO),
// its entry [(m_b, m_{b+1}), (k_b, k_{b+1})] is A[(n_b n_{b+1}), (k_b k_{b+1})]
// B[(k'_b k'_{b+1}), (n'_b n'_{b+1})].  The bond generator is
//   Lv_b = -i [h_b, .] + w_l D_b + w_r D_{b+1},
//   D_i rho = sum_k gamma_k (L_k rho L_k^+ - 1/2 L_k^+L_k rho - 1/2 rho L_k^+L_k),
// which in (x) form carries L (x) conj(L) and 1 (x) h^T (Eq. Liouvillian read
// with the conjugate and transpose the map produces).  Loss sigma-, gain sigma+,
// dephasing n; the weights split the site terms as for the trajectory gates.
// A fermionic loss or gain is accepted on the chain ends only, where its string
// acts as the total parity, which commutes with every state reached from a
// product state, so the local operator gives the same evolution.
typedef std::vector<cd> Mat;

Mat mat_mul(const Mat& a, const Mat& b, int n) {
  Mat r((size_t)n * n, cd(0.0, 0.0));
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const cd x = a[(size_t)i * n + k];
      if (x == cd(0.0, 0.0)) continue;
      for (int j = 0; j < n; ++j) r[(size_t)i * n + j] += x * b[(size_t)k * n + j];
    }
  return r;
}

// exp(A) for an n x n matrix, the same scaling-and-squaring Taylor rule as expm4
Mat expm_n(Mat A, int n) {
  double nrm = 0.0;
  for (int j = 0; j < n; ++j) {
    double col = 0.0;
    for (int i = 0; i < n; ++i) col += std::abs(A[(size_t)i * n + j]);
    nrm = col > nrm ? col : nrm;
  }
  int s = 0;
  while (nrm > 0.5) {
    nrm *= 0.5;
    ++s;
  }
  const double scale = std::ldexp(1.0, -s);
  for (auto& x : A) x *= scale;
  Mat E((size_t)n * n, cd(0.0, 0.0)), term;
  for (int i = 0; i < n; ++i) E[(size_t)i * n + i] = 1.0;
  term = E;
  for (int k = 1; k < 40; ++k) {
    term = mat_mul(term, A, n);
    double mx = 0.0;
    for (auto& x : term) {
      x /= (double)k;
      mx = std::abs(x) > mx ? std::abs(x) : mx;
    }
    for (size_t i = 0; i < E.size(); ++i) E[i] += term[i];
    if (mx < 1e-18) break;
  }
  for (int k = 0; k < s; ++k) E = mat_mul(E, E, n);
  return E;
}

// S += coef * (rho -> A rho B) on the 16-dimensional two-site space
void add_superop(Mat& S, const M4& A, const M4& B, cd coef) {
  for (int nb = 0; nb < 2; ++nb)
    for (int pb = 0; pb < 2; ++pb)
      for (int nc = 0; nc < 2; ++nc)
        for (int pc = 0; pc < 2; ++pc) {
          const int row = (2 * nb + pb) * 4 + (2 * nc + pc);
          for (int kb = 0; kb < 2; ++kb)
            for (int qb = 0; qb < 2; ++qb)
              for (int kc = 0; kc < 2; ++kc)
                for (int qc = 0; qc < 2; ++qc) {
                  const int col = (2 * kb + qb) * 4 + (2 * kc + qc);
                  S[(size_t)row * 16 + col] += coef * A.v[(nb * 2 + nc) * 4 + (kb * 2 + kc)] *
                                               B.v[(qb * 2 + qc) * 4 + (pb * 2 + pc)];
                }
        }
}

// one-site 2x2 operator on the left (side 0) or right (side 1) site of a bond
M4 on_site(const cd op[4], int side) {
  M4 r;
  for (auto& x : r.v) x = 0;
  for (int sb = 0; sb < 2; ++sb)
    for (int sc = 0; sc < 2; ++sc)
      for (int tb = 0; tb < 2; ++tb)
        for (int tc = 0; tc < 2; ++tc) {
          cd v = side == 0 ? (sc == tc ? op[sb * 2 + tb] : cd(0.0, 0.0))
                           : (sb == tb ? op[sc * 2 + tc] : cd(0.0, 0.0));
          r.v[(sb * 2 + sc) * 4 + (tb * 2 + tc)] = v;
        }
  return r;
}

M4 adjoint(const M4& a) {
  M4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r.v[i * 4 + j] = std::conj(a.v[j * 4 + i]);
  return r;
}

void build_liouvillian_gates(const lt_ctx_s* c, double tau, std::vector<double2>& out) {
  const int L = c->L;
  out.assign((size_t)(L - 1) * 256, make_double2(0, 0));
  M4 one, h;
  for (int i = 0; i < 16; ++i) {
    one.v[i] = (i % 5 == 0) ? 1.0 : 0.0;
    h.v[i] = 0.0;
  }
  h.v[2 * 4 + 1] = -c->J;  // |10><01|
  h.v[1 * 4 + 2] = -c->J;  // |01><10|
  M4 mih, pih;
  for (int i = 0; i < 16; ++i) {
    mih.v[i] = cd(0.0, -1.0) * h.v[i];
    pih.v[i] = cd(0.0, 1.0) * h.v[i];
  }
  const cd sminus[4] = {0.0, 1.0, 0.0, 0.0}, splus[4] = {0.0, 0.0, 1.0, 0.0},
           number[4] = {0.0, 0.0, 0.0, 1.0};
  for (int b = 0; b < L - 1; ++b) {
    Mat S(256, cd(0.0, 0.0));
    add_superop(S, mih, one, 1.0);  // -i h rho
    add_superop(S, one, pih, 1.0);  // +i rho h
    const double w[2] = {b == 0 ? 1.0 : 0.5, b + 1 == L - 1 ? 1.0 : 0.5};
    for (int side = 0; side < 2; ++side) {
      const int site = b + side;
      const double g[3] = {c->gl[site], c->gg[site], c->gd[site]};
      const cd* ops[3] = {sminus, splus, number};
      for (int k = 0; k < 3; ++k) {
        if (!(g[k] > 0.0)) continue;
        const M4 Lk = on_site(ops[k], side), Ld = adjoint(Lk);
        const M4 LdL = mmul(Ld, Lk);
        const double wg = w[side] * g[k];
        add_superop(S, Lk, Ld, wg);
        add_superop(S, LdL, one, -0.5 * wg);
        add_superop(S, one, LdL, -0.5 * wg);
      }
    }
    for (auto& x : S) x *= tau;
    const Mat G = expm_n(S, 16);
    for (int i = 0; i < 256; ++i)
      out[(size_t)b * 256 + i] = make_double2(G[i].real(), G[i].imag());
  }
}

// Purified density matrix (Sec. 3.2, Eq. ThetaPurified): the effective-Hamiltonian
// gate over the physical indices times the identity over the Kraus indices, on
// s = 2n + k: F[(s_b, s_{b+1}), (t_b, t_{b+1})] = G[(n_b n_{b+1}), (m_b m_{b+1})]
// delta(k_b, k'_b) delta(k_{b+1}, k'_{b+1}).
void build_purified_gates(const lt_ctx_s* c, double tau, std::vector<double2>& out) {
  std::vector<double2> g4;
  build_gates(c, tau, g4);
  const int L = c->L;
  out.assign((size_t)(L - 1) * 256, make_double2(0, 0));
  for (int b = 0; b < L - 1; ++b)
    for (int nb = 0; nb < 2; ++nb)
      for (int kb = 0; kb < 2; ++kb)
        for (int nc = 0; nc < 2; ++nc)
          for (int kc = 0; kc < 2; ++kc)
            for (int mb = 0; mb < 2; ++mb)
              for (int mc = 0; mc < 2; ++mc) {
                const int row = (2 * nb + kb) * 4 + (2 * nc + kc);
                const int col = (2 * mb + kb) * 4 + (2 * mc + kc);
                out[(size_t)b * 256 + row * 16 + col] = g4[(size_t)b * 16 + (nb * 2 + nc) * 4 + (mb * 2 + mc)];
              }
}

lt_status gate_ptr(lt_ctx_s* c, double tau, const double2** out) {
  const size_t per = (size_t)(c->L - 1) * c->d * c->d * c->d * c->d;
  for (size_t i = 0; i < c->gate_taus.size(); ++i)
    if (c->gate_taus[i] == tau) {
      *out = c->gates + i * per;
      return LT_OK;
    }
  if (c->gate_taus.size() >= 8) return fail(c, LT_ERR_ARG, "lt_apply_layer", "more than 8 distinct tau values");
  std::vector<double2> h;
  if (c->method == LT_MPDO) build_liouvillian_gates(c, tau, h);
  else if (c->method == LT_PURIFIED) build_purified_gates(c, tau, h);
  else build_gates(c, tau, h);
  const size_t i = c->gate_taus.size();
  double2* dst = c->gates + i * per;
  LT_CK(cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaStreamSynchronize(c->stream));
  c->gate_taus.push_back(tau);
  *out = dst;
  return LT_OK;
}

lt_status check_device_error(lt_ctx_s* c) {
  int err = 0;
  LT_CK(cudaMemcpyAsync(&err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LT_CK(cudaStreamSynchronize(c->stream));
  if (err & LT_EBIT_THETA_ZERO) return fail(c, LT_ERR_NUMERICAL, "bond update", "theta vanished");
  if (err & LT_EBIT_PROB)
    return fail(c, LT_ERR_NUMERICAL, "jump decision", "jump probability per step >= 0.5; reduce dt");
  if (err & LT_EBIT_WORKSPACE)
    return fail(c, LT_ERR_NUMERICAL, "bond update", "a task exceeded its workspace");
  if (err & LT_EBIT_TIMEOUT)
    return fail(c, LT_ERR_TIMEOUT, "bond update", "a bounded wait on the tensor cores ran out");
  if (err & LT_EBIT_BADARG) {
    c->last_error = "replayed channel out of range";
    int zero = 0;
    LT_CK(cudaMemcpyAsync(c->err_dev, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    return LT_ERR_ARG;
  }
  return LT_OK;
}

template <typename T> lt_status dalloc(lt_ctx_s* c, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, LT_ERR_OOM, "cudaMalloc", cudaGetErrorString(e));
  }
  c->dev_bytes += n * sizeof(T);
  return LT_OK;
}

void free_all(lt_ctx_s* c) {
  void* ptrs[] = {c->B, c->lam, c->dims, c->trunc, c->evolve, c->channel, c->replay,
                  c->active_list, c->jumped_list, c->counts, c->density, c->logw, c->rates, c->gam,
                  c->err_dev, c->sweep_hist, c->counters, c->gates, c->bond_scratch, c->bond_cl_state,
                  c->env_scratch,
                  c->corr, c->red, c->step_dev};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

lt_status guard(lt_ctx_s* c) {
  if (!c) return LT_ERR_ARG;
  if (c->poisoned) return LT_ERR_STATE;
  return LT_OK;
}

}  // namespace

extern "C" {

const char* lt_status_str(lt_status s) {
  switch (s) {
    case LT_OK: return "ok";
    case LT_ERR_ARG: return "invalid argument";
    case LT_ERR_OOM: return "device out of memory";
    case LT_ERR_CUDA: return "CUDA error";
    case LT_ERR_NUMERICAL: return "numerical failure";
    case LT_ERR_TIMEOUT: return "device wait timed out";
    case LT_ERR_STATE: return "context poisoned by an earlier error";
    case LT_ERR_UNSUPPORTED: return "unsupported method or option";
  }
  return "unknown status";
}

const char* lt_last_error(lt_ctx ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int64_t lt_launch_count(lt_ctx ctx) { return ctx ? ctx->launches : 0; }

int64_t lt_cluster_launches(lt_ctx ctx) { return ctx ? ctx->cluster_launches : 0; }

lt_status lt_get_sweep_histogram(lt_ctx c, int32_t* hist, int32_t clear) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (hist) LT_CK(cudaMemcpyAsync(hist, c->sweep_hist, 64 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (clear) LT_CK(cudaMemsetAsync(c->sweep_hist, 0, 64 * sizeof(int), c->stream));
  LT_CK(cudaStreamSynchronize(c->stream));
  return LT_OK;
}

lt_status lt_get_counters(lt_ctx c, uint64_t* out, int32_t clear) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (out)
    LT_CK(cudaMemcpyAsync(out, c->counters, LT_NCOUNTERS * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, c->stream));
  if (clear) LT_CK(cudaMemsetAsync(c->counters, 0, LT_NCOUNTERS * sizeof(unsigned long long), c->stream));
  LT_CK(cudaStreamSynchronize(c->stream));
  return LT_OK;
}

void* lt_stream(lt_ctx ctx) { return ctx ? (void*)ctx->stream : nullptr; }

int64_t lt_get_step(lt_ctx ctx) { return ctx ? ctx->step_counter : 0; }

lt_status lt_create(const lt_config* cfg, void* stream, lt_ctx* out) {
  if (!out) return LT_ERR_ARG;
  *out = nullptr;
  if (!cfg) return LT_ERR_ARG;
  if (cfg->method != LT_TRAJ && cfg->method != LT_QSD && cfg->method != LT_MPDO &&
      cfg->method != LT_PURIFIED)
    return LT_ERR_UNSUPPORTED;
  // theta of the vectorised and of the purified density matrix is 4 chi x 4 chi:
  // the two-site update holds sides up to LT_MAX_DIM; the purified form is built
  // for a Kraus dimension of 2 (0 selects it)
  const bool four = cfg->method == LT_MPDO || cfg->method == LT_PURIFIED;
  if (four && cfg->chi_max > LT_MAX_DIM / 4 && cfg->chi_max <= LT_MAX_CHI) return LT_ERR_UNSUPPORTED;
  if (cfg->method == LT_PURIFIED && cfg->kraus_dim != 0 && cfg->kraus_dim != 2)
    return LT_ERR_UNSUPPORTED;
  if (cfg->L < 2 || cfg->L > 1024 || cfg->chi_max < 1 || cfg->chi_max > LT_MAX_CHI ||
      cfg->n_traj < 1 || (cfg->precision != LT_FP64 && cfg->precision != LT_MIXED) ||
      (cfg->trotter_order != 1 && cfg->trotter_order != 2) || !(cfg->dt > 0.0) ||
      !(cfg->svd_cut >= 0.0) || cfg->max_sweeps < 0 || cfg->max_sweeps > 1000 ||
      !(cfg->jacobi_tol >= 0.0 && cfg->jacobi_tol < 1.0) || cfg->init < LT_INIT_VACUUM || cfg->init > LT_INIT_PRODUCT ||
      cfg->theta_path < 0 || cfg->theta_path > 2 ||
      cfg->env_ctas_per_sm < 0 || cfg->env_ctas_per_sm > 8 ||
      (cfg->init == LT_INIT_PRODUCT && !cfg->product_occ) || !std::isfinite(cfg->J))
    return LT_ERR_ARG;
  lt_ctx_s* c = new (std::nothrow) lt_ctx_s();
  if (!c) return LT_ERR_OOM;
  const int L = cfg->L;
  c->L = L;
  c->chi = cfg->chi_max;
  c->n_traj = cfg->n_traj;
  c->method = cfg->method;
  c->prec = cfg->precision;
  c->order = cfg->trotter_order;
  c->fermionic = cfg->fermionic_jumps ? 1 : 0;
  c->J = cfg->J;
  c->dt = cfg->dt;
  c->cut = cfg->svd_cut;
  c->max_sweeps = cfg->max_sweeps > 0 ? cfg->max_sweeps : 40;
  c->jacobi_tol = cfg->jacobi_tol;
  {
    // the schedule: explicit fields, else the tuned table's entry, else the defaults
    int path = 1, env = 0;
    lt_schedule_lookup(c->method == LT_MPDO || c->method == LT_PURIFIED ? 4 : 2, cfg->precision,
                       cfg->chi_max, &path, &env);
    if (cfg->theta_path) path = cfg->theta_path;
    if (cfg->env_ctas_per_sm) env = cfg->env_ctas_per_sm;
    c->theta_tc = path == 2 ? 0 : 1;
    c->env_occ = env;
  }
  c->seed = cfg->seed;
  c->traj_offset = cfg->traj_offset;
  c->init = cfg->init;
  c->gl.assign(L, 0.0);
  c->gg.assign(L, 0.0);
  c->gd.assign(L, 0.0);
  for (int i = 0; i < L; ++i) {
    if (cfg->gamma_loss) c->gl[i] = cfg->gamma_loss[i];
    if (cfg->gamma_gain) c->gg[i] = cfg->gamma_gain[i];
    if (cfg->gamma_deph) c->gd[i] = cfg->gamma_deph[i];
    if (!(c->gl[i] >= 0.0) || !(c->gg[i] >= 0.0) || !(c->gd[i] >= 0.0)) {
      delete c;
      return LT_ERR_ARG;
    }
    // quantum state diffusion applies 1 + eta sqrt(gamma dt) L_k: with the
    // Jordan-Wigner string (fermionic loss or gain beyond site 0) that is a sum
    // of non-local products, which the site-local noise step does not cover
    if (c->method == LT_QSD && c->fermionic && i > 0 && (c->gl[i] > 0.0 || c->gg[i] > 0.0)) {
      delete c;
      return LT_ERR_UNSUPPORTED;
    }
    // the vectorised density matrix takes c_i and c_i^+ as local operators on
    // the chain ends only (there the string acts as the total parity)
    if ((c->method == LT_MPDO || c->method == LT_PURIFIED) && c->fermionic && i > 0 && i < L - 1 &&
        (c->gl[i] > 0.0 || c->gg[i] > 0.0)) {
      delete c;
      return LT_ERR_UNSUPPORTED;
    }
  }
  c->occ.assign(L, 0);
  for (int i = 0; i < L; ++i) {
    switch (cfg->init) {
      case LT_INIT_VACUUM: c->occ[i] = 0; break;
      case LT_INIT_NEEL: c->occ[i] = (i % 2 == 0); break;
      case LT_INIT_DOMAIN_WALL: c->occ[i] = (i < L / 2); break;
      default: c->occ[i] = cfg->product_occ[i] ? 1 : 0;
    }
  }
  c->d = c->method == LT_MPDO || c->method == LT_PURIFIED ? 4 : 2;
  c->slot = c->d * c->chi * c->chi;
  c->celt = c->prec == LT_MIXED ? sizeof(float2) : sizeof(double2);
  lt_status st = LT_OK;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return LT_ERR_CUDA;
  }
  if (stream) {
    c->stream = (cudaStream_t)stream;
    c->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return LT_ERR_CUDA;
    }
    c->own_stream = true;
  }
  const size_t nt = c->n_traj, nb = L - 1;
  e = configure_bond(c);
  if (e != cudaSuccess) st = fail(c, LT_ERR_CUDA, "configure_bond", cudaGetErrorString(e));
  c->env_grid = env_grid(c);
  c->env_scratch_stride = c->method == LT_MPDO
                              ? (long long)(mpdo_scratch_bytes(L, c->chi) / c->celt)
                          : c->method == LT_PURIFIED
                              ? (long long)(purified_scratch_bytes(L, c->chi) / c->celt)
                              : (long long)env_scratch_elems(L, c->chi);
  if (st == LT_OK) st = dalloc(c, (char**)&c->B, nt * L * c->slot * c->celt);
  if (st == LT_OK) st = dalloc(c, &c->lam, nt * nb * c->chi);
  if (st == LT_OK) st = dalloc(c, &c->dims, nt * nb);
  if (st == LT_OK) st = dalloc(c, &c->trunc, nt * nb);
  if (st == LT_OK) st = dalloc(c, &c->evolve, nt);
  if (st == LT_OK) st = dalloc(c, &c->channel, nt);
  if (st == LT_OK) st = dalloc(c, &c->replay, nt);
  if (st == LT_OK) st = dalloc(c, &c->active_list, nt);
  if (st == LT_OK) st = dalloc(c, &c->jumped_list, nt);
  if (st == LT_OK) st = dalloc(c, &c->counts, 2);
  if (st == LT_OK) st = dalloc(c, &c->density, nt * L);
  if (st == LT_OK) st = dalloc(c, &c->logw, nt);
  if (st == LT_OK) st = dalloc(c, &c->rates, nt * 3 * L);
  if (st == LT_OK) st = dalloc(c, &c->gam, 3 * (size_t)L);
  if (st == LT_OK) st = dalloc(c, &c->err_dev, 1);
  if (st == LT_OK) st = dalloc(c, &c->sweep_hist, 64);
  if (st == LT_OK) st = dalloc(c, &c->counters, LT_NCOUNTERS);
  if (st == LT_OK) st = dalloc(c, &c->gates, 8 * nb * (size_t)(c->d * c->d * c->d * c->d));
  if (st == LT_OK) st = dalloc(c, &c->red, 2 * (size_t)L * L + 2 * (size_t)L);
  if (st == LT_OK && c->bond_scratch_stride > 0)
    st = dalloc(c, (char**)&c->bond_scratch, (size_t)c->bond_grid * c->bond_scratch_stride * c->celt);
  // the shared Jacobi state of the clusters, as many as can be resident
  const int ncl_max = std::max(c->bond_ncl[2], std::max(c->bond_ncl[4], c->bond_ncl[8]));
  if (st == LT_OK && ncl_max > 0)
    st = dalloc(c, &c->bond_cl_state, (size_t)ncl_max * LT_CL_STATE);
  if (st == LT_OK)
    st = dalloc(c, (char**)&c->env_scratch, (size_t)c->env_grid * c->env_scratch_stride * c->celt);
  uint8_t* occ_dev = nullptr;
  if (st == LT_OK) st = dalloc(c, &occ_dev, L);
  if (st == LT_OK) {
    std::vector<double> g(3 * (size_t)L);
    for (int i = 0; i < L; ++i) {
      g[i] = c->gl[i];
      g[L + i] = c->gg[i];
      g[2 * L + i] = c->gd[i];
    }
    e = cudaMemcpyAsync(c->gam, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(occ_dev, c->occ.data(), L, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->B, 0, nt * L * c->slot * c->celt, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->lam, 0, nt * nb * c->chi * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->logw, 0, nt * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sweep_hist, 0, 64 * sizeof(int), c->stream);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(c->counters, 0, LT_NCOUNTERS * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = launch_init_state(c, occ_dev);
    if (e == cudaSuccess) e = launch_compact(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(c, LT_ERR_CUDA, "lt_create", cudaGetErrorString(e));
  }
  if (occ_dev) {
    cudaFree(occ_dev);
    c->dev_bytes -= L;
  }
  if (st != LT_OK) {
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return st;
  }
  *out = c;
  return LT_OK;
}

lt_status lt_destroy(lt_ctx c) {
  if (!c) return LT_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
  free_all(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return LT_OK;
}

lt_status lt_apply_layer(lt_ctx c, int32_t parity, double tau) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if ((parity != 0 && parity != 1) || !std::isfinite(tau)) return LT_ERR_ARG;
  if (parity > c->L - 2) return LT_OK;
  const double2* g = nullptr;
  st = gate_ptr(c, tau, &g);
  if (st != LT_OK) return st;
  const int nb = (c->L - 2 - parity) / 2 + 1;
  LT_CK(launch_bond(c, c->active_list, c->counts, parity, nb, g, 0));
  return LT_OK;
}

lt_status lt_apply_jumps(lt_ctx c, int64_t step, const int32_t* replay, int32_t* out_channel) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (step < 0) return LT_ERR_ARG;
  if (c->method != LT_TRAJ) {
    c->last_error = "jumps belong to the quantum-trajectory method";
    return LT_ERR_UNSUPPORTED;
  }
  if (replay) {
    // stage through pageable host memory: the caller's array is consumed before return
    c->replay_host.assign(replay, replay + c->n_traj);
    LT_CK(cudaMemcpyAsync(c->replay, c->replay_host.data(), sizeof(int) * c->n_traj,
                          cudaMemcpyHostToDevice, c->stream));
  }
  LT_CK(launch_env(c, 1, step, replay ? c->replay : nullptr));
  LT_CK(launch_compact(c));
  LT_CK(launch_jump_apply(c));
  // restore the canonical form of the jumped histories by one-site SVDs: right
  // to left over every bond (B_{b+1} right-canonical), then left to right
  // (Lambda_b the Schmidt spectrum)
  for (int b = c->L - 2; b >= 0; --b) LT_CK(launch_bond(c, c->jumped_list, c->counts + 1, b, 1, nullptr, 1));
  for (int b = 0; b <= c->L - 2; ++b) LT_CK(launch_bond(c, c->jumped_list, c->counts + 1, b, 1, nullptr, 2));
  if (replay) {
    st = check_device_error(c);
    if (st != LT_OK) return st;
  }
  if (out_channel) {
    LT_CK(cudaMemcpyAsync(out_channel, c->channel, sizeof(int) * c->n_traj, cudaMemcpyDeviceToHost, c->stream));
    st = check_device_error(c);
    if (st != LT_OK) return st;
  }
  return LT_OK;
}

lt_status lt_apply_noise(lt_ctx c, int64_t step) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (step < 0) return LT_ERR_ARG;
  if (c->method != LT_QSD) {
    c->last_error = "the noise step belongs to quantum state diffusion";
    return LT_ERR_UNSUPPORTED;
  }
  LT_CK(launch_qsd_noise(c, step));
  // exact canonical form of every history (the active list holds all of them:
  // no jumps are drawn); bond 0 of the left-to-right sweep moves <psi|psi> into
  // the log weight
  for (int b = c->L - 2; b >= 0; --b) LT_CK(launch_bond(c, c->active_list, c->counts, b, 1, nullptr, 1));
  for (int b = 0; b <= c->L - 2; ++b) LT_CK(launch_bond(c, c->active_list, c->counts, b, 1, nullptr, 2));
  return LT_OK;
}

lt_status lt_apply_kraus(lt_ctx c) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (c->method != LT_PURIFIED) {
    c->last_error = "the R step belongs to the purified density matrix";
    return LT_ERR_UNSUPPORTED;
  }
  LT_CK(launch_kraus(c));
  return LT_OK;
}

lt_status lt_get_log_weights(lt_ctx c, double* out) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (!out) return LT_ERR_ARG;
  LT_CK(cudaMemcpyAsync(out, c->logw, sizeof(double) * c->n_traj, cudaMemcpyDeviceToHost, c->stream));
  return check_device_error(c);
}

// the launches of one time step (no host synchronisation once the gates are cached)
static lt_status one_step(lt_ctx c, long long step) {
  lt_status st;
  if (c->method == LT_TRAJ) {
    st = lt_apply_jumps(c, step, nullptr, nullptr);
    if (st != LT_OK) return st;
  }
  if (c->order == 1) {
    if ((st = lt_apply_layer(c, 0, c->dt)) != LT_OK) return st;
    if ((st = lt_apply_layer(c, 1, c->dt)) != LT_OK) return st;
  } else {
    if ((st = lt_apply_layer(c, 0, 0.5 * c->dt)) != LT_OK) return st;
    if ((st = lt_apply_layer(c, 1, c->dt)) != LT_OK) return st;
    if ((st = lt_apply_layer(c, 0, 0.5 * c->dt)) != LT_OK) return st;
  }
  if (c->method == LT_QSD) {
    st = lt_apply_noise(c, step);
    if (st != LT_OK) return st;
  }
  if (c->method == LT_PURIFIED) {
    st = lt_apply_kraus(c);
    if (st != LT_OK) return st;
  }
  return LT_OK;
}

lt_status lt_step(lt_ctx c, int32_t n_steps) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (n_steps < 0) return LT_ERR_ARG;
  for (int s = 0; s < n_steps; ++s) {
    st = one_step(c, c->step_counter);
    if (st != LT_OK) return st;
    c->step_counter++;
  }
  return LT_OK;
}

lt_status lt_gates(const lt_config* cfg, double tau, double* out, int64_t capacity) {
  if (!cfg || !out || cfg->L < 2 || cfg->L > 1024 || !std::isfinite(tau) || !std::isfinite(cfg->J))
    return LT_ERR_ARG;
  if (cfg->method < LT_TRAJ || cfg->method > LT_PURIFIED) return LT_ERR_UNSUPPORTED;
  lt_ctx_s c{};
  c.L = cfg->L;
  c.J = cfg->J;
  c.method = cfg->method;
  c.d = cfg->method == LT_MPDO || cfg->method == LT_PURIFIED ? 4 : 2;
  c.gl.assign(c.L, 0.0);
  c.gg.assign(c.L, 0.0);
  c.gd.assign(c.L, 0.0);
  for (int i = 0; i < c.L; ++i) {
    if (cfg->gamma_loss) c.gl[i] = cfg->gamma_loss[i];
    if (cfg->gamma_gain) c.gg[i] = cfg->gamma_gain[i];
    if (cfg->gamma_deph) c.gd[i] = cfg->gamma_deph[i];
    if (!(c.gl[i] >= 0.0) || !(c.gg[i] >= 0.0) || !(c.gd[i] >= 0.0)) return LT_ERR_ARG;
  }
  const int64_t per = (int64_t)c.d * c.d * c.d * c.d;
  if (capacity < 2 * per * (c.L - 1)) return LT_ERR_ARG;
  std::vector<double2> g;
  if (c.method == LT_MPDO) build_liouvillian_gates(&c, tau, g);
  else if (c.method == LT_PURIFIED) build_purified_gates(&c, tau, g);
  else build_gates(&c, tau, g);
  for (size_t i = 0; i < g.size(); ++i) {
    out[2 * i] = g[i].x;
    out[2 * i + 1] = g[i].y;
  }
  return LT_OK;
}

lt_status lt_step_graph(lt_ctx c, int32_t n_steps) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (n_steps < 0) return LT_ERR_ARG;
  if (n_steps == 0) return LT_OK;
  if (!c->step_graph) {
    // the gates of the schedule are uploaded before the capture: an upload
    // synchronises the stream, which a capture does not allow
    const double2* g = nullptr;
    if (c->order == 1) {
      if ((st = gate_ptr(c, c->dt, &g)) != LT_OK) return st;
    } else {
      if ((st = gate_ptr(c, 0.5 * c->dt, &g)) != LT_OK) return st;
      if ((st = gate_ptr(c, c->dt, &g)) != LT_OK) return st;
    }
    if (!c->step_dev) {
      st = dalloc(c, &c->step_dev, 1);
      if (st != LT_OK) return st;
    }
    cudaGraph_t graph = nullptr;
    const long long before = c->launches;
    c->use_step_dev = true;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      c->use_step_dev = false;
      cudaGetLastError();
      c->last_error = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
      return LT_ERR_UNSUPPORTED;  // e.g. the legacy default stream
    }
    st = one_step(c, 0);
    cudaError_t e2 = st == LT_OK ? launch_step_advance(c) : cudaSuccess;
    e = cudaStreamEndCapture(c->stream, &graph);
    c->use_step_dev = false;
    if (st != LT_OK || e2 != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      c->launches = before;
      if (st != LT_OK) return st;
      return fail(c, LT_ERR_CUDA, "step capture", cudaGetErrorString(e2 != cudaSuccess ? e2 : e));
    }
    e = cudaGraphInstantiate(&c->step_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->step_graph = nullptr;
      c->launches = before;
      return fail(c, LT_ERR_CUDA, "cudaGraphInstantiate", cudaGetErrorString(e));
    }
    c->graph_launches = c->launches - before;
    c->launches = before;
  }
  // the device counter starts at this context's step; each replay advances it
  c->step_host = c->step_counter;
  LT_CK(cudaMemcpyAsync(c->step_dev, &c->step_host, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
  for (int s = 0; s < n_steps; ++s) LT_CK(cudaGraphLaunch(c->step_graph, c->stream));
  c->step_counter += n_steps;
  c->launches += (long long)n_steps * c->graph_launches;
  return LT_OK;
}

lt_status lt_measure_density(lt_ctx c, double* mean, double* sem, double* per_traj) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (c->method == LT_MPDO) LT_CK(launch_mpdo_trace(c, false));
  else if (c->method == LT_PURIFIED) LT_CK(launch_purified_env(c, false));
  else LT_CK(launch_env(c, 0, 0, nullptr));
  LT_CK(launch_reduce_density(c, c->red, c->red + c->L));
  if (mean) LT_CK(cudaMemcpyAsync(mean, c->red, sizeof(double) * c->L, cudaMemcpyDeviceToHost, c->stream));
  if (sem) LT_CK(cudaMemcpyAsync(sem, c->red + c->L, sizeof(double) * c->L, cudaMemcpyDeviceToHost, c->stream));
  if (per_traj)
    LT_CK(cudaMemcpyAsync(per_traj, c->density, sizeof(double) * c->L * (size_t)c->n_traj,
                          cudaMemcpyDeviceToHost, c->stream));
  return check_device_error(c);
}

lt_status lt_measure_corr(lt_ctx c, double* C_re, double* C_im, double* per_re, double* per_im) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  const size_t LL = (size_t)c->L * c->L;
  if (!c->corr) {
    st = dalloc(c, &c->corr, LL * c->n_traj);
    if (st != LT_OK) return st;
  }
  if (c->method == LT_MPDO) LT_CK(launch_mpdo_trace(c, true));
  else if (c->method == LT_PURIFIED) LT_CK(launch_purified_env(c, true));
  else LT_CK(launch_corr(c));
  LT_CK(launch_reduce_corr(c, c->red));
  std::vector<double> m(2 * LL);
  LT_CK(cudaMemcpyAsync(m.data(), c->red, sizeof(double) * 2 * LL, cudaMemcpyDeviceToHost, c->stream));
  std::vector<double2> per;
  if (per_re || per_im) {
    per.resize(LL * c->n_traj);
    LT_CK(cudaMemcpyAsync(per.data(), c->corr, sizeof(double2) * per.size(), cudaMemcpyDeviceToHost, c->stream));
  }
  st = check_device_error(c);
  if (st != LT_OK) return st;
  for (size_t i = 0; i < LL; ++i) {
    if (C_re) C_re[i] = m[2 * i];
    if (C_im) C_im[i] = m[2 * i + 1];
  }
  for (size_t i = 0; i < per.size(); ++i) {
    if (per_re) per_re[i] = per[i].x;
    if (per_im) per_im[i] = per[i].y;
  }
  return LT_OK;
}

lt_status lt_get_stats(lt_ctx c, double* trunc_weight, int32_t* bond_dims) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  const size_t nb = c->L - 1, nt = c->n_traj;
  std::vector<double> tr;
  if (trunc_weight) {
    tr.resize(nt * nb);
    LT_CK(cudaMemcpyAsync(tr.data(), c->trunc, sizeof(double) * tr.size(), cudaMemcpyDeviceToHost, c->stream));
  }
  if (bond_dims)
    LT_CK(cudaMemcpyAsync(bond_dims, c->dims, sizeof(int) * nt * nb, cudaMemcpyDeviceToHost, c->stream));
  st = check_device_error(c);
  if (st != LT_OK) return st;
  for (size_t t = 0; trunc_weight && t < nt; ++t) {
    double s = 0.0;
    for (size_t b = 0; b < nb; ++b) s += tr[t * nb + b];
    trunc_weight[t] = s;
  }
  return LT_OK;
}

lt_status lt_set_state(lt_ctx c, int32_t traj0, int32_t n, const int32_t* dims, const double* lam,
                       const double* B) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (traj0 < 0 || n < 0 || traj0 + (long long)n > c->n_traj || !dims || !lam || !B) return LT_ERR_ARG;
  const size_t nb = c->L - 1;
  for (size_t i = 0; i < (size_t)n * nb; ++i)
    if (dims[i] < 1 || dims[i] > c->chi) return LT_ERR_ARG;
  LT_CK(cudaStreamSynchronize(c->stream));
  LT_CK(cudaMemcpyAsync(c->dims + (size_t)traj0 * nb, dims, sizeof(int) * n * nb, cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaMemcpyAsync(c->lam + (size_t)traj0 * nb * c->chi, lam, sizeof(double) * n * nb * c->chi, cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaMemsetAsync(c->trunc + (size_t)traj0 * nb, 0, sizeof(double) * n * nb, c->stream));
  LT_CK(cudaMemsetAsync(c->logw + traj0, 0, sizeof(double) * n, c->stream));
  const long long per_traj = (long long)c->L * c->slot;
  const int chunk = 8;
  double* stage = nullptr;
  st = dalloc(c, &stage, 2 * (size_t)per_traj * chunk);
  if (st != LT_OK) return st;
  for (int t = 0; t < n && st == LT_OK; t += chunk) {
    const int m = n - t < chunk ? n - t : chunk;
    cudaError_t e = cudaMemcpyAsync(stage, B + 2 * (size_t)per_traj * t, sizeof(double) * 2 * per_traj * m, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_convert_in(c, stage, per_traj * m, per_traj * (traj0 + t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(c, LT_ERR_CUDA, "lt_set_state", cudaGetErrorString(e));
  }
  cudaFree(stage);
  c->dev_bytes -= 2 * (size_t)per_traj * chunk * sizeof(double);
  return st;
}

lt_status lt_get_state(lt_ctx c, int32_t traj0, int32_t n, int32_t* dims, double* lam, double* B) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (traj0 < 0 || n < 0 || traj0 + (long long)n > c->n_traj) return LT_ERR_ARG;
  const size_t nb = c->L - 1;
  LT_CK(cudaStreamSynchronize(c->stream));
  if (dims) LT_CK(cudaMemcpyAsync(dims, c->dims + (size_t)traj0 * nb, sizeof(int) * n * nb, cudaMemcpyDeviceToHost, c->stream));
  if (lam)
    LT_CK(cudaMemcpyAsync(lam, c->lam + (size_t)traj0 * nb * c->chi, sizeof(double) * n * nb * c->chi, cudaMemcpyDeviceToHost, c->stream));
  LT_CK(cudaStreamSynchronize(c->stream));
  if (!B) return LT_OK;
  const long long per_traj = (long long)c->L * c->slot;
  const int chunk = 8;
  double* stage = nullptr;
  st = dalloc(c, &stage, 2 * (size_t)per_traj * chunk);
  if (st != LT_OK) return st;
  for (int t = 0; t < n && st == LT_OK; t += chunk) {
    const int m = n - t < chunk ? n - t : chunk;
    cudaError_t e = launch_convert_out(c, stage, per_traj * m, per_traj * (traj0 + t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B + 2 * (size_t)per_traj * t, stage, sizeof(double) * 2 * per_traj * m, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) st = fail(c, LT_ERR_CUDA, "lt_get_state", cudaGetErrorString(e));
  }
  cudaFree(stage);
  c->dev_bytes -= 2 * (size_t)per_traj * chunk * sizeof(double);
  return st;
}

// checkpoint file: magic, header ints, step, then dims, lam, trunc and the raw
// site tensors in the context's precision
lt_status lt_save(lt_ctx c, const char* path) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (!path) return LT_ERR_ARG;
  const size_t nb = c->L - 1, nt = c->n_traj;
  std::vector<int> dims(nt * nb);
  std::vector<double> lam(nt * nb * c->chi), tr(nt * nb), lw(nt);
  std::vector<char> B(nt * c->L * c->slot * c->celt);
  LT_CK(cudaStreamSynchronize(c->stream));
  LT_CK(cudaMemcpyAsync(lw.data(), c->logw, lw.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LT_CK(cudaMemcpyAsync(dims.data(), c->dims, dims.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LT_CK(cudaMemcpyAsync(lam.data(), c->lam, lam.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LT_CK(cudaMemcpyAsync(tr.data(), c->trunc, tr.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LT_CK(cudaMemcpyAsync(B.data(), c->B, B.size(), cudaMemcpyDeviceToHost, c->stream));
  LT_CK(cudaStreamSynchronize(c->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, LT_ERR_ARG, "lt_save", "cannot open file");
  const char magic[8] = {'L', 'T', 'C', 'K', 'P', 'T', '0', '2'};
  const int hdr[5] = {c->L, c->chi, c->n_traj, c->prec, c->method};
  const long long stepc = c->step_counter;
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 5, f) == 5 &&
            std::fwrite(&stepc, sizeof(stepc), 1, f) == 1 &&
            std::fwrite(dims.data(), sizeof(int), dims.size(), f) == dims.size() &&
            std::fwrite(lam.data(), sizeof(double), lam.size(), f) == lam.size() &&
            std::fwrite(tr.data(), sizeof(double), tr.size(), f) == tr.size() &&
            std::fwrite(B.data(), 1, B.size(), f) == B.size() &&
            std::fwrite(lw.data(), sizeof(double), lw.size(), f) == lw.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? LT_OK : fail(c, LT_ERR_ARG, "lt_save", "short write");
}

lt_status lt_load(lt_ctx c, const char* path) {
  lt_status st = guard(c);
  if (st != LT_OK) return st;
  if (!path) return LT_ERR_ARG;
  const size_t nb = c->L - 1, nt = c->n_traj;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, LT_ERR_ARG, "lt_load", "cannot open file");
  char magic[8];
  int hdr[5];
  long long stepc = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "LTCKPT02", 8) == 0 &&
            std::fread(hdr, sizeof(int), 5, f) == 5 && hdr[0] == c->L && hdr[1] == c->chi &&
            hdr[2] == c->n_traj && hdr[3] == c->prec && hdr[4] == c->method &&
            std::fread(&stepc, sizeof(stepc), 1, f) == 1;
  std::vector<int> dims(nt * nb);
  std::vector<double> lam(nt * nb * c->chi), tr(nt * nb), lw(nt);
  std::vector<char> B(nt * c->L * c->slot * c->celt);
  ok = ok && std::fread(dims.data(), sizeof(int), dims.size(), f) == dims.size() &&
       std::fread(lam.data(), sizeof(double), lam.size(), f) == lam.size() &&
       std::fread(tr.data(), sizeof(double), tr.size(), f) == tr.size() &&
       std::fread(B.data(), 1, B.size(), f) == B.size() &&
       std::fread(lw.data(), sizeof(double), lw.size(), f) == lw.size();
  std::fclose(f);
  if (!ok) return fail(c, LT_ERR_ARG, "lt_load", "checkpoint does not match this context");
  for (int d : dims)
    if (d < 1 || d > c->chi) return fail(c, LT_ERR_ARG, "lt_load", "bond dimension out of range");
  LT_CK(cudaStreamSynchronize(c->stream));
  LT_CK(cudaMemcpyAsync(c->dims, dims.data(), dims.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaMemcpyAsync(c->lam, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaMemcpyAsync(c->trunc, tr.data(), tr.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaMemcpyAsync(c->B, B.data(), B.size(), cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaMemcpyAsync(c->logw, lw.data(), lw.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LT_CK(cudaStreamSynchronize(c->stream));
  c->step_counter = stepc;
  return LT_OK;
}

}  // extern "C"
