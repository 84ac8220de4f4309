"""MPS quantum-trajectory integrator in Vidal-Hastings form (plain FP64).

State (Sec. 2.2, Eqs. MPS, MPSMixte; Vidal form as in Sec. 2.3): per site a tensor
B_i = Gamma_i Lambda_i of shape (chi_{i-1}, 2, chi_i), per bond the Schmidt values
Lambda_i (length chi_i), chi_{-1} = chi_{L-1} = 1, Lambda_{-1} = [1].  The state is
psi = B_0 B_1 ... B_{L-1}.

Two-site update (Sec. 2.3, Eq. Theta, with the Hastings variant that avoids
dividing by Lambda):
  theta~[(a,s'),(t',c)] = sum_{s,t} G[s't',st] sum_m B_b[a,s,m] B_{b+1}[m,t,c]
  theta = Lambda_{b-1}[a] theta~                      (rows weighted)
  theta = U S V^+  (SVD, S descending)
  keep k = min(chi_max, #{S_j > cut * S_0}) >= 1     (keep the chi largest, Sec. 2.2)
  discarded weight w = sum_{j>=k} S_j^2 / sum_j S_j^2 (Eq. HilbertSchmidtNorm)
  Lambda_b <- S_k / ||S_k||                            (renormalise, Sec. 2.3 end)
  B_{b+1} <- V_k^+,  B_b <- theta~ V_k / ||S_k||

One time step of a trajectory (Sec. 4.1, after Eq. ErrorCLT's preceding text):
  rates W_k = gamma_k <L_k^+ L_k> for every channel (Eq. TransitionRate), with
  <n_k> = <psi|n_k|psi>/<psi|psi> contracted with left and right environments
  (equal to the Fig. 3 local formula when the form is exactly canonical);
  draw r ~ U[0,1) (Philox, purpose 0); if r < P = sum_k W_k dt the channel is the
  least k with cumulative sum of W dt above r: apply L_k, renormalise and restore
  the canonical form; otherwise apply the Trotter layers of exp(-i H_eff dt)
  (Eq. QJump1), the norm being restored by each bond's renormalisation.

Canonical form after a jump: L_k changes only B_k (plus a sign on the occupied
component of every B_j, j < k, for the fermionic string, a unitary).  One-site
SVDs shift the orthogonality centre (Sec. 2.2, Eq. ShiftCenter): right to left
over bonds L-2, ..., 0 each B_{b+1} is made right-canonical and its U S absorbed
into B_b; then left to right over bonds 0, ..., L-2 the SVD of Lambda_{b-1} B_b
restores Lambda_b as the exact Schmidt spectrum.  With B_{b+1} right-canonical
this equals the two-site update with the identity gate.  The sweep covers the
whole chain because the effective-Hamiltonian layers before the jump leave the
form only approximately canonical.
"""
import numpy as np

from . import model
from .philox import uniform01, noise, PURPOSE_JUMP

IDENTITY4 = np.eye(4, dtype=complex)


class TrajectoryConfig:
    """Parameters of the trajectory integrator (one chain, many trajectories)."""

    def __init__(self, L, J=1.0, dt=0.05, chi_max=16, svd_cut=1e-12,
                 gamma_loss=0.0, gamma_gain=0.0, gamma_deph=0.0,
                 fermionic=True, trotter_order=2, occupation=None, seed=0):
        self.L = int(L)
        self.J = float(J)
        self.dt = float(dt)
        self.chi_max = int(chi_max)
        self.svd_cut = float(svd_cut)
        self.gamma_loss = np.broadcast_to(np.asarray(gamma_loss, float), (L,)).copy()
        self.gamma_gain = np.broadcast_to(np.asarray(gamma_gain, float), (L,)).copy()
        self.gamma_deph = np.broadcast_to(np.asarray(gamma_deph, float), (L,)).copy()
        self.fermionic = bool(fermionic)
        self.trotter_order = int(trotter_order)
        self.occupation = (np.zeros(L, int) if occupation is None
                           else np.asarray(occupation, int).copy())
        self.seed = int(seed)

    def layers(self):
        """Trotter schedule as (parity, tau): parity 0 = even bonds, 1 = odd bonds."""
        dt = self.dt
        if self.trotter_order == 1:
            return [(0, dt), (1, dt)]
        if self.trotter_order == 2:
            return [(0, dt / 2), (1, dt), (0, dt / 2)]
        raise ValueError("trotter_order must be 1 or 2")

    def gates(self, tau):
        return model.bond_gates(self.L, self.J, tau, self.gamma_loss,
                                self.gamma_gain, self.gamma_deph)


class Trajectory:
    """One MPS history |psi_alpha(t)> in Vidal-Hastings form."""

    def __init__(self, cfg):
        self.cfg = cfg
        L = cfg.L
        self.B = []
        for i in range(L):
            t = np.zeros((1, 2, 1), dtype=complex)
            t[0, int(cfg.occupation[i]), 0] = 1.0
            self.B.append(t)
        self.lam = [np.ones(1) for _ in range(L - 1)]
        self.trunc_weight = 0.0
        self.log_weight = 0.0   # ln <psi|psi> of the unnormalised QSD state (Sec. 5.2)

    @classmethod
    def from_tensors(cls, cfg, B, lam):
        self = cls.__new__(cls)
        self.cfg = cfg
        self.B = [np.array(b, dtype=complex) for b in B]
        self.lam = [np.array(x, dtype=float) for x in lam]
        self.trunc_weight = 0.0
        self.log_weight = 0.0
        return self

    def bond_dims(self):
        return [len(x) for x in self.lam]

    def left_weight(self, b):
        return self.lam[b - 1] if b > 0 else np.ones(1)

    # ---- Sec. 2.3, Eq. Theta (Hastings form) --------------------------------
    def update_bond(self, b, G, keep_norm=False):
        """Two-site update.  With keep_norm (quantum state diffusion) B_b keeps
        the factor ||S_k||, so the represented state carries the norm change of
        the non-unitary gate; Lambda_b is normalised either way."""
        cfg = self.cfg
        Bl, Br = self.B[b], self.B[b + 1]
        chiL, chiR = Bl.shape[0], Br.shape[2]
        P = np.tensordot(Bl, Br, axes=(2, 0))                  # [a, s, t, c]
        tt = np.einsum('uvst,astc->auvc', G.reshape(2, 2, 2, 2), P)
        tt = tt.reshape(chiL * 2, 2 * chiR)                     # theta~
        th = tt * np.repeat(self.left_weight(b), 2)[:, None]    # theta
        U, S, Vh = np.linalg.svd(th, full_matrices=False)
        if not S[0] > 0.0:
            raise FloatingPointError("theta vanished at bond %d" % b)
        k = int(np.count_nonzero(S > cfg.svd_cut * S[0]))
        k = max(1, min(cfg.chi_max, k))
        total = float(np.sum(S ** 2))
        kept = float(np.sum(S[:k] ** 2))
        norm = np.sqrt(kept)
        self.trunc_weight += (total - kept) / total
        Vk_h = Vh[:k]
        self.B[b + 1] = Vk_h.reshape(k, 2, chiR).copy()
        self.B[b] = (tt @ Vk_h.conj().T / (1.0 if keep_norm else norm)).reshape(chiL, 2, k)
        self.lam[b] = S[:k] / norm

    def apply_layer(self, parity, gates, keep_norm=False):
        for b in range(parity, self.cfg.L - 1, 2):
            self.update_bond(b, gates[b], keep_norm)

    def apply_site_operator(self, i, M):
        """B_i <- M B_i on the physical index (M a 2 x 2 matrix)."""
        self.B[i] = np.einsum('uv,avc->auc', M, self.B[i])

    # ---- expectation values (Fig. 3, with exact environments) ---------------
    def environments(self):
        """Left and right transfer-matrix environments of <psi|psi>.

        Lenv[i][b', b] = sum conj(psi-left)_{b'} (psi-left)_b over sites < i,
        Renv[i][a, a'] = sum over sites >= i, Lenv[0] = Renv[L] = [[1]].
        Under the non-unitary effective-Hamiltonian gates the bond-parallel
        update leaves the neighbouring Lambda only approximately canonical, so
        expectation values contract the full environments instead of assuming
        Lenv = diag(Lambda^2) and Renv = 1 (they coincide in canonical form)."""
        L = self.cfg.L
        Lenv = [None] * (L + 1)
        Renv = [None] * (L + 1)
        Lenv[0] = np.ones((1, 1), dtype=complex)
        Renv[L] = np.ones((1, 1), dtype=complex)
        for i in range(L):
            Bi = self.B[i]
            Lenv[i + 1] = sum(Bi[:, s, :].conj().T @ Lenv[i] @ Bi[:, s, :] for s in range(2))
        for i in range(L - 1, -1, -1):
            Bi = self.B[i]
            Renv[i] = sum(Bi[:, s, :] @ Renv[i + 1] @ Bi[:, s, :].conj().T for s in range(2))
        return Lenv, Renv

    def norm2(self):
        return float(np.real(self.environments()[1][0][0, 0]))

    def density(self):
        """<n_i> = <psi|n_i|psi> / <psi|psi> for every site."""
        Lenv, Renv = self.environments()
        nrm = np.real(Renv[0][0, 0])
        out = np.empty(self.cfg.L)
        for i in range(self.cfg.L):
            B1 = self.B[i][:, 1, :]
            out[i] = np.real(np.sum(B1.conj() * (Lenv[i] @ B1 @ Renv[i + 1]))) / nrm
        return out

    def channel_rates(self):
        """W_k = gamma_k <L_k^+ L_k> for channel k = 3 * site + kind (Eq. TransitionRate)."""
        cfg = self.cfg
        n = self.density()
        W = np.zeros(3 * cfg.L)
        W[0::3] = cfg.gamma_loss * n
        W[1::3] = cfg.gamma_gain * (1.0 - n)
        W[2::3] = cfg.gamma_deph * n
        return W

    def apply_jump(self, channel):
        """|psi> <- L_k |psi>, then renormalise and restore the canonical form."""
        cfg = self.cfg
        site, kind = divmod(int(channel), model.N_KINDS)
        O = model.jump_operator(kind)
        self.B[site] = np.einsum('uv,avc->auc', O, self.B[site])
        if model.has_string(kind, cfg.fermionic):
            for j in range(site):
                self.B[j] = self.B[j].copy()
                self.B[j][:, 1, :] *= -1.0
        self.recanonicalize(site)

    def recanonicalize(self, site=None):
        """Restore the exact canonical form (every B right-canonical, every Lambda
        the Schmidt spectrum of its bond).  The sweep covers the whole chain: the
        effective-Hamiltonian layers before a jump leave the form only
        approximately canonical on both sides of the jump site.  Returns the
        squared norm the state had (found at bond 0, where everything to the
        right is right-canonical, and divided out there)."""
        for b in range(self.cfg.L - 2, -1, -1):
            self.shift_left(b)
        norm2 = 1.0
        for b in range(0, self.cfg.L - 1):
            kept = self.restore_bond(b)
            if b == 0:
                norm2 = kept
        return norm2

    # ---- moving the orthogonality centre by one-site SVDs (Sec. 2.2, Eq. ShiftCenter)
    def _keep(self, S):
        k = int(np.count_nonzero(S > self.cfg.svd_cut * S[0]))
        return max(1, min(self.cfg.chi_max, k))

    def shift_left(self, b):
        """Make B_{b+1} right-canonical: B_{b+1} = U S V^+ as a chi_b x (2 chi_{b+1})
        matrix, B_{b+1} <- V_k^+, B_b <- B_b U_k S_k (the state is unchanged up to
        the discarded singular values; no renormalisation)."""
        Bl, Br = self.B[b], self.B[b + 1]
        chiL, chiM, chiR = Bl.shape[0], Br.shape[0], Br.shape[2]
        U, S, Vh = np.linalg.svd(Br.reshape(chiM, 2 * chiR), full_matrices=False)
        if not S[0] > 0.0:
            raise FloatingPointError("site tensor vanished at %d" % (b + 1))
        k = min(self._keep(S), len(S))
        self.B[b + 1] = Vh[:k].reshape(k, 2, chiR).copy()
        self.B[b] = (Bl.reshape(2 * chiL, chiM) @ (U[:, :k] * S[:k])).reshape(chiL, 2, k)
        self.lam[b] = S[:k] / np.sqrt(np.sum(S[:k] ** 2))

    def restore_bond(self, b):
        """With Lambda_{b-1} exact and B_{b+1}, B_{b+2}, ... right-canonical, the
        SVD of Lambda_{b-1} B_b (a 2 chi_{b-1} x chi_b matrix) gives the Schmidt
        values of bond b: Lambda_b <- S_k / ||S_k||, B_b <- B_b V_k / ||S_k||,
        B_{b+1} <- V_k^+ B_{b+1}; the discarded weight is recorded."""
        Bl, Br = self.B[b], self.B[b + 1]
        chiL, chiM, chiR = Bl.shape[0], Bl.shape[2], Br.shape[2]
        Bm = Bl.reshape(2 * chiL, chiM)
        M = np.repeat(self.left_weight(b), 2)[:, None] * Bm
        U, S, Vh = np.linalg.svd(M, full_matrices=False)
        if not S[0] > 0.0:
            raise FloatingPointError("site tensor vanished at %d" % b)
        k = min(self._keep(S), len(S))
        total = float(np.sum(S ** 2))
        kept = float(np.sum(S[:k] ** 2))
        norm = np.sqrt(kept)
        self.trunc_weight += (total - kept) / total
        Vk_h = Vh[:k]
        self.B[b] = (Bm @ Vk_h.conj().T / norm).reshape(chiL, 2, k)
        self.B[b + 1] = (Vk_h @ Br.reshape(chiM, 2 * chiR)).reshape(k, 2, chiR)
        self.lam[b] = S[:k] / norm
        return kept

    # ---- <c_i^+ c_j> by transfer matrices -------------------------------------
    def correlation(self):
        """C_ij = <c_i^+ c_j> = <s+_i prod_{i<l<j} (-1)^{n_l} s-_j> / <psi|psi>
        for i < j, C_ji = conj(C_ij), C_ii = <n_i> (Jordan-Wigner, Sec. 2.1)."""
        L = self.cfg.L
        Lenv, Renv = self.environments()
        nrm = np.real(Renv[0][0, 0])
        C = np.zeros((L, L), dtype=complex)
        C[np.diag_indices(L)] = self.density()
        for i in range(L):
            Bi = self.B[i]
            # s+ = |1><0|: bra component 1, ket component 0
            E = Bi[:, 1, :].conj().T @ Lenv[i] @ Bi[:, 0, :]
            for j in range(i + 1, L):
                Bj = self.B[j]
                # close with s- = |0><1|: bra component 0, ket component 1
                C[i, j] = np.sum(Bj[:, 0, :].conj() * (E @ Bj[:, 1, :] @ Renv[j + 1])) / nrm
                C[j, i] = np.conj(C[i, j])
                # carry the string (-1)^n through site j
                E = (Bj[:, 0, :].conj().T @ E @ Bj[:, 0, :]
                     - Bj[:, 1, :].conj().T @ E @ Bj[:, 1, :])
        return C

    def to_dense(self):
        """Contract B_0 ... B_{L-1} into the 2^L vector (site 0 most significant)."""
        v = self.B[0].reshape(2, -1)
        for i in range(1, self.cfg.L):
            Bi = self.B[i]
            v = (v @ Bi.reshape(Bi.shape[0], -1)).reshape(-1, Bi.shape[2])
        return v.reshape(-1)


def draw_channel(rates, dt, r):
    """Jump-or-evolve decision (Sec. 4.1): -1 if r >= P = sum W dt, else the least
    channel whose cumulative probability exceeds r."""
    p = rates * dt
    total = float(np.sum(p))
    if total >= 0.5:
        raise ValueError("jump probability per step %.3g >= 0.5: reduce dt" % total)
    if not r < total:
        return -1
    csum = np.cumsum(p)
    return int(np.argmax(csum > r))


class StepGates:
    """The gates of one Trotter step, built once per run."""

    def __init__(self, cfg):
        self.layers = [(parity, cfg.gates(tau)) for parity, tau in cfg.layers()]


def step_trajectory(traj, gates, traj_id, step, replay=None):
    """One time step of one history; returns the applied channel or -1."""
    cfg = traj.cfg
    if replay is None or replay == -2:
        r = uniform01(cfg.seed, traj_id, step, PURPOSE_JUMP)
        ch = draw_channel(traj.channel_rates(), cfg.dt, r)
    else:
        ch = int(replay)
    if ch >= 0:
        traj.apply_jump(ch)
    else:
        for parity, g in gates.layers:
            traj.apply_layer(parity, g)
    return ch


def run_trajectories(cfg, n_steps, traj_ids, replay=None, measure_corr=False,
                     initial=None):
    """Integrate the histories traj_ids for n_steps steps.

    replay: optional array [len(traj_ids), n_steps] of channels (-1 none, -2 draw).
    initial: optional list of (B, lam) per trajectory (default: the product state).
    Returns dict(density [n, L], corr [n, L, L] or None, jumps [n, n_steps],
    trunc [n], bond_dims [n, L-1]).
    """
    gates = StepGates(cfg)
    n = len(traj_ids)
    dens = np.zeros((n, cfg.L))
    corr = np.zeros((n, cfg.L, cfg.L), dtype=complex) if measure_corr else None
    jumps = np.full((n, n_steps), -1, dtype=np.int64)
    trunc = np.zeros(n)
    dims = np.zeros((n, cfg.L - 1), dtype=np.int64)
    for idx, tid in enumerate(traj_ids):
        if initial is None:
            traj = Trajectory(cfg)
        else:
            traj = Trajectory.from_tensors(cfg, *initial[idx])
        for step in range(n_steps):
            rep = None if replay is None else replay[idx][step]
            jumps[idx, step] = step_trajectory(traj, gates, tid, step, rep)
        dens[idx] = traj.density()
        if measure_corr:
            corr[idx] = traj.correlation()
        trunc[idx] = traj.trunc_weight
        dims[idx] = traj.bond_dims()
    return dict(density=dens, corr=corr, jumps=jumps, trunc=trunc, bond_dims=dims)


# ---- quantum state diffusion (Sec. 5.2) -------------------------------------------
def qsd_check(cfg):
    """The noise operators 1 + eta sqrt(gamma dt) L_k must act on one site: a
    loss or gain channel with the Jordan-Wigner string (fermionic c_k for k > 0)
    would make them sums of non-local products."""
    if cfg.fermionic and (np.any(cfg.gamma_loss[1:] > 0) or np.any(cfg.gamma_gain[1:] > 0)):
        raise ValueError("quantum state diffusion needs local jump operators: fermionic "
                         "loss or gain only on site 0, or spin operators")


def qsd_site_operator(cfg, site, eta):
    """prod_k (1 + eta_k sqrt(gamma_k dt) L_k) over the channels k = 3 site + kind
    of one site, applied in increasing k (loss, then gain, then dephasing);
    eta = (eta_loss, eta_gain, eta_deph)."""
    gam = (cfg.gamma_loss[site], cfg.gamma_gain[site], cfg.gamma_deph[site])
    M = model.IDENTITY2.copy()
    for kind in (model.LOSS, model.GAIN, model.DEPHASING):
        if gam[kind] > 0:
            a = eta[kind] * np.sqrt(gam[kind] * cfg.dt)
            M = (model.IDENTITY2 + a * model.jump_operator(kind)) @ M
    return M


def step_qsd(traj, gates, traj_id, step):
    """One step of the first-order scheme of Sec. 5.2: |psi> <- prod_k (1 +
    eta_k sqrt(gamma_k dt) L_k) exp(-i H_eff dt) |psi>, with the exponential by the
    Trotter layers (no renormalisation, so the state keeps its norm change), the
    noise eta_k from the Philox Gaussian pairs of (trajectory, step), then the
    exact canonical form; the squared norm removed there multiplies the weight
    w = <psi|psi> (log_weight += ln)."""
    cfg = traj.cfg
    for parity, g in gates.layers:
        traj.apply_layer(parity, g, keep_norm=True)
    eta = noise(cfg.seed, traj_id, step, 3 * cfg.L)
    for i in range(cfg.L):
        traj.apply_site_operator(i, qsd_site_operator(cfg, i, eta[3 * i:3 * i + 3]))
    traj.log_weight += float(np.log(traj.recanonicalize()))


def run_qsd(cfg, n_steps, traj_ids, measure_corr=False, initial=None):
    """Integrate the QSD histories traj_ids for n_steps steps.  Returns
    dict(density [n, L] and corr [n, L, L] of the normalised states, log_weight
    [n] = ln <psi|psi>, trunc [n], bond_dims [n, L-1])."""
    qsd_check(cfg)
    gates = StepGates(cfg)
    n = len(traj_ids)
    dens = np.zeros((n, cfg.L))
    corr = np.zeros((n, cfg.L, cfg.L), dtype=complex) if measure_corr else None
    logw = np.zeros(n)
    trunc = np.zeros(n)
    dims = np.zeros((n, cfg.L - 1), dtype=np.int64)
    for idx, tid in enumerate(traj_ids):
        traj = Trajectory(cfg) if initial is None else Trajectory.from_tensors(cfg, *initial[idx])
        for step in range(n_steps):
            step_qsd(traj, gates, tid, step)
        dens[idx] = traj.density()
        if measure_corr:
            corr[idx] = traj.correlation()
        logw[idx] = traj.log_weight
        trunc[idx] = traj.trunc_weight
        dims[idx] = traj.bond_dims()
    return dict(density=dens, corr=corr, log_weight=logw, trunc=trunc, bond_dims=dims)


def qsd_estimate(values, log_weight):
    """Sec. 5.2: the average density matrix is the mean of |psi><psi| over the
    unnormalised histories, so <O> = mean_t(w_t <O>_t) with w_t = <psi_t|psi_t> and
    <O>_t the normalised expectation; returns that mean and its CLT error."""
    w = np.exp(np.asarray(log_weight))
    x = np.asarray(values) * w.reshape((-1,) + (1,) * (np.ndim(values) - 1))
    return ensemble_stats(x)


def ensemble_stats(values):
    """Monte Carlo mean and its CLT error sqrt(var / n_conf) (Eq. ErrorCLT)."""
    values = np.asarray(values)
    n = values.shape[0]
    mean = values.mean(axis=0)
    if n < 2:
        return mean, np.zeros_like(np.real(mean))
    var = np.mean(np.abs(values - mean) ** 2, axis=0)
    return mean, np.sqrt(var / n)
