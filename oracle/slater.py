"""Exact per-trajectory reference for the free-fermion chain: the history as a
Slater determinant (plain FP64, no truncation).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every operation of a quantum-trajectory step on the chain of Sec. 2.1 maps a
Slater determinant to a Slater determinant, so a history with N particles is
the span of N orbitals, an L x N matrix Phi, and the MPS integrator of
``tebd`` (same Trotter gates, same jump record) must reproduce it up to its
truncation error:

  * the two-site gate exp(-i h_b^eff tau) (Sec. 2.3; h_b^eff of Eq.
    EffHamiltonian with the site terms shared between bonds as in Eq.
    LindbladLocal) is the exponential of a quadratic form c^+ h1 c; on
    orbitals it is the 2 x 2 matrix exp(-i tau h1) acting on rows b, b+1 with
    h1 = [[-i w_b k_b / 2, -J], [-J, -i w_{b+1} k_{b+1} / 2]], k_i = gamma_loss
    + gamma_deph - gamma_gain (L^+L = n for loss and dephasing, 1 - n for
    gain; the constant only rescales the state) and w the bond's share of the
    site term (1/2 in the bulk, 1 at a chain end);
  * a loss jump c_k (Sec. 4.1) keeps the orbitals of span(Phi) that vanish on
    site k; a gain jump c_k^+ adds the orbital e_k; dephasing n_k = c_k^+ c_k
    does both;
  * <c_i^+ c_j> = sum_n conj(Phi_in) Phi_jn for orthonormal columns (Sec. 2.1,
    the correlation matrix of Eq. eqCorr for a pure Gaussian state).

The norm is not tracked (every observable here is normalised); after each
operation the columns are re-orthonormalised.  The jump operators are the
fermionic ones (the Jordan-Wigner string is part of c_k); spin operators
sigma^- with no string are not Gaussian in general and are not covered.
"""
import numpy as np

from . import model


def _orthonormal(Phi):
    if Phi.shape[1] == 0:
        return Phi
    Q, _ = np.linalg.qr(Phi)
    return Q


def _expm2(A):
    """exp(A) of a 2 x 2 complex matrix by its eigendecomposition (A = h1 times
    -i tau is diagonalisable except at isolated exceptional points, where the
    series below takes over)."""
    w, V = np.linalg.eig(A)
    if abs(w[0] - w[1]) > 1e-6 * max(1.0, abs(w[0])):
        return V @ np.diag(np.exp(w)) @ np.linalg.inv(V)
    out = np.eye(2, dtype=complex)
    term = np.eye(2, dtype=complex)
    for n in range(1, 40):
        term = term @ A / n
        out = out + term
    return out


class SlaterHistory:
    """One trajectory as the span of N orthonormal orbitals (columns of Phi)."""

    def __init__(self, cfg):
        if not cfg.fermionic:
            raise ValueError("the Slater reference covers fermionic jump operators only")
        self.cfg = cfg
        L = cfg.L
        occ = [i for i in range(L) if cfg.occupation[i]]
        self.Phi = np.zeros((L, len(occ)), dtype=complex)
        for n, i in enumerate(occ):
            self.Phi[i, n] = 1.0
        kappa = cfg.gamma_loss + cfg.gamma_deph - cfg.gamma_gain
        self._blocks = {}
        self._kappa = kappa

    def block(self, b, tau):
        key = (b, tau)
        if key not in self._blocks:
            cfg = self.cfg
            wl, wr = model.site_weights(cfg.L)[b]
            h1 = np.array([[-0.5j * wl * self._kappa[b], -cfg.J],
                           [-cfg.J, -0.5j * wr * self._kappa[b + 1]]], dtype=complex)
            self._blocks[key] = _expm2(-1j * tau * h1)
        return self._blocks[key]

    def apply_layer(self, parity, tau):
        for b in range(parity, self.cfg.L - 1, 2):
            self.Phi[b:b + 2, :] = self.block(b, tau) @ self.Phi[b:b + 2, :]
        self.Phi = _orthonormal(self.Phi)

    def apply_jump(self, channel):
        site, kind = divmod(int(channel), model.N_KINDS)
        L = self.cfg.L
        if kind in (model.LOSS, model.DEPHASING):
            # orbitals of span(Phi) with no weight on `site`: the null space of row `site`
            r = self.Phi[site:site + 1, :]
            if np.linalg.norm(r) == 0.0:
                raise FloatingPointError("jump on an empty site")
            _, _, Vh = np.linalg.svd(r)
            Z = Vh[1:].conj().T                   # N x (N-1), orthonormal, r Z = 0
            self.Phi = self.Phi @ Z
        if kind in (model.GAIN, model.DEPHASING):
            e = np.zeros((L, 1), dtype=complex)
            e[site, 0] = 1.0
            # c_k^+ on a state with site k empty in every orbital (after the loss part
            # of n_k, or for gain when the site is empty): add the orbital e_k
            rest = e - self.Phi @ (self.Phi.conj().T @ e)
            if np.linalg.norm(rest) < 1e-14:
                raise FloatingPointError("gain jump on a full site")
            self.Phi = np.hstack([self.Phi, e])
        self.Phi = _orthonormal(self.Phi)

    def correlation(self):
        """C_ij = <c_i^+ c_j> = sum_n conj(Phi_in) Phi_jn."""
        return self.Phi.conj() @ self.Phi.T

    def number(self):
        return self.Phi.shape[1]


def run_slater(cfg, jumps_per_traj, n_steps=None):
    """Exact (untruncated) C of each history for its recorded channels
    (jumps_per_traj [n, n_steps], -1 = Trotter layers).  Returns [n, L, L]."""
    jumps_per_traj = np.asarray(jumps_per_traj)
    n_steps = jumps_per_traj.shape[1] if n_steps is None else n_steps
    out = np.zeros((jumps_per_traj.shape[0], cfg.L, cfg.L), dtype=complex)
    for t, rec in enumerate(jumps_per_traj):
        h = SlaterHistory(cfg)
        for s in range(n_steps):
            if rec[s] >= 0:
                h.apply_jump(rec[s])
            else:
                for parity, tau in cfg.layers():
                    h.apply_layer(parity, tau)
        out[t] = h.correlation()
    return out
