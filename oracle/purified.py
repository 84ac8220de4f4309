"""Locally purified density matrix in plain FP64 (Sec. 3.2).

TEST INFRASTRUCTURE ONLY (see the package header): the product path never
imports this module.

State (Eqs. Purified, Purified1): rho = X X^+, X an MPO whose site tensors carry
a physical index n (d = 2) and a Kraus index k (chi_k values).  Here n and k are
grouped into one index s = n chi_k + k, so X is an MPS with D = 2 chi_k values
per site, held in Vidal-Hastings form like the pure states: B_i of shape
(chi_{i-1}, D, chi_i).  The product start |occ><occ| has k = 0 on every site.

One time step, the first-order splitting e^{dt Lv} ~ e^{dt Lv1} e^{dt Lv2} of
Eq. LindbladLocal, in the order the paper's summary gives (the effective
Hamiltonian sweep, then every site's R step):
1. The Trotter layers of exp(-i h_b^eff tau) (x) 1 over the Kraus indices
   (Eq. ThetaPurified: the gate does not touch k), each bond by the two-site
   update of Eq. Theta with theta of (D chi) x (D chi).  The norm is not
   enforced (H_eff is not Hermitian): B_b <- theta~ V_k, B_{b+1} <- V_k^+,
   Lambda_b <- S_k / ||S_k||; truncation keeps the chi_max largest values
   above svd_cut.  h_b^eff splits the site terms as the trajectory gates do.
2. The jump part on every site: rho -> rho + dt sum_c gamma_c L_c rho L_c^+ over
   the site's channels (loss sigma-, gain sigma+, dephasing n; the paper writes
   1 + gamma_i dt L_i (x) L_i^+ with one channel per site, and its Eq. MatrixR
   leaves out the factor gamma_i dt, which the operator carries).  It replaces
   sum_k A^{n,k} (A^{n',k})^* by the tensor R of Eq. MatrixR.  R = A~ A~^+ for
   the enlarged Kraus set A~ = [A^{.,k} ; sqrt(gamma_c dt) L_c A^{.,k}] (columns
   over k, then over the channels), so the eigenvectors of R with the chi_k
   largest eigenvalues, scaled by sqrt(lambda_k) (Eq. NewPurified), are the
   columns of A~ V_k with V_k the leading eigenvectors of the small Hermitian
   matrix A~^+ A~: the same numbers as diagonalising the d chi^2 x d chi^2 matrix
   R, which the paper does.  The R steps of different sites commute and act on
   one tensor each.
   Which chi_k directions to keep depends on the site's environment.  The paper
   diagonalises R at the site a sweep has reached, where the environment is the
   identity.  In the Vidal-Hastings form the left environment of B_i is
   Lambda_{i-1}^2 (B_i itself carries the right weights), so the kept directions
   are the leading eigenvectors of the weighted A~^+ W^2 A~ (W = Lambda_{i-1} on
   the left bond index), applied to the unweighted A~: new A = A~ V_k.  This is
   the same weighting the two-site update gives theta (theta = Lambda theta~).
   Unweighted, the local cut in this gauge is far from optimal: on a 3-site chain
   it left X X^+ 8e-2 away from the untruncated scheme at chi_k = 8, against
   5e-5 weighted (a reading: the paper works at the orthogonality centre).
Observables: <O> = Tr(O X X^+) / Tr(X X^+) = <X|O (x) 1|X> / <X|X> by exact
environment contractions; C_ij with the Jordan-Wigner string as for pure states.

Fermionic jumps: as in the MPDO, c_0 and c_{L-1} act as the local sigma-+ (the
string of site L-1 is the total parity times a one-site factor, and every state
here commutes with the parity); a bulk fermionic loss or gain raises ValueError.
"""
import numpy as np

from . import model


def check_channels(cfg):
    if not cfg.fermionic:
        return
    for i in range(1, cfg.L - 1):
        if cfg.gamma_loss[i] > 0 or cfg.gamma_gain[i] > 0:
            raise ValueError("fermionic loss/gain on bulk site %d is non-local" % i)


def full_gate(G, kraus):
    """The 4x4 gate over (n_b, n_{b+1}) times the identity on (k_b, k_{b+1}),
    as a (D^2 x D^2) matrix over (s_b, s_{b+1}), s = n kraus + k."""
    D = 2 * kraus
    I = np.eye(kraus)
    F = np.einsum('uvst,ab,cd->uavcsbtd', G.reshape(2, 2, 2, 2), I, I)
    return F.reshape(D * D, D * D)


def site_channels(cfg, i):
    """(sqrt(gamma dt), one-site L) of the channels of site i with gamma > 0,
    in the order loss, gain, dephasing."""
    out = []
    for kind, g in ((model.LOSS, cfg.gamma_loss[i]), (model.GAIN, cfg.gamma_gain[i]),
                    (model.DEPHASING, cfg.gamma_deph[i])):
        if g > 0:
            out.append((np.sqrt(g * cfg.dt), model.jump_operator(kind)))
    return out


class Purified:
    def __init__(self, cfg, kraus):
        self.cfg = cfg
        self.kraus = int(kraus)
        self.D = 2 * self.kraus
        self.B = []
        for i in range(cfg.L):
            t = np.zeros((1, self.D, 1), dtype=complex)
            t[0, int(cfg.occupation[i]) * self.kraus, 0] = 1.0
            self.B.append(t)
        self.lam = [np.ones(1) for _ in range(cfg.L - 1)]
        self.trunc_weight = 0.0

    def bond_dims(self):
        return [len(x) for x in self.lam]

    def left_weight(self, b):
        return self.lam[b - 1] if b > 0 else np.ones(1)

    # ---- Eq. ThetaPurified: the two-site update over s = (n, k), norm kept -----------
    def update_bond(self, b, G):
        cfg, D = self.cfg, self.D
        Bl, Br = self.B[b], self.B[b + 1]
        chiL, chiR = Bl.shape[0], Br.shape[2]
        P = np.tensordot(Bl, Br, axes=(2, 0))                    # [a, s, t, c]
        tt = np.einsum('uvst,astc->auvc', G.reshape(D, D, D, D), P).reshape(chiL * D, D * chiR)
        th = tt * np.repeat(self.left_weight(b), D)[:, None]
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
        self.B[b + 1] = Vk_h.reshape(k, D, chiR).copy()
        self.B[b] = (tt @ Vk_h.conj().T).reshape(chiL, D, k)
        self.lam[b] = S[:k] / norm

    def apply_layer(self, parity, gates):
        for b in range(parity, self.cfg.L - 1, 2):
            self.update_bond(b, gates[b])

    # ---- Eqs. MatrixR, NewPurified: the jump part on one site ----------------------
    def enlarged_kraus(self, i):
        """A~ as a matrix: rows (a, n, c), columns p kraus + k for the operators
        p = 0 (identity), 1.. (sqrt(gamma dt) L_c of the site's channels)."""
        K = self.kraus
        A = self.B[i].reshape(self.B[i].shape[0], 2, K, self.B[i].shape[2])
        ops = [(1.0, np.eye(2))] + site_channels(self.cfg, i)
        cols = []
        for a, O in ops:
            OA = a * np.einsum('nm,amkc->ankc', O, A)
            for k in range(K):
                cols.append(OA[:, :, k, :].reshape(-1))
        return np.stack(cols, axis=1)

    def kraus_step(self, i):
        K = self.kraus
        chiL, chiR = self.B[i].shape[0], self.B[i].shape[2]
        M = self.enlarged_kraus(i)
        Mw = M * np.repeat(self.left_weight(i), 2 * chiR)[:, None]   # rows (a, n, c)
        lam, V = np.linalg.eigh(Mw.conj().T @ Mw)
        order = np.argsort(lam)[::-1][:K]
        new = M @ V[:, order]                                      # (chiL 2 chiR) x K
        A = new.reshape(chiL, 2, chiR, K).transpose(0, 1, 3, 2)    # [a, n, k, c]
        self.B[i] = A.reshape(chiL, 2 * K, chiR).copy()

    def kraus_steps(self):
        for i in range(self.cfg.L):
            self.kraus_step(i)

    # ---- expectation values ----------------------------------------------------------
    def environments(self):
        L = self.cfg.L
        Lenv = [None] * (L + 1)
        Renv = [None] * (L + 1)
        Lenv[0] = np.ones((1, 1), dtype=complex)
        Renv[L] = np.ones((1, 1), dtype=complex)
        for i in range(L):
            Bi = self.B[i]
            Lenv[i + 1] = sum(Bi[:, s, :].conj().T @ Lenv[i] @ Bi[:, s, :] for s in range(self.D))
        for i in range(L - 1, -1, -1):
            Bi = self.B[i]
            Renv[i] = sum(Bi[:, s, :] @ Renv[i + 1] @ Bi[:, s, :].conj().T for s in range(self.D))
        return Lenv, Renv

    def trace(self):
        """Tr(X X^+) = <X|X>."""
        return float(np.real(self.environments()[1][0][0, 0]))

    def density(self):
        L, K = self.cfg.L, self.kraus
        Lenv, Renv = self.environments()
        nrm = np.real(Renv[0][0, 0])
        out = np.empty(L)
        for i in range(L):
            acc = 0.0
            for k in range(K):
                B1 = self.B[i][:, K + k, :]
                acc += np.real(np.sum(B1.conj() * (Lenv[i] @ B1 @ Renv[i + 1])))
            out[i] = acc / nrm
        return out

    def correlation(self):
        L, K = self.cfg.L, self.kraus
        Lenv, Renv = self.environments()
        nrm = np.real(Renv[0][0, 0])
        C = np.zeros((L, L), dtype=complex)
        C[np.diag_indices(L)] = self.density()
        for i in range(L):
            Bi = self.B[i]
            # s+_i: bra n = 1, ket n = 0, the same Kraus index on both sides
            E = sum(Bi[:, K + k, :].conj().T @ Lenv[i] @ Bi[:, k, :] for k in range(K))
            for j in range(i + 1, L):
                Bj = self.B[j]
                C[i, j] = sum(np.sum(Bj[:, k, :].conj() * (E @ Bj[:, K + k, :] @ Renv[j + 1]))
                              for k in range(K)) / nrm
                C[j, i] = np.conj(C[i, j])
                E = sum(Bj[:, k, :].conj().T @ E @ Bj[:, k, :]
                        - Bj[:, K + k, :].conj().T @ E @ Bj[:, K + k, :] for k in range(K))
        return C

    def to_dense(self):
        """rho = X X^+ as a 2^L x 2^L matrix (site 0 most significant)."""
        L, K = self.cfg.L, self.kraus
        v = self.B[0].reshape(self.D, -1)
        for i in range(1, L):
            Bi = self.B[i]
            v = (v @ Bi.reshape(Bi.shape[0], -1)).reshape(-1, Bi.shape[2])
        T = v.reshape([2, K] * L)                       # n_0 k_0 n_1 k_1 ...
        T = T.transpose(list(range(0, 2 * L, 2)) + list(range(1, 2 * L, 2)))
        X = T.reshape(2 ** L, K ** L)
        return X @ X.conj().T


def run_purified(cfg, kraus, n_steps, measure_corr=False, state=None):
    """n_steps of (Trotter layers, then the R step on every site)."""
    check_channels(cfg)
    m = Purified(cfg, kraus) if state is None else state
    gates = {}
    for _ in range(n_steps):
        for parity, tau in cfg.layers():
            if tau not in gates:
                gates[tau] = [full_gate(G, kraus) for G in cfg.gates(tau)]
            m.apply_layer(parity, gates[tau])
        m.kraus_steps()
    out = {"state": m, "density": m.density(), "bond_dims": m.bond_dims(),
           "trunc_weight": m.trunc_weight, "trace": m.trace()}
    if measure_corr:
        out["corr"] = m.correlation()
    return out
