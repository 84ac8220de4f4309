"""Vectorised density matrix (MPDO) integrator in plain FP64 (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see the package header): the product path never
imports this module.

Vectorisation (Eq. Choi): rho = sum_ij rho_ij |i><j| becomes the vector
|rho>> = sum_ij rho_ij |i> (x) |j>.  With that map rho -> A rho B becomes the
matrix A (x) B^T, so the Lindblad equation (Eq. LindbladChoi) has the generator

  Lv = -i (H (x) 1 - 1 (x) H^T)
       + sum_k gamma_k [ L_k (x) conj(L_k) - 1/2 L_k^+L_k (x) 1 - 1/2 1 (x) (L_k^+L_k)^T ].

Eq. Liouvillian prints L_k (x) L_k^+ and 1 (x) H; the conjugate and transpose
above are what the map gives for L rho L^+ and rho H (the printed form would
send rho to c rho c, whose trace is zero, so it cannot preserve the trace).
Below every superoperator is built as "rho -> A rho B" (`superop`), which is the
definition itself; the (x) forms follow from it.

Local basis (Eq. MPDO): per site the ket index n and the bra index n' are
grouped into m = 2 n + n' (d = 2, d^2 = 4 values), so |rho>> is an MPS with
four physical values per site.  Vector index: sum_i m_i 4^(L-1-i).

Per bond (the TEBD split of Sec. 2.3, with the site terms shared as in the
trajectory gates: half a bulk site's dissipator on each of its two bonds, the
whole of an end site's on its one bond):
  Lv_b = -i [h_b, .] + w_l D_b (x) id + w_r id (x) D_{b+1},
  D_i rho = sum_k gamma_k (L_k rho L_k^+ - 1/2 {L_k^+L_k, rho})  on site i,
and the gate is exp(tau Lv_b), a 16 x 16 matrix over (m_b, m_{b+1}).

Jump operators per site: loss sigma-, gain sigma+, dephasing n.  With
fermionic jumps, loss and gain carry the Jordan-Wigner string and are accepted
on the two chain ends only: c_0 has no string, and the string of site L-1 is
the total parity P times a one-site factor ((-1)^n sigma- = sigma-,
(-1)^n sigma+ = -sigma+), so c rho c^+ = P sigma- rho sigma+ P, which equals
sigma- rho sigma+ whenever rho commutes with P.  Every state here does: the
initial states are diagonal in the occupation basis, and the hopping and each
site dissipator preserve [rho, P] = 0.  (The paper writes the sink of the
source/sink chain in exactly this string form, Sec. 2.1.)  A bulk fermionic
loss or gain raises ValueError.

State update (Eq. Theta in the Hastings form, as for pure states): theta~ =
G (B_b B_{b+1}), theta = Lambda_{b-1} theta~, SVD, keep k values,
B_{b+1} <- V_k^+, B_b <- theta~ V_k / ||S_k||, Lambda_b <- S_k / ||S_k||.
Truncation keeps the largest values as for pure states, except that it never
splits a multiplet of equal singular values: rho = rho^+ maps the coherences of
particle-number difference q onto those of -q, so the Schmidt spectrum of
|rho>> holds exactly degenerate pairs, and keeping one member of a pair would
pick an arbitrary vector of the pair and leave a non-Hermitian rho.  k is
lowered while S_{k-1} - S_k <= MULTIPLET_TOL S_0 (the paper is silent on this;
it is a reading).  The
scale of |rho>> is thereby not tracked (the renormalisation fixes its
Hilbert-Schmidt norm, not its trace), so every observable is a ratio
Tr(O rho) / Tr rho.

Traces: for a product operator O = (x)_i O_i,
Tr(O rho) = sum_{n,n'} O[n', n] rho[n, n'] is the contraction of |rho>> with the
site vectors o_i[2n + n'] = O_i[n', n]: identity (1,0,0,1), n (0,0,0,1),
sigma+ = |1><0| (0,1,0,0), sigma- = |0><1| (0,0,1,0), parity (1,0,0,-1).
C_ij = Tr(c_i^+ c_j rho) / Tr rho = Tr(s+_i prod_{i<l<j} (-1)^{n_l} s-_j rho) /
Tr rho for i < j, C_ji = conj(C_ij), C_ii = <n_i>.
"""
import numpy as np

from . import model

E_ID = np.array([1.0, 0.0, 0.0, 1.0], dtype=complex)
E_N = np.array([0.0, 0.0, 0.0, 1.0], dtype=complex)
E_SPLUS = np.array([0.0, 1.0, 0.0, 0.0], dtype=complex)
E_SMINUS = np.array([0.0, 0.0, 1.0, 0.0], dtype=complex)
E_PARITY = np.array([1.0, 0.0, 0.0, -1.0], dtype=complex)

# singular values closer than this (relative to the largest) count as one multiplet
MULTIPLET_TOL = 1e-9


def keep_multiplets(S, k, tol=MULTIPLET_TOL):
    """Largest k' <= k (at least 1) whose cut does not split a multiplet of the
    descending singular values S."""
    while 1 < k < len(S) and S[k - 1] - S[k] <= tol * S[0]:
        k -= 1
    return k


def superop(A, B):
    """Matrix of rho -> A rho B on `ns` sites in the site-grouped basis
    (m_0, ..., m_{ns-1}), m = 2 n + n'.  A and B are 2^ns x 2^ns."""
    ns = int(round(np.log2(A.shape[0])))
    dims = [2] * ns
    # S[(n, n'), (k, k')] = A[n, k] B[k', n'] over multi-indices n = (n_0..), ...
    S = np.einsum('ac,db->abcd', A, B)          # a = n, b = n', c = k, d = k'
    S = S.reshape(dims * 4)
    # axes: n_0..n_{ns-1}, n'_0.., k_0.., k'_0..  ->  (n_0 n'_0 n_1 n'_1 ..), (k_0 k'_0 ..)
    out_axes = [x for i in range(ns) for x in (i, ns + i)]
    in_axes = [x for i in range(ns) for x in (2 * ns + i, 3 * ns + i)]
    return S.transpose(out_axes + in_axes).reshape(4 ** ns, 4 ** ns)


def site_jump_ops(g_loss, g_gain, g_deph):
    """(rate, one-site L_k) of one site's channels with non-zero rate."""
    out = []
    for kind, g in ((model.LOSS, g_loss), (model.GAIN, g_gain), (model.DEPHASING, g_deph)):
        if g > 0:
            out.append((g, model.jump_operator(kind)))
    return out


def dissipator_superop(ops, ns=1, where=0):
    """D rho = sum_k gamma_k (L rho L^+ - 1/2 L^+L rho - 1/2 rho L^+L) with the
    one-site L_k of `ops` placed on site `where` of `ns` sites."""
    dim = 2 ** ns
    S = np.zeros((4 ** ns, 4 ** ns), dtype=complex)
    one = np.eye(dim, dtype=complex)
    for g, Lk in ops:
        Lf = np.kron(np.kron(np.eye(2 ** where), Lk), np.eye(2 ** (ns - where - 1)))
        LdL = Lf.conj().T @ Lf
        S += g * (superop(Lf, Lf.conj().T) - 0.5 * superop(LdL, one) - 0.5 * superop(one, LdL))
    return S


def check_channels(cfg):
    """Bulk fermionic loss or gain would need the string inside the bond
    superoperators; only the chain ends reduce to local operators."""
    if not cfg.fermionic:
        return
    for i in range(1, cfg.L - 1):
        if cfg.gamma_loss[i] > 0 or cfg.gamma_gain[i] > 0:
            raise ValueError("fermionic loss/gain on bulk site %d is non-local" % i)


def bond_liouvillian(cfg, b):
    """Lv_b (16 x 16) of bond b: the hopping commutator plus the weighted site
    dissipators of sites b and b+1."""
    L = cfg.L
    J = cfg.J
    hop = -J * (np.kron(model.SIGMA_PLUS, model.SIGMA_MINUS)
                + np.kron(model.SIGMA_MINUS, model.SIGMA_PLUS))
    one = np.eye(4, dtype=complex)
    S = superop(-1j * hop, one) + superop(one, 1j * hop)     # -i (h rho - rho h)
    wl, wr = model.site_weights(L)[b]
    for site, w, where in ((b, wl, 0), (b + 1, wr, 1)):
        ops = site_jump_ops(cfg.gamma_loss[site], cfg.gamma_gain[site], cfg.gamma_deph[site])
        S += w * dissipator_superop(ops, ns=2, where=where)
    return S


def bond_gates(cfg, tau):
    """exp(tau Lv_b) for every bond (16 x 16 each)."""
    return [model.expm_taylor(tau * bond_liouvillian(cfg, b)) for b in range(cfg.L - 1)]


class MPDO:
    """|rho>> in Vidal-Hastings form: B_i of shape (chi_{i-1}, 4, chi_i)."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.B = []
        for i in range(cfg.L):
            t = np.zeros((1, 4, 1), dtype=complex)
            t[0, 3 * int(cfg.occupation[i]), 0] = 1.0   # |n><n| has m = 2n + n = 3n
            self.B.append(t)
        self.lam = [np.ones(1) for _ in range(cfg.L - 1)]
        self.trunc_weight = 0.0

    def bond_dims(self):
        return [len(x) for x in self.lam]

    def left_weight(self, b):
        return self.lam[b - 1] if b > 0 else np.ones(1)

    def update_bond(self, b, G):
        cfg = self.cfg
        Bl, Br = self.B[b], self.B[b + 1]
        chiL, chiR = Bl.shape[0], Br.shape[2]
        P = np.tensordot(Bl, Br, axes=(2, 0))                   # [a, m, n, c]
        tt = np.einsum('uvst,astc->auvc', G.reshape(4, 4, 4, 4), P)
        tt = tt.reshape(chiL * 4, 4 * chiR)                      # theta~
        th = tt * np.repeat(self.left_weight(b), 4)[:, None]     # theta
        U, S, Vh = np.linalg.svd(th, full_matrices=False)
        if not S[0] > 0.0:
            raise FloatingPointError("theta vanished at bond %d" % b)
        k = int(np.count_nonzero(S > cfg.svd_cut * S[0]))
        k = keep_multiplets(S, max(1, min(cfg.chi_max, k)))
        total = float(np.sum(S ** 2))
        kept = float(np.sum(S[:k] ** 2))
        norm = np.sqrt(kept)
        self.trunc_weight += (total - kept) / total
        Vk_h = Vh[:k]
        self.B[b + 1] = Vk_h.reshape(k, 4, chiR).copy()
        self.B[b] = (tt @ Vk_h.conj().T / norm).reshape(chiL, 4, k)
        self.lam[b] = S[:k] / norm

    def apply_layer(self, parity, gates):
        for b in range(parity, self.cfg.L - 1, 2):
            self.update_bond(b, gates[b])

    # ---- traces -------------------------------------------------------------------
    def _T(self, i, o):
        """sum_m o[m] B_i[:, m, :]"""
        return np.tensordot(self.B[i], o, axes=(1, 0))

    def trace_vectors(self):
        """left[i] = contraction of sites < i with the identity vectors (a row),
        right[i] = of sites >= i (a column); left[L] = right[0] = Tr rho."""
        L = self.cfg.L
        left = [None] * (L + 1)
        right = [None] * (L + 1)
        left[0] = np.ones(1, dtype=complex)
        right[L] = np.ones(1, dtype=complex)
        for i in range(L):
            left[i + 1] = left[i] @ self._T(i, E_ID)
        for i in range(L - 1, -1, -1):
            right[i] = self._T(i, E_ID) @ right[i + 1]
        return left, right

    def trace(self):
        return complex(self.trace_vectors()[0][self.cfg.L][0])

    def density(self):
        left, right = self.trace_vectors()
        tr = left[self.cfg.L][0]
        return np.array([np.real(left[i] @ self._T(i, E_N) @ right[i + 1] / tr)
                         for i in range(self.cfg.L)])

    def correlation(self):
        L = self.cfg.L
        left, right = self.trace_vectors()
        tr = left[L][0]
        C = np.zeros((L, L), dtype=complex)
        C[np.diag_indices(L)] = self.density()
        for i in range(L):
            v = left[i] @ self._T(i, E_SPLUS)
            for j in range(i + 1, L):
                C[i, j] = v @ self._T(j, E_SMINUS) @ right[j + 1] / tr
                C[j, i] = np.conj(C[i, j])
                v = v @ self._T(j, E_PARITY)
        return C

    def to_dense(self):
        """rho as a 2^L x 2^L matrix (site 0 most significant on both sides)."""
        L = self.cfg.L
        v = self.B[0].reshape(4, -1)
        for i in range(1, L):
            Bi = self.B[i]
            v = (v @ Bi.reshape(Bi.shape[0], -1)).reshape(-1, Bi.shape[2])
        T = v.reshape([2] * (2 * L))                    # n_0 n'_0 n_1 n'_1 ...
        T = T.transpose(list(range(0, 2 * L, 2)) + list(range(1, 2 * L, 2)))
        return T.reshape(2 ** L, 2 ** L)


def current(C):
    """<j_i> = i (C_{i,i-1} - C_{i-1,i}) for i = 1..L-1 (Sec. 2.1)."""
    L = C.shape[0]
    return np.array([np.real(1j * (C[i, i - 1] - C[i - 1, i])) for i in range(1, L)])


def run_mpdo(cfg, n_steps, measure_corr=False, state=None):
    """n_steps Trotter steps of cfg.layers() from the product state (or from
    `state`, which is advanced in place).  Returns a dict with the MPDO, its
    density, correlation (optional), bond dims and discarded weight."""
    check_channels(cfg)
    m = MPDO(cfg) if state is None else state
    gates = {}
    for _ in range(n_steps):
        for parity, tau in cfg.layers():
            if tau not in gates:
                gates[tau] = bond_gates(cfg, tau)
            m.apply_layer(parity, gates[tau])
    out = {"state": m, "density": m.density(), "bond_dims": m.bond_dims(),
           "trunc_weight": m.trunc_weight}
    if measure_corr:
        out["corr"] = m.correlation()
    return out
