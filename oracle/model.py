"""Free-fermion chain, jump channels and two-site effective-Hamiltonian gates.

Sec. 2.1 (Eq. Hamiltonian): H = -J sum_i (c_{i+1}^+ c_i + c_i^+ c_{i+1}); after a
Jordan-Wigner map the nearest-neighbour hopping carries no string, so the bond
term is h_b = -J (s+_b s-_{b+1} + s-_b s+_{b+1}) on sites (b, b+1).
Eq. EffHamiltonian: H_eff = H - (i/2) sum_k gamma_k L_k^+ L_k.  Per site the
channels are loss L = c (L^+L = n), gain L = c^+ (L^+L = 1 - n) and dephasing
L = n (L^+L = n).  The site term is shared between the two bonds that touch the
site (weight 1/2) and given whole to the single bond at a chain end (the split
the paper uses for the purified scheme, Eq. LindbladLocal).
Sec. 2.3: the two-site gate exp(-i h_b^eff tau) is a 4x4 matrix, computed here by
Taylor series with scaling and squaring.

Single-site basis: |0> empty, |1> occupied.  Two-site index s_b * 2 + s_{b+1}.
"""
import numpy as np

SIGMA_MINUS = np.array([[0, 1], [0, 0]], dtype=complex)   # |0><1| removes a particle
SIGMA_PLUS = SIGMA_MINUS.T.copy()                          # |1><0| adds a particle
NUMBER = np.diag([0.0, 1.0]).astype(complex)
PARITY = np.diag([1.0, -1.0]).astype(complex)              # (-1)^n, the Jordan-Wigner string
IDENTITY2 = np.eye(2, dtype=complex)

# jump channel kinds; channel index = 3 * site + kind
LOSS, GAIN, DEPHASING = 0, 1, 2
N_KINDS = 3


def jump_operator(kind):
    """Single-site part of L for a channel kind."""
    return {LOSS: SIGMA_MINUS, GAIN: SIGMA_PLUS, DEPHASING: NUMBER}[kind]


def has_string(kind, fermionic):
    """Loss c_k and gain c_k^+ carry the string prod_{j<k} (-1)^{n_j}; n_k does not."""
    return bool(fermionic) and kind in (LOSS, GAIN)


def site_dissipator(g_loss, g_gain, g_deph):
    """sum over the site's channels of gamma L^+L, a 2x2 diagonal matrix."""
    return (g_loss * NUMBER + g_gain * (IDENTITY2 - NUMBER) + g_deph * NUMBER)


def site_weights(L):
    """Fraction of each site's dissipator carried by each bond: w[b] = (left, right)."""
    w = []
    for b in range(L - 1):
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b + 1 == L - 1 else 0.5
        w.append((wl, wr))
    return w


def bond_heff(J, K_left, K_right, w_left, w_right):
    """h_b^eff = h_b - (i/2)(w_l K_l x 1 + w_r 1 x K_r), a 4x4 matrix."""
    hop = -J * (np.kron(SIGMA_PLUS, SIGMA_MINUS) + np.kron(SIGMA_MINUS, SIGMA_PLUS))
    damp = w_left * np.kron(K_left, IDENTITY2) + w_right * np.kron(IDENTITY2, K_right)
    return hop - 0.5j * damp


def expm_taylor(A):
    """exp(A) by scaling and squaring: halve A until its 1-norm is below 1/2,
    sum the Taylor series to convergence, then square back."""
    A = np.asarray(A, dtype=complex)
    nrm = np.abs(A).sum(axis=0).max()
    s = 0
    while nrm > 0.5:
        nrm *= 0.5
        s += 1
    X = A / (2.0 ** s)
    E = np.eye(A.shape[0], dtype=complex)
    term = np.eye(A.shape[0], dtype=complex)
    for n in range(1, 40):
        term = term @ X / n
        E = E + term
        if np.abs(term).max() < 1e-18:
            break
    for _ in range(s):
        E = E @ E
    return E


def bond_gates(L, J, tau, g_loss, g_gain, g_deph):
    """Gates G_b(tau) = exp(-i h_b^eff tau) for every bond b = 0..L-2."""
    g_loss = np.broadcast_to(np.asarray(g_loss, float), (L,))
    g_gain = np.broadcast_to(np.asarray(g_gain, float), (L,))
    g_deph = np.broadcast_to(np.asarray(g_deph, float), (L,))
    K = [site_dissipator(g_loss[i], g_gain[i], g_deph[i]) for i in range(L)]
    gates = []
    for b, (wl, wr) in enumerate(site_weights(L)):
        h = bond_heff(J, K[b], K[b + 1], wl, wr)
        gates.append(expm_taylor(-1j * tau * h))
    return gates
