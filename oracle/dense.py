"""Brute-force references on the full 2^L Hilbert space (small L only).

dense_trajectory   the same Trotterised, jump-or-evolve history as the MPS
                   integrator, on the full state vector, with no truncation.
lindblad_rk4       the Lindblad equation (Eq. Lindblad) for rho (2^L x 2^L),
                   integrated by classical RK4.
corr_rk4           the closed linear equation of motion of C_ij = <c_i^+ c_j>
                   (Eq. eqCorr, generalised to loss, gain and dephasing on every
                   site), integrated by RK4.
corr_uniform_loss  its closed form for uniform loss gamma and no gain or
                   dephasing: C(t) = exp(-gamma t) U C(0) U^+, U = exp(-i A t),
                   with A = J x adjacency (Eq. SoleqCorr with Gamma = 0).
dense_qsd          a quantum-state-diffusion history (Sec. 5.2) on the full
                   vector: the same Trotter layers and noise operators as the
                   MPS integrator, unnormalised.
qsd_mean_map       the exact noise average of one QSD step on rho: E[eta] = 0
                   and E[eta^2] = 1 turn each factor 1 + eta a L into
                   rho -> rho + a^2 L rho L^+, applied channel by channel.
Basis index: sum_i s_i 2^(L-1-i) (site 0 most significant).
"""
import numpy as np

from . import model


def site_op(L, i, O):
    return np.kron(np.kron(np.eye(2 ** i), O), np.eye(2 ** (L - i - 1)))


def bond_op(L, b, G):
    return np.kron(np.kron(np.eye(2 ** b), G), np.eye(2 ** (L - b - 2)))


def fermion_annihilator(L, i, fermionic=True):
    """c_i = (prod_{j<i} (-1)^{n_j}) s-_i (Jordan-Wigner)."""
    op = np.eye(1)
    for j in range(L):
        if j < i:
            f = model.PARITY if fermionic else model.IDENTITY2
        elif j == i:
            f = model.SIGMA_MINUS
        else:
            f = model.IDENTITY2
        op = np.kron(op, f)
    return op


def jump_ops(L, g_loss, g_gain, g_deph, fermionic=True):
    """List of (rate, L_k) for every channel with non-zero rate."""
    ops = []
    for i in range(L):
        c = fermion_annihilator(L, i, fermionic)
        if g_loss[i] > 0:
            ops.append((g_loss[i], c))
        if g_gain[i] > 0:
            ops.append((g_gain[i], c.conj().T))
        if g_deph[i] > 0:
            ops.append((g_deph[i], site_op(L, i, model.NUMBER)))
    return ops


def hamiltonian(L, J):
    H = np.zeros((2 ** L, 2 ** L), dtype=complex)
    hop = -J * (np.kron(model.SIGMA_PLUS, model.SIGMA_MINUS)
                + np.kron(model.SIGMA_MINUS, model.SIGMA_PLUS))
    for b in range(L - 1):
        H += bond_op(L, b, hop)
    return H


def product_state(L, occupation):
    idx = 0
    for i in range(L):
        idx = idx * 2 + int(occupation[i])
    v = np.zeros(2 ** L, dtype=complex)
    v[idx] = 1.0
    return v


def dense_trajectory(cfg, jumps):
    """Full-vector history with the given channel record (-1 = Trotter step)."""
    L = cfg.L
    layer_ops = []
    for parity, tau in cfg.layers():
        gates = cfg.gates(tau)
        op = np.eye(2 ** L, dtype=complex)
        for b in range(parity, L - 1, 2):
            op = bond_op(L, b, gates[b]) @ op
        layer_ops.append(op)
    psi = product_state(L, cfg.occupation)
    for ch in jumps:
        if ch >= 0:
            site, kind = divmod(int(ch), model.N_KINDS)
            op = site_op(L, site, model.jump_operator(kind))
            if model.has_string(kind, cfg.fermionic):
                for j in range(site):
                    op = site_op(L, j, model.PARITY) @ op
            psi = op @ psi
        else:
            for op in layer_ops:
                psi = op @ psi
        psi = psi / np.linalg.norm(psi)
    return psi


def dense_correlation(L, psi_or_rho, fermionic=True):
    """C_ij = <c_i^+ c_j> of a state vector or density matrix."""
    cs = [fermion_annihilator(L, i, fermionic) for i in range(L)]
    C = np.zeros((L, L), dtype=complex)
    x = psi_or_rho
    for i in range(L):
        for j in range(L):
            op = cs[i].conj().T @ cs[j]
            if x.ndim == 1:
                C[i, j] = np.vdot(x, op @ x)
            else:
                C[i, j] = np.trace(op @ x)
    return C


def lindblad_rhs(H, ops, rho):
    """-i[H, rho] + sum_k gamma_k (L rho L^+ - 1/2 {L^+L, rho})  (Eq. Lindblad)."""
    out = -1j * (H @ rho - rho @ H)
    for g, Lk in ops:
        LdL = Lk.conj().T @ Lk
        out += g * (Lk @ rho @ Lk.conj().T - 0.5 * (LdL @ rho + rho @ LdL))
    return out


def lindblad_rk4(L, J, g_loss, g_gain, g_deph, rho0, t_end, h, fermionic=True):
    H = hamiltonian(L, J)
    ops = jump_ops(L, g_loss, g_gain, g_deph, fermionic)
    n = int(round(t_end / h))
    rho = rho0.astype(complex)
    for _ in range(n):
        k1 = lindblad_rhs(H, ops, rho)
        k2 = lindblad_rhs(H, ops, rho + 0.5 * h * k1)
        k3 = lindblad_rhs(H, ops, rho + 0.5 * h * k2)
        k4 = lindblad_rhs(H, ops, rho + h * k3)
        rho = rho + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return rho


def adjacency(L, J):
    A = np.zeros((L, L))
    for i in range(L - 1):
        A[i, i + 1] = A[i + 1, i] = J
    return A


def corr_rhs(Heff, Gam, gd, C):
    """dC/dt = -i Heff C + i C Heff^+ + Gamma - dephasing on the off-diagonal."""
    out = -1j * (Heff @ C) + 1j * (C @ Heff.conj().T) + Gam
    D = 0.5 * (gd[:, None] + gd[None, :])
    np.fill_diagonal(D, 0.0)
    return out - D * C


def corr_rk4(L, J, g_loss, g_gain, g_deph, C0, t_end, h):
    """Eq. eqCorr with H^eff = J adj - (i/2) diag(g_loss + g_gain), Gamma =
    diag(g_gain); dephasing L = n damps C_ij (i != j) at (g_i + g_j)/2."""
    g_loss = np.asarray(g_loss, float)
    g_gain = np.asarray(g_gain, float)
    g_deph = np.asarray(g_deph, float)
    Heff = adjacency(L, J) - 0.5j * np.diag(g_loss + g_gain)
    Gam = np.diag(g_gain).astype(complex)
    n = int(round(t_end / h))
    C = C0.astype(complex)
    for _ in range(n):
        k1 = corr_rhs(Heff, Gam, g_deph, C)
        k2 = corr_rhs(Heff, Gam, g_deph, C + 0.5 * h * k1)
        k3 = corr_rhs(Heff, Gam, g_deph, C + 0.5 * h * k2)
        k4 = corr_rhs(Heff, Gam, g_deph, C + h * k3)
        C = C + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return C


def corr_uniform_loss(L, J, gamma, C0, t):
    """C(t) = exp(-gamma t) U C(0) U^+ with U = exp(-i A t); the open-chain
    adjacency has eigenvectors sqrt(2/(L+1)) sin(pi q a/(L+1)) and eigenvalues
    2 J cos(pi q/(L+1)), q = 1..L."""
    a = np.arange(1, L + 1)
    q = np.arange(1, L + 1)
    V = np.sqrt(2.0 / (L + 1)) * np.sin(np.pi * np.outer(a, q) / (L + 1))
    eps = 2.0 * J * np.cos(np.pi * q / (L + 1))
    U = (V * np.exp(-1j * eps * t)) @ V.T
    return np.exp(-gamma * t) * (U @ C0 @ U.conj().T)


def _layer_ops(cfg):
    L = cfg.L
    ops = []
    for parity, tau in cfg.layers():
        gates = cfg.gates(tau)
        op = np.eye(2 ** L, dtype=complex)
        for b in range(parity, L - 1, 2):
            op = bond_op(L, b, gates[b]) @ op
        ops.append(op)
    return ops


def _qsd_site_factors(cfg, site):
    """[(a, L_k)] of one site in the order the factors are applied (loss, gain,
    dephasing), a = sqrt(gamma_k dt); L_k acts on that site only."""
    gam = (cfg.gamma_loss[site], cfg.gamma_gain[site], cfg.gamma_deph[site])
    out = []
    for kind in (model.LOSS, model.GAIN, model.DEPHASING):
        if gam[kind] > 0:
            out.append((np.sqrt(gam[kind] * cfg.dt), site_op(cfg.L, site, model.jump_operator(kind))))
    return out


def dense_qsd(cfg, traj_id, n_steps, psi0=None):
    """Unnormalised QSD history on the full vector with the Philox noise of
    (traj_id, step); returns psi (its squared norm is the weight w)."""
    from .philox import noise
    L = cfg.L
    layers = _layer_ops(cfg)
    psi = product_state(L, cfg.occupation) if psi0 is None else psi0.copy()
    for step in range(n_steps):
        for op in layers:
            psi = op @ psi
        eta = noise(cfg.seed, traj_id, step, 3 * L)
        for i in range(L):
            kinds = [k for k, g in ((model.LOSS, cfg.gamma_loss[i]), (model.GAIN, cfg.gamma_gain[i]),
                                    (model.DEPHASING, cfg.gamma_deph[i])) if g > 0]
            for kind, (a, Lk) in zip(kinds, _qsd_site_factors(cfg, i)):
                psi = psi + eta[3 * i + kind] * a * (Lk @ psi)
    return psi


def qsd_mean_map(cfg, rho0, n_steps):
    """rho_bar after n_steps exact noise-averaged QSD steps (see module doc)."""
    layers = _layer_ops(cfg)
    rho = rho0.copy()
    for _ in range(n_steps):
        for op in layers:
            rho = op @ rho @ op.conj().T
        for i in range(cfg.L):
            for a, Lk in _qsd_site_factors(cfg, i):
                rho = rho + a * a * (Lk @ rho @ Lk.conj().T)
    return rho
