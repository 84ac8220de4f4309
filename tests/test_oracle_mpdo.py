"""Pins of the vectorised-density-matrix (MPDO) oracle (Sec. 3.1) against
things other than itself: the definition of the vectorisation (rho -> A rho B
is a matrix on |rho>>), the dense Lindblad generator (Eq. Lindblad) written
with 2^L x 2^L matrices, trace and hermiticity preservation of every gate,
the dense product of the same gates, second-order convergence of the Strang
step to the Lindblad solution, the closed equation of motion of C_ij for the
paper's source/sink chain (Eq. eqCorr), positivity of the untruncated state
and the best rank-k approximation of one truncated bond (Eckart-Young)."""
import numpy as np
import pytest

import workloads
from oracle import dense, model, mpdo, tebd


def vec(rho):
    """Site-grouped |rho>>: index sum_i (2 n_i + n'_i) 4^(L-1-i)."""
    L = int(round(np.log2(rho.shape[0])))
    T = rho.reshape([2] * (2 * L))
    axes = [x for i in range(L) for x in (i, L + i)]
    return T.transpose(axes).reshape(-1)


def unvec(v):
    L = int(round(np.log(v.size) / np.log(4)))
    T = v.reshape([2] * (2 * L))
    T = T.transpose(list(range(0, 2 * L, 2)) + list(range(1, 2 * L, 2)))
    return T.reshape(2 ** L, 2 ** L)


def cfg_of(L, dt=0.05, chi=64, loss=0.0, gain=0.0, deph=0.0, fermionic=False, occ="domain_wall",
           order=2):
    return tebd.TrajectoryConfig(L, J=1.0, dt=dt, chi_max=chi, svd_cut=1e-14, gamma_loss=loss,
                                 gamma_gain=gain, gamma_deph=deph, fermionic=fermionic,
                                 trotter_order=order, occupation=workloads.occupation(L, occ))


def rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def full_generator(cfg):
    """sum_b of every bond Liouvillian embedded in the 4^L space."""
    L = cfg.L
    S = np.zeros((4 ** L, 4 ** L), dtype=complex)
    for b in range(L - 1):
        S += np.kron(np.kron(np.eye(4 ** b), mpdo.bond_liouvillian(cfg, b)), np.eye(4 ** (L - b - 2)))
    return S


def dense_rhs(cfg, rho):
    H = dense.hamiltonian(cfg.L, cfg.J)
    ops = dense.jump_ops(cfg.L, cfg.gamma_loss, cfg.gamma_gain, cfg.gamma_deph, cfg.fermionic)
    return dense.lindblad_rhs(H, ops, rho)


def test_superop_is_the_matrix_of_a_rho_b():
    rng = np.random.default_rng(1)
    for ns in (1, 2, 3):
        d = 2 ** ns
        A, B, rho = rand_c(rng, d, d), rand_c(rng, d, d), rand_c(rng, d, d)
        assert np.allclose(mpdo.superop(A, B) @ vec(rho), vec(A @ rho @ B), atol=1e-12)
    assert np.allclose(unvec(vec(rho)), rho)


def test_bond_generators_sum_to_the_dense_lindbladian():
    # spin jumps with unequal rates on every site: the matrices must agree exactly
    rng = np.random.default_rng(2)
    L = 4
    cfg = cfg_of(L, loss=rng.uniform(0.1, 0.9, L), gain=rng.uniform(0.1, 0.9, L),
                 deph=rng.uniform(0.1, 0.9, L))
    S = full_generator(cfg)
    M = np.zeros_like(S)
    for col in range(4 ** L):
        e = np.zeros(4 ** L, dtype=complex)
        e[col] = 1.0
        M[:, col] = vec(dense_rhs(cfg, unvec(e)))
    assert np.abs(S - M).max() < 1e-13


def test_fermionic_chain_ends_act_locally_on_parity_symmetric_states():
    # source c_0^+ and sink c_{L-1} with the string (Sec. 2.1), dephasing in the
    # bulk: equal to the dense generator on every rho that commutes with the parity
    rng = np.random.default_rng(3)
    L = 4
    loss = np.zeros(L)
    gain = np.zeros(L)
    loss[-1], gain[0] = 0.7, 0.4
    loss[0] = 0.3                      # c_0 has no string either
    cfg = cfg_of(L, loss=loss, gain=gain, deph=0.25, fermionic=True)
    S = full_generator(cfg)
    par = np.diag([(-1) ** bin(s).count("1") for s in range(2 ** L)]).astype(complex)
    for _ in range(3):
        X = rand_c(rng, 2 ** L, 2 ** L)
        rho = X @ X.conj().T
        rho = 0.5 * (rho + par @ rho @ par)          # commutes with the parity
        assert np.abs(unvec(S @ vec(rho)) - dense_rhs(cfg, rho)).max() < 1e-12
    # and the string matters off that sector
    X = rand_c(rng, 2 ** L, 2 ** L)
    rho = X @ X.conj().T
    assert np.abs(unvec(S @ vec(rho)) - dense_rhs(cfg, rho)).max() > 1e-3


def test_bulk_fermionic_loss_is_rejected():
    cfg = cfg_of(5, loss=0.1, fermionic=True)
    with pytest.raises(ValueError):
        mpdo.run_mpdo(cfg, 1)


def test_gates_preserve_trace_and_hermiticity():
    L = 5
    cfg = cfg_of(L, loss=[0.3, 0.1, 0.2, 0.1, 0.5], gain=0.15, deph=0.2)
    ee = np.kron(mpdo.E_ID, mpdo.E_ID)
    swap = np.zeros((4, 4))
    for n in range(2):
        for n2 in range(2):
            swap[2 * n2 + n, 2 * n + n2] = 1.0
    SW = np.kron(swap, swap)
    for G in mpdo.bond_gates(cfg, 0.07):
        assert np.abs(ee @ G - ee).max() < 1e-14             # Tr(G rho) = Tr rho
        assert np.abs(SW @ G.conj() @ SW - G).max() < 1e-14  # (G rho)^+ = G rho^+


def dense_trotter(cfg, n_steps, rho0):
    L = cfg.L
    v = vec(rho0).astype(complex)
    for _ in range(n_steps):
        for parity, tau in cfg.layers():
            gates = mpdo.bond_gates(cfg, tau)
            for b in range(parity, L - 1, 2):
                v = np.kron(np.kron(np.eye(4 ** b), gates[b]), np.eye(4 ** (L - b - 2))) @ v
    return unvec(v)


def test_untruncated_mpdo_equals_the_dense_gate_product():
    L, steps = 5, 6
    cfg = cfg_of(L, dt=0.08, loss=0.3, gain=0.1, deph=0.2, occ="neel")
    res = mpdo.run_mpdo(cfg, steps, measure_corr=True)
    m = res["state"]
    psi0 = dense.product_state(L, cfg.occupation)
    want = dense_trotter(cfg, steps, np.outer(psi0, psi0.conj()))
    got = m.to_dense()
    tr = np.trace(got)
    assert abs(tr - m.trace()) < 1e-12 * abs(tr)
    assert np.abs(got / tr - want / np.trace(want)).max() < 1e-12
    rho = want / np.trace(want)
    n = np.array([np.trace(dense.site_op(L, i, model.NUMBER) @ rho).real for i in range(L)])
    assert np.abs(res["density"] - n).max() < 1e-12
    C = dense.dense_correlation(L, rho, fermionic=True)
    assert np.abs(res["corr"] - C).max() < 1e-12
    assert max(res["bond_dims"]) > 4 and res["trunc_weight"] < 1e-20


def test_untruncated_state_is_a_density_matrix():
    L = 5
    cfg = cfg_of(L, dt=0.1, loss=0.4, gain=0.2, deph=0.3, occ="neel")
    rho = mpdo.run_mpdo(cfg, 10)["state"].to_dense()
    rho = rho / np.trace(rho)
    assert np.abs(rho - rho.conj().T).max() < 1e-12
    w = np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))
    assert w.min() > -1e-12 and abs(w.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("order,ratio", [(2, 0.25), (1, 0.5)])
def test_trotter_step_converges_to_lindblad(order, ratio):
    L, T = 4, 1.0
    errs = []
    for dt in (0.1, 0.05):
        cfg = cfg_of(L, dt=dt, loss=[0.5, 0.2, 0.3, 0.6], gain=0.2, deph=0.3, occ="neel",
                     order=order)
        res = mpdo.run_mpdo(cfg, int(round(T / dt)))
        rho = res["state"].to_dense()
        psi0 = dense.product_state(L, cfg.occupation)
        exact = dense.lindblad_rk4(L, 1.0, cfg.gamma_loss, cfg.gamma_gain, cfg.gamma_deph,
                                   np.outer(psi0, psi0.conj()), T, 1e-3, fermionic=False)
        errs.append(np.abs(rho / np.trace(rho) - exact).max())
    assert errs[0] < 0.05
    assert 0.7 * ratio < errs[1] / errs[0] < 1.3 * ratio, errs


def test_source_sink_chain_follows_the_closed_correlation_equation():
    # the paper's model (Sec. 2.1): source c_0^+ and sink c_{L-1} at the same
    # gamma, vacuum start; C(t) from Eq. eqCorr, Strang error O(dt^2)
    L, T, g = 6, 2.0, 0.8
    loss = np.zeros(L)
    gain = np.zeros(L)
    gain[0], loss[-1] = g, g
    errs = []
    for dt in (0.04, 0.02):
        cfg = cfg_of(L, dt=dt, loss=loss, gain=gain, fermionic=True, occ="vacuum")
        res = mpdo.run_mpdo(cfg, int(round(T / dt)), measure_corr=True)
        want = dense.corr_rk4(L, 1.0, loss, gain, np.zeros(L), np.zeros((L, L), complex), T, 1e-3)
        errs.append(np.abs(res["corr"] - want).max())
        j = mpdo.current(res["corr"])
        j_want = mpdo.current(want)
        assert np.abs(j - j_want).max() < 2 * errs[-1] + 1e-9
    assert errs[1] < 2e-3
    assert 0.18 < errs[1] / errs[0] < 0.32, errs


def test_one_truncated_bond_is_the_best_rank_k_approximation():
    # L = 2: one bond, theta = G |rho>> as a 4 x 4 matrix; keeping k = 2 values
    # must give its best rank-2 approximation divided by the kept norm
    rng = np.random.default_rng(5)
    cfg = cfg_of(2, chi=2, loss=0.3, gain=0.2, deph=0.4)
    m = mpdo.MPDO(cfg)
    X = rand_c(rng, 4, 4)
    U, S, Vh = np.linalg.svd(X)
    m.B = [U.reshape(1, 4, 4), (np.diag(S) @ Vh).reshape(4, 4, 1)]
    m.lam = [np.ones(4)]   # bond 0 has no left weight; Lambda_0 is not read
    G = mpdo.bond_gates(cfg, 0.3)[0]
    m.update_bond(0, G)
    th = (G @ X.reshape(-1)).reshape(4, 4)
    u, s, vh = np.linalg.svd(th)
    best = (u[:, :2] * s[:2]) @ vh[:2]
    got = (m.B[0].reshape(4, 2) @ m.B[1].reshape(2, 4))
    assert np.abs(got - best / np.sqrt(np.sum(s[:2] ** 2))).max() < 1e-13
    assert np.allclose(m.lam[0], s[:2] / np.sqrt(np.sum(s[:2] ** 2)))
    assert abs(m.trunc_weight - np.sum(s[2:] ** 2) / np.sum(s ** 2)) < 1e-15


def test_bulk_truncation_is_the_best_rank_k_approximation_of_the_state():
    # three sites in exact canonical form (B_0 = U_0 Lambda_0, B_1 and B_2
    # right-canonical); truncating bond 1 to k = 2 must give the best rank-2
    # approximation of G_{12}|v> across the cut {0,1} | {2}, which weights the
    # rows of theta~ by Lambda_0 (Eckart-Young on the full vector)
    rng = np.random.default_rng(6)
    cfg = cfg_of(3, chi=2, loss=0.3, gain=0.2, deph=0.4)
    v = rand_c(rng, 64)
    v /= np.linalg.norm(v)
    U0, S0, V0 = np.linalg.svd(v.reshape(4, 16), full_matrices=False)
    U1, S1, V1 = np.linalg.svd(V0.reshape(16, 4), full_matrices=False)
    m = mpdo.MPDO(cfg)
    m.B = [(U0 * S0).reshape(1, 4, 4), (V0.reshape(16, 4) @ V1.conj().T).reshape(4, 4, 4),
           V1.reshape(4, 4, 1)]
    m.lam = [S0, S1 / np.linalg.norm(S1)]
    G = mpdo.bond_gates(cfg, 0.3)[1]
    w = np.kron(np.eye(4), G) @ v
    u, s, vh = np.linalg.svd(w.reshape(16, 4), full_matrices=False)
    best = ((u[:, :2] * s[:2]) @ vh[:2]).reshape(-1) / np.sqrt(np.sum(s[:2] ** 2))
    m.update_bond(1, G)
    got = (m.B[0].reshape(4, -1) @ m.B[1].reshape(m.B[1].shape[0], -1)).reshape(16, -1)
    got = (got @ m.B[2].reshape(m.B[2].shape[0], -1)).reshape(-1)
    assert np.abs(got - best).max() < 1e-13


def test_truncation_keeps_degenerate_pairs_and_hermiticity():
    # the Schmidt spectrum of |rho>> comes in equal pairs (coherences q and -q);
    # with chi_max = 8 the plain cut would split the pair at 7/8 and leave a
    # non-Hermitian rho (error ~1e-2): the truncation keeps fewer values instead
    L = 6
    for chi in (4, 6, 8, 12):
        cfg = cfg_of(L, dt=0.1, chi=chi, loss=0.3, gain=0.2, deph=0.1, occ="neel")
        m = mpdo.run_mpdo(cfg, 8)["state"]
        rho = m.to_dense()
        rho = rho / np.trace(rho)
        assert np.abs(rho - rho.conj().T).max() < 1e-12, chi
        assert max(m.bond_dims()) <= chi
    cfg = cfg_of(L, dt=0.1, chi=8, loss=0.3, gain=0.2, deph=0.1, occ="neel")
    assert max(mpdo.run_mpdo(cfg, 8)["bond_dims"]) < 8     # pairs dropped, not split
    S = np.array([3.0, 2.0, 2.0, 1.0, 1.0, 0.5])
    assert [mpdo.keep_multiplets(S, k) for k in range(1, 7)] == [1, 1, 3, 3, 5, 6]
