"""Pins of the locally purified density matrix oracle (Sec. 3.2) against things
other than itself: the same scheme on dense 2^L x 2^L matrices, the paper's own
route through the d chi^2 x d chi^2 matrix R (Eq. MatrixR) and its
eigenvectors, first-order convergence to the Lindblad equation, the closed
equation of motion of C_ij (Eq. eqCorr) for the source/sink chain, and
positivity and Hermiticity of X X^+ under truncation."""
import numpy as np
import pytest

import workloads
from oracle import dense, model, purified, tebd


def cfg_of(L, dt=0.05, chi=64, loss=0.0, gain=0.0, deph=0.0, fermionic=False, occ="neel",
           order=2, cut=1e-14):
    return tebd.TrajectoryConfig(L, J=1.0, dt=dt, chi_max=chi, svd_cut=cut, gamma_loss=loss,
                                 gamma_gain=gain, gamma_deph=deph, fermionic=fermionic,
                                 trotter_order=order, occupation=workloads.occupation(L, occ))


def dense_scheme(cfg, n_steps):
    """Layers of the H_eff gates as dense operators, then on each site
    rho -> rho + dt sum_c gamma_c L_c rho L_c^+, written with 2^L matrices."""
    L = cfg.L
    psi0 = dense.product_state(L, cfg.occupation)
    rho = np.outer(psi0, psi0.conj())
    layer_ops = []
    for parity, tau in cfg.layers():
        gates = cfg.gates(tau)
        op = np.eye(2 ** L, dtype=complex)
        for b in range(parity, L - 1, 2):
            op = dense.bond_op(L, b, gates[b]) @ op
        layer_ops.append(op)
    rates = {model.LOSS: cfg.gamma_loss, model.GAIN: cfg.gamma_gain,
             model.DEPHASING: cfg.gamma_deph}
    for _ in range(n_steps):
        for op in layer_ops:
            rho = op @ rho @ op.conj().T
        for i in range(L):
            add = np.zeros_like(rho)
            for kind, g in rates.items():
                if g[i] > 0:
                    Li = dense.site_op(L, i, model.jump_operator(kind))
                    add += cfg.dt * g[i] * (Li @ rho @ Li.conj().T)
            rho = rho + add
    return rho


def test_untruncated_purification_equals_the_dense_scheme():
    # L = 4, loss on every site and dephasing on site 1, two steps: at most
    # (1 + 2)^2 = 9 Kraus vectors per site, so kraus = 9 and a large chi keep
    # everything
    L = 4
    cfg = cfg_of(L, dt=0.1, chi=400, loss=0.3, deph=[0, 0.2, 0, 0])
    res = purified.run_purified(cfg, 9, 2, measure_corr=True)
    rho = res["state"].to_dense()
    want = dense_scheme(cfg, 2)
    assert np.abs(rho - want).max() < 1e-12
    assert abs(res["trace"] - np.trace(want).real) < 1e-12
    n = np.array([np.trace(dense.site_op(L, i, model.NUMBER) @ want).real for i in range(L)])
    assert np.abs(res["density"] - n / np.trace(want).real).max() < 1e-12
    C = dense.dense_correlation(L, want, fermionic=True) / np.trace(want).real
    assert np.abs(res["corr"] - C).max() < 1e-12


def test_r_step_equals_the_eigenvectors_of_r():
    # the paper's route: R (Eq. MatrixR) as a (d chi_l chi_r)^2 Hermitian matrix,
    # its chi_k leading eigenvectors scaled by sqrt(lambda) (Eq. NewPurified),
    # taken with the left environment Lambda_{i-1}^2: R_w = W R W, and the kept
    # part W^-1 (R_w)_k W^-1
    rng = np.random.default_rng(3)
    K, chiL, chiR = 2, 3, 4
    cfg = cfg_of(3, dt=0.07, loss=0.4, gain=0.3, deph=0.2)
    m = purified.Purified(cfg, K)
    A = rng.standard_normal((chiL, 2, K, chiR)) + 1j * rng.standard_normal((chiL, 2, K, chiR))
    m.B[1] = A.reshape(chiL, 2 * K, chiR).copy()
    lam0 = np.array([0.8, 0.5, 0.33])
    m.lam[0] = lam0 / np.linalg.norm(lam0)
    vecs = [A]
    for kind, g in ((model.LOSS, 0.4), (model.GAIN, 0.3), (model.DEPHASING, 0.2)):
        vecs.append(np.sqrt(g * cfg.dt) * np.einsum('nm,amkc->ankc', model.jump_operator(kind), A))
    R = np.zeros((2 * chiL * chiR,) * 2, dtype=complex)
    for V in vecs:
        for k in range(K):
            x = V[:, :, k, :].transpose(1, 0, 2).reshape(-1)    # rows (n, a, c)
            R += np.outer(x, x.conj())
    W = np.kron(np.eye(2), np.kron(np.diag(m.lam[0]), np.eye(chiR)))   # rows (n, a, c)
    lam, phi = np.linalg.eigh(W @ R @ W)
    top = np.argsort(lam)[::-1][:K]
    Wi = np.linalg.inv(W)
    R_k = Wi @ ((phi[:, top] * lam[top]) @ phi[:, top].conj().T) @ Wi
    m.kraus_step(1)
    An = m.B[1].reshape(chiL, 2, K, chiR)
    got = np.zeros_like(R)
    for k in range(K):
        x = An[:, :, k, :].transpose(1, 0, 2).reshape(-1)
        got += np.outer(x, x.conj())
    assert np.abs(got - R_k).max() < 1e-12 * np.abs(R_k).max()


def test_bulk_fermionic_loss_is_rejected():
    with pytest.raises(ValueError):
        purified.run_purified(cfg_of(5, loss=0.1, fermionic=True), 2, 1)


def test_truncated_state_stays_a_density_matrix():
    # chi = 4 and chi_k = 2 truncate both kinds of bonds; X X^+ stays Hermitian,
    # positive semidefinite, with the trace the oracle reports
    L = 5
    cfg = cfg_of(L, dt=0.1, chi=4, loss=0.3, gain=0.2, deph=0.2)
    res = purified.run_purified(cfg, 2, 8)
    rho = res["state"].to_dense()
    assert np.abs(rho - rho.conj().T).max() < 1e-13
    w = np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))
    assert w.min() > -1e-13 * w.max()
    assert abs(np.trace(rho).real - res["trace"]) < 1e-12 * res["trace"]
    assert res["trunc_weight"] > 0 and max(res["bond_dims"]) == 4


def test_scheme_converges_to_lindblad_at_first_order():
    L, T = 3, 0.6
    errs = []
    for dt in (0.04, 0.02):
        cfg = cfg_of(L, dt=dt, chi=64, loss=[0.5, 0.2, 0.4], gain=0.1, deph=0.3)
        rho = purified.run_purified(cfg, 8, int(round(T / dt)))["state"].to_dense()
        assert np.abs(rho / np.trace(rho) - dense_scheme(cfg, int(round(T / dt)))
                      / np.trace(dense_scheme(cfg, int(round(T / dt))))).max() < 2e-4
        psi0 = dense.product_state(L, cfg.occupation)
        exact = dense.lindblad_rk4(L, 1.0, cfg.gamma_loss, cfg.gamma_gain, cfg.gamma_deph,
                                   np.outer(psi0, psi0.conj()), T, 1e-3, fermionic=False)
        errs.append(np.abs(rho / np.trace(rho) - exact).max())
    assert errs[0] < 0.02
    assert 0.4 < errs[1] / errs[0] < 0.6, errs


def test_source_sink_chain_follows_the_closed_correlation_equation():
    # the paper's chain (Sec. 2.1): source c_0^+ and sink c_{L-1} at the same gamma
    L, T, g = 5, 1.0, 0.6
    loss = np.zeros(L)
    gain = np.zeros(L)
    gain[0], loss[-1] = g, g
    errs = []
    for dt in (0.04, 0.02):
        cfg = cfg_of(L, dt=dt, chi=64, loss=loss, gain=gain, fermionic=True, occ="vacuum")
        res = purified.run_purified(cfg, 4, int(round(T / dt)), measure_corr=True)
        want = dense.corr_rk4(L, 1.0, loss, gain, np.zeros(L), np.zeros((L, L), complex), T, 1e-3)
        errs.append(np.abs(res["corr"] - want).max())
    assert errs[1] < 5e-3
    assert 0.4 < errs[1] / errs[0] < 0.6, errs
