"""Pins of the quantum-state-diffusion oracle (Sec. 5.2) against things other
than itself: the moments of the Gaussian noise, the brute-force state vector,
the exact noise average of a step (from E[eta] = 0 and E[eta^2] = 1), the
Lindblad equation it must reproduce as dt -> 0 (Eq. Lindblad), and the closed
equation of motion of C_ij for dephasing with boundary loss."""
import numpy as np
import pytest

import workloads
from oracle import dense, model, philox, tebd


def cfg_qsd(L, dt, seed=3, loss0=0.3, deph=0.2, chi=64, occ="neel", fermionic=True):
    g_loss = np.zeros(L)
    g_loss[0] = loss0
    return tebd.TrajectoryConfig(L, J=1.0, dt=dt, chi_max=chi, svd_cut=1e-14, gamma_loss=g_loss,
                                 gamma_deph=deph, fermionic=fermionic,
                                 occupation=workloads.occupation(L, occ), seed=seed)


def test_gaussian_noise_moments():
    # 2 x 12000 numbers: mean 0, variance 1, fourth moment 3, pair members and
    # neighbouring steps uncorrelated (5 sigma bounds)
    pairs = np.array([philox.gaussian_pair(7, t, s, j)
                      for t in range(30) for s in range(20) for j in range(20)])
    x = pairs.reshape(-1)
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(x ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)
    assert abs(np.mean(pairs[:, 0] * pairs[:, 1])) < 5 / np.sqrt(n / 2)
    assert abs(np.mean(x[:-1] * x[1:])) < 5 / np.sqrt(n)
    # noise() lays the pairs out in order
    assert philox.noise(7, 2, 5, 5) == list(philox.gaussian_pair(7, 2, 5, 0)) + \
        list(philox.gaussian_pair(7, 2, 5, 1)) + [philox.gaussian_pair(7, 2, 5, 2)[0]]


@pytest.mark.parametrize("L,dt,fermionic", [(5, 0.05, True), (6, 0.02, False)])
def test_mps_qsd_equals_the_state_vector(L, dt, fermionic):
    cfg = cfg_qsd(L, dt, fermionic=fermionic)
    if not fermionic:
        cfg.gamma_loss[:] = 0.15   # spin loss on every site is local
    steps = 8
    res = tebd.run_qsd(cfg, steps, [0, 1, 2], measure_corr=True)
    for t in range(3):
        psi = dense.dense_qsd(cfg, t, steps)
        w = float(np.vdot(psi, psi).real)
        assert abs(np.log(w) - res["log_weight"][t]) < 1e-12
        n = np.array([np.vdot(psi, dense.site_op(L, i, model.NUMBER) @ psi).real / w
                      for i in range(L)])
        assert np.abs(n - res["density"][t]).max() < 1e-12
        C = dense.dense_correlation(L, psi / np.sqrt(w), fermionic=True)
        assert np.abs(C - res["corr"][t]).max() < 1e-12


def test_noise_step_leaves_the_canonical_form():
    # after every noise step (one-site SVDs right to left, then left to right) each
    # B_{b+1} is right-canonical and Lambda_{b-1} B_b has orthogonal columns whose
    # norms are Lambda_b, normalised to sum(Lambda_b^2) = 1, while the log weight
    # keeps <psi|psi>
    L = 7
    cfg = cfg_qsd(L, 0.05, fermionic=False, chi=8)
    cfg.gamma_loss[:] = 0.2
    cfg.svd_cut = 1e-10
    tr = tebd.Trajectory(cfg)
    gates = tebd.StepGates(cfg)
    for s in range(10):
        tebd.step_qsd(tr, gates, 1, s)
        for b in range(L - 1):
            X = np.repeat(tr.left_weight(b), 2)[:, None] * tr.B[b].reshape(-1, tr.B[b].shape[2])
            assert np.abs(X.conj().T @ X - np.diag(tr.lam[b] ** 2)).max() < 1e-12
            assert abs(np.sum(tr.lam[b] ** 2) - 1.0) < 1e-12
            M = tr.B[b + 1].reshape(tr.B[b + 1].shape[0], -1)
            assert np.abs(M @ M.conj().T - np.eye(M.shape[0])).max() < 1e-12
    assert max(tr.bond_dims()) == 8, "truncation should act"
    assert abs(tr.log_weight) > 1e-3, "the weight should move"


def test_bulk_fermionic_loss_is_rejected():
    cfg = cfg_qsd(4, 0.05)
    cfg.gamma_loss[2] = 0.1
    with pytest.raises(ValueError):
        tebd.run_qsd(cfg, 1, [0])


def test_monte_carlo_average_matches_the_exact_mean_map():
    # L = 3, 2500 dense histories, 6 steps: mean_t(w_t <n_i>_t) and mean_t(w_t)
    # within 4 sigma of Tr(n_i rho_bar) and Tr(rho_bar)
    L, dt, steps, n = 3, 0.1, 6, 2500
    cfg = cfg_qsd(L, dt, seed=11, loss0=0.6, deph=0.5)
    nums = [dense.site_op(L, i, model.NUMBER) for i in range(L)]
    vals = np.empty((n, L + 1))
    for t in range(n):
        psi = dense.dense_qsd(cfg, t, steps)
        vals[t, :L] = [np.vdot(psi, o @ psi).real for o in nums]
        vals[t, L] = np.vdot(psi, psi).real
    psi0 = dense.product_state(L, cfg.occupation)
    rho = dense.qsd_mean_map(cfg, np.outer(psi0, psi0.conj()), steps)
    want = np.array([np.trace(o @ rho).real for o in nums] + [np.trace(rho).real])
    mean = vals.mean(0)
    sem = vals.std(0) / np.sqrt(n)
    assert np.all(np.abs(mean - want) < 4 * sem + 1e-12), (mean, want, sem)
    assert np.all(sem > 0)


def test_mean_map_converges_to_lindblad_at_first_order():
    # Eq. EqMvtStochPsi reproduces Eq. Lindblad up to O(dt): the error of the
    # averaged scheme at T = 1 halves when dt halves, and Tr(rho_bar) - 1 too
    L, T = 4, 1.0
    occ = workloads.occupation(L, "neel")
    psi0 = dense.product_state(L, occ)
    rho0 = np.outer(psi0, psi0.conj())
    errs, tr = [], []
    for dt in (0.04, 0.02):
        cfg = cfg_qsd(L, dt, loss0=0.5, deph=0.3)
        rho = dense.qsd_mean_map(cfg, rho0, int(round(T / dt)))
        exact = dense.lindblad_rk4(L, 1.0, cfg.gamma_loss, cfg.gamma_gain, cfg.gamma_deph,
                                   rho0, T, 1e-3)
        errs.append(np.abs(rho - exact).max())
        tr.append(abs(np.trace(rho).real - 1.0))
    assert errs[0] < 0.05
    assert 0.4 < errs[1] / errs[0] < 0.6, errs
    assert 0.3 < tr[1] / tr[0] < 0.6, tr


def test_mean_map_correlations_follow_the_closed_equation():
    # dephasing on every site plus loss on site 0 (no string there): C_ij obeys
    # the closed linear equation; the averaged scheme approaches it at O(dt)
    L, T = 5, 0.8
    errs = []
    for dt in (0.02, 0.01):
        cfg = cfg_qsd(L, dt, loss0=0.4, deph=0.25)
        psi0 = dense.product_state(L, cfg.occupation)
        rho = dense.qsd_mean_map(cfg, np.outer(psi0, psi0.conj()), int(round(T / dt)))
        C = dense.dense_correlation(L, rho)
        C0 = np.diag(cfg.occupation.astype(float)).astype(complex)
        want = dense.corr_rk4(L, 1.0, cfg.gamma_loss, cfg.gamma_gain, cfg.gamma_deph, C0, T, 1e-3)
        errs.append(np.abs(C - want).max())
    assert errs[1] < 0.004
    assert 0.4 < errs[1] / errs[0] < 0.6, errs
