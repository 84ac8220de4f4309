"""Pins of the FP64 oracle against things other than itself: published
known-answer vectors, closed forms, brute force on the full Hilbert space, and
invariants of the quantum-trajectory method."""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import dense, model, tebd
from oracle.philox import philox4x32_10, uniform01
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- Philox4x32-10 -------------------------------------------------------------
def test_philox_known_answer_vectors():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])
        n += 1
    assert n == 3


def test_uniform_draws_cover_unit_interval():
    u = np.array([uniform01(7, t, s) for t in range(50) for s in range(200)])
    assert u.min() >= 0.0 and u.max() < 1.0
    # mean 1/2 and variance 1/12 of U[0,1) within 5 sigma for 10^4 draws
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / u.size)
    assert uniform01(7, 3, 5) != uniform01(7, 3, 6) != uniform01(8, 3, 5)


# ---- gates (Sec. 2.3) ------------------------------------------------------------
def test_expm_taylor_matches_eigendecomposition_and_scipy():
    h = model.bond_heff(1.3, model.site_dissipator(0, 0, 0),
                        model.site_dissipator(0, 0, 0), 0.5, 0.5)
    w, V = np.linalg.eigh(h)
    for tau in (0.01, 0.37, 3.0):
        ref = (V * np.exp(-1j * tau * w)) @ V.conj().T
        assert np.abs(model.expm_taylor(-1j * tau * h) - ref).max() < 1e-14
    K1 = model.site_dissipator(0.3, 0.1, 0.2)
    K2 = model.site_dissipator(0.05, 0.4, 0.0)
    h = model.bond_heff(0.8, K1, K2, 1.0, 0.5)
    for tau in (0.02, 1.5):
        assert np.abs(model.expm_taylor(-1j * tau * h)
                      - scipy.linalg.expm(-1j * tau * h)).max() < 1e-13


def test_gates_unitary_without_dissipation():
    for G in model.bond_gates(6, 1.0, 0.05, 0.0, 0.0, 0.0):
        assert np.abs(G.conj().T @ G - np.eye(4)).max() < 1e-15


def test_hopping_gate_closed_form():
    # |10> -> cos(J tau)|10> + i sin(J tau)|01>  for h = -J (s+ s- + s- s+)
    J, tau = 0.9, 0.3
    G = model.bond_gates(2, J, tau, 0.0, 0.0, 0.0)[0]
    v = G[:, 2]
    assert abs(v[2] - np.cos(J * tau)) < 1e-15
    assert abs(v[1] - 1j * np.sin(J * tau)) < 1e-15
    assert abs(v[0]) < 1e-15 and abs(v[3]) < 1e-15


@pytest.mark.parametrize("L", [5, 6])
def test_site_damping_split_over_a_second_order_step(L):
    # J = 0: gates are diagonal; over A(dt/2) B(dt) A(dt/2) every site must
    # receive exp(-(dt/2) K_i) exactly once (edges whole, bulk halves).
    rng = np.random.default_rng(L)
    gl, gg, gd = rng.random(L), rng.random(L), rng.random(L)
    cfg = tebd.TrajectoryConfig(L, J=0.0, dt=0.07, gamma_loss=gl, gamma_gain=gg,
                                gamma_deph=gd)
    op = np.eye(2 ** L, dtype=complex)
    for parity, tau in cfg.layers():
        g = cfg.gates(tau)
        for b in range(parity, L - 1, 2):
            op = dense.bond_op(L, b, g[b]) @ op
    want = np.eye(2 ** L, dtype=complex)
    for i in range(L):
        K = model.site_dissipator(gl[i], gg[i], gd[i])
        want = want @ dense.site_op(L, i, np.diag(np.exp(-0.5 * cfg.dt * np.diag(K))))
    assert np.abs(op - want).max() < 1e-14


# ---- correlation matrix (Sec. 2.1) -------------------------------------------
def test_correlation_equation_matches_dense_lindblad():
    L = 4
    gl = np.array([0.1, 0.2, 0.05, 0.15])
    gg = np.array([0.05, 0.0, 0.1, 0.02])
    gd = np.array([0.03, 0.07, 0.0, 0.1])
    occ = [1, 0, 1, 0]
    psi0 = dense.product_state(L, occ)
    rho = dense.lindblad_rk4(L, 1.0, gl, gg, gd, np.outer(psi0, psi0.conj()), 1.0, 1e-3)
    assert abs(np.trace(rho) - 1) < 1e-12
    assert np.abs(rho - rho.conj().T).max() < 1e-14
    C = dense.corr_rk4(L, 1.0, gl, gg, gd, np.diag(occ).astype(complex), 1.0, 1e-3)
    assert np.abs(dense.dense_correlation(L, rho) - C).max() < 1e-12


def test_correlation_equation_matches_closed_form():
    L = 7
    C0 = np.diag(workloads.occupation(L, "neel")).astype(complex)
    C = dense.corr_rk4(L, 1.0, [0.2] * L, [0] * L, [0] * L, C0, 1.5, 1e-3)
    assert np.abs(C - dense.corr_uniform_loss(L, 1.0, 0.2, C0, 1.5)).max() < 1e-11


def test_two_site_correlation_by_hand():
    # L = 2, |10>, one step: state cos(J dt)|10> + i sin(J dt)|01>, so
    # <n_1> = sin^2, C_01 = conj(cos) * i sin.
    cfg = tebd.TrajectoryConfig(2, J=1.0, dt=0.2, chi_max=4, occupation=[1, 0])
    tr = tebd.Trajectory(cfg)
    g = tebd.StepGates(cfg)
    tebd.step_trajectory(tr, g, 0, 0, replay=-1)
    C = tr.correlation()
    c, s = np.cos(0.2), np.sin(0.2)
    assert abs(C[1, 1] - s * s) < 1e-15 and abs(C[0, 0] - c * c) < 1e-15
    assert abs(C[0, 1] - 1j * c * s) < 1e-15


# ---- MPS integrator against the full state vector ------------------------------
def _cfg_l6(**kw):
    base = dict(dt=0.05, chi_max=64, svd_cut=0.0, gamma_loss=0.3, gamma_gain=0.1,
                gamma_deph=0.05, occupation=[1, 0] * 3, seed=3)
    base.update(kw)
    return tebd.TrajectoryConfig(6, **base)


@pytest.mark.parametrize("fermionic,order", [(True, 2), (False, 2), (True, 1)])
def test_untruncated_mps_equals_dense_trajectory(fermionic, order):
    cfg = _cfg_l6(fermionic=fermionic, trotter_order=order)
    res = tebd.run_trajectories(cfg, 30, [0, 1, 2, 3])
    assert (res["jumps"] >= 0).sum() > 0
    for idx in range(4):
        tr = tebd.Trajectory(cfg)
        g = tebd.StepGates(cfg)
        for s, ch in enumerate(res["jumps"][idx]):
            tebd.step_trajectory(tr, g, idx, s, ch)
        v = tr.to_dense()
        v = v / np.linalg.norm(v)
        psi = dense.dense_trajectory(cfg, res["jumps"][idx])
        assert abs(abs(np.vdot(v, psi)) - 1) < 1e-12
        Cx = dense.dense_correlation(6, psi)   # C_ij is fermionic whatever the jumps are
        assert np.abs(tr.correlation() - Cx).max() < 1e-12
        assert np.abs(tr.density() - np.real(np.diag(Cx))).max() < 1e-12


def test_jump_record_is_reproducible_and_replayable():
    cfg = _cfg_l6()
    a = tebd.run_trajectories(cfg, 25, [5, 9])
    b = tebd.run_trajectories(cfg, 25, [5, 9], replay=a["jumps"])
    assert np.array_equal(a["jumps"], b["jumps"])
    assert np.abs(a["density"] - b["density"]).max() == 0.0


def test_bond_update_canonical_and_exact_without_truncation():
    Bl, Br, lam = workloads.random_theta_inputs(5, 7, 3, seed=11)
    cfg = tebd.TrajectoryConfig(3, chi_max=64, svd_cut=0.0)
    G = model.bond_gates(3, 1.0, 0.1, 0.2, 0.1, 0.0)[1]
    B0 = np.ones((1, 2, 5), complex) / np.sqrt(10)
    tr = tebd.Trajectory.from_tensors(cfg, [B0, Bl, Br], [lam, np.ones(7)])
    before = np.einsum('uvst,astc->auvc', G.reshape(2, 2, 2, 2),
                       np.tensordot(Bl, Br, axes=(2, 0))).reshape(10, 6)
    tr.update_bond(1, G)
    lam1, Bl1, Br1 = tr.lam[1], tr.B[1], tr.B[2]
    assert abs(np.sum(lam1 ** 2) - 1) < 1e-14
    V = Br1.reshape(len(lam1), -1)
    assert np.abs(V @ V.conj().T - np.eye(len(lam1))).max() < 1e-14
    # B_b' B_{b+1}' reproduces G (B_b B_{b+1}) up to the renormalisation factor
    after = Bl1.reshape(10, -1) @ V
    ratio = np.linalg.norm(after) / np.linalg.norm(before)
    assert np.abs(after - ratio * before).max() < 1e-13 * np.abs(before).max()
    # Lambda_b are the singular values of Lambda_{b-1}-weighted theta (renormalised):
    # compare the squared spectrum with the eigenvalues of theta^+ theta
    th = np.repeat(lam, 2)[:, None] * before
    ev = np.sort(np.linalg.eigvalsh(th.conj().T @ th))[::-1]
    assert np.abs(lam1 ** 2 - ev[:len(lam1)] / ev.sum()).max() < 1e-13
    assert tr.trunc_weight < 1e-28


def test_truncation_weight_is_discarded_hilbert_schmidt_norm():
    Bl, Br, lam = workloads.random_theta_inputs(6, 6, 6, seed=5)
    cfg = tebd.TrajectoryConfig(3, chi_max=4, svd_cut=0.0)
    G = np.eye(4, dtype=complex)
    tr = tebd.Trajectory.from_tensors(cfg, [np.ones((1, 2, 6)) / np.sqrt(12), Bl, Br],
                                      [lam, np.ones(6)])
    th = np.repeat(lam, 2)[:, None] * np.tensordot(Bl, Br, axes=(2, 0)).reshape(12, 12)
    tr.update_bond(1, G)
    k = len(tr.lam[1])
    assert k == 4
    # rank-4 projection of theta onto the kept right vectors: the squared Frobenius
    # distance over ||theta||^2 is the recorded discarded weight (Eq. HilbertSchmidtNorm)
    V = tr.B[2].reshape(k, -1)
    resid = th - th @ V.conj().T @ V
    assert abs(np.linalg.norm(resid) ** 2 / np.linalg.norm(th) ** 2 - tr.trunc_weight) < 1e-13


def test_particle_number_drops_by_one_per_loss_jump():
    cfg = tebd.TrajectoryConfig(8, dt=0.05, chi_max=16, svd_cut=0.0, gamma_loss=0.3,
                                occupation=workloads.occupation(8, "neel"), seed=1)
    res = tebd.run_trajectories(cfg, 40, list(range(6)))
    for idx in range(6):
        n_jumps = int((res["jumps"][idx] >= 0).sum())
        assert abs(res["density"][idx].sum() - (4 - n_jumps)) < 1e-11


def test_density_bounds_and_hermitian_correlation():
    cfg = _cfg_l6(chi_max=4, svd_cut=1e-12)
    res = tebd.run_trajectories(cfg, 30, [0, 1], measure_corr=True)
    for C in res["corr"]:
        assert np.abs(C - C.conj().T).max() < 1e-14
        assert np.all(np.real(np.diag(C)) > -1e-14) and np.all(np.real(np.diag(C)) < 1 + 1e-14)
        assert np.linalg.eigvalsh(C).min() > -1e-12   # C is a Gram matrix of c_j|psi>


def test_ensemble_matches_exact_correlation_within_clt_error():
    # uniform loss: C(t) = exp(-gamma t) U C(0) U^+ (closed form); Trotter and
    # the first-order jump-or-evolve bias are far below the CLT error here.
    L, n_traj, n_steps, dt, g = 6, 160, 40, 0.025, 0.5
    occ = workloads.occupation(L, "neel")
    cfg = tebd.TrajectoryConfig(L, dt=dt, chi_max=8, gamma_loss=g, occupation=occ, seed=4)
    res = tebd.run_trajectories(cfg, n_steps, list(range(n_traj)))
    mean, sem = tebd.ensemble_stats(res["density"])
    exact = np.real(np.diag(dense.corr_uniform_loss(L, 1.0, g, np.diag(occ).astype(complex),
                                                     n_steps * dt)))
    assert np.all(np.abs(mean - exact) < 4.5 * sem + 2e-3)


def test_one_site_recanonicalisation_equals_two_site_identity_sweep():
    # After a jump, shifting the orthogonality centre with one-site SVDs must give
    # the same Schmidt spectra (gauge invariant) as two-site identity-gate updates
    # over the whole chain; afterwards every B is right-canonical.
    L, chi = 10, 32
    cfg = tebd.TrajectoryConfig(L, dt=0.05, chi_max=chi, svd_cut=1e-13, gamma_loss=0.3,
                                occupation=workloads.occupation(L, "neel"), seed=2)
    tr = tebd.Trajectory(cfg)
    g = tebd.StepGates(cfg)
    for s in range(12):
        tebd.step_trajectory(tr, g, 0, s, replay=-1)
    for site in (0, 4, L - 1):
        a = tebd.Trajectory.from_tensors(cfg, tr.B, tr.lam)
        b = tebd.Trajectory.from_tensors(cfg, tr.B, tr.lam)
        a.apply_jump(3 * site)                      # one-site sweep
        O = model.jump_operator(model.LOSS)
        b.B[site] = np.einsum('uv,avc->auc', O, b.B[site])
        for j in range(site):
            b.B[j] = b.B[j].copy()
            b.B[j][:, 1, :] *= -1.0
        for bond in range(L - 2, 0, -1):
            b.update_bond(bond, tebd.IDENTITY4)
        for bond in range(L - 1):
            b.update_bond(bond, tebd.IDENTITY4)
        assert a.bond_dims() == b.bond_dims()
        for la, lb in zip(a.lam, b.lam):
            assert np.abs(la - lb).max() < 1e-12
        assert np.abs(a.correlation() - b.correlation()).max() < 1e-12
        for Bi in a.B[1:]:
            M = Bi.reshape(Bi.shape[0], -1)
            assert np.abs(M @ M.conj().T - np.eye(M.shape[0])).max() < 1e-12
        # and Lambda_{b-1} B_b has orthogonal columns whose norms are Lambda_b (the
        # left half of the canonical form, which fixes Lambda_b by the stored tensors)
        for bond in range(L - 1):
            X = np.repeat(a.left_weight(bond), 2)[:, None] * a.B[bond].reshape(-1, a.B[bond].shape[2])
            assert np.abs(X.conj().T @ X - np.diag(a.lam[bond] ** 2)).max() < 1e-12
