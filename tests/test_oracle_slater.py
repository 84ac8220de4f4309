"""Pins of the Slater-determinant reference (oracle/slater.py): the exact
untruncated history of the free-fermion chain for a given jump record.  It is
checked against brute force on the full 2^L state vector (the same Trotter
layers and jump operators, Sec. 2.3 and Sec. 4.1), and against the invariants
of a Gaussian pure state (C Hermitian, a projector of trace N, N lowered by one
per loss jump)."""
import numpy as np
import pytest

import workloads
from oracle import dense, slater, tebd


def _cfg(L, gl, gg, gd, seed, init="neel", dt=0.05):
    return tebd.TrajectoryConfig(L, J=1.0, dt=dt, chi_max=2 ** (L // 2), svd_cut=1e-12,
                                 gamma_loss=gl, gamma_gain=gg, gamma_deph=gd,
                                 occupation=workloads.occupation(L, init), seed=seed)


@pytest.mark.parametrize("L,gl,gg,gd,seed,init", [
    (8, 0.3, 0.0, 0.0, 1, "neel"),            # loss only, the configuration's channel
    (8, 0.2, 0.1, 0.15, 2, "neel"),           # loss, gain and dephasing on every site
    (7, [0.5, 0, 0, 0, 0, 0, 0.2], 0.0, 0.0, 3, "domain_wall"),  # odd chain, uneven rates
])
def test_slater_history_equals_the_dense_state_vector(L, gl, gg, gd, seed, init):
    cfg = _cfg(L, gl, gg, gd, seed, init)
    res = tebd.run_trajectories(cfg, 30, list(range(5)))
    assert (res["jumps"] >= 0).sum() > 0
    Cs = slater.run_slater(cfg, res["jumps"])
    for t in range(5):
        psi = dense.dense_trajectory(cfg, res["jumps"][t])
        Cd = dense.dense_correlation(L, psi)
        assert np.abs(Cs[t] - Cd).max() < 1e-12


def test_slater_correlation_is_a_projector_of_the_particle_number():
    cfg = _cfg(16, 0.3, 0.0, 0.0, 5, dt=0.05)
    res = tebd.run_trajectories(cfg, 40, list(range(4)))
    n0 = int(cfg.occupation.sum())
    for t in range(4):
        C = slater.run_slater(cfg, res["jumps"][t:t + 1])[0]
        assert np.abs(C - C.conj().T).max() < 1e-13
        assert np.abs(C @ C - C).max() < 1e-12          # pure Gaussian state
        n_loss = int((res["jumps"][t] >= 0).sum())
        assert abs(np.trace(C).real - (n0 - n_loss)) < 1e-12


def test_untruncated_mps_history_equals_the_slater_history():
    # the MPS integrator with no truncation (chi_max = 2^(L/2)) is exact for the
    # represented state, so the two references agree to rounding
    cfg = _cfg(10, 0.25, 0.0, 0.0, 7)
    res = tebd.run_trajectories(cfg, 40, list(range(3)), measure_corr=True)
    Cs = slater.run_slater(cfg, res["jumps"])
    assert np.abs(Cs - res["corr"]).max() < 1e-10
