"""The host-side gate build (the first step of every method) against the oracle's
gates, on the CPU: exp(-i h_b^eff tau) with the site terms split between bonds
(Eq. EffHamiltonian, Eq. LindbladLocal), the Liouvillian gates exp(tau Lv_b) of
the vectorised density matrix (Eq. Liouvillian, L (x) conj(L) reading) and the
purified gates exp(-i h_b^eff tau) (x) 1 over the Kraus indices (Eq.
ThetaPurified).  Both sides exponentiate by their own scaling-and-squaring
series, so they agree to rounding."""
import numpy as np
import pytest

import workloads
from oracle import model, mpdo, purified, tebd
from paper_2609_18841_b300 import lindtebd as lt


def _rates(L, seed):
    rng = np.random.default_rng(seed)
    loss = rng.uniform(0.0, 0.6, L) * (rng.random(L) < 0.8)
    gain = rng.uniform(0.0, 0.4, L) * (rng.random(L) < 0.6)
    deph = rng.uniform(0.0, 0.5, L) * (rng.random(L) < 0.7)
    return loss, gain, deph


@pytest.mark.parametrize("L,tau,seed", [(2, 0.05, 1), (5, 0.01, 2), (9, 0.2, 3), (16, 0.5, 4)])
def test_pure_state_gates(L, tau, seed):
    loss, gain, deph = _rates(L, seed)
    got = lt.lt_gates(L, tau, J=0.7, gamma_loss=loss, gamma_gain=gain, gamma_deph=deph)
    want = model.bond_gates(L, 0.7, tau, loss, gain, deph)
    for b in range(L - 1):
        assert np.abs(got[b] - want[b]).max() < 1e-14


@pytest.mark.parametrize("L,tau,seed", [(2, 0.05, 5), (6, 0.02, 6), (9, 0.3, 7)])
def test_liouvillian_gates(L, tau, seed):
    loss, gain, deph = _rates(L, seed)
    got = lt.lt_gates(L, tau, J=1.3, method=lt.LT_MPDO, gamma_loss=loss, gamma_gain=gain,
                      gamma_deph=deph, fermionic_jumps=0)
    cfg = tebd.TrajectoryConfig(L, J=1.3, gamma_loss=loss, gamma_gain=gain, gamma_deph=deph,
                                fermionic=False, occupation=workloads.occupation(L, "neel"))
    want = mpdo.bond_gates(cfg, tau)
    for b in range(L - 1):
        assert np.abs(got[b] - want[b]).max() < 1e-13


@pytest.mark.parametrize("L,tau,seed", [(3, 0.05, 8), (7, 0.1, 9)])
def test_purified_gates(L, tau, seed):
    loss, gain, deph = _rates(L, seed)
    got = lt.lt_gates(L, tau, method=lt.LT_PURIFIED, kraus_dim=2, gamma_loss=loss,
                      gamma_gain=gain, gamma_deph=deph, fermionic_jumps=0)
    want = [purified.full_gate(G, 2) for G in model.bond_gates(L, 1.0, tau, loss, gain, deph)]
    for b in range(L - 1):
        assert np.abs(got[b] - want[b]).max() < 1e-14


def test_gate_arguments_are_checked():
    with pytest.raises(lt.LtError):
        lt.lt_gates(1, 0.1)
    with pytest.raises(lt.LtError):
        lt.lt_gates(4, 0.1, gamma_loss=[0.1, -0.2, 0.0, 0.0])
