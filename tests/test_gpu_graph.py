"""Time steps replayed from a captured CUDA graph (lt_step_graph) are bit-identical
to plain lt_step for every method, also when the two are interleaved: the
captured launches read the Philox step from a device counter that each replay
advances, and everything else is the same kernels with the same arguments."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lt():
    from paper_2609_18841_b300 import lindtebd
    return lindtebd


def _configs():
    lt = _lt()
    return {
        "trajectories_fp64": (10, 16, 16, dict(precision=lt.LT_FP64, gamma_loss=0.3, gamma_deph=0.1,
                                                   seed=3)),
        "trajectories_mixed": (10, 16, 16, dict(precision=lt.LT_MIXED, gamma_loss=0.3, seed=4,
                                                    svd_cut=1e-6)),
        "qsd": (8, 16, 8, dict(method=lt.LT_QSD, precision=lt.LT_FP64, gamma_loss=[0.3] + [0] * 7,
                               gamma_deph=0.2, seed=5)),
        "mpdo": (8, 16, 2, dict(method=lt.LT_MPDO, precision=lt.LT_MIXED, gamma_loss=0.1,
                                gamma_gain=0.05, fermionic_jumps=0, svd_cut=1e-6)),
        "purified": (8, 16, 1, dict(method=lt.LT_PURIFIED, kraus_dim=2, precision=lt.LT_FP64,
                                    gamma_loss=0.2, gamma_deph=0.07, fermionic_jumps=0)),
    }


@pytest.mark.parametrize("name", ["trajectories_fp64", "trajectories_mixed", "qsd", "mpdo",
                                  "purified"])
def test_graph_steps_equal_plain_steps(name):
    lt = _lt()
    L, chi, n, kw = _configs()[name]
    kw = dict(kw, init="neel", dt=0.05)
    with lt.Ensemble(L, chi, n, **kw) as a, lt.Ensemble(L, chi, n, **kw) as b:
        a.step(6)
        b.step_graph(2)
        b.step(1)
        b.step_graph(3)
        assert lt.lt_get_step(a.ctx) == lt.lt_get_step(b.ctx) == 6
        da, db = a.density(per_traj=True)[2], b.density(per_traj=True)[2]
        ca, cb = a.corr(per_traj=True)[1], b.corr(per_traj=True)[1]
        sa, sb = a.stats(), b.stats()
        assert np.array_equal(da, db) and np.array_equal(ca, cb)
        assert np.array_equal(sa[1], sb[1]) and np.array_equal(sa[0], sb[0])
        if name == "qsd":
            assert np.array_equal(a.log_weights(), b.log_weights())
        assert b.launches() == a.launches() + 5   # one counter advance per replayed step
