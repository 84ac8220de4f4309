"""The request server on the GPU: requests of different methods, precisions and
sizes run side by side must give exactly the results each gives alone;
admission respects the device-memory budget; a request larger than the budget
fails with LT_ERR_OOM."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REQUESTS = [
    dict(n_steps=12, L=16, chi_max=16, n_traj=8, precision=1, dt=0.05, gamma_loss=0.2, seed=1),
    dict(n_steps=9, L=12, chi_max=8, n_traj=5, precision=0, method=1, dt=0.05, gamma_deph=0.2,
         gamma_loss=[0.3] + [0.0] * 11, seed=2),
    dict(n_steps=7, L=10, chi_max=8, n_traj=3, precision=0, dt=0.05, gamma_loss=0.3,
         gamma_deph=0.1, seed=3),
    dict(n_steps=5, L=20, chi_max=32, n_traj=16, precision=1, dt=0.02, gamma_loss=0.1, seed=4,
         init="domain_wall"),
    # a vectorised density matrix: two chains, spin loss and gain on every site
    dict(n_steps=6, L=10, chi_max=16, n_traj=2, precision=1, method=2, dt=0.05,
         gamma_loss=0.1, gamma_gain=0.05, fermionic_jumps=0, seed=5, init="domain_wall"),
    # a purified density matrix (Kraus dimension 2)
    dict(n_steps=5, L=9, chi_max=16, n_traj=1, precision=0, method=3, kraus_dim=2, dt=0.05,
         gamma_loss=0.1, gamma_deph=0.07, fermionic_jumps=0, seed=6),
]


def _alone(lt, req):
    kw = dict(req)
    n_steps = kw.pop("n_steps")
    with lt.Ensemble(kw.pop("L"), kw.pop("chi_max"), kw.pop("n_traj"), **kw) as e:
        e.step(n_steps)
        mean, sem, _ = e.density()
    return mean, sem


def _served(lt, budget, max_active=16):
    with lt.Server(budget, max_active) as s:
        ids = [s.submit(**r) for r in REQUESTS]
        peak = 0
        for _ in range(10000):
            q, a, f = s.tick()
            peak = max(peak, a)
            used, _ = s.usage()
            assert used <= budget
            if q == 0 and a == 0:
                break
        out = [s.result(i) for i in ids]
    return out, peak


def test_requests_served_together_equal_each_alone():
    from paper_2609_18841_b300 import lindtebd as lt
    alone = [_alone(lt, r) for r in REQUESTS]
    served, peak = _served(lt, 8 << 30)
    assert peak > 1, "requests should run side by side"
    for (st, mean, sem, t), (m0, s0) in zip(served, alone):
        assert st == lt.LT_OK
        assert np.array_equal(mean, m0) and np.array_equal(sem, s0)
        assert t[0] <= t[1] <= t[2]


def test_staggered_arrivals_of_different_chi():
    """Requests admitted while others run (a large-chi request first, smaller ones
    arriving during it) all finish with the results they give alone."""
    from paper_2609_18841_b300 import lindtebd as lt
    order = [3, 0, 4, 5, 2, 1]
    alone = {i: _alone(lt, REQUESTS[i]) for i in order}
    with lt.Server(8 << 30, 16) as s:
        ids = {}
        for i in order:
            ids[i] = s.submit(**REQUESTS[i])
            s.tick()
            s.tick()
        s.run()
        for i in order:
            st, mean, sem, _ = s.result(ids[i])
            assert st == lt.LT_OK, s.error(ids[i])
            assert np.array_equal(mean, alone[i][0]) and np.array_equal(sem, alone[i][1])


def test_admission_cap_estimate_and_oversize():
    from paper_2609_18841_b300 import lindtebd as lt
    sizes = [lt.lt_context_bytes(r["L"], r["chi_max"], r["n_traj"], num_sms=148,
                                 precision=r["precision"], method=r.get("method", 0),
                                 kraus_dim=r.get("kraus_dim", 0))
             for r in REQUESTS]
    alone = [_alone(lt, r) for r in REQUESTS]
    # one at a time (active cap 1) under a budget that fits the largest request
    served, peak = _served(lt, max(sizes) + 1, max_active=1)
    assert peak == 1
    for (st, mean, sem, _), (m0, s0) in zip(served, alone):
        assert st == lt.LT_OK
        assert np.array_equal(mean, m0) and np.array_equal(sem, s0)
    # the admission estimate bounds what a context allocates
    for r, est in zip(REQUESTS, sizes):
        with lt.Server(8 << 30) as s:
            s.submit(**r)
            s.tick()
            used, _ = s.usage()
            assert 0 < used <= est
            s.run()
    # a request larger than the budget fails instead of blocking the queue
    with lt.Server(1 << 20) as s:
        big = s.submit(n_steps=1, L=64, chi_max=64, n_traj=64, precision=1)
        small = s.submit(n_steps=1, L=4, chi_max=2, n_traj=1, precision=1)
        s.run()
        assert s.result(big)[0] == lt.LT_ERR_OOM
        assert s.result(small)[0] == lt.LT_OK
