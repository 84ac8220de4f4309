"""GPU parity of the locally purified density matrix (Sec. 3.2) through the C ABI
against the FP64 oracle: rho = X X^+ with X an MPS over s = 2n + k (Kraus
dimension 2), effective-Hamiltonian layers that keep the norm, then the R step
on every site (Eqs. MatrixR, NewPurified).  Per chain <n_i> and C_ij within 1e-10
in FP64 and within the single-precision bound below in mixed precision.  The
R step keeps two eigenvectors; the rates are chosen unequal so that no two
eigenvalues tie at that cut (a tie makes the kept Kraus vector arbitrary)."""
import numpy as np
import pytest

import workloads
from oracle import purified, tebd

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 5e-5


def _lt():
    from paper_2609_18841_b300 import lindtebd
    return lindtebd


def cfg_of(L, chi, dt=0.05, loss=0.0, gain=0.0, deph=0.0, fermionic=False, occ="neel",
           cut=1e-12):
    return tebd.TrajectoryConfig(L, J=1.0, dt=dt, chi_max=chi, svd_cut=cut, gamma_loss=loss,
                                 gamma_gain=gain, gamma_deph=deph, fermionic=fermionic,
                                 occupation=workloads.occupation(L, occ))


def source_sink(L, chi, g=0.6, deph=0.13, dt=0.05):
    loss = np.zeros(L)
    gain = np.zeros(L)
    gain[0], loss[-1] = g, 0.9 * g
    return cfg_of(L, chi, dt=dt, loss=loss, gain=gain, deph=deph, fermionic=True, occ="vacuum")


def ensemble(cfg, n, precision, cut=None):
    lt = _lt()
    return lt.Ensemble(cfg.L, cfg.chi_max, n, method=lt.LT_PURIFIED, kraus_dim=2,
                       precision=precision, init="product",
                       product_occ=cfg.occupation.astype(np.uint8), J=cfg.J, dt=cfg.dt,
                       gamma_loss=cfg.gamma_loss, gamma_gain=cfg.gamma_gain,
                       gamma_deph=cfg.gamma_deph, fermionic_jumps=int(cfg.fermionic),
                       svd_cut=cfg.svd_cut if cut is None else cut)


def close(got, want, tol, what):
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(got - want).max())
    assert err <= tol * scale, "%s: max |diff| %.3e > %.1e" % (what, err, tol * scale)
    return err


CASES = [
    ("source_sink_chi16", lambda: source_sink(8, 16), 10),
    ("loss_gain_deph_chi32", lambda: cfg_of(9, 32, loss=0.1, gain=0.05, deph=0.07), 8),
    ("loss_gain_chi64", lambda: cfg_of(8, 64, dt=0.1, loss=0.3, gain=0.2, deph=0.11), 6),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    name, make, steps = request.param
    cfg = make()
    return cfg, steps, purified.run_purified(cfg, 2, steps, measure_corr=True)


def test_purified_fp64_matches_the_oracle(case):
    cfg, steps, res = case
    lt = _lt()
    with ensemble(cfg, 2, lt.LT_FP64) as e:
        e.step(steps)
        _, sem, per = e.density(per_traj=True)
        _, Cp = e.corr(per_traj=True)
        tw, dims = e.stats()
    for t in range(2):
        close(per[t], res["density"], FP64_TOL, "density")
        close(Cp[t], res["corr"], FP64_TOL, "correlation")
        assert list(dims[t]) == list(res["bond_dims"])
    assert np.all(sem < 1e-12)


def test_purified_mixed_precision(case):
    cfg, steps, res = case
    lt = _lt()
    with ensemble(cfg, 1, lt.LT_MIXED, cut=1e-6) as e:
        e.step(steps)
        _, _, per = e.density(per_traj=True)
        _, Cp = e.corr(per_traj=True)
    close(per[0], res["density"], MIXED_TOL, "mixed density")
    close(Cp[0], res["corr"], MIXED_TOL, "mixed correlation")


def test_step_equals_layers_then_r_step():
    lt = _lt()
    cfg = cfg_of(7, 16, loss=0.2, gain=0.1, deph=0.05)
    with ensemble(cfg, 1, lt.LT_FP64) as a, ensemble(cfg, 1, lt.LT_FP64) as b:
        a.step(4)
        for _ in range(4):
            for parity, tau in cfg.layers():
                b.apply_layer(parity, tau)
            b.apply_kraus()
        assert np.array_equal(a.density(per_traj=True)[2], b.density(per_traj=True)[2])
    with lt.Ensemble(6, 8, 1, precision=lt.LT_FP64, gamma_loss=0.1) as t:
        with pytest.raises(lt.LtError) as err:
            t.apply_kraus()
        assert err.value.status == lt.LT_ERR_UNSUPPORTED


def test_chain_of_64_sites_sampled():
    # 64 sites, spin loss, gain and dephasing on every site, chi_max = 64,
    # the first steps through the oracle site by site
    lt = _lt()
    cfg = cfg_of(64, 64, dt=0.02, loss=0.1, gain=0.05, deph=0.03)
    steps = 3
    res = purified.run_purified(cfg, 2, steps, measure_corr=True)
    for prec, tol, cut in ((lt.LT_FP64, FP64_TOL, 1e-12), (lt.LT_MIXED, MIXED_TOL, 1e-6)):
        with ensemble(cfg, 1, prec, cut=cut) as e:
            e.step(steps)
            _, _, per = e.density(per_traj=True)
            _, Cp = e.corr(per_traj=True)
        close(per[0], res["density"], tol, "density")
        close(Cp[0], res["corr"], tol, "corr")


def _edge_cases():
    def ss(L, chi, order=2):
        c = source_sink(L, chi, g=0.5, deph=0.1)
        c.trotter_order = order
        return c
    spin = cfg_of(5, 8, loss=0.3, gain=0.12, deph=0.07, occ="domain_wall")
    spin.trotter_order = 1
    return [("one_bond_source_sink", ss(2, 4), 6), ("odd_first_order", ss(3, 8, order=1), 6),
            ("chi_1", cfg_of(6, 1, loss=0.2, gain=0.1, deph=0.05), 5),
            ("first_order_spin", spin, 7)]


@pytest.mark.parametrize("name,cfg,steps", _edge_cases(), ids=[c[0] for c in _edge_cases()])
def test_purified_edges(name, cfg, steps):
    lt = _lt()
    res = purified.run_purified(cfg, 2, steps, measure_corr=True)
    with lt.Ensemble(cfg.L, cfg.chi_max, 1, method=lt.LT_PURIFIED, kraus_dim=2,
                     precision=lt.LT_FP64, init="product",
                     product_occ=cfg.occupation.astype(np.uint8), J=cfg.J, dt=cfg.dt,
                     trotter_order=cfg.trotter_order, gamma_loss=cfg.gamma_loss,
                     gamma_gain=cfg.gamma_gain, gamma_deph=cfg.gamma_deph,
                     fermionic_jumps=int(cfg.fermionic), svd_cut=cfg.svd_cut) as e:
        e.step(steps)
        _, _, per = e.density(per_traj=True)
        _, Cp = e.corr(per_traj=True)
        _, dims = e.stats()
    close(per[0], res["density"], FP64_TOL, "density")
    close(Cp[0], res["corr"], FP64_TOL, "corr")
    assert list(dims[0]) == list(res["bond_dims"])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_configured_chi96_theta_384(precision, tol):
    # chi_max = 96, the purified form's configured bond dimension: bond 4 of a 10-site
    # chain with dims 96 | 96 | 96 has theta 384 x 384 (s = 2n + k, four values per
    # site); the layer keeps the norm change.  Synthetic state.
    from paper_2609_18841_b300.lindtebd import unpack_state
    lt = _lt()
    L, chi = 10, 96
    dims = [4, 16, 64, 96, 96, 96, 64, 16, 4]
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=17, d=4, dims=dims)
    cut = 1e-12 if precision == "fp64" else 1e-6
    cfg = cfg_of(L, chi, loss=0.1, deph=0.05, cut=cut)
    ref = purified.Purified(cfg, 2)
    ref.B, ref.lam = [b.copy() for b in B], [x.copy() for x in lam]
    ref.apply_layer(0, [purified.full_gate(G, 2) for G in cfg.gates(0.01)])
    prec = lt.LT_FP64 if precision == "fp64" else lt.LT_MIXED
    with ensemble(cfg, 1, prec) as e:
        e.set_state(0, [(B, lam, dims)])
        e.apply_layer(0, 0.01)
        gd, gl, gB = e.get_state(0, 1)
    gBs, gls = unpack_state(gd[0], gl[0], gB[0], L, d=4)
    for b in (0, 2, 4, 6, 8):
        X = np.tensordot(ref.B[b], ref.B[b + 1], axes=(2, 0)).reshape(4 * ref.B[b].shape[0], -1)
        Y = np.tensordot(gBs[b], gBs[b + 1], axes=(2, 0)).reshape(4 * gBs[b].shape[0], -1)
        w = np.repeat(ref.lam[b - 1], 4)[:, None] if b > 0 else np.ones((4, 1))
        err = np.abs(w * (Y - X)).max() / np.abs(w * X).max()
        assert err < tol, "bond %d: relative error %.2e" % (b, err)
    if precision == "fp64":
        assert list(gd[0]) == ref.bond_dims()


def test_cluster_launch_equals_the_one_cta_launch():
    # one chain: its single-precision layers go out as thread-block clusters that share
    # the wide Jacobi, the preconditioning, V_k^+ and the split of the 384 x 384 theta (the
    # purified form keeps the norm change, so the split is not rescaled); inside 96 chains
    # each task has one CTA.  The same arithmetic either way: equal bit for bit.
    lt = _lt()
    L, chi = 10, 96
    dims = [4, 16, 64, 96, 96, 96, 64, 16, 4]
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=23, d=4, dims=dims)
    cfg = cfg_of(L, chi, loss=0.1, deph=0.05, cut=1e-6)
    runs = []
    for n in (1, 96):
        with ensemble(cfg, n, lt.LT_MIXED) as e:
            e.set_state(0, [(B, lam, dims)] * n)
            e.apply_layer(0, 0.01)
            e.apply_layer(1, 0.01)
            runs.append((e.get_state(0, 1), lt.lt_cluster_launches(e.ctx)))
    (d1, l1, b1), c1 = runs[0]
    (d2, l2, b2), c2 = runs[1]
    assert c1 == 2 and c2 == 0
    assert np.array_equal(d1, d2)
    assert np.array_equal(l1, l2)
    assert np.array_equal(b1, b2)
