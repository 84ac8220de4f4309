"""GPU parity of the vectorised density matrix (MPDO, Sec. 3.1) through the C ABI
against the FP64 oracle: Liouvillian gates exp(tau Lv_b) on |rho>> with four
local values per site, densities Tr(n_i rho)/Tr rho and correlations C_ij per
chain.  FP64 within 1e-10; mixed precision within the single-precision bound
stated below.  Sizes span the register path (4 chi <= 128) and the
shared/global-memory path (4 chi up to 256), ragged starting states, the
paper's source/sink chain and the 32-site loss/gain chain."""
import numpy as np
import pytest

import workloads
from oracle import dense, mpdo, tebd

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
# single precision: theta, the Jacobi rotations and the site tensors in FP32
# (relative rounding 6e-8 per operation over a few hundred layers); the
# observables are ratios of traces accumulated in double
MIXED_TOL = 5e-5


def _lt():
    from paper_2609_18841_b300 import lindtebd
    return lindtebd


def cfg_of(L, chi, dt=0.05, loss=0.0, gain=0.0, deph=0.0, fermionic=False, occ="domain_wall",
           cut=1e-12):
    return tebd.TrajectoryConfig(L, J=1.0, dt=dt, chi_max=chi, svd_cut=cut, gamma_loss=loss,
                                 gamma_gain=gain, gamma_deph=deph, fermionic=fermionic,
                                 occupation=workloads.occupation(L, occ))


def source_sink(L, chi, g=0.5, deph=0.0, dt=0.05):
    loss = np.zeros(L)
    gain = np.zeros(L)
    gain[0], loss[-1] = g, g
    return cfg_of(L, chi, dt=dt, loss=loss, gain=gain, deph=deph, fermionic=True, occ="vacuum")


def ensemble(cfg, n, precision, cut=None, **kw):
    lt = _lt()
    occ = cfg.occupation.astype(np.uint8)
    return lt.Ensemble(cfg.L, cfg.chi_max, n, method=lt.LT_MPDO, precision=precision,
                       init="product", product_occ=occ, J=cfg.J, dt=cfg.dt,
                       gamma_loss=cfg.gamma_loss, gamma_gain=cfg.gamma_gain,
                       gamma_deph=cfg.gamma_deph, fermionic_jumps=int(cfg.fermionic),
                       svd_cut=cfg.svd_cut if cut is None else cut, **kw)


def close(got, want, tol, what):
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(got - want).max())
    assert err <= tol * scale, "%s: max |diff| %.3e > %.1e" % (what, err, tol * scale)
    return err


CASES = [
    # (name, cfg, steps): the paper's source/sink chain with bulk dephasing,
    # truncated at chi 16; spin loss/gain on every site at chi 32 (register
    # path in single precision); chi 64 (theta 256 x 256 on the middle bonds)
    ("source_sink_chi16", lambda: source_sink(8, 16, g=0.7, deph=0.1), 12),
    ("loss_gain_chi32", lambda: cfg_of(9, 32, loss=0.1, gain=0.05, deph=0.02), 8),
    ("loss_gain_chi64", lambda: cfg_of(8, 64, dt=0.1, loss=0.3, gain=0.2, occ="neel"), 6),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    name, make, steps = request.param
    cfg = make()
    return cfg, steps, mpdo.run_mpdo(cfg, steps, measure_corr=True)


def test_mpdo_fp64_matches_the_oracle(case):
    cfg, steps, res = case
    lt = _lt()
    with ensemble(cfg, 2, lt.LT_FP64) as e:
        e.step(steps)
        mean, sem, per = e.density(per_traj=True)
        C, Cp = e.corr(per_traj=True)
        tw, dims = e.stats()
    for t in range(2):
        close(per[t], res["density"], FP64_TOL, "density")
        close(Cp[t], res["corr"], FP64_TOL, "correlation")
        assert list(dims[t]) == list(res["bond_dims"])
        assert abs(tw[t] - res["trunc_weight"]) <= 1e-10 + 1e-6 * res["trunc_weight"]
    close(mean, res["density"], FP64_TOL, "chain mean")
    assert np.all(sem < 1e-12)   # identical chains


def test_mpdo_mixed_precision(case):
    cfg, steps, res = case
    lt = _lt()
    with ensemble(cfg, 1, lt.LT_MIXED, cut=1e-6) as e:
        e.step(steps)
        _, _, per = e.density(per_traj=True)
        _, Cp = e.corr(per_traj=True)
    close(per[0], res["density"], MIXED_TOL, "mixed density")
    close(Cp[0], res["corr"], MIXED_TOL, "mixed correlation")


def test_ragged_chains_from_different_states():
    # three chains continue from oracle states with different occupations and
    # ragged, truncated bond dimensions; each must follow its own oracle history
    lt = _lt()
    L, chi = 7, 12
    occs = ["neel", "domain_wall", "vacuum"]
    starts = []
    for k, occ in enumerate(occs):
        cfg = cfg_of(L, chi, loss=0.2, gain=0.1 + 0.05 * k, deph=0.05, occ=occ)
        m = mpdo.run_mpdo(cfg, (1, 1, 2)[k])["state"]
        starts.append(([b.copy() for b in m.B], [x.copy() for x in m.lam], m.bond_dims()))
    # one context holds all three chains and applies one set of rates (those
    # of chain 0) to all of them from here on
    cfg0 = cfg_of(L, chi, loss=0.2, gain=0.1, deph=0.05)
    want = []
    for B, lam, _ in starts:
        m = mpdo.MPDO(cfg0)
        m.B = [b.copy() for b in B]
        m.lam = [x.copy() for x in lam]
        want.append(mpdo.run_mpdo(cfg0, 5, measure_corr=True, state=m))
    with ensemble(cfg0, 3, lt.LT_FP64) as e:
        e.set_state(0, starts)
        dims0, _, _ = e.get_state(0, 3)
        assert [list(d) for d in dims0] == [s[2] for s in starts]
        e.step(5)
        _, _, per = e.density(per_traj=True)
        _, Cp = e.corr(per_traj=True)
        _, dims = e.stats()
    for t in range(3):
        close(per[t], want[t]["density"], FP64_TOL, "density chain %d" % t)
        close(Cp[t], want[t]["corr"], FP64_TOL, "corr chain %d" % t)
        assert list(dims[t]) == list(want[t]["bond_dims"])
    assert len({tuple(s[2]) for s in starts}) == 3   # the chains started ragged


def test_paper_source_sink_chain_second_order_in_dt():
    # the paper's chain: N = 24, source c_1^+ and sink c_N at the same gamma,
    # vacuum start, chi = 32; against the closed equation Eq. eqCorr (RK4 at a
    # step ten times finer than the MPDO's): the error at t = 2 falls about
    # fourfold when dt halves (Strang splitting) and stays below 1e-3
    lt = _lt()
    L, T, g = 24, 2.0, 0.5
    errs = []
    for dt in (0.04, 0.02):
        cfg = source_sink(L, 32, g=g, dt=dt)
        with ensemble(cfg, 1, lt.LT_FP64) as e:
            e.step(int(round(T / dt)))
            C, _ = e.corr()
        want = dense.corr_rk4(L, 1.0, cfg.gamma_loss, cfg.gamma_gain, cfg.gamma_deph,
                              np.zeros((L, L), complex), T, dt / 10)
        errs.append(float(np.abs(C - want).max()))
        j = mpdo.current(C)
        assert np.abs(j - mpdo.current(want)).max() < 2 * errs[-1] + 1e-12
    assert errs[1] < 1e-3, errs
    assert 0.15 < errs[1] / errs[0] < 0.35, errs


def test_loss_gain_chain_of_32_sites_sampled():
    # 32 sites, spin loss 0.1 and gain 0.05 on every site, dt = 0.02, domain
    # wall; the first steps through the oracle site by site
    lt = _lt()
    cfg = cfg_of(32, 64, dt=0.02, loss=0.1, gain=0.05)
    steps = 4
    res = mpdo.run_mpdo(cfg, steps, measure_corr=True)
    for prec, tol in ((lt.LT_FP64, FP64_TOL), (lt.LT_MIXED, MIXED_TOL)):
        with ensemble(cfg, 1, prec, cut=1e-12 if prec == lt.LT_FP64 else 1e-6) as e:
            e.step(steps)
            _, _, per = e.density(per_traj=True)
            _, Cp = e.corr(per_traj=True)
        close(per[0], res["density"], tol, "density")
        close(Cp[0], res["corr"], tol, "corr")


def test_mpdo_checkpoint_and_method_errors(tmp_path):
    lt = _lt()
    cfg = source_sink(8, 16, deph=0.1)
    with ensemble(cfg, 2, lt.LT_MIXED) as a:
        a.step(7)
        da = a.density(per_traj=True)[2]
        with pytest.raises(lt.LtError) as e:
            a.apply_jumps(0)
        assert e.value.status == lt.LT_ERR_UNSUPPORTED
        with pytest.raises(lt.LtError) as e:
            a.apply_noise(0)
        assert e.value.status == lt.LT_ERR_UNSUPPORTED
    with ensemble(cfg, 2, lt.LT_MIXED) as b:
        b.step(3)
        lt.lt_save(b.ctx, str(tmp_path / "m.bin"))
    with ensemble(cfg, 2, lt.LT_MIXED) as c:
        lt.lt_load(c.ctx, str(tmp_path / "m.bin"))
        c.step(4)
        dc = c.density(per_traj=True)[2]
    assert np.array_equal(da, dc)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_wide_theta_whose_factor_takes_the_blocked_rows(precision, tol):
    # bond 3 of an 8-site chain with dims 19 | 40 | 36: theta is 76 x 144 (wider
    # than the register path holds) and its 76 x 76 factor takes the blocked
    # Jacobi layout with rows rounded up to 80; a synthetic (non-physical) state
    from paper_2609_18841_b300.lindtebd import unpack_state
    lt = _lt()
    L, chi = 8, 64
    dims = [4, 16, 19, 40, 36, 16, 4]
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=6, d=4, dims=dims)
    cut = 1e-12 if precision == "fp64" else 1e-6
    cfg = cfg_of(L, chi, loss=0.1, gain=0.05, cut=cut)
    ref = mpdo.MPDO(cfg)
    ref.B, ref.lam = [b.copy() for b in B], [x.copy() for x in lam]
    ref.apply_layer(1, mpdo.bond_gates(cfg, 0.05))
    prec = lt.LT_FP64 if precision == "fp64" else lt.LT_MIXED
    with ensemble(cfg, 1, prec) as e:
        e.set_state(0, [(B, lam, dims)])
        e.apply_layer(1, 0.05)
        gd, gl, gB = e.get_state(0, 1)
    gBs, gls = unpack_state(gd[0], gl[0], gB[0], L, d=4)
    for b in (1, 3, 5):
        X = np.tensordot(ref.B[b], ref.B[b + 1], axes=(2, 0)).reshape(4 * ref.B[b].shape[0], -1)
        Y = np.tensordot(gBs[b], gBs[b + 1], axes=(2, 0)).reshape(4 * gBs[b].shape[0], -1)
        w = np.repeat(ref.lam[b - 1], 4)[:, None]
        err = np.abs(w * (Y - X)).max() / np.abs(w * X).max()
        assert err < tol, "bond %d: relative error %.2e" % (b, err)
    if precision == "fp64":
        assert list(gd[0]) == ref.bond_dims()


def _edge_cases():
    def ss(L, chi, order=2):
        loss = np.zeros(L)
        gain = np.zeros(L)
        gain[0], loss[-1] = 0.5, 0.45
        c = cfg_of(L, chi, loss=loss, gain=gain, deph=0.1, fermionic=True, occ="vacuum")
        c.trotter_order = order
        return c
    spin = cfg_of(5, 8, loss=0.3, gain=0.12, deph=0.07, occ="domain_wall")
    spin.trotter_order = 1
    return [("one_bond_source_sink", ss(2, 4), 6), ("odd_first_order", ss(3, 8, order=1), 6),
            ("chi_1", cfg_of(6, 1, loss=0.2, gain=0.1, deph=0.05, occ="neel"), 5),
            ("first_order_spin", spin, 7)]


@pytest.mark.parametrize("name,cfg,steps", _edge_cases(), ids=[c[0] for c in _edge_cases()])
def test_mpdo_edges(name, cfg, steps):
    # one bond, an odd chain, chi_max = 1 (product states only) and the first-order
    # Trotter step, each through the oracle in FP64
    lt = _lt()
    res = mpdo.run_mpdo(cfg, steps, measure_corr=True)
    with lt.Ensemble(cfg.L, cfg.chi_max, 1, method=lt.LT_MPDO, precision=lt.LT_FP64,
                     init="product", product_occ=cfg.occupation.astype(np.uint8), J=cfg.J,
                     dt=cfg.dt, trotter_order=cfg.trotter_order, gamma_loss=cfg.gamma_loss,
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
def test_configured_chi128_theta_512(precision, tol):
    # chi_max = 128, the vectorised density matrix's configured bond dimension: bond 4
    # of a 10-site chain with dims 128 | 128 | 128 has theta 512 x 512 (in FP64 rows
    # longer than one Jacobi group's span, handled in chunks; in single precision the
    # wide block Jacobi, shared by a thread-block cluster since one chain has few
    # tasks); bond 2 is 64 x 512.  Synthetic state.
    from paper_2609_18841_b300.lindtebd import unpack_state
    lt = _lt()
    L, chi = 10, 128
    dims = [4, 16, 64, 128, 128, 128, 64, 16, 4]
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=16, d=4, dims=dims)
    cut = 1e-12 if precision == "fp64" else 1e-6
    cfg = cfg_of(L, chi, loss=0.1, gain=0.05, cut=cut)
    ref = mpdo.MPDO(cfg)
    ref.B, ref.lam = [b.copy() for b in B], [x.copy() for x in lam]
    ref.apply_layer(0, mpdo.bond_gates(cfg, 0.02))
    prec = lt.LT_FP64 if precision == "fp64" else lt.LT_MIXED
    with ensemble(cfg, 1, prec) as e:
        e.set_state(0, [(B, lam, dims)])
        e.apply_layer(0, 0.02)
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


@pytest.mark.parametrize("chi", [64, 96, 128])
def test_cluster_launch_equals_the_one_cta_launch(chi):
    # One chain gives a layer few tasks, so its single-precision layers go out as
    # thread-block clusters whose CTAs share the wide Jacobi (theta 4 chi x 4 chi = 256,
    # 384, 512: warp groups of 2, 3, 4 slices); the same chain inside an ensemble of 96
    # chains takes one CTA per task.  Both run the same block rounds with the same
    # arithmetic, so the results must agree bit for bit.
    lt = _lt()
    L = 10
    dims = [4, 16, 64, chi, chi, chi, 64, 16, 4]
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=19, d=4, dims=dims)
    cfg = cfg_of(L, chi, loss=0.1, gain=0.05, cut=1e-6)
    runs = []
    for n in (1, 96):
        with ensemble(cfg, n, lt.LT_MIXED) as e:
            e.set_state(0, [(B, lam, dims)] * n)
            e.apply_layer(0, 0.02)
            e.apply_layer(1, 0.02)
            runs.append((e.get_state(0, 1), lt.lt_cluster_launches(e.ctx)))
    (d1, l1, b1), c1 = runs[0]
    (d2, l2, b2), c2 = runs[1]
    assert c1 == 2 and c2 == 0
    assert np.array_equal(d1, d2)
    assert np.array_equal(l1, l2)
    assert np.array_equal(b1, b2)
