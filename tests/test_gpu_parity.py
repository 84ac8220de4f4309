"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  FP64 mode must agree per trajectory within 1e-10 (scaled
by the largest |value|); decisions drawn from Philox on both sides must agree
exactly; mixed mode is held to the per-observable bounds stated below."""
import numpy as np
import pytest

import workloads
from oracle import tebd

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _lt():
    from paper_2609_18841_b300 import lindtebd
    return lindtebd


def oracle_cfg(w, L=None, chi=None, cut=1e-12, **over):
    L = L or w["L"]
    d = dict(J=w["J"], dt=w["dt"], chi_max=chi or w["chi_max"], svd_cut=cut,
             gamma_loss=w["gamma_loss"], gamma_gain=w["gamma_gain"],
             gamma_deph=w["gamma_deph"], fermionic=bool(w["fermionic"]),
             trotter_order=w["trotter_order"], occupation=workloads.occupation(L, w["init"]),
             seed=w["seed"])
    d.update(over)
    return tebd.TrajectoryConfig(L, **d)


def gpu_ensemble(cfg, n_traj, precision, init="neel", **kw):
    lt = _lt()
    return lt.Ensemble(cfg.L, cfg.chi_max, n_traj, precision=precision, init=init, J=cfg.J,
                       dt=cfg.dt, trotter_order=cfg.trotter_order, gamma_loss=cfg.gamma_loss,
                       gamma_gain=cfg.gamma_gain, gamma_deph=cfg.gamma_deph,
                       fermionic_jumps=int(cfg.fermionic), svd_cut=cfg.svd_cut, seed=cfg.seed,
                       **kw)


def gpu_steps(ens, cfg, n_steps, replay=None, step0=0):
    chans = []
    for s in range(n_steps):
        rep = None if replay is None else np.ascontiguousarray(replay[:, step0 + s], np.int32)
        chans.append(ens.apply_jumps(step0 + s, rep))
        for parity, tau in cfg.layers():
            ens.apply_layer(parity, tau)
    return np.stack(chans, axis=1)


def assert_close(got, want, tol, what):
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(got - want).max())
    assert err <= tol * scale, "%s: max |diff| %.3e > %.1e" % (what, err, tol * scale)
    return err


# ---- W1: L=8, chi=16, fermionic loss 0.1, Neel, dt=0.05, 40 steps ----------------------
@pytest.fixture(scope="module")
def w1_oracle():
    cfg = oracle_cfg(workloads.W1)
    n = 24
    res = tebd.run_trajectories(cfg, workloads.W1["n_steps"], list(range(n)), measure_corr=True)
    return cfg, n, res


def test_w1_fp64_sampled_decisions_and_observables(w1_oracle):
    cfg, n, res = w1_oracle
    lt = _lt()
    with gpu_ensemble(cfg, n, lt.LT_FP64) as ens:
        chans = gpu_steps(ens, cfg, workloads.W1["n_steps"])
        assert np.array_equal(chans, res["jumps"])
        mean, sem, dens = ens.density(per_traj=True)
        C, Cp = ens.corr(per_traj=True)
        tw, dims = ens.stats()
    assert_close(dens, res["density"], FP64_TOL, "density")
    assert_close(Cp, res["corr"], FP64_TOL, "corr")
    assert np.abs(mean - res["density"].mean(0)).max() < FP64_TOL
    assert np.array_equal(dims, res["bond_dims"])
    assert np.abs(tw - res["trunc"]).max() < 1e-12


def test_w1_fp64_replay(w1_oracle):
    cfg, n, res = w1_oracle
    lt = _lt()
    with gpu_ensemble(cfg, n, lt.LT_FP64) as ens:
        chans = gpu_steps(ens, cfg, workloads.W1["n_steps"], replay=res["jumps"])
        assert np.array_equal(chans, res["jumps"])
        _, _, dens = ens.density(per_traj=True)
    assert_close(dens, res["density"], FP64_TOL, "density")


@pytest.mark.parametrize("theta_path", [1, 2], ids=["theta_tensor_cores", "theta_fma"])
def test_w1_mixed_replay_error_bounds(w1_oracle, theta_path):
    # mixed: single-precision tensors, theta contractions and Jacobi rotations;
    # double-precision singular values, norms, Schmidt values and rates; the kept
    # right singular vectors re-orthonormalised after the Jacobi and the gates
    # applied as their single-precision value plus its rounding residual.  Bound:
    # the 1e-6 ensemble target for <c_i^+ c_j>.  Per trajectory the floor is the
    # single-precision accumulation of the theta contractions (about 3x the
    # rounding of the stored tensors in a CPU emulation of the same steps).
    # theta_path: theta from exact digit products on the tensor cores (1), or from
    # single-precision FMAs (2)
    cfg, n, res = w1_oracle
    lt = _lt()
    with gpu_ensemble(cfg, n, lt.LT_MIXED, theta_path=theta_path) as ens:
        gpu_steps(ens, cfg, workloads.W1["n_steps"], replay=res["jumps"])
        mean, _, dens = ens.density(per_traj=True)
        C, Cp = ens.corr(per_traj=True)
    e1 = assert_close(dens, res["density"], 5e-6, "mixed density per trajectory")
    e2 = assert_close(Cp, res["corr"], 5e-6, "mixed corr per trajectory")
    e3 = assert_close(mean, res["density"].mean(0), 1e-6, "mixed density ensemble")
    e4 = assert_close(C, res["corr"].mean(0), 1e-6, "mixed corr ensemble")
    print("mixed errors: dens %.2e corr %.2e mean %.2e Cmean %.2e" % (e1, e2, e3, e4))


def test_w3_full_run_mixed_against_fp64_and_the_exact_histories():
    """The W3 chain (L=64, chi_max=64, fermionic loss 0.2, dt=0.02, Neel) for all
    200 steps with 64 trajectories: the FP64 path samples the jumps, the mixed
    path replays them, both with svd_cut = 1e-6.  The exact untruncated history
    of each trajectory (the Slater-determinant reference) sizes the truncation
    error.  Bounds, from measurement:
      step 50:        ensemble C_ij of mixed and FP64 within 1e-6;
      steps 100, 150: within 4e-6: the single-precision rounding of the theta
                      contractions grows with the number of updates and is
                      correlated across trajectories whose histories differ only
                      near their jump sites (measured 1.6e-6 and 2.5e-6);
      step 200:       the chi_max = 64 truncation dominates and its dynamics
                      amplifies any perturbation (two FP64 runs whose Jacobi
                      thresholds differ part by up to 7e-4 per trajectory), so
                      the mixed ensemble must be as close to the exact histories
                      as the FP64 one (within 1.5x plus 1e-5) and the two
                      precisions closer to each other than FP64 is to exact."""
    from oracle import slater
    lt = _lt()
    w = workloads.W3
    L, chi, n = w["L"], w["chi_max"], 64
    cfg = oracle_cfg(w, cut=1e-6)
    checkpoints = (50, 100, 150, 200)
    kw = dict(init="neel", dt=w["dt"], gamma_loss=w["gamma_loss"], seed=w["seed"], svd_cut=1e-6)
    c64, chans = {}, []
    with lt.Ensemble(L, chi, n, precision=lt.LT_FP64, **kw) as ea:
        s0 = 0
        for ck in checkpoints:
            chans.append(gpu_steps(ea, cfg, ck - s0, step0=s0))
            s0 = ck
            c64[ck] = ea.corr(per_traj=True)[1]
    rec = np.concatenate(chans, axis=1)
    assert (rec >= 0).sum() > 500, "the run should hold many jumps"
    cmx = {}
    with lt.Ensemble(L, chi, n, precision=lt.LT_MIXED, **kw) as em:
        s0 = 0
        for ck in checkpoints:
            got = gpu_steps(em, cfg, ck - s0, replay=rec, step0=s0)
            assert np.array_equal(got, rec[:, s0:ck])
            s0 = ck
            cmx[ck] = em.corr(per_traj=True)[1]
    ens = {ck: float(np.abs(cmx[ck].mean(0) - c64[ck].mean(0)).max()) for ck in checkpoints}
    print("W3 ensemble |C_mixed - C_fp64|:", {k: "%.2e" % v for k, v in ens.items()})
    assert ens[50] <= 1e-6
    assert ens[100] <= 4e-6 and ens[150] <= 4e-6
    exact = slater.run_slater(cfg, rec, n_steps=200).mean(0)
    e64 = float(np.abs(c64[200].mean(0) - exact).max())
    emx = float(np.abs(cmx[200].mean(0) - exact).max())
    print("step 200: FP64 vs exact %.2e, mixed vs exact %.2e" % (e64, emx))
    assert emx <= 1.5 * e64 + 1e-5
    assert ens[200] <= e64


# ---- synthetic states: ragged dims, several tiles, truncation active ---------------------
@pytest.mark.parametrize("L,chi,ragged,seed", [(10, 8, True, 1), (12, 16, True, 2),
                                               (9, 5, False, 3), (16, 32, True, 4),
                                               (16, 128, False, 5)])
def test_synthetic_state_one_step_fp64(L, chi, ragged, seed):
    w = dict(workloads.W3, L=L, chi_max=chi, gamma_loss=0.3, gamma_gain=0.05, gamma_deph=0.1)
    cfg = oracle_cfg(w, L=L, chi=chi, dt=0.05, seed=seed)
    n = 3
    states = [workloads.synthetic_mps(L, chi, seed=100 * seed + t, ragged=ragged) for t in range(n)]
    res = tebd.run_trajectories(cfg, 2, list(range(n)), measure_corr=True,
                                initial=[(B, lam) for B, lam, _ in states])
    lt = _lt()
    with gpu_ensemble(cfg, n, lt.LT_FP64) as ens:
        ens.set_state(0, states)
        chans = gpu_steps(ens, cfg, 2)
        _, _, dens = ens.density(per_traj=True)
        _, Cp = ens.corr(per_traj=True)
        tw, dims = ens.stats()
    assert np.array_equal(chans, res["jumps"])
    assert np.array_equal(dims, res["bond_dims"])
    assert_close(dens, res["density"], FP64_TOL, "density")
    assert_close(Cp, res["corr"], FP64_TOL, "corr")
    assert np.abs(tw - res["trunc"]).max() < 1e-11


def test_forced_jump_then_recanonicalise_fp64():
    L, chi = 12, 16
    cfg = oracle_cfg(dict(workloads.W3, gamma_gain=0.1, gamma_deph=0.1), L=L, chi=chi, dt=0.05)
    n = 6
    states = [workloads.synthetic_mps(L, chi, seed=70 + t, ragged=True) for t in range(n)]
    # every channel kind at several sites, including both chain ends
    replay = np.array([[0], [3 * 5 + 1], [3 * 11 + 0], [3 * 7 + 2], [3 * 11 + 1], [-1]])
    res = tebd.run_trajectories(cfg, 1, list(range(n)), replay=replay, measure_corr=True,
                                initial=[(B, lam) for B, lam, _ in states])
    lt = _lt()
    with gpu_ensemble(cfg, n, lt.LT_FP64) as ens:
        ens.set_state(0, states)
        gpu_steps(ens, cfg, 1, replay=replay)
        _, _, dens = ens.density(per_traj=True)
        _, Cp = ens.corr(per_traj=True)
        tw, dims = ens.stats()
    assert np.array_equal(dims, res["bond_dims"])
    assert_close(dens, res["density"], FP64_TOL, "density")
    assert_close(Cp, res["corr"], FP64_TOL, "corr")


# ---- the W3 chain at full size (L=64, chi_max=64) on sampled outputs -------------------
def test_w3_full_size_sampled_trajectories_fp64_and_mixed():
    L, chi, n = 64, 64, 2
    cfg = oracle_cfg(workloads.W3)
    states = [workloads.synthetic_mps(L, chi, seed=900 + t) for t in range(n)]
    res = tebd.run_trajectories(cfg, 1, list(range(n)),
                                initial=[(B, lam) for B, lam, _ in states])
    lt = _lt()
    for prec, tol in ((lt.LT_FP64, FP64_TOL), (lt.LT_MIXED, 2e-5)):
        with gpu_ensemble(cfg, n, prec) as ens:
            ens.set_state(0, states)
            chans = gpu_steps(ens, cfg, 1, replay=res["jumps"])
            _, _, dens = ens.density(per_traj=True)
            _, dims = ens.stats()
        assert np.array_equal(chans, res["jumps"])
        if prec == lt.LT_FP64:
            assert np.array_equal(dims, res["bond_dims"])
        assert_close(dens, res["density"], tol, "density %d" % prec)


# ---- edge cases --------------------------------------------------------------------------
@pytest.mark.parametrize("L,chi,init", [(2, 1, "neel"), (2, 2, "domain_wall"), (3, 1, "neel"),
                                        (5, 2, "vacuum"), (7, 64, "neel")])
def test_edge_cases_fp64(L, chi, init):
    w = dict(workloads.W1, L=L, chi_max=chi, gamma_gain=0.2, init=init)
    cfg = oracle_cfg(w, L=L, chi=chi)
    n, steps = 5, 12
    res = tebd.run_trajectories(cfg, steps, list(range(n)), measure_corr=True)
    lt = _lt()
    with gpu_ensemble(cfg, n, lt.LT_FP64, init=init) as ens:
        chans = gpu_steps(ens, cfg, steps)
        _, _, dens = ens.density(per_traj=True)
        _, Cp = ens.corr(per_traj=True)
    assert np.array_equal(chans, res["jumps"])
    assert_close(dens, res["density"], FP64_TOL, "density")
    assert_close(Cp, res["corr"], FP64_TOL, "corr")


def test_lt_step_matches_manual_schedule_and_checkpoint(tmp_path):
    cfg = oracle_cfg(workloads.W1, L=10, chi=8)
    lt = _lt()
    n = 16
    with gpu_ensemble(cfg, n, lt.LT_FP64) as a:
        a.step(10)
        da = a.density(per_traj=True)[2]
        assert lt.lt_get_step(a.ctx) == 10
    with gpu_ensemble(cfg, n, lt.LT_FP64) as b:
        b.step(4)
        lt.lt_save(b.ctx, str(tmp_path / "ck.bin"))
    with gpu_ensemble(cfg, n, lt.LT_FP64) as c:
        lt.lt_load(c.ctx, str(tmp_path / "ck.bin"))
        assert lt.lt_get_step(c.ctx) == 4
        c.step(6)
        dc = c.density(per_traj=True)[2]
    assert np.array_equal(da, dc)
    res = tebd.run_trajectories(cfg, 10, list(range(n)))
    assert_close(da, res["density"], FP64_TOL, "lt_step density")


def test_large_dt_is_reported_and_poisons_the_context():
    lt = _lt()
    ens = lt.Ensemble(6, 4, 2, precision=lt.LT_FP64, dt=2.0, gamma_loss=1.0)
    with pytest.raises(lt.LtError) as e:
        ens.apply_jumps(0)
    assert e.value.status == lt.LT_ERR_NUMERICAL
    with pytest.raises(lt.LtError) as e:
        ens.step(1)
    assert e.value.status == lt.LT_ERR_STATE
    ens.close()


@pytest.mark.parametrize("precision_name", ["fp64", "mixed"])
def test_trajectory_shards_reproduce_the_unsharded_ensemble(precision_name):
    """Ranks own contiguous ranges of global trajectory ids (traj_offset); the
    jump draws are keyed by the global id, so two shards must give exactly the
    trajectories of one context holding all of them."""
    from paper_2609_18841_b300 import shard
    lt = _lt()
    prec = lt.LT_FP64 if precision_name == "fp64" else lt.LT_MIXED
    L, chi, n_total, steps = 10, 8, 9, 8
    kw = dict(precision=prec, init="neel", dt=0.05, gamma_loss=0.6, seed=5)
    with lt.Ensemble(L, chi, n_total, **kw) as whole:
        whole_j = gpu_steps(whole, oracle_cfg(workloads.W1, L=L, chi=chi, dt=0.05), steps)
        _, _, whole_d = whole.density(per_traj=True)
    parts_j, parts_d = [], []
    for r in range(2):
        off, n = shard.shard_range(n_total, r, 2)
        with lt.Ensemble(L, chi, n, traj_offset=off, **kw) as e:
            parts_j.append(gpu_steps(e, oracle_cfg(workloads.W1, L=L, chi=chi, dt=0.05), steps))
            parts_d.append(e.density(per_traj=True)[2])
    assert whole_j.max() >= 0, "the case should contain jumps"
    assert np.array_equal(np.concatenate(parts_j), whole_j)
    assert np.array_equal(np.concatenate(parts_d), whole_d)


def test_w3s_mixed_ensemble_agrees_with_fp64_to_1e6():
    """L=64, chi=64 from 16 distinct synthetic start states (32 trajectories),
    two full steps with the same svd_cut in both precisions: the FP64 path
    samples the jumps, the mixed path replays them; the ensemble <n_i> and C_ij
    must agree to 1e-6 (per trajectory the single-precision floor, 2e-5,
    applies)."""
    lt = _lt()
    L, chi, n, steps = 64, 64, 32, 2
    mps = [workloads.synthetic_mps(L, chi, seed=1234 + t) for t in range(16)]
    packed = lt.pack_state(mps, L, chi)
    kw = dict(init="neel", dt=0.02, gamma_loss=0.2)
    layers = [(0, 0.01), (1, 0.02), (0, 0.01)]

    def upload(e):
        for t0 in range(0, n, 16):
            lt.lt_set_state(e.ctx, t0, packed[0], packed[1], packed[2])

    with lt.Ensemble(L, chi, n, precision=lt.LT_FP64, svd_cut=1e-6, **kw) as ea, \
            lt.Ensemble(L, chi, n, precision=lt.LT_MIXED, svd_cut=1e-6, **kw) as em:
        upload(ea)
        upload(em)
        jumps = 0
        for s in range(steps):
            ch = np.ascontiguousarray(ea.apply_jumps(s), np.int32)
            em.apply_jumps(s, ch)
            jumps += int((ch >= 0).sum())
            for parity, tau in layers:
                ea.apply_layer(parity, tau)
                em.apply_layer(parity, tau)
        m64, _, d64 = ea.density(per_traj=True)
        mmx, _, dmx = em.density(per_traj=True)
        c64, cp64 = ea.corr(per_traj=True)
        cmx, cpmx = em.corr(per_traj=True)
    assert jumps > 0, "the case should contain jumps"
    assert_close(dmx, d64, 2e-5, "W3s mixed density per trajectory")
    assert_close(cpmx, cp64, 2e-5, "W3s mixed corr per trajectory")
    assert_close(mmx, m64, 1e-6, "W3s mixed density ensemble")
    assert_close(cmx, c64, 1e-6, "W3s mixed corr ensemble")


def test_contexts_of_different_chi_live_side_by_side():
    """The bond kernel's shared-memory ceiling is shared by all contexts of a
    process: creating a small-chi context must not break a live large-chi one."""
    lt = _lt()
    cfg_big = oracle_cfg(workloads.W1, L=12, chi=32)
    with gpu_ensemble(cfg_big, 4, lt.LT_MIXED) as big:
        gpu_steps(big, cfg_big, 3)
        cfg_small = oracle_cfg(workloads.W1, L=8, chi=4)
        with gpu_ensemble(cfg_small, 2, lt.LT_MIXED) as small:
            gpu_steps(small, cfg_small, 2)
            gpu_steps(big, cfg_big, 3, step0=3)
            gpu_steps(small, cfg_small, 2, step0=2)
            d_small = small.density(per_traj=True)[2]
        d_big = big.density(per_traj=True)[2]
    with gpu_ensemble(cfg_big, 4, lt.LT_MIXED) as ref:
        gpu_steps(ref, cfg_big, 6)
        assert np.array_equal(ref.density(per_traj=True)[2], d_big)
    with gpu_ensemble(cfg_small, 2, lt.LT_MIXED) as ref:
        gpu_steps(ref, cfg_small, 4)
        assert np.array_equal(ref.density(per_traj=True)[2], d_small)



def test_chi128_mixed_two_steps():
    """chi_max = 128 (theta up to 256 x 256, beyond the register paths) in mixed
    precision, jump records replayed from the oracle."""
    L, chi, n = 16, 128, 2
    w = dict(workloads.W3, L=L, chi_max=chi, gamma_loss=0.3, gamma_deph=0.1)
    cfg = oracle_cfg(w, L=L, chi=chi, dt=0.05, seed=6)
    states = [workloads.synthetic_mps(L, chi, seed=700 + t) for t in range(n)]
    res = tebd.run_trajectories(cfg, 2, list(range(n)), initial=[(B, lam) for B, lam, _ in states])
    lt = _lt()
    with gpu_ensemble(cfg, n, lt.LT_MIXED) as ens:
        ens.set_state(0, states)
        gpu_steps(ens, cfg, 2, replay=res["jumps"])
        _, _, dens = ens.density(per_traj=True)
    assert_close(dens, res["density"], 2e-5, "chi 128 mixed density")


def _two_site_blocks(B, lam, bonds, d):
    """Lambda_{b-1} B_b B_{b+1} as (d chi_{b-1}) x (d chi_{b+1}) matrices: after a
    two-site update this is theta~ V_k V_k^+ / |S_k| weighted, independent of the
    phases (and of rotations within degenerate subspaces) of the singular vectors."""
    out = {}
    for b in bonds:
        X = np.tensordot(B[b], B[b + 1], axes=(2, 0))
        X = X.reshape(X.shape[0] * d, -1)
        w = lam[b - 1] if b > 0 else np.ones(1)
        out[b] = X * np.repeat(w, d)[:, None]
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_wide_theta_whose_factor_takes_the_blocked_rows(precision, tol):
    # bond 7 of a 16-site chain with dims 38 | 100 | 70: theta is 76 x 140, too
    # wide for the register path, while its 76 x 76 triangular factor takes the
    # blocked Jacobi layout, whose rows are rounded up to 80
    from paper_2609_18841_b300.lindtebd import unpack_state
    lt = _lt()
    L, chi = 16, 128
    dims = [min(2 ** (b + 1), 2 ** (L - b - 1), 64) for b in range(L - 1)]
    dims[6], dims[7], dims[8] = 38, 100, 70
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=5, dims=dims)
    cut = 1e-12 if precision == "fp64" else 1e-6
    cfg = tebd.TrajectoryConfig(L, J=1.0, dt=0.05, chi_max=chi, svd_cut=cut, gamma_loss=0.2,
                                occupation=workloads.occupation(L, "neel"))
    ref = tebd.Trajectory.from_tensors(cfg, B, lam)
    ref.apply_layer(1, cfg.gates(0.05))
    prec = lt.LT_FP64 if precision == "fp64" else lt.LT_MIXED
    with lt.Ensemble(L, chi, 1, precision=prec, dt=0.05, gamma_loss=0.2, svd_cut=cut) as e:
        e.set_state(0, [(B, lam, dims)])
        e.apply_layer(1, 0.05)
        gd, gl, gB = e.get_state(0, 1)
    gBs, gls = unpack_state(gd[0], gl[0], gB[0], L)
    bonds = list(range(1, L - 1, 2))
    want = _two_site_blocks(ref.B, ref.lam, bonds, 2)
    got = _two_site_blocks(gBs, gls, bonds, 2)
    for b in bonds:
        err = np.abs(got[b] - want[b]).max() / np.abs(want[b]).max()
        assert err < tol, "bond %d: relative error %.2e" % (b, err)
    if precision == "fp64":
        assert list(gd[0]) == ref.bond_dims()


def test_w1_sampled_decisions_agree_between_precisions():
    """Both precisions sample their own jumps (no replay): a decision differs only
    when the Philox draw falls within the single-precision error of the rates
    (computed from single-precision environments, accumulated in double) of a
    channel boundary, after which the histories go apart.  On W1 (100
    trajectories x 40 steps) at most 2 % of the trajectories may part, and the
    trajectory-steps up to the first difference must agree exactly."""
    cfg = oracle_cfg(workloads.W1)
    lt = _lt()
    n = workloads.W1["n_traj"]
    recs = {}
    for prec in (lt.LT_FP64, lt.LT_MIXED):
        with gpu_ensemble(cfg, n, prec) as ens:
            recs[prec] = gpu_steps(ens, cfg, workloads.W1["n_steps"])
    a, b = recs[lt.LT_FP64], recs[lt.LT_MIXED]
    assert (a >= 0).sum() > 20, "the case should contain jumps"
    parted = np.nonzero((a != b).any(axis=1))[0]
    print("W1 sampled decisions: %d of %d trajectories part, %d of %d trajectory-steps differ"
          % (len(parted), n, int((a != b).sum()), a.size))
    assert len(parted) <= 0.02 * n


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_chi256_theta_512(precision, tol):
    # chi_max = 256 (the serving mix's largest): bond 8 of an 18-site chain with dims
    # 256 | 256 | 256 has theta 512 x 512; one layer against the oracle's update of the
    # same synthetic state (the gauge-invariant two-site blocks, as above)
    from paper_2609_18841_b300.lindtebd import unpack_state
    lt = _lt()
    L, chi = 18, 256
    dims = [min(2 ** (b + 1), 2 ** (L - b - 1), chi) for b in range(L - 1)]
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=18, dims=dims)
    cut = 1e-12 if precision == "fp64" else 1e-6
    cfg = tebd.TrajectoryConfig(L, J=1.0, dt=0.02, chi_max=chi, svd_cut=cut, gamma_loss=0.2,
                                occupation=workloads.occupation(L, "neel"))
    ref = tebd.Trajectory.from_tensors(cfg, B, lam)
    ref.apply_layer(0, cfg.gates(0.02))
    prec = lt.LT_FP64 if precision == "fp64" else lt.LT_MIXED
    with lt.Ensemble(L, chi, 1, precision=prec, dt=0.02, gamma_loss=0.2, svd_cut=cut) as e:
        e.set_state(0, [(B, lam, dims)])
        e.apply_layer(0, 0.02)
        gd, gl, gB = e.get_state(0, 1)
    gBs, gls = unpack_state(gd[0], gl[0], gB[0], L)
    bonds = list(range(0, L - 1, 2))
    want = _two_site_blocks(ref.B, ref.lam, bonds, 2)
    got = _two_site_blocks(gBs, gls, bonds, 2)
    for b in bonds:
        err = np.abs(got[b] - want[b]).max() / np.abs(want[b]).max()
        assert err < tol, "bond %d: relative error %.2e" % (b, err)
    if precision == "fp64":
        assert list(gd[0]) == ref.bond_dims()


@pytest.mark.parametrize("method", ["trajectory", "qsd"])
@pytest.mark.parametrize("chi", [128, 256])
def test_cluster_launch_equals_the_one_cta_launch_pure_state(chi, method):
    # One 18-site trajectory at chi_max = 128 or 256 (theta up to 256 or 512) gives a
    # layer 9 tasks: its single-precision layers go out as thread-block clusters that
    # share the wide Jacobi, the preconditioning, V_k^+ and the split; within 16
    # trajectories (144 tasks) each task has one CTA.  Same arithmetic: equal bit for
    # bit.  QSD keeps the norm change in B_b (the split is not rescaled).
    lt = _lt()
    L = 18
    dims = [min(2 ** (b + 1), 2 ** (L - b - 1), chi) for b in range(L - 1)]
    B, lam, dims = workloads.synthetic_mps(L, chi, seed=21, dims=dims)
    kw = dict(method=lt.LT_QSD, gamma_deph=0.1, fermionic_jumps=0) if method == "qsd" else {}
    runs = []
    for n in (1, 16):
        with lt.Ensemble(L, chi, n, precision=lt.LT_MIXED, dt=0.02, gamma_loss=0.2,
                         svd_cut=1e-6, **kw) as e:
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
