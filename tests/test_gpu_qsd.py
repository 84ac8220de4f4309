"""GPU parity of quantum state diffusion (Sec. 5.2) through the C ABI against the
FP64 oracle: same Philox Gaussian noise on both sides, so every unnormalised
history, its log weight ln <psi|psi> and the weighted ensemble estimator
mean_t(w_t <O>_t) must agree (FP64 within 1e-10; mixed precision within the
single-precision bounds of the trajectory tests)."""
import numpy as np
import pytest

import workloads
from oracle import tebd

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _lt():
    from paper_2609_18841_b300 import lindtebd
    return lindtebd


def qsd_cfg(L, chi, dt=0.05, loss=None, deph=0.2, fermionic=True, seed=4, occ="neel"):
    g_loss = np.zeros(L)
    if loss is None:
        g_loss[0] = 0.3
    else:
        g_loss[:] = loss
    return tebd.TrajectoryConfig(L, J=1.0, dt=dt, chi_max=chi, svd_cut=1e-12, gamma_loss=g_loss,
                                 gamma_deph=deph, fermionic=fermionic,
                                 occupation=workloads.occupation(L, occ), seed=seed)


def gpu_qsd(cfg, n, precision, cut=None):
    lt = _lt()
    return lt.Ensemble(cfg.L, cfg.chi_max, n, method=lt.LT_QSD, precision=precision, init="neel",
                       J=cfg.J, dt=cfg.dt, gamma_loss=cfg.gamma_loss, gamma_deph=cfg.gamma_deph,
                       fermionic_jumps=int(cfg.fermionic), svd_cut=cfg.svd_cut if cut is None else cut,
                       seed=cfg.seed)


def run_gpu(ens, cfg, n_steps):
    for s in range(n_steps):
        for parity, tau in cfg.layers():
            ens.apply_layer(parity, tau)
        ens.apply_noise(s)


def close(got, want, tol, what):
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(got - want).max())
    assert err <= tol * scale, "%s: max |diff| %.3e > %.1e" % (what, err, tol * scale)
    return err


@pytest.fixture(scope="module")
def qsd_oracle():
    cfg = qsd_cfg(8, 16)
    n, steps = 12, 10
    return cfg, n, steps, tebd.run_qsd(cfg, steps, list(range(n)), measure_corr=True)


def test_qsd_fp64_histories_weights_and_estimator(qsd_oracle):
    cfg, n, steps, res = qsd_oracle
    lt = _lt()
    with gpu_qsd(cfg, n, lt.LT_FP64) as ens:
        run_gpu(ens, cfg, steps)
        mean, sem, dens = ens.density(per_traj=True)
        C, Cp = ens.corr(per_traj=True)
        logw = ens.log_weights()
    close(logw, res["log_weight"], FP64_TOL, "log weight")
    close(dens, res["density"], FP64_TOL, "density per history")
    close(Cp, res["corr"], FP64_TOL, "corr per history")
    want_mean, want_sem = tebd.qsd_estimate(res["density"], res["log_weight"])
    close(mean, want_mean, FP64_TOL, "weighted density estimator")
    close(sem, want_sem, FP64_TOL, "its CLT error")
    want_C, _ = tebd.qsd_estimate(res["corr"], res["log_weight"])
    close(C, want_C, FP64_TOL, "weighted corr estimator")
    assert np.abs(res["log_weight"]).max() > 1e-3, "the weights should move"


def test_qsd_mixed_histories(qsd_oracle):
    cfg, n, steps, res = qsd_oracle
    lt = _lt()
    with gpu_qsd(cfg, n, lt.LT_MIXED, cut=1e-6) as ens:
        run_gpu(ens, cfg, steps)
        mean, _, dens = ens.density(per_traj=True)
        logw = ens.log_weights()
    close(logw, res["log_weight"], 2e-5, "mixed log weight")
    close(dens, res["density"], 2e-5, "mixed density per history")
    want_mean, _ = tebd.qsd_estimate(res["density"], res["log_weight"])
    close(mean, want_mean, 2e-5, "mixed weighted estimator")


def test_qsd_mixed_log_weight_does_not_drift():
    # ln <psi|psi> of single-precision histories against the FP64 path on the same
    # Philox noise (32 sites, spin loss and dephasing everywhere, 40 steps).  The
    # single-precision steps bias the norm the same way in every history, so the
    # mean difference grows step by step; measured -3.9e-5 after 40 steps (2.5e-5
    # of it from step 20 on).  Taking the restored Schmidt spectrum from the singular
    # values instead of from the norms of the tensors the sweep stores doubles it
    # (-7.7e-5, 5.0e-5 from step 20 on), which these bounds reject.
    cfg = qsd_cfg(32, 64, dt=0.01, loss=0.05, deph=0.1, fermionic=False)
    n, marks = 32, (10, 20, 30, 40)
    lt = _lt()
    logw = {}
    for prec in (lt.LT_FP64, lt.LT_MIXED):
        with gpu_qsd(cfg, n, prec, cut=1e-6) as ens:
            for s in range(marks[-1]):
                for parity, tau in cfg.layers():
                    ens.apply_layer(parity, tau)
                ens.apply_noise(s)
                if s + 1 in marks:
                    logw[prec, s + 1] = ens.log_weights().copy()
    d = [logw[lt.LT_MIXED, t] - logw[lt.LT_FP64, t] for t in marks]
    mean = [float(x.mean()) for x in d]
    print("mixed - FP64 ln w, mean over histories at steps", marks, mean,
          "max", float(np.abs(d[-1]).max()))
    assert np.abs(logw[lt.LT_FP64, marks[-1]]).max() > 1e-2, "the weights should move"
    assert abs(mean[-1]) <= 5e-5 and abs(mean[-1] - mean[1]) <= 3.5e-5, mean


def test_qsd_spin_loss_from_truncated_synthetic_states():
    # spin loss on every site (local), dephasing, ragged start states, chi = 8
    # truncation active
    L, chi, n, steps = 12, 8, 4, 6
    cfg = qsd_cfg(L, chi, dt=0.04, loss=0.15, deph=0.1, fermionic=False)
    lt = _lt()
    states = [workloads.synthetic_mps(L, chi, seed=900 + t, ragged=True) for t in range(n)]
    res = tebd.run_qsd(cfg, steps, list(range(n)), initial=[(B, lam) for B, lam, _ in states])
    with gpu_qsd(cfg, n, lt.LT_FP64) as ens:
        ens.set_state(0, states)
        run_gpu(ens, cfg, steps)
        _, _, dens = ens.density(per_traj=True)
        logw = ens.log_weights()
        tw, dims = ens.stats()
    close(logw, res["log_weight"], FP64_TOL, "log weight")
    close(dens, res["density"], FP64_TOL, "density")
    assert np.array_equal(dims, res["bond_dims"])


def test_qsd_step_checkpoint_and_method_errors(tmp_path):
    cfg = qsd_cfg(8, 8)
    lt = _lt()
    n = 6
    with gpu_qsd(cfg, n, lt.LT_FP64) as a:
        a.step(5)
        da, wa = a.density(per_traj=True)[2], a.log_weights()
        with pytest.raises(lt.LtError) as e:
            a.apply_jumps(5)
        assert e.value.status == lt.LT_ERR_UNSUPPORTED
    with gpu_qsd(cfg, n, lt.LT_FP64) as b:
        run_gpu(b, cfg, 2)
        lt.lt_save(b.ctx, str(tmp_path / "q.bin"))
    with gpu_qsd(cfg, n, lt.LT_FP64) as c:
        lt.lt_load(c.ctx, str(tmp_path / "q.bin"))
        for s in range(2, 5):
            for parity, tau in cfg.layers():
                c.apply_layer(parity, tau)
            c.apply_noise(s)
        dc, wc = c.density(per_traj=True)[2], c.log_weights()
    assert np.array_equal(da, dc) and np.array_equal(wa, wc)
    with lt.Ensemble(8, 8, 2, precision=lt.LT_FP64, gamma_deph=0.1) as t:
        with pytest.raises(lt.LtError) as e:
            t.apply_noise(0)
        assert e.value.status == lt.LT_ERR_UNSUPPORTED
    with pytest.raises(lt.LtError) as e:
        lt.Ensemble(8, 8, 2, method=lt.LT_QSD, gamma_loss=0.1, fermionic_jumps=1)
    assert e.value.status == lt.LT_ERR_UNSUPPORTED


@pytest.mark.parametrize("L,chi,fermionic,loss,gain,deph", [
    (2, 1, True, [0.3, 0.0], 0.0, 0.2),          # one bond, product states only
    (6, 8, False, 0.1, 0.2, 0.1),                # spin gain and loss on every site
    (7, 4, True, [0.4] + [0.0] * 6, 0.0, 0.15),  # odd length, truncation at chi 4
])
def test_qsd_gain_edges_and_small_chains(L, chi, fermionic, loss, gain, deph):
    cfg = tebd.TrajectoryConfig(L, J=1.0, dt=0.05, chi_max=chi, svd_cut=1e-12, gamma_loss=loss,
                                gamma_gain=gain, gamma_deph=deph, fermionic=fermionic,
                                occupation=workloads.occupation(L, "neel"), seed=9)
    n, steps = 3, 6
    res = tebd.run_qsd(cfg, steps, list(range(n)))
    lt = _lt()
    with lt.Ensemble(L, chi, n, method=lt.LT_QSD, precision=lt.LT_FP64, init="neel", J=1.0,
                     dt=0.05, gamma_loss=cfg.gamma_loss, gamma_gain=cfg.gamma_gain,
                     gamma_deph=cfg.gamma_deph, fermionic_jumps=int(fermionic), svd_cut=1e-12,
                     seed=9) as ens:
        ens.step(steps)
        _, _, dens = ens.density(per_traj=True)
        logw = ens.log_weights()
    close(logw, res["log_weight"], FP64_TOL, "log weight")
    close(dens, res["density"], FP64_TOL, "density")
