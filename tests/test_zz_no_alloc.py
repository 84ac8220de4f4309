"""The allocation-free density entry point, for callers that cannot call
cudaMalloc (their device memory belongs to another allocator, or they cannot
take the synchronisation an allocation may cause).  Its results must equal
what the context-based lt_measure_density returns per trajectory, on two calls
in a row that share the library's static scratch array.  This file is collected
last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 parity tolerance of the other GPU tests, scaled by max |value|


@pytest.mark.parametrize("precision_name", ["fp64", "mixed"])
def test_noalloc_density_matches_context_measurement(precision_name):
    import torch
    from paper_2609_18841_b300 import lindtebd as lt

    prec = lt.LT_FP64 if precision_name == "fp64" else lt.LT_MIXED
    L, chi, n = 14, 16, 6
    states = [workloads.synthetic_mps(L, chi, seed=600 + t, ragged=True) for t in range(n)]
    with lt.Ensemble(L, chi, n, precision=prec, init="neel", dt=0.05, gamma_loss=0.3,
                     gamma_deph=0.1, seed=7) as ens:
        ens.set_state(0, states)
        ens.step(3)
        _, _, want = ens.density(per_traj=True)
        dims, lam, B = ens.get_state(0, n)

    dev = torch.device("cuda", 0)
    cdt = torch.complex128 if prec == lt.LT_FP64 else torch.complex64
    d_B = torch.from_numpy(B).to(device=dev, dtype=cdt).contiguous()
    d_dims = torch.from_numpy(dims).to(device=dev).contiguous()
    d_out = torch.empty((n, L), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    scale = max(1.0, float(np.abs(want).max()))
    for call in range(2):
        d_out.fill_(float("nan"))
        st = lt.lt_measure_density_noalloc(prec, L, chi, n, d_B.data_ptr(), d_dims.data_ptr(),
                                           d_out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        assert st == lt.LT_OK, "call %d returned %d" % (call, st)
        got = d_out.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = float(np.abs(got - want).max())
        assert err <= TOL * scale, "call %d: max |diff| %.3e" % (call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2609_18841_b300 import lindtebd as lt

    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    # (L + 8) chi^2 complex128 per trajectory: L = 600, chi = 64 needs 38 MiB > 32 MiB
    assert lt.lt_measure_density_noalloc(lt.LT_FP64, 600, 64, 1, p, p, p, None) == lt.LT_ERR_ARG
    assert lt.lt_measure_density_noalloc(lt.LT_FP64, 8, 257, 1, p, p, p, None) == lt.LT_ERR_ARG
    assert lt.lt_measure_density_noalloc(lt.LT_MIXED, 8, 8, 1, p, None, p, None) == lt.LT_ERR_ARG
    assert lt.lt_measure_density_noalloc(lt.LT_FP64, 8, 8, 0, p, p, p, None) == lt.LT_ERR_ARG


def test_noalloc_skips_trajectories_with_dimensions_out_of_range():
    # the kernel checks every bond dimension of a trajectory against [1, chi_max]
    # before it reads a site: a trajectory outside it gets NaN densities, the
    # others are measured as usual
    import torch
    from paper_2609_18841_b300 import lindtebd as lt

    L, chi, n = 10, 8, 4
    states = [workloads.synthetic_mps(L, chi, seed=700 + t, ragged=True) for t in range(n)]
    with lt.Ensemble(L, chi, n, precision=lt.LT_MIXED, init="neel", dt=0.05, gamma_loss=0.3,
                     seed=3) as ens:
        ens.set_state(0, states)
        _, _, want = ens.density(per_traj=True)
        dims, lam, B = ens.get_state(0, n)
    dims = dims.copy()
    dims[1, 3] = chi + 5
    dims[3, 0] = 0
    dev = torch.device("cuda", 0)
    d_B = torch.from_numpy(B).to(device=dev, dtype=torch.complex64).contiguous()
    d_dims = torch.from_numpy(dims).to(device=dev).contiguous()
    d_out = torch.zeros((n, L), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = lt.lt_measure_density_noalloc(lt.LT_MIXED, L, chi, n, d_B.data_ptr(), d_dims.data_ptr(),
                                       d_out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    assert st == lt.LT_OK
    got = d_out.cpu().numpy()
    assert np.all(np.isnan(got[1])) and np.all(np.isnan(got[3]))
    ok = [0, 2]
    assert np.abs(got[ok] - want[ok]).max() <= TOL * max(1.0, float(np.abs(want).max()))
