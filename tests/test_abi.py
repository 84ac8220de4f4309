"""Host-side checks of the C ABI: the library loads, exports every function that
include/lindtebd.h declares, and rejects invalid configurations before it
touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lindtebd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lt_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2609_18841_b300 import lindtebd
    names = _declared()
    assert len(names) >= 21
    for n in names:
        assert hasattr(lindtebd._lib, n), n
    assert set(names) == set(lindtebd.EXPORTS)


def test_config_struct_layout_matches_header():
    from paper_2609_18841_b300.lindtebd import lt_config
    assert ctypes.sizeof(lt_config) == 128
    assert lt_config.J.offset == 40 and lt_config.svd_cut.offset == 88
    assert lt_config.traj_offset.offset == 104 and lt_config.jacobi_tol.offset == 112
    assert lt_config.theta_path.offset == 120 and lt_config.env_ctas_per_sm.offset == 124


@pytest.mark.parametrize("kw,status", [
    (dict(L=1), 1), (dict(chi_max=0), 1), (dict(chi_max=257), 1), (dict(n_traj=0), 1),
    (dict(dt=0.0), 1), (dict(trotter_order=3), 1), (dict(precision=5), 1),
    (dict(method=1, gamma_loss=0.1), 7), (dict(method=4), 7), (dict(gamma_loss=-0.1), 1),
    # the purified density matrix: Kraus dimension 2 only, chi_max <= 128, local jumps
    (dict(method=3, kraus_dim=3), 7), (dict(method=3, chi_max=129), 7),
    (dict(method=3, gamma_gain=[0, 0.1, 0, 0, 0, 0, 0, 0]), 7),
    # the vectorised density matrix: theta is 4 chi wide (chi_max <= 128), and a
    # fermionic loss or gain is local only on the chain ends
    (dict(method=2, chi_max=129), 7), (dict(method=2, chi_max=257), 1),
    (dict(method=2, gamma_loss=[0, 0, 0.1, 0, 0, 0, 0, 0]), 7),
    (dict(method=2, gamma_gain=[0, 0, 0, 0, 0, 0, 0.2, 0]), 7),
    (dict(init="product"), 1),
    # schedules: theta path 0..2, 0..8 CTAs per SM
    (dict(theta_path=3), 1), (dict(env_ctas_per_sm=9), 1),
])
def test_invalid_configurations_are_rejected_on_the_host(kw, status):
    from paper_2609_18841_b300 import lindtebd as lt
    args = dict(L=8, chi_max=16, n_traj=4)
    args.update(kw)
    L = args.pop("L")
    chi = args.pop("chi_max")
    n = args.pop("n_traj")
    with pytest.raises(lt.LtError) as e:
        lt.lt_create(L, chi, n, **args)
    assert e.value.status == status


def test_status_strings_and_null_context():
    from paper_2609_18841_b300 import lindtebd as lt
    for s in range(8):
        assert lt._lib.lt_status_str(s)
    assert lt._lib.lt_destroy(None) == lt.LT_ERR_ARG
    assert lt._lib.lt_step(None, 1) == lt.LT_ERR_ARG
    assert lt._lib.lt_step_graph(None, 1) == lt.LT_ERR_ARG
    assert lt._lib.lt_apply_kraus(None) == lt.LT_ERR_ARG
    assert lt._lib.lt_launch_count(None) == 0
    assert lt._lib.lt_cluster_launches(None) == 0
    out = ctypes.c_void_p(1)
    assert lt._lib.lt_create(None, None, ctypes.byref(out)) == lt.LT_ERR_ARG
    assert out.value is None


def test_pack_unpack_roundtrip():
    import workloads
    from paper_2609_18841_b300 import lindtebd as lt
    B, lam, dims = workloads.synthetic_mps(10, 8, seed=2, ragged=True)
    d, l, Bp = lt.pack_state([(B, lam, dims)], 10, 8)
    B2, lam2 = lt.unpack_state(d[0], l[0], Bp[0], 10)
    for x, y in zip(B, B2):
        assert np.array_equal(x, y)
    for x, y in zip(lam, lam2):
        assert np.array_equal(x, y)
