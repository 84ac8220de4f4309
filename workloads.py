"""Seeded synthetic inputs shared by the tests, the smoke run and the benchmark.

This module holds parameters and random-number draws only: no step of the TEBD
method's arithmetic.  Both the oracle and the CUDA library receive what it
returns, so the two never exchange data.

Workloads (the paper's free-fermion chain, Sec. 2.1, with fermionic jumps):
  W1  XX chain L=8, J=1, loss 0.1 on every site, Neel start, chi_max=16,
      second-order Trotter dt=0.05 to T=2 (40 steps), 100 trajectories, seed 0.
  W3  L=64, chi_max=64, loss 0.2 on every site, Neel start, dt=0.02 to T=4
      (200 steps), 4096 trajectories, seeds (0, trajectory id).
  W3s the W3 chain started from a synthetic right-canonical MPS (below) so that
      every step runs at the bond dimensions chi_max allows.
"""
import numpy as np

W1 = dict(name="W1", L=8, J=1.0, dt=0.05, n_steps=40, chi_max=16, n_traj=100,
          gamma_loss=0.1, gamma_gain=0.0, gamma_deph=0.0, fermionic=1,
          trotter_order=2, init="neel", seed=0)

W3 = dict(name="W3", L=64, J=1.0, dt=0.02, n_steps=200, chi_max=64, n_traj=4096,
          gamma_loss=0.2, gamma_gain=0.0, gamma_deph=0.0, fermionic=1,
          trotter_order=2, init="neel", seed=0)


def occupation(L, init):
    """Initial product state: Neel |1010...>, domain wall (left half full), vacuum."""
    occ = np.zeros(L, dtype=np.int64)
    if init == "neel":
        occ[0::2] = 1
    elif init == "domain_wall":
        occ[: L // 2] = 1
    elif init != "vacuum":
        raise ValueError(init)
    return occ


def structural_caps(L, chi_max, d=2):
    """chi_b <= min(d^(b+1), d^(L-1-b), chi_max) for bond b = 0..L-2."""
    caps = []
    for b in range(L - 1):
        left = d ** min(b + 1, 62)
        right = d ** min(L - 1 - b, 62)
        caps.append(int(min(left, right, chi_max)))
    return np.array(caps, dtype=np.int64)


def bond_dims(L, chi_max, rng=None, ragged=False, d=2):
    """Full (every bond at its cap) or ragged (uniform in 1..cap, then clamped so
    that neighbouring bonds differ by at most a factor d)."""
    caps = structural_caps(L, chi_max, d)
    if not ragged:
        return caps
    dims = np.array([rng.integers(1, c + 1) for c in caps], dtype=np.int64)
    for _ in range(2):
        for b in range(1, L - 1):
            dims[b] = min(dims[b], d * dims[b - 1])
        for b in range(L - 3, -1, -1):
            dims[b] = min(dims[b], d * dims[b + 1])
    dims[0] = min(dims[0], d)
    dims[-1] = min(dims[-1], d)
    return dims


def synthetic_mps(L, chi_max, seed, ragged=False, d=2, decay=8.0, dims=None):
    """Random MPS in (approximate) Vidal-Hastings form.

    B_i: i.i.d. complex Gaussian entries, made right-canonical by a QR
    factorisation of the conjugate transpose (rows orthonormal; needs
    chi_{i-1} <= d chi_i);
    Lambda_b,a proportional to exp(-a/decay), normalised to sum Lambda^2 = 1.
    dims: explicit bond dimensions [L-1] instead of drawn ones.
    Returns (B list of (chi_{i-1}, d, chi_i) complex128, lam list, dims)."""
    rng = np.random.default_rng(seed)
    if dims is None:
        dims = bond_dims(L, chi_max, rng, ragged, d)
    else:
        dims = np.asarray(dims, dtype=np.int64)
    full = [1] + [int(x) for x in dims] + [1]
    B = []
    for i in range(L):
        cl, cr = full[i], full[i + 1]
        X = (rng.standard_normal((d * cr, cl)) + 1j * rng.standard_normal((d * cr, cl)))
        Q, _ = np.linalg.qr(X)                        # (d cr) x cl, orthonormal columns
        B.append(Q.conj().T.reshape(cl, d, cr))       # rows orthonormal
    lam = []
    for b in range(L - 1):
        x = np.exp(-np.arange(full[b + 1]) / decay)
        lam.append(x / np.sqrt(np.sum(x ** 2)))
    return B, lam, dims


def random_theta_inputs(chiL, chiM, chiR, seed, d=2):
    """Two random site tensors and a random left weight for single-bond tests."""
    rng = np.random.default_rng(seed)
    Bl = rng.standard_normal((chiL, d, chiM)) + 1j * rng.standard_normal((chiL, d, chiM))
    Br = rng.standard_normal((chiM, d, chiR)) + 1j * rng.standard_normal((chiM, d, chiR))
    lam = np.sort(rng.random(chiL))[::-1] + 0.05
    return Bl, Br, lam / np.sqrt(np.sum(lam ** 2))
