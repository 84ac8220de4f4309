"""ctypes binding of the lindtebd C ABI (include/lindtebd.h).

Argument marshalling only: every step of the integrator runs in the CUDA
library.  Importing this module loads liblindtebd.so and raises ImportError if
it has not been built (there is no fallback implementation).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblindtebd.so")

LT_OK, LT_ERR_ARG, LT_ERR_OOM, LT_ERR_CUDA, LT_ERR_NUMERICAL, LT_ERR_TIMEOUT, \
    LT_ERR_STATE, LT_ERR_UNSUPPORTED = range(8)
LT_TRAJ, LT_QSD, LT_MPDO, LT_PURIFIED = range(4)
LT_FP64, LT_MIXED = 0, 1
LT_INIT_VACUUM, LT_INIT_NEEL, LT_INIT_DOMAIN_WALL, LT_INIT_PRODUCT = range(4)
INIT_NAMES = {"vacuum": LT_INIT_VACUUM, "neel": LT_INIT_NEEL,
              "domain_wall": LT_INIT_DOMAIN_WALL, "product": LT_INIT_PRODUCT}


class lt_config(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32), ("chi_max", ctypes.c_int32), ("n_traj", ctypes.c_int32),
        ("kraus_dim", ctypes.c_int32), ("method", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("init", ctypes.c_int32),
        ("trotter_order", ctypes.c_int32), ("product_occ", ctypes.c_void_p),
        ("J", ctypes.c_double), ("dt", ctypes.c_double),
        ("gamma_loss", ctypes.c_void_p), ("gamma_gain", ctypes.c_void_p),
        ("gamma_deph", ctypes.c_void_p), ("fermionic_jumps", ctypes.c_int32),
        ("max_sweeps", ctypes.c_int32), ("svd_cut", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("traj_offset", ctypes.c_int64),
        ("jacobi_tol", ctypes.c_double), ("theta_path", ctypes.c_int32),
        ("env_ctas_per_sm", ctypes.c_int32),
    ]


EXPORTS = ["lt_create", "lt_destroy", "lt_apply_layer", "lt_apply_jumps", "lt_apply_noise",
           "lt_apply_kraus", "lt_get_log_weights",
           "lt_step", "lt_step_graph", "lt_gates", "lt_measure_density", "lt_measure_corr", "lt_get_stats", "lt_set_state",
           "lt_get_state", "lt_save", "lt_load", "lt_get_sweep_histogram", "lt_get_counters", "lt_measure_density_noalloc", "lt_launch_count", "lt_cluster_launches", "lt_stream", "lt_get_step", "lt_pipe_peaks",
           "lt_status_str", "lt_last_error", "lt_context_bytes", "lt_admit_plan",
           "lt_server_create", "lt_server_destroy", "lt_server_submit", "lt_server_tick",
           "lt_server_result", "lt_server_error", "lt_server_usage", "lt_server_updates"]


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("liblindtebd.so is not built (run paper_2609_18841_b300/build.py)")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "lt_create": ([ctypes.POINTER(lt_config), P, ctypes.POINTER(P)], I32),
        "lt_destroy": ([P], I32),
        "lt_apply_layer": ([P, I32, D], I32),
        "lt_apply_jumps": ([P, I64, P, P], I32),
        "lt_apply_noise": ([P, I64], I32),
        "lt_apply_kraus": ([P], I32),
        "lt_get_log_weights": ([P, P], I32),
        "lt_step": ([P, I32], I32),
        "lt_step_graph": ([P, I32], I32),
        "lt_gates": ([ctypes.POINTER(lt_config), D, P, I64], I32),
        "lt_measure_density": ([P, P, P, P], I32),
        "lt_measure_corr": ([P, P, P, P, P], I32),
        "lt_get_stats": ([P, P, P], I32),
        "lt_set_state": ([P, I32, I32, P, P, P], I32),
        "lt_get_state": ([P, I32, I32, P, P, P], I32),
        "lt_save": ([P, ctypes.c_char_p], I32),
        "lt_load": ([P, ctypes.c_char_p], I32),
        "lt_get_sweep_histogram": ([P, P, I32], I32),
        "lt_get_counters": ([P, P, I32], I32),
        "lt_measure_density_noalloc": ([I32, I32, I32, I32, P, P, P, P], I32),
        "lt_launch_count": ([P], I64),
        "lt_cluster_launches": ([P], I64),
        "lt_pipe_peaks": ([P], I32),
        "lt_stream": ([P], P),
        "lt_get_step": ([P], I64),
        "lt_status_str": ([I32], ctypes.c_char_p),
        "lt_context_bytes": ([ctypes.POINTER(lt_config), I32, P], I32),
        "lt_admit_plan": ([ctypes.c_uint64, ctypes.c_uint64, I32, I32, P, I32, P], I32),
        "lt_server_create": ([ctypes.c_uint64, I32, ctypes.POINTER(P)], I32),
        "lt_server_destroy": ([P], I32),
        "lt_server_submit": ([P, ctypes.POINTER(lt_config), I32, P], I32),
        "lt_server_tick": ([P, P, P, P], I32),
        "lt_server_result": ([P, I64, P, P, P], I32),
        "lt_server_usage": ([P, P, P], I32),
        "lt_server_updates": ([P, I64, P], I32),
        "lt_server_error": ([P, I64], ctypes.c_char_p),
        "lt_last_error": ([P], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = load_library()


class LtError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = "%s failed: %s" % (where, _lib.lt_status_str(status).decode())
        if detail:
            msg += " (%s)" % detail
        super().__init__(msg)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(status, where, ctx=None):
    if status != LT_OK:
        detail = _lib.lt_last_error(ctx).decode() if ctx else ""
        raise LtError(status, where, detail)


def _arr(x, L, dtype=np.float64):
    if x is None:
        return None
    return np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype), (L,)))


def make_config(L, chi_max, n_traj, precision=LT_FP64, init="neel", J=1.0, dt=0.05,
                trotter_order=2, gamma_loss=None, gamma_gain=None, gamma_deph=None,
                fermionic_jumps=1, svd_cut=1e-12, seed=0, traj_offset=0, product_occ=None,
                method=LT_TRAJ, max_sweeps=0, jacobi_tol=0.0, kraus_dim=0, theta_path=0,
                env_ctas_per_sm=0):
    """An lt_config and the arrays it points to (keep both alive while it is used)."""
    cfg = lt_config()
    cfg.L, cfg.chi_max, cfg.n_traj = L, chi_max, n_traj
    cfg.kraus_dim, cfg.method, cfg.precision = kraus_dim, method, precision
    cfg.init = INIT_NAMES[init] if isinstance(init, str) else int(init)
    cfg.trotter_order, cfg.J, cfg.dt = trotter_order, J, dt
    keep = [_arr(gamma_loss, L), _arr(gamma_gain, L), _arr(gamma_deph, L),
            None if product_occ is None else np.ascontiguousarray(product_occ, np.uint8)]
    cfg.gamma_loss, cfg.gamma_gain, cfg.gamma_deph = (_ptr(k) for k in keep[:3])
    cfg.product_occ = _ptr(keep[3])
    cfg.fermionic_jumps, cfg.svd_cut = int(fermionic_jumps), svd_cut
    cfg.seed, cfg.traj_offset = seed, traj_offset
    cfg.max_sweeps, cfg.jacobi_tol = max_sweeps, jacobi_tol
    cfg.theta_path, cfg.env_ctas_per_sm = int(theta_path), int(env_ctas_per_sm)
    return cfg, keep


def lt_create(L, chi_max, n_traj, stream=None, **kw):
    """Create a context (keyword arguments as make_config)."""
    cfg, keep = make_config(L, chi_max, n_traj, **kw)
    h = ctypes.c_void_p()
    _check(_lib.lt_create(ctypes.byref(cfg), stream, ctypes.byref(h)), "lt_create")
    return h


def lt_destroy(ctx):
    _check(_lib.lt_destroy(ctx), "lt_destroy")


def lt_apply_layer(ctx, parity, tau):
    _check(_lib.lt_apply_layer(ctx, parity, tau), "lt_apply_layer", ctx)


def lt_apply_jumps(ctx, step, replay=None, n_traj=None, want_channels=False):
    rep = None if replay is None else np.ascontiguousarray(replay, np.int32)
    out = None
    if want_channels:
        out = np.empty(n_traj if n_traj is not None else len(rep), np.int32)
    _check(_lib.lt_apply_jumps(ctx, step, _ptr(rep), _ptr(out)), "lt_apply_jumps", ctx)
    return out


def lt_apply_noise(ctx, step):
    _check(_lib.lt_apply_noise(ctx, step), "lt_apply_noise", ctx)


def lt_apply_kraus(ctx):
    _check(_lib.lt_apply_kraus(ctx), "lt_apply_kraus", ctx)


def lt_get_log_weights(ctx, n_traj):
    out = np.empty(n_traj)
    _check(_lib.lt_get_log_weights(ctx, _ptr(out)), "lt_get_log_weights", ctx)
    return out


def lt_step(ctx, n_steps):
    _check(_lib.lt_step(ctx, n_steps), "lt_step", ctx)


def lt_gates(L, tau, **kw):
    """The gates a context of these settings builds for time step tau (host only):
    (L-1, D^2, D^2) complex, D = 2 or 4 by method."""
    cfg, keep = make_config(L, 1, 1, **kw)
    D = 4 if cfg.method in (LT_MPDO, LT_PURIFIED) else 2
    out = np.empty(2 * D ** 4 * (L - 1))
    _check(_lib.lt_gates(ctypes.byref(cfg), tau, _ptr(out), out.size), "lt_gates")
    return out.view(np.complex128).reshape(L - 1, D * D, D * D)


def lt_step_graph(ctx, n_steps):
    _check(_lib.lt_step_graph(ctx, n_steps), "lt_step_graph", ctx)


def lt_measure_density(ctx, L, n_traj, per_traj=False, out=None):
    mean = np.empty(L) if out is None else out[0]
    sem = np.empty(L) if out is None else out[1]
    pt = np.empty((n_traj, L)) if per_traj else None
    _check(_lib.lt_measure_density(ctx, _ptr(mean), _ptr(sem), _ptr(pt)), "lt_measure_density", ctx)
    return mean, sem, pt


def lt_measure_corr(ctx, L, n_traj, per_traj=False):
    re, im = np.empty((L, L)), np.empty((L, L))
    pre = np.empty((n_traj, L, L)) if per_traj else None
    pim = np.empty((n_traj, L, L)) if per_traj else None
    _check(_lib.lt_measure_corr(ctx, _ptr(re), _ptr(im), _ptr(pre), _ptr(pim)),
           "lt_measure_corr", ctx)
    return re + 1j * im, (None if pre is None else pre + 1j * pim)


def lt_get_stats(ctx, L, n_traj):
    tw = np.empty(n_traj)
    dims = np.empty((n_traj, L - 1), np.int32)
    _check(_lib.lt_get_stats(ctx, _ptr(tw), _ptr(dims)), "lt_get_stats", ctx)
    return tw, dims


def lt_set_state(ctx, traj0, dims, lam, B):
    """dims [n, L-1] int32, lam [n, L-1, chi] float64, B [n, L, d chi^2] complex128
    (d = 2 for pure states, 4 for the vectorised density matrix)."""
    dims = np.ascontiguousarray(dims, np.int32)
    lam = np.ascontiguousarray(lam, np.float64)
    B = np.ascontiguousarray(B, np.complex128)
    _check(_lib.lt_set_state(ctx, traj0, dims.shape[0], _ptr(dims), _ptr(lam), _ptr(B)),
           "lt_set_state", ctx)


def lt_get_state(ctx, traj0, n, L, chi, d=2):
    dims = np.empty((n, L - 1), np.int32)
    lam = np.empty((n, L - 1, chi))
    B = np.empty((n, L, d * chi * chi), np.complex128)
    _check(_lib.lt_get_state(ctx, traj0, n, _ptr(dims), _ptr(lam), _ptr(B)), "lt_get_state", ctx)
    return dims, lam, B


def lt_save(ctx, path):
    _check(_lib.lt_save(ctx, path.encode()), "lt_save", ctx)


def lt_load(ctx, path):
    _check(_lib.lt_load(ctx, path.encode()), "lt_load", ctx)


def lt_get_sweep_histogram(ctx, clear=False):
    h = np.zeros(64, np.int32)
    _check(_lib.lt_get_sweep_histogram(ctx, _ptr(h), int(clear)), "lt_get_sweep_histogram", ctx)
    return h


COUNTER_NAMES = ("updates", "rotations", "pair_dots", "layer_flops", "sweep_flops",
                 "layer_updates")


def lt_get_counters(ctx, clear=False):
    c = np.zeros(6, np.uint64)
    _check(_lib.lt_get_counters(ctx, _ptr(c), int(clear)), "lt_get_counters", ctx)
    return dict(zip(COUNTER_NAMES, (int(x) for x in c)))


def lt_measure_density_noalloc(precision, L, chi_max, n_traj, B_ptr, dims_ptr, density_ptr,
                               stream=None):
    """Device pointers in, densities written to density_ptr; returns the status."""
    return int(_lib.lt_measure_density_noalloc(precision, L, chi_max, n_traj, B_ptr, dims_ptr,
                                               density_ptr, stream))


def lt_pipe_peaks():
    """Measured SIMT peaks of the current device: dict(fp32_tflops, fp64_tflops,
    sm_clock_mhz, sms)."""
    out = np.zeros(4)
    _check(_lib.lt_pipe_peaks(_ptr(out)), "lt_pipe_peaks")
    return dict(fp32_tflops=float(out[0]), fp64_tflops=float(out[1]),
                sm_clock_mhz=float(out[2]), sms=int(out[3]))


def lt_launch_count(ctx):
    return int(_lib.lt_launch_count(ctx))


def lt_cluster_launches(ctx):
    return int(_lib.lt_cluster_launches(ctx))


def lt_stream(ctx):
    return _lib.lt_stream(ctx)


def lt_get_step(ctx):
    return int(_lib.lt_get_step(ctx))


# ---- packing helpers: list-of-tensors MPS <-> the library's padded layout ---------------
def pack_state(mps_list, L, chi, d=2):
    """mps_list: per trajectory (B list of (chi_l, d, chi_r), lam list, dims)."""
    n = len(mps_list)
    dims = np.zeros((n, L - 1), np.int32)
    lam = np.zeros((n, L - 1, chi))
    Bp = np.zeros((n, L, d * chi * chi), np.complex128)
    for t, (B, lm, dm) in enumerate(mps_list):
        dims[t] = dm
        for b in range(L - 1):
            lam[t, b, :len(lm[b])] = lm[b]
        for i in range(L):
            flat = np.asarray(B[i]).reshape(-1)
            Bp[t, i, :flat.size] = flat
    return dims, lam, Bp


def unpack_state(dims, lam, Bp, L, d=2):
    """Inverse of pack_state for one trajectory."""
    full = [1] + [int(x) for x in dims] + [1]
    B = [Bp[i, :full[i] * d * full[i + 1]].reshape(full[i], d, full[i + 1]) for i in range(L)]
    lm = [lam[b, :full[b + 1]] for b in range(L - 1)]
    return B, lm


class Ensemble:
    """Owner of one context: holds the handle and its sizes."""

    def __init__(self, L, chi_max, n_traj, **kw):
        self.L, self.chi, self.n_traj = L, chi_max, n_traj
        self.d = 4 if kw.get("method", LT_TRAJ) in (LT_MPDO, LT_PURIFIED) else 2
        self.ctx = lt_create(L, chi_max, n_traj, **kw)

    def close(self):
        if self.ctx is not None:
            lt_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lt_step(self.ctx, n)

    def step_graph(self, n=1):
        lt_step_graph(self.ctx, n)

    def apply_jumps(self, step, replay=None, want_channels=True):
        return lt_apply_jumps(self.ctx, step, replay, self.n_traj, want_channels)

    def apply_layer(self, parity, tau):
        lt_apply_layer(self.ctx, parity, tau)

    def apply_noise(self, step):
        lt_apply_noise(self.ctx, step)

    def apply_kraus(self):
        lt_apply_kraus(self.ctx)

    def log_weights(self):
        return lt_get_log_weights(self.ctx, self.n_traj)

    def density(self, per_traj=False):
        return lt_measure_density(self.ctx, self.L, self.n_traj, per_traj)

    def corr(self, per_traj=False):
        return lt_measure_corr(self.ctx, self.L, self.n_traj, per_traj)

    def stats(self):
        return lt_get_stats(self.ctx, self.L, self.n_traj)

    def set_state(self, traj0, mps_list):
        dims, lam, B = pack_state(mps_list, self.L, self.chi, self.d)
        lt_set_state(self.ctx, traj0, dims, lam, B)

    def get_state(self, traj0, n):
        return lt_get_state(self.ctx, traj0, n, self.L, self.chi, self.d)

    def launches(self):
        return lt_launch_count(self.ctx)

    def counters(self, clear=False):
        return lt_get_counters(self.ctx, clear)

    def sweep_histogram(self, clear=False):
        return lt_get_sweep_histogram(self.ctx, clear)


# ---- request server ------------------------------------------------------------------
def lt_context_bytes(L, chi_max, n_traj, num_sms, **kw):
    cfg, keep = make_config(L, chi_max, n_traj, **kw)
    out = np.zeros(1, np.uint64)
    _check(_lib.lt_context_bytes(ctypes.byref(cfg), num_sms, _ptr(out)), "lt_context_bytes")
    return int(out[0])


def lt_admit_plan(budget, used, max_active, n_active, queued_bytes):
    q = np.ascontiguousarray(queued_bytes, np.uint64)
    k = np.zeros(1, np.int32)
    _check(_lib.lt_admit_plan(budget, used, max_active, n_active, _ptr(q), len(q), _ptr(k)),
           "lt_admit_plan")
    return int(k[0])


class Server:
    """Continuous-batching request server (include/lindtebd.h, lt_server_*)."""

    def __init__(self, hbm_budget_bytes, max_active=64):
        h = ctypes.c_void_p()
        _check(_lib.lt_server_create(int(hbm_budget_bytes), max_active, ctypes.byref(h)),
               "lt_server_create")
        self.h = h
        self.L = {}

    def submit(self, n_steps, L, chi_max, n_traj, **kw):
        cfg, keep = make_config(L, chi_max, n_traj, **kw)
        rid = np.zeros(1, np.int64)
        _check(_lib.lt_server_submit(self.h, ctypes.byref(cfg), n_steps, _ptr(rid)),
               "lt_server_submit")
        self.L[int(rid[0])] = L
        return int(rid[0])

    def tick(self):
        c = np.zeros(3, np.int32)
        _check(_lib.lt_server_tick(self.h, _ptr(c[0:]), _ptr(c[1:]), _ptr(c[2:])), "lt_server_tick")
        return int(c[0]), int(c[1]), int(c[2])

    def result(self, rid):
        """(status, mean, sem, times) of a finished request; status LT_ERR_STATE while it runs."""
        L = self.L[rid]
        mean, sem, t = np.empty(L), np.empty(L), np.empty(3)
        st = _lib.lt_server_result(self.h, rid, _ptr(mean), _ptr(sem), _ptr(t))
        return st, mean, sem, t

    def error(self, rid):
        return _lib.lt_server_error(self.h, rid).decode()

    def updates(self, rid):
        """Two-site updates a request executed (so far, while it is active)."""
        u = np.zeros(1, np.uint64)
        _check(_lib.lt_server_updates(self.h, rid, _ptr(u)), "lt_server_updates")
        return int(u[0])

    def usage(self):
        u = np.zeros(2, np.uint64)
        _check(_lib.lt_server_usage(self.h, _ptr(u[0:]), _ptr(u[1:])), "lt_server_usage")
        return int(u[0]), int(u[1])

    def run(self, max_ticks=1_000_000):
        """Tick until nothing is queued or active; returns the tick count."""
        for n in range(max_ticks):
            q, a, _ = self.tick()
            if q == 0 and a == 0:
                return n + 1
        raise RuntimeError("server did not drain")

    def close(self):
        if self.h is not None:
            _lib.lt_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
