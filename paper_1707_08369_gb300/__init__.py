"""GB300 rank-one SVD update (Gandhi & Rajgor, arXiv 1707.08369, Alg. 6.1).

Thin Python binding over the C ABI in include/svdup.h (libsvdup.so): it only
marshals arguments.  Every step of the update runs in the library's CUDA
kernels; PyTorch is used for device memory and streams.  There is no CPU
fallback: if the shared library is missing or fails to load, every call raises.

Names follow the C ABI: create / destroy / sync / update / update_host /
rank_one_eig / secular / secular_static / cauchy_product / batch_create (batch_plan) /
batch_launch / update_batched / autotune / tuning / error_string / launch_count.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvdup.so")

OK, EINVAL, ENOMEM, ENOCONV, ENONFINITE, ECUDA, EORDER, ETIMEOUT = 0, 1, 2, 3, 4, 5, 6, 7
FP64, MIXED_BF16X3, MIXED_FP16X2 = 0, 1, 2  # update modes (split BF16 x3, scaled FP16 x2)
DENSE, REFINE = 0x100, 0x200                 # flags: dense product; gated refinement
TIMING_STAGES, TIMING_KERNELS = 1, 2      # svdup_timing modes

_lib = None


class SvdupError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (code %d)" % (where, error_string(code) if _lib else "?", code))


def load(path: str = LIB_PATH):
    """Load libsvdup.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsvdup.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.svdup_create.argtypes = [ctypes.POINTER(P), I, P, ctypes.c_uint]
    lib.svdup_destroy.argtypes = [P]
    lib.svdup_sync.argtypes = [P]
    lib.svdup_error_string.argtypes = [I]
    lib.svdup_error_string.restype = ctypes.c_char_p
    lib.svdup_launch_count.argtypes = [P]
    lib.svdup_launch_count.restype = ctypes.c_longlong
    lib.svdup_timing.argtypes = [P, I]
    lib.svdup_timing_read.argtypes = [P, P, P, P, P, I]
    lib.svdup_timing_read_alg.argtypes = [P, P, I]
    lib.svdup_update.argtypes = [P, I, I, P, I, P, P, I, P, P, D, I]
    lib.svdup_update_host.argtypes = [P, I, I, P, I, P, P, I, P, P, D, I]
    lib.svdup_rank_one_eig.argtypes = [P, I, P, P, D, P, P, P, P, P, P, P, P]
    lib.svdup_secular.argtypes = [P, I, P, P, D, P, P]
    lib.svdup_cauchy_product.argtypes = [P, I, I, P, I, P, P, D, P, I, P, D, I]
    lib.svdup_secular_static.argtypes = [P, I, P, P, D, P, P, P]
    lib.svdup_refine.argtypes = [P, I, I, P, I, D, P]
    lib.svdup_check_rcp.argtypes = [P, I, P, P, P]
    lib.svdup_check_timeout.argtypes = [P, I, I, P, I, P, P, D, P, I, P]
    lib.svdup_set_refine_tol.argtypes = [P, D]
    lib.svdup_refine_residuals.argtypes = [P, P]
    lib.svdup_batch_create.argtypes = [P, I, P, D, I, I, ctypes.POINTER(P)]
    lib.svdup_batch_launch.argtypes = [P]
    lib.svdup_batch_kernels.argtypes = [P]
    lib.svdup_batch_kernels.restype = ctypes.c_longlong
    lib.svdup_batch_destroy.argtypes = [P]
    lib.svdup_update_batched.argtypes = [P, I, P, D, I, I]
    lib.svdup_autotune.argtypes = [P, I, I]
    lib.svdup_tuning_get.argtypes = [P, I, P, P]
    lib.svdup_tuning_set.argtypes = [P, I, I, I]
    lib.svdup_tuning_get_tile.argtypes = [P, I, P]
    lib.svdup_tuning_set_tile.argtypes = [P, I, I]
    lib.svdup_set_far_sums.argtypes = [P, I, I]
    lib.svdup_rank_one_apply.argtypes = [P, I, P, P, D, P, P, P]
    S_T = ctypes.c_size_t
    lib.svdup_update_workspace.argtypes = [P, I, I, D, I, ctypes.POINTER(S_T)]
    lib.svdup_server_create.argtypes = [I, I, S_T, D, I, ctypes.POINTER(P)]
    lib.svdup_server_register.argtypes = [P, I, I, P, I, P, P, I, ctypes.POINTER(I)]
    lib.svdup_server_submit.argtypes = [P, I, P, P, ctypes.POINTER(ctypes.c_longlong)]
    lib.svdup_server_wait.argtypes = [P, ctypes.c_longlong, D, ctypes.POINTER(D)]
    lib.svdup_server_drain.argtypes = [P]
    lib.svdup_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D),
                                       ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(S_T)]
    lib.svdup_server_destroy.argtypes = [P]
    lib.svdup_server_set_group.argtypes = [P, I]
    lib.svdup_server_group_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I)]
    _lib = lib
    return lib


class Problem(ctypes.Structure):
    """svdup_problem: the arguments of svdup_update for one member of a batch."""
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("U", ctypes.c_void_p),
                ("ldu", ctypes.c_int), ("S", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("ldv", ctypes.c_int), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p)]


def _problems(items):
    """ctypes array of Problem from (U, S, V, a, b) device-tensor tuples."""
    arr = (Problem * len(items))()
    for i, (U, S, V, a, b) in enumerate(items):
        m, n = S.numel(), b.numel()
        for t, nm in ((U, "U"), (S, "S"), (V, "V"), (a, "a"), (b, "b")):
            _dev_f64(t, nm)
        arr[i] = Problem(m, n, U.data_ptr(), _colmajor_ld(U, m, m, "U"), S.data_ptr(), V.data_ptr(),
                         _colmajor_ld(V, n, n, "V"), a.data_ptr(), b.data_ptr())
    return arr


def error_string(code: int) -> str:
    return load().svdup_error_string(int(code)).decode()


def _check(code: int, where: str):
    if code != OK:
        raise SvdupError(code, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev_f64(t, name, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("%s must be a float64 CUDA tensor" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements" % (name, numel))
    return t


def _colmajor_ld(t, rows, cols, name):
    """Leading dimension of a column-major (Fortran-ordered) 2-D tensor."""
    if t.dim() != 2 or t.shape[0] != rows or t.shape[1] != cols:
        raise ValueError("%s must be %d x %d" % (name, rows, cols))
    if t.stride(0) != 1:
        raise ValueError("%s must be column-major (stride(0) == 1)" % name)
    return max(t.stride(1), rows)


class Handle:
    """A library handle bound to a device and a CUDA stream (torch's current stream
    by default)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.device = device
        h = ctypes.c_void_p()
        _check(lib.svdup_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream.cuda_stream), 0),
               "svdup_create")
        self._h = h

    def close(self):
        if self._h:
            load().svdup_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self) -> int:
        return int(load().svdup_sync(self._h))

    def launch_count(self) -> int:
        return int(load().svdup_launch_count(self._h))

    STAGES = ("gemv", "solve", "sign", "gather", "setup", "p2m", "m2l", "out")

    def timing(self, enable=True):
        """Timer mode: True / TIMING_STAGES (every stage, one stream), TIMING_KERNELS (the
        product-stage kernels on their own streams, schedule unchanged), False / 0 off."""
        mode = TIMING_STAGES if enable is True else int(enable)
        _check(load().svdup_timing(self._h, mode), "svdup_timing")

    def timing_read_alg(self):
        """{stage: algorithmic flops (App. D's operation count)} since timing was enabled."""
        n = len(self.STAGES)
        fl = (ctypes.c_double * n)()
        _check(load().svdup_timing_read_alg(self._h, fl, n), "svdup_timing_read_alg")
        return {s: fl[i] for i, s in enumerate(self.STAGES)}

    def timing_read(self):
        """{stage: (ms, intervals, useful flops, executed tensor-core flops)} since
        timing was enabled."""
        n = len(self.STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        fl = (ctypes.c_double * n)()
        mfl = (ctypes.c_double * n)()
        _check(load().svdup_timing_read(self._h, ms, cnt, fl, mfl, n), "svdup_timing_read")
        return {s: (ms[i], cnt[i], fl[i], mfl[i]) for i, s in enumerate(self.STAGES)}

    def update(self, U, S, V, a, b, eps: float = 1e-12, mode: int = FP64, check: bool = True):
        """In-place Alg. 6.1 on device tensors: U (m x m) and V (n x n) column-major
        float64, S (m, descending), a (m), b (n).  Queues the work; with check=True
        waits and raises on a device error."""
        m, n = S.numel(), b.numel()
        for t, nm in ((U, "U"), (S, "S"), (V, "V"), (a, "a"), (b, "b")):
            _dev_f64(t, nm)
        ldu = _colmajor_ld(U, m, m, "U")
        ldv = _colmajor_ld(V, n, n, "V")
        _check(load().svdup_update(self._h, m, n, _ptr(U), ldu, _ptr(S), _ptr(V), ldv, _ptr(a),
                                   _ptr(b), float(eps), int(mode)), "svdup_update")
        if check:
            _check(self.sync(), "svdup_update (device)")

    def update_host(self, U, S, V, a, b, eps: float = 1e-12, mode: int = FP64):
        """The same update on host numpy arrays (copied in and out inside the call)."""
        import numpy as np
        for t, nm in ((U, "U"), (S, "S"), (V, "V"), (a, "a"), (b, "b")):
            if not isinstance(t, np.ndarray) or t.dtype != np.float64:
                raise TypeError("%s must be a float64 numpy array" % nm)
        if not (U.flags.f_contiguous and V.flags.f_contiguous):
            raise ValueError("U and V must be column-major (Fortran order)")
        m, n = S.size, b.size
        p = lambda x: ctypes.c_void_p(x.ctypes.data)
        _check(load().svdup_update_host(self._h, m, n, p(U), m, p(S), p(V), n, p(a), p(b),
                                        float(eps), int(mode)), "svdup_update_host")

    def batch_plan(self, items, eps: float = 1e-12, mode: int = FP64, lanes: int = 0):
        """Record a batch of independent updates (a list of (U, S, V, a, b) device
        tensors, as in update) into a CUDA graph; returns a Batch to launch."""
        arr = _problems(items)
        out = ctypes.c_void_p()
        _check(load().svdup_batch_create(self._h, len(items), arr, float(eps), int(mode), int(lanes),
                                         ctypes.byref(out)), "svdup_batch_create")
        return Batch(self, out, items)

    def update_batched(self, items, eps: float = 1e-12, mode: int = FP64, lanes: int = 0):
        """The same batch without a graph; waits and raises on any error."""
        arr = _problems(items)
        _check(load().svdup_update_batched(self._h, len(items), arr, float(eps), int(mode), int(lanes)),
               "svdup_update_batched")

    def update_workspace(self, m: int, n: int, eps: float = 1e-12, mode: int = FP64) -> int:
        """Workspace bytes svdup_update needs for an m x n problem."""
        v = ctypes.c_size_t()
        _check(load().svdup_update_workspace(self._h, int(m), int(n), float(eps), int(mode),
                                             ctypes.byref(v)), "svdup_update_workspace")
        return v.value

    def autotune(self, mode: int = FP64, nmax: int = 4096):
        """Measure the product-path choices for `mode`; returns (dense_max, leaf128_min)."""
        _check(load().svdup_autotune(self._h, int(mode), int(nmax)), "svdup_autotune")
        return self.tuning(mode)

    def tuning(self, mode: int = FP64):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().svdup_tuning_get(self._h, int(mode), ctypes.byref(a), ctypes.byref(b)),
               "svdup_tuning_get")
        return a.value, b.value

    def tile_tuning(self, mode: int = FP64) -> int:
        """Smallest N at which the mixed dense product uses 128-column output tiles."""
        a = ctypes.c_int()
        _check(load().svdup_tuning_get_tile(self._h, int(mode), ctypes.byref(a)),
               "svdup_tuning_get_tile")
        return a.value

    def set_tile_tuning(self, mode: int, dense_tile128_min: int):
        _check(load().svdup_tuning_set_tile(self._h, int(mode), int(dense_tile128_min)),
               "svdup_tuning_set_tile")

    def set_far_sums(self, kmin: int, kmin_pairs: int = None):
        kp = kmin if kmin_pairs is None else kmin_pairs
        _check(load().svdup_set_far_sums(self._h, int(kmin), int(kp)), "svdup_set_far_sums")

    def set_tuning(self, mode: int, dense_max: int, leaf128_min: int):
        _check(load().svdup_tuning_set(self._h, int(mode), int(dense_max), int(leaf128_min)),
               "svdup_tuning_set")

    def rank_one_eig(self, d, z, rho: float):
        """Compact eigen-system of diag(d) + rho z z^T (device tensors).  Returns a dict
        with k, idx, dk, org, tau, zhat, inv_norm (first k valid) and lam (all N)."""
        import torch
        N = d.numel()
        _dev_f64(d, "d"); _dev_f64(z, "z", N)
        dev = d.device
        out = dict(k=torch.zeros(1, dtype=torch.int32, device=dev),
                   idx=torch.zeros(N, dtype=torch.int32, device=dev),
                   dk=torch.zeros(N, dtype=torch.float64, device=dev),
                   org=torch.zeros(N, dtype=torch.int32, device=dev),
                   tau=torch.zeros(N, dtype=torch.float64, device=dev),
                   zhat=torch.zeros(N, dtype=torch.float64, device=dev),
                   inv_norm=torch.zeros(N, dtype=torch.float64, device=dev),
                   lam=torch.zeros(N, dtype=torch.float64, device=dev))
        _check(load().svdup_rank_one_eig(self._h, N, _ptr(d), _ptr(z), float(rho), _ptr(out["k"]),
                                         _ptr(out["idx"]), _ptr(out["dk"]), _ptr(out["org"]),
                                         _ptr(out["tau"]), _ptr(out["zhat"]), _ptr(out["inv_norm"]),
                                         _ptr(out["lam"])), "svdup_rank_one_eig")
        _check(self.sync(), "svdup_rank_one_eig (device)")
        return out

    def rank_one_apply(self, d, z, rho: float, x):
        """y = Q x for the eigenvectors Q of diag(d) + rho z z^T (device tensors; x in
        the order of the ascending eigenvalues, y in the order of d).  Returns (y, lam)."""
        import torch
        N = d.numel()
        _dev_f64(d, "d"); _dev_f64(z, "z", N); _dev_f64(x, "x", N)
        y = torch.zeros(N, dtype=torch.float64, device=d.device)
        lam = torch.zeros(N, dtype=torch.float64, device=d.device)
        _check(load().svdup_rank_one_apply(self._h, N, _ptr(d), _ptr(z), float(rho), _ptr(x),
                                           _ptr(y), _ptr(lam)), "svdup_rank_one_apply")
        _check(self.sync(), "svdup_rank_one_apply (device)")
        return y, lam

    def secular(self, d, z, rho: float):
        """Roots of the secular equation for strictly ascending d and nonzero z."""
        import torch
        k = d.numel()
        _dev_f64(d, "d"); _dev_f64(z, "z", k)
        org = torch.zeros(k, dtype=torch.int32, device=d.device)
        tau = torch.zeros(k, dtype=torch.float64, device=d.device)
        _check(load().svdup_secular(self._h, k, _ptr(d), _ptr(z), float(rho), _ptr(org), _ptr(tau)),
               "svdup_secular")
        _check(self.sync(), "svdup_secular (device)")
        return org, tau

    def refine(self, X, tol: float = 0.0):
        """One gated Newton-Schulz step on X (device, rows x cols column-major) in place;
        returns the probe residual measured before the step (0-d device tensor)."""
        import torch
        rows, cols = X.shape
        _dev_f64(X, "X")
        ldx = _colmajor_ld(X, rows, cols, "X")
        res = torch.zeros((), dtype=torch.float64, device=X.device)
        _check(load().svdup_refine(self._h, rows, cols, _ptr(X), ldx, float(tol), _ptr(res)),
               "svdup_refine")
        _check(self.sync(), "svdup_refine (device)")
        return res

    def set_refine_tol(self, tol: float):
        _check(load().svdup_set_refine_tol(self._h, float(tol)), "svdup_set_refine_tol")

    def refine_residuals(self):
        """Probe residuals of Uhat and Vhat measured by the last REFINE update."""
        out = (ctypes.c_double * 2)()
        _check(load().svdup_refine_residuals(self._h, out), "svdup_refine_residuals")
        return out[0], out[1]

    def cauchy_product(self, X, d, z, rho: float, eps: float = 1e-12, mode: int = FP64):
        """Y = X Q for diag(d) + rho z z^T = Q diag(lam) Q^T; returns (lam, Y)."""
        import torch
        rows, N = X.shape
        _dev_f64(X, "X"); _dev_f64(d, "d", N); _dev_f64(z, "z", N)
        ldx = _colmajor_ld(X, rows, N, "X")
        Y = torch.zeros((N, rows), dtype=torch.float64, device=X.device).t()
        lam = torch.zeros(N, dtype=torch.float64, device=X.device)
        _check(load().svdup_cauchy_product(self._h, rows, N, _ptr(X), ldx, _ptr(d), _ptr(z),
                                           float(rho), _ptr(Y), rows, _ptr(lam), float(eps),
                                           int(mode)), "svdup_cauchy_product")
        _check(self.sync(), "svdup_cauchy_product (device)")
        return lam, Y


class Batch:
    """A planned batch (svdup_batch_t): launch() queues one graph launch on the
    handle's stream; the problems' tensors must stay alive while it exists."""

    def __init__(self, handle, ptr, items):
        self.handle = handle
        self._b = ptr
        self._items = items

    def launch(self, check: bool = True):
        _check(load().svdup_batch_launch(self._b), "svdup_batch_launch")
        if check:
            _check(self.handle.sync(), "svdup_batch_launch (device)")

    def kernels(self) -> int:
        return int(load().svdup_batch_kernels(self._b))

    def close(self):
        if self._b:
            load().svdup_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving engine (svdup_server_*): register resident SVDs (device tensors as
    in Handle.update, kept alive by this object), submit updates with host vectors,
    wait for tickets, read latency statistics."""

    def __init__(self, device: int = 0, lanes: int = 8, hbm_budget: int = 0, eps: float = 1e-12,
                 mode: int = FP64):
        out = ctypes.c_void_p()
        _check(load().svdup_server_create(int(device), int(lanes), int(hbm_budget), float(eps),
                                          int(mode), ctypes.byref(out)), "svdup_server_create")
        self._s = out
        self._mats = []

    def register(self, U, S, V) -> int:
        m, n = S.numel(), V.shape[0]
        for t, nm in ((U, "U"), (S, "S"), (V, "V")):
            _dev_f64(t, nm)
        mid = ctypes.c_int()
        _check(load().svdup_server_register(self._s, m, n, _ptr(U), _colmajor_ld(U, m, m, "U"),
                                            _ptr(S), _ptr(V), _colmajor_ld(V, n, n, "V"),
                                            ctypes.byref(mid)), "svdup_server_register")
        self._mats.append((U, S, V))
        return mid.value

    def submit(self, mid: int, a, b) -> int:
        import numpy as np
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        t = ctypes.c_longlong()
        _check(load().svdup_server_submit(self._s, int(mid), ctypes.c_void_p(a.ctypes.data),
                                          ctypes.c_void_p(b.ctypes.data), ctypes.byref(t)),
               "svdup_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        """(status, latency_ms) of a request."""
        lat = ctypes.c_double()
        st = load().svdup_server_wait(self._s, int(ticket), float(timeout_ms), ctypes.byref(lat))
        return int(st), lat.value

    def drain(self):
        _check(load().svdup_server_drain(self._s), "svdup_server_drain")

    def stats(self):
        c, p50, p99 = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        mif, mws = ctypes.c_int(), ctypes.c_size_t()
        _check(load().svdup_server_stats(self._s, ctypes.byref(c), ctypes.byref(p50), ctypes.byref(p99),
                                         ctypes.byref(mif), ctypes.byref(mws)), "svdup_server_stats")
        return {"completed": c.value, "p50_ms": p50.value, "p99_ms": p99.value,
                "max_in_flight": mif.value, "max_ws_bytes": mws.value}

    def set_group(self, group_max: int):
        """Requests of one size class a lane takes per cycle (1..16)."""
        _check(load().svdup_server_set_group(self._s, int(group_max)), "svdup_server_set_group")

    def group_stats(self):
        g, r, m = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        _check(load().svdup_server_group_stats(self._s, ctypes.byref(g), ctypes.byref(r),
                                               ctypes.byref(m)), "svdup_server_group_stats")
        return {"groups": g.value, "grouped": r.value, "max_group": m.value}

    def close(self):
        if self._s:
            load().svdup_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SECULAR_STATIC_MAX_K = 16384


def secular_static(d, z, rho: float, stream=None):
    """Secular roots through svdup_secular_static, the entry point that allocates no
    device memory (its scratch is a fixed array inside the library; at most
    SECULAR_STATIC_MAX_K roots).  Queued on `stream` (torch's current stream by
    default) of d's device; returns (org, tau, info) device tensors without waiting,
    info holding the device status once the stream has run."""
    import torch
    k = d.numel()
    _dev_f64(d, "d"); _dev_f64(z, "z", k)
    if stream is None:
        stream = torch.cuda.current_stream(d.device)
    org = torch.empty(k, dtype=torch.int32, device=d.device)
    tau = torch.empty(k, dtype=torch.float64, device=d.device)
    info = torch.empty(1, dtype=torch.int32, device=d.device)
    with torch.cuda.device(d.device):
        _check(load().svdup_secular_static(ctypes.c_void_p(stream.cuda_stream), k, _ptr(d), _ptr(z),
                                           float(rho), _ptr(org), _ptr(tau), _ptr(info)),
               "svdup_secular_static")
    return org, tau, info


def colmajor(t):
    """A column-major copy of a 2-D tensor (what the library expects for matrices)."""
    return t.t().contiguous().t()
