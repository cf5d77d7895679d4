"""GB300-native (sm_103a) IB-GM time step of Wiens & Stockie (arxiv 1305.3976).

Python binding of the C ABI in include/ib_gb300.h: the functions below carry
the C names and only marshal arguments; every step of the method runs in the
CUDA kernels of libibgb300.so.  There is no CPU fallback: if the library is
missing or cannot be built, the first call raises.

PyTorch is optional plumbing: torch CUDA tensors may be passed wherever the ABI
takes a device pointer, and by default a Grid works on torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

IB_OK, IB_ERR_ARG, IB_ERR_OOM, IB_ERR_CUDA, IB_ERR_NONFINITE, IB_ERR_TIMEOUT, IB_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
IB_FP32, IB_FP64 = 0, 1
IB_DELTA_PESKIN4, IB_DELTA_COS4 = 0, 1
IB_GM2, IB_GM1 = 0, 1
IB_FIELD_U, IB_FIELD_V, IB_FIELD_W, IB_FIELD_P, IB_FIELD_PSI, IB_FIELD_DIV = 1, 2, 4, 8, 16, 32
FIELD_BITS = ("u", "v", "w", "p", "psi", "div")

EXPORTS = ("ib_create_grid", "ib_add_fiber", "ib_set_velocity", "ib_step", "ib_read_fields", "ib_read_markers",
           "ib_set_markers", "ib_diagnostics", "ib_destroy_grid", "ib_error_string", "ib_last_error",
           "ib_cyclic_solve_lines", "ib_split_solve", "ib_split_solve_noalloc", "ib_profile_step",
           "ib_kernel_name", "ib_create_ensemble", "ib_ensemble_step", "ib_destroy_ensemble",
           "ib_sweep_config", "ib_fix_sweep_config", "ib_adjoint_run", "ib_selftest_wait_timeout",
           "ib_state_size", "ib_save_state", "ib_load_state", "ib_measure_peak", "ib_resort_markers",
           "ib_set_resort_interval")
IB_PEAK_FP64_FMA, IB_PEAK_FP32_FMA, IB_PEAK_L2_ATOMIC = 0, 1, 2


class ib_grid_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("H", C.c_double), ("rho", C.c_double),
                ("mu", C.c_double), ("dt", C.c_double), ("chi", C.c_double), ("precision", C.c_int),
                ("kernel", C.c_int), ("rotate_split", C.c_int), ("stream", C.c_void_p), ("scheme", C.c_int)]


class ib_diag(C.Structure):
    _fields_ = [("volume", C.c_double), ("div_l2", C.c_double), ("div_max", C.c_double),
                ("kinetic", C.c_double), ("elastic", C.c_double), ("step", C.c_int64)]


_lib = None


def library_path() -> str:
    return os.path.join(HERE, "libibgb300.so")


def lib():
    """Load libibgb300.so (building it with nvcc first if it is stale)."""
    global _lib
    if _lib is None:
        from . import _build
        path = _build.build()
        L = C.CDLL(path)
        vp, dp, ip, i64 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_int64
        L.ib_create_grid.argtypes = [C.POINTER(ib_grid_desc), C.POINTER(vp)]
        L.ib_add_fiber.argtypes = [vp, dp, i64, ip, dp, dp, i64, ip, i64, C.POINTER(C.c_int32)]
        L.ib_set_velocity.argtypes = [vp, C.c_int, vp, C.c_int]
        L.ib_step.argtypes = [vp, C.c_int]
        L.ib_read_fields.argtypes = [vp, C.c_uint, vp, C.c_size_t, C.c_int]
        L.ib_read_markers.argtypes = [vp, vp, i64, C.c_int]
        L.ib_set_markers.argtypes = [vp, vp, i64, C.c_int]
        L.ib_diagnostics.argtypes = [vp, C.POINTER(ib_diag)]
        L.ib_destroy_grid.argtypes = [vp]
        L.ib_error_string.argtypes = [C.c_int]
        L.ib_error_string.restype = C.c_char_p
        L.ib_last_error.argtypes = []
        L.ib_last_error.restype = C.c_char_p
        L.ib_cyclic_solve_lines.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_double, vp, vp, vp]
        L.ib_split_solve.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), dp, vp, vp, vp]
        L.ib_split_solve_noalloc.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), dp, vp, vp, vp]
        L.ib_profile_step.argtypes = [vp, C.c_int, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]
        L.ib_create_ensemble.argtypes = [C.POINTER(vp), C.c_int, vp, C.POINTER(vp)]
        L.ib_ensemble_step.argtypes = [vp, C.c_int]
        L.ib_destroy_ensemble.argtypes = [vp]
        L.ib_measure_peak.argtypes = [C.c_int, vp, dp]
        L.ib_resort_markers.argtypes = [vp]
        L.ib_set_resort_interval.argtypes = [vp, C.c_int]
        L.ib_sweep_config.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.ib_fix_sweep_config.argtypes = [vp, C.c_int, C.c_int]
        L.ib_adjoint_run.argtypes = [vp, C.c_int, C.c_int, dp, dp, dp]
        L.ib_selftest_wait_timeout.argtypes = [vp, C.POINTER(C.c_int)]
        L.ib_state_size.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.ib_save_state.argtypes = [vp, vp, C.c_size_t]
        L.ib_load_state.argtypes = [vp, vp, C.c_size_t]
        L.ib_kernel_name.argtypes = [C.c_int]
        L.ib_kernel_name.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("ib_error_string", "ib_last_error", "ib_kernel_name"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class IBError(RuntimeError):
    def __init__(self, code, where):
        L = lib()
        super().__init__(f"{where}: {L.ib_error_string(code).decode()} ({code}): {L.ib_last_error().decode()}")
        self.code = code


def _check(rc, where):
    if rc != IB_OK:
        raise IBError(rc, where)


# ---------------------------------------------------------------------------
# pointer helpers: numpy arrays are host memory, torch CUDA tensors device


def _is_torch_cuda(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x):
    if _is_torch_cuda(x) or (hasattr(x, "data_ptr") and hasattr(x, "is_cuda")):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), int(x.is_cuda)
    return C.c_void_p(x.ctypes.data), 0


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point


def ib_create_grid(dim, n, H=1.0, rho=1.0, mu=0.1, dt=1e-3, chi=0.6, precision=IB_FP32,
                   kernel=IB_DELTA_PESKIN4, rotate_split=1, stream="current", scheme=IB_GM2):
    d = ib_grid_desc()
    d.dim = dim
    n = [int(n)] * dim if np.isscalar(n) else list(n)
    n = n + [1] * (3 - len(n))
    d.n[0], d.n[1], d.n[2] = n
    d.H, d.rho, d.mu, d.dt, d.chi = H, rho, mu, dt, chi
    d.precision, d.kernel, d.rotate_split = precision, kernel, int(rotate_split)
    d.stream = _current_stream() if stream == "current" else stream
    d.scheme = scheme
    h = C.c_void_p()
    _check(lib().ib_create_grid(C.byref(d), C.byref(h)), "ib_create_grid")
    return h


def ib_add_fiber(g, X0, edges, kappa, rest_len=None, tris=None):
    """Arrays may be numpy (host) or contiguous torch CUDA tensors (device) of
    the C types: X0 float64 [n][dim], edges int32 [n_edges][2], kappa and
    rest_len float64 [n_edges], tris int32 [n_tris][3]."""
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)

    def arr(x, dtype, cols, ctype):
        if x is None:
            return None, 0
        if _is_torch_cuda(x):
            if not x.is_contiguous() or x.element_size() != np.dtype(dtype).itemsize:
                raise ValueError("device arrays must be contiguous tensors of the C type")
            return C.cast(C.c_void_p(x.data_ptr()), ctype), x.numel() // cols
        a = np.ascontiguousarray(x, dtype=dtype)
        keep.append(a)
        return a.ctypes.data_as(ctype), a.size // cols

    keep = []
    X0p, nm = arr(X0, np.float64, X0.shape[-1] if hasattr(X0, "shape") else 1, dp)
    ep, ne = arr(edges, np.int32, 2, ip)
    kp, _ = arr(kappa, np.float64, 1, dp)
    rp, _ = arr(rest_len, np.float64, 1, dp)
    tp, nt = arr(tris, np.int32, 3, ip)
    fid = C.c_int32()
    _check(lib().ib_add_fiber(g, X0p, nm, ep, kp, rp, ne, tp, nt, C.byref(fid)), "ib_add_fiber")
    return fid.value


def ib_set_velocity(g, comp, src):
    p, dev = _ptr(src)
    _check(lib().ib_set_velocity(g, comp, p, dev), "ib_set_velocity")


def ib_step(g, n_steps=1):
    _check(lib().ib_step(g, int(n_steps)), "ib_step")


def ib_read_fields(g, field_mask, dst):
    p, dev = _ptr(dst)
    nbytes = dst.numel() * dst.element_size() if dev else dst.nbytes
    _check(lib().ib_read_fields(g, field_mask, p, nbytes, dev), "ib_read_fields")
    return dst


def ib_read_markers(g, dst):
    p, dev = _ptr(dst)
    n = dst.shape[0]
    _check(lib().ib_read_markers(g, p, n, dev), "ib_read_markers")
    return dst


def ib_set_markers(g, src):
    p, dev = _ptr(src)
    _check(lib().ib_set_markers(g, p, src.shape[0], dev), "ib_set_markers")


def ib_diagnostics(g, check=True):
    d = ib_diag()
    rc = lib().ib_diagnostics(g, C.byref(d))
    if check:
        _check(rc, "ib_diagnostics")
    return {k: getattr(d, k) for k, _ in ib_diag._fields_}, rc


def ib_resort_markers(g):
    _check(lib().ib_resort_markers(g), "ib_resort_markers")


def ib_set_resort_interval(g, every):
    _check(lib().ib_set_resort_interval(g, int(every)), "ib_set_resort_interval")


def ib_measure_peak(kind, stream="current"):
    """Throughput of one of the GPU's units (IB_PEAK_*): FLOP/s or atomic
    updates/s."""
    v = C.c_double()
    st = _current_stream() if stream == "current" else stream
    _check(lib().ib_measure_peak(int(kind), st, C.byref(v)), "ib_measure_peak")
    return v.value


def ib_destroy_grid(g):
    _check(lib().ib_destroy_grid(g), "ib_destroy_grid")


def ib_save_state(g):
    """The grid's state S^n as a bytes object (see include/ib_gb300.h)."""
    n = C.c_size_t()
    _check(lib().ib_state_size(g, C.byref(n)), "ib_state_size")
    buf = (C.c_char * n.value)()
    _check(lib().ib_save_state(g, buf, n.value), "ib_save_state")
    return bytes(buf)


def ib_load_state(g, image):
    buf = C.create_string_buffer(bytes(image), len(image))
    _check(lib().ib_load_state(g, buf, len(image)), "ib_load_state")


def ib_selftest_wait_timeout(stream="current"):
    """1 if a device wait that cannot complete ran out and was reported."""
    flag = C.c_int(-1)
    s = _current_stream() if stream == "current" else stream
    _check(lib().ib_selftest_wait_timeout(C.c_void_p(s), C.byref(flag)), "ib_selftest_wait_timeout")
    return flag.value


def ib_adjoint_run(g, n_steps, checkpoint_every, X_target, n_edges):
    """Returns (loss, dkappa[n_edges]); X_target is [n_markers][dim] FP64."""
    T = np.ascontiguousarray(X_target, dtype=np.float64)
    loss = C.c_double()
    dk = np.zeros(int(n_edges), dtype=np.float64)
    dp = C.POINTER(C.c_double)
    _check(lib().ib_adjoint_run(g, int(n_steps), int(checkpoint_every), T.ctypes.data_as(dp), C.byref(loss),
                                dk.ctypes.data_as(dp)), "ib_adjoint_run")
    return loss.value, dk


def ib_cyclic_solve_lines(precision, dim, n, axis, r, src, dst, stream="current"):
    na = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    s = _current_stream() if stream == "current" else stream
    _check(lib().ib_cyclic_solve_lines(precision, dim, na, axis, float(r), _ptr(src)[0], _ptr(dst)[0],
                                       C.c_void_p(s)), "ib_cyclic_solve_lines")


def ib_split_solve(precision, dim, n, r, f, psi, stream="current"):
    na = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    ra = (C.c_double * 3)(*(list(r) + [0.0] * (3 - len(r))))
    s = _current_stream() if stream == "current" else stream
    _check(lib().ib_split_solve(precision, dim, na, ra, _ptr(f)[0], _ptr(psi)[0], C.c_void_p(s)), "ib_split_solve")


def ib_split_solve_noalloc(precision, dim, n, r, f, psi, stream="current"):
    """ib_split_solve without any device allocation (fixed scratch inside the
    library, lines up to IB_NOALLOC_MAX_N = 512)."""
    na = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    ra = (C.c_double * 3)(*(list(r) + [0.0] * (3 - len(r))))
    s = _current_stream() if stream == "current" else stream
    _check(lib().ib_split_solve_noalloc(precision, dim, na, ra, _ptr(f)[0], _ptr(psi)[0], C.c_void_p(s)),
           "ib_split_solve_noalloc")


def ib_sweep_config(g, axis):
    cfg = (C.c_int * 4)()
    _check(lib().ib_sweep_config(g, axis, cfg), "ib_sweep_config")
    return tuple(cfg)


def ib_fix_sweep_config(g, axis, cfg_id):
    _check(lib().ib_fix_sweep_config(g, int(axis), int(cfg_id)), "ib_fix_sweep_config")


def ib_profile_step(g, n_steps):
    ms = (C.c_float * 16)()
    nk = C.c_int()
    _check(lib().ib_profile_step(g, int(n_steps), ms, 16, C.byref(nk)), "ib_profile_step")
    return {lib().ib_kernel_name(i).decode(): float(ms[i]) for i in range(nk.value)}


def ib_create_ensemble(members, stream="current"):
    arr = (C.c_void_p * len(members))(*[m.value if isinstance(m, C.c_void_p) else m for m in members])
    h = C.c_void_p()
    st = _current_stream() if stream == "current" else stream
    _check(lib().ib_create_ensemble(arr, len(members), C.c_void_p(st), C.byref(h)), "ib_create_ensemble")
    return h


def ib_ensemble_step(e, n_steps=1):
    _check(lib().ib_ensemble_step(e, int(n_steps)), "ib_ensemble_step")


def ib_destroy_ensemble(e):
    _check(lib().ib_destroy_ensemble(e), "ib_destroy_ensemble")


# ---------------------------------------------------------------------------
# convenience wrapper


class Grid:
    """An ib_grid_t with numpy/torch conveniences (argument marshalling only)."""

    def __init__(self, dim, n, H=1.0, rho=1.0, mu=0.1, dt=1e-3, chi=0.6, precision="fp32",
                 kernel="peskin4", rotate_split=True, stream="current", scheme="gm2"):
        self.dim = dim
        self.n = [int(n)] * dim if np.isscalar(n) else list(n)[:dim]
        self.precision = IB_FP32 if precision in ("fp32", IB_FP32) else IB_FP64
        self.dtype = np.float32 if self.precision == IB_FP32 else np.float64
        k = {"peskin4": IB_DELTA_PESKIN4, "cos4": IB_DELTA_COS4}.get(kernel, kernel)
        s = {"gm2": IB_GM2, "gm1": IB_GM1}.get(scheme, scheme)
        self.h = ib_create_grid(dim, self.n, H, rho, mu, dt, chi, self.precision, k, rotate_split, stream, s)
        self.n_markers = 0
        self.n_edges = 0

    @property
    def field_shape(self):
        return tuple(reversed(self.n))

    def add_fiber(self, X, edges, kappa, rest=None, tris=None):
        fid = ib_add_fiber(self.h, X, edges, kappa, rest, tris)
        self.n_markers += len(X)
        self.n_edges += (edges if hasattr(edges, "reshape") else np.asarray(edges)).reshape(-1, 2).shape[0]
        return fid

    def set_velocity(self, u):
        for c in range(self.dim):
            src = u[c]
            if not _is_torch_cuda(src):
                src = np.ascontiguousarray(src, dtype=self.dtype)
            ib_set_velocity(self.h, c, src)

    def step(self, n=1):
        ib_step(self.h, n)

    def fields(self, names=FIELD_BITS):
        """Host copies of the named fields ('u', 'v', 'w', 'p', 'psi', 'div')."""
        out = {}
        for name in names:
            b = FIELD_BITS.index(name)
            if b == 2 and self.dim == 2:
                continue
            arr = np.empty(self.field_shape, dtype=self.dtype)
            ib_read_fields(self.h, 1 << b, arr)
            out[name] = arr
        return out

    def velocity(self):
        f = self.fields(("u", "v", "w")[:self.dim])
        return np.stack([f[k] for k in ("u", "v", "w")[:self.dim]])

    def markers(self):
        X = np.empty((self.n_markers, self.dim), dtype=np.float64)
        return ib_read_markers(self.h, X)

    def set_markers(self, X):
        ib_set_markers(self.h, np.ascontiguousarray(X, dtype=np.float64))

    def diagnostics(self, check=True):
        return ib_diagnostics(self.h, check)[0]

    def profile(self, n_steps=1):
        return ib_profile_step(self.h, n_steps)

    def adjoint(self, n_steps, X_target, checkpoint_every=20):
        """Advance n_steps; return (sum |X - X_target|^2, d loss / d kappa per connection)."""
        return ib_adjoint_run(self.h, n_steps, checkpoint_every, X_target, self.n_edges)

    def resort_markers(self):
        """Re-number the markers internally by their current positions."""
        ib_resort_markers(self.h)

    def set_resort_interval(self, every):
        ib_set_resort_interval(self.h, every)

    def save_state(self):
        return ib_save_state(self.h)

    def load_state(self, image):
        ib_load_state(self.h, image)

    def sweep_configs(self):
        """Autotuned line-solve configuration per axis: (id, a, b, c)."""
        return [ib_sweep_config(self.h, a) for a in range(self.dim)]

    def fix_sweep_configs(self, ids):
        """Use these configuration ids (one per axis) instead of timing candidates."""
        for a, i in enumerate(ids):
            ib_fix_sweep_config(self.h, a, i)

    def close(self):
        if self.h:
            ib_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Independent Grids advanced together (one CUDA graph launch per step)."""

    def __init__(self, grids, stream="current"):
        self.grids = list(grids)
        self.h = ib_create_ensemble([g.h for g in self.grids], stream)

    def step(self, n=1):
        ib_ensemble_step(self.h, n)

    def close(self):
        if self.h:
            ib_destroy_ensemble(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_KAPPA_LOSS = None


def kappa_loss(kappa, build, n_steps, X_target, checkpoint_every=20):
    """Differentiable loss(kappa) = sum_k |X_k^{n_steps} - X_target_k|^2 for
    torch.autograd: `kappa` is a tensor of connection stiffnesses, `build`
    maps a numpy copy of it to a fresh Grid with its fibers added.  One call of
    ib_adjoint_run gives the loss and its gradient; backward returns
    grad_output * dkappa."""
    global _KAPPA_LOSS
    import torch

    if _KAPPA_LOSS is None:
        class _KappaLoss(torch.autograd.Function):
            @staticmethod
            def forward(ctx, kap, build_fn, steps, target, ck):
                g = build_fn(kap.detach().cpu().numpy().astype(np.float64))
                try:
                    loss, dk = g.adjoint(steps, target, ck)
                finally:
                    g.close()
                ctx.save_for_backward(torch.from_numpy(dk).to(dtype=kap.dtype, device=kap.device))
                return kap.new_tensor(loss)

            @staticmethod
            def backward(ctx, grad_out):
                (dk,) = ctx.saved_tensors
                return grad_out * dk, None, None, None, None

        _KAPPA_LOSS = _KappaLoss
    return _KAPPA_LOSS.apply(kappa, build, n_steps, X_target, checkpoint_every)
