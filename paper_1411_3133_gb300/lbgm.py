"""Python binding of liblbgm.so (include/lbgm.h): argument marshalling only.

Every function of the C ABI is exposed under its own name; ``LBContext`` is a
small convenience wrapper that owns an ``lb_ctx``. PyTorch supplies the CUDA
stream and, through ``torch.cuda.caching_allocator_alloc``, the device memory.
All numerical work happens in the library's CUDA kernels; there is no fallback:
a missing or unloadable library raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbgm.so")

LB_Q = 41
LB_GEO_STRIDE = 44

LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_NONFINITE, LB_ERR_TIMEOUT, LB_ERR_STATE = range(6)
STATUS_NAMES = {0: "LB_OK", 1: "LB_ERR_ARG", 2: "LB_ERR_CUDA", 3: "LB_ERR_NONFINITE",
                4: "LB_ERR_TIMEOUT", 5: "LB_ERR_STATE"}
METRICS = {"flat": 0, "cylindrical": 1, "ellipsoidal": 2, "ellipsoidal_theta": 3}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16_shifted": 2, "bf16_shifted": 3}
LB_OPT_CHECK_EVERY, LB_OPT_BLOCK_THREADS, LB_OPT_USE_GRAPH, LB_OPT_STEP_KERNEL = 0, 1, 2, 3
LB_OPT_SCHEDULE, LB_OPT_TILE_BLOCKS, LB_OPT_STORAGE_REFERENCE = 4, 5, 6


class lb_geometry_desc(ctypes.Structure):
    _fields_ = [("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double),
                ("b", ctypes.c_double), ("nr", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("n3", ctypes.c_int), ("periodic3", ctypes.c_int),
                ("dtheta_scale", ctypes.c_double), ("d3_scale", ctypes.c_double),
                ("wall", ctypes.c_int)]


class lb_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("force_G", ctypes.c_double),
                ("old_forcing", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("noise_amp", ctypes.c_double), ("init_base_flow", ctypes.c_int)]


class lb_diag(ctypes.Structure):
    _fields_ = [("mass_rho_prime", ctypes.c_double), ("mass_physical", ctypes.c_double),
                ("mean_v_theta", ctypes.c_double), ("dean", ctypes.c_double),
                ("mean_vorticity", ctypes.c_double), ("vortex_amp", ctypes.c_double),
                ("vortex_amp_x3", ctypes.c_double), ("max_speed", ctypes.c_double),
                ("nonfinite", ctypes.c_longlong), ("step", ctypes.c_longlong)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class lb_tune(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("schedule", ctypes.c_int),
                ("tile_nodes", ctypes.c_int), ("ms_per_step", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class lb_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


# C signatures: name -> (restype, argtypes)
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
SIGNATURES = {
    "lb_velocity_set": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), _D]),
    "lb_geometry_eval": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(lb_geometry_desc), _D,
                                        ctypes.c_size_t]),
    "lb_force_for_dean": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(lb_geometry_desc),
                                         ctypes.c_double, ctypes.c_double, _D]),
    "lb_create_geometry": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(lb_geometry_desc),
                                          ctypes.c_int, ctypes.c_int, _P,
                                          ctypes.POINTER(lb_allocator), ctypes.POINTER(_P)]),
    "lb_init": (ctypes.c_int, [_P, ctypes.POINTER(lb_params)]),
    "lb_init_fields": (ctypes.c_int, [_P, ctypes.POINTER(lb_params), _P, _P, ctypes.c_int]),
    "lb_step": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "lb_macros": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "lb_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(lb_diag)]),
    "lb_get_populations": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "lb_capture_reference": (ctypes.c_int, [_P]),
    "lb_velocity_change": (ctypes.c_int, [_P, _P, _D, _D]),
    "lb_set_populations": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "lb_state_bytes": (ctypes.c_size_t, [_P]),
    "lb_get_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.c_int]),
    "lb_set_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.c_int]),
    "lb_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong]),
    "lb_step_count": (ctypes.c_longlong, [_P]),
    "lb_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(lb_geometry_desc),
                                              ctypes.c_int, _D, _P, _P, _P,
                                              ctypes.POINTER(lb_diag)]),
    "lb_fma_peak": (ctypes.c_int, [ctypes.c_int, _P, _D]),
    "lb_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(lb_tune), ctypes.POINTER(lb_tune),
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "lb_destroy": (None, [_P]),
    "lb_last_error": (ctypes.c_char_p, [_P]),
    "lb_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "lb_batch_step": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "lb_batch_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong]),
    "lb_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(lb_tune),
                                         ctypes.POINTER(lb_tune), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "lb_batch_nodes": (ctypes.c_longlong, [_P]),
    "lb_batch_step_count": (ctypes.c_longlong, [_P]),
    "lb_batch_destroy": (None, [_P]),
    "lb_batch_last_error": (ctypes.c_char_p, [_P]),
    "lb_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_ulonglong, _P, ctypes.POINTER(_P)]),
    "lb_mlp_param_count": (ctypes.c_size_t, [_P]),
    "lb_mlp_set_output_scale": (ctypes.c_int, [_P, _F, _F]),
    "lb_mlp_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_float, _F]),
    "lb_mlp_predict": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "lb_mlp_get_params": (ctypes.c_int, [_P, _F, ctypes.c_size_t]),
    "lb_mlp_set_params": (ctypes.c_int, [_P, _F, ctypes.c_size_t]),
    "lb_mlp_get_grads": (ctypes.c_int, [_P, _F, ctypes.c_size_t]),
    "lb_mlp_destroy": (None, [_P]),
    "lb_mlp_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblbgm.so (raises RuntimeError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_1411_3133_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LBError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status, ctx=None):
    if status != LB_OK:
        msg = load_library().lb_last_error(ctx).decode()
        raise LBError(status, msg)


def _check_batch(status, batch):
    if status != LB_OK:
        raise LBError(status, load_library().lb_batch_last_error(batch).decode())


def _tune_call(fn, handle, steps_per_trial, check):
    best = lb_tune()
    trials = (lb_tune * 64)()
    n = ctypes.c_int()
    check(fn(handle, int(steps_per_trial), ctypes.byref(best), trials, 64, ctypes.byref(n)), handle)
    return best.as_dict(), [trials[i].as_dict() for i in range(min(n.value, 64))]


def _ptr(a):
    """Device or host address of a torch tensor / numpy array (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------------------
# functions under their C names
# ---------------------------------------------------------------------------
def lb_velocity_set():
    """(c (41, 3) int, w (41,) float64) in the library's population order."""
    c = np.zeros(LB_Q * 3, dtype=np.int32)
    w = np.zeros(LB_Q, dtype=np.float64)
    load_library().lb_velocity_set(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   w.ctypes.data_as(_D))
    return c.reshape(LB_Q, 3).astype(np.int64), w


WALLS = {"bounceback": 0, "equilibrium": 1}


def make_desc(r_inner, r_outer, nr, ntheta, n3, b=1.0, periodic3=True, dtheta_scale=1.0,
              d3_scale=1.0, wall="bounceback") -> lb_geometry_desc:
    return lb_geometry_desc(float(r_inner), float(r_outer), float(b), int(nr), int(ntheta),
                            int(n3), int(bool(periodic3)), float(dtheta_scale), float(d3_scale),
                            WALLS[wall])


def lb_geometry_eval(metric: str, desc: lb_geometry_desc) -> np.ndarray:
    """Host-only geometry rows, shape (nr, n3, LB_GEO_STRIDE), or (nr, ntheta,
    n3, LB_GEO_STRIDE) for the theta-resolved ellipsoid."""
    shape = (desc.nr, desc.ntheta, desc.n3) if metric == "ellipsoidal_theta" else (desc.nr, desc.n3)
    out = np.zeros(int(np.prod(shape)) * LB_GEO_STRIDE)
    _check(load_library().lb_geometry_eval(METRICS[metric], ctypes.byref(desc),
                                           out.ctypes.data_as(_D), out.size))
    return out.reshape(shape + (LB_GEO_STRIDE,))


def lb_force_for_dean(metric: str, desc: lb_geometry_desc, tau: float, De: float) -> float:
    G = ctypes.c_double()
    _check(load_library().lb_force_for_dean(METRICS[metric], ctypes.byref(desc), tau, De,
                                            ctypes.byref(G)))
    return G.value


FORCING_IMPROVED, FORCING_OLD, FORCING_HALF_FORCE_VELOCITY = 0, 1, 2


def make_params(tau, force_G=0.0, old_forcing=False, seed=0, noise_amp=0.0,
                init_base_flow=False) -> lb_params:
    """old_forcing: False / 0 improved forcing (Sec. II), True / 1 the earlier
    method, 2 the half-force velocity variant (see include/lbgm.h)."""
    return lb_params(float(tau), float(force_G), int(old_forcing), int(seed),
                     float(noise_amp), int(bool(init_base_flow)))


def _params_array(params):
    arr = (lb_params * len(params))()
    for i, p in enumerate(params):
        arr[i] = p
    return arr


def torch_allocator(device=None):
    """lb_allocator backed by torch's CUDA caching allocator."""
    import torch
    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:   # the library sees NULL and reports LB_ERR_CUDA
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a_fn, f_fn = ALLOC_FN(_alloc), FREE_FN(_free)
    alloc = lb_allocator(a_fn, f_fn, None)
    alloc._keep = (a_fn, f_fn)   # keep the callbacks alive
    return alloc


def lb_diagnostics_noalloc(metric: str, desc: lb_geometry_desc, taus, rho, u, stream=None):
    """Observables from device fields rho [B*N], u [B*3*N] (torch tensors)
    without any device allocation by the library; see include/lbgm.h.

    The fields are checked here, before the call: CUDA float64 tensors,
    contiguous, holding at least B*N and 3*B*N values (the C side reads
    exactly that many and cannot check a raw pointer)."""
    import torch
    taus = np.ascontiguousarray(taus, dtype=np.float64)
    n = int(desc.nr) * int(desc.ntheta) * int(desc.n3) * len(taus)
    for name, t, need in (("rho", rho, n), ("u", u, 3 * n)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise LBError(LB_ERR_ARG, f"{name} must be a CUDA tensor")
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise LBError(LB_ERR_ARG, f"{name} must be a contiguous float64 tensor")
        if t.numel() < need:
            raise LBError(LB_ERR_ARG, f"{name} holds {t.numel()} values, needs {need}")
    out = (lb_diag * len(taus))()
    handle = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(load_library().lb_diagnostics_noalloc(METRICS[metric], ctypes.byref(desc), len(taus),
                                                 taus.ctypes.data_as(_D), _ptr(rho), _ptr(u),
                                                 handle, out))
    return [d.as_dict() for d in out]


def lb_fma_peak(precision: str = "fp64", stream=None) -> float:
    """Measured FMA peak of the current device in flop/s (see include/lbgm.h)."""
    out = ctypes.c_double()
    handle = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(load_library().lb_fma_peak(PRECISIONS[precision], handle, ctypes.byref(out)))
    return out.value


# ---------------------------------------------------------------------------
# context wrapper
# ---------------------------------------------------------------------------
@dataclass
class ChannelSpec:
    metric: str
    r_inner: float
    r_outer: float
    nr: int
    ntheta: int
    n3: int
    b: float = 1.0
    periodic3: bool = True
    dtheta_scale: float = 1.0
    d3_scale: float = 1.0
    wall: str = "bounceback"

    def desc(self) -> lb_geometry_desc:
        return make_desc(self.r_inner, self.r_outer, self.nr, self.ntheta, self.n3, self.b,
                         self.periodic3, self.dtheta_scale, self.d3_scale, self.wall)

    @property
    def ncells(self):
        return self.nr * self.ntheta * self.n3


class LBContext:
    """One lb_ctx: `batch` instances of a channel on the current CUDA device.

    The context runs on its own torch CUDA stream (``self.stream``) and takes
    its device memory from torch's caching allocator.
    """

    def __init__(self, spec: ChannelSpec, batch: int = 1, precision: str = "fp32",
                 stream=None, use_torch_allocator: bool = True):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("LBContext needs a CUDA device")
        self.spec = spec
        self.batch = batch
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._desc = spec.desc()
        self._alloc = torch_allocator() if use_torch_allocator else None
        ctx = ctypes.c_void_p()
        _check(lib.lb_create_geometry(METRICS[spec.metric], ctypes.byref(self._desc), batch,
                                      PRECISIONS[precision], ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(self._alloc) if self._alloc else None,
                                      ctypes.byref(ctx)))
        self.ctx = ctx
        self._params = None

    # lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            load_library().lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # entry points ----------------------------------------------------------
    def lb_init(self, params):
        self._params = _params_array(params)
        _check(load_library().lb_init(self.ctx, self._params), self.ctx)

    def lb_init_fields(self, params, rho, u, on_device=False):
        self._params = _params_array(params)
        _check(load_library().lb_init_fields(self.ctx, self._params, _ptr(rho), _ptr(u),
                                             int(on_device)), self.ctx)

    def lb_step(self, n=1):
        _check(load_library().lb_step(self.ctx, int(n)), self.ctx)

    def lb_macros(self, rho=None, u=None, on_device=False):
        """Fill caller buffers; with no buffers, return host numpy arrays."""
        N = self.spec.ncells
        if rho is None and u is None and not on_device:
            rho = np.zeros(self.batch * N)
            u = np.zeros(self.batch * 3 * N)
            _check(load_library().lb_macros(self.ctx, _ptr(rho), _ptr(u), 0), self.ctx)
            return rho.reshape(self.batch, N), u.reshape(self.batch, 3, N)
        _check(load_library().lb_macros(self.ctx, _ptr(rho), _ptr(u), int(on_device)), self.ctx)
        return rho, u

    def lb_diagnostics(self):
        out = (lb_diag * self.batch)()
        _check(load_library().lb_diagnostics(self.ctx, out), self.ctx)
        return [d.as_dict() for d in out]

    def lb_get_populations(self, out=None, on_device=False):
        N = self.spec.ncells
        if out is None:
            out = np.zeros(self.batch * LB_Q * N)
            _check(load_library().lb_get_populations(self.ctx, _ptr(out), 0), self.ctx)
            return out.reshape(self.batch, LB_Q, N)
        _check(load_library().lb_get_populations(self.ctx, _ptr(out), int(on_device)), self.ctx)
        return out

    def lb_velocity_change(self, u_prev):
        """(change, umax) per instance against the device array u_prev, which
        is updated to the current velocity."""
        ch = np.zeros(self.batch)
        um = np.zeros(self.batch)
        _check(load_library().lb_velocity_change(self.ctx, _ptr(u_prev), ch.ctypes.data_as(_D),
                                                 um.ctypes.data_as(_D)), self.ctx)
        return ch, um

    def lb_capture_reference(self):
        _check(load_library().lb_capture_reference(self.ctx), self.ctx)

    def lb_set_populations(self, f, on_device=False):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
        _check(load_library().lb_set_populations(self.ctx, _ptr(f), int(on_device)), self.ctx)

    def lb_state_bytes(self):
        return int(load_library().lb_state_bytes(self.ctx))

    def lb_get_state(self, buf, on_device=False):
        _check(load_library().lb_get_state(self.ctx, _ptr(buf), self.lb_state_bytes(),
                                           int(on_device)), self.ctx)
        return buf

    def lb_set_state(self, buf, on_device=False):
        _check(load_library().lb_set_state(self.ctx, _ptr(buf), self.lb_state_bytes(),
                                           int(on_device)), self.ctx)

    def lb_set_option(self, option, value):
        _check(load_library().lb_set_option(self.ctx, int(option), int(value)), self.ctx)

    def lb_step_count(self):
        return int(load_library().lb_step_count(self.ctx))

    def lb_autotune(self, steps_per_trial=20):
        """(best, trials): measured launch configurations; the trial steps
        advance the simulation."""
        return _tune_call(load_library().lb_autotune, self.ctx, steps_per_trial, _check)


class LBBatch:
    """One lb_batch over LBContext members that share precision and stream
    (see include/lbgm.h); the members stay usable on their own."""

    def __init__(self, members):
        lib = load_library()
        self.members = list(members)
        arr = (_P * len(self.members))(*[m.ctx.value for m in self.members])
        h = ctypes.c_void_p()
        _check_batch(lib.lb_batch_create(arr, len(self.members), ctypes.byref(h)), None)
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load_library().lb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def lb_batch_step(self, n=1):
        _check_batch(load_library().lb_batch_step(self.handle, int(n)), self.handle)

    def lb_batch_set_option(self, option, value):
        _check_batch(load_library().lb_batch_set_option(self.handle, int(option), int(value)),
                     self.handle)

    def lb_batch_autotune(self, steps_per_trial=20):
        return _tune_call(load_library().lb_batch_autotune, self.handle, steps_per_trial,
                          _check_batch)

    def lb_batch_nodes(self):
        return int(load_library().lb_batch_nodes(self.handle))

    def lb_batch_step_count(self):
        return int(load_library().lb_batch_step_count(self.handle))


def _check_mlp(status, net):
    if status != LB_OK:
        raise LBError(status, load_library().lb_mlp_last_error(net).decode())


class LBMlp:
    """One lb_mlp (see include/lbgm.h): inputs x (n, n_plain + 1) and fields
    y (n, 4) are torch CUDA float32 tensors."""

    def __init__(self, n_fourier=4, width=256, depth=5, max_batch=16384, seed=20241111, stream=None, n_plain=2):
        import torch
        lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check_mlp(lib.lb_mlp_create(int(n_plain), int(n_fourier), int(width), int(depth), int(max_batch),
                                     int(seed), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), None)
        self.handle = h
        self.n_plain = n_plain
        self.n_fourier, self.width, self.depth, self.max_batch = n_fourier, width, depth, max_batch

    def close(self):
        if getattr(self, "handle", None):
            load_library().lb_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def param_count(self):
        return int(load_library().lb_mlp_param_count(self.handle))

    def set_output_scale(self, mean, std):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(std, dtype=np.float32)
        _check_mlp(load_library().lb_mlp_set_output_scale(self.handle, m.ctypes.data_as(_F),
                                                          s.ctypes.data_as(_F)), self.handle)

    def train_step(self, x, y, lr, want_loss=True):
        loss = ctypes.c_float()
        _check_mlp(load_library().lb_mlp_train_step(self.handle, _ptr(x), _ptr(y), int(x.shape[0]),
                                                    float(lr), ctypes.byref(loss) if want_loss else None),
                   self.handle)
        return loss.value if want_loss else None

    def predict(self, x, out=None):
        import torch
        if out is None:
            out = torch.empty((x.shape[0], 4), dtype=torch.float32, device=x.device)
        _check_mlp(load_library().lb_mlp_predict(self.handle, _ptr(x), int(x.shape[0]), _ptr(out)),
                   self.handle)
        return out

    def _host_call(self, fn, arr=None):
        n = self.param_count()
        a = np.zeros(n, dtype=np.float32) if arr is None else np.ascontiguousarray(arr, dtype=np.float32)
        _check_mlp(fn(self.handle, a.ctypes.data_as(_F), n), self.handle)
        return a

    def get_params(self):
        return self._host_call(load_library().lb_mlp_get_params)

    def set_params(self, p):
        self._host_call(load_library().lb_mlp_set_params, p)

    def get_grads(self):
        return self._host_call(load_library().lb_mlp_get_grads)
