"""Python binding of the C ABI in include/psatd.h (ctypes; argument marshalling only).

Every step of the method runs in the CUDA library libpsatd.so.  Importing this
module loads the library and raises if it is missing: there is no fallback.
Device memory and streams come from PyTorch.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpsatd.so")

OK = 0
ERR_ARG, ERR_SIZE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5, -6
FLAT_TOP, GAUSSIAN, PROFILE = 0, 1, 2
FORWARD, INVERSE = -1, +1
FLAG_NO_FIELD_ALLOC = 1
FLAG_REAL_FIELDS = 2

# every symbol include/psatd.h declares
EXPORTS = (
    "psatd_init_grid", "psatd_destroy", "psatd_set_dt", "psatd_bind_fields", "psatd_fields",
    "psatd_set_field", "psatd_get_field", "psatd_init_pulse", "psatd_advance", "psatd_fft",
    "psatd_sample_focal_plane", "psatd_diagnostics", "psatd_time", "psatd_set_time",
    "psatd_synchronize", "psatd_d_min", "psatd_last_error", "psatd_status_string",
    "psatd_launch_count", "psatd_profile_enable", "psatd_profile_read", "psatd_kernel_name",
    "psatd_set_kernel_path", "psatd_selftest_wait_timeout", "psatd_energy_noalloc",
    "psatd_focal_one_shot", "psatd_batch_begin", "psatd_batch_end", "psatd_batch_launch",
    "psatd_batch_nodes", "psatd_batch_destroy", "psatd_autotune",
    "psatd_fno_create", "psatd_fno_destroy", "psatd_fno_num_params", "psatd_fno_buffers", "psatd_fno_forward",
    "psatd_fno_loss_backward", "psatd_fno_adam_step", "psatd_fno_synchronize", "psatd_fno_last_error",
    "psatd_gemm_bf16", "psatd_set_mapping", "psatd_set_pulse_profile", "psatd_fp64_fma_probe",
    "psatd_multi_advance", "psatd_multi_autotune", "psatd_selftest_grid_barrier_timeout",
    "psatd_debug_set_alloc_limit", "psatd_debug_alloc_live", "psatd_debug_inject_cuda_error",
    "psatd_debug_bounds_report", "psatd_gemm_bf16_tma", "psatd_gemm_synchronize",
)
PATH_AUTO, PATH_GENERIC, PATH_REGISTER = 0, 1, 2

KERNEL_KINDS = ("fft_x", "fft_y", "fft_z", "kspace_z", "init_pulse", "sample_plane", "diagnostics",
                "plane_xy")


class PsatdGrid(C.Structure):
    _fields_ = [("Nx", C.c_int), ("Ny", C.c_int), ("Nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x_min", C.c_double), ("y_min", C.c_double), ("z_min", C.c_double),
                ("c", C.c_double)]


class PsatdMapping(C.Structure):
    _fields_ = [("R0", C.c_double), ("L", C.c_double)]


class PsatdPulse(C.Structure):
    _fields_ = [("kind", C.c_int), ("div_project", C.c_int),
                ("lambda_", C.c_double), ("theta", C.c_double), ("eps", C.c_double),
                ("P0", C.c_double), ("n_cycles", C.c_double), ("cep", C.c_double),
                ("ellipticity", C.c_double), ("pol_angle", C.c_double)]


class PsatdFnoConfig(C.Structure):
    _fields_ = [("in_params", C.c_int), ("width", C.c_int), ("layers", C.c_int), ("patch", C.c_int),
                ("modes", C.c_int), ("hidden", C.c_int), ("out_channels", C.c_int), ("max_batch", C.c_int)]


class PsatdDiag(C.Structure):
    _fields_ = [("energy", C.c_double), ("energy_E", C.c_double), ("energy_B", C.c_double),
                ("max_div_E", C.c_double), ("max_div_B", C.c_double),
                ("max_E_hat", C.c_double), ("max_B_hat", C.c_double)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError("libpsatd.so is not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "psatd_init_grid": (C.c_int, [C.POINTER(PsatdGrid), C.POINTER(PsatdMapping), C.c_double, C.c_int, P, C.c_int, C.POINTER(P)]),
        "psatd_destroy": (None, [P]),
        "psatd_set_dt": (C.c_int, [P, C.c_double]),
        "psatd_bind_fields": (C.c_int, [P, P, C.c_size_t]),
        "psatd_fields": (C.c_int, [P, C.POINTER(P), C.POINTER(C.c_size_t)]),
        "psatd_set_field": (C.c_int, [P, C.c_int, P, C.c_int]),
        "psatd_get_field": (C.c_int, [P, C.c_int, P, C.c_int]),
        "psatd_init_pulse": (C.c_int, [P, C.POINTER(PsatdPulse)]),
        "psatd_set_pulse_profile": (C.c_int, [P, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_double]),
        "psatd_advance": (C.c_int, [P, C.c_int]),
        "psatd_fft": (C.c_int, [P, C.c_int]),
        "psatd_sample_focal_plane": (C.c_int, [P, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double,
                                               C.c_double, C.c_double, C.c_int, P, C.c_int]),
        "psatd_diagnostics": (C.c_int, [P, C.POINTER(PsatdDiag)]),
        "psatd_time": (C.c_double, [P]),
        "psatd_set_time": (C.c_int, [P, C.c_double]),
        "psatd_synchronize": (C.c_int, [P]),
        "psatd_d_min": (C.c_double, [C.c_double, C.c_double, C.c_double]),
        "psatd_last_error": (C.c_char_p, [P]),
        "psatd_status_string": (C.c_char_p, [C.c_int]),
        "psatd_launch_count": (C.c_longlong, [P]),
        "psatd_profile_enable": (C.c_int, [P, C.c_int]),
        "psatd_profile_read": (C.c_int, [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
        "psatd_kernel_name": (C.c_char_p, [C.c_int]),
        "psatd_set_kernel_path": (C.c_int, [P, C.c_int]),
        "psatd_selftest_wait_timeout": (C.c_int, [P]),
        "psatd_energy_noalloc": (C.c_int, [P, C.c_int, C.c_longlong, C.POINTER(C.c_double), C.c_int, P]),
        "psatd_focal_one_shot": (C.c_int, [P, C.POINTER(PsatdPulse), C.c_double, C.c_double, C.c_int, C.c_int,
                                           C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, P, C.c_int]),
        "psatd_batch_begin": (C.c_int, [P, C.POINTER(P)]),
        "psatd_batch_end": (C.c_int, [P]),
        "psatd_batch_launch": (C.c_int, [P]),
        "psatd_batch_nodes": (C.c_longlong, [P]),
        "psatd_batch_destroy": (None, [P]),
        "psatd_autotune": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "psatd_fno_create": (C.c_int, [C.POINTER(PsatdFnoConfig), C.c_ulonglong, P, C.POINTER(P)]),
        "psatd_fno_destroy": (None, [P]),
        "psatd_fno_num_params": (C.c_longlong, [P]),
        "psatd_fno_buffers": (C.c_int, [P, C.POINTER(P), C.POINTER(P), C.POINTER(P)]),
        "psatd_fno_forward": (C.c_int, [P, P, C.c_int, P]),
        "psatd_fno_loss_backward": (C.c_int, [P, P, C.c_int, P, C.POINTER(C.c_double)]),
        "psatd_fno_adam_step": (C.c_int, [P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float]),
        "psatd_fno_synchronize": (C.c_int, [P]),
        "psatd_fno_last_error": (C.c_char_p, [P]),
        "psatd_set_mapping": (C.c_int, [P, C.POINTER(PsatdMapping)]),
        "psatd_fp64_fma_probe": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P]),
        "psatd_multi_advance": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.c_int)]),
        "psatd_multi_autotune": (C.c_int, [C.POINTER(P), C.c_int, C.c_int, C.POINTER(C.c_double)]),
        "psatd_selftest_grid_barrier_timeout": (C.c_int, [P]),
        "psatd_debug_set_alloc_limit": (None, [C.c_longlong]),
        "psatd_debug_alloc_live": (C.c_longlong, []),
        "psatd_debug_inject_cuda_error": (None, [C.c_int, C.c_int]),
        "psatd_debug_bounds_report": (C.c_longlong, [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "psatd_gemm_bf16_tma": (C.c_int, [C.c_int, C.c_int, C.c_int, P, P, P, P]),
        "psatd_gemm_synchronize": (C.c_int, [P]),
        "psatd_gemm_bf16": (C.c_int, [C.c_int, C.c_int, C.c_int, P, C.c_longlong, C.c_longlong, P, C.c_longlong,
                                      C.c_longlong, P, C.c_longlong, C.c_longlong, C.c_float, C.c_float, C.c_int, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class PsatdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (lib().psatd_status_string(status).decode(), msg))
        self.status = status


def _check(status: int, ctx_ptr=None):
    if status != OK:
        raise PsatdError(status, lib().psatd_last_error(ctx_ptr).decode())


def d_min(R0: float, L: float, theta: float) -> float:
    """Eq. 12 through the library."""
    return lib().psatd_d_min(R0, L, theta)


def make_grid(g) -> PsatdGrid:
    return PsatdGrid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def make_pulse(p) -> PsatdPulse:
    return PsatdPulse(p.kind, p.div_project, p.lam, p.theta, p.eps, p.P0, p.n_cycles, p.cep,
                      p.ellipticity, p.pol_angle)


class Batch:
    """A CUDA graph of library calls recorded on one stream (see psatd_batch_*).

        with Batch(stream) as b:        # records
            ctx1.advance(4); ctx2.focal_one_shot(..., out=dev_tensor)
        b.launch()                      # replays with one graph launch
    """

    def __init__(self, stream):
        self.stream = stream
        self._ptr = C.c_void_p()

    def __enter__(self):
        _check(lib().psatd_batch_begin(C.c_void_p(self.stream.cuda_stream), C.byref(self._ptr)), None)
        return self

    def __exit__(self, exc_type, exc, tb):
        st = lib().psatd_batch_end(self._ptr)
        if exc_type is None:
            _check(st, None)

    def launch(self):
        _check(lib().psatd_batch_launch(self._ptr), None)

    @property
    def nodes(self) -> int:
        return lib().psatd_batch_nodes(self._ptr)

    def close(self):
        if self._ptr and self._ptr.value:
            lib().psatd_batch_destroy(self._ptr)
            self._ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Fno:
    """The surrogate network (psatd_fno_*): parameters, gradients and output are
    device tensors owned by the model and exposed as torch views."""

    def __init__(self, in_params, width=32, layers=4, patch=64, modes=12, hidden=64, out_channels=3,
                 max_batch=8, seed=0, stream=None):
        import torch
        self._torch = torch
        self.cfg = PsatdFnoConfig(in_params, width, layers, patch, modes, hidden, out_channels, max_batch)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._ptr = C.c_void_p()
        st = lib().psatd_fno_create(C.byref(self.cfg), seed, C.c_void_p(self.stream.cuda_stream), C.byref(self._ptr))
        if st != OK:
            raise PsatdError(st, "psatd_fno_create failed")
        self.n_params = lib().psatd_fno_num_params(self._ptr)
        pp, gp, op = C.c_void_p(), C.c_void_p(), C.c_void_p()
        lib().psatd_fno_buffers(self._ptr, C.byref(pp), C.byref(gp), C.byref(op))
        self._bufs = (pp.value, gp.value, op.value)
        self.device = dev

    @property
    def params(self):
        return _device_view(self._bufs[0], self.n_params, self.device)

    @property
    def grads(self):
        return _device_view(self._bufs[1], self.n_params, self.device)

    def output(self, batch):
        c = self.cfg
        return _device_view(self._bufs[2], batch * c.out_channels * c.patch ** 3, self.device).view(
            batch, c.out_channels, c.patch, c.patch, c.patch)

    def _check(self, st):
        if st != OK:
            raise PsatdError(st, lib().psatd_fno_last_error(self._ptr).decode())

    def forward(self, prm):
        """prm: float32 CUDA tensor [B][in_params]; returns the output view."""
        B = prm.shape[0]
        self._check(lib().psatd_fno_forward(self._ptr, C.c_void_p(prm.data_ptr()), B, None))
        return self.output(B)

    def loss_backward(self, prm, target, want_loss=True):
        loss = C.c_double()
        self._check(lib().psatd_fno_loss_backward(self._ptr, C.c_void_p(prm.data_ptr()), prm.shape[0],
                                                  C.c_void_p(target.data_ptr()), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        self._check(lib().psatd_fno_adam_step(self._ptr, lr, beta1, beta2, eps, weight_decay))

    def synchronize(self):
        self._check(lib().psatd_fno_synchronize(self._ptr))

    def close(self):
        if self._ptr and self._ptr.value:
            lib().psatd_fno_destroy(self._ptr)
            self._ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(addr, n, device):
    """A float32 torch tensor aliasing n floats of device memory at addr (the
    owner keeps the memory alive)."""
    import torch

    class _Holder:
        def __init__(self, ptr, size):
            self.__cuda_array_interface__ = {"shape": (size,), "typestr": "<f4", "data": (ptr, False),
                                             "version": 2, "strides": None}
    return torch.as_tensor(_Holder(addr, n), device=device)


def gemm_bf16(A, B, Cout, alpha=1.0, beta=0.0, ksplit=1, stream=None):
    """Cout = alpha A B + beta Cout on float32 CUDA tensors (2-D, any strides)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    M, K = A.shape
    K2, N = B.shape
    assert K == K2 and tuple(Cout.shape) == (M, N)
    st = lib().psatd_gemm_bf16(M, N, K, C.c_void_p(A.data_ptr()), A.stride(0), A.stride(1), C.c_void_p(B.data_ptr()),
                               B.stride(0), B.stride(1), C.c_void_p(Cout.data_ptr()), Cout.stride(0), Cout.stride(1),
                               alpha, beta, ksplit, C.c_void_p(s.cuda_stream))
    _check(st, None)
    return Cout


def gemm_bf16_tma(A, B, Cout, stream=None):
    """Cout = A @ B.T on the tensor cores: A (M x K), B (N x K) bfloat16 CUDA
    tensors, Cout (M x N) float32, all contiguous; M % 128, N % 256, K % 64 == 0."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    M, K = A.shape
    N = B.shape[0]
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and Cout.dtype == torch.float32
    assert A.is_contiguous() and B.is_contiguous() and Cout.is_contiguous() and B.shape[1] == K
    assert tuple(Cout.shape) == (M, N)
    _check(lib().psatd_gemm_bf16_tma(M, N, K, C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                     C.c_void_p(Cout.data_ptr()), C.c_void_p(s.cuda_stream)), None)
    return Cout


def gemm_synchronize(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().psatd_gemm_synchronize(C.c_void_p(s.cuda_stream)), None)


def fp64_fma_probe(out, blocks, threads, iters, stream=None):
    """Launch the float64 FMA rate probe (16 * iters flops per thread) writing
    one float64 per thread to the CUDA tensor out (blocks * threads elements)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    assert out.dtype == torch.float64 and out.is_cuda and out.numel() >= blocks * threads
    _check(lib().psatd_fp64_fma_probe(C.c_void_p(out.data_ptr()), blocks, threads, iters,
                                      C.c_void_p(s.cuda_stream)), None)
    return out


def _ctx_array(ctxs):
    arr = (C.c_void_p * len(ctxs))(*[c._ptr.value for c in ctxs])
    return arr


def multi_advance(ctxs, n_steps):
    """Advance the contexts in one persistent launch: n_steps is one count for
    all or a list with one count per context (the contexts share one stream and
    precision; errors come from ctxs[0])."""
    counts = [int(n_steps)] * len(ctxs) if np.isscalar(n_steps) else [int(n) for n in n_steps]
    assert len(counts) == len(ctxs)
    arr = (C.c_int * len(ctxs))(*counts)
    _check(lib().psatd_multi_advance(_ctx_array(ctxs), len(ctxs), arr), ctxs[0]._ptr)


def multi_autotune(ctxs, trial_steps: int = 1) -> float:
    """Tune the batched advance's radix schedules and tile widths per axis
    length; returns the best time per step in ms."""
    ms = C.c_double()
    _check(lib().psatd_multi_autotune(_ctx_array(ctxs), len(ctxs), trial_steps, C.byref(ms)), ctxs[0]._ptr)
    return ms.value


class Context:
    """One periodic box on the current CUDA device; fields are a torch tensor
    [6, Nz, Ny, Nx] (complex64 or complex128, or float32 with real=True) bound
    to the library.  Sampled planes are complex of the context's precision."""

    def __init__(self, grid, mapping=None, dt: float = 0.0, precision: int = 64, stream=None,
                 fields=None, real: bool = False):
        import torch
        self._torch = torch
        self.grid = grid
        self.precision = precision
        self.real = real
        self.cdtype = torch.complex128 if precision == 64 else torch.complex64
        self.dtype = torch.float32 if real else self.cdtype
        self._np_field = np.float32 if real else (np.complex128 if precision == 64 else np.complex64)
        self._np_sample = np.complex128 if precision == 64 else np.complex64
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        m = PsatdMapping(mapping.R0, mapping.L) if mapping is not None else None
        ptr = C.c_void_p()
        flags = FLAG_NO_FIELD_ALLOC | (FLAG_REAL_FIELDS if real else 0)
        st = lib().psatd_init_grid(C.byref(make_grid(grid)), C.byref(m) if m is not None else None, dt,
                                   precision, C.c_void_p(self.stream.cuda_stream), flags, C.byref(ptr))
        _check(st, None)
        self._ptr = ptr
        if fields is None:
            fields = torch.zeros((6, grid.Nz, grid.Ny, grid.Nx), dtype=self.dtype, device=dev)
        assert fields.dtype == self.dtype and fields.is_contiguous() and fields.is_cuda
        self.fields = fields
        _check(lib().psatd_bind_fields(self._ptr, C.c_void_p(fields.data_ptr()),
                                       fields.numel() * fields.element_size()), self._ptr)

    # -- lifetime
    def close(self):
        if getattr(self, "_ptr", None) is not None and self._ptr.value:
            lib().psatd_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def set_mapping(self, mapping):
        m = PsatdMapping(mapping.R0, mapping.L)
        _check(lib().psatd_set_mapping(self._ptr, C.byref(m)), self._ptr)

    def set_dt(self, dt: float):
        _check(lib().psatd_set_dt(self._ptr, dt), self._ptr)

    def set_field(self, comp: int, src):
        """src: numpy array (host) or torch tensor (device), layout of the storage."""
        if isinstance(src, np.ndarray):
            a = np.ascontiguousarray(src, dtype=self._np_field)
            _check(lib().psatd_set_field(self._ptr, comp, a.ctypes.data_as(C.c_void_p), 0), self._ptr)
        else:
            t = src.to(self.dtype).contiguous()
            _check(lib().psatd_set_field(self._ptr, comp, C.c_void_p(t.data_ptr()), 1), self._ptr)

    def set_fields(self, src):
        self.set_field(-1, src)

    def get_field(self, comp: int = -1) -> np.ndarray:
        shape = (self.grid.Nz, self.grid.Ny, self.grid.Nx)
        out = np.empty(((6,) if comp < 0 else ()) + shape, dtype=self._np_field)
        _check(lib().psatd_get_field(self._ptr, comp, out.ctypes.data_as(C.c_void_p), 0), self._ptr)
        return out

    def set_pulse_profile(self, a, zeta0: float, dzeta: float):
        """Longitudinal profile of PROFILE pulses: complex samples a_k = a(zeta0 + k dzeta)."""
        z = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
        buf = z.view(np.float64)
        _check(lib().psatd_set_pulse_profile(self._ptr, buf.ctypes.data_as(C.POINTER(C.c_double)), int(z.size),
                                             float(zeta0), float(dzeta)), self._ptr)

    def init_pulse(self, pulse):
        _check(lib().psatd_init_pulse(self._ptr, C.byref(make_pulse(pulse))), self._ptr)

    def advance(self, n: int):
        _check(lib().psatd_advance(self._ptr, n), self._ptr)

    def fft(self, direction: int):
        _check(lib().psatd_fft(self._ptr, direction), self._ptr)

    def sample_focal_plane(self, x_phys, ny, nz, y0, y1, z0, z1, comps=(0, 1, 2), out=None):
        mask = 0
        for c in comps:
            mask |= 1 << c
        nc = bin(mask).count("1")
        if out is None:
            out = np.empty((nc, nz, ny), dtype=self._np_sample)
            _check(lib().psatd_sample_focal_plane(self._ptr, x_phys, ny, nz, y0, y1, z0, z1, mask,
                                                  out.ctypes.data_as(C.c_void_p), 0), self._ptr)
            return out
        assert out.dtype == self.cdtype and out.is_cuda and out.numel() >= nc * ny * nz
        _check(lib().psatd_sample_focal_plane(self._ptr, x_phys, ny, nz, y0, y1, z0, z1, mask,
                                              C.c_void_p(out.data_ptr()), 1), self._ptr)
        return out

    def focal_one_shot(self, pulse, T, x_phys, ny, nz, y0, y1, z0, z1, comps=(0, 1, 2), out=None):
        mask = 0
        for c in comps:
            mask |= 1 << c
        nc = bin(mask).count("1")
        if out is None:
            out = np.empty((nc, nz, ny), dtype=self._np_sample)
            _check(lib().psatd_focal_one_shot(self._ptr, C.byref(make_pulse(pulse)), T, x_phys, ny, nz, y0, y1,
                                              z0, z1, mask, out.ctypes.data_as(C.c_void_p), 0), self._ptr)
            return out
        assert out.dtype == self.cdtype and out.is_cuda and out.numel() >= nc * ny * nz
        _check(lib().psatd_focal_one_shot(self._ptr, C.byref(make_pulse(pulse)), T, x_phys, ny, nz, y0, y1, z0,
                                          z1, mask, C.c_void_p(out.data_ptr()), 1), self._ptr)
        return out

    def diagnostics(self) -> dict:
        d = PsatdDiag()
        _check(lib().psatd_diagnostics(self._ptr, C.byref(d)), self._ptr)
        return {k: getattr(d, k) for k, _ in PsatdDiag._fields_}

    @property
    def time(self) -> float:
        return lib().psatd_time(self._ptr)

    def set_time(self, t: float):
        _check(lib().psatd_set_time(self._ptr, t), self._ptr)

    def synchronize(self):
        _check(lib().psatd_synchronize(self._ptr), self._ptr)

    @property
    def launch_count(self) -> int:
        return lib().psatd_launch_count(self._ptr)

    def autotune(self, trial_steps: int = 2):
        path, shift, ms = C.c_int(), C.c_int(), C.c_double()
        _check(lib().psatd_autotune(self._ptr, trial_steps, C.byref(path), C.byref(shift), C.byref(ms)), self._ptr)
        return path.value, shift.value, ms.value

    def selftest_grid_barrier_timeout(self) -> int:
        """Status of the batched advance's barrier self-test (ERR_TIMEOUT expected)."""
        return lib().psatd_selftest_grid_barrier_timeout(self._ptr)

    def set_kernel_path(self, path: int):
        _check(lib().psatd_set_kernel_path(self._ptr, path), self._ptr)

    def profile_enable(self, on: bool = True):
        _check(lib().psatd_profile_enable(self._ptr, 1 if on else 0), self._ptr)

    def profile_read(self) -> dict:
        """{kernel name: (total ms, timed launches)} since profiling was enabled."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            ms, n = C.c_double(), C.c_longlong()
            _check(lib().psatd_profile_read(self._ptr, k, C.byref(ms), C.byref(n)), self._ptr)
            if n.value:
                out[name] = (ms.value, n.value)
        return out
