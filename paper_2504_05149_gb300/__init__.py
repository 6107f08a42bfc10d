"""Fast SE(2) convolutions on Z^2\\SE(2) for GB300 -- Python binding.

A thin ctypes layer over the C ABI of libse2.so (include/se2.h): it checks
tensor shapes/dtypes/devices, passes raw device pointers and the current
CUDA stream, and raises on any non-OK status.  Every step of the path runs in
the library's CUDA kernels; PyTorch only provides device memory and streams.
There is no CPU fallback: if the library is missing this module raises.

The operation (arXiv 2504.05149, Algorithm 3 at output grid N = L):
    out = iDFT( W . DFT(f) . C ),   C = DFT(P) / |L|
for f, P sampled on the grid Omega_L ([M][N][N] = [theta][y][x]).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libse2.so")

F64 = 0
F32 = 1
SPLIT_BF16 = 2
BF16 = 3
SPLIT_F16 = 4
_PRECISIONS = {"f64": F64, "f32": F32, "split_bf16": SPLIT_BF16, "bf16": BF16, "split_f16": SPLIT_F16}
SHARED_KERNEL = 0x1
PERSISTENT = 0x2
GRID_ORIGIN_ZERO = 0x4        # grids sampled at x_i = i/N: the plain cyclic convolution (no W)
MASS_RENORM = 0x8             # FP64 mass renormalisation of convolve / convolve_chain outputs
KERNEL_YSYM = 0x10            # kernel spectra mirror-symmetric in y (radial kernels): half the C rows read
HOST_STAGING = 0x20           # convolve_host staging allocated with the plan
CHECK_FINITE = 0x40           # outputs checked for NaN / infinity (status(): SE2_ERR_NUMERIC)

_STATUS = {0: "SE2_OK", 1: "SE2_ERR_INVALID_ARG", 2: "SE2_ERR_UNSUPPORTED", 3: "SE2_ERR_OOM",
           4: "SE2_ERR_CUDA", 5: "SE2_ERR_TIMEOUT", 6: "SE2_ERR_NUMERIC"}

_lib = None


class SE2Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH):
    """Load libse2.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libse2.so not found at {path}; run paper_2504_05149_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.se2_plan_create.argtypes = [ctypes.POINTER(vp), ip, ip, ip, ip, ctypes.c_uint, ip]
    lib.se2_plan_destroy.argtypes = [vp]
    lib.se2_plan_workspace_bytes.argtypes = [vp]
    lib.se2_plan_workspace_bytes.restype = ctypes.c_size_t
    lib.se2_coeffs.argtypes = [vp, vp, ip, vp, vp, vp]
    lib.se2_convolve.argtypes = [vp, vp, ip, vp, vp, vp, vp]
    lib.se2_convolve_host.argtypes = [vp, vp, ip, vp, vp, vp, vp]
    lib.se2_convolve_chain_all.argtypes = [vp, vp, ip, ctypes.POINTER(vp), ctypes.POINTER(vp), ip, vp, vp]
    lib.se2_convolve_chain.argtypes = [vp, vp, ip, ctypes.POINTER(vp), ctypes.POINTER(vp), ip, vp, vp]
    lib.se2_plan_status.argtypes = [vp, vp]
    lib.se2_separable_tables.argtypes = [vp, vp, vp, ip, ip, vp, vp]
    lib.se2_convolve_separable.argtypes = [vp, vp, ip, vp, vp, vp]
    lib.se2_backward.argtypes = [vp, vp, vp, ip, vp, vp, ip, ctypes.POINTER(vp), vp, vp, vp]
    lib.se2_sample_radial_gaussian.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp]
    dptr = ctypes.POINTER(ctypes.c_double)
    lib.se2_sample_se2_gaussian.argtypes = [vp, dptr, dptr, ctypes.c_int, vp, vp]
    lib.se2_sample_deformed_gaussian.argtypes = [vp, dptr, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, vp]
    i3 = ctypes.POINTER(ctypes.c_int)
    lib.se2_grid_plan_create.argtypes = [ctypes.POINTER(vp), i3, i3, ip, ip, ctypes.c_uint, ip]
    lib.se2_grid_plan_destroy.argtypes = [vp]
    lib.se2_grid_plan_launches.argtypes = [vp]
    lib.se2_grid_plan_launches.restype = ctypes.c_ulonglong
    lib.se2_grid_coeffs.argtypes = [vp, vp, ip, vp, vp]
    lib.se2_grid_ffc_at.argtypes = [vp, vp, ip, ip, ip, ip, vp, vp]
    lib.se2_debug_alloc_stats.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.se2_debug_fail_alloc.argtypes = [ctypes.c_longlong]
    lib.se2_grid_convolve_chain.argtypes = [vp, vp, ip, ctypes.POINTER(vp), ip, vp, vp]
    lib.se2_grid_convolve_chain_all.argtypes = [vp, vp, ip, ctypes.POINTER(vp), ip, vp, vp]
    lib.se2_grid_sample_se2_gaussian.argtypes = [vp, dptr, dptr, ctypes.c_int, vp, vp]
    lib.se2_grid_sample_deformed_gaussian.argtypes = [vp, dptr, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, vp]
    lib.se2_accuracy_order.argtypes = [ctypes.c_double, ctypes.c_double, ip, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_longlong)]
    lib.se2_debug_wait_timeout.argtypes = [vp, vp, vp, vp, vp]
    lib.se2_plan_timing.argtypes = [vp, ip]
    lib.se2_plan_timing_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.se2_plan_launches.argtypes = [vp]
    lib.se2_plan_launches.restype = ctypes.c_ulonglong
    lib.se2_last_error.restype = ctypes.c_char_p
    lib.se2_version.restype = ctypes.c_char_p
    for name in ("se2_plan_create", "se2_plan_destroy", "se2_coeffs", "se2_convolve", "se2_convolve_host",
                 "se2_convolve_chain", "se2_convolve_chain_all",
                 "se2_plan_status", "se2_debug_wait_timeout", "se2_backward", "se2_sample_radial_gaussian",
                 "se2_sample_se2_gaussian", "se2_sample_deformed_gaussian",
                 "se2_grid_plan_create", "se2_grid_plan_destroy", "se2_grid_coeffs", "se2_grid_ffc_at",
                 "se2_grid_convolve_chain", "se2_grid_convolve_chain_all",
                 "se2_accuracy_order", "se2_plan_timing", "se2_plan_timing_read", "se2_grid_sample_se2_gaussian", "se2_grid_sample_deformed_gaussian",
                 "se2_separable_tables", "se2_convolve_separable", "se2_debug_alloc_stats", "se2_debug_fail_alloc"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise SE2Error(status, load_library().se2_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Plan:
    """Twiddle tables and scratch for batches of up to `batch` N x N x M grids."""

    def __init__(self, N: int, M: int, batch: int = 1, precision: str = "f32", flags: int = 0,
                 device: Optional[int] = None):
        lib = load_library()
        if precision not in _PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(_PRECISIONS)}")
        self.N, self.M, self.batch, self.flags = N, M, batch, flags
        self.precision = precision
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.cdtype = torch.complex128 if precision == "f64" else torch.complex64
        h = ctypes.c_void_p()
        _check(lib.se2_plan_create(ctypes.byref(h), N, M, batch, _PRECISIONS[precision], flags, self.device))
        self._h = h

    @property
    def handle(self):
        return self._h

    def launches(self) -> int:
        """Kernels launched through this plan so far (se2_plan_launches)."""
        return int(load_library().se2_plan_launches(self._h))

    def timing(self, on: bool = True):
        """Record per-launch durations of the FP32 fast path's units (and clear
        earlier records); see timing_read."""
        _check(load_library().se2_plan_timing(self._h, 1 if on else 0))

    def timing_read(self):
        """[(summed ms, launches)] for units 0 (kf_fwd_xt), 1 (kf_lines),
        2 (kf_inv_tx) since timing was switched on."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_longlong * 4)()
        _check(load_library().se2_plan_timing_read(self._h, ms, n))
        return [(float(ms[i]), int(n[i])) for i in range(4)]

    def workspace_bytes(self) -> int:
        return int(load_library().se2_plan_workspace_bytes(self._h))

    def status(self):
        """Synchronise the current stream and raise SE2Error if a bounded
        device-side wait of the persistent kernel gave up since the last call."""
        _check(load_library().se2_plan_status(self._h, _stream(self.device)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().se2_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shape helpers -------------------------------------------------------
    def grid_shape(self, B: int):
        return (B, self.M, self.N, self.N)

    def spec_shape(self, B: int):
        return (B, self.M, self.N, self.N // 2 + 1)

    def _check_grid(self, t: torch.Tensor, name: str) -> int:
        if t.dim() != 4 or tuple(t.shape[1:]) != (self.M, self.N, self.N):
            raise ValueError(f"{name}: expected [B, {self.M}, {self.N}, {self.N}], got {tuple(t.shape)}")
        if t.dtype != self.dtype or not t.is_cuda or t.device.index != self.device or not t.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {self.dtype} tensor on cuda:{self.device}")
        return t.shape[0]

    def _check_spec(self, t: torch.Tensor, name: str, B: int):
        shared = bool(self.flags & SHARED_KERNEL)
        want = (1 if shared else B, self.M, self.N, self.N // 2 + 1)
        if t.dim() == 3 and shared:
            t = t.unsqueeze(0)
        if tuple(t.shape) != want:
            raise ValueError(f"{name}: expected {want}, got {tuple(t.shape)}")
        if t.dtype != self.cdtype or not t.is_cuda or t.device.index != self.device or not t.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {self.cdtype} tensor on cuda:{self.device}")
        return t


def coeffs(plan: Plan, samples: torch.Tensor, normalize: bool = False):
    """C = DFT(P)/|L| of each kernel in `samples` ([n, M, N, N] real).
    Returns (C [n, M, N, N/2+1] complex, log_scale [n] float64 or None)."""
    n = plan._check_grid(samples, "samples")
    C = torch.empty(plan.spec_shape(n), dtype=plan.cdtype, device=samples.device)
    ls = torch.empty(n, dtype=torch.float64, device=samples.device) if normalize else None
    _check(load_library().se2_coeffs(plan.handle, _ptr(samples), n, _ptr(C), _ptr(ls), _stream(samples.device)))
    return C, ls


def convolve(plan: Plan, f: torch.Tensor, C: torch.Tensor, log_scale: Optional[torch.Tensor] = None,
             out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """S_K[f, rho] on Omega_L for a batch f [B, M, N, N]."""
    return convolve_chain(plan, f, [C], None if log_scale is None else [log_scale], out)


def convolve_host(plan: Plan, f: torch.Tensor, C: torch.Tensor, log_scale: Optional[torch.Tensor] = None,
                  out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """se2_convolve with f and out in host memory (se2_convolve_host): copies
    in, convolutions and copies out of problem groups overlap on the device.
    f: contiguous CPU tensor [B, M, N, N] of the plan's real type (pin it for
    asynchronous copies); out: same, allocated pinned if not given.  Returns
    out after synchronising the current stream."""
    if f.dim() != 4 or tuple(f.shape[1:]) != (plan.M, plan.N, plan.N) or f.dtype != plan.dtype \
            or f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f: need a contiguous CPU {plan.dtype} tensor [B, {plan.M}, {plan.N}, {plan.N}]")
    B = f.shape[0]
    if out is None:
        out = torch.empty(f.shape, dtype=f.dtype, pin_memory=True)
    elif tuple(out.shape) != tuple(f.shape) or out.dtype != f.dtype or out.is_cuda or not out.is_contiguous():
        raise ValueError("out: need a contiguous CPU tensor shaped like f")
    C = plan._check_spec(C, "coeffs", B)
    if log_scale is not None and (log_scale.dtype != torch.float64 or not log_scale.is_cuda
                                  or not log_scale.is_contiguous()):
        raise ValueError("log_scale: need a contiguous float64 CUDA tensor")
    stream = _stream(plan.device)
    _check(load_library().se2_convolve_host(plan.handle, _ptr(f), B, _ptr(C), _ptr(log_scale), _ptr(out), stream))
    torch.cuda.current_stream(plan.device).synchronize()
    return out


def convolve_chain(plan: Plan, f: torch.Tensor, Cs: Sequence[torch.Tensor],
                   log_scales: Optional[Sequence[Optional[torch.Tensor]]] = None,
                   out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """f * rho_1 * ... * rho_k via W^k . DFT(f) . C_1 ... C_k."""
    B = plan._check_grid(f, "f")
    if out is None:
        out = torch.empty_like(f)
    else:
        plan._check_grid(out, "out")
    k = len(Cs)
    Cs = [plan._check_spec(C, f"coeffs[{i}]", B) for i, C in enumerate(Cs)]
    cp = (ctypes.c_void_p * k)(*[C.data_ptr() for C in Cs])
    if log_scales is not None:
        if len(log_scales) != k:
            raise ValueError("log_scales must have one entry per kernel")
        for ls in log_scales:
            if ls is not None and (ls.dtype != torch.float64 or not ls.is_cuda or not ls.is_contiguous()):
                raise ValueError("log_scale: need a contiguous float64 CUDA tensor")
        lp = (ctypes.c_void_p * k)(*[0 if ls is None else ls.data_ptr() for ls in log_scales])
    else:
        lp = None
    _check(load_library().se2_convolve_chain(plan.handle, _ptr(f), B, cp, lp, k, _ptr(out), _stream(f.device)))
    return out


def convolve_chain_all(plan: Plan, f: torch.Tensor, Cs: Sequence[torch.Tensor],
                       log_scales: Optional[Sequence[Optional[torch.Tensor]]] = None,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Every intermediate V_p = f * rho_1 * ... * rho_p, p = 1..k (Algorithm 6),
    from one forward transform: returns [k, B, M, N, N]."""
    B = plan._check_grid(f, "f")
    k = len(Cs)
    if out is None:
        out = torch.empty((k,) + tuple(f.shape), dtype=f.dtype, device=f.device)
    elif tuple(out.shape) != (k,) + tuple(f.shape) or out.dtype != f.dtype or not out.is_contiguous():
        raise ValueError("out: need a contiguous tensor [k, B, M, N, N] like f")
    Cs = [plan._check_spec(C, f"coeffs[{i}]", B) for i, C in enumerate(Cs)]
    cp = (ctypes.c_void_p * k)(*[C.data_ptr() for C in Cs])
    lp = None
    if log_scales is not None:
        if len(log_scales) != k:
            raise ValueError("log_scales must have one entry per kernel")
        lp = (ctypes.c_void_p * k)(*[0 if ls is None else ls.data_ptr() for ls in log_scales])
    _check(load_library().se2_convolve_chain_all(plan.handle, _ptr(f), B, cp, lp, k, _ptr(out), _stream(f.device)))
    return out


def backward(plan: Plan, grad_out: torch.Tensor, C: torch.Tensor, f: Optional[torch.Tensor] = None,
             dCs: Sequence[torch.Tensor] = (), log_scale: Optional[torch.Tensor] = None,
             want_grad_f: bool = True):
    """Adjoint of convolve: returns (grad_f or None, grad_params [len(dCs)] float64)."""
    B = plan._check_grid(grad_out, "grad_out")
    C = plan._check_spec(C, "coeffs", B)
    n = len(dCs)
    dCs = [plan._check_spec(d, f"dcoeffs[{i}]", B) for i, d in enumerate(dCs)]
    if n > 0:
        if f is None:
            raise ValueError("parameter gradients need f")
        plan._check_grid(f, "f")
    gf = torch.empty_like(grad_out) if want_grad_f else None
    gp = torch.zeros(max(n, 1), dtype=torch.float64, device=grad_out.device)
    dp = (ctypes.c_void_p * max(n, 1))(*([d.data_ptr() for d in dCs] or [0]))
    _check(load_library().se2_backward(plan.handle, _ptr(grad_out), _ptr(f), B, _ptr(C), _ptr(log_scale), n,
                                       dp if n else None, _ptr(gp) if n else None, _ptr(gf),
                                       _stream(grad_out.device)))
    return gf, gp[:n]


def sample_radial_gaussian(plan: Plan, sigma: float, sigma_theta: float, nu: float = 0.0, derivs: bool = False):
    """The radial Gaussian x wrapped-normal kernel on the plan's grid
    ([1, M, N, N]); with derivs=True also d/dsigma and d/dsigma_theta."""
    dev = torch.device("cuda", plan.device)
    shape = plan.grid_shape(1)
    P = torch.empty(shape, dtype=plan.dtype, device=dev)
    dPs = torch.empty(shape, dtype=plan.dtype, device=dev) if derivs else None
    dPt = torch.empty(shape, dtype=plan.dtype, device=dev) if derivs else None
    _check(load_library().se2_sample_radial_gaussian(plan.handle, float(sigma), float(sigma_theta), float(nu),
                                                     _ptr(P), _ptr(dPs), _ptr(dPt), _stream(dev)))
    return (P, dPs, dPt) if derivs else P


def _host_doubles(vals, n: int, name: str):
    if len(vals) != n:
        raise ValueError(f"{name} needs {n} values")
    return (ctypes.c_double * n)(*[float(v) for v in vals])


def _sigma_list(Sigma, sigma2):
    if (Sigma is None) == (sigma2 is None):
        raise ValueError("give exactly one of Sigma and sigma2")
    if Sigma is None:
        return [float(sigma2) if r == c else 0.0 for r in range(3) for c in range(3)]
    return [float(v) for row in Sigma for v in row]


def sample_se2_gaussian(plan, beta=(0.0, 0.0, 0.0), Sigma=None, sigma2: float | None = None, images: int = 1):
    """The Gaussian on SE(2) (Eq. fbS) with mean beta = (b1, b2, nu) and
    covariance Sigma (3x3), or Sigma = sigma2 * I (the kernel of Eq. gbS0
    shifted by nu), sampled on the plan's grid: [1, M, N, N] for a Plan,
    [1, Lr, Ly, Lx] (Omega_L) for a GridPlan."""
    S = _sigma_list(Sigma, sigma2)
    dev = torch.device("cuda", plan.device)
    grid = isinstance(plan, GridPlan)
    P = torch.empty(plan.sample_shape(1) if grid else plan.grid_shape(1), dtype=plan.dtype, device=dev)
    lib = load_library()
    fn = lib.se2_grid_sample_se2_gaussian if grid else lib.se2_sample_se2_gaussian
    _check(fn(plan.handle, _host_doubles(list(beta), 3, "beta"), _host_doubles(S, 9, "Sigma"), int(images), _ptr(P),
              _stream(dev)))
    return P


def sample_deformed_gaussian(plan, H, nu: float, s: float, images: int = 1):
    """The 3D deformed Gaussian exp(-x^T H x) exp(-(theta - nu)^2 / s)
    (Eq. fHsnu) on the plan's grid ([1, M, N, N], or [1, Lr, Ly, Lx] for a
    GridPlan)."""
    Hs = [float(v) for row in H for v in row]
    dev = torch.device("cuda", plan.device)
    grid = isinstance(plan, GridPlan)
    P = torch.empty(plan.sample_shape(1) if grid else plan.grid_shape(1), dtype=plan.dtype, device=dev)
    lib = load_library()
    fn = lib.se2_grid_sample_deformed_gaussian if grid else lib.se2_sample_deformed_gaussian
    _check(fn(plan.handle, _host_doubles(Hs, 4, "H"), float(nu), float(s), int(images), _ptr(P), _stream(dev)))
    return P


class GridPlan:
    """Odd sampling grid L = (Lx, Ly, Lr) (each 2K+1) with output on the
    N-grid N = (Nx, Ny, Nr) >= L (se2_grid_plan_create)."""

    def __init__(self, L: Sequence[int], N: Optional[Sequence[int]] = None, batch: int = 1,
                 precision: str = "f32", flags: int = 0, device: Optional[int] = None):
        lib = load_library()
        if precision not in ("f32", "f64"):
            raise ValueError("precision must be 'f32' or 'f64'")
        N = tuple(L) if N is None else tuple(N)
        if len(L) != 3 or len(N) != 3:
            raise ValueError("L and N need three sizes (x, y, theta)")
        self.Lx, self.Ly, self.Lr = (int(v) for v in L)
        self.Nx, self.Ny, self.Nr = (int(v) for v in N)
        self.Hx = (self.Lx - 1) // 2 + 1
        self.batch, self.flags, self.precision = batch, flags, precision
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.cdtype = torch.complex128 if precision == "f64" else torch.complex64
        h = ctypes.c_void_p()
        _check(lib.se2_grid_plan_create(ctypes.byref(h), (ctypes.c_int * 3)(self.Lx, self.Ly, self.Lr),
                                        (ctypes.c_int * 3)(self.Nx, self.Ny, self.Nr), batch,
                                        _PRECISIONS[precision], flags, self.device))
        self._h = h

    @property
    def handle(self):
        return self._h

    def launches(self) -> int:
        return int(load_library().se2_grid_plan_launches(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().se2_grid_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample_shape(self, B: int):
        return (B, self.Lr, self.Ly, self.Lx)

    def out_shape(self, B: int):
        return (B, self.Nr, self.Ny, self.Nx)

    def spec_shape(self, B: int):
        return (B, self.Lr, self.Ly, self.Hx)

    def _check_tensor(self, t: torch.Tensor, name: str, shape_tail, dtype) -> int:
        if t.dim() != 4 or tuple(t.shape[1:]) != tuple(shape_tail):
            raise ValueError(f"{name}: expected [B, {', '.join(map(str, shape_tail))}], got {tuple(t.shape)}")
        if t.dtype != dtype or not t.is_cuda or t.device.index != self.device or not t.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {dtype} tensor on cuda:{self.device}")
        return t.shape[0]


def grid_coeffs(plan: GridPlan, samples: torch.Tensor) -> torch.Tensor:
    """C = DFT(P)/|L| of [n, Lr, Ly, Lx] real samples: [n, Lr, Ly, Kx+1] complex."""
    n = plan._check_tensor(samples, "samples", plan.sample_shape(1)[1:], plan.dtype)
    C = torch.empty(plan.spec_shape(n), dtype=plan.cdtype, device=samples.device)
    _check(load_library().se2_grid_coeffs(plan.handle, _ptr(samples), n, _ptr(C), _stream(samples.device)))
    return C


def grid_convolve_chain(plan: GridPlan, f: torch.Tensor, Cs: Sequence[torch.Tensor],
                        out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Re S_K[f, rho_1..rho_k] on the N-grid ([B, Nr, Ny, Nx]); k = 0 gives the
    finite Fourier series S_K[f] itself."""
    B = plan._check_tensor(f, "f", plan.sample_shape(1)[1:], plan.dtype)
    if out is None:
        out = torch.empty(plan.out_shape(B), dtype=plan.dtype, device=f.device)
    else:
        plan._check_tensor(out, "out", plan.out_shape(1)[1:], plan.dtype)
    nb = 1 if plan.flags & SHARED_KERNEL else B
    for i, C in enumerate(Cs):
        plan._check_tensor(C, f"coeffs[{i}]", plan.spec_shape(1)[1:], plan.cdtype)
        if C.shape[0] != nb:
            raise ValueError(f"coeffs[{i}]: expected {nb} arrays, got {C.shape[0]}")
    k = len(Cs)
    cp = (ctypes.c_void_p * max(k, 1))(*[C.data_ptr() for C in Cs])
    _check(load_library().se2_grid_convolve_chain(plan.handle, _ptr(f), B, cp if k else None, k, _ptr(out),
                                                  _stream(f.device)))
    return out


def grid_convolve_chain_all(plan: GridPlan, f: torch.Tensor, Cs: Sequence[torch.Tensor],
                            out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Every V_p = Re S_K[f, rho_1..rho_p], p = 1..k, on the N-grid from one
    forward transform (Algorithm 6): returns [k, B, Nr, Ny, Nx]."""
    B = plan._check_tensor(f, "f", plan.sample_shape(1)[1:], plan.dtype)
    k = len(Cs)
    if k < 1:
        raise ValueError("need at least one kernel")
    shape = (k,) + plan.out_shape(B)
    if out is None:
        out = torch.empty(shape, dtype=plan.dtype, device=f.device)
    elif tuple(out.shape) != shape or out.dtype != plan.dtype or not out.is_contiguous():
        raise ValueError(f"out: need a contiguous {plan.dtype} tensor {shape}")
    nb = 1 if plan.flags & SHARED_KERNEL else B
    for i, C in enumerate(Cs):
        plan._check_tensor(C, f"coeffs[{i}]", plan.spec_shape(1)[1:], plan.cdtype)
        if C.shape[0] != nb:
            raise ValueError(f"coeffs[{i}]: expected {nb} arrays, got {C.shape[0]}")
    cp = (ctypes.c_void_p * k)(*[C.data_ptr() for C in Cs])
    _check(load_library().se2_grid_convolve_chain_all(plan.handle, _ptr(f), B, cp, k, _ptr(out), _stream(f.device)))
    return out


def accuracy_order(eps: float, grad_inf: float, k=(0, 0, 0), constant: float = 32.0) -> int:
    """Algorithm 1: the smallest K with K >= max(constant ||grad f||_inf / eps,
    ||k||_inf); f^[k; 2K+1] is then within eps of f^[k] (Theorem fkLmain)."""
    K = ctypes.c_longlong()
    _check(load_library().se2_accuracy_order(float(eps), float(grad_inf), int(max(abs(int(v)) for v in k)),
                                             float(constant), ctypes.byref(K)))
    return int(K.value)


def ffc_at(plan: GridPlan, C: torch.Tensor, k, index: int = 0) -> complex:
    """f^[k; L] = (-1)^(k1+k2) C(tau(k)) (Eq. FkLv) read from grid coefficients
    C = DFT(P)/|L| ([n, Lr, Ly, Kx+1]) of real samples by se2_grid_ffc_at;
    k = (k1, k2, k3) with |k_i| <= K_i (negative k1: the Hermitian partner)."""
    k1, k2, k3 = (int(v) for v in k)
    out = torch.empty(2, dtype=torch.float64, device=C.device)
    _check(load_library().se2_grid_ffc_at(plan.handle, _ptr(C), int(index), k1, k2, k3, _ptr(out),
                                          _stream(C.device)))
    re, im = out.cpu().tolist()
    return complex(re, im)


def ffc_convergence(sample, k, Ks, precision: str = "f64", device: Optional[int] = None):
    """FFC convergence report (Corollary fkOK): f^[k; 2K+1] for each K in Ks,
    computed on the GPU from `sample(L)` ([Lr, Ly, Lx] samples on Omega_L,
    L = (2K+1,)*3).  Returns [(K, value, |value - previous value|)]."""
    out, prev = [], None
    for K in Ks:
        L = 2 * int(K) + 1
        plan = GridPlan((L, L, L), batch=1, precision=precision, device=device)
        dev = torch.device("cuda", plan.device)
        P = torch.as_tensor(sample((L, L, L)), dtype=plan.dtype).reshape(1, L, L, L).contiguous().to(dev)
        v = ffc_at(plan, grid_coeffs(plan, P), k)
        out.append((int(K), v, None if prev is None else abs(v - prev)))
        prev = v
        plan.close()
    return out


def alloc_stats():
    """(live, total) device allocations the library has made (se2_debug_alloc_stats)."""
    live, total = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load_library().se2_debug_alloc_stats(ctypes.byref(live), ctypes.byref(total)))
    return int(live.value), int(total.value)


def fail_alloc(n: int):
    """Make the n-th next device allocation of the library fail (0: off)."""
    _check(load_library().se2_debug_fail_alloc(int(n)))


def table_len(plan: Plan) -> int:
    return plan.N // 2 + 1 + plan.N + plan.M


def separable_tables(plan: Plan, params: torch.Tensor, k: torch.Tensor) -> torch.Tensor:
    """Factored chain coefficients (se2_separable_tables).  params: float64
    [B, kmax, 3] (sigma, sigma_theta, nu) on the plan's device; k: int32 [B]
    chain lengths.  Returns [B, N/2+1+N+M] complex."""
    if params.dim() != 3 or params.shape[2] != 3 or params.dtype != torch.float64 or not params.is_contiguous():
        raise ValueError("params: contiguous float64 [B, kmax, 3]")
    B, kmax = params.shape[0], params.shape[1]
    if k.dtype != torch.int32 or k.shape != (B,) or not k.is_contiguous():
        raise ValueError("k: contiguous int32 [B]")
    tab = torch.empty((B, table_len(plan)), dtype=plan.cdtype, device=params.device)
    _check(load_library().se2_separable_tables(plan.handle, _ptr(params), _ptr(k), kmax, B, _ptr(tab),
                                               _stream(params.device)))
    return tab


def convolve_separable(plan: Plan, f: torch.Tensor, tables: torch.Tensor, out: Optional[torch.Tensor] = None):
    """se2_convolve with factored coefficient tables."""
    B = plan._check_grid(f, "f")
    if out is None:
        out = torch.empty_like(f)
    else:
        plan._check_grid(out, "out")
    nt = 1 if plan.flags & SHARED_KERNEL else B
    if tables.shape != (nt, table_len(plan)) or tables.dtype != plan.cdtype or not tables.is_contiguous():
        raise ValueError(f"tables: expected contiguous {plan.cdtype} [{nt}, {table_len(plan)}]")
    _check(load_library().se2_convolve_separable(plan.handle, _ptr(f), B, _ptr(tables), _ptr(out),
                                                 _stream(f.device)))
    return out


class SE2Conv(torch.autograd.Function):
    """out = f * rho(sigma, sigma_theta) for a batch f [B, M, N, N] and the
    radial Gaussian x wrapped-normal kernel shared by the batch, differentiable
    in f and in params = tensor([sigma, sigma_theta]) (float64).  The plan must
    have the SHARED_KERNEL flag."""

    @staticmethod
    def _spectra(plan, params):
        """C, dC/dsigma, dC/dsigma_theta for params, cached on the plan: while
        the params tensor is unchanged (same storage and version counter) the
        spectra are reused without reading its values, so a step that trains
        only f neither synchronises nor resamples.  params may live on the CPU
        (no device read at all) or on the device (read when they change)."""
        key = (params.data_ptr(), params._version, params.device)
        cache = getattr(plan, "_se2conv_cache", None)
        if cache is not None and cache[0] == key:
            return cache[1]
        sigma, sigma_t = (float(v) for v in params.detach().cpu().tolist())
        P, dPs, dPt = sample_radial_gaussian(plan, sigma, sigma_t, 0.0, derivs=True)
        spectra = (coeffs(plan, P)[0], coeffs(plan, dPs)[0], coeffs(plan, dPt)[0])
        plan._se2conv_cache = (key, spectra)
        return spectra

    @staticmethod
    def forward(ctx, f, params, plan):
        if not plan.flags & SHARED_KERNEL:
            raise ValueError("SE2Conv needs a plan with SHARED_KERNEL")
        C, dCs, dCt = SE2Conv._spectra(plan, params)
        out = convolve(plan, f.contiguous(), C)
        ctx.plan = plan
        ctx.save_for_backward(f, C, dCs, dCt)
        ctx.params_dtype = params.dtype
        ctx.params_device = params.device
        return out

    @staticmethod
    def backward(ctx, grad_out):
        f, C, dCs, dCt = ctx.saved_tensors
        gf, gp = backward(ctx.plan, grad_out.contiguous(), C, f, [dCs, dCt],
                          want_grad_f=ctx.needs_input_grad[0])
        return gf, gp.to(ctx.params_device, ctx.params_dtype), None


__all__ = ["Plan", "SE2Error", "coeffs", "convolve", "convolve_host", "convolve_chain", "convolve_chain_all",
           "backward",
           "sample_radial_gaussian", "sample_se2_gaussian", "sample_deformed_gaussian",
           "GridPlan", "grid_coeffs", "grid_convolve_chain", "grid_convolve_chain_all", "accuracy_order", "ffc_at", "ffc_convergence",
           "SE2Conv", "separable_tables", "convolve_separable", "table_len", "load_library", "LIB_PATH",
           "SHARED_KERNEL", "PERSISTENT", "GRID_ORIGIN_ZERO", "MASS_RENORM",
           "KERNEL_YSYM", "HOST_STAGING", "CHECK_FINITE", "alloc_stats", "fail_alloc"]
