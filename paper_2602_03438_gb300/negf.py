"""ctypes binding of libnegf (include/negf.h): argument marshalling only.

Every arithmetic step of the path runs in the CUDA kernels of libnegf.so; this
module converts torch tensors to raw device pointers and back.  It refuses to
run without the compiled library (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libnegf.so")

NEGF_OK = 0
NEGF_ERR_ARG = -1
NEGF_ERR_CUDA = -2
NEGF_ERR_NOMEM = -3
NEGF_ERR_NOCONV = -4
NEGF_ERR_SINGULAR = -5
NEGF_ERR_TIMEOUT = -6
FP64 = 0
MIXED = 1
MIXED_TF32 = 2

EXPORTS = ["negf_ctx_create", "negf_ctx_destroy", "negf_last_error", "negf_ctx_sync", "negf_layout", "negf_worklist",
           "negf_obc", "negf_rgf_retarded", "negf_rgf_lesser", "negf_rgf_keldysh", "negf_rgf_partitioned",
           "negf_observables", "negf_energy_convolution", "negf_scba", "negf_rgf_observables",
           "negf_rgf_arrowhead",
           "negf_profile_enable",
           "negf_profile_read", "negf_profile_reset", "negf_block_gemm", "negf_block_inverse",
           "negf_block_gemm_noalloc", "negf_mlp_get_dims", "negf_mlp_workspace_bytes", "negf_mlp_pack",
           "negf_mlp_forward", "negf_mlp_train_step", "negf_sliced_digits", "negf_tune_products",
           "negf_set_product_variant", "negf_selftest_wait_timeout"]
KERNEL_CLASSES = ["gemm_tc", "gemm_f64", "inv_f32", "inv_f64", "other", "gemm_oz", "gemm_oz_lo"]


class NegfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libnegf status {code}: {msg}")
        self.code = code


class _System(C.Structure):
    _fields_ = [("ndev", C.c_int32), ("nb", C.POINTER(C.c_int32)), ("bs", C.POINTER(C.c_int32)),
                ("ne", C.POINTER(C.c_int32)), ("H_diag", C.c_void_p), ("H_up", C.c_void_p),
                ("S_diag", C.c_void_p), ("S_up", C.c_void_p), ("energy", C.c_void_p), ("eta", C.c_double)]


class MlpDims(C.Structure):
    """negf_mlp_dims (include/negf_warmstart.h)."""
    _fields_ = [("b", C.c_int32), ("hidden", C.c_int32), ("k0", C.c_int32), ("k0p", C.c_int32),
                ("nout", C.c_int32), ("off_W1", C.c_int64), ("off_c1", C.c_int64), ("off_W2", C.c_int64),
                ("off_c2", C.c_int64), ("off_W3", C.c_int64), ("off_c3", C.c_int64), ("n_params", C.c_int64)]


class _BosonKernel(C.Structure):
    _fields_ = [("M", C.c_int32), ("w_lesser", C.POINTER(C.c_double)), ("w_greater", C.POINTER(C.c_double))]


class _Scattering(C.Structure):
    _fields_ = [("sigR", C.c_void_p), ("sigL", C.c_void_p), ("sigL_scale", C.c_void_p),
                ("per_energy", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libnegf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libnegf.so not found at {path}: run __graft_entry__.build() first")
    lib = C.CDLL(path)
    vp, i32, dbl, sz = C.c_void_p, C.c_int32, C.c_double, C.c_size_t
    lib.negf_ctx_create.argtypes = [C.POINTER(vp), C.c_int, sz]
    lib.negf_ctx_destroy.argtypes = [vp]
    lib.negf_last_error.argtypes = [vp]
    lib.negf_last_error.restype = C.c_char_p
    lib.negf_ctx_sync.argtypes = [vp, vp]
    lib.negf_layout.argtypes = [C.POINTER(_System), C.POINTER(C.c_int64)]
    lib.negf_worklist.argtypes = [C.POINTER(_System), i32, C.POINTER(i32), vp, vp, vp, vp]
    lib.negf_obc.argtypes = [vp, C.POINTER(_System), C.c_int, dbl, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.negf_mlp_get_dims.argtypes = [i32, i32, C.POINTER(MlpDims)]
    lib.negf_mlp_workspace_bytes.argtypes = [C.POINTER(MlpDims), i32]
    lib.negf_mlp_workspace_bytes.restype = sz
    lib.negf_mlp_pack.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.negf_mlp_forward.argtypes = [vp, C.POINTER(MlpDims), vp, i32, vp, vp, vp]
    lib.negf_mlp_train_step.argtypes = [vp, C.POINTER(MlpDims), vp, vp, vp, vp, i32, C.c_float, i32, vp, i32, vp,
                                        vp, vp, i32, vp]
    lib.negf_rgf_retarded.argtypes = [vp, C.POINTER(_System), C.c_int, vp, vp, C.POINTER(_Scattering),
                                      vp, vp, vp, vp, vp]
    lib.negf_rgf_lesser.argtypes = [vp, C.POINTER(_System), C.c_int, vp, vp, vp, vp, C.POINTER(_Scattering),
                                    vp, vp, vp, vp, vp, vp, vp]
    lib.negf_rgf_partitioned.argtypes = [vp, C.POINTER(_System), C.c_int, i32, vp, vp, C.POINTER(_Scattering),
                                         vp, vp, vp, vp, vp]
    lib.negf_rgf_arrowhead.argtypes = [vp, C.POINTER(_System), C.c_int, vp, vp, vp, vp, C.POINTER(_Scattering),
                                       vp, vp, vp, vp, vp, vp, vp, vp]
    lib.negf_rgf_observables.argtypes = [vp, C.POINTER(_System), C.c_int, vp, vp, vp, vp, C.POINTER(_Scattering),
                                         vp, vp, vp, vp, vp, vp, vp]
    lib.negf_energy_convolution.argtypes = [vp, i32, C.c_int64, C.c_int64, i32, C.POINTER(C.c_double), vp, vp, vp]
    lib.negf_scba.argtypes = [vp, C.POINTER(_System), C.c_int, vp, vp, vp, vp, C.POINTER(_BosonKernel), dbl, dbl,
                              i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(i32), C.POINTER(dbl), vp]
    lib.negf_rgf_keldysh.argtypes = [vp, C.POINTER(_System), C.c_int, vp, vp, vp, vp, C.POINTER(_Scattering),
                                     vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.negf_observables.argtypes = [vp, C.POINTER(_System), i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.negf_block_gemm.argtypes = [vp, C.c_int, i32, i32, i32, i32, vp, vp, C.c_int64, vp, C.c_int64, vp, vp,
                                    C.c_int64, vp, C.c_int64, vp]
    lib.negf_block_inverse.argtypes = [vp, C.c_int, i32, i32, vp, vp, vp, vp]
    lib.negf_block_gemm_noalloc.argtypes = [i32, i32, i32, i32, vp, vp, C.c_int64, vp, C.c_int64, vp, vp,
                                            C.c_int64, vp, C.c_int64, vp, vp]
    lib.negf_profile_enable.argtypes = [vp, C.c_int]
    lib.negf_profile_read.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.negf_profile_reset.argtypes = [vp]
    lib.negf_sliced_digits.argtypes = []
    lib.negf_tune_products.argtypes = [vp, i32, i32, C.POINTER(i32), C.POINTER(dbl), vp]
    lib.negf_set_product_variant.argtypes = [vp, i32, i32]
    lib.negf_selftest_wait_timeout.argtypes = [vp, C.c_int64, vp]
    for name in EXPORTS:
        if name not in ("negf_last_error", "negf_mlp_workspace_bytes"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libnegf takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libnegf takes contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """A libnegf context bound to one CUDA device with its own workspace."""

    def __init__(self, device: int = 0, workspace_bytes: int = 1 << 30):
        self.lib = load_library()
        self.h = C.c_void_p()
        st = self.lib.negf_ctx_create(C.byref(self.h), int(device), C.c_size_t(int(workspace_bytes)))
        if st != NEGF_OK:
            raise NegfError(st, self.lib.negf_last_error(None).decode())
        self.device = device

    def close(self):
        if self.h:
            self.lib.negf_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        if st != NEGF_OK:
            raise NegfError(st, self.lib.negf_last_error(self.h).decode())

    def profile(self, enable: bool):
        self.check(self.lib.negf_profile_enable(self.h, 1 if enable else 0))

    def profile_reset(self):
        self.check(self.lib.negf_profile_reset(self.h))

    def profile_read(self) -> dict:
        """Kernel launches and per-class event timings accumulated since the last reset."""
        n = len(KERNEL_CLASSES)
        tot = C.c_int64()
        kl = (C.c_int64 * n)()
        ms = (C.c_double * n)()
        fl = (C.c_double * n)()
        by = (C.c_double * n)()
        self.check(self.lib.negf_profile_read(self.h, C.byref(tot), kl, ms, fl, by))
        return dict(launches=int(tot.value),
                    classes={k: dict(launches=int(kl[i]), ms=float(ms[i]), flops=float(fl[i]), bytes=float(by[i]))
                             for i, k in enumerate(KERNEL_CLASSES)})

    def sync(self, stream=None) -> int:
        """Synchronize the stream; returns the worst device-side status (0 = OK)."""
        return int(self.lib.negf_ctx_sync(self.h, _stream(stream)))

    def selftest_wait_timeout(self, wait_ns: int, stream=None):
        """Launch the failure-detection self test: one bounded device wait that runs
        out after wait_ns and raises NEGF_ERR_TIMEOUT (read it with sync())."""
        self.check(self.lib.negf_selftest_wait_timeout(self.h, int(wait_ns), _stream(stream)))


@dataclass
class System:
    """Device-resident packed batch of BT devices (the negf_system of the C ABI)."""
    nb: List[int]
    bs: List[int]
    ne: List[int]
    H_diag: torch.Tensor
    H_up: torch.Tensor
    S_diag: Optional[torch.Tensor]
    S_up: Optional[torch.Tensor]
    energy: torch.Tensor
    eta: float
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _System:
        n = len(self.nb)
        arrs = [(C.c_int32 * n)(*self.nb), (C.c_int32 * n)(*self.bs), (C.c_int32 * n)(*self.ne)]
        self._keep = arrs
        return _System(n, arrs[0], arrs[1], arrs[2], _ptr(self.H_diag), _ptr(self.H_up),
                       _ptr(self.S_diag), _ptr(self.S_up), _ptr(self.energy), float(self.eta))

    @property
    def ndev(self):
        return len(self.nb)

    def layout(self) -> np.ndarray:
        """Integer offsets of the packing, [ndev+1, 8] (see negf_layout)."""
        lib = load_library()
        out = (C.c_int64 * (8 * (self.ndev + 1)))()
        s = self.c()
        st = lib.negf_layout(C.byref(s), out)
        if st != NEGF_OK:
            raise NegfError(st, lib.negf_last_error(None).decode())
        return np.frombuffer(out, dtype=np.int64).reshape(self.ndev + 1, 8).copy()


def system_layout(nb: Sequence[int], bs: Sequence[int], ne: Sequence[int]) -> np.ndarray:
    """negf_layout for shapes only (no device memory touched)."""
    lib = load_library()
    n = len(nb)
    arrs = [(C.c_int32 * n)(*nb), (C.c_int32 * n)(*bs), (C.c_int32 * n)(*ne)]
    s = _System(n, arrs[0], arrs[1], arrs[2], None, None, None, None, None, 1.0)
    out = (C.c_int64 * (8 * (n + 1)))()
    st = lib.negf_layout(C.byref(s), out)
    if st != NEGF_OK:
        raise NegfError(st, lib.negf_last_error(None).decode())
    return np.frombuffer(out, dtype=np.int64).reshape(n + 1, 8).copy()


def system_worklist(nb: Sequence[int], bs: Sequence[int], ne: Sequence[int], block_size: int) -> dict:
    """negf_worklist for shapes only: the (device, energy) units of the devices with
    `block_size` and their output offsets (host arrays)."""
    lib = load_library()
    n = len(nb)
    arrs = [(C.c_int32 * n)(*nb), (C.c_int32 * n)(*bs), (C.c_int32 * n)(*ne)]
    s = _System(n, arrs[0], arrs[1], arrs[2], None, None, None, None, None, 1.0)
    cnt = C.c_int32(0)
    st = lib.negf_worklist(C.byref(s), int(block_size), C.byref(cnt), None, None, None, None)
    if st != NEGF_OK:
        raise NegfError(st, lib.negf_last_error(None).decode())
    k = cnt.value
    out = dict(unit_dev=np.zeros(k, np.int32), unit_e=np.zeros(k, np.int32), off_d=np.zeros(k, np.int64),
               off_o=np.zeros(k, np.int64))
    st = lib.negf_worklist(C.byref(s), int(block_size), C.byref(cnt),
                           *(C.c_void_p(out[key].ctypes.data) for key in ("unit_dev", "unit_e", "off_d", "off_o")))
    if st != NEGF_OK:
        raise NegfError(st, lib.negf_last_error(None).decode())
    return out


def _dev_tensor(a, device, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device)


def upload(devices, device="cuda") -> System:
    """Pack one or several ``workloads.Device`` objects onto the GPU."""
    if not isinstance(devices, (list, tuple)):
        devices = [devices]
    eta = devices[0].eta
    if any(d.eta != eta for d in devices):
        raise ValueError("all devices of a batch share eta")
    flat = lambda xs: np.concatenate([x.reshape(-1) for x in xs]) if xs else np.zeros(0, np.complex128)
    has_s = [d.S_diag is not None for d in devices]
    if any(has_s) and not all(has_s):
        raise ValueError("either every device has an overlap matrix or none")
    Hd = _dev_tensor(flat([d.H_diag for d in devices]), device)
    Hu = _dev_tensor(flat([d.H_up for d in devices]), device)
    Sd = _dev_tensor(flat([d.S_diag for d in devices]), device) if all(has_s) else None
    Su = _dev_tensor(flat([d.S_up for d in devices]), device) if all(has_s) else None
    E = _dev_tensor(np.concatenate([d.energy for d in devices]), device)
    return System([d.nb for d in devices], [d.b for d in devices], [d.ne for d in devices],
                  Hd, Hu if Hu.numel() else None, Sd, Su, E, eta)


class Scattering:
    """Block-diagonal scattering self-energies (negf_scattering)."""

    def __init__(self, sigR=None, sigL=None, sigL_scale=None, per_energy=False):
        self.sigR, self.sigL, self.sigL_scale, self.per_energy = sigR, sigL, sigL_scale, per_energy

    def c(self):
        return _Scattering(_ptr(self.sigR), _ptr(self.sigL), _ptr(self.sigL_scale), 1 if self.per_energy else 0)

    @staticmethod
    def from_devices(devices, device="cuda"):
        if not isinstance(devices, (list, tuple)):
            devices = [devices]
        if all(d.sigR_scat is None and d.sigL_base is None for d in devices):
            return None
        cat = lambda xs: np.concatenate([x.reshape(-1) for x in xs])
        sR = _dev_tensor(cat([d.sigR_scat for d in devices]), device) if devices[0].sigR_scat is not None else None
        sL = _dev_tensor(cat([d.sigL_base for d in devices]), device) if devices[0].sigL_base is not None else None
        sc = (_dev_tensor(cat([d.sigL_scale for d in devices]), device)
              if devices[0].sigL_scale is not None else None)
        return Scattering(sR, sL, sc, False)


def _scat_ptr(scat):
    return C.byref(scat.c()) if scat is not None else None


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def negf_obc(ctx: Context, sys: System, sigma_L, sigma_R, iters=None, status=None, tol=1e-12, max_iter=100,
             stream=None, g0_L=None, g0_R=None, gs_L=None, gs_R=None, newton=None, prec=FP64):
    s = sys.c()
    ctx.check(ctx.lib.negf_obc(ctx.h, C.byref(s), int(prec), float(tol), int(max_iter), _ptr(g0_L), _ptr(g0_R),
                               _ptr(sigma_L), _ptr(sigma_R), _ptr(gs_L), _ptr(gs_R), _ptr(iters), _ptr(newton),
                               _ptr(status), _stream(stream)))


def negf_rgf_retarded(ctx: Context, sys: System, prec, sigma_L, sigma_R, scat=None, GR_diag=None, GR_up=None,
                      GR_low=None, status=None, stream=None):
    s = sys.c()
    sc = scat.c() if scat is not None else None
    ctx.check(ctx.lib.negf_rgf_retarded(ctx.h, C.byref(s), int(prec), _ptr(sigma_L), _ptr(sigma_R),
                                        C.byref(sc) if sc is not None else None, _ptr(GR_diag), _ptr(GR_up),
                                        _ptr(GR_low), _ptr(status), _stream(stream)))


def negf_rgf_lesser(ctx: Context, sys: System, prec, sigma_L, sigma_R, f_L, f_R, scat=None, GR_diag=None,
                    GR_up=None, GR_low=None, GL_diag=None, GL_low=None, status=None, stream=None):
    s = sys.c()
    sc = scat.c() if scat is not None else None
    ctx.check(ctx.lib.negf_rgf_lesser(ctx.h, C.byref(s), int(prec), _ptr(sigma_L), _ptr(sigma_R), _ptr(f_L),
                                      _ptr(f_R), C.byref(sc) if sc is not None else None, _ptr(GR_diag),
                                      _ptr(GR_up), _ptr(GR_low), _ptr(GL_diag), _ptr(GL_low), _ptr(status),
                                      _stream(stream)))


def negf_rgf_partitioned(ctx: Context, sys: System, prec, P: int, sigma_L, sigma_R, scat=None, GR_diag=None,
                         GR_up=None, GR_low=None, status=None, stream=None):
    s = sys.c()
    sc = scat.c() if scat is not None else None
    ctx.check(ctx.lib.negf_rgf_partitioned(ctx.h, C.byref(s), int(prec), int(P), _ptr(sigma_L), _ptr(sigma_R),
                                           C.byref(sc) if sc is not None else None, _ptr(GR_diag), _ptr(GR_up),
                                           _ptr(GR_low), _ptr(status), _stream(stream)))


def negf_rgf_arrowhead(ctx: Context, sys: System, prec, H_tip, H_arrow, sigma_L, sigma_R, scat=None, GR_diag=None,
                       GR_up=None, GR_low=None, G_tip=None, G_row=None, G_col=None, status=None, stream=None):
    s = sys.c()
    sc = scat.c() if scat is not None else None
    ctx.check(ctx.lib.negf_rgf_arrowhead(ctx.h, C.byref(s), int(prec), _ptr(H_tip), _ptr(H_arrow), _ptr(sigma_L),
                                         _ptr(sigma_R), C.byref(sc) if sc is not None else None, _ptr(GR_diag),
                                         _ptr(GR_up), _ptr(GR_low), _ptr(G_tip), _ptr(G_row), _ptr(G_col),
                                         _ptr(status), _stream(stream)))


def negf_rgf_observables(ctx: Context, sys: System, prec, sigma_L, sigma_R, f_L, f_R, scat=None, e_weight=None,
                         T=None, dos=None, current=None, density=None, status=None, stream=None):
    s = sys.c()
    sc = scat.c() if scat is not None else None
    ctx.check(ctx.lib.negf_rgf_observables(ctx.h, C.byref(s), int(prec), _ptr(sigma_L), _ptr(sigma_R), _ptr(f_L),
                                           _ptr(f_R), C.byref(sc) if sc is not None else None, _ptr(e_weight),
                                           _ptr(T), _ptr(dos), _ptr(current), _ptr(density), _ptr(status),
                                           _stream(stream)))


def negf_energy_convolution(ctx: Context, X, Y, w, ne=None, stream=None):
    """Eq. (3) along the first axis of X ([ne, ...] complex128 device tensor) into Y."""
    ne = X.shape[0] if ne is None else ne
    nelem = X[0].numel() if X.dim() > 1 else 1
    wa = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    M = (wa.size - 1) // 2
    ctx.check(ctx.lib.negf_energy_convolution(ctx.h, int(ne), int(nelem), int(nelem), int(M),
                                              wa.ctypes.data_as(C.POINTER(C.c_double)), _ptr(X), _ptr(Y),
                                              _stream(stream)))


def negf_scba(ctx: Context, sys: System, prec, sigma_L, sigma_R, f_L, f_R, w_lesser, w_greater, sigR, sigL, sigG,
              GR_diag, GL_diag, GG_diag, GR_up=None, GR_low=None, GL_low=None, GG_low=None, status=None,
              mixing=0.5, tol=1e-8, max_iter=100, stream=None):
    """The self-consistent scattering loop; returns (sweeps, last change)."""
    s = sys.c()
    wl = np.ascontiguousarray(np.asarray(w_lesser, dtype=np.float64))
    wg = np.ascontiguousarray(np.asarray(w_greater, dtype=np.float64))
    if wl.size != wg.size or wl.size % 2 == 0:
        raise ValueError("kernels of equal odd length 2M+1")
    k = _BosonKernel((wl.size - 1) // 2, wl.ctypes.data_as(C.POINTER(C.c_double)),
                     wg.ctypes.data_as(C.POINTER(C.c_double)))
    it = C.c_int32(0)
    ch = C.c_double(0.0)
    ctx.check(ctx.lib.negf_scba(ctx.h, C.byref(s), int(prec), _ptr(sigma_L), _ptr(sigma_R), _ptr(f_L), _ptr(f_R),
                                C.byref(k), float(mixing), float(tol), int(max_iter), _ptr(sigR), _ptr(sigL),
                                _ptr(sigG), _ptr(GR_diag), _ptr(GR_up), _ptr(GR_low), _ptr(GL_diag), _ptr(GL_low),
                                _ptr(GG_diag), _ptr(GG_low), _ptr(status), C.byref(it), C.byref(ch),
                                _stream(stream)))
    return int(it.value), float(ch.value)


def negf_rgf_keldysh(ctx: Context, sys: System, prec, sigma_L, sigma_R, f_L, f_R, scat=None, GR_diag=None,
                     GR_up=None, GR_low=None, GL_diag=None, GL_low=None, GG_diag=None, GG_low=None, status=None,
                     stream=None):
    s = sys.c()
    sc = scat.c() if scat is not None else None
    ctx.check(ctx.lib.negf_rgf_keldysh(ctx.h, C.byref(s), int(prec), _ptr(sigma_L), _ptr(sigma_R), _ptr(f_L),
                                       _ptr(f_R), C.byref(sc) if sc is not None else None, _ptr(GR_diag),
                                       _ptr(GR_up), _ptr(GR_low), _ptr(GL_diag), _ptr(GL_low), _ptr(GG_diag),
                                       _ptr(GG_low), _ptr(status), _stream(stream)))


def negf_observables(ctx: Context, sys: System, sigma_L=None, e_weight=None, GR_diag=None, GR_up=None,
                     GR_low=None, GL_diag=None, GL_low=None, T=None, dos=None, current=None, density=None,
                     stream=None, prec: int = FP64):
    s = sys.c()
    ctx.check(ctx.lib.negf_observables(ctx.h, C.byref(s), int(prec), _ptr(sigma_L), _ptr(e_weight), _ptr(GR_diag),
                                       _ptr(GR_up), _ptr(GR_low), _ptr(GL_diag), _ptr(GL_low), _ptr(T), _ptr(dos),
                                       _ptr(current), _ptr(density), _stream(stream)))


# ---------------------------------------------------------------------------
# output allocation helper (torch is the allocator)
# ---------------------------------------------------------------------------

def allocate_outputs(sys: System, lesser=True, device="cuda", want_up_low=True, greater=False):
    L = sys.layout()
    tot = L[-1]
    z = lambda n: torch.empty(int(n), dtype=torch.complex128, device=device)
    out = dict(
        sigma_L=z(tot[3]), sigma_R=z(tot[3]),
        iters=torch.zeros(2 * int(tot[2]), dtype=torch.int32, device=device),
        obc_status=torch.zeros(int(tot[2]), dtype=torch.int32, device=device),
        status=torch.zeros(int(tot[2]), dtype=torch.int32, device=device),
        GR_diag=z(tot[4]),
        GR_up=z(tot[5]) if want_up_low else None,
        GR_low=z(tot[5]) if want_up_low else None,
        T=torch.zeros(int(tot[2]), dtype=torch.float64, device=device),
        dos=torch.zeros(int(tot[2]), dtype=torch.float64, device=device),
    )
    if lesser:
        out.update(GL_diag=z(tot[4]), GL_low=z(tot[5]),
                   current=torch.zeros(int(tot[6]), dtype=torch.float64, device=device),
                   density=torch.zeros(int(tot[7]), dtype=torch.float64, device=device))
        if greater:
            out.update(GG_diag=z(tot[4]), GG_low=z(tot[5]))
    return out


def negf_block_gemm(ctx: Context, prec, A, B, D, opA=0, opB=0, alpha=1.0, beta=0.0, C_=None, stream=None):
    """Batched D[u] = alpha op(A[u]) op(B[u]) + beta C[u] on [units, n, n] complex128 tensors
    (a [n, n] tensor is shared by all units)."""
    n = D.shape[-1]
    units = D.shape[0] if D.dim() == 3 else 1
    st = lambda t: 0 if t.dim() == 2 else n * n
    al = (C.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (C.c_double * 2)(complex(beta).real, complex(beta).imag)
    ctx.check(ctx.lib.negf_block_gemm(ctx.h, int(prec), n, units, int(opA), int(opB), al, _ptr(A), st(A), _ptr(B),
                                      st(B), be, _ptr(C_), st(C_) if C_ is not None else 0, _ptr(D), st(D),
                                      _stream(stream)))


def negf_block_inverse(ctx: Context, prec, M, X, status=None, stream=None):
    """Batched X[u] = M[u]^{-1} on [units, n, n] complex128 tensors."""
    n = M.shape[-1]
    units = M.shape[0] if M.dim() == 3 else 1
    ctx.check(ctx.lib.negf_block_inverse(ctx.h, int(prec), n, units, _ptr(M), _ptr(X), _ptr(status),
                                         _stream(stream)))


def sliced_digits() -> int:
    """Digits per value of the NEGF_MIXED sliced product in the loaded build."""
    return int(load_library().negf_sliced_digits())


def negf_block_gemm_noalloc(A, B, D, opA=0, opB=0, alpha=1.0, beta=0.0, C_=None, status=None, stream=None):
    """The NEGF_MIXED block product without a context or any allocation (static
    device scratch); same operands as negf_block_gemm."""
    lib = load_library()
    n = D.shape[-1]
    units = D.shape[0] if D.dim() == 3 else 1
    st = lambda t: 0 if t.dim() == 2 else n * n
    al = (C.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (C.c_double * 2)(complex(beta).real, complex(beta).imag)
    rc = lib.negf_block_gemm_noalloc(n, units, int(opA), int(opB), al, _ptr(A), st(A), _ptr(B), st(B), be,
                                     _ptr(C_), st(C_) if C_ is not None else 0, _ptr(D), st(D), _ptr(status),
                                     _stream(stream))
    if rc != NEGF_OK:
        raise NegfError(rc, lib.negf_last_error(None).decode())


# ---------------------------------------------------------------------------
# warm-start network (include/negf_warmstart.h)
# ---------------------------------------------------------------------------

def negf_mlp_get_dims(b: int, hidden: int = 512) -> MlpDims:
    lib = load_library()
    d = MlpDims()
    rc = lib.negf_mlp_get_dims(int(b), int(hidden), C.byref(d))
    if rc != NEGF_OK:
        raise NegfError(rc, lib.negf_last_error(None).decode())
    return d


def negf_mlp_workspace_bytes(dims: MlpDims, n: int) -> int:
    return int(load_library().negf_mlp_workspace_bytes(C.byref(dims), int(n)))


def mlp_rows(n: int) -> int:
    """Rows of the feature / activation buffers for n samples (multiple of 128)."""
    return (int(n) + 127) // 128 * 128


def negf_mlp_pack(ctx: Context, b: int, H00, H01, lead, E, X=None, stream=None):
    """Feature rows (BF16, returned as a torch.bfloat16 [NP, K0P] tensor) of the samples
    (lead[s], E[s]); H00/H01 are [nlead, b, b] complex128 device tensors."""
    n = int(lead.numel())
    d = negf_mlp_get_dims(b, 128)
    if X is None:
        X = torch.empty((mlp_rows(n), d.k0p), dtype=torch.bfloat16, device=lead.device)
    ctx.check(ctx.lib.negf_mlp_pack(ctx.h, int(b), n, int(H00.shape[0]), _ptr(H00), _ptr(H01), _ptr(lead),
                                    _ptr(E), _ptr(X), _stream(stream)))
    return X


def negf_mlp_forward(ctx: Context, dims: MlpDims, params, n: int, X, g0=None, stream=None):
    if g0 is None:
        g0 = torch.empty((int(n), dims.b, dims.b), dtype=torch.complex128, device=params.device)
    ctx.check(ctx.lib.negf_mlp_forward(ctx.h, C.byref(dims), _ptr(params), int(n), _ptr(X), _ptr(g0),
                                       _stream(stream)))
    return g0


def negf_mlp_train_step(ctx: Context, dims: MlpDims, params, adam_m, adam_v, grad, step: int, lr: float, n: int, X,
                        g_target, loss, update: bool = True, rows=None, n_set: int = 0, stream=None):
    ctx.check(ctx.lib.negf_mlp_train_step(ctx.h, C.byref(dims), _ptr(params), _ptr(adam_m), _ptr(adam_v),
                                          _ptr(grad), int(step), float(lr), int(n), _ptr(rows), int(n_set), _ptr(X),
                                          _ptr(g_target), _ptr(loss), int(bool(update)), _stream(stream)))
