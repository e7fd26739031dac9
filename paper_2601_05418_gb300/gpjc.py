"""Python binding of the gpjc C ABI (include/gpjc.h).

Argument marshalling only: every step of the compression and reconstruction
runs in the CUDA kernels of libgpjc.so.  PyTorch supplies device memory and
the current stream.  Importing this module fails loudly when the library has
not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpjc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = C.CDLL(LIB_PATH)

GPJC_OK, GPJC_EINVAL, GPJC_ENOMEM, GPJC_ECUDA, GPJC_ETIMEOUT, GPJC_ENONFINITE, GPJC_EUNSUPPORTED = range(7)
FP32, BF16, FP16 = 0, 1, 2
CG, FISTA, DECOUPLED = 0, 1, 2
_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)


class GpjcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gpjc status {status} ({_lib.gpjc_strerror(status).decode()}): {msg}")
        self.status = status


class Geom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nc", C.c_int32), ("os", C.c_int32),
                ("w", C.c_int32), ("n_groups", C.c_int32), ("patch_group", _I32P), ("keep", _I32P),
                ("n_lines", C.c_int32), ("line_ky", _I32P), ("line_kz", _I32P),
                ("cycles", C.c_double), ("kappa_y", C.c_double), ("kappa_z", C.c_double)]


class BuildParams(C.Structure):
    _fields_ = [("eig_iters", C.c_int32), ("block", C.c_int32), ("keep_gram", C.c_int32),
                ("eig_iters_fp32", C.c_int32)]


class GroupsInfo(C.Structure):
    _fields_ = [("roi_pixels", C.c_int64), ("block", C.c_int32), ("max_residual", C.c_double)]


class ReconParams(C.Structure):
    _fields_ = [("alg", C.c_int32), ("iters", C.c_int32), ("lambda_", C.c_double), ("lipschitz", C.c_double),
                ("power_iters", C.c_int32), ("haar_levels", C.c_int32), ("use_x0", C.c_int32),
                ("use_graph", C.c_int32), ("lambda_tv", C.c_double), ("tv_eps", C.c_double)]


class ReconInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("lipschitz", C.c_double), ("h_history", C.POINTER(C.c_double))]


def _sig(name, args, res=C.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_lib.gpjc_strerror.argtypes = [C.c_int]
_lib.gpjc_strerror.restype = C.c_char_p
_sig("gpjc_last_error", [], C.c_char_p)
_sig("gpjc_version", [], C.c_char_p)
_sig("gpjc_plan_create", [C.POINTER(Geom), C.POINTER(_P)])
_sig("gpjc_plan_destroy", [_P], None)
_sig("gpjc_plan_ntx_c", [_P, _I32P])
_sig("gpjc_plan_sets", [_P, _I32P, _I32P])
_sig("gpjc_plan_tables", [_P, _I32P, _I32P, _I32P])
_sig("gpjc_build_groups", [_P, _P, _P, _P, C.POINTER(BuildParams), _P, C.POINTER(_P)])
_sig("gpjc_groups_rebuild", [_P, _P, _P, _P, _P])
_sig("gpjc_groups_from_matrices", [_P, _P, C.POINTER(_P)])
_sig("gpjc_launch_count", [], C.c_uint64)
_sig("gpjc_op_profile", [_P, C.c_int32])
_sig("gpjc_op_profile_read", [_P, C.c_int32, C.POINTER(C.c_double), _I32P])
_sig("gpjc_groups_destroy", [_P], None)
_sig("gpjc_groups_info_get", [_P, C.POINTER(GroupsInfo)])
_sig("gpjc_groups_get", [_P, _P, _P])
_sig("gpjc_keep_from_energy", [_P, C.c_int32, C.c_int32, _P, C.c_double, _P])
_sig("gpjc_tv_grad", [_P, C.c_int32, C.c_int32, C.c_int32, C.c_double, _P, _P])
_sig("gpjc_groups_gram", [_P, _P])
_sig("gpjc_groups_roi", [_P, _I32P])
_sig("gpjc_compress", [_P, _P, _P, C.c_int, _P])
_sig("gpjc_op_create", [_P, _P, C.c_int, C.c_int32, C.POINTER(_P)])
_sig("gpjc_op_destroy", [_P], None)
_sig("gpjc_op_autotune", [_P, _P, _I32P])
_sig("gpjc_apply_E", [_P, _P, _P, _P])
_sig("gpjc_apply_EH", [_P, _P, _P, _P])
_sig("gpjc_apply_normal", [_P, _P, _P, _P, _P])
_sig("gpjc_simulate", [_P, _P, _P, _P])
_sig("gpjc_simulate_adjoint", [_P, _P, _P, _P])
_sig("gpjc_recon", [_P, _P, _P, C.POINTER(ReconParams), C.POINTER(ReconInfo), _P])
_sig("gpjc_apply_EH_static", [_P, _P, _P, _P, _P])
_sig("gpjc_query", [_P, C.c_int32, C.c_int32, _I32P, C.POINTER(C.c_uint64)])
_sig("gpjc_debug_fail_allocations", [C.c_int64], None)
_sig("gpjc_probe_fp32_tflops", [C.c_int32, C.POINTER(C.c_double)])
_sig("gpjc_op_create_local_b0", [_P, _P, C.c_int32, _P, _P, C.POINTER(_P)])
_sig("gpjc_multi_create", [C.c_int32, C.POINTER(_P), C.c_int32, C.POINTER(_P)])
_sig("gpjc_op_tuning", [_P, _I32P, _I32P, _I32P])
_sig("gpjc_op_set_tuning", [_P, C.c_int32, C.c_int32, C.c_int32])
_sig("gpjc_multi_destroy", [_P], None)
_sig("gpjc_recon_multi", [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(ReconParams), _I32P, _P])
_sig("gpjc_batch_create", [C.c_int32, C.POINTER(_P), C.c_int32, C.POINTER(_P)])
_sig("gpjc_batch_destroy", [_P], None)
_sig("gpjc_recon_batched", [_P, C.POINTER(_P), C.POINTER(_P), C.c_int32, _I32P, _P])
_sig("gpjc_batch_set_wait_budget", [_P, C.c_int64])
_sig("gpjc_batch_info", [_P, _I32P, C.POINTER(C.c_int64)])


def check(status: int) -> None:
    if status != GPJC_OK:
        raise GpjcError(status, _lib.gpjc_last_error().decode())


def probe_fp32_tflops(iters: int = 200000) -> float:
    """Measured FP32 FMA throughput (TFLOP/s) of the current device."""
    v = C.c_double(0.0)
    check(_lib.gpjc_probe_fp32_tflops(int(iters), C.byref(v)))
    return float(v.value)


def debug_fail_allocations(n: int) -> None:
    """Test hook: the library's (n+1)-th and later device allocations fail
    with GPJC_ENOMEM; n < 0 restores normal allocation."""
    _lib.gpjc_debug_fail_allocations(int(n))


def lib():
    """The loaded ctypes library (for tests of the raw ABI)."""
    return _lib


def version() -> str:
    return _lib.gpjc_version().decode()


def launch_count() -> int:
    """Kernels launched by libgpjc so far in this process."""
    return int(_lib.gpjc_launch_count())


def tv_grad(x: torch.Tensor, eps: float, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Gradient of the smoothed isotropic TV of each z-slice of a
    [nz][ny][nx] complex64 image on the device."""
    nz, ny, nx = x.shape
    if out is None:
        out = torch.empty_like(x)
    if out.shape != x.shape or out.device != x.device:
        raise ValueError(f"out must have the shape {tuple(x.shape)} and device of x")
    check(_lib.gpjc_tv_grad(_dptr(x, torch.complex64), nz, ny, nx, float(eps), _dptr(out, torch.complex64),
                            _stream(stream)))
    return out


def keep_from_energy(eigvals, threshold: float, trace=None) -> np.ndarray:
    """Kept dimension per group: the smallest k whose leading eigenvalues of
    P_g hold `threshold` of trace(P_g) (-1 if the given values do not reach
    it).  eigvals [G][m] descending (e.g. Groups.matrices()[1]); trace: None
    (sum of the given values), a scalar (|ROI|, the trace of every P_g) or
    [G]."""
    ev = np.ascontiguousarray(np.asarray(eigvals, dtype=np.float64))
    G, m = ev.shape
    tr = None
    if trace is not None:
        tr = np.ascontiguousarray(np.broadcast_to(np.asarray(trace, dtype=np.float64), (G,)))
    keep = np.zeros(G, np.int32)
    check(_lib.gpjc_keep_from_energy(ev.ctypes.data_as(_P), G, m, None if tr is None else tr.ctypes.data_as(_P),
                                     float(threshold), keep.ctypes.data_as(_P)))
    return keep


STAGE_READOUT_FWD, STAGE_PHASE_ENCODE, STAGE_READOUT_ADJ = 0, 1, 2


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor, dtype=None) -> C.c_void_p:
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_I32P)


class Plan:
    """Geometry + bookkeeping tables (gpjc_plan_create)."""

    def __init__(self, geom):
        self._keep_alive = [_i32(geom.patch_group), _i32(geom.keep), _i32(geom.line_ky), _i32(geom.line_kz)]
        pg, keep, ky, kz = self._keep_alive
        self.geom = geom
        self.c = Geom(int(geom.nx), int(geom.ny), int(geom.nz), int(geom.nc), int(geom.os), int(geom.w),
                      int(geom.n_groups), _iptr(pg), _iptr(keep), int(len(ky)), _iptr(ky), _iptr(kz),
                      float(geom.cycles), float(geom.kappa_y), float(geom.kappa_z))
        self.h = _P()
        check(_lib.gpjc_plan_create(C.byref(self.c), C.byref(self.h)))

    def __del__(self):
        if getattr(self, "h", None):
            _lib.gpjc_plan_destroy(self.h)
            self.h = None

    @property
    def ntx_c(self) -> int:
        v = C.c_int32()
        check(_lib.gpjc_plan_ntx_c(self.h, C.byref(v)))
        return v.value

    def sets(self):
        """(number of aliased sets, set index of every phase-encode row [nz*ny])."""
        g = self.geom
        sor = np.zeros(g.nz * g.ny, np.int32)
        n = C.c_int32()
        check(_lib.gpjc_plan_sets(self.h, _iptr(sor), C.byref(n)))
        return int(n.value), sor

    def tables(self):
        g = self.geom
        off = np.zeros(g.ntx // g.w, np.int32)
        ref = np.zeros(g.n_groups, np.int32)
        lof = np.zeros(g.nz * g.ny, np.int32)
        check(_lib.gpjc_plan_tables(self.h, _iptr(off), _iptr(ref), _iptr(lof)))
        return off, ref, lof


class Groups:
    """Compression matrices A_g (gpjc_build_groups / gpjc_groups_from_matrices)."""

    def __init__(self, plan: Plan, handle):
        self.plan, self.h = plan, handle

    @classmethod
    def build(cls, plan: Plan, coil: torch.Tensor, roi: torch.Tensor, T: Optional[np.ndarray] = None,
              eig_iters: int = 0, block: int = 0, keep_gram: bool = False, eig_iters_fp32: int = 0,
              stream=None) -> "Groups":
        h = _P()
        bp = BuildParams(eig_iters, block, 1 if keep_gram else 0, eig_iters_fp32)
        Tp = None
        if T is not None:
            Tc = np.ascontiguousarray(np.asarray(T, np.complex64))
            Tp = Tc.ctypes.data_as(_P)
        check(_lib.gpjc_build_groups(plan.h, _dptr(coil, torch.complex64), _dptr(roi, torch.uint8), Tp,
                                     C.byref(bp), _stream(stream), C.byref(h)))
        return cls(plan, h)

    def rebuild(self, coil: torch.Tensor, roi: torch.Tensor, T: Optional[np.ndarray] = None, stream=None):
        """Recompute in place from new coil maps / ROI (asynchronous, no allocation)."""
        Tp = None
        if T is not None:
            self._T = np.ascontiguousarray(np.asarray(T, np.complex64))
            Tp = self._T.ctypes.data_as(_P)
        check(_lib.gpjc_groups_rebuild(self.h, _dptr(coil, torch.complex64), _dptr(roi, torch.uint8), Tp,
                                       _stream(stream)))
        return self

    @classmethod
    def from_matrices(cls, plan: Plan, As: Sequence[np.ndarray]) -> "Groups":
        packed = np.ascontiguousarray(np.concatenate([np.asarray(A, np.complex64).ravel() for A in As]))
        h = _P()
        check(_lib.gpjc_groups_from_matrices(plan.h, packed.ctypes.data_as(_P), C.byref(h)))
        return cls(plan, h)

    def __del__(self):
        if getattr(self, "h", None):
            _lib.gpjc_groups_destroy(self.h)
            self.h = None

    def info(self) -> GroupsInfo:
        i = GroupsInfo()
        check(_lib.gpjc_groups_info_get(self.h, C.byref(i)))
        return i

    def matrices(self):
        """(list of A_g [keep_g][N_s] complex64, Ritz values [G][b] or None)."""
        g = self.plan.geom
        ns = g.nc * g.w
        total = int(sum(int(k) * ns for k in g.keep))
        A = np.zeros(total, np.complex64)
        info = self.info()
        ritz = np.zeros((g.n_groups, max(info.block, 1)), np.float64)
        check(_lib.gpjc_groups_get(self.h, A.ctypes.data_as(_P), ritz.ctypes.data_as(_P)))
        out, o = [], 0
        for k in g.keep:
            out.append(A[o:o + int(k) * ns].reshape(int(k), ns))
            o += int(k) * ns
        return out, (ritz if info.block > 0 else None)

    def query(self, precision: int = FP32, nchunk: int = 0):
        """(N'_tx, device bytes an Operator(self, ..., precision, nchunk) allocates)."""
        ntxc = C.c_int32(0)
        nbytes = C.c_uint64(0)
        check(_lib.gpjc_query(self.h, precision, nchunk, C.byref(ntxc), C.byref(nbytes)))
        return int(ntxc.value), int(nbytes.value)

    def gram(self) -> np.ndarray:
        g = self.plan.geom
        ns = g.nc * g.w
        P = np.zeros((g.n_groups, ns, ns), np.complex128)
        check(_lib.gpjc_groups_gram(self.h, P.ctypes.data_as(_P)))
        return P

    def roi(self) -> np.ndarray:
        n = self.info().roi_pixels
        pix = np.zeros(n, np.int32)
        check(_lib.gpjc_groups_roi(self.h, _iptr(pix)))
        return pix


def compress(groups: Groups, S: torch.Tensor, precision: int = FP32, out: Optional[torch.Tensor] = None,
             stream=None) -> torch.Tensor:
    g = groups.plan.geom
    if out is None:
        out = torch.empty((g.n_lines, groups.plan.ntx_c), dtype=torch.complex64, device=S.device)
    check(_lib.gpjc_compress(groups.h, _dptr(S, torch.complex64), _dptr(out, torch.complex64), precision,
                             _stream(stream)))
    return out


class Operator:
    """E_c and E_c^H bound to groups and coil maps (gpjc_op_create)."""

    def __init__(self, groups: Groups, coil: torch.Tensor, precision: int = FP32, nchunk: int = 0):
        self.groups, self.coil, self.precision = groups, coil, precision
        self.plan = groups.plan
        self.h = _P()
        check(_lib.gpjc_op_create(groups.h, _dptr(coil, torch.complex64), precision, nchunk, C.byref(self.h)))

    @classmethod
    def local_b0(cls, groups: Groups, coil: torch.Tensor, fields: torch.Tensor, amps: np.ndarray) -> "Operator":
        """Nonlinear local-B0 operator: stored compressed readout matrices
        built from A_g, coil maps, fields [n_fields][nz][ny][nx] (float32,
        device) and drive amps [n_fields][ntx] (host)."""
        op = cls.__new__(cls)
        op.groups, op.coil, op.precision = groups, coil, FP32
        op.plan = groups.plan
        op.h = _P()
        a = np.ascontiguousarray(np.asarray(amps, np.float64))
        f = fields.contiguous()
        if f.dtype != torch.float32 or f.device != coil.device:
            raise ValueError("fields must be float32 on the coil maps' device")
        check(_lib.gpjc_op_create_local_b0(groups.h, _dptr(coil, torch.complex64), int(a.shape[0]),
                                           C.c_void_p(f.data_ptr()), a.ctypes.data_as(_P), C.byref(op.h)))
        return op

    def __del__(self):
        if getattr(self, "h", None):
            _lib.gpjc_op_destroy(self.h)
            self.h = None

    @property
    def image_shape(self):
        g = self.plan.geom
        return (g.nz, g.ny, g.nx)

    @property
    def data_shape(self):
        return (self.plan.geom.n_lines, self.plan.ntx_c)

    def profile(self, enable: bool = True) -> None:
        check(_lib.gpjc_op_profile(self.h, 1 if enable else 0))

    def profile_read(self, stage: int):
        """(total device ms, launches) of a stage since the last reset."""
        ms, n = C.c_double(), C.c_int32()
        check(_lib.gpjc_op_profile_read(self.h, stage, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def autotune(self, stream=None) -> int:
        n = C.c_int32()
        check(_lib.gpjc_op_autotune(self.h, _stream(stream), C.byref(n)))
        return n.value

    def tuning(self):
        """(forward coil chunks, adjoint coil chunks, adjoint row pieces)."""
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        check(_lib.gpjc_op_tuning(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def set_tuning(self, nchunk: int, nchunk_adj: int, adj_pieces: int) -> None:
        check(_lib.gpjc_op_set_tuning(self.h, int(nchunk), int(nchunk_adj), int(adj_pieces)))

    def shape_class(self) -> str:
        """Key of the operator's shape class for persisted tuning results."""
        g = self.plan.geom
        return (f"{g.nz}x{g.ny}x{g.nx}_c{g.nc}_os{g.os}_w{g.w}_G{g.n_groups}_k{int(max(g.keep))}"
                f"_l{g.n_lines}_p{self.precision}")

    def autotune_cached(self, path: str, stream=None):
        """gpjc_op_autotune with a JSON cache of the chosen knobs per shape
        class: a cached class is set directly, a new one is timed and
        stored.  Returns the knobs."""
        import json
        import os

        cache = {}
        if os.path.exists(path):
            with open(path) as f:
                cache = json.load(f)
        key = self.shape_class()
        if key in cache:
            self.set_tuning(*cache[key])
        else:
            self.autotune(stream)
            cache[key] = list(self.tuning())
            tmp = path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        return self.tuning()

    def E(self, x: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.data_shape, dtype=torch.complex64, device=x.device)
        check(_lib.gpjc_apply_E(self.h, _dptr(x, torch.complex64), _dptr(out, torch.complex64), _stream(stream)))
        return out

    def EH(self, y: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.complex64, device=y.device)
        check(_lib.gpjc_apply_EH(self.h, _dptr(y, torch.complex64), _dptr(out, torch.complex64), _stream(stream)))
        return out

    def normal(self, x: torch.Tensor, out=None, qq: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.complex64, device=x.device)
        q = _dptr(qq, torch.float64) if qq is not None else None
        check(_lib.gpjc_apply_normal(self.h, _dptr(x, torch.complex64), _dptr(out, torch.complex64), q,
                                     _stream(stream)))
        return out

    def simulate(self, x: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        g = self.plan.geom
        if out is None:
            out = torch.empty((g.n_lines, g.nc, g.ntx), dtype=torch.complex64, device=x.device)
        check(_lib.gpjc_simulate(self.h, _dptr(x, torch.complex64), _dptr(out, torch.complex64), _stream(stream)))
        return out

    def simulate_adjoint(self, S: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.complex64, device=S.device)
        check(_lib.gpjc_simulate_adjoint(self.h, _dptr(S, torch.complex64), _dptr(out, torch.complex64),
                                         _stream(stream)))
        return out

    def recon(self, Sc: torch.Tensor, alg: int = CG, iters: int = 20, lam: float = 0.0, lipschitz: float = 0.0,
              power_iters: int = 20, haar_levels: int = 4, x0: Optional[torch.Tensor] = None,
              use_graph: bool = True, history: bool = False, sync: bool = True, out=None, stream=None,
              lam_tv: float = 0.0, tv_eps: float = 1e-3):
        """Returns (x, info dict).  With sync=False nothing is read back.
        FISTA: lam weights the Haar l1 term, lam_tv the smoothed TV term."""
        if out is None:
            out = (x0.clone() if x0 is not None else
                   torch.empty(self.image_shape, dtype=torch.complex64, device=Sc.device))
        elif x0 is not None:
            out.copy_(x0)
        rp = ReconParams(alg, iters, float(lam), float(lipschitz), power_iters, haar_levels,
                         1 if x0 is not None else 0, 1 if use_graph else 0, float(lam_tv), float(tv_eps))
        hist = np.zeros(iters + 1, np.float64) if history else None
        info = ReconInfo(0, 0.0, hist.ctypes.data_as(C.POINTER(C.c_double)) if hist is not None else None)
        check(_lib.gpjc_recon(self.h, _dptr(Sc, torch.complex64), _dptr(out, torch.complex64), C.byref(rp),
                              C.byref(info) if sync else None, _stream(stream)))
        return out, {"status": info.status, "lipschitz": info.lipschitz, "history": hist}


def apply_EH_static(groups: Groups, coil: torch.Tensor, y: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """E_c^H y with the library's static scratch: no operator, no allocation
    inside the call (for callers that cannot allocate device memory there)."""
    g = groups.plan.geom
    if out is None:
        out = torch.empty((g.nz, g.ny, g.nx), dtype=torch.complex64, device=y.device)
    if tuple(coil.shape) != (g.nc, g.nz, g.ny, g.nx):
        raise ValueError(f"coil must have shape {(g.nc, g.nz, g.ny, g.nx)}, got {tuple(coil.shape)}")
    if tuple(y.shape) != (g.n_lines, groups.plan.ntx_c):
        raise ValueError(f"y must have shape {(g.n_lines, groups.plan.ntx_c)}, got {tuple(y.shape)}")
    if tuple(out.shape) != (g.nz, g.ny, g.nx):
        raise ValueError(f"out must have shape {(g.nz, g.ny, g.nx)}, got {tuple(out.shape)}")
    if not (y.device == coil.device == out.device) or y.device.type != "cuda":
        raise ValueError("coil, y and out must be on one CUDA device")
    with torch.cuda.device(y.device):
        check(_lib.gpjc_apply_EH_static(groups.h, _dptr(coil, torch.complex64), _dptr(y, torch.complex64),
                                        _dptr(out, torch.complex64), _stream(stream)))
    return out


class Batch:
    """Batched CG over many FP32 operators in one persistent launch."""

    def __init__(self, ops: Sequence[Operator], iters: int):
        self.ops = list(ops)
        arr = (_P * len(self.ops))(*[op.h for op in self.ops])
        self.h = _P()
        check(_lib.gpjc_batch_create(len(self.ops), arr, iters, C.byref(self.h)))
        self.iters = iters

    def __del__(self):
        if getattr(self, "h", None):
            _lib.gpjc_batch_destroy(self.h)
            self.h = None

    def info(self):
        grid, items = C.c_int32(), C.c_int64()
        check(_lib.gpjc_batch_info(self.h, C.byref(grid), C.byref(items)))
        return grid.value, items.value

    def set_wait_budget(self, cycles: int) -> None:
        check(_lib.gpjc_batch_set_wait_budget(self.h, cycles))

    def recon(self, Scs: Sequence[torch.Tensor], xs: Optional[Sequence[torch.Tensor]] = None,
              use_graph: bool = True, sync: bool = True, stream=None):
        if xs is None:
            xs = [torch.empty(op.image_shape, dtype=torch.complex64, device=Sc.device)
                  for op, Sc in zip(self.ops, Scs)]
        sp = (_P * len(Scs))(*[_dptr(t, torch.complex64) for t in Scs])
        xp = (_P * len(xs))(*[_dptr(t, torch.complex64) for t in xs])
        st = C.c_int32(0)
        check(_lib.gpjc_recon_batched(self.h, sp, xp, 1 if use_graph else 0, C.byref(st) if sync else None,
                                      _stream(stream)))
        return xs, st.value


class Multi:
    """Many reconstructions (any operators) in one CUDA graph on parallel
    branches (gpjc_multi_create / gpjc_recon_multi)."""

    def __init__(self, ops: Sequence[Operator], n_branches: int = 8):
        self.ops = list(ops)
        arr = (_P * len(self.ops))(*[op.h for op in self.ops])
        self.h = _P()
        check(_lib.gpjc_multi_create(len(self.ops), arr, int(n_branches), C.byref(self.h)))

    def __del__(self):
        if getattr(self, "h", None):
            _lib.gpjc_multi_destroy(self.h)
            self.h = None

    def recon(self, Scs: Sequence[torch.Tensor], xs: Optional[Sequence[torch.Tensor]] = None, alg: int = CG,
              iters: int = 30, sync: bool = True, stream=None):
        if xs is None:
            xs = [torch.empty(op.image_shape, dtype=torch.complex64, device=Sc.device)
                  for op, Sc in zip(self.ops, Scs)]
        sp = (_P * len(Scs))(*[_dptr(t, torch.complex64) for t in Scs])
        xp = (_P * len(xs))(*[_dptr(t, torch.complex64) for t in xs])
        rp = ReconParams(alg, iters, 0.0, 0.0, 0, 0, 0, 1, 0.0, 1e-3)
        st = C.c_int32(0)
        check(_lib.gpjc_recon_multi(self.h, sp, xp, C.byref(rp), C.byref(st) if sync else None, _stream(stream)))
        return xs, st.value


def plan_from(geom) -> Plan:
    return Plan(geom)
