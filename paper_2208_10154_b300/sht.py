"""Thin ctypes binding of libsht (include/sht.h).

Argument marshalling only: every step of a transform runs in libsht's CUDA
kernels. Device memory comes from torch (outputs and workspaces), and calls
are issued on torch's current CUDA stream. There is no CPU fallback: if the
library is missing or fails to load, every call raises.

Low-level names mirror the C ABI (``sht_plan_create``, ``sht_alm2map``, ...);
``Plan`` wraps a plan handle with tensor-in / tensor-out methods.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsht.so")

SHT_OK, SHT_EINVAL, SHT_ENOMEM, SHT_ECUDA, SHT_EUNSUPPORTED, SHT_ETIMEOUT = range(6)
SHT_FP64, SHT_SPLIT_F16X4 = 0, 1
PRECISIONS = {"fp64": SHT_FP64, "split": SHT_SPLIT_F16X4, "f16x4": SHT_SPLIT_F16X4}

_lock = threading.Lock()
_lib = None


class ShtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libsht status {status}: {msg}")
        self.status = status


def load() -> ctypes.CDLL:
    """Load libsht.so (build it with ``python -m paper_2208_10154_b300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsht.so not found at {LIB_PATH}; build it with "
                              "`python -m paper_2208_10154_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        LL = ctypes.c_longlong
        lib.sht_plan_create.argtypes = [I, I, I, I, I, I, ctypes.POINTER(P)]
        lib.sht_plan_create.restype = I
        lib.sht_plan_destroy.argtypes = [P]
        lib.sht_plan_destroy.restype = None
        lib.sht_workspace_bytes.argtypes = [P, I]
        lib.sht_workspace_bytes.restype = S
        lib.sht_workspace_bytes_iter.argtypes = [P, I, I]
        lib.sht_workspace_bytes_iter.restype = S
        for n in ("nside", "lmax", "mmax", "spin", "precision"):
            f = getattr(lib, "sht_plan_" + n)
            f.argtypes = [P]
            f.restype = I
        for n in ("npix", "nalm"):
            f = getattr(lib, "sht_plan_" + n)
            f.argtypes = [P]
            f.restype = LL
        lib.sht_plan_device_bytes.argtypes = [P]
        lib.sht_plan_device_bytes.restype = S
        lib.sht_plan_terms_kept.argtypes = [P]
        lib.sht_plan_terms_kept.restype = ctypes.c_double
        lib.sht_plan_first_pairs.argtypes = [P, P]
        lib.sht_plan_first_pairs.restype = I
        lib.sht_alm2map.argtypes = [P, P, P, I, P, S, P]
        lib.sht_map2alm.argtypes = [P, P, P, I, I, P, S, P]
        lib.sht_alm2map_adjoint.argtypes = [P, P, P, I, P, S, P]
        lib.sht_map2alm_adjoint.argtypes = [P, P, P, I, P, S, P]
        lib.sht_alm2map_host.argtypes = [P, P, P, I, P]
        lib.sht_map2alm_host.argtypes = [P, P, P, I, I, P]
        lib.sht_map2alm_eb.argtypes = [P, P, P, I, I, P, S, P]
        lib.sht_map2alm_eb.restype = I
        lib.sht_alm2map_eb.argtypes = [P, P, P, I, I, P, S, P]
        lib.sht_alm2map_eb.restype = I
        lib.sht_workspace_bytes_eb.argtypes = [P, I]
        lib.sht_workspace_bytes_eb.restype = S
        lib.sht_map2alm_immediate.argtypes = [P, P, P, I, I, P, S, P]
        lib.sht_map2alm_immediate.restype = I
        lib.sht_workspace_bytes_immediate.argtypes = [P, I]
        lib.sht_workspace_bytes_immediate.restype = S
        lib.sht_alm_to_square.argtypes = [P, P, P, I, P]
        lib.sht_square_to_alm.argtypes = [P, P, P, I, P]
        lib.sht_eb_project.argtypes = [P, P, P, I, I, I, P, S, P]
        lib.sht_workspace_bytes_project.argtypes = [P, I, I]
        lib.sht_workspace_bytes_project.restype = S
        for f in (lib.sht_alm2map, lib.sht_map2alm, lib.sht_alm2map_adjoint,
                  lib.sht_map2alm_adjoint, lib.sht_alm2map_host, lib.sht_map2alm_host,
                  lib.sht_alm_to_square, lib.sht_square_to_alm, lib.sht_eb_project):
            f.restype = I
        lib.sht_last_error.restype = ctypes.c_char_p
        lib.sht_last_launch_count.restype = I
        lib.sht_plan_device_status.argtypes = [P, ctypes.POINTER(I)]
        lib.sht_plan_device_status.restype = I
        lib.sht_version.restype = ctypes.c_char_p
        lib.sht_profile_begin.restype = None
        lib.sht_profile_end.argtypes = [ctypes.c_char_p, I]
        lib.sht_profile_end.restype = I
        _lib = lib
        return lib


def _check(status: int):
    if status != SHT_OK:
        raise ShtError(status, load().sht_last_error().decode())


def sht_last_error() -> str:
    return load().sht_last_error().decode()


def sht_last_launch_count() -> int:
    return load().sht_last_launch_count()


def sht_plan_device_status(h) -> int:
    """Device word of the plan's bounded waits (0 = fine); raises ShtError on a timeout."""
    code = ctypes.c_int(0)
    _check(load().sht_plan_device_status(h, ctypes.byref(code)))
    return code.value


def sht_profile_begin() -> None:
    load().sht_profile_begin()


def sht_profile_end() -> dict:
    """Per-kernel {name: {"launches": n, "ms": total}} since sht_profile_begin()."""
    import json
    lib = load()
    buf = ctypes.create_string_buffer(1 << 16)
    n = lib.sht_profile_end(buf, len(buf))
    if n > len(buf):
        raise RuntimeError("profile buffer too small")
    return json.loads(buf.value.decode())


def sht_plan_create(nside, lmax, mmax=-1, spin=0, precision=SHT_FP64, device=0):
    h = ctypes.c_void_p()
    _check(load().sht_plan_create(int(nside), int(lmax), int(mmax), int(spin), int(precision),
                                  int(device), ctypes.byref(h)))
    return h


def sht_plan_destroy(h):
    load().sht_plan_destroy(h)


def sht_workspace_bytes(h, nmaps: int, niter: int = 0) -> int:
    lib = load()
    return lib.sht_workspace_bytes_iter(h, nmaps, niter) if niter else lib.sht_workspace_bytes(h, nmaps)


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def sht_alm2map(h, alm_ptr, map_ptr, nmaps, ws_ptr, ws_bytes, stream_ptr):
    _check(load().sht_alm2map(h, alm_ptr, map_ptr, nmaps, ws_ptr, ws_bytes, stream_ptr))


def sht_map2alm(h, map_ptr, alm_ptr, nmaps, niter, ws_ptr, ws_bytes, stream_ptr):
    _check(load().sht_map2alm(h, map_ptr, alm_ptr, nmaps, niter, ws_ptr, ws_bytes, stream_ptr))


def sht_alm2map_adjoint(h, map_ptr, alm_ptr, nmaps, ws_ptr, ws_bytes, stream_ptr):
    _check(load().sht_alm2map_adjoint(h, map_ptr, alm_ptr, nmaps, ws_ptr, ws_bytes, stream_ptr))


def sht_map2alm_adjoint(h, alm_ptr, map_ptr, nmaps, ws_ptr, ws_bytes, stream_ptr):
    _check(load().sht_map2alm_adjoint(h, alm_ptr, map_ptr, nmaps, ws_ptr, ws_bytes, stream_ptr))


def sht_alm2map_host(h, alm_ptr, map_ptr, nmaps, stream_ptr):
    _check(load().sht_alm2map_host(h, alm_ptr, map_ptr, nmaps, stream_ptr))


def sht_map2alm_host(h, map_ptr, alm_ptr, nmaps, niter, stream_ptr):
    _check(load().sht_map2alm_host(h, map_ptr, alm_ptr, nmaps, niter, stream_ptr))


class Plan:
    """A resident transform plan (ring tables, recurrence tables, FFT tables).

    Tensors: alm complex128 [nmaps, ncomp, nalm] (m-major packed), map float64
    [nmaps, ncomp, npix] (HEALPix RING), both contiguous on the plan's device.
    """

    def __init__(self, nside: int, lmax: int, mmax: int | None = None, spin: int = 0,
                 precision="fp64", device: int | None = None):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.handle = sht_plan_create(nside, lmax, -1 if mmax is None else mmax, spin, precision,
                                      self.device)
        lib = load()
        self.nside, self.lmax, self.mmax = nside, lmax, lib.sht_plan_mmax(self.handle)
        self.spin, self.precision = spin, precision
        self.ncomp = 2 if spin else 1
        self.npix = lib.sht_plan_npix(self.handle)
        self.nalm = lib.sht_plan_nalm(self.handle)
        self._ws = None

    def close(self):
        if getattr(self, "handle", None) is not None:
            sht_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self) -> int:
        """0 if every bounded device wait of this plan's kernels succeeded; raises otherwise."""
        return sht_plan_device_status(self.handle)

    def device_bytes(self) -> int:
        """Device memory held by the plan itself (tables, host-path staging)."""
        return int(load().sht_plan_device_bytes(self.handle))

    def first_pairs(self):
        """First ring pair contracted for each order m (numpy int32 [mmax + 1])."""
        import numpy as np
        out = np.zeros(self.mmax + 1, dtype=np.int32)
        _check(load().sht_plan_first_pairs(self.handle, ctypes.c_void_p(out.ctypes.data)))
        return out

    def terms_kept(self) -> float:
        """Share of the (m, l, ring pair) Legendre terms the contraction evaluates."""
        return float(load().sht_plan_terms_kept(self.handle))

    def workspace_bytes(self, nmaps: int, niter: int = 0) -> int:
        return sht_workspace_bytes(self.handle, nmaps, niter)

    def _workspace(self, nmaps: int, niter: int = 0, workspace=None):
        need = self.workspace_bytes(nmaps, niter)
        if workspace is not None:
            nb = workspace.numel() * workspace.element_size()
            if nb < need:
                raise ValueError(f"workspace too small: need {need} bytes")
            return workspace, nb
        if self._ws is None or self._ws.numel() < need + 256:
            self._ws = None
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        base = self._ws.data_ptr()
        off = (-base) % 256
        return self._ws[off:], self._ws.numel() - off

    def _in(self, x, dtype, last):
        if not (x.is_cuda and x.dtype == dtype and x.is_contiguous()):
            raise ValueError(f"expected a contiguous {dtype} CUDA tensor")
        if x.shape[-1] != last:
            raise ValueError(f"last dimension must be {last}")
        return x

    def alm2map(self, alm: torch.Tensor, out=None, workspace=None) -> torch.Tensor:
        alm = self._in(alm, torch.complex128, self.nalm)
        nmaps = alm.numel() // (self.ncomp * self.nalm)
        if out is None:
            out = torch.empty((nmaps, self.ncomp, self.npix), dtype=torch.float64, device=alm.device)
        ws, wsb = self._workspace(nmaps, 0, workspace)
        sht_alm2map(self.handle, ctypes.c_void_p(alm.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                    nmaps, ctypes.c_void_p(ws.data_ptr()), wsb, _stream())
        return out

    def map2alm(self, maps: torch.Tensor, niter: int = 0, out=None, workspace=None) -> torch.Tensor:
        maps = self._in(maps, torch.float64, self.npix)
        nmaps = maps.numel() // (self.ncomp * self.npix)
        if out is None:
            out = torch.empty((nmaps, self.ncomp, self.nalm), dtype=torch.complex128, device=maps.device)
        ws, wsb = self._workspace(nmaps, niter, workspace)
        sht_map2alm(self.handle, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                    nmaps, int(niter), ctypes.c_void_p(ws.data_ptr()), wsb, _stream())
        return out

    def map2alm_eb(self, maps: torch.Tensor, which: str = "E", out=None, workspace=None) -> torch.Tensor:
        """One component (E or B) of the spin-2 map2alm: [nmaps, 2, npix] -> [nmaps, 1, nalm]."""
        maps = self._in(maps, torch.float64, self.npix)
        nmaps = maps.numel() // (2 * self.npix)
        if out is None:
            out = torch.empty((nmaps, 1, self.nalm), dtype=torch.complex128, device=maps.device)
        ws, wsb = self._workspace(nmaps, 0, workspace)
        _check(load().sht_map2alm_eb(self.handle, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     nmaps, {"E": 0, "B": 1}[which], ctypes.c_void_p(ws.data_ptr()), wsb,
                                     _stream()))
        return out

    def alm2map_eb(self, alm: torch.Tensor, which: str = "E", out=None) -> torch.Tensor:
        """Q/U maps [nmaps, 2, npix] from one component's a_lm [nmaps, 1, nalm] (the other zero)."""
        alm = self._in(alm, torch.complex128, self.nalm)
        nmaps = alm.numel() // self.nalm
        if out is None:
            out = torch.empty((nmaps, 2, self.npix), dtype=torch.float64, device=alm.device)
        lib = load()
        need = lib.sht_workspace_bytes_eb(self.handle, nmaps)
        ws = torch.empty(need + 256, dtype=torch.uint8, device=alm.device)
        off = (-ws.data_ptr()) % 256
        _check(lib.sht_alm2map_eb(self.handle, ctypes.c_void_p(alm.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  nmaps, {"E": 0, "B": 1}[which], ctypes.c_void_p(ws.data_ptr() + off), need,
                                  _stream()))
        return out

    def map2alm_immediate(self, maps: torch.Tensor, npass: int, out=None) -> torch.Tensor:
        """Algorithm 3 (immediate iteration): npass >= 1 Gauss-Seidel sweeps
        over m from a = 0 (FP64 plans, spin 0 or 2)."""
        maps = self._in(maps, torch.float64, self.npix)
        nmaps = maps.numel() // (self.ncomp * self.npix)
        if out is None:
            out = torch.empty((nmaps, self.ncomp, self.nalm), dtype=torch.complex128, device=maps.device)
        lib = load()
        need = lib.sht_workspace_bytes_immediate(self.handle, nmaps)
        ws = torch.empty(need + 256, dtype=torch.uint8, device=maps.device)
        off = (-ws.data_ptr()) % 256
        _check(lib.sht_map2alm_immediate(self.handle, ctypes.c_void_p(maps.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), nmaps, int(npass),
                                         ctypes.c_void_p(ws.data_ptr() + off), need, _stream()))
        return out

    def alm2map_adjoint(self, maps: torch.Tensor, out=None, workspace=None) -> torch.Tensor:
        maps = self._in(maps, torch.float64, self.npix)
        nmaps = maps.numel() // (self.ncomp * self.npix)
        if out is None:
            out = torch.empty((nmaps, self.ncomp, self.nalm), dtype=torch.complex128, device=maps.device)
        ws, wsb = self._workspace(nmaps, 0, workspace)
        sht_alm2map_adjoint(self.handle, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                            nmaps, ctypes.c_void_p(ws.data_ptr()), wsb, _stream())
        return out

    def map2alm_adjoint(self, alm: torch.Tensor, out=None, workspace=None) -> torch.Tensor:
        alm = self._in(alm, torch.complex128, self.nalm)
        nmaps = alm.numel() // (self.ncomp * self.nalm)
        if out is None:
            out = torch.empty((nmaps, self.ncomp, self.npix), dtype=torch.float64, device=alm.device)
        ws, wsb = self._workspace(nmaps, 0, workspace)
        sht_map2alm_adjoint(self.handle, ctypes.c_void_p(alm.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                            nmaps, ctypes.c_void_p(ws.data_ptr()), wsb, _stream())
        return out

    def alm2map_host(self, alm_host, out_host=None):
        """End to end on host numpy arrays (staged through pinned memory by libsht)."""
        import numpy as np
        a = np.ascontiguousarray(alm_host, dtype=np.complex128)
        nmaps = a.size // (self.ncomp * self.nalm)
        out = np.empty((nmaps, self.ncomp, self.npix)) if out_host is None else out_host
        sht_alm2map_host(self.handle, ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                         nmaps, _stream())
        return out

    def map2alm_host(self, map_host, niter: int = 0, out_host=None):
        import numpy as np
        x = np.ascontiguousarray(map_host, dtype=np.float64)
        nmaps = x.size // (self.ncomp * self.npix)
        out = np.empty((nmaps, self.ncomp, self.nalm), dtype=np.complex128) if out_host is None else out_host
        sht_map2alm_host(self.handle, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                         nmaps, int(niter), _stream())
        return out

    # ---- the paper's compact square a_lm storage and E / B projection ----
    def alm_to_square(self, alm: torch.Tensor, out=None) -> torch.Tensor:
        """a_lm [..., ncomp, nalm] -> compact square [nmaps, ncomp, lmax+1, lmax+1] (float64)."""
        alm = self._in(alm, torch.complex128, self.nalm)
        nmaps = alm.numel() // (self.ncomp * self.nalm)
        L = self.lmax + 1
        if out is None:
            out = torch.empty((nmaps, self.ncomp, L, L), dtype=torch.float64, device=alm.device)
        _check(load().sht_alm_to_square(self.handle, ctypes.c_void_p(alm.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), nmaps, _stream()))
        return out

    def square_to_alm(self, sq: torch.Tensor, out=None) -> torch.Tensor:
        """compact square [..., ncomp, lmax+1, lmax+1] (float64) -> a_lm [nmaps, ncomp, nalm]."""
        L = self.lmax + 1
        if not (sq.is_cuda and sq.dtype == torch.float64 and sq.is_contiguous()) or sq.shape[-2:] != (L, L):
            raise ValueError(f"expected a contiguous float64 CUDA tensor [..., {L}, {L}]")
        nmaps = sq.numel() // (self.ncomp * L * L)
        if out is None:
            out = torch.empty((nmaps, self.ncomp, self.nalm), dtype=torch.complex128, device=sq.device)
        _check(load().sht_square_to_alm(self.handle, ctypes.c_void_p(sq.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), nmaps, _stream()))
        return out

    def eb_project(self, maps: torch.Tensor, which: str = "E", niter: int = 0, out=None) -> torch.Tensor:
        """Pixel-domain E (which="E") or B ("B") part of Q/U maps [nmaps, 2, npix] (spin-2 plans)."""
        maps = self._in(maps, torch.float64, self.npix)
        nmaps = maps.numel() // (self.ncomp * self.npix)
        if out is None:
            out = torch.empty((nmaps, self.ncomp, self.npix), dtype=torch.float64, device=maps.device)
        lib = load()
        need = lib.sht_workspace_bytes_project(self.handle, nmaps, int(niter))
        ws = torch.empty(need + 256, dtype=torch.uint8, device=maps.device)
        off = (-ws.data_ptr()) % 256
        _check(lib.sht_eb_project(self.handle, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  nmaps, {"E": 0, "B": 1}[which], int(niter), ctypes.c_void_p(ws.data_ptr() + off),
                                  need, _stream()))
        return out
