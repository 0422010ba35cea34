"""Python binding of libmcd (the C ABI in include/mcd.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels (or, for the basis sampler, its host threads).  Device vectors are
torch tensors; the context runs on torch's current CUDA stream.  The library
must have been built (``paper_2509_22975_gb300.build.build()``); importing an
entry point without it raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from .build import LIB as LIB_PATH, build  # noqa: F401

MCD_OK, MCD_W_SHORT = 0, 1
MCD_F64, MCD_F32 = 0, 1
MCD_SAMPLE_NEW_ONLY = 1
MCD_OPT_HV_ALGO, MCD_OPT_KERNEL_TIMING, MCD_OPT_SAMPLER_THREADS, MCD_OPT_HASH_ITEM = 1, 2, 3, 4
MCD_OPT_SAMPLER_DEVICE = 5
MCD_OPT_HV_CACHE = 6
MCD_OPT_APPLY_SYNC, MCD_OPT_WAIT_TEST, MCD_OPT_KRYLOV_STORE, MCD_OPT_HV_COLS = 7, 8, 9, 10
HV_COLS_AUTO, HV_COLS_TILES, HV_COLS_ITEMS = 0, 1, 2
MCD_OPT_BATCH_SPLIT, MCD_OPT_BATCH_MODE = 11, 12
BATCH_POOL, BATCH_LOCKSTEP = 0, 1
MCD_E_NOT_CONVERGED, MCD_E_TIMEOUT = -5, -7
CACHE_AUTO, CACHE_OFF, CACHE_REQUIRED = 0, 1, 2
SAMPLER_AUTO, SAMPLER_HOST, SAMPLER_DEVICE = 0, 1, 2
HV_AUTO, HV_PLAIN, HV_SEARCH, HV_HASH = 0, 1, 2, 3
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mcd.h")

_lib = None
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_dp = ctypes.POINTER(ctypes.c_double)
c_u64p = ctypes.POINTER(ctypes.c_uint64)
c_vp = ctypes.c_void_p

_SIGS = {
    "mcd_create": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int, c_vp]),
    "mcd_destroy": (ctypes.c_int, [c_vp]),
    "mcd_set_stream": (ctypes.c_int, [c_vp, c_vp]),
    "mcd_set_option": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int64]),
    "mcd_last_error": (ctypes.c_char_p, [c_vp]),
    "mcd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mcd_set_hamiltonian": (ctypes.c_int, [c_vp, ctypes.c_int, c_dp, c_dp, c_dp, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int]),
    "mcd_build_basis": (ctypes.c_int, [c_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, c_u64p,
                                       ctypes.c_int64, ctypes.c_int, c_i64p]),
    "mcd_set_basis": (ctypes.c_int, [c_vp, c_u64p, ctypes.c_int64]),
    "mcd_set_basis_device": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int64]),
    "mcd_get_basis": (ctypes.c_int, [c_vp, c_u64p, ctypes.c_int64, c_i64p]),
    "mcd_save_basis": (ctypes.c_int, [c_vp, ctypes.c_char_p]),
    "mcd_load_basis": (ctypes.c_int, [c_vp, ctypes.c_char_p]),
    "mcd_launch_count": (ctypes.c_int, [c_vp, c_i64p]),
    "mcd_hv_cache_info": (ctypes.c_int, [c_vp, c_i64p, c_i64p, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "mcd_basis_info": (ctypes.c_int, [c_vp, c_i64p, c_i64p, c_i64p, c_i64p]),
    "mcd_apply": (ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mcd_diagonal": (ctypes.c_int, [c_vp, c_vp]),
    "mcd_connections": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, ctypes.c_int64, c_i64p]),
    "mcd_connections_noalloc": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, ctypes.c_int64, c_i64p]),
    "mcd_lanczos_ground": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                          c_dp, c_vp, ctypes.POINTER(ctypes.c_int), c_dp]),
    "mcd_lanczos_coeffs": (ctypes.c_int, [c_vp, c_dp, c_dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mcd_kernel_times": (ctypes.c_int, [c_vp, c_dp, c_i64p, ctypes.c_int, ctypes.c_int]),
    "mcd_band_lanczos_green": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, c_dp, c_dp,
                                              ctypes.c_int, c_dp, c_dp, c_i64p, c_i64p]),
    "mcd_symeig": (ctypes.c_int, [ctypes.c_int, c_dp, c_dp, ctypes.c_int, c_dp]),
    "mcd_hv_adjoint": (ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_dp, c_dp, c_dp]),
    "mcd_green_gradient": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.c_int, ctypes.c_int, ctypes.c_double, c_dp, c_dp, ctypes.c_int, c_dp,
                                          c_dp, ctypes.c_double, c_dp, c_dp, c_dp, ctypes.POINTER(ctypes.c_int)]),
    "mcd_batch_apply": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int, c_vp, c_vp, ctypes.c_int]),
    "mcd_batch_band_lanczos_green": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                    ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_double, ctypes.c_int, c_dp, c_dp, ctypes.c_int, c_dp,
                                                    c_dp, c_i64p, c_i64p]),
    "mcd_batch_green_gradient": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, c_dp, c_dp, ctypes.c_int, c_dp, c_dp, ctypes.c_double,
                                                c_dp, c_dp, c_dp, ctypes.POINTER(ctypes.c_int)]),
    "mcd_batch_lanczos_ground": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_uint64, ctypes.c_int, c_dp, ctypes.POINTER(ctypes.c_int),
                                                c_dp, ctypes.POINTER(c_vp)]),
}


class MCDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mcd status {status}: {msg}")
        self.status = status


def lib():
    """The loaded libmcd.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmcd.so is not built ({LIB_PATH}); call paper_2509_22975_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions include/mcd.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcd_[a-z0-9_]+)\s*\(", text)))


def mcd_symeig(A, rows: int | None = None):
    """Eigenvalues (ascending) and the first `rows` rows of the eigenvectors."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    rows = n if rows is None else rows
    w = np.zeros(n)
    X = np.zeros((rows, n))
    st = lib().mcd_symeig(n, A.ctypes.data_as(c_dp), w.ctypes.data_as(c_dp), rows, X.ctypes.data_as(c_dp))
    if st != MCD_OK:
        raise MCDError(st, "mcd_symeig")
    return w, X


def _ctx_array(ctxs):
    arr = (c_vp * len(ctxs))()
    for i, c in enumerate(ctxs):
        arr[i] = c.h
    return arr


def _batch_check(ctxs, st, name, ok=(0,)):
    if st not in ok:
        msg = lib().mcd_last_error(ctxs[0].h) if ctxs else b""
        raise MCDError(st, f"{name}: {(msg or b'').decode()}")
    return st


def mcd_batch_apply(ctxs, x, y):
    """y_i = H~_i x_i for every context; x, y: 1-D device tensors holding the
    instances' vectors back to back (float32 or float64)."""
    for c in ctxs:
        c._sync_stream()
    st = lib().mcd_batch_apply(_ctx_array(ctxs), len(ctxs), _ptr(x), _ptr(y), _dtype_code(x))
    return _batch_check(ctxs, st, "mcd_batch_apply")


def mcd_batch_lanczos_ground(ctxs, max_iter: int, tol: float, seed: int, dtype: int, psi=None,
                             allow_not_converged: bool = False):
    """Lanczos ground states of all contexts (concurrent per-instance solves,
    or lockstep launches with MCD_OPT_BATCH_MODE = 1 on ctxs[0]); returns dict
    with E0, iters, residual (numpy arrays) and status.  psi: None or a list of
    device tensors (or None entries) receiving the normalised Ritz vectors."""
    for c in ctxs:
        c._sync_stream()
    n = len(ctxs)
    E0 = np.zeros(n)
    it = (ctypes.c_int * n)()
    res = np.zeros(n)
    parr = None
    if psi is not None:
        parr = (c_vp * n)()
        for i, p in enumerate(psi):
            parr[i] = _ptr(p) or None
    st = lib().mcd_batch_lanczos_ground(_ctx_array(ctxs), n, max_iter, tol, seed, dtype, E0.ctypes.data_as(c_dp), it,
                                        res.ctypes.data_as(c_dp), parr)
    _batch_check(ctxs, st, "mcd_batch_lanczos_ground", ok=(0, -5) if allow_not_converged else (0,))
    return {"E0": E0, "iters": np.array(list(it)), "residual": res, "status": st}


def _orbitals(orbitals):
    L = len(orbitals)
    return (L, (ctypes.c_int * L)(*[int(o[0]) for o in orbitals]), (ctypes.c_int * L)(*[int(o[1]) for o in orbitals]))


def _zpoints(z):
    z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.complex128)
    return z, np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)


def mcd_batch_band_lanczos_green(ctxs, orbitals, n_block_iter: int, w_t: float, z, dtype: int = MCD_F64):
    """G[n_inst, nz, L, L] (complex) of every context's last ground state, the
    instances run concurrently; returns (G, dim_plus[n_inst], dim_minus[n_inst])."""
    for c in ctxs:
        c._sync_stream()
    n = len(ctxs)
    L, site, spin = _orbitals(orbitals)
    z, zr, zi = _zpoints(z)
    gr = np.zeros((n, len(z), L, L))
    gi = np.zeros((n, len(z), L, L))
    dp = np.zeros(n, dtype=np.int64)
    dm = np.zeros(n, dtype=np.int64)
    st = lib().mcd_batch_band_lanczos_green(_ctx_array(ctxs), n, site, spin, L, n_block_iter, w_t, dtype,
                                            zr.ctypes.data_as(c_dp), zi.ctypes.data_as(c_dp), len(z),
                                            gr.ctypes.data_as(c_dp), gi.ctypes.data_as(c_dp),
                                            dp.ctypes.data_as(c_i64p), dm.ctypes.data_as(c_i64p))
    _batch_check(ctxs, st, "mcd_batch_band_lanczos_green")
    return gr + 1j * gi, dp, dm


def mcd_batch_green_gradient(ctxs, orbitals, n_block_iter: int, w_t: float, z, gG, cg_tol: float = 1e-11,
                             allow_not_converged: bool = False):
    """mcd_green_gradient of every context, the instances run concurrently;
    gG: complex [n_inst, nz, L, L].  Returns (grad_t [n_inst, n, n],
    grad_eps [n_inst, n], grad_U [n_inst, n], cg_iters [n_inst])."""
    for c in ctxs:
        c._sync_stream()
    n_inst = len(ctxs)
    L, site, spin = _orbitals(orbitals)
    z, zr, zi = _zpoints(z)
    gG = np.asarray(gG, dtype=np.complex128).reshape(n_inst, len(z), L, L)
    gr, gi = np.ascontiguousarray(gG.real), np.ascontiguousarray(gG.imag)
    n = ctxs[0].n_sites
    gt, ge, gu = np.zeros((n_inst, n, n)), np.zeros((n_inst, n)), np.zeros((n_inst, n))
    it = (ctypes.c_int * n_inst)()
    st = lib().mcd_batch_green_gradient(_ctx_array(ctxs), n_inst, site, spin, L, n_block_iter, w_t,
                                        zr.ctypes.data_as(c_dp), zi.ctypes.data_as(c_dp), len(z),
                                        gr.ctypes.data_as(c_dp), gi.ctypes.data_as(c_dp), cg_tol,
                                        gt.ctypes.data_as(c_dp), ge.ctypes.data_as(c_dp), gu.ctypes.data_as(c_dp), it)
    _batch_check(ctxs, st, "mcd_batch_green_gradient", ok=(0, -5) if allow_not_converged else (0,))
    return gt, ge, gu, np.array(list(it))


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return MCD_F64
    if t.dtype == torch.float32:
        return MCD_F32
    raise TypeError("vectors must be float32 or float64")


class Context:
    """An mcd_ctx.  device=-1 gives a host-only context (sampler, basis)."""

    def __init__(self, device: int = 0, stream=None):
        self.L = lib()
        self.device = device
        h = c_vp()
        if device >= 0 and stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        st = self.L.mcd_create(ctypes.byref(h), device, stream or None)
        if st != MCD_OK:
            raise MCDError(st, self.L.mcd_last_error(None).decode())
        self.h = h

    # -- helpers ---------------------------------------------------------------
    def _check(self, st: int, ok=(MCD_OK,)) -> int:
        if st not in ok:
            raise MCDError(st, self.L.mcd_last_error(self.h).decode())
        return st

    def _sync_stream(self):
        if self.device >= 0:
            import torch
            self.L.mcd_set_stream(self.h, torch.cuda.current_stream(self.device).cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            self.L.mcd_destroy(self.h)
            self.h = None

    __del__ = close

    # -- ABI mirror -------------------------------------------------------------
    def mcd_set_option(self, option: int, value: int):
        return self._check(self.L.mcd_set_option(self.h, option, value))

    def mcd_set_hamiltonian(self, t, eps, U, n_up: int, n_dn: int):
        t = np.ascontiguousarray(t, dtype=np.float64)
        n = t.shape[0]
        e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        u = np.ascontiguousarray(np.atleast_1d(U), dtype=np.float64)
        ep = e.ctypes.data_as(c_dp) if e is not None else None
        st = self._check(self.L.mcd_set_hamiltonian(self.h, n, t.ctypes.data_as(c_dp), ep,
                                                    u.ctypes.data_as(c_dp), len(u), n_up, n_dn))
        self.n_sites, self.n_up, self.n_dn = n, n_up, n_dn
        return st

    def mcd_build_basis(self, seed: int, n_target: int, beta: float, seed_states, flags: int = 0):
        s = np.ascontiguousarray(np.atleast_1d(seed_states), dtype=np.uint64)
        n = ctypes.c_int64(0)
        st = self.L.mcd_build_basis(self.h, seed, n_target, beta, s.ctypes.data_as(c_u64p), len(s), flags,
                                    ctypes.byref(n))
        self._check(st, ok=(MCD_OK, MCD_W_SHORT))
        return st, n.value

    def mcd_set_basis(self, words):
        """Install a basis of host words: a numpy array / sequence, or a
        contiguous 64-bit CPU torch tensor (pinned memory copies by DMA)."""
        dev = getattr(words, "device", None)
        if dev is not None and getattr(dev, "type", None) == "cpu" and hasattr(words, "data_ptr"):
            if words.element_size() != 8 or not words.is_contiguous():
                raise ValueError("basis tensor must be contiguous 64-bit words")
            return self._check(self.L.mcd_set_basis(self.h, ctypes.cast(words.data_ptr(), c_u64p), words.numel()))
        w = np.ascontiguousarray(words, dtype=np.uint64)
        return self._check(self.L.mcd_set_basis(self.h, w.ctypes.data_as(c_u64p), len(w)))

    def mcd_set_basis_device(self, words):
        """Install a basis held in a device uint64/int64 torch tensor."""
        self._sync_stream()
        return self._check(self.L.mcd_set_basis_device(self.h, _ptr(words), words.numel()))

    def mcd_save_basis(self, path):
        self._check(self.L.mcd_save_basis(self.h, os.fsencode(path)))

    def mcd_load_basis(self, path):
        self._sync_stream()
        self._check(self.L.mcd_load_basis(self.h, os.fsencode(path)))

    def mcd_launch_count(self) -> int:
        n = ctypes.c_int64(0)
        self._check(self.L.mcd_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def mcd_get_basis(self) -> np.ndarray:
        n = ctypes.c_int64(0)
        self._check(self.L.mcd_get_basis(self.h, None, 0, ctypes.byref(n)))
        out = np.empty(n.value, dtype=np.uint64)
        self._check(self.L.mcd_get_basis(self.h, out.ctypes.data_as(c_u64p), len(out), ctypes.byref(n)))
        return out

    def mcd_hv_cache_info(self) -> dict:
        """Connection cache of the current basis: record bytes (with padding),
        stored hops, bytes per record (zeros when none is built) and whether a
        bounded wait in a cached kernel ran out."""
        b, n, r, w = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_int(0)
        self._sync_stream()
        self._check(self.L.mcd_hv_cache_info(self.h, ctypes.byref(b), ctypes.byref(n), ctypes.byref(r),
                                             ctypes.byref(w)))
        return {"bytes": b.value, "n_conn": n.value, "rec_bytes": r.value, "wait_errors": w.value}

    def mcd_basis_info(self, nnz: bool = True) -> dict:
        v = [ctypes.c_int64(0) for _ in range(4)]
        self._sync_stream()
        self._check(self.L.mcd_basis_info(self.h, *(ctypes.byref(x) for x in v[:3]),
                                          ctypes.byref(v[3]) if nnz else None))
        return {"n_states": v[0].value, "n_up_blocks": v[1].value, "n_dn_blocks": v[2].value,
                "nnz_offdiag": v[3].value if nnz else None}

    def mcd_apply(self, x, y, ncols: int | None = None, ld: int | None = None):
        """y = H~ x for torch tensors [n] or [n, ld] on this device."""
        if x.dim() == 1:
            nc, l = 1, 1
        else:
            nc, l = x.shape[1], x.stride(0)
        nc = nc if ncols is None else ncols
        l = l if ld is None else ld
        self._sync_stream()
        return self._check(self.L.mcd_apply(self.h, _ptr(x), _ptr(y), nc, l, _dtype_code(x)))

    def mcd_hv_adjoint(self, u, v):
        """(grad_t [n, n], grad_eps [n], grad_U [n]) of <u, H~ v> (torch device tensors)."""
        n = self.n_sites
        gt, ge, gu = np.zeros((n, n)), np.zeros(n), np.zeros(n)
        nc, l = (1, 1) if u.dim() == 1 else (u.shape[1], u.stride(0))
        self._sync_stream()
        self._check(self.L.mcd_hv_adjoint(self.h, _ptr(u), _ptr(v), nc, l, _dtype_code(u),
                                          gt.ctypes.data_as(c_dp), ge.ctypes.data_as(c_dp),
                                          gu.ctypes.data_as(c_dp)))
        return gt, ge, gu

    def mcd_diagonal(self, out):
        self._sync_stream()
        return self._check(self.L.mcd_diagonal(self.h, _ptr(out)))

    def mcd_connections(self, rows=None, cols=None, vals=None) -> int:
        n = ctypes.c_int64(0)
        cap = 0 if rows is None else rows.numel()
        self._sync_stream()
        self._check(self.L.mcd_connections(self.h, _ptr(rows) or None, _ptr(cols) or None,
                                           _ptr(vals) or None, cap, ctypes.byref(n)))
        return n.value

    def mcd_connections_noalloc(self, rows=None, cols=None, vals=None) -> int:
        """mcd_connections without any device allocation (fixed scratch, at
        most 262144 states)."""
        n = ctypes.c_int64(0)
        cap = 0 if rows is None else rows.numel()
        self._sync_stream()
        self._check(self.L.mcd_connections_noalloc(self.h, _ptr(rows) or None, _ptr(cols) or None,
                                                   _ptr(vals) or None, cap, ctypes.byref(n)))
        return n.value

    def mcd_lanczos_ground(self, max_iter: int, tol: float, seed: int, dtype: int, psi=None,
                           allow_not_converged: bool = False) -> dict:
        E0, res = ctypes.c_double(0), ctypes.c_double(0)
        it = ctypes.c_int(0)
        self._sync_stream()
        st = self.L.mcd_lanczos_ground(self.h, max_iter, tol, seed, dtype, ctypes.byref(E0),
                                       _ptr(psi) or None, ctypes.byref(it), ctypes.byref(res))
        self._check(st, ok=(MCD_OK, -5) if allow_not_converged else (MCD_OK,))
        return {"status": st, "E0": E0.value, "iters": it.value, "residual": res.value}

    def mcd_lanczos_coeffs(self):
        m = ctypes.c_int(0)
        self._check(self.L.mcd_lanczos_coeffs(self.h, None, None, 0, ctypes.byref(m)))
        a, b = np.zeros(m.value), np.zeros(m.value)
        self._check(self.L.mcd_lanczos_coeffs(self.h, a.ctypes.data_as(c_dp), b.ctypes.data_as(c_dp),
                                              m.value, ctypes.byref(m)))
        return a, b

    def mcd_band_lanczos_green(self, orbitals, n_block_iter: int, w_t: float, z, dtype: int = MCD_F64):
        """G[nz, L, L] (complex) of the last ground state; orbitals = [(site, spin)]."""
        L = len(orbitals)
        site = (ctypes.c_int * L)(*[int(o[0]) for o in orbitals])
        spin = (ctypes.c_int * L)(*[int(o[1]) for o in orbitals])
        z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.complex128)
        zr, zi = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        gr = np.zeros((len(z), L, L))
        gi = np.zeros((len(z), L, L))
        dp, dm = ctypes.c_int64(0), ctypes.c_int64(0)
        self._sync_stream()
        self._check(self.L.mcd_band_lanczos_green(self.h, site, spin, L, n_block_iter, w_t, dtype,
                                                  zr.ctypes.data_as(c_dp), zi.ctypes.data_as(c_dp), len(z),
                                                  gr.ctypes.data_as(c_dp), gi.ctypes.data_as(c_dp),
                                                  ctypes.byref(dp), ctypes.byref(dm)))
        return gr + 1j * gi, dp.value, dm.value

    def mcd_green_gradient(self, orbitals, n_block_iter: int, w_t: float, z, gG, cg_tol: float = 1e-11,
                           allow_not_converged: bool = False):
        """Gradient of sum Re(conj(gG) G) = sum gG.re Re G + gG.im Im G with respect
        to (t [n, n], eps [n], U [n]); gG: complex [nz, L, L].  Returns
        (grad_t, grad_eps, grad_U, cg_iters)."""
        L = len(orbitals)
        site = (ctypes.c_int * L)(*[int(o[0]) for o in orbitals])
        spin = (ctypes.c_int * L)(*[int(o[1]) for o in orbitals])
        z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.complex128)
        zr, zi = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        gG = np.asarray(gG, dtype=np.complex128).reshape(len(z), L, L)
        gr, gi = np.ascontiguousarray(gG.real), np.ascontiguousarray(gG.imag)
        n = self.n_sites
        gt, ge, gu = np.zeros((n, n)), np.zeros(n), np.zeros(n)
        it = ctypes.c_int(0)
        self._sync_stream()
        st = self.L.mcd_green_gradient(self.h, site, spin, L, n_block_iter, w_t, zr.ctypes.data_as(c_dp),
                                       zi.ctypes.data_as(c_dp), len(z), gr.ctypes.data_as(c_dp),
                                       gi.ctypes.data_as(c_dp), cg_tol, gt.ctypes.data_as(c_dp),
                                       ge.ctypes.data_as(c_dp), gu.ctypes.data_as(c_dp), ctypes.byref(it))
        self._check(st, ok=(MCD_OK, MCD_E_NOT_CONVERGED) if allow_not_converged else (MCD_OK,))
        return gt, ge, gu, it.value

    def mcd_kernel_times(self, reset: bool = False):
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_int64 * 4)()
        self._check(self.L.mcd_kernel_times(self.h, ms, cnt, 4, int(reset)))
        return list(ms), list(cnt)
