"""Thin Python binding of libfnl (ctypes): argument marshalling only.

Every step of the path runs in the CUDA kernels behind the C ABI declared in
``include/fnl.h``; PyTorch only provides device memory and the current stream.
Importing this module raises if ``libfnl.so`` has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfnl.so")

FNL_FP64, FNL_FP32, FNL_BF16X2, FNL_BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": FNL_FP64, "fp32": FNL_FP32, "bf16x2": FNL_BF16X2, "bf16x3": FNL_BF16X3}
STATUS = {0: "FNL_OK", 1: "FNL_EINVAL", 2: "FNL_ENOMEM", 3: "FNL_ECUDA", 4: "FNL_EUNSUPPORTED", 5: "FNL_ETIMEOUT"}

# Every symbol include/fnl.h declares.
EXPORTS = [
    "fnl_version", "fnl_last_error", "fnl_make_shells", "fnl_shells_destroy", "fnl_shells_info",
    "fnl_shells_mu", "fnl_generate", "fnl_filter", "fnl_synth", "fnl_analyse", "fnl_square",
    "fnl_accumulate", "fnl_gauss_legendre", "fnl_covariance", "fnl_cholesky_filters",
    "fnl_profile_enable", "fnl_profile_read", "fnl_generate_host", "fnl_device_status",
    "fnl_accumulate_noalloc", "fnl_generate_backward", "fnl_batch_create", "fnl_batch_destroy",
    "fnl_batch_info", "fnl_generate_batch", "fnl_shells_autotune", "fnl_shells_set_tiles", "fnl_batch_tiles",
    "fnl_maps_prepare", "fnl_maps", "fnl_ksw_create", "fnl_ksw_destroy", "fnl_ksw_info", "fnl_ksw_statistic",
    "fnl_quad_create", "fnl_quad_destroy", "fnl_quad_moments", "fnl_quad_greedy", "fnl_quad_fit", "fnl_quad_error",
    "fnl_make_shells_healpix", "fnl_shells_set_sm_limits", "fnl_test_fail_alloc", "fnl_test_wait_expiry",
    "fnl_measure_fma_peaks", "fnl_make_shells_shard", "fnl_shells_shard", "fnl_shells_gemm_work",
]
STAGES = ["filter", "synthesis_gemm", "ring_fft_square", "analysis_gemm", "quadrature"]


class FnlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class ShellDesc(ctypes.Structure):
    _fields_ = [
        ("lmax", ctypes.c_int), ("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("nphi", ctypes.c_int),
        ("r", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
        ("K", ctypes.POINTER(ctypes.c_double)),
        ("A", ctypes.c_double), ("ns", ctypes.c_double), ("kmin", ctypes.c_double), ("kmax", ctypes.c_double),
        ("nk", ctypes.c_int), ("jitter_rel", ctypes.c_double),
        ("alphaT", ctypes.POINTER(ctypes.c_double)), ("alphaE", ctypes.POINTER(ctypes.c_double)),
        ("mu", ctypes.POINTER(ctypes.c_double)), ("prec", ctypes.c_int),
    ]


class QuadDesc(ctypes.Structure):
    _fields_ = [
        ("lmax", ctypes.c_int), ("ntot", ctypes.c_int),
        ("r", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
        ("alphaT", ctypes.POINTER(ctypes.c_double)), ("alphaE", ctypes.POINTER(ctypes.c_double)),
        ("P", ctypes.POINTER(ctypes.c_double)),
        ("A", ctypes.c_double), ("ns", ctypes.c_double), ("kmin", ctypes.c_double), ("kmax", ctypes.c_double),
        ("nk", ctypes.c_int), ("jitter_rel", ctypes.c_double),
    ]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfnl.so (built in-tree by paper_0909_0009_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_0909_0009_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, d, u64, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    lib.fnl_version.restype = ctypes.c_char_p
    lib.fnl_last_error.restype = ctypes.c_char_p
    lib.fnl_make_shells.argtypes = [ctypes.POINTER(ShellDesc), i, ctypes.POINTER(vp)]
    lib.fnl_shells_destroy.argtypes = [vp]
    lib.fnl_shells_destroy.restype = None
    lib.fnl_shells_info.argtypes = [vp] + [ctypes.POINTER(i)] * 5 + [ctypes.POINTER(ctypes.c_size_t)]
    lib.fnl_shells_mu.argtypes = [vp, dp]
    lib.fnl_generate.argtypes = [vp, u64, u64, d, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.fnl_filter.argtypes = [vp, u64, u64, vp, vp, vp]
    lib.fnl_synth.argtypes = [vp, vp, vp, vp]
    lib.fnl_analyse.argtypes = [vp, vp, vp, vp]
    lib.fnl_square.argtypes = [vp, vp, vp, vp]
    lib.fnl_accumulate.argtypes = [vp, vp, vp, d, vp, vp, vp, vp, vp, vp, vp]
    lib.fnl_gauss_legendre.argtypes = [i, dp, dp]
    lib.fnl_covariance.argtypes = [i, i, dp, d, d, d, d, i, dp]
    lib.fnl_cholesky_filters.argtypes = [i, i, dp, d, dp]
    lib.fnl_profile_enable.argtypes = [vp, i]
    lib.fnl_profile_read.argtypes = [vp, dp, i, ctypes.POINTER(i)]
    lib.fnl_generate_host.argtypes = [vp, u64, u64, d, vp, vp, vp, vp, vp]
    lib.fnl_device_status.argtypes = [vp]
    lib.fnl_test_fail_alloc.argtypes = [ctypes.c_long]
    lib.fnl_test_wait_expiry.argtypes = [vp, ctypes.c_uint, vp]
    lib.fnl_measure_fma_peaks.argtypes = [i, dp, dp]
    lib.fnl_accumulate_noalloc.argtypes = [i, i, vp, vp, vp, vp, vp, vp, d, vp, vp, vp, vp, vp, vp, vp]
    lib.fnl_generate_backward.argtypes = [vp, u64, u64, d, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.fnl_batch_create.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(vp)]
    lib.fnl_batch_destroy.argtypes = [vp]
    lib.fnl_batch_destroy.restype = None
    lib.fnl_batch_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.fnl_generate_batch.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), dp, ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), vp]
    lib.fnl_shells_autotune.argtypes = [vp, vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.fnl_shells_set_tiles.argtypes = [vp, i, i]
    lib.fnl_batch_tiles.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.fnl_maps_prepare.argtypes = [vp]
    lib.fnl_maps.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.fnl_ksw_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.fnl_ksw_destroy.argtypes = [vp]
    lib.fnl_ksw_destroy.restype = None
    lib.fnl_ksw_info.argtypes = [vp, dp, dp, ctypes.POINTER(i)]
    lib.fnl_ksw_statistic.argtypes = [vp, vp, vp, vp, vp]
    lib.fnl_quad_create.argtypes = [ctypes.POINTER(QuadDesc), i, ctypes.POINTER(vp)]
    lib.fnl_quad_destroy.argtypes = [vp]
    lib.fnl_quad_destroy.restype = None
    lib.fnl_quad_moments.argtypes = [vp, dp, dp]
    lib.fnl_quad_greedy.argtypes = [vp, i, ctypes.POINTER(i), dp, dp, dp, dp]
    lib.fnl_quad_error.argtypes = [vp, i, ctypes.POINTER(i), dp, dp]
    lib.fnl_quad_fit.argtypes = [vp, i, ctypes.POINTER(i), dp, dp]
    lib.fnl_make_shells_healpix.argtypes = [ctypes.POINTER(ShellDesc), i, i, ctypes.POINTER(vp)]
    lib.fnl_shells_set_sm_limits.argtypes = [vp, i, i]
    lib.fnl_make_shells_shard.argtypes = [ctypes.POINTER(ShellDesc), i, i, i, ctypes.POINTER(vp)]
    lib.fnl_shells_shard.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.fnl_shells_gemm_work.argtypes = [vp, dp, dp]
    for name in EXPORTS:
        if name not in ("fnl_version", "fnl_last_error", "fnl_shells_destroy", "fnl_batch_destroy", "fnl_ksw_destroy",
                        "fnl_quad_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != 0:
        raise FnlError(code, _lib.fnl_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- host helpers (no GPU needed) -----------------------------------------------------

def gauss_legendre(n: int):
    lib = load_library()
    x = np.empty(n)
    w = np.empty(n)
    _check(lib.fnl_gauss_legendre(n, _dptr(x), _dptr(w)))
    return x, w


def covariance(lmax, r, A, ns, kmin, kmax, nk):
    lib = load_library()
    r = np.ascontiguousarray(r, dtype=np.float64)
    C = np.empty((lmax + 1, r.size, r.size))
    _check(lib.fnl_covariance(lmax, r.size, _dptr(r), A, ns, kmin, kmax, nk, _dptr(C)))
    return C


def cholesky_filters(C, jitter_rel):
    lib = load_library()
    C = np.ascontiguousarray(C, dtype=np.float64)
    K = np.empty_like(C)
    _check(lib.fnl_cholesky_filters(C.shape[0] - 1, C.shape[1], _dptr(C), jitter_rel, _dptr(K)))
    return K


# ---- device objects -----------------------------------------------------------------

def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Cov:
    A: float = 1.6e-8
    ns: float = 0.96
    kmin: float = 1e-4
    kmax: float = 0.3
    nk: int = 4096
    jitter_rel: float = 1e-10


class Shells:
    """Device tables and scratch for one configuration (wraps fnl_make_shells)."""

    def __init__(self, lmax, nr, ntheta, nphi, r, w, alphaT, alphaE, K=None, cov: Cov | None = None,
                 mu=None, prec="fp64", device=0, nside: int | None = None, shard: tuple | None = None):
        """Gauss-Legendre ring grid of ntheta x nphi; or, with nside, the HEALPix grid of
        12 nside^2 pixels (fnl_make_shells_healpix; ntheta and nphi are then ignored and maps are
        [nr][npix] in RING order).  With shard = (j0, j1) the object is the shell shard
        [j0, j1) of the nr-shell configuration described (fnl_make_shells_shard): its per-shell
        arrays have j1 - j0 shells and fnl_generate returns its partial sums."""
        lib = load_library()
        if nside:
            ntheta, nphi = 4 * nside - 1, 4 * nside
        cov = cov or Cov()
        self._keep = []

        def arr(a, shape):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(shape)
            self._keep.append(a)
            return _dptr(a)

        d = ShellDesc()
        d.lmax, d.nr, d.ntheta, d.nphi = lmax, nr, ntheta, nphi
        d.r, d.w = arr(r, (nr,)), arr(w, (nr,))
        d.K = arr(K, (lmax + 1, nr, nr))
        d.A, d.ns, d.kmin, d.kmax, d.nk, d.jitter_rel = cov.A, cov.ns, cov.kmin, cov.kmax, cov.nk, cov.jitter_rel
        d.alphaT, d.alphaE = arr(alphaT, (lmax + 1, nr)), arr(alphaE, (lmax + 1, nr))
        d.mu = arr(mu, (nr,))
        d.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        h = ctypes.c_void_p()
        if nside:
            assert shard is None, "shell shards are made on the Gauss-Legendre grid"
            _check(lib.fnl_make_shells_healpix(ctypes.byref(d), int(nside), device, ctypes.byref(h)))
        elif shard is not None:
            _check(lib.fnl_make_shells_shard(ctypes.byref(d), int(shard[0]), int(shard[1]), device,
                                             ctypes.byref(h)))
        else:
            _check(lib.fnl_make_shells(ctypes.byref(d), device, ctypes.byref(h)))
        self.nside = nside or 0
        self.npix = 12 * nside * nside if nside else ntheta * nphi
        self._keep = []
        self.handle = h
        self.j0, self.nr_total = (int(shard[0]), nr) if shard is not None else (0, nr)
        nr = int(shard[1]) - int(shard[0]) if shard is not None else nr
        self.lmax, self.nr, self.ntheta, self.nphi = lmax, nr, ntheta, nphi
        self.nalm = (lmax + 1) * (lmax + 2) // 2
        self.device = device
        self.prec = d.prec

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.fnl_shells_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def mu(self) -> np.ndarray:
        out = np.empty(self.nr)
        _check(_lib.fnl_shells_mu(self.handle, _dptr(out)))
        return out

    def device_status(self):
        """Synchronise and raise FnlError(FNL_ETIMEOUT) if a bounded device wait expired."""
        _check(_lib.fnl_device_status(self.handle))

    @property
    def device_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(_lib.fnl_shells_info(self.handle, None, None, None, None, None, ctypes.byref(b)))
        return b.value

    def profile(self, slots: int = 256):
        """Time the stages of fnl_generate with CUDA events on the launching stream
        (a ring of `slots` calls; 0 turns profiling off)."""
        _check(_lib.fnl_profile_enable(self.handle, int(slots)))

    def stage_ms(self) -> tuple[dict, int]:
        """Stage durations (ms) summed over the profiled calls since the last read, and their count."""
        ms = np.zeros(len(STAGES))
        n = ctypes.c_int()
        _check(_lib.fnl_profile_read(self.handle, _dptr(ms), len(STAGES), ctypes.byref(n)))
        return dict(zip(STAGES, ms.tolist())), n.value

    def generate_host(self, seed: int, realisation: int, fnl: float, aT: np.ndarray, aE: np.ndarray,
                      aNLT=None, aNLE=None, stream=None):
        """fnl_generate with host outputs (complex128 arrays of nalm, any but aT/aE may be None):
        page-locked arrays are written by the path's last kernel, others receive a copy.  The
        caller synchronises the stream before reading them."""
        def hp(a):
            if a is None:
                return None
            assert a.dtype == np.complex128 and a.flags.c_contiguous and a.size == self.nalm
            return ctypes.c_void_p(a.ctypes.data)
        _check(_lib.fnl_generate_host(self.handle, seed, realisation, float(fnl), hp(aT), hp(aE), hp(aNLT),
                                      hp(aNLE), _stream(stream)))

    def set_sm_limits(self, gemm: int = 0, ring: int = 0):
        """SMs the persistent GEMM and ring kernels may occupy (0: all)."""
        _check(_lib.fnl_shells_set_sm_limits(self.handle, int(gemm), int(ring)))

    def autotune(self, stream=None) -> tuple[int, int]:
        """fnl_shells_autotune: time the candidate tile shapes, keep the fastest; returns
        (synthesis width, analysis width cap)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(_lib.fnl_shells_autotune(self.handle, _stream(stream), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_tiles(self, syn_cap: int, ana_cap: int):
        _check(_lib.fnl_shells_set_tiles(self.handle, int(syn_cap), int(ana_cap)))

    def gemm_work(self) -> tuple[float, float]:
        """fnl_shells_gemm_work: the shares of the dense Legendre work the synthesis and the
        analysis GEMMs execute (the polar ring pairs of negligible lambda are left out)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(_lib.fnl_shells_gemm_work(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # -- tensors
    def _alm(self, n=None):
        """complex128 [nalm] (n None) or [nalm, n] on the object's device."""
        torch = _torch()
        return torch.empty((self.nalm,) if n is None else (self.nalm, n), dtype=torch.complex128,
                           device=f"cuda:{self.device}")

    def generate(self, seed: int, realisation: int, fnl: float, noise=None, parts: bool = True,
                 out: dict | None = None, stream=None) -> dict:
        """One realisation; returns complex128 tensors aT, aE (and aLT, aLE, aNLT, aNLE if parts)."""
        names = ["aT", "aE"] + (["aLT", "aLE", "aNLT", "aNLE"] if parts else [])
        if out is None:
            out = {k: self._alm() for k in names}
        ptrs = [_ptr(out.get(k)) for k in ["aT", "aE", "aLT", "aLE", "aNLT", "aNLE"]]
        if noise is not None:  # shells 0 .. j0 + nr - 1 of the configuration
            assert (noise.dtype == _torch().complex128 and noise.is_contiguous()
                    and noise.shape == (self.j0 + self.nr, self.nalm))
        _check(_lib.fnl_generate(self.handle, seed, realisation, float(fnl), _ptr(noise), *ptrs, _stream(stream)))
        return out

    def generate_backward(self, seed: int, realisation: int, fnl: float, gT=None, gE=None, noise=None,
                          aNLT=None, aNLE=None, want_noise: bool = True, want_fnl: bool = True, stream=None):
        """Adjoint of ``generate`` (fnl_generate_backward): given gX = dL/da^X of a real loss
        (complex128 [nalm], dL/dRe + i dL/dIm, or None for zero), returns (dL/dn as complex128
        [nr, nalm] or None, dL/df_NL as a float64 0-d tensor or None) for the noise of the same
        call (explicit ``noise``, else the Philox draw of seed and realisation).  aNLT/aNLE from
        the forward call spare one forward pass when dL/df_NL is wanted."""
        torch = _torch()
        for t in (gT, gE, noise, aNLT, aNLE):
            if t is not None:
                assert t.dtype == torch.complex128 and t.is_contiguous()
        gn = torch.empty((self.nr, self.nalm), dtype=torch.complex128,
                         device=f"cuda:{self.device}") if want_noise else None
        gf = torch.empty((), dtype=torch.float64, device=f"cuda:{self.device}") if want_fnl else None
        _check(_lib.fnl_generate_backward(self.handle, seed, realisation, float(fnl), _ptr(noise), _ptr(gT),
                                          _ptr(gE), _ptr(aNLT), _ptr(aNLE), _ptr(gn), _ptr(gf), _stream(stream)))
        return gn, gf

    def filter(self, seed: int = 0, realisation: int = 0, noise=None, stream=None):
        phi = self._alm(self.nr)
        _check(_lib.fnl_filter(self.handle, seed, realisation, _ptr(noise), _ptr(phi), _stream(stream)))
        return phi

    def synth(self, alm, stream=None):
        torch = _torch()
        assert alm.dtype == torch.complex128 and alm.is_contiguous() and alm.shape == (self.nalm, self.nr)
        shape = (self.nr, self.npix) if self.nside else (self.nr, self.ntheta, self.nphi)
        maps = torch.empty(shape, dtype=torch.float64, device=alm.device)
        _check(_lib.fnl_synth(self.handle, _ptr(alm), _ptr(maps), _stream(stream)))
        return maps

    def analyse(self, maps, stream=None):
        torch = _torch()
        shape = (self.nr, self.npix) if self.nside else (self.nr, self.ntheta, self.nphi)
        assert maps.dtype == torch.float64 and maps.is_contiguous() and maps.shape == shape
        alm = self._alm(self.nr)
        _check(_lib.fnl_analyse(self.handle, _ptr(maps), _ptr(alm), _stream(stream)))
        return alm

    def square(self, phiL, stream=None):
        torch = _torch()
        assert phiL.dtype == torch.complex128 and phiL.is_contiguous() and phiL.shape == (self.nalm, self.nr)
        out = self._alm(self.nr)
        _check(_lib.fnl_square(self.handle, _ptr(phiL), _ptr(out), _stream(stream)))
        return out

    def maps_prepare(self):
        """Spin-0 and spin-2 tables of the Stokes maps (fnl_maps_prepare; synchronous, allocates)."""
        _check(_lib.fnl_maps_prepare(self.handle))

    def maps(self, aT, aE, aB=None, out=None, stream=None):
        """Stokes maps [3, ntheta, nphi] = (I, Q, U) of aT, aE and aB (complex128 [nalm] on the
        device; aB None for zero B modes) on the object's grid (fnl_maps)."""
        torch = _torch()
        for a in (aT, aE) + ((aB,) if aB is not None else ()):
            assert a.dtype == torch.complex128 and a.is_contiguous() and a.shape == (self.nalm,)
        if out is None:
            out = torch.empty((3, self.ntheta, self.nphi), dtype=torch.float64, device=aT.device)
        assert out.dtype == torch.float64 and out.is_contiguous() and out.shape == (3, self.ntheta, self.nphi)
        _check(_lib.fnl_maps(self.handle, _ptr(aT), _ptr(aE), _ptr(aB), _ptr(out), _stream(stream)))
        return out

    def accumulate(self, phiL=None, phiNL=None, fnl: float = 0.0, stream=None) -> dict:
        out = {k: self._alm() for k in ["aT", "aE", "aLT", "aLE", "aNLT", "aNLE"]}
        ptrs = [_ptr(out[k]) for k in ["aT", "aE", "aLT", "aLE", "aNLT", "aNLE"]]
        _check(_lib.fnl_accumulate(self.handle, _ptr(phiL), _ptr(phiNL), float(fnl), *ptrs, _stream(stream)))
        return out


class Ksw:
    """The fast cubic f_NL estimator of Sect. 5 (fnl_ksw_*) for the configuration of a shells
    object: S_prim of a sky (a^T, a^E) and the normalisation N, f_NL = S_prim / N."""

    def __init__(self, shells: "Shells"):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.fnl_ksw_create(shells.handle, ctypes.byref(h)))
        self.handle = h
        self.shells = shells  # the estimator keeps pointers into it
        norm, secs = ctypes.c_double(), ctypes.c_double()
        rank = (ctypes.c_int * (shells.lmax + 1))()
        _check(lib.fnl_ksw_info(h, ctypes.byref(norm), ctypes.byref(secs), rank))
        self.norm = norm.value
        self.norm_seconds = secs.value
        self.rank = np.array(rank[:], dtype=int)

    def statistic(self, aT, aE, out=None, stream=None):
        """S_prim as a 0-d float64 device tensor (asynchronous)."""
        torch = _torch()
        for a in (aT, aE):
            assert a.dtype == torch.complex128 and a.is_contiguous() and a.shape == (self.shells.nalm,)
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=aT.device)
        _check(_lib.fnl_ksw_statistic(self.handle, _ptr(aT), _ptr(aE), _ptr(out), _stream(stream)))
        return out

    def fnl(self, aT, aE, stream=None) -> float:
        """The estimate S_prim / N (synchronises)."""
        return float(self.statistic(aT, aE, stream=stream).item()) / self.norm

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.fnl_ksw_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Quadrature:
    """Optimal radial quadrature of Sect. 3 (fnl_quad_*): the fine-grid covariance and moments
    are built at construction (on the device unless P is given); greedy() selects nodes and
    optimal weights, error() evaluates any rule."""

    def __init__(self, lmax: int, r, w, alphaT, alphaE, P=None, cov: "Cov" = None, device: int = 0):
        lib = load_library()
        cov = cov or Cov()
        self.lmax, self.ntot = lmax, len(r)
        keep = []

        def arr(a, shape):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(shape)
            keep.append(a)
            return _dptr(a)

        d = QuadDesc()
        d.lmax, d.ntot = lmax, self.ntot
        d.r, d.w = arr(r, (self.ntot,)), arr(w, (self.ntot,))
        d.alphaT, d.alphaE = arr(alphaT, (lmax + 1, self.ntot)), arr(alphaE, (lmax + 1, self.ntot))
        d.P = arr(P, (lmax + 1, self.ntot, self.ntot))
        d.A, d.ns, d.kmin, d.kmax, d.nk, d.jitter_rel = cov.A, cov.ns, cov.kmin, cov.kmax, cov.nk, cov.jitter_rel
        h = ctypes.c_void_p()
        _check(lib.fnl_quad_create(ctypes.byref(d), device, ctypes.byref(h)))
        self.handle = h
        I2 = np.zeros((2, lmax + 1))
        sec = ctypes.c_double()
        _check(lib.fnl_quad_moments(h, _dptr(I2), ctypes.byref(sec)))
        self.I2, self.create_seconds = I2, sec.value

    def greedy(self, nsel: int) -> dict:
        nodes = (ctypes.c_int * nsel)()
        W = np.zeros((2, self.lmax + 1, nsel))
        obj = np.zeros(nsel)
        rel = np.zeros((2, self.lmax + 1))
        sec = ctypes.c_double()
        _check(_lib.fnl_quad_greedy(self.handle, nsel, nodes, _dptr(W), _dptr(obj), _dptr(rel), ctypes.byref(sec)))
        return {"nodes": list(nodes), "weights": W, "objective": obj, "rel_err": rel, "seconds": sec.value}

    def fit(self, nodes) -> dict:
        """Optimal weights and relative errors of the given distinct fine nodes."""
        n = len(nodes)
        nd = (ctypes.c_int * n)(*[int(x) for x in nodes])
        W = np.zeros((2, self.lmax + 1, n))
        rel = np.zeros((2, self.lmax + 1))
        _check(_lib.fnl_quad_fit(self.handle, n, nd, _dptr(W), _dptr(rel)))
        return {"weights": W, "rel_err": rel}

    def error(self, nodes, weights) -> np.ndarray:
        n = len(nodes)
        nd = (ctypes.c_int * n)(*[int(x) for x in nodes])
        W = np.ascontiguousarray(weights, dtype=np.float64).reshape(2, self.lmax + 1, n)
        rel = np.zeros((2, self.lmax + 1))
        _check(_lib.fnl_quad_error(self.handle, n, nd, _dptr(W), _dptr(rel)))
        return rel

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.fnl_quad_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batching form (fnl_batch_create / fnl_generate_batch): n instances over shells objects
    of any l_max and N_r, launched as one captured CUDA graph per call."""

    def __init__(self, shells: list, nstreams: int = 0):
        lib = load_library()
        self.shells = list(shells)  # keeps the objects alive as long as the batch
        arr = (ctypes.c_void_p * len(self.shells))(*[s.handle.value for s in self.shells])
        h = ctypes.c_void_p()
        _check(lib.fnl_batch_create(arr, len(self.shells), int(nstreams), ctypes.byref(h)))
        self.handle = h
        self.n = len(self.shells)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.fnl_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def multi(self) -> bool:
        """True when every stage runs as one launch over all instances."""
        n, ns = ctypes.c_int(), ctypes.c_int()
        _check(_lib.fnl_batch_info(self.handle, ctypes.byref(n), ctypes.byref(ns), None))
        return ns.value == 0

    def tiles(self) -> tuple[int, int]:
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(_lib.fnl_batch_tiles(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def lanes(self) -> list:
        n, ns = ctypes.c_int(), ctypes.c_int()
        lanes = (ctypes.c_int * self.n)()
        _check(_lib.fnl_batch_info(self.handle, ctypes.byref(n), ctypes.byref(ns), lanes))
        return list(lanes)

    def generate(self, seeds, realisations, fnl, out=None, stream=None) -> list:
        """Returns (or fills) a list of (aT, aE) complex128 tensors, one pair per instance."""
        if out is None:
            out = [(s._alm(), s._alm()) for s in self.shells]
        n = self.n
        sd = (ctypes.c_uint64 * n)(*[int(x) for x in seeds])
        rl = (ctypes.c_uint64 * n)(*[int(x) for x in realisations])
        fv = np.ascontiguousarray(fnl, dtype=np.float64)
        assert fv.size == n
        pT = (ctypes.c_void_p * n)(*[o[0].data_ptr() for o in out])
        pE = (ctypes.c_void_p * n)(*[o[1].data_ptr() for o in out])
        _check(_lib.fnl_generate_batch(self.handle, sd, rl, _dptr(fv), pT, pE, _stream(stream)))
        return out


def measure_fma_peaks(device: int = 0) -> tuple[float, float]:
    """(FP64, FP32) fused multiply-add rates of the device in TFLOP/s, measured by the library."""
    lib = load_library()
    d64, d32 = ctypes.c_double(), ctypes.c_double()
    _check(lib.fnl_measure_fma_peaks(int(device), ctypes.byref(d64), ctypes.byref(d32)))
    return d64.value, d32.value


NOALLOC_OUTPUTS = ["aT", "aE", "aLT", "aLE", "aNLT", "aNLE"]


def accumulate_noalloc(lmax, nr, r, w, alphaT, alphaE, phiL=None, phiNL=None, fnl: float = 0.0, out=None,
                       stream=None):
    """Step (v) through fnl_accumulate_noalloc, which allocates no device memory.

    For callers that may not allocate (their device memory belongs to another allocator,
    or cudaMalloc's device synchronisation is not acceptable where they run): every array
    is the caller's, on the current device -- r, w (float64 [nr]), alphaT, alphaE (float64
    [lmax+1, nr]), phiL, phiNL (complex128 [nalm, nr] or None) -- and ``out`` maps any of
    aT, aE, aLT, aLE, aNLT, aNLE to a complex128 [nalm] tensor the call fills.  This wrapper
    allocates nothing either.  Calls share one scratch array in the library: calls that
    overlap on the GPU race.
    """
    lib = load_library()
    torch = _torch()
    out = out or {}
    bad = set(out) - set(NOALLOC_OUTPUTS)
    if bad:
        raise ValueError(f"unknown outputs {sorted(bad)}")
    lmax, nr = int(lmax), int(nr)
    nalm = (lmax + 1) * (lmax + 2) // 2
    dev = torch.cuda.current_device()

    def need(t, name, dtype, shape, nullable=False):
        # the library sees bare pointers: a wrong dtype, shape or device would make its
        # kernels read or write past the caller's buffers, so check before the call
        if t is None:
            if not nullable:
                raise ValueError(f"{name} must be given")
            return
        if t.dtype != dtype or tuple(t.shape) != shape:
            raise ValueError(f"{name} must be {dtype} of shape {shape}, got {t.dtype} {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device.type != "cuda" or t.device.index != dev:
            raise ValueError(f"{name} must be on the current device cuda:{dev}")

    need(r, "r", torch.float64, (nr,))
    need(w, "w", torch.float64, (nr,))
    need(alphaT, "alphaT", torch.float64, (lmax + 1, nr))
    need(alphaE, "alphaE", torch.float64, (lmax + 1, nr))
    need(phiL, "phiL", torch.complex128, (nalm, nr), nullable=True)
    need(phiNL, "phiNL", torch.complex128, (nalm, nr), nullable=True)
    for k, t in out.items():
        need(t, k, torch.complex128, (nalm,), nullable=True)
    ptrs = [_ptr(out.get(k)) for k in NOALLOC_OUTPUTS]
    _check(lib.fnl_accumulate_noalloc(lmax, nr, _ptr(r), _ptr(w), _ptr(alphaT), _ptr(alphaE), _ptr(phiL),
                                      _ptr(phiNL), float(fnl), *ptrs, _stream(stream)))
    return out
