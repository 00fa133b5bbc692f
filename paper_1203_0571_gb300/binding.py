"""ctypes binding of libfse (include/fse.h): argument marshalling only.

Every computation runs in the CUDA kernels behind the C ABI.  There is no
CPU path: if libfse.so cannot be built or loaded the import of a compute
entry point raises.

Names follow the ABI: ``Context.fit_batch`` calls ``fse_fit_batch``,
``Context.centroid`` calls ``fse_centroid`` and so on; the module-level
``fse_*`` functions take the context as their first argument, like the C
calls.  Device arrays are torch CUDA tensors; the stream is the current
torch stream unless one is given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _build

FSE_OK, FSE_EINVAL, FSE_ENOMEM, FSE_ECUDA, FSE_ETIMEOUT, FSE_EUNSUPPORTED = range(6)
FSE_F32, FSE_BF16 = 0, 1
FSE_FLAG_GRAPH = 1 << 0
FSE_MAX_PIX = 128 * 128

ST = dict(MOM_CONVERGED=1 << 0, FIT_CONVERGED=1 << 1, MOM_MAXITER=1 << 2, FIT_MAXITER=1 << 3,
          NONFINITE=1 << 4, BAD_SIZE=1 << 5, MOM_FAILED=1 << 6, FIT_BOUND=1 << 7,
          FIT_SINGULAR=1 << 8, NONPOS_FLUX=1 << 9, SIGW_CLAMPED=1 << 10, INIT_FALLBACK=1 << 11,
          TIMEOUT=1 << 12, MOM_REFINE2=1 << 13, FIT_REFINE2=1 << 14, NO_ROOM=1 << 15)

# exported symbols, in the order include/fse.h declares them
EXPORTS = ["fse_create", "fse_destroy", "fse_last_error", "fse_opts_default", "fse_centroid",
           "fse_ellipticity", "fse_sersic_fit", "fse_fit_batch", "fse_fit_batch_plain",
           "fse_fit_batch_host", "fse_fit_batch_ragged", "fse_autotune", "fse_tuning_save",
           "fse_tuning_load", "fse_tuning_read", "fse_tuned_warps", "fse_star_fit", "fse_moment_vjp", "fse_moment_jvp",
           "fse_cutout", "fse_sersic_b", "fse_sersic_chi2_grad", "fse_partition", "fse_sync_check",
           "fse_fit_batch_static"]
CUTOUT_DTYPE = np.dtype([("row0", "<i4"), ("col0", "<i4"), ("h", "<i4"), ("w", "<i4"), ("r50", "<f4"),
                         ("status", "<u4")])
FSE_MOM_ELLIP, FSE_MOM_SIGW_FIXED, FSE_MOM_SIGW_R50 = 1, 2, 4
FSE_STAR_GAUSS, FSE_STAR_MOFFAT = 0, 1
STAR_DTYPE = np.dtype([("size", "<f4"), ("beta", "<f4"), ("I0", "<f4"), ("flux", "<f4"), ("r50", "<f4"),
                       ("iters", "<i4"), ("status", "<u4"), ("reserved", "<f4")])


class Opts(ctypes.Structure):
    _fields_ = [("size", ctypes.c_size_t), ("tol_pos", ctypes.c_double), ("tol_g", ctypes.c_double),
                ("tol_sig", ctypes.c_double), ("tol_fit", ctypes.c_double),
                ("max_iter_mom", ctypes.c_int32), ("max_iter_fit", ctypes.c_int32),
                ("k_gain", ctypes.c_double), ("sigw_mode", ctypes.c_int32),
                ("max_pix", ctypes.c_int32), ("n_min", ctypes.c_double), ("n_max", ctypes.c_double),
                ("re_min", ctypes.c_double), ("re_max_frac", ctypes.c_double),
                ("lm_lambda0", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("warps_per_cta", ctypes.c_int32), ("warps_per_stamp", ctypes.c_int32),
                ("supersample", ctypes.c_int32)]


RESULT_DTYPE = np.dtype([("x0", "<f4"), ("y0", "<f4"), ("e1", "<f4"), ("e2", "<f4"), ("I0", "<f4"),
                         ("re", "<f4"), ("n", "<f4"), ("flux", "<f4"), ("chi2", "<f8"),
                         ("npix", "<i4"), ("it_mom", "<i4"), ("it_fit", "<i4"), ("status", "<u4"),
                         ("sigma_w", "<f4"), ("r50", "<f4")])
assert RESULT_DTYPE.itemsize == 64
STAMP_DTYPE = np.dtype([("offset", "<i8"), ("h", "<i4"), ("w", "<i4")])

_lib = None
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build: bool = True, path: str | None = None) -> ctypes.CDLL:
    """Load libfse.so (building it with nvcc first if it is missing or stale).

    `path` loads another build of the same ABI instead (for A/B comparisons)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libfse.so not found at {path}; run paper_1203_0571_gb300._build.build()")
    L = ctypes.CDLL(path)
    L.fse_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
    L.fse_destroy.argtypes = [_vp]
    L.fse_destroy.restype = None
    L.fse_last_error.argtypes = [_vp]
    L.fse_last_error.restype = ctypes.c_char_p
    L.fse_opts_default.argtypes = [ctypes.POINTER(Opts)]
    L.fse_opts_default.restype = None
    dev_sig = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp, ctypes.POINTER(Opts), _vp, _vp]
    for f in ("fse_centroid", "fse_ellipticity", "fse_sersic_fit", "fse_fit_batch",
              "fse_fit_batch_plain", "fse_fit_batch_ragged", "fse_autotune"):
        getattr(L, f).argtypes = dev_sig
        getattr(L, f).restype = ctypes.c_int
    L.fse_fit_batch_host.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int, _vp, _vp,
                                     ctypes.c_int64, _vp, ctypes.POINTER(Opts), _vp, _vp]
    L.fse_fit_batch_host.restype = ctypes.c_int
    L.fse_sersic_b.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp]
    L.fse_sersic_b.restype = ctypes.c_int
    L.fse_star_fit.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int,
                               ctypes.POINTER(Opts), _vp, _vp]
    L.fse_star_fit.restype = ctypes.c_int
    for f in ("fse_moment_vjp", "fse_moment_jvp"):
        getattr(L, f).argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int,
                                  _vp, _vp, _vp, _vp]
        getattr(L, f).restype = ctypes.c_int
    L.fse_cutout.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp]
    L.fse_cutout.restype = ctypes.c_int
    L.fse_tuned_warps.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32)]
    L.fse_tuned_warps.restype = ctypes.c_int
    L.fse_sersic_chi2_grad.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp, _vp,
                                       _vp, _vp, _vp, _vp, _vp]
    L.fse_sersic_chi2_grad.restype = ctypes.c_int
    L.fse_sync_check.argtypes = [_vp, _vp]
    L.fse_sync_check.restype = ctypes.c_int
    L.fse_fit_batch_static.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp,
                                       ctypes.POINTER(Opts), _vp, _vp, ctypes.c_char_p,
                                       ctypes.c_size_t]
    L.fse_fit_batch_static.restype = ctypes.c_int
    L.fse_partition.argtypes = [_vp, ctypes.c_int64, ctypes.c_int32, _vp]
    L.fse_partition.restype = ctypes.c_int
    for f in ("fse_tuning_save", "fse_tuning_load"):
        getattr(L, f).argtypes = [_vp, ctypes.c_char_p]
        getattr(L, f).restype = ctypes.c_int
    L.fse_tuning_read.argtypes = [ctypes.c_char_p, ctypes.c_char_p, _vp]
    L.fse_tuning_read.restype = ctypes.c_int
    _lib = L
    return L


def use_library(path: str) -> ctypes.CDLL:
    """Replace the loaded libfse with another build of the same ABI."""
    global _lib
    _lib = None
    return load(path=path)


def partition(index, parts: int) -> np.ndarray:
    """fse_partition: boundaries (parts + 1 int64) of contiguous index ranges of
    about equal total pixels, for replicas over stamp ranges.  index is a host
    array (make_index on the CPU, or a STAMP_DTYPE / int64 [N, 2] numpy array)."""
    if isinstance(index, torch.Tensor):
        index = index.detach().cpu().contiguous()
    ip, n = _index(index, where="cpu")
    starts = np.zeros(parts + 1, dtype=np.int64)
    rc = load().fse_partition(ip, n, int(parts), _vp(starts.ctypes.data))
    if rc != FSE_OK:
        raise FseError(rc, f"fse_partition(count={n}, parts={parts})")
    return starts


def tuning_read(path: str, device: str):
    """fse_tuning_read: the launch shapes a saved cache file holds for a device
    name, without a context or a GPU.  Returns (entries read, shapes) with
    shapes an int32 array [dtype, inv_var, class, (warps per CTA, warps per
    stamp)], -1 where the file has no entry for that dtype and setting."""
    shapes = np.zeros((2, 2, 7, 2), dtype=np.int32)
    n = load().fse_tuning_read(os.fsencode(path), device.encode(), _vp(shapes.ctypes.data))
    if n < 0:
        raise FseError(-n, f"fse_tuning_read({path!r})")
    return n, shapes


def default_opts(**kw) -> Opts:
    o = Opts()
    load().fse_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"fse_opts has no field {k}")
        setattr(o, k, v)
    return o


class FseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfse error {code}: {msg}")
        self.code = code


def make_index(offset, h, w, device="cuda") -> torch.Tensor:
    """fse_stamp array as an int64 tensor [N, 2]: (offset, h | w << 32)."""
    off = torch.as_tensor(offset, dtype=torch.int64)
    hh = torch.as_tensor(h, dtype=torch.int64)
    ww = torch.as_tensor(w, dtype=torch.int64)
    return torch.stack([off, hh | (ww << 32)], dim=1).contiguous().to(device)


def star_results(out: torch.Tensor) -> np.ndarray:
    """Copy a star result tensor (uint8 [N, 32]) to a numpy structured array."""
    return out.detach().cpu().contiguous().numpy().view(STAR_DTYPE).reshape(-1)


def cutout_info(info: torch.Tensor) -> np.ndarray:
    """Copy cut-out records (uint8 [N, 24]) to a numpy structured array."""
    return info.detach().cpu().contiguous().numpy().view(CUTOUT_DTYPE).reshape(-1)


def results(out: torch.Tensor) -> np.ndarray:
    """Copy a result tensor (uint8 [N, 64]) to a numpy structured array."""
    return out.detach().cpu().contiguous().numpy().view(RESULT_DTYPE).reshape(-1)


def _stream(stream) -> _vp:
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _index(index, where: str = "cuda"):
    """Pointer and count of an fse_stamp array, after checking its layout: a
    contiguous int64 tensor [N, 2] (see make_index) on the device type the call
    reads it from; for host calls also a C-contiguous numpy array of STAMP_DTYPE
    or int64 [N, 2].  Anything else raises TypeError before the library sees it."""
    if isinstance(index, torch.Tensor):
        if index.dtype != torch.int64 or index.dim() != 2 or index.shape[1] != 2:
            raise TypeError(f"index must be an int64 tensor [N, 2] (make_index), "
                            f"got {index.dtype} {tuple(index.shape)}")
        if not index.is_contiguous():
            raise TypeError("index must be contiguous")
        if index.device.type != where:
            raise TypeError(f"index must be on {where}, got {index.device}")
        return _vp(index.data_ptr()), int(index.shape[0])
    if isinstance(index, np.ndarray) and where == "cpu":
        ok = (index.dtype == STAMP_DTYPE and index.ndim == 1) or \
             (index.dtype == np.int64 and index.ndim == 2 and index.shape[1] == 2)
        if not ok or not index.flags.c_contiguous:
            raise TypeError(f"index must be a C-contiguous STAMP_DTYPE array or int64 [N, 2], "
                            f"got {index.dtype} {index.shape}")
        return _vp(index.ctypes.data), int(index.shape[0])
    raise TypeError(f"index must be a tensor{' or numpy array' if where == 'cpu' else ''} "
                    f"on {where}, got {type(index).__name__}")


def _dtype_of(pix: torch.Tensor) -> int:
    if pix.dtype == torch.float32:
        return FSE_F32
    if pix.dtype == torch.bfloat16:
        return FSE_BF16
    raise TypeError("pixels must be float32 or bfloat16")


class Context:
    """An fse_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        L = load()
        h = _vp()
        rc = L.fse_create(ctypes.byref(h), int(device))
        if rc != FSE_OK:
            raise FseError(rc, f"fse_create(device={device}) failed")
        self._h = h
        self.device = int(device)

    def close(self):
        if getattr(self, "_h", None):
            load().fse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != FSE_OK:
            raise FseError(rc, load().fse_last_error(self._h).decode())

    def _dev_call(self, fname, pix, index, out, scale, inv_var, opts, stream):
        ip, n = _index(index)
        if out is None:
            out = torch.zeros((n, 64), dtype=torch.uint8, device=pix.device)
        rc = getattr(load(), fname)(self._h, _ptr(pix), _dtype_of(pix), _ptr(scale), ip, n,
                                    _ptr(inv_var), ctypes.byref(opts or default_opts()), _ptr(out),
                                    _stream(stream))
        self._check(rc)
        return out

    # --- the C ABI, one method per entry point --------------------------------
    def centroid(self, pix, index, *, scale=None, inv_var=None, opts=None, out=None, stream=None):
        """fse_centroid: Sec. 2 centroid. Returns the result tensor (uint8 [N, 64])."""
        return self._dev_call("fse_centroid", pix, index, out, scale, inv_var, opts, stream)

    def ellipticity(self, pix, index, inout, *, scale=None, inv_var=None, opts=None, stream=None):
        """fse_ellipticity: Secs. 2-3 from inout's centre and sigma_w (in place)."""
        return self._dev_call("fse_ellipticity", pix, index, inout, scale, inv_var, opts, stream)

    def sersic_fit(self, pix, index, inout, *, scale=None, inv_var=None, opts=None, stream=None):
        """fse_sersic_fit: Sec. 4.1 fit with inout's centre and ellipticity (in place)."""
        return self._dev_call("fse_sersic_fit", pix, index, inout, scale, inv_var, opts, stream)

    def fit_batch(self, pix, index, *, scale=None, inv_var=None, opts=None, out=None, stream=None):
        """fse_fit_batch: the whole chain in three persistent launches (start-up, moments, fit)."""
        return self._dev_call("fse_fit_batch", pix, index, out, scale, inv_var, opts, stream)

    def fit_batch_plain(self, pix, index, *, scale=None, inv_var=None, opts=None, out=None,
                        stream=None):
        """fse_fit_batch_plain: the same chain, one launch pair per stamp."""
        return self._dev_call("fse_fit_batch_plain", pix, index, out, scale, inv_var, opts, stream)

    def fit_batch_ragged(self, pix, index, *, scale=None, inv_var=None, opts=None, out=None,
                         stream=None):
        """fse_fit_batch_ragged: size-class launches (opts.flags |= 1 replays a CUDA graph)."""
        return self._dev_call("fse_fit_batch_ragged", pix, index, out, scale, inv_var, opts, stream)

    def autotune(self, pix, index, *, scale=None, inv_var=None, opts=None, out=None, stream=None):
        """fse_autotune: time the launch shapes of each size class on this batch."""
        return self._dev_call("fse_autotune", pix, index, out, scale, inv_var, opts, stream)

    def tuned_warps(self, dtype: int = FSE_F32, inv_var: bool = False) -> list:
        """fse_tuned_warps: (warps per CTA, warps per stamp) of the seven size classes."""
        w = (ctypes.c_int32 * 7)()
        n = (ctypes.c_int32 * 7)()
        self._check(load().fse_tuned_warps(self._h, dtype, int(inv_var), w, n))
        return list(zip(w, n))

    def tuning_save(self, path: str) -> None:
        """fse_tuning_save: write this context's autotuned launch shapes to a JSON file."""
        self._check(load().fse_tuning_save(self._h, os.fsencode(path)))

    def tuning_load(self, path: str) -> bool:
        """fse_tuning_load: apply the saved launch shapes for this device; False
        when the file holds none that apply (or cannot be read)."""
        return load().fse_tuning_load(self._h, os.fsencode(path)) == FSE_OK

    def star_fit(self, pix, index, moments, *, profile: str = "gauss", scale=None, opts=None,
                 out=None, stream=None):
        """fse_star_fit: Sec. 4.2 star profile at the moments' centre and ellipticity.
        moments is a result tensor (uint8 [N, 64]); returns uint8 [N, 32]."""
        ip, n = _index(index)
        if out is None:
            out = torch.zeros((n, 32), dtype=torch.uint8, device=pix.device)
        rc = load().fse_star_fit(self._h, _ptr(pix), _dtype_of(pix), _ptr(scale), ip, n,
                                 _ptr(moments), {"gauss": FSE_STAR_GAUSS, "moffat": FSE_STAR_MOFFAT}[profile],
                                 ctypes.byref(opts or default_opts()), _ptr(out), _stream(stream))
        self._check(rc)
        return out

    def moment_vjp(self, pix, index, moments, v, *, mode: int = FSE_MOM_ELLIP | FSE_MOM_SIGW_R50,
                   scale=None, out=None, status=None, stream=None):
        """fse_moment_vjp: dL/dI (float32, laid out like pix) for v = dL/d(x0, y0,
        e1, e2, sigma_w) (float32 [N, 5]) at the moment fixed point in moments."""
        ip, n = _index(index)
        v = v.to(torch.float32).contiguous()
        if v.shape != (n, 5):
            raise TypeError("v must be [N, 5]")
        if out is None:
            out = torch.zeros(pix.numel(), dtype=torch.float32, device=pix.device)
        self._check(load().fse_moment_vjp(self._h, _ptr(pix), _dtype_of(pix), _ptr(scale), ip, n,
                                          _ptr(moments), mode, _ptr(v), _ptr(out), _ptr(status),
                                          _stream(stream)))
        return out

    def moment_jvp(self, pix, index, moments, tangent, *, mode: int = FSE_MOM_ELLIP | FSE_MOM_SIGW_R50,
                   scale=None, out=None, status=None, stream=None):
        """fse_moment_jvp: d(x0, y0, e1, e2, sigma_w) (float32 [N, 5]) along the
        pixel tangent (float32, laid out like pix)."""
        ip, n = _index(index)
        tangent = tangent.to(torch.float32).contiguous()
        if out is None:
            out = torch.empty((n, 5), dtype=torch.float32, device=pix.device)
        self._check(load().fse_moment_jvp(self._h, _ptr(pix), _dtype_of(pix), _ptr(scale), ip, n,
                                          _ptr(moments), mode, _ptr(tangent), _ptr(out), _ptr(status),
                                          _stream(stream)))
        return out

    def cutout(self, images, img_index, *, side_factor: float = 6.0, min_side: int = 8, max_side: int = 128,
               scale=None, out=None, stream=None):
        """fse_cutout (Sec. 4.1): the square of side side_factor * r50 around the
        brightest pixel of each image, packed back to back.  Returns (pix,
        index, info): the cut-out pixels (dtype of the images), their fse_stamp
        index (int64 [N, 2] view, see make_index) and the per-image
        fse_cutout_info records (uint8 [N, 24]).  Without `out` a first launch
        sizes the buffer (and the stream is synchronised once)."""
        ip, n = _index(img_index)
        dev = images.device
        info = torch.zeros((n, 24), dtype=torch.uint8, device=dev)
        idx = torch.zeros((n, 2), dtype=torch.int64, device=dev)
        total = torch.zeros(1, dtype=torch.int64, device=dev)
        L = load()
        args = lambda o, cap: (self._h, _ptr(images), _dtype_of(images), _ptr(scale), ip, n,
                               float(side_factor), int(min_side), int(max_side), _ptr(info), _ptr(idx), _ptr(o),
                               int(cap), _ptr(total), _stream(stream))
        if out is None:
            self._check(L.fse_cutout(*args(None, 0)))
            torch.cuda.synchronize(dev)
            out = torch.empty(max(int(total.item()), 1), dtype=images.dtype, device=dev)
            cap = int(total.item())
        else:
            cap = out.numel()
        self._check(L.fse_cutout(*args(out, cap)))
        return out, idx, info

    def fit_batch_host(self, pix: np.ndarray | torch.Tensor, index: np.ndarray | torch.Tensor, *,
                       scale=None, inv_var=None, opts=None, out=None, stream=None) -> np.ndarray:
        """fse_fit_batch_host: host buffers in, host results out (synchronous)."""
        if isinstance(pix, torch.Tensor):
            assert pix.device.type == "cpu" and pix.is_contiguous()
            dtype = _dtype_of(pix)
            pix_ptr, npix = pix.data_ptr(), pix.numel()
        else:
            assert pix.dtype == np.float32 and pix.flags.c_contiguous
            dtype, pix_ptr, npix = FSE_F32, pix.ctypes.data, pix.size
        idx_ptr, n = _index(index, "cpu")
        if out is None:
            out = np.zeros(n, dtype=RESULT_DTYPE)
        out_ptr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
        sp = None if scale is None else _vp(scale.data_ptr() if isinstance(scale, torch.Tensor)
                                             else scale.ctypes.data)
        ivp = None if inv_var is None else _vp(inv_var.data_ptr() if isinstance(inv_var, torch.Tensor)
                                                else inv_var.ctypes.data)
        rc = load().fse_fit_batch_host(self._h, _vp(pix_ptr), int(npix), dtype, sp, idx_ptr,
                                       int(n), ivp, ctypes.byref(opts or default_opts()),
                                       _vp(out_ptr), _stream(stream))
        self._check(rc)
        return out

    def sersic_b(self, n: torch.Tensor, stream=None):
        """fse_sersic_b: (b(n), b'(n)) from the device table, float64 CUDA tensors."""
        n = n.to(torch.float64).contiguous()
        b = torch.empty_like(n)
        db = torch.empty_like(n)
        self._check(load().fse_sersic_b(self._h, _ptr(n), _ptr(b), _ptr(db), n.numel(),
                                        _stream(stream)))
        return b, db

    def chi2_grad(self, pix, index, params, *, scale=None, inv_var=None, gout=None,
                  want_chi2=True, want_dparams=True, want_dpix=False, stream=None):
        """fse_sersic_chi2_grad: chi^2 and its gradient at params (float32 [N, 7]).

        Returns (chi2 float64 [N] or None, dparams float32 [N, 7] or None,
        dpix float32 like pix or None)."""
        ip, n = _index(index)
        dev = pix.device
        chi2 = torch.empty(n, dtype=torch.float64, device=dev) if want_chi2 else None
        dpar = torch.empty((n, 7), dtype=torch.float32, device=dev) if want_dparams else None
        dpix = torch.zeros(pix.numel(), dtype=torch.float32, device=dev) if want_dpix else None
        params = params.contiguous()
        if params.dtype != torch.float32 or params.shape != (n, 7):
            raise TypeError("params must be float32 [N, 7]")
        if gout is not None:
            gout = gout.to(torch.float64).contiguous()
        rc = load().fse_sersic_chi2_grad(self._h, _ptr(pix), _dtype_of(pix), _ptr(scale), ip,
                                         n, _ptr(inv_var), _ptr(params), _ptr(gout), _ptr(chi2),
                                         _ptr(dpar), _ptr(dpix), _stream(stream))
        self._check(rc)
        return chi2, dpar, dpix

    def sync_check(self, stream=None):
        """fse_sync_check: wait for the stream and raise if a bounded device wait expired."""
        self._check(load().fse_sync_check(self._h, _stream(stream)))


# module-level forms with the ABI's names (context first)
def fse_centroid(ctx: Context, *a, **k):
    return ctx.centroid(*a, **k)


def fse_ellipticity(ctx: Context, *a, **k):
    return ctx.ellipticity(*a, **k)


def fse_sersic_fit(ctx: Context, *a, **k):
    return ctx.sersic_fit(*a, **k)


def fse_fit_batch(ctx: Context, *a, **k):
    return ctx.fit_batch(*a, **k)


def fse_fit_batch_plain(ctx: Context, *a, **k):
    return ctx.fit_batch_plain(*a, **k)


def fse_fit_batch_host(ctx: Context, *a, **k):
    return ctx.fit_batch_host(*a, **k)


def fse_fit_batch_ragged(ctx: Context, *a, **k):
    return ctx.fit_batch_ragged(*a, **k)


def fse_autotune(ctx: Context, *a, **k):
    return ctx.autotune(*a, **k)


def fse_tuned_warps(ctx: Context, *a, **k):
    return ctx.tuned_warps(*a, **k)


def fse_star_fit(ctx: Context, *a, **k):
    return ctx.star_fit(*a, **k)


def fse_moment_vjp(ctx: Context, *a, **k):
    return ctx.moment_vjp(*a, **k)


def fse_moment_jvp(ctx: Context, *a, **k):
    return ctx.moment_jvp(*a, **k)


def fse_cutout(ctx: Context, *a, **k):
    return ctx.cutout(*a, **k)


def fse_sersic_b(ctx: Context, *a, **k):
    return ctx.sersic_b(*a, **k)


def fse_sersic_chi2_grad(ctx: Context, *a, **k):
    return ctx.chi2_grad(*a, **k)


def fse_sync_check(ctx: Context, *a, **k):
    return ctx.sync_check(*a, **k)


def fit_batch_static(pix, index, *, scale=None, inv_var=None, opts=None, out=None, stream=None):
    """fse_fit_batch_static: the whole chain on the current device with no context
    and no device allocation inside the call (scratch in static device memory)."""
    ip, n = _index(index)
    if out is None:
        out = torch.zeros((n, 64), dtype=torch.uint8, device=pix.device)
    err = ctypes.create_string_buffer(512)
    rc = load().fse_fit_batch_static(_ptr(pix), _dtype_of(pix), _ptr(scale), ip, n,
                                     _ptr(inv_var), ctypes.byref(opts or default_opts()), _ptr(out),
                                     _stream(stream), err, len(err))
    if rc != FSE_OK:
        raise FseError(rc, err.value.decode())
    return out


fse_fit_batch_static = fit_batch_static
