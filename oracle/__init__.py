"""ctypes front end of the FP64 oracle (``fse_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product path
(``paper_1203_0571_gb300``) never imports it.  It shares no code with the CUDA
library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fse_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfse_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no -march flags: same code on x86 and Arm)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                           "-D_GNU_SOURCE", "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class Opts(ctypes.Structure):
    _fields_ = [("tol_pos", ctypes.c_double), ("tol_g", ctypes.c_double),
                ("tol_sig", ctypes.c_double), ("tol_fit", ctypes.c_double),
                ("max_iter_mom", ctypes.c_int), ("max_iter_fit", ctypes.c_int),
                ("k_gain", ctypes.c_double), ("sigw_mode", ctypes.c_int),
                ("n_min", ctypes.c_double), ("n_max", ctypes.c_double),
                ("re_min", ctypes.c_double), ("re_max_frac", ctypes.c_double),
                ("lm_lambda0", ctypes.c_double), ("supersample", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("x0", "y0", "e1", "e2", "sigma_w", "r50", "I0", "re", "n", "flux", "chi2")] + \
               [("npix", ctypes.c_int32), ("it_mom", ctypes.c_int32), ("it_fit", ctypes.c_int32),
                ("status", ctypes.c_uint32)]


class StarResult(ctypes.Structure):
    _fields_ = [("size", ctypes.c_double), ("beta", ctypes.c_double), ("I0", ctypes.c_double),
                ("flux", ctypes.c_double), ("r50", ctypes.c_double), ("iters", ctypes.c_int32),
                ("status", ctypes.c_uint32)]


RESULT_DTYPE = np.dtype([(k, "f8") for k in
                         ("x0", "y0", "e1", "e2", "sigma_w", "r50", "I0", "re", "n", "flux", "chi2")] +
                        [("npix", "i4"), ("it_mom", "i4"), ("it_fit", "i4"), ("status", "u4")])
assert RESULT_DTYPE.itemsize == ctypes.sizeof(Result)

# status bits
MOM_CONVERGED, FIT_CONVERGED, MOM_MAXITER, FIT_MAXITER = 1, 2, 4, 8
NONFINITE, BAD_SIZE, MOM_FAILED, FIT_BOUND = 16, 32, 64, 128
FIT_SINGULAR, NONPOS_FLUX, SIGW_CLAMPED, INIT_FALLBACK = 256, 512, 1024, 2048

# implicit-gradient modes: g a parameter (Secs. 2-3); sigma_w held, or from
# the start-up growth curve (else the matched weight)
MOM_ELLIP, MOM_SIGW_FIXED, MOM_SIGW_R50 = 1, 2, 4

_dp = ctypes.POINTER(ctypes.c_double)


class CutoutInfo(ctypes.Structure):
    _fields_ = [("row0", ctypes.c_int32), ("col0", ctypes.c_int32), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("r50", ctypes.c_double), ("status", ctypes.c_uint32)]


class Oracle:
    """The oracle's entry points, bound to one compiled copy of fse_oracle.c."""

    MOM_ELLIP, MOM_SIGW_FIXED, MOM_SIGW_R50 = MOM_ELLIP, MOM_SIGW_FIXED, MOM_SIGW_R50

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        L.orc_default_opts.argtypes = [ctypes.POINTER(Opts)]
        for f in ("orc_sersic_b", "orc_sersic_db"):
            getattr(L, f).argtypes = [ctypes.c_double]
            getattr(L, f).restype = ctypes.c_double
        L.orc_gamma_p.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_gamma_p.restype = ctypes.c_double
        L.orc_sersic_flux.argtypes = [ctypes.c_double] * 4
        L.orc_sersic_flux.restype = ctypes.c_double
        for f in ("orc_centroid", "orc_ellipticity"):
            getattr(L, f).argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts),
                                      ctypes.POINTER(Result)]
        for f in ("orc_sersic_fit", "orc_measure"):
            getattr(L, f).argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts),
                                      ctypes.POINTER(Result)]
        L.orc_sersic_fit_from.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts),
                                          ctypes.c_double, ctypes.c_double, ctypes.POINTER(Result)]
        L.orc_moment_step.argtypes = [_dp, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 6 + \
                                     [ctypes.c_int, _dp]
        L.orc_fit_eval.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + \
                                  [_dp, _dp]
        L.orc_fit_eval_ss.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + \
                                     [_dp, ctypes.c_int, _dp]
        L.orc_star.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts), ctypes.c_int] + \
            [ctypes.c_double] * 5 + [ctypes.POINTER(StarResult)]
        L.orc_star.restype = None
        L.orc_chi2_grad.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        L.orc_chi2_grad.restype = None
        L.orc_moment_jacobian.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.orc_moment_jacobian.restype = None
        L.orc_moment_jvp.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
        L.orc_moment_jvp.restype = ctypes.c_int
        L.orc_moment_vjp.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
        L.orc_moment_vjp.restype = ctypes.c_int
        L.orc_cutout.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(CutoutInfo)]
        L.orc_cutout.restype = None
        L.orc_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(Opts), ctypes.c_int,
                                ctypes.c_void_p, ctypes.c_int]
        L.orc_batch.restype = ctypes.c_int
        self.L = L
        self.path = path

    def default_opts(self, **kw) -> Opts:
        o = Opts()
        self.L.orc_default_opts(ctypes.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def sersic_b(self, n: float) -> float:
        return self.L.orc_sersic_b(float(n))

    def sersic_db(self, n: float) -> float:
        return self.L.orc_sersic_db(float(n))

    def gamma_p(self, a: float, x: float) -> float:
        return self.L.orc_gamma_p(float(a), float(x))

    def sersic_flux(self, I0, re, n, gabs) -> float:
        return self.L.orc_sersic_flux(float(I0), float(re), float(n), float(gabs))

    def measure(self, I, ivar=None, opts: Opts | None = None) -> dict:
        """Whole chain on one stamp (float64 array (h, w))."""
        I = _img(I)
        iv = None if ivar is None else _img(ivar)
        r = Result()
        self.L.orc_measure(_as_dp(I), None if iv is None else _as_dp(iv), I.shape[0], I.shape[1],
                           ctypes.byref(opts or self.default_opts()), ctypes.byref(r))
        return _res_dict(r)

    def centroid(self, I, opts: Opts | None = None) -> dict:
        I = _img(I)
        r = Result()
        self.L.orc_centroid(_as_dp(I), I.shape[0], I.shape[1],
                            ctypes.byref(opts or self.default_opts()), ctypes.byref(r))
        return _res_dict(r)

    def ellipticity(self, I, x0, y0, sigma_w, opts: Opts | None = None) -> dict:
        I = _img(I)
        r = Result()
        r.x0, r.y0, r.sigma_w = x0, y0, sigma_w
        self.L.orc_ellipticity(_as_dp(I), I.shape[0], I.shape[1],
                               ctypes.byref(opts or self.default_opts()), ctypes.byref(r))
        return _res_dict(r)

    def sersic_fit(self, I, x0, y0, e1, e2, sigma_w, ivar=None, opts: Opts | None = None) -> dict:
        I = _img(I)
        iv = None if ivar is None else _img(ivar)
        r = Result()
        r.x0, r.y0, r.e1, r.e2, r.sigma_w = x0, y0, e1, e2, sigma_w
        self.L.orc_sersic_fit(_as_dp(I), None if iv is None else _as_dp(iv), I.shape[0],
                              I.shape[1], ctypes.byref(opts or self.default_opts()), ctypes.byref(r))
        return _res_dict(r)

    def sersic_fit_from(self, I, x0, y0, e1, e2, re0, n0, ivar=None, opts: Opts | None = None) -> dict:
        """The Sec. 4.1 fit at a fixed centre and ellipticity, started from (re0, n0)."""
        I = _img(I)
        iv = None if ivar is None else _img(ivar)
        r = Result()
        r.x0, r.y0, r.e1, r.e2 = x0, y0, e1, e2
        self.L.orc_sersic_fit_from(_as_dp(I), None if iv is None else _as_dp(iv), I.shape[0], I.shape[1],
                                   ctypes.byref(opts or self.default_opts()), re0, n0, ctypes.byref(r))
        return _res_dict(r)

    def moment_step(self, I, xc, yc, g1, g2, sw, k_gain=0.75, ellip=True) -> dict:
        I = _img(I)
        out = np.zeros(8)
        self.L.orc_moment_step(_as_dp(I), I.shape[0], I.shape[1], xc, yc, g1, g2, sw, k_gain,
                               int(ellip), _as_dp(out))
        return dict(dx=out[0], dy=out[1], dg1=out[2], dg2=out[3], e1=out[4], e2=out[5],
                    sigw_new=out[6], ok=bool(out[7]))

    def fit_eval(self, I, xc, yc, g1, g2, p, ivar=None, supersample: int = 1):
        """chi^2, J^T r and J^T J at p = (I0, r_e, n) with centre and g fixed;
        with supersample S the model of a pixel is the mean of S x S samples."""
        I = _img(I)
        iv = None if ivar is None else _img(ivar)
        pp = np.ascontiguousarray(p, dtype=np.float64)
        out = np.zeros(13)
        self.L.orc_fit_eval_ss(_as_dp(I), None if iv is None else _as_dp(iv), I.shape[0], I.shape[1],
                               xc, yc, g1, g2, _as_dp(pp), int(supersample), _as_dp(out))
        return out[0], out[1:4].copy(), out[4:].reshape(3, 3).copy()

    def star(self, I, xc, yc, g1, g2, size0, profile: str = "gauss", opts: Opts | None = None) -> dict:
        """Sec. 4.2 star profile from weighted radial moments at a fixed centre and
        ellipticity: size (Gaussian sigma or Moffat r_d along the major axis),
        beta (Moffat), I0, flux, r50, iters, status."""
        I = _img(I)
        r = StarResult()
        self.L.orc_star(_as_dp(I), I.shape[0], I.shape[1], ctypes.byref(opts or self.default_opts()),
                        {"gauss": 0, "moffat": 1}[profile], xc, yc, g1, g2, size0, ctypes.byref(r))
        return {k: getattr(r, k) for k, _ in StarResult._fields_}

    def chi2_grad(self, I, p, ivar=None, pixels: bool = False, scales: bool = False):
        """chi^2 and its gradient with respect to p = (x0, y0, g1, g2, I0, r_e, n)
        for one stamp; with pixels=True also the pixel gradient, with scales=True
        also the first-order error scales (8 values: 7 parameters, chi^2)."""
        I = _img(I)
        iv = None if ivar is None else _img(ivar)
        pp = np.ascontiguousarray(p, dtype=np.float64)
        chi2 = np.zeros(1)
        g = np.zeros(7)
        dp = np.zeros(I.shape) if pixels else None
        sc = np.zeros(8) if scales else None
        self.L.orc_chi2_grad(_as_dp(I), None if iv is None else _as_dp(iv), I.shape[0], I.shape[1],
                             _as_dp(pp), _as_dp(chi2), _as_dp(g), None if dp is None else _as_dp(dp),
                             None if sc is None else _as_dp(sc))
        out = (float(chi2[0]), g)
        if pixels:
            out += (dp,)
        if scales:
            out += (sc,)
        return out

    def moment_jacobian(self, I, theta):
        """F(theta) and J = dF/dtheta (5 x 5) of the moment fixed-point equations
        at theta = (xc, yc, g1, g2, sigma_w)."""
        I = _img(I)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        F, J = np.zeros(5), np.zeros(25)
        self.L.orc_moment_jacobian(_as_dp(I), I.shape[0], I.shape[1], _as_dp(th), _as_dp(F), _as_dp(J))
        return F, J.reshape(5, 5)

    def moment_jvp(self, I, theta, u, mode: int = MOM_ELLIP):
        """d theta along the pixel tangent u (implicit function theorem).
        Returns (dtheta[5], singular)."""
        I = _img(I)
        uu = _img(u)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        d = np.zeros(5)
        rc = self.L.orc_moment_jvp(_as_dp(I), I.shape[0], I.shape[1], _as_dp(th), mode, _as_dp(uu), _as_dp(d))
        return d, bool(rc)

    def moment_vjp(self, I, theta, v, mode: int = MOM_ELLIP):
        """dL/dI for dL/dtheta = v (implicit function theorem).  Returns
        (dI[h, w], singular)."""
        I = _img(I)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        vv = np.ascontiguousarray(v, dtype=np.float64)
        d = np.zeros(I.shape)
        rc = self.L.orc_moment_vjp(_as_dp(I), I.shape[0], I.shape[1], _as_dp(th), mode, _as_dp(vv), _as_dp(d))
        return d, bool(rc)

    def cutout(self, I, side_factor: float = 6.0, min_side: int = 8, max_side: int = 128) -> dict:
        """Sec. 4.1 cut-out of a large image: the square of side side_factor * r50
        around the brightest pixel.  Returns row0, col0, h, w, r50, status."""
        I = _img(I)
        r = CutoutInfo()
        self.L.orc_cutout(_as_dp(I), I.shape[0], I.shape[1], side_factor, min_side, max_side, ctypes.byref(r))
        return {k: getattr(r, k) for k, _ in CutoutInfo._fields_}

    def batch(self, pix, offset, h, w, stage: str = "measure", ivar=None,
              opts: Opts | None = None, init=None, threads: int = 0):
        """Run a stage over a flat fp32 stamp buffer.  Returns (results, threads_used)."""
        pix = np.ascontiguousarray(pix, dtype=np.float32)
        offset = np.ascontiguousarray(offset, dtype=np.int64)
        h = np.ascontiguousarray(h, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int32)
        iv = None if ivar is None else np.ascontiguousarray(ivar, dtype=np.float32)
        out = np.zeros(offset.size, dtype=RESULT_DTYPE) if init is None else \
            np.ascontiguousarray(init, dtype=RESULT_DTYPE).copy()
        used = self.L.orc_batch(pix.ctypes.data, offset.ctypes.data, h.ctypes.data, w.ctypes.data,
                                offset.size, None if iv is None else iv.ctypes.data,
                                ctypes.byref(opts or self.default_opts()), STAGES[stage],
                                out.ctypes.data, threads)
        return out, used


def _as_dp(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _img(I) -> np.ndarray:
    return np.ascontiguousarray(I, dtype=np.float64)


def _res_dict(r: Result) -> dict:
    return {k: getattr(r, k) for k, _ in Result._fields_}


_default = None


def get() -> Oracle:
    """The oracle built from the committed source."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def compile_variant(source_text: str, out_dir: str) -> Oracle:
    """Compile a modified copy of the oracle source (used to plant mistakes in tests)."""
    src = os.path.join(out_dir, "fse_oracle_variant.c")
    lib_path = os.path.join(out_dir, "libfse_oracle_variant.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                           "-D_GNU_SOURCE", "-o", lib_path, src, "-lm"])
    return Oracle(lib_path)


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


STAGES = {"measure": 0, "centroid": 1, "ellipticity": 2, "fit": 3}


def __getattr__(name):
    """Module-level access to the default oracle's methods (oracle.measure(...), ...)."""
    if name in ("default_opts", "sersic_b", "sersic_db", "gamma_p", "sersic_flux", "measure",
                "centroid", "ellipticity", "sersic_fit", "moment_step", "fit_eval", "batch"):
        return getattr(get(), name)
    raise AttributeError(name)
