"""GPU-versus-oracle comparison used by the GPU parity tests.

Tolerances (the estimator's parity gate): centroid 1e-4 px, e1/e2 1e-5
absolute, r_e, n and flux 1e-4 relative, chi^2 1e-5 relative.

A stamp enters the gate when both sides report converged moments (and, for
the fit, a converged fit), neither fit ended on a bound, and the fit is not
degenerate: the Jacobi-scaled J^T J of the oracle's optimum has condition
number <= 1e10, and the GPU did not find a lower chi^2 than the oracle by more
than the tolerance (that would be a different local minimum).  Excluded
stamps are counted and reported, never silently dropped.
"""
from __future__ import annotations

import json
import os

import numpy as np

TOL = dict(x0=1e-4, y0=1e-4, e1=1e-5, e2=1e-5, re=1e-4, n=1e-4, flux=1e-4, chi2=1e-5)
ABS = {"x0", "y0", "e1", "e2"}
MOM_CONVERGED, FIT_CONVERGED, FIT_BOUND = 1, 2, 128


def oracle_results(O, batch, ids, stage="measure", init=None, ivar=None, threads=0, opts=None):
    """Oracle results for stamps `ids` of a StampBatch (pixels decoded to fp32 as the kernel does)."""
    offs, hs, ws, chunks, ivs = [], [], [], [], []
    pos = 0
    for i in ids:
        a = batch.stamp(int(i)).astype(np.float32).ravel()
        chunks.append(a)
        offs.append(pos)
        hs.append(int(batch.h[int(i)]))
        ws.append(int(batch.w[int(i)]))
        if ivar is not None:
            o = int(batch.offset[int(i)])
            ivs.append(ivar[o:o + a.size])
        pos += a.size
    pix = np.concatenate(chunks) if chunks else np.zeros(0, np.float32)
    iv = np.concatenate(ivs).astype(np.float32) if ivar is not None else None
    res, _ = O.batch(pix, np.array(offs), np.array(hs), np.array(ws), stage=stage, init=init,
                     ivar=iv, threads=threads, opts=opts)
    return res


def jtj_condition(O, stamp, r, ivar=None, supersample=1):
    """Condition number of the Jacobi-scaled J^T J at the oracle's optimum."""
    _, _, H = O.fit_eval(stamp, r["x0"], r["y0"], r["e1"], r["e2"], [r["I0"], r["re"], r["n"]], ivar=ivar,
                         supersample=supersample)
    d = np.sqrt(np.abs(np.diag(H)))
    if not np.all(d > 0):
        return np.inf
    S = H / np.outer(d, d)
    ev = np.linalg.eigvalsh(S)
    return np.inf if ev[0] <= 0 else float(ev[-1] / ev[0])


def compare(gpu, orc, keys=("x0", "y0", "e1", "e2", "re", "n", "flux", "chi2"), fit=True,
            O=None, batch=None, ids=None, ivar=None, supersample=1):
    """Per-stamp errors and the gate verdict.  Returns a report dict."""
    gs, os_ = gpu["status"].astype(np.int64), orc["status"].astype(np.int64)
    conv = (gs & MOM_CONVERGED).astype(bool) & (os_ & MOM_CONVERGED).astype(bool)
    if fit:
        conv &= (gs & FIT_CONVERGED).astype(bool) & (os_ & FIT_CONVERGED).astype(bool)
        conv &= ~((gs & FIT_BOUND).astype(bool) | (os_ & FIT_BOUND).astype(bool))
    err = {}
    for k in keys:
        g = gpu[k].astype(np.float64)
        o = orc[k].astype(np.float64)
        if k in ABS:
            err[k] = np.abs(g - o)
        else:
            err[k] = np.abs(g - o) / np.maximum(np.abs(o), 1e-300)
    excluded_cond = np.zeros(len(gs), bool)
    excluded_basin = np.zeros(len(gs), bool)
    if fit and "chi2" in keys:
        excluded_basin = conv & (gpu["chi2"] < orc["chi2"] * (1 - TOL["chi2"]))
        if O is not None and batch is not None:
            for j in np.nonzero(conv)[0]:
                i = int(ids[j])
                iv = None
                if ivar is not None:
                    o = int(batch.offset[i])
                    iv = ivar[o:o + int(batch.h[i]) * int(batch.w[i])].reshape(batch.h[i], batch.w[i])
                excluded_cond[j] = jtj_condition(O, batch.stamp(i), orc[j], iv, supersample) > 1e10
    gate = conv & ~excluded_cond & ~excluded_basin
    ok = np.ones(len(gs), bool)
    for k in keys:
        ok &= err[k] <= TOL[k]
    within = gate & ok
    status_bits = MOM_CONVERGED | (FIT_CONVERGED if fit else 0)
    rep = {
        "n": int(len(gs)),
        "status_agree": float(np.mean((gs & status_bits) == (os_ & status_bits))) if len(gs) else 1.0,
        "both_converged": int(conv.sum()),
        "excluded_condition": int(excluded_cond.sum()),
        "excluded_other_minimum": int(excluded_basin.sum()),
        "gated": int(gate.sum()),
        "within_tolerance": int(within.sum()),
        "max_err": {k: float(err[k][gate].max()) if gate.any() else 0.0 for k in keys},
        "p99_err": {k: float(np.percentile(err[k][gate], 99)) if gate.any() else 0.0 for k in keys},
        "failing": [int(j) for j in np.nonzero(gate & ~ok)[0][:50]],
    }
    bad = np.nonzero((gate & ~ok) | excluded_basin)[0][:40]
    rep["detail"] = [{"j": int(j), "id": int(ids[j]) if ids is not None else int(j),
                      "excluded_other_minimum": bool(excluded_basin[j]),
                      "gpu": {k: float(gpu[k][j]) for k in gpu.dtype.names},
                      "orc": {k: float(orc[k][j]) for k in orc.dtype.names},
                      "err": {k: float(err[k][j]) for k in keys}} for j in bad]
    rep["_err"] = err
    rep["_gate"] = gate
    return rep


def dump(name: str, rep: dict, extra: dict | None = None):
    """Write the report as parity_<name>.json into the folder named by the
    environment variable FSE_PARITY_DIR, when it is set and exists."""
    d = os.environ.get("FSE_PARITY_DIR", "")
    if not d or not os.path.isdir(d):
        return
    clean = {k: v for k, v in rep.items() if not k.startswith("_")}
    if extra:
        clean.update(extra)
    with open(os.path.join(d, f"parity_{name}.json"), "w") as f:
        json.dump(clean, f, indent=1)
