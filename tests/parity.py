"""GPU-versus-oracle comparison used by the GPU parity tests.

Tolerances (the estimator's parity gate): centroid 1e-4 px, e1/e2 1e-5
absolute, r_e, n and flux 1e-4 relative, chi^2 1e-5 relative.

Every stamp of a comparison is accounted for, in exactly one class:

  gated          both sides converged their moments (and, for the fit, a fit
                 that did not end on a bound); every gated stamp must be within
                 tolerance.
  both_not_ok    neither side converged (the same verdict on both sides).
  cond           both converged, but the Jacobi-scaled J^T J of the oracle's
                 optimum has condition number > 1e10: the r_e - n valley is too
                 flat for a unique minimum at these tolerances.
  other_minimum  the GPU found a chi^2 lower than the oracle's by more than the
                 tolerance.  It counts as excluded only when the oracle,
                 restarted from the GPU's (r_e, n), reaches the GPU's minimum
                 (within tolerance): a second local minimum of the r_e - n
                 degeneracy (Sec. 4.1).  Otherwise it is a failure.
  clamped_fixed_point
                 both converged with sigma_w held at its lower clamp of 0.5 px,
                 but at different centres or ellipticities: a weight narrower
                 than a pixel does not determine a unique fixed point of
                 Secs. 2-3.  Excluded only when the oracle confirms that the
                 GPU's point is a fixed point (its moment step there below
                 1e-5, sigma_w held) and the oracle's own fit from the GPU's
                 moments agrees with the GPU's fit.  Otherwise a failure.
  other_fixed_point
                 the same without the clamp: both converged, at different
                 centres or ellipticities, each a fixed point of Secs. 2-3 (at
                 low SNR the iteration has several).  Confirmed as above, and
                 allowed up to assert_gate's max_other_fixed_point (0 unless a
                 test states otherwise).
  disagree       the two sides disagree on whether the moments, or the fit,
                 converged.  Each such stamp carries its reason:
                   oracle_*   the GPU converged and the oracle did not.  It is
                              excluded only when the oracle confirms the GPU's
                              result: a moment step of the oracle at the GPU's
                              centre, g and sigma_w below 1e-5 (a fixed point of
                              Secs. 2-3), or the oracle's fit restarted from the
                              GPU's (r_e, n) converging to the GPU's values
                              within tolerance.  Otherwise it is a failure.
                   gpu_*      the oracle converged and the GPU did not (its pass
                              cap, a bound, a failed step).  Allowed up to a
                              stated count per test (assert_gate's max_gpu_short),
                              each listed.
                   subpixel_* either side holds sigma_w at its lower clamp of
                              0.5 px: the weight is narrower than a pixel, the
                              iteration has several fixed points and which one
                              (or a failure) it reaches depends on its path.
                              Counted apart, up to assert_gate's max_subpixel.

assert_gate() checks all of this; the report (dumped with FSE_PARITY_DIR) lists
every excluded or disagreeing stamp with its reason.
"""
from __future__ import annotations

import json
import os

import numpy as np

TOL = dict(x0=1e-4, y0=1e-4, e1=1e-5, e2=1e-5, re=1e-4, n=1e-4, flux=1e-4, chi2=1e-5)
ABS = {"x0", "y0", "e1", "e2"}
MOM_CONVERGED, FIT_CONVERGED, MOM_MAXITER, FIT_MAXITER = 1, 2, 4, 8
MOM_FAILED, FIT_BOUND, FIT_SINGULAR, SIGW_CLAMPED = 64, 128, 256, 1024
FIXED_POINT_STEP = 1e-5     # largest oracle moment step at a point accepted as its fixed point


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


def _stamp_ivar(batch, i, ivar):
    if ivar is None:
        return None
    o = int(batch.offset[i])
    return ivar[o:o + int(batch.h[i]) * int(batch.w[i])].reshape(int(batch.h[i]), int(batch.w[i]))


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


def _rel(a, b):
    return abs(float(a) - float(b)) / max(abs(float(b)), 1e-300)


def _fit_agrees(g, o):
    return all(_rel(g[k], o[k]) <= TOL[k] for k in ("re", "n", "flux", "chi2"))


def _oracle_refit(O, batch, i, orc_row, gpu_row, ivar, supersample, opts):
    """The oracle's fit at its own centre and ellipticity, restarted from the GPU's (r_e, n)."""
    kw = {} if opts is None else {"opts": opts}
    if supersample > 1:
        kw["opts"] = O.default_opts(supersample=supersample) if opts is None else opts
    return O.sersic_fit_from(batch.stamp(i), orc_row["x0"], orc_row["y0"], orc_row["e1"], orc_row["e2"],
                             float(gpu_row["re"]), float(gpu_row["n"]), ivar=_stamp_ivar(batch, i, ivar), **kw)


def _clamped_low(row):
    """sigma_w held at its lower clamp of 0.5 px (a weight narrower than a pixel)."""
    return bool(int(row["status"]) & SIGW_CLAMPED) and abs(float(row["sigma_w"]) - 0.5) <= 1e-6


def _confirm_fixed_point(O, batch, i, gpu_row, ellip, sigw_mode):
    """The oracle's moment step at the GPU's converged centre, g and sigma_w.
    For the matched weight (sigw_mode 0) sigma_w must also be the rule's fixed
    point, or, where the GPU holds it at a clamp, the rule must point past
    that clamp."""
    g1, g2 = (float(gpu_row["e1"]), float(gpu_row["e2"])) if ellip else (0.0, 0.0)
    sw = float(gpu_row["sigma_w"])
    st = O.moment_step(batch.stamp(i), float(gpu_row["x0"]), float(gpu_row["y0"]), g1, g2,
                       sw, k_gain=0.0, ellip=ellip)
    size = max(abs(st["dx"]), abs(st["dy"]))
    if ellip:
        size = max(size, abs(st["dg1"]), abs(st["dg2"]))
    ok = bool(st["ok"])
    if sigw_mode == 0:
        h, w = int(batch.h[i]), int(batch.w[i])
        if _clamped_low(gpu_row):
            ok = ok and st["sigw_new"] <= 0.5
        elif int(gpu_row["status"]) & SIGW_CLAMPED and abs(sw - 0.5 * min(h, w)) <= 1e-6 * sw:
            ok = ok and st["sigw_new"] >= sw
        else:
            size = max(size, abs(st["sigw_new"] / sw - 1.0))
    return ok and size <= FIXED_POINT_STEP, float(size)


def _bits(s):
    names = [(MOM_CONVERGED, "MOM_CONVERGED"), (FIT_CONVERGED, "FIT_CONVERGED"), (MOM_MAXITER, "MOM_MAXITER"),
             (FIT_MAXITER, "FIT_MAXITER"), (16, "NONFINITE"), (32, "BAD_SIZE"), (MOM_FAILED, "MOM_FAILED"),
             (FIT_BOUND, "FIT_BOUND"), (FIT_SINGULAR, "FIT_SINGULAR"), (512, "NONPOS_FLUX")]
    return [n for b, n in names if int(s) & b]


def _gpu_short_reason(gs, fit_level):
    if not fit_level:
        if gs & MOM_MAXITER:
            return "gpu_mom_pass_cap"
        if gs & MOM_FAILED:
            return "gpu_mom_failed"
        return "gpu_mom_other"
    if gs & FIT_BOUND:
        return "gpu_fit_bound"
    if gs & FIT_SINGULAR:
        return "gpu_fit_singular"
    if gs & FIT_MAXITER:
        return "gpu_fit_pass_cap"
    return "gpu_fit_other"


def compare(gpu, orc, keys=("x0", "y0", "e1", "e2", "re", "n", "flux", "chi2"), fit=True,
            O=None, batch=None, ids=None, ivar=None, supersample=1, ellip=True, sigw_mode=1,
            orc_opts=None, same_pixels=True):
    """Per-stamp errors, the class of every stamp and the gate verdict.  Returns a report.

    O, batch and ids (stamp j of gpu/orc is stamp ids[j] of batch) let the
    oracle check the exclusions; without them every exclusion that needs a
    check counts as unconfirmed.  same_pixels=False (the two sides measured
    different pixels, e.g. bf16 storage against fp32) keeps every jointly
    converged stamp in the gate: its differences are the measurement, not
    another fixed point."""
    gs, os_ = gpu["status"].astype(np.int64), orc["status"].astype(np.int64)
    n = len(gs)
    mom_g, mom_o = (gs & MOM_CONVERGED) != 0, (os_ & MOM_CONVERGED) != 0
    fit_g = mom_g & ((gs & FIT_CONVERGED) != 0) & ((gs & FIT_BOUND) == 0)
    fit_o = mom_o & ((os_ & FIT_CONVERGED) != 0) & ((os_ & FIT_BOUND) == 0)
    ok_g, ok_o = (fit_g, fit_o) if fit else (mom_g, mom_o)
    conv = ok_g & ok_o
    err = {}
    for k in keys:
        g = gpu[k].astype(np.float64)
        o = orc[k].astype(np.float64)
        if k in ABS:
            err[k] = np.abs(g - o)
        else:
            err[k] = np.abs(g - o) / np.maximum(np.abs(o), 1e-300)
    checkable = O is not None and batch is not None and ids is not None
    klass = np.array(["gated"] * n, dtype=object)
    klass[~ok_g & ~ok_o] = "both_not_ok"
    reason = [""] * n
    confirmed = np.zeros(n, bool)
    extra = [dict() for _ in range(n)]
    # condition-number and other-minimum exclusions among the jointly converged
    if fit and "chi2" in keys:
        basin = conv & (gpu["chi2"] < orc["chi2"] * (1 - TOL["chi2"]))
        for j in np.nonzero(conv)[0]:
            if not checkable:
                break
            i = int(ids[j])
            c = jtj_condition(O, batch.stamp(i), orc[j], _stamp_ivar(batch, i, ivar), supersample)
            if c > 1e10:
                klass[j] = "cond"
                reason[j] = "jtj_condition"
                extra[j]["condition"] = c
                confirmed[j] = True
        for j in np.nonzero(basin)[0]:
            if klass[j] != "gated":
                continue
            klass[j] = "other_minimum"
            reason[j] = "other_minimum"
            if checkable:
                r = _oracle_refit(O, batch, int(ids[j]), orc[j], gpu[j], ivar, supersample, orc_opts)
                extra[j]["oracle_restarted"] = {k: float(r[k]) for k in ("re", "n", "flux", "chi2", "status")}
                rok = (r["status"] & FIT_CONVERGED) and not (r["status"] & FIT_BOUND)
                confirmed[j] = bool(rok and r["chi2"] < orc["chi2"][j] * (1 - TOL["chi2"])
                                    and _fit_agrees(gpu[j], r))
    # both converged at the sub-pixel weight clamp, on different fixed points
    mkeys = [k for k in ("x0", "y0", "e1", "e2") if k in keys]
    for j in np.nonzero(conv)[0]:
        if klass[j] not in ("gated", "other_minimum") or not mkeys or not same_pixels:
            continue
        if all(err[k][j] <= TOL[k] for k in mkeys):
            continue
        kind = "clamped_fixed_point" if _clamped_low(gpu[j]) and _clamped_low(orc[j]) else "other_fixed_point"
        klass[j] = kind
        reason[j] = kind
        confirmed[j] = False
        if not checkable:
            continue
        i = int(ids[j])
        confirmed[j], extra[j]["oracle_step_at_gpu"] = _confirm_fixed_point(O, batch, i, gpu[j], ellip, sigw_mode)
        if confirmed[j] and fit:
            fo = orc_opts if orc_opts is not None else (
                O.default_opts(supersample=supersample) if supersample > 1 else None)
            r = O.sersic_fit(batch.stamp(i), float(gpu["x0"][j]), float(gpu["y0"][j]), float(gpu["e1"][j]),
                             float(gpu["e2"][j]), float(gpu["sigma_w"][j]), ivar=_stamp_ivar(batch, i, ivar), opts=fo)
            rok = (r["status"] & FIT_CONVERGED) and not (r["status"] & FIT_BOUND)
            extra[j]["oracle_fit_at_gpu_moments"] = {k: float(r[k]) for k in ("re", "n", "chi2", "status")}
            confirmed[j] = bool(rok and _fit_agrees(gpu[j], r))
    # status disagreements
    for j in np.nonzero(ok_g != ok_o)[0]:
        klass[j] = "disagree"
        fit_level = bool(mom_g[j] and mom_o[j])
        extra[j]["gpu_bits"] = _bits(gs[j])
        extra[j]["oracle_bits"] = _bits(os_[j])
        extra[j]["it_mom"] = [int(gpu["it_mom"][j]), int(orc["it_mom"][j])]
        if fit_level:
            extra[j]["it_fit"] = [int(gpu["it_fit"][j]), int(orc["it_fit"][j])]
        if _clamped_low(gpu[j]) or _clamped_low(orc[j]):
            reason[j] = "subpixel_" + ("gpu_short" if ok_o[j] else "oracle_short")
            continue
        if ok_o[j]:
            reason[j] = _gpu_short_reason(gs[j], fit_level)
            continue
        # the GPU converged and the oracle did not: the oracle must confirm the GPU's result
        reason[j] = "oracle_fit_short" if fit_level else "oracle_mom_short"
        if not checkable:
            continue
        i = int(ids[j])
        if not fit_level:
            confirmed[j], extra[j]["oracle_step_at_gpu"] = _confirm_fixed_point(O, batch, i, gpu[j], ellip,
                                                                               sigw_mode)
            if confirmed[j] and fit:
                # the oracle's own fit from the GPU's moments must agree too
                fo = orc_opts if orc_opts is not None else (
                    O.default_opts(supersample=supersample) if supersample > 1 else None)
                r = O.sersic_fit(batch.stamp(i), float(gpu["x0"][j]), float(gpu["y0"][j]), float(gpu["e1"][j]),
                                 float(gpu["e2"][j]), float(gpu["sigma_w"][j]), ivar=_stamp_ivar(batch, i, ivar),
                                 opts=fo)
                rok = (r["status"] & FIT_CONVERGED) and not (r["status"] & FIT_BOUND)
                extra[j]["oracle_fit_at_gpu_moments"] = {k: float(r[k]) for k in ("re", "n", "chi2", "status")}
                confirmed[j] = bool(rok and _fit_agrees(gpu[j], r)) if "chi2" in keys else confirmed[j]
        else:
            r = _oracle_refit(O, batch, i, orc[j], gpu[j], ivar, supersample, orc_opts)
            rok = (r["status"] & FIT_CONVERGED) and not (r["status"] & FIT_BOUND)
            extra[j]["oracle_restarted"] = {k: float(r[k]) for k in ("re", "n", "flux", "chi2", "status")}
            confirmed[j] = bool(rok and _fit_agrees(gpu[j], r))
    gate = klass == "gated"
    ok = np.ones(n, bool)
    for k in keys:
        ok &= err[k] <= TOL[k]
    within = gate & ok
    gpu_short = np.array([r.startswith("gpu_") for r in reason], bool)
    subpixel = np.array([r.startswith("subpixel_") for r in reason], bool)
    unconfirmed = (np.isin(klass, ["other_minimum", "disagree", "clamped_fixed_point", "other_fixed_point"])
                   & ~confirmed & ~gpu_short
                   & ~subpixel)
    counts = {}
    for j in range(n):
        if reason[j]:
            key = reason[j] + ("" if reason[j].startswith(("gpu_", "subpixel_")) or confirmed[j] else "_unconfirmed")
            counts[key] = counts.get(key, 0) + 1
    rep = {
        "n": int(n),
        "status_agree": float(np.mean(ok_g == ok_o)) if n else 1.0,
        "both_converged": int(conv.sum()),
        "both_not_ok": int((klass == "both_not_ok").sum()),
        "excluded_condition": int((klass == "cond").sum()),
        "excluded_other_minimum": int(((klass == "other_minimum") & confirmed).sum()),
        "excluded_clamped_fixed_point": int(((klass == "clamped_fixed_point") & confirmed).sum()),
        "excluded_other_fixed_point": int(((klass == "other_fixed_point") & confirmed).sum()),
        "disagree_confirmed": int(((klass == "disagree") & confirmed).sum()),
        "gpu_short": int(gpu_short.sum()),
        "subpixel": int(subpixel.sum()),
        "unconfirmed": int(unconfirmed.sum()),
        "reasons": counts,
        "gated": int(gate.sum()),
        "within_tolerance": int(within.sum()),
        "max_err": {k: float(err[k][gate].max()) if gate.any() else 0.0 for k in keys},
        "p99_err": {k: float(np.percentile(err[k][gate], 99)) if gate.any() else 0.0 for k in keys},
        "failing": [int(j) for j in np.nonzero(gate & ~ok)[0][:50]],
    }
    listed = np.nonzero((gate & ~ok) | np.isin(klass, ["other_minimum", "disagree", "cond", "clamped_fixed_point",
                                                       "other_fixed_point"]))[0]
    rep["detail"] = [{"j": int(j), "id": int(ids[j]) if ids is not None else int(j),
                      "class": str(klass[j]), "reason": reason[j], "confirmed": bool(confirmed[j]),
                      **extra[j],
                      "gpu": {k: float(gpu[k][j]) for k in gpu.dtype.names},
                      "orc": {k: float(orc[k][j]) for k in orc.dtype.names},
                      "err": {k: float(err[k][j]) for k in keys}} for j in listed[:200]]
    rep["_err"] = err
    rep["_gate"] = gate
    return rep


def summary(rep: dict) -> dict:
    return {k: v for k, v in rep.items() if not k.startswith("_") and k != "detail"}


def assert_gate(rep: dict, max_gpu_short: int = 0, min_gated: float = 0.5, max_subpixel: int = 0,
                max_other_fixed_point: int = 0):
    """Every gated stamp within tolerance; every exclusion confirmed by the
    oracle; at most max_gpu_short stamps that the oracle converged and the GPU
    did not, at most max_subpixel disagreements at the sub-pixel weight clamp
    and at most max_other_fixed_point other fixed points (each listed in the
    report with its reason); and, as a guard against a gate that excludes
    everything, at least min_gated of the stamps gated."""
    s = summary(rep)
    bad = [d for d in rep["detail"] if d["class"] in ("other_minimum", "disagree", "clamped_fixed_point",
                                                      "other_fixed_point")
           and not d["confirmed"] and not d["reason"].startswith(("gpu_", "subpixel_"))]
    assert rep["unconfirmed"] == 0, (s, bad[:5])
    short = [d for d in rep["detail"] if d["reason"].startswith("gpu_")]
    assert rep["gpu_short"] <= max_gpu_short, (s, short[:10])
    sub = [d for d in rep["detail"] if d["reason"].startswith("subpixel_")]
    assert rep["subpixel"] <= max_subpixel, (s, sub[:10])
    other = [d for d in rep["detail"] if d["class"] == "other_fixed_point"]
    assert rep["excluded_other_fixed_point"] <= max_other_fixed_point, (s, other[:10])
    assert rep["within_tolerance"] == rep["gated"], (rep["failing"], rep["max_err"], s)
    assert rep["gated"] >= min_gated * rep["n"], s


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
        json.dump(clean, f, indent=1, default=float)
