"""Seeded synthetic postage stamps for the shape estimator.

This module renders the simulated images of Sec. 4.1 (Sérsic galaxies, Eq. 10)
and Sec. 4.2.1 (Gaussian stars) on small pixel grids and adds Gaussian noise.
It is an input generator only: it holds none of the estimator's arithmetic
(no moments, no fit).  Both the CUDA path and the FP64 oracle consume what it
produces; neither is used here.

Randomness is counter based.  Every random number is a SplitMix64 hash of
(seed, stream, counter), so any stamp of any workload can be regenerated on its
own, on any device, without drawing the stamps before it.  The Sérsic constant
b(n) used for rendering comes from ``scipy.special.gammaincinv`` (a library
routine), independently of the estimator's own b(n) code.

Conventions (shared with the C ABI): a stamp is row-major, pixel (row i,
column j) has its centre at (x=j, y=i); the ellipticity g=(g1, g2) enters the
elliptical radius R^2 = [(1-g1)^2+g2^2] dx^2 + [(1+g1)^2+g2^2] dy^2 - 4 g2 dx dy
(Eq. A1), and the Sérsic radius is r = R/(1-|g|), so r_e is the
half-light radius along the major axis.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch
from scipy import special

# ---------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64 finaliser, wrapping int64 maths).
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def _s64(v: int) -> int:
    """Reinterpret an unsigned 64-bit constant as a signed int64."""
    v &= _M64
    return v - (1 << 64) if v >= (1 << 63) else v


_GOLD = _s64(0x9E3779B97F4A7C15)
_C1 = _s64(0xBF58476D1CE4E5B9)
_C2 = _s64(0x94D049BB133111EB)


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _mix(x: torch.Tensor) -> torch.Tensor:
    x = x + _GOLD
    x = (x ^ _srl(x, 30)) * _C1
    x = (x ^ _srl(x, 27)) * _C2
    return x ^ _srl(x, 31)


def _key(seed: int, stream: int) -> int:
    z = torch.tensor([_s64(seed * 0x100000001B3 + stream)], dtype=torch.int64)
    return int(_mix(_mix(z))[0])


def uniform(seed: int, stream: int, counter: torch.Tensor) -> torch.Tensor:
    """U(0,1) doubles, one per int64 counter (never exactly 0 or 1)."""
    z = _mix(counter.to(torch.int64) ^ _key(seed, stream))
    return (_srl(z, 11).to(torch.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, counter: torch.Tensor) -> torch.Tensor:
    """N(0,1) doubles by Box-Muller from two independent uniform streams."""
    u1 = uniform(seed, 2 * stream, counter)
    u2 = uniform(seed, 2 * stream + 1, counter)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


# Streams: parameters use counter = stamp*16 + slot, noise counter = stamp<<15 | pixel.
_S_PARAM = 1
_S_NOISE = 2


def _param_uniform(seed: int, ids: np.ndarray, slot: int) -> np.ndarray:
    c = torch.from_numpy(ids.astype(np.int64) * 16 + slot)
    return uniform(seed, _S_PARAM, c).numpy()


# ---------------------------------------------------------------------------
# Workloads.
# ---------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    count: int
    seed: int
    description: str


WORKLOADS = {
    0: Workload("small-32px", 256, 0,
                "256 single-galaxy Sersic stamps, 32x32 fp32, flux logU[1e3,1e5], noise sigma=1"),
    1: Workload("uniform-48px", 100_000, 1,
                "100,000 stamps 48x48 fp32: 80% Sersic galaxies (SNR U[15,200]), "
                "20% Gaussian stars (FWHM U[2,4] px, |g|<0.05), shuffled"),
    2: Workload("ragged-16-128px", 1_000_000, 2,
                "1,000,000 stamps, side clip(round(8 r_e),16,128), r_e logU[1,15], packed flat fp32"),
    3: Workload("grad-64px", 65_536, 3,
                "65,536 stamps 64x64 fp32, n U[0.5,6], forward chi2 + adjoint"),
    4: Workload("precision-32-64px", 4_000_000, 4,
                "4,000,000 stamps, side U{32..64}, pixels bf16 (per-stamp scale) or fp32"),
    5: Workload("precision-lowsnr", 10_000, 5,
                "10,000 stamps, side U{32..64}, SNR U[10,30], n U[0.5,8] (error subsample)"),
    6: Workload("stars-gauss-32px", 20_000, 6,
                "20,000 Gaussian stars 32x32 fp32 (Sec. 4.2): r50 U[1.5,2.5] px, |g| U[0,0.25], SNR 300"),
    7: Workload("stars-moffat-48px", 20_000, 7,
                "20,000 Moffat stars 48x48 fp32 (Sec. 4.2): beta U[3,5], r50 U[1.5,2.5] px, |g| U[0,0.25], SNR 300"),
    8: Workload("images-512px", 500, 8,
                "500 images 512x512 fp32, one galaxy each (the large images of Sec. 4.1): base galaxy "
                "recipe, SNR U[15,200], centre offset U(-20,20) px from the image centre"),
}


@dataclasses.dataclass
class StampBatch:
    """A flat pixel buffer plus its index and the generating parameters."""
    pix: torch.Tensor            # flat float32 (or bf16 when encoded), all stamps back to back
    offset: torch.Tensor         # int64 [N], element offset of each stamp in pix
    h: torch.Tensor              # int32 [N]
    w: torch.Tensor              # int32 [N]
    truth: dict                  # numpy float64 arrays: n, re, g1, g2, xc, yc, I0, flux, b, star
    scale: torch.Tensor | None = None   # float32 [N] per-stamp scale for bf16 pixels

    @property
    def count(self) -> int:
        return int(self.offset.numel())

    def stamp(self, i: int) -> np.ndarray:
        """Stamp i as a float64 (h, w) numpy array (decoded if bf16)."""
        o, hh, ww = int(self.offset[i]), int(self.h[i]), int(self.w[i])
        a = self.pix[o:o + hh * ww].to(torch.float32).cpu().numpy().astype(np.float64)
        if self.scale is not None:
            a = a * float(self.scale[i])
        return a.reshape(hh, ww)

    def to(self, device) -> "StampBatch":
        return dataclasses.replace(
            self, pix=self.pix.to(device), offset=self.offset.to(device),
            h=self.h.to(device), w=self.w.to(device),
            scale=None if self.scale is None else self.scale.to(device))


def sersic_b(n: np.ndarray) -> np.ndarray:
    """b(n) with P(2n, b) = 1/2 (Eq. 10: r_e is the half-light radius), via scipy."""
    return special.gammaincinv(2.0 * np.asarray(n, dtype=np.float64), 0.5)


def sersic_flux(I0, re, n, gabs):
    """Total flux of the elliptical Sérsic profile: 2 pi n Gamma(2n) b^-2n I0 r_e^2 q."""
    b = sersic_b(n)
    q = (1.0 - gabs) / (1.0 + gabs)
    return 2.0 * np.pi * n * np.exp(special.gammaln(2 * n) - 2 * n * np.log(b)) * I0 * re * re * q


def _draw_params(wl: Workload, ids: np.ndarray) -> dict:
    """Per-stamp generating parameters (numpy float64), keyed on stamp id."""
    s = wl.seed
    U = lambda slot, lo, hi: lo + (hi - lo) * _param_uniform(s, ids, slot)
    logU = lambda slot, lo, hi: np.exp(U(slot, math.log(lo), math.log(hi)))
    N = ids.size
    star = np.zeros(N, dtype=bool)
    if wl.seed == 1:
        # exactly 20% stars, shuffled: a stamp is a star when its rank under a
        # seeded permutation key falls in the lowest fifth.
        key = _param_uniform(s, np.arange(wl.count), 15)
        rank = np.empty(wl.count, dtype=np.int64)
        rank[np.argsort(key, kind="stable")] = np.arange(wl.count)
        star = rank[ids] < wl.count // 5
    n = U(0, 0.5, 4.0)
    re = U(1, 1.5, 5.0)
    gabs = U(2, 0.0, 0.5)
    if wl.seed == 2:
        re = logU(1, 1.0, 15.0)
    if wl.seed == 3:
        n = U(0, 0.5, 6.0)
    if wl.seed == 5:
        n = U(0, 0.5, 8.0)
    phi = U(3, 0.0, math.pi)
    dx = U(4, -1.0, 1.0)
    dy = U(5, -1.0, 1.0)
    flux = logU(6, 1e3, 1e5)
    snr = U(7, 15.0, 200.0)
    if wl.seed == 5:
        snr = U(7, 10.0, 30.0)
    if wl.seed == 8:
        dx = U(4, -20.0, 20.0)
        dy = U(5, -20.0, 20.0)
    if star.any():
        fwhm = U(8, 2.0, 4.0)
        n = np.where(star, 0.5, n)
        re = np.where(star, fwhm / 2.0, re)
        gabs = np.where(star, U(9, 0.0, 0.05), gabs)
    beta = np.zeros(N)
    if wl.seed in (6, 7):
        # Sec. 4.2 star simulations: r50 1.5-2.5 px, |g| up to 0.25, SNR 300.
        # Gaussian: the n = 0.5 Sersic profile, whose r_e is r50.  Moffat: r_d
        # from r50 = r_d sqrt(2^(1/(beta-1)) - 1), kept in `re`.
        star[:] = True
        r50 = U(1, 1.5, 2.5)
        gabs = U(2, 0.0, 0.25)
        snr = np.full(N, 300.0)
        n = np.full(N, 0.5)
        re = r50
        if wl.seed == 7:
            beta = U(11, 3.0, 5.0)
            re = r50 / np.sqrt(2.0 ** (1.0 / (beta - 1.0)) - 1.0)
    if wl.seed in (0, 1, 3, 6, 7, 8):
        side = np.full(N, {0: 32, 1: 48, 3: 64, 6: 32, 7: 48, 8: 512}[wl.seed], dtype=np.int64)
    elif wl.seed == 2:
        side = np.clip(np.rint(8.0 * re), 16, 128).astype(np.int64)
    else:
        side = np.floor(U(10, 32.0, 65.0)).astype(np.int64).clip(32, 64)
    return dict(n=n, re=re, gabs=gabs, phi=phi, dx=dx, dy=dy, flux=flux, snr=snr,
                star=star, side=side, beta=beta, by_snr=np.full(N, wl.seed in (1, 5, 6, 7, 8)))


def _render(side: int, p: dict, sel: np.ndarray, ids: np.ndarray, seed: int,
            device, noise: bool) -> torch.Tensor:
    """Render the stamps `sel` (all of one side length); float64 [k, side, side]."""
    f64 = dict(dtype=torch.float64, device=device)
    k = sel.size
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a[sel]), **f64).view(k, 1, 1)
    n, re, gabs, phi = t(p["n"]), t(p["re"]), t(p["gabs"]), t(p["phi"])
    g1, g2 = gabs * torch.cos(2 * phi), gabs * torch.sin(2 * phi)
    c = (side - 1) / 2.0
    xc, yc = c + t(p["dx"]), c + t(p["dy"])
    b = torch.as_tensor(sersic_b(p["n"][sel]), **f64).view(k, 1, 1)
    yy, xx = torch.meshgrid(torch.arange(side, **f64), torch.arange(side, **f64), indexing="ij")
    d1, d2 = xx - xc, yy - yc
    R2 = ((1 - g1) ** 2 + g2 ** 2) * d1 * d1 + ((1 + g1) ** 2 + g2 ** 2) * d2 * d2 - 4 * g2 * d1 * d2
    r = torch.sqrt(torch.clamp(R2, min=0.0)) / (1 - gabs)
    prof = torch.exp(-b * (r / re) ** (1.0 / n))
    beta = t(p["beta"])
    if bool((beta > 0).any()):
        # Moffat stars (Sec. 4.2): re holds r_d
        prof = torch.where(beta > 0, (1.0 + (r / re) ** 2) ** (-beta), prof)
    by_snr = torch.as_tensor(p["by_snr"][sel], device=device).view(k, 1, 1)
    amp_snr = t(p["snr"]) / torch.sqrt((prof * prof).sum(dim=(1, 2), keepdim=True))
    I0_flux = t(p["flux"]) / torch.as_tensor(
        sersic_flux(1.0, p["re"][sel], p["n"][sel], p["gabs"][sel]), **f64).view(k, 1, 1)
    I0 = torch.where(by_snr, amp_snr, I0_flux)
    img = I0 * prof
    if noise:
        pix = torch.arange(side * side, device=device, dtype=torch.int64).view(1, side, side)
        # a stamp's noise counters: id << 15 up to 181 x 181 pixels, id << 20 for larger images
        shift = 15 if side * side <= (1 << 15) else 20
        cnt = (torch.as_tensor(ids[sel], device=device, dtype=torch.int64).view(k, 1, 1) << shift) + pix
        img = img + normal(seed, _S_NOISE, cnt)
    return img, I0.view(k).cpu().numpy(), g1.view(k).cpu().numpy(), g2.view(k).cpu().numpy(), \
        xc.view(k).cpu().numpy(), yc.view(k).cpu().numpy(), b.view(k).cpu().numpy()


def make_workload(which: int, count: int | None = None, first: int = 0, device="cpu",
                  noise: bool = True, ids: np.ndarray | None = None) -> StampBatch:
    """Stamps `first .. first+count-1` (or the explicit `ids`) of workload `which`.

    Pixels are fp32, packed back to back in stamp order (no padding, so offsets
    are generally not 16-byte aligned for ragged workloads)."""
    wl = WORKLOADS[which]
    if ids is None:
        count = wl.count - first if count is None else count
        ids = np.arange(first, first + count, dtype=np.int64)
    ids = np.asarray(ids, dtype=np.int64)
    p = _draw_params(wl, ids)
    N = ids.size
    side = p["side"]
    area = side * side
    offset = np.zeros(N, dtype=np.int64)
    if N:
        offset[1:] = np.cumsum(area)[:-1]
    total = int(area.sum())
    pix = torch.empty(total, dtype=torch.float32, device=device)
    truth = {k: np.zeros(N) for k in ("I0", "g1", "g2", "xc", "yc", "b")}
    for s in np.unique(side):
        sel = np.nonzero(side == s)[0]
        # chunk to bound temporary memory (float64 [k, s, s] tensors)
        step = max(1, (1 << 24) // int(s * s))
        for c0 in range(0, sel.size, step):
            cs = sel[c0:c0 + step]
            img, I0, g1, g2, xc, yc, b = _render(int(s), p, cs, ids, wl.seed, device, noise)
            img32 = img.to(torch.float32).reshape(cs.size, -1)
            # scatter each stamp to its offset (stamps of one side are not contiguous)
            o = torch.as_tensor(offset[cs], device=device).view(-1, 1)
            dst = o + torch.arange(int(s * s), device=device).view(1, -1)
            pix[dst.reshape(-1)] = img32.reshape(-1)
            for k_, v in (("I0", I0), ("g1", g1), ("g2", g2), ("xc", xc), ("yc", yc), ("b", b)):
                truth[k_][cs] = v
    truth.update(n=p["n"], re=p["re"], star=p["star"], beta=p["beta"], id=ids)
    truth["flux"] = sersic_flux(truth["I0"], p["re"], p["n"], p["gabs"])
    return StampBatch(pix=pix,
                      offset=torch.as_tensor(offset, device=device),
                      h=torch.as_tensor(side.astype(np.int32), device=device),
                      w=torch.as_tensor(side.astype(np.int32), device=device),
                      truth=truth)


def encode_bf16(batch: StampBatch) -> StampBatch:
    """Store pixels as bf16 scaled per stamp by max|I| (the decoded value is bf16 * scale)."""
    N = batch.count
    dev = batch.pix.device
    scale = torch.empty(N, dtype=torch.float32, device=dev)
    out = torch.empty(batch.pix.numel(), dtype=torch.bfloat16, device=dev)
    offs = batch.offset.to("cpu").numpy()
    area = (batch.h.to(torch.int64) * batch.w.to(torch.int64)).to("cpu").numpy()
    if N and np.array_equal(offs[1:], offs[:-1] + area[:-1]):
        # stamps back to back: per-stamp maxima over chunks of about 2^24 pixels
        i0 = 0
        while i0 < N:
            i1 = int(np.searchsorted(offs, offs[i0] + (1 << 24), side="left"))
            i1 = max(i1, i0 + 1)
            a = torch.as_tensor(area[i0:i1], device=dev)
            o0, o1 = int(offs[i0]), int(offs[i1 - 1] + area[i1 - 1])
            seg = batch.pix[o0:o1]
            sid = torch.repeat_interleave(torch.arange(i1 - i0, device=dev), a)
            mx = torch.zeros(i1 - i0, dtype=torch.float32, device=dev)
            mx = mx.scatter_reduce(0, sid, seg.abs(), reduce="amax", include_self=True).clamp(min=1e-30)
            scale[i0:i1] = mx
            out[o0:o1] = (seg / mx[sid]).to(torch.bfloat16)
            i0 = i1
        return dataclasses.replace(batch, pix=out, scale=scale)
    for i in range(N):
        o, a = int(batch.offset[i]), int(batch.h[i]) * int(batch.w[i])
        seg = batch.pix[o:o + a]
        s = seg.abs().max().clamp(min=1e-30)
        scale[i] = s
        out[o:o + a] = (seg / s).to(torch.bfloat16)
    return dataclasses.replace(batch, pix=out, scale=scale)


def moffat_stamp(h: int, w: int, *, beta: float, rd: float, g1: float, g2: float,
                 xc: float, yc: float, I0: float, noise_sigma: float = 0.0,
                 seed: int = 0) -> np.ndarray:
    """One elliptical Moffat star (Sec. 4.2), I0 (1 + (r / r_d)^2)^-beta with the
    semi-major-axis radius r = R(g) / (1 - |g|), sampled at pixel centres,
    float64 (h, w); noise from the same counter-based normals as single_stamp."""
    gabs = math.hypot(g1, g2)
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    d1, d2 = xx - xc, yy - yc
    R2 = ((1 - g1) ** 2 + g2 ** 2) * d1 * d1 + ((1 + g1) ** 2 + g2 ** 2) * d2 * d2 - 4 * g2 * d1 * d2
    r2 = np.maximum(R2, 0.0) / (1 - gabs) ** 2
    img = I0 * (1.0 + r2 / (rd * rd)) ** (-beta)
    if noise_sigma:
        cnt = torch.arange(h * w, dtype=torch.int64)
        img = img + noise_sigma * normal(seed, 7, cnt).numpy().reshape(h, w)
    return img


def single_stamp(h: int, w: int, *, n: float, re: float, g1: float, g2: float,
                 xc: float, yc: float, I0: float, noise_sigma: float = 0.0,
                 seed: int = 0, supersample: int = 1) -> np.ndarray:
    """One noiseless (or noisy) elliptical Sérsic stamp, float64 (h, w), for pins.

    With supersample=s each pixel is the mean of s x s point samples on a
    regular sub-grid (used only by brute-force flux pins)."""
    gabs = math.hypot(g1, g2)
    b = float(sersic_b(np.array([n]))[0])
    s = supersample
    sub = (np.arange(s) + 0.5) / s - 0.5
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    acc = np.zeros((h, w))
    for oy in sub:
        for ox in sub:
            d1, d2 = xx + ox - xc, yy + oy - yc
            R2 = ((1 - g1) ** 2 + g2 ** 2) * d1 * d1 + ((1 + g1) ** 2 + g2 ** 2) * d2 * d2 - 4 * g2 * d1 * d2
            r = np.sqrt(np.maximum(R2, 0.0)) / (1 - gabs)
            acc += I0 * np.exp(-b * (r / re) ** (1.0 / n))
    img = acc / (s * s)
    if noise_sigma:
        cnt = torch.arange(h * w, dtype=torch.int64)
        img = img + noise_sigma * normal(seed, 7, cnt).numpy().reshape(h, w)
    return img
