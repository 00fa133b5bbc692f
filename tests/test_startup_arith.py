"""The integer arithmetic of the estimator's start-up growth curve (Sec. 4.1),
restated with numpy and checked exhaustively on the CPU:

- the ring index ceil(sqrt(d2)) from one approximate square root, with the
  root rounded through the bits of 2^23 and corrected by one comparison, over
  every d2 a stamp of sides <= 128 can produce, with the root off by up to
  2^-21 relative (the hardware approximation is within about 2^-22);
- the three 32-bit pieces of each 64-bit fixed-point pixel value, whose sums
  over a stamp stay inside 32 bits and rebuild the 64-bit sum exactly;
- the number of rings the tile reserves, against a brute-force maximum over
  all stamp shapes;
- the cut-out's ring index for images of sides up to 32768 (d2 < 2^31): the
  truncated approximate root and two conditional increments, next to every
  perfect square and on random d2.
"""
import math

import numpy as np


def ring_fast(d2, rel_err):
    f = (np.int32(0x4B000000) | d2.astype(np.int32)).view(np.float32) - np.float32(8388608.0)
    assert np.array_equal(f.astype(np.int64), d2)        # the float of d2, exactly
    r = (np.sqrt(f.astype(np.float64)) * (1.0 + rel_err)).astype(np.float32)
    k0 = (r + np.float32(8388608.0)).view(np.int32).astype(np.int64) - 0x4B000000
    return k0 + (k0 * k0 < d2)


def test_ring_index_exhaustive():
    d2 = np.arange(0, 2 * 127 * 127 + 1, dtype=np.int64)
    want = np.array([math.isqrt(int(x)) + (0 if math.isqrt(int(x)) ** 2 == int(x) else 1) for x in d2])
    for rel in (-2.0 ** -21, -2.0 ** -23, 0.0, 2.0 ** -23, 2.0 ** -21):
        assert np.array_equal(ring_fast(d2, rel), want), rel


def pieces(q, npix):
    b = 31 - (0 if npix == 1 else int(math.ceil(math.log2(npix))))
    mask = (1 << b) - 1
    q0 = np.array([int(x) & mask for x in q], dtype=np.int64)
    q1 = np.array([(int(x) >> b) & mask for x in q], dtype=np.int64)   # >> of a negative int floors
    q2 = np.array([int(x) >> (2 * b) for x in q], dtype=np.int64)
    return b, q0, q1, q2


def test_fixed_point_pieces():
    rng = np.random.default_rng(0)
    for npix in (1, 2, 3, 255, 256, 2304, 9999, 16384):
        lim = (1 << 62) // npix          # |q| of one pixel: amax * npix * 2^S < 2^62
        for trial in range(6):
            if trial == 0:
                q = [lim - 1] * npix
            elif trial == 1:
                q = [-(lim - 1)] * npix
            else:
                q = [int(x) for x in rng.integers(-lim + 1, lim, npix)]
            b, q0, q1, q2 = pieces(q, npix)
            for x, a0, a1, a2 in zip(q[:50], q0[:50], q1[:50], q2[:50]):
                assert int(a2) * (1 << (2 * b)) + int(a1) * (1 << b) + int(a0) == x
            s0, s1, s2 = int(q0.sum()), int(q1.sum()), int(q2.sum())
            assert 0 <= s0 < 2 ** 32 and 0 <= s1 < 2 ** 32, (npix, s0, s1)
            assert -2 ** 31 <= s2 < 2 ** 31, (npix, s2)
            assert s0 + (s1 << b) + (s2 << (2 * b)) == sum(q)


def ring_slots(max_pix):
    best = 0
    for h in range(1, 129):
        w = max_pix // h
        if w < 1:
            break
        w = min(w, 128)
        best = max(best, (h - 1) ** 2 + (w - 1) ** 2)
    k = 0
    while k * k < best:
        k += 1
    return k + 2


def test_ring_slots_cover_every_shape():
    # every stamp h x w (sides <= 128, h w <= max_pix) with any brightest pixel
    # needs kmax + 1 = ceil(corner distance) + 2 rings at most
    need = {}
    for h in range(1, 129):
        for w in range(1, 129):
            k = math.isqrt((h - 1) ** 2 + (w - 1) ** 2)
            if k * k < (h - 1) ** 2 + (w - 1) ** 2:
                k += 1
            need[(h, w)] = k + 2
    for max_pix in (1, 2, 16, 100, 128, 129, 256, 576, 1024, 2300, 2304, 4096, 9216, 16384):
        worst = max(v for (h, w), v in need.items() if h * w <= max_pix)
        assert ring_slots(max_pix) == worst, max_pix
    assert ring_slots(48 * 48) == 131 and ring_slots(128 * 128) == 182


def ring_ceil32(d2, rel_err):
    """The cut-out's ring index for d2 < 2^31: the float nearest d2, its root
    off by rel_err, truncated, and two conditional increments (uint32)."""
    f = d2.astype(np.float32)                                   # round to nearest
    r = (np.sqrt(f.astype(np.float64)) * (1.0 + rel_err)).astype(np.float32)
    k = r.astype(np.uint64)                                     # truncation
    d = d2.astype(np.uint64)
    for _ in range(2):
        k = k + ((k * k) < d).astype(np.uint64)
    assert np.all(k * k < 2 ** 32)
    return k.astype(np.int64)


def test_cutout_ring_index_near_squares():
    """Images with both sides <= 32768: d2 <= 2 * 32767^2 < 2^31.  The hard
    cases sit next to perfect squares, where the root is closest to an
    integer; every square up to the largest d2 is taken with its neighbours,
    plus random d2, and the root is perturbed by up to 2^-21 relative."""
    dmax = 2 * 32767 ** 2
    k = np.arange(0, math.isqrt(dmax) + 2, dtype=np.int64)
    d2 = np.concatenate([k * k - 1, k * k, k * k + 1,
                         np.random.default_rng(1).integers(0, dmax + 1, 200000)])
    d2 = d2[(d2 >= 0) & (d2 <= dmax)]
    root = np.array([math.isqrt(int(x)) for x in d2], dtype=np.int64)
    want = root + (root * root != d2)
    for rel in (-2.0 ** -21, -2.0 ** -23, 0.0, 2.0 ** -23, 2.0 ** -21):
        assert np.array_equal(ring_ceil32(d2, rel), want), rel
