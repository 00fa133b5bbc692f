"""The box the moment passes sum over (the pixels whose Gaussian weight is at
least 2^-40), restated with numpy in fp32 and checked on the CPU: over random
weight states (centre, g, s_w) and stamp shapes, every pixel with
R^2 <= 80 ln 2 s_w^2 (Eq. A1's R^2) lies inside the box, and the box is inside
the stamp."""
import numpy as np

CUT = np.float32(7.4446500)   # sqrt(80 ln 2)


def weight_box(xi, yi, xf, yf, g1, g2, sw, h, w):
    f = np.float32
    g1, g2, sw, xf, yf = f(g1), f(g2), f(sw), f(xf), f(yf)
    gg = g1 * g1 + g2 * g2
    rc = CUT * sw / (f(1) - gg)
    hx = min(rc * np.sqrt(f(1) + gg + f(2) * g1) + f(1), f(4096))
    hy = min(rc * np.sqrt(f(1) + gg - f(2) * g1) + f(1), f(4096))
    xc, yc = f(xi) + xf, f(yi) + yf
    c0 = max(0, int(np.floor(xc - hx)))
    r0 = max(0, int(np.floor(yc - hy)))
    c1 = min(w - 1, int(np.ceil(xc + hx)))
    r1 = min(h - 1, int(np.ceil(yc + hy)))
    if not (c1 >= c0 and r1 >= r0):
        return 0, 0, h, w
    return r0, c0, r1 - r0 + 1, c1 - c0 + 1


def test_box_holds_every_pixel_above_the_cut():
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(3000):
        h, w = rng.integers(1, 129, 2)
        gabs = rng.uniform(0, 0.949)
        phi = rng.uniform(0, 2 * np.pi)
        g1, g2 = gabs * np.cos(phi), gabs * np.sin(phi)
        sw = rng.uniform(0.5, max(0.5, min(h, w) / 2))
        xi, yi = rng.integers(0, w), rng.integers(0, h)
        xf, yf = rng.uniform(-0.5, 0.5, 2)
        r0, c0, bh, bw = weight_box(xi, yi, xf, yf, g1, g2, sw, h, w)
        assert 0 <= r0 and 0 <= c0 and bh >= 1 and bw >= 1 and r0 + bh <= h and c0 + bw <= w
        t1 = np.arange(w)[None, :] - (xi + xf)
        t2 = np.arange(h)[:, None] - (yi + yf)
        gg = g1 * g1 + g2 * g2
        R2 = (1 + gg - 2 * g1) * t1 ** 2 + (1 + gg + 2 * g1) * t2 ** 2 - 4 * g2 * t1 * t2
        inside = R2 <= 80 * np.log(2) * sw * sw
        box = np.zeros((h, w), bool)
        box[r0:r0 + bh, c0:c0 + bw] = True
        assert not np.any(inside & ~box), (h, w, g1, g2, sw, xi, yi)
        worst = max(worst, box.sum() / (h * w))
    assert worst <= 1.0


def test_box_saves_work_on_compact_objects():
    # a round weight of s_w = 1 px in the middle of a 48 x 48 stamp: a box of
    # side 2 * ceil(7.44 + 1) + 1 = 19 at most
    r0, c0, bh, bw = weight_box(24, 24, 0.0, 0.0, 0.0, 0.0, 1.0, 48, 48)
    assert bh <= 19 and bw <= 19
    # a weight wider than the stamp: the whole stamp
    assert weight_box(24, 24, 0.1, -0.2, 0.3, 0.1, 12.0, 48, 48) == (0, 0, 48, 48)


def test_bench_counts_the_same_box():
    """bench.py's operation count takes the moment passes over the same box."""
    import bench
    rng = np.random.default_rng(3)
    n = 500
    rec = np.zeros(n, dtype=[("x0", "f4"), ("y0", "f4"), ("e1", "f4"), ("e2", "f4"), ("sigma_w", "f4")])
    rec["x0"] = rng.uniform(0, 47, n)
    rec["y0"] = rng.uniform(0, 47, n)
    gabs, phi = rng.uniform(0, 0.9, n), rng.uniform(0, 2 * np.pi, n)
    rec["e1"], rec["e2"] = gabs * np.cos(phi), gabs * np.sin(phi)
    rec["sigma_w"] = rng.uniform(0.5, 6, n)
    got = bench.box_pixels(rec, 48, 48)
    for j in range(n):
        xi, yi = int(np.rint(rec["x0"][j])), int(np.rint(rec["y0"][j]))
        r0, c0, bh, bw = weight_box(xi, yi, rec["x0"][j] - xi, rec["y0"][j] - yi, rec["e1"][j], rec["e2"][j],
                                    rec["sigma_w"][j], 48, 48)
        # fp32 versus fp64 rounding of the edges moves a side by a pixel at most
        assert abs(got[j] - bh * bw) <= bh + bw + 1, (j, got[j], bh * bw)
