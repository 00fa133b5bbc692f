"""The seeded synthetic inputs follow their stated recipes (CPU only).

The generator holds none of the method's arithmetic; these checks pin the
workload shapes and distributions that the parity tests and the benchmark
rely on: parameter ranges, the star fraction, side rules, the matched-filter
SNR and the per-stamp regeneration."""
import numpy as np
import torch

from paper_1203_0571_gb300 import synth


def params(which, ids=None):
    wl = synth.WORKLOADS[which]
    ids = np.arange(wl.count, dtype=np.int64) if ids is None else np.asarray(ids, dtype=np.int64)
    return synth._draw_params(wl, ids)


def test_uniform48_recipe():
    p = params(1)
    star = p["star"]
    assert star.sum() == 100_000 // 5                      # exactly 20% stars
    gal = ~star
    assert np.all((p["n"][gal] >= 0.5) & (p["n"][gal] <= 4.0))
    assert np.all((p["re"][gal] >= 1.5) & (p["re"][gal] <= 5.0))
    assert np.all(p["gabs"][gal] <= 0.5)
    assert np.all((p["snr"] >= 15.0) & (p["snr"] <= 200.0))
    # stars: n = 0.5 (a Gaussian), r_e = FWHM / 2 with FWHM in [2, 4], |g| < 0.05
    assert np.all(p["n"][star] == 0.5)
    assert np.all((p["re"][star] >= 1.0) & (p["re"][star] <= 2.0))
    assert np.all(p["gabs"][star] < 0.05)
    assert np.all(p["side"] == 48)
    assert np.all((np.abs(p["dx"]) <= 1.0) & (np.abs(p["dy"]) <= 1.0))
    # shuffled: stars spread over the whole index range
    q = np.nonzero(star)[0]
    assert q.min() < 1000 and q.max() > 99_000


def test_ragged_and_precision_sides():
    p = params(2, np.arange(200_000))
    assert np.all((p["re"] >= 1.0) & (p["re"] <= 15.0))
    assert np.array_equal(p["side"], np.clip(np.rint(8.0 * p["re"]), 16, 128).astype(np.int64))
    # 8 r_e <= 120 with r_e <= 15: the upper clip at 128 never applies
    assert p["side"].min() == 16 and p["side"].max() == 120
    p = params(4, np.arange(200_000))
    assert p["side"].min() == 32 and p["side"].max() == 64
    assert len(np.unique(p["side"])) == 33
    p = params(5)
    assert np.all((p["snr"] >= 10.0) & (p["snr"] <= 30.0)) and p["n"].max() <= 8.0


def test_star_workloads_follow_sec42():
    for which in (6, 7):
        p = params(which, np.arange(5000))
        assert p["star"].all() and np.all(p["snr"] == 300.0)
        assert np.all(p["gabs"] <= 0.25)
        if which == 6:
            r50 = p["re"]                                  # n = 0.5: r_e is r50
        else:
            beta = p["beta"]
            assert np.all((beta >= 3.0) & (beta <= 5.0))
            r50 = p["re"] * np.sqrt(2.0 ** (1.0 / (beta - 1.0)) - 1.0)
        assert np.all((r50 >= 1.5) & (r50 <= 2.5))


def test_matched_filter_snr_sets_the_amplitude():
    """sqrt(sum m^2) / sigma equals the drawn SNR on noiseless stamps."""
    ids = np.arange(0, 100_000, 997)
    b = synth.make_workload(1, ids=ids, noise=False)
    p = params(1, ids)
    for i in range(b.count):
        m = b.stamp(i)
        assert abs(np.sqrt((m * m).sum()) / p["snr"][i] - 1.0) < 1e-6


def test_any_stamp_regenerates_alone():
    full = synth.make_workload(2, count=300)
    some = synth.make_workload(2, ids=[7, 150, 299])
    for j, i in enumerate((7, 150, 299)):
        assert np.array_equal(full.stamp(i), some.stamp(j))
    assert np.array_equal(full.truth["re"][[7, 150, 299]], some.truth["re"])


def test_noise_is_standard_normal():
    b = synth.make_workload(0, count=64)
    clean = synth.make_workload(0, count=64, noise=False)
    r = (b.pix.double() - clean.pix.double()).numpy()
    assert abs(r.mean()) < 0.01 and abs(r.std() - 1.0) < 0.01      # 65,536 samples
    # stamps draw different noise
    a0 = r[:32 * 32]
    a1 = r[32 * 32:2 * 32 * 32]
    assert abs(np.corrcoef(a0, a1)[0, 1]) < 0.1


def test_bf16_encoding_decodes_within_bf16_rounding():
    b = synth.make_workload(4, count=50)
    e = synth.encode_bf16(b)
    assert e.pix.dtype == torch.bfloat16 and e.scale.shape == (50,)
    for i in range(50):
        x, y = b.stamp(i), e.stamp(i)
        assert np.max(np.abs(x - y)) <= 2.0 ** -8 * np.max(np.abs(x))
