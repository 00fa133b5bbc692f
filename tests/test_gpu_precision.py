"""Low-SNR precision subsample (SNR 10-30, n up to 8, 32-64 px), needs a GB300.

At this noise level a few fits lie in valleys so flat (condition numbers
1e5-1e6, n above 6) that the fp32 rounding of the model values moves the
minimum by more than 1e-4 in r_e or n while chi^2 agrees to 1e-8: on the full
10,000-stamp subsample 10 of 7,611 gated stamps.  The test therefore asks for
99.8 % of the gated stamps within the parity tolerance on every output, on
fp32 pixels and for the arithmetic on bf16 pixels, and for bf16 storage to
move r_e and n by far less than their statistical error.  The full report is
tests/precision_report.py."""
import pytest

import precision_report as PRR

pytestmark = pytest.mark.gpu


def test_lowsnr_precision_subsample():
    rep = PRR.run(1000)
    print(PRR.markdown(rep))
    f = rep["fp32"]
    assert f["gated"] >= 0.7 * f["total"], f["gated"]
    for k in PRR.KEYS:
        assert f[k]["within"] >= 0.998, (k, f[k])
    # the arithmetic on bf16 pixels is held to the same gate as on fp32
    c = rep["bf16_compute"]
    for k in PRR.KEYS:
        assert c[k]["within"] >= 0.998, (k, c[k])
    # storage: the median change of r_e and n stays far below the noise
    s = rep["oracle_sigma_median"]
    t = rep["bf16_total"]
    assert t["re"]["median"] <= 0.1 * s["re"] and t["n"]["median"] <= 0.1 * s["n"], (t["re"], t["n"], s)
