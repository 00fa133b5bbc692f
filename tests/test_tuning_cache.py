"""The launch-shape cache file (fse_tuning_save / fse_tuning_load), read on
the CPU through fse_tuning_read: the file is the JSON document the save call
writes (one entry per line), and an entry is taken only for the named device,
the library's size classes and shapes the autotuner could have chosen."""
import json

import numpy as np
import pytest

from paper_1203_0571_gb300 import binding as B

CLASS_PIX = [16 * 16, 24 * 24, 32 * 32, 48 * 48, 64 * 64, 96 * 96, 128 * 128]


def entry(device, dtype="f32", inv_var=0, cta=(4, 4, 4, 4, 4, 4, 8), nw=(1, 1, 1, 1, 2, 4, 8), pix=CLASS_PIX):
    return json.dumps({"device": device, "dtype": dtype, "inv_var": inv_var, "class_pix": list(pix),
                       "warps_per_cta": list(cta), "warps_per_stamp": list(nw)})


def write(path, entries, fmt="libfse-launch-shapes/1"):
    with open(path, "w") as f:
        f.write(json.dumps({"format": fmt})[:-1] + ', "entries": [\n')
        f.write(",\n".join(entries) + "\n]}\n")
    # the file is valid JSON, as the save call writes it
    json.load(open(path))


def test_entries_are_read_for_their_device(tmp_path):
    p = str(tmp_path / "shapes.json")
    write(p, [entry("GPU A"), entry("GPU A", dtype="bf16", cta=(2, 2, 2, 2, 4, 4, 8)),
              entry("GPU B", cta=(8, 8, 8, 8, 4, 4, 8), nw=(1, 1, 1, 1, 2, 4, 8))])
    n, s = B.tuning_read(p, "GPU A")
    assert n == 2
    assert s[0, 0, :, 0].tolist() == [4, 4, 4, 4, 4, 4, 8]
    assert s[0, 0, :, 1].tolist() == [1, 1, 1, 1, 2, 4, 8]
    assert s[1, 0, :, 0].tolist() == [2, 2, 2, 2, 4, 4, 8]
    assert np.all(s[:, 1] == -1)                   # no inverse-variance entries in the file
    n, s = B.tuning_read(p, "GPU B")
    assert n == 1 and s[0, 0, 0].tolist() == [8, 1]
    assert B.tuning_read(p, "GPU C")[0] == 0


def test_default_shapes_are_zero(tmp_path):
    p = str(tmp_path / "shapes.json")
    write(p, [entry("GPU A", inv_var=1, cta=(0,) * 7, nw=(0,) * 7)])
    n, s = B.tuning_read(p, "GPU A")
    assert n == 1 and np.all(s[0, 1] == 0) and np.all(s[0, 0] == -1)


@pytest.mark.parametrize("bad", [
    dict(cta=(3, 4, 4, 4, 4, 4, 8)),                       # not a power of two
    dict(cta=(4, 4, 4, 4, 4, 2, 8), nw=(1, 1, 1, 1, 2, 4, 8)),   # fewer warps per CTA than per stamp
    dict(cta=(4, 4, 4, 4, 4, 4, 8), nw=(1, 1, 1, 1, 2, 4, 1)),   # eight 128^2 tiles: past 227 KB
    dict(pix=CLASS_PIX[:-1] + [100 * 100]),                # another library's size classes
    dict(dtype="f16"),                                     # unknown dtype
])
def test_invalid_entries_are_skipped(tmp_path, bad):
    p = str(tmp_path / "shapes.json")
    write(p, [entry("GPU A", **bad)])
    assert B.tuning_read(p, "GPU A")[0] == 0


def test_other_formats_and_missing_files(tmp_path):
    p = str(tmp_path / "shapes.json")
    write(p, [entry("GPU A")], fmt="libfse-launch-shapes/0")
    assert B.tuning_read(p, "GPU A")[0] == 0
    with pytest.raises(B.FseError):
        B.tuning_read(str(tmp_path / "missing.json"), "GPU A")
