"""Run the pipe-throughput microbenchmark (libfse_peaks.so) and print JSON.

    python -m paper_1203_0571_gb300.pipe_peaks [device]
"""
from __future__ import annotations

import ctypes
import json
import sys

from . import _build


def measure(device: int = 0) -> dict:
    _build.build()
    lib = ctypes.CDLL(_build.PEAKS_LIB)
    lib.fse_pipe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    out = (ctypes.c_double * 7)()
    rc = lib.fse_pipe_peaks(out, device)
    if rc:
        raise RuntimeError(f"fse_pipe_peaks failed ({rc})")
    sms, mhz = out[5], out[6]
    per_clk = lambda g: g * 1e9 / (sms * mhz * 1e6)
    return {"ffma_gops": out[0], "ex2_gops": out[1], "lg2_gops": out[2], "dfma_gops_32lanes": out[3],
            "dfma_warp_instr_per_s_1lane_e9": out[4], "sms": sms, "sm_max_mhz": mhz,
            "per_sm_per_clk_at_max": {"ffma": per_clk(out[0]), "ex2": per_clk(out[1]),
                                      "lg2": per_clk(out[2]), "dfma_32lanes": per_clk(out[3]),
                                      "dfma_1lane_warp_instr": per_clk(out[4])}}


if __name__ == "__main__":
    print(json.dumps(measure(int(sys.argv[1]) if len(sys.argv) > 1 else 0), indent=1))
