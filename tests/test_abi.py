"""The C ABI library builds, loads and exports what include/fse.h declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1203_0571_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fse.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(fse_\w+)\s*\(", text, flags=re.M)


@pytest.fixture(scope="module")
def lib():
    return binding.load()


def test_header_declares_binding_exports():
    assert declared_functions() == binding.EXPORTS


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layout_matches_c(tmp_path):
    """sizeof/offsetof of the ABI structs from a C compiler equal the ctypes/numpy views."""
    src = tmp_path / "layout.c"
    fields_r = [n for n in binding.RESULT_DTYPE.names]
    fields_o = [f for f, _ in binding.Opts._fields_]
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "fse.h"', 'int main(void){',
            'printf("%zu %zu %zu\\n", sizeof(fse_result), sizeof(fse_opts), sizeof(fse_stamp));']
    body += [f'printf("%zu ", offsetof(fse_result, {f}));' for f in fields_r]
    body += ['printf("\\n");']
    body += [f'printf("%zu ", offsetof(fse_opts, {f}));' for f in fields_o]
    body += ['printf("\\n"); return 0; }']
    src.write_text("\n".join(body))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    assert sizes == [64, ctypes.sizeof(binding.Opts), 16]
    assert [int(x) for x in lines[1].split()] == [binding.RESULT_DTYPE.fields[f][1] for f in fields_r]
    assert [int(x) for x in lines[2].split()] == [getattr(binding.Opts, f).offset for f in fields_o]
    assert binding.STAMP_DTYPE.itemsize == 16


def test_opts_defaults(lib):
    o = binding.default_opts()
    assert o.size == ctypes.sizeof(binding.Opts)
    assert o.k_gain == 0.0 and o.sigw_mode == 1 and o.max_pix == 0
    assert o.n_min == 0.2 and o.n_max == 10.0


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.fse_create(ctypes.byref(h), 0) != 0
    assert not h.value


def test_index_packing():
    import torch
    idx = binding.make_index([0, 1024, 5], [32, 16, 3], [32, 64, 7], device="cpu")
    arr = idx.numpy().view(binding.STAMP_DTYPE).reshape(-1)
    assert arr["offset"].tolist() == [0, 1024, 5]
    assert arr["h"].tolist() == [32, 16, 3] and arr["w"].tolist() == [32, 64, 7]


def test_static_entry_rejects_oversized_batch(lib):
    """The batch limit of the static-scratch entry is checked before any CUDA call."""
    err = ctypes.create_string_buffer(256)
    rc = lib.fse_fit_batch_static(None, binding.FSE_F32, None, None, 1 << 31, None,
                                  ctypes.byref(binding.default_opts()), None, None, err, len(err))
    assert rc == binding.FSE_EINVAL
    assert b"static work counter" in err.value


def test_null_context_is_rejected_by_every_entry_point(lib):
    """Every entry point that takes a context returns FSE_EINVAL for a NULL one,
    before any CUDA call, so it is safe on a machine without a GPU."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    takes_ctx = re.findall(r"^\s*int\s+(fse_\w+)\s*\(\s*(?:const\s+)?fse_ctx\s*\*", text, flags=re.M)
    takes_ctx = [f for f in takes_ctx if f not in ("fse_create",)]
    assert {"fse_fit_batch", "fse_fit_batch_host", "fse_star_fit", "fse_moment_vjp", "fse_cutout",
            "fse_sersic_chi2_grad", "fse_sync_check"} <= set(takes_ctx), takes_ctx
    for name in takes_ctx:
        fn = getattr(lib, name)
        types = fn.argtypes
        assert types, f"{name} has no ctypes signature in the binding"
        args = []
        for t in types:
            if t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t):
                args.append(0)
            elif t in (ctypes.c_float, ctypes.c_double):
                args.append(0.0)
            else:
                args.append(None)
        assert fn(*args) == binding.FSE_EINVAL, name
    assert lib.fse_last_error(None) == b"null context"


def test_index_layout_is_checked_before_the_library():
    """Only the fse_stamp layout reaches the C ABI: int64 [N, 2] (make_index) on
    the call's device type, contiguous; numpy STAMP_DTYPE or int64 [N, 2] on the
    host.  Other layouts raise TypeError in the binding."""
    import torch
    idx = binding.make_index([0, 1024, 5], [32, 16, 3], [32, 64, 7], device="cpu")
    ptr, n = binding._index(idx, "cpu")
    assert n == 3 and ptr.value == idx.data_ptr()
    assert binding._index(idx[1:], "cpu")[1] == 2 and binding._index(idx[:0], "cpu")[1] == 0
    arr = idx.numpy().view(binding.STAMP_DTYPE).reshape(-1)
    ptr, n = binding._index(arr, "cpu")
    assert n == 3 and ptr.value == arr.ctypes.data
    assert binding._index(idx.numpy(), "cpu")[1] == 3
    bad = [idx.to(torch.int32), idx.float(), idx.reshape(-1), torch.zeros((3, 3), dtype=torch.int64),
           idx.t().contiguous().t(), [[0, 1]]]
    for b in bad:
        with pytest.raises(TypeError):
            binding._index(b, "cpu")
    with pytest.raises(TypeError):
        binding._index(idx, "cuda")          # a host tensor handed to a device call
    with pytest.raises(TypeError):
        binding._index(idx.numpy(), "cuda")  # numpy only for host calls
    with pytest.raises(TypeError):
        binding._index(idx.numpy()[:, :1].copy(), "cpu")
