"""The C ABI without a GPU: the library builds, loads, exports every symbol the
header declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1506_07933_gb300 import afft
from paper_1506_07933_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "afft.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return afft.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(afft_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("afft_plan_create", "afft_execute_forward", "afft_execute_backward", "afft_plan_destroy",
              "afft_plan_workspace_bytes", "afft_status_string"):
        assert s in syms
    assert sorted(afft.EXPORTS) == syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def _create(lib, n, kind, prec):
    p = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 3)(*n)
    return lib.afft_plan_create(ctypes.byref(p), arr, kind, prec), p


@pytest.mark.parametrize("n,kind,prec,code", [
    ((8, 8, 7), 0, 0, 2),        # prime factor 7
    ((0, 8, 8), 0, 0, 2),        # zero size
    ((8, -4, 8), 0, 1, 2),       # negative size
    ((8, 8, 11), 1, 0, 2),       # size check precedes the parity check
    ((8, 8, 9), 1, 0, 3),        # r2c with odd n2
    ((8, 8, 8), 5, 0, 4),        # kind
    ((8, 8, 8), 0, 7, 5),        # precision
    ((8, 8, 7), 0, 2, 2),        # split precision: same size rules
    ((8, 8, 9), 1, 2, 3),        # split precision: r2c with odd n2
    ((8, 8, 3 ** 15), 0, 0, 9),  # no split into two factors <= 4096
    ((8, 8, 16384), 1, 1, 9),    # r2c half length 8192
])
def test_plan_create_rejects_bad_arguments(lib, n, kind, prec, code):
    st, p = _create(lib, n, kind, prec)
    assert st == code, (st, afft.status_string(st))
    assert not p.value


def test_null_arguments(lib):
    arr = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.afft_plan_create(None, arr, 0, 0) == 1
    p = ctypes.c_void_p()
    assert lib.afft_plan_create(ctypes.byref(p), None, 0, 0) == 1
    assert lib.afft_plan_destroy(None) == 0
    assert lib.afft_execute_forward(None, None, None, None) == 1
    assert lib.afft_execute_backward(None, None, None, None) == 1
    assert lib.afft_execute_forward_host(None, None, None, None, None, None) == 1
    assert lib.afft_fill_uniform(None, 4, 1, 0, None) == 1
    assert lib.afft_plan_workspace_bytes(None) == 0
    assert lib.afft_plan_input_bytes(None) == 0
    assert lib.afft_plan_launches(None, 0) == 0
    assert lib.afft_plan_wait_probe(None, 1000, None) == 1


def test_status_strings(lib):
    seen = set()
    for code in range(10):
        s = afft.status_string(code)
        assert s and s != "unknown status"
        seen.add(s)
    assert len(seen) == 10
    assert afft.status_string(99) == "unknown status"


def test_error_is_raised_from_python(lib):
    with pytest.raises(afft.AfftError) as e:
        afft.afft_plan_create((8, 8, 7), afft.C2C, afft.F32)
    assert e.value.status == 2


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(afft, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        afft.load(str(tmp_path / "libafft.so"))


def test_tuning_calls_reject_null(lib):
    cfg = (ctypes.c_int64 * 6)()
    assert lib.afft_plan_get_tuning(None, cfg) == 1
    assert lib.afft_plan_set_tuning(None, cfg) == 1
    assert lib.afft_plan_set_blocked(None, 1) == 1


def test_tuning_cache_file(tmp_path):
    """The autotuner cache: per-key entries, kept across stores, and malformed files or entries
    read as missing (the plan then tunes again)."""
    path = str(tmp_path / "tune.json")
    k1 = afft.tuning_key((512, 512, 512), afft.R2C, afft.F32, None, "GPU A")
    k2 = afft.tuning_key((512, 512, 512), afft.R2C, afft.F32, 4, "GPU A")
    k3 = afft.tuning_key((512, 512, 512), afft.R2C, afft.F32, None, "GPU B")
    assert len({k1, k2, k3}) == 3 and "512x512x512/r2c/f32/batch1/GPU A" == k1
    assert afft.tuning_cache_lookup(path, k1) is None
    afft.tuning_cache_store(path, k1, [4096, 1, 1, 0])
    afft.tuning_cache_store(path, k2, [2048, 0, 1, 33554432, 0, 1])
    assert afft.tuning_cache_lookup(path, k1) == [4096, 1, 1, 0, 0, 0]      # a 4-entry record, padded
    assert afft.tuning_cache_lookup(path, k2) == [2048, 0, 1, 33554432, 0, 1]
    assert afft.tuning_cache_lookup(path, k3) is None
    afft.tuning_cache_store(path, k1, [1024, 0, 0, 0, 0, 0])
    assert afft.tuning_cache_lookup(path, k1) == [1024, 0, 0, 0, 0, 0]
    with open(path, "w") as fh:
        fh.write('{"%s": [1, 2]}' % k1)
    assert afft.tuning_cache_lookup(path, k1) is None
    with open(path, "w") as fh:
        fh.write("not json")
    assert afft.tuning_cache_lookup(path, k1) is None
    afft.tuning_cache_store(path, k1, [4096, 1, 1, 0, 1, 0])
    assert afft.tuning_cache_lookup(path, k1) == [4096, 1, 1, 0, 1, 0]


def test_noalloc_source_calls_no_allocator():
    """The no-allocation entry point's translation unit names no allocating CUDA call in its code
    (comments aside), so a later edit that adds one fails here before it reaches a GPU."""
    path = os.path.join(os.path.dirname(libbuild.__file__), "csrc", "noalloc.cu")
    src = open(path).read()
    code = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    code = re.sub(r"//[^\n]*", "", code)
    for name in ("cudaMalloc", "cudaMallocAsync", "cudaMallocManaged", "cudaMallocHost", "cudaHostAlloc",
                 "cudaFree", "cudaFreeAsync", "cudaMallocPitch", "cudaMalloc3D", "cuMemAlloc", "cuMemCreate",
                 "malloc(", "new "):
        assert name not in code, name
    assert "cudaGetSymbolAddress" in code


@pytest.mark.parametrize("n,kind,axes,code", [
    ((8, 8, 8), 0, 0, 12),        # empty axis set
    ((8, 8, 8), 0, 8, 12),        # bit beyond axis 2
    ((8, 8, 8), 1, 3, 12),        # r2c without the halved contiguous axis
    ((8, 8, 7), 0, 7, 2),         # a transformed axis must be 2/3/5-smooth
    ((8, 8, 0), 0, 3, 2),         # an untransformed one must still have a length
    ((7, 8, 9), 1, 6, 3),         # an untransformed n0 = 7 is fine, an odd r2c n2 is not
])
def test_plan_create_axes_rejects_bad_arguments(lib, n, kind, axes, code):
    p = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 3)(*n)
    assert lib.afft_plan_create_axes(ctypes.byref(p), arr, 1, kind, 0, axes) == code
    assert not p.value


def test_backward_scale_and_copy_2d_argument_checks(lib):
    assert lib.afft_plan_set_backward_scale(None, 1.0) == 1
    assert lib.afft_plan_backward_scale(None) == 0.0
    assert lib.afft_copy_2d(None, 16, None, 16, 8, 0, None) == 0      # nothing to copy
    assert lib.afft_copy_2d(None, 16, None, 16, 8, 2, None) == 1
    buf = ctypes.create_string_buffer(64)
    assert lib.afft_copy_2d(buf, 8, buf, 16, 16, 2, None) == 2        # width beyond the pitch
    assert afft.status_string(12) != "unknown status"
