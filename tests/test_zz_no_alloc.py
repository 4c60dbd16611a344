"""afft_c2r_noalloc: the c2r backward transform for callers that cannot allocate.

Callers such as a framework that owns all device memory through its own arena,
or a service loop that must never wait on the CUDA allocator, cannot create a
plan (plan creation calls cudaMalloc).  The no-allocation entry point keeps its
twiddles and intermediate in one fixed device array instead.  These tests call
it through the C ABI and compare it with the plan-based c2r of the same size and
with the FP64 CPU oracle's c2r, within the tolerances the parity tests use, on
consecutive calls that share the array, and check that calls after the first
leave the device's free memory unchanged.  This file is collected last so that
a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1506_07933_gb300 import afft, synth
from paper_1506_07933_gb300 import build as libbuild

pytestmark = pytest.mark.gpu

TOL = {afft.F32: 2e-6, afft.F64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    libbuild.build()
    return afft.load()


def noalloc(lib, shape, prec, X, out):
    n = (ctypes.c_int64 * 3)(*shape)
    return lib.afft_c2r_noalloc(n, prec, X.data_ptr(), out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)


def rel(a, b):
    a, b = a.double(), b.double()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("prec", [afft.F32, afft.F64])
def test_matches_plan_backward_on_consecutive_calls(lib, prec):
    rdt = np.float32 if prec == afft.F32 else np.float64
    # two calls in a row on the same shape, then a different shape reusing the same array
    for shape, seed in (((64, 48, 96), 1), ((64, 48, 96), 2), ((30, 40, 128), 3)):
        with afft.Plan(shape, "r2c", prec) as p:
            x = torch.from_numpy(synth.uniform_real(shape, seed).astype(rdt)).cuda()
            X = p.forward(x)
            ref = p.backward(X)
            X_before = X.clone()
            out = torch.full(shape, float("nan"), dtype=ref.dtype, device="cuda")
            assert noalloc(lib, shape, prec, X, out) == 0
            torch.cuda.synchronize()
            assert torch.equal(X, X_before), "input modified"
            err = rel(out, ref)
            ref_orc = oracle.c2r(X.cpu().numpy(), shape[2])
            err_orc = oracle.rel_l2(out.cpu().numpy(), ref_orc)
            print("\n[no-alloc] %s %s rel_l2 vs plan c2r = %.3e, vs oracle c2r = %.3e"
                  % (shape, "f32" if prec == 0 else "f64", err, err_orc))
            assert err <= TOL[prec]
            assert err_orc <= TOL[prec]
            assert rel(out, x) <= TOL[prec]


@pytest.mark.parametrize("prec", [afft.F32, afft.F64])
def test_calls_allocate_no_device_memory(lib, prec):
    """After a first call (which looks up the array's address and loads the kernels), further
    calls leave the device's free memory exactly where it was."""
    shape = (64, 48, 96)
    cdt = np.complex64 if prec == afft.F32 else np.complex128
    X = torch.from_numpy(oracle.r2c(synth.uniform_real(shape, 5)).astype(cdt)).cuda()
    out = torch.empty(shape, dtype=torch.float32 if prec == afft.F32 else torch.float64, device="cuda")
    assert noalloc(lib, shape, prec, X, out) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        assert noalloc(lib, shape, prec, X, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_rejects_what_does_not_fit(lib):
    # 256^3 float32: the 256*256*129 complex intermediate (64.5 MiB) exceeds the scratch array;
    # rejected before any launch
    big_in = torch.empty((256, 256, 129), dtype=torch.complex64, device="cuda")
    big_out = torch.empty((256, 256, 256), dtype=torch.float32, device="cuda")
    assert noalloc(lib, (256, 256, 256), afft.F32, big_in, big_out) == 10    # AFFT_ERR_SCRATCH
    del big_in, big_out
    X = torch.empty(16, dtype=torch.complex64, device="cuda")
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    assert afft.status_string(10) != "unknown status"
    assert noalloc(lib, (8, 8, 7), afft.F32, X, out) == 2           # odd size with factor 7
    assert noalloc(lib, (8, 8, 9), afft.F32, X, out) == 3           # odd n2
    # lines longer than 4096 points (n2/2 = 8192 here) would need the four-step split's buffer
    long_in = torch.empty(8193, dtype=torch.complex64, device="cuda")
    long_out = torch.empty(16384, dtype=torch.float32, device="cuda")
    assert noalloc(lib, (1, 1, 16384), afft.F32, long_in, long_out) == 9   # AFFT_ERR_UNSUPPORTED
    assert noalloc(lib, (8192, 1, 2), afft.F32, long_in, long_out) == 9
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.afft_c2r_noalloc(n, afft.F32, None, out.data_ptr(), None) == 1
    assert lib.afft_c2r_noalloc(n, afft.F32, X.data_ptr(), X.data_ptr(), None) == 7
