"""The split-precision path (AFFT_F32_SPLIT): complex64 storage, radix-16 passes as FP16
tensor-core MMAs on hi + lo split operands with FP32 accumulation, other radices in FP32.
Against the FP64 oracle with the path's tolerance, relative L2 <= 2e-5; each error printed."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_07933_gb300 import afft, synth

pytestmark = pytest.mark.gpu

TOL = 2e-5
P = "f32_split"


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    afft.load()
    yield


def report(name, err, tol=TOL):
    print("\n[split] %-48s rel_l2 = %.3e (tol %.0e)" % (name, err, tol))
    assert err <= tol, (name, err, tol)


def run_c2c(x, direction=-1, prec=P):
    with afft.Plan(x.shape, "c2c", prec) as p:
        t = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        y = p.forward(t) if direction < 0 else p.backward(t)
        torch.cuda.synchronize()
        return y.cpu().numpy()


def test_plan_reports_split_precision():
    with afft.Plan((64, 64, 64), "c2c", P) as p:
        d = p.describe()
    assert d["precision"] == "f32split"
    assert d["radix"] == ["16x4"] * 3      # the split sequences lead with radix-16 passes


# lengths whose radix plans have radix-16 passes (and a few without, which stay on CUDA cores)
LENGTHS = [16, 32, 48, 64, 80, 128, 256, 512, 1024, 2048, 4096, 8, 40, 96]


@pytest.mark.parametrize("n", LENGTHS)
def test_c2c_each_length_on_each_axis(n):
    other = (6, 10) if n <= 512 else (2, 3)
    for shape in ((n,) + other, (other[0], n, other[1]), other + (n,)):
        x = synth.uniform_complex(shape, 7 * n).astype(np.complex64)
        ref = oracle.c2c(x, -1, "fft")
        report("c2c %s fwd" % (shape,), oracle.rel_l2(run_c2c(x), ref))
        Xr = ref.astype(np.complex64)
        report("c2c %s bwd" % (shape,), oracle.rel_l2(run_c2c(Xr, +1), oracle.c2c(Xr, +1, "fft")))


@pytest.mark.parametrize("shape", [(8192, 2, 3), (2, 3, 8192)])
def test_four_step_long_lines(shape):
    x = synth.uniform_complex(shape, 81).astype(np.complex64)
    report("c2c four-step %s" % (shape,), oracle.rel_l2(run_c2c(x), oracle.c2c(x, -1, "fft")))


@pytest.mark.parametrize("m", [16, 64, 128, 256, 512, 1024])
def test_r2c_c2r_each_half_length(m):
    shape = (6, 5, 2 * m) if m <= 512 else (2, 3, 2 * m)
    x = synth.uniform_real(shape, m).astype(np.float32)
    ref = oracle.r2c(x)
    with afft.Plan(shape, "r2c", P) as p:
        X = p.forward(torch.from_numpy(x).cuda())
        Xr = ref.astype(np.complex64)
        y = p.backward(torch.from_numpy(Xr).cuda())
        torch.cuda.synchronize()
    report("r2c %s" % (shape,), oracle.rel_l2(X.cpu().numpy(), ref))
    report("c2r %s" % (shape,), oracle.rel_l2(y.cpu().numpy(), oracle.c2r(Xr, shape[2])))


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1e3, 1e30])
def test_magnitudes_across_the_float_range(scale):
    """Every butterfly is scaled by a power of two into FP16 range before the split."""
    shape = (32, 16, 64)
    x = (synth.uniform_complex(shape, 5) * scale).astype(np.complex64)
    report("c2c scale %.0e" % scale, oracle.rel_l2(run_c2c(x), oracle.c2c(x, -1, "fft")))


def test_zeros_and_an_impulse():
    shape = (16, 32, 64)
    x = np.zeros(shape, np.complex64)
    assert not np.any(run_c2c(x))
    x[3, 5, 7] = 2.5 - 1.0j
    report("impulse", oracle.rel_l2(run_c2c(x), oracle.c2c(x, -1, "naive")))


def test_subcase_256cubed_splitmix_input():
    """The 1024^3 workload's error on its 256^3 sub-case (same generator), split and FP32 side by
    side (the FP32 CUDA-core path must stay within 2e-6)."""
    shape = (256, 256, 256)
    t = torch.empty(shape, dtype=torch.complex64, device="cuda")
    afft.fill_uniform(t, 2560)
    ref = oracle.c2c(synth.splitmix64_uniform(256 ** 3, 2560).reshape(shape), -1, "fft")
    errs = {}
    for prec in ("f32", P):
        with afft.Plan(shape, "c2c", prec) as p:
            X = p.forward(t)
            torch.cuda.synchronize()
        errs[prec] = oracle.rel_l2(X.cpu().numpy(), ref)
    report("c2c 256^3 split (1024^3 sub-case)", errs[P])
    report("c2c 256^3 f32 (same input)", errs["f32"], 2e-6)


def test_c2c_1024cubed_full_size_against_the_fp32_path():
    """1024^3 complex64 (8 GB): round trip and Parseval on the splitmix input, and the split
    spectrum against the FP32 path's spectrum (both within their tolerances of the exact one)."""
    n = 1024
    shape = (n, n, n)
    N = float(n) ** 3
    x = torch.empty(shape, dtype=torch.complex64, device="cuda")
    afft.fill_uniform(x, 10240)
    with afft.Plan(shape, "c2c", P) as p:
        X = p.forward(x)
        torch.cuda.synchronize()
        px = float(torch.sum(torch.abs(x.to(torch.complex128)) ** 2))
        pX = float(torch.sum(torch.abs(X.to(torch.complex128)) ** 2))
        report("c2c 1024^3 split Parseval", abs(pX / (N * px) - 1))
        y = p.backward(X)
        torch.cuda.synchronize()
        rt = float(torch.linalg.vector_norm((y - x).to(torch.complex128)) / torch.linalg.vector_norm(x.to(torch.complex128)))
        report("c2c 1024^3 split round trip", rt)
        del y
    with afft.Plan(shape, "c2c", "f32") as p:
        Y = p.forward(x)
        torch.cuda.synchronize()
    d = float(torch.linalg.vector_norm((X - Y).to(torch.complex128)) / torch.linalg.vector_norm(Y.to(torch.complex128)))
    report("c2c 1024^3 split vs FP32 path", d)


def test_batched_split_plan_and_poisson():
    shape, B = (32, 32, 32), 3
    fs = np.stack([synth.manufactured_poisson(shape, 40 + b, n_modes=6)[0] for b in range(B)]).astype(np.float32)
    us = np.stack([synth.manufactured_poisson(shape, 40 + b, n_modes=6)[1] for b in range(B)])
    with afft.Plan(shape, "r2c", P, batch=B) as p:
        got = p.poisson(torch.from_numpy(fs).cuda())
        torch.cuda.synchronize()
    for b in range(B):
        report("poisson batched split [%d]" % b, oracle.rel_l2(got[b].cpu().numpy(), us[b]))
