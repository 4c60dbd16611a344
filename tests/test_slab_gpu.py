"""GPU parity of the distributed-form building blocks against the FP64 CPU oracle:
axis-subset plans, the slab decomposition (Algorithm 3) at one process over NCCL,
and d-dimensional transforms (Algorithm 2), at the tolerances of the other
parity tests (relative L2: 1e-12 FP64, 2e-6 FP32)."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist

import oracle
from paper_1506_07933_gb300 import afft, ndim, slab, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}
CDT = {"f64": np.complex128, "f32": np.complex64}
RDT = {"f64": np.float64, "f32": np.float32}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    afft.load()


def report(name, err, tol):
    print("\n[parity] %-52s rel_l2 = %.3e (tol %.0e)" % (name, err, tol))
    assert err <= tol, (name, err, tol)


def oracle_axes(x, axes, sign, kind="c2c"):
    """The separable DFT along the selected axes (N2 first forward, N0 first backward), by the
    oracle's 1-D transforms; r2c keeps bins 0 .. n2/2 of the contiguous axis."""
    a = np.asarray(x, dtype=np.complex128)
    order = (2, 1, 0) if sign < 0 else (0, 1, 2)
    for ax in order:
        if (axes >> ax) & 1:
            a = oracle.dft_axis(a, ax, sign)
    if kind == "r2c":
        a = a[..., : x.shape[2] // 2 + 1]
    return np.ascontiguousarray(a)


@pytest.mark.parametrize("axes", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_c2c_axis_subsets(axes, prec):
    shape = (12, 10, 16)
    x = synth.uniform_complex(shape, 100 + axes).astype(CDT[prec])
    with afft.Plan(shape, "c2c", prec, axes=axes) as p:
        X = p.forward(torch.from_numpy(x).cuda())
        y = p.backward(X)
        torch.cuda.synchronize()
        report("c2c axes %d %s forward" % (axes, prec), oracle.rel_l2(X.cpu().numpy(), oracle_axes(x, axes, -1)),
               TOL[prec])
        report("c2c axes %d %s round trip" % (axes, prec), oracle.rel_l2(y.cpu().numpy(), x), TOL[prec])
        assert p.backward_scale == pytest.approx(1.0 / math.prod(n for a, n in enumerate(shape) if (axes >> a) & 1))


@pytest.mark.parametrize("axes", [4, 5, 6, 7])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_r2c_axis_subsets(axes, prec):
    shape = (6, 20, 24)
    x = synth.uniform_real(shape, 200 + axes).astype(RDT[prec])
    with afft.Plan(shape, "r2c", prec, axes=axes) as p:
        X = p.forward(torch.from_numpy(x).cuda())
        y = p.backward(X)
        torch.cuda.synchronize()
        report("r2c axes %d %s forward" % (axes, prec), oracle.rel_l2(X.cpu().numpy(), oracle_axes(x, axes, -1, "r2c")),
               TOL[prec])
        report("r2c axes %d %s round trip" % (axes, prec), oracle.rel_l2(y.cpu().numpy(), x), TOL[prec])


def test_untransformed_axes_may_have_any_length_and_scale_is_settable():
    """Axis 2 of length 257 (prime) left alone; the axis-0 transform of a [n0][n1][257] array, with
    the backward factor set to 1 (unnormalised) and to 1/n0."""
    shape = (64, 6, 257)
    x = synth.uniform_complex(shape, 9).astype(np.complex64)
    with afft.Plan(shape, "c2c", "f32", axes=1) as p:
        xt = torch.from_numpy(x).cuda()
        X = p.forward(xt)
        report("c2c axes 1 with n2 = 257", oracle.rel_l2(X.cpu().numpy(), oracle_axes(x, 1, -1)), TOL["f32"])
        p.set_backward_scale(1.0)
        y = p.backward(X)
        torch.cuda.synchronize()
        report("axes 1 unnormalised backward", oracle.rel_l2(y.cpu().numpy(), 64 * x), TOL["f32"])
        p.set_backward_scale(1.0 / 64)
        y = p.backward(X)
        torch.cuda.synchronize()
        report("axes 1 backward x 1/n0", oracle.rel_l2(y.cpu().numpy(), x), TOL["f32"])
        assert p.launches(True) == 2      # the strided stage and the scaling pass
        assert p.describe()["stage_kernels_forward"][0] == "none"


def test_copy_2d_moves_pitched_blocks():
    src = torch.arange(6 * 10, dtype=torch.float32, device="cuda").view(6, 10)
    dst = torch.full((6, 4), -1.0, device="cuda")
    afft.afft_copy_2d(dst.data_ptr(), 16, src.data_ptr() + 3 * 4, 40, 16, 6, afft._stream_handle(None))
    torch.cuda.synchronize()
    assert torch.equal(dst, src[:, 3:7])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("shape,kind,prec", [((32, 24, 40), "r2c", "f64"), ((16, 48, 64), "c2c", "f32"),
                                             ((64, 64, 64), "r2c", "f32")])
def test_slab_fft_one_process_over_nccl(shape, kind, prec):
    """The slab decomposition's whole path (axes {1, 2} plan, pitched pack, NCCL all-to-all,
    axes {0} plan, and back) with one process: the result is the full 3-D transform."""
    own = not dist.is_initialized()
    if own:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
        dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        x = (synth.uniform_real(shape, 5) if kind == "r2c" else synth.uniform_complex(shape, 5))
        x = x.astype(RDT[prec] if kind == "r2c" else CDT[prec])
        f = slab.SlabFFT(shape, kind, prec)
        Z = f.forward(torch.from_numpy(x).cuda())
        back = f.backward(Z)
        torch.cuda.synchronize()
        ref = oracle.r2c(x) if kind == "r2c" else oracle.c2c(x, -1)
        report("slab P=1 %s %s %s forward" % (shape, kind, prec), oracle.rel_l2(Z.cpu().numpy(), ref), TOL[prec])
        report("slab P=1 %s %s %s round trip" % (shape, kind, prec), oracle.rel_l2(back.cpu().numpy(), x), TOL[prec])
        f.close()
    finally:
        if own:
            dist.destroy_process_group()


@pytest.mark.parametrize("shape,kind,prec", [((6, 8, 10, 12), "c2c", "f64"), ((4, 6, 10, 16), "r2c", "f32"),
                                             ((3, 5, 8, 6, 10), "c2c", "f32"), ((16, 12, 10, 8), "r2c", "f64")])
def test_fftn_against_oracle(shape, kind, prec):
    """d-D transforms (Algorithm 2): every axis by the oracle's 1-D DFT."""
    rng = np.random.default_rng(len(shape) * 100 + shape[0])
    if kind == "r2c":
        x = rng.uniform(-1, 1, shape).astype(RDT[prec])
    else:
        x = (rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)).astype(CDT[prec])
    ref = np.asarray(x, dtype=np.complex128)
    for ax in range(len(shape) - 1, -1, -1):
        ref = oracle.dft_axis(ref, ax, -1)
    if kind == "r2c":
        ref = ref[..., : shape[-1] // 2 + 1]
    f = ndim.FFTN(shape, kind, prec)
    X = f.forward(torch.from_numpy(x).cuda())
    y = f.backward(X)
    torch.cuda.synchronize()
    report("fftn %s %s %s forward" % (shape, kind, prec), oracle.rel_l2(X.cpu().numpy(), ref), TOL[prec])
    report("fftn %s %s %s round trip" % (shape, kind, prec), oracle.rel_l2(y.cpu().numpy(), x), TOL[prec])
    f.close()


def test_fftn_4d_paper_size_plane_wave():
    """The 4-D case of Section 3 (512 x 256 x 128 x 64, c2c FP32, 8.6 GB): a plane wave must come
    out as a single delta of height N, and the round trip must return the input."""
    shape = (512, 256, 128, 64)
    N = float(math.prod(shape))
    k = (5, 250, 3, 40)
    e = [torch.exp(2j * np.pi * torch.remainder(torch.arange(n, device="cuda", dtype=torch.float64) * kk, n) / n)
         for n, kk in zip(shape, k)]
    a = (e[0][:, None] * e[1][None, :]).to(torch.complex64)          # [512, 256]
    b = (e[2][:, None] * e[3][None, :]).to(torch.complex64)          # [128, 64]
    x = (a[:, :, None, None] * b[None, None, :, :]).contiguous()
    assert tuple(x.shape) == shape
    f = ndim.FFTN(shape, "c2c", "f32")
    X = f.forward(x)
    torch.cuda.synchronize()
    peak = complex(X[k].item())
    X[k] = 0
    report("fftn 512x256x128x64 f32 plane-wave peak", abs(peak - N) / N, TOL["f32"])
    report("fftn 512x256x128x64 f32 plane-wave leakage", float(torch.linalg.vector_norm(X.to(torch.complex128))) / N,
           TOL["f32"])
    X[k] = peak
    y = f.backward(X)
    torch.cuda.synchronize()
    x64 = x.to(torch.complex128)
    report("fftn 512x256x128x64 f32 round trip",
           float(torch.linalg.vector_norm(y.to(torch.complex128) - x64) / torch.linalg.vector_norm(x64)), TOL["f32"])
    f.close()
