"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle.

Tolerances are relative L2 errors ||y - y_oracle|| / ||y_oracle||: 1e-12 for
FP64 and 2e-6 for FP32.  FP32 results are compared with the oracle run in
FP64 on the same FP32-rounded input, so the tolerance measures the kernels'
rounding only.  Each error is printed (pytest -s shows them).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_07933_gb300 import afft, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}
CDT = {"f64": np.complex128, "f32": np.complex64}
RDT = {"f64": np.float64, "f32": np.float32}

# every line length with specialised kernels, and some that take the generic ones
SPEC_LENGTHS = [1, 2, 4, 8, 16, 24, 32, 48, 60, 64, 80, 96, 120, 128, 160, 192, 256, 384, 512, 1024]
GENERIC_LENGTHS = [3, 5, 6, 9, 10, 12, 18, 25, 27, 36, 45, 50, 72, 81, 100, 125, 150, 243, 250, 320,
                   640, 729, 768, 2048, 4096]


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    afft.load()
    yield


def report(name, err, tol):
    print("\n[parity] %-48s rel_l2 = %.3e (tol %.0e)" % (name, err, tol))
    assert err <= tol, (name, err, tol)


def gpu_c2c(x, prec, direction=-1):
    with afft.Plan(x.shape, "c2c", prec) as p:
        t = torch.from_numpy(np.ascontiguousarray(x.astype(CDT[prec]))).cuda()
        y = p.forward(t) if direction < 0 else p.backward(t)
        torch.cuda.synchronize()
        return y.cpu().numpy()


def gpu_r2c(x, prec):
    with afft.Plan(x.shape, "r2c", prec) as p:
        y = p.forward(torch.from_numpy(np.ascontiguousarray(x.astype(RDT[prec]))).cuda())
        torch.cuda.synchronize()
        return y.cpu().numpy()


def gpu_c2r(X, shape, prec):
    with afft.Plan(shape, "r2c", prec) as p:
        t = torch.from_numpy(np.ascontiguousarray(X.astype(CDT[prec]))).cuda()
        before = t.clone()
        y = p.backward(t)
        torch.cuda.synchronize()
        assert torch.equal(t, before), "c2r modified its input"
        return y.cpu().numpy()


# --- the small c2c configuration: 32^3 complex128 against the naive DFT ---------

def test_c2c_32cubed_complex128_against_naive_dft():
    x = synth.uniform_complex((32, 32, 32), 1506)
    ref = oracle.c2c(x, -1, "naive")
    X = gpu_c2c(x, "f64")
    report("c2c 32^3 f64 forward vs naive", oracle.rel_l2(X, ref), 1e-12)
    back = gpu_c2c(ref, "f64", +1)
    report("c2c 32^3 f64 backward vs naive", oracle.rel_l2(back, oracle.c2c(ref, +1, "naive")), 1e-12)
    report("c2c 32^3 f64 round trip", oracle.rel_l2(gpu_c2c(X, "f64", +1), x), 1e-12)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_c2c_32cubed_both_precisions(prec):
    x = synth.uniform_complex((32, 32, 32), 1506).astype(CDT[prec])
    report("c2c 32^3 %s forward" % prec, oracle.rel_l2(gpu_c2c(x, prec), oracle.c2c(x, -1, "naive")), TOL[prec])


# --- every line length, on every axis --------------------------------------------

@pytest.mark.parametrize("n", SPEC_LENGTHS + GENERIC_LENGTHS)
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_c2c_each_length_on_each_axis(n, prec):
    other = (6, 10) if n <= 512 else (2, 3)
    for shape in ((n,) + other, (other[0], n, other[1]), other + (n,)):
        x = synth.uniform_complex(shape, n).astype(CDT[prec])
        ref = oracle.c2c(x, -1, "fft")
        report("c2c %s %s fwd" % (shape, prec), oracle.rel_l2(gpu_c2c(x, prec), ref), TOL[prec])
        report("c2c %s %s bwd" % (shape, prec),
               oracle.rel_l2(gpu_c2c(ref.astype(CDT[prec]), prec, +1),
                             oracle.c2c(ref.astype(CDT[prec]), +1, "fft")), TOL[prec])


@pytest.mark.parametrize("m", SPEC_LENGTHS + [3, 5, 12, 36, 100, 2048])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_r2c_c2r_each_half_length(m, prec):
    shape = (6, 5, 2 * m) if m <= 512 else (2, 3, 2 * m)
    x = synth.uniform_real(shape, m).astype(RDT[prec])
    ref = oracle.r2c(x)
    X = gpu_r2c(x, prec)
    report("r2c %s %s" % (shape, prec), oracle.rel_l2(X, ref), TOL[prec])
    Xr = ref.astype(CDT[prec])
    report("c2r %s %s" % (shape, prec), oracle.rel_l2(gpu_c2r(Xr, shape, prec), oracle.c2r(Xr, shape[2])),
           TOL[prec])


# --- edge cases ----------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 8), (1, 8, 1), (8, 1, 1), (5, 1, 3), (1, 1, 2),
                                   (2, 2, 2), (3, 1, 2), (16, 3, 1)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_degenerate_shapes(shape, prec):
    x = synth.uniform_complex(shape, 7).astype(CDT[prec])
    report("c2c %s %s" % (shape, prec), oracle.rel_l2(gpu_c2c(x, prec), oracle.c2c(x, -1, "fft")), TOL[prec])
    report("c2c bwd %s %s" % (shape, prec),
           oracle.rel_l2(gpu_c2c(x, prec, +1), oracle.c2c(x, +1, "fft")), TOL[prec])
    if shape[2] % 2 == 0:
        r = x.real.copy()
        report("r2c %s %s" % (shape, prec), oracle.rel_l2(gpu_r2c(r, prec), oracle.r2c(r)), TOL[prec])
        H = oracle.r2c(r).astype(CDT[prec])
        report("c2r %s %s" % (shape, prec), oracle.rel_l2(gpu_c2r(H, shape, prec), oracle.c2r(H, shape[2])),
               TOL[prec])


@pytest.mark.parametrize("shape", [(6, 10, 36), (5, 9, 540), (3, 40, 160), (32, 3, 96)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ragged_tiles(shape, prec):
    """Column counts that do not fill the last tile (n2/2+1 odd, few lines per CTA)."""
    x = synth.uniform_real(shape, 21).astype(RDT[prec])
    ref = oracle.r2c(x)
    report("r2c ragged %s %s" % (shape, prec), oracle.rel_l2(gpu_r2c(x, prec), ref), TOL[prec])
    H = ref.astype(CDT[prec])
    report("c2r ragged %s %s" % (shape, prec), oracle.rel_l2(gpu_c2r(H, shape, prec), oracle.c2r(H, shape[2])),
           TOL[prec])


@pytest.mark.parametrize("shape", [(16, 24, 40), (64, 48, 96), (32, 3, 96), (120, 8, 12), (8, 1, 24),
                                   (8, 512, 512), (4, 256, 64), (6, 48, 36), (2, 32, 8), (3, 16, 120),
                                   (5, 160, 72), (2, 384, 40), (5, 32, 108), (40, 64, 64)])
def test_r2c_odd_width_rows(shape):
    """FP32 r2c plans whose half-spectrum width n2/2+1 is odd: complex64 rows of odd width,
    read as row pairs through TMA in the N1 stage where n1 allows (a multiple of 16, at most
    512), by per-element copies otherwise; results must not change.  The last tile of each row
    holds W mod 16 columns: one (W = 49, 257, 33), three (19), five (37, 21), seven (55) or
    thirteen (61)."""
    x = synth.uniform_real(shape, 31).astype(np.float32)
    ref = oracle.r2c(x)
    report("r2c odd rows %s f32" % (shape,), oracle.rel_l2(gpu_r2c(x, "f32"), ref), TOL["f32"])
    H = ref.astype(np.complex64)
    report("c2r odd rows %s f32" % (shape,), oracle.rel_l2(gpu_c2r(H, shape, "f32"), oracle.c2r(H, shape[2])),
           TOL["f32"])


@pytest.mark.parametrize("shape", [(8, 512, 512), (4, 256, 64), (6, 48, 36), (5, 160, 72), (5, 32, 108),
                                   (40, 64, 64)])
def test_r2c_odd_width_rows_early_release(shape):
    """The row-pair N1 tiles with their load buffer released after the first pass (a tuning
    choice): the same results as the oracle, both directions."""
    x = synth.uniform_real(shape, 33).astype(np.float32)
    ref = oracle.r2c(x)
    H = ref.astype(np.complex64)
    with afft.Plan(shape, "r2c", "f32") as p:
        cfg = p.tuning
        cfg[5] = 1
        p.set_tuning(cfg)
        assert p.describe()["rp_early"][1] == 1
        X = p.forward(torch.from_numpy(x).cuda())
        y = p.backward(torch.from_numpy(H).cuda())
        torch.cuda.synchronize()
    report("r2c odd rows early release %s" % (shape,), oracle.rel_l2(X.cpu().numpy(), ref), TOL["f32"])
    report("c2r odd rows early release %s" % (shape,), oracle.rel_l2(y.cpu().numpy(), oracle.c2r(H, shape[2])),
           TOL["f32"])


@pytest.mark.parametrize("shape,kind", [((4, 64, 32), "r2c"), ((6, 48, 64), "r2c"), ((6, 96, 160), "r2c"),
                                        ((3, 128, 256), "r2c"), ((4, 512, 512), "r2c"), ((32, 3, 20), "r2c"),
                                        ((4, 32, 81), "c2c"), ((3, 64, 225), "c2c")])
@pytest.mark.parametrize("early", [0, 1])
def test_row_pair_tiles_with_a_one_column_tail(shape, kind, early):
    """Rows of W = 16k + 1 complex64 columns (half spectra of 17, 33, 81, 129, 257 bins; c2c rows
    of 81 and 225; an N0 stage over planes of 3 x 11 bins) run k full row-pair tiles and a last
    tile of one column, whose boxes reach past the row pair's end: both directions against the
    oracle, with the load buffer released early or not."""
    if kind == "c2c":
        x = synth.uniform_complex(shape, 47).astype(np.complex64)
        ref = oracle.c2c(x)
    else:
        x = synth.uniform_real(shape, 47).astype(np.float32)
        ref = oracle.r2c(x)
    H = ref.astype(np.complex64)
    with afft.Plan(shape, kind, "f32") as p:
        cfg = p.tuning
        cfg[4] = early if p.describe()["stage_kernels_forward"][2] == "k_strided_pipe_rp" else cfg[4]
        cfg[5] = early if p.describe()["stage_kernels_forward"][1] == "k_strided_pipe_rp" else cfg[5]
        p.set_tuning(cfg)
        assert "k_strided_pipe_rp" in p.describe()["stage_kernels_forward"]
        X = p.forward(torch.from_numpy(x).cuda())
        y = p.backward(torch.from_numpy(H).cuda())
        torch.cuda.synchronize()
    back = oracle.c2c(H, +1) if kind == "c2c" else oracle.c2r(H, shape[2])
    report("rp tail %s %s early %d" % (shape, kind, early), oracle.rel_l2(X.cpu().numpy(), ref), TOL["f32"])
    report("rp tail backward %s %s early %d" % (shape, kind, early), oracle.rel_l2(y.cpu().numpy(), back), TOL["f32"])


@pytest.mark.parametrize("shape", [(3, 2, 8192), (8, 10, 160), (4, 6, 500)])
def test_c2r_staged_and_direct_tiles(shape):
    """The specialised complex64 c2r kernels copy a CTA's run of half-spectrum lines into shared
    memory when the run starts 16-byte aligned and read global memory otherwise.  One-line CTAs
    of n2/2 = 4096 (4097 bins) alternate between the two; 81 bins (n2 = 160) take 50 of the 51
    lines a CTA would hold, so every run is aligned; n2/2 = 250 runs the generic kernel."""
    x = synth.uniform_real(shape, 41).astype(np.float32)
    H = oracle.r2c(x).astype(np.complex64)
    report("c2r staging %s f32" % (shape,), oracle.rel_l2(gpu_c2r(H, shape, "f32"), oracle.c2r(H, shape[2])),
           TOL["f32"])


def test_c2r_drops_imaginary_parts_of_self_conjugate_bins():
    shape = (4, 6, 16)
    H = oracle.r2c(synth.uniform_real(shape, 3))
    G = H.copy()
    G[:, :, 0] += 0.5j
    G[:, :, 8] -= 0.25j
    report("c2r non-Hermitian bins", oracle.rel_l2(gpu_c2r(G, shape, "f64"), oracle.c2r(G, 16)), 1e-12)


# --- the r2c/c2r configuration: 256^3 and 512^3 random-mode fields -------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_r2c_c2r_256cubed_random_modes(prec):
    shape = (256, 256, 256)
    f = synth.random_mode_field(shape, 2561, n_modes=64, noise=1e-3)
    x = f.astype(RDT[prec])
    ref = oracle.r2c(x)
    with afft.Plan(shape, "r2c", prec) as p:
        X = p.forward(torch.from_numpy(x).cuda())
        y = p.backward(X)
        torch.cuda.synchronize()
        Xh, yh = X.cpu().numpy(), y.cpu().numpy()
    report("r2c 256^3 %s forward" % prec, oracle.rel_l2(Xh, ref), TOL[prec])
    Hr = ref.astype(CDT[prec])
    with afft.Plan(shape, "r2c", prec) as p:
        yb = p.backward(torch.from_numpy(Hr).cuda())
        torch.cuda.synchronize()
    report("c2r 256^3 %s backward" % prec, oracle.rel_l2(yb.cpu().numpy(), oracle.c2r(Hr, 256)), TOL[prec])
    report("r2c+c2r 256^3 %s round trip" % prec, oracle.rel_l2(yh, x), TOL[prec])


def closed_form_half_spectrum(n, modes):
    ks, amp, phase = modes
    N = float(n) ** 3
    H = {}
    for k, a, ph in zip(ks, amp, phase):
        for sgn in (1, -1):
            kk = sgn * k
            if kk[2] >= 0 and 2 * kk[2] <= n:
                key = (int(kk[0] % n), int(kk[1] % n), int(kk[2]))
                H[key] = H.get(key, 0) + N / 2 * a * np.exp(sgn * 1j * ph)
    return H


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_r2c_512cubed_full_size(prec):
    """512^3 in the benchmark's launch configuration.  Noise-free field: the whole
    spectrum is known in closed form.  Noisy field: sampled bins from the DFT
    definition, plus the round trip."""
    n = 512
    shape = (n, n, n)
    f, modes = synth.random_mode_field(shape, 5121, n_modes=64, noise=0.0, return_modes=True)
    H = closed_form_half_spectrum(n, modes)
    x = torch.from_numpy(f.astype(RDT[prec])).cuda()
    with afft.Plan(shape, "r2c", prec) as p:
        X = p.forward(x)
        torch.cuda.synchronize()
        keys = list(H.keys())
        idx = torch.tensor(keys, device="cuda").T
        vals = torch.tensor([H[k] for k in keys], dtype=torch.complex128, device="cuda")
        got = X[idx[0], idx[1], idx[2]].to(torch.complex128)
        Xe = X.to(torch.complex128, copy=True)   # never an alias of X (X is complex128 for f64)
        Xe[idx[0], idx[1], idx[2]] -= vals
        err = float(torch.linalg.vector_norm(Xe) / torch.linalg.vector_norm(vals))
        del Xe, got
        # the noise-free input is rounded to FP32 for the f32 case: measure against the closed
        # form of the rounded field only through the bound it must still meet
        report("r2c 512^3 %s vs closed form" % prec, err, TOL[prec])
        y = p.backward(X)
        torch.cuda.synchronize()
        rt = float(torch.linalg.vector_norm((y - x).to(torch.float64)) / torch.linalg.vector_norm(x.to(torch.float64)))
        report("r2c+c2r 512^3 %s round trip" % prec, rt, TOL[prec])
        del X, y
    g = synth.random_mode_field(shape, 5121, n_modes=64, noise=1e-3).astype(RDT[prec])
    rng = np.random.default_rng(512)
    ks = np.stack([rng.integers(0, n, 6), rng.integers(0, n, 6), rng.integers(0, n // 2 + 1, 6)], 1)
    ks = np.concatenate([ks, np.array(list(H.keys())[:6])])
    ref = oracle.dft_bins(g, ks)
    with afft.Plan(shape, "r2c", prec) as p:
        G = p.forward(torch.from_numpy(g).cuda())
        torch.cuda.synchronize()
        got = G[ks[:, 0], ks[:, 1], ks[:, 2]].cpu().numpy()
    report("r2c 512^3 %s sampled bins (%d)" % (prec, len(ks)), oracle.rel_l2(got, ref), TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c2r_512cubed_full_size(prec):
    """The c2r backward of the 512^3 workload over the whole array, in the benchmark's launch
    configuration: (1) the closed-form half spectrum of the noise-free field must come back as
    the field itself (its values on the grid, evaluated without any transform); (2) on the
    noisy field, the c2r of the oracle's half spectrum against the oracle's own c2r."""
    n = 512
    shape = (n, n, n)
    f, modes = synth.random_mode_field(shape, 5121, n_modes=64, noise=0.0, return_modes=True)
    H = closed_form_half_spectrum(n, modes)
    keys = list(H.keys())
    Hd = torch.zeros((n, n, n // 2 + 1), dtype=torch.complex128, device="cuda")
    idx = torch.tensor(keys, device="cuda").T
    Hd[idx[0], idx[1], idx[2]] = torch.tensor([H[k] for k in keys], dtype=torch.complex128, device="cuda")
    Hd = Hd.to(torch.complex64 if prec == "f32" else torch.complex128)
    fd = torch.from_numpy(f).cuda()
    with afft.Plan(shape, "r2c", prec) as p:
        y = p.backward(Hd)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(y.to(torch.float64) - fd) / torch.linalg.vector_norm(fd))
        report("c2r 512^3 %s closed-form spectrum -> field" % prec, err, TOL[prec])
        del y, Hd, fd
        g = synth.random_mode_field(shape, 5121, n_modes=64, noise=1e-3).astype(RDT[prec])
        G = oracle.r2c(g).astype(CDT[prec])
        ref = oracle.c2r(G, n)
        yb = p.backward(torch.from_numpy(G).cuda())
        torch.cuda.synchronize()
        report("c2r 512^3 %s vs oracle c2r (noisy field)" % prec, oracle.rel_l2(yb.cpu().numpy(), ref), TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c2c_512cubed_full_size(prec):
    """512^3 c2c over the whole array.  (1) A sum of 64 complex plane waves c_m exp(+i k_m.x):
    the forward spectrum is exactly N c_m at k_m and zero elsewhere.  (2) The splitmix64 input
    of the c2c workload, forward against the oracle's full 3-D transform, and the backward
    transform of the oracle's spectrum against the oracle's backward transform."""
    n = 512
    shape = (n, n, n)
    N = float(n) ** 3
    tdt = torch.complex64 if prec == "f32" else torch.complex128
    ks, amp, phase = synth.draw_modes(shape, 64, 5122)
    coef = amp * np.exp(1j * phase)
    spec = {}
    for k, c in zip(ks, coef):
        key = tuple(int(v) % n for v in k)
        spec[key] = spec.get(key, 0) + N * c
    keys = list(spec.keys())
    idx = torch.tensor(keys, device="cuda").T
    vals = torch.tensor([spec[k] for k in keys], dtype=torch.complex128, device="cuda")
    x = synth.plane_wave_sum_torch(shape, ks, coef).to(tdt)
    with afft.Plan(shape, "c2c", prec) as p:
        assert p.describe()["blocked"] == 0   # the benchmark's row-major stages
        X = p.forward(x)
        torch.cuda.synchronize()
        Xe = X.to(torch.complex128, copy=True)
        Xe[idx[0], idx[1], idx[2]] -= vals
        report("c2c 512^3 %s plane waves vs closed form" % prec,
               float(torch.linalg.vector_norm(Xe) / torch.linalg.vector_norm(vals)), TOL[prec])
        del Xe
        y = p.backward(X)
        torch.cuda.synchronize()
        x64 = x.to(torch.complex128)
        report("c2c 512^3 %s round trip" % prec,
               float(torch.linalg.vector_norm(y.to(torch.complex128) - x64) / torch.linalg.vector_norm(x64)),
               TOL[prec])
        del X, y, x, x64
        t = torch.empty(shape, dtype=tdt, device="cuda")
        afft.fill_uniform(t, 5120)
        xh = t.cpu().numpy()
        ref = oracle.c2c(xh, -1, "fft")
        Xg = p.forward(t)
        torch.cuda.synchronize()
        report("c2c 512^3 %s forward vs oracle (splitmix input)" % prec,
               oracle.rel_l2(Xg.cpu().numpy(), ref), TOL[prec])
        del Xg, t, xh
        R = ref.astype(CDT[prec])
        refb = oracle.c2c(R, +1, "fft")
        yb = p.backward(torch.from_numpy(R).cuda())
        torch.cuda.synchronize()
        report("c2c 512^3 %s backward vs oracle" % prec, oracle.rel_l2(yb.cpu().numpy(), refb), TOL[prec])


# --- the large c2c configuration: 1024^3 complex64 ------------------------------------

def test_c2c_1024_subcase_256cubed_splitmix_input():
    """The 1024^3 workload's error is stated on its 256^3 sub-case (same generator)."""
    shape = (256, 256, 256)
    x = synth.splitmix64_uniform(256 ** 3, 2560).reshape(shape)
    t = torch.empty(shape, dtype=torch.complex64, device="cuda")
    afft.fill_uniform(t, 2560)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), x), "device generator differs from its CPU definition"
    ref = oracle.c2c(x, -1, "fft")
    with afft.Plan(shape, "c2c", "f32") as p:
        X = p.forward(t)
        torch.cuda.synchronize()
    report("c2c 256^3 f32 (1024^3 sub-case)", oracle.rel_l2(X.cpu().numpy(), ref), TOL["f32"])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_c2c_1024cubed_full_size_properties(prec):
    """1024^3 c2c (8.6 GB complex64, 17.2 GB complex128) in the default launch configuration,
    the blocked layout: round trip and Parseval on the splitmix input, and a plane wave that must
    come out as a single delta of height N with no leakage anywhere else in the array."""
    n = 1024
    shape = (n, n, n)
    N = float(n) ** 3
    tdt = torch.complex64 if prec == "f32" else torch.complex128
    x = torch.empty(shape, dtype=tdt, device="cuda")
    afft.fill_uniform(x, 10240)
    with afft.Plan(shape, "c2c", prec) as p:
        assert p.describe()["blocked"] == 1
        X = p.forward(x)
        torch.cuda.synchronize()
        px = float(torch.sum(torch.abs(x.to(torch.complex128)) ** 2))
        pX = float(torch.sum(torch.abs(X.to(torch.complex128)) ** 2))
        report("c2c 1024^3 %s Parseval" % prec, abs(pX / (N * px) - 1), TOL[prec])
        y = p.backward(X)
        torch.cuda.synchronize()
        del X
        rt = float(torch.linalg.vector_norm((y - x).to(torch.complex128)) / torch.linalg.vector_norm(x.to(torch.complex128)))
        report("c2c 1024^3 %s round trip" % prec, rt, TOL[prec])
        del y
        k = (3, 1000, 17)
        j = torch.arange(n, device="cuda", dtype=torch.float64)
        e = [torch.exp(2j * np.pi * torch.remainder(j * kk, n) / n) for kk in k]
        x.copy_(e[0][:, None, None] * e[1][None, :, None] * e[2][None, None, :])
        X = p.forward(x)
        torch.cuda.synchronize()
        peak = complex(X[k].item())
        X[k] = 0
        rest = float(torch.linalg.vector_norm(X.to(torch.complex128)))
        report("c2c 1024^3 %s plane-wave peak" % prec, abs(peak - N) / N, TOL[prec])
        report("c2c 1024^3 %s plane-wave leakage" % prec, rest / N, TOL[prec])


def test_c2c_1024_point_rows_megabytes_apart_separable_input():
    """An N0 stage of 1024-point lines whose rows lie more than 1 MB apart, checked over the
    whole array: a separable input a[j0] b[j1] c[j2] has the separable spectrum A[k0] B[k1] C[k2]
    (the oracle's 1-D DFTs); both directions."""
    n0, n1, n2 = 1024, 384, 384
    a = synth.uniform_complex((n0, 1, 1), 901)
    b = synth.uniform_complex((1, n1, 1), 902)
    c = synth.uniform_complex((1, 1, n2), 903)
    A, B, C = (oracle.c2c(v, -1, "fft") for v in (a, b, c))
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    x = (dev(a) * dev(b) * dev(c)).to(torch.complex64)
    with afft.Plan((n0, n1, n2), "c2c", "f32") as p:
        X = p.forward(x)
        y = p.backward(X)
        torch.cuda.synchronize()
    ref = dev(A) * dev(B) * dev(C)
    err = float(torch.linalg.vector_norm(X.to(torch.complex128) - ref) / torch.linalg.vector_norm(ref))
    del ref
    report("c2c 1024x384x384 separable", err, TOL["f32"])
    x64 = x.to(torch.complex128)
    rt = float(torch.linalg.vector_norm(y.to(torch.complex128) - x64) / torch.linalg.vector_norm(x64))
    report("c2c 1024x384x384 round trip", rt, TOL["f32"])


# --- the boundary's behaviour on a GPU ------------------------------------------------

def test_in_place_and_overlap_are_rejected():
    with afft.Plan((8, 8, 8), "c2c", "f32") as p:
        t = torch.zeros((8, 8, 8), dtype=torch.complex64, device="cuda")
        ptr = t.data_ptr()
        with pytest.raises(afft.AfftError) as e:
            afft.afft_execute_forward(p._p, ptr, ptr, 0)
        assert e.value.status == 7
        with pytest.raises(afft.AfftError) as e:
            afft.afft_execute_forward(p._p, ptr, ptr + 8, 0)
        assert e.value.status == 7


def test_sizes_and_workspace():
    with afft.Plan((16, 8, 32), "r2c", "f64") as p:
        assert p.input_bytes == 16 * 8 * 32 * 8
        assert p.output_bytes == 16 * 8 * 17 * 16
        assert p.workspace_bytes == 16 * 8 * 17 * 16
        assert p.launches(False) == 3 and p.launches(True) == 3
    with afft.Plan((16, 8, 32), "c2c", "f32") as p:
        assert p.workspace_bytes == 0


def test_runs_on_a_side_stream():
    shape = (32, 48, 64)
    x = synth.uniform_complex(shape, 99).astype(np.complex64)
    s = torch.cuda.Stream()
    with afft.Plan(shape, "c2c", "f32") as p:
        t = torch.from_numpy(x).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            X = p.forward(t)
        s.synchronize()
        report("c2c on a side stream", oracle.rel_l2(X.cpu().numpy(), oracle.c2c(x)), TOL["f32"])


@pytest.mark.parametrize("kind,prec", [("c2c", "f32"), ("r2c", "f64")])
def test_host_buffer_entry_points(kind, prec):
    shape = (16, 20, 24)
    with afft.Plan(shape, kind, prec) as p:
        if kind == "c2c":
            x = torch.from_numpy(synth.uniform_complex(shape, 5).astype(CDT[prec]))
        else:
            x = torch.from_numpy(synth.uniform_real(shape, 5).astype(RDT[prec]))
        hin = x.pin_memory()
        hout = torch.empty(p.spectral_shape, dtype=p.spectral_dtype).pin_memory()
        din = torch.empty(p.spatial_shape, dtype=p.spatial_dtype, device="cuda")
        dout = torch.empty(p.spectral_shape, dtype=p.spectral_dtype, device="cuda")
        p.forward_host(hin, hout, din, dout)
        torch.cuda.synchronize()
        ref = p.forward(x.cuda()).cpu()
        torch.cuda.synchronize()
        assert torch.equal(hout, ref)
        back = torch.empty(p.spatial_shape, dtype=p.spatial_dtype).pin_memory()
        p.backward_host(hout, back, dout.clone(), din)
        torch.cuda.synchronize()
        report("host-buffer round trip %s %s" % (kind, prec), oracle.rel_l2(back.numpy(), x.numpy()), TOL[prec])


def test_fill_uniform_matches_cpu_definition():
    t = torch.empty(1000, dtype=torch.complex128, device="cuda")
    afft.fill_uniform(t, 77)
    torch.cuda.synchronize()
    ref = synth.splitmix64_uniform(1000, 77).astype(np.complex128)
    assert np.array_equal(t.cpu().numpy(), ref)


def test_bounded_wait_reports_a_timeout_and_the_device_stays_usable():
    """Failure detection without a fault: a wait that nothing can satisfy runs out after its
    limit, the plan's status reports AFFT_ERR_TIMEOUT once, and transforms keep working."""
    shape = (16, 24, 32)
    x = synth.uniform_complex(shape, 77).astype(np.complex64)
    with afft.Plan(shape, "c2c", "f32") as p:
        assert p.device_status() == 0
        p.wait_probe(2000)
        torch.cuda.synchronize()
        assert p.device_status() == 11
        assert p.device_status() == 0          # reported once, then cleared
        y = p.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert p.device_status() == 0
    report("c2c after a probed timeout", oracle.rel_l2(y.cpu().numpy(), oracle.c2c(x, -1, "fft")), TOL["f32"])
    with pytest.raises(afft.AfftError):
        with afft.Plan(shape, "c2c", "f32") as p:
            p.wait_probe(0)


def test_plans_are_independent():
    a = afft.Plan((8, 12, 16), "c2c", "f32")
    b = afft.Plan((8, 12, 16), "r2c", "f64")
    x = synth.uniform_complex((8, 12, 16), 1).astype(np.complex64)
    ya = a.forward(torch.from_numpy(x).cuda())
    b.close()
    ya2 = a.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert torch.equal(ya, ya2)
    a.close()


def test_stage_timing_records_every_execution():
    shape = (64, 96, 128)
    with afft.Plan(shape, "r2c", "f32") as p:
        x = torch.from_numpy(synth.uniform_real(shape, 4).astype(np.float32)).cuda()
        p.timing_begin(4)
        for _ in range(3):
            X = p.forward(x)
            p.backward(X)
        rows = p.timing_end()
        assert len(rows) == 4 and all(len(r) == 3 for r in rows)
        assert all(t > 0 for r in rows for t in r)
        y = p.backward(p.forward(x))   # recording is off again
        torch.cuda.synchronize()
        assert p.timing_end() == []
        report("round trip with timing on", float(torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x)),
               TOL["f32"])


@pytest.mark.parametrize("shape,kind,prec", [((64, 48, 96), "r2c", "f32"), ((40, 30, 64), "c2c", "f32"),
                                             ((24, 16, 32), "r2c", "f64"), ((36, 20, 24), "c2c", "f64")])
@pytest.mark.parametrize("planes", [1, 3, 7])
def test_l2_fused_slabs_match_unfused(shape, kind, prec, planes):
    """The N2/N1 stages run slab by slab on two streams; results equal the unfused schedule
    bit for bit and the oracle within tolerance, with a ragged last slab."""
    if kind == "c2c":
        x = synth.uniform_complex(shape, 41).astype(CDT[prec])
    else:
        x = synth.uniform_real(shape, 41).astype(RDT[prec])
    with afft.Plan(shape, kind, prec) as p:
        p.set_l2_chunk(0)
        assert p.l2_chunk == 0
        t = torch.from_numpy(x).cuda()
        ref_f = p.forward(t)
        ref_b = p.backward(ref_f)
        n_unfused = p.launches(False)
        plane = shape[1] * (p.spectral_shape[2] + (1 if (kind == "r2c" and prec == "f32" and
                                                          p.spectral_shape[2] % 2 == 1) else 0)) \
            * (8 if prec == "f32" else 16)
        p.set_l2_chunk(planes * plane)
        assert p.l2_chunk > 0
        assert p.launches(False) > n_unfused
        f = p.forward(t)
        b = p.backward(f)
        torch.cuda.synchronize()
        assert torch.equal(f, ref_f) and torch.equal(b, ref_b)
    ref = oracle.r2c(x) if kind == "r2c" else oracle.c2c(x)
    report("fused %s %s %s planes=%d" % (shape, kind, prec, planes), oracle.rel_l2(f.cpu().numpy(), ref), TOL[prec])


@pytest.mark.parametrize("shape,kind,prec", [((64, 48, 96), "r2c", "f32"), ((40, 30, 64), "c2c", "f32"),
                                             ((24, 16, 32), "r2c", "f64"), ((36, 20, 24), "c2c", "f64"),
                                             ((8, 512, 512), "r2c", "f32"), ((6, 10, 36), "r2c", "f32"),
                                             ((5, 243, 40), "c2c", "f32"), ((3, 2, 8192), "r2c", "f32")])
def test_alternating_stage_order_is_bit_exact(shape, kind, prec):
    """By default consecutive stages walk their tiles in alternating order, so each starts on the
    part of the array the previous stage wrote last (still in L2).  Only the order of independent
    tiles changes: both transforms must equal the first-to-last order bit for bit (pipelined,
    row-pair, plain strided, generic and r2c/c2r kernels, both precisions), and the oracle."""
    if kind == "c2c":
        x = synth.uniform_complex(shape, 43).astype(CDT[prec])
    else:
        x = synth.uniform_real(shape, 43).astype(RDT[prec])
    with afft.Plan(shape, kind, prec) as p:
        assert p.l2_order and p.describe()["l2_order"] == 1
        t = torch.from_numpy(x).cuda()
        f = p.forward(t)
        b = p.backward(f)
        u = p.poisson(t) if kind == "r2c" else None
        p.set_l2_order(False)
        assert not p.l2_order
        f0 = p.forward(t)
        b0 = p.backward(f0)
        u0 = p.poisson(t) if kind == "r2c" else None
        torch.cuda.synchronize()
        assert torch.equal(f, f0) and torch.equal(b, b0)
        assert u is None or torch.equal(u, u0)
    ref = oracle.r2c(x) if kind == "r2c" else oracle.c2c(x)
    report("alternating order %s %s %s" % (shape, kind, prec), oracle.rel_l2(f.cpu().numpy(), ref), TOL[prec])
    report("alternating order round trip %s %s %s" % (shape, kind, prec), oracle.rel_l2(b.cpu().numpy(), x),
           TOL[prec])


@pytest.mark.parametrize("shape", [(8192, 2, 3), (2, 8192, 3), (2, 3, 8192), (3, 2, 6000), (1, 2, 65536),
                                   (5000, 3, 4)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_four_step_long_lines_c2c(shape, prec):
    """Lines longer than 4096 points are split n = n_a n_b (four-step, with the twiddle and
    transposed store fused into the second half) on every axis."""
    x = synth.uniform_complex(shape, 51).astype(CDT[prec])
    ref = oracle.c2c(x, -1, "fft")
    report("four-step c2c %s %s fwd" % (shape, prec), oracle.rel_l2(gpu_c2c(x, prec), ref), TOL[prec])
    R = ref.astype(CDT[prec])
    report("four-step c2c %s %s bwd" % (shape, prec), oracle.rel_l2(gpu_c2c(R, prec, +1), oracle.c2c(R, +1, "fft")),
           TOL[prec])


@pytest.mark.parametrize("shape", [(8192, 4, 16), (4, 10000, 8), (6000, 2, 36)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_four_step_long_lines_r2c(shape, prec):
    x = synth.uniform_real(shape, 52).astype(RDT[prec])
    ref = oracle.r2c(x)
    report("four-step r2c %s %s" % (shape, prec), oracle.rel_l2(gpu_r2c(x, prec), ref), TOL[prec])
    H = ref.astype(CDT[prec])
    report("four-step c2r %s %s" % (shape, prec), oracle.rel_l2(gpu_c2r(H, shape, prec), oracle.c2r(H, shape[2])),
           TOL[prec])


@pytest.mark.parametrize("scale", [1e-300, 1e-30, 1e30, 1e200])
@pytest.mark.parametrize("kind", ["c2c", "r2c"])
def test_fp64_extreme_magnitudes(scale, kind):
    """FP64 kernels compute in float-float when every value of a tile lies in its range
    (2^-74 .. 2^127) and redo the tile in FP64 otherwise; results stay within 1e-12 for inputs
    far outside float range, including a field where only some tiles are extreme."""
    shape = (64, 48, 96)
    if kind == "c2c":
        x = synth.uniform_complex(shape, 61) * scale
    else:
        x = synth.uniform_real(shape, 61) * scale
    x[:4] /= scale   # a few planes of ordinary magnitude: mixed tiles
    if kind == "c2c":
        report("c2c f64 x %g" % scale, oracle.rel_l2(gpu_c2c(x, "f64"), oracle.c2c(x)), TOL["f64"])
        report("c2c bwd f64 x %g" % scale, oracle.rel_l2(gpu_c2c(x, "f64", +1), oracle.c2c(x, +1)), TOL["f64"])
    else:
        ref = oracle.r2c(x)
        report("r2c f64 x %g" % scale, oracle.rel_l2(gpu_r2c(x, "f64"), ref), TOL["f64"])
        report("c2r f64 x %g" % scale, oracle.rel_l2(gpu_c2r(ref, shape, "f64"), oracle.c2r(ref, shape[2])),
               TOL["f64"])


def test_fp64_tiny_values_mixed_with_ordinary_ones():
    """Values below float-float precision range inside tiles that also hold ordinary values stay on
    the fast path (their contribution is negligible); accuracy must hold."""
    shape = (64, 48, 96)
    x = synth.uniform_complex(shape, 62)
    x[:, :, ::3] *= 1e-30
    x[:, ::5, :] *= 1e-200
    report("c2c f64 tiny mixed", oracle.rel_l2(gpu_c2c(x, "f64"), oracle.c2c(x)), TOL["f64"])
    r = x.real.copy()
    report("r2c f64 tiny mixed", oracle.rel_l2(gpu_r2c(r, "f64"), oracle.r2c(r)), TOL["f64"])


@pytest.mark.parametrize("shape,batch,kind,prec", [((24, 20, 30), 3, "c2c", "f32"), ((16, 24, 40), 5, "r2c", "f32"),
                                                   ((12, 10, 16), 4, "r2c", "f64"), ((64, 8, 8), 2, "c2c", "f64")])
def test_batched_plan_matches_per_field_oracle(shape, batch, kind, prec):
    if kind == "c2c":
        xs = np.stack([synth.uniform_complex(shape, 70 + b) for b in range(batch)]).astype(CDT[prec])
    else:
        xs = np.stack([synth.uniform_real(shape, 70 + b) for b in range(batch)]).astype(RDT[prec])
    with afft.Plan(shape, kind, prec, batch=batch) as p:
        X = p.forward(torch.from_numpy(xs).cuda())
        y = p.backward(X)
        torch.cuda.synchronize()
        Xh, yh = X.cpu().numpy(), y.cpu().numpy()
    for b in range(batch):
        ref = oracle.c2c(xs[b]) if kind == "c2c" else oracle.r2c(xs[b])
        report("batched %s %s %s [%d]" % (shape, kind, prec, b), oracle.rel_l2(Xh[b], ref), TOL[prec])
        report("batched %s %s %s round trip [%d]" % (shape, kind, prec, b), oracle.rel_l2(yh[b], xs[b]), TOL[prec])


def test_multi_plan_graph_matches_separate_executes():
    sizes = [(48, 48, 48, 3), (64, 64, 64, 2), (120, 120, 120, 1)]
    plans = [afft.Plan(s[:3], "r2c", "f32", batch=s[3]) for s in sizes]
    xs = [torch.from_numpy(np.stack([synth.random_mode_field(s[:3], 80 + b, n_modes=8)
                                     for b in range(s[3])]).astype(np.float32)).cuda() for s in sizes]
    ref = [p.forward(x) for p, x in zip(plans, xs)]
    refb = [p.backward(r) for p, r in zip(plans, ref)]
    outs = [torch.empty_like(r) for r in ref]
    backs = [torch.empty_like(x) for x in xs]
    m = afft.Multi(plans)
    for _ in range(3):        # capture once, then replay
        m.forward(xs, outs)
        m.backward(outs, backs)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    for a, b in zip(backs, refb):
        assert torch.equal(a, b)
    outs2 = [torch.empty_like(r) for r in ref]   # new buffers: a second graph
    m.forward(xs, outs2)
    torch.cuda.synchronize()
    for a, b in zip(outs2, ref):
        assert torch.equal(a, b)
    m.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("shape,kind,prec", [((128, 128, 128), "r2c", "f32"), ((96, 96, 96), "c2c", "f64")])
def test_autotune_keeps_results(shape, kind, prec):
    if kind == "c2c":
        x = synth.uniform_complex(shape, 90).astype(CDT[prec])
        ref = oracle.c2c(x)
    else:
        x = synth.uniform_real(shape, 90).astype(RDT[prec])
        ref = oracle.r2c(x)
    with afft.Plan(shape, kind, prec) as p:
        before = p.describe()
        p.tune()
        after = p.describe()
        assert set(after) == set(before) and after["n"] == list(shape)
        X = p.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
    print("\n[tune] %s -> %s" % (before, after))
    report("tuned %s %s %s" % (shape, kind, prec), oracle.rel_l2(X.cpu().numpy(), ref), TOL[prec])


@pytest.mark.parametrize("shape,prec", [((64, 64, 64), "f32"), ((96, 48, 64), "f64"), ((6, 10, 16), "f32"),
                                        ((32, 48, 40), "f32"), ((1, 16, 16), "f64"), ((40, 24, 30), "f64"),
                                        ((128, 120, 96), "f32")])
def test_poisson_solve_matches_oracle(shape, prec):
    """u = -Lap^{-1} f through the fused N0 operator (pipelined N0 stages) or the separate multiply
    (other N0 lengths), against the oracle's spectral solve on the same input."""
    f = synth.uniform_real(shape, 101)
    f -= f.mean()
    x = f.astype(RDT[prec])
    with afft.Plan(shape, "r2c", prec) as p:
        u = p.poisson(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
    report("poisson %s %s" % (shape, prec), oracle.rel_l2(u.cpu().numpy(), oracle.poisson(x)), TOL[prec])


@pytest.mark.parametrize("n,prec", [(128, "f32"), (128, "f64"), (192, "f32")])
def test_poisson_manufactured_solution(n, prec):
    """f from a band-limited manufactured u (16 modes, |k| <= n/4): the solve returns u itself."""
    f, u = synth.manufactured_poisson((n, n, n), 7, n_modes=16)
    with afft.Plan((n, n, n), "r2c", prec) as p:
        got = p.poisson(torch.from_numpy(f.astype(RDT[prec])).cuda())
        torch.cuda.synchronize()
    tol = TOL[prec] if prec == "f64" else 2e-6
    report("poisson manufactured %d^3 %s" % (n, prec), oracle.rel_l2(got.cpu().numpy(), u), tol)


def test_poisson_batched():
    shape, B = (32, 32, 32), 3
    fs = np.stack([synth.manufactured_poisson(shape, 20 + b, n_modes=6)[0] for b in range(B)]).astype(np.float32)
    us = np.stack([synth.manufactured_poisson(shape, 20 + b, n_modes=6)[1] for b in range(B)])
    with afft.Plan(shape, "r2c", "f32", batch=B) as p:
        got = p.poisson(torch.from_numpy(fs).cuda())
        torch.cuda.synchronize()
    for b in range(B):
        report("poisson batched [%d]" % b, oracle.rel_l2(got[b].cpu().numpy(), us[b]), 2e-6)


# --- blocked c2c layout ([n1/32][batch n0][32][n2] workspace) --------------------------

@pytest.mark.parametrize("shape,batch,prec", [((64, 64, 256), 1, "f32"), ((32, 96, 128), 1, "f32"),
                                              ((16, 64, 128), 3, "f32"), ((64, 32, 128), 1, "f64"),
                                              ((512, 32, 128), 1, "f32"), ((24, 64, 1024), 2, "f64")])
def test_c2c_blocked_layout_matches_oracle(shape, batch, prec):
    """The blocked layout (N2 stage into the workspace, N0 stage on rows 32 n2 apart, N1 stage
    reading runs of 32 rows back to row-major) gives the oracle's transform, forward and back."""
    xs = np.stack([synth.uniform_complex(shape, 90 + b) for b in range(batch)]).astype(CDT[prec])
    with afft.Plan(shape, "c2c", prec, batch=batch if batch > 1 else None) as p:
        p.set_blocked(True)
        assert p.describe()["blocked"] == 1
        n = int(np.prod(shape)) * batch
        assert afft.load().afft_plan_workspace_bytes(p._p) >= n * np.dtype(CDT[prec]).itemsize
        t = torch.from_numpy(xs if batch > 1 else xs[0]).cuda()
        before = t.clone()
        X = p.forward(t)
        y = p.backward(X)
        torch.cuda.synchronize()
        assert torch.equal(t, before), "the blocked forward modified its input"
        Xh = X.cpu().numpy().reshape((batch,) + shape)
        yh = y.cpu().numpy().reshape((batch,) + shape)
    for b in range(batch):
        ref = oracle.c2c(xs[b], -1, "fft")
        report("blocked c2c %s %s fwd [%d]" % (shape, prec, b), oracle.rel_l2(Xh[b], ref), TOL[prec])
        report("blocked c2c %s %s round trip [%d]" % (shape, prec, b), oracle.rel_l2(yh[b], xs[b]), TOL[prec])


def test_c2c_blocked_backward_alone_matches_oracle():
    shape = (64, 64, 256)
    X = synth.uniform_complex(shape, 95).astype(np.complex64)
    with afft.Plan(shape, "c2c", "f32") as p:
        p.set_blocked(True)
        y = p.backward(torch.from_numpy(X).cuda())
        torch.cuda.synchronize()
    report("blocked c2c %s backward" % (shape,), oracle.rel_l2(y.cpu().numpy(), oracle.c2c(X, +1, "fft")), TOL["f32"])


def test_c2c_blocked_split_precision():
    shape = (32, 64, 256)
    x = synth.uniform_complex(shape, 97).astype(np.complex64)
    with afft.Plan(shape, "c2c", "f32_split") as p:
        p.set_blocked(True)
        X = p.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
    report("blocked c2c %s split fwd" % (shape,), oracle.rel_l2(X.cpu().numpy(), oracle.c2c(x, -1, "fft")), 2e-5)


def test_blocked_layout_eligibility_and_default():
    """Refused where the shapes do not allow it; on by default where N0 rows lie beyond 4 MB
    apart (1024^3 complex64: the plan's workspace is the array's size); off again on request."""
    with afft.Plan((64, 64, 256), "r2c", "f32") as p:
        with pytest.raises(afft.AfftError):
            p.set_blocked(True)
    with afft.Plan((64, 48, 256), "c2c", "f32") as p:   # n1 not a multiple of 32
        with pytest.raises(afft.AfftError):
            p.set_blocked(True)
    with afft.Plan((512, 512, 512), "c2c", "f32") as p:  # N0 rows 2 MB apart: row-major
        assert p.describe()["blocked"] == 0
    with afft.Plan((1024, 1024, 1024), "c2c", "f32") as p:
        assert p.describe()["blocked"] == 1
        assert afft.load().afft_plan_workspace_bytes(p._p) == 1024 ** 3 * 8
        p.set_blocked(False)
        assert p.describe()["blocked"] == 0
        assert afft.load().afft_plan_workspace_bytes(p._p) == 0


def test_tune_with_cache_file(tmp_path):
    """A tuned configuration is stored under the plan's key and applied, without tuning, to a
    new plan of the same key; results do not change beyond rounding."""
    path = str(tmp_path / "tune.json")
    shape = (64, 64, 128)
    x = synth.uniform_real(shape, 61).astype(np.float32)
    with afft.Plan(shape, "r2c", "f32") as p:
        assert p.tune(cache=path) is False
        cfg = p.tuning
        ref = p.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    with afft.Plan(shape, "r2c", "f32") as q:
        assert q.tune(cache=path) is True
        assert q.tuning == cfg
        got = q.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    report("tuned from cache %s" % (shape,), oracle.rel_l2(got, oracle.r2c(x)), TOL["f32"])
    report("tuned from cache vs tuned", oracle.rel_l2(got, ref), TOL["f32"])
    with afft.Plan(shape, "r2c", "f32") as r:
        r.set_tuning([1024, 1, 1, 0])
        assert r.tuning[0] == 1024
        with pytest.raises(afft.AfftError):
            r.set_tuning([-1, 0, 0, 0])
