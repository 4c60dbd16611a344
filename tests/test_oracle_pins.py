"""Pins for the FP64 CPU oracle: facts fixed by the mathematics, not by the oracle.

The paper prints no numeric transform values (every result figure of AccFFT
Section 3 is a timing plot), so nothing here is a value from the paper.  Each
test checks the oracle against a closed form, an exact special case, an
invariant or brute force, chosen so that a plausible mistake (a dropped term,
a flipped sign, a transposed axis, a missing 1/N) fails at least one of them;
``test_planted_mistakes_are_caught`` shows that on mutated oracles.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1506_07933_gb300 import synth

TOL = 1e-13
SHAPES = [(4, 6, 5), (8, 12, 30), (3, 5, 16), (1, 7, 9)]
METHODS = ["naive", "fft"]


def grid(shape):
    return np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")


# --- closed forms ------------------------------------------------------------

@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", SHAPES)
def test_impulse_at_origin_gives_flat_spectrum(shape, method):
    x = np.zeros(shape, complex)
    x[0, 0, 0] = 1.0
    X = oracle.c2c(x, -1, method)
    assert np.max(np.abs(X - 1.0)) < TOL


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape,pos", [((4, 6, 5), (1, 2, 3)), ((8, 12, 30), (5, 7, 11)),
                                       ((3, 5, 16), (2, 4, 9))])
def test_shift_theorem(shape, pos, method):
    """An impulse at (a, b, c) has spectrum exp(-2 pi i (k0 a/n0 + k1 b/n1 + k2 c/n2))."""
    x = np.zeros(shape, complex)
    x[pos] = 1.0
    X = oracle.c2c(x, -1, method)
    k0, k1, k2 = grid(shape)
    ph = (k0 * pos[0] % shape[0]) / shape[0] + (k1 * pos[1] % shape[1]) / shape[1] \
        + (k2 * pos[2] % shape[2]) / shape[2]
    expect = np.exp(-2j * np.pi * ph)
    assert np.max(np.abs(X - expect)) < TOL


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape,kstar", [((4, 6, 5), (1, 5, 2)), ((8, 12, 30), (3, 0, 29)),
                                         ((16, 3, 10), (15, 2, 5))])
def test_plane_wave_is_a_delta(shape, kstar, method):
    """exp(+2 pi i k*.j/n) transforms to N at k* and 0 elsewhere."""
    j0, j1, j2 = grid(shape)
    ph = (j0 * kstar[0] % shape[0]) / shape[0] + (j1 * kstar[1] % shape[1]) / shape[1] \
        + (j2 * kstar[2] % shape[2]) / shape[2]
    x = np.exp(2j * np.pi * ph)
    X = oracle.c2c(x, -1, method)
    N = np.prod(shape)
    expect = np.zeros(shape, complex)
    expect[kstar] = N
    assert np.max(np.abs(X - expect)) < TOL * N


@pytest.mark.parametrize("method", METHODS)
def test_real_cosine_gives_conjugate_pair(method):
    shape = (8, 12, 10)
    k = np.array([3, -2, 4])
    a, phi = 1.7, 0.6
    j0, j1, j2 = grid(shape)
    x = a * np.cos(2 * np.pi * (k[0] * j0 / 8 + k[1] * j1 / 12 + k[2] * j2 / 10) + phi)
    X = oracle.c2c(x.astype(complex), -1, method)
    N = np.prod(shape)
    expect = np.zeros(shape, complex)
    expect[tuple(k % shape)] += N / 2 * a * np.exp(1j * phi)
    expect[tuple(-k % shape)] += N / 2 * a * np.exp(-1j * phi)
    assert np.max(np.abs(X - expect)) < 1e-12 * N


# --- exact special cases -----------------------------------------------------

def dft_matrix_exact(n):
    """Exact DFT matrices for n in {1, 2, 4}: entries are powers of -i."""
    if n == 1:
        return np.ones((1, 1), complex)
    powers = {0: 1, 1: -1j, 2: -1, 3: 1j}  # (-i)^m for the 4th roots; n=2 uses m even
    step = 4 // n
    return np.array([[powers[(step * j * k) % 4] for k in range(n)] for j in range(n)])


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", [(2, 2, 2), (4, 2, 4), (4, 4, 4), (1, 4, 2)])
def test_small_power_of_two_sizes_match_exact_integer_dft(shape, method):
    """For n in {1, 2, 4} the DFT matrix has entries in {1, -1, i, -i}: integer in, Gaussian
    integers out.  The 3-D DFT is the Kronecker product F_n0 x F_n1 x F_n2 (row-major)."""
    rng = np.random.default_rng(7)
    x = rng.integers(-9, 10, size=shape) + 1j * rng.integers(-9, 10, size=shape)
    F = np.kron(np.kron(dft_matrix_exact(shape[0]), dft_matrix_exact(shape[1])),
                dft_matrix_exact(shape[2]))
    expect = (F @ x.ravel()).reshape(shape)
    X = oracle.c2c(x, -1, method)
    assert np.max(np.abs(X - expect)) < 1e-12
    assert np.array_equal(np.round(X.real), expect.real) and np.array_equal(np.round(X.imag), expect.imag)


# --- invariants --------------------------------------------------------------

@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", SHAPES)
def test_parseval(shape, method):
    x = synth.uniform_complex(shape, 11)
    X = oracle.c2c(x, -1, method)
    N = np.prod(shape)
    assert abs(np.sum(np.abs(X) ** 2) / (N * np.sum(np.abs(x) ** 2)) - 1) < TOL


@pytest.mark.parametrize("method", METHODS)
def test_linearity(method):
    shape = (6, 10, 8)
    x, y = synth.uniform_complex(shape, 1), synth.uniform_complex(shape, 2)
    a, b = 0.3 - 1.1j, -2.0 + 0.5j
    lhs = oracle.c2c(a * x + b * y, -1, method)
    rhs = a * oracle.c2c(x, -1, method) + b * oracle.c2c(y, -1, method)
    assert oracle.rel_l2(lhs, rhs) < TOL


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", SHAPES)
def test_backward_inverts_forward(shape, method):
    x = synth.uniform_complex(shape, 3)
    assert oracle.rel_l2(oracle.c2c(oracle.c2c(x, -1, method), +1, method), x) < TOL
    assert oracle.rel_l2(oracle.c2c(oracle.c2c(x, +1, method), -1, method), x) < TOL


@pytest.mark.parametrize("method", METHODS)
def test_hermitian_symmetry_for_real_input(method):
    shape = (6, 5, 8)
    x = synth.uniform_real(shape, 4)
    X = oracle.c2c(x.astype(complex), -1, method)
    k = [np.arange(n) for n in shape]
    mirror = X[np.ix_(-k[0] % 6, -k[1] % 5, -k[2] % 8)]
    assert np.max(np.abs(X - np.conj(mirror))) < TOL * np.max(np.abs(X))


def test_stage_order_is_immaterial():
    """The 3-D DFT factors into 1-D DFTs along each axis in any order (Algorithm 1's
    factorisation); the oracle's order N2, N1, N0 equals N0, N1, N2."""
    x = synth.uniform_complex((6, 10, 15), 5)
    y = x
    for ax in (0, 1, 2):
        y = oracle.dft_axis(y, ax, -1, "naive")
    assert oracle.rel_l2(oracle.c2c(x, -1, "naive"), y) < TOL


# --- brute force: fft engine against the naive definition --------------------

SIZES = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 15, 16, 20, 24, 25, 27, 30, 32, 48, 60, 64]


@pytest.mark.parametrize("n", SIZES)
def test_fft_engine_matches_definition_1d(n):
    x = synth.uniform_complex((3, n), 100 + n)
    a = oracle.dft_axis(x, 1, -1, "naive")
    b = oracle.dft_axis(x, 1, -1, "fft")
    assert oracle.rel_l2(b, a) < 1e-14
    a = oracle.dft_axis(x, 1, +1, "naive")
    b = oracle.dft_axis(x, 1, +1, "fft")
    assert oracle.rel_l2(b, a) < 1e-14


@pytest.mark.parametrize("shape", [(8, 12, 30), (5, 9, 16), (32, 32, 32), (2, 3, 60)])
def test_fft_engine_matches_definition_3d(shape):
    x = synth.uniform_complex(shape, 9)
    for d in (-1, +1):
        assert oracle.rel_l2(oracle.c2c(x, d, "fft"), oracle.c2c(x, d, "naive")) < 1e-14


@pytest.mark.parametrize("real", [False, True])
def test_dft_bins_match_full_transform(real):
    """The per-bin definition (used for sampled checks at sizes too big for the CPU FFT)
    agrees with the naive separable transform on every bin of a small mixed shape."""
    shape = (6, 10, 8)
    x = synth.uniform_complex(shape, 3)
    if real:
        x = x.real.copy()
    full = oracle.c2c(x.astype(complex), -1, "naive")
    ks = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), -1).reshape(-1, 3)
    assert oracle.rel_l2(oracle.dft_bins(x, ks), full.ravel()) < 1e-14


# --- r2c / c2r -----------------------------------------------------------------

@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", [(4, 6, 8), (3, 5, 10), (6, 4, 7), (8, 8, 2), (2, 3, 1)])
def test_r2c_is_sliced_c2c(shape, method):
    x = synth.uniform_real(shape, 6)
    H = oracle.r2c(x, method)
    full = oracle.c2c(x.astype(complex), -1, method)
    assert H.shape == shape[:2] + (shape[2] // 2 + 1,)
    assert oracle.rel_l2(H, full[:, :, : shape[2] // 2 + 1]) < TOL


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", [(4, 6, 8), (3, 5, 10), (6, 4, 7), (8, 8, 2), (2, 3, 1)])
def test_c2r_inverts_r2c(shape, method):
    x = synth.uniform_real(shape, 8)
    y = oracle.c2r(oracle.r2c(x, method), shape[2], method)
    assert oracle.rel_l2(y, x) < TOL


def test_c2r_ignores_imaginary_parts_of_self_conjugate_bins():
    """Bins k2 = 0 and k2 = n2/2 are their own mirrors; c2r keeps only their real parts."""
    shape = (4, 6, 8)
    H = oracle.r2c(synth.uniform_real(shape, 12))
    G = H.copy()
    G[:, :, 0] += 0.25j
    G[:, :, 4] -= 0.5j
    assert np.array_equal(oracle.c2r(G, 8, "naive"), oracle.c2r(H, 8, "naive"))


@pytest.mark.parametrize("n", [16, 32])
def test_random_mode_field_spectrum_closed_form(n):
    """Noise-free sum of modes a cos(k.x + phi): the r2c spectrum is N/2 a e^{i phi} at +k and
    its conjugate at -k (folded into the half space k2 >= 0), zero elsewhere."""
    shape = (n, n, n)
    f, (ks, amp, phase) = synth.random_mode_field(shape, 2561, n_modes=64, noise=0.0,
                                                  return_modes=True)
    H = oracle.r2c(f, "fft")
    N = n ** 3
    expect = np.zeros_like(H)
    for k, a, p in zip(ks, amp, phase):
        for sgn in (1, -1):
            kk = sgn * k
            c = N / 2 * a * np.exp(sgn * 1j * p)
            if kk[2] >= 0 and 2 * kk[2] <= n:
                expect[kk[0] % n, kk[1] % n, kk[2]] += c
    assert np.max(np.abs(H - expect)) < 1e-12 * N


# --- the Poisson operator ------------------------------------------------------

@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 20, 24), (32, 16, 8)])
def test_poisson_reproduces_manufactured_solution(shape):
    """-Lap u = f with u a band-limited sum of modes: the spectral solve is exact up to rounding."""
    f, u = synth.manufactured_poisson(shape, 5, n_modes=8)
    assert oracle.rel_l2(oracle.poisson(f), u) < 1e-13
    assert oracle.rel_l2(oracle.poisson(f, "naive"), u) < 1e-13


def test_poisson_annihilates_constants_and_inverts_second_difference():
    """A constant f has zero-mean solution 0; for f = sin(x0) (k = (1,0,0)) u = sin(x0)."""
    shape = (16, 8, 10)
    assert np.max(np.abs(oracle.poisson(np.full(shape, 3.0)))) < 1e-14
    x0 = 2 * np.pi * np.arange(16) / 16
    f = np.broadcast_to(np.sin(x0)[:, None, None], shape).copy()
    assert oracle.rel_l2(oracle.poisson(f), f) < 1e-14
    f2 = np.broadcast_to(np.cos(3 * x0)[:, None, None], shape).copy()
    assert oracle.rel_l2(oracle.poisson(f2), f2 / 9.0) < 1e-14


# --- an independent library as a third opinion ---------------------------------

@pytest.mark.parametrize("shape", [(16, 24, 30), (48, 20, 64)])
def test_cross_check_numpy_fft(shape):
    x = synth.uniform_complex(shape, 13)
    assert oracle.rel_l2(oracle.c2c(x, -1, "fft"), np.fft.fftn(x)) < 1e-13
    assert oracle.rel_l2(oracle.c2c(x, +1, "fft"), np.fft.ifftn(x)) < 1e-13
    r = x.real.copy()
    assert oracle.rel_l2(oracle.r2c(r, "fft"), np.fft.rfftn(r)) < 1e-13
    H = np.fft.rfftn(r)
    assert oracle.rel_l2(oracle.c2r(H, shape[2], "fft"), np.fft.irfftn(H, s=shape, axes=(0, 1, 2))) < 1e-13


# --- the pins discriminate: mistakes planted in the oracle fail them ----------------

def _pin_errors(c2c_fwd):
    """Run a subset of the pins against a forward c2c function; return their errors."""
    errs = {}
    shape, pos = (4, 6, 5), (1, 2, 3)
    x = np.zeros(shape, complex)
    x[pos] = 1.0
    k0, k1, k2 = grid(shape)
    expect = np.exp(-2j * np.pi * (k0 * 1 / 4 + k1 * 2 / 6 + k2 * 3 / 5))
    errs["shift"] = np.max(np.abs(c2c_fwd(x) - expect))
    y = synth.uniform_complex(shape, 3)
    errs["parseval"] = abs(np.sum(np.abs(c2c_fwd(y)) ** 2) / (120 * np.sum(np.abs(y) ** 2)) - 1)
    errs["numpy"] = oracle.rel_l2(c2c_fwd(y), np.fft.fftn(y))
    return errs


def test_planted_mistakes_are_caught():
    good = _pin_errors(lambda v: oracle.c2c(v, -1, "fft"))
    assert max(good.values()) < TOL
    mutants = {
        "flipped sign": lambda v: oracle.c2c(v, +1, "fft") * np.prod(v.shape),
        "dropped axis": lambda v: oracle.dft_axis(oracle.dft_axis(v, 2, -1), 1, -1),
        "transposed axes": lambda v: oracle.c2c(v.transpose(0, 2, 1).copy(), -1)
        .reshape(v.shape) if v.shape[1] == v.shape[2] else
        oracle.c2c(v.reshape(v.shape[0], v.shape[2], v.shape[1]), -1).reshape(v.shape),
        "spurious 1/N": lambda v: oracle.c2c(v, -1, "fft") / np.prod(v.shape),
        "index off by one": lambda v: np.roll(oracle.c2c(v, -1, "fft"), 1, axis=2),
    }
    for name, fn in mutants.items():
        errs = _pin_errors(fn)
        assert max(errs.values()) > 1e-3, (name, errs)


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.c2c(np.zeros((4, 4)), -1)
    with pytest.raises(RuntimeError):
        oracle.c2c(np.zeros((4, 4, 4), complex), 0)
    with pytest.raises(ValueError):
        oracle.c2r(np.zeros((4, 4, 3), complex), 8)


def test_splitmix64_reference_values():
    """splitmix64 seeded with 0 yields the published first outputs
    0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F (states gamma*i, i = 0, 1, 2)."""
    gamma = 0x9E3779B97F4A7C15
    states = np.array([(gamma * i) % 2 ** 64 for i in range(3)], dtype=np.uint64)
    out = synth.splitmix64(states)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# --- golden fixture: a 2x4x4 Gaussian-integer DFT (tests/golden/dft_2x4x4.txt) -----------

def _golden_rows():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dft_2x4x4.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def _golden_input_ints():
    return {(j0, j1, j2): ((j0 + 2 * j1 + 3 * j2) % 5 - 2, (j0 * j1 + j2) % 3 - 1)
            for j0 in range(2) for j1 in range(4) for j2 in range(4)}


def _unit_root_pow(m, n):
    """exp(-2 pi i m / n) for n in {1, 2, 4}, exactly, as a Gaussian integer (re, im)."""
    q = (m * (4 // n)) % 4            # the same angle in quarter turns
    return [(1, 0), (0, -1), (-1, 0), (0, 1)][q]


def test_golden_2x4x4_fixture_is_the_exact_definition():
    """Every bin of the fixture equals the 3-D DFT definition evaluated in exact Gaussian-integer
    arithmetic (no floating point, no oracle code)."""
    x = _golden_input_ints()
    rows = _golden_rows()
    assert len(rows) == 32
    for k0, k1, k2, re, im in rows:
        sr = si = 0
        for (j0, j1, j2), (a, b) in x.items():
            w = (1, 0)
            for m, n in ((j0 * k0, 2), (j1 * k1, 4), (j2 * k2, 4)):
                c, d = _unit_root_pow(m, n)
                w = (w[0] * c - w[1] * d, w[0] * d + w[1] * c)
            sr += a * w[0] - b * w[1]
            si += a * w[1] + b * w[0]
        assert (sr, si) == (re, im), (k0, k1, k2)


@pytest.mark.parametrize("method", ["naive", "fft"])
def test_oracle_reproduces_golden_2x4x4(method):
    x = np.zeros((2, 4, 4), dtype=np.complex128)
    for (j0, j1, j2), (a, b) in _golden_input_ints().items():
        x[j0, j1, j2] = complex(a, b)
    X = oracle.c2c(x, -1, method)
    for k0, k1, k2, re, im in _golden_rows():
        assert abs(X[k0, k1, k2] - complex(re, im)) < 1e-12
