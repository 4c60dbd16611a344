"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws numbers and nothing else: it holds none of the transform's
arithmetic, so both the CUDA library and the CPU oracle can be fed from it
without either depending on the other.  The paper runs on synthetic arrays
of given sizes and names no dataset (AccFFT Section 3, "Parameters in the
Experiments"); the recipes below fix what those arrays contain.

* ``uniform_complex``: re and im iid U[-1, 1) from ``numpy.random.default_rng``.
* ``random_mode_field``: a real field that is a sum of random Fourier modes,
  a_m cos(k_m . x + phi_m) on the grid x_j = 2 pi j / n, with integer
  wavevectors |k_m| <= n/4 (k_m != 0, rejection-sampled from the cube),
  a_m ~ N(0, 1), phi_m ~ U[0, 2 pi), plus optional 1e-3 N(0, 1) noise.
  The field is evaluated as a rank-M sum of outer products of 1-D complex
  exponentials (a matrix product), never through a Fourier transform.
* ``plane_wave_sum_torch`` / ``random_mode_field_torch``: the same kind of
  fields evaluated with torch on the GPU, for sizes too large for the host.
* ``splitmix64_uniform``: the counter-based generator used for inputs too
  large to draw on the host.  value(i, part) =
  (splitmix64(seed ^ (2 i + part)) >> 40) * 2**-24 * 2 - 1, with splitmix64
  as published by Steele, Lea and Flood (2014): z = x + 0x9E3779B97F4A7C15,
  z = (z ^ z>>30) * 0xBF58476D1CE4E5B9, z = (z ^ z>>27) * 0x94D049BB133111EB,
  z ^ z>>31.  The CUDA library carries its own implementation of the same
  definition; the two are compared bit for bit in the tests.
"""
from __future__ import annotations

import numpy as np

SPLITMIX_GAMMA = np.uint64(0x9E3779B97F4A7C15)
SPLITMIX_M1 = np.uint64(0xBF58476D1CE4E5B9)
SPLITMIX_M2 = np.uint64(0x94D049BB133111EB)


def uniform_complex(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """re, im iid U[-1, 1) from default_rng(seed); re drawn first, then im."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=shape)
    im = rng.uniform(-1.0, 1.0, size=shape)
    return (re + 1j * im).astype(dtype)


def uniform_real(shape, seed: int, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=shape).astype(dtype)


def draw_modes(shape, n_modes: int, seed: int):
    """Integer wavevectors |k| <= min(shape)/4, k != 0; amplitudes and phases."""
    rng = np.random.default_rng(seed)
    kmax = min(shape) // 4
    if kmax < 1:
        raise ValueError("grid too small for |k| <= n/4 modes")
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        r2 = int(k[0] * k[0] + k[1] * k[1] + k[2] * k[2])
        if r2 == 0 or r2 > kmax * kmax:
            continue
        ks.append(k)
    ks = np.array(ks, dtype=np.int64).reshape(n_modes, 3)
    amp = rng.standard_normal(n_modes)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return ks, amp, phase


def mode_sum(shape, ks, amp, phase) -> np.ndarray:
    """sum_m amp_m cos(k_m . x + phase_m) on x_j = 2 pi j / n, in float64."""
    n0, n1, n2 = shape
    j0, j1, j2 = (np.arange(n, dtype=np.float64) for n in shape)
    # e_d[m, j] = exp(i k_md 2 pi j / n_d); the exact-integer phase (k j mod n)
    # keeps the argument small.
    def exps(d, jv, n):
        ph = np.mod(np.outer(ks[:, d], np.arange(n, dtype=np.int64)), n).astype(np.float64)
        return np.exp(2j * np.pi * ph / n)
    e0, e1, e2 = exps(0, j0, n0), exps(1, j1, n1), exps(2, j2, n2)
    c = amp * np.exp(1j * phase)                        # [m]
    a = (c[:, None, None] * e0[:, :, None] * e1[:, None, :]).reshape(len(c), n0 * n1)
    field = (a.T @ e2).real                              # [(n0 n1), n2]
    return np.ascontiguousarray(field.reshape(n0, n1, n2))


def random_mode_field(shape, seed: int, n_modes: int = 64, noise: float = 1e-3,
                      dtype=np.float64, return_modes: bool = False):
    """The sum-of-random-modes real field; noise drawn from default_rng(seed + 1)."""
    shape = tuple(int(s) for s in shape)
    ks, amp, phase = draw_modes(shape, n_modes, seed)
    f = mode_sum(shape, ks, amp, phase)
    if noise:
        f += noise * np.random.default_rng(seed + 1).standard_normal(shape)
    f = f.astype(dtype)
    if return_modes:
        return f, (ks, amp, phase)
    return f


def plane_wave_sum_torch(shape, ks, coef, device="cuda"):
    """sum_m coef_m exp(+i k_m . x) on x_j = 2 pi j / n as a complex128 torch tensor on `device`:
    a rank-M sum of outer products of 1-D exponentials (exact-integer phases k j mod n), never a
    Fourier transform.  For inputs too large to build on the host; torch is imported here only."""
    import torch
    n0, n1, n2 = (int(s) for s in shape)
    ks = np.asarray(ks, dtype=np.int64).reshape(-1, 3)

    def exps(d, n):
        j = torch.arange(n, device=device, dtype=torch.int64)
        k = torch.tensor(ks[:, d], device=device, dtype=torch.int64)
        ph = torch.remainder(k[:, None] * j[None, :], n).to(torch.float64)
        return torch.exp(2j * torch.pi * ph / n)

    e0, e1, e2 = exps(0, n0), exps(1, n1), exps(2, n2)
    c = torch.tensor(np.asarray(coef, dtype=np.complex128), device=device)
    a = (c[:, None, None] * e0[:, :, None] * e1[:, None, :]).reshape(len(c), n0 * n1)
    return (a.T @ e2).reshape(n0, n1, n2)


def random_mode_field_torch(shape, seed: int, n_modes: int = 64, noise: float = 1e-3, device="cuda"):
    """random_mode_field (same modes) evaluated with torch on `device` in float64; the noise comes
    from a torch generator seeded with seed + 1 (so it differs from the numpy recipe's noise)."""
    import torch
    shape = tuple(int(s) for s in shape)
    ks, amp, phase = draw_modes(shape, n_modes, seed)
    f = plane_wave_sum_torch(shape, ks, amp * np.exp(1j * phase), device).real.contiguous()
    if noise:
        g = torch.Generator(device=device)
        g.manual_seed(seed + 1)
        f += noise * torch.randn(f.shape, device=device, dtype=torch.float64, generator=g)
    return f


def manufactured_poisson(shape, seed: int, n_modes: int = 16):
    """A zero-mean u = sum of n_modes random modes a cos(k.x + phi) with |k| <= min(n)/4 and the
    matching f = -Lap u = sum |k|^2 a cos(k.x + phi), both in float64.  Returns (f, u)."""
    shape = tuple(int(s) for s in shape)
    ks, amp, phase = draw_modes(shape, n_modes, seed)
    u = mode_sum(shape, ks, amp, phase)
    k2 = (ks * ks).sum(axis=1).astype(np.float64)
    f = mode_sum(shape, ks, amp * k2, phase)
    return f, u


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 output for state values x (uint64 array), wrapping arithmetic."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + SPLITMIX_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * SPLITMIX_M1
        z = (z ^ (z >> np.uint64(27))) * SPLITMIX_M2
        return z ^ (z >> np.uint64(31))


def splitmix64_uniform(count: int, seed: int, start: int = 0) -> np.ndarray:
    """Interleaved complex64 U[-1, 1) values for complex indices start..start+count-1."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    out = np.empty(2 * count, dtype=np.float32)
    for part in (0, 1):
        h = splitmix64(np.uint64(seed) ^ (np.uint64(2) * idx + np.uint64(part)))
        out[part::2] = ((h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24 * 2.0 - 1.0)
    return out.view(np.complex64)


def batched_sizes(count: int = 200, seed: int = 200, choices=(48, 64, 96, 120, 128, 160, 256)):
    """Cubic sizes drawn uniformly from ``choices`` with default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return [int(choices[i]) for i in rng.integers(0, len(choices), size=count)]
