"""Slab decomposition (Algorithm 3) bookkeeping with gloo ranks on the CPU.

Each rank holds n0/P planes; the product's SlabFFT computes the pack offsets and
pitches, runs the all-to-all and places the pieces, while the local 1-D FFT
stages come from an engine.  Here the engine computes those stages with the
oracle's 1-D DFT (and numpy's irfft for the final real axis), standing in for
the GPU kernels, which the GPU tests cover.  Every rank's block of the result is
compared with the oracle's full 3-D transform of the global array, and the
backward transform with the rank's own slab.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1506_07933_gb300 import slab, synth


class OracleEngine:
    """Local stages by the oracle on CPU tensors (complex128 / float64)."""

    def __init__(self, shape, kind):
        self.shape, self.kind = shape, kind
        self.N = float(np.prod(shape))

    def empty(self, shape, complex_=True):
        return torch.empty(shape, dtype=torch.complex128 if complex_ else torch.float64)

    def forward_zy(self, x, out):
        a = x.numpy().astype(np.complex128)
        A = oracle.dft_axis(a, 2, -1)
        if self.kind == "r2c":
            A = A[..., : self.shape[2] // 2 + 1]
        out.copy_(torch.from_numpy(oracle.dft_axis(np.ascontiguousarray(A), 1, -1)))

    def forward_x(self, y, out):
        out.copy_(torch.from_numpy(oracle.dft_axis(y.numpy(), 0, -1)))

    def backward_x(self, z, out):
        out.copy_(torch.from_numpy(oracle.dft_axis(z.numpy(), 0, +1)))

    def backward_zy(self, y, out):
        B = oracle.dft_axis(y.numpy(), 1, +1)
        n2 = self.shape[2]
        if self.kind == "r2c":
            r = np.fft.irfft(B, n=n2, axis=2) * n2 / self.N
        else:
            r = oracle.dft_axis(B, 2, +1) / self.N
        out.copy_(torch.from_numpy(np.ascontiguousarray(r)))

    @staticmethod
    def copy_2d(dst, dst_off, dpitch, src, src_off, spitch, width, rows):
        d, s = dst.view(-1), src.view(-1)
        for i in range(rows):
            d[dst_off + i * dpitch: dst_off + i * dpitch + width] = s[src_off + i * spitch: src_off + i * spitch + width]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, shape, kind, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x = synth.uniform_real(shape, 77) if kind == "r2c" else synth.uniform_complex(shape, 77)
        f = slab.SlabFFT(shape, kind, "f64", engine=OracleEngine(shape, kind))
        n0p, n1p = f.n0p, f.n1p
        mine = torch.from_numpy(np.ascontiguousarray(x[rank * n0p:(rank + 1) * n0p]))
        assert tuple(mine.shape) == f.input_shape
        Z = f.forward(mine)
        assert tuple(Z.shape) == f.output_shape
        ref = oracle.r2c(x) if kind == "r2c" else oracle.c2c(x, -1)
        e_fwd = oracle.rel_l2(Z.numpy(), ref[:, rank * n1p:(rank + 1) * n1p, :])
        back = f.backward(Z)
        e_bwd = oracle.rel_l2(back.numpy(), mine.numpy())
        out[rank] = (e_fwd, e_bwd)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,kind", [(2, (8, 6, 10), "r2c"), (2, (6, 4, 10), "c2c"),
                                               (3, (6, 9, 8), "r2c"), (3, (9, 6, 5), "c2c")])
def test_slab_forward_and_backward_with_gloo_ranks(world, shape, kind):
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, port, shape, kind, out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == list(range(world))
    for r in range(world):
        e_fwd, e_bwd = out[r]
        assert e_fwd < 1e-13 and e_bwd < 1e-13, (r, e_fwd, e_bwd)


def test_pack_plan_covers_every_element_once():
    """The pitched copies of the pack move each element of the rank's [n0/P][n1][n2h] planes to
    exactly one place of the send buffer, and the unpack inverts them (P = 1 .. 4)."""
    for P in (1, 2, 3, 4):
        shape = (2 * P, 3 * P, 6)
        f = slab.SlabFFT.__new__(slab.SlabFFT)
        f.shape, f.world, f.rank, f.kind = shape, P, 0, "c2c"
        f.n0p, f.n1p, f.nh = shape[0] // P, shape[1] // P, shape[2]
        y = torch.arange(f.n0p * shape[1] * f.nh, dtype=torch.float64)
        send = torch.full((P * f.n0p * f.n1p * f.nh,), -1.0)
        for d_off, dp, s_off, sp, w, rows in f.pack_plan():
            OracleEngine.copy_2d(send, d_off, dp, y, s_off, sp, w, rows)
        assert sorted(send.tolist()) == y.tolist()
        yy = y.view(f.n0p, shape[1], f.nh)
        for s in range(P):
            piece = send[s * f.n0p * f.n1p * f.nh:(s + 1) * f.n0p * f.n1p * f.nh].view(f.n0p, f.n1p, f.nh)
            assert torch.equal(piece, yy[:, s * f.n1p:(s + 1) * f.n1p, :])
        back = torch.full_like(y, -1.0)
        for d_off, dp, s_off, sp, w, rows in f.pack_plan():
            OracleEngine.copy_2d(back, s_off, sp, send, d_off, dp, w, rows)
        assert torch.equal(back, y)
