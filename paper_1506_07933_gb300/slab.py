"""Slab decomposition of the 3-D FFT over P processes (AccFFT Algorithm 3).

Each process holds n0/P consecutive planes of the spatial array, [n0/P][n1][n2]
(real for r2c, complex for c2c).  The forward transform:

1. runs the 1-D FFTs along N2 and N1 of its planes (an axes {1, 2} plan: the
   contiguous stage, r2c or c2c, then the strided N1 stage);
2. packs, for every process s, the block [n0/P][rows s n1/P ...][n2h] of its
   planes into one contiguous piece (one pitched copy per s: n0/P rows of
   n1/P * n2h elements, n1 * n2h elements apart);
3. exchanges the pieces with one all-to-all (NCCL on GPUs), so that process r
   receives from s the planes s n0/P ... of rows r n1/P ... -- contiguous in
   its [n0][n1/P][n2h] array, which therefore needs no unpack;
4. runs the 1-D FFTs along N0 (an axes {0} c2c plan over [n0][n1/P][n2h]).

The output is distributed as N0 x N1/P x N2h (Algorithm 3's output layout): rank
r holds X[:, r n1/P : (r+1) n1/P, :].  The backward transform runs the same steps
in reverse: N0 inverse (unscaled), the all-to-all (each rank's planes s n0/P ...
are already contiguous), an unpack of the received [P][n0/P][n1/P][n2h] into
[n0/P][n1][n2h] (pitched copies), then the N1 inverse and the contiguous inverse
(c2r or c2c) carrying the global 1/N.  Remote data lands in local memory before
any kernel reads it: no kernel touches another GPU's memory.

The local stages, copies and buffers come from an engine: ``GpuEngine`` runs them
through the C ABI of libafft (PyTorch supplies memory and streams).  Tests on the
CPU pass an engine of their own to check the partition and exchange bookkeeping
with gloo ranks; the bookkeeping here is the same for both.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import afft


class GpuEngine:
    """Local stages through libafft: an axes {1, 2} plan over the rank's planes and an axes {0}
    c2c plan over its rows after the exchange."""

    def __init__(self, shape, kind, precision, world):
        n0, n1, n2 = shape
        self.kind = afft.KINDS[kind] if isinstance(kind, str) else int(kind)
        self.precision = afft.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        nh = n2 // 2 + 1 if self.kind == afft.R2C else n2
        self.zy = afft.Plan((n0 // world, n1, n2), self.kind, self.precision, axes=6)
        self.x = afft.Plan((n0, n1 // world, nh), afft.C2C, self.precision, axes=1)
        # the whole backward transform carries 1/N once, in its last (contiguous) stage
        self.zy.set_backward_scale(1.0 / (float(n0) * n1 * n2))
        self.x.set_backward_scale(1.0)
        self.cdtype = afft._CDT[self.precision]
        self.rdtype = afft._RDT[self.precision] if self.kind == afft.R2C else self.cdtype
        self.device = self.zy.device

    def empty(self, shape, complex_=True):
        return torch.empty(shape, dtype=self.cdtype if complex_ else self.rdtype, device=self.device)

    def forward_zy(self, x, out):
        self.zy.forward(x, out)

    def forward_x(self, y, out):
        self.x.forward(y, out)

    def backward_x(self, z, out):
        self.x.backward(z, out)

    def backward_zy(self, y, out):
        self.zy.backward(y, out)

    @staticmethod
    def copy_2d(dst, dst_off, dpitch, src, src_off, spitch, width, rows):
        """Element offsets and pitches (complex elements) into contiguous tensors of one dtype."""
        e = dst.element_size()
        afft.afft_copy_2d(dst.data_ptr() + dst_off * e, dpitch * e, src.data_ptr() + src_off * e, spitch * e,
                          width * e, rows, afft._stream_handle(None))

    def close(self):
        self.zy.close()
        self.x.close()


class SlabFFT:
    """3-D FFT of an n0 x n1 x n2 array distributed in slabs of n0/P planes over the processes of
    `group` (torch.distributed, initialised by the caller; one GPU per process).  n0 and n1 must
    be multiples of P."""

    def __init__(self, shape, kind="r2c", precision="f32", group=None, engine=None):
        self.shape = tuple(int(s) for s in shape)
        n0, n1, n2 = self.shape
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        P = self.world
        if n0 % P or n1 % P:
            raise ValueError("n0 = %d and n1 = %d must be multiples of the %d processes" % (n0, n1, P))
        self.kind = kind
        self.n0p, self.n1p = n0 // P, n1 // P
        self.nh = n2 // 2 + 1 if kind == "r2c" else n2
        self.engine = engine if engine is not None else GpuEngine(self.shape, kind, precision, P)

    # local shapes
    @property
    def input_shape(self):
        """This rank's spatial slab: planes rank * n0/P ... of the global array."""
        return (self.n0p,) + self.shape[1:]

    @property
    def output_shape(self):
        """This rank's spectral block: all k0, rows rank * n1/P ..., all k2 (N0 x N1/P x N2h)."""
        return (self.shape[0], self.n1p, self.nh)

    def _exchange(self, recv, send):
        if not dist.is_initialized():      # one process and no process group: a local copy
            n = send.numel()
            self.engine.copy_2d(recv, 0, n, send, 0, n, n, 1)
        else:
            flat = lambda t: torch.view_as_real(t).view(-1) if t.is_complex() else t.view(-1)
            dist.all_to_all_single(flat(recv), flat(send), group=self.group)

    def pack_plan(self):
        """(dst_off, dpitch, src_off, spitch, width, rows) of the pitched copy for each rank s, in
        complex elements: the block of rows s n1/P ... of every local plane [n0/P][n1][n2h] into
        piece s of the send buffer [P][n0/P][n1/P][n2h].  The unpack uses the same copies with
        source and destination exchanged."""
        n1, nh, n0p, n1p = self.shape[1], self.nh, self.n0p, self.n1p
        return [(s * n0p * n1p * nh, n1p * nh, s * n1p * nh, n1 * nh, n1p * nh, n0p) for s in range(self.world)]

    def forward(self, x):
        """Forward transform of this rank's slab `x` [n0/P][n1][n2]; returns [n0][n1/P][n2h]."""
        E = self.engine
        y = E.empty((self.n0p, self.shape[1], self.nh))
        E.forward_zy(x, y)
        send = E.empty((self.world, self.n0p, self.n1p, self.nh))
        for d_off, dp, s_off, sp, w, rows in self.pack_plan():
            E.copy_2d(send, d_off, dp, y, s_off, sp, w, rows)
        del y
        recv = E.empty(self.output_shape)
        self._exchange(recv, send)
        del send
        out = E.empty(self.output_shape)
        E.forward_x(recv, out)
        return out

    def backward(self, z):
        """Backward transform of this rank's block `z` [n0][n1/P][n2h] (times 1/N); returns the
        rank's slab [n0/P][n1][n2]."""
        E = self.engine
        t = E.empty(self.output_shape)
        E.backward_x(z, t)
        recv = E.empty((self.world, self.n0p, self.n1p, self.nh))
        self._exchange(recv, t)           # planes s n0/P ... of t are piece s, already contiguous
        del t
        y = E.empty((self.n0p, self.shape[1], self.nh))
        for d_off, dp, s_off, sp, w, rows in self.pack_plan():
            E.copy_2d(y, s_off, sp, recv, d_off, dp, w, rows)
        del recv
        out = E.empty(self.input_shape, complex_=self.kind != "r2c")
        E.backward_zy(y, out)
        return out

    def close(self):
        if hasattr(self.engine, "close"):
            self.engine.close()
