"""d-dimensional FFTs (d >= 3) from the 3-D stage kernels (AccFFT Algorithm 2).

Algorithm 2 transforms a d-dimensional array by batched 1-D FFTs along one axis
at a time, with the leading axes treated as a batch while the trailing ones are
transformed.  On one GPU that is:

* the trailing three axes as a batched 3-D plan (batch = product of the leading
  axes; c2c, or r2c halving the last axis);
* each leading axis a as one strided stage of an axes {0} c2c plan over the view
  [outer][n_a][inner], outer = product of the axes before a, inner = product of
  the (already transformed) axes after it.

Forward: trailing 3-D transform, then the leading axes from the innermost to the
outermost (Algorithm 1's order generalised: contiguous axis first).  Backward:
the reverse, the 1/N of the whole array applied once, by the last stage (the
trailing plan's contiguous one).  Every step runs in libafft's kernels.
"""
from __future__ import annotations

import math

import torch

from . import afft


class FFTN:
    """Forward/backward d-D transform, d >= 3: ``FFTN(shape, "c2c" | "r2c", "f32" | "f64")``."""

    def __init__(self, shape, kind="c2c", precision="f32"):
        self.shape = tuple(int(s) for s in shape)
        if len(self.shape) < 3:
            raise ValueError("FFTN needs at least 3 axes (use Plan for 3-D)")
        self.kind = kind
        self.precision = precision
        lead, trail = self.shape[:-3], self.shape[-3:]
        batch = math.prod(lead) if lead else 1
        self.trail = afft.Plan(trail, kind, precision, batch=batch, axes=7)
        self.trail.set_backward_scale(1.0 / math.prod(self.shape))
        nh = trail[2] // 2 + 1 if kind == "r2c" else trail[2]
        self.spec_shape = self.shape[:-1] + (nh,)
        self.lead = []   # (axis, plan over [outer][n_a][inner])
        for a in range(len(lead) - 1, -1, -1):
            outer = math.prod(self.shape[:a]) if a else 1
            inner = math.prod(self.spec_shape[a + 1:])
            p = afft.Plan((self.shape[a], 1, inner), "c2c", precision, batch=outer, axes=1)
            p.set_backward_scale(1.0)
            self.lead.append((a, p))

    @property
    def spectral_dtype(self):
        return self.trail.spectral_dtype

    @property
    def spatial_dtype(self):
        return self.trail.spatial_dtype

    def forward(self, x, out=None):
        """Unscaled forward transform; `out` (optional) receives the spectrum."""
        if tuple(x.shape) != self.shape:
            raise ValueError("input must have shape %s" % (self.shape,))
        if out is None:
            out = torch.empty(self.spec_shape, dtype=self.spectral_dtype, device=x.device)
        # the stages ping-pong between `out` and one buffer so that the last one writes `out`
        bufs = [out, torch.empty_like(out)] if self.lead else [out]
        k = len(self.lead) % 2
        y = self.trail.forward(x.view(self.trail.spatial_shape), bufs[k].view(self.trail.spectral_shape))
        for _, p in self.lead:
            k ^= 1
            p.forward(y.view(p.spectral_shape), bufs[k].view(p.spectral_shape))
            y = bufs[k]
        return out

    def backward(self, X, out=None):
        """Backward transform times 1/N of the whole array; `X` is not modified."""
        if tuple(X.shape) != self.spec_shape:
            raise ValueError("input must have shape %s" % (self.spec_shape,))
        y = X
        if self.lead:
            bufs = [torch.empty_like(X), torch.empty_like(X)]
            for i, (_, p) in enumerate(reversed(self.lead)):
                p.backward(y.view(p.spectral_shape), bufs[i % 2].view(p.spectral_shape))
                y = bufs[i % 2]
        if out is None:
            out = torch.empty(self.shape, dtype=self.spatial_dtype, device=X.device)
        self.trail.backward(y.view(self.trail.spectral_shape), out.view(self.trail.spatial_shape))
        return out

    def close(self):
        self.trail.close()
        for _, p in self.lead:
            p.close()
