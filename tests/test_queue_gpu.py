"""The persistent uneven-size executor (afft_queue_*): one kernel launch per direction for a set
of batched r2c plans of different sizes.  Every field is compared with the FP64 CPU oracle (the
forward spectrum, the backward transform of the oracle's spectrum, the round trip), at the FP32
tolerance of the parity tests, on two consecutive executions (the counters restart each time)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_07933_gb300 import afft, synth

pytestmark = pytest.mark.gpu
TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    afft.load()


def report(name, err):
    print("\n[parity] %-56s rel_l2 = %.3e (tol %.0e)" % (name, err, TOL))
    assert err <= TOL, (name, err)


# (shape, batch): every family of the executor, cubic and not
GROUPS = [((48, 48, 48), 3), ((64, 64, 64), 2), ((96, 96, 96), 2), ((120, 120, 120), 1),
          ((128, 128, 128), 1), ((160, 160, 160), 1), ((256, 256, 256), 1), ((48, 160, 256), 2),
          ]


def test_queue_matches_oracle_field_by_field():
    plans = [afft.Plan(shape, "r2c", "f32", batch=b) for shape, b in GROUPS]
    fields = [np.stack([synth.random_mode_field(shape, 9000 + 17 * i + j, n_modes=16, noise=1e-3)
                        for j in range(b)]).astype(np.float32) for i, (shape, b) in enumerate(GROUPS)]
    q = afft.Queue(plans)
    assert q.items(False) > 0 and q.items(True) > 0
    ins = [torch.from_numpy(f).cuda() for f in fields]
    specs = [torch.full(p.spectral_shape, float("nan"), dtype=torch.complex64, device="cuda") for p in plans]
    backs = [torch.full(p.spatial_shape, float("nan"), dtype=torch.float32, device="cuda") for p in plans]
    refs = [np.stack([oracle.r2c(f[j]) for j in range(f.shape[0])]) for f in fields]
    for rep in range(2):
        q.forward(ins, specs)
        q.backward(specs, backs)
        torch.cuda.synchronize()
        assert q.status() == 0
        for (shape, b), f, S, B, R in zip(GROUPS, fields, specs, backs, refs):
            Sh, Bh = S.cpu().numpy(), B.cpu().numpy()
            for j in range(b):
                report("queue r2c %s field %d (run %d)" % (shape, j, rep), oracle.rel_l2(Sh[j], R[j]))
                report("queue round trip %s field %d (run %d)" % (shape, j, rep), oracle.rel_l2(Bh[j], f[j]))
        for S in specs:
            S.fill_(float("nan"))
    # backward alone, from the oracle's spectrum (rounded to complex64)
    ospec = [torch.from_numpy(R.astype(np.complex64)).cuda() for R in refs]
    q.backward(ospec, backs)
    torch.cuda.synchronize()
    for (shape, b), B, R in zip(GROUPS, backs, refs):
        Bh = B.cpu().numpy()
        for j in range(b):
            ref = oracle.c2r(R[j].astype(np.complex64), shape[2])
            report("queue c2r %s field %d vs oracle" % (shape, j), oracle.rel_l2(Bh[j], ref))
    q.close()
    for p in plans:
        p.close()


def test_queue_matches_the_plans_own_transforms_on_the_batched_workload_sizes():
    """The 200-field size mix at reduced counts: the executor's spectra equal (to rounding) what
    each plan computes on its own."""
    sizes = synth.batched_sizes(40, 200)
    groups = sorted({n: sizes.count(n) for n in sizes}.items())
    plans = [afft.Plan((n, n, n), "r2c", "f32", batch=c) for n, c in groups]
    xs = [torch.empty(p.spatial_shape, dtype=torch.float32, device="cuda").uniform_(-1, 1) for p in plans]
    mine = [torch.empty(p.spectral_shape, dtype=torch.complex64, device="cuda") for p in plans]
    q = afft.Queue(plans)
    q.forward(xs, mine)
    ref = [p.forward(x) for p, x in zip(plans, xs)]
    back = [torch.empty_like(x) for x in xs]
    q.backward(ref, back)
    torch.cuda.synchronize()
    assert q.status() == 0
    for (n, c), a, b, x, y in zip(groups, mine, ref, xs, back):
        e = float(torch.linalg.vector_norm((a - b).to(torch.complex128)) / torch.linalg.vector_norm(b.to(torch.complex128)))
        report("queue vs plan forward %d^3 x %d" % (n, c), e)
        e = float(torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double()))
        report("queue backward of the plan's spectrum %d^3 x %d" % (n, c), e)
    q.close()
    for p in plans:
        p.close()


def test_queue_rejects_what_it_does_not_run():
    ok = afft.Plan((64, 64, 64), "r2c", "f32")
    for bad in (afft.Plan((64, 64, 64), "c2c", "f32"), afft.Plan((64, 64, 64), "r2c", "f64"),
                afft.Plan((64, 64, 72), "r2c", "f32"), afft.Plan((40, 64, 64), "r2c", "f32")):
        with pytest.raises(afft.AfftError) as e:
            afft.Queue([ok, bad])
        assert e.value.status == 9
        bad.close()
    ok.close()
