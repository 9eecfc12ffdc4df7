"""Parity of the batched form at the full size of the uneven-batch workload (256
convection-diffusion problems, sides 64..256, p 1..4) in the launch configuration that
bench.py times: all inputs packed in one device buffer, one persistent launch replayed
as a CUDA graph, the team size from the batch's work distribution.  The oracle checks a
sample of the outputs one by one (evenly spaced problems)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
from oracle import phipm_oracle as O
from paper_0907_4631_gb300 import phipm as pm

pytestmark = pytest.mark.gpu

SAMPLE = [0, 51, 102, 153, 204, 255]


@pytest.mark.parametrize("name,prec,bar", [("batched_convdiff_256", "f64pair", 1e-8),
                                            ("batched_convdiff_256_f32", "f32", 1e-5)])
def test_full_uneven_batch_sampled(name, prec, bar):
    probs = bench.make_batch(name)
    assert len(probs) == 256
    solver = pm.Phipm(prec)
    pk = bench.PackedBatch(probs)
    batch = solver.batch([p.t_end for p in probs], pk.ops, pk.bs, [p.tol for p in probs],
                         [p.symm for p in probs], outs=pk.outs)
    batch.run()
    batch.run()                      # the replayed graph gives the same answers
    torch.cuda.synchronize()
    assert all(s == pm.OK for s in batch.statuses())
    for i in SAMPLE:
        pr = probs[i]
        ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, pr.symm)
        u = pk.outs[i].cpu().numpy()
        assert np.linalg.norm(u - ref) <= bar * np.linalg.norm(ref), i
