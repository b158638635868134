"""GPU parity on launches shaped like the paper's applications (Circuit,
PENNANT, stencil, Cannon, SUMMA, PUMMA, Johnson/COSMA) at full size:
sampled ids against the oracle point by point, the histogram against a
PyTorch bincount of the ids, the halo total against the oracle's closed
form and the per-processor bytes summing to it."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2507_17087_gb300 import native as N
from paper_2507_17087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("w", W.application_shapes(), ids=lambda w: w["name"])
def test_application_launch_full_size(w):
    L, machine = w["L"], w["machine"]
    npts, P = math.prod(L), machine[0] * machine[1]
    ids = torch.empty(npts, dtype=torch.int32, device=DEV)
    hist = torch.empty(P, dtype=torch.int64, device=DEV)
    total = torch.empty(1, dtype=torch.int64, device=DEV)
    recv = torch.empty(P, dtype=torch.int64, device=DEV)
    N.map_launch(L, machine, w["chain"], w["dist"], ids=ids, hist=hist, face_bytes=w["face"], total=total,
                 recv=recv)
    torch.cuda.synchronize()
    ref = O.Launch(L, machine, w["chain"], w["dist"])
    g = torch.Generator().manual_seed(3)
    lins = torch.randint(0, npts, (50000,), generator=g).numpy().astype(np.int64)
    lins = np.concatenate([lins, np.arange(0, 2048), np.arange(npts - 2048, npts)])
    got = ids[torch.from_numpy(lins).to(DEV)].cpu().numpy()
    assert np.array_equal(got, ref.owner_of(lins))
    assert torch.equal(torch.bincount(ids.long(), minlength=P), hist)
    assert int(total.item()) == ref.halo_closed_form(w["face"])
    assert int(recv.sum().item()) == int(total.item())
    del ids
    torch.cuda.empty_cache()
