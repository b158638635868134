"""GPU parity of mp_halo_volume (per-dimension halo widths) against the CPU
oracle.

The element count is an integer; totals and per-processor received bytes must
match the oracle bit-exactly on seeded launches of every distribution kind.
At the 1024x1024x512 size the block variant is checked against the
appendix's closed form and the cyclic variants against a plain PyTorch
recount from the id array (itself checked point by point against the oracle
in tests/test_gpu_map.py).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2507_17087_gb300 import native as N
from paper_2507_17087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"
THREADS = 8


def gpu_halo(L, machine, chain, dist, width, eb, elements=True):
    P = machine[0] * machine[1]
    total = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    recv = torch.full((P,), -7, dtype=torch.int64, device=DEV)
    N.halo_volume(L, machine, chain, dist, width, eb, total=total, recv=recv, elements=elements)
    torch.cuda.synchronize()
    return int(total.item()), recv.cpu().numpy()


def check(L, machine, chain, dist, width, eb):
    tot, recv = gpu_halo(L, machine, chain, dist, width, eb)
    ref = O.Launch(L, machine, chain, dist)
    rtot, rrecv = ref.halo_elements(width, eb, threads=THREADS)
    assert tot == rtot, (L, machine, chain, dist, width)
    assert np.array_equal(recv.astype(np.uint64), rrecv), (L, machine, chain, dist, width)


def random_case(rng, max_points, max_width):
    k = rng.randint(1, 4)
    L = [rng.randint(1, 40) for _ in range(k)]
    while math.prod(L) > max_points:
        L = [max(1, v // 2) for v in L]
    machine = (rng.randint(1, 24), rng.randint(1, 8))
    draws = [rng.next() for _ in range(rng.randint(0, 5))]
    chain = N.chain_from_draws(machine[0], machine[1], draws)
    kind = rng.choice(W.DIST_KINDS)
    dist = ("block_cyclic", rng.randint(1, 5)) if kind == "block_cyclic" else (kind,)
    width = [rng.randint(0, max_width) for _ in range(k)]
    eb = [rng.randint(1, 64) for _ in range(k)]
    return tuple(L), machine, chain, dist, width, eb


@pytest.mark.parametrize("seed", range(8))
def test_random_launches_bit_exact(seed):
    rng = W.rng(700 + seed)
    for _ in range(20):
        check(*random_case(rng, 20000, 6))


@pytest.mark.parametrize("kind", ["block", "cyclic", "block_cyclic", "hier", "linear_cyclic"])
def test_widest_halos_and_small_machines(kind):
    # widths up to the limit on machines with few processors per dimension:
    # the dilated runs overlap, wrap residues and reach past the launch
    rng = W.rng(760)
    for L, machine in (((300,), (1, 3)), ((37, 41), (2, 2)), ((17, 5, 23), (3, 2)), ((16,), (4, 4))):
        for _ in range(3):
            cfg = W.scaled_launch(L, machine, kind, rng.randint(0, 10 ** 6))
            chain = N.chain_from_draws(*machine, cfg["draws"])
            width = [rng.randint(0, N.MAX_HALO_WIDTH) for _ in L]
            check(L, machine, chain, cfg["dist"], width, [3] * len(L))


def test_width_one_block_equals_faces_and_zero_width_is_zero():
    cfg = W.scaled_launch((33, 47, 9), (4, 4), "block", 3)
    chain = N.chain_from_draws(4, 4, cfg["draws"])
    e, re_ = gpu_halo(cfg["L"], (4, 4), chain, cfg["dist"], (1, 1, 1), (8, 8, 8))
    f, rf = gpu_halo(cfg["L"], (4, 4), chain, cfg["dist"], (1, 1, 1), (8, 8, 8), elements=False)
    assert e == f and np.array_equal(re_, rf)
    z, rz = gpu_halo(cfg["L"], (4, 4), chain, cfg["dist"], (0, 0, 0), (8, 8, 8))
    assert z == 0 and not rz.any()


def test_invalid_widths_rejected():
    L, machine = (8, 8), (2, 2)
    total = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    for width in ((17, 1), (-1, 1)):
        with pytest.raises(N.MapleError):
            N.halo_volume(L, machine, [], ("block",), width, (1, 1), total=total)
    torch.cuda.synchronize()
    assert int(total.item()) == -7


def _recount(ids_view, width, eb, P):
    """Plain PyTorch: per element and dimension, the distinct other owners
    within the halo width, in chunks of the first dimension."""
    L = tuple(ids_view.shape)
    total = 0
    recv = torch.zeros(P, dtype=torch.int64, device=DEV)
    for t in range(len(L)):
        w = width[t]
        if w == 0:
            continue
        u = 1 if t == 0 else 0
        step = 64
        for c0 in range(0, L[u], step):
            c1 = min(L[u], c0 + step)
            a = ids_view.narrow(u, c0, c1 - c0)
            nb = []
            for dlt in list(range(-w, 0)) + list(range(1, w + 1)):
                sh = torch.full_like(a, -1)
                if abs(dlt) < L[t]:
                    n = L[t] - abs(dlt)
                    src = a.narrow(t, max(dlt, 0), n)
                    sh.narrow(t, max(-dlt, 0), n).copy_(src)
                sh[sh == a] = -1
                nb.append(sh)
            s, _ = torch.sort(torch.stack(nb), dim=0)
            first = s >= 0
            first[1:] &= s[1:] != s[:-1]
            got = s[first].long()
            total += eb[t] * got.numel()
            recv += eb[t] * torch.bincount(got, minlength=P)
            del nb, s, first, got
    return total, recv


@pytest.mark.parametrize("variant", ["block", "cyclic", "block_cyclic"])
def test_full_size_1024x1024x512(variant):
    cfg = W.large_config(variant)
    L, machine = cfg["L"], cfg["machine"]
    chain = N.chain_from_draws(*machine, cfg["draws"])
    P = machine[0] * machine[1]
    width, eb = (2, 1, 3), (8, 8, 8)
    total = torch.empty(1, dtype=torch.int64, device=DEV)
    recv = torch.empty(P, dtype=torch.int64, device=DEV)
    N.halo_volume(L, machine, chain, cfg["dist"], width, eb, total=total, recv=recv)
    torch.cuda.synchronize()
    if variant == "block":
        # the appendix's volume on a grid that divides the extents, interior
        # cuts only: sum_t 2 (s_t - 1) h_t prod_{u != t} L_u
        s, _ = N.plan(L, machine, chain, cfg["dist"])
        want = sum(2 * (s[t] - 1) * width[t] * eb[t] * math.prod(L[u] for u in range(3) if u != t)
                   for t in range(3))
        assert int(total.item()) == want
        assert int(recv.sum().item()) == want
    else:
        ids = torch.empty(math.prod(L), dtype=torch.int32, device=DEV)
        N.map_points(L, machine, chain, cfg["dist"], ids=ids)
        tot, rc = _recount(ids.view(*L), width, eb, P)
        assert int(total.item()) == tot
        assert torch.equal(recv, rc)


def test_mid_size_linear_cyclic_against_oracle():
    for q, machine in ((1, (6, 4)), (2, (8, 8))):
        cfg = W.scaled_launch((64, 48, 40), machine, "linear_cyclic", 500 + q)
        chain = N.chain_from_draws(*machine, cfg["draws"])
        check(cfg["L"], machine, chain, cfg["dist"], (3, 0, 5), (4, 8, 16))


def test_decompose_vs_greedy_study_grid():
    # the 180-configuration stencil grid of the paper's decompose study: the
    # engine's halo volume of both grids against the oracle's closed form
    total = torch.empty(1, dtype=torch.int64, device=DEV)
    for c in W.stencil_study_configs():
        g = N.greedy_grid(c["gpus"], 2)
        assert g == O.greedy(c["gpus"], 2)
        for chain in ([("merge", 0, 1), ("split", 0, g[0])], [("merge", 0, 1), ("decompose", 0, c["L"])]):
            N.halo_volume(c["L"], c["machine"], chain, ("block",), (1, 1), (8, 8), total=total)
            ref = O.Launch(c["L"], c["machine"], chain, ("block",)).halo_closed_form((8, 8))
            assert int(total.item()) == ref, (c["name"], chain)
