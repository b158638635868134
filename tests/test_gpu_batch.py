"""GPU parity of the batched, graph-captured mapping path.

Every query of a batch must produce exactly what the oracle gives: ids,
histogram, halo total and per-processor received bytes -- for the whole
10,000-query batch the benchmark runs, every query in full.
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
from paper_2507_17087_gb300 import native as N
from paper_2507_17087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def batch_outputs(b):
    info = b.info()
    ids = torch.full((max(1, int(info["total_ids"])),), -9, dtype=torch.int32, device=DEV)
    hist = torch.full((int(info["total_procs"]),), -9, dtype=torch.int64, device=DEV)
    recv = torch.full((int(info["total_procs"]),), -9, dtype=torch.int64, device=DEV)
    halo = torch.full((b.n,), -9, dtype=torch.int64, device=DEV)
    return info, ids, hist, halo, recv


def launches_from(queries):
    out = []
    for q in queries:
        chain = N.chain_from_draws(*q["machine"], q["draws"])
        out.append((q["L"], q["machine"], chain, q["dist"], q["face"]))
    return out


def small_queries(count, seed):
    rng = W.rng(seed)
    res = []
    for _ in range(count):
        k = rng.randint(1, 4)
        L = [rng.randint(1, 30) for _ in range(k)]
        while math.prod(L) > 20000:
            L = [max(1, v // 2) for v in L]
        machine = (rng.randint(1, 40), rng.randint(1, 8))
        draws = [rng.next() for _ in range(rng.randint(0, 5))]
        kind = rng.choice(W.DIST_KINDS)
        dist = ("block_cyclic", rng.randint(1, 5)) if kind == "block_cyclic" else (kind,)
        face = [rng.randint(1, 64) for _ in range(k)]
        res.append({"L": tuple(L), "machine": machine, "draws": draws, "dist": dist, "face": face})
    return res


def check_query(info, ids, hist, halo, recv, q, launch, ref_ids, ref_hist, ref_tot, ref_recv):
    io, po = int(info["ids_offsets"][q]), int(info["proc_offsets"][q])
    npts = math.prod(launch[0])
    P = launch[1][0] * launch[1][1]
    assert np.array_equal(ids[io:io + npts], ref_ids), f"ids of query {q}: {launch}"
    assert np.array_equal(hist[po:po + P].astype(np.uint64), ref_hist)
    assert int(halo[q]) == ref_tot
    assert np.array_equal(recv[po:po + P].astype(np.uint64), ref_recv)


@pytest.mark.parametrize("graph", [True, False])
def test_small_batch_against_oracle(graph):
    launches = launches_from(small_queries(300, 4000))
    b = N.Batch(launches)
    info, ids, hist, halo, recv = batch_outputs(b)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv, graph=graph)
    torch.cuda.synchronize()
    ids, hist, halo, recv = (t.cpu().numpy() for t in (ids, hist, halo, recv))
    for q, launch in enumerate(launches):
        ref = O.Launch(*launch[:4])
        rids, rhist = ref.map_points(threads=8)
        rtot, rrecv = ref.comm_volume(launch[4], threads=8)
        check_query(info, ids, hist, halo, recv, q, launch, rids, rhist, rtot, rrecv)
    b.close()


def test_replay_autotune_and_pointer_change():
    launches = launches_from(small_queries(120, 4100))
    b = N.Batch(launches)
    info, ids, hist, halo, recv = batch_outputs(b)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv, autotune=True)
    first = [t.clone() for t in (ids, hist, halo, recv)]
    assert b.info()["tile_groups"] in (8192, 32768, 65536, 131072)
    for _ in range(3):   # graph replays
        b.run(ids=ids, hist=hist, halo=halo, recv=recv)
    torch.cuda.synchronize()
    for a, c in zip(first, (ids, hist, halo, recv)):
        assert torch.equal(a, c)
    _, ids2, hist2, halo2, recv2 = batch_outputs(b)   # new pointers: the graph is captured again
    b.run(ids=ids2, hist=hist2, halo=halo2, recv=recv2)
    torch.cuda.synchronize()
    for a, c in zip(first, (ids2, hist2, halo2, recv2)):
        assert torch.equal(a, c)
    # only some outputs
    hist3 = torch.zeros_like(hist)
    b.run(hist=hist3)
    torch.cuda.synchronize()
    assert torch.equal(hist3, hist)
    b.close()


def test_batched_recipe_against_single_launch_path():
    # the first 400 queries of the 10,000-query recipe (up to 2^24 points each)
    qs = W.batched_queries(count=400)
    launches = launches_from(qs)
    b = N.Batch(launches)
    info, ids, hist, halo, recv = batch_outputs(b)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv, autotune=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for q in list(range(40)) + list(rng.integers(40, 400, 40)):
        L, machine, chain, dist, face = launches[q]
        npts, P = math.prod(L), machine[0] * machine[1]
        rid = torch.empty(npts, dtype=torch.int32, device=DEV)
        rh = torch.empty(P, dtype=torch.int64, device=DEV)
        rt = torch.empty(1, dtype=torch.int64, device=DEV)
        rr = torch.empty(P, dtype=torch.int64, device=DEV)
        N.map_points(L, machine, chain, dist, ids=rid, hist=rh)
        N.comm_volume(L, machine, chain, dist, face, total=rt, recv=rr)
        io, po = int(info["ids_offsets"][q]), int(info["proc_offsets"][q])
        assert torch.equal(ids[io:io + npts], rid), (q, L, machine, chain, dist)
        assert torch.equal(hist[po:po + P], rh)
        assert torch.equal(recv[po:po + P], rr)
        assert int(halo[q].item()) == int(rt.item())
        # and a sample of ids against the oracle, point by point
        lins = rng.integers(0, npts, 200).astype(np.int64)
        ref = O.Launch(L, machine, chain, dist)
        assert np.array_equal(rid[torch.from_numpy(lins).to(DEV)].cpu().numpy(), ref.owner_of(lins))
    b.close()


# launch shapes that select each way a batched row finds its contributions:
# rows fused into a table (multiple of 4 points or not, short or long),
# two-level rows (a fused table under 128 points joined by the next
# dimension's table; inner tables of 1 to 3 points cross several boundaries
# within one 4-point group), rows computed in place (last extent above the
# fused limit, aligned or not, above the table limit), 16-byte table rows
ROW_SHAPES = [
    (3, 5000, 7), (2, 4097, 1), (5, 2500, 2), (7, 3000, 3), (4, 1100, 4), (9, 33, 127), (6, 40, 4500, 2),
    (3, 700, 100), (2, 3, 1500, 5), (11, 4097, 6), (40, 50, 60), (7, 2049), (13, 4093), (3, 66000),
    (5, 40000), (2, 70001), (9, 8192), (4, 12, 5000), (2, 2, 2, 9001),
]


def test_row_shapes_against_oracle():
    rng = W.rng(4300)
    launches = []
    for L in ROW_SHAPES:
        for kind in W.DIST_KINDS:
            machine = (rng.randint(1, 24), rng.randint(1, 8))
            draws = [rng.next() for _ in range(rng.randint(0, 5))]
            dist = ("block_cyclic", rng.randint(1, 7)) if kind == "block_cyclic" else (kind,)
            launches.append((L, machine, N.chain_from_draws(*machine, draws), dist, [8] * len(L)))
    b = N.Batch(launches)
    info, ids, hist, halo, recv = batch_outputs(b)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv, autotune=True)
    torch.cuda.synchronize()
    ids, hist, halo, recv = (t.cpu().numpy() for t in (ids, hist, halo, recv))
    for q, launch in enumerate(launches):
        ref = O.Launch(*launch[:4])
        rids, rhist = ref.map_points(threads=8)
        rtot, rrecv = ref.comm_volume(launch[4], threads=8)
        check_query(info, ids, hist, halo, recv, q, launch, rids, rhist, rtot, rrecv)
    b.close()


def test_batch_rejects_invalid_queries():
    with pytest.raises(N.MapleError):
        N.Batch([((4, 4), (2, 2), [("split", 0, 3)], ("block",), (1, 1))])
    with pytest.raises(N.MapleError):
        N.Batch([((4, 4), (1 << 15, 1), [], ("block",), (1, 1))])   # P > 16384


def test_full_10000_query_batch_every_query():
    # the whole 10,000-query batch as the benchmark runs it (1.2e10 points,
    # 49 GB of ids, autotuned, graph replay), every query against the oracle:
    # all of its ids, its histogram, its halo total and its received bytes
    # (the oracle evaluates each point's owner once and looks each
    # neighbour's owner up in its own ids; the queries run on all host cores)
    qs = W.batched_queries(10000)
    launches = launches_from(qs)
    b = N.Batch(launches)
    info, ids, hist, halo, recv = batch_outputs(b)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv, autotune=True)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv)
    torch.cuda.synchronize()
    io = np.asarray(info["ids_offsets"], dtype=np.int64)
    po = np.asarray(info["proc_offsets"], dtype=np.int64)
    hist, halo, recv = (t.cpu().numpy() for t in (hist, halo, recv))
    npts = [math.prod(q["L"]) for q in qs]

    def check(q, host_ids, base):
        L, machine, chain, dist, face = launches[q]
        assert chain == O.chain_from_draws(*machine, qs[q]["draws"])
        rids, rhist, rtot, rrecv = O.Launch(L, machine, chain, dist).map_launch(face, threads=1)
        P = machine[0] * machine[1]
        lo = int(io[q]) - base
        assert np.array_equal(host_ids[lo:lo + npts[q]], rids), (q, L, machine, chain, dist)
        assert np.array_equal(hist[po[q]:po[q] + P].astype(np.uint64), rhist), q
        assert int(halo[q]) == rtot, q
        assert np.array_equal(recv[po[q]:po[q] + P].astype(np.uint64), rrecv), q
        return npts[q]

    checked = 0
    with ThreadPoolExecutor(os.cpu_count() or 8) as pool:
        q = 0
        while q < len(qs):
            # consecutive queries holding about 2^28 ids, copied to the host together
            q1 = q
            while q1 < len(qs) and (q1 == q or int(io[q1]) + npts[q1] - int(io[q]) <= 1 << 28):
                q1 += 1
            base, end = int(io[q]), int(io[q1 - 1]) + npts[q1 - 1]
            host_ids = ids[base:end].cpu().numpy()
            checked += sum(pool.map(lambda j: check(j, host_ids, base), range(q, q1)))
            q = q1
    assert checked == sum(npts)
    b.close()
    del ids
    torch.cuda.empty_cache()
