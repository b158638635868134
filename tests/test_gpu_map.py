"""GPU parity of map_points / comm_volume against the CPU oracle.

Every case runs the CUDA engine through the C ABI and compares, element by
element, with the oracle on the same seeded launch: ids and histograms are
integers and must match bit-exactly; so must the halo totals and the
per-processor received bytes.  At the 1024x1024x512 size the call the
benchmark times is compared with the oracle in full: every id, the whole
histogram, the halo total and the received bytes of every processor.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2507_17087_gb300 import native as N
from paper_2507_17087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"
THREADS = 8
CORES = os.cpu_count() or 8


def gpu_run(L, machine, chain, dist, face):
    P = machine[0] * machine[1]
    npts = math.prod(L)
    ids = torch.full((npts,), -7, dtype=torch.int32, device=DEV)
    hist = torch.full((P,), -7, dtype=torch.int64, device=DEV)
    total = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    recv = torch.full((P,), -7, dtype=torch.int64, device=DEV)
    N.map_points(L, machine, chain, dist, ids=ids, hist=hist)
    N.comm_volume(L, machine, chain, dist, face, total=total, recv=recv)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), hist.cpu().numpy(), int(total.item()), recv.cpu().numpy()


def check_against_oracle(L, machine, chain, dist, face):
    ids, hist, total, recv = gpu_run(L, machine, chain, dist, face)
    ref = O.Launch(L, machine, chain, dist)
    rids, rhist = ref.map_points(threads=THREADS)
    rtot, rrecv = ref.comm_volume(face, threads=THREADS)
    assert np.array_equal(ids, rids), f"ids differ for {L} {machine} {chain} {dist}"
    assert np.array_equal(hist.astype(np.uint64), rhist)
    assert total == rtot
    assert np.array_equal(recv.astype(np.uint64), rrecv)


def random_launch(rng, max_points):
    k = rng.randint(1, 4)
    L = [rng.randint(1, 40) for _ in range(k)]
    while math.prod(L) > max_points:
        L = [max(1, v // 2) for v in L]
    machine = (rng.randint(1, 40), rng.randint(1, 8))
    draws = [rng.next() for _ in range(rng.randint(0, 5))]
    chain = N.chain_from_draws(machine[0], machine[1], draws)
    kind = rng.choice(W.DIST_KINDS)
    dist = ("block_cyclic", rng.randint(1, 5)) if kind == "block_cyclic" else (kind,)
    face = [rng.randint(1, 100) for _ in range(k)]
    return tuple(L), machine, chain, dist, face


@pytest.mark.parametrize("seed", range(12))
def test_random_launches_bit_exact(seed):
    rng = W.rng(100 + seed)
    for _ in range(25):
        check_against_oracle(*random_launch(rng, 30000))


def test_plain_64x64_on_2x4():
    cfg = W.plain_config()
    check_against_oracle(cfg["L"], cfg["machine"], cfg["chain"], cfg["dist"], cfg["face"])
    _, _, total, _ = gpu_run(cfg["L"], cfg["machine"], cfg["chain"], cfg["dist"], cfg["face"])
    assert total == 1048576


@pytest.mark.parametrize("variant", ["block", "cyclic", "block_cyclic", "hier", "linear_cyclic"])
def test_scaled_large_recipe(variant):
    # the large-launch recipe (random depth-4 chain) at sizes spanning many
    # tiles with ragged tails
    for q, L in enumerate([(37, 41, 29), (64, 33, 130), (5, 7, 3001), (2, 3, 1, 4099)]):
        cfg = W.scaled_launch(L, (64, 8), variant, 300 + q)
        chain = N.chain_from_draws(64, 8, cfg["draws"])
        assert chain == O.chain_from_draws(64, 8, cfg["draws"])
        check_against_oracle(cfg["L"], cfg["machine"], chain, cfg["dist"], cfg["face"])


@pytest.mark.parametrize("L", [(1,), (3,), (5, 1), (1, 1, 1, 1), (7, 3), (2, 2, 2, 3), (4099,), (3, 8191)])
def test_ragged_and_degenerate_shapes(L):
    for dist in [("block",), ("cyclic",), ("block_cyclic", 3), ("hier",), ("linear_cyclic",)]:
        for machine in [(1, 1), (3, 5), (16, 8)]:
            check_against_oracle(L, machine, [], dist, [3] * len(L))


def test_explicit_chains():
    cases = [
        ((12, 18), (3, 2), [], ("block",)),
        ((18, 12), (2, 3), [("swap", 0, 1)], ("block",)),
        ((64, 64), (2, 4), [("merge", 0, 1), ("decompose", 0, (64, 64))], ("block",)),
        ((8, 8), (4, 4), [("decompose", 0, (8, 8)), ("decompose", 2, (4, 4))], ("hier",)),
        ((4, 4, 4), (2, 4), [("split", 0, 2), ("split", 1, 1), ("split", 3, 1), ("split", 4, 2)], ("hier",)),
        ((17, 5), (3, 4), [("merge", 0, 1), ("split", 0, 12)], ("block",)),
        ((30, 20, 10), (6, 4), [("balance_split", 1, 2), ("merge", 0, 2)], ("cyclic",)),
        ((9, 9), (6, 6), [("split", 0, 3), ("merge", 1, 2), ("swap", 0, 1), ("merge", 0, 1)], ("linear_cyclic",)),
    ]
    for L, machine, chain, dist in cases:
        check_against_oracle(L, machine, chain, dist, [5] * len(L))


def test_large_processor_count_uses_global_tables():
    # P > 16384 keeps T in HBM/L2 instead of shared memory
    for dist in [("block",), ("cyclic",), ("linear_cyclic",), ("hier",)]:
        check_against_oracle((130, 257), (4096, 8), [("swap", 0, 1)], dist, [8, 8])


def test_long_fastest_dimension_paths():
    # c_last from the HBM table (8192 < L_last <= 2^22) and computed (> 2^22)
    for L in [(3, 20011), ((1 << 22) + 5,)]:
        for dist in [("block",), ("cyclic",), ("block_cyclic", 7)]:
            check_against_oracle(L, (5, 3), [("swap", 0, 1)], dist, [2] * len(L))


def test_host_buffers_and_unaligned_device_buffers():
    L, machine, chain, dist, face = (33, 65), (6, 4), [("merge", 0, 1)], ("block_cyclic", 2), [4, 4]
    ref = O.Launch(L, machine, chain, dist)
    rids, rhist = ref.map_points()
    rtot, rrecv = ref.comm_volume(face)
    ids = np.zeros(math.prod(L), dtype=np.int32)
    hist = np.zeros(24, dtype=np.uint64)
    N.map_points(L, machine, chain, dist, ids=ids, hist=hist)
    assert np.array_equal(ids, rids) and np.array_equal(hist, rhist)
    total = np.zeros(1, dtype=np.uint64)
    recv = np.zeros(24, dtype=np.uint64)
    N.comm_volume(L, machine, chain, dist, face, total=total, recv=recv)
    assert int(total[0]) == rtot and np.array_equal(recv, rrecv)
    pinned = torch.zeros(math.prod(L), dtype=torch.int32).pin_memory()
    N.map_points(L, machine, chain, dist, ids=pinned)
    assert np.array_equal(pinned.numpy(), rids)
    # device pointer offset by one element: not 16-byte aligned
    big = torch.zeros(math.prod(L) + 1, dtype=torch.int32, device=DEV)
    N.map_points(L, machine, chain, dist, ids=big[1:])
    assert np.array_equal(big[1:].cpu().numpy(), rids)


def test_invalid_arguments_write_nothing():
    ids = torch.full((16,), -3, dtype=torch.int32, device=DEV)
    bad = [
        ((0, 4), (2, 2), [], ("block",)),
        ((4, 4), (2, 2), [("split", 0, 3)], ("block",)),
        ((4, 4), (2, 2), [("merge", 1, 0)], ("block",)),
        ((4, 4), (2, 2), [("swap", 0, 0)], ("block",)),
        ((4, 4), (2, 2), [], ("block_cyclic", 0)),
        ((4, 4), (0, 2), [], ("block",)),
    ]
    for L, machine, chain, dist in bad:
        with pytest.raises(N.MapleError) as e:
            N.map_points(L, machine, chain, dist, ids=ids)
        assert e.value.status == 1
    assert (ids == -3).all()


@pytest.mark.parametrize("variant", ["block", "cyclic", "block_cyclic"])
def test_full_size_1024x1024x512(variant):
    # the call the benchmark times (ids, histogram, halo total and received
    # bytes in one map_launch, on the current stream) at full size, compared
    # element by element with the oracle: all 2^29 ids, the whole histogram,
    # the halo total and every processor's received bytes, the neighbour's
    # owner evaluated independently for every directed pair
    cfg = W.large_config(variant)
    L, machine, face = cfg["L"], cfg["machine"], cfg["face"]
    chain = N.chain_from_draws(*machine, cfg["draws"])
    assert chain == O.chain_from_draws(*machine, cfg["draws"])
    P = machine[0] * machine[1]
    npts = math.prod(L)
    ids = torch.full((npts,), -7, dtype=torch.int32, device=DEV)
    hist = torch.full((P,), -7, dtype=torch.int64, device=DEV)
    total = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    recv = torch.full((P,), -7, dtype=torch.int64, device=DEV)
    N.map_launch(L, machine, chain, cfg["dist"], ids=ids, hist=hist, face_bytes=face, total=total, recv=recv,
                 stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    got_ids = ids.cpu().numpy()
    got_hist, got_total, got_recv = hist.cpu().numpy(), int(total.item()), recv.cpu().numpy()
    del ids
    torch.cuda.empty_cache()
    ref = O.Launch(L, machine, chain, cfg["dist"])
    rids, rhist = ref.map_points(threads=CORES)
    assert np.array_equal(got_ids, rids)
    del rids, got_ids
    assert np.array_equal(got_hist.astype(np.uint64), rhist)
    rtot, rrecv = ref.comm_volume(face, threads=CORES)
    assert got_total == rtot == ref.halo_closed_form(face)
    assert np.array_equal(got_recv.astype(np.uint64), rrecv)


def test_extent_limit():
    # an extent of 2^38 or more is MP_ENOTSUP (the distributions' products
    # x * s must stay below 2^64); nothing is written
    hist = torch.full((6,), -3, dtype=torch.int64, device=DEV)
    for L in [(1 << 38,), (2, 1 << 40)]:
        with pytest.raises(N.MapleError) as e:
            N.map_points(L, (2, 3), [], ("block",), hist=hist)
        assert e.value.status == 6
    assert (hist == -3).all()
    # just below the limit, without ids: only the closed-form per-dimension
    # counts run.  Histogram: every final index a owns prod_t H_t(a_t)
    # points, H(a) = ceil((a+1) L / s) - ceil(a L / s) for block and
    # floor((L - 1 - a) / s) + 1 for cyclic; halo total: the oracle's closed
    # form; received bytes sum to it
    for L, machine, dist in [(((1 << 38) - 1,), (2, 3), ("block",)), (((1 << 38) - 3,), (5, 1), ("cyclic",)),
                             ((3, (1 << 38) - 5), (2, 4), ("block",)), ((7, (1 << 38) - 1), (3, 2), ("cyclic",))]:
        P = machine[0] * machine[1]
        face = [8] * len(L)
        hist = torch.full((P,), -3, dtype=torch.int64, device=DEV)
        total = torch.full((1,), -3, dtype=torch.int64, device=DEV)
        recv = torch.full((P,), -3, dtype=torch.int64, device=DEV)
        N.map_launch(L, machine, [], dist, hist=hist, face_bytes=face, total=total, recv=recv)
        torch.cuda.synchronize()
        ref = O.Launch(L, machine, [], dist)
        shape = ref.final_shape()
        a = np.array(list(itertools.product(*[range(v) for v in shape])), dtype=np.int64)
        node, proc = ref.resolve(a)
        want = np.zeros(P, dtype=np.int64)
        for row, nd, pr in zip(a, node, proc):
            cnt = 1
            for t, at in enumerate(row):
                if dist[0] == "block":
                    cnt *= -(-(int(at) + 1) * L[t] // shape[t]) - -(-int(at) * L[t] // shape[t])
                else:
                    cnt *= (L[t] - 1 - int(at)) // shape[t] + 1
            want[nd * machine[1] + pr] = cnt
        assert hist.cpu().numpy().tolist() == want.tolist(), (L, dist)
        assert int(total.item()) == ref.halo_closed_form(face), (L, dist)
        assert int(recv.sum().item()) == int(total.item())


def test_wide_index_launch_sampled():
    # more than 2^32 points: 64-bit point indexing
    L, machine = (65536, 65537), (7, 3)
    for dist in [("block",), ("linear_cyclic",)]:
        npts = math.prod(L)
        ids = torch.empty(npts, dtype=torch.int32, device=DEV)
        hist = torch.empty(21, dtype=torch.int64, device=DEV)
        N.map_points(L, machine, [("swap", 0, 1)], dist, ids=ids, hist=hist)
        torch.cuda.synchronize()
        ref = O.Launch(L, machine, [("swap", 0, 1)], dist)
        g = torch.Generator().manual_seed(3)
        lins = torch.randint(0, npts, (50000,), generator=g).numpy().astype(np.int64)
        lins = np.concatenate([lins, np.arange(npts - 1000, npts)])
        got = ids[torch.from_numpy(lins).to(DEV)].cpu().numpy()
        assert np.array_equal(got, ref.owner_of(lins))
        assert int(hist.sum().item()) == npts
        del ids
        torch.cuda.empty_cache()


def test_map_launch_equals_separate_calls():
    # one call for ids, histogram and halo gives what the separate calls give
    rng = W.rng(150)
    for _ in range(30):
        L, machine, chain, dist, face = random_launch(rng, 30000)
        P = machine[0] * machine[1]
        npts = math.prod(L)
        ids, rid = (torch.full((npts,), -7, dtype=torch.int32, device=DEV) for _ in range(2))
        hist, rh = (torch.full((P,), -7, dtype=torch.int64, device=DEV) for _ in range(2))
        tot, rt = (torch.full((1,), -7, dtype=torch.int64, device=DEV) for _ in range(2))
        recv, rr = (torch.full((P,), -7, dtype=torch.int64, device=DEV) for _ in range(2))
        N.map_launch(L, machine, chain, dist, ids=ids, hist=hist, face_bytes=face, total=tot, recv=recv)
        N.map_points(L, machine, chain, dist, ids=rid, hist=rh)
        N.comm_volume(L, machine, chain, dist, face, total=rt, recv=rr)
        width = [rng.randint(0, 4) for _ in L]
        et, er = (torch.full((1,), -7, dtype=torch.int64, device=DEV) for _ in range(2))
        e_recv, e_rr = (torch.full((P,), -7, dtype=torch.int64, device=DEV) for _ in range(2))
        N.map_launch(L, machine, chain, dist, face_bytes=face, total=et, recv=e_recv, width=width, elements=True)
        N.halo_volume(L, machine, chain, dist, width, face, total=er, recv=e_rr)
        torch.cuda.synchronize()
        for a, b in ((ids, rid), (hist, rh), (tot, rt), (recv, rr), (et, er), (e_recv, e_rr)):
            assert torch.equal(a, b), (L, machine, chain, dist)


@pytest.mark.parametrize("L,machine", [((300, 200, 2), (64, 8)), ((2, 9082, 7), (7, 8)), ((97, 2, 3, 171), (16, 4)),
                                       ((4096, 3), (1, 6)), ((5, 1, 4096), (3, 5)), ((65537,), (13, 1))])
def test_linear_cyclic_deficits_in_closed_form(L, machine):
    # the linear-cyclic face deficits are counted per residue run and, for the
    # last dimension, from a linear congruence: degenerate extents against the
    # oracle's per-neighbour count
    rng = W.rng(sum(L))
    chain = N.chain_from_draws(*machine, [rng.next() for _ in range(3)])
    face = [3 + t for t in range(len(L))]
    check_against_oracle(L, machine, chain, ("linear_cyclic",), face)


@pytest.mark.parametrize("kind", ["block", "linear_cyclic"])
def test_map_launch_captured_in_a_cuda_graph(kind):
    # the call's kernels run on two streams (the reductions beside the id
    # writer) and join before the call's work ends: captured into a caller's
    # CUDA graph and replayed, it gives what the eager call gives
    L, machine = (96, 40, 37), (6, 4)
    cfg = W.scaled_launch(L, machine, kind, 77)
    chain = N.chain_from_draws(*machine, cfg["draws"])
    P = machine[0] * machine[1]
    face = (8, 16, 4)

    def outputs():
        return (torch.full((math.prod(L),), -3, dtype=torch.int32, device="cuda"),
                torch.full((P,), -3, dtype=torch.int64, device="cuda"),
                torch.full((1,), -3, dtype=torch.int64, device="cuda"),
                torch.full((P,), -3, dtype=torch.int64, device="cuda"))

    want = outputs()
    N.map_launch(L, machine, chain, cfg["dist"], ids=want[0], hist=want[1], face_bytes=face, total=want[2],
                 recv=want[3])
    torch.cuda.synchronize()
    got = outputs()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):   # warm on the capture stream (workspace, second stream)
        N.map_launch(L, machine, chain, cfg["dist"], ids=got[0], hist=got[1], face_bytes=face, total=got[2],
                     recv=got[3], stream=s.cuda_stream)
    torch.cuda.synchronize()
    for t in got:
        t.fill_(-3)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        N.map_launch(L, machine, chain, cfg["dist"], ids=got[0], hist=got[1], face_bytes=face, total=got[2],
                     recv=got[3], stream=s.cuda_stream)
    for t in got:
        t.fill_(-3)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(want, got):
        assert torch.equal(a, b)
    # and the oracle agrees with the eager call
    ref = O.Launch(L, machine, chain, cfg["dist"])
    rids, rhist = ref.map_points(threads=8)
    assert np.array_equal(want[0].cpu().numpy(), rids)
    assert np.array_equal(want[1].cpu().numpy().astype(np.uint64), rhist)
