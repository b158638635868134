"""GPU parity of decompose_search and candidate_costs against the CPU oracle.

The exhaustive argmin (index, primary, secondary) must equal the oracle's
exhaustive search exactly, with and without the primary-bound dismissal, on
small queries and on every full-size 3-D matmul query (P up to 4096, up to
3.79 M candidates); a sample of 10^5 candidates per full-size query checks
the engine's own per-candidate costs.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2507_17087_gb300 import native as N
from paper_2507_17087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = 512 * 512 * 4
CORES = os.cpu_count() or 8


def oracle_best(q, threads=16):
    M, N_, K = q["MNK"]
    return O.search(M, N_, K, q["machine"], q["max_depth"], threads=threads)


@pytest.mark.parametrize("full", [False, True])
def test_small_queries_exhaustive(full):
    for q in W.search_query_small(count=24):
        got = N.decompose_search([q], full=full)[0]
        ref = oracle_best(q)
        assert got["index"] == ref["index"], (q, got, ref)
        assert got["primary_bytes"] == ref["primary"] * TILE
        assert got["secondary_bytes"] == ref["secondary"] * TILE
        assert got["n_candidates"] == ref["n_candidates"]
        assert got["f"] == ref["f"]


def test_worked_shapes():
    # (4,8,4) on 16 processors.  Among factorisations with f <= (M,N,K) the
    # least primary cost is decompose's (2,4,2) (Fig. 10); the moved-tile cost
    # has no load-balance term, so (1,1,16) -- four idle processor rows along
    # K -- moves fewer tiles (96 < 112) and wins the unrestricted search.
    q = {"MNK": (4, 8, 4), "machine": (2, 8), "max_depth": 2, "tile_bytes": TILE}
    got = N.decompose_search([q])[0]
    ref = oracle_best(q)
    assert (got["index"], got["f"]) == (ref["index"], ref["f"]) and got["f"] == (1, 1, 16)
    assert got["primary_bytes"] == 96 * TILE
    assert O.matmul_cost(4, 8, 4, (2, 8), (), (2, 4, 2))[0] == 112
    fits = [f for f in O.factorisations(16, 3) if all(a <= b for a, b in zip(f, (4, 8, 4)))]
    assert min(fits, key=lambda f: (O.matmul_cost(4, 8, 4, (2, 8), (), f)[0], f)) == (2, 4, 2)
    # the plain 64x64 case as a degenerate 3-D grid (K = 1): 8 processors
    q = {"MNK": (64, 64, 1), "machine": (2, 4), "max_depth": 1, "tile_bytes": TILE}
    assert N.decompose_search([q])[0]["index"] == oracle_best(q)["index"]


def test_search_kernel_paths():
    # shapes that take the search kernels' special paths, exhaustively against
    # the oracle, with and without the primary bound: extents below their
    # factors (blocks holding one tile or none), uneven blocks (A or A + 1
    # tiles), families with fewer than 32 long fibres, precounted families
    # read by fibre number
    shapes = [((5, 1000, 7), (90, 8)), ((250, 333, 97), (45, 16)), ((3, 3, 3), (64, 1)),
              ((1000, 2, 1000), (30, 24)), ((64, 4096, 2), (8, 8))]
    for MNK, machine in shapes:
        q = {"MNK": MNK, "machine": machine, "max_depth": 3, "tile_bytes": TILE}
        ref = oracle_best(q, threads=CORES)
        for full in (False, True):
            got = N.decompose_search([q], full=full)[0]
            assert (got["index"], got["f"]) == (ref["index"], ref["f"]), (q, full, got, ref)
            assert got["primary_bytes"] == ref["primary"] * TILE
            assert got["secondary_bytes"] == ref["secondary"] * TILE


@pytest.mark.parametrize("qi", range(8))
def test_matmul_queries_full_size(qi):
    # every full-size query (P = 512, 2520, 3600, 4096; up to 3.79 M
    # candidates) against the oracle's exhaustive search over all host
    # cores, with and without the primary bound; then 10^5 random candidates:
    # the engine's own costs equal the oracle's and none beats the winner
    q = W.search_queries(8)[qi]
    M, N_, K = q["MNK"]
    n, g = q["machine"]
    P = n * g
    got = N.decompose_search([q])[0]
    full = N.decompose_search([q], full=True)[0]
    nf, nc = N.search_space(P, g, q["max_depth"])
    assert got["n_candidates"] == nf * nc == len(O.factorisations(P, 3)) * len(O.chains(n, g, 3))
    ref = oracle_best(q, threads=CORES)
    want = (ref["index"], ref["primary"] * TILE, ref["secondary"] * TILE, ref["n_candidates"])
    for r in (got, full):
        assert (r["index"], r["primary_bytes"], r["secondary_bytes"], r["n_candidates"]) == want
        assert r["f"] == ref["f"]
    rng = np.random.default_rng(qi)
    sample = rng.integers(0, got["n_candidates"], 100000, dtype=np.int64)
    sp, ss = O.candidate_costs(M, N_, K, q["machine"], 3, sample, threads=CORES)
    key = (ref["primary"], ref["secondary"], ref["index"])
    assert min(zip(sp.tolist(), ss.tolist(), sample.tolist())) >= key
    gp = np.zeros(len(sample), dtype=np.uint64)
    gs = np.zeros(len(sample), dtype=np.uint64)
    N.candidate_costs(q, sample, gp, gs)
    assert np.array_equal(gp, sp.astype(np.uint64) * TILE)
    assert np.array_equal(gs, ss.astype(np.uint64) * TILE)


def test_candidate_costs_device_buffers_and_out_of_range():
    q = W.search_query_small(count=1)[0]
    nf, nc = N.search_space(q["machine"][0] * q["machine"][1], q["machine"][1], q["max_depth"])
    idx = torch.tensor([0, nf * nc - 1, 5 % (nf * nc), nf * nc, -1], dtype=torch.int64, device="cuda")
    p = torch.zeros(5, dtype=torch.int64, device="cuda")
    s = torch.zeros(5, dtype=torch.int64, device="cuda")
    N.candidate_costs(q, idx, p, s)
    torch.cuda.synchronize()
    M, N_, K = q["MNK"]
    rp, rs = O.candidate_costs(M, N_, K, q["machine"], q["max_depth"], idx[:3].cpu().numpy())
    assert p[:3].cpu().numpy().tolist() == (rp * TILE).tolist()
    assert s[:3].cpu().numpy().tolist() == (rs * TILE).tolist()
    # out-of-range indices are flagged, not evaluated
    assert p[3:].cpu().numpy().astype(np.uint64).tolist() == [2 ** 64 - 1] * 2
    with pytest.raises(N.MapleError):
        N.candidate_costs(q, np.array([nf * nc], dtype=np.int64), np.zeros(1, np.uint64), np.zeros(1, np.uint64))


def test_space_cache_eviction_and_reuse():
    # more distinct candidate spaces (P, g, depth) than the device cache
    # keeps, each searched twice in a row and again after it was evicted,
    # with and without the primary bound: every answer equals the oracle's
    shapes = [((n, g), d) for (n, g) in ((2, 2), (3, 2), (4, 2), (6, 1), (5, 2), (3, 4), (7, 1), (2, 8), (9, 2), (4, 4))
              for d in (2,)]
    queries = [{"MNK": (16, 8, 64), "machine": m, "max_depth": d, "tile_bytes": TILE} for m, d in shapes]
    refs = [oracle_best(q) for q in queries]
    for rnd in range(2):
        for q, ref in zip(queries, refs):
            for full in (False, True):
                got = N.decompose_search([q], full=full)[0]
                assert (got["index"], got["secondary_bytes"]) == (ref["index"], ref["secondary"] * TILE), (rnd, q)
    # listed candidates through the cached tables, against the oracle's costs
    q = queries[0]
    nf, nc = N.search_space(q["machine"][0] * q["machine"][1], q["machine"][1], q["max_depth"])
    idx = np.arange(nf * nc, dtype=np.int64)
    p = np.zeros(nf * nc, dtype=np.uint64)
    s = np.zeros(nf * nc, dtype=np.uint64)
    N.candidate_costs(q, idx, p, s)
    rp, rs = O.candidate_costs(*q["MNK"], q["machine"], q["max_depth"], idx)
    assert np.array_equal(p, rp.astype(np.uint64) * TILE) and np.array_equal(s, rs.astype(np.uint64) * TILE)
