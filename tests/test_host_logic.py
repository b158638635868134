"""Host-side logic of the engine, on CPU (no kernel launches).

The C-ABI library loads without a GPU; its planner (validation, decompose
expansion, rank fix-up), random-chain builder and search-space enumeration
must agree with the oracle's independent implementations.
"""
import ctypes
import math
import os
import re

import pytest

import oracle as O
from paper_2507_17087_gb300 import native as N
from paper_2507_17087_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "mapple.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(N.library_path())
    names = declared_functions()
    assert "mp_map_points" in names and "mp_comm_volume" in names and "mp_decompose_search" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/mapple.h but not exported"


def test_status_strings():
    for code in range(7):
        assert N.strerror(code) and N.strerror(code) != "unknown status"


def _random_case(rng):
    k = rng.randint(1, 4)
    L = tuple(rng.randint(1, 50) for _ in range(k))
    machine = (rng.randint(1, 64), rng.randint(1, 8))
    draws = [rng.next() for _ in range(rng.randint(0, 5))]
    chain = O.chain_from_draws(*machine, draws)
    if rng.randint(0, 3) == 0:
        kk = rng.randint(1, 3)
        T = tuple(rng.randint(1, 30) for _ in range(kk))
        r = rng.randint(0, 3)
        if r == 0:     # the appendix's generalised objective: widths and transposes
            h = tuple(rng.randint(0, 6) for _ in range(kk))
            tr = tuple(m for m in range(kk) if rng.randint(0, 2) == 0)
            chain = chain + [("decompose", 0, T, h, tr)]
        else:
            chain = chain + [("decompose", 0, T)]
    if rng.randint(0, 5) == 0:
        chain = chain + [("balance_split", 0, rng.randint(1, 3))]
    kind = rng.choice(W.DIST_KINDS)
    dist = ("block_cyclic", rng.randint(1, 5)) if kind == "block_cyclic" else (kind,)
    return L, machine, chain, dist


def test_plan_matches_oracle_expansion():
    rng = W.rng(900)
    for _ in range(400):
        L, machine, chain, dist = _random_case(rng)
        shape, prims = N.plan(L, machine, chain, dist)
        ref = O.Launch(L, machine, chain, dist)
        assert shape == ref.final_shape()
        want = [(op, p, q if op != "split" else -1, d if op == "split" else 0) for op, p, q, d in ref.expand()]
        got = [(op, p, q if op != "split" else -1, d if op == "split" else 0) for op, p, q, d in prims]
        assert got == want


def test_chain_from_draws_matches_oracle():
    rng = W.rng(901)
    for _ in range(300):
        machine = (rng.randint(1, 300), rng.randint(1, 8))
        draws = [rng.next() for _ in range(rng.randint(0, 6))]
        assert N.chain_from_draws(*machine, draws) == O.chain_from_draws(*machine, draws)


@pytest.mark.parametrize("P,g,D", [(512, 8, 3), (2520, 8, 2), (4096, 8, 2), (3600, 8, 1), (16, 2, 3),
                                   (6, 3, 3), (1, 1, 2), (7, 7, 3)])
def test_search_space_matches_oracle(P, g, D):
    nf, nc = N.search_space(P, g, D)
    assert nf == len(O.factorisations(P, 3))
    assert nc == len(O.chains(P // g, g, D))


def test_search_candidate_decoding_matches_oracle_order():
    for P, g, D in [(16, 2, 3), (24, 4, 2), (512, 8, 2)]:
        q = N.make_query(8, 8, 8, P, g, D)
        fs = O.factorisations(P, 3)
        chains = O.chains(P // g, g, D)
        rng = W.rng(P)
        for _ in range(200):
            idx = rng.next() % (len(fs) * len(chains))
            f, chain = N.search_candidate(q, idx)
            assert f == fs[idx // len(chains)]
            assert chain == chains[idx % len(chains)]


def test_invalid_plans_rejected():
    cases = [
        (((0, 4), (2, 2), [], ("block",)), 1),
        (((4, 4), (2, 2), [("split", 0, 3)], ("block",)), 1),
        (((4, 4), (2, 2), [("split", 2, 1)], ("block",)), 1),
        (((4, 4), (2, 2), [("merge", 1, 0)], ("block",)), 1),
        (((4, 4), (2, 2), [("merge", 0, 2)], ("block",)), 1),
        (((4, 4), (2, 2), [("swap", 1, 1)], ("block",)), 1),
        (((4, 4), (2, 2), [("decompose", 0, (0, 2))], ("block",)), 1),
        (((4, 4), (2, 2), [("decompose", 0, (4, 2), (1, -1))], ("block",)), 1),
        (((4, 4), (2, 2), [("decompose", 0, (4, 2), None, (2,))], ("block",)), 1),
        (((4, 4), (2, 2), [("balance_split", 0, 5)], ("block",)), 1),
        (((4, 4), (2, 2), [], ("block_cyclic", 0)), 1),
        (((4, 4), (0, 2), [], ("block",)), 1),
        (((1 << 31, 1 << 31, 1 << 2), (2, 2), [], ("block",)), 2),
        (((1 << 39,), (2, 2), [], ("block",)), 6),
        (((4, 4), (1 << 20, 1 << 10), [], ("block",)), 6),
        (((1, 2, 3, 4, 5), (2, 2), [], ("block",)), 1),
    ]
    for (L, machine, chain, dist), want in cases:
        if len(L) > 4:
            sp = N.mp_space()
            sp.rank = 5
            mc, ds = N.make_machine(machine), N.make_dist(dist)
            rc = N.lib().mp_plan(ctypes.byref(sp), ctypes.byref(mc), None, 0, ctypes.byref(ds),
                                 None, None, None, None, 0)
        else:
            rc = N.plan_status(L, machine, chain, dist)
        assert rc == want, (L, machine, chain, dist, rc)


def test_invalid_search_queries_rejected():
    lib = N.lib()
    out = (N.mp_search_result * 1)()
    for q in [N.make_query(0, 4, 4, 8, 2), N.make_query(4, 4, 4, 9, 2), N.make_query(4, 4, 4, 8, 2, 5),
              N.make_query(4, 4, 4, 1 << 15, 8), N.make_query(1 << 21, 4, 4, 8, 2)]:
        arr = (N.mp_search_query * 1)(q)
        assert lib.mp_decompose_search(arr, 1, out, None) != 0


def test_weighted_decompose_matches_oracle():
    # the appendix's generalised objective, engine planner vs oracle
    rng = W.rng(905)
    for _ in range(300):
        k = rng.randint(1, 4)
        d = rng.choice((6, 12, 16, 24, 36, 48, 64, 96, 128, 360, 512, 720, 1024))
        T = tuple(rng.randint(1, 4096) for _ in range(k))
        h = tuple(rng.randint(0, 16) for _ in range(k))
        tr = tuple(m for m in range(k) if rng.randint(0, 2) == 0)
        chain = [("merge", 0, 1), ("decompose", 0, T, h, tr)]
        shape, _ = N.plan((8,) * k, (d, 1), chain, ("block",))
        hw = h if any(h) else (1,) * k
        assert shape == O.decompose(d, T, h=hw, transposes=tr), (d, T, h, tr)


def test_greedy_grid_matches_oracle():
    # Algorithm A1, engine vs oracle (the oracle's version is pinned to the
    # paper's Sec. 4.1 example and the Sec. 4.3 counterexample)
    for d in list(range(1, 300)) + [512, 720, 2520, 3600, 4096, 65536, 9699690]:
        for k in (1, 2, 3, 4):
            assert N.greedy_grid(d, k) == O.greedy(d, k), (d, k)


def test_hier_chain_matches_the_pinned_construction():
    # the engine's two-level chains equal the test-side construction (the
    # one the oracle pins use), and plan to the expected final spaces
    import hier_chains as T
    rng = W.rng(906)
    for _ in range(60):
        k = rng.randint(1, 4)
        n, g = rng.choice((1, 2, 4, 6, 12, 64)), rng.choice((1, 2, 4, 8))
        fa, fb = O.factorisations(n, k), O.factorisations(g, k)
        a, b = fa[rng.randint(0, len(fa) - 1)], fb[rng.randint(0, len(fb) - 1)]
        for variant in ("block", "cyclic"):
            ch, dist = N.hier_chain(a, b, variant)
            want_ch, want_dist = T.hier_chain(k, a, b, variant)
            assert (ch, dist) == (want_ch, want_dist)
            shape, _ = N.plan((8,) * k, (n, g), ch, dist)
            want = tuple(a[t] * b[t] for t in range(k)) if variant == "block" else tuple(a) + tuple(b)
            assert shape == want


def _pool_min_secondaries(q):
    """Least secondary (tiles) over every chain, per factorisation, from the
    oracle's exact costs."""
    import numpy as np
    M, Nn, K = q["MNK"]
    n, g = q["machine"]
    fs = O.factorisations(n * g, 3)
    nch = len(O.chains(n, g, q["max_depth"]))
    out = {}
    for i, f in enumerate(fs):
        idx = np.arange(i * nch, (i + 1) * nch, dtype=np.int64)
        _, s = O.candidate_costs(M, Nn, K, (n, g), q["max_depth"], idx)
        out[f] = int(s.min())
    return out


def test_secondary_lower_bound_is_a_lower_bound():
    # never above the least secondary any chain reaches (oracle, every chain)
    checked = 0
    for q in W.search_query_small(count=8):
        mins = _pool_min_secondaries(q)
        for f, smin in mins.items():
            lb = N.secondary_lower_bound(q, f) // q["tile_bytes"]
            assert lb <= smin, (q, f, lb, smin)
            checked += lb > 0
    assert checked > 0


def test_secondary_lower_bound_is_reached_on_divisible_grids():
    # extents divisible by the factors on 64 x 8: an optimal chain gives every
    # node an optimal down-set, so the bound equals the least secondary for
    # the factorisations of least primary cost
    import math
    for MNK in ((1024, 4096, 1024), (4096, 4096, 1024)):
        q = {"MNK": MNK, "machine": (64, 8), "max_depth": 3, "tile_bytes": 512 * 512 * 4}
        fs = O.factorisations(512, 3)

        def primary(f):
            return sum((min(MNK[v], f[v]) - 1) * math.prod(MNK[t] for t in range(3) if t != v) for v in range(3))

        pmin = min(primary(f) for f in fs)
        pool = [f for f in fs if primary(f) == pmin]
        import numpy as np
        nch = len(O.chains(64, 8, 3))
        for f in pool:
            i = fs.index(f)
            idx = np.arange(i * nch, (i + 1) * nch, dtype=np.int64)
            _, s = O.candidate_costs(*MNK, (64, 8), 3, idx)
            assert N.secondary_lower_bound(q, f) // q["tile_bytes"] == int(s.min()), (MNK, f)


def test_batch_query_records_match_the_c_structs():
    # the numpy records handed to mp_batch_create hold, byte for byte, what
    # the field-by-field ctypes structures hold (chain pointers aside, which
    # must point at the same transforms)
    from paper_2507_17087_gb300 import workloads as W
    qs = W.batched_queries(400)
    launches = [(q["L"], q["machine"], N.chain_from_draws(*q["machine"], q["draws"]), q["dist"], q["face"])
                for q in qs]
    launches.append(((5, 6), (2, 3), [("decompose", 0, (5, 6), (2, 1), (1,))], ("block_cyclic", 3), (4, 8)))
    xf, rec = N.query_records(launches)
    for q, (L, machine, chain, dist, face) in enumerate(launches):
        ch, n = N.make_chain(chain)
        a = N.mp_query()
        a.space, a.machine, a.n_xf, a.dist = N.make_space(L), N.make_machine(machine), n, N.make_dist(dist)
        for t, v in enumerate(face):
            a.face_bytes[t] = int(v)
        got, want = bytearray(rec[q].tobytes()), bytearray(bytes(a))
        off = N.mp_query.chain.offset
        got[off:off + 8] = want[off:off + 8] = bytes(8)
        assert got == want, q
        first = (int(rec[q]["chain"]) - xf.ctypes.data) // ctypes.sizeof(N.mp_xform)
        assert xf[first:first + n].tobytes() == bytes(ch)[:ctypes.sizeof(N.mp_xform) * n], q
