"""Pins the CPU oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints (tests/golden/paper_values.txt), a closed form derived from the
paper's surface formula, an invariant of the transforms, or brute force on tiny
inputs.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from hier_chains import hier_chain, node_chain
from paper_2507_17087_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, value, _cite = (s.strip() for s in line.split("|"))
        vals[name] = value
    return vals


G = golden()


def ints(s):
    return tuple(int(v) for v in s.split())


# ------------------------------------------------------------ worked examples

def test_fig3_block2d_point():
    # Fig. 3: (6,6) on (2,2); point (2,3) -> node 0, GPU 1
    L = O.Launch((6, 6), (2, 2), [], ("block",))
    node, gpu = ints(G["fig3_block2d_point_2_3"])
    ids = L.owner_of([2 * 6 + 3])
    assert ids[0] == node * 2 + gpu
    n, p = L.resolve(np.array([[2 * 2 // 6, 3 * 2 // 6]]))
    assert (n[0], p[0]) == (node, gpu)


def test_sec41_factorisations_and_greedy():
    want = sorted(tuple(int(v) for v in t.split()) for t in G["sec41_factorisations_6_k2"].split(";"))
    assert O.factorisations(6, 2) == want
    assert O.greedy(6, 2) == ints(G["sec41_greedy_grid_6"])


@pytest.mark.parametrize("L,key", [((12, 18), "sec41_volume_12x18_grid_3x2"),
                                   ((18, 12), "sec41_volume_18x12_grid_3x2")])
def test_sec41_volumes(L, key):
    # grid (3,2): machine (3,2) with the plain block mapping; 1 element per face
    launch = O.Launch(L, (3, 2), [], ("block",))
    tot, recv = launch.comm_volume((1, 1))
    assert tot == int(G[key])
    assert int(recv.sum()) == tot


def test_sec41_better_grid_and_decompose():
    # decompose picks (2,3) for (12,18) and (3,2) for (18,12); (2,3) gives 84
    assert O.decompose(6, (12, 18)) == ints(G["sec41_better_grid_12x18"])
    assert O.decompose(6, (18, 12)) == (3, 2)
    launch = O.Launch((12, 18), (2, 3), [], ("block",))
    assert launch.comm_volume((1, 1))[0] == int(G["sec41_volume_18x12_grid_3x2"])
    w = tuple(Fraction(l, d) for l, d in zip((18, 12), O.decompose(6, (18, 12))))
    assert w == tuple(Fraction(v) for v in ints(G["sec42_workload_18x12"]))


def test_fig10_3d_example():
    parts = [ints(s) for s in G["sec42_fig10_3d"].split(";")]
    l, d, w = parts[0], parts[1][0], parts[2]
    f = O.decompose(d, l)
    assert tuple(Fraction(a, b) for a, b in zip(l, f)) == tuple(Fraction(v) for v in w)
    # 2S = SA(w) d - SA(l), SA(x) = 2 (prod x)(sum 1/x): the directed face count
    SA = lambda x: 2 * math.prod(x) * sum(Fraction(1, v) for v in x)
    two_s = SA(w) * d - SA(l)
    launch = O.Launch(l, (4, 4), [("merge", 0, 1), ("decompose", 0, l)], ("block",))
    assert launch.final_shape() == f
    assert launch.comm_volume((1, 1, 1))[0] == two_s == 224


def test_sec43_counts():
    assert len(O.factorisations(16, 3)) == int(G["sec43_count_16_k3"])
    # general count prod_j C(a_j + k - 1, k - 1), checked against brute force
    for d in (1, 2, 12, 16, 48, 72, 360, 512, 2520, 3600, 4096):
        for k in (1, 2, 3, 4):
            fac = O.factorisations(d, k)
            want = math.prod(math.comb(a + k - 1, k - 1) for a in _exponents(d))
            assert len(fac) == want
            if d <= 360 and k <= 3:
                brute = sorted(t for t in itertools.product(_divisors(d), repeat=k)
                               if math.prod(t) == d)
                assert fac == brute
    assert [len(O.factorisations(p, 3)) for p in (512, 2520, 3600, 4096)] == [55, 540, 540, 91]


def _exponents(d):
    out, p = [], 2
    while p * p <= d:
        e = 0
        while d % p == 0:
            d //= p
            e += 1
        if e:
            out.append(e)
        p += 1
    if d > 1:
        out.append(1)
    return out


def _divisors(d):
    return [v for v in range(1, d + 1) if d % v == 0]


def test_sec43_greedy_counterexample():
    greedy = O.greedy_workload(72, (8, 9))
    want = tuple(Fraction(s) for s in G["sec43_greedy_72_8x9"].split())
    assert tuple(Fraction(l, d) for l, d in zip((8, 9), greedy)) == want
    best = O.decompose(72, (8, 9))
    want = tuple(Fraction(s) for s in G["sec43_exhaustive_72_8x9"].split())
    assert tuple(Fraction(l, d) for l, d in zip((8, 9), best)) == want


def test_decompose_brute_force():
    rng = W.rng(11)
    for _ in range(200):
        k = rng.randint(1, 3)
        d = rng.randint(1, 200)
        l = tuple(rng.randint(1, 40) for _ in range(k))
        got = O.decompose(d, l)
        cands = [t for t in itertools.product(_divisors(d), repeat=k) if math.prod(t) == d]
        best = min(cands, key=lambda t: (sum(Fraction(a, b) for a, b in zip(t, l)), t))
        assert got == best


def test_plain_config_decompose_tie_break():
    # 8 processors over 64x64: (2,4) and (4,2) tie; lexicographic -> (2,4)
    assert O.decompose(8, (64, 64)) == (2, 4)


# ------------------------------------------------------------ transforms

def test_split_then_merge_is_identity():
    # Sec. 3.3: m.split(0, d).merge(0, 1) == m
    for (n, g) in [(6, 4), (12, 2), (8, 8)]:
        for d in _divisors(n):
            L = O.Launch((n, g), (n, g), [("split", 0, d), ("merge", 0, 1)], ("block",))
            assert L.final_shape() == (n, g)
            a = np.array([[i, j] for i in range(n) for j in range(g)])
            node, proc = L.resolve(a)
            assert np.array_equal(node, a[:, 0]) and np.array_equal(proc, a[:, 1])


def test_merge_then_split_is_identity():
    for (n, g) in [(6, 4), (3, 5)]:
        L = O.Launch((n, g), (n, g), [("merge", 0, 1), ("split", 0, n)], ("block",))
        a = np.array([[i, j] for i in range(n) for j in range(g)])
        node, proc = L.resolve(a)
        assert np.array_equal(node, a[:, 0]) and np.array_equal(proc, a[:, 1])


def test_block1d_x_worked_translation():
    # Sec. 5.2: m.merge(0,1).split(0, n g) -> (n g, 1); point (ix, iy) goes to
    # (a mod n, a div n), a = floor(ix * n g / Lx)
    n, g, Lx, Ly = 3, 4, 17, 5
    chain = [("merge", 0, 1), ("split", 0, n * g)]
    L = O.Launch((Lx, Ly), (n, g), chain, ("block",))
    assert L.final_shape() == (n * g, 1)
    ids, _ = L.map_points()
    for ix in range(Lx):
        for iy in range(Ly):
            a = ix * n * g // Lx
            assert ids[ix * Ly + iy] == (a % n) * g + a // n


def test_swap_chain_closed_form():
    n, g = 3, 4
    L = O.Launch((7, 9), (n, g), [("swap", 0, 1)], ("block",))
    assert L.final_shape() == (g, n)
    ids, _ = L.map_points()
    for x in range(7):
        for y in range(9):
            a0, a1 = x * g // 7, y * n // 9
            assert ids[x * 9 + y] == a1 * g + a0


def test_merge_formula_three_dims():
    # Fig. 4 merge(0, 2) on (2, 3, 4): a' = (a0 + 2 a2, a1)
    L = O.Launch((8, 3), (2, 12), [("split", 1, 3), ("merge", 0, 2)], ("block",))
    assert L.final_shape() == (8, 3)
    a = np.array([[i, j] for i in range(8) for j in range(3)])
    node, proc = L.resolve(a)
    for (i, j), nd, pr in zip(a, node, proc):
        b0, b1, b2 = i % 2, j, i // 2       # inverse merge(0,2)
        assert (nd, pr) == (b0, b1 + b2 * 3)  # inverse split(1, 3)


def test_solomonik_split_structure():
    # Fig. 5b: 2 nodes x 4 GPUs, four splits -> 6-D (2,1,1) x (1,2,2); nodes
    # split the x axis in halves, the GPUs of a node block the y-z plane.
    chain = [("split", 0, 2), ("split", 1, 1), ("split", 3, 1), ("split", 4, 2)]
    L = O.Launch((4, 4, 4), (2, 4), chain, ("block",))
    X = 4
    pts = [(x, y, z) for x in range(X) for y in range(X) for z in range(X)]
    a = np.array([[x * 2 // X, 0, 0, 0, y * 2 // X, z * 2 // X] for x, y, z in pts])
    lp = O.Launch((4, 4, 4), (2, 4), chain, ("hier",))  # rank-6 final space, no fix-up
    assert lp.final_shape() == (2, 1, 1, 1, 2, 2)
    node, proc = lp.resolve(a)
    for (x, y, z), nd, pr in zip(pts, node, proc):
        assert nd == x * 2 // X
        assert pr == (y * 2 // X) + 2 * (z * 2 // X)


def test_cannon_hierarchical_mapper():
    # Appendix A.1: m3d = machine.decompose(0, is); m4d = m3d.decompose(2,
    # is / m3d[:-1]); upper = ip * m4d[0:2] / is; lower = ip % m4d[2:4]
    n, g, Lx, Ly = 4, 4, 8, 8
    L = O.Launch((Lx, Ly), (n, g), [], ("hier",))
    assert L.final_shape() == (2, 2, 2, 2)
    ids, _ = L.map_points()
    for i in range(Lx):
        for j in range(Ly):
            u0, u1 = i * 2 // Lx, j * 2 // Ly
            l0, l1 = i % 2, j % 2
            node, gpu = u0 + 2 * u1, l0 + 2 * l1   # inverse of the two decomposes
            assert ids[i * Ly + j] == node * g + gpu
    # the explicit two-decompose chain gives the same ids
    explicit = [("decompose", 0, (Lx, Ly)), ("decompose", 2, (Lx // 2, Ly // 2))]
    ids2, _ = O.Launch((Lx, Ly), (n, g), explicit, ("hier",)).map_points()
    assert np.array_equal(ids, ids2)


def test_linear_cyclic_subdiagonal():
    # Fig. 5: merge(0,1) -> 1-D of size 4; linearised points round robin.
    # With a 4-wide task space in C order, (i, j) -> (4 i + j) mod 4 = j.
    L = O.Launch((4, 4), (2, 2), [("merge", 0, 1)], ("linear_cyclic",))
    ids, hist = L.map_points()
    a = np.array([[(i * 4 + j) % 4] for i in range(4) for j in range(4)])
    node, proc = L.resolve(a)
    assert np.array_equal(ids, node * 2 + proc)
    assert list(hist) == [4, 4, 4, 4]


def test_balance_split_is_shape_agnostic_decompose():
    # balance_split(i, k) (read as decompose(i, (1,)*k)) == decompose(i, (c,)*k) for any cube
    for P in (8, 12, 36, 64):
        for k in (2, 3):
            a = O.Launch((5,) * k, (P, 1), [("balance_split", 0, k)], ("block",)).final_shape()
            b = O.Launch((5,) * k, (P, 1), [("decompose", 0, (7,) * k)], ("block",)).final_shape()
            assert a[:k] == b[:k]


# ------------------------------------------------------------ invariants

def _random_launch(rng, max_points=600, dists=W.DIST_KINDS):
    k = rng.randint(1, 3)
    L = tuple(rng.randint(1, 12) for _ in range(k))
    while math.prod(L) > max_points:
        L = tuple(max(1, v // 2) for v in L)
    machine = (rng.randint(1, 6), rng.randint(1, 4))
    draws = [rng.next() for _ in range(rng.randint(0, 4))]
    chain = O.chain_from_draws(machine[0], machine[1], draws)
    kind = rng.choice(dists)
    dist = ("block_cyclic", rng.randint(1, 4)) if kind == "block_cyclic" else (kind,)
    return L, machine, chain, dist


def test_every_point_one_in_range_processor():
    rng = W.rng(21)
    for _ in range(150):
        L, machine, chain, dist = _random_launch(rng)
        launch = O.Launch(L, machine, chain, dist)
        ids, hist = launch.map_points()
        P = machine[0] * machine[1]
        assert ids.min() >= 0 and ids.max() < P
        assert int(hist.sum()) == math.prod(L)
        assert np.array_equal(np.bincount(ids, minlength=P), hist.astype(np.int64))


def test_resolution_is_a_bijection():
    rng = W.rng(22)
    for _ in range(100):
        L, machine, chain, dist = _random_launch(rng)
        launch = O.Launch(L, machine, chain, dist)
        shape = launch.final_shape()
        assert math.prod(shape) == launch.P
        a = np.array(list(itertools.product(*[range(s) for s in shape])))
        node, proc = launch.resolve(a)
        ids = node * machine[1] + proc
        assert sorted(ids.tolist()) == list(range(launch.P))


def test_block_histogram_is_product_of_interval_lengths():
    rng = W.rng(23)
    for _ in range(60):
        L, machine, chain, _ = _random_launch(rng)
        launch = O.Launch(L, machine, chain, ("block",))
        shape = launch.final_shape()
        _, hist = launch.map_points(want_ids=False)
        a = np.array(list(itertools.product(*[range(s) for s in shape])))
        node, proc = launch.resolve(a)
        for row, nd, pr in zip(a, node, proc):
            want = 1
            for t, at in enumerate(row):
                lo = -(-at * L[t] // shape[t])
                hi = -(-(at + 1) * L[t] // shape[t])
                want *= hi - lo
            assert hist[nd * machine[1] + pr] == want


def test_halo_closed_form_matches_brute_force():
    rng = W.rng(24)
    for _ in range(150):
        L, machine, chain, dist = _random_launch(rng)
        launch = O.Launch(L, machine, chain, dist)
        face = tuple(rng.randint(1, 9) for _ in L)
        tot, recv = launch.comm_volume(face)
        assert tot == launch.halo_closed_form(face)
        assert int(recv.sum()) == tot


def test_block_halo_closed_form_by_hand():
    # BLOCK: V = 2 sum_t (min(s_t, L_t) - 1) prod_{u != t} L_u faces
    rng = W.rng(25)
    for _ in range(60):
        L, machine, chain, _ = _random_launch(rng)
        launch = O.Launch(L, machine, chain, ("block",))
        s = launch.final_shape()
        want = sum(2 * (min(s[t], L[t]) - 1) * math.prod(L) // L[t] for t in range(len(L)))
        assert launch.comm_volume([1] * len(L))[0] == want


def test_map_launch_equals_per_pair_evaluation():
    # the one-pass form (owners evaluated once, each neighbour's owner looked
    # up) against map_points and against comm_volume, which evaluates the
    # neighbour's owner again for every directed pair; all five
    # distributions, threads or not
    rng = W.rng(26)
    for it in range(200):
        L, machine, chain, dist = _random_launch(rng, max_points=5000)
        launch = O.Launch(L, machine, chain, dist)
        face = tuple(rng.randint(1, 9) for _ in L)
        threads = 1 + it % 3
        ids, hist, tot, recv = launch.map_launch(face, threads=threads)
        rids, rhist = launch.map_points()
        rtot, rrecv = launch.comm_volume(face)
        assert np.array_equal(ids, rids) and np.array_equal(hist, rhist)
        assert tot == rtot and np.array_equal(recv, rrecv), (L, machine, chain, dist)


def test_map_launch_halo_by_numpy_neighbour_comparison():
    # directed faces counted from the ids array with plain numpy slicing
    rng = W.rng(27)
    for _ in range(60):
        L, machine, chain, dist = _random_launch(rng, max_points=4000)
        launch = O.Launch(L, machine, chain, dist)
        face = tuple(rng.randint(1, 9) for _ in L)
        ids, _, tot, recv = launch.map_launch(face)
        v = ids.reshape(L)
        P = machine[0] * machine[1]
        want = np.zeros(P, dtype=np.int64)
        for t in range(len(L)):
            a = np.take(v, np.arange(L[t] - 1), axis=t)
            b = np.take(v, np.arange(1, L[t]), axis=t)
            cross = a != b
            want += face[t] * (np.bincount(a[cross], minlength=P) + np.bincount(b[cross], minlength=P))
        assert np.array_equal(recv.astype(np.int64), want) and tot == int(want.sum())


def test_halo_and_histogram_multiset_independent_of_chain():
    L, machine = (9, 7, 5), (4, 3)
    ref = None
    for chain in [[], [("swap", 0, 1)], [("merge", 0, 1), ("split", 0, 6)],
                  [("split", 0, 2), ("merge", 1, 2), ("swap", 0, 1)]]:
        launch = O.Launch(L, machine, chain + [("merge", 0, 1), ("decompose", 0, L)], ("block",))
        tot, _ = launch.comm_volume((1, 1, 1))
        _, hist = launch.map_points(want_ids=False)
        key = (tot, sorted(hist.tolist()))
        ref = ref or key
        assert key == ref


def test_plain_and_large_halo_values():
    cfg = W.plain_config()
    launch = O.Launch(cfg["L"], cfg["machine"], cfg["chain"], cfg["dist"])
    assert launch.final_shape() == (2, 4)
    tot, _ = launch.comm_volume(cfg["face"])
    assert tot == 512 * 2048 == 1048576
    # 1024x1024x512 on (8,8,8): 29,360,128 directed faces of 8 bytes (closed form)
    big = O.Launch((1024, 1024, 512), (64, 8), [("merge", 0, 1), ("decompose", 0, (1024, 1024, 512))],
                   ("block",))
    assert big.final_shape() == (8, 8, 8)
    assert big.halo_closed_form((8, 8, 8)) == 29360128 * 8 == 234881024


# ------------------------------------------------------------ canonical chains

def test_chain_enumeration_matches_alphabet_recursion():
    # re-derive the canonical order independently in Python for small machines
    def alphabet(shape):
        ops = []
        for i, s in enumerate(shape):
            ops += [("split", i, d) for d in range(2, s) if s % d == 0]
        r = len(shape)
        ops += [("merge", p, q) for p in range(r) for q in range(p + 1, r)]
        ops += [("swap", p, q) for p in range(r) for q in range(p + 1, r)]
        return ops

    def apply(shape, op):
        s = list(shape)
        if op[0] == "split":
            i, d = op[1], op[2]
            return tuple(s[:i] + [d, s[i] // d] + s[i + 1:])
        if op[0] == "merge":
            p, q = op[1], op[2]
            t = s[:]
            t[p] = s[p] * s[q]
            del t[q]
            return tuple(t)
        t = s[:]
        t[op[1]], t[op[2]] = t[op[2]], t[op[1]]
        return tuple(t)

    def enum(shape, depth):
        if depth == 0:
            return [()]
        out = []
        for op in alphabet(shape):
            out += [(op,) + rest for rest in enum(apply(shape, op), depth - 1)]
        return out

    for n, g, D in [(2, 4, 3), (6, 2, 2), (4, 8, 2), (3, 1, 3)]:
        want = [c for depth in range(D + 1) for c in enum((n, g), depth)]
        assert O.chains(n, g, D) == want


def test_chain_from_draws():
    draws = [5, 17, 3, 99]
    ch = O.chain_from_draws(64, 8, draws)
    assert len(ch) == 4
    all1 = O.chains(64, 8, 1)[1:]   # depth-1 chains = the alphabet at (64, 8)
    assert ch[0] == all1[5 % len(all1)][0]


# ------------------------------------------------------------ matmul cost / search

def test_matmul_grouped_equals_literal():
    rng = W.rng(31)
    for _ in range(40):
        n, g = rng.randint(1, 4), rng.choice((1, 2, 4))
        P = n * g
        M, N, K = (rng.randint(1, 9) for _ in range(3))
        chains = O.chains(n, g, 2)
        chain = chains[rng.next() % len(chains)]
        fs = O.factorisations(P, 3)
        f = fs[rng.next() % len(fs)]
        assert O.matmul_cost(M, N, K, (n, g), chain, f, literal=True) == \
            O.matmul_cost(M, N, K, (n, g), chain, f, literal=False)


def test_matmul_primary_closed_form_and_decompose_argmin():
    for (M, N, K), (n, g) in [((8, 16, 4), (4, 4)), ((256, 1024, 4096), (64, 8)),
                              ((1024, 256, 256), (315, 8)), ((4096, 4096, 1024), (450, 8))]:
        P = n * g
        fs = O.factorisations(P, 3)
        prim = {}
        for f in fs:
            p, _ = O.matmul_cost(M, N, K, (n, g), (), f)
            want = M * K * (min(N, f[1]) - 1) + K * N * (min(M, f[0]) - 1) + M * N * (min(K, f[2]) - 1)
            assert p == want
            prim[f] = p
        best = min(fs, key=lambda f: (prim[f], f))
        if all(fm <= lm for fm, lm in zip(best, (M, N, K))):
            assert best == O.decompose(P, (M, N, K))


def test_search_equals_brute_force_min():
    for q in W.search_query_small(count=6):
        M, N, K = q["MNK"]
        n, g = q["machine"]
        D = q["max_depth"]
        res = O.search(M, N, K, (n, g), D)
        fs = O.factorisations(n * g, 3)
        chains = O.chains(n, g, D)
        best = None
        for fr, f in enumerate(fs):
            for c, chain in enumerate(chains):
                p, s = O.matmul_cost(M, N, K, (n, g), chain, f)
                key = (p, s, fr * len(chains) + c)
                best = key if best is None or key < best else best
        assert (res["primary"], res["secondary"], res["index"]) == best
        assert res["n_candidates"] == len(fs) * len(chains)


def test_search_literal_brute_force_tiny():
    # every candidate's cost by the literal per-tile definition on a tiny grid
    M, N, K, n, g = 3, 4, 2, 2, 2
    fs = O.factorisations(4, 3)
    chains = O.chains(n, g, 2)
    best = None
    for fr, f in enumerate(fs):
        for c, chain in enumerate(chains):
            p, s = O.matmul_cost(M, N, K, (n, g), chain, f, literal=True)
            key = (p, s, fr * len(chains) + c)
            best = key if best is None or key < best else best
    res = O.search(M, N, K, (n, g), 2)
    assert (res["primary"], res["secondary"], res["index"]) == best


def test_secondary_worked_by_hand():
    # 4 x 2 x 2 tiles (M, N, K) on Machine(GPU) = (2 nodes, 2 GPUs), f = (2, 2, 1).
    # Block coordinates: a0 = floor(2 i / 4) (i = 0,1 -> 0; i = 2,3 -> 1),
    # a1 = j, a2 = 0; flat index b = a0 + 2 a1.  Flattening (node, gpu) with
    # merge(0, 1) puts the node fastest (Sec. 5.2): node(b) = b mod 2,
    # gpu(b) = b div 2.
    #   A(i, k), 8 tiles, fibre over j: b in {a0, a0 + 2} -> 2 processors, 1 node
    #   B(k, j), 4 tiles, fibre over i: b in {2j, 2j + 1} -> 2 processors, 2 nodes
    #   C(i, j), 8 tiles, fibre over k: one block -> 1 processor, 1 node
    # primary = 8 (2 - 1) + 4 (2 - 1) + 0 = 12; secondary = 0 + 4 (2 - 1) + 0 = 4.
    # With swap(0, 1) first, the flattened space is (gpu, node) merged gpu
    # fastest: node(b) = b div 2 = a1 = j.
    #   A: nodes {0, 1} -> 8 (2 - 1) = 8;  B: node j only -> 0;  C: 0
    # secondary = 8 (the primary does not depend on the chain).
    for literal in (False, True):
        assert O.matmul_cost(4, 2, 2, (2, 2), (), (2, 2, 1), literal=literal) == (12, 4)
        assert O.matmul_cost(4, 2, 2, (2, 2), (("swap", 0, 1),), (2, 2, 1), literal=literal) == (12, 8)


def test_secondary_depends_on_chain():
    # splits followed by the flattening merges are the identity (Sec. 3.3), so
    # only merge / swap reorderings matter; an asymmetric grid exposes them
    M, N, K, n, g = 64, 256, 16, 8, 8
    f = (4, 4, 4)
    vals = {O.matmul_cost(M, N, K, (n, g), ch, f)[1] for ch in O.chains(n, g, 1)}
    assert len(vals) > 1


# ------------------------------------------- anisotropic halo and transposes
# The appendix's "Generalization of the Decompose Primitive": halo width h_n
# along dimension n gives V = sum_n d_n h_n prod_{m != n} l_m, and an
# all-to-all transpose along n adds V*_n = (1 - 1/d_n) (prod_m w_m) d.

def _grid_chain(f):
    """A chain whose final space is the grid f on Machine(1, P)."""
    ch = [("merge", 0, 1)]
    for t in range(len(f) - 1):
        ch.append(("split", t, f[t]))
    return ch


@pytest.mark.parametrize("L,f,h", [((12, 18), (2, 3), (2, 3)), ((16, 16), (4, 2), (1, 4)),
                                   ((8, 12, 6), (2, 3, 2), (2, 1, 3)), ((30,), (5,), (3,))])
def test_halo_elements_match_the_appendix_volume(L, f, h):
    # BLOCK, extents divisible by the grid, width <= block width: every
    # interior cut moves h_n layers each way.  The appendix's V counts d_n
    # cuts per dimension (the outer surface included): the exact
    # count is 2 V - 2 sum_n h_n prod_{m != n} l_m.
    P = math.prod(f)
    ln = O.Launch(L, (1, P), _grid_chain(f), ("block",))
    assert ln.final_shape() == tuple(f)
    tot, recv = ln.halo_elements(h, [1] * len(L))
    V = sum(f[n] * h[n] * math.prod(L[m] for m in range(len(L)) if m != n) for n in range(len(L)))
    outer = sum(h[n] * math.prod(L[m] for m in range(len(L)) if m != n) for n in range(len(L)))
    assert tot == 2 * V - 2 * outer
    assert int(recv.sum()) == tot


@pytest.mark.parametrize("dist", [("block",), ("block_cyclic", 3)])
def test_halo_elements_width_one_equals_faces_for_blocks(dist):
    # with width 1 the de-duplicated count and the directed-face
    # count differ only where both neighbours of an element belong to one
    # other owner; with runs of at least two points per owner along every
    # dimension (block, block-cyclic with b >= 2) that cannot happen
    for q in range(4):
        cfg = W.scaled_launch((9, 14, 5), (2, 3), dist[0], 300 + q)
        ch = O.chain_from_draws(*cfg["machine"], cfg["draws"])
        ln = O.Launch(cfg["L"], cfg["machine"], ch, dist)
        assert ln.halo_elements((1, 1, 1), (8, 8, 8))[0] == ln.comm_volume((8, 8, 8))[0]


def test_halo_elements_width_one_cyclic_pairs():
    # CYCLIC over 2 residues: an interior element's two neighbours share one
    # owner, so it is sent once (the face count sends it twice)
    ln = O.Launch((10,), (1, 2), [], ("cyclic",))
    assert ln.halo_elements((1,), (1,))[0] == 10
    assert ln.comm_volume((1,))[0] == 18


def test_halo_elements_cyclic_closed_form():
    # CYCLIC with s_t > 2 w_t: all 2 w_t neighbours of an element along t
    # have distinct residues, none equal to its own, so the element goes to
    # min(y, w) + min(L - 1 - y, w) receivers; summed over y: 2 L w - w^2 - w
    for L, w in (((40, 33), (3, 2)), ((25, 50), (1, 5))):
        ln = O.Launch(L, (16, 16), [], ("cyclic",))
        s = ln.final_shape()
        assert all(s[t] > 2 * w[t] for t in range(2)), s
        tot, _ = ln.halo_elements(w, (1, 1), want_recv=False)
        want = sum((2 * L[t] * w[t] - w[t] * w[t] - w[t]) * L[1 - t] for t in range(2))
        assert tot == want


def _brute_elements(ids, L, width, eb, P):
    """Brute force from an id array: per element and dimension, the set of
    other owners within the halo width."""
    a = ids.reshape(L)
    tot = 0
    recv = np.zeros(P, dtype=np.int64)
    for y in itertools.product(*(range(e) for e in L)):
        me = a[y]
        for t in range(len(L)):
            owners = set()
            for dlt in range(-width[t], width[t] + 1):
                z = list(y)
                z[t] += dlt
                if dlt == 0 or not 0 <= z[t] < L[t]:
                    continue
                o = int(a[tuple(z)])
                if o != me:
                    owners.add(o)
            tot += eb[t] * len(owners)
            for o in owners:
                recv[o] += eb[t]
    return tot, recv


@pytest.mark.parametrize("kind", ["block", "cyclic", "block_cyclic", "hier", "linear_cyclic"])
def test_halo_elements_brute_force(kind):
    for q in range(3):
        L = ((7, 9), (5, 4, 6), (23,))[q]
        width = ((2, 3), (1, 2, 3), (4,))[q]
        eb = ((3, 5), (1, 2, 4), (7,))[q]
        cfg = W.scaled_launch(L, (2, 3), kind, 400 + q)
        ch = O.chain_from_draws(*cfg["machine"], cfg["draws"])
        ln = O.Launch(L, cfg["machine"], ch, cfg["dist"])
        ids, _ = ln.map_points()
        tot, recv = ln.halo_elements(width, eb)
        bt, br = _brute_elements(ids, L, width, eb, ln.P)
        assert tot == bt
        assert np.array_equal(recv.astype(np.int64), br)


def test_weighted_decompose_reduces_to_sec42():
    # unit widths and no transposes: the Sec. 4.2 objective (pinned above);
    # any uniform width scales it and keeps the argmin
    for d, l in ((16, (64, 64)), (512, (1024, 1024, 512)), (3600, (256, 1024, 4096)), (6, (12, 18))):
        base = O.decompose(d, l)
        assert O.decompose(d, l, h=(1,) * len(l)) == base
        assert O.decompose(d, l, h=(7,) * len(l)) == base


def test_weighted_decompose_worked_values():
    # d = 16, l = (64, 64), f = (4, 4), h = (1, 1), transpose along dim 0:
    # V = 4*1*64 + 4*1*64 = 512; V*_0 = (1 - 1/4) * (16 * 16) * 16 = 3072;
    # the oracle compares d * (V + V*_0) = 16 * 3584 = 57344
    assert O.weighted_objective(16, (4, 4), (64, 64), (1, 1), (0,)) == 57344
    # (1, 16): V = 64 + 1024 = 1088, V*_0 = 0 -> 17408, the argmin
    assert O.weighted_objective(16, (1, 16), (64, 64), (1, 1), (0,)) == 17408
    assert O.decompose(16, (64, 64), transposes=(0,)) == (1, 16)
    # a wide halo along dim 0 keeps it uncut; (2, 8) wins for h = (4, 1):
    # V(2,8) = 4*2*64 + 8*64 = 1024 < V(4,4) = V(1,16) = 1280
    assert O.decompose(16, (64, 64), h=(1000, 1)) == (1, 16)
    assert O.decompose(16, (64, 64), h=(4, 1)) == (2, 8)


def test_weighted_decompose_transposes_only():
    # no halo and a transpose along every dimension: minimise
    # sum_n (1 - 1/d_n), i.e. put all of d on one dimension; the
    # lexicographically smallest such tuple is (1, ..., 1, d)
    for d, k in ((12, 2), (64, 3), (360, 4)):
        assert O.decompose(d, (5,) * k, h=(0,) * k, transposes=tuple(range(k))) == (1,) * (k - 1) + (d,)


def test_weighted_decompose_minimises_the_exact_halo_count():
    # for BLOCK grids that divide the extents the exact element count is an
    # affine function of V with a d-independent offset, so the weighted
    # argmin is the grid of least exact volume (first in lexicographic order)
    for L, P, h in (((24, 36), 12, (3, 1)), ((16, 48), 16, (1, 2)), ((12, 12, 24), 8, (2, 1, 1))):
        best = None
        for f in O.factorisations(P, len(L)):
            if any(L[t] % f[t] or L[t] // f[t] < h[t] for t in range(len(L))):
                continue
            v, _ = O.Launch(L, (1, P), _grid_chain(f), ("block",)).halo_elements(h, [1] * len(L), want_recv=False)
            if best is None or v < best[0]:
                best = (v, f)
        assert O.decompose(P, L, h=h) == best[1]


def test_weighted_decompose_in_a_chain():
    # the chain form applies the generalised objective to the machine
    ln = O.Launch((64, 64), (4, 4), [("merge", 0, 1), ("decompose", 0, (64, 64), (4, 1))], ("block",))
    assert ln.final_shape() == (2, 8)
    ln = O.Launch((64, 64), (4, 4), [("merge", 0, 1), ("decompose", 0, (64, 64), None, (0,))], ("block",))
    assert ln.final_shape() == (1, 16)


# ------------------------------------------------------ hierarchical search
# Two-level (node grid a x GPU grid b) mappings: node u_t = floor(x_t a_t / L_t),
# GPU block-within-node floor(x_t a_t b_t / L_t) mod b_t or cyclic x_t mod b_t.

@pytest.mark.parametrize("N", [4, 6, 8])
def test_hier_search_recovers_the_fig5b_mapper(N):
    # Fig. 5b: on 2 nodes x 4 GPUs a 3-D launch longer along x maps with node
    # space (2,1,1) and GPU space (1,2,2); the search's optimum is that pair
    r = O.hier_search((2 * N, N, N), (2, 4), "block", (1, 1, 1), (1, 1, 1), threads=8)
    assert r["a"] == ints(G["fig5b_solomonik_node_space"])
    assert r["b"] == ints(G["fig5b_solomonik_gpu_space"])
    assert r["primary"] == 2 * N * N   # one node cut of N x N, both directions


@pytest.mark.parametrize("variant", ["block", "cyclic"])
def test_hier_costs_match_chain_mappings(variant):
    # the direct formulas against the same mappings written as
    # split / swap / merge chains with the block or hierarchical distribution
    rng = W.rng(810)
    for _ in range(12):
        k = rng.randint(1, 3)
        n, g = rng.choice((1, 2, 3, 4, 6)), rng.choice((1, 2, 4, 8))
        L = tuple(rng.randint(1, 13) for _ in range(k))
        fa, fb = O.factorisations(n, k), O.factorisations(g, k)
        a, b = fa[rng.randint(0, len(fa) - 1)], fb[rng.randint(0, len(fb) - 1)]
        width = tuple(rng.randint(0, 3) for _ in range(k))
        eb = tuple(rng.randint(1, 9) for _ in range(k))
        p, s = O.hier_costs(L, (n, g), a, b, variant, width, eb)
        ch, dist = hier_chain(k, a, b, variant)
        ln = O.Launch(L, (n, g), ch, dist)
        assert s == ln.halo_elements(width, eb, want_recv=False)[0], (L, n, g, a, b)
        lnode = O.Launch(L, (n, 1), node_chain(k, a), ("block",))
        assert p == lnode.halo_elements(width, eb, want_recv=False)[0], (L, n, g, a, b)


def test_hier_primary_closed_form():
    # extents divisible by the node grid: interior node cuts only
    for L, a, w in (((12, 8, 6), (3, 2, 1), (1, 2, 1)), ((16, 16), (4, 2), (3, 1))):
        n = math.prod(a)
        p, _ = O.hier_costs(L, (n, 2), a, (2,) + (1,) * (len(L) - 1), "block", w, (1,) * len(L))
        assert p == sum(2 * (a[t] - 1) * w[t] * math.prod(L[u] for u in range(len(L)) if u != t)
                        for t in range(len(L)))


def test_hier_cyclic_lower_is_worst_for_stencils():
    # within a node the cyclic lower level puts every neighbour on another
    # GPU once b_t >= 2: its processor volume is never below the block one
    for L in ((16, 8, 8), (12, 12, 6)):
        rb = O.hier_search(L, (2, 4), "block", (1, 1, 1), (1, 1, 1), threads=8)
        rc = O.hier_search(L, (2, 4), "cyclic", (1, 1, 1), (1, 1, 1), threads=8)
        assert rb["primary"] == rc["primary"] and rb["secondary"] <= rc["secondary"]
