"""CPU oracle for the Mapple index-mapping hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (``paper_2507_17087_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``mapple_oracle.cpp`` (plain C++, one point and one
transform at a time, exact integers); this module compiles it with g++ and
wraps it with ctypes.  ``mlp.py`` holds the float64 numpy forward/backward of
the learned cost model.

Chain vocabulary (plain tuples, shared with the tests):
  ("split", i, d)            Fig. 4 split(i, d)
  ("merge", p, q)            Fig. 4 merge(p, q), p < q
  ("swap", p, q)             Fig. 4 swap(p, q)
  ("decompose", i, (l1..lk)) Sec. 4.2 decompose(i, T)
  ("decompose", i, (l1..lk), (h1..hk), (n, ...))
                             the appendix's generalised objective: halo
                             widths h and all-to-all transposes along the
                             listed target dimensions
  ("balance_split", i, k)    read as decompose(i, (1,)*k)
Distributions: ("block",), ("cyclic",), ("block_cyclic", b), ("hier",),
("linear_cyclic",).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mapple_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPS = {"split": 0, "merge": 1, "swap": 2, "decompose": 3, "balance_split": 4}
OP_NAMES = {v: k for k, v in OPS.items()}
DISTS = {"block": 0, "cyclic": 1, "block_cyclic": 2, "hier": 3, "linear_cyclic": 4}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            V, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            launch = [V, I, I, I, V, I, I, I]   # L, k, n, g, xf, nxf, dist, b
            sig = {
                "or_final_shape": (I, launch + [V, V]),
                "or_expand": (I, launch + [V, I]),
                "or_resolve": (I, launch + [V, I64, V, V]),
                "or_map_points": (I, launch + [V, V, I]),
                "or_owner_of": (I, launch + [V, I64, V]),
                "or_map_range": (I, launch + [V, I64, I64, I, V, V]),
                "or_comm_volume": (I, launch + [V, V, V, I]),
                "or_map_launch": (I, launch + [V, V, V, V, V, I]),
                "or_halo_elements": (I, launch + [V, V, V, V, I]),
                "or_decompose_weighted": (I, [I64, I, V, V, I, V]),
                "or_weighted_objective": (I, [I64, I, V, V, V, I, V]),
                "or_halo_closed_form": (I, launch + [V, V]),
                "or_factorisations": (I64, [I64, I, V, I64]),
                "or_decompose": (I, [I64, I, V, V]),
                "or_greedy": (I, [I64, I, V]),
                "or_greedy_workload": (I, [I64, I, V, V]),
                "or_chains": (I64, [I, I, I, V, I64]),
                "or_chain_from_draws": (I, [I, I, I, V, V]),
                "or_matmul_cost": (I, [I64, I64, I64, I, I, V, I, V, I, V, V]),
                "or_search": (I, [I64, I64, I64, I, I, I, I, V]),
                "or_candidate_costs": (I, [I64, I64, I64, I, I, I, V, I64, V, V, I]),
                "or_hier_costs": (I, [V, I, I, I, V, V, I, V, V, I, V, V]),
                "or_hier_search": (I, [V, I, I, I, I, V, V, I, V]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


XF_W = 14


def encode_chain(chain) -> np.ndarray:
    """Chain tuples -> the oracle's 14-int64-per-op array
    [op, i, j, k, d, T0..T3, h0..h3, transpose_mask]."""
    out = np.zeros((max(len(chain), 1), XF_W), dtype=np.int64)
    for o, op in enumerate(chain):
        name = op[0]
        out[o, 0] = OPS[name]
        if name == "split":
            out[o, 1], out[o, 4] = op[1], op[2]
        elif name in ("merge", "swap"):
            out[o, 1], out[o, 2] = op[1], op[2]
        elif name == "decompose":
            T = tuple(op[2])
            out[o, 1], out[o, 3] = op[1], len(T)
            out[o, 5:5 + len(T)] = T
            if len(op) > 3 and op[3] is not None:
                out[o, 9:9 + len(T)] = tuple(op[3])
            if len(op) > 4:
                out[o, 13] = sum(1 << int(n) for n in op[4])
        elif name == "balance_split":
            out[o, 1], out[o, 3] = op[1], op[2]
        else:
            raise ValueError(name)
    return out


def _dist(dist):
    return DISTS[dist[0]], (int(dist[1]) if len(dist) > 1 else 1)


class Launch:
    """One index launch: task space L, machine (n, g), chain, distribution."""

    def __init__(self, L, machine, chain, dist):
        self.L = np.asarray(L, dtype=np.int64)
        self.k = len(L)
        self.n, self.g = int(machine[0]), int(machine[1])
        self.P = self.n * self.g
        self.chain = list(chain)
        self.xf = encode_chain(self.chain)
        self.dk, self.db = _dist(dist)
        self.npoints = int(np.prod(self.L))

    def _args(self):
        return (_p(self.L), self.k, self.n, self.g, _p(self.xf), len(self.chain), self.dk, self.db)

    def final_shape(self):
        lib = _load()
        shape = np.zeros(32, dtype=np.int64)
        r = ctypes.c_int(0)
        rc = lib.or_final_shape(*self._args(), _p(shape), ctypes.byref(r))
        if rc:
            raise ValueError("invalid chain or distribution")
        return tuple(int(v) for v in shape[: r.value])

    def expand(self):
        lib = _load()
        out = np.zeros((256, 4), dtype=np.int64)
        m = lib.or_expand(*self._args(), _p(out), 256)
        if m < 0:
            raise ValueError("invalid chain or distribution")
        return [(OP_NAMES[int(o)], int(p), int(q), int(d)) for o, p, q, d in out[:m]]

    def resolve(self, a):
        """Final-space indices (m x rank) -> (node, proc) arrays."""
        lib = _load()
        a = np.ascontiguousarray(a, dtype=np.int64)
        m = a.shape[0]
        node = np.zeros(m, dtype=np.int64)
        proc = np.zeros(m, dtype=np.int64)
        rc = lib.or_resolve(*self._args(), _p(a), m, _p(node), _p(proc))
        if rc:
            raise ValueError("invalid chain or distribution")
        return node, proc

    def map_points(self, want_ids=True, want_hist=True, threads=1):
        lib = _load()
        ids = np.zeros(self.npoints, dtype=np.int32) if want_ids else None
        hist = np.zeros(self.P, dtype=np.uint64) if want_hist else None
        rc = lib.or_map_points(*self._args(), _p(ids) if ids is not None else None,
                               _p(hist) if hist is not None else None, threads)
        if rc:
            raise ValueError("invalid chain or distribution")
        return ids, hist

    def owner_of(self, lins):
        lib = _load()
        lins = np.ascontiguousarray(lins, dtype=np.int64)
        out = np.zeros(lins.shape[0], dtype=np.int32)
        rc = lib.or_owner_of(*self._args(), _p(lins), lins.shape[0], _p(out))
        if rc:
            raise ValueError("invalid chain or distribution")
        return out

    def map_range(self, face_bytes, lo, count, threads=1):
        """Owners of points [lo, lo+count) and the halo bytes they receive."""
        lib = _load()
        fb = np.zeros(4, dtype=np.uint64)
        fb[: self.k] = face_bytes
        ids = np.zeros(count, dtype=np.int32)
        halo = np.zeros(1, dtype=np.uint64)
        rc = lib.or_map_range(*self._args(), _p(fb), lo, count, threads, _p(ids), _p(halo))
        if rc:
            raise ValueError("invalid chain or distribution")
        return ids, int(halo[0])

    def comm_volume(self, face_bytes, want_recv=True, threads=1):
        lib = _load()
        fb = np.zeros(4, dtype=np.uint64)
        fb[: self.k] = face_bytes
        tot = np.zeros(1, dtype=np.uint64)
        recv = np.zeros(self.P, dtype=np.uint64) if want_recv else None
        rc = lib.or_comm_volume(*self._args(), _p(fb), _p(tot),
                                _p(recv) if recv is not None else None, threads)
        if rc:
            raise ValueError("invalid chain or distribution")
        return int(tot[0]), recv

    def map_launch(self, face_bytes, ids=None, threads=1):
        """ids, histogram, halo total and received bytes in one pass: every
        point's owner evaluated once, each neighbour's owner looked up from
        those ids.  `ids` may be a caller's int32 array of npoints."""
        lib = _load()
        fb = np.zeros(4, dtype=np.uint64)
        fb[: self.k] = face_bytes
        if ids is None:
            ids = np.empty(self.npoints, dtype=np.int32)
        assert ids.dtype == np.int32 and ids.size == self.npoints and ids.flags.c_contiguous
        hist = np.zeros(self.P, dtype=np.uint64)
        tot = np.zeros(1, dtype=np.uint64)
        recv = np.zeros(self.P, dtype=np.uint64)
        rc = lib.or_map_launch(*self._args(), _p(fb), _p(ids), _p(hist), _p(tot), _p(recv), threads)
        if rc:
            raise ValueError("invalid chain or distribution")
        return ids, hist, int(tot[0]), recv

    def halo_elements(self, width, elem_bytes, want_recv=True, threads=1):
        """Anisotropic halo volume in elements: per element and
        dimension, one copy to each other owner within the halo width."""
        lib = _load()
        wd = np.zeros(4, dtype=np.int64)
        wd[: self.k] = width
        eb = np.zeros(4, dtype=np.uint64)
        eb[: self.k] = elem_bytes
        tot = np.zeros(1, dtype=np.uint64)
        recv = np.zeros(self.P, dtype=np.uint64) if want_recv else None
        rc = lib.or_halo_elements(*self._args(), _p(wd), _p(eb), _p(tot),
                                  _p(recv) if recv is not None else None, threads)
        if rc:
            raise ValueError("invalid chain, distribution or width")
        return int(tot[0]), recv

    def halo_closed_form(self, face_bytes):
        lib = _load()
        fb = np.zeros(4, dtype=np.uint64)
        fb[: self.k] = face_bytes
        tot = np.zeros(1, dtype=np.uint64)
        rc = lib.or_halo_closed_form(*self._args(), _p(fb), _p(tot))
        if rc:
            raise ValueError("invalid chain or distribution")
        return int(tot[0])


def factorisations(d: int, k: int):
    lib = _load()
    cnt = lib.or_factorisations(d, k, None, 0)
    out = np.zeros((max(cnt, 1), k), dtype=np.int64)
    lib.or_factorisations(d, k, _p(out), cnt)
    return [tuple(int(v) for v in row) for row in out[:cnt]]


def decompose(d: int, l, h=None, transposes=()):
    """Sec. 4.2 decompose argmin; with halo widths h and/or transposes, the
    appendix's generalised objective."""
    lib = _load()
    l = np.asarray(l, dtype=np.int64)
    out = np.zeros(len(l), dtype=np.int64)
    if h is None and not transposes:
        if lib.or_decompose(d, len(l), _p(l), _p(out)):
            raise ValueError("bad decompose")
    else:
        hw = np.asarray(h if h is not None else [1] * len(l), dtype=np.int64)
        mask = sum(1 << int(n) for n in transposes)
        rc = lib.or_decompose_weighted(d, len(l), _p(l), _p(hw), mask, _p(out))
        if rc:
            raise (OverflowError if rc == 2 else ValueError)("bad decompose")
    return tuple(int(v) for v in out)


def weighted_objective(d: int, f, l, h, transposes=()):
    """d * (V + sum_T V*_n) of one factorisation f (exact integer)."""
    lib = _load()
    f = np.asarray(f, dtype=np.int64)
    l = np.asarray(l, dtype=np.int64)
    hw = np.asarray(h, dtype=np.int64)
    out = np.zeros(2, dtype=np.int64)
    mask = sum(1 << int(n) for n in transposes)
    if lib.or_weighted_objective(d, len(l), _p(f), _p(l), _p(hw), mask, _p(out)):
        raise OverflowError("objective overflow")
    return (int(out[0]) << 64) + (int(out[1]) & ((1 << 64) - 1))


def greedy(d: int, k: int):
    lib = _load()
    out = np.zeros(k, dtype=np.int64)
    if lib.or_greedy(d, k, _p(out)):
        raise ValueError("bad greedy")
    return tuple(int(v) for v in out)


def chains(n: int, g: int, max_depth: int):
    """Canonical chains of depth <= max_depth on (n, g) as tuples of ops."""
    lib = _load()
    cnt = lib.or_chains(n, g, max_depth, None, 0)
    D = max(max_depth, 1)
    out = np.zeros((cnt, D, 4), dtype=np.int64)
    lib.or_chains(n, g, max_depth, _p(out), cnt)
    res = []
    for c in range(cnt):
        ops = []
        for o in range(max_depth):
            op, p, q, d = (int(v) for v in out[c, o])
            if op < 0:
                break
            ops.append(("split", p, d) if op == 0 else (OP_NAMES[op], p, q))
        res.append(tuple(ops))
    return res


def chain_from_draws(n: int, g: int, draws):
    lib = _load()
    draws = np.ascontiguousarray(draws, dtype=np.uint64)
    out = np.zeros((max(len(draws), 1), XF_W), dtype=np.int64)
    m = lib.or_chain_from_draws(n, g, len(draws), _p(draws), _p(out))
    res = []
    for o in range(m):
        op = int(out[o, 0])
        if op == 0:
            res.append(("split", int(out[o, 1]), int(out[o, 4])))
        else:
            res.append((OP_NAMES[op], int(out[o, 1]), int(out[o, 2])))
    return res


def _chain_ops(chain, depth):
    arr = np.full((max(depth, 1), 4), 0, dtype=np.int64)
    arr[:, 0] = -1
    for o, op in enumerate(chain):
        if op[0] == "split":
            arr[o] = (0, op[1], -1, op[2])
        else:
            arr[o] = (OPS[op[0]], op[1], op[2], 0)
    return arr


def matmul_cost(M, N, K, machine, chain, f, literal=False):
    """(primary, secondary) moved tiles of one candidate: per operand tile,
    distinct processors - 1 and distinct nodes - 1."""
    lib = _load()
    n, g = machine
    depth = max(len(chain), 1)
    ch = _chain_ops(chain, depth)
    f = np.asarray(f, dtype=np.int64)
    p = ctypes.c_int64(0)
    s = ctypes.c_int64(0)
    rc = lib.or_matmul_cost(M, N, K, n, g, _p(ch), depth, _p(f), 0 if literal else 1,
                            ctypes.byref(p), ctypes.byref(s))
    if rc:
        raise ValueError("bad candidate")
    return p.value, s.value


def search(M, N, K, machine, max_depth=3, threads=1):
    """Exhaustive lexicographic argmin over (factorisation, chain).  Costs in tiles."""
    lib = _load()
    n, g = machine
    out = np.zeros(8, dtype=np.int64)
    lib.or_search(M, N, K, n, g, max_depth, threads, _p(out))
    return {"index": int(out[0]), "f": tuple(int(v) for v in out[1:4]), "chain_rank": int(out[4]),
            "primary": int(out[5]), "secondary": int(out[6]), "n_candidates": int(out[7])}


def candidate_costs(M, N, K, machine, max_depth, indices, threads=1):
    lib = _load()
    n, g = machine
    idx = np.ascontiguousarray(indices, dtype=np.int64)
    p = np.zeros(idx.shape[0], dtype=np.int64)
    s = np.zeros(idx.shape[0], dtype=np.int64)
    if lib.or_candidate_costs(M, N, K, n, g, max_depth, _p(idx), idx.shape[0], _p(p), _p(s), threads):
        raise ValueError("bad candidate index")
    return p, s


def greedy_workload(d: int, l):
    """Sec. 4.3's workload-balancing greedy (the counterexample to greedy)."""
    lib = _load()
    l = np.asarray(l, dtype=np.int64)
    out = np.zeros(len(l), dtype=np.int64)
    if lib.or_greedy_workload(d, len(l), _p(l), _p(out)):
        raise ValueError("bad greedy")
    return tuple(int(v) for v in out)


HIER_VARIANTS = {"block": 0, "cyclic": 1}


def _hier_args(L, width, elem_bytes):
    k = len(L)
    Lv = np.asarray(L, dtype=np.int64)
    wd = np.zeros(4, dtype=np.int64)
    wd[:k] = width
    eb = np.zeros(4, dtype=np.uint64)
    eb[:k] = elem_bytes
    return k, Lv, wd, eb


def hier_costs(L, machine, a, b, variant, width, elem_bytes, threads=1):
    """(inter-node, inter-processor) element halo bytes of the two-level
    mapping with node grid a and GPU grid b."""
    lib = _load()
    k, Lv, wd, eb = _hier_args(L, width, elem_bytes)
    av = np.asarray(a, dtype=np.int64)
    bv = np.asarray(b, dtype=np.int64)
    p = np.zeros(1, dtype=np.uint64)
    s = np.zeros(1, dtype=np.uint64)
    if lib.or_hier_costs(_p(Lv), k, machine[0], machine[1], _p(av), _p(bv), HIER_VARIANTS[variant], _p(wd), _p(eb),
                         threads, _p(p), _p(s)):
        raise ValueError("bad hierarchical candidate")
    return int(p[0]), int(s[0])


def hier_search(L, machine, variant, width, elem_bytes, threads=1):
    """Exhaustive lexicographic argmin over (node grid, GPU grid)."""
    lib = _load()
    k, Lv, wd, eb = _hier_args(L, width, elem_bytes)
    out = np.zeros(12, dtype=np.int64)
    if lib.or_hier_search(_p(Lv), k, machine[0], machine[1], HIER_VARIANTS[variant], _p(wd), _p(eb), threads,
                          _p(out)):
        raise ValueError("bad hierarchical query")
    return {"index": int(out[0]), "a": tuple(int(v) for v in out[1:1 + k]),
            "b": tuple(int(v) for v in out[5:5 + k]), "primary": int(out[9]), "secondary": int(out[10]),
            "n_candidates": int(out[11])}
