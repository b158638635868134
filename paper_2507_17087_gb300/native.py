"""Thin ctypes binding of the engine's C ABI (include/mapple.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libmapple_gb300.so``.  There is no CPU fallback: if the library
has not been built, every call raises.

Buffers may be torch tensors (CUDA or CPU), numpy arrays, or raw integer
pointers.  ``stream`` defaults to torch's current CUDA stream.

Chain vocabulary (plain tuples):
  ("split", i, d), ("merge", p, q), ("swap", p, q),
  ("decompose", i, (l1..lk)), ("balance_split", i, k)
Distributions: ("block",), ("cyclic",), ("block_cyclic", b), ("hier",),
("linear_cyclic",).
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

OPS = {"split": 0, "merge": 1, "swap": 2, "decompose": 3, "balance_split": 4}
OP_NAMES = {v: k for k, v in OPS.items()}
DISTS = {"block": 0, "cyclic": 1, "block_cyclic": 2, "hier": 3, "linear_cyclic": 4}
STATUS = {0: "MP_OK", 1: "MP_EINVAL", 2: "MP_EOVERFLOW", 3: "MP_ENOMEM", 4: "MP_ECUDA",
          5: "MP_ETIMEOUT", 6: "MP_ENOTSUP"}


class MapleError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = ""
        if status == 4:
            try:
                detail = " at " + lib().mp_last_error_detail().decode()
            except Exception:  # noqa: BLE001 - formatting another error
                pass
        super().__init__(f"{where}: {STATUS.get(status, status)} ({strerror(status)}){detail}")


class mp_space(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("reserved", ctypes.c_int32), ("ext", ctypes.c_int64 * 4)]


class mp_machine(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_int32), ("procs_per_node", ctypes.c_int32)]


class mp_xform(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("i", ctypes.c_int32), ("j", ctypes.c_int32),
                ("k", ctypes.c_int32), ("d", ctypes.c_int64), ("T", ctypes.c_int64 * 4),
                ("h", ctypes.c_int32 * 4), ("transpose", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mp_halo(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("width", ctypes.c_int32 * 4), ("reserved", ctypes.c_int32),
                ("bytes", ctypes.c_uint64 * 4)]


HALO_FACES = 0
HALO_ELEMENTS = 1
MAX_HALO_WIDTH = 16
HIER_VARIANTS = {"block": 0, "cyclic": 1}


class mp_dist(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("b", ctypes.c_int32)]


class mp_hier_query(ctypes.Structure):
    _fields_ = [("space", mp_space), ("machine", mp_machine), ("variant", ctypes.c_int32),
                ("width", ctypes.c_int32 * 4), ("bytes", ctypes.c_uint64 * 4)]


class mp_hier_result(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int64), ("a", ctypes.c_int64 * 4), ("b", ctypes.c_int64 * 4),
                ("primary_bytes", ctypes.c_uint64), ("secondary_bytes", ctypes.c_uint64),
                ("n_candidates", ctypes.c_int64)]


class mp_query(ctypes.Structure):
    _fields_ = [("space", mp_space), ("machine", mp_machine), ("chain", ctypes.c_void_p),
                ("n_xf", ctypes.c_int32), ("reserved", ctypes.c_int32), ("dist", mp_dist),
                ("face_bytes", ctypes.c_uint64 * 4)]


class mp_search_query(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64),
                ("procs", ctypes.c_int32), ("procs_per_node", ctypes.c_int32),
                ("max_depth", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tile_bytes", ctypes.c_uint64)]


class mp_search_result(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int64), ("f", ctypes.c_int64 * 3), ("chain_rank", ctypes.c_int64),
                ("chain_len", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("chain", mp_xform * 4), ("primary_bytes", ctypes.c_uint64),
                ("secondary_bytes", ctypes.c_uint64), ("n_candidates", ctypes.c_int64),
                ("n_chains", ctypes.c_int64), ("n_factorisations", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded engine library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libmapple_gb300.so is not built: run __graft_entry__.build() "
                                   "(the engine has no CPU fallback)")
            L = ctypes.CDLL(_build.LIB)
            V, I, I64, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
            sig = {
                "mp_map_points": (I, [V, V, V, I, V, V, V, V]),
                "mp_map_points_noalloc": (I, [V, V, V, I, V, V, V, V]),
                "mp_comm_volume": (I, [V, V, V, I, V, V, V, V, V]),
                "mp_halo_volume": (I, [V, V, V, I, V, V, V, V, V]),
                "mp_map_launch": (I, [V, V, V, I, V, V, V, V, V, V, V]),
                "mp_greedy_grid": (I, [I64, I, V]),
                "mp_batch_set_tile": (I, [V, I]),
                "mp_mlp_save": (I, [V, ctypes.c_char_p]),
                "mp_mlp_load": (I, [V, ctypes.c_char_p]),
                "mp_selftest_wait_timeout": (I, [ctypes.c_uint32, V]),
                "mp_debug_fail_allocations": (I, [I]),
                "mp_secondary_lower_bound": (I, [V, V, V]),
                "mp_hier_search": (I, [V, V, V]),
                "mp_hier_chain": (I, [I, V, V, I, V, V, V]),
                "mp_decompose_search": (I, [V, I, V, V]),
                "mp_candidate_costs": (I, [V, V, I64, V, V, V]),
                "mp_plan": (I, [V, V, V, I, V, V, V, V, V, I]),
                "mp_chain_from_draws": (I, [I, I, I, V, V, V]),
                "mp_search_space": (I, [I, I, I, V, V]),
                "mp_search_candidate": (I, [V, I64, V, V, V]),
                "mp_strerror": (ctypes.c_char_p, [I]),
                "mp_last_error_detail": (ctypes.c_char_p, []),
                "mp_kernel_launches": (U64, []),
                "mp_workspace_bytes": (U64, []),
                "mp_set_kernel_timer": (I, [V, V]),
                "mp_set_layer_timer": (I, [V, V]),
                "mp_batch_create": (I, [V, I, V]),
                "mp_batch_info": (I, [V, V, V, V, V, V]),
                "mp_batch_run": (I, [V, V, V, V, V, I, V]),
                "mp_batch_destroy": (I, [V]),
                "mp_gemm_bf16": (I, [V, V, V, I, I, I, V]),
                "mp_mlp_create": (I, [ctypes.c_uint64, V]),
                "mp_mlp_destroy": (I, [V]),
                "mp_mlp_num_params": (I, []),
                "mp_mlp_set_params": (I, [V, V]),
                "mp_mlp_get_params": (I, [V, V, V]),
                "mp_mlp_forward": (I, [V, V, V, I, V]),
                "mp_mlp_train_step": (I, [V, V, V, I, ctypes.c_float, V, V]),
                "mp_mlp_train_search": (I, [V, V, I, I, I, I, ctypes.c_float, ctypes.c_uint64, V, V]),
                "mp_learned_search": (I, [V, V, I, I, V, V, V]),
                "mp_mlp_calibrate": (I, [V, V, I, V, V]),
                "mp_mlp_set_margin_bound": (I, [V, ctypes.c_double]),
                "mp_learned_scores": (I, [V, V, V, V, V, V]),
                "mp_descriptor_bytes": (U64, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().mp_strerror(status).decode()
    except Exception:  # noqa: BLE001 - used while formatting another error
        return "?"


def _check(rc: int, where: str):
    if rc != 0:
        raise MapleError(rc, where)


# ----------------------------------------------------------------- marshalling

def make_space(L) -> mp_space:
    s = mp_space()
    s.rank = len(L)
    for t, v in enumerate(L):
        s.ext[t] = int(v)
    return s


def make_machine(machine) -> mp_machine:
    m = mp_machine()
    m.nodes, m.procs_per_node = int(machine[0]), int(machine[1])
    return m


def make_chain(chain):
    n = len(chain)
    arr = (mp_xform * max(n, 1))()
    for o, op in enumerate(chain):
        x = arr[o]
        name = op[0]
        x.op = OPS[name]
        if name == "split":
            x.i, x.d = int(op[1]), int(op[2])
        elif name in ("merge", "swap"):
            x.i, x.j = int(op[1]), int(op[2])
        elif name == "decompose":
            T = tuple(op[2])
            x.i, x.k = int(op[1]), len(T)
            for m, v in enumerate(T):
                x.T[m] = int(v)
            if len(op) > 3 and op[3] is not None:
                for m, v in enumerate(op[3]):
                    x.h[m] = int(v)
            if len(op) > 4:
                x.transpose = sum(1 << int(m) for m in op[4])
        elif name == "balance_split":
            x.i, x.k = int(op[1]), int(op[2])
        else:
            raise ValueError(f"unknown transform {name!r}")
    return arr, n


_XFORM_DTYPE = np.dtype(mp_xform)
_QUERY_DTYPE = np.dtype(mp_query)


def _xform_row(op):
    """One transform as a record of mp_xform's layout (see make_chain)."""
    name = op[0]
    i = j = k = d = tr = 0
    T, h = (0, 0, 0, 0), (0, 0, 0, 0)
    if name == "split":
        i, d = int(op[1]), int(op[2])
    elif name in ("merge", "swap"):
        i, j = int(op[1]), int(op[2])
    elif name == "decompose":
        Tl = tuple(int(v) for v in op[2])
        i, k = int(op[1]), len(Tl)
        T = Tl + (0,) * (4 - k)
        if len(op) > 3 and op[3] is not None:
            hl = tuple(int(v) for v in op[3])
            h = hl + (0,) * (4 - len(hl))
        if len(op) > 4:
            tr = sum(1 << int(m) for m in op[4])
    elif name == "balance_split":
        i, k = int(op[1]), int(op[2])
    else:
        raise ValueError(f"unknown transform {name!r}")
    return (OPS[name], i, j, k, d, T, h, tr, 0)


def query_records(launches):
    """(L, machine, chain, dist, face_bytes) tuples as numpy records with the
    layouts of mp_xform (every chain, one after the other) and mp_query (the
    chain field pointing into the first array, which must outlive the use)."""
    xrows, qrows = [], []
    for L, machine, chain, dist, face in launches:
        first = len(xrows)
        xrows.extend(_xform_row(op) for op in chain)
        ext = tuple(int(v) for v in L) + (0,) * (4 - len(L))
        fb = tuple(int(v) for v in face) + (0,) * (4 - len(face))
        qrows.append(((len(L), 0, ext), (int(machine[0]), int(machine[1])), first, len(chain), 0,
                      (DISTS[dist[0]], int(dist[1]) if len(dist) > 1 else 1), fb))
    xf = np.array(xrows or [_xform_row(("split", 0, 1))], dtype=_XFORM_DTYPE)
    qs = np.array(qrows, dtype=_QUERY_DTYPE)
    qs["chain"] = xf.ctypes.data + qs["chain"] * _XFORM_DTYPE.itemsize
    return xf, qs


def make_dist(dist) -> mp_dist:
    d = mp_dist()
    d.kind = DISTS[dist[0]]
    d.b = int(dist[1]) if len(dist) > 1 else 1
    return d


def _ptr(buf):
    """Raw address of a torch tensor, numpy array or int (None -> NULL)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _stream(stream):
    if stream is not None:
        return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def resolve_chain(machine, chain=None, draws=None):
    """Explicit chain tuples, or a canonical chain built from draws."""
    if chain is not None:
        return list(chain)
    return chain_from_draws(machine[0], machine[1], draws or [])


# ----------------------------------------------------------------- entry points

def map_points(L, machine, chain, dist, ids=None, hist=None, stream=None):
    """ids[lin] (int32, C order) and hist[P] (uint64) of one launch."""
    sp, mc, ds = make_space(L), make_machine(machine), make_dist(dist)
    ch, n = make_chain(chain)
    rc = lib().mp_map_points(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds),
                             _ptr(ids), _ptr(hist), _stream(stream))
    _check(rc, "mp_map_points")


def map_points_noalloc(L, machine, chain, dist, ids=None, hist=None, stream=None):
    """map_points with its scratch in the library's fixed 8 MiB device array.

    For callers that cannot allocate device memory (a framework that owns the
    whole device budget, latency-critical loops that cannot absorb
    cudaMalloc's device-wide synchronisation).  ids / hist must be device
    memory.  Calls share the one array: do not overlap them on the GPU.
    """
    sp, mc, ds = make_space(L), make_machine(machine), make_dist(dist)
    ch, n = make_chain(chain)
    rc = lib().mp_map_points_noalloc(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds),
                                     _ptr(ids), _ptr(hist), _stream(stream))
    _check(rc, "mp_map_points_noalloc")


def comm_volume(L, machine, chain, dist, face_bytes, total, recv=None, stream=None):
    """total[0] (uint64) = halo bytes; recv[P] = bytes received per processor."""
    sp, mc, ds = make_space(L), make_machine(machine), make_dist(dist)
    ch, n = make_chain(chain)
    fb = (ctypes.c_uint64 * 4)(*([int(v) for v in face_bytes] + [0] * (4 - len(face_bytes))))
    rc = lib().mp_comm_volume(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds), fb,
                              _ptr(total), _ptr(recv), _stream(stream))
    _check(rc, "mp_comm_volume")


def _halo(width, elem_bytes, elements):
    h = mp_halo()
    h.mode = HALO_ELEMENTS if elements else HALO_FACES
    for t, v in enumerate(width):
        h.width[t] = int(v)
    for t, v in enumerate(elem_bytes):
        h.bytes[t] = int(v)
    return h


def map_launch(L, machine, chain, dist, ids=None, hist=None, face_bytes=None, total=None, recv=None,
               width=None, elements=False, stream=None):
    """mp_map_launch: ids, histogram and halo of one launch in one call
    (face_bytes per dimension; width for the element count)."""
    sp, mc, ds = make_space(L), make_machine(machine), make_dist(dist)
    ch, n = make_chain(chain)
    h = None
    if face_bytes is not None:
        h = _halo(width if width is not None else [1] * len(L), face_bytes, elements)
    rc = lib().mp_map_launch(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds),
                             ctypes.byref(h) if h is not None else None, _ptr(ids), _ptr(hist), _ptr(total),
                             _ptr(recv), _stream(stream))
    _check(rc, "mp_map_launch")


def halo_volume(L, machine, chain, dist, width, elem_bytes, total, recv=None, elements=True, stream=None):
    """mp_halo_volume: the element count with per-dimension halo widths
    (elements=True) or the directed face count."""
    sp, mc, ds = make_space(L), make_machine(machine), make_dist(dist)
    ch, n = make_chain(chain)
    h = mp_halo()
    h.mode = HALO_ELEMENTS if elements else HALO_FACES
    for t, v in enumerate(width):
        h.width[t] = int(v)
    for t, v in enumerate(elem_bytes):
        h.bytes[t] = int(v)
    rc = lib().mp_halo_volume(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds), ctypes.byref(h),
                              _ptr(total), _ptr(recv), _stream(stream))
    _check(rc, "mp_halo_volume")


def hier_chain(a, b, variant):
    """(chain, distribution) realising the two-level candidate (a, b)."""
    k = len(a)
    av = (ctypes.c_int64 * 4)(*[int(v) for v in a], *([0] * (4 - k)))
    bv = (ctypes.c_int64 * 4)(*[int(v) for v in b], *([0] * (4 - k)))
    ch = (mp_xform * 16)()
    n = ctypes.c_int32(0)
    d = mp_dist()
    _check(lib().mp_hier_chain(k, av, bv, HIER_VARIANTS[variant], ch, ctypes.byref(n), ctypes.byref(d)),
           "mp_hier_chain")
    kind = {v: k_ for k_, v in DISTS.items()}[d.kind]
    return [xform_tuple(ch[o]) for o in range(n.value)], (kind,)


def hier_search(L, machine, variant, width, elem_bytes, stream=None):
    """mp_hier_search: the two-level (node grid, GPU grid) argmin."""
    q = mp_hier_query()
    q.space = make_space(L)
    q.machine = make_machine(machine)
    q.variant = HIER_VARIANTS[variant]
    for t, v in enumerate(width):
        q.width[t] = int(v)
    for t, v in enumerate(elem_bytes):
        q.bytes[t] = int(v)
    r = mp_hier_result()
    _check(lib().mp_hier_search(ctypes.byref(q), ctypes.byref(r), _stream(stream)), "mp_hier_search")
    k = len(L)
    return {"index": r.index, "a": tuple(r.a[:k]), "b": tuple(r.b[:k]), "primary": r.primary_bytes,
            "secondary": r.secondary_bytes, "n_candidates": r.n_candidates}


def selftest_wait_timeout(limit=1000, stream=None):
    """Status of a bounded wait that nothing completes (MP_ETIMEOUT)."""
    return lib().mp_selftest_wait_timeout(int(limit), _stream(stream))


def debug_fail_allocations(n):
    """Make the next n device workspace requests fail (host-side injection)."""
    _check(lib().mp_debug_fail_allocations(int(n)), "mp_debug_fail_allocations")


def greedy_grid(d, k):
    """Algorithm A1's processor grid (host only)."""
    out = (ctypes.c_int64 * 4)()
    _check(lib().mp_greedy_grid(int(d), int(k), out), "mp_greedy_grid")
    return tuple(out[m] for m in range(k))


def plan(L, machine, chain, dist):
    """(final shape, expanded primitives) -- host planning only, no GPU."""
    sp, mc, ds = make_space(L), make_machine(machine), make_dist(dist)
    ch, n = make_chain(chain)
    rank = ctypes.c_int32(0)
    shape = (ctypes.c_int64 * 32)()
    nprim = ctypes.c_int32(0)
    prims = (ctypes.c_int64 * (4 * 256))()
    rc = lib().mp_plan(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds),
                       ctypes.byref(rank), shape, ctypes.byref(nprim), prims, 256)
    _check(rc, "mp_plan")
    out = []
    for o in range(min(nprim.value, 256)):
        op, p, q, d = prims[4 * o:4 * o + 4]
        out.append((OP_NAMES[op], p, q, d))
    return tuple(shape[: rank.value]), out


def plan_status(L, machine, chain, dist) -> int:
    sp, mc, ds = make_space(L), make_machine(machine), make_dist(dist)
    ch, n = make_chain(chain)
    return lib().mp_plan(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds),
                         None, None, None, None, 0)


def chain_from_draws(nodes, procs_per_node, draws):
    d = np.ascontiguousarray(np.asarray(draws, dtype=np.uint64))
    out = (mp_xform * max(len(d), 1))()
    n = ctypes.c_int32(0)
    rc = lib().mp_chain_from_draws(int(nodes), int(procs_per_node), len(d),
                                   d.ctypes.data if len(d) else None, out, ctypes.byref(n))
    _check(rc, "mp_chain_from_draws")
    return [xform_tuple(out[o]) for o in range(n.value)]


def xform_tuple(x):
    name = OP_NAMES[x.op]
    if name == "split":
        return ("split", x.i, x.d)
    if name in ("merge", "swap"):
        return (name, x.i, x.j)
    if name == "decompose":
        T = tuple(x.T[m] for m in range(x.k))
        h = tuple(x.h[m] for m in range(x.k))
        tr = tuple(m for m in range(x.k) if (x.transpose >> m) & 1)
        if any(h) or tr:
            return ("decompose", x.i, T, h if any(h) else None, tr)
        return ("decompose", x.i, T)
    return ("balance_split", x.i, x.k)


def search_space(procs, procs_per_node, max_depth):
    nf, nc = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().mp_search_space(procs, procs_per_node, max_depth, ctypes.byref(nf), ctypes.byref(nc)),
           "mp_search_space")
    return nf.value, nc.value


SEARCH_FULL = 1


def make_query(M, N, K, procs, procs_per_node, max_depth=3, tile_bytes=512 * 512 * 4, full=False):
    q = mp_search_query()
    q.flags = SEARCH_FULL if full else 0
    q.M, q.N, q.K = int(M), int(N), int(K)
    q.procs, q.procs_per_node, q.max_depth = int(procs), int(procs_per_node), int(max_depth)
    q.tile_bytes = int(tile_bytes)
    return q


def decompose_search(queries, full=False, stream=None):
    """queries: list of mp_search_query (or dicts from workloads.search_queries)."""
    qs = [q if isinstance(q, mp_search_query) else
          make_query(*q["MNK"], q["machine"][0] * q["machine"][1], q["machine"][1],
                     q["max_depth"], q["tile_bytes"], full=full) for q in queries]
    arr = (mp_search_query * len(qs))(*qs)
    out = (mp_search_result * len(qs))()
    _check(lib().mp_decompose_search(arr, len(qs), out, _stream(stream)), "mp_decompose_search")
    res = []
    for r in out:
        res.append({"index": r.index, "f": tuple(r.f), "chain_rank": r.chain_rank,
                    "chain": tuple(xform_tuple(r.chain[o]) for o in range(r.chain_len)),
                    "primary_bytes": r.primary_bytes, "secondary_bytes": r.secondary_bytes,
                    "n_candidates": r.n_candidates, "n_chains": r.n_chains,
                    "n_factorisations": r.n_factorisations})
    return res


def _query(q, full=False):
    if isinstance(q, mp_search_query):
        return q
    return make_query(*q["MNK"], q["machine"][0] * q["machine"][1], q["machine"][1], q["max_depth"],
                      q["tile_bytes"], full=full)


def secondary_lower_bound(query, f):
    """Lower bound (bytes) on the secondary cost of factorisation f over
    every chain (host only)."""
    q = _query(query)
    fv = (ctypes.c_int64 * 3)(*[int(v) for v in f])
    lb = ctypes.c_uint64(0)
    _check(lib().mp_secondary_lower_bound(ctypes.byref(q), fv, ctypes.byref(lb)), "mp_secondary_lower_bound")
    return lb.value


def search_candidate(query, index):
    """(f, chain) of candidate `index` of a search query (host only)."""
    q = _query(query)
    f = (ctypes.c_int64 * 3)()
    ch = (mp_xform * 4)()
    n = ctypes.c_int32(0)
    _check(lib().mp_search_candidate(ctypes.byref(q), int(index), f, ch, ctypes.byref(n)),
           "mp_search_candidate")
    return tuple(f), tuple(xform_tuple(ch[o]) for o in range(n.value))


def candidate_costs(query, indices, primary, secondary, stream=None):
    q = query if isinstance(query, mp_search_query) else \
        make_query(*query["MNK"], query["machine"][0] * query["machine"][1], query["machine"][1],
                   query["max_depth"], query["tile_bytes"])
    n = len(indices)
    _check(lib().mp_candidate_costs(ctypes.byref(q), _ptr(indices), n, _ptr(primary), _ptr(secondary),
                                    _stream(stream)), "mp_candidate_costs")


def kernel_launches() -> int:
    return int(lib().mp_kernel_launches())


def workspace_bytes() -> int:
    """Device workspace the library holds on the current device."""
    return int(lib().mp_workspace_bytes())


def set_kernel_timer(start_event, stop_event):
    """Time the next id-writer kernel with two cudaEvent_t handles (or torch events)."""
    h = lambda e: None if e is None else (e.cuda_event if hasattr(e, "cuda_event") else int(e))
    _check(lib().mp_set_kernel_timer(h(start_event), h(stop_event)), "mp_set_kernel_timer")


def set_layer_timer(start_event, stop_event):
    """Time the learned scorer's next layer-kernel launch (mp_set_layer_timer)."""
    h = lambda e: None if e is None else (e.cuda_event if hasattr(e, "cuda_event") else int(e))
    _check(lib().mp_set_layer_timer(h(start_event), h(stop_event)), "mp_set_layer_timer")


def descriptor_bytes() -> int:
    return int(lib().mp_descriptor_bytes())


BATCH_AUTOTUNE = 1
BATCH_NO_GRAPH = 2


class Batch:
    """A planned batch of mapping queries (mp_batch_create / mp_batch_run).

    launches: iterable of (L, machine, chain, dist, face_bytes) tuples.
    """

    def __init__(self, launches):
        launches = list(launches)
        self.n = len(launches)
        self._launches = launches
        self._signature = None
        self._xf, self._qs = query_records(launches)
        self._h = ctypes.c_void_p()
        _check(lib().mp_batch_create(self._qs.ctypes.data, self.n, ctypes.byref(self._h)), "mp_batch_create")

    @property
    def signature(self):
        """Identifies the batch's queries (for the persisted autotune choice)."""
        if self._signature is None:
            self._signature = hashlib.sha256(repr([(tuple(L), tuple(m), [tuple(o) for o in ch], tuple(d), tuple(f))
                                                   for L, m, ch, d, f in self._launches]).encode()).hexdigest()
        return self._signature

    def info(self):
        ti, tp = ctypes.c_uint64(0), ctypes.c_uint64(0)
        io = np.zeros(self.n + 1, dtype=np.uint64)
        po = np.zeros(self.n + 1, dtype=np.uint64)
        tg = ctypes.c_int32(0)
        _check(lib().mp_batch_info(self._h, ctypes.byref(ti), ctypes.byref(tp), io.ctypes.data,
                                   po.ctypes.data, ctypes.byref(tg)), "mp_batch_info")
        return {"total_ids": ti.value, "total_procs": tp.value, "ids_offsets": io, "proc_offsets": po,
                "tile_groups": tg.value}

    def set_tile(self, tile_groups):
        _check(lib().mp_batch_set_tile(self._h, int(tile_groups)), "mp_batch_set_tile")

    def autotune_cached(self, cache_path, ids, stream=None):
        """The id writer's tile size from a JSON cache (version 1, keyed by
        the batch signature), or autotuned now and recorded there."""
        cache = {"version": 1, "tiles": {}}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                loaded = json.load(f)
            if loaded.get("version") == 1 and isinstance(loaded.get("tiles"), dict):
                cache = loaded
        tile = cache["tiles"].get(self.signature)
        if tile is not None:
            self.set_tile(tile)
            return int(tile)
        self.run(ids=ids, autotune=True, stream=stream)
        cache["tiles"][self.signature] = int(self.info()["tile_groups"])
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, cache_path)
        return cache["tiles"][self.signature]

    def run(self, ids=None, hist=None, halo=None, recv=None, autotune=False, graph=True, stream=None):
        flags = (BATCH_AUTOTUNE if autotune else 0) | (0 if graph else BATCH_NO_GRAPH)
        _check(lib().mp_batch_run(self._h, _ptr(ids), _ptr(hist), _ptr(halo), _ptr(recv), flags,
                                  _stream(stream)), "mp_batch_run")

    def close(self):
        if self._h:
            lib().mp_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def gemm_bf16(A, B, C, stream=None):
    """C = A @ B.T on the tcgen05 tensor cores (A, B bfloat16, C float32)."""
    M, K = A.shape
    N = B.shape[0]
    _check(lib().mp_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), M, N, K, _stream(stream)), "mp_gemm_bf16")


class mp_learned_stats(ctypes.Structure):
    _fields_ = [("n_scored", ctypes.c_int64), ("n_exact", ctypes.c_int64), ("n_selected", ctypes.c_int64),
                ("certified", ctypes.c_int32), ("fallback", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("margin", ctypes.c_double), ("max_overestimate", ctypes.c_double),
                ("margin_bound", ctypes.c_double), ("ms_prepare", ctypes.c_double), ("ms_model", ctypes.c_double),
                ("ms_exact", ctypes.c_double), ("ms_wall", ctypes.c_double), ("ms_fallback", ctypes.c_double)]


CERTIFIED = {0: "none", 1: "every threat evaluated", 2: "secondary lower bound", 3: "margin rule"}


LEARNED_NO_FALLBACK = 1
LEARNED_SCORE_ALL = 2
PARAM_BLOCKS = [("W1", (256, 64)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
                ("b3", (256,)), ("w4", (256,)), ("b4", (1,))]


def _search_result(r):
    return {"index": r.index, "f": tuple(r.f), "chain_rank": r.chain_rank,
            "chain": tuple(xform_tuple(r.chain[o]) for o in range(r.chain_len)),
            "primary_bytes": r.primary_bytes, "secondary_bytes": r.secondary_bytes,
            "n_candidates": r.n_candidates, "n_chains": r.n_chains, "n_factorisations": r.n_factorisations}


class MLP:
    """The learned cost model (mp_mlp_*), parameters on the current device."""

    def __init__(self, seed=0):
        self._h = ctypes.c_void_p()
        _check(lib().mp_mlp_create(int(seed), ctypes.byref(self._h)), "mp_mlp_create")
        self.nparams = lib().mp_mlp_num_params()

    def set_params(self, params: dict):
        flat = np.concatenate([np.asarray(params[k], dtype=np.float32).reshape(-1) for k, _ in PARAM_BLOCKS])
        assert flat.size == self.nparams
        _check(lib().mp_mlp_set_params(self._h, flat.ctypes.data), "mp_mlp_set_params")

    def get_params(self, grads=False):
        p = np.zeros(self.nparams, dtype=np.float32)
        g = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().mp_mlp_get_params(self._h, p.ctypes.data, g.ctypes.data), "mp_mlp_get_params")
        out, o = {}, 0
        src = g if grads else p
        for k, shape in PARAM_BLOCKS:
            n = int(np.prod(shape))
            out[k] = src[o:o + n].reshape(shape).astype(np.float64)
            o += n
        return out

    def forward(self, X, y, stream=None):
        _check(lib().mp_mlp_forward(self._h, _ptr(X), _ptr(y), X.shape[0], _stream(stream)), "mp_mlp_forward")

    def train_step(self, X, target, lr, stream=None):
        loss = ctypes.c_float(0)
        _check(lib().mp_mlp_train_step(self._h, _ptr(X), _ptr(target), X.shape[0], ctypes.c_float(lr),
                                       ctypes.byref(loss), _stream(stream)), "mp_mlp_train_step")
        return loss.value

    def train_search(self, queries, samples_per_query=2048, epochs=4, batch=4096, lr=1e-3, seed=1, stream=None):
        qs = [_query(q) for q in queries]
        arr = (mp_search_query * len(qs))(*qs)
        loss = ctypes.c_float(0)
        _check(lib().mp_mlp_train_search(self._h, arr, len(qs), samples_per_query, epochs, batch,
                                         ctypes.c_float(lr), int(seed), ctypes.byref(loss), _stream(stream)),
               "mp_mlp_train_search")
        return loss.value

    def learned_search(self, query, K=1024, fallback=True, score_all=False, stream=None):
        q = _query(query)
        out = mp_search_result()
        st = mp_learned_stats()
        flags = (0 if fallback else LEARNED_NO_FALLBACK) | (LEARNED_SCORE_ALL if score_all else 0)
        _check(lib().mp_learned_search(self._h, ctypes.byref(q), int(K), flags, ctypes.byref(out),
                                       ctypes.byref(st), _stream(stream)), "mp_learned_search")
        res = _search_result(out)
        res.update({"n_scored": st.n_scored, "n_exact": st.n_exact, "n_selected": st.n_selected,
                    "certified": int(st.certified), "fallback": bool(st.fallback), "rounds": st.rounds,
                    "margin": st.margin, "max_overestimate": st.max_overestimate, "margin_bound": st.margin_bound,
                    "ms": {"prepare": st.ms_prepare, "model": st.ms_model, "exact": st.ms_exact,
                           "wall": st.ms_wall, "fallback": st.ms_fallback}})
        return res

    def calibrate(self, queries, stream=None):
        """Sets (and returns) the margin rule's overestimation bound from
        queries held out of training (mp_mlp_calibrate)."""
        qs = [_query(q) for q in queries]
        arr = (mp_search_query * len(qs))(*qs)
        bound = ctypes.c_double(0)
        _check(lib().mp_mlp_calibrate(self._h, arr, len(qs), ctypes.byref(bound), _stream(stream)),
               "mp_mlp_calibrate")
        return bound.value

    def set_margin_bound(self, bound):
        _check(lib().mp_mlp_set_margin_bound(self._h, ctypes.c_double(bound)), "mp_mlp_set_margin_bound")

    def save(self, path):
        """Checkpoint: parameters, Adam moments and step (versioned header)."""
        _check(lib().mp_mlp_save(self._h, os.fsencode(path)), "mp_mlp_save")

    def load(self, path):
        _check(lib().mp_mlp_load(self._h, os.fsencode(path)), "mp_mlp_load")

    def scores(self, query, scores, features=None, stream=None):
        q = _query(query)
        n = ctypes.c_int64(0)
        _check(lib().mp_learned_scores(self._h, ctypes.byref(q), _ptr(scores), _ptr(features), ctypes.byref(n),
                                       _stream(stream)), "mp_learned_scores")
        return n.value

    def close(self):
        if self._h:
            lib().mp_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
