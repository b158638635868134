"""The allocation-free map_points entry point, against the regular one.

mp_map_points_noalloc serves callers that cannot allocate device memory (a
framework whose allocator owns the whole device budget, or a latency-critical
loop that cannot absorb cudaMalloc's device-wide synchronisation).  Its
results must equal mp_map_points' exactly (ids and histograms are integers),
on two calls in a row -- the second call finds the first call's contents in
the shared scratch array.  This file is collected last on purpose.
"""
import ctypes
import math

import pytest

from paper_2507_17087_gb300 import native as N

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ((1024, 96, 130), (64, 8), [("split", 1, 4), ("swap", 0, 2)], ("block",)),
    ((37, 41, 29), (6, 4), [("merge", 0, 1)], ("block_cyclic", 3)),
    ((300, 7), (5, 3), [], ("hier",)),
    ((9, 9, 9), (6, 6), [("split", 0, 3)], ("linear_cyclic",)),
]


def call_noalloc(L, machine, chain, dist, ids, hist):
    """Straight through the C ABI."""
    sp, mc, ds = N.make_space(L), N.make_machine(machine), N.make_dist(dist)
    ch, n = N.make_chain(chain)
    return N.lib().mp_map_points_noalloc(ctypes.byref(sp), ctypes.byref(mc), ch, n, ctypes.byref(ds),
                                         ids.data_ptr() if ids is not None else None,
                                         hist.data_ptr() if hist is not None else None,
                                         torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_map_points_on_consecutive_calls():
    for L, machine, chain, dist in CASES:
        P = machine[0] * machine[1]
        npts = math.prod(L)
        ref_ids = torch.empty(npts, dtype=torch.int32, device="cuda")
        ref_hist = torch.empty(P, dtype=torch.int64, device="cuda")
        N.map_points(L, machine, chain, dist, ids=ref_ids, hist=ref_hist)
        outs = [(torch.full((npts,), -1, dtype=torch.int32, device="cuda"),
                 torch.full((P,), -1, dtype=torch.int64, device="cuda")) for _ in range(2)]
        torch.cuda.synchronize()
        # nothing is allocated by the calls: neither the device's free memory
        # nor the library's workspace changes around them
        free0, ws0 = torch.cuda.mem_get_info()[0], N.workspace_bytes()
        for ids, hist in outs:
            assert call_noalloc(L, machine, chain, dist, ids, hist) == 0
            torch.cuda.synchronize()
            assert torch.equal(ids, ref_ids)
            assert torch.equal(hist, ref_hist)
        assert (torch.cuda.mem_get_info()[0], N.workspace_bytes()) == (free0, ws0)


def test_noalloc_rejects_host_buffers_and_oversized_scratch():
    L, machine, chain, dist = (16, 16), (2, 4), [], ("block",)
    host = torch.zeros(256, dtype=torch.int32)
    assert call_noalloc(L, machine, chain, dist, host, None) == 1            # MP_EINVAL
    # P = 2^22 processors: the chain table alone (4 P bytes = 16 MiB) exceeds 8 MiB
    assert call_noalloc((8, 8), (1 << 19, 8), [], ("cyclic",), None,
                        torch.empty(1 << 22, dtype=torch.int64, device="cuda")) == 6   # MP_ENOTSUP
