"""Failure reporting, fault injection and checkpoints, on the GPU without a
fault: a bounded device-side wait that runs out, injected allocation
failures, the model checkpoint (resume) and the persisted autotune choice."""
import math
import os

import numpy as np
import pytest

from paper_2507_17087_gb300 import native as N
from paper_2507_17087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"
MP_ENOMEM, MP_ETIMEOUT = 3, 5


def _small_map():
    cfg = W.plain_config()
    ids = torch.full((math.prod(cfg["L"]),), -5, dtype=torch.int32, device=DEV)
    hist = torch.full((8,), -5, dtype=torch.int64, device=DEV)
    return cfg, ids, hist


def test_bounded_wait_reports_timeout_and_context_survives():
    assert N.selftest_wait_timeout(2000) == MP_ETIMEOUT
    cfg, ids, hist = _small_map()
    N.map_points(cfg["L"], cfg["machine"], cfg["chain"], cfg["dist"], ids=ids, hist=hist)
    torch.cuda.synchronize()
    assert int(hist.sum().item()) == math.prod(cfg["L"])


def test_injected_allocation_failure_writes_nothing():
    cfg, ids, hist = _small_map()
    N.debug_fail_allocations(1)
    with pytest.raises(N.MapleError) as err:
        N.map_points(cfg["L"], cfg["machine"], cfg["chain"], cfg["dist"], ids=ids, hist=hist)
    assert err.value.status == MP_ENOMEM
    torch.cuda.synchronize()
    assert (ids == -5).all() and (hist == -5).all()
    N.map_points(cfg["L"], cfg["machine"], cfg["chain"], cfg["dist"], ids=ids, hist=hist)
    torch.cuda.synchronize()
    assert int(hist.sum().item()) == math.prod(cfg["L"])
    N.debug_fail_allocations(0)


def _batch(seed, B=256):
    rng = np.random.default_rng(seed)
    X = torch.from_numpy(rng.standard_normal((B, 64)).astype(np.float32)).to(torch.bfloat16).to(DEV)
    t = torch.from_numpy(rng.standard_normal(B).astype(np.float32)).to(DEV)
    return X, t


def test_model_checkpoint_resumes_training(tmp_path):
    a = N.MLP(seed=21)
    for s in range(3):
        a.train_step(*_batch(s), lr=1e-3)
    path = os.fspath(tmp_path / "model.ckpt")
    a.save(path)
    b = N.MLP(seed=99)
    b.load(path)
    pa, pb = a.get_params(), b.get_params()
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    # the Adam state came along: one more identical step keeps them together
    la = a.train_step(*_batch(7), lr=1e-3)
    lb = b.train_step(*_batch(7), lr=1e-3)
    assert abs(la - lb) <= 1e-6 * max(1.0, abs(la))
    pa, pb = a.get_params(), b.get_params()
    for k in pa:
        assert np.allclose(pa[k], pb[k], rtol=1e-5, atol=1e-7), k
    a.close()
    b.close()


def test_checkpoint_carries_the_margin_bound(tmp_path):
    # format 2 stores the calibrated margin bound after the header; a
    # format-1 file (no bound) loads as an uncalibrated model
    q = {"MNK": (64, 256, 16), "machine": (4, 8), "max_depth": 2, "tile_bytes": 512 * 512 * 4}
    a = N.MLP(seed=23)
    a.set_margin_bound(0.5)
    path = tmp_path / "model.ckpt"
    a.save(os.fspath(path))
    b = N.MLP(seed=24)
    b.load(os.fspath(path))
    assert b.learned_search(q, K=64)["margin_bound"] == pytest.approx(1.25 * 0.5 + 0.01)
    raw = bytearray(path.read_bytes())
    v1 = raw[:8] + (1).to_bytes(4, "little") + raw[12:24] + raw[32:]   # version 1, bound dropped
    p1 = tmp_path / "v1.ckpt"
    p1.write_bytes(bytes(v1))
    b.load(os.fspath(p1))
    assert b.learned_search(q, K=64)["margin_bound"] == np.inf
    pa, pb = a.get_params(), b.get_params()
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    a.close()
    b.close()


def test_corrupt_checkpoints_rejected(tmp_path):
    a = N.MLP(seed=22)
    path = tmp_path / "model.ckpt"
    a.save(os.fspath(path))
    raw = bytearray(path.read_bytes())
    for mutate in (lambda r: r.__setitem__(0, ord("X")),            # magic
                   lambda r: r.__setitem__(8, 7),                   # format version
                   lambda r: r.__setitem__(12, r[12] ^ 1)):         # parameter count
        bad = bytearray(raw)
        mutate(bad)
        p = tmp_path / "bad.ckpt"
        p.write_bytes(bytes(bad))
        with pytest.raises(N.MapleError):
            a.load(os.fspath(p))
    p = tmp_path / "short.ckpt"
    p.write_bytes(bytes(raw[: len(raw) // 2]))
    with pytest.raises(N.MapleError):
        a.load(os.fspath(p))
    a.close()


def test_persisted_autotune_choice(tmp_path):
    qs = W.batched_queries(120, max_points=1 << 20)
    launches = [(q["L"], q["machine"], N.chain_from_draws(*q["machine"], q["draws"]), q["dist"], q["face"])
                for q in qs]
    cache = os.fspath(tmp_path / "tiles.json")
    b1 = N.Batch(launches)
    # (ids between queries pad each query to 4 points and are not written)
    ids1 = torch.full((int(b1.info()["total_ids"]),), -1, dtype=torch.int32, device=DEV)
    t1 = b1.autotune_cached(cache, ids1)
    b1.run(ids=ids1)
    b2 = N.Batch(launches)
    ids2 = torch.full_like(ids1, -1)
    assert b2.autotune_cached(cache, ids2) == t1
    assert b2.info()["tile_groups"] == t1
    b2.run(ids=ids2)
    torch.cuda.synchronize()
    assert torch.equal(ids1, ids2)
    b1.close()
    b2.close()


def test_kernel_timers_are_one_shot_and_record_on_the_call_stream():
    # the id writer's and the layer kernel's measurement hooks: armed, the
    # next launch records both events (a positive elapsed time); then they
    # disarm themselves, so a second call does not record them again
    def events():
        # recorded once here, so that torch will read them after the library
        # records them again
        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        for x in e:
            x.record()
        torch.cuda.synchronize()
        return e

    a, b = events()
    ids = torch.empty(64 * 64, dtype=torch.int32, device="cuda")
    N.set_kernel_timer(a, b)
    N.map_points((64, 64), (2, 4), [("merge", 0, 1)], ("block",), ids=ids)
    torch.cuda.synchronize()
    assert a.elapsed_time(b) > 0
    model = N.MLP(seed=2)
    q = {"MNK": (64, 64, 64), "machine": (4, 4), "max_depth": 2, "tile_bytes": 512 * 512 * 4}
    nf, nc = N.search_space(16, 4, 2)
    scores = torch.empty(nf * nc, dtype=torch.float32, device="cuda")
    c, d = events()
    N.set_layer_timer(c, d)
    assert model.scores(q, scores) == nf * nc
    torch.cuda.synchronize()
    t1 = c.elapsed_time(d)
    assert t1 > 0
    model.scores(q, scores)
    N.map_points((64, 64), (2, 4), [("merge", 0, 1)], ("block",), ids=ids)
    torch.cuda.synchronize()
    assert c.elapsed_time(d) == t1
    model.close()
