"""Tensor-core MLP kernels against the float64 reference (oracle/mlp.py).

The GEMM is checked against a float64 product of the same bfloat16 values
(FP32 accumulation: relative error well below 1e-4).  The forward pass and
the fused scorer are checked element by element: every output y_i against
the float64 forward y64_i, |y_i - y64_i| <= 1e-2 max(|y64_i|, floor), where
the floor is a fixed fraction of the outputs' scale (an output near zero
carries the absolute rounding error of its 256-term sums).  The backward
pass is checked element by element against the float64 gradients with the
engine's BF16 rounding points (the float64 gradients are themselves pinned
to finite differences in tests/test_mlp_oracle.py).
"""
import numpy as np
import pytest

from paper_2507_17087_gb300 import native as N

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N_,K", [(128, 64, 64), (128, 256, 64), (256, 256, 256), (384, 128, 192),
                                    (1024, 256, 4096), (128, 64, 1024),
                                    # K split over CTAs (few output tiles, long K), unevenly for K = 576
                                    (256, 256, 4096), (256, 64, 4096), (128, 128, 576)])
def test_gemm_bf16_against_float64(M, N_, K):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N_ * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N_, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N_), float("nan"), dtype=torch.float32, device="cuda")
    N.gemm_bf16(A, B, C)
    ref = A.double() @ B.double().T
    err = (C.double() - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * scale * max(1.0, K / 256), (err, scale)


import oracle as O  # noqa: E402
from oracle import mlp as R  # noqa: E402
from paper_2507_17087_gb300 import workloads as W  # noqa: E402


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def rounded_params(p):
    q = dict(p)
    for k in ("W1", "W2", "W3"):
        q[k] = bf16_round(p[k])
    return q


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def max_rel(a, ref, floor):
    """max over elements of |a_i - ref_i| / max(|ref_i|, floor)."""
    a, ref = np.asarray(a, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return float((np.abs(a - ref) / np.maximum(np.abs(ref), floor)).max())


def rms(v):
    return float(np.sqrt(np.mean(np.square(v))))


def test_forward_against_float64():
    model = N.MLP(seed=3)
    p = R.init_params(3)
    rng = np.random.default_rng(3)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    p["b4"] = np.array([0.2])
    model.set_params(p)
    X = torch.from_numpy(rng.standard_normal((4096, 64)).astype(np.float32)).to(torch.bfloat16).cuda()
    y = torch.empty(4096, dtype=torch.float32, device="cuda")
    model.forward(X, y)
    y = y.double().cpu().numpy()
    xs = X.double().cpu().numpy()
    # the float64 forward of the same BF16 inputs and weights, element by
    # element (floor: the outputs' root mean square)
    ref, _ = R.forward(rounded_params(p), xs)
    assert max_rel(y, ref, rms(ref)) <= 1e-2
    # with the engine's BF16 rounding points (the stored activations): only
    # the FP32 accumulation order differs
    ref, _ = R.forward(rounded_params(p), xs, rnd=bf16_round)
    assert max_rel(y, ref, 1e-3 * np.abs(ref).max()) <= 1e-2


def test_gradients_against_float64():
    model = N.MLP(seed=4)
    p = R.init_params(4)
    rng = np.random.default_rng(4)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    model.set_params(p)
    B = 256
    X = torch.from_numpy(rng.standard_normal((B, 64)).astype(np.float32)).to(torch.bfloat16).cuda()
    t = torch.from_numpy(rng.standard_normal(B).astype(np.float32)).cuda()
    loss = model.train_step(X, t, lr=0.0)
    g = model.get_params(grads=True)
    pr = rounded_params(p)
    xs, ts = X.double().cpu().numpy(), t.double().cpu().numpy()
    # float64 with the engine's BF16 rounding points: tight
    y, cache = R.forward(pr, xs, rnd=bf16_round)
    ref = R.backward(pr, cache, y, ts, rnd=bf16_round)
    assert abs(loss - R.loss(y, ts)) <= 1e-3 * abs(loss)
    # element by element, floor: the root mean square of each block
    for k in ref:
        assert max_rel(g[k], ref[k], rms(ref[k])) <= 1e-2, k
    # pure float64 (no rounding points): each gradient sums products of five
    # BF16-rounded operands with cancellation, so only its norm is held to
    # the BF16 budget
    y, cache = R.forward(pr, xs)
    ref = R.backward(pr, cache, y, ts)
    for k in ref:
        assert rel(g[k], ref[k]) <= 6e-2, k


def test_adam_step_against_float64():
    model = N.MLP(seed=5)
    p = model.get_params()
    rng = np.random.default_rng(5)
    X = torch.from_numpy(rng.standard_normal((128, 64)).astype(np.float32)).to(torch.bfloat16).cuda()
    t = torch.from_numpy(rng.standard_normal(128).astype(np.float32)).cuda()
    model.train_step(X, t, lr=1e-3)
    g = model.get_params(grads=True)
    after = model.get_params()
    want = R.adam_step({k: v.copy() for k, v in p.items()}, g, {}, lr=1e-3)
    for k in p:
        assert np.allclose(after[k], want[k], rtol=0, atol=2e-6), k


def test_fused_scores_match_unfused_forward_and_float64():
    model = N.MLP(seed=6)
    q = {"MNK": (256, 1024, 256), "machine": (16, 8), "max_depth": 2, "tile_bytes": 512 * 512 * 4}
    nf, nc = N.search_space(128, 8, 2)
    n = nf * nc
    npad = (n + 127) // 128 * 128
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    feats = torch.zeros(npad, 64, dtype=torch.bfloat16, device="cuda")
    assert model.scores(q, scores, feats) == n
    y = torch.empty(npad, dtype=torch.float32, device="cuda")
    model.forward(feats, y)
    sc = scores.double().cpu().numpy()
    unfused = y[:n].double().cpu().numpy()
    assert max_rel(sc, unfused, 1e-3 * np.abs(unfused).max()) <= 1e-3
    ref, _ = R.forward(rounded_params(model.get_params()), feats[:n].double().cpu().numpy())
    assert max_rel(sc, ref, rms(ref)) <= 1e-2


def test_fused_scores_full_run_against_float64():
    # every candidate of a P = 3600 query (3.79 M: seven full runs of 2^19
    # candidates and a ragged last one, each through the feature and layer
    # kernels) scored by a trained model, against the float64 forward of the
    # kernel's own BF16 features, element by element; and the unfused forward
    # of all 3.79 M feature rows (row tiles far beyond 65,535 x 32) against
    # the fused scores
    model = N.MLP(seed=11)
    model.train_search(W.search_training_queries(128), samples_per_query=4096, epochs=4, batch=4096, lr=1e-3,
                       seed=3)
    q = [q for q in W.search_queries(16) if q["machine"][0] * q["machine"][1] == 3600][0]
    n = 3787020
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    feats = torch.zeros((n + 127) // 128 * 128, 64, dtype=torch.bfloat16, device="cuda")
    assert model.scores(q, scores, feats) == n
    sc = scores.double().cpu().numpy()
    F = feats[:n].double().cpu().numpy()
    pr = rounded_params(model.get_params())
    ref = np.empty(n)
    for lo in range(0, n, 1 << 18):
        ref[lo:lo + (1 << 18)], _ = R.forward(pr, F[lo:lo + (1 << 18)])
    assert max_rel(sc, ref, 1.0) <= 1e-2
    y = torch.empty(feats.shape[0], dtype=torch.float32, device="cuda")
    model.forward(feats, y)
    assert max_rel(y[:n].double().cpu().numpy(), sc, 1.0) <= 1e-4
    model.close()


def test_learned_search_gains_over_the_search_without_it():
    # on 100 held-out queries: the trained, calibrated network against the
    # same network untrained and against the exact search without a network
    # (the primary-bound search).  Every returned cost is the exact cost of
    # the returned candidate; results certified (every threat evaluated, or
    # the secondary lower bound reached) or from the fallback are optimal;
    # with the calibrated margin rule at least 99 % are; the trained model's
    # top K alone hold the optimum far more often than the untrained one's
    # (at least 90 % of the time), and it falls back to the exhaustive search
    # less often.
    # the benchmark's recipe: two training runs, the one with the smaller
    # calibration bound on the held-out calibration queries kept
    calq = W.search_training_queries(64, first_index=40000)
    model, bound = None, None
    for seed in (2, 3):
        m = N.MLP(seed=7 + seed)
        loss0 = m.train_search(W.search_training_queries(4), samples_per_query=512, epochs=1, batch=512, lr=1e-3,
                               seed=1)
        loss = m.train_search(W.search_training_queries(512), samples_per_query=4096, epochs=8, batch=4096,
                              lr=1e-3, seed=seed)
        assert np.isfinite(loss) and loss < loss0
        b = m.calibrate(calq)
        assert np.isfinite(b)
        if model is None or b < bound:
            if model is not None:
                model.close()
            model, bound = m, b
        else:
            m.close()
    untrained = N.MLP(seed=99)
    assert untrained.learned_search(W.search_queries(1, first_index=9000)[0], K=1024)["margin_bound"] == np.inf
    stats = {"trained": [0, 0, 0], "untrained": [0, 0, 0]}   # zero regret, top-K zero regret, fallbacks
    evalq = W.search_queries(100, first_index=9000)
    for q in evalq:
        exact = N.decompose_search([q])[0]
        want = (exact["primary_bytes"], exact["secondary_bytes"])
        for name, m in (("trained", model), ("untrained", untrained)):
            got = m.learned_search(q, K=1024, fallback=True)
            cost = (got["primary_bytes"], got["secondary_bytes"])
            p = np.zeros(1, dtype=np.uint64)
            s = np.zeros(1, dtype=np.uint64)
            N.candidate_costs(q, np.array([got["index"]], dtype=np.int64), p, s)
            assert (int(p[0]), int(s[0])) == cost   # the returned costs are exact
            if got["fallback"]:
                assert got["index"] == exact["index"]
            if got["fallback"] or got["certified"] in (1, 2):
                assert cost == want, (name, q, got["certified"])
            raw = m.learned_search(q, K=1024, fallback=False)
            st = stats[name]
            st[0] += cost == want
            st[1] += (raw["primary_bytes"], raw["secondary_bytes"]) == want
            st[2] += got["fallback"]
    print("trained / untrained (zero regret, top-K zero regret, fallbacks):", stats, "bound", bound)
    assert stats["trained"][0] >= 99   # the search as deployed (certificates, margin rule, fallback)
    assert stats["trained"][1] >= 90 and stats["untrained"][1] <= stats["trained"][1] - 10
    assert stats["trained"][2] < stats["untrained"][2]
    # scoring every candidate instead
    q = evalq[0]
    exact = N.decompose_search([q])[0]
    got = model.learned_search(q, K=1024, fallback=True, score_all=True)
    assert got["n_scored"] == exact["n_candidates"]
    assert (got["primary_bytes"], got["secondary_bytes"]) == (exact["primary_bytes"], exact["secondary_bytes"])
    model.close()
    untrained.close()


def test_learned_search_edge_cases():
    # pools smaller than K (every candidate of least primary evaluated: the
    # first certificate), K = 1, one node, one processor per node; every
    # result's cost tuple equals the exact search's, and the exhaustive
    # oracle's on the small machines
    model = N.MLP(seed=12)
    model.train_search(W.search_training_queries(8), samples_per_query=1024, epochs=2, batch=1024, lr=1e-3, seed=4)
    cases = [{"MNK": (16, 8, 64), "machine": (2, 4), "max_depth": 2},
             {"MNK": (64, 64, 1), "machine": (1, 8), "max_depth": 1},
             {"MNK": (5, 7, 3), "machine": (6, 1), "max_depth": 2},
             {"MNK": (256, 1024, 256), "machine": (16, 8), "max_depth": 2}]
    for q in cases:
        q = dict(q, tile_bytes=512 * 512 * 4)
        exact = N.decompose_search([q])[0]
        want = (exact["primary_bytes"], exact["secondary_bytes"])
        for K in (1, 64, 65536):
            got = model.learned_search(q, K=K, fallback=True)
            assert (got["primary_bytes"], got["secondary_bytes"]) == want, (q, K)
            if K >= got["n_scored"]:
                assert got["certified"] == 1 and not got["fallback"]
        if q["machine"][0] * q["machine"][1] <= 16:
            ref = O.search(*q["MNK"], q["machine"], q["max_depth"], threads=8)
            assert want == (ref["primary"] * q["tile_bytes"], ref["secondary"] * q["tile_bytes"])
    with pytest.raises(N.MapleError):
        model.learned_search(cases[0] | {"tile_bytes": 512 * 512 * 4}, K=0)
    model.close()


def test_fibre_features_against_oracle_nodes():
    # features 53..58 of a candidate (factorisation f, chain c): whether the
    # node changes one step along each fibre, and how many distinct nodes its
    # first four points reach; recomputed from the oracle's owner of each flat
    # index of the chain space (values 0, 1/4 .. 1 are exact in BF16)
    model = N.MLP(seed=8)
    n, g = 30, 8
    P = n * g
    q = {"MNK": (256, 1024, 256), "machine": (n, g), "max_depth": 2, "tile_bytes": 512 * 512 * 4}
    nf, nc = N.search_space(P, g, 2)
    facts = O.factorisations(P, 3)
    chains = O.chains(n, g, 2)
    assert (len(facts), len(chains)) == (nf, nc)
    npad = (nf * nc + 127) // 128 * 128
    scores = torch.empty(nf * nc, dtype=torch.float32, device="cuda")
    feats = torch.zeros(npad, 64, dtype=torch.bfloat16, device="cuda")
    assert model.scores(q, scores, feats) == nf * nc
    got = feats[:, 53:59].float().cpu().numpy()
    rng = np.random.default_rng(8)
    node_cache = {}
    for c in rng.choice(nc, 40, replace=False):
        if c not in node_cache:
            own = O.Launch((P,), (n, g), list(chains[c]), ("block",)).owner_of(np.arange(P, dtype=np.int64))
            node_cache[c] = own // g
        node = node_cache[c]
        for fr in rng.choice(nf, 25, replace=False):
            f = facts[fr]
            want = []
            stride = (1, f[0], f[0] * f[1])
            ch, dist = [0.0] * 3, [0.25] * 3
            for v in range(3):
                if f[v] > 1 and stride[v] < P:
                    seen = [node[0]]
                    j = 1
                    while j < 4 and j < f[v] and j * stride[v] < P:
                        nd = node[j * stride[v]]
                        if j == 1:
                            ch[v] = float(nd != node[0])
                        if nd not in seen:
                            seen.append(nd)
                        j += 1
                    dist[v] = len(seen) / 4.0
            want = ch + dist
            assert np.array_equal(got[fr * nc + c], np.array(want, dtype=np.float32)), (fr, c, f, chains[c])
