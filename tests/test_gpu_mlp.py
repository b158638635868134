"""Tensor-core MLP kernels against the float64 reference (oracle/mlp.py).

The GEMM is checked against a float64 product of the same bfloat16 values
(FP32 accumulation: relative error well below 1e-4); the forward pass of the
model against the float64 forward to 1e-2 relative (BF16 operands); the
backward pass against the float64 gradients, which are themselves pinned to
finite differences in tests/test_mlp_oracle.py.
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


def test_forward_against_float64():
    model = N.MLP(seed=3)
    p = R.init_params(3)
    rng = np.random.default_rng(3)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    p["b4"] = np.array([0.2])
    model.set_params(p)
    X = torch.from_numpy(rng.standard_normal((512, 64)).astype(np.float32)).to(torch.bfloat16).cuda()
    y = torch.empty(512, dtype=torch.float32, device="cuda")
    model.forward(X, y)
    ref, _ = R.forward(rounded_params(p), X.double().cpu().numpy())
    assert rel(y.double().cpu().numpy(), ref) <= 1e-2


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
    for k in ref:
        assert rel(g[k], ref[k]) <= 1e-2, k
    # pure float64: within the BF16 rounding of five stored operands
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
    assert rel(scores.double().cpu().numpy(), y[:n].double().cpu().numpy()) <= 1e-3
    ref, _ = R.forward(rounded_params(model.get_params()), feats[:n].double().cpu().numpy())
    assert rel(scores.double().cpu().numpy(), ref) <= 1e-2


def test_learned_search_trains_and_finds_the_optimum():
    model = N.MLP(seed=7)
    train = W.search_training_queries(48)
    loss0 = model.train_search(train[:4], samples_per_query=512, epochs=1, batch=512, lr=1e-3, seed=1)
    loss = model.train_search(train, samples_per_query=4096, epochs=6, batch=4096, lr=1e-3, seed=2)
    print(f"training loss {loss0:.4f} -> {loss:.4f}")
    assert np.isfinite(loss) and loss < loss0
    evalq = W.search_queries(12, first_index=9000)
    zero_regret = 0
    for q in evalq:
        exact = N.decompose_search([q])[0]
        got = model.learned_search(q, K=1024, fallback=True)
        # exact with the fallback: the optimal cost tuple (among
        # exact ties the index may differ unless the exhaustive search ran)
        assert (got["primary_bytes"], got["secondary_bytes"]) == \
            (exact["primary_bytes"], exact["secondary_bytes"])
        if got["fallback"]:
            assert got["index"] == exact["index"]
        raw = model.learned_search(q, K=1024, fallback=False)
        zero_regret += (raw["primary_bytes"], raw["secondary_bytes"]) == \
            (exact["primary_bytes"], exact["secondary_bytes"])
        # the model ranks the candidates of least primary cost, at most all
        assert raw["n_exact"] <= 1024 and raw["n_scored"] <= exact["n_candidates"]
    print(f"zero-regret without fallback: {zero_regret}/{len(evalq)}")
    assert zero_regret >= len(evalq) // 2
    # scoring every candidate instead
    q = evalq[0]
    exact = N.decompose_search([q])[0]
    got = model.learned_search(q, K=1024, fallback=True, score_all=True)
    assert got["n_scored"] == exact["n_candidates"]
    assert (got["primary_bytes"], got["secondary_bytes"]) == (exact["primary_bytes"], exact["secondary_bytes"])


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
