"""GPU parity of the learned-proposal kernels.

Truth vectors against the oracle's evaluation of every pointed model; the
Hamming k-NN against numpy brute force; the MLP's FP32 forward pass and
gradient against the float64 reference (oracle/mlp.py); the BF16 scoring
kernel against the reference with W1 rounded to BF16; and Adam training on a
learnable labelling.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as ref
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk
from paper_2606_15437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()
    assert torch.cuda.is_available()


def E():
    from paper_2606_15437_gb300 import engine
    return engine


def test_truth_vectors_match_oracle():
    texts = W.proposal_formulas(5, count=2100, bases=2000)[::50] + [W.alpha(2), "p -> []<>p", W.K_AXIOM]
    models, groups = W.pointed_models(5)
    bits = E().truth_vectors(texts, models=models, groups=groups).cpu().numpy().view(np.uint32)
    for i, t in enumerate(texts):
        for j in range(0, len(models), 7):
            m = models[j]
            n = int(m["n"])
            R = oracle.frame_matrix(int(m["frame"]), n)
            V = np.array([[(int(m["val"]) >> (v * n + w)) & 1 for w in range(n)] for v in range(4)], np.uint8)
            want = oracle.eval_model(t, R, V)[int(m["world"])]
            got = (int(bits[i, j // 32]) >> (j % 32)) & 1
            assert got == want, (t, j)


def test_hamming_knn_matches_brute_force():
    rng = np.random.default_rng(2)
    n, words, k = 700, 8, 12
    v = rng.integers(0, 2 ** 32, size=(n, words), dtype=np.uint64).astype(np.uint32)
    v[100:120] = v[100]              # ties and zero distances
    v[300:310, 0] = 0
    bits = torch.from_numpy(v.view(np.int32).copy()).cuda()
    nbr, dist = E().hamming_knn(bits, k)
    pop = np.unpackbits(v.view(np.uint8), axis=1)
    for q in range(0, n, 3):
        d = (pop ^ pop[q]).sum(1)
        order = sorted((int(d[j]), j) for j in range(n) if j != q)
        t = order[k - 1][0]
        want = [j for dd, j in order if dd < t] + [j for dd, j in order if dd == t][:k - sum(1 for dd, _ in order if dd < t)]
        assert sorted(nbr[q].tolist()) == sorted(want), q
        assert all(int(dist[q, i]) == int(d[nbr[q, i]]) for i in range(k))


def _small_problem(F=256, H=256, B=96, seed=3):
    rng = np.random.default_rng(seed)
    words = F // 64
    vec = rng.integers(0, 2 ** 32, size=(40, words), dtype=np.uint64).astype(np.uint32)
    pa = rng.integers(0, 40, size=B).astype(np.int32)
    pb = rng.integers(0, 40, size=B).astype(np.int32)
    y = (rng.random(B) < 0.3).astype(np.float32)
    w = (0.5 + rng.random(B)).astype(np.float32)
    return vec, pa, pb, y, w


@pytest.mark.parametrize("F,B", [(256, 96), (8192, 64)])
def test_mlp_forward_and_gradient_match_float64(F, B):
    """The FP32 forward pass and gradient against float64, at a small feature
    dimension and at the production one (8,192 features: 128 words per pair
    operand, the K of the FP32 training GEMMs).  FP32 sums of K products
    err by about sqrt(K) ulps, so the tolerance grows with sqrt(F / 256)."""
    H = 256
    vec, pa, pb, y, w = _small_problem(F, H, B=B)
    net = E().MLP(F, H, seed=4)
    widen = np.sqrt(F / 256)
    dv = torch.from_numpy(vec.view(np.int32).copy()).cuda()
    tpa, tpb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
    z = net.forward(dv, tpa, tpb).cpu().numpy()
    params = net.params.cpu().numpy().astype(np.float64)
    zr = ref.forward(params, F, H, vec, pa, pb)
    assert np.allclose(z, zr, rtol=1e-4 * widen, atol=1e-4 * widen)
    loss = net.gradient(dv, tpa, tpb, torch.from_numpy(y).cuda(), torch.from_numpy(w).cuda())
    g = net.grad.cpu().numpy().astype(np.float64)
    lr, gr = ref.loss_and_grad(params, F, H, vec, pa, pb, y, w)
    assert abs(float(loss.item()) - lr) <= 1e-4 * widen * max(1.0, abs(lr))
    # FP32 sums of up to B*F products: compare relative to the gradient's scale
    scale = np.abs(gr).max()
    assert np.abs(g - gr).max() <= 2e-4 * widen * scale
    # the W1 block (the tiled GEMM with features generated in its loader) on its own scale
    g1, r1 = g[:F * H], gr[:F * H]
    assert np.abs(g1 - r1).max() <= 2e-4 * widen * max(np.abs(r1).max(), 1e-30)


def test_bf16_scoring_matches_rounded_reference():
    F, H = 256, 256
    vec, pa, pb, _, _ = _small_problem(F, H, B=200, seed=5)
    net = E().MLP(F, H, seed=6)
    dv = torch.from_numpy(vec.view(np.int32).copy()).cuda()
    tpa, tpb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
    s = net.score(dv, tpa, tpb, batch=64).cpu().numpy()
    params = net.params.cpu().numpy().astype(np.float64)
    w1 = torch.from_numpy(params[:F * H].astype(np.float32)).to(torch.bfloat16).float().numpy()
    p2 = params.copy()
    p2[:F * H] = w1
    zr = ref.forward(p2, F, H, vec, pa, pb)
    assert np.allclose(s, zr, rtol=1e-3, atol=1e-3)


def test_training_learns_a_labelling():
    # label = whether the pair's vectors share bit 7 (a and b), learnable from x
    F, H = 256, 256
    rng = np.random.default_rng(7)
    vec = rng.integers(0, 2 ** 32, size=(300, F // 64), dtype=np.uint64).astype(np.uint32)
    pa = rng.integers(0, 300, size=8192).astype(np.int32)
    pb = rng.integers(0, 300, size=8192).astype(np.int32)
    y = (((vec[pa, 0] & vec[pb, 0]) >> 7) & 1).astype(np.float32)
    net = E().MLP(F, H, seed=8)
    dv = torch.from_numpy(vec.view(np.int32).copy()).cuda()
    tpa, tpb, ty = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda(), torch.from_numpy(y).cuda()
    hist = net.train(dv, tpa, tpb, ty, epochs=6, batch=1024, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    acc = ((net.forward(dv, tpa, tpb).cpu().numpy() > 0) == (y > 0.5)).mean()
    assert acc > 0.95


def test_learned_proposal_gain():
    """What the trained network gains over the method without it: at an
    equal exact-evaluation budget, the MLP's ranking of the candidate
    universe yields more certified late splits per 1e12 evaluations than a
    random ranking of the same universe.  Every late split reported by the
    exact search is accepted by mk_certify."""
    r = E().proposal_experiment(n_formulas=4000, universe=500_000, k=256, train_identical=40_000,
                                train_other=40_000, budget=4e12, frames_per_n=1 << 18, epochs=6,
                                methods=("mlp", "random", "random_identical"))
    for m in ("mlp", "random", "random_identical"):
        assert r[m]["certified"] == r[m]["late_splits"], m
    assert r["train_late"] > 0
    assert r["mlp"]["certified_per_1e12_evals"] > r["random"]["certified_per_1e12_evals"]
    assert r["mlp"]["certified"] > 0
    # the trivial filter (identical truth vectors first) is not what the network learns
    assert r["mlp"]["certified_per_1e12_evals"] > r["random_identical"]["certified_per_1e12_evals"]
    print("certified per 1e12 evals: mlp %.3f, random among identical-vector pairs %.3f, random %.3f" % (
        r["mlp"]["certified_per_1e12_evals"], r["random_identical"]["certified_per_1e12_evals"],
        r["random"]["certified_per_1e12_evals"]))


def test_learned_workload_full_size_sampled_outputs():
    """The learned-proposal workload at its full size (10,000 formulas,
    4,096 pointed models, 1,024-NN universe of 5,467,766 pairs), checked on
    sampled outputs the references can compute one by one: truth-vector bits
    against the oracle's evaluation of the model, neighbour lists against
    brute-force Hamming distances over all 10,000 vectors, and BF16 scores of
    universe pairs against float64 with the same BF16-rounded weights."""
    E_ = E()
    texts = W.proposal_formulas(5, 10000)
    models, groups = W.pointed_models(5)
    bits = E_.truth_vectors(texts, models=models, groups=groups)
    bits_np = bits.cpu().numpy().view(np.uint32)
    assert bits_np.shape == (10000, len(models) // 32) and len(models) == 4096
    rng = np.random.default_rng(17)
    for i, j in zip(rng.integers(0, 10000, 300), rng.integers(0, 4096, 300)):
        m = models[j]
        n = int(m["n"])
        R = oracle.frame_matrix(int(m["frame"]), n)
        V = np.array([[(int(m["val"]) >> (v * n + w)) & 1 for w in range(n)] for v in range(4)], np.uint8)
        assert ((int(bits_np[i, j // 32]) >> (j % 32)) & 1) == oracle.eval_model(texts[i], R, V)[int(m["world"])]
    k = 1024
    nbr, dist = E_.hamming_knn(bits, k)
    pop = np.unpackbits(bits_np.view(np.uint8), axis=1)
    for q in rng.integers(0, 10000, 4):
        d = (pop ^ pop[q]).sum(1)
        d[q] = 1 << 30
        kth = np.sort(d)[k - 1]
        got = nbr[q]
        assert np.array_equal(np.sort(d[got]), np.sort(d)[:k])           # the k least distances
        assert (d[got] <= kth).all() and len(set(got.tolist())) == k and q not in got
        assert np.array_equal(dist[q].astype(np.int64), d[got])
    pa, pb = E_.knn_universe(nbr, 5_467_766, 5)
    assert len(pa) == 5_467_766
    F, H = bits_np.shape[1] * 64, 256
    net = E_.MLP(F, H, seed=6)
    pick = rng.integers(0, len(pa), 512)
    tpa = torch.from_numpy(pa[pick]).cuda()
    tpb = torch.from_numpy(pb[pick]).cuda()
    s = net.score(bits, tpa, tpb).cpu().numpy()
    params = net.params.cpu().numpy().astype(np.float64)
    w1 = torch.from_numpy(params[:F * H].astype(np.float32)).to(torch.bfloat16).float().numpy()
    p2 = params.copy()
    p2[:F * H] = w1
    zr = ref.forward(p2, F, H, bits_np, pa[pick], pb[pick])
    # FP32 sums over 8,192 features: the F = 256 tolerance widened by sqrt(8192 / 256)
    assert np.abs(s - zr).max() <= 1e-3 * np.sqrt(F / 256) * max(1.0, float(np.abs(zr).max()))
