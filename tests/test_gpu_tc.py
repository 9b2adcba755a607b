"""GPU parity of the tcgen05 first MLP layer (tensor memory accumulator)
against a float64 reference of the same BF16-rounded weights, against the
legacy mma.sync layer, and end to end through mk_mlp_infer_tc; sizes span
one and several CTAs, ragged batches, the shortest and the full feature
dimension."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 256


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()
    assert torch.cuda.is_available()


def E():
    from paper_2606_15437_gb300 import engine
    return engine


def _problem(F, B, seed):
    rng = np.random.default_rng(seed)
    words = F // 64
    vec = rng.integers(0, 2 ** 32, size=(50, words), dtype=np.uint64).astype(np.uint32)
    pa = rng.integers(0, 50, size=B).astype(np.int32)
    pb = rng.integers(0, 50, size=B).astype(np.int32)
    return vec, pa, pb


def _features(vec, pa, pb):
    words = vec.shape[1]
    a, b = vec[pa], vec[pb]
    x = np.concatenate([a ^ b, a & b], axis=1)                    # [B, words] words
    bits = (x[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1  # bit i of word j = feature 32j + i
    return bits.reshape(len(pa), 64 * words).astype(np.float64)


def _layer1(F, B, seed, impl):
    vec, pa, pb = _problem(F, B, seed)
    net = E().MLP(F, H, seed=seed + 1)
    dv = torch.from_numpy(vec.view(np.int32).copy()).cuda()
    tpa, tpb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
    w1t = torch.empty((H, F), dtype=torch.bfloat16, device="cuda")
    mk.mlp_w1t_bf16_raw(net.params.data_ptr(), F, H, w1t.data_ptr(), 0)
    b1 = net.params[F * H:F * H + H]
    h1 = torch.full((B, H), -7.0, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    if impl == "tc":
        mk.mlp_layer1_tc_raw(dv.data_ptr(), F, tpa.data_ptr(), tpb.data_ptr(), B, w1t.data_ptr(), b1.data_ptr(),
                             h1.data_ptr(), st.data_ptr(), 0)
    elif impl == "ws":
        tiles = torch.empty(mk.mlp_w1_tiles_bytes(F), dtype=torch.uint8, device="cuda")
        mk.mlp_w1_tiles_raw(net.params.data_ptr(), F, H, tiles.data_ptr(), 0)
        mk.mlp_layer1_tc_ws_raw(dv.data_ptr(), F, tpa.data_ptr(), tpb.data_ptr(), B, tiles.data_ptr(), b1.data_ptr(),
                                h1.data_ptr(), st.data_ptr(), 0)
    else:
        mk.mlp_layer1_mma_raw(dv.data_ptr(), F, tpa.data_ptr(), tpb.data_ptr(), B, w1t.data_ptr(), b1.data_ptr(),
                              h1.data_ptr(), 0)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    X = _features(vec, pa, pb)
    W1 = w1t.float().cpu().numpy().astype(np.float64).T            # [F, H], BF16 values
    want = np.maximum(X @ W1 + b1.cpu().numpy().astype(np.float64), 0.0)
    return h1.cpu().numpy(), want


@pytest.mark.parametrize("impl", ["tc", "ws"])
@pytest.mark.parametrize("F,B", [(128, 128), (256, 1), (256, 300), (1024, 129), (8192, 700)])
def test_layer1_tc_matches_float64(F, B, impl):
    got, want = _layer1(F, B, F + B, impl)
    scale = max(1.0, float(np.abs(want).max()))
    assert np.abs(got - want).max() <= 2e-5 * scale * np.sqrt(F / 128)


def test_layer1_tc_agrees_with_mma_sync():
    a, want = _layer1(8192, 512, 11, "tc")
    b, _ = _layer1(8192, 512, 11, "mma")
    c, _ = _layer1(8192, 512, 11, "ws")
    scale = float(np.abs(want).max())
    assert np.abs(a - b).max() <= 1e-4 * scale
    assert np.abs(c - b).max() <= 1e-4 * scale


def test_w1_tiles_layout():
    F = 256
    net = E().MLP(F, H, seed=2)
    tiles = torch.empty(mk.mlp_w1_tiles_bytes(F), dtype=torch.uint8, device="cuda")
    mk.mlp_w1_tiles_raw(net.params.data_ptr(), F, H, tiles.data_ptr(), 0)
    got = tiles.cpu().numpy().view(np.uint16).reshape(F // 64, H, 64)
    w1 = torch.from_numpy(net.params.cpu().numpy()[:F * H].reshape(F, H)).to(torch.bfloat16).view(torch.int16)
    w1 = w1.numpy().view(np.uint16)
    for kb in range(F // 64):
        for n in (0, 1, 7, 8, 100, 255):
            for c in range(8):
                chunk = got[kb, n, 8 * (c ^ (n & 7)):8 * (c ^ (n & 7)) + 8]
                assert np.array_equal(chunk, w1[kb * 64 + 8 * c:kb * 64 + 8 * c + 8, n])


def test_infer_tc_matches_rounded_reference():
    F = 256
    rng = np.random.default_rng(5)
    vec = rng.integers(0, 2 ** 32, size=(40, F // 64), dtype=np.uint64).astype(np.uint32)
    pa = rng.integers(0, 40, size=333).astype(np.int32)
    pb = rng.integers(0, 40, size=333).astype(np.int32)
    net = E().MLP(F, H, seed=6)
    dv = torch.from_numpy(vec.view(np.int32).copy()).cuda()
    tpa, tpb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
    s_tc = net.score(dv, tpa, tpb, batch=200, impl="tc").cpu().numpy()
    s_mma = net.score(dv, tpa, tpb, batch=200, impl="mma").cpu().numpy()
    params = net.params.cpu().numpy().astype(np.float64)
    w1 = torch.from_numpy(params[:F * H].astype(np.float32)).to(torch.bfloat16).float().numpy()
    p2 = params.copy()
    p2[:F * H] = w1
    zr = ref.forward(p2, F, H, vec, pa, pb)
    assert np.allclose(s_tc, zr, rtol=1e-3, atol=1e-3)
    assert np.allclose(s_tc, s_mma, rtol=1e-4, atol=1e-4)


def test_layer1_tc_rejects_bad_shapes():
    with pytest.raises(mk.MkError):
        mk.mlp_layer1_tc_raw(8, 192, 8, 8, 4, 16, 8, 16, 8, 0)       # features % 128


def test_timeout_path_aborts_cleanly_and_next_call_is_exact():
    """Every pipeline wait of the warp-specialised layer is bounded.  With a
    limit of one test per wait the waits run out (a bulk copy or an MMA takes
    longer than one test): the call must report MK_ST_TIMEOUT through the
    status word (MK_E_TIMEOUT), drain its copies and MMAs, free its tensor
    memory and leave the context usable, so that the next normal call on the
    same stream gives the float64-checked result."""
    F, B = 8192, 700
    vec, pa, pb = _problem(F, B, 31)
    net = E().MLP(F, H, seed=32)
    dv = torch.from_numpy(vec.view(np.int32).copy()).cuda()
    tpa, tpb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
    tiles = torch.empty(mk.mlp_w1_tiles_bytes(F), dtype=torch.uint8, device="cuda")
    mk.mlp_w1_tiles_raw(net.params.data_ptr(), F, H, tiles.data_ptr(), 0)
    b1 = net.params[F * H:F * H + H]
    h1 = torch.zeros((B, H), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = (dv.data_ptr(), F, tpa.data_ptr(), tpb.data_ptr(), B, tiles.data_ptr(), b1.data_ptr(), h1.data_ptr(),
            st.data_ptr())
    for _ in range(2):
        st.zero_()
        mk.mlp_layer1_tc_ws_bounded_raw(*args, 1, 0)
        torch.cuda.synchronize()
        assert mk.status_error(int(st.item())) == -11          # MK_E_TIMEOUT
    with pytest.raises(mk.MkError):
        mk.mlp_layer1_tc_ws_bounded_raw(*args, 0, 0)            # a zero limit is rejected
    st.zero_()
    h1.fill_(-7.0)
    mk.mlp_layer1_tc_ws_raw(*args, 0)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    X = _features(vec, pa, pb)
    w1t = torch.empty((H, F), dtype=torch.bfloat16, device="cuda")
    mk.mlp_w1t_bf16_raw(net.params.data_ptr(), F, H, w1t.data_ptr(), 0)
    W1 = w1t.float().cpu().numpy().astype(np.float64).T
    want = np.maximum(X @ W1 + b1.cpu().numpy().astype(np.float64), 0.0)
    scale = max(1.0, float(np.abs(want).max()))
    assert np.abs(h1.cpu().numpy() - want).max() <= 2e-5 * scale * np.sqrt(F / 128)
