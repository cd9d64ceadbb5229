"""GPU parity of the features, scaling, selector network and its training kernels."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sp = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global sp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_11938_gb300 as m

    m.lib()
    sp = m


def _long_row_missed(m=40_000, long_len=5000):
    """Rows of one entry and one row of long_len entries at row 1, which the
    8192-row sample (rows floor(k*M/8192)) skips."""
    lens = np.ones(m, np.int32)
    lens[1] = long_len
    return synth.from_lengths_random_cols(lens, 7000, 13, "long_row_missed")


def _sampled_long_rest_empty(m=40_000):
    sampled = np.unique((np.arange(8192, dtype=np.int64) * m) // 8192)
    lens = np.zeros(m, np.int32)
    lens[sampled] = 40
    return synth.from_lengths_random_cols(lens, 100, 14, "sampled_long_rest_empty")


def _feature_cases():
    lens = np.array([0, 0, 700, 0, 3, 0, 0, 70, 1, 0] * 50, np.int32)
    return [
        synth.config1(),
        synth.powerlaw(20_000, 3, xmax=3000, lmax=3000),  # sampled rows (M > 8192)
        synth.powerlaw(8_192, 4),                         # exactly the sample size
        synth.banded(100_000, 40, 5),
        synth.stencil(synth.STENCIL_7PT_3D, 30, 30, 30, 6),
        synth.blockdiag(777, 64, 7),
        synth.from_lengths_random_cols(lens, 800, 8, "empty_mix"),
        synth.tiny_random(3, 2, 0.5, 9),
        synth.uniform_random(40_000, 600, 10),            # every row longer than the 512 cap
        synth.from_lengths_random_cols(np.zeros(50, np.int32), 10, 11, "all_empty"),  # nnz = 0, idx NULL
        synth.from_lengths_random_cols(np.zeros(20_000, np.int32), 10, 12, "all_empty_sampled"),
        _long_row_missed(),                               # exact max sees a row the sample skips
        _sampled_long_rest_empty(),                       # exact statistics differ from the sample's
        synth.powerlaw(2_000_003, 15, xmax=5000, lmax=5000),  # M not a multiple of 4: the scalar tail of the pass
    ]


@pytest.mark.parametrize("ci", range(14))
def test_features_match_oracle(ci):
    a = _feature_cases()[ci]
    f = sp.spmv_features(sp.DeviceCSR.from_host(a)).cpu().numpy()
    ref = oracle.features(a).astype(np.float32)
    assert np.allclose(f, ref, rtol=2e-6, atol=0), np.stack([f, ref])


def _xy(seed, B=800):
    X = synth.vector(B * 16, seed, 0, 1).reshape(B, 16)
    y = (synth.vector(B, seed + 1, 0, 5).astype(np.int64)) % 5
    return X, y


def _theta(seed):
    return mlp.glorot_init(synth.vector(mlp.N_PARAMS, seed))


@pytest.mark.parametrize("B", [1, 63, 64, 65, 800])
def test_loss_grad_matches_oracle(B):
    theta = _theta(3)
    X, y = _xy(4, B)
    Xf = X.astype(np.float32)
    th32 = theta.astype(np.float32)
    loss_ref, g_ref = mlp.loss_and_grad(th32.astype(np.float64), Xf.astype(np.float64), y)
    loss, g = sp.spmv_mlp_loss_grad(torch.as_tensor(th32).cuda(), torch.as_tensor(Xf).cuda(),
                                    torch.as_tensor(y.astype(np.int32)).cuda())
    g = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.cpu()) - loss_ref) <= 1e-5 * abs(loss_ref)
    scale = np.abs(g_ref).max()
    assert np.all(np.abs(g - g_ref) <= 1e-4 * np.maximum(np.abs(g_ref), 1e-2 * scale))


def test_adam_matches_oracle():
    theta = _theta(5)
    g = synth.vector(mlp.N_PARAMS, 6) * 1e-2
    m0 = synth.vector(mlp.N_PARAMS, 7) * 1e-3
    v0 = np.abs(synth.vector(mlp.N_PARAMS, 8)) * 1e-5
    th_ref, m_ref, v_ref = mlp.adam_step(theta, g, m0, v0, 3, lr=1e-3)
    T = [torch.as_tensor(a.astype(np.float32)).cuda() for a in (theta, g, m0, v0)]
    sp.spmv_mlp_adam(T[0], T[1], T[2], T[3], 3, lr=1e-3)
    assert np.allclose(T[0].cpu().numpy(), th_ref, rtol=1e-5, atol=1e-7)
    assert np.allclose(T[2].cpu().numpy(), m_ref, rtol=1e-5, atol=1e-9)
    assert np.allclose(T[3].cpu().numpy(), v_ref, rtol=1e-5, atol=1e-12)


def test_train_matches_oracle_steps():
    """Ten fused full-batch Adam steps on the device follow ten oracle steps."""
    theta = _theta(9)
    X, y = _xy(10, 300)
    th = theta.astype(np.float32).astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    losses = []
    for t in range(1, 11):
        l, g = mlp.loss_and_grad(th, X.astype(np.float32).astype(np.float64), y)
        losses.append(l)
        th, m, v = mlp.adam_step(th, g, m, v, t, lr=3e-3)
    T = torch.as_tensor(theta.astype(np.float32)).cuda()
    M = torch.zeros_like(T)
    V = torch.zeros_like(T)
    hist = sp.spmv_mlp_train(T, M, V, torch.as_tensor(X.astype(np.float32)).cuda(),
                             torch.as_tensor(y.astype(np.int32)).cuda(), 10, 0, lr=3e-3).cpu().numpy()
    assert np.allclose(hist, losses, rtol=1e-4)
    assert np.allclose(T.cpu().numpy(), th, rtol=1e-3, atol=1e-5)


def test_forward_and_predict():
    theta = _theta(11)
    X, _ = _xy(12, 500)
    z_ref, _ = mlp.forward(theta.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    logits, pred = sp.spmv_mlp_forward(torch.as_tensor(theta.astype(np.float32)).cuda(),
                                       torch.as_tensor(X.astype(np.float32)).cuda())
    z = logits.cpu().numpy()
    assert np.allclose(z, z_ref, rtol=1e-4, atol=1e-5)
    srt = np.sort(z_ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-3  # argmax decided away from ties
    assert np.array_equal(pred.cpu().numpy()[clear], np.argmax(z_ref, axis=1)[clear])


def test_scale_matches_oracle():
    feats = np.stack([oracle.features(a) for a in _feature_cases()]).astype(np.float32)
    t = mlp.transform(feats.astype(np.float64))
    lo, hi = mlp.fit_scaling(t[:6])
    ref = mlp.scale(t, lo, hi)
    X = sp.spmv_mlp_scale(torch.as_tensor(feats).cuda(), torch.as_tensor(lo.astype(np.float32)).cuda(),
                          torch.as_tensor(hi.astype(np.float32)).cuda()).cpu().numpy()
    assert np.allclose(X, ref, atol=2e-6)


def test_select_matches_oracle():
    theta = _theta(13).astype(np.float32)
    cases = _feature_cases()
    feats = np.stack([oracle.features(a) for a in cases]).astype(np.float32)
    t = mlp.transform(feats.astype(np.float64))
    lo, hi = mlp.fit_scaling(t)
    model = sp.Model(theta, lo, hi)
    lo32, hi32 = lo.astype(np.float32).astype(np.float64), hi.astype(np.float32).astype(np.float64)
    for a, f in zip(cases, feats):
        x = mlp.scale(mlp.transform(f.astype(np.float64)), lo32, hi32).astype(np.float32)
        z_ref, _ = mlp.forward(theta.astype(np.float64), x[None, :].astype(np.float64))
        d = sp.DeviceCSR.from_host(a)
        fmt_out = torch.zeros(1, dtype=torch.int32, device="cuda")
        logits = torch.zeros(5, dtype=torch.float32, device="cuda")
        sp.spmv_select_async(d, model, fmt_out, logits)
        assert np.allclose(logits.cpu().numpy(), z_ref[0], rtol=1e-4, atol=1e-5)
        srt = np.sort(z_ref[0])
        if srt[-1] - srt[-2] > 1e-3:
            assert int(fmt_out.cpu()) == int(np.argmax(z_ref[0]))
            assert sp.spmv_select(d, model) == int(np.argmax(z_ref[0]))


def test_select_without_model():
    d = sp.DeviceCSR.from_host(synth.config1())
    with pytest.raises(sp.SpmvError) as ei:
        sp.spmv_select(d, None)
    assert ei.value.name == "NO_MODEL"


@pytest.mark.parametrize("name", ["selector_mlp.json", "selector_mlp_batch.json"])
def test_committed_model_on_corpus_matrices(name):
    """spmv_select with a shipped model picks, on regenerated corpus matrices, what the
    oracle's network picks from the features stored when the table was profiled."""
    import json
    import os

    data = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_11938_gb300", "data")
    with open(os.path.join(data, name)) as f:
        md = json.load(f)
    with open(os.path.join(data, "corpus_table.jsonl")) as f:
        recs = {json.loads(l)["index"]: json.loads(l) for l in f}
    model = sp.Model.load(os.path.join(data, name))
    theta = np.array(md["params"], np.float64)
    lo, hi = np.array(md["lo"], np.float64), np.array(md["hi"], np.float64)
    small = [i for i in sorted(recs) if recs[i]["nnz"] < 2_000_000][:12]
    for i in small:
        a = synth.corpus_matrix(i)
        d = sp.DeviceCSR.from_host(a)
        f = sp.spmv_features(d).cpu().numpy()
        assert np.array_equal(f, np.array(recs[i]["features"], np.float32)), i  # the table's features, bit for bit
        x = mlp.scale(mlp.transform(f.astype(np.float64)), lo, hi)
        z, _ = mlp.forward(theta, x[None, :])
        srt = np.sort(z[0])
        if srt[-1] - srt[-2] > 1e-3:
            assert sp.spmv_select(d, model) == int(np.argmax(z[0])), i


def test_features_exact_pass_unaligned_ptr_and_slot_reuse():
    """The pass over ptr with ptr 4 bytes off a 16-byte boundary (the scalar
    loads), and more calls than the ring has slots (each call finds its
    slot's accumulators at zero again)."""
    cases = [_long_row_missed(), _sampled_long_rest_empty(), synth.powerlaw(30_001, 16, xmax=900, lmax=900)]
    refs = [oracle.features(a).astype(np.float32) for a in cases]
    devs = []
    for a in cases:
        d = sp.DeviceCSR.from_host(a)
        buf = torch.empty(a.m + 2, dtype=torch.int32, device="cuda")
        buf[1:].copy_(d.ptr)
        assert buf[1:].data_ptr() % 16 == 4
        devs.append((d, sp.DeviceCSR(a.m, a.n, buf[1:], d.idx, d.val)))
    for rep in range(70):
        k = rep % len(cases)
        d_al, d_un = devs[k]
        for d in (d_al, d_un):
            f = sp.spmv_features(d).cpu().numpy()
            assert np.allclose(f, refs[k], rtol=2e-6, atol=0), (rep, cases[k].name, np.stack([f, refs[k]]))


def _forced_model(b3):
    """Zero weights: every logit is its bias, whatever the features."""
    p = np.zeros(sp.MLP_PARAMS, np.float32)
    p[5568:5573] = b3
    return sp.Model(p, np.zeros(16, np.float32), np.ones(16, np.float32))


def test_select_never_returns_ell_over_the_cap():
    """A network that always prefers ELL, then SELL: on a matrix with one long
    row the row sample misses, selection names ELL exactly while ELL's padded
    layout fits the model's cap and SELL from one byte below it -- the same
    footprint at which spmv_convert refuses ELL."""
    a = _long_row_missed()
    d = sp.DeviceCSR.from_host(a)
    model = _forced_model([0.0, 0.0, 1.0, 0.5, 0.0])
    ld = (a.m + 3) // 4 * 4
    foot = ld * 5000 * 12 + ld * 4
    model.set_max_bytes(foot)
    assert sp.spmv_select(d, model) == sp.SPMV_ELL
    fmt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    logits = torch.zeros(5, dtype=torch.float32, device="cuda")
    model.set_max_bytes(foot - 1)
    assert sp.spmv_select(d, model) == sp.SPMV_SELL
    sp.spmv_select_async(d, model, fmt, logits)
    assert int(fmt.item()) == sp.SPMV_SELL and logits.cpu().numpy().tolist() == [0.0, 0.0, 1.0, 0.5, 0.0]
    with pytest.raises(sp.SpmvError) as ei:
        sp.spmv_convert(sp.SPMV_ELL, d, {"max_bytes": foot - 1})
    assert ei.value.name == "TOO_LARGE"
    assert sp.spmv_convert(sp.SPMV_ELL, d, {"max_bytes": foot}).info()["stored_slots"] == ld * 5000
    with pytest.raises(sp.SpmvError):
        model.set_max_bytes(0)
