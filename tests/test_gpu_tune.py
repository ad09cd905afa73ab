"""GPU checks of the schedule machinery: the cost model's kernels against the
oracle's FP64 twin (forward, gradient within 1e-4 relative, Adam), every
schedule candidate against the oracle, the exhaustive tuner, predictions from
two host threads at once, and a small regret study of the learned picker
against the exhaustive tuner on held-out size buckets."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import mlp as OMLP
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu
F, H = D.NUM_FEATURES, 64


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield desc_lib
    D.desc_tune_clear()


def data(rows, seed):
    X = synth.normal_f32(rows * F, seed=seed).reshape(rows, F)
    t = synth.normal_f32(rows, seed=seed + 1)
    return X, t


def test_forward_matches_fp64_twin():
    p = synth.mlp_init(F, H, seed=1)
    X, _ = data(300, 2)
    m = D.CostModel(p)
    y = m.forward(X.cuda()).cpu().double().numpy()
    want, _ = OMLP.forward(p.double().numpy(), X.double().numpy(), F, H)
    assert np.max(np.abs(y - want)) <= 1e-5 * max(1.0, np.max(np.abs(want)))


def test_gradient_matches_fp64_twin():
    p = synth.mlp_init(F, H, seed=3)
    p[H * F:H * F + H] = 0.05
    X, t = data(257, 4)
    m = D.CostModel(p)
    g = m.backward(X.cuda(), t.cuda()).cpu().double().numpy()
    _, want = OMLP.backward(p.double().numpy(), X.double().numpy(), t.double().numpy(), F, H)
    assert np.linalg.norm(g - want) <= 1e-4 * np.linalg.norm(want)


def test_adam_matches_fp64_twin_and_zero_lr_is_a_no_op():
    p = synth.mlp_init(F, H, seed=5)
    X, t = data(64, 6)
    m = D.CostModel(p)
    g = m.backward(X.cuda(), t.cuda()).clone()
    m.adam(1, 1e-3)
    want, _, _ = OMLP.adam(p.double().numpy(), g.cpu().double().numpy(), np.zeros(p.numel()), np.zeros(p.numel()),
                           1, 1e-3)
    assert np.max(np.abs(m.p.cpu().double().numpy() - want)) <= 1e-6
    m2 = D.CostModel(p)
    m2.backward(X.cuda(), t.cuda())
    m2.adam(1, 0.0)
    assert torch.equal(m2.p.cpu(), p)


def test_training_fits_and_pick_is_argmin():
    p = synth.mlp_init(F, H, seed=7)
    X, t = data(8, 8)
    m = D.CostModel(p)
    l0 = float(np.mean((OMLP.forward(p.double().numpy(), X.double().numpy(), F, H)[0] - t.numpy()) ** 2))
    loss = m.train(X.cuda(), t.cuda(), epochs=2000, batch=8, lr=3e-3)
    assert loss < 1e-2 * l0
    best, pred = m.pick(X[:5].cuda())
    want, _ = OMLP.forward(m.p.cpu().double().numpy(), X[:5].double().numpy(), F, H)
    assert best == int(np.argmin(want))
    assert np.allclose(pred.cpu().numpy(), want, atol=1e-4)


def test_every_candidate_is_correct():
    """Each schedule candidate, forced, matches the oracle."""
    n = (1 << 20) + 77
    xi = synth.ints_pm1000(n, seed=9)
    xf = synth.uniform_grid(n, seed=9)
    for c in range(D.candidate_count(D.OP_REDUCE)):
        D.desc_force_candidate(D.OP_REDUCE, c)
        assert int(D.desc_reduce(xi.cuda(), [n], [], V.GRID).item()) == int(O.reduce(xi.numpy(), [n], [], V.GRID)[0][0])
        g = 64
        got = D.desc_reduce(xi[: g * 16384].cuda(), [g * 16384], [("group", 16384, 0), ("select", V.BLOCK, V.X)],
                            V.BLOCK, (g, 1, 1), (1, 1, 1)).cpu().numpy()
        want, _ = O.reduce(xi[: g * 16384].numpy(), [g * 16384], [("group", 16384, 0), ("select", V.BLOCK, V.X)],
                           V.BLOCK)
        assert np.array_equal(got, want)
    D.desc_force_candidate(D.OP_REDUCE, -1)
    for c in range(D.candidate_count(D.OP_SCAN)):
        D.desc_force_candidate(D.OP_SCAN, c)
        got = D.desc_scan(xi.cuda(), [n], [], V.GRID).cpu().numpy()
        want, _ = O.scan(xi.numpy(), np.zeros(n, np.int32), [n], [], V.GRID)
        assert np.array_equal(got, want)
        gotf = D.desc_scan(xf.cuda(), [n], [], V.GRID).cpu().numpy()
        wantf, pa = O.scan(xf.numpy(), np.zeros(n, np.float32), [n], [], V.GRID)
        assert np.all(np.abs(gotf - wantf) <= 1e-5 * pa)
    D.desc_force_candidate(D.OP_SCAN, -1)
    L = synth.loguniform_lengths(500, seed=10, max_len=20000)
    off = synth.offsets_from_lengths(L)
    x = synth.ints_pm1000(int(off[-1]), seed=10)
    want, wsum, _, _ = O.segmented_reduce_scan(x.numpy(), off.numpy())
    for c in range(D.candidate_count(D.OP_SEGMENTED)):
        D.desc_force_candidate(D.OP_SEGMENTED, c)
        s, sums = D.desc_segmented_reduce_scan(x.cuda(), off.cuda())
        assert np.array_equal(s.cpu().numpy(), want) and np.array_equal(sums.cpu().numpy(), wsum)
    D.desc_force_candidate(D.OP_SEGMENTED, -1)
    R, C = 300, 1000
    xt = synth.normal_f32(R * C, seed=11).reshape(R, C)
    for c in range(D.candidate_count(D.OP_TRANSPOSE)):
        D.desc_force_candidate(D.OP_TRANSPOSE, c)
        out = torch.empty(C, R, device="cuda")
        D.desc_transpose(xt.cuda(), [R, C], [("transpose", 0)], out, [C, R], [])
        assert torch.equal(out.cpu(), xt.t())
    D.desc_force_candidate(D.OP_TRANSPOSE, -1)


def test_exhaustive_tuner_records_the_fastest():
    arena = D.TuneArena(1 << 22, 1000, max_mm=2048)
    D.desc_tune_clear()
    for prob in [dict(op=1, dtype=1, n=1 << 22, aux=0, lengths=None), dict(op=0, dtype=0, n=1 << 21, aux=0, lengths=None),
                 dict(op=2, dtype=1, n=1 << 22, aux=1 << 11, lengths=None),
                 dict(op=4, dtype=1, n=2048, aux=1024, lengths=None, k=512)]:
        us = D.desc_tune_measure(prob, arena, reps=5)
        assert len(us) == D.candidate_count(prob["op"]) and min(us) > 0
        best = D.desc_tune_exhaustive(prob, arena, reps=5)
        assert 0 <= best < len(us)
        assert D.desc_tune_lookup(prob) == best
    D.desc_tune_clear()


@pytest.mark.parametrize("M,N,K", [(512, 768, 320), (384, 256, 200), (1000, 700, 129)])
def test_every_matmul_candidate_is_correct(M, N, K):
    """Each matmul schedule (CTA pairs or single CTAs, wide or narrow
    rasterisation groups), forced, gives the same BF16 products."""
    from oracle import matmul as OM
    A = synth.normal_f32(M * K, seed=M, stream=1).reshape(M, K)
    B = synth.normal_f32(K * N, seed=M, stream=2).reshape(K, N)
    emul = OM.matmul_f64(OM.bf16_rne(A.numpy()), OM.bf16_rne(B.numpy()))
    for c in range(D.candidate_count(D.OP_MATMUL)):
        D.desc_force_candidate(D.OP_MATMUL, c)
        for prec in (D.MM_BF16, D.MM_SPLIT3):
            C = D.desc_matmul(A.cuda(), B.cuda(), prec).cpu().numpy()
            if prec == D.MM_BF16:
                assert OM.rel_frobenius(C, emul) <= 2e-6, c
            else:
                assert OM.rel_frobenius(C, OM.split3_product_f64(A.numpy(), B.numpy())) <= 2e-6, c
    D.desc_force_candidate(D.OP_MATMUL, -1)


def test_learned_picker_small_regret_study():
    """A small version of the regret study the bench runs at full size: the
    held-out problems share no tuned-table bucket with the training ones."""
    import bench
    arena = D.TuneArena(1 << 27, 5000, max_mm=4096)
    train = synth.tune_problems(160, seed=21, part="even")
    test = synth.tune_problems(60, seed=22, part="odd")
    model = D.CostModel(synth.mlp_init(F, H, seed=23))
    r = bench.regret_study(D, train, test, arena, model, epochs=200, batch=64, lr=2e-3, reps=3, retime_reps=7)
    print(r)
    assert r["overlap"] == {"bucket": 0, "shape": 0}
    assert r["final_loss"] < 0.5
    assert r["mean_regret"] <= 0.15
    # what the trained model gains over the method without it (always the default candidate)
    assert r["mean_regret"] < r["default_mean_regret"]
    # the model predicts for a problem through the library's own picker too
    model.install()
    c = model.predict_problem(test[0])
    assert D.desc_tune_lookup(test[0]) == c
    D.lib().desc_tune_set_model(None, 0, 0)


def test_predictions_from_two_threads():
    """desc_tune_predict from two host threads on two streams at once: every
    pick is the argmin of the oracle twin's predictions for that problem."""
    import threading
    p = synth.mlp_init(F, H, seed=31)
    model = D.CostModel(p)
    model.install()
    probs = synth.tune_problems(60, seed=32)
    want = []
    for prob in probs:
        rows = np.array(D.feature_rows(prob), dtype=np.float32).astype(np.float64)
        y, _ = OMLP.forward(p.double().numpy(), rows, F, H)
        want.append(int(np.argmin(y)))
    got = [[None] * len(probs) for _ in range(2)]
    errors = []

    def worker(t):
        try:
            s = torch.cuda.Stream()
            order = range(len(probs)) if t == 0 else reversed(range(len(probs)))
            for _ in range(3):
                for i in order:
                    c = model.predict_problem(probs[i], stream=s)
                    if got[t][i] is not None and got[t][i] != c:
                        errors.append((t, i, "unstable"))
                    got[t][i] = c
        except Exception as e:          # noqa: BLE001 -- reported below
            errors.append((t, repr(e)))

    th = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    D.lib().desc_tune_set_model(None, 0, 0)
    D.desc_tune_clear()
    assert not errors, errors[:5]
    # near-ties of the FP32 kernel and the FP64 twin may pick differently; allow
    # only those
    for t in range(2):
        for i, prob in enumerate(probs):
            if got[t][i] != want[i]:
                rows = np.array(D.feature_rows(prob), dtype=np.float64)
                y, _ = OMLP.forward(p.double().numpy(), rows, F, H)
                assert abs(y[got[t][i]] - y[want[i]]) <= 1e-5 * max(1.0, abs(y[want[i]])), (t, i)
