"""Schedule selection on the host (no GPU): candidate tables, cost-model
features, the tuned table and its file round trip."""
import os

import pytest

import paper_2305_03448_gb300 as D
import synth


def test_candidate_counts(desc_lib):
    assert [D.candidate_count(o) for o in range(5)] == [8, 3, 2, 3, 6]
    with pytest.raises(D.DescError):
        D.candidate_count(7)


def test_features_encode_problem_and_candidate(desc_lib):
    # layout: [0,5) op, [5,7) dtype, [7] log2 n, [8] log2(aux+1), [9] log2 ratio, [10,18) histogram,
    # [18] log2 tile, [19] vectors, [20] log2 CTAs / group, [21,29) candidate, [29] load path,
    # [30] log2(K+1), [31] CTA pairs
    p = D.make_problem(D.OP_SCAN, D.F32, 1 << 20)
    rows = [D.desc_features(p, c) for c in range(3)]
    for c, f in enumerate(rows):
        assert len(f) == D.NUM_FEATURES
        assert f[0:5] == [0.0, 1.0, 0.0, 0.0, 0.0] and f[5:7] == [0.0, 1.0]
        assert abs(f[7] - 20 / 32) < 1e-6
        assert f[21 + c] == 1.0 and sum(f[21:29]) == 1.0
    assert rows[0][18] > rows[1][18] > rows[2][18]          # tile sizes 16384 > 8192 > 4096
    L = synth.loguniform_lengths(100, seed=1, max_len=1 << 12)
    ps = D.make_problem(D.OP_SEGMENTED, D.I32, int(L.sum()), 100, L)
    f = D.desc_features(ps, 0)
    assert abs(sum(f[10:18]) - 1.0) < 1e-6 and f[5] == 1.0 and f[3] == 1.0
    with pytest.raises(D.DescError):
        D.desc_features(p, 3)                               # scan has 3 candidates
    pm = D.make_problem(D.OP_MATMUL, D.F32, 2048, 1024, k=4096)
    mm = [D.desc_features(pm, c) for c in range(6)]
    for c, f in enumerate(mm):
        assert f[4] == 1.0 and abs(f[7] - 11 / 32) < 1e-6 and abs(f[30] - 12 / 32) < 1e-3
        assert f[21 + c] == 1.0
    assert [f[31] for f in mm] == [1.0, 0.0, 1.0, 0.0, 1.0, 1.0]   # CTA pairs
    assert mm[0][18] > mm[1][18] and mm[0][20] > mm[2][20]   # pair tiles larger; narrow groups
    assert mm[4][18] > mm[0][18] and mm[4][20] > mm[5][20]   # 256 x 512 pair tiles; narrow groups


def test_table_record_lookup_save_load(desc_lib, tmp_path):
    D.desc_tune_clear()
    p = D.make_problem(D.OP_REDUCE, D.I32, 1 << 22, 0)
    assert D.desc_tune_lookup(p) == -1
    D.desc_tune_record(p, 3)
    assert D.desc_tune_lookup(p) == 3
    q = D.make_problem(D.OP_REDUCE, D.I32, (1 << 22) + 5, 0)   # same log2 bucket
    assert D.desc_tune_lookup(q) == 3
    r = D.make_problem(D.OP_REDUCE, D.F32, 1 << 22, 0)         # other dtype: not recorded
    assert D.desc_tune_lookup(r) == -1
    path = os.path.join(tmp_path, "sched.txt")
    D.desc_tune_save(path)
    D.desc_tune_clear()
    assert D.desc_tune_lookup(p) == -1
    D.desc_tune_load(path)
    assert D.desc_tune_lookup(p) == 3
    with pytest.raises(D.DescError):
        D.desc_tune_record(p, 8)                            # out of range
    open(path, "w").write("0 0 22 0 9\n")
    with pytest.raises(D.DescError):
        D.desc_tune_load(path)
    D.desc_tune_clear()


def test_problem_sampler_is_seeded():
    a = synth.tune_problems(30, seed=5)
    b = synth.tune_problems(30, seed=5)
    assert [(x["op"], x["n"], x["aux"]) for x in a] == [(x["op"], x["n"], x["aux"]) for x in b]
    assert {x["op"] for x in synth.tune_problems(200, seed=1)} == {0, 1, 2, 3, 4}
