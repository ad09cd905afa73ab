"""Schedule selection on the host (no GPU): candidate tables, cost-model
features (the segment-length histogram against the oracle's restatement, the
view-composition features), the tuned table keyed by GPU model and its file
round trip, and the held-out split of the problem sampler."""
import os

import pytest

import paper_2305_03448_gb300 as D
import synth
from oracle import mlp as OMLP

V = D


def test_candidate_counts(desc_lib):
    assert [D.candidate_count(o) for o in range(5)] == [8, 3, 2, 5, 6]
    with pytest.raises(D.DescError):
        D.candidate_count(7)


def test_features_encode_problem_and_candidate(desc_lib):
    # layout: [0,5) op, [5,7) dtype, [7] log2 n, [8] log2(aux+1), [9] log2 ratio, [10,18) histogram,
    # [18] log2 tile, [19] vectors, [20] log2 CTAs / group, [21,29) candidate, [29] load path,
    # [30] log2(K+1), [31] CTA pairs, [32,37) view counts, [37] depth, [38] hand-indexed, [39] dims
    p = D.make_problem(D.OP_SCAN, D.F32, 1 << 20)
    rows = [D.desc_features(p, c) for c in range(3)]
    for c, f in enumerate(rows):
        assert len(f) == D.NUM_FEATURES == 40
        assert f[0:5] == [0.0, 1.0, 0.0, 0.0, 0.0] and f[5:7] == [0.0, 1.0]
        assert abs(f[7] - 20 / 32) < 1e-6
        assert f[21 + c] == 1.0 and sum(f[21:29]) == 1.0
        assert f[32:37] == [0.0] * 5 and f[38] == 1.0 and f[39] == 1 / 8
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


def test_length_histogram_is_computed_behind_the_abi(desc_lib):
    """desc_features bins the raw segment lengths itself; the bins match the
    oracle's restatement of the bucket rule, including empty segments and
    lengths beyond the last bucket."""
    for seed, mx in ((1, 1 << 12), (2, 1 << 20), (3, 1 << 8)):
        L = synth.loguniform_lengths(777, seed=seed, max_len=mx)
        L[::13] = 0
        L[5] = 1 << 30
        p = D.make_problem(D.OP_SEGMENTED, D.F32, int(L.sum()), L.numel(), L)
        got = D.desc_features(p, 1)[10:18]
        want = OMLP.length_histogram(L.tolist())
        assert max(abs(a - b) for a, b in zip(got, want)) <= 1e-7
    # no lengths: the histogram stays zero
    assert D.desc_features(D.make_problem(D.OP_SEGMENTED, D.F32, 1000, 10), 0)[10:18] == [0.0] * 8


def test_view_composition_features(desc_lib):
    n = 1 << 20
    hier = [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
            ("select", V.THREAD, V.X)]
    f = D.desc_features(D.make_problem(D.OP_REDUCE, D.I32, n, view=([n], hier), grid=(n // 1024, 1, 1),
                                       block=(1024, 1, 1), level=V.BLOCK), 0)
    assert f[32:37] == [2 / 8, 0.0, 0.0, 0.0, 3 / 8] and f[38] == 1.0
    assert abs(f[7] - 20 / 32) < 1e-6 and abs(f[8] - 10 / 32) < 1e-4      # 1024 outputs
    # a column reduce of a row-major matrix: strided, the general kernel
    f = D.desc_features(D.make_problem(D.OP_REDUCE, D.F32, n, view=([1024, 1024], [("transpose", 0),
                                                                                 ("select", V.BLOCK, V.X)]),
                                       grid=(1024, 1, 1), block=(1, 1, 1), level=V.BLOCK), 0)
    assert f[34] == 1 / 8 and f[36] == 1 / 8 and f[38] == 0.0 and f[39] == 2 / 8
    # a reversed scan takes the general path; a split-off tail stays contiguous
    f = D.desc_features(D.make_problem(D.OP_SCAN, D.F32, n, view=([n], [("reverse", 0)])), 0)
    assert f[35] == 1 / 8 and f[38] == 0.0
    f = D.desc_features(D.make_problem(D.OP_SCAN, D.F32, n, view=([n], [("split_snd", 5, 0)])), 0)
    assert f[33] == 1 / 8 and f[38] == 1.0 and abs(f[7] - 19.99999 / 32) < 1e-4
    # a map(reverse) nested one level deep
    f = D.desc_features(D.make_problem(D.OP_SCAN, D.F32, n, view=([n], [("group", 64, 0), ("reverse", 1)])), 0)
    assert f[37] == 1 / 4


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
    # the same call through a view that lowers to the plain array shares the bucket
    n = 1 << 22
    hier = [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
            ("select", V.THREAD, V.X)]
    assert D.desc_tune_lookup(D.make_problem(D.OP_REDUCE, D.I32, n, view=([n], hier), grid=(n // 1024, 1, 1),
                                             block=(1024, 1, 1), level=V.GRID)) == 3
    path = os.path.join(tmp_path, "sched.txt")
    D.desc_tune_save(path)
    lines = [x for x in open(path) if not x.startswith("#")]
    assert len(lines) == 1 and len(lines[0].split()) == 6
    model = lines[0].split()[0]
    D.desc_tune_clear()
    assert D.desc_tune_lookup(p) == -1
    D.desc_tune_load(path)
    assert D.desc_tune_lookup(p) == 3
    # a table taken on another GPU model is not used here
    D.desc_tune_clear()
    open(path, "w").write("Some_Other_GPU " + " ".join(lines[0].split()[1:]) + "\n")
    D.desc_tune_load(path)
    assert D.desc_tune_lookup(p) == -1
    open(path, "w").write(model + " " + " ".join(lines[0].split()[1:]) + "\n")
    D.desc_tune_load(path)
    assert D.desc_tune_lookup(p) == 3
    with pytest.raises(D.DescError):
        D.desc_tune_record(p, 8)                            # out of range
    open(path, "w").write(model + " 0 0 22 0 9\n")
    with pytest.raises(D.DescError):
        D.desc_tune_load(path)
    open(path, "w").write("0 0 22 0 1\n")                   # the old five-field format
    with pytest.raises(D.DescError):
        D.desc_tune_load(path)
    D.desc_tune_clear()


def test_problem_sampler_is_seeded_and_splits_by_size_bucket():
    a = synth.tune_problems(30, seed=5)
    b = synth.tune_problems(30, seed=5)
    assert [(x["op"], x["n"], x["aux"]) for x in a] == [(x["op"], x["n"], x["aux"]) for x in b]
    assert {x["op"] for x in synth.tune_problems(200, seed=1)} == {0, 1, 2, 3, 4}
    import bench
    even = synth.tune_problems(300, seed=7, part="even")
    odd = synth.tune_problems(300, seed=8, part="odd")
    be = {bench.bucket_of(p) for p in even}
    bo = {bench.bucket_of(p) for p in odd}
    assert not be & bo
    assert all(k[2] % 2 == 0 for k in be) and all(k[2] % 2 == 1 for k in bo)
    assert sum(1 for p in odd if p["view"] is not None) > 30          # view compositions are drawn


def test_bucket_of_matches_the_library(desc_lib):
    """The bench's bucket rule agrees with the library's table keys: a
    problem recorded under its own bucket is found by every problem the rule
    puts in that bucket, and by no problem it puts elsewhere."""
    import bench
    probs = synth.tune_problems(120, seed=9)
    for p in probs:
        D.desc_tune_clear()
        D.desc_tune_record(p, 0)
        for q in probs[:40]:
            same = bench.bucket_of(q) == bench.bucket_of(p)
            assert (D.desc_tune_lookup(q) == 0) == same, (p, q)
    D.desc_tune_clear()
