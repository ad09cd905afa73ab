"""Parity at the benchmark's full sizes, in the launch configurations that
bench.py times (every schedule candidate the autotuner may pick):

  reduce    2^30 int32 through group(1024)[[block]].group(32)[[warp]][[thread]]
            -- bit-exact against the oracle's int64 sum
  scan      2^28 FP32 -- every element within 1e-5 * sum_{q<=p}|x_q|
  transpose 16384^2 FP32 -- 2^20 sampled elements bit-exact
  matmul    8192^3 (SPLIT3 and BF16) -- 64 sampled rows against the FP64 product
  segmented 20,000 log-uniform segments (about 1.5e9 elements) -- 64 sampled
            segments in full, and the sums of all segments against their scans
  arg scan  2^28 FP32 arg-maximum, plain and through a reversed view -- sampled
            prefixes against the oracle's selection
  per-block 2^28 FP32 sums in segments of 1024 and 2^20 -- sampled segments in full
"""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import matmul as OM
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield desc_lib
    for op in range(4):
        D.desc_force_candidate(op, -1)
    torch.cuda.empty_cache()


def test_reduce_2_30_all_candidates():
    n = 1 << 30
    x = synth.ints_pm1000(n, seed=1, device="cuda")
    want, _ = O.reduce(x.cpu().numpy(), [n], [], V.GRID)
    ops = [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
           ("select", V.THREAD, V.X)]
    for c in range(D.candidate_count(D.OP_REDUCE)):
        D.desc_force_candidate(D.OP_REDUCE, c)
        got = D.desc_reduce(x, [n], ops, V.GRID, (n // 1024, 1, 1), (1024, 1, 1))
        assert int(got.item()) == int(want[0]), c
    D.desc_force_candidate(D.OP_REDUCE, -1)


def test_scan_2_28_all_candidates():
    n = 1 << 28
    x = synth.uniform_grid(n, seed=2, device="cuda")
    xh = x.cpu().numpy()
    want, pabs = O.scan(xh, np.zeros(n, np.float32), [n], [], V.GRID)
    out = torch.empty_like(x)
    for c in range(D.candidate_count(D.OP_SCAN)):
        D.desc_force_candidate(D.OP_SCAN, c)
        D.desc_scan(x, [n], [], V.GRID, out=out)
        err = np.abs(out.cpu().numpy().astype(np.float64) - want)
        assert np.all(err <= 1e-5 * pabs + 1e-30), (c, err.max())
    D.desc_force_candidate(D.OP_SCAN, -1)


def test_transpose_16384_sampled():
    T = 16384
    x = synth.normal_f32(T * T, seed=3, device="cuda").reshape(T, T)
    out = torch.empty(T, T, device="cuda")
    idx = synth.splitmix64(synth.stream_key(3, 5), 0, 1 << 20, device="cuda") & ((1 << 28) - 1)
    r, c = idx // T, idx % T
    for cand in range(D.candidate_count(D.OP_TRANSPOSE)):
        D.desc_force_candidate(D.OP_TRANSPOSE, cand)
        D.desc_transpose(x, [T, T], [("transpose", 0)], out, [T, T], [])
        # out[j][i] == in[i][j] at the sampled (i, j), compared as bit patterns
        assert torch.equal(out[c, r].view(torch.int32), x[r, c].view(torch.int32))
    D.desc_force_candidate(D.OP_TRANSPOSE, -1)


@pytest.mark.parametrize("prec,bound", [(D.MM_SPLIT3, 1e-5), (D.MM_BF16, 1e-2)])
def test_matmul_8192_sampled_rows(prec, bound):
    n = 8192
    A = synth.normal_f32(n * n, seed=1, stream=1, device="cuda").reshape(n, n)
    B = synth.normal_f32(n * n, seed=1, stream=2, device="cuda").reshape(n, n)
    C = D.desc_matmul(A, B, prec)
    rows = np.arange(7, n, n // 64)
    ref = OM.matmul_rows_f64(A.cpu().numpy(), B.cpu().numpy(), rows)
    assert OM.rel_frobenius(C.cpu().numpy()[rows], ref) <= bound


def test_segmented_20000_sampled_segments():
    nseg = 20000
    L = synth.loguniform_lengths(nseg, seed=7, device="cuda")
    off = synth.offsets_from_lengths(L)
    total = int(off[-1])
    x = synth.uniform_grid(total, seed=8, device="cuda")
    out = torch.empty_like(x)
    sums = torch.empty(nseg, device="cuda")
    g = D.SegmentedGraph(x, off, out, sums)
    g.launch()
    torch.cuda.synchronize()
    g.close()
    offh = off.cpu().numpy()
    pick = (synth.splitmix64(synth.stream_key(7, 9), 0, 64) & 0x7FFFFFFF).numpy() % nseg
    for s in pick:
        a, b = int(offh[s]), int(offh[s + 1])
        seg = x[a:b].cpu().numpy()
        want, wsum, pa, sabs = O.segmented_reduce_scan(seg, [0, b - a])
        got = out[a:b].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want) <= 1e-5 * pa + 1e-30)
        assert abs(float(sums[s]) - wsum[0]) <= 1e-5 * sabs[0] + 1e-30
    # every segment's total equals the scan at its last element
    nz = offh[1:] > offh[:-1]
    last = torch.from_numpy(offh[1:][nz] - 1).cuda()
    assert torch.equal(sums[torch.from_numpy(nz).cuda()], out[last])


def test_arg_scan_2_28_sampled():
    """The arg-maximum scan of 2^28 FP32 (the operators benchmark), plain and
    through a reversed view: sampled outputs against the oracle's selection
    over each prefix (ties to the smallest element index), and the last
    output against the arg-maximum reduce of the whole array."""
    n = 1 << 28
    x = synth.uniform_grid(n, seed=81, device="cuda")
    xn = x.cpu().numpy()
    rng = np.random.default_rng(3)
    # mostly short prefixes (the oracle converts each prefix to FP64), three long ones
    picks = [0, 1, 8191, 8192, 1 << 20, n - 1, int(rng.integers(0, n)), int(rng.integers(0, n))] + \
        [int(p) for p in rng.integers(0, 1 << 22, 4)]
    got = D.desc_scan(x, [n], [], V.GRID, flags=D.ARGMAX).cpu().numpy()
    for p in picks:
        assert int(got[p]) == O.arg_pick(xn[:p + 1], np.arange(p + 1), "argmax"), p
    assert int(got[n - 1]) == D.desc_reduce(x, [n], [], V.GRID, flags=D.ARGMAX).item()
    # reversed: point p is element n-1-p, its prefix the elements n-1-p .. n-1, written at n-1-p
    got = D.desc_scan(x, [n], [("reverse", 0)], V.GRID, flags=D.ARGMAX).cpu().numpy()
    for p in picks:
        e = n - 1 - p
        assert int(got[e]) == O.arg_pick(xn[e:], np.arange(e, n), "argmax"), p
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("m", [1024, 1 << 20])
def test_scan_per_block_2_28_sampled(m):
    """FP32 sum scans of 2^28 segmented per block of group(m)[[block]] (the
    operators benchmark): 24 sampled segments, each against the oracle's scan
    of that segment, every element within 1e-5 * sum_{q<=p}|x_q|."""
    n = 1 << 28
    x = synth.uniform_grid(n, seed=91, device="cuda")
    ops = [("group", m, 0), ("select", V.BLOCK, V.X)]
    got = D.desc_scan(x, [n], ops, V.BLOCK, (n // m, 1, 1), (1, 1, 1)).cpu().numpy()
    xn = x.cpu().numpy()
    rng = np.random.default_rng(5)
    segs = sorted({0, n // m - 1} | {int(s) for s in rng.integers(0, n // m, 22)})
    for sgi in segs:
        a, b = sgi * m, (sgi + 1) * m
        want, pa = O.scan(xn[a:b], np.zeros(m, np.float32), [m], [], V.GRID)
        err = np.abs(got[a:b].astype(np.float64) - want)
        assert np.all(err <= 1e-5 * pa + 1e-30), (sgi, float(err.max()))
    del x
    torch.cuda.empty_cache()
