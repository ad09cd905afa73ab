"""GPU parity of the batched segmented reduce + scan (one launch, CSR
offsets), its CUDA-graph replay and the one-launch-per-segment baseline,
against the oracle's per-segment sums and prefix sums."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import ops as O

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return desc_lib


def segments(nseg, max_len, seed, zero_every=0):
    L = synth.loguniform_lengths(nseg, seed=seed, max_len=max_len)
    if zero_every:
        L[::zero_every] = 0
    L[1::7] = 1
    return synth.offsets_from_lengths(L)


def check(x, off, scan, sums):
    want, wsum, pabs, sabs = O.segmented_reduce_scan(x.numpy(), off.numpy())
    if x.dtype == torch.int32:
        assert np.array_equal(scan.cpu().numpy(), want)
        assert np.array_equal(sums.cpu().numpy(), wsum)
    else:
        e = np.abs(scan.cpu().numpy().astype(np.float64) - want)
        assert np.all(e <= TOL * pabs + 1e-30), e.max()
        es = np.abs(sums.cpu().numpy().astype(np.float64) - wsum)
        assert np.all(es <= TOL * sabs + 1e-30), es.max()


@pytest.mark.parametrize("dt", ["i32", "f32"])
@pytest.mark.parametrize("nseg,max_len,zero", [(1, 100000, 0), (50, 5000, 5), (700, 300, 3), (300, 70000, 0),
                                               (2000, 40, 2)])
def test_batched_matches_oracle(dt, nseg, max_len, zero):
    off = segments(nseg, max_len, seed=nseg + max_len, zero_every=zero)
    n = int(off[-1])
    x = synth.ints_pm1000(n, seed=nseg) if dt == "i32" else synth.uniform_grid(n, seed=nseg)
    scan, sums = D.desc_segmented_reduce_scan(x.cuda(), off.cuda(), flags=D.CHECK_OFFSETS)
    check(x, off, scan, sums)


def test_graph_replay_and_per_segment_baseline():
    off = segments(400, 20000, seed=3, zero_every=9)
    n = int(off[-1])
    x = synth.uniform_grid(n, seed=3).cuda()
    offd = off.cuda()
    out = torch.full_like(x, 9.0)
    sums = torch.full((400,), 9.0, device="cuda")
    g = D.SegmentedGraph(x, offd, out, sums)
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    check(x.cpu(), off, out, sums)
    out2, sums2 = D.desc_segmented_reduce_scan_per_segment(x, off.tolist())
    check(x.cpu(), off, out2, sums2)
    g.close()
    xi = synth.ints_pm1000(n, seed=4).cuda()
    a, sa = D.desc_segmented_reduce_scan(xi, offd)
    b, sb = D.desc_segmented_reduce_scan_per_segment(xi, off.tolist())
    assert torch.equal(a, b) and torch.equal(sa, sb)


def test_in_place_and_all_empty():
    off = segments(100, 3000, seed=5)
    n = int(off[-1])
    x = synth.ints_pm1000(n, seed=5)
    xd = x.cuda()
    scan, sums = D.desc_segmented_reduce_scan(xd, off.cuda(), out=xd)
    check(x, off, scan, sums)
    z = torch.zeros(4, dtype=torch.int64).cuda()
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    _, s = D.desc_segmented_reduce_scan(e, z, sums=torch.full((3,), 5.0, device="cuda"))
    assert s.tolist() == [0.0, 0.0, 0.0]


def test_bad_offsets_are_rejected_when_checked():
    off = torch.tensor([0, 10, 5, 20], dtype=torch.int64).cuda()
    x = torch.zeros(20, device="cuda")
    with pytest.raises(D.DescError) as e:
        D.desc_segmented_reduce_scan(x, off, flags=D.CHECK_OFFSETS)
    assert e.value.status == 2
    with pytest.raises(D.DescError):
        D.SegmentedGraph(x, off, torch.empty_like(x), torch.empty(3, device="cuda"))


@pytest.mark.parametrize("cand", range(5))
@pytest.mark.parametrize("lens", ["short", "mixed", "long"])
def test_every_segment_schedule(cand, lens):
    """Each schedule of the batched call, forced -- the look-back scan over
    tiles of 16384 / 8192 / 4096 points, one warp per segment, one CTA per
    segment -- with sums, maxima, minima and exclusive scans, empty and
    one-point segments, against the oracle."""
    spec = {"short": (3000, 40, 4), "mixed": (600, 20000, 7), "long": (6, 300000, 0)}[lens]
    off = segments(spec[0], spec[1], seed=cand + spec[0], zero_every=spec[2])
    n = int(off[-1])
    D.desc_force_candidate(D.OP_SEGMENTED, cand)
    try:
        for dt in ("i32", "f32"):
            x = synth.ints_pm1000(n, seed=cand + 1) if dt == "i32" else synth.uniform_grid(n, seed=cand + 2)
            scan, sums = D.desc_segmented_reduce_scan(x.cuda(), off.cuda())
            check(x, off, scan, sums)
            for op, flag in (("max", D.MAX), ("min", D.MIN), ("sum", D.EXCLUSIVE), ("max", D.MAX | D.EXCLUSIVE)):
                sc, tot = D.desc_segmented_reduce_scan(x.cuda(), off.cuda(), flags=flag)
                want, wtot, pa, sa = O.segmented_op(x.numpy(), off.numpy(), op, bool(flag & D.EXCLUSIVE))
                if dt == "i32" or op != "sum":
                    assert np.array_equal(sc.cpu().numpy().astype(np.float64), want.astype(np.float64))
                    assert np.array_equal(tot.cpu().numpy().astype(np.float64), wtot.astype(np.float64))
                else:
                    assert np.all(np.abs(sc.cpu().numpy().astype(np.float64) - want) <= TOL * pa + 1e-30)
                    assert np.all(np.abs(tot.cpu().numpy().astype(np.float64) - wtot) <= TOL * sa + 1e-30)
    finally:
        D.desc_force_candidate(D.OP_SEGMENTED, -1)
