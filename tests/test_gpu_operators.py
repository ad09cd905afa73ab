"""Maximum, minimum and exclusive scans on the GPU against the oracle
(flags DESC_MAX, DESC_MIN, DESC_EXCLUSIVE): bit-exact for the maximum and
minimum in both dtypes and for int32 sums, FP32 exclusive sums within
1e-5 * sum |x| of the points before each one."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu
TOL = 1e-5
OPS = [("max", D.MAX), ("min", D.MIN)]


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return desc_lib


def signed_floats(n, seed):
    return synth.uniform_grid(n, seed=seed) - 2.0        # all negative: the maximum is not 0


@pytest.mark.parametrize("n", [1, 77, 4097, (1 << 20) + 5, 50_000_000])
@pytest.mark.parametrize("op,flag", OPS)
def test_reduce_max_min(n, op, flag):
    for x in (synth.ints_pm1000(n, seed=n), signed_floats(n, n + 1)):
        got = D.desc_reduce(x.cuda(), [n], [], V.GRID, flags=flag).cpu().numpy()
        want = O.reduce_op(x.numpy(), [n], [], V.GRID, op)
        assert np.array_equal(got.astype(np.float64), want.astype(np.float64))


@pytest.mark.parametrize("op,flag", OPS)
def test_reduce_max_min_views(op, flag):
    n = 1 << 20
    x = synth.ints_pm1000(n, seed=3)
    views = [([("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
               ("select", V.THREAD, V.X)], V.BLOCK, (1024, 1, 1), (1024, 1, 1)),
             ([("group", 16, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (n // 16, 1, 1), (1, 1, 1)),
             ([("reverse", 0), ("group", 4096, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (256, 1, 1), (1, 1, 1)),
             ([("group", 64, 0), ("reverse", 0), ("select", V.BLOCK, V.X)], V.BLOCK, (n // 64, 1, 1), (1, 1, 1))]
    for ops, lvl, g, b in views:
        got = D.desc_reduce(x.cuda(), [n], ops, lvl, g, b, flags=flag).cpu().numpy()
        assert np.array_equal(got, O.reduce_op(x.numpy(), [n], ops, lvl, op, g, b))
    D.desc_force_generic(True)
    try:
        got = D.desc_reduce(x.cuda(), [n], views[0][0], V.BLOCK, views[0][2], views[0][3], flags=flag).cpu().numpy()
        assert np.array_equal(got, O.reduce_op(x.numpy(), [n], views[0][0], V.BLOCK, op))
    finally:
        D.desc_force_generic(False)


def test_reduce_nan_and_empty():
    x = torch.tensor([float("nan"), -3.0, float("nan"), -5.0])
    assert D.desc_reduce(x.cuda(), [4], [], V.GRID, flags=D.MAX).item() == -3.0
    assert D.desc_reduce(x.cuda(), [4], [], V.GRID, flags=D.MIN).item() == -5.0
    e = torch.zeros(0, dtype=torch.int32)
    # an empty split of the array reduces to the identity
    out = D.desc_reduce(torch.zeros(8, dtype=torch.int32).cuda(), [8], [("split_fst", 0, 0)], V.GRID, flags=D.MAX)
    assert int(out.item()) == -(2 ** 31)
    out = D.desc_reduce(torch.zeros(8).cuda(), [8], [("split_fst", 0, 0)], V.GRID, flags=D.MIN)
    assert out.item() == float("inf")
    with pytest.raises(D.DescError):
        D.desc_reduce(torch.zeros(8).cuda(), [8], [], V.GRID, flags=D.MAX | D.MIN)
    with pytest.raises(D.DescError):
        D.desc_reduce(torch.zeros(8).cuda(), [8], [], V.GRID, kahan=True, flags=D.MAX)
    del e


def check_scan(x, op, excl, ops=(), lvl=V.GRID, g=None, b=None, inplace=False):
    n = x.numel()
    flags = ({"max": D.MAX, "min": D.MIN}.get(op, 0)) | (D.EXCLUSIVE if excl else 0)
    xd = x.cuda()
    out = xd if inplace else torch.zeros_like(xd)
    got = D.desc_scan(xd, [n], list(ops), lvl, g, b, out=out, flags=flags).cpu().numpy()
    want, pa = O.scan_op(x.numpy(), x.numpy() if inplace else np.zeros_like(x.numpy()), [n], list(ops), lvl, op,
                         excl, g, b)
    if x.dtype == torch.int32 or op != "sum":
        assert np.array_equal(got.astype(np.float64), want.astype(np.float64))
    else:
        assert np.all(np.abs(got.astype(np.float64) - want) <= TOL * pa + 1e-30)


@pytest.mark.parametrize("n", [1, 5, 4096, 4097, 16384, 16385, 3 * 16384 + 11, (1 << 20) + 3, 20_000_000])
@pytest.mark.parametrize("op,excl", [("sum", True), ("max", False), ("max", True), ("min", False), ("min", True)])
def test_scan_operators(n, op, excl):
    check_scan(synth.ints_pm1000(n, seed=n), op, excl)
    check_scan(signed_floats(n, n + 3) if op != "sum" else synth.uniform_grid(n, seed=n + 3), op, excl)


@pytest.mark.parametrize("m", [7, 4096, 5000, 16384, 70000])
@pytest.mark.parametrize("op,excl", [("sum", True), ("max", False), ("min", True)])
def test_scan_operators_segments(m, op, excl):
    g = max(1, 600000 // m)
    x = synth.ints_pm1000(g * m, seed=m)
    check_scan(x, op, excl, [("group", m, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (g, 1, 1), (1, 1, 1))


def test_exclusive_in_place_and_generic_views():
    n = 300001
    check_scan(synth.ints_pm1000(n, seed=4), "sum", True, inplace=True)
    check_scan(synth.uniform_grid(n, seed=5), "max", True, [("reverse", 0)])
    check_scan(synth.ints_pm1000(n, seed=6), "min", True, [("split_snd", 3, 0)])


@pytest.mark.parametrize("op,excl", [("sum", True), ("max", False), ("max", True), ("min", False)])
def test_segmented_operators(op, excl):
    L = synth.loguniform_lengths(900, seed=12, max_len=40000)
    L[::7] = 0
    off = synth.offsets_from_lengths(L)
    flags = ({"max": D.MAX, "min": D.MIN}.get(op, 0)) | (D.EXCLUSIVE if excl else 0)
    for x in (synth.ints_pm1000(int(off[-1]), seed=13), synth.uniform_grid(int(off[-1]), seed=14)):
        sc, tot = D.desc_segmented_reduce_scan(x.cuda(), off.cuda(), flags=flags)
        want, wtot, pa, sa = O.segmented_op(x.numpy(), off.numpy(), op, excl)
        if x.dtype == torch.int32 or op != "sum":
            assert np.array_equal(sc.cpu().numpy().astype(np.float64), want.astype(np.float64))
            assert np.array_equal(tot.cpu().numpy().astype(np.float64), wtot.astype(np.float64))
        else:
            assert np.all(np.abs(sc.cpu().numpy().astype(np.float64) - want) <= TOL * pa + 1e-30)
            assert np.all(np.abs(tot.cpu().numpy().astype(np.float64) - wtot) <= TOL * sa + 1e-30)
    # all segments empty: totals are the identity
    off0 = torch.zeros(4, dtype=torch.int64)
    _, tot = D.desc_segmented_reduce_scan(torch.zeros(0).cuda(), off0.cuda(), flags=flags)
    assert np.array_equal(tot.cpu().numpy(), np.full(3, O.identity(op, False), np.float32))
