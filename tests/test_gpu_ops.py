"""GPU parity of reduce, scan and transpose against the oracle, through the
C ABI.  Sizes span several tiles with ragged tails; integers must match bit
for bit, FP32 within 1e-5 * sum|x| (reduce: total, scan: per prefix)."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return desc_lib


def dev(t):
    return t.to("cuda")


def check_reduce(x, base, ops, lvl, grid=None, block=None, kahan=False):
    got = D.desc_reduce(dev(x), base, ops, lvl, grid, block, kahan=kahan).cpu().numpy()
    want, sabs = O.reduce(x.numpy(), base, ops, lvl, grid, block)
    if x.dtype == torch.int32:
        assert np.array_equal(got, want)
    else:
        err = np.abs(got.astype(np.float64) - want)
        assert np.all(err <= TOL * sabs + 1e-30), (err.max(), sabs.max())


# ------------------------------------------------------------------ reduce
def test_reduce_hierarchical_view_int32():
    """group(1024) per block, group(32) per warp, one element per lane."""
    n = 1 << 22
    x = synth.ints_pm1000(n, seed=1)
    ops = [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
           ("select", V.THREAD, V.X)]
    for lvl in (V.GRID, V.BLOCK, V.WARP, V.THREAD):
        check_reduce(x, [n], ops, lvl, (n // 1024, 1, 1), (1024, 1, 1))


@pytest.mark.parametrize("n", [1, 3, 4, 5, 31, 4095, 4096, 4097, 65537, 100003, (1 << 20) + 7])
@pytest.mark.parametrize("dt", ["i32", "f32", "kahan"])
def test_reduce_full(n, dt):
    x = synth.ints_pm1000(n, seed=n) if dt == "i32" else synth.uniform_grid(n, seed=n)
    check_reduce(x, [n], [], V.GRID, kahan=(dt == "kahan"))


@pytest.mark.parametrize("off", [1, 2, 3, 5])
def test_reduce_misaligned_start(off):
    n = 50000
    x = synth.uniform_grid(n, seed=off)
    check_reduce(x, [n], [("split_snd", off, 0)], V.GRID)
    xi = synth.ints_pm1000(n, seed=off)
    check_reduce(xi, [n], [("split_snd", off, 0), ("split_fst", n - 2 * off, 0)], V.GRID)


@pytest.mark.parametrize("m", [1, 5, 16, 17, 32, 1000, 4096, 5000, 100000])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_reduce_segments(m, dt):
    g = max(1, 400000 // m)
    n = g * m
    x = synth.ints_pm1000(n, seed=m) if dt == "i32" else synth.uniform_grid(n, seed=m)
    check_reduce(x, [n], [("group", m, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (g, 1, 1), (1, 1, 1))


@pytest.mark.parametrize("R,C", [(3, 5), (64, 100), (1000, 37), (37, 20000)])
def test_reduce_affine_paths(R, C):
    xi = synth.ints_pm1000(R * C, seed=R + C)
    # column sums: transpose, one block per column
    ops = [("transpose", 0), ("select", V.BLOCK, V.X)]
    check_reduce(xi, [R, C], ops, V.BLOCK, (C, 1, 1), (1, 1, 1))
    # everything through a reversed, transposed view
    check_reduce(xi, [R, C], [("reverse", 1), ("transpose", 0)], V.GRID)
    xf = synth.uniform_grid(R * C, seed=R * C)
    check_reduce(xf, [R, C], ops, V.BLOCK, (C, 1, 1), (1, 1, 1))
    check_reduce(xf, [R, C], [("transpose", 0)], V.GRID, kahan=True)


def test_reduce_empty_and_zero_extent():
    x = synth.ints_pm1000(64, seed=2)
    got = D.desc_reduce(dev(x), [64], [("split_fst", 0, 0)], V.GRID).cpu()
    assert got.tolist() == [0]


def test_reduce_kahan_beats_plain_on_hard_data():
    # one large value and many small ones of the opposite sign
    n = 1 << 22
    x = torch.full((n,), 1e-4, dtype=torch.float32)
    x[0] = 1e4
    exact = 1e4 + (n - 1) * float(np.float32(1e-4))
    p = D.desc_reduce(dev(x), [n], [], V.GRID).item()
    k = D.desc_reduce(dev(x), [n], [], V.GRID, kahan=True).item()
    assert abs(k - exact) <= abs(p - exact)
    assert abs(k - exact) <= 1e-6 * exact


# ------------------------------------------------------------------ scan
def check_scan(x, base, ops, lvl, grid=None, block=None, inplace=False, out0=None):
    xd = dev(x)
    if out0 is None:
        out0 = torch.zeros_like(x)
    out = xd if inplace else dev(out0.clone())
    got = D.desc_scan(xd, base, ops, lvl, grid, block, out=out).cpu().numpy()
    want, pabs = O.scan(x.numpy(), out0.numpy() if not inplace else x.numpy(), base, ops, lvl, grid, block)
    if x.dtype == torch.int32:
        assert np.array_equal(got, want)
    else:
        err = np.abs(got.astype(np.float64) - want)
        assert np.all(err <= TOL * pabs + 1e-30), err.max()


@pytest.mark.parametrize("n", [1, 17, 4096, 4097, 3 * 4096 + 5, 131072, (1 << 20) + 3, 5_000_000])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_scan_plain(n, dt):
    x = synth.ints_pm1000(n, seed=n) if dt == "i32" else synth.uniform_grid(n, seed=n)
    check_scan(x, [n], [], V.GRID)


@pytest.mark.parametrize("m", [1, 7, 16, 1000, 1024, 4096, 5000, 70000])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_scan_segments(m, dt):
    g = max(1, 300000 // m)
    n = g * m
    x = synth.ints_pm1000(n, seed=m) if dt == "i32" else synth.uniform_grid(n, seed=m)
    check_scan(x, [n], [("group", m, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (g, 1, 1), (1, 1, 1))


def test_scan_general_views():
    R, C = 300, 257
    x = synth.ints_pm1000(R * C, seed=5).reshape(R, C)
    # column scans through a transpose, one segment per column
    check_scan(x, [R, C], [("transpose", 0), ("select", V.BLOCK, V.X)], V.BLOCK, (C, 1, 1), (1, 1, 1))
    # suffix scan through reverse
    check_scan(x.reshape(-1), [R * C], [("reverse", 0)], V.GRID)
    xf = synth.uniform_grid(R * C, seed=6).reshape(R, C)
    check_scan(xf, [R, C], [("transpose", 0), ("select", V.BLOCK, V.X)], V.BLOCK, (C, 1, 1), (1, 1, 1))
    # part of the array only: untouched elements keep their value
    guard = torch.full((R * C,), -77, dtype=torch.int32)
    check_scan(x.reshape(-1), [R * C], [("split_snd", 1000, 0), ("split_fst", 5000, 0)], V.GRID, out0=guard)


def test_scan_misaligned_and_in_place():
    n = 100000
    x = synth.uniform_grid(n, seed=9)
    check_scan(x, [n], [("split_snd", 1, 0)], V.GRID)
    check_scan(x, [n], [], V.GRID, inplace=True)
    xi = synth.ints_pm1000(n, seed=9)
    check_scan(xi, [n], [("split_snd", 3, 0)], V.GRID, inplace=True)


def test_scan_hard_fp_carry():
    """2^24 ones: the running sum leaves the exact FP32 integer range, so
    only a compensated carry keeps every prefix within the tolerance."""
    n = 1 << 24
    x = torch.ones(n, dtype=torch.float32)
    x[::3] = 0.1
    check_scan(x, [n], [], V.GRID)


def test_scan_timeout_is_reported_not_hung():
    """A tile that never publishes: the waits give up, the call reports
    DESC_ERR_DEVICE_TIMEOUT, and the context stays usable."""
    n = 1 << 22
    x = dev(synth.ints_pm1000(n, seed=3))
    assert D.desc_stream_status() == 0
    D.desc_scan(x, [n], [], V.GRID, flags=D.DEBUG_STALL_TILE)
    assert D.desc_stream_status() == 9
    assert D.desc_stream_status() == 0      # read and cleared
    check_scan(x.cpu(), [n], [], V.GRID)


# ------------------------------------------------------------------ transpose
@pytest.mark.parametrize("R,C", [(1, 1), (33, 65), (1, 17), (17, 1), (64, 64), (1000, 3000), (4099, 4101)])
def test_transpose_2d(R, C):
    x = synth.normal_f32(R * C, seed=R * 7 + C).reshape(R, C)
    out = torch.zeros(C, R, dtype=torch.float32, device="cuda")
    D.desc_transpose(dev(x), [R, C], [("transpose", 0)], out, [C, R], [])
    assert torch.equal(out.cpu(), torch.from_numpy(O.transpose2d(x.numpy())))


def test_transpose_nan_payloads_and_ints():
    R, C = 129, 67
    bits = (synth.splitmix64(synth.stream_key(4), 0, R * C) & 0x7FFFFFFF).to(torch.int32).reshape(R, C)
    out = torch.zeros(C, R, dtype=torch.int32, device="cuda")
    D.desc_transpose(dev(bits), [R, C], [("transpose", 0)], out, [C, R], [])
    assert torch.equal(out.cpu(), bits.t())


def test_transpose_through_tile_views():
    """The transpose written with tile views selected by blocks and
    threads (32 x 32 tiles, 32 x 8 threads, 4 items per thread)."""
    N = 128
    x = synth.normal_f32(N * N, seed=11).reshape(N, N)
    tiles = [("group", 32, 0), ("group", 32, 2), ("transpose", 1)]           # [N/32][N/32][32][32]
    sel_b = [("select", V.BLOCK, V.Y), ("select", V.BLOCK, V.X)]
    rows = [("group", 8, 0), ("transpose", 0), ("transpose", 1),
            ("select", V.THREAD, V.Y), ("select", V.THREAD, V.X)]            # thread (x,y) item i: (y+8i, x)
    in_ops = tiles + [("transpose", 0)] + sel_b + [("transpose", 0)] + rows
    out_ops = tiles + sel_b + rows
    grid, block = (N // 32, N // 32, 1), (32, 8, 1)
    want = O.view_copy(x.numpy(), np.zeros((N, N), np.float32), [N, N], in_ops, [N, N], out_ops)
    assert np.array_equal(want, x.numpy().T)
    out = torch.zeros(N, N, dtype=torch.float32, device="cuda")
    D.desc_transpose(dev(x), [N, N], in_ops, out, [N, N], out_ops, grid, block)
    assert torch.equal(out.cpu(), torch.from_numpy(want))


def test_transpose_batched_and_general_copies():
    B, R, C = 3, 50, 70
    x = synth.normal_f32(B * R * C, seed=12).reshape(B, R, C)
    out = torch.zeros(B, C, R, device="cuda")
    D.desc_transpose(dev(x), [B, R, C], [("transpose", 1)], out, [B, C, R], [])
    assert torch.equal(out.cpu(), x.transpose(1, 2))
    # reversed rows and guard band: only part of the output is written
    guard = torch.full((R + 2, C), -5.0)
    out = dev(guard.clone())
    D.desc_transpose(dev(x[0]), [R, C], [("reverse", 0)], out, [R + 2, C], [("split_snd", 1, 0), ("split_fst", R, 0)])
    want = O.view_copy(x[0].numpy(), guard.numpy(), [R, C], [("reverse", 0)], [R + 2, C],
                       [("split_snd", 1, 0), ("split_fst", R, 0)])
    assert np.array_equal(out.cpu().numpy(), want)


# ------------------------------------------------------------------ rejected calls
def test_rejections_launch_nothing():
    n = 4096
    x = dev(synth.ints_pm1000(n, seed=1))
    host = torch.zeros(n, dtype=torch.int32)
    with pytest.raises(D.DescError) as e:                       # host pointer (Section 2.3)
        D.desc_scan(host, [n], [], V.GRID, out=dev(host))
    assert e.value.status == 4
    out = torch.full((n,), 123, dtype=torch.int32, device="cuda")
    with pytest.raises(D.DescError) as e:                       # sizes in bytes vs elements
        D.desc_scan(x, [n * 4], [], V.GRID, out=out)
    assert e.value.status == 5
    with pytest.raises(D.DescError) as e:                       # overlapping writes (narrowing)
        D.desc_scan(x, [n], [("group", 32, 0), ("select", V.THREAD, V.X)], V.GRID, (4, 1, 1), (128, 1, 1), out=out)
    assert e.value.status == 3
    with pytest.raises(D.DescError) as e:                       # in-place transpose races
        D.desc_transpose(x, [64, 64], [("transpose", 0)], x, [64, 64], [])
    assert e.value.status == 3
    with pytest.raises(D.DescError) as e:                       # workspace too small
        D.desc_scan(x, [n], [], V.GRID, out=out, ws=torch.empty(8, dtype=torch.uint8, device="cuda"))
    assert e.value.status == 10
    torch.cuda.synchronize()
    assert torch.all(out.cpu() == 123)


@pytest.mark.parametrize("m,g", [(16, 4096), (4096, 64), (8192, 37)])
def test_reversed_outer_groups(m, g):
    """Groups taken in reverse order (the kept dimension walks backwards):
    per-group reduce and segmented scan stay on the right elements."""
    n = m * g
    x = synth.ints_pm1000(n, seed=m + g)
    for ops in ([("group", m, 0), ("reverse", 0), ("select", V.BLOCK, V.X)],
                [("reverse", 0), ("group", m, 0), ("select", V.BLOCK, V.X)]):
        got = D.desc_reduce(x.cuda(), [n], ops, V.BLOCK, (g, 1, 1), (1, 1, 1)).cpu().numpy()
        want, _ = O.reduce(x.numpy(), [n], ops, V.BLOCK, (g, 1, 1), (1, 1, 1))
        assert np.array_equal(got, want)
        check_scan(x, [n], ops, V.BLOCK, (g, 1, 1), (1, 1, 1))
