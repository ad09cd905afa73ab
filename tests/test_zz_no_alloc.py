"""desc_scan_noalloc: the scan for callers that may not allocate device
memory when they call (a plugin whose host framework owns every device
allocation, an allocator or out-of-memory callback, a real-time loop that
allocates nothing after start-up).  It uses the library's static scratch
array instead of a caller-provided workspace.

Checked here through the C ABI: on two calls in a row its output matches
desc_scan's (bit for bit for int32, within 1e-5 * sum_{q<=p} |x_q| for
FP32) and the CPU oracle's; a view whose scan is not one contiguous run is
refused, and so is a scan longer than the static scratch allows, both
without touching the output.  This file is collected last on purpose."""
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


def _compare(x, got, want):
    if x.dtype == torch.int32:
        assert torch.equal(got.cpu(), want.cpu())
    else:
        pabs = torch.cumsum(x.double().abs(), 0).cpu().numpy()
        err = np.abs(got.double().cpu().numpy() - want.double().cpu().numpy())
        assert np.all(err <= TOL * pabs + 1e-30), err.max()


@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_noalloc_matches_desc_scan_twice(dt):
    for call, n in enumerate([(1 << 20) + 13, 3 * 4096 + 1]):
        gen = synth.ints_pm1000 if dt == "i32" else synth.uniform_grid
        x = gen(n, seed=100 + call).cuda()
        want = D.desc_scan(x, [n], [], D.GRID)
        got = torch.full_like(x, 7)
        D.desc_scan_noalloc(x, [n], [], D.GRID, out=got)
        assert D.desc_stream_status() == 0
        _compare(x, got, want)
        # and against the oracle: int32 bit for bit, FP32 within 1e-5 * sum |x| of each prefix
        xo = x.cpu().numpy()
        ref, pa = O.scan(xo, np.zeros(n, xo.dtype), [n], [], D.GRID)
        if dt == "i32":
            assert np.array_equal(got.cpu().numpy(), ref)
        else:
            assert np.all(np.abs(got.cpu().numpy().astype(np.float64) - ref) <= TOL * pa + 1e-30)


def test_noalloc_segments_and_split_views():
    m, g = 1000, 300
    n = m * g
    x = synth.uniform_grid(n, seed=7).cuda()
    ops = [("group", m, 0), ("select", D.BLOCK, D.X)]
    pabs = torch.cumsum(x.double().abs().reshape(g, m), 1).reshape(-1).cpu().numpy()
    for _ in range(2):
        want = D.desc_scan(x, [n], ops, D.BLOCK, (g, 1, 1), (1, 1, 1))
        got = D.desc_scan_noalloc(x, [n], ops, D.BLOCK, (g, 1, 1), (1, 1, 1))
        err = np.abs(got.double().cpu().numpy() - want.double().cpu().numpy())
        assert np.all(err <= TOL * pabs + 1e-30), err.max()
    xi = synth.ints_pm1000(n, seed=8).cuda()
    ops = [("split_snd", 3, 0), ("split_fst", n - 10, 0)]
    want = D.desc_scan(xi, [n], ops, D.GRID, out=torch.zeros_like(xi))
    got = D.desc_scan_noalloc(xi, [n], ops, D.GRID, out=torch.zeros_like(xi))
    assert torch.equal(got.cpu(), want.cpu())


def test_noalloc_refuses_views_that_are_not_one_run():
    n = 5000
    x = synth.ints_pm1000(n, seed=9).cuda()
    for ops in ([("reverse", 0)], [("group", 50, 0), ("transpose", 0)]):
        out = torch.full((n,), 5, dtype=torch.int32, device="cuda")
        with pytest.raises(D.DescError) as e:
            D.desc_scan_noalloc(x, [n], ops, D.GRID, out=out)
        assert e.value.status == 7                       # DESC_ERR_UNSUPPORTED
        torch.cuda.synchronize()
        assert torch.equal(out.cpu(), torch.full((n,), 5, dtype=torch.int32))


def test_noalloc_refuses_more_than_its_scratch():
    n = (1 << 28) + 4096
    x = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.full((n,), 5, dtype=torch.int32, device="cuda")
    with pytest.raises(D.DescError) as e:
        D.desc_scan_noalloc(x, [n], [], D.GRID, out=out)
    assert e.value.status == 10
    torch.cuda.synchronize()
    assert int(out[0]) == 5 and int(out[-1]) == 5
    del x, out
    torch.cuda.empty_cache()
