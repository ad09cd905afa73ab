"""Every scan schedule, forced, against the oracle: tiles of 4096 x 4,
x 2 and x 1 elements, each scanned by one CTA and chained by decoupled
look-back (Section 5's grid-level scan).  Sizes put the ragged tail at
every sub-tile boundary of a tile, periods cross tile boundaries, and CSR
segments include empty ones."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu
TOL = 1e-5
PART = 4 * 4096          # elements per tile of the largest schedule


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield desc_lib
    D.desc_force_candidate(D.OP_SCAN, -1)
    D.desc_force_candidate(D.OP_SEGMENTED, -1)


def _check(x, base, ops, lvl, grid=None, block=None, inplace=False):
    xd = x.cuda()
    out = xd if inplace else torch.zeros_like(xd)
    got = D.desc_scan(xd, base, ops, lvl, grid, block, out=out).cpu().numpy()
    want, pabs = O.scan(x.numpy(), x.numpy() if inplace else np.zeros_like(x.numpy()), base, ops, lvl, grid, block)
    if x.dtype == torch.int32:
        assert np.array_equal(got, want)
    else:
        assert np.all(np.abs(got.astype(np.float64) - want) <= TOL * pabs + 1e-30)


CANDS = range(3)
SIZES = [1, 4097, PART - 1, PART + 1, 2 * PART + 3, 3 * PART, 4 * PART + 1, 9 * PART + 77, (1 << 22) + 5]


@pytest.mark.parametrize("cand", CANDS)
@pytest.mark.parametrize("n", SIZES)
def test_plain(cand, n):
    assert D.candidate_count(D.OP_SCAN) == len(CANDS)
    D.desc_force_candidate(D.OP_SCAN, cand)
    _check(synth.ints_pm1000(n, seed=n), [n], [], V.GRID)
    _check(synth.uniform_grid(n, seed=n + 1), [n], [], V.GRID)


@pytest.mark.parametrize("cand", CANDS)
@pytest.mark.parametrize("m", [7, 4096, 5000, PART, 3 * PART + 1, 70000])
def test_periodic(cand, m):
    D.desc_force_candidate(D.OP_SCAN, cand)
    g = max(1, 600000 // m)
    n = g * m
    for x in (synth.ints_pm1000(n, seed=m), synth.uniform_grid(n, seed=m)):
        _check(x, [n], [("group", m, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (g, 1, 1), (1, 1, 1))


@pytest.mark.parametrize("cand", CANDS)
def test_misaligned_in_place_and_hard_carry(cand):
    D.desc_force_candidate(D.OP_SCAN, cand)
    n = 200003
    _check(synth.uniform_grid(n, seed=9), [n], [("split_snd", 1, 0)], V.GRID)
    _check(synth.ints_pm1000(n, seed=9), [n], [("split_snd", 3, 0)], V.GRID, inplace=True)
    x = torch.ones(1 << 24, dtype=torch.float32)
    x[::3] = 0.1
    _check(x, [1 << 24], [], V.GRID)


@pytest.mark.parametrize("cand", CANDS)
@pytest.mark.parametrize("maxlen", [3, 2000, 100000])
def test_segmented_csr(cand, maxlen):
    D.desc_force_candidate(D.OP_SEGMENTED, cand)
    L = synth.loguniform_lengths(700, seed=maxlen, max_len=maxlen)
    L[::11] = 0                                   # empty segments
    off = synth.offsets_from_lengths(L)
    for x in (synth.ints_pm1000(int(off[-1]), seed=3), synth.uniform_grid(int(off[-1]), seed=4)):
        s, sums = D.desc_segmented_reduce_scan(x.cuda(), off.cuda())
        want, wsum, pa, sa = O.segmented_reduce_scan(x.numpy(), off.numpy())
        if x.dtype == torch.int32:
            assert np.array_equal(s.cpu().numpy(), want) and np.array_equal(sums.cpu().numpy(), wsum)
        else:
            assert np.all(np.abs(s.cpu().numpy().astype(np.float64) - want) <= TOL * pa + 1e-30)
            assert np.all(np.abs(sums.cpu().numpy().astype(np.float64) - wsum) <= TOL * sa + 1e-30)


@pytest.mark.parametrize("cand", CANDS)
def test_timeout_is_reported_not_hung(cand):
    """A tile that never publishes: the look-backs behind it give up, and the
    call reports DESC_ERR_DEVICE_TIMEOUT with the context usable."""
    D.desc_force_candidate(D.OP_SCAN, cand)
    n = 1 << 22
    x = synth.ints_pm1000(n, seed=3).cuda()
    assert D.desc_stream_status() == 0
    D.desc_scan(x, [n], [], V.GRID, flags=D.DEBUG_STALL_TILE)
    assert D.desc_stream_status() == 9
    assert D.desc_stream_status() == 0
    _check(x.cpu(), [n], [], V.GRID)
