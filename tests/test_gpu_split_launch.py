"""One launch, two ops (desc_split_reduce_transpose): the first blocks
reduce, the others transpose (Section 3.3's split of an execution resource
running different code).  Results against the oracle and against the two
separate calls."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield desc_lib
    D.desc_force_candidate(D.OP_REDUCE, -1)


CASES = [
    ((1 << 20) + 5, [], V.GRID, None, None, (1000, 3000)),
    (64 * 8192, [("group", 8192, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (64, 1, 1), (1, 1, 1), (257, 129)),
    (37 * 5000, [("reverse", 0), ("group", 5000, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (37, 1, 1), (1, 1, 1),
     (64, 64)),
    (1 << 16, [], V.GRID, None, None, (1, 1)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_split_launch_matches_oracle_and_separate_calls(case):
    n, ops, lvl, g, b, (R, C) = CASES[case]
    D.desc_force_candidate(D.OP_REDUCE, 0)          # the split launch runs the default reduce schedule
    for x in (synth.ints_pm1000(n, seed=n), synth.uniform_grid(n, seed=n + 1)):
        t = synth.normal_f32(R * C, seed=R + C).reshape(R, C)
        tout = torch.empty(C, R, device="cuda")
        got = D.desc_split_reduce_transpose(x.cuda(), [n], ops, lvl, g, b, t.cuda(), tout).cpu()
        assert np.array_equal(tout.cpu().numpy().view(np.int32), O.transpose2d(t.numpy()).view(np.int32))
        want, sabs = O.reduce(x.numpy(), [n], ops, lvl, g, b)
        if x.dtype == torch.int32:
            assert np.array_equal(got.numpy(), want)
        else:
            assert np.all(np.abs(got.numpy().astype(np.float64) - want) <= 1e-5 * sabs + 1e-30)
        sep = D.desc_reduce(x.cuda(), [n], ops, lvl, g, b).cpu()
        assert torch.equal(got.view(torch.int32), sep.view(torch.int32))   # same bits as the separate call
    D.desc_force_candidate(D.OP_REDUCE, -1)


def test_split_launch_rejections():
    x = synth.ints_pm1000(1 << 20, seed=1).cuda()
    t = torch.zeros(64, 64, device="cuda")
    with pytest.raises(D.DescError) as e:           # the transpose writes over its input
        D.desc_split_reduce_transpose(x, [1 << 20], [], V.GRID, None, None, t, t)
    assert e.value.status == 3
    with pytest.raises(D.DescError) as e:           # short runs: not the chunked schedule
        D.desc_split_reduce_transpose(x, [1 << 20], [("group", 16, 0), ("select", V.BLOCK, V.X)], V.BLOCK,
                                      ((1 << 20) // 16, 1, 1), (1, 1, 1), t, torch.zeros(64, 64, device="cuda"))
    assert e.value.status == 7
