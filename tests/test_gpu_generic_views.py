"""The general path (desc_force_generic): reduce, scan and transpose evaluate
their lowered affine maps element by element instead of running the
hand-indexed kernels, with the same results against the oracle.  This is
the other arm of Section 5's view-overhead comparison."""
import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import ops as O
from oracle import views as V

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(autouse=True)
def _generic(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    D.desc_force_generic(True)
    yield
    D.desc_force_generic(False)


RED_VIEWS = [
    ([1 << 20], [], V.GRID, None, None),
    ([1 << 20], [("group", 1024, 0), ("select", V.BLOCK, V.X), ("group", 32, 0), ("select", V.WARP, V.X),
                 ("select", V.THREAD, V.X)], V.GRID, (1024, 1, 1), (1024, 1, 1)),
    ([1 << 20], [("group", 1024, 0), ("select", V.BLOCK, V.X)], V.BLOCK, (1024, 1, 1), (1, 1, 1)),
    ([300 * 257], [("reverse", 0)], V.GRID, None, None),
]


@pytest.mark.parametrize("case", range(len(RED_VIEWS)))
def test_reduce_generic(case):
    base, ops, lvl, grid, block = RED_VIEWS[case]
    n = base[0]
    x = synth.ints_pm1000(n, seed=case + 1)
    got = D.desc_reduce(x.cuda(), base, ops, lvl, grid, block).cpu().numpy()
    want, _ = O.reduce(x.numpy(), base, ops, lvl, grid, block)
    assert np.array_equal(got, want)
    xf = synth.uniform_grid(n, seed=case + 11)
    gotf = D.desc_reduce(xf.cuda(), base, ops, lvl, grid, block).cpu().numpy().astype(np.float64)
    wantf, sabs = O.reduce(xf.numpy(), base, ops, lvl, grid, block)
    assert np.all(np.abs(gotf - wantf) <= TOL * sabs + 1e-30)


@pytest.mark.parametrize("n", [1, 4097, (1 << 20) + 3])
def test_scan_generic(n):
    for x in (synth.ints_pm1000(n, seed=n), synth.uniform_grid(n, seed=n + 1)):
        out = torch.zeros_like(x).cuda()
        got = D.desc_scan(x.cuda(), [n], [], V.GRID, out=out).cpu().numpy()
        want, pabs = O.scan(x.numpy(), np.zeros_like(x.numpy()), [n], [], V.GRID)
        if x.dtype == torch.int32:
            assert np.array_equal(got, want)
        else:
            assert np.all(np.abs(got.astype(np.float64) - want) <= TOL * pabs + 1e-30)


def test_scan_generic_segments():
    m, g = 5000, 60
    x = synth.uniform_grid(m * g, seed=3)
    ops = [("group", m, 0), ("select", V.BLOCK, V.X)]
    got = D.desc_scan(x.cuda(), [m * g], ops, V.BLOCK, (g, 1, 1), (1, 1, 1)).cpu().numpy()
    want, pabs = O.scan(x.numpy(), np.zeros(m * g, np.float32), [m * g], ops, V.BLOCK, (g, 1, 1), (1, 1, 1))
    assert np.all(np.abs(got.astype(np.float64) - want) <= TOL * pabs + 1e-30)


@pytest.mark.parametrize("R,C", [(1, 1), (33, 65), (1000, 3000), (4096, 2048)])
def test_transpose_generic(R, C):
    x = synth.normal_f32(R * C, seed=R + C).reshape(R, C)
    out = torch.empty(C, R, device="cuda")
    D.desc_transpose(x.cuda(), [R, C], [("transpose", 0)], out, [C, R], [])
    assert np.array_equal(out.cpu().numpy().view(np.int32), O.transpose2d(x.numpy()).view(np.int32))


def test_switch_is_per_thread_and_restored():
    """The specialised path is back once the switch is off: same results."""
    n = 1 << 18
    x = synth.ints_pm1000(n, seed=5).cuda()
    a = D.desc_reduce(x, [n], [], V.GRID).cpu()
    D.desc_force_generic(False)
    b = D.desc_reduce(x, [n], [], V.GRID).cpu()
    assert torch.equal(a, b)


@pytest.mark.parametrize("shape", [(5, 7, 9), (3, 1, 4097), (37, 41, 43)])
def test_copy_generic_3d_permutation(shape):
    """Odd extents exercise the 32-bit invariant division of the decoder."""
    A, B, C = shape
    x = synth.normal_f32(A * B * C, seed=A + B + C).reshape(A, B, C)
    out = torch.empty(A, C, B, device="cuda")
    D.desc_transpose(x.cuda(), [A, B, C], [("transpose", 1)], out, [A, C, B], [])
    want = np.ascontiguousarray(x.numpy().transpose(0, 2, 1))
    assert np.array_equal(out.cpu().numpy().view(np.int32), want.view(np.int32))


@pytest.mark.parametrize("m,g", [(3, 1001), (7, 4099), (1000, 3)])
def test_reduce_generic_odd_groups_reversed(m, g):
    n = m * g
    x = synth.ints_pm1000(n, seed=m)
    ops = [("reverse", 0), ("group", m, 0), ("select", V.BLOCK, V.X)]
    got = D.desc_reduce(x.cuda(), [n], ops, V.BLOCK, (g, 1, 1), (1, 1, 1)).cpu().numpy()
    want, _ = O.reduce(x.numpy(), [n], ops, V.BLOCK, (g, 1, 1), (1, 1, 1))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape,in_ops,perm", [
    ((6, 40, 5, 48), [("transpose", 0), ("transpose", 2)], (1, 0, 3, 2)),    # two batch dims, tiled
    ((70000, 16, 16), [("transpose", 1)], (0, 2, 1)),                       # batch above the grid's z limit
    ((17, 33, 70), [("transpose", 0), ("transpose", 1)], (1, 2, 0)),        # a rotation of the dims
    ((64, 96), [("reverse", 1), ("transpose", 0)], None),                    # reversed rows: element path
])
def test_copy_generic_tiled_and_batched(shape, in_ops, perm):
    """General copies through the tiled path (the input's and the output's
    unit-stride dims tiled through shared memory, the other dims decoded per
    CTA) and through the element path, bit-exact against the oracle."""
    n = int(np.prod(shape))
    x = synth.normal_f32(n, seed=n % 1000).reshape(shape)
    dom = V.domain_shape(list(shape), in_ops)
    out = torch.zeros(*dom, device="cuda")
    D.desc_transpose(x.cuda(), list(shape), in_ops, out, dom, [])
    want = O.view_copy(x.numpy(), np.zeros(dom, np.float32), list(shape), in_ops, dom, [])
    assert np.array_equal(out.cpu().numpy().view(np.int32), want.astype(np.float32).view(np.int32))
    if perm is not None:
        assert np.array_equal(out.cpu().numpy(), np.ascontiguousarray(x.numpy().transpose(perm)))
