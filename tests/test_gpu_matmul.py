"""GPU parity of desc_matmul against the oracle (FP64 products).

Two kinds of check per tensor-core form: against the exact FP64 product
(the stated error bounds: SPLIT3 <= 1e-5, BF16 <= 1e-2 relative Frobenius),
and against the FP64 product of the same BF16 terms (oracle's bit-level
rounding and split), which isolates the tensor-core arithmetic: only FP32
accumulation error may remain there."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2305_03448_gb300 as D
import synth
from oracle import matmul as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return desc_lib


def mats(M, N, K, seed):
    A = synth.normal_f32(M * K, seed=seed, stream=1).reshape(M, K)
    B = synth.normal_f32(K * N, seed=seed, stream=2).reshape(K, N)
    return A, B


# Tile rows (128) odd or even: even counts run as pairs of CTAs sharing B;
# (4096, 2048, 256) gives each pair of an SM pair several tiles in turn.
SHAPES = [(128, 256, 64), (256, 512, 128), (100, 300, 70), (1, 1, 1), (257, 513, 129), (384, 256, 1024),
          (1000, 700, 300), (4096, 2048, 256)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_simt_fp32(M, N, K):
    A, B = mats(M, N, K, seed=M + N + K)
    C = D.desc_matmul(A.cuda(), B.cuda(), D.MM_FP32_SIMT).cpu().numpy()
    ref = OM.matmul_f64(A.numpy(), B.numpy())
    assert OM.rel_frobenius(C, ref) <= 1e-6


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_bf16_tensor_cores(M, N, K):
    A, B = mats(M, N, K, seed=M * 3 + N + K)
    C = D.desc_matmul(A.cuda(), B.cuda(), D.MM_BF16).cpu().numpy()
    a, b = A.numpy(), B.numpy()
    emul = OM.matmul_f64(OM.bf16_rne(a), OM.bf16_rne(b))     # same BF16 inputs, exact products
    assert OM.rel_frobenius(C, emul) <= 2e-6
    assert OM.rel_frobenius(C, OM.matmul_f64(a, b)) <= 1e-2


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_split3_tensor_cores(M, N, K):
    A, B = mats(M, N, K, seed=M + N * 5 + K)
    C = D.desc_matmul(A.cuda(), B.cuda(), D.MM_SPLIT3).cpu().numpy()
    a, b = A.numpy(), B.numpy()
    assert OM.rel_frobenius(C, OM.split3_product_f64(a, b)) <= 2e-6
    assert OM.rel_frobenius(C, OM.matmul_f64(a, b)) <= 1e-5


def test_split2_between_bf16_and_split3():
    M, N, K = 256, 256, 512
    A, B = mats(M, N, K, seed=9)
    ref = OM.matmul_f64(A.numpy(), B.numpy())
    e = {p: OM.rel_frobenius(D.desc_matmul(A.cuda(), B.cuda(), p).cpu().numpy(), ref)
         for p in (D.MM_BF16, D.MM_SPLIT2, D.MM_SPLIT3)}
    assert e[D.MM_SPLIT3] < e[D.MM_SPLIT2] < e[D.MM_BF16]
    assert e[D.MM_SPLIT2] <= 1e-4


def test_closed_forms_on_tensor_cores():
    # identity: A = I gives B exactly when B holds BF16 values (one term), and
    # within the split's representation for general B
    K, N = 256, 512
    B = synth.normal_f32(K * N, seed=3).reshape(K, N)
    Bb = torch.from_numpy(OM.bf16_rne(B.numpy()))
    eye = torch.eye(K, dtype=torch.float32)
    C = D.desc_matmul(eye.cuda(), Bb.cuda(), D.MM_BF16).cpu()
    assert torch.equal(C, Bb)
    C3 = D.desc_matmul(eye.cuda(), B.cuda(), D.MM_SPLIT3).cpu().numpy()
    assert np.max(np.abs(C3 - B.numpy())) <= 2.0 ** -23 * np.max(np.abs(B.numpy()))
    ones = torch.ones(128, 300)
    C = D.desc_matmul(ones.cuda(), torch.ones(300, 256).cuda(), D.MM_BF16).cpu()
    assert torch.all(C == 300.0)


def test_transposed_operand_views():
    M, N, K = 200, 300, 160
    A, B = mats(M, N, K, seed=4)
    At = A.t().contiguous()                     # buffer holds A^T (K x M)
    ref = OM.matmul_f64(A.numpy(), B.numpy())
    for p in (D.MM_BF16, D.MM_SPLIT3):
        C = D.desc_matmul(At.cuda(), B.cuda(), p, a_view=([K, M], [("transpose", 0)]), b_view=([K, N], []),
                          M=M, N=N, K=K).cpu().numpy()
        assert OM.rel_frobenius(C, ref) <= (1e-5 if p == D.MM_SPLIT3 else 1e-2)
    with pytest.raises(D.DescError) as e:     # the CUDA-core form needs unit stride along K
        D.desc_matmul(At.cuda(), B.cuda(), D.MM_FP32_SIMT, a_view=([K, M], [("transpose", 0)]),
                      b_view=([K, N], []), M=M, N=N, K=K)
    assert e.value.status == 7


def test_rejections():
    A, B = mats(64, 64, 64, seed=5)
    with pytest.raises(D.DescError) as e:       # host pointer
        D.desc_matmul(A, B.cuda(), D.MM_BF16, out=torch.empty(64, 64, device="cuda"))
    assert e.value.status == 4
    Ad = A.cuda()
    with pytest.raises(D.DescError) as e:       # C overlapping A
        D.desc_matmul(Ad, B.cuda(), D.MM_FP32_SIMT, out=Ad)
    assert e.value.status == 3
    assert D.desc_stream_status() == 0


# The last, partial wave of pair tiles is cut along K into pieces (at least
# 24 K blocks x products each) whose partial tiles the last-arriving piece
# adds in order.  With 76 resident pairs (the cases of test_mm_plan.py):
# 16 tiles of 256 x 256 -> SPLIT3 in 4 pieces of 4 K blocks, SPLIT2 in 2;
# K = 1090 -> 18 K blocks, SPLIT3 pieces of 4, 5, 4, 5; 2560^2 on 256 x 256
# tiles (candidate 0) -> 76 whole tiles and 24 in 3 pieces (SPLIT3), on
# 256 x 512 tiles 50 whole tiles; K = 3100 -> 49 K blocks, BF16 pieces of 24
# and 25.
PIECE_SHAPES = [(1024, 1024, 1024), (1000, 1000, 1090), (2560, 2560, 1024), (1000, 1000, 3100)]


@pytest.mark.parametrize("cand", [-1, 0, 4])           # the default schedule; 256 x 256; 256 x 512
@pytest.mark.parametrize("M,N,K", PIECE_SHAPES)
def test_last_wave_pieces(M, N, K, cand):
    D.desc_force_candidate(D.OP_MATMUL, cand)
    try:
        _check_pieces(M, N, K)
    finally:
        D.desc_force_candidate(D.OP_MATMUL, -1)


def _check_pieces(M, N, K):
    A, B = mats(M, N, K, seed=M + 2 * N + K)
    a, b = A.numpy(), B.numpy()
    Ad, Bd = A.cuda(), B.cuda()
    exact = OM.matmul_f64(a, b)
    emul = OM.matmul_f64(OM.bf16_rne(a), OM.bf16_rne(b))
    split3 = OM.split3_product_f64(a, b)
    for p, ref, tol, tol_exact in ((D.MM_BF16, emul, 2e-6, 1e-2), (D.MM_SPLIT3, split3, 2e-6, 1e-5),
                                   (D.MM_SPLIT2, None, None, 1e-4)):
        nb = ctypes.c_size_t(0)
        assert D.lib().desc_matmul_workspace_size(M, N, K, p, ctypes.byref(nb)) == 0
        ws = torch.full((nb.value,), 0xFF, dtype=torch.uint8, device="cuda")   # stale counters
        C1 = D.desc_matmul(Ad, Bd, p, ws=ws)
        C2 = D.desc_matmul(Ad, Bd, p, ws=ws)
        assert torch.equal(C1, C2)                  # independent of which piece finishes last
        c = C1.cpu().numpy()
        if ref is not None:
            assert OM.rel_frobenius(c, ref) <= tol
        assert OM.rel_frobenius(c, exact) <= tol_exact
    assert D.desc_stream_status() == 0


@pytest.mark.parametrize("M,N,K,p", [(1024, 1024, 1024, D.MM_SPLIT3), (1000, 1000, 3100, D.MM_BF16),
                                     (384, 520, 300, D.MM_SPLIT3)])
def test_matmul_captured_in_cuda_graph(M, N, K, p):
    """The tensor-core call issues kernel launches only (split passes, the
    counters cleared by the A pass, the GEMM with its last-wave pieces), so it
    replays from a CUDA graph with the same bits as the direct call."""
    A, B = mats(M, N, K, seed=M + N + K + 11)
    Ad, Bd = A.cuda(), B.cuda()
    nb = ctypes.c_size_t(0)
    assert D.lib().desc_matmul_workspace_size(M, N, K, p, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    ref = D.desc_matmul(Ad, Bd, p, ws=ws)              # direct call (also the first call on the device)
    C = torch.full_like(ref, float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        D.desc_matmul(Ad, Bd, p, out=C, ws=ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, ref)
    C.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, ref)
    assert D.desc_stream_status() == 0


@pytest.mark.parametrize("M", [640, 768])              # odd / even 128-row tile counts: single CTAs / pairs
@pytest.mark.parametrize("p", [D.MM_BF16, D.MM_SPLIT3])
def test_operands_and_output_off_16_byte_alignment(p, M):
    """A, B and C each start one float past a 16-byte boundary: the split
    passes take the general kernel and C cannot be stored by TMA, so the
    epilogue stores from registers."""
    N, K = 768, 320
    A, B = mats(M, N, K, seed=31)
    bufA = torch.zeros(M * K + 1, device="cuda")
    bufB = torch.zeros(K * N + 1, device="cuda")
    bufC = torch.full((M * N + 1,), float("nan"), device="cuda")
    Ad, Bd, Cd = bufA[1:].view(M, K), bufB[1:].view(K, N), bufC[1:].view(M, N)
    Ad.copy_(A.cuda())
    Bd.copy_(B.cuda())
    assert Ad.data_ptr() % 16 == 4 and Cd.data_ptr() % 16 == 4
    D.desc_matmul(Ad, Bd, p, out=Cd)
    ref = D.desc_matmul(A.cuda(), B.cuda(), p).cpu()
    assert torch.equal(Cd.cpu(), ref)                   # same terms, same products, same order
    assert torch.isnan(bufC[0].cpu())                   # nothing written before C
    a, b = A.numpy(), B.numpy()
    assert OM.rel_frobenius(Cd.cpu().numpy(), OM.matmul_f64(a, b)) <= (1e-5 if p == D.MM_SPLIT3 else 1e-2)


# K of one and two K blocks (no second phase / halves of one block); N = 256:
# the second MMA of each 512-wide tile reads only zero padding.
@pytest.mark.parametrize("M,N,K", [(512, 1024, 320), (768, 1280, 256), (1000, 700, 200), (512, 512, 64),
                                   (512, 768, 100), (512, 256, 128)])
def test_wide_pair_tiles_give_the_same_bits(M, N, K):
    """256 x 512 pair tiles (two N256 MMAs per K step, one accumulator set)
    against 256 x 256 tiles: the split forms run each tile's K range in two
    phases (first halves of every product, then second halves), so every sum
    adds the same products in the same order -- bit-identical results.  K is
    too short here for the last wave's pieces, which depend on the tile count."""
    A, B = mats(M, N, K, seed=M + N + 3 * K)
    Ad, Bd = A.cuda(), B.cuda()
    for p in (D.MM_BF16, D.MM_SPLIT2, D.MM_SPLIT3):
        out = {}
        for cand in (0, 4, 2, 5):
            D.desc_force_candidate(D.OP_MATMUL, cand)
            try:
                out[cand] = D.desc_matmul(Ad, Bd, p).cpu()
            finally:
                D.desc_force_candidate(D.OP_MATMUL, -1)
        assert torch.equal(out[0], out[4]) and torch.equal(out[2], out[5]) and torch.equal(out[0], out[2]), p
    assert D.desc_stream_status() == 0


@pytest.mark.parametrize("M,N,K", [(896, 768, 320), (1152, 640, 200), (128, 512, 256), (1000, 520, 64)])
def test_odd_tile_rows_padded_to_pairs(M, N, K):
    """An odd count of 128-row tiles is padded with a zero tile row so that CTA
    pairs take it (split forms always, BF16 from nine tile rows): same bits as
    the single-CTA kernel, no row of C past M written.  K is too short here
    for the last wave's pieces."""
    A, B = mats(M, N, K, seed=M + 5 * N + K)
    Ad, Bd = A.cuda(), B.cuda()
    for p in (D.MM_BF16, D.MM_SPLIT2, D.MM_SPLIT3):
        buf = torch.full(((M + 1) * N,), float("nan"), device="cuda")
        C = buf[:M * N].view(M, N)
        D.desc_matmul(Ad, Bd, p, out=C)
        assert torch.isnan(buf[M * N:]).all()              # the row after C untouched
        D.desc_force_candidate(D.OP_MATMUL, 1)             # single CTAs, no padding
        try:
            ref = D.desc_matmul(Ad, Bd, p)
        finally:
            D.desc_force_candidate(D.OP_MATMUL, -1)
        assert torch.equal(C, ref), p
    assert D.desc_stream_status() == 0


def test_simt_fp32_wide_tiles_sampled_rows():
    """Enough 128 x 256 tiles for eight waves (152 SMs): the CUDA-core form
    takes its 8 x 16-outputs-per-thread kernel; sampled rows against FP64."""
    M, N, K = 4864, 8192, 96
    A, B = mats(M, N, K, seed=77)
    C = D.desc_matmul(A.cuda(), B.cuda(), D.MM_FP32_SIMT).cpu().numpy()
    rows = np.array([0, 1, 127, 128, 2437, 4800, 4863])
    ref = OM.matmul_f64(A.numpy()[rows], B.numpy())
    assert OM.rel_frobenius(C[rows], ref) <= 1e-6
    assert np.isfinite(C).all()
