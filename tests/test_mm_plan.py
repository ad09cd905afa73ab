"""The matmul schedule decided on the host (desc_matmul_plan): CTA pairs or
single CTAs, 256- or 512-column pair tiles, padding of an odd count of
128-row tiles, and the last wave's K pieces.  Pure host logic, run with an
explicit number of resident CTA pairs (76 on a GB300)."""
import itertools

import pytest
import torch

import paper_2305_03448_gb300 as D

PAIRS = 76


@pytest.fixture(scope="module", autouse=True)
def _lib(desc_lib):
    return desc_lib


def plan(M, N, K, p, cand=-1, pairs=PAIRS):
    return D.desc_matmul_plan(M, N, K, p, candidate=cand, max_pairs=pairs)


def nprod(p):
    return {D.MM_BF16: 1, D.MM_SPLIT2: 3, D.MM_SPLIT3: 6}[p]


@pytest.mark.parametrize("M,N,K,p,expect", [
    # large squares: 256 x 512 pair tiles, 32 x 16 of them, no pieces (76 / 56 < 2)
    (8192, 8192, 8192, D.MM_SPLIT3, dict(candidate=4, pairs=1, tile_n=512, padded=0, tiles=512, pieces=1)),
    (8192, 8192, 8192, D.MM_BF16, dict(candidate=4, pairs=1, tile_n=512, tiles=512, pieces=1)),
    # 2048^3, 32 wide tiles: one product keeps 256 x 256 tiles, the split forms take the wide ones in 2 pieces
    (2048, 2048, 2048, D.MM_BF16, dict(candidate=0, tile_n=256, tiles=64, whole_tiles=64, pieces=1)),
    (2048, 2048, 2048, D.MM_SPLIT3, dict(candidate=4, tile_n=512, tiles=32, whole_tiles=0, pieces=2)),
    # 16 tiles of 256 x 256: four K pieces each
    (1024, 1024, 1024, D.MM_SPLIT3, dict(candidate=0, tile_n=256, tiles=16, whole_tiles=0, pieces=4)),
    # 63 tile rows padded to 64 for the split forms and for one product (>= 9 rows)
    (8064, 8192, 8192, D.MM_SPLIT3, dict(pairs=1, padded=1, rows=8192, tile_n=512, tiles=512)),
    (8064, 8192, 8192, D.MM_BF16, dict(pairs=1, padded=1, rows=8192)),
    # 5 tile rows: one product stays on single CTAs, the split forms pad and take 24 wide tiles in 3 pieces
    (640, 4096, 4096, D.MM_BF16, dict(pairs=0, padded=0, rows=640, tile_n=256, tiles=80, pieces=1)),
    (640, 4096, 4096, D.MM_SPLIT3, dict(pairs=1, padded=1, rows=768, tile_n=512, tiles=24, whole_tiles=0,
                                        pieces=3)),
    # ragged M: 1000 rows round up to 8 tile rows, already even
    (1000, 1000, 3100, D.MM_BF16, dict(pairs=1, padded=0, rows=1024, tile_n=256, tiles=16, pieces=2)),
])
def test_size_rule(M, N, K, p, expect):
    got = plan(M, N, K, p)
    assert got["max_pairs"] == PAIRS
    for key, value in expect.items():
        assert got[key] == value, (key, got)


def test_forced_candidates():
    # 2560^2 x 1024 on 256 x 256 tiles: 100 tiles, 76 whole, 24 in 3 pieces
    g = plan(2560, 2560, 1024, D.MM_SPLIT3, cand=0)
    assert (g["tile_n"], g["tiles"], g["whole_tiles"], g["pieces"]) == (256, 100, 76, 3)
    g = plan(2560, 2560, 1024, D.MM_SPLIT3, cand=4)                 # 50 wide tiles fit one wave
    assert (g["tile_n"], g["tiles"], g["whole_tiles"], g["pieces"]) == (512, 50, 50, 1)
    for cand in (1, 3):                                              # single CTAs: never padded, no pieces
        g = plan(8064, 8192, 8192, D.MM_SPLIT3, cand=cand)
        assert (g["pairs"], g["padded"], g["rows"], g["tile_n"], g["pieces"]) == (0, 0, 8064, 256, 1)
        assert g["tiles"] == 63 * 32
    g = plan(640, 4096, 4096, D.MM_BF16, cand=4)                     # 5 rows, one product: not padded
    assert (g["pairs"], g["padded"], g["tile_n"]) == (0, 0, 256)
    assert plan(4096, 4096, 4096, D.MM_BF16, cand=2)["candidate"] == 2


def test_one_resident_pair():
    g = plan(4096, 4096, 4096, D.MM_SPLIT3, pairs=1)                 # still pairs and wide tiles, no pieces
    assert g["pairs"] == 1 and g["pieces"] == 1


@pytest.mark.parametrize("p", [D.MM_BF16, D.MM_SPLIT2, D.MM_SPLIT3])
def test_pieces_invariants(p):
    """Over many shapes: pieces only on pair tiles, at most four, at most one
    piece unit per resident pair, only for the partial last wave, and each
    piece holds at least 24 K blocks x products."""
    for m, n, k in itertools.product([128, 384, 1000, 1536, 2560, 4096], [256, 700, 2048, 5000],
                                     [64, 320, 1024, 4096]):
        g = plan(m, n, k, p)
        tail = g["tiles"] - g["whole_tiles"]
        r128 = -(-m // 128) * 128                                   # M in whole 128-row tiles
        assert g["rows"] == (r128 + 128 if g["padded"] else r128)
        assert not g["padded"] or (r128 // 128) % 2 == 1
        tile_m = 256 if g["pairs"] else 128
        assert g["rows"] % tile_m == 0
        assert g["tiles"] == (g["rows"] // tile_m) * -(-(-(-n // 256) * 256) // g["tile_n"])
        if g["pieces"] == 1:
            assert tail == 0
            continue
        assert g["pairs"] == 1 and 2 <= g["pieces"] <= 4
        assert tail == g["tiles"] % PAIRS and tail * g["pieces"] <= PAIRS
        assert ((k + 63) // 64) * nprod(p) // g["pieces"] >= 24


def test_rejections():
    with pytest.raises(D.DescError) as e:
        plan(64, 64, 64, D.MM_FP32_SIMT)                             # not a tensor-core form
    assert e.value.status == 1
    for bad in [dict(M=0), dict(K=-1), dict(cand=6), dict(cand=-2), dict(pairs=-1)]:
        a = dict(M=64, N=64, K=64, p=D.MM_BF16, cand=-1, pairs=PAIRS)
        a.update(bad)
        with pytest.raises(D.DescError) as e:
            plan(a["M"], a["N"], a["K"], a["p"], a["cand"], a["pairs"])
        assert e.value.status == 1
    if not torch.cuda.is_available():
        with pytest.raises(D.DescError) as e:                        # 0 asks the device: there is none
            D.desc_matmul_plan(64, 64, 64, D.MM_BF16)
        assert e.value.status == 8
