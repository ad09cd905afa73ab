"""Oracle of the kernel-body checker, pinned to the paper's examples and to
cases whose verdict follows directly from the rules (Section 2.2
"Synchronization", Section 3.3 "Narrowing" / "Synchronization", Section 4
access_safety_check).  Statuses: 0 safe, 2 shape, 3 conflict, 11 barrier."""
from oracle import program as P
from oracle.views import BLOCK, GRID, THREAD, WARP, X, Y

W, R = True, False


def thr(n):            # arr[[thread]] on an n-element array
    return [("select", THREAD, X)]


def test_section_2_2_barrier_inside_split_block():
    # split(X) block at 32 { first_32_threads => { sync } } with 64 threads: rejected
    prog = [("split", THREAD, X, 32, [("sync", BLOCK)], [])]
    assert P.check_program(prog, (1, 1, 1), (64, 1, 1)) == (11, 1, None)
    # the same barrier outside the split is reached by every thread
    assert P.check_program([("sync", BLOCK)], (1, 1, 1), (64, 1, 1)) == (0, -1, None)


def test_section_2_2_conflicting_reverse_selection():
    # arr[[thread]] = arr.rev[[thread]]: thread t writes element t and reads n-1-t
    n = 64
    prog = [("access", 0, [n], [("reverse", 0), ("select", THREAD, X)], R),
            ("access", 0, [n], thr(n), W)]
    st, idx, e = P.check_program(prog, (1, 1, 1), (n, 1, 1))
    assert (st, idx, e) == (3, 1, 0)


def test_section_3_3_narrowing_examples():
    g, b = (32, 1, 1), (32, 1, 1)
    n = 1024
    # a block writing the whole array after the blocks were scheduled
    assert P.check_program([("access", 0, [n], [], W)], g, b)[0] == 3
    # arr.group<32>[[thread]] without a block selection: every block's threads share
    assert P.check_program([("access", 0, [n], [("group", 32, 0), ("select", THREAD, X)], W)], g, b)[0] == 3
    # arr.group<32>[[block]][[thread]]: correct narrowing
    ok = [("access", 0, [n], [("group", 32, 0), ("select", BLOCK, X), ("select", THREAD, X)], W)]
    assert P.check_program(ok, g, b) == (0, -1, None)


def test_section_3_3_barrier_releases_shared_memory_exchange():
    # write tmp[[thread]], sync, read tmp.rev[[thread]]: safe only with the barrier
    n = 128
    w = ("access", 7, [n], thr(n), W)
    r = ("access", 7, [n], [("reverse", 0), ("select", THREAD, X)], R)
    assert P.check_program([w, ("sync", BLOCK), r], (1, 1, 1), (n, 1, 1)) == (0, -1, None)
    assert P.check_program([w, r], (1, 1, 1), (n, 1, 1)) == (3, 1, 0)
    # another buffer never conflicts
    r2 = ("access", 8, [n], [("reverse", 0), ("select", THREAD, X)], R)
    assert P.check_program([w, r2], (1, 1, 1), (n, 1, 1)) == (0, -1, None)


def test_block_barrier_does_not_order_blocks_grid_boundary_does():
    n, g, b = 64, (2, 1, 1), (32, 1, 1)
    wv = ("access", 0, [n], [("group", 32, 0), ("select", BLOCK, X), ("select", THREAD, X)], W)
    # every thread then reads element (t + 32) mod 64: the other block's data
    rv = ("access", 0, [n], [("group", 32, 0), ("reverse", 0), ("select", BLOCK, X), ("select", THREAD, X)], R)
    assert P.check_program([wv, ("sync", BLOCK), rv], g, b)[0] == 3
    assert P.check_program([wv, ("sync", GRID), rv], g, b) == (0, -1, None)


def test_block_split_parts_and_barriers():
    g, b = (4, 1, 1), (32, 1, 1)
    # blocks 0-1 write the first 64 elements, blocks 2-3 the last 64: disjoint
    first = [("access", 0, [128], [("split_fst", 64, 0), ("group", 32, 0), ("select", BLOCK, X),
                                   ("select", THREAD, X)], W), ("sync", BLOCK)]
    second = [("access", 0, [128], [("split_snd", 64, 0), ("group", 32, 0), ("select", BLOCK, X),
                                    ("select", THREAD, X)], W)]
    assert P.check_program([("split", BLOCK, X, 2, first, second)], g, b) == (0, -1, None)
    # both parts on the same half: the second part's write conflicts
    second_bad = [("access", 0, [128], [("split_fst", 64, 0), ("group", 32, 0), ("select", BLOCK, X),
                                        ("select", THREAD, X)], W)]
    assert P.check_program([("split", BLOCK, X, 2, first, second_bad)], g, b) == (3, 3, 0)
    # a kernel boundary inside a split is rejected
    assert P.check_program([("split", BLOCK, X, 2, [("sync", GRID)], [])], g, b) == (11, 1, None)


def test_warp_barriers():
    b = (128, 1, 1)
    lanes = [("group", 32, 0), ("select", WARP, X), ("select", THREAD, X)]
    lanes_rev = [("group", 32, 0), ("select", WARP, X), ("reverse", 0), ("select", THREAD, X)]
    w = ("access", 0, [128], lanes, W)
    r_same_warp = ("access", 0, [128], lanes_rev, R)
    assert P.check_program([w, ("sync", WARP), r_same_warp], (1, 1, 1), b) == (0, -1, None)
    assert P.check_program([w, r_same_warp], (1, 1, 1), b)[0] == 3
    # a warp barrier does not order different warps: read the next warp's data
    r_other_warp = ("access", 0, [128], [("group", 32, 0), ("reverse", 0), ("select", WARP, X),
                                         ("select", THREAD, X)], R)
    assert P.check_program([w, ("sync", WARP), r_other_warp], (1, 1, 1), b)[0] == 3
    # a warp barrier inside a split of the threads, and a block barrier inside a split of the warps
    assert P.check_program([("split", THREAD, X, 16, [("sync", WARP)], [])], (1, 1, 1), b) == (11, 1, None)
    assert P.check_program([("split", WARP, X, 1, [("sync", BLOCK)], [])], (1, 1, 1), b) == (11, 1, None)
    assert P.check_program([("split", WARP, X, 1, [("sync", WARP)], [])], (1, 1, 1), b) == (0, -1, None)


def test_shapes_of_splits_and_selects():
    b = (64, 1, 1)
    assert P.check_program([("split", THREAD, X, 64, [], [])], (1, 1, 1), b) == (2, 0, None)
    assert P.check_program([("split", THREAD, X, 0, [], [])], (1, 1, 1), b) == (2, 0, None)
    # inside the first 32 threads a [[thread]] select needs 32 elements
    assert P.check_program([("split", THREAD, X, 32, [("access", 0, [64], thr(64), W)], [])],
                           (1, 1, 1), b) == (2, 1, None)
    assert P.check_program([("split", THREAD, X, 32, [("access", 0, [32], thr(32), W)],
                             [("access", 1, [32], thr(32), W)])], (1, 1, 1), b) == (0, -1, None)
    # warp selects where the threads are split
    assert P.check_program([("split", THREAD, X, 32, [("access", 0, [32], [("select", WARP, X)], W)], [])],
                           (1, 1, 1), b)[0] == 2


def test_two_dimensional_blocks():
    # 16 x 4 threads: a split along Y at 2 gives two halves of 16 x 2
    b = (16, 4, 1)
    sel = [("select", THREAD, Y), ("select", THREAD, X)]
    first = [("access", 0, [2, 16], sel, W)]
    second = [("access", 0, [2, 16], sel, W)]
    assert P.check_program([("split", THREAD, Y, 2, first, second)], (1, 1, 1), b) == (3, 2, 0)
    assert P.check_program([("split", THREAD, Y, 2, first, [("access", 1, [2, 16], sel, W)])],
                           (1, 1, 1), b) == (0, -1, None)
