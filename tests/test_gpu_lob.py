"""GPU parity: batched limit-order-book matching and order placement (Section
5.3) vs the oracle, element by element and bit-exact (all arithmetic is
integer). Books span ragged caps (1 slot to the 2048-slot maximum), more books
than the launch has CTAs (grid-stride), ties on price and time, extreme
prices, times and quantities, empty / one-sided / non-crossing books, and the
full 65536 x 1024 benchmark workload."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    return engine


def copy(book):
    return {f: np.ascontiguousarray(v.copy()) for f, v in book.items()}


def check_match(eng, book):
    dev = eng.OrderBooks(book)
    ref = copy(book)
    vol_o, px_o = oracle.lob_match(ref)
    vol, px = dev.match()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(vol.cpu().numpy(), vol_o)
    np.testing.assert_array_equal(px.cpu().numpy(), px_o)
    got = dev.numpy()
    for f in ("active", "side", "price", "time"):
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    # a filled order's qty is left as the oracle leaves it (0 for filled ones)
    np.testing.assert_array_equal(got["qty"], ref["qty"])
    return vol_o


@pytest.mark.parametrize("n_books,cap", [(1, 1), (5, 2), (64, 7), (300, 255), (300, 256), (129, 257),
                                         (40, 1000), (17, 1024), (9, 2047), (6, 2048), (3000, 64)])
@pytest.mark.parametrize("fill", [0.3, 0.9])
def test_match_random(eng, n_books, cap, fill):
    book = workloads.random_books(n_books, cap, fill, seed=n_books * 7 + cap)
    vol = check_match(eng, book)
    if n_books * cap >= 1000:
        assert (vol > 0).any()  # the generator's books do cross


def test_match_ties(eng):
    # every order at one price and one time: priority by slot alone
    book = workloads.random_books(200, 300, 0.7, seed=3, price_spread=0)
    book["price"][:] = 100
    book["time"][:] = 5
    check_match(eng, book)


def test_match_extremes(eng):
    rng = np.random.default_rng(11)
    book = workloads.random_books(100, 512, 0.8, seed=12)
    book["price"] = rng.choice(np.array([1, 2, 2**31 - 2, 2**31 - 1], np.int32), size=book["price"].shape)
    book["time"] = rng.choice(np.array([-2**31, -1, 0, 2**31 - 1], np.int32), size=book["time"].shape)
    book["qty"] = rng.choice(np.array([1, 2**31 - 1], np.int32), size=book["qty"].shape)
    vol = check_match(eng, book)
    assert vol.max() > 2**32  # share sums past 32 bits


def test_match_degenerate(eng):
    cap = 300
    books = []
    empty = workloads.random_books(1, cap, 0.0, seed=1)
    books.append(empty)
    bids = workloads.random_books(1, cap, 0.9, seed=2)
    bids["side"][:] = 0
    books.append(bids)
    asks = workloads.random_books(1, cap, 0.9, seed=3)
    asks["side"][:] = 1
    books.append(asks)
    apart = workloads.random_books(1, cap, 0.9, seed=4)
    apart["price"] = np.where(apart["side"] == 0, 50, 60).astype(np.int32)  # never cross
    books.append(apart)
    one = workloads.random_books(1, cap, 0.0, seed=5)
    one["active"][0, [3, 200]] = 1
    one["side"][0, 3], one["side"][0, 200] = 0, 1
    one["price"][0, 3], one["price"][0, 200] = 10, 10
    one["qty"][0, 3], one["qty"][0, 200] = 4, 9
    books.append(one)
    book = {f: np.concatenate([b[f] for b in books]) for f in books[0]}
    vol = check_match(eng, book)
    assert list(vol) == [0, 0, 0, 0, 4]


def test_zero_books(eng):
    dev = eng.OrderBooks(workloads.random_books(0, 16, 0.5, seed=1))
    vol, px = dev.match()
    assert dev.add(torch.zeros((0, 4, 4), dtype=torch.int32), torch.zeros(0, dtype=torch.int32)).numel() == 0
    torch.cuda.synchronize()
    assert vol.numel() == 0 and px.numel() == 0


@pytest.mark.parametrize("n_books,cap,kmax", [(1, 1, 3), (70, 33, 40), (300, 257, 64), (2000, 128, 100),
                                              (8, 2048, 2048), (50, 64, 0)])
def test_add(eng, n_books, cap, kmax):
    book = workloads.random_books(n_books, cap, 0.6, seed=cap + kmax)
    orders, k = workloads.random_new_orders(n_books, kmax, seed=kmax + 1)
    if n_books > 2:
        k[0], k[1] = -3, kmax + 5  # clamped to [0, kmax]
    dev = eng.OrderBooks(book)
    ref = copy(book)
    added_o = oracle.lob_add(ref, orders, k)
    added = dev.add(torch.from_numpy(orders), torch.from_numpy(k))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(added.cpu().numpy(), added_o)
    got = dev.numpy()
    for f in ref:
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)


def test_market_rounds(eng):
    """Alternating order placement and matching for several rounds, the whole
    book state compared after every call."""
    n_books, cap, kmax = 500, 512, 96
    book = workloads.random_books(n_books, cap, 0.4, seed=31)
    dev = eng.OrderBooks(book)
    ref = copy(book)
    for r in range(6):
        orders, k = workloads.random_new_orders(n_books, kmax, seed=100 + r, time0=(1 << 20) + r * kmax)
        a_o = oracle.lob_add(ref, orders, k)
        a = dev.add(torch.from_numpy(orders), torch.from_numpy(k))
        v_o, p_o = oracle.lob_match(ref)
        v, p = dev.match()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), a_o)
        np.testing.assert_array_equal(v.cpu().numpy(), v_o)
        np.testing.assert_array_equal(p.cpu().numpy(), p_o)
        got = dev.numpy()
        for f in ref:
            np.testing.assert_array_equal(got[f], ref[f], err_msg=f"{f} round {r}")


def test_full_size_workload(eng):
    """The 65536 books x 1024 slots benchmark workload, every book compared."""
    W = workloads.LOB
    book = workloads.random_books(W["n_books"], W["cap"], W["fill"], W["seed"])
    check_match(eng, book)


def test_match_sort_path_crowded_level(eng):
    """More than 256 orders on one marginal price level: those books are
    matched by the sort path; others in the same launch by price levels."""
    book = workloads.random_books(64, 2048, 0.9, seed=41, price_spread=0)
    book["price"][::2] = 100  # even books: one price level for both sides
    check_match(eng, book)


def test_match_unaligned_rows(eng):
    """Rows that are not 16-byte aligned (4-byte staging copies)."""
    from paper_2508_16508_gb300 import abm
    nb, cap = 300, 512
    book = workloads.random_books(nb, cap, 0.6, seed=43)
    ref = copy(book)
    vol_o, px_o = oracle.lob_match(ref)
    t = {}
    for f, v in book.items():
        base = torch.zeros(nb * cap + 1, dtype=torch.int32, device="cuda")
        base[1:] = torch.from_numpy(v.reshape(-1)).cuda()
        t[f] = base[1:]  # 4 bytes past a 256-byte boundary
    vol = torch.empty(nb, dtype=torch.int64, device="cuda")
    px = torch.empty(nb, dtype=torch.int32, device="cuda")
    abm.call("abm_lob_match", nb, cap, *[abm.ptr(t[f]) for f in ("active", "side", "price", "qty", "time")],
             abm.ptr(vol), abm.ptr(px), abm.stream_handle(None))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(vol.cpu().numpy(), vol_o)
    np.testing.assert_array_equal(px.cpu().numpy(), px_o)
    for f in ("active", "qty"):
        np.testing.assert_array_equal(t[f].cpu().numpy().reshape(nb, cap), ref[f], err_msg=f)


def test_market_paper_scale(eng):
    """The finance model's scale (500 books x 1000 slots, 100 steps of up to
    10 new orders per book and a matching round), every output compared."""
    M = workloads.LOB_MARKET
    orders, ks = workloads.market_orders(M["n_books"], M["traders"], M["steps"], M["seed"])
    book = workloads.random_books(M["n_books"], M["cap"], M["fill"], M["seed"])
    dev = eng.OrderBooks(book)
    ref = copy(book)
    d_orders, d_k = torch.from_numpy(orders).cuda(), torch.from_numpy(ks).cuda()
    vols, pxs, adds = [], [], []
    for st in range(M["steps"]):
        adds.append(dev.add(d_orders[st], d_k[st]))
        v, p = dev.match()
        vols.append(v)
        pxs.append(p)
    torch.cuda.synchronize()
    traded = 0
    for st in range(M["steps"]):
        a_o = oracle.lob_add(ref, orders[st], ks[st])
        v_o, p_o = oracle.lob_match(ref)
        np.testing.assert_array_equal(adds[st].cpu().numpy(), a_o)
        np.testing.assert_array_equal(vols[st].cpu().numpy(), v_o)
        np.testing.assert_array_equal(pxs[st].cpu().numpy(), p_o)
        traded += int(v_o.sum())
    got = dev.numpy()
    for f in ref:
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    assert traded > 0


@pytest.mark.parametrize("warps", [1, 2, 4])
@pytest.mark.parametrize("cap", [7, 128, 257, 1000, 1024, 2048])
def test_match_every_launch_shape(eng, warps, cap):
    """The price-level path with 1, 2 or 4 warps per book (results must not
    depend on it), ragged and full caps, crowded and wide books mixed in."""
    eng.OrderBooks.tune(warps)
    try:
        book = workloads.random_books(97, cap, 0.7, seed=cap * 3 + warps)
        book["price"][5::7] = 100  # some books on one price level
        book["price"][3::11] = np.where(book["side"][3::11] == 0, 10**6, 10)  # some with a wide range
        check_match(eng, book)
    finally:
        eng.OrderBooks.tune(0)


def test_market_graph_replay_equals_eager(eng):
    """Placement + matching steps captured in a CUDA graph and replayed give
    the eager calls' results (every call enqueues on the capturing stream)."""
    n_books, cap, kmax, steps = 200, 500, 10, 12
    orders, ks = workloads.market_orders(n_books, kmax, steps, seed=77)
    book = workloads.random_books(n_books, cap, 0.3, seed=78)
    d_orders, d_k = torch.from_numpy(orders).cuda(), torch.from_numpy(ks).cuda()
    outs = [torch.empty(steps, n_books, dtype=t, device="cuda") for t in (torch.int32, torch.int64, torch.int32)]
    eager = eng.OrderBooks(book)
    for st in range(steps):
        eager.add(d_orders[st], d_k[st], out=outs[0][st])
        eager.match(outs[1][st], outs[2][st])
    torch.cuda.synchronize()
    want = [o.clone() for o in outs]
    replay = eng.OrderBooks(book)
    start = {f: replay.t[f].clone() for f in replay.FIELDS}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for st in range(steps):
                replay.add(d_orders[st], d_k[st], out=outs[0][st])
                replay.match(outs[1][st], outs[2][st])
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for f in replay.FIELDS:
            replay.t[f].copy_(start[f])
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, w in zip(outs, want):
            assert torch.equal(o, w)
        for f in replay.FIELDS:
            assert torch.equal(replay.t[f], eager.t[f]), f
