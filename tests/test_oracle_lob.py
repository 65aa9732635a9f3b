"""Pins of the order-book oracle (Section 5.3; the rules are the engine's own,
restated in orc_lob_match): an independent share-by-share matcher on small
books, invariants, special cases, and the free-slot allocator for new orders."""
import numpy as np
import pytest

import oracle
import workloads


def brute_match(book):
    """Continuous matching one share at a time: while the best bid (highest
    price, then earliest time, then lowest slot) is priced at or above the
    best ask (lowest price, ...), one share trades between them."""
    nb, cap = book["active"].shape
    vol = np.zeros(nb, np.int64)
    px = np.full(nb, -1, np.int32)
    for b in range(nb):
        left = {i: int(book["qty"][b, i]) for i in range(cap) if book["active"][b, i]}
        while True:
            bids = [i for i in left if left[i] > 0 and book["side"][b, i] == 0]
            asks = [i for i in left if left[i] > 0 and book["side"][b, i] == 1]
            if not bids or not asks:
                break
            bi = min(bids, key=lambda i: (-book["price"][b, i], book["time"][b, i], i))
            ai = min(asks, key=lambda i: (book["price"][b, i], book["time"][b, i], i))
            if book["price"][b, bi] < book["price"][b, ai]:
                break
            left[bi] -= 1
            left[ai] -= 1
            vol[b] += 1
            px[b] = book["price"][b, ai]
        for i, q in left.items():
            book["qty"][b, i] = q
            if q == 0:
                book["active"][b, i] = 0
    return vol, px


def copy(book):
    return {k: v.copy() for k, v in book.items()}


@pytest.mark.parametrize("seed", range(12))
def test_match_vs_share_by_share(seed):
    book = workloads.random_books(16, 24, 0.7, seed, price_spread=3, qty_max=5)
    if seed % 3 == 0:  # ties in price and time (time ties broken by slot)
        book["time"][:] = 0
    a, b = copy(book), copy(book)
    vol, px = oracle.lob_match(a)
    bvol, bpx = brute_match(b)
    np.testing.assert_array_equal(vol, bvol)
    np.testing.assert_array_equal(px, bpx)
    np.testing.assert_array_equal(a["qty"], b["qty"])
    np.testing.assert_array_equal(a["active"], b["active"])


@pytest.mark.parametrize("seed", range(6))
def test_match_invariants(seed):
    book = workloads.random_books(64, 200, 0.6, 100 + seed)
    before = copy(book)
    vol, px = oracle.lob_match(book)
    for b in range(64):
        for s in (0, 1):
            was = (before["active"][b] != 0) & (before["side"][b] == s)
            traded = (before["qty"][b][was].astype(np.int64) - np.where(book["active"][b][was] != 0,
                                                                        book["qty"][b][was], 0)).sum()
            assert traded == vol[b]  # both sides trade V shares
        live = book["active"][b] != 0
        bids = book["price"][b][live & (book["side"][b] == 0)]
        asks = book["price"][b][live & (book["side"][b] == 1)]
        if bids.size and asks.size:
            assert bids.max() < asks.min()  # the book no longer crosses
        assert (book["qty"][b][live] > 0).all()
        if vol[b] == 0:
            assert px[b] == -1
        else:
            assert px[b] in before["price"][b][(before["active"][b] != 0) & (before["side"][b] == 1)]


def test_match_special_cases():
    def one(orders, cap=4):
        book = {k: np.zeros((1, cap), np.int32) for k in ("active", "side", "price", "qty", "time")}
        for i, (s, p, q, t) in enumerate(orders):
            book["active"][0, i], book["side"][0, i], book["price"][0, i] = 1, s, p
            book["qty"][0, i], book["time"][0, i] = q, t
        vol, px = oracle.lob_match(book)
        return int(vol[0]), int(px[0]), book
    assert one([])[:2] == (0, -1)
    assert one([(0, 100, 5, 0)])[:2] == (0, -1)  # bids only
    assert one([(0, 99, 5, 0), (1, 100, 5, 1)])[:2] == (0, -1)  # no crossing
    v, p, bk = one([(0, 100, 5, 0), (1, 100, 3, 1)])  # equal prices trade min(qty)
    assert (v, p) == (3, 100) and bk["qty"][0, 0] == 2 and bk["active"][0, 1] == 0
    v, p, bk = one([(0, 105, 4, 0), (0, 101, 4, 1), (1, 100, 3, 2), (1, 103, 10, 3)])
    # shares 1-3: bid 105 vs ask 100; share 4: bid 105 vs ask 103; shares 5-8: bid 101 < 103
    assert (v, p) == (4, 103)


def test_add_into_lowest_free_slots():
    rng = np.random.default_rng(5)
    book = workloads.random_books(30, 40, 0.5, 9)
    new, k = workloads.random_new_orders(30, 25, 10)
    k[0], k[1], k[2] = -4, 25 + 7, 0  # counts outside [0, kmax] are clamped to it
    book["active"][1] = 0  # 40 free slots: only kmax = 25 orders exist to place
    before = copy(book)
    added = oracle.lob_add(book, new, k)
    for b in range(30):
        free = [i for i in range(40) if not before["active"][b, i]]  # ascending
        r = min(max(int(k[b]), 0), 25, len(free))
        assert added[b] == r
        for j, slot in enumerate(free[:r]):
            assert book["active"][b, slot] == 1
            assert [book[f][b, slot] for f in ("side", "price", "qty", "time")] == new[b, j].tolist()
        untouched = np.setdiff1d(np.arange(40), free[:r])
        for f in ("active", "side", "price", "qty", "time"):
            np.testing.assert_array_equal(book[f][b, untouched], before[f][b, untouched])
    del rng
    assert added[0] == 0 and added[1] == 25 and added[2] == 0


@pytest.mark.parametrize("seed", range(8))
def test_volume_is_max_over_prices_of_min_demand_supply(seed):
    """A second characterisation of the traded volume: with D(p) the bid
    shares priced at or above p and S(p) the ask shares priced at or below p,
    V = max over p of min(D(p), S(p)) (the bid holding share min(D, S) is
    priced >= p, the ask holding it <= p; at the clearing price both reach
    V). The clearing price is the smallest p with S(p) >= V."""
    book = workloads.random_books(40, 200, 0.2 + 0.1 * seed, seed=500 + seed, price_spread=3 + seed)
    ref = copy(book)
    vol, px = oracle.lob_match(ref)
    for b in range(40):
        live = book["active"][b] != 0
        bid = live & (book["side"][b] == 0)
        ask = live & (book["side"][b] != 0)
        prices = np.unique(book["price"][b][live])
        D = np.array([book["qty"][b][bid & (book["price"][b] >= p)].sum() for p in prices], dtype=np.int64)
        S = np.array([book["qty"][b][ask & (book["price"][b] <= p)].sum() for p in prices], dtype=np.int64)
        v = int(np.minimum(D, S).max()) if len(prices) else 0
        assert vol[b] == v
        assert px[b] == (int(prices[np.argmax(S >= v)]) if v > 0 else -1)
