// Limit order books (ABMax Section 5.3): many books matched in parallel, and
// traders' new orders placed into each book's vacant slots (the add primitive
// of Section 4 per book).
//
// Matching rule (the paper gives none; the oracle restates the same): bids in
// priority order (price descending, then time, then slot), asks likewise
// (price ascending). The traded volume V is the largest share count v such
// that the bid holding share v is priced at or above the ask holding share v;
// the first V shares of each side trade, so an order fills clamp(V - shares
// ahead of it, 0, qty) and filled orders leave the book. The price is that of
// the ask holding share V.
//
// The paper matches by sorting both sides by price and taking cumulative sums
// of shares. Here most books need no sort: with D(p) = bid shares priced >= p
// and S(p) = ask shares priced <= p,
//   V = max over p of min(D(p), S(p)),
// because the bid holding share min(D(p), S(p)) is priced >= p and the ask
// holding it <= p, while at p = the price of the ask holding share V both sums
// reach V. Only prices in [lowest ask, highest bid] matter.
//
// Level path (k_lob_match_levels): a CTA of G warps matches one book at a
// time. It stages the book's active, side, price and qty words into shared
// memory with cp.async, moves each thread's slots into registers (and starts
// staging its next book), builds per-price histograms of the range (shares |
// orders << 21, one shared atomic per order), scans them into D and S, and
// takes V, the bid level pb holding share V (largest p with D(p) >= V) and the
// ask level pa holding it (smallest p with S(p) >= V). Bids above pb and asks
// below pa fill whole, those beyond fill nothing, and only the orders on the
// two marginal levels are ranked by (time, slot), by counting.
//
// Sort path (k_lob_deferred): a book whose range is wider than kWarpLevels
// prices, whose marginal level holds more than kWarpMarginal orders, or whose
// bid or ask shares reach 2^21 is left untouched by the level path (its
// volume set to -1) and matched by a second kernel, one CTA per book: bitonic
// sort of the whole book in shared memory, cumulative sums, a binary search
// per bid.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"

namespace abm {

constexpr int kLobThreads = 256;        // sort path: threads per book
constexpr int kLobWarps = kLobThreads / 32;
constexpr int kWarpLevels = 256;        // level path: prices in [lowest ask, highest bid], at most
constexpr int kWarpMarginal = 64;       // level path: orders on one marginal level, at most
constexpr u32 kShareBits = 21;          // level words: shares in the low 21 bits, orders above
constexpr u32 kShareMask = (1u << kShareBits) - 1u;
constexpr u32 kLive = 1u << 31, kAsk = 1u << 30;  // packed slot word: live | ask | qty


// order-preserving map of int32 onto u32
__device__ __forceinline__ u32 ord32(int32_t p) { return (u32)p ^ 0x80000000u; }

// Block-wide exclusive scan of a u64 (every thread gets its prefix and the
// total). Three barriers; the buffer is free again when it returns.
__device__ __forceinline__ u64 block_sum_scan_u64(u64 v, u64& total, u64* s_warp /* [kLobWarps + 1] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const u64 w = lane < kLobWarps ? s_warp[lane] : 0ull;
    u64 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kLobWarps) s_warp[lane] = wi - w;
    if (lane == kLobWarps - 1) s_warp[kLobWarps] = wi;
  }
  __syncthreads();
  const u64 ex = s_warp[warp] + incl - v;
  total = s_warp[kLobWarps];
  __syncthreads();
  return ex;
}

// One book's words in shared memory (n entries each; slots >= cap hold
// active = 0).
struct LobBook {
  int32_t* act;
  int32_t* sid;
  int32_t* px;
  int32_t* qt;
};

// The sort path for one book (see the file comment). n = R * kLobThreads
// padded slots; key/cum share one u64 array and ord a u32 array, both [n], in
// the work area. nbid/nask: live orders per side.
__device__ void lob_match_sorted(const LobBook& d, int n, int b, int cap, int nbid, int nask, int32_t* active,
                                 int32_t* qty, const int32_t* __restrict__ time, long long* out_volume,
                                 int32_t* out_price, u64* key, u32* ord, u64* s_scan, unsigned long long* s_v) {
  const size_t o = (size_t)b * cap;
  __syncthreads();  // the work area may still be read as level tables
  if (threadIdx.x == 0) *s_v = 0ull;
  // key: side | price (bids descending; prices positive) | time (signed
  // order); ties by slot, empty slots (slot + n) last
  for (int i = threadIdx.x; i < n; i += kLobThreads) {
    u64 k = kNoKey;
    u32 r = (u32)(i + n);
    if (d.act[i]) {
      const u32 s = d.sid[i] != 0;
      const u32 p = s ? (u32)d.px[i] : 0x7FFFFFFFu - (u32)d.px[i];
      k = ((u64)s << 63) | ((u64)(p & 0x7FFFFFFFu) << 32) | (u64)ord32(time[o + i]);
      r = (u32)i;
    }
    key[i] = k;
    ord[i] = r;
  }
  __syncthreads();
  for (int kk = 2; kk <= n; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += kLobThreads) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & kk) == 0;
          const bool gt = key[i] > key[l] || (key[i] == key[l] && ord[i] > ord[l]);
          if (gt == up) {
            const u64 tk = key[i];
            key[i] = key[l];
            key[l] = tk;
            const u32 to = ord[i];
            ord[i] = ord[l];
            ord[l] = to;
          }
        }
      }
      __syncthreads();
    }
  }
  // sorted: bids [0, nbid), asks [nbid, nbid + nask), empty slots after. The
  // keys are dead now: cum[e] (same array) = shares of entries [0, e].
  u64* cum = key;
  const int nl = nbid + nask, per = n / kLobThreads;
  u64 local = 0;
  for (int e = threadIdx.x * per; e < (threadIdx.x + 1) * per; ++e)
    local += e < nl ? (u64)(u32)d.qt[ord[e]] : 0ull;
  u64 tot;
  u64 run = block_sum_scan_u64(local, tot, s_scan);
  for (int e = threadIdx.x * per; e < (threadIdx.x + 1) * per; ++e) {
    run += e < nl ? (u64)(u32)d.qt[ord[e]] : 0ull;
    cum[e] = run;
  }
  __syncthreads();
  const u64 bid_total = nbid > 0 ? cum[nbid - 1] : 0ull;
  // V: bid i may trade the shares in (QB_{i-1}, min(QB_i, QA(J_i))], J_i = the
  // asks priced at or below it
  u64 vbest = 0;
  for (int i = threadIdx.x; i < nbid; i += kLobThreads) {
    const int32_t p = d.px[ord[i]];
    int lo = 0, hi = nask;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (d.px[ord[nbid + mid]] <= p) lo = mid + 1;
      else hi = mid;
    }
    const u64 qa = lo > 0 ? cum[nbid + lo - 1] - bid_total : 0ull;
    const u64 qb = cum[i], before = i > 0 ? cum[i - 1] : 0ull;
    const u64 c = qa < qb ? qa : qb;
    if (c > before && c > vbest) vbest = c;
  }
  if (vbest) atomicMax(s_v, (unsigned long long)vbest);
  __syncthreads();
  const u64 V = *s_v;
  if (threadIdx.x == 0) {
    out_volume[b] = (long long)V;
    if (V == 0) out_price[b] = -1;
  }
  for (int e = threadIdx.x; e < nl; e += kLobThreads) {
    const bool is_bid = e < nbid;
    const u64 start = is_bid ? (e > 0 ? cum[e - 1] : 0ull) : (e > nbid ? cum[e - 1] - bid_total : 0ull);
    const u64 end = is_bid ? cum[e] : cum[e] - bid_total;
    const u64 q = end - start;
    const u64 fill = V > start ? (V - start < q ? V - start : q) : 0ull;
    if (!is_bid && V > start && V <= end) out_price[b] = d.px[ord[e]];
    if (fill || q == 0) {
      const u32 s = ord[e];
      const int32_t left = (int32_t)(q - fill);
      qty[o + s] = left;
      if (left == 0) active[o + s] = 0;
    }
  }
}

// Shared memory of one CTA of the level path (one book at a time): the staged
// book (4 arrays of n words; slots >= cap hold active = 0), the level words of
// both sides, and the marginal lists (qty, key = time | slot) of both sides.
__host__ __device__ constexpr size_t grp_smem_bytes(int n) {
  return 16 * (size_t)n + 2 * kWarpLevels * sizeof(u32) + 2 * kWarpMarginal * (sizeof(u32) + sizeof(u64));
}

__device__ __forceinline__ int popc_mask(u32 m) { return __popc(m); }
__device__ __forceinline__ int popc_mask(u64 m) { return __popcll(m); }
__device__ __forceinline__ int ffs_mask(u32 m) { return __ffs(m); }
__device__ __forceinline__ int ffs_mask(u64 m) { return __ffsll((long long)m); }

// Inclusive warp scan of a u32.
__device__ __forceinline__ u32 warp_incl_scan(u32 v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Barrier of the G warps matching one book.
template <int G>
__device__ __forceinline__ void grp_sync() {
  if (G == 1) __syncwarp();
  else __syncthreads();
}

// Three sums, a min, a max and an or over the G warps (every thread gets
// them). One barrier; the exchange buffer alternates between calls.
struct Agg6 {
  u32 s0, s1, s2, mn, mx, orr;
};
template <int G>
__device__ __forceinline__ Agg6 grp_agg6(Agg6 a, u32 (*x)[G][8], int& par) {
  a.s0 = __reduce_add_sync(0xFFFFFFFFu, a.s0);
  a.s1 = __reduce_add_sync(0xFFFFFFFFu, a.s1);
  a.s2 = __reduce_add_sync(0xFFFFFFFFu, a.s2);
  a.mn = __reduce_min_sync(0xFFFFFFFFu, a.mn);
  a.mx = __reduce_max_sync(0xFFFFFFFFu, a.mx);
  a.orr = __reduce_or_sync(0xFFFFFFFFu, a.orr);
  if (G == 1) return a;
  if ((threadIdx.x & 31) == 0) {
    u32* d = x[par][threadIdx.x >> 5];
    d[0] = a.s0;
    d[1] = a.s1;
    d[2] = a.s2;
    d[3] = a.mn;
    d[4] = a.mx;
    d[5] = a.orr;
  }
  __syncthreads();
  Agg6 r{0u, 0u, 0u, 0xFFFFFFFFu, 0u, 0u};
#pragma unroll
  for (int w = 0; w < G; ++w) {
    const u32* d = x[par][w];
    r.s0 += d[0];
    r.s1 += d[1];
    r.s2 += d[2];
    r.mn = min(r.mn, d[3]);
    r.mx = max(r.mx, d[4]);
    r.orr |= d[5];
  }
  par ^= 1;
  return r;
}

// Exclusive scan of two u32 over the G warps' threads, with the totals.
template <int G>
__device__ __forceinline__ void grp_scan2(u32 a, u32 b, u32& ex_a, u32& ex_b, u32& tot_a, u32& tot_b,
                                          u32 (*x)[G][8], int& par) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 ia = warp_incl_scan(a, lane), ib = warp_incl_scan(b, lane);
  if (G == 1) {
    ex_a = ia - a;
    ex_b = ib - b;
    tot_a = __shfl_sync(0xFFFFFFFFu, ia, 31);
    tot_b = __shfl_sync(0xFFFFFFFFu, ib, 31);
    return;
  }
  if (lane == 31) {
    x[par][warp][0] = ia;
    x[par][warp][1] = ib;
  }
  __syncthreads();
  u32 pa = 0, pb = 0, ta = 0, tb = 0;
#pragma unroll
  for (int w = 0; w < G; ++w) {
    const u32 wa = x[par][w][0], wb = x[par][w][1];
    pa += w < warp ? wa : 0u;
    pb += w < warp ? wb : 0u;
    ta += wa;
    tb += wb;
  }
  ex_a = pa + ia - a;
  ex_b = pb + ib - b;
  tot_a = ta;
  tot_b = tb;
  par ^= 1;
}

// Book b's words into the staging arrays (asynchronous; committed). T
// threads copy.
template <int T, bool kVec16>
__device__ __forceinline__ void grp_stage(int32_t* s_act, int n, int b, int cap, const int32_t* active,
                                          const int32_t* side, const int32_t* price, const int32_t* qty) {
  const size_t o = (size_t)b * cap;
  if (kVec16) {
    for (int c = threadIdx.x; c < (cap >> 2); c += T) {
      cp_async16(s_act + 4 * c, active + o + 4 * c);
      cp_async16(s_act + n + 4 * c, side + o + 4 * c);
      cp_async16(s_act + 2 * n + 4 * c, price + o + 4 * c);
      cp_async16(s_act + 3 * n + 4 * c, qty + o + 4 * c);
    }
  } else {
    for (int c = threadIdx.x; c < cap; c += T) {
      cp_async4(s_act + c, active + o + c);
      cp_async4(s_act + n + c, side + o + c);
      cp_async4(s_act + 2 * n + c, price + o + c);
      cp_async4(s_act + 3 * n + c, qty + o + c);
    }
  }
  cp_async_commit();
}

// Level path: a CTA of G warps (T = 32 G threads) matches one book at a time;
// SPL = slots per thread (cap <= T * SPL), thread t holding slots
// 4 * (g * T + t) + c. The book's words move from the staging arrays into
// registers, and the next book is staged at once. Deferred books get
// out_volume = -1 and are left untouched.
template <int G, int SPL, bool kVec16>
__global__ void __launch_bounds__(G * 32)
    k_lob_match_levels(int n_books, int cap, int32_t* active, const int32_t* __restrict__ side,
                       const int32_t* __restrict__ price, int32_t* qty, const int32_t* __restrict__ time,
                       long long* out_volume, int32_t* out_price) {
  constexpr int T = G * 32;
  constexpr int LPT = kWarpLevels / T;  // levels per thread in the scan
  constexpr int n = T * SPL;            // staged words per array
  extern __shared__ __align__(16) unsigned char lob_smem[];
  __shared__ u32 s_x[2][G][8];
  int32_t* s_act = reinterpret_cast<int32_t*>(lob_smem);  // then side, price, qty at +n, +2n, +3n
  u32* lvb = reinterpret_cast<u32*>(s_act + 4 * n);        // bid level words, then D | orders << 21
  u32* lva = lvb + kWarpLevels;                            // ask level words, then S | orders << 21
  u32* m_qty = lva + kWarpLevels;                          // [2][kWarpMarginal]
  u64* m_key = reinterpret_cast<u64*>(m_qty + 2 * kWarpMarginal);  // [2][kWarpMarginal]
  const int t = threadIdx.x;
  int par = 0;
  for (int i = cap + t; i < n; i += T) s_act[i] = 0;  // padding slots: never copied, never live
  if ((int)blockIdx.x < n_books) grp_stage<T, kVec16>(s_act, n, blockIdx.x, cap, active, side, price, qty);
  for (int b = blockIdx.x; b < n_books; b += gridDim.x) {
    const size_t o = (size_t)b * cap;
    cp_async_wait_0();
    grp_sync<G>();

    // this thread's slots into registers: price and live | ask | qty
    int32_t px[SPL];
    u32 w[SPL];
    u32 cnt = 0, mn = 0xFFFFFFFFu, mx = 0u, sb = 0, sa = 0, flags = 0;
#pragma unroll
    for (int g = 0; g < SPL / 4; ++g) {
      const int v = g * T + t;
      const int4 a4 = reinterpret_cast<const int4*>(s_act)[v];
      const int4 s4 = reinterpret_cast<const int4*>(s_act + n)[v];
      const int4 p4 = reinterpret_cast<const int4*>(s_act + 2 * n)[v];
      const int4 q4 = reinterpret_cast<const int4*>(s_act + 3 * n)[v];
      const int av[4] = {a4.x, a4.y, a4.z, a4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
      const int pv[4] = {p4.x, p4.y, p4.z, p4.w}, qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k = 4 * g + c;
        const bool live = av[c] != 0, ask = sv[c] != 0;
        const bool lbid = live && !ask, lask = live && ask;
        const u32 q = (u32)qv[c], qm = q & kShareMask;
        flags |= (live && q > kShareMask) ? 1u : 0u;  // too large (or negative) for the level words
        flags |= (live && q == 0) ? 2u : 0u;
        px[k] = pv[c];
        w[k] = live ? (kLive | (ask ? kAsk : 0u) | qm) : 0u;
        cnt += lask ? 0x10000u : (lbid ? 1u : 0u);
        sa += lask ? qm : 0u;
        sb += lbid ? qm : 0u;
        mn = min(mn, lask ? ord32(pv[c]) : 0xFFFFFFFFu);
        mx = max(mx, lbid ? ord32(pv[c]) : 0u);
      }
    }
    // share sums saturate per thread, so the sums cannot wrap; for G > 1 the
    // barrier inside also frees the staging arrays
    const Agg6 r1 = grp_agg6<G>(Agg6{cnt, min(sb, 1u << kShareBits), min(sa, 1u << kShareBits), mn, mx, flags}, s_x,
                                par);
    if (G == 1) __syncwarp();
    if (b + (int)gridDim.x < n_books)
      grp_stage<T, kVec16>(s_act, n, b + gridDim.x, cap, active, side, price, qty);
    const bool zq = r1.orr & 2u;
    const bool cross = (r1.s0 & 0xFFFFu) != 0 && (r1.s0 >> 16) != 0 && r1.mx >= r1.mn;
    const int32_t pmin = (int32_t)(r1.mn ^ 0x80000000u), pmax = (int32_t)(r1.mx ^ 0x80000000u);
    const long long L = cross ? (long long)pmax - (long long)pmin + 1 : 0;
    if (cross && ((r1.orr & 1u) || r1.s1 > kShareMask || r1.s2 > kShareMask || L > kWarpLevels)) {
      if (t == 0) out_volume[b] = -1;  // the sort path takes it
      continue;
    }
    u32 V = 0;
    int32_t pb = 0, pa = 0;
    u32 Dn = 0, Sp = 0;
    if (cross) {
      for (int l = t; l < L; l += T) {
        lvb[l] = 0u;
        lva[l] = 0u;
      }
      grp_sync<G>();
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const bool ask = w[k] & kAsk;
        const bool in = (w[k] & kLive) && (ask ? px[k] <= pmax : px[k] >= pmin);
        if (in) atomicAdd((ask ? lva : lvb) + (px[k] - pmin), (w[k] & kShareMask) | (1u << kShareBits));
      }
      grp_sync<G>();
      // D(l) = bid shares at levels >= l, S(l) = ask shares at levels <= l;
      // thread t owns levels [LPT * t, LPT * t + LPT)
      u32 hb[LPT], ha[LPT];
      u32 tb = 0, ta = 0;
      const int l0 = t * LPT;
#pragma unroll
      for (int j = 0; j < LPT; ++j) {
        hb[j] = l0 + j < L ? lvb[l0 + j] : 0u;
        ha[j] = l0 + j < L ? lva[l0 + j] : 0u;
        tb += hb[j] & kShareMask;
        ta += ha[j] & kShareMask;
      }
      u32 pre_b, pre_a, BT, AT;
      grp_scan2<G>(tb, ta, pre_b, pre_a, BT, AT, s_x, par);
      u32 best = 0;
      u32 Dl[LPT], Sl[LPT];
#pragma unroll
      for (int j = 0; j < LPT; ++j) {
        Dl[j] = BT - pre_b;
        pre_b += hb[j] & kShareMask;
        pre_a += ha[j] & kShareMask;
        Sl[j] = pre_a;
        if (l0 + j < L) best = max(best, min(Dl[j], Sl[j]));
      }
      if (G == 1) __syncwarp();  // (G > 1: the scan's barrier came after every read)
#pragma unroll
      for (int j = 0; j < LPT; ++j) {
        if (l0 + j < L) {
          lvb[l0 + j] = Dl[j] | (hb[j] & ~kShareMask);
          lva[l0 + j] = Sl[j] | (ha[j] & ~kShareMask);
        }
      }
      V = grp_agg6<G>(Agg6{0u, 0u, 0u, 0xFFFFFFFFu, best, 0u}, s_x, par).mx;
      if (V > 0) {
        // D falls and S rises with the level: count the levels at or above V
        u32 cb = 0, ca = 0;
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
          cb += (l0 + j < L) && Dl[j] >= V;
          ca += (l0 + j < L) && Sl[j] >= V;
        }
        const Agg6 r3 = grp_agg6<G>(Agg6{cb, ca, 0u, 0xFFFFFFFFu, 0u, 0u}, s_x, par);
        const int lb = (int)r3.s0 - 1, la = (int)L - (int)r3.s1;
        grp_sync<G>();
        if ((lvb[lb] >> kShareBits) > kWarpMarginal || (lva[la] >> kShareBits) > kWarpMarginal) {
          if (t == 0) out_volume[b] = -1;  // a crowded marginal level: the sort path takes it
          continue;
        }
        pb = pmin + lb;
        pa = pmin + la;
        Dn = lb + 1 < L ? lvb[lb + 1] & kShareMask : 0u;  // bid shares priced above pb
        Sp = la > 0 ? lva[la - 1] & kShareMask : 0u;      // ask shares priced below pa
      }
    }
    if (V == 0 && !zq) {
      if (t == 0) {
        out_volume[b] = 0;
        out_price[b] = -1;
      }
      continue;
    }
    // whole fills (and zero-qty orders) written here; marginal orders marked
    // in per-thread bit masks (bit k = this thread's slot k), listed below
    using Mask = typename std::conditional<(SPL > 32), u64, u32>::type;
    Mask mmb = 0, mma = 0;
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
      const int i = 4 * ((k >> 2) * T + t) + (k & 3);
      const bool live = w[k] & kLive, ask = w[k] & kAsk;
      const u32 q = w[k] & kShareMask;
      const bool whole = live && (q == 0 || (V > 0 && (ask ? px[k] < pa : px[k] > pb)));
      const bool marg = live && q > 0 && V > 0 && px[k] == (ask ? pa : pb);
      if (whole) {
        qty[o + i] = 0;
        active[o + i] = 0;
      }
      mmb |= (Mask)(marg && !ask) << k;
      mma |= (Mask)(marg && ask) << k;
    }
    if (V > 0) {
      // list positions: scan of the per-thread counts; qty and time of the
      // marginal orders from global memory (neither written by this kernel)
      const u32 cb = (u32)popc_mask(mmb), ca = (u32)popc_mask(mma);
      u32 eb, ea, nm0, nm1;
      grp_scan2<G>(cb, ca, eb, ea, nm0, nm1, s_x, par);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        Mask m = s ? mma : mmb;
        u32 pos = s ? ea : eb;
        while (m) {
          const int k = ffs_mask(m) - 1;
          m &= m - 1;
          const u32 i = 4u * (u32)((k >> 2) * T + t) + (u32)(k & 3);
          m_qty[s * kWarpMarginal + pos] = (u32)qty[o + i];
          m_key[s * kWarpMarginal + pos] = ((u64)ord32(time[o + i]) << 32) | i;
          ++pos;
        }
      }
      grp_sync<G>();
      for (int e = t; e < (int)(nm0 + nm1); e += T) {
        const int s = e >= (int)nm0, f = e - (s ? (int)nm0 : 0), m = s ? (int)nm1 : (int)nm0;
        const u32* mq = m_qty + s * kWarpMarginal;
        const u64* mk = m_key + s * kWarpMarginal;
        const u64 mine = mk[f];
        u32 before = s ? Sp : Dn;
        for (int h = 0; h < m; ++h) before += mk[h] < mine ? mq[h] : 0u;
        const u32 q = mq[f];
        const u32 fill = V > before ? min(V - before, q) : 0u;
        if (fill) {
          const u32 slot = (u32)mine;
          qty[o + slot] = (int32_t)(q - fill);
          if (fill == q) active[o + slot] = 0;
        }
      }
    }
    if (t == 0) {
      out_volume[b] = (long long)V;
      out_price[b] = V > 0 ? pa : -1;
    }
  }
  cp_async_wait_0();
}

// Sort path for the books the level path deferred (out_volume < 0), one CTA
// per book; n = R * kLobThreads padded slots. Shared memory: the book's words
// (4 x n int32), then key u64[n] and ord u32[n].
template <int R>
__global__ void __launch_bounds__(kLobThreads)
    k_lob_deferred(int n_books, int cap, int32_t* active, const int32_t* __restrict__ side,
                   const int32_t* __restrict__ price, int32_t* qty, const int32_t* __restrict__ time,
                   long long* out_volume, int32_t* out_price) {
  constexpr int n = R * kLobThreads;
  extern __shared__ __align__(16) unsigned char lob_smem[];
  int32_t* w = reinterpret_cast<int32_t*>(lob_smem);
  const LobBook d{w, w + n, w + 2 * n, w + 3 * n};
  u64* key = reinterpret_cast<u64*>(w + 4 * n);
  u32* ord = reinterpret_cast<u32*>(key + n);
  __shared__ int s_list[kLobThreads];
  __shared__ int s_cnt;
  __shared__ u64 s_scan[kLobWarps + 1];
  __shared__ unsigned long long s_v;
  for (int c0 = blockIdx.x * kLobThreads; c0 < n_books; c0 += gridDim.x * kLobThreads) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int bq = c0 + threadIdx.x;
    if (bq < n_books && out_volume[bq] < 0) s_list[atomicAdd(&s_cnt, 1)] = bq;
    __syncthreads();
    const int m = s_cnt;
    for (int j = 0; j < m; ++j) {
      const int b = s_list[j];
      const size_t o = (size_t)b * cap;
      int nbid = 0, nask = 0;
      for (int i = threadIdx.x; i < n; i += kLobThreads) {
        const bool in = i < cap;
        const int32_t a = in ? active[o + i] : 0;
        const int32_t s = in ? side[o + i] : 0;
        d.act[i] = a;
        d.sid[i] = s;
        d.px[i] = in ? price[o + i] : 0;
        d.qt[i] = in ? qty[o + i] : 0;
        nbid += __syncthreads_count(a != 0 && s == 0);
        nask += __syncthreads_count(a != 0 && s != 0);
      }
      lob_match_sorted(d, n, b, cap, nbid, nask, active, qty, time, out_volume, out_price, key, ord, s_scan, &s_v);
      __syncthreads();  // shared arrays are reused by the next book
    }
  }
}

// new orders into each book's lowest free slots: order j < k[b] -> j-th free
// slot; per = slots per thread (cap padded to n = per * kLobThreads)
__global__ void __launch_bounds__(kLobThreads) k_lob_add(int n_books, int cap, int n, int32_t* active, int32_t* side,
                                                         int32_t* price, int32_t* qty, int32_t* time,
                                                         const int32_t* __restrict__ orders,
                                                         const int32_t* __restrict__ k, int kmax,
                                                         int32_t* out_added) {
  __shared__ u64 s_warp[kLobWarps + 1];
  const int per = n / kLobThreads;
  for (int b = blockIdx.x; b < n_books; b += gridDim.x) {
    const size_t o = (size_t)b * cap;
    const int kb = min(max(k[b], 0), kmax);
    u64 local = 0;
    for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per; ++i) local += (i < cap && !active[o + i]) ? 1 : 0;
    u64 tot;
    u64 rank = block_sum_scan_u64(local, tot, s_warp);
    for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per; ++i) {
      if (i >= cap || active[o + i]) continue;
      if ((int)rank < kb) {
        const int32_t* r = orders + ((size_t)b * kmax + rank) * 4;
        side[o + i] = r[0];
        price[o + i] = r[1];
        qty[o + i] = r[2];
        time[o + i] = r[3];
        active[o + i] = 1;
      }
      ++rank;
    }
    if (threadIdx.x == 0) out_added[b] = (int32_t)min((u64)kb, tot);
  }
}


static int lob_pad(int cap) {
  int n = kLobThreads;
  while (n < cap) n <<= 1;
  return n;
}

static std::atomic<int> g_lob_warps_per_book{2};  // level path: warps per book (1, 2 or 4)

template <int G, int SPL, bool kVec16>
static abm_status lob_launch_levels(int n_books, int cap, int32_t* active, const int32_t* side, const int32_t* price,
                                    int32_t* qty, const int32_t* time, long long* vol, int32_t* px, cudaStream_t st) {
  // the shared-memory limit and the occupancy are per device: looked up once for each
  static std::atomic<unsigned long long> attr{0};
  static std::atomic<int> occ_dev[64];
  const size_t smem = grp_smem_bytes(G * 32 * SPL);
  ABM_CUDA_TRY(smem_attr_once(k_lob_match_levels<G, SPL, kVec16>, (int)smem, attr));
  int dev = 0;
  ABM_CUDA_TRY(cudaGetDevice(&dev));
  int blocks_per_sm = (dev >= 0 && dev < 64) ? occ_dev[dev].load(std::memory_order_relaxed) : 0;
  if (!blocks_per_sm) {
    int occ = 0;
    ABM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lob_match_levels<G, SPL, kVec16>, G * 32,
                                                               smem));
    blocks_per_sm = std::max(occ, 1);
    if (dev >= 0 && dev < 64) occ_dev[dev].store(blocks_per_sm, std::memory_order_relaxed);
  }
  const int grid = (int)std::min<long long>(n_books, (long long)num_sms() * blocks_per_sm);
  k_lob_match_levels<G, SPL, kVec16><<<grid, G * 32, smem, st>>>(n_books, cap, active, side, price, qty, time, vol,
                                                                  px);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

// the smallest slots-per-thread (a multiple of 4) that covers cap
template <int G, bool kVec16>
static abm_status lob_launch_g(int n_books, int cap, int32_t* active, const int32_t* side, const int32_t* price,
                               int32_t* qty, const int32_t* time, long long* vol, int32_t* px, cudaStream_t st) {
  constexpr int T = G * 32;
  if (cap <= 4 * T) return lob_launch_levels<G, 4, kVec16>(n_books, cap, active, side, price, qty, time, vol, px, st);
  if (cap <= 8 * T) return lob_launch_levels<G, 8, kVec16>(n_books, cap, active, side, price, qty, time, vol, px, st);
  if (cap <= 16 * T)
    return lob_launch_levels<G, 16, kVec16>(n_books, cap, active, side, price, qty, time, vol, px, st);
  if (G <= 2 && cap <= 32 * T)
    return lob_launch_levels<G, (G <= 2 ? 32 : 16), kVec16>(n_books, cap, active, side, price, qty, time, vol, px,
                                                             st);
  return lob_launch_levels<G, (G == 1 ? 64 : 16), kVec16>(n_books, cap, active, side, price, qty, time, vol, px,
                                                           st);
}

template <int R>
static abm_status lob_launch_deferred(int n_books, int cap, int32_t* active, const int32_t* side,
                                      const int32_t* price, int32_t* qty, const int32_t* time, long long* vol,
                                      int32_t* px, cudaStream_t st) {
  constexpr size_t smem = (size_t)R * kLobThreads * (4 * sizeof(int32_t) + sizeof(u64) + sizeof(u32));
  static std::atomic<unsigned long long> attr{0};
  ABM_CUDA_TRY(smem_attr_once(k_lob_deferred<R>, (int)smem, attr));
  const long long chunks = ((long long)n_books + kLobThreads - 1) / kLobThreads;
  const int grid = (int)std::min<long long>(chunks, (long long)num_sms() * 2);
  k_lob_deferred<R><<<grid, kLobThreads, smem, st>>>(n_books, cap, active, side, price, qty, time, vol, px);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

static abm_status lob_launch(bool vec16, int n_books, int cap, int32_t* active, const int32_t* side,
                             const int32_t* price, int32_t* qty, const int32_t* time, long long* vol, int32_t* px,
                             cudaStream_t st) {
  abm_status e;
  switch (g_lob_warps_per_book.load(std::memory_order_relaxed)) {
    case 1:
      e = vec16 ? lob_launch_g<1, true>(n_books, cap, active, side, price, qty, time, vol, px, st)
                : lob_launch_g<1, false>(n_books, cap, active, side, price, qty, time, vol, px, st);
      break;
    case 4:
      e = vec16 ? lob_launch_g<4, true>(n_books, cap, active, side, price, qty, time, vol, px, st)
                : lob_launch_g<4, false>(n_books, cap, active, side, price, qty, time, vol, px, st);
      break;
    default:
      e = vec16 ? lob_launch_g<2, true>(n_books, cap, active, side, price, qty, time, vol, px, st)
                : lob_launch_g<2, false>(n_books, cap, active, side, price, qty, time, vol, px, st);
  }
  if (e != ABM_OK) return e;
  switch (lob_pad(cap) / kLobThreads) {
    case 1: return lob_launch_deferred<1>(n_books, cap, active, side, price, qty, time, vol, px, st);
    case 2: return lob_launch_deferred<2>(n_books, cap, active, side, price, qty, time, vol, px, st);
    case 4: return lob_launch_deferred<4>(n_books, cap, active, side, price, qty, time, vol, px, st);
    default: return lob_launch_deferred<8>(n_books, cap, active, side, price, qty, time, vol, px, st);
  }
}

}  // namespace abm

using namespace abm;

extern "C" abm_status abm_lob_match(int32_t n_books, int32_t cap, int32_t* active, const int32_t* side,
                                    const int32_t* price, int32_t* qty, const int32_t* time, int64_t* out_volume,
                                    int32_t* out_price, void* stream) {
  if (n_books < 0 || cap < 1 || cap > ABM_LOB_MAX_CAP) return ABM_ERR_ARG;
  if (n_books == 0) return ABM_OK;
  if (!active || !side || !price || !qty || !time || !out_volume || !out_price) return ABM_ERR_ARG;
  // 16-byte copies need every book's rows 16-byte aligned
  const bool vec16 =
      cap % 4 == 0 && ((uintptr_t)active | (uintptr_t)side | (uintptr_t)price | (uintptr_t)qty) % 16 == 0;
  long long* vol = reinterpret_cast<long long*>(out_volume);
  const cudaStream_t st = (cudaStream_t)stream;
  return lob_launch(vec16, n_books, cap, active, side, price, qty, time, vol, out_price, st);
}

extern "C" abm_status abm_lob_tune(int32_t warps_per_book) {
  if (warps_per_book != 0 && warps_per_book != 1 && warps_per_book != 2 && warps_per_book != 4) return ABM_ERR_ARG;
  g_lob_warps_per_book.store(warps_per_book ? warps_per_book : 2, std::memory_order_relaxed);
  return ABM_OK;
}

extern "C" abm_status abm_lob_add(int32_t n_books, int32_t cap, int32_t* active, int32_t* side, int32_t* price,
                                  int32_t* qty, int32_t* time, const int32_t* new_orders, const int32_t* k,
                                  int32_t kmax, int32_t* out_added, void* stream) {
  if (n_books < 0 || cap < 1 || cap > ABM_LOB_MAX_CAP || kmax < 0) return ABM_ERR_ARG;
  if (n_books == 0) return ABM_OK;
  if (!active || !side || !price || !qty || !time || !k || !out_added || (kmax > 0 && !new_orders))
    return ABM_ERR_ARG;
  const int grid = std::min(n_books, num_sms() * 8);
  k_lob_add<<<grid, kLobThreads, 0, (cudaStream_t)stream>>>(n_books, cap, lob_pad(cap), active, side, price, qty,
                                                             time, new_orders, k, kmax, out_added);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}
