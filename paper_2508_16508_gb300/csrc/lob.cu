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
// of shares. Here one CTA matches one book at a time, and most books need no
// sort: with D(p) = bid shares priced >= p and S(p) = ask shares priced <= p,
//   V = max over p of min(D(p), S(p)),
// because the bid holding share min(D(p), S(p)) is priced >= p and the ask
// holding it <= p, while at p = the price of the ask holding share V both sums
// reach V. Only prices in [lowest ask, highest bid] matter, so the level path
// builds per-price share histograms of that range in shared memory (one
// atomic per order), scans them into D and S, and takes V, the bid level pb
// holding share V (largest p with D(p) >= V) and the ask level pa holding it
// (smallest p with S(p) >= V). Bids above pb and asks below pa fill whole,
// those beyond fill nothing, and only the orders on the two marginal levels
// are ranked by (time, slot) -- by counting, they are few. A book whose range
// is wider than kLobLevels prices, whose marginal levels hold more than
// kLobMarginal orders, or with a qty >= kLobQtyMax takes the sort path:
// bitonic sort of the whole book in shared memory, cumulative sums, and a
// binary search per bid.
//
// Each CTA streams the next book's active, side, price and qty words into a
// second shared-memory buffer with cp.async while it matches the current one.
#include <algorithm>

#include "common.cuh"

namespace abm {

constexpr int kLobThreads = 256;
constexpr int kLobWarps = kLobThreads / 32;
constexpr int kLobLevels = 1024;       // prices in the level path's range, at most
constexpr int kLobLevelsPerThread = kLobLevels / kLobThreads;
constexpr int kLobMarginal = 256;      // orders on one marginal level, at most
constexpr u32 kLobQtyMax = 1u << 20;   // every qty below this keeps share sums in 32 bits
constexpr size_t kLobLevelBytes = 2 * kLobLevels * sizeof(u32) + 2 * kLobMarginal * (sizeof(u64) + sizeof(u32));

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// order-preserving map of int32 onto u32
__device__ __forceinline__ u32 ord32(int32_t p) { return (u32)p ^ 0x80000000u; }

// Block-wide (sum, sum, min, max) of u32 values; every thread gets the result.
// One barrier; two alternating buffers make back-to-back calls safe.
struct Red4 {
  u32 a, b, mn, mx;
};
__device__ __forceinline__ Red4 block_red4(u32 a, u32 b, u32 mn, u32 mx, uint4 (*s)[kLobWarps], int& par) {
  a = __reduce_add_sync(0xFFFFFFFFu, a);
  b = __reduce_add_sync(0xFFFFFFFFu, b);
  mn = __reduce_min_sync(0xFFFFFFFFu, mn);
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  if ((threadIdx.x & 31) == 0) s[par][threadIdx.x >> 5] = make_uint4(a, b, mn, mx);
  __syncthreads();
  Red4 r{0u, 0u, 0xFFFFFFFFu, 0u};
#pragma unroll
  for (int w = 0; w < kLobWarps; ++w) {
    const uint4 v = s[par][w];
    r.a += v.x;
    r.b += v.y;
    r.mn = min(r.mn, v.z);
    r.mx = max(r.mx, v.w);
  }
  par ^= 1;
  return r;
}

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

// One book's staged words in shared memory (n entries each; slots >= cap hold
// active = 0).
struct LobBook {
  int32_t* act;
  int32_t* sid;
  int32_t* px;
  int32_t* qt;
};

// Book b's words into the staging buffer (asynchronous; the caller commits).
template <bool kVec16>
__device__ __forceinline__ void lob_issue(const LobBook& d, int b, int cap, const int32_t* active,
                                          const int32_t* side, const int32_t* price, const int32_t* qty) {
  const size_t o = (size_t)b * cap;
  const int32_t* src[4] = {active + o, side + o, price + o, qty + o};
  int32_t* dst[4] = {d.act, d.sid, d.px, d.qt};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (kVec16) {
      for (int c = threadIdx.x; c < (cap >> 2); c += kLobThreads) cp_async16(dst[a] + 4 * c, src[a] + 4 * c);
    } else {
      for (int c = threadIdx.x; c < cap; c += kLobThreads) cp_async4(dst[a] + c, src[a] + c);
    }
  }
}

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

// Dynamic shared memory: two staging buffers of 4 * n int32, then the work
// area (level tables and marginal lists, or the sort path's key/ord arrays).
template <int R, bool kVec16>
__global__ void __launch_bounds__(kLobThreads, R >= 8 ? 2 : 4)
    k_lob_match(int n_books, int cap, int32_t* active, const int32_t* __restrict__ side,
                const int32_t* __restrict__ price, int32_t* qty, const int32_t* __restrict__ time,
                long long* out_volume, int32_t* out_price) {
  constexpr int n = R * kLobThreads;
  extern __shared__ __align__(16) unsigned char lob_smem[];
  int32_t* stage = reinterpret_cast<int32_t*>(lob_smem);
  auto staged = [&](int s) -> LobBook {
    int32_t* q = stage + 4 * n * s;
    return LobBook{q, q + n, q + 2 * n, q + 3 * n};
  };
  unsigned char* work = lob_smem + 8 * (size_t)n * sizeof(int32_t);
  u32* hb = reinterpret_cast<u32*>(work);  // bid shares per level, then D
  u32* ha = hb + kLobLevels;               // ask shares per level, then S
  u64* mk = reinterpret_cast<u64*>(ha + kLobLevels);  // marginal keys [2][kLobMarginal]
  u32* mq = reinterpret_cast<u32*>(mk + 2 * kLobMarginal);  // marginal qty [2][kLobMarginal]
  u64* skey = reinterpret_cast<u64*>(work);
  u32* sord = reinterpret_cast<u32*>(skey + n);
  __shared__ uint4 s_red[2][kLobWarps];
  __shared__ u64 s_scan[2][kLobWarps + 1];
  __shared__ int s_nm[2];
  __shared__ unsigned long long s_v;
  int par = 0, spar = 0;

  // padding slots stay inactive in both buffers (the copies never reach them)
  for (int i = cap + threadIdx.x; i < n; i += kLobThreads) {
    stage[i] = 0;
    stage[4 * n + i] = 0;
  }
  if ((int)blockIdx.x < n_books) lob_issue<kVec16>(staged(0), blockIdx.x, cap, active, side, price, qty);
  cp_async_commit();
  int it = 0;
  for (int b = blockIdx.x; b < n_books; b += gridDim.x, ++it) {
    const LobBook d = staged(it & 1);
    const int nxt = b + gridDim.x;
    if (nxt < n_books) lob_issue<kVec16>(staged((it & 1) ^ 1), nxt, cap, active, side, price, qty);
    cp_async_commit();
    cp_async_wait_1();  // this thread's copies of book b have landed
    __syncthreads();    // everyone's have
    const size_t o = (size_t)b * cap;

    // this thread's slots: live flag, side, price, qty
    int32_t px[R];
    u32 qv[R], fl[R];  // fl: bit 0 live, bit 1 ask
    u32 big = 0, cnt = 0, mn = 0xFFFFFFFFu, mx = 0u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = threadIdx.x + r * kLobThreads;
      const bool live = d.act[i] != 0;
      const bool ask = d.sid[i] != 0;
      px[r] = d.px[i];
      qv[r] = (u32)d.qt[i];
      fl[r] = live ? (ask ? 3u : 1u) : 0u;
      if (live) {
        big += qv[r] >= kLobQtyMax;
        cnt += ask ? 0x10000u : 1u;  // bids in the low half, asks in the high half
        if (ask) mn = min(mn, ord32(px[r]));
        else mx = max(mx, ord32(px[r]));
      }
    }
    const Red4 r1 = block_red4(big, cnt, mn, mx, s_red, par);
    const int nbid = (int)(r1.b & 0xFFFFu), nask = (int)(r1.b >> 16);
    const int32_t pmin = (int32_t)(r1.mn ^ 0x80000000u), pmax = (int32_t)(r1.mx ^ 0x80000000u);
    const bool cross = nbid > 0 && nask > 0 && r1.mx >= r1.mn;
    const long long L = cross ? (long long)pmax - (long long)pmin + 1 : 0;
    bool sorted = cross && (r1.a != 0 || L > kLobLevels);
    u32 V = 0;
    int32_t pa = 0, pb = 0;
    u32 Dn = 0, Sp = 0;
    if (cross && !sorted) {
      // level path: share histograms of [pmin, pmax]
      for (int l = threadIdx.x; l < L; l += kLobThreads) {
        hb[l] = 0u;
        ha[l] = 0u;
      }
      if (threadIdx.x == 0) {
        s_nm[0] = 0;
        s_nm[1] = 0;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(fl[r] & 1u)) continue;
        const bool ask = fl[r] & 2u;
        if (ask ? px[r] <= pmax : px[r] >= pmin) atomicAdd((ask ? ha : hb) + (px[r] - pmin), qv[r]);
      }
      __syncthreads();
      // D(l) = bid shares at levels >= l, S(l) = ask shares at levels <= l
      u32 Dl[kLobLevelsPerThread], Sl[kLobLevelsPerThread];
      u32 sb = 0, sa = 0;
      const int l0 = threadIdx.x * kLobLevelsPerThread;
#pragma unroll
      for (int j = 0; j < kLobLevelsPerThread; ++j) {
        Dl[j] = l0 + j < L ? hb[l0 + j] : 0u;
        Sl[j] = l0 + j < L ? ha[l0 + j] : 0u;
        sb += Dl[j];
        sa += Sl[j];
      }
      // packed exclusive scan (both totals stay below 2^31)
      const u64 v = ((u64)sb << 32) | sa;
      u64 incl = v;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const u64 t = __shfl_up_sync(0xFFFFFFFFu, incl, o2);
        if (lane >= o2) incl += t;
      }
      if (lane == 31) s_scan[spar][warp] = incl;
      __syncthreads();
      u64 ex = incl - v, tot = 0;
#pragma unroll
      for (int w = 0; w < kLobWarps; ++w) {
        const u64 t = s_scan[spar][w];
        ex += w < warp ? t : 0ull;
        tot += t;
      }
      spar ^= 1;
      const u32 HB = (u32)(tot >> 32);
      u32 pre_b = (u32)(ex >> 32), pre_a = (u32)ex, best = 0;
#pragma unroll
      for (int j = 0; j < kLobLevelsPerThread; ++j) {
        const u32 hbj = Dl[j];
        pre_a += Sl[j];
        Dl[j] = HB - pre_b;
        Sl[j] = pre_a;
        pre_b += hbj;
        if (l0 + j < L) {
          hb[l0 + j] = Dl[j];
          ha[l0 + j] = Sl[j];
          best = max(best, min(Dl[j], Sl[j]));
        }
      }
      V = block_red4(0u, 0u, 0xFFFFFFFFu, best, s_red, par).mx;
      if (V > 0) {
        // D falls and S rises with the level: count the levels at or above V
        u32 cb = 0, ca = 0;
#pragma unroll
        for (int j = 0; j < kLobLevelsPerThread; ++j) {
          cb += (l0 + j < L) && Dl[j] >= V;
          ca += (l0 + j < L) && Sl[j] >= V;
        }
        const Red4 r3 = block_red4(cb, ca, 0xFFFFFFFFu, 0u, s_red, par);
        const int lb = (int)r3.a - 1, la = (int)L - (int)r3.b;
        pb = pmin + lb;
        pa = pmin + la;
        Dn = lb + 1 < L ? hb[lb + 1] : 0u;  // bid shares priced above pb
        Sp = la > 0 ? ha[la - 1] : 0u;      // ask shares priced below pa
        // the marginal orders, ranked by (time, slot) below
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (!(fl[r] & 1u) || qv[r] == 0) continue;
          const int s = (fl[r] >> 1) & 1;
          if (px[r] != (s ? pa : pb)) continue;
          const int i = threadIdx.x + r * kLobThreads;
          const int k = atomicAdd(&s_nm[s], 1);
          if (k < kLobMarginal) {
            mk[s * kLobMarginal + k] = ((u64)ord32(time[o + i]) << 32) | (u32)i;
            mq[s * kLobMarginal + k] = qv[r];
          }
        }
        __syncthreads();
        sorted = s_nm[0] > kLobMarginal || s_nm[1] > kLobMarginal;
      }
    }
    if (sorted) {
      lob_match_sorted(d, n, b, cap, nbid, nask, active, qty, time, out_volume, out_price, skey, sord,
                       s_scan[0], &s_v);
    } else {
      if (threadIdx.x == 0) {
        out_volume[b] = (long long)V;
        out_price[b] = V > 0 ? pa : -1;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(fl[r] & 1u)) continue;
        const int i = threadIdx.x + r * kLobThreads;
        const bool ask = fl[r] & 2u;
        const u32 q = qv[r];
        u32 fill = 0;
        if (V > 0 && q > 0) {
          const int32_t edge = ask ? pa : pb;
          const bool whole = ask ? px[r] < edge : px[r] > edge;
          if (whole) {
            fill = q;
          } else if (px[r] == edge) {
            const int s = ask ? 1 : 0;
            const u64 mine = ((u64)ord32(time[o + i]) << 32) | (u32)i;
            u32 before = ask ? Sp : Dn;
            const int m = s_nm[s];
            for (int e = 0; e < m; ++e) before += mk[s * kLobMarginal + e] < mine ? mq[s * kLobMarginal + e] : 0u;
            fill = V > before ? min(V - before, q) : 0u;
          }
        }
        if (fill || q == 0) {
          qty[o + i] = (int32_t)(q - fill);
          if (q == fill) active[o + i] = 0;
        }
      }
    }
    __syncthreads();  // the staging buffer and work area are reused
  }
  cp_async_wait_0();
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

static size_t lob_smem_bytes(int n) {
  return 8 * (size_t)n * sizeof(int32_t) + std::max(kLobLevelBytes, (size_t)n * (sizeof(u64) + sizeof(u32)));
}

template <int R, bool kVec16>
static abm_status lob_launch(int n_books, int cap, int32_t* active, const int32_t* side, const int32_t* price,
                             int32_t* qty, const int32_t* time, long long* vol, int32_t* px, cudaStream_t st) {
  static int grid_per_sm = 0;
  const size_t smem = lob_smem_bytes(R * kLobThreads);
  if (!grid_per_sm) {
    ABM_CUDA_TRY(cudaFuncSetAttribute(k_lob_match<R, kVec16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    int occ = 0;
    ABM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lob_match<R, kVec16>, kLobThreads, smem));
    grid_per_sm = std::max(occ, 1);
  }
  const int grid = (int)std::min<long long>(n_books, (long long)num_sms() * grid_per_sm);
  k_lob_match<R, kVec16><<<grid, kLobThreads, smem, st>>>(n_books, cap, active, side, price, qty, time, vol, px);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

template <int R>
static abm_status lob_launch_r(bool vec16, int n_books, int cap, int32_t* active, const int32_t* side,
                               const int32_t* price, int32_t* qty, const int32_t* time, long long* vol, int32_t* px,
                               cudaStream_t st) {
  return vec16 ? lob_launch<R, true>(n_books, cap, active, side, price, qty, time, vol, px, st)
               : lob_launch<R, false>(n_books, cap, active, side, price, qty, time, vol, px, st);
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
  switch (lob_pad(cap) / kLobThreads) {
    case 1: return lob_launch_r<1>(vec16, n_books, cap, active, side, price, qty, time, vol, out_price, st);
    case 2: return lob_launch_r<2>(vec16, n_books, cap, active, side, price, qty, time, vol, out_price, st);
    case 4: return lob_launch_r<4>(vec16, n_books, cap, active, side, price, qty, time, vol, out_price, st);
    default: return lob_launch_r<8>(vec16, n_books, cap, active, side, price, qty, time, vol, out_price, st);
  }
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
