// Batched predation: thousands of independent wolf-sheep-grass models of
// uneven size in one persistent launch (ABMax vectorises many models with
// vmap over Sets, Section 2 and Table 2; here each model gets a CTA).
//
// A CTA takes the next model from a ticket (models ordered largest first),
// runs the requested steps of it -- every phase separated by __syncthreads,
// compaction by block scans -- and takes the next. Each model has its own
// capacity slabs at offsets in shared arrays. The sweep over a model's slab is
// either its full capacity (the static shapes of the paper: placeholders are
// visited every step) or its extent (highest slot ever used + 1); both give
// the same results, and the capacity sweep is what a tighter capacity speeds
// up. A CTA never waits for another CTA.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "pred_rules.cuh"

namespace abm {

constexpr int kBatchLiveWordsMax = 1 << 15;  // 128 KiB: live-flag bitmask of up to 1Mi slots per CTA

struct BModel {
  int side, ncells;
  u32 seed, model;
  int prm[8];
  int cap[2];       // slots per species (capacity)
  int cap_pad[2];   // allocated slots (multiple of 16)
  int n0[2];
  long long oa[2];  // slot offset of each species' slab
  long long oc;     // cell offset
};

struct BCtr {
  int n_active[2], next_id[2], hw[2], overflow[2], extent[2], step, pad;
  long long agent_steps;  // sum over steps run of the live agents at step start
};

struct BatchDev {
  const BModel* models;
  BCtr* ctr;
  int nmodels;
  int32_t* active[2];
  int4* agent[2];
  int32_t* plist[2];
  int32_t* flist[2];
  int32_t* regrow;
  u64* gclaim;
  u64* victim;
  u64* wclaim;
  const int32_t* order;
  u32* ctrl;  // [0] model ticket, [1] CTAs finished, [2] epoch
  int* err;
};

// the model a CTA is working on, in shared memory
struct MCtx {
  BModel m;
  int n_active[2], next_id[2], hw[2], overflow[2], extent[2], step;
  long long agent_steps;
  int n_start[2], P[2], F[2], starved[2], eaten, grass;
};

// Models per CTA: a CTA of N threads runs G models at once, each on a group
// of T = N / G threads (thread gt of group g) with its own barrier -- the CTA
// barrier when G = 1, else the named barrier 1 + g -- and its own shared arrays.
template <int G>
__device__ __forceinline__ void gsync(int g, int nthreads) {
  if (G == 1) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(nthreads) : "memory");
  }
}

// gsync that also returns whether pred holds in any thread of the group
template <int G>
__device__ __forceinline__ int gsync_or(int g, int nthreads, int pred) {
  if (G == 1) return __syncthreads_or(pred);
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.s32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(pred), "r"(1 + g), "r"(nthreads)
      : "memory");
  return r;
}

// exclusive scan of two counts (packed in one u64) over a group of T threads
template <int T, int G>
__device__ __forceinline__ void group_scan2(int g, int gt, u32 a, u32 b, u32& ex_a, u32& ex_b, u32& tot_a,
                                            u32& tot_b, u64* s_warp /* [T / 32 + 1] */) {
  constexpr int W = T / 32;
  const int lane = gt & 31, warp = gt >> 5;
  const u64 v = ((u64)a << 32) | b;
  u64 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) s_warp[warp] = incl;
  gsync<G>(g, T);
  if (warp == 0) {
    const u64 w = lane < W ? s_warp[lane] : 0ull;
    u64 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 x = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += x;
    }
    if (lane < W) s_warp[lane] = wi - w;
    if (lane == W - 1) s_warp[W] = wi;
  }
  gsync<G>(g, T);
  const u64 ex = s_warp[warp] + incl - v;
  const u64 tot = s_warp[W];
  ex_a = (u32)(ex >> 32);
  ex_b = (u32)ex;
  tot_a = (u32)(tot >> 32);
  tot_b = (u32)tot;
}

// Live agents of a chunk of A * T slots (A = slots per thread, 8, 16 or 32),
// listed in shared memory (offsets within the chunk, in the order of the
// threads' masks) so that all T threads share the work whatever the chunk's
// density. m = the thread's A-bit live mask; returns the list's length.
template <int T, int G>
__device__ __forceinline__ int chunk_list(int g, int gt, u32 m, int first_off, int stride_off, unsigned short* s_list, u64* s_warp) {
  u32 ex, ex2, tot, tot2;
  group_scan2<T, G>(g, gt, (u32)__popc(m), 0u, ex, ex2, tot, tot2, s_warp);
  u32 pos = ex;
  while (m) {
    const int j = __ffs(m) - 1;
    m &= m - 1;
    s_list[pos++] = (unsigned short)(first_off + j * stride_off);
  }
  gsync<G>(g, T);
  return (int)tot;
}

template <int T, int G>
__device__ __forceinline__ void move_agent(const BatchDev& b, const MCtx& c, int S, int t, int slot, int4 a) {
  int4* ag = b.agent[S] + c.m.oa[S];
  u64* victim = b.victim + c.m.oc;
  if (!in_range(a.x, c.m.ncells, b.err)) return;  // check builds: a cell outside the model's lattice
  if (S == 0) victim[a.x] = kNoKey;
  const u32 dir = draw(c.m.seed, c.m.model, (u32)t, (u32)slot, ABM_P_MOVE, (u32)S) >> 29;
  const int cell = step_cell(a.x, c.m.side, dir);
  a.x = cell;
  a.y -= c.m.prm[PRM_SHEEP_METAB + S];
  a.w += 1;
  ag[slot] = a;
  if (S == 0) {
    if (b.regrow[c.m.oc + cell] <= t)
      atomicMin(&b.gclaim[c.m.oc + cell], claim_key(draw(c.m.seed, c.m.model, (u32)t, (u32)slot, ABM_P_PRIO, 0u), slot));
  } else {
    if (victim[cell] != kNoKey)
      atomicMin(&b.wclaim[c.m.oc + cell], claim_key(draw(c.m.seed, c.m.model, (u32)t, (u32)slot, ABM_P_PRIO, 1u), slot));
  }
}

template <int T, int G, int A>
__device__ __forceinline__ void b_move(int g, int gt, const BatchDev& b, MCtx& c, int S, int sweep, int t, unsigned short* s_list,
                                       u64* s_warp, u32* s_live, int live_words) {
  static_assert(A == 8 || A == 16 || A == 32, "slots per thread per chunk: 8, 16 or 32");
  const int32_t* act = b.active[S] + c.m.oa[S];
  const int4* ag = b.agent[S] + c.m.oa[S];
  // the sweep's live flags also go into a shared-memory bitmask (when it fits)
  // that the scan of the same species reads instead of the flags: nothing
  // changes this species' flags between its move and its scan
  const bool keep = sweep <= 32 * live_words;
  // per chunk: A / 4 128-bit loads of live flags per thread (int4 q0 + u*T),
  // the live slots listed, then two agents in flight per thread (copying the
  // next chunk's flags into shared memory ahead, with cp.async, measured slower
  // overall: faster at full capacity, slower with extent sweeps)
  for (int c0 = 0; c0 < sweep; c0 += A * T) {
    const int q0 = (c0 >> 2) + gt;
    const int nq = (sweep + 3) >> 2;
    u32 m = 0;
#pragma unroll
    for (int u = 0; u < A / 4; ++u) {
      const int q = q0 + u * T;
      const int4 a = q < nq ? reinterpret_cast<const int4*>(act)[q] : make_int4(0, 0, 0, 0);
      m |= ((u32)(a.x != 0) | ((u32)(a.y != 0) << 1) | ((u32)(a.z != 0) << 2) | ((u32)(a.w != 0) << 3)) << (4 * u);
    }
    // bit 4u + j of m is slot 4 (q0 + u T) + j = c0 + 4 tid + 4 u T + j
    if (keep) {
      // the nibbles of 8 neighbouring threads make one bitmask word (slots 4 (q0 + u T) .. + 32)
#pragma unroll
      for (int u = 0; u < A / 4; ++u) {
        u32 v = ((m >> (4 * u)) & 0xFu) << (4 * (gt & 7));
        v |= __shfl_xor_sync(0xFFFFFFFFu, v, 1);
        v |= __shfl_xor_sync(0xFFFFFFFFu, v, 2);
        v |= __shfl_xor_sync(0xFFFFFFFFu, v, 4);
        const int wd = (c0 + 4 * (gt + u * T)) >> 5;
        if ((gt & 7) == 0 && wd < live_words) s_live[wd] = v;
      }
    }
    if (!gsync_or<G>(g, T, m != 0)) continue;  // no live agent in the chunk
    u32 ex, ex2, tot, tot2;
    group_scan2<T, G>(g, gt, (u32)__popc(m), 0u, ex, ex2, tot, tot2, s_warp);
    {
      u32 pos = ex, mb = m;
      while (mb) {
        const int bit = __ffs(mb) - 1;
        mb &= mb - 1;
        s_list[pos++] = (unsigned short)(4 * gt + 4 * (bit >> 2) * T + (bit & 3));
      }
    }
    gsync<G>(g, T);
    for (int e = gt; e < (int)tot; e += 2 * T) {
      const int sa = c0 + s_list[e];
      const int sb = e + T < (int)tot ? c0 + s_list[e + T] : -1;
      const int4 aa = ag[sa];
      int4 ab = make_int4(0, 0, 0, 0);
      if (sb >= 0) ab = ag[sb];
      move_agent<T, G>(b, c, S, t, sa, aa);
      if (sb >= 0) move_agent<T, G>(b, c, S, t, sb, ab);
    }
    gsync<G>(g, T);  // the list is rewritten by the next chunk
  }
}

// eat (claim winners), select parents or die; returns bit 0 = parent, bit 1 =
// died, bit 2 = ate
template <int T, int G>
__device__ __forceinline__ u32 scan_agent(const BatchDev& b, const MCtx& c, int S, int t, int slot) {
  int32_t* act = b.active[S] + c.m.oa[S];
  int4* ag = b.agent[S] + c.m.oa[S];
  u64* claim = (S == 0 ? b.gclaim : b.wclaim) + c.m.oc;
  u64* victim = b.victim + c.m.oc;
  int4 a = ag[slot];
  const int cell = a.x;
  if (!in_range(cell, c.m.ncells, b.err)) return 0u;  // check builds only
  const u64 cl = claim[cell];
  u32 r = 0;
  if (cl != kNoKey && (u32)cl == (u32)slot) {
    a.y += c.m.prm[S];
    ag[slot].y = a.y;
    claim[cell] = kNoKey;
    r |= 4u;
    if (S == 0) {
      b.regrow[c.m.oc + cell] = t + c.m.prm[PRM_REGROWTH];
    } else {
      const u64 v = victim[cell];
      if (in_range((u32)v, c.m.cap[0], b.err)) b.active[0][c.m.oa[0] + (u32)v] = 0;
      victim[cell] = kNoKey;
    }
  }
  if (a.y < 0) {
    act[slot] = 0;
    r |= 2u;
  } else {
    if (draw(c.m.seed, c.m.model, (u32)t, (u32)slot, ABM_P_REPRO, (u32)S) < (u32)c.m.prm[PRM_SHEEP_T + S]) r |= 1u;
    if (S == 0)
      atomicMin(&victim[cell], claim_key(draw(c.m.seed, c.m.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u), slot));
  }
  return r;
}

// eat (claim winners), select parents, kill the starving, compact the free
// slots and the parents (ranks by block scans, chunk by chunk). Thread i holds
// the A contiguous slots A i.. of a chunk for the ranks; the live agents of
// the chunk are listed and shared by all threads.
template <int T, int G, int A>
__device__ __forceinline__ void b_scan(int g, int gt, const BatchDev& b, MCtx& c, int S, int sweep, int t, u64* s_warp,
                                       int* s_acc, unsigned short* s_list, u32* s_par, const u32* s_live,
                                       int live_words) {
  const int32_t* act = b.active[S] + c.m.oa[S];
  int32_t* plist = b.plist[S] + c.m.oa[S];
  int32_t* flist = b.flist[S] + c.m.oa[S];
  const int bound = c.n_active[S];
  const bool kept = sweep <= 32 * live_words;  // the move left this sweep's flags in s_live
  int starved = 0, won = 0;
  u32 pf = 0, pp = 0;
  constexpr u32 kMaskA = A == 32 ? 0xFFFFFFFFu : (1u << (A & 31)) - 1u;
  for (int c0 = 0; c0 < sweep; c0 += A * T) {
    const int base = c0 + A * gt;
    u32 m = 0, valid = 0;
    if (kept) {
      if (base < sweep) m = (s_live[base >> 5] >> (base & 31)) & kMaskA;
    } else {
#pragma unroll
      for (int v = 0; v < A / 4; ++v) {
        int4 q = make_int4(0, 0, 0, 0);
        if (base + 4 * v < sweep) q = reinterpret_cast<const int4*>(act)[(base >> 2) + v];
        m |= ((u32)(q.x != 0) | ((u32)(q.y != 0) << 1) | ((u32)(q.z != 0) << 2) | ((u32)(q.w != 0) << 3)) << (4 * v);
      }
    }
#pragma unroll
    for (int j = 0; j < A; ++j) valid |= (u32)(base + j < sweep) << j;
    m &= valid;
    const u32 fr = ~m & valid;
    // a chunk without live agents whose free slots all rank past the free-list
    // bound only adds to the free count
    if ((int)pf >= bound && !gsync_or<G>(g, T, m != 0)) {
      pf += (u32)min(A * T, sweep - c0);
      continue;
    }
    const int tot = chunk_list<T, G>(g, gt, m, A * gt, 1, s_list, s_warp);
    for (int e = gt; e < tot; e += T) {
      const int off = s_list[e];
      const u32 r = scan_agent<T, G>(b, c, S, t, c0 + off);
      if (r & 1u) atomicOr(&s_par[off >> 5], 1u << (off & 31));
      starved += (r >> 1) & 1u;
      won += (r >> 2) & 1u;
    }
    gsync<G>(g, T);
    u32 par = (s_par[(A * gt) >> 5] >> ((A * gt) & 31)) & kMaskA;
    u32 ex_f, ex_p, tot_f, tot_p;
    group_scan2<T, G>(g, gt, __popc(fr), __popc(par), ex_f, ex_p, tot_f, tot_p, s_warp);
    if (((A * gt) & 31) == 0) s_par[(A * gt) >> 5] = 0u;  // the word's parts were read before the scan's barrier
    u32 rf = pf + ex_f, rp = pp + ex_p;
    u32 frm = fr;
    while (frm) {
      const int j = __ffs(frm) - 1;
      frm &= frm - 1;
      if ((int)rf < bound && in_range(rf, c.m.cap_pad[S], b.err)) flist[rf] = base + j;
      ++rf;
    }
    while (par) {
      const int j = __ffs(par) - 1;
      par &= par - 1;
      if (in_range(rp, c.m.cap_pad[S], b.err)) plist[rp] = base + j;
      ++rp;
    }
    pf += tot_f;
    pp += tot_p;
    gsync<G>(g, T);  // the list and the parent words are rewritten by the next chunk
  }
  // per-CTA sums of the winners and the starved
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    starved += __shfl_xor_sync(0xFFFFFFFFu, starved, o);
    won += __shfl_xor_sync(0xFFFFFFFFu, won, o);
  }
  if ((gt & 31) == 0) {
    if (starved) atomicAdd(&s_acc[0], starved);
    if (won) atomicAdd(&s_acc[1], won);
  }
  if (gt == 0) {
    c.P[S] = (int)pp;
    c.F[S] = (int)pf;
  }
}

// children: the i-th parent (ascending slot) fills the i-th free slot
template <int T, int G>
__device__ __forceinline__ void b_births(int g, int gt, const BatchDev& b, MCtx& c, int S, int r, int t) {
  int32_t* act = b.active[S] + c.m.oa[S];
  int4* ag = b.agent[S] + c.m.oa[S];
  const int32_t* plist = b.plist[S] + c.m.oa[S];
  const int32_t* flist = b.flist[S] + c.m.oa[S];
  const int Fin = c.F[S], ext = c.extent[S];
  const int id0 = c.next_id[S];
  for (int i = gt; i < r; i += T) {
    const int p = plist[i];
    const int slot = i < Fin ? flist[i] : ext + (i - Fin);
    if (!in_range(p, c.m.cap[S], b.err) || !in_range(slot, c.m.cap[S], b.err)) continue;
    const int4 pa = ag[p];
    const int half = pa.y >> 1;
    ag[p].y = pa.y - half;
    ag[slot] = make_int4(pa.x, half, (int)((u32)id0 + (u32)i), 0);
    act[slot] = 1;
    if (S == 0)
      atomicMin(&b.victim[c.m.oc + pa.x], claim_key(draw(c.m.seed, c.m.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u), slot));
  }
}

// after a species' births (thread 0): its counters. avail = free slots in
// the whole capacity (both sweeps count them the same way).
__device__ __forceinline__ void b_count_births(const BatchDev& b, MCtx& c, int S, int r, int starved, int avail) {
  const int Fin = c.F[S], ext = c.extent[S];
  const int n_after = c.n_start[S] + r;
  if (n_after > c.hw[S]) c.hw[S] = n_after;
  c.n_active[S] = n_after - starved;
  c.next_id[S] += r;
  if (r > Fin) {
    c.extent[S] = ext + (r - Fin);
  } else if (r > 0) {
    const int last = b.flist[S][c.m.oa[S] + r - 1] + 1;  // children fill free slots below the extent
    if (last > c.extent[S]) c.extent[S] = last;
  }
  if (c.P[S] > avail) c.overflow[S] = 1;
}

// N threads per CTA, G models per CTA (groups of N / G threads), A slots per
// thread in a chunk of the sweeps
template <int N, int G, int A>
__global__ void __launch_bounds__(N, (1024 / N > 0 ? 1024 / N : 1)) k_batch_run(BatchDev b, int nsteps, int sweep_extent,
                                                                        int live_words) {
  constexpr int T = N / G;
  extern __shared__ u32 s_live_all[];  // [G][live_words]: one species' live flags per group, move -> scan
  __shared__ MCtx s_c[G];
  __shared__ u64 s_warp_all[G][T / 32 + 1];
  __shared__ int s_acc_all[G][4];
  __shared__ int s_idx_all[G];
  __shared__ unsigned short s_list_all[G][A * T];  // live agents of a chunk
  __shared__ u32 s_par_all[G][A * T / 32];         // parent bits of a chunk
  const int g = (int)threadIdx.x / T, gt = (int)threadIdx.x % T;
  MCtx& c = s_c[g];
  u64* s_warp = s_warp_all[g];
  int* s_acc = s_acc_all[g];
  int& s_idx = s_idx_all[g];
  unsigned short* s_list = s_list_all[g];
  u32* s_par = s_par_all[g];
  u32* s_live = s_live_all + (size_t)g * live_words;
  if (gt < A * T / 32) s_par[gt] = 0u;
  while (true) {
    gsync<G>(g, T);
    if (gt == 0) s_idx = (int)atomicAdd(&b.ctrl[0], 1u);
    gsync<G>(g, T);
    const int idx = s_idx;
    if (idx >= b.nmodels) break;
    const int mi = b.order[idx];
    if (gt == 0) {
      c.m = b.models[mi];
      const BCtr k = b.ctr[mi];
      for (int s = 0; s < 2; ++s) {
        c.n_active[s] = k.n_active[s];
        c.next_id[s] = k.next_id[s];
        c.hw[s] = k.hw[s];
        c.overflow[s] = k.overflow[s];
        c.extent[s] = k.extent[s];
      }
      c.step = k.step;
      c.agent_steps = k.agent_steps;
    }
    gsync<G>(g, T);
    for (int it = 0; it < nsteps; ++it) {
      const int t = c.step;
      if (gt == 0) {
        c.n_start[0] = c.n_active[0];
        c.n_start[1] = c.n_active[1];
        c.agent_steps += c.n_active[0] + c.n_active[1];
        s_acc[0] = s_acc[1] = s_acc[2] = s_acc[3] = 0;
      }
      const int sw0 = sweep_extent ? c.extent[0] : c.m.cap[0];
      gsync<G>(g, T);
      // sheep: move + grass claims; eat, select, die, compact
      b_move<T, G, A>(g, gt, b, c, 0, sw0, t, s_list, s_warp, s_live, live_words);
      gsync<G>(g, T);
      b_scan<T, G, A>(g, gt, b, c, 0, sw0, t, s_warp, s_acc, s_list, s_par, s_live, live_words);
      gsync<G>(g, T);
      const int avail0 = c.F[0] + (sweep_extent ? c.m.cap[0] - c.extent[0] : 0);
      const int r0 = min(c.P[0], avail0);
      const int sw1 = sweep_extent ? c.extent[1] : c.m.cap[1];
      // sheep births, concurrently the wolves' move + victim claims (a wolf's
      // claim only needs the cell to hold a live sheep; every newborn lamb
      // sits with its live parent)
      b_births<T, G>(g, gt, b, c, 0, r0, t);
      b_move<T, G, A>(g, gt, b, c, 1, sw1, t, s_list, s_warp, s_live, live_words);
      gsync<G>(g, T);
      if (gt == 0) {
        b_count_births(b, c, 0, r0, s_acc[0], avail0);
        c.starved[0] = s_acc[0];
        c.grass = s_acc[1];
        s_acc[0] = s_acc[1] = 0;
      }
      gsync<G>(g, T);
      b_scan<T, G, A>(g, gt, b, c, 1, sw1, t, s_warp, s_acc, s_list, s_par, s_live, live_words);
      gsync<G>(g, T);
      const int avail1 = c.F[1] + (sweep_extent ? c.m.cap[1] - c.extent[1] : 0);
      const int r1 = min(c.P[1], avail1);
      b_births<T, G>(g, gt, b, c, 1, r1, t);
      gsync<G>(g, T);
      if (gt == 0) {
        b_count_births(b, c, 1, r1, s_acc[0], avail1);
        c.starved[1] = s_acc[0];
        c.eaten = s_acc[1];
        c.n_active[0] -= s_acc[1];
        c.step = t + 1;
      }
      gsync<G>(g, T);
    }
    if (gt == 0) {
      BCtr k;
      for (int s = 0; s < 2; ++s) {
        k.n_active[s] = c.n_active[s];
        k.next_id[s] = c.next_id[s];
        k.hw[s] = c.hw[s];
        k.overflow[s] = c.overflow[s];
        k.extent[s] = c.extent[s];
      }
      k.step = c.step;
      k.pad = 0;
      k.agent_steps = c.agent_steps;
      b.ctr[mi] = k;
    }
  }
  last_cta_out(b.ctrl);  // its barrier waits for every group of the CTA
}

// one CTA per model: initial agents, grass, empty claim tables, counters
__global__ void k_batch_init(BatchDev b) {
  const int mi = blockIdx.x;
  const BModel m = b.models[mi];
  for (int s = 0; s < 2; ++s) {
    const int gain = m.prm[s];
    for (int k = threadIdx.x; k < m.cap_pad[s]; k += blockDim.x) {
      const long long g = m.oa[s] + k;
      if (k < m.n0[s]) {
        const uint4 u = draw4(m.seed, m.model, ABM_INIT_STEP, (u32)k, ABM_P_INIT_AGENT, (u32)s);
        b.agent[s][g] = make_int4(uniform_below(u.x, m.ncells), uniform_below(u.y, 2 * gain), k, 0);
        b.active[s][g] = 1;
      } else {
        // check builds: canaries in the fields past the capacity (the flags stay 0)
        b.agent[s][g] = (kCheck && k >= m.cap[s]) ? make_int4(kCanary, kCanary, kCanary, kCanary) : make_int4(0, 0, 0, 0);
        b.active[s][g] = 0;
      }
    }
  }
  for (int cidx = threadIdx.x; cidx < m.ncells; cidx += blockDim.x) {
    const uint4 u = draw4(m.seed, m.model, ABM_INIT_STEP, (u32)cidx, ABM_P_GRASS_INIT, 2u);
    const bool grown = u.x < (u32)m.prm[PRM_GRASS_T];
    const int wait = uniform_below(u.y, m.prm[PRM_REGROWTH]);
    const long long g = m.oc + cidx;
    b.regrow[g] = grown ? 0 : max(wait, 1);
    b.gclaim[g] = kNoKey;
    b.victim[g] = kNoKey;
    b.wclaim[g] = kNoKey;
  }
  if (threadIdx.x == 0) {
    BCtr k;
    std::memset(&k, 0, sizeof(k));
    for (int s = 0; s < 2; ++s) {
      k.n_active[s] = m.n0[s];
      k.next_id[s] = m.n0[s];
      k.hw[s] = m.n0[s];
      k.extent[s] = m.n0[s];
    }
    b.ctr[mi] = k;
  }
}

__global__ void k_batch_grass(BatchDev b, int mi, int which, int32_t* dst) {
  const BModel m = b.models[mi];
  const int T = b.ctr[mi].step;
  for (int cidx = blockIdx.x * blockDim.x + threadIdx.x; cidx < m.ncells; cidx += gridDim.x * blockDim.x) {
    const int r = b.regrow[m.oc + cidx];
    dst[cidx] = which == 0 ? (r <= T ? 1 : 0) : (r <= T ? 0 : r - T);
  }
}

// list of the models whose births were ever truncated (device-side, one CTA)
__global__ void k_batch_overflowed(BatchDev b, int32_t* list, int32_t* count) {
  __shared__ int n;
  if (threadIdx.x == 0) n = 0;
  __syncthreads();
  for (int base = 0; base < b.nmodels; base += blockDim.x) {
    const int m = base + threadIdx.x;
    const bool ov = m < b.nmodels && (b.ctr[m].overflow[0] | b.ctr[m].overflow[1]);
    const u32 bal = __ballot_sync(0xFFFFFFFFu, ov);
    __shared__ int warp_base[32];
    if ((threadIdx.x & 31) == 0) warp_base[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = n;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const int x = warp_base[w];
        warp_base[w] = acc;
        acc += x;
      }
      n = acc;
    }
    __syncthreads();
    if (ov) list[warp_base[threadIdx.x >> 5] + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = m;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = n;
}

// check builds: one CTA per model verifies the padding past each capacity
__global__ void k_batch_canaries(BatchDev b) {
  const BModel m = b.models[blockIdx.x];
  bool bad = false;
  for (int s = 0; s < 2; ++s)
    for (int k = m.cap[s] + (int)threadIdx.x; k < m.cap_pad[s]; k += blockDim.x) {
      const int4 a = b.agent[s][m.oa[s] + k];
      bad |= b.active[s][m.oa[s] + k] != 0 || a.x != kCanary || a.y != kCanary || a.z != kCanary || a.w != kCanary;
    }
  if (bad) atomicCAS(b.err, 0, kErrCheck);
}

// order-independent digest of one model's observable state (digest_* terms)
__global__ void k_batch_digest(BatchDev b, u64* out) {
  __shared__ u64 s[32];
  const int mi = blockIdx.x;
  const BModel m = b.models[mi];
  const BCtr k = b.ctr[mi];
  u64 h = 0;
  for (int sp = 0; sp < 2; ++sp) {
    for (int i = threadIdx.x; i < k.extent[sp]; i += blockDim.x) {
      if (!b.active[sp][m.oa[sp] + i]) continue;
      h += digest_agent(sp, i, b.agent[sp][m.oa[sp] + i]);
    }
  }
  for (int c = threadIdx.x; c < m.ncells; c += blockDim.x) h += digest_cell(c, b.regrow[m.oc + c], k.step);
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = h;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    out[mi] = t + digest_counters(k.n_active, k.next_id, k.hw);
  }
}

}  // namespace abm

// ============================================================================
using namespace abm;

struct abm_batch {
  BatchDev d;
  BModel* models_dev;
  std::vector<BModel> models;
  long long slots[2], cells;
  int threads, ctas_per_sm, steps_per_launch, models_per_cta, agents_per_thread;
  // fixed-capacity rerun of the models whose slabs overflowed (abm_batch_rerun_overflowed)
  abm_batch* rerun;
  std::vector<int> rerun_of;  // per model: its index in `rerun`, or -1
  int32_t* rerun_idx;         // device [rerun->n]: model index in this batch of rerun model j
  u64* rerun_dig;             // device [rerun->n]: digests of the rerun models
};

// digest j of the rerun batch -> entry idx[j] of this batch's digests
__global__ void k_scatter_u64(const u64* src, const int32_t* idx, int n, u64* dst) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) dst[idx[j]] = src[j];
}

static void batch_free(abm_batch* b) {
  for (int s = 0; s < 2; ++s) {
    cudaFree(b->d.active[s]);
    cudaFree(b->d.agent[s]);
    cudaFree(b->d.plist[s]);
    cudaFree(b->d.flist[s]);
  }
  cudaFree(b->d.regrow);
  cudaFree(b->d.gclaim);
  cudaFree(b->d.victim);
  cudaFree(b->d.wclaim);
  cudaFree(b->d.ctr);
  cudaFree(b->models_dev);
  cudaFree((void*)b->d.order);
  cudaFree(b->d.ctrl);
  cudaFree(b->d.err);
  if (b->rerun) batch_free(b->rerun);
  cudaFree(b->rerun_idx);
  cudaFree(b->rerun_dig);
  delete b;
}

extern "C" abm_status abm_batch_destroy(abm_batch* b) {
  if (!b) return ABM_ERR_ARG;
  batch_free(b);
  return ABM_OK;
}

extern "C" abm_status abm_batch_create(const abm_batch_model* models, int32_t n, void* stream, abm_batch** out) {
  if (!models || n < 1 || !out) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  abm_batch* b = new (std::nothrow) abm_batch();
  if (!b) return ABM_ERR_OOM;
  b->models.resize((size_t)n);
  long long oa[2] = {0, 0}, oc = 0;
  for (int i = 0; i < n; ++i) {
    const abm_batch_model& in = models[i];
    if (in.side < 1 || in.side > 46340 || in.params[4] < 1) {
      delete b;
      return ABM_ERR_ARG;
    }
    BModel& m = b->models[(size_t)i];
    std::memset(&m, 0, sizeof(m));
    m.side = in.side;
    m.ncells = in.side * in.side;
    m.seed = in.seed;
    m.model = in.model;
    std::memcpy(m.prm, in.params, sizeof(m.prm));
    for (int s = 0; s < 2; ++s) {
      if (in.cap[s] < 1 || in.cap[s] > (1 << 28) - 1 || in.n0[s] < 0 || in.n0[s] > in.cap[s] || in.params[s] < 0 ||
          in.params[5 + s] < 0) {
        delete b;
        return ABM_ERR_ARG;
      }
      m.cap[s] = in.cap[s];
      m.cap_pad[s] = (in.cap[s] + 15) & ~15;
      m.n0[s] = in.n0[s];
      m.oa[s] = oa[s];
      oa[s] += m.cap_pad[s];
    }
    m.oc = oc;
    oc += m.ncells;
  }
  b->slots[0] = oa[0];
  b->slots[1] = oa[1];
  b->cells = oc;
  BatchDev& d = b->d;
  d.nmodels = n;
  bool ok = true;
  for (int s = 0; s < 2; ++s) {
    ok = ok && cudaMalloc(&d.active[s], sizeof(int32_t) * (size_t)oa[s]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.agent[s], sizeof(int4) * (size_t)oa[s]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.plist[s], sizeof(int32_t) * (size_t)oa[s]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.flist[s], sizeof(int32_t) * (size_t)oa[s]) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&d.regrow, sizeof(int32_t) * (size_t)oc) == cudaSuccess;
  ok = ok && cudaMalloc(&d.gclaim, sizeof(u64) * (size_t)oc) == cudaSuccess;
  ok = ok && cudaMalloc(&d.victim, sizeof(u64) * (size_t)oc) == cudaSuccess;
  ok = ok && cudaMalloc(&d.wclaim, sizeof(u64) * (size_t)oc) == cudaSuccess;
  ok = ok && cudaMalloc(&d.ctr, sizeof(BCtr) * (size_t)n) == cudaSuccess;
  ok = ok && cudaMalloc(&b->models_dev, sizeof(BModel) * (size_t)n) == cudaSuccess;
  int32_t* order = nullptr;
  ok = ok && cudaMalloc(&order, sizeof(int32_t) * (size_t)n) == cudaSuccess;
  d.order = order;
  ok = ok && cudaMalloc(&d.ctrl, sizeof(u32) * 4) == cudaSuccess;
  ok = ok && cudaMalloc(&d.err, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    batch_free(b);
    return ABM_ERR_OOM;
  }
  d.models = b->models_dev;
  // largest models first: they bound the tail of the persistent launch
  std::vector<int32_t> ord((size_t)n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    const BModel &a = b->models[(size_t)x], &c = b->models[(size_t)y];
    return (long long)a.cap[0] + a.cap[1] + a.ncells > (long long)c.cap[0] + c.cap[1] + c.ncells;
  });
  if (cudaMemcpyAsync(b->models_dev, b->models.data(), sizeof(BModel) * (size_t)n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(order, ord.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(d.ctrl, 0, sizeof(u32) * 4, st) != cudaSuccess ||
      cudaMemsetAsync(d.err, 0, sizeof(int), st) != cudaSuccess) {
    batch_free(b);
    return ABM_ERR_CUDA;
  }
  k_batch_init<<<n, 256, 0, st>>>(d);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    batch_free(b);
    return ABM_ERR_CUDA;
  }
  b->threads = 256;
  b->ctas_per_sm = 4;
  b->steps_per_launch = 1 << 30;
  b->models_per_cta = 1;
  b->agents_per_thread = 16;
  *out = b;
  return ABM_OK;
}

extern "C" abm_status abm_batch_tune(abm_batch* b, int32_t threads, int32_t ctas_per_sm, int32_t steps_per_launch) {
  if (!b || (threads != 128 && threads != 256 && threads != 512 && threads != 1024) || ctas_per_sm < 1 ||
      threads * ctas_per_sm > 2048 || steps_per_launch < 1)
    return ABM_ERR_ARG;
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  b->steps_per_launch = steps_per_launch;
  if (threads / b->models_per_cta < 128) b->models_per_cta = 1;
  if (threads > 512 && b->agents_per_thread == 32) b->agents_per_thread = 16;
  return ABM_OK;
}

// One launch of the run kernel with N threads and G models per CTA. Its
// dynamic shared memory (G live-flag bitmasks) is set per device, raised when
// a batch needs more; the bitmasks shrink (their models then read their flags
// twice) when the CTA's shared memory is short.
template <int N, int GG, int A>
static abm_status batch_launch(const BatchDev& d, int grid, int nsteps, int ext, int live_words, cudaStream_t st) {
  static std::atomic<int> limit_set[64];
  static std::atomic<int> max_dyn[64];
  int dev = 0;
  ABM_CUDA_TRY(cudaGetDevice(&dev));
  const bool cache = dev >= 0 && dev < 64;
  int maxd = cache ? max_dyn[dev].load(std::memory_order_relaxed) : 0;
  if (maxd == 0) {
    int optin = 0;
    cudaFuncAttributes fa;
    ABM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    ABM_CUDA_TRY(cudaFuncGetAttributes(&fa, k_batch_run<N, GG, A>));
    maxd = std::max(0, optin - (int)fa.sharedSizeBytes);
    if (cache) max_dyn[dev].store(maxd, std::memory_order_relaxed);
  }
  while (live_words > 0 && sizeof(u32) * (size_t)live_words * GG > (size_t)maxd) live_words /= 2;
  const int smem = (int)(sizeof(u32) * (size_t)live_words * GG);
  if (!cache || limit_set[dev].load(std::memory_order_acquire) < smem) {
    ABM_CUDA_TRY(cudaFuncSetAttribute(k_batch_run<N, GG, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    if (cache) {
      int cur = limit_set[dev].load(std::memory_order_relaxed);
      while (cur < smem && !limit_set[dev].compare_exchange_weak(cur, smem)) {
      }
    }
  }
  k_batch_run<N, GG, A><<<grid, N, smem, st>>>(d, nsteps, ext, live_words);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

// the launch shapes instantiated: (threads, models per CTA) for A slots per
// thread (32 slots only up to 512 threads: a chunk's list must fit the CTA's
// static shared memory)
template <int A>
static abm_status batch_shape(const abm_batch* b, int grid, int s, int ext, int live_words, cudaStream_t st) {
  if constexpr (A == 32) {
    switch (b->threads * 10 + b->models_per_cta) {
      case 1281: return batch_launch<128, 1, A>(b->d, grid, s, ext, live_words, st);
      case 2561: return batch_launch<256, 1, A>(b->d, grid, s, ext, live_words, st);
      case 2562: return batch_launch<256, 2, A>(b->d, grid, s, ext, live_words, st);
      case 5121: return batch_launch<512, 1, A>(b->d, grid, s, ext, live_words, st);
      case 5122: return batch_launch<512, 2, A>(b->d, grid, s, ext, live_words, st);
      case 5124: return batch_launch<512, 4, A>(b->d, grid, s, ext, live_words, st);
      default: return ABM_ERR_ARG;
    }
  } else {
    switch (b->threads * 10 + b->models_per_cta) {
      case 1281: return batch_launch<128, 1, A>(b->d, grid, s, ext, live_words, st);
      case 2561: return batch_launch<256, 1, A>(b->d, grid, s, ext, live_words, st);
      case 2562: return batch_launch<256, 2, A>(b->d, grid, s, ext, live_words, st);
      case 5121: return batch_launch<512, 1, A>(b->d, grid, s, ext, live_words, st);
      case 5122: return batch_launch<512, 2, A>(b->d, grid, s, ext, live_words, st);
      case 5124: return batch_launch<512, 4, A>(b->d, grid, s, ext, live_words, st);
      case 10242: return batch_launch<1024, 2, A>(b->d, grid, s, ext, live_words, st);
      case 10244: return batch_launch<1024, 4, A>(b->d, grid, s, ext, live_words, st);
      default: return batch_launch<1024, 1, A>(b->d, grid, s, ext, live_words, st);
    }
  }
}

extern "C" abm_status abm_batch_agents_per_thread(abm_batch* b, int32_t agents_per_thread) {
  if (!b || (agents_per_thread != 8 && agents_per_thread != 16 && agents_per_thread != 32)) return ABM_ERR_ARG;
  if (agents_per_thread == 32 && b->threads > 512) return ABM_ERR_ARG;
  b->agents_per_thread = agents_per_thread;
  return ABM_OK;
}

extern "C" abm_status abm_batch_models_per_cta(abm_batch* b, int32_t models_per_cta) {
  if (!b || (models_per_cta != 1 && models_per_cta != 2 && models_per_cta != 4)) return ABM_ERR_ARG;
  // groups of at least 128 threads (the launch shapes instantiated)
  if (b->threads / models_per_cta < 128) return ABM_ERR_ARG;
  b->models_per_cta = models_per_cta;
  return ABM_OK;
}

extern "C" abm_status abm_batch_run(abm_batch* b, int32_t nsteps, int32_t sweep, void* stream) {
  if (!b || nsteps < 0 || (sweep != ABM_SWEEP_CAPACITY && sweep != ABM_SWEEP_EXTENT)) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = std::max(1, std::min(b->d.nmodels, num_sms() * b->ctas_per_sm));
  const int ext = sweep == ABM_SWEEP_EXTENT;
  // the live-flag bitmask of the largest sweep of the batch, per model run at
  // once (at most 1Mi slots per CTA, and as much as the CTA's shared memory
  // allows; larger models read their flags twice)
  const int G = b->models_per_cta;
  int live_words = 0;
  for (const BModel& m : b->models) live_words = std::max(live_words, (std::max(m.cap[0], m.cap[1]) + 31) / 32);
  live_words = std::min(live_words, kBatchLiveWordsMax / G);
  for (int done = 0; done < nsteps;) {
    const int s = std::min(nsteps - done, b->steps_per_launch);
    const abm_status e = b->agents_per_thread == 8    ? batch_shape<8>(b, grid, s, ext, live_words, st)
                         : b->agents_per_thread == 32 ? batch_shape<32>(b, grid, s, ext, live_words, st)
                                                      : batch_shape<16>(b, grid, s, ext, live_words, st);
    if (e != ABM_OK) return e;
    ABM_LAUNCH_CHECK();
    done += s;
  }
  // rerun models continue at their fixed capacities
  if (b->rerun) return abm_batch_run(b->rerun, nsteps, sweep, stream);
  return ABM_OK;
}

extern "C" abm_status abm_batch_counters_get(abm_batch* b, abm_batch_counters* out, void* stream) {
  if (!b || !out) return ABM_ERR_ARG;
  std::vector<BCtr> h((size_t)b->d.nmodels);
  cudaStream_t st = (cudaStream_t)stream;
  ABM_CUDA_TRY(cudaMemcpyAsync(h.data(), b->d.ctr, sizeof(BCtr) * h.size(), cudaMemcpyDeviceToHost, st));
  ABM_CUDA_TRY(cudaStreamSynchronize(st));
  for (size_t i = 0; i < h.size(); ++i) {
    abm_batch_counters& o = out[i];
    for (int s = 0; s < 2; ++s) {
      o.n_active[s] = h[i].n_active[s];
      o.next_id[s] = h[i].next_id[s];
      o.hw[s] = h[i].hw[s];
      o.overflow[s] = h[i].overflow[s];
      o.extent[s] = h[i].extent[s];
    }
    o.step = h[i].step;
    o.reserved = 0;
    o.agent_steps = h[i].agent_steps;
  }
  if (b->rerun) {
    std::vector<abm_batch_counters> r((size_t)b->rerun->d.nmodels);
    const abm_status e = abm_batch_counters_get(b->rerun, r.data(), stream);
    if (e != ABM_OK) return e;
    for (size_t i = 0; i < h.size(); ++i)
      if (b->rerun_of[i] >= 0) out[i] = r[(size_t)b->rerun_of[i]];
  }
  return ABM_OK;
}

extern "C" abm_status abm_batch_read_agents(abm_batch* b, int32_t m, int32_t species, int32_t which, int32_t* dst,
                                            void* stream) {
  if (!b || !dst || m < 0 || m >= b->d.nmodels || species < 0 || species > 1 || which < 0 || which > 4)
    return ABM_ERR_ARG;
  if (b->rerun && b->rerun_of[(size_t)m] >= 0)
    return abm_batch_read_agents(b->rerun, b->rerun_of[(size_t)m], species, which, dst, stream);
  const BModel& mm = b->models[(size_t)m];
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)mm.cap[species];
  if (which == 0) {
    ABM_CUDA_TRY(cudaMemcpyAsync(dst, b->d.active[species] + mm.oa[species], sizeof(int32_t) * n,
                                 cudaMemcpyDeviceToDevice, st));
  } else {
    const int32_t* src = reinterpret_cast<const int32_t*>(b->d.agent[species] + mm.oa[species]) + (which - 1);
    ABM_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(int32_t), src, sizeof(int4), sizeof(int32_t), n,
                                   cudaMemcpyDeviceToDevice, st));
  }
  return ABM_OK;
}

extern "C" abm_status abm_batch_read_grass(abm_batch* b, int32_t m, int32_t which, int32_t* dst, void* stream) {
  if (!b || !dst || m < 0 || m >= b->d.nmodels || which < 0 || which > 1) return ABM_ERR_ARG;
  if (b->rerun && b->rerun_of[(size_t)m] >= 0)
    return abm_batch_read_grass(b->rerun, b->rerun_of[(size_t)m], which, dst, stream);
  k_batch_grass<<<std::max(1, std::min(num_sms() * 4, (b->models[(size_t)m].ncells + 255) / 256)), 256, 0,
                  (cudaStream_t)stream>>>(b->d, m, which, dst);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_batch_overflowed(abm_batch* b, int32_t* list, int32_t* count, void* stream) {
  if (!b || !list || !count) return ABM_ERR_ARG;
  k_batch_overflowed<<<1, 1024, 0, (cudaStream_t)stream>>>(b->d, list, count);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_batch_digest(abm_batch* b, uint64_t* out, void* stream) {
  if (!b || !out) return ABM_ERR_ARG;
  k_batch_digest<<<b->d.nmodels, 256, 0, (cudaStream_t)stream>>>(b->d, (u64*)out);
  ABM_LAUNCH_CHECK();
  if (b->rerun) {
    const int nr = b->rerun->d.nmodels;
    k_batch_digest<<<nr, 256, 0, (cudaStream_t)stream>>>(b->rerun->d, b->rerun_dig);
    ABM_LAUNCH_CHECK();
    k_scatter_u64<<<std::max(1, std::min((nr + 255) / 256, num_sms() * 4)), 256, 0, (cudaStream_t)stream>>>(
        b->rerun_dig, b->rerun_idx, nr, (u64*)out);
    ABM_LAUNCH_CHECK();
  }
  return ABM_OK;
}

extern "C" abm_status abm_batch_check(abm_batch* b, void* stream) {
  if (!b) return ABM_ERR_ARG;
  if (kCheck) {
    k_batch_canaries<<<b->d.nmodels, 128, 0, (cudaStream_t)stream>>>(b->d);
    ABM_LAUNCH_CHECK();
  }
  ABM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int err = 0;
  ABM_CUDA_TRY(cudaMemcpy(&err, b->d.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return ABM_ERR_OF(err);
  return b->rerun ? abm_batch_check(b->rerun, stream) : ABM_OK;
}

extern "C" abm_status abm_batch_capacity(abm_batch* b, int32_t m, int32_t* cap) {
  if (!b || !cap || m < 0 || m >= b->d.nmodels) return ABM_ERR_ARG;
  if (b->rerun && b->rerun_of[(size_t)m] >= 0) return abm_batch_capacity(b->rerun, b->rerun_of[(size_t)m], cap);
  cap[0] = b->models[(size_t)m].cap[0];
  cap[1] = b->models[(size_t)m].cap[1];
  return ABM_OK;
}

// The learned-capacity recovery path: the models whose births were truncated
// are run again from their initial state, at their fixed capacities, in a
// second batch that this one keeps and reports through.
extern "C" abm_status abm_batch_rerun_overflowed(abm_batch* b, const int32_t* cap_fixed, int32_t sweep,
                                                 int32_t* out_rerun, int32_t* out_unrecovered, void* stream) {
  if (!b || !cap_fixed || (sweep != ABM_SWEEP_CAPACITY && sweep != ABM_SWEEP_EXTENT)) return ABM_ERR_ARG;
  if (b->rerun) return ABM_ERR_STATE;
  const int n = b->d.nmodels;
  for (int i = 0; i < n; ++i)
    if (cap_fixed[2 * i] < b->models[(size_t)i].n0[0] || cap_fixed[2 * i + 1] < b->models[(size_t)i].n0[1] ||
        cap_fixed[2 * i] > (1 << 28) - 1 || cap_fixed[2 * i + 1] > (1 << 28) - 1)
      return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // the overflow flags and the steps run so far, read on the host to size the rerun
  std::vector<BCtr> h((size_t)n);
  ABM_CUDA_TRY(cudaMemcpyAsync(h.data(), b->d.ctr, sizeof(BCtr) * (size_t)n, cudaMemcpyDeviceToHost, st));
  ABM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<abm_batch_model> rm;
  std::vector<int32_t> idx;
  int steps = -1;
  for (int i = 0; i < n; ++i) {
    if (!(h[(size_t)i].overflow[0] | h[(size_t)i].overflow[1])) continue;
    if (steps >= 0 && h[(size_t)i].step != steps) return ABM_ERR_STATE;  // models are always advanced together
    steps = h[(size_t)i].step;
    const BModel& m = b->models[(size_t)i];
    abm_batch_model x;
    std::memset(&x, 0, sizeof(x));
    x.side = m.side;
    x.seed = m.seed;
    x.model = m.model;
    std::memcpy(x.params, m.prm, sizeof(x.params));
    for (int s = 0; s < 2; ++s) {
      x.cap[s] = cap_fixed[2 * i + s];
      x.n0[s] = m.n0[s];
    }
    rm.push_back(x);
    idx.push_back(i);
  }
  if (out_rerun) *out_rerun = (int32_t)rm.size();
  if (out_unrecovered) *out_unrecovered = 0;
  if (rm.empty()) return ABM_OK;
  abm_batch* r = nullptr;
  abm_status e = abm_batch_create(rm.data(), (int32_t)rm.size(), stream, &r);
  if (e != ABM_OK) return e;
  r->threads = b->threads;
  r->ctas_per_sm = b->ctas_per_sm;
  r->steps_per_launch = b->steps_per_launch;
  r->models_per_cta = b->models_per_cta;
  r->agents_per_thread = b->agents_per_thread;
  e = abm_batch_run(r, steps, sweep, stream);
  const int nr = (int)rm.size();
  if (e == ABM_OK && (cudaMalloc(&b->rerun_idx, sizeof(int32_t) * (size_t)nr) != cudaSuccess ||
                      cudaMalloc(&b->rerun_dig, sizeof(u64) * (size_t)nr) != cudaSuccess)) {
    cudaGetLastError();
    e = ABM_ERR_OOM;
  }
  if (e == ABM_OK &&
      cudaMemcpyAsync(b->rerun_idx, idx.data(), sizeof(int32_t) * (size_t)nr, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    e = ABM_ERR_CUDA;
  std::vector<BCtr> hr((size_t)nr);
  if (e == ABM_OK &&
      (cudaMemcpyAsync(hr.data(), r->d.ctr, sizeof(BCtr) * (size_t)nr, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    e = ABM_ERR_CUDA;
  if (e != ABM_OK) {
    batch_free(r);
    cudaFree(b->rerun_idx);
    cudaFree(b->rerun_dig);
    b->rerun_idx = nullptr;
    b->rerun_dig = nullptr;
    return e;
  }
  b->rerun = r;
  b->rerun_of.assign((size_t)n, -1);
  for (int j = 0; j < nr; ++j) b->rerun_of[(size_t)idx[(size_t)j]] = j;
  int unrec = 0;
  for (int j = 0; j < nr; ++j) unrec += (hr[(size_t)j].overflow[0] | hr[(size_t)j].overflow[1]) != 0;
  if (out_unrecovered) *out_unrecovered = unrec;
  return ABM_OK;
}

extern "C" abm_status abm_batch_info(abm_batch* b, int64_t* slots_sheep, int64_t* slots_wolf, int64_t* cells) {
  if (!b) return ABM_ERR_ARG;
  if (slots_sheep) *slots_sheep = b->slots[0];
  if (slots_wolf) *slots_wolf = b->slots[1];
  if (cells) *cells = b->cells;
  return ABM_OK;
}
