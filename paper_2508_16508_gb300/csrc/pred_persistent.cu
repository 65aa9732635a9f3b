// Persistent step kernel for one large predation world (ABMax Section 5.1):
// all phases of many steps in one cooperative launch, separated by a bounded
// grid barrier instead of kernel boundaries.
//
// Per step, five barrier-separated phases (each species: move + claims;
// eat / select / die with flags into bit-planes and per-unit counts; ranks ->
// parent list and the first P free slots (P = parents); births), with the
// wolves' ranks and births shifted by one step and run by two warps of each
// CTA while the other fourteen move and feed the sheep (the schedule is
// spelled out in k_persistent).
// Move and count phases deal 128-slot units to warps round-robin over the
// CTAs (the live agents crowd the low slots) and list the live agents of a
// CTA's units in shared memory for all its threads; the rank phases give CTA
// b a contiguous run of units, so a rank is a prefix over per-run sums, a
// block scan of the unit counts and a warp scan: no look-back chains.
// Every thread keeps the world counters in registers and updates them from
// the same totals, so no counter needs a broadcast.
#include <algorithm>

#include "pred_world.cuh"

namespace abm {

constexpr int kPT = 512;                  // threads per CTA
constexpr int kPWarps = kPT / 32;
constexpr int kBarSpin = 1 << 24;         // bounded barrier wait (polls; a few seconds)
constexpr int kPhases = 5;                // grid barriers per step (plus one closing a launch)

// Grid barrier (all CTAs co-resident: cooperative launch) over a monotonic
// arrival counter: the k-th barrier of a launch is passed once the counter
// reaches base + k * G, base = the arrivals of all earlier launches (kept by
// the host, which knows that each step has kPhases barriers). Each CTA arrives with
// a release add after its threads meet at __syncthreads and waits with
// acquire loads, so everything written before the barrier anywhere in the
// grid is visible after it. A wait that runs out records an error and
// proceeds (results are then invalid, but the kernel ends). Returns, in every
// thread, whether an error was recorded (by the time this CTA arrived, or
// during its wait): the error word is read while waiting, not after.
__device__ __forceinline__ u32 ld_acquire32(const u32* p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(u32* p, u32 v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A grid barrier in two halves, so that independent work can run between
// them: grid_arrive counts this CTA in (after its threads meet), grid_wait
// waits for the whole grid.
__device__ __forceinline__ void grid_arrive(u32* bar, u32& target, u32 expected = 0) {
  target += expected == 0 ? gridDim.x : expected;
  __syncthreads();
  if (threadIdx.x == 0) red_release_add(bar, 1u);
}

__device__ __forceinline__ bool grid_wait(u32* bar, int* err, u32 target, int limit = kBarSpin) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) {
    // in flight during the first polls
    int bad = ld_relaxed32(reinterpret_cast<const u32*>(err)) != 0u;
    int spins = 0;
    u32 backoff = 8;
    while ((int)(ld_acquire32(bar) - target) < 0) {
      if (++spins > limit) {
        atomicCAS(err, 0, kErrTimeout);  // the first error recorded is the one reported
        bad = 1;
        break;
      }
      // another CTA gave up (checked now and then: one round trip per poll)
      if ((spins & 63) == 0 && ld_relaxed32(reinterpret_cast<const u32*>(err)) != 0u) {
        bad = 1;
        break;
      }
      __nanosleep(backoff);
      if (backoff < 32) backoff <<= 1;
    }
    s_bad = bad;
  }
  __syncthreads();
  return s_bad != 0;
}

__device__ __forceinline__ bool grid_sync(u32* bar, int* err, u32& target, u32 expected = 0, int limit = kBarSpin) {
  grid_arrive(bar, target, expected);
  return grid_wait(bar, err, target, limit);
}

// Teams: in phases 1 and 2 a CTA splits into a sheep team (warps 0 ..
// kSheepWarps - 1, named barrier 1) and a wolf team (the last kWolfWarps warps,
// named barrier 2), so that the previous step's wolf ranks and births run
// beside the sheep work instead of before it; in the other phases all warps
// form one team (the CTA barrier). NW = warps of the team (it starts at warp 0
// for the sheep team and the whole CTA).
constexpr int kWolfWarps = 2;
constexpr int kSheepWarps = kPWarps - kWolfWarps;

template <int NW>
__device__ __forceinline__ void tsync() {
  if (NW == kPWarps) {
    __syncthreads();
  } else if (NW == kSheepWarps) {
    asm volatile("bar.sync 1, %0;" ::"n"(kSheepWarps * 32) : "memory");
  } else {
    asm volatile("bar.sync 2, %0;" ::"n"(kWolfWarps * 32) : "memory");
  }
}

// Work compaction over a CTA: in one round every warp loads the live flags of
// kQ 128-slot units (lane l: slots 4l..4l+3 of each, live mask m[q]); the live
// slots of the CTA's kQ * 16 units go into one shared list, entry = v << 7 |
// offset with v = q * 16 + warp the unit's place in the round, so that all 512
// threads then work on whole live agents instead of the warps of dense units
// working while the others idle on placeholders.
constexpr int kQ = 2;                  // units per warp per round
constexpr int kRoundUnits = kQ * kPWarps;

struct CtaList {
  unsigned short* list;  // [kRoundUnits * 128]
  int* wcnt;             // [kRoundUnits]
  // carried from a move phase to the count phase of the same species when
  // all its units fit in one round: the live words of the round's units and,
  // per list entry, the moved agent's cell and energy
  u32* live;             // [kRoundUnits * 4]
  int* cell;             // [kRoundUnits * 128]
  int* energy;           // [kRoundUnits * 128]
};

template <int NW>
__device__ __forceinline__ int cta_list_live(const u32 (&m)[kQ], const CtaList& cl) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  int pre[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const u32 b0 = __ballot_sync(0xFFFFFFFFu, m[q] & 1u), b1 = __ballot_sync(0xFFFFFFFFu, m[q] & 2u);
    const u32 b2 = __ballot_sync(0xFFFFFFFFu, m[q] & 4u), b3 = __ballot_sync(0xFFFFFFFFu, m[q] & 8u);
    pre[q] = __popc(b0 & lt) + __popc(b1 & lt) + __popc(b2 & lt) + __popc(b3 & lt);
    if (lane == 0) cl.wcnt[q * NW + warp] = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
  }
  tsync<NW>();
  int tot = 0;
#pragma unroll
  for (int k = 0; k < kQ * NW; ++k) {
    const int c = cl.wcnt[k];
#pragma unroll
    for (int q = 0; q < kQ; ++q)
      if (k < q * NW + warp) pre[q] += c;
    tot += c;
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (m[q] & (1u << j)) cl.list[pre[q]++] = (unsigned short)(((q * NW + warp) << 7) | (4 * lane + j));
  tsync<NW>();
  return tot;
}

__device__ __forceinline__ u32 live_mask(int4 a) {
  return (u32)(a.x != 0) | ((u32)(a.y != 0) << 1) | ((u32)(a.z != 0) << 2) | ((u32)(a.w != 0) << 3);
}

// unit at place v of round r of this CTA (a team of NW warps deals kQ * NW
// units per round): units are dealt round-robin over the CTAs (unit i -> CTA
// i mod G), so the crowded low slots spread over all SMs
template <int NW>
__device__ __forceinline__ int unit_at(int v, int round) {
  return (int)blockIdx.x + (int)gridDim.x * (v + kQ * NW * round);
}

template <int NW>
__device__ __forceinline__ int slot_of(u32 entry, int round) {
  return (unit_at<NW>((int)(entry >> 7), round) << 7) + (int)(entry & 127u);
}

// ---- several-wolves variant: per-cell lists tagged with the step
__device__ __forceinline__ void list_push(u64* head, u64* next, u64* keys, int cell, int slot, int t, u64 key) {
  keys[slot] = key;
  next[slot] = atomicExch(reinterpret_cast<unsigned long long*>(head + cell),
                          (unsigned long long)(((u64)(u32)t << 32) | (u32)slot));
}

template <int S>
__device__ __forceinline__ int4 move_one(const WorldDev& w, int t, int slot, int4 ag, int L, int metab) {
  const SpeciesDev& sp = w.sp[S];
  if (!in_range(ag.x, w.ncells, w.err)) return ag;  // check builds: a cell outside the lattice
  if (S == 0 && !(w.variant & ABM_VARIANT_MANY_WOLVES)) w.victim[ag.x] = kNoKey;  // last step's victim entry here
  const u32 dir = draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_MOVE, (u32)S) >> 29;
  const int cell = step_cell(ag.x, L, dir);
  ag.x = cell;
  ag.y -= metab;
  ag.w += 1;
  sp.agent[slot] = ag;
  if (S == 0) {
    if (!(w.variant & ABM_VARIANT_GRASS_OFF) && w.regrow[cell] <= t)
      atomicMin(&w.gclaim[cell], claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_PRIO, 0u), slot));
  } else {
    const u64 key = claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_PRIO, 1u), slot);
    if (w.variant & ABM_VARIANT_MANY_WOLVES)  // every wolf joins its cell's list
      list_push(w.wclaim, w.wnext, w.wkey, cell, slot, t, key);
    else if (w.victim[cell] != kNoKey)
      atomicMin(&w.wclaim[cell], key);
  }
  return ag;
}

// phase 1/4: move every live agent; claims for the cell's grass (sheep) or
// the cell's victim (wolves)
// A world whose units fit in one round leaves the round's list, live words and
// moved records in shared memory; `carried` = the list's length (-1 if not).
// live masks of this thread's slots in round `round` of the unit dealing
template <int S, int NW>
__device__ __forceinline__ void round_flags(const WorldDev& w, int ext, int round, u32 (&m)[kQ]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (ext + 127) >> 7;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int i = unit_at<NW>(q * NW + warp, round);
    const int base = (i << 7) + 4 * lane;
    int4 act = make_int4(0, 0, 0, 0);
    if (i < nblk && base < ext) act = reinterpret_cast<const int4*>(w.sp[S].active)[base >> 2];
    m[q] = live_mask(act);
  }
}

// m0 = round_flags(round 0), loaded by the caller ahead of other work
template <int S, int NW>
__device__ __forceinline__ void p_move(const WorldDev& w, int t, int ext, const CtaList& cl, int& carried,
                                       const u32 (&m0)[kQ]) {
  constexpr int NT = NW * 32;
  carried = -1;
  const SpeciesDev& sp = w.sp[S];
  const int L = w.side;
  // without grass (variant) sheep neither spend energy nor claim grass
  const int metab = (S == 0 && (w.variant & ABM_VARIANT_GRASS_OFF)) ? 0 : w.params[PRM_SHEEP_METAB + S];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (ext + 127) >> 7;
  for (int round = 0; unit_at<NW>(0, round) < nblk; ++round) {
    u32 m[kQ];
    if (round == 0) {
#pragma unroll
      for (int q = 0; q < kQ; ++q) m[q] = m0[q];
    } else {
      round_flags<S, NW>(w, ext, round, m);
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {  // live words of the round's units, for the count phase
      u32 vm = m[q] << (4 * (lane & 7));
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) vm |= __shfl_xor_sync(0xFFFFFFFFu, vm, o);
      if ((lane & 7) == 0) cl.live[4 * (q * NW + warp) + (lane >> 3)] = vm;
    }
    const int tot = cta_list_live<NW>(m, cl);
    for (int e = threadIdx.x; e < tot; e += 2 * NT) {
      const int sa = slot_of<NW>(cl.list[e], round);
      const int sb = e + NT < tot ? slot_of<NW>(cl.list[e + NT], round) : -1;
      const int4 aa = sp.agent[sa];
      int4 ab = make_int4(0, 0, 0, 0);
      if (sb >= 0) ab = sp.agent[sb];
      const int4 ma = move_one<S>(w, t, sa, aa, L, metab);
      cl.cell[e] = ma.x;
      cl.energy[e] = ma.y;
      if (sb >= 0) {
        const int4 mb = move_one<S>(w, t, sb, ab, L, metab);
        cl.cell[e + NT] = mb.x;
        cl.energy[e + NT] = mb.y;
      }
    }
    carried = tot;
    tsync<NW>();  // the list is rewritten by the next round
  }
}

// The wolf `slot` on `cell` eats if its rank among the cell's wolves (by key)
// is below the number of sheep there; it eats the sheep of the same rank.
// Lists only hold this step's entries (tag = t); a walk longer than the
// species' capacity means a broken list: the error flag is set.
__device__ __forceinline__ bool eat_rank_matched(const WorldDev& w, int t, int slot, int cell) {
  const u64 tag = (u64)(u32)t;
  const u64 mine = w.wkey[slot];
  int rank = 0, n = 0;
  for (u64 e = w.wclaim[cell]; (e >> 32) == tag; e = w.wnext[(u32)e]) {
    if (++n > w.sp[1].cap) {
      atomicExch(w.err, kErrTimeout);
      return false;
    }
    rank += w.wkey[(u32)e] < mine;
  }
  n = 0;
  for (u64 e = w.victim[cell]; (e >> 32) == tag; e = w.snext[(u32)e]) {
    if (++n > w.sp[0].cap) {
      atomicExch(w.err, kErrTimeout);
      return false;
    }
    const u64 k = w.skey[(u32)e];
    int below = 0, m = 0;
    for (u64 f = w.victim[cell]; (f >> 32) == tag && m <= w.sp[0].cap; f = w.snext[(u32)f], ++m)
      below += w.skey[(u32)f] < k;
    if (below == rank) {
      w.sp[0].active[(u32)e] = 0;
      return true;
    }
  }
  return false;
}

// one live agent of phase 2/5: eat if it won its cell, then die (energy
// below zero) or be drawn as a parent. Returns bit 0 = parent, bit 1 = died,
// bit 2 = ate.
template <int S>
__device__ __forceinline__ u32 count_one(const WorldDev& w, int t, int slot, int4 ag, u64 cl, int gain, u32 Tr,
                                         int regrowth) {
  const SpeciesDev& sp = w.sp[S];
  const int cell = ag.x;
  u32 r = 0;
  if (S == 1 && (w.variant & ABM_VARIANT_MANY_WOLVES)) {
    if (eat_rank_matched(w, t, slot, cell)) {
      ag.y += gain;
      sp.agent[slot].y = ag.y;
      r |= 4u;
    }
  } else if (cl != kNoKey && (u32)cl == (u32)slot) {
    ag.y += gain;
    sp.agent[slot].y = ag.y;
    r |= 4u;
    if (S == 0) {
      w.gclaim[cell] = kNoKey;
      w.regrow[cell] = t + regrowth;
    } else {
      w.wclaim[cell] = kNoKey;
      const u64 v = w.victim[cell];
      if (in_range((u32)v, w.sp[0].cap, w.err)) w.sp[0].active[(u32)v] = 0;
      w.victim[cell] = kNoKey;
    }
  }
  if (ag.y < 0) {
    sp.active[slot] = 0;
    r |= 2u;
  } else {
    if (draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_REPRO, (u32)S) < Tr) r |= 1u;
    if (S == 0) {
      const u64 key = claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u), slot);
      if (w.variant & ABM_VARIANT_MANY_WOLVES)
        list_push(w.victim, w.snext, w.skey, cell, slot, t, key);
      else
        atomicMin(&w.victim[cell], key);
    }
  }
  return r;
}

// phase 2/5: eat, select parents, kill the starving. Units are dealt and
// their live agents listed as for the moves. Each unit then writes its free /
// parent bits into the bit-planes (word = 32 slots = 8 lanes x 4 slots) and
// its two counts, which are also summed per run of kseg units (the CTA
// segments of the rank phase).
template <int S, int NW>
__device__ __forceinline__ void p_count(const WorldDev& w, int t, int ext, int kseg, int* acc, const CtaList& cl,
                                        int carried, u32* s_upar /* [kRoundUnits][4], zero on entry and exit */,
                                        int* s_acc /* [2 * kPWarps] */) {
  constexpr int NT = NW * 32;
  const SpeciesDev& sp = w.sp[S];
  const PersistDev& ps = w.ps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (ext + 127) >> 7;
  const int gain = w.params[S];
  const u32 Tr = (u32)w.params[PRM_SHEEP_T + S];
  const int regrowth = w.params[PRM_REGROWTH];
  const u64* claim = S == 0 ? w.gclaim : w.wclaim;
  int starved = 0, won = 0;
  // one round and the move phase's list still in shared memory: neither the
  // live flags nor the agent records need reading again
  const bool reuse = carried >= 0 && unit_at<NW>(0, 1) >= nblk;
  for (int round = 0; unit_at<NW>(0, round) < nblk; ++round) {
    u32 m[kQ], fr[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int i = unit_at<NW>(q * NW + warp, round);
      const int base = (i << 7) + 4 * lane;
      if (reuse) {
        m[q] = (cl.live[4 * (q * NW + warp) + (lane >> 3)] >> (4 * (lane & 7))) & 0xFu;
      } else {
        int4 act = make_int4(0, 0, 0, 0);
        if (i < nblk && base < ext) act = reinterpret_cast<const int4*>(sp.active)[base >> 2];
        m[q] = live_mask(act);
      }
      const u32 valid = (i >= nblk || base >= ext) ? 0u : (ext - base >= 4 ? 0xFu : (1u << (ext - base)) - 1u);
      fr[q] = ~m[q] & valid;
    }
    const int tot = reuse ? carried : cta_list_live<NW>(m, cl);
    for (int e = threadIdx.x; e < tot; e += 2 * NT) {
      const u32 ea = cl.list[e];
      const int eb = e + NT < tot ? (int)cl.list[e + NT] : -1;
      const int sa = slot_of<NW>(ea, round);
      const int sb = eb >= 0 ? slot_of<NW>((u32)eb, round) : -1;
      int4 aa, ab = make_int4(0, 0, 0, 0);
      if (reuse) {
        aa = make_int4(cl.cell[e], cl.energy[e], 0, 0);
        if (sb >= 0) ab = make_int4(cl.cell[e + NT], cl.energy[e + NT], 0, 0);
      } else {
        aa = sp.agent[sa];
        if (sb >= 0) ab = sp.agent[sb];
      }
      if (!in_range(aa.x, w.ncells, w.err)) aa.x = 0;  // check builds only (recorded, then harmless)
      if (sb >= 0 && !in_range(ab.x, w.ncells, w.err)) ab.x = 0;
      const u64 ca = claim[aa.x];
      const u64 cb = sb >= 0 ? claim[ab.x] : kNoKey;
      u32 r = count_one<S>(w, t, sa, aa, ca, gain, Tr, regrowth);
      if (r & 1u) atomicOr(&s_upar[4 * (ea >> 7) + ((ea & 127u) >> 5)], 1u << (ea & 31u));
      starved += (r >> 1) & 1u;
      won += (r >> 2) & 1u;
      if (sb >= 0) {
        r = count_one<S>(w, t, sb, ab, cb, gain, Tr, regrowth);
        if (r & 1u) atomicOr(&s_upar[4 * (eb >> 7) + ((eb & 127) >> 5)], 1u << (eb & 31));
        starved += (r >> 1) & 1u;
        won += (r >> 2) & 1u;
      }
    }
    tsync<NW>();
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int v = q * NW + warp;
      const int i = unit_at<NW>(v, round);
      if (i >= nblk) continue;
      const int base = (i << 7) + 4 * lane;
      const u32 pw = s_upar[4 * v + (lane >> 3)];
      const u32 par = (pw >> (4 * (lane & 7))) & 0xFu;
      // 8 lanes x 4 bits -> one plane word
      u32 vf = fr[q] << (4 * (lane & 7));
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) vf |= __shfl_xor_sync(0xFFFFFFFFu, vf, o);
      if ((lane & 7) == 0 && base < ext) {
        ps.plane[S][0][base >> 5] = vf;
        ps.plane[S][1][base >> 5] = pw;
      }
      u32 cu = ((u32)__popc(fr[q]) << 16) | (u32)__popc(par);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cu += __shfl_xor_sync(0xFFFFFFFFu, cu, o);
      if (lane == 0) {
        const u64 val = ((u64)(cu >> 16) << 32) | (cu & 0xFFFFu);
        ps.blk[S][i] = val;
        atomicAdd(reinterpret_cast<unsigned long long*>(&ps.seg[S][i / kseg]), (unsigned long long)val);
      }
      __syncwarp();
      if (lane < 4) s_upar[4 * v + lane] = 0u;
    }
    tsync<NW>();  // the list and the unit words are rewritten by the next round
  }
  // accumulators: summed over the CTA first, so that the two counters see one
  // atomic per CTA, not one per warp (same-address atomics serialise in L2)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    starved += __shfl_xor_sync(0xFFFFFFFFu, starved, o);
    won += __shfl_xor_sync(0xFFFFFFFFu, won, o);
  }
  if (lane == 0) {
    s_acc[2 * warp] = starved;
    s_acc[2 * warp + 1] = won;
  }
  tsync<NW>();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      a += s_acc[2 * k];
      b += s_acc[2 * k + 1];
    }
    if (a) atomicAdd(&acc[S], a);
    if (b) atomicAdd(&acc[S == 0 ? 3 : 2], b);
  }
}

// grand totals of the per-segment counts: (free, parents) over all segments
// and over the segments before this CTA's, in every thread
template <int S>
__device__ __forceinline__ void grand_totals(const PersistDev& ps, u32& F, u32& P, u32& preF, u32& preP,
                                             u64* s_red) {
  u64 tot = 0, pre = 0;
  for (int j = threadIdx.x; j < (int)gridDim.x; j += kPT) {
    const u64 x = ps.seg[S][j];
    tot += x;
    if (j < (int)blockIdx.x) pre += x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    s_red[2 * (threadIdx.x >> 5)] = tot;
    s_red[2 * (threadIdx.x >> 5) + 1] = pre;
  }
  __syncthreads();
  tot = pre = 0;
  for (int i = 0; i < kPWarps; ++i) {
    tot += s_red[2 * i];
    pre += s_red[2 * i + 1];
  }
  F = (u32)(tot >> 32);
  P = (u32)tot;
  preF = (u32)(pre >> 32);
  preP = (u32)pre;
  __syncthreads();  // s_red is reused by the caller
}

// One unit's ranks: a warp scan of the lanes' (free, parent) counts taken
// from the unit's plane words wf / wp (zero past the extent) and its prefix
// pr = free << 32 | parents, then the list writes: the parent list takes
// every parent, the free list only the ranks below P (the only free slots a
// child can receive).
template <int S>
__device__ __forceinline__ void rank_unit(const WorldDev& w, int base, int ext, u32 wf, u32 wp, u64 pr, u32 P,
                                          int lane) {
  const SpeciesDev& sp = w.sp[S];
  const int sh = 4 * (lane & 7);
  u32 fr = base < ext ? (wf >> sh) & 0xFu : 0u;
  u32 par = base < ext ? (wp >> sh) & 0xFu : 0u;
  const u32 c = (u32)__popc(fr) | ((u32)__popc(par) << 16);
  u32 inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 x = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += x;
  }
  const u32 ex = inc - c;
  u32 rf = (u32)(pr >> 32) + (ex & 0xFFFFu), rp = (u32)pr + (ex >> 16);
  while (fr && rf < P) {
    const int jj = __ffs(fr) - 1;
    fr &= fr - 1;
    if (in_range(rf, sp.cap, w.err)) sp.freel[rf] = base + jj;
    ++rf;
  }
  while (par) {
    const int jj = __ffs(par) - 1;
    par &= par - 1;
    if (in_range(rp, sp.cap, w.err)) sp.parents[rp] = base + jj;
    ++rp;
  }
}

// phase 3/6: ranks -> parent list (all) and free list (ranks below P only).
// CTA b owns units [b*kseg, (b+1)*kseg); the unit ranks are the segment's
// prefix plus a block scan of the unit counts; inside a unit, a warp scan.
template <int S>
__device__ __forceinline__ void p_ranks(const WorldDev& w, int ext, int kseg, u32 P, u32 preF, u32 preP,
                                        u64* s_red, u64* s_pre) {
  const PersistDev& ps = w.ps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (ext + 127) >> 7;
  const int j0 = blockIdx.x * kseg, j1 = min(nblk, j0 + kseg);
  u32 cf = preF, cp = preP;
  for (int c0 = j0; c0 < j1; c0 += kPT) {
    const int j = c0 + threadIdx.x;
    const u64 v = j < j1 ? ps.blk[S][j] : 0ull;
    u32 exf, exp_, tf, tp;
    block_scan2<kPT>((u32)(v >> 32), (u32)v, exf, exp_, tf, tp, s_red);
    s_pre[threadIdx.x] = ((u64)(cf + exf) << 32) | (u64)(cp + exp_);
    __syncthreads();
    const int cn = min(kPT, j1 - c0);
    for (int q = warp; q < cn; q += kPWarps) {
      const int base = ((c0 + q) << 7) + 4 * lane;
      u32 wf = 0, wp = 0;
      if (base < ext) {
        wf = ps.plane[S][0][base >> 5];
        wp = ps.plane[S][1][base >> 5];
      }
      rank_unit<S>(w, base, ext, wf, wp, s_pre[q], P, lane);
    }
    cf += tf;
    cp += tp;
    __syncthreads();  // s_pre and s_red are rewritten by the next pass
  }
}

// Stage the two plane-word quads (free, parent: the 4 words of 128 slots) of
// units j0 .. j0 + min(n, nu) - 1 into s_pw[8 * q + 4 * plane + word] with
// 16-byte cp.async, threads tid < 2 * nu (one quad each); commits a group.
template <int S>
__device__ __forceinline__ void stage_planes(const PersistDev& ps, int j0, int n, int nu, int tid, u32* s_pw) {
  if (tid < 2 * nu) {
    const int q = tid >> 1, pl = tid & 1;
    if (q < n) cp_async16(s_pw + 8 * q + 4 * pl, ps.plane[S][pl] + 4 * (j0 + q));
  }
  cp_async_commit();
}

// A rank phase (grand totals + ranks). When this CTA's run of units is short
// (kseg <= kPWarps * kRankU, the common case) every load -- the segment sums,
// the unit counts, the plane words (cp.async into shared memory) -- is issued
// up front, so the phase costs one memory round trip instead of three.
constexpr int kRankU = 4;

template <int S>
__device__ __forceinline__ void rank_phase(const WorldDev& w, int ext, int kseg, u32& F, u32& P, u64* s_red,
                                           u64* s_pre, u32* s_pw /* [kPWarps * kRankU][2][4], 16-byte aligned */) {
  const PersistDev& ps = w.ps;
  if (kseg > kPWarps * kRankU || (int)gridDim.x > kPT) {
    u32 preF, preP;
    grand_totals<S>(ps, F, P, preF, preP, s_red);
    p_ranks<S>(w, ext, kseg, P, preF, preP, s_red, s_pre);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (ext + 127) >> 7;
  const int j0 = blockIdx.x * kseg, j1 = min(nblk, j0 + kseg);
  const int n = max(0, j1 - j0);
  stage_planes<S>(ps, j0, n, kPWarps * kRankU, threadIdx.x, s_pw);
  const u64 sv = threadIdx.x < (int)gridDim.x ? ps.seg[S][threadIdx.x] : 0ull;
  const u64 bv = threadIdx.x < n ? ps.blk[S][j0 + threadIdx.x] : 0ull;
  // grand totals and the sums of the segments before this CTA's
  u64 tot = sv, pre = (int)threadIdx.x < (int)blockIdx.x ? sv : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
  }
  __syncthreads();
  if (lane == 0) {
    s_red[2 * warp] = tot;
    s_red[2 * warp + 1] = pre;
  }
  __syncthreads();
  tot = pre = 0;
  for (int i = 0; i < kPWarps; ++i) {
    tot += s_red[2 * i];
    pre += s_red[2 * i + 1];
  }
  F = (u32)(tot >> 32);
  P = (u32)tot;
  const u32 preF = (u32)(pre >> 32), preP = (u32)pre;
  cp_async_wait_0();  // the staged plane words: visible to the CTA after the barrier
  __syncthreads();  // s_red is reused by the scan
  // unit prefixes inside the run
  u32 exf, exp_, tf, tp;
  block_scan2<kPT>((u32)(bv >> 32), (u32)bv, exf, exp_, tf, tp, s_red);
  s_pre[threadIdx.x] = ((u64)(preF + exf) << 32) | (u64)(preP + exp_);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kRankU; ++k) {
    const int q = warp + kPWarps * k;
    if (q >= n) break;
    rank_unit<S>(w, ((j0 + q) << 7) + 4 * lane, ext, s_pw[8 * q + (lane >> 3)], s_pw[8 * q + 4 + (lane >> 3)],
                 s_pre[q], P, lane);
  }
  __syncthreads();  // s_pre and s_red are reused
}

// A rank phase on the wolf team (kWolfWarps warps, named barrier 2) while the
// sheep team moves the sheep: the same lists as rank_phase. The segment sums,
// the first pass's unit counts and the plane words of the first
// kRankTU * kWolfWarps units are all requested up front, in one round trip
// (the plane words by cp.async into shared memory, 32 bytes a unit, so that
// they hold no registers); longer runs of units take further passes of one
// unit count per team thread.
constexpr int kRankTU = 8;

template <int S>
__device__ __forceinline__ void rank_team(const WorldDev& w, int ext, int kseg, u32& F, u32& P,
                                          u64* s_red /* [2 * kWolfWarps] */,
                                          u64* s_pre /* [kWolfWarps * 32 + 2 * kRankTU * kWolfWarps] */) {
  constexpr int NW = kWolfWarps, NT = NW * 32, NU = kRankTU * NW;
  const PersistDev& ps = w.ps;
  const int tt = (int)threadIdx.x - kSheepWarps * 32;
  const int warp = tt >> 5, lane = tt & 31;
  const int nblk = (ext + 127) >> 7;
  const int j0 = blockIdx.x * kseg, j1 = min(nblk, j0 + kseg);
  const int n = max(0, j1 - j0);
  u32* s_pw = reinterpret_cast<u32*>(s_pre + NT);  // [NU][2][4] plane words of the first NU units
  stage_planes<S>(ps, j0, n, NU, tt, s_pw);
  const u64 bv0 = tt < n ? ps.blk[S][j0 + tt] : 0ull;
  // grand totals and the sums of the segments before this CTA's
  u64 tot = 0, pre = 0;
  for (int j = tt; j < (int)gridDim.x; j += NT) {
    const u64 x = ps.seg[S][j];
    tot += x;
    if (j < (int)blockIdx.x) pre += x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
  }
  if (lane == 0) {
    s_red[2 * warp] = tot;
    s_red[2 * warp + 1] = pre;
  }
  cp_async_wait_0();  // the staged plane words: visible to the team after the barrier
  tsync<NW>();
  tot = pre = 0;
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    tot += s_red[2 * i];
    pre += s_red[2 * i + 1];
  }
  F = (u32)(tot >> 32);
  P = (u32)tot;
  tsync<NW>();  // s_red is reused by the scan
  // unit prefixes, packed (free << 32 | parents: the parent sums stay below
  // the capacity, so the low half never carries into the high one)
  for (int c0 = 0; c0 < n; c0 += NT) {
    const u64 v = c0 == 0 ? bv0 : (c0 + tt < n ? ps.blk[S][j0 + c0 + tt] : 0ull);
    u64 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 x = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += x;
    }
    if (lane == 31) s_red[warp] = inc;
    tsync<NW>();
    u64 wpre = 0, ptot = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      const u64 x = s_red[i];
      if (i < warp) wpre += x;
      ptot += x;
    }
    s_pre[tt] = pre + wpre + inc - v;
    tsync<NW>();
    const int cn = min(NT, n - c0);
    int q = warp;
    if (c0 == 0) {
#pragma unroll
      for (int k = 0; k < kRankTU; ++k, q += NW)
        if (q < cn)
          rank_unit<S>(w, ((j0 + q) << 7) + 4 * lane, ext, s_pw[8 * q + (lane >> 3)], s_pw[8 * q + 4 + (lane >> 3)],
                       s_pre[q], P, lane);
    }
    for (; q < cn; q += NW) {
      const int base = ((j0 + c0 + q) << 7) + 4 * lane;
      u32 a = 0, b = 0;
      if (base < ext) {
        a = ps.plane[S][0][base >> 5];
        b = ps.plane[S][1][base >> 5];
      }
      rank_unit<S>(w, base, ext, a, b, s_pre[q], P, lane);
    }
    pre += ptot;
    tsync<NW>();  // s_pre and s_red are rewritten by the next pass
  }
}

// births on a team of NT threads (tid = the thread's place in it)
template <int S, int NT>
__device__ __forceinline__ void p_births(const WorldDev& w, int t, int r, int F, int ext, int id0, int tid) {
  const SpeciesDev& sp = w.sp[S];
  // birth i -> CTA i mod G: the births spread over all SMs
  for (int i = blockIdx.x + gridDim.x * tid; i < r; i += gridDim.x * NT) {
    const int p = sp.parents[i];
    const int slot = i < F ? sp.freel[i] : ext + (i - F);
    if (!in_range(p, sp.cap, w.err) || !in_range(slot, sp.cap, w.err)) continue;
    const int4 pa = sp.agent[p];
    const int half = pa.y >> 1;
    sp.agent[p].y = pa.y - half;
    sp.agent[slot] = make_int4(pa.x, half, (int)((u32)id0 + (u32)i), 0);
    sp.active[slot] = 1;
    if (S == 0) {
      const u64 key = claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u), slot);
      if (w.variant & ABM_VARIANT_MANY_WOLVES)
        list_push(w.victim, w.snext, w.skey, pa.x, slot, t, key);
      else
        atomicMin(&w.victim[pa.x], key);
    }
  }
}

struct Births {
  int r, F, ext, id0;
};

__device__ __forceinline__ u64 globaltimer() {
  u64 t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bookkeeping that no phase reads: the live counts, high-water marks,
// overflow flags and per-step statistics. Block 0's thread 0 keeps it in
// shared memory, so that it takes no registers of the other threads (a
// register spilled to local memory costs a round trip at a phase boundary).
struct StepBook {
  int nact[2], hw[2], ovf[2];
  int nstart0, r0p, P0p, starved0p, grassp;  // of the previous step's sheep
  abm_step_stats* stp;                       // statistics row of the previous step
  u64 clk_last;                              // phase timing (block 0)
};

__device__ __forceinline__ bool book_thread() { return blockIdx.x == 0 && threadIdx.x == 0; }

// phase timing by block 0 (nanoseconds from one barrier exit to the next)
struct PhaseClock {
  unsigned long long* acc;
  StepBook& b;
  __device__ __forceinline__ void start() {
    if (acc && book_thread()) b.clk_last = globaltimer();
  }
  __device__ __forceinline__ void lap(int k) {
    if (acc && book_thread()) {
      const u64 now = globaltimer();
      acc[k] += now - b.clk_last;
      b.clk_last = now;
    }
  }
};

// MINB = resident CTAs per SM the register budget is cut for (1: up to 128
// registers a thread, 2: 64).
template <int MINB>
__global__ void __launch_bounds__(kPT, MINB) k_persistent(WorldDev w, int nsteps, abm_step_stats* stats,
                                                     unsigned long long* phase_ns) {
  __shared__ u64 s_red[2 * kPWarps];
  __shared__ __align__(16) u64 s_pre[kPT];
  __shared__ unsigned short s_clist[kRoundUnits * 128];
  __shared__ int s_wcnt[kRoundUnits];
  __shared__ u32 s_upar[kRoundUnits * 4];
  __shared__ int s_acc[2 * kPWarps];
  __shared__ u32 s_live[kRoundUnits * 4];
  __shared__ __align__(16) int s_cell[kRoundUnits * 128];
  __shared__ int s_energy[kRoundUnits * 128];
  __shared__ int s_wolf[4];  // the wolf team's F, P, starved and eaten, for the whole CTA
  __shared__ StepBook s_book;
  const CtaList cl{s_clist, s_wcnt, s_live, s_cell, s_energy};
  const bool wolf_team = (int)threadIdx.x >= kSheepWarps * 32;
  int carried = -1;
  if (threadIdx.x < kRoundUnits * 4) s_upar[threadIdx.x] = 0u;
  PhaseClock clk{phase_ns, s_book};
  u32 bar_target = w.bar_base;  // arrival count that completes the next barrier
  WorldCtr* c = w.ctr;
  const PersistDev& ps = w.ps;
  // counters the phases read: one copy per thread, all updated identically
  int t = c->step;
  int ext[2] = {c->extent[0], c->extent[1]};
  int nid[2] = {c->next_id[0], c->next_id[1]};
  if (book_thread()) {
    for (int s2 = 0; s2 < 2; ++s2) {
      s_book.nact[s2] = c->n_active[s2];
      s_book.hw[s2] = c->hw[s2];
      s_book.ovf[s2] = c->overflow[s2];
    }
    s_book.nstart0 = s_book.r0p = s_book.P0p = s_book.starved0p = s_book.grassp = 0;
    s_book.stp = nullptr;
  }
  clk.start();
  // Wolf ranks of step t-1 run beside the sheep moves of step t, and the wolf
  // moves of step t beside the sheep ranks: neither needs the other's
  // results, so a step takes five barrier-separated phases:
  //   P1  wolf team: wolf ranks (t-1) | sheep team: sheep move (t)
  //   P2  wolf counters and statistics (t-1) in every thread, then
  //       wolf team: wolf births (t-1) | sheep team: sheep eat / select / die (t)
  //   P3  sheep ranks (t) | wolves move + victim claims (t) (a wolf only
  //       needs a live sheep on its cell: the survivors registered in P2)
  //   P4  sheep births (t) (lambs register as victims before wolves eat)
  //   P5  wolves eat / kill / select / die (t)
  // and the last step's wolf ranks and births close the launch. In P1 and P2
  // the two teams meet only at the grid barriers; P3 to P5 use every warp.
  // The barrier between P3 and P4 is split: a CTA counts itself in once its
  // ranks are written and waits only after its wolf moves, so the wait
  // overlaps the wolf moves (births touch no wolf, and a lamb lands on its
  // parent's cell, which already holds a victim key, so no claim condition of
  // the wolf move changes under it).
  // wolf team: the ranks of step tw's wolves and that step's counters, left in s_wolf
  auto wolf_ranks = [&](int tw) {
    const int* accw = ps.acc + 4 * (tw & 1);
    // complete since the last barrier; loaded ahead of the rank phase's own
    // loads (for the bookkeeping of block 0 only)
    const int starved1 = blockIdx.x == 0 ? accw[1] : 0, eaten = blockIdx.x == 0 ? accw[2] : 0;
    u32 F1, P1;
    const int kseg1 = (((ext[1] + 127) >> 7) + (int)gridDim.x - 1) / (int)gridDim.x;  // as in the count phase
    rank_team<1>(w, ext[1], kseg1, F1, P1, s_red, s_pre);
    if ((int)threadIdx.x == kSheepWarps * 32) {
      s_wolf[0] = (int)F1;
      s_wolf[1] = (int)P1;
      s_wolf[2] = starved1;
      s_wolf[3] = eaten;
    }
  };
  // every thread: the counters after step tw's wolf births, from s_wolf
  // (the bookkeeping and step tw's statistics: block 0's thread 0); returns
  // the births to place
  auto wolf_counters = [&](int tw) -> Births {
    const int F1 = s_wolf[0], P1 = s_wolf[1];
    const int avail1 = F1 + (w.sp[1].cap - ext[1]);
    const int r1 = min(P1, avail1);
    const Births wb = {r1, F1, ext[1], nid[1]};
    nid[1] += r1;
    if (r1 > F1) ext[1] += r1 - F1;
    if (book_thread()) {
      StepBook& b = s_book;
      const int starved1 = s_wolf[2], eaten = s_wolf[3];
      const int n_after = b.nact[1] + r1;
      if (n_after > b.hw[1]) b.hw[1] = n_after;
      b.nact[1] = n_after - starved1;
      if (P1 > avail1) b.ovf[1] = 1;
      b.nact[0] -= eaten;
      if (abm_step_stats* stp = b.stp) {
        stp->parents[0] = b.P0p;
        stp->parents[1] = P1;
        stp->births[0] = b.r0p;
        stp->births[1] = r1;
        stp->starved[0] = b.starved0p;
        stp->starved[1] = starved1;
        stp->eaten = eaten;
        stp->grass_eaten = b.grassp;
        for (int s2 = 0; s2 < 2; ++s2) {
          stp->n_end[s2] = b.nact[s2];
          stp->hw[s2] = b.hw[s2];
          stp->overflow[s2] = b.ovf[s2];
        }
        stp->step = tw;
      }
    }
    return wb;
  };
  for (int it = 0; it < nsteps; ++it) {
    int* acc = ps.acc + 4 * (t & 1);
    // ---- P1: wolf ranks of the previous step | sheep move
    if (wolf_team) {
      if (it > 0) wolf_ranks(t - 1);
    } else {
      u32 mf[kQ];
      round_flags<0, kSheepWarps>(w, ext[0], 0, mf);
      if (blockIdx.x == 0 && threadIdx.x == 0) acc[0] = acc[1] = acc[2] = acc[3] = 0;  // last read in P1 of step t-1
      p_move<0, kSheepWarps>(w, t, ext[0], cl, carried, mf);
    }
    const bool bad = grid_sync(ps.bar, w.err, bar_target);
    clk.lap(0);
    if (bad) return;
    // ---- P2: wolf counters (t-1) | wolf births (t-1) beside sheep eat / select / die / flags
    const Births wb = it > 0 ? wolf_counters(t - 1) : Births{0, 0, 0, 0};
    if (book_thread()) {
      s_book.nstart0 = s_book.nact[0];
      if (stats) {
        abm_step_stats* st = stats + it;
        st->n_start[0] = s_book.nact[0];
        st->n_start[1] = s_book.nact[1];
        st->extent[0] = ext[0];
        st->extent[1] = ext[1];
      }
    }
    const int kseg0 = (((ext[0] + 127) >> 7) + (int)gridDim.x - 1) / (int)gridDim.x;
    if (wolf_team) {
      if (it > 0)
        p_births<1, kWolfWarps * 32>(w, t - 1, wb.r, wb.F, wb.ext, wb.id0, (int)threadIdx.x - kSheepWarps * 32);
    } else {
      if (blockIdx.x == 0)  // wolf segment sums: last read in P1
        for (int j = threadIdx.x; j < (int)gridDim.x; j += kSheepWarps * 32) ps.seg[1][j] = 0ull;
      p_count<0, kSheepWarps>(w, t, ext[0], kseg0, acc, cl, carried, s_upar, s_acc);
    }
    grid_sync(ps.bar, w.err, bar_target);
    clk.lap(1);
    // ---- P3: sheep ranks and lists | wolves move + claims
    u32 mf[kQ];
    round_flags<1, kPWarps>(w, ext[1], 0, mf);  // issued before the sheep ranks, used by the wolf move
    u32 F0, P0;
    // (s_cell is free between the count phase and the wolf move: plane staging)
    rank_phase<0>(w, ext[0], kseg0, F0, P0, s_red, s_pre, reinterpret_cast<u32*>(s_cell));
    const int avail0 = (int)F0 + (w.sp[0].cap - ext[0]);
    const int r0 = min((int)P0, avail0);
    const Births sb = {r0, (int)F0, ext[0], nid[0]};
    // the ranks' half of the barrier; the wolf move needs none of them
    grid_arrive(ps.bar, bar_target);
    p_move<1, kPWarps>(w, t, ext[1], cl, carried, mf);
    grid_wait(ps.bar, w.err, bar_target);
    clk.lap(2);
    // ---- P4: sheep births (every CTA's lists are complete: the split barrier's wait); sheep counters
    int starved0 = 0, grass = 0;
    if (book_thread()) {  // written in P2: loaded ahead of the births' own loads
      starved0 = acc[0];
      grass = acc[3];
    }
    p_births<0, kPT>(w, t, sb.r, sb.F, sb.ext, sb.id0, threadIdx.x);
    if (blockIdx.x == 0)  // sheep segment sums: last read by the rank phases
      for (int j = threadIdx.x; j < (int)gridDim.x; j += kPT) ps.seg[0][j] = 0ull;
    nid[0] += r0;
    if (r0 > (int)F0) ext[0] += r0 - (int)F0;
    if (book_thread()) {
      StepBook& b = s_book;
      const int n_after = b.nstart0 + r0;
      if (n_after > b.hw[0]) b.hw[0] = n_after;
      b.nact[0] = n_after - starved0;
      if ((int)P0 > avail0) b.ovf[0] = 1;
      b.r0p = r0;
      b.P0p = (int)P0;
      b.starved0p = starved0;
      b.grassp = grass;
    }
    grid_sync(ps.bar, w.err, bar_target);
    clk.lap(3);
    // ---- P5: wolves eat / kill / select / die / flags
    const int kseg1 = (((ext[1] + 127) >> 7) + (int)gridDim.x - 1) / (int)gridDim.x;
    p_count<1, kPWarps>(w, t, ext[1], kseg1, acc, cl, carried, s_upar, s_acc);
    if (book_thread()) s_book.stp = stats ? stats + it : nullptr;
    ++t;
    grid_sync(ps.bar, w.err, bar_target);
    clk.lap(4);
  }
  // the last step's wolf ranks and births (every warp is free: the whole CTA ranks)
  if (nsteps > 0) {
    const int* accw = ps.acc + 4 * ((t - 1) & 1);
    const int starved1 = book_thread() ? accw[1] : 0, eaten = book_thread() ? accw[2] : 0;
    const int kseg1 = (((ext[1] + 127) >> 7) + (int)gridDim.x - 1) / (int)gridDim.x;  // as in the count phase
    u32 F1, P1;
    rank_phase<1>(w, ext[1], kseg1, F1, P1, s_red, s_pre, reinterpret_cast<u32*>(s_cell));
    if (threadIdx.x == 0) {
      s_wolf[0] = (int)F1;
      s_wolf[1] = (int)P1;
      s_wolf[2] = starved1;
      s_wolf[3] = eaten;
    }
    __syncthreads();
    const Births wb = wolf_counters(t - 1);
    grid_sync(ps.bar, w.err, bar_target);
    clk.lap(5);
    p_births<1, kPT>(w, t - 1, wb.r, wb.F, wb.ext, wb.id0, threadIdx.x);
    if (blockIdx.x == 0)  // wolf segment sums, for the next launch
      for (int j = threadIdx.x; j < (int)gridDim.x; j += kPT) ps.seg[1][j] = 0ull;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->step = t;
    for (int s = 0; s < 2; ++s) {
      c->extent[s] = ext[s];
      c->n_active[s] = s_book.nact[s];
      c->next_id[s] = nid[s];
      c->hw[s] = s_book.hw[s];
      c->overflow[s] = s_book.ovf[s];
    }
  }
}

// Failure-detection check: a grid barrier that waits for one CTA more than
// the grid has, so that the wait must run out; every CTA records the timeout
// and returns. Used to show that a wait which never completes ends the kernel
// with an error status instead of hanging the GPU.
__global__ void k_barrier_timeout(u32* bar, int* err, int limit) {
  u32 target = 0;
  grid_sync(bar, err, target, gridDim.x + 1, limit);
}

int persistent_max_ctas() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<2>, kPT, 0) != cudaSuccess) return 0;
  return nb * num_sms();
}

int persistent_warps() { return kPWarps; }

abm_status launch_persistent(const WorldDev& d, u32* bar_next, int grid, int nsteps, abm_step_stats* stats,
                             cudaStream_t st, unsigned long long* phase_ns) {
  WorldDev dd = d;
  dd.bar_base = *bar_next;
  void* args[] = {(void*)&dd, (void*)&nsteps, (void*)&stats, (void*)&phase_ns};
  // one CTA per SM: the variant with the larger register budget
  const void* fn = grid <= num_sms() ? (const void*)k_persistent<1> : (const void*)k_persistent<2>;
  ABM_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kPT), args, 0, st));
  // arrivals this launch adds to the counter
  if (nsteps > 0) *bar_next += ((u32)kPhases * (u32)nsteps + 1u) * (u32)grid;
  return ABM_OK;
}

}  // namespace abm

extern "C" abm_status abm_diag_barrier_timeout(int32_t spin_limit, void* stream) {
  using namespace abm;
  if (spin_limit < 1 || spin_limit > (1 << 24)) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  u32* bar = nullptr;
  int* err = nullptr;
  ABM_CUDA_TRY(cudaMalloc(&bar, sizeof(u32) * 2));
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaFree(bar);
    return ABM_ERR_OOM;
  }
  abm_status rc = ABM_OK;
  if (cudaMemsetAsync(bar, 0, sizeof(u32) * 2, st) != cudaSuccess || cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    rc = ABM_ERR_CUDA;
  if (rc == ABM_OK) {
    void* args[] = {(void*)&bar, (void*)&err, (void*)&spin_limit};
    if (cudaLaunchCooperativeKernel((const void*)k_barrier_timeout, dim3((unsigned)num_sms()), dim3(32), args, 0, st) !=
        cudaSuccess)
      rc = ABM_ERR_CUDA;
  }
  int herr = 0;
  if (rc == ABM_OK && (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
    rc = ABM_ERR_CUDA;
  cudaFree(bar);
  cudaFree(err);
  if (rc != ABM_OK) return rc;
  return herr ? ABM_ERR_DEVICE_TIMEOUT : ABM_OK;
}
