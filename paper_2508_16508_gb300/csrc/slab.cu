// Generic fixed-capacity agent set ("Set", ABMax Section 2) and the selection /
// compaction / distinct-update primitives of Section 4 (Algorithms 1 and 2).
//
// Every rank-matched operation is count -> scatter -> apply over a static
// partition of the slab: pass 1 evaluates the per-slot flags (from 128-bit
// loads of live flags) into bit-planes and per-warp / per-CTA counts; pass 2
// turns a slot's position into its rank (prefix of the CTA counts + prefix of
// the warp counts + a warp scan) and writes rank-ordered slot lists; pass 3
// moves the records. The i-th selected slot receiving the i-th record is
// exactly Rank-Match's pairing (cumsum(mask) * mask on both sides, matched on
// equal nonzero ranks), computed in O(n + k) instead of O(n * k). The passes
// are chained with programmatic dependent launch; no pass spins on another CTA.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>

#include "slab.cuh"

namespace abm {

// SM count per device, looked up once per device (a process may drive
// several GPUs from several host threads: relaxed atomics, idempotent writes)
constexpr int kSmCacheDevices = 64;
static std::atomic<int> g_num_sms[kSmCacheDevices];
int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < kSmCacheDevices) {
    n = g_num_sms[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
  }
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
  if (dev >= 0 && dev < kSmCacheDevices) g_num_sms[dev].store(n, std::memory_order_relaxed);
  return n;
}

constexpr int kSlabThreads = 256;    // default CTA size of the slab passes
constexpr int kMaxFields = 16;



struct PredDev {
  int kind;
  u32 threshold, step, purpose, species;
  const int32_t* mask;
  int field, cmp, and_mask, value;
};

__device__ __forceinline__ bool eval_pred(const PredDev& p, const SlabDev& s, int slot, int live) {
  switch (p.kind) {
    case ABM_PRED_LIVE: return live != 0;
    case ABM_PRED_FREE: return live == 0;
    case ABM_PRED_BERNOULLI:
      return live && draw(s.seed, s.model, p.step, (u32)slot, p.purpose, p.species) < p.threshold;
    case ABM_PRED_MASK: return live && p.mask[slot] != 0;
    case ABM_PRED_FIELD: {
      if (!live) return false;
      const int v = s.fields[(size_t)slot * s.Fp + p.field] & p.and_mask;
      switch (p.cmp) {
        case ABM_CMP_EQ: return v == p.value;
        case ABM_CMP_NE: return v != p.value;
        case ABM_CMP_LT: return v < p.value;
        default: return v >= p.value;
      }
    }
  }
  return false;
}

enum Op { OP_SELECT = 0, OP_REMOVE = 1, OP_ADD = 2, OP_UPDATE = 3, OP_FUSED = 4, OP_ARRAY = 5 };

struct ScanArgs {
  SlabDev s;
  PredDev pred;
  u32* ctrl;               // [1] CTAs finished, [2] epoch (last-CTA-out bookkeeping)
  u32* planeA;             // n/32 words each: selected / free
  u32* planeB;             // chosen (fused call)
  u32* totals;             // [2 * G] per-CTA counts
  u32* wtotals;            // [2 * G * warps] per-warp counts
  int n;                   // slots (or array entries for OP_ARRAY)
  int chunk;               // slots per CTA (a multiple of the sub-tile)
  int G;                   // CTAs = number of chunks
  const int32_t* src;      // OP_ARRAY: mask array
  const int32_t* rec;      // records [k][F]
  const int32_t* rec2;     // OP_FUSED: deltas [k][F]
  int k;
  int op_kind;             // ABM_OP_ADD / ABM_OP_SET for OP_UPDATE
  int id_field;            // OP_ADD
  int use_rec_idx;         // OP_UPDATE with a record mask
  u32 step, threshold;     // OP_FUSED
  u32 rk[20];              // OP_FUSED: Philox round keys of the slab's key (seed, model), round r at 2r, 2r+1
  u32 mk[5];               // OP_FUSED: the call's mask draws' constant parts (mask_pair_consts)
  int32_t* list_a;         // slots by rank: selected / free (caller's out_idx or scratch)
  int32_t* list_b;         // slots by rank: chosen (fused call)
  int32_t* out_count;      // device outputs (nullable)
  int negate;              // OP_SELECT: select where the predicate is false
  const int32_t* list_base;  // OP_SELECT: device offset added to every rank (nullable)
};

// copy or add one record into a slot's fields
__device__ __forceinline__ void apply_record(int32_t* dst, const int32_t* src, int F, bool add) {
  if ((F & 3) == 0 && ((((uintptr_t)src) & 15) == 0)) {
    for (int f = 0; f < F; f += 4) {
      int4 r = *reinterpret_cast<const int4*>(src + f);
      int4* d = reinterpret_cast<int4*>(dst + f);
      if (add) {
        int4 o = *d;
        r.x = (int)((u32)o.x + (u32)r.x);
        r.y = (int)((u32)o.y + (u32)r.y);
        r.z = (int)((u32)o.z + (u32)r.z);
        r.w = (int)((u32)o.w + (u32)r.w);
      }
      *d = r;
    }
  } else {
    for (int f = 0; f < F; ++f) dst[f] = add ? (int)((u32)dst[f] + (u32)src[f]) : src[f];
  }
}

template <int THREADS>
__device__ __forceinline__ void block_sum2(u32& a, u32& b, u64* s_red) {
  u64 v = ((u64)a << 32) | b;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  u64 t = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) t += s_red[w];
  a = (u32)(t >> 32);
  b = (u32)t;
}

// 32-byte (256-bit) global accesses: one instruction moves a whole 8-field
// row, so a row written to DRAM is one full sector (two 16-byte stores to a
// sector make L2 fetch it first when the first half arrives alone)
__device__ __forceinline__ void ld_v8_nc(const int32_t* p, int (&r)[8]) {
  asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(p));
}
__device__ __forceinline__ void ld_v8(const int32_t* p, int (&r)[8]) {
  asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st_v8(int32_t* p, const int (&r)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(r[0]), "r"(r[1]), "r"(r[2]),
               "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// Flags live in two bit-planes of one bit per slot: A = selected / free,
// B = chosen (fused call); word w of a plane covers slots [32w, 32w + 32).
//
// Both passes use the same static partition: CTA b owns the slots
// [b*chunk, (b+1)*chunk) and warp w of it the contiguous segment
// [b*chunk + w*seg, ... + seg), seg a multiple of 512 slots. In each 512-slot
// step, lane l handles the 16 consecutive slots [16l, 16l + 16).
constexpr int kLaneSlots = 16;
constexpr int kWarpStep = 32 * kLaneSlots;

// Pass 1: flags from four 128-bit loads of live flags per lane; the lane's
// 16-bit masks are paired with the neighbour lane's into plane words.
template <int OP, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_count(ScanArgs a) {
  constexpr int WARPS = THREADS / 32;
  __shared__ u64 s_red[WARPS];
  const SlabDev& s = a.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = a.chunk / WARPS;
  const int wlo = blockIdx.x * a.chunk + warp * seg;
  const int whi = min(a.n, wlo + seg);
  const int32_t* flag_src = OP == OP_ARRAY ? a.src : s.active;
  const bool vec = (((uintptr_t)flag_src) & 15) == 0;  // a caller's mask array may start anywhere
  u32 ca = 0, cb = 0;
  for (int b0 = wlo; b0 < whi; b0 += kWarpStep) {
    const int base = b0 + lane * kLaneSlots;
    int live[kLaneSlots];
#pragma unroll
    for (int v = 0; v < kLaneSlots / 4; ++v) {
      const int b = base + 4 * v;
      int4 q = make_int4(0, 0, 0, 0);
      if (vec && b + 3 < a.n) {
        q = *reinterpret_cast<const int4*>(flag_src + b);
      } else {
        if (b + 0 < a.n) q.x = flag_src[b + 0];
        if (b + 1 < a.n) q.y = flag_src[b + 1];
        if (b + 2 < a.n) q.z = flag_src[b + 2];
        if (b + 3 < a.n) q.w = flag_src[b + 3];
      }
      live[4 * v + 0] = q.x; live[4 * v + 1] = q.y; live[4 * v + 2] = q.z; live[4 * v + 3] = q.w;
    }
    u32 ma = 0, mb = 0, mr = 0;  // 16-bit masks over the lane's slots
#pragma unroll
    for (int j = 0; j < kLaneSlots; ++j) {
      const int slot = base + j;
      bool f = false;
      if (slot < a.n) {
        if (OP == OP_ARRAY) f = live[j] != 0;
        else if (OP == OP_ADD) f = live[j] == 0;
        else f = eval_pred(a.pred, s, slot, live[j]) != (a.negate != 0);
      }
      ma |= (u32)f << j;
    }
    if (OP == OP_REMOVE) mr = ma;
    // removed slots become placeholders now: rewrite only the 4-slot groups
    // that changed (the other flags keep their values)
    if (OP == OP_REMOVE) {
#pragma unroll
      for (int v = 0; v < kLaneSlots / 4; ++v) {
        const u32 g = (mr >> (4 * v)) & 0xFu;
        if (!g) continue;
        const int b = base + 4 * v;
        const int4 q = make_int4((g & 1u) ? 0 : live[4 * v], (g & 2u) ? 0 : live[4 * v + 1],
                                 (g & 4u) ? 0 : live[4 * v + 2], (g & 8u) ? 0 : live[4 * v + 3]);
        if (b + 3 < a.n) {
          *reinterpret_cast<int4*>(s.active + b) = q;
        } else {
          if (b + 0 < a.n) s.active[b + 0] = q.x;
          if (b + 1 < a.n) s.active[b + 1] = q.y;
          if (b + 2 < a.n) s.active[b + 2] = q.z;
        }
      }
    }
    ca += __popc(ma);
    cb += __popc(mb);
    if (OP != OP_REMOVE) {
      const u32 na = __shfl_down_sync(0xFFFFFFFFu, ma, 1);
      if (!(lane & 1) && base < a.n) a.planeA[base >> 5] = ma | (na << 16);
    }
  }
  u64 v = ((u64)ca << 32) | cb;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) {
    a.wtotals[2 * (blockIdx.x * WARPS + warp)] = (u32)(v >> 32);
    a.wtotals[2 * (blockIdx.x * WARPS + warp) + 1] = (u32)v;
  }
  block_sum2<THREADS>(ca, cb, s_red);
  if (threadIdx.x == 0) {
    a.totals[2 * blockIdx.x] = ca;
    a.totals[2 * blockIdx.x + 1] = cb;
  }
  if (OP == OP_REMOVE) {
    if (last_cta_out(a.ctrl)) {
      int A = 0;
      for (int b = 0; b < a.G; ++b) A += (int)a.totals[2 * b];
      s.counters[0] -= A;
      if (a.out_count) *a.out_count = A;
      __threadfence();
    }
  }
}

// The selective-update call's mask draws are Philox4x32-10 blocks on the
// counter (step, j, MASK, 0), j = slot >> 1: only the second word varies
// within a call, so the first round, one multiply of the second and one of
// the third depend on the call alone. mask_pair_consts works them out on the
// host (round r: (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)), M0 = 0xD2511F53, M1 = 0xCD9E8D57, round keys k = rk); the
// device finishes the block from them. Same outputs as philox_rk.
static void mask_pair_consts(u32 step, const u32 (&rk)[20], u32 (&mk)[5]) {
  const auto wide = [](u32 m, u32 x, u32& hi, u32& lo) {
    const uint64_t p = (uint64_t)m * (uint64_t)x;
    hi = (u32)(p >> 32);
    lo = (u32)p;
  };
  u32 h0, l0, h1, l1;
  // round 0 on (step, j, MASK, 0) -> (A ^ j, B, C, D)
  wide(0xD2511F53u, step, h0, l0);
  wide(0xCD9E8D57u, (u32)ABM_P_MASK, h1, l1);
  const u32 A = h1 ^ rk[0], B = l1, C = h0 ^ 0u ^ rk[1], D = l0;
  // round 1: the third word C is constant -> (E, F, hi(M0 (A ^ j)) ^ G, lo(M0 (A ^ j)))
  wide(0xCD9E8D57u, C, h1, l1);
  const u32 E = h1 ^ B ^ rk[2], F = l1, G = D ^ rk[3];
  // round 2: the first word E is constant -> (hi(M1 z) ^ H, lo(M1 z), I ^ w, J)
  wide(0xD2511F53u, E, h0, l0);
  mk[0] = A;
  mk[1] = G;
  mk[2] = F ^ rk[4];  // H
  mk[3] = h0 ^ rk[5];  // I
  mk[4] = l0;          // J
}

__device__ __forceinline__ uint4 mask_pair_draw(u32 j, const u32 (&mk)[5], const u32 (&rk)[20]) {
  const u32 x = mk[0] ^ j;                                         // round 0
  const u32 a_lo = 0xD2511F53u * x, a_hi = __umulhi(0xD2511F53u, x);  // round 1
  const u32 z = a_hi ^ mk[1];
  const u32 b_lo = 0xCD9E8D57u * z, b_hi = __umulhi(0xCD9E8D57u, z);  // round 2
  uint4 c = make_uint4(b_hi ^ mk[2], b_lo, mk[3] ^ a_lo, mk[4]);
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const u32 p0_lo = 0xD2511F53u * c.x, p0_hi = __umulhi(0xD2511F53u, c.x);
    const u32 p1_lo = 0xCD9E8D57u * c.z, p1_hi = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(p1_hi ^ c.y ^ rk[2 * r], p1_lo, p0_hi ^ c.w ^ rk[2 * r + 1], p0_lo);
  }
  return c;
}

// Pass 1 of the selective-update call: as k_count, with the live flags as a
// 16-bit mask per lane (any nonzero flag is live) read by two 32-byte loads
// and written back as 0/1 in whole 8-slot (32-byte) groups; the lane's eight
// draws are independent and all in flight together. The pass is bound by the
// Philox draws (one per pair of slots): fewer draws in flight at a higher
// occupancy measured slower.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_count_fused(ScanArgs a) {
  constexpr int WARPS = THREADS / 32;
  __shared__ u64 s_red[WARPS];
  const SlabDev& s = a.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = a.chunk / WARPS;
  const int wlo = blockIdx.x * a.chunk + warp * seg;
  const int whi = min(a.n, wlo + seg);
  u32 ca = 0, cb = 0;
  for (int b0 = wlo; b0 < whi; b0 += kWarpStep) {
    const int base = b0 + lane * kLaneSlots;
    // the selective-update call: live flags as a 16-bit mask (any nonzero
    // flag is live), read with two 32-byte loads, written back as 0/1 in
    // whole 8-slot (32-byte) groups
    u32 ml = 0;
    if (base + kLaneSlots <= a.n) {
      int f[8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        ld_v8(s.active + base + 8 * h, f);
#pragma unroll
        for (int j = 0; j < 8; ++j) ml |= (u32)(f[j] != 0) << (8 * h + j);
      }
    } else {
      for (int j = 0; j < kLaneSlots; ++j)
        if (base + j < a.n) ml |= (u32)(s.active[base + j] != 0) << j;
    }
    // the draws' outcomes as 16-bit masks (bit j: slot base + j), combined
    // with the live mask once per 16 slots
    u32 dr = 0, dc = 0;
#pragma unroll
    for (int m = 0; m < kLaneSlots / 2; ++m) {
      const int slot = base + 2 * m;
      // slots 2j and 2j+1 share draw j: words (x, y) and (z, w) = (remove, choose)
      const uint4 u = mask_pair_draw((u32)slot >> 1, a.mk, a.rk);
      dr |= (u.x < a.threshold ? 1u << (2 * m) : 0u) | (u.z < a.threshold ? 2u << (2 * m) : 0u);
      dc |= (u.y < a.threshold ? 1u << (2 * m) : 0u) | (u.w < a.threshold ? 2u << (2 * m) : 0u);
    }
    const u32 valid = base + kLaneSlots <= a.n ? 0xFFFFu : (base < a.n ? (1u << (a.n - base)) - 1u : 0u);
    const u32 mr = ml & dr;         // removed: live and drawn
    const u32 al = ml & ~dr;        // still live
    const u32 ma = valid & ~al;     // free after the removals
    const u32 mb = al & dc;         // chosen among the live
    const u32 nl = ml & ~mr;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!((mr >> (8 * h)) & 0xFFu)) continue;
      const int b = base + 8 * h;
      if (b + 8 <= a.n) {
        int f[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = (int)((nl >> (8 * h + j)) & 1u);
        st_v8(s.active + b, f);
      } else {
        for (int j = 0; j < 8; ++j)
          if (b + j < a.n) s.active[b + j] = (int)((nl >> (8 * h + j)) & 1u);
      }
    }
    ca += __popc(ma);
    cb += __popc(mb);
    const u32 na = __shfl_down_sync(0xFFFFFFFFu, ma, 1);
    const u32 nb = __shfl_down_sync(0xFFFFFFFFu, mb, 1);
    if (!(lane & 1) && base < a.n) {
      a.planeA[base >> 5] = ma | (na << 16);
      a.planeB[base >> 5] = mb | (nb << 16);
    }
  }
  u64 v = ((u64)ca << 32) | cb;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) {
    a.wtotals[2 * (blockIdx.x * WARPS + warp)] = (u32)(v >> 32);
    a.wtotals[2 * (blockIdx.x * WARPS + warp) + 1] = (u32)v;
  }
  block_sum2<THREADS>(ca, cb, s_red);
  if (threadIdx.x == 0) {
    a.totals[2 * blockIdx.x] = ca;
    a.totals[2 * blockIdx.x + 1] = cb;
  }
}

// Pass 2: ranks from the CTA prefix + warp prefix + a warp scan per step.
// Each 512-slot step of a warp stages its flagged slots in shared memory in
// rank order (each lane writes its own, 16 slots at most) and the warp copies
// them out coalesced; steps with no rank below the limit are skipped. The add
// passes also write the final live flags of every 16-slot group that receives
// a new agent, whole (0/1), so no flag sector is written in part.
// The selective-update call's records moved by the pass that ranks them:
// the staged slots [0, n) of a warp step take records r0 + i (ADDROW: added
// to the row, wrapping), two 32-byte rows per lane in flight. With a slab
// that is mostly live, free and chosen slots spread evenly over it, so the
// static slot partition also balances the record moves.
template <bool ADDROW>
__device__ __forceinline__ void move_staged(const ScanArgs& a, const int* stage, u32 n, u32 r0, const int32_t* rec,
                                            int lane) {
  constexpr int U = 2;
  for (u32 i0 = lane; i0 < n; i0 += 32 * U) {
    int slot[U];
    int r[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const u32 i = i0 + 32 * u;
      slot[u] = -1;
      if (i < n) {
        slot[u] = stage[i];
        if (!in_range(slot[u], a.s.cap, a.s.err)) slot[u] = -1;
        ld_v8_nc(rec + (size_t)(r0 + i) * 8, r[u]);
      }
    }
    if (ADDROW) {
      int o[U][8];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (slot[u] >= 0) ld_v8(a.s.fields + (size_t)slot[u] * 8, o[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int f = 0; f < 8; ++f) r[u][f] = (int)((u32)o[u][f] + (u32)r[u][f]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (slot[u] >= 0) st_v8(a.s.fields + (size_t)slot[u] * 8, r[u]);
  }
}

// MOVE (selective-update call, 8 fields, 32-byte aligned records): the pass
// moves the records itself instead of writing the rank-ordered slot lists, and
// no apply pass follows.
template <int OP, int THREADS, bool MOVE = false>
__global__ void __launch_bounds__(THREADS, MOVE ? (768 / THREADS > 0 ? 768 / THREADS : 1) : 1) k_scatter(ScanArgs a) {
  constexpr int WARPS = THREADS / 32;
  __shared__ u64 s_red[WARPS];
  __shared__ int s_stage[WARPS * kWarpStep];
  griddep_wait();
  const SlabDev& s = a.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = a.chunk / WARPS;
  const int wlo = blockIdx.x * a.chunk + warp * seg;
  const int whi = min(a.n, wlo + seg);
  // the plane words of the warp's first step, requested ahead of the prefix
  // sums; each step then requests the next step's words before its own work,
  // so a warp waits for one round trip in all, not one per step
  u32 wa_next = 0, wb_next = 0;
  {
    const int base = wlo + lane * kLaneSlots;
    if (wlo < whi && base < a.n) {
      wa_next = a.planeA[base >> 5];
      if (OP == OP_FUSED) wb_next = a.planeB[base >> 5];
    }
  }
  u32 pa = 0, pb = 0, ta = 0, tb = 0;
  for (int j = threadIdx.x; j < a.G; j += THREADS) {
    const u32 x = a.totals[2 * j], y = a.totals[2 * j + 1];
    if (j < (int)blockIdx.x) {
      pa += x;
      pb += y;
    }
    ta += x;
    tb += y;
  }
  block_sum2<THREADS>(pa, pb, s_red);
  block_sum2<THREADS>(ta, tb, s_red);
  {
    u32 x = 0, y = 0;
    if (lane < warp) {
      x = a.wtotals[2 * (blockIdx.x * WARPS + lane)];
      y = a.wtotals[2 * (blockIdx.x * WARPS + lane) + 1];
    }
    u64 v = ((u64)x << 32) | y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    pa += (u32)(v >> 32);
    pb += (u32)v;
  }
  const int nrec = (OP == OP_UPDATE && a.use_rec_idx) ? s.counters[3] : a.k;
  const u32 limit = (u32)(OP == OP_UPDATE ? nrec : (OP == OP_SELECT || OP == OP_ARRAY ? 0x7FFFFFFF : a.k));
  const u32 limit_b = (u32)a.k;
  // ranks land at list_a + *list_base (the permutation's second half)
  int32_t* const list_a = a.list_a + (OP == OP_SELECT && a.list_base ? *a.list_base : 0);
  int* const stage = s_stage + warp * kWarpStep;
  for (int b0 = wlo; b0 < whi; b0 += kWarpStep) {
    const int base = b0 + lane * kLaneSlots;
    const u32 wa = wa_next, wb = wb_next;
    {
      const int nbase = base + kWarpStep;
      wa_next = wb_next = 0;
      if (b0 + kWarpStep < whi && nbase < a.n) {
        wa_next = a.planeA[nbase >> 5];
        if (OP == OP_FUSED) wb_next = a.planeB[nbase >> 5];
      }
    }
    u32 ma = 0, mb = 0;
    if (base < a.n) {
      ma = (wa >> (16 * (lane & 1))) & 0xFFFFu;
      if (OP == OP_FUSED) mb = (wb >> (16 * (lane & 1))) & 0xFFFFu;
    }
    const u32 c = (u32)__popc(ma) | ((u32)__popc(mb) << 16);
    u32 inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += t;
    }
    const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const u32 ex = inc - c;
    const u32 sa = pa, sb = pb;  // ranks of the step's first flagged slots
    pa += tot & 0xFFFFu;
    pb += tot >> 16;
    // plane A: the step's ranks [sa, sa + na) are below the limit
    if (sa < limit && (tot & 0xFFFFu)) {
      const u32 na = min(tot & 0xFFFFu, limit - sa);
      const u32 off = ex & 0xFFFFu;
      // plane A is dense: every flagged slot of the lane goes to its place
      // below na, unrolled (no loop over the set bits)
#pragma unroll
      for (int j = 0; j < kLaneSlots; ++j) {
        const u32 pos = off + (u32)__popc(ma & ((1u << j) - 1u));
        if (((ma >> j) & 1u) && pos < na) stage[pos] = base + j;
      }
      __syncwarp();
      if constexpr (MOVE) move_staged<false>(a, stage, na, sa, a.rec, lane);
      else for (u32 i = lane; i < na; i += 32) list_a[sa + i] = stage[i];
      if (OP == OP_ADD || OP == OP_FUSED) {
        // flags of the lane's 16 slots after the adds: live 1, free 0, and the
        // free slots with a rank below the limit 1
        const u32 mine = (ex & 0xFFFFu) < na ? min((u32)__popc(ma), na - (ex & 0xFFFFu)) : 0u;
        if (mine) {
          const u32 added = mine == (u32)__popc(ma) ? ma : ma & ((1u << __fns(ma, 0, (int)mine + 1)) - 1u);
          const u32 valid = base + kLaneSlots <= a.n ? 0xFFFFu : (1u << (a.n - base)) - 1u;
          const u32 nl = ((~ma & valid) | added) & valid;
          if (valid == 0xFFFFu) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              int f[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) f[j] = (int)((nl >> (8 * h + j)) & 1u);
              st_v8(s.active + base + 8 * h, f);
            }
          } else {
            for (int j = 0; j < kLaneSlots; ++j)
              if ((valid >> j) & 1u) s.active[base + j] = (int)((nl >> j) & 1u);
          }
        }
      }
      __syncwarp();  // the stage is rewritten next
    }
    // plane B (the fused call's chosen survivors), the same way
    if (OP == OP_FUSED && sb < limit_b && (tot >> 16)) {
      const u32 nb = min(tot >> 16, limit_b - sb);
      u32 off = ex >> 16;
      u32 m = mb;
      while (m && off < nb) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        stage[off++] = base + j;
      }
      __syncwarp();
      if constexpr (MOVE) move_staged<true>(a, stage, nb, sb, a.rec2, lane);
      else for (u32 i = lane; i < nb; i += 32) a.list_b[sb + i] = stage[i];
      __syncwarp();
    }
  }
  if (last_cta_out(a.ctrl)) {
    const int A = (int)ta, B = (int)tb;
    if (OP == OP_SELECT || OP == OP_ARRAY) {
      if (a.out_count) *a.out_count = A;
      if (OP == OP_ARRAY) s.counters[3] = A;
    } else if (OP == OP_ADD) {
      const int r = min(a.k, A);
      s.meta[0] = r;
      s.meta[1] = 0;
      s.meta[2] = s.counters[1];  // first id of this batch
      s.counters[0] += r;
      if (a.id_field >= 0) s.counters[1] += r;
      if (a.k > A) s.counters[2] = 1;
      if (a.out_count) *a.out_count = r;
    } else if (OP == OP_UPDATE) {
      const int r = min(A, nrec);
      s.meta[0] = r;
      s.meta[1] = 0;
      if (a.out_count) *a.out_count = r;
    } else if (OP == OP_FUSED) {  // A = free after removal, B = chosen survivors
      const int n_before = s.counters[0];
      const int added = min(a.k, A);
      s.meta[0] = added;
      s.meta[1] = min(a.k, B);
      s.counters[0] = s.cap - A + added;
      if (a.k > A) s.counters[2] = 1;
      if (a.out_count) {
        a.out_count[0] = A - (s.cap - n_before);
        a.out_count[1] = added;
        a.out_count[2] = min(a.k, B);
      }
    }
    __threadfence();
  }
}

// Whole 8-field rows, 32-byte aligned: records [j0, j1) of `rec` (or their
// rec_idx entries) go to the slots list[j], U rows in flight per thread, all
// loads issued before the stores. ADDROW: the slot's row is read and the
// record added to it field-wise (wrapping).
template <int U, bool ADDROW, bool STAMP, bool IDX>
__device__ __forceinline__ void move_rows_v8(const ScanArgs& a, const int32_t* rec, const int32_t* list, int j1,
                                             int id_field, int id0) {
  const SlabDev& s = a.s;
  const int stride = gridDim.x * blockDim.x;
  for (int j0 = blockIdx.x * blockDim.x + threadIdx.x; j0 < j1; j0 += U * stride) {
    int slot[U];
    int r[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * stride;
      slot[u] = -1;
      if (j < j1) {
        slot[u] = list[j];
        if (!in_range(slot[u], s.cap, s.err)) slot[u] = -1;
        ld_v8_nc(rec + (size_t)(IDX ? s.rec_idx[j] : j) * 8, r[u]);
      }
    }
    if (ADDROW) {
      int o[U][8];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (slot[u] >= 0) ld_v8(s.fields + (size_t)slot[u] * 8, o[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int f = 0; f < 8; ++f) r[u][f] = (int)((u32)o[u][f] + (u32)r[u][f]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (slot[u] < 0) continue;
      if (STAMP) {  // the id of an added agent: next id + its rank
        const int id = (int)((u32)id0 + (u32)(j0 + u * stride));
#pragma unroll
        for (int f = 0; f < 8; ++f)
          if (f == id_field) r[u][f] = id;
      }
      st_v8(s.fields + (size_t)slot[u] * 8, r[u]);
    }
  }
}

// Pass 3: record j goes to (or is added to) the slot at rank j, four records
// per thread in flight, all loads issued before the stores; coalesced record
// reads, one field run written per slot (one 32-byte store for 8 fields).
// Two CTAs of 256 threads per SM (96 registers) measured faster than three
// with two rows in flight where rows are read.
template <int OP>
__global__ void __launch_bounds__(256, 2) k_apply(ScanArgs a) {
  griddep_wait();
  const SlabDev& s = a.s;
  const int ra = s.meta[0], rb = s.meta[1];
  const int id0 = s.meta[2];
  const int total = ra + rb;
  const int stride = gridDim.x * blockDim.x;
  const bool f8 = s.F == 8 && s.Fp == 8 && ((((uintptr_t)a.rec) | ((uintptr_t)a.rec2)) & 15) == 0;
  // 8 fields, records 32-byte aligned (the rows always are): whole rows per instruction
  if (f8 && ((((uintptr_t)a.rec) | ((uintptr_t)a.rec2) | ((uintptr_t)s.fields)) & 31) == 0) {
    if (OP == OP_UPDATE) {
      const bool idx = a.use_rec_idx != 0;
      if (a.op_kind == ABM_OP_ADD) {
        if (idx) move_rows_v8<4, true, false, true>(a, a.rec, a.list_a, ra, -1, 0);
        else move_rows_v8<4, true, false, false>(a, a.rec, a.list_a, ra, -1, 0);
      } else {
        if (idx) move_rows_v8<4, false, false, true>(a, a.rec, a.list_a, ra, -1, 0);
        else move_rows_v8<4, false, false, false>(a, a.rec, a.list_a, ra, -1, 0);
      }
    } else if (OP == OP_ADD && a.id_field >= 0) {
      move_rows_v8<4, false, true, false>(a, a.rec, a.list_a, ra, a.id_field, id0);
    } else {
      move_rows_v8<4, false, false, false>(a, a.rec, a.list_a, ra, -1, 0);
    }
    if (OP == OP_FUSED) move_rows_v8<4, true, false, false>(a, a.rec2, a.list_b, rb, -1, 0);
    return;
  }
  for (int j0 = blockIdx.x * blockDim.x + threadIdx.x; j0 < total; j0 += 4 * stride) {
    if (f8) {
      int slot[4];
      int4 r0[4], r1[4];
      bool add[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u * stride;
        slot[u] = -1;
        add[u] = false;
        if (j < total) {
          const int32_t* src;
          if (j < ra) {
            slot[u] = a.list_a[j];
            const int rj = (OP == OP_UPDATE && a.use_rec_idx) ? s.rec_idx[j] : j;
            src = a.rec + (size_t)rj * 8;
            add[u] = OP == OP_UPDATE && a.op_kind == ABM_OP_ADD;
          } else {
            slot[u] = a.list_b[j - ra];
            src = a.rec2 + (size_t)(j - ra) * 8;
            add[u] = true;
          }
          r0[u] = __ldg(reinterpret_cast<const int4*>(src));
          r1[u] = __ldg(reinterpret_cast<const int4*>(src) + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (slot[u] < 0) continue;
        int4* d = reinterpret_cast<int4*>(s.fields + (size_t)slot[u] * 8);
        if (OP == OP_ADD && a.id_field >= 0) {  // stamp the id into the record before storing it
          const int j = j0 + u * stride;
          const int id = (int)((u32)id0 + (u32)j);
          int4& r = a.id_field < 4 ? r0[u] : r1[u];
          switch (a.id_field & 3) {
            case 0: r.x = id; break;
            case 1: r.y = id; break;
            case 2: r.z = id; break;
            default: r.w = id; break;
          }
        }
        if (add[u]) {
          const int4 o0 = d[0], o1 = d[1];
          r0[u] = make_int4((int)((u32)o0.x + (u32)r0[u].x), (int)((u32)o0.y + (u32)r0[u].y),
                            (int)((u32)o0.z + (u32)r0[u].z), (int)((u32)o0.w + (u32)r0[u].w));
          r1[u] = make_int4((int)((u32)o1.x + (u32)r1[u].x), (int)((u32)o1.y + (u32)r1[u].y),
                            (int)((u32)o1.z + (u32)r1[u].z), (int)((u32)o1.w + (u32)r1[u].w));
        }
        d[0] = r0[u];
        d[1] = r1[u];
      }
      continue;
    }
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u * stride;
      if (j >= total) break;
      if (j < ra) {
        const int slot = a.list_a[j];
        int32_t* dst = s.fields + (size_t)slot * s.Fp;
        if (OP == OP_UPDATE) {
          const int rj = a.use_rec_idx ? s.rec_idx[j] : j;
          apply_record(dst, a.rec + (size_t)rj * s.F, s.F, a.op_kind == ABM_OP_ADD);
        } else {
          apply_record(dst, a.rec + (size_t)j * s.F, s.F, false);
          if (OP == OP_ADD && a.id_field >= 0) dst[a.id_field] = (int)((u32)id0 + (u32)j);
        }
      } else {
        const int i = j - ra;
        apply_record(s.fields + (size_t)a.list_b[i] * s.Fp, a.rec2 + (size_t)i * s.F, s.F, true);
      }
    }
  }
}

// --------------------------------------------------------------------------
// check builds: the fields past the capacity hold the canary, the live flags
// there stay 0; k_canary_check records kErrCheck if either changed
__global__ void k_canary_fill(int32_t* fields, int Fp, int cap, int n_pad) {
  const long long n = (long long)(n_pad - cap) * Fp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    fields[(long long)cap * Fp + i] = kCanary;
}

__global__ void k_canary_check(const int32_t* active, const int32_t* fields, int Fp, int cap, int n_pad, int* err) {
  const long long n = (long long)(n_pad - cap) * Fp;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= fields[(long long)cap * Fp + i] != kCanary;
  for (int i = cap + blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
    bad |= active[i] != 0;
  if (bad) atomicCAS(err, 0, kErrCheck);
}

__global__ void k_check_index(long long i, long long n, int* err) { in_range(i, n, err); }

__global__ void k_slab_init(SlabDev s, int init, int n_pad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
    const bool inside = i < s.cap;
    int live = 0;
    if (inside && init == ABM_INIT_HALF_LIVE)
      live = draw(s.seed, s.model, ABM_INIT_STEP, (u32)i, ABM_P_INIT_ACTIVE, 0u) < 0x80000000u;
    s.active[i] = live;
    int32_t* dst = s.fields + (size_t)i * s.Fp;
    uint4 w0 = make_uint4(0, 0, 0, 0), w1 = w0, w2 = w0, w3 = w0;
    if (inside && init == ABM_INIT_HALF_LIVE) {
      w0 = draw4(s.seed, s.model, ABM_INIT_STEP, (u32)i, ABM_P_NEWREC0, 0u);
      if (s.F > 4) w1 = draw4(s.seed, s.model, ABM_INIT_STEP, (u32)i, ABM_P_NEWREC1, 0u);
      if (s.F > 8) w2 = draw4(s.seed, s.model, ABM_INIT_STEP, (u32)i, ABM_P_NEWREC1 + 1, 0u);
      if (s.F > 12) w3 = draw4(s.seed, s.model, ABM_INIT_STEP, (u32)i, ABM_P_NEWREC1 + 2, 0u);
    }
    const uint4 w[4] = {w0, w1, w2, w3};
    for (int f = 0; f < s.Fp; f += 4) {
      const uint4 q = f < s.F ? w[f >> 2] : make_uint4(0, 0, 0, 0);
      int4 o = make_int4((int)q.x, (int)q.y, (int)q.z, (int)q.w);
      if (f + 1 >= s.F) o.y = 0;
      if (f + 2 >= s.F) o.z = 0;
      if (f + 3 >= s.F) o.w = 0;
      if (f >= s.F) o.x = 0;
      *reinterpret_cast<int4*>(dst + f) = o;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s.counters[1] = 0;
    s.counters[2] = 0;
    s.counters[3] = 0;
  }
}

// n_active after init (a plain count)
__global__ void k_count_live(SlabDev s) {
  int c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.cap; i += gridDim.x * blockDim.x)
    c += s.active[i] != 0;
  warp_add(&s.counters[0], c);
}

__global__ void k_philox_records(SlabDev s, u32 step, u32 p0, u32 p1, int k, int32_t* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
    int32_t* dst = out + (size_t)j * s.F;
    const uint4 a = draw4(s.seed, s.model, step, (u32)j, p0, 0u);
    const u32 wa[4] = {a.x, a.y, a.z, a.w};
    uint4 b = make_uint4(0, 0, 0, 0);
    if (s.F > 4) b = draw4(s.seed, s.model, step, (u32)j, p1, 0u);
    const u32 wb[4] = {b.x, b.y, b.z, b.w};
    for (int f = 0; f < s.F && f < 8; ++f) dst[f] = (int)(f < 4 ? wa[f] : wb[f - 4]);
  }
}

}  // namespace abm

// ============================================================================
// host side
using namespace abm;



extern "C" const char* abm_strerror(abm_status st) {
  switch (st) {
    case ABM_OK: return "ok";
    case ABM_ERR_ARG: return "invalid argument";
    case ABM_ERR_OOM: return "device allocation failed";
    case ABM_ERR_CUDA: return "CUDA runtime error";
    case ABM_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case ABM_ERR_OVERFLOW: return "more agents asked for a slot than were free";
    case ABM_ERR_STATE: return "operation not valid for this handle";
    case ABM_ERR_TOO_LARGE: return "size beyond the fixed maximum of this entry point";
    case ABM_ERR_CHECK: return "check build: an index out of range or a damaged canary was recorded";
  }
  return "unknown status";
}

extern "C" int32_t abm_version(void) { return kCheck ? -101 : 101; }

static void slab_free(abm_slab* s) {
  if (!s->view) {
    cudaFree(s->d.active);
    cudaFree(s->d.fields);
  }
  cudaFree(s->d.counters);
  cudaFree(s->d.rec_idx);
  cudaFree(s->d.err);
  cudaFree(s->planes);
  cudaFree(s->planes2);
  cudaFree(s->totals);
  cudaFree(s->totals2);
  cudaFree(s->wtotals);
  cudaFree(s->wtotals2);
  cudaFree(s->lista);
  cudaFree(s->listb);
  cudaFree(s->d.meta);
  cudaFree(s->ctrl);
  sort_scratch_free(s->sort);
  delete s;
}

extern "C" abm_status abm_slab_destroy(abm_slab* s) {
  if (!s) return ABM_ERR_ARG;
  if (s->view) return ABM_ERR_STATE;  // a world's view lives as long as the world
  slab_free(s);
  return ABM_OK;
}

void abm::slab_free_view(abm_slab* s) {
  if (s) slab_free(s);
}

// host part of slab creation: the struct, its scratch and counters, and the
// live flags and fields unless they are borrowed (active != nullptr)
static abm_status slab_alloc(int capacity, int n_fields, u32 seed, u32 model, int32_t* active, int32_t* fields,
                             abm_slab** out) {
  abm_slab* s = new (std::nothrow) abm_slab();
  if (!s) return ABM_ERR_OOM;
  std::memset(s, 0, sizeof(*s));
  s->d.cap = capacity;
  s->d.F = n_fields;
  s->d.Fp = (n_fields + 3) & ~3;
  s->d.seed = seed;
  s->d.model = model;
  s->n_pad = ((capacity + kSlabTileMax - 1) / kSlabTileMax) * kSlabTileMax;
  s->max_ctas = num_sms() * 16;
  s->fused_threads = 256;
  s->fused_ctas_per_sm = 8;
  s->view = active != nullptr;
  bool ok = true;
  if (s->view) {
    s->d.active = active;
    s->d.fields = fields;
  } else {
    ok = cudaMalloc(&s->d.active, sizeof(int32_t) * (size_t)s->n_pad) == cudaSuccess &&
         cudaMalloc(&s->d.fields, sizeof(int32_t) * (size_t)s->n_pad * s->d.Fp) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&s->d.counters, sizeof(int32_t) * 4) == cudaSuccess &&
            cudaMalloc(&s->d.rec_idx, sizeof(int32_t) * (size_t)capacity) == cudaSuccess &&
            cudaMalloc(&s->d.err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&s->planes, sizeof(u32) * 2 * (size_t)(s->n_pad / 32)) == cudaSuccess &&
            cudaMalloc(&s->planes2, sizeof(u32) * (size_t)(s->n_pad / 32)) == cudaSuccess &&
            cudaMalloc(&s->totals, sizeof(u32) * 2 * (size_t)s->max_ctas) == cudaSuccess &&
            cudaMalloc(&s->totals2, sizeof(u32) * 2 * (size_t)s->max_ctas) == cudaSuccess &&
            cudaMalloc(&s->wtotals, sizeof(u32) * 32 * (size_t)s->max_ctas) == cudaSuccess &&
            cudaMalloc(&s->wtotals2, sizeof(u32) * 32 * (size_t)s->max_ctas) == cudaSuccess &&
            cudaMalloc(&s->lista, sizeof(int32_t) * (size_t)capacity) == cudaSuccess &&
            cudaMalloc(&s->listb, sizeof(int32_t) * (size_t)capacity) == cudaSuccess &&
            cudaMalloc(&s->d.meta, sizeof(int32_t) * 4) == cudaSuccess &&
            cudaMalloc(&s->ctrl, sizeof(u32) * 8) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    slab_free(s);
    return ABM_ERR_OOM;
  }
  *out = s;
  return ABM_OK;
}

abm_status abm::slab_create_view(int cap, u32 seed, u32 model, int32_t* active, int32_t* fields, abm_slab** out) {
  if (!active || !fields || !out || cap < 1 || cap > (1 << 28) - 1) return ABM_ERR_ARG;
  abm_slab* s = nullptr;
  const abm_status e = slab_alloc(cap, 4, seed, model, active, fields, &s);
  if (e != ABM_OK) return e;
  // zeroed synchronously: a view is made once, outside any stream order
  if (cudaMemset(s->d.counters, 0, sizeof(int32_t) * 4) != cudaSuccess ||
      cudaMemset(s->d.err, 0, sizeof(int)) != cudaSuccess || cudaMemset(s->ctrl, 0, sizeof(u32) * 8) != cudaSuccess) {
    slab_free(s);
    return ABM_ERR_CUDA;
  }
  *out = s;
  return ABM_OK;
}

extern "C" abm_status abm_slab_create(int32_t capacity, int32_t n_fields, uint32_t seed,
                                      uint32_t model, int32_t init, void* stream, abm_slab** out) {
  if (!out || capacity < 1 || capacity > (1 << 28) - 1 || n_fields < 1 || n_fields > kMaxFields ||
      (init != ABM_INIT_EMPTY && init != ABM_INIT_HALF_LIVE))
    return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  abm_slab* s = nullptr;
  const abm_status e = slab_alloc(capacity, n_fields, seed, model, nullptr, nullptr, &s);
  if (e != ABM_OK) return e;
  if (cudaMemsetAsync(s->d.counters, 0, sizeof(int32_t) * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->d.err, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(s->ctrl, 0, sizeof(u32) * 8, st) != cudaSuccess) {
    slab_free(s);
    return ABM_ERR_CUDA;
  }
  k_slab_init<<<num_sms() * 4, 256, 0, st>>>(s->d, init, s->n_pad);
  k_count_live<<<num_sms() * 4, 256, 0, st>>>(s->d);
  if (kCheck) k_canary_fill<<<num_sms() * 4, 256, 0, st>>>(s->d.fields, s->d.Fp, s->d.cap, s->n_pad);
  if (cudaGetLastError() != cudaSuccess) {
    slab_free(s);
    return ABM_ERR_CUDA;
  }
  *out = s;
  return ABM_OK;
}

extern "C" abm_status abm_slab_check(abm_slab* s, void* stream) {
  if (!s) return ABM_ERR_ARG;
  // check builds: the padding of a slab's own arrays (a world's view has none of its own)
  if (kCheck && !s->view && s->n_pad > s->d.cap) {
    k_canary_check<<<num_sms() * 4, 256, 0, (cudaStream_t)stream>>>(s->d.active, s->d.fields, s->d.Fp, s->d.cap,
                                                                    s->n_pad, s->d.err);
    ABM_LAUNCH_CHECK();
  }
  ABM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int err = 0;
  ABM_CUDA_TRY(cudaMemcpy(&err, s->d.err, sizeof(int), cudaMemcpyDeviceToHost));
  return ABM_ERR_OF(err);
}

abm_status abm::slab_canary_fill(int32_t* fields, int Fp, int cap, int n_pad, cudaStream_t st) {
  if (!kCheck || n_pad <= cap) return ABM_OK;
  k_canary_fill<<<num_sms() * 4, 256, 0, st>>>(fields, Fp, cap, n_pad);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

abm_status abm::canary_check(const int32_t* active, const int32_t* fields, int Fp, int cap, int n_pad, int* err,
                             cudaStream_t st) {
  if (!kCheck || n_pad <= cap) return ABM_OK;
  k_canary_check<<<num_sms() * 4, 256, 0, st>>>(active, fields, Fp, cap, n_pad, err);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_diag_check_index(int64_t i, int64_t n, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  ABM_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
  abm_status rc = ABM_OK;
  int h = 0;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) rc = ABM_ERR_CUDA;
  if (rc == ABM_OK) {
    k_check_index<<<1, 1, 0, st>>>((long long)i, (long long)n, err);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = ABM_ERR_CUDA;
  }
  cudaFree(err);
  return rc != ABM_OK ? rc : ABM_ERR_OF(h);
}

extern "C" abm_status abm_slab_arrays(abm_slab* s, int32_t** active, int32_t** fields, int32_t* stride) {
  if (!s) return ABM_ERR_ARG;
  if (active) *active = s->d.active;
  if (fields) *fields = s->d.fields;
  if (stride) *stride = s->d.Fp;
  return ABM_OK;
}

extern "C" abm_status abm_slab_read(abm_slab* s, int32_t field, int32_t* dst, int32_t n, void* stream) {
  if (!s || !dst || n < 0 || n > s->d.cap || field < -1 || field >= s->d.F) return ABM_ERR_ARG;
  if (n == 0) return ABM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (field < 0) {
    ABM_CUDA_TRY(cudaMemcpyAsync(dst, s->d.active, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  } else {
    ABM_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(int32_t), s->d.fields + field, sizeof(int32_t) * s->d.Fp,
                                   sizeof(int32_t), (size_t)n, cudaMemcpyDeviceToDevice, st));
  }
  return ABM_OK;
}

extern "C" abm_status abm_slab_write(abm_slab* s, int32_t field, const int32_t* src, int32_t n, void* stream) {
  if (!s || !src || n < 0 || n > s->d.cap || field < -1 || field >= s->d.F) return ABM_ERR_ARG;
  if (n == 0) return ABM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (field < 0) {
    ABM_CUDA_TRY(cudaMemcpyAsync(s->d.active, src, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    ABM_CUDA_TRY(cudaMemsetAsync(s->d.counters, 0, sizeof(int32_t), st));
    k_count_live<<<num_sms() * 4, 256, 0, st>>>(s->d);
    ABM_LAUNCH_CHECK();
  } else {
    ABM_CUDA_TRY(cudaMemcpy2DAsync(s->d.fields + field, sizeof(int32_t) * s->d.Fp, src, sizeof(int32_t),
                                   sizeof(int32_t), (size_t)n, cudaMemcpyDeviceToDevice, st));
  }
  return ABM_OK;
}

static bool pred_ok(const abm_slab* s, const abm_pred* p) {
  if (!p) return false;
  switch (p->kind) {
    case ABM_PRED_LIVE:
    case ABM_PRED_FREE:
    case ABM_PRED_BERNOULLI: return true;
    case ABM_PRED_MASK: return p->mask != nullptr;
    case ABM_PRED_FIELD: return p->field >= 0 && p->field < s->d.F && p->cmp >= 0 && p->cmp <= 3;
  }
  return false;
}

static PredDev to_dev(const abm_pred* p) {
  PredDev d;
  std::memset(&d, 0, sizeof(d));
  if (!p) return d;
  d.kind = p->kind;
  d.threshold = p->threshold;
  d.step = p->step;
  d.purpose = p->purpose;
  d.species = p->species;
  d.mask = p->mask;
  d.field = p->field;
  d.cmp = p->cmp;
  d.and_mask = p->and_mask;
  d.value = p->value;
  return d;
}

// The apply pass runs one wave: as many CTAs as fit on the device at once
// (looked up once per device), each striding over the records.
template <int OP>
static int apply_grid() {
  static std::atomic<int> per_sm[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  int b = (dev >= 0 && dev < 64) ? per_sm[dev].load(std::memory_order_relaxed) : 0;
  if (!b) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_apply<OP>, 256, 0) != cudaSuccess || b < 1) b = 1;
    if (dev >= 0 && dev < 64) per_sm[dev].store(b, std::memory_order_relaxed);
  }
  return num_sms() * b;
}

// Up to three launches per operation: flags + per-warp / per-CTA counts, then
// ranks + slot lists, then the record moves. Each warp owns one static
// segment of slots in the first two passes; no CTA waits for another.
template <int OP, int THREADS = kSlabThreads>
static abm_status launch_scan(abm_slab* s, const ScanArgs& a, bool aux, cudaStream_t st,
                              int ctas_per_sm = 8) {
  ScanArgs b = a;
  const size_t words = (size_t)(s->n_pad / 32);
  b.planeA = aux ? s->planes2 : s->planes;
  b.planeB = s->planes + words;
  b.totals = aux ? s->totals2 : s->totals;
  b.wtotals = aux ? s->wtotals2 : s->wtotals;
  b.ctrl = aux ? s->ctrl + 4 : s->ctrl;
  constexpr int SUB = (THREADS / 32) * kWarpStep;  // chunks are whole warp steps
  if (b.n <= 0) {
    if (b.out_count) ABM_CUDA_TRY(cudaMemsetAsync(b.out_count, 0, sizeof(int32_t), st));
    if (OP == OP_ARRAY) ABM_CUDA_TRY(cudaMemsetAsync(s->d.counters + 3, 0, sizeof(int32_t), st));
    return ABM_OK;
  }
  const int target = std::max(1, std::min(num_sms() * ctas_per_sm, s->max_ctas));
  const long per = ((long)b.n + target - 1) / target;
  b.chunk = (int)(((per + SUB - 1) / SUB) * SUB);
  b.G = (int)(((long)b.n + b.chunk - 1) / b.chunk);
  if constexpr (OP == OP_FUSED) k_count_fused<THREADS><<<b.G, THREADS, 0, st>>>(b);
  else k_count<OP, THREADS><<<b.G, THREADS, 0, st>>>(b);
  ABM_LAUNCH_CHECK();
  // the next passes may launch while the previous one drains; they wait on
  // it (griddepcontrol) before reading its results
  if constexpr (OP == OP_FUSED) {
    // many records (k >= capacity / 8), 8 fields, 32-byte aligned records and
    // deltas: the ranking pass moves them. With fewer records a warp step holds
    // too few to keep memory busy, and the separate apply pass (four records
    // per thread over the whole grid) measured faster.
    if ((long long)b.k * 8 >= (long long)s->d.cap && s->d.F == 8 && s->d.Fp == 8 &&
        ((((uintptr_t)b.rec) | ((uintptr_t)b.rec2)) & 31) == 0) {
      ABM_CUDA_TRY(launch_pdl(k_scatter<OP, THREADS, true>, b.G, THREADS, st, b));
      return ABM_OK;
    }
  }
  if (OP != OP_REMOVE) ABM_CUDA_TRY(launch_pdl(k_scatter<OP, THREADS>, b.G, THREADS, st, b));
  if (OP == OP_ADD || OP == OP_UPDATE || OP == OP_FUSED)
    ABM_CUDA_TRY(launch_pdl(k_apply<OP>, apply_grid<OP>(), 256, st, b));
  return ABM_OK;
}

static abm_status launch_fused(abm_slab* s, const ScanArgs& a, cudaStream_t st) {
  const int c = s->fused_ctas_per_sm;
  switch (s->fused_threads) {
    case 128: return launch_scan<OP_FUSED, 128>(s, a, false, st, c);
    case 256: return launch_scan<OP_FUSED, 256>(s, a, false, st, c);
    case 512: return launch_scan<OP_FUSED, 512>(s, a, false, st, c);
  }
  return ABM_ERR_ARG;
}

static ScanArgs base_args(abm_slab* s) {
  ScanArgs a;
  std::memset(&a, 0, sizeof(a));
  a.s = s->d;
  a.n = s->d.cap;
  a.id_field = -1;
  return a;
}

extern "C" abm_status abm_select(abm_slab* s, const abm_pred* pred, int32_t* out_idx, int32_t* out_count,
                                 void* stream) {
  if (!s || !pred_ok(s, pred) || !out_idx || !out_count) return ABM_ERR_ARG;
  ScanArgs a = base_args(s);
  a.pred = to_dev(pred);
  a.list_a = out_idx;
  a.out_count = out_count;
  return launch_scan<OP_SELECT>(s, a, false, (cudaStream_t)stream);
}

extern "C" abm_status abm_select_permutation(abm_slab* s, const abm_pred* pred, int32_t* out_perm,
                                             int32_t* out_count, void* stream) {
  if (!s || !pred_ok(s, pred) || !out_perm || !out_count) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ScanArgs a = base_args(s);
  a.pred = to_dev(pred);
  a.list_a = out_perm;
  a.out_count = out_count;
  abm_status e = launch_scan<OP_SELECT>(s, a, false, st);
  if (e != ABM_OK) return e;
  // the complement, ranked from *out_count on (read on the device by the
  // second compaction, after the first one has finished in stream order)
  ScanArgs b = base_args(s);
  b.pred = to_dev(pred);
  b.negate = 1;
  b.list_a = out_perm;
  b.list_base = out_count;
  b.out_count = s->d.meta + 3;
  return launch_scan<OP_SELECT>(s, b, false, st);
}

extern "C" abm_status abm_remove(abm_slab* s, const abm_pred* pred, int32_t* out_removed, void* stream) {
  if (!s || !pred_ok(s, pred) || pred->kind == ABM_PRED_FREE) return ABM_ERR_ARG;
  ScanArgs a = base_args(s);
  a.pred = to_dev(pred);
  a.out_count = out_removed;
  return launch_scan<OP_REMOVE>(s, a, false, (cudaStream_t)stream);
}

extern "C" abm_status abm_add(abm_slab* s, const int32_t* records, int32_t k, int32_t id_field,
                              int32_t* out_slots, int32_t* out_added, void* stream) {
  if (!s || k < 0 || (k > 0 && !records) || id_field < -1 || id_field >= s->d.F) return ABM_ERR_ARG;
  ScanArgs a = base_args(s);
  a.rec = records;
  a.k = k;
  a.id_field = id_field;
  a.list_a = out_slots ? out_slots : s->lista;
  a.out_count = out_added;
  return launch_scan<OP_ADD>(s, a, false, (cudaStream_t)stream);
}

extern "C" abm_status abm_update_distinct(abm_slab* s, const abm_pred* pred, const int32_t* records,
                                          const int32_t* record_mask, int32_t k, int32_t op,
                                          int32_t* out_slots, int32_t* out_applied, void* stream) {
  if (!s || !pred_ok(s, pred) || k < 0 || (k > 0 && !records) || (op != ABM_OP_ADD && op != ABM_OP_SET))
    return ABM_ERR_ARG;
  if (record_mask && k > s->d.cap) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (record_mask) {
    ScanArgs r = base_args(s);
    r.n = k;
    r.src = record_mask;
    r.list_a = s->d.rec_idx;
    abm_status e = launch_scan<OP_ARRAY>(s, r, true, st);
    if (e != ABM_OK) return e;
  }
  ScanArgs a = base_args(s);
  a.pred = to_dev(pred);
  a.rec = records;
  a.k = k;
  a.op_kind = op;
  a.use_rec_idx = record_mask != nullptr;
  a.list_a = out_slots ? out_slots : s->lista;
  a.out_count = out_applied;
  return launch_scan<OP_UPDATE>(s, a, false, st);
}

extern "C" abm_status abm_selective_update(abm_slab* s, uint32_t step, uint32_t threshold,
                                           const int32_t* records, const int32_t* deltas, int32_t k,
                                           int32_t* out_counts, void* stream) {
  if (!s || k < 0 || (k > 0 && (!records || !deltas))) return ABM_ERR_ARG;
  ScanArgs a = base_args(s);
  philox_round_keys(s->d.seed, s->d.model, a.rk);
  mask_pair_consts(step, a.rk, a.mk);
  a.rec = records;
  a.rec2 = deltas;
  a.k = k;
  a.step = step;
  a.threshold = threshold;
  a.out_count = out_counts;
  a.list_a = s->lista;
  a.list_b = s->listb;
  return launch_fused(s, a, (cudaStream_t)stream);
}

extern "C" abm_status abm_slab_tune(abm_slab* s, int32_t threads, int32_t ctas_per_sm, void* stream) {
  (void)stream;
  if (!s || (threads != 128 && threads != 256 && threads != 512) || ctas_per_sm < 1 || ctas_per_sm > 16 ||
      threads * ctas_per_sm > 2048)
    return ABM_ERR_ARG;
  s->fused_threads = threads;
  s->fused_ctas_per_sm = ctas_per_sm;
  return ABM_OK;
}

extern "C" abm_status abm_philox_records(abm_slab* s, uint32_t step, uint32_t purpose0, uint32_t purpose1,
                                         int32_t k, int32_t* out, void* stream) {
  if (!s || k < 0 || (k > 0 && !out) || s->d.F > 8) return ABM_ERR_ARG;
  if (k == 0) return ABM_OK;
  const int grid = std::min((k + 255) / 256, num_sms() * 8);
  k_philox_records<<<grid, 256, 0, (cudaStream_t)stream>>>(s->d, step, purpose0, purpose1, k, out);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_slab_counters_get(abm_slab* s, abm_slab_counters* out, void* stream) {
  if (!s || !out) return ABM_ERR_ARG;
  int32_t c[4];
  ABM_CUDA_TRY(cudaMemcpyAsync(c, s->d.counters, sizeof(c), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  ABM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  out->n_active = c[0];
  out->next_id = c[1];
  out->overflow = c[2];
  out->reserved = 0;
  return ABM_OK;
}
