// Persistent step kernel for one large predation world (ABMax Section 5.1):
// all phases of many steps in one cooperative launch, separated by a bounded
// grid barrier instead of kernel boundaries.
//
// Per step, six barrier-separated phases:
//   1. sheep move + grass claims            (and the previous step's wolf births)
//   2. sheep eat / select / die, flags into bit-planes, per-warp and per-CTA counts
//   3. sheep ranks -> parent list and the first P free slots (P = parents)
//   4. sheep births, wolves move + victim claims
//   5. wolves eat / select / die, flags, counts
//   6. wolves ranks -> lists; counters and statistics of the step
//   (7. wolf births run together with phase 1 of the next step)
// Every CTA owns one static chunk of [0, extent) in phases 2/3 and 5/6, so a
// rank is a prefix over per-CTA totals plus a warp scan: no look-back chains.
// Every thread keeps the world counters in registers and updates them from
// the same totals, so no counter needs a broadcast.
#include <algorithm>

#include "pred_world.cuh"

namespace abm {

constexpr int kPT = 512;                  // threads per CTA
constexpr int kPWarps = kPT / 32;
constexpr int kPCStep = kPWarps * 128;    // chunks are multiples of 128 slots per warp
constexpr int kBarSpin = 1 << 24;         // bounded barrier wait (~2 s with the back-off)

// Grid barrier (all CTAs co-resident: cooperative launch). Generation-based:
// the last CTA to arrive resets the arrival count and bumps the generation.
// A wait that runs out records an error and proceeds (results are then
// invalid, but the kernel ends).
__device__ __forceinline__ void grid_sync(u32* bar, int* err, u32 expected = 0, int limit = kBarSpin) {
  if (expected == 0) expected = gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    const u32 gen = ld_relaxed32(bar + 1);
    __threadfence();
    const u32 arrived = atomicAdd(bar, 1u);
    if (arrived == expected - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      int spins = 0;
      u32 backoff = 16;
      while (ld_relaxed32(bar + 1) == gen) {
        if (++spins > limit) {
          atomicExch(err, kErrTimeout);
          break;
        }
        if (ld_relaxed32(reinterpret_cast<const u32*>(err)) != 0u) break;  // another CTA gave up
        __nanosleep(backoff);
        if (backoff < 128) backoff <<= 1;
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <int S>
__device__ __forceinline__ void p_move(const WorldDev& w, int t, int ext) {
  const SpeciesDev& sp = w.sp[S];
  const int L = w.side;
  const int metab = w.params[PRM_SHEEP_METAB + S];
  const int nq = (ext + 3) >> 2;
  for (int q = blockIdx.x * kPT + threadIdx.x; q < nq; q += gridDim.x * kPT) {
    const int4 act = reinterpret_cast<const int4*>(sp.active)[q];
    const int a4[4] = {act.x, act.y, act.z, act.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!a4[j]) continue;
      const int slot = 4 * q + j;
      int4 ag = sp.agent[slot];
      if (S == 0) w.victim[ag.x] = kNoKey;  // last step's victim entry for this cell
      const u32 dir = draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_MOVE, (u32)S) >> 29;
      const int cell = step_cell(ag.x, L, dir);
      ag.x = cell;
      ag.y -= metab;
      ag.w += 1;
      sp.agent[slot] = ag;
      if (S == 0) {
        if (w.regrow[cell] <= t)
          atomicMin(&w.gclaim[cell], claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_PRIO, 0u), slot));
      } else {
        if (w.victim[cell] != kNoKey)
          atomicMin(&w.wclaim[cell], claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_PRIO, 1u), slot));
      }
    }
  }
}

__device__ __forceinline__ int chunk_of(int ext) {
  const int per = (ext + (int)gridDim.x - 1) / (int)gridDim.x;
  const int c = ((per + kPCStep - 1) / kPCStep) * kPCStep;
  return c > kPCStep ? c : kPCStep;
}

// phase 2/5: eat, select parents, kill the starving; free / parent flags into
// bit-planes (word = 32 slots = 8 lanes x 4 slots), per-warp and per-CTA counts
template <int S>
__device__ __forceinline__ void p_count(const WorldDev& w, int t, int ext, int* acc, u64* s_red) {
  const SpeciesDev& sp = w.sp[S];
  const PersistDev& ps = w.ps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = chunk_of(ext);
  const int seg = chunk / kPWarps;
  const int wlo = blockIdx.x * chunk + warp * seg;
  const int whi = min(ext, wlo + seg);
  const int gain = w.params[S];
  const u32 Tr = (u32)w.params[PRM_SHEEP_T + S];
  const int regrowth = w.params[PRM_REGROWTH];
  u64* claim = S == 0 ? w.gclaim : w.wclaim;
  u32 cf = 0, cp = 0;
  int starved = 0, won = 0;
  for (int b0 = wlo; b0 < whi; b0 += 128) {
    const int base = b0 + 4 * lane;
    int4 act = make_int4(0, 0, 0, 0);
    if (base < ext) act = reinterpret_cast<const int4*>(sp.active)[base >> 2];
    int a4[4] = {act.x, act.y, act.z, act.w};
    u32 fr = 0, par = 0;
    bool died = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int slot = base + j;
      if (slot >= ext) continue;
      if (!a4[j]) {
        fr |= 1u << j;
        continue;
      }
      int4 ag = sp.agent[slot];
      const int cell = ag.x;
      const u64 cl = claim[cell];
      if (cl != kNoKey && (u32)cl == (u32)slot) {
        ag.y += gain;
        sp.agent[slot].y = ag.y;
        claim[cell] = kNoKey;
        ++won;
        if (S == 0) {
          w.regrow[cell] = t + regrowth;
        } else {
          const u64 v = w.victim[cell];
          w.sp[0].active[(u32)v] = 0;
          w.victim[cell] = kNoKey;
        }
      }
      if (ag.y < 0) {
        a4[j] = 0;
        died = true;
        ++starved;
      } else {
        if (draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_REPRO, (u32)S) < Tr) par |= 1u << j;
        if (S == 0)
          atomicMin(&w.victim[cell], claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u), slot));
      }
    }
    if (died) reinterpret_cast<int4*>(sp.active)[base >> 2] = make_int4(a4[0], a4[1], a4[2], a4[3]);
    cf += __popc(fr);
    cp += __popc(par);
    // 8 lanes x 4 bits -> one plane word
    u32 vf = fr << (4 * (lane & 7)), vp = par << (4 * (lane & 7));
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      vf |= __shfl_xor_sync(0xFFFFFFFFu, vf, o);
      vp |= __shfl_xor_sync(0xFFFFFFFFu, vp, o);
    }
    if ((lane & 7) == 0 && base < ext) {
      ps.plane[S][0][base >> 5] = vf;
      ps.plane[S][1][base >> 5] = vp;
    }
  }
  u64 v = ((u64)cf << 32) | cp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) {
    ps.wtotals[2 * (blockIdx.x * kPWarps + warp)] = (u32)(v >> 32);
    ps.wtotals[2 * (blockIdx.x * kPWarps + warp) + 1] = (u32)v;
  }
  // per-CTA totals
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 tt = 0;
    for (int i = 0; i < kPWarps; ++i) tt += s_red[i];
    ps.totals[2 * blockIdx.x] = (u32)(tt >> 32);
    ps.totals[2 * blockIdx.x + 1] = (u32)tt;
  }
  // accumulators (warp-aggregated)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    starved += __shfl_xor_sync(0xFFFFFFFFu, starved, o);
    won += __shfl_xor_sync(0xFFFFFFFFu, won, o);
  }
  if (lane == 0) {
    if (starved) atomicAdd(&acc[S], starved);
    if (won) atomicAdd(&acc[S == 0 ? 3 : 2], won);
  }
}

// grand totals of the per-CTA counts: (free, parents), in every thread
__device__ __forceinline__ void grand_totals(const PersistDev& ps, u32& F, u32& P, u32& preF, u32& preP,
                                             u64* s_red) {
  u64 tot = 0, pre = 0;
  for (int j = threadIdx.x; j < (int)gridDim.x; j += kPT) {
    const u64 x = ((u64)ps.totals[2 * j] << 32) | ps.totals[2 * j + 1];
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
}

// phase 3/6: ranks -> parent list (all) and free list (ranks below P only)
template <int S>
__device__ __forceinline__ void p_scatter(const WorldDev& w, int ext, u32 P, u32 preF, u32 preP) {
  const SpeciesDev& sp = w.sp[S];
  const PersistDev& ps = w.ps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  u32 pf = preF, pp = preP;
  {
    u32 x = 0, y = 0;
    if (lane < warp) {
      x = ps.wtotals[2 * (blockIdx.x * kPWarps + lane)];
      y = ps.wtotals[2 * (blockIdx.x * kPWarps + lane) + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
      y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
    }
    pf += x;
    pp += y;
  }
  const int chunk = chunk_of(ext);
  const int seg = chunk / kPWarps;
  const int wlo = blockIdx.x * chunk + warp * seg;
  const int whi = min(ext, wlo + seg);
  for (int b0 = wlo; b0 < whi; b0 += 128) {
    const int base = b0 + 4 * lane;
    u32 fr = 0, par = 0;
    if (base < ext) {
      const int sh = 4 * (lane & 7);
      fr = (ps.plane[S][0][base >> 5] >> sh) & 0xFu;
      par = (ps.plane[S][1][base >> 5] >> sh) & 0xFu;
    }
    const u32 c = (u32)__popc(fr) | ((u32)__popc(par) << 16);
    u32 inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 x = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += x;
    }
    const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const u32 ex = inc - c;
    u32 rf = pf + (ex & 0xFFFFu), rp = pp + (ex >> 16);
    pf += tot & 0xFFFFu;
    pp += tot >> 16;
    while (fr && rf < P) {  // only the first P free slots can receive a child
      const int j = __ffs(fr) - 1;
      fr &= fr - 1;
      sp.freel[rf++] = base + j;
    }
    while (par) {
      const int j = __ffs(par) - 1;
      par &= par - 1;
      sp.parents[rp++] = base + j;
    }
  }
}

template <int S>
__device__ __forceinline__ void p_births(const WorldDev& w, int t, int r, int F, int ext, int id0) {
  const SpeciesDev& sp = w.sp[S];
  for (int i = blockIdx.x * kPT + threadIdx.x; i < r; i += gridDim.x * kPT) {
    const int p = sp.parents[i];
    const int slot = i < F ? sp.freel[i] : ext + (i - F);
    const int4 pa = sp.agent[p];
    const int half = pa.y >> 1;
    sp.agent[p].y = pa.y - half;
    sp.agent[slot] = make_int4(pa.x, half, (int)((u32)id0 + (u32)i), 0);
    sp.active[slot] = 1;
    if (S == 0)
      atomicMin(&w.victim[pa.x], claim_key(draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u), slot));
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

// phase timing by block 0 (nanoseconds from one barrier exit to the next)
struct PhaseClock {
  unsigned long long* acc;
  u64 last;
  __device__ __forceinline__ void start() {
    if (acc && blockIdx.x == 0 && threadIdx.x == 0) last = globaltimer();
  }
  __device__ __forceinline__ void lap(int k) {
    if (acc && blockIdx.x == 0 && threadIdx.x == 0) {
      const u64 now = globaltimer();
      acc[k] += now - last;
      last = now;
    }
  }
};

__global__ void __launch_bounds__(kPT) k_persistent(WorldDev w, int nsteps, abm_step_stats* stats,
                                                     unsigned long long* phase_ns) {
  __shared__ u64 s_red[2 * kPWarps];
  PhaseClock clk{phase_ns, 0};
  clk.start();
  WorldCtr* c = w.ctr;
  const PersistDev& ps = w.ps;
  // counters: one copy per thread, all updated identically
  int t = c->step;
  int ext[2] = {c->extent[0], c->extent[1]};
  int nact[2] = {c->n_active[0], c->n_active[1]};
  int nid[2] = {c->next_id[0], c->next_id[1]};
  int hw[2] = {c->hw[0], c->hw[1]};
  int ovf[2] = {c->overflow[0], c->overflow[1]};
  const int cap[2] = {w.sp[0].cap, w.sp[1].cap};
  Births wb = {0, 0, 0, 0};  // wolf births pending from the previous step
  for (int it = 0; it < nsteps; ++it) {
    int* acc = ps.acc + 4 * (t & 1);
    abm_step_stats* st = stats ? stats + it : nullptr;
    const int nstart0 = nact[0], nstart1 = nact[1];
    // ---- phase 1: sheep move (+ wolf births of the previous step)
    if (it > 0) p_births<1>(w, t - 1, wb.r, wb.F, wb.ext, wb.id0);
    if (blockIdx.x == 0 && threadIdx.x == 0) acc[0] = acc[1] = acc[2] = acc[3] = 0;  // unused since step t-2
    p_move<0>(w, t, ext[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0 && st) {
      st->n_start[0] = nstart0;
      st->n_start[1] = nstart1;
      st->extent[0] = ext[0];
      st->extent[1] = ext[1];
    }
    grid_sync(ps.bar, w.err);
    clk.lap(0);
    if (*(volatile int*)w.err) return;
    // ---- phase 2: sheep eat / select / die / flags
    p_count<0>(w, t, ext[0], acc, s_red);
    grid_sync(ps.bar, w.err);
    clk.lap(1);
    // ---- phase 3: sheep ranks and lists; sheep counters
    u32 F0, P0, preF, preP;
    grand_totals(ps, F0, P0, preF, preP, s_red);
    p_scatter<0>(w, ext[0], P0, preF, preP);
    const int avail0 = (int)F0 + (cap[0] - ext[0]);
    const int r0 = min((int)P0, avail0);
    const Births sb = {r0, (int)F0, ext[0], nid[0]};
    grid_sync(ps.bar, w.err);
    clk.lap(2);
    // ---- phase 4: sheep births, wolves move + claims (a wolf only needs a live
    // sheep on its cell; every newborn lamb sits with its live parent)
    p_births<0>(w, t, sb.r, sb.F, sb.ext, sb.id0);
    p_move<1>(w, t, ext[1]);
    const int starved0 = acc[0], grass = acc[3];
    {
      const int n_after = nstart0 + r0;
      if (n_after > hw[0]) hw[0] = n_after;
      nact[0] = n_after - starved0;
      nid[0] += r0;
      if (r0 > (int)F0) ext[0] += r0 - (int)F0;
      if ((int)P0 > avail0) ovf[0] = 1;
    }
    grid_sync(ps.bar, w.err);
    clk.lap(3);
    // ---- phase 5: wolves eat / kill / select / die / flags
    p_count<1>(w, t, ext[1], acc, s_red);
    grid_sync(ps.bar, w.err);
    clk.lap(4);
    // ---- phase 6: wolf ranks and lists; counters; statistics
    u32 F1, P1, preF1, preP1;
    grand_totals(ps, F1, P1, preF1, preP1, s_red);
    p_scatter<1>(w, ext[1], P1, preF1, preP1);
    const int starved1 = acc[1], eaten = acc[2];
    const int avail1 = (int)F1 + (cap[1] - ext[1]);
    const int r1 = min((int)P1, avail1);
    wb = {r1, (int)F1, ext[1], nid[1]};
    {
      const int n_after = nstart1 + r1;
      if (n_after > hw[1]) hw[1] = n_after;
      nact[1] = n_after - starved1;
      nid[1] += r1;
      if (r1 > (int)F1) ext[1] += r1 - (int)F1;
      if ((int)P1 > avail1) ovf[1] = 1;
      nact[0] -= eaten;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && st) {
      st->parents[0] = (int)P0;
      st->parents[1] = (int)P1;
      st->births[0] = r0;
      st->births[1] = r1;
      st->starved[0] = starved0;
      st->starved[1] = starved1;
      st->eaten = eaten;
      st->grass_eaten = grass;
      for (int s = 0; s < 2; ++s) {
        st->n_end[s] = nact[s];
        st->hw[s] = hw[s];
        st->overflow[s] = ovf[s];
      }
      st->step = t;
    }
    ++t;
    grid_sync(ps.bar, w.err);
    clk.lap(5);
  }
  // the last step's wolf births
  if (nsteps > 0) p_births<1>(w, t - 1, wb.r, wb.F, wb.ext, wb.id0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->step = t;
    for (int s = 0; s < 2; ++s) {
      c->extent[s] = ext[s];
      c->n_active[s] = nact[s];
      c->next_id[s] = nid[s];
      c->hw[s] = hw[s];
      c->overflow[s] = ovf[s];
    }
  }
}

// Failure-detection check: a grid barrier that waits for one CTA more than
// the grid has, so that the wait must run out; every CTA records the timeout
// and returns. Used to show that a wait which never completes ends the kernel
// with an error status instead of hanging the GPU.
__global__ void k_barrier_timeout(u32* bar, int* err, int limit) {
  grid_sync(bar, err, gridDim.x + 1, limit);
}

int persistent_max_ctas() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent, kPT, 0) != cudaSuccess) return 0;
  return nb * num_sms();
}

int persistent_warps() { return kPWarps; }

abm_status launch_persistent(const WorldDev& d, int grid, int nsteps, abm_step_stats* stats, cudaStream_t st,
                             unsigned long long* phase_ns) {
  WorldDev dd = d;
  void* args[] = {(void*)&dd, (void*)&nsteps, (void*)&stats, (void*)&phase_ns};
  ABM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_persistent, dim3((unsigned)grid), dim3(kPT), args, 0, st));
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
