// Wolf-sheep-grass predation (ABMax Section 5.1, Fig. 3) on one GPU: the
// model that drives the selective-update hot path.
//
// Per species and step the engine runs three kernels:
//   move    - random 8-neighbour move, metabolism, ageing; then the claim on
//             this step's resource (sheep: grown grass; wolves: a cell that
//             holds a victim) by atomicMin of (PRIO draw << 32 | slot);
//   scan    - the claim's winner eats; live agents with energy >= 0 and a
//             REPRO draw below T are selected as parents, agents with energy
//             < 0 die; one decoupled-look-back pass ranks parents and free
//             slots together and compacts both lists; surviving sheep enter
//             their cell's victim draw;
//   births  - the i-th parent puts a child in the i-th free slot (Rank-Match
//             pairing) and gives it floor(e/2) energy; the last CTA out
//             updates the counters.
// Sweeps cover [0, extent), the highest slot ever used + 1. Because children
// always fill the lowest free slots, extent never exceeds the high-water mark
// of the population, and the slots beyond it are free by construction.
//
// Grass is stored as the step from which each cell is edible again, so no
// per-cell regrowth pass is needed. The per-cell claim tables are returned to
// "empty" by the agents that consumed them (winners, eaters, and each live
// sheep resetting its cell's victim entry at the start of the next step), so
// no table is ever swept either.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "pred_world.cuh"
#include "slab.cuh"

namespace abm {

template <int S>
__global__ void __launch_bounds__(kPredThreads) k_move(WorldDev w, abm_step_stats* st) {
  const int t = w.ctr->step;
  const int ext = w.ctr->extent[S];
  const int L = w.side;
  const int metab = w.params[5 + S];
  const SpeciesDev sp = w.sp[S];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int n = w.ctr->n_active[S];
    w.ctr->n_start[S] = n;
    if (st) {
      st->n_start[S] = n;
      st->extent[S] = ext;
    }
  }
  const int nq = (ext + 3) >> 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const int4 act = reinterpret_cast<const int4*>(sp.active)[q];
    const int a4[4] = {act.x, act.y, act.z, act.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!a4[j]) continue;
      const int slot = 4 * q + j;
      int4 ag = sp.agent[slot];
      if (!in_range(ag.x, w.ncells, w.err)) continue;  // check builds: a cell outside the lattice
      if (S == 0) w.victim[ag.x] = kNoKey;  // last step's victim entry for this cell
      const u32 dir = draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_MOVE, (u32)S) >> 29;
      const int cell = step_cell(ag.x, L, dir);
      ag.x = cell;
      ag.y -= metab;
      ag.w += 1;
      sp.agent[slot] = ag;
      if (S == 0) {
        if (w.regrow[cell] <= t) {
          const u64 key = ((u64)draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_PRIO, 0u) << 32) | (u32)slot;
          atomicMin(&w.gclaim[cell], key);
        }
      } else {
        if (w.victim[cell] != kNoKey) {
          const u64 key = ((u64)draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_PRIO, 1u) << 32) | (u32)slot;
          atomicMin(&w.wclaim[cell], key);
        }
      }
    }
  }
}

template <int S>
__global__ void __launch_bounds__(kPredThreads) k_scan(WorldDev w) {
  __shared__ u64 s_warp[kPredThreads / 32 + 1];
  __shared__ u32 s_bcast[2];
  __shared__ int s_tile;
  const SpeciesDev sp = w.sp[S];
  const ScanCtl ctl{sp.tiles, sp.ctrl, w.err};
  const u32 tag = launch_tag(sp.ctrl);
  const int t = w.ctr->step;
  const int ext = w.ctr->extent[S];
  const int bound = w.ctr->n_active[S];  // parents <= live agents: free slots past this rank are never used
  const int ntiles = (ext + kPredTile - 1) / kPredTile;
  const int gain = w.params[S];
  const u32 T = (u32)w.params[2 + S];
  const int regrowth = w.params[4];
  int grass = 0, eaten = 0, starved = 0;

  while (true) {
    const int tile = next_tile(sp.ctrl, &s_tile);
    if (tile >= ntiles) break;
    const int base = tile * kPredTile + threadIdx.x * kPredItems;
    const int4 act = reinterpret_cast<const int4*>(sp.active)[base >> 2];
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
      if (!in_range(cell, w.ncells, w.err)) continue;  // check builds only
      u64* claim = S == 0 ? w.gclaim : w.wclaim;
      const u64 cl = claim[cell];
      if (cl != kNoKey && (u32)cl == (u32)slot) {
        ag.y += gain;
        sp.agent[slot].y = ag.y;
        claim[cell] = kNoKey;
        if (S == 0) {
          w.regrow[cell] = t + regrowth;
          ++grass;
        } else {
          const u64 v = w.victim[cell];
          if (in_range((u32)v, w.sp[0].cap, w.err)) w.sp[0].active[(u32)v] = 0;
          w.victim[cell] = kNoKey;
          ++eaten;
        }
      }
      if (ag.y < 0) {
        a4[j] = 0;
        died = true;
        ++starved;
      } else {
        if (draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_REPRO, (u32)S) < T) par |= 1u << j;
        if (S == 0) {
          const u64 key = ((u64)draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u) << 32) | (u32)slot;
          atomicMin(&w.victim[cell], key);
        }
      }
    }
    u32 ex_f, ex_p, tot_f, tot_p, pre_f, pre_p;
    block_scan2<kPredThreads>(__popc(fr), __popc(par), ex_f, ex_p, tot_f, tot_p, s_warp);
    tile_prefix<kPredThreads>(ctl, tile, tag, tot_f, tot_p, pre_f, pre_p, s_bcast);
    if (tile == ntiles - 1 && threadIdx.x == 0) {
      w.ctr->free_in[S] = (int)(pre_f + tot_f);
      w.ctr->parents[S] = (int)(pre_p + tot_p);
    }
    u32 rf = pre_f + ex_f, rp = pre_p + ex_p;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((fr >> j) & 1u) {
        if ((int)rf < bound && in_range(rf, sp.cap, w.err)) sp.freel[rf] = base + j;
        ++rf;
      }
      if ((par >> j) & 1u) {
        if (in_range(rp, sp.cap, w.err)) sp.parents[rp] = base + j;
        ++rp;
      }
    }
    if (died) reinterpret_cast<int4*>(sp.active)[base >> 2] = make_int4(a4[0], a4[1], a4[2], a4[3]);
  }
  if (ntiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    w.ctr->free_in[S] = 0;
    w.ctr->parents[S] = 0;
  }
  if (S == 0) warp_add(&w.ctr->grass_eaten, grass);
  if (S == 1) warp_add(&w.ctr->eaten, eaten);
  warp_add(&w.ctr->starved[S], starved);
  last_cta_out(sp.ctrl);
}

template <int S>
__global__ void __launch_bounds__(kPredThreads) k_births(WorldDev w, abm_step_stats* st) {
  const SpeciesDev sp = w.sp[S];
  WorldCtr* c = w.ctr;
  const int t = c->step;
  const int P = c->parents[S], Fin = c->free_in[S], ext = c->extent[S];
  const int avail = Fin + (sp.cap - ext);
  const int r = min(P, avail);
  const int next_id = c->next_id[S];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x) {
    const int p = sp.parents[i];
    const int slot = i < Fin ? sp.freel[i] : ext + (i - Fin);
    if (!in_range(p, sp.cap, w.err) || !in_range(slot, sp.cap, w.err)) continue;
    const int4 pa = sp.agent[p];
    const int half = pa.y >> 1;
    sp.agent[p].y = pa.y - half;
    sp.agent[slot] = make_int4(pa.x, half, (int)((u32)next_id + (u32)i), 0);
    sp.active[slot] = 1;
    if (S == 0) {
      const u64 key = ((u64)draw(w.seed, w.model, (u32)t, (u32)slot, ABM_P_VICTIM, 0u) << 32) | (u32)slot;
      atomicMin(&w.victim[pa.x], key);
    }
  }
  if (last_cta_out(sp.ctrl + 4)) {
    const int n_after = c->n_start[S] + r;
    if (n_after > c->hw[S]) c->hw[S] = n_after;
    c->n_active[S] = n_after - c->starved[S];
    c->next_id[S] = next_id + r;
    if (r > Fin) c->extent[S] = ext + (r - Fin);
    if (P > avail) c->overflow[S] = 1;
    if (st) {
      st->parents[S] = P;
      st->births[S] = r;
      st->starved[S] = c->starved[S];
    }
    if (S == 1) {
      c->n_active[0] -= c->eaten;
      if (st) {
        st->eaten = c->eaten;
        st->grass_eaten = c->grass_eaten;
        for (int s = 0; s < 2; ++s) {
          st->n_end[s] = c->n_active[s];
          st->hw[s] = c->hw[s];
          st->overflow[s] = c->overflow[s];
        }
        st->step = t;
      }
      c->step = t + 1;
      c->starved[0] = c->starved[1] = 0;
      c->eaten = 0;
      c->grass_eaten = 0;
    }
    __threadfence();
  }
}

// total live energy per species (optional statistics)
__global__ void k_energy(WorldDev w, abm_step_stats* st) {
  for (int s = 0; s < 2; ++s) {
    const int ext = w.ctr->extent[s];
    long long e = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ext; i += gridDim.x * blockDim.x)
      if (w.sp[s].active[i]) e += w.sp[s].agent[i].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    if ((threadIdx.x & 31) == 0 && e) atomicAdd((unsigned long long*)&w.ctr->energy[s], (unsigned long long)e);
  }
  if (last_cta_out(w.ctr->energy_exit)) {
    for (int s = 0; s < 2; ++s) {
      if (st) st->energy[s] = w.ctr->energy[s];
      w.ctr->energy[s] = 0;
    }
    __threadfence();
  }
}

__global__ void k_world_init(WorldDev w, int n0s, int n0w) {
  const int n0[2] = {n0s, n0w};
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int s = 0; s < 2; ++s) {
    const int gain = w.params[s];
    for (int k = tid; k < n0[s]; k += stride) {
      const uint4 u = draw4(w.seed, w.model, ABM_INIT_STEP, (u32)k, ABM_P_INIT_AGENT, (u32)s);
      w.sp[s].agent[k] = make_int4(uniform_below(u.x, w.ncells), uniform_below(u.y, 2 * gain), k, 0);
      w.sp[s].active[k] = 1;
    }
  }
  for (int c = tid; c < w.ncells; c += stride) {
    const uint4 u = draw4(w.seed, w.model, ABM_INIT_STEP, (u32)c, ABM_P_GRASS_INIT, 2u);
    const bool grown = u.x < (u32)w.params[7];
    const int wait = uniform_below(u.y, w.params[4]);
    w.regrow[c] = grown ? 0 : max(wait, 1);
    w.gclaim[c] = kNoKey;
    w.victim[c] = kNoKey;
    w.wclaim[c] = kNoKey;
  }
}

__global__ void k_read_grass(WorldDev w, int which, int32_t* dst) {
  const int T = w.ctr->step;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < w.ncells; c += gridDim.x * blockDim.x) {
    const int r = w.regrow[c];
    dst[c] = which == 0 ? (r <= T ? 1 : 0) : (r <= T ? 0 : r - T);
  }
}

// digest of the whole world (digest_* terms): per-CTA sums added atomically
// into *out (zeroed by the caller), the counters' term by CTA 0
__global__ void k_world_digest(WorldDev w, u64* out) {
  __shared__ u64 s[kPredThreads / 32];
  const WorldCtr* c = w.ctr;
  const int step = c->step;
  u64 h = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int sp = 0; sp < 2; ++sp) {
    const int ext = c->extent[sp];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ext; i += stride)
      if (w.sp[sp].active[i]) h += digest_agent(sp, i, w.sp[sp].agent[i]);
  }
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < w.ncells; cell += stride)
    h += digest_cell(cell, w.regrow[cell], step);
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = h;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int k = 0; k < kPredThreads / 32; ++k) t += s[k];
    if (blockIdx.x == 0) {
      const int na[2] = {c->n_active[0], c->n_active[1]}, ni[2] = {c->next_id[0], c->next_id[1]};
      const int hw[2] = {c->hw[0], c->hw[1]};
      t += digest_counters(na, ni, hw);
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)t);
  }
}

// a species' slab view takes the world's live count, next id and overflow flag
__global__ void k_view_open(const WorldCtr* c, int sp, int32_t* counters) {
  counters[0] = c->n_active[sp];
  counters[1] = c->next_id[sp];
  counters[2] = c->overflow[sp];
  counters[3] = 0;
}

// live slots and the highest live slot + 1 of a species, into scan[0], scan[1] (zeroed)
__global__ void k_view_scan(const int32_t* active, int cap, int* scan) {
  int n = 0, top = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
    if (active[i]) {
      ++n;
      top = i + 1;
    }
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
    top = max(top, __shfl_xor_sync(0xFFFFFFFFu, top, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (n) atomicAdd(&scan[0], n);
    if (top) atomicMax(&scan[1], top);
  }
}

// fold an edited species back into the world's counters
__global__ void k_view_commit(WorldCtr* c, int sp, const int32_t* counters, const int* scan) {
  const int n = scan[0];
  c->n_active[sp] = n;
  c->next_id[sp] = counters[1];
  if (counters[2]) c->overflow[sp] = 1;
  if (n > c->hw[sp]) c->hw[sp] = n;
  if (scan[1] > c->extent[sp]) c->extent[sp] = scan[1];
}

}  // namespace abm

// ============================================================================
using namespace abm;

struct abm_world {
  WorldDev d;
  int cap_pad[2];
  int grid;
  int engine;       // ABM_ENGINE_PERSISTENT or ABM_ENGINE_KERNELS
  int pgrid;        // CTAs of the persistent kernel
  u32 bar_next;     // value of the persistent kernel's barrier counter after the launches so far
  int pgrid_max;
  int64_t steps_host;
  // cached graph
  cudaGraphExec_t gexec;
  int g_nsteps;
  abm_step_stats* g_stats;
  abm_slab* view[2];  // per species, made by the first abm_world_slab call
};

static void world_free(abm_world* w) {
  for (int s = 0; s < 2; ++s) {
    cudaFree(w->d.sp[s].active);
    cudaFree(w->d.sp[s].agent);
    cudaFree(w->d.sp[s].parents);
    cudaFree(w->d.sp[s].freel);
    cudaFree(w->d.sp[s].tiles);
    cudaFree(w->d.sp[s].ctrl);
  }
  cudaFree(w->d.regrow);
  cudaFree(w->d.gclaim);
  cudaFree(w->d.victim);
  cudaFree(w->d.wclaim);
  cudaFree(w->d.ctr);
  cudaFree(w->d.err);
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 2; ++k) cudaFree(w->d.ps.plane[s][k]);
  for (int s = 0; s < 2; ++s) {
    cudaFree(w->d.ps.blk[s]);
    cudaFree(w->d.ps.seg[s]);
  }
  cudaFree(w->d.ps.bar);
  cudaFree(w->d.ps.acc);
  cudaFree(w->d.skey);
  cudaFree(w->d.snext);
  cudaFree(w->d.wkey);
  cudaFree(w->d.wnext);
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  slab_free_view(w->view[0]);
  slab_free_view(w->view[1]);
  delete w;
}

extern "C" abm_status abm_destroy(abm_world* w) {
  if (!w) return ABM_ERR_ARG;
  world_free(w);
  return ABM_OK;
}

extern "C" abm_status abm_create(const abm_config* cfg, void* stream, abm_world** out) {
  if (!cfg || !out || cfg->side < 1 || cfg->side > 46340) return ABM_ERR_ARG;
  for (int s = 0; s < 2; ++s) {
    if (cfg->cap[s] < 1 || cfg->cap[s] > (1 << 28) - 1 || cfg->n0[s] < 0 || cfg->n0[s] > cfg->cap[s])
      return ABM_ERR_ARG;
    if (cfg->params[s] < 0 || cfg->params[5 + s] < 0) return ABM_ERR_ARG;
  }
  if (cfg->params[4] < 1) return ABM_ERR_ARG;
  if (cfg->variant & ~(ABM_VARIANT_MANY_WOLVES | ABM_VARIANT_GRASS_OFF)) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  abm_world* w = new (std::nothrow) abm_world();
  if (!w) return ABM_ERR_OOM;
  std::memset(w, 0, sizeof(*w));
  WorldDev& d = w->d;
  d.side = cfg->side;
  d.ncells = cfg->side * cfg->side;
  d.seed = cfg->seed;
  d.model = cfg->model;
  d.variant = cfg->variant;
  std::memcpy(d.params, cfg->params, sizeof(d.params));
  bool ok = true;
  for (int s = 0; s < 2; ++s) {
    const int cap = cfg->cap[s];
    const int ntiles = (cap + kPredTile - 1) / kPredTile;
    w->cap_pad[s] = ntiles * kPredTile;
    d.sp[s].cap = cap;
    ok = ok && cudaMalloc(&d.sp[s].active, sizeof(int32_t) * (size_t)w->cap_pad[s]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.sp[s].agent, sizeof(int4) * (size_t)w->cap_pad[s]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.sp[s].parents, sizeof(int32_t) * (size_t)cap) == cudaSuccess;
    ok = ok && cudaMalloc(&d.sp[s].freel, sizeof(int32_t) * (size_t)cap) == cudaSuccess;
    ok = ok && cudaMalloc(&d.sp[s].tiles, sizeof(u64) * (size_t)ntiles) == cudaSuccess;
    ok = ok && cudaMalloc(&d.sp[s].ctrl, sizeof(u32) * 8) == cudaSuccess;
    if (ok) {
      ok = cudaMemsetAsync(d.sp[s].active, 0, sizeof(int32_t) * (size_t)w->cap_pad[s], st) == cudaSuccess &&
           cudaMemsetAsync(d.sp[s].agent, 0, sizeof(int4) * (size_t)w->cap_pad[s], st) == cudaSuccess &&
           cudaMemsetAsync(d.sp[s].tiles, 0, sizeof(u64) * (size_t)ntiles, st) == cudaSuccess &&
           cudaMemsetAsync(d.sp[s].ctrl, 0, sizeof(u32) * 8, st) == cudaSuccess;
    }
  }
  ok = ok && cudaMalloc(&d.regrow, sizeof(int32_t) * (size_t)d.ncells) == cudaSuccess;
  ok = ok && cudaMalloc(&d.gclaim, sizeof(u64) * (size_t)d.ncells) == cudaSuccess;
  ok = ok && cudaMalloc(&d.victim, sizeof(u64) * (size_t)d.ncells) == cudaSuccess;
  ok = ok && cudaMalloc(&d.wclaim, sizeof(u64) * (size_t)d.ncells) == cudaSuccess;
  ok = ok && cudaMalloc(&d.ctr, sizeof(WorldCtr)) == cudaSuccess;
  ok = ok && cudaMalloc(&d.err, sizeof(int)) == cudaSuccess;
  w->pgrid_max = persistent_max_ctas();
  if (w->pgrid_max < 1) ok = false;
  const int pmax = std::max(1, w->pgrid_max);
  for (int s = 0; s < 2 && ok; ++s)
    for (int k = 0; k < 2 && ok; ++k)
      ok = cudaMalloc(&d.ps.plane[s][k], sizeof(u32) * (size_t)(w->cap_pad[s] / 32)) == cudaSuccess;
  for (int s = 0; s < 2 && ok; ++s) {
    ok = cudaMalloc(&d.ps.blk[s], sizeof(u64) * (size_t)(w->cap_pad[s] / 128)) == cudaSuccess &&
         cudaMalloc(&d.ps.seg[s], sizeof(u64) * (size_t)pmax) == cudaSuccess &&
         cudaMemsetAsync(d.ps.seg[s], 0, sizeof(u64) * (size_t)pmax, st) == cudaSuccess;
  }
  if (d.variant & ABM_VARIANT_MANY_WOLVES) {
    ok = ok && cudaMalloc(&d.skey, sizeof(u64) * (size_t)cfg->cap[0]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.snext, sizeof(u64) * (size_t)cfg->cap[0]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.wkey, sizeof(u64) * (size_t)cfg->cap[1]) == cudaSuccess;
    ok = ok && cudaMalloc(&d.wnext, sizeof(u64) * (size_t)cfg->cap[1]) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&d.ps.bar, sizeof(u32) * 2) == cudaSuccess;
  ok = ok && cudaMalloc(&d.ps.acc, sizeof(int) * 8) == cudaSuccess;
  ok = ok && cudaMemsetAsync(d.ps.bar, 0, sizeof(u32) * 2, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(d.ps.acc, 0, sizeof(int) * 8, st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    world_free(w);
    return ABM_ERR_OOM;
  }
  WorldCtr h;
  std::memset(&h, 0, sizeof(h));
  for (int s = 0; s < 2; ++s) {
    h.n_active[s] = cfg->n0[s];
    h.next_id[s] = cfg->n0[s];
    h.hw[s] = cfg->n0[s];
    h.extent[s] = cfg->n0[s];
  }
  if (cudaMemcpyAsync(d.ctr, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(d.err, 0, sizeof(int), st) != cudaSuccess) {
    world_free(w);
    return ABM_ERR_CUDA;
  }
  w->grid = num_sms() * 8;
  w->engine = ABM_ENGINE_PERSISTENT;
  w->pgrid = std::min(w->pgrid_max, num_sms() * 2);
  k_world_init<<<num_sms() * 4, 256, 0, st>>>(d, cfg->n0[0], cfg->n0[1]);
  for (int s = 0; s < 2; ++s)  // check builds: canaries past the capacity
    if (slab_canary_fill(reinterpret_cast<int32_t*>(d.sp[s].agent), 4, d.sp[s].cap, w->cap_pad[s], st) != ABM_OK)
      ok = false;
  if (!ok || cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    world_free(w);
    return ABM_ERR_CUDA;
  }
  *out = w;
  return ABM_OK;
}

// ev (nullable): 7 events recorded around the six kernels of the step
static abm_status enqueue_step(abm_world* w, abm_step_stats* st_ptr, int want_energy, cudaStream_t st,
                               cudaEvent_t* ev = nullptr) {
  const int g = w->grid;
  if (ev) cudaEventRecord(ev[0], st);
  k_move<0><<<g, kPredThreads, 0, st>>>(w->d, st_ptr);
  if (ev) cudaEventRecord(ev[1], st);
  k_scan<0><<<g, kPredThreads, 0, st>>>(w->d);
  if (ev) cudaEventRecord(ev[2], st);
  k_births<0><<<g, kPredThreads, 0, st>>>(w->d, st_ptr);
  if (ev) cudaEventRecord(ev[3], st);
  k_move<1><<<g, kPredThreads, 0, st>>>(w->d, st_ptr);
  if (ev) cudaEventRecord(ev[4], st);
  k_scan<1><<<g, kPredThreads, 0, st>>>(w->d);
  if (ev) cudaEventRecord(ev[5], st);
  k_births<1><<<g, kPredThreads, 0, st>>>(w->d, st_ptr);
  if (ev) cudaEventRecord(ev[6], st);
  if (want_energy) k_energy<<<g, kPredThreads, 0, st>>>(w->d, st_ptr);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_step_profiled(abm_world* w, int32_t nsteps, abm_step_stats* stats, float* phase_ms,
                                        void* stream) {
  if (!w || nsteps < 0 || !phase_ms) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (w->engine == ABM_ENGINE_PERSISTENT) {
    // one launch; block 0 times its phases with the global timer, the whole
    // launch is timed with events
    unsigned long long* ns = nullptr;
    ABM_CUDA_TRY(cudaMallocAsync((void**)&ns, sizeof(unsigned long long) * 8, st));
    ABM_CUDA_TRY(cudaMemsetAsync(ns, 0, sizeof(unsigned long long) * 8, st));
    cudaEvent_t e0, e1;
    ABM_CUDA_TRY(cudaEventCreate(&e0));
    ABM_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    abm_status rc = nsteps > 0 ? launch_persistent(w->d, &w->bar_next, w->pgrid, nsteps, stats, st, ns) : ABM_OK;
    cudaEventRecord(e1, st);
    unsigned long long h[8] = {0};
    if (rc == ABM_OK) {
      w->steps_host += nsteps;
      if (cudaMemcpyAsync(h, ns, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = ABM_ERR_CUDA;
    }
    float total = 0.f;
    if (rc == ABM_OK && cudaEventElapsedTime(&total, e0, e1) != cudaSuccess) rc = ABM_ERR_CUDA;
    for (int k = 0; k < 8; ++k) phase_ms[k] = k < 6 ? (float)(h[k] * 1e-6) : 0.f;
    phase_ms[7] = total;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(ns, st);
    return rc;
  }
  std::vector<cudaEvent_t> ev((size_t)nsteps * 7);
  for (auto& e : ev) ABM_CUDA_TRY(cudaEventCreate(&e));
  abm_status rc = ABM_OK;
  for (int i = 0; i < nsteps && rc == ABM_OK; ++i)
    rc = enqueue_step(w, stats ? stats + i : nullptr, 0, st, &ev[(size_t)i * 7]);
  if (rc == ABM_OK) {
    w->steps_host += nsteps;
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = ABM_ERR_CUDA;
  }
  for (int k = 0; k < 8; ++k) phase_ms[k] = 0.f;
  for (int i = 0; i < nsteps && rc == ABM_OK; ++i) {
    for (int k = 0; k < 6; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[(size_t)i * 7 + k], ev[(size_t)i * 7 + k + 1]) != cudaSuccess) {
        rc = ABM_ERR_CUDA;
        break;
      }
      phase_ms[k] += ms;
    }
  }
  if (rc == ABM_OK && nsteps > 0) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[0], ev[(size_t)(nsteps - 1) * 7 + 6]) == cudaSuccess) phase_ms[7] = ms;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}

extern "C" abm_status abm_step(abm_world* w, int32_t nsteps, abm_step_stats* stats, int32_t want_energy,
                               void* stream) {
  if (!w || nsteps < 0) return ABM_ERR_ARG;
  // the per-phase kernels (which also compute the energy statistics) do not
  // implement the several-wolves variant
  if (want_energy && w->d.variant != ABM_VARIANT_ONE_WOLF) return ABM_ERR_ARG;
  if (w->engine == ABM_ENGINE_PERSISTENT && !want_energy) {
    if (nsteps == 0) return ABM_OK;
    abm_status e = launch_persistent(w->d, &w->bar_next, w->pgrid, nsteps, stats, (cudaStream_t)stream);
    if (e == ABM_OK) w->steps_host += nsteps;
    return e;
  }
  for (int i = 0; i < nsteps; ++i) {
    abm_status e = enqueue_step(w, stats ? stats + i : nullptr, want_energy, (cudaStream_t)stream);
    if (e != ABM_OK) return e;
  }
  w->steps_host += nsteps;
  return ABM_OK;
}

extern "C" abm_status abm_step_graph(abm_world* w, int32_t nsteps, int32_t reps, abm_step_stats* stats,
                                     void* stream) {
  if (!w || nsteps < 1 || reps < 0 || !stream) return ABM_ERR_ARG;
  if (w->d.variant != ABM_VARIANT_ONE_WOLF) return ABM_ERR_STATE;  // per-phase kernels only
  cudaStream_t st = (cudaStream_t)stream;
  if (!w->gexec || w->g_nsteps != nsteps || w->g_stats != stats) {
    if (w->gexec) {
      cudaGraphExecDestroy(w->gexec);
      w->gexec = nullptr;
    }
    cudaGraph_t graph;
    ABM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    abm_status e = ABM_OK;
    for (int i = 0; i < nsteps && e == ABM_OK; ++i) e = enqueue_step(w, stats ? stats + i : nullptr, 0, st);
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (e != ABM_OK) return e;
    if (ce != cudaSuccess) return ABM_ERR_CUDA;
    ce = cudaGraphInstantiate(&w->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      w->gexec = nullptr;
      return ABM_ERR_CUDA;
    }
    w->g_nsteps = nsteps;
    w->g_stats = stats;
  }
  for (int r = 0; r < reps; ++r) ABM_CUDA_TRY(cudaGraphLaunch(w->gexec, st));
  w->steps_host += (int64_t)nsteps * reps;
  return ABM_OK;
}

extern "C" abm_status abm_world_tune(abm_world* w, int32_t engine, int32_t ctas_per_sm) {
  if (!w || (engine != ABM_ENGINE_PERSISTENT && engine != ABM_ENGINE_KERNELS) || ctas_per_sm < 1) return ABM_ERR_ARG;
  if (engine == ABM_ENGINE_KERNELS && w->d.variant != ABM_VARIANT_ONE_WOLF) return ABM_ERR_ARG;
  const int g = num_sms() * ctas_per_sm;
  if (engine == ABM_ENGINE_PERSISTENT && g > w->pgrid_max) return ABM_ERR_ARG;
  w->engine = engine;
  if (engine == ABM_ENGINE_PERSISTENT) w->pgrid = g;
  return ABM_OK;
}

extern "C" abm_status abm_world_check(abm_world* w, void* stream) {
  if (!w) return ABM_ERR_ARG;
  for (int s = 0; s < 2; ++s) {
    const abm_status e = canary_check(w->d.sp[s].active, reinterpret_cast<const int32_t*>(w->d.sp[s].agent), 4,
                                      w->d.sp[s].cap, w->cap_pad[s], w->d.err, (cudaStream_t)stream);
    if (e != ABM_OK) return e;
  }
  ABM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int err = 0;
  ABM_CUDA_TRY(cudaMemcpy(&err, w->d.err, sizeof(int), cudaMemcpyDeviceToHost));
  return ABM_ERR_OF(err);
}

extern "C" abm_status abm_read_agents(abm_world* w, int32_t species, int32_t which, int32_t* dst, void* stream) {
  if (!w || !dst || species < 0 || species > 1 || which < 0 || which > 4) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)w->d.sp[species].cap;
  if (which == 0) {
    ABM_CUDA_TRY(cudaMemcpyAsync(dst, w->d.sp[species].active, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
  } else {
    const int32_t* src = reinterpret_cast<const int32_t*>(w->d.sp[species].agent) + (which - 1);
    ABM_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(int32_t), src, sizeof(int4), sizeof(int32_t), n,
                                   cudaMemcpyDeviceToDevice, st));
  }
  return ABM_OK;
}

extern "C" abm_status abm_read_grass(abm_world* w, int32_t which, int32_t* dst, void* stream) {
  if (!w || !dst || which < 0 || which > 1) return ABM_ERR_ARG;
  k_read_grass<<<num_sms() * 4, 256, 0, (cudaStream_t)stream>>>(w->d, which, dst);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_world_counters_get(abm_world* w, abm_world_counters* out, void* stream) {
  if (!w || !out) return ABM_ERR_ARG;
  WorldCtr h;
  cudaStream_t st = (cudaStream_t)stream;
  ABM_CUDA_TRY(cudaMemcpyAsync(&h, w->d.ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
  ABM_CUDA_TRY(cudaStreamSynchronize(st));
  for (int s = 0; s < 2; ++s) {
    out->n_active[s] = h.n_active[s];
    out->next_id[s] = h.next_id[s];
    out->hw[s] = h.hw[s];
    out->overflow[s] = h.overflow[s];
    out->extent[s] = h.extent[s];
  }
  out->step = h.step;
  out->reserved = 0;
  return ABM_OK;
}

// checkpoint image: [WorldCtr][active0][agent0][active1][agent1][regrow],
// each species' arrays cut at its extent (slots at or past the extent are
// empty: never written, or emptied by abm_load)
static size_t image_bytes(const abm_world* w, const WorldCtr& h) {
  size_t b = sizeof(WorldCtr);
  for (int s = 0; s < 2; ++s) b += (size_t)h.extent[s] * (sizeof(int32_t) + sizeof(int4));
  return b + (size_t)w->d.ncells * sizeof(int32_t);
}

extern "C" abm_status abm_image_capacity(abm_world* w, size_t* bytes) {
  if (!w || !bytes) return ABM_ERR_ARG;
  WorldCtr h;
  std::memset(&h, 0, sizeof(h));
  h.extent[0] = w->d.sp[0].cap;
  h.extent[1] = w->d.sp[1].cap;
  *bytes = image_bytes(w, h);
  return ABM_OK;
}

extern "C" abm_status abm_save(abm_world* w, void* buf, size_t* bytes, void* stream) {
  if (!w || !bytes) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  WorldCtr h;
  ABM_CUDA_TRY(cudaMemcpyAsync(&h, w->d.ctr, sizeof(WorldCtr), cudaMemcpyDeviceToHost, st));
  ABM_CUDA_TRY(cudaStreamSynchronize(st));
  const size_t need = image_bytes(w, h);
  if (!buf) {
    *bytes = need;
    return ABM_OK;
  }
  if (*bytes < need) return ABM_ERR_ARG;
  char* p = (char*)buf;
  std::memcpy(p, &h, sizeof(WorldCtr));
  p += sizeof(WorldCtr);
  for (int s = 0; s < 2; ++s) {
    const size_t n = (size_t)h.extent[s];
    if (n) {
      ABM_CUDA_TRY(cudaMemcpyAsync(p, w->d.sp[s].active, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      p += n * sizeof(int32_t);
      ABM_CUDA_TRY(cudaMemcpyAsync(p, w->d.sp[s].agent, n * sizeof(int4), cudaMemcpyDeviceToHost, st));
      p += n * sizeof(int4);
    }
  }
  ABM_CUDA_TRY(cudaMemcpyAsync(p, w->d.regrow, (size_t)w->d.ncells * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  ABM_CUDA_TRY(cudaStreamSynchronize(st));
  *bytes = need;
  return ABM_OK;
}

__global__ void k_reset_tables(WorldDev w) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < w.ncells; c += gridDim.x * blockDim.x) {
    w.gclaim[c] = kNoKey;
    w.victim[c] = kNoKey;
    w.wclaim[c] = kNoKey;
  }
}

extern "C" abm_status abm_load(abm_world* w, const void* buf, size_t bytes, void* stream) {
  if (!w || !buf || bytes < sizeof(WorldCtr)) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const char* p = (const char*)buf;
  WorldCtr h;
  std::memcpy(&h, p, sizeof(h));
  for (int s = 0; s < 2; ++s)
    if (h.extent[s] < 0 || h.extent[s] > w->d.sp[s].cap) return ABM_ERR_ARG;
  if (bytes < image_bytes(w, h)) return ABM_ERR_ARG;
  ABM_CUDA_TRY(cudaMemcpyAsync(w->d.ctr, p, sizeof(WorldCtr), cudaMemcpyHostToDevice, st));
  p += sizeof(WorldCtr);
  for (int s = 0; s < 2; ++s) {
    const size_t n = (size_t)h.extent[s], cap = (size_t)w->d.sp[s].cap;
    if (n) {
      ABM_CUDA_TRY(cudaMemcpyAsync(w->d.sp[s].active, p, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      p += n * sizeof(int32_t);
      ABM_CUDA_TRY(cudaMemcpyAsync(w->d.sp[s].agent, p, n * sizeof(int4), cudaMemcpyHostToDevice, st));
      p += n * sizeof(int4);
    }
    if (n < cap) {  // past the extent: empty slots, as in a world that never used them
      ABM_CUDA_TRY(cudaMemsetAsync(w->d.sp[s].active + n, 0, (cap - n) * sizeof(int32_t), st));
      ABM_CUDA_TRY(cudaMemsetAsync(w->d.sp[s].agent + n, 0, (cap - n) * sizeof(int4), st));
    }
    const int ntiles = w->cap_pad[s] / kPredTile;
    ABM_CUDA_TRY(cudaMemsetAsync(w->d.sp[s].tiles, 0, sizeof(u64) * (size_t)ntiles, st));
  }
  ABM_CUDA_TRY(cudaMemcpyAsync(w->d.regrow, p, (size_t)w->d.ncells * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  k_reset_tables<<<num_sms() * 4, 256, 0, st>>>(w->d);
  ABM_LAUNCH_CHECK();
  ABM_CUDA_TRY(cudaMemsetAsync(w->d.ps.acc, 0, sizeof(int) * 8, st));
  for (int s = 0; s < 2; ++s)
    ABM_CUDA_TRY(cudaMemsetAsync(w->d.ps.seg[s], 0, sizeof(u64) * (size_t)std::max(1, w->pgrid_max), st));
  ABM_CUDA_TRY(cudaMemsetAsync(w->d.ps.bar, 0, sizeof(u32) * 2, st));
  w->bar_next = 0;
  ABM_CUDA_TRY(cudaStreamSynchronize(st));
  w->steps_host = h.step;
  return ABM_OK;
}

extern "C" abm_status abm_digest(abm_world* w, uint64_t* out, void* stream) {
  if (!w || !out) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ABM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
  k_world_digest<<<num_sms() * 4, kPredThreads, 0, st>>>(w->d, (u64*)out);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_world_slab(abm_world* w, int32_t species, abm_slab** out, void* stream) {
  if (!w || !out || species < 0 || species > 1) return ABM_ERR_ARG;
  if (!w->view[species]) {
    abm_status e = slab_create_view(w->d.sp[species].cap, w->d.seed, w->d.model, w->d.sp[species].active,
                                    reinterpret_cast<int32_t*>(w->d.sp[species].agent), &w->view[species]);
    if (e != ABM_OK) return e;
  }
  k_view_open<<<1, 1, 0, (cudaStream_t)stream>>>(w->d.ctr, species, w->view[species]->d.counters);
  ABM_LAUNCH_CHECK();
  *out = w->view[species];
  return ABM_OK;
}

extern "C" abm_status abm_world_slab_commit(abm_world* w, int32_t species, void* stream) {
  if (!w || species < 0 || species > 1) return ABM_ERR_ARG;
  abm_slab* v = w->view[species];
  if (!v) return ABM_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  int* scan = v->d.meta;  // free between the view's calls
  ABM_CUDA_TRY(cudaMemsetAsync(scan, 0, sizeof(int) * 2, st));
  const int cap = w->d.sp[species].cap;
  k_view_scan<<<std::max(1, std::min((cap + 255) / 256, num_sms() * 4)), 256, 0, st>>>(w->d.sp[species].active, cap,
                                                                                       scan);
  ABM_LAUNCH_CHECK();
  k_view_commit<<<1, 1, 0, st>>>(w->d.ctr, species, v->d.counters, scan);
  ABM_LAUNCH_CHECK();
  // the per-cell claim tables are rebuilt by the next step, as after abm_load
  k_reset_tables<<<num_sms() * 4, 256, 0, st>>>(w->d);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}
