// Device state of one predation world, shared by the per-phase kernels
// (predation.cu) and the persistent step kernel (pred_persistent.cu).
#pragma once

#include "pred_rules.cuh"

namespace abm {

constexpr int kPredThreads = 256;
constexpr int kPredItems = 4;  // one 128-bit load of live flags per thread
constexpr int kPredTile = kPredThreads * kPredItems;

struct SpeciesDev {
  int32_t* active;   // [cap_pad]
  int4* agent;       // [cap_pad]: cell, energy, id, age
  int32_t* parents;  // [cap] compacted parent slots
  int32_t* freel;    // [cap] compacted free slots (only the first n_active are written)
  u64* tiles;        // decoupled look-back states
  u32* ctrl;         // [0..4) scan control, [4..8) births exit counter
  int cap;
};

struct WorldCtr {
  int n_active[2], next_id[2], hw[2], overflow[2], extent[2], step;
  int parents[2], free_in[2];
  int starved[2], eaten, grass_eaten;
  int n_start[2];
  u32 energy_exit[4];
  long long energy[2];
};

// scratch of the persistent step kernel
struct PersistDev {
  u32* plane[2][2];   // per species: [0] free, [1] parent bit-planes (cap/32 words)
  u64* blk[2];        // per species: (free << 32 | parents) of each 128-slot unit (cap/128)
  u64* seg[2];        // per species: the same summed over each CTA's run of units (max CTAs)
  u32* bar;           // [0] grid-barrier arrivals (monotonic, wraps)
  int* acc;           // [2][4] per-step accumulators by step parity: starved0, starved1, eaten, grass
};

struct WorldDev {
  SpeciesDev sp[2];
  PersistDev ps;
  int32_t* regrow;  // first step at which the cell's grass is edible
  u64* gclaim;      // per-cell grass claims (sheep)
  u64* victim;      // per-cell victim keys (sheep)
  u64* wclaim;      // per-cell wolf claims
  WorldCtr* ctr;
  int* err;
  int side, ncells;
  u32 seed, model;
  u32 bar_base;     // barrier arrivals before this launch (persistent kernel)
  int params[8];
  // ABM_VARIANT_MANY_WOLVES: per-cell lists of this step's live sheep and
  // wolves. Heads reuse `victim` (sheep) and `wclaim` (wolves); a head or link
  // is (step << 32 | slot), so entries of earlier steps end a list and no list
  // is ever cleared. key = the agent's (draw, slot) key.
  int variant;
  u64* skey;        // [cap sheep]
  u64* snext;       // [cap sheep]
  u64* wkey;        // [cap wolves]
  u64* wnext;       // [cap wolves]
};

// persistent step kernel (pred_persistent.cu)
int persistent_max_ctas();
int persistent_warps();
abm_status launch_persistent(const WorldDev& d, u32* bar_next, int grid, int nsteps, abm_step_stats* stats,
                             cudaStream_t st,
                             unsigned long long* phase_ns = nullptr);

}  // namespace abm
