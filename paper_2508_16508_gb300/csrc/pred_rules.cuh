// Predation rules shared by the single-model and the batched kernels
// (ABMax Section 5.1, Fig. 3): the neighbour move and the claim keys.
#pragma once

#include "common.cuh"

namespace abm {

// Parameter slots of a model (int32; the thresholds are u32 bit patterns).
enum {
  PRM_SHEEP_GAIN = 0, PRM_WOLF_GAIN = 1, PRM_SHEEP_T = 2, PRM_WOLF_T = 3,
  PRM_REGROWTH = 4, PRM_SHEEP_METAB = 5, PRM_WOLF_METAB = 6, PRM_GRASS_T = 7
};

// Random move to one of the 8 neighbours on the periodic lattice, indexed by
// the top three bits of the MOVE draw, one nibble (offset + 1) per direction:
// (-1,-1) (0,-1) (1,-1) (-1,0) (1,0) (-1,1) (0,1) (1,1).
__device__ __forceinline__ int step_cell(int cell, int L, u32 dir) {
  const int dx = (int)((0x21020210u >> (4u * dir)) & 0xFu) - 1;
  const int dy = (int)((0x22211000u >> (4u * dir)) & 0xFu) - 1;
  const int y = cell / L;
  int x = cell - y * L + dx;
  int yy = y + dy;
  if (x < 0) x += L;
  if (x >= L) x -= L;
  if (yy < 0) yy += L;
  if (yy >= L) yy -= L;
  return yy * L + x;
}

// claim key: lexicographic (priority draw, slot) packed into 64 bits
__device__ __forceinline__ u64 claim_key(u32 prio, int slot) { return ((u64)prio << 32) | (u32)slot; }

// State digest of a model (abm_digest, abm_batch_digest): the wrapping sum of
// one hash per live agent (species, slot, cell, energy, id, age), per cell
// (steps until its grass is edible) and per species counter (live, next id,
// high-water mark). A sum does not depend on the order of its terms, so any
// parallel reduction gives the same value, and nothing in it depends on the
// capacity. The hash is the splitmix64 finaliser (Steele, Lea, Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014).
__device__ __forceinline__ u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ u64 digest_agent(int sp, int slot, int4 a) {
  u64 z = mix64(((u64)sp << 40) ^ (u64)(u32)slot);
  z = mix64(z ^ (((u64)(u32)a.x << 32) | (u32)a.y));
  return mix64(z ^ (((u64)(u32)a.z << 32) | (u32)a.w));
}

// regrow = the first step the cell's grass is edible, step = the current step
__device__ __forceinline__ u64 digest_cell(int c, int regrow, int step) {
  const u32 wait = regrow <= step ? 0u : (u32)(regrow - step);
  return mix64((2ull << 40) ^ ((u64)(u32)c << 8) ^ ((u64)wait << 40));
}

__device__ __forceinline__ u64 digest_counters(const int (&n_active)[2], const int (&next_id)[2], const int (&hw)[2]) {
  u64 t = 0;
  for (int sp = 0; sp < 2; ++sp) {
    t += mix64(0xC0FFEEull + sp * 7 + ((u64)(u32)n_active[sp] << 20));
    t += mix64(0xBADull + sp * 11 + ((u64)(u32)next_id[sp] << 20));
    t += mix64(0xF00Dull + sp * 13 + ((u64)(u32)hw[sp] << 20));
  }
  return t;
}

}  // namespace abm
