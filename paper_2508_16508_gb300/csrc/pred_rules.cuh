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

}  // namespace abm
