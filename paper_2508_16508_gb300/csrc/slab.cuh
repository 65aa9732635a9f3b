// Device and host state of a slab (a fixed-capacity agent set), shared by the
// slab passes (slab.cu) and the slab sort (sort.cu).
#pragma once
#include "common.cuh"

namespace abm {

constexpr int kSlabTileMax = 16384;  // slab arrays are padded to a multiple of this

struct SlabDev {
  int32_t* active;
  int32_t* fields;   // cap x Fp, agent-major
  int32_t* counters; // [0] n_active [1] next_id [2] overflow [3] scratch count
  int32_t* rec_idx;  // [cap] compacted record indices (scratch)
  int32_t* meta;     // [4] pass-2 results for pass 3: rank counts, first id
  int* err;
  int cap, F, Fp;
  u32 seed, model;
};

struct SortScratch;
void sort_scratch_free(SortScratch* p);

}  // namespace abm

struct abm_slab {
  abm::SlabDev d;
  abm::u32* planes;    // 2 x n_pad / 32 words: bit-planes A, B of the slab passes
  abm::u32* planes2;   // n_pad / 32 words: plane A of record-mask compaction
  abm::u32* totals;    // [2 * max CTAs] per-CTA counts (slab passes)
  abm::u32* totals2;   // the same for record-mask compaction
  abm::u32* wtotals;   // [2 * max CTAs * 16 warps] per-warp counts
  abm::u32* wtotals2;
  int32_t* lista;  // [cap] scratch slot lists when the caller wants none
  int32_t* listb;
  abm::u32* ctrl;      // [0..4) slab passes, [4..8) record-mask compaction
  int n_pad;
  int max_ctas;
  // shape of the fused selective-update pass (abm_slab_tune)
  int fused_threads, fused_ctas_per_sm;
  abm::SortScratch* sort;  // buffers of abm_sort, allocated by its first call
  int view;                // 1: active / fields belong to a predation world (abm_world_slab)
};

namespace abm {
// A slab over arrays owned by someone else (a world's species): own scratch
// and counters, borrowed live flags and fields (F = Fp = 4). Freed by
// slab_free_view, never by abm_slab_destroy.
abm_status slab_create_view(int cap, u32 seed, u32 model, int32_t* active, int32_t* fields, abm_slab** out);
void slab_free_view(abm_slab* s);
// check builds: canaries in the fields past the capacity (fields: n_pad x Fp)
abm_status slab_canary_fill(int32_t* fields, int Fp, int cap, int n_pad, cudaStream_t st);
// check builds: records kErrCheck in *err if the canaries past the capacity changed
abm_status canary_check(const int32_t* active, const int32_t* fields, int Fp, int cap, int n_pad, int* err,
                        cudaStream_t st);
}  // namespace abm
