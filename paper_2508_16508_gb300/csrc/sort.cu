// sort_agents (ABMax Section 2 API list): reorder a slab so that its live
// agents come first, ascending by one int32 field with ties kept in slot
// order, and the placeholders after them in slot order.
//
// LSD radix sort of (key, value) pairs, key = the field with its sign bit
// flipped (so unsigned order is signed order), value = the slot with the
// placeholder flag in bit 31: four passes over the key bytes, then one pass
// over the flag. Each pass: per-tile digit histograms -> one exclusive scan
// over (digit, tile) -> each tile ranks its items stably per digit in shared
// memory (warp match + per-warp digit counts) and writes them at their global
// positions. Finally every agent's row (fields + live flag) is gathered into
// spare arrays, which then become the slab's arrays.
#include <algorithm>
#include <new>

#include "slab.cuh"

namespace abm {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kBins = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;
constexpr u32 kPlaceholder = 0x80000000u;  // value bit: the slot holds no agent

struct SortScratch {
  int cap, n_pad, Fp, G;
  u32* key[2];
  u32* val[2];
  u32* hist;        // [kBins * G], scanned in place
  u32* sums;        // per scan block
  int32_t* fields;  // [n_pad * Fp]: the next fields array
  int32_t* active;  // [n_pad]: the next live-flag array
  int* nonbinary;   // set when a live flag is neither 0 nor 1 (the gather then copies them)
};

void sort_scratch_free(SortScratch* p) {
  if (!p) return;
  for (int b = 0; b < 2; ++b) {
    cudaFree(p->key[b]);
    cudaFree(p->val[b]);
  }
  cudaFree(p->hist);
  cudaFree(p->sums);
  cudaFree(p->fields);
  cudaFree(p->active);
  cudaFree(p->nonbinary);
  delete p;
}

__global__ void k_sort_init(SlabDev s, int field, u32* key, u32* val, int* nonbinary) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.cap; i += gridDim.x * blockDim.x) {
    const int a = s.active[i];
    if (a != 0 && a != 1) *nonbinary = 1;
    const bool live = a != 0;
    key[i] = live ? ((u32)s.fields[(size_t)i * s.Fp + field] ^ 0x80000000u) : 0u;
    val[i] = (u32)i | (live ? 0u : kPlaceholder);
  }
}

__device__ __forceinline__ u32 digit_of(u32 key, u32 val, int pass) {
  return pass < 4 ? (key >> (8 * pass)) & 0xFFu : val >> 31;
}

// per-tile digit counts, digit-major: hist[d * G + tile]
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const u32* __restrict__ key, const u32* __restrict__ val,
                                                            int n, int pass, int G, u32* hist) {
  __shared__ u32 s_cnt[kBins];
  s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  const int t = blockIdx.x;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int i = t * kSortTile + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&s_cnt[pass < 4 ? digit_of(key[i], 0u, pass) : digit_of(0u, val[i], pass)], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * G + t] = s_cnt[threadIdx.x];
}

// exclusive scan of a[0..n): blocks of kScanBlock, their sums, the offsets
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(u32* a, int n, u32* sums) {
  __shared__ u64 s_warp[kScanThreads / 32 + 1];
  const int b0 = blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  u32 v[kScanItems];
  u32 local = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = b0 + j < n ? a[b0 + j] : 0u;
    local += v[j];
  }
  u32 ex, ex2, tot, tot2;
  block_scan2<kScanThreads>(local, 0u, ex, ex2, tot, tot2, s_warp);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (b0 + j < n) a[b0 + j] = ex;
    ex += v[j];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(u32* sums, int nb) {
  __shared__ u64 s_warp[kScanThreads / 32 + 1];
  u32 carry = 0;
  for (int c0 = 0; c0 < nb; c0 += kScanThreads) {
    const int i = c0 + threadIdx.x;
    const u32 v = i < nb ? sums[i] : 0u;
    u32 ex, ex2, tot, tot2;
    block_scan2<kScanThreads>(v, 0u, ex, ex2, tot, tot2, s_warp);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(u32* a, int n, const u32* sums) {
  const u32 add = sums[blockIdx.x];
  const int b0 = blockIdx.x * kScanBlock;
  for (int j = threadIdx.x; j < kScanBlock; j += kScanThreads)
    if (b0 + j < n) a[b0 + j] += add;
}

// Stable scatter of one pass. The tile's items are taken in rounds of 256
// (slot order within the tile = round, warp, lane); an item's rank among the
// tile's items with its digit = the count from earlier rounds + the counts of
// lower warps in this round + the lower lanes of its warp with that digit.
// The items are first placed in shared memory in (digit, rank) order, then
// written out in that order, so that consecutive threads write consecutive
// addresses of one digit's run.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const u32* __restrict__ key, const u32* __restrict__ val,
                                                               int n, int pass, int G, const u32* __restrict__ off,
                                                               u32* key_out, u32* val_out) {
  __shared__ u32 s_key[kSortTile], s_val[kSortTile];  // the tile in (digit, rank) order
  __shared__ u32 s_run[kBins];                // items of each digit in earlier rounds
  __shared__ u32 s_off[kBins];                // the tile's global offset of each digit
  __shared__ u32 s_start[kBins];              // a digit's first position in the tile order
  __shared__ unsigned short s_wc[kSortWarps][kBins];  // this round's count per warp and digit
  __shared__ u64 s_warp[kSortWarps + 1];
  const int t = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tile = min(kSortTile, n - t * kSortTile);
  {
    // the tile's count of digit d: the next (digit, tile) entry's offset minus its own
    const size_t e = (size_t)threadIdx.x * G + t;
    const u32 o = off[e];
    const u32 next = e + 1 < (size_t)kBins * G ? off[e + 1] : (u32)n;
    u32 ex, ex2, tot, tot2;
    block_scan2<kSortThreads>(next - o, 0u, ex, ex2, tot, tot2, s_warp);
    s_off[threadIdx.x] = o;
    s_start[threadIdx.x] = ex;
    s_run[threadIdx.x] = 0u;
  }
  for (int w = 0; w < kSortWarps; ++w) s_wc[w][threadIdx.x] = 0;
  __syncthreads();
  const u32 lt = (1u << lane) - 1u;
  u32 kr[kSortItems], vr[kSortItems];  // all of the thread's items in flight at once
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int j = r * kSortThreads + threadIdx.x;
    kr[r] = j < n_tile ? key[t * kSortTile + j] : 0u;
    vr[r] = j < n_tile ? val[t * kSortTile + j] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int j = r * kSortThreads + threadIdx.x;
    const bool ok = j < n_tile;
    const u32 k = kr[r], v = vr[r];
    const u32 d = ok ? digit_of(k, v, pass) : (u32)kBins;  // kBins: no item
    const u32 peers = __match_any_sync(0xFFFFFFFFu, d);
    const u32 below = (u32)__popc(peers & lt);
    if (ok && below == 0) s_wc[warp][d] = (unsigned short)__popc(peers);
    __syncthreads();
    if (ok) {
      u32 pos = s_start[d] + s_run[d] + below;
      for (int w = 0; w < warp; ++w) pos += s_wc[w][d];
      s_key[pos] = k;
      s_val[pos] = v;
    }
    __syncthreads();
    {
      u32 add = 0;
      for (int w = 0; w < kSortWarps; ++w) {
        add += s_wc[w][threadIdx.x];
        s_wc[w][threadIdx.x] = 0;
      }
      s_run[threadIdx.x] += add;
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n_tile; j += kSortThreads) {
    const u32 k = s_key[j], v = s_val[j];
    const u32 d = digit_of(k, v, pass);
    const u32 pos = s_off[d] + ((u32)j - s_start[d]);
    key_out[pos] = k;
    val_out[pos] = v;
  }
}

// row i of the sorted slab <- row (val[i] without the flag) of the old one
__global__ void k_sort_gather(SlabDev s, const u32* __restrict__ val, int32_t* fields_out, int32_t* active_out,
                              int32_t* perm_out, const int* nonbinary) {
  const bool exact = *nonbinary != 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.cap; i += gridDim.x * blockDim.x) {
    const u32 v = val[i];
    const int src = (int)(v & ~kPlaceholder);
    // the flag travels with the value; only other nonzero live values need the old array
    active_out[i] = exact ? s.active[src] : ((v & kPlaceholder) ? 0 : 1);
    const int32_t* a = s.fields + (size_t)src * s.Fp;
    int32_t* b = fields_out + (size_t)i * s.Fp;
    for (int f = 0; f < s.Fp; f += 4) *reinterpret_cast<int4*>(b + f) = *reinterpret_cast<const int4*>(a + f);
    if (perm_out) perm_out[i] = src;
  }
}

static abm_status sort_scratch(abm_slab* s, SortScratch** out) {
  if (s->sort) {
    *out = s->sort;
    return ABM_OK;
  }
  SortScratch* p = new (std::nothrow) SortScratch();
  if (!p) return ABM_ERR_OOM;
  p->cap = s->d.cap;
  p->n_pad = s->n_pad;
  p->Fp = s->d.Fp;
  p->G = (s->d.cap + kSortTile - 1) / kSortTile;
  const size_t nh = (size_t)kBins * p->G;
  const size_t nb = (nh + kScanBlock - 1) / kScanBlock;
  bool ok = true;
  for (int b = 0; b < 2 && ok; ++b)
    ok = cudaMalloc(&p->key[b], sizeof(u32) * (size_t)p->cap) == cudaSuccess &&
         cudaMalloc(&p->val[b], sizeof(u32) * (size_t)p->cap) == cudaSuccess;
  ok = ok && cudaMalloc(&p->hist, sizeof(u32) * nh) == cudaSuccess;
  ok = ok && cudaMalloc(&p->sums, sizeof(u32) * nb) == cudaSuccess;
  ok = ok && cudaMalloc(&p->fields, sizeof(int32_t) * (size_t)p->n_pad * p->Fp) == cudaSuccess;
  ok = ok && cudaMalloc(&p->active, sizeof(int32_t) * (size_t)p->n_pad) == cudaSuccess;
  ok = ok && cudaMalloc(&p->nonbinary, sizeof(int)) == cudaSuccess;
  // rows past the capacity are never gathered: keep them as the slab keeps its own
  ok = ok && cudaMemset(p->fields, 0, sizeof(int32_t) * (size_t)p->n_pad * p->Fp) == cudaSuccess;
  ok = ok && cudaMemset(p->active, 0, sizeof(int32_t) * (size_t)p->n_pad) == cudaSuccess;
  if (kCheck && ok)  // check builds: the spare arrays carry the canaries too (they become the slab's)
    ok = slab_canary_fill(p->fields, p->Fp, s->d.cap, p->n_pad, 0) == ABM_OK && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sort_scratch_free(p);
    return ABM_ERR_OOM;
  }
  s->sort = p;
  *out = p;
  return ABM_OK;
}

}  // namespace abm

using namespace abm;

extern "C" abm_status abm_sort(abm_slab* s, int32_t field, int32_t* out_perm, void* stream) {
  if (!s || field < 0 || field >= s->d.F) return ABM_ERR_ARG;
  if (s->view) return ABM_ERR_STATE;  // the sort swaps the slab's arrays, which a world's view does not own
  SortScratch* p = nullptr;
  abm_status e = sort_scratch(s, &p);
  if (e != ABM_OK) return e;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = s->d.cap, G = p->G;
  const int nh = kBins * G;
  const int nb = (nh + kScanBlock - 1) / kScanBlock;
  const int grid = std::max(1, std::min((n + 255) / 256, num_sms() * 8));
  ABM_CUDA_TRY(cudaMemsetAsync(p->nonbinary, 0, sizeof(int), st));
  k_sort_init<<<grid, 256, 0, st>>>(s->d, field, p->key[0], p->val[0], p->nonbinary);
  ABM_LAUNCH_CHECK();
  int cur = 0;
  for (int pass = 0; pass < 5; ++pass) {
    k_sort_hist<<<G, kSortThreads, 0, st>>>(p->key[cur], p->val[cur], n, pass, G, p->hist);
    ABM_LAUNCH_CHECK();
    k_scan_blocks<<<nb, kScanThreads, 0, st>>>(p->hist, nh, p->sums);
    ABM_LAUNCH_CHECK();
    k_scan_sums<<<1, kScanThreads, 0, st>>>(p->sums, nb);
    ABM_LAUNCH_CHECK();
    k_scan_add<<<nb, kScanThreads, 0, st>>>(p->hist, nh, p->sums);
    ABM_LAUNCH_CHECK();
    k_sort_scatter<<<G, kSortThreads, 0, st>>>(p->key[cur], p->val[cur], n, pass, G, p->hist, p->key[cur ^ 1],
                                               p->val[cur ^ 1]);
    ABM_LAUNCH_CHECK();
    cur ^= 1;
  }
  k_sort_gather<<<grid, 256, 0, st>>>(s->d, p->val[cur], p->fields, p->active, out_perm, p->nonbinary);
  ABM_LAUNCH_CHECK();
  // the gathered arrays become the slab's; the old ones are the next sort's targets
  std::swap(s->d.fields, p->fields);
  std::swap(s->d.active, p->active);
  return ABM_OK;
}
