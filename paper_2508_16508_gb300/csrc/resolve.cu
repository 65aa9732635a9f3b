// Conflict resolution: several agents claim one resource (ABMax Section 1;
// the per-cell priority of Section 5.2). Winner per resource = the claim with
// the smallest packed key (priority << 32 | claim index), i.e. the
// lexicographic minimum of (priority, index). atomicMin on a unique 64-bit
// key is order-independent, so the result is deterministic.
//
// Skewed (Zipf) claim distributions put a large share of the claims on a few
// resources; each CTA therefore first folds its chunk of claims into a
// shared-memory hash table (open addressing, smem 64-bit atomicMin) and then
// issues one global atomicMin per distinct resource it saw.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace abm {

constexpr int kResThreads = 512;
constexpr int kResPerThread = 8;
constexpr int kResChunk = kResThreads * kResPerThread;
constexpr int kHashBits = 13;
constexpr int kHash = 1 << kHashBits;  // 8192 entries x 12 B = 96 KiB of shared memory
constexpr int kMaxProbe = 64;

__global__ void k_table_fill(u64* table, int R) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) table[i] = kNoKey;
}

__global__ void __launch_bounds__(kResThreads) k_claims(const int32_t* __restrict__ res,
                                                        const u32* __restrict__ prio, int M, int R,
                                                        u64* table) {
  extern __shared__ unsigned char smem[];
  u64* s_best = reinterpret_cast<u64*>(smem);
  int* s_tag = reinterpret_cast<int*>(s_best + kHash);
  __shared__ int s_used;  // distinct resources in the table
  for (int h = threadIdx.x; h < kHash; h += kResThreads) {
    s_tag[h] = -1;
    s_best[h] = kNoKey;
  }
  if (threadIdx.x == 0) s_used = 0;
  __syncthreads();
  const int nchunks = (M + kResChunk - 1) / kResChunk;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int m0 = c * kResChunk;
#pragma unroll
    for (int j = 0; j < kResPerThread; ++j) {
      const int m = m0 + j * kResThreads + threadIdx.x;  // coalesced
      if (m >= M) continue;
      const int r = res[m];
      if (r < 0 || r >= R) continue;
      const u64 key = ((u64)prio[m] << 32) | (u32)m;
      u32 h = ((u32)r * 2654435761u) >> (32 - kHashBits);
      bool done = false;
      for (int p = 0; p < kMaxProbe; ++p) {
        int t = s_tag[h];
        if (t == -1) {
          t = atomicCAS(&s_tag[h], -1, r);
          if (t == -1) atomicAdd(&s_used, 1);
        }
        if (t == -1 || t == r) {
          atomicMin(&s_best[h], key);
          done = true;
          break;
        }
        h = (h + 1) & (kHash - 1);
      }
      if (!done) atomicMin(&table[r], key);  // table full around h: go straight to global
    }
    __syncthreads();
    // The table is folded into global memory only when it is half full or the
    // CTA has no chunks left: skewed claims (a few hot resources) then cost
    // one global atomic per distinct resource per CTA, not per chunk.
    if (s_used > kHash / 2 || c + (int)gridDim.x >= nchunks) {
      for (int h = threadIdx.x; h < kHash; h += kResThreads) {
        const int t = s_tag[h];
        if (t >= 0) {
          atomicMin(&table[t], s_best[h]);
          s_tag[h] = -1;
          s_best[h] = kNoKey;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_used = 0;
    }
    __syncthreads();
  }
}

// winner per resource, then restore the table to "no claim"
__global__ void k_winners(u64* table, int R, int32_t* winner) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) {
    const u64 v = table[i];
    winner[i] = v == kNoKey ? -1 : (int32_t)(u32)v;
    if (v != kNoKey) table[i] = kNoKey;
  }
}

__global__ void k_is_winner(const int32_t* __restrict__ res, int M, int R, const int32_t* __restrict__ winner,
                            uint8_t* is_winner) {
  // 4 claims per thread: one 128-bit load of resource ids, one 32-bit store of flags
  const int n4 = M >> 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
    const int4 r = reinterpret_cast<const int4*>(res)[q];
    const int m = q << 2;
    u32 f = 0;
    f |= (u32)(r.x >= 0 && r.x < R && winner[r.x] == m + 0) << 0;
    f |= (u32)(r.y >= 0 && r.y < R && winner[r.y] == m + 1) << 8;
    f |= (u32)(r.z >= 0 && r.z < R && winner[r.z] == m + 2) << 16;
    f |= (u32)(r.w >= 0 && r.w < R && winner[r.w] == m + 3) << 24;
    reinterpret_cast<u32*>(is_winner)[q] = f;
  }
  if (blockIdx.x == 0 && threadIdx.x < (M & 3)) {
    const int m = (n4 << 2) + threadIdx.x;
    const int r = res[m];
    is_winner[m] = (r >= 0 && r < R && winner[r] == m) ? 1 : 0;
  }
}

__global__ void k_is_winner_scalar(const int32_t* __restrict__ res, int M, int R,
                                   const int32_t* __restrict__ winner, uint8_t* is_winner) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    const int r = res[m];
    is_winner[m] = (r >= 0 && r < R && winner[r] == m) ? 1 : 0;
  }
}

static std::atomic<unsigned long long> g_res_attr{0};  // devices whose k_claims has its smem limit

abm_status resolve_launch(const int32_t* claim_res, const uint32_t* claim_prio, int32_t M, int32_t R,
                          uint64_t* table, int32_t* out_winner, uint8_t* out_is_winner, cudaStream_t st) {
  const size_t smem = (size_t)kHash * (sizeof(u64) + sizeof(int));
  ABM_CUDA_TRY(smem_attr_once(k_claims, (int)smem, g_res_attr));
  const int sms = num_sms();
  if (M > 0) {
    const int nchunks = (M + kResChunk - 1) / kResChunk;
    const int grid = std::max(1, std::min(nchunks, sms * 2));
    k_claims<<<grid, kResThreads, smem, st>>>(claim_res, claim_prio, M, R, (u64*)table);
    ABM_LAUNCH_CHECK();
  }
  k_winners<<<std::max(1, std::min((R + 255) / 256, sms * 8)), 256, 0, st>>>((u64*)table, R, out_winner);
  ABM_LAUNCH_CHECK();
  if (out_is_winner && M > 0) {
    if ((((uintptr_t)claim_res) & 15) == 0 && (((uintptr_t)out_is_winner) & 3) == 0) {
      k_is_winner<<<std::max(1, std::min((M / 4 + 255) / 256, sms * 8)), 256, 0, st>>>(
          claim_res, M, R, out_winner, out_is_winner);
    } else {
      k_is_winner_scalar<<<std::max(1, std::min((M + 255) / 256, sms * 8)), 256, 0, st>>>(
          claim_res, M, R, out_winner, out_is_winner);
    }
    ABM_LAUNCH_CHECK();
  }
  return ABM_OK;
}

}  // namespace abm

using namespace abm;

extern "C" abm_status abm_resolve_table_init(uint64_t* table, int32_t R, void* stream) {
  if (!table || R < 1) return ABM_ERR_ARG;
  k_table_fill<<<std::max(1, std::min((R + 255) / 256, num_sms() * 8)), 256, 0, (cudaStream_t)stream>>>(
      (u64*)table, R);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_resolve(const int32_t* claim_res, const uint32_t* claim_prio, int32_t M, int32_t R,
                                  uint64_t* table, int32_t* out_winner, uint8_t* out_is_winner, void* stream) {
  if (M < 0 || R < 1 || !table || !out_winner || (M > 0 && (!claim_res || !claim_prio))) return ABM_ERR_ARG;
  return resolve_launch(claim_res, claim_prio, M, R, table, out_winner, out_is_winner, (cudaStream_t)stream);
}

// ----------------------------------------------------------------------------
// Resolve without allocation: the scratch table lives in a fixed-size
// file-scope device array instead of caller- or library-allocated memory.
namespace abm {

static __device__ __align__(256) unsigned long long g_resolve_scratch[ABM_RESOLVE_STATIC_MAX_R];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static u64* g_scratch_ptr[kMaxDevices] = {};

// Device address of this device's copy of the array, looked up once per
// device (the array's name is only a host-side handle in host code).
static abm_status static_scratch(u64** out) {
  int dev = 0;
  ABM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return ABM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_resolve_scratch) != cudaSuccess || !p) return ABM_ERR_CUDA;
    g_scratch_ptr[dev] = (u64*)p;
  }
  *out = g_scratch_ptr[dev];
  return ABM_OK;
}

}  // namespace abm

extern "C" abm_status abm_resolve_static(const int32_t* claim_res, const uint32_t* claim_prio, int32_t M, int32_t R,
                                         int32_t* out_winner, uint8_t* out_is_winner, void* stream) {
  if (M < 0 || R < 1 || !out_winner || (M > 0 && (!claim_res || !claim_prio))) return ABM_ERR_ARG;
  if (R > ABM_RESOLVE_STATIC_MAX_R) return ABM_ERR_TOO_LARGE;
  u64* table = nullptr;
  abm_status e = static_scratch(&table);
  if (e != ABM_OK) return e;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps whatever the previous call left: empty the R entries used here
  k_table_fill<<<std::max(1, std::min((R + 255) / 256, num_sms() * 8)), 256, 0, st>>>(table, R);
  ABM_LAUNCH_CHECK();
  return resolve_launch(claim_res, claim_prio, M, R, (uint64_t*)table, out_winner, out_is_winner, st);
}
