// Device-side building blocks shared by the engine's kernels (sm_103a).
//
//  - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
//    "Parallel random numbers: as easy as 1, 2, 3", SC'11).
//  - Single-pass stable compaction: per-thread flag counts, warp shuffles and
//    a block scan, then a decoupled look-back across tiles whose states carry
//    two 28-bit counts, an "inclusive" bit and a 7-bit launch tag (so tile
//    states never need clearing between launches). Every spin is bounded.
//  - "Last CTA out" bookkeeping that resets per-launch counters on device,
//    which keeps the kernels CUDA-graph replayable without memset nodes.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/abm.h"

namespace abm {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u64 kNoKey = 0xFFFFFFFFFFFFFFFFull;
constexpr int kMaxSpin = 1 << 23;  // bounded waits: ~2 s with the back-off below

// Device error codes written into a handle's error word.
constexpr int kErrTimeout = 1;
constexpr int kErrCheck = 2;  // check builds: an index out of range or a damaged canary

// Check builds (compiled with -DABM_CHECK into libabm_check.so; a stand-in for
// a memory checker): data-dependent indices are tested before they are used,
// and the padding past each slab's capacity holds canaries that the *_check
// calls verify. Other builds compile every test away.
#ifdef ABM_CHECK
constexpr bool kCheck = true;
#else
constexpr bool kCheck = false;
#endif
constexpr int kCanary = 0x7E57CA11;  // agent fields past the capacity (live flags there stay 0)

// true iff 0 <= i < n; in a check build a violation is recorded in *err (the
// first error word set wins) and false is returned, so that the caller skips
// the access. Always true in other builds.
__device__ __forceinline__ bool in_range(long long i, long long n, int* err) {
  if constexpr (kCheck) {
    if (i < 0 || i >= n) {
      if (err) atomicCAS(err, 0, kErrCheck);
      return false;
    }
  }
  return true;
}

// ----------------------------------------------------------------------------
// Philox4x32-10: ten rounds; each multiplies counter words 0 and 2 by the two
// round constants, xors the high halves with the other two counter words and
// the key, and keeps the low halves; the key advances by the Weyl constants.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const u32 p0_lo = 0xD2511F53u * c.x, p0_hi = __umulhi(0xD2511F53u, c.x);
    const u32 p1_lo = 0xCD9E8D57u * c.z, p1_hi = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(p1_hi ^ c.y ^ k.x, p1_lo, p0_hi ^ c.w ^ k.y, p0_lo);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the ten rounds' key words given (rk[2r], rk[2r+1] =
// the key after r Weyl steps), e.g. from a kernel's parameters, so that each
// round's key is an operand instead of an addition.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const u32 (&rk)[20]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const u32 p0_lo = 0xD2511F53u * c.x, p0_hi = __umulhi(0xD2511F53u, c.x);
    const u32 p1_lo = 0xCD9E8D57u * c.z, p1_hi = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(p1_hi ^ c.y ^ rk[2 * r], p1_lo, p0_hi ^ c.w ^ rk[2 * r + 1], p0_lo);
  }
  return c;
}

// host: the round keys of key (seed, model) for philox_rk
inline void philox_round_keys(u32 seed, u32 model, u32 (&rk)[20]) {
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = seed + (u32)r * 0x9E3779B9u;
    rk[2 * r + 1] = model + (u32)r * 0xBB67AE85u;
  }
}

__device__ __forceinline__ uint4 draw4(u32 seed, u32 model, u32 step, u32 slot, u32 purpose,
                                       u32 species) {
  return philox(make_uint4(step, slot, purpose, species), make_uint2(seed, model));
}

__device__ __forceinline__ u32 draw(u32 seed, u32 model, u32 step, u32 slot, u32 purpose,
                                    u32 species) {
  return draw4(seed, model, step, slot, purpose, species).x;
}

// asynchronous global -> shared copies (16 bytes: both addresses 16-byte
// aligned; 4 bytes: 4-byte aligned), completed by cp_async_wait_0
__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// uniform integer in [0, n) by multiply-shift
__device__ __forceinline__ int uniform_below(u32 u, int n) {
  return (int)(((u64)u * (u64)(u32)n) >> 32);
}

// ----------------------------------------------------------------------------
// relaxed GPU-scope 64-bit accesses for the tile states
__device__ __forceinline__ u64 ld_relaxed(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u32 ld_relaxed32(const u32* p) {
  u32 v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// tile state: [63:57] tag, [56] inclusive, [55:28] count a, [27:0] count b
__device__ __forceinline__ u64 tile_pack(u32 tag, u32 incl, u32 a, u32 b) {
  return ((u64)tag << 57) | ((u64)incl << 56) | ((u64)(a & 0xFFFFFFFu) << 28) | (u64)(b & 0xFFFFFFFu);
}
__device__ __forceinline__ u32 tile_tag(u64 v) { return (u32)(v >> 57); }
__device__ __forceinline__ u32 tile_incl(u64 v) { return (u32)(v >> 56) & 1u; }
__device__ __forceinline__ u32 tile_a(u64 v) { return (u32)(v >> 28) & 0xFFFFFFFu; }
__device__ __forceinline__ u32 tile_b(u64 v) { return (u32)v & 0xFFFFFFFu; }

// Per-scan control words (device u32[4]):
//   [0] tile ticket  [1] CTAs finished  [2] launch epoch  [3] spare
struct ScanCtl {
  u64* tiles;
  u32* ctrl;
  int* err;
};

__device__ __forceinline__ u32 launch_tag(const u32* ctrl) { return (ld_relaxed32(ctrl + 2) % 127u) + 1u; }

// Block-wide exclusive scan of two per-thread counts at once (packed into one
// u64 as a << 32 | b; block totals stay below 2^32 so the halves never mix).
template <int THREADS>
__device__ __forceinline__ void block_scan2(u32 a, u32 b, u32& ex_a, u32& ex_b, u32& tot_a, u32& tot_b,
                                            u64* s_warp /* [THREADS/32 + 1] */) {
  constexpr int W = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 v = ((u64)a << 32) | b;
  u64 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    u64 w = lane < W ? s_warp[lane] : 0ull;
    u64 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u64 t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < W) s_warp[lane] = wi - w;  // exclusive warp offsets
    if (lane == W - 1) s_warp[W] = wi;    // block total
  }
  __syncthreads();
  const u64 ex = s_warp[warp] + incl - v;
  const u64 tot = s_warp[W];
  ex_a = (u32)(ex >> 32);
  ex_b = (u32)ex;
  tot_a = (u32)(tot >> 32);
  tot_b = (u32)tot;
}

// Decoupled look-back. Called by every thread of the CTA after block_scan2;
// returns the exclusive prefix (a, b) of this tile. Warp 0 does the waiting.
template <int THREADS>
__device__ __forceinline__ void tile_prefix(const ScanCtl& ctl, int tile, u32 tag, u32 agg_a, u32 agg_b,
                                            u32& pre_a, u32& pre_b, u32* s_bcast /* [2] */) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    if (tile == 0) {
      if (lane == 0) {
        st_relaxed(&ctl.tiles[0], tile_pack(tag, 1u, agg_a, agg_b));
        s_bcast[0] = 0u;
        s_bcast[1] = 0u;
      }
    } else {
      if (lane == 0) st_relaxed(&ctl.tiles[tile], tile_pack(tag, 0u, agg_a, agg_b));
      u32 sa = 0, sb = 0;
      int pred = tile - 1;
      int spins = 0;
      bool timed_out = false;
      u32 backoff = 32;
      while (true) {
        const int idx = pred - lane;
        u64 v;
        while (true) {
          v = idx >= 0 ? ld_relaxed(&ctl.tiles[idx]) : tile_pack(tag, 1u, 0u, 0u);
          const bool ok = tile_tag(v) == tag;
          if (__all_sync(0xFFFFFFFFu, ok)) break;
          if (++spins > kMaxSpin) {
            timed_out = true;
            break;
          }
          if (spins > 16) __nanosleep(backoff);  // short spins first: the wait is usually brief
          if (spins > 64 && backoff < 256) backoff <<= 1;
        }
        if (timed_out) break;
        const u32 incl_mask = __ballot_sync(0xFFFFFFFFu, tile_incl(v) != 0u);
        const int stop = incl_mask ? (__ffs(incl_mask) - 1) : 31;
        u32 a = lane <= stop ? tile_a(v) : 0u;
        u32 b = lane <= stop ? tile_b(v) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
          b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
        }
        sa += a;
        sb += b;
        if (incl_mask) break;
        pred -= 32;
      }
      if (lane == 0) {
        if (timed_out) atomicExch(ctl.err, kErrTimeout);
        st_relaxed(&ctl.tiles[tile], tile_pack(tag, 1u, sa + agg_a, sb + agg_b));
        s_bcast[0] = sa;
        s_bcast[1] = sb;
      }
    }
  }
  __syncthreads();
  pre_a = s_bcast[0];
  pre_b = s_bcast[1];
}

// Next tile for this CTA (dynamic, in acquisition order: every predecessor of
// a tile was handed to a CTA that is already running).
__device__ __forceinline__ int next_tile(u32* ctrl, int* s_tile) {
  __syncthreads();
  if (threadIdx.x == 0) *s_tile = (int)atomicAdd(ctrl, 1u);
  __syncthreads();
  return *s_tile;
}

// Called by every CTA once it has finished all of its work. The last CTA out
// resets the ticket and the exit count and advances the epoch; it returns
// true in thread 0 of that CTA only, after a fence, so that the caller can do
// launch-wide finishing work (totals written by other CTAs are visible).
__device__ __forceinline__ bool last_cta_out(u32* ctrl) {
  __syncthreads();
  bool last = false;
  if (threadIdx.x == 0) {
    __threadfence();
    const u32 done = atomicAdd(ctrl + 1, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      ctrl[0] = 0u;
      ctrl[1] = 0u;
      ctrl[2] = ctrl[2] + 1u;
      last = true;
    }
  }
  return last;
}

// warp-aggregated atomic add of a per-thread count into *dst
__device__ __forceinline__ void warp_add(int* dst, int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// Programmatic dependent launch: a kernel launched with launch_pdl() may
// start before its predecessor in the stream has finished; it must call
// griddep_wait() before touching anything the predecessor writes.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace abm

// host-side helpers
#define ABM_CUDA_TRY(expr)                     \
  do {                                         \
    cudaError_t _e = (expr);                   \
    if (_e != cudaSuccess) return ABM_ERR_CUDA; \
  } while (0)

// status of a handle's device error word
#define ABM_ERR_OF(word) ((word) == 0 ? ABM_OK : ((word) == abm::kErrCheck ? ABM_ERR_CHECK : ABM_ERR_DEVICE_TIMEOUT))

#define ABM_LAUNCH_CHECK()                      \
  do {                                          \
    if (cudaGetLastError() != cudaSuccess) return ABM_ERR_CUDA; \
  } while (0)

namespace abm {
int num_sms();  // multiprocessor count of the current device (cached per device)

// A kernel's dynamic shared-memory limit is a per-device setting: set it once
// for each device a process uses (bit d of `done` records device d; devices
// beyond 63 set it on every call). Two threads that race on a device's first
// call both set it, which is harmless.
template <typename K>
inline cudaError_t smem_attr_once(K* kernel, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}
}
