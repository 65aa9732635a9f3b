// Generic fixed-capacity agent set ("Set", ABMax Section 2) and the selection /
// compaction / distinct-update primitives of Section 4 (Algorithms 1 and 2),
// plus per-resource conflict resolution.
//
// Every rank-matched operation is ONE pass over the slab: each CTA takes a
// tile, computes per-slot flags from the 128-bit loaded live flags, ranks them
// with a block scan plus a decoupled look-back, and scatters the records at
// those ranks while the tile is still in registers. The i-th selected slot
// receiving the i-th record is exactly Rank-Match's pairing (cumsum(mask) *
// mask on both sides, matched on equal nonzero ranks), computed in O(n + k)
// instead of O(n * k).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.cuh"

namespace abm {

static int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    g_num_sms = n > 0 ? n : 1;
  }
  return g_num_sms;
}

constexpr int kSlabThreads = 256;
constexpr int kSlabItems = 8;  // 8 slots per thread: two 128-bit loads of live flags
constexpr int kSlabTile = kSlabThreads * kSlabItems;
constexpr int kMaxFields = 16;

struct SlabDev {
  int32_t* active;
  int32_t* fields;   // cap x Fp, agent-major
  int32_t* counters; // [0] n_active [1] next_id [2] overflow [3] scratch count
  int32_t* rec_idx;  // [cap] compacted record indices (scratch)
  int32_t* pending;  // [2] scan totals handed from the last tile to the last CTA out
  int* err;
  int cap, F, Fp;
  u32 seed, model;
};

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
  ScanCtl ctl;
  int n;                   // slots (or array entries for OP_ARRAY)
  const int32_t* src;      // OP_ARRAY: mask array
  const int32_t* rec;      // records [k][F]
  const int32_t* rec2;     // OP_FUSED: deltas [k][F]
  int k;
  int op_kind;             // ABM_OP_ADD / ABM_OP_SET for OP_UPDATE
  int id_field;            // OP_ADD
  int use_rec_idx;         // OP_UPDATE with a record mask
  u32 step, threshold;     // OP_FUSED
  int32_t* out_idx;        // OP_SELECT / OP_ARRAY: compacted indices; OP_ADD/OP_UPDATE: slots
  int32_t* out_count;      // device outputs (nullable)
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

template <int OP>
__global__ void __launch_bounds__(kSlabThreads) k_scan_op(ScanArgs a, int ntiles) {
  __shared__ u64 s_warp[kSlabThreads / 32 + 1];
  __shared__ u32 s_bcast[2];
  __shared__ int s_tile;
  const u32 tag = launch_tag(a.ctl.ctrl);
  const SlabDev& s = a.s;

  while (true) {
    const int tile = next_tile(a.ctl.ctrl, &s_tile);
    if (tile >= ntiles) break;
    const int base = tile * kSlabTile + threadIdx.x * kSlabItems;

    int live[kSlabItems];
    u32 fa = 0, fb = 0, removed = 0;  // bit masks over the thread's items
    const int32_t* flag_src = OP == OP_ARRAY ? a.src : s.active;
#pragma unroll
    for (int v = 0; v < kSlabItems / 4; ++v) {
      int4 q = make_int4(0, 0, 0, 0);
      if (base + 4 * v + 3 < a.n) {
        q = *reinterpret_cast<const int4*>(flag_src + base + 4 * v);
      } else {
        if (base + 4 * v + 0 < a.n) q.x = flag_src[base + 4 * v + 0];
        if (base + 4 * v + 1 < a.n) q.y = flag_src[base + 4 * v + 1];
        if (base + 4 * v + 2 < a.n) q.z = flag_src[base + 4 * v + 2];
      }
      live[4 * v + 0] = q.x; live[4 * v + 1] = q.y; live[4 * v + 2] = q.z; live[4 * v + 3] = q.w;
    }
#pragma unroll
    for (int j = 0; j < kSlabItems; ++j) {
      const int slot = base + j;
      const bool valid = slot < a.n;
      bool fA = false, fB = false;
      if (OP == OP_ARRAY) {
        fA = valid && live[j] != 0;
      } else if (OP == OP_SELECT || OP == OP_REMOVE || OP == OP_UPDATE) {
        fA = valid && eval_pred(a.pred, s, slot, live[j]);
      } else if (OP == OP_ADD) {
        fA = valid && live[j] == 0;
      } else {  // OP_FUSED
        if (valid) {
          const uint4 u = draw4(s.seed, s.model, a.step, (u32)slot, ABM_P_MASK, 0u);
          const bool rm = live[j] && u.x < a.threshold;
          const bool alive = live[j] && !rm;
          fA = !alive;
          fB = alive && u.y < a.threshold;
          if (rm) removed |= 1u << j;
        }
      }
      fa |= (u32)fA << j;
      fb |= (u32)fB << j;
    }
    u32 ex_a, ex_b, tot_a, tot_b, pre_a, pre_b;
    block_scan2<kSlabThreads>(__popc(fa), __popc(fb), ex_a, ex_b, tot_a, tot_b, s_warp);
    tile_prefix<kSlabThreads>(a.ctl, tile, tag, tot_a, tot_b, pre_a, pre_b, s_bcast);
    u32 ra = pre_a + ex_a, rb = pre_b + ex_b;

    // the last tile knows the totals; the last CTA out applies them
    if (tile == ntiles - 1 && threadIdx.x == 0) {
      s.pending[0] = (int)(pre_a + tot_a);
      s.pending[1] = (int)(pre_b + tot_b);
    }

    // scatter
    const int next_id = (OP == OP_ADD && a.id_field >= 0) ? s.counters[1] : 0;
    const int nrec = (OP == OP_UPDATE && a.use_rec_idx) ? s.counters[3] : a.k;
    int newlive[kSlabItems];
    bool dirty = false;
#pragma unroll
    for (int j = 0; j < kSlabItems; ++j) {
      const int slot = base + j;
      newlive[j] = live[j];
      if (!((fa >> j) & 1u)) {
        if (OP == OP_FUSED && ((removed >> j) & 1u)) { newlive[j] = 0; dirty = true; }
        if (OP == OP_FUSED && ((fb >> j) & 1u)) {
          if ((int)rb < a.k)
            apply_record(s.fields + (size_t)slot * s.Fp, a.rec2 + (size_t)rb * s.F, s.F, true);
          ++rb;
        }
        continue;
      }
      const u32 rank = ra++;
      if (OP == OP_SELECT || OP == OP_ARRAY) {
        a.out_idx[rank] = slot;
      } else if (OP == OP_REMOVE) {
        newlive[j] = 0;
        dirty = true;
      } else if (OP == OP_ADD || OP == OP_FUSED) {
        if ((int)rank < a.k) {
          int32_t* dst = s.fields + (size_t)slot * s.Fp;
          apply_record(dst, a.rec + (size_t)rank * s.F, s.F, false);
          if (OP == OP_ADD && a.id_field >= 0) dst[a.id_field] = (int)((u32)next_id + rank);
          if (OP == OP_ADD && a.out_idx) a.out_idx[rank] = slot;
          newlive[j] = 1;
          dirty = true;
        } else if (OP == OP_FUSED && ((removed >> j) & 1u)) {
          newlive[j] = 0;
          dirty = true;
        }
      } else if (OP == OP_UPDATE) {
        if ((int)rank < nrec) {
          const int rj = a.use_rec_idx ? s.rec_idx[rank] : (int)rank;
          apply_record(s.fields + (size_t)slot * s.Fp, a.rec + (size_t)rj * s.F, s.F,
                       a.op_kind == ABM_OP_ADD);
          if (a.out_idx) a.out_idx[rank] = slot;
        }
      }
    }
    if (OP == OP_REMOVE || OP == OP_ADD || OP == OP_FUSED) {
      if (dirty) {
#pragma unroll
        for (int v = 0; v < kSlabItems / 4; ++v) {
          const int b0 = base + 4 * v;
          if (b0 + 3 < a.n) {
            *reinterpret_cast<int4*>(s.active + b0) =
                make_int4(newlive[4 * v], newlive[4 * v + 1], newlive[4 * v + 2], newlive[4 * v + 3]);
          } else {
            for (int j = 0; j < 4; ++j)
              if (b0 + j < a.n) s.active[b0 + j] = newlive[4 * v + j];
          }
        }
      }
    }
  }
  if (last_cta_out(a.ctl.ctrl)) {
    const int A = ntiles > 0 ? s.pending[0] : 0;
    const int B = ntiles > 0 ? s.pending[1] : 0;
    if (OP == OP_SELECT || OP == OP_ARRAY) {
      if (a.out_count) *a.out_count = A;
      if (OP == OP_ARRAY) s.counters[3] = A;
    } else if (OP == OP_REMOVE) {
      s.counters[0] -= A;
      if (a.out_count) *a.out_count = A;
    } else if (OP == OP_ADD) {
      const int r = min(a.k, A);
      s.counters[0] += r;
      if (a.id_field >= 0) s.counters[1] += r;
      if (a.k > A) s.counters[2] = 1;
      if (a.out_count) *a.out_count = r;
    } else if (OP == OP_UPDATE) {
      const int nrec = a.use_rec_idx ? s.counters[3] : a.k;
      if (a.out_count) *a.out_count = min(A, nrec);
    } else {  // OP_FUSED: A = free after removal, B = chosen survivors
      const int n_before = s.counters[0];
      const int added = min(a.k, A);
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

// --------------------------------------------------------------------------
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

struct abm_slab {
  SlabDev d;
  u64* tiles;
  u32* ctrl;      // [4] main scan, [4..8) array scan
  u64* tiles2;
  int ntiles_max;
  int n_pad;
  int grid;
};

static ScanCtl ctl_main(abm_slab* s) { return ScanCtl{s->tiles, s->ctrl, s->d.err}; }
static ScanCtl ctl_aux(abm_slab* s) { return ScanCtl{s->tiles2, s->ctrl + 4, s->d.err}; }

extern "C" const char* abm_strerror(abm_status st) {
  switch (st) {
    case ABM_OK: return "ok";
    case ABM_ERR_ARG: return "invalid argument";
    case ABM_ERR_OOM: return "device allocation failed";
    case ABM_ERR_CUDA: return "CUDA runtime error";
    case ABM_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case ABM_ERR_OVERFLOW: return "more agents asked for a slot than were free";
    case ABM_ERR_STATE: return "operation not valid for this handle";
  }
  return "unknown status";
}

extern "C" int32_t abm_version(void) { return 100; }

extern "C" abm_status abm_slab_destroy(abm_slab* s) {
  if (!s) return ABM_ERR_ARG;
  cudaFree(s->d.active);
  cudaFree(s->d.fields);
  cudaFree(s->d.counters);
  cudaFree(s->d.rec_idx);
  cudaFree(s->d.pending);
  cudaFree(s->d.err);
  cudaFree(s->tiles);
  cudaFree(s->tiles2);
  cudaFree(s->ctrl);
  delete s;
  return ABM_OK;
}

extern "C" abm_status abm_slab_create(int32_t capacity, int32_t n_fields, uint32_t seed,
                                      uint32_t model, int32_t init, void* stream, abm_slab** out) {
  if (!out || capacity < 1 || capacity > (1 << 28) - 1 || n_fields < 1 || n_fields > kMaxFields ||
      (init != ABM_INIT_EMPTY && init != ABM_INIT_HALF_LIVE))
    return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  abm_slab* s = new (std::nothrow) abm_slab();
  if (!s) return ABM_ERR_OOM;
  std::memset(s, 0, sizeof(*s));
  s->d.cap = capacity;
  s->d.F = n_fields;
  s->d.Fp = (n_fields + 3) & ~3;
  s->d.seed = seed;
  s->d.model = model;
  s->ntiles_max = (capacity + kSlabTile - 1) / kSlabTile;
  s->n_pad = s->ntiles_max * kSlabTile;
  bool ok = cudaMalloc(&s->d.active, sizeof(int32_t) * (size_t)s->n_pad) == cudaSuccess &&
            cudaMalloc(&s->d.fields, sizeof(int32_t) * (size_t)s->n_pad * s->d.Fp) == cudaSuccess &&
            cudaMalloc(&s->d.counters, sizeof(int32_t) * 4) == cudaSuccess &&
            cudaMalloc(&s->d.rec_idx, sizeof(int32_t) * (size_t)capacity) == cudaSuccess &&
            cudaMalloc(&s->d.err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&s->d.pending, sizeof(int32_t) * 2) == cudaSuccess &&
            cudaMalloc(&s->tiles, sizeof(u64) * (size_t)s->ntiles_max) == cudaSuccess &&
            cudaMalloc(&s->tiles2, sizeof(u64) * (size_t)s->ntiles_max) == cudaSuccess &&
            cudaMalloc(&s->ctrl, sizeof(u32) * 8) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    abm_slab_destroy(s);
    return ABM_ERR_OOM;
  }
  s->grid = num_sms() * 8;
  if (cudaMemsetAsync(s->d.counters, 0, sizeof(int32_t) * 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->d.err, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(s->tiles, 0, sizeof(u64) * (size_t)s->ntiles_max, st) != cudaSuccess ||
      cudaMemsetAsync(s->tiles2, 0, sizeof(u64) * (size_t)s->ntiles_max, st) != cudaSuccess ||
      cudaMemsetAsync(s->ctrl, 0, sizeof(u32) * 8, st) != cudaSuccess) {
    abm_slab_destroy(s);
    return ABM_ERR_CUDA;
  }
  k_slab_init<<<num_sms() * 4, 256, 0, st>>>(s->d, init, s->n_pad);
  k_count_live<<<num_sms() * 4, 256, 0, st>>>(s->d);
  if (cudaGetLastError() != cudaSuccess) {
    abm_slab_destroy(s);
    return ABM_ERR_CUDA;
  }
  *out = s;
  return ABM_OK;
}

extern "C" abm_status abm_slab_check(abm_slab* s, void* stream) {
  if (!s) return ABM_ERR_ARG;
  ABM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int err = 0;
  ABM_CUDA_TRY(cudaMemcpy(&err, s->d.err, sizeof(int), cudaMemcpyDeviceToHost));
  return err ? ABM_ERR_DEVICE_TIMEOUT : ABM_OK;
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

template <int OP>
static abm_status launch_scan(abm_slab* s, const ScanArgs& a, const ScanCtl& ctl, cudaStream_t st) {
  ScanArgs b = a;
  b.ctl = ctl;
  const int ntiles = (b.n + kSlabTile - 1) / kSlabTile;
  const int grid = std::max(1, std::min(ntiles, s->grid));
  k_scan_op<OP><<<grid, kSlabThreads, 0, st>>>(b, ntiles);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
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
  a.out_idx = out_idx;
  a.out_count = out_count;
  return launch_scan<OP_SELECT>(s, a, ctl_main(s), (cudaStream_t)stream);
}

extern "C" abm_status abm_remove(abm_slab* s, const abm_pred* pred, int32_t* out_removed, void* stream) {
  if (!s || !pred_ok(s, pred) || pred->kind == ABM_PRED_FREE) return ABM_ERR_ARG;
  ScanArgs a = base_args(s);
  a.pred = to_dev(pred);
  a.out_count = out_removed;
  return launch_scan<OP_REMOVE>(s, a, ctl_main(s), (cudaStream_t)stream);
}

extern "C" abm_status abm_add(abm_slab* s, const int32_t* records, int32_t k, int32_t id_field,
                              int32_t* out_slots, int32_t* out_added, void* stream) {
  if (!s || k < 0 || (k > 0 && !records) || id_field < -1 || id_field >= s->d.F) return ABM_ERR_ARG;
  ScanArgs a = base_args(s);
  a.rec = records;
  a.k = k;
  a.id_field = id_field;
  a.out_idx = out_slots;
  a.out_count = out_added;
  return launch_scan<OP_ADD>(s, a, ctl_main(s), (cudaStream_t)stream);
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
    r.out_idx = s->d.rec_idx;
    abm_status e = launch_scan<OP_ARRAY>(s, r, ctl_aux(s), st);
    if (e != ABM_OK) return e;
  }
  ScanArgs a = base_args(s);
  a.pred = to_dev(pred);
  a.rec = records;
  a.k = k;
  a.op_kind = op;
  a.use_rec_idx = record_mask != nullptr;
  a.out_idx = out_slots;
  a.out_count = out_applied;
  return launch_scan<OP_UPDATE>(s, a, ctl_main(s), st);
}

extern "C" abm_status abm_selective_update(abm_slab* s, uint32_t step, uint32_t threshold,
                                           const int32_t* records, const int32_t* deltas, int32_t k,
                                           int32_t* out_counts, void* stream) {
  if (!s || k < 0 || (k > 0 && (!records || !deltas))) return ABM_ERR_ARG;
  ScanArgs a = base_args(s);
  a.rec = records;
  a.rec2 = deltas;
  a.k = k;
  a.step = step;
  a.threshold = threshold;
  a.out_count = out_counts;
  return launch_scan<OP_FUSED>(s, a, ctl_main(s), (cudaStream_t)stream);
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
