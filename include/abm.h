/*
 * abm.h -- C ABI of the GB300 selective-update engine for agent-based models.
 *
 * The engine implements the hot path of ABMax (Chaturvedi, El-Gazzar, van
 * Gerven, arXiv 2508.16508): distinct updates to a dynamically selected,
 * variable-size subset of agents held in fixed-capacity arrays (Section 4),
 * driven by the wolf-sheep-grass predation model (Section 5.1).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an abm_status; ABM_OK is 0. abm_strerror() names it.
 *  - Pointers documented as "device" are CUDA device (or managed) pointers;
 *    "host" pointers are ordinary CPU memory. Nothing takes ownership of a
 *    caller's buffer; handles own the memory they allocate and free it in
 *    their destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). All work is enqueued asynchronously on it; device outputs are
 *    valid once the stream reaches that point. Calls that return host values
 *    synchronise the stream and say so.
 *  - Counts returned through device pointers are int32. A NULL output pointer
 *    means "not wanted" unless the argument is documented as required.
 *  - Argument errors (NULL where required, negative sizes, sizes beyond a
 *    documented limit) return ABM_ERR_ARG before anything is enqueued.
 *  - Spin-waits inside kernels are bounded. A wait that runs out sets a
 *    device error word and the kernel returns; abm_*_check() reports
 *    ABM_ERR_DEVICE_TIMEOUT and the handle's results are then undefined.
 *  - Check build (libabm_check.so, the same sources compiled with -DABM_CHECK,
 *    slower): every data-dependent index (a slot from a list, a cell from an
 *    agent record, a parent, a victim) is tested before use; a violation is
 *    recorded in the handle's error word and the access skipped. The padding
 *    past each slab's capacity holds canaries (agent fields 0x7E57CA11, live
 *    flags 0). abm_slab_check / abm_world_check / abm_batch_check then report
 *    ABM_ERR_CHECK for a recorded violation or a damaged canary. abm_version()
 *    is negative in a check build.
 *  - Randomness is Philox4x32-10 (Salmon et al., SC'11) with counter
 *    (step, slot, purpose, species) and key (seed, model); a probability p is
 *    an integer threshold T = floor(p * 2^32) and an event happens iff the
 *    32-bit draw is below T.
 */
#ifndef ABM_H
#define ABM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t abm_status;
#define ABM_OK 0
#define ABM_ERR_ARG 1            /* invalid argument; nothing was enqueued */
#define ABM_ERR_OOM 2            /* device allocation failed */
#define ABM_ERR_CUDA 3           /* a CUDA runtime call failed */
#define ABM_ERR_DEVICE_TIMEOUT 4 /* a bounded device-side wait ran out */
#define ABM_ERR_OVERFLOW 5       /* informational: more agents asked for a slot than were free */
#define ABM_ERR_STATE 6          /* operation not valid for this handle */
#define ABM_ERR_TOO_LARGE 7      /* size beyond a fixed, documented maximum */
#define ABM_ERR_CHECK 8          /* check build only: an index out of range or a damaged canary was recorded */

const char* abm_strerror(abm_status s);
/* Library version: major * 10000 + minor * 100 + patch. */
int32_t abm_version(void);

/* Philox purposes (counter word 2). Species word 3: 0 sheep or generic slab,
 * 1 wolf, 2 grass. Initialisation draws use step ABM_INIT_STEP. */
#define ABM_P_MOVE 1
#define ABM_P_PRIO 2
#define ABM_P_REPRO 3
#define ABM_P_VICTIM 4
#define ABM_P_INIT_AGENT 5
#define ABM_P_GRASS_INIT 6
#define ABM_P_MASK 7
#define ABM_P_NEWREC0 9
#define ABM_P_NEWREC1 10
#define ABM_P_DELTA0 11
#define ABM_P_DELTA1 12
#define ABM_P_RESOURCE 13
#define ABM_P_INIT_ACTIVE 14
#define ABM_INIT_STEP 0xFFFFFFFFu

/* ========================================================================== */
/* Generic fixed-capacity agent set ("Set", Section 2)                        */
/* ========================================================================== */
/*
 * A slab holds `capacity` slots. Slot i has an int32 live flag and F int32
 * fields. Device layout: active[capacity] (int32, 0/1) and fields stored
 * agent-major, capacity x Fp int32 with Fp = F rounded up to a multiple of 4
 * (so one agent's fields are one 16/32-byte run). Placeholders (inactive
 * slots) keep their last field values. Limits: 1 <= capacity <= 2^28 - 1,
 * 1 <= F <= 16. Every call reads a nonzero flag as live. abm_add and
 * abm_selective_update write the flags of the 16-slot groups they fill (and
 * abm_selective_update those of the 8-slot groups it empties) whole, as 0/1,
 * so a flag other than 0 or 1 stored there by abm_slab_write becomes 1; the
 * other calls leave such values as they are.
 */
typedef struct abm_slab abm_slab;

#define ABM_INIT_EMPTY 0     /* all slots free, fields zero */
#define ABM_INIT_HALF_LIVE 1 /* slot i live iff draw(INIT_STEP, i, INIT_ACTIVE, 0).w0 < 2^31;
                                field f = word f%4 of draw(INIT_STEP, i, NEWREC0 + f/4, 0) */

abm_status abm_slab_create(int32_t capacity, int32_t n_fields, uint32_t seed, uint32_t model,
                           int32_t init, void* stream, abm_slab** out);
abm_status abm_slab_destroy(abm_slab* s);
/* Synchronises `stream`, then reports any device-side error recorded for the slab. */
abm_status abm_slab_check(abm_slab* s, void* stream);
/* Device pointers to the slab's arrays (valid until destroy or abm_sort,
 * which replaces them). */
abm_status abm_slab_arrays(abm_slab* s, int32_t** active, int32_t** fields, int32_t* fields_stride);
/* Copy `n` slots starting at slot 0 of field `field` (or the live flags for
 * field = -1) into / out of a device buffer of n int32. */
abm_status abm_slab_read(abm_slab* s, int32_t field, int32_t* dst, int32_t n, void* stream);
abm_status abm_slab_write(abm_slab* s, int32_t field, const int32_t* src, int32_t n, void* stream);

/* Selection predicates (select_agents, Section 2; the masks of Algorithms 1/2). */
#define ABM_PRED_LIVE 0      /* live slots */
#define ABM_PRED_FREE 1      /* placeholder slots */
#define ABM_PRED_BERNOULLI 2 /* live and word 0 of draw(step, slot, purpose, species) < threshold */
#define ABM_PRED_MASK 3      /* live and mask[slot] != 0 (device int32[capacity]) */
#define ABM_PRED_FIELD 4     /* live and ((field value & and_mask) <cmp> value) */
#define ABM_CMP_EQ 0
#define ABM_CMP_NE 1
#define ABM_CMP_LT 2
#define ABM_CMP_GE 3
typedef struct abm_pred {
  int32_t kind;
  uint32_t threshold, step, purpose, species; /* BERNOULLI */
  const int32_t* mask;                        /* MASK (device) */
  int32_t field, cmp, and_mask, value;        /* FIELD */
} abm_pred;

/* select_agents (Section 2): the slots satisfying `pred`, ascending, written
 * to out_idx[0..count) (device int32[capacity], required); the count goes to
 * *out_count (device int32, required). Stable stream compaction. */
abm_status abm_select(abm_slab* s, const abm_pred* pred, int32_t* out_idx, int32_t* out_count,
                      void* stream);

/* sort_agents (Section 2 API list): reorder the slab so that the live agents
 * come first, ascending by the int32 `field` (signed order; ties keep their
 * slot order), and the placeholders after them in slot order. Every row
 * moves whole (all fields and the live flag); counters are unchanged.
 * out_perm (device int32[capacity], nullable): out_perm[i] = the old slot of
 * the row now in slot i. The first call allocates the sort's buffers (about
 * 16 bytes a slot plus one spare copy of the slab, kept until destroy); the
 * slab's arrays are replaced by the sorted copies (abm_slab_arrays changes).
 * LSD radix sort: four passes over the key bytes and one over the live flag. */
abm_status abm_sort(abm_slab* s, int32_t field, int32_t* out_perm, void* stream);

/* ========================================================================== */
/* Limit order books (Section 5.3: noisy traders' limit orders in fixed-size   */
/* books, all books matched in parallel by price sorting and share cumsums)    */
/* ========================================================================== */
/*
 * n_books books of `cap` order slots (1 <= cap <= ABM_LOB_MAX_CAP), each
 * array device int32[n_books][cap] (book-major): active (0/1), side (0 buy,
 * any other value sell), price (ticks, 1 .. 2^31 - 1), qty (shares >= 1),
 * time (any int32; priority among equal prices). Values outside these ranges
 * give unspecified books but no out-of-bounds access. ABM_ERR_ARG for
 * n_books < 0, cap outside [1, ABM_LOB_MAX_CAP], kmax < 0 or a null array;
 * n_books = 0 launches nothing. Asynchronous on `stream`; the caller owns
 * every buffer. The paper gives no exact rules; these are:
 *
 * abm_lob_match -- one matching round of every book. Bids in priority order
 * (price descending, then time, then slot), asks likewise (price ascending);
 * the traded volume V is the largest share count such that the bid holding
 * share V is priced at or above the ask holding share V (0 if none), and the
 * first V shares of each side trade: an order fills clamp(V - shares ahead of
 * it, 0, qty); filled orders become inactive, the others keep the rest of
 * their qty. out_volume (device int64[n_books]) = V; out_price (device
 * int32[n_books]) = the price of the ask holding share V, -1 if V = 0.
 * One CTA per book, sorted in shared memory.
 *
 * abm_lob_add -- new orders into each book's vacant slots (the add of
 * Section 4 per book; the stock-exchange case of Section 4's example): order
 * j < k[b] of book b (new_orders device int32[n_books][kmax][4] = side,
 * price, qty, time; k device int32[n_books], values clamped to [0, kmax])
 * goes into the j-th free slot of book b, ascending, j < min(k[b], free);
 * new_orders may be null when kmax = 0. out_added device int32[n_books] =
 * orders placed.
 */
#define ABM_LOB_MAX_CAP 2048
/* Launch shape of abm_lob_match's price-level path for the rest of the
 * process: warps matching one book (1, 2 or 4; 0 = the default, 2). Results
 * never depend on it. ABM_ERR_ARG for other values. Host only. */
abm_status abm_lob_tune(int32_t warps_per_book);
abm_status abm_lob_match(int32_t n_books, int32_t cap, int32_t* active, const int32_t* side, const int32_t* price,
                         int32_t* qty, const int32_t* time, int64_t* out_volume, int32_t* out_price, void* stream);
abm_status abm_lob_add(int32_t n_books, int32_t cap, int32_t* active, int32_t* side, int32_t* price, int32_t* qty,
                       int32_t* time, const int32_t* new_orders, const int32_t* k, int32_t kmax, int32_t* out_added,
                       void* stream);

/* select_agents with SCI's index exposure (Algorithm 2, Section 4): a
 * permutation of all slots, those satisfying `pred` first, then the others,
 * each group ascending -- the stable argsort of the mask with true first.
 * out_perm: device int32[capacity] (required); *out_count (device int32,
 * required) = the number satisfying `pred`. Two stream compactions on
 * `stream`. */
abm_status abm_select_permutation(abm_slab* s, const abm_pred* pred, int32_t* out_perm, int32_t* out_count,
                                  void* stream);

/* set_agents_mask (Section 2) as removal: every slot satisfying `pred` becomes
 * a placeholder. *out_removed (device, nullable) = number removed. */
abm_status abm_remove(abm_slab* s, const abm_pred* pred, int32_t* out_removed, void* stream);

/* Adding agents with distinct initial states (Section 4 toy task with free
 * slots as targets; Algorithm 1 rank matching): record j (records = device
 * int32[k][F], row-major) goes to the j-th free slot in ascending order, for
 * j < r = min(k, #free). If id_field >= 0 that field is set to the slab's
 * next id + j and next id advances by r. out_slots (device int32[k],
 * nullable) receives the slots; *out_added (device, nullable) = r. When
 * k > #free the slab's overflow flag is set (abm_slab_counters). */
abm_status abm_add(abm_slab* s, const int32_t* records, int32_t k, int32_t id_field,
                   int32_t* out_slots, int32_t* out_added, void* stream);

/* Distinct updates (Algorithms 1 and 2, set_agents_rm / set_agents_sci): the
 * i-th slot satisfying `pred` (ascending) receives the i-th selected record,
 * for i < r = min(#selected slots, #selected records). Records are device
 * int32[k][F]; record_mask (device int32[k], nullable = all) selects records.
 * op ABM_OP_ADD adds field-wise with 32-bit wrap-around; ABM_OP_SET
 * overwrites. out_slots (device int32[min(k,capacity)], nullable) gets the
 * updated slots; *out_applied (device, nullable) = r. A non-NULL record_mask
 * needs k <= capacity. */
#define ABM_OP_ADD 0
#define ABM_OP_SET 1
abm_status abm_update_distinct(abm_slab* s, const abm_pred* pred, const int32_t* records,
                               const int32_t* record_mask, int32_t k, int32_t op,
                               int32_t* out_slots, int32_t* out_applied, void* stream);

/* Selective-update call, fused into one pass over the slab (the microbenchmark
 * of the selection / add / remove / distinct-update primitives). With one
 * draw u = draw(step, slot, MASK, 0) per slot:
 *   1. remove every live slot with u.w0 < threshold;
 *   2. the i-th slot still live with u.w1 < threshold (ascending) gets delta
 *      record i added field-wise (wrapping), i < min(k, #chosen);
 *   3. record j goes to the j-th free slot (after 1), j < min(k, #free).
 * Steps 2 and 3 touch disjoint slots, so the result equals abm_remove,
 * abm_update_distinct and abm_add issued in that order with those
 * predicates. records and deltas are device int32[k][F]. out_counts (device
 * int32[3], nullable) = removed, added, updated. */
abm_status abm_selective_update(abm_slab* s, uint32_t step, uint32_t threshold,
                                const int32_t* records, const int32_t* deltas, int32_t k,
                                int32_t* out_counts, void* stream);

/* Launch shape of abm_selective_update's passes: `threads` per CTA (128, 256
 * or 512) and `ctas_per_sm` CTAs per SM (threads * ctas_per_sm <= 2048).
 * Results never depend on it; the autotuner picks it. Default 256, 8. */
abm_status abm_slab_tune(abm_slab* s, int32_t threads, int32_t ctas_per_sm, void* stream);

/* Fill out[k][F] (device int32) with record j field f = word f%4 of
 * draw(step, j, purpose0 + (f >= 4 ? purpose1 - purpose0 : 0), 0) under the
 * slab's key -- the Philox-generated records of the microbenchmark. */
abm_status abm_philox_records(abm_slab* s, uint32_t step, uint32_t purpose0, uint32_t purpose1,
                              int32_t k, int32_t* out, void* stream);

typedef struct abm_slab_counters {
  int32_t n_active, next_id, overflow, reserved;
} abm_slab_counters;
/* Host copy of the slab's counters (synchronises `stream`). */
abm_status abm_slab_counters_get(abm_slab* s, abm_slab_counters* out, void* stream);

/* ========================================================================== */
/* Conflict resolution (Section 1: several agents claim one resource;         */
/* Section 5.2: per-cell priority)                                            */
/* ========================================================================== */
/* Claim m (0 <= m < M) asks for resource claim_res[m]; a claim whose resource
 * is outside [0, R) is ignored. Per resource the claim with the
 * lexicographically smallest (claim_prio[m], m) wins.
 *  claim_res, claim_prio: device int32[M] / uint32[M] (required when M > 0).
 *  table: device uint64[R] scratch; every entry must be 0xFFFFFFFFFFFFFFFF
 *         before the call (abm_resolve_table_init) and is left so after it.
 *  out_winner: device int32[R] (required): winning claim index or -1.
 *  out_is_winner: device uint8[M] (nullable): 1 for winning claims.
 * Limits: 0 <= M, 1 <= R <= 2^31 - 1. */
abm_status abm_resolve_table_init(uint64_t* table, int32_t R, void* stream);
abm_status abm_resolve(const int32_t* claim_res, const uint32_t* claim_prio, int32_t M, int32_t R,
                       uint64_t* table, int32_t* out_winner, uint8_t* out_is_winner, void* stream);

/* abm_resolve for callers that cannot allocate device memory. (The paper has
 * no counterpart; this is a deployment variant.) Some hosts of this library
 * must not call cudaMalloc once they are running: an engine that owns a fixed
 * device-memory budget and hands out every byte itself, a serving loop where
 * an allocation's implicit synchronisation would stall other streams, or an
 * embedding that forbids the CUDA allocator outright. This entry point
 * allocates nothing -- no cudaMalloc, cudaFree or allocating library call --
 * and takes no scratch argument: its per-resource table is a file-scope
 * device array of ABM_RESOLVE_STATIC_MAX_R 64-bit entries (2 MiB). The caller
 * still passes the inputs and outputs (same meaning as abm_resolve).
 *  - R above ABM_RESOLVE_STATIC_MAX_R returns ABM_ERR_TOO_LARGE.
 *  - The array belongs to the library's device code, which CUDA loads onto a
 *    device lazily (by default) the first time the library touches that
 *    device: from then on the device holds the 2 MiB until the process exits.
 *  - The first call on a device also looks the array's device address up
 *    (cudaGetSymbolAddress) with that device current, and may be the moment
 *    the module is loaded (one driver allocation). So make one call on each
 *    device -- a warm-up with M = 0 will do -- before any stream capture and
 *    before the period in which the host forbids allocation; later calls
 *    allocate nothing.
 *  - All calls share the one array. Each call empties the entries it uses
 *    before claiming, so nothing carries over between calls, but calls that
 *    overlap on the GPU (different streams, or different host threads on the
 *    same device) race on it and give undefined results. */
#define ABM_RESOLVE_STATIC_MAX_R (1 << 18)
abm_status abm_resolve_static(const int32_t* claim_res, const uint32_t* claim_prio, int32_t M, int32_t R,
                              int32_t* out_winner, uint8_t* out_is_winner, void* stream);

/* ========================================================================== */
/* Predation model (Section 5.1, Fig. 3)                                      */
/* ========================================================================== */
/*
 * Wolves, sheep and grass on a periodic side x side lattice (cell = y*side+x).
 * Per step, in this order: sheep move to a random 8-neighbour (word 0 of the
 * MOVE draw, top 3 bits), lose `metabolism` energy, age by 1; sheep on grown
 * grass claim it and the smallest (PRIO draw, slot) sheep per cell eats
 * (+gain, grass regrows `regrowth` steps later); live sheep with energy >= 0
 * and REPRO draw < T reproduce in ascending slot order into the lowest free
 * slots (r = min(parents, free); child on the parent's cell with floor(e/2)
 * energy, age 0, id next_id + i; the parent keeps e - floor(e/2)); sheep with
 * energy < 0 die. Wolves then do the same, except that eating means: per
 * cell, the live sheep with the smallest (VICTIM draw, slot) is the victim
 * and the smallest (PRIO draw, slot) wolf on that cell eats it (+gain, the
 * sheep is removed).
 *
 * params[8] (int32; thresholds are u32 bit patterns): sheep gain, wolf gain,
 * sheep reproduction T, wolf reproduction T, grass regrowth delay, sheep
 * metabolism, wolf metabolism, initial-grass T. Initial agent k of species s
 * sits in slot k with cell = (w0 * side^2) >> 32 and energy =
 * (w1 * 2 * gain) >> 32 of draw(INIT_STEP, k, INIT_AGENT, s); cell c's grass
 * is grown iff w0 < initial-grass T and otherwise waits (w1 * regrowth) >> 32
 * steps, from draw(INIT_STEP, c, GRASS_INIT, 2).
 *
 * Limits: 1 <= side <= 46340, 0 <= n0[s] <= cap[s] <= 2^28 - 1.
 */
typedef struct abm_world abm_world;

/* Rule variants (bits; the paper fixes neither):
 * 0 (ONE_WOLF): per cell, the live wolf with the smallest (PRIO draw, slot)
 *   eats the live sheep with the smallest (VICTIM draw, slot); at most one per
 *   cell and step.
 * MANY_WOLVES: per cell, the i-th wolf by (PRIO draw, slot) eats the i-th
 *   sheep by (VICTIM draw, slot), i < min(#wolves, #sheep) (NetLogo lets every
 *   wolf eat; Algorithm 1's rank matching inside each cell).
 * GRASS_OFF: sheep neither eat grass nor spend energy moving (Wilensky's
 *   model without grass); the grass state still evolves.
 * Any variant bit: persistent engine only (abm_world_tune refuses the
 * per-phase kernels for such a world, and so do energy statistics). */
#define ABM_VARIANT_ONE_WOLF 0
#define ABM_VARIANT_MANY_WOLVES 1
#define ABM_VARIANT_GRASS_OFF 2

typedef struct abm_config {
  int32_t side;
  uint32_t seed, model;
  int32_t params[8];
  int32_t cap[2];
  int32_t n0[2];
  int32_t variant; /* ABM_VARIANT_* */
} abm_config;

/* Per-step statistics, written by the device (one record per step). */
typedef struct abm_step_stats {
  int32_t n_start[2];   /* live agents when the step started */
  int32_t parents[2];   /* agents selected to reproduce */
  int32_t births[2];    /* children placed */
  int32_t starved[2];   /* agents removed with energy < 0 */
  int32_t eaten;        /* sheep eaten by wolves */
  int32_t grass_eaten;  /* cells grazed */
  int32_t n_end[2];     /* live agents at the end of the step */
  int32_t hw[2];        /* maximum post-birth population so far */
  int32_t overflow[2];  /* 1 once parents outnumbered free slots */
  int32_t step;         /* index of this step */
  int32_t extent[2];    /* highest slot ever used + 1, when the step started */
  int32_t reserved;
  int64_t energy[2];    /* total live energy at the end of the step (only when requested) */
} abm_step_stats;

abm_status abm_create(const abm_config* cfg, void* stream, abm_world** out);
abm_status abm_destroy(abm_world* w);
/* Advance `nsteps` steps. stats: abm_step_stats[nsteps] (nullable) in memory
 * the kernels can write: device memory, or pinned host memory mapped into the
 * device's address space (cudaHostAlloc; with unified addressing its host
 * pointer serves), which the host may read once the call's work on `stream`
 * has completed -- the statistics then reach the host with no copy.
 * want_energy != 0 also fills the energy totals (one extra reduction per step). */
abm_status abm_step(abm_world* w, int32_t nsteps, abm_step_stats* stats, int32_t want_energy,
                    void* stream);
/* Capture `nsteps` steps into a CUDA graph once and replay it `reps` times
 * (stats, if given, is device abm_step_stats[nsteps] and is overwritten by each replay). */
abm_status abm_step_graph(abm_world* w, int32_t nsteps, int32_t reps, abm_step_stats* stats,
                          void* stream);
/* abm_step that also reports where the time goes; phase_ms (host float[8],
 * required) receives milliseconds summed over the steps. Kernel engine: CUDA
 * events between the launches, [0] sheep move, [1] sheep eat/select/compact,
 * [2] sheep births, [3] wolf move, [4] wolf eat/select/compact, [5] wolf
 * births. Persistent engine: block 0's global-timer laps between the grid
 * barriers, [0] previous step's wolf ranks + sheep move, [1] previous step's
 * wolf births + sheep eat/select/flags, [2] sheep ranks + wolf move, [3]
 * sheep births, [4] wolf eat/select/flags, [5] the last step's wolf ranks
 * (once per call). Both: [7] whole call by events, [6] = 0.
 * Synchronises `stream`. */
abm_status abm_step_profiled(abm_world* w, int32_t nsteps, abm_step_stats* stats, float* phase_ms,
                             void* stream);
/* Execution engine of abm_step: ABM_ENGINE_PERSISTENT (default) runs all
 * requested steps in one cooperative launch of `ctas_per_sm` CTAs per SM
 * with bounded grid barriers between the phases; ABM_ENGINE_KERNELS runs six
 * kernels per step (and is what abm_step_profiled, energy statistics and
 * abm_step_graph use). Results are identical. */
#define ABM_ENGINE_PERSISTENT 0
#define ABM_ENGINE_KERNELS 1
abm_status abm_world_tune(abm_world* w, int32_t engine, int32_t ctas_per_sm);
/* Failure-detection self-check (no counterpart in the paper): runs the
 * bounded grid barrier of the persistent engine with one arrival more than
 * the grid provides, so its wait runs out after `spin_limit` polls (1..2^24;
 * ~100 ns each). Returns ABM_ERR_DEVICE_TIMEOUT when the timeout was detected
 * and reported -- the expected outcome -- and leaves the context usable.
 * Synchronises `stream`. */
abm_status abm_diag_barrier_timeout(int32_t spin_limit, void* stream);
/* Self-check of the check build's index test (no counterpart in the paper):
 * tests index i against [0, n) on the device, the way the kernels test their
 * indices, without any access. Check build: ABM_ERR_CHECK if i is out of
 * range, else ABM_OK. Other builds: ABM_OK (nothing is tested). Synchronises
 * `stream`. */
abm_status abm_diag_check_index(int64_t i, int64_t n, void* stream);
/* Synchronises `stream`; reports a recorded device error (e.g. a timed-out wait). */
abm_status abm_world_check(abm_world* w, void* stream);

/* Digest of the world's observable state (the checkpoint/digest call of the
 * Section 2 API list): the wrapping 64-bit sum of one hash per live agent
 * (species, slot, cell, energy, id, age), per cell (steps until its grass is
 * edible) and per species counter (live agents, next id, high-water mark).
 * Independent of the capacity and of the engine; a batch model run with the
 * same configuration has the same digest (abm_batch_digest). out: device
 * uint64 (required), written asynchronously on `stream`. */
abm_status abm_digest(abm_world* w, uint64_t* out, void* stream);

/* A species of the world as a Set (Section 2), so that the Set calls --
 * abm_select, abm_select_permutation, abm_remove, abm_add,
 * abm_update_distinct, abm_slab_read / write -- edit the world's agents
 * between steps. The slab has F = 4 fields (0 cell, 1 energy, 2 id, 3 age)
 * over the world's own arrays; its Bernoulli draws use the world's key. The
 * first call for a species allocates the view's scratch (about 12 bytes a
 * slot, kept until abm_destroy); every call copies the world's live count,
 * next id and overflow flag into the view (asynchronously on `stream`). The
 * view belongs to the world: abm_slab_destroy and abm_sort refuse it
 * (ABM_ERR_STATE). Cells must stay in [0, side^2) and ids are the caller's
 * business. After editing, call abm_world_slab_commit before the next step. */
abm_status abm_world_slab(abm_world* w, int32_t species, abm_slab** out, void* stream);
/* Fold a species' edits back into the world: live count recounted from the
 * live flags, next id and overflow taken from the view, the high-water mark
 * raised to the live count, the extent raised to the highest live slot + 1,
 * and the per-cell claim tables emptied (they are rebuilt by the next step,
 * as after abm_load). ABM_ERR_STATE if abm_world_slab was never called for
 * the species. Asynchronous on `stream`. */
abm_status abm_world_slab_commit(abm_world* w, int32_t species, void* stream);

/* State export into device int32 buffers of the slab capacity (agents) or
 * side^2 (grass). which: 0 active, 1 cell, 2 energy, 3 id, 4 age. Grass:
 * 0 grown (0/1), 1 wait = steps until the cell is edible (0 when grown). */
abm_status abm_read_agents(abm_world* w, int32_t species, int32_t which, int32_t* dst, void* stream);
abm_status abm_read_grass(abm_world* w, int32_t which, int32_t* dst, void* stream);
typedef struct abm_world_counters {
  int32_t n_active[2], next_id[2], hw[2], overflow[2], extent[2], step, reserved;
} abm_world_counters;
/* Host copy of the counters (synchronises `stream`). */
abm_status abm_world_counters_get(abm_world* w, abm_world_counters* out, void* stream);

/* Checkpoint: the state as a flat byte image in host memory -- the counters,
 * then per species the live flags and records of slots [0, extent), then the
 * grass. Slots at or past a species' extent hold no agent (the extent is the
 * high-water mark of occupied slots; edits made through abm_world_slab count
 * once abm_world_slab_commit has folded them back), so the image carries only
 * what the state depends on and its size follows the extent, not the capacity.
 * abm_save with buf = NULL returns the size the current state needs in
 * *bytes; with a buffer of *bytes >= that size it writes the image and sets
 * *bytes to its size (ABM_ERR_ARG for a smaller buffer). abm_load restores a
 * world created with the same config from an image of `bytes` >= its size;
 * slots at or past the image's extents come back empty (flag and record
 * zero, as in a world that never used them). abm_image_capacity gives the
 * largest image the world can produce (every slot below the capacity in
 * use), a size that fits any later state. abm_save and abm_load synchronise
 * `stream` (abm_save also to read the counters). */
abm_status abm_save(abm_world* w, void* buf, size_t* bytes, void* stream);
abm_status abm_load(abm_world* w, const void* buf, size_t bytes, void* stream);
abm_status abm_image_capacity(abm_world* w, size_t* bytes);

/* ========================================================================== */
/* Batched predation: many independent models in one persistent launch        */
/* (ABMax vectorises models with vmap over Sets, Section 2, Table 2)          */
/* ========================================================================== */
/*
 * Every model follows the rules of abm_step with its own side, key
 * (seed, model), params, capacities and initial populations. One CTA runs one
 * model at a time (largest models first); per-model slabs sit at offsets in
 * shared device arrays. Limits per model as for abm_create.
 */
typedef struct abm_batch abm_batch;

typedef struct abm_batch_model {
  int32_t side;
  uint32_t seed, model;
  int32_t params[8];
  int32_t cap[2];
  int32_t n0[2];
} abm_batch_model;

typedef struct abm_batch_counters {
  int32_t n_active[2], next_id[2], hw[2], overflow[2], extent[2], step, reserved;
  int64_t agent_steps; /* sum over the steps run of the live agents at step start */
} abm_batch_counters;

/* Sweep of a model's slabs in every phase: the whole capacity (the paper's
 * static shapes, placeholders included) or the extent (highest slot ever
 * used + 1). Results are identical; only the work differs. */
#define ABM_SWEEP_CAPACITY 0
#define ABM_SWEEP_EXTENT 1

/* models: host array of n. Allocates and initialises every model (synchronises `stream`). */
abm_status abm_batch_create(const abm_batch_model* models, int32_t n, void* stream, abm_batch** out);
abm_status abm_batch_destroy(abm_batch* b);
/* Launch shape: CTA size (128..1024), CTAs per SM, and steps per launch
 * (a run of nsteps is split into ceil(nsteps / steps_per_launch) launches,
 * each replayable in a CUDA graph). Results never depend on it. */
abm_status abm_batch_tune(abm_batch* b, int32_t threads, int32_t ctas_per_sm, int32_t steps_per_launch);
/* Launch shape: models run at once by one CTA (1, 2 or 4), each on a group of
 * threads / models_per_cta threads with its own barrier, so that small models
 * need not occupy a whole CTA; the groups take models from the same queue
 * (largest first). Groups must keep at least 128 threads (ABM_ERR_ARG
 * otherwise; abm_batch_tune resets it to 1 when a new CTA size would break
 * that). Results never depend on it. Host only. */
abm_status abm_batch_models_per_cta(abm_batch* b, int32_t models_per_cta);
/* Launch shape: agent slots per thread in each chunk of the per-species
 * sweeps (8, 16 or 32, default 16; 32 only with at most 512 threads per CTA,
 * ABM_ERR_ARG otherwise, and abm_batch_tune resets it to 16 when a larger CTA
 * is chosen): a group of T threads reads the live flags of
 * agents_per_thread * T slots (128-bit loads), lists the live ones and shares
 * them out, chunk by chunk. Results never depend on it. Host only. */
abm_status abm_batch_agents_per_thread(abm_batch* b, int32_t agents_per_thread);
/* Advance every model by nsteps (asynchronous on `stream`). */
abm_status abm_batch_run(abm_batch* b, int32_t nsteps, int32_t sweep, void* stream);
/* Host copy of every model's counters (out: host abm_batch_counters[n]; synchronises `stream`). */
abm_status abm_batch_counters_get(abm_batch* b, abm_batch_counters* out, void* stream);
/* State of model m, as abm_read_agents / abm_read_grass (dst: device int32[cap] / [side^2]). */
abm_status abm_batch_read_agents(abm_batch* b, int32_t m, int32_t species, int32_t which, int32_t* dst,
                                 void* stream);
abm_status abm_batch_read_grass(abm_batch* b, int32_t m, int32_t which, int32_t* dst, void* stream);
/* Device-side list of the models whose births were truncated by a full slab
 * (list: device int32[n], count: device int32). */
abm_status abm_batch_overflowed(abm_batch* b, int32_t* list, int32_t* count, void* stream);
/* Per-model digest (device uint64[n]): an order-independent hash of the
 * live agents (species, slot, cell, energy, id, age), the grass (steps
 * until edible) and the counters. It does not depend on the capacity, so
 * runs of the same models at different capacities compare equal iff their
 * observable states are equal (up to hash collisions). */
abm_status abm_batch_digest(abm_batch* b, uint64_t* out, void* stream);
abm_status abm_batch_check(abm_batch* b, void* stream);
/* Total slots per species and total cells allocated by the batch (its own
 * slabs; a rerun's are not counted). */
abm_status abm_batch_info(abm_batch* b, int64_t* slots_sheep, int64_t* slots_wolf, int64_t* cells);
/* Current capacities of model m (host int32[2]): its own, or the fixed
 * capacities of its rerun. */
abm_status abm_batch_capacity(abm_batch* b, int32_t m, int32_t* cap);

/* Recovery of a learned-capacity batch (Section 4: the maximum number of
 * agents must be known in advance; a predicted capacity can be too small).
 * Every model whose births were ever truncated by its slab (overflow flag,
 * as listed by abm_batch_overflowed) is run again from its initial state, to
 * the step the batch has reached, at the capacities cap_fixed[m] (host
 * int32[n][2]; cap_fixed[m][s] >= n0[s], entries of models that did not
 * overflow are not read beyond that check) with `sweep` and the batch's
 * launch shape, in a second batch that `b` keeps. From then on
 * abm_batch_counters_get, abm_batch_digest, abm_batch_read_agents,
 * abm_batch_read_grass and abm_batch_capacity report the rerun for those
 * models, abm_batch_run advances both, and abm_batch_check checks both;
 * abm_batch_overflowed and abm_batch_info still describe b's own slabs.
 * *out_rerun (host, nullable) = models rerun; *out_unrecovered (host,
 * nullable) = rerun models whose births were truncated again (cap_fixed too
 * small as well; their counters say so). Synchronises `stream` (the overflow
 * flags are read on the host to size the rerun). ABM_ERR_STATE on a second
 * call. */
abm_status abm_batch_rerun_overflowed(abm_batch* b, const int32_t* cap_fixed, int32_t sweep, int32_t* out_rerun,
                                      int32_t* out_unrecovered, void* stream);

/* ========================================================================== */
/* Learned capacity: an FP32 MLP predicting a high quantile of a model's peak */
/* population, which sizes its slabs (no counterpart in the paper; Section 4 */
/* requires the maximum number of agents in advance)                          */
/* ========================================================================== */
/*
 * n_in -> `layers` hidden layers of `hidden` ReLU units -> n_out, row-major
 * FP32. Parameters are one flat device array: for each linear map l,
 * W_l[din][dout] then b_l[dout]. He-uniform initial weights from Philox
 * (purpose 15, key (seed, 0x4D4C50)), zero biases. Inputs and outputs are
 * device float[B][n_in] / [B][n_out]; B <= max_batch.
 */
typedef struct abm_mlp abm_mlp;
abm_status abm_mlp_create(int32_t n_in, int32_t hidden, int32_t layers, int32_t n_out, uint32_t seed,
                          int32_t max_batch, void* stream, abm_mlp** out);
abm_status abm_mlp_destroy(abm_mlp* n);
abm_status abm_mlp_forward(abm_mlp* n, const float* x, int32_t B, float* y, void* stream);
/* Pinball (quantile tau) loss averaged over the B x n_out outputs and its
 * gradient w.r.t. every parameter (readable via abm_mlp_params). Row r of
 * the batch is row (perm_a * (perm_m0 + r) + perm_c) mod perm_rows of x and
 * y when perm_rows > 0 (a cheap shuffle), else row r. loss_out: device
 * float, nullable. */
abm_status abm_mlp_gradients(abm_mlp* n, const float* x, const float* y, int32_t B, float tau,
                             int64_t perm_rows, int64_t perm_a, int64_t perm_c, int64_t perm_m0,
                             float* loss_out, void* stream);
/* abm_mlp_gradients followed by one Adam step (beta 0.9 / 0.999, eps 1e-8). */
abm_status abm_mlp_train_step(abm_mlp* n, const float* x, const float* y, int32_t B, float tau, float lr,
                              int64_t perm_rows, int64_t perm_a, int64_t perm_c, int64_t perm_m0,
                              float* loss_out, void* stream);
/* Device pointers to the flat parameter and gradient arrays, and their length. */
abm_status abm_mlp_params(abm_mlp* n, float** params, float** grads, int64_t* count);
abm_status abm_mlp_reset_adam(abm_mlp* n, void* stream);
/* Copy `count` (= the parameter count) floats between a device buffer and the parameters / gradients. */
abm_status abm_mlp_set_params(abm_mlp* n, const float* src, int64_t count, void* stream);
abm_status abm_mlp_get_params(abm_mlp* n, float* dst, int64_t count, void* stream);
abm_status abm_mlp_get_grads(abm_mlp* n, float* dst, int64_t count, void* stream);
/* Features of models: table = device int32[B][12] (side, n0 sheep, n0 wolves,
 * the 8 params, horizon); x[b] = log1p(side), log1p(n0 sheep), log1p(n0
 * wolves), params[j] / nominal[j] (as unsigned), horizon / 500.
 * nominal: device int32[8]. */
abm_status abm_capacity_features(const int32_t* table, int32_t B, const int32_t* nominal, float* x, void* stream);
/* Capacities from predicted log peaks yhat[B][2]: cap = min(cap_max,
 * roundup(ceil(exp(yhat) * (1 + margin)), round_to)), at least n0 and round_to. */
abm_status abm_capacity_from_prediction(const float* yhat, int32_t B, float margin, int32_t round_to,
                                        const int32_t* cap_max, const int32_t* n0, int32_t* cap, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ABM_H */
