/*
 * CPU oracle for the selective-update hot path of ABMax (arXiv 2508.16508).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, sequential restatement of
 * what the GPU path computes. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it. It shares no code,
 * header or constant table with the CUDA library; every constant here is
 * written out again from its definition.
 *
 * Everything is integer arithmetic; results must agree with the GPU path bit
 * for bit.
 *
 * Parity pins (see tests/): Philox against Triton's interpreter and cuRAND;
 * the distinct-update primitive against literal Rank-Match (Alg. 1) and
 * Sort-Count-Iterate (Alg. 2) and numpy.flatnonzero; resolve against a
 * lexicographic min over brute-force groups; the predation step against an
 * independent list-of-agents simulator on tiny worlds plus invariants (the
 * paper prints no trajectory values, so the predation dynamics are pinned
 * only by those, not by numbers from the paper).
 */
#ifndef ABM_ORACLE_H
#define ABM_ORACLE_H
#include <stdint.h>

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------- */
/* counter = (c0 step, c1 slot, c2 purpose, c3 species), key = (seed, model) */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* out[i] = word `word` of philox((step, slot0+i, purpose, species), (seed, model)) */
void orc_philox_words(uint32_t seed, uint32_t model, uint32_t step, uint32_t purpose,
                      uint32_t species, uint32_t slot0, int64_t n, int word, uint32_t* out);

/* Purposes (the c2 counter word). Species word c3: 0 sheep / slab, 1 wolf, 2 grass. */
enum {
  ORC_P_MOVE = 1, ORC_P_PRIO = 2, ORC_P_REPRO = 3, ORC_P_VICTIM = 4,
  ORC_P_INIT_AGENT = 5, ORC_P_GRASS_INIT = 6, ORC_P_MASK = 7,
  ORC_P_NEWREC0 = 9, ORC_P_NEWREC1 = 10, ORC_P_DELTA0 = 11, ORC_P_DELTA1 = 12,
  ORC_P_RESOURCE = 13, ORC_P_INIT_ACTIVE = 14
};
#define ORC_INIT_STEP 0xFFFFFFFFu

/* ---- primitives (Section 4: select, Rank-Match / Sort-Count-Iterate) ---- */
int64_t orc_flatnonzero(const int32_t* mask, int64_t n, int32_t* out_idx);
/* a[sel_a[i]] <- b[sel_b[i]] for i < r = min(#sel_a, #sel_b); returns r. */
int64_t orc_assign_ranked(int32_t* a, const int32_t* mask_a, int64_t n,
                          const int32_t* b, const int32_t* mask_b, int64_t m);
/* Generic slab = active[n] + fields[F][n] (field-major). */
int64_t orc_remove(int32_t* active, const int32_t* mask, int64_t n);
int64_t orc_add(int32_t* active, int32_t* fields, int64_t n, int F, const int32_t* rec,
                int64_t k, int id_field, int32_t id_base, int32_t* out_slots);
/* op 0 = wrapping add, 1 = overwrite. rec_mask may be NULL (all records used). */
int64_t orc_update_distinct(int32_t* fields, int64_t n, int F, const int32_t* target_mask,
                            const int32_t* rec, const int32_t* rec_mask, int64_t k, int op,
                            int32_t* out_slots);
void orc_resolve(const int32_t* res, const uint32_t* prio, int64_t M, int64_t R,
                 int32_t* winner, uint8_t* is_winner);

/* Selective-update microbenchmark call c: remove, then distinct update of the
 * survivors, then add (the update and the add touch disjoint slots). */
void orc_c1_init(int32_t* active, int32_t* fields, int64_t n, int F, uint32_t seed, uint32_t model);
void orc_c1_records(uint32_t seed, uint32_t model, uint32_t step, uint32_t p0, uint32_t p1,
                    int64_t k, int F, int32_t* out);
void orc_c1_call(int32_t* active, int32_t* fields, int64_t n, int F, uint32_t seed,
                 uint32_t model, uint32_t step, uint32_t T, int64_t k, int64_t out_counts[3]);

/* ---- predation (Section 5.1, Fig. 3) ------------------------------------ */
typedef struct orc_stats {
  int32_t n_start[2];   /* live agents when the step starts */
  int32_t parents[2];   /* agents selected to reproduce */
  int32_t births[2];    /* children placed (r = min(parents, free)) */
  int32_t starved[2];   /* removed with energy < 0 */
  int32_t eaten;        /* sheep removed by wolves */
  int32_t grass_eaten;
  int32_t n_end[2];
  int32_t hw[2];        /* high-water mark of the post-birth count so far */
  int32_t overflow[2];  /* 1 once parents > free slots has happened */
  int32_t pad;
  int64_t energy[2];    /* sum of live energy at the end of the step */
} orc_stats;

/* sort_agents: live agents first ascending by fields[field] (signed, ties in
 * slot order), then the placeholders in slot order; rows move whole. fields
 * is F rows of n; perm[i] = old slot of new slot i. */
void orc_sort(int32_t* active, int32_t* fields, int64_t n, int F, int field, int32_t* perm);

/* limit order books: one matching round of every book, and new orders into
 * the books' free slots (arrays [nbooks][cap]) */
void orc_lob_match(int32_t nbooks, int32_t cap, int32_t* active, const int32_t* side, const int32_t* price,
                   int32_t* qty, const int32_t* time, int64_t* out_volume, int32_t* out_price);
void orc_lob_add(int32_t nbooks, int32_t cap, int32_t* active, int32_t* side, int32_t* price, int32_t* qty,
                 int32_t* time, const int32_t* new_orders, const int32_t* k, int32_t kmax, int32_t* out_added);

typedef struct orc_world orc_world;
orc_world* orc_pred_create(int32_t side, uint32_t seed, uint32_t model, const int32_t params[8],
                           const int32_t cap[2], const int32_t n0[2]);
void orc_pred_free(orc_world* w);
void orc_pred_step(orc_world* w, orc_stats* st);
/* Rule variants of a world, as bits (0 = the default rules):
 * ORC_VARIANT_MANY_WOLVES: the i-th wolf of a cell eats its i-th sheep, both
 *   ordered by their keys (default: at most one wolf eats per cell per step);
 * ORC_VARIANT_GRASS_OFF: sheep neither eat grass nor spend energy moving
 *   (Wilensky's model without grass). */
enum { ORC_VARIANT_ONE_WOLF = 0, ORC_VARIANT_MANY_WOLVES = 1, ORC_VARIANT_GRASS_OFF = 2 };
void orc_pred_set_variant(orc_world* w, int32_t variant);
/* which: 0 active, 1 cell, 2 energy, 3 id, 4 age */
int32_t* orc_pred_agents(orc_world* w, int species, int which);
/* which: 0 grown, 1 countdown */
int32_t* orc_pred_grass(orc_world* w, int which);
/* out: n_active[2], next_id[2], hw[2], overflow[2], step */
void orc_pred_counters(const orc_world* w, int32_t out[9]);
void orc_pred_set_counters(orc_world* w, int species, int32_t n_active, int32_t next_id, int32_t hw,
                           int32_t overflow);

#endif
