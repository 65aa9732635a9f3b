/*
 * CPU oracle (test infrastructure only; see oracle.h). Plain sequential C.
 *
 * Every function cites the passage of the ABMax paper (arXiv 2508.16508) it
 * restates. Where the paper is silent, the reading used is written beside the
 * code.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al., "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 products
 * whose halves are xored into the other counter words together with the key;
 * the key is advanced by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)prod1;
    uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)prod0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t draw(uint32_t seed, uint32_t model, uint32_t step, uint32_t slot,
                     uint32_t purpose, uint32_t species, int word) {
  uint32_t ctr[4] = {step, slot, purpose, species};
  uint32_t key[2] = {seed, model};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[word];
}

void orc_philox_words(uint32_t seed, uint32_t model, uint32_t step, uint32_t purpose,
                      uint32_t species, uint32_t slot0, int64_t n, int word, uint32_t* out) {
  for (int64_t i = 0; i < n; i++)
    out[i] = draw(seed, model, step, slot0 + (uint32_t)i, purpose, species, word);
}

/* uniform integer in [0, n): multiply-shift of a 32-bit draw */
static int32_t uniform_below(uint32_t u, int32_t n) {
  return (int32_t)(((uint64_t)u * (uint64_t)(uint32_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* select_agents (Section 2): indices of the selected agents, in ascending
 * order -- the "true first, stable" permutation's front part. */
int64_t orc_flatnonzero(const int32_t* mask, int64_t n, int32_t* out_idx) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++)
    if (mask[i]) out_idx[c++] = (int32_t)i;
  return c;
}

/* Sort-Count-Iterate (Algorithm 2): r = min of the two selection counts;
 * the i-th selected target receives the i-th selected update. Rank-Match
 * (Algorithm 1) computes the same result (reading: ranks match only when
 * both are nonzero). */
int64_t orc_assign_ranked(int32_t* a, const int32_t* mask_a, int64_t n,
                          const int32_t* b, const int32_t* mask_b, int64_t m) {
  int32_t* ia = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* ib = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int64_t na = orc_flatnonzero(mask_a, n, ia);
  int64_t nb = orc_flatnonzero(mask_b, m, ib);
  int64_t r = na < nb ? na : nb;
  for (int64_t i = 0; i < r; i++) a[ia[i]] = b[ib[i]];
  free(ia);
  free(ib);
  return r;
}

/* set_agents_mask (Section 2): independent masked change -- here, removal of
 * the masked live agents (they become placeholders, Section 4). */
int64_t orc_remove(int32_t* active, const int32_t* mask, int64_t n) {
  int64_t removed = 0;
  for (int64_t i = 0; i < n; i++) {
    if (active[i] && mask[i]) {
      active[i] = 0;
      removed++;
    }
  }
  return removed;
}

/* Adding agents with distinct initial states (Section 4 toy task, with the
 * free placeholder slots as targets): record j goes to the j-th free slot in
 * ascending order, j < r = min(k, #free). id_field >= 0 stamps id_base + j. */
int64_t orc_add(int32_t* active, int32_t* fields, int64_t n, int F, const int32_t* rec,
                int64_t k, int id_field, int32_t id_base, int32_t* out_slots) {
  int64_t j = 0;
  for (int64_t i = 0; i < n && j < k; i++) {
    if (active[i]) continue;
    for (int f = 0; f < F; f++) fields[(int64_t)f * n + i] = rec[j * F + f];
    if (id_field >= 0) fields[(int64_t)id_field * n + i] = (int32_t)((uint32_t)id_base + (uint32_t)j);
    active[i] = 1;
    if (out_slots) out_slots[j] = (int32_t)i;
    j++;
  }
  return j;
}

/* Distinct updates to the selected agents (Algorithms 1 and 2): the i-th
 * selected target (ascending slot) gets the i-th selected record. op 0 adds
 * field-wise with 32-bit wrap-around, op 1 overwrites. */
int64_t orc_update_distinct(int32_t* fields, int64_t n, int F, const int32_t* target_mask,
                            const int32_t* rec, const int32_t* rec_mask, int64_t k, int op,
                            int32_t* out_slots) {
  int32_t* targets = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* recs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
  int64_t nt = orc_flatnonzero(target_mask, n, targets);
  int64_t nr = 0;
  for (int64_t j = 0; j < k; j++)
    if (rec_mask == NULL || rec_mask[j]) recs[nr++] = (int32_t)j;
  int64_t r = nt < nr ? nt : nr;
  for (int64_t i = 0; i < r; i++) {
    int64_t slot = targets[i];
    int64_t j = recs[i];
    for (int f = 0; f < F; f++) {
      int32_t* dst = &fields[(int64_t)f * n + slot];
      if (op == 0)
        *dst = (int32_t)((uint32_t)*dst + (uint32_t)rec[j * F + f]);
      else
        *dst = rec[j * F + f];
    }
    if (out_slots) out_slots[i] = (int32_t)slot;
  }
  free(targets);
  free(recs);
  return r;
}

/* Conflict resolution (Section 1's shared-resource case; Section 5.2's
 * per-cell priority): among the claims on one resource, the lexicographically
 * smallest (priority, claim index) wins. Claims with a resource outside
 * [0, R) are not claims. */
void orc_resolve(const int32_t* res, const uint32_t* prio, int64_t M, int64_t R,
                 int32_t* winner, uint8_t* is_winner) {
  for (int64_t r = 0; r < R; r++) winner[r] = -1;
  for (int64_t m = 0; m < M; m++) {
    int64_t r = res[m];
    if (r < 0 || r >= R) continue;
    int32_t w = winner[r];
    if (w < 0 || prio[m] < prio[w] || (prio[m] == prio[w] && m < w)) winner[r] = (int32_t)m;
  }
  for (int64_t m = 0; m < M; m++) {
    int64_t r = res[m];
    is_winner[m] = (r >= 0 && r < R && winner[r] == (int32_t)m) ? 1 : 0;
  }
}

/* ------------------------------------------------------------------------ */
/* Selective-update microbenchmark (a slab of n slots x F int32 fields). */
void orc_c1_records(uint32_t seed, uint32_t model, uint32_t step, uint32_t p0, uint32_t p1,
                    int64_t k, int F, int32_t* out) {
  for (int64_t j = 0; j < k; j++)
    for (int f = 0; f < F; f++) {
      uint32_t purpose = f < 4 ? p0 : p1;
      out[j * F + f] = (int32_t)draw(seed, model, step, (uint32_t)j, purpose, 0, f & 3);
    }
}

/* Initial slab: each slot is live with probability 1/2; every slot's fields
 * hold its own Philox record (live or not). */
void orc_c1_init(int32_t* active, int32_t* fields, int64_t n, int F, uint32_t seed, uint32_t model) {
  for (int64_t i = 0; i < n; i++) {
    active[i] = draw(seed, model, ORC_INIT_STEP, (uint32_t)i, ORC_P_INIT_ACTIVE, 0, 0) < 0x80000000u;
    for (int f = 0; f < F; f++) {
      uint32_t purpose = f < 4 ? ORC_P_NEWREC0 : ORC_P_NEWREC1;
      fields[(int64_t)f * n + i] = (int32_t)draw(seed, model, ORC_INIT_STEP, (uint32_t)i, purpose, 0, f & 3);
    }
  }
}

/* One microbenchmark call at step c with threshold T and k records. Slots 2j
 * and 2j+1 share the MASK draw with counter slot word j: slot 2j decides
 * removal on word 0 and the choice on word 1, slot 2j+1 on words 2 and 3.
 *   1. remove live slots whose removal word is below T;
 *   2. chosen = slots live after 1 whose choice word is below T; the i-th
 *      chosen slot (i < min(k, #chosen)) gets DELTA record i added;
 *   3. NEWREC record j goes to the j-th slot free after 1, j < min(k, #free).
 * Steps 2 and 3 touch disjoint slots. out_counts = removed, added, updated. */
void orc_c1_call(int32_t* active, int32_t* fields, int64_t n, int F, uint32_t seed,
                 uint32_t model, uint32_t step, uint32_t T, int64_t k, int64_t out_counts[3]) {
  int32_t* mask = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  int32_t* rec = (int32_t*)calloc((size_t)(k > 0 ? k : 1) * (size_t)F, sizeof(int32_t));
  for (int64_t i = 0; i < n; i++)
    mask[i] = draw(seed, model, step, (uint32_t)(i >> 1), ORC_P_MASK, 0, 2 * (int)(i & 1)) < T;
  out_counts[0] = orc_remove(active, mask, n);

  for (int64_t i = 0; i < n; i++)
    mask[i] = active[i] && draw(seed, model, step, (uint32_t)(i >> 1), ORC_P_MASK, 0, 2 * (int)(i & 1) + 1) < T;
  orc_c1_records(seed, model, step, ORC_P_DELTA0, ORC_P_DELTA1, k, F, rec);
  out_counts[2] = orc_update_distinct(fields, n, F, mask, rec, NULL, k, 0, NULL);

  orc_c1_records(seed, model, step, ORC_P_NEWREC0, ORC_P_NEWREC1, k, F, rec);
  out_counts[1] = orc_add(active, fields, n, F, rec, k, -1, 0, NULL);
  free(mask);
  free(rec);
}

/* sort_agents (Section 2 API list): the live agents first, ascending by the
 * signed int32 `field` with ties in slot order, then the placeholders in slot
 * order; every row (live flag and all fields) moves whole. fields is F rows
 * of n. perm[i] = the old slot of the row placed in slot i. */
typedef struct {
  int32_t placeholder, key, slot;
} orc_sortkey;

static int cmp_sortkey(const void* a, const void* b) {
  const orc_sortkey* x = (const orc_sortkey*)a;
  const orc_sortkey* y = (const orc_sortkey*)b;
  if (x->placeholder != y->placeholder) return x->placeholder < y->placeholder ? -1 : 1;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->slot < y->slot ? -1 : x->slot > y->slot;
}

void orc_sort(int32_t* active, int32_t* fields, int64_t n, int F, int field, int32_t* perm) {
  orc_sortkey* k = (orc_sortkey*)malloc(sizeof(orc_sortkey) * (size_t)(n > 0 ? n : 1));
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; i++) {
    k[i].placeholder = active[i] ? 0 : 1;
    k[i].key = active[i] ? fields[(int64_t)field * n + i] : 0;
    k[i].slot = (int32_t)i;
  }
  qsort(k, (size_t)n, sizeof(orc_sortkey), cmp_sortkey);
  for (int64_t i = 0; i < n; i++) perm[i] = k[i].slot;
  for (int f = -1; f < F; f++) {
    int32_t* row = f < 0 ? active : fields + (int64_t)f * n;
    for (int64_t i = 0; i < n; i++) tmp[i] = row[perm[i]];
    memcpy(row, tmp, sizeof(int32_t) * (size_t)n);
  }
  free(k);
  free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Limit order books (Section 5.3: noisy traders place limit orders into the
 * vacant slots of an order book; all books are matched in parallel by sorting
 * the buy and sell orders by price and taking cumulative sums of shares). The
 * paper gives no exact rules; the ones restated here are the engine's:
 * a book is a fixed-capacity set of orders (active, side 0 buy / 1 sell,
 * price > 0, qty > 0, time); priority = price (bids descending, asks
 * ascending), then time, then slot. */

typedef struct {
  int32_t price, time, slot;
  int64_t qty;
} orc_order;

static int cmp_bid(const void* a, const void* b) {
  const orc_order* x = (const orc_order*)a;
  const orc_order* y = (const orc_order*)b;
  if (x->price != y->price) return x->price > y->price ? -1 : 1;
  if (x->time != y->time) return x->time < y->time ? -1 : 1;
  return x->slot < y->slot ? -1 : x->slot > y->slot;
}

static int cmp_ask(const void* a, const void* b) {
  const orc_order* x = (const orc_order*)a;
  const orc_order* y = (const orc_order*)b;
  if (x->price != y->price) return x->price < y->price ? -1 : 1;
  if (x->time != y->time) return x->time < y->time ? -1 : 1;
  return x->slot < y->slot ? -1 : x->slot > y->slot;
}

/* One matching round of every book (arrays [nbooks][cap], updated in place).
 * With the bids and asks in priority order and QB_i, QA_j their cumulative
 * quantities, the traded volume V is the largest v such that the bid holding
 * share v (QB_{i-1} < v <= QB_i) is priced at or above the ask holding share v
 * (0 if none): bid prices fall and ask prices rise along the shares, so the
 * first V shares of each side trade. Order k fills clamp(V - Q_{k-1}, 0,
 * qty_k); filled orders leave the book. out_volume[b] = V; out_price[b] = the
 * price of the ask holding share V (-1 if V = 0). */
void orc_lob_match(int32_t nbooks, int32_t cap, int32_t* active, const int32_t* side, const int32_t* price,
                   int32_t* qty, const int32_t* time, int64_t* out_volume, int32_t* out_price) {
  orc_order* bid = (orc_order*)malloc(sizeof(orc_order) * (size_t)(cap > 0 ? cap : 1));
  orc_order* ask = (orc_order*)malloc(sizeof(orc_order) * (size_t)(cap > 0 ? cap : 1));
  for (int32_t b = 0; b < nbooks; b++) {
    const int64_t o = (int64_t)b * cap;
    int32_t nb = 0, na = 0;
    for (int32_t i = 0; i < cap; i++) {
      if (!active[o + i]) continue;
      const orc_order e = {price[o + i], time[o + i], i, qty[o + i]};
      if (side[o + i] == 0)
        bid[nb++] = e;
      else
        ask[na++] = e;
    }
    qsort(bid, (size_t)nb, sizeof(orc_order), cmp_bid);
    qsort(ask, (size_t)na, sizeof(orc_order), cmp_ask);
    /* walk the shares: the two fronts trade while the bid front is priced at
     * or above the ask front */
    int64_t v = 0;
    int32_t i = 0, j = 0, last_ask_price = -1;
    int64_t left_b = nb > 0 ? bid[0].qty : 0, left_a = na > 0 ? ask[0].qty : 0;
    while (i < nb && j < na && bid[i].price >= ask[j].price) {
      const int64_t t = left_b < left_a ? left_b : left_a;
      v += t;
      last_ask_price = ask[j].price;
      left_b -= t;
      left_a -= t;
      if (left_b == 0 && ++i < nb) left_b = bid[i].qty;
      if (left_a == 0 && ++j < na) left_a = ask[j].qty;
    }
    out_volume[b] = v;
    out_price[b] = v > 0 ? last_ask_price : -1;
    /* the first v shares of each side fill */
    for (int s = 0; s < 2; s++) {
      orc_order* q = s == 0 ? bid : ask;
      const int32_t n = s == 0 ? nb : na;
      int64_t before = 0;
      for (int32_t k = 0; k < n; k++) {
        int64_t fill = v - before;
        if (fill < 0) fill = 0;
        if (fill > q[k].qty) fill = q[k].qty;
        before += q[k].qty;
        const int64_t slot = o + q[k].slot;
        qty[slot] = (int32_t)(q[k].qty - fill);
        if (qty[slot] == 0) active[slot] = 0;
      }
    }
  }
  free(bid);
  free(ask);
}

/* Traders' new orders into each book: order j < k[b] of book b (rows of
 * new_orders[b][kmax][4] = side, price, qty, time) goes into the j-th free
 * slot of book b (ascending), j < min(k[b], free) -- the add primitive of
 * Section 4 per book. out_added[b] = orders placed. */
void orc_lob_add(int32_t nbooks, int32_t cap, int32_t* active, int32_t* side, int32_t* price, int32_t* qty,
                 int32_t* time, const int32_t* new_orders, const int32_t* k, int32_t kmax, int32_t* out_added) {
  for (int32_t b = 0; b < nbooks; b++) {
    const int64_t o = (int64_t)b * cap;
    const int32_t kb = k[b] < 0 ? 0 : (k[b] < kmax ? k[b] : kmax); /* [0, kmax] rows */
    int32_t j = 0;
    for (int32_t i = 0; i < cap && j < kb; i++) {
      if (active[o + i]) continue;
      const int32_t* r = new_orders + ((int64_t)b * kmax + j) * 4;
      active[o + i] = 1;
      side[o + i] = r[0];
      price[o + i] = r[1];
      qty[o + i] = r[2];
      time[o + i] = r[3];
      j++;
    }
    out_added[b] = j;
  }
}

/* ------------------------------------------------------------------------ */
/* Predation (Section 5.1 and Fig. 3: grass, sheep and wolves on a periodic
 * 2-D lattice; random moves; sheep eat grass, wolves eat sheep; grass regrows
 * after a fixed delay; asexual reproduction with a given probability, the
 * child on the parent's cell). Numbers the paper does not give are params:
 *   0 sheep gain, 1 wolf gain, 2 sheep reproduction threshold (u32),
 *   3 wolf reproduction threshold (u32), 4 grass regrowth delay,
 *   5 sheep metabolism, 6 wolf metabolism, 7 initial-grass threshold (u32). */
struct orc_world {
  int32_t side, ncells;
  uint32_t seed, model;
  int32_t params[8];
  int32_t cap[2];
  int32_t* agent[2][5]; /* active, cell, energy, id, age */
  int32_t* grown;
  int32_t* countdown;
  uint64_t* best;      /* per-cell minimum claim key */
  uint64_t* victim;    /* per-cell minimum victim key */
  int32_t n_active[2], next_id[2], hw[2], overflow[2];
  uint32_t t;
  int32_t variant;     /* ORC_VARIANT_* bits */
};

enum { A_ACTIVE = 0, A_CELL = 1, A_ENERGY = 2, A_ID = 3, A_AGE = 4 };
#define NO_KEY 0xFFFFFFFFFFFFFFFFull

orc_world* orc_pred_create(int32_t side, uint32_t seed, uint32_t model, const int32_t params[8],
                           const int32_t cap[2], const int32_t n0[2]) {
  if (side <= 0 || (int64_t)side * side > 0x7FFFFFFF) return NULL;
  orc_world* w = (orc_world*)calloc(1, sizeof(orc_world));
  w->side = side;
  w->ncells = side * side;
  w->seed = seed;
  w->model = model;
  memcpy(w->params, params, sizeof(w->params));
  for (int s = 0; s < 2; s++) {
    if (n0[s] < 0 || n0[s] > cap[s]) { orc_pred_free(w); return NULL; }
    w->cap[s] = cap[s];
    for (int a = 0; a < 5; a++)
      w->agent[s][a] = (int32_t*)calloc((size_t)(cap[s] > 0 ? cap[s] : 1), sizeof(int32_t));
  }
  w->grown = (int32_t*)calloc((size_t)w->ncells, sizeof(int32_t));
  w->countdown = (int32_t*)calloc((size_t)w->ncells, sizeof(int32_t));
  w->best = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)w->ncells);
  w->victim = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)w->ncells);

  /* create_agents (Section 2): agent k of species s sits in slot k; cell and
   * energy are uniform draws (cell in [0, L^2), energy in [0, 2 gain)). */
  for (int s = 0; s < 2; s++) {
    int32_t gain = params[s];
    for (int32_t k = 0; k < n0[s]; k++) {
      uint32_t u0 = draw(seed, model, ORC_INIT_STEP, (uint32_t)k, ORC_P_INIT_AGENT, (uint32_t)s, 0);
      uint32_t u1 = draw(seed, model, ORC_INIT_STEP, (uint32_t)k, ORC_P_INIT_AGENT, (uint32_t)s, 1);
      w->agent[s][A_ACTIVE][k] = 1;
      w->agent[s][A_CELL][k] = uniform_below(u0, w->ncells);
      w->agent[s][A_ENERGY][k] = uniform_below(u1, 2 * gain);
      w->agent[s][A_ID][k] = k;
      w->agent[s][A_AGE][k] = 0;
    }
    w->n_active[s] = n0[s];
    w->next_id[s] = n0[s];
    w->hw[s] = n0[s];
  }
  /* grass: grown with the initial-grass probability, countdown uniform in
   * [0, regrowth) */
  for (int32_t c = 0; c < w->ncells; c++) {
    uint32_t u0 = draw(seed, model, ORC_INIT_STEP, (uint32_t)c, ORC_P_GRASS_INIT, 2, 0);
    uint32_t u1 = draw(seed, model, ORC_INIT_STEP, (uint32_t)c, ORC_P_GRASS_INIT, 2, 1);
    w->grown[c] = u0 < (uint32_t)params[7];
    w->countdown[c] = uniform_below(u1, params[4]);
  }
  w->t = 0;
  return w;
}

void orc_pred_free(orc_world* w) {
  if (!w) return;
  for (int s = 0; s < 2; s++)
    for (int a = 0; a < 5; a++) free(w->agent[s][a]);
  free(w->grown);
  free(w->countdown);
  free(w->best);
  free(w->victim);
  free(w);
}

int32_t* orc_pred_agents(orc_world* w, int species, int which) { return w->agent[species][which]; }

/* Counters of a species whose arrays were edited between steps with the Set
 * operations of Section 2 (select, remove, add, distinct update). */
void orc_pred_set_counters(orc_world* w, int species, int32_t n_active, int32_t next_id, int32_t hw,
                           int32_t overflow) {
  w->n_active[species] = n_active;
  w->next_id[species] = next_id;
  w->hw[species] = hw;
  w->overflow[species] = overflow;
}
int32_t* orc_pred_grass(orc_world* w, int which) { return which == 0 ? w->grown : w->countdown; }
void orc_pred_counters(const orc_world* w, int32_t out[9]) {
  for (int s = 0; s < 2; s++) {
    out[0 + s] = w->n_active[s];
    out[2 + s] = w->next_id[s];
    out[4 + s] = w->hw[s];
    out[6 + s] = w->overflow[s];
  }
  out[8] = (int32_t)w->t;
}

/* Neighbour offsets of the 8-neighbourhood, indexed by the top three bits of
 * the MOVE draw. */
static const int DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

/* step_agents (Section 2): random 8-neighbour move on the periodic lattice,
 * metabolism, ageing -- for every live agent of the species. */
static void move_species(orc_world* w, int s) {
  int32_t L = w->side;
  /* without grass (variant), sheep neither eat nor spend energy */
  int32_t metab = (s == 0 && (w->variant & ORC_VARIANT_GRASS_OFF)) ? 0 : w->params[5 + s];
  for (int32_t i = 0; i < w->cap[s]; i++) {
    if (!w->agent[s][A_ACTIVE][i]) continue;
    uint32_t u = draw(w->seed, w->model, w->t, (uint32_t)i, ORC_P_MOVE, (uint32_t)s, 0);
    int d = (int)(u >> 29);
    int32_t cell = w->agent[s][A_CELL][i];
    int32_t x = cell % L, y = cell / L;
    x = (x + DX[d] + L) % L;
    y = (y + DY[d] + L) % L;
    w->agent[s][A_CELL][i] = y * L + x;
    w->agent[s][A_ENERGY][i] -= metab;
    w->agent[s][A_AGE][i] += 1;
  }
}

static uint64_t make_key(uint32_t prio, int32_t slot) {
  return ((uint64_t)prio << 32) | (uint32_t)slot;
}

/* Sheep eat grass: the live sheep on a grown cell claim it; the smallest
 * (PRIO draw, slot) key wins (reading: one grass per cell per step). */
static void sheep_eat(orc_world* w, orc_stats* st) {
  for (int32_t c = 0; c < w->ncells; c++) w->best[c] = NO_KEY;
  for (int32_t i = 0; i < w->cap[0]; i++) {
    if (!w->agent[0][A_ACTIVE][i]) continue;
    int32_t c = w->agent[0][A_CELL][i];
    if (!w->grown[c]) continue;
    uint64_t key = make_key(draw(w->seed, w->model, w->t, (uint32_t)i, ORC_P_PRIO, 0, 0), i);
    if (key < w->best[c]) w->best[c] = key;
  }
  for (int32_t c = 0; c < w->ncells; c++) {
    if (w->best[c] == NO_KEY) continue;
    int32_t i = (int32_t)(uint32_t)w->best[c];
    w->agent[0][A_ENERGY][i] += w->params[0];
    w->grown[c] = 0;
    w->countdown[c] = w->params[4];
    st->grass_eaten++;
  }
}

/* Reproduction = select + compact + distinct update + add (Section 4's
 * predation example): parents are live agents with energy >= 0 whose REPRO
 * draw is below the threshold, in ascending slot order; the i-th parent
 * (i < r = min(#parents, #free)) places a child in the i-th free slot. The
 * child takes floor(e/2) of the parent's energy e, the parent keeps the rest;
 * the child sits on the parent's cell with age 0 and id next_id + i. */
static void reproduce(orc_world* w, int s, orc_stats* st) {
  int32_t cap = w->cap[s];
  int32_t* parents = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
  int32_t* freeslots = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
  int32_t np = 0, nf = 0;
  for (int32_t i = 0; i < cap; i++) {
    if (w->agent[s][A_ACTIVE][i]) {
      if (w->agent[s][A_ENERGY][i] >= 0 &&
          draw(w->seed, w->model, w->t, (uint32_t)i, ORC_P_REPRO, (uint32_t)s, 0) < (uint32_t)w->params[2 + s])
        parents[np++] = i;
    } else {
      freeslots[nf++] = i;
    }
  }
  int32_t r = np < nf ? np : nf;
  if (np > nf) w->overflow[s] = 1;
  for (int32_t j = 0; j < r; j++) {
    int32_t p = parents[j], c = freeslots[j];
    int32_t e = w->agent[s][A_ENERGY][p];
    int32_t half = e >> 1;
    w->agent[s][A_ENERGY][p] = e - half;
    w->agent[s][A_ACTIVE][c] = 1;
    w->agent[s][A_CELL][c] = w->agent[s][A_CELL][p];
    w->agent[s][A_ENERGY][c] = half;
    w->agent[s][A_ID][c] = w->next_id[s] + j;
    w->agent[s][A_AGE][c] = 0;
  }
  w->next_id[s] += r;
  w->n_active[s] += r;
  if (w->n_active[s] > w->hw[s]) w->hw[s] = w->n_active[s];
  st->parents[s] = np;
  st->births[s] = r;
  free(parents);
  free(freeslots);
}

/* Death: live agents with negative energy become placeholders. */
static void die(orc_world* w, int s, orc_stats* st) {
  for (int32_t i = 0; i < w->cap[s]; i++) {
    if (w->agent[s][A_ACTIVE][i] && w->agent[s][A_ENERGY][i] < 0) {
      w->agent[s][A_ACTIVE][i] = 0;
      w->n_active[s]--;
      st->starved[s]++;
    }
  }
}

/* Wolves eat sheep: on every cell, the live sheep with the smallest (VICTIM
 * draw, slot) key is that cell's victim; the live wolves on cells with a
 * victim claim it, and the smallest (PRIO draw, slot) wolf wins (reading: at
 * most one wolf eats per cell per step). The winner gains energy, the victim
 * is removed. */
static void wolves_eat(orc_world* w, orc_stats* st) {
  for (int32_t c = 0; c < w->ncells; c++) {
    w->victim[c] = NO_KEY;
    w->best[c] = NO_KEY;
  }
  for (int32_t i = 0; i < w->cap[0]; i++) {
    if (!w->agent[0][A_ACTIVE][i]) continue;
    int32_t c = w->agent[0][A_CELL][i];
    uint64_t key = make_key(draw(w->seed, w->model, w->t, (uint32_t)i, ORC_P_VICTIM, 0, 0), i);
    if (key < w->victim[c]) w->victim[c] = key;
  }
  for (int32_t i = 0; i < w->cap[1]; i++) {
    if (!w->agent[1][A_ACTIVE][i]) continue;
    int32_t c = w->agent[1][A_CELL][i];
    if (w->victim[c] == NO_KEY) continue;
    uint64_t key = make_key(draw(w->seed, w->model, w->t, (uint32_t)i, ORC_P_PRIO, 1, 0), i);
    if (key < w->best[c]) w->best[c] = key;
  }
  for (int32_t c = 0; c < w->ncells; c++) {
    if (w->best[c] == NO_KEY) continue;
    int32_t wolf = (int32_t)(uint32_t)w->best[c];
    int32_t sheep = (int32_t)(uint32_t)w->victim[c];
    w->agent[1][A_ENERGY][wolf] += w->params[1];
    w->agent[0][A_ACTIVE][sheep] = 0;
    w->n_active[0]--;
    st->eaten++;
  }
}

/* (key, slot) pairs of one cell, ascending by key (keys are unique: the slot
 * is in the low half). */
typedef struct {
  uint64_t key;
  int32_t slot;
} orc_keyed;

static int cmp_keyed(const void* a, const void* b) {
  const uint64_t x = ((const orc_keyed*)a)->key, y = ((const orc_keyed*)b)->key;
  return x < y ? -1 : x > y;
}

/* Variant: several wolves per cell (NetLogo lets every wolf eat). On every
 * cell, order the live sheep by (VICTIM draw, slot) and the live wolves by
 * (PRIO draw, slot); the i-th wolf eats the i-th sheep for i < min(#sheep,
 * #wolves) -- Algorithm 1's rank matching applied inside each cell. Each
 * eating wolf gains energy; each eaten sheep is removed. */
static void wolves_eat_many(orc_world* w, orc_stats* st) {
  const int32_t n = w->ncells;
  int32_t* start[2];
  orc_keyed* items[2];
  for (int s = 0; s < 2; s++) {
    /* bucket the live agents by cell (counting sort), in slot order */
    start[s] = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < w->cap[s]; i++)
      if (w->agent[s][A_ACTIVE][i]) start[s][w->agent[s][A_CELL][i] + 1]++;
    for (int32_t c = 0; c < n; c++) start[s][c + 1] += start[s][c];
    items[s] = (orc_keyed*)malloc(sizeof(orc_keyed) * (size_t)(start[s][n] > 0 ? start[s][n] : 1));
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    memcpy(fill, start[s], sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < w->cap[s]; i++) {
      if (!w->agent[s][A_ACTIVE][i]) continue;
      const uint32_t purpose = s == 0 ? ORC_P_VICTIM : ORC_P_PRIO;
      const orc_keyed e = {make_key(draw(w->seed, w->model, w->t, (uint32_t)i, purpose, (uint32_t)s, 0), i), i};
      items[s][fill[w->agent[s][A_CELL][i]]++] = e;
    }
    free(fill);
  }
  for (int32_t c = 0; c < n; c++) {
    const int32_t ns = start[0][c + 1] - start[0][c], nw = start[1][c + 1] - start[1][c];
    if (ns == 0 || nw == 0) continue;
    orc_keyed* sh = items[0] + start[0][c];
    orc_keyed* wo = items[1] + start[1][c];
    qsort(sh, (size_t)ns, sizeof(orc_keyed), cmp_keyed);
    qsort(wo, (size_t)nw, sizeof(orc_keyed), cmp_keyed);
    for (int32_t i = 0; i < ns && i < nw; i++) {
      w->agent[1][A_ENERGY][wo[i].slot] += w->params[1];
      w->agent[0][A_ACTIVE][sh[i].slot] = 0;
      w->n_active[0]--;
      st->eaten++;
    }
  }
  for (int s = 0; s < 2; s++) {
    free(start[s]);
    free(items[s]);
  }
}

void orc_pred_set_variant(orc_world* w, int32_t variant) { w->variant = variant; }

/* Grass regrowth after a fixed delay: a cell eaten at step t is grown again
 * from step t + delay on. */
static void grass(orc_world* w) {
  for (int32_t c = 0; c < w->ncells; c++) {
    if (w->grown[c]) continue;
    w->countdown[c] -= 1;
    if (w->countdown[c] <= 0) w->grown[c] = 1;
  }
}

/* One step of Sim.step (Section 3), species order of Wilensky's model:
 * sheep move, eat, reproduce, die; wolves move, eat, reproduce, die; grass. */
void orc_pred_step(orc_world* w, orc_stats* st) {
  memset(st, 0, sizeof(*st));
  st->n_start[0] = w->n_active[0];
  st->n_start[1] = w->n_active[1];
  move_species(w, 0);
  if (!(w->variant & ORC_VARIANT_GRASS_OFF)) sheep_eat(w, st);
  reproduce(w, 0, st);
  die(w, 0, st);
  move_species(w, 1);
  if (w->variant & ORC_VARIANT_MANY_WOLVES)
    wolves_eat_many(w, st);
  else
    wolves_eat(w, st);
  reproduce(w, 1, st);
  die(w, 1, st);
  grass(w);
  w->t++;
  for (int s = 0; s < 2; s++) {
    st->n_end[s] = w->n_active[s];
    st->hw[s] = w->hw[s];
    st->overflow[s] = w->overflow[s];
    int64_t e = 0;
    for (int32_t i = 0; i < w->cap[s]; i++)
      if (w->agent[s][A_ACTIVE][i]) e += w->agent[s][A_ENERGY][i];
    st->energy[s] = e;
  }
}
