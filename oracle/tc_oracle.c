/*
 * CPU oracle for temporal 3-path sampling (Pu et al., "Accurate and Fast
 * Estimation of Temporal Motifs using Path Sampling", ICDM 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA library: no headers, no helpers, no tables.  Everything here is plain,
 * serial and written to be read against the paper:
 *
 *   - time-sorted adjacency lists and per-pair lists   (Sec. III, III-B)
 *   - windowed degrees and path weights w_e             (Def. 6, Claim 1, Alg. 1)
 *   - exact prefix / total W                            (Alg. 1)
 *   - Philox4x32-10 counter RNG (Salmon et al., SC'11) and Lemire's bounded
 *     integer draw (Lemire, ACM TOMACS 2019) as the random source of Alg. 2
 *   - Sample                                            (Alg. 2)
 *   - CheckMotif / ListCount                            (Alg. 3, Alg. 4)
 *   - exhaustive path-sum counter  sum_P CheckMotif(P)  (Claim 2's proof)
 *   - chronological backtracking exact enumerator of M-matches (Def. 2)
 *
 * Conventions shared with the library by specification (not by code):
 *   canonical edge order = out-lists: sort by (src, t, input index)
 *   in-lists             = sort by (dst, t, input index)
 *   pair lists           = sort by (src, dst, t, input index)
 * Windows: "strict" (default) follows the class definition (Def. 5), where the
 * end edge is strictly before/after the middle edge; "closed" follows the
 * closed intervals of Claim 1 / Alg. 1.  Both are unbiased because CheckMotif
 * rejects ties among anchor edges.
 *
 * Status codes: 0 ok, 3 overflow, 6 RNG attempts exhausted, 1 invalid.
 *
 * Threads: serial by default.  or_set_threads(n > 1) runs the per-edge loop
 * of the weights, the per-sample loop of the sampler, the per-middle-edge
 * loop of the path sum and the first-edge loop of the backtracking count on
 * n OpenMP threads.  Every iteration is independent and every sum is an
 * integer, so the results are identical to the serial ones.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define OR_OK 0
#define OR_INVALID 1
#define OR_OVERFLOW 3
#define OR_RNG_EXHAUSTED 6

static int or_threads = 1;

/* Threads of the parallel loops (1 = serial); returns the number in use. */
int or_set_threads(int n) {
#ifdef _OPENMP
  or_threads = n > 1 ? n : 1;
#else
  (void)n;
  or_threads = 1;
#endif
  return or_threads;
}

/* ------------------------------------------------------------------------ */
/* Sorting into the three list orders (Sec. III: lists sorted by timestamp). */

static const int32_t *g_src, *g_dst;
static const int64_t *g_t;

static int cmp_i64(int64_t a, int64_t b) { return (a > b) - (a < b); }

static int cmp_out(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  int c = cmp_i64(g_src[a], g_src[b]);
  if (!c) c = cmp_i64(g_t[a], g_t[b]);
  if (!c) c = cmp_i64(a, b);
  return c;
}
static int cmp_in(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  int c = cmp_i64(g_dst[a], g_dst[b]);
  if (!c) c = cmp_i64(g_t[a], g_t[b]);
  if (!c) c = cmp_i64(a, b);
  return c;
}
static int cmp_pair(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  int c = cmp_i64(g_src[a], g_src[b]);
  if (!c) c = cmp_i64(g_dst[a], g_dst[b]);
  if (!c) c = cmp_i64(g_t[a], g_t[b]);
  if (!c) c = cmp_i64(a, b);
  return c;
}
static int cmp_time(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  int c = cmp_i64(g_t[a], g_t[b]);
  if (!c) c = cmp_i64(a, b);
  return c;
}

/*
 * Build the out-, in- and pair-lists.  All arrays are caller-allocated:
 *   out_perm[m], out_off[n+1], in_perm[m], in_off[n+1], in_eid[m],
 *   pair_perm[m], pair_off[n+1], pair_dst[m], pair_eoff[m+1]; *P_out = #pairs.
 * *_perm map a list position to the input edge index; in_eid maps an in-list
 * position to the canonical (out-list) position of the same edge.  With
 * presorted != 0 the three permutations are taken as given (computed by a
 * library sort with the same keys) and only the rest is built.
 */
int or_build_csr(int64_t n, int64_t m, int presorted, const int32_t *src, const int32_t *dst,
                 const int64_t *t, int64_t *out_perm, int64_t *out_off,
                 int64_t *in_perm, int64_t *in_off, int64_t *in_eid,
                 int64_t *pair_perm, int64_t *pair_off, int32_t *pair_dst,
                 int64_t *pair_eoff, int64_t *P_out) {
  g_src = src; g_dst = dst; g_t = t;
  if (!presorted) {
    for (int64_t i = 0; i < m; i++) out_perm[i] = in_perm[i] = pair_perm[i] = i;
    qsort(out_perm, (size_t)m, sizeof(int64_t), cmp_out);
    qsort(in_perm, (size_t)m, sizeof(int64_t), cmp_in);
    qsort(pair_perm, (size_t)m, sizeof(int64_t), cmp_pair);
  }

  /* offsets by counting */
  for (int64_t v = 0; v <= n; v++) out_off[v] = in_off[v] = 0;
  for (int64_t i = 0; i < m; i++) { out_off[src[i] + 1]++; in_off[dst[i] + 1]++; }
  for (int64_t v = 0; v < n; v++) { out_off[v + 1] += out_off[v]; in_off[v + 1] += in_off[v]; }

  /* canonical position of each input edge, then in_eid */
  int64_t *canon = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
  for (int64_t p = 0; p < m; p++) canon[out_perm[p]] = p;
  for (int64_t p = 0; p < m; p++) in_eid[p] = canon[in_perm[p]];
  free(canon);

  /* unique (src,dst) pairs in pair order */
  int64_t P = 0;
  for (int64_t v = 0; v <= n; v++) pair_off[v] = 0;
  for (int64_t p = 0; p < m; p++) {
    int64_t e = pair_perm[p];
    int fresh = (p == 0) || src[pair_perm[p - 1]] != src[e] || dst[pair_perm[p - 1]] != dst[e];
    if (fresh) {
      pair_dst[P] = dst[e];
      pair_eoff[P] = p;
      pair_off[src[e] + 1]++;
      P++;
    }
  }
  pair_eoff[P] = m;
  for (int64_t v = 0; v < n; v++) pair_off[v + 1] += pair_off[v];
  *P_out = P;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Searching a time-sorted list: the binary searches of Alg. 1 and Alg. 2.   */

/* number of leading positions p in [lo,hi) whose time is < x (lower bound) */
static int64_t first_ge(const int64_t *perm, const int64_t *t, int64_t lo, int64_t hi, int64_t x) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (t[perm[mid]] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
static int64_t first_gt(const int64_t *perm, const int64_t *t, int64_t lo, int64_t hi, int64_t x) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (t[perm[mid]] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

static int64_t sat_add(int64_t a, int64_t d) { return (a > INT64_MAX - d) ? INT64_MAX : a + d; }
static int64_t sat_sub(int64_t a, int64_t d) { return (a < INT64_MIN + d) ? INT64_MIN : a - d; }

/*
 * The graph view the estimator needs (all caller-owned).
 */
typedef struct {
  int64_t n, m;
  const int32_t *src, *dst;
  const int64_t *t;
  const int64_t *out_perm, *out_off, *in_perm, *in_off;
  const int64_t *pair_perm, *pair_off, *pair_eoff;
  const int32_t *pair_dst;
} or_graph;

/*
 * Motif plan, produced by the oracle's Python motif compiler:
 *   plan[0]        r = number of motif edges (3..16); edge i has time rank i
 *   plan[1..16]    motif edge sources (vertex labels 0..3)
 *   plan[17..32]   motif edge destinations
 *   plan[33..35]   anchor edges: e1, middle, e3 (motif edge indices)
 *   plan[36..39]   alpha1, alpha3 (-1 = in-list, +1 = out-list),
 *                  beta1, beta3   (-1 = before the middle edge, +1 = after)
 *   plan[40]       1 = closed windows (Claim 1 literally), 0 = strict
 *   plan[41..44]   motif vertex labels of u', u, v, v'
 *   plan[45]       kind: 0 = 3-path anchor (4-vertex motif); 1 or 2 = wedge
 *                  anchor (3-vertex motif, Sec. "Brief Description of Wedge
 *                  Sampling"): the base is motif edge 0 (the sampled edge,
 *                  stored as the middle) and the second edge shares the
 *                  base's source (1; stored as e1 with alpha1, beta1 = +1,
 *                  third vertex label in slot u') or its destination (2;
 *                  stored as e3 with alpha3, beta3 = +1, label in slot v').
 *                  The unused end has index -1, alpha = beta = 0, label -1.
 */
typedef struct {
  int r;
  int msrc[16], mdst[16];
  int e1, mid, e3;
  int alpha1, alpha3, beta1, beta3;
  int closed;
  int lab[4];
  int kind;
} or_plan;

static void read_plan(const int32_t *p, or_plan *pl) {
  pl->r = p[0];
  for (int i = 0; i < 16; i++) { pl->msrc[i] = p[1 + i]; pl->mdst[i] = p[17 + i]; }
  pl->e1 = p[33]; pl->mid = p[34]; pl->e3 = p[35];
  pl->alpha1 = p[36]; pl->alpha3 = p[37]; pl->beta1 = p[38]; pl->beta3 = p[39];
  pl->closed = p[40];
  for (int i = 0; i < 4; i++) pl->lab[i] = p[41 + i];
  pl->kind = p[45];
}

/*
 * Windowed list of vertex x around time t (Def. 6): positions [*lo, *hi) of
 * x's in-list (alpha = -1) or out-list (alpha = +1) whose time lies in
 *   beta = -1:  [t - delta, t)   strict,   [t - delta, t]  closed
 *   beta = +1:  (t, t + delta]   strict,   [t, t + delta]  closed
 */
static void window_list(const or_graph *g, int alpha, int beta, int closed, int64_t x,
                        int64_t t, int64_t delta, int64_t *lo, int64_t *hi) {
  const int64_t *perm = alpha < 0 ? g->in_perm : g->out_perm;
  const int64_t *off = alpha < 0 ? g->in_off : g->out_off;
  int64_t a = off[x], b = off[x + 1];
  if (beta < 0) {
    *lo = first_ge(perm, g->t, a, b, sat_sub(t, delta));
    *hi = closed ? first_gt(perm, g->t, a, b, t) : first_ge(perm, g->t, a, b, t);
  } else {
    *lo = closed ? first_ge(perm, g->t, a, b, t) : first_gt(perm, g->t, a, b, t);
    *hi = first_gt(perm, g->t, a, b, sat_add(t, delta));
  }
}

/*
 * Wedge anchor: the window of the base edge e's shared vertex in which its
 * second edge lies, (t, t + delta] strict or [t, t + delta] closed, taken
 * from the shared vertex's out-list (alpha = +1) or in-list (-1).  The
 * wedge weight is its size (for the paper's <+,>> wedge, d+_u[t, t+delta]).
 * It is returned as [a, b) for a wedge at the base's source and [c, d) for
 * one at its destination; the unused side is [0, 1).
 */
static void wedge_window(const or_graph *g, const or_plan *pl, int64_t e, int64_t delta,
                         int64_t *a, int64_t *b, int64_t *c, int64_t *d) {
  *a = 0; *b = 1; *c = 0; *d = 1;
  if (pl->kind == 1)
    window_list(g, pl->alpha1, pl->beta1, pl->closed, g->src[e], g->t[e], delta, a, b);
  else
    window_list(g, pl->alpha3, pl->beta3, pl->closed, g->dst[e], g->t[e], delta, c, d);
}

/* The anchor's windows around middle (base) edge e: the two end windows of
 * a 3-path, or a wedge's window and the single dummy position [0, 1). */
static void anchor_windows(const or_graph *g, const or_plan *pl, int64_t e, int64_t delta,
                           int64_t *a, int64_t *b, int64_t *c, int64_t *d) {
  if (pl->kind == 0) {
    window_list(g, pl->alpha1, pl->beta1, pl->closed, g->src[e], g->t[e], delta, a, b);
    window_list(g, pl->alpha3, pl->beta3, pl->closed, g->dst[e], g->t[e], delta, c, d);
  } else {
    wedge_window(g, pl, e, delta, a, b, c, d);
  }
}

/*
 * Path weights (Claim 1, Alg. 1, one entry per edge in canonical order):
 *   w[i] = d^{alpha1}_u[window1(t)] * d^{alpha3}_v[window3(t)]
 * together with the list positions of both windows (used by Sample).
 */
int or_path_weights(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                    const int64_t *t, const int64_t *out_perm, const int64_t *out_off,
                    const int64_t *in_perm, const int64_t *in_off, const int32_t *plan_arr,
                    int64_t delta, uint64_t *w, int64_t *lo1, int64_t *d1, int64_t *lo3,
                    int64_t *d3) {
  or_graph g = {n, m, src, dst, t, out_perm, out_off, in_perm, in_off, 0, 0, 0, 0};
  or_plan pl;
  read_plan(plan_arr, &pl);
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1)
  for (int64_t i = 0; i < m; i++) {
    int64_t e = out_perm[i];
    int64_t a, b, c, d;
    anchor_windows(&g, &pl, e, delta, &a, &b, &c, &d);
    /* a wedge's unused window is [0, 1): w is the size of its one window */
    w[i] = (uint64_t)(b - a) * (uint64_t)(d - c);
    if (lo1) { lo1[i] = a; d1[i] = b - a; lo3[i] = c; d3[i] = d - c; }
  }
  return OR_OK;
}

/* Exact prefix sum over w (Alg. 1's running total W): prefix[0] = 0. */
int or_prefix(int64_t m, const uint64_t *w, uint64_t *prefix) {
  prefix[0] = 0;
  for (int64_t i = 0; i < m; i++) {
    uint64_t s = prefix[i] + w[i];
    if (s < prefix[i]) return OR_OVERFLOW;
    prefix[i + 1] = s;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with the  */
/* published multipliers and Weyl key increments.                            */

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; round++) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Uniform integer in [0, range) for sample id s and draw number d.
 * Attempt a uses the Philox block with counter (s_lo, s_hi, d, a) and key
 * (seed_lo, seed_hi); its words 0 and 1 form x = w0 | w1 << 32.  Following
 * Lemire (2019), x * range is split into high and low 64-bit halves; the draw
 * is accepted when low >= 2^64 mod range, and the result is the high half.
 */
static int bounded_words(uint64_t seed, uint64_t s, uint32_t d, int upper, uint64_t range, uint64_t *r) {
  if (range == 0) return OR_INVALID;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint64_t reject_below = (uint64_t)(-range) % range; /* = 2^64 mod range */
  for (uint32_t a = 0; a < 64; a++) {
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), d, a}, o[4];
    or_philox4x32_10(ctr, key, o);
    uint64_t x = upper ? ((uint64_t)o[2] | ((uint64_t)o[3] << 32)) : ((uint64_t)o[0] | ((uint64_t)o[1] << 32));
    u128 prod = (u128)x * range;
    if ((uint64_t)prod >= reject_below) { *r = (uint64_t)(prod >> 64); return OR_OK; }
  }
  return OR_RNG_EXHAUSTED;
}

/* x from words 0-1 of block (s, d, a) */
int or_bounded(uint64_t seed, uint64_t s, uint32_t d, uint64_t range, uint64_t *r) {
  return bounded_words(seed, s, d, 0, range, r);
}

/* the same draw from words 2-3 of the block: the two end edges of a sample
 * share block d = 1, e1 the lower half, e3 the upper half */
int or_bounded_hi(uint64_t seed, uint64_t s, uint32_t d, uint64_t range, uint64_t *r) {
  return bounded_words(seed, s, d, 1, range, r);
}

/* ------------------------------------------------------------------------ */
/* ListCount (Alg. 4).  The printed listing restarts its inner pointer for    */
/* every i and adds cnt before moving it; the reading used here is the one   */
/* the text and Claim 5 describe: cnt_1[i] = 1 and                            */
/*   cnt_r[i] = sum of cnt_{r-1}[j] over j with t(L_{r-1}[j]) < t(L_r[i]),    */
/* with a pointer that only moves forward (strict order, as Def. 2 needs).   */

uint64_t or_list_count(int l, const int64_t *const *lists, const int64_t *lens, int *ovf) {
  if (l == 0) return 1;
  for (int r = 0; r < l; r++) if (lens[r] == 0) return 0;
  uint64_t *prev = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)lens[0]);
  for (int64_t i = 0; i < lens[0]; i++) prev[i] = 1;
  for (int r = 1; r < l; r++) {
    uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)lens[r]);
    int64_t j = 0;
    uint64_t cursum = 0;
    for (int64_t i = 0; i < lens[r]; i++) {
      while (j < lens[r - 1] && lists[r - 1][j] < lists[r][i]) {
        uint64_t s = cursum + prev[j];
        if (s < cursum) *ovf = 1;
        cursum = s;
        j++;
      }
      cur[i] = cursum;
    }
    free(prev);
    prev = cur;
  }
  uint64_t total = 0;
  for (int64_t i = 0; i < lens[l - 1]; i++) {
    uint64_t s = total + prev[i];
    if (s < total) *ovf = 1;
    total = s;
  }
  free(prev);
  return total;
}

/* ------------------------------------------------------------------------ */
/* CheckMotif (Alg. 3) for one sampled path.                                  */
/* The path is given by the canonical middle edge i2 and the list positions  */
/* p1 (in x's alpha1 list) and p3 (in v's alpha3 list).                       */

static int64_t edge_of_pos(const or_graph *g, int alpha, int64_t p) {
  return alpha < 0 ? g->in_perm[p] : g->out_perm[p];
}

/* pair list of (x, y) restricted to times in (lo_excl, hi] or (lo_excl, hi):
 * positions [*a, *b) of pair_perm */
static void pair_window(const or_graph *g, int64_t x, int64_t y, int64_t lo_excl, int64_t hi,
                        int hi_inclusive, int64_t *a, int64_t *b) {
  *a = *b = 0;
  /* the pairs of x are pair_dst[pair_off[x] .. pair_off[x+1]), sorted by dst */
  int64_t lo = g->pair_off[x], up = g->pair_off[x + 1];
  while (lo < up) {
    int64_t mid = lo + (up - lo) / 2;
    if (g->pair_dst[mid] < y) lo = mid + 1; else up = mid;
  }
  if (lo >= g->pair_off[x + 1] || g->pair_dst[lo] != y) return;
  int64_t s = g->pair_eoff[lo], e = g->pair_eoff[lo + 1];
  *a = first_gt(g->pair_perm, g->t, s, e, lo_excl);
  *b = hi_inclusive ? first_gt(g->pair_perm, g->t, s, e, hi) : first_ge(g->pair_perm, g->t, s, e, hi);
}

static uint64_t check_motif(const or_graph *g, const or_plan *pl, int64_t delta, int64_t i2,
                            int64_t p1, int64_t p3, int *ovf) {
  int64_t e2 = g->out_perm[i2];
  int64_t e1 = edge_of_pos(g, pl->alpha1, p1);
  int64_t e3 = edge_of_pos(g, pl->alpha3, p3);
  int64_t u = g->src[e2], v = g->dst[e2];
  int64_t up = pl->alpha1 < 0 ? g->src[e1] : g->dst[e1];
  int64_t vp = pl->alpha3 < 0 ? g->src[e3] : g->dst[e3];
  /* the 3-path must span four distinct vertices */
  if (up == u || up == v || up == vp || u == v || u == vp || v == vp) return 0;

  /* phi: motif vertex label -> graph vertex */
  int64_t phi[4];
  phi[pl->lab[0]] = up; phi[pl->lab[1]] = u; phi[pl->lab[2]] = v; phi[pl->lab[3]] = vp;

  /* anchor times in rank order must be strictly increasing and within delta */
  int64_t anchor_rank[3] = {pl->e1, pl->mid, pl->e3};
  int64_t anchor_time[3] = {g->t[e1], g->t[e2], g->t[e3]};
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      if (anchor_rank[a] < anchor_rank[b] && !(anchor_time[a] < anchor_time[b])) return 0;
  int64_t tmin = anchor_time[0], tmax = anchor_time[0];
  for (int a = 1; a < 3; a++) {
    if (anchor_time[a] < tmin) tmin = anchor_time[a];
    if (anchor_time[a] > tmax) tmax = anchor_time[a];
  }
  if ((uint64_t)tmax - (uint64_t)tmin > (uint64_t)delta) return 0;

  /* the anchor's ranks sorted: a0 < a1 < a2 (a0 = 0 by the anchor rule) */
  int64_t rk[3] = {pl->e1, pl->mid, pl->e3}, tk[3] = {anchor_time[0], anchor_time[1], anchor_time[2]};
  for (int a = 0; a < 3; a++)
    for (int b = a + 1; b < 3; b++)
      if (rk[b] < rk[a]) {
        int64_t x = rk[a]; rk[a] = rk[b]; rk[b] = x;
        x = tk[a]; tk[a] = tk[b]; tk[b] = x;
      }

  /* gap g holds the non-anchor edges with ranks between rk[g] and rk[g+1]
   * (the last gap: ranks above rk[2], bounded by t(first edge) + delta) */
  uint64_t X = 1;
  for (int gap = 0; gap < 3; gap++) {
    int64_t rlo = rk[gap], rhi = gap < 2 ? rk[gap + 1] : pl->r;
    int64_t tlo = tk[gap];
    int64_t thi = gap < 2 ? tk[gap + 1] : sat_add(tk[0], delta);
    int hi_incl = gap == 2;
    const int64_t *lists[16];
    int64_t lens[16];
    int64_t *buf[16];
    int l = 0;
    for (int64_t f = rlo + 1; f < rhi; f++) {
      int64_t a, b;
      pair_window(g, phi[pl->msrc[f]], phi[pl->mdst[f]], tlo, thi, hi_incl, &a, &b);
      buf[l] = (int64_t *)malloc(sizeof(int64_t) * (size_t)((b - a) ? (b - a) : 1));
      for (int64_t q = a; q < b; q++) buf[l][q - a] = g->t[g->pair_perm[q]];
      lists[l] = buf[l];
      lens[l] = b - a;
      l++;
    }
    uint64_t c = or_list_count(l, lists, lens, ovf);
    for (int q = 0; q < l; q++) free(buf[q]);
    u128 prod = (u128)X * c;
    if (prod >> 64) *ovf = 1;
    X = (uint64_t)prod;
  }
  return X;
}

/*
 * CheckMotif for a sampled wedge of a 3-vertex motif: base edge i2 (motif
 * edge 0) and second edge at list position p of the shared vertex.  The
 * three vertices must be distinct, the second edge strictly later than the
 * base and within delta of it; the remaining motif edges fall in two gaps,
 * ranks between the base and the second edge (times strictly between the
 * two) and ranks after the second edge (times after it, up to t(base) +
 * delta), and X is the product of the gaps' ListCounts.
 */
static uint64_t check_wedge(const or_graph *g, const or_plan *pl, int64_t delta, int64_t i2, int64_t p,
                            int *ovf) {
  int64_t e0 = g->out_perm[i2];
  int at_src = pl->kind == 1;
  int alpha = at_src ? pl->alpha1 : pl->alpha3;
  int64_t e = edge_of_pos(g, alpha, p);
  int64_t u = g->src[e0], v = g->dst[e0];
  int64_t y = alpha < 0 ? g->src[e] : g->dst[e]; /* the end away from the shared vertex */
  if (u == v || y == u || y == v) return 0;
  int64_t phi[4];
  phi[pl->lab[1]] = u;
  phi[pl->lab[2]] = v;
  phi[at_src ? pl->lab[0] : pl->lab[3]] = y;
  int j = at_src ? pl->e1 : pl->e3;
  int64_t t0 = g->t[e0], tj = g->t[e];
  if (!(t0 < tj) || (uint64_t)tj - (uint64_t)t0 > (uint64_t)delta) return 0;
  uint64_t X = 1;
  for (int gap = 0; gap < 2; gap++) {
    int64_t rlo = gap == 0 ? 0 : j, rhi = gap == 0 ? j : pl->r;
    int64_t tlo = gap == 0 ? t0 : tj, thi = gap == 0 ? tj : sat_add(t0, delta);
    const int64_t *lists[16];
    int64_t lens[16];
    int64_t *buf[16];
    int l = 0;
    for (int64_t f = rlo + 1; f < rhi; f++) {
      int64_t a, b;
      pair_window(g, phi[pl->msrc[f]], phi[pl->mdst[f]], tlo, thi, gap == 1, &a, &b);
      buf[l] = (int64_t *)malloc(sizeof(int64_t) * (size_t)((b - a) ? (b - a) : 1));
      for (int64_t q = a; q < b; q++) buf[l][q - a] = g->t[g->pair_perm[q]];
      lists[l] = buf[l];
      lens[l] = b - a;
      l++;
    }
    uint64_t c = or_list_count(l, lists, lens, ovf);
    for (int q = 0; q < l; q++) free(buf[q]);
    u128 prod = (u128)X * c;
    if (prod >> 64) *ovf = 1;
    X = (uint64_t)prod;
  }
  return X;
}

/* CheckMotif of the anchor drawn at middle (base) edge i2 with end-edge list
 * positions p1 and p3 (a wedge uses the one on its side). */
static uint64_t anchor_check(const or_graph *g, const or_plan *pl, int64_t delta, int64_t i2, int64_t p1,
                             int64_t p3, int *ovf) {
  if (pl->kind == 0) return check_motif(g, pl, delta, i2, p1, p3, ovf);
  return check_wedge(g, pl, delta, i2, pl->kind == 1 ? p1 : p3, ovf);
}

/*
 * One sample (Alg. 2, then Alg. 3): sample id s draws the middle edge and the
 * two end edges; *X receives CheckMotif of the path and (i2, p1, p3) its
 * canonical middle edge and end-edge list positions.  Returns a status.
 */
static int sample_one(const or_graph *g, const or_plan *pl, int64_t delta, const uint64_t *prefix,
                      uint64_t W, uint64_t seed, uint64_t s, int64_t *i2_out, int64_t *p1_out,
                      int64_t *p3_out, uint64_t *X, int *ovf) {
  uint64_t r2, r1, r3;
  int st = or_bounded(seed, s, 0, W, &r2);
  if (st) return st;
  /* middle edge: the unique i2 with prefix[i2] <= r2 < prefix[i2+1] */
  int64_t lo = 0, hi = g->m; /* invariant: prefix[lo] <= r2 < prefix[hi] */
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (prefix[mid] <= r2) lo = mid; else hi = mid;
  }
  int64_t i2 = lo, e2 = g->out_perm[i2];
  int64_t a, b, c, d;
  anchor_windows(g, pl, e2, delta, &a, &b, &c, &d);
  /* e1 and e3 from the two halves of block 1; a wedge's unused end has
   * range 1 (r = 0) */
  st = or_bounded(seed, s, 1, (uint64_t)(b - a), &r1);
  if (st) return st;
  st = or_bounded_hi(seed, s, 1, (uint64_t)(d - c), &r3);
  if (st) return st;
  *i2_out = i2;
  *p1_out = a + (int64_t)r1;
  *p3_out = c + (int64_t)r3;
  *X = anchor_check(g, pl, delta, i2, *p1_out, *p3_out, ovf);
  return OR_OK;
}

/*
 * Sample + CheckMotif for sample ids offset .. offset+k-1 (Alg. 2, Alg. 5's
 * loop).  prefix has m+1 entries (prefix[m] = W).  Optional trace[4*k]
 * receives (i2, p1, p3, X) per sample.  sums[0..4] = (sum X, sum X^2 low,
 * sum X^2 high, hits = #(X > 0), k).
 */
int or_sample_run(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t,
                  const int64_t *out_perm, const int64_t *out_off, const int64_t *in_perm,
                  const int64_t *in_off, const int64_t *pair_perm, const int64_t *pair_off,
                  const int32_t *pair_dst, const int64_t *pair_eoff, const int32_t *plan_arr,
                  int64_t delta, const uint64_t *prefix, uint64_t k, uint64_t seed,
                  uint64_t offset, uint64_t *trace, uint64_t *sums) {
  or_graph g = {n, m, src, dst, t, out_perm, out_off, in_perm, in_off,
                pair_perm, pair_off, pair_eoff, pair_dst};
  or_plan pl;
  read_plan(plan_arr, &pl);
  uint64_t W = prefix[m];
  uint64_t sx = 0, hits = 0;
  u128 sx2 = 0;
  int ovf = 0, status = OR_OK;
  if (W == 0) { sums[0] = sums[1] = sums[2] = sums[3] = 0; sums[4] = k; return OR_OK; }
#pragma omp parallel num_threads(or_threads) if (or_threads > 1)
  {
    uint64_t tsx = 0, thits = 0;
    u128 tsx2 = 0;
    int tovf = 0, tst = OR_OK;
#pragma omp for schedule(static)
    for (uint64_t i = 0; i < k; i++) {
      if (tst) continue;
      int64_t i2, p1, p3;
      uint64_t X;
      int st = sample_one(&g, &pl, delta, prefix, W, seed, offset + i, &i2, &p1, &p3, &X, &tovf);
      if (st) { tst = st; continue; }
      if (trace) {
        trace[4 * i + 0] = (uint64_t)i2; trace[4 * i + 1] = (uint64_t)p1;
        trace[4 * i + 2] = (uint64_t)p3; trace[4 * i + 3] = X;
      }
      uint64_t s1 = tsx + X;
      if (s1 < tsx) tovf = 1;
      tsx = s1;
      u128 x2 = (u128)X * X, s2 = tsx2 + x2;
      if (s2 < tsx2) tovf = 1;
      tsx2 = s2;
      thits += X > 0;
    }
#pragma omp critical
    {
      uint64_t s1 = sx + tsx;
      if (s1 < sx) ovf = 1;
      sx = s1;
      u128 s2 = sx2 + tsx2;
      if (s2 < sx2) ovf = 1;
      sx2 = s2;
      hits += thits;
      ovf |= tovf;
      if (tst && !status) status = tst;
    }
  }
  if (status) return status;
  sums[0] = sx; sums[1] = (uint64_t)sx2; sums[2] = (uint64_t)(sx2 >> 64); sums[3] = hits; sums[4] = k;
  return ovf ? OR_OVERFLOW : OR_OK;
}

/*
 * Exhaustive path-sum: sum over every delta-centered 3-path P of the anchor's
 * class of CheckMotif(P).  By the proof of Claim 2 every M-match has exactly
 * one anchor path, so the sum equals the exact count C; the sum of squares
 * gives the exact variance of one sample.  out[0] = sum X, out[1..2] = sum X^2
 * (low, high), out[3] = number of paths (must equal W).
 */
int or_path_sum(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t,
                const int64_t *out_perm, const int64_t *out_off, const int64_t *in_perm,
                const int64_t *in_off, const int64_t *pair_perm, const int64_t *pair_off,
                const int32_t *pair_dst, const int64_t *pair_eoff, const int32_t *plan_arr,
                int64_t delta, uint64_t *out) {
  or_graph g = {n, m, src, dst, t, out_perm, out_off, in_perm, in_off,
                pair_perm, pair_off, pair_eoff, pair_dst};
  or_plan pl;
  read_plan(plan_arr, &pl);
  uint64_t sx = 0, paths = 0;
  u128 sx2 = 0;
  int ovf = 0;
#pragma omp parallel num_threads(or_threads) if (or_threads > 1)
  {
    uint64_t tsx = 0, tpaths = 0;
    u128 tsx2 = 0;
    int tovf = 0;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t i2 = 0; i2 < m; i2++) {
      int64_t e2 = out_perm[i2];
      int64_t a, b, c, d;
      anchor_windows(&g, &pl, e2, delta, &a, &b, &c, &d);
      for (int64_t p1 = a; p1 < b; p1++)
        for (int64_t p3 = c; p3 < d; p3++) {
          uint64_t X = anchor_check(&g, &pl, delta, i2, p1, p3, &tovf);
          tsx += X;
          tsx2 += (u128)X * X;
          tpaths++;
        }
    }
#pragma omp critical
    {
      sx += tsx;
      sx2 += tsx2;
      paths += tpaths;
      ovf |= tovf;
    }
  }
  out[0] = sx; out[1] = (uint64_t)sx2; out[2] = (uint64_t)(sx2 >> 64); out[3] = paths;
  return ovf ? OR_OVERFLOW : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact count by chronological backtracking over the motif's edges in rank  */
/* order (Def. 2: injective phi, strictly increasing times, span <= delta).  */

typedef struct {
  const or_graph *g;
  const int64_t *tperm; /* all edges sorted by (t, index) */
  int r;
  const int *msrc, *mdst;
  int64_t delta;
  int64_t phi[4];
  int mapped[4];
  int ovf;
} bt_state;

static int used_vertex(const bt_state *S, int64_t x) {
  for (int a = 0; a < 4; a++) if (S->mapped[a] && S->phi[a] == x) return 1;
  return 0;
}

static uint64_t bt(bt_state *S, int i, int64_t tfirst, int64_t tprev) {
  if (i == S->r) return 1;
  const or_graph *g = S->g;
  int x = S->msrc[i], y = S->mdst[i];
  int64_t tmax = i == 0 ? INT64_MAX : sat_add(tfirst, S->delta);
  uint64_t total = 0;
  const int64_t *perm;
  int64_t a, b;
  if (S->mapped[x] && S->mapped[y]) {
    pair_window(g, S->phi[x], S->phi[y], tprev, tmax, 1, &a, &b);
    perm = g->pair_perm;
  } else if (S->mapped[x]) {
    perm = g->out_perm;
    a = first_gt(perm, g->t, g->out_off[S->phi[x]], g->out_off[S->phi[x] + 1], tprev);
    b = first_gt(perm, g->t, g->out_off[S->phi[x]], g->out_off[S->phi[x] + 1], tmax);
  } else if (S->mapped[y]) {
    perm = g->in_perm;
    a = first_gt(perm, g->t, g->in_off[S->phi[y]], g->in_off[S->phi[y] + 1], tprev);
    b = first_gt(perm, g->t, g->in_off[S->phi[y]], g->in_off[S->phi[y] + 1], tmax);
  } else {
    perm = S->tperm;
    a = i == 0 ? 0 : first_gt(perm, g->t, 0, g->m, tprev);
    b = i == 0 ? g->m : first_gt(perm, g->t, 0, g->m, tmax);
  }
  for (int64_t p = a; p < b; p++) {
    int64_t e = perm[p];
    int64_t gs = g->src[e], gd = g->dst[e];
    int newx = !S->mapped[x], newy = !S->mapped[y];
    if (!newx && S->phi[x] != gs) continue;
    if (!newy && S->phi[y] != gd) continue;
    if (gs == gd) continue; /* x != y in the motif, phi is 1-1 */
    if (newx && used_vertex(S, gs)) continue;
    if (newy && used_vertex(S, gd)) continue;
    if (newx) { S->mapped[x] = 1; S->phi[x] = gs; }
    if (newy) { S->mapped[y] = 1; S->phi[y] = gd; }
    uint64_t c = bt(S, i + 1, i == 0 ? g->t[e] : tfirst, g->t[e]);
    uint64_t s = total + c;
    if (s < total) S->ovf = 1;
    total = s;
    if (newx) S->mapped[x] = 0;
    if (newy) S->mapped[y] = 0;
  }
  return total;
}

int or_exact_count(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t,
                   const int64_t *out_perm, const int64_t *out_off, const int64_t *in_perm,
                   const int64_t *in_off, const int64_t *pair_perm, const int64_t *pair_off,
                   const int32_t *pair_dst, const int64_t *pair_eoff, int32_t r,
                   const int32_t *msrc, const int32_t *mdst, int64_t delta, uint64_t *count) {
  or_graph g = {n, m, src, dst, t, out_perm, out_off, in_perm, in_off,
                pair_perm, pair_off, pair_eoff, pair_dst};
  int64_t *tperm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
  g_src = src; g_dst = dst; g_t = t;
  for (int64_t i = 0; i < m; i++) tperm[i] = i;
  qsort(tperm, (size_t)m, sizeof(int64_t), cmp_time);
  int ms[16], md[16];
  for (int i = 0; i < r; i++) { ms[i] = msrc[i]; md[i] = mdst[i]; }
  uint64_t total = 0;
  int ovf = 0;
  if (or_threads <= 1) {
    bt_state S;
    memset(&S, 0, sizeof S);
    S.g = &g; S.tperm = tperm; S.r = r; S.msrc = ms; S.mdst = md; S.delta = delta;
    total = m ? bt(&S, 0, 0, INT64_MIN) : 0;
    ovf = S.ovf;
  } else {
    /* the first motif edge's loop of bt() split over threads: iteration p
     * maps motif edge 0 to the p-th edge in time order and counts the
     * completions of that partial match */
#pragma omp parallel num_threads(or_threads)
    {
      bt_state S;
      memset(&S, 0, sizeof S);
      S.g = &g; S.tperm = tperm; S.r = r; S.msrc = ms; S.mdst = md; S.delta = delta;
      uint64_t part = 0;
#pragma omp for schedule(dynamic, 256)
      for (int64_t p = 0; p < m; p++) {
        int64_t e = tperm[p];
        int64_t gs = g.src[e], gd = g.dst[e];
        if (gs == gd) continue;
        S.mapped[ms[0]] = 1; S.phi[ms[0]] = gs;
        S.mapped[md[0]] = 1; S.phi[md[0]] = gd;
        uint64_t c = bt(&S, 1, g.t[e], g.t[e]);
        S.mapped[ms[0]] = 0;
        S.mapped[md[0]] = 0;
        uint64_t s2 = part + c;
        if (s2 < part) S.ovf = 1;
        part = s2;
      }
#pragma omp critical
      {
        uint64_t s2 = total + part;
        if (s2 < total) ovf = 1;
        total = s2;
        ovf |= S.ovf;
      }
    }
  }
  *count = total;
  free(tperm);
  return ovf ? OR_OVERFLOW : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Learned proposal (not in the paper; the estimator stays that of Alg. 5    */
/* with the middle edge drawn proportional to w_e * h_e instead of w_e).     */

/* Edge features, all log1p of counts, per canonical edge (row-major [m][12]):
 *  0 d1 and 1 d3 (the anchor's windows, Claim 1), 2 w = d1 * d3,
 *  3..6 in- and out-degree of u, then of v, over [t - delta, t + delta],
 *  7 multiplicity sigma_{u,v}[t - delta, t + delta] (Def. 3),
 *  8 sigma_{v,u}[t - delta, t + delta],
 *  9 total out-degree of u, 10 total in-degree of v, 11 total in-degree of u.
 * Counts are taken from the plain definitions on the lists. */
int or_edge_features(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t,
                     const int64_t *out_perm, const int64_t *out_off, const int64_t *in_perm,
                     const int64_t *in_off, const int64_t *pair_perm, const int64_t *pair_off,
                     const int32_t *pair_dst, const int64_t *pair_eoff, const int32_t *plan_arr,
                     int64_t delta, double *feat) {
  or_graph g = {n, m, src, dst, t, out_perm, out_off, in_perm, in_off,
                pair_perm, pair_off, pair_eoff, pair_dst};
  or_plan pl;
  read_plan(plan_arr, &pl);
  for (int64_t i = 0; i < m; i++) {
    int64_t e = out_perm[i];
    int64_t u = src[e], v = dst[e], te = t[e];
    int64_t a, b, c, d;
    anchor_windows(&g, &pl, e, delta, &a, &b, &c, &d);
    double *f = feat + 12 * i;
    int64_t lo = sat_sub(te, delta), hi = sat_add(te, delta);
    f[0] = (double)(b - a);
    f[1] = (double)(d - c);
    f[2] = (double)((uint64_t)(b - a) * (uint64_t)(d - c));
    f[3] = (double)(first_gt(in_perm, t, in_off[u], in_off[u + 1], hi) - first_ge(in_perm, t, in_off[u], in_off[u + 1], lo));
    f[4] = (double)(first_gt(out_perm, t, out_off[u], out_off[u + 1], hi) - first_ge(out_perm, t, out_off[u], out_off[u + 1], lo));
    f[5] = (double)(first_gt(in_perm, t, in_off[v], in_off[v + 1], hi) - first_ge(in_perm, t, in_off[v], in_off[v + 1], lo));
    f[6] = (double)(first_gt(out_perm, t, out_off[v], out_off[v + 1], hi) - first_ge(out_perm, t, out_off[v], out_off[v + 1], lo));
    int64_t pa, pb;
    pair_window(&g, u, v, lo == INT64_MIN ? INT64_MIN : lo - 1, hi, 1, &pa, &pb);
    f[7] = (double)(pb - pa);
    pair_window(&g, v, u, lo == INT64_MIN ? INT64_MIN : lo - 1, hi, 1, &pa, &pb);
    f[8] = (double)(pb - pa);
    f[9] = (double)(out_off[u + 1] - out_off[u]);
    f[10] = (double)(in_off[v + 1] - in_off[v]);
    f[11] = (double)(in_off[u + 1] - in_off[u]);
  }
  return OR_OK;
}

/*
 * Sampling with the proposal q_e = w_e * h_e: the middle edge is the unique
 * e with qprefix[e] <= r < qprefix[e+1] for r uniform in [0, Q); e1 and e3
 * uniform in their windows as in Alg. 2.  Per sample Y = X * Q / h_e is
 * unbiased; it is accumulated exactly per value of h:
 *   bins[3*(h - h_lo) + 0] = sum of X, + 1 = sum of X^2 (low), + 2 = (high)
 * for h in [h_lo, h_hi].  trace (optional) as in or_sample_run.
 * sums[0..2] = (hits, checked-free count of samples, k).
 */
int or_sample_run_q(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t,
                    const int64_t *out_perm, const int64_t *out_off, const int64_t *in_perm,
                    const int64_t *in_off, const int64_t *pair_perm, const int64_t *pair_off,
                    const int32_t *pair_dst, const int64_t *pair_eoff, const int32_t *plan_arr,
                    int64_t delta, const uint64_t *qprefix, const uint16_t *h, uint32_t h_lo, uint32_t h_hi,
                    uint64_t k, uint64_t seed, uint64_t offset, uint64_t *trace, uint64_t *bins,
                    uint64_t *sums) {
  or_graph g = {n, m, src, dst, t, out_perm, out_off, in_perm, in_off,
                pair_perm, pair_off, pair_eoff, pair_dst};
  or_plan pl;
  read_plan(plan_arr, &pl);
  uint64_t Q = qprefix[m], hits = 0;
  int ovf = 0;
  for (uint64_t b = 0; b < 3ull * (h_hi - h_lo + 1); b++) bins[b] = 0;
  sums[0] = sums[1] = 0; sums[2] = k;
  if (Q == 0) return OR_OK;
  for (uint64_t i = 0; i < k; i++) {
    uint64_t s = offset + i, r2, r1, r3;
    int st = or_bounded(seed, s, 0, Q, &r2);
    if (st) return st;
    int64_t lo = 0, hi = m; /* qprefix[lo] <= r2 < qprefix[hi] */
    while (hi - lo > 1) {
      int64_t mid = lo + (hi - lo) / 2;
      if (qprefix[mid] <= r2) lo = mid; else hi = mid;
    }
    int64_t i2 = lo, e2 = out_perm[i2];
    int64_t a, b, c, d;
    anchor_windows(&g, &pl, e2, delta, &a, &b, &c, &d);
    /* e1 and e3 from the two halves of block 1; a wedge's unused end has
     * range 1 (r = 0) */
    st = or_bounded(seed, s, 1, (uint64_t)(b - a), &r1);
    if (st) return st;
    st = or_bounded_hi(seed, s, 1, (uint64_t)(d - c), &r3);
    if (st) return st;
    int64_t p1 = a + (int64_t)r1, p3 = c + (int64_t)r3;
    uint64_t X = anchor_check(&g, &pl, delta, i2, p1, p3, &ovf);
    if (trace) {
      trace[4 * i + 0] = (uint64_t)i2; trace[4 * i + 1] = (uint64_t)p1;
      trace[4 * i + 2] = (uint64_t)p3; trace[4 * i + 3] = X;
    }
    uint32_t hv = h[i2];
    if (hv < h_lo || hv > h_hi) return OR_INVALID;
    uint64_t *bin = bins + 3 * (hv - h_lo);
    uint64_t s1 = bin[0] + X;
    if (s1 < bin[0]) ovf = 1;
    bin[0] = s1;
    u128 x2 = ((u128)bin[2] << 64 | bin[1]) + (u128)X * X;
    bin[1] = (uint64_t)x2; bin[2] = (uint64_t)(x2 >> 64);
    hits += X > 0;
  }
  sums[0] = hits;
  return ovf ? OR_OVERFLOW : OR_OK;
}

/* Exhaustive sums for the proposal: out[0..1] = sum over all class paths P
 * of C_P^2 / h_{e(P)} as a fraction num / den is not exact in integers, so
 * the per-h sums are returned instead: acc[3*(h - h_lo) + 0] = sum of C_P,
 * + 1 / + 2 = sum of C_P^2 (low, high), over paths whose middle edge has h. */
int or_path_sum_q(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t,
                  const int64_t *out_perm, const int64_t *out_off, const int64_t *in_perm,
                  const int64_t *in_off, const int64_t *pair_perm, const int64_t *pair_off,
                  const int32_t *pair_dst, const int64_t *pair_eoff, const int32_t *plan_arr,
                  int64_t delta, const uint16_t *h, uint32_t h_lo, uint32_t h_hi, uint64_t *acc) {
  or_graph g = {n, m, src, dst, t, out_perm, out_off, in_perm, in_off,
                pair_perm, pair_off, pair_eoff, pair_dst};
  or_plan pl;
  read_plan(plan_arr, &pl);
  int ovf = 0;
  for (uint64_t b = 0; b < 3ull * (h_hi - h_lo + 1); b++) acc[b] = 0;
  for (int64_t i2 = 0; i2 < m; i2++) {
    int64_t e2 = out_perm[i2];
    int64_t a, b, c, d;
    anchor_windows(&g, &pl, e2, delta, &a, &b, &c, &d);
    if (a == b || c == d) continue;
    uint32_t hv = h[i2];
    if (hv < h_lo || hv > h_hi) return OR_INVALID;
    uint64_t *bin = acc + 3 * (hv - h_lo);
    for (int64_t p1 = a; p1 < b; p1++)
      for (int64_t p3 = c; p3 < d; p3++) {
        uint64_t X = anchor_check(&g, &pl, delta, i2, p1, p3, &ovf);
        bin[0] += X;
        u128 x2 = ((u128)bin[2] << 64 | bin[1]) + (u128)X * X;
        bin[1] = (uint64_t)x2; bin[2] = (uint64_t)(x2 >> 64);
      }
  }
  return ovf ? OR_OVERFLOW : OR_OK;
}
