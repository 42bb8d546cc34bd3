/*
 * Seeded input generators shared by the CUDA path and the oracle: a PRNG and the
 * Progressive Edge-Growth (PEG) construction of sparse parity-check matrices.
 *
 * This file holds none of the decoding arithmetic. It only builds the u m x n
 * matrices H_l that the multi-matrix method assumes are given (Section 2 of the
 * paper: "u matrices generated by PEG"), in CSR form.
 *
 * PRNG: splitmix64 (Steele, Lea & Flood, OOPSLA 2014) expands a 64-bit seed into
 * the state of xoshiro256** (Blackman & Vigna, 2018); both written here from their
 * published definitions.
 *
 * PEG (Hu, Eleftheriou & Arnold, IEEE Trans. IT 51(1), 2005): variable nodes are
 * processed in the order given (the caller sorts them by non-decreasing degree).
 * The first edge of a variable goes to a check of minimum current degree. Every
 * later edge goes to a check of minimum current degree among the checks that a
 * breadth-first search from the variable does not reach; if the search reaches
 * every check, the candidates are the checks first reached in its last layer.
 * Ties are broken uniformly at random with the seeded PRNG. An optional depth
 * cap stops the search after `depth_cap` expansions (depth 1 forbids 4-cycles,
 * depth 2 forbids 4- and 6-cycles); a negative cap means unlimited.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } xo256;

static uint64_t splitmix64_next(uint64_t* x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void xo_seed(xo256* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static uint64_t xo_next(xo256* r) {
  uint64_t* s = r->s;
  uint64_t out = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

/* uniform integer in [0, bound) by rejection of the biased tail */
static uint64_t xo_below(xo256* r, uint64_t bound) {
  uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
  for (;;) {
    uint64_t v = xo_next(r);
    if (v < lim) return v % bound;
  }
}

/* exported for tests: n raw 64-bit outputs of xoshiro256** seeded via splitmix64 */
void mbpin_xoshiro_stream(uint64_t seed, int count, uint64_t* out) {
  xo256 r;
  xo_seed(&r, seed);
  for (int i = 0; i < count; ++i) out[i] = xo_next(&r);
}

typedef struct { int32_t* v; int32_t len, cap; } ivec;

static int iv_push(ivec* a, int32_t x) {
  if (a->len == a->cap) {
    int32_t nc = a->cap ? a->cap * 2 : 8;
    int32_t* nv = (int32_t*)realloc(a->v, (size_t)nc * sizeof(int32_t));
    if (!nv) return -1;
    a->v = nv;
    a->cap = nc;
  }
  a->v[a->len++] = x;
  return 0;
}

typedef struct {
  int n, m;
  const int32_t* var_deg;
  int64_t* var_off;     /* n+1 */
  int32_t* var_cnt;     /* n */
  int32_t* var_adj;     /* sum var_deg */
  ivec* chk_adj;        /* m */
  int32_t* chk_deg;     /* m */
  ivec* bucket;         /* checks grouped by current degree */
  int32_t nbucket;
  int32_t* pos_in_bucket;
  int32_t* chk_seen;    /* BFS stamps */
  int32_t* var_seen;
  int32_t gen;
  ivec frontier, next, scratch;
  xo256 rng;
} peg_state;

static int bucket_ensure(peg_state* S, int32_t d) {
  if (d < S->nbucket) return 0;
  int32_t nb = S->nbucket ? S->nbucket : 8;
  while (nb <= d) nb *= 2;
  ivec* b = (ivec*)realloc(S->bucket, (size_t)nb * sizeof(ivec));
  if (!b) return -1;
  memset(b + S->nbucket, 0, (size_t)(nb - S->nbucket) * sizeof(ivec));
  S->bucket = b;
  S->nbucket = nb;
  return 0;
}

static int add_edge(peg_state* S, int32_t v, int32_t c) {
  S->var_adj[S->var_off[v] + S->var_cnt[v]++] = c;
  if (iv_push(&S->chk_adj[c], v)) return -1;
  int32_t d = S->chk_deg[c];
  /* move c from bucket d to bucket d+1 */
  ivec* b = &S->bucket[d];
  int32_t p = S->pos_in_bucket[c];
  int32_t last = b->v[b->len - 1];
  b->v[p] = last;
  S->pos_in_bucket[last] = p;
  b->len--;
  if (bucket_ensure(S, d + 1)) return -1;
  S->pos_in_bucket[c] = S->bucket[d + 1].len;
  if (iv_push(&S->bucket[d + 1], c)) return -1;
  S->chk_deg[c] = d + 1;
  return 0;
}

/* minimum-degree check not stamped with the current generation; -1 if none */
static int32_t pick_unreached(peg_state* S) {
  for (int32_t d = 0; d < S->nbucket; ++d) {
    ivec* b = &S->bucket[d];
    if (b->len == 0) continue;
    for (int t = 0; t < 32; ++t) {
      int32_t c = b->v[xo_below(&S->rng, (uint64_t)b->len)];
      if (S->chk_seen[c] != S->gen) return c;
    }
    S->scratch.len = 0;
    for (int32_t i = 0; i < b->len; ++i)
      if (S->chk_seen[b->v[i]] != S->gen)
        if (iv_push(&S->scratch, b->v[i])) return -2;
    if (S->scratch.len) return S->scratch.v[xo_below(&S->rng, (uint64_t)S->scratch.len)];
  }
  return -1;
}

/* minimum-degree member of a given list, random tie-break */
static int32_t pick_min_of(peg_state* S, const ivec* L) {
  int32_t best = INT32_MAX;
  for (int32_t i = 0; i < L->len; ++i)
    if (S->chk_deg[L->v[i]] < best) best = S->chk_deg[L->v[i]];
  S->scratch.len = 0;
  for (int32_t i = 0; i < L->len; ++i)
    if (S->chk_deg[L->v[i]] == best)
      if (iv_push(&S->scratch, L->v[i])) return -2;
  if (!S->scratch.len) return -1;
  return S->scratch.v[xo_below(&S->rng, (uint64_t)S->scratch.len)];
}

static int32_t choose_check(peg_state* S, int32_t v, int depth_cap) {
  S->gen++;
  S->var_seen[v] = S->gen;
  S->frontier.len = 0;
  int32_t reached = 0;
  for (int32_t k = 0; k < S->var_cnt[v]; ++k) {
    int32_t c = S->var_adj[S->var_off[v] + k];
    if (S->chk_seen[c] != S->gen) {
      S->chk_seen[c] = S->gen;
      reached++;
      if (iv_push(&S->frontier, c)) return -2;
    }
  }
  if (reached == S->m) return -1; /* v already touches every check */
  int depth = 0;
  for (;;) {
    if (S->var_cnt[v] == 0 || (depth_cap >= 0 && depth >= depth_cap)) return pick_unreached(S);
    S->next.len = 0;
    for (int32_t i = 0; i < S->frontier.len; ++i) {
      ivec* cv = &S->chk_adj[S->frontier.v[i]];
      for (int32_t a = 0; a < cv->len; ++a) {
        int32_t w = cv->v[a];
        if (S->var_seen[w] == S->gen) continue;
        S->var_seen[w] = S->gen;
        for (int32_t k = 0; k < S->var_cnt[w]; ++k) {
          int32_t c = S->var_adj[S->var_off[w] + k];
          if (S->chk_seen[c] == S->gen) continue;
          S->chk_seen[c] = S->gen;
          reached++;
          if (iv_push(&S->next, c)) return -2;
        }
      }
    }
    if (S->next.len == 0) return pick_unreached(S); /* search stopped growing */
    if (reached == S->m) return pick_min_of(S, &S->next); /* last layer */
    ivec t = S->frontier;
    S->frontier = S->next;
    S->next = t;
    depth++;
  }
}

static void peg_free(peg_state* S) {
  if (S->chk_adj)
    for (int i = 0; i < S->m; ++i) free(S->chk_adj[i].v);
  if (S->bucket)
    for (int i = 0; i < S->nbucket; ++i) free(S->bucket[i].v);
  free(S->var_off); free(S->var_cnt); free(S->var_adj); free(S->chk_adj); free(S->chk_deg);
  free(S->bucket); free(S->pos_in_bucket); free(S->chk_seen); free(S->var_seen);
  free(S->frontier.v); free(S->next.v); free(S->scratch.v);
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Build one m x n matrix. var_deg[i] is the degree of column i (columns are
 * processed in index order). Writes row_ptr[m+1] and col_idx[sum var_deg], rows
 * with ascending column indices. Returns 0, or -1 (impossible degrees),
 * -2 (out of memory), -3 (bad arguments).
 */
int mbpin_peg(int n, int m, const int32_t* var_deg, int depth_cap, uint64_t seed,
              int32_t* row_ptr, int32_t* col_idx) {
  if (n <= 0 || m <= 0 || !var_deg || !row_ptr || !col_idx) return -3;
  peg_state S;
  memset(&S, 0, sizeof S);
  S.n = n; S.m = m; S.var_deg = var_deg;
  xo_seed(&S.rng, seed);
  int rc = -2;
  S.var_off = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
  S.var_cnt = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  S.chk_adj = (ivec*)calloc((size_t)m, sizeof(ivec));
  S.chk_deg = (int32_t*)calloc((size_t)m, sizeof(int32_t));
  S.pos_in_bucket = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  S.chk_seen = (int32_t*)calloc((size_t)m, sizeof(int32_t));
  S.var_seen = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!S.var_off || !S.var_cnt || !S.chk_adj || !S.chk_deg || !S.pos_in_bucket || !S.chk_seen || !S.var_seen) goto done;
  S.var_off[0] = 0;
  for (int i = 0; i < n; ++i) {
    if (var_deg[i] < 0 || var_deg[i] > m) { rc = -1; goto done; }
    S.var_off[i + 1] = S.var_off[i] + var_deg[i];
  }
  if (S.var_off[n] > INT32_MAX) { rc = -1; goto done; }
  S.var_adj = (int32_t*)malloc((size_t)(S.var_off[n] ? S.var_off[n] : 1) * sizeof(int32_t));
  if (!S.var_adj || bucket_ensure(&S, 0)) goto done;
  for (int c = 0; c < m; ++c) {
    S.pos_in_bucket[c] = c;
    if (iv_push(&S.bucket[0], c)) goto done;
  }
  for (int v = 0; v < n; ++v) {
    for (int k = 0; k < var_deg[v]; ++k) {
      int32_t c = choose_check(&S, v, depth_cap);
      if (c == -2) goto done;
      if (c < 0) { rc = -1; goto done; }
      if (add_edge(&S, v, c)) goto done;
    }
  }
  row_ptr[0] = 0;
  for (int c = 0; c < m; ++c) {
    row_ptr[c + 1] = row_ptr[c] + S.chk_adj[c].len;
    memcpy(col_idx + row_ptr[c], S.chk_adj[c].v, (size_t)S.chk_adj[c].len * sizeof(int32_t));
    qsort(col_idx + row_ptr[c], (size_t)S.chk_adj[c].len, sizeof(int32_t), cmp_i32);
  }
  rc = 0;
done:
  peg_free(&S);
  return rc;
}
