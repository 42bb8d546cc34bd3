/*
 * FP64 CPU oracle for multi-matrix belief-propagation reconciliation (MBP).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load this library. It shares no
 * code, header, table or helper with the CUDA library, and it is written for a
 * reader who checks it against the paper by eye, not for speed.
 *
 * What it computes (arXiv 2001.07979):
 *  - eq. (1), Section 2: Alice's syndromes z^l = H_l x (mod 2), l = 1..u.
 *  - eq. (5), Section 3B: Bob's priors from his bit y_i and the QBER e, and the
 *    channel LLR L_P,i = ln(P_i^0 / P_i^1) named in Section 2.
 *  - Algorithm 1, Section 3A, with flooding over all u matrices:
 *      initialise V2C = L_P (C2V = 0); then per iteration the check-node update
 *      of eq. (6) for every check of every H_l, the variable-node update, the
 *      soft decision of eq. (2) (sum over all u matrices), the hard decision and
 *      the stopping rule "z^l = H_l y for every l" of Section 2.
 *
 * Readings of the paper used here (the paper is silent or garbled on these):
 *  - eq. (5) as printed gives P^1 = -(y - e) < 0 for y = 1; it is read as
 *    P^1 = |y - e|, P^0 = 1 - |y - e|, so L_P = (1 - 2y) ln((1 - e)/e).
 *  - LLR sign: positive means bit 0 (forced by the (-1)^{z_j} factor of eq. 6).
 *  - The u matrices interact through the shared posterior of eq. (2): the
 *    variable-to-check message to check j of H_l is L_P,i plus every incoming
 *    check-to-variable message of every matrix except the one from (l, j)
 *    itself. All checks of an iteration use the previous iteration's messages.
 *  - Messages are clipped to [-L_max, L_max] (V2C before the check update, C2V
 *    after it); the empty product of a degree-1 check gives +inf, clipped.
 *  - A check's extrinsic combination excludes its own edge by prefix/suffix
 *    combination, never by division.
 *  - Hard decision: bit 1 iff L_V < 0 (a tie gives 0).
 *  - Variants (orc_decode_ex): the min-sum check rule and the matrix-by-matrix
 *    schedule of Algorithm 1's loop nesting, for comparison with the flooding
 *    sum-product decoder the paper's text describes.
 *  - The syndrome is tested before the first iteration (iters = 0 on success);
 *    iters counts full check+variable iterations; on failure the result is the
 *    last iteration's hard decision with iters = max_iter.
 *
 * Layouts (shared with the library boundary, not with its code): bits are
 * packed LSB first in uint32 words, bit i of a frame in word i >> 5 at i & 31.
 * Matrices arrive concatenated: m[l] rows each, row_ptr blocks of m[l] + 1
 * entries, col_idx blocks of nnz_l entries. Syndromes are [u][F][ceil(m_l/32)].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int bit_of(const uint32_t* w, int64_t i) { return (int)((w[i >> 5] >> (i & 31)) & 1u); }
static void set_bit(uint32_t* w, int64_t i, int b) {
  if (b) w[i >> 5] |= 1u << (i & 31);
  else w[i >> 5] &= ~(1u << (i & 31));
}
static int64_t nwords(int64_t nbits) { return (nbits + 31) / 32; }

/* ------------------------------------------------------------------ code */

typedef struct {
  int u, n;
  int32_t m_tot;
  int64_t e_tot;
  int32_t* m;            /* [u] */
  int32_t* row_first;    /* [u+1] first stacked row of each matrix */
  int64_t* row_ptr;      /* [m_tot+1] stacked rows */
  int32_t* row_mat;      /* [m_tot] matrix of each stacked row */
  int32_t* row_local;    /* [m_tot] row index inside its matrix */
  int32_t* edge_col;     /* [e_tot] */
  int64_t* col_ptr;      /* [n+1] */
  int64_t* col_edge;     /* [e_tot] edges of each column in stacked-row order */
} orc_code;

static void code_free(orc_code* C) {
  free(C->m); free(C->row_first); free(C->row_ptr); free(C->row_mat); free(C->row_local);
  free(C->edge_col); free(C->col_ptr); free(C->col_edge);
  memset(C, 0, sizeof *C);
}

static int code_build(orc_code* C, int u, int n, const int32_t* m, const int32_t* row_ptr_cat,
                      const int32_t* col_idx_cat) {
  memset(C, 0, sizeof *C);
  if (u <= 0 || n <= 0) return -1;
  C->u = u;
  C->n = n;
  C->m = (int32_t*)malloc(sizeof(int32_t) * u);
  C->row_first = (int32_t*)malloc(sizeof(int32_t) * (u + 1));
  if (!C->m || !C->row_first) return -2;
  C->row_first[0] = 0;
  for (int l = 0; l < u; ++l) {
    if (m[l] < 0) return -1;
    C->m[l] = m[l];
    C->row_first[l + 1] = C->row_first[l] + m[l];
  }
  C->m_tot = C->row_first[u];
  /* total edges */
  int64_t etot = 0, rp_off = 0;
  for (int l = 0; l < u; ++l) {
    etot += row_ptr_cat[rp_off + m[l]] - row_ptr_cat[rp_off];
    rp_off += m[l] + 1;
  }
  C->e_tot = etot;
  C->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (C->m_tot + 1));
  C->row_mat = (int32_t*)malloc(sizeof(int32_t) * (C->m_tot > 0 ? C->m_tot : 1));
  C->row_local = (int32_t*)malloc(sizeof(int32_t) * (C->m_tot > 0 ? C->m_tot : 1));
  C->edge_col = (int32_t*)malloc(sizeof(int32_t) * (etot > 0 ? etot : 1));
  C->col_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  C->col_edge = (int64_t*)malloc(sizeof(int64_t) * (etot > 0 ? etot : 1));
  if (!C->row_ptr || !C->row_mat || !C->row_local || !C->edge_col || !C->col_ptr || !C->col_edge) return -2;
  int64_t e = 0, ci_off = 0;
  rp_off = 0;
  C->row_ptr[0] = 0;
  for (int l = 0; l < u; ++l) {
    const int32_t* rp = row_ptr_cat + rp_off;
    const int32_t* ci = col_idx_cat + ci_off;
    for (int32_t j = 0; j < m[l]; ++j) {
      int32_t r = C->row_first[l] + j;
      C->row_mat[r] = l;
      C->row_local[r] = j;
      for (int32_t k = rp[j]; k < rp[j + 1]; ++k) {
        int32_t col = ci[k - rp[0]];
        if (col < 0 || col >= n) return -1;
        C->edge_col[e++] = col;
      }
      C->row_ptr[r + 1] = e;
    }
    ci_off += rp[m[l]] - rp[0];
    rp_off += m[l] + 1;
  }
  /* column lists: edges visited in stacked-row order, so each list is sorted by (l, j) */
  for (int64_t k = 0; k < etot; ++k) C->col_ptr[C->edge_col[k] + 1]++;
  for (int i = 0; i < n; ++i) C->col_ptr[i + 1] += C->col_ptr[i];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * n);
  if (!fill) return -2;
  memcpy(fill, C->col_ptr, sizeof(int64_t) * n);
  for (int64_t k = 0; k < etot; ++k) C->col_edge[fill[C->edge_col[k]]++] = k;
  free(fill);
  return 0;
}

/* ------------------------------------------------------------ eq. (1) */

/* z^l_j = sum over the columns i of row j of H_l of x_i, mod 2 (eq. 1) */
static int syndrome_bit(const orc_code* C, int32_t r, const uint32_t* x) {
  int p = 0;
  for (int64_t k = C->row_ptr[r]; k < C->row_ptr[r + 1]; ++k) p ^= bit_of(x, C->edge_col[k]);
  return p;
}

static int64_t z_offset(const orc_code* C, int F, int l, int f) {
  int64_t off = 0;
  for (int q = 0; q < l; ++q) off += (int64_t)F * nwords(C->m[q]);
  return off + (int64_t)f * nwords(C->m[l]);
}

int orc_syndrome(int u, int n, const int32_t* m, const int32_t* row_ptr_cat, const int32_t* col_idx_cat,
                 int F, const uint32_t* x_bits, uint32_t* z_bits) {
  orc_code C;
  int rc = code_build(&C, u, n, m, row_ptr_cat, col_idx_cat);
  if (rc) { code_free(&C); return rc; }
  int64_t wn = nwords(n);
  for (int f = 0; f < F; ++f) {
    const uint32_t* x = x_bits + (int64_t)f * wn;
    for (int32_t r = 0; r < C.m_tot; ++r) {
      int l = C.row_mat[r];
      uint32_t* z = z_bits + z_offset(&C, F, l, f);
      set_bit(z, C.row_local[r], syndrome_bit(&C, r, x));
    }
  }
  code_free(&C);
  return 0;
}

/* ------------------------------------------------------------ eq. (5) */

/* P_i^1 = |y_i - e|, P_i^0 = 1 - |y_i - e| (eq. 5, sign repaired); L_P = ln(P^0 / P^1) */
void orc_bsc_llr(int n, const uint32_t* y_bits, double e, double* L_P) {
  for (int i = 0; i < n; ++i) {
    double y = (double)bit_of(y_bits, i);
    double p1 = fabs(y - e);
    double p0 = 1.0 - fabs(y - e);
    L_P[i] = log(p0 / p1);
  }
}

/* ------------------------------------------------------------ eq. (6) */

static double sgn(double a) { return a < 0 ? -1.0 : 1.0; }

/*
 * a [+] b = 2 atanh(tanh(a/2) tanh(b/2)), evaluated in the Jacobian-logarithm
 * form sgn(a) sgn(b) min(|a|,|b|) + log1p(e^{-|a+b|}) - log1p(e^{-|a-b|}),
 * which stays accurate where tanh saturates.
 */
double orc_boxplus(double a, double b) {
  double mn = fmin(fabs(a), fabs(b));
  return sgn(a) * sgn(b) * mn + log1p(exp(-fabs(a + b))) - log1p(exp(-fabs(a - b)));
}

static double clip(double v, double L) { return v > L ? L : (v < -L ? -L : v); }

/*
 * Check-node update of eq. (6) for one check of degree d with syndrome bit z:
 * c2v[k] = clip((-1)^z [+]_{r != k} v2c[r]). The extrinsic combination of each
 * edge joins the prefix (edges before k) and suffix (edges after k); an empty
 * combination is +inf.
 */
int orc_check_node(int d, const double* v2c, int z, double L_max, double* c2v) {
  if (d <= 0) return 0;
  double* pre = (double*)malloc(sizeof(double) * d);
  double* suf = (double*)malloc(sizeof(double) * d);
  if (!pre || !suf) { free(pre); free(suf); return -2; }
  for (int k = 0; k < d; ++k) pre[k] = k == 0 ? INFINITY : (k == 1 ? v2c[0] : orc_boxplus(pre[k - 1], v2c[k - 1]));
  for (int k = d - 1; k >= 0; --k)
    suf[k] = k == d - 1 ? INFINITY : (k == d - 2 ? v2c[d - 1] : orc_boxplus(suf[k + 1], v2c[k + 1]));
  double s = z ? -1.0 : 1.0;
  for (int k = 0; k < d; ++k) {
    double ext;
    if (isinf(pre[k]) && isinf(suf[k])) ext = INFINITY;
    else if (isinf(pre[k])) ext = suf[k];
    else if (isinf(suf[k])) ext = pre[k];
    else ext = orc_boxplus(pre[k], suf[k]);
    c2v[k] = clip(s * ext, L_max);
  }
  free(pre);
  free(suf);
  return 0;
}

/* eq. (6) as printed: (-1)^z 2 atanh(prod_{r != k} tanh(v2c[r] / 2)), clipped */
int orc_check_node_tanh(int d, const double* v2c, int z, double L_max, double* c2v) {
  double s = z ? -1.0 : 1.0;
  for (int k = 0; k < d; ++k) {
    double p = 1.0;
    for (int r = 0; r < d; ++r)
      if (r != k) p *= tanh(v2c[r] / 2.0);
    c2v[k] = clip(s * 2.0 * atanh(p), L_max);
  }
  return 0;
}

/*
 * Min-sum check-node rule (an algorithm variant, not in the paper): the
 * magnitude of the extrinsic combination is replaced by the smallest magnitude
 * among the other incoming messages, the sign kept:
 * c2v[k] = (-1)^z prod_{r != k} sgn(v2c[r]) * min_{r != k} |v2c[r]|, clipped.
 */
int orc_check_node_minsum(int d, const double* v2c, int z, double L_max, double* c2v) {
  for (int k = 0; k < d; ++k) {
    double s = z ? -1.0 : 1.0, mn = INFINITY;
    for (int r = 0; r < d; ++r) {
      if (r == k) continue;
      s *= sgn(v2c[r]);
      if (fabs(v2c[r]) < mn) mn = fabs(v2c[r]);
    }
    c2v[k] = clip(s * mn, L_max);
  }
  return 0;
}

/* ------------------------------------------------------ Algorithm 1 */

typedef struct {
  const orc_code* C;
  int F, T, early_exit;
  int rule;                 /* 0: sum-product (eq. 6), 1: min-sum */
  int serial;               /* 0: flooding over all matrices, 1: matrix by matrix (Algorithm 1's nesting) */
  double L_max;
  const double* L_P;        /* [F][n] */
  const uint32_t* z_bits;   /* [u][F][words(m_l)] */
  uint32_t* x_hat_bits;     /* [F][words(n)] */
  int32_t* iters;           /* [F] */
  uint8_t* success;         /* [F] */
  uint8_t* synd_ok;         /* [F][u] or NULL */
  double* L_V_out;          /* [F][n] or NULL */
  double* c2v_out;          /* [F][e_tot] or NULL */
  int f_begin, f_end, rc;
} job_t;

/* every matrix's syndrome of the hard decision equals Alice's (stopping rule, Section 2) */
static int all_syndromes_ok(const orc_code* C, const uint32_t* z_all, int F, int f, const uint32_t* xhat,
                            uint8_t* per_matrix) {
  int ok = 1;
  for (int l = 0; l < C->u; ++l) {
    const uint32_t* z = z_all + z_offset(C, F, l, f);
    int okl = 1;
    for (int32_t j = 0; j < C->m[l]; ++j)
      if (syndrome_bit(C, C->row_first[l] + j, xhat) != bit_of(z, j)) { okl = 0; break; }
    if (per_matrix) per_matrix[l] = (uint8_t)okl;
    ok &= okl;
  }
  return ok;
}

static int decode_one(const job_t* J, int f, double* c2v, double* v2c, double* LV, uint32_t* xhat,
                      double* vin, double* vout) {
  const orc_code* C = J->C;
  const int n = C->n;
  const double* LP = J->L_P + (int64_t)f * n;
  const double L = J->L_max;
  int t = 0, ok = 0;
  /* t = 0: L_V = L_P, hard decision, syndrome test */
  for (int i = 0; i < n; ++i) LV[i] = LP[i];
  memset(xhat, 0, sizeof(uint32_t) * nwords(n));
  for (int i = 0; i < n; ++i) set_bit(xhat, i, LV[i] < 0.0);
  if (J->early_exit && all_syndromes_ok(C, J->z_bits, J->F, f, xhat, NULL)) {
    ok = 1;
  } else {
    for (int64_t e = 0; e < C->e_tot; ++e) c2v[e] = 0.0; /* Algorithm 1: V2C starts at L_P */
    for (t = 1; t <= J->T; ++t) {
      /* flooding: one step over every check of every matrix; matrix-serial: one step per matrix, each
         using the posterior that the previous matrix's step left */
      const int steps = J->serial ? C->u : 1;
      for (int step = 0; step < steps; ++step) {
        const int32_t r0 = J->serial ? C->row_first[step] : 0;
        const int32_t r1 = J->serial ? C->row_first[step + 1] : C->m_tot;
        /* variable-to-check: L_P plus every other incoming check message, all matrices */
        for (int32_t r = r0; r < r1; ++r)
          for (int64_t a = C->row_ptr[r]; a < C->row_ptr[r + 1]; ++a) {
            const int i = C->edge_col[a];
            double s = LP[i];
            for (int64_t b = C->col_ptr[i]; b < C->col_ptr[i + 1]; ++b)
              if (C->col_edge[b] != a) s += c2v[C->col_edge[b]];
            v2c[a] = clip(s, L);
          }
        /* check-to-variable, eq. (6) (or the min-sum rule), for every check of the step */
        for (int32_t r = r0; r < r1; ++r) {
          int l = C->row_mat[r];
          int zj = bit_of(J->z_bits + z_offset(C, J->F, l, f), C->row_local[r]);
          int d = (int)(C->row_ptr[r + 1] - C->row_ptr[r]);
          for (int k = 0; k < d; ++k) vin[k] = v2c[C->row_ptr[r] + k];
          if (J->rule == 1) orc_check_node_minsum(d, vin, zj, L, vout);
          else if (orc_check_node(d, vin, zj, L, vout)) return -2;
          for (int k = 0; k < d; ++k) c2v[C->row_ptr[r] + k] = vout[k];
        }
        /* soft decision, eq. (2): L_V = L_P + sum over l and checks of C2V, in (l, j) order */
        for (int i = 0; i < n; ++i) {
          double s = LP[i];
          for (int64_t a = C->col_ptr[i]; a < C->col_ptr[i + 1]; ++a) s += c2v[C->col_edge[a]];
          LV[i] = s;
        }
      }
      /* hard decision */
      for (int i = 0; i < n; ++i) set_bit(xhat, i, LV[i] < 0.0);
      /* stopping rule */
      if (J->early_exit && all_syndromes_ok(C, J->z_bits, J->F, f, xhat, NULL)) { ok = 1; break; }
    }
    if (t > J->T) t = J->T;
    if (!J->early_exit) ok = all_syndromes_ok(C, J->z_bits, J->F, f, xhat, NULL);
  }
  J->iters[f] = t;
  J->success[f] = (uint8_t)ok;
  if (J->synd_ok) all_syndromes_ok(C, J->z_bits, J->F, f, xhat, J->synd_ok + (int64_t)f * C->u);
  memcpy(J->x_hat_bits + (int64_t)f * nwords(n), xhat, sizeof(uint32_t) * nwords(n));
  if (J->L_V_out) memcpy(J->L_V_out + (int64_t)f * n, LV, sizeof(double) * n);
  if (J->c2v_out) {
    if (ok && t == 0) memset(J->c2v_out + (int64_t)f * C->e_tot, 0, sizeof(double) * C->e_tot);
    else memcpy(J->c2v_out + (int64_t)f * C->e_tot, c2v, sizeof(double) * C->e_tot);
  }
  return 0;
}

static void* run_job(void* arg) {
  job_t* J = (job_t*)arg;
  const orc_code* C = J->C;
  int dmax = 1;
  for (int32_t r = 0; r < C->m_tot; ++r) {
    int d = (int)(C->row_ptr[r + 1] - C->row_ptr[r]);
    if (d > dmax) dmax = d;
  }
  double* c2v = (double*)malloc(sizeof(double) * (C->e_tot ? C->e_tot : 1));
  double* v2c = (double*)malloc(sizeof(double) * (C->e_tot ? C->e_tot : 1));
  double* LV = (double*)malloc(sizeof(double) * C->n);
  uint32_t* xhat = (uint32_t*)malloc(sizeof(uint32_t) * nwords(C->n));
  double* vin = (double*)malloc(sizeof(double) * dmax);
  double* vout = (double*)malloc(sizeof(double) * dmax);
  J->rc = 0;
  if (!c2v || !v2c || !LV || !xhat || !vin || !vout) J->rc = -2;
  for (int f = J->f_begin; f < J->f_end && !J->rc; ++f) J->rc = decode_one(J, f, c2v, v2c, LV, xhat, vin, vout);
  free(c2v); free(v2c); free(LV); free(xhat); free(vin); free(vout);
  return NULL;
}

/*
 * Decode F frames. L_P [F][n] (double), z_bits [u][F][ceil(m_l/32)].
 * early_exit = 1 applies the stopping rule after every iteration (and at t = 0);
 * early_exit = 0 runs exactly max_iter iterations and reports the final syndrome
 * test as success. Optional outputs (NULL to skip): synd_ok [F][u], L_V_out
 * [F][n], c2v_out [F][e_tot] in stacked CSR edge order (matrix 1's edges, then
 * matrix 2's, ...). Frames are spread over n_threads POSIX threads.
 * rule: 0 = sum-product (eq. 6), 1 = min-sum. serial: 0 = flooding over every
 * matrix; 1 = matrix by matrix, the literal nesting of Algorithm 1 (for each H_l
 * in turn the V2C of its edges, its checks and the soft decision of eq. 2;
 * the stopping rule after all u). Both are variants; the paper's decoder is
 * rule 0 with flooding.
 * Returns 0, -1 (bad arguments) or -2 (out of memory).
 */
int orc_decode_ex(int u, int n, const int32_t* m, const int32_t* row_ptr_cat, const int32_t* col_idx_cat,
                  int F, const double* L_P, const uint32_t* z_bits, int max_iter, double L_max,
                  int early_exit, int rule, int serial, int n_threads, uint32_t* x_hat_bits, int32_t* iters,
                  uint8_t* success, uint8_t* synd_ok, double* L_V_out, double* c2v_out) {
  if (F < 0 || max_iter < 0 || !(L_max > 0) || rule < 0 || rule > 1 || serial < 0 || serial > 1) return -1;
  orc_code C;
  int rc = code_build(&C, u, n, m, row_ptr_cat, col_idx_cat);
  if (rc) { code_free(&C); return rc; }
  if (n_threads < 1) n_threads = 1;
  if (n_threads > F) n_threads = F > 0 ? F : 1;
  job_t* jobs = (job_t*)calloc((size_t)n_threads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); code_free(&C); return -2; }
  for (int k = 0; k < n_threads; ++k) {
    job_t* J = &jobs[k];
    J->C = &C; J->F = F; J->T = max_iter; J->early_exit = early_exit; J->L_max = L_max;
    J->rule = rule; J->serial = serial;
    J->L_P = L_P; J->z_bits = z_bits; J->x_hat_bits = x_hat_bits; J->iters = iters; J->success = success;
    J->synd_ok = synd_ok; J->L_V_out = L_V_out; J->c2v_out = c2v_out;
    J->f_begin = (int)((int64_t)F * k / n_threads);
    J->f_end = (int)((int64_t)F * (k + 1) / n_threads);
  }
  for (int k = 1; k < n_threads; ++k) pthread_create(&th[k], NULL, run_job, &jobs[k]);
  run_job(&jobs[0]);
  for (int k = 1; k < n_threads; ++k) pthread_join(th[k], NULL);
  rc = 0;
  for (int k = 0; k < n_threads; ++k)
    if (jobs[k].rc) rc = jobs[k].rc;
  free(jobs);
  free(th);
  code_free(&C);
  return rc;
}

/* Algorithm 1 as above: flooding, sum-product (eq. 6). */
int orc_decode(int u, int n, const int32_t* m, const int32_t* row_ptr_cat, const int32_t* col_idx_cat,
               int F, const double* L_P, const uint32_t* z_bits, int max_iter, double L_max,
               int early_exit, int n_threads, uint32_t* x_hat_bits, int32_t* iters, uint8_t* success,
               uint8_t* synd_ok, double* L_V_out, double* c2v_out) {
  return orc_decode_ex(u, n, m, row_ptr_cat, col_idx_cat, F, L_P, z_bits, max_iter, L_max, early_exit, 0, 0,
                       n_threads, x_hat_bits, iters, success, synd_ok, L_V_out, c2v_out);
}
