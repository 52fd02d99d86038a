/*
 * tc_oracle.c -- plain, slow FP64 CPU oracle for the general tensor contraction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file; only the tests, the package's smoke check and the bench's CPU
 * baseline leg do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Section 4, eq. (gen-contraction), with the alpha/beta form of
 * Section 3):
 *
 *   C[pi_C(I J)] := alpha * sum_P A[pi_A(I P)] * B[pi_B(P J)] + beta * C[pi_C(I J)]
 *
 * for every multi-index (I, J) of C.  Each element of A, B and C is addressed
 * through its own strides, loc(T[u0..ud-1]) = sum_k u_k * s_k(T) (Section 6.1,
 * "generic layout"), so any layout of A, B or C is contracted in place.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  - a label must occur in exactly two of A, B, C (Section 4 defines I, J, P that
 *    way); a label in one tensor only, in all three, or twice in one tensor is
 *    rejected (OR_ERR_LABEL);
 *  - beta == 0: C is written, never read; alpha == 0: A and B are not read;
 *  - an empty contracted range (some extent in P is 0) gives C = beta * C;
 *  - the sum over P runs in colexicographic order of the P labels taken in the
 *    order in which they first appear in A (the paper fixes no order).
 *
 * Alongside C the oracle can return, per element, the magnitude
 *   mag = |alpha| * sum_P |A||B| + |beta| * |C_old|
 * used to normalise errors.  mag[e] is stored at e = the colexicographic rank
 * of the element's multi-index over C's dimensions in C's own order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_MAX_RANK 16

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_LABEL = -2, OR_ERR_EXTENT = -3 };

typedef struct {
  /* one entry per dimension of C, in C's own order; s_A (s_B) is 0 when the
     label is not an index of A (B) */
  int nc;
  int64_t c_len[OR_MAX_RANK], c_sC[OR_MAX_RANK], c_sA[OR_MAX_RANK], c_sB[OR_MAX_RANK];
  /* the contracted (P) labels, in the order they first appear in A */
  int np;
  int64_t p_len[OR_MAX_RANK], p_sA[OR_MAX_RANK], p_sB[OR_MAX_RANK];
  int64_t p_count;
  double alpha, beta;
  const double *A, *B;
  double *C, *mag;
  int64_t begin, end;
} or_problem;

static int find_label(int r, const char* labels, char x) {
  for (int d = 0; d < r; ++d)
    if (labels[d] == x) return d;
  return -1;
}

static int repeats(int r, const char* labels) {
  for (int d = 0; d < r; ++d)
    for (int e = d + 1; e < r; ++e)
      if (labels[d] == labels[e]) return 1;
  return 0;
}

/* Classify every label into I (A and C), J (B and C) or P (A and B), Section 4. */
static int classify(or_problem* p, int rA, const int64_t* lA, const int64_t* sA, const char* labA,
                    int rB, const int64_t* lB, const int64_t* sB, const char* labB,
                    int rC, const int64_t* lC, const int64_t* sC, const char* labC) {
  if (rA < 0 || rB < 0 || rC < 0 || rA > OR_MAX_RANK || rB > OR_MAX_RANK || rC > OR_MAX_RANK)
    return OR_ERR_ARG;
  for (int d = 0; d < rA; ++d) if (lA[d] < 0) return OR_ERR_ARG;
  for (int d = 0; d < rB; ++d) if (lB[d] < 0) return OR_ERR_ARG;
  for (int d = 0; d < rC; ++d) if (lC[d] < 0) return OR_ERR_ARG;
  if (repeats(rA, labA) || repeats(rB, labB) || repeats(rC, labC)) return OR_ERR_LABEL;

  p->nc = rC;
  for (int d = 0; d < rC; ++d) {
    int ia = find_label(rA, labA, labC[d]);
    int ib = find_label(rB, labB, labC[d]);
    if ((ia < 0) == (ib < 0)) return OR_ERR_LABEL; /* in neither, or in all three */
    if (ia >= 0 && lA[ia] != lC[d]) return OR_ERR_EXTENT;
    if (ib >= 0 && lB[ib] != lC[d]) return OR_ERR_EXTENT;
    p->c_len[d] = lC[d];
    p->c_sC[d] = sC[d];
    p->c_sA[d] = ia >= 0 ? sA[ia] : 0;
    p->c_sB[d] = ib >= 0 ? sB[ib] : 0;
  }
  p->np = 0;
  for (int d = 0; d < rA; ++d) {
    if (find_label(rC, labC, labA[d]) >= 0) continue;
    int ib = find_label(rB, labB, labA[d]);
    if (ib < 0) return OR_ERR_LABEL; /* a label of A alone */
    if (lB[ib] != lA[d]) return OR_ERR_EXTENT;
    p->p_len[p->np] = lA[d];
    p->p_sA[p->np] = sA[d];
    p->p_sB[p->np] = sB[ib];
    p->np++;
  }
  for (int d = 0; d < rB; ++d) {
    if (find_label(rC, labC, labB[d]) >= 0) continue;
    if (find_label(rA, labA, labB[d]) < 0) return OR_ERR_LABEL; /* a label of B alone */
  }
  p->p_count = 1;
  for (int d = 0; d < p->np; ++d) p->p_count *= p->p_len[d];
  return OR_OK;
}

/* Elements [e0, e1) of C, in colexicographic order over C's dimensions. */
static void contract_range(const or_problem* p, int64_t e0, int64_t e1) {
  for (int64_t e = e0; e < e1; ++e) {
    int64_t rem = e, offA = 0, offB = 0, offC = 0;
    for (int d = 0; d < p->nc; ++d) {
      int64_t i = rem % p->c_len[d];
      rem /= p->c_len[d];
      offA += i * p->c_sA[d];
      offB += i * p->c_sB[d];
      offC += i * p->c_sC[d];
    }
    double acc = 0.0, macc = 0.0;
    if (p->alpha != 0.0) {
      for (int64_t q = 0; q < p->p_count; ++q) {
        int64_t r = q, pa = 0, pb = 0;
        for (int d = 0; d < p->np; ++d) {
          int64_t k = r % p->p_len[d];
          r /= p->p_len[d];
          pa += k * p->p_sA[d];
          pb += k * p->p_sB[d];
        }
        double prod = p->A[offA + pa] * p->B[offB + pb];
        acc += prod;
        macc += fabs(prod);
      }
    }
    double cold = 0.0, cnew;
    if (p->beta != 0.0) {
      cold = p->C[offC];
      cnew = p->alpha * acc + p->beta * cold;
    } else {
      cnew = p->alpha * acc;
    }
    p->C[offC] = cnew;
    if (p->mag) p->mag[e] = fabs(p->alpha) * macc + fabs(p->beta) * fabs(cold);
  }
}

typedef struct {
  const or_problem* p;
  int64_t e0, e1;
} or_chunk;

static void* worker(void* arg) {
  const or_chunk* c = (const or_chunk*)arg;
  contract_range(c->p, c->e0, c->e1);
  return NULL;
}

int oracle_num_threads(int requested) {
  if (requested > 0) return requested;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/*
 * Contract in place into C.  Strides are in elements and may be any int64
 * (negative or zero for A and B); each data pointer addresses the element whose
 * indices are all 0.  Only elements with colexicographic rank in [begin, end) are
 * computed (end < 0 means all); mag may be NULL.  nthreads <= 0 uses every
 * online core.  Returns 0 or a negative error code.
 */
int oracle_contract(double alpha, int rA, const int64_t* lenA, const int64_t* strideA,
                    const char* labA, const double* A, int rB, const int64_t* lenB,
                    const int64_t* strideB, const char* labB, const double* B, double beta,
                    int rC, const int64_t* lenC, const int64_t* strideC, const char* labC,
                    double* C, double* mag, int64_t begin, int64_t end, int nthreads) {
  or_problem p;
  memset(&p, 0, sizeof p);
  int rc = classify(&p, rA, lenA, strideA, labA, rB, lenB, strideB, labB, rC, lenC, strideC, labC);
  if (rc != OR_OK) return rc;
  int64_t numel = 1;
  for (int d = 0; d < rC; ++d) numel *= lenC[d];
  if (end < 0 || end > numel) end = numel;
  if (begin < 0) begin = 0;
  if (begin >= end) return OR_OK;
  p.alpha = alpha;
  p.beta = beta;
  p.A = A;
  p.B = B;
  p.C = C;
  p.mag = mag;

  int nt = oracle_num_threads(nthreads);
  int64_t span = end - begin;
  if (nt > span) nt = (int)span;
  if (nt <= 1) {
    contract_range(&p, begin, end);
    return OR_OK;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
  or_chunk* ch = (or_chunk*)malloc(sizeof(or_chunk) * nt);
  for (int t = 0; t < nt; ++t) {
    ch[t].p = &p;
    ch[t].e0 = begin + span * t / nt;
    ch[t].e1 = begin + span * (t + 1) / nt;
    pthread_create(&th[t], NULL, worker, &ch[t]);
  }
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  free(th);
  free(ch);
  return OR_OK;
}

/*
 * Scatter vector of one index bundle (Section 6.1, generic-stride scatter
 * vectors): for the linearised index x of the bundle dims (len[0] fastest),
 *   scat[x] = sum_k u_k(x) * stride[k].
 */
void oracle_scatter(int nd, const int64_t* len, const int64_t* stride, int64_t* out) {
  int64_t n = 1;
  for (int k = 0; k < nd; ++k) n *= len[k];
  for (int64_t x = 0; x < n; ++x) {
    int64_t rem = x, v = 0;
    for (int k = 0; k < nd; ++k) {
      v += (rem % len[k]) * stride[k];
      rem /= len[k];
    }
    out[x] = v;
  }
}

/*
 * Block-scatter vector with blocking parameter b (Section 6.2): entry i is s > 0
 * when scat[j] - scat[j-1] == s for every i*b < j < min(l, (i+1)*b), else 0.  A
 * block of one element has no differences; it is given stride 1.
 */
void oracle_block_scatter(const int64_t* scat, int64_t l, int64_t b, int64_t* out) {
  int64_t nb = (l + b - 1) / b;
  for (int64_t i = 0; i < nb; ++i) {
    int64_t lo = i * b, hi = (i + 1) * b < l ? (i + 1) * b : l;
    if (hi - lo == 1) {
      out[i] = 1;
      continue;
    }
    int64_t s = scat[lo + 1] - scat[lo];
    int ok = s > 0;
    for (int64_t j = lo + 1; j < hi && ok; ++j)
      if (scat[j] - scat[j - 1] != s) ok = 0;
    out[i] = ok ? s : 0;
  }
}
