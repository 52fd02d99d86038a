// Host planner: validation, index bundling and the dimension heuristic.
//
// Section 4 defines the bundles: labels of A and C form I, of B and C form J,
// of A and B form P; each label lies in exactly two tensors with one length.
// Section 7.3 gives the purely logical reordering applied here, in order:
//   1. length-1 dims are discarded;
//   2. dims x, y of a bundle merge when s_y(T) == s_x(T) * n_x in both tensors
//      T carrying the bundle;
//   3. I and J dims are ordered by |stride| in C, smallest first (stable in
//      C's label order);
//   4. when the first J dim has unit stride in C, A and B (and I and J) trade
//      roles, i.e. C^T = B^T A^T is computed, so C's unit stride runs along M;
//   5. P dims are ordered by |stride| in A, smallest first (stable in the
//      original A's label order).
// No data moves; the result only fixes the iteration order of the kernels.
// One GPU-specific step follows the paper's five:
//   6. if A's smallest |stride| lies outside P (A is read along its rows, so
//      the P order does not affect it) and B's smallest |stride| lies in P,
//      re-sort P by |stride| in B, so that B's k-runs are contiguous.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "tc_internal.h"

namespace tc {
namespace {

struct LDim {
  int64_t len;
  int64_t s0, s1;
  char labels[kMaxRank + 1];
  int nlab;
};

int find(const tc_tensor* T, char x) {
  for (int d = 0; d < T->rank; ++d)
    if (T->labels[d] == x) return d;
  return -1;
}

int check_tensor(const tc_tensor* T) {
  if (!T) return TC_ERR_ARG;
  if (T->rank < 0 || T->rank > kMaxRank) return TC_ERR_ARG;
  if (T->rank > 0 && (!T->len || !T->stride || !T->labels)) return TC_ERR_ARG;
  for (int d = 0; d < T->rank; ++d)
    if (T->len[d] < 0) return TC_ERR_ARG;
  for (int d = 0; d < T->rank; ++d) {
    if (T->labels[d] == 0) return TC_ERR_LABEL;  // the folded label strings end at a NUL
    for (int e = d + 1; e < T->rank; ++e)
      if (T->labels[d] == T->labels[e]) return TC_ERR_LABEL;
  }
  return TC_OK;
}

int64_t numel(const tc_tensor* T) {
  int64_t n = 1;
  for (int d = 0; d < T->rank; ++d) n *= T->len[d];
  return n;
}

// C must not overlap itself.  Sufficient test: with its dims of length > 1
// sorted by |stride|, every |stride| exceeds the largest offset reachable with
// the dims before it.
bool self_overlaps(const tc_tensor* C) {
  if (numel(C) == 0) return false;
  int64_t ls[kMaxRank][2];
  int n = 0;
  for (int d = 0; d < C->rank; ++d)
    if (C->len[d] > 1) {
      ls[n][0] = std::llabs(C->stride[d]);
      ls[n][1] = C->len[d];
      ++n;
    }
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && ls[j][0] < ls[j - 1][0]; --j) std::swap(ls[j], ls[j - 1]);
  // span = 1 + largest offset reachable with the dims so far
  int64_t span = 1;
  for (int i = 0; i < n; ++i) {
    if (ls[i][0] < span) return true;
    span += (ls[i][1] - 1) * ls[i][0];
  }
  return false;
}

// Byte range [lo, hi] touched by a tensor (empty tensors touch nothing).
bool byte_range(const tc_tensor* T, size_t es, intptr_t* lo, intptr_t* hi) {
  if (numel(T) == 0) return false;
  int64_t mn = 0, mx = 0;
  for (int d = 0; d < T->rank; ++d) {
    int64_t ext = (T->len[d] - 1) * T->stride[d];
    if (ext < 0) mn += ext; else mx += ext;
  }
  *lo = reinterpret_cast<intptr_t>(T->data) + mn * (int64_t)es;
  *hi = reinterpret_cast<intptr_t>(T->data) + mx * (int64_t)es + (intptr_t)es - 1;
  return true;
}

void fold(LDim* d, int& n) {
  bool merged = true;
  while (merged) {
    merged = false;
    for (int i = 0; i < n && !merged; ++i)
      for (int j = 0; j < n && !merged; ++j) {
        if (i == j) continue;
        if (d[j].s0 == d[i].s0 * d[i].len && d[j].s1 == d[i].s1 * d[i].len) {
          LDim x = d[i];
          x.len = d[i].len * d[j].len;
          for (int q = 0; q < d[j].nlab; ++q) x.labels[x.nlab++] = d[j].labels[q];
          x.labels[x.nlab] = 0;
          d[i] = x;
          for (int q = j; q + 1 < n; ++q) d[q] = d[q + 1];
          --n;
          merged = true;
        }
      }
  }
}

template <typename Key>
void stable_sort(LDim* d, int n, Key key) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && key(d[j]) < key(d[j - 1]); --j) std::swap(d[j], d[j - 1]);
}

}  // namespace

int plan_problem(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, Planned* out) {
  int rc;
  if ((rc = check_tensor(A)) || (rc = check_tensor(B)) || (rc = check_tensor(C))) return rc;
  std::memset(out, 0, sizeof(*out));

  LDim I[kMaxRank], J[kMaxRank], P[kMaxRank];
  int nI = 0, nJ = 0, nP = 0;
  // a1: classify (Section 4)
  for (int d = 0; d < C->rank; ++d) {
    int ia = find(A, C->labels[d]), ib = find(B, C->labels[d]);
    if ((ia < 0) == (ib < 0)) return TC_ERR_LABEL;
    LDim x;
    x.len = C->len[d];
    x.s1 = C->stride[d];
    x.labels[0] = C->labels[d];
    x.labels[1] = 0;
    x.nlab = 1;
    if (ia >= 0) {
      if (A->len[ia] != C->len[d]) return TC_ERR_EXTENT;
      x.s0 = A->stride[ia];
      I[nI++] = x;
    } else {
      if (B->len[ib] != C->len[d]) return TC_ERR_EXTENT;
      x.s0 = B->stride[ib];
      J[nJ++] = x;
    }
  }
  for (int d = 0; d < A->rank; ++d) {
    if (find(C, A->labels[d]) >= 0) continue;
    int ib = find(B, A->labels[d]);
    if (ib < 0) return TC_ERR_LABEL;
    if (B->len[ib] != A->len[d]) return TC_ERR_EXTENT;
    LDim x;
    x.len = A->len[d];
    x.s0 = A->stride[d];
    x.s1 = B->stride[ib];
    x.labels[0] = A->labels[d];
    x.labels[1] = 0;
    x.nlab = 1;
    P[nP++] = x;
  }
  for (int d = 0; d < B->rank; ++d)
    if (find(C, B->labels[d]) < 0 && find(A, B->labels[d]) < 0) return TC_ERR_LABEL;
  if (self_overlaps(C)) return TC_ERR_OVERLAP;

  // a2 step 1: drop length-one dims
  auto drop1 = [](LDim* d, int& n) {
    int w = 0;
    for (int i = 0; i < n; ++i)
      if (d[i].len != 1) d[w++] = d[i];
    n = w;
  };
  drop1(I, nI);
  drop1(J, nJ);
  drop1(P, nP);
  // step 2: merge sequentially contiguous dims
  fold(I, nI);
  fold(J, nJ);
  fold(P, nP);
  // step 3: sort I and J by |stride| in C
  stable_sort(I, nI, [](const LDim& x) { return std::llabs(x.s1); });
  stable_sort(J, nJ, [](const LDim& x) { return std::llabs(x.s1); });
  // step 4: swap when C's unit stride lies in J
  bool swapped = false;
  if (nJ > 0 && J[0].s1 == 1) {
    swapped = true;
    LDim t[kMaxRank];
    int nt = nI;
    std::memcpy(t, I, sizeof(LDim) * nI);
    std::memcpy(I, J, sizeof(LDim) * nJ);
    nI = nJ;
    std::memcpy(J, t, sizeof(LDim) * nt);
    nJ = nt;
    for (int i = 0; i < nP; ++i) std::swap(P[i].s0, P[i].s1);
  }
  // step 5: sort P by |stride| in A
  stable_sort(P, nP, [](const LDim& x) { return std::llabs(x.s0); });
  // step 6 (GPU): B's unit stride orders P when A's lies outside P
  if (nP > 0) {
    int64_t minAP = INT64_MAX, minAI = INT64_MAX, minBP = INT64_MAX, minBJ = INT64_MAX;
    for (int i = 0; i < nP; ++i) {
      minAP = std::min<int64_t>(minAP, std::llabs(P[i].s0));
      minBP = std::min<int64_t>(minBP, std::llabs(P[i].s1));
    }
    for (int i = 0; i < nI; ++i) minAI = std::min<int64_t>(minAI, std::llabs(I[i].s0));
    for (int i = 0; i < nJ; ++i) minBJ = std::min<int64_t>(minBJ, std::llabs(J[i].s0));
    const bool a_rows = nI > 0 && minAI <= minAP;
    const bool b_k = nJ == 0 || minBP < minBJ;
    if (a_rows && b_k) stable_sort(P, nP, [](const LDim& x) { return std::llabs(x.s1); });
  }
  // step 7 (GPU): an operand read along its rows orders its row bundle by its
  // own strides, so that the loaders' consecutive rows are its unit-stride
  // run.  For J and B this costs little: after step 4 C's unit stride lies
  // in I, and the epilogue's threads run along I (each store instruction
  // still covers whole lines; only the distance between a tile's columns
  // grows), and ordering J by C instead can cost B its box form.  For I and A
  // it moves C's unit-stride dim away from the epilogue's threads: every
  // store of C then lands in its own sector, where otherwise every load of A
  // does.  A is read once per output tile across from it (about k x
  // ceil(n / 128) loads per row against n stores), and a scattered store
  // costs about two and a half scattered loads (measured), so I is sorted by
  // A's strides only when k ceil(n / 128) >= 2.5 n.  Otherwise A's
  // smallest-stride dim moves up to second place, right after C's: a tile's
  // rows then span C's first dim and a few steps of A's, so the tiles that
  // run side by side read every sector of A whole between them (from L2)
  // instead of one element of it each.
  int64_t kprod = 1, nprod = 1;
  for (int i = 0; i < nP; ++i) kprod *= P[i].len;
  for (int i = 0; i < nJ; ++i) nprod *= J[i].len;
  {
    int64_t minAP = INT64_MAX, minAI = INT64_MAX, minBP = INT64_MAX, minBJ = INT64_MAX;
    for (int i = 0; i < nP; ++i) {
      minAP = std::min<int64_t>(minAP, std::llabs(P[i].s0));
      minBP = std::min<int64_t>(minBP, std::llabs(P[i].s1));
    }
    for (int i = 0; i < nI; ++i) minAI = std::min<int64_t>(minAI, std::llabs(I[i].s0));
    for (int i = 0; i < nJ; ++i) minBJ = std::min<int64_t>(minBJ, std::llabs(J[i].s0));
    if (nI > 0 && minAI <= minAP) {
      const double loads = (double)kprod * (double)((nprod + 127) / 128);
      if (2.0 * loads >= 5.0 * (double)nprod) {
        stable_sort(I, nI, [](const LDim& x) { return std::llabs(x.s0); });
      } else {
        int u = 0;
        for (int i = 1; i < nI; ++i)
          if (std::llabs(I[i].s0) < std::llabs(I[u].s0)) u = i;
        if (u > 1) {
          const LDim t = I[u];
          for (int i = u; i > 1; --i) I[i] = I[i - 1];
          I[1] = t;
        }
      }
    }
    if (nJ > 0 && minBJ <= minBP) stable_sort(J, nJ, [](const LDim& x) { return std::llabs(x.s0); });
  }

  Layout& L = out->L;
  tc_plan_info& info = out->info;
  auto put = [](Bundle& b, const LDim* d, int n, int64_t* len, int64_t* s0, int64_t* s1,
                char (*labs)[kMaxRank + 1]) {
    b.nd = n;
    int64_t prod = 1;
    for (int i = 0; i < n; ++i) {
      b.len[i] = len[i] = d[i].len;
      b.s0[i] = s0[i] = d[i].s0;
      b.s1[i] = s1[i] = d[i].s1;
      std::memcpy(labs[i], d[i].labels, kMaxRank + 1);
      prod *= d[i].len;
    }
    return prod;
  };
  L.m = put(L.I, I, nI, info.I_len, info.I_sA, info.I_sC, info.I_labels);
  L.n = put(L.J, J, nJ, info.J_len, info.J_sB, info.J_sC, info.J_labels);
  L.k = put(L.P, P, nP, info.P_len, info.P_sA, info.P_sB, info.P_labels);
  // a length-0 dim was kept by step 1, so a product of 0 means an empty range
  info.swapped = swapped;
  info.nI = nI;
  info.nJ = nJ;
  info.nP = nP;
  info.m = L.m;
  info.n = L.n;
  info.k = L.k;

  // a3: stride-1 preference per operand
  auto minabs = [](const int64_t* s, int n) {
    int64_t v = INT64_MAX;
    for (int i = 0; i < n; ++i) v = std::min<int64_t>(v, std::llabs(s[i]));
    return v;
  };
  info.a_k_contig = nP > 0 && (nI == 0 || minabs(L.P.s0, nP) < minabs(L.I.s0, nI));
  info.b_k_contig = nP > 0 && (nJ == 0 || minabs(L.P.s1, nP) < minabs(L.J.s0, nJ));
  info.c_m_contig = nJ == 0 || (nI > 0 && minabs(L.I.s1, nI) <= minabs(L.J.s1, nJ));

  out->a = swapped ? B->data : A->data;
  out->b = swapped ? A->data : B->data;
  out->c = C->data;
  return TC_OK;
}


// Exposed for the API layer.
int aliases(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, size_t es) {
  intptr_t clo, chi, lo, hi;
  if (!byte_range(C, es, &clo, &chi)) return 0;
  if (byte_range(A, es, &lo, &hi) && !(hi < clo || chi < lo)) return 1;
  if (byte_range(B, es, &lo, &hi) && !(hi < clo || chi < lo)) return 1;
  return 0;
}

}  // namespace tc

namespace tc {

bool block_row_bundle(const Layout& L, bool a_k_contig, Layout* out) {
  const Bundle& I = L.I;
  constexpr int64_t B0 = 16, B1 = 8;
  if (a_k_contig || I.nd < 2 || I.nd + 2 > kMaxRank || L.n <= 0 || L.k <= 0) return false;
  // C's unit stride leads the row bundle, A's is the second row dim
  if (std::llabs(I.s1[0]) != 1 || std::llabs(I.s0[1]) != 1 || std::llabs(I.s0[0]) == 1)
    return false;
  const int64_t e0 = I.len[0], e1 = I.len[1];
  if (e0 < B0 || e1 < B1) return false;
  const int64_t h0 = (e0 + B0 - 1) / B0, h1 = (e1 + B1 - 1) / B1;
  int64_t rest = 1;
  for (int d = 2; d < I.nd; ++d) rest *= I.len[d];
  const int64_t mb = B0 * B1 * h0 * h1 * rest;
  // the holes may not cost more than a quarter of the rows
  if ((double)mb > 1.25 * (double)L.m) return false;
  *out = L;
  Bundle& b = out->I;
  auto set = [&](int d, int64_t len, int64_t s0, int64_t s1) {
    b.len[d] = len;
    b.s0[d] = s0;
    b.s1[d] = s1;
  };
  set(0, B0, I.s0[0], I.s1[0]);
  set(1, B1, I.s0[1], I.s1[1]);
  set(2, h0, B0 * I.s0[0], B0 * I.s1[0]);
  set(3, h1, B1 * I.s0[1], B1 * I.s1[1]);
  for (int d = 2; d < I.nd; ++d) set(d + 2, I.len[d], I.s0[d], I.s1[d]);
  b.nd = I.nd + 2;
  b.nblk = 2;
  b.blk_lo[0] = 0;
  b.blk_hi[0] = 2;
  b.blk_b[0] = B0;
  b.blk_lim[0] = e0;
  b.blk_lo[1] = 1;
  b.blk_hi[1] = 3;
  b.blk_b[1] = B1;
  b.blk_lim[1] = e1;
  out->m = mb;
  return true;
}

}  // namespace tc

namespace tc {

void swap_roles(Planned* p) {
  Layout& L = p->L;
  std::swap(L.I, L.J);
  std::swap(L.m, L.n);
  for (int i = 0; i < L.P.nd; ++i) std::swap(L.P.s0[i], L.P.s1[i]);
  std::swap(p->a, p->b);
  tc_plan_info& f = p->info;
  f.swapped = !f.swapped;
  std::swap(f.a_k_contig, f.b_k_contig);
  std::swap(f.m, f.n);
}

}  // namespace tc

