// a3: the access plan of the tensor-core mainloop's operands.
//
// Section 7.3 prefers, for each operand, the dimension of unit stride as the
// fast index of the packed panels, and Section 6.2 recognises with the
// block-scatter vectors the blocks of a panel whose stride is regular, which
// the packing then reads as dense vectors.  On GB300 the widest such block is
// a whole tile: when the rows of a tile and one k-tile of an operand form a
// box in the operand's own dims, one TMA box load (cp.async.bulk.tensor, up
// to 5 dims, strides of any order) moves the tile into shared memory with no
// scatter entry at all.  This file decides, per operand, whether its tiles
// are such boxes and encodes the tensor map; operands that are not keep the
// scatter-vector gather of Section 6.1.  It also carries the process-wide
// settings of the tensor-core path: the access (boxes where tiles are boxes
// (default), block gathers only, or element gathers only) and the form of the
// k-split reduction.
//
// A tile of T consecutive linear indices of a bundle (dims d0, d1, ... with
// extents n0, n1, ..., d0 fastest, tiles starting at multiples of T) is a box
// when it covers d0..d(t-1) whole and q = T / (n0...n(t-1)) consecutive
// indices of d(t), with q dividing n(t) -- or d(t) the bundle's last dim, whose
// excess the box reads as zeros.  The smem image of the box is then the tile
// in the mainloop's raw layout: for a k-contiguous operand rows of 32 FP32
// (128 bytes) with the 128-byte swizzle (chunk ^ (row & 7)), for a
// row-contiguous operand 32 k-rows of T FP32 each.
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace tc {
namespace {

std::atomic<int> g_access{TC_ACCESS_AUTO};

constexpr int kTileK = 32;  // k-tile of the tensor-core mainloop
constexpr int kTileM = 128; // rows of an A tile

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Box extents over a bundle for tiles of T consecutive linear indices (see
// the file comment); false when such a tile is not a box.  *end = the dim the
// tile ends in (the next tile's box starts box[*end] further along it).
bool tile_box(const int64_t* len, int nd, int64_t T, uint32_t* box, int* end) {
  int64_t rem = T;
  *end = 0;
  for (int d = 0; d < nd; ++d) {
    if (rem == 1) {
      box[d] = 1;
    } else if (d == nd - 1) {
      box[d] = (uint32_t)rem;  // the last dim may run past its end
      rem = 1;
      *end = d;
    } else if (len[d] >= rem) {
      if (len[d] % rem) return false;
      box[d] = (uint32_t)rem;
      rem = 1;
      *end = d;
    } else {
      if (rem % len[d]) return false;
      box[d] = (uint32_t)len[d];
      rem /= len[d];
    }
  }
  return rem == 1;
}

// One operand: rows = I (A) or J (B), k = P; strides in this operand.
bool make_box(const Bundle& R, const int64_t* rs, const Bundle& K, const int64_t* ks,
              const void* base, int rows, bool kcontig, CUtensorMap* map, BoxAccess* out) {
  std::memset(out, 0, sizeof *out);
  const int nr = R.nd, nk = K.nd;
  if (nr < 1 || nk < 1 || nr > 4 || nk > 4 || nr + nk > 5) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  // the unit-stride dim must lead the bundle the access flag names
  if (kcontig ? ks[0] != 1 : rs[0] != 1) return false;
  const int64_t lim = int64_t(1) << 31;
  int64_t tr = 1, tk = 1;
  for (int i = 0; i < nr; ++i) {
    if (R.len[i] <= 0 || R.len[i] >= lim) return false;
    tr *= R.len[i];
  }
  for (int i = 0; i < nk; ++i) {
    if (K.len[i] <= 0 || K.len[i] >= lim) return false;
    tk *= K.len[i];
  }
  if (tr >= lim || tk >= lim) return false;  // coordinates are 32-bit
  uint32_t rbox[4], kbox[4];
  int rend = 0, kend = 0;
  if (!tile_box(R.len, nr, rows, rbox, &rend) || !tile_box(K.len, nk, kTileK, kbox, &kend))
    return false;
  if (kcontig ? kbox[0] != (uint32_t)kTileK : (rbox[0] % 4) != 0) return false;
  // every box extent within its dim's length (a tile may still run past the
  // end of a bundle's last dim, whose excess the box reads as zeros): boxes
  // larger than their tensor are not taken
  for (int i = 0; i < nr; ++i)
    if ((int64_t)rbox[i] > R.len[i]) return false;
  for (int i = 0; i < nk; ++i)
    if ((int64_t)kbox[i] > K.len[i]) return false;

  // tensor-map dims: the unit-stride bundle first, each bundle fastest dim first
  const int rank = nr + nk;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5];
  int64_t st[5];
  int j = 0;
  auto put = [&](const Bundle& B, const int64_t* s, const uint32_t* bx, int n) {
    for (int i = 0; i < n; ++i, ++j) {
      dims[j] = (cuuint64_t)B.len[i];
      st[j] = s[i];
      box[j] = bx[i];
      estr[j] = 1;
    }
  };
  if (kcontig) {
    put(K, ks, kbox, nk);
    put(R, rs, rbox, nr);
  } else {
    put(R, rs, rbox, nr);
    put(K, ks, kbox, nk);
  }
  for (int i = 1; i < rank; ++i) {
    if (st[i] <= 0 || (st[i] % 4) != 0 || st[i] * 4 >= (int64_t(1) << 40)) return false;
    strides[i - 1] = (cuuint64_t)(st[i] * 4);
  }
  if (map) {  // null: the eligibility alone (no driver needed)
    auto fn = encoder();
    if (!fn) return false;
    const CUresult r =
        fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), dims,
           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           kcontig ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  out->rank = rank;
  out->nfirst = kcontig ? nk : nr;
  out->kfirst = kcontig ? 1 : 0;
  out->bytes = rows * kTileK * 4;
  for (int i = 0; i < rank; ++i) out->len[i] = (int32_t)dims[i];
  const int k0 = kcontig ? 0 : nr;  // map index of the k bundle's first dim
  out->klast = k0 + nk - 1;
  out->kstep_dim = k0 + kend;
  out->kstep = (int32_t)kbox[kend];
  return true;
}

}  // namespace

void plan_access(const Layout& L, DevProblem& d, CUtensorMap* maps, bool allow_box, bool pair) {
  std::memset(&d.boxA, 0, sizeof d.boxA);
  std::memset(&d.boxB, 0, sizeof d.boxB);
  d.pair = 0;
  const int acc = g_access.load();
  d.elem_gather = acc == TC_ACCESS_SCATTER ? 1 : 0;
  if (!allow_box || (acc != TC_ACCESS_BOX && acc != TC_ACCESS_AUTO) || L.m <= 0 || L.n <= 0 ||
      L.k <= 0)
    return;
  // both operands or neither: with one operand boxed and the other gathered
  // the kernel would need loader warps and the box warp on one stage, which
  // measured slower than gathering both
  const bool a_ok = make_box(L.I, L.I.s0, L.P, L.P.s0, d.a, kTileM, d.a_kc != 0,
                             maps ? &maps[0] : nullptr, &d.boxA);
  const bool b_ok = make_box(L.J, L.J.s0, L.P, L.P.s1, d.b, pair ? d.bn / 2 : d.bn,
                             d.b_kc != 0, maps ? &maps[1] : nullptr, &d.boxB);
  if (!(a_ok && b_ok)) {
    std::memset(&d.boxA, 0, sizeof d.boxA);
    std::memset(&d.boxB, 0, sizeof d.boxB);
  } else {
    d.pair = pair ? 1 : 0;
  }
}

bool box_encoder_available() { return encoder() != nullptr; }

}  // namespace tc

namespace tc {
namespace {
std::atomic<int> g_reduce{TC_REDUCE_COMPENSATED};
std::atomic<int> g_checks{0};
}
bool split_reduction_f64() { return g_reduce.load() == TC_REDUCE_F64; }
bool checks_on() { return g_checks.load() != 0; }
}  // namespace tc

extern "C" int tc_set_checks(int on) {
  if (on != 0 && on != 1) return TC_ERR_ARG;
  return tc::g_checks.exchange(on);
}

extern "C" int tc_set_split_reduction(int reduce) {
  if (reduce != TC_REDUCE_COMPENSATED && reduce != TC_REDUCE_F64) return TC_ERR_ARG;
  return tc::g_reduce.exchange(reduce);
}

namespace tc {
int access_setting() { return g_access.load(); }
}  // namespace tc

extern "C" int tc_set_access(int access) {
  if (access != TC_ACCESS_BLOCK && access != TC_ACCESS_SCATTER && access != TC_ACCESS_BOX &&
      access != TC_ACCESS_PACKED && access != TC_ACCESS_AUTO)
    return TC_ERR_ARG;
  return tc::g_access.exchange(access);
}
