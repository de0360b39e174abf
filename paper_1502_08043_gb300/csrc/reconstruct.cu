// K2: reconstruction of (IJ|KL) from the per-node tables (Sec. II Eq. 14) with the
// momentum-conservation bookkeeping of planewaves (Sec. I and III: the product of two
// planewaves is a planewave, so (IJ|KL) vanishes unless n_J - n_I + n_L - n_K = 0).
//
// SEPARABLE: V(q) = sum_s c_s T_s[|q_x|] c_s T_s[|q_y|] c_s T_s[|q_z|] with c_s^3 = pref w_s
// folded into the table.  A warp takes 32 quadruples; lane l owns the S_pad/32 consecutive
// nodes starting at l S_pad/32; for every quadruple all lanes read one table row (one
// vector load per axis, conflict free), and a 31-shuffle butterfly transposes and sums
// the 32 x 32 partial sums so that lane l ends with the total of quadruple l.
// COLLAPSED (periodic kernel): prod_x exp(-a_s q_x^2) = exp(-a_s |q|^2), so the node sum
// is a function of the integer m = |q|^2 <= 4 R^2 only; one table of 4R^2 + 1 values,
// one shared-memory gather per integral; the kernel streams 16 B in and 4 B out.
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.cuh"

namespace cc {

constexpr unsigned kFull = 0xffffffffu;
enum : int { kNonCons = 1, kQZero = 2, kRange = 4, kInvalid = 8 };

__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }

// A planewave index vector is one 32-bit word of signed bytes (n_x, n_y, n_z, -), both in
// the basis table and in the int8x4 quadruple form, and the bookkeeping runs on the packed
// words with byte-wise SIMD arithmetic (|n_i| <= 63, so every sum and difference below
// stays inside a signed byte, and the conservation residual inside (-256, 256)).
constexpr uint32_t kXYZ = 0x00ffffffu;

__device__ __forceinline__ uint32_t ld_word(const char4* b, int i) {
  return *reinterpret_cast<const uint32_t*>(b + i);  // one 32-bit load per gather
}

// q = n_J - n_I; conservation n_J - n_I + n_L - n_K == 0; flags; qa = (|q_x|, |q_y|, |q_z|)
// as unsigned bytes
template <bool kPeriodic>
__device__ __forceinline__ int classify(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                        uint32_t& qa) {
  const uint32_t resid = __vsub4(__vadd4(b, d), __vadd4(a, c)) & kXYZ;
  qa = __vabsdiffs4(b, a) & kXYZ;
  int f = 0;
  if (resid != 0) f = kNonCons;
  else if (kPeriodic && qa == 0) f = kQZero;
  return f;
}

// k_col's classification: flags and m = |q|^2 (the sources below, from q's byte magnitudes)
template <bool kPeriodic, typename Src>
__device__ __forceinline__ int classify_m(const Src& src, const int4 v, uint32_t& m) {
  if constexpr (Src::kOwnClassify) {
    return src.template classify_m<kPeriodic>(v, m);
  } else {
    uint32_t qa;
    const int f = src.template classify_raw<kPeriodic>(v, qa);
    m = __dp4a(qa, qa, 0u);
    return f;
  }
}

struct IdsSrc {
  static constexpr bool kHint = false;
  static constexpr bool kOwnClassify = false, kOffsetWords = false;
  const int4* q;
  const char4* basis;
  int Nb;
  __device__ __forceinline__ int4 raw(int64_t i) const { return ld_stream(q + i); }
  template <bool kPeriodic>
  __device__ __forceinline__ int decode(int64_t i, uint32_t& qa) const {
    return classify_raw<kPeriodic>(raw(i), qa);
  }
  template <bool kPeriodic>
  __device__ __forceinline__ int classify_raw(const int4 v, uint32_t& qa) const {
    if ((unsigned)v.x >= (unsigned)Nb || (unsigned)v.y >= (unsigned)Nb ||
        (unsigned)v.z >= (unsigned)Nb || (unsigned)v.w >= (unsigned)Nb) {
      qa = 0;
      return kRange;
    }
    return classify<kPeriodic>(ld_word(basis, v.x), ld_word(basis, v.y), ld_word(basis, v.z),
                               ld_word(basis, v.w), qa);
  }
  // the four index vectors of quadruple i; false if an id is out of range
  __device__ __forceinline__ bool fetch(int64_t i, uint32_t w[4]) const {
    const int4 v = raw(i);
    if ((unsigned)v.x >= (unsigned)Nb || (unsigned)v.y >= (unsigned)Nb ||
        (unsigned)v.z >= (unsigned)Nb || (unsigned)v.w >= (unsigned)Nb)
      return false;
    w[0] = ld_word(basis, v.x);
    w[1] = ld_word(basis, v.y);
    w[2] = ld_word(basis, v.z);
    w[3] = ld_word(basis, v.w);
    return true;
  }
};

// uint16 ids: 8 bytes per quadruple (basis of at most 65536 functions)
struct Ids16Src {
  static constexpr bool kHint = false;
  static constexpr bool kOwnClassify = false, kOffsetWords = false;
  const uint2* q;
  const char4* basis;
  int Nb;
  __device__ __forceinline__ int4 raw(int64_t i) const {
    const uint2 v = __ldcs(q + i);
    return make_int4((int)(v.x & 0xffffu), (int)(v.x >> 16), (int)(v.y & 0xffffu),
                     (int)(v.y >> 16));
  }
  template <bool kPeriodic>
  __device__ __forceinline__ int decode(int64_t i, uint32_t& qa) const {
    return classify_raw<kPeriodic>(raw(i), qa);
  }
  template <bool kPeriodic>
  __device__ __forceinline__ int classify_raw(const int4 v, uint32_t& qa) const {
    if (v.x >= Nb || v.y >= Nb || v.z >= Nb || v.w >= Nb) {
      qa = 0;
      return kRange;
    }
    return classify<kPeriodic>(ld_word(basis, v.x), ld_word(basis, v.y), ld_word(basis, v.z),
                               ld_word(basis, v.w), qa);
  }
  __device__ __forceinline__ bool fetch(int64_t i, uint32_t w[4]) const {
    const int4 v = raw(i);
    if (v.x >= Nb || v.y >= Nb || v.z >= Nb || v.w >= Nb) return false;
    w[0] = ld_word(basis, v.x);
    w[1] = ld_word(basis, v.y);
    w[2] = ld_word(basis, v.z);
    w[3] = ld_word(basis, v.w);
    return true;
  }
};

struct VecSrc {
  static constexpr bool kHint = false;
  static constexpr bool kOwnClassify = false, kOffsetWords = false;
  const int4* q;
  const char4* basis;  // unused
  int R2;
  __device__ __forceinline__ bool in_sphere(uint32_t a) const {
    const int v = (int)(a & kXYZ);
    return __dp4a(v, v, 0) <= R2;
  }
  __device__ __forceinline__ int4 raw(int64_t i) const { return ld_stream(q + i); }
  template <bool kPeriodic>
  __device__ __forceinline__ int decode(int64_t i, uint32_t& qa) const {
    return classify_raw<kPeriodic>(raw(i), qa);
  }
  template <bool kPeriodic>
  __device__ __forceinline__ int classify_raw(const int4 v, uint32_t& qa) const {
    const uint32_t a = (uint32_t)v.x, b = (uint32_t)v.y, c = (uint32_t)v.z, d = (uint32_t)v.w;
    if (!in_sphere(a) || !in_sphere(b) || !in_sphere(c) || !in_sphere(d)) {
      qa = 0;
      return kRange;
    }
    return classify<kPeriodic>(a, b, c, d, qa);
  }
  __device__ __forceinline__ bool fetch(int64_t i, uint32_t w[4]) const {
    const int4 v = raw(i);
    w[0] = (uint32_t)v.x;
    w[1] = (uint32_t)v.y;
    w[2] = (uint32_t)v.z;
    w[3] = (uint32_t)v.w;
    return in_sphere(w[0]) && in_sphere(w[1]) && in_sphere(w[2]) && in_sphere(w[3]);
  }
};

// Ids of a basis too large for shared memory (|n| <= 63: 1047331 functions, 4.2 MB) are
// decoded on chip from the hint of their bucket of 32 ids (make_id_hint), staged in shared
// memory, instead of a random gather from the basis in L2.  The basis is the lexicographic
// list of the lines (x, y) inside the sphere, line (x, y) holding the ids of
// z = -z_max .. z_max, z_max = floor(sqrt(R^2 - x^2 - y^2)).  The hint places the bucket's
// first id on its line and gives the next line's z_max; ids further on (about 0.2 % at
// |n| <= 63) walk over whole lines, at most 31 of them.  The words carry every component
// offset by +R (bytes 0 .. 126): the bookkeeping only takes differences of words, so the
// offsets cancel.
__device__ __forceinline__ int isqrt_small(int v) {  // floor(sqrt(v)), 0 <= v < 2^24
  int h = v > 0 ? (int)((float)v * rsqrtf((float)v)) : 0;
  if (h * h > v) --h;
  if ((h + 1) * (h + 1) <= v) ++h;
  return h;
}

__device__ __noinline__ uint32_t id_vector_walk(int R, int x, int y, int pos) {
  // pos = place of the id counted from the first id of the line after (x, y)
  for (int it = 0; it < 32; ++it) {
    ++y;
    int r2 = R * R - x * x - y * y;
    if (r2 < 0) {  // past the plane's last line: first line of the next plane
      ++x;
      y = -isqrt_small(R * R - x * x);
      r2 = R * R - x * x - y * y;
    }
    const int zm = isqrt_small(r2);
    if (pos <= 2 * zm) return (uint32_t)(x + R) | (uint32_t)(y + R) << 8 |
                              (uint32_t)(pos - zm + R) << 16;
    pos -= 2 * zm + 1;
  }
  return 0u;  // not reached for ids below Nb
}

__device__ __forceinline__ uint32_t id_vector(const uint32_t* hint, int R, int id) {
  const uint32_t e = hint[id >> kIdHintShift];
  const int k = id & ((1 << kIdHintShift) - 1);
  const int rest = (int)((e >> 21) & 31u), zm1 = (int)(e >> 26);
  const int k1 = k - rest - 1;  // place on the next line (x, y + 1) when >= 0
  const bool next = k1 >= 0;
  if (next && (zm1 == 63 || k1 > 2 * zm1))
    return id_vector_walk(R, (int)(e & 127u) - R, (int)((e >> 7) & 127u) - R, k1);
  const uint32_t xy = (e & 127u) | ((e << 1) & 0x7f00u);  // bytes x + R, y + R
  const uint32_t zR = next ? (uint32_t)(R - zm1 + k1) : ((e >> 14) & 127u) + (uint32_t)k;
  return xy + (next ? 256u : 0u) + (zR << 16);
}

template <bool k16>  // uint16 ids (8 bytes per quadruple) or int32 ids (16 bytes)
struct IdsDecSrc {
  static constexpr bool kHint = true;
  static constexpr bool kOwnClassify = true, kOffsetWords = false;
  const void* q;
  const uint32_t* hint;  // [nhint], moved to shared memory by the kernel
  int Nb, R, nhint;
  __device__ __forceinline__ int4 raw(int64_t i) const {
    if constexpr (k16) {
      const uint2 v = __ldcs(reinterpret_cast<const uint2*>(q) + i);
      return make_int4((int)(v.x & 0xffffu), (int)(v.x >> 16), (int)(v.y & 0xffffu),
                       (int)(v.y >> 16));
    } else {
      return ld_stream(reinterpret_cast<const int4*>(q) + i);
    }
  }
  __device__ __forceinline__ bool in_range(const int4 v) const {
    return (unsigned)v.x < (unsigned)Nb && (unsigned)v.y < (unsigned)Nb &&
           (unsigned)v.z < (unsigned)Nb && (unsigned)v.w < (unsigned)Nb;
  }
  template <bool kPeriodic>
  __device__ __forceinline__ int decode(int64_t i, uint32_t& qa) const {
    return classify_raw<kPeriodic>(raw(i), qa);
  }
  template <bool kPeriodic>
  __device__ __forceinline__ int classify_raw(const int4 v, uint32_t& qa) const {
    if (!in_range(v)) {
      qa = 0;
      return kRange;
    }
    return classify<kPeriodic>(id_vector(hint, R, v.x), id_vector(hint, R, v.y),
                               id_vector(hint, R, v.z), id_vector(hint, R, v.w), qa);
  }
  // The decoded words have bytes in [0, 2R] (offset by +R), so byte sums stay below 256
  // and plain 32-bit arithmetic is exact byte by byte: conservation is b + d == a + c, and
  // ((b | 0x80..) - a) ^ 0x80.. holds the signed bytes of q = n_J - n_I, whose dot product
  // with itself is |q|^2.
  template <bool kPeriodic>
  __device__ __forceinline__ int classify_m(const int4 v, uint32_t& m) const {
    if (!in_range(v)) {
      m = 0;
      return kRange;
    }
    const uint32_t a = id_vector(hint, R, v.x), b = id_vector(hint, R, v.y),
                   c = id_vector(hint, R, v.z), d = id_vector(hint, R, v.w);
    const uint32_t q = ((b | 0x80808080u) - a) ^ 0x80808080u;
    m = (uint32_t)__dp4a((int)q, (int)q, 0);
    if (b + d != a + c) return kNonCons;
    if (kPeriodic && m == 0) return kQZero;
    return 0;
  }
  __device__ __forceinline__ bool fetch(int64_t i, uint32_t w[4]) const {
    const int4 v = raw(i);
    if (!in_range(v)) return false;
    w[0] = id_vector(hint, R, v.x);
    w[1] = id_vector(hint, R, v.y);
    w[2] = id_vector(hint, R, v.z);
    w[3] = id_vector(hint, R, v.w);
    return true;
  }
};

// uint16 or int32 ids of a basis staged in shared memory by k_col with every component
// offset by +R (bytes 0 .. 2R): the bookkeeping runs on whole words without carries, as for
// decoded ids (conservation b + d == a + c; q's signed bytes from one subtraction)
template <class Base>
struct OffsetIds : Base {
  static constexpr bool kOwnClassify = true, kOffsetWords = true;
  int R;
  template <bool kPeriodic>
  __device__ __forceinline__ int classify_m(const int4 v, uint32_t& m) const {
    if ((unsigned)v.x >= (unsigned)this->Nb || (unsigned)v.y >= (unsigned)this->Nb ||
        (unsigned)v.z >= (unsigned)this->Nb || (unsigned)v.w >= (unsigned)this->Nb) {
      m = 0;
      return kRange;
    }
    const uint32_t a = ld_word(this->basis, v.x), b = ld_word(this->basis, v.y),
                   c = ld_word(this->basis, v.z), d = ld_word(this->basis, v.w);
    const uint32_t q = ((b | 0x80808080u) - a) ^ 0x80808080u;
    m = (uint32_t)__dp4a((int)q, (int)q, 0);
    if (b + d != a + c) return kNonCons;
    if (kPeriodic && m == 0) return kQZero;
    return 0;
  }
};

// exchange-type pairs (ij|ji): item = row * Nb + col, q = n_col - n_row
struct PairSrc {
  static constexpr bool kHint = false;
  static constexpr bool kOwnClassify = false, kOffsetWords = false;
  const int4* q;  // unused
  const char4* basis;
  int Nb;
  int64_t row0;
  template <bool kPeriodic>
  __device__ __forceinline__ int decode(int64_t i, uint32_t& qa) const {
    const int64_t r = row0 + i / Nb;
    const int c = (int)(i % Nb);
    const uint32_t a = ld_word(basis, (int)r), b = ld_word(basis, c);
    return classify<kPeriodic>(a, b, b, a, qa);
  }
};

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ void flush_counts(unsigned long long* counters, unsigned c0,
                                             unsigned c1, unsigned c2) {
  if (!counters) return;
  if (c0) atomicAdd(counters + 0, (unsigned long long)c0);
  if (c1) atomicAdd(counters + 1, (unsigned long long)c1);
  if (c2) atomicAdd(counters + 2, (unsigned long long)c2);
}

// ---------------------------------------------------------------- separable kernel
// NCH consecutive nodes per lane (S_pad = 32 NCH); NCH = 0 selects a runtime loop.  The
// products are always accumulated in ascending node order, a = fma(x_c y_c, z_c, a).
template <typename T, int NCH>
__device__ __forceinline__ T node_chunk(const T* rx, const T* ry, const T* rz, int nch) {
  T a = T(0);
  if constexpr (sizeof(T) == 4 && NCH > 0 && (NCH % 4 == 0 || NCH % 2 == 0)) {
    // the lane's chunk starts at a multiple of NCH words: vector loads per axis
    constexpr int W = NCH % 4 == 0 ? 4 : 2;
    using V = typename std::conditional<W == 4, float4, float2>::type;
#pragma unroll
    for (int c = 0; c < NCH; c += W) {
      const V x = *reinterpret_cast<const V*>(rx + c);
      const V y = *reinterpret_cast<const V*>(ry + c);
      const V z = *reinterpret_cast<const V*>(rz + c);
      const float* xf = reinterpret_cast<const float*>(&x);
      const float* yf = reinterpret_cast<const float*>(&y);
      const float* zf = reinterpret_cast<const float*>(&z);
#pragma unroll
      for (int e = 0; e < W; ++e) a = fma_t(xf[e] * yf[e], zf[e], a);
    }
  } else if constexpr (NCH > 0) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) a = fma_t(rx[c] * ry[c], rz[c], a);
  } else {
    for (int c = 0; c < nch; ++c) a = fma_t(rx[c] * ry[c], rz[c], a);
  }
  return a;
}

template <typename T, typename Src, bool kPeriodic, int NCH, int kThreads = 256>
__global__ void __launch_bounds__(kThreads) k_sep(Src src, int64_t n, const T* __restrict__ gtab,
                                                  int Dmax, int S_pad, T* __restrict__ out,
                                                  unsigned long long* counters,
                                                  int basis_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* tab = reinterpret_cast<T*>(smem);
  const int tab_elems = (Dmax + 1) * S_pad;
  for (int i = threadIdx.x; i < tab_elems; i += blockDim.x) tab[i] = gtab[i];
  const size_t off = ((size_t)tab_elems * sizeof(T) + 15) & ~(size_t)15;
  if constexpr (Src::kHint) {  // decoded ids: the words carry +R offsets, |q| is unchanged
    uint32_t* sh = reinterpret_cast<uint32_t*>(smem + off);
    for (int i = threadIdx.x; i < src.nhint; i += blockDim.x) sh[i] = src.hint[i];
    src.hint = sh;
  } else if (basis_smem > 0) {
    char4* sb = reinterpret_cast<char4*>(smem + off);
    for (int i = threadIdx.x; i < basis_smem; i += blockDim.x) sb[i] = src.basis[i];
    src.basis = sb;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nch = S_pad >> 5;
  unsigned c0 = 0, c1 = 0, c2 = 0;
  for (int64_t base = ((int64_t)blockIdx.x * nw + warp) * 32; base < n;
       base += (int64_t)gridDim.x * nw * 32) {
    const int64_t i = base + lane;
    uint32_t qa = 0;
    int flag = kInvalid;
    if (i < n) flag = src.template decode<kPeriodic>(i, qa);
    const unsigned pk = flag ? 0u : qa;  // (|q_x|, |q_y|, |q_z|) bytes
    c0 += __popc(__ballot_sync(kFull, flag == kNonCons));
    c1 += __popc(__ballot_sync(kFull, flag == kQZero));
    c2 += __popc(__ballot_sync(kFull, flag == kRange));
    T acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const unsigned p = __shfl_sync(kFull, pk, k);
      const int lo = lane * nch;  // this lane's nodes lane*nch .. lane*nch + nch - 1
      const T* rx = tab + (p & 255u) * S_pad + lo;
      const T* ry = tab + ((p >> 8) & 255u) * S_pad + lo;
      const T* rz = tab + ((p >> 16) & 255u) * S_pad + lo;
      acc[k] = node_chunk<T, NCH>(rx, ry, rz, nch);
    }
    // butterfly transpose-reduce: afterwards lane l holds the sum over lanes of acc[l]
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int j = 0; j < o; ++j) {
        const T send = up ? acc[j] : acc[j + o];
        const T keep = up ? acc[j + o] : acc[j];
        acc[j] = keep + __shfl_xor_sync(kFull, send, o);
      }
    }
    if (i < n) out[i] = flag ? T(0) : acc[0];
  }
  if (lane == 0) flush_counts(counters, c0, c1, c2);
}

// ---------------------------------------------------------------- general box kernel
// Any quadruple, conserving or not (Sec. II Eq. 8 with the node sum of Eq. 14):
//   (IJ|KL) = sum_s prod_{x,y,z} c_s A(alpha_s, D1, D2),  D1 = n_J - n_I, D2 = n_L - n_K,
// c_s^3 = pref w_s folded into the table.  A is unchanged by swapping D1, D2 and by negating
// both, so the table has one row per canonical pair d1 >= |d2|, code d1^2 + d1 + d2.
__device__ __forceinline__ int gen_code(int d1, int d2) {
  int a = d1, b = d2;
  if (abs(b) > abs(a)) {
    a = d2;
    b = d1;
  }
  if (a < 0) {
    a = -a;
    b = -b;
  }
  return a * a + a + b;
}

__device__ __forceinline__ int sbyte(uint32_t w, int k) { return (int)(int8_t)(w >> (8 * k)); }

// The same warp organisation as k_sep (lane l owns nodes l S_pad/32 ..; butterfly
// transpose-reduce).  The table [codes][S_pad] is staged in shared memory when it fits
// (tab_smem), otherwise read through the L1 cache from global memory.
template <typename T, typename Src, int NCH>
__global__ void __launch_bounds__(256) k_gen(Src src, int64_t n, const T* __restrict__ gtab,
                                             int codes, int S_pad, T* __restrict__ out,
                                             unsigned long long* counters, int tab_smem,
                                             int basis_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  const T* tab = gtab;
  size_t off = 0;
  if (tab_smem) {
    T* st = reinterpret_cast<T*>(smem);
    const int tab_elems = codes * S_pad;
    for (int i = threadIdx.x; i < tab_elems; i += blockDim.x) st[i] = gtab[i];
    tab = st;
    off = ((size_t)tab_elems * sizeof(T) + 15) & ~(size_t)15;
  }
  if (basis_smem > 0) {
    char4* sb = reinterpret_cast<char4*>(smem + off);
    for (int i = threadIdx.x; i < basis_smem; i += blockDim.x) sb[i] = src.basis[i];
    src.basis = sb;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nch = S_pad >> 5;
  unsigned c0 = 0, c2 = 0;
  for (int64_t base = ((int64_t)blockIdx.x * nw + warp) * 32; base < n;
       base += (int64_t)gridDim.x * nw * 32) {
    const int64_t i = base + lane;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    const bool live = i < n;
    const bool ok = live && src.fetch(i, w);
    uint32_t pxy = 0, pz = 0;  // codes (x | y << 16, z); 0 (a valid row) for dead lanes
    bool noncons = false;
    if (ok) {
      int cx[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int d1 = sbyte(w[1], k) - sbyte(w[0], k), d2 = sbyte(w[3], k) - sbyte(w[2], k);
        noncons |= d1 + d2 != 0;
        cx[k] = gen_code(d1, d2);
      }
      pxy = (uint32_t)cx[0] | ((uint32_t)cx[1] << 16);
      pz = (uint32_t)cx[2];
    }
    c0 += __popc(__ballot_sync(kFull, ok && noncons));
    c2 += __popc(__ballot_sync(kFull, live && !ok));
    T acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const uint32_t p = __shfl_sync(kFull, pxy, k), q = __shfl_sync(kFull, pz, k);
      const int lo = lane * nch;
      const T* rx = tab + (size_t)(p & 0xffffu) * S_pad + lo;
      const T* ry = tab + (size_t)(p >> 16) * S_pad + lo;
      const T* rz = tab + (size_t)q * S_pad + lo;
      acc[k] = node_chunk<T, NCH>(rx, ry, rz, nch);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int j = 0; j < o; ++j) {
        const T send = up ? acc[j] : acc[j + o];
        const T keep = up ? acc[j + o] : acc[j];
        acc[j] = keep + __shfl_xor_sync(kFull, send, o);
      }
    }
    if (live) out[i] = ok ? acc[0] : T(0);
  }
  if (lane == 0) flush_counts(counters, c0, 0, c2);
}

// ---------------------------------------------------------------- collapsed kernel
// kRep copies of the table V_m in shared memory, copy c holding entry m at word kRep m + c,
// and lane l reading copy l % kRep: a warp's gathers of V_m then conflict at most
// 32 / kRep ways (kRep = 16: lanes l and l + 16 share a copy), instead of landing on random
// banks.  kRep = 1 is the plain table.
template <typename T, typename Src, int kRep, int kThreads>
__global__ void __launch_bounds__(kThreads) k_col(Src src, int64_t n, const T* __restrict__ gVm,
                                             int m_max, T* __restrict__ out,
                                             unsigned long long* counters, int basis_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* Vm = reinterpret_cast<T*>(smem);
  for (int i = threadIdx.x; i < (m_max + 1) * kRep; i += blockDim.x) Vm[i] = gVm[i / kRep];
  const size_t off = ((size_t)(m_max + 1) * kRep * sizeof(T) + 15) & ~(size_t)15;
  if constexpr (Src::kHint) {
    uint32_t* sh = reinterpret_cast<uint32_t*>(smem + off);
    for (int i = threadIdx.x; i < src.nhint; i += blockDim.x) sh[i] = src.hint[i];
    src.hint = sh;
  } else if (basis_smem > 0) {
    char4* sb = reinterpret_cast<char4*>(smem + off);
    if constexpr (Src::kOffsetWords) {
      const uint32_t offR = (uint32_t)src.R * 0x010101u;
      uint32_t* sw = reinterpret_cast<uint32_t*>(sb);
      for (int i = threadIdx.x; i < basis_smem; i += blockDim.x)
        sw[i] = __vadd4(ld_word(src.basis, i), offR) & kXYZ;
    } else {
      for (int i = threadIdx.x; i < basis_smem; i += blockDim.x) sb[i] = src.basis[i];
    }
    src.basis = sb;
  }
  __syncthreads();
  const T* Vl = Vm + (threadIdx.x & (kRep - 1));  // this lane's copy
  unsigned c0 = 0, c1 = 0, c2 = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = 8;  // 8 streaming loads in flight per thread before any use
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (U - 1) * stride < n; i += U * stride) {
    int4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = src.raw(i + u * stride);
    int f[U];
    uint32_t m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) f[u] = classify_m<true>(src, v[u], m[u]);  // m = |q|^2
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (f[u]) {  // rare
        c0 += f[u] == kNonCons;
        c1 += f[u] == kQZero;
        c2 += f[u] == kRange;
      }
      __stcs(out + i + u * stride, f[u] ? T(0) : Vl[m[u] * kRep]);
    }
  }
  for (; i < n; i += stride) {
    uint32_t mm;
    const int f = classify_m<true>(src, src.raw(i), mm);
    c0 += f == kNonCons;
    c1 += f == kQZero;
    c2 += f == kRange;
    __stcs(out + i, f ? T(0) : Vl[mm * kRep]);
  }
  c0 = __reduce_add_sync(kFull, c0);
  c1 = __reduce_add_sync(kFull, c1);
  c2 = __reduce_add_sync(kFull, c2);
  if ((threadIdx.x & 31) == 0) flush_counts(counters, c0, c1, c2);
}

// all-pairs, collapsed: out[r][j] = V_m[|n_j - n_{row0+r}|^2]
template <typename T>
__global__ void __launch_bounds__(256) k_pair_col(const char4* __restrict__ gbasis, int Nb,
                                                  int64_t row0, int64_t nrows,
                                                  const T* __restrict__ gVm, int m_max,
                                                  T* __restrict__ out, int basis_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* Vm = reinterpret_cast<T*>(smem);
  for (int i = threadIdx.x; i <= m_max; i += blockDim.x) Vm[i] = gVm[i];
  const char4* basis = gbasis;
  if (basis_smem > 0) {
    const size_t off = ((size_t)(m_max + 1) * sizeof(T) + 15) & ~(size_t)15;
    char4* sb = reinterpret_cast<char4*>(smem + off);
    for (int i = threadIdx.x; i < basis_smem; i += blockDim.x) sb[i] = gbasis[i];
    basis = sb;
  }
  __syncthreads();
  for (int64_t r = blockIdx.y; r < nrows; r += gridDim.y) {
    const uint32_t a = ld_word(gbasis, (int)(row0 + r));
    T* orow = out + r * (int64_t)Nb;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Nb; j += gridDim.x * blockDim.x) {
      const uint32_t qa = __vabsdiffs4(ld_word(basis, j), a) & kXYZ;
      __stcs(orow + j, Vm[__dp4a(qa, qa, 0u)]);
    }
  }
}

// ---------------------------------------------------------------- launch helpers
static int g_num_sms = 0;

static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

template <typename K>
static cc_status grid_for(K kernel, int threads, size_t smem, int64_t work_items, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) {
    set_last_error("cudaFuncSetAttribute", e);
    return CC_ERR_CUDA;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess || per_sm <= 0) {
    set_last_error("occupancy", e);
    return CC_ERR_CUDA;
  }
  int64_t b = (int64_t)per_sm * num_sms();
  const int64_t need = (work_items + threads - 1) / threads;
  if (need < b) b = need < 1 ? 1 : need;
  *blocks = (int)b;
  return CC_OK;
}

static constexpr size_t kSmemCap = 200 * 1024;

template <typename T, typename Src, bool kPeriodic>
static cc_status launch_sep(cc_tables t, Src src, int64_t n, T* out,
                            unsigned long long* counters, cudaStream_t st) {
  const T* tab;
  if constexpr (sizeof(T) == 4) tab = reinterpret_cast<const T*>(t->d.sep32);
  else tab = reinterpret_cast<const T*>(t->d.sep64);
  const size_t tb = (((size_t)(t->Dmax + 1) * t->S_pad * sizeof(T)) + 15) & ~(size_t)15;
  if (tb > kSmemCap) return CC_ERR_RANGE;
  int basis_smem = 0;
  size_t smem = tb;
  if constexpr (Src::kHint) {
    smem = tb + (size_t)src.nhint * 4;
  } else if (tb + (size_t)t->Nb * 4 <= 96 * 1024) {
    basis_smem = t->Nb;
    smem = tb + (size_t)basis_smem * 4;
  }
  const int nch = t->S_pad / 32;
  // decoding sources hold one 512-thread block per SM (table and hints fill shared memory)
  constexpr int kThr = Src::kHint ? 512 : 256;
  auto kern = nch == 1 ? k_sep<T, Src, kPeriodic, 1, kThr>
            : nch == 2 ? k_sep<T, Src, kPeriodic, 2, kThr>
            : nch == 3 ? k_sep<T, Src, kPeriodic, 3, kThr>
            : nch == 4 ? k_sep<T, Src, kPeriodic, 4, kThr>
                       : k_sep<T, Src, kPeriodic, 0, kThr>;
  int blocks = 0;
  CC_TRY(grid_for(kern, kThr, smem, (n + 7) / 8, &blocks));
  kern<<<blocks, kThr, smem, st>>>(src, n, tab, t->Dmax, t->S_pad, out, counters, basis_smem);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

template <typename T, typename Src>
static cc_status launch_gen(cc_tables t, Src src, int64_t n, T* out,
                            unsigned long long* counters, cudaStream_t st) {
  const T* tab;
  if constexpr (sizeof(T) == 4) tab = reinterpret_cast<const T*>(t->d.sepG32);
  else tab = reinterpret_cast<const T*>(t->d.sepG64);
  if (!tab) return CC_ERR_NOTSUPP;
  const size_t tb = (((size_t)t->Gc * t->S_pad * sizeof(T)) + 15) & ~(size_t)15;
  const int tab_smem = tb <= kSmemCap ? 1 : 0;
  const size_t tsm = tab_smem ? tb : 0;
  int basis_smem = 0;
  if (src.basis && tsm + (size_t)t->Nb * 4 <= (tab_smem ? kSmemCap : 96 * 1024)) basis_smem = t->Nb;
  const size_t smem = tsm + (size_t)basis_smem * 4;
  const int nch = t->S_pad / 32;
  auto kern = nch == 1 ? k_gen<T, Src, 1>
            : nch == 2 ? k_gen<T, Src, 2>
            : nch == 4 ? k_gen<T, Src, 4>
            : nch == 6 ? k_gen<T, Src, 6>
                       : k_gen<T, Src, 0>;
  int blocks = 0;
  CC_TRY(grid_for(kern, 256, smem, (n + 7) / 8, &blocks));
  kern<<<blocks, 256, smem, st>>>(src, n, tab, t->Gc, t->S_pad, out, counters, tab_smem,
                                  basis_smem);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

// 1: int32 ids of bases too large for shared memory are decoded on chip (IdsDecSrc);
// 0: gathered from the basis in global memory (L2)
static int g_id_decode = 1;

template <typename T, typename Src>
static cc_status launch_col(cc_tables t, Src src, int64_t n, T* out, unsigned long long* counters,
                            cudaStream_t st, bool uses_basis) {
  const T* Vm;
  if constexpr (sizeof(T) == 4) Vm = reinterpret_cast<const T*>(t->d.Vm32);
  else Vm = reinterpret_cast<const T*>(t->d.Vm64);
  const size_t tb1 = (((size_t)(t->m_max + 1) * sizeof(T)) + 15) & ~(size_t)15;
  if (tb1 > kSmemCap) return CC_ERR_RANGE;
  // the replicated table when it and the basis fit in 96 KB (two 512-thread blocks per SM)
  constexpr int kRep = 16;
  const size_t tbr = (((size_t)(t->m_max + 1) * kRep * sizeof(T)) + 15) & ~(size_t)15;
  size_t staged = uses_basis ? (size_t)t->Nb * 4 : 0;
  if constexpr (Src::kHint) staged = (size_t)src.nhint * 4;
  const bool rep = tbr + staged <= 96 * 1024;
  const size_t tb = rep ? tbr : tb1;
  int basis_smem = 0;
  if (uses_basis && tb + (size_t)t->Nb * 4 <= (rep ? 96 * 1024 : 48 * 1024)) basis_smem = t->Nb;
  size_t smem = tb + (size_t)basis_smem * 4;
  if constexpr (Src::kHint) smem = tb + (size_t)src.nhint * 4;
  // decoding sources hold one 1024-thread block per SM (the hints fill shared memory)
  constexpr int kThreads = Src::kHint ? 1024 : 512;
  auto go = [&](auto s) -> cc_status {
    using S = decltype(s);
    auto kern = rep ? k_col<T, S, kRep, kThreads> : k_col<T, S, 1, kThreads>;
    int blocks = 0;
    CC_TRY(grid_for(kern, kThreads, smem, (n + 7) / 8, &blocks));
    kern<<<blocks, kThreads, smem, st>>>(s, n, Vm, t->m_max, out, counters, basis_smem);
    CC_CUDA(cudaGetLastError());
    return CC_OK;
  };
  // ids whose basis is staged: offset words, carry-free bookkeeping
  if constexpr (std::is_same<Src, IdsSrc>::value || std::is_same<Src, Ids16Src>::value) {
    if (basis_smem > 0) {
      OffsetIds<Src> os;
      static_cast<Src&>(os) = src;
      os.R = t->p.R;
      return go(os);
    }
  }
  return go(src);
}

template <typename T>
static cc_status reconstruct_t(cc_tables t, const void* quads, int64_t n, int format, int lookup,
                               T* out, unsigned long long* counters, cudaStream_t st) {
  const bool periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  const char4* basis = reinterpret_cast<const char4*>(t->d.basis);
  const int4* q = reinterpret_cast<const int4*>(quads);
  const uint2* q16 = reinterpret_cast<const uint2*>(quads);
  if (lookup == CC_LOOKUP_GENERAL) {
    if (format == CC_QUAD_IDS_U16)
      return launch_gen<T>(t, Ids16Src{q16, basis, t->Nb}, n, out, counters, st);
    if (format == CC_QUAD_IDS_I32)
      return launch_gen<T>(t, IdsSrc{q, basis, t->Nb}, n, out, counters, st);
    return launch_gen<T>(t, VecSrc{q, nullptr, t->p.R * t->p.R}, n, out, counters, st);
  }
  // collapsed lookups decode ids on chip when the basis cannot be staged but the hints can
  const size_t tbc = (((size_t)(t->m_max + 1) * sizeof(T)) + 15) & ~(size_t)15;
  const int nhint = (t->Nb + (1 << kIdHintShift) - 1) >> kIdHintShift;
  const bool dec = tbc + (size_t)t->Nb * 4 > 48 * 1024 && tbc + (size_t)nhint * 4 <= kSmemCap &&
                   __atomic_load_n(&g_id_decode, __ATOMIC_ACQUIRE);
  // ... and so do separable lookups, with their table
  const size_t tbs = (((size_t)(t->Dmax + 1) * t->S_pad * sizeof(T)) + 15) & ~(size_t)15;
  const bool dec_s = tbs + (size_t)t->Nb * 4 > 96 * 1024 &&
                     tbs + (size_t)nhint * 4 <= kSmemCap &&
                     __atomic_load_n(&g_id_decode, __ATOMIC_ACQUIRE);
  if (format == CC_QUAD_IDS_U16) {
    if (lookup == CC_LOOKUP_COLLAPSED && dec)
      return launch_col<T>(t, IdsDecSrc<true>{quads, t->d.idhint, t->Nb, t->p.R, nhint}, n,
                           out, counters, st, false);
    if (lookup == CC_LOOKUP_COLLAPSED)
      return launch_col<T>(t, Ids16Src{q16, basis, t->Nb}, n, out, counters, st, true);
    if (dec_s) {
      const IdsDecSrc<true> d{quads, t->d.idhint, t->Nb, t->p.R, nhint};
      if (periodic) return launch_sep<T, IdsDecSrc<true>, true>(t, d, n, out, counters, st);
      return launch_sep<T, IdsDecSrc<true>, false>(t, d, n, out, counters, st);
    }
    if (periodic) return launch_sep<T, Ids16Src, true>(t, Ids16Src{q16, basis, t->Nb}, n, out, counters, st);
    return launch_sep<T, Ids16Src, false>(t, Ids16Src{q16, basis, t->Nb}, n, out, counters, st);
  }
  if (lookup == CC_LOOKUP_COLLAPSED) {
    if (format == CC_QUAD_IDS_I32 && dec)
      return launch_col<T>(t, IdsDecSrc<false>{quads, t->d.idhint, t->Nb, t->p.R, nhint}, n,
                           out, counters, st, false);
    if (format == CC_QUAD_IDS_I32) return launch_col<T>(t, IdsSrc{q, basis, t->Nb}, n, out, counters, st, true);
    return launch_col<T>(t, VecSrc{q, basis, t->p.R * t->p.R}, n, out, counters, st, false);
  }
  if (format == CC_QUAD_IDS_I32) {
    if (dec_s) {
      const IdsDecSrc<false> d{quads, t->d.idhint, t->Nb, t->p.R, nhint};
      if (periodic) return launch_sep<T, IdsDecSrc<false>, true>(t, d, n, out, counters, st);
      return launch_sep<T, IdsDecSrc<false>, false>(t, d, n, out, counters, st);
    }
    if (periodic) return launch_sep<T, IdsSrc, true>(t, IdsSrc{q, basis, t->Nb}, n, out, counters, st);
    return launch_sep<T, IdsSrc, false>(t, IdsSrc{q, basis, t->Nb}, n, out, counters, st);
  }
  if (periodic)
    return launch_sep<T, VecSrc, true>(t, VecSrc{q, basis, t->p.R * t->p.R}, n, out, counters, st);
  return launch_sep<T, VecSrc, false>(t, VecSrc{q, basis, t->p.R * t->p.R}, n, out, counters, st);
}

template <typename T>
static cc_status pairs_t(cc_tables t, int64_t row0, int64_t nrows, int lookup, T* out,
                         cudaStream_t st) {
  const char4* basis = reinterpret_cast<const char4*>(t->d.basis);
  if (lookup == CC_LOOKUP_COLLAPSED) {
    const T* Vm;
    if constexpr (sizeof(T) == 4) Vm = reinterpret_cast<const T*>(t->d.Vm32);
    else Vm = reinterpret_cast<const T*>(t->d.Vm64);
    const size_t tb = (((size_t)(t->m_max + 1) * sizeof(T)) + 15) & ~(size_t)15;
    if (tb > kSmemCap) return CC_ERR_RANGE;
    int basis_smem = tb + (size_t)t->Nb * 4 <= 48 * 1024 ? t->Nb : 0;
    const size_t smem = tb + (size_t)basis_smem * 4;
    auto kern = k_pair_col<T>;
    CC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
    const int bx = (t->Nb + 255) / 256 < 8 ? (t->Nb + 255) / 256 : 8;
    int64_t by = ((int64_t)per_sm * num_sms() + bx - 1) / bx;
    if (by > nrows) by = nrows;
    if (by > 65535) by = 65535;
    if (by < 1) by = 1;
    kern<<<dim3(bx, (unsigned)by), 256, smem, st>>>(basis, t->Nb, row0, nrows, Vm, t->m_max, out,
                                                    basis_smem);
    CC_CUDA(cudaGetLastError());
    return CC_OK;
  }
  const int64_t n = nrows * (int64_t)t->Nb;
  if (t->p.kernel == CC_KERNEL_PERIODIC)
    return launch_sep<T, PairSrc, true>(t, PairSrc{nullptr, basis, t->Nb, row0}, n, out, nullptr, st);
  return launch_sep<T, PairSrc, false>(t, PairSrc{nullptr, basis, t->Nb, row0}, n, out, nullptr, st);
}

}  // namespace cc

using namespace cc;

extern "C" cc_status cc_set_id_decode(int on) {
  if (on != 0 && on != 1) return CC_ERR_ARG;
  __atomic_store_n(&g_id_decode, on, __ATOMIC_RELEASE);
  return CC_OK;
}

extern "C" cc_status cc_reconstruct_integrals(cc_tables t, const void* quads_dev, int64_t n,
                                              int format, int lookup, int precision,
                                              void* out_dev, unsigned long long* counters_dev,
                                              void* stream) {
  if (!t || n < 0) return CC_ERR_ARG;
  if (format != CC_QUAD_IDS_I32 && format != CC_QUAD_VEC_I8X4 && format != CC_QUAD_IDS_U16)
    return CC_ERR_ARG;
  if (format == CC_QUAD_IDS_U16 && t->Nb > 65536) return CC_ERR_RANGE;
  if (lookup != CC_LOOKUP_SEPARABLE && lookup != CC_LOOKUP_COLLAPSED &&
      lookup != CC_LOOKUP_GENERAL)
    return CC_ERR_ARG;
  if (precision != CC_PREC_FP32 && precision != CC_PREC_FP64) return CC_ERR_NOTSUPP;
  if (lookup == CC_LOOKUP_COLLAPSED && t->p.kernel != CC_KERNEL_PERIODIC) return CC_ERR_NOTSUPP;
  if (lookup == CC_LOOKUP_GENERAL && t->p.kernel != CC_KERNEL_BOX) return CC_ERR_NOTSUPP;
  if (n == 0) return CC_OK;
  if (!quads_dev || !out_dev) return CC_ERR_ARG;
  if (((uintptr_t)quads_dev & (format == CC_QUAD_IDS_U16 ? 7 : 15)) != 0) return CC_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (precision == CC_PREC_FP32)
    return reconstruct_t<float>(t, quads_dev, n, format, lookup, (float*)out_dev, counters_dev, st);
  return reconstruct_t<double>(t, quads_dev, n, format, lookup, (double*)out_dev, counters_dev, st);
}

extern "C" cc_status cc_pair_matrix(cc_tables t, int64_t row0, int64_t nrows, int lookup,
                                    int precision, void* out_dev, void* stream) {
  if (!t || row0 < 0 || nrows < 0 || row0 + nrows > t->Nb) return CC_ERR_ARG;
  if (lookup != CC_LOOKUP_SEPARABLE && lookup != CC_LOOKUP_COLLAPSED) return CC_ERR_ARG;
  if (precision != CC_PREC_FP32 && precision != CC_PREC_FP64) return CC_ERR_NOTSUPP;
  if (lookup == CC_LOOKUP_COLLAPSED && t->p.kernel != CC_KERNEL_PERIODIC) return CC_ERR_NOTSUPP;
  if (nrows == 0) return CC_OK;
  if (!out_dev) return CC_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (precision == CC_PREC_FP32) return pairs_t<float>(t, row0, nrows, lookup, (float*)out_dev, st);
  return pairs_t<double>(t, row0, nrows, lookup, (double*)out_dev, st);
}
