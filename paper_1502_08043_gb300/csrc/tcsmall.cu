// Tensor-core exchange sums for grids of side up to 64 (bf16 hi + lo), the transposed slab
// form: two slabs share every 128-row MMA.
//
// Sec. III exchange of the uniform electron gas with the node sum of Sec. II Eq. 14; the
// periodic kernel uses the D_s = T_s - I split, so with the Fermi-sphere occupation O
//   E[x] = sum_s w_s (T_s R_{s,x} + A_{s,x}) T_s  +  (I x I x Dbar term),
// where, for the slab x (matrices over y, z):
//   R_{s,x}[y][z] = F_s[x][h(y, z)]     the first mode product of O (line along x),
//   A_{s,x}[y][z] = F_s[y][h(x, z)]     O x2 D_s restricted to the slab (line along y),
//   F_s[a][h]     = sum_{k = R-h}^{R+h} D_s[a][k]   (window sums, FP64, 0 for h < 0),
//   h(u, v)       = floor(sqrt(R_F^2 - (u-R)^2 - (v-R)^2)), -1 outside the sphere.
// The box kernel has F_s from T_s, no A term and no Dbar term.
//
// With the grid padded to 64, a unit (slab pair x_0 = 2p, x_1 = 2p + 1; node s) is
//   MMA1  D1[(j, z)][y] = sum_y' R_{s,x_j}[y'][z] T_s[y][y']  +  sum_h P_j[z][h] F_s[y][h]
//         (M = 128 rows (j, z): both slabs; A = R^T built in shared memory, B = T_s and
//         F_s by TMA; P_j[z][h] = [h(x_j, z) = h] is a one-hot matrix fixed per pair)
//   epi   U_{x_j}[y][z] = w_s D1[(j, z)][y], split into bf16 hi + lo and written as the
//         MN-major A operand of MMA2 (row (j, y), K index z)
//   MMA2  E[(j, y)][z'] += sum_z U_{x_j}[y][z] T_s[z][z']   (M = 128 rows (j, y))
// so every MMA uses all 128 rows for grids of side up to 64.  Both remaining mode products
// run over the band |y - R|, |z - R| <= R_F only (K steps of 16), and each is bf16x3:
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory.  E of the pair stays in
// tensor memory over the CTA's run of nodes and leaves once as a partial; a second kernel
// adds the partials of each pair in a fixed order, the Dbar term, and forms eps and E_x.
//
// Pipeline: one warp issues MMA1 of unit after unit, another MMA2, while the builders form
// R^T of unit i + 1 and the epilogue converts D1 of unit i; with two issuing warps neither
// product waits for the other's issue (an N = 64 MMA issues no faster than the pipe runs
// it, and the hand-offs between them would otherwise leave the pipe idle).  T_s (read by
// both products) has three buffers, so the TMA load of unit i + 2 needs only MMA2(i - 1) to
// have finished; F_s, R^T, D1 and the U operand have two each.  The issuers first test all
// the barriers of a product at once (independent test_waits) and only then wait for what
// is not ready, and every role steps its unit's (pair, node) place without a 64-bit
// division.
// Tensor memory (256 columns): [0, 64) D1[0], [64, 128) D1[1], [128, 192) E.
// Warps: 0-7 epilogue (warp w: lanes 32 (w % 4) .., columns 32 (w / 4) ..), 8-10 and 12-14
// build R^T and P, 11 TMA producer, 15 issues MMA1 and 16 MMA2.  Every wait is bounded
// (global timer); on expiry the error word is set, all roles stop, the MMA issuers drain
// their MMAs and tensor memory is freed before the CTA returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "slab_finalize.cuh"
#include "tc_prims.cuh"

namespace cc {

namespace {

constexpr int kThreads = 544;
constexpr int kEpiWarps = 8;
constexpr int kBldWarps = 6;
constexpr int kBldThreads = 32 * kBldWarps;
constexpr int kProdWarp = 11;
constexpr int kMmaWarp = 15;   // issues MMA1
constexpr int kMma2Warp = 16;  // issues MMA2
constexpr int kG = 64;                        // padded grid side
constexpr int kHMax = 64;                     // window half-lengths h = 0 .. R_F <= 31
constexpr uint32_t kPl64 = kG * kG * 2;       // 64 x 64 bf16 plane: 8 KB
constexpr uint32_t kPl128 = 128 * kG * 2;     // 128 x 64 bf16 plane: 16 KB
// shared memory (1024-byte aligned base)
constexpr uint32_t kNT = 3;                         // T buffers
constexpr uint32_t kNF = 2;                         // F buffers
constexpr uint32_t kNU = 2;                         // U buffers
constexpr uint32_t kOffU = 0;                       // 2 x (U hi, U lo) MN-major: 64 KB
constexpr uint32_t kOffT = kOffU + 2 * kNU * kPl128; // 3 x (T hi, T lo): 48 KB
constexpr uint32_t kOffF = kOffT + 2 * kNT * kPl64; // 2 x (F hi, F lo): 32 KB
constexpr uint32_t kOffA = kOffF + 2 * kNF * kPl64; // 2 x (R^T hi, R^T lo): 64 KB
constexpr uint32_t kOffP = kOffA + 4 * kPl128;      // P one-hot: 16 KB
constexpr uint32_t kOffBar = kOffP + kPl128;        // mbarriers, tensor-memory slot
constexpr int kNumBars = 36;
constexpr uint32_t kOffIsq = kOffBar + 8 * kNumBars + 16;  // floor(sqrt(v)), v <= R_F^2
constexpr uint32_t kSmemBytes = kOffIsq + 1024 + 1024;     // isq (R_F <= 31) + alignment
constexpr uint32_t kTmemCols = 256;

// one box of a launch (single boxes: the only one, from the kernel parameters; batches:
// a table in global memory, boxes in unit order)
struct SBox {
  int R, RF, Mg, S;
  long long unit0;  // first work unit (units of a box: pair-major, node-minor)
  long long fr0;    // FR / F / T planes: node s of the box at plane row (fr0 / 64) + 64 s
  long long w0;     // w: node s at w0 + s
  long long part0;  // part: pair p, segment k at part0 + (p * maxseg + k) * 128 * 64
  int maxseg, pad;
};

struct Args {
  const SBox* boxes;  // batches: nbox entries; single boxes: nullptr (b0 is used)
  SBox b0;
  const long long* cta0;  // batches: first unit of CTA c at cta0[c] (grid + 1 entries)
  int nbox, units, rf_max;
  const uint32_t* FR;  // [nodes][64][64] F_s[a][h] as bf16 hi (low half) | lo (high half)
  const float* w;      // [nodes]
  float* part;         // partial E of a slab pair: [128][64] per (pair, segment)
  int* err;
  int stall_test;
};

// the CTA that owns unit u: an equal split of the units, or the table of CTA starts
__host__ __device__ inline int owner_of(long long u, const long long* cta0, int units, int grid) {
  if (!cta0) return owner_cta(u, units, grid);
  int lo = 0, hi = grid - 1;  // last c with cta0[c] <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta0[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the box of a role's current unit; batches walk the table forward as units increase
template <bool kBatch>
struct BoxCursor {
  SBox X;
  int b = 0;
  long long next = 0;
  __device__ __forceinline__ void init(const Args& g, long long u) {
    if constexpr (kBatch) {
      int lo = 0, hi = g.nbox - 1;  // last box with unit0 <= u
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.boxes[mid].unit0 <= u) lo = mid;
        else hi = mid - 1;
      }
      b = lo;
      X = g.boxes[b];
      next = b + 1 < g.nbox ? g.boxes[b + 1].unit0 : 0x7fffffffffffffffll;
    } else {
      X = g.b0;
      next = 0x7fffffffffffffffll;
    }
  }
  // true when u starts a new box
  __device__ __forceinline__ bool advance(const Args& g, long long u) {
    if constexpr (kBatch) {
      if (u < next) return false;
      while (b + 1 < g.nbox && g.boxes[b + 1].unit0 <= u) ++b;
      X = g.boxes[b];
      next = b + 1 < g.nbox ? g.boxes[b + 1].unit0 : 0x7fffffffffffffffll;
      return true;
    } else {
      return false;
    }
  }
};

// place of a unit in its box: node s and slab pair p (a box's units are pair-major,
// node-minor), stepped from unit to unit without a 64-bit division in the loops
struct UnitPos {
  int s = 0, p = 0;
  __device__ __forceinline__ void set(long long loc, int S) {
    p = (int)(loc / S);
    s = (int)(loc - (long long)p * S);
  }
  __device__ __forceinline__ void step(int S) {
    if (++s == S) {
      s = 0;
      ++p;
    }
  }
  // the place of unit u: the box cursor moved to u (set at a new box), else one step on
  template <bool kBatch>
  __device__ __forceinline__ void next(BoxCursor<kBatch>& C, const Args& g, long long u,
                                       long long u0, bool* new_box = nullptr) {
    const bool nb = C.advance(g, u);
    if (new_box) *new_box = nb;
    if (nb) set(u - C.X.unit0, C.X.S);
    else if (u != u0) step(C.X.S);
  }
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_k, float hi_k) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo_f(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// MN-major 128-byte-swizzle descriptor: atoms of 64 M elements x 8 K rows (1 KB), atoms
// along K 1 KB apart (stride byte offset), the two 64-row M blocks 8 KB apart (leading
// byte offset)
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(8192 >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// D += A B + A B2 with A and both B in shared memory (A exact in 16 bits), warp-converged
__device__ __forceinline__ void mma_x2_ss_w(uint32_t tmem_d, uint64_t a, uint64_t b, uint64_t db,
                                            uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p, t, e;\n .reg .b64 b1;\n setp.ne.b32 p, %4, 0;\n"
      " setp.eq.u32 t, 0, 0;\n add.u64 b1, %2, %5;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, b1, %3, t;\n}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum), "l"(db)
      : "memory");
}

// kX1: hi * hi products only (no lo-plane correction; a diagnostic of single boxes)
template <bool kPeriodic, bool kBatch, bool kX1>
__global__ void __launch_bounds__(kThreads, 1)
    k_tcs(const __grid_constant__ CUtensorMap mTh, const __grid_constant__ CUtensorMap mTl,
          const __grid_constant__ CUtensorMap mFh, const __grid_constant__ CUtensorMap mFl,
          Args g) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gb = smem_raw + (base - raw);
  const uint8_t* isq = gb + kOffIsq;
  const uint32_t bar = base + kOffBar;
  auto ffull = [&](int k) { return bar + 8u * (0 + k); };    // 0, 1, 2 (F buffer k)
  auto ffree = [&](int k) { return bar + 8u * (3 + k); };    // 3, 4, 5
  auto afull = [&](int k) { return bar + 8u * (6 + k); };    // 6, 7
  auto afree = [&](int k) { return bar + 8u * (8 + k); };    // 8, 9
  auto d1full = [&](int k) { return bar + 8u * (10 + k); };  // 10, 11
  auto d1free = [&](int k) { return bar + 8u * (12 + k); };  // 12, 13
  auto ufull = [&](uint32_t k) { return bar + 8u * (31 + k); };  // 31, 32 (U buffer k)
  auto ufree = [&](uint32_t k) { return bar + 8u * (33 + k); };  // 33, 34
  const uint32_t efull = bar + 8u * 16, edone = bar + 8u * 17;
  const uint32_t pfull = bar + 8u * 18, pfree = bar + 8u * 19;
  const uint32_t never = bar + 8u * 20, drain = bar + 8u * 21, drain2 = bar + 8u * 35;
  auto tfull = [&](int k) { return bar + 8u * (22 + k); };   // 22 .. 25 (T buffer k)
  auto tfree = [&](int k) { return bar + 8u * (26 + k); };   // 26 .. 29
  const uint32_t zbar = bar + 8u * 30;  // builders: an R^T buffer is cleared for a new box
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gb + kOffBar + 8 * kNumBars);
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    s_abort = 0;
    for (int k = 0; k < (int)kNT; ++k) {
      mbar_init(tfull(k), 1);
      mbar_init(tfree(k), 1);
    }
    for (int k = 0; k < (int)kNF; ++k) {
      mbar_init(ffull(k), 1);
      mbar_init(ffree(k), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(afull(k), kBldWarps);
      mbar_init(afree(k), 1);
      mbar_init(d1full(k), 1);
      mbar_init(d1free(k), kEpiWarps);
    }
    for (int k = 0; k < (int)kNU; ++k) {
      mbar_init(ufull(k), kEpiWarps);
      mbar_init(ufree(k), 1);
    }
    mbar_init(efull, 1);
    mbar_init(edone, kEpiWarps);
    mbar_init(pfull, kBldWarps);
    mbar_init(pfree, 1);
    mbar_init(never, 1);
    mbar_init(drain, 1);
    mbar_init(drain2, 1);
    mbar_init(zbar, kBldWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int v = tid; v <= g.rf_max * g.rf_max; v += kThreads) {
    int h = (int)sqrtf((float)v);
    while (h * h > v) --h;
    while ((h + 1) * (h + 1) <= v) ++h;
    gb[kOffIsq + v] = (uint8_t)h;
  }
  // R^T operands start all zero (builders only ever write the band of the current box and
  // clear a buffer when a new box starts using it), and so do the U operands (the epilogue
  // writes every K index of the band it reads)
  for (uint32_t o = 16u * tid; o < 4 * kPl128; o += 16u * kThreads)
    *reinterpret_cast<uint4*>(gb + kOffA + o) = make_uint4(0u, 0u, 0u, 0u);
  for (uint32_t o = 16u * tid; o < 2 * kNU * kPl128; o += 16u * kThreads)
    *reinterpret_cast<uint4*>(gb + kOffU + o) = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const long long u0 =
      g.cta0 ? g.cta0[blockIdx.x] : (long long)blockIdx.x * g.units / gridDim.x;
  const long long u1 =
      g.cta0 ? g.cta0[blockIdx.x + 1] : (long long)(blockIdx.x + 1) * g.units / gridDim.x;
  // the band [zs, ze) of y, y' and z of box X in 16-aligned K steps
  auto band_lo = [](const SBox& X) { return (X.R - X.RF) & ~15; };
  auto band_hi = [](const SBox& X) {
    const int e = (X.R + X.RF + 16) & ~15;
    return e < kG ? e : kG;
  };

  if (warp == kProdWarp) {
    if (lane == 0) {
      // ---------------- TMA producer: T_s hi + lo into T buffer (unit % 4), F_s hi + lo
      // (periodic) into F buffer (unit % 3)
      BoxCursor<kBatch> C;
      UnitPos P;
      if (u0 < u1) {
        C.init(g, u0);
        P.set(u0 - C.X.unit0, C.X.S);
      }
      uint32_t n = 0;
      for (long long u = u0; u < u1 && !s_abort; ++u, ++n) {
        P.next(C, g, u, u0);
        const int s = P.s, kt = (int)(n % kNT), kf = (int)(n % kNF);
        const int row = (int)(C.X.fr0 / kG) + s * kG;
        if (!mbar_wait(tfree(kt), ((n / kNT) & 1u) ^ 1u, g.err, 41, &s_abort)) {
          s_abort = 1;
          break;
        }
        const uint32_t dt = base + kOffT + kt * 2 * kPl64;
        mbar_expect_tx(tfull(kt), 2 * kPl64);
        tma_load_2d(dt, &mTh, 0, row, tfull(kt));
        tma_load_2d(dt + kPl64, &mTl, 0, row, tfull(kt));
        if (kPeriodic) {
          if (!mbar_wait(ffree(kf), ((n / kNF) & 1u) ^ 1u, g.err, 41, &s_abort)) {
            s_abort = 1;
            break;
          }
          const uint32_t df = base + kOffF + kf * 2 * kPl64;
          mbar_expect_tx(ffull(kf), 2 * kPl64);
          tma_load_2d(df, &mFh, 0, row, ffull(kf));
          tma_load_2d(df + kPl64, &mFl, 0, row, ffull(kf));
        }
      }
      // copies still in flight land before the CTA leaves
      for (uint32_t m = n > kNT ? n - kNT : 0; m < n; ++m)
        mbar_wait(tfull(m % kNT), (m / kNT) & 1u, g.err, 42, nullptr, 100000000ull);
      if (kPeriodic)
        for (uint32_t m = n > kNF ? n - kNF : 0; m < n; ++m)
          mbar_wait(ffull(m % kNF), (m / kNF) & 1u, g.err, 42, nullptr, 100000000ull);
    }
  } else if (warp == kMmaWarp || warp == kMma2Warp) {
    // ---------------- MMA issuers: warp 15 issues MMA1, warp 16 MMA2, so that neither
    // product waits for the other's issue (whole warps; every wait result warp-uniform)
    auto all = [](bool v) { return __all_sync(0xffffffffu, v); };
    constexpr uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 4) << 24);
    if (warp == kMmaWarp && g.stall_test &&
        !all(mbar_wait(never, 0, g.err, 5, nullptr, 20000000ull)))
      s_abort = 1;
    const uint64_t dP = sdesc(base + kOffP);
    // K steps and N of the box of each MMA (unit i's box for MMA1, i - 1's for MMA2)
    struct Geo {
      int ms, me, nh;
      uint32_t idesc1, idesc2;
    };
    auto geo = [&](const SBox& X) {
      Geo q;
      q.ms = band_lo(X) >> 4;
      q.me = band_hi(X) >> 4;
      q.nh = (X.RF + 16) >> 4;  // K steps of h in the A term
      const uint32_t N2 = (uint32_t)((X.Mg + 15) & ~15);
      q.idesc1 = idesc0 | ((N2 >> 3) << 17);              // A, B K-major
      q.idesc2 = idesc0 | (1u << 15) | ((N2 >> 3) << 17);  // A MN-major
      return q;
    };
    auto mma1 = [&](uint32_t i, const Geo& q) {
      const uint32_t k = i & 1u, d = tmem + 64u * k;
      const uint64_t dA = sdesc(base + kOffA + k * 2 * kPl128);
      const uint64_t dT = sdesc(base + kOffT + (i % kNT) * 2 * kPl64);
#pragma unroll 1
      for (int m = q.ms; m < q.me; ++m) {
        if constexpr (kX1) mma_x1_w(d, dA + 2u * m, dT + 2u * m, q.idesc1, m > q.ms ? 1u : 0u);
        else mma_x3_w(d, dA + 2u * m, dT + 2u * m, kPl128 >> 4, kPl64 >> 4, q.idesc1,
                      m > q.ms ? 1u : 0u);
      }
      if constexpr (kPeriodic) {
        const uint64_t dF = sdesc(base + kOffF + (i % kNF) * 2 * kPl64);
#pragma unroll 1
        for (int m = 0; m < q.nh; ++m) {
          if constexpr (kX1) mma_x1_w(d, dP + 2u * m, dF + 2u * m, q.idesc1, 1u);
          else mma_x2_ss_w(d, dP + 2u * m, dF + 2u * m, kPl64 >> 4, q.idesc1, 1u);
        }
      }
    };
    auto mma2 = [&](uint32_t i, bool first, const Geo& q) {
      const uint64_t dU = sdesc_mn(base + kOffU + (i % kNU) * 2 * kPl128);
      const uint64_t dT = sdesc(base + kOffT + (i % kNT) * 2 * kPl64);
#pragma unroll 1
      for (int m = q.ms; m < q.me; ++m) {
        const uint32_t acc = (first && m == q.ms) ? 0u : 1u;
        if constexpr (kX1) mma_x1_w(tmem + 128u, dU + 128u * m, dT + 2u * m, q.idesc2, acc);
        else mma_x3_w(tmem + 128u, dU + 128u * m, dT + 2u * m, kPl128 >> 4, kPl64 >> 4,
                      q.idesc2, acc);
      }
    };
    bool ok = all(!s_abort);
    uint32_t pc = 0, segc = 0;
    BoxCursor<kBatch> C;
    UnitPos P;
    if (u0 < u1) {
      C.init(g, u0);
      P.set(u0 - C.X.unit0, C.X.S);
    }
    Geo q = geo(C.X);
    uint32_t i = 0;
    if (warp == kMmaWarp) {
      for (long long u = u0; u < u1 && ok; ++u, ++i) {
        bool nbox = false;
        P.next(C, g, u, u0, &nbox);
        if (nbox) q = geo(C.X);
        const bool first = u == u0 || P.s == 0;
        const bool last = u + 1 == u1 || P.s + 1 == C.X.S;
        // MMA1(i): the operands are usually ready by now, so all of them are first tested
        // together (independent test_waits, no chain of dependent waits), and only what is
        // not ready is waited for
        const bool ready1 =
            all(mbar_test(tfull(i % kNT), (i / kNT) & 1u) &
                (!kPeriodic || mbar_test(ffull(i % kNF), (i / kNF) & 1u)) &
                mbar_test(afull(i & 1u), (i >> 1) & 1u) &
                (!first || !kPeriodic || mbar_test(pfull, pc & 1u)) &
                (i < 2 || mbar_test(d1free(i & 1u), ((i >> 1) & 1u) ^ 1u)));
        if (!ready1)
          ok = all(mbar_wait(tfull(i % kNT), (i / kNT) & 1u, g.err, 43, &s_abort) &&
                   (!kPeriodic || mbar_wait(ffull(i % kNF), (i / kNF) & 1u, g.err, 43, &s_abort)) &&
                   mbar_wait(afull(i & 1u), (i >> 1) & 1u, g.err, 44, &s_abort) &&
                   (!first || !kPeriodic || mbar_wait(pfull, pc & 1u, g.err, 45, &s_abort)) &&
                   (i < 2 || mbar_wait(d1free(i & 1u), ((i >> 1) & 1u) ^ 1u, g.err, 46, &s_abort)));
        if (!ok) break;
        if (first) ++pc;
        tc_fence_after();
        mma1(i, q);
        mma_commit_w(afree(i & 1u));
        if (kPeriodic) mma_commit_w(ffree(i % kNF));
        mma_commit_w(d1full(i & 1u));
        if (last && kPeriodic) mma_commit_w(pfree);
      }
      if (!ok) s_abort = 1;
      mma_commit_w(drain);
      mbar_wait(drain, 0, g.err, 49, nullptr, 100000000ull);
    } else {
      // MMA2(i) once the epilogue has written U(i) (which follows MMA1(i)); T(i) is free
      // when MMA2(i) completes, since MMA1(i) completed before U(i) was written
      for (long long u = u0; u < u1 && ok; ++u, ++i) {
        bool nbox = false;
        P.next(C, g, u, u0, &nbox);
        if (nbox) q = geo(C.X);
        const bool first = u == u0 || P.s == 0;
        const bool last = u + 1 == u1 || P.s + 1 == C.X.S;
        const bool ready2 = all(mbar_test(ufull(i % kNU), (i / kNU) & 1u) &
                                (!first || segc == 0 || mbar_test(edone, (segc - 1) & 1u)));
        if (!ready2)
          ok = all(mbar_wait(ufull(i % kNU), (i / kNU) & 1u, g.err, 47, &s_abort) &&
                   (!first || segc == 0 ||
                    mbar_wait(edone, (segc - 1) & 1u, g.err, 48, &s_abort)));
        if (!ok) break;
        tc_fence_after();
        mma2(i, first, q);
        mma_commit_w(ufree(i % kNU));
        mma_commit_w(tfree(i % kNT));
        if (last) {
          mma_commit_w(efull);
          ++segc;
        }
      }
      if (!ok) s_abort = 1;
      mma_commit_w(drain2);
      mbar_wait(drain2, 0, g.err, 49, nullptr, 100000000ull);
    }
  } else if (warp >= kEpiWarps) {
    // ---------------- R^T and P builders (warps 8-10, 12-14)
    // R^T[(j, z)][y'] = F_s[x_j][h(y', z)]: rows z and 2R - z are equal, so a task forms one
    // 16-byte chunk (8 consecutive y') of a row z <= R for both slabs j and stores it into
    // the mirror rows too.
    // The h values of a task are fixed for a box; the row of F_s comes from one register per
    // lane (h = lane; R_F <= 31) by shuffles.
    const int bw = warp < kProdWarp ? warp - kEpiWarps : warp - kEpiWarps - 1;
    const int bt = 32 * bw + lane;
    constexpr int kMaxTasks = 2;  // (R_F + 1 rows, halved by the mirror) 8 chunks <= 256
    uint32_t hb[kMaxTasks][2];
    int zlo = 0, nzh = 0, clo = 0, nc = 0, tasks = 0;
    auto setup = [&](const SBox& X) {
      zlo = X.R - X.RF;
      nzh = X.RF + 1;
      clo = (X.R - X.RF) >> 3;
      nc = ((X.R + X.RF) >> 3) - clo + 1;
      tasks = nzh * nc;
#pragma unroll
      for (int k = 0; k < kMaxTasks; ++k) {
        const int t = bt + k * kBldThreads;
        hb[k][0] = hb[k][1] = 0xffffffffu;
        if (t < tasks) {
          const int z = zlo + t / nc, c = clo + t % nc, dz = z - X.R;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int dy = 8 * c + e - X.R;
            const int q = X.RF * X.RF - dy * dy - dz * dz;
            const uint32_t h = q >= 0 ? (uint32_t)isq[q] : 0xffu;
            hb[k][e >> 2] = (hb[k][e >> 2] & ~(0xffu << (8 * (e & 3)))) | (h << (8 * (e & 3)));
          }
        }
      }
    };
    BoxCursor<kBatch> C, Cn;  // the box of this unit and of the next (F rows loaded ahead)
    UnitPos P, Pn;
    if (u0 < u1) {
      C.init(g, u0);
      Cn.init(g, u0);
      P.set(u0 - C.X.unit0, C.X.S);
      Pn = P;
      setup(C.X);
    }
    auto frow = [&](const SBox& X, const UnitPos& Q, int j) {
      return g.FR + X.fr0 + ((long long)Q.s * kG + 2 * Q.p + j) * kHMax;
    };
    uint32_t nf0 = 0, nf1 = 0;
    if (u0 < u1) {
      nf0 = __ldg(frow(C.X, P, 0) + lane);
      nf1 = __ldg(frow(C.X, P, 1) + lane);
    }
    int abox[2] = {0, 0};  // the box each R^T buffer was last built for (zero at start)
    if (kBatch && u0 < u1) abox[0] = abox[1] = C.b;
    uint32_t pc = 0, i = 0, zc = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u, ++i) {
      bool nbox = false;
      P.next(C, g, u, u0, &nbox);
      if (nbox) setup(C.X);
      const bool first = u == u0 || P.s == 0;
      const uint32_t f0 = nf0, f1 = nf1;
      if (u + 1 < u1) {
        Pn = P;
        Pn.next(Cn, g, u + 1, u0);
        nf0 = __ldg(frow(Cn.X, Pn, 0) + lane);
        nf1 = __ldg(frow(Cn.X, Pn, 1) + lane);
      }
      if (kPeriodic && first) {
        // P_j[z][h] = [h(x_j, z) = h] for the pair of u: row r = 64 j + z, one thread a row
        if (pc > 0) ok = mbar_wait(pfree, (pc - 1) & 1u, g.err, 51, &s_abort);
        if (!ok) break;
        if (bt < 128) {
          const int j = bt >> 6, z = bt & 63;
          const int dx = 2 * P.p + j - C.X.R, dz = z - C.X.R;
          const int q = C.X.RF * C.X.RF - dx * dx - dz * dz;
          const int h = q >= 0 ? (int)isq[q] : -1;
          uint8_t* row = gb + kOffP + bt * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (h >= 0 && (h >> 3) == c) {
              const uint32_t one = 0x3F80u << (16 * (h & 1)), wi = (uint32_t)(h & 7) >> 1;
              v = make_uint4(wi == 0 ? one : 0u, wi == 1 ? one : 0u, wi == 2 ? one : 0u,
                             wi == 3 ? one : 0u);
            }
            *reinterpret_cast<uint4*>(row + ((c ^ (bt & 7)) << 4)) = v;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(pfull);
        ++pc;
      }
      ok = mbar_wait(afree(i & 1u), ((i >> 1) & 1u) ^ 1u, g.err, 52, &s_abort);
      if (!ok) break;
      uint8_t* A = gb + kOffA + (i & 1u) * 2 * kPl128;
      if (kBatch && abox[i & 1u] != C.b) {
        // a new box in this buffer: clear what the previous box's band left, and let no
        // builder write its chunks before every builder has finished clearing
        for (uint32_t o = 16u * bt; o < 2 * kPl128; o += 16u * kBldThreads)
          *reinterpret_cast<uint4*>(A + o) = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        if (lane == 0) mbar_arrive(zbar);
        ok = mbar_wait(zbar, zc & 1u, g.err, 53, &s_abort);
        ++zc;
        if (!ok) break;
        abox[i & 1u] = C.b;
      }
#pragma unroll
      for (int k = 0; k < kMaxTasks; ++k) {
        const int t = bt + k * kBldThreads;
        if (k * kBldThreads >= tasks) break;  // warp-uniform
        // every lane shuffles (the source lane is its h); idle lanes use h = 0.  The h of a
        // chunk does not depend on the slab, so one task fills the chunk in both slabs' rows.
        uint32_t v0[8], v1[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint32_t h = (hb[k][e >> 2] >> (8 * (e & 3))) & 0xffu;
          const uint32_t a = __shfl_sync(0xffffffffu, f0, (int)(h & 31u));
          const uint32_t b = __shfl_sync(0xffffffffu, f1, (int)(h & 31u));
          v0[e] = h == 0xffu ? 0u : a;
          v1[e] = h == 0xffu ? 0u : b;
        }
        if (t < tasks) {
          const int z = zlo + t / nc, c = clo + t % nc;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint32_t* v = j ? v1 : v0;
            uint4 hi, lo;
            hi.x = __byte_perm(v[0], v[1], 0x5410);
            hi.y = __byte_perm(v[2], v[3], 0x5410);
            hi.z = __byte_perm(v[4], v[5], 0x5410);
            hi.w = __byte_perm(v[6], v[7], 0x5410);
            lo.x = __byte_perm(v[0], v[1], 0x7632);
            lo.y = __byte_perm(v[2], v[3], 0x7632);
            lo.z = __byte_perm(v[4], v[5], 0x7632);
            lo.w = __byte_perm(v[6], v[7], 0x7632);
            const int r = 64 * j + z, rm = 64 * j + 2 * C.X.R - z;
            const uint32_t off = (uint32_t)r * 128u + ((uint32_t)((c & 7) ^ (r & 7)) << 4);
            *reinterpret_cast<uint4*>(A + off) = hi;
            *reinterpret_cast<uint4*>(A + off + kPl128) = lo;
            if (rm != r) {
              const uint32_t offm = (uint32_t)rm * 128u + ((uint32_t)((c & 7) ^ (rm & 7)) << 4);
              *reinterpret_cast<uint4*>(A + offm) = hi;
              *reinterpret_cast<uint4*>(A + offm + kPl128) = lo;
            }
          }
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(afull(i & 1u));
    }
    if (!ok) s_abort = 1;
  } else {
    // ---------------- epilogue warps 0-7: lanes (j, z) of D1 (and (j, y) of E), 32 columns
    const int quad = warp & 3, half = warp >> 2;
    const int j = quad >> 1, zr = 32 * (quad & 1) + lane;  // D1 row (j, z = zr)
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    BoxCursor<kBatch> C;
    UnitPos P;
    if (u0 < u1) {
      C.init(g, u0);
      P.set(u0 - C.X.unit0, C.X.S);
    }
    bool in_band = zr >= band_lo(C.X) && zr < band_hi(C.X);
    uint32_t i = 0, segc = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u, ++i) {
      bool nbox = false;
      P.next(C, g, u, u0, &nbox);
      if (nbox) in_band = zr >= band_lo(C.X) && zr < band_hi(C.X);
      const bool last = u + 1 == u1 || P.s + 1 == C.X.S;
      const float ws = g.w[C.X.w0 + P.s];
      ok = mbar_wait(d1full(i & 1u), (i >> 1) & 1u, g.err, 61, &s_abort);
      if (!ok) break;
      tc_fence_after();
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + 64u * (i & 1u) + 32u * half, v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(d1free(i & 1u));
      // the U buffer of unit i was last read by MMA2(i - kNU)
      ok = mbar_wait(ufree(i % kNU), ((i / kNU) & 1u) ^ 1u, g.err, 62, &s_abort);
      if (!ok) break;
      if (in_band) {
        // U[(j, y)][z] for y = 32 half + e: MN-major atom row z & 7 of K atom z >> 3 in
        // M block j, 16-byte chunk c = y >> 3 at position c ^ (z & 7)
        uint8_t* U = gb + kOffU + (i % kNU) * 2 * kPl128 + j * 8192 + (zr >> 3) * 1024 +
                     (zr & 7) * 128;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float x0 = __uint_as_float(v[8 * cc + 2 * e]) * ws;
            const float x1 = __uint_as_float(v[8 * cc + 2 * e + 1]) * ws;
            hi[e] = pack_bf16x2(x0, x1);
            lo[e] = pack_bf16x2(x0 - bf16_lo_f(hi[e]), x1 - bf16_hi_f(hi[e]));
          }
          const int c = 4 * half + cc;
          const uint32_t o = (uint32_t)((c ^ (zr & 7)) << 4);
          *reinterpret_cast<uint4*>(U + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(U + kPl128 + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(ufull(i % kNU));
      if (!last) continue;
      // the pair's E leaves tensor memory once, as a partial of this CTA
      ok = mbar_wait(efull, segc & 1u, g.err, 63, &s_abort);
      if (!ok) break;
      tc_fence_after();
      const long long p = P.p;
      const int kseg =
          (int)blockIdx.x - owner_of(C.X.unit0 + p * C.X.S, g.cta0, g.units, gridDim.x);
      tmem_ld32(tmem + lane_off + 128u + 32u * half, v);
      float4* o = reinterpret_cast<float4*>(
          g.part + C.X.part0 + ((p * C.X.maxseg + kseg) * 128 + 32 * quad + lane) * (long long)kG +
          32 * half);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        o[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                           __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(edone);
      ++segc;
    }
    if (!ok) s_abort = 1;
  }
  tc_fence_before();
  __syncthreads();
  signal_finalizer();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// F_s window sums (FP64) of every row a < 64: packed bf16 hi | lo pairs for the builders,
// and planar bf16 hi / lo [s][a][h] for the A-term MMA.  One thread per (s, a).
__global__ void k_tcs_prep(const double* Tm, int S, int Mg, int R, int RF, int periodic,
                           uint32_t* FR, __nv_bfloat16* Fh, __nv_bfloat16* Fl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * kG) return;
  const int s = i / kG, a = i % kG;
  const double* row = Tm + ((long long)s * Mg + (a < Mg ? a : 0)) * Mg;
  auto X = [&](int k) { return (periodic && k == a) ? 0.0 : row[k]; };
  double acc = 0.0;
  for (int h = 0; h < kHMax; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? X(R) : X(R - h) + X(R + h);
      f = acc;
    }
    const __nv_bfloat16 hb = __double2bfloat16(f);
    const __nv_bfloat16 lb = __double2bfloat16(f - (double)__bfloat162float(hb));
    FR[(long long)i * kHMax + h] = (uint32_t)__bfloat16_as_ushort(hb) |
                                   ((uint32_t)__bfloat16_as_ushort(lb) << 16);
    Fh[(long long)i * kHMax + h] = hb;
    Fl[(long long)i * kHMax + h] = lb;
  }
}

// T_s as bf16 hi + lo planes padded to 64 x 64
__global__ void k_tcs_tplanes(const double* Tm, int S, int Mg, __nv_bfloat16* hi,
                              __nv_bfloat16* lo) {
  const long long n = (long long)S * kG * kG;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / (kG * kG)), a = (int)((i / kG) % kG), c = (int)(i % kG);
    const double t = (a < Mg && c < Mg) ? Tm[((long long)s * Mg + a) * Mg + c] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16_rn((float)t);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn((float)t - __bfloat162float(h));
  }
}

// window sums of Dbar (I x I x Dbar term), FB[h][z'] = sum_{k=R-h}^{R+h} Dbar[z'][k]
__global__ void k_tcs_dbar(const double* Dbar, int Mg, int R, int RF, float* FB) {
  const int a = threadIdx.x;
  double acc = 0.0;
  for (int h = 0; h < kHMax; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? Dbar[a * Mg + R] : Dbar[a * Mg + R - h] + Dbar[a * Mg + R + h];
      f = acc;
    }
    FB[h * kG + a] = (float)f;
  }
}

// batches: one block per slab (box, x), eight warps over the rows y, two z per lane; the
// block's FP64 sum of eps over the Fermi sphere (rows in order, then warps in order), and the
// last block of a box (ticket) adds its slab sums in order into the box's E_x
struct FBox {
  int R, RF, Mg, S, maxseg, slab0;
  long long unit0, part0, eps_off;
  double pref;
};

__global__ void __launch_bounds__(256)
    k_tcsb_finalize(const FBox* __restrict__ boxes, const int* __restrict__ slab_box,
                    const long long* cta0, const float* part, const float* FB, int units,
                    int grid, float* eps, double* slab_ex, unsigned* ticket, double* Ex) {
  const int gx = blockIdx.x, b = slab_box[gx];
  const FBox X = boxes[b];
  const int x = gx - X.slab0, Mg = X.Mg, R = X.R, RF = X.RF;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = x >> 1, j = x & 1;
  const int c0 = owner_of(X.unit0 + (long long)p * X.S, cta0, units, grid);
  const int nseg = owner_of(X.unit0 + (long long)(p + 1) * X.S - 1, cta0, units, grid) - c0 + 1;
  const int dx = x - R;
  double wacc = 0.0;
  for (int y = warp; y < Mg; y += 8) {
    const int dy = y - R;
    const int qb = RF * RF - dx * dx - dy * dy;
    const float* fb = qb >= 0 ? FB + (long long)b * kG * kHMax + isqrt_int(qb) * kG : nullptr;
    const float* pp = part + X.part0 + ((long long)p * X.maxseg * 128 + 64 * j + y) * kG;
    double acc = 0.0;
#pragma unroll
    for (int k2 = 0; k2 < 2; ++k2) {
      const int z = lane + 32 * k2;
      if (z >= Mg) continue;
      float sum = 0.0f;
      for (int k = 0; k < nseg; ++k) sum += __ldg(pp + (long long)k * 128 * kG + z);
      if (fb) sum += __ldg(fb + z);
      const int dz = z - R, m = dx * dx + dy * dy + dz * dz;
      const float v = m <= R * R ? (float)(-X.pref * (double)sum) : 0.0f;
      eps[X.eps_off + ((long long)x * Mg + y) * Mg + z] = v;
      if (m <= RF * RF) acc += (double)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    wacc += acc;
  }
  __shared__ double s_w[8];
  __shared__ bool s_last;
  if (lane == 0) s_w[warp] = wacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += s_w[k];
    slab_ex[gx] = t;
    __threadfence();
    s_last = atomicAdd(ticket + b, 1u) == (unsigned)(Mg - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double tot = 0.0;
  for (int k = 0; k < Mg; ++k) tot += __ldcg(slab_ex + X.slab0 + k);
  Ex[2 * b] = 0.5 * tot;
  Ex[2 * b + 1] = tot;
  ticket[b] = 0u;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

cc_status set_smem_attrs() {
  static bool done = false;
  if (done) return CC_OK;
  const void* ks[] = {(const void*)k_tcs<true, false, false>, (const void*)k_tcs<false, false, false>,
                      (const void*)k_tcs<true, false, true>, (const void*)k_tcs<false, false, true>,
                      (const void*)k_tcs<true, true, false>};
  for (const void* k : ks)
    CC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  done = true;
  return CC_OK;
}

// the largest number of CTAs that one slab pair's units are spread over
int max_segments(long long unit0, int pairs, int S, int units, int grid,
                 const long long* cta0 = nullptr) {
  int m = 1;
  for (int p = 0; p < pairs; ++p) {
    const int c0 = owner_of(unit0 + (long long)p * S, cta0, units, grid);
    const int c1 = owner_of(unit0 + (long long)(p + 1) * S - 1, cta0, units, grid);
    m = std::max(m, c1 - c0 + 1);
  }
  return m;
}

}  // namespace

struct TcSmallWs {
  int grid = 0, units = 0, maxseg = 0, RF_built = -1;
  uint32_t* FR = nullptr;
  void* F[2] = {nullptr, nullptr};
  void* T[2] = {nullptr, nullptr};
  float* FB = nullptr;
  float* part = nullptr;
  double* blk_ex = nullptr;
  float* w32 = nullptr;
  unsigned* ticket = nullptr;
  alignas(64) unsigned char map_th[128], map_tl[128], map_fh[128], map_fl[128];
  std::vector<void*> allocs;
};

bool tc_small_supported(cc_tables t) { return t->Mg <= kG; }

void tc_small_free(void* p) {
  TcSmallWs* w = reinterpret_cast<TcSmallWs*>(p);
  if (!w) return;
  for (void* a : w->allocs) cudaFree(a);
  delete w;
}

cc_status tc_small_alloc(cc_tables t, void** out) {
  *out = nullptr;
  if (!tc_small_supported(t)) return CC_OK;
  CC_TRY(set_smem_attrs());
  TcSmallWs* w = new (std::nothrow) TcSmallWs();
  if (!w) return CC_ERR_ALLOC;
  const int S = t->S_eff, pairs = (t->Mg + 1) / 2;
  w->units = pairs * S;
  w->grid = std::min(sm_count(), w->units);
  w->maxseg = max_segments(0, pairs, S, w->units, w->grid);
  auto alloc = [&](void** p, size_t bytes) -> cc_status {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      set_last_error("cudaMalloc(small-grid tensor-core workspace)", e);
      return CC_ERR_ALLOC;
    }
    w->allocs.push_back(*p);
    t->ws.mx_bytes += bytes;
    t->device_bytes += bytes;
    return CC_OK;
  };
  const size_t plane = sizeof(__nv_bfloat16) * (size_t)S * kG * kG;
  cc_status st = CC_OK;
  if ((st = alloc((void**)&w->FR, sizeof(uint32_t) * S * kG * kHMax)) != CC_OK ||
      (st = alloc(&w->F[0], plane)) != CC_OK || (st = alloc(&w->F[1], plane)) != CC_OK ||
      (st = alloc(&w->T[0], plane)) != CC_OK || (st = alloc(&w->T[1], plane)) != CC_OK ||
      (st = alloc((void**)&w->FB, sizeof(float) * kG * kHMax)) != CC_OK ||
      (st = alloc((void**)&w->part, sizeof(float) * 128 * kG * pairs * w->maxseg)) != CC_OK ||
      (st = alloc((void**)&w->blk_ex, sizeof(double) * kG * kG)) != CC_OK ||
      (st = alloc((void**)&w->w32, sizeof(float) * S)) != CC_OK ||
      (st = alloc((void**)&w->ticket, sizeof(unsigned))) != CC_OK) {
    tc_small_free(w);
    return st;
  }
  static_assert(sizeof(CUtensorMap) <= 128, "tensor map size");
  if ((st = tc_make_map_bf16(w->map_th, w->T[0], (long long)S * kG, kG, kG)) != CC_OK ||
      (st = tc_make_map_bf16(w->map_tl, w->T[1], (long long)S * kG, kG, kG)) != CC_OK ||
      (st = tc_make_map_bf16(w->map_fh, w->F[0], (long long)S * kG, kG, kG)) != CC_OK ||
      (st = tc_make_map_bf16(w->map_fl, w->F[1], (long long)S * kG, kG, kG)) != CC_OK) {
    tc_small_free(w);
    return st;
  }
  k_tcs_tplanes<<<512, 256>>>(t->d.Tm64, S, t->Mg, (__nv_bfloat16*)w->T[0],
                              (__nv_bfloat16*)w->T[1]);
  std::vector<float> w32(S);
  for (int i = 0; i < S; ++i) w32[i] = (float)t->w[t->kept_idx[i]];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpy(w->w32, w32.data(), sizeof(float) * S, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(w->ticket, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    set_last_error("small-grid tensor-core planes", e);
    tc_small_free(w);
    return CC_ERR_CUDA;
  }
  *out = w;
  return CC_OK;
}

cc_status tc_small_run(cc_tables t, void* ws, int* err, int stall_test, int R_F, float* eps,
                       double* Ex, cudaStream_t st, int x1) {
  TcSmallWs* w = reinterpret_cast<TcSmallWs*>(ws);
  if (!w || !tc_small_supported(t) || R_F > 31) return CC_ERR_NOTSUPP;
  const int S = t->S_eff, Mg = t->Mg, R = t->p.R;
  const int periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  if (w->RF_built != R_F) {
    k_tcs_prep<<<(S * kG + 127) / 128, 128, 0, st>>>(t->d.Tm64, S, Mg, R, R_F, periodic, w->FR,
                                                      (__nv_bfloat16*)w->F[0],
                                                      (__nv_bfloat16*)w->F[1]);
    if (periodic) k_tcs_dbar<<<1, kG, 0, st>>>(t->d.Dbar64, Mg, R, R_F, w->FB);
    CC_CUDA(cudaGetLastError());
    w->RF_built = R_F;
  }
  Args a{};
  a.boxes = nullptr;
  a.b0 = SBox{R, R_F, Mg, S, 0, 0, 0, 0, w->maxseg, 0};
  a.cta0 = nullptr;
  a.nbox = 1;
  a.units = w->units;
  a.rf_max = R_F;
  a.FR = w->FR;
  a.w = w->w32;
  a.part = w->part;
  a.err = err;
  a.stall_test = stall_test;
  const CUtensorMap& th = *reinterpret_cast<const CUtensorMap*>(w->map_th);
  const CUtensorMap& tl = *reinterpret_cast<const CUtensorMap*>(w->map_tl);
  const CUtensorMap& fh = *reinterpret_cast<const CUtensorMap*>(w->map_fh);
  const CUtensorMap& fl = *reinterpret_cast<const CUtensorMap*>(w->map_fl);
  if (periodic && x1)
    k_tcs<true, false, true><<<w->grid, kThreads, kSmemBytes, st>>>(th, tl, fh, fl, a);
  else if (periodic)
    k_tcs<true, false, false><<<w->grid, kThreads, kSmemBytes, st>>>(th, tl, fh, fl, a);
  else if (x1)
    k_tcs<false, false, true><<<w->grid, kThreads, kSmemBytes, st>>>(th, tl, fh, fl, a);
  else
    k_tcs<false, false, false><<<w->grid, kThreads, kSmemBytes, st>>>(th, tl, fh, fl, a);
  CC_CUDA((launch_slab_finalize<kG, 2 * kG, true>(
      Mg, st, (const float*)w->part, (const float*)w->FB, R, R_F, S, 1, w->units, w->grid,
      w->maxseg, periodic, t->pref, eps, w->blk_ex, w->ticket, Ex, (const int*)err, err + 1)));
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

// ---------------------------------------------------------------- batches of boxes
// The work decomposition of a batch is tunable (cc_batch_tune): the order of the boxes in
// the unit sequence (as given, or by decreasing cost) and how the sequence is cut among the
// CTAs (equal unit counts, or equal estimated cost: per unit a fixed latency of about
// kUnitFixed cycles plus the MMA time, 48 cycles per 128 x 16 x N2 / 64 operand step).
constexpr double kUnitFixed = 2400.0;

struct TcSmallBatch {
  int nbox = 0, units = 0, grid = 0, rf_max = 0, slabs = 0;
  int order = 0, split = 0;  // the current plan (see above)
  std::vector<cc_tables> tabs;
  std::vector<int> R_F;
  std::vector<long long> eps_off;
  std::vector<long long> node0;  // first node of box b in the concatenated planes
  SBox* boxes = nullptr;
  FBox* fboxes = nullptr;
  int* slab_box = nullptr;
  long long* cta0 = nullptr;
  uint32_t* FR = nullptr;
  void* F[2] = {nullptr, nullptr};
  void* T[2] = {nullptr, nullptr};
  float* FB = nullptr;
  float* part = nullptr;
  size_t part_cap = 0;
  double* slab_ex = nullptr;
  float* w = nullptr;
  unsigned* ticket = nullptr;
  alignas(64) unsigned char map_th[128], map_tl[128], map_fh[128], map_fl[128];
  std::vector<void*> allocs;
};

bool tc_small_batch_supported(const std::vector<cc_tables>& tabs, const std::vector<int>& R_F) {
  for (size_t b = 0; b < tabs.size(); ++b)
    if (tabs[b]->Mg > kG || R_F[b] > 31 || tabs[b]->p.kernel != CC_KERNEL_PERIODIC) return false;
  return !tabs.empty();
}

void tc_small_batch_free(void* p) {
  TcSmallBatch* m = reinterpret_cast<TcSmallBatch*>(p);
  if (!m) return;
  for (void* a : m->allocs) cudaFree(a);
  cudaFree(m->part);
  delete m;
}

static double unit_cost(int R, int RF, int Mg) {
  const int steps = (std::min(kG, (R + RF + 16) & ~15) - ((R - RF) & ~15)) / 16;
  const int nh = (RF + 16) >> 4, N2 = (Mg + 15) & ~15;
  return kUnitFixed + 48.0 * (6 * steps + 2 * nh) * N2 / 64.0;
}

// unit sequence, CTA cuts, partial layout and finaliser tables for (order, split)
static cc_status small_batch_plan(TcSmallBatch* m, int order, int split) {
  const int nb = m->nbox;
  std::vector<int> seq(nb);
  for (int b = 0; b < nb; ++b) seq[b] = b;
  auto cost_of = [&](int b) {
    const cc_tables t = m->tabs[b];
    return unit_cost(t->p.R, m->R_F[b], t->Mg) * ((t->Mg + 1) / 2) * t->S_eff;
  };
  if (order == 1)
    std::stable_sort(seq.begin(), seq.end(), [&](int a, int b) { return cost_of(a) > cost_of(b); });
  std::vector<SBox> bx(nb);  // in unit order
  std::vector<FBox> fb(nb);  // by box index
  std::vector<double> ucost;
  long long units = 0;
  for (int k = 0; k < nb; ++k) {
    const int b = seq[k];
    const cc_tables t = m->tabs[b];
    const int pairs = (t->Mg + 1) / 2;
    bx[k] = SBox{t->p.R, m->R_F[b], t->Mg, t->S_eff, units, m->node0[b] * kG * kG,
                 m->node0[b], 0, 1, 0};
    units += (long long)pairs * t->S_eff;
    if (split == 1) ucost.push_back(unit_cost(t->p.R, m->R_F[b], t->Mg));
  }
  const int grid = (int)std::min<long long>(sm_count(), units);
  std::vector<long long> cuts(grid + 1);
  if (split == 1) {  // equal estimated cost per CTA
    double total = 0.0;
    for (int k = 0; k < nb; ++k) total += ucost[k] * (double)((bx[k].Mg + 1) / 2) * bx[k].S;
    double acc = 0.0;
    int c = 1;
    cuts[0] = 0;
    for (int k = 0; k < nb && c < grid; ++k) {
      const long long n = (long long)((bx[k].Mg + 1) / 2) * bx[k].S;
      for (long long i = 0; i < n && c < grid; ++i) {
        acc += ucost[k];
        if (acc >= total * c / grid) cuts[c++] = bx[k].unit0 + i + 1;
      }
    }
    for (; c < grid; ++c) cuts[c] = units;
    cuts[grid] = units;
    for (int c2 = 1; c2 <= grid; ++c2) cuts[c2] = std::max(cuts[c2], cuts[c2 - 1]);
  } else {
    for (int c = 0; c <= grid; ++c) cuts[c] = (long long)c * units / grid;
  }
  long long part = 0;
  std::vector<int> slab_box(m->slabs);
  std::vector<int> slab0(nb);
  for (int b = 0, sl = 0; b < nb; ++b) {
    slab0[b] = sl;
    for (int x = 0; x < m->tabs[b]->Mg; ++x) slab_box[sl++] = b;
  }
  for (int k = 0; k < nb; ++k) {
    const int b = seq[k];
    const int pairs = (bx[k].Mg + 1) / 2;
    bx[k].maxseg = max_segments(bx[k].unit0, pairs, bx[k].S, (int)units, grid, cuts.data());
    bx[k].part0 = part;
    part += (long long)pairs * bx[k].maxseg * 128 * kG;
    fb[b] = FBox{bx[k].R, bx[k].RF, bx[k].Mg, bx[k].S, bx[k].maxseg, slab0[b], bx[k].unit0,
                 bx[k].part0, m->eps_off[b], m->tabs[b]->pref};
  }
  const size_t pbytes = sizeof(float) * (size_t)part;
  if (pbytes > m->part_cap) {
    cudaFree(m->part);
    m->part = nullptr;
    m->part_cap = 0;
    if (cudaMalloc((void**)&m->part, pbytes) != cudaSuccess) {
      set_last_error("cudaMalloc(small-grid batch partials)", cudaErrorMemoryAllocation);
      return CC_ERR_ALLOC;
    }
    m->part_cap = pbytes;
  }
  m->units = (int)units;
  m->grid = grid;
  m->order = order;
  m->split = split;
  CC_CUDA(cudaMemcpy(m->boxes, bx.data(), sizeof(SBox) * nb, cudaMemcpyHostToDevice));
  CC_CUDA(cudaMemcpy(m->fboxes, fb.data(), sizeof(FBox) * nb, cudaMemcpyHostToDevice));
  CC_CUDA(cudaMemcpy(m->slab_box, slab_box.data(), sizeof(int) * m->slabs, cudaMemcpyHostToDevice));
  CC_CUDA(cudaMemcpy(m->cta0, cuts.data(), sizeof(long long) * (grid + 1), cudaMemcpyHostToDevice));
  return CC_OK;
}

cc_status tc_small_batch_create(const std::vector<cc_tables>& tabs, const std::vector<int>& R_F,
                                const std::vector<long long>& eps_off, void** out) {
  *out = nullptr;
  if (!tc_small_batch_supported(tabs, R_F)) return CC_ERR_NOTSUPP;
  CC_TRY(set_smem_attrs());
  TcSmallBatch* m = new (std::nothrow) TcSmallBatch();
  if (!m) return CC_ERR_ALLOC;
  const int nb = (int)tabs.size();
  m->nbox = nb;
  m->tabs = tabs;
  m->R_F = R_F;
  m->eps_off = eps_off;
  long long nodes = 0;
  for (int b = 0; b < nb; ++b) {
    m->node0.push_back(nodes);
    nodes += tabs[b]->S_eff;
    m->slabs += tabs[b]->Mg;
    m->rf_max = std::max(m->rf_max, R_F[b]);
  }
  auto alloc = [&](void** p, size_t bytes) -> cc_status {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      set_last_error("cudaMalloc(small-grid tensor-core batch)", e);
      return CC_ERR_ALLOC;
    }
    m->allocs.push_back(*p);
    return CC_OK;
  };
  const size_t plane = sizeof(__nv_bfloat16) * (size_t)nodes * kG * kG;
  cc_status st = CC_OK;
  if ((st = alloc((void**)&m->boxes, sizeof(SBox) * nb)) != CC_OK ||
      (st = alloc((void**)&m->fboxes, sizeof(FBox) * nb)) != CC_OK ||
      (st = alloc((void**)&m->slab_box, sizeof(int) * m->slabs)) != CC_OK ||
      (st = alloc((void**)&m->cta0, sizeof(long long) * (sm_count() + 1))) != CC_OK ||
      (st = alloc((void**)&m->FR, sizeof(uint32_t) * (size_t)nodes * kG * kHMax)) != CC_OK ||
      (st = alloc(&m->F[0], plane)) != CC_OK || (st = alloc(&m->F[1], plane)) != CC_OK ||
      (st = alloc(&m->T[0], plane)) != CC_OK || (st = alloc(&m->T[1], plane)) != CC_OK ||
      (st = alloc((void**)&m->FB, sizeof(float) * nb * kG * kHMax)) != CC_OK ||
      (st = alloc((void**)&m->slab_ex, sizeof(double) * m->slabs)) != CC_OK ||
      (st = alloc((void**)&m->w, sizeof(float) * nodes)) != CC_OK ||
      (st = alloc((void**)&m->ticket, sizeof(unsigned) * nb)) != CC_OK) {
    tc_small_batch_free(m);
    return st;
  }
  const long long rows = nodes * kG;
  if ((st = tc_make_map_bf16(m->map_th, m->T[0], rows, kG, kG)) != CC_OK ||
      (st = tc_make_map_bf16(m->map_tl, m->T[1], rows, kG, kG)) != CC_OK ||
      (st = tc_make_map_bf16(m->map_fh, m->F[0], rows, kG, kG)) != CC_OK ||
      (st = tc_make_map_bf16(m->map_fl, m->F[1], rows, kG, kG)) != CC_OK) {
    tc_small_batch_free(m);
    return st;
  }
  std::vector<float> w(nodes);
  for (int b = 0; b < nb; ++b) {
    const cc_tables t = tabs[b];
    const long long o = m->node0[b] * kG * kG;
    k_tcs_prep<<<(t->S_eff * kG + 127) / 128, 128>>>(t->d.Tm64, t->S_eff, t->Mg, t->p.R, R_F[b], 1,
                                                      m->FR + o, (__nv_bfloat16*)m->F[0] + o,
                                                      (__nv_bfloat16*)m->F[1] + o);
    k_tcs_tplanes<<<128, 256>>>(t->d.Tm64, t->S_eff, t->Mg, (__nv_bfloat16*)m->T[0] + o,
                                (__nv_bfloat16*)m->T[1] + o);
    k_tcs_dbar<<<1, kG>>>(t->d.Dbar64, t->Mg, t->p.R, R_F[b], m->FB + (long long)b * kG * kHMax);
    for (int i = 0; i < t->S_eff; ++i) w[m->node0[b] + i] = (float)t->w[t->kept_idx[i]];
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpy(m->w, w.data(), sizeof(float) * nodes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->ticket, 0, sizeof(unsigned) * nb);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_last_error("small-grid tensor-core batch planes", e);
    tc_small_batch_free(m);
    return CC_ERR_CUDA;
  }
  if ((st = small_batch_plan(m, 0, 0)) != CC_OK) {
    tc_small_batch_free(m);
    return st;
  }
  *out = m;
  return CC_OK;
}

cc_status tc_small_batch_run(void* p, int* err, float* eps, double* Ex, cudaStream_t st) {
  TcSmallBatch* m = reinterpret_cast<TcSmallBatch*>(p);
  if (!m) return CC_ERR_NOTSUPP;
  Args a{};
  a.boxes = m->boxes;
  a.cta0 = m->cta0;
  a.nbox = m->nbox;
  a.units = m->units;
  a.rf_max = m->rf_max;
  a.FR = m->FR;
  a.w = m->w;
  a.part = m->part;
  a.err = err;
  a.stall_test = 0;
  const CUtensorMap& th = *reinterpret_cast<const CUtensorMap*>(m->map_th);
  const CUtensorMap& tl = *reinterpret_cast<const CUtensorMap*>(m->map_tl);
  const CUtensorMap& fh = *reinterpret_cast<const CUtensorMap*>(m->map_fh);
  const CUtensorMap& fl = *reinterpret_cast<const CUtensorMap*>(m->map_fl);
  k_tcs<true, true, false><<<m->grid, kThreads, kSmemBytes, st>>>(th, tl, fh, fl, a);
  k_tcsb_finalize<<<m->slabs, 256, 0, st>>>(m->fboxes, m->slab_box, m->cta0, m->part, m->FB,
                                            m->units, m->grid, eps, m->slab_ex, m->ticket, Ex);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

// Times every (order, split) plan with CUDA events (median of reps runs) and keeps the
// fastest.  choice[0] = order (0 as given, 1 by decreasing cost), choice[1] = split (0 equal
// units, 1 equal estimated cost).  Writes valid sums into eps / Ex while timing.
cc_status tc_small_batch_tune(void* p, int* err, float* eps, double* Ex, int reps,
                              int* choice, float* ms_out, cudaStream_t st) {
  TcSmallBatch* m = reinterpret_cast<TcSmallBatch*>(p);
  if (!m || reps < 1) return CC_ERR_ARG;
  cudaEvent_t e0, e1;
  CC_CUDA(cudaEventCreate(&e0));
  CC_CUDA(cudaEventCreate(&e1));
  float best = -1.0f;
  int bo = 0, bs = 0;
  cc_status s = CC_OK;
  for (int order = 0; order < 2 && s == CC_OK; ++order)
    for (int split = 0; split < 2 && s == CC_OK; ++split) {
      if ((s = small_batch_plan(m, order, split)) != CC_OK) break;
      if ((s = tc_small_batch_run(m, err, eps, Ex, st)) != CC_OK) break;
      std::vector<float> t(reps);
      for (int r = 0; r < reps && s == CC_OK; ++r) {
        cudaEventRecord(e0, st);
        s = tc_small_batch_run(m, err, eps, Ex, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = CC_ERR_CUDA;
        cudaEventElapsedTime(&t[r], e0, e1);
      }
      if (s != CC_OK) break;
      std::sort(t.begin(), t.end());
      if (best < 0.0f || t[reps / 2] < best) {
        best = t[reps / 2];
        bo = order;
        bs = split;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == CC_OK) s = small_batch_plan(m, bo, bs);
  if (s != CC_OK) return s;
  if (choice) {
    choice[0] = bo;
    choice[1] = bs;
  }
  if (ms_out) *ms_out = best;
  return CC_OK;
}

}  // namespace cc
