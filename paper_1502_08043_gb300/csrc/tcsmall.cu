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
// Pipeline: the node planes (T_s, F_s), the R^T operand, D1 and the U operand are all
// double buffered, so the MMA warp issues MMA1(i), MMA2(i - 1), MMA1(i + 1), ... while the
// builders form R^T of unit i + 1 and the epilogue converts D1 of unit i.
// Tensor memory (256 columns): [0, 64) D1[0], [64, 128) D1[1], [128, 192) E.
// Warps: 0-7 epilogue (warp w: lanes 32 (w % 4) .., columns 32 (w / 4) ..), 8-10 and 12-14
// build R^T and P, 11 TMA producer, 15 MMA issuer.  Every wait is bounded (global timer);
// on expiry the error word is set, all roles stop, the MMA issuer drains its MMAs and tensor
// memory is freed before the CTA returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "tc_prims.cuh"

namespace cc {

namespace {

constexpr int kThreads = 512;
constexpr int kEpiWarps = 8;
constexpr int kBldWarps = 6;
constexpr int kBldThreads = 32 * kBldWarps;
constexpr int kProdWarp = 11;
constexpr int kMmaWarp = 15;
constexpr int kG = 64;                        // padded grid side
constexpr int kHMax = 64;                     // window half-lengths h = 0 .. R_F <= 31
constexpr uint32_t kPl64 = kG * kG * 2;       // 64 x 64 bf16 plane: 8 KB
constexpr uint32_t kPl128 = 128 * kG * 2;     // 128 x 64 bf16 plane: 16 KB
// shared memory (1024-byte aligned base)
constexpr uint32_t kOffU = 0;                       // 2 x (U hi, U lo) MN-major: 64 KB
constexpr uint32_t kOffNode = kOffU + 4 * kPl128;   // 2 x (T hi, T lo, F hi, F lo): 64 KB
constexpr uint32_t kOffA = kOffNode + 8 * kPl64;    // 2 x (R^T hi, R^T lo): 64 KB
constexpr uint32_t kOffP = kOffA + 4 * kPl128;      // P one-hot: 16 KB
constexpr uint32_t kOffBar = kOffP + kPl128;        // mbarriers, tensor-memory slot
constexpr int kNumBars = 22;
constexpr uint32_t kOffIsq = kOffBar + 8 * kNumBars + 16;  // floor(sqrt(v)), v <= R_F^2
constexpr uint32_t kSmemBytes = kOffIsq + 1024 + 1024;     // isq (R_F <= 31) + alignment
constexpr uint32_t kTmemCols = 256;

struct Args {
  int R, R_F, Mg, S, periodic;
  int units, maxseg;
  const uint32_t* FR;  // [S][64][64] F_s[a][h] as bf16 hi (low half) | lo (high half)
  const float* w;      // [S]
  float* part;         // [pairs * maxseg][128][64] partial E of a slab pair
  int* err;
  int stall_test;
};

__host__ __device__ inline int owner_cta(long long u, int units, int grid) {
  int c = (int)((u * grid) / units);
  while (c + 1 < grid && (long long)(c + 1) * units / grid <= u) ++c;
  while (c > 0 && (long long)c * units / grid > u) --c;
  return c;
}

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

template <bool kPeriodic>
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
  auto nfull = [&](int k) { return bar + 8u * k; };          // 0, 1
  auto nfree = [&](int k) { return bar + 8u * (2 + k); };    // 2, 3
  auto afull = [&](int k) { return bar + 8u * (4 + k); };    // 4, 5
  auto afree = [&](int k) { return bar + 8u * (6 + k); };    // 6, 7
  auto d1full = [&](int k) { return bar + 8u * (8 + k); };   // 8, 9
  auto d1free = [&](int k) { return bar + 8u * (10 + k); };  // 10, 11
  auto ufull = [&](int k) { return bar + 8u * (12 + k); };   // 12, 13
  auto ufree = [&](int k) { return bar + 8u * (14 + k); };   // 14, 15
  const uint32_t efull = bar + 8u * 16, edone = bar + 8u * 17;
  const uint32_t pfull = bar + 8u * 18, pfree = bar + 8u * 19;
  const uint32_t never = bar + 8u * 20, drain = bar + 8u * 21;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gb + kOffBar + 8 * kNumBars);
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = g.R, RF = g.R_F, S = g.S;
  if (tid == 0) {
    s_abort = 0;
    for (int k = 0; k < 2; ++k) {
      mbar_init(nfull(k), 1);
      mbar_init(nfree(k), 1);
      mbar_init(afull(k), kBldWarps);
      mbar_init(afree(k), 1);
      mbar_init(d1full(k), 1);
      mbar_init(d1free(k), kEpiWarps);
      mbar_init(ufull(k), kEpiWarps);
      mbar_init(ufree(k), 1);
    }
    mbar_init(efull, 1);
    mbar_init(edone, kEpiWarps);
    mbar_init(pfull, kBldWarps);
    mbar_init(pfree, 1);
    mbar_init(never, 1);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int v = tid; v <= RF * RF; v += kThreads) {
    int h = (int)sqrtf((float)v);
    while (h * h > v) --h;
    while ((h + 1) * (h + 1) <= v) ++h;
    gb[kOffIsq + v] = (uint8_t)h;
  }
  // R^T operands start all zero (builders only ever write the band), and so do the U
  // operands (the epilogue writes every K index of the band it reads)
  for (uint32_t o = 16u * tid; o < 4 * kPl128; o += 16u * kThreads) {
    *reinterpret_cast<uint4*>(gb + kOffA + o) = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(gb + kOffU + o) = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // the band [zs, ze) of y, y' and z in 16-aligned K steps
  const int zs = (R - RF) & ~15, ze0 = (R + RF + 16) & ~15, ze = ze0 < kG ? ze0 : kG;
  const long long u0 = (long long)blockIdx.x * g.units / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * g.units / gridDim.x;

  if (warp == kProdWarp) {
    if (lane == 0) {
      // ---------------- TMA producer: T_s (and F_s) hi + lo into node buffer (unit & 1)
      const uint32_t bytes = kPeriodic ? 4 * kPl64 : 2 * kPl64;
      uint32_t n = 0;
      for (long long u = u0; u < u1 && !s_abort; ++u, ++n) {
        const int s = (int)(u % S), k = (int)(n & 1u);
        if (!mbar_wait(nfree(k), ((n >> 1) & 1u) ^ 1u, g.err, 41, &s_abort)) {
          s_abort = 1;
          break;
        }
        const uint32_t dst = base + kOffNode + k * 4 * kPl64;
        mbar_expect_tx(nfull(k), bytes);
        tma_load_2d(dst, &mTh, 0, s * kG, nfull(k));
        tma_load_2d(dst + kPl64, &mTl, 0, s * kG, nfull(k));
        if (kPeriodic) {
          tma_load_2d(dst + 2 * kPl64, &mFh, 0, s * kG, nfull(k));
          tma_load_2d(dst + 3 * kPl64, &mFl, 0, s * kG, nfull(k));
        }
      }
      for (uint32_t m = n > 2 ? n - 2 : 0; m < n; ++m)
        mbar_wait(nfull(m & 1u), (m >> 1) & 1u, g.err, 42, nullptr, 100000000ull);
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer (the whole warp; every wait result made warp-uniform)
    auto all = [](bool v) { return __all_sync(0xffffffffu, v); };
    const uint32_t N2 = (uint32_t)((g.Mg + 15) & ~15);
    constexpr uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t idesc1 = idesc0 | ((N2 >> 3) << 17);              // A, B K-major
    const uint32_t idesc2 = idesc0 | (1u << 15) | ((N2 >> 3) << 17);  // A MN-major
    if (g.stall_test && !all(mbar_wait(never, 0, g.err, 5, nullptr, 20000000ull))) s_abort = 1;
    const int ms = zs >> 4, me = ze >> 4;
    const int nh = (RF + 16) >> 4;  // K steps of h in the A term
    const uint64_t dP = sdesc(base + kOffP);
    auto mma1 = [&](uint32_t i) {
      const uint32_t k = i & 1u, d = tmem + 64u * k;
      const uint32_t nb = base + kOffNode + k * 4 * kPl64;
      const uint64_t dA = sdesc(base + kOffA + k * 2 * kPl128), dT = sdesc(nb);
#pragma unroll 1
      for (int m = ms; m < me; ++m)
        mma_x3_w(d, dA + 2u * m, dT + 2u * m, kPl128 >> 4, kPl64 >> 4, idesc1, m > ms ? 1u : 0u);
      if constexpr (kPeriodic) {
        const uint64_t dF = sdesc(nb + 2 * kPl64);
#pragma unroll 1
        for (int m = 0; m < nh; ++m) mma_x2_ss_w(d, dP + 2u * m, dF + 2u * m, kPl64 >> 4, idesc1, 1u);
      }
    };
    auto mma2 = [&](uint32_t i, bool first) {
      const uint32_t k = i & 1u;
      const uint64_t dU = sdesc_mn(base + kOffU + k * 2 * kPl128);
      const uint64_t dT = sdesc(base + kOffNode + k * 4 * kPl64);
#pragma unroll 1
      for (int m = ms; m < me; ++m)
        mma_x3_w(tmem + 128u, dU + 128u * m, dT + 2u * m, kPl128 >> 4, kPl64 >> 4, idesc2,
                 (first && m == ms) ? 0u : 1u);
    };
    bool ok = all(!s_abort);
    uint32_t pc = 0, segc = 0;
    long long prev = -1;  // unit of the MMA2 still to issue
    bool prev_first = false, prev_last = false;
    uint32_t i = 0;
    for (long long u = u0; u < u1 && ok; ++u, ++i) {
      const bool first = u == u0 || u % S == 0;
      const bool last = u + 1 == u1 || (u + 1) % S == 0;
      // MMA1(i)
      ok = all(mbar_wait(nfull(i & 1u), (i >> 1) & 1u, g.err, 43, &s_abort) &&
               mbar_wait(afull(i & 1u), (i >> 1) & 1u, g.err, 44, &s_abort) &&
               (!first || !kPeriodic || mbar_wait(pfull, pc & 1u, g.err, 45, &s_abort)) &&
               (i < 2 || mbar_wait(d1free(i & 1u), ((i >> 1) & 1u) ^ 1u, g.err, 46, &s_abort)));
      if (!ok) break;
      if (first) ++pc;
      tc_fence_after();
      mma1(i);
      mma_commit_w(afree(i & 1u));
      mma_commit_w(d1full(i & 1u));
      if (last && kPeriodic) mma_commit_w(pfree);
      // MMA2(i - 1)
      if (prev >= 0) {
        const uint32_t ip = i - 1;
        ok = all(mbar_wait(ufull(ip & 1u), (ip >> 1) & 1u, g.err, 47, &s_abort) &&
                 (!prev_first || segc == 0 ||
                  mbar_wait(edone, (segc - 1) & 1u, g.err, 48, &s_abort)));
        if (!ok) break;
        tc_fence_after();
        mma2(ip, prev_first);
        mma_commit_w(ufree(ip & 1u));
        mma_commit_w(nfree(ip & 1u));
        if (prev_last) {
          mma_commit_w(efull);
          ++segc;
        }
      }
      prev = u;
      prev_first = first;
      prev_last = last;
    }
    if (ok && prev >= 0) {
      const uint32_t ip = i - 1;
      ok = all(mbar_wait(ufull(ip & 1u), (ip >> 1) & 1u, g.err, 47, &s_abort) &&
               (!prev_first || segc == 0 ||
                mbar_wait(edone, (segc - 1) & 1u, g.err, 48, &s_abort)));
      if (ok) {
        tc_fence_after();
        mma2(ip, prev_first);
        mma_commit_w(ufree(ip & 1u));
        mma_commit_w(nfree(ip & 1u));
        mma_commit_w(efull);
        ++segc;
      }
    }
    if (!ok) s_abort = 1;
    mma_commit_w(drain);
    mbar_wait(drain, 0, g.err, 49, nullptr, 100000000ull);
  } else if (warp >= kEpiWarps) {
    // ---------------- R^T and P builders (warps 8-10, 12-14)
    // R^T[(j, z)][y'] = F_s[x_j][h(y', z)]: rows z and 2R - z are equal, so a task forms one
    // 16-byte chunk (8 consecutive y') of a row z <= R and stores it into both mirror rows.
    // The h values of a task never change; the row of F_s comes from two registers per lane
    // (h < 32 and h >= 32; R_F <= 31, so only the first) by shuffles.
    const int bw = warp < kProdWarp ? warp - kEpiWarps : warp - kEpiWarps - 1;
    const int bt = 32 * bw + lane;
    const int zlo = R - RF, nzh = RF + 1;
    const int clo = (R - RF) >> 3, nc = ((R + RF) >> 3) - clo + 1;
    const int tasks = 2 * nzh * nc;  // <= 2 x 32 x 8 = 512 < 3 x 192
    constexpr int kMaxTasks = 3;
    uint32_t hb[kMaxTasks][2];
#pragma unroll
    for (int k = 0; k < kMaxTasks; ++k) {
      const int t = bt + k * kBldThreads;
      hb[k][0] = hb[k][1] = 0xffffffffu;
      if (t < tasks) {
        const int tt = t % (nzh * nc);
        const int z = zlo + tt / nc, c = clo + tt % nc, dz = z - R;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int dy = 8 * c + e - R;
          const int q = RF * RF - dy * dy - dz * dz;
          const uint32_t h = q >= 0 ? (uint32_t)isq[q] : 0xffu;
          hb[k][e >> 2] = (hb[k][e >> 2] & ~(0xffu << (8 * (e & 3)))) | (h << (8 * (e & 3)));
        }
      }
    }
    auto frow = [&](long long u, int j) {
      return g.FR + ((long long)(u % S) * kG + 2 * (u / S) + j) * kHMax;
    };
    // F rows of the next unit, loaded a unit ahead (row x_j: lane l holds h = l)
    uint32_t nf0 = 0, nf1 = 0;
    if (u0 < u1) {
      nf0 = __ldg(frow(u0, 0) + lane);
      nf1 = __ldg(frow(u0, 1) + lane);
    }
    uint32_t pc = 0, i = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u, ++i) {
      const bool first = u == u0 || u % S == 0;
      const uint32_t f0 = nf0, f1 = nf1;
      if (u + 1 < u1) {
        nf0 = __ldg(frow(u + 1, 0) + lane);
        nf1 = __ldg(frow(u + 1, 1) + lane);
      }
      if (kPeriodic && first) {
        // P_j[z][h] = [h(x_j, z) = h] for the pair of u: row r = 64 j + z, one thread a row
        if (pc > 0) ok = mbar_wait(pfree, (pc - 1) & 1u, g.err, 51, &s_abort);
        if (!ok) break;
        if (bt < 128) {
          const int j = bt >> 6, z = bt & 63;
          const int dx = (int)(2 * (u / S) + j) - R, dz = z - R;
          const int q = RF * RF - dx * dx - dz * dz;
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
#pragma unroll
      for (int k = 0; k < kMaxTasks; ++k) {
        const int t = bt + k * kBldThreads;
        if (k * kBldThreads >= tasks) break;  // warp-uniform
        // every lane shuffles (the source lane is its h); idle lanes use h = 0
        const int j = t < tasks ? t / (nzh * nc) : 0;
        uint32_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint32_t h = (hb[k][e >> 2] >> (8 * (e & 3))) & 0xffu;
          const uint32_t a = __shfl_sync(0xffffffffu, f0, (int)(h & 31u));
          const uint32_t b = __shfl_sync(0xffffffffu, f1, (int)(h & 31u));
          v[e] = h == 0xffu ? 0u : (j ? b : a);
        }
        if (t < tasks) {
          const int tt = t % (nzh * nc);
          const int z = zlo + tt / nc, c = clo + tt % nc;
          uint4 hi, lo;
          hi.x = __byte_perm(v[0], v[1], 0x5410);
          hi.y = __byte_perm(v[2], v[3], 0x5410);
          hi.z = __byte_perm(v[4], v[5], 0x5410);
          hi.w = __byte_perm(v[6], v[7], 0x5410);
          lo.x = __byte_perm(v[0], v[1], 0x7632);
          lo.y = __byte_perm(v[2], v[3], 0x7632);
          lo.z = __byte_perm(v[4], v[5], 0x7632);
          lo.w = __byte_perm(v[6], v[7], 0x7632);
          const int r = 64 * j + z, rm = 64 * j + 2 * R - z;
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
    const bool in_band = zr >= zs && zr < ze;
    uint32_t i = 0, segc = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u, ++i) {
      const bool last = u + 1 == u1 || (u + 1) % S == 0;
      const float ws = g.w[(int)(u % S)];
      ok = mbar_wait(d1full(i & 1u), (i >> 1) & 1u, g.err, 61, &s_abort);
      if (!ok) break;
      tc_fence_after();
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + 64u * (i & 1u) + 32u * half, v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(d1free(i & 1u));
      ok = mbar_wait(ufree(i & 1u), ((i >> 1) & 1u) ^ 1u, g.err, 62, &s_abort);
      if (!ok) break;
      if (in_band) {
        // U[(j, y)][z] for y = 32 half + e: MN-major atom row z & 7 of K atom z >> 3 in
        // M block j, 16-byte chunk c = y >> 3 at position c ^ (z & 7)
        uint8_t* U = gb + kOffU + (i & 1u) * 2 * kPl128 + j * 8192 + (zr >> 3) * 1024 +
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
      if (lane == 0) mbar_arrive(ufull(i & 1u));
      if (!last) continue;
      // the pair's E leaves tensor memory once, as a partial of this CTA
      ok = mbar_wait(efull, segc & 1u, g.err, 63, &s_abort);
      if (!ok) break;
      tc_fence_after();
      const long long p = u / S;
      const int kseg = (int)blockIdx.x - owner_cta(p * S, g.units, gridDim.x);
      tmem_ld32(tmem + lane_off + 128u + 32u * half, v);
      float4* o = reinterpret_cast<float4*>(
          g.part + ((p * g.maxseg + kseg) * 128 + 32 * quad + lane) * (long long)kG + 32 * half);
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

__device__ __forceinline__ int isqrt_int(int v) {
  int h = (int)sqrtf((float)v);
  while (h * h > v) --h;
  while ((h + 1) * (h + 1) <= v) ++h;
  return h;
}

// one warp per grid row (x, y), two z per lane: partials of the pair in order, + Dbar term,
// eps on the basis sphere; FP64 sum of the row's eps over the Fermi sphere
__global__ void __launch_bounds__(256)
    k_tcs_finalize(const float* part, const float* FB, int R, int RF, int S, int units, int grid,
                   int maxseg, int periodic, double pref, float* eps, double* row_ex) {
  const int Mg = 2 * R + 1;
  const int x = blockIdx.y, y = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (y >= Mg) return;  // whole warps
  const int p = x >> 1, j = x & 1;
  const int c0 = owner_cta((long long)p * S, units, grid);
  const int nseg = owner_cta((long long)(p + 1) * S - 1, units, grid) - c0 + 1;
  const int dx = x - R, dy = y - R;
  const int qb = RF * RF - dx * dx - dy * dy;
  const float* fb = (periodic && qb >= 0) ? FB + isqrt_int(qb) * kG : nullptr;
  const float* pp = part + ((long long)p * maxseg * 128 + 64 * j + y) * kG;
  double acc = 0.0;
#pragma unroll
  for (int k2 = 0; k2 < 2; ++k2) {
    const int z = lane + 32 * k2;
    if (z >= Mg) continue;
    float sum = 0.0f;
    for (int k = 0; k < nseg; ++k) sum += __ldg(pp + (long long)k * 128 * kG + z);
    if (fb) sum += __ldg(fb + z);
    const int dz = z - R, m = dx * dx + dy * dy + dz * dz;
    const float v = m <= R * R ? (float)(-pref * (double)sum) : 0.0f;
    eps[((long long)x * Mg + y) * Mg + z] = v;
    if (m <= RF * RF) acc += (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) row_ex[(long long)x * Mg + y] = acc;
}

__global__ void __launch_bounds__(1024)
    k_tcs_ex(const double* row_ex, int n, double* Ex, const int* err, int* status) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) acc += row_ex[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Ex[0] = 0.5 * red[0];
    Ex[1] = red[0];
    if (status) *status = *err;
  }
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

}  // namespace

struct TcSmallWs {
  int grid = 0, units = 0, maxseg = 0, RF_built = -1;
  uint32_t* FR = nullptr;
  void* F[2] = {nullptr, nullptr};
  void* T[2] = {nullptr, nullptr};
  float* FB = nullptr;
  float* part = nullptr;
  double* row_ex = nullptr;
  float* w32 = nullptr;
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
  TcSmallWs* w = new (std::nothrow) TcSmallWs();
  if (!w) return CC_ERR_ALLOC;
  const int S = t->S_eff, pairs = (t->Mg + 1) / 2;
  w->units = pairs * S;
  w->grid = std::min(sm_count(), w->units);
  for (int p = 0; p < pairs; ++p) {
    const int c0 = owner_cta((long long)p * S, w->units, w->grid);
    const int c1 = owner_cta((long long)(p + 1) * S - 1, w->units, w->grid);
    w->maxseg = std::max(w->maxseg, c1 - c0 + 1);
  }
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
      (st = alloc((void**)&w->row_ex, sizeof(double) * kG * kG)) != CC_OK ||
      (st = alloc((void**)&w->w32, sizeof(float) * S)) != CC_OK) {
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
  if (e != cudaSuccess) {
    set_last_error("small-grid tensor-core planes", e);
    tc_small_free(w);
    return CC_ERR_CUDA;
  }
  *out = w;
  return CC_OK;
}

cc_status tc_small_run(cc_tables t, void* ws, int* err, int stall_test, int R_F, float* eps,
                       double* Ex, cudaStream_t st) {
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
  a.R = R;
  a.R_F = R_F;
  a.Mg = Mg;
  a.S = S;
  a.periodic = periodic;
  a.units = w->units;
  a.maxseg = w->maxseg;
  a.FR = w->FR;
  a.w = w->w32;
  a.part = w->part;
  a.err = err;
  a.stall_test = stall_test;
  static bool attr = false;
  if (!attr) {
    CC_CUDA(cudaFuncSetAttribute(k_tcs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes));
    CC_CUDA(cudaFuncSetAttribute(k_tcs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes));
    attr = true;
  }
  const CUtensorMap& th = *reinterpret_cast<const CUtensorMap*>(w->map_th);
  const CUtensorMap& tl = *reinterpret_cast<const CUtensorMap*>(w->map_tl);
  const CUtensorMap& fh = *reinterpret_cast<const CUtensorMap*>(w->map_fh);
  const CUtensorMap& fl = *reinterpret_cast<const CUtensorMap*>(w->map_fl);
  if (periodic)
    k_tcs<true><<<w->grid, kThreads, kSmemBytes, st>>>(th, tl, fh, fl, a);
  else
    k_tcs<false><<<w->grid, kThreads, kSmemBytes, st>>>(th, tl, fh, fl, a);
  k_tcs_finalize<<<dim3((Mg + 7) / 8, Mg), 256, 0, st>>>(w->part, w->FB, R, R_F, S, w->units,
                                                         w->grid, w->maxseg, periodic, t->pref,
                                                         eps, w->row_ex);
  k_tcs_ex<<<1, 1024, 0, st>>>(w->row_ex, Mg * Mg, Ex, err, err + 1);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

}  // namespace cc
