// Fused tensor-core exchange sums, bf16 or fp16 hi + lo, any grid side up to 127 (operands
// padded to 128).
//
// Sec. III exchange of the uniform electron gas with the node sum of Sec. II Eq. 14; the
// periodic kernel uses the D_s = T_s - I split, so with the Fermi-sphere occupation O
//   E[x] = sum_s w_s (T_s R_{s,x} + A_{s,x}) T_s  +  (I x I x Dbar term),
// where, for the slab x (all matrices Mg x Mg, indices y, z):
//   R_{s,x}[y][z] = F_s[x][h(y, z)]     the first mode product of O (line along x),
//   A_{s,x}[y][z] = F_s[y][h(x, z)]     O x2 D_s restricted to the slab (line along y),
//   F_s[a][h]     = sum_{k = R-h}^{R+h} D_s[a][k]   (window sums, FP64, 0 for h < 0),
//   h(u, v)       = floor(sqrt(R_F^2 - (u-R)^2 - (v-R)^2)), -1 outside the sphere.
// The box kernel has F_s from T_s, no A term and no Dbar term.
//
// One CTA per SM walks a contiguous run of work units (slab pair, node).  For every unit:
//   MMA1  U_j = T_s R_{s,x_j}                 (A = T_s, B = R from shared memory)
//   epi   U_j <- w_s U_j + w_s A_{s,x_j}, split into bf16 hi + lo, written back into the
//         same tensor-memory columns (each 16-column piece becomes 8 hi + 8 lo columns)
//   MMA2  E_j += U_j T_s                      (A = U_j from tensor memory, B = T_s)
// for the two slabs x_0 = 2p, x_1 = 2p + 1 of the pair, issued in the order
//   MMA1(i, 0), MMA2(i-1, 1), MMA1(i, 1), MMA2(i, 0)
// so that the epilogue of one slab always overlaps two GEMMs of the other, the single
// R operand buffer has one GEMM of slack for its rebuild, and T_s (two buffers) is
// loaded by TMA two GEMMs ahead.  E_0, E_1 stay in tensor memory (FP32) for the whole run
// of nodes of the pair on this CTA and leave once, as a partial; a second kernel adds
// the partials of each pair in a fixed order (deterministic), adds the Dbar term and
// forms eps and E_x.  Each product is bf16x3: hi*hi + hi*lo + lo*hi, FP32 accumulate.
//
// Periodic boxes whose band is at most 96 columns wide form the A term on the tensor cores
// instead of in the epilogue: A_{s,x} = F_s P_x with the one-hot P_x[z][h] = [h(x, z) = h],
// exact in 16 bits, built with R; MMA1 adds F_s P_x (F_s hi and lo from the tensor-memory
// columns the band leaves free, staged once per node by the epilogue warps) to U_j, and
// the epilogue only scales and re-splits (fp16: F' = 2^j F and ones of 2^a, so the sum is
// 2^(a + j) (T R + A) like T' R').  Both terms are non-negative, so the sum has no
// cancellation.
//
// Tensor memory (512 columns): [0,128) U_0, [128,256) U_1, [256,384) E_0, [384,512) E_1;
// with the A term on the tensor cores F_s hi in [96,128), lo in [224,256).
// Warps: 0-7 epilogue (warp w: lanes 32 (w % 4) ..; warps w and w + 4 share the band's
// 16-column pieces evenly), 8-10 and 12-14 build R, 11 TMA producer, 15 MMA issuer.
// Warp w runs on scheduler w % 4, and the MMA issue rate drops with every busy warp on the
// MMA warp's scheduler: that scheduler hosts besides it the two quadrant-3 epilogue warps
// and the mostly idle producer, and the MMA warp issues converged, one K step (three MMAs)
// per elected instruction block.  Every wait is bounded (global timer); on expiry the error
// word is set, all roles stop, the MMA issuer drains its MMAs and tensor memory is freed
// before the CTA returns.
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

constexpr int kThreads = 512;
constexpr int kEpiWarps = 8;
constexpr int kBldWarps = 6;
constexpr int kBldThreads = 32 * kBldWarps;
constexpr int kProdWarp = 11;
constexpr int kMmaWarp = 15;
constexpr int kN = 128;                 // padded grid side
constexpr int kHMax = 64;               // window half-lengths h = 0 .. R_F <= 63
constexpr uint32_t kPlane = 128 * 64 * 2;   // one 64-wide K block of one plane: 16 KB
constexpr uint32_t kOp = 4 * kPlane;        // 128 x 128 operand, hi + lo: 64 KB
constexpr uint32_t kOffT = 0;               // two T_s buffers
constexpr uint32_t kOffR = 2 * kOp;         // the R operand
// the row of F_s of a build, replicated 32 times so that lane l reads its copy from bank
// l (entry h of copy l at word 32 h + l): conflict-free gathers; two of them alternate
constexpr uint32_t kFtabBytes = kHMax * 32 * 4;  // 8 KB
constexpr uint32_t kOffFtab = 3 * kOp;
// periodic boxes whose band is at most 96 columns wide add the A term on the tensor
// cores: A_{s,x} = F_s P_x with the one-hot P_x[z][h] = [h(x, z) = h] (band rows z, K = h),
// F_s as bf16 hi and lo in the tensor-memory columns the band leaves free in U_0 and U_1
constexpr int kMmaABand = 96;
constexpr uint32_t kOffP = kOffFtab + 2 * kFtabBytes;   // P_x, band rows x 128 bytes
constexpr uint32_t kFhi = 96, kFlo = 224;               // F_s hi / lo columns
constexpr uint32_t kOffBar = kOffP + kMmaABand * 128;  // mbarriers, tensor-memory slot
constexpr int kNumBars = 17;
constexpr uint32_t kOffIsq = kOffBar + 8 * kNumBars + 16;  // floor(sqrt(v)), v <= R_F^2
__host__ __device__ constexpr uint32_t slab_smem_bytes(int R_F) {
  return kOffIsq + (((uint32_t)(R_F * R_F + 1) + 15u) & ~15u) + 1024u;
}

struct Args {
  int R, R_F, Mg, S, periodic;
  int units, maxseg;
  const uint32_t* FR;  // [S][128][64] F_s[x][h] as bf16 hi (low half) | lo (high half)
  const float* FW;     // [S][64][128] w_s F_s[y][h], h-major (periodic)
  const float* w;      // [S]
  const int* aexp;     // [S] fp16: T' = 2^a T, the one-hot entries of P are 2^a
  float* part;         // [pairs * maxseg][2][128][128] partial E of a slab pair
  int* err;
  int stall_test;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_k, float hi_k) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_lo_f(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// x0, x1 -> (hi pair, lo pair) of 16-bit values, bf16 or fp16
template <bool kHalf>
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  if constexpr (kHalf) {
    __half2 h = __floats2half2_rn(x0, x1);
    __half2 l = __floats2half2_rn(x0 - __low2float(h), x1 - __high2float(h));
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
  } else {
    hi = pack_bf16x2(x0, x1);
    lo = pack_bf16x2(x0 - bf16_lo_f(hi), x1 - bf16_hi_f(hi));
  }
}

// kX1: hi * hi products only (no lo-plane correction; a diagnostic, bf16)
template <bool kHalf, bool kMmaA, bool kX1>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_slab(const __grid_constant__ CUtensorMap mTh, const __grid_constant__ CUtensorMap mTl,
              Args g) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gb = smem_raw + (base - raw);
  const uint8_t* isq = gb + kOffIsq;
  const uint32_t bar = base + kOffBar;
  auto tfull = [&](int k) { return bar + 8u * k; };          // 0, 1
  auto tfree = [&](int k) { return bar + 8u * (2 + k); };    // 2, 3
  const uint32_t rfull = bar + 8u * 4, rfree = bar + 8u * 5;
  auto d1full = [&](int j) { return bar + 8u * (6 + j); };   // 6, 7
  auto a2full = [&](int j) { return bar + 8u * (8 + j); };   // 8, 9
  const uint32_t efull = bar + 8u * 10, edone = bar + 8u * 11;
  const uint32_t never = bar + 8u * 12, drain = bar + 8u * 13;
  auto ftfull = [&](int k) { return bar + 8u * (14 + k); };  // 14, 15
  const uint32_t ffull = bar + 8u * 16;  // F_s of the next unit is in tensor memory
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gb + kOffBar + 8 * kNumBars);
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = g.R, RF = g.R_F, S = g.S;
  if (tid == 0) {
    s_abort = 0;
    for (int k = 0; k < 2; ++k) {
      mbar_init(tfull(k), 1);
      mbar_init(tfree(k), 1);
      mbar_init(d1full(k), 1);
      mbar_init(a2full(k), kEpiWarps);
    }
    mbar_init(rfull, kBldWarps);
    mbar_init(rfree, 1);
    mbar_init(efull, 1);
    mbar_init(edone, kEpiWarps);
    mbar_init(never, 1);
    mbar_init(drain, 1);
    mbar_init(ftfull(0), kBldWarps);
    mbar_init(ftfull(1), kBldWarps);
    mbar_init(ffull, kEpiWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // isqrt table and a zero R operand (the builders only ever write the square
  // |y - R|, |z - R| <= R_F; the rest of the operand stays zero)
  for (int v = tid; v <= RF * RF; v += kThreads) {
    int h = (int)sqrtf((float)v);
    while (h * h > v) --h;
    while ((h + 1) * (h + 1) <= v) ++h;
    gb[kOffIsq + v] = (uint8_t)h;
  }
  for (uint32_t o = 16u * tid; o < kOp; o += 16u * kThreads)
    *reinterpret_cast<uint4*>(gb + kOffR + o) = make_uint4(0u, 0u, 0u, 0u);
  if (kMmaA)  // P starts all zero; every build then moves the one of each row
    for (uint32_t o = 16u * tid; o < kMmaABand * 128u; o += 16u * kThreads)
      *reinterpret_cast<uint4*>(gb + kOffP + o) = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // U and R vanish outside the band [R - R_F, R + R_F] of z (and of y for R): the products
  // run over the 16-aligned band [zs, ze) only (U column n holds z = zs + n)
  const int zs = (R - RF) & ~15, ze = (R + RF + 16) & ~15, nact = ze - zs;
  const long long u0 = (long long)blockIdx.x * g.units / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * g.units / gridDim.x;

  if (warp == kProdWarp) {
    if (lane == 0) {
      // ---------------- TMA producer: T_s hi + lo, both K blocks, into buffer (unit & 1)
      uint32_t n = 0;
      int s = (int)(u0 % S);  // node of unit u, stepped (no 64-bit division per unit)
      for (long long u = u0; u < u1 && !s_abort; ++u, ++n, s = s + 1 == S ? 0 : s + 1) {
        const int k = (int)(n & 1u);
        if (!mbar_wait(tfree(k), ((n >> 1) & 1u) ^ 1u, g.err, 11, &s_abort)) {
          s_abort = 1;
          break;
        }
        const uint32_t dst = base + kOffT + k * kOp;
        mbar_expect_tx(tfull(k), kOp);
        for (int kb = 0; kb < 2; ++kb) {
          tma_load_2d(dst + kb * 2 * kPlane, &mTh, kb * 64, s * kN, tfull(k));
          tma_load_2d(dst + kb * 2 * kPlane + kPlane, &mTl, kb * 64, s * kN, tfull(k));
        }
      }
      // copies still in flight land before the CTA leaves
      for (uint32_t m = n > 2 ? n - 2 : 0; m < n; ++m)
        mbar_wait(tfull(m & 1u), (m >> 1) & 1u, g.err, 12, nullptr, 100000000ull);
    }
  } else if (warp == kMmaWarp) {
    {
      // ---------------- MMA issuer (the whole warp; every wait result made warp-uniform)
      auto all = [](bool v) { return __all_sync(0xffffffffu, v); };
      // F32 accumulate; A and B both bf16 (format 1) or both fp16 (format 0)
      constexpr uint32_t fmt = kHalf ? 0u : 1u;
      constexpr uint32_t idesc0 =
          (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(128 >> 4) << 24);
      const uint32_t idesc1 = idesc0 | ((uint32_t)(nact >> 3) << 17);  // N = band width
      // N = the grid side rounded up to 16 (columns z' >= Mg are never read)
      const uint32_t idesc2 = idesc0 | ((uint32_t)(((g.Mg + 15) & ~15) >> 3) << 17);
      if (g.stall_test && !all(mbar_wait(never, 0, g.err, 5, nullptr, 20000000ull))) s_abort = 1;
      uint32_t n = 0, r = 0, segc = 0;
      // descriptors as base + constant: the start-address field holds address / 16, so a
      // byte offset o (all addresses < 256 KB) adds o / 16
      const int ms = zs >> 4, me = ze >> 4;
      const uint64_t dR = sdesc(base + kOffR + zs * 128u);  // B rows z = zs ..
      // the A-term MMAs: K = h < 16 nh (h <= R_F), B = P_x (band rows), A = F_s hi and lo
      const int nh = (RF + 16) >> 4;
      const uint64_t dP = sdesc(base + kOffP);
      auto mma1 = [&](uint32_t tb, int j) {
        const uint32_t d = tmem + (uint32_t)(j * 128);
        const uint64_t dT = sdesc(tb);
#pragma unroll
        for (int m = 0; m < 8; ++m) {  // K step m covers y = 16 m .. 16 m + 15
          if (m < ms || m >= me) continue;
          constexpr uint64_t kPl = kPlane >> 4;
          const uint64_t o = (uint64_t)((m >> 2) * 2 * (kPlane >> 4) + 2 * (m & 3));
          const uint32_t acc = m > ms ? 1u : 0u;
          if constexpr (kX1) mma_x1_w(d, dT + o, dR + o, idesc1, acc);
          else mma_x3_w(d, dT + o, dR + o, kPl, kPl, idesc1, acc);
        }
        if constexpr (kMmaA) {
#pragma unroll
          for (int m = 0; m < 4; ++m)
            if (m < nh) {
              if constexpr (kX1) mma_x1_ts_w(d, tmem + kFhi + 8u * m, dP + 2u * m, idesc1, 1u);
              else mma_x2_ts_w(d, tmem + kFhi + 8u * m, tmem + kFlo + 8u * m, dP + 2u * m,
                               idesc1);
            }
        }
      };
      auto mma2 = [&](uint32_t tb, int j, bool first) {
        const uint32_t d = tmem + 256u + (uint32_t)(j * 128);
        const uint32_t a0 = tmem + (uint32_t)(j * 128) - (uint32_t)(16 * ms);
        const uint64_t dT = sdesc(tb);
#pragma unroll
        for (int m = 0; m < 8; ++m) {  // K step m covers z = 16 m .. 16 m + 15
          if (m < ms || m >= me) continue;
          constexpr uint64_t kPl = kPlane >> 4;
          const uint64_t o = (uint64_t)((m >> 2) * 2 * (kPlane >> 4) + 2 * (m & 3));
          // U piece of z = 16 m ..: columns 16 (m - zs / 16) .., 8 hi then 8 lo
          const uint32_t aH = a0 + (uint32_t)(16 * m);
          if constexpr (kX1) mma_x1_ts_w(d, aH, dT + o, idesc2, (first && m == ms) ? 0u : 1u);
          else mma_x3_ts_w(d, aH, dT + o, kPl, idesc2, (first && m == ms) ? 0u : 1u);
        }
      };
      bool ok = all(!s_abort);
      for (long long u = u0; u < u1 && ok;) {
        const long long p = u / S;
        const long long ue = u1 < (p + 1) * S ? u1 : (p + 1) * S;
        const int U = (int)(ue - u);
        for (int i = 0; i < U && ok; ++i, ++n) {
          const uint32_t k = n & 1u, tb = base + kOffT + k * kOp;
          const uint32_t tbp = base + kOffT + (k ^ 1u) * kOp;
          // MMA1(i, 0): the three barriers are tested together first; otherwise waited for
          // with the R operand (the critical path) last, so that its completion is followed
          // by the issue without further waits
          if (!all(mbar_test(tfull(k), (n >> 1) & 1u) & mbar_test(rfull, r & 1u) &
                   (!kMmaA || mbar_test(ffull, n & 1u))))
            ok = all(mbar_wait(tfull(k), (n >> 1) & 1u, g.err, 14, &s_abort) &&
                     (!kMmaA || mbar_wait(ffull, n & 1u, g.err, 18, &s_abort)) &&
                     mbar_wait(rfull, r & 1u, g.err, 15, &s_abort));
          if (!ok) break;
          tc_fence_after();
          mma1(tb, 0);
          mma_commit_w(rfree);
          mma_commit_w(d1full(0));
          ++r;
          // MMA2(i - 1, 1)
          if (i > 0) {
            ok = all(mbar_wait(a2full(1), (n - 1) & 1u, g.err, 16, &s_abort));
            if (!ok) break;
            tc_fence_after();
            mma2(tbp, 1, i - 1 == 0);
            mma_commit_w(tfree(k ^ 1u));
          }
          // MMA1(i, 1)
          ok = all(mbar_wait(rfull, r & 1u, g.err, 15, &s_abort));
          if (!ok) break;
          tc_fence_after();
          mma1(tb, 1);
          mma_commit_w(rfree);
          mma_commit_w(d1full(1));
          ++r;
          // MMA2(i, 0); the first one of a pair also waits until the previous pair's E
          // has left tensor memory
          ok = all(mbar_wait(a2full(0), n & 1u, g.err, 16, &s_abort) &&
                   (i > 0 || segc == 0 || mbar_wait(edone, (segc - 1) & 1u, g.err, 13, &s_abort)));
          if (!ok) break;
          tc_fence_after();
          mma2(tb, 0, i == 0);
        }
        if (!ok) break;
        // MMA2(U - 1, 1), then E of the pair is complete
        const uint32_t kl = (n - 1) & 1u;
        ok = all(mbar_wait(a2full(1), (n - 1) & 1u, g.err, 16, &s_abort));
        if (!ok) break;
        tc_fence_after();
        mma2(base + kOffT + kl * kOp, 1, U == 1);
        mma_commit_w(tfree(kl));
        mma_commit_w(efull);
        ++segc;
        u = ue;
      }
      if (!ok) s_abort = 1;
      // every MMA issued has finished before tensor memory is released
      mma_commit_w(drain);
      mbar_wait(drain, 0, g.err, 17, nullptr, 100000000ull);
    }
  } else if (warp >= kEpiWarps) {
    // ---------------- R operand builders (warps 8-10, 12-14)
    // R_{s,x}[y][z] = F_s[x][h(y, z)]: the x line of the sphere at (y, z) does not depend
    // on x, only the row of F_s does, and rows z and 2R - z of the operand are equal.  A
    // builder thread always forms the same 16-byte chunks (row z <= R of the square
    // |y - R|, |z - R| <= R_F, 8 consecutive y) and stores each into both mirror rows, so
    // it keeps their h values in registers (packed bytes) from the start.  The row of F_s
    // of a build is written by all builder warps into a replicated table (copy l in bank
    // l) and every element is one conflict-free shared-memory load away.
    const int bw = warp < kProdWarp ? warp - kEpiWarps : warp - kEpiWarps - 1;
    const int bt = 32 * bw + lane;
    const int zlo = R - RF, nzh = RF + 1;
    const int clo = (R - RF) >> 3, nc = ((R + RF) >> 3) - clo + 1;
    const int tasks = nzh * nc;  // <= 64 x 16 = 1024 = 5.3 x 192
    constexpr int kMaxTasks = 6;
    uint32_t hb[kMaxTasks][2];
#pragma unroll
    for (int k = 0; k < kMaxTasks; ++k) {
      const int t = bt + k * kBldThreads;
      hb[k][0] = hb[k][1] = 0xffffffffu;
      if (t < tasks) {
        const int z = zlo + t / nc, c = clo + t % nc, dz = z - R;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int dy = 8 * c + e - R;
          const int q = RF * RF - dy * dy - dz * dz;
          const uint32_t h = q >= 0 ? (uint32_t)isq[q] : 0xffu;
          hb[k][e >> 2] = (hb[k][e >> 2] & ~(0xffu << (8 * (e & 3)))) | (h << (8 * (e & 3)));
        }
      }
    }
    // the window-sum row of slab 2 p + j at node s; the unit's (node, pair) place is stepped
    // from unit to unit (no 64-bit division per build)
    auto frow = [&](int sn, int pn, int j) {
      return g.FR + ((long long)sn * kN + 2 * pn + j) * kHMax;
    };
    int su = (int)(u0 % S), pu = (int)(u0 / S);  // place of unit u
    // this warp fills entries h = hw0 .. hw0 + 10 (11 per warp, 6 warps cover 64)
    const int hw0 = 11 * bw;
    uint32_t nf0 = __ldg(frow(su, pu, 0) + lane), nf1 = __ldg(frow(su, pu, 0) + lane + 32);
    uint32_t r = 0;
    int p_h = -1;  // the h of this thread's row of P as it stands (-1: zero row)
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u) {
      const int sn = su + 1 == S ? 0 : su + 1, pn = su + 1 == S ? pu + 1 : pu;  // unit u + 1
      for (int j = 0; j < 2 && ok; ++j, ++r) {
        const uint32_t f0 = nf0, f1 = nf1;
        const long long un = j == 0 ? u : u + 1;
        if (un < u1) {  // the next build's row
          const int ss = j == 0 ? su : sn, ps = j == 0 ? pu : pn;
          nf0 = __ldg(frow(ss, ps, j ^ 1) + lane);
          nf1 = __ldg(frow(ss, ps, j ^ 1) + lane + 32);
        }
        // every warp has finished build r - 2, so table (r & 1) is free
        uint32_t* ft = reinterpret_cast<uint32_t*>(gb + kOffFtab + (r & 1u) * kFtabBytes);
#pragma unroll
        for (int i = 0; i < 11; ++i) {
          const int h = hw0 + i;
          const uint32_t a = __shfl_sync(0xffffffffu, f0, h & 31);
          const uint32_t b = __shfl_sync(0xffffffffu, f1, h & 31);
          if (h < kHMax) ft[32 * h + lane] = h < 32 ? a : b;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(ftfull(r & 1u));
        ok = mbar_wait(ftfull(r & 1u), (r >> 1) & 1u, g.err, 22, &s_abort) &&
             mbar_wait(rfree, (r & 1u) ^ 1u, g.err, 21, &s_abort);
        if (!ok) break;
#pragma unroll
        for (int k = 0; k < kMaxTasks; ++k) {
          const int t = bt + k * kBldThreads;
          if (k * kBldThreads >= tasks) break;  // warp-uniform
          if (t < tasks) {
            uint32_t v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const uint32_t h = (hb[k][e >> 2] >> (8 * (e & 3))) & 0xffu;
              v[e] = h == 0xffu ? 0u : ft[32 * h + lane];
            }
            const int z = zlo + t / nc, c = clo + t % nc;
            uint4 hi, lo;
            hi.x = __byte_perm(v[0], v[1], 0x5410);
            hi.y = __byte_perm(v[2], v[3], 0x5410);
            hi.z = __byte_perm(v[4], v[5], 0x5410);
            hi.w = __byte_perm(v[6], v[7], 0x5410);
            lo.x = __byte_perm(v[0], v[1], 0x7632);
            lo.y = __byte_perm(v[2], v[3], 0x7632);
            lo.z = __byte_perm(v[4], v[5], 0x7632);
            lo.w = __byte_perm(v[6], v[7], 0x7632);
            const uint32_t kb = (uint32_t)(c >> 3) * 2 * kPlane;
            const int zm = 2 * R - z;
            const uint32_t off = kOffR + kb + (uint32_t)z * 128u +
                                 ((uint32_t)((c & 7) ^ (z & 7)) << 4);
            *reinterpret_cast<uint4*>(gb + off) = hi;
            *reinterpret_cast<uint4*>(gb + off + kPlane) = lo;
            if (zm != z) {
              const uint32_t offm = kOffR + kb + (uint32_t)zm * 128u +
                                    ((uint32_t)((c & 7) ^ (zm & 7)) << 4);
              *reinterpret_cast<uint4*>(gb + offm) = hi;
              *reinterpret_cast<uint4*>(gb + offm + kPlane) = lo;
            }
          }
        }
        if constexpr (kMmaA) {
          // P_x for x = 2 p + j: band row rr (z = zs + rr) is one-hot at h(x, z), zero
          // outside the sphere; 16-byte chunk c holds h = 8 c .. 8 c + 7 (128-byte swizzle).
          // The one is bf16 1 or, fp16, the node's 2^a (so that F' = 2^j F times P gives
          // 2^(a + j) A, the scale of T' R').  Builder thread rr owns row rr: the chunk of
          // the previous h is cleared, the chunk of the new h written (at most two 16-byte
          // stores; bf16 skips both while h stays)
          if (bt < nact) {
            const int rr = bt, dz = zs + rr - R, dx = 2 * pu + j - R;
            const int q = RF * RF - dx * dx - dz * dz;
            const int h = q >= 0 ? (int)isq[q] : -1;
            if (p_h >= 0 && p_h != h)
              *reinterpret_cast<uint4*>(gb + kOffP + rr * 128 + (((p_h >> 3) ^ (rr & 7)) << 4)) =
                  make_uint4(0u, 0u, 0u, 0u);
            if (h >= 0 && (kHalf || h != p_h)) {
              const uint32_t v1 =
                  kHalf ? (uint32_t)(0x3C00 + 1024 * g.aexp[su]) : 0x3F80u;
              const uint32_t one = v1 << (16 * (h & 1)), wi = (uint32_t)(h & 7) >> 1;
              *reinterpret_cast<uint4*>(gb + kOffP + rr * 128 + (((h >> 3) ^ (rr & 7)) << 4)) =
                  make_uint4(wi == 0 ? one : 0u, wi == 1 ? one : 0u, wi == 2 ? one : 0u,
                             wi == 3 ? one : 0u);
            }
            p_h = h;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(rfull);
      }
      su = sn;
      pu = pn;
    }
    if (!ok) s_abort = 1;
  } else {
    // ---------------- epilogue warps 0-7
    const int quad = warp & 3, half = warp >> 2;
    const int yrow = 32 * quad + lane;
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    // the band's 16-column pieces split evenly between the two warps of a lane quadrant:
    // this warp's np pieces start at band column c0
    const int npc = nact >> 4, n0 = (npc + 1) >> 1;
    const int c0 = half ? 16 * n0 : 0, np = half ? npc - n0 : n0;
    uint32_t n = 0, segc = 0;
    bool ok = true;
    // the A-term MMAs read F_s of unit uu from tensor memory: lane y, column kFhi + c
    // (kFlo + c) holds the bf16 hi (lo) pair of h = 2 c, 2 c + 1; this warp writes
    // h = 32 half .. 32 half + 31 of its lanes from the window-sum rows F_s[y][.]
    uint4 fpre[8];  // the next unit's row segment, loaded a unit ahead of its staging
    auto load_f = [&](int su) {  // node su
      const uint4* src = reinterpret_cast<const uint4*>(
          g.FR + ((long long)su * kN + yrow) * kHMax + 32 * half);
#pragma unroll
      for (int i = 0; i < 8; ++i) fpre[i] = __ldg(src + i);
    };
    auto stage_f = [&]() {
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint4 f = fpre[i];
        hi[2 * i] = __byte_perm(f.x, f.y, 0x5410);
        lo[2 * i] = __byte_perm(f.x, f.y, 0x7632);
        hi[2 * i + 1] = __byte_perm(f.z, f.w, 0x5410);
        lo[2 * i + 1] = __byte_perm(f.z, f.w, 0x7632);
      }
      tmem_st16(tmem + lane_off + kFhi + 16u * half, hi);
      tmem_st16(tmem + lane_off + kFlo + 16u * half, lo);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(ffull);
    };
    if constexpr (kMmaA) {
      if (u0 < u1) {
        load_f((int)(u0 % S));
        stage_f();
      }
    }
    for (long long u = u0; u < u1 && ok;) {
      const long long p = u / S;
      const long long ue = u1 < (p + 1) * S ? u1 : (p + 1) * S;
      // h(x_j, z) for the columns z = zs + c0 + 32 k + lane of this warp's two chunks (fixed
      // for the whole pair; broadcast by shuffle per column), -1 outside the sphere
      int hz[2][2];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int dx = (int)(2 * p + j) - R, dz = zs + c0 + 32 * k + lane - R;
          const int q = RF * RF - dx * dx - dz * dz;
          hz[j][k] = q >= 0 ? (int)isq[q] : -1;
        }
      for (; u < ue && ok; ++u, ++n) {
        const int s = (int)(u - p * S);
        const float ws = g.w[s];
        const float* FWs = g.FW + (long long)s * kHMax * kN + yrow;
        if constexpr (kMmaA) {
          if (u + 1 < u1) load_f(s + 1 == S ? 0 : s + 1);
        }
        for (int j = 0; j < 2; ++j) {
          // the A-term values of this warp's columns, requested before the MMA result is
          // waited for (their L2 latency hides behind the wait)
          float a[2][32];
          if constexpr (!kMmaA) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              const int hzk = j == 0 ? hz[0][k] : hz[1][k];
#pragma unroll
              for (int e = 0; e < 32; ++e) {
                const int h = __shfl_sync(0xffffffffu, hzk, e);
                a[k][e] = (g.periodic && h >= 0) ? __ldg(FWs + h * kN) : 0.0f;
              }
            }
          }
          ok = mbar_wait(d1full(j), n & 1u, g.err, 31, &s_abort);
          if (!ok) break;
          tc_fence_after();
          // the second first mode product of this unit is done with F_s: the next unit's
          // goes into tensor memory (the MMA warp waits for it before that unit's first MMA)
          if constexpr (kMmaA) {
            if (j == 1 && u + 1 < u1) stage_f();
          }
          // in place, 16 columns at a time: FP32 U of the piece z = zs + 16 m .. in columns
          // 16 m .. 16 m + 15 becomes 8 columns of bf16 hi pairs followed by 8 of lo pairs
#pragma unroll
          for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int sub = 0; sub < 2; ++sub) {
              if (2 * k + sub >= np) continue;  // beyond this warp's pieces
              const uint32_t ta = tmem + lane_off + (uint32_t)(j * 128 + c0 + 32 * k + 16 * sub);
              uint32_t v[16];
              tmem_ld16(ta, v);
              uint32_t hi[8], lo[8];
#pragma unroll
              for (int e = 0; e < 16; e += 2) {
                float x0, x1;
                if constexpr (kMmaA) {  // U already holds T_s R + A
                  x0 = __uint_as_float(v[e]) * ws;
                  x1 = __uint_as_float(v[e + 1]) * ws;
                } else {
                  x0 = fmaf(__uint_as_float(v[e]), ws, a[k][16 * sub + e]);
                  x1 = fmaf(__uint_as_float(v[e + 1]), ws, a[k][16 * sub + e + 1]);
                }
                split_pair<kHalf>(x0, x1, hi[e >> 1], lo[e >> 1]);
              }
              tmem_st8(ta, hi);
              tmem_st8(ta + 8u, lo);
            }
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(a2full(j));
        }
      }
      if (!ok) break;
      // the pair's E leaves tensor memory once, as a partial of this CTA
      ok = mbar_wait(efull, segc & 1u, g.err, 32, &s_abort);
      if (!ok) break;
      tc_fence_after();
      const int kseg = (int)blockIdx.x - owner_cta(p * S, g.units, gridDim.x);
      float* P = g.part + ((p * g.maxseg + kseg) * 2) * (long long)(kN * kN);
      for (int j = 0; j < 2; ++j) {
#pragma unroll 1
        for (int cc = 2 * half; cc < 2 * half + 2; ++cc) {
          uint32_t v[32];
          tmem_ld32(tmem + lane_off + (uint32_t)(256 + j * 128 + 32 * cc), v);
          float4* o = reinterpret_cast<float4*>(P + (long long)j * kN * kN + yrow * kN + 32 * cc);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            o[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                               __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
        }
      }
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }
}

// F_s window sums (FP64) of every row a < Mg: the bf16 hi | lo pairs for the R operand and,
// periodic, w_s F_s transposed for the A term.  One thread per (s, a).
__global__ void k_tc_slab_prep(const double* Tm, const double* w, int S, int Mg, int R, int RF,
                               int periodic, uint32_t* FR, float* FW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * kN) return;
  const int s = i / kN, a = i % kN;
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
    if (periodic) FW[((long long)s * kHMax + h) * kN + a] = (float)(w[s] * f);
  }
}

// T_s as bf16 hi + lo planes padded to 128 x 128 (grids of side <= 64, whose step-chain
// planes are 64 x 64)
__global__ void k_tc_slab_tplanes(const double* Tm, int S, int Mg, __nv_bfloat16* hi,
                                  __nv_bfloat16* lo) {
  const long long n = (long long)S * kN * kN;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / (kN * kN)), a = (int)((i / kN) % kN), c = (int)(i % kN);
    const double t = (a < Mg && c < Mg) ? Tm[((long long)s * Mg + a) * Mg + c] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16_rn((float)t);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn((float)t - __bfloat162float(h));
  }
}

// fp16x3 keeps every operand inside fp16's range with power-of-two scales per node s:
//   R' = 2^j F (largest value 2^14), T' = 2^a T for both products, and the epilogue forms
//   U'' = 2^-a w (T R + A) = (T' R') w 2^(-2a-j) + (2^-a w F) so that U'' T' = w (T R + A) T;
//   a balances the largest T' (2^a) and U'' (2^-a w (Mg + 1) max F).
// The largest window sum of each node (F grows with h, so it is reached at h = R_F), as the
// bits of a non-negative float.  One thread per (s, a).
__global__ void k_tc_slab_fmax(const double* Tm, int S, int Mg, int R, int RF, int periodic,
                               unsigned* fmax_bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * Mg) return;
  const int s = i / Mg, a = i % Mg;
  const double* row = Tm + ((long long)s * Mg + a) * Mg;
  double f = 0.0;
  for (int k = R - RF; k <= R + RF; ++k) f += (periodic && k == a) ? 0.0 : row[k];
  atomicMax(fmax_bits + s, __float_as_uint((float)f));
}

__global__ void k_tc_slab_scales(const unsigned* fmax_bits, const double* w, int S, int Mg,
                                 int* jexp, int* aexp, float* wsc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double fm = (double)__uint_as_float(fmax_bits[s]);
  int j = 0, a = 0;
  if (fm > 0.0) {
    int e;
    frexp(fm, &e);  // fm < 2^e
    j = 14 - e;
    frexp(w[s] * (Mg + 1) * fm, &e);
    a = (int)floor(0.5 * e + 0.5);
    a = a < -14 ? -14 : (a > 14 ? 14 : a);
  }
  jexp[s] = j;
  aexp[s] = a;
  wsc[s] = (float)ldexp(w[s], -2 * a - j);
}

// fp16: R' = 2^j F as fp16 hi | lo pairs, 2^-a w F for the A term
__global__ void k_tc_slab_prep16(const double* Tm, const double* w, int S, int Mg, int R,
                                 int RF, int periodic, const int* jexp, const int* aexp,
                                 uint32_t* FR, float* FW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * kN) return;
  const int s = i / kN, a = i % kN;
  const double* row = Tm + ((long long)s * Mg + (a < Mg ? a : 0)) * Mg;
  auto X = [&](int k) { return (periodic && k == a) ? 0.0 : row[k]; };
  const int js = jexp[s], as = aexp[s];
  double acc = 0.0;
  for (int h = 0; h < kHMax; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? X(R) : X(R - h) + X(R + h);
      f = acc;
    }
    const double fs = ldexp(f, js);
    const __half hb = __float2half_rn((float)fs);
    const __half lb = __float2half_rn((float)(fs - (double)__half2float(hb)));
    FR[(long long)i * kHMax + h] = (uint32_t)__half_as_ushort(hb) |
                                   ((uint32_t)__half_as_ushort(lb) << 16);
    if (periodic) FW[((long long)s * kHMax + h) * kN + a] = (float)ldexp(w[s] * f, -as);
  }
}

// fp16: T' = 2^a T as fp16 hi + lo planes padded to 128 x 128
__global__ void k_tc_slab_tplanes16(const double* Tm, int S, int Mg, const int* aexp,
                                    __half* hi, __half* lo) {
  const long long n = (long long)S * kN * kN;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / (kN * kN)), a = (int)((i / kN) % kN), c = (int)(i % kN);
    const double t =
        (a < Mg && c < Mg) ? ldexp(Tm[((long long)s * Mg + a) * Mg + c], aexp[s]) : 0.0;
    const __half h = __float2half_rn((float)t);
    hi[i] = h;
    lo[i] = __float2half_rn((float)(t - (double)__half2float(h)));
  }
}

// window sums of Dbar (I x I x Dbar term), FB[h][z'] = sum_{k=R-h}^{R+h} Dbar[z'][k]
__global__ void k_tc_slab_dbar(const double* Dbar, int Mg, int R, int RF, float* FB) {
  const int a = threadIdx.x;
  double acc = 0.0;
  for (int h = 0; h < kHMax; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? Dbar[a * Mg + R] : Dbar[a * Mg + R - h] + Dbar[a * Mg + R + h];
      f = acc;
    }
    FB[h * kN + a] = (float)f;
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

struct TcSlabWs {
  int grid = 0, units = 0, maxseg = 0, RF_built = -1;
  uint32_t* FR = nullptr;
  float* FW = nullptr;
  float* FB = nullptr;
  float* part = nullptr;
  double* blk_ex = nullptr;
  unsigned* ticket = nullptr;  // blocks of the finaliser done (0 between calls)
  float* w32 = nullptr;
  // grids of side <= 64: own 128-padded T planes and their maps (else the step chain's)
  void* T128[2] = {nullptr, nullptr};
  alignas(64) unsigned char map_hi[128], map_lo[128];
  // fp16x3: scaled operands of their own (see k_tc_slab_scales)
  int RF16_built = -1;
  uint32_t* FR16 = nullptr;
  float* FW16 = nullptr;
  float* FB16 = nullptr;
  float* w16 = nullptr;
  unsigned* fmax = nullptr;
  int* jexp = nullptr;
  int* aexp = nullptr;
  void* T16[2] = {nullptr, nullptr};
  alignas(64) unsigned char map16_hi[128], map16_lo[128];
  std::vector<void*> allocs;
};

bool tc_slab_supported(cc_tables t) { return t->Mg <= 127 && t->p.R <= 63; }

cc_status tc_slab_alloc(cc_tables t, void** out) {
  *out = nullptr;
  if (!tc_slab_supported(t)) return CC_OK;
  TcSlabWs* w = new (std::nothrow) TcSlabWs();
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
      set_last_error("cudaMalloc(tensor-core slab workspace)", e);
      return CC_ERR_ALLOC;
    }
    w->allocs.push_back(*p);
    t->ws.mx_bytes += bytes;
    t->device_bytes += bytes;
    return CC_OK;
  };
  cc_status st = CC_OK;
  if ((st = alloc((void**)&w->FR, sizeof(uint32_t) * S * kN * kHMax)) != CC_OK ||
      (st = alloc((void**)&w->FW, sizeof(float) * S * kN * kHMax)) != CC_OK ||
      (st = alloc((void**)&w->FB, sizeof(float) * kN * kHMax)) != CC_OK ||
      (st = alloc((void**)&w->part, sizeof(float) * 2 * kN * kN * pairs * w->maxseg)) != CC_OK ||
      (st = alloc((void**)&w->blk_ex, sizeof(double) * kN * kN)) != CC_OK ||
      (st = alloc((void**)&w->ticket, sizeof(unsigned))) != CC_OK ||
      (st = alloc((void**)&w->w32, sizeof(float) * S)) != CC_OK) {
    tc_slab_free(w);
    return st;
  }
  if (cudaMemset(w->ticket, 0, sizeof(unsigned)) != cudaSuccess) {
    set_last_error("cudaMemset(finaliser ticket)", cudaGetLastError());
    tc_slab_free(w);
    return CC_ERR_CUDA;
  }
  if (t->Mg <= 64) {
    const size_t plane = sizeof(__nv_bfloat16) * (size_t)S * kN * kN;
    if ((st = alloc(&w->T128[0], plane)) != CC_OK || (st = alloc(&w->T128[1], plane)) != CC_OK) {
      tc_slab_free(w);
      return st;
    }
    static_assert(sizeof(CUtensorMap) <= 128, "tensor map size");
    if ((st = tc_make_map_bf16(w->map_hi, w->T128[0], (long long)S * kN, kN, kN)) != CC_OK ||
        (st = tc_make_map_bf16(w->map_lo, w->T128[1], (long long)S * kN, kN, kN)) != CC_OK) {
      tc_slab_free(w);
      return st;
    }
    k_tc_slab_tplanes<<<1024, 256>>>(t->d.Tm64, S, t->Mg, (__nv_bfloat16*)w->T128[0],
                                     (__nv_bfloat16*)w->T128[1]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_last_error("k_tc_slab_tplanes", e);
      tc_slab_free(w);
      return CC_ERR_CUDA;
    }
  }
  {
    const size_t plane = sizeof(__half) * (size_t)S * kN * kN;
    if ((st = alloc((void**)&w->FR16, sizeof(uint32_t) * S * kN * kHMax)) != CC_OK ||
        (st = alloc((void**)&w->FW16, sizeof(float) * S * kN * kHMax)) != CC_OK ||
        (st = alloc((void**)&w->FB16, sizeof(float) * kN * kHMax)) != CC_OK ||
        (st = alloc((void**)&w->w16, sizeof(float) * S)) != CC_OK ||
        (st = alloc((void**)&w->fmax, sizeof(unsigned) * S)) != CC_OK ||
        (st = alloc((void**)&w->jexp, sizeof(int) * S)) != CC_OK ||
        (st = alloc((void**)&w->aexp, sizeof(int) * S)) != CC_OK ||
        (st = alloc(&w->T16[0], plane)) != CC_OK || (st = alloc(&w->T16[1], plane)) != CC_OK ||
        (st = tc_make_map_16(w->map16_hi, w->T16[0], (long long)S * kN, kN, kN, false)) !=
            CC_OK ||
        (st = tc_make_map_16(w->map16_lo, w->T16[1], (long long)S * kN, kN, kN, false)) !=
            CC_OK) {
      tc_slab_free(w);
      return st;
    }
  }
  std::vector<float> w32(S);
  for (int i = 0; i < S; ++i) w32[i] = (float)t->w[t->kept_idx[i]];
  cudaError_t e = cudaMemcpy(w->w32, w32.data(), sizeof(float) * S, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_last_error("cudaMemcpy(node weights)", e);
    tc_slab_free(w);
    return CC_ERR_CUDA;
  }
  *out = w;
  return CC_OK;
}

void tc_slab_free(void* p) {
  TcSlabWs* w = reinterpret_cast<TcSlabWs*>(p);
  if (!w) return;
  for (void* a : w->allocs) cudaFree(a);
  delete w;
}

cc_status tc_slab_run(cc_tables t, void* ws, const void* map_hi, const void* map_lo, int* err,
                      int stall_test, int R_F, float* eps, double* Ex, cudaStream_t st,
                      bool half, int x1) {
  TcSlabWs* w = reinterpret_cast<TcSlabWs*>(ws);
  if (!w || !tc_slab_supported(t) || R_F > 63) return CC_ERR_NOTSUPP;
  const int S = t->S_eff, Mg = t->Mg, R = t->p.R;
  const int periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  if (half && w->RF16_built != R_F) {
    CC_CUDA(cudaMemsetAsync(w->fmax, 0, sizeof(unsigned) * S, st));
    k_tc_slab_fmax<<<(S * Mg + 127) / 128, 128, 0, st>>>(t->d.Tm64, S, Mg, R, R_F, periodic,
                                                         w->fmax);
    k_tc_slab_scales<<<(S + 127) / 128, 128, 0, st>>>(w->fmax, t->d.w64, S, Mg, w->jexp,
                                                      w->aexp, w->w16);
    k_tc_slab_prep16<<<(S * kN + 127) / 128, 128, 0, st>>>(t->d.Tm64, t->d.w64, S, Mg, R, R_F,
                                                            periodic, w->jexp, w->aexp, w->FR16,
                                                            w->FW16);
    k_tc_slab_tplanes16<<<1024, 256, 0, st>>>(t->d.Tm64, S, Mg, w->aexp, (__half*)w->T16[0],
                                              (__half*)w->T16[1]);
    if (periodic) k_tc_slab_dbar<<<1, kN, 0, st>>>(t->d.Dbar64, Mg, R, R_F, w->FB16);
    CC_CUDA(cudaGetLastError());
    w->RF16_built = R_F;
  }
  if (!half && w->RF_built != R_F) {
    k_tc_slab_prep<<<(S * kN + 127) / 128, 128, 0, st>>>(t->d.Tm64, t->d.w64, S, Mg, R, R_F,
                                                          periodic, w->FR, w->FW);
    if (periodic) k_tc_slab_dbar<<<1, kN, 0, st>>>(t->d.Dbar64, Mg, R, R_F, w->FB);
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
  a.FR = half ? w->FR16 : w->FR;
  a.FW = half ? w->FW16 : w->FW;
  a.w = half ? w->w16 : w->w32;
  a.aexp = half ? w->aexp : nullptr;
  a.part = w->part;
  a.err = err;
  a.stall_test = stall_test;
  const uint32_t smem = slab_smem_bytes(R_F);
  static uint32_t attr = 0;
  if (attr < smem) {
    const void* ks[] = {(const void*)k_tc_slab<false, false, false>,
                        (const void*)k_tc_slab<false, true, false>,
                        (const void*)k_tc_slab<true, false, false>,
                        (const void*)k_tc_slab<true, true, false>,
                        (const void*)k_tc_slab<false, false, true>,
                        (const void*)k_tc_slab<false, true, true>};
    for (const void* k : ks)
      CC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)slab_smem_bytes(63)));
    attr = slab_smem_bytes(63);
  }
  // the A term on the tensor cores where the band leaves tensor memory free for F_s
  const bool mma_a = periodic && ((R + R_F + 16) & ~15) - ((R - R_F) & ~15) <= kMmaABand;
  if (half) {  // fp16x3 (the hi * hi diagnostic is a bf16 one)
    const CUtensorMap& mh = *reinterpret_cast<const CUtensorMap*>(w->map16_hi);
    const CUtensorMap& ml = *reinterpret_cast<const CUtensorMap*>(w->map16_lo);
    if (mma_a)
      k_tc_slab<true, true, false><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
    else
      k_tc_slab<true, false, false><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
  } else {
    const CUtensorMap& mh =
        *reinterpret_cast<const CUtensorMap*>(w->T128[0] ? (const void*)w->map_hi : map_hi);
    const CUtensorMap& ml =
        *reinterpret_cast<const CUtensorMap*>(w->T128[0] ? (const void*)w->map_lo : map_lo);
    if (mma_a && x1)
      k_tc_slab<false, true, true><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
    else if (mma_a)
      k_tc_slab<false, true, false><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
    else if (x1)
      k_tc_slab<false, false, true><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
    else
      k_tc_slab<false, false, false><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
  }
  CC_CUDA((launch_slab_finalize<kN, 2 * kN, true>(
      Mg, st, (const float*)w->part, (const float*)(half ? w->FB16 : w->FB), R, R_F, S, 1,
      w->units, w->grid, w->maxseg, periodic, t->pref, eps, w->blk_ex, w->ticket, Ex,
      (const int*)err, err + 1)));
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

}  // namespace cc
