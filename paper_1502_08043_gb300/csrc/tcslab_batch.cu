// The batched form of the fused tensor-core exchange kernel of tcslab.cu (bf16 hi + lo):
// many boxes of grid side up to 127 (operands padded to 128) in one launch.
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
// One CTA per SM walks a contiguous run of work units (box, slab pair, node); the boxes of a
// batch follow each other in the unit order and every role reads the parameters of the
// box it is in from a small table.  For every unit:
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
// When every box of the batch is periodic with a band of at most 96 columns, the A term is
// formed on the tensor cores as in tcslab.cu: A_{s,x} = F_s P_x with the one-hot
// P_x[z][h] = [h(x, z) = h] built with R (cleared with R when the box changes), F_s hi and
// lo staged per node into the tensor-memory columns the band leaves free, two more MMAs per
// K step of h <= R_F added to U in MMA1; the epilogue then only scales and re-splits.
//
// Tensor memory (512 columns): [0,128) U_0, [128,256) U_1, [256,384) E_0, [384,512) E_1;
// with the A term on the tensor cores F_s hi in [96,128), lo in [224,256).
// Warps: 0-7 epilogue (warp w: lanes 32 (w % 4) .., columns 64 (w / 4) ..), 8-10 and 12-14
// build R, 11 TMA producer, 15 MMA issuer (converged, one K step per elected asm block; no
// builder shares the MMA warp's scheduler).  Every wait is bounded (global timer); on
// expiry the error word is set, all roles stop, the MMA issuer drains its MMAs and tensor
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
// batches whose boxes are all periodic with bands of at most 96 columns add the A term on
// the tensor cores: A_{s,x} = F_s P_x with the one-hot P_x[z][h] = [h(x, z) = h] (band rows
// of the box, K = h), F_s as bf16 hi and lo in the tensor-memory columns the band leaves
// free in U_0 and U_1
constexpr int kMmaABand = 96;
constexpr uint32_t kOffP = kOffFtab + 2 * kFtabBytes;   // P_x, band rows x 128 bytes
constexpr uint32_t kFhi = 96, kFlo = 224;               // F_s hi / lo columns
constexpr uint32_t kOffBar = kOffP + kMmaABand * 128;  // mbarriers, tensor-memory slot
constexpr int kNumBars = 17;
constexpr uint32_t kOffIsq = kOffBar + 8 * kNumBars + 16;  // floor(sqrt(v)), v <= R_F^2
__host__ __device__ constexpr uint32_t slab_smem_bytes(int R_F) {
  return kOffIsq + (((uint32_t)(R_F * R_F + 1) + 15u) & ~15u) + 1024u;
}

// one box of the launch (element offsets into the shared arrays of Args)
struct SlabBox {
  int R, RF, Mg, S;
  int periodic, frs, fws, ld;  // F row stride (>= R_F + 1), FW/FB row stride, partial row stride
  int t_rpn;                   // rows per node of the T planes (64 or 128)
  long long unit0;             // first work unit of the box
  long long t_row0;            // T plane row of node 0
  long long fr_off;            // FR: [S][Mg + 1][frs] packed bf16 hi | lo of F_s[x][h]
  long long fw_off;            // FW: [S][frs][fws] w_s F_s[y][h] (periodic)
  long long fb_off;            // FB: [frs][fws] window sums of Dbar (periodic)
  long long w_off;             // w:  [S]
  long long part_off;          // part: [pairs][maxseg][2][Mg][ld]
  long long eps_off;           // eps: [Mg][Mg][Mg]
  long long rows0;             // row_ex: [Mg][Mg]
  double pref;
};

struct Args {
  const SlabBox* __restrict__ boxes;  // nbox entries in unit order (batch launches)
  SlabBox b0;
  int nbox, units, maxseg, rf_max;
  const uint32_t* FR;
  const float* FW;
  const float* w;
  float* part;
  int* err;
  int stall_test;
};

// a single box reads its fields straight from the kernel parameters, a batch copies the
// entry of the box it is in from the table in global memory
template <bool kBatch>
__device__ __forceinline__ SlabBox box_ref(const Args& g, int b) {
  if constexpr (kBatch) return g.boxes[b];
  else return g.b0;
}
__device__ __forceinline__ SlabBox get_box(const Args& g, int b) {
  return g.boxes ? g.boxes[b] : g.b0;
}
// the box of unit u, walking forward from box b (units only increase along a CTA's run)
template <bool kBatch>
__device__ __forceinline__ int advance_box(const Args& g, int b, long long u) {
  if constexpr (kBatch)
    while (b + 1 < g.nbox && g.boxes[b + 1].unit0 <= u) ++b;
  return b;
}

// CTA c owns work units [c U / G, (c + 1) U / G); the CTA that owns unit u
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

template <bool kBatch, bool kMmaA>
__global__ void __launch_bounds__(kThreads, 1)
    k_tcb_slab(const __grid_constant__ CUtensorMap mTh, const __grid_constant__ CUtensorMap mTl,
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
  // |y - R|, |z - R| <= R_F of the current box; they clear it when the box changes)
  for (int v = tid; v <= g.rf_max * g.rf_max; v += kThreads) {
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

  const long long u0 = (long long)blockIdx.x * g.units / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * g.units / gridDim.x;
  // U and R vanish outside the band [R - R_F, R + R_F] of z (and of y for R): the products
  // of a box run over its 16-aligned band [zs, ze) only (U column n holds z = zs + n)
  auto band_lo = [](const SlabBox& b) { return (b.R - b.RF) & ~15; };
  auto band_hi = [](const SlabBox& b) { return (b.R + b.RF + 16) & ~15; };

  if (warp == kProdWarp) {
    if (lane == 0) {
      // ---------------- TMA producer: T_s hi + lo, the K blocks of the band, into buffer
      // (unit & 1); rows of the 128-row box past the node's own rows only feed output rows
      // y' >= Mg, which are never read
      uint32_t n = 0;
      int b = 0;
      for (long long u = u0; u < u1 && !s_abort; ++u, ++n) {
        b = advance_box<kBatch>(g, b, u);
        const SlabBox bx = box_ref<kBatch>(g, b);
        const int s = (int)((u - bx.unit0) % bx.S), k = (int)(n & 1u);
        const int kb0 = band_lo(bx) >> 6, kb1 = (band_hi(bx) - 1) >> 6;
        if (!mbar_wait(tfree(k), ((n >> 1) & 1u) ^ 1u, g.err, 11, &s_abort)) {
          s_abort = 1;
          break;
        }
        const uint32_t dst = base + kOffT + k * kOp;
        const int row = (int)(bx.t_row0 + (long long)s * bx.t_rpn);
        mbar_expect_tx(tfull(k), (uint32_t)(kb1 - kb0 + 1) * 2u * kPlane);
        for (int kb = kb0; kb <= kb1; ++kb) {
          tma_load_2d(dst + kb * 2 * kPlane, &mTh, kb * 64, row, tfull(k));
          tma_load_2d(dst + kb * 2 * kPlane + kPlane, &mTl, kb * 64, row, tfull(k));
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
      constexpr uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 4) << 24);
      if (g.stall_test && !all(mbar_wait(never, 0, g.err, 5, nullptr, 20000000ull))) s_abort = 1;
      uint32_t n = 0, r = 0, segc = 0;
      // per box: band [zs, ze) in K steps [ms, me); first MMA N = band width, second MMA
      // N = the grid side rounded up to 16 (columns z' >= Mg are never read).  Descriptors
      // as base + constant: the start-address field holds address / 16, so a byte offset o
      // (all addresses < 256 KB) adds o / 16
      int ms = 0, me = 0, nh = 0;  // nh: K steps of the A-term MMAs (h < 16 nh)
      uint32_t idesc1 = 0, idesc2 = 0;
      uint64_t dR = 0;  // B rows z = zs ..
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
          mma_x3_w(d, dT + o, dR + o, kPl, kPl, idesc1, acc);
        }
        if constexpr (kMmaA) {  // + F_s P_x: A = F_s hi and lo from tensor memory
#pragma unroll
          for (int m = 0; m < 4; ++m)
            if (m < nh)
              mma_x2_ts_w(d, tmem + kFhi + 8u * m, tmem + kFlo + 8u * m, dP + 2u * m, idesc1);
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
          mma_x3_ts_w(d, aH, dT + o, kPl, idesc2, (first && m == ms) ? 0u : 1u);
        }
      };
      bool ok = all(!s_abort);
      int b = 0;
      for (long long u = u0; u < u1 && ok;) {
        b = advance_box<kBatch>(g, b, u);
        const SlabBox bx = box_ref<kBatch>(g, b);
        const long long p = (u - bx.unit0) / bx.S;
        const long long pe = bx.unit0 + (p + 1) * bx.S;
        const long long ue = u1 < pe ? u1 : pe;
        const int U = (int)(ue - u);
        const int zs = band_lo(bx), ze = band_hi(bx);
        ms = zs >> 4;
        me = ze >> 4;
        nh = (kMmaA && bx.periodic) ? (bx.RF + 16) >> 4 : 0;
        idesc1 = idesc0 | ((uint32_t)((ze - zs) >> 3) << 17);
        idesc2 = idesc0 | ((uint32_t)(((bx.Mg + 15) & ~15) >> 3) << 17);
        dR = sdesc(base + kOffR + (uint32_t)zs * 128u);
        for (int i = 0; i < U && ok; ++i, ++n) {
          const uint32_t k = n & 1u, tb = base + kOffT + k * kOp;
          const uint32_t tbp = base + kOffT + (k ^ 1u) * kOp;
          // MMA1(i, 0)
          ok = all(mbar_wait(tfull(k), (n >> 1) & 1u, g.err, 14, &s_abort) &&
                   mbar_wait(rfull, r & 1u, g.err, 15, &s_abort) &&
                   (!kMmaA || mbar_wait(ffull, n & 1u, g.err, 18, &s_abort)));
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
    // builder thread always forms the same 16-byte chunks of a box (row z <= R of the
    // square |y - R|, |z - R| <= R_F, 8 consecutive y) and stores each into both mirror
    // rows, so it keeps their h values in registers (packed bytes) for the whole box.  The
    // row of F_s of a build is written by all builder warps into a replicated table (copy
    // l in bank l) and every element is one conflict-free shared-memory load away.
    const int bw = warp < kProdWarp ? warp - kEpiWarps : warp - kEpiWarps - 1;
    const int bt = 32 * bw + lane;
    constexpr int kMaxTasks = 6;  // (R_F + 1) x chunks <= 64 x 16 = 1024 = 5.3 x 192
    uint32_t hb[kMaxTasks][2];
    int cur = -1, R = 0, RF = 0, zlo = 0, clo = 0, nc = 1, tasks = 0;
    int zsb = 0, nactb = 0, perb = 0, Sb = 1;  // the box's band, kernel and node count
    long long unit0b = 0;
    int p_h = -1;  // the h of this thread's row of P as it stands (-1: zero row)
    auto frow = [&](int b, long long u, int j) {
      const SlabBox bx = box_ref<kBatch>(g, b);
      const long long l = u - bx.unit0;
      return g.FR + bx.fr_off + ((l % bx.S) * (bx.Mg + 1) + 2 * (l / bx.S) + j) * bx.frs;
    };
    // this warp fills entries h = hw0 .. hw0 + 10 (11 per warp, 6 warps cover 64)
    const int hw0 = 11 * bw;
    int bn = advance_box<kBatch>(g, 0, u0);
    uint32_t nf0 = __ldg(frow(bn, u0, 0) + lane), nf1 = __ldg(frow(bn, u0, 0) + lane + 32);
    uint32_t r = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u) {
      const int b = advance_box<kBatch>(g, cur < 0 ? 0 : cur, u);
      const bool fresh = b != cur;
      if (fresh) {
        const SlabBox bx = box_ref<kBatch>(g, b);
        R = bx.R;
        RF = bx.RF;
        zsb = band_lo(bx);
        nactb = band_hi(bx) - zsb;
        perb = bx.periodic;
        Sb = bx.S;
        unit0b = bx.unit0;
        zlo = R - RF;
        clo = (R - RF) >> 3;
        nc = ((R + RF) >> 3) - clo + 1;
        tasks = (RF + 1) * nc;
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
      }
      for (int j = 0; j < 2 && ok; ++j, ++r) {
        const uint32_t f0 = nf0, f1 = nf1;
        const long long un = j == 0 ? u : u + 1;
        if (un < u1) {  // the next build's row
          bn = advance_box<kBatch>(g, b, un);
          nf0 = __ldg(frow(bn, un, j ^ 1) + lane);
          nf1 = __ldg(frow(bn, un, j ^ 1) + lane + 32);
        }
        const bool clear = fresh && j == 0 && cur >= 0;
        if (clear) {
          // a new box: the previous box's square may reach beyond this one's, so the
          // operand is cleared (once it is free) before the table is published
          ok = mbar_wait(rfree, (r & 1u) ^ 1u, g.err, 21, &s_abort);
          if (!ok) break;
          for (uint32_t o = 16u * bt; o < kOp; o += 16u * kBldThreads)
            *reinterpret_cast<uint4*>(gb + kOffR + o) = make_uint4(0u, 0u, 0u, 0u);
          if (kMmaA) {  // and P: its rows are band rows of the previous box
            for (uint32_t o = 16u * bt; o < kMmaABand * 128u; o += 16u * kBldThreads)
              *reinterpret_cast<uint4*>(gb + kOffP + o) = make_uint4(0u, 0u, 0u, 0u);
            p_h = -1;
          }
        }
        // every warp has finished build r - 2, so table (r & 1) is free
        uint32_t* ft = reinterpret_cast<uint32_t*>(gb + kOffFtab + (r & 1u) * kFtabBytes);
#pragma unroll
        for (int i = 0; i < 11; ++i) {
          const int h = hw0 + i;
          const uint32_t a = __shfl_sync(0xffffffffu, f0, h & 31);
          const uint32_t c = __shfl_sync(0xffffffffu, f1, h & 31);
          if (h < kHMax) ft[32 * h + lane] = h < 32 ? a : c;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(ftfull(r & 1u));
        ok = mbar_wait(ftfull(r & 1u), (r >> 1) & 1u, g.err, 22, &s_abort) &&
             (clear || mbar_wait(rfree, (r & 1u) ^ 1u, g.err, 21, &s_abort));
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
          // P_x for x = 2 p + j: band row rr (z = zs + rr) is one-hot (bf16 1) at h(x, z),
          // zero outside the sphere; 16-byte chunk c holds h = 8 c .. 8 c + 7 (128-byte
          // swizzle).  Builder thread rr owns row rr and moves its one.
          if (perb && bt < nactb) {
            const int rr = bt, dz = zsb + rr - R;
            const int dx = (int)(2 * ((u - unit0b) / Sb) + j) - R;
            const int q = RF * RF - dx * dx - dz * dz;
            const int h = q >= 0 ? (int)isq[q] : -1;
            if (p_h >= 0 && p_h != h)
              *reinterpret_cast<uint4*>(gb + kOffP + rr * 128 + (((p_h >> 3) ^ (rr & 7)) << 4)) =
                  make_uint4(0u, 0u, 0u, 0u);
            if (h >= 0 && h != p_h) {
              const uint32_t one = 0x3F80u << (16 * (h & 1)), wi = (uint32_t)(h & 7) >> 1;
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
      cur = b;
    }
    if (!ok) s_abort = 1;
  } else {
    // ---------------- epilogue warps 0-7
    const int quad = warp & 3, half = warp >> 2;
    const int yrow = 32 * quad + lane;
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    uint32_t n = 0, segc = 0;
    bool ok = true;
    int b = 0;
    // the A-term MMAs read F_s of unit uu from tensor memory: lane y, column kFhi + c
    // (kFlo + c) holds the bf16 hi (lo) pair of h = 2 c, 2 c + 1; this warp writes
    // h = 32 half .. 32 half + 31 of its lanes from the box's rows F_s[y][h], y <= Mg,
    // h <= R_F (zero elsewhere), loaded a unit ahead of the staging
    uint32_t fpre[32];
    auto load_f = [&](long long uu, int bb) {
      const SlabBox fx = box_ref<kBatch>(g, bb);
      const long long l = uu - fx.unit0;
      const uint32_t* row = g.FR + fx.fr_off + ((l % fx.S) * (fx.Mg + 1) + yrow) * fx.frs;
      const bool rowok = yrow <= fx.Mg;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int h = 32 * half + i;
        fpre[i] = (rowok && h <= fx.RF) ? __ldg(row + h) : 0u;
      }
    };
    auto stage_f = [&]() {
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        hi[c] = __byte_perm(fpre[2 * c], fpre[2 * c + 1], 0x5410);
        lo[c] = __byte_perm(fpre[2 * c], fpre[2 * c + 1], 0x7632);
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
        load_f(u0, advance_box<kBatch>(g, 0, u0));
        stage_f();
      }
    }
    for (long long u = u0; u < u1 && ok;) {
      b = advance_box<kBatch>(g, b, u);
      const SlabBox bx = box_ref<kBatch>(g, b);
      const int R = bx.R, RF = bx.RF, S = bx.S, zs = band_lo(bx), nact = band_hi(bx) - zs;
      const long long p = (u - bx.unit0) / S;
      const long long pe = bx.unit0 + (p + 1) * S;
      const long long ue = u1 < pe ? u1 : pe;
      // h(x_j, z) for the columns z = zs + 32 cc + lane of this warp's two chunks (fixed
      // for the whole pair; broadcast by shuffle per column), -1 outside the sphere
      int hz[2][2];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int dx = (int)(2 * p + j) - R, dz = zs + 32 * (2 * half + k) + lane - R;
          const int q = RF * RF - dx * dx - dz * dz;
          hz[j][k] = (!kMmaA && q >= 0) ? (int)isq[q] : -1;
        }
      const long long fw_node = (long long)bx.frs * bx.fws;
      const int fws = bx.fws, periodic = bx.periodic;
      const long long unit0 = bx.unit0;
      const float* FWb = g.FW + bx.fw_off;
      const float* wb = g.w + bx.w_off;
      for (; u < ue && ok; ++u, ++n) {
        const int s = (int)((u - unit0) % S);
        const float ws = wb[s];
        const float* FWs = FWb + s * fw_node + yrow;
        if constexpr (kMmaA) {
          if (u + 1 < u1) load_f(u + 1, advance_box<kBatch>(g, b, u + 1));
        }
        if (!kMmaA && periodic && u + 1 < ue) {
          // the next unit's A-term table into L1 ahead of its use
          const long long lines = (fw_node * 4 + 127) / 128;
          if (tid < lines) {
            const float* nx = FWb + (s + 1) * fw_node + tid * 32;
            asm volatile("prefetch.global.L1 [%0];" ::"l"(nx));
          }
        }
        for (int j = 0; j < 2; ++j) {
          // the A-term values of this warp's columns, requested before the MMA result is
          // waited for (their L2 latency hides behind the wait): both 32-column chunks for a
          // single box; for a batch (box fields held in registers) the second chunk's right
          // after the first chunk is converted
          constexpr int kAC = kBatch ? 1 : 2;
          float a[kAC][32];
          auto load_a = [&](int k) {
            const int hzk = j == 0 ? hz[0][k] : hz[1][k];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int h = __shfl_sync(0xffffffffu, hzk, e);
              a[kBatch ? 0 : k][e] = (periodic && h >= 0) ? __ldg(FWs + h * fws) : 0.0f;
            }
          };
          if constexpr (!kMmaA) {
            load_a(0);
            if (!kBatch) load_a(1);
          }
          ok = mbar_wait(d1full(j), n & 1u, g.err, 31, &s_abort);
          if (!ok) break;
          tc_fence_after();
          // the unit's second first mode product is done with F_s: the next unit's goes
          // into tensor memory (the MMA warp waits for it before that unit's first MMA)
          if constexpr (kMmaA) {
            if (j == 1 && u + 1 < u1) stage_f();
          }
          // in place, 16 columns at a time: FP32 U of the piece z = zs + 16 m .. in columns
          // 16 m .. 16 m + 15 becomes 8 columns of bf16 hi pairs followed by 8 of lo pairs
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            if (!kMmaA && kBatch && k == 1) load_a(1);
#pragma unroll
            for (int sub = 0; sub < 2; ++sub) {
              if (32 * (2 * half + k) + 16 * sub >= nact) continue;  // beyond the band
              const uint32_t ta = tmem + lane_off +
                                  (uint32_t)(j * 128 + 32 * (2 * half + k) + 16 * sub);
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
                  x0 = fmaf(__uint_as_float(v[e]), ws, a[kBatch ? 0 : k][16 * sub + e]);
                  x1 = fmaf(__uint_as_float(v[e + 1]), ws, a[kBatch ? 0 : k][16 * sub + e + 1]);
                }
                const uint32_t h = pack_bf16x2(x0, x1);
                hi[e >> 1] = h;
                lo[e >> 1] = pack_bf16x2(x0 - bf16_lo_f(h), x1 - bf16_hi_f(h));
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
      // the pair's E leaves tensor memory once, as a partial of this CTA: rows y < Mg,
      // columns z' < ld (a multiple of 4 within the computed N = Mg rounded up to 16)
      ok = mbar_wait(efull, segc & 1u, g.err, 32, &s_abort);
      if (!ok) break;
      tc_fence_after();
      const int kseg = (int)blockIdx.x - owner_cta(bx.unit0 + p * S, g.units, gridDim.x);
      float* P = g.part + bx.part_off +
                 (long long)((p * g.maxseg + kseg) * 2) * bx.Mg * bx.ld;
      for (int j = 0; j < 2; ++j) {
#pragma unroll 1
        for (int cc = 2 * half; cc < 2 * half + 2; ++cc) {
          if (32 * cc >= bx.ld) continue;  // warp-uniform
          uint32_t v[32];
          tmem_ld32(tmem + lane_off + (uint32_t)(256 + j * 128 + 32 * cc), v);
          if (yrow < bx.Mg) {
            float4* o = reinterpret_cast<float4*>(P + ((long long)j * bx.Mg + yrow) * bx.ld +
                                                  32 * cc);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (32 * cc + 4 * e < bx.ld)
                o[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                   __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
          }
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
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }
}

// F_s window sums (FP64) of every row a <= Mg (row Mg: zero, the padding slab of an odd
// grid): the bf16 hi | lo pairs for the R operand and, periodic, w_s F_s transposed for the
// A term.  One thread per (s, a).
__global__ void k_tcb_prep(const double* Tm, const double* w, int S, int Mg, int R, int RF,
                               int periodic, int frs, int fws, uint32_t* FR, float* FW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * (Mg + 1)) return;
  const int s = i / (Mg + 1), a = i % (Mg + 1);
  const double* row = Tm + ((long long)s * Mg + (a < Mg ? a : 0)) * Mg;
  auto X = [&](int k) { return (periodic && k == a) ? 0.0 : row[k]; };
  double acc = 0.0;
  for (int h = 0; h < frs; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? X(R) : X(R - h) + X(R + h);
      f = acc;
    }
    const __nv_bfloat16 hb = __double2bfloat16(f);
    const __nv_bfloat16 lb = __double2bfloat16(f - (double)__bfloat162float(hb));
    FR[(long long)i * frs + h] = (uint32_t)__bfloat16_as_ushort(hb) |
                                 ((uint32_t)__bfloat16_as_ushort(lb) << 16);
    if (periodic && a < fws) FW[((long long)s * frs + h) * fws + a] = (float)(w[s] * f);
  }
}

// window sums of Dbar (I x I x Dbar term), FB[h][z'] = sum_{k=R-h}^{R+h} Dbar[z'][k]
__global__ void k_tcb_dbar(const double* Dbar, int Mg, int R, int RF, int frs, int fws,
                               float* FB) {
  const int a = threadIdx.x;
  if (a >= fws) return;
  double acc = 0.0;
  for (int h = 0; h < frs; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? Dbar[a * Mg + R] : Dbar[a * Mg + R - h] + Dbar[a * Mg + R + h];
      f = acc;
    }
    FB[h * fws + a] = (float)f;
  }
}

__device__ __forceinline__ int isqrt_int(int v) {
  int h = (int)sqrtf((float)v);
  while (h * h > v) --h;
  while ((h + 1) * (h + 1) <= v) ++h;
  return h;
}

// one warp per grid row (box, x, y) of the flattened rows of all boxes, four z per lane:
// partials of the pair in order, + Dbar term, eps on the basis sphere; FP64 sum of the
// row's eps over the Fermi sphere (fixed butterfly order)
__global__ void __launch_bounds__(256)
    k_tcb_finalize(Args g, int kgrid, const float* FB, long long rows, float* eps,
                       double* row_ex) {
  const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;  // whole warps
  int lo = 0, hi = g.nbox - 1;  // the box whose rows hold r
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.boxes[mid].rows0 <= r) lo = mid;
    else hi = mid - 1;
  }
  const SlabBox bx = get_box(g, lo);
  const int R = bx.R, RF = bx.RF, Mg = bx.Mg, S = bx.S;
  const int x = (int)((r - bx.rows0) / Mg), y = (int)((r - bx.rows0) % Mg);
  const int p = x >> 1, j = x & 1;
  const int c0 = owner_cta(bx.unit0 + (long long)p * S, g.units, kgrid);
  const int nseg = owner_cta(bx.unit0 + (long long)(p + 1) * S - 1, g.units, kgrid) - c0 + 1;
  const int dx = x - R, dy = y - R;
  const int qb = RF * RF - dx * dx - dy * dy;  // z line at (x, y) for the Dbar term
  const float* fb = (bx.periodic && qb >= 0) ? FB + bx.fb_off + isqrt_int(qb) * bx.fws : nullptr;
  const long long slab = (long long)Mg * bx.ld;
  const float* pp = g.part + bx.part_off + ((long long)p * g.maxseg * 2 + j) * slab +
                    (long long)y * bx.ld;
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int z = lane + 32 * i;
    if (z >= Mg) continue;
    float sum = 0.0f;
    for (int k = 0; k < nseg; ++k) sum += __ldg(pp + (long long)k * 2 * slab + z);
    if (fb) sum += __ldg(fb + z);
    const int dz = z - R, m = dx * dx + dy * dy + dz * dz;
    const float v = m <= R * R ? (float)(-bx.pref * (double)sum) : 0.0f;
    eps[bx.eps_off + ((long long)x * Mg + y) * Mg + z] = v;
    if (m <= RF * RF) acc += (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) row_ex[r] = acc;
}

// E_x of box blockIdx.x from its Mg^2 row sums, fixed order: thread t adds rows t,
// t + 1024, ..., then a tree
__global__ void __launch_bounds__(1024)
    k_tcb_ex(Args g, const double* row_ex, double* Ex, const int* err, int* status) {
  __shared__ double red[1024];
  const SlabBox bx = get_box(g, blockIdx.x);
  const long long n = (long long)bx.Mg * bx.Mg;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += 1024) acc += row_ex[bx.rows0 + i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Ex[2 * blockIdx.x] = 0.5 * red[0];
    Ex[2 * blockIdx.x + 1] = red[0];
    if (status && blockIdx.x == 0) *status = *err;
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

namespace {

// The arrays and the box table of one batch launch (fixed Fermi radii).  T planes are the
// step chain's ([nodes x 64][64] bf16 hi, lo, concatenated over boxes), read through maps
// with 128-row boxes: rows past a node only feed output rows y' >= Mg, never read.
struct SlabPlan {
  int grid = 0, units = 0, maxseg = 0, rf_max = 0, nbox = 0;
  bool mma_a = false;  // every box periodic with a band of at most 96 columns
  long long rows = 0;
  uint32_t* FR = nullptr;
  float* FW = nullptr;
  float* FB = nullptr;
  float* part = nullptr;
  double* row_ex = nullptr;
  float* w32 = nullptr;
  SlabBox* boxes_dev = nullptr;
  alignas(64) unsigned char map_hi[128], map_lo[128];
  std::vector<void*> allocs;
};

cc_status plan_alloc(SlabPlan* w, void** p, size_t bytes, cc_tables t) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_last_error("cudaMalloc(tensor-core slab workspace)", e);
    return CC_ERR_ALLOC;
  }
  w->allocs.push_back(*p);
  if (t) {
    t->ws.mx_bytes += bytes;
    t->device_bytes += bytes;
  }
  return CC_OK;
}

// the fixed geometry of box b: units, strides; offsets are filled by the caller
SlabBox box_geometry(cc_tables t, int R_F, int frs, int t_rpn) {
  SlabBox b{};
  b.R = t->p.R;
  b.RF = R_F;
  b.Mg = t->Mg;
  b.S = t->S_eff;
  b.periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  b.frs = frs;
  b.fws = (t->Mg + 3) & ~3;
  b.ld = b.fws;
  b.t_rpn = t_rpn;
  b.pref = t->pref;
  return b;
}

// units, grid and segments per pair of a list of boxes (unit0 filled in)
void plan_partition(SlabPlan* w, std::vector<SlabBox>& boxes) {
  long long units = 0;
  for (auto& b : boxes) {
    b.unit0 = units;
    units += (long long)((b.Mg + 1) / 2) * b.S;
  }
  w->units = (int)units;
  w->grid = (int)std::min<long long>(sm_count(), units);
  w->maxseg = 1;
  for (const auto& b : boxes)
    for (int p = 0; p < (b.Mg + 1) / 2; ++p) {
      const int c0 = owner_cta(b.unit0 + (long long)p * b.S, w->units, w->grid);
      const int c1 = owner_cta(b.unit0 + (long long)(p + 1) * b.S - 1, w->units, w->grid);
      w->maxseg = std::max(w->maxseg, c1 - c0 + 1);
    }
}

// element offsets of every box in the shared arrays; returns the array sizes
void plan_offsets(SlabPlan* w, std::vector<SlabBox>& boxes, long long* nFR, long long* nFW,
                  long long* nFB, long long* nW, long long* nPart) {
  long long fr = 0, fw = 0, fb = 0, ww = 0, part = 0, rows = 0;
  for (auto& b : boxes) {
    b.fr_off = fr;
    b.fw_off = fw;
    b.fb_off = fb;
    b.w_off = ww;
    b.part_off = part;
    b.rows0 = rows;
    fr += (long long)b.S * (b.Mg + 1) * b.frs;
    fw += (long long)b.S * b.frs * b.fws;
    fb += (long long)b.frs * b.fws;
    ww += b.S;
    part += (long long)((b.Mg + 1) / 2) * w->maxseg * 2 * b.Mg * b.ld;  // multiple of 4
    rows += (long long)b.Mg * b.Mg;
  }
  w->rows = rows;
  *nFR = fr + 64;    // the builders read 64 words from any row start
  *nFW = fw + 128;   // the epilogue reads up to 128 rows of the last table
  *nFB = fb;
  *nW = ww;
  *nPart = part;
}

cc_status plan_arrays(SlabPlan* w, long long nFR, long long nFW, long long nFB, long long nW,
                      long long nPart, cc_tables t) {
  CC_TRY(plan_alloc(w, (void**)&w->FR, sizeof(uint32_t) * nFR, t));
  CC_TRY(plan_alloc(w, (void**)&w->FW, sizeof(float) * nFW, t));
  CC_TRY(plan_alloc(w, (void**)&w->FB, sizeof(float) * std::max<long long>(nFB, 1), t));
  CC_TRY(plan_alloc(w, (void**)&w->part, sizeof(float) * nPart, t));
  CC_TRY(plan_alloc(w, (void**)&w->row_ex, sizeof(double) * w->rows, t));
  CC_TRY(plan_alloc(w, (void**)&w->w32, sizeof(float) * nW, t));
  CC_CUDA(cudaMemset(w->FR, 0, sizeof(uint32_t) * nFR));
  CC_CUDA(cudaMemset(w->FW, 0, sizeof(float) * nFW));
  return CC_OK;
}

// node weights of box t at offset off
cc_status plan_weights(SlabPlan* w, cc_tables t, long long off) {
  std::vector<float> w32(t->S_eff);
  for (int i = 0; i < t->S_eff; ++i) w32[i] = (float)t->w[t->kept_idx[i]];
  CC_CUDA(cudaMemcpy(w->w32 + off, w32.data(), sizeof(float) * t->S_eff,
                     cudaMemcpyHostToDevice));
  return CC_OK;
}

// window sums of box t (Fermi radius b.RF) into the box's slices
cc_status plan_prep(SlabPlan* w, cc_tables t, const SlabBox& b, cudaStream_t st) {
  const int n = b.S * (b.Mg + 1);
  k_tcb_prep<<<(n + 127) / 128, 128, 0, st>>>(t->d.Tm64, t->d.w64, b.S, b.Mg, b.R, b.RF,
                                                  b.periodic, b.frs, b.fws, w->FR + b.fr_off,
                                                  w->FW + b.fw_off);
  if (b.periodic)
    k_tcb_dbar<<<1, 128, 0, st>>>(t->d.Dbar64, b.Mg, b.R, b.RF, b.frs, b.fws,
                                      w->FB + b.fb_off);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

cc_status plan_maps(SlabPlan* w, void* tt_hi, void* tt_lo, long long rows, int Np) {
  static_assert(sizeof(CUtensorMap) <= 128, "tensor map size");
  CC_TRY(tc_make_map_bf16(w->map_hi, tt_hi, rows, Np, kN));
  CC_TRY(tc_make_map_bf16(w->map_lo, tt_lo, rows, Np, kN));
  return CC_OK;
}

cc_status plan_launch(SlabPlan* w, int* err, int stall_test, float* eps, double* Ex,
                      cudaStream_t st) {
  Args a{};
  a.boxes = w->boxes_dev;
  a.nbox = w->nbox;
  a.units = w->units;
  a.maxseg = w->maxseg;
  a.rf_max = w->rf_max;
  a.FR = w->FR;
  a.FW = w->FW;
  a.w = w->w32;
  a.part = w->part;
  a.err = err;
  a.stall_test = stall_test;
  const uint32_t smem = slab_smem_bytes(w->rf_max);
  const CUtensorMap& mh = *reinterpret_cast<const CUtensorMap*>(w->map_hi);
  const CUtensorMap& ml = *reinterpret_cast<const CUtensorMap*>(w->map_lo);
  if (w->mma_a)
    k_tcb_slab<true, true><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
  else
    k_tcb_slab<true, false><<<w->grid, kThreads, smem, st>>>(mh, ml, a);
  k_tcb_finalize<<<(unsigned)((w->rows + 7) / 8), 256, 0, st>>>(a, w->grid, w->FB, w->rows,
                                                                    eps, w->row_ex);
  k_tcb_ex<<<w->nbox, 1024, 0, st>>>(a, w->row_ex, Ex, err, err + 1);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

cc_status set_smem_attr() {
  static bool done = false;
  if (!done) {
    CC_CUDA(cudaFuncSetAttribute(k_tcb_slab<true, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)slab_smem_bytes(63)));
    CC_CUDA(cudaFuncSetAttribute(k_tcb_slab<true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)slab_smem_bytes(63)));
    done = true;
  }
  return CC_OK;
}

}  // namespace

static bool box_supported(cc_tables t) { return t->Mg <= 127 && t->p.R <= 63; }

void tc_slab_batch_free(void* p) {
  SlabPlan* w = reinterpret_cast<SlabPlan*>(p);
  if (!w) return;
  for (void* a : w->allocs) cudaFree(a);
  delete w;
}

cc_status tc_slab_batch_create(const std::vector<cc_tables>& tabs, const std::vector<int>& R_F,
                               const std::vector<long long>& eps_off, void* tt_hi, void* tt_lo,
                               long long tt_rows, const std::vector<long long>& t_row0, int Np,
                               void** out) {
  *out = nullptr;
  const int nb = (int)tabs.size();
  SlabPlan* w = new (std::nothrow) SlabPlan();
  if (!w) return CC_ERR_ALLOC;
  std::vector<SlabBox> boxes;
  cc_status st = CC_OK;
  for (int b = 0; b < nb; ++b) {
    if (!box_supported(tabs[b]) || R_F[b] > 63 || R_F[b] < 1 || R_F[b] > tabs[b]->p.R)
      st = CC_ERR_NOTSUPP;
    boxes.push_back(box_geometry(tabs[b], R_F[b], R_F[b] + 1, Np));
    boxes.back().t_row0 = t_row0[b];
    boxes.back().eps_off = eps_off[b];
    w->rf_max = std::max(w->rf_max, R_F[b]);
  }
  w->mma_a = true;
  for (const SlabBox& bx : boxes)
    if (!bx.periodic || ((bx.R + bx.RF + 16) & ~15) - ((bx.R - bx.RF) & ~15) > kMmaABand)
      w->mma_a = false;
  if (st == CC_OK) {
    plan_partition(w, boxes);
    long long nFR, nFW, nFB, nW, nPart;
    plan_offsets(w, boxes, &nFR, &nFW, &nFB, &nW, &nPart);
    w->nbox = nb;
    st = plan_arrays(w, nFR, nFW, nFB, nW, nPart, nullptr);
  }
  for (int b = 0; b < nb && st == CC_OK; ++b) {
    st = plan_weights(w, tabs[b], boxes[b].w_off);
    if (st == CC_OK) st = plan_prep(w, tabs[b], boxes[b], 0);
  }
  if (st == CC_OK) st = plan_alloc(w, (void**)&w->boxes_dev, sizeof(SlabBox) * nb, nullptr);
  if (st == CC_OK &&
      cudaMemcpy(w->boxes_dev, boxes.data(), sizeof(SlabBox) * nb, cudaMemcpyHostToDevice) !=
          cudaSuccess)
    st = CC_ERR_CUDA;
  if (st == CC_OK) st = plan_maps(w, tt_hi, tt_lo, tt_rows, Np);
  if (st == CC_OK) st = set_smem_attr();
  if (st == CC_OK && cudaDeviceSynchronize() != cudaSuccess) st = CC_ERR_CUDA;
  if (st != CC_OK) {
    tc_slab_batch_free(w);
    return st;
  }
  *out = w;
  return CC_OK;
}

cc_status tc_slab_batch_run(void* p, int* err, float* eps, double* Ex, cudaStream_t st) {
  SlabPlan* w = reinterpret_cast<SlabPlan*>(p);
  if (!w) return CC_ERR_NOTSUPP;
  return plan_launch(w, err, 0, eps, Ex, st);
}

}  // namespace cc
