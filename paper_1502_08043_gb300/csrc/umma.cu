// Mixed-precision exchange mode products on the 5th-generation tensor cores (tcgen05):
// the step chain below (fp16x3, the batched engine, and bf16x3 on request) and the routing
// to the fused slab kernel of tcslab.cu (bf16x3 single boxes, grid side up to 127).
//
// Same sums as exchange.cu (Sec. III exchange of the uniform electron gas, node sum of
// Sec. II Eq. 14 with the D = T - I split for the periodic kernel), reordered so that
// every contraction is a dense GEMM whose two operands are K-major in memory:
//   step 5 (once)  E[x][y][z']  = sum_z O[x][y][z] Dbar[z'][z]            (I x I x D)
//   per node s (Dx = D_s periodic, T_s box):
//   step 1  R_s[x][y][z]   = sum_x' Dx[x][x'] O[x'][y][z]               (x mode first)
//   step 2  W1_s[x][z'][y] = sum_z T_s[z'][z] R_s[x][y][z]               (z mode)
//   step 3  W2_s[x][z'][y] = sum_z T_s[z'][z] O[x][y][z]                 (z mode)
//   step 4  E[x][y'][z'] += sum_s sum_y (w T_s)[y'][y] W1_s[x][z'][y]
//                                   + (w D_s)[y'][y] W2_s[x][z'][y]     (y mode)
// which is D x T x T + I x D x T + I x I x D (mode products commute).  The box kernel
// keeps only W1 with Dx = T_s and no step 3 / step 5.
// Every GEMM has a 128-row operand A (rows of an Np^2 x Np slab stack) and an Np x Np
// operand B (a Toeplitz matrix), Np = 64 or 128 (the grid side padded with zeros).
// Operands are bf16 (or fp16) hi + lo planes: x = hi + lo with hi = bf16(x),
// lo = bf16(x - hi); the product keeps hi*hi + hi*lo + lo*hi (3 MMAs, the lo*lo term is
// below 2^-18 relative for bf16, 2^-22 for fp16).  fp16 has a narrow exponent range,
// so its y-mode operands carry a per-node power-of-two scale (see build_planes).  Intermediates leave TMEM as FP32, are re-split into hi + lo (the FP32
// residual x - hi carried as the correction operand) and stored for the next GEMM.
// O, O^T are exact in bf16 (0/1) and have no lo plane.
//
// Kernel anatomy (persistent: one CTA per SM walks 128 x Np output tiles, 6 warps):
//   warp 4 / lane 0  TMA producer: 2D tiled cp.async.bulk.tensor loads of 64-wide K
//                    blocks (128-byte swizzle) into a 3-stage shared-memory ring that
//                    runs on across tiles;
//   warp 5 / lane 0  MMA issuer: tcgen05.mma.cta_group::1.kind::f16, M = 128, N = Np,
//                    K = 16 per instruction, FP32 accumulators in TMEM (two of them, used
//                    alternately); tcgen05.commit frees a ring slot when its MMAs have
//                    read it and hands a finished accumulator to the epilogue;
//   warps 0-3        allocate / free 2 Np TMEM columns; epilogue: tcgen05.ld 32 lanes x 32
//                    columns, scale, store FP32 (accumulation by reductions) or split into
//                    hi / lo planes, then release the accumulator.
// Every mbarrier wait is bounded by the global timer (about 2 s); on expiry the kernel
// sets an error word, the other roles of the CTA stop waiting, and the CTA returns through
// the normal teardown (TMEM freed), leaving the context usable.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <type_traits>
#include <vector>

#include "internal.cuh"
#include "tc_prims.cuh"

namespace cc {

// ------------------------------------------------------------------ the GEMM kernel
struct TcArgs {
  int m_tiles, batches; // output tiles: m_tiles 128-row tiles in each of `batches`
  int nk;               // 64-wide K blocks per product
  int J;                // products stacked along K (accumulated in one TMEM tile)
  long long a_base, a_sb, a_sj;  // A row of (batch b, product j): base + b*sb + j*sj (+ m0)
  long long b_base, b_sb, b_sj;
  int a_lo, b_lo;       // lo planes present
  int out_split;        // 0: FP32 output, 1: hi/lo planes of E
  int beta;             // FP32 output: accumulate into the existing value
  void* out;
  void* out_lo;
  long long o_base, o_sb;              // element offset of batch b
  long long s_mhi, s_mlo, s_n;         // element (m, n) -> (m / Np) s_mhi + (m % Np) s_mlo + n s_n
  const float* scale;   // per-batch factor applied before the store (nullptr: 1)
  // optional per-batch table (overrides the affine forms above): for batch b,
  // btab[4b] = A row base, btab[4b+1] = B row base, btab[4b+2] = output element offset,
  // btab[4b+3] = number of stacked products J_b
  const long long* btab;
  int stall_test;  // test hook: the MMA warp first waits on a barrier nothing arrives at
  // tile_b (Np = 128 only): the tile index walks the rows of B (N side) instead of A;
  // output element (m, n) of tile `tile` goes to obase + tile*s_tile + m*s_mlo + n*s_n
  int tile_b;
  long long s_tile;
  // resident (J = 1, not tile_b): a CTA takes a contiguous run of tiles; the fixed N-side
  // operand of a batch (all K blocks, hi and lo) is loaded once and stays in shared
  // memory while only the M-side tiles stream through a ring of A slots
  int resident;
  int* err;
};

struct TcBatch {
  long long abase, bbase, obase;
  int J;
};

__device__ __forceinline__ TcBatch tc_batch(const TcArgs& g, int b) {
  if (g.btab) {
    const long long* e = g.btab + 4 * b;
    return {e[0], e[1], e[2], (int)e[3]};
  }
  return {g.a_base + b * g.a_sb, g.b_base + b * g.b_sb, g.o_base + b * g.o_sb, g.J};
}

constexpr int kStages = 3;
constexpr int kTileM = 128;
constexpr int kKB = 64;  // K elements per block = one 128-byte swizzle atom of 16-bit values
constexpr int kTcThreads = 192;  // warps 0-3 epilogue, warp 4 TMA producer, warp 5 MMA issuer

template <int NP>
struct TcSmem {
  static constexpr int kA = kTileM * kKB * 2;  // 16 KB
  static constexpr int kB = NP * kKB * 2;      // 8 / 16 KB
  static constexpr int kStage = 2 * kA + 2 * kB;
  static constexpr int kBytes = kStages * kStage + 1024 /*barriers*/ + 1024 /*alignment*/;
};

// Persistent, warp-specialised GEMM: CTA c takes output tiles c, c + grid, ... of the
// m_tiles x batches tile space.  The producer streams operands through a kStages ring
// continuously across tiles; the MMA warp alternates between two TMEM accumulators so
// that the epilogue of one tile overlaps the MMAs (and loads) of the next.
template <int NP, typename E>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mAlo,
              const __grid_constant__ CUtensorMap mB, const __grid_constant__ CUtensorMap mBlo,
              TcArgs g) {
  using L = TcSmem<NP>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned ring (swizzle atoms)
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t bar0 = base + kStages * L::kStage;
  constexpr int kRing = 4;  // barrier slots (3 used by the normal ring, 4 by the resident one)
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (kRing + s); };
  auto tfull = [&](int a) { return bar0 + 8u * (2 * kRing + a); };
  auto tempty = [&](int a) { return bar0 + 8u * (2 * kRing + 2 + a); };
  const uint32_t never = bar0 + 8u * (2 * kRing + 4);
  const uint32_t a_full = bar0 + 8u * (2 * kRing + 5);
  const uint32_t a_empty = bar0 + 8u * (2 * kRing + 6);
  uint32_t* tmem_slot =
      reinterpret_cast<uint32_t*>(gbase + kStages * L::kStage + 8 * (2 * kRing + 7));
  // resident mode: the N-side operand at base (nk x (hi, lo) of kB), ring of A slots after it
  const uint32_t rb = base;
  constexpr int kResBytes = 2 * 2 * L::kB;  // up to two K blocks of hi + lo
  const uint32_t ring0 = base + (uint32_t)kResBytes;
  constexpr int kResSlots0 = (kStages * L::kStage - kResBytes) / (2 * L::kA);
  constexpr int kResSlots = kResSlots0 < kRing ? kResSlots0 : kRing;
  static_assert(kResSlots >= 2, "resident ring");
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = g.m_tiles * g.batches;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kRing; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(a_full, 1);
    mbar_init(a_empty, 1);
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull(a), 1);
      mbar_init(tempty(a), 4);  // one arrival per epilogue warp
    }
    mbar_init(never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * NP))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // tiles of this CTA: strided, or a contiguous run in resident mode
  int t_first = blockIdx.x, t_step = gridDim.x, t_end = total;
  if (g.resident) {
    const int per = (total + gridDim.x - 1) / gridDim.x;
    t_first = blockIdx.x * per;
    t_step = 1;
    t_end = min(total, t_first + per);
  }

  if (warp == 4) {
    if (lane == 0) {
      // ---------------- TMA producer
      const uint32_t bytes = (uint32_t)(L::kA * (g.a_lo ? 2 : 1) + L::kB * (g.b_lo ? 2 : 1));
      uint32_t n = 0;
      if (g.resident) {
        const uint32_t rbytes = (uint32_t)(g.nk * L::kB * (g.b_lo ? 2 : 1));
        const uint32_t abytes = (uint32_t)(L::kA * (g.a_lo ? 2 : 1));
        uint32_t loads = 0;
        int cur = -1;
        for (int t = t_first; t < t_end && !s_abort; t += t_step) {
          const int b = t / g.m_tiles;
          const TcBatch bt = tc_batch(g, b);
          const long long m0 = (long long)(t % g.m_tiles) * kTileM;
          if (b != cur) {
            if (!mbar_wait(a_empty, (loads & 1u) ^ 1u, g.err, 6, &s_abort)) {
              s_abort = 1;
              break;
            }
            mbar_expect_tx(a_full, rbytes);
            for (int kb = 0; kb < g.nk; ++kb) {
              tma_load_2d(rb + kb * 2 * L::kB, &mB, kb * kKB, (int)bt.bbase, a_full);
              if (g.b_lo) tma_load_2d(rb + kb * 2 * L::kB + L::kB, &mBlo, kb * kKB, (int)bt.bbase, a_full);
            }
            cur = b;
            ++loads;
          }
          for (int kb = 0; kb < g.nk; ++kb, ++n) {
            const int s = (int)(n % kResSlots);
            const uint32_t ph = (n / kResSlots) & 1u;
            if (!mbar_wait(empty(s), ph ^ 1u, g.err, 1, &s_abort)) {
              s_abort = 1;
              break;
            }
            const uint32_t st = ring0 + s * 2 * L::kA;
            mbar_expect_tx(full(s), abytes);
            tma_load_2d(st, &mA, kb * kKB, (int)(bt.abase + m0), full(s));
            if (g.a_lo) tma_load_2d(st + L::kA, &mAlo, kb * kKB, (int)(bt.abase + m0), full(s));
          }
        }
      }
      for (int t = blockIdx.x; t < total && !s_abort && !g.resident; t += gridDim.x) {
        const int b = t / g.m_tiles;
        const TcBatch bt = tc_batch(g, b);
        const int iters = bt.J * g.nk;
        const long long m0 = (long long)(t % g.m_tiles) * kTileM;
        for (int it = 0; it < iters; ++it, ++n) {
          const int s = (int)(n % kStages);
          const uint32_t ph = (n / kStages) & 1u;
          if (!mbar_wait(empty(s), ph ^ 1u, g.err, 1, &s_abort)) {
            s_abort = 1;
            break;
          }
          const int j = it / g.nk, kb = it % g.nk;
          const int arow = (int)(bt.abase + j * g.a_sj + (g.tile_b ? 0 : m0));
          const int brow = (int)(bt.bbase + j * g.b_sj + (g.tile_b ? m0 : 0));
          const uint32_t st = base + s * L::kStage;
          mbar_expect_tx(full(s), bytes);
          tma_load_2d(st, &mA, kb * kKB, arow, full(s));
          if (g.a_lo) tma_load_2d(st + L::kA, &mAlo, kb * kKB, arow, full(s));
          tma_load_2d(st + 2 * L::kA, &mB, kb * kKB, brow, full(s));
          if (g.b_lo) tma_load_2d(st + 2 * L::kA + L::kB, &mBlo, kb * kKB, brow, full(s));
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t fmt = std::is_same<E, __nv_bfloat16>::value ? 1u : 0u;
      constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) |
                                 ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
      uint32_t n = 0, lt = 0;
      if (g.stall_test && !mbar_wait(never, 0, g.err, 5, nullptr, 20000000ull)) s_abort = 1;
      if (g.resident) {
        uint32_t loads = 0;
        int cur = -1;
        for (int t = t_first; t < t_end && !s_abort; t += t_step, ++lt) {
          const int b = t / g.m_tiles;
          if (b != cur) {
            if (cur >= 0) mma_commit(a_empty);  // frees the old operand once its MMAs finish
            if (!mbar_wait(a_full, loads & 1u, g.err, 7, &s_abort)) {
              s_abort = 1;
              break;
            }
            ++loads;
            cur = b;
          }
          const uint32_t acc = lt & 1u, use = lt >> 1;
          if (!mbar_wait(tempty(acc), (use & 1u) ^ 1u, g.err, 4, &s_abort)) {
            s_abort = 1;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + acc * (uint32_t)NP;
          bool ok = true;
          for (int kb = 0; kb < g.nk; ++kb, ++n) {
            const int s = (int)(n % kResSlots);
            const uint32_t ph = (n / kResSlots) & 1u;
            if (!mbar_wait(full(s), ph, g.err, 2, &s_abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = ring0 + s * 2 * L::kA;
            const uint64_t dA = sdesc(st), dAl = sdesc(st + L::kA);
            const uint64_t dB = sdesc(rb + kb * 2 * L::kB), dBl = sdesc(rb + kb * 2 * L::kB + L::kB);
#pragma unroll
            for (int k = 0; k < kKB / 16; ++k) {
              const uint64_t adv = (uint64_t)((k * 32) >> 4);
              mma_f16(d, dA + adv, dB + adv, idesc, (kb > 0 || k > 0) ? 1u : 0u);
              if (g.b_lo) mma_f16(d, dA + adv, dBl + adv, idesc, 1u);
              if (g.a_lo) mma_f16(d, dAl + adv, dB + adv, idesc, 1u);
            }
            mma_commit(empty(s));
          }
          if (!ok) {
            s_abort = 1;
            break;
          }
          mma_commit(tfull(acc));
        }
      }
      for (int t = blockIdx.x; t < total && !s_abort && !g.resident; t += gridDim.x, ++lt) {
        const uint32_t acc = lt & 1u, use = lt >> 1;
        if (!mbar_wait(tempty(acc), (use & 1u) ^ 1u, g.err, 4, &s_abort)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + acc * (uint32_t)NP;
        const int iters = tc_batch(g, t / g.m_tiles).J * g.nk;
        bool ok = true;
        for (int it = 0; it < iters; ++it, ++n) {
          const int s = (int)(n % kStages);
          const uint32_t ph = (n / kStages) & 1u;
          if (!mbar_wait(full(s), ph, g.err, 2, &s_abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + s * L::kStage;
          const uint64_t dA = sdesc(st), dAl = sdesc(st + L::kA);
          const uint64_t dB = sdesc(st + 2 * L::kA), dBl = sdesc(st + 2 * L::kA + L::kB);
#pragma unroll
          for (int k = 0; k < kKB / 16; ++k) {
            const uint64_t adv = (uint64_t)((k * 32) >> 4);  // 32 bytes per K = 16 step
            mma_f16(d, dA + adv, dB + adv, idesc, (it > 0 || k > 0) ? 1u : 0u);
            if (g.b_lo) mma_f16(d, dA + adv, dBl + adv, idesc, 1u);
            if (g.a_lo) mma_f16(d, dAl + adv, dB + adv, idesc, 1u);
          }
          mma_commit(empty(s));
        }
        if (!ok) {
          s_abort = 1;
          break;
        }
        mma_commit(tfull(acc));
      }
    }
  } else {
    // ---------------- epilogue (warps 0-3; warp w owns TMEM lanes 32w .. 32w + 31)
    uint32_t lt = 0;
    for (int t = t_first; t < t_end; t += t_step, ++lt) {
      const uint32_t acc = lt & 1u, use = lt >> 1;
      const bool have = mbar_wait(tfull(acc), use & 1u, g.err, 3, &s_abort);
      tc_fence_after();
      if (!have || s_abort) break;
      const int b = t / g.m_tiles;
      const int tile = t % g.m_tiles;
      const long long m = g.tile_b ? (long long)(warp * 32 + lane)
                                   : (long long)tile * kTileM + warp * 32 + lane;
      const long long mh = m / NP, ml = m % NP;
      const long long row_off = tc_batch(g, b).obase + (g.tile_b ? tile * g.s_tile : 0) +
                                mh * g.s_mhi + ml * g.s_mlo;
      const float sc = g.scale ? g.scale[b] : 1.0f;
#pragma unroll 1
      for (int c0 = 0; c0 < NP; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + acc * (uint32_t)NP + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (!g.out_split) {
          float* o = reinterpret_cast<float*>(g.out) + row_off + c0 * g.s_n;
          if (g.beta) {
            // accumulate with fire-and-forget reductions (every element has one owner)
#pragma unroll
            for (int i = 0; i < 32; ++i) atomicAdd(o + i * g.s_n, __uint_as_float(v[i]) * sc);
          } else if (g.s_n == 1) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(o + i) =
                  make_float4(__uint_as_float(v[i]) * sc, __uint_as_float(v[i + 1]) * sc,
                              __uint_as_float(v[i + 2]) * sc, __uint_as_float(v[i + 3]) * sc);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) o[i * g.s_n] = __uint_as_float(v[i]) * sc;
          }
        } else {
          E* oh = reinterpret_cast<E*>(g.out) + row_off + c0 * g.s_n;
          E* ol = reinterpret_cast<E*>(g.out_lo) + row_off + c0 * g.s_n;
          if (g.s_n == 1) {
#pragma unroll
            for (int i = 0; i < 32; i += 8) {
              E h[8], l[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) split2<E>(__uint_as_float(v[i + u]) * sc, h[u], l[u]);
              *reinterpret_cast<uint4*>(oh + i) = *reinterpret_cast<uint4*>(h);
              *reinterpret_cast<uint4*>(ol + i) = *reinterpret_cast<uint4*>(l);
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              E h, l;
              split2<E>(__uint_as_float(v[i]) * sc, h, l);
              oh[i * g.s_n] = h;
              ol[i * g.s_n] = l;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(acc));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * NP))
                 : "memory");
  }
}

// ------------------------------------------------------------------ element kernels
// operand planes of the Toeplitz matrices, padded to Np x Np:
// X1[s] = D_s (periodic) or T_s (box), TT[s] = T_s, WTD[s][0] = w_s T_s, WTD[s][1] = w_s D_s
template <typename E>
__global__ void k_mx_tables(const double* Tm, const double* WDm, const double* w, int S_eff,
                            int Mg, int Np, int periodic, const float* cs, E* x1h, E* x1l,
                            E* tth, E* ttl, E* wtdh, E* wtdl) {
  const long long n = (long long)S_eff * Np * Np;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / ((long long)Np * Np));
    const int a = (int)((i / Np) % Np), c = (int)(i % Np);
    double t = 0.0, d = 0.0;
    if (a < Mg && c < Mg) {
      t = Tm[((long long)s * Mg + a) * Mg + c];
      d = (periodic && a == c) ? 0.0 : t;
    }
    // fp16: the weight is split as (w_s / c_s) here and c_s on the intermediates
    const double ws = cs ? w[s] / (double)cs[s] : w[s];
    const double wt = ws * t, wd = ws * d;
    E h, l;
    split2<E>((float)(periodic ? d : t), h, l);
    x1h[i] = h;
    x1l[i] = l;
    split2<E>((float)t, h, l);
    tth[i] = h;
    ttl[i] = l;
    const long long j0 = (((long long)s * 2 + 0) * Np + a) * Np + c;
    const long long j1 = (((long long)s * 2 + 1) * Np + a) * Np + c;
    split2<E>((float)wt, h, l);
    wtdh[j0] = h;
    wtdl[j0] = l;
    split2<E>((float)wd, h, l);
    wtdh[j1] = h;
    wtdl[j1] = l;
    (void)WDm;
  }
}

template <typename E>
__global__ void k_mx_dbar(const double* Dbar, int Mg, int Np, E* h, E* l) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np * Np) return;
  const int a = i / Np, c = i % Np;
  const double v = (a < Mg && c < Mg) ? Dbar[a * Mg + c] : 0.0;
  E hh, ll;
  split2<E>((float)v, hh, ll);
  h[i] = hh;
  l[i] = ll;
}

// occupation O[x][y][z] and its x-last transpose OT[y][z][x], padded to Np^3 (exact)
template <typename E>
__global__ void k_mx_occ(int R, int R_F, int Np, E* O, E* OT) {
  const long long n = (long long)Np * Np * Np;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i / ((long long)Np * Np)), y = (int)((i / Np) % Np), z = (int)(i % Np);
    const int Mg = 2 * R + 1;
    float v = 0.0f;
    if (x < Mg && y < Mg && z < Mg) {
      const int a = x - R, bb = y - R, c = z - R;
      v = (a * a + bb * bb + c * c <= R_F * R_F) ? 1.0f : 0.0f;
    }
    O[i] = (E)v;
    OT[((long long)y * Np + z) * Np + x] = (E)v;
  }
}

// eps = -pref E on the basis sphere (unpadded grid), FP64 partials over the Fermi sphere
__global__ void k_mx_finalize(const float* E, int Np, int R, int R_F, double pref, float* eps,
                              double* part) {
  const int Mg = 2 * R + 1;
  const long long G3 = (long long)Mg * Mg * Mg;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G3;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i / ((long long)Mg * Mg)), y = (int)((i / Mg) % Mg), z = (int)(i % Mg);
    const int a = x - R, bb = y - R, c = z - R;
    const int m = a * a + bb * bb + c * c;
    float v = 0.0f;
    if (m <= R * R) v = (float)(-pref * (double)E[((long long)x * Np + y) * Np + z]);
    eps[i] = v;
    if (m <= R_F * R_F) acc += (double)v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_mx_reduce(const double* part, int n, double* Ex, const int* err, int* status) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Ex[0] = 0.5 * red[0];
    Ex[1] = red[0];
    if (status) *status = *err;
  }
}

// ------------------------------------------------------------------ host side
struct MxPlanes {  // one element type
  void* X1[2];   // [S_eff][Np][Np] hi, lo
  void* TT[2];   // [S_eff][Np][Np]
  void* WTD[2];  // [S_eff][2][Np][Np]
  void* DB[2];   // [Np][Np]
  void* O;       // [Np^3]
  void* OT;      // [Np^3]
  void* R[2];    // [C][Np^3]
  void* W[2];    // [C][2][Np^3]
  CUtensorMap mO, mOT, mR[2], mW[2], mX1[2], mTT[2], mWTD[2], mDB[2];
  float* cs = nullptr;  // fp16: per-node power-of-two scale of the y-mode operands
};

struct MxWorkspace {
  int Np = 0, C = 0, R_F_built = -1, R_F_built16 = -1;
  void* slab = nullptr;   // fused slab kernel workspace (Np = 128), tcslab.cu
  void* small = nullptr;  // small-grid kernel workspace (grid side <= 64), tcsmall.cu
  float* E = nullptr;     // [Np^3]
  int* err = nullptr;     // device error word
  MxPlanes bf, hf;
  std::vector<void*> allocs;
};

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static cc_status get_encoder() {
  if (g_encode) return CC_OK;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    set_last_error("cuTensorMapEncodeTiled entry point", e);
    return CC_ERR_CUDA;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return CC_OK;
}

// 2D map over a row-major [rows][Np] array of 16-bit values; box = 64 columns x box_rows
static cc_status make_map(CUtensorMap* m, void* ptr, long long rows, int Np, int box_rows,
                          bool bf16) {
  cuuint64_t dims[2] = {(cuuint64_t)Np, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Np * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1u, 1u};
  CUresult r = g_encode(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                        2, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled", cudaErrorInvalidValue);
    return CC_ERR_CUDA;
  }
  return CC_OK;
}

// for tcslab.cu: a 2D bf16 map over [rows][cols], 64-column x box_rows boxes, 128-byte swizzle
cc_status tc_make_map_bf16(void* map, void* ptr, long long rows, int cols, int box_rows) {
  CC_TRY(get_encoder());
  return make_map(reinterpret_cast<CUtensorMap*>(map), ptr, rows, cols, box_rows, true);
}
cc_status tc_make_map_16(void* map, void* ptr, long long rows, int cols, int box_rows,
                         bool bf16) {
  CC_TRY(get_encoder());
  return make_map(reinterpret_cast<CUtensorMap*>(map), ptr, rows, cols, box_rows, bf16);
}

static cc_status mx_alloc(cc_tables t, MxWorkspace* w, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_last_error("cudaMalloc(mixed workspace)", e);
    return CC_ERR_ALLOC;
  }
  w->allocs.push_back(*p);
  t->ws.mx_bytes += bytes;
  t->device_bytes += bytes;
  return CC_OK;
}

template <typename E>
static cc_status build_planes(cc_tables t, MxWorkspace* w, MxPlanes* P, bool bf16) {
  const int Np = w->Np, S = t->S_eff, C = w->C;
  const size_t e2 = 2;
  const size_t mat = (size_t)Np * Np * e2;
  const size_t vol = (size_t)Np * Np * Np * e2;
  for (int h = 0; h < 2; ++h) {
    CC_TRY(mx_alloc(t, w, &P->X1[h], mat * S));
    CC_TRY(mx_alloc(t, w, &P->TT[h], mat * S));
    CC_TRY(mx_alloc(t, w, &P->WTD[h], mat * S * 2));
    CC_TRY(mx_alloc(t, w, &P->DB[h], mat));
    CC_TRY(mx_alloc(t, w, &P->R[h], vol * C));
    CC_TRY(mx_alloc(t, w, &P->W[h], vol * C * 2));
  }
  CC_TRY(mx_alloc(t, w, &P->O, vol));
  CC_TRY(mx_alloc(t, w, &P->OT, vol));
  const long long NN = (long long)Np * Np;
  CC_TRY(make_map(&P->mO, P->O, NN, Np, kTileM, bf16));
  CC_TRY(make_map(&P->mOT, P->OT, NN, Np, kTileM, bf16));
  for (int h = 0; h < 2; ++h) {
    CC_TRY(make_map(&P->mR[h], P->R[h], (long long)C * NN, Np, kTileM, bf16));
    CC_TRY(make_map(&P->mW[h], P->W[h], (long long)C * 2 * NN, Np, kTileM, bf16));
    CC_TRY(make_map(&P->mX1[h], P->X1[h], (long long)S * Np, Np, Np, bf16));
    CC_TRY(make_map(&P->mTT[h], P->TT[h], (long long)S * Np, Np, Np, bf16));
    CC_TRY(make_map(&P->mWTD[h], P->WTD[h], (long long)S * 2 * Np, Np, Np, bf16));
    CC_TRY(make_map(&P->mDB[h], P->DB[h], (long long)Np, Np, Np, bf16));
  }
  const int periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  if (!bf16) {
    // per-node exponent scaling for fp16: the products w_s T_s W_s are formed as
    // (w_s / c_s) T_s (c_s W_s) with c_s = 2^min(1, floor(log2 w_s) + 14): the weight
    // factor stays in fp16's normal range (>= 2^-14 for T ~ 1) and c_s W_s <= 2 Np^2
    // stays below 65504 (W_s <= Np^2 since every T_s, D_s entry is <= 1)
    std::vector<float> c(S);
    for (int i = 0; i < S; ++i) {
      const double wv = t->w[t->kept_idx[i]];
      int e = (int)floor(log2(wv)) + 14;
      if (e > 1) e = 1;
      c[i] = ldexpf(1.0f, e);
    }
    CC_TRY(mx_alloc(t, w, (void**)&P->cs, sizeof(float) * S));
    CC_CUDA(cudaMemcpy(P->cs, c.data(), sizeof(float) * S, cudaMemcpyHostToDevice));
  }
  k_mx_tables<E><<<1024, 256>>>(t->d.Tm64, t->d.WDm64, t->d.w64, S, t->Mg, Np, periodic, P->cs,
                                (E*)P->X1[0], (E*)P->X1[1], (E*)P->TT[0], (E*)P->TT[1],
                                (E*)P->WTD[0], (E*)P->WTD[1]);
  k_mx_dbar<E><<<(Np * Np + 255) / 256, 256>>>(t->d.Dbar64, t->Mg, Np, (E*)P->DB[0],
                                               (E*)P->DB[1]);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

cc_status mixed_workspace_alloc(cc_tables t) {
  if (t->ws.mx) return CC_OK;
  if (t->Mg > 128) return CC_ERR_NOTSUPP;
  CC_TRY(get_encoder());
  MxWorkspace* w = new (std::nothrow) MxWorkspace();
  if (!w) return CC_ERR_ALLOC;
  t->ws.mx = w;
  w->Np = t->Mg <= 64 ? 64 : 128;
  w->C = t->S_eff < 8 ? t->S_eff : 8;
  const int Np = w->Np;
  CC_TRY(mx_alloc(t, w, (void**)&w->E, sizeof(float) * Np * Np * Np));
  CC_TRY(mx_alloc(t, w, (void**)&w->err, sizeof(int) * 2));
  CC_CUDA(cudaMemset(w->err, 0, sizeof(int) * 2));
  CC_TRY(build_planes<__nv_bfloat16>(t, w, &w->bf, true));
  CC_TRY(build_planes<__half>(t, w, &w->hf, false));
  CC_TRY(tc_slab_alloc(t, &w->slab));
  CC_TRY(tc_small_alloc(t, &w->small));
  CC_CUDA(cudaDeviceSynchronize());
  return CC_OK;
}

void mixed_workspace_free(cc_tables t) {
  MxWorkspace* w = reinterpret_cast<MxWorkspace*>(t->ws.mx);
  if (!w) return;
  tc_slab_free(w->slab);
  tc_small_free(w->small);
  for (void* p : w->allocs) cudaFree(p);
  delete w;
  t->ws.mx = nullptr;
}

static int tc_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

static int g_stall_next = 0;
// 0: automatic, 1: step chain, 2: fused slab kernel, 3: small-grid kernel (bf16x3)
static int g_mixed_variant = 0;
static int g_mixed_terms = 3;  // 3: hi*hi + hi*lo + lo*hi; 1: hi*hi only (slab kernels)

template <int NP, typename E>
static cc_status launch_tc(const CUtensorMap& A, const CUtensorMap& Alo, const CUtensorMap& B,
                           const CUtensorMap& Blo, TcArgs g, int m_tiles, int batches,
                           cudaStream_t st) {
  g.stall_test = __atomic_exchange_n(&g_stall_next, 0, __ATOMIC_ACQ_REL);
  auto kern = k_tc_gemm<NP, E>;
  const int smem = TcSmem<NP>::kBytes;
  static bool attr = false;
  if (!attr) {
    CC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  g.m_tiles = m_tiles;
  g.batches = batches;
  const int total = m_tiles * batches;
  const int grid = total < tc_sm_count() ? total : tc_sm_count();  // one CTA per SM, persistent
  kern<<<grid, kTcThreads, smem, st>>>(A, Alo, B, Blo, g);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

template <int NP, typename E>
static cc_status run_mixed(cc_tables t, MxWorkspace* w, MxPlanes& P, int R_F, float* eps,
                           double* Ex, cudaStream_t st) {
  const long long NN = (long long)NP * NP, VOL = NN * NP;
  const int m_tiles = (int)(NN / kTileM);
  const bool periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  const int S = t->S_eff, C = w->C;
  k_mx_occ<E><<<1024, 256, 0, st>>>(t->p.R, R_F, NP, (E*)P.O, (E*)P.OT);
  CC_CUDA(cudaGetLastError());
  const long long nat_mhi = NN, nat_mlo = NP;
  bool first = true;
  if (periodic) {
    // step 5: E[x][y][z'] = sum_z O[(x,y)][z] Dbar[z'][z]
    TcArgs g{};
    g.nk = NP / kKB; g.J = 1; g.resident = 1;
    g.a_base = 0; g.a_lo = 0; g.b_base = 0; g.b_lo = 1;
    g.out_split = 0; g.beta = 0; g.out = w->E;
    g.o_base = 0; g.o_sb = 0; g.s_mhi = nat_mhi; g.s_mlo = nat_mlo; g.s_n = 1;
    g.err = w->err;
    CC_TRY((launch_tc<NP, E>(P.mO, P.mO, P.mDB[0], P.mDB[1], g, m_tiles, 1, st)));
    first = false;
  }
  for (int s0 = 0; s0 < S; s0 += C) {
    const int cs = S - s0 < C ? S - s0 : C;
    // step 1: R_s[x][(y,z)] = sum_x' X1_s[x][x'] OT[(y,z)][x']   (stored transposed)
    {
      TcArgs g{};
      g.nk = NP / kKB; g.J = 1; g.resident = 1;
      g.a_base = 0; g.a_sb = 0; g.a_lo = 0;
      g.b_base = (long long)s0 * NP; g.b_sb = NP; g.b_lo = 1;
      g.out_split = 1; g.out = P.R[0]; g.out_lo = P.R[1];
      g.o_base = 0; g.o_sb = VOL; g.s_mhi = NP; g.s_mlo = 1; g.s_n = NN;
      g.err = w->err;
      CC_TRY((launch_tc<NP, E>(P.mOT, P.mOT, P.mX1[0], P.mX1[1], g, m_tiles, cs, st)));
    }
    // step 2: W1_s[x][z'][y] = sum_z T_s[z'][z] R_s[(x,y)][z]      (slab transposed)
    {
      TcArgs g{};
      g.nk = NP / kKB; g.J = 1; g.resident = 1;
      g.a_base = 0; g.a_sb = NN; g.a_lo = 1;
      g.b_base = (long long)s0 * NP; g.b_sb = NP; g.b_lo = 1;
      g.out_split = 1; g.out = P.W[0]; g.out_lo = P.W[1];
      g.o_base = 0; g.o_sb = 2 * VOL; g.s_mhi = NN; g.s_mlo = 1; g.s_n = NP;
      g.scale = P.cs ? P.cs + s0 : nullptr;
      g.err = w->err;
      CC_TRY((launch_tc<NP, E>(P.mR[0], P.mR[1], P.mTT[0], P.mTT[1], g, m_tiles, cs, st)));
    }
    if (periodic) {
      // step 3: W2_s[x][z'][y] = sum_z T_s[z'][z] O[(x,y)][z]
      TcArgs g{};
      g.nk = NP / kKB; g.J = 1; g.resident = 1;
      g.a_base = 0; g.a_sb = 0; g.a_lo = 0;
      g.b_base = (long long)s0 * NP; g.b_sb = NP; g.b_lo = 1;
      g.out_split = 1; g.out = P.W[0]; g.out_lo = P.W[1];
      g.o_base = VOL; g.o_sb = 2 * VOL; g.s_mhi = NN; g.s_mlo = 1; g.s_n = NP;
      g.scale = P.cs ? P.cs + s0 : nullptr;
      g.err = w->err;
      CC_TRY((launch_tc<NP, E>(P.mO, P.mO, P.mTT[0], P.mTT[1], g, m_tiles, cs, st)));
    }
    // step 4: E[x][y'][z'] += sum_j sum_y WTD_j[y'][y] W_j[(x,z')][y]   (slab transposed)
    {
      TcArgs g{};
      g.nk = NP / kKB;
      g.J = periodic ? 2 * cs : cs;
      g.a_base = 0; g.a_sb = 0; g.a_sj = periodic ? NN : 2 * NN; g.a_lo = 1;
      g.b_base = (long long)s0 * 2 * NP; g.b_sb = 0; g.b_sj = periodic ? NP : 2 * NP; g.b_lo = 1;
      g.out_split = 0; g.beta = first ? 0 : 1; g.out = w->E;
      g.o_base = 0; g.o_sb = 0; g.s_mhi = NN; g.s_mlo = 1; g.s_n = NP;
      g.err = w->err;
      CC_TRY((launch_tc<NP, E>(P.mW[0], P.mW[1], P.mWTD[0], P.mWTD[1], g, m_tiles, 1, st)));
      first = false;
    }
  }
  k_mx_finalize<<<kRedBlocks, 256, 0, st>>>(w->E, NP, t->p.R, R_F, t->pref, eps, t->ws.part);
  k_mx_reduce<<<1, 256, 0, st>>>(t->ws.part, kRedBlocks, Ex, w->err, w->err + 1);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

cc_status exchange_mixed(cc_tables t, int R_F, int precision, float* eps, double* Ex,
                         cudaStream_t st) {
  if (precision != CC_PREC_BF16X3 && precision != CC_PREC_FP16X3) return CC_ERR_NOTSUPP;
  if (t->Mg > 128) return CC_ERR_NOTSUPP;
  MxWorkspace* w = reinterpret_cast<MxWorkspace*>(t->ws.mx);
  if (!w) return CC_ERR_NOTSUPP;  // handle built without workspaces
  if (precision == CC_PREC_FP16X3) {
    if (w->slab && g_mixed_variant != 1) {
      const int stall = __atomic_exchange_n(&g_stall_next, 0, __ATOMIC_ACQ_REL);
      return tc_slab_run(t, w->slab, nullptr, nullptr, w->err, stall, R_F, eps, Ex, st, true,
                         __atomic_load_n(&g_mixed_terms, __ATOMIC_ACQUIRE) == 1);
    }
    if (g_mixed_variant == 2) return CC_ERR_NOTSUPP;
    if (w->Np == 64) return run_mixed<64, __half>(t, w, w->hf, R_F, eps, Ex, st);
    return run_mixed<128, __half>(t, w, w->hf, R_F, eps, Ex, st);
  }
  const int variant = __atomic_load_n(&g_mixed_variant, __ATOMIC_ACQUIRE);
  if (w->small && (variant == 0 || variant == 3)) {
    const int stall = __atomic_exchange_n(&g_stall_next, 0, __ATOMIC_ACQ_REL);
    return tc_small_run(t, w->small, w->err, stall, R_F, eps, Ex, st,
                        __atomic_load_n(&g_mixed_terms, __ATOMIC_ACQUIRE) == 1);
  }
  if (variant == 3) return CC_ERR_NOTSUPP;
  if (w->slab && variant != 1) {
    const int stall = __atomic_exchange_n(&g_stall_next, 0, __ATOMIC_ACQ_REL);
    return tc_slab_run(t, w->slab, &w->bf.mTT[0], &w->bf.mTT[1], w->err, stall, R_F, eps, Ex,
                       st, false, __atomic_load_n(&g_mixed_terms, __ATOMIC_ACQUIRE) == 1);
  }
  if (variant == 2) return CC_ERR_NOTSUPP;
  if (w->Np == 64) return run_mixed<64, __nv_bfloat16>(t, w, w->bf, R_F, eps, Ex, st);
  return run_mixed<128, __nv_bfloat16>(t, w, w->bf, R_F, eps, Ex, st);
}

}  // namespace cc

// Choice of the tensor-core exchange form (0 automatic: the small-grid kernel for bf16x3 at
// grid sides up to 64, the 128-row slab kernel above and for fp16x3; 1 the step chain;
// 2 the 128-row slab kernel; 3 the small-grid kernel).
extern "C" cc_status cc_set_mixed_variant(int variant) {
  if (variant < 0 || variant > 3) return CC_ERR_ARG;
  __atomic_store_n(&cc::g_mixed_variant, variant, __ATOMIC_RELEASE);
  return CC_OK;
}

extern "C" cc_status cc_set_mixed_terms(int terms) {
  if (terms != 1 && terms != 3) return CC_ERR_ARG;
  __atomic_store_n(&cc::g_mixed_terms, terms, __ATOMIC_RELEASE);
  return CC_OK;
}

// Device error word of the mixed path (0: fine, 1-3: a bounded wait ran out in the
// producer, MMA issuer or epilogue).  Reads back synchronously; clears it when asked.
extern "C" cc_status cc_mixed_status(cc_tables t, int* code_host, int clear) {
  if (!t || !code_host) return CC_ERR_ARG;
  cc::MxWorkspace* w = reinterpret_cast<cc::MxWorkspace*>(t->ws.mx);
  *code_host = 0;
  if (!w) return CC_OK;
  CC_CUDA(cudaMemcpy(code_host, w->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (clear) CC_CUDA(cudaMemset(w->err, 0, sizeof(int) * 2));
  return *code_host ? CC_ERR_TIMEOUT : CC_OK;
}

// ------------------------------------------------------------------ batched boxes (bf16x3)
// The tensor-core form of the batched engine: every box (grid side <= 49, padded to
// Np = 64) goes through the same step 5 / 1 / 2 / 3 / 4 chain as a single box, but each
// launch covers all boxes at once through a per-batch table of row bases (TcArgs.btab):
// rounds of C nodes per box, the boxes' planes concatenated in shared arrays.  The whole
// sequence is enqueued on one stream and captured in one CUDA graph by the caller.
namespace cc {

struct MxBatchImpl {
  int nbox = 0, C = 4, rounds = 0;
  std::vector<int> S;
  int* R_dev = nullptr;
  int* RF_dev = nullptr;
  double* pref_dev = nullptr;
  long long* eps_off_dev = nullptr;
  MxPlanes P;  // X1, TT, WTD, DB concatenated over boxes; O, OT [nbox][Np^3]; R, W slots
  float* E = nullptr;
  int* err = nullptr;
  long long* t5 = nullptr;
  std::vector<long long*> t123[3], t4;
  std::vector<int> n123, n4;
  std::vector<void*> allocs;
  void* small = nullptr;  // the batch through the small-grid kernel (tcsmall.cu)
};

__global__ void k_mxb_occ(int nbox, const int* R, const int* RF, __nv_bfloat16* O,
                          __nv_bfloat16* OT) {
  constexpr int Np = 64;
  const long long per = (long long)Np * Np * Np;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per * nbox;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per);
    const long long j = i % per;
    const int x = (int)(j / (Np * Np)), y = (int)((j / Np) % Np), z = (int)(j % Np);
    const int Rb = R[b], Mg = 2 * Rb + 1;
    float v = 0.0f;
    if (x < Mg && y < Mg && z < Mg) {
      const int a = x - Rb, bb = y - Rb, c = z - Rb;
      v = (a * a + bb * bb + c * c <= RF[b] * RF[b]) ? 1.0f : 0.0f;
    }
    O[i] = __float2bfloat16_rn(v);
    OT[b * per + ((long long)y * Np + z) * Np + x] = __float2bfloat16_rn(v);
  }
}

// one CTA per box: eps = -pref E on the basis sphere, E_x in FP64
__global__ void k_mxb_finalize(const int* R, const int* RF, const double* pref,
                               const long long* eps_off, const float* E, float* eps,
                               double* Ex) {
  constexpr int Np = 64;
  const int b = blockIdx.x;
  const int Rb = R[b], Mg = 2 * Rb + 1;
  const long long G3 = (long long)Mg * Mg * Mg;
  const float* Eb = E + (long long)b * Np * Np * Np;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < G3; i += blockDim.x) {
    const int x = (int)(i / ((long long)Mg * Mg)), y = (int)((i / Mg) % Mg), z = (int)(i % Mg);
    const int a = x - Rb, bb = y - Rb, c = z - Rb;
    const int m = a * a + bb * bb + c * c;
    float v = 0.0f;
    if (m <= Rb * Rb) v = (float)(-pref[b] * (double)Eb[((long long)x * Np + y) * Np + z]);
    eps[eps_off[b] + i] = v;
    if (m <= RF[b] * RF[b]) acc += (double)v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Ex[2 * b] = 0.5 * red[0];
    Ex[2 * b + 1] = red[0];
  }
}

static cc_status mxb_alloc(MxBatchImpl* m, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    set_last_error("cudaMalloc(mixed batch)", e);
    return CC_ERR_ALLOC;
  }
  m->allocs.push_back(*p);
  return CC_OK;
}

template <typename V>
static cc_status mxb_upload(MxBatchImpl* m, V** dst, const std::vector<V>& src) {
  CC_TRY(mxb_alloc(m, (void**)dst, sizeof(V) * src.size()));
  CC_CUDA(cudaMemcpy(*dst, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice));
  return CC_OK;
}

void mixed_batch_free(void* p) {
  MxBatchImpl* m = reinterpret_cast<MxBatchImpl*>(p);
  if (!m) return;
  tc_small_batch_free(m->small);
  for (void* q : m->allocs) cudaFree(q);
  delete m;
}

cc_status mixed_batch_create(const std::vector<cc_tables>& tabs, const std::vector<int>& R_F,
                             const std::vector<long long>& eps_off, void** out) {
  *out = nullptr;
  CC_TRY(get_encoder());
  constexpr int Np = 64;
  const long long NN = (long long)Np * Np, VOL = NN * Np;
  MxBatchImpl* m = new (std::nothrow) MxBatchImpl();
  if (!m) return CC_ERR_ALLOC;
  m->nbox = (int)tabs.size();
  const int nb = m->nbox;
  cc_status s = CC_OK;
  std::vector<int> Rv(nb);
  std::vector<double> pref(nb);
  std::vector<long long> off_x1(nb), off_wtd(nb);
  long long rows_x1 = 0;
  int max_s = 0;
  for (int b = 0; b < nb; ++b) {
    const cc_tables t = tabs[b];
    if (t->Mg > Np || t->p.kernel != CC_KERNEL_PERIODIC) s = CC_ERR_NOTSUPP;
    Rv[b] = t->p.R;
    pref[b] = t->pref;
    m->S.push_back(t->S_eff);
    off_x1[b] = rows_x1;
    off_wtd[b] = 2 * rows_x1;
    rows_x1 += (long long)t->S_eff * Np;
    max_s = std::max(max_s, t->S_eff);
  }
  const int C = m->C;
  m->rounds = (max_s + C - 1) / C;
  const size_t e2 = 2;
  MxPlanes& P = m->P;
  for (int h = 0; h < 2 && s == CC_OK; ++h) {
    if (s == CC_OK) s = mxb_alloc(m, &P.X1[h], rows_x1 * Np * e2);
    if (s == CC_OK) s = mxb_alloc(m, &P.TT[h], rows_x1 * Np * e2);
    if (s == CC_OK) s = mxb_alloc(m, &P.WTD[h], 2 * rows_x1 * Np * e2);
    if (s == CC_OK) s = mxb_alloc(m, &P.DB[h], (size_t)nb * NN * e2);
    if (s == CC_OK) s = mxb_alloc(m, &P.R[h], (size_t)nb * C * VOL * e2);
    if (s == CC_OK) s = mxb_alloc(m, &P.W[h], (size_t)nb * C * 2 * VOL * e2);
  }
  if (s == CC_OK) s = mxb_alloc(m, &P.O, (size_t)nb * VOL * e2);
  if (s == CC_OK) s = mxb_alloc(m, &P.OT, (size_t)nb * VOL * e2);
  if (s == CC_OK) s = mxb_alloc(m, (void**)&m->E, (size_t)nb * VOL * sizeof(float));
  if (s == CC_OK) s = mxb_alloc(m, (void**)&m->err, sizeof(int) * 2);
  if (s == CC_OK) s = make_map(&P.mO, P.O, nb * NN, Np, kTileM, true);
  if (s == CC_OK) s = make_map(&P.mOT, P.OT, nb * NN, Np, kTileM, true);
  for (int h = 0; h < 2 && s == CC_OK; ++h) {
    if (s == CC_OK) s = make_map(&P.mR[h], P.R[h], (long long)nb * C * NN, Np, kTileM, true);
    if (s == CC_OK) s = make_map(&P.mW[h], P.W[h], (long long)nb * C * 2 * NN, Np, kTileM, true);
    if (s == CC_OK) s = make_map(&P.mX1[h], P.X1[h], rows_x1, Np, Np, true);
    if (s == CC_OK) s = make_map(&P.mTT[h], P.TT[h], rows_x1, Np, Np, true);
    if (s == CC_OK) s = make_map(&P.mWTD[h], P.WTD[h], 2 * rows_x1, Np, Np, true);
    if (s == CC_OK) s = make_map(&P.mDB[h], P.DB[h], (long long)nb * Np, Np, Np, true);
  }
  // Toeplitz planes of every box, written at the box's row offsets
  for (int b = 0; b < nb && s == CC_OK; ++b) {
    const cc_tables t = tabs[b];
    using E = __nv_bfloat16;
    k_mx_tables<E><<<256, 256>>>(t->d.Tm64, t->d.WDm64, t->d.w64, t->S_eff, t->Mg, Np, 1,
                                 nullptr, (E*)P.X1[0] + off_x1[b] * Np,
                                 (E*)P.X1[1] + off_x1[b] * Np, (E*)P.TT[0] + off_x1[b] * Np,
                                 (E*)P.TT[1] + off_x1[b] * Np, (E*)P.WTD[0] + off_wtd[b] * Np,
                                 (E*)P.WTD[1] + off_wtd[b] * Np);
    k_mx_dbar<E><<<(Np * Np + 255) / 256, 256>>>(t->d.Dbar64, t->Mg, Np,
                                                  (E*)P.DB[0] + (long long)b * NN,
                                                  (E*)P.DB[1] + (long long)b * NN);
    if (cudaGetLastError() != cudaSuccess) s = CC_ERR_CUDA;
  }
  // per-step tables
  std::vector<long long> t5;
  for (int b = 0; b < nb; ++b) t5.insert(t5.end(), {b * NN, (long long)b * Np, b * VOL, 1});
  if (s == CC_OK) s = mxb_upload(m, &m->t5, t5);
  for (int r = 0; r < m->rounds && s == CC_OK; ++r) {
    std::vector<long long> a1, a2, a3, a4;
    for (int b = 0; b < nb; ++b) {
      const int s0 = r * C;
      const int cnt = std::min(C, m->S[b] - s0);
      if (cnt <= 0) continue;
      for (int c = 0; c < cnt; ++c) {
        const long long slot = (long long)b * C + c, node = s0 + c;
        a1.insert(a1.end(), {b * NN, off_x1[b] + node * Np, slot * VOL, 1});
        a2.insert(a2.end(), {slot * NN, off_x1[b] + node * Np, slot * 2 * VOL, 1});
        a3.insert(a3.end(), {b * NN, off_x1[b] + node * Np, slot * 2 * VOL + VOL, 1});
      }
      a4.insert(a4.end(), {(long long)b * C * 2 * NN, off_wtd[b] + 2LL * s0 * Np, b * VOL,
                           2LL * cnt});
    }
    long long* d[4] = {nullptr, nullptr, nullptr, nullptr};
    if (s == CC_OK) s = mxb_upload(m, &d[0], a1);
    if (s == CC_OK) s = mxb_upload(m, &d[1], a2);
    if (s == CC_OK) s = mxb_upload(m, &d[2], a3);
    if (s == CC_OK) s = mxb_upload(m, &d[3], a4);
    m->t123[0].push_back(d[0]);
    m->t123[1].push_back(d[1]);
    m->t123[2].push_back(d[2]);
    m->t4.push_back(d[3]);
    m->n123.push_back((int)(a1.size() / 4));
    m->n4.push_back((int)(a4.size() / 4));
  }
  if (s == CC_OK) s = mxb_upload(m, &m->R_dev, Rv);
  if (s == CC_OK) s = mxb_upload(m, &m->RF_dev, R_F);
  if (s == CC_OK) s = mxb_upload(m, &m->pref_dev, pref);
  if (s == CC_OK) s = mxb_upload(m, &m->eps_off_dev, eps_off);
  if (s == CC_OK && cudaMemset(m->err, 0, sizeof(int) * 2) != cudaSuccess) s = CC_ERR_CUDA;
  if (s == CC_OK && cudaDeviceSynchronize() != cudaSuccess) s = CC_ERR_CUDA;
  // the same boxes through the small-grid kernel (every grid side <= 64)
  if (s == CC_OK && tc_small_batch_supported(tabs, R_F))
    s = tc_small_batch_create(tabs, R_F, eps_off, &m->small);
  if (s != CC_OK) {
    mixed_batch_free(m);
    return s;
  }
  *out = m;
  return CC_OK;
}

cc_status mixed_batch_tune(void* p, float* eps, double* Ex, int reps, int* choice, float* ms,
                           cudaStream_t st) {
  MxBatchImpl* m = reinterpret_cast<MxBatchImpl*>(p);
  if (!m || !m->small) return CC_ERR_NOTSUPP;
  return tc_small_batch_tune(m->small, m->err, eps, Ex, reps, choice, ms, st);
}

cc_status mixed_batch_run(void* p, float* eps, double* Ex, cudaStream_t st) {
  MxBatchImpl* m = reinterpret_cast<MxBatchImpl*>(p);
  if (!m) return CC_ERR_NOTSUPP;
  const int variant = __atomic_load_n(&g_mixed_variant, __ATOMIC_ACQUIRE);
  if (m->small && variant != 1) return tc_small_batch_run(m->small, m->err, eps, Ex, st);
  constexpr int Np = 64;
  using E = __nv_bfloat16;
  const long long NN = (long long)Np * Np;
  const int m_tiles = (int)(NN / kTileM);
  MxPlanes& P = m->P;
  k_mxb_occ<<<1216, 256, 0, st>>>(m->nbox, m->R_dev, m->RF_dev, (E*)P.O, (E*)P.OT);
  CC_CUDA(cudaGetLastError());
  {  // step 5: E_b = O_b x3 Dbar_b
    TcArgs g{};
    g.nk = 1; g.J = 1; g.resident = 1; g.a_lo = 0; g.b_lo = 1;
    g.out_split = 0; g.beta = 0; g.out = m->E;
    g.s_mhi = NN; g.s_mlo = Np; g.s_n = 1;
    g.btab = m->t5; g.err = m->err;
    CC_TRY((launch_tc<Np, E>(P.mO, P.mO, P.mDB[0], P.mDB[1], g, m_tiles, m->nbox, st)));
  }
  for (int r = 0; r < m->rounds; ++r) {
    TcArgs g{};
    g.nk = 1; g.J = 1; g.resident = 1; g.err = m->err;
    g.a_lo = 0; g.b_lo = 1; g.out_split = 1; g.out = P.R[0]; g.out_lo = P.R[1];
    g.s_mhi = Np; g.s_mlo = 1; g.s_n = NN; g.btab = m->t123[0][r];
    CC_TRY((launch_tc<Np, E>(P.mOT, P.mOT, P.mX1[0], P.mX1[1], g, m_tiles, m->n123[r], st)));
    g.a_lo = 1; g.out = P.W[0]; g.out_lo = P.W[1];
    g.s_mhi = NN; g.s_mlo = 1; g.s_n = Np; g.btab = m->t123[1][r];
    CC_TRY((launch_tc<Np, E>(P.mR[0], P.mR[1], P.mTT[0], P.mTT[1], g, m_tiles, m->n123[r], st)));
    g.a_lo = 0; g.btab = m->t123[2][r];
    CC_TRY((launch_tc<Np, E>(P.mO, P.mO, P.mTT[0], P.mTT[1], g, m_tiles, m->n123[r], st)));
    TcArgs g4{};
    g4.nk = 1; g4.J = 1; g4.a_sj = NN; g4.b_sj = Np; g4.a_lo = 1; g4.b_lo = 1;
    g4.out_split = 0; g4.beta = 1; g4.out = m->E;
    g4.s_mhi = NN; g4.s_mlo = 1; g4.s_n = Np; g4.btab = m->t4[r]; g4.err = m->err;
    CC_TRY((launch_tc<Np, E>(P.mW[0], P.mW[1], P.mWTD[0], P.mWTD[1], g4, m_tiles, m->n4[r], st)));
  }
  k_mxb_finalize<<<m->nbox, 256, 0, st>>>(m->R_dev, m->RF_dev, m->pref_dev, m->eps_off_dev, m->E,
                                          eps, Ex);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

}  // namespace cc

// Test hook (no counterpart in the paper): the next tensor-core GEMM launch makes its MMA
// warp wait on a barrier that nothing arrives at; the 20 ms bound runs out, the kernel
// records error code 5 and returns through its normal teardown.
extern "C" cc_status cc_test_stall_next_mixed(void) {
  __atomic_store_n(&cc::g_stall_next, 1, __ATOMIC_RELEASE);
  return CC_OK;
}
