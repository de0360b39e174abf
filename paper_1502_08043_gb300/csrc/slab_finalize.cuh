// Work split and deterministic finaliser shared by the single-box slab kernels of the
// exchange sums (Sec. III, with the node sum of Sec. II Eq. 14): the fused tensor-core slab
// kernels of grid side <= 127 and <= 63, and the FP32 SIMT slab kernel.
//
// A persistent grid of G CTAs walks U work units; CTA c owns the contiguous run
// [c U / G, (c + 1) U / G).  Units come in groups (a slab pair, or a row block of one slab)
// of S units, one per node s; every CTA that touches a group leaves one partial E plane of
// it, its "segment".  The finaliser adds, for each grid row (x, y), the segments of its
// group in CTA order, adds the I x I x Dbar term of the periodic kernel, writes eps on the
// basis sphere (0 outside), and sums the row's eps over the Fermi sphere in FP64 (fixed
// butterfly order); a block adds its eight rows in order.  The last block to finish
// (ticket) adds the block sums in a fixed order into E_x = (E_x / 2, E_x), copies the error
// word into the status word, and resets the ticket for the next call, so the result does
// not depend on which block finishes last.
#pragma once

#include <cuda_runtime.h>

namespace cc {
namespace {

// the CTA that owns unit u under the equal split of `units` units over `grid` CTAs
__host__ __device__ inline int owner_cta(long long u, int units, int grid) {
  int c = (int)((u * grid) / units);
  while (c + 1 < grid && (long long)(c + 1) * units / grid <= u) ++c;
  while (c > 0 && (long long)c * units / grid > u) --c;
  return c;
}

// floor(sqrt(v)) for v >= 0, exact for every int
__device__ __forceinline__ int isqrt_int(int v) {
  int h = (int)sqrtf((float)v);
  while (h * h > v) --h;
  while ((h + 1) * (h + 1) <= v) ++h;
  return h;
}

// part is [groups][maxseg][GR][W] floats (W = padded grid side, a multiple of 32); the row
// (x, y) is row r of group g:
//   kPairs:   g = x / 2,        r = (x % 2) W + y    (a slab pair per group, GR = 2 W)
//   !kPairs:  g = x nh + y / GR, r = y % GR          (nh row blocks of GR rows per slab)
// FB is [h][W], the Dbar windows sum_{k=R-h}^{R+h} Dbar[z][k] of the periodic kernel.
// blk_ex holds one double per block.  Launch: grid ((Mg + 7) / 8, Mg), 256 threads, one warp
// per row y.
template <int W, int GR, bool kPairs>
__global__ void __launch_bounds__(256)
    k_slab_finalize(const float* part, const float* FB, int R, int RF, int S, int nh,
                    int units, int grid, int maxseg, int periodic, double pref, float* eps,
                    double* blk_ex, unsigned* ticket, double* Ex, const int* err,
                    int* status) {
  static_assert(W % 32 == 0, "row width must be whole warps");
  // launched as a programmatic dependent of the slab kernel: wait until that grid has
  // completed and its partials are visible (no-op for an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int Mg = 2 * R + 1;
  const int x = blockIdx.y, y = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  __shared__ double wsum[8];
  __shared__ double red[256];
  __shared__ bool s_last;
  if (y < Mg) {
    const int g = kPairs ? x >> 1 : x * nh + y / GR;
    const int r = kPairs ? (x & 1) * W + y : y % GR;
    const int c0 = owner_cta((long long)g * S, units, grid);
    const int nseg = owner_cta((long long)(g + 1) * S - 1, units, grid) - c0 + 1;
    const int dx = x - R, dy = y - R;
    const int qb = RF * RF - dx * dx - dy * dy;  // z line at (x, y) of the Dbar term
    const float* fb = (periodic && qb >= 0) ? FB + isqrt_int(qb) * W : nullptr;
    const float* pp = part + ((long long)g * maxseg * GR + r) * W;
    constexpr int kZ = W / 32;  // z values per lane
    float sum[kZ];
#pragma unroll
    for (int i = 0; i < kZ; ++i) sum[i] = 0.0f;
    // segments in order, four at a time with every load issued before the adds
    for (int k0 = 0; k0 < nseg; k0 += 4) {
      float v[4][kZ];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int i = 0; i < kZ; ++i)
          v[kk][i] = k0 + kk < nseg && lane + 32 * i < Mg
                         ? __ldg(pp + (long long)(k0 + kk) * GR * W + lane + 32 * i)
                         : 0.0f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int i = 0; i < kZ; ++i)
          if (k0 + kk < nseg) sum[i] += v[kk][i];
    }
    // eps scaled in FP32 (FP64 arithmetic runs at a small fraction of the FP32 rate on
    // GB300; rounding pref adds at most 2^-24 relative), the E_x row sum in FP64
    const float npref = (float)(-pref);
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < kZ; ++i) {
      const int z = lane + 32 * i;
      if (z >= Mg) continue;
      float s = sum[i];
      if (fb) s += __ldg(fb + z);
      const int dz = z - R, m = dx * dx + dy * dy + dz * dz;
      const float v = m <= R * R ? npref * s : 0.0f;
      eps[((long long)x * Mg + y) * Mg + z] = v;
      if (m <= RF * RF) acc += (double)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[threadIdx.x >> 5] = acc;
  } else if (lane == 0) {
    wsum[threadIdx.x >> 5] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the block's rows in order, then the ticket
    double b = 0.0;
    for (int k = 0; k < 8; ++k) b += wsum[k];
    blk_ex[blockIdx.y * gridDim.x + blockIdx.x] = b;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nblk = gridDim.x * gridDim.y;
  double a = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 256) a += __ldcg(blk_ex + i);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Ex[0] = 0.5 * red[0];
    Ex[1] = red[0];
    if (status) *status = err ? *err : 0;
    *ticket = 0u;
  }
}

// the finaliser, launched as a programmatic dependent of the slab kernel launched just
// before it on st (its launch overlaps that kernel's last CTAs; every CTA of the slab kernel
// signals with griddepcontrol.launch_dependents when its own work is done)
template <int W, int GR, bool kPairs, typename... Args>
inline cudaError_t launch_slab_finalize(int Mg, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((Mg + 7) / 8, Mg);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_slab_finalize<W, GR, kPairs>, args...);
}

// a slab kernel's CTA is done with everything the finaliser reads
__device__ __forceinline__ void signal_finalizer() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace
}  // namespace cc
