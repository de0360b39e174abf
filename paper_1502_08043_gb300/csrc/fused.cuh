// Slab-wise exchange sums on the SIMT cores (FP32 / FP64), grid side Mg <= 63, used for
// single boxes and for the batched engine.
//
// Sec. III exchange of the uniform electron gas with the node sum of Sec. II Eq. 14.
// Periodic kernel, D_s = T_s - I (no self term, no cancellation):
//   E = sum_s w_s (O x1 D x2 T x3 T + O x2 D x3 T) + O x3 Dbar,   Dbar = sum_s w_s D_s
//     = sum_s w_s [ (R_s x2 T_s + A_s) x3 T_s ] + O x3 Dbar,
//   R_s = O x1 D_s,  A_s = O x2 D_s.
// Box kernel: E = sum_s w_s (R_s x2 T_s) x3 T_s with R_s = O x1 T_s, no A, no Dbar term.
// The occupation is a Fermi sphere, so every line of O along an axis is 1 on one
// contiguous range [R - h, R + h] (h = floor(sqrt(R_F^2 - u^2 - v^2)) for the other two
// coordinates u, v).  A mode product of O with M therefore takes, per line, the window sum
// F[a][h] = sum_{k = R - h}^{R + h} M[a][k]; the table builder forms these in FP64 once
// (k_windows), rounded to T only here.  What is left per node and x slab are two
// Mg x Mg x Mg products (U = T R_x + A_x, then U T), all in shared memory.
// Work item = (box, x slab, group of nodes); the item's slab of E (Kahan-summed over
// its nodes) goes to a partial buffer; the CTA that completes the last group of a slab
// adds the slab's partials (Kahan), writes its eps and its FP64 share of E_x, and the
// CTA that completes the last slab of a box adds the shares in slab order.  Items are
// taken from an atomic counter by a persistent grid; no CTA ever waits for another.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace cc {

constexpr int kSlabMaxMg = 63;

template <typename T>
struct FusedBox {
  int R, R_F, Mg, S_eff, periodic, n_groups, n_items;
  double pref;
  const T* Tm;         // [S_eff][Mg][Mg]  T_s
  const T* Fw;         // [S_eff][Mg][R + 1]  window sums of the rows of D_s (T_s for the box)
  const double* w64;   // [S_eff]
  const T* FDb;        // [Mg][R + 1]  window sums of the rows of sum_s w_s D_s (periodic)
  T* part;             // [n_groups][Mg][Mg][Mg] slab partials
  int* slab_done;      // [Mg] finished groups per slab
  double* slab_ex;     // [Mg] FP64 sum of eps over the Fermi sphere, per slab
  long long eps_off;   // offset of this box's eps block in the output
  int ex_idx;          // this box's E_x pair in the output
};

struct FusedItem {
  int box, x, s0, s1, g;
};

constexpr int kFusedThreads = 256;
constexpr int kFusedMaxGroups = 16;  // node groups per box at most

// shared-memory layout of one item (Mg = 2R + 1 = the box's grid side, mm = Mg * Mg):
//   T      sT[mm], sR[mm], sU[mm], sE[mm], sC[mm]
//   T      sF[Mg][R + 1]     the node's window sums (periodic: the A term)
//   short  H[Mg][Mg]         sphere half-lengths, -1 for an empty line
template <typename T>
__host__ __device__ inline size_t slab_smem_bytes(int Mg) {
  const size_t mm = (size_t)Mg * Mg;
  return (5 * mm + (size_t)Mg * ((Mg + 1) / 2)) * sizeof(T) + sizeof(short) * mm;
}

__device__ __forceinline__ int isqrt_floor(int v) {
  int h = (int)sqrtf((float)v);
  while (h * h > v) --h;
  while ((h + 1) * (h + 1) <= v) ++h;
  return h;
}

template <typename T>
__device__ __forceinline__ void kahan_add(T* e, T* c, int o, T v) {
  const T yv = v - c[o];
  const T t = e[o] + yv;
  c[o] = (t - e[o]) - yv;
  e[o] = t;
}

template <typename T>
__global__ void __launch_bounds__(kFusedThreads)
    k_fused_exchange(const FusedBox<T>* __restrict__ boxes, const FusedItem* __restrict__ items,
                     int n_items, int* work, int* done, int rf_override, T* eps_out,
                     double* ex_out) {
  extern __shared__ __align__(16) unsigned char fsmem[];
  __shared__ int s_item, s_last;
  __shared__ double s_red[kFusedThreads];
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const FusedItem item = items[it];
    FusedBox<T> bx = boxes[item.box];
    if (rf_override > 0) bx.R_F = rf_override;
    const int Mg = bx.Mg, R = bx.R, nh = R + 1, mm = Mg * Mg, x = item.x;
    T* sT = reinterpret_cast<T*>(fsmem);
    T* sR = sT + mm;
    T* sU = sR + mm;
    T* sE = sU + mm;
    T* sC = sE + mm;
    T* sF = sC + mm;
    short* H = reinterpret_cast<short*>(sF + Mg * nh);
    for (int i = threadIdx.x; i < mm; i += blockDim.x) {
      const int u = i / Mg - R, v = i % Mg - R;
      const int h2 = bx.R_F * bx.R_F - u * u - v * v;
      H[i] = (short)(h2 >= 0 ? isqrt_floor(h2) : -1);
      sE[i] = T(0);
      sC[i] = T(0);
    }
    __syncthreads();
    const int cb = (Mg + 3) / 4;
    for (int s = item.s0; s < item.s1; ++s) {
      // T_s; R_x[y][z] = sum_{x' on the x line at (y, z)} X[x][x'] = F_s[x][h(y, z)] with
      // X = D_s (periodic) or T_s (box); the node's window sums for the A term
      const T* Fs = bx.Fw + (long long)s * Mg * nh;
      for (int i = threadIdx.x; i < mm; i += blockDim.x) {
        sT[i] = bx.Tm[(long long)s * mm + i];
        const int h = H[i];
        sR[i] = h < 0 ? T(0) : Fs[x * nh + h];
      }
      if (bx.periodic)
        for (int i = threadIdx.x; i < Mg * nh; i += blockDim.x) sF[i] = Fs[i];
      __syncthreads();
      // U[y'][z] = sum_y T[y'][y] R_x[y][z] + A_x[y'][z],
      // A_x[y'][z] = sum_{y on the y line at (x, z)} D[y'][y]   (periodic only)
      for (int blk = threadIdx.x; blk < Mg * cb; blk += blockDim.x) {
        const int yp = blk / cb, z0 = (blk % cb) * 4;
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int y = 0; y < Mg; ++y) {
          const T tv = sT[yp * Mg + y];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (z0 + j < Mg) acc[j] += tv * sR[y * Mg + z0 + j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int z = z0 + j;
          if (z >= Mg) continue;
          T a = T(0);
          if (bx.periodic) {
            const int h = H[x * Mg + z];
            if (h >= 0) a = sF[yp * nh + h];
          }
          sU[yp * Mg + z] = acc[j] + a;
        }
      }
      __syncthreads();
      // E[y'][z'] += w_s sum_z U[y'][z] T[z][z']   (Kahan over the item's nodes)
      const T ws = (T)bx.w64[s];
      for (int blk = threadIdx.x; blk < Mg * cb; blk += blockDim.x) {
        const int yp = blk / cb, z0 = (blk % cb) * 4;
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int z = 0; z < Mg; ++z) {
          const T uv = sU[yp * Mg + z];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (z0 + j < Mg) acc[j] += uv * sT[z * Mg + z0 + j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (z0 + j < Mg) kahan_add(sE, sC, yp * Mg + z0 + j, ws * acc[j]);
      }
      __syncthreads();
    }
    // I x I x D term (periodic, once per slab): E[y][z'] += sum_{z on the z line at (x, y)}
    // Dbar[z'][z]
    if (bx.periodic && item.g == 0) {
      for (int i = threadIdx.x; i < mm; i += blockDim.x) {
        const int y = i / Mg, zp = i % Mg;
        const int h = H[x * Mg + y];
        if (h < 0) continue;
        kahan_add(sE, sC, i, bx.FDb[zp * nh + h]);
      }
      __syncthreads();
    }
    // publish the slab partial; the last group of the slab finalises the slab, the last
    // slab of the box finalises E_x
    const long long G3 = (long long)mm * Mg;
    T* P = bx.part + (long long)item.g * G3 + (long long)x * mm;
    for (int i = threadIdx.x; i < mm; i += blockDim.x) P[i] = sE[i] - sC[i];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(bx.slab_done + x, 1) == bx.n_groups - 1);
    __syncthreads();
    if (s_last) {
      __threadfence();
      double acc = 0.0;
      const long long base = (long long)x * mm;
      for (int i = threadIdx.x; i < mm; i += blockDim.x) {
        // every group's partial in flight at once, then added in group order
        T pv[kFusedMaxGroups];
#pragma unroll
        for (int g = 0; g < kFusedMaxGroups; ++g)
          pv[g] = g < bx.n_groups ? __ldcg(bx.part + (long long)g * G3 + base + i) : T(0);
        T sum = T(0), cmp = T(0);
#pragma unroll
        for (int g = 0; g < kFusedMaxGroups; ++g) {
          if (g >= bx.n_groups) break;
          const T yv = pv[g] - cmp;
          const T t = sum + yv;
          cmp = (t - sum) - yv;
          sum = t;
        }
        const int a = x - R, b = i / Mg - R, c = i % Mg - R;
        const int m = a * a + b * b + c * c;
        T v = T(0);
        if (m <= R * R) v = (T)(-bx.pref * (double)sum);
        eps_out[bx.eps_off + base + i] = v;
        if (m <= bx.R_F * bx.R_F) acc += (double)v;
      }
      s_red[threadIdx.x] = acc;
      __syncthreads();
      for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_red[threadIdx.x] += s_red[threadIdx.x + o];
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        bx.slab_ex[x] = s_red[0];
        __threadfence();
        s_last = (atomicAdd(done + item.box, 1) == Mg - 1);
      }
      __syncthreads();
      if (s_last) {  // the box's last slab: its shares read at once, added in slab order
        __threadfence();
        for (int k = threadIdx.x; k < Mg; k += blockDim.x) s_red[k] = __ldcg(bx.slab_ex + k);
        __syncthreads();
        if (threadIdx.x == 0) {
          double tot = 0.0;
          for (int k = 0; k < Mg; ++k) tot += s_red[k];
          ex_out[2 * bx.ex_idx] = 0.5 * tot;
          ex_out[2 * bx.ex_idx + 1] = tot;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace cc
