// Fused exchange-sum work items for small grids (grid side Mg <= 49): one CTA computes
// the contribution of a group of quadrature nodes of one box to the exchange sums
// (Sec. III; node sum of Sec. II Eq. 14 with the D = T - I split of the periodic
// kernel), keeping the per-node intermediates P_s = O x3 T_s and Q_s = P_s x2 T_s in
// shared memory when they fit, else in a per-CTA slice of global scratch.  The last
// CTA to finish a box adds the item partials, writes eps and reduces E_x (FP64).
// Work items are handed out by an atomic counter to a persistent grid; nothing waits
// on another CTA, so the scheme cannot deadlock whatever the residency.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace cc {

template <typename T>
struct FusedBox {
  int R, R_F, Mg, S_eff, periodic, n_items;
  double pref;
  const T* Tm;   // [S_eff][Mg][Mg]  T_s
  const T* WD;   // [S_eff][Mg][Mg]  w_s D_s (periodic) or w_s T_s (box)
  const T* Db;   // [Mg][Mg] sum_s w_s D_s (periodic)
  T* part;       // [n_items][2][Mg^3]  Kahan sum and compensation per item
  long long eps_off;  // offset of this box's eps block in the output
  int ex_idx;         // this box's E_x pair in the output
};

struct FusedItem {
  int box, s0, s1, g;
};

constexpr int kFusedThreads = 512;

template <typename T>
__device__ __forceinline__ void kahan_add(T* e, T* c, long long i, T v) {
  const T y = v - c[i];
  const T t = e[i] + y;
  c[i] = (t - e[i]) - y;
  e[i] = t;
}

__device__ __forceinline__ bool occ_at(int x, int y, int z, int R, int R_F) {
  const int a = x - R, b = y - R, c = z - R;
  return a * a + b * b + c * c <= R_F * R_F;
}

// z mode on the occupation tensor: P[(x,y)][z'] = sum_z O[x][y][z] M[z][z'] (M symmetric);
// row (x,y) of O is 1 exactly on the contiguous z range zr[row] = (z_lo, z_hi) of the
// Fermi sphere (empty when z_lo > z_hi); written (overwrite) or Kahan-added into (E, C)
template <typename T, bool kAcc>
__device__ void zmode_occ(const T* __restrict__ M, int Mg, const short2* zr, T* P, T* E, T* C) {
  const int rows = Mg * Mg;
  const int rb = (rows + 3) / 4, cb = (Mg + 3) / 4;
  for (int blk = threadIdx.x; blk < rb * cb; blk += blockDim.x) {
    const int r0 = (blk / cb) * 4, c0 = (blk % cb) * 4;
    T acc[4][4] = {};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + i;
      if (r >= rows) continue;
      const short2 z = zr[r];
      for (int zz = z.x; zz <= z.y; ++zz) {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += (c0 + j < Mg) ? M[zz * Mg + c0 + j] : T(0);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + i;
      if (r >= rows) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (c0 + j >= Mg) continue;
        const long long o = (long long)r * Mg + c0 + j;
        if (kAcc) kahan_add(E, C, o, acc[i][j]);
        else P[o] = acc[i][j];
      }
    }
  }
}

// y mode: out[x][y'][z] (=|+=) sum_y M[y'][y] X[x][y][z]
template <typename T, bool kAcc>
__device__ void ymode(const T* __restrict__ M, const T* X, int Mg, T* out, T* E, T* C) {
  const int yb = (Mg + 3) / 4, zb = (Mg + 3) / 4;
  const int nblk = Mg * yb * zb;
  for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) {
    const int x = blk / (yb * zb);
    const int rem = blk % (yb * zb);
    const int y0 = (rem / zb) * 4, z0 = (rem % zb) * 4;
    T acc[4][4] = {};
    const T* Xx = X + (long long)x * Mg * Mg;
    for (int y = 0; y < Mg; ++y) {
      T m[4], v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) m[i] = (y0 + i < Mg) ? M[(y0 + i) * Mg + y] : T(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = (z0 + j < Mg) ? Xx[y * Mg + z0 + j] : T(0);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += m[i] * v[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (y0 + i >= Mg) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (z0 + j >= Mg) continue;
        const long long o = ((long long)x * Mg + y0 + i) * Mg + z0 + j;
        if (kAcc) kahan_add(E, C, o, acc[i][j]);
        else out[o] = acc[i][j];
      }
    }
  }
}

// x mode (accumulating): E[x][(y,z)] += sum_x' M[x][x'] X[x'][(y,z)]
template <typename T>
__device__ void xmode_acc(const T* __restrict__ M, const T* X, int Mg, T* E, T* C) {
  const int N = Mg * Mg;
  const int xb = (Mg + 3) / 4, nb = (N + 3) / 4;
  for (int blk = threadIdx.x; blk < xb * nb; blk += blockDim.x) {
    const int x0 = (blk / nb) * 4, n0 = (blk % nb) * 4;
    T acc[4][4] = {};
    for (int xp = 0; xp < Mg; ++xp) {
      T m[4], v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) m[i] = (x0 + i < Mg) ? M[(x0 + i) * Mg + xp] : T(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = (n0 + j < N) ? X[(long long)xp * N + n0 + j] : T(0);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += m[i] * v[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (x0 + i >= Mg) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (n0 + j >= N) continue;
        kahan_add(E, C, (long long)(x0 + i) * N + n0 + j, acc[i][j]);
      }
    }
  }
}

// One persistent launch over all items of all boxes.  Scratch for P and Q: dynamic
// shared memory when smem_pq != 0, else gscratch + blockIdx.x * 2 * max_g3.
template <typename T>
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_fused_exchange(const FusedBox<T>* __restrict__ boxes, const FusedItem* __restrict__ items,
                     int n_items, int* work, int* done, T* gscratch, long long max_g3,
                     int smem_pq, int rf_override, T* eps_out, double* ex_out) {
  extern __shared__ __align__(16) unsigned char fsmem[];
  __shared__ int s_item, s_last;
  __shared__ double s_red[kFusedThreads];
  // dynamic shared memory: [Ts | Ws | Db : 3 Mg_max^2] [z ranges: Mg_max^2 short2] [P | Q]
  const int mgmax = (int)llround(cbrt((double)max_g3));
  T* sT = reinterpret_cast<T*>(fsmem);
  T* sW = sT + mgmax * mgmax;
  T* sD = sW + mgmax * mgmax;
  short2* zr = reinterpret_cast<short2*>(sD + mgmax * mgmax);
  T* P;
  T* Q;
  if (smem_pq) {
    const size_t off = ((size_t)3 * mgmax * mgmax * sizeof(T) + (size_t)mgmax * mgmax * 4 + 15) &
                       ~(size_t)15;
    P = reinterpret_cast<T*>(fsmem + off);
    Q = P + max_g3;
  } else {
    P = gscratch + (long long)blockIdx.x * 2 * max_g3;
    Q = P + max_g3;
  }
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const FusedItem item = items[it];
    FusedBox<T> bx = boxes[item.box];
    if (rf_override > 0) bx.R_F = rf_override;
    const int Mg = bx.Mg;
    const long long G3 = (long long)Mg * Mg * Mg, M2 = (long long)Mg * Mg;
    T* E = bx.part + (long long)item.g * 2 * G3;
    T* C = E + G3;
    for (long long i = threadIdx.x; i < 2 * G3; i += blockDim.x) E[i] = T(0);
    for (int r = threadIdx.x; r < M2; r += blockDim.x) {   // Fermi-sphere z range per row
      const int x = r / Mg - bx.R, y = r % Mg - bx.R;
      const int h2 = bx.R_F * bx.R_F - x * x - y * y;
      short2 z = make_short2(1, 0);
      if (h2 >= 0) {
        int h = (int)sqrtf((float)h2);
        while (h * h > h2) --h;
        while ((h + 1) * (h + 1) <= h2) ++h;
        z = make_short2((short)(bx.R - h), (short)(bx.R + h));
      }
      zr[r] = z;
    }
    __syncthreads();
    for (int s = item.s0; s < item.s1; ++s) {
      for (int i = threadIdx.x; i < M2; i += blockDim.x) {
        sT[i] = bx.Tm[s * M2 + i];
        sW[i] = bx.WD[s * M2 + i];
      }
      __syncthreads();
      zmode_occ<T, false>(sT, Mg, zr, P, nullptr, nullptr);             // P = O x3 T
      __syncthreads();
      ymode<T, false>(sT, P, Mg, Q, nullptr, nullptr);                   // Q = P x2 T
      if (bx.periodic) ymode<T, true>(sW, P, Mg, nullptr, E, C);         // E += P x2 wD
      __syncthreads();
      xmode_acc<T>(sW, Q, Mg, E, C);                                     // E += Q x1 wD
      __syncthreads();
    }
    if (bx.periodic && item.g == 0) {
      for (int i = threadIdx.x; i < M2; i += blockDim.x) sD[i] = bx.Db[i];
      __syncthreads();
      zmode_occ<T, true>(sD, Mg, zr, nullptr, E, C);                    // E += O x3 Dbar
      __syncthreads();
    }
    // publish this item; the last item of the box finalises it
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(done + item.box, 1) == bx.n_items - 1);
    __syncthreads();
    if (s_last) {
      __threadfence();
      double acc = 0.0;
      const int R = bx.R;
      for (long long i = threadIdx.x; i < G3; i += blockDim.x) {
        T sum = T(0), cmp = T(0);
        for (int g = 0; g < bx.n_items; ++g) {
          const T* Eg = bx.part + (long long)g * 2 * G3;
          const T v = __ldcg(Eg + i) - __ldcg(Eg + G3 + i);
          const T y = v - cmp;
          const T t = sum + y;
          cmp = (t - sum) - y;
          sum = t;
        }
        const int x = (int)(i / M2) - R, y = (int)((i / Mg) % Mg) - R, z = (int)(i % Mg) - R;
        const int m = x * x + y * y + z * z;
        T v = T(0);
        if (m <= R * R) v = (T)(-bx.pref * (double)sum);
        eps_out[bx.eps_off + i] = v;
        if (m <= bx.R_F * bx.R_F) acc += (double)v;
      }
      s_red[threadIdx.x] = acc;
      __syncthreads();
      for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_red[threadIdx.x] += s_red[threadIdx.x + o];
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        ex_out[2 * bx.ex_idx] = 0.5 * s_red[0];
        ex_out[2 * bx.ex_idx + 1] = s_red[0];
      }
    }
    __syncthreads();
  }
}

}  // namespace cc
