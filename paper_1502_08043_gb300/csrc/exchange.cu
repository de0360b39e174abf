// Exchange sums of the uniform electron gas (Sec. III) as Toeplitz mode products, plain
// FP32 / FP64 path on the SIMT cores.
//
// eps(k) = -sum_{j in F} V(k - n_j) is a 3D convolution of the occupation tensor O with
// V; with the node sum of Eq. 14 each node is a separable Gaussian, so
//   sum_j O(j) V(k - j) = pref sum_s w_s (O x1 T_s x2 T_s x3 T_s)(k)
// with T_s[a][b] = T_s[|a - b|] the Mg x Mg Toeplitz matrix of node s.
// PERIODIC kernel: the j = k term (q = 0) is excluded.  Subtracting sum_s w_s O(k) after
// the fact would cancel catastrophically (sum_s w_s is the quadrature of a divergent
// integral), so the identity
//   T x T x T - I x I x I = D x T x T + I x D x T + I x I x D,   D_s = T_s - I,
// is used instead: every term is a product of non-negative entries and the excluded
// term never appears.  Per chunk of nodes:
//   P_s = O x3 T_s,  Q_s = P_s x2 T_s,
//   E  += sum_s w_s D_s x2 P_s          (I x D x T)
//   E  += sum_s w_s D_s x1 Q_s          (D x T x T)
// and once:  E += O x3 (sum_s w_s D_s)  (I x I x D).
// BOX kernel: D_s = T_s and only the x1 term is kept (the full triple product).
// Then eps = -pref E on the basis sphere, E_x^sigma = 1/2 sum_{k in F} eps(k) in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace cc {

// ---------------------------------------------------------------- strided batched GEMM
// C[b1,b2](m,n) = beta C + sum_{j<J} sum_{k<K} A[b1,b2,j](m,k) B[b1,b2,j](k,n)
struct GemmDesc {
  const void* A;
  const void* B;
  void* C;
  int M, N, K, J, nb1, nb2;
  long long sAm, sAk, sAj, sAb1, sAb2;
  long long sBk, sBn, sBj, sBb1, sBb2;
  long long sCm, sCn, sCb1, sCb2;
  int beta;  // 0: overwrite, 1: accumulate
};

template <typename T, int BM, int BN, int NT>
__global__ void __launch_bounds__(NT) k_gemm(GemmDesc g) {
  constexpr int BK = 16;
  constexpr int TX = BN / 4, TY = BM / 4;  // NT == TX * TY threads, 4 x 4 outputs each
  static_assert(TX * TY == NT, "tile");
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int b1 = blockIdx.z / g.nb2, b2 = blockIdx.z % g.nb2;
  const T* A = reinterpret_cast<const T*>(g.A) + b1 * g.sAb1 + b2 * g.sAb2;
  const T* B = reinterpret_cast<const T*>(g.B) + b1 * g.sBb1 + b2 * g.sBb2;
  T* C = reinterpret_cast<T*>(g.C) + b1 * g.sCb1 + b2 * g.sCb2;
  const bool a_kc = g.sAk == 1, b_nc = g.sBn == 1;
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;
  T ra[LA], rb[LB];
  // running sum with a Kahan compensation term; every K tile of 16 products is summed
  // into fresh partials first, so the rounding error stays O(BK/2 + 3) ulps however long
  // the stacked K dimension (J nodes x K) is
  T acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = T(0);
  const int ktiles = (g.K + BK - 1) / BK;
  const int total = ktiles * g.J;
  auto load = [&](int t) {
    const int j = t / ktiles, k0 = (t % ktiles) * BK;
    const T* Aj = A + j * g.sAj;
    const T* Bj = B + j * g.sBj;
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int m, k;
      if (a_kc) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
      const int gm = m0 + m, gk = k0 + k;
      ra[r] = (gm < g.M && gk < g.K) ? Aj[gm * g.sAm + gk * g.sAk] : T(0);
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * NT;
      int n, k;
      if (b_nc) { n = e % BN; k = e / BN; } else { k = e % BK; n = e / BK; }
      const int gn = n0 + n, gk = k0 + k;
      rb[r] = (gn < g.N && gk < g.K) ? Bj[gk * g.sBk + gn * g.sBn] : T(0);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int m, k;
      if (a_kc) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
      As[k][m] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * NT;
      int n, k;
      if (b_nc) { n = e % BN; k = e / BN; } else { k = e % BK; n = e / BK; }
      Bs[k][n] = rb[r];
    }
  };
  if (total > 0) load(0);
  for (int t = 0; t < total; ++t) {
    __syncthreads();
    store();
    __syncthreads();
    if (t + 1 < total) load(t + 1);
    // two interleaved partial sums (even / odd k): 8-term chains, then one pairwise add
    T part[2][4][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[h][i][j] = T(0);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[k][ty + i * TY];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + j * TX];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[k & 1][i][j] += av[i] * bv[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const T y = (part[0][i][j] + part[1][i][j]) - cmp[i][j];
        const T s = acc[i][j] + y;
        cmp[i][j] = (s - acc[i][j]) - y;
        acc[i][j] = s;
      }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + i * TY;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + j * TX;
      if (gn >= g.N) continue;
      T* c = C + gm * g.sCm + gn * g.sCn;
      *c = g.beta ? *c + (acc[i][j] - cmp[i][j]) : acc[i][j] - cmp[i][j];
    }
  }
}

// tile configurations the autotuner chooses from
enum GemmTile { kTile64 = 0, kTile32 = 1, kTile64x32 = 2 };

template <typename T>
static cc_status gemm(const GemmDesc& g, int tile, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.nb1 * g.nb2 <= 0) return CC_OK;
  if ((long long)g.nb1 * g.nb2 > 65535) return CC_ERR_RANGE;
  if (tile == kTile32) {
    dim3 grid((g.N + 31) / 32, (g.M + 31) / 32, g.nb1 * g.nb2);
    k_gemm<T, 32, 32, 64><<<grid, 64, 0, st>>>(g);
  } else if (tile == kTile64x32) {
    dim3 grid((g.N + 31) / 32, (g.M + 63) / 64, g.nb1 * g.nb2);
    k_gemm<T, 64, 32, 128><<<grid, 128, 0, st>>>(g);
  } else {
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.nb1 * g.nb2);
    k_gemm<T, 64, 64, 256><<<grid, 256, 0, st>>>(g);
  }
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

// ---------------------------------------------------------------- element kernels
template <typename T>
__global__ void k_occ(T* occ, int R, int R_F) {
  const int Mg = 2 * R + 1;
  const long long G3 = (long long)Mg * Mg * Mg;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G3;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i / (Mg * Mg)) - R, y = (int)((i / Mg) % Mg) - R, z = (int)(i % Mg) - R;
    occ[i] = (x * x + y * y + z * z <= R_F * R_F) ? T(1) : T(0);
  }
}

// eps = -pref E on the basis sphere, 0 elsewhere; FP64 partial sums over the Fermi sphere
template <typename T, typename TO>
__global__ void k_finalize(const T* E, TO* eps, int R, int R_F, double pref, double* part) {
  const int Mg = 2 * R + 1;
  const long long G3 = (long long)Mg * Mg * Mg;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G3;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i / (Mg * Mg)) - R, y = (int)((i / Mg) % Mg) - R, z = (int)(i % Mg) - R;
    const int m = x * x + y * y + z * z;
    TO v = TO(0);
    if (m <= R * R) v = (TO)(-pref * (double)E[i]);
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

__global__ void k_reduce_ex(const double* part, int n, double* Ex) {
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
  }
}

// ---------------------------------------------------------------- workspace
static constexpr size_t kWorkspaceBudget = 512ull << 20;

cc_status workspace_alloc(cc_tables t) {
  Workspace& w = t->ws;
  const size_t G3 = (size_t)t->Mg * t->Mg * t->Mg;
  size_t chunk = kWorkspaceBudget / (2 * G3 * sizeof(double));
  if (chunk < 1) chunk = 1;
  if (chunk > (size_t)t->S_eff) chunk = t->S_eff;
  w.chunk = (int)chunk;
  const size_t pq = chunk * G3 * sizeof(double);
  void** slots[] = {&w.occ, &w.P, &w.Q, &w.E};
  const size_t sizes[] = {G3 * sizeof(double), pq, pq, G3 * sizeof(double)};
  for (int i = 0; i < 4; ++i) {
    cudaError_t e = cudaMalloc(slots[i], sizes[i]);
    if (e != cudaSuccess) {
      set_last_error("cudaMalloc(workspace)", e);
      return CC_ERR_ALLOC;
    }
    w.bytes += sizes[i];
  }
  cudaError_t e = cudaMalloc((void**)&w.part, sizeof(double) * kRedBlocks);
  if (e != cudaSuccess) {
    set_last_error("cudaMalloc(workspace)", e);
    return CC_ERR_ALLOC;
  }
  w.bytes += sizeof(double) * kRedBlocks;
  t->device_bytes += w.bytes;
  return CC_OK;
}

void workspace_free(cc_tables t) {
  Workspace& w = t->ws;
  void* ptrs[] = {w.occ, w.P, w.Q, w.E, w.part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  w.occ = w.P = w.Q = w.E = nullptr;
  w.part = nullptr;
}

// ---------------------------------------------------------------- tile choice
// Tile per GEMM class: a choice measured by cc_autotune_gemm for this (grid side,
// precision) when there is one; otherwise the process-wide setting (cc_set_gemm_tiles):
// 32x32 tiles for grid sides up to the threshold (40), above it 32x32 for the Mg x Mg
// products and 64x64 for the products with an Mg^2-long side.
static int g_tile_small[2] = {kTile32, kTile32};   // [fp32, fp64] the Mg x Mg products
static int g_tile_large[2] = {kTile64, kTile64};   // the Mg^2-long products
static int g_tile_threshold = 40;
// measured choices: [precision][grid side] -> small_tile + 3 * large_tile + 1 (0 = none)
static unsigned char g_tuned[2][256] = {};

static int tile_for(int Mg, bool long_dim, bool fp64) {
  const int tc = (Mg >= 0 && Mg < 256) ? __atomic_load_n(&g_tuned[fp64][Mg], __ATOMIC_ACQUIRE) : 0;
  if (tc) return long_dim ? (tc - 1) / 3 : (tc - 1) % 3;
  if (Mg <= g_tile_threshold) return kTile32;
  return long_dim ? g_tile_large[fp64] : g_tile_small[fp64];
}

// The plain path on an explicit workspace: occ, E ([Mg^3] each), P, Q ([chunk][Mg^3]
// each) of element type T, and part[kRedBlocks] doubles.
template <typename T>
static cc_status exchange_simt_ws(cc_tables t, const Workspace& w, int chunk, int R_F, T* eps,
                                  double* Ex, cudaStream_t st) {
  const int Mg = t->Mg, R = t->p.R;
  const long long M2 = (long long)Mg * Mg, G3 = M2 * Mg;
  const bool periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  const bool f64 = sizeof(T) == 8;
  T* occ = reinterpret_cast<T*>(w.occ);
  T* P = reinterpret_cast<T*>(w.P);
  T* Q = reinterpret_cast<T*>(w.Q);
  T* E = reinterpret_cast<T*>(w.E);
  const T* Tm = f64 ? reinterpret_cast<const T*>(t->d.Tm64) : reinterpret_cast<const T*>(t->d.Tm32);
  const T* WD = f64 ? reinterpret_cast<const T*>(t->d.WDm64) : reinterpret_cast<const T*>(t->d.WDm32);
  const T* Db = f64 ? reinterpret_cast<const T*>(t->d.Dbar64) : reinterpret_cast<const T*>(t->d.Dbar32);
  k_occ<T><<<1024, 256, 0, st>>>(occ, R, R_F);
  CC_CUDA(cudaMemsetAsync(E, 0, sizeof(T) * G3, st));
  const int tS = tile_for(Mg, false, f64), tL = tile_for(Mg, true, f64);
  for (int s0 = 0; s0 < t->S_eff; s0 += chunk) {
    const int cs = t->S_eff - s0 < chunk ? t->S_eff - s0 : chunk;
    const T* Tc = Tm + s0 * M2;
    const T* Wc = WD + s0 * M2;
    GemmDesc g{};
    // 1. P_s[(x,y)][z'] = sum_z O[(x,y)][z] T_s[z][z']
    g = GemmDesc{occ, Tc, P, (int)M2, Mg, Mg, 1, cs, 1,
                 Mg, 1, 0, 0, 0,
                 Mg, 1, 0, M2, 0,
                 Mg, 1, G3, 0, 0};
    CC_TRY(gemm<T>(g, tL, st));
    // 2. Q_s[x][y'][z] = sum_y T_s[y'][y] P_s[x][y][z]
    g = GemmDesc{Tc, P, Q, Mg, Mg, Mg, 1, cs, Mg,
                 Mg, 1, 0, M2, 0,
                 Mg, 1, 0, G3, M2,
                 Mg, 1, G3, M2, 0};
    CC_TRY(gemm<T>(g, tS, st));
    if (periodic) {
      // 3. E[x][y'][z] += sum_s sum_y w_s D_s[y'][y] P_s[x][y][z]
      g = GemmDesc{Wc, P, E, Mg, Mg, Mg, cs, Mg, 1,
                   Mg, 1, M2, 0, 0,
                   Mg, 1, G3, M2, 0,
                   Mg, 1, M2, 0, 1};
      CC_TRY(gemm<T>(g, tS, st));
    }
    // 4. E[x][(y,z)] += sum_s sum_x' w_s D_s[x][x'] Q_s[x'][(y,z)]
    g = GemmDesc{Wc, Q, E, Mg, (int)M2, Mg, cs, 1, 1,
                 Mg, 1, M2, 0, 0,
                 M2, 1, G3, 0, 0,
                 M2, 1, 0, 0, 1};
    CC_TRY(gemm<T>(g, tL, st));
  }
  if (periodic) {
    // 5. E[(x,y)][z] += sum_z' O[(x,y)][z'] Dbar[z'][z]
    GemmDesc g{occ, Db, E, (int)M2, Mg, Mg, 1, 1, 1,
               Mg, 1, 0, 0, 0,
               Mg, 1, 0, 0, 0,
               Mg, 1, 0, 0, 1};
    CC_TRY(gemm<T>(g, tL, st));
  }
  k_finalize<T, T><<<kRedBlocks, 256, 0, st>>>(E, eps, R, R_F, t->pref, w.part);
  k_reduce_ex<<<1, 256, 0, st>>>(w.part, kRedBlocks, Ex);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

// the plain path on the handle's own workspace (sized in doubles at build time)
template <typename T>
static cc_status exchange_simt(cc_tables t, int R_F, T* eps, double* Ex, cudaStream_t st) {
  const int chunk = (int)((size_t)t->ws.chunk * sizeof(double) / sizeof(T));
  return exchange_simt_ws<T>(t, t->ws, chunk, R_F, eps, Ex, st);
}

}  // namespace cc

using namespace cc;

// which form the plain FP32 exchange takes at grid sides 50..127 (process-wide)
static int g_simt_variant = 0;  // 0: automatic (SIMT slab kernel), 1: dense GEMM chain

extern "C" cc_status cc_exchange_sums(cc_tables t, int R_F, int precision, void* eps_dev,
                                      double* Ex_dev, void* stream) {
  if (!t || !eps_dev || !Ex_dev) return CC_ERR_ARG;
  if (R_F < 1 || R_F > t->p.R) return CC_ERR_RANGE;
  cudaStream_t st = as_stream(stream);
  // grids up to 49 per side: fused per-node work items with shared-memory intermediates
  if (t->fused && (precision == CC_PREC_FP32 || precision == CC_PREC_FP64))
    return fused_single_exchange(t, R_F, precision, eps_dev, Ex_dev, st);
  // FP32 at grid sides 50..127: the slab algorithm on the SIMT cores
  if (precision == CC_PREC_FP32 && t->simt &&
      __atomic_load_n(&g_simt_variant, __ATOMIC_ACQUIRE) == 0)
    return simt_slab_run(t, t->simt, R_F, (float*)eps_dev, Ex_dev, st);
  switch (precision) {
    case CC_PREC_FP32: return exchange_simt<float>(t, R_F, (float*)eps_dev, Ex_dev, st);
    case CC_PREC_FP64: return exchange_simt<double>(t, R_F, (double*)eps_dev, Ex_dev, st);
    case CC_PREC_BF16X3:
    case CC_PREC_FP16X3: return exchange_mixed(t, R_F, precision, (float*)eps_dev, Ex_dev, st);
  }
  return CC_ERR_ARG;
}

extern "C" cc_status cc_set_simt_variant(int variant) {
  if (variant < 0 || variant > 1) return CC_ERR_ARG;
  __atomic_store_n(&g_simt_variant, variant, __ATOMIC_RELEASE);
  return CC_OK;
}

// Autotuner of the SIMT GEMM tiles: times the dense chain of mode products of this handle
// with every (small, large) tile pair and keeps the fastest for this grid side and precision.
extern "C" cc_status cc_autotune_gemm(cc_tables t, int precision, int R_F, int reps,
                                      int* choice_host, float* ms_host, void* stream) {
  if (!t || (precision != CC_PREC_FP32 && precision != CC_PREC_FP64) || reps < 1) return CC_ERR_ARG;
  if (R_F < 1 || R_F > t->p.R) return CC_ERR_RANGE;
  if (t->Mg >= 256) return CC_ERR_RANGE;
  cudaStream_t st = as_stream(stream);
  const bool f64 = precision == CC_PREC_FP64;
  const size_t G3 = (size_t)t->Mg * t->Mg * t->Mg;
  void* eps = nullptr;
  double* Ex = nullptr;
  if (cudaMalloc(&eps, G3 * (f64 ? 8 : 4)) != cudaSuccess ||
      cudaMalloc((void**)&Ex, 2 * sizeof(double)) != cudaSuccess) {
    cudaFree(eps);
    return CC_ERR_ALLOC;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = -1.0f;
  int bs = 0, bl = 0;
  cc_status s = CC_OK;
  for (int ts = 0; ts < 3 && s == CC_OK; ++ts)
    for (int tl = 0; tl < 3 && s == CC_OK; ++tl) {
      __atomic_store_n(&g_tuned[f64][t->Mg], (unsigned char)(ts + 3 * tl + 1), __ATOMIC_RELEASE);
      auto run = [&]() {
        return f64 ? exchange_simt<double>(t, R_F, (double*)eps, Ex, st)
                   : exchange_simt<float>(t, R_F, (float*)eps, Ex, st);
      };
      s = run();  // warm-up
      if (s != CC_OK) break;
      std::vector<float> ms(reps);
      for (int r = 0; r < reps && s == CC_OK; ++r) {
        cudaEventRecord(e0, st);
        s = run();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = CC_ERR_CUDA;
        cudaEventElapsedTime(&ms[r], e0, e1);
      }
      if (s != CC_OK) break;
      std::sort(ms.begin(), ms.end());
      const float med = ms[reps / 2];
      if (best < 0.0f || med < best) {
        best = med;
        bs = ts;
        bl = tl;
      }
    }
  __atomic_store_n(&g_tuned[f64][t->Mg], (unsigned char)(s == CC_OK ? bs + 3 * bl + 1 : 0),
                   __ATOMIC_RELEASE);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(eps);
  cudaFree(Ex);
  if (s != CC_OK) return s;
  if (choice_host) {
    choice_host[0] = bs;
    choice_host[1] = bl;
  }
  if (ms_host) *ms_host = best;
  return CC_OK;
}

// The measured tile choice for a grid side and precision: small_tile, large_tile, or -1, -1
// when none has been measured in this process.
extern "C" cc_status cc_gemm_tiles_tuned(int precision, int Mg, int* small_tile, int* large_tile) {
  if ((precision != CC_PREC_FP32 && precision != CC_PREC_FP64) || !small_tile || !large_tile)
    return CC_ERR_ARG;
  if (Mg < 0 || Mg >= 256) return CC_ERR_RANGE;
  const int tc = __atomic_load_n(&g_tuned[precision == CC_PREC_FP64][Mg], __ATOMIC_ACQUIRE);
  *small_tile = tc ? (tc - 1) % 3 : -1;
  *large_tile = tc ? (tc - 1) / 3 : -1;
  return CC_OK;
}

// Tile selection for the SIMT mode products: small = Mg x Mg batched products, large =
// products with an Mg^2-long dimension; threshold = grid side up to which 32 x 32 tiles
// are always used.  Values: 0 = 64x64, 1 = 32x32, 2 = 64x32.  Set by the autotuner.
extern "C" cc_status cc_set_gemm_tiles(int precision, int small_tile, int large_tile,
                                       int threshold) {
  if (precision != CC_PREC_FP32 && precision != CC_PREC_FP64) return CC_ERR_ARG;
  if (small_tile < 0 || small_tile > 2 || large_tile < 0 || large_tile > 2) return CC_ERR_ARG;
  const int f = precision == CC_PREC_FP64;
  g_tile_small[f] = small_tile;
  g_tile_large[f] = large_tile;
  if (threshold >= 0) g_tile_threshold = threshold;
  return CC_OK;
}

// ---------------------------------------------------------------- allocation-free variant
// Some callers cannot call cudaMalloc when they need the exchange sums: code that runs
// under a framework's caching allocator which owns the device memory and must not have
// memory taken behind its back, and latency-critical loops where cudaMalloc's implicit
// device synchronisation would stall every other stream.  cc_exchange_sums_noalloc serves
// them: it runs the plain FP32 path of cc_exchange_sums with its scratch (occupation
// tensor, accumulator, node-chunk intermediates, reduction partials) in the fixed device
// array below instead of the handle's workspace.  The array lives in the library image,
// so every GPU that loads the library holds it until the process exits.
namespace cc {
constexpr size_t kNoAllocScratchBytes = 16ull << 20;  // 16 MiB per device
constexpr int kNoAllocMaxR = 31;                      // grid side (2R + 1) <= 63
constexpr int kNoAllocMaxDevices = 64;
}  // namespace cc

static __device__ __align__(256) unsigned char g_noalloc_scratch[cc::kNoAllocScratchBytes];

namespace cc {
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (with
// that device current) and cached for the process (one primary context per device).  The
// handle's tables must live on that same device.
static cc_status noalloc_scratch(cc_tables t, void** out) {
  int dev = 0;
  CC_CUDA(cudaGetDevice(&dev));
  if (dev != t->device) return CC_ERR_ARG;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return CC_ERR_RANGE;
  void* p = __atomic_load_n(&g_noalloc_ptr[dev], __ATOMIC_ACQUIRE);
  if (!p) {
    CC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    __atomic_store_n(&g_noalloc_ptr[dev], p, __ATOMIC_RELEASE);
  }
  *out = p;
  return CC_OK;
}

// Called when a handle is built, where allocating is allowed.  With lazy module loading
// (the CUDA default) the first use of this file's module allocates the scratch array and
// loads the kernels; an allocation-free call that came first would pay for both.  So the
// array's address is resolved and the FP32 chain's kernels are loaded here.  Best effort:
// a failure leaves the lookup to the first call and clears the error.
void noalloc_preload(cc_tables t) {
  if (t->p.R > kNoAllocMaxR) return;
  void* p = nullptr;
  if (noalloc_scratch(t, &p) != CC_OK) {
    (void)cudaGetLastError();
    return;
  }
  const void* kernels[] = {(const void*)k_occ<float>, (const void*)k_gemm<float, 32, 32, 64>,
                           (const void*)k_gemm<float, 64, 32, 128>,
                           (const void*)k_gemm<float, 64, 64, 256>,
                           (const void*)k_finalize<float, float>, (const void*)k_reduce_ex};
  for (const void* k : kernels) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, k) != cudaSuccess) (void)cudaGetLastError();
  }
}
}  // namespace cc

extern "C" cc_status cc_exchange_sums_noalloc(cc_tables t, int R_F, float* eps_dev,
                                              double* Ex_dev, void* stream) {
  if (!t || !eps_dev || !Ex_dev) return CC_ERR_ARG;
  if (t->p.R > kNoAllocMaxR) return CC_ERR_RANGE;
  if (R_F < 1 || R_F > t->p.R) return CC_ERR_RANGE;
  void* base = nullptr;
  CC_TRY(noalloc_scratch(t, &base));
  // layout: occ | E | part (each start 256-byte aligned) | P[chunk][Mg^3] | Q[chunk][Mg^3]
  const size_t G3 = (size_t)t->Mg * t->Mg * t->Mg;
  const size_t tensor = G3 * sizeof(float);
  const size_t vol = (tensor + 255) & ~(size_t)255;
  const size_t fixed = 2 * vol + ((sizeof(double) * kRedBlocks + 255) & ~(size_t)255);
  if (fixed + 2 * tensor > kNoAllocScratchBytes) return CC_ERR_RANGE;
  size_t chunk = (kNoAllocScratchBytes - fixed) / (2 * tensor);
  if (chunk > (size_t)t->S_eff) chunk = t->S_eff;
  unsigned char* b = static_cast<unsigned char*>(base);
  Workspace w;
  w.occ = b;
  w.E = b + vol;
  w.part = reinterpret_cast<double*>(b + 2 * vol);
  w.P = b + fixed;
  w.Q = b + fixed + chunk * tensor;
  return exchange_simt_ws<float>(t, w, (int)chunk, R_F, eps_dev, Ex_dev, as_stream(stream));
}
