// Plain FP32 exchange sums on the SIMT cores by the algorithm of the fused tensor-core slab
// kernel (tcslab.cu), for single boxes of grid side 50..127.
//
// Sec. III exchange of the uniform electron gas with the node sum of Sec. II Eq. 14; the
// periodic kernel uses the D_s = T_s - I split, so with the Fermi-sphere occupation O
//   E[x] = sum_s (T_s R'_{s,x} + A'_{s,x}) T_s  +  (I x I x Dbar term),
// for the slab x (matrices over y, z):
//   R'_{s,x}[y][z] = w_s F_s[x][h(y, z)]   the first mode product of O (line along x),
//   A'_{s,x}[y][z] = w_s F_s[y][h(x, z)]   O x2 D_s restricted to the slab (line along y),
//   F_s[a][h]      = sum_{k = R-h}^{R+h} D_s[a][k]  (window sums in FP64, rounded once),
//   h(u, v)        = floor(sqrt(R_F^2 - (u-R)^2 - (v-R)^2)), -1 outside the sphere.
// The box kernel has F_s from T_s, no A' term and no Dbar term.  R' and U = T R' + A'
// vanish outside the band |y - R|, |z - R| <= R_F, so both remaining mode products run
// over the band only: U (rows y', band columns z) = T[:, band] R' + A', then
// E[y'][z'] += sum_{z in band} U[y'][z] T[z][z'].  Everything is FP32 with FMA chains of at
// most 2 R_F + 1 terms per product; the node sum of each output is Kahan-compensated.
//
// Work unit = (slab x, half of the rows y', node s); a persistent grid, each CTA a
// contiguous run of units (slab-major), so consecutive units of a CTA share (x, half) and
// accumulate E in registers over their nodes; the run leaves one partial per (x, half) and
// CTA, which a second kernel adds in a fixed order (deterministic) with the Dbar term to
// form eps and the FP64 row sums of E_x.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "slab_finalize.cuh"

namespace cc {

namespace {

constexpr int kThreads = 256;   // 16 x 16 thread grid
constexpr int kRows = 64;       // rows y' of one unit
constexpr int kHMax = 64;       // window half-lengths h = 0 .. R_F <= 63
constexpr int kCols = 128;      // columns of the padded grid (grid side <= 127)
constexpr int kUtStride = kRows + 4;  // padded row of the transposed U

struct SArgs {
  int R, RF, Mg, S, nh, units, maxseg;
  const float* Tm;  // [S][Mg][Mg] T_s
  const float* FW;  // [S][kHMax][kCols] w_s F_s[a][h], h-major
  float* part;      // [Mg * nh][maxseg][kRows][kCols] partial E of a (slab, half)
};


// shared memory of one CTA: Tb[nb][16 EW] | Rm[nb][16 ZW] | Ut[16 ZW][kUtStride] | ftab[64]
// | hyz[nb][nb] (bytes)
__host__ __device__ inline size_t simt_smem_bytes(int nb, int ZW, int EW) {
  return sizeof(float) * ((size_t)nb * 16 * EW + (size_t)nb * 16 * ZW +
                          (size_t)16 * ZW * kUtStride + kHMax) +
         (((size_t)nb * nb + 15) & ~(size_t)15);
}

// ZW: band columns of U per thread (band padded to 16 ZW); EW: E columns per thread
// (grid padded to 16 EW)
template <int ZW, int EW, bool kPeriodic>
__global__ void __launch_bounds__(kThreads, 2) k_simt_slab(SArgs g) {
  extern __shared__ __align__(16) float sm[];
  constexpr int NBP = 16 * ZW, NCP = 16 * EW;
  const int R = g.R, RF = g.RF, Mg = g.Mg, S = g.S;
  const int zlo = R - RF, nb = 2 * RF + 1;
  float* Tb = sm;                        // T_s rows z in the band, every column z'
  float* Rm = Tb + nb * NCP;             // R'[y][z], band x band
  float* Ut = Rm + nb * NBP;             // U[y'][z] stored as [z][y']
  float* ftab = Ut + NBP * kUtStride;    // w_s F_s[x][h]
  signed char* hyz = reinterpret_cast<signed char*>(ftab + kHMax);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  // h(y, z) on the band square; zero the padding once (never written afterwards)
  for (int i = tid; i < nb * nb; i += kThreads) {
    const int dy = i / nb - RF, dz = i % nb - RF;
    const int q = RF * RF - dy * dy - dz * dz;
    hyz[i] = (signed char)(q >= 0 ? isqrt_int(q) : -1);
  }
  for (int i = tid; i < nb * NCP; i += kThreads) Tb[i] = 0.0f;
  for (int i = tid; i < nb * NBP; i += kThreads) Rm[i] = 0.0f;

  const long long u0 = (long long)blockIdx.x * g.units / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * g.units / gridDim.x;
  float E[4][EW], C[4][EW];
  for (long long u = u0; u < u1; ++u) {
    const int xh = (int)(u / S), s = (int)(u % S);
    const int x = xh / g.nh, row0 = kRows * (xh % g.nh);
    if (u == u0 || s == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < EW; ++j) E[i][j] = C[i][j] = 0.0f;
    }
    __syncthreads();  // the previous unit is done with Tb, Rm, Ut, ftab
    // 1. T_s band rows, w_s F_s[x][.]
    const float* Ts = g.Tm + (long long)s * Mg * Mg;
    for (int i = tid; i < nb * Mg; i += kThreads) {
      const int r = i / Mg, c = i % Mg;
      Tb[r * NCP + c] = __ldg(Ts + (long long)(zlo + r) * Mg + c);
    }
    const float* FWs = g.FW + (long long)s * kHMax * kCols;
    if (tid <= RF) ftab[tid] = __ldg(FWs + tid * kCols + x);
    __syncthreads();
    // 2. R'[y][z] = w_s F_s[x][h(y, z)]
    for (int i = tid; i < nb * nb; i += kThreads) {
      const int h = hyz[i];
      Rm[(i / nb) * NBP + i % nb] = h >= 0 ? ftab[h] : 0.0f;
    }
    __syncthreads();
    // 3. U[y'][z] = sum_{y in band} T[y'][y] R'[y][z] + A'[y'][z]   (T symmetric:
    //    T[y'][y] = Tb[y - zlo][y']), rows y' = row0 + 4 ty + i, band columns ZW tx + j
    {
      float acc[4][ZW];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < ZW; ++j) acc[i][j] = 0.0f;
      const float* ta = Tb + row0 + 4 * ty;
      const float* rb = Rm + ZW * tx;
#pragma unroll 2
      for (int k = 0; k < nb; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(ta + k * NCP);
        float b[ZW];
#pragma unroll
        for (int j = 0; j < ZW; j += 2) {
          const float2 v = *reinterpret_cast<const float2*>(rb + k * NBP + j);
          b[j] = v.x;
          b[j + 1] = v.y;
        }
#pragma unroll
        for (int j = 0; j < ZW; ++j) {
          acc[0][j] = fmaf(a.x, b[j], acc[0][j]);
          acc[1][j] = fmaf(a.y, b[j], acc[1][j]);
          acc[2][j] = fmaf(a.z, b[j], acc[2][j]);
          acc[3][j] = fmaf(a.w, b[j], acc[3][j]);
        }
      }
#pragma unroll
      for (int j = 0; j < ZW; ++j) {
        const int zi = ZW * tx + j;
        if (zi >= nb) continue;
        float4 v = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        if (kPeriodic) {
          // A'[y'][z] = w_s F_s[y'][h(x, z)]: the x line must cross the sphere
          const int dx = x - R;
          const int h = (dx >= -RF && dx <= RF) ? hyz[(dx + RF) * nb + zi] : -1;
          if (h >= 0) {
            const float4 f =
                __ldg(reinterpret_cast<const float4*>(FWs + h * kCols + row0 + 4 * ty));
            v.x += f.x;
            v.y += f.y;
            v.z += f.z;
            v.w += f.w;
          }
        }
        *reinterpret_cast<float4*>(Ut + zi * kUtStride + 4 * ty) = v;
      }
    }
    __syncthreads();
    // 4. E[y'][z'] += sum_{z in band} U[y'][z] T[z][z'], columns z' = EW tx + j
    {
      float P[4][EW];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < EW; ++j) P[i][j] = 0.0f;
      const float* ua = Ut + 4 * ty;
      const float* tb = Tb + EW * tx;
#pragma unroll 2
      for (int k = 0; k < nb; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(ua + k * kUtStride);
        float b[EW];
#pragma unroll
        for (int j = 0; j < EW; j += 4) {
          const float4 v = *reinterpret_cast<const float4*>(tb + k * NCP + j);
          b[j] = v.x;
          b[j + 1] = v.y;
          b[j + 2] = v.z;
          b[j + 3] = v.w;
        }
#pragma unroll
        for (int j = 0; j < EW; ++j) {
          P[0][j] = fmaf(a.x, b[j], P[0][j]);
          P[1][j] = fmaf(a.y, b[j], P[1][j]);
          P[2][j] = fmaf(a.z, b[j], P[2][j]);
          P[3][j] = fmaf(a.w, b[j], P[3][j]);
        }
      }
      // Kahan-compensated node sum
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < EW; ++j) {
          const float yv = P[i][j] - C[i][j];
          const float t = E[i][j] + yv;
          C[i][j] = (t - E[i][j]) - yv;
          E[i][j] = t;
        }
    }
    // the last node of this (slab, half) on this CTA: publish the partial
    if (u + 1 == u1 || (u + 1) % S == 0) {
      const int kseg = (int)blockIdx.x - owner_cta((long long)xh * S, g.units, gridDim.x);
      float* P = g.part + (((long long)xh * g.maxseg + kseg) * kRows + 4 * ty) * kCols + EW * tx;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < EW; j += 4)
          *reinterpret_cast<float4*>(P + i * kCols + j) =
              make_float4(E[i][j] - C[i][j], E[i][j + 1] - C[i][j + 1],
                          E[i][j + 2] - C[i][j + 2], E[i][j + 3] - C[i][j + 3]);
    }
  }
  signal_finalizer();
}

// w_s F_s[a][h] (FP64 window sums of D_s = T_s - I, or of T_s for the box kernel, rounded
// once), h-major; and the Dbar window sums.  One thread per (s, a).
__global__ void k_simt_prep(const double* Tm, const double* w, int S, int Mg, int R, int RF,
                            int periodic, float* FW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * kCols) return;
  const int s = i / kCols, a = i % kCols;
  const double* row = Tm + ((long long)s * Mg + (a < Mg ? a : 0)) * Mg;
  auto X = [&](int k) { return (periodic && k == a) ? 0.0 : row[k]; };
  double acc = 0.0;
  for (int h = 0; h < kHMax; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? X(R) : X(R - h) + X(R + h);
      f = acc;
    }
    FW[((long long)s * kHMax + h) * kCols + a] = (float)(w[s] * f);
  }
}

__global__ void k_simt_dbar(const double* Dbar, int Mg, int R, int RF, float* FB) {
  const int a = threadIdx.x;
  double acc = 0.0;
  for (int h = 0; h < kHMax; ++h) {
    double f = 0.0;
    if (a < Mg && h <= RF) {
      acc += h == 0 ? Dbar[a * Mg + R] : Dbar[a * Mg + R - h] + Dbar[a * Mg + R + h];
      f = acc;
    }
    FB[h * kCols + a] = (float)f;
  }
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int ZW, int EW, bool P>
cc_status launch_zw(const SArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto k = k_simt_slab<ZW, EW, P>;
  CC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<grid, kThreads, smem, st>>>(a);
  return CC_OK;
}

template <int EW, bool P>
cc_status launch_ew(const SArgs& a, int zw, int grid, size_t smem, cudaStream_t st) {
  switch (zw) {
    case 2: return launch_zw<2, EW, P>(a, grid, smem, st);
    case 4: return launch_zw<4, EW, P>(a, grid, smem, st);
    case 6: return launch_zw<6, EW, P>(a, grid, smem, st);
    default: return launch_zw<8, EW, P>(a, grid, smem, st);
  }
}

}  // namespace

struct SimtSlabWs {
  int RF_built = -1;
  int nh = 0, units = 0, grid = 0, maxseg = 0;
  float* FW = nullptr;
  float* FB = nullptr;
  float* part = nullptr;
  double* blk_ex = nullptr;
  unsigned* ticket = nullptr;  // blocks of the finaliser done (0 between calls)
  std::vector<void*> allocs;
};

bool simt_slab_supported(cc_tables t) { return t->Mg > kFusedMaxMg && t->Mg <= 127; }

void simt_slab_free(void* p) {
  SimtSlabWs* w = reinterpret_cast<SimtSlabWs*>(p);
  if (!w) return;
  for (void* a : w->allocs) cudaFree(a);
  delete w;
}

cc_status simt_slab_alloc(cc_tables t, void** out) {
  *out = nullptr;
  if (!simt_slab_supported(t)) return CC_OK;
  SimtSlabWs* w = new (std::nothrow) SimtSlabWs();
  if (!w) return CC_ERR_ALLOC;
  const int S = t->S_eff, Mg = t->Mg;
  w->nh = (Mg + kRows - 1) / kRows;
  w->units = Mg * w->nh * S;
  w->grid = std::min(2 * num_sms(), w->units);
  for (int xh = 0; xh < Mg * w->nh; ++xh) {
    const int c0 = owner_cta((long long)xh * S, w->units, w->grid);
    const int c1 = owner_cta((long long)(xh + 1) * S - 1, w->units, w->grid);
    w->maxseg = std::max(w->maxseg, c1 - c0 + 1);
  }
  auto alloc = [&](void** p, size_t bytes) -> cc_status {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      set_last_error("cudaMalloc(SIMT slab workspace)", e);
      return CC_ERR_ALLOC;
    }
    w->allocs.push_back(*p);
    t->device_bytes += bytes;
    return CC_OK;
  };
  cc_status st = CC_OK;
  if ((st = alloc((void**)&w->FW, sizeof(float) * S * kHMax * kCols)) != CC_OK ||
      (st = alloc((void**)&w->FB, sizeof(float) * kHMax * kCols)) != CC_OK ||
      (st = alloc((void**)&w->part, sizeof(float) * (size_t)Mg * w->nh * w->maxseg * kRows *
                                        kCols)) != CC_OK ||
      (st = alloc((void**)&w->blk_ex, sizeof(double) * Mg * Mg)) != CC_OK ||
      (st = alloc((void**)&w->ticket, sizeof(unsigned))) != CC_OK) {
    simt_slab_free(w);
    return st;
  }
  if (cudaMemset(w->ticket, 0, sizeof(unsigned)) != cudaSuccess) {
    set_last_error("cudaMemset(finaliser ticket)", cudaGetLastError());
    simt_slab_free(w);
    return CC_ERR_CUDA;
  }
  *out = w;
  return CC_OK;
}

cc_status simt_slab_run(cc_tables t, void* ws, int R_F, float* eps, double* Ex,
                        cudaStream_t st) {
  SimtSlabWs* w = reinterpret_cast<SimtSlabWs*>(ws);
  if (!w || !simt_slab_supported(t) || R_F > 63) return CC_ERR_NOTSUPP;
  const int S = t->S_eff, Mg = t->Mg, R = t->p.R;
  const int periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  if (w->RF_built != R_F) {
    k_simt_prep<<<(S * kCols + 127) / 128, 128, 0, st>>>(t->d.Tm64, t->d.w64, S, Mg, R, R_F,
                                                          periodic, w->FW);
    if (periodic) k_simt_dbar<<<1, kCols, 0, st>>>(t->d.Dbar64, Mg, R, R_F, w->FB);
    CC_CUDA(cudaGetLastError());
    w->RF_built = R_F;
  }
  const int nb = 2 * R_F + 1;
  const int zw = std::min(8, 2 * ((nb + 31) / 32));  // band padded to 16 ZW >= nb
  const int ew = Mg <= 64 ? 4 : 8;                    // grid padded to 16 EW >= Mg
  if (16 * zw < nb || 16 * ew < Mg) return CC_ERR_NOTSUPP;
  SArgs a{R, R_F, Mg, S, w->nh, w->units, w->maxseg, t->d.Tm32, w->FW, w->part};
  const size_t smem = simt_smem_bytes(nb, zw, ew);
  if (ew == 4) {
    if (periodic) CC_TRY((launch_ew<4, true>(a, zw, w->grid, smem, st)));
    else CC_TRY((launch_ew<4, false>(a, zw, w->grid, smem, st)));
  } else {
    if (periodic) CC_TRY((launch_ew<8, true>(a, zw, w->grid, smem, st)));
    else CC_TRY((launch_ew<8, false>(a, zw, w->grid, smem, st)));
  }
  CC_CUDA((launch_slab_finalize<kCols, kRows, false>(
      Mg, st, (const float*)w->part, (const float*)w->FB, R, R_F, S, w->nh, w->units, w->grid,
      w->maxseg, periodic, t->pref, eps, w->blk_ex, w->ticket, Ex, (const int*)nullptr,
      (int*)nullptr)));
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

}  // namespace cc
