// Device twin of coulomb_inputs.quads(): counter-based SplitMix64 quadruple generator.
// Input generation only (no arithmetic of the Coulomb method).  Bit-identical to the
// numpy version: quadruple i, attempt a, component c uses counter (i * 64 + a) * 4 + c;
// I, J, K uniform ids by multiply-high; L = id of n_I + n_K - n_J if inside the sphere.
// Mode 2 (coulomb_inputs.quads_uniform): four independent uniform ids, counter 4 i + c.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kAttempts = 64;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1) * kGamma);
}
__device__ __forceinline__ int lemire(uint64_t u, int n) {
  return (int)(((u >> 32) * (uint64_t)n) >> 32);
}

__global__ void k_quads(int R, int Nb, const char4* __restrict__ vec, const int* __restrict__ idmap,
                        uint64_t key, int64_t start, int64_t count, int planted, int4* out) {
  const int G = 2 * R + 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t i = (uint64_t)(start + t);
    if (planted == 2) {
      out[t] = make_int4(lemire(draw(key, 4 * i), Nb), lemire(draw(key, 4 * i + 1), Nb),
                         lemire(draw(key, 4 * i + 2), Nb), lemire(draw(key, 4 * i + 3), Nb));
      continue;
    }
    int4 q = make_int4(0, 0, 0, 0);
    bool done = false;
    int I0 = 0, K0 = 0;
    for (int a = 0; a < kAttempts && !done; ++a) {
      const uint64_t base = (i * kAttempts + a) * 4;
      const int I = lemire(draw(key, base), Nb);
      const int J = lemire(draw(key, base + 1), Nb);
      const int K = lemire(draw(key, base + 2), Nb);
      if (a == 0) { I0 = I; K0 = K; }
      const char4 vi = vec[I], vj = vec[J], vk = vec[K];
      const int x = vi.x + vk.x - vj.x, y = vi.y + vk.y - vj.y, z = vi.z + vk.z - vj.z;
      if (x * x + y * y + z * z <= R * R) {
        q = make_int4(I, J, K, idmap[((x + R) * G + (y + R)) * G + (z + R)]);
        done = true;
      }
    }
    if (!done) q = make_int4(I0, I0, K0, K0);
    if (planted) {
      const uint64_t b0 = i * kAttempts * 4 + 3;
      const uint64_t u = draw(key, b0) >> 32;
      if (u < (uint64_t)(0.05 * 4294967296.0)) {
        q.w = lemire(draw(key, b0 + 4), Nb);
      } else if (u < (uint64_t)(0.06 * 4294967296.0)) {
        q.y = q.x;
        q.w = q.z;
      }
    }
    out[t] = q;
  }
}
}  // namespace

extern "C" int ccgen_quads(int R, int Nb, const void* vec_dev, const void* idmap_dev,
                           unsigned long long key, long long start, long long count, int planted,
                           void* out_dev, void* stream) {
  if (count <= 0) return 0;
  if (!vec_dev || !idmap_dev || !out_dev || R < 1 || R > 127 || Nb < 1) return 1;
  k_quads<<<1216, 256, 0, (cudaStream_t)stream>>>(R, Nb, (const char4*)vec_dev,
                                                  (const int*)idmap_dev, key, start, count,
                                                  planted, (int4*)out_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
