// Internal declarations shared by the translation units of libcoulomb.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "coulomb.h"

namespace cc {

// ---------------------------------------------------------------- error plumbing
void set_last_error(const char* what, cudaError_t e);

#define CC_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      ::cc::set_last_error(#call, e_);                 \
      return CC_ERR_CUDA;                              \
    }                                                  \
  } while (0)

#define CC_TRY(call)                  \
  do {                                \
    cc_status s_ = (call);            \
    if (s_ != CC_OK) return s_;       \
  } while (0)

// limits
constexpr int kMaxR = 127;          // Delta = 0..254 fits the 8-bit packed deltas
constexpr int kMaxS = 1024;
constexpr int kBoxGLPoints = 1200;  // Gauss-Legendre points of one box axis integral
constexpr int kFusedMaxMg = 49;     // grid side served by the fused small-grid exchange

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Device buffers owned by a table handle.  All tables are for the kept nodes only.
struct DevTables {
  double* T64 = nullptr;      // [S_eff][Dmax+1]  T_s[Delta]
  double* w64 = nullptr;      // [S_eff]
  double* a64 = nullptr;      // [S_eff]
  double* sep64 = nullptr;    // [Dmax+1][S_pad]  cbrt(pref w_s) T_s[Delta], 0 padded
  float* sep32 = nullptr;     // same, FP32
  double* Vm64 = nullptr;     // [m_max+1] collapsed pref sum_s w_s exp(-a_s m) (PERIODIC)
  float* Vm32 = nullptr;
  int8_t* basis = nullptr;    // [Nb][4]
  uint32_t* idhint = nullptr; // [ceil(Nb / 64)] decode hints of the ids (make_id_hint)
  // dense Mg x Mg Toeplitz matrices for the mode products
  double* Tm64 = nullptr;     // [S_eff][Mg][Mg]  T_s[|a-b|]
  double* WDm64 = nullptr;    // [S_eff][Mg][Mg]  w_s D_s (D = T - I periodic, T box)
  double* Dbar64 = nullptr;   // [Mg][Mg] sum_s w_s D_s (periodic)
  float* Tm32 = nullptr;
  float* WDm32 = nullptr;
  float* Dbar32 = nullptr;
  // window sums over the centred ranges [R - h, R + h], h = 0..R, of the rows of D_s
  // (periodic; T_s for the box kernel) and of Dbar: the product of a Fermi-sphere line of
  // the occupation with those matrices (grid side <= kFusedMaxMg only)
  double* FW64 = nullptr;     // [S_eff][Mg][R + 1]
  float* FW32 = nullptr;
  double* FDb64 = nullptr;    // [Mg][R + 1]
  float* FDb32 = nullptr;
  // BOX kernel, general (not necessarily momentum-conserving) integrals: the two-index
  // per-axis tables A(alpha_s, D1, D2) of Sec. II Eq. 8 over the canonical codes
  // c = d1^2 + d1 + d2 (d1 >= |d2|, see gen_code), Gc = (2R + 1)^2 codes per node
  double* G64 = nullptr;      // [S_eff][Gc]      A(alpha_s, d1, d2)
  double* sepG64 = nullptr;   // [Gc][S_pad]      cbrt(pref w_s) A(alpha_s, d1, d2), 0 padded
  float* sepG32 = nullptr;    // same, FP32
};

// Exchange workspace (allocated with the handle; a chunk of nodes at a time).
struct Workspace {
  int chunk = 0;              // nodes per chunk
  void* occ = nullptr;        // [Mg^3] occupation tensor (float or double, by call)
  void* P = nullptr;          // [chunk][Mg^3]
  void* Q = nullptr;          // [chunk][Mg^3]
  void* E = nullptr;          // [Mg^3] accumulator
  double* part = nullptr;     // [kRedBlocks] FP64 partial sums of E_x
  size_t bytes = 0;
  // mixed-precision (tensor core) workspace, see umma.cu
  void* mx = nullptr;
  size_t mx_bytes = 0;
};

constexpr int kRedBlocks = 608;

}  // namespace cc

struct cc_tables_s {
  cc_table_params p;          // resolved parameters
  int device = 0;
  int S = 0, S_eff = 0, S_pad = 0, Nb = 0, Mg = 0, Dmax = 0, m_max = 0;
  double pref = 0.0;          // 1/(pi L) periodic, 1/(2 pi^2) box
  std::vector<double> alpha, w;   // full node set (host copy)
  std::vector<int> part, kept;    // part: 0 interval 1, 1 tail; kept flags
  std::vector<int> kept_idx;      // indices of kept nodes
  cc::DevTables d;
  cc::Workspace ws;
  void* fused = nullptr;          // fused small-grid exchange plan (grid side <= 49)
  void* simt = nullptr;           // SIMT slab exchange workspace (FP32, grid side 50..127)
  size_t table_bytes = 0;
  size_t device_bytes = 0;
  int Gc = 0;                     // codes of the general box tables per node (0: periodic)
  size_t general_table_bytes = 0; // FP32 general box lookup tables
};

namespace cc {
// tables.cu
cc_status resolve_params(const cc_table_params* in, cc_table_params* out);
void default_mesh(int S, int R, int* n_sub, int* q_tail);
std::vector<int8_t> make_basis(int R);
// Decode hints for basis ids in lexicographic (n_x, n_y, n_z) order, one per bucket of 32
// ids; entry b describes id 32 b, the first id of bucket b, on its line (x, y) of
// z = -z_max .. z_max, z_max = floor(sqrt(R^2 - x^2 - y^2)):
//   bits 0-6  x + R,  bits 7-13  y + R,  bits 14-20  z + R of id 32 b,
//   bits 21-25  min(z_max - z, 31)  (ids after id 32 b that are still on its line),
//   bits 26-31  z_max of the next line when it is (x, y + 1), else 63 (also when that
//               z_max is 63, which only costs a walk)
constexpr int kIdHintShift = 5;
std::vector<uint32_t> make_id_hint(int R);
cc_status build_tables_internal(const cc_table_params* params, cudaStream_t st,
                                bool workspaces, cc_tables* out);
// batched.cu
cc_status fused_single_alloc(cc_tables t);
void noalloc_preload(cc_tables t);  // exchange.cu: the allocation-free path's module
void fused_single_free(cc_tables t);
cc_status fused_single_exchange(cc_tables t, int R_F, int precision, void* eps, double* Ex,
                                cudaStream_t st);
// exchange.cu
cc_status workspace_alloc(cc_tables t);
void workspace_free(cc_tables t);
// umma.cu
cc_status mixed_batch_create(const std::vector<cc_tables>& tabs, const std::vector<int>& R_F,
                             const std::vector<long long>& eps_off, void** out);
cc_status mixed_batch_run(void* mb, float* eps, double* Ex, cudaStream_t st);
cc_status mixed_batch_tune(void* mb, float* eps, double* Ex, int reps, int* choice, float* ms,
                           cudaStream_t st);
void mixed_batch_free(void* mb);
cc_status mixed_workspace_alloc(cc_tables t);
void mixed_workspace_free(cc_tables t);
cc_status exchange_mixed(cc_tables t, int R_F, int precision, float* eps, double* Ex,
                         cudaStream_t st);
cc_status tc_make_map_bf16(void* map, void* ptr, long long rows, int cols, int box_rows);
cc_status tc_make_map_16(void* map, void* ptr, long long rows, int cols, int box_rows, bool bf16);
// tcslab.cu (fused tensor-core exchange, bf16x3, grid side up to 127)
bool tc_slab_supported(cc_tables t);
cc_status tc_slab_alloc(cc_tables t, void** out);
void tc_slab_free(void* ws);
cc_status tc_slab_run(cc_tables t, void* ws, const void* map_hi, const void* map_lo, int* err,
                      int stall_test, int R_F, float* eps, double* Ex, cudaStream_t st,
                      bool half, int x1 = 0);
// tcsmall.cu (tensor-core exchange, bf16x3, grid side up to 64: two slabs per 128-row MMA)
bool tc_small_supported(cc_tables t);
cc_status tc_small_alloc(cc_tables t, void** out);
void tc_small_free(void* ws);
cc_status tc_small_run(cc_tables t, void* ws, int* err, int stall_test, int R_F, float* eps,
                       double* Ex, cudaStream_t st, int x1 = 0);
bool tc_small_batch_supported(const std::vector<cc_tables>& tabs, const std::vector<int>& R_F);
cc_status tc_small_batch_create(const std::vector<cc_tables>& tabs, const std::vector<int>& R_F,
                                const std::vector<long long>& eps_off, void** out);
cc_status tc_small_batch_run(void* p, int* err, float* eps, double* Ex, cudaStream_t st);
cc_status tc_small_batch_tune(void* p, int* err, float* eps, double* Ex, int reps, int* choice,
                              float* ms, cudaStream_t st);
void tc_small_batch_free(void* p);
// simtslab.cu (plain FP32 exchange by the slab algorithm, grid side 50..127)
bool simt_slab_supported(cc_tables t);
cc_status simt_slab_alloc(cc_tables t, void** out);
void simt_slab_free(void* ws);
cc_status simt_slab_run(cc_tables t, void* ws, int R_F, float* eps, double* Ex, cudaStream_t st);
}  // namespace cc
