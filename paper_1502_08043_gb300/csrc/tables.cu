// K1: quadrature nodes, weights and per-node 1D tables, built on the GPU in FP64.
//
// Sec. II, Eqs. 5-7: 1/p^2 = int_0^inf exp(-alpha p^2) d alpha, split at alpha_c.
// Eq. 11: on [alpha_c, inf) the variable t = alpha^{-1/2} maps the interval onto
// (0, alpha_c^{-1/2}]; d alpha = -2 t^{-3} dt, so a Gauss-Legendre point (t, w_t) becomes
// the node alpha = 1/t^2 with weight 2 w_t / t^3 (the printed Eq. 13 weight is garbled).
// Eq. 12 and the Table I discussion: Gauss-Legendre on [0, alpha_c], optionally split
// geometrically at alpha_c rho^-k (the paper's Mesh 2: rho = 5).  Eq. 14: one node sum over
// both intervals.
// Sec. III: for planewaves the per-axis tables depend on one index difference only.
//
// Gauss-Legendre points: Newton iteration on the three-term Legendre recurrence
// (Bonnet), started from the asymptotic guess cos(pi (j + 3/4) / (n + 1/2)) for the
// j-th largest root; weight 2 / ((1 - x^2) P_n'(x)^2).  Textbook method, FP64.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "internal.cuh"

namespace cc {

static constexpr double kPi = 3.14159265358979323846;

static thread_local std::string g_last_error;

void set_last_error(const char* what, cudaError_t e) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                 ")";
}

// ---------------------------------------------------------------- device: nodes
__host__ __device__ void gl_node(int n, int i, double* x, double* w) {
  // i-th node in ascending order on [-1, 1]
  const int j = n - 1 - i;
  double z = cos(kPi * (j + 0.75) / (n + 0.5));
  double p1 = 1.0, p2 = 0.0, dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    p1 = 1.0;
    p2 = 0.0;
    for (int k = 1; k <= n; ++k) {
      const double p3 = p2;
      p2 = p1;
      p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
    }
    dp = n * (z * p1 - p2) / (z * z - 1.0);
    const double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) <= 4e-16) break;
  }
  // derivative at the converged root
  p1 = 1.0;
  p2 = 0.0;
  for (int k = 1; k <= n; ++k) {
    const double p3 = p2;
    p2 = p1;
    p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
  }
  dp = n * (z * p1 - p2) / (z * z - 1.0);
  *x = z;
  *w = 2.0 / ((1.0 - z * z) * dp * dp);
}

struct NodeSpec {
  int n, i, tail;
  double lo, hi;
};

__global__ void k_mesh_nodes(const NodeSpec* spec, int S, int periodic, double keep_thresh,
                             double* alpha, double* w, int* keep) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const NodeSpec sp = spec[s];
  double x, wx;
  gl_node(sp.n, sp.i, &x, &wx);
  const double half = 0.5 * (sp.hi - sp.lo);
  double a = half * x + 0.5 * (sp.hi + sp.lo);
  double ww = half * wx;
  if (sp.tail) {  // a here is t; alpha = 1/t^2, weight 2 w_t / t^3
    const double t = a;
    a = 1.0 / (t * t);
    ww = 2.0 * ww / (t * t * t);
  }
  alpha[s] = a;
  w[s] = ww;
  keep[s] = periodic ? (ww * exp(-a) >= keep_thresh ? 1 : 0) : 1;
}

__global__ void k_gl_rule(int n, double* x, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  gl_node(n, i, &x[i], &w[i]);
}

// ---------------------------------------------------------------- device: tables
__global__ void k_periodic_table(const double* a, int S, int Dmax, double* T) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * (Dmax + 1)) return;
  const int s = idx / (Dmax + 1), D = idx % (Dmax + 1);
  T[idx] = exp(-a[s] * (double)D * (double)D);
}

// A(alpha, Delta) = 2/L^2 int_0^L (L - u) cos(2 pi Delta u / L) sqrt(pi/alpha)
//                   exp(-u^2 / (4 alpha)) du on [0, min(L, 14 sqrt(alpha))].
// One block per (node, Delta); fixed-order tree reduction.
__global__ void k_box_table(const double* a, int Dmax, double L, const double* glx,
                            const double* glw, int ngl, double* T) {
  const int s = blockIdx.x / (Dmax + 1), D = blockIdx.x % (Dmax + 1);
  const double al = a[s];
  const double ub = fmin(L, 14.0 * sqrt(al));
  const double h = 0.5 * ub;
  const double g0 = sqrt(kPi / al);
  double acc = 0.0;
  for (int i = threadIdx.x; i < ngl; i += blockDim.x) {
    const double u = h * glx[i] + h;
    acc += glw[i] * (L - u) * cos(2.0 * kPi * D * u / L) * g0 * exp(-u * u / (4.0 * al));
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) T[s * (Dmax + 1) + D] = 2.0 / (L * L) * h * red[0];
}

// Sine integrals of the general box tables, Sn(alpha, D) = int_0^L sqrt(pi/alpha)
// exp(-u^2 / (4 alpha)) sin(2 pi D u / L) du on [0, min(L, 14 sqrt(alpha))], D = 0..2R.
// One block per (node, D); fixed-order tree reduction.
__global__ void k_box_sin_table(const double* a, int Dmax, double L, const double* glx,
                                const double* glw, int ngl, double* Sn) {
  const int s = blockIdx.x / (Dmax + 1), D = blockIdx.x % (Dmax + 1);
  const double al = a[s];
  const double ub = fmin(L, 14.0 * sqrt(al));
  const double h = 0.5 * ub;
  const double g0 = sqrt(kPi / al);
  double acc = 0.0;
  for (int i = threadIdx.x; i < ngl; i += blockDim.x) {
    const double u = h * glx[i] + h;
    acc += glw[i] * sin(2.0 * kPi * D * u / L) * g0 * exp(-u * u / (4.0 * al));
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) Sn[s * (Dmax + 1) + D] = h * red[0];
}

// General per-axis box tables (Sec. II Eq. 8 for a pair difference D1 = J_x - I_x at r and
// D2 = L_x - K_x at r'):  A(alpha, D1, D2) = 1/L^2 int int g(x - x') e^{2 pi i (D1 x + D2 x')/L}.
// With u = x - x' the x integral is elementary because D1 + D2 is an integer:
//   D1 + D2 = 0:  the conserving table A(alpha, |D1|) (T64),
//   otherwise:    -(Sn(D1) + Sn(D2)) / (pi (D1 + D2) L),   Sn odd in D.
// A is unchanged by swapping D1, D2 and by negating both, so one entry per canonical code
// c = d1^2 + d1 + d2 with d1 >= |d2| (d1 = floor(sqrt(c))).  One thread per (node, code).
__global__ void k_general_tables(const double* T64, const double* Sn, const double* w, int S_eff,
                                 int S_pad, int Dmax, int Gc, double L, double pref,
                                 double* G64, double* sepG64, float* sepG32) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Gc * S_pad) return;
  const int c = (int)(idx / S_pad), s = (int)(idx % S_pad);
  double v = 0.0;
  if (s < S_eff) {
    int d1 = (int)sqrt((double)c);
    while (d1 * d1 > c) --d1;
    while ((d1 + 1) * (d1 + 1) <= c) ++d1;
    const int d2 = c - d1 * d1 - d1;
    const double* sn = Sn + (long long)s * (Dmax + 1);
    auto sodd = [&](int d) { return d >= 0 ? sn[d] : -sn[-d]; };
    const int sig = d1 + d2;
    const double g = sig == 0 ? T64[(long long)s * (Dmax + 1) + d1]
                              : -(sodd(d1) + sodd(d2)) / (kPi * (double)sig * L);
    G64[(long long)s * Gc + c] = g;
    v = cbrt(pref * w[s]) * g;
  }
  sepG64[idx] = v;
  sepG32[idx] = (float)v;
}

// separable lookup tables [Delta][S_pad] with cbrt(pref w_s) folded into every axis
__global__ void k_sep_tables(const double* T, const double* w, int S_eff, int S_pad, int Dmax,
                             double pref, double* sep64, float* sep32) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (Dmax + 1) * S_pad) return;
  const int D = idx / S_pad, s = idx % S_pad;
  double v = 0.0;
  if (s < S_eff) v = cbrt(pref * w[s]) * T[s * (Dmax + 1) + D];
  sep64[idx] = v;
  sep32[idx] = (float)v;
}

// collapsed periodic table: V_m = pref sum_s w_s exp(-a_s m), V_0 = 0 (excluded term)
__global__ void k_collapsed(const double* a, const double* w, int S_eff, int m_max, double pref,
                            double* Vm64, float* Vm32) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > m_max) return;
  double acc = 0.0;
  if (m > 0)
    for (int s = 0; s < S_eff; ++s) acc += w[s] * exp(-a[s] * (double)m);
  Vm64[m] = pref * acc;
  Vm32[m] = (float)(pref * acc);
}

// dense Toeplitz matrices for the mode products
__global__ void k_toeplitz(const double* T, const double* w, int S_eff, int Dmax, int Mg,
                           int periodic, double* Tm64, double* WDm64, float* Tm32, float* WDm32) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long tot = (long)S_eff * Mg * Mg;
  if (idx >= tot) return;
  const int s = (int)(idx / ((long)Mg * Mg));
  const int ab = (int)(idx % ((long)Mg * Mg));
  const int a = ab / Mg, b = ab % Mg;
  const int D = a > b ? a - b : b - a;
  const double t = T[s * (Dmax + 1) + D];
  const double d = (periodic && D == 0) ? 0.0 : t;
  Tm64[idx] = t;
  WDm64[idx] = w[s] * d;
  Tm32[idx] = (float)t;
  WDm32[idx] = (float)(w[s] * d);
}

__global__ void k_dbar(const double* WDm64, int S_eff, int Mg, double* D64, float* D32) {
  const int ab = blockIdx.x * blockDim.x + threadIdx.x;
  if (ab >= Mg * Mg) return;
  double acc = 0.0;
  for (int s = 0; s < S_eff; ++s) acc += WDm64[(long)s * Mg * Mg + ab];
  D64[ab] = acc;
  D32[ab] = (float)acc;
}

// Window sums F_s[a][h] = sum_{k = R - h}^{R + h} X_s[a][k], h = 0..R, in FP64, for
// X_s = D_s (periodic: T_s without its diagonal) or T_s (box), and for Dbar (the row
// after the last node).  A line of the Fermi-sphere occupation O along one axis is 1 on
// [R - h, R + h], so these are the entries of the mode products O x_k X_s of the Sec. III
// exchange; they depend on the table only, not on the Fermi radius (h <= R_F <= R).
__global__ void k_windows(const double* Tm64, const double* Dbar64, int S_eff, int Mg, int R,
                          int periodic, double* FW64, float* FW32, double* FDb64,
                          float* FDb32) {
  const int nh = R + 1;
  const long long n = (long long)(S_eff + 1) * Mg * nh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int h = (int)(i % nh);
    const long long r = i / nh;
    const int a = (int)(r % Mg), s = (int)(r / Mg);
    const bool bar = s == S_eff;
    const double* X = bar ? Dbar64 + (long long)a * Mg : Tm64 + ((long long)s * Mg + a) * Mg;
    double acc = 0.0;
    for (int k = R - h; k <= R + h; ++k)
      if (bar || !periodic || k != a) acc += X[k];
    if (bar) {
      FDb64[a * nh + h] = acc;
      FDb32[a * nh + h] = (float)acc;
    } else {
      FW64[i] = acc;
      FW32[i] = (float)acc;
    }
  }
}

// ---------------------------------------------------------------- host helpers
// Host copy of the node set of a mesh (same construction as k_mesh_nodes).
static void host_mesh(int S, int n_sub, int q_tail, double alpha_c, double ratio,
                      std::vector<double>& a, std::vector<double>& w);

// max_m |sum_s w_s exp(-a_s m) - 1/m| m over m_k = 1 + floor((12R^2 - 1) k^3 / 95^3),
// k = 0..95: the relative error of the node sum of 1/m (periodic kernel, index units)
static double mesh_error(int S, int n_sub, int q_tail, int R, double alpha_c = 1.0,
                         double ratio = 5.0) {
  std::vector<double> a, w;
  host_mesh(S, n_sub, q_tail, alpha_c, ratio, a, w);
  const long long top = 12LL * R * R - 1;
  long long prev = -1;
  double worst = 0.0;
  for (long long k = 0; k < 96; ++k) {
    const long long m = 1 + (top * k * k * k) / 857375LL;
    if (m == prev) continue;
    prev = m;
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += w[s] * exp(-a[s] * (double)m);
    const double e = fabs(v - 1.0 / (double)m) * (double)m;
    if (e > worst) worst = e;
  }
  return worst;
}

// Default mesh of the periodic kernel: explicit choices for (S, R) = (32, 4), (64, 13),
// (96, 31), (128, 63); otherwise the pair (n_sub, q_tail) with the smallest mesh_error
// among n_sub in {r, r + 1}, r = max(1, floor(log5(12 R^2)) - 1), and q_tail in
// 3 .. max(3, round(0.45 S)) with S - q_tail >= n_sub + 1 (errors floored at 1e-10,
// where FP64 rounding noise starts to decide), visited n_sub then q_tail
// ascending, replacing the best only when smaller by more than 0.1 % relative.  Fewer
// than 5 nodes: one interval and a tail of S / 2.  (A value given explicitly is kept.)
void default_mesh(int S, int R, int* n_sub, int* q_tail) {
  struct E { int S, R, n, q; };
  static const E tab[] = {{32, 4, 2, 10}, {64, 13, 3, 21}, {96, 31, 4, 29}, {128, 63, 5, 34}};
  if (*n_sub >= 0 && *q_tail >= 0) return;
  for (const E& e : tab)
    if (e.S == S && e.R == R) {
      if (*n_sub < 0) *n_sub = e.n;
      if (*q_tail < 0) *q_tail = e.q;
      return;
    }
  int r = (int)floor(log(12.0 * R * R) / log(5.0)) - 1;
  if (r < 1) r = 1;
  double best = -1.0;
  int bn = -1, bq = -1;
  const int qmax = std::max(3, (int)lrint(0.45 * S));
  for (int n = r; n <= r + 1; ++n) {
    if (*n_sub >= 0 && n != *n_sub) continue;
    for (int q = 3; q <= qmax; ++q) {
      if (*q_tail >= 0 && q != *q_tail) continue;
      if (S - q < n + 1) continue;
      const double e = std::max(mesh_error(S, n, q, R), 1e-10);  // below: rounding noise
      if (best < 0 || e < best * (1.0 - 1e-3)) {
        best = e;
        bn = n;
        bq = q;
      }
    }
  }
  if (bn < 0) {
    bn = 0;
    bq = std::max(1, S / 2);
  }
  if (*n_sub < 0) *n_sub = bn;
  if (*q_tail < 0) *q_tail = bq;
}

cc_status resolve_params(const cc_table_params* in, cc_table_params* out) {
  if (!in || !out) return CC_ERR_ARG;
  cc_table_params p = *in;
  if (p.kernel != CC_KERNEL_PERIODIC && p.kernel != CC_KERNEL_BOX) return CC_ERR_ARG;
  if (p.R < 1 || p.R > kMaxR) return CC_ERR_RANGE;
  if (!(p.L > 0.0) || !isfinite(p.L)) return CC_ERR_ARG;
  if (p.S < 2 || p.S > kMaxS) return CC_ERR_RANGE;
  default_mesh(p.S, p.R, &p.n_sub, &p.q_tail);
  if (p.n_sub > 30) return CC_ERR_RANGE;
  if (p.q_tail < 0 || p.q_tail >= p.S) return CC_ERR_ARG;
  if (!(p.alpha_c > 0.0)) p.alpha_c = 1.0;
  if (!(p.ratio > 1.0)) p.ratio = 5.0;
  if (!std::isfinite(p.alpha_c) || !std::isfinite(p.ratio)) return CC_ERR_ARG;
  if (p.prune_tol < 0.0) p.prune_tol = 1e-9;
  if (p.kernel == CC_KERNEL_BOX) p.prune_tol = 0.0;
  if (p.S - p.q_tail < p.n_sub + 1) return CC_ERR_ARG;  // every sub-interval gets a point
  *out = p;
  return CC_OK;
}

std::vector<int8_t> make_basis(int R) {
  std::vector<int8_t> v;
  for (int x = -R; x <= R; ++x)
    for (int y = -R; y <= R; ++y)
      for (int z = -R; z <= R; ++z)
        if (x * x + y * y + z * z <= R * R) {
          v.push_back((int8_t)x);
          v.push_back((int8_t)y);
          v.push_back((int8_t)z);
          v.push_back(0);
        }
  return v;
}

std::vector<uint32_t> make_id_hint(int R) {
  struct Line { int x, y, zm; };
  std::vector<Line> lines;
  for (int x = -R; x <= R; ++x)
    for (int y = -R; y <= R; ++y) {
      const int r2 = R * R - x * x - y * y;
      if (r2 < 0) continue;
      int zm = 0;
      while ((zm + 1) * (zm + 1) <= r2) ++zm;
      lines.push_back({x, y, zm});
    }
  std::vector<uint32_t> h;
  long long id = 0;  // first id of the current line
  for (size_t l = 0; l < lines.size(); ++l) {
    const Line& L = lines[l];
    const long long len = 2 * L.zm + 1;
    const uint32_t zm1 = l + 1 < lines.size() && lines[l + 1].x == L.x ? lines[l + 1].zm : 63;
    // every bucket whose first id falls on this line
    const long long B = 1LL << kIdHintShift;
    for (long long b = (id + B - 1) >> kIdHintShift; (b << kIdHintShift) < id + len; ++b) {
      const int z = (int)((b << kIdHintShift) - id) - L.zm;
      const int rest = L.zm - z < 31 ? L.zm - z : 31;
      h.push_back((uint32_t)(L.x + R) | (uint32_t)(L.y + R) << 7 | (uint32_t)(z + R) << 14 |
                  (uint32_t)rest << 21 | zm1 << 26);
    }
    id += len;
  }
  return h;
}

static std::vector<NodeSpec> node_specs(const cc_table_params& p) {
  std::vector<NodeSpec> out;
  std::vector<double> edges;
  edges.push_back(0.0);
  for (int k = p.n_sub; k >= 1; --k) edges.push_back(p.alpha_c * pow(p.ratio, -k));
  edges.push_back(p.alpha_c);
  const int n1 = p.S - p.q_tail, ns = p.n_sub + 1;
  for (int i = 0; i < ns; ++i) {
    const int q = n1 / ns + (i < n1 % ns ? 1 : 0);
    for (int j = 0; j < q; ++j) out.push_back({q, j, 0, edges[i], edges[i + 1]});
  }
  for (int j = 0; j < p.q_tail; ++j) out.push_back({p.q_tail, j, 1, 0.0, 1.0 / sqrt(p.alpha_c)});
  return out;
}

static void host_mesh(int S, int n_sub, int q_tail, double alpha_c, double ratio,
                      std::vector<double>& a, std::vector<double>& w) {
  cc_table_params p{};
  p.S = S;
  p.n_sub = n_sub;
  p.q_tail = q_tail;
  p.alpha_c = alpha_c;
  p.ratio = ratio;
  std::vector<NodeSpec> spec = node_specs(p);
  a.resize(spec.size());
  w.resize(spec.size());
  for (size_t s = 0; s < spec.size(); ++s) {
    double x, wx;
    gl_node(spec[s].n, spec[s].i, &x, &wx);
    const double half = 0.5 * (spec[s].hi - spec[s].lo);
    double al = half * x + 0.5 * (spec[s].hi + spec[s].lo);
    double ww = half * wx;
    if (spec[s].tail) {
      const double t = al;
      al = 1.0 / (t * t);
      ww = 2.0 * ww / (t * t * t);
    }
    a[s] = al;
    w[s] = ww;
  }
}

template <typename T>
static cc_status dmalloc(cc_tables t, T** ptr, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    set_last_error("cudaMalloc", e);
    return CC_ERR_ALLOC;
  }
  t->device_bytes += count * sizeof(T);
  return CC_OK;
}

static void free_tables(cc_tables t) {
  DevTables& d = t->d;
  void* ptrs[] = {d.T64, d.w64, d.a64, d.sep64, d.sep32, d.Vm64, d.Vm32, d.basis, d.idhint,
                  d.Tm64, d.WDm64, d.Dbar64, d.Tm32, d.WDm32, d.Dbar32,
                  d.FW64, d.FW32, d.FDb64, d.FDb32, d.G64, d.sepG64, d.sepG32};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  d = DevTables();
}

// General box tables (any quadruple, Sec. II Eq. 8): the sine integrals of every kept node
// with the library's Gauss-Legendre rule, then one entry per (canonical code, node).
static cc_status build_general(cc_tables t, cudaStream_t st) {
  const int S_eff = t->S_eff, Dmax = t->Dmax;
  DevTables& d = t->d;
  t->Gc = (2 * t->p.R + 1) * (2 * t->p.R + 1);
  CC_TRY(dmalloc(t, &d.G64, (size_t)S_eff * t->Gc));
  CC_TRY(dmalloc(t, &d.sepG64, (size_t)t->Gc * t->S_pad));
  CC_TRY(dmalloc(t, &d.sepG32, (size_t)t->Gc * t->S_pad));
  double *gx = nullptr, *gw = nullptr, *sn = nullptr;
  if (cudaMalloc((void**)&gx, sizeof(double) * kBoxGLPoints) != cudaSuccess ||
      cudaMalloc((void**)&gw, sizeof(double) * kBoxGLPoints) != cudaSuccess ||
      cudaMalloc((void**)&sn, sizeof(double) * S_eff * (Dmax + 1)) != cudaSuccess) {
    cudaFree(gx);
    cudaFree(gw);
    return CC_ERR_ALLOC;
  }
  k_gl_rule<<<(kBoxGLPoints + 127) / 128, 128, 0, st>>>(kBoxGLPoints, gx, gw);
  k_box_sin_table<<<S_eff * (Dmax + 1), 256, 0, st>>>(d.a64, Dmax, t->p.L, gx, gw, kBoxGLPoints,
                                                      sn);
  const long long n = (long long)t->Gc * t->S_pad;
  k_general_tables<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      d.T64, sn, d.w64, S_eff, t->S_pad, Dmax, t->Gc, t->p.L, t->pref, d.G64, d.sepG64,
      d.sepG32);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(gx);
  cudaFree(gw);
  cudaFree(sn);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error("general box tables", e);
    return CC_ERR_CUDA;
  }
  t->general_table_bytes = sizeof(float) * (size_t)t->Gc * t->S_pad;
  return CC_OK;
}

// Everything downstream of the FP64 tables T64 (shared by build and load).
static cc_status build_derived(cc_tables t, cudaStream_t st) {
  const int S_eff = t->S_eff, Dmax = t->Dmax, Mg = t->Mg;
  DevTables& d = t->d;
  CC_TRY(dmalloc(t, &d.sep64, (size_t)(Dmax + 1) * t->S_pad));
  CC_TRY(dmalloc(t, &d.sep32, (size_t)(Dmax + 1) * t->S_pad));
  CC_TRY(dmalloc(t, &d.Vm64, (size_t)t->m_max + 1));
  CC_TRY(dmalloc(t, &d.Vm32, (size_t)t->m_max + 1));
  const size_t mm = (size_t)S_eff * Mg * Mg;
  CC_TRY(dmalloc(t, &d.Tm64, mm));
  CC_TRY(dmalloc(t, &d.WDm64, mm));
  CC_TRY(dmalloc(t, &d.Tm32, mm));
  CC_TRY(dmalloc(t, &d.WDm32, mm));
  CC_TRY(dmalloc(t, &d.Dbar64, (size_t)Mg * Mg));
  CC_TRY(dmalloc(t, &d.Dbar32, (size_t)Mg * Mg));
  const int n1 = (Dmax + 1) * t->S_pad;
  k_sep_tables<<<(n1 + 255) / 256, 256, 0, st>>>(d.T64, d.w64, S_eff, t->S_pad, Dmax, t->pref,
                                                  d.sep64, d.sep32);
  const int periodic = t->p.kernel == CC_KERNEL_PERIODIC;
  if (periodic)
    k_collapsed<<<(t->m_max + 1 + 255) / 256, 256, 0, st>>>(d.a64, d.w64, S_eff, t->m_max,
                                                             t->pref, d.Vm64, d.Vm32);
  else {
    CC_CUDA(cudaMemsetAsync(d.Vm64, 0, sizeof(double) * (t->m_max + 1), st));
    CC_CUDA(cudaMemsetAsync(d.Vm32, 0, sizeof(float) * (t->m_max + 1), st));
  }
  k_toeplitz<<<(unsigned)((mm + 255) / 256), 256, 0, st>>>(d.T64, d.w64, S_eff, Dmax, Mg, periodic,
                                                           d.Tm64, d.WDm64, d.Tm32, d.WDm32);
  k_dbar<<<(Mg * Mg + 255) / 256, 256, 0, st>>>(d.WDm64, S_eff, Mg, d.Dbar64, d.Dbar32);
  if (Mg <= kFusedMaxMg) {
    const size_t nh = (size_t)t->p.R + 1;
    CC_TRY(dmalloc(t, &d.FW64, (size_t)S_eff * Mg * nh));
    CC_TRY(dmalloc(t, &d.FW32, (size_t)S_eff * Mg * nh));
    CC_TRY(dmalloc(t, &d.FDb64, (size_t)Mg * nh));
    CC_TRY(dmalloc(t, &d.FDb32, (size_t)Mg * nh));
    const long long n = (long long)(S_eff + 1) * Mg * nh;
    k_windows<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(
        d.Tm64, d.Dbar64, S_eff, Mg, t->p.R, periodic, d.FW64, d.FW32, d.FDb64, d.FDb32);
  }
  CC_CUDA(cudaGetLastError());
  std::vector<int8_t> b = make_basis(t->p.R);
  CC_TRY(dmalloc(t, &d.basis, b.size()));
  CC_CUDA(cudaMemcpyAsync(d.basis, b.data(), b.size(), cudaMemcpyHostToDevice, st));
  const std::vector<uint32_t> hint = make_id_hint(t->p.R);
  CC_TRY(dmalloc(t, &d.idhint, hint.size()));
  CC_CUDA(cudaMemcpyAsync(d.idhint, hint.data(), sizeof(uint32_t) * hint.size(),
                          cudaMemcpyHostToDevice, st));
  t->table_bytes = sizeof(float) * ((size_t)(Dmax + 1) * t->S_pad + t->m_max + 1);
  if (!periodic) CC_TRY(build_general(t, st));
  return CC_OK;
}

static void init_sizes(cc_tables t) {
  const int R = t->p.R;
  t->Mg = 2 * R + 1;
  t->Dmax = 2 * R;
  t->m_max = 4 * R * R;
  t->Nb = (int)(make_basis(R).size() / 4);
  t->pref = t->p.kernel == CC_KERNEL_PERIODIC ? 1.0 / (kPi * t->p.L) : 1.0 / (2.0 * kPi * kPi);
}

static cc_status finish_kept(cc_tables t) {
  t->kept_idx.clear();
  for (int s = 0; s < t->S; ++s)
    if (t->kept[s]) t->kept_idx.push_back(s);
  t->S_eff = (int)t->kept_idx.size();
  if (t->S_eff == 0) return CC_ERR_ARG;
  t->S_pad = (t->S_eff + 31) / 32 * 32;
  return CC_OK;
}

static cc_status build_impl(const cc_table_params* params, cudaStream_t st, cc_tables t,
                            bool workspaces) {
  CC_TRY(resolve_params(params, &t->p));
  CC_CUDA(cudaGetDevice(&t->device));
  const cc_table_params& p = t->p;
  t->S = p.S;
  init_sizes(t);
  // 1. nodes and weights (FP64, device)
  std::vector<NodeSpec> spec = node_specs(p);
  NodeSpec* dspec = nullptr;
  double *da = nullptr, *dw = nullptr;
  int* dk = nullptr;
  cc_status s = CC_OK;
  const double thresh = p.prune_tol > 0 ? p.prune_tol / (12.0 * p.R * p.R) : -1.0;
  if (cudaMalloc((void**)&dspec, sizeof(NodeSpec) * p.S) != cudaSuccess ||
      cudaMalloc((void**)&da, sizeof(double) * p.S) != cudaSuccess ||
      cudaMalloc((void**)&dw, sizeof(double) * p.S) != cudaSuccess ||
      cudaMalloc((void**)&dk, sizeof(int) * p.S) != cudaSuccess) {
    s = CC_ERR_ALLOC;
  }
  t->alpha.assign(p.S, 0.0);
  t->w.assign(p.S, 0.0);
  t->kept.assign(p.S, 0);
  t->part.assign(p.S, 0);
  for (int i = 0; i < p.S; ++i) t->part[i] = spec[i].tail;
  if (s == CC_OK) {
    cudaMemcpyAsync(dspec, spec.data(), sizeof(NodeSpec) * p.S, cudaMemcpyHostToDevice, st);
    k_mesh_nodes<<<(p.S + 127) / 128, 128, 0, st>>>(dspec, p.S, p.kernel == CC_KERNEL_PERIODIC,
                                                   thresh, da, dw, dk);
    cudaMemcpyAsync(t->alpha.data(), da, sizeof(double) * p.S, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(t->w.data(), dw, sizeof(double) * p.S, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(t->kept.data(), dk, sizeof(int) * p.S, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_last_error("node kernel", e);
      s = CC_ERR_CUDA;
    }
  }
  cudaFree(dspec);
  cudaFree(da);
  cudaFree(dw);
  cudaFree(dk);
  CC_TRY(s);
  CC_TRY(finish_kept(t));
  // 2. per-node tables of the kept nodes
  const int S_eff = t->S_eff, Dmax = t->Dmax;
  std::vector<double> ka(S_eff), kw(S_eff);
  for (int i = 0; i < S_eff; ++i) {
    ka[i] = t->alpha[t->kept_idx[i]];
    kw[i] = t->w[t->kept_idx[i]];
  }
  DevTables& d = t->d;
  CC_TRY(dmalloc(t, &d.a64, S_eff));
  CC_TRY(dmalloc(t, &d.w64, S_eff));
  CC_TRY(dmalloc(t, &d.T64, (size_t)S_eff * (Dmax + 1)));
  CC_CUDA(cudaMemcpyAsync(d.a64, ka.data(), sizeof(double) * S_eff, cudaMemcpyHostToDevice, st));
  CC_CUDA(cudaMemcpyAsync(d.w64, kw.data(), sizeof(double) * S_eff, cudaMemcpyHostToDevice, st));
  if (p.kernel == CC_KERNEL_PERIODIC) {
    const int n = S_eff * (Dmax + 1);
    k_periodic_table<<<(n + 255) / 256, 256, 0, st>>>(d.a64, S_eff, Dmax, d.T64);
  } else {
    double *gx = nullptr, *gw = nullptr;
    if (cudaMalloc((void**)&gx, sizeof(double) * kBoxGLPoints) != cudaSuccess ||
        cudaMalloc((void**)&gw, sizeof(double) * kBoxGLPoints) != cudaSuccess) {
      cudaFree(gx);
      return CC_ERR_ALLOC;
    }
    k_gl_rule<<<(kBoxGLPoints + 127) / 128, 128, 0, st>>>(kBoxGLPoints, gx, gw);
    k_box_table<<<S_eff * (Dmax + 1), 256, 0, st>>>(d.a64, Dmax, p.L, gx, gw, kBoxGLPoints, d.T64);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(gx);
    cudaFree(gw);
    if (e != cudaSuccess) {
      set_last_error("box table kernel", e);
      return CC_ERR_CUDA;
    }
  }
  CC_CUDA(cudaGetLastError());
  CC_TRY(build_derived(t, st));
  CC_CUDA(cudaStreamSynchronize(st));
  if (workspaces) {
    CC_TRY(workspace_alloc(t));
    if (t->Mg <= 128) CC_TRY(mixed_workspace_alloc(t));
    CC_TRY(fused_single_alloc(t));
    noalloc_preload(t);
    CC_TRY(simt_slab_alloc(t, &t->simt));
  }
  return CC_OK;
}

cc_status build_tables_internal(const cc_table_params* params, cudaStream_t st, bool workspaces,
                                cc_tables* out) {
  *out = nullptr;
  cc_tables t = new (std::nothrow) cc_tables_s();
  if (!t) return CC_ERR_ALLOC;
  cc_status s = build_impl(params, st, t, workspaces);
  if (s != CC_OK) {
    cc_tables_free(t);
    return s;
  }
  *out = t;
  return CC_OK;
}

// ---------------------------------------------------------------- checkpoint format
// little-endian: "CCTB" u32 version | params | S, S_eff | alpha[S] w[S] part[S] kept[S] |
// T64[S_eff][Dmax+1] | u64 FNV-1a of everything before it
static const uint32_t kMagic = 0x42544343u;  // "CCTB"
static const uint32_t kVersion = 2;  // 2: parameters carry the sub-interval ratio

static uint64_t fnv1a(const std::vector<uint8_t>& b) {
  uint64_t h = 1469598103934665603ull;
  for (uint8_t c : b) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

template <typename T>
static void put(std::vector<uint8_t>& b, const T* v, size_t n) {
  const uint8_t* p = reinterpret_cast<const uint8_t*>(v);
  b.insert(b.end(), p, p + sizeof(T) * n);
}

template <typename T>
static bool get(const std::vector<uint8_t>& b, size_t& off, T* v, size_t n) {
  if (off + sizeof(T) * n > b.size()) return false;
  memcpy(v, b.data() + off, sizeof(T) * n);
  off += sizeof(T) * n;
  return true;
}

}  // namespace cc

using namespace cc;

extern "C" {

const char* cc_status_string(cc_status s) {
  switch (s) {
    case CC_OK: return "ok";
    case CC_ERR_ARG: return "invalid argument";
    case CC_ERR_RANGE: return "size beyond limit";
    case CC_ERR_CUDA: return "CUDA error";
    case CC_ERR_ALLOC: return "allocation failed";
    case CC_ERR_TIMEOUT: return "device wait timed out";
    case CC_ERR_NOTSUPP: return "not supported";
    case CC_ERR_IO: return "I/O or format error";
  }
  return "unknown status";
}

const char* cc_last_error(void) { return g_last_error.c_str(); }

cc_status cc_default_mesh(int S, int R, int* n_sub, int* q_tail) {
  if (!n_sub || !q_tail) return CC_ERR_ARG;
  if (R < 1 || R > kMaxR || S < 2 || S > kMaxS) return CC_ERR_RANGE;
  *n_sub = -1;
  *q_tail = -1;
  default_mesh(S, R, n_sub, q_tail);
  return CC_OK;
}

// Smallest node count S in 2 .. S_max whose default mesh (default_mesh above, the
// tabulated workloads included) has mesh_error <= target: the inverse of the default rule,
// fewest nodes for a stated method error (Sec. II: the node count follows from the
// accuracy wanted over the range of |q|^2 the cutoff allows).
cc_status cc_mesh_for_error(int R, double target, int S_max, int* S, int* n_sub, int* q_tail,
                            double* err) {
  if (!S || !n_sub || !q_tail || !(target > 0.0) || !std::isfinite(target)) return CC_ERR_ARG;
  if (R < 1 || R > kMaxR || S_max < 2 || S_max > kMaxS) return CC_ERR_RANGE;
  for (int s = 2; s <= S_max; ++s) {
    int n = -1, q = -1;
    default_mesh(s, R, &n, &q);
    const double e = mesh_error(s, n, q, R);
    if (e <= target) {
      *S = s;
      *n_sub = n;
      *q_tail = q;
      if (err) *err = e;
      return CC_OK;
    }
  }
  return CC_ERR_RANGE;
}

// Mesh tuning for a stated periodic-kernel error (Sec. II: the split point alpha_c and the
// sub-intervals decide how many nodes the accuracy needs).  Candidates: sub-interval ratio
// rho in {3, 4, 5, 6, 8}, alpha_c in {0.5, 1, 2} (index units), n_sub = max(1,
// floor(log_rho(12 R^2)) - 1) (from the smallest split edge alpha_c rho^-n_sub near
// 1 / (12 R^2)) and the next one, q_tail in 3 .. max(3, round(0.45 S)) with
// S - q_tail >= n_sub + 1; node counts S from max(2, floor(0.8 S_d)) up to S_d, where S_d is
// cc_mesh_for_error's count for the same target (which the default rho = 5, alpha_c = 1
// mesh reaches).  The first S whose best candidate reaches the target wins; within an S the
// smallest error wins (errors floored at 1e-10, a candidate replaces the best only when
// smaller by more than 0.1 %, visiting rho, alpha_c, n_sub, q_tail ascending).
static const double kTuneRatios[] = {3.0, 4.0, 5.0, 6.0, 8.0};
static const double kTuneAlphas[] = {0.5, 1.0, 2.0};

static bool mesh_tune(int R, double target, int S_max, int* S, int* n_sub, int* q_tail,
                      double* alpha_c, double* ratio, double* err) {
  int Sd = -1, nd = -1, qd = -1;
  for (int s = 2; s <= S_max; ++s) {
    int n = -1, q = -1;
    default_mesh(s, R, &n, &q);
    if (mesh_error(s, n, q, R) <= target) {
      Sd = s;
      nd = n;
      qd = q;
      break;
    }
  }
  if (Sd < 0) return false;
  const double m = 12.0 * R * R;
  for (int s = std::max(2, (int)(0.8 * Sd)); s <= Sd; ++s) {
    double best = -1.0, bestraw = 0.0;
    int bn = -1, bq = -1;
    double ba = 1.0, br = 5.0;
    for (double rho : kTuneRatios)
      for (double ac : kTuneAlphas) {
        const int r = std::max(1, (int)floor(log(m) / log(rho)) - 1);
        for (int n = r; n <= r + 1; ++n)
          for (int q = 3; q <= std::max(3, (int)lrint(0.45 * s)); ++q) {
            if (s - q < n + 1) continue;
            const double raw = mesh_error(s, n, q, R, ac, rho);
            const double e = std::max(raw, 1e-10);
            if (best < 0 || e < best * (1.0 - 1e-3)) {
              best = e;
              bestraw = raw;
              bn = n;
              bq = q;
              ba = ac;
              br = rho;
            }
          }
      }
    if (bn >= 0 && bestraw <= target) {
      *S = s;
      *n_sub = bn;
      *q_tail = bq;
      *alpha_c = ba;
      *ratio = br;
      *err = bestraw;
      return true;
    }
  }
  // S_d itself with the default mesh reaches the target
  *S = Sd;
  *n_sub = nd;
  *q_tail = qd;
  *alpha_c = 1.0;
  *ratio = 5.0;
  *err = mesh_error(Sd, nd, qd, R);
  return true;
}

cc_status cc_mesh_tune(int R, double target, int S_max, int* S, int* n_sub, int* q_tail,
                       double* alpha_c, double* ratio, double* err) {
  if (!S || !n_sub || !q_tail || !alpha_c || !ratio || !(target > 0.0) || !std::isfinite(target))
    return CC_ERR_ARG;
  if (R < 1 || R > kMaxR || S_max < 2 || S_max > kMaxS) return CC_ERR_RANGE;
  double e = 0.0;
  if (!mesh_tune(R, target, S_max, S, n_sub, q_tail, alpha_c, ratio, &e)) return CC_ERR_RANGE;
  if (err) *err = e;
  return CC_OK;
}

cc_status cc_build_tables_for_error(int kernel, int R, double L, double target, int S_max,
                                    void* stream, cc_tables* out) {
  if (!out) return CC_ERR_ARG;
  cc_table_params p{};
  p.kernel = kernel;
  p.R = R;
  p.L = L;
  p.prune_tol = -1.0;
  double e = 0.0;
  CC_TRY(cc_mesh_tune(R, target, S_max, &p.S, &p.n_sub, &p.q_tail, &p.alpha_c, &p.ratio, &e));
  return build_tables_internal(&p, as_stream(stream), true, out);
}

cc_status cc_basis(int R, int* Nb, int8_t* vec_host) {
  if (!Nb) return CC_ERR_ARG;
  if (R < 1 || R > kMaxR) return CC_ERR_RANGE;
  std::vector<int8_t> b = make_basis(R);
  *Nb = (int)(b.size() / 4);
  if (vec_host) memcpy(vec_host, b.data(), b.size());
  return CC_OK;
}

cc_status cc_build_tables(const cc_table_params* params, void* stream, cc_tables* out) {
  if (!params || !out) return CC_ERR_ARG;
  return build_tables_internal(params, as_stream(stream), true, out);
}

cc_status cc_tables_info(cc_tables t, cc_tables_info_t* info) {
  if (!t || !info) return CC_ERR_ARG;
  info->kernel = t->p.kernel;
  info->R = t->p.R;
  info->S = t->p.S;
  info->n_sub = t->p.n_sub;
  info->q_tail = t->p.q_tail;
  info->L = t->p.L;
  info->alpha_c = t->p.alpha_c;
  info->ratio = t->p.ratio;
  info->prune_tol = t->p.prune_tol;
  info->S_eff = t->S_eff;
  info->Nb = t->Nb;
  info->Mg = t->Mg;
  info->m_max = t->m_max;
  info->device_bytes = t->device_bytes;
  info->table_bytes = t->table_bytes;
  info->general_codes = t->Gc;
  info->general_table_bytes = t->general_table_bytes;
  return CC_OK;
}

cc_status cc_tables_nodes(cc_tables t, double* alpha_host, double* w_host, int* part_host,
                          int* kept_host) {
  if (!t) return CC_ERR_ARG;
  for (int s = 0; s < t->S; ++s) {
    if (alpha_host) alpha_host[s] = t->alpha[s];
    if (w_host) w_host[s] = t->w[s];
    if (part_host) part_host[s] = t->part[s];
    if (kept_host) kept_host[s] = t->kept[s];
  }
  return CC_OK;
}

cc_status cc_tables_values(cc_tables t, double* table_host) {
  if (!t || !table_host) return CC_ERR_ARG;
  CC_CUDA(cudaMemcpy(table_host, t->d.T64, sizeof(double) * t->S_eff * (t->Dmax + 1),
                     cudaMemcpyDeviceToHost));
  return CC_OK;
}

cc_status cc_tables_general_values(cc_tables t, double* table_host) {
  if (!t || !table_host) return CC_ERR_ARG;
  if (t->p.kernel != CC_KERNEL_BOX || !t->d.G64) return CC_ERR_NOTSUPP;
  CC_CUDA(cudaMemcpy(table_host, t->d.G64, sizeof(double) * t->S_eff * t->Gc,
                     cudaMemcpyDeviceToHost));
  return CC_OK;
}

cc_status cc_tables_free(cc_tables t) {
  if (!t) return CC_ERR_ARG;
  workspace_free(t);
  mixed_workspace_free(t);
  fused_single_free(t);
  simt_slab_free(t->simt);
  t->simt = nullptr;
  free_tables(t);
  delete t;
  return CC_OK;
}

cc_status cc_tables_save(cc_tables t, const char* path) {
  if (!t || !path) return CC_ERR_ARG;
  std::vector<double> T((size_t)t->S_eff * (t->Dmax + 1));
  CC_CUDA(cudaMemcpy(T.data(), t->d.T64, sizeof(double) * T.size(), cudaMemcpyDeviceToHost));
  std::vector<uint8_t> b;
  put(b, &kMagic, 1);
  put(b, &kVersion, 1);
  put(b, &t->p, 1);
  put(b, &t->S, 1);
  put(b, &t->S_eff, 1);
  put(b, t->alpha.data(), t->S);
  put(b, t->w.data(), t->S);
  put(b, t->part.data(), t->S);
  put(b, t->kept.data(), t->S);
  put(b, T.data(), T.size());
  const uint64_t h = fnv1a(b);
  put(b, &h, 1);
  FILE* f = fopen(path, "wb");
  if (!f) return CC_ERR_IO;
  const size_t wr = fwrite(b.data(), 1, b.size(), f);
  const int rc = fclose(f);
  return (wr == b.size() && rc == 0) ? CC_OK : CC_ERR_IO;
}

cc_status cc_tables_load(const char* path, void* stream, cc_tables* out) {
  if (!path || !out) return CC_ERR_ARG;
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return CC_ERR_IO;
  std::vector<uint8_t> b;
  uint8_t buf[1 << 16];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0) b.insert(b.end(), buf, buf + n);
  fclose(f);
  if (b.size() < 8 + sizeof(uint64_t)) return CC_ERR_IO;
  uint64_t h;
  memcpy(&h, b.data() + b.size() - 8, 8);
  b.resize(b.size() - 8);
  if (fnv1a(b) != h) return CC_ERR_IO;
  size_t off = 0;
  uint32_t magic, ver;
  cc_table_params p;
  int S, S_eff;
  if (!get(b, off, &magic, 1) || !get(b, off, &ver, 1) || magic != kMagic || ver != kVersion ||
      !get(b, off, &p, 1) || !get(b, off, &S, 1) || !get(b, off, &S_eff, 1))
    return CC_ERR_IO;
  cc_table_params chk;
  if (resolve_params(&p, &chk) != CC_OK || S != p.S) return CC_ERR_IO;
  cc_tables t = new (std::nothrow) cc_tables_s();
  if (!t) return CC_ERR_ALLOC;
  t->p = p;
  t->S = S;
  t->alpha.resize(S);
  t->w.resize(S);
  t->part.resize(S);
  t->kept.resize(S);
  bool ok = get(b, off, t->alpha.data(), S) && get(b, off, t->w.data(), S) &&
            get(b, off, t->part.data(), S) && get(b, off, t->kept.data(), S);
  cc_status s = ok ? CC_OK : CC_ERR_IO;
  cudaStream_t st = as_stream(stream);
  if (s == CC_OK) {
    init_sizes(t);
    s = finish_kept(t);
  }
  if (s == CC_OK && t->S_eff != S_eff) s = CC_ERR_IO;
  std::vector<double> T;
  if (s == CC_OK) {
    T.resize((size_t)S_eff * (t->Dmax + 1));
    if (!get(b, off, T.data(), T.size()) || off != b.size()) s = CC_ERR_IO;
  }
  if (s == CC_OK) {
    cudaGetDevice(&t->device);
    std::vector<double> ka(S_eff), kw(S_eff);
    for (int i = 0; i < S_eff; ++i) {
      ka[i] = t->alpha[t->kept_idx[i]];
      kw[i] = t->w[t->kept_idx[i]];
    }
    s = dmalloc(t, &t->d.a64, S_eff);
    if (s == CC_OK) s = dmalloc(t, &t->d.w64, S_eff);
    if (s == CC_OK) s = dmalloc(t, &t->d.T64, T.size());
    if (s == CC_OK) {
      if (cudaMemcpyAsync(t->d.a64, ka.data(), 8 * S_eff, cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(t->d.w64, kw.data(), 8 * S_eff, cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(t->d.T64, T.data(), 8 * T.size(), cudaMemcpyHostToDevice, st) !=
              cudaSuccess)
        s = CC_ERR_CUDA;
    }
    if (s == CC_OK) s = build_derived(t, st);
    if (s == CC_OK) s = workspace_alloc(t);
    if (s == CC_OK && cudaStreamSynchronize(st) != cudaSuccess) s = CC_ERR_CUDA;
    if (s == CC_OK && t->Mg <= 128) s = mixed_workspace_alloc(t);
    if (s == CC_OK) s = fused_single_alloc(t);
    if (s == CC_OK) noalloc_preload(t);
    if (s == CC_OK) s = simt_slab_alloc(t, &t->simt);
  }
  if (s != CC_OK) {
    cc_tables_free(t);
    return s;
  }
  *out = t;
  return CC_OK;
}

}  // extern "C"
