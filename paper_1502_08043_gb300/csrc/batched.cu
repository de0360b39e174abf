// Slab-wise exchange sums (single box, grid side <= 49) and the batched engine:
// many independent boxes with uneven cutoffs, Fermi radii and quadrature orders in one
// persistent launch, captured once in a CUDA graph and replayed.
//
// Work items are (box, group of consecutive nodes); a persistent grid takes them from an
// atomic counter in order of decreasing cost (longest-processing-time first), and the
// CTA that completes the last item of a box finalises that box (see fused.cuh).  The
// granularity of the items (how many node groups each box is cut into) and the number of
// CTAs per SM are chosen by cc_batch_tune, which times each candidate with CUDA events.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fused.cuh"

namespace cc {

struct FusedPlan {
  int n_boxes = 0, n_items = 0, grid = 0, ctas_per_sm = 4, oversub = 1, max_mg = 0;
  int n_slabs = 0;
  FusedBox<float>* boxes32 = nullptr;
  FusedBox<double>* boxes64 = nullptr;
  FusedItem* items = nullptr;
  int* counters = nullptr;  // [1 + n_boxes + n_slabs]: work, per-box and per-slab done
  double* slab_ex = nullptr;
  void* part = nullptr;     // slab partials (sized for double)
  size_t bytes = 0;
};

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

static void plan_free(FusedPlan* p) {
  void* ptrs[] = {p->boxes32, p->boxes64, p->items, p->counters, p->slab_ex, p->part};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  *p = FusedPlan();
}

struct BoxIn {
  cc_tables t;
  int R_F;
  long long eps_off;
};

constexpr int kMaxGroups = kFusedMaxGroups;

// Build a plan: about slots x oversub items in total, shared among the boxes in
// proportion to their cost Mg^4 S; a box gets Mg slabs x n_groups node groups
// (n_groups <= min(S, 16)); items are ordered by decreasing cost.
static cc_status plan_build(const std::vector<BoxIn>& boxes, int ctas_per_sm, int oversub,
                            FusedPlan* out) {
  FusedPlan p;
  p.n_boxes = (int)boxes.size();
  p.ctas_per_sm = ctas_per_sm;
  p.oversub = oversub;
  double total = 0.0;
  for (const BoxIn& b : boxes) {
    const double mg = b.t->Mg;
    total += mg * mg * mg * mg * b.t->S_eff;
    p.max_mg = std::max(p.max_mg, b.t->Mg);
  }
  const double want = (double)sm_count() * ctas_per_sm * oversub;
  std::vector<FusedItem> items;
  std::vector<double> cost;
  std::vector<int> groups(boxes.size()), slab0(boxes.size());
  std::vector<long long> part_off(boxes.size());
  long long acc = 0;
  int slabs = 0;
  for (size_t b = 0; b < boxes.size(); ++b) {
    const cc_tables t = boxes[b].t;
    const double mg = t->Mg;
    const double share = want * mg * mg * mg * mg * t->S_eff / std::max(total, 1.0);
    int k = (int)std::lround(share / mg);
    k = std::max(1, std::min(k, std::min(t->S_eff, kMaxGroups)));
    groups[b] = k;
    slab0[b] = slabs;
    slabs += t->Mg;
    part_off[b] = acc;
    acc += (long long)k * t->Mg * t->Mg * t->Mg;
    for (int g = 0; g < k; ++g) {
      const int s0 = (int)((long long)t->S_eff * g / k), s1 = (int)((long long)t->S_eff * (g + 1) / k);
      for (int x = 0; x < t->Mg; ++x) {
        items.push_back({(int)b, x, s0, s1, g});
        cost.push_back(mg * mg * mg * (s1 - s0));
      }
    }
  }
  std::vector<int> order(items.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<FusedItem> sorted(items.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
  p.n_items = (int)sorted.size();
  p.n_slabs = slabs;
  p.grid = std::max(1, std::min(p.n_items, sm_count() * ctas_per_sm));
  auto alloc = [&](void** ptr, size_t bytes) -> cc_status {
    cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      set_last_error("cudaMalloc(fused plan)", e);
      return CC_ERR_ALLOC;
    }
    p.bytes += bytes;
    return CC_OK;
  };
  cc_status s = CC_OK;
  if (s == CC_OK) s = alloc((void**)&p.boxes32, sizeof(FusedBox<float>) * boxes.size());
  if (s == CC_OK) s = alloc((void**)&p.boxes64, sizeof(FusedBox<double>) * boxes.size());
  if (s == CC_OK) s = alloc((void**)&p.items, sizeof(FusedItem) * sorted.size());
  if (s == CC_OK) s = alloc((void**)&p.counters, sizeof(int) * (1 + boxes.size() + slabs));
  if (s == CC_OK) s = alloc((void**)&p.slab_ex, sizeof(double) * slabs);
  if (s == CC_OK) s = alloc(&p.part, (size_t)acc * sizeof(double));
  if (s != CC_OK) {
    plan_free(&p);
    return s;
  }
  int* slab_done = p.counters + 1 + boxes.size();
  std::vector<FusedBox<float>> b32(boxes.size());
  std::vector<FusedBox<double>> b64(boxes.size());
  for (size_t b = 0; b < boxes.size(); ++b) {
    const cc_tables t = boxes[b].t;
    const int periodic = t->p.kernel == CC_KERNEL_PERIODIC;
    const int n_items = t->Mg * groups[b];
    b32[b] = FusedBox<float>{t->p.R, boxes[b].R_F, t->Mg, t->S_eff, periodic, groups[b], n_items,
                             t->pref, t->d.Tm32, t->d.FW32, t->d.w64, t->d.FDb32,
                             reinterpret_cast<float*>(p.part) + part_off[b],
                             slab_done + slab0[b], p.slab_ex + slab0[b], boxes[b].eps_off,
                             (int)b};
    b64[b] = FusedBox<double>{t->p.R, boxes[b].R_F, t->Mg, t->S_eff, periodic, groups[b],
                              n_items, t->pref, t->d.Tm64, t->d.FW64, t->d.w64, t->d.FDb64,
                              reinterpret_cast<double*>(p.part) + part_off[b],
                              slab_done + slab0[b], p.slab_ex + slab0[b], boxes[b].eps_off,
                              (int)b};
  }
  if (cudaMemcpy(p.boxes32, b32.data(), sizeof(FusedBox<float>) * b32.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p.boxes64, b64.data(), sizeof(FusedBox<double>) * b64.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p.items, sorted.data(), sizeof(FusedItem) * sorted.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    plan_free(&p);
    return CC_ERR_CUDA;
  }
  *out = p;
  return CC_OK;
}

template <typename T>
static cc_status plan_launch(const FusedPlan& p, int rf_override, T* eps, double* Ex,
                             cudaStream_t st) {
  const size_t smem = slab_smem_bytes<T>(p.max_mg);
  auto kern = k_fused_exchange<T>;
  CC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFusedThreads, smem));
  const int grid = std::min(p.grid, std::max(1, per_sm) * sm_count());
  CC_CUDA(cudaMemsetAsync(p.counters, 0, sizeof(int) * (1 + p.n_boxes + p.n_slabs), st));
  const FusedBox<T>* boxes;
  if constexpr (sizeof(T) == 4) boxes = reinterpret_cast<const FusedBox<T>*>(p.boxes32);
  else boxes = reinterpret_cast<const FusedBox<T>*>(p.boxes64);
  kern<<<grid, kFusedThreads, smem, st>>>(boxes, p.items, p.n_items, p.counters, p.counters + 1,
                                          rf_override, eps, Ex);
  CC_CUDA(cudaGetLastError());
  return CC_OK;
}

// ---------------------------------------------------------------- single box hook
cc_status fused_single_alloc(cc_tables t) {
  if (t->Mg > kFusedMaxMg || t->fused) return CC_OK;
  FusedPlan* p = new (std::nothrow) FusedPlan();
  if (!p) return CC_ERR_ALLOC;
  std::vector<BoxIn> one{{t, 1, 0}};
  cc_status s = plan_build(one, 4, 1, p);
  if (s != CC_OK) {
    delete p;
    return s;
  }
  t->fused = p;
  t->device_bytes += p->bytes;
  return CC_OK;
}

void fused_single_free(cc_tables t) {
  FusedPlan* p = reinterpret_cast<FusedPlan*>(t->fused);
  if (!p) return;
  plan_free(p);
  delete p;
  t->fused = nullptr;
}

cc_status fused_single_exchange(cc_tables t, int R_F, int precision, void* eps, double* Ex,
                                cudaStream_t st) {
  FusedPlan* p = reinterpret_cast<FusedPlan*>(t->fused);
  if (!p) return CC_ERR_NOTSUPP;
  if (precision == CC_PREC_FP32) return plan_launch<float>(*p, R_F, (float*)eps, Ex, st);
  return plan_launch<double>(*p, R_F, (double*)eps, Ex, st);
}

}  // namespace cc

// ---------------------------------------------------------------- batch handle
struct cc_batch_s {
  std::vector<cc_tables> tabs;
  std::vector<cc_box> spec;
  std::vector<long long> eps_off;  // nbox + 1
  cc::FusedPlan plan;
  struct Graph {
    int prec;
    void* eps;
    double* Ex;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  int device = 0;
  void* mixed = nullptr;  // tensor-core form (periodic boxes), built on first use
};

using namespace cc;

static void batch_drop_graphs(cc_batch b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

static cc_status batch_plan(cc_batch b, int ctas_per_sm, int oversub) {
  std::vector<BoxIn> in;
  for (size_t i = 0; i < b->tabs.size(); ++i) in.push_back({b->tabs[i], b->spec[i].R_F, b->eps_off[i]});
  FusedPlan p;
  CC_TRY(plan_build(in, ctas_per_sm, oversub, &p));
  batch_drop_graphs(b);
  plan_free(&b->plan);
  b->plan = p;
  return CC_OK;
}

extern "C" cc_status cc_batch_create(const cc_box* boxes_host, int nbox, void* stream,
                                     cc_batch* out) {
  if (!boxes_host || !out || nbox < 1 || nbox > 65536) return CC_ERR_ARG;
  *out = nullptr;
  cc_batch b = new (std::nothrow) cc_batch_s();
  if (!b) return CC_ERR_ALLOC;
  cudaGetDevice(&b->device);
  cc_status s = CC_OK;
  long long off = 0;
  for (int i = 0; i < nbox && s == CC_OK; ++i) {
    const cc_box& bx = boxes_host[i];
    if (bx.p.R < 1 || 2 * bx.p.R + 1 > kFusedMaxMg || bx.R_F < 1 || bx.R_F > bx.p.R) {
      s = CC_ERR_RANGE;
      break;
    }
    cc_tables t = nullptr;
    s = build_tables_internal(&bx.p, as_stream(stream), false, &t);
    if (s != CC_OK) break;
    b->tabs.push_back(t);
    b->spec.push_back(bx);
    b->eps_off.push_back(off);
    off += (long long)t->Mg * t->Mg * t->Mg;
  }
  b->eps_off.push_back(off);
  if (s == CC_OK) s = batch_plan(b, 4, 2);
  if (s != CC_OK) {
    cc_batch_free(b);
    return s;
  }
  *out = b;
  return CC_OK;
}

extern "C" cc_status cc_batch_info(cc_batch b, int* nbox, long long* eps_offsets_host,
                                   int* n_items, size_t* device_bytes) {
  if (!b) return CC_ERR_ARG;
  if (nbox) *nbox = (int)b->tabs.size();
  if (eps_offsets_host)
    for (size_t i = 0; i < b->eps_off.size(); ++i) eps_offsets_host[i] = b->eps_off[i];
  if (n_items) *n_items = b->plan.n_items;
  if (device_bytes) {
    size_t s = b->plan.bytes;
    for (cc_tables t : b->tabs) s += t->device_bytes;
    *device_bytes = s;
  }
  return CC_OK;
}

extern "C" cc_status cc_batch_set_plan(cc_batch b, int ctas_per_sm, int oversub) {
  if (!b || ctas_per_sm < 1 || ctas_per_sm > 16 || oversub < 1 || oversub > 64) return CC_ERR_ARG;
  return batch_plan(b, ctas_per_sm, oversub);
}

extern "C" cc_status cc_batch_exchange(cc_batch b, int precision, void* eps_dev, double* Ex_dev,
                                       void* stream) {
  if (!b || !eps_dev || !Ex_dev) return CC_ERR_ARG;
  if (precision != CC_PREC_FP32 && precision != CC_PREC_FP64 && precision != CC_PREC_BF16X3)
    return CC_ERR_NOTSUPP;
  cudaStream_t st = as_stream(stream);
  if (precision == CC_PREC_BF16X3 && !b->mixed) {
    std::vector<int> rf;
    std::vector<long long> off(b->eps_off.begin(), b->eps_off.end() - 1);
    for (const cc_box& bx : b->spec) rf.push_back(bx.R_F);
    CC_TRY(mixed_batch_create(b->tabs, rf, off, &b->mixed));
  }
  for (auto& g : b->graphs)
    if (g.prec == precision && g.eps == eps_dev && g.Ex == Ex_dev) {
      CC_CUDA(cudaGraphLaunch(g.exec, st));
      return CC_OK;
    }
  // capture the whole batch (counter reset + one persistent launch) once per outputs
  cudaStream_t cap;
  CC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cc_status s = CC_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = CC_ERR_CUDA;
  if (s == CC_OK) {
    s = precision == CC_PREC_FP32    ? plan_launch<float>(b->plan, 0, (float*)eps_dev, Ex_dev, cap)
        : precision == CC_PREC_FP64  ? plan_launch<double>(b->plan, 0, (double*)eps_dev, Ex_dev, cap)
                                     : mixed_batch_run(b->mixed, (float*)eps_dev, Ex_dev, cap);
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (s == CC_OK && e != cudaSuccess) {
      set_last_error("cudaStreamEndCapture", e);
      s = CC_ERR_CUDA;
    }
  }
  cudaGraphExec_t exec = nullptr;
  if (s == CC_OK) {
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
      set_last_error("cudaGraphInstantiate", e);
      s = CC_ERR_CUDA;
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  CC_TRY(s);
  b->graphs.push_back({precision, eps_dev, Ex_dev, exec});
  CC_CUDA(cudaGraphLaunch(exec, st));
  return CC_OK;
}

// Autotuner: time every (CTAs per SM, oversubscription) candidate with CUDA events
// (median of `reps` graph replays after one warm-up) and keep the fastest.  Writes the
// choice to choice_host[2] and its time to *ms_host.
extern "C" cc_status cc_batch_tune(cc_batch b, int precision, void* eps_dev, double* Ex_dev,
                                   int reps, int* choice_host, float* ms_host, void* stream) {
  if (!b || !eps_dev || !Ex_dev || reps < 1) return CC_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (precision == CC_PREC_BF16X3) {
    // the tensor-core form: order of the boxes and cut of the unit sequence among the CTAs
    if (!b->mixed) CC_TRY(cc_batch_exchange(b, precision, eps_dev, Ex_dev, stream));
    CC_CUDA(cudaStreamSynchronize(st));
    batch_drop_graphs(b);  // captured launches hold the old plan's arguments
    CC_TRY(mixed_batch_tune(b->mixed, (float*)eps_dev, Ex_dev, reps, choice_host, ms_host, st));
    batch_drop_graphs(b);
    return CC_OK;
  }
  if (precision != CC_PREC_FP32 && precision != CC_PREC_FP64) return CC_ERR_NOTSUPP;
  const int cps[] = {2, 4, 8};
  const int ovs[] = {1, 2, 4};
  float best = 1e30f;
  int bc[2] = {4, 2};
  cudaEvent_t e0, e1;
  CC_CUDA(cudaEventCreate(&e0));
  CC_CUDA(cudaEventCreate(&e1));
  cc_status s = CC_OK;
  for (int c : cps)
    for (int o : ovs) {
      if (s != CC_OK) break;
      s = batch_plan(b, c, o);
      if (s != CC_OK) break;
      s = cc_batch_exchange(b, precision, eps_dev, Ex_dev, stream);
      std::vector<float> tm;
      for (int r = 0; r < reps && s == CC_OK; ++r) {
        cudaEventRecord(e0, st);
        s = cc_batch_exchange(b, precision, eps_dev, Ex_dev, stream);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = CC_ERR_CUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        tm.push_back(ms);
      }
      if (s != CC_OK) break;
      std::sort(tm.begin(), tm.end());
      const float med = tm[tm.size() / 2];
      if (med < best) {
        best = med;
        bc[0] = c;
        bc[1] = o;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CC_TRY(s);
  CC_TRY(batch_plan(b, bc[0], bc[1]));
  if (choice_host) memcpy(choice_host, bc, sizeof(bc));
  if (ms_host) *ms_host = best;
  return CC_OK;
}

extern "C" cc_status cc_batch_free(cc_batch b) {
  if (!b) return CC_ERR_ARG;
  batch_drop_graphs(b);
  plan_free(&b->plan);
  mixed_batch_free(b->mixed);
  for (cc_tables t : b->tabs) cc_tables_free(t);
  delete b;
  return CC_OK;
}
