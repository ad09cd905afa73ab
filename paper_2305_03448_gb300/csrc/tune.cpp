// Schedule selection: candidate counts, the tuned table, forced candidates,
// cost-model features, exhaustive measurement and the learned picker.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "desc_internal.h"

namespace desc {
int32_t mlp_pick_device(const float *params, int32_t F, int32_t H, const float *Xhost, int32_t ncand,
                        desc_stream_t s, int32_t *best);
}

using namespace desc;

namespace {

constexpr int kOps = 5;
constexpr int kMaxDevices = 64;
// (GPU model, op, dtype, floor(log2 n), floor(log2(aux + 1)))
using Key = std::tuple<std::string, int32_t, int32_t, int32_t, int32_t>;

std::mutex g_mu;
std::map<Key, int32_t> g_table;
thread_local int32_t g_force[kOps] = {-1, -1, -1, -1, -1};
const float *g_model = nullptr;
int32_t g_model_F = 0, g_model_H = 0;

int32_t ilog2(int64_t x) {
  int32_t r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

// The GPU model of the current device, spaces replaced by '_' ("none" without
// a device), looked up once per device.
std::string device_model() {
  static std::mutex mu;
  static std::string names[kMaxDevices];
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return "none";
  }
  std::lock_guard<std::mutex> lock(mu);
  if (names[dev].empty()) {
    cudaDeviceProp prop;
    std::string s = "none";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
      s = prop.name;
      for (char &c : s)
        if (c == ' ' || c == '\t' || c == '\n') c = '_';
      if (s.empty()) s = "unnamed";
    } else {
      (void)cudaGetLastError();
    }
    names[dev] = s;
  }
  return names[dev];
}

Key key_of(const std::string &dev, int32_t op, int32_t dtype, int64_t n, int64_t aux) {
  return Key(dev, op, dtype, ilog2(std::max<int64_t>(n, 1)), ilog2(aux + 1));
}

int ncand(int32_t op) {
  switch (op) {
    case DESC_OP_REDUCE: return reduce_candidates();
    case DESC_OP_SCAN: return scan_candidates();
    case DESC_OP_TRANSPOSE: return transpose_candidates();
    case DESC_OP_SEGMENTED: return kNumSegCands;
    case DESC_OP_MATMUL: return mm_candidates();
    default: return 0;
  }
}

bool problem_ok(const desc_problem *p) {
  if (!p || p->op < 0 || p->op >= kOps || !dtype_size(p->dtype) || p->n < 0 || p->aux < 0 || p->k < 0) return false;
  if (p->view && p->op != DESC_OP_REDUCE && p->op != DESC_OP_SCAN) return false;
  if (p->view && (p->level < DESC_LEVEL_GRID || p->level > DESC_LEVEL_THREAD)) return false;
  return true;
}

// What a problem's call looks like after lowering: the (n, aux) the op call
// passes to its schedule lookup, the (n, aux) the features describe, and the
// view composition.
struct Shape {
  int64_t key_n, key_aux;      // bucket of the tuned table
  int64_t n, aux;              // features [7..9]
  int counts[5];               // group, split, transpose, reverse, select views
  int depth;                   // deepest map nesting
  int hand;                    // the op's hand-indexed kernel applies
  int dims;                    // lowered dims after merging neighbours
  int64_t base_elems;          // elements of the view's base array
};

// Dims of a lowered map once extent-1 dims are dropped and neighbours that
// its strides walk as one are merged.
int merged_dims(const desc_lowered &L) {
  int m = 0;
  int64_t pe = 0, ps = 0;
  for (int i = 0; i < L.ndims; ++i) {
    if (L.extent[i] == 1) continue;
    if (m > 0 && ps == L.stride[i] * L.extent[i]) {
      pe *= L.extent[i];
      ps = L.stride[i];
    } else {
      ++m;
      pe = L.extent[i];
      ps = L.stride[i];
    }
  }
  (void)pe;
  return m;
}

void count_view(const desc_view &v, Shape *s) {
  for (int i = 0; i < v.nops && i < DESC_MAX_OPS; ++i) {
    const desc_view_op &o = v.ops[i];
    switch (o.kind) {
      case DESC_V_GROUP: ++s->counts[0]; break;
      case DESC_V_SPLIT_FST:
      case DESC_V_SPLIT_SND: ++s->counts[1]; break;
      case DESC_V_TRANSPOSE: ++s->counts[2]; break;
      case DESC_V_REVERSE: ++s->counts[3]; break;
      case DESC_V_SELECT: ++s->counts[4]; break;
      default: break;
    }
    s->depth = std::max(s->depth, (int)o.depth);
  }
}

// The plain form's view (see desc_problem), for reduce and scan.
void plain_view(const desc_problem *p, desc_view *v, desc_exec *ex, bool *has_ex) {
  std::memset(v, 0, sizeof(*v));
  v->rank = 1;
  v->shape[0] = p->n;
  *has_ex = false;
  if (p->op == DESC_OP_REDUCE && p->aux > 1) {
    v->nops = 2;
    v->ops[0].kind = DESC_V_GROUP;
    v->ops[0].k = p->aux ? p->n / p->aux : 0;
    v->ops[1].kind = DESC_V_SELECT;
    v->ops[1].level = DESC_LEVEL_BLOCK;
    v->ops[1].dim = DESC_DIM_X;
    *ex = desc_exec{{p->aux, 1, 1}, {1, 1, 1}};
    *has_ex = true;
  }
}

int32_t shape_of(const desc_problem *p, Shape *s) {
  std::memset(s, 0, sizeof(*s));
  s->key_n = s->n = p->n;
  s->key_aux = s->aux = p->aux;
  s->hand = 1;
  s->dims = 1;
  s->base_elems = p->n;
  if (p->op == DESC_OP_TRANSPOSE) {
    s->counts[2] = 1;
    s->dims = 2;
    return DESC_OK;
  }
  if (p->op != DESC_OP_REDUCE && p->op != DESC_OP_SCAN) return DESC_OK;
  desc_view pv;
  desc_exec pex;
  bool has_ex = false;
  const desc_view *v = p->view;
  const desc_exec *ex = p->ex;
  int32_t level = p->level;
  if (!v) {
    if (p->op == DESC_OP_REDUCE && p->aux > 1 && p->n % p->aux) return DESC_ERR_SHAPE;
    plain_view(p, &pv, &pex, &has_ex);
    v = &pv;
    ex = has_ex ? &pex : nullptr;
    level = has_ex ? DESC_LEVEL_BLOCK : DESC_LEVEL_GRID;
  }
  count_view(*v, s);
  desc_lowered L;
  const int32_t r = desc_lower_view(v, ex, &L);
  if (r != DESC_OK) return r;
  const Plan pl = split_plan(L, level);
  s->n = s->key_n = pl.n_keep * pl.n_rest;
  s->aux = pl.n_keep > 1 ? pl.n_keep : 0;
  s->base_elems = L.base_elems;
  s->dims = merged_dims(L);
  int64_t start0 = 0, seg = 0;
  if (p->op == DESC_OP_REDUCE) {
    s->key_aux = s->aux;
    s->hand = rest_contiguous(pl, true, &start0, &seg) ? 1 : 0;
  } else {
    s->key_aux = 0;                                    // desc_scan's lookup ignores segments
    s->hand = (rest_contiguous(pl, false, &start0, &seg) && (pl.n_keep <= 1 || seg == pl.n_rest)) ? 1 : 0;
  }
  return DESC_OK;
}

// Fraction of segments per floor(log2 len) bucket of width 3, empty
// segments in the first bucket.
void length_histogram(const int64_t *len, int64_t count, float *h) {
  for (int i = 0; i < 8; ++i) h[i] = 0.f;
  if (!len || count <= 0) return;
  std::vector<int64_t> c(8, 0);
  for (int64_t i = 0; i < count; ++i) {
    const int b = len[i] <= 0 ? 0 : std::min(ilog2(len[i]) / 3, 7);
    ++c[size_t(b)];
  }
  for (int i = 0; i < 8; ++i) h[i] = float(double(c[size_t(i)]) / double(count));
}

}  // namespace

namespace desc {
int32_t schedule_for(int32_t op, int32_t dtype, int64_t n, int64_t aux) {
  if (op < 0 || op >= kOps) return -1;
  if (g_force[op] >= 0) return g_force[op];
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_table.empty()) return -1;
  }
  const std::string dev = device_model();
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(key_of(dev, op, dtype, n, aux));
  return it == g_table.end() ? -1 : it->second;
}
}  // namespace desc

extern "C" int32_t desc_candidate_count(int32_t op, int32_t *count) {
  if (!count || op < 0 || op >= kOps) return DESC_ERR_INVALID_ARG;
  *count = ncand(op);
  return DESC_OK;
}

extern "C" int32_t desc_force_candidate(int32_t op, int32_t cand) {
  if (op < 0 || op >= kOps || cand >= ncand(op)) return DESC_ERR_INVALID_ARG;
  g_force[op] = cand < 0 ? -1 : cand;
  return DESC_OK;
}

extern "C" int32_t desc_features(const desc_problem *p, int32_t cand, float *out, int32_t nout) {
  if (!problem_ok(p) || !out || nout < DESC_NUM_FEATURES || cand < 0 || cand >= ncand(p->op))
    return DESC_ERR_INVALID_ARG;
  Shape sh;
  const int32_t r = shape_of(p, &sh);
  if (r != DESC_OK) return r;
  for (int i = 0; i < DESC_NUM_FEATURES; ++i) out[i] = 0.f;
  auto lg = [](double x) { return (float)std::log2(std::max(x, 1.0)); };
  out[p->op] = 1.f;
  out[5 + (p->dtype == DESC_F32 ? 1 : 0)] = 1.f;
  out[7] = lg((double)sh.n) / 32.f;
  out[8] = lg((double)sh.aux + 1.0) / 32.f;
  out[9] = lg((double)sh.n / ((double)sh.aux + 1.0) + 1.0) / 32.f;
  if (p->op == DESC_OP_SEGMENTED) length_histogram(p->seg_lengths, p->aux, out + 10);
  if (p->op == DESC_OP_REDUCE) {
    const ReduceCand &c = kReduceCands[cand];
    out[18] = lg(256.0 * 4 * c.unroll) / 32.f;
    out[19] = c.unroll / 16.f;
    out[20] = lg((double)c.target_ctas) / 16.f;
    out[29] = (float)c.nc;
  } else if (p->op == DESC_OP_TRANSPOSE) {
    const double td = kTransposeTiles[cand];
    out[18] = lg(td * td) / 32.f;
  } else if (p->op == DESC_OP_MATMUL) {
    const MmCand &c = kMmCands[cand];
    out[18] = lg(c.pairs ? 256.0 * 256.0 * c.width : 128.0 * 256.0) / 32.f;
    out[20] = lg((double)c.group_rows) / 16.f;
    out[30] = lg((double)p->k + 1.0) / 32.f;
    out[31] = (float)c.pairs;
  } else if (p->op == DESC_OP_SEGMENTED) {
    const SegCand &c = kSegCands[cand];
    out[18] = lg(c.threads ? double(c.threads) * 4 : double(kScanSubTile) * c.sub) / 32.f;   // points per step
    out[19] = (c.threads ? 4.f : 16.f) / 16.f;                                            // items per thread
    out[20] = c.threads ? lg((double)c.threads) / 16.f : 0.f;                              // threads per segment
  } else {
    out[18] = lg(double(kScanSubTile) * kScanSubCands[cand]) / 32.f;
    out[19] = 16.f / 16.f;
  }
  out[21 + cand] = 1.f;
  for (int i = 0; i < 5; ++i) out[32 + i] = sh.counts[i] / 8.f;
  out[37] = sh.depth / 4.f;
  out[38] = (float)sh.hand;
  out[39] = sh.dims / 8.f;
  return DESC_OK;
}

namespace {

// One launch of the problem's call with the current forced candidate.
int32_t run_problem(const desc_problem *p, const desc_tune_buffers *b, desc_stream_t s) {
  if (p->view) {
    Shape sh;
    int32_t r = shape_of(p, &sh);
    if (r != DESC_OK) return r;
    const size_t nb = size_t(sh.base_elems) * 4;
    if (p->op == DESC_OP_REDUCE) {
      const size_t ob = size_t(std::max<int64_t>(sh.aux, 1)) * 4;
      return desc_reduce(p->view, p->ex, p->level, p->dtype, b->in, nb, b->out, ob, 0, b->ws, b->ws_bytes, s);
    }
    return desc_scan(p->view, p->ex, p->level, p->dtype, b->in, nb, b->out, nb, 0, b->ws, b->ws_bytes, s);
  }
  desc_view v;
  desc_exec ex;
  bool has_ex = false;
  const size_t nb = size_t(p->n) * 4;
  switch (p->op) {
    case DESC_OP_REDUCE: {
      if (p->aux > 1 && p->n % p->aux) return DESC_ERR_SHAPE;
      plain_view(p, &v, &ex, &has_ex);
      if (has_ex)
        return desc_reduce(&v, &ex, DESC_LEVEL_BLOCK, p->dtype, b->in, nb, b->out, size_t(p->aux) * 4, 0, b->ws,
                           b->ws_bytes, s);
      return desc_reduce(&v, nullptr, DESC_LEVEL_GRID, p->dtype, b->in, nb, b->out, 4, 0, b->ws, b->ws_bytes, s);
    }
    case DESC_OP_SCAN:
      plain_view(p, &v, &ex, &has_ex);
      return desc_scan(&v, nullptr, DESC_LEVEL_GRID, p->dtype, b->in, nb, b->out, nb, 0, b->ws, b->ws_bytes, s);
    case DESC_OP_TRANSPOSE: {
      if (p->aux <= 0 || p->n % p->aux) return DESC_ERR_SHAPE;
      const int64_t R = p->aux, C = p->n / p->aux;
      desc_view vi, vo;
      std::memset(&vi, 0, sizeof(vi));
      std::memset(&vo, 0, sizeof(vo));
      vi.rank = vo.rank = 2;
      vi.shape[0] = R; vi.shape[1] = C;
      vo.shape[0] = C; vo.shape[1] = R;
      vi.nops = 1;
      vi.ops[0].kind = DESC_V_TRANSPOSE;
      return desc_transpose(&vi, &vo, nullptr, p->dtype, b->in, nb, b->out, nb, s);
    }
    case DESC_OP_SEGMENTED:
      return desc_segmented_reduce_scan(b->offsets, p->aux, p->n, p->dtype, b->in, b->out, b->sums, 0, b->ws,
                                        b->ws_bytes, s);
    case DESC_OP_MATMUL: {
      const int64_t M = p->n, N = p->aux, K = p->k;
      return desc_matmul(nullptr, nullptr, M, N, K, static_cast<const float *>(b->in), size_t(M * K) * 4,
                         static_cast<const float *>(b->in2), size_t(K * N) * 4, static_cast<float *>(b->out),
                         size_t(M * N) * 4, DESC_MM_BF16, b->ws, b->ws_bytes, s);
    }
    default:
      return DESC_ERR_INVALID_ARG;
  }
}

// Medians of `reps` timed launches of each listed candidate; rounds visit
// every candidate once (with a warm-up launch before each candidate's first
// round).
int32_t measure(const desc_problem *p, const desc_tune_buffers *b, const int32_t *cands, int nc, int reps,
                desc_stream_t s, float *us) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  std::vector<cudaEvent_t> ev(size_t(2 * nc));
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return DESC_ERR_CUDA;
  const int32_t saved = g_force[p->op];
  int32_t r = DESC_OK;
  std::vector<std::vector<float>> t(static_cast<size_t>(nc));
  for (int c = 0; c < nc && r == DESC_OK; ++c) {   // warm-up
    g_force[p->op] = cands[c];
    r = run_problem(p, b, s);
  }
  for (int i = 0; i < reps && r == DESC_OK; ++i) {
    for (int c = 0; c < nc && r == DESC_OK; ++c) {
      g_force[p->op] = cands[c];
      cudaEventRecord(ev[size_t(2 * c)], st);
      r = run_problem(p, b, s);
      cudaEventRecord(ev[size_t(2 * c + 1)], st);
    }
    if (r != DESC_OK) break;
    if (cudaEventSynchronize(ev[size_t(2 * nc - 1)]) != cudaSuccess) { r = DESC_ERR_CUDA; break; }
    for (int c = 0; c < nc; ++c) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[size_t(2 * c)], ev[size_t(2 * c + 1)]);
      t[size_t(c)].push_back(ms);
    }
  }
  g_force[p->op] = saved;
  for (auto &e : ev) cudaEventDestroy(e);
  if (r != DESC_OK) return r;
  for (int c = 0; c < nc; ++c) {
    std::vector<float> &v = t[size_t(c)];
    std::nth_element(v.begin(), v.begin() + reps / 2, v.end());
    us[c] = v[size_t(reps / 2)] * 1000.f;
  }
  return DESC_OK;
}

}  // namespace

extern "C" int32_t desc_tune_measure(const desc_problem *p, const desc_tune_buffers *b, int32_t reps,
                                     desc_stream_t s, float *us) {
  if (!problem_ok(p) || !b || !us || reps < 1) return DESC_ERR_INVALID_ARG;
  const int nc = ncand(p->op);
  std::vector<int32_t> all(static_cast<size_t>(nc));
  for (int c = 0; c < nc; ++c) all[size_t(c)] = c;
  return measure(p, b, all.data(), nc, reps, s, us);
}

extern "C" int32_t desc_tune_measure_cands(const desc_problem *p, const desc_tune_buffers *b, const int32_t *cands,
                                           int32_t ncands, int32_t reps, desc_stream_t s, float *us) {
  if (!problem_ok(p) || !b || !us || !cands || ncands < 1 || reps < 1) return DESC_ERR_INVALID_ARG;
  for (int i = 0; i < ncands; ++i)
    if (cands[i] < 0 || cands[i] >= ncand(p->op)) return DESC_ERR_INVALID_ARG;
  return measure(p, b, cands, ncands, reps, s, us);
}

namespace {
int32_t problem_key(const desc_problem *p, Key *k) {
  Shape sh;
  const int32_t r = shape_of(p, &sh);
  if (r != DESC_OK) return r;
  *k = key_of(device_model(), p->op, p->dtype, sh.key_n, sh.key_aux);
  return DESC_OK;
}
}  // namespace

extern "C" int32_t desc_tune_record(const desc_problem *p, int32_t cand) {
  if (!problem_ok(p) || cand < 0 || cand >= ncand(p->op)) return DESC_ERR_INVALID_ARG;
  Key k;
  const int32_t r = problem_key(p, &k);
  if (r != DESC_OK) return r;
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[k] = cand;
  return DESC_OK;
}

extern "C" int32_t desc_tune_lookup(const desc_problem *p, int32_t *cand) {
  if (!problem_ok(p) || !cand) return DESC_ERR_INVALID_ARG;
  Key k;
  const int32_t r = problem_key(p, &k);
  if (r != DESC_OK) return r;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(k);
  *cand = it == g_table.end() ? -1 : it->second;
  return DESC_OK;
}

extern "C" int32_t desc_tune_exhaustive(const desc_problem *p, const desc_tune_buffers *b, int32_t reps,
                                        desc_stream_t s, int32_t *best) {
  if (!best) return DESC_ERR_INVALID_ARG;
  float us[16];
  if (!problem_ok(p) || ncand(p->op) > 16) return DESC_ERR_INVALID_ARG;
  const int32_t r = desc_tune_measure(p, b, reps, s, us);
  if (r != DESC_OK) return r;
  int c = 0;
  for (int i = 1; i < ncand(p->op); ++i)
    if (us[i] < us[c]) c = i;                 // strict: ties keep the lower index
  *best = c;
  return desc_tune_record(p, c);
}

extern "C" int32_t desc_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
  return DESC_OK;
}

extern "C" int32_t desc_tune_save(const char *path) {
  if (!path) return DESC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  FILE *f = std::fopen(path, "w");
  if (!f) return DESC_ERR_INVALID_ARG;
  std::fprintf(f, "# libdesc schedule table: gpu_model op dtype log2_n log2_aux1 candidate\n");
  for (auto &kv : g_table)
    std::fprintf(f, "%s %d %d %d %d %d\n", std::get<0>(kv.first).c_str(), std::get<1>(kv.first),
                 std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second);
  std::fclose(f);
  return DESC_OK;
}

extern "C" int32_t desc_tune_load(const char *path) {
  if (!path) return DESC_ERR_INVALID_ARG;
  FILE *f = std::fopen(path, "r");
  if (!f) return DESC_ERR_INVALID_ARG;
  std::map<Key, int32_t> t;
  char line[512];
  int32_t r = DESC_OK;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    char dev[256];
    int op, dt, ln, la, c;
    if (std::sscanf(line, "%255s %d %d %d %d %d", dev, &op, &dt, &ln, &la, &c) != 6 || op < 0 || op >= kOps ||
        c < 0 || c >= ncand(op)) {
      r = DESC_ERR_INVALID_ARG;
      break;
    }
    t[Key(std::string(dev), op, dt, ln, la)] = c;
  }
  std::fclose(f);
  if (r != DESC_OK) return r;
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto &kv : t) g_table[kv.first] = kv.second;
  return DESC_OK;
}

extern "C" int32_t desc_tune_set_model(const float *params, int32_t F, int32_t H) {
  if ((params && (F != DESC_NUM_FEATURES || H < 32 || H > 64 || H % 32)) ) return DESC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  g_model = params;
  g_model_F = F;
  g_model_H = H;
  return DESC_OK;
}

extern "C" int32_t desc_tune_predict(const desc_problem *p, desc_stream_t s, int32_t *best) {
  if (!problem_ok(p) || !best) return DESC_ERR_INVALID_ARG;
  const float *model;
  int32_t F, H;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    model = g_model;
    F = g_model_F;
    H = g_model_H;
  }
  if (!model) return DESC_ERR_INVALID_ARG;
  const int nc = ncand(p->op);
  std::vector<float> X(size_t(nc) * F);
  for (int c = 0; c < nc; ++c) {
    const int32_t r = desc_features(p, c, &X[size_t(c) * F], F);
    if (r != DESC_OK) return r;
  }
  const int32_t r = mlp_pick_device(model, F, H, X.data(), nc, s, best);
  if (r != DESC_OK) return r;
  return desc_tune_record(p, *best);
}
