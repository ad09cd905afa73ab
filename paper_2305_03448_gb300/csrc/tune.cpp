// Schedule selection: candidate counts, the tuned table, forced candidates,
// cost-model features, exhaustive measurement and the learned picker.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
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
using Key = std::tuple<int32_t, int32_t, int32_t, int32_t>;

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

Key key_of(int32_t op, int32_t dtype, int64_t n, int64_t aux) {
  return Key(op, dtype, ilog2(std::max<int64_t>(n, 1)), ilog2(aux + 1));
}

int ncand(int32_t op) {
  switch (op) {
    case DESC_OP_REDUCE: return reduce_candidates();
    case DESC_OP_SCAN: return scan_candidates();
    case DESC_OP_TRANSPOSE: return transpose_candidates();
    case DESC_OP_SEGMENTED: return scan_candidates();
    case DESC_OP_MATMUL: return mm_candidates();
    default: return 0;
  }
}

bool problem_ok(const desc_problem *p) {
  return p && p->op >= 0 && p->op < kOps && dtype_size(p->dtype) && p->n >= 0 && p->aux >= 0 && p->k >= 0;
}

}  // namespace

namespace desc {
int32_t schedule_for(int32_t op, int32_t dtype, int64_t n, int64_t aux) {
  if (op < 0 || op >= kOps) return -1;
  if (g_force[op] >= 0) return g_force[op];
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_table.empty()) return -1;
  auto it = g_table.find(key_of(op, dtype, n, aux));
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
  // [0, 5) op, [5, 7) dtype, [7] log2 n, [8] log2 (aux + 1), [9] log2 (n / (aux + 1) + 1),
  // [10, 18) segment histogram, [18] log2 tile, [19] vectors, [20] log2 CTAs or group,
  // [21, 29) candidate, [29] load path, [30] log2 (K + 1), [31] CTA pairs
  for (int i = 0; i < DESC_NUM_FEATURES; ++i) out[i] = 0.f;
  auto lg = [](double x) { return (float)std::log2(std::max(x, 1.0)); };
  out[p->op] = 1.f;
  out[5 + (p->dtype == DESC_F32 ? 1 : 0)] = 1.f;
  out[7] = lg((double)p->n) / 32.f;
  out[8] = lg((double)p->aux + 1.0) / 32.f;
  out[9] = lg((double)p->n / ((double)p->aux + 1.0) + 1.0) / 32.f;
  if (p->op == DESC_OP_SEGMENTED)
    for (int i = 0; i < 8; ++i) out[10 + i] = p->seg_hist[i];
  static const int unroll[8] = {8, 4, 8, 4, 8, 8, 4, 8};
  static const int ctas[8] = {1216, 1216, 608, 2432, 2432, 304, 2432, 1216};
  static const int nc[8] = {0, 0, 0, 0, 0, 0, 1, 1};
  static const int subs[3] = {4, 2, 1};
  if (p->op == DESC_OP_REDUCE) {
    out[18] = lg(256.0 * 4 * unroll[cand]) / 32.f;
    out[19] = unroll[cand] / 16.f;
    out[20] = lg((double)ctas[cand]) / 16.f;
    out[29] = (float)nc[cand];
  } else if (p->op == DESC_OP_TRANSPOSE) {
    const double td = cand == 0 ? 64 : 32;
    out[18] = lg(td * td) / 32.f;
  } else if (p->op == DESC_OP_MATMUL) {
    int pairs = 0, group = 0, width = 1;
    mm_candidate(cand, &pairs, &group, &width);
    out[18] = lg(pairs ? 256.0 * 256.0 * width : 128.0 * 256.0) / 32.f;
    out[20] = lg((double)group) / 16.f;
    out[30] = lg((double)p->k + 1.0) / 32.f;
    out[31] = (float)pairs;
  } else {
    out[18] = lg(4096.0 * subs[cand]) / 32.f;
    out[19] = 16.f / 16.f;
  }
  out[21 + cand] = 1.f;
  return DESC_OK;
}

namespace {

// One launch of the problem's canonical call with the current forced candidate.
int32_t run_problem(const desc_problem *p, const desc_tune_buffers *b, desc_stream_t s) {
  desc_view v;
  std::memset(&v, 0, sizeof(v));
  v.rank = 1;
  v.shape[0] = p->n;
  const size_t nb = size_t(p->n) * 4;
  switch (p->op) {
    case DESC_OP_REDUCE: {
      if (p->aux > 1) {
        if (p->n % p->aux) return DESC_ERR_SHAPE;
        v.nops = 2;
        v.ops[0].kind = DESC_V_GROUP;
        v.ops[0].k = p->n / p->aux;
        v.ops[1].kind = DESC_V_SELECT;
        v.ops[1].level = DESC_LEVEL_BLOCK;
        v.ops[1].dim = DESC_DIM_X;
        desc_exec ex = {{p->aux, 1, 1}, {1, 1, 1}};
        return desc_reduce(&v, &ex, DESC_LEVEL_BLOCK, p->dtype, b->in, nb, b->out, size_t(p->aux) * 4, 0, b->ws,
                           b->ws_bytes, s);
      }
      return desc_reduce(&v, nullptr, DESC_LEVEL_GRID, p->dtype, b->in, nb, b->out, 4, 0, b->ws, b->ws_bytes, s);
    }
    case DESC_OP_SCAN:
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

}  // namespace

extern "C" int32_t desc_tune_measure(const desc_problem *p, const desc_tune_buffers *b, int32_t reps,
                                     desc_stream_t s, float *us) {
  if (!problem_ok(p) || !b || !us || reps < 1) return DESC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  const int nc = ncand(p->op);
  std::vector<cudaEvent_t> ev(size_t(reps) + 1);
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return DESC_ERR_CUDA;
  const int32_t saved = g_force[p->op];
  int32_t r = DESC_OK;
  for (int c = 0; c < nc && r == DESC_OK; ++c) {
    g_force[p->op] = c;
    if ((r = run_problem(p, b, s)) != DESC_OK) break;   // warm-up
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < reps && r == DESC_OK; ++i) {
      r = run_problem(p, b, s);
      cudaEventRecord(ev[size_t(i) + 1], st);
    }
    if (r != DESC_OK) break;
    if (cudaEventSynchronize(ev[size_t(reps)]) != cudaSuccess) { r = DESC_ERR_CUDA; break; }
    std::vector<float> t(reps);
    for (int i = 0; i < reps; ++i) cudaEventElapsedTime(&t[i], ev[size_t(i)], ev[size_t(i) + 1]);
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    us[c] = t[size_t(reps / 2)] * 1000.f;
  }
  g_force[p->op] = saved;
  for (auto &e : ev) cudaEventDestroy(e);
  return r;
}

extern "C" int32_t desc_tune_record(const desc_problem *p, int32_t cand) {
  if (!problem_ok(p) || cand < 0 || cand >= ncand(p->op)) return DESC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[key_of(p->op, p->dtype, p->n, p->aux)] = cand;
  return DESC_OK;
}

extern "C" int32_t desc_tune_lookup(const desc_problem *p, int32_t *cand) {
  if (!problem_ok(p) || !cand) return DESC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(key_of(p->op, p->dtype, p->n, p->aux));
  *cand = it == g_table.end() ? -1 : it->second;
  return DESC_OK;
}

extern "C" int32_t desc_tune_exhaustive(const desc_problem *p, const desc_tune_buffers *b, int32_t reps,
                                        desc_stream_t s, int32_t *best) {
  if (!best) return DESC_ERR_INVALID_ARG;
  float us[8];
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
  std::fprintf(f, "# libdesc schedule table: op dtype log2_n log2_aux1 candidate\n");
  for (auto &kv : g_table)
    std::fprintf(f, "%d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                 std::get<3>(kv.first), kv.second);
  std::fclose(f);
  return DESC_OK;
}

extern "C" int32_t desc_tune_load(const char *path) {
  if (!path) return DESC_ERR_INVALID_ARG;
  FILE *f = std::fopen(path, "r");
  if (!f) return DESC_ERR_INVALID_ARG;
  std::map<Key, int32_t> t;
  char line[256];
  int32_t r = DESC_OK;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int op, dt, ln, la, c;
    if (std::sscanf(line, "%d %d %d %d %d", &op, &dt, &ln, &la, &c) != 5 || op < 0 || op >= kOps || c < 0 ||
        c >= ncand(op)) {
      r = DESC_ERR_INVALID_ARG;
      break;
    }
    t[Key(op, dt, ln, la)] = c;
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
