// View lowering and the access-conflict check: host code of libdesc.
//
// Lowering (Section 3.2 views, Section 5 index generation).  Every basic
// view maps an index of its output affinely to an index of its input, so a
// chain of views composed onto a row-major base array is one affine map
// from the logical domain to the base.  The map is built forwards, view by
// view, keeping for every current axis its extent and its stride in the
// base array, plus one offset:
//   group k      axis (n, s)       -> (n/k, k*s), (k, s)
//   split fst k  axis (n, s)       -> (k, s)
//   split snd k  axis (n, s)       -> (n-k, s), offset += k*s
//   transpose    axes a, b         -> b, a
//   reverse      axis (n, s)       -> (n, -s), offset += (n-1)*s
//   select       outermost axis    -> moved to the selected dims
//
// Access conflicts (Section 3.3 narrowing, Section 4 access_safety_check):
// an element must not be written by two threads, nor written by one thread
// and read by another, within one phase.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "desc_internal.h"

namespace {

constexpr int64_t kMaxElems = int64_t(1) << 46;
constexpr int64_t kMaxEnum = int64_t(1) << 24;

bool mul_ok(int64_t a, int64_t b, int64_t *r) {
  if (a < 0 || b < 0) return false;
  if (a != 0 && b > kMaxElems / a) return false;
  *r = a * b;
  return true;
}

struct Axis {
  int64_t extent, stride;
};

struct SelDim {
  int64_t extent, stride;
  int32_t level, dim;
};

// Number of sub-resources a select at (level, dim) distributes over.
int64_t resource_count(const desc_exec &ex, int32_t level, int32_t dim) {
  const int64_t nt = ex.block[0] * ex.block[1] * ex.block[2];
  if (level == DESC_LEVEL_BLOCK) return ex.grid[dim];
  if (level == DESC_LEVEL_WARP) return nt / 32;
  if (dim == DESC_DIM_LANE) return 32;
  return ex.block[dim];
}

bool exec_ok(const desc_exec &ex) {
  for (int d = 0; d < 3; ++d)
    if (ex.grid[d] < 1 || ex.block[d] < 1 || ex.grid[d] > (int64_t(1) << 31) ||
        ex.block[d] > 4096)
      return false;
  return true;
}

}  // namespace

extern "C" const char *desc_status_string(int32_t s) {
  switch (s) {
    case DESC_OK: return "DESC_OK";
    case DESC_ERR_INVALID_ARG: return "DESC_ERR_INVALID_ARG";
    case DESC_ERR_SHAPE: return "DESC_ERR_SHAPE";
    case DESC_ERR_OVERLAP: return "DESC_ERR_OVERLAP";
    case DESC_ERR_HOST_POINTER: return "DESC_ERR_HOST_POINTER";
    case DESC_ERR_SIZE_MISMATCH: return "DESC_ERR_SIZE_MISMATCH";
    case DESC_ERR_ALIGNMENT: return "DESC_ERR_ALIGNMENT";
    case DESC_ERR_UNSUPPORTED: return "DESC_ERR_UNSUPPORTED";
    case DESC_ERR_CUDA: return "DESC_ERR_CUDA";
    case DESC_ERR_DEVICE_TIMEOUT: return "DESC_ERR_DEVICE_TIMEOUT";
    case DESC_ERR_WORKSPACE: return "DESC_ERR_WORKSPACE";
    case DESC_ERR_BARRIER: return "DESC_ERR_BARRIER";
    default: return "DESC_ERR_UNKNOWN";
  }
}

extern "C" int32_t desc_version(void) { return (1 << 16) | 0; }

extern "C" int32_t desc_lower_view(const desc_view *v, const desc_exec *ex, desc_lowered *out) {
  if (!v || !out) return DESC_ERR_INVALID_ARG;
  if (v->rank < 1 || v->rank > DESC_MAX_RANK) return DESC_ERR_SHAPE;
  if (v->nops < 0 || v->nops > DESC_MAX_OPS) return DESC_ERR_INVALID_ARG;
  if (ex && !exec_ok(*ex)) return DESC_ERR_INVALID_ARG;

  std::vector<Axis> ax(v->rank);
  int64_t n_base = 1;
  for (int i = 0; i < v->rank; ++i)
    if (!mul_ok(n_base, v->shape[i], &n_base)) return DESC_ERR_SHAPE;
  int64_t s = 1;
  for (int i = v->rank - 1; i >= 0; --i) {
    ax[i] = {v->shape[i], s};
    s *= std::max<int64_t>(v->shape[i], 1);
  }
  int64_t off = 0;
  std::vector<SelDim> sel;
  int32_t last_level = DESC_LEVEL_BLOCK;
  bool after_warp = false;
  bool seen[4][4] = {};

  for (int i = 0; i < v->nops; ++i) {
    const desc_view_op &op = v->ops[i];
    if (op.kind == DESC_V_SELECT) {
      if (op.depth != 0 || ax.empty()) return DESC_ERR_SHAPE;
      if (op.level < DESC_LEVEL_BLOCK || op.level > DESC_LEVEL_THREAD) return DESC_ERR_SHAPE;
      if (op.dim < DESC_DIM_X || op.dim > DESC_DIM_Z) return DESC_ERR_SHAPE;
      if (op.level < last_level) return DESC_ERR_SHAPE;   // must narrow
      int32_t dim = op.dim;
      if (op.level == DESC_LEVEL_WARP && dim != DESC_DIM_X) return DESC_ERR_SHAPE;
      if (op.level == DESC_LEVEL_THREAD && after_warp) {
        if (dim != DESC_DIM_X) return DESC_ERR_SHAPE;
        dim = DESC_DIM_LANE;
      }
      if (seen[op.level][dim]) return DESC_ERR_SHAPE;
      seen[op.level][dim] = true;
      if (ex) {
        if (op.level == DESC_LEVEL_WARP && (ex->block[0] * ex->block[1] * ex->block[2]) % 32)
          return DESC_ERR_SHAPE;
        if (ax[0].extent != resource_count(*ex, op.level, dim)) return DESC_ERR_SHAPE;
      }
      sel.push_back({ax[0].extent, ax[0].stride, op.level, dim});
      ax.erase(ax.begin());
      if (op.level == DESC_LEVEL_WARP) after_warp = true;
      last_level = op.level;
      continue;
    }
    const int d = op.depth;
    if (d < 0 || d >= (int)ax.size()) return DESC_ERR_SHAPE;
    const int64_t n = ax[d].extent, st = ax[d].stride;
    switch (op.kind) {
      case DESC_V_GROUP:
        if (op.k < 1 || n % op.k != 0) return DESC_ERR_SHAPE;
        ax[d] = {n / op.k, op.k * st};
        ax.insert(ax.begin() + d + 1, Axis{op.k, st});
        break;
      case DESC_V_SPLIT_FST:
        if (op.k < 0 || op.k > n) return DESC_ERR_SHAPE;
        ax[d].extent = op.k;
        break;
      case DESC_V_SPLIT_SND:
        if (op.k < 0 || op.k > n) return DESC_ERR_SHAPE;
        ax[d].extent = n - op.k;
        off += op.k * st;
        break;
      case DESC_V_TRANSPOSE:
        if (d + 1 >= (int)ax.size()) return DESC_ERR_SHAPE;
        std::swap(ax[d], ax[d + 1]);
        break;
      case DESC_V_REVERSE:
        if (n > 0) off += (n - 1) * st;
        ax[d].stride = -st;
        break;
      default:
        return DESC_ERR_INVALID_ARG;
    }
    if ((int)(sel.size() + ax.size()) > DESC_MAX_DIMS) return DESC_ERR_UNSUPPORTED;
  }
  if ((int)(sel.size() + ax.size()) > DESC_MAX_DIMS) return DESC_ERR_UNSUPPORTED;

  desc_lowered L;
  std::memset(&L, 0, sizeof(L));
  L.nsel = (int32_t)sel.size();
  L.ndims = (int32_t)(sel.size() + ax.size());
  int k = 0;
  for (auto &sd : sel) {
    L.extent[k] = sd.extent; L.stride[k] = sd.stride; L.level[k] = sd.level; L.dim[k] = sd.dim;
    ++k;
  }
  for (auto &a : ax) {
    L.extent[k] = a.extent; L.stride[k] = a.stride; L.level[k] = -1; L.dim[k] = -1;
    ++k;
  }
  L.offset = off;
  L.base_elems = n_base;
  *out = L;
  return DESC_OK;
}

namespace desc {

bool affine_injective(const int64_t *extent, const int64_t *stride, int n) {
  std::vector<Dim> d;
  for (int i = 0; i < n; ++i) {
    if (extent[i] == 0) return true;        // empty domain
    if (extent[i] > 1) d.push_back({extent[i], std::llabs(stride[i])});
  }
  std::sort(d.begin(), d.end(), [](const Dim &a, const Dim &b) { return a.stride < b.stride; });
  int64_t span = 0;   // largest distance reachable with the smaller strides
  for (auto &x : d) {
    if (x.stride <= span) return false;
    span += x.stride * (x.extent - 1);
  }
  return true;
}

Plan split_plan(const desc_lowered &L, int32_t cut) {
  Plan p;
  std::memset(&p, 0, sizeof(p));
  p.offset = L.offset;
  p.n_keep = 1;
  p.n_rest = 1;
  for (int i = 0; i < L.ndims; ++i) {
    const bool keep = i < L.nsel && L.level[i] <= cut;
    if (keep) {
      p.keep[p.nkeep++] = {L.extent[i], L.stride[i]};
      p.n_keep *= L.extent[i];
    } else {
      p.rest[p.nrest++] = {L.extent[i], L.stride[i]};
      p.n_rest *= L.extent[i];
    }
  }
  return p;
}

bool rest_contiguous(const Plan &p, bool any_order, int64_t *start0, int64_t *seg_stride) {
  // The remaining dims must cover one contiguous run of n_rest elements:
  // in logical order with stride +1 after merging (any_order == false, the
  // scan), or as a set (any_order == true, the reduce: dims may come in any
  // order and with negative strides).
  std::vector<Dim> r;
  for (int i = 0; i < p.nrest; ++i)
    if (p.rest[i].extent != 1) r.push_back(p.rest[i]);
  int64_t lo_adj = 0;   // offset of the lowest element of the run
  if (any_order) {
    for (auto &d : r)
      if (d.stride < 0 && d.extent > 0) lo_adj += (d.extent - 1) * d.stride;
    for (auto &d : r) d.stride = std::llabs(d.stride);
    std::sort(r.begin(), r.end(), [](const Dim &a, const Dim &b) { return a.stride > b.stride; });
  }
  int64_t ext = 1, st = 1;
  bool have = false;
  for (int i = (int)r.size() - 1; i >= 0; --i) {     // innermost first
    if (!have) {
      ext = r[i].extent;
      st = r[i].stride;
      have = true;
    } else {
      if (r[i].stride != st * ext) return false;
      ext *= r[i].extent;
    }
  }
  if (have && st != 1) return false;
  // Kept dims must be regular: output o starts at start0 + o * seg_stride
  // (seg_stride may be negative: kept dims walked backwards).
  int64_t expect = 0, cum = 1;
  bool have_keep = false;
  for (int i = p.nkeep - 1; i >= 0; --i) {
    const Dim &d = p.keep[i];
    if (d.extent == 1) continue;
    if (!have_keep) {
      expect = d.stride;
      cum = d.extent;
      have_keep = true;
    } else {
      if (d.stride != expect * cum) return false;
      cum *= d.extent;
    }
  }
  *seg_stride = have_keep ? expect : p.n_rest;
  *start0 = p.offset + lo_adj;
  return true;
}

}  // namespace desc

// ----------------------------------------------------------------------------
// desc_check_disjoint
// ----------------------------------------------------------------------------
namespace {

struct Ent {
  int64_t elem;
  int64_t tid;
  int32_t w;
};

bool same_map(const desc_lowered &a, const desc_lowered &b) {
  if (a.ndims != b.ndims || a.nsel != b.nsel || a.offset != b.offset) return false;
  for (int i = 0; i < a.ndims; ++i)
    if (a.extent[i] != b.extent[i] || a.stride[i] != b.stride[i] || a.level[i] != b.level[i] ||
        a.dim[i] != b.dim[i])
      return false;
  return true;
}

// Extent of the execution coordinate a selected dim binds.
int64_t bound_count(const desc_exec &ex, int32_t level, int32_t dim) {
  return resource_count(ex, level, dim);
}

// Threads that share every bound coordinate (the replication of an access),
// or -1 when a bound extent differs from its resource count.
int64_t replication(const desc_lowered &m, const desc_exec &ex) {
  bool bb[3] = {}, bt[3] = {}, warp = false, lane = false;
  for (int i = 0; i < m.nsel; ++i) {
    if (m.extent[i] != bound_count(ex, m.level[i], m.dim[i])) return -1;
    if (m.level[i] == DESC_LEVEL_BLOCK) bb[m.dim[i]] = true;
    else if (m.level[i] == DESC_LEVEL_WARP) warp = true;
    else if (m.dim[i] == DESC_DIM_LANE) lane = true;
    else bt[m.dim[i]] = true;
  }
  int64_t r = 1;
  for (int d = 0; d < 3; ++d)
    if (!bb[d]) r *= ex.grid[d];
  const int64_t nt = ex.block[0] * ex.block[1] * ex.block[2];
  if (warp || lane) {
    if (!warp) r *= nt / 32;
    if (!lane) r *= 32;
  } else {
    for (int d = 0; d < 3; ++d)
      if (!bt[d]) r *= ex.block[d];
  }
  return r;
}

int64_t min_element(const desc_lowered &m) {
  int64_t e = m.offset;
  for (int i = 0; i < m.ndims; ++i)
    if (m.stride[i] < 0 && m.extent[i] > 0) e += (m.extent[i] - 1) * m.stride[i];
  return e;
}

bool empty_domain(const desc_lowered &m) {
  for (int i = 0; i < m.ndims; ++i)
    if (m.extent[i] == 0) return true;
  return false;
}

// Every (element, thread) pair of an access, appended to `out`.  Returns
// false if more than kMaxEnum pairs would be needed.
bool enumerate(const desc_lowered &m, const desc_exec &ex, int32_t w, std::vector<Ent> &out) {
  if (empty_domain(m)) return true;
  const int64_t nb = ex.grid[0] * ex.grid[1] * ex.grid[2];
  const int64_t nt = ex.block[0] * ex.block[1] * ex.block[2];
  int64_t nloc = 1;
  for (int i = m.nsel; i < m.ndims; ++i) nloc *= m.extent[i];
  if (nb * nt > kMaxEnum || nloc > kMaxEnum || nb * nt * nloc + (int64_t)out.size() > kMaxEnum)
    return false;
  std::vector<int64_t> loc(nloc);
  for (int64_t q = 0; q < nloc; ++q) {
    int64_t r = q, e = 0;
    for (int i = m.ndims - 1; i >= m.nsel; --i) {
      e += (r % m.extent[i]) * m.stride[i];
      r /= m.extent[i];
    }
    loc[q] = e;
  }
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t bc[3] = {b % ex.grid[0], (b / ex.grid[0]) % ex.grid[1], b / (ex.grid[0] * ex.grid[1])};
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t tc[3] = {t % ex.block[0], (t / ex.block[0]) % ex.block[1],
                             t / (ex.block[0] * ex.block[1])};
      int64_t e0 = m.offset;
      bool reach = true;
      for (int i = 0; i < m.nsel; ++i) {
        int64_t c;
        if (m.level[i] == DESC_LEVEL_BLOCK) c = bc[m.dim[i]];
        else if (m.level[i] == DESC_LEVEL_WARP) c = t / 32;
        else if (m.dim[i] == DESC_DIM_LANE) c = t % 32;
        else c = tc[m.dim[i]];
        if (c >= m.extent[i]) { reach = false; break; }   // resource beyond the extent
        e0 += c * m.stride[i];
      }
      if (!reach) continue;
      const int64_t tid = b * nt + t;
      for (int64_t q = 0; q < nloc; ++q) out.push_back({e0 + loc[q], tid, w});
    }
  }
  return true;
}

}  // namespace

extern "C" int32_t desc_check_disjoint_ex(const desc_access *acc, int32_t n, const desc_exec *ex,
                                          int64_t *first_conflict, int32_t *method) {
  if (method) *method = 0;
  if (n < 0 || (n > 0 && !acc) || !ex) return DESC_ERR_INVALID_ARG;
  if (!exec_ok(*ex)) return DESC_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const desc_lowered &m = acc[i].map;
    if (m.ndims < 0 || m.ndims > DESC_MAX_DIMS || m.nsel < 0 || m.nsel > m.ndims)
      return DESC_ERR_INVALID_ARG;
    for (int j = 0; j < m.ndims; ++j) {
      if (m.extent[j] < 0) return DESC_ERR_INVALID_ARG;
      if (j < m.nsel) {
        const int32_t l = m.level[j], d = m.dim[j];
        const bool ok = (l == DESC_LEVEL_BLOCK && d >= 0 && d < 3) ||
                        (l == DESC_LEVEL_WARP && d == DESC_DIM_X) ||
                        (l == DESC_LEVEL_THREAD && d >= 0 && d <= DESC_DIM_LANE);
        if (!ok) return DESC_ERR_INVALID_ARG;
      }
    }
  }
  std::vector<int32_t> bufs;
  for (int i = 0; i < n; ++i) bufs.push_back(acc[i].buffer);
  std::sort(bufs.begin(), bufs.end());
  bufs.erase(std::unique(bufs.begin(), bufs.end()), bufs.end());

  bool found = false;
  int64_t worst = 0;
  int32_t how = 0;
  auto report = [&](int64_t e) {
    if (!found || e < worst) worst = e;
    found = true;
  };
  for (int32_t b : bufs) {
    std::vector<const desc_access *> W, R;
    for (int i = 0; i < n; ++i)
      if (acc[i].buffer == b) (acc[i].is_write ? W : R).push_back(&acc[i]);
    if (W.empty()) continue;
    // Structural path: one write map, reads (if any) through the same map.
    bool structural = W.size() == 1;
    for (auto *r : R) structural = structural && same_map(r->map, W[0]->map);
    if (structural) {
      const desc_lowered &m = W[0]->map;
      if (empty_domain(m)) continue;
      const int64_t rep = replication(m, *ex);
      if (rep > 1) {            // several threads write every element
        report(min_element(m));
        how |= DESC_DECIDED_STRUCTURAL;
        continue;
      }
      if (rep == 1 && desc::affine_injective(m.extent, m.stride, m.ndims)) {
        how |= DESC_DECIDED_STRUCTURAL;
        continue;
      }
    }
    how |= DESC_DECIDED_ENUMERATION;
    std::vector<Ent> ents;
    for (auto *a : W)
      if (!enumerate(a->map, *ex, 1, ents)) return DESC_ERR_UNSUPPORTED;
    for (auto *a : R)
      if (!enumerate(a->map, *ex, 0, ents)) return DESC_ERR_UNSUPPORTED;
    std::sort(ents.begin(), ents.end(), [](const Ent &x, const Ent &y) {
      return x.elem != y.elem ? x.elem < y.elem : (x.tid != y.tid ? x.tid < y.tid : x.w > y.w);
    });
    for (size_t i = 0; i < ents.size();) {
      size_t j = i;
      int64_t writer = -1;
      bool bad = false;
      while (j < ents.size() && ents[j].elem == ents[i].elem) {
        if (ents[j].w) {
          if (writer >= 0 && writer != ents[j].tid) bad = true;
          writer = ents[j].tid;
        }
        ++j;
      }
      if (!bad && writer >= 0)
        for (size_t q = i; q < j; ++q)
          if (!ents[q].w && ents[q].tid != writer) bad = true;
      if (bad) {
        report(ents[i].elem);
        break;          // elements are sorted: the first bad one is the smallest
      }
      i = j;
    }
  }
  if (method) *method = how;
  if (found) {
    if (first_conflict) *first_conflict = worst;
    return DESC_ERR_OVERLAP;
  }
  return DESC_OK;
}

extern "C" int32_t desc_check_disjoint(const desc_access *acc, int32_t n, const desc_exec *ex,
                                       int64_t *first_conflict) {
  return desc_check_disjoint_ex(acc, n, ex, first_conflict, nullptr);
}

namespace desc {
bool injective_quick(const desc_lowered &w) { return affine_injective(w.extent, w.stride, w.ndims); }
bool same_map_quick(const desc_lowered &a, const desc_lowered &b) { return same_map(a, b); }
}  // namespace desc
