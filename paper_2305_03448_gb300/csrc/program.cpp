// desc_check_program: access safety across a whole kernel body.
//
// Section 3.3 (narrowing, synchronization) and Section 4
// (access_safety_check) keep an access environment that maps execution
// resources to the places they accessed; a barrier removes the entries of
// the threads it synchronises.  Section 2.2 rejects a barrier that not every
// thread of its scope reaches (a sync inside a split of the block's threads).
//
// The body is a flattened statement tree (ACCESS, SYNC, SPLIT).  Every
// access is enumerated exactly: for each thread of the current sub-resource,
// the elements it reaches.  Each (buffer, element) keeps the list of earlier
// (thread, read/write, barrier counts) entries; a new entry conflicts with an
// earlier one from another thread when one of the two writes and neither a
// block barrier of their common block nor a warp barrier of their common
// warp has been passed since the earlier entry.  A grid-level sync (a kernel
// boundary) clears the environment.
#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "desc_internal.h"

namespace {

constexpr int64_t kMaxPairs = int64_t(1) << 22;

// A sub-resource: a box of blocks, and within each block either a box of
// threads or a range of warps.
struct Sub {
  int64_t blo[3], bhi[3];
  int64_t tlo[3], thi[3];
  int64_t wlo, whi;
  bool thread_split, warp_split, in_split;
};

struct Entry {
  int64_t tid;
  uint32_t bs, ws;     // barrier counts of the thread's block and warp at the access
  uint8_t w;
};

struct Key {
  int32_t buf;
  int64_t elem;
  bool operator==(const Key &o) const { return buf == o.buf && elem == o.elem; }
};
struct KeyHash {
  size_t operator()(const Key &k) const {
    uint64_t x = uint64_t(k.elem) * 0x9E3779B97F4A7C15ull ^ uint64_t(uint32_t(k.buf)) * 0xC2B2AE3D27D4EB4Full;
    return size_t(x ^ (x >> 29));
  }
};

struct Checker {
  desc_exec ex;
  int64_t nb = 0, nt = 0, nw = 0;
  std::vector<uint32_t> bsync, wsync;
  std::unordered_map<Key, std::vector<Entry>, KeyHash> env;
  int64_t pairs = 0;
  int32_t bad_stmt = -1;
  int64_t bad_elem = 0;

  uint32_t warp_count(int64_t tid) const { return wsync[size_t((tid / nt) * nw + (tid % nt) / 32)]; }

  // Count of the sub-resource along a select (level, dim), or -1 when that
  // coordinate is not defined there.
  int64_t count(const Sub &s, int32_t level, int32_t dim) const {
    if (level == DESC_LEVEL_BLOCK) return s.bhi[dim] - s.blo[dim];
    if (level == DESC_LEVEL_WARP) {
      if (s.thread_split) return -1;
      return s.warp_split ? s.whi - s.wlo : nt / 32;
    }
    if (dim == DESC_DIM_LANE) return s.thread_split ? -1 : 32;
    if (s.warp_split) return -1;
    return s.thi[dim] - s.tlo[dim];
  }

  int32_t access(const desc_access &a, const Sub &s, int32_t index) {
    const desc_lowered &m = a.map;
    if (m.ndims < 0 || m.ndims > DESC_MAX_DIMS || m.nsel < 0 || m.nsel > m.ndims) return DESC_ERR_INVALID_ARG;
    bool empty = false;
    for (int i = 0; i < m.ndims; ++i) {
      if (m.extent[i] < 0) return DESC_ERR_INVALID_ARG;
      empty = empty || m.extent[i] == 0;
      if (i < m.nsel) {
        const int32_t l = m.level[i], d = m.dim[i];
        const bool ok = (l == DESC_LEVEL_BLOCK && d >= 0 && d < 3) || (l == DESC_LEVEL_WARP && d == DESC_DIM_X) ||
                        (l == DESC_LEVEL_THREAD && d >= 0 && d <= DESC_DIM_LANE);
        if (!ok) return DESC_ERR_INVALID_ARG;
        if (m.extent[i] != count(s, l, d)) {
          bad_stmt = index;
          return DESC_ERR_SHAPE;
        }
      }
    }
    if (empty) return DESC_OK;
    int64_t nloc = 1;
    for (int i = m.nsel; i < m.ndims; ++i) nloc *= m.extent[i];
    if (nloc > kMaxPairs) return DESC_ERR_UNSUPPORTED;
    std::vector<int64_t> loc(static_cast<size_t>(nloc));
    for (int64_t q = 0; q < nloc; ++q) {
      int64_t r = q, e = 0;
      for (int i = m.ndims - 1; i >= m.nsel; --i) {
        e += (r % m.extent[i]) * m.stride[i];
        r /= m.extent[i];
      }
      loc[size_t(q)] = e;
    }
    bool conflict = false;
    int64_t worst = 0;
    for (int64_t bz = s.blo[2]; bz < s.bhi[2]; ++bz)
      for (int64_t by = s.blo[1]; by < s.bhi[1]; ++by)
        for (int64_t bx = s.blo[0]; bx < s.bhi[0]; ++bx) {
          const int64_t bc[3] = {bx - s.blo[0], by - s.blo[1], bz - s.blo[2]};
          const int64_t b = bx + ex.grid[0] * (by + ex.grid[1] * bz);
          for (int64_t t = 0; t < nt; ++t) {
            const int64_t tc[3] = {t % ex.block[0], (t / ex.block[0]) % ex.block[1], t / (ex.block[0] * ex.block[1])};
            bool in = true;
            if (s.warp_split) {
              in = t / 32 >= s.wlo && t / 32 < s.whi;
            } else {
              for (int d = 0; d < 3; ++d) in = in && tc[d] >= s.tlo[d] && tc[d] < s.thi[d];
            }
            if (!in) continue;
            int64_t e0 = m.offset;
            bool reach = true;
            for (int i = 0; i < m.nsel && reach; ++i) {
              int64_t c;
              const int32_t l = m.level[i], d = m.dim[i];
              if (l == DESC_LEVEL_BLOCK) c = bc[d];
              else if (l == DESC_LEVEL_WARP) c = t / 32 - (s.warp_split ? s.wlo : 0);
              else if (d == DESC_DIM_LANE) c = t % 32;
              else c = tc[d] - s.tlo[d];
              if (c >= m.extent[i]) reach = false;   // resource beyond the extent
              e0 += c * m.stride[i];
            }
            if (!reach) continue;
            const int64_t tid = b * nt + t;
            for (int64_t q = 0; q < nloc; ++q) {
              if (++pairs > kMaxPairs) return DESC_ERR_UNSUPPORTED;
              const Key k{a.buffer, e0 + loc[size_t(q)]};
              std::vector<Entry> &list = env[k];
              for (const Entry &h : list) {
                if (h.tid == tid || !(h.w || a.is_write)) continue;
                const bool same_block = h.tid / nt == b;
                if (same_block && bsync[size_t(b)] > h.bs) continue;          // a block barrier since
                if (same_block && (h.tid % nt) / 32 == t / 32 && warp_count(tid) > h.ws) continue;
                if (!conflict || k.elem < worst) worst = k.elem;
                conflict = true;
                break;
              }
              list.push_back({tid, bsync[size_t(b)], warp_count(tid), uint8_t(a.is_write ? 1 : 0)});
            }
          }
        }
    if (conflict) {
      bad_stmt = index;
      bad_elem = worst;
      return DESC_ERR_OVERLAP;
    }
    return DESC_OK;
  }

  int32_t sync(const desc_stmt &st, const Sub &s, int32_t index) {
    if (st.level == DESC_LEVEL_GRID) {
      if (s.in_split) {
        bad_stmt = index;
        return DESC_ERR_BARRIER;
      }
      env.clear();
      pairs = 0;
      return DESC_OK;
    }
    if (st.level == DESC_LEVEL_BLOCK) {
      if (s.thread_split || s.warp_split) {
        bad_stmt = index;
        return DESC_ERR_BARRIER;
      }
      for (int64_t bz = s.blo[2]; bz < s.bhi[2]; ++bz)
        for (int64_t by = s.blo[1]; by < s.bhi[1]; ++by)
          for (int64_t bx = s.blo[0]; bx < s.bhi[0]; ++bx) ++bsync[size_t(bx + ex.grid[0] * (by + ex.grid[1] * bz))];
      return DESC_OK;
    }
    if (st.level == DESC_LEVEL_WARP) {
      if (s.thread_split || nt % 32 != 0) {
        bad_stmt = index;
        return DESC_ERR_BARRIER;
      }
      const int64_t w0 = s.warp_split ? s.wlo : 0, w1 = s.warp_split ? s.whi : nw;
      for (int64_t bz = s.blo[2]; bz < s.bhi[2]; ++bz)
        for (int64_t by = s.blo[1]; by < s.bhi[1]; ++by)
          for (int64_t bx = s.blo[0]; bx < s.bhi[0]; ++bx) {
            const int64_t b = bx + ex.grid[0] * (by + ex.grid[1] * bz);
            for (int64_t w = w0; w < w1; ++w) ++wsync[size_t(b * nw + w)];
          }
      return DESC_OK;
    }
    return DESC_ERR_INVALID_ARG;
  }

  // Statements [i0, i1) on sub-resource s.
  int32_t run(const desc_stmt *p, int32_t i0, int32_t i1, const Sub &s) {
    for (int32_t i = i0; i < i1;) {
      const desc_stmt &st = p[i];
      int32_t r = DESC_OK;
      if (st.kind == DESC_STMT_ACCESS) {
        r = access(st.access, s, i);
        ++i;
      } else if (st.kind == DESC_STMT_SYNC) {
        r = sync(st, s, i);
        ++i;
      } else if (st.kind == DESC_STMT_SPLIT) {
        if (st.n_first < 0 || st.n_second < 0 || int64_t(i) + 1 + st.n_first + st.n_second > i1)
          return DESC_ERR_INVALID_ARG;
        Sub a = s, b = s;
        a.in_split = b.in_split = true;
        const int32_t d = st.dim;
        if (st.level == DESC_LEVEL_BLOCK || st.level == DESC_LEVEL_THREAD) {
          if (d < 0 || d > 2) return DESC_ERR_INVALID_ARG;
          if (st.level == DESC_LEVEL_THREAD && s.warp_split) {
            bad_stmt = i;
            return DESC_ERR_SHAPE;
          }
          int64_t *lo_a = st.level == DESC_LEVEL_BLOCK ? a.blo : a.tlo, *hi_a = st.level == DESC_LEVEL_BLOCK ? a.bhi : a.thi;
          int64_t *lo_b = st.level == DESC_LEVEL_BLOCK ? b.blo : b.tlo;
          const int64_t lo = lo_a[d], hi = hi_a[d];
          if (st.at <= 0 || st.at >= hi - lo) {
            bad_stmt = i;
            return DESC_ERR_SHAPE;
          }
          hi_a[d] = lo + st.at;
          lo_b[d] = lo + st.at;
          if (st.level == DESC_LEVEL_THREAD) a.thread_split = b.thread_split = true;
        } else if (st.level == DESC_LEVEL_WARP) {
          if (d != DESC_DIM_X) return DESC_ERR_INVALID_ARG;
          if (s.thread_split || nt % 32 != 0) {
            bad_stmt = i;
            return DESC_ERR_SHAPE;
          }
          const int64_t lo = s.warp_split ? s.wlo : 0, hi = s.warp_split ? s.whi : nw;
          if (st.at <= 0 || st.at >= hi - lo) {
            bad_stmt = i;
            return DESC_ERR_SHAPE;
          }
          a.warp_split = b.warp_split = true;
          a.wlo = lo;
          a.whi = lo + st.at;
          b.wlo = lo + st.at;
          b.whi = hi;
        } else {
          return DESC_ERR_INVALID_ARG;
        }
        const int32_t f0 = i + 1, f1 = f0 + st.n_first, s1 = f1 + st.n_second;
        if ((r = run(p, f0, f1, a)) != DESC_OK) return r;
        if ((r = run(p, f1, s1, b)) != DESC_OK) return r;
        i = s1;
      } else {
        return DESC_ERR_INVALID_ARG;
      }
      if (r != DESC_OK) return r;
    }
    return DESC_OK;
  }
};

}  // namespace

extern "C" int32_t desc_check_program(const desc_stmt *prog, int32_t n, const desc_exec *ex, int32_t *bad_stmt,
                                      int64_t *first_conflict) {
  if (n < 0 || (n > 0 && !prog) || !ex) return DESC_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (ex->grid[d] < 1 || ex->block[d] < 1 || ex->block[d] > 4096 || ex->grid[d] > (int64_t(1) << 31))
      return DESC_ERR_INVALID_ARG;
  Checker c;
  c.ex = *ex;
  c.nb = ex->grid[0] * ex->grid[1] * ex->grid[2];
  c.nt = ex->block[0] * ex->block[1] * ex->block[2];
  c.nw = (c.nt + 31) / 32;
  if (c.nb * c.nt > kMaxPairs) return DESC_ERR_UNSUPPORTED;
  c.bsync.assign(size_t(c.nb), 0u);
  c.wsync.assign(size_t(c.nb * c.nw), 0u);
  Sub all{};
  for (int d = 0; d < 3; ++d) {
    all.blo[d] = 0;
    all.bhi[d] = ex->grid[d];
    all.tlo[d] = 0;
    all.thi[d] = ex->block[d];
  }
  all.wlo = 0;
  all.whi = c.nw;
  const int32_t r = c.run(prog, 0, n, all);
  if (bad_stmt) *bad_stmt = c.bad_stmt;
  if (r == DESC_ERR_OVERLAP && first_conflict) *first_conflict = c.bad_elem;
  return r;
}
