// regrid.cpp -- host side of regridding: marking and 2:1 balance of the new
// octree, and the new block list with the transfer map.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- the Grid unit owns the
// (PARAMESH-style) octree and its refinement.  Rules: a leaf whose indicator
// exceeds the refine cutoff is split (below the maximum level); a parent
// whose children are all leaves under the derefine cutoff (none split) is
// coarsened; then, until nothing changes, of any two touching leaf regions
// (faces, edges, corners; periodic axes wrap) whose new levels differ by two
// or more the coarser is split, or its coarsening cancelled.
//
// Balance is enforced on the adjacency of the current leaves: two new leaf
// regions touch exactly when the current leaves they come from touch, so it
// suffices that touching current leaves b, c satisfy |t(b) - t(c)| <= 1 for
// the new level t of the region holding each.
#include "fx_internal.h"

#include <algorithm>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace fx {

namespace {

// (level, block x, y, z) packed into 64 bits: 6 bits of level, 19 per axis.
constexpr int kAxisBits = 19;
uint64_t key(int level, long long x, long long y, long long z) {
  return ((uint64_t)level << (3 * kAxisBits)) | ((uint64_t)z << (2 * kAxisBits)) |
         ((uint64_t)y << kAxisBits) | (uint64_t)x;
}
using Where = std::unordered_map<uint64_t, int>;

}  // namespace

int regrid_plan(int ndim, int nxb, const int nroot[3], const int bc[6], int nb,
                const std::vector<int> &level, const std::vector<int> &origin,
                const std::vector<int> &parent, const std::vector<double> &err, double rc,
                double dc, int max_level, RegridPlan *out, std::string *msg) {
  const int nch = 1 << ndim;
  // block indices at the finest level present or planned must fit the key
  int lcap = max_level + 1;
  for (int b = 0; b < nb; ++b) lcap = std::max(lcap, level[b]);
  for (int d = 0; d < 3; ++d)
    if (((long long)nroot[d] << lcap) > (1LL << kAxisBits)) {
      *msg = "regrid: block lattice too large";
      return FX_ERR_ARG;
    }
  std::vector<int> leaf(nb, 1), child(8 * (size_t)nb, -1);
  Where where;
  where.reserve(2 * (size_t)nb);
  for (int b = 0; b < nb; ++b)
    where[key(level[b], origin[3 * b] / nxb, origin[3 * b + 1] / nxb, origin[3 * b + 2] / nxb)] = b;
  for (int b = 0; b < nb; ++b) {
    const int p = parent[b];
    if (p < 0) continue;
    leaf[p] = 0;
    int oct = 0;
    for (int d = 0; d < ndim; ++d)
      if (origin[3 * b + d] != 2 * origin[3 * p + d]) oct |= 1 << d;
    child[8 * p + oct] = b;
  }
  // ---- touching leaves of every leaf
  std::vector<std::vector<int>> nbr(nb);
  std::vector<int> found;
  for (int b = 0; b < nb; ++b) {
    if (!leaf[b]) continue;
    const int L = level[b];
    long long B[3] = {origin[3 * b] / nxb, origin[3 * b + 1] / nxb, origin[3 * b + 2] / nxb};
    found.clear();
    for (int sz = (ndim == 3 ? -1 : 0); sz <= (ndim == 3 ? 1 : 0); ++sz)
      for (int sy = -1; sy <= 1; ++sy)
        for (int sx = -1; sx <= 1; ++sx) {
          const int s[3] = {sx, sy, sz};
          if (!sx && !sy && !sz) continue;
          long long Q[3];
          bool outside = false;
          for (int d = 0; d < 3; ++d) {
            Q[d] = B[d] + s[d];
            if (d >= ndim) continue;
            const long long N = (long long)nroot[d] << L;
            if (Q[d] < 0 || Q[d] >= N) {
              if (bc[2 * d] == FX_BC_PERIODIC) Q[d] = (Q[d] + N) % N;
              else outside = true;
            }
          }
          if (outside) continue;
          auto it = where.find(key(L, Q[0], Q[1], Q[2]));
          if (it != where.end()) {
            const int q = it->second;
            if (leaf[q]) { found.push_back(q); continue; }
            for (int oct = 0; oct < nch; ++oct) {   // children of q on b's side
              bool touches = true;
              for (int d = 0; d < ndim; ++d) {
                const int bit = (oct >> d) & 1;
                if ((s[d] > 0 && bit) || (s[d] < 0 && !bit)) touches = false;
              }
              const int c = child[8 * q + oct];
              if (!touches) continue;
              if (c < 0 || !leaf[c]) { *msg = "regrid: mesh not 2:1 balanced"; return FX_ERR_MESH; }
              found.push_back(c);
            }
          } else {
            if (L == 0) { *msg = "regrid: mesh does not cover the domain"; return FX_ERR_MESH; }
            auto up = where.find(key(L - 1, Q[0] >> 1, Q[1] >> 1, ndim == 3 ? Q[2] >> 1 : 0));
            if (up == where.end() || !leaf[up->second]) {
              *msg = "regrid: mesh not 2:1 balanced";
              return FX_ERR_MESH;
            }
            found.push_back(up->second);
          }
        }
    std::sort(found.begin(), found.end());
    found.erase(std::unique(found.begin(), found.end()), found.end());
    nbr[b].assign(found.begin(), found.end());
  }
  // ---- requests
  std::vector<char> split(nb, 0), merge(nb, 0);
  for (int b = 0; b < nb; ++b)
    if (leaf[b] && err[b] > rc && level[b] < max_level) split[b] = 1;
  for (int p = 0; p < nb; ++p) {
    if (leaf[p]) continue;
    bool all = true;
    for (int oct = 0; oct < nch; ++oct) {
      const int c = child[8 * p + oct];
      all = all && c >= 0 && leaf[c] && err[c] < dc && !split[c];
    }
    merge[p] = all;
  }
  auto target = [&](int b) {
    const int p = parent[b];
    if (p >= 0 && merge[p]) return level[p];
    return level[b] + split[b];
  };
  // ---- balance
  for (bool changed = true; changed;) {
    changed = false;
    for (int b = 0; b < nb; ++b) {
      if (!leaf[b]) continue;
      for (int c : nbr[b]) {
        if (target(c) <= target(b) + 1) continue;
        const int p = parent[b];
        if (p >= 0 && merge[p]) merge[p] = 0;
        else if (!split[b]) split[b] = 1;
        else { *msg = "regrid: balance cannot be restored"; return FX_ERR_MESH; }
        changed = true;
        break;
      }
    }
  }
  // ---- the new block list, sorted by (level, z, y, x)
  struct Entry {
    int level;
    long long o[3];
    int kind, src, oct;
  };
  std::vector<Entry> e;
  for (int b = 0; b < nb; ++b) {
    if (parent[b] >= 0 && merge[parent[b]]) continue;
    e.push_back({level[b], {origin[3 * b], origin[3 * b + 1], origin[3 * b + 2]}, 0, b, 0});
    if (leaf[b] && split[b])
      for (int oct = 0; oct < nch; ++oct) {
        Entry c{level[b] + 1, {0, 0, 0}, 1, b, oct};
        for (int d = 0; d < ndim; ++d)
          c.o[d] = 2LL * origin[3 * b + d] + (((oct >> d) & 1) ? nxb : 0);
        e.push_back(c);
      }
  }
  std::sort(e.begin(), e.end(), [](const Entry &a, const Entry &b) {
    if (a.level != b.level) return a.level < b.level;
    if (a.o[2] != b.o[2]) return a.o[2] < b.o[2];
    if (a.o[1] != b.o[1]) return a.o[1] < b.o[1];
    return a.o[0] < b.o[0];
  });
  const int nn = (int)e.size();
  Where at;
  at.reserve(2 * (size_t)nn);
  for (int j = 0; j < nn; ++j)
    at[key(e[j].level, e[j].o[0] / nxb, e[j].o[1] / nxb, e[j].o[2] / nxb)] = j;
  out->level.resize(nn);
  out->origin.resize(3 * (size_t)nn);
  out->parent.resize(nn);
  out->map.resize(nn);
  for (int j = 0; j < nn; ++j) {
    out->level[j] = e[j].level;
    for (int d = 0; d < 3; ++d) out->origin[3 * j + d] = e[j].o[d];
    out->map[j] = make_int4(e[j].kind, e[j].src, e[j].oct, 0);
    out->parent[j] = -1;
    if (e[j].level > 0) {
      auto it = at.find(key(e[j].level - 1, (e[j].o[0] / nxb) >> 1, (e[j].o[1] / nxb) >> 1,
                            ndim == 3 ? (e[j].o[2] / nxb) >> 1 : 0));
      if (it == at.end()) { *msg = "regrid: block without parent"; return FX_ERR_MESH; }
      out->parent[j] = it->second;
    }
  }
  return FX_OK;
}

}  // namespace fx
