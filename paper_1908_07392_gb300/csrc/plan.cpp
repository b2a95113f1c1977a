// Tree validation and adaptive FMM interaction lists on the level-restricted
// quadtree (Sec. 3.2.1, "Tree structure": boxes split into four children,
// adjacent leaves within one level of each other).
//
// Lists, for a box b at level l (standard adaptive-FMM definitions, reduced by
// the level restriction):
//   U(b), b a leaf: leaves adjacent to b (levels l-1, l, l+1) and b itself;
//   V(b), l >= 2:   children of the colleagues of b's parent that are not
//                   adjacent to b (same level, offsets in [-3,3]^2 \ [-1,1]^2);
//   W(b), b a leaf: children of b's non-leaf colleagues not adjacent to b;
//   X(b):           leaves at level l-1 adjacent to b's parent but not to b
//                   (the dual of W).
// Every pair (target leaf, source leaf) is covered exactly once by U(t),
// W(t), X(a) or V(a) for a an ancestor-or-self of t (with the sources being
// the leaves under the listed box).
#include "plan.h"

#include <unordered_map>
#include <unordered_set>

#include "vp_internal.h"

namespace vp {

namespace {
inline uint64_t key(int l, int x, int y) {
  return ((uint64_t)(uint32_t)l << 50) | ((uint64_t)(uint32_t)x << 25) | (uint64_t)(uint32_t)y;
}
}  // namespace

int build_plan(int n_leaves, const int32_t* level, const int32_t* ix, const int32_t* iy, int max_allowed_level,
               TreePlan& out) {
  out = TreePlan();
  if (n_leaves < 1 || !level || !ix || !iy) return VP_ERR_ARG;
  std::unordered_map<uint64_t, int> leafmap;
  leafmap.reserve(n_leaves * 2);
  int maxl = 0;
  for (int k = 0; k < n_leaves; ++k) {
    const int l = level[k];
    if (l < 0 || l > 24) return VP_ERR_ARG;
    const int64_t lim = (int64_t)1 << l;
    if (ix[k] < 0 || iy[k] < 0 || ix[k] >= lim || iy[k] >= lim) return VP_ERR_TREE;
    if (!leafmap.emplace(key(l, ix[k], iy[k]), k).second) return VP_ERR_TREE;
    maxl = std::max(maxl, l);
  }
  if (maxl > max_allowed_level) return VP_ERR_LEVELS;
  // internal boxes = strict ancestors of leaves; an ancestor that is a leaf means overlap
  std::unordered_set<uint64_t> internal;
  internal.reserve(n_leaves * 2);
  for (int k = 0; k < n_leaves; ++k) {
    int l = level[k], x = ix[k], y = iy[k];
    while (l > 0) {
      --l; x >>= 1; y >>= 1;
      const uint64_t kk = key(l, x, y);
      if (leafmap.count(kk)) return VP_ERR_TREE;
      if (!internal.insert(kk).second) break;
    }
  }
  // breadth-first numbering from the root; every internal box needs all four children
  std::vector<Box>& B = out.boxes;
  std::unordered_map<uint64_t, int> boxmap;
  boxmap.reserve((n_leaves + internal.size()) * 2);
  {
    const uint64_t rk = key(0, 0, 0);
    const auto lf = leafmap.find(rk);
    if (lf == leafmap.end() && !internal.count(rk)) return VP_ERR_TREE;
    B.push_back({0, 0, 0, -1, -1, lf == leafmap.end() ? -1 : lf->second});
    boxmap[rk] = 0;
  }
  for (size_t i = 0; i < B.size(); ++i) {
    if (B[i].leaf >= 0) continue;
    const int l = B[i].level + 1;
    B[i].child0 = (int)B.size();
    for (int q = 0; q < 4; ++q) {
      const int x = 2 * B[i].ix + (q & 1), y = 2 * B[i].iy + (q >> 1);
      const uint64_t kk = key(l, x, y);
      const auto lf = leafmap.find(kk);
      int leaf = -1;
      if (lf != leafmap.end()) leaf = lf->second;
      else if (!internal.count(kk)) return VP_ERR_TREE;  // gap
      boxmap[kk] = (int)B.size();
      B.push_back({l, x, y, (int)i, -1, leaf});
    }
  }
  out.leaf_box.assign(n_leaves, -1);
  for (size_t i = 0; i < B.size(); ++i)
    if (B[i].leaf >= 0) out.leaf_box[B[i].leaf] = (int)i;
  out.max_level = maxl;

  auto find = [&](int l, int x, int y) -> int {
    if (l < 0) return -1;
    const int64_t lim = (int64_t)1 << l;
    if (x < 0 || y < 0 || x >= lim || y >= lim) return -1;
    const auto it = boxmap.find(key(l, x, y));
    return it == boxmap.end() ? -1 : it->second;
  };
  const Positions& P = positions();

  // level restriction: no non-leaf box of level l+1 may touch a leaf of level l
  for (size_t i = 0; i < B.size(); ++i) {
    const Box& b = B[i];
    if (b.leaf < 0) continue;
    for (int Y = -1; Y <= 2; ++Y)
      for (int X = -1; X <= 2; ++X) {
        if (P.near_fine[Y + 1][X + 1] < 0) continue;
        const int j = find(b.level + 1, 2 * b.ix + X, 2 * b.iy + Y);
        if (j >= 0 && B[j].leaf < 0) return VP_ERR_TREE_UNBALANCED;
      }
  }

  for (size_t i = 0; i < B.size(); ++i) {
    const Box& b = B[i];
    const int l = b.level;
    if (b.leaf >= 0) {
      // U list
      out.U.push_back({(int)i, (int)i, P.near_same[1][1]});
      int coarse_seen[8];
      int n_coarse = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy) continue;
          const int64_t lim = (int64_t)1 << l;
          const int nx = b.ix + dx, ny = b.iy + dy;
          if (nx < 0 || ny < 0 || nx >= lim || ny >= lim) continue;
          const int j = find(l, nx, ny);
          if (j >= 0) {
            if (B[j].leaf >= 0) {
              out.U.push_back({(int)i, j, P.near_same[dy + 1][dx + 1]});
            } else {
              for (int q = 0; q < 4; ++q) {
                const int c = B[j].child0 + q;
                const int X = B[c].ix - 2 * b.ix, Y = B[c].iy - 2 * b.iy;
                if (X >= -1 && X <= 2 && Y >= -1 && Y <= 2) {
                  const int pos = P.near_fine[Y + 1][X + 1];
                  if (pos >= 0) {
                    if (B[c].leaf < 0) return VP_ERR_TREE_UNBALANCED;
                    out.U.push_back({(int)i, c, pos});
                  }
                } else {
                  const int wp = P.w_idx[Y + 2][X + 2];
                  if (wp >= 0) out.W.push_back({(int)i, c, wp});
                }
              }
            }
          } else {
            const int c = find(l - 1, nx >> 1, ny >> 1);
            if (c < 0 || B[c].leaf < 0) return VP_ERR_TREE_UNBALANCED;
            bool seen = false;
            for (int s = 0; s < n_coarse; ++s) seen |= (coarse_seen[s] == c);
            if (seen) continue;
            coarse_seen[n_coarse++] = c;
            const int X = 2 * B[c].ix - b.ix, Y = 2 * B[c].iy - b.iy;
            const int pos = (X >= -2 && X <= 1 && Y >= -2 && Y <= 1) ? P.near_coarse[Y + 2][X + 2] : -1;
            if (pos < 0) return VP_ERR_TREE;
            out.U.push_back({(int)i, c, pos});
          }
        }
    }
    if (l >= 2) {
      const Box& par = B[b.parent];
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int j = find(l - 1, par.ix + dx, par.iy + dy);
          if (j < 0) continue;
          if (B[j].leaf < 0) {
            // V list: children of the parent's colleagues, not adjacent
            for (int q = 0; q < 4; ++q) {
              const int c = B[j].child0 + q;
              const int ox = B[c].ix - b.ix, oy = B[c].iy - b.iy;
              if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1) continue;
              out.V.push_back({(int)i, c, P.v_idx[oy + 3][ox + 3]});
            }
          } else {
            // X list: leaf colleagues of the parent, not adjacent to b
            const int X = 2 * B[j].ix - b.ix, Y = 2 * B[j].iy - b.iy;
            if (X >= -3 && X <= 2 && Y >= -3 && Y <= 2) {
              const int xp = P.x_idx[Y + 3][X + 3];
              if (xp >= 0) out.X.push_back({(int)i, j, xp});
            }
          }
        }
    }
  }
  return VP_OK;
}

}  // namespace vp

// Host-only planning export (no GPU needed): the interaction lists of a leaf
// list, expanded to (target leaf, source leaf, mechanism) triples so that the
// coverage of the pair set can be checked. mechanism: 0 = U (near table),
// 1 = V (multipole-to-local), 2 = W (multipole-to-target), 3 = X (source-to-local).
// Call with out arrays NULL to get the count in *n_out.
extern "C" int vp_plan_pairs(int n_leaves, const int32_t* level, const int32_t* ix, const int32_t* iy,
                             int64_t* n_out, int32_t* tgt, int32_t* src, int32_t* mech) {
  if (!n_out) return VP_ERR_ARG;
  vp::TreePlan T;
  const int rc = vp::build_plan(n_leaves, level, ix, iy, 24, T);
  if (rc != VP_OK) return rc;
  const auto& B = T.boxes;
  // leaves under each box
  std::vector<std::vector<int>> under(B.size());
  for (int i = (int)B.size() - 1; i >= 0; --i) {
    if (B[i].leaf >= 0) under[i].push_back(B[i].leaf);
    else
      for (int q = 0; q < 4; ++q) {
        const auto& c = under[B[i].child0 + q];
        under[i].insert(under[i].end(), c.begin(), c.end());
      }
  }
  int64_t cnt = 0;
  auto emit = [&](int t, int s, int m) {
    if (tgt) { tgt[cnt] = t; src[cnt] = s; mech[cnt] = m; }
    ++cnt;
  };
  for (const auto& p : T.U) emit(B[p.tgt].leaf, B[p.src].leaf, 0);
  for (const auto& p : T.V)
    for (int t : under[p.tgt])
      for (int s : under[p.src]) emit(t, s, 1);
  for (const auto& p : T.W)
    for (int s : under[p.src]) emit(B[p.tgt].leaf, s, 2);
  for (const auto& p : T.X)
    for (int t : under[p.tgt]) emit(t, B[p.src].leaf, 3);
  *n_out = cnt;
  return VP_OK;
}
