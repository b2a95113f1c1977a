// Host-side tree planning: validation, interaction lists, grouping by operator.
#pragma once

#include <cstdint>
#include <vector>

namespace vp {

struct Box {
  int level, ix, iy;
  int parent;  // -1 for the root
  int child0;  // first of 4 consecutive children, -1 for a leaf
  int leaf;    // index into the caller's leaf list, -1 for an internal box
};

// One interaction (target, source, relative-position index).
struct Pair {
  int tgt, src, pos;
};

struct TreePlan {
  std::vector<Box> boxes;        // breadth first: levels ascending, siblings consecutive
  std::vector<int> leaf_box;     // caller leaf index -> box index
  int max_level = 0;
  // lists (box indices)
  std::vector<Pair> U;  // target leaf box, source leaf box, near position (0..32)
  std::vector<Pair> V;  // target box, source box (same level), offset (0..39)
  std::vector<Pair> W;  // target leaf box (level l), source box (level l+1), W position (0..19)
  std::vector<Pair> X;  // target box (level l), source leaf box (level l-1), X position (0..19)
};

// Returns VP_OK or VP_ERR_ARG / VP_ERR_TREE / VP_ERR_TREE_UNBALANCED / VP_ERR_LEVELS.
int build_plan(int n_leaves, const int32_t* level, const int32_t* ix, const int32_t* iy, int max_allowed_level,
               TreePlan& out);

}  // namespace vp
