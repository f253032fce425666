// Host BVH builder interface.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace ccs {

struct BvhHost {
    std::vector<float> nodes;        // 16 floats per binary node, 32 per 4-wide node (layouts of ccs_internal.h)
    std::vector<int> leaf_parent;    // per patch: (node << 1) | slot, or (node << 2) | slot when 4-wide
    int max_depth = 0;
};

bool build_bvh(const std::vector<float> &leaf_lo, const std::vector<float> &leaf_hi, uint32_t n, int bins,
               BvhHost &out, std::string &err);

// Collapse a binary BVH into a 4-wide one: each node keeps up to four subtrees, opening the child of
// largest surface area while fewer than four are present.  Leaves and their boxes are unchanged.
bool collapse_bvh4(const BvhHost &bin, uint32_t n, BvhHost &out, std::string &err);

}  // namespace ccs
