// Host BVH builder interface.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace ccs {

struct BvhHost {
    std::vector<float> nodes;        // 16 floats per node (layout of ccs_internal.h)
    std::vector<int> leaf_parent;    // per patch: (node << 1) | slot
    int max_depth = 0;
};

bool build_bvh(const std::vector<float> &leaf_lo, const std::vector<float> &leaf_hi, uint32_t n, int bins,
               BvhHost &out, std::string &err);

}  // namespace ccs
