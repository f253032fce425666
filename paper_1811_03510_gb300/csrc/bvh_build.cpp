// Host binned-SAH build of a binary BVH with one patch per leaf (Sec. 4: "simple binary BVH,
// recursively constructed using bins to split approximately according to the SAH").
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <vector>

#include "bvh_build.h"

namespace ccs {

namespace {

struct Aabb {
    float lo[3], hi[3];
    void reset() {
        for (int k = 0; k < 3; ++k) { lo[k] = FLT_MAX; hi[k] = -FLT_MAX; }
    }
    void grow(const Aabb &b) {
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); }
    }
    float area() const {
        float e[3];
        for (int k = 0; k < 3; ++k) e[k] = std::max(0.0f, hi[k] - lo[k]);
        return 2.0f * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0]);
    }
};

struct Task {
    uint32_t first, count;
    int parent, slot, depth;
};

void set_child(std::vector<float> &nodes, int node, int slot, const Aabb &b, int child)
{
    float *nd = &nodes[(size_t)node * 16];
    for (int a = 0; a < 3; ++a) {   // float4 a = axis a: (c0.lo, c0.hi, c1.lo, c1.hi)
        nd[4 * a + 2 * slot] = b.lo[a];
        nd[4 * a + 2 * slot + 1] = b.hi[a];
    }
    std::memcpy(nd + 12 + slot, &child, 4);
}

}  // namespace

bool build_bvh(const std::vector<float> &leaf_lo, const std::vector<float> &leaf_hi, uint32_t n, int bins,
               BvhHost &out, std::string &err)
{
    out.nodes.clear();
    out.leaf_parent.assign(n, 0);
    out.max_depth = 0;
    if (n == 0) return true;
    std::vector<Aabb> box(n);
    std::vector<float> cen(3 * (size_t)n);
    for (uint32_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            box[i].lo[k] = leaf_lo[3 * (size_t)i + k];
            box[i].hi[k] = leaf_hi[3 * (size_t)i + k];
            cen[3 * (size_t)i + k] = 0.5f * (box[i].lo[k] + box[i].hi[k]);
        }
    }
    std::vector<uint32_t> idx(n);
    for (uint32_t i = 0; i < n; ++i) idx[i] = i;
    const int kEmpty = 0x7FFFFFFF;
    auto new_node = [&](int parent, int slot) {
        const int id = (int)(out.nodes.size() / 16);
        out.nodes.resize(out.nodes.size() + 16, 0.0f);
        float *nd = &out.nodes[(size_t)id * 16];
        std::memcpy(nd + 12, &kEmpty, 4);
        std::memcpy(nd + 13, &kEmpty, 4);
        std::memcpy(nd + 14, &parent, 4);
        std::memcpy(nd + 15, &slot, 4);
        return id;
    };
    if (n == 1) {   // root with a single leaf child
        new_node(-1, 0);
        set_child(out.nodes, 0, 0, box[0], ~0);
        Aabb e;
        e.reset();
        set_child(out.nodes, 0, 1, e, kEmpty);
        out.leaf_parent[0] = (0 << 1) | 0;
        out.max_depth = 1;
        return true;
    }
    std::vector<Task> stack;
    stack.push_back({0, n, -1, 0, 0});
    std::vector<Aabb> bl(bins), br(bins);
    std::vector<uint32_t> cl(bins);
    while (!stack.empty()) {
        Task t = stack.back();
        stack.pop_back();
        const int node = new_node(t.parent, t.slot);
        if (t.parent >= 0) std::memcpy(&out.nodes[(size_t)t.parent * 16 + 12 + t.slot], &node, 4);
        out.max_depth = std::max(out.max_depth, t.depth + 1);
        // centroid bounds
        float clo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, chi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
        for (uint32_t i = t.first; i < t.first + t.count; ++i)
            for (int k = 0; k < 3; ++k) {
                clo[k] = std::min(clo[k], cen[3 * (size_t)idx[i] + k]);
                chi[k] = std::max(chi[k], cen[3 * (size_t)idx[i] + k]);
            }
        int best_axis = -1, best_split = -1;
        float best_cost = FLT_MAX;
        for (int ax = 0; ax < 3; ++ax) {
            const float ext = chi[ax] - clo[ax];
            if (!(ext > 0.0f)) continue;
            std::vector<Aabb> bb(bins);
            std::vector<uint32_t> bc(bins, 0);
            for (auto &b : bb) b.reset();
            const float scale = (float)bins / ext;
            for (uint32_t i = t.first; i < t.first + t.count; ++i) {
                int b = (int)((cen[3 * (size_t)idx[i] + ax] - clo[ax]) * scale);
                b = std::min(std::max(b, 0), bins - 1);
                bb[b].grow(box[idx[i]]);
                bc[b]++;
            }
            Aabb acc;
            acc.reset();
            uint32_t cnt = 0;
            for (int b = 0; b < bins; ++b) {
                acc.grow(bb[b]);
                cnt += bc[b];
                bl[b] = acc;
                cl[b] = cnt;
            }
            acc.reset();
            cnt = 0;
            for (int b = bins - 1; b > 0; --b) {
                acc.grow(bb[b]);
                cnt += bc[b];
                const uint32_t nl = cl[b - 1], nr = cnt;
                if (nl == 0 || nr == 0) continue;
                const float cost = bl[b - 1].area() * nl + acc.area() * nr;
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = ax;
                    best_split = b;
                }
            }
        }
        uint32_t mid;
        if (best_axis < 0) {
            mid = t.first + t.count / 2;   // all centroids coincide: split by index
        } else {
            const float ext = chi[best_axis] - clo[best_axis];
            const float scale = (float)bins / ext;
            auto it = std::partition(idx.begin() + t.first, idx.begin() + t.first + t.count, [&](uint32_t p) {
                int b = (int)((cen[3 * (size_t)p + best_axis] - clo[best_axis]) * scale);
                b = std::min(std::max(b, 0), bins - 1);
                return b < best_split;
            });
            mid = (uint32_t)(it - idx.begin());
            if (mid == t.first || mid == t.first + t.count) mid = t.first + t.count / 2;
        }
        const uint32_t cnt[2] = {mid - t.first, t.first + t.count - mid};
        const uint32_t beg[2] = {t.first, mid};
        for (int s = 0; s < 2; ++s) {
            Aabb b;
            b.reset();
            for (uint32_t i = beg[s]; i < beg[s] + cnt[s]; ++i) b.grow(box[idx[i]]);
            if (cnt[s] == 1) {
                const uint32_t p = idx[beg[s]];
                set_child(out.nodes, node, s, b, ~(int)p);
                out.leaf_parent[p] = (node << 1) | s;
                out.max_depth = std::max(out.max_depth, t.depth + 2);
            } else {
                set_child(out.nodes, node, s, b, kEmpty);   // child index patched when the task runs
                stack.push_back({beg[s], cnt[s], node, s, t.depth + 1});
            }
        }
    }
    if (out.max_depth > 62) {
        err = "BVH deeper than the traversal stack (62 levels)";
        return false;
    }
    return true;
}

namespace {

// One subtree below a node of the binary BVH: its box and child word (node index, or ~patch).
struct Sub {
    Aabb box;
    int child;
};

Sub binary_child(const std::vector<float> &nodes, int node, int slot)
{
    const float *nd = &nodes[(size_t)node * 16];
    Sub s;
    for (int a = 0; a < 3; ++a) {
        s.box.lo[a] = nd[4 * a + 2 * slot];
        s.box.hi[a] = nd[4 * a + 2 * slot + 1];
    }
    std::memcpy(&s.child, nd + 12 + slot, 4);
    return s;
}

// 4-wide node = 32 floats: [8a .. 8a+3] lo of the four children along axis a, [8a+4 .. 8a+7] hi, then
// the four child words, then (parent, slot in parent, children present, 0).
void set_child4(std::vector<float> &nodes, int node, int slot, const Aabb &b, int child)
{
    float *nd = &nodes[(size_t)node * 32];
    for (int a = 0; a < 3; ++a) {
        nd[8 * a + slot] = b.lo[a];
        nd[8 * a + 4 + slot] = b.hi[a];
    }
    std::memcpy(nd + 24 + slot, &child, 4);
}

}  // namespace

bool collapse_bvh4(const BvhHost &bin, uint32_t n, BvhHost &out, std::string &err)
{
    out.nodes.clear();
    out.leaf_parent.assign(n, 0);
    out.max_depth = 0;
    if (n == 0 || bin.nodes.empty()) return true;
    const int kEmpty = 0x7FFFFFFF;
    struct Task {
        int bin_node, parent, slot, depth;
    };
    std::vector<Task> stack{{0, -1, 0, 1}};
    while (!stack.empty()) {
        const Task t = stack.back();
        stack.pop_back();
        const int id = (int)(out.nodes.size() / 32);
        out.nodes.resize(out.nodes.size() + 32, 0.0f);
        if (t.parent >= 0) std::memcpy(&out.nodes[(size_t)t.parent * 32 + 24 + t.slot], &id, 4);
        out.max_depth = std::max(out.max_depth, t.depth);
        std::vector<Sub> subs;
        for (int s = 0; s < 2; ++s) {
            Sub c = binary_child(bin.nodes, t.bin_node, s);
            if (c.child != kEmpty) subs.push_back(c);
        }
        while (subs.size() < 4) {   // open the internal subtree of largest surface area
            int pick = -1;
            float best = -1.0f;
            for (size_t i = 0; i < subs.size(); ++i)
                if (subs[i].child >= 0 && subs[i].box.area() > best) {
                    best = subs[i].box.area();
                    pick = (int)i;
                }
            if (pick < 0) break;
            const int b = subs[pick].child;
            subs.erase(subs.begin() + pick);
            for (int s = 0; s < 2; ++s) {
                Sub c = binary_child(bin.nodes, b, s);
                if (c.child != kEmpty) subs.insert(subs.begin() + pick + s, c);
            }
        }
        float *nd = &out.nodes[(size_t)id * 32];
        const int present = (int)subs.size();
        std::memcpy(nd + 28, &t.parent, 4);
        std::memcpy(nd + 29, &t.slot, 4);
        std::memcpy(nd + 30, &present, 4);
        Aabb empty;
        empty.reset();
        for (int s = 0; s < 4; ++s) {
            if (s >= present) {
                set_child4(out.nodes, id, s, empty, kEmpty);
                continue;
            }
            const Sub &c = subs[s];
            if (c.child < 0) {
                set_child4(out.nodes, id, s, c.box, c.child);
                out.leaf_parent[~c.child] = (id << 2) | s;
                out.max_depth = std::max(out.max_depth, t.depth + 1);
            } else {
                set_child4(out.nodes, id, s, c.box, kEmpty);   // child word patched when the task runs
                stack.push_back({c.child, id, s, t.depth + 1});
            }
        }
    }
    // a traversal path pushes at most three siblings per level onto a 64-entry stack
    if (3 * out.max_depth > 64) {
        err = "4-wide BVH deeper than the traversal stack (21 levels)";
        return false;
    }
    return true;
}

}  // namespace ccs
