// Host BVH construction: binned surface-area-heuristic build (Wald, "On fast
// construction of SAH-based bounding volume hierarchies", 2007) into the
// two-wide node layout the traversal kernels read.  Depth is bounded so the
// fixed traversal stack cannot overflow: past kMaxSahDepth levels the build
// falls back to median splits, which halve the triangle count per level.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "ddgi_internal.h"

namespace ddgi {
namespace {

constexpr int kBins = 32;
constexpr int kMaxLeaf = 4;   // at most kMaxLeafTris
constexpr int kMaxSahDepth = 30;   // + log2(2^28 / 4) median levels < 64 stack slots
static_assert(kMaxLeaf <= kMaxLeafTris, "leaf size beyond what the traversal encodes");
constexpr float kTraversalCost = 1.0f;
constexpr float kIntersectCost = 1.0f;

struct Aabb {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const Aabb& b) {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], b.lo[a]); hi[a] = std::max(hi[a], b.hi[a]); }
    }
    void grow(const float* p) {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
    }
    bool empty() const { return lo[0] > hi[0]; }
    float area() const {
        if (empty()) return 0.0f;
        float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0f * (dx * dy + dy * dz + dz * dx);
    }
};

struct Work {
    int32_t begin, end;     // range in the reference array
    int32_t parent;         // node index whose child slot we fill
    int32_t slot;           // 0 or 1
    int32_t depth;
};

struct Builder {
    std::vector<Aabb> tri_box;
    std::vector<float> centroid;   // 3 per triangle
    std::vector<int32_t> ref;
    std::vector<float4> nodes;
    std::vector<int32_t> leaf_order;   // triangle order of the final array
    int64_t n_leaves = 0;
    int32_t max_depth = 0;

    Aabb range_box(int32_t b, int32_t e) const {
        Aabb r;
        for (int32_t i = b; i < e; ++i) r.grow(tri_box[ref[i]]);
        return r;
    }

    // Choose a split; returns the partition point or -1 for a leaf.
    int32_t split(int32_t b, int32_t e, int32_t depth, const Aabb& box) {
        int32_t n = e - b;
        if (n <= 1) return -1;
        Aabb cb;
        for (int32_t i = b; i < e; ++i) cb.grow(&centroid[3 * ref[i]]);
        int axis = 0;
        float ext = cb.hi[0] - cb.lo[0];
        for (int a = 1; a < 3; ++a)
            if (cb.hi[a] - cb.lo[a] > ext) { ext = cb.hi[a] - cb.lo[a]; axis = a; }
        if (depth >= kMaxSahDepth || !(ext > 0.0f)) {
            if (n <= kMaxLeaf) return -1;
            int32_t mid = b + n / 2;
            std::nth_element(ref.begin() + b, ref.begin() + mid, ref.begin() + e,
                             [&](int32_t x, int32_t y) {
                                 return centroid[3 * x + axis] < centroid[3 * y + axis];
                             });
            return mid;
        }
        float best_cost = FLT_MAX;
        int best_axis = -1, best_bin = -1;
        for (int a = 0; a < 3; ++a) {
            float lo = cb.lo[a], w = cb.hi[a] - cb.lo[a];
            if (!(w > 0.0f)) continue;
            float scale = kBins / w;
            Aabb bins[kBins];
            int32_t cnt[kBins] = {0};
            for (int32_t i = b; i < e; ++i) {
                int k = std::min(kBins - 1, (int)((centroid[3 * ref[i] + a] - lo) * scale));
                bins[k].grow(tri_box[ref[i]]);
                cnt[k]++;
            }
            float left_area[kBins];
            int32_t left_cnt[kBins];
            Aabb acc;
            int32_t c = 0;
            for (int k = 0; k < kBins; ++k) {
                acc.grow(bins[k]);
                c += cnt[k];
                left_area[k] = acc.area();
                left_cnt[k] = c;
            }
            Aabb racc;
            int32_t rc = 0;
            for (int k = kBins - 1; k > 0; --k) {
                racc.grow(bins[k]);
                rc += cnt[k];
                int32_t lc = left_cnt[k - 1];
                if (lc == 0 || rc == 0) continue;
                float cost = left_area[k - 1] * lc + racc.area() * rc;
                if (cost < best_cost) { best_cost = cost; best_axis = a; best_bin = k; }
            }
        }
        float parent_area = box.area();
        float leaf_cost = kIntersectCost * n;
        float split_cost = kTraversalCost + kIntersectCost * best_cost / std::max(parent_area, 1e-30f);
        if (best_axis < 0 || (n <= kMaxLeaf && split_cost >= leaf_cost)) {
            if (n <= kMaxLeaf) return -1;
            int32_t mid = b + n / 2;
            std::nth_element(ref.begin() + b, ref.begin() + mid, ref.begin() + e,
                             [&](int32_t x, int32_t y) {
                                 return centroid[3 * x + axis] < centroid[3 * y + axis];
                             });
            return mid;
        }
        float lo = cb.lo[best_axis], scale = kBins / (cb.hi[best_axis] - cb.lo[best_axis]);
        int32_t* mid = std::partition(ref.data() + b, ref.data() + e, [&](int32_t t) {
            int k = std::min(kBins - 1, (int)((centroid[3 * t + best_axis] - lo) * scale));
            return k < best_bin;
        });
        int32_t m = (int32_t)(mid - ref.data());
        if (m == b || m == e) m = b + n / 2;
        return m;
    }

    int32_t new_node() {
        int32_t id = (int32_t)(nodes.size() / 4);
        nodes.resize(nodes.size() + 4);
        // empty children: inverted boxes never hit, count 0
        float4 inv = make_float4(FLT_MAX, -FLT_MAX, FLT_MAX, -FLT_MAX);
        nodes[4 * id + 0] = inv;
        nodes[4 * id + 1] = inv;
        nodes[4 * id + 2] = make_float4(FLT_MAX, -FLT_MAX, FLT_MAX, -FLT_MAX);
        int32_t z[4] = {~0, ~0, 0, 0};
        std::memcpy(&nodes[4 * id + 3], z, sizeof(z));
        return id;
    }

    void set_child(int32_t node, int slot, const Aabb& box, int32_t child, int32_t count) {
        float4& xy = nodes[4 * node + slot];
        xy = make_float4(box.lo[0], box.hi[0], box.lo[1], box.hi[1]);
        float4& z = nodes[4 * node + 2];
        if (slot == 0) { z.x = box.lo[2]; z.y = box.hi[2]; } else { z.z = box.lo[2]; z.w = box.hi[2]; }
        int32_t meta[4];
        std::memcpy(meta, &nodes[4 * node + 3], sizeof(meta));
        meta[slot] = child;
        meta[2 + slot] = count;
        std::memcpy(&nodes[4 * node + 3], meta, sizeof(meta));
    }

    void run(int32_t n) {
        ref.resize(n);
        for (int32_t i = 0; i < n; ++i) ref[i] = i;
        int32_t root = new_node();
        Aabb all = range_box(0, n);
        std::vector<Work> stack;
        int32_t m = split(0, n, 0, all);
        if (m < 0) {
            // whole scene is one leaf hanging off the root
            set_child(root, 0, all, ~(int32_t)leaf_order.size(), n);
            for (int32_t i = 0; i < n; ++i) leaf_order.push_back(ref[i]);
            n_leaves = 1;
            return;
        }
        stack.push_back({m, n, root, 1, 1});
        stack.push_back({0, m, root, 0, 1});
        while (!stack.empty()) {
            Work w = stack.back();
            stack.pop_back();
            max_depth = std::max(max_depth, w.depth);
            Aabb box = range_box(w.begin, w.end);
            int32_t s = split(w.begin, w.end, w.depth, box);
            if (s < 0) {
                set_child(w.parent, w.slot, box, ~(int32_t)leaf_order.size(), w.end - w.begin);
                for (int32_t i = w.begin; i < w.end; ++i) leaf_order.push_back(ref[i]);
                n_leaves++;
                continue;
            }
            int32_t id = new_node();
            set_child(w.parent, w.slot, box, id, 0);
            stack.push_back({s, w.end, id, 1, w.depth + 1});
            stack.push_back({w.begin, s, id, 0, w.depth + 1});
        }
    }
};

// One binary child: box, reference (node >= 0 or ~first), triangle count.
struct Kid {
    float lo[3], hi[3];
    int32_t ref, cnt;
    float area() const {
        float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0f * (dx * dy + dy * dz + dz * dx);
    }
};

void binary_kids(const std::vector<float4>& n2, int32_t i, std::vector<Kid>& out) {
    int32_t meta[4];
    std::memcpy(meta, &n2[4 * (size_t)i + 3], sizeof(meta));
    const float4 z = n2[4 * (size_t)i + 2];
    for (int slot = 0; slot < 2; ++slot) {
        if (meta[slot] < 0 && meta[2 + slot] == 0) continue;   // empty slot
        const float4 xy = n2[4 * (size_t)i + slot];
        Kid k;
        k.lo[0] = xy.x; k.hi[0] = xy.y;
        k.lo[1] = xy.z; k.hi[1] = xy.w;
        k.lo[2] = slot ? z.z : z.x; k.hi[2] = slot ? z.w : z.y;
        k.ref = meta[slot];
        k.cnt = meta[2 + slot];
        out.push_back(k);
    }
}

// Collapse of the binary hierarchy into 4-wide nodes: a node starts from a
// binary node's two children and repeatedly replaces its internal child of
// largest surface area by that child's two children until it holds four
// (two below kWideFullDepth).  Layout, 8 float4 per node: the children's
// lo_x, hi_x, lo_y, hi_y, lo_z, hi_z (one float4 each, child c in lane c),
// an int4 of child references, one float4 of padding.  An empty slot has
// the box lo = hi = (+inf, +inf, +inf), which no ray enters, and reference
// kRefDone.
void collapse_wide(const std::vector<float4>& n2, std::vector<float4>& n4, int32_t& max_depth4) {
    n4.clear();
    max_depth4 = 0;
    if (n2.empty()) return;
    struct Job {
        int32_t n2, n4, depth;
    };
    std::vector<Job> jobs{{0, 0, 1}};
    n4.resize(8);
    std::vector<Kid> kids, sub;
    while (!jobs.empty()) {
        Job j = jobs.back();
        jobs.pop_back();
        max_depth4 = std::max(max_depth4, j.depth);
        kids.clear();
        binary_kids(n2, j.n2, kids);
        const size_t width = j.depth <= kWideFullDepth ? 4 : 2;
        while (kids.size() < width) {
            int best = -1;
            float best_area = -1.0f;
            for (size_t k = 0; k < kids.size(); ++k)
                if (kids[k].ref >= 0 && kids[k].area() > best_area) { best_area = kids[k].area(); best = (int)k; }
            if (best < 0) break;
            sub.clear();
            binary_kids(n2, kids[best].ref, sub);
            kids.erase(kids.begin() + best);
            kids.insert(kids.end(), sub.begin(), sub.end());
        }
        float lo[3][4], hi[3][4];
        int32_t ref[4];
        for (int c = 0; c < 4; ++c) {
            if (c < (int)kids.size()) {
                const Kid& k = kids[c];
                for (int a = 0; a < 3; ++a) { lo[a][c] = k.lo[a]; hi[a][c] = k.hi[a]; }
                if (k.ref >= 0) {
                    int32_t id = (int32_t)(n4.size() / 8);
                    n4.resize(n4.size() + 8);
                    jobs.push_back({k.ref, id, j.depth + 1});
                    ref[c] = id;
                } else {
                    ref[c] = ~(((~k.ref) << kLeafBits) | (k.cnt - 1));
                }
            } else {
                for (int a = 0; a < 3; ++a) { lo[a][c] = INFINITY; hi[a][c] = INFINITY; }
                ref[c] = kRefDone;
            }
        }
        float4* N = &n4[8 * (size_t)j.n4];
        for (int a = 0; a < 3; ++a) {
            N[2 * a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
            N[2 * a + 1] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
        }
        std::memcpy(&N[6], ref, sizeof(ref));
        N[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

}  // namespace

int64_t wide_stack_bound(const std::vector<float4>& n4) {
    if (n4.empty()) return 0;
    std::vector<int32_t> st{0};
    int64_t deepest = 1;
    while (!st.empty()) {
        const int32_t ref = st.back();
        st.pop_back();
        if (ref < 0) continue;   // a leaf
        int32_t kid[4];
        std::memcpy(kid, &n4[8 * (size_t)ref + 6], sizeof(kid));
        for (int c = 0; c < 4; ++c)
            if (kid[c] != kRefDone) st.push_back(kid[c]);
        deepest = std::max<int64_t>(deepest, (int64_t)st.size());
    }
    return deepest;
}

bool build_bvh(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
               const int32_t* tri_flags, BvhHost& out, std::string& err) {
    out = BvhHost();
    if (n_tris == 0) return true;
    if (n_tris > (int64_t)(1 << 30)) { err = "too many triangles"; return false; }
    Builder b;
    int32_t n = (int32_t)n_tris;
    b.tri_box.resize(n);
    b.centroid.resize(3 * (size_t)n);
    for (int32_t t = 0; t < n; ++t) {
        Aabb box;
        for (int k = 0; k < 3; ++k) {
            int32_t vi = tris[3 * (int64_t)t + k];
            if (vi < 0 || vi >= n_verts) { err = "triangle vertex index out of range"; return false; }
            box.grow(verts + 3 * (int64_t)vi);
        }
        b.tri_box[t] = box;
        for (int a = 0; a < 3; ++a) b.centroid[3 * t + a] = 0.5f * (box.lo[a] + box.hi[a]);
    }
    b.run(n);
    out.nodes = std::move(b.nodes);
    out.n_leaves = b.n_leaves;
    out.max_depth = b.max_depth;
    out.tris.resize(3 * (size_t)n);
    for (int32_t k = 0; k < n; ++k) {
        int32_t t = b.leaf_order[k];
        const float* v[3];
        for (int c = 0; c < 3; ++c) v[c] = verts + 3 * (int64_t)tris[3 * (int64_t)t + c];
        float id_bits, flag_bits;
        int32_t flags = tri_flags ? tri_flags[t] : 1;
        std::memcpy(&id_bits, &t, 4);
        std::memcpy(&flag_bits, &flags, 4);
        out.tris[3 * k + 0] = make_float4(v[0][0], v[0][1], v[0][2], id_bits);
        out.tris[3 * k + 1] = make_float4(v[1][0], v[1][1], v[1][2], flag_bits);
        out.tris[3 * k + 2] = make_float4(v[2][0], v[2][1], v[2][2], 0.0f);
    }
    if (out.max_depth > 62) { err = "BVH too deep"; return false; }
    collapse_wide(out.nodes, out.nodes4, out.max_depth4);
    return true;
}

}  // namespace ddgi
