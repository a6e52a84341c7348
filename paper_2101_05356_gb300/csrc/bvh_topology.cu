// Static BVH topology for a fixed-connectivity mesh, built once on the host
// when the mesh is set (like the edge and vertex->face lists): a binned
// surface-area-heuristic split of the mean face's triangles (model space),
// single-triangle leaves, internal nodes numbered in pre-order (root 0) and
// leaves numbered left to right.  Every call then refits the boxes of this
// topology to the morphed, posed face on the GPU (k_boxes / k_pack in
// lbvh.cu); the per-call LBVH rebuild remains available (FR_FLAG_LBVH) for
// deformations the mean-face topology does not suit.
//
// Depth is capped: below depth SAH_MAX_DEPTH a node is split at the median of
// its centroids along the widest axis instead, so the tree is at most
// 40 + log2(T) deep (57 at 100,000 triangles) and the 64-entry traversal stack
// cannot overflow whatever the SAH prefers.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "kernels.h"

namespace {

constexpr int SAH_BINS = 32;      // 128 or 512 bins cut node visits by 0.5% only (measured)
constexpr int SAH_MAX_DEPTH = 40;

struct Box {
    float lo[3] = {INFINITY, INFINITY, INFINITY};
    float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    double area() const {
        if (!(hi[0] >= lo[0])) return 0.0;
        const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return dx * dy + dy * dz + dz * dx;
    }
};

struct Builder {
    const std::vector<Box>& box;
    const std::vector<float>& cen;          // [T][3]
    std::vector<int> prim;
    BvhTopology& out;
    int next_internal = 0, next_leaf = 0;

    Builder(const std::vector<Box>& b, const std::vector<float>& c, BvhTopology& o) : box(b), cen(c), out(o) {}

    // child code of the subtree over prim[s, e): ~leaf slot or internal index
    int build(int s, int e, int parent, int depth) {
        if (e - s == 1) {
            const int slot = next_leaf++;
            out.vals[slot] = prim[s];
            out.parent_leaf[slot] = parent;
            return ~slot;
        }
        const int id = next_internal++;
        out.parent_int[id] = parent;
        const int mid = split(s, e, depth);
        const int l = build(s, mid, id, depth + 1);
        const int r = build(mid, e, id, depth + 1);
        out.child[2 * id] = l;
        out.child[2 * id + 1] = r;
        return id;
    }

    // partition prim[s, e) and return the split point (s < mid < e)
    int split(int s, int e, int depth) {
        float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int i = s; i < e; ++i)
            for (int k = 0; k < 3; ++k) {
                clo[k] = std::min(clo[k], cen[3 * prim[i] + k]);
                chi[k] = std::max(chi[k], cen[3 * prim[i] + k]);
            }
        int best_axis = -1, best_bin = -1;
        double best_cost = INFINITY;
        if (depth < SAH_MAX_DEPTH) {
            for (int ax = 0; ax < 3; ++ax) {
                const float ext = chi[ax] - clo[ax];
                if (!(ext > 0.0f)) continue;
                Box bb[SAH_BINS];
                int cnt[SAH_BINS] = {0};
                for (int i = s; i < e; ++i) {
                    const int b = bin_of(prim[i], ax, clo[ax], ext);
                    cnt[b]++;
                    bb[b].grow(box[prim[i]]);
                }
                double right_area[SAH_BINS];
                int right_cnt[SAH_BINS];
                Box acc;
                int n = 0;
                for (int b = SAH_BINS - 1; b > 0; --b) {
                    acc.grow(bb[b]);
                    n += cnt[b];
                    right_area[b] = acc.area();
                    right_cnt[b] = n;
                }
                Box left;
                int nl = 0;
                for (int b = 0; b < SAH_BINS - 1; ++b) {      // split after bin b
                    left.grow(bb[b]);
                    nl += cnt[b];
                    const int nr = right_cnt[b + 1];
                    if (nl == 0 || nr == 0) continue;
                    const double cost = left.area() * nl + right_area[b + 1] * nr;
                    if (cost < best_cost) {
                        best_cost = cost;
                        best_axis = ax;
                        best_bin = b;
                    }
                }
            }
        }
        if (best_axis >= 0) {
            const float lo = clo[best_axis], ext = chi[best_axis] - clo[best_axis];
            const auto it = std::stable_partition(prim.begin() + s, prim.begin() + e, [&](int p) {
                return bin_of(p, best_axis, lo, ext) <= best_bin;
            });
            return (int)(it - prim.begin());
        }
        // median of the centroids along the widest axis (ties by triangle index)
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
        std::stable_sort(prim.begin() + s, prim.begin() + e, [&](int a, int b) {
            const float ca = cen[3 * a + ax], cb = cen[3 * b + ax];
            return ca < cb || (ca == cb && a < b);
        });
        return s + (e - s) / 2;
    }

    int bin_of(int p, int ax, float lo, float ext) const {
        const int b = (int)((cen[3 * p + ax] - lo) / ext * SAH_BINS);
        return std::min(std::max(b, 0), SAH_BINS - 1);
    }
};

}  // namespace

void build_bvh_topology(const float* v, const int* faces, int T, BvhTopology& out) {
    out.child.assign(2 * (size_t)std::max(T - 1, 1), -1);
    out.parent_int.assign((size_t)std::max(T - 1, 1), -1);
    out.parent_leaf.assign((size_t)T, -1);
    out.vals.assign((size_t)T, 0);
    if (T == 1) {
        out.vals[0] = 0;
        return;
    }
    std::vector<Box> box((size_t)T);
    std::vector<float> cen(3 * (size_t)T);
    for (int f = 0; f < T; ++f) {
        for (int q = 0; q < 3; ++q) {
            const float* p = v + 3 * (size_t)faces[3 * f + q];
            for (int k = 0; k < 3; ++k) {
                box[f].lo[k] = std::min(box[f].lo[k], p[k]);
                box[f].hi[k] = std::max(box[f].hi[k], p[k]);
            }
        }
        for (int k = 0; k < 3; ++k) cen[3 * f + k] = 0.5f * (box[f].lo[k] + box[f].hi[k]);
    }
    Builder b(box, cen, out);
    b.prim.resize((size_t)T);
    for (int f = 0; f < T; ++f) b.prim[f] = f;
    b.build(0, T, -1, 0);
}
