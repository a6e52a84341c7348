// Linear BVH over the camera-space triangles (the per-call rebuild; the
// default refits a static SAH topology built at set-up, bvh_topology.cu, with
// the same box and pack kernels): Morton keys
// of the centroids (geometry.cu), a stable LSD radix sort (4 x 8-bit passes),
// the radix-tree construction of Karras (HPG 2012) with index tie-breaks, and a
// bottom-up box pass with one atomic flag per internal node.  Leaves are single
// triangles; nodes store both children's boxes for two-wide tests.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int SORT_TILE = 256;

__global__ void __launch_bounds__(SORT_TILE) k_hist(const DevItem* items, int pass, int n, int shift,
                                                    int n_tiles) {
    __shared__ int h[256];
    const BvhScratch& B = items[blockIdx.y].B;
    const uint32_t* keys = (pass & 1) ? B.keys_alt : B.keys;
    int* hist = B.hist;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * SORT_TILE + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    __syncthreads();
    hist[threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of hist[256][n_tiles] in digit-major order in two launches:
// one block per (digit, item) scans its row and records the row total; one
// block per item scans the 256 totals into digit bases (hist_base), which the
// scatter adds.
FR_D int block_scan_excl(int v, int* warp_tot, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    const int r = (wid ? warp_tot[wid - 1] : 0) + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(512) k_scan_rows(const DevItem* items, int n_tiles) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const BvhScratch& B = items[blockIdx.y].B;
    int* row = B.hist + blockIdx.x * n_tiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_tiles; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const int v = t < n_tiles ? row[t] : 0;
        int tot;
        const int ex = block_scan_excl(v, warp_tot, tot);
        if (t < n_tiles) row[t] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) B.hist_base[blockIdx.x] = carry;       // row total for now
}

__global__ void __launch_bounds__(256) k_scan_digits(const DevItem* items) {
    __shared__ int warp_tot[32];
    const BvhScratch& B = items[blockIdx.x].B;
    int tot;
    const int ex = block_scan_excl(B.hist_base[threadIdx.x], warp_tot, tot);
    B.hist_base[threadIdx.x] = ex;
}

// Stable scatter: rank among equal digits = earlier warps' counts + earlier
// lanes of the same warp with that digit.
__global__ void __launch_bounds__(SORT_TILE) k_scatter(const DevItem* items, int pass, int n, int shift,
                                                       int n_tiles) {
    constexpr int NW = SORT_TILE / 32;
    const BvhScratch& B = items[blockIdx.y].B;
    const uint32_t* keys = (pass & 1) ? B.keys_alt : B.keys;
    const int* vals = (pass & 1) ? B.vals_alt : B.vals;
    uint32_t* keys_out = (pass & 1) ? B.keys : B.keys_alt;
    int* vals_out = (pass & 1) ? B.vals : B.vals_alt;
    const int* off = B.hist;
    const int* dbase = B.hist_base;
    __shared__ int cnt[NW][256];
    for (int k = threadIdx.x; k < NW * 256; k += SORT_TILE) (&cnt[0][0])[k] = 0;
    __syncthreads();
    const int i = blockIdx.x * SORT_TILE + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool ok = i < n;
    const uint32_t key = ok ? keys[i] : 0u;
    const int digit = ok ? (int)((key >> shift) & 255u) : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && rank == 0) cnt[wid][digit] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < 256) {
        int s = 0;
        for (int w = 0; w < NW; ++w) {
            const int c = cnt[w][threadIdx.x];
            cnt[w][threadIdx.x] = s;
            s += c;
        }
    }
    __syncthreads();
    if (ok) {
        const int pos = dbase[digit] + off[digit * n_tiles + blockIdx.x] + cnt[wid][digit] + rank;
        keys_out[pos] = key;
        vals_out[pos] = vals[i];
    }
}

// common prefix length of sorted keys i and j, ties broken by index
FR_D int delta(const uint32_t* k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = k[i], b = k[j];
    if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clz(a ^ b);
}

// Karras 2012: internal node i covers a key range found from the direction of
// the larger common prefix and split at the highest differing bit.
__global__ void __launch_bounds__(256) k_karras(const DevItem* items, int n, int* status) {
    const BvhScratch& B = items[blockIdx.y].B;
    const uint32_t* k = B.keys;
    int* child = B.child;
    int* parent_int = B.parent_int;
    int* parent_leaf = B.parent_leaf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int left = (lo == gamma) ? ~gamma : gamma;
    const int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    if (gamma < 0 || gamma + 1 > n - 1 || (left >= 0 && left >= n - 1) || (right >= 0 && right >= n - 1)) {
        set_status(status, FR_STATUS_BAD_BVH);      // cannot happen for sorted keys
        return;
    }
    child[2 * i] = left;
    child[2 * i + 1] = right;
    if (left < 0) parent_leaf[~left] = i; else parent_int[left] = i;
    if (right < 0) parent_leaf[~right] = i; else parent_int[right] = i;
}

__global__ void k_flag_reset(const DevItem* items, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n - 1) items[blockIdx.y].B.flag[i] = 0;
}

// flags 0; parents and child codes -1 (an unwritten child reads as leaf 0,
// never as an ancestor)
__global__ void k_bvh_init(const DevItem* items, int n) {
    const BvhScratch& B = items[blockIdx.y].B;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n - 1) {
        B.flag[i] = 0;
        B.parent_int[i] = -1;
        B.child[2 * i] = -1;
        B.child[2 * i + 1] = -1;
    }
    if (i < n) B.parent_leaf[i] = -1;
}

// Arrival count at a node, with release (this thread's box writes happen
// before it) and acquire (the sibling's box writes, released by its own
// arrival, are visible after it) at GPU scope: one round trip per level
// instead of an atomic between two full fences.
__device__ __forceinline__ int arrive_acq_rel(int* flag) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(flag) : "memory");
    return old;
}

// Leaf boxes + sorted triangle records, then climb: the second child to arrive
// at a node merges its own box with the sibling's (read from memory) and
// continues upward.
__global__ void __launch_bounds__(256) k_boxes(const DevItem* items, const int4* __restrict__ faces, int n,
                                               int* status) {
    const DevItem& it = items[blockIdx.y];
    const float4* v = it.v_cam;
    const int* vals = it.B.vals;
    const int* child = it.B.child;
    const int* parent_int = it.B.parent_int;
    const int* parent_leaf = it.B.parent_leaf;
    int* flag = it.B.flag;
    float4* box_int = it.B.box_int;
    float4* box_leaf = it.B.box_leaf;
    float4* tris = it.tris;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int id = vals[s];
    const int4 t = faces[id];
    const float4 a = v[t.x], b = v[t.y], c = v[t.z];
    tris[3 * s] = make_float4(a.x, a.y, a.z, __int_as_float(id));
    it.slot_of[id] = s;
    tris[3 * s + 1] = make_float4(b.x, b.y, b.z, 0.0f);
    tris[3 * s + 2] = make_float4(c.x, c.y, c.z, 0.0f);
    float3 lo = f3(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z)));
    float3 hi = f3(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z)));
    // pad so that the FP32 slab test never culls a triangle the exact test hits
    lo = f3(lo.x - 1e-5f - 1e-6f * fabsf(lo.x), lo.y - 1e-5f - 1e-6f * fabsf(lo.y), lo.z - 1e-5f - 1e-6f * fabsf(lo.z));
    hi = f3(hi.x + 1e-5f + 1e-6f * fabsf(hi.x), hi.y + 1e-5f + 1e-6f * fabsf(hi.y), hi.z + 1e-5f + 1e-6f * fabsf(hi.z));
    box_leaf[2 * s] = make_float4(lo.x, lo.y, lo.z, 0.0f);
    box_leaf[2 * s + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
    if (n == 1) return;
    int me = ~s;                                        // child code of the box in (lo, hi)
    int node = parent_leaf[s];
    for (int guard = 0; node >= 0; ++guard) {
        if (guard > 128 || node >= n - 1) { set_status(status, FR_STATUS_BAD_BVH); return; }
        if (arrive_acq_rel(&flag[node]) == 0) return;   // sibling not done yet
        const int c0 = child[2 * node], c1 = child[2 * node + 1];
        const int ch = c0 == me ? c1 : c0;
        if ((c0 != me && c1 != me) || ch >= n - 1 || ~ch >= n) { set_status(status, FR_STATUS_BAD_BVH); return; }
        const float4* bx = ch < 0 ? &box_leaf[2 * (~ch)] : &box_int[2 * ch];
        const float4 cl = __ldcg(bx), chh = __ldcg(bx + 1);
        lo = f3(fminf(lo.x, cl.x), fminf(lo.y, cl.y), fminf(lo.z, cl.z));
        hi = f3(fmaxf(hi.x, chh.x), fmaxf(hi.y, chh.y), fmaxf(hi.z, chh.z));
        __stcg(&box_int[2 * node], make_float4(lo.x, lo.y, lo.z, 0.0f));
        __stcg(&box_int[2 * node + 1], make_float4(hi.x, hi.y, hi.z, 0.0f));
        me = node;
        node = node == 0 ? -1 : parent_int[node];
    }
}

__global__ void __launch_bounds__(256) k_pack(const DevItem* items, int n) {
    const DevItem& it = items[blockIdx.y];
    const int* child = it.B.child;
    const float4* box_int = it.B.box_int;
    const float4* box_leaf = it.B.box_leaf;
    BvhNode* nodes = it.nodes;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 1) {
        if (i == 0) {
            const float4 l = box_leaf[0], h = box_leaf[1];
            nodes[0].a = make_float4(l.x, l.y, l.z, h.x);
            nodes[0].b = make_float4(h.y, h.z, INFINITY, INFINITY);
            nodes[0].c = make_float4(INFINITY, -INFINITY, -INFINITY, -INFINITY);
            nodes[0].d = make_int4(~0, ~0, 0, 0);
        }
        return;
    }
    if (i >= n - 1) return;
    const int c0 = child[2 * i], c1 = child[2 * i + 1];
    const float4* b0 = c0 < 0 ? &box_leaf[2 * (~c0)] : &box_int[2 * c0];
    const float4* b1 = c1 < 0 ? &box_leaf[2 * (~c1)] : &box_int[2 * c1];
    const float4 l0 = b0[0], h0 = b0[1], l1 = b1[0], h1 = b1[1];
    nodes[i].a = make_float4(l0.x, l0.y, l0.z, h0.x);
    nodes[i].b = make_float4(h0.y, h0.z, l1.x, l1.y);
    nodes[i].c = make_float4(l1.z, h1.x, h1.y, h1.z);
    nodes[i].d = make_int4(c0, c1, 0, 0);
}

// Validity: every leaf referenced exactly once, child boxes inside the parent's
// stored box, depth of each leaf.
__global__ void k_check(const DevItem* items, int n, int* out) {
    const DevItem& it = items[0];
    const BvhNode* nodes = it.nodes;
    const int* parent_int = it.B.parent_int;
    const int* parent_leaf = it.B.parent_leaf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 1) { if (i == 0) { out[0] = 1; out[1] = 0; out[2] = 1; } return; }
    if (i < n - 1) {
        const int cc[2] = {nodes[i].d.x, nodes[i].d.y};
        for (int q = 0; q < 2; ++q) {
            if (cc[q] < 0) { atomicAdd(&out[0], 1); continue; }
            // the child's own children boxes must lie inside this node's box for it
            const BvhNode& ch = nodes[cc[q]];
            const float4 pa = nodes[i].a, pb = nodes[i].b, pc = nodes[i].c;
            const float3 plo = q == 0 ? f3(pa.x, pa.y, pa.z) : f3(pb.z, pb.w, pc.x);
            const float3 phi = q == 0 ? f3(pa.w, pb.x, pb.y) : f3(pc.y, pc.z, pc.w);
            const float3 lo0 = f3(ch.a.x, ch.a.y, ch.a.z), hi0 = f3(ch.a.w, ch.b.x, ch.b.y);
            const float3 lo1 = f3(ch.b.z, ch.b.w, ch.c.x), hi1 = f3(ch.c.y, ch.c.z, ch.c.w);
            const bool in = lo0.x >= plo.x && lo0.y >= plo.y && lo0.z >= plo.z && hi0.x <= phi.x && hi0.y <= phi.y &&
                            hi0.z <= phi.z && lo1.x >= plo.x && lo1.y >= plo.y && lo1.z >= plo.z && hi1.x <= phi.x &&
                            hi1.y <= phi.y && hi1.z <= phi.z;
            if (!in) atomicAdd(&out[1], 1);
        }
    }
    if (i < n) {
        int depth = 1, node = parent_leaf[i];
        while (node > 0 && depth < 4096) { node = parent_int[node]; ++depth; }
        atomicMax(&out[2], depth);
    }
}

int nb(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

void launch_lbvh(const DevItem* items, int n, const int4* faces, int T, int* status, bool rebuild,
                 cudaStream_t st) {
    if (!rebuild) {                                  // refit a fixed topology: reset the climb flags only
        if (T > 1) {
            k_flag_reset<<<dim3(nb(T - 1, 256), n), 256, 0, st>>>(items, T);
            fr_count_launches(1);
        }
        k_boxes<<<dim3(nb(T, 256), n), 256, 0, st>>>(items, faces, T, status);
        k_pack<<<dim3(nb(T > 1 ? T - 1 : 1, 256), n), 256, 0, st>>>(items, T);
        fr_count_launches(2);
        return;
    }
    const int n_tiles = nb(T, SORT_TILE);
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        k_hist<<<dim3(n_tiles, n), SORT_TILE, 0, st>>>(items, pass, T, shift, n_tiles);
        k_scan_rows<<<dim3(256, n), 512, 0, st>>>(items, n_tiles);
        k_scan_digits<<<n, 256, 0, st>>>(items);
        k_scatter<<<dim3(n_tiles, n), SORT_TILE, 0, st>>>(items, pass, T, shift, n_tiles);
        fr_count_launches(4);
    }
    // after an even number of passes the sorted data is back in keys/vals
    if (T > 1) {
        k_bvh_init<<<dim3(nb(T, 256), n), 256, 0, st>>>(items, T);
        k_karras<<<dim3(nb(T - 1, 256), n), 256, 0, st>>>(items, T, status);
        fr_count_launches(2);
    }
    k_boxes<<<dim3(nb(T, 256), n), 256, 0, st>>>(items, faces, T, status);
    k_pack<<<dim3(nb(T > 1 ? T - 1 : 1, 256), n), 256, 0, st>>>(items, T);
    fr_count_launches(2);
}

void launch_bvh_check(const DevItem* items, int T, int* out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, sizeof(int) * 3, st);
    k_check<<<nb(T, 256), 256, 0, st>>>(items, T, out);
    fr_count_launches(1);
}
