// Broad phase: candidate triangle pairs whose closed bounding boxes overlap.
//
// §1.2 accelerates the pair tests with a spatial structure that "eliminates
// redundant computations" (spatial hashing there).  Here: a linear BVH built
// from 63-bit Morton codes (Karras' radix-tree construction), refitted
// bottom-up, then traversed without a stack: every node stores its left child
// and its "rope" (the next node of a depth-first walk once its subtree is done),
// which in a Karras tree follows from the node's leaf range alone.  One pass
// counts each leaf's partners and keeps the first kSpill of them; offsets come
// from a scan, the kept pairs are copied out, and only leaves with more partners
// are walked again.  The pair list comes out in a deterministic order (leaf
// order, then depth-first order) without a global sort.  Topologically adjacent
// pairs (a shared vertex index, §1) are dropped.
#include <algorithm>

#include "common.cuh"

namespace ttie {

namespace {

constexpr int kThreads = 256;
constexpr int kStack = 96;    // bound on the refit's climb (tree depth) before it reports a malformed tree
constexpr int kSpill = 16;    // partners kept per leaf by the counting pass

__device__ __forceinline__ unsigned long long ordered_bits(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered(unsigned long long u) {
    u = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    return __longlong_as_double((long long)u);
}

template <typename T> __device__ __forceinline__ bool finite3(T a, T b, T c) { return isfinite(a) && isfinite(b) && isfinite(c); }

template <typename T>
__global__ void k_pack_positions(const T *__restrict__ x, int stride, int64_t V, vec4_t<T> *__restrict__ out,
                                 DevScalars *ds) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        T a = x[i * stride], b = x[i * stride + 1], c = x[i * stride + 2];
        vec4_t<T> v;
        v.x = a; v.y = b; v.z = c; v.w = T(0);
        out[i] = v;
        if (!finite3(a, b, c)) atomicOr(&ds->err, ERR_NONFINITE);
    }
}

__global__ void k_pack_topology(const int32_t *__restrict__ tri, const int32_t *__restrict__ grp_in, int64_t F,
                                int64_t V, int4 *__restrict__ tri4, int32_t *__restrict__ grp, DevScalars *ds) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        int a = tri[3 * f], b = tri[3 * f + 1], c = tri[3 * f + 2];
        if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V) {
            atomicOr(&ds->err, ERR_BAD_INDEX);
            a = b = c = 0;
        }
        tri4[f] = make_int4(a, b, c, 0);
        if (grp_in) {
            int g = grp_in[f];
            if (g < 0 || g >= (1 << 20)) {
                atomicOr(&ds->err, ERR_BAD_INDEX);
                g = 0;
            }
            grp[f] = g;
            atomicMax(&ds->max_group, g);
        }
    }
}

__global__ void k_init_bounds(DevScalars *ds) {
    if (threadIdx.x < 3) {
        ds->bounds_lo[threadIdx.x] = ~0ull;
        ds->bounds_hi[threadIdx.x] = 0ull;
    }
}

template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// Box of each triangle (over the vertices at x0 and, when x1 is given, also at x1:
// the box swept by a straight-line motion) and the scene bounds of the box centres.  The
// centres and their bounds only place the Morton codes, so they are taken in the positions'
// own precision (FP32 for FP32 positions, not the slow FP64 pipe).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_tri_boxes(const vec4_t<T> *__restrict__ x0, const vec4_t<T> *__restrict__ x1,
                                                        const int4 *__restrict__ tri4, int64_t F, Box<T> *__restrict__ box,
                                                        DevScalars *ds) {
    constexpr T kBig = sizeof(T) == 4 ? T(3e38) : T(1e300);
    T clo[3] = {kBig, kBig, kBig}, chi[3] = {-kBig, -kBig, -kBig};
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        int4 t = tri4[f];
        vec4_t<T> a = x0[t.x], b = x0[t.y], c = x0[t.z];
        Box<T> bx;
        bx.lo.x = tmin(a.x, tmin(b.x, c.x)); bx.lo.y = tmin(a.y, tmin(b.y, c.y)); bx.lo.z = tmin(a.z, tmin(b.z, c.z));
        bx.hi.x = tmax(a.x, tmax(b.x, c.x)); bx.hi.y = tmax(a.y, tmax(b.y, c.y)); bx.hi.z = tmax(a.z, tmax(b.z, c.z));
        if (x1) {
            a = x1[t.x]; b = x1[t.y]; c = x1[t.z];
            bx.lo.x = tmin(bx.lo.x, tmin(a.x, tmin(b.x, c.x)));
            bx.lo.y = tmin(bx.lo.y, tmin(a.y, tmin(b.y, c.y)));
            bx.lo.z = tmin(bx.lo.z, tmin(a.z, tmin(b.z, c.z)));
            bx.hi.x = tmax(bx.hi.x, tmax(a.x, tmax(b.x, c.x)));
            bx.hi.y = tmax(bx.hi.y, tmax(a.y, tmax(b.y, c.y)));
            bx.hi.z = tmax(bx.hi.z, tmax(a.z, tmax(b.z, c.z)));
        }
        bx.lo.w = T(0);
        bx.hi.w = T(0);
        box[f] = bx;
        const T cx = T(0.5) * (bx.lo.x + bx.hi.x), cy = T(0.5) * (bx.lo.y + bx.hi.y), cz = T(0.5) * (bx.lo.z + bx.hi.z);
        clo[0] = tmin(clo[0], cx); clo[1] = tmin(clo[1], cy); clo[2] = tmin(clo[2], cz);
        chi[0] = tmax(chi[0], cx); chi[1] = tmax(chi[1], cy); chi[2] = tmax(chi[2], cz);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o; o >>= 1) {
            clo[k] = tmin(clo[k], __shfl_xor_sync(0xffffffffu, clo[k], o));
            chi[k] = tmax(chi[k], __shfl_xor_sync(0xffffffffu, chi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0 && clo[0] <= chi[0]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(&ds->bounds_lo[k], ordered_bits((double)clo[k]));
            atomicMax(&ds->bounds_hi[k], ordered_bits((double)chi[k]));
        }
    }
}

__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
    // insert two zero bits between the low 21 bits of v
    v &= 0x1fffffull;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}

template <typename T>
__global__ void k_morton(const Box<T> *__restrict__ box, int64_t F, const int32_t *__restrict__ grp, int group_bits,
                         const DevScalars *ds, unsigned long long *__restrict__ key, uint32_t *__restrict__ perm) {
    // quantised in FP32 (the codes only order the leaves; any deterministic rounding does)
    const int b = (63 - group_bits) / 3;
    const float scale = (float)((1u << b) - 1u);
    float lo[3], inv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double l = from_ordered(ds->bounds_lo[k]), h = from_ordered(ds->bounds_hi[k]);
        lo[k] = (float)l;
        const float e = (float)(h - l);
        inv[k] = e > 0.0f ? 1.0f / e : 1.0f;
    }
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        Box<T> bx = box[f];
        const float c[3] = {(float)(T(0.5) * (bx.lo.x + bx.hi.x)), (float)(T(0.5) * (bx.lo.y + bx.hi.y)),
                            (float)(T(0.5) * (bx.lo.z + bx.hi.z))};
        unsigned long long q[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float u = fminf(fmaxf((c[k] - lo[k]) * inv[k], 0.0f), 1.0f);
            q[k] = (unsigned long long)(u * scale);
        }
        unsigned long long m = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
        if (group_bits) m |= (unsigned long long)grp[f] << (3 * b);
        key[f] = m;
        perm[f] = (uint32_t)f;
    }
}

__global__ void k_leaf_group(const uint32_t *__restrict__ perm, const int32_t *__restrict__ grp, int64_t n,
                             int32_t *__restrict__ leaf_group) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        leaf_group[s] = grp[perm[s]];
}

__global__ void k_group_ranges(const int32_t *__restrict__ lg, int64_t n, int2 *__restrict__ range) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        int g = lg[s];
        if (s == 0 || lg[s - 1] != g) range[g].x = (int)s;
        if (s == n - 1 || lg[s + 1] != g) range[g].y = (int)s;
    }
}

__global__ void k_fill_int2(int2 *p, int64_t n, int2 v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// Length of the common prefix of sorted keys i and j; ties broken by the index.
__device__ __forceinline__ int delta(const unsigned long long *__restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned long long a = k[i], b = k[j];
    if (a == b) return 64 + __clz((unsigned)(i ^ j));
    return __clzll(a ^ b);
}

// Internal node i of the radix tree over n sorted keys (Karras 2012).  Leaves are nodes
// n-1 .. 2n-2; the root is internal node 0.
__global__ void k_karras(const unsigned long long *__restrict__ key, int n, int2 *__restrict__ child,
                         int *__restrict__ parent, int2 *__restrict__ range) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x) {
        const int d = (delta(key, n, i, i + 1) - delta(key, n, i, i - 1)) >= 0 ? 1 : -1;
        const int dmin = delta(key, n, i, i - d);
        int lmax = 2;
        while (delta(key, n, i, i + lmax * d) > dmin) lmax <<= 1;
        int l = 0;
        for (int t = lmax >> 1; t >= 1; t >>= 1)
            if (delta(key, n, i, i + (l + t) * d) > dmin) l += t;
        const int j = i + l * d;
        const int dnode = delta(key, n, i, j);
        int s = 0, t = l;
        do {
            t = (t + 1) >> 1;
            if (delta(key, n, i, i + (s + t) * d) > dnode) s += t;
        } while (t > 1);
        const int gamma = i + s * d + (d < 0 ? -1 : 0);
        const int lo = min(i, j), hi = max(i, j);
        const int left = (lo == gamma) ? (n - 1 + gamma) : gamma;
        const int right = (hi == gamma + 1) ? (n - 1 + gamma + 1) : gamma + 1;
        child[i] = make_int2(left, right);
        parent[left] = i;
        parent[right] = i;
        range[i] = make_int2(lo, hi);
        if (i == 0) parent[0] = -1;
    }
}

template <typename T>
__global__ void k_leaf_boxes(const Box<T> *__restrict__ tbox, const uint32_t *__restrict__ perm, int n,
                             Box<T> *__restrict__ node_box, int2 *__restrict__ range) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        node_box[n - 1 + s] = tbox[perm[s]];
        range[n - 1 + s] = make_int2(s, s);
    }
}

template <typename T> __device__ __forceinline__ vec4_t<T> ld_cg(const vec4_t<T> *p);
template <> __device__ __forceinline__ float4 ld_cg<float>(const float4 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ dvec4 ld_cg<double>(const dvec4 *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    dvec4 r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}

// Bottom-up refit: the second child to arrive at a node writes its box and moves up.
template <typename T>
__global__ void k_refit(int n, const int *__restrict__ parent, const int2 *__restrict__ child, Box<T> *node_box,
                        unsigned int *visit, DevScalars *ds) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        int node = parent[n - 1 + s];
        for (int level = 0; node >= 0; ++level) {
            if (level > 2 * kStack) {   // deeper than any valid tree: malformed, stop
                atomicOr(&ds->err, ERR_STACK);
                break;
            }
            // the first child to arrive stops; the second sees both boxes: leaf boxes come from
            // an earlier launch, an inner node's box was written and fenced before its counter
            if (atomicAdd(&visit[node], 1u) == 0u) break;
            int2 ch = child[node];
            vec4_t<T> alo = ld_cg<T>(&node_box[ch.x].lo), ahi = ld_cg<T>(&node_box[ch.x].hi);
            vec4_t<T> blo = ld_cg<T>(&node_box[ch.y].lo), bhi = ld_cg<T>(&node_box[ch.y].hi);
            Box<T> u;
            u.lo.x = tmin(alo.x, blo.x); u.lo.y = tmin(alo.y, blo.y); u.lo.z = tmin(alo.z, blo.z); u.lo.w = T(0);
            u.hi.x = tmax(ahi.x, bhi.x); u.hi.y = tmax(ahi.y, bhi.y); u.hi.z = tmax(ahi.z, bhi.z); u.hi.w = T(0);
            node_box[node] = u;
            __threadfence();   // this box before the parent's counter
            node = parent[node];
        }
    }
}

template <typename T>
__device__ __forceinline__ bool overlap(const vec4_t<T> &alo, const vec4_t<T> &ahi, const vec4_t<T> &blo,
                                        const vec4_t<T> &bhi) {
    return alo.x <= bhi.x && blo.x <= ahi.x && alo.y <= bhi.y && blo.y <= ahi.y && alo.z <= bhi.z && blo.z <= ahi.z;
}

// Each leaf's triangle in leaf order: its vertex indices and, in w, the triangle's index.
__global__ void k_leaf_tri(const uint32_t *__restrict__ perm, const int4 *__restrict__ tri4, int64_t n,
                           int4 *__restrict__ leaf_tri) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = perm[i];
        int4 v = tri4[t];
        v.w = (int)t;
        leaf_tri[i] = v;
    }
}

__device__ __forceinline__ bool share_vertex(int4 a, int4 b) {
    return a.x == b.x || a.x == b.y || a.x == b.z || a.y == b.x || a.y == b.y || a.y == b.z || a.z == b.x ||
           a.z == b.y || a.z == b.z;
}

// Links stored in the unused w lanes of the node boxes: lo.w = left child (-1 for a leaf),
// hi.w = rope.  A node covering leaves [lo, hi] is followed, once its subtree is done, by the
// right sibling of its lowest ancestor-or-self that is a left child; that sibling covers a range
// starting at hi + 1 and is internal node hi + 1 when that node's range starts there (in a
// Karras tree internal node k has k as one end of its range), else leaf hi + 1.
template <typename T> __device__ __forceinline__ void set_link(T &w, int v);
template <> __device__ __forceinline__ void set_link<float>(float &w, int v) { w = __int_as_float(v); }
template <> __device__ __forceinline__ void set_link<double>(double &w, int v) { w = __longlong_as_double((long long)v); }
template <typename T> __device__ __forceinline__ int get_link(T w);
template <> __device__ __forceinline__ int get_link<float>(float w) { return __float_as_int(w); }
template <> __device__ __forceinline__ int get_link<double>(double w) { return (int)__double_as_longlong(w); }

template <typename T>
__global__ void k_links(int n, const int2 *__restrict__ child, const int2 *__restrict__ range, Box<T> *node_box) {
    const int nodes = 2 * n - 1;
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nodes; node += gridDim.x * blockDim.x) {
        const int2 r = range[node];
        int rope = -1;
        if (r.y < n - 1) {
            const int k = r.y + 1;
            rope = (k < n - 1 && range[k].x == k) ? k : n - 1 + k;
        }
        set_link<T>(node_box[node].lo.w, node < n - 1 ? child[node].x : -1);
        set_link<T>(node_box[node].hi.w, rope);
    }
}

// One thread per leaf s: every leaf s' > s in the pair-mode window whose box overlaps, in
// depth-first order.  kPass 0 counts them and keeps the first kSpill in spill[s]; kPass 1
// writes all of them at offset[s], for the leaves with more than kSpill.
// kOneWalk (counting pass only): the walk starts at the node that follows leaf lo - 1 in
// depth-first order (its rope) and stops at the first node past hi.  The walk from the root
// reaches that node before any output, having only descended ancestors of lo - 1 and skipped
// subtrees below lo, and past it ranges only grow, so the partners and their order are the
// same.  Partners past the first kSpill go to kChunk-pair chunks taken from the pool by one
// atomic each and linked per leaf (head[s], next[chunk]); a chunk index past pool_chunks is not
// written, and the host then runs kPass 1 for the list instead.
constexpr int kChunk = 32;
template <typename T, int kPass, bool kOneWalk = false>
__global__ void __launch_bounds__(kThreads) k_traverse(int n, const int2 *__restrict__ range,
                                                       const Box<T> *__restrict__ node_box,
                                                       const int4 *__restrict__ leaf_tri,
                                                       const int32_t *__restrict__ leaf_group,
                                                       const int2 *__restrict__ group_range, int mode,
                                                       uint32_t *__restrict__ count,
                                                       const unsigned long long *__restrict__ offset,
                                                       int2 *__restrict__ spill, int2 *__restrict__ pairs,
                                                       DevScalars *ds, int2 *__restrict__ pool = nullptr,
                                                       int *__restrict__ pool_next = nullptr,
                                                       int *__restrict__ pool_head = nullptr,
                                                       unsigned long long pool_chunks = 0) {
    static_assert(!(kOneWalk && kPass != 0), "the one-walk traversal is a counting pass");
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        if (kPass == 1 && count[s] <= (uint32_t)kSpill) continue;
        int lo = s + 1, hi = n - 1;
        if (mode == TTIE_PAIRS_INTRA_GROUP) {
            hi = group_range[leaf_group[s]].y;
        } else if (mode == TTIE_PAIRS_INTER_GROUP) {
            lo = max(lo, group_range[leaf_group[s]].y + 1);
        }
        uint32_t cnt = 0;
        int chunk = -1;
        const unsigned long long out = kPass == 1 ? offset[s] : 0ull;
        if (lo <= hi) {
            const int4 tq = leaf_tri[s];
            const uint32_t qi = (uint32_t)tq.w;
            const Box<T> qb = node_box[n - 1 + s];
            int node = kOneWalk ? get_link<T>(node_box[n - 1 + lo - 1].hi.w) : 0;
            for (int steps = 0; node >= 0; ++steps) {
                if (steps > 2 * n) {   // a walk visits every node at most once: malformed links
                    atomicOr(&ds->err, ERR_STACK);
                    break;
                }
                // a leaf's triangle is loaded with its box (leaves are the nodes from n - 1 on), so
                // the shared-vertex test waits for no further load
                int4 lt = make_int4(-1, -1, -1, -1);
                if (node >= n - 1) lt = leaf_tri[node - (n - 1)];
                const Box<T> nb = node_box[node];
                const int2 r = range[node];
                if (kOneWalk && r.x > hi) break;
                int next = get_link<T>(nb.hi.w);
                if (r.y >= lo && r.x <= hi && overlap<T>(qb.lo, qb.hi, nb.lo, nb.hi)) {
                    const int left = get_link<T>(nb.lo.w);
                    if (left >= 0) {
                        next = left;
                    } else {
                        const uint32_t tj = (uint32_t)lt.w;
                        if (!share_vertex(tq, lt)) {
                            const int2 pr = make_int2((int)min(qi, tj), (int)max(qi, tj));
                            if (kPass == 0) {
                                if (cnt < (uint32_t)kSpill) {
                                    spill[(size_t)s * kSpill + cnt] = pr;
                                } else if (kOneWalk) {
                                    const uint32_t q = cnt - (uint32_t)kSpill, slot = q & (uint32_t)(kChunk - 1);
                                    if (slot == 0) {
                                        const unsigned long long cid = atomicAdd(&ds->ovf_cursor, 1ull);
                                        const int nc = cid < pool_chunks ? (int)cid : -1;
                                        if (q == 0) pool_head[s] = nc;
                                        else if (chunk >= 0) pool_next[chunk] = nc;
                                        chunk = nc;
                                    }
                                    if (chunk >= 0) pool[(size_t)chunk * kChunk + slot] = pr;
                                }
                            } else if (!TTIE_BAD(ds, out + cnt < offset[s + 1], 61, out + cnt)) {
                                pairs[out + cnt] = pr;
                            }
                            ++cnt;
                        }
                    }
                }
                node = next;
            }
        }
        if (kPass == 0) count[s] = cnt;
    }
}

// One-walk traversal: the partners of each leaf past its first kSpill, from its chunk chain
// (in walk order) to their place after the kept ones.  Runs only when no chunk index ran past
// the pool; the copy still stops at a chunk index outside the pool.
__global__ void k_chunk_copy(int n, const uint32_t *__restrict__ count, const unsigned long long *__restrict__ offset,
                             const int2 *__restrict__ pool, const int *__restrict__ pool_next,
                             const int *__restrict__ pool_head, unsigned long long pool_chunks,
                             int2 *__restrict__ pairs) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint32_t cnt = count[s];
        if (cnt <= (uint32_t)kSpill) continue;
        unsigned long long out = offset[s] + kSpill, end = offset[s + 1];
        uint32_t rem = cnt - (uint32_t)kSpill;
        int chunk = pool_head[s];
        while (rem > 0) {
            if (chunk < 0 || (unsigned long long)chunk >= pool_chunks) break;
            const uint32_t take = min(rem, (uint32_t)kChunk);
            for (uint32_t i = 0; i < take && out + i < end; ++i) pairs[out + i] = pool[(size_t)chunk * kChunk + i];
            out += take;
            rem -= take;
            if (rem > 0) chunk = pool_next[chunk];
        }
    }
}

// Copy the kept partners of every leaf to its place in the pair list.
__global__ void k_spill_copy(int n, const uint32_t *__restrict__ count, const unsigned long long *__restrict__ offset,
                             const int2 *__restrict__ spill, int2 *__restrict__ pairs) {
    const long long total = (long long)n * kSpill;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / kSpill), k = (int)(i - (long long)s * kSpill);
        if ((uint32_t)k < min(count[s], (uint32_t)kSpill)) pairs[offset[s] + k] = spill[i];
    }
}

// Brute force: every pair i<j of the mode sharing no vertex (no box test).
template <bool kWrite>
__global__ void k_brute(int n, const int4 *__restrict__ tri4, const int32_t *__restrict__ grp, int mode,
                        uint32_t *__restrict__ count, const unsigned long long *__restrict__ offset,
                        int2 *__restrict__ pairs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 ti = tri4[i];
        const int gi = grp ? grp[i] : 0;
        uint32_t cnt = 0;
        unsigned long long out = kWrite ? offset[i] : 0ull;
        for (int j = i + 1; j < n; ++j) {
            if (mode == TTIE_PAIRS_INTER_GROUP && grp[j] == gi) continue;
            if (mode == TTIE_PAIRS_INTRA_GROUP && grp[j] != gi) continue;
            if (share_vertex(ti, tri4[j])) continue;
            if (kWrite) pairs[out + cnt] = make_int2(i, j);
            ++cnt;
        }
        if (!kWrite) count[i] = cnt;
    }
}

}  // namespace

template <typename T> cudaError_t pack_positions(Ctx &c, const T *x, int stride, vec4_t<T> *out) {
    launch(c, k_pack_positions<T>, dim3(grid_for(c.V, kThreads)), dim3(kThreads), x, stride, c.V, out, c.ds);
    return cudaGetLastError();
}
template cudaError_t pack_positions<float>(Ctx &, const float *, int, float4 *);
template cudaError_t pack_positions<double>(Ctx &, const double *, int, dvec4 *);

cudaError_t pack_topology(Ctx &c, const int32_t *tri, const int32_t *group) {
    TTIE_CUDA_TRY(ensure(c, c.tri4, (size_t)c.F * sizeof(int4)));
    if (group) TTIE_CUDA_TRY(ensure(c, c.grp, (size_t)c.F * sizeof(int32_t)));
    launch(c, k_pack_topology, dim3(grid_for(c.F, kThreads)), dim3(kThreads), tri, group, c.F, c.V, (int4 *)c.tri4.p,
                                                                      (int32_t *)c.grp.p, c.ds);
    return cudaGetLastError();
}

static int mode_of(const Ctx &c) { return c.prm.pair_mode & 3; }

template <typename T>
cudaError_t build_candidates(Ctx &c, const vec4_t<T> *x0, const vec4_t<T> *x1, Buf &out_pairs, int64_t *n_out,
                             int64_t cap, bool refit_only) {
    const int n = (int)c.F;
    const int mode = mode_of(c);
    *n_out = 0;
    if (n < 2) return cudaSuccess;
    TTIE_CUDA_TRY(ensure(c, c.tbox, (size_t)n * sizeof(Box<T>)));
    TTIE_CUDA_TRY(ensure(c, c.mkey, (size_t)n * 8));
    TTIE_CUDA_TRY(ensure(c, c.mkey2, (size_t)n * 8));
    TTIE_CUDA_TRY(ensure(c, c.perm, (size_t)n * 4));
    TTIE_CUDA_TRY(ensure(c, c.perm2, (size_t)n * 4));
    TTIE_CUDA_TRY(ensure(c, c.node_box, (size_t)(2 * n - 1) * sizeof(Box<T>)));
    TTIE_CUDA_TRY(ensure(c, c.node_child, (size_t)(n - 1) * sizeof(int2)));
    TTIE_CUDA_TRY(ensure(c, c.node_parent, (size_t)(2 * n - 1) * sizeof(int)));
    TTIE_CUDA_TRY(ensure(c, c.node_range, (size_t)(2 * n - 1) * sizeof(int2)));
    TTIE_CUDA_TRY(ensure(c, c.visit, (size_t)(n - 1) * sizeof(unsigned int)));
    TTIE_CUDA_TRY(ensure(c, c.cand_cnt, (size_t)n * 4));
    TTIE_CUDA_TRY(ensure(c, c.cand_off, (size_t)(n + 1) * 8));
    const bool grouped = mode != TTIE_PAIRS_SELF;
    if (grouped) {
        TTIE_CUDA_TRY(ensure(c, c.leaf_group, (size_t)n * 4));
        TTIE_CUDA_TRY(ensure(c, c.group_range, (size_t)c.n_groups * sizeof(int2)));
    }
    Box<T> *tbox = (Box<T> *)c.tbox.p;
    auto *key = (unsigned long long *)c.mkey.p;
    auto *perm = (uint32_t *)c.perm.p;
    const unsigned g = grid_for(n, kThreads);

    int2 *child = (int2 *)c.node_child.p;
    int *parent = (int *)c.node_parent.p;
    int2 *range = (int2 *)c.node_range.p;
    Box<T> *nbox = (Box<T> *)c.node_box.p;
    if (!refit_only) c.tree_leaves = -1;
    launch(c, k_init_bounds, dim3(1), dim3(32), c.ds);
    launch(c, k_tri_boxes<T>, dim3(g), dim3(kThreads), x0, x1, (const int4 *)c.tri4.p, n, tbox, c.ds);
    if (c.prm.pair_mode & TTIE_PAIRS_HASH) {   // spatial hashing instead of the LBVH (hash.cu)
        c.tree_leaves = -1;
        return hash_candidates<T>(c, (const Box<T> *)tbox, out_pairs, n_out, cap);
    }
    if (!(refit_only && c.tree_leaves == n)) {
        const int gbits = grouped ? c.group_bits : 0;
        launch(c, k_morton<T>, dim3(g), dim3(kThreads), tbox, n, (const int32_t *)c.grp.p, gbits, c.ds, key, perm);
        TTIE_CUDA_TRY(cudaGetLastError());
        const int key_bits = 3 * ((63 - gbits) / 3) + gbits;
        TTIE_CUDA_TRY(radix_sort_graph(c, key, perm, (unsigned long long *)c.mkey2.p, (uint32_t *)c.perm2.p, n, key_bits));
        if (grouped) {
            launch(c, k_leaf_group, dim3(g), dim3(kThreads), perm, (const int32_t *)c.grp.p, n, (int32_t *)c.leaf_group.p);
            launch(c, k_fill_int2, dim3(grid_for(c.n_groups, kThreads)), dim3(kThreads), (int2 *)c.group_range.p,
                   c.n_groups, make_int2(1, 0));
            launch(c, k_group_ranges, dim3(g), dim3(kThreads), (const int32_t *)c.leaf_group.p, n,
                   (int2 *)c.group_range.p);
        }
        launch(c, k_karras, dim3(grid_for(n - 1, kThreads)), dim3(kThreads), key, n, child, parent, range);
        TTIE_CUDA_TRY(ensure(c, c.leaf_tri, (size_t)n * sizeof(int4)));
        launch(c, k_leaf_tri, dim3(g), dim3(kThreads), (const uint32_t *)perm, (const int4 *)c.tri4.p, n,
               (int4 *)c.leaf_tri.p);
        c.tree_leaves = n;
    }
    // a refit-only build keeps the hierarchy (and leaf order) of the last full build: any
    // hierarchy over the new boxes yields the same overlapping pairs
    launch(c, k_leaf_boxes<T>, dim3(g), dim3(kThreads), tbox, perm, n, nbox, range);
    TTIE_CUDA_TRY(cudaMemsetAsync(c.visit.p, 0, (size_t)(n - 1) * sizeof(unsigned int), c.stream));
    launch(c, k_refit<T>, dim3(g), dim3(kThreads), n, parent, child, nbox, (unsigned int *)c.visit.p, c.ds);
    launch(c, k_links<T>, dim3(grid_for(2 * (int64_t)n - 1, kThreads)), dim3(kThreads), n, (const int2 *)child,
           (const int2 *)range, nbox);
    auto *cnt = (uint32_t *)c.cand_cnt.p;
    auto *off = (unsigned long long *)c.cand_off.p;
    TTIE_CUDA_TRY(ensure(c, c.spill, (size_t)n * kSpill * sizeof(int2)));
    const bool one_walk = c.prm.traversal_mode == TTIE_TRAVERSAL_ONE_WALK;
    // the pool: n / 4 + 1024 chunks, or what the last walk needed (+ 25 %) if more; a walk that
    // runs past it falls back to the second walk and sizes the next pool
    const unsigned long long pool_chunks = std::max((unsigned long long)n / 4 + 1024, c.ovf_chunks);
    if (one_walk) {
        TTIE_CUDA_TRY(ensure(c, c.ovf_pool, (size_t)pool_chunks * kChunk * sizeof(int2)));
        TTIE_CUDA_TRY(ensure(c, c.ovf_next, (size_t)pool_chunks * sizeof(int)));
        TTIE_CUDA_TRY(ensure(c, c.ovf_head, (size_t)n * sizeof(int)));
        TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->ovf_cursor, 0, sizeof(unsigned long long), c.stream));
        launch(c, k_traverse<T, 0, true>, dim3(g), dim3(kThreads), n, (const int2 *)range, (const Box<T> *)nbox,
               (const int4 *)c.leaf_tri.p, (const int32_t *)c.leaf_group.p,
               (const int2 *)c.group_range.p, mode, cnt, (const unsigned long long *)nullptr, (int2 *)c.spill.p,
               (int2 *)nullptr, c.ds, (int2 *)c.ovf_pool.p, (int *)c.ovf_next.p, (int *)c.ovf_head.p, pool_chunks);
    } else {
        launch(c, k_traverse<T, 0>, dim3(g), dim3(kThreads), n, (const int2 *)range, (const Box<T> *)nbox,
               (const int4 *)c.leaf_tri.p, (const int32_t *)c.leaf_group.p,
               (const int2 *)c.group_range.p, mode, cnt, (const unsigned long long *)nullptr, (int2 *)c.spill.p,
               (int2 *)nullptr, c.ds, (int2 *)nullptr, (int *)nullptr, (int *)nullptr, 0ull);
    }
    TTIE_CUDA_TRY(cudaGetLastError());
    TTIE_CUDA_TRY(scan_u32_u64(c, cnt, off, n));
    unsigned long long total = 0;
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_cand, off + n, 8, cudaMemcpyDeviceToHost, c.stream));
    if (one_walk)
        TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->ovf_cursor, &c.ds->ovf_cursor, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    total = c.hs->n_cand;
    if (one_walk && c.hs->ovf_cursor > pool_chunks) c.ovf_chunks = c.hs->ovf_cursor + c.hs->ovf_cursor / 4;
    if ((int64_t)total > cap) {
        *n_out = (int64_t)total;
        return cudaSuccess;
    }
    TTIE_CUDA_TRY(ensure(c, out_pairs, (size_t)(total > 0 ? total : 1) * sizeof(int2)));
    if (total > 0) {
        launch(c, k_spill_copy, dim3(grid_for((int64_t)n * kSpill, kThreads)), dim3(kThreads), n, (const uint32_t *)cnt,
               (const unsigned long long *)off, (const int2 *)c.spill.p, (int2 *)out_pairs.p);
        if (one_walk && c.hs->ovf_cursor <= pool_chunks)
            launch(c, k_chunk_copy, dim3(g), dim3(kThreads), n, (const uint32_t *)cnt, (const unsigned long long *)off,
                   (const int2 *)c.ovf_pool.p, (const int *)c.ovf_next.p, (const int *)c.ovf_head.p, pool_chunks,
                   (int2 *)out_pairs.p);
        else
            launch(c, k_traverse<T, 1>, dim3(g), dim3(kThreads), n, (const int2 *)range, (const Box<T> *)nbox,
                   (const int4 *)c.leaf_tri.p, (const int32_t *)c.leaf_group.p,
                   (const int2 *)c.group_range.p, mode, cnt, (const unsigned long long *)off, (int2 *)nullptr,
                   (int2 *)out_pairs.p, c.ds, (int2 *)nullptr, (int *)nullptr, (int *)nullptr, 0ull);
    }
    *n_out = (int64_t)total;
    return cudaGetLastError();
}
template cudaError_t build_candidates<float>(Ctx &, const float4 *, const float4 *, Buf &, int64_t *, int64_t, bool);
template cudaError_t build_candidates<double>(Ctx &, const dvec4 *, const dvec4 *, Buf &, int64_t *, int64_t, bool);

namespace {
// Per-block sums of edge lengths, then one block adds the block sums in order.
template <typename T>
__global__ void k_edge_sum(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4, int64_t F,
                           double *partials) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        const int4 t = tri4[f];
        const v3<T> a = xyz<T>(x[t.x]), b = xyz<T>(x[t.y]), c = xyz<T>(x[t.z]);
        const v3<T> e0 = b - a, e1 = c - b, e2 = a - c;
        s += sqrt((double)dot(e0, e0)) + sqrt((double)dot(e1, e1)) + sqrt((double)dot(e2, e2));
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        partials[blockIdx.x] = t;
    }
}
__global__ void k_edge_mean(const double *partials, int n, int64_t F, double *out) {
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += partials[i];
        *out = F > 0 ? t / (3.0 * (double)F) : 0.0;
    }
}
}  // namespace

// Mean edge length over all triangles (fixed summation order).
template <typename T> cudaError_t mean_edge_length(Ctx &c, const vec4_t<T> *x, double *out_dev) {
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)kNumSMs * 16 * 4 * sizeof(double)));
    const unsigned g = grid_for(c.F, kThreads, kNumSMs * 4);
    launch(c, k_edge_sum<T>, dim3(g), dim3(kThreads), x, (const int4 *)c.tri4.p, c.F, (double *)c.partials.p);
    launch(c, k_edge_mean, dim3(1), dim3(32), (const double *)c.partials.p, (int)g, c.F, out_dev);
    return cudaGetLastError();
}
template cudaError_t mean_edge_length<float>(Ctx &, const float4 *, double *);
template cudaError_t mean_edge_length<double>(Ctx &, const dvec4 *, double *);

cudaError_t brute_candidates(Ctx &c, Buf &out_pairs, int64_t *n_out) {
    const int n = (int)c.F;
    const int mode = mode_of(c);
    *n_out = 0;
    if (n < 2) return cudaSuccess;
    TTIE_CUDA_TRY(ensure(c, c.cand_cnt, (size_t)n * 4));
    TTIE_CUDA_TRY(ensure(c, c.cand_off, (size_t)(n + 1) * 8));
    auto *cnt = (uint32_t *)c.cand_cnt.p;
    auto *off = (unsigned long long *)c.cand_off.p;
    const unsigned g = grid_for(n, 128);
    launch(c, k_brute<false>, dim3(g), dim3(128), n, (const int4 *)c.tri4.p, (const int32_t *)c.grp.p, mode, cnt, nullptr,
                                            nullptr);
    TTIE_CUDA_TRY(cudaGetLastError());
    TTIE_CUDA_TRY(scan_u32_u64(c, cnt, off, n));
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_cand, off + n, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    unsigned long long total = c.hs->n_cand;
    TTIE_CUDA_TRY(ensure(c, out_pairs, (size_t)(total > 0 ? total : 1) * sizeof(int2)));
    if (total > 0)
        launch(c, k_brute<true>, dim3(g), dim3(128), n, (const int4 *)c.tri4.p, (const int32_t *)c.grp.p, mode, nullptr,
                                               off, (int2 *)out_pairs.p);
    *n_out = (int64_t)total;
    return cudaGetLastError();
}

}  // namespace ttie
