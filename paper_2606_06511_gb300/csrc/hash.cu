// Spatial-hashing broad phase (§1.2 names spatial hashing as the structure that eliminates
// redundant pair tests), selected with the pair-mode flag TTIE_PAIRS_HASH.  Same contract as
// the LBVH: every pair i < j of the pair mode whose closed bounding boxes overlap and which
// shares no vertex index, each pair once.
//
// A uniform grid of cubic cells (side h = the mean of the boxes' largest sides): each triangle
// is listed in every cell its box touches, the (cell, triangle) list is sorted by cell (stable
// radix sort, so a cell's triangles stay in index order), and the pairs of each cell are tested.
// A pair whose boxes overlap is reported by one cell only: the cell holding the lower corner of
// the boxes' intersection, which both boxes touch.  The output order (cell, then triangle,
// then partner) is deterministic.  In the intra-group mode the group id prefixes the cell key,
// so cells never mix groups.
#include <algorithm>

#include "common.cuh"

namespace ttie {

namespace {

constexpr int kThreads = 256;
constexpr long long kMaxCellsPerTri = 1 << 16;

// Per-block minima of the box lower corners, maxima of the upper corners and sums of the
// boxes' largest sides (7 values per block).
template <typename T>
__global__ void k_hash_partials(const Box<T> *__restrict__ box, int64_t F, double *partials) {
    __shared__ double sh[7][kThreads / 32];
    double v[7] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0.0};
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        const Box<T> b = box[f];
        v[0] = fmin(v[0], (double)b.lo.x); v[1] = fmin(v[1], (double)b.lo.y); v[2] = fmin(v[2], (double)b.lo.z);
        v[3] = fmax(v[3], (double)b.hi.x); v[4] = fmax(v[4], (double)b.hi.y); v[5] = fmax(v[5], (double)b.hi.z);
        v[6] += fmax((double)b.hi.x - b.lo.x, fmax((double)b.hi.y - b.lo.y, (double)b.hi.z - b.lo.z));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            v[k] = fmin(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
            v[3 + k] = fmax(v[3 + k], __shfl_xor_sync(0xffffffffu, v[3 + k], o));
        }
        v[6] += __shfl_xor_sync(0xffffffffu, v[6], o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 7; ++k) sh[k][w] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[7] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0.0};
        for (int q = 0; q < kThreads / 32; ++q) {
            for (int k = 0; k < 3; ++k) {
                r[k] = fmin(r[k], sh[k][q]);
                r[3 + k] = fmax(r[3 + k], sh[3 + k][q]);
            }
            r[6] += sh[6][q];
        }
        for (int k = 0; k < 7; ++k) partials[blockIdx.x * 7 + k] = r[k];
    }
}

// Grid: origin, cell side, and the bits per axis of the cell coordinates.
struct Grid {
    double org[3], h;
    int bits;
};

// Cell side = the mean of the boxes' largest sides, enlarged when the scene would need more
// cells along an axis than the key holds.  Partials added in block order (deterministic).
__global__ void k_hash_grid(const double *partials, int n_blocks, int64_t F, int group_bits, Grid *grid) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, ext = 0.0;
    for (int b = 0; b < n_blocks; ++b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], partials[b * 7 + k]);
            hi[k] = fmax(hi[k], partials[b * 7 + 3 + k]);
        }
        ext += partials[b * 7 + 6];
    }
    Grid g;
    g.bits = min(20, (64 - group_bits) / 3);
    double h = F > 0 ? ext / (double)F : 1.0;
    double span = 0.0;
    for (int k = 0; k < 3; ++k) span = fmax(span, hi[k] - lo[k]);
    const double cells = (double)((1ll << g.bits) - 2);
    if (!(h > 0.0)) h = span > 0.0 ? span / cells : 1.0;
    if (span / h > cells) h = span / cells;
    for (int k = 0; k < 3; ++k) g.org[k] = lo[k];
    g.h = h;
    *grid = g;
}

template <typename T>
__device__ __forceinline__ void cell_range(const Box<T> &b, const Grid &g, int lo[3], int hi[3]) {
    const double bl[3] = {(double)b.lo.x, (double)b.lo.y, (double)b.lo.z};
    const double bh[3] = {(double)b.hi.x, (double)b.hi.y, (double)b.hi.z};
    const int cmax = (1 << g.bits) - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = min(cmax, max(0, (int)floor((bl[k] - g.org[k]) / g.h)));
        hi[k] = min(cmax, max(0, (int)floor((bh[k] - g.org[k]) / g.h)));
    }
}

template <typename T>
__global__ void k_cell_count(const Box<T> *__restrict__ box, int64_t F, const Grid *grid, uint32_t *__restrict__ cnt,
                             DevScalars *ds) {
    const Grid g = *grid;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        int lo[3], hi[3];
        cell_range<T>(box[f], g, lo, hi);
        const long long n = (long long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
        if (n > kMaxCellsPerTri) {
            atomicOr(&ds->err, ERR_STACK);
            cnt[f] = 0;
        } else {
            cnt[f] = (uint32_t)n;
        }
    }
}

__device__ __forceinline__ unsigned long long cell_key(int cx, int cy, int cz, int bits, unsigned long long gprefix) {
    return gprefix | ((unsigned long long)cx << (2 * bits)) | ((unsigned long long)cy << bits) | (unsigned long long)cz;
}

template <typename T>
__global__ void k_cell_emit(const Box<T> *__restrict__ box, int64_t F, const Grid *grid, const int32_t *__restrict__ grp,
                            int group_bits, const uint32_t *__restrict__ cnt, const unsigned long long *__restrict__ off,
                            unsigned long long *__restrict__ key, uint32_t *__restrict__ val) {
    const Grid g = *grid;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        if (cnt[f] == 0) continue;
        int lo[3], hi[3];
        cell_range<T>(box[f], g, lo, hi);
        const unsigned long long gp = group_bits ? (unsigned long long)grp[f] << (3 * g.bits) : 0ull;
        unsigned long long o = off[f];
        for (int cx = lo[0]; cx <= hi[0]; ++cx)
            for (int cy = lo[1]; cy <= hi[1]; ++cy)
                for (int cz = lo[2]; cz <= hi[2]; ++cz) {
                    key[o] = cell_key(cx, cy, cz, g.bits, gp);
                    val[o] = (uint32_t)f;
                    ++o;
                }
    }
}

template <typename T>
__device__ __forceinline__ bool closed_overlap(const Box<T> &a, const Box<T> &b) {
    return a.lo.x <= b.hi.x && b.lo.x <= a.hi.x && a.lo.y <= b.hi.y && b.lo.y <= a.hi.y && a.lo.z <= b.hi.z &&
           b.lo.z <= a.hi.z;
}

__device__ __forceinline__ bool shares_vertex(int4 a, int4 b) {
    return a.x == b.x || a.x == b.y || a.x == b.z || a.y == b.x || a.y == b.y || a.y == b.z || a.z == b.x ||
           a.z == b.y || a.z == b.z;
}

// Pairs of every (cell, triangle) entry with the later entries of the same cell.  Pass 0
// counts, pass 1 writes at offset[e].
template <typename T, int kPass>
__global__ void k_cell_pairs(const unsigned long long *__restrict__ key, const uint32_t *__restrict__ val, int64_t n,
                             const Box<T> *__restrict__ box, const int4 *__restrict__ tri4,
                             const int32_t *__restrict__ grp, int mode, const Grid *grid, uint32_t *__restrict__ cnt,
                             const unsigned long long *__restrict__ offset, int2 *__restrict__ pairs, DevScalars *ds) {
    const Grid g = *grid;
    const unsigned long long cmask = (1ull << g.bits) - 1ull;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[e];
        const int cx = (int)((k >> (2 * g.bits)) & cmask), cy = (int)((k >> g.bits) & cmask), cz = (int)(k & cmask);
        const uint32_t i = val[e];
        const Box<T> bi = box[i];
        const int4 ti = tri4[i];
        const int gi = grp ? grp[i] : 0;
        uint32_t c = 0;
        const unsigned long long out = kPass == 1 ? offset[e] : 0ull;
        for (int64_t e2 = e + 1; e2 < n && key[e2] == k; ++e2) {
            const uint32_t j = val[e2];
            if (mode == TTIE_PAIRS_INTER_GROUP && grp[j] == gi) continue;
            const Box<T> bj = box[j];
            if (!closed_overlap<T>(bi, bj)) continue;
            // report in the cell of the lower corner of the intersection only
            Box<T> ix;
            ix.lo.x = bi.lo.x > bj.lo.x ? bi.lo.x : bj.lo.x;
            ix.lo.y = bi.lo.y > bj.lo.y ? bi.lo.y : bj.lo.y;
            ix.lo.z = bi.lo.z > bj.lo.z ? bi.lo.z : bj.lo.z;
            ix.hi = ix.lo;
            int lo[3], hi[3];
            cell_range<T>(ix, g, lo, hi);
            if (lo[0] != cx || lo[1] != cy || lo[2] != cz) continue;
            if (shares_vertex(ti, tri4[j])) continue;
            if (kPass == 1 && !TTIE_BAD(ds, out + c < offset[e + 1], 62, out + c))
                pairs[out + c] = make_int2((int)min(i, j), (int)max(i, j));
            ++c;
        }
        if (kPass == 0) cnt[e] = c;
    }
}

}  // namespace

template <typename T>
cudaError_t hash_candidates(Ctx &c, const Box<T> *box, Buf &out_pairs, int64_t *n_out, int64_t cap) {
    const int64_t F = c.F;
    const int mode = c.prm.pair_mode & 3;
    const int gbits = mode == TTIE_PAIRS_INTRA_GROUP ? c.group_bits : 0;
    *n_out = 0;
    if (F < 2) return cudaSuccess;
    const unsigned gb = grid_for(F, kThreads, (int64_t)kNumSMs * 4);
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)gb * 7 * sizeof(double)));
    TTIE_CUDA_TRY(ensure(c, c.hgrid, sizeof(Grid)));
    launch(c, k_hash_partials<T>, dim3(gb), dim3(kThreads), box, F, (double *)c.partials.p);
    launch(c, k_hash_grid, dim3(1), dim3(32), (const double *)c.partials.p, (int)gb, F, gbits, (Grid *)c.hgrid.p);
    TTIE_CUDA_TRY(ensure(c, c.cand_cnt, (size_t)F * 4));
    TTIE_CUDA_TRY(ensure(c, c.cand_off, (size_t)(F + 1) * 8));
    auto *cnt = (uint32_t *)c.cand_cnt.p;
    auto *off = (unsigned long long *)c.cand_off.p;
    launch(c, k_cell_count<T>, dim3(grid_for(F, kThreads)), dim3(kThreads), box, F, (const Grid *)c.hgrid.p, cnt, c.ds);
    TTIE_CUDA_TRY(scan_u32_u64(c, cnt, off, F));
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_cand, off + F, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    const int64_t n_ent = (int64_t)c.hs->n_cand;
    if (n_ent < 2) return cudaSuccess;
    TTIE_CUDA_TRY(ensure(c, c.hkey, (size_t)n_ent * 8));
    TTIE_CUDA_TRY(ensure(c, c.hkey2, (size_t)n_ent * 8));
    TTIE_CUDA_TRY(ensure(c, c.hval, (size_t)n_ent * 4));
    TTIE_CUDA_TRY(ensure(c, c.hval2, (size_t)n_ent * 4));
    auto *key = (unsigned long long *)c.hkey.p;
    auto *val = (uint32_t *)c.hval.p;
    launch(c, k_cell_emit<T>, dim3(grid_for(F, kThreads)), dim3(kThreads), box, F, (const Grid *)c.hgrid.p,
           (const int32_t *)c.grp.p, gbits, (const uint32_t *)cnt, (const unsigned long long *)off, key, val);
    TTIE_CUDA_TRY(cudaGetLastError());
    // bits of the key: 3 x bits per axis + group bits (bits per axis is at most 20 and
    // (64 - group bits) / 3; the grid kernel chose it, recompute the same value here)
    const int bits = std::min(20, (64 - gbits) / 3);
    TTIE_CUDA_TRY(radix_sort(c, key, val, (unsigned long long *)c.hkey2.p, (uint32_t *)c.hval2.p, n_ent, 3 * bits + gbits));
    TTIE_CUDA_TRY(ensure(c, c.hcnt, (size_t)n_ent * 4));
    TTIE_CUDA_TRY(ensure(c, c.hoff, (size_t)(n_ent + 1) * 8));
    auto *pc = (uint32_t *)c.hcnt.p;
    auto *po = (unsigned long long *)c.hoff.p;
    const int32_t *grp = c.have_group ? (const int32_t *)c.grp.p : nullptr;
    launch(c, k_cell_pairs<T, 0>, dim3(grid_for(n_ent, kThreads)), dim3(kThreads), (const unsigned long long *)key,
           (const uint32_t *)val, n_ent, box, (const int4 *)c.tri4.p, grp, mode, (const Grid *)c.hgrid.p, pc,
           (const unsigned long long *)nullptr, (int2 *)nullptr, c.ds);
    TTIE_CUDA_TRY(scan_u32_u64(c, pc, po, n_ent));
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_cand, po + n_ent, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    const int64_t total = (int64_t)c.hs->n_cand;
    if (total > cap) {
        *n_out = total;
        return cudaSuccess;
    }
    TTIE_CUDA_TRY(ensure(c, out_pairs, (size_t)(total > 0 ? total : 1) * sizeof(int2)));
    if (total > 0)
        launch(c, k_cell_pairs<T, 1>, dim3(grid_for(n_ent, kThreads)), dim3(kThreads), (const unsigned long long *)key,
               (const uint32_t *)val, n_ent, box, (const int4 *)c.tri4.p, grp, mode, (const Grid *)c.hgrid.p, pc,
               (const unsigned long long *)po, (int2 *)out_pairs.p, c.ds);
    *n_out = total;
    return cudaGetLastError();
}
template cudaError_t hash_candidates<float>(Ctx &, const Box<float> *, Buf &, int64_t *, int64_t);
template cudaError_t hash_candidates<double>(Ctx &, const Box<double> *, Buf &, int64_t *, int64_t);

}  // namespace ttie
