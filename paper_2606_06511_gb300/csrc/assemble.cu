// Assembly of the PSD Hessian and gradient into 3x3 block CSR, and the PCG solve.
//
// Per intersecting pair with a = t_c^0, b = t_c^1, u = grad a, v = grad b:
//   gradient (Eq. 3)      g  = 2ab (b u + a v)
//   Hessian (Eq. 4)       H  = 2b^2 uu' + 2a^2 vv' + 4ab (vu' + uv')
// Eigen-analysis (§1.1): parts 1 and 2 are PSD; part 3 = 4ab(uv' + vu') has the
// eigenpairs 4ab(u.v +- |u||v|) on u^ +- v^, and on an intersecting pair (ab < 0)
// only 4ab(u.v - |u||v|) >= 0 survives the projection.  So
//   H+ = z1 z1' + z2 z2' + z3 z3',  z1 = sqrt2 |b| u,  z2 = sqrt2 |a| v,
//   z3 = sqrt(2 |ab| |u||v|) (u^ - v^)          (z3 = 0 for DROP_CROSS)
// and no 18x18 eigen-solve is needed.  WHOLE projects the sum instead: H = G M G' with
// G = [u v] and M = [[2b^2, 4ab], [4ab, 2a^2]] (det M = -12 a^2 b^2 < 0), so with G = QR
// (Gram-Schmidt) the non-zero spectrum of H is that of the 2x2 S = R M R', which has one
// positive eigenvalue; H+ = z1 z1' with z1 = sqrt(lambda+) Q e+.
//
// Assembly: 36 vertex-block keys (row, col) per pair, a stable radix sort, and
// one thread per distinct key summing its run in sorted order, so both the
// pattern and the values are deterministic.
#include "common.cuh"
#include "pcg_common.cuh"

namespace ttie {

namespace {

constexpr int kThreads = 256;
// Per intersecting pair, for each of its 6 vertices r: [z1 (3), z2 (3), z3 (3), g (3)] (the
// rows 3r..3r+2 of the three PSD factors and of the gradient), so a 3x3 block (r, c) reads
// two contiguous 36-byte runs.
constexpr int kZStride = 72;
constexpr int kZVertex = 12;

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
    __shared__ T sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T r = T(0);
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
#pragma unroll
        for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// Deterministic grid sums of N values; the last block to finish runs `fin` on the totals.
template <int N, typename Fin>
__device__ __forceinline__ void grid_sums(const double (&v)[N], double *partials, unsigned int *ticket, Fin fin) {
    __shared__ bool last;
    double b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] = block_sum(v[i]);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) partials[(size_t)i * gridDim.x + blockIdx.x] = b[i];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        double tot[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (unsigned j = threadIdx.x; j < gridDim.x; j += blockDim.x) s += __ldcg(&partials[(size_t)i * gridDim.x + j]);
            tot[i] = block_sum(s);
        }
        if (threadIdx.x == 0) {
            fin(tot);
            *ticket = 0u;
        }
    }
}

__global__ void k_mark_vertices(const int4 *__restrict__ tri4, const int2 *__restrict__ pairs,
                                const uint32_t *__restrict__ active, const DevScalars *ds, uint32_t *__restrict__ vflag) {
    const unsigned long long n = ds->n_active;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        int2 pr = pairs[active[k]];
        int4 a = tri4[pr.x], b = tri4[pr.y];
        vflag[a.x] = 1; vflag[a.y] = 1; vflag[a.z] = 1;
        vflag[b.x] = 1; vflag[b.y] = 1; vflag[b.z] = 1;
    }
}

__global__ void k_row_vertex(const uint32_t *__restrict__ vflag, const unsigned long long *__restrict__ vrow, int64_t V,
                             int32_t *__restrict__ row_vertex, DevScalars *ds) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        if (vflag[v]) row_vertex[vrow[v]] = (int32_t)v;
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->n_rows = vrow[V];
}

// Rank-one projection of the whole Eq. 4 Hessian: z = alpha u + beta v.
template <typename T>
__device__ __forceinline__ void whole_projection(T a, T b, T uu, T uv, T vv, T &alpha, T &beta) {
    alpha = beta = T(0);
    const T m11 = T(2) * b * b, m12 = T(4) * a * b, m22 = T(2) * a * a;
    if (!(uu > T(0))) {                       // G = [0 v]: H = 2a^2 vv'
        if (vv > T(0)) beta = sqrt(m22);
        return;
    }
    const T nu = sqrt(uu);
    const T r12 = uv / nu;                    // R = [[|u|, u.v/|u|], [0, |w|]], w = v - (v.q1) q1
    const T w2 = vv - r12 * r12;
    const T r22 = w2 > T(0) ? sqrt(w2) : T(0);
    // S = R M R'
    const T s11 = nu * nu * m11 + T(2) * nu * r12 * m12 + r12 * r12 * m22;
    const T s12 = r22 * (nu * m12 + r12 * m22);
    const T s22 = r22 * r22 * m22;
    const T hm = T(0.5) * (s11 + s22), hd = T(0.5) * (s11 - s22);
    const T lam = hm + sqrt(hd * hd + s12 * s12);
    if (!(lam > T(0))) return;
    // eigenvector of the larger eigenvalue: the better conditioned of (s12, lam - s11), (lam - s22, s12)
    T e1 = s12, e2 = lam - s11;
    const T f1 = lam - s22, f2 = s12;
    if (f1 * f1 + f2 * f2 > e1 * e1 + e2 * e2) { e1 = f1; e2 = f2; }
    const T en = sqrt(e1 * e1 + e2 * e2);
    if (!(en > T(0))) { alpha = sqrt(lam) / nu; return; }
    const T c = sqrt(lam) / en;
    // Q e = e1 u/|u| + e2 (v - (u.v/|u|^2) u)/|w|
    if (r22 > T(0)) {
        beta = c * e2 / r22;
        alpha = c * e1 / nu - beta * uv / uu;
    } else {
        alpha = c * e1 / nu;
    }
}

// PSD factors z1, z2, z3 and the gradient of each intersecting pair; trace of H+.
template <typename T>
__global__ void k_factors(const T *__restrict__ fac, int psd_mode, T *__restrict__ z, double *partials, DevScalars *ds) {
    const unsigned long long n = ds->n_active;
    double tr = 0.0;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const T *r = fac + k * kFacStride;
        const T a = r[0], b = r[1];
        T uu = 0, vv = 0, uv = 0;
#pragma unroll
        for (int i = 0; i < 18; ++i) {
            uu += r[2 + i] * r[2 + i];
            vv += r[20 + i] * r[20 + i];
            uv += r[2 + i] * r[20 + i];
        }
        const T nu = sqrt(uu), nv = sqrt(vv);
        T c1 = sqrt(T(2)) * fabs(b), c2 = sqrt(T(2)) * fabs(a);
        T c3 = T(0), iu = T(0), iv = T(0), wa = T(0), wb = T(0);
        if (psd_mode == TTIE_PSD_PER_PART && nu > T(0) && nv > T(0)) {
            c3 = sqrt(T(2) * fabs(a * b) * nu * nv);
            iu = T(1) / nu;
            iv = T(1) / nv;
        } else if (psd_mode == TTIE_PSD_WHOLE) {
            whole_projection(a, b, uu, uv, vv, wa, wb);
            c1 = c2 = T(0);
        }
        T *o = z + k * kZStride;
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < 18; ++i) {
            const T u = r[2 + i], v = r[20 + i];
            const T z1 = c1 * u + (wa * u + wb * v), z2 = c2 * v, z3 = c3 * (u * iu - v * iv);
            T *ov = o + (i / 3) * kZVertex + i % 3;
            ov[0] = z1;
            ov[3] = z2;
            ov[6] = z3;
            ov[9] = T(2) * a * b * (b * u + a * v);
            t += (double)z1 * z1 + (double)z2 * z2 + (double)z3 * z3;
        }
        tr += t;
    }
    double v[1] = {tr};
    grid_sums<1>(v, partials, &ds->done_counter[1], [&](const double *tot) { ds->trace = tot[0]; });
}

__device__ __forceinline__ int vid(int4 a, int4 b, int r) {
    return r == 0 ? a.x : r == 1 ? a.y : r == 2 ? a.z : r == 3 ? b.x : r == 4 ? b.y : b.z;
}

// One thread per block entry (pair k, vertex rows r and c), so the keys and values are written
// contiguously.
__global__ void k_block_keys(const int4 *__restrict__ tri4, const int2 *__restrict__ pairs,
                             const uint32_t *__restrict__ active, const unsigned long long *__restrict__ vrow,
                             const DevScalars *ds, unsigned long long *__restrict__ key, uint32_t *__restrict__ val) {
    const unsigned long long n = ds->n_active * 36, nr = ds->n_rows;
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; e < n;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long k = e / 36;
        const int rc = (int)(e - k * 36), r = rc / 6, c = rc - r * 6;
        const int2 pr = pairs[active[k]];
        const int4 a = tri4[pr.x], b = tri4[pr.y];
        unsigned long long rr = vrow[vid(a, b, r)], cc = vrow[vid(a, b, c)];
        if (TTIE_BAD((DevScalars *)ds, rr < nr, 11, rr)) rr = 0;
        if (TTIE_BAD((DevScalars *)ds, cc < nr, 11, cc)) cc = 0;
        key[e] = rr * nr + cc;
        val[e] = (uint32_t)e;
    }
}

// ---------------------------------------------------------------- elastic term
// The quasi-static simulation of Fig. 2 adds an elastic term to sum T; the paper does not
// state its model, so it is a mass-spring term here: springs k/2 (|x_i - x_j| - L)^2 and
// anchors k_a/2 |x_v - t_v|^2.  Per spring, with l = |x_i - x_j| and n = (x_i - x_j)/l: the
// gradient is k (l - L) n on i (minus that on j) and the Hessian [[K, -K], [-K, K]] with
// K = k (n n' + (1 - L/l)(I - n n')).  Its spectrum is twice K's (k along n, k (1 - L/l)
// twice across n) and three zeros, so the PSD projection only clamps 1 - L/l at 0:
// K+ = k (c I + (1 - c) n n'), c = max(0, 1 - L/l).  At l = 0: K+ = k I, gradient 0.  An
// anchor adds k_a I and k_a (x_v - t_v).  In the assembly a spring contributes four block
// entries (+K+ on (i,i) and (j,j), -K+ on (i,j) and (j,i)) and an anchor one, after the
// pairs' 36 per pair, so the same sort and segmented sums merge both patterns.
constexpr int kElStride = 12;   // per spring: K+ (9, row-major), gradient on i (3)

// Energy of the term at x (and, with sfac, each spring's K+ and gradient, each anchor's
// gradient, and the term's trace added to ds->trace).
template <typename T>
__global__ void k_el_factors(const vec4_t<T> *__restrict__ x, const int2 *__restrict__ edges,
                             const T *__restrict__ rest, int64_t n_edges, T k, const int32_t *__restrict__ anchors,
                             const T *__restrict__ targets, int64_t n_anchors, T ka, T *__restrict__ sfac,
                             T *__restrict__ afac, double *partials, DevScalars *ds) {
    double en = 0.0, tr = 0.0;
    const int64_t n = n_edges + n_anchors;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n_edges) {
            const int2 e = edges[i];
            const vec4_t<T> xi = x[e.x], xj = x[e.y];
            const T d[3] = {xi.x - xj.x, xi.y - xj.y, xi.z - xj.z};
            const T l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const T L = rest[i];
            en += 0.5 * (double)k * ((double)l - (double)L) * ((double)l - (double)L);
            if (sfac) {
                T *o = sfac + (size_t)i * kElStride;
                if (l > T(0)) {
                    const T nv[3] = {d[0] / l, d[1] / l, d[2] / l};
                    const T c = max(T(0), T(1) - L / l);
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) o[3 * r + q] = k * ((r == q ? c : T(0)) + (T(1) - c) * nv[r] * nv[q]);
                        o[9 + r] = k * (l - L) * nv[r];
                    }
                    tr += 2.0 * (double)k * (1.0 + 2.0 * (double)c);
                } else {
#pragma unroll
                    for (int r = 0; r < 9; ++r) o[r] = (r % 4 == 0) ? k : T(0);
                    o[9] = o[10] = o[11] = T(0);
                    tr += 6.0 * (double)k;
                }
            }
        } else {
            const int64_t a = i - n_edges;
            const vec4_t<T> xv = x[anchors[a]];
            const T d[3] = {xv.x - targets[3 * a], xv.y - targets[3 * a + 1], xv.z - targets[3 * a + 2]};
            en += 0.5 * (double)ka * ((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
            if (sfac) {
#pragma unroll
                for (int r = 0; r < 3; ++r) afac[3 * a + r] = ka * d[r];
                tr += 3.0 * (double)ka;
            }
        }
    }
    double v[2] = {en, tr};
    const bool with_trace = sfac != nullptr;
    grid_sums<2>(v, partials, &ds->done_counter[6], [&](const double *tot) {
        ds->el_energy = tot[0];
        if (with_trace) ds->trace += tot[1];
    });
}

// Vertices of springs and anchors are rows of the system.
__global__ void k_el_mark(const int2 *__restrict__ edges, int64_t n_edges, const int32_t *__restrict__ anchors,
                          int64_t n_anchors, uint32_t *__restrict__ vflag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_edges + n_anchors;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n_edges) {
            const int2 e = edges[i];
            vflag[e.x] = 1;
            vflag[e.y] = 1;
        } else {
            vflag[anchors[i - n_edges]] = 1;
        }
    }
}

// Block entries of springs (4 each) and anchors (1 each) at base + ..., values index themselves.
__global__ void k_el_keys(const int2 *__restrict__ edges, int64_t n_edges, const int32_t *__restrict__ anchors,
                          int64_t n_anchors, const unsigned long long *__restrict__ vrow, const DevScalars *ds,
                          unsigned long long base, unsigned long long *__restrict__ key, uint32_t *__restrict__ val) {
    const unsigned long long nr = ds->n_rows;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_edges + n_anchors;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n_edges) {
            const int2 e = edges[i];
            const unsigned long long ri = vrow[e.x], rj = vrow[e.y], o = base + 4 * (unsigned long long)i;
            key[o] = ri * nr + ri;
            key[o + 1] = ri * nr + rj;
            key[o + 2] = rj * nr + ri;
            key[o + 3] = rj * nr + rj;
#pragma unroll
            for (int q = 0; q < 4; ++q) val[o + q] = (uint32_t)(o + q);
        } else {
            const unsigned long long r = vrow[anchors[i - n_edges]], o = base + 4 * (unsigned long long)n_edges + (i - n_edges);
            key[o] = r * nr + r;
            val[o] = (uint32_t)o;
        }
    }
}

// Spring endpoints distinct and in [0, V), anchors in [0, V).
__global__ void k_el_check(const int2 *__restrict__ edges, int64_t n_edges, const int32_t *__restrict__ anchors,
                           int64_t n_anchors, int64_t V, DevScalars *ds) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_edges + n_anchors;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool ok;
        if (i < n_edges) {
            const int2 e = edges[i];
            ok = e.x >= 0 && e.x < V && e.y >= 0 && e.y < V && e.x != e.y;
        } else {
            const int a = anchors[i - n_edges];
            ok = a >= 0 && a < V;
        }
        if (!ok) atomicOr(&ds->err, ERR_BAD_INDEX);
    }
}

__global__ void k_run_flags(const unsigned long long *__restrict__ key, int64_t n, uint32_t *__restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

__global__ void k_run_starts(const uint32_t *__restrict__ flag, const unsigned long long *__restrict__ pos, int64_t n,
                             uint32_t *__restrict__ run_start, DevScalars *ds) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) run_start[pos[i]] = (uint32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long nb = pos[n];
        run_start[nb] = (uint32_t)n;
        ds->nnzb = nb;
    }
}

// One thread per stored block: pattern, then the sum over its run in sorted order.
// One entry of a block (row, col), added in place.  Pair entry (pk, r, c): z_t[r] z_t[c]^T for
// the three PSD factors t, and on the diagonal the gradient rows of r.  Spring entry q (0: (i, i),
// 1: (i, j), 2: (j, i), 3: (j, j)): +-K+, and on the diagonal +-the gradient on i.  Anchor: k_a I
// and its gradient.
template <typename T>
__device__ __forceinline__ void add_pair_entry(const T *__restrict__ z, uint32_t pk, uint32_t r, uint32_t c, bool diag,
                                               T (&m)[9], T &g0, T &g1, T &g2) {
    const T *zr = z + (size_t)pk * kZStride + r * kZVertex, *zc = z + (size_t)pk * kZStride + c * kZVertex;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const T x0 = zr[3 * t], x1 = zr[3 * t + 1], x2 = zr[3 * t + 2];
        const T y0 = zc[3 * t], y1 = zc[3 * t + 1], y2 = zc[3 * t + 2];
        m[0] += x0 * y0; m[1] += x0 * y1; m[2] += x0 * y2;
        m[3] += x1 * y0; m[4] += x1 * y1; m[5] += x1 * y2;
        m[6] += x2 * y0; m[7] += x2 * y1; m[8] += x2 * y2;
    }
    if (diag) {
        g0 += zr[9]; g1 += zr[10]; g2 += zr[11];
    }
}
template <typename T>
__device__ __forceinline__ void add_spring_entry(const T *__restrict__ sfac, unsigned long long sp, unsigned q, bool diag,
                                                 T (&m)[9], T &g0, T &g1, T &g2) {
    const T *K = sfac + sp * kElStride;
    const T sg = (q == 0 || q == 3) ? T(1) : T(-1);
#pragma unroll
    for (int t = 0; t < 9; ++t) m[t] += sg * K[t];
    if (diag) {   // (i, i): the gradient on i; (j, j): on j, its negative
        const T gs = q == 0 ? T(1) : T(-1);
        g0 += gs * K[9]; g1 += gs * K[10]; g2 += gs * K[11];
    }
}
template <typename T>
__device__ __forceinline__ void add_anchor_entry(const T *__restrict__ afac, unsigned long long an, T ka, bool diag,
                                                 T (&m)[9], T &g0, T &g1, T &g2) {
    m[0] += ka; m[4] += ka; m[8] += ka;
    if (diag) { g0 += afac[3 * an]; g1 += afac[3 * an + 1]; g2 += afac[3 * an + 2]; }
}

template <typename T>
__global__ void k_block_values(const unsigned long long *__restrict__ key, const uint32_t *__restrict__ val,
                               const uint32_t *__restrict__ run_start, const T *__restrict__ z, const DevScalars *ds,
                               int32_t *__restrict__ row_ptr, int32_t *__restrict__ col_idx, T *__restrict__ bval,
                               T *__restrict__ grad_rows, const int32_t *__restrict__ row_vertex,
                               T *__restrict__ grad_full, unsigned long long n_entries, const T *__restrict__ sfac,
                               int64_t n_springs, const T *__restrict__ afac, T ka) {
    const unsigned long long nb = ds->nnzb, nr = ds->n_rows, n_pair = ds->n_active * 36;
    for (unsigned long long bi = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; bi < nb;
         bi += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t s = run_start[bi], e = run_start[bi + 1];
        if (TTIE_BAD((DevScalars *)ds, s < e && e <= n_entries, 21, ((long long)s << 32) | e)) continue;
        const unsigned long long kk = key[s];
        const unsigned long long row = kk / nr, col = kk - row * nr;
        if (TTIE_BAD((DevScalars *)ds, row < nr, 22, row)) continue;
        col_idx[bi] = (int32_t)col;
        if (bi == 0 || key[run_start[bi - 1]] / nr != row) row_ptr[row] = (int32_t)bi;
        if (bi == nb - 1) row_ptr[nr] = (int32_t)nb;
        T m[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) m[i] = T(0);
        T g0 = 0, g1 = 0, g2 = 0;
        for (uint32_t i = s; i < e; ++i) {
            const uint32_t v = val[i];
            if (v >= n_pair) {   // elastic entries
                const unsigned long long w = v - n_pair;
                if (w < 4ull * (unsigned long long)n_springs) {
                    const unsigned long long sp = w / 4, q = w - sp * 4;
                    add_spring_entry<T>(sfac, sp, (unsigned)q, row == col, m, g0, g1, g2);
                } else {
                    add_anchor_entry<T>(afac, w - 4ull * (unsigned long long)n_springs, ka, row == col, m, g0, g1, g2);
                }
                continue;
            }
            const uint32_t pk = v / 36, rc = v - pk * 36, r = rc / 6, c = rc - r * 6;
            if (TTIE_BAD((DevScalars *)ds, pk < ds->n_active, 23, pk)) continue;
            add_pair_entry<T>(z, pk, r, c, row == col, m, g0, g1, g2);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) bval[bi * 9 + i] = m[i];
        if (row == col) {
            grad_rows[row * 3] = g0; grad_rows[row * 3 + 1] = g1; grad_rows[row * 3 + 2] = g2;
            if (grad_full) {
                const int64_t v = row_vertex[row];
                grad_full[v * 3] = g0; grad_full[v * 3 + 1] = g1; grad_full[v * 3 + 2] = g2;
            }
        }
    }
}

// ---------------------------------------------------------------- assembly by row buckets
// The same system without a global sort.  An item is what one row receives from one source:
// pair k's vertex r (code 6k + r, six entries: columns of the pair's six vertices), spring s's
// end (code 6 n_act + 2s + side, two entries: columns of i and j) or anchor a (code
// 6 n_act + 2 n_springs + a, one entry).  Items are counted and bucketed per row (in arrival
// order), then one warp per row orders its items by code, lists each item's entry columns,
// and finds the distinct columns in ascending order; after a scan of their counts, one warp
// per row sums, for each distinct column, the entries in item order.  Within a block (row, col)
// a source has one entry, so item order is the entry order of the sorted-key assembly (pair
// index, then springs, then anchors) and every value is the same sum in the same order.

// the row and the number of entries of item code
__device__ __forceinline__ void item_row(uint32_t code, unsigned long long n_pair_items, int64_t n_springs,
                                         const int4 *__restrict__ tri4, const int2 *__restrict__ pairs,
                                         const uint32_t *__restrict__ active, const unsigned long long *__restrict__ vrow,
                                         const int2 *__restrict__ edges, const int32_t *__restrict__ anchors,
                                         unsigned long long &row) {
    if (code < n_pair_items) {
        const uint32_t k = code / 6, r = code - k * 6;
        const int2 pr = pairs[active[k]];
        row = vrow[vid(tri4[pr.x], tri4[pr.y], (int)r)];
    } else if ((unsigned long long)code - n_pair_items < 2ull * (unsigned long long)n_springs) {
        const unsigned long long w = code - n_pair_items, sp = w / 2;
        const int2 e = edges[sp];
        row = vrow[(w - 2 * sp) ? e.y : e.x];
    } else {
        row = vrow[anchors[code - n_pair_items - 2ull * (unsigned long long)n_springs]];
    }
}

// count (fill = false) or place (fill = true) every item in its row's bucket
template <bool kFill>
__global__ void k_row_items(const int4 *__restrict__ tri4, const int2 *__restrict__ pairs,
                            const uint32_t *__restrict__ active, const unsigned long long *__restrict__ vrow,
                            const int2 *__restrict__ edges, int64_t n_springs, const int32_t *__restrict__ anchors,
                            int64_t n_anchors, DevScalars *ds, uint32_t *__restrict__ cnt,
                            const unsigned long long *__restrict__ off, uint32_t *__restrict__ items) {
    const unsigned long long n_pair_items = ds->n_active * 6, nr = ds->n_rows;
    const unsigned long long n = n_pair_items + 2ull * (unsigned long long)n_springs + (unsigned long long)n_anchors;
    for (unsigned long long code = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; code < n;
         code += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long row;
        item_row((uint32_t)code, n_pair_items, n_springs, tri4, pairs, active, vrow, edges, anchors, row);
        // (these kernels guard every write in all builds; the checked build also records it)
        if (TTIE_BAD(ds, row < nr, 61, row) || row >= nr) continue;
        const uint32_t slot = atomicAdd(&cnt[row], 1u);
        if (kFill) {
            if (TTIE_BAD(ds, off[row] + slot < off[row + 1], 62, row) || off[row] + slot >= off[row + 1]) continue;
            items[off[row] + slot] = (uint32_t)code;
        }
    }
}

// One group per row: items in code order (each item's rank among the row's codes, which are
// distinct), each item's entry columns (6 slots, -1 where an item has fewer), the first entry
// of each column (no earlier entry in item order has that column) and the distinct columns in
// ascending order (a first entry's place is the number of first entries with a smaller
// column).  All of a row's scratch lies in its items' range (x6 for entries).  The work per row
// grows with the square of its entries, so a row with more than kBigItems items goes to a
// block (kBig: kBigThreads threads) and the others to a warp.
constexpr int kRowWarps = 4;
constexpr int kBigThreads = 512;
constexpr unsigned long long kBigItems = 48;
template <bool kBig> __device__ __forceinline__ void group_sync() {
    if (kBig) __syncthreads();
    else __syncwarp();
}

template <bool kBig>
__global__ void __launch_bounds__(kBig ? kBigThreads : 32 * kRowWarps)
    k_row_columns(const uint32_t *__restrict__ items, const unsigned long long *__restrict__ off,
                  const int4 *__restrict__ tri4, const int2 *__restrict__ pairs, const uint32_t *__restrict__ active,
                  const unsigned long long *__restrict__ vrow, const int2 *__restrict__ edges, int64_t n_springs,
                  const int32_t *__restrict__ anchors, DevScalars *ds, uint32_t *__restrict__ items2,
                  int32_t *__restrict__ ecol, uint8_t *__restrict__ efirst, int32_t *__restrict__ dlist,
                  uint32_t *__restrict__ dcnt) {
    constexpr int G = kBig ? kBigThreads : 32;
    __shared__ unsigned int s_nd;
    const int tid = kBig ? (int)threadIdx.x : (int)(threadIdx.x & 31);
    const unsigned long long nr = ds->n_rows, n_pair_items = ds->n_active * 6;
    const unsigned long long row0 = kBig ? blockIdx.x : blockIdx.x * (unsigned long long)kRowWarps + (threadIdx.x >> 5);
    const unsigned long long stride = kBig ? gridDim.x : (unsigned long long)gridDim.x * kRowWarps;
    for (unsigned long long row = row0; row < nr; row += stride) {
        const unsigned long long base = off[row], n = off[row + 1] - base;
        if ((n > kBigItems) != kBig) continue;   // the same for the whole group
        if (kBig && tid == 0) s_nd = 0;
        for (unsigned long long i = tid; i < n; i += G) {
            const uint32_t code = items[base + i];
            unsigned long long rank = 0;
            for (unsigned long long j = 0; j < n; ++j) rank += items[base + j] < code;
            if (rank < n) items2[base + rank] = code;
        }
        group_sync<kBig>();
        for (unsigned long long i = tid; i < n; i += G) {
            const uint32_t code = items2[base + i];
            int32_t cols[6] = {-1, -1, -1, -1, -1, -1};
            if (code < n_pair_items) {
                const uint32_t k = code / 6;
                const int2 pr = pairs[active[k]];
                const int4 a = tri4[pr.x], b = tri4[pr.y];
#pragma unroll
                for (int c = 0; c < 6; ++c) cols[c] = (int32_t)vrow[vid(a, b, c)];
            } else if ((unsigned long long)code - n_pair_items < 2ull * (unsigned long long)n_springs) {
                const int2 e = edges[(code - n_pair_items) / 2];
                cols[0] = (int32_t)vrow[e.x];
                cols[1] = (int32_t)vrow[e.y];
            } else {
                cols[0] = (int32_t)vrow[anchors[code - n_pair_items - 2ull * (unsigned long long)n_springs]];
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) ecol[(base + i) * 6 + c] = cols[c];
        }
        group_sync<kBig>();
        const unsigned long long ne = 6 * n;
        int32_t *ec = ecol + base * 6;
        for (unsigned long long q = tid; q < ne; q += G) {
            const int32_t col = ec[q];
            bool first = col >= 0;
            for (unsigned long long p = 0; p < q && first; ++p) first = ec[p] != col;
            efirst[base * 6 + q] = first ? 1 : 0;
        }
        group_sync<kBig>();
        uint32_t nd = 0;
        for (unsigned long long q = tid; q < ne; q += G) {
            if (!efirst[base * 6 + q]) continue;
            const int32_t col = ec[q];
            unsigned long long place = 0;
            for (unsigned long long p = 0; p < ne; ++p) place += efirst[base * 6 + p] && ec[p] < col;
            if (place < ne) dlist[base * 6 + place] = col;
            ++nd;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) nd += __shfl_xor_sync(0xffffffffu, nd, o);
        if (kBig) {
            if ((threadIdx.x & 31) == 0) atomicAdd(&s_nd, nd);
            __syncthreads();
            if (tid == 0) dcnt[row] = s_nd;
        } else if (tid == 0) {
            dcnt[row] = nd;
        }
        group_sync<kBig>();
    }
}

// One group per row (as above), a thread per distinct column: the block (row, col) as the sum
// of its entries in item order, its column index and, on the diagonal, the gradient rows;
// row_ptr from the scanned distinct counts (dptr[V] = nnzb).
template <typename T, bool kBig>
__global__ void __launch_bounds__(kBig ? kBigThreads : 32 * kRowWarps)
    k_row_values(const uint32_t *__restrict__ items2, const unsigned long long *__restrict__ off,
                 const int32_t *__restrict__ ecol, const int32_t *__restrict__ dlist, const uint32_t *__restrict__ dcnt,
                 const unsigned long long *__restrict__ dptr, int64_t V, unsigned long long cap, const T *__restrict__ z,
                 const T *__restrict__ sfac, int64_t n_springs, const T *__restrict__ afac, T ka, DevScalars *ds,
                 int32_t *__restrict__ row_ptr, int32_t *__restrict__ col_idx, T *__restrict__ bval,
                 T *__restrict__ grad_rows, const int32_t *__restrict__ row_vertex, T *__restrict__ grad_full) {
    constexpr int G = kBig ? kBigThreads : 32;
    const int tid = kBig ? (int)threadIdx.x : (int)(threadIdx.x & 31);
    const unsigned long long nr = ds->n_rows, n_pair_items = ds->n_active * 6;
    const unsigned long long row0 = kBig ? blockIdx.x : blockIdx.x * (unsigned long long)kRowWarps + (threadIdx.x >> 5);
    const unsigned long long stride = kBig ? gridDim.x : (unsigned long long)gridDim.x * kRowWarps;
    if (!kBig && blockIdx.x == 0 && threadIdx.x == 0) {
        ds->nnzb = dptr[V];
        if (nr <= (unsigned long long)V) row_ptr[nr] = (int32_t)dptr[V];
    }
    for (unsigned long long row = row0; row < nr; row += stride) {
        const unsigned long long base = off[row], n = off[row + 1] - base, rp = dptr[row];
        if ((n > kBigItems) != kBig) continue;
        const uint32_t nd = dcnt[row];
        if (tid == 0) row_ptr[row] = (int32_t)rp;
        for (uint32_t d = tid; d < nd && rp + d < cap; d += G) {
            const int32_t col = dlist[base * 6 + d];
            const bool diag = (unsigned long long)col == row;
            T m[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) m[i] = T(0);
            T g0 = 0, g1 = 0, g2 = 0;
            for (unsigned long long i = 0; i < n; ++i) {
                const uint32_t code = items2[base + i];
                const int32_t *ci = ecol + (base + i) * 6;
                for (int c = 0; c < 6; ++c) {
                    if (ci[c] != col) continue;
                    if (code < n_pair_items) {
                        const uint32_t k = code / 6;
                        add_pair_entry<T>(z, k, code - k * 6, (uint32_t)c, diag, m, g0, g1, g2);
                    } else if ((unsigned long long)code - n_pair_items < 2ull * (unsigned long long)n_springs) {
                        const unsigned long long w = code - n_pair_items, sp = w / 2;
                        const unsigned q = (w - 2 * sp) ? (c == 0 ? 2u : 3u) : (c == 0 ? 0u : 1u);
                        add_spring_entry<T>(sfac, sp, q, diag, m, g0, g1, g2);
                    } else {
                        add_anchor_entry<T>(afac, code - n_pair_items - 2ull * (unsigned long long)n_springs, ka, diag,
                                            m, g0, g1, g2);
                    }
                }
            }
            col_idx[rp + d] = col;
#pragma unroll
            for (int i = 0; i < 9; ++i) bval[(rp + d) * 9 + i] = m[i];
            if (diag) {
                grad_rows[row * 3] = g0; grad_rows[row * 3 + 1] = g1; grad_rows[row * 3 + 2] = g2;
                if (grad_full) {
                    const int64_t v = row_vertex[row];
                    grad_full[v * 3] = g0; grad_full[v * 3 + 1] = g1; grad_full[v * 3 + 2] = g2;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- PCG

// Words that one block publishes to the others carry a tag in their two lowest significand
// bits (the value is the tagged word itself, on both sides), so a reader that loads a word
// also learns whether it is the current one: no separate flag or epoch is read first.
__device__ __forceinline__ float tag_word(float v, unsigned t) { return __uint_as_float((__float_as_uint(v) & ~3u) | t); }
__device__ __forceinline__ double tag_word(double v, unsigned t) {
    return __longlong_as_double((long long)(((unsigned long long)__double_as_longlong(v) & ~3ull) | t));
}
__device__ __forceinline__ unsigned word_tag(float v) { return __float_as_uint(v) & 3u; }
__device__ __forceinline__ unsigned word_tag(double v) { return (unsigned)__double_as_longlong(v) & 3u; }

// Rows of the block-resident PCG's G blocks: part[b] .. part[b + 1], balanced by the work
// of a block, nnz + row_weight * rows (the first row r whose prefix row_ptr[r] +
// row_weight * r reaches b / G of the total), then clamped to at most r_cap rows per block
// (a forward pass bounds each block by its predecessor, a backward pass the tail; r_cap * G
// >= n_rows makes both feasible).  One block of the setup grid.
__device__ void resident_partition(const int32_t *__restrict__ row_ptr, long long nr, int G, int r_cap, int row_weight,
                                   int *__restrict__ part) {
    const long long total = (long long)row_ptr[nr] + (long long)row_weight * nr;
    for (int b = threadIdx.x; b <= G; b += blockDim.x) {
        long long lo = 0, hi = nr;
        if (b == G) lo = nr;
        else if (b > 0) {
            const long long target = total * b / G;
            while (lo < hi) {
                const long long mid = (lo + hi) / 2;
                if ((long long)row_ptr[mid] + (long long)row_weight * mid >= target) hi = mid;
                else lo = mid + 1;
            }
        }
        part[b] = (int)lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int b = 1; b < G; ++b) part[b] = min(max(part[b], part[b - 1]), part[b - 1] + r_cap);
        for (int b = G - 1; b >= 1; --b) part[b] = max(part[b], part[b + 1] - r_cap);
    }
}

// p = z = M^-1 r0, r = r0, x = 0; r.z and r.r summed.  For the block-resident kernel also the
// tagged mirror z4 of z (tag 0: the first iteration's vector), its reduction words cleared
// (tag 0 never marks a published reduction word) and its row partition (block 0).
template <typename T>
__global__ void k_pcg_setup(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                            const T *__restrict__ bval, double mu_rel, T *__restrict__ dinv, const T *__restrict__ rhs,
                            T *__restrict__ x, T *__restrict__ r, T *__restrict__ z, T *__restrict__ p, double *partials,
                            vec4_t<T> *__restrict__ z4, unsigned long long *__restrict__ sync_words, int n_sync_words,
                            int *__restrict__ part, int part_blocks, int r_cap, int row_weight, DevScalars *ds) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_sync_words; i += gridDim.x * blockDim.x) sync_words[i] = 0ull;
    if (part && blockIdx.x == 0) resident_partition(row_ptr, (long long)ds->n_rows, part_blocks, r_cap, row_weight, part);
    const unsigned long long nr = ds->n_rows;
    const T mu = (T)(nr ? mu_rel * ds->trace / (3.0 * (double)nr) : 0.0);
    double rz = 0.0, rr = 0.0;
    for (unsigned long long row = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; row < nr;
         row += (unsigned long long)gridDim.x * blockDim.x) {
        const T zero9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        const T *diag = zero9;
        if (TTIE_BAD(ds, row_ptr[row] <= row_ptr[row + 1] && (unsigned long long)row_ptr[row + 1] <= ds->nnzb, 31,
                     row))
            continue;
        for (int b = row_ptr[row]; b < row_ptr[row + 1]; ++b)
            if ((unsigned long long)col_idx[b] == row) { diag = bval + (size_t)b * 9; break; }
        T di[9];
        inv3(diag, mu, di);
#pragma unroll
        for (int i = 0; i < 9; ++i) dinv[row * 9 + i] = di[i];
        const T r0 = rhs[row * 3], r1 = rhs[row * 3 + 1], r2 = rhs[row * 3 + 2];
        const T z0 = di[0] * r0 + di[1] * r1 + di[2] * r2, z1 = di[3] * r0 + di[4] * r1 + di[5] * r2,
                z2 = di[6] * r0 + di[7] * r1 + di[8] * r2;
        x[row * 3] = 0; x[row * 3 + 1] = 0; x[row * 3 + 2] = 0;
        r[row * 3] = r0; r[row * 3 + 1] = r1; r[row * 3 + 2] = r2;
        z[row * 3] = z0; z[row * 3 + 1] = z1; z[row * 3 + 2] = z2;
        p[row * 3] = z0; p[row * 3 + 1] = z1; p[row * 3 + 2] = z2;
        if (z4) {
            vec4_t<T> t;
            t.x = tag_word(z0, 0u); t.y = tag_word(z1, 0u); t.z = tag_word(z2, 0u); t.w = T(0);
            z4[row] = t;
        }
        rz += (double)r0 * z0 + (double)r1 * z1 + (double)r2 * z2;
        rr += (double)r0 * r0 + (double)r1 * r1 + (double)r2 * r2;
    }
    double v[2] = {rz, rr};
    grid_sums<2>(v, partials, &ds->done_counter[2], [&](const double *t) {
        ds->mu = (double)mu;
        ds->red[0] = t[0];   // r.z
        ds->red[1] = t[1];   // r0.r0
        ds->red[4] = t[1];   // r.r
        ds->pcg_iters = 0;
        ds->pcg_done = (t[1] == 0.0) ? 1 : 0;
    });
}

// ---------------------------------------------------------------- persistent PCG
// All PCG iterations in one cooperative launch (every block resident), for systems whose rows
// do not fit the block-resident kernels.  Blocks meet at a grid reduction twice per iteration
// (p.q, then r.z and r.r); each wait is bounded and, when it runs out, sets ERR_BARRIER and
// the kernel returns.  Reductions: block partials, then the last block to arrive sums them in
// block order and publishes the totals, so all blocks take the same decisions and the result
// does not depend on timing.
// Every wait of the PCG kernels gives up after kWaitNs of elapsed time (the GPU's global
// timer, read every 64 polls), so a block that never arrives ends the others' waits, and the
// launch, with ERR_BARRIER in about a second.
constexpr unsigned long long kWaitNs = 1000000000ull;
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
struct WaitClock {
    unsigned long long t0 = 0;
    unsigned polls = 0;
    __device__ __forceinline__ bool out() {   // true once the wait has run for more than kWaitNs
        if ((polls++ & 63u) != 0u) return false;
        const unsigned long long t = global_ns();
        if (t0 == 0) t0 = t;
        return t - t0 > kWaitNs;
    }
};

// Sum of per-block values v[0..N) over the grid, identical in every block, fused with a
// grid barrier.  Each block writes its partial sums and arrives on one counter; the last
// block to arrive adds all partials in block order (a fixed order, so the result does not
// depend on timing), publishes the totals and bumps the generation the others poll; they
// then read the totals.  Waits are bounded (kWaitNs); on timeout ERR_BARRIER is set
// and false returned.  part holds N x gridDim.x partials followed by N totals.
template <int N>
__device__ __forceinline__ bool grid_allreduce(double (&v)[N], double *part, DevScalars *ds) {
    __shared__ double tot[N];
    __shared__ int s_last, s_fail;
    __shared__ unsigned s_gen;
    const unsigned G = gridDim.x;
    double b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] = block_sum(v[i]);
    if (threadIdx.x == 0) {
        s_fail = 0;
        s_gen = *(volatile unsigned int *)&ds->bar_gen;   // before arriving: the release bumps it
#pragma unroll
        for (int i = 0; i < N; ++i) part[(size_t)i * G + blockIdx.x] = b[i];
        __threadfence();
        s_last = atomicAdd(&ds->bar_count, 1u) == G - 1;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned g = s_gen;
        if (s_last) {
            __threadfence();
#pragma unroll
            for (int i = 0; i < N; ++i) {
                double s = 0.0;
                for (unsigned j = threadIdx.x; j < G; j += 32) s += __ldcg(&part[(size_t)i * G + j]);
#pragma unroll
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                tot[i] = s;
            }
            if (threadIdx.x == 0) {
#pragma unroll
                for (int i = 0; i < N; ++i) part[(size_t)N * G + i] = tot[i];
                ds->bar_count = 0u;
                __threadfence();
                atomicAdd(&ds->bar_gen, 1u);
            }
        } else if (threadIdx.x == 0) {
            WaitClock wc;
            while (*(volatile unsigned int *)&ds->bar_gen == g) {
                if (wc.out()) {
                    atomicOr(&ds->err, ERR_BARRIER);
                    s_fail = 1;
                    break;
                }
                __nanosleep(20);
            }
            __threadfence();
#pragma unroll
            for (int i = 0; i < N; ++i) tot[i] = __ldcg(&part[(size_t)N * G + i]);
        }
    }
    __syncthreads();
    const bool ok = s_fail == 0;
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = tot[i];
    __syncthreads();
    return ok;
}

// One block's partial sums for the resident PCG's reductions: the bits of its accumulators,
// each word tagged (its lowest bits) with the reduction that wrote it.
struct __align__(32) RedSlot {
    unsigned long long v[4];   // v[3] unused
};

template <typename T> struct PcgArgs {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const T *bval;
    const T *dinv;
    T *x, *r, *z, *p, *q;
    vec4_t<T> *z4;           // z mirrored as one tagged 16/32-byte vector per row (resident kernel)
    vec4_t<T> *z4b;          // resident kernel with the Chebyshev preconditioner: odd publications
    int cheb_degree;         // degree of the Chebyshev preconditioner (that kernel only)
    double *partA, *partB;
    RedSlot *slots;          // resident kernel: 2 x kMaxGridPcg tagged reduction slots, then 2 total slots
    const int *part;         // resident kernel: rows of block b are part[b] .. part[b + 1]
    int withhold;            // test switch: block 0 never publishes its partial sums
    double rtol2;
    int max_it;
    DevScalars *ds;
};

// 8 consecutive lanes share a row in the product w = (H + mu I) z: each takes every 8th
// block of the row and the partial products are summed by shuffles.  Lane 0 of the group
// owns the row in the vector updates, so x, r, z, p, q of a row are written by one thread
// only; z of other rows is read through L2 (__ldcg) after the barrier that follows its
// update.  With w = A z, the search direction's product follows from q = A p = w + beta q,
// so an iteration needs two grid reductions (p.q, then r.z and r.r) and no third barrier.
constexpr int kLanesPerRow = 8;
constexpr int kPcgThreads = 1024;

template <typename T>
__device__ __forceinline__ void spmv_row(const PcgArgs<T> &a, unsigned long long row, int sub, unsigned gmask, T mu,
                                         T &y0, T &y1, T &y2) {
    const int b0 = a.row_ptr[row], b1 = a.row_ptr[row + 1];
    y0 = 0; y1 = 0; y2 = 0;
    for (int b = b0 + sub; b < b1; b += kLanesPerRow) {
        if (TTIE_BAD(a.ds, b >= 0 && (unsigned long long)b < a.ds->nnzb, 51, b)) break;
        const T *m = a.bval + (size_t)b * 9;
        const int c = a.col_idx[b];
        if (TTIE_BAD(a.ds, c >= 0 && (unsigned long long)c < a.ds->n_rows, 52, c)) break;
        const T c0 = __ldcg(&a.z[c * 3]), c1 = __ldcg(&a.z[c * 3 + 1]), c2 = __ldcg(&a.z[c * 3 + 2]);
        y0 += m[0] * c0 + m[1] * c1 + m[2] * c2;
        y1 += m[3] * c0 + m[4] * c1 + m[5] * c2;
        y2 += m[6] * c0 + m[7] * c1 + m[8] * c2;
    }
#pragma unroll
    for (int o = kLanesPerRow / 2; o; o >>= 1) {
        y0 += __shfl_xor_sync(gmask, y0, o, kLanesPerRow);
        y1 += __shfl_xor_sync(gmask, y1, o, kLanesPerRow);
        y2 += __shfl_xor_sync(gmask, y2, o, kLanesPerRow);
    }
    y0 += mu * a.z[row * 3]; y1 += mu * a.z[row * 3 + 1]; y2 += mu * a.z[row * 3 + 2];
}

// p = z + beta p, q = A z + beta q (p = z, q = A z when first: p and q hold nothing yet),
// returns the row's p.q
template <typename T>
__device__ __forceinline__ double direction_phase(const PcgArgs<T> &a, unsigned long long nr, unsigned long long group,
                                                  unsigned long long n_groups, int sub, unsigned gmask, T mu, T beta,
                                                  bool first) {
    double pq = 0.0;
    for (unsigned long long row = group; row < nr; row += n_groups) {
        T w0, w1, w2;
        spmv_row(a, row, sub, gmask, mu, w0, w1, w2);
        if (sub == 0) {
            const T w[3] = {w0, w1, w2};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T pi = first ? a.z[row * 3 + i] : a.z[row * 3 + i] + beta * a.p[row * 3 + i];
                const T qi = first ? w[i] : w[i] + beta * a.q[row * 3 + i];
                a.p[row * 3 + i] = pi;
                a.q[row * 3 + i] = qi;
                pq += (double)pi * qi;
            }
        }
    }
    return pq;
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads) k_pcg_persistent(PcgArgs<T> a) {
    DevScalars *ds = a.ds;
    if (ds->pcg_done) return;
    const unsigned long long nr = ds->n_rows;
    const T mu = (T)ds->mu;
    const double rr0 = ds->red[1];
    double rz = ds->red[0], rr = rr0;
    const int lane = threadIdx.x & 31, sub = lane & (kLanesPerRow - 1);
    const unsigned gmask = 0xffu << (lane & ~(kLanesPerRow - 1));
    const unsigned long long group = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) / kLanesPerRow;
    const unsigned long long n_groups = (unsigned long long)gridDim.x * blockDim.x / kLanesPerRow;
    // p = z, q = A z (z comes from the setup kernel, an earlier launch)
    double v1[1] = {direction_phase(a, nr, group, n_groups, sub, gmask, mu, T(0), true)};
    if (!grid_allreduce<1>(v1, a.partA, ds)) return;
    int it = 0;
    for (; it < a.max_it; ++it) {
        const double pq = v1[0];
        const bool ok = pq > 0.0 && isfinite(pq);
        // breakdown at the first iteration keeps x = p = M^-1 r0 (preconditioned gradient)
        const T alpha = (T)(ok ? rz / pq : (it == 0 ? 1.0 : 0.0));
        double v2[2] = {0.0, 0.0};
        if (sub == 0) {
            for (unsigned long long row = group; row < nr; row += n_groups) {
                T rv[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    a.x[row * 3 + i] += alpha * a.p[row * 3 + i];
                    rv[i] = a.r[row * 3 + i] - alpha * a.q[row * 3 + i];
                    a.r[row * 3 + i] = rv[i];
                }
                const T *di = a.dinv + row * 9;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T zi = di[3 * i] * rv[0] + di[3 * i + 1] * rv[1] + di[3 * i + 2] * rv[2];
                    a.z[row * 3 + i] = zi;
                    v2[0] += (double)rv[i] * zi;
                    v2[1] += (double)rv[i] * rv[i];
                }
            }
        }
        if (!grid_allreduce<2>(v2, a.partB, ds)) return;
        if (!ok) { ++it; break; }
        const double beta = rz != 0.0 ? v2[0] / rz : 0.0;
        rz = v2[0];
        rr = v2[1];
        if (rr <= a.rtol2 * rr0 || !isfinite(rr)) { ++it; break; }
        v1[0] = direction_phase(a, nr, group, n_groups, sub, gmask, mu, (T)beta, false);
        if (!grid_allreduce<1>(v1, a.partA, ds)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ds->pcg_iters = it;
        ds->red[0] = rz;
        ds->red[4] = rr;
        ds->pcg_done = 1;
    }
}

// ---------------------------------------------------------------- PCG, block-resident rows
// Each block owns the contiguous rows [row0, row0 + nrow) for the whole solve.  Their x, r,
// u = M^-1 r, p, s = A p, w = A u, the inverse diagonal blocks, the row offsets and, when
// they fit, the matrix rows and the gathered u of their columns live in shared memory.
//
// Iteration (Chronopoulos and Gear's form of preconditioned CG: one reduction per
// iteration).  With gamma = r.u, delta = w.u:
//   beta = gamma / gamma_prev,  alpha = gamma / (delta - beta gamma / alpha_prev)
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,  u = M^-1 r,  w = A u.
// The product needs u of other blocks' rows.  Each block publishes its u as one 16/32-byte
// vector per row whose words carry the iteration's tag (k mod 4); a reader loads the words
// of its columns and loads again those whose tag is not yet k.  The three dot products are
// summed through per-block slots whose words carry the reduction's tag (8 + k mod 8): block
// 0 adds all slots in a fixed order and publishes the totals, tagged the same way, which
// every block reads, so all blocks take the same decisions.
//
// Why the tags cannot be mistaken, with no fences: all published words are written and read
// with relaxed gpu-scope accesses, and a thread reads the same words in every iteration (its
// columns, its slots).  Coherence per location: having waited for the tag of iteration
// k - 1 in a word, the same thread's next load of it returns that write or a later one.  No
// block writes u of iteration k + 1 before it has read the totals of reduction k, which
// follow the reader's sums, which follow its product (a causality cycle otherwise).  So a
// reader of u sees iteration k - 1 or k.  Slots and totals alternate between two buffers by
// reduction parity: no block publishes sums of reduction k + 2 before it has read the totals
// of k + 1, which block 0 publishes after it has read every slot of k + 1 (so after those of
// k), so block 0 sees reduction k - 2 or k in a slot and every block sees k - 2 or k in the
// totals.  The setup kernel (an earlier launch) writes u of iteration 0 with tag 0 and
// clears slots and totals (tag 0 is never a reduction's).  Every wait is bounded; on
// timeout ERR_BARRIER is set and the kernel returns.
constexpr int kResidentSmem = 220 * 1024;   // dynamic shared memory per block
constexpr int kMaxGridPcg = 160;            // at least the SM count; slots per lane of the root's poll: 5
constexpr int kRowWeight = 8;   // work of a row in the partition, in matrix blocks (lane-group pass, shuffles, update)

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// a block's row range that does not fit its layout: recorded as a failed check, rows dropped
__device__ __forceinline__ void partition_fail(DevScalars *ds, int code) {
    if (threadIdx.x == 0) {
        atomicCAS(&ds->check_code, 0, code);
        atomicOr(&ds->err, ERR_CHECK);
    }
}

// relaxed (coherent, never cached in L1) load of one published row vector
template <typename T> __device__ __forceinline__ vec4_t<T> ld_row(const vec4_t<T> *p);
template <> __device__ __forceinline__ float4 ld_row<float>(const float4 *p) {
    float4 r;
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}
template <> __device__ __forceinline__ dvec4 ld_row<double>(const dvec4 *p) {
    dvec4 r;
    asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(r.z) : "l"(reinterpret_cast<const double *>(p) + 2));
    r.w = 0.0;
    return r;
}
template <typename T> __device__ __forceinline__ void st_row(vec4_t<T> *p, const vec4_t<T> &v);
template <> __device__ __forceinline__ void st_row<float>(float4 *p, const float4 &v) {
    asm volatile("st.relaxed.gpu.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
template <> __device__ __forceinline__ void st_row<double>(dvec4 *p, const dvec4 &v) {
    asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v.x), "d"(v.y) : "memory");
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(reinterpret_cast<double *>(p) + 2), "d"(v.z) : "memory");
}
template <typename T> __device__ __forceinline__ bool row_tagged(const vec4_t<T> &g, unsigned t) {
    return (word_tag(g.x) == t) & (word_tag(g.y) == t) & (word_tag(g.z) == t);
}
// reload g from p until its words carry tag t; bounded (sets *bad)
template <typename T>
__device__ __forceinline__ void settle_row(vec4_t<T> &g, const vec4_t<T> *p, unsigned t, int *bad) {
    WaitClock wc;
    while (!row_tagged<T>(g, t)) {
        if (wc.out() || *(volatile int *)bad) { *bad = 1; return; }
        g = ld_row<T>(p);
    }
}

// a reduction word with tag t in the four lowest significand bits of its smaller part
template <typename T> __device__ __forceinline__ unsigned long long tag_bits(unsigned long long b, unsigned t) {
    constexpr int s = Acc<T>::kTagShift;
    return (b & ~(15ull << s)) | ((unsigned long long)t << s);
}
template <typename T> __device__ __forceinline__ unsigned bits_tag(unsigned long long b) {
    return (unsigned)(b >> Acc<T>::kTagShift) & 15u;
}

// one reduction slot, all four words in one 32-byte load (each word read atomically)
__device__ __forceinline__ void ld_slot(const RedSlot *p, unsigned long long (&w)[4]) {
    asm volatile("ld.relaxed.gpu.global.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3])
                 : "l"(p));
}

// Grid sums of N <= 3 accumulators, identical in every block, through tagged words (tag
// t = 8 + k mod 8 for reduction k, buffers by k mod 2).  After the warps' partial sums meet
// in shared memory, warp i < N adds word i over the warps and publishes it in the block's
// slot.  Block 0 alone loads all slots (one 32-byte load each) until every word carries t,
// adds them in slot order and publishes the totals in one slot of their own; every other
// block polls that one slot.  So each poll round costs the memory system one load per block
// instead of one per block and slot.  Thread 0 then runs fin(totals).  A block that gave up
// (*bad), or withholds (the failure-path test switch), publishes nothing.  Returns false
// (ERR_BARRIER set) when a wait ran out.
template <int N, typename T, typename Fin>
__device__ __forceinline__ bool slot_allreduce(Acc<T> (&a)[N], RedSlot *slots, unsigned k, const int *bad,
                                               bool withhold, DevScalars *ds, Fin fin) {
    static_assert(N <= 3, "three words per slot");
    __shared__ int s_fail;
    __shared__ unsigned long long s_part[N][32];
    __shared__ unsigned long long s_w[kMaxGridPcg][N];
    const unsigned G = gridDim.x;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int o = 16; o; o >>= 1) a[i].add(a[i].shfl_xor(0xffffffffu, o, 32));
        if (lane == 0) s_part[i][wi] = a[i].bits();
    }
    __syncthreads();   // also makes *bad visible
    RedSlot *buf = slots + (size_t)(k & 1u) * kMaxGridPcg;
    RedSlot *tot = slots + 2 * kMaxGridPcg + (k & 1u);
    const unsigned t = 8u | (k & 7u);
    const bool gave_up = *(const volatile int *)bad != 0;
    if (wi < N) {
        Acc<T> mine = lane < (int)(blockDim.x >> 5) ? Acc<T>::from_bits(s_part[wi][lane]) : Acc<T>();
#pragma unroll
        for (int o = 16; o; o >>= 1) mine.add(mine.shfl_xor(0xffffffffu, o, 32));
        if (lane == 0 && !gave_up && !withhold) st_relaxed_u64(&buf[blockIdx.x].v[wi], tag_bits<T>(mine.bits(), t));
    }
    if (wi == 0) {
        bool fail = gave_up;
        unsigned long long tw[4];
        if (blockIdx.x == 0) {
            // the root: every slot, all loads of a lane in flight together
            unsigned ready = 0, want = 0;
#pragma unroll
            for (int q = 0; q < kMaxGridPcg / 32; ++q)
                if (lane + 32u * q < G) want |= 1u << q;
            WaitClock wc;
            while (!fail) {
#pragma unroll
                for (int q = 0; q < kMaxGridPcg / 32; ++q)
                    if ((want & ~ready) >> q & 1u) {
                        unsigned long long w[4];
                        ld_slot(&buf[lane + 32 * q], w);
                        bool ok = true;
#pragma unroll
                        for (int i = 0; i < N; ++i) ok &= bits_tag<T>(w[i]) == t;
                        if (ok) {
#pragma unroll
                            for (int i = 0; i < N; ++i) s_w[lane + 32 * q][i] = w[i];
                            ready |= 1u << q;
                        }
                    }
                if (__all_sync(0xffffffffu, ready == want)) break;
                if (wc.out()) { fail = true; break; }
                __nanosleep(20);
            }
            fail = __any_sync(0xffffffffu, fail);
            __syncwarp();
            Acc<T> sum[N];
#pragma unroll
            for (int q = 0; q < kMaxGridPcg / 32; ++q)
                if (want >> q & 1u)
#pragma unroll
                    for (int i = 0; i < N; ++i) sum[i].add(Acc<T>::from_bits(s_w[lane + 32 * q][i]));
#pragma unroll
            for (int i = 0; i < N; ++i) {
#pragma unroll
                for (int o = 16; o; o >>= 1) sum[i].add(sum[i].shfl_xor(0xffffffffu, o, 32));
                tw[i] = tag_bits<T>(sum[i].bits(), t);
            }
            if (lane == 0 && !fail)
#pragma unroll
                for (int i = 0; i < N; ++i) st_relaxed_u64(&tot->v[i], tw[i]);
        } else if (lane == 0) {
            WaitClock wc;
            while (!fail) {
                ld_slot(tot, tw);
                bool ok = true;
#pragma unroll
                for (int i = 0; i < N; ++i) ok &= bits_tag<T>(tw[i]) == t;
                if (ok) break;
                if (wc.out()) { fail = true; break; }
                __nanosleep(20);
            }
        }
        if (lane == 0) {
            s_fail = fail ? 1 : 0;
            if (fail) atomicOr(&ds->err, ERR_BARRIER);
            else {
                Acc<T> tt[N];
#pragma unroll
                for (int i = 0; i < N; ++i) tt[i] = Acc<T>::from_bits(tw[i]);
                fin(tt);
            }
        }
    }
    __syncthreads();
    return s_fail == 0;
}

template <typename T>
__device__ __forceinline__ void block_times(const T *m, T v0, T v1, T v2, T &y0, T &y1, T &y2) {
    y0 += m[0] * v0 + m[1] * v1 + m[2] * v2;
    y1 += m[3] * v0 + m[4] * v1 + m[5] * v2;
    y2 += m[6] * v0 + m[7] * v1 + m[8] * v2;
}

template <typename T> struct ResidentView {
    T *x, *r, *u, *p, *s, *w, *di;   // 3 (9 for di) values per local row
    int *rp;                          // local row offsets (nrow + 1)
    T *val;                           // matrix rows (9 per block) when cached
    int *col;                         // their columns when cached
    T *gu;                            // u at each block's column (3 per block) when gathered
    T *d, *rr;                        // Chebyshev preconditioner: direction and D^-1 residual (3 each)
    bool cached, gathered;
    int nrow, nnz, b_begin;
};

// w = (A + mu I) u on the block's rows, u of every row read from the published vectors src
// with tag t (loc: the block's own rows of u, for the shift); returns the rows' w.u.  A load
// that never sees tag t sets *bad.
template <typename T>
__device__ __forceinline__ Acc<T> resident_product(const PcgArgs<T> &a, const ResidentView<T> &v,
                                                   const vec4_t<T> *src, const T *loc, T mu, unsigned t, int *bad) {
    if (v.gathered) {
        // gather every block's column vector first: all loads of a thread in flight together
        // words not yet tagged t are loaded again, all of a thread's together
        constexpr int U = 4;
        for (int j0 = threadIdx.x; j0 < v.nnz; j0 += U * kPcgThreads) {
            vec4_t<T> g[U];
            unsigned pend = 0;
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int j = j0 + k * kPcgThreads;
                if (j < v.nnz) {
                    g[k] = ld_row<T>(&src[v.col[j]]);
                    pend |= 1u << k;
                }
            }
            WaitClock wc;
            while (true) {
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if ((pend >> k & 1u) && row_tagged<T>(g[k], t)) {
                        const int j = j0 + k * kPcgThreads;
                        v.gu[3 * j] = g[k].x; v.gu[3 * j + 1] = g[k].y; v.gu[3 * j + 2] = g[k].z;
                        pend &= ~(1u << k);
                    }
                if (!pend) break;
                if (wc.out() || *(volatile int *)bad) { *bad = 1; break; }
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (pend >> k & 1u) g[k] = ld_row<T>(&src[v.col[j0 + k * kPcgThreads]]);
            }
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, sub = lane & (kLanesPerRow - 1);
    const unsigned gmask = 0xffu << (lane & ~(kLanesPerRow - 1));
    Acc<T> wu;
    for (int lr = threadIdx.x / kLanesPerRow; lr < v.nrow; lr += kPcgThreads / kLanesPerRow) {
        T y0 = 0, y1 = 0, y2 = 0;
        const int be = v.rp[lr + 1];
        if (v.gathered) {
            for (int b = v.rp[lr] + sub; b < be; b += kLanesPerRow)
                block_times(v.val + (size_t)b * 9, v.gu[3 * b], v.gu[3 * b + 1], v.gu[3 * b + 2], y0, y1, y2);
        } else {
            // up to four of the lane's blocks at a time: every load in flight before any tag
            // is checked (a check is a branch on the loaded value)
            constexpr int U = 4;
            for (int b0 = v.rp[lr] + sub; b0 < be; b0 += U * kLanesPerRow) {
                int cc[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int b = b0 + k * kLanesPerRow;
                    cc[k] = -1;
                    if (b < be) {
                        if (v.cached) {
                            cc[k] = v.col[b];
                        } else {
                            if (TTIE_BAD(a.ds, (unsigned long long)(v.b_begin + b) < a.ds->nnzb, 41, b)) continue;
                            const int c = a.col_idx[v.b_begin + b];
                            if (TTIE_BAD(a.ds, c >= 0 && (unsigned long long)c < a.ds->n_rows, 42, c)) continue;
                            cc[k] = c;
                        }
                    }
                }
                vec4_t<T> g[U];
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (cc[k] >= 0) g[k] = ld_row<T>(&src[cc[k]]);
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (cc[k] >= 0) {
                        settle_row<T>(g[k], &src[cc[k]], t, bad);
                        const int b = b0 + k * kLanesPerRow;
                        const T *m = v.cached ? v.val + (size_t)b * 9 : a.bval + (size_t)(v.b_begin + b) * 9;
                        block_times(m, g[k].x, g[k].y, g[k].z, y0, y1, y2);
                    }
            }
        }
#pragma unroll
        for (int o = kLanesPerRow / 2; o; o >>= 1) {
            y0 += __shfl_xor_sync(gmask, y0, o, kLanesPerRow);
            y1 += __shfl_xor_sync(gmask, y1, o, kLanesPerRow);
            y2 += __shfl_xor_sync(gmask, y2, o, kLanesPerRow);
        }
        if (sub == 0) {
            const T w0 = y0 + mu * loc[lr * 3], w1 = y1 + mu * loc[lr * 3 + 1], w2 = y2 + mu * loc[lr * 3 + 2];
            v.w[lr * 3] = w0; v.w[lr * 3 + 1] = w1; v.w[lr * 3 + 2] = w2;
            wu.add_prod(w0, loc[lr * 3]);
            wu.add_prod(w1, loc[lr * 3 + 1]);
            wu.add_prod(w2, loc[lr * 3 + 2]);
        }
    }
    return wu;
}

// Chebyshev preconditioner (TTIE_PCG_CHEBYSHEV): block-Jacobi iterations before the estimate
// of lambda_max(D^-1 A), the margin on that estimate, lambda_max / lambda_min of the interval
// and the largest degree.
constexpr int kChebWarm = 6;
constexpr double kChebSafety = 1.1;
constexpr double kChebRatio = 10.0;
constexpr int kChebMaxDeg = 8;

// Eigenvalues below x of the symmetric tridiagonal (diagonal dg, squared off-diagonal e2):
// the number of negative pivots of its LDL^T factorisation shifted by x (Sturm sequence).
__device__ __forceinline__ int sturm_below(const double *dg, const double *e2, int m, double x) {
    int below = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
        q = dg[i] - x - (i ? e2[i - 1] / q : 0.0);
        if (q == 0.0) q = 1e-300;
        below += q < 0.0;
    }
    return below;
}

// From the first kChebWarm CG coefficients (al[j], be[j]: alpha and beta of iteration j; be[0]
// unused), the Lanczos tridiagonal of D^-1 A: diagonal 1/al[j] + be[j]/al[j-1], off-diagonal
// sqrt(be[j+1])/al[j].  Its largest eigenvalue (a lower bound of lambda_max, by bisection on
// the Sturm count from its Gershgorin bound) times kChebSafety is the interval's top; the
// Chebyshev iteration y = p_k(D^-1 A) D^-1 v on [top / kChebRatio, top] then runs
//   rr = D^-1 v,  d = rr / theta,  y = d;  for j < k: rr -= D^-1 A d,
//   d = c1[j] d + c2[j] rr,  y += d
// with theta, delta the interval's centre and half-width, sigma = theta / delta,
// rho_0 = 1 / sigma, rho_{j+1} = 1 / (2 sigma - rho_j), c1[j] = rho_{j+1} rho_j and
// c2[j] = 2 rho_{j+1} / delta.  Same inputs in every block, same coefficients.  False (keep
// block Jacobi) when a coefficient is not positive and finite.
template <typename T>
__device__ __noinline__ bool cheb_coefficients(const double *al, const double *be, int deg, T *c1, T *c2, T *theta_inv) {
    double dg[kChebWarm], e2[kChebWarm];
    for (int j = 0; j < kChebWarm; ++j) {
        if (!(al[j] > 0.0) || !isfinite(al[j]) || (j > 0 && (!(be[j] > 0.0) || !isfinite(be[j])))) return false;
        dg[j] = 1.0 / al[j] + (j ? be[j] / al[j - 1] : 0.0);
        if (j > 0) e2[j - 1] = be[j] / (al[j - 1] * al[j - 1]);
    }
    double hi = 0.0;
    for (int i = 0; i < kChebWarm; ++i)
        hi = fmax(hi, dg[i] + (i ? sqrt(e2[i - 1]) : 0.0) + (i + 1 < kChebWarm ? sqrt(e2[i]) : 0.0));
    if (!(hi > 0.0) || !isfinite(hi)) return false;
    double lo = 0.0;
    for (int s = 0; s < 60; ++s) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_below(dg, e2, kChebWarm, mid) < kChebWarm) lo = mid;
        else hi = mid;
    }
    const double top = hi * kChebSafety, bot = top / kChebRatio;
    const double th = 0.5 * (top + bot), de = 0.5 * (top - bot), sig = th / de;
    double rho = 1.0 / sig;
    for (int j = 0; j < deg; ++j) {
        const double rn = 1.0 / (2.0 * sig - rho);
        c1[j] = (T)(rn * rho);
        c2[j] = (T)(2.0 * rn / de);
        rho = rn;
    }
    *theta_inv = (T)(1.0 / th);
    return true;
}

template <typename T, bool kCheb>
__global__ void __launch_bounds__(kPcgThreads) k_pcg_resident(PcgArgs<T> a, int smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ T s_alpha, s_beta;
    __shared__ int s_stop, s_bad;
    DevScalars *ds = a.ds;
    if (ds->pcg_done) return;
    const long long nr = (long long)ds->n_rows;
    const long long row0 = a.part[blockIdx.x];
    ResidentView<T> v;
    v.nrow = a.part[blockIdx.x + 1] - (int)row0;
    const auto vec_size = [](int rows, int per_row) {
        return ((size_t)rows * per_row * sizeof(T) + (size_t)(rows + 1) * sizeof(int) + 15) / 16 * 16;
    };
    // the Chebyshev preconditioner's d and rr, after the other vectors
    const auto cheb_size = [](int rows) { return kCheb ? ((size_t)rows * 6 * sizeof(T) + 15) / 16 * 16 : (size_t)0; };
    if (!(row0 >= 0 && v.nrow >= 0 && row0 + v.nrow <= nr &&
          vec_size(v.nrow, 15) + cheb_size(v.nrow) <= (size_t)smem_bytes)) {
        partition_fail(ds, 45);   // checked in every build: the rows index shared memory
        v.nrow = 0;
    }
    const int R = v.nrow;
    // lean: x and the inverse diagonal blocks (read or written once per row and iteration) stay
    // in global memory so that larger row ranges fit
    const bool lean = vec_size(R, 27) + cheb_size(R) > (size_t)smem_bytes;
    size_t vec_bytes;
    if (lean) {
        v.r = (T *)smem; v.u = v.r + 3 * R; v.p = v.u + 3 * R; v.s = v.p + 3 * R; v.w = v.s + 3 * R;
        v.rp = (int *)(v.w + 3 * R);
        v.x = a.x + row0 * 3;
        v.di = (T *)a.dinv + row0 * 9;
        vec_bytes = vec_size(R, 15);
    } else {
        v.x = (T *)smem; v.r = v.x + 3 * R; v.u = v.r + 3 * R; v.p = v.u + 3 * R; v.s = v.p + 3 * R; v.w = v.s + 3 * R;
        v.di = v.w + 3 * R;
        v.rp = (int *)(v.di + 9 * R);
        vec_bytes = vec_size(R, 27);
    }
    if constexpr (kCheb) {
        v.d = (T *)(smem + vec_bytes);
        v.rr = v.d + 3 * R;
        vec_bytes += cheb_size(R);
    }
    v.b_begin = v.nrow ? a.row_ptr[row0] : 0;
    v.nnz = v.nrow ? a.row_ptr[row0 + v.nrow] - v.b_begin : 0;
    const size_t mat_bytes = ((size_t)v.nnz * (9 * sizeof(T) + sizeof(int)) + 15) / 16 * 16;
    v.cached = vec_bytes + mat_bytes <= (size_t)smem_bytes;
    v.gathered = v.cached && vec_bytes + mat_bytes + (size_t)v.nnz * 3 * sizeof(T) <= (size_t)smem_bytes;
    v.val = (T *)(smem + vec_bytes);
    v.col = (int *)(v.val + (size_t)9 * v.nnz);
    v.gu = (T *)(smem + vec_bytes + mat_bytes);
    // load the block's rows (x = 0, r, u = M^-1 r as published with tag 0 by the setup kernel,
    // M^-1; p = s = 0)
    for (int i = threadIdx.x; i < 3 * v.nrow; i += blockDim.x) {
        if (!lean) v.x[i] = a.x[row0 * 3 + i];
        v.r[i] = a.r[row0 * 3 + i];
        v.u[i] = reinterpret_cast<const T *>(a.z4 + row0 + i / 3)[i % 3];
        v.p[i] = T(0);
        v.s[i] = T(0);
    }
    if (!lean)
        for (int i = threadIdx.x; i < 9 * v.nrow; i += blockDim.x) v.di[i] = a.dinv[row0 * 9 + i];
    for (int i = threadIdx.x; i <= v.nrow; i += blockDim.x) {
        v.rp[i] = a.row_ptr[row0 + i] - v.b_begin;
        if (TTIE_BAD(ds, v.rp[i] >= 0 && v.rp[i] <= v.nnz, 43, v.rp[i])) v.rp[i] = 0;
    }
    if (v.cached)
        for (int i = threadIdx.x; i < v.nnz; i += blockDim.x) {
            int c = a.col_idx[v.b_begin + i];
            if (TTIE_BAD(ds, c >= 0 && (long long)c < nr, 44, c)) c = 0;
            for (int k = 0; k < 9; ++k) v.val[(size_t)i * 9 + k] = a.bval[(size_t)(v.b_begin + i) * 9 + k];
            v.col[i] = c;
        }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const T mu = (T)ds->mu;
    // local r.u and r.r of the current residual (thread per row)
    Acc<T> gl, rl;
    for (int lr = threadIdx.x; lr < v.nrow; lr += blockDim.x)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gl.add_prod(v.r[lr * 3 + i], v.u[lr * 3 + i]);
            rl.add_prod(v.r[lr * 3 + i], v.r[lr * 3 + i]);
        }
    // the recurrence's scalars, kept and decided by thread 0 of each block (identical inputs,
    // identical decisions) and broadcast through shared memory
    Acc<T> gamma, rr;
    T rr0 = T(0), gamma_prev = T(1), alpha_prev = T(1);
    const T rtol2 = (T)a.rtol2;
    bool stop_next = false;
    int it = 0;
    // Chebyshev preconditioner: kit counts the iterations since CG (re)started, pub the
    // published vectors (the setup kernel's u is publication 0).  Publication q goes to z4
    // when q is even and to z4b when odd, tagged q mod 4: a block publishes q + 1 only after
    // it has read q of every block it shares a matrix block with, so a reader of q finds q,
    // q - 2 (other tag) or, first, z4b's zeros (tag 0, never an odd publication's).
    int kit = 0;
    unsigned pub = 0;
    bool cheb_on = false, cheb_tried = false;
    __shared__ T s_c1[kChebMaxDeg], s_c2[kChebMaxDeg], s_thi;
    __shared__ double s_al[kChebWarm], s_be[kChebWarm];
    __shared__ int s_restart;
    auto decide = [&](const Acc<T> *t) {
        gamma = t[0];
        rr = t[2];
        const T g = gamma.approx(), d = t[1].approx(), r2 = rr.approx();
        if (it == 0) rr0 = r2;
        int stop = (stop_next || it >= a.max_it || r2 <= rtol2 * rr0 || !isfinite(r2)) ? 1 : 0;
        T alpha = T(0), beta = T(0);
        if (!stop) {
            bool ok;
            if ((kCheb ? kit : it) == 0) {
                alpha = g / d;
                ok = d > T(0) && isfinite(alpha);
            } else {
                // den = delta - beta gamma / alpha_prev in the accumulator's precision
                beta = g / gamma_prev;
                const T den = t[1].minus(gamma.over(alpha_prev).times(beta)).approx();
                alpha = g / den;
                ok = den > T(0) && isfinite(alpha);
            }
            if (!ok) {
                if (it > 0) stop = 1;
                alpha = T(1);      // breakdown at the first step keeps x = M^-1 r0 (preconditioned gradient)
                beta = T(0);
                stop_next = true;
            }
        }
        if constexpr (kCheb) {
            // the block-Jacobi iterations' coefficients; after the last of them the Chebyshev
            // polynomial's, and CG restarts with it (unless they are unusable)
            s_restart = 0;
            if (!stop && !stop_next && !cheb_tried && kit < kChebWarm) {
                s_al[kit] = (double)alpha;
                s_be[kit] = (double)beta;
                if (kit == kChebWarm - 1) {
                    cheb_tried = true;
                    s_restart = cheb_coefficients<T>(s_al, s_be, a.cheb_degree, s_c1, s_c2, &s_thi) ? 1 : 0;
                }
            }
        }
        gamma_prev = g;
        alpha_prev = alpha;
        s_alpha = alpha;
        s_beta = beta;
        s_stop = stop;
    };
    // jstep (Chebyshev): 0 when the next product is w = A u of an iteration, j + 1 when it is
    // the product of the polynomial's j-th direction
    int jstep = 0;
    unsigned long long n_prod = 0;
    while (true) {
        const bool inner = kCheb && jstep > 0;
        const vec4_t<T> *src = (kCheb && (pub & 1u)) ? a.z4b : a.z4;
        const unsigned tu = kCheb ? (pub & 3u) : ((unsigned)it & 3u);
        const Acc<T> wu = resident_product(a, v, src, inner ? v.d : v.u, mu, tu, &s_bad);
        if constexpr (kCheb) ++n_prod;
        if (inner) {
            // the polynomial's next step: rr -= D^-1 (A + mu I) d, d = c1 d + c2 rr, y += d;
            // each d but the last published for the next product, then u = y
            __syncthreads();
            const int j = jstep - 1;
            const bool last = j + 1 == a.cheb_degree;
            const T c1 = s_c1[j], c2 = s_c2[j];
            const unsigned tq = (pub + 1u) & 3u;
            vec4_t<T> *dq = ((pub + 1u) & 1u) ? a.z4b : a.z4;
            for (int lr = threadIdx.x; lr < v.nrow; lr += blockDim.x) {
                const T *di = v.di + lr * 9;
                const T w0 = v.w[lr * 3], w1 = v.w[lr * 3 + 1], w2 = v.w[lr * 3 + 2];
                T o[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int k = lr * 3 + i;
                    const T rri = v.rr[k] - (di[3 * i] * w0 + di[3 * i + 1] * w1 + di[3 * i + 2] * w2);
                    v.rr[k] = rri;
                    const T dn = c1 * v.d[k] + c2 * rri;
                    if (!last) {
                        o[i] = tag_word(dn, tq);
                        v.d[k] = o[i];
                        v.u[k] += o[i];
                    } else {
                        o[i] = tag_word(v.u[k] + dn, tq);
                        v.u[k] = o[i];
                        gl.add_prod(v.r[k], o[i]);
                    }
                }
                vec4_t<T> ov;
                ov.x = o[0]; ov.y = o[1]; ov.z = o[2]; ov.w = T(0);
                st_row<T>(&dq[row0 + lr], ov);
            }
            ++pub;
            jstep = last ? 0 : jstep + 1;
            __syncthreads();
            continue;
        }
        Acc<T> red[3] = {gl, wu, rl};
        if (!slot_allreduce<3, T>(red, a.slots, (unsigned)it, &s_bad, a.withhold && blockIdx.x == 0, ds, decide)) return;
        if (s_stop) break;
        const T al = s_alpha, be = s_beta;
        // with the Chebyshev preconditioner (from the restart on) the update publishes the
        // polynomial's first direction d = D^-1 r / theta instead of u
        const bool cheb_now = kCheb && (cheb_on || s_restart);
        const T thi = kCheb ? s_thi : T(0);
        const unsigned tn = kCheb ? ((pub + 1u) & 3u) : ((unsigned)(it + 1) & 3u);
        vec4_t<T> *dst = (kCheb && ((pub + 1u) & 1u)) ? a.z4b : a.z4;
        gl = Acc<T>();
        rl = Acc<T>();
        for (int lr = threadIdx.x; lr < v.nrow; lr += blockDim.x) {
            T rv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int k = lr * 3 + i;
                const T pi = v.u[k] + be * v.p[k];
                const T si = v.w[k] + be * v.s[k];
                v.p[k] = pi;
                v.s[k] = si;
                v.x[k] += al * pi;
                rv[i] = v.r[k] - al * si;
                v.r[k] = rv[i];
            }
            const T *di = v.di + lr * 9;
            vec4_t<T> z4;
            T zv[3];
            if (!cheb_now) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    // the published (tagged) word is the value on every side
                    zv[i] = tag_word(di[3 * i] * rv[0] + di[3 * i + 1] * rv[1] + di[3 * i + 2] * rv[2], tn);
                    v.u[lr * 3 + i] = zv[i];
                    gl.add_prod(rv[i], zv[i]);
                    rl.add_prod(rv[i], rv[i]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int k = lr * 3 + i;
                    const T q = di[3 * i] * rv[0] + di[3 * i + 1] * rv[1] + di[3 * i + 2] * rv[2];
                    v.rr[k] = q;
                    zv[i] = tag_word(q * thi, tn);
                    v.d[k] = zv[i];
                    v.u[k] = zv[i];    // y = d
                    rl.add_prod(rv[i], rv[i]);
                }
            }
            z4.x = zv[0]; z4.y = zv[1]; z4.z = zv[2]; z4.w = T(0);
            st_row<T>(&dst[row0 + lr], z4);
        }
        ++it;
        __syncthreads();
        if constexpr (kCheb) {
            ++pub;
            if (cheb_now) {
                kit = cheb_on ? kit + 1 : 0;   // CG restarts with the polynomial
                cheb_on = true;
                jstep = 1;
            } else {
                ++kit;
            }
        }
    }
    if (!lean)
        for (int i = threadIdx.x; i < 3 * v.nrow; i += blockDim.x) a.x[row0 * 3 + i] = v.x[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ds->pcg_iters = it;
        ds->red[0] = gamma.value();
        ds->red[1] = (double)rr0;
        ds->red[4] = rr.value();
        ds->pcg_done = 1;
        if constexpr (kCheb) ds->pcg_products = n_prod;
    }
}

template <typename T>
__global__ void k_axpy_positions(const vec4_t<T> *__restrict__ x, const T *__restrict__ d, T alpha, int64_t V,
                                 vec4_t<T> *__restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        vec4_t<T> a = x[v];
        a.x += alpha * d[v * 3]; a.y += alpha * d[v * 3 + 1]; a.z += alpha * d[v * 3 + 2];
        out[v] = a;
    }
}

template <typename T>
__global__ void k_scatter_rows(const T *__restrict__ d_rows, const int32_t *__restrict__ row_vertex, const DevScalars *ds,
                               T *__restrict__ d_full) {
    const unsigned long long nr = ds->n_rows;
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < nr;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        const int64_t v = row_vertex[r];
        d_full[v * 3] = d_rows[r * 3]; d_full[v * 3 + 1] = d_rows[r * 3 + 1]; d_full[v * 3 + 2] = d_rows[r * 3 + 2];
    }
}

template <typename T>
__global__ void k_update_positions(T *__restrict__ x, int stride, const T *__restrict__ d, T alpha, int64_t V) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        x[v * stride] += alpha * d[v * 3];
        x[v * stride + 1] += alpha * d[v * 3 + 1];
        x[v * stride + 2] += alpha * d[v * 3 + 2];
    }
}

// g.d and max_r |d_r| of a Newton direction: deterministic sum, order-free max.
template <typename T>
__global__ void k_dir_stats(const T *__restrict__ g, const T *__restrict__ d, double *partials, DevScalars *ds,
                            double *out) {
    const unsigned long long nr = ds->n_rows;
    double s = 0.0, m = 0.0;
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < nr;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        const double d0 = d[3 * r], d1 = d[3 * r + 1], d2 = d[3 * r + 2];
        s += (double)g[3 * r] * d0 + (double)g[3 * r + 1] * d1 + (double)g[3 * r + 2] * d2;
        m = fmax(m, d0 * d0 + d1 * d1 + d2 * d2);
    }
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax((unsigned long long *)&out[1], (unsigned long long)__double_as_longlong(m));
    double v[1] = {s};
    grid_sums<1>(v, partials, &ds->done_counter[5], [&](const double *t) { out[0] = t[0]; });
}

#ifdef TTIE_CHECKS
__global__ void k_check_sorted(const unsigned long long *key, int64_t n, DevScalars *ds) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x + 1; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (TTIE_BAD(ds, key[i - 1] <= key[i], 71, i)) return;
}
__global__ void k_check_runs(const uint32_t *run_start, const unsigned long long *pos, const uint32_t *flag, int64_t n,
                             DevScalars *ds) {
    const unsigned long long nb = ds->nnzb;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < nb;
         k += (unsigned long long)gridDim.x * blockDim.x)
        if (TTIE_BAD(ds, run_start[k] < run_start[k + 1], 72, k)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x + 1; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        if (TTIE_BAD(ds, pos[i] == pos[i - 1] + flag[i - 1], 73, i)) return;
}
#endif

// Sum of per-pair 18-vectors per vertex, over the diagonal block runs of the last
// assembly (each lists every (pair, vertex) of that vertex once, in sorted order).
template <typename T>
__global__ void k_vertex_sums(const unsigned long long *__restrict__ key, const uint32_t *__restrict__ val,
                              const uint32_t *__restrict__ run_start, const T *__restrict__ h,
                              const int32_t *__restrict__ row_vertex, const DevScalars *ds, T *__restrict__ out) {
    const unsigned long long nb = ds->nnzb, nr = ds->n_rows;
    for (unsigned long long bi = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; bi < nb;
         bi += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t s = run_start[bi], e = run_start[bi + 1];
        const unsigned long long kk = key[s];
        const unsigned long long row = kk / nr, col = kk - row * nr;
        if (row != col) continue;
        T g0 = 0, g1 = 0, g2 = 0;
        for (uint32_t i = s; i < e; ++i) {
            const uint32_t v = val[i];
            const uint32_t pk = v / 36, r = (v - pk * 36) / 6;
            const T *hp = h + (size_t)pk * 18 + 3 * r;
            g0 += hp[0]; g1 += hp[1]; g2 += hp[2];
        }
        const int64_t vx = row_vertex[row];
        out[vx * 3] = g0; out[vx * 3 + 1] = g1; out[vx * 3 + 2] = g2;
    }
}

// The same sums from the row-bucket assembly: a row's pair items in code order are its
// (pair, vertex) entries of the diagonal block in the same order.
template <typename T>
__global__ void k_vertex_sums_rows(const uint32_t *__restrict__ items2, const unsigned long long *__restrict__ off,
                                   const T *__restrict__ h, const int32_t *__restrict__ row_vertex, const DevScalars *ds,
                                   T *__restrict__ out) {
    const unsigned long long nr = ds->n_rows, n_pair_items = ds->n_active * 6;
    for (unsigned long long row = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; row < nr;
         row += (unsigned long long)gridDim.x * blockDim.x) {
        T g0 = 0, g1 = 0, g2 = 0;
        for (unsigned long long i = off[row]; i < off[row + 1]; ++i) {
            const uint32_t code = items2[i];
            if (code >= n_pair_items) continue;
            const uint32_t pk = code / 6, r = code - pk * 6;
            const T *hp = h + (size_t)pk * 18 + 3 * r;
            g0 += hp[0]; g1 += hp[1]; g2 += hp[2];
        }
        const int64_t vx = row_vertex[row];
        out[vx * 3] = g0; out[vx * 3 + 1] = g1; out[vx * 3 + 2] = g2;
    }
}

// out (V x 3) = H+ v on the assembled rows (vertices of intersecting pairs); other rows 0.
template <typename T>
__global__ void k_bsr_matvec(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                             const T *__restrict__ bval, const int32_t *__restrict__ row_vertex,
                             const T *__restrict__ v, const DevScalars *ds, T *__restrict__ out) {
    const unsigned long long nr = ds->n_rows;
    for (unsigned long long row = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; row < nr;
         row += (unsigned long long)gridDim.x * blockDim.x) {
        T y0 = 0, y1 = 0, y2 = 0;
        for (int b = row_ptr[row]; b < row_ptr[row + 1]; ++b) {
            const T *m = bval + (size_t)b * 9;
            const int64_t cv = row_vertex[col_idx[b]];
            const T c0 = v[cv * 3], c1 = v[cv * 3 + 1], c2 = v[cv * 3 + 2];
            y0 += m[0] * c0 + m[1] * c1 + m[2] * c2;
            y1 += m[3] * c0 + m[4] * c1 + m[5] * c2;
            y2 += m[6] * c0 + m[7] * c1 + m[8] * c2;
        }
        const int64_t rv = row_vertex[row];
        out[rv * 3] = y0; out[rv * 3 + 1] = y1; out[rv * 3 + 2] = y2;
    }
}

int bits_for(unsigned long long v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0ull) ++b;
    return b;
}

}  // namespace

// The row-bucket assembly (TTIE_ASSEMBLY_ROW_BUCKETS), after the factor kernels: buffers sized
// by V and the entry count so that no size is read before the end, then one read of n_rows and
// nnzb.
template <typename T>
static cudaError_t assemble_rows(Ctx &c, T *grad_full, int64_t n_springs, int64_t n_anchors) {
    const int64_t n_act = c.n_active, V = c.V;
    const int64_t n_items = n_act * 6 + 2 * n_springs + n_anchors;
    const int64_t nk = n_act * 36 + 4 * n_springs + n_anchors;
    if (n_items >= (int64_t)UINT32_MAX) return cudaErrorInvalidValue;   // item codes are 32-bit
    const size_t vb = (size_t)(V > 0 ? V : 1), ib = (size_t)(n_items > 0 ? n_items : 1), kb = (size_t)(nk > 0 ? nk : 1);
    TTIE_CUDA_TRY(ensure(c, c.it_cnt, vb * 4));
    TTIE_CUDA_TRY(ensure(c, c.it_fill, vb * 4));
    TTIE_CUDA_TRY(ensure(c, c.dcnt, vb * 4));
    TTIE_CUDA_TRY(ensure(c, c.it_off, (vb + 1) * 8));
    TTIE_CUDA_TRY(ensure(c, c.dptr, (vb + 1) * 8));
    TTIE_CUDA_TRY(ensure(c, c.items, ib * 4));
    TTIE_CUDA_TRY(ensure(c, c.items2, ib * 4));
    TTIE_CUDA_TRY(ensure(c, c.ecol, ib * 6 * 4));
    TTIE_CUDA_TRY(ensure(c, c.eflag, ib * 6));
    TTIE_CUDA_TRY(ensure(c, c.dlist, ib * 6 * 4));
    TTIE_CUDA_TRY(ensure(c, c.row_ptr, (vb + 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.col_idx, kb * 4));
    TTIE_CUDA_TRY(ensure(c, c.bsr_val, kb * 9 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.rhs, vb * 3 * sizeof(T)));
    TTIE_CUDA_TRY(cudaMemsetAsync(c.it_cnt.p, 0, vb * 4, c.stream));
    TTIE_CUDA_TRY(cudaMemsetAsync(c.it_fill.p, 0, vb * 4, c.stream));
    TTIE_CUDA_TRY(cudaMemsetAsync(c.dcnt.p, 0, vb * 4, c.stream));
    if (grad_full) TTIE_CUDA_TRY(cudaMemsetAsync(grad_full, 0, (size_t)V * 3 * sizeof(T), c.stream));
    const int4 *tri4 = (const int4 *)c.tri4.p;
    const int2 *pairs = (const int2 *)c.cand.p;
    const uint32_t *active = (const uint32_t *)c.active.p;
    const unsigned long long *vrow = (const unsigned long long *)c.vrow.p;
    const int2 *edges = (const int2 *)c.el_edges.p;
    const int32_t *anchors = (const int32_t *)c.el_anchor.p;
    const unsigned gI = grid_for(n_items, kThreads);
    launch(c, k_row_items<false>, dim3(gI), dim3(kThreads), tri4, pairs, active, vrow, edges, n_springs, anchors,
           n_anchors, c.ds, (uint32_t *)c.it_cnt.p, (const unsigned long long *)nullptr, (uint32_t *)nullptr);
    TTIE_CUDA_TRY(scan_u32_u64(c, (const uint32_t *)c.it_cnt.p, (unsigned long long *)c.it_off.p, V));
    launch(c, k_row_items<true>, dim3(gI), dim3(kThreads), tri4, pairs, active, vrow, edges, n_springs, anchors,
           n_anchors, c.ds, (uint32_t *)c.it_fill.p, (const unsigned long long *)c.it_off.p, (uint32_t *)c.items.p);
    // rows of up to kBigItems items: a warp each; larger rows: a block each (the big-row
    // launches skip the small rows, one load per row)
    const unsigned gR = grid_for((V + kRowWarps - 1) / kRowWarps, 1, kNumSMs * 16);
    const unsigned gB = grid_for(V, 1, kNumSMs * 2);
    launch(c, k_row_columns<false>, dim3(gR), dim3(32 * kRowWarps), (const uint32_t *)c.items.p,
           (const unsigned long long *)c.it_off.p, tri4, pairs, active, vrow, edges, n_springs, anchors, c.ds,
           (uint32_t *)c.items2.p, (int32_t *)c.ecol.p, (uint8_t *)c.eflag.p, (int32_t *)c.dlist.p,
           (uint32_t *)c.dcnt.p);
    launch(c, k_row_columns<true>, dim3(gB), dim3(kBigThreads), (const uint32_t *)c.items.p,
           (const unsigned long long *)c.it_off.p, tri4, pairs, active, vrow, edges, n_springs, anchors, c.ds,
           (uint32_t *)c.items2.p, (int32_t *)c.ecol.p, (uint8_t *)c.eflag.p, (int32_t *)c.dlist.p,
           (uint32_t *)c.dcnt.p);
    TTIE_CUDA_TRY(scan_u32_u64(c, (const uint32_t *)c.dcnt.p, (unsigned long long *)c.dptr.p, V));
    launch(c, k_row_values<T, false>, dim3(gR), dim3(32 * kRowWarps), (const uint32_t *)c.items2.p,
           (const unsigned long long *)c.it_off.p, (const int32_t *)c.ecol.p, (const int32_t *)c.dlist.p,
           (const uint32_t *)c.dcnt.p, (const unsigned long long *)c.dptr.p, V, (unsigned long long)kb, (const T *)c.zfac.p,
           (const T *)c.el_sfac.p, n_springs, (const T *)c.el_afac.p, (T)c.el_ka, c.ds, (int32_t *)c.row_ptr.p,
           (int32_t *)c.col_idx.p, (T *)c.bsr_val.p, (T *)c.rhs.p, (const int32_t *)c.row_vertex.p, grad_full);
    launch(c, k_row_values<T, true>, dim3(gB), dim3(kBigThreads), (const uint32_t *)c.items2.p,
           (const unsigned long long *)c.it_off.p, (const int32_t *)c.ecol.p, (const int32_t *)c.dlist.p,
           (const uint32_t *)c.dcnt.p, (const unsigned long long *)c.dptr.p, V, (unsigned long long)kb, (const T *)c.zfac.p,
           (const T *)c.el_sfac.p, n_springs, (const T *)c.el_afac.p, (T)c.el_ka, c.ds, (int32_t *)c.row_ptr.p,
           (int32_t *)c.col_idx.p, (T *)c.bsr_val.p, (T *)c.rhs.p, (const int32_t *)c.row_vertex.p, grad_full);
    TTIE_CUDA_TRY(cudaGetLastError());
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_rows, &c.ds->n_rows, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->nnzb, &c.ds->nnzb, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    c.n_rows = (int64_t)c.hs->n_rows;
    c.nnzb = nk > 0 ? (int64_t)c.hs->nnzb : 0;
    return cudaSuccess;
}

template <typename T>
cudaError_t assemble_system(Ctx &c, T *grad_full, bool with_elastic) {
    const int64_t n_act = c.n_active;
    const int64_t V = c.V;
    const bool el = with_elastic && c.have_elastic;
    const int64_t n_springs = el ? c.el_n_edges : 0, n_anchors = el ? c.el_n_anchors : 0;
    TTIE_CUDA_TRY(ensure(c, c.vflag, (size_t)V * 4));
    TTIE_CUDA_TRY(ensure(c, c.vrow, (size_t)(V + 1) * 8));
    TTIE_CUDA_TRY(cudaMemsetAsync(c.vflag.p, 0, (size_t)V * 4, c.stream));
    const int4 *tri4 = (const int4 *)c.tri4.p;
    const int2 *pairs = (const int2 *)c.cand.p;
    const uint32_t *active = (const uint32_t *)c.active.p;
    const unsigned gA = grid_for(n_act, kThreads);
    launch(c, k_mark_vertices, dim3(gA), dim3(kThreads), tri4, pairs, active, c.ds, (uint32_t *)c.vflag.p);
    if (el)
        launch(c, k_el_mark, dim3(grid_for(n_springs + n_anchors, kThreads)), dim3(kThreads), (const int2 *)c.el_edges.p,
               n_springs, (const int32_t *)c.el_anchor.p, n_anchors, (uint32_t *)c.vflag.p);
    TTIE_CUDA_TRY(scan_u32_u64(c, (const uint32_t *)c.vflag.p, (unsigned long long *)c.vrow.p, V));
    TTIE_CUDA_TRY(ensure(c, c.row_vertex, (size_t)(V > 0 ? V : 1) * 4));
    launch(c, k_row_vertex, dim3(grid_for(V, kThreads)), dim3(kThreads), (const uint32_t *)c.vflag.p,
                                                                  (const unsigned long long *)c.vrow.p, V,
                                                                  (int32_t *)c.row_vertex.p, c.ds);
    TTIE_CUDA_TRY(ensure(c, c.zfac, (size_t)(n_act > 0 ? n_act : 1) * kZStride * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)kNumSMs * 16 * 4 * sizeof(double)));
    launch(c, k_factors<T>, dim3(grid_for(n_act, 128, kNumSMs * 8)), dim3(128), (const T *)c.fac.p, c.prm.psd_mode,
           (T *)c.zfac.p, (double *)c.partials.p, c.ds);
    if (el) {   // after k_factors: adds the term's trace to the pairs'
        TTIE_CUDA_TRY(ensure(c, c.el_sfac, (size_t)(n_springs > 0 ? n_springs : 1) * kElStride * sizeof(T)));
        TTIE_CUDA_TRY(ensure(c, c.el_afac, (size_t)(n_anchors > 0 ? n_anchors : 1) * 3 * sizeof(T)));
        launch(c, k_el_factors<T>, dim3(grid_for(n_springs + n_anchors, kThreads, kNumSMs * 4)), dim3(kThreads),
               (const vec4_t<T> *)c.xp.p, (const int2 *)c.el_edges.p, (const T *)c.el_rest.p, n_springs, (T)c.el_k,
               (const int32_t *)c.el_anchor.p, (const T *)c.el_target.p, n_anchors, (T)c.el_ka, (T *)c.el_sfac.p,
               (T *)c.el_afac.p, (double *)c.partials.p, c.ds);
    }
    c.asm_rows = c.prm.assembly_mode == TTIE_ASSEMBLY_ROW_BUCKETS;
    if (c.asm_rows) return assemble_rows<T>(c, grad_full, n_springs, n_anchors);
    const int64_t nk = n_act * 36 + 4 * n_springs + n_anchors;
    if (nk >= (int64_t)UINT32_MAX) return cudaErrorInvalidValue;   // entry indices are 32-bit
    TTIE_CUDA_TRY(ensure(c, c.bkey, (size_t)(nk > 0 ? nk : 1) * 8));
    TTIE_CUDA_TRY(ensure(c, c.bkey2, (size_t)(nk > 0 ? nk : 1) * 8));
    TTIE_CUDA_TRY(ensure(c, c.bval, (size_t)(nk > 0 ? nk : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.bval2, (size_t)(nk > 0 ? nk : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.bflag, (size_t)(nk > 0 ? nk : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.run_start, (size_t)(nk + 1) * 8));
    // the row count decides the key width: one sync
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_rows, &c.ds->n_rows, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    const int64_t nr = (int64_t)c.hs->n_rows;
    c.n_rows = nr;
    launch(c, k_block_keys, dim3(grid_for(n_act * 36, kThreads)), dim3(kThreads), tri4, pairs, active,
           (const unsigned long long *)c.vrow.p, c.ds, (unsigned long long *)c.bkey.p, (uint32_t *)c.bval.p);
    if (el)
        launch(c, k_el_keys, dim3(grid_for(n_springs + n_anchors, kThreads)), dim3(kThreads), (const int2 *)c.el_edges.p,
               n_springs, (const int32_t *)c.el_anchor.p, n_anchors, (const unsigned long long *)c.vrow.p, c.ds,
               (unsigned long long)n_act * 36, (unsigned long long *)c.bkey.p, (uint32_t *)c.bval.p);
    TTIE_CUDA_TRY(cudaGetLastError());
    const int kbits = bits_for((unsigned long long)nr * (unsigned long long)nr);
    TTIE_CUDA_TRY(radix_sort(c, (unsigned long long *)c.bkey.p, (uint32_t *)c.bval.p, (unsigned long long *)c.bkey2.p,
                             (uint32_t *)c.bval2.p, nk, kbits));
#ifdef TTIE_CHECKS
    launch(c, k_check_sorted, dim3(grid_for(nk, kThreads)), dim3(kThreads), (const unsigned long long *)c.bkey.p, nk, c.ds);
#endif
    // run boundaries: flags -> positions
    launch(c, k_run_flags, dim3(grid_for(nk, kThreads)), dim3(kThreads), (const unsigned long long *)c.bkey.p, nk,
                                                                  (uint32_t *)c.bflag.p);
    TTIE_CUDA_TRY(ensure(c, c.gtmp, (size_t)(nk + 1) * 8));
    TTIE_CUDA_TRY(scan_u32_u64(c, (const uint32_t *)c.bflag.p, (unsigned long long *)c.gtmp.p, nk));
    launch(c, k_run_starts, dim3(grid_for(nk, kThreads)), dim3(kThreads), (const uint32_t *)c.bflag.p,
                                                                   (const unsigned long long *)c.gtmp.p, nk,
                                                                   (uint32_t *)c.run_start.p, c.ds);
#ifdef TTIE_CHECKS
    launch(c, k_check_runs, dim3(grid_for(nk, kThreads)), dim3(kThreads), (const uint32_t *)c.run_start.p,
           (const unsigned long long *)c.gtmp.p, (const uint32_t *)c.bflag.p, nk, c.ds);
#endif
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->nnzb, &c.ds->nnzb, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    const int64_t nnzb = nk > 0 ? (int64_t)c.hs->nnzb : 0;
    c.nnzb = nnzb;
    TTIE_CUDA_TRY(ensure(c, c.row_ptr, (size_t)(nr + 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.col_idx, (size_t)(nnzb > 0 ? nnzb : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.bsr_val, (size_t)(nnzb > 0 ? nnzb : 1) * 9 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.rhs, (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T)));
    if (grad_full) TTIE_CUDA_TRY(cudaMemsetAsync(grad_full, 0, (size_t)V * 3 * sizeof(T), c.stream));
    if (nk == 0) {
        TTIE_CUDA_TRY(cudaMemsetAsync(c.row_ptr.p, 0, 4, c.stream));
        return cudaGetLastError();
    }
    launch(c, k_block_values<T>, dim3(grid_for(nnzb, 128, kNumSMs * 16)), dim3(128), 
        (const unsigned long long *)c.bkey.p, (const uint32_t *)c.bval.p, (const uint32_t *)c.run_start.p,
        (const T *)c.zfac.p, c.ds, (int32_t *)c.row_ptr.p, (int32_t *)c.col_idx.p, (T *)c.bsr_val.p, (T *)c.rhs.p,
        (const int32_t *)c.row_vertex.p, grad_full, (unsigned long long)nk, (const T *)c.el_sfac.p, n_springs,
        (const T *)c.el_afac.p, (T)c.el_ka);
    return cudaGetLastError();
}
template cudaError_t assemble_system<float>(Ctx &, float *, bool);
template cudaError_t assemble_system<double>(Ctx &, double *, bool);

// Energy of the elastic term at x into ds->el_energy.
template <typename T> cudaError_t elastic_energy(Ctx &c, const vec4_t<T> *x) {
    const int64_t n = c.el_n_edges + c.el_n_anchors;
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)kNumSMs * 16 * 4 * sizeof(double)));
    launch(c, k_el_factors<T>, dim3(grid_for(n, kThreads, kNumSMs * 4)), dim3(kThreads), x, (const int2 *)c.el_edges.p,
           (const T *)c.el_rest.p, c.el_n_edges, (T)c.el_k, (const int32_t *)c.el_anchor.p, (const T *)c.el_target.p,
           c.el_n_anchors, (T)c.el_ka, (T *)nullptr, (T *)nullptr, (double *)c.partials.p, c.ds);
    return cudaGetLastError();
}
template cudaError_t elastic_energy<float>(Ctx &, const float4 *);
template cudaError_t elastic_energy<double>(Ctx &, const dvec4 *);

// Copies the term's arrays into the context and checks its indices against V (ERR_BAD_INDEX).
template <typename T> cudaError_t elastic_set(Ctx &c, const ttie_elastic *e) {
    const int64_t E = e->n_edges, A = e->n_anchors;
    TTIE_CUDA_TRY(ensure(c, c.el_edges, (size_t)(E > 0 ? E : 1) * sizeof(int2)));
    TTIE_CUDA_TRY(ensure(c, c.el_rest, (size_t)(E > 0 ? E : 1) * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.el_anchor, (size_t)(A > 0 ? A : 1) * sizeof(int32_t)));
    TTIE_CUDA_TRY(ensure(c, c.el_target, (size_t)(A > 0 ? A : 1) * 3 * sizeof(T)));
    if (E > 0) {
        TTIE_CUDA_TRY(cudaMemcpyAsync(c.el_edges.p, e->edges, (size_t)E * sizeof(int2), cudaMemcpyDeviceToDevice, c.stream));
        TTIE_CUDA_TRY(cudaMemcpyAsync(c.el_rest.p, e->rest, (size_t)E * sizeof(T), cudaMemcpyDeviceToDevice, c.stream));
    }
    if (A > 0) {
        TTIE_CUDA_TRY(cudaMemcpyAsync(c.el_anchor.p, e->anchors, (size_t)A * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                      c.stream));
        TTIE_CUDA_TRY(cudaMemcpyAsync(c.el_target.p, e->targets, (size_t)A * 3 * sizeof(T), cudaMemcpyDeviceToDevice,
                                      c.stream));
    }
    if (E + A > 0)
        launch(c, k_el_check, dim3(grid_for(E + A, kThreads)), dim3(kThreads), (const int2 *)c.el_edges.p, E,
               (const int32_t *)c.el_anchor.p, A, c.V, c.ds);
    return cudaGetLastError();
}
template cudaError_t elastic_set<float>(Ctx &, const ttie_elastic *);
template cudaError_t elastic_set<double>(Ctx &, const ttie_elastic *);

template <typename T>
cudaError_t pcg_solve(Ctx &c, const T *rhs, T *out, double rtol, int max_it) {
    const int64_t nr = c.n_rows;
    TTIE_CUDA_TRY(ensure(c, c.dinv, (size_t)(nr > 0 ? nr : 1) * 9 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.pcg_r, (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.pcg_z, (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.pcg_p, (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.pcg_q, (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.pcg_z4, (size_t)(nr > 0 ? nr : 1) * sizeof(vec4_t<T>)));
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)kNumSMs * 16 * 4 * sizeof(double)));
    // reduction slots, then the resident kernel's row partition
    TTIE_CUDA_TRY(ensure(c, c.pcg_sync, (2 * (size_t)kMaxGridPcg + 2) * sizeof(RedSlot) + (kMaxGridPcg + 1) * sizeof(int)));
    const int sms = c.num_sms > 0 ? c.num_sms : kNumSMs;
    // one block per SM at most: fewer participants in every reduction
    int64_t blocks = (nr * kLanesPerRow + kPcgThreads - 1) / kPcgThreads;
    if (blocks > (int64_t)sms) blocks = sms;
    if (blocks > kMaxGridPcg) blocks = kMaxGridPcg;
    if (blocks < 1) blocks = 1;
    // rows resident in shared memory when every block's vectors fit (lean layout: 15 values
    // per row); blocks are balanced by nnz + kRowWeight * rows within that cap; else the
    // global-memory kernel
    // (the Chebyshev preconditioner keeps 6 more values per row, rounded up separately)
    const bool cheb = c.prm.pcg_precond == TTIE_PCG_CHEBYSHEV;
    const int64_t r_cap = cheb ? ((int64_t)kResidentSmem - 4 - 15 - 15) / (21 * (int64_t)sizeof(T) + 4)
                               : ((int64_t)kResidentSmem - 4 - 15) / (15 * (int64_t)sizeof(T) + 4);
    const bool resident = (nr + blocks - 1) / blocks <= r_cap;
    if (cheb && resident) {
        // odd publications; zeros carry tag 0, which no odd publication has
        TTIE_CUDA_TRY(ensure(c, c.pcg_z4b, (size_t)(nr > 0 ? nr : 1) * sizeof(vec4_t<T>)));
        TTIE_CUDA_TRY(cudaMemsetAsync(c.pcg_z4b.p, 0, (size_t)(nr > 0 ? nr : 1) * sizeof(vec4_t<T>), c.stream));
        TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->pcg_products, 0, sizeof(unsigned long long), c.stream));
    }
    RedSlot *slots = (RedSlot *)c.pcg_sync.p;
    int *rpart = (int *)(slots + 2 * kMaxGridPcg + 2);
    double *part = (double *)c.partials.p;
    const unsigned g = grid_for(nr, kThreads, kNumSMs * 4);
    TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->bar_count, 0, 2 * sizeof(unsigned int), c.stream));
    launch(c, k_pcg_setup<T>, dim3(g), dim3(kThreads), (const int32_t *)c.row_ptr.p, (const int32_t *)c.col_idx.p,
                                                 (const T *)c.bsr_val.p, c.prm.mu_rel, (T *)c.dinv.p, rhs, out,
                                                 (T *)c.pcg_r.p, (T *)c.pcg_z.p, (T *)c.pcg_p.p, part,
                                                 (vec4_t<T> *)c.pcg_z4.p, (unsigned long long *)slots,
                                                 (int)((2 * kMaxGridPcg + 2) * sizeof(RedSlot) / sizeof(unsigned long long)),
                                                 resident ? rpart : nullptr, (int)blocks, (int)r_cap, kRowWeight, c.ds);
    TTIE_CUDA_TRY(cudaGetLastError());
    PcgArgs<T> args;
    args.row_ptr = (const int32_t *)c.row_ptr.p;
    args.col_idx = (const int32_t *)c.col_idx.p;
    args.bval = (const T *)c.bsr_val.p;
    args.dinv = (const T *)c.dinv.p;
    args.x = out;
    args.r = (T *)c.pcg_r.p;
    args.z = (T *)c.pcg_z.p;
    args.p = (T *)c.pcg_p.p;
    args.q = (T *)c.pcg_q.p;
    args.z4 = (vec4_t<T> *)c.pcg_z4.p;
    args.z4b = cheb && resident ? (vec4_t<T> *)c.pcg_z4b.p : nullptr;
    args.cheb_degree = c.prm.pcg_cheb_degree > 0 ? c.prm.pcg_cheb_degree : 2;
    c.pcg_cheb = cheb && resident;
    args.partA = part;
    args.partB = part + 2 * kNumSMs * 8;
    args.rtol2 = rtol * rtol;
    args.max_it = max_it;
    args.ds = c.ds;
    args.slots = slots;
    args.part = rpart;
    args.withhold = c.prm.test_withhold;
    ++c.n_launch;
    if (c.prm.profile) cudaEventRecord(c.ev[8], c.stream);
    if (resident) {
        const void *kern = cheb ? (const void *)k_pcg_resident<T, true> : (const void *)k_pcg_resident<T, false>;
        TTIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kResidentSmem));
        int smem = kResidentSmem;
        void *kargs[] = {&args, &smem};
        TTIE_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3((unsigned)blocks), dim3(kPcgThreads), kargs,
                                                  (size_t)kResidentSmem, c.stream));
    } else {
        void *kargs[] = {&args};
        TTIE_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_pcg_persistent<T>, dim3((unsigned)blocks),
                                                  dim3(kPcgThreads), kargs, 0, c.stream));
    }
    if (c.prm.profile) cudaEventRecord(c.ev[9], c.stream);
    return cudaGetLastError();
}
template cudaError_t pcg_solve<float>(Ctx &, const float *, float *, double, int);
template cudaError_t pcg_solve<double>(Ctx &, const double *, double *, double, int);

template <typename T>
cudaError_t axpy_positions(Ctx &c, const vec4_t<T> *x, const T *d, T alpha, vec4_t<T> *out) {
    launch(c, k_axpy_positions<T>, dim3(grid_for(c.V, kThreads)), dim3(kThreads), x, d, alpha, c.V, out);
    return cudaGetLastError();
}
template cudaError_t axpy_positions<float>(Ctx &, const float4 *, const float *, float, float4 *);
template cudaError_t axpy_positions<double>(Ctx &, const dvec4 *, const double *, double, dvec4 *);

template <typename T>
cudaError_t scatter_direction(Ctx &c, const T *d_rows, T *d_full) {
    TTIE_CUDA_TRY(cudaMemsetAsync(d_full, 0, (size_t)c.V * 3 * sizeof(T), c.stream));
    launch(c, k_scatter_rows<T>, dim3(grid_for(c.n_rows, kThreads)), dim3(kThreads), d_rows, (const int32_t *)c.row_vertex.p,
                                                                              c.ds, d_full);
    return cudaGetLastError();
}
template cudaError_t scatter_direction<float>(Ctx &, const float *, float *);
template cudaError_t scatter_direction<double>(Ctx &, const double *, double *);

template <typename T>
cudaError_t update_positions(Ctx &c, T *x, int stride, const T *d_full, T alpha) {
    launch(c, k_update_positions<T>, dim3(grid_for(c.V, kThreads)), dim3(kThreads), x, stride, d_full, alpha, c.V);
    return cudaGetLastError();
}
template cudaError_t update_positions<float>(Ctx &, float *, int, const float *, float);
template cudaError_t update_positions<double>(Ctx &, double *, int, const double *, double);

// out_dev[0] = g.d, out_dev[1] = max_r |d_r| (d given per assembled row)
template <typename T> cudaError_t direction_stats(Ctx &c, const T *g, const T *d, double *out_dev) {
    TTIE_CUDA_TRY(cudaMemsetAsync(out_dev, 0, 2 * sizeof(double), c.stream));
    launch(c, k_dir_stats<T>, dim3(grid_for(c.n_rows, kThreads, kNumSMs * 4)), dim3(kThreads), g, d,
           (double *)c.partials.p, c.ds, out_dev);
    TTIE_CUDA_TRY(cudaGetLastError());
    // the max was accumulated on the squared norm
    return cudaSuccess;
}
template cudaError_t direction_stats<float>(Ctx &, const float *, const float *, double *);
template cudaError_t direction_stats<double>(Ctx &, const double *, const double *, double *);

// PCG on explicit buffers (no context): the setup and persistent kernels above, on
// caller-provided work vectors and state.  ds must hold n_rows and trace (mu = mu_rel *
// trace / (3 n_rows)) with its counters, tickets and barrier words zeroed.
cudaError_t pcg_run_raw(cudaStream_t stream, int num_sms, const int32_t *row_ptr, const int32_t *col_idx,
                        const float *bval, int64_t n_rows, double mu_rel, const float *rhs, float *out, float *dinv,
                        float *r, float *z, float *p, float *q, double *partials, DevScalars *ds, double rtol,
                        int max_it) {
    const unsigned g = grid_for(n_rows, kThreads, kNumSMs * 4);
    k_pcg_setup<float><<<g, kThreads, 0, stream>>>(row_ptr, col_idx, bval, mu_rel, dinv, rhs, out, r, z, p, partials,
                                                   nullptr, nullptr, 0, nullptr, 0, 0, 0, ds);
    TTIE_CUDA_TRY(cudaGetLastError());
    PcgArgs<float> args;
    args.row_ptr = row_ptr;
    args.col_idx = col_idx;
    args.bval = bval;
    args.dinv = dinv;
    args.x = out;
    args.r = r;
    args.z = z;
    args.p = p;
    args.q = q;
    args.z4 = nullptr;   // only the block-resident kernel uses the vector mirror, slots and partition
    args.slots = nullptr;
    args.part = nullptr;
    args.withhold = 0;
    args.partA = partials;
    args.partB = partials + 2 * kNumSMs * 8;
    args.rtol2 = rtol * rtol;
    args.max_it = max_it;
    args.ds = ds;
    int blocks = (int)((n_rows * kLanesPerRow + kPcgThreads - 1) / kPcgThreads);
    if (blocks > num_sms) blocks = num_sms;
    if (blocks < 1) blocks = 1;
    void *kargs[] = {&args};
    return cudaLaunchCooperativeKernel((const void *)k_pcg_persistent<float>, dim3((unsigned)blocks),
                                       dim3(kPcgThreads), kargs, 0, stream);
}

template <typename T> cudaError_t vertex_sums(Ctx &c, const T *h, T *out) {
    TTIE_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)c.V * 3 * sizeof(T), c.stream));
    if (c.nnzb == 0) return cudaSuccess;
    if (c.asm_rows)
        launch(c, k_vertex_sums_rows<T>, dim3(grid_for(c.n_rows, kThreads)), dim3(kThreads), (const uint32_t *)c.items2.p,
               (const unsigned long long *)c.it_off.p, h, (const int32_t *)c.row_vertex.p, c.ds, out);
    else
        launch(c, k_vertex_sums<T>, dim3(grid_for(c.nnzb, kThreads)), dim3(kThreads), (const unsigned long long *)c.bkey.p,
               (const uint32_t *)c.bval.p, (const uint32_t *)c.run_start.p, h, (const int32_t *)c.row_vertex.p, c.ds, out);
    return cudaGetLastError();
}
template cudaError_t vertex_sums<float>(Ctx &, const float *, float *);
template cudaError_t vertex_sums<double>(Ctx &, const double *, double *);

template <typename T> cudaError_t bsr_matvec(Ctx &c, const T *v, T *out) {
    TTIE_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)c.V * 3 * sizeof(T), c.stream));
    if (c.n_rows == 0) return cudaSuccess;
    launch(c, k_bsr_matvec<T>, dim3(grid_for(c.n_rows, kThreads)), dim3(kThreads), (const int32_t *)c.row_ptr.p,
           (const int32_t *)c.col_idx.p, (const T *)c.bsr_val.p, (const int32_t *)c.row_vertex.p, v, c.ds, out);
    return cudaGetLastError();
}
template cudaError_t bsr_matvec<float>(Ctx &, const float *, float *);
template cudaError_t bsr_matvec<double>(Ctx &, const double *, double *);

}  // namespace ttie
