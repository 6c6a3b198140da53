// Assembly of the PSD Hessian and gradient into 3x3 block CSR (the PCG that solves the
// system is in pcg.cu).
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
#include "reduce.cuh"

namespace ttie {

namespace {

// Per intersecting pair, for each of its 6 vertices r: [z1 (3), z2 (3), z3 (3), g (3)] (the
// rows 3r..3r+2 of the three PSD factors and of the gradient), so a 3x3 block (r, c) reads
// two contiguous 36-byte runs.
constexpr int kZStride = 72;
constexpr int kZVertex = 12;


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

// PSD factors z1, z2, z3 and the gradient of each intersecting pair; trace of H+.  A block of
// fac_threads threads handles as many pairs: their rows of t_c values and gradients are read
// into shared memory and their factor rows written out of it, each by the whole block in
// consecutive words (a thread's own row is kFacStride or kZStride values long, so direct
// per-thread row accesses would touch a separate sector per thread and word).
// (32 pairs per block for FP64 rows, so the staging stays at 29 KB of static shared memory)
template <typename T> __host__ __device__ constexpr int fac_threads() { return sizeof(T) == 4 ? 64 : 32; }

template <typename T>
__global__ void __launch_bounds__(fac_threads<T>()) k_factors(const T *__restrict__ fac, int psd_mode, T *__restrict__ z,
                                                              double *partials, DevScalars *ds) {
    constexpr int kFacThreads = fac_threads<T>();
    __shared__ T s_in[kFacThreads * kFacStride];
    __shared__ T s_out[kFacThreads * kZStride];
    const unsigned long long n = ds->n_active;
    double tr = 0.0;
    for (unsigned long long k0 = (unsigned long long)blockIdx.x * kFacThreads; k0 < n;
         k0 += (unsigned long long)gridDim.x * kFacThreads) {
        const int rows = (int)min((unsigned long long)kFacThreads, n - k0);
        for (int i = threadIdx.x; i < rows * kFacStride; i += kFacThreads) s_in[i] = fac[k0 * kFacStride + i];
        __syncthreads();
        if (threadIdx.x < rows) {
            const T *r = s_in + threadIdx.x * kFacStride;
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
            T *o = s_out + threadIdx.x * kZStride;
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
        __syncthreads();
        for (int i = threadIdx.x; i < rows * kZStride; i += kFacThreads) z[k0 * kZStride + i] = s_out[i];
        __syncthreads();
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
// The 12 values of one vertex's factors, [z1 (3), z2 (3), z3 (3), g (3)], 16-byte aligned (a
// pair's row is 72 values): three 16-byte loads for FP32, six for FP64.
template <typename T> __device__ __forceinline__ void load_vertex_factors(const T *__restrict__ p, T (&o)[12]);
template <> __device__ __forceinline__ void load_vertex_factors<float>(const float *__restrict__ p, float (&o)[12]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float4 v = __ldg(q + i);
        o[4 * i] = v.x; o[4 * i + 1] = v.y; o[4 * i + 2] = v.z; o[4 * i + 3] = v.w;
    }
}
template <> __device__ __forceinline__ void load_vertex_factors<double>(const double *__restrict__ p, double (&o)[12]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double2 v = __ldg(q + i);
        o[2 * i] = v.x; o[2 * i + 1] = v.y;
    }
}
static_assert(kZStride % 4 == 0 && kZVertex % 4 == 0, "factor rows and vertices start on 16 bytes");

template <typename T>
__device__ __forceinline__ void add_pair_entry(const T *__restrict__ z, uint32_t pk, uint32_t r, uint32_t c, bool diag,
                                               T (&m)[9], T &g0, T &g1, T &g2) {
    T zr[12], zc[12];
    load_vertex_factors<T>(z + (size_t)pk * kZStride + r * kZVertex, zr);
    load_vertex_factors<T>(z + (size_t)pk * kZStride + c * kZVertex, zc);
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
    launch(c, k_factors<T>, dim3(grid_for(n_act, fac_threads<T>(), kNumSMs * 16)), dim3(fac_threads<T>()),
           (const T *)c.fac.p, c.prm.psd_mode, (T *)c.zfac.p, (double *)c.partials.p, c.ds);
    if (el) {   // after k_factors: adds the term's trace to the pairs'
        TTIE_CUDA_TRY(ensure(c, c.el_sfac, (size_t)(n_springs > 0 ? n_springs : 1) * kElStride * sizeof(T)));
        TTIE_CUDA_TRY(ensure(c, c.el_afac, (size_t)(n_anchors > 0 ? n_anchors : 1) * 3 * sizeof(T)));
        launch(c, k_el_factors<T>, dim3(grid_for(n_springs + n_anchors, kThreads, kNumSMs * 4)), dim3(kThreads),
               (const vec4_t<T> *)c.xp.p, (const int2 *)c.el_edges.p, (const T *)c.el_rest.p, n_springs, (T)c.el_k,
               (const int32_t *)c.el_anchor.p, (const T *)c.el_target.p, n_anchors, (T)c.el_ka, (T *)c.el_sfac.p,
               (T *)c.el_afac.p, (double *)c.partials.p, c.ds);
    }
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
    bool in_second = false;
    TTIE_CUDA_TRY(radix_sort(c, (unsigned long long *)c.bkey.p, (uint32_t *)c.bval.p, (unsigned long long *)c.bkey2.p,
                             (uint32_t *)c.bval2.p, nk, kbits, &in_second));
    if (in_second) {   // the sorted entries are in the scratch buffers: they become bkey / bval
        std::swap(c.bkey, c.bkey2);
        std::swap(c.bval, c.bval2);
    }
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

template <typename T> cudaError_t vertex_sums(Ctx &c, const T *h, T *out) {
    TTIE_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)c.V * 3 * sizeof(T), c.stream));
    if (c.nnzb == 0) return cudaSuccess;
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
