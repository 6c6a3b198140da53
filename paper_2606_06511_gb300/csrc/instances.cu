// Batched independent instances (pair mode TTIE_PAIRS_INTRA_GROUP).
//
// When pairs never cross groups, the assembled system is block-diagonal by group and every
// group is its own problem.  One Newton step then solves them all at once but independently:
//   * the PCG of every instance runs in one launch, one thread block per instance, with
//     block-local reductions only (no grid-wide synchronisation), each instance with its
//     own regulariser mu_i = mu_rel * mean diag(H+_i), its own stopping test and its own
//     step cap (max_step * the instance's mean edge length);
//   * the line search walks the same ladder of trial steps for all instances, and each
//     instance accepts the first trial that meets its own Armijo test (or leaves it without
//     intersecting pairs); its energy is the sum of T over its own pairs, added in a fixed
//     order.
// Layout: every instance's vertices must be numbered contiguously (rows of the block-CSR
// system are sorted by vertex, so an instance's rows are then a contiguous range); the pair
// lists come out of the LBVH with group-prefixed Morton keys, so an instance's pairs are a
// contiguous range of every pair list too.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "pcg_common.cuh"

namespace ttie {

namespace {

constexpr int kThreads = 256;
constexpr int kInstLanes = 4;             // lanes sharing a row in the product
constexpr int kInstSmemMax = 220 * 1024;  // dynamic shared memory per instance block, at most

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// group of every vertex; a vertex used by triangles of two groups is an error
__global__ void k_vertex_group(const int4 *__restrict__ tri4, const int32_t *__restrict__ grp, int64_t F,
                               int32_t *vgroup, DevScalars *ds) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        const int4 t = tri4[f];
        const int g = grp[f];
        const int v[3] = {t.x, t.y, t.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int old = atomicCAS(&vgroup[v[k]], -1, g);
            if (old != -1 && old != g) atomicOr(&ds->err, ERR_GROUP);
        }
    }
}

// mean edge length of every group's triangles (leaves of the group in LBVH order, fixed order)
template <typename T>
__global__ void k_group_edges(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4,
                              const uint32_t *__restrict__ perm, const int2 *__restrict__ group_range, int G,
                              double *edge) {
    const int lane = threadIdx.x & 31;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += (gridDim.x * blockDim.x) >> 5) {
        const int2 r = group_range[g];
        double s = 0.0;
        for (int i = r.x + lane; i <= r.y; i += 32) {
            const int4 t = tri4[perm[i]];
            const v3<T> a = xyz<T>(x[t.x]), b = xyz<T>(x[t.y]), c = xyz<T>(x[t.z]);
            const v3<T> e0 = b - a, e1 = c - b, e2 = a - c;
            s += sqrt((double)dot(e0, e0)) + sqrt((double)dot(e1, e1)) + sqrt((double)dot(e2, e2));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) edge[g] = r.y >= r.x ? s / (3.0 * (r.y - r.x + 1)) : 0.0;
    }
}

__global__ void k_inst_init(Inst *inst, int G) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        Inst I = {};
        I.first = INT_MAX;
        I.last = -1;
        inst[g] = I;
    }
}

__global__ void k_inst_rows(const int32_t *__restrict__ row_vertex, const int32_t *__restrict__ vgroup, DevScalars *ds,
                            int G, Inst *inst) {
    const long long nr = (long long)ds->n_rows;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr; r += (long long)gridDim.x * blockDim.x) {
        const int g = vgroup[row_vertex[r]];
        if (TTIE_BAD(ds, g >= 0 && g < G, 81, g)) continue;
        atomicMin(&inst[g].first, (int)r);
        atomicMax(&inst[g].last, (int)r);
        atomicAdd(&inst[g].count, 1);
    }
}

__global__ void k_inst_check(Inst *inst, int G, const int32_t *__restrict__ row_ptr, DevScalars *ds) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        Inst &I = inst[g];
        if (I.count > 0 && I.last - I.first + 1 != I.count) {
            atomicOr(&ds->err, ERR_GROUP);
            I.count = 0;   // not solved: the error is reported after the step's kernels
        }
        if (I.count == 0) I.first = 0;
        I.nnz = I.count > 0 ? row_ptr[I.first + I.count] - row_ptr[I.first] : 0;
    }
}

// Per-instance ranges of the active-pair list of the last evaluation (pairs of a group are
// contiguous there).
__global__ void k_inst_segments(const int2 *__restrict__ pairs, const uint32_t *__restrict__ active,
                                const int32_t *__restrict__ grp, const DevScalars *ds, Inst *inst) {
    const long long n = (long long)ds->n_active;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int g = grp[pairs[active[k]].x];
        if (k == 0 || grp[pairs[active[k - 1]].x] != g) inst[g].seg_lo = (int)k;
        if (k == n - 1 || grp[pairs[active[k + 1]].x] != g) inst[g].seg_hi = (int)(k + 1);
    }
}

__global__ void k_inst_clear_segments(Inst *inst, int G) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        inst[g].seg_lo = 0;
        inst[g].seg_hi = 0;
    }
}

// Energy (sum of T = (a b)^2 over the instance's intersecting pairs, fixed order) and count,
// one warp per instance; into e0/n0 (at x) or et/nt (at a trial).
template <typename T>
__global__ void k_inst_energy(const T *__restrict__ fac, int fac_stride, int G, int at_trial, Inst *inst) {
    const int lane = threadIdx.x & 31;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += (gridDim.x * blockDim.x) >> 5) {
        const int lo = inst[g].seg_lo, hi = inst[g].seg_hi;
        double s = 0.0;
        for (int k = lo + lane; k < hi; k += 32) {
            const double ab = (double)fac[(size_t)k * fac_stride] * (double)fac[(size_t)k * fac_stride + 1];
            s += ab * ab;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (at_trial) {
                inst[g].et = s;
                inst[g].nt = hi - lo;
            } else {
                inst[g].e0 = s;
                inst[g].n0 = hi - lo;
            }
        }
    }
}

template <typename T> struct InstPcgArgs {
    const int32_t *row_ptr, *col_idx;
    const T *bval, *rhs;          // rhs = -g on the rows
    T *x;                         // the direction d on the rows (output)
    T *r, *u, *p, *s, *w, *dinv;  // row vectors of instances kept in global memory
    T *cd, *crr;                  // the Chebyshev preconditioner's d and D^-1 residual (global layout)
    unsigned long long *acc;      // their row partials: 3 x rows
    const double *edge;           // mean edge length per instance
    const int32_t *ids;           // the instances of this launch, in the order they are taken
    int n_ids;
    unsigned int *queue;          // next position of ids to take (zeroed before the launch)
    Inst *inst;
    double mu_rel, rtol2, max_step;
    int max_it;
    long long n_rows;
    int cheb;                     // Chebyshev preconditioner: 0 never, 1 instances in shared memory, 2 all
    int cheb_degree;
};

template <typename T> struct InstView {
    T *x, *r, *u, *p, *s, *w, *di;
    T *d, *rr;                    // Chebyshev: the polynomial's direction and D^-1 residual
    unsigned long long *pg, *pd, *pr;   // per-row partials of r.u, w.u, r.r (accumulator bits)
    const T *val;
    bool resident;
    int nrow, nnz, r0, b0;
    int *rp, *col;                // local row offsets and local columns (resident only)
};

template <typename T>
__device__ __forceinline__ int inst_rowp(const InstPcgArgs<T> &a, const InstView<T> &v, int i) {
    return v.resident ? v.rp[i] : a.row_ptr[v.r0 + i] - v.b0;
}
template <typename T>
__device__ __forceinline__ int inst_col(const InstPcgArgs<T> &a, const InstView<T> &v, int b) {
    return v.resident ? v.col[b] : a.col_idx[v.b0 + b] - v.r0;
}

// Sums of N per-row accumulator arrays part[i][0..n) in an order fixed by n alone (not by the
// block's size): 256 virtual lanes each add rows l, l + 256, ... in order, then warp 0 adds the
// lanes (lane j: virtual lanes j, j + 32, ..., then a shuffle tree).  Every thread gets the
// totals.
template <typename T, int THREADS, int N>
__device__ __forceinline__ void rows_totals(const unsigned long long *const (&part)[N], int n, Acc<T> (&out)[N]) {
    constexpr int VL = 256;
    __shared__ unsigned long long lanes[N][VL];
    __shared__ unsigned long long total[N];
    for (int l = threadIdx.x; l < VL; l += THREADS) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            Acc<T> s;
            for (int i = l; i < n; i += VL) s.add(Acc<T>::from_bits(part[k][i]));
            lanes[k][l] = s.bits();
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            Acc<T> s;
#pragma unroll
            for (int j = 0; j < VL / 32; ++j) s.add(Acc<T>::from_bits(lanes[k][threadIdx.x + 32 * j]));
#pragma unroll
            for (int o = 16; o; o >>= 1) s.add(s.shfl_xor(0xffffffffu, o, 32));
            if (threadIdx.x == 0) total[k] = s.bits();
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = Acc<T>::from_bits(total[k]);
}

template <typename T, int THREADS>
__device__ __forceinline__ Acc<T> rows_total(const unsigned long long *part, int n) {
    const unsigned long long *const p[1] = {part};
    Acc<T> out[1];
    rows_totals<T, THREADS, 1>(p, n, out);
    return out[0];
}

// The PCG of instance gid by the whole block (k_pcg_instances takes the instances).  With the
// Chebyshev preconditioner (a.cheb: every instance, or the ones whose rows sit in shared
// memory) the first kChebWarm iterations use 3x3 block Jacobi; their CG coefficients give the
// Lanczos estimate of lambda_max(D^-1 A), and CG restarts with M^-1 = p_k(D^-1 A) D^-1, the
// degree-k Chebyshev polynomial on [lambda_max / kChebRatio, lambda_max] (cheb_coefficients),
// applied by k more products per iteration.  In one block the polynomial's products need
// only block barriers, while each iteration's reductions and barriers are what an instance's
// solve waits on, so fewer iterations pay.
template <typename T, int THREADS>
__device__ __forceinline__ void inst_pcg_one(const InstPcgArgs<T> &a, int gid, int smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ T s_c1[kChebMaxDeg], s_c2[kChebMaxDeg], s_thi;
    __shared__ int s_restart;
    Inst *I = a.inst + gid;
    InstView<T> v;
    v.nrow = I->count;
    if (v.nrow <= 0) return;
    v.r0 = I->first;
    v.b0 = a.row_ptr[v.r0];
    v.nnz = a.row_ptr[v.r0 + v.nrow] - v.b0;
    // resident layout: 3 accumulator words, 27 values (x r u p s w, 9 of M^-1) per row, 6 more
    // (d, rr) when the Chebyshev preconditioner may run, the local row offsets, then the matrix
    const int per_row = 27 + (a.cheb ? 6 : 0);
    const size_t vec_bytes = ((size_t)v.nrow * (per_row * sizeof(T) + 24) + (size_t)(v.nrow + 1) * 4 + 15) / 16 * 16;
    const size_t mat_bytes = (size_t)v.nnz * (9 * sizeof(T) + 4);
    v.resident = vec_bytes + mat_bytes <= (size_t)smem_bytes;
    const bool cheb = a.cheb == 2 || (a.cheb == 1 && v.resident);
    if (v.resident) {
        v.pg = (unsigned long long *)smem; v.pd = v.pg + v.nrow; v.pr = v.pd + v.nrow;
        v.x = (T *)(v.pr + v.nrow); v.r = v.x + 3 * v.nrow; v.u = v.r + 3 * v.nrow; v.p = v.u + 3 * v.nrow;
        v.s = v.p + 3 * v.nrow; v.w = v.s + 3 * v.nrow; v.di = v.w + 3 * v.nrow;
        v.d = v.di + 9 * v.nrow; v.rr = v.d + 3 * v.nrow;   // inside the layout only when a.cheb
        v.rp = (int *)(v.di + (size_t)(per_row - 18) * v.nrow);
        T *val = (T *)(smem + vec_bytes);
        v.col = (int *)(val + (size_t)9 * v.nnz);
        for (int i = threadIdx.x; i < 9 * v.nnz; i += THREADS) val[i] = a.bval[(size_t)v.b0 * 9 + i];
        for (int i = threadIdx.x; i < v.nnz; i += THREADS) v.col[i] = a.col_idx[v.b0 + i] - v.r0;
        for (int i = threadIdx.x; i <= v.nrow; i += THREADS) v.rp[i] = a.row_ptr[v.r0 + i] - v.b0;
        v.val = val;
    } else {
        const size_t o = (size_t)v.r0 * 3;
        v.x = a.x + o; v.r = a.r + o; v.u = a.u + o; v.p = a.p + o; v.s = a.s + o; v.w = a.w + o;
        v.d = a.cd + o; v.rr = a.crr + o;
        v.di = a.dinv + (size_t)v.r0 * 9;
        v.pg = a.acc + v.r0; v.pd = a.acc + a.n_rows + v.r0; v.pr = a.acc + 2 * a.n_rows + v.r0;
        v.rp = nullptr;
        v.col = nullptr;
        v.val = a.bval + (size_t)v.b0 * 9;
    }
    __syncthreads();
    // mu_i from the instance's own trace, then M^-1, r = rhs, u = M^-1 r, x = p = s = 0
    for (int lr = threadIdx.x; lr < v.nrow; lr += THREADS) {
        Acc<T> t;
        for (int b = inst_rowp(a, v, lr); b < inst_rowp(a, v, lr + 1); ++b)
            if (inst_col(a, v, b) == lr) {
                const T *m = v.val + (size_t)b * 9;
                t.add_prod(m[0] + m[4] + m[8], T(1));
                break;
            }
        v.pg[lr] = t.bits();
    }
    __syncthreads();
    const T mu = (T)(a.mu_rel * rows_total<T, THREADS>(v.pg, v.nrow).value() / (3.0 * v.nrow));
    for (int lr = threadIdx.x; lr < v.nrow; lr += THREADS) {
        const T zero9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        const T *diag = zero9;
        for (int b = inst_rowp(a, v, lr); b < inst_rowp(a, v, lr + 1); ++b)
            if (inst_col(a, v, b) == lr) { diag = v.val + (size_t)b * 9; break; }
        T di[9];
        inv3(diag, mu, di);
#pragma unroll
        for (int i = 0; i < 9; ++i) v.di[lr * 9 + i] = di[i];
        const T r0 = a.rhs[(size_t)(v.r0 + lr) * 3], r1 = a.rhs[(size_t)(v.r0 + lr) * 3 + 1],
                r2 = a.rhs[(size_t)(v.r0 + lr) * 3 + 2];
        const T u[3] = {di[0] * r0 + di[1] * r1 + di[2] * r2, di[3] * r0 + di[4] * r1 + di[5] * r2,
                        di[6] * r0 + di[7] * r1 + di[8] * r2};
        const T rv[3] = {r0, r1, r2};
        Acc<T> g, q;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            v.x[lr * 3 + i] = T(0);
            v.r[lr * 3 + i] = rv[i];
            v.u[lr * 3 + i] = u[i];
            v.p[lr * 3 + i] = T(0);
            v.s[lr * 3 + i] = T(0);
            g.add_prod(rv[i], u[i]);
            q.add_prod(rv[i], rv[i]);
        }
        v.pg[lr] = g.bits();
        v.pr[lr] = q.bits();
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, sub = lane & (kInstLanes - 1);
    const unsigned gmask = ((1u << kInstLanes) - 1u) << (lane & ~(kInstLanes - 1));
    // dst = (A + mu I) src on the instance's rows, kInstLanes lanes per row summed in a fixed
    // order; with pd, each row's dst.src too
    const auto product = [&](const T *src, T *dst, unsigned long long *pd) {
        for (int lr = threadIdx.x / kInstLanes; lr < v.nrow; lr += THREADS / kInstLanes) {
            T y0 = 0, y1 = 0, y2 = 0;
            const int be = inst_rowp(a, v, lr + 1);
            for (int b = inst_rowp(a, v, lr) + sub; b < be; b += kInstLanes) {
                const int c = inst_col(a, v, b);
                const T *m = v.val + (size_t)b * 9;
                const T c0 = src[c * 3], c1 = src[c * 3 + 1], c2 = src[c * 3 + 2];
                y0 += m[0] * c0 + m[1] * c1 + m[2] * c2;
                y1 += m[3] * c0 + m[4] * c1 + m[5] * c2;
                y2 += m[6] * c0 + m[7] * c1 + m[8] * c2;
            }
#pragma unroll
            for (int o = kInstLanes / 2; o; o >>= 1) {
                y0 += __shfl_xor_sync(gmask, y0, o, kInstLanes);
                y1 += __shfl_xor_sync(gmask, y1, o, kInstLanes);
                y2 += __shfl_xor_sync(gmask, y2, o, kInstLanes);
            }
            if (sub == 0) {
                const T w0 = y0 + mu * src[lr * 3], w1 = y1 + mu * src[lr * 3 + 1], w2 = y2 + mu * src[lr * 3 + 2];
                dst[lr * 3] = w0; dst[lr * 3 + 1] = w1; dst[lr * 3 + 2] = w2;
                if (pd) {
                    Acc<T> wu;
                    wu.add_prod(w0, src[lr * 3]);
                    wu.add_prod(w1, src[lr * 3 + 1]);
                    wu.add_prod(w2, src[lr * 3 + 2]);
                    pd[lr] = wu.bits();
                }
            }
        }
    };
    const T rtol2 = (T)a.rtol2;
    T rr0 = T(0), gamma_prev = T(1), alpha_prev = T(1), rr_last = T(0);
    bool stop_next = false;
    int it = 0, prods = 0;
    // Chebyshev: kit counts the iterations since CG (re)started; al, be the block-Jacobi ones'
    int kit = 0;
    bool cheb_on = false, cheb_tried = false;
    double al[kChebWarm], be[kChebWarm];
    while (true) {
        // w = (A + mu I) u and the rows' w.u
        product(v.u, v.w, v.pd);
        ++prods;
        __syncthreads();
        Acc<T> tot[3];
        {
            const unsigned long long *const parts[3] = {v.pg, v.pd, v.pr};
            rows_totals<T, THREADS, 3>(parts, v.nrow, tot);
        }
        const Acc<T> gam = tot[0], del = tot[1], rr = tot[2];
        const T g = gam.approx(), d = del.approx(), r2 = rr.approx();
        if (it == 0) rr0 = r2;
        rr_last = r2;
        if (stop_next || it >= a.max_it || r2 <= rtol2 * rr0 || !isfinite(r2)) break;
        T alpha, beta = T(0);
        bool ok;
        if ((cheb ? kit : it) == 0) {
            alpha = g / d;
            ok = d > T(0) && isfinite(alpha);
        } else {
            beta = g / gamma_prev;
            const T den = del.minus(gam.over(alpha_prev).times(beta)).approx();
            alpha = g / den;
            ok = den > T(0) && isfinite(alpha);
        }
        if (!ok) {
            if (it > 0) break;
            alpha = T(1);      // breakdown at the first step keeps x = M^-1 r0 (preconditioned gradient)
            beta = T(0);
            stop_next = true;
        }
        gamma_prev = g;
        alpha_prev = alpha;
        // the block-Jacobi iterations' coefficients; after the last of them the polynomial's
        // (thread 0, from the same values every thread holds), and CG restarts with it
        bool restart = false;
        if (cheb && !cheb_tried && !stop_next && kit < kChebWarm) {
            al[kit] = (double)alpha;
            be[kit] = (double)beta;
            if (kit == kChebWarm - 1 && it + 1 < a.max_it) {
                cheb_tried = true;
                if (threadIdx.x == 0)
                    s_restart = cheb_coefficients<T>(al, be, a.cheb_degree, s_c1, s_c2, &s_thi) ? 1 : 0;
                __syncthreads();
                restart = s_restart != 0;
            }
        }
        const bool cheb_now = cheb_on || restart;
        const T thi = cheb_now ? s_thi : T(0);
        for (int lr = threadIdx.x; lr < v.nrow; lr += THREADS) {
            T rv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int k = lr * 3 + i;
                const T pi = v.u[k] + beta * v.p[k];
                const T si = v.w[k] + beta * v.s[k];
                v.p[k] = pi;
                v.s[k] = si;
                v.x[k] += alpha * pi;
                rv[i] = v.r[k] - alpha * si;
                v.r[k] = rv[i];
            }
            const T *di = v.di + lr * 9;
            Acc<T> gp, qp;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T zi = di[3 * i] * rv[0] + di[3 * i + 1] * rv[1] + di[3 * i + 2] * rv[2];
                if (cheb_now) {
                    v.rr[lr * 3 + i] = zi;   // D^-1 r; the polynomial's first direction and y
                    v.d[lr * 3 + i] = zi * thi;
                    v.u[lr * 3 + i] = zi * thi;
                } else {
                    v.u[lr * 3 + i] = zi;
                    gp.add_prod(rv[i], zi);
                }
                qp.add_prod(rv[i], rv[i]);
            }
            if (!cheb_now) v.pg[lr] = gp.bits();
            v.pr[lr] = qp.bits();
        }
        ++it;
        if (cheb_now) {
            // u = p_k(D^-1 A) D^-1 r: rr -= D^-1 (A + mu I) d, d = c1 d + c2 rr, u += d
            for (int j = 0; j < a.cheb_degree; ++j) {
                __syncthreads();
                product(v.d, v.w, nullptr);   // w is free until the next iteration's product
                ++prods;
                __syncthreads();
                const T c1 = s_c1[j], c2 = s_c2[j];
                for (int lr = threadIdx.x; lr < v.nrow; lr += THREADS) {
                    const T *di = v.di + lr * 9;
                    const T w0 = v.w[lr * 3], w1 = v.w[lr * 3 + 1], w2 = v.w[lr * 3 + 2];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const int k = lr * 3 + i;
                        const T rri = v.rr[k] - (di[3 * i] * w0 + di[3 * i + 1] * w1 + di[3 * i + 2] * w2);
                        v.rr[k] = rri;
                        const T dn = c1 * v.d[k] + c2 * rri;
                        v.d[k] = dn;
                        v.u[k] += dn;
                    }
                }
            }
            for (int lr = threadIdx.x; lr < v.nrow; lr += THREADS) {
                Acc<T> gp;
#pragma unroll
                for (int i = 0; i < 3; ++i) gp.add_prod(v.r[lr * 3 + i], v.u[lr * 3 + i]);
                v.pg[lr] = gp.bits();
            }
            kit = cheb_on ? kit + 1 : 0;   // CG restarts with the polynomial
            cheb_on = true;
        } else {
            ++kit;
        }
        __syncthreads();
    }
    // g.d and max |d_r| of the instance's direction; the step cap; the direction out
    T dm = T(0);
    for (int lr = threadIdx.x; lr < v.nrow; lr += THREADS) {
        T n2 = T(0);
        Acc<T> gd;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T di = v.x[lr * 3 + i];
            gd.add_prod(-a.rhs[(size_t)(v.r0 + lr) * 3 + i], di);
            n2 += di * di;
        }
        v.pg[lr] = gd.bits();
        dm = fmax(dm, n2);
    }
    __shared__ T s_max[THREADS / 32];
#pragma unroll
    for (int o = 16; o; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (lane == 0) s_max[threadIdx.x >> 5] = dm;
    __syncthreads();
    const Acc<T> gdt = rows_total<T, THREADS>(v.pg, v.nrow);
    dm = T(0);
    for (int k = 0; k < THREADS / 32; ++k) dm = fmax(dm, s_max[k]);
    const double dmax = sqrt((double)dm);
    const double cap = a.max_step * a.edge[gid];
    const double scale = (cap > 0.0 && dmax > cap) ? cap / dmax : 1.0;
    for (int i = threadIdx.x; i < 3 * v.nrow; i += THREADS) {
        const T di = v.x[i] * (T)scale;
        a.x[(size_t)v.r0 * 3 + i] = di;
    }
    if (threadIdx.x == 0) {
        I->iters = it;
        I->prods = prods;
        I->rel = rr0 > T(0) ? sqrt((double)rr_last / (double)rr0) : 0.0;
        I->gd = gdt.value() * scale;
    }
}

// PCG (Chronopoulos-Gear form, as in the grid-wide solver) of one instance at a time per
// block: a persistent launch whose blocks take the instances from a queue in the order of ids
// (one atomic per instance), so one launch covers every instance, whatever their sizes.  Each
// row's product is summed by kInstLanes lanes in a fixed order and every reduction goes
// through rows_total, so the result depends neither on THREADS nor on which block takes an
// instance (the tuner picks THREADS, the blocks per SM and the order).
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) k_pcg_instances(InstPcgArgs<T> a, int smem_bytes) {
    __shared__ int s_take;
    while (true) {
        __syncthreads();   // s_take of the previous instance has been read by every thread
        if (threadIdx.x == 0) s_take = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int take = s_take;
        if (take >= a.n_ids) return;
        inst_pcg_one<T, THREADS>(a, a.ids[take], smem_bytes);
    }
}

// Line search bookkeeping per instance
__global__ void k_ls_init(Inst *inst, int G) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        Inst &I = inst[g];
        I.pending = I.n0 > 0 ? 1 : 0;
        I.alpha = 0.0;
        I.e_new = I.e0;
        I.n_new = I.n0;
    }
}

__global__ void k_ls_accept(Inst *inst, int G, double alpha, double armijo_c, int last, unsigned int *n_pending) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        Inst &I = inst[g];
        if (!I.pending) continue;
        if (I.nt == 0 || I.et <= I.e0 + armijo_c * alpha * I.gd || last) {
            I.alpha = alpha;
            I.e_new = I.et;
            I.n_new = I.nt;
            I.pending = 0;
        } else {
            atomicAdd(n_pending, 1u);
        }
    }
}

// Candidate pairs of the instances whose line search is still open (order kept).
__global__ void k_pending_flags(const int2 *__restrict__ pairs, int64_t n, const int32_t *__restrict__ grp,
                                const Inst *__restrict__ inst, uint32_t *__restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = inst[grp[pairs[i].x]].pending ? 1u : 0u;
}
__global__ void k_pending_scatter(const int2 *__restrict__ pairs, int64_t n, const uint32_t *__restrict__ flag,
                                  const unsigned long long *__restrict__ off, int2 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[off[i]] = pairs[i];
}

// Trial positions x + alpha d with the step read from device memory (graph replays).
template <typename T>
__global__ void k_axpy_dev(const vec4_t<T> *__restrict__ x, const T *__restrict__ d, const DevScalars *ds, int64_t V,
                           vec4_t<T> *__restrict__ out) {
    const T a = (T)ds->ls_alpha;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        vec4_t<T> p = x[v];
        p.x += a * d[v * 3]; p.y += a * d[v * 3 + 1]; p.z += a * d[v * 3 + 2];
        out[v] = p;
    }
}

__global__ void k_ls_accept_dev(Inst *inst, int G, double armijo_c, DevScalars *ds) {
    const double alpha = ds->ls_alpha;
    const bool last = ds->ls_last != 0.0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        Inst &I = inst[g];
        if (!I.pending) continue;
        if (I.nt == 0 || I.et <= I.e0 + armijo_c * alpha * I.gd || last) {
            I.alpha = alpha;
            I.e_new = I.et;
            I.n_new = I.nt;
            I.pending = 0;
        } else {
            atomicAdd(&ds->n_pending, 1u);
        }
    }
}

template <typename T>
__global__ void k_update_grouped(T *__restrict__ x, int stride, const T *__restrict__ d,
                                 const int32_t *__restrict__ vgroup, const Inst *__restrict__ inst, int64_t V) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int g = vgroup[v];
        if (g < 0) continue;
        const T a = (T)inst[g].alpha;
        x[v * stride] += a * d[v * 3];
        x[v * stride + 1] += a * d[v * 3 + 1];
        x[v * stride + 2] += a * d[v * 3 + 2];
    }
}

// Totals of a batched step in fixed order: energy and pairs after the step, largest PCG
// iteration count and relative residual, sum of g.d, smallest accepted step, instances
// solved, and the PCG work (iterations x 3x3 blocks, iterations x rows) summed over them.
constexpr int kTotThreads = 512;
__global__ void __launch_bounds__(kTotThreads) k_inst_totals(const Inst *inst, int G, const int32_t *row_ptr,
                                                             double *out) {
    // per thread over instances g = tid, tid + kTotThreads, ..., then a tree over the threads:
    // a fixed order, so the sums do not depend on timing
    double e = 0.0, gd = 0.0, rel = 0.0, amin = 1e300, wb = 0.0, wr = 0.0, n = 0.0;
    int it = 0, solved = 0;
    for (int g = threadIdx.x; g < G; g += kTotThreads) {
        const Inst &I = inst[g];
        e += I.e_new;
        n += (double)I.n_new;
        if (I.n0 > 0) {
            gd += I.gd;
            rel = fmax(rel, I.rel);
            it = max(it, I.iters);
            amin = fmin(amin, I.alpha);
            ++solved;
        }
        if (I.count > 0) {
            wb += (double)I.prods * (row_ptr[I.first + I.count] - row_ptr[I.first]);
            wr += (double)I.prods * I.count;
        }
    }
    __shared__ double s_d[7][kTotThreads];
    __shared__ int s_i[2][kTotThreads];
    const int t = threadIdx.x;
    s_d[0][t] = e; s_d[1][t] = gd; s_d[2][t] = rel; s_d[3][t] = amin; s_d[4][t] = wb; s_d[5][t] = wr; s_d[6][t] = n;
    s_i[0][t] = it; s_i[1][t] = solved;
    __syncthreads();
    for (int h = kTotThreads / 2; h; h >>= 1) {
        if (t < h) {
            s_d[0][t] += s_d[0][t + h];
            s_d[1][t] += s_d[1][t + h];
            s_d[2][t] = fmax(s_d[2][t], s_d[2][t + h]);
            s_d[3][t] = fmin(s_d[3][t], s_d[3][t + h]);
            s_d[4][t] += s_d[4][t + h];
            s_d[5][t] += s_d[5][t + h];
            s_d[6][t] += s_d[6][t + h];
            s_i[0][t] = max(s_i[0][t], s_i[0][t + h]);
            s_i[1][t] += s_i[1][t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[7] = s_d[4][0];
        out[8] = s_d[5][0];
        out[0] = s_d[0][0];
        out[1] = s_d[6][0];
        out[2] = (double)s_i[0][0];
        out[3] = s_d[2][0];
        out[4] = s_d[1][0];
        out[5] = s_i[1][0] ? s_d[3][0] : 0.0;
        out[6] = (double)s_i[1][0];
    }
}

}  // namespace

cudaError_t instance_vertex_groups(Ctx &c) {
    TTIE_CUDA_TRY(ensure(c, c.vgroup, (size_t)c.V * 4));
    launch(c, k_fill_i32, dim3(grid_for(c.V, kThreads)), dim3(kThreads), (int32_t *)c.vgroup.p, c.V, -1);
    launch(c, k_vertex_group, dim3(grid_for(c.F, kThreads)), dim3(kThreads), (const int4 *)c.tri4.p,
           (const int32_t *)c.grp.p, c.F, (int32_t *)c.vgroup.p, c.ds);
    return cudaGetLastError();
}

template <typename T> cudaError_t instance_edges(Ctx &c, const vec4_t<T> *x) {
    TTIE_CUDA_TRY(ensure(c, c.iedge, (size_t)(c.n_groups > 0 ? c.n_groups : 1) * sizeof(double)));
    launch(c, k_group_edges<T>, dim3(grid_for((int64_t)c.n_groups * 32, kThreads)), dim3(kThreads), x,
           (const int4 *)c.tri4.p, (const uint32_t *)c.perm.p, (const int2 *)c.group_range.p, c.n_groups,
           (double *)c.iedge.p);
    return cudaGetLastError();
}
template cudaError_t instance_edges<float>(Ctx &, const float4 *);
template cudaError_t instance_edges<double>(Ctx &, const dvec4 *);

cudaError_t instance_layout(Ctx &c) {
    const int G = c.n_groups;
    TTIE_CUDA_TRY(ensure(c, c.inst, (size_t)(G > 0 ? G : 1) * sizeof(Inst)));
    launch(c, k_inst_init, dim3(grid_for(G, kThreads)), dim3(kThreads), (Inst *)c.inst.p, G);
    launch(c, k_inst_rows, dim3(grid_for(c.n_rows, kThreads)), dim3(kThreads), (const int32_t *)c.row_vertex.p,
           (const int32_t *)c.vgroup.p, c.ds, G, (Inst *)c.inst.p);
    launch(c, k_inst_check, dim3(grid_for(G, kThreads)), dim3(kThreads), (Inst *)c.inst.p, G,
           (const int32_t *)c.row_ptr.p, c.ds);
    return cudaGetLastError();
}

template <typename T> cudaError_t instance_energies(Ctx &c, const int2 *pairs, int at_trial) {
    const int G = c.n_groups;
    launch(c, k_inst_clear_segments, dim3(grid_for(G, kThreads)), dim3(kThreads), (Inst *)c.inst.p, G);
    if (c.n_active > 0)
        launch(c, k_inst_segments, dim3(grid_for(c.n_active, kThreads)), dim3(kThreads), pairs,
               (const uint32_t *)c.active.p, (const int32_t *)c.grp.p, (const DevScalars *)c.ds, (Inst *)c.inst.p);
    launch(c, k_inst_energy<T>, dim3(grid_for((int64_t)G * 32, kThreads)), dim3(kThreads), (const T *)c.fac.p,
           kFacStride, G, at_trial, (Inst *)c.inst.p);
    return cudaGetLastError();
}
template cudaError_t instance_energies<float>(Ctx &, const int2 *, int);
template cudaError_t instance_energies<double>(Ctx &, const int2 *, int);

// The batched PCG is one persistent launch over all instances (k_pcg_instances takes them from
// a queue).  Its schedule is tuned on the first batched step of a context by timing every
// candidate on the actual system: threads per block, blocks per SM (each block's shared
// memory is the SM's divided among them; an instance whose rows and matrix do not fit runs
// from global memory) and the order of the queue (largest instance first, or as numbered).
// Results do not depend on the schedule, only the time does.  With the environment variable
// TTIE_TUNE_CACHE naming a file, the choice is kept there (one line per device, precision,
// instance count and row count) and read back by later contexts instead of tuning again.
constexpr int kTunerThreads[] = {256, 512, 1024};
constexpr int kTunerBlocksPerSM[] = {1, 2, 4};

template <typename T, int THREADS>
cudaError_t launch_inst(Ctx &c, const InstPcgArgs<T> &a, int bps, cudaStream_t st) {
    // per block: the SM's shared memory divided among bps blocks, beside the kernel's static share
    cudaFuncAttributes fa;
    TTIE_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void *)k_pcg_instances<T, THREADS>));
    int optin = 0, per_sm = 0;
    TTIE_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
    TTIE_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c.device));
    int smem = std::min(optin, per_sm / bps - 1024) - (int)fa.sharedSizeBytes;
    smem = std::max(0, std::min(smem, kInstSmemMax)) / 16 * 16;
    TTIE_CUDA_TRY(cudaFuncSetAttribute((const void *)k_pcg_instances<T, THREADS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int resident = 0;
    TTIE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_pcg_instances<T, THREADS>, THREADS,
                                                                (size_t)smem));
    if (resident < 1) resident = 1;
    const int sms = c.num_sms > 0 ? c.num_sms : kNumSMs;
    const int grid = std::max(1, std::min(a.n_ids, std::min(resident, bps) * sms));
    TTIE_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), st));
    ++c.n_launch;
    k_pcg_instances<T, THREADS><<<dim3((unsigned)grid), dim3(THREADS), (size_t)smem, st>>>(a, smem);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inst_threads(Ctx &c, const InstPcgArgs<T> &a, int threads, int bps, cudaStream_t st) {
    switch (threads) {
    case 128: return launch_inst<T, 128>(c, a, bps, st);
    case 256: return launch_inst<T, 256>(c, a, bps, st);
    case 512: return launch_inst<T, 512>(c, a, bps, st);
    default: return launch_inst<T, 1024>(c, a, bps, st);
    }
}

static std::string tune_key(Ctx &c, int n_inst, long long rows) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c.device) != cudaSuccess) prop.name[0] = 0;
    std::string dev(prop.name);
    for (char &ch : dev)
        if (ch == ' ' || ch == '"') ch = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "inst_pcg %s f%d pc%d n%d rows%lld", dev.c_str(), c.prm.precision == TTIE_F64 ? 64 : 32,
             c.prm.pcg_precond, n_inst, rows);
    return buf;
}

// the cache file holds one JSON object per line: {"key": "...", "threads": T, "blocks_per_sm": B, "order": O}
static bool tune_read(const std::string &key, int *threads, int *bps, int *order) {
    const char *path = getenv("TTIE_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    const std::string want = "{\"key\": \"" + key + "\",";
    while (fgets(line, sizeof line, f)) {
        if (strncmp(line, want.c_str(), want.size()) != 0) continue;
        int t = 0, b = 0, o = 0;
        if (sscanf(line + want.size(), " \"threads\": %d, \"blocks_per_sm\": %d, \"order\": %d", &t, &b, &o) == 3 &&
            (t == 256 || t == 512 || t == 1024) && (b == 1 || b == 2 || b == 4) && (o == 0 || o == 1)) {
            *threads = t; *bps = b; *order = o;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void tune_write(const std::string &key, int threads, int bps, int order, float ms) {
    const char *path = getenv("TTIE_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"threads\": %d, \"blocks_per_sm\": %d, \"order\": %d, \"ms\": %.4f}\n", key.c_str(),
            threads, bps, order, ms);
    fclose(f);
}

template <typename T> cudaError_t instance_pcg(Ctx &c, const T *rhs, T *out) {
    const int64_t nr = c.n_rows;
    const int G = c.n_groups;
    const size_t n3 = (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T);
    TTIE_CUDA_TRY(ensure(c, c.pcg_r, n3));
    TTIE_CUDA_TRY(ensure(c, c.pcg_z, n3));
    TTIE_CUDA_TRY(ensure(c, c.pcg_p, n3));
    TTIE_CUDA_TRY(ensure(c, c.pcg_q, n3));
    TTIE_CUDA_TRY(ensure(c, c.pcg_w, n3));
    TTIE_CUDA_TRY(ensure(c, c.dinv, (size_t)(nr > 0 ? nr : 1) * 9 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.inst_acc, (size_t)(nr > 0 ? nr : 1) * 3 * 8));
    const int cheb = c.prm.pcg_precond == TTIE_PCG_CHEBYSHEV ? 2 : c.prm.pcg_precond == TTIE_PCG_AUTO ? 1 : 0;
    if (cheb == 2) {   // instances outside shared memory keep d and rr in global memory
        TTIE_CUDA_TRY(ensure(c, c.inst_cd, n3));
        TTIE_CUDA_TRY(ensure(c, c.inst_crr, n3));
    }
    TTIE_CUDA_TRY(ensure(c, c.inst_ids, (size_t)(G > 0 ? G : 1) * 4 * 2));
    // the instances with rows, in the two queue orders: largest first (by rows, then nnz), as numbered
    std::vector<Inst> h(G);
    TTIE_CUDA_TRY(cudaMemcpyAsync(h.data(), c.inst.p, (size_t)G * sizeof(Inst), cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    std::vector<int32_t> ids;
    for (int g = 0; g < G; ++g)
        if (h[g].count > 0) ids.push_back(g);
    const int n = (int)ids.size();
    std::vector<int32_t> both(ids);
    std::stable_sort(both.begin(), both.end(), [&](int32_t x, int32_t y) {
        return h[x].count != h[y].count ? h[x].count > h[y].count : h[x].nnz > h[y].nnz;
    });
    both.insert(both.end(), ids.begin(), ids.end());
    if (n > 0)
        TTIE_CUDA_TRY(cudaMemcpyAsync(c.inst_ids.p, both.data(), both.size() * 4, cudaMemcpyHostToDevice, c.stream));
    InstPcgArgs<T> a;
    a.row_ptr = (const int32_t *)c.row_ptr.p;
    a.col_idx = (const int32_t *)c.col_idx.p;
    a.bval = (const T *)c.bsr_val.p;
    a.rhs = rhs;
    a.x = out;
    a.r = (T *)c.pcg_r.p;
    a.u = (T *)c.pcg_z.p;
    a.p = (T *)c.pcg_p.p;
    a.s = (T *)c.pcg_q.p;
    a.w = (T *)c.pcg_w.p;
    a.dinv = (T *)c.dinv.p;
    a.acc = (unsigned long long *)c.inst_acc.p;
    a.edge = (const double *)c.iedge.p;
    a.inst = (Inst *)c.inst.p;
    a.n_ids = n;
    a.queue = &c.ds->inst_queue;
    a.mu_rel = c.prm.mu_rel;
    a.rtol2 = c.prm.pcg_rtol * c.prm.pcg_rtol;
    a.max_step = c.prm.max_step;
    a.max_it = c.prm.pcg_max_it;
    a.cheb = cheb;
    a.cheb_degree = c.prm.pcg_cheb_degree > 0 ? c.prm.pcg_cheb_degree : 2;
    a.cd = (T *)c.inst_cd.p;
    a.crr = (T *)c.inst_crr.p;
    a.n_rows = nr;
    if (n == 0) return cudaSuccess;
    // the schedule: a caller's block size with the tuned rest, the cache, or a timed sweep
    if (c.inst_tuned[0] == 0) {
        const std::string key = tune_key(c, n, (long long)nr);
        int t = 0, b = 0, o = 0;
        if (tune_read(key, &t, &b, &o)) {
            c.inst_tuned[0] = t; c.inst_tuned[1] = b; c.inst_tuned[2] = o;
        } else {
            cudaEvent_t e0, e1;
            TTIE_CUDA_TRY(cudaEventCreate(&e0));
            TTIE_CUDA_TRY(cudaEventCreate(&e1));
            float best = -1.f;
            for (int tt : kTunerThreads) {
                if (c.prm.inst_threads > 0 && tt != c.prm.inst_threads) continue;
                for (int bb : kTunerBlocksPerSM)
                    for (int oo = 0; oo < 2; ++oo) {
                        a.ids = (const int32_t *)c.inst_ids.p + (oo ? n : 0);
                        TTIE_CUDA_TRY(cudaEventRecord(e0, c.stream));
                        TTIE_CUDA_TRY(launch_inst_threads<T>(c, a, tt, bb, c.stream));
                        TTIE_CUDA_TRY(cudaEventRecord(e1, c.stream));
                        TTIE_CUDA_TRY(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (best < 0.f || ms < best) {
                            best = ms; c.inst_tuned[0] = tt; c.inst_tuned[1] = bb; c.inst_tuned[2] = oo;
                        }
                    }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (c.inst_tuned[0] == 0) { c.inst_tuned[0] = 512; c.inst_tuned[1] = 1; c.inst_tuned[2] = 0; }
            else tune_write(key, c.inst_tuned[0], c.inst_tuned[1], c.inst_tuned[2], best);
        }
    }
    const int threads = c.prm.inst_threads > 0 ? c.prm.inst_threads : c.inst_tuned[0];
    a.ids = (const int32_t *)c.inst_ids.p + (c.inst_tuned[2] ? n : 0);
    if (c.prm.profile) cudaEventRecord(c.ev[8], c.stream);
    TTIE_CUDA_TRY(launch_inst_threads<T>(c, a, threads, c.inst_tuned[1], c.stream));
    if (c.prm.profile) cudaEventRecord(c.ev[9], c.stream);
    return cudaGetLastError();
}
template cudaError_t instance_pcg<float>(Ctx &, const float *, float *);
template cudaError_t instance_pcg<double>(Ctx &, const double *, double *);

cudaError_t instance_ls_init(Ctx &c) {
    launch(c, k_ls_init, dim3(grid_for(c.n_groups, kThreads)), dim3(kThreads), (Inst *)c.inst.p, c.n_groups);
    return cudaGetLastError();
}

cudaError_t instance_ls_accept(Ctx &c, double alpha, int last, unsigned int *d_pending) {
    TTIE_CUDA_TRY(cudaMemsetAsync(d_pending, 0, sizeof(unsigned int), c.stream));
    launch(c, k_ls_accept, dim3(grid_for(c.n_groups, kThreads)), dim3(kThreads), (Inst *)c.inst.p, c.n_groups, alpha,
           c.prm.armijo_c, last, d_pending);
    return cudaGetLastError();
}

cudaError_t instance_pending_pairs(Ctx &c, const int2 *pairs, int64_t n, Buf &out, int64_t *n_out) {
    *n_out = 0;
    if (n <= 0) return cudaSuccess;
    TTIE_CUDA_TRY(ensure(c, c.gtmp, (size_t)n * 4));
    TTIE_CUDA_TRY(ensure(c, c.word_off, (size_t)(n + 1) * 8));
    auto *flag = (uint32_t *)c.gtmp.p;
    auto *off = (unsigned long long *)c.word_off.p;
    launch(c, k_pending_flags, dim3(grid_for(n, kThreads)), dim3(kThreads), pairs, n, (const int32_t *)c.grp.p,
           (const Inst *)c.inst.p, flag);
    TTIE_CUDA_TRY(scan_u32_u64(c, flag, off, n));
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_cand, off + n, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    const int64_t m = (int64_t)c.hs->n_cand;
    TTIE_CUDA_TRY(ensure(c, out, (size_t)(m > 0 ? m : 1) * sizeof(int2)));
    if (m > 0)
        launch(c, k_pending_scatter, dim3(grid_for(n, kThreads)), dim3(kThreads), pairs, n, (const uint32_t *)flag,
               (const unsigned long long *)off, (int2 *)out.p);
    *n_out = m;
    return cudaGetLastError();
}

template <typename T>
cudaError_t instance_trial_graph(Ctx &c, const vec4_t<T> *xp, const T *dir, vec4_t<T> *xt, const int2 *cand,
                                 int64_t ns, cudaGraphExec_t *exec, unsigned long long *kernels) {
    const int G = c.n_groups;
    // everything sized before the capture: nothing may be allocated inside it
    TTIE_CUDA_TRY(prepare_energy_eval<T>(c, ns));
    TTIE_CUDA_TRY(ensure(c, c.ls_flag, (size_t)(ns > 0 ? ns : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.ls_off, (size_t)(ns + 1) * 8));
    TTIE_CUDA_TRY(ensure(c, c.ls_cand, (size_t)(ns > 0 ? ns : 1) * sizeof(int2)));
    auto *flag = (uint32_t *)c.ls_flag.p;
    auto *off = (unsigned long long *)c.ls_off.p;
    const unsigned long long launches0 = c.n_launch;
    cudaGraph_t graph = nullptr;
    // captured on a stream of the context's own (the caller's stream may be the legacy default
    // stream, which cannot be captured); the graph is then launched on the caller's stream
    if (!c.cap_stream) TTIE_CUDA_TRY(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    const cudaStream_t main_stream = c.stream;
    c.stream = c.cap_stream;
    cudaError_t eb = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
    if (eb != cudaSuccess) {
        c.stream = main_stream;
        return eb;
    }
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMemcpyAsync(&c.ds->ls_alpha, &c.hs->ls_alpha, 2 * sizeof(double), cudaMemcpyHostToDevice,
                                 c.stream)) != cudaSuccess) break;
        // the candidates of the instances still open (their count stays on the device)
        if (ns > 0) {
            launch(c, k_pending_flags, dim3(grid_for(ns, kThreads)), dim3(kThreads), cand, ns, (const int32_t *)c.grp.p,
                   (const Inst *)c.inst.p, flag);
            if ((e = scan_u32_u64(c, (const uint32_t *)flag, off, ns)) != cudaSuccess) break;
            launch(c, k_pending_scatter, dim3(grid_for(ns, kThreads)), dim3(kThreads), cand, ns, (const uint32_t *)flag,
                   (const unsigned long long *)off, (int2 *)c.ls_cand.p);
        }
        launch(c, k_axpy_dev<T>, dim3(grid_for(c.V, kThreads)), dim3(kThreads), xp, dir, (const DevScalars *)c.ds, c.V,
               xt);
        if ((e = energy_eval_nosync<T>(c, xt, (const int2 *)c.ls_cand.p, ns, (const unsigned long long *)off + ns)) !=
            cudaSuccess)
            break;
        launch(c, k_inst_clear_segments, dim3(grid_for(G, kThreads)), dim3(kThreads), (Inst *)c.inst.p, G);
        if (ns > 0)
            launch(c, k_inst_segments, dim3(grid_for(ns, kThreads)), dim3(kThreads), (const int2 *)c.ls_cand.p,
                   (const uint32_t *)c.active.p, (const int32_t *)c.grp.p, (const DevScalars *)c.ds, (Inst *)c.inst.p);
        launch(c, k_inst_energy<T>, dim3(grid_for((int64_t)G * 32, kThreads)), dim3(kThreads), (const T *)c.ab.p, 2, G, 1,
               (Inst *)c.inst.p);
        if ((e = cudaMemsetAsync(&c.ds->n_pending, 0, sizeof(unsigned int), c.stream)) != cudaSuccess) break;
        launch(c, k_ls_accept_dev, dim3(grid_for(G, kThreads)), dim3(kThreads), (Inst *)c.inst.p, G, c.prm.armijo_c,
               c.ds);
        if ((e = cudaMemcpyAsync(&c.hs->n_pending, &c.ds->n_pending, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                 c.stream)) != cudaSuccess) break;
        e = cudaGetLastError();
    } while (false);
    const cudaError_t ec = cudaStreamEndCapture(c.stream, &graph);
    c.stream = main_stream;
    *kernels = c.n_launch - launches0;
    c.n_launch = launches0;   // captured, not launched: every replay counts them
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return e;
}
template cudaError_t instance_trial_graph<float>(Ctx &, const float4 *, const float *, float4 *, const int2 *, int64_t,
                                                 cudaGraphExec_t *, unsigned long long *);
template cudaError_t instance_trial_graph<double>(Ctx &, const dvec4 *, const double *, dvec4 *, const int2 *, int64_t,
                                                  cudaGraphExec_t *, unsigned long long *);

template <typename T> cudaError_t instance_update(Ctx &c, T *x, int stride, const T *d_full) {
    launch(c, k_update_grouped<T>, dim3(grid_for(c.V, kThreads)), dim3(kThreads), x, stride, d_full,
           (const int32_t *)c.vgroup.p, (const Inst *)c.inst.p, c.V);
    return cudaGetLastError();
}
template cudaError_t instance_update<float>(Ctx &, float *, int, const float *);
template cudaError_t instance_update<double>(Ctx &, double *, int, const double *);

cudaError_t instance_totals(Ctx &c, double *d_out) {
    launch(c, k_inst_totals, dim3(1), dim3(kTotThreads), (const Inst *)c.inst.p, c.n_groups, (const int32_t *)c.row_ptr.p,
           d_out);
    return cudaGetLastError();
}

}  // namespace ttie
