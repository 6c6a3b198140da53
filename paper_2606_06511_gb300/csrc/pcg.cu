// The PCG solve of the assembled Newton system (H+ + mu I) d = -g: the setup kernel
// (inverse diagonal blocks, first residual and preconditioned vector, the block-resident
// kernel's row partition), the persistent global-memory kernel and the block-resident kernel
// (block-Jacobi or Chebyshev preconditioner), and their host entry points.
#include <algorithm>

#include "common.cuh"
#include "pcg_common.cuh"
#include "reduce.cuh"

namespace ttie {

namespace {

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
    int no_cache;            // resident kernel: matrix rows read from global memory even where they fit
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

// Hint: bring [b, e) of global memory into L2 (one bulk prefetch; the 16-byte-aligned part
// inside the range, so no byte outside [b, e) rounded down to 16 bytes is touched).
__device__ __forceinline__ void prefetch_l2(const void *b, const void *e) {
    const size_t lo = __cvta_generic_to_global(b) & ~(size_t)15, hi = __cvta_generic_to_global(e) & ~(size_t)15;
    if (hi > lo) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}
// waves of rows ahead that a warp prefetches its matrix rows when they are not cached
constexpr int kPrefetchWaves = 2;

// w = (A + mu I) u on the block's rows (THREADS threads), u of every row read from the
// published vectors src with tag t (loc: the block's own rows of u, for the shift); returns the
// rows' w.u.  A load that never sees tag t sets *bad.  rev: the rows in reverse order.
// Successive products alternate the order, so that a matrix streamed from global memory
// (larger than L2) starts each pass on the part the previous pass left in L2 (noisy sphere,
// 201 MB of blocks: 20.8 -> 19.2 ms for 200 iterations).
template <typename T, int THREADS>
__device__ __forceinline__ Acc<T> resident_product(const PcgArgs<T> &a, const ResidentView<T> &v,
                                                   const vec4_t<T> *src, const T *loc, T mu, unsigned t, int *bad,
                                                   bool rev) {
    if (v.gathered) {
        // gather every block's column vector first: all loads of a thread in flight together
        // words not yet tagged t are loaded again, all of a thread's together
        constexpr int U = 4;
        for (int j0 = threadIdx.x; j0 < v.nnz; j0 += U * THREADS) {
            vec4_t<T> g[U];
            unsigned pend = 0;
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int j = j0 + k * THREADS;
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
                        const int j = j0 + k * THREADS;
                        v.gu[3 * j] = g[k].x; v.gu[3 * j + 1] = g[k].y; v.gu[3 * j + 2] = g[k].z;
                        pend &= ~(1u << k);
                    }
                if (!pend) break;
                if (wc.out() || *(volatile int *)bad) { *bad = 1; break; }
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (pend >> k & 1u) g[k] = ld_row<T>(&src[v.col[j0 + k * THREADS]]);
            }
        }
        __syncthreads();
    }
    // lanes per row: 2, 4, 16 and 32 measured slower (noisy sphere, 200 iterations: 40.7, 33.1,
    // 37.5 and 51.0 ms against 18.4 ms with fixed turns)
    constexpr int LPR = kLanesPerRow;
    const int lane = threadIdx.x & 31, sub = lane & (LPR - 1);
    const unsigned gmask = ((1u << LPR) - 1u) << (lane & ~(LPR - 1));
    Acc<T> wu;
    // Streamed rows (1024 threads) are handed out to warps as they finish, 32 / LPR
    // consecutive rows at a time in loop order, not dealt in fixed turns: the rows' costs
    // differ, and every warp waits for the slowest one at the reduction that follows (noisy
    // sphere, 200 iterations: 18.1 -> 15.1 ms).  Rows in shared memory (512 threads) keep the
    // fixed turns, whose products are too short to repay the counter's two barriers (cloth:
    // 1.90 against 2.04 ms for 85 iterations).
    constexpr bool kHandOut = THREADS >= 1024;
    __shared__ int s_next_row;
    if (kHandOut) {
        __syncthreads();   // the previous product's last reads of the counter are done
        if (threadIdx.x == 0) s_next_row = 0;
        __syncthreads();
    }
    for (int turn = 0;; ++turn) {
        int wbase;
        if (kHandOut) {
            wbase = 0;
            if (lane == 0) wbase = atomicAdd(&s_next_row, 32 / LPR);
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
        } else {
            wbase = turn * (THREADS / LPR) + (threadIdx.x >> 5) * (32 / LPR);
        }
        if (wbase >= v.nrow) break;
        const int lr0 = wbase + lane / LPR;
        if (lr0 < v.nrow) {
            const int lr = rev ? v.nrow - 1 - lr0 : lr0;
            if (!v.cached && lane == 0) {
                // the warp's rows kPrefetchWaves waves on, [w0, w1) in loop order, [ra, rb) local
                const int w0 = lr0 + kPrefetchWaves * (THREADS / LPR);
                if (w0 < v.nrow) {
                    const int w1 = min(w0 + 32 / LPR, v.nrow);
                    const int ra = rev ? v.nrow - w1 : w0, rb = rev ? v.nrow - w0 : w1;
                    prefetch_l2(a.bval + (size_t)(v.b_begin + v.rp[ra]) * 9, a.bval + (size_t)(v.b_begin + v.rp[rb]) * 9);
                    prefetch_l2(a.col_idx + v.b_begin + v.rp[ra], a.col_idx + v.b_begin + v.rp[rb]);
                }
            }
            T y0 = 0, y1 = 0, y2 = 0;
            const int be = v.rp[lr + 1];
            if (v.gathered) {
                for (int b = v.rp[lr] + sub; b < be; b += LPR)
                    block_times(v.val + (size_t)b * 9, v.gu[3 * b], v.gu[3 * b + 1], v.gu[3 * b + 2], y0, y1, y2);
            } else {
                // matrix rows cached, u not gathered: up to four of the lane's blocks at a time,
                // every load in flight before any tag is checked (a check is a branch on the value)
                constexpr int U = 4;
                for (int b0 = v.rp[lr] + sub; b0 < be; b0 += U * LPR) {
                    int cc[U];
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        const int b = b0 + k * LPR;
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
                            const int b = b0 + k * LPR;
                            const T *m = v.cached ? v.val + (size_t)b * 9 : a.bval + (size_t)(v.b_begin + b) * 9;
                            block_times(m, g[k].x, g[k].y, g[k].z, y0, y1, y2);
                        }
                }
            }
#pragma unroll
            for (int o = LPR / 2; o; o >>= 1) {
                y0 += __shfl_xor_sync(gmask, y0, o, LPR);
                y1 += __shfl_xor_sync(gmask, y1, o, LPR);
                y2 += __shfl_xor_sync(gmask, y2, o, LPR);
            }
            if (sub == 0) {
                const T w0 = y0 + mu * loc[lr * 3], w1 = y1 + mu * loc[lr * 3 + 1], w2 = y2 + mu * loc[lr * 3 + 2];
                v.w[lr * 3] = w0; v.w[lr * 3 + 1] = w1; v.w[lr * 3 + 2] = w2;
                wu.add_prod(w0, loc[lr * 3]);
                wu.add_prod(w1, loc[lr * 3 + 1]);
                wu.add_prod(w2, loc[lr * 3 + 2]);
            }
        }
    }
    return wu;
}

// THREADS: 512 when the matrix rows are cached in shared memory (the product and its
// exchanges are latency-bound and fewer warps meet sooner: cloth 2.02 -> 1.78 ms for 85
// iterations), 1024 when they stream from global memory (more loads in flight: noisy sphere
// 19.2 against 29.0 ms with 512).
template <typename T, bool kCheb, int THREADS>
__global__ void __launch_bounds__(THREADS) k_pcg_resident(PcgArgs<T> a, int smem_bytes) {
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
    v.cached = !a.no_cache && vec_bytes + mat_bytes <= (size_t)smem_bytes;
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
                if (kit == kChebWarm - 1 && it + 1 < a.max_it) {   // an iteration follows the restart
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
    unsigned n_calls = 0;   // products so far (their parity sets the order of the next)
    while (true) {
        const bool inner = kCheb && jstep > 0;
        const vec4_t<T> *src = (kCheb && (pub & 1u)) ? a.z4b : a.z4;
        const unsigned tu = kCheb ? (pub & 3u) : ((unsigned)it & 3u);
        const Acc<T> wu = resident_product<T, THREADS>(a, v, src, inner ? v.d : v.u, mu, tu, &s_bad, (n_calls++ & 1u) != 0);
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

// ---------------------------------------------------------------- PCG, streamed
// Systems whose matrix rows do not fit the solver blocks' shared memory (the matrix streams
// from HBM every product anyway): Chronopoulos and Gear's recurrence as two kernels per
// iteration, replayed from a CUDA graph.  k_cg_spmv forms w = (A + mu I) u with 8 lanes per
// row and the read-only path for u (u does not change during that kernel, so its gathers can
// hit L1 and the neighbouring rows' shared columns), sums delta = w.u, and its last block
// decides the step from gamma = r.u, delta and r.r (the same decisions as the block-resident
// kernel); k_cg_update updates p, s, x, r, u = M^-1 r and sums the next gamma and r.r.  All
// sums are block partials added in block order by the last block, so the result does not
// depend on timing.  A kernel of an iteration after the stop returns at once.
constexpr int kCgThreads = 256;

template <typename T>
__device__ __forceinline__ void cg_decide(DevScalars *ds, double gamma, double delta, double rr, double rtol2,
                                          int max_it) {
    const int it = ds->pcg_iters;
    if (it == 0) ds->red[1] = rr;
    const double rr0 = ds->red[1];
    bool stop = ds->cg_stop_next || it >= max_it || rr <= rtol2 * rr0 || !isfinite(rr);
    double alpha = 0.0, beta = 0.0;
    if (!stop) {
        bool ok;
        if (it == 0) {
            alpha = gamma / delta;
            ok = delta > 0.0 && isfinite(alpha);
        } else {
            beta = gamma / ds->cg_gamma_prev;
            const double den = delta - beta * gamma / ds->cg_alpha_prev;
            alpha = gamma / den;
            ok = den > 0.0 && isfinite(alpha);
        }
        if (!ok) {
            if (it > 0) stop = true;
            alpha = 1.0;   // breakdown at the first step keeps x = M^-1 r0 (preconditioned gradient)
            beta = 0.0;
            ds->cg_stop_next = 1;
        }
    }
    ds->cg_gamma_prev = gamma;
    ds->cg_alpha_prev = alpha;
    ds->cg_alpha = alpha;
    ds->cg_beta = beta;
    ds->red[0] = gamma;
    ds->red[4] = rr;
    if (stop) ds->pcg_done = 1;
}

template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_spmv(const int32_t *__restrict__ row_ptr,
                                                        const int32_t *__restrict__ col_idx,
                                                        const T *__restrict__ bval, const T *__restrict__ u,
                                                        T *__restrict__ w, double *partials, double rtol2, int max_it,
                                                        DevScalars *ds) {
    if (*(volatile int *)&ds->pcg_done) return;
    const unsigned long long nr = ds->n_rows;
    const T mu = (T)ds->mu;
    const int lane = threadIdx.x & 31, sub = lane & (kLanesPerRow - 1);
    const unsigned gmask = 0xffu << (lane & ~(kLanesPerRow - 1));
    const unsigned long long group = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) / kLanesPerRow;
    const unsigned long long n_groups = (unsigned long long)gridDim.x * blockDim.x / kLanesPerRow;
    Acc<T> wu;
    for (unsigned long long row = group; row < nr; row += n_groups) {
        T y0 = 0, y1 = 0, y2 = 0;
        const int be = row_ptr[row + 1];
        for (int b = row_ptr[row] + sub; b < be; b += kLanesPerRow) {
            if (TTIE_BAD(ds, b >= 0 && (unsigned long long)b < ds->nnzb, 51, b)) break;
            const int c = __ldg(col_idx + b);
            if (TTIE_BAD(ds, c >= 0 && (unsigned long long)c < nr, 52, c)) break;
            const T *m = bval + (size_t)b * 9;
            const T c0 = __ldg(u + 3 * (size_t)c), c1 = __ldg(u + 3 * (size_t)c + 1), c2 = __ldg(u + 3 * (size_t)c + 2);
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
        if (sub == 0) {
            const T u0 = u[row * 3], u1 = u[row * 3 + 1], u2 = u[row * 3 + 2];
            const T w0 = y0 + mu * u0, w1 = y1 + mu * u1, w2 = y2 + mu * u2;
            w[row * 3] = w0; w[row * 3 + 1] = w1; w[row * 3 + 2] = w2;
            wu.add_prod(w0, u0);
            wu.add_prod(w1, u1);
            wu.add_prod(w2, u2);
        }
    }
    double v[1] = {wu.value()};
    grid_sums<1>(v, partials, &ds->done_counter[3], [&](const double *t) {
        cg_decide<T>(ds, ds->red[0], t[0], ds->red[4], rtol2, max_it);
    });
}

template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_update(const T *__restrict__ dinv, T *__restrict__ x,
                                                          T *__restrict__ r, T *__restrict__ u, T *__restrict__ p,
                                                          T *__restrict__ s, const T *__restrict__ w,
                                                          double *partials, DevScalars *ds) {
    if (*(volatile int *)&ds->pcg_done) return;
    const unsigned long long nr = ds->n_rows;
    const T al = (T)ds->cg_alpha, be = (T)ds->cg_beta;
    Acc<T> g, q;
    for (unsigned long long row = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; row < nr;
         row += (unsigned long long)gridDim.x * blockDim.x) {
        T rv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t k = row * 3 + i;
            const T pi = u[k] + be * p[k];
            const T si = w[k] + be * s[k];
            p[k] = pi;
            s[k] = si;
            x[k] += al * pi;
            rv[i] = r[k] - al * si;
            r[k] = rv[i];
        }
        const T *di = dinv + row * 9;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T zi = di[3 * i] * rv[0] + di[3 * i + 1] * rv[1] + di[3 * i + 2] * rv[2];
            u[row * 3 + i] = zi;
            g.add_prod(rv[i], zi);
            q.add_prod(rv[i], rv[i]);
        }
    }
    double v[2] = {g.value(), q.value()};
    grid_sums<2>(v, partials, &ds->done_counter[4], [&](const double *t) {
        ds->red[0] = t[0];
        ds->red[4] = t[1];
        ds->pcg_iters += 1;
    });
}

}  // namespace

// The streamed PCG (kernels above): setup, then iterations of (k_cg_spmv, k_cg_update) from a
// graph of kCgGraphIters iterations captured once per call and replayed until max_it is
// covered; iterations after the stop return at once, so nothing is read back in between.
constexpr int kCgGraphIters = 10;

template <typename T>
cudaError_t pcg_streamed(Ctx &c, const T *rhs, T *out, double rtol, int max_it) {
    const int64_t nr = c.n_rows;
    TTIE_CUDA_TRY(ensure(c, c.pcg_w, (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T)));
    const int sms = c.num_sms > 0 ? c.num_sms : kNumSMs;
    const unsigned gs = grid_for(nr * kLanesPerRow, kCgThreads, (int64_t)sms * 8);
    const unsigned gu = grid_for(nr, kCgThreads, (int64_t)sms * 8);
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)kNumSMs * 16 * 4 * sizeof(double)));
    double *part = (double *)c.partials.p;
    // tickets of the two kernels' grid sums, the decision state and the iteration count
    TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->done_counter[3], 0, 2 * sizeof(unsigned int), c.stream));
    TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->cg_stop_next, 0, sizeof(int), c.stream));
    TTIE_CUDA_TRY(cudaMemsetAsync(c.pcg_q.p, 0, (size_t)(nr > 0 ? nr : 1) * 3 * sizeof(T), c.stream));   // s
    const unsigned g = grid_for(nr, kThreads, kNumSMs * 4);
    launch(c, k_pcg_setup<T>, dim3(g), dim3(kThreads), (const int32_t *)c.row_ptr.p, (const int32_t *)c.col_idx.p,
           (const T *)c.bsr_val.p, c.prm.mu_rel, (T *)c.dinv.p, rhs, out, (T *)c.pcg_r.p, (T *)c.pcg_z.p,
           (T *)c.pcg_p.p, part, (vec4_t<T> *)nullptr, (unsigned long long *)nullptr, 0, (int *)nullptr, 0, 0, 0,
           c.ds);
    TTIE_CUDA_TRY(cudaGetLastError());
    if (c.prm.profile) cudaEventRecord(c.ev[8], c.stream);
    const double rtol2 = rtol * rtol;
    const auto one_iteration = [&](cudaStream_t st) {
        ++c.n_launch;
        k_cg_spmv<T><<<gs, kCgThreads, 0, st>>>((const int32_t *)c.row_ptr.p, (const int32_t *)c.col_idx.p,
                                               (const T *)c.bsr_val.p, (const T *)c.pcg_z.p, (T *)c.pcg_w.p, part,
                                               rtol2, max_it, c.ds);
        ++c.n_launch;
        k_cg_update<T><<<gu, kCgThreads, 0, st>>>((const T *)c.dinv.p, out, (T *)c.pcg_r.p, (T *)c.pcg_z.p,
                                                 (T *)c.pcg_p.p, (T *)c.pcg_q.p, (const T *)c.pcg_w.p,
                                                 part + 2 * (size_t)kNumSMs * 16, c.ds);
    };
    // max_it + 1 products: the last decides the stop at max_it
    const int iters = max_it + 1;
#ifndef TTIE_CHECKS
    if (!c.cap_stream) TTIE_CUDA_TRY(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    TTIE_CUDA_TRY(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    const unsigned long long n0 = c.n_launch;
    for (int i = 0; i < kCgGraphIters; ++i) one_iteration(c.cap_stream);
    const unsigned long long per_graph = c.n_launch - n0;
    c.n_launch = n0;
    cudaError_t e = cudaGetLastError();
    const cudaError_t ec = cudaStreamEndCapture(c.cap_stream, &graph);
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (int done = 0; e == cudaSuccess && done < iters; done += kCgGraphIters) {
        e = cudaGraphLaunch(exec, c.stream);
        c.n_launch += per_graph;
    }
    if (exec) cudaGraphExecDestroy(exec);
    TTIE_CUDA_TRY(e);
#else
    for (int i = 0; i < iters; ++i) one_iteration(c.stream);
#endif
    if (c.prm.profile) cudaEventRecord(c.ev[9], c.stream);
    c.pcg_cheb = false;
    c.pcg_streamed = true;
    return cudaGetLastError();
}

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
    int64_t blocks = (nr * kLanesPerRow + 1023) / 1024;
    if (blocks > (int64_t)sms) blocks = sms;
    if (blocks > kMaxGridPcg) blocks = kMaxGridPcg;
    if (blocks < 1) blocks = 1;
    // rows resident in shared memory when every block's vectors fit (lean layout: 15 values
    // per row); blocks are balanced by nnz + kRowWeight * rows within that cap; else the
    // global-memory kernel
    // (the Chebyshev preconditioner keeps 6 more values per row, rounded up separately)
    // blk_bytes: a block's share of the matrix rows (with a quarter to spare for the
    // partition's imbalance) beside its vectors, which decides whether the rows are cached
    const int64_t blk_bytes = (int64_t)((double)c.nnzb * (9 * sizeof(T) + 4) * 1.25 / (double)blocks) +
                              (nr + blocks - 1) / blocks * (27 + 6) * (int64_t)sizeof(T);
    // AUTO: the polynomial preconditioner whenever the block-resident kernel can hold its two
    // more vectors per row (rows cached or streamed).  With block Jacobi the noisy sphere's
    // system stops at the cap of 200 iterations at a relative residual of 3.7e-3; Chebyshev
    // reaches 1e-3 in 68 (204 products) for 0.5 ms more, and its Newton step lowers the energy
    // by 46 % against 22 %.
    const int64_t r_cap_cheb = ((int64_t)kResidentSmem - 4 - 15 - 15) / (21 * (int64_t)sizeof(T) + 4);
    const bool cheb = c.prm.pcg_precond == TTIE_PCG_CHEBYSHEV ||
                      (c.prm.pcg_precond == TTIE_PCG_AUTO && (nr + blocks - 1) / blocks <= r_cap_cheb);
    const int64_t r_cap = cheb ? r_cap_cheb : ((int64_t)kResidentSmem - 4 - 15) / (15 * (int64_t)sizeof(T) + 4);
    const bool resident = (nr + blocks - 1) / blocks <= r_cap;
    // the streamed kernels for systems whose rows do not fit the block-resident kernel's lean
    // layout (in place of the global-memory persistent kernel), or when asked for: the noisy
    // sphere's FP32 system (386k rows) fits the lean layout, its FP64 system only the streamed
    // kernels
    const bool streamed = !(cheb && resident) && c.prm.test_withhold == 0 &&
                          (c.prm.pcg_kernel == TTIE_PCG_KERNEL_STREAMED ||
                           (c.prm.pcg_kernel == TTIE_PCG_KERNEL_AUTO && !resident));
    if (streamed) return pcg_streamed<T>(c, rhs, out, rtol, max_it);
    // 512 threads when the blocks' matrix rows are expected in shared memory, else 1024 with
    // the rows streamed from global memory; then the launch asks for just the shared memory of
    // the lean layout (the partition's rows capped at 1/8 above the mean) and leaves the rest
    // of the SM's 256 KB of L1 and shared memory to L1, which holds the streamed rows' loads
    // (L1 28 -> about 60 KB on the noisy sphere: 18.8 -> 18.5 ms for 200 iterations)
    const bool no_cache = c.prm.pcg_kernel == TTIE_PCG_KERNEL_RESIDENT_UNCACHED;
    const bool narrow = blk_bytes <= (int64_t)kResidentSmem && !no_cache;
    int64_t r_cap_run = r_cap, smem_run = kResidentSmem;
    if (resident && !narrow) {
        const int64_t per_row = (cheb ? 21 : 15) * (int64_t)sizeof(T) + 4;
        r_cap_run = std::min<int64_t>(r_cap, (nr + blocks - 1) / blocks * 9 / 8 + 32);
        smem_run = std::min<int64_t>(kResidentSmem, (r_cap_run * per_row + 64 + 1023) / 1024 * 1024);
    }
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
                                                 resident ? rpart : nullptr, (int)blocks, (int)r_cap_run, kRowWeight, c.ds);
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
    c.pcg_streamed = false;
    args.partA = part;
    args.partB = part + 2 * kNumSMs * 8;
    args.rtol2 = rtol * rtol;
    args.max_it = max_it;
    args.ds = c.ds;
    args.slots = slots;
    args.part = rpart;
    args.withhold = c.prm.test_withhold;
    args.no_cache = no_cache ? 1 : 0;
    ++c.n_launch;
    if (c.prm.profile) cudaEventRecord(c.ev[8], c.stream);
    if (resident) {
        const void *kern = cheb ? (narrow ? (const void *)k_pcg_resident<T, true, 512> : (const void *)k_pcg_resident<T, true, 1024>)
                                : (narrow ? (const void *)k_pcg_resident<T, false, 512> : (const void *)k_pcg_resident<T, false, 1024>);
        TTIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kResidentSmem));
        // the carve-out: the launch's shared memory with the static part, the rest L1
        const int carve = (int)std::min<int64_t>(100, (smem_run + 8192) * 100 / (228 * 1024) + 1);
        TTIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
        int smem = (int)smem_run;
        void *kargs[] = {&args, &smem};
        TTIE_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3((unsigned)blocks), dim3(narrow ? 512 : 1024), kargs,
                                                  (size_t)smem_run, c.stream));
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
    args.z4b = nullptr;
    args.cheb_degree = 0;
    args.slots = nullptr;
    args.part = nullptr;
    args.withhold = 0;
    args.no_cache = 0;
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

}  // namespace ttie
