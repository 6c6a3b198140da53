// Narrow phase and energy (§1, Eq. 1-3, Appendix A).
//
// 1. k_classify: one thread per candidate pair.  The pair intersects iff each
//    triangle has vertices strictly on both sides of the other's plane and the
//    open intervals I_a, I_b on the intersection line overlap (0 inside I_c).
//    Every sign of that test is certified: an FP32 determinant with a forward
//    error bound, then FP64 with its bound; signs neither can certify send the
//    pair to k_resolve (exact expansions).  The interval comparison is recast
//    as orientation signs: with p1 the vertex of A alone on its side of plane B
//    and q1 the vertex of B alone on its side of plane A, the endpoint on edge
//    (p1, p_u) and the endpoint on edge (q1, q_v) compare as
//        sign(t_v - t_u) = -s_p s_q sign det[p_u - p1, q_v - q1, q1 - p1]
//    (s_p, s_q the sides of p1 and q1), and the intervals overlap openly iff
//    these four signs include both a positive and a negative one.
// 2. k_compact: intersecting pairs in candidate order.
// 3. k_derivs: t_c^0, t_c^1 (Eq. 1), T (Eq. 2) and the analytic gradients of
//    t_c^0 and t_c^1 for each intersecting pair (manual chain rule through the
//    Möller construction, as §1.2 describes), plus the FP64 energy sum.
#include "common.cuh"
#include "exact.cuh"

namespace ttie {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------- certified signs
// Every sign below is +1, -1, 0 (certified zero) or kUndec (not certified).
constexpr int kUndec = 2;

// Sign of det[e1, e2, f] = (e1 x e2) . f, given n = e1 x e2 and N = |e1| x |e2|
// (componentwise absolute cross product).  The rounding error of the computed value
// is below ~8u times the permanent N.|f| (u: unit roundoff), so a sign is trusted
// only beyond 1e-6 (FP32, ~17u) or 2e-15 (FP64, ~18u) times the permanent.
__device__ __forceinline__ int filt_f32(v3<float> n, v3<float> N, v3<float> f) {
    float d = dot(n, f);
    float perm = dot(N, vabs(f));
    if (!(perm > 1e-30f) || !(perm < 1e30f)) return kUndec;
    float bound = 1e-6f * perm;
    return d > bound ? 1 : (d < -bound ? -1 : kUndec);
}
__device__ __forceinline__ int filt_f64(v3<double> n, v3<double> N, v3<double> f) {
    double d = dot(n, f);
    double perm = dot(N, vabs(f));
    if (!(perm > 1e-280) || !(perm < 1e280)) return kUndec;
    double bound = 2e-15 * perm;
    return d > bound ? 1 : (d < -bound ? -1 : kUndec);
}
__device__ __forceinline__ v3<double> to_d(v3<float> a) { return {(double)a.x, (double)a.y, (double)a.z}; }
__device__ __forceinline__ v3<double> to_d(v3<double> a) { return a; }

// det[e1, e2, f] is exactly zero when each of its six terms e1_i e2_j f_k has a factor
// that is exactly zero (a difference of floating-point numbers is exactly zero only
// when they are equal).  Aligned meshes (a grid keeping one coordinate exact) produce
// such determinants at every crossing of two sheets.
__device__ __forceinline__ bool structural_zero(v3<double> a, v3<double> b, v3<double> f) {
    const bool ax = a.x == 0.0, ay = a.y == 0.0, az = a.z == 0.0;
    const bool bx = b.x == 0.0, by = b.y == 0.0, bz = b.z == 0.0;
    const bool fx = f.x == 0.0, fy = f.y == 0.0, fz = f.z == 0.0;
    return (ax || by || fz) && (ax || bz || fy) && (ay || bx || fz) && (ay || bz || fx) && (az || bx || fy) &&
           (az || by || fx);
}

// a * b == c * d exactly: the rounded products and their errors (fma) both equal.  Only
// where the errors are exact (no product near underflow) and a zero product has a zero factor.
__device__ __forceinline__ bool prod_eq(double a, double b, double c, double d) {
    const double p = a * b, q = c * d;
    if (p != q) return false;
    if (p == 0.0) return (a == 0.0 || b == 0.0) && (c == 0.0 || d == 0.0);
    if (!(fabs(p) > 0x1p-960) || !(fabs(p) < 0x1p+1000)) return false;
    return fma(a, b, -p) == fma(c, d, -q);
}

// det[e1, e2, f] (entries exact) is exactly zero when, expanded along one of its rows w with
// the other two rows u, v in cyclic order, every term w_i (u x v)_i vanishes: w_i = 0, or the
// minor u_j v_k - u_k v_j has two exactly equal products.  Meshes with mirror symmetry
// (a vertex quadruple symmetric about a coordinate plane: an isosceles trapezoid, coplanar)
// give such determinants, which neither filter can certify.
__device__ __forceinline__ bool terms_vanish(v3<double> u, v3<double> v, v3<double> w) {
    return (w.x == 0.0 || prod_eq(u.y, v.z, u.z, v.y)) && (w.y == 0.0 || prod_eq(u.z, v.x, u.x, v.z)) &&
           (w.z == 0.0 || prod_eq(u.x, v.y, u.y, v.x));
}
__device__ __forceinline__ bool minor_zero(v3<double> e1, v3<double> e2, v3<double> f) {
    return terms_vanish(e1, e2, f) || terms_vanish(e2, f, e1) || terms_vanish(f, e1, e2);
}

// b - a, and whether it is exact (Knuth's two-sum error of b + (-a) is zero).
__device__ __forceinline__ double sub_exact(double b, double a, bool &exact) {
    const double s = b - a, bp = s + a, ap = s - bp;
    exact &= ((b - bp) + (-a - ap)) == 0.0;
    return s;
}
__device__ __forceinline__ v3<double> sub_exact(v3<double> b, v3<double> a, bool &exact) {
    return {sub_exact(b.x, a.x, exact), sub_exact(b.y, a.y, exact), sub_exact(b.z, a.z, exact)};
}

// FP64 stage: filter, then the structural-zero certificate, then (differences exact) the
// exact sign in 128-bit integers where the entries fit, else the vanishing-terms certificate.
// Only what none of these settles goes to the expansion arithmetic.
__device__ __noinline__ int det_sign_f64(v3<double> e1, v3<double> e2, v3<double> f, bool exact) {
    const int s = filt_f64(cross(e1, e2), abs_cross(e1, e2), f);
    if (s != kUndec) return s;
    if (structural_zero(e1, e2, f)) return 0;
    if (!exact) return kUndec;
    const double a[3] = {e1.x, e1.y, e1.z}, b[3] = {e2.x, e2.y, e2.z}, c[3] = {f.x, f.y, f.z};
    int si;
    if (exact::det3_int_sign(a, b, c, si)) return si;
    return minor_zero(e1, e2, f) ? 0 : kUndec;
}

__device__ __forceinline__ int orient_exact(v3<double> a, v3<double> b, v3<double> c, v3<double> d) {
    double A[3] = {a.x, a.y, a.z}, B[3] = {b.x, b.y, b.z}, C[3] = {c.x, c.y, c.z}, D[3] = {d.x, d.y, d.z};
    return exact::orient3d_exact(A, B, C, D);
}

struct Stats {
    unsigned long long f32 = 0, f64 = 0, ex = 0;
};

// Sign providers.  side(P0, P1, P2, q) = sign det[P1-P0, P2-P0, q-P0] (side of q w.r.t. the
// plane of P); over(p1, pu, q1, qv) = sign det[pu-p1, qv-q1, q1-p1].  kF32Only (FP32
// positions): a sign the FP32 filter cannot certify is left undecided instead of going to the
// FP64 filter, so the classification of all candidates never issues FP64 instructions: on
// GB300 the FP64 pipe runs at a small fraction of the FP32 rate and a warp pays for the
// FP64 path whenever one of its lanes takes it.  Those pairs go to the resolve pass.
template <typename T, bool kF32Only = false> struct Filtered {
    bool exact_only;
    Stats &st;
    __device__ __forceinline__ int side(v3<T> P0, v3<T> P1, v3<T> P2, v3<T> q) {
        if (exact_only) return kUndec;
        int s = kUndec;
        if (sizeof(T) == 4) {
            const v3<T> e1 = P1 - P0, e2 = P2 - P0, f = q - P0;
            s = filt_f32(to_f(cross(e1, e2)), to_f(abs_cross(e1, e2)), to_f(f));
            if (s != kUndec) { ++st.f32; return s; }
            if (kF32Only) return kUndec;
            if (int_sign(P0, P1, P2, q, s)) { ++st.f64; return s; }
        }
        const v3<double> a = to_d(P0);
        bool exact = true;
        const v3<double> e1 = sub_exact(to_d(P1), a, exact), e2 = sub_exact(to_d(P2), a, exact),
                         f = sub_exact(to_d(q), a, exact);
        s = det_sign_f64(e1, e2, f, exact);
        if (s != kUndec) ++st.f64;
        return s;
    }
    __device__ __forceinline__ int over(v3<T> p1, v3<T> pu, v3<T> q1, v3<T> qv) {
        if (exact_only) return kUndec;
        int s = kUndec;
        if (sizeof(T) == 4) {
            const v3<T> e1 = pu - p1, e2 = qv - q1;
            s = filt_f32(to_f(cross(e1, e2)), to_f(abs_cross(e1, e2)), to_f(q1 - p1));
            if (s != kUndec) { ++st.f32; return s; }
            if (kF32Only) return kUndec;
            if (int_sign(p1, pu, qv, q1, s)) { ++st.f64; return s; }   // det[pu - p1, qv - p1, q1 - p1]
        }
        bool exact = true;
        const v3<double> e1 = sub_exact(to_d(pu), to_d(p1), exact), e2 = sub_exact(to_d(qv), to_d(q1), exact),
                         f = sub_exact(to_d(q1), to_d(p1), exact);
        s = det_sign_f64(e1, e2, f, exact);
        if (s != kUndec) ++st.f64;
        return s;
    }
    __device__ __forceinline__ static v3<float> to_f(v3<T> a) { return {(float)a.x, (float)a.y, (float)a.z}; }
    // float32 points: the exact sign in integers, cheaper than the FP64 filter on a part whose
    // FP64 rate is a small fraction of its integer rate (false where the span does not fit)
    __device__ __forceinline__ static bool int_sign(v3<T> a, v3<T> b, v3<T> c, v3<T> d, int &s) {
        const float A[3] = {(float)a.x, (float)a.y, (float)a.z}, B[3] = {(float)b.x, (float)b.y, (float)b.z},
                    C[3] = {(float)c.x, (float)c.y, (float)c.z}, D[3] = {(float)d.x, (float)d.y, (float)d.z};
        return exact::orient3d_f32_int(A, B, C, D, s);
    }
};

// The undecided pairs' signs: each one through the FP32 and FP64 filters again (certified,
// so the same decisions), and only the signs neither certifies through exact expansions.
// Counts the signs decided by FP64 and by exact arithmetic (the FP32 ones were counted by the
// first pass).  With exact_only every sign is exact.
// Exact signs for what the filters leave: float32 points in 256-bit integers where their span
// allows, else (and for FP64 points) expansion arithmetic.  exact_mode 1: no filters; 2: no
// filters and expansions only (test switches).
template <typename T> struct Cascade {
    int exact_mode;
    Stats &st;
    __device__ int exact_sign(v3<T> a, v3<T> b, v3<T> c, v3<T> d) {
        ++st.ex;
        if constexpr (sizeof(T) == 4) {
            if (exact_mode != 2) {
                const float A[3] = {(float)a.x, (float)a.y, (float)a.z}, B[3] = {(float)b.x, (float)b.y, (float)b.z},
                            C[3] = {(float)c.x, (float)c.y, (float)c.z}, D[3] = {(float)d.x, (float)d.y, (float)d.z};
                int s;
                if (exact::orient3d_f32_int(A, B, C, D, s)) return s;
            }
        }
        return orient_exact(to_d(a), to_d(b), to_d(c), to_d(d));
    }
    __device__ int side(v3<T> P0, v3<T> P1, v3<T> P2, v3<T> q) {
        if (!exact_mode) {
            Stats inner;
            Filtered<T> f{false, inner};
            const int s = f.side(P0, P1, P2, q);
            st.f64 += inner.f64;
            if (s != kUndec) return s;
        }
        return exact_sign(P0, P1, P2, q);
    }
    // det[pu - p1, qv - q1, q1 - p1] = det[pu - p1, qv - p1, q1 - p1]
    __device__ int over(v3<T> p1, v3<T> pu, v3<T> q1, v3<T> qv) {
        if (!exact_mode) {
            Stats inner;
            Filtered<T> f{false, inner};
            const int s = f.over(p1, pu, q1, qv);
            st.f64 += inner.f64;
            if (s != kUndec) return s;
        }
        return exact_sign(p1, pu, qv, q1);
    }
};

template <typename T>
__device__ __forceinline__ void load_pair(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4, int2 pr,
                                          v3<T> A[3], v3<T> B[3]) {
    int4 ta = tri4[pr.x], tb = tri4[pr.y];
    A[0] = xyz<T>(x[ta.x]); A[1] = xyz<T>(x[ta.y]); A[2] = xyz<T>(x[ta.z]);
    B[0] = xyz<T>(x[tb.x]); B[1] = xyz<T>(x[tb.y]); B[2] = xyz<T>(x[tb.z]);
}

// First vertex whose side is non-zero and shared by no other vertex.
__device__ __forceinline__ int lone_of(const int s[3]) {
    for (int i = 0; i < 3; ++i) {
        const int same = (s[i] == s[0]) + (s[i] == s[1]) + (s[i] == s[2]);
        if (s[i] != 0 && same == 1) return i;
    }
    return 0;
}

// 1: intersecting, 0: not, -1: undecided (some deciding sign not certified).
template <typename T, typename Signs>
__device__ __forceinline__ int classify(const v3<T> A[3], const v3<T> B[3], Signs &sg) {
    int sB[3], sA[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sB[k] = sg.side(A[0], A[1], A[2], B[k]);
    int pos = (sB[0] == 1) + (sB[1] == 1) + (sB[2] == 1);
    int neg = (sB[0] == -1) + (sB[1] == -1) + (sB[2] == -1);
    const int undB = (sB[0] == kUndec) + (sB[1] == kUndec) + (sB[2] == kUndec);
    if (!(pos + undB >= 1 && neg + undB >= 1)) return 0;   // B cannot straddle plane A
#pragma unroll
    for (int k = 0; k < 3; ++k) sA[k] = sg.side(B[0], B[1], B[2], A[k]);
    pos = (sA[0] == 1) + (sA[1] == 1) + (sA[2] == 1);
    neg = (sA[0] == -1) + (sA[1] == -1) + (sA[2] == -1);
    const int undA = (sA[0] == kUndec) + (sA[1] == kUndec) + (sA[2] == kUndec);
    if (!(pos + undA >= 1 && neg + undA >= 1)) return 0;
    if (undA || undB) return -1;
    // both straddle: compare the interval endpoints through orientation signs
    const int ip = lone_of(sA), iq = lone_of(sB);
    const int f = -sA[ip] * sB[iq];
    const v3<T> p1 = A[ip], pu = A[(ip + 1) % 3], pw = A[(ip + 2) % 3];
    const v3<T> q1 = B[iq], qv = B[(iq + 1) % 3], qw = B[(iq + 2) % 3];
    int s[4];
    s[0] = sg.over(p1, pu, q1, qv);
    s[1] = sg.over(p1, pu, q1, qw);
    s[2] = sg.over(p1, pw, q1, qv);
    s[3] = sg.over(p1, pw, q1, qw);
    bool any_pos = false, any_neg = false, und = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (s[k] == kUndec) { und = true; continue; }
        any_pos |= f * s[k] > 0;
        any_neg |= f * s[k] < 0;
    }
    if (any_pos && any_neg) return 1;
    return und ? -1 : 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_classify(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4,
                                                       const int2 *__restrict__ pairs, int64_t n,
                                                       const unsigned long long *__restrict__ d_n, int exact_only,
                                                       uint32_t *__restrict__ bits, uint32_t *__restrict__ defer,
                                                       DevScalars *ds) {
    const int lane = threadIdx.x & 31;
    const int64_t n_words = (n + 31) / 32;   // words of the list's capacity n; pairs at or past *d_n count as 0
    if (d_n) n = (int64_t)min((unsigned long long)n, *d_n);
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Stats st;
    Filtered<T, true> sg{exact_only != 0, st};
    for (int64_t w = warp0; w < n_words; w += n_warps) {
        const int64_t p = w * 32 + lane;
        int r = 0;
        if (p < n) {
            v3<T> A[3], B[3];
            load_pair<T>(x, tri4, pairs[p], A, B);
            r = classify<T>(A, B, sg);
        }
        const unsigned act = __ballot_sync(0xffffffffu, r == 1);
        const unsigned und = __ballot_sync(0xffffffffu, r == -1);
        if (lane == 0) bits[w] = act;
        if (und) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ds->n_defer, (unsigned long long)__popc(und));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (r == -1) defer[base + __popc(und & ((1u << lane) - 1u))] = (uint32_t)p;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        st.f32 += __shfl_xor_sync(0xffffffffu, st.f32, o);
        st.f64 += __shfl_xor_sync(0xffffffffu, st.f64, o);
    }
    if (lane == 0 && (st.f32 | st.f64)) {
        atomicAdd(&ds->filter_stats[0], st.f32);
        atomicAdd(&ds->filter_stats[1], st.f64);
    }
}

// Pairs the FP32 pass left undecided, compacted: the test again with the FP32 then FP64
// filters.  Pairs still undecided go to defer2 for the exact pass, which keeps the
// registers of the exact expansions (and their low occupancy) off the many pairs that FP64
// decides.
template <typename T>
__global__ void __launch_bounds__(128, 4) k_resolve_f64(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4,
                              const int2 *__restrict__ pairs, const uint32_t *__restrict__ defer, int exact_only,
                              uint32_t *__restrict__ bits, uint32_t *__restrict__ defer2, DevScalars *ds) {
    const unsigned long long m = ds->n_defer;
    Stats st;
    Filtered<T> sg{exact_only != 0, st};
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < m;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = defer[k];
        v3<T> A[3], B[3];
        load_pair<T>(x, tri4, pairs[p], A, B);
        const int r = classify<T>(A, B, sg);
        if (r == 1) atomicOr(&bits[p >> 5], 1u << (p & 31));
        else if (r == -1) defer2[atomicAdd(&ds->n_defer2, 1ull)] = p;
    }
    if (st.f64) atomicAdd(&ds->filter_stats[1], st.f64);
}

// Decision of the pairs neither filter decided: the same test, every sign the filters
// cannot certify from exact expansion arithmetic (a vertex exactly on a plane counts as
// zero, touching intervals do not overlap).
template <typename T>
__global__ void k_resolve(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4, const int2 *__restrict__ pairs,
                          const uint32_t *__restrict__ defer2, int exact_only, uint32_t *__restrict__ bits,
                          DevScalars *ds) {
    const unsigned long long m = ds->n_defer2;
    Stats st;
    Cascade<T> sg{exact_only, st};
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < m;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t p = defer2[k];
        v3<T> A[3], B[3];
        load_pair<T>(x, tri4, pairs[p], A, B);
        if (classify<T>(A, B, sg) == 1) atomicOr(&bits[p >> 5], 1u << (p & 31));
    }
    if (st.ex) atomicAdd(&ds->filter_stats[2], st.ex);   // its FP64 signs were counted by k_resolve_f64
}

__global__ void k_popc(const uint32_t *__restrict__ bits, int64_t n_words, uint32_t *__restrict__ cnt) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_words; w += (int64_t)gridDim.x * blockDim.x)
        cnt[w] = __popc(bits[w]);
}

__global__ void k_compact(const uint32_t *__restrict__ bits, int64_t n_words, const unsigned long long *__restrict__ off,
                          uint32_t *__restrict__ active, DevScalars *ds) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = bits[w];
        unsigned long long o = off[w];
        while (b) {
            int i = __ffs(b) - 1;
            active[o++] = (uint32_t)(w * 32 + i);
            b &= b - 1;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->n_active = off[n_words];
}

// ---------------------------------------------------------------- reductions
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
    return r;   // valid in thread 0
}

// Deterministic grid sum: block partials, then the last block to finish adds them in order.
__device__ __forceinline__ void grid_sum(double v, double *partials, unsigned int *ticket, double *out) {
    __shared__ bool last;
    double b = block_sum(v);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        double s = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) s += __ldcg(&partials[i]);
        s = block_sum(s);
        if (threadIdx.x == 0) {
            *out = s;
            *ticket = 0u;
        }
    }
}

// ---------------------------------------------------------------- derivatives
template <typename T> struct Cut {
    // Segment endpoint on edge (m, p) of the cut triangle: S = (1 - lam) q_m + lam q_p
    int m0, p0, m1, p1;
    T lam0, lam1;
    v3<T> S0, S1;
};

// The discrete choices of one pair's construction: the lone vertex of the cut of B by
// plane A (mB) and of A by plane B (mA), and which end of each segment has the smaller line
// parameter.  The FP32 evaluation takes them from an FP64 evaluation of the same pair, so
// the values and the gradients follow the same branch.
struct Branch {
    int mB, mA;
    bool a0min, b0min;
};

// Plane-side values and the cut of triangle Q by the plane of P (values only; the
// sides were certified during classification, here they only pick the edges).
// m_in >= 0: the lone vertex is given; the chosen one is returned in m_out.
template <typename T>
__device__ __forceinline__ Cut<T> cut_by(const v3<T> P[3], const v3<T> Q[3], v3<T> nP, int m_in, int &m_out) {
    T d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = dot(nP, Q[k] - P[0]);
    const int s0 = d[0] >= T(0), s1 = d[1] >= T(0), s2 = d[2] >= T(0);
    int m;
    const int pos = s0 + s1 + s2;
    if (m_in >= 0) m = m_in;
    else if (pos == 1) m = s0 ? 0 : (s1 ? 1 : 2);
    else if (pos == 2) m = !s0 ? 0 : (!s1 ? 1 : 2);
    else {   // not straddling in this precision (near-degenerate): farthest vertex
        T a0 = fabs(d[0]), a1 = fabs(d[1]), a2 = fabs(d[2]);
        m = (a0 >= a1 && a0 >= a2) ? 0 : (a1 >= a2 ? 1 : 2);
    }
    m_out = m;
    Cut<T> c;
    const int u = (m + 1) % 3, v = (m + 2) % 3;   // the other two, in increasing order
    c.m0 = m; c.p0 = u < v ? u : v;
    c.m1 = m; c.p1 = u < v ? v : u;
    T den0 = d[m] - d[c.p0], den1 = d[m] - d[c.p1];
    c.lam0 = den0 != T(0) ? d[m] / den0 : T(0.5);
    c.lam1 = den1 != T(0) ? d[m] / den1 : T(0.5);
    c.S0 = Q[m] + c.lam0 * (Q[c.p0] - Q[m]);
    c.S1 = Q[m] + c.lam1 * (Q[c.p1] - Q[m]);
    return c;
}

// g[off_Q + 3v + k] += coefficients of d(D.S)/d(vertex) for the endpoint S on edge (m, p) of
// Q cut by the plane (P, nP), scaled by w:
//   q_m: (1 - lam) Pd, q_p: lam Pd with Pd = D + rho nP, rho = -(D.e)/(nP.e), e = q_p - q_m
//   P_k: rho (S - P_0) x (P_{k+2} - P_{k+1}), and P_0 additionally -rho nP
template <typename T>
__device__ __forceinline__ void add_endpoint(T *g, int offQ, int offP, const v3<T> P[3], const v3<T> Q[3], v3<T> nP,
                                             v3<T> D, int m, int p, T lam, v3<T> S, T w) {
    const v3<T> e = Q[p] - Q[m];
    const T ne = dot(nP, e);
    const T rho = ne != T(0) ? -dot(D, e) / ne : T(0);
    const v3<T> Pd = D + rho * nP;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const T cv = w * ((v == m ? T(1) - lam : T(0)) + (v == p ? lam : T(0)));
        g[offQ + 3 * v + 0] += cv * Pd.x;
        g[offQ + 3 * v + 1] += cv * Pd.y;
        g[offQ + 3 * v + 2] += cv * Pd.z;
    }
    const v3<T> c = S - P[0];
    const T wr = w * rho;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v3<T> t = cross(c, P[(k + 2) % 3] - P[(k + 1) % 3]);
        if (k == 0) t = t - nP;
        g[offP + 3 * k + 0] += wr * t.x;
        g[offP + 3 * k + 1] += wr * t.y;
        g[offP + 3 * k + 2] += wr * t.z;
    }
}

// g += w * d(D.Delta)/dx through D = (nB x nA)/|nB x nA| with Delta fixed:
//   c = (Delta - (D.Delta) D)/|w|;  b_k: (nA x c) x (b_{k+2} - b_{k+1});  a_k: (c x nB) x (a_{k+2} - a_{k+1})
template <typename T>
__device__ __forceinline__ void add_direction(T *g, const v3<T> A[3], const v3<T> B[3], v3<T> nA, v3<T> nB, v3<T> D,
                                              T inv_w, v3<T> Delta, T w) {
    const v3<T> c = (w * inv_w) * (Delta - dot(D, Delta) * D);
    const v3<T> cb = cross(nA, c), ca = cross(c, nB);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const v3<T> tb = cross(cb, B[(k + 2) % 3] - B[(k + 1) % 3]);
        const v3<T> ta = cross(ca, A[(k + 2) % 3] - A[(k + 1) % 3]);
        g[9 + 3 * k + 0] += tb.x; g[9 + 3 * k + 1] += tb.y; g[9 + 3 * k + 2] += tb.z;
        g[3 * k + 0] += ta.x; g[3 * k + 1] += ta.y; g[3 * k + 2] += ta.z;
    }
}

// Dual number (value, tangent) for forward-mode differentiation; comparisons use values.
template <typename T> struct Dual {
    T v, t;
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(T a) : v(a), t(T(0)) {}
    __device__ __forceinline__ Dual(T a, T b) : v(a), t(b) {}
};
template <typename T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.t + b.t}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.t - b.t}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.t}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) {
    return {a.v * b.v, a.t * b.v + a.v * b.t};
}
template <typename T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
    const T q = a.v / b.v;
    return {q, (a.t - q * b.t) / b.v};
}
template <typename T> __device__ __forceinline__ Dual<T> &operator+=(Dual<T> &a, Dual<T> b) { return a = a + b; }
template <typename T> __device__ __forceinline__ Dual<T> &operator-=(Dual<T> &a, Dual<T> b) { return a = a - b; }
template <typename T> __device__ __forceinline__ bool operator<(Dual<T> a, Dual<T> b) { return a.v < b.v; }
template <typename T> __device__ __forceinline__ bool operator>(Dual<T> a, Dual<T> b) { return a.v > b.v; }
template <typename T> __device__ __forceinline__ bool operator>=(Dual<T> a, Dual<T> b) { return a.v >= b.v; }
template <typename T> __device__ __forceinline__ bool operator!=(Dual<T> a, Dual<T> b) { return a.v != b.v; }
template <typename T> __device__ __forceinline__ Dual<T> sqrt(Dual<T> a) {
    const T r = sqrt(a.v);
    return {r, r > T(0) ? a.t / (T(2) * r) : T(0)};
}
template <typename T> __device__ __forceinline__ Dual<T> fabs(Dual<T> a) { return a.v < T(0) ? -a : a; }
using ::sqrt;   // keep the float / double overloads visible next to the dual ones
using ::fabs;

// Output row per intersecting pair: [t_c^0, t_c^1, d t_c^0 (18), d t_c^1 (18), pad 2].

// t_c^0, t_c^1 of one intersecting pair and, with kGrad, their gradients (18 each) by the
// chain rule through the construction above.  S is float, double or a dual number (the
// exact Hessian-vector product differentiates this function once more in forward mode).
// br: the branch taken (out), or with given = true the branch to take (in).
template <typename S, bool kGrad>
__device__ __forceinline__ void pair_tc(v3<S> A[3], v3<S> B[3], S tc_scale, S &a, S &b, S *ga, S *gb, Branch &br,
                                        bool given = false) {
    // local frame at A0: T and its gradient are translation invariant, and small
    // coordinates keep the cancellations in t_c at the size of the triangles
    const v3<S> o = A[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) { A[i] = A[i] - o; B[i] = B[i] - o; }
    const v3<S> nA = cross(A[1] - A[0], A[2] - A[0]);
    const v3<S> nB = cross(B[1] - B[0], B[2] - B[0]);
    const Cut<S> cB = cut_by<S>(A, B, nA, given ? br.mB : -1, br.mB);   // segment on B (plane of A)
    const Cut<S> cA = cut_by<S>(B, A, nB, given ? br.mA : -1, br.mA);   // segment on A (plane of B)
    const v3<S> wv = cross(nB, nA);
    const S wn = sqrt(dot(wv, wv));
    const S inv_w = wn > S(0) ? S(1) / wn : S(0);
    const v3<S> D = inv_w * wv;
    const S tA0 = dot(D, cA.S0), tA1 = dot(D, cA.S1), tB0 = dot(D, cB.S0), tB1 = dot(D, cB.S1);
    if (!given) {
        br.a0min = !(tA1 < tA0);
        br.b0min = !(tB1 < tB0);
    }
    const bool a0min = br.a0min, b0min = br.b0min;
    a = tc_scale * ((a0min ? tA0 : tA1) - (b0min ? tB1 : tB0));
    b = tc_scale * ((a0min ? tA1 : tA0) - (b0min ? tB0 : tB1));
    if (kGrad) {
#pragma unroll
        for (int i = 0; i < 18; ++i) { ga[i] = S(0); gb[i] = S(0); }
        // t_c^0 = s (t_A,min - t_B,max), t_c^1 = s (t_A,max - t_B,min)
        const int amin_m = a0min ? cA.m0 : cA.m1, amin_p = a0min ? cA.p0 : cA.p1;
        const int amax_m = a0min ? cA.m1 : cA.m0, amax_p = a0min ? cA.p1 : cA.p0;
        const S amin_l = a0min ? cA.lam0 : cA.lam1, amax_l = a0min ? cA.lam1 : cA.lam0;
        const v3<S> amin_S = a0min ? cA.S0 : cA.S1, amax_S = a0min ? cA.S1 : cA.S0;
        const int bmin_m = b0min ? cB.m0 : cB.m1, bmin_p = b0min ? cB.p0 : cB.p1;
        const int bmax_m = b0min ? cB.m1 : cB.m0, bmax_p = b0min ? cB.p1 : cB.p0;
        const S bmin_l = b0min ? cB.lam0 : cB.lam1, bmax_l = b0min ? cB.lam1 : cB.lam0;
        const v3<S> bmin_S = b0min ? cB.S0 : cB.S1, bmax_S = b0min ? cB.S1 : cB.S0;
        add_endpoint<S>(ga, 0, 9, B, A, nB, D, amin_m, amin_p, amin_l, amin_S, tc_scale);
        add_endpoint<S>(ga, 9, 0, A, B, nA, D, bmax_m, bmax_p, bmax_l, bmax_S, -tc_scale);
        add_direction<S>(ga, A, B, nA, nB, D, inv_w, amin_S - bmax_S, tc_scale);
        add_endpoint<S>(gb, 0, 9, B, A, nB, D, amax_m, amax_p, amax_l, amax_S, tc_scale);
        add_endpoint<S>(gb, 9, 0, A, B, nA, D, bmin_m, bmin_p, bmin_l, bmin_S, -tc_scale);
        add_direction<S>(gb, A, B, nA, nB, D, inv_w, amax_S - bmin_S, tc_scale);
    }
}

// t_c^0 and t_c^1 are differences of positions of the pair's size L, so an FP32 evaluation
// carries an absolute error of a few u32 L in them: relative 1e-3 and more on pairs whose
// |t_c| is 1e-6 of the scene.  Their gradients carry errors that grow with the inverse sines
// of the angles between the planes and between the cut edges and the cutting planes, and with
// the cancellation between the two terms of Eq. 3: up to 1.4e-4 relative on the crossing
// cloth, and no cheap estimate of those factors kept every FP32 gradient within 1e-4 (one
// missed 1.1e-4 after a few Newton steps).  So for FP32 positions the derivatives of the
// intersecting pairs are evaluated in FP64 from the exactly converted FP32 inputs and
// rounded to FP32; the classification of all candidates (k_classify) stays in FP32.  This runs
// on the intersecting pairs only (about 9 % of the candidates).
template <typename T, bool kGrad>
__device__ __forceinline__ void pair_values(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4, int2 pr,
                                            T tc_scale, double &a, double &b, T *ga, T *gb) {
    v3<T> A[3], B[3];
    load_pair<T>(x, tri4, pr, A, B);
    v3<double> Ad[3], Bd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) { Ad[i] = to_d(A[i]); Bd[i] = to_d(B[i]); }
    double gad[18], gbd[18];
    Branch br;
    pair_tc<double, kGrad>(Ad, Bd, (double)tc_scale, a, b, gad, gbd, br);
    if (kGrad) {
#pragma unroll
        for (int i = 0; i < 18; ++i) { ga[i] = (T)gad[i]; gb[i] = (T)gbd[i]; }
    }
}

template <typename T, bool kGrad>
__global__ void __launch_bounds__(128) k_derivs(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4,
                                                const int2 *__restrict__ pairs, const uint32_t *__restrict__ active,
                                                T tc_scale, T *__restrict__ fac, int stride, double *partials,
                                                DevScalars *ds) {
    const unsigned long long n_act = ds->n_active;
    double e_sum = 0.0;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n_act;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        double a, b;
        T ga[18], gb[18];
        pair_values<T, kGrad>(x, tri4, pairs[active[k]], tc_scale, a, b, ga, gb);
        e_sum += (a * b) * (a * b);
        T *row = fac + k * stride;
        row[0] = (T)a;
        row[1] = (T)b;
        if (kGrad) {
#pragma unroll
            for (int i = 0; i < 18; ++i) {
                row[2 + i] = ga[i];
                row[20 + i] = gb[i];
            }
        }
    }
    grid_sum(e_sum, partials, &ds->done_counter[0], &ds->energy);
}

// Exact Hessian-vector product per intersecting pair: the pair gradient of Eq. 3,
// g = 2ab (b grad a + a grad b), evaluated in dual numbers whose tangents are the
// direction v, gives H_pair v (the full Hessian of T, including the terms Eq. 4 drops).
template <typename T>
__global__ void __launch_bounds__(128) k_hvp_pairs(const vec4_t<T> *__restrict__ x, const T *__restrict__ v,
                                                   const int4 *__restrict__ tri4, const int2 *__restrict__ pairs,
                                                   const uint32_t *__restrict__ active, T tc_scale,
                                                   T *__restrict__ h, const DevScalars *ds) {
    typedef Dual<T> S;
    const unsigned long long n_act = ds->n_active;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n_act;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const int2 pr = pairs[active[k]];
        const int4 ta = tri4[pr.x], tb = tri4[pr.y];
        const int vid[6] = {ta.x, ta.y, ta.z, tb.x, tb.y, tb.z};
        v3<S> P[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const vec4_t<T> p = x[vid[i]];
            const T *d = v + 3 * (size_t)vid[i];
            P[i] = {S(p.x, d[0]), S(p.y, d[1]), S(p.z, d[2])};
        }
        v3<S> A[3] = {P[0], P[1], P[2]}, B[3] = {P[3], P[4], P[5]};
        S a, b, ga[18], gb[18];
        Branch br;
        pair_tc<S, true>(A, B, S(tc_scale), a, b, ga, gb, br);
        const S w = S(2) * a * b;
#pragma unroll
        for (int i = 0; i < 18; ++i) h[k * 18 + i] = (w * (b * ga[i] + a * gb[i])).t;
    }
}

// The appendix's route to the derivatives, as an independent FP64 check of the analytic
// chain rule: t_c^0 and t_c^1 of every intersecting pair evaluated in forward-mode dual
// numbers (FP64 values and tangents), once per coordinate with that coordinate's tangent
// seeded to 1.  out[k] = [d t_c^0 (18), d t_c^1 (18)] in the pair's vertex order.
template <typename T>
__global__ void __launch_bounds__(128) k_dual_gradients(const vec4_t<T> *__restrict__ x, const int4 *__restrict__ tri4,
                                                        const int2 *__restrict__ pairs,
                                                        const uint32_t *__restrict__ active, double tc_scale,
                                                        double *__restrict__ out, const DevScalars *ds) {
    typedef Dual<double> S;
    const unsigned long long n_act = ds->n_active;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n_act;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const int2 pr = pairs[active[k]];
        const int4 ta = tri4[pr.x], tb = tri4[pr.y];
        const int vid[6] = {ta.x, ta.y, ta.z, tb.x, tb.y, tb.z};
        double pv[18];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const vec4_t<T> p = x[vid[i]];
            pv[3 * i] = (double)p.x; pv[3 * i + 1] = (double)p.y; pv[3 * i + 2] = (double)p.z;
        }
        for (int j = 0; j < 18; ++j) {
            v3<S> P[6];
#pragma unroll
            for (int i = 0; i < 6; ++i)
                P[i] = {S(pv[3 * i], 3 * i == j ? 1.0 : 0.0), S(pv[3 * i + 1], 3 * i + 1 == j ? 1.0 : 0.0),
                        S(pv[3 * i + 2], 3 * i + 2 == j ? 1.0 : 0.0)};
            v3<S> A[3] = {P[0], P[1], P[2]}, B[3] = {P[3], P[4], P[5]};
            S a, b, ga[18], gb[18];
            Branch br;
            pair_tc<S, false>(A, B, S(tc_scale), a, b, ga, gb, br);
            out[k * 36 + j] = a.t;
            out[k * 36 + 18 + j] = b.t;
        }
    }
}

}  // namespace

// Blocks of k_classify that are resident on the whole GPU at once: one wave of a latency-bound
// kernel (a second, partial wave would leave SMs idle at its end).
template <typename T> static int64_t classify_wave(Ctx &c) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_classify<T>, kThreads, 0) != cudaSuccess || b < 1) b = 1;
        per_sm = b;
    }
    return (int64_t)per_sm * (c.num_sms > 0 ? c.num_sms : kNumSMs);
}

template <typename T>
cudaError_t eval_candidates(Ctx &c, const vec4_t<T> *x, const int2 *pairs, int64_t n, unsigned what) {
    const int64_t n_words = (n + 31) / 32;
    TTIE_CUDA_TRY(ensure(c, c.act_bits, (size_t)(n_words > 0 ? n_words : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.word_off, (size_t)(n_words + 1) * 8));
    TTIE_CUDA_TRY(ensure(c, c.defer, (size_t)(n > 0 ? n : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.defer2, (size_t)(n > 0 ? n : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.active, (size_t)(n > 0 ? n : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)kNumSMs * 16 * sizeof(double)));
    TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->n_defer, 0, 16, c.stream));   // n_defer, n_defer2
    TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->filter_stats[0], 0, 3 * 8, c.stream));
    auto *bits = (uint32_t *)c.act_bits.p;
    const int4 *tri4 = (const int4 *)c.tri4.p;
    if (n > 0) {
        const unsigned g = grid_for(n_words * 32, kThreads, classify_wave<T>(c));
        if (c.time_kernels) cudaEventRecord(c.ev[6], c.stream);
        launch(c, k_classify<T>, dim3(g), dim3(kThreads), x, tri4, pairs, n, (const unsigned long long *)nullptr,
               c.prm.exact_only, bits, (uint32_t *)c.defer.p, c.ds);
        if (c.time_kernels) cudaEventRecord(c.ev[7], c.stream);
        launch(c, k_resolve_f64<T>, dim3(kNumSMs * 8), dim3(128), x, tri4, pairs, (const uint32_t *)c.defer.p,
               c.prm.exact_only, bits, (uint32_t *)c.defer2.p, c.ds);
        launch(c, k_resolve<T>, dim3(kNumSMs * 4), dim3(64), x, tri4, pairs, (const uint32_t *)c.defer2.p,
               c.prm.exact_only, bits, c.ds);
        TTIE_CUDA_TRY(ensure(c, c.gtmp, (size_t)(n_words > 0 ? n_words : 1) * 4));
        launch(c, k_popc, dim3(grid_for(n_words, kThreads)), dim3(kThreads), bits, n_words, (uint32_t *)c.gtmp.p);
        TTIE_CUDA_TRY(scan_u32_u64(c, (const uint32_t *)c.gtmp.p, (unsigned long long *)c.word_off.p, n_words));
        launch(c, k_compact, dim3(grid_for(n_words, kThreads)), dim3(kThreads), 
            bits, n_words, (const unsigned long long *)c.word_off.p, (uint32_t *)c.active.p, c.ds);
    } else {
        TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->n_active, 0, 8, c.stream));
    }
    TTIE_CUDA_TRY(cudaGetLastError());
    const bool grad = (what & (TTIE_EVAL_G | TTIE_EVAL_H)) != 0;
    // read the count (one sync) so the per-pair rows are sized by the active set
    TTIE_CUDA_TRY(cudaMemcpyAsync(&c.hs->n_active, &c.ds->n_active, 8, cudaMemcpyDeviceToHost, c.stream));
    TTIE_CUDA_TRY(cudaStreamSynchronize(c.stream));
    const int64_t n_act = (int64_t)c.hs->n_active;
    TTIE_CUDA_TRY(ensure(c, c.fac, (size_t)(n_act > 0 ? n_act : 1) * kFacStride * sizeof(T)));
    const unsigned gd = grid_for(n_act, 128, (int64_t)kNumSMs * 8);
    if (grad)
        launch(c, k_derivs<T, true>, dim3(gd), dim3(128), x, tri4, pairs, (const uint32_t *)c.active.p, (T)c.prm.tc_scale,
               (T *)c.fac.p, kFacStride, (double *)c.partials.p, c.ds);
    else
        launch(c, k_derivs<T, false>, dim3(gd), dim3(128), x, tri4, pairs, (const uint32_t *)c.active.p, (T)c.prm.tc_scale,
               (T *)c.fac.p, kFacStride, (double *)c.partials.p, c.ds);
    c.n_active = n_act;
    return cudaGetLastError();
}
template cudaError_t eval_candidates<float>(Ctx &, const float4 *, const int2 *, int64_t, unsigned);
template cudaError_t eval_candidates<double>(Ctx &, const dvec4 *, const int2 *, int64_t, unsigned);

// Energy and intersecting pairs over a candidate list without reading anything back on the
// host, so that the sequence can be captured into a CUDA graph: launch sizes follow the
// list's capacity n_cap, the actual length is *d_n on the device (nullptr: n_cap), and t_c^0,
// t_c^1 of the intersecting pairs go to ab (2 per pair, room for n_cap).  Results in
// ds->energy and ds->n_active.  prepare_energy_eval sizes every buffer for n_cap first
// (nothing may be allocated while a graph is captured).
template <typename T> cudaError_t prepare_energy_eval(Ctx &c, int64_t n_cap) {
    const int64_t n_words = (n_cap + 31) / 32;
    TTIE_CUDA_TRY(ensure(c, c.act_bits, (size_t)(n_words > 0 ? n_words : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.word_off, (size_t)(n_words + 1) * 8));
    TTIE_CUDA_TRY(ensure(c, c.defer, (size_t)(n_cap > 0 ? n_cap : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.defer2, (size_t)(n_cap > 0 ? n_cap : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.active, (size_t)(n_cap > 0 ? n_cap : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.partials, (size_t)kNumSMs * 16 * sizeof(double)));
    TTIE_CUDA_TRY(ensure(c, c.gtmp, (size_t)(n_cap > 0 ? n_cap : 1) * 4));
    TTIE_CUDA_TRY(ensure(c, c.ab, (size_t)(n_cap > 0 ? n_cap : 1) * 2 * sizeof(T)));
    TTIE_CUDA_TRY(ensure(c, c.scan_tmp, (size_t)((n_cap + 2047) / 2048 + 2) * 8));
    return cudaSuccess;
}
template cudaError_t prepare_energy_eval<float>(Ctx &, int64_t);
template cudaError_t prepare_energy_eval<double>(Ctx &, int64_t);

template <typename T>
cudaError_t energy_eval_nosync(Ctx &c, const vec4_t<T> *x, const int2 *pairs, int64_t n_cap,
                               const unsigned long long *d_n) {
    const int64_t n_words = (n_cap + 31) / 32;
    TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->n_defer, 0, 16, c.stream));   // n_defer, n_defer2
    TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->filter_stats[0], 0, 3 * 8, c.stream));
    auto *bits = (uint32_t *)c.act_bits.p;
    const int4 *tri4 = (const int4 *)c.tri4.p;
    if (n_cap > 0) {
        const unsigned g = grid_for(n_words * 32, kThreads, classify_wave<T>(c));
        launch(c, k_classify<T>, dim3(g), dim3(kThreads), x, tri4, pairs, n_cap, d_n, c.prm.exact_only, bits,
               (uint32_t *)c.defer.p, c.ds);
        launch(c, k_resolve_f64<T>, dim3(kNumSMs * 8), dim3(128), x, tri4, pairs, (const uint32_t *)c.defer.p,
               c.prm.exact_only, bits, (uint32_t *)c.defer2.p, c.ds);
        launch(c, k_resolve<T>, dim3(kNumSMs * 4), dim3(64), x, tri4, pairs, (const uint32_t *)c.defer2.p,
               c.prm.exact_only, bits, c.ds);
        launch(c, k_popc, dim3(grid_for(n_words, kThreads)), dim3(kThreads), (const uint32_t *)bits, n_words,
               (uint32_t *)c.gtmp.p);
        TTIE_CUDA_TRY(scan_u32_u64(c, (const uint32_t *)c.gtmp.p, (unsigned long long *)c.word_off.p, n_words));
        launch(c, k_compact, dim3(grid_for(n_words, kThreads)), dim3(kThreads), (const uint32_t *)bits, n_words,
               (const unsigned long long *)c.word_off.p, (uint32_t *)c.active.p, c.ds);
    } else {
        TTIE_CUDA_TRY(cudaMemsetAsync(&c.ds->n_active, 0, 8, c.stream));
    }
    launch(c, k_derivs<T, false>, dim3(grid_for(n_cap, 128, (int64_t)kNumSMs * 8)), dim3(128), x, tri4, pairs,
           (const uint32_t *)c.active.p, (T)c.prm.tc_scale, (T *)c.ab.p, 2, (double *)c.partials.p, c.ds);
    return cudaGetLastError();
}
template cudaError_t energy_eval_nosync<float>(Ctx &, const float4 *, const int2 *, int64_t, const unsigned long long *);
template cudaError_t energy_eval_nosync<double>(Ctx &, const dvec4 *, const int2 *, int64_t, const unsigned long long *);

// Per intersecting pair of the last evaluation: the exact Hessian of T times the direction v
// (V x 3), 18 values per pair in the order of the pair's vertices.
template <typename T> cudaError_t hvp_pairs(Ctx &c, const vec4_t<T> *x, const T *v, T *h) {
    launch(c, k_hvp_pairs<T>, dim3(grid_for(c.n_active, 128, (int64_t)kNumSMs * 8)), dim3(128), x, v,
           (const int4 *)c.tri4.p, (const int2 *)c.cand.p, (const uint32_t *)c.active.p, (T)c.prm.tc_scale, h, c.ds);
    return cudaGetLastError();
}
template cudaError_t hvp_pairs<float>(Ctx &, const float4 *, const float *, float *);

template <typename T> cudaError_t dual_gradients(Ctx &c, const vec4_t<T> *x, double *out) {
    launch(c, k_dual_gradients<T>, dim3(grid_for(c.n_active, 128, (int64_t)kNumSMs * 8)), dim3(128), x,
           (const int4 *)c.tri4.p, (const int2 *)c.cand.p, (const uint32_t *)c.active.p, c.prm.tc_scale, out,
           (const DevScalars *)c.ds);
    return cudaGetLastError();
}
template cudaError_t dual_gradients<float>(Ctx &, const float4 *, double *);
template cudaError_t dual_gradients<double>(Ctx &, const dvec4 *, double *);
template cudaError_t hvp_pairs<double>(Ctx &, const dvec4 *, const double *, double *);

}  // namespace ttie
