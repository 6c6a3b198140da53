// Internal declarations shared by the translation units of libttie.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <string>

#include "ttie.h"

namespace ttie {

// ------------------------------------------------------------------ vector types
struct alignas(32) dvec4 { double x, y, z, w; };

template <typename T> struct vec4_of;
template <> struct vec4_of<float> { typedef float4 type; };
template <> struct vec4_of<double> { typedef dvec4 type; };
template <typename T> using vec4_t = typename vec4_of<T>::type;

template <typename T> struct v3 { T x, y, z; };

template <typename T> __host__ __device__ __forceinline__ v3<T> mk(T x, T y, T z) { return {x, y, z}; }
template <typename T> __host__ __device__ __forceinline__ v3<T> xyz(const vec4_t<T> &a) { return {a.x, a.y, a.z}; }
template <typename T> __host__ __device__ __forceinline__ v3<T> operator+(v3<T> a, v3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T> __host__ __device__ __forceinline__ v3<T> operator-(v3<T> a, v3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T> __host__ __device__ __forceinline__ v3<T> operator*(T s, v3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T> __host__ __device__ __forceinline__ T dot(v3<T> a, v3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T> __host__ __device__ __forceinline__ v3<T> cross(v3<T> a, v3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T> __host__ __device__ __forceinline__ v3<T> vabs(v3<T> a) { return {fabs(a.x), fabs(a.y), fabs(a.z)}; }
// |a| x |b| componentwise "absolute cross product": the permanent of the cross product
template <typename T> __host__ __device__ __forceinline__ v3<T> abs_cross(v3<T> a, v3<T> b) {
    return {fabs(a.y * b.z) + fabs(a.z * b.y), fabs(a.z * b.x) + fabs(a.x * b.z), fabs(a.x * b.y) + fabs(a.y * b.x)};
}

template <typename T> struct Box { vec4_t<T> lo, hi; };

// ------------------------------------------------------------------ device scalars
// One small block of device memory holding counters and reduction results; it is
// copied to a pinned host mirror when the host needs a value.
enum ErrBits : int {
    ERR_NONFINITE = 1,      // NaN / Inf in positions
    ERR_BAD_INDEX = 2,      // triangle index outside [0, V) or group outside [0, 2^20)
    ERR_STACK = 4,          // traversal stack overflow
    ERR_DEFER = 8,          // exact-resolve list overflow
    ERR_BARRIER = 16,       // a grid barrier wait ran out of its iteration limit
    ERR_CHECK = 32,         // a bounds check of a TTIE_CHECKS build failed (see check_code)
    ERR_GROUP = 64,         // batched instances: a vertex in two groups, or a group's vertices not contiguous
};


// Per-pair rows of the evaluation: [a, b, grad a (18), grad b (18), pad 2] (a = t_c^0, b = t_c^1)
constexpr int kFacStride = 40;

// One instance of a batched solve (intra-group pair mode): its rows of the assembled system,
// its PCG result, its energies and its line-search state.
struct Inst {
    int first, last, count;   // rows [first, last] of the system (contiguous), count of them
    int nnz;                  // 3x3 blocks of its rows
    int iters;                // PCG iterations
    int prods;                // products with the matrix (iterations, plus the polynomial's with Chebyshev)
    double rel;               // PCG relative residual
    double gd;                // g . d after the step cap
    double e0, et, e_new;     // energy at x, at the current trial, at the accepted step
    int n0, nt, n_new;        // intersecting pairs at x, at the trial, at the accepted step
    int seg_lo, seg_hi;       // its range in the active-pair list of the last evaluation
    int pending;              // line search not yet accepted
    double alpha;             // accepted step
};

struct DevScalars {
    unsigned long long n_cand;
    unsigned long long n_active;
    unsigned long long n_defer;           // pairs the FP32 pass left undecided
    unsigned long long n_defer2;          // pairs the FP64 filter left undecided (cleared with n_defer)
    unsigned long long n_rows;
    unsigned long long nnzb;
    unsigned long long n_groups_seen;
    unsigned long long filter_stats[3];   // signs decided by FP32 filter, FP64 filter, exact
    int err;
    int max_group;
    unsigned int done_counter[8];         // "last block" reduction tickets
    unsigned long long bounds_lo[3];      // scene bounds as order-preserving integers
    unsigned long long bounds_hi[3];
    double energy;
    double trace;                          // sum of diag(H+) over active DOFs
    double mu;
    double red[8];                         // PCG scalars
    int pcg_done;
    int pcg_iters;
    int check_code;                        // first failed bounds check (TTIE_CHECKS builds)
    long long check_value;                 // the offending index
    unsigned int bar_count;                // arrivals at the PCG kernels' grid all-reduce
    unsigned int bar_gen;                  // its generation (bumped on release)
    unsigned int n_pending;                // batched line search: instances still open
    double ls_alpha, ls_last;              // batched line search: trial step, 1 on the last trial
    double batch[10];                      // batched step totals (instance_totals)
    double el_energy;                      // energy of the elastic term at the last evaluation
    unsigned long long pcg_products;       // Chebyshev-preconditioned PCG: products computed
    unsigned long long ovf_cursor;         // one-walk traversal: overflow chunks taken
    unsigned int inst_queue;               // batched PCG: next instance to take
    double cg_alpha, cg_beta;              // streamed PCG: the step's coefficients (decided on the device)
    double cg_gamma_prev, cg_alpha_prev;   //   the previous iteration's r.u and alpha
    int cg_stop_next;                      //   breakdown at the first iteration: stop after its update
};

static_assert(offsetof(DevScalars, n_defer2) == offsetof(DevScalars, n_defer) + sizeof(unsigned long long),
              "n_defer and n_defer2 are cleared by one 16-byte memset");

// ------------------------------------------------------------------ buffers
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Ctx;
cudaError_t ensure(Ctx &c, Buf &b, size_t bytes);   // grow-only, contents not kept

#define TTIE_BUFS(X)                                                                       \
    X(tri4) X(grp) X(xp) X(xq) X(tbox) X(mkey) X(mkey2) X(perm) X(perm2) X(sort_cnt)       \
    X(node_box) X(node_child) X(node_parent) X(node_range) X(visit) X(leaf_group)          \
    X(group_range) X(cand_cnt) X(cand_off) X(cand) X(scan_tmp) X(act_bits) X(word_off)     \
    X(defer) X(active) X(fac) X(partials) X(vflag) X(vrow) X(row_vertex) X(bkey) X(bkey2)   \
    X(bval) X(bval2) X(bflag) X(run_start) X(row_ptr) X(col_idx) X(bsr_val) X(rhs)         \
    X(zfac) X(dinv) X(pcg_x) X(pcg_r) X(pcg_z) X(pcg_p) X(pcg_q) X(dir) X(xt) X(gtmp)      \
    X(xsave) X(sweep_cand) X(pcg_z4) X(pcg_z4b) X(hbuf) X(pcg_sync) X(spill) X(pcg_w) X(vgroup) X(iedge)  \
    X(el_edges) X(el_rest) X(el_anchor) X(el_target) X(el_sfac) X(el_afac) X(defer2)          \
    X(inst) X(ls_cand) X(inst_acc) X(inst_ids) X(ab) X(ls_flag)  \
    X(ls_off) X(ls_scalars) X(hgrid) X(hkey) X(hkey2) X(hval) X(hval2) X(hcnt) X(hoff)   \
    X(ovf_pool) X(ovf_next) X(ovf_head) X(leaf_tri) X(inst_cd) X(inst_crr)

struct Ctx {
    ttie_params prm;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    // topology recorded by ttie_build_bvh
    bool have_mesh = false;
    int64_t V = 0, F = 0;
    int x_stride = 3;
    bool have_group = false;
    int n_groups = 1;
    int group_bits = 0;
    // state of the last calls
    bool have_cand = false;
    int64_t n_cand = 0;
    bool have_eval = false;
    unsigned eval_what = 0;
    int64_t n_active = 0;
    bool have_bsr = false;
    bool pcg_cheb = false;   // the last PCG ran the Chebyshev-preconditioned kernel
    bool pcg_streamed = false;   // the last PCG ran the streamed kernels
    unsigned long long ovf_chunks = 0;   // one-walk traversal: chunks the last walk needed, + 25 %
    int64_t n_rows = 0, nnzb = 0;
    bool have_dir = false;
    double mean_edge = 0.0;   // mean edge length at the last ttie_build_bvh
    double eta_cur = 0.0;     // overshoot of the next line search (adaptive with TTIE_LS_FEWER)
    // memory
    DevScalars *ds = nullptr;     // device
    DevScalars *hs = nullptr;     // pinned host mirror
#define TTIE_DECL_BUF(name) Buf name;
    TTIE_BUFS(TTIE_DECL_BUF)
#undef TTIE_DECL_BUF
    cudaEvent_t ev[12] = {};
    cudaStream_t cap_stream = nullptr;         // stream that graphs are captured on (lazily made)
    int num_sms = 0;
    unsigned long long n_launch = 0;   // kernels launched through this context
    bool time_kernels = false;         // profile: events around the classification / PCG kernels
    int64_t tree_leaves = -1;          // leaves of the hierarchy in the BVH buffers (-1: none)
    int inst_tuned[4] = {0, 0, 0, 0};  // batched PCG schedule: threads, blocks per SM, order (0: not tuned)
    unsigned long long mark_launch[6] = {};   // n_launch at the step's stage marks
    // elastic term of the quasi-static simulation (ttie_set_elastic)
    bool have_elastic = false;
    int64_t el_n_edges = 0, el_n_anchors = 0, el_V = -1;
    int el_prec = 0;
    // the Morton sort of a full LBVH build, captured once as a graph and replayed while its
    // arguments and scratch buffers stay the same
    cudaGraphExec_t sort_exec = nullptr;
    const void *sort_key[7] = {};       // keys, vals, keys2, vals2, count and scan scratch, (n, bits)
    long long sort_n = -1;
    int sort_bits = -1;
    unsigned long long sort_kernels = 0;
    double el_k = 0.0, el_ka = 0.0;
};

// Every kernel of the library is launched through this helper on the context's
// stream, which also counts the launches.  A TTIE_CHECKS build also synchronises after
// every launch and reports the kernel's signature when it failed.
template <typename... KArgs, typename... Args>
inline void launch(Ctx &c, void (*kernel)(KArgs...), dim3 grid, dim3 block, Args &&...args) {
    ++c.n_launch;
    kernel<<<grid, block, 0, c.stream>>>(static_cast<KArgs>(args)...);
#ifdef TTIE_CHECKS
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) fprintf(stderr, "TTIE_CHECKS: launch %llu failed (%s) in %s\n", c.n_launch, cudaGetErrorString(e), __PRETTY_FUNCTION__);
#endif
}

// Bounds checks of TTIE_CHECKS builds: record the first failure and let the caller skip the
// access.  In other builds they compile to nothing.
#ifdef TTIE_CHECKS
__device__ __forceinline__ bool ttie_check_fail(DevScalars *ds, int code, long long v) {
    if (atomicCAS(&ds->check_code, 0, code) == 0) ds->check_value = v;
    atomicOr(&ds->err, ERR_CHECK);
    return true;
}
#define TTIE_BAD(ds, cond, code, v) (!(cond) && ttie_check_fail((ds), (code), (long long)(v)))
#else
#define TTIE_BAD(ds, cond, code, v) false
#endif

// ------------------------------------------------------------------ launch helpers
constexpr int kNumSMs = 152;
inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 16) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ------------------------------------------------------------------ primitives (sort_scan.cu)
// Exclusive scan of n uint32 counts into uint64 offsets; out[n] = total.
cudaError_t scan_u32_u64(Ctx &c, const uint32_t *in, unsigned long long *out, int64_t n);
// Stable LSD radix sort of (key, value) by the low `bits` bits of key; keys2/vals2 are scratch
// of the same size.  The result is left in keys/vals, or, with in_second, wherever the last
// pass wrote it: *in_second tells whether that is keys2/vals2 (no copy back).
cudaError_t radix_sort(Ctx &c, unsigned long long *keys, uint32_t *vals, unsigned long long *keys2,
                       uint32_t *vals2, int64_t n, int bits, bool *in_second = nullptr);
// The same sort replayed from a graph captured on the first call with these arguments.
cudaError_t radix_sort_graph(Ctx &c, unsigned long long *keys, uint32_t *vals, unsigned long long *keys2,
                             uint32_t *vals2, int64_t n, int bits);

// ------------------------------------------------------------------ broad phase (bvh.cu)
template <typename T> cudaError_t pack_positions(Ctx &c, const T *x, int stride, vec4_t<T> *out);
cudaError_t pack_topology(Ctx &c, const int32_t *tri, const int32_t *group);
// Candidate pairs whose boxes (over x0, or swept from x0 to x1) overlap.  When the count
// exceeds `cap` nothing is written and *n_out receives the count.
// refit_only: keep the hierarchy of the last full build of this mesh (the line search's swept
// boxes reuse the tree built at x) and only refit it to the new boxes.
// spatial-hashing broad phase over the triangle boxes of the last k_tri_boxes (hash.cu)
template <typename T> cudaError_t hash_candidates(Ctx &c, const Box<T> *box, Buf &out_pairs, int64_t *n_out, int64_t cap);
template <typename T> cudaError_t build_candidates(Ctx &c, const vec4_t<T> *x0, const vec4_t<T> *x1,
                                                   Buf &out_pairs, int64_t *n_out, int64_t cap,
                                                   bool refit_only = false);

// batched independent instances (instances.cu)
cudaError_t instance_vertex_groups(Ctx &c);
template <typename T> cudaError_t instance_edges(Ctx &c, const vec4_t<T> *x);
cudaError_t instance_layout(Ctx &c);
template <typename T> cudaError_t instance_energies(Ctx &c, const int2 *pairs, int at_trial);
template <typename T> cudaError_t instance_pcg(Ctx &c, const T *rhs, T *out);
cudaError_t instance_ls_init(Ctx &c);
cudaError_t instance_ls_accept(Ctx &c, double alpha, int last, unsigned int *d_pending);
cudaError_t instance_pending_pairs(Ctx &c, const int2 *pairs, int64_t n, Buf &out, int64_t *n_out);
// One line-search trial of every open instance as a CUDA graph (capture once per Newton step,
// replay per trial after writing the step into the host mirror's ls_alpha / ls_last).
template <typename T>
cudaError_t instance_trial_graph(Ctx &c, const vec4_t<T> *xp, const T *dir, vec4_t<T> *xt, const int2 *cand,
                                 int64_t ns, cudaGraphExec_t *exec, unsigned long long *kernels);
template <typename T> cudaError_t instance_update(Ctx &c, T *x, int stride, const T *d_full);
cudaError_t instance_totals(Ctx &c, double *d_out);   // 10 values
cudaError_t brute_candidates(Ctx &c, Buf &out_pairs, int64_t *n_out);
template <typename T> cudaError_t mean_edge_length(Ctx &c, const vec4_t<T> *x, double *out_dev);

// ------------------------------------------------------------------ narrow phase (pair_eval.cu)
// what: TTIE_EVAL_* bits.  Classifies the n candidate pairs at x, compacts the
// intersecting ones (ctx.active), and with G|H writes their t_c and gradients (ctx.fac).
// Energy lands in ds->energy, count in ds->n_active.
template <typename T> cudaError_t eval_candidates(Ctx &c, const vec4_t<T> *x, const int2 *pairs, int64_t n,
                                                  unsigned what);
template <typename T> cudaError_t prepare_energy_eval(Ctx &c, int64_t n_cap);
template <typename T>
cudaError_t energy_eval_nosync(Ctx &c, const vec4_t<T> *x, const int2 *pairs, int64_t n_cap,
                               const unsigned long long *d_n);

// ------------------------------------------------------------------ assembly (assemble.cu)
// with_elastic: the elastic term (ttie_set_elastic) is added to the pairs' system
template <typename T> cudaError_t assemble_system(Ctx &c, T *grad_out_V3, bool with_elastic = false);
template <typename T> cudaError_t elastic_energy(Ctx &c, const vec4_t<T> *x);   // -> ds->el_energy
template <typename T> cudaError_t elastic_set(Ctx &c, const ttie_elastic *e);
// ------------------------------------------------------------------ solve (pcg.cu)
template <typename T> cudaError_t pcg_solve(Ctx &c, const T *rhs, T *out, double rtol, int max_it);
// ------------------------------------------------------------------ (assemble.cu)
// Hessian-vector products: per-pair exact products (pair_eval.cu), their per-vertex sums over
// the last assembly's diagonal runs, and the assembled PSD Hessian times v.
template <typename T> cudaError_t hvp_pairs(Ctx &c, const vec4_t<T> *x, const T *v, T *h);
template <typename T> cudaError_t dual_gradients(Ctx &c, const vec4_t<T> *x, double *out);
template <typename T> cudaError_t vertex_sums(Ctx &c, const T *h, T *out);
template <typename T> cudaError_t bsr_matvec(Ctx &c, const T *v, T *out);
// out_dev[0] = g.d, out_dev[1] = max over rows of |d_r|^2 (rows of the assembled system)
template <typename T> cudaError_t direction_stats(Ctx &c, const T *g, const T *d, double *out_dev);
template <typename T> cudaError_t axpy_positions(Ctx &c, const vec4_t<T> *x, const T *d, T alpha, vec4_t<T> *out);
template <typename T> cudaError_t scatter_direction(Ctx &c, const T *d_rows, T *d_full);
template <typename T> cudaError_t update_positions(Ctx &c, T *x, int stride, const T *d_full, T alpha);

}  // namespace ttie

#define TTIE_CUDA_TRY(expr)                              \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) return _e;                \
    } while (0)
