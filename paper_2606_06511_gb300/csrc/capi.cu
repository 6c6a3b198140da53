// C ABI of libttie: argument checks, context memory, and the order of the stages.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "common.cuh"

namespace ttie {

cudaError_t ensure(Ctx &c, Buf &b, size_t bytes) {
    (void)c;
    if (b.bytes >= bytes) return cudaSuccess;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);   // waits for pending work that may still use it
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return e;
    }
    const size_t nb = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.bytes = nb;
    return cudaSuccess;
}


namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void k_copy_neg(const T *__restrict__ a, T *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = -a[i];
}

template <typename T> __global__ void k_scale(T *a, int64_t n, double s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (T)(a[i] * s);
}

__global__ void k_gather_active(const int2 *__restrict__ cand, const uint32_t *__restrict__ active, int64_t n,
                                int2 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cand[active[i]];
}

template <typename T>
__global__ void k_split_fac(const T *__restrict__ fac, int64_t n, T *__restrict__ tc, T *__restrict__ dtc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T *r = fac + i * 40;
        if (tc) { tc[2 * i] = r[0]; tc[2 * i + 1] = r[1]; }
        if (dtc)
            for (int k = 0; k < 36; ++k) dtc[36 * i + k] = r[2 + k];
    }
}

}  // namespace

template <typename T> cudaError_t scale(Ctx &c, T *a, int64_t n, double s) {
    launch(c, k_scale<T>, dim3(grid_for(n, kThreads)), dim3(kThreads), a, n, s);
    return cudaGetLastError();
}

}  // namespace ttie

using namespace ttie;

struct ttie_ctx {
    Ctx c;
};

static ttie_status set_err(Ctx &c, ttie_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c.err = buf;
    return s;
}

static ttie_status cuda_err(Ctx &c, cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(c, TTIE_ERR_OOM, "%s: device allocation failed", where);
    }
    return set_err(c, TTIE_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(expr, where)                                      \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return cuda_err(c, _e, where); \
    } while (0)

static ttie_status check_params(Ctx &c, const ttie_params *p) {
    if (!p) return set_err(c, TTIE_ERR_INVALID, "params is NULL");
    if (p->precision != TTIE_F32 && p->precision != TTIE_F64) return set_err(c, TTIE_ERR_INVALID, "precision");
    const int m = p->pair_mode & 3;
    if (m == 3 || (p->pair_mode & ~15) || ((p->pair_mode & TTIE_PAIRS_BRUTE) && (p->pair_mode & TTIE_PAIRS_HASH)))
        return set_err(c, TTIE_ERR_INVALID, "pair_mode");
    if (p->psd_mode != TTIE_PSD_PER_PART && p->psd_mode != TTIE_PSD_DROP_CROSS && p->psd_mode != TTIE_PSD_WHOLE)
        return set_err(c, TTIE_ERR_INVALID, "psd_mode");
    if (!(p->tc_scale > 0.0) || !(p->mu_rel >= 0.0) || !(p->pcg_rtol > 0.0) || p->pcg_max_it < 1 ||
        p->newton_max_it < 0 || p->ls_max_halvings < 0 || p->ls_max_halvings > 60 || !(p->armijo_c >= 0.0) ||
        !(p->push_eta >= 0.0) || !(p->max_step >= 0.0) || p->max_candidates < 0 ||
        (p->inst_threads != 0 && p->inst_threads != 128 && p->inst_threads != 256 && p->inst_threads != 512 &&
         p->inst_threads != 1024) ||
        (p->test_withhold != 0 && p->test_withhold != 1) ||
        (p->pcg_precond != TTIE_PCG_BLOCK_JACOBI && p->pcg_precond != TTIE_PCG_CHEBYSHEV &&
         p->pcg_precond != TTIE_PCG_AUTO) ||
        p->pcg_cheb_degree < 0 || p->pcg_cheb_degree > 8 ||
        (p->traversal_mode != TTIE_TRAVERSAL_TWO_WALKS && p->traversal_mode != TTIE_TRAVERSAL_ONE_WALK) ||
        (p->ls_rule != TTIE_LS_ARMIJO && p->ls_rule != TTIE_LS_FEWER) ||
        !(p->push_eta_max >= 0.0) || p->push_eta_max > 1e3 ||
        p->pcg_kernel < TTIE_PCG_KERNEL_AUTO || p->pcg_kernel > TTIE_PCG_KERNEL_RESIDENT_UNCACHED ||
        p->exact_only < 0 || p->exact_only > 2)
        return set_err(c, TTIE_ERR_INVALID, "numeric parameter out of range");
    return TTIE_OK;
}

extern "C" {

void ttie_default_params(ttie_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->precision = TTIE_F32;
    p->pair_mode = TTIE_PAIRS_SELF;
    p->psd_mode = TTIE_PSD_PER_PART;
    p->tc_scale = 1.0;
    p->mu_rel = 1e-3;
    p->pcg_rtol = 1e-3;
    p->pcg_max_it = 200;
    p->newton_max_it = 200;
    p->ls_max_halvings = 20;
    p->armijo_c = 1e-4;
    p->push_eta = 0.5;
    p->max_step = 1.0;
    p->max_candidates = 0;
    p->inst_threads = 0;
    p->test_withhold = 0;
    p->pcg_precond = TTIE_PCG_AUTO;
    p->pcg_cheb_degree = 0;
    p->traversal_mode = TTIE_TRAVERSAL_ONE_WALK;
    p->ls_rule = TTIE_LS_ARMIJO;
    p->push_eta_max = 1.5;
    p->pcg_kernel = TTIE_PCG_KERNEL_AUTO;
}

ttie_status ttie_create(ttie_ctx **out, const ttie_params *p, void *stream) {
    if (!out) return TTIE_ERR_INVALID;
    *out = nullptr;
    ttie_ctx *h = new (std::nothrow) ttie_ctx;
    if (!h) return TTIE_ERR_OOM;
    Ctx &c = h->c;
    ttie_params def;
    ttie_default_params(&def);
    if (check_params(c, p ? p : &def) != TTIE_OK) {
        delete h;
        return TTIE_ERR_INVALID;
    }
    c.prm = p ? *p : def;
    c.stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
    if (e == cudaSuccess) e = cudaMalloc(&c.ds, sizeof(DevScalars));
    if (e == cudaSuccess) e = cudaMallocHost(&c.hs, sizeof(DevScalars));
    if (e == cudaSuccess) e = cudaMemsetAsync(c.ds, 0, sizeof(DevScalars), c.stream);
    for (int i = 0; i < 12 && e == cudaSuccess; ++i) e = cudaEventCreate(&c.ev[i]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        ttie_status s = e == cudaErrorMemoryAllocation ? TTIE_ERR_OOM : TTIE_ERR_CUDA;
        cudaGetLastError();
        ttie_destroy(h);
        return s;
    }
    std::memset(c.hs, 0, sizeof(DevScalars));
    *out = h;
    return TTIE_OK;
}

void ttie_destroy(ttie_ctx *h) {
    if (!h) return;
    Ctx &c = h->c;
    if (c.stream || c.ds) cudaStreamSynchronize(c.stream);
#define TTIE_FREE_BUF(name) if (c.name.p) cudaFree(c.name.p);
    TTIE_BUFS(TTIE_FREE_BUF)
#undef TTIE_FREE_BUF
    if (c.ds) cudaFree(c.ds);
    if (c.hs) cudaFreeHost(c.hs);
    for (int i = 0; i < 12; ++i)
        if (c.ev[i]) cudaEventDestroy(c.ev[i]);
    if (c.sort_exec) cudaGraphExecDestroy(c.sort_exec);
    if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
    delete h;
}

const char *ttie_last_error(const ttie_ctx *h) {
    if (!h) return "null context";
    return h->c.err.c_str();
}

ttie_status ttie_set_params(ttie_ctx *h, const ttie_params *p) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    ttie_status s = check_params(c, p);
    if (s != TTIE_OK) return s;
    if (c.have_mesh && p->precision != c.prm.precision)
        return set_err(c, TTIE_ERR_STATE, "precision cannot change after ttie_build_bvh");
    c.prm = *p;
    return TTIE_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ stage helpers
static int64_t cand_cap(const Ctx &c) {
    return c.prm.max_candidates > 0 ? c.prm.max_candidates : 64 * c.F + 1000000;
}

static ttie_status read_err(Ctx &c, const char *where) {
    CK(cudaMemcpyAsync(&c.hs->err, &c.ds->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream), where);
    CK(cudaStreamSynchronize(c.stream), where);
    const int e = c.hs->err;
    if (e) CK(cudaMemsetAsync(&c.ds->err, 0, sizeof(int), c.stream), where);
    if (e & ERR_BAD_INDEX)
        return set_err(c, TTIE_ERR_INVALID, "%s: index out of range (triangle, group, spring or anchor)", where);
    if (e & ERR_NONFINITE) return set_err(c, TTIE_ERR_NONFINITE, "%s: non-finite vertex position", where);
    if (e & ERR_STACK)
        return set_err(c, TTIE_ERR_CAPACITY, "%s: broad-phase capacity exceeded (BVH depth or hash cells per triangle)",
                       where);
    if (e & ERR_BARRIER) return set_err(c, TTIE_ERR_CUDA, "%s: PCG grid barrier timed out", where);
    if (e & ERR_GROUP)
        return set_err(c, TTIE_ERR_INVALID,
                       "%s: batched instances need every vertex in one group and each group's vertices numbered "
                       "contiguously", where);
    if (e & ERR_CHECK) {
        CK(cudaMemcpyAsync(c.hs, c.ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.stream), where);
        CK(cudaStreamSynchronize(c.stream), where);
        return set_err(c, TTIE_ERR_CAPACITY, "%s: bounds check %d failed (value %lld)", where, c.hs->check_code,
                       c.hs->check_value);
    }
    return TTIE_OK;
}

// Intra-group pairs over an LBVH: every group is an independent problem (instances.cu).
static bool batched(const Ctx &c) {
    return (c.prm.pair_mode & 3) == TTIE_PAIRS_INTRA_GROUP && c.have_group &&
           !(c.prm.pair_mode & (TTIE_PAIRS_BRUTE | TTIE_PAIRS_HASH));
}

template <typename T>
static ttie_status build_impl(Ctx &c, const T *x, const int32_t *tri, const int32_t *group, int64_t *n_cand) {
    c.have_cand = c.have_eval = c.have_bsr = c.have_dir = false;
    CK(cudaMemsetAsync(&c.ds->max_group, 0, sizeof(int), c.stream), "build");
    CK(pack_topology(c, tri, group), "build: topology");
    CK(ensure(c, c.xp, (size_t)(c.V > 0 ? c.V : 1) * sizeof(vec4_t<T>)), "build");
    CK(pack_positions<T>(c, x, c.x_stride, (vec4_t<T> *)c.xp.p), "build: positions");
    ttie_status s = read_err(c, "ttie_build_bvh");
    if (s != TTIE_OK) return s;
    c.have_group = group != nullptr;
    c.n_groups = 1;
    c.group_bits = 0;
    if (group) {
        CK(cudaMemcpyAsync(&c.hs->max_group, &c.ds->max_group, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "build");
        CK(cudaStreamSynchronize(c.stream), "build");
        c.n_groups = c.hs->max_group + 1;
        while ((1 << c.group_bits) < c.n_groups) ++c.group_bits;
        if (c.group_bits == 0) c.group_bits = 1;
    }
    c.have_mesh = true;
    c.eta_cur = c.prm.push_eta;
    int64_t n = 0;
    CK(mean_edge_length<T>(c, (const vec4_t<T> *)c.xp.p, &c.ds->red[7]), "build");
    CK(cudaMemcpyAsync(&c.hs->red[7], &c.ds->red[7], sizeof(double), cudaMemcpyDeviceToHost, c.stream), "build");
    CK(cudaStreamSynchronize(c.stream), "build");
    c.mean_edge = c.hs->red[7];
    if (c.prm.pair_mode & TTIE_PAIRS_BRUTE)
        CK(brute_candidates(c, c.cand, &n), "build: brute-force pairs");
    else
        CK(build_candidates<T>(c, (const vec4_t<T> *)c.xp.p, nullptr, c.cand, &n, cand_cap(c)), "build: LBVH");
    if (batched(c) && n <= cand_cap(c)) {
        CK(instance_vertex_groups(c), "build: instances");
        CK(instance_edges<T>(c, (const vec4_t<T> *)c.xp.p), "build: instances");
    }
    s = read_err(c, "ttie_build_bvh");
    if (s != TTIE_OK) return s;
    if (n > cand_cap(c))
        return set_err(c, TTIE_ERR_CAPACITY, "ttie_build_bvh: %lld candidate pairs exceed max_candidates %lld",
                       (long long)n, (long long)cand_cap(c));
    c.n_cand = n;
    c.have_cand = true;
    if (n_cand) *n_cand = n;
    return TTIE_OK;
}

template <typename T>
static ttie_status eval_impl(Ctx &c, const T *x, unsigned what, double *energy, int64_t *n_active, T *grad) {
    c.have_eval = c.have_bsr = false;
    CK(pack_positions<T>(c, x, c.x_stride, (vec4_t<T> *)c.xp.p), "eval: positions");
    ttie_status s = read_err(c, "ttie_eval_pairs");
    if (s != TTIE_OK) return s;
    CK(eval_candidates<T>(c, (const vec4_t<T> *)c.xp.p, (const int2 *)c.cand.p, c.n_cand, what), "eval");
    c.have_eval = true;
    c.eval_what = what;
    if (grad) {
        CK(assemble_system<T>(c, grad), "eval: gradient");
        c.have_bsr = true;
    }
    CK(cudaMemcpyAsync(&c.hs->energy, &c.ds->energy, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "eval");
    CK(cudaStreamSynchronize(c.stream), "eval");
    if (!std::isfinite(c.hs->energy)) return set_err(c, TTIE_ERR_NONFINITE, "ttie_eval_pairs: energy is not finite");
    if (energy) *energy = c.hs->energy;
    if (n_active) *n_active = c.n_active;
    return TTIE_OK;
}

// Energy and intersecting-pair count at positions xt over the given candidate list.
// Energy (sum T, plus the elastic term when one is set) and intersecting-pair count at
// positions xt over the given candidate list.
template <typename T>
static ttie_status energy_at(Ctx &c, const vec4_t<T> *xt, const int2 *pairs, int64_t n, double *E, int64_t *n_act,
                             double *E_el = nullptr) {
    CK(eval_candidates<T>(c, xt, pairs, n, TTIE_EVAL_E), "line search");
    if (c.have_elastic) {
        CK(elastic_energy<T>(c, xt), "line search: elastic term");
        CK(cudaMemcpyAsync(&c.hs->el_energy, &c.ds->el_energy, sizeof(double), cudaMemcpyDeviceToHost, c.stream),
           "line search");
    }
    CK(cudaMemcpyAsync(&c.hs->energy, &c.ds->energy, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "line search");
    CK(cudaStreamSynchronize(c.stream), "line search");
    const double el = c.have_elastic ? c.hs->el_energy : 0.0;
    *E = c.hs->energy + el;
    if (E_el) *E_el = el;
    *n_act = c.n_active;
    return TTIE_OK;
}

// The elastic term is usable with the current mesh and precision.
static ttie_status elastic_ok(Ctx &c, const char *where) {
    if (!c.have_elastic) return TTIE_OK;
    if (c.el_prec != c.prm.precision)
        return set_err(c, TTIE_ERR_STATE, "%s: the elastic term was set for the other precision", where);
    return TTIE_OK;
}

static float ms_between(Ctx &c, int a, int b) {
    float ms = 0.f;
    if (c.prm.profile) cudaEventElapsedTime(&ms, c.ev[a], c.ev[b]);
    return ms;
}

static void mark(Ctx &c, int i) {
    if (c.prm.profile) cudaEventRecord(c.ev[i], c.stream);
    if (i < 6) c.mark_launch[i] = c.n_launch;
}

// per-stage launch counts (and, batched, the PCG schedule) into a step's info
static void stage_info(const Ctx &c, ttie_step_info &inf, bool batched_step) {
    for (int k = 0; k < 5; ++k) inf.stage_launches[k] = (int64_t)(c.mark_launch[k + 1] - c.mark_launch[k]);
    if (batched_step) {
        inf.inst_threads = c.prm.inst_threads > 0 ? c.prm.inst_threads : c.inst_tuned[0];
        inf.inst_blocks_per_sm = c.inst_tuned[1];
        inf.inst_order = c.inst_tuned[2];
    }
}

template <typename T> static cudaError_t negate_copy(Ctx &c, const T *a, T *b, int64_t n) {
    launch(c, ttie::k_copy_neg<T>, dim3(grid_for(n, 256)), dim3(256), a, b, n);
    return cudaGetLastError();
}

template <typename T> static ttie_status newton_batched(Ctx &c, T *x, ttie_step_info *info);

template <typename T>
static ttie_status newton_impl(Ctx &c, T *x, ttie_step_info *info) {
    if (batched(c)) {
        if (c.have_elastic)
            return set_err(c, TTIE_ERR_INVALID, "ttie_newton_step: the elastic term is not available with batched instances");
        return newton_batched<T>(c, x, info);
    }
    {
        const ttie_status se = elastic_ok(c, "ttie_newton_step");
        if (se != TTIE_OK) return se;
    }
    ttie_step_info inf;
    std::memset(&inf, 0, sizeof inf);
    c.have_dir = false;
    mark(c, 0);
    // candidates and evaluation at x
    CK(pack_positions<T>(c, x, c.x_stride, (vec4_t<T> *)c.xp.p), "newton: positions");
    ttie_status s = read_err(c, "ttie_newton_step");
    if (s != TTIE_OK) return s;
    int64_t n = 0;
    if (c.prm.pair_mode & TTIE_PAIRS_BRUTE)
        CK(brute_candidates(c, c.cand, &n), "newton: pairs");
    else
        CK(build_candidates<T>(c, (const vec4_t<T> *)c.xp.p, nullptr, c.cand, &n, cand_cap(c)), "newton: LBVH");
    if (n > cand_cap(c)) {
        c.have_cand = false;
        return set_err(c, TTIE_ERR_CAPACITY, "ttie_newton_step: %lld candidate pairs exceed max_candidates %lld",
                       (long long)n, (long long)cand_cap(c));
    }
    c.n_cand = n;
    c.have_cand = true;
    inf.n_candidates = n;
    mark(c, 1);
    c.time_kernels = c.prm.profile != 0;
    CK(eval_candidates<T>(c, (const vec4_t<T> *)c.xp.p, (const int2 *)c.cand.p, n, TTIE_EVAL_E | TTIE_EVAL_H), "newton: eval");
    c.time_kernels = false;
    c.have_eval = true;
    c.eval_what = TTIE_EVAL_E | TTIE_EVAL_H;
    if (c.have_elastic) {
        CK(elastic_energy<T>(c, (const vec4_t<T> *)c.xp.p), "newton: elastic term");
        CK(cudaMemcpyAsync(&c.hs->el_energy, &c.ds->el_energy, sizeof(double), cudaMemcpyDeviceToHost, c.stream),
           "newton");
    }
    CK(cudaMemcpyAsync(&c.hs->energy, &c.ds->energy, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "newton");
    CK(cudaStreamSynchronize(c.stream), "newton");
    inf.energy_elastic = c.have_elastic ? c.hs->el_energy : 0.0;
    const double E = c.hs->energy + inf.energy_elastic;
    inf.energy = E;
    inf.n_active = c.n_active;
    mark(c, 2);
    if (!std::isfinite(E)) return set_err(c, TTIE_ERR_NONFINITE, "ttie_newton_step: energy is not finite");
    if (c.n_active == 0) {
        inf.energy_new = E;
        mark(c, 3); mark(c, 4); mark(c, 5);
        if (c.prm.profile) cudaEventSynchronize(c.ev[5]);
        inf.ms_build = ms_between(c, 0, 1);
        inf.ms_eval = ms_between(c, 1, 2);
        inf.ms_classify = c.n_cand > 0 ? ms_between(c, 6, 7) : 0.f;
        stage_info(c, inf, false);
        if (info) *info = inf;
        return TTIE_OK;
    }
    // assembly (with the elastic term when one is set) and PCG for (H+ + mu I) d = -g
    CK(assemble_system<T>(c, nullptr, true), "newton: assembly");
    c.have_bsr = !c.have_elastic;   // ttie_assemble's system is the pairs' alone
    inf.n_rows = c.n_rows;
    inf.nnzb = c.nnzb;
    mark(c, 3);
    const int64_t n3 = c.n_rows * 3;
    CK(ensure(c, c.pcg_x, (size_t)(n3 > 0 ? n3 : 1) * sizeof(T)), "newton");
    CK(ensure(c, c.xsave, (size_t)(n3 > 0 ? n3 : 1) * sizeof(T)), "newton");
    CK(negate_copy(c, (const T *)c.rhs.p, (T *)c.xsave.p, n3), "newton");
    CK(pcg_solve<T>(c, (const T *)c.xsave.p, (T *)c.pcg_x.p, c.prm.pcg_rtol, c.prm.pcg_max_it), "newton: PCG");
    s = read_err(c, "ttie_newton_step");
    if (s != TTIE_OK) return s;
    CK(direction_stats<T>(c, (const T *)c.rhs.p, (const T *)c.pcg_x.p, &c.ds->red[5]), "newton");
    CK(cudaMemcpyAsync(c.hs, c.ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.stream), "newton");
    CK(cudaStreamSynchronize(c.stream), "newton");
    double gd = c.hs->red[5];
    const double dmax = std::sqrt(c.hs->red[6]);
    if (!std::isfinite(gd) || !std::isfinite(dmax))
        return set_err(c, TTIE_ERR_NONFINITE, "ttie_newton_step: Newton direction is not finite");
    const double cap = c.prm.max_step * c.mean_edge;
    if (cap > 0.0 && dmax > cap) {   // step cap: no vertex moves more than max_step mean edges
        CK(scale<T>(c, (T *)c.pcg_x.p, n3, cap / dmax), "newton");
        gd *= cap / dmax;
    }
    CK(ensure(c, c.dir, (size_t)c.V * 3 * sizeof(T)), "newton");
    CK(scatter_direction<T>(c, (const T *)c.pcg_x.p, (T *)c.dir.p), "newton");
    c.have_dir = true;
    inf.grad_dot_dir = gd;
    inf.pcg_iters = c.hs->pcg_iters;
    inf.pcg_rel_residual = c.hs->red[1] > 0.0 ? std::sqrt(c.hs->red[4] / c.hs->red[1]) : 0.0;
    // the Chebyshev-preconditioned kernel multiplies k + 1 times per iteration after its restart
    const int64_t passes = c.pcg_cheb ? (int64_t)c.hs->pcg_products : (int64_t)inf.pcg_iters;
    inf.pcg_kernel = c.pcg_streamed ? TTIE_PCG_KERNEL_STREAMED
                     : c.prm.pcg_kernel == TTIE_PCG_KERNEL_RESIDENT_UNCACHED ? TTIE_PCG_KERNEL_RESIDENT_UNCACHED
                                                                             : TTIE_PCG_KERNEL_RESIDENT;
    inf.pcg_block_iters = passes * c.nnzb;
    inf.pcg_row_iters = passes * c.n_rows;
    mark(c, 4);
    // line search on candidates from the boxes swept between x and x + a_max d
    if (!(c.eta_cur >= c.prm.push_eta)) c.eta_cur = c.prm.push_eta;
    double a_max = 1.0 + (c.prm.ls_rule == TTIE_LS_FEWER ? c.eta_cur : c.prm.push_eta);
    const double a_top = a_max;
    CK(ensure(c, c.xq, (size_t)c.V * sizeof(vec4_t<T>)), "newton");
    CK(ensure(c, c.xt, (size_t)c.V * sizeof(vec4_t<T>)), "newton");
    int64_t ns = 0;
    if (c.prm.pair_mode & TTIE_PAIRS_BRUTE) {
        ns = c.n_cand;
        CK(ensure(c, c.sweep_cand, (size_t)(ns > 0 ? ns : 1) * sizeof(int2)), "newton");
        CK(cudaMemcpyAsync(c.sweep_cand.p, c.cand.p, (size_t)ns * sizeof(int2), cudaMemcpyDeviceToDevice, c.stream), "newton");
    } else {
        // a swept list beyond the cap shrinks the largest trial step until it fits
        for (int tries = 0;; ++tries) {
            CK(axpy_positions<T>(c, (const vec4_t<T> *)c.xp.p, (const T *)c.dir.p, (T)a_max, (vec4_t<T> *)c.xq.p), "newton");
            CK(build_candidates<T>(c, (const vec4_t<T> *)c.xp.p, (const vec4_t<T> *)c.xq.p, c.sweep_cand, &ns,
                                   cand_cap(c), true), "newton: sweep");
            if (ns <= cand_cap(c)) break;
            if (tries >= 12)
                return set_err(c, TTIE_ERR_CAPACITY, "ttie_newton_step: swept candidates %lld exceed max_candidates",
                               (long long)ns);
            a_max *= 0.5;
        }
    }
    s = read_err(c, "ttie_newton_step");
    if (s != TTIE_OK) return s;
    inf.n_candidates_swept = ns;
    double alpha = 0.0, E_new = E;
    int64_t n_new = c.n_active;
    int trials = 0;
    bool accepted = false;
    for (int k = -1; k <= c.prm.ls_max_halvings; ++k) {
        const double a = k < 0 ? a_max : std::ldexp(1.0, -k);
        if (k < 0 && !(a_max > 1.0)) continue;
        if (a > a_max) continue;   // beyond the swept range
        CK(axpy_positions<T>(c, (const vec4_t<T> *)c.xp.p, (const T *)c.dir.p, (T)a, (vec4_t<T> *)c.xt.p), "newton");
        double Et = 0.0;
        int64_t nt = 0;
        s = energy_at<T>(c, (const vec4_t<T> *)c.xt.p, (const int2 *)c.sweep_cand.p, ns, &Et, &nt);
        if (s != TTIE_OK) return s;
        ++trials;
        const bool armijo = Et <= E + c.prm.armijo_c * a * gd;
        const bool fewer = nt < c.n_active && Et <= E;
        const bool ok = nt == 0 || armijo || (c.prm.ls_rule == TTIE_LS_FEWER && fewer);
        alpha = a;   // the last (smallest) trial is taken when none is accepted
        E_new = Et;
        n_new = nt;
        if (ok) {
            accepted = true;
            break;
        }
    }
    // adaptive overshoot: the overshoot trial taken without lowering the count (the pairs
    // approach touching without crossing, e.g. held back by the regulariser or an elastic
    // term) doubles eta for the next step; a lower count resets it
    if (c.prm.ls_rule == TTIE_LS_FEWER) {
        if (n_new < c.n_active) c.eta_cur = c.prm.push_eta;
        else if (accepted && alpha == a_top && a_top > 1.0)
            c.eta_cur = std::min(std::max(c.prm.push_eta_max, c.prm.push_eta), 2.0 * c.eta_cur);
    }
    CK(update_positions<T>(c, x, c.x_stride, (const T *)c.dir.p, (T)alpha), "newton: update");
    c.have_eval = false;   // the last evaluation ran on the line-search candidates
    mark(c, 5);
    CK(cudaStreamSynchronize(c.stream), "newton");
    inf.alpha = alpha;
    inf.energy_new = E_new;
    inf.n_active_new = n_new;
    inf.ls_trials = trials;
    inf.ms_build = ms_between(c, 0, 1);
    inf.ms_eval = ms_between(c, 1, 2);
    inf.ms_assemble = ms_between(c, 2, 3);
    inf.ms_pcg = ms_between(c, 3, 4);
    inf.ms_line_search = ms_between(c, 4, 5);
    inf.ms_classify = c.n_cand > 0 ? ms_between(c, 6, 7) : 0.f;
    inf.ms_pcg_kernel = ms_between(c, 8, 9);
    stage_info(c, inf, false);
    if (info) *info = inf;
    return TTIE_OK;
}

// One Newton step of every instance at once, each instance on its own (instances.cu): per-
// instance PCG in one launch, per-instance step cap and line search over a shared ladder of
// trial steps.
template <typename T>
static ttie_status newton_batched(Ctx &c, T *x, ttie_step_info *info) {
    ttie_step_info inf;
    std::memset(&inf, 0, sizeof inf);
    c.have_dir = false;
    mark(c, 0);
    CK(pack_positions<T>(c, x, c.x_stride, (vec4_t<T> *)c.xp.p), "newton: positions");
    ttie_status s = read_err(c, "ttie_newton_step");
    if (s != TTIE_OK) return s;
    int64_t n = 0;
    CK(build_candidates<T>(c, (const vec4_t<T> *)c.xp.p, nullptr, c.cand, &n, cand_cap(c)), "newton: LBVH");
    if (n > cand_cap(c)) {
        c.have_cand = false;
        return set_err(c, TTIE_ERR_CAPACITY, "ttie_newton_step: %lld candidate pairs exceed max_candidates %lld",
                       (long long)n, (long long)cand_cap(c));
    }
    c.n_cand = n;
    c.have_cand = true;
    inf.n_candidates = n;
    mark(c, 1);
    c.time_kernels = c.prm.profile != 0;
    CK(eval_candidates<T>(c, (const vec4_t<T> *)c.xp.p, (const int2 *)c.cand.p, n, TTIE_EVAL_E | TTIE_EVAL_H), "newton: eval");
    c.time_kernels = false;
    c.have_eval = true;
    c.eval_what = TTIE_EVAL_E | TTIE_EVAL_H;
    CK(cudaMemcpyAsync(&c.hs->energy, &c.ds->energy, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "newton");
    CK(cudaStreamSynchronize(c.stream), "newton");
    const double E = c.hs->energy;
    inf.energy = E;
    inf.n_active = c.n_active;
    mark(c, 2);
    if (!std::isfinite(E)) return set_err(c, TTIE_ERR_NONFINITE, "ttie_newton_step: energy is not finite");
    if (c.n_active == 0) {
        inf.energy_new = E;
        mark(c, 3); mark(c, 4); mark(c, 5);
        if (c.prm.profile) cudaEventSynchronize(c.ev[5]);
        inf.ms_build = ms_between(c, 0, 1);
        inf.ms_eval = ms_between(c, 1, 2);
        inf.ms_classify = c.n_cand > 0 ? ms_between(c, 6, 7) : 0.f;
        stage_info(c, inf, true);
        if (info) *info = inf;
        return TTIE_OK;
    }
    // assembly, instance layout and energies at x, per-instance PCG for (H+_i + mu_i I) d_i = -g_i
    CK(assemble_system<T>(c, nullptr), "newton: assembly");
    c.have_bsr = true;
    inf.n_rows = c.n_rows;
    inf.nnzb = c.nnzb;
    CK(instance_layout(c), "newton: instances");
    CK(instance_energies<T>(c, (const int2 *)c.cand.p, 0), "newton: instances");
    mark(c, 3);
    const int64_t n3 = c.n_rows * 3;
    CK(ensure(c, c.pcg_x, (size_t)(n3 > 0 ? n3 : 1) * sizeof(T)), "newton");
    CK(ensure(c, c.xsave, (size_t)(n3 > 0 ? n3 : 1) * sizeof(T)), "newton");
    CK(negate_copy(c, (const T *)c.rhs.p, (T *)c.xsave.p, n3), "newton");
    CK(instance_pcg<T>(c, (const T *)c.xsave.p, (T *)c.pcg_x.p), "newton: PCG");
    s = read_err(c, "ttie_newton_step");
    if (s != TTIE_OK) return s;
    CK(ensure(c, c.dir, (size_t)c.V * 3 * sizeof(T)), "newton");
    CK(scatter_direction<T>(c, (const T *)c.pcg_x.p, (T *)c.dir.p), "newton");
    c.have_dir = true;
    mark(c, 4);
    // line search: candidates from the boxes swept to the largest trial step (tree of x refitted)
    double a_max = 1.0 + c.prm.push_eta;
    CK(ensure(c, c.xq, (size_t)c.V * sizeof(vec4_t<T>)), "newton");
    CK(ensure(c, c.xt, (size_t)c.V * sizeof(vec4_t<T>)), "newton");
    int64_t ns = 0;
    for (int tries = 0;; ++tries) {
        CK(axpy_positions<T>(c, (const vec4_t<T> *)c.xp.p, (const T *)c.dir.p, (T)a_max, (vec4_t<T> *)c.xq.p), "newton");
        CK(build_candidates<T>(c, (const vec4_t<T> *)c.xp.p, (const vec4_t<T> *)c.xq.p, c.sweep_cand, &ns, cand_cap(c), true),
           "newton: sweep");
        if (ns <= cand_cap(c)) break;
        if (tries >= 12)
            return set_err(c, TTIE_ERR_CAPACITY, "ttie_newton_step: swept candidates %lld exceed max_candidates",
                           (long long)ns);
        a_max *= 0.5;
    }
    inf.n_candidates_swept = ns;
    CK(instance_ls_init(c), "newton: line search");
    int trials = 0;
#ifndef TTIE_CHECKS
    // every trial (the candidates of the instances still open, trial positions, energies per
    // instance, acceptance) is one CUDA graph, captured here and replayed with the next step
    cudaGraphExec_t exec = nullptr;
    unsigned long long graph_kernels = 0;
    CK(instance_trial_graph<T>(c, (const vec4_t<T> *)c.xp.p, (const T *)c.dir.p, (vec4_t<T> *)c.xt.p,
                               (const int2 *)c.sweep_cand.p, ns, &exec, &graph_kernels), "line search: graph");
    cudaError_t ge = cudaSuccess;
    for (int k = -1; k <= c.prm.ls_max_halvings; ++k) {
        const double a = k < 0 ? a_max : std::ldexp(1.0, -k);
        if (k < 0 && !(a_max > 1.0)) continue;
        if (a > a_max) continue;   // beyond the swept range
        c.hs->ls_alpha = a;
        c.hs->ls_last = k == c.prm.ls_max_halvings ? 1.0 : 0.0;
        if ((ge = cudaGraphLaunch(exec, c.stream)) != cudaSuccess) break;
        if ((ge = cudaStreamSynchronize(c.stream)) != cudaSuccess) break;
        c.n_launch += graph_kernels;
        ++trials;
        if (c.hs->n_pending == 0) break;
    }
    cudaGraphExecDestroy(exec);
    CK(ge, "line search: graph replay");
#else
    // self-checking builds synchronise after every launch, which a capture does not allow
    const int2 *tp = (const int2 *)c.sweep_cand.p;
    int64_t tn = ns;
    for (int k = -1; k <= c.prm.ls_max_halvings; ++k) {
        const double a = k < 0 ? a_max : std::ldexp(1.0, -k);
        if (k < 0 && !(a_max > 1.0)) continue;
        if (a > a_max) continue;
        CK(axpy_positions<T>(c, (const vec4_t<T> *)c.xp.p, (const T *)c.dir.p, (T)a, (vec4_t<T> *)c.xt.p), "newton");
        CK(eval_candidates<T>(c, (const vec4_t<T> *)c.xt.p, tp, tn, TTIE_EVAL_E), "line search");
        CK(instance_energies<T>(c, tp, 1), "line search");
        CK(instance_ls_accept(c, a, k == c.prm.ls_max_halvings ? 1 : 0, &c.ds->n_pending), "line search");
        CK(cudaMemcpyAsync(&c.hs->n_pending, &c.ds->n_pending, sizeof(unsigned int), cudaMemcpyDeviceToHost, c.stream),
           "line search");
        CK(cudaStreamSynchronize(c.stream), "line search");
        ++trials;
        if (c.hs->n_pending == 0) break;
        CK(instance_pending_pairs(c, (const int2 *)c.sweep_cand.p, ns, c.ls_cand, &tn), "line search");
        tp = (const int2 *)c.ls_cand.p;
    }
#endif
    CK(instance_update<T>(c, x, c.x_stride, (const T *)c.dir.p), "newton: update");
    CK(instance_totals(c, c.ds->batch), "newton");
    c.have_eval = false;   // the last evaluation ran on the line-search candidates
    s = read_err(c, "ttie_newton_step");
    if (s != TTIE_OK) return s;
    mark(c, 5);
    CK(cudaMemcpyAsync(c.hs->batch, c.ds->batch, sizeof(c.hs->batch), cudaMemcpyDeviceToHost, c.stream), "newton");
    CK(cudaStreamSynchronize(c.stream), "newton");
    inf.energy_new = c.hs->batch[0];
    inf.n_active_new = (int64_t)c.hs->batch[1];
    inf.pcg_iters = (int)c.hs->batch[2];
    inf.pcg_rel_residual = c.hs->batch[3];
    inf.grad_dot_dir = c.hs->batch[4];
    inf.alpha = c.hs->batch[5];
    inf.pcg_block_iters = (int64_t)c.hs->batch[7];
    inf.pcg_row_iters = (int64_t)c.hs->batch[8];
    inf.ls_trials = trials;
    inf.ms_build = ms_between(c, 0, 1);
    inf.ms_eval = ms_between(c, 1, 2);
    inf.ms_assemble = ms_between(c, 2, 3);
    inf.ms_pcg = ms_between(c, 3, 4);
    inf.ms_line_search = ms_between(c, 4, 5);
    inf.ms_classify = c.n_cand > 0 ? ms_between(c, 6, 7) : 0.f;
    inf.ms_pcg_kernel = ms_between(c, 8, 9);
    stage_info(c, inf, true);
    if (info) *info = inf;
    return TTIE_OK;
}

template <typename T>
static ttie_status hvp_impl(Ctx &c, const T *x, const T *v, T *out, int exact) {
    if (!c.have_bsr) {
        CK(assemble_system<T>(c, nullptr), "ttie_hvp: assembly");
        c.have_bsr = true;
    }
    if (exact) {
        CK(pack_positions<T>(c, x, c.x_stride, (vec4_t<T> *)c.xp.p), "ttie_hvp");
        ttie_status s = read_err(c, "ttie_hvp");
        if (s != TTIE_OK) return s;
        CK(ensure(c, c.hbuf, (size_t)(c.n_active > 0 ? c.n_active : 1) * 18 * sizeof(T)), "ttie_hvp");
        CK(hvp_pairs<T>(c, (const vec4_t<T> *)c.xp.p, v, (T *)c.hbuf.p), "ttie_hvp");
        CK(vertex_sums<T>(c, (const T *)c.hbuf.p, out), "ttie_hvp");
    } else {
        CK(bsr_matvec<T>(c, v, out), "ttie_hvp");
    }
    CK(cudaStreamSynchronize(c.stream), "ttie_hvp");
    return TTIE_OK;
}

extern "C" {

ttie_status ttie_build_bvh(ttie_ctx *h, const void *d_x, int64_t V, int x_stride, const int32_t *d_tri, int64_t F,
                           const int32_t *d_group, int64_t *n_candidates) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!d_x || (!d_tri && F > 0)) return set_err(c, TTIE_ERR_INVALID, "ttie_build_bvh: null pointer");
    if (V < 1 || V > (int64_t)INT32_MAX) return set_err(c, TTIE_ERR_INVALID, "ttie_build_bvh: V out of range");
    if (F < 0 || F > (int64_t)INT32_MAX / 2) return set_err(c, TTIE_ERR_INVALID, "ttie_build_bvh: F out of range");
    if (x_stride != 3 && x_stride != 4) return set_err(c, TTIE_ERR_INVALID, "ttie_build_bvh: x_stride must be 3 or 4");
    const int mode = c.prm.pair_mode & 3;
    if (mode != TTIE_PAIRS_SELF && !d_group)
        return set_err(c, TTIE_ERR_INVALID, "ttie_build_bvh: the group pair modes need d_group");
    if (c.have_elastic && V != c.el_V) c.have_elastic = false;   // the term was set for another mesh
    c.V = V;
    c.F = F;
    c.x_stride = x_stride;
    c.have_mesh = false;
    if (c.prm.precision == TTIE_F64) return build_impl<double>(c, (const double *)d_x, d_tri, d_group, n_candidates);
    return build_impl<float>(c, (const float *)d_x, d_tri, d_group, n_candidates);
}

ttie_status ttie_eval_pairs(ttie_ctx *h, const void *d_x, unsigned what, double *energy, int64_t *n_active, void *d_grad) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_cand) return set_err(c, TTIE_ERR_STATE, "ttie_eval_pairs: call ttie_build_bvh first");
    if (!d_x) return set_err(c, TTIE_ERR_INVALID, "ttie_eval_pairs: null positions");
    if (what & ~7u) return set_err(c, TTIE_ERR_INVALID, "ttie_eval_pairs: unknown flags");
    if (d_grad && !(what & TTIE_EVAL_G)) return set_err(c, TTIE_ERR_INVALID, "ttie_eval_pairs: d_grad needs TTIE_EVAL_G");
    if (c.prm.precision == TTIE_F64)
        return eval_impl<double>(c, (const double *)d_x, what, energy, n_active, (double *)d_grad);
    return eval_impl<float>(c, (const float *)d_x, what, energy, n_active, (float *)d_grad);
}

ttie_status ttie_assemble(ttie_ctx *h, ttie_bsr_view *out) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!out) return set_err(c, TTIE_ERR_INVALID, "ttie_assemble: null output");
    if (!c.have_eval || !(c.eval_what & (TTIE_EVAL_H | TTIE_EVAL_G)))
        return set_err(c, TTIE_ERR_STATE, "ttie_assemble: needs a ttie_eval_pairs with TTIE_EVAL_H");
    if (!c.have_bsr) {
        cudaError_t e = c.prm.precision == TTIE_F64 ? assemble_system<double>(c, nullptr) : assemble_system<float>(c, nullptr);
        if (e != cudaSuccess) return cuda_err(c, e, "ttie_assemble");
        c.have_bsr = true;
    }
    CK(cudaStreamSynchronize(c.stream), "ttie_assemble");
    out->n_rows = c.n_rows;
    out->nnzb = c.nnzb;
    out->row_ptr = (const int32_t *)c.row_ptr.p;
    out->col_idx = (const int32_t *)c.col_idx.p;
    out->val = c.bsr_val.p;
    out->vertex_of_row = (const int32_t *)c.row_vertex.p;
    out->grad = c.rhs.p;
    return TTIE_OK;
}

ttie_status ttie_copy_bsr(ttie_ctx *h, int32_t *d_row_ptr, int32_t *d_col_idx, void *d_val, int32_t *d_vertex_of_row,
                         void *d_grad) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_bsr) return set_err(c, TTIE_ERR_STATE, "ttie_copy_bsr: call ttie_assemble first");
    const size_t es = c.prm.precision == TTIE_F64 ? 8 : 4;
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (d_row_ptr) CK(cudaMemcpyAsync(d_row_ptr, c.row_ptr.p, (size_t)(c.n_rows + 1) * 4, k, c.stream), "ttie_copy_bsr");
    if (d_col_idx && c.nnzb) CK(cudaMemcpyAsync(d_col_idx, c.col_idx.p, (size_t)c.nnzb * 4, k, c.stream), "ttie_copy_bsr");
    if (d_val && c.nnzb) CK(cudaMemcpyAsync(d_val, c.bsr_val.p, (size_t)c.nnzb * 9 * es, k, c.stream), "ttie_copy_bsr");
    if (d_vertex_of_row && c.n_rows)
        CK(cudaMemcpyAsync(d_vertex_of_row, c.row_vertex.p, (size_t)c.n_rows * 4, k, c.stream), "ttie_copy_bsr");
    if (d_grad && c.n_rows) CK(cudaMemcpyAsync(d_grad, c.rhs.p, (size_t)c.n_rows * 3 * es, k, c.stream), "ttie_copy_bsr");
    CK(cudaStreamSynchronize(c.stream), "ttie_copy_bsr");
    return TTIE_OK;
}

ttie_status ttie_hvp(ttie_ctx *h, const void *d_x, const void *d_v, void *d_out, int exact) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_eval || !(c.eval_what & (TTIE_EVAL_G | TTIE_EVAL_H)))
        return set_err(c, TTIE_ERR_STATE, "ttie_hvp: needs a ttie_eval_pairs with TTIE_EVAL_G or TTIE_EVAL_H");
    if (!d_v || !d_out || (exact && !d_x)) return set_err(c, TTIE_ERR_INVALID, "ttie_hvp: null pointer");
    if (c.prm.precision == TTIE_F64)
        return hvp_impl<double>(c, (const double *)d_x, (const double *)d_v, (double *)d_out, exact);
    return hvp_impl<float>(c, (const float *)d_x, (const float *)d_v, (float *)d_out, exact);
}

ttie_status ttie_dual_gradients(ttie_ctx *h, const void *d_x, double *d_out) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_eval) return set_err(c, TTIE_ERR_STATE, "ttie_dual_gradients: needs a ttie_eval_pairs");
    if (!d_x || !d_out) return set_err(c, TTIE_ERR_INVALID, "ttie_dual_gradients: null pointer");
    if (c.prm.precision == TTIE_F64) {
        CK(pack_positions<double>(c, (const double *)d_x, c.x_stride, (dvec4 *)c.xp.p), "ttie_dual_gradients");
        CK(dual_gradients<double>(c, (const dvec4 *)c.xp.p, d_out), "ttie_dual_gradients");
    } else {
        CK(pack_positions<float>(c, (const float *)d_x, c.x_stride, (float4 *)c.xp.p), "ttie_dual_gradients");
        CK(dual_gradients<float>(c, (const float4 *)c.xp.p, d_out), "ttie_dual_gradients");
    }
    CK(cudaStreamSynchronize(c.stream), "ttie_dual_gradients");
    return read_err(c, "ttie_dual_gradients");
}

ttie_status ttie_pcg(ttie_ctx *h, const void *d_rhs, void *d_out, double rtol, int max_it, int *iters, double *rel_residual) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_bsr) return set_err(c, TTIE_ERR_STATE, "ttie_pcg: call ttie_assemble first");
    if (!d_rhs || !d_out || !(rtol > 0.0) || max_it < 1) return set_err(c, TTIE_ERR_INVALID, "ttie_pcg: arguments");
    cudaError_t e = c.prm.precision == TTIE_F64
                        ? pcg_solve<double>(c, (const double *)d_rhs, (double *)d_out, rtol, max_it)
                        : pcg_solve<float>(c, (const float *)d_rhs, (float *)d_out, rtol, max_it);
    if (e != cudaSuccess) return cuda_err(c, e, "ttie_pcg");
    ttie_status st = read_err(c, "ttie_pcg");
    if (st != TTIE_OK) return st;
    CK(cudaMemcpyAsync(c.hs, c.ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.stream), "ttie_pcg");
    CK(cudaStreamSynchronize(c.stream), "ttie_pcg");
    if (iters) *iters = c.hs->pcg_iters;
    const double rel = c.hs->red[1] > 0.0 ? std::sqrt(c.hs->red[4] / c.hs->red[1]) : 0.0;
    if (rel_residual) *rel_residual = rel;
    if (!std::isfinite(rel)) return set_err(c, TTIE_ERR_NONFINITE, "ttie_pcg: residual is not finite");
    return TTIE_OK;
}

ttie_status ttie_set_elastic(ttie_ctx *h, const ttie_elastic *el) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_mesh) return set_err(c, TTIE_ERR_STATE, "ttie_set_elastic: call ttie_build_bvh first");
    if (!el || (el->n_edges == 0 && el->n_anchors == 0)) {
        c.have_elastic = false;
        return TTIE_OK;
    }
    if (el->n_edges < 0 || el->n_anchors < 0 || el->n_edges > (int64_t)INT32_MAX || el->n_anchors > (int64_t)INT32_MAX)
        return set_err(c, TTIE_ERR_INVALID, "ttie_set_elastic: counts out of range");
    if (!(el->k_edge >= 0.0) || !(el->k_anchor >= 0.0) || !std::isfinite(el->k_edge) || !std::isfinite(el->k_anchor))
        return set_err(c, TTIE_ERR_INVALID, "ttie_set_elastic: stiffness must be finite and >= 0");
    if ((el->n_edges > 0 && (!el->edges || !el->rest)) || (el->n_anchors > 0 && (!el->anchors || !el->targets)))
        return set_err(c, TTIE_ERR_INVALID, "ttie_set_elastic: null array");
    if (batched(c))
        return set_err(c, TTIE_ERR_INVALID, "ttie_set_elastic: the elastic term is not available with batched instances");
    c.have_elastic = false;
    CK(c.prm.precision == TTIE_F64 ? elastic_set<double>(c, el) : elastic_set<float>(c, el), "ttie_set_elastic");
    ttie_status s = read_err(c, "ttie_set_elastic");
    if (s != TTIE_OK) return s;
    c.el_n_edges = el->n_edges;
    c.el_n_anchors = el->n_anchors;
    c.el_k = el->k_edge;
    c.el_ka = el->k_anchor;
    c.el_V = c.V;
    c.el_prec = c.prm.precision;
    c.have_elastic = true;
    return TTIE_OK;
}

ttie_status ttie_newton_step(ttie_ctx *h, void *d_x_inout, ttie_step_info *info) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_mesh) return set_err(c, TTIE_ERR_STATE, "ttie_newton_step: call ttie_build_bvh first");
    if (!d_x_inout) return set_err(c, TTIE_ERR_INVALID, "ttie_newton_step: null positions");
    if (c.prm.precision == TTIE_F64) return newton_impl<double>(c, (double *)d_x_inout, info);
    return newton_impl<float>(c, (float *)d_x_inout, info);
}

ttie_status ttie_solve(ttie_ctx *h, void *d_x_inout, ttie_solve_info *info) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_mesh) return set_err(c, TTIE_ERR_STATE, "ttie_solve: call ttie_build_bvh first");
    if (!d_x_inout) return set_err(c, TTIE_ERR_INVALID, "ttie_solve: null positions");
    ttie_solve_info inf;
    std::memset(&inf, 0, sizeof inf);
    const auto t0 = std::chrono::steady_clock::now();
    ttie_status s = TTIE_OK;
    int it = 0;
    c.eta_cur = c.prm.push_eta;
    for (;; ++it) {
        ttie_step_info st;
        s = ttie_newton_step(h, d_x_inout, &st);
        if (s != TTIE_OK) break;
        if (it == 0) {
            inf.energy_initial = st.energy;
            inf.n_active_initial = st.n_active;
        }
        inf.energy_final = st.energy;
        inf.n_active_final = st.n_active;
        if (st.n_active == 0) {
            inf.converged = 1;
            break;
        }
        if (it >= c.prm.newton_max_it) {
            s = set_err(c, TTIE_ERR_NOT_CONVERGED, "ttie_solve: %d iterations, %lld pairs still intersect", it,
                        (long long)st.n_active);
            break;
        }
    }
    inf.iterations = it;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return s;
}

ttie_status ttie_get_candidates(ttie_ctx *h, int32_t *d_out, int64_t capacity, int64_t *n) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_cand) return set_err(c, TTIE_ERR_STATE, "ttie_get_candidates: no candidates");
    if (n) *n = c.n_cand;
    if (!d_out) return TTIE_OK;
    if (capacity < c.n_cand) return set_err(c, TTIE_ERR_INVALID, "ttie_get_candidates: capacity %lld < %lld",
                                            (long long)capacity, (long long)c.n_cand);
    if (c.n_cand) CK(cudaMemcpyAsync(d_out, c.cand.p, (size_t)c.n_cand * sizeof(int2), cudaMemcpyDeviceToDevice, c.stream), "get");
    CK(cudaStreamSynchronize(c.stream), "ttie_get_candidates");
    return TTIE_OK;
}

ttie_status ttie_get_active(ttie_ctx *h, int32_t *d_pairs, void *d_tc, void *d_dtc, int64_t capacity, int64_t *n) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_eval) return set_err(c, TTIE_ERR_STATE, "ttie_get_active: no evaluation");
    if (n) *n = c.n_active;
    if (!d_pairs && !d_tc && !d_dtc) return TTIE_OK;
    if (capacity < c.n_active) return set_err(c, TTIE_ERR_INVALID, "ttie_get_active: capacity too small");
    if ((d_tc || d_dtc) && !(c.eval_what & (TTIE_EVAL_G | TTIE_EVAL_H)))
        return set_err(c, TTIE_ERR_STATE, "ttie_get_active: t_c and gradients need TTIE_EVAL_G or TTIE_EVAL_H");
    const int64_t na = c.n_active;
    if (na > 0) {
        if (d_pairs)
            launch(c, k_gather_active, dim3(grid_for(na, kThreads)), dim3(kThreads), (const int2 *)c.cand.p,
                                                                              (const uint32_t *)c.active.p, na,
                                                                              (int2 *)d_pairs);
        if (d_tc || d_dtc) {
            if (c.prm.precision == TTIE_F64)
                launch(c, k_split_fac<double>, dim3(grid_for(na, kThreads)), dim3(kThreads), (const double *)c.fac.p, na,
                                                                                      (double *)d_tc, (double *)d_dtc);
            else
                launch(c, k_split_fac<float>, dim3(grid_for(na, kThreads)), dim3(kThreads), (const float *)c.fac.p, na,
                                                                                     (float *)d_tc, (float *)d_dtc);
        }
        CK(cudaGetLastError(), "ttie_get_active");
    }
    CK(cudaStreamSynchronize(c.stream), "ttie_get_active");
    return TTIE_OK;
}

ttie_status ttie_get_direction(ttie_ctx *h, void *d_out) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!c.have_dir) return set_err(c, TTIE_ERR_STATE, "ttie_get_direction: no Newton direction");
    if (!d_out) return set_err(c, TTIE_ERR_INVALID, "ttie_get_direction: null output");
    const size_t es = c.prm.precision == TTIE_F64 ? 8 : 4;
    CK(cudaMemcpyAsync(d_out, c.dir.p, (size_t)c.V * 3 * es, cudaMemcpyDeviceToDevice, c.stream), "ttie_get_direction");
    CK(cudaStreamSynchronize(c.stream), "ttie_get_direction");
    return TTIE_OK;
}

void ttie_struct_sizes(int64_t *out5) {
    if (!out5) return;
    out5[0] = (int64_t)sizeof(ttie_params);
    out5[1] = (int64_t)sizeof(ttie_bsr_view);
    out5[2] = (int64_t)sizeof(ttie_step_info);
    out5[3] = (int64_t)sizeof(ttie_elastic);
    out5[4] = (int64_t)sizeof(ttie_solve_info);
}

ttie_status ttie_get_filter_stats(ttie_ctx *h, int64_t *out3) {
    if (!h) return TTIE_ERR_INVALID;
    Ctx &c = h->c;
    if (!out3) return set_err(c, TTIE_ERR_INVALID, "ttie_get_filter_stats: null output");
    CK(cudaMemcpyAsync(c.hs->filter_stats, c.ds->filter_stats, 3 * 8, cudaMemcpyDeviceToHost, c.stream), "stats");
    CK(cudaStreamSynchronize(c.stream), "stats");
    for (int i = 0; i < 3; ++i) out3[i] = (int64_t)c.hs->filter_stats[i];
    return TTIE_OK;
}

ttie_status ttie_get_launch_count(ttie_ctx *h, int64_t *n) {
    if (!h || !n) return TTIE_ERR_INVALID;
    *n = (int64_t)h->c.n_launch;
    return TTIE_OK;
}

}  // extern "C"
