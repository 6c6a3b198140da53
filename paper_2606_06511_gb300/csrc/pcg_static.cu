// ttie_pcg_static: the block-Jacobi PCG solve for callers that cannot allocate device
// memory.  Its work vectors live in one file-scope device array of fixed size; nothing
// here allocates.
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace ttie {
// the setup and persistent PCG kernels on explicit buffers (pcg.cu)
cudaError_t pcg_run_raw(cudaStream_t stream, int num_sms, const int32_t *row_ptr, const int32_t *col_idx,
                        const float *bval, int64_t n_rows, double mu_rel, const float *rhs, float *out, float *dinv,
                        float *r, float *z, float *p, float *q, double *partials, DevScalars *ds, double rtol,
                        int max_it);
}

using namespace ttie;

namespace {

constexpr int64_t kMaxRows = TTIE_PCG_STATIC_MAX_ROWS;
constexpr size_t kPartials = (size_t)kNumSMs * 16 * 4;   // doubles, as the context's partial sums

// Layout of the static scratch (byte offsets, each 256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffState = 0;
constexpr size_t kOffPart = align256(kOffState + sizeof(DevScalars));
constexpr size_t kOffDinv = align256(kOffPart + kPartials * sizeof(double));
constexpr size_t kOffR = align256(kOffDinv + (size_t)kMaxRows * 9 * sizeof(float));
constexpr size_t kOffZ = align256(kOffR + (size_t)kMaxRows * 3 * sizeof(float));
constexpr size_t kOffP = align256(kOffZ + (size_t)kMaxRows * 3 * sizeof(float));
constexpr size_t kOffQ = align256(kOffP + (size_t)kMaxRows * 3 * sizeof(float));
constexpr size_t kScratchBytes = align256(kOffQ + (size_t)kMaxRows * 3 * sizeof(float));

// Held by every GPU that loads the library, until the process exits (about 1.4 MB).
static __device__ __align__(256) unsigned char g_pcg_scratch[kScratchBytes];

// Device address of g_pcg_scratch per device.  In host code the symbol names a host-side
// stand-in, not device memory, so the address must come from cudaGetSymbolAddress, taken
// once per device with that device current.
std::mutex g_mutex;
void *g_addr[64] = {};
int g_sms[64] = {};

cudaError_t scratch_for_current_device(unsigned char **out, int *sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_pcg_scratch);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_addr[dev] = ptr;
    }
    *out = (unsigned char *)g_addr[dev];
    *sms = g_sms[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ttie_status ttie_pcg_static(const int32_t *d_row_ptr, const int32_t *d_col_idx, const float *d_val,
                                       int64_t n_rows, double mu, const float *d_rhs, float *d_out, double rtol,
                                       int max_it, void *stream, int *iters, double *rel_residual) {
    if (!d_row_ptr || !d_col_idx || !d_val || !d_rhs || !d_out) return TTIE_ERR_INVALID;
    if (n_rows < 1 || n_rows > kMaxRows) return TTIE_ERR_INVALID;   // beyond the static scratch
    if (!(mu >= 0.0) || !(rtol > 0.0) || max_it < 1) return TTIE_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    int sms = 0;
    if (scratch_for_current_device(&base, &sms) != cudaSuccess) {
        cudaGetLastError();
        return TTIE_ERR_CUDA;
    }
    DevScalars *ds = (DevScalars *)(base + kOffState);
    // The previous call's state stays in the array: zero the counters, tickets, barrier
    // words and flags, then set the row count and the trace that gives mu (mu_rel = 1).
    DevScalars init;
    memset(&init, 0, sizeof init);
    init.n_rows = (unsigned long long)n_rows;
    init.trace = mu * 3.0 * (double)n_rows;
    cudaError_t e = cudaMemcpyAsync(ds, &init, sizeof init, cudaMemcpyHostToDevice, st);
    // the block count row_ptr[n_rows] into the low half of ds->nnzb (zeroed just above): the
    // kernels' bounds checks in self-checking builds test column positions against it
    static_assert(sizeof(int32_t) <= sizeof(init.nnzb), "nnzb holds an int32 count");
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&ds->nnzb, d_row_ptr + n_rows, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = pcg_run_raw(st, sms, d_row_ptr, d_col_idx, d_val, n_rows, 1.0, d_rhs, d_out,
                        (float *)(base + kOffDinv), (float *)(base + kOffR), (float *)(base + kOffZ),
                        (float *)(base + kOffP), (float *)(base + kOffQ), (double *)(base + kOffPart), ds, rtol,
                        max_it);
    DevScalars fin;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fin, ds, sizeof fin, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TTIE_ERR_CUDA;
    }
    if (fin.err & ERR_CHECK) return TTIE_ERR_INVALID;   // the caller's arrays failed a bounds check
    if (fin.err) return TTIE_ERR_CUDA;                  // the bounded grid-barrier wait ran out
    const double rel = fin.red[1] > 0.0 ? sqrt(fin.red[4] / fin.red[1]) : 0.0;
    if (iters) *iters = fin.pcg_iters;
    if (rel_residual) *rel_residual = rel;
    return isfinite(rel) ? TTIE_OK : TTIE_ERR_NONFINITE;
}
