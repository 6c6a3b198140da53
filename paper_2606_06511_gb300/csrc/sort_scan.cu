// Exclusive scan and stable LSD radix sort.
//
// Both are tile-based three-kernel schemes (per-tile reduction, one-block scan of
// the tile totals, per-tile rescan / scatter).  They need no inter-block waiting,
// so every launch is independent and deterministic.
#include "common.cuh"

namespace ttie {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // 2048 elements per tile
constexpr int kWarps = kThreads / 32;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Exclusive block scan of one value per thread (up to 32 warps); returns the block total
// in *total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total) {
    __shared__ T warp_tot[32];
    __shared__ T block_tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = lane < nw ? warp_tot[lane] : T(0);
        T ti = warp_inclusive_scan(t);
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) block_tot = ti;
    }
    __syncthreads();
    T res = warp_tot[w] + inc - v;
    *total = block_tot;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kThreads) k_tile_sums(const uint32_t *__restrict__ in, int64_t n,
                                                        unsigned long long *__restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    unsigned long long tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// One block: exclusive scan of the tile totals in place; total into ts[n_tiles].
__global__ void __launch_bounds__(1024) k_scan_tile_sums(unsigned long long *ts, int64_t n_tiles) {
    unsigned long long carry = 0;
    for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        unsigned long long v = i < n_tiles ? ts[i] : 0ull, tot;
        unsigned long long ex = block_exclusive_scan(v, &tot);
        if (i < n_tiles) ts[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) ts[n_tiles] = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_tiles(const uint32_t *__restrict__ in, int64_t n,
                                                         const unsigned long long *__restrict__ tile_off,
                                                         int64_t n_tiles, unsigned long long *__restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;  // blocked
    uint32_t v[kItems];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    unsigned long long tot;
    unsigned long long run = tile_off[blockIdx.x] + block_exclusive_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_off[n_tiles];
}

// ---------------------------------------------------------------- radix sort
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

__global__ void __launch_bounds__(kThreads) k_radix_hist(const unsigned long long *__restrict__ keys, int64_t n,
                                                         int shift, int64_t n_tiles, uint32_t *__restrict__ cnt) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    cnt[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];   // digit-major
}

// Stable scatter.  Warp w of tile t owns elements [t*kTile + w*32*kItems, +32*kItems) and
// walks them in rounds of 32 in order, so (warp, round, lane) order is input order.  The tile
// is first reordered by digit in shared memory (same stable order), then written out in that
// order, so consecutive threads write consecutive positions of one digit's run instead of
// scattering every element to a different bucket.
__global__ void __launch_bounds__(kThreads) k_radix_scatter(
    const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
    unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
    int64_t n_tiles, const unsigned long long *__restrict__ off) {
    __shared__ uint32_t wh[kWarps][kRadix];
    __shared__ uint32_t dbase[kRadix];            // start of each digit in the reordered tile
    __shared__ unsigned long long s_key[kTile];
    __shared__ uint32_t s_val[kTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wh[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * kTile;
    const int64_t wbase = tbase + (int64_t)w * 32 * kItems;
    unsigned long long key[kItems];
    uint32_t val[kItems], rank[kItems];
    int dig[kItems];
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = wbase + r * 32 + lane;
        bool ok = i < n;
        key[r] = ok ? kin[i] : 0ull;
        val[r] = ok ? vin[i] : 0u;
        int d = ok ? (int)((key[r] >> shift) & (kRadix - 1)) : kRadix;   // kRadix = invalid
        dig[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = (d < kRadix) ? wh[w][d] : 0u;
        rank[r] = before + __popc(peers & lt_mask);
        __syncwarp();
        if (d < kRadix && (peers & lt_mask) == 0) wh[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps per digit, then over digits of the tile's counts
    {
        const int d = threadIdx.x;   // kThreads == kRadix
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            uint32_t t = wh[ww][d];
            wh[ww][d] = run;
            run += t;
        }
        uint32_t tot;
        dbase[d] = block_exclusive_scan(run, &tot);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int d = dig[r];
        if (d < kRadix) {
            const uint32_t lp = dbase[d] + wh[w][d] + rank[r];
            s_key[lp] = key[r];
            s_val[lp] = val[r];
        }
    }
    __syncthreads();
    const int n_valid = (int)min((int64_t)kTile, n - tbase);
    for (int i = threadIdx.x; i < n_valid; i += kThreads) {
        const unsigned long long k = s_key[i];
        const int d = (int)((k >> shift) & (kRadix - 1));
        const unsigned long long pos = off[(int64_t)d * n_tiles + blockIdx.x] + (uint32_t)(i - dbase[d]);
        kout[pos] = k;
        vout[pos] = s_val[i];
    }
}

}  // namespace

cudaError_t scan_u32_u64(Ctx &c, const uint32_t *in, unsigned long long *out, int64_t n) {
    int64_t n_tiles = (n + kTile - 1) / kTile;
    if (n_tiles < 1) n_tiles = 1;
    TTIE_CUDA_TRY(ensure(c, c.scan_tmp, (size_t)(n_tiles + 1) * sizeof(unsigned long long)));
    auto *ts = (unsigned long long *)c.scan_tmp.p;
    launch(c, k_tile_sums, dim3((unsigned)n_tiles), dim3(kThreads), in, n, ts);
    launch(c, k_scan_tile_sums, dim3(1), dim3(1024), ts, n_tiles);
    launch(c, k_scan_tiles, dim3((unsigned)n_tiles), dim3(kThreads), in, n, ts, n_tiles, out);
    return cudaGetLastError();
}

cudaError_t radix_sort(Ctx &c, unsigned long long *keys, uint32_t *vals, unsigned long long *keys2, uint32_t *vals2,
                       int64_t n, int bits, bool *in_second) {
    if (in_second) *in_second = false;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    const int64_t n_cnt = n_tiles * kRadix;
    TTIE_CUDA_TRY(ensure(c, c.sort_cnt, (size_t)n_cnt * sizeof(uint32_t) + (size_t)(n_cnt + 1) * sizeof(unsigned long long)));
    auto *cnt = (uint32_t *)c.sort_cnt.p;
    auto *off = (unsigned long long *)((char *)c.sort_cnt.p + ((n_cnt * sizeof(uint32_t) + 15) / 16) * 16);
    unsigned long long *ka = keys, *kb = keys2;
    uint32_t *va = vals, *vb = vals2;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += kRadixBits, ++passes) {
        launch(c, k_radix_hist, dim3((unsigned)n_tiles), dim3(kThreads), ka, n, shift, n_tiles, cnt);
        TTIE_CUDA_TRY(scan_u32_u64(c, cnt, off, n_cnt));
        launch(c, k_radix_scatter, dim3((unsigned)n_tiles), dim3(kThreads), ka, va, kb, vb, n, shift, n_tiles, off);
        TTIE_CUDA_TRY(cudaGetLastError());
        unsigned long long *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if ((passes & 1) && in_second) {
        *in_second = true;   // the caller takes the result from keys2 / vals2
    } else if (passes & 1) {
        TTIE_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, c.stream));
        TTIE_CUDA_TRY(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c.stream));
    }
    return cudaSuccess;
}

}  // namespace ttie

namespace ttie {

// radix_sort replayed from a graph: 5 launches per 8-bit pass (63-bit Morton keys: 40) become one
// graph launch.  Captured on the context's capture stream on the first call, and again whenever
// an argument or a scratch buffer changes (the graph holds their addresses); every buffer is
// sized before the capture, so nothing is allocated inside it.
cudaError_t radix_sort_graph(Ctx &c, unsigned long long *keys, uint32_t *vals, unsigned long long *keys2,
                             uint32_t *vals2, int64_t n, int bits) {
#ifdef TTIE_CHECKS
    return radix_sort(c, keys, vals, keys2, vals2, n, bits);   // checked builds synchronise after every launch
#endif
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    const int64_t n_cnt = n_tiles * kRadix;
    TTIE_CUDA_TRY(ensure(c, c.sort_cnt, (size_t)n_cnt * sizeof(uint32_t) + (size_t)(n_cnt + 1) * sizeof(unsigned long long)));
    TTIE_CUDA_TRY(ensure(c, c.scan_tmp, (size_t)((n_cnt + kTile - 1) / kTile + 1) * sizeof(unsigned long long)));
    const void *key[6] = {keys, vals, keys2, vals2, c.sort_cnt.p, c.scan_tmp.p};
    bool same = c.sort_exec && c.sort_n == n && c.sort_bits == bits;
    for (int i = 0; i < 6; ++i) same = same && c.sort_key[i] == key[i];
    if (!same) {
        if (c.sort_exec) {
            cudaGraphExecDestroy(c.sort_exec);
            c.sort_exec = nullptr;
        }
        if (!c.cap_stream) TTIE_CUDA_TRY(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
        const cudaStream_t main_stream = c.stream;
        c.stream = c.cap_stream;
        cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c.stream = main_stream;
            return e;
        }
        const unsigned long long launches0 = c.n_launch;
        e = radix_sort(c, keys, vals, keys2, vals2, n, bits);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c.stream, &graph);
        c.stream = main_stream;
        c.sort_kernels = c.n_launch - launches0;
        c.n_launch = launches0;   // captured, not launched: every replay counts them
        if (e == cudaSuccess) e = ec;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c.sort_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c.sort_exec = nullptr;
            return e;
        }
        for (int i = 0; i < 6; ++i) c.sort_key[i] = key[i];
        c.sort_n = n;
        c.sort_bits = bits;
    }
    TTIE_CUDA_TRY(cudaGraphLaunch(c.sort_exec, c.stream));
    c.n_launch += c.sort_kernels;
    return cudaSuccess;
}

}  // namespace ttie
