// y = A x and x^T A x without a handle and without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while the CUDA caching
// allocator of a host framework owns all device memory, an embedded or
// real-time host whose memory budget is fixed at start-up, or a kernel
// library called from inside another library's critical section.  For them
// this entry point takes every input and output from the caller and keeps
// its only scratch -- the per-block partial sums and the ticket counter of
// the deterministic reduction -- in one file-scope static device array,
// which every GPU that loads this library holds until the process exits.
//
// The arithmetic is that of the library's thread-per-row FP64 CSR SpMV with
// the fused p^T A p of the CG recurrence: y[g] = sum_e val[e] x[col[e]] in
// column order, and the reduction sums one partial per block in block order,
// so the result is deterministic.  The paper has no counterpart of this call.
#include <mutex>

#include "ddg_internal.cuh"
#include "dev_common.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = DDG_NOALLOC_MAX_ROWS / NA_THREADS;   // 4096
constexpr size_t NA_SCRATCH_BYTES = NA_MAX_BLOCKS * sizeof(double) + 256;

// partial sums at offset 0 (one double per block), ticket counter at the end
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

__global__ void __launch_bounds__(NA_THREADS) spmv_dot_noalloc_kernel(
    int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
    double* __restrict__ xAx, double* partials, unsigned* ticket) {
    __shared__ double sh[NA_THREADS / 32];
    __shared__ bool last;
    const int64_t g = (int64_t)blockIdx.x * NA_THREADS + threadIdx.x;
    double acc = 0.0;
    if (g < n) {
        double s = 0.0;
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) s = fma(val[e], x[col[e]], s);
        y[g] = s;
        acc = x[g] * s;
    }
    const double bs = ddgdev::block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += NA_THREADS) s += __ldcg(partials + b);
    const double tot = ddgdev::block_sum(s, sh);
    if (threadIdx.x == 0) {
        *xAx = tot;
        *ticket = 0u;
    }
}

// Device addresses of the scratch array, looked up once per device with
// that device current (a host-side reference to the array is only a
// stand-in for it, not a device address).
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

}  // namespace

extern "C" ddg_status ddg_spmv_dot_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                                           const double* val, const double* x, double* y,
                                           double* xAx, void* stream) {
    if (n < 0 || n > DDG_NOALLOC_MAX_ROWS) {
        ddg::set_handleless_error(
            "ddg_spmv_dot_noalloc: n must be in [0, DDG_NOALLOC_MAX_ROWS = 1048576]");
        return DDG_EINVAL;
    }
    if (!xAx || (n > 0 && (!rowptr || !col || !val || !x || !y))) {
        ddg::set_handleless_error("ddg_spmv_dot_noalloc: null pointer");
        return DDG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        ddg::set_handleless_error("ddg_spmv_dot_noalloc: no usable current device");
        return DDG_ECUDA;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            e = cudaGetSymbolAddress((void**)&base, g_noalloc_scratch);
            if (e != cudaSuccess) {
                ddg::set_handleless_error(cudaGetErrorString(e));
                return DDG_ECUDA;
            }
            g_na_ptr[dev] = base;
        }
        base = g_na_ptr[dev];
    }
    double* partials = reinterpret_cast<double*>(base);
    unsigned* ticket = reinterpret_cast<unsigned*>(base + NA_MAX_BLOCKS * sizeof(double));
    // the ticket must start at zero; a previous call that failed part-way
    // may have left it elsewhere
    e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && n == 0) e = cudaMemsetAsync(xAx, 0, sizeof(double), s);
    if (e == cudaSuccess && n > 0) {
        const unsigned blocks = (unsigned)((n + NA_THREADS - 1) / NA_THREADS);
        spmv_dot_noalloc_kernel<<<blocks, NA_THREADS, 0, s>>>(n, rowptr, col, val, x, y, xAx,
                                                              partials, ticket);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        ddg::set_handleless_error(cudaGetErrorString(e));
        return DDG_ECUDA;
    }
    return DDG_OK;
}
