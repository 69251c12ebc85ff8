// k_noalloc.cu -- population totals without any device allocation.
//
// Same reduction as the conservation sums of clbm_residual (sum N', sum c^1 N',
// sum c^2 N'), but over a caller-provided FP64 population array and with its
// block partials in a fixed static device array instead of a grid workspace.
// It exists for callers that must not allocate device memory: code that runs
// while a stream is being captured into a CUDA graph (cudaMalloc cannot be
// captured), and processes that work inside a fixed, pre-reserved memory
// budget where any further allocation may fail or is forbidden.
#include <cstdio>
#include <mutex>

#include "../../include/clbm.h"
#include "clbm_internal.cuh"

namespace clbm {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 8192;                  // scratch holds this many partials
constexpr long long NA_MAX_CELLS = (long long)NA_MAX_BLOCKS * NA_THREADS;

// Block partials (3 per block) followed by the 3 final sums.  Every slot a
// call reads is written earlier in the same call, so nothing needs clearing.
static __device__ __align__(256) double g_na_scratch[NA_MAX_BLOCKS * 3 + 3];

std::mutex g_na_mu;
double* g_na_ptr[64] = {nullptr};  // device address of g_na_scratch, per device
void* g_na_ctx[64] = {nullptr};    // the context that address belongs to

// The calling thread's current context (the driver's cuCtxGetCurrent, found
// through the runtime so the library needs no link to the driver library);
// nullptr when it cannot be asked.  A device reset or a new primary context
// loads the module again, and the array's address with it, so the address
// is resolved again whenever the context differs from the one it came from.
void* current_context() {
    using Fn = int (*)(void**);
    static Fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (Fn)f;
        tried = true;
    }
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

template <int Q>
__global__ void __launch_bounds__(NA_THREADS) k_totals_partial(const double* __restrict__ Np,
                                                              long long ncell,
                                                              double* __restrict__ part) {
    const long long m = (long long)blockIdx.x * NA_THREADS + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (m < ncell) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double x = Np[(long long)a * ncell + m];
            v[0] += x;
            v[1] += c1_of(a) * x;
            v[2] += c2_of(a) * x;
        }
    }
    __shared__ double sh[NA_THREADS / 32][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) x += sh[w][threadIdx.x];
        part[(size_t)blockIdx.x * 3 + threadIdx.x] = x;
    }
}

__global__ void __launch_bounds__(NA_THREADS) k_totals_final(double* __restrict__ part, int nb) {
    __shared__ double sh[NA_THREADS];
    for (int k = 0; k < 3; ++k) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nb; b += NA_THREADS) x += part[(size_t)b * 3 + k];
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)NA_MAX_BLOCKS * 3 + k] = sh[0];
        __syncthreads();
    }
}

}  // namespace
}  // namespace clbm

using namespace clbm;

extern "C" clbm_status clbm_totals_noalloc(int lattice, const double* Np, int n1, int n2,
                                           double* out, int out_is_device, void* stream) {
    if (lattice != 9 && lattice != 21) {
        set_last_error("clbm_totals_noalloc: lattice must be 9 or 21");
        return CLBM_EINVAL;
    }
    if (!Np || !out || n1 < 1 || n2 < 1) {
        set_last_error("clbm_totals_noalloc: NULL pointer or empty grid");
        return CLBM_EINVAL;
    }
    const long long ncell = (long long)n1 * n2;
    if (ncell > NA_MAX_CELLS) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "clbm_totals_noalloc: %lld cells exceed the static scratch limit of %lld cells",
                 ncell, NA_MAX_CELLS);
        set_last_error(msg);
        return CLBM_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_last_error("clbm_totals_noalloc: no current CUDA device");
        return CLBM_ECUDA;
    }
    // an error left by earlier work is not this call's: report it, untouched
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "clbm_totals_noalloc: an earlier CUDA error is pending: %s",
                 cudaGetErrorString(pending));
        set_last_error(msg);
        return CLBM_ECUDA;
    }
    double* scratch = nullptr;
    {
        // First call on a device (or in a new context of it): resolve the
        // device address of the static scratch (host code may not use the
        // symbol itself as a pointer).
        std::lock_guard<std::mutex> lk(g_na_mu);
        void* ctx = current_context();
        if (!g_na_ptr[dev] || ctx != g_na_ctx[dev] || !ctx) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
                set_last_error("clbm_totals_noalloc: cudaGetSymbolAddress failed");
                return CLBM_ECUDA;
            }
            g_na_ptr[dev] = (double*)p;
            g_na_ctx[dev] = ctx;
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((ncell + NA_THREADS - 1) / NA_THREADS);
    if (lattice == 9) k_totals_partial<9><<<nb, NA_THREADS, 0, s>>>(Np, ncell, scratch);
    else k_totals_partial<21><<<nb, NA_THREADS, 0, s>>>(Np, ncell, scratch);
    k_totals_final<<<1, NA_THREADS, 0, s>>>(scratch, nb);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("clbm_totals_noalloc: kernel launch failed");
        return CLBM_ECUDA;
    }
    const double* res = scratch + (size_t)NA_MAX_BLOCKS * 3;
    if (out_is_device) {
        if (cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            set_last_error("clbm_totals_noalloc: result copy failed");
            return CLBM_ECUDA;
        }
    } else {
        if (cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            set_last_error("clbm_totals_noalloc: result copy failed");
            return CLBM_ECUDA;
        }
    }
    return CLBM_OK;
}
