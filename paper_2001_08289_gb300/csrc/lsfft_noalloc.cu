// Volume averages of a field without any device allocation.
//
// Some callers cannot call cudaMalloc: code that must not block (cudaMalloc and
// cudaFree may synchronise the device), code whose device memory belongs to
// another allocator under a fixed budget (a framework's caching allocator),
// and code that runs where allocation is not permitted.  For them this entry
// point recomputes the volume averages that lsfft_solve reports (<E>, <J> with
// J = sigma E, <|E|^2> and sigma_* = <J>.e / <E>.e) for a field and mask the
// caller already holds, keeping its block partial sums in a file-scope
// __device__ array instead of allocated scratch.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "lsfft.h"
#include "lsfft_fft.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_CHUNK = 65536;          // voxels per partial sum
constexpr int NA_MAX_PARTIALS = 4096;        // so at most 268,435,456 voxels per call
constexpr int NA_NV = 16;                    // slots per partial (4 d + 1 <= 13 used)

// Shared by every call on a device and kept until the process exits (512 KiB).
// Host code must not use this name as an address: the device address comes
// from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_PARTIALS * NA_NV];

thread_local std::string g_noalloc_error;

template <typename T>
__global__ void __launch_bounds__(NA_THREADS)
noalloc_partials(const lsfft::cx<T>* __restrict__ E, const uint8_t* __restrict__ mask, int d, int64_t N,
                 double s1re, double s1im, double* __restrict__ scratch) {
    const int64_t begin = blockIdx.x * NA_CHUNK;
    const int64_t end = begin + NA_CHUNK < N ? begin + NA_CHUNK : N;
    double acc[13];
#pragma unroll
    for (int v = 0; v < 13; ++v) acc[v] = 0.0;
    for (int64_t i = begin + threadIdx.x; i < end; i += NA_THREADS) {
        const bool inc = mask[i] != 0;
        for (int c = 0; c < d; ++c) {
            const double er = (double)E[c * N + i].x, ei = (double)E[c * N + i].y;
            const double jr = inc ? s1re * er - s1im * ei : er;
            const double ji = inc ? s1re * ei + s1im * er : ei;
            acc[4 * c + 0] += er;
            acc[4 * c + 1] += ei;
            acc[4 * c + 2] += jr;
            acc[4 * c + 3] += ji;
            acc[12] += er * er + ei * ei;
        }
    }
    __shared__ double red[NA_THREADS / 32][13];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < 13; ++v) {
        double x = acc[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) s += red[w][threadIdx.x];
        scratch[(int64_t)blockIdx.x * NA_NV + threadIdx.x] = s;
    }
}

__global__ void noalloc_finish(const double* __restrict__ scratch, int nparts, int d, int64_t N, double e0, double e1,
                               double e2, double* __restrict__ out) {
    __shared__ double tot[13];
    if (threadIdx.x < 13) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += scratch[(int64_t)b * NA_NV + threadIdx.x];   // fixed order
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double e[3] = {e0, e1, e2};
    double ee_re = 0, ee_im = 0, je_re = 0, je_im = 0;
    for (int c = 0; c < d; ++c) {
        out[4 * c + 0] = tot[4 * c + 0] / (double)N;
        out[4 * c + 1] = tot[4 * c + 1] / (double)N;
        out[4 * c + 2] = tot[4 * c + 2] / (double)N;
        out[4 * c + 3] = tot[4 * c + 3] / (double)N;
        ee_re += tot[4 * c + 0] * e[c];
        ee_im += tot[4 * c + 1] * e[c];
        je_re += tot[4 * c + 2] * e[c];
        je_im += tot[4 * c + 3] * e[c];
    }
    out[4 * d] = tot[12] / (double)N;
    // sigma_* is undefined when <E>.e vanishes: report NaN rather than divide by zero
    const double den = ee_re * ee_re + ee_im * ee_im;
    out[4 * d + 1] = den > 0.0 ? (je_re * ee_re + je_im * ee_im) / den : nan("");
    out[4 * d + 2] = den > 0.0 ? (je_im * ee_re - je_re * ee_im) / den : nan("");
}

// Device address of the scratch array on the current device.  It is looked
// up on every call (the lookup allocates nothing and is cheap), so that an
// address never outlives a device reset or a rebuilt primary context.
int scratch_on_current_device(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        g_noalloc_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return LSFFT_ECUDA;
    }
    *out = static_cast<double*>(p);
    return LSFFT_OK;
}

// Launch check that leaves the thread's error state alone: an error pending from
// earlier work is reported as such, not as this call's, and the caller's own
// cudaGetLastError still sees it.
int check_launch(const char* what) {
    const cudaError_t e = cudaPeekAtLastError();
    if (e == cudaSuccess) return LSFFT_OK;
    g_noalloc_error = std::string("CUDA error after launching ") + what +
                      " (it may stem from earlier work on this thread): " + cudaGetErrorString(e);
    return LSFFT_ECUDA;
}

}  // namespace

extern "C" {

const char* lsfft_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

int lsfft_field_averages_noalloc(int d, const int64_t n[3], const void* E_device, int precision,
                                 const uint8_t* mask_device, lsfft_c128 sigma1, const double* e,
                                 double* out_device, void* cuda_stream) {
    if (!n || !E_device || !mask_device || !e || !out_device || (d != 2 && d != 3) ||
        (precision != LSFFT_FP32 && precision != LSFFT_FP64)) {
        g_noalloc_error = "null pointer, d not in {2, 3} or unknown precision";
        return LSFFT_EINVAL;
    }
    double e2 = 0.0;
    for (int c = 0; c < d; ++c) e2 += e[c] * e[c];
    if (!(e2 > 0.0) || !std::isfinite(e2)) {
        g_noalloc_error = "the applied field e must be finite and non-zero";
        return LSFFT_EINVAL;
    }
    int64_t N = 1;
    for (int a = 0; a < d; ++a) {
        if (n[a] < 1) {
            g_noalloc_error = "every n[a] must be >= 1";
            return LSFFT_EINVAL;
        }
        N *= n[a];
    }
    if (N > (int64_t)NA_MAX_PARTIALS * NA_CHUNK) {
        g_noalloc_error = "field larger than the no-allocation limit of 268435456 voxels (4096 partial sums of 65536)";
        return LSFFT_EINVAL;
    }
    double* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != LSFFT_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nparts = (int)((N + NA_CHUNK - 1) / NA_CHUNK);
    if (precision == LSFFT_FP32)
        noalloc_partials<float><<<nparts, NA_THREADS, 0, s>>>((const float2*)E_device, mask_device, d, N, sigma1.re,
                                                              sigma1.im, scratch);
    else
        noalloc_partials<double><<<nparts, NA_THREADS, 0, s>>>((const double2*)E_device, mask_device, d, N, sigma1.re,
                                                               sigma1.im, scratch);
    rc = check_launch("the partial-sum kernel");
    if (rc != LSFFT_OK) return rc;
    noalloc_finish<<<1, 32, 0, s>>>(scratch, nparts, d, N, e[0], e[1], d > 2 ? e[2] : 0.0, out_device);
    rc = check_launch("the final-sum kernel");
    if (rc != LSFFT_OK) return rc;
    return LSFFT_OK;
}

}  // extern "C"
