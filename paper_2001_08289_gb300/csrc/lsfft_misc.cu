// Small kernels around the passes: initial state and the FP64 finalize step
// (volume averages, sigma_k of Eq. J13, stop rule), small device-to-host
// transfers, Lanczos vector operations and the gradient.
#include <math.h>

#include "lsfft_finalize.cuh"
#include "lsfft_misc.h"
#include "lsfft_pdl.cuh"
#include "lsfft_reduce.cuh"

namespace lsfft {

// Initial state.  Complex layout: Q = iq e, S = is e, T = it e (S, T on phase 1).
// Packed real layout (d = 2): one plane z = iq (e_x + i e_y), with S = i s and
// T = i tau stored as s = Im(is) (e_x + i e_y), tau = Im(it) (e_x + i e_y).
template <typename T>
__global__ void init_state_kernel(cx<T>* __restrict__ X, cx<T>* __restrict__ S, cx<T>* __restrict__ Tf,
                                  const uint8_t* __restrict__ mask, const SchemeParams P, int64_t Ntot, int d,
                                  int packed, const cx<T>* __restrict__ sigma) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Ntot; i += (int64_t)gridDim.x * blockDim.x) {
        const bool inc = mask[i] != 0;
        // (packed layout: the first row pass forms the initial Q itself)
        if (sigma) {   // per-voxel mode: MS starts from E = e, EM from P = (sigma + sigma_0) e
            const double qr = P.scheme == SCHEME_EM ? (double)sigma[i].x + P.s0[0] : 1.0;
            const double qi = P.scheme == SCHEME_EM ? (double)sigma[i].y + P.s0[1] : 0.0;
            if (!packed)
                for (int c = 0; c < d; ++c) X[c * Ntot + i] = mkc((T)(qr * P.e[c]), (T)(qi * P.e[c]));
            continue;
        }
        if (packed) {
            if (S) S[i] = inc ? mkc((T)(P.is_in[1] * P.e[0]), (T)(P.is_in[1] * P.e[1])) : mkc((T)0, (T)0);
            if (Tf) Tf[i] = inc ? mkc((T)(P.it_in[1] * P.e[0]), (T)(P.it_in[1] * P.e[1])) : mkc((T)0, (T)0);
            continue;
        }
        const double* q = inc ? P.iq_in : P.iq_out;
        for (int c = 0; c < d; ++c) {
            const double e = P.e[c];
            X[c * Ntot + i] = mkc((T)(q[0] * e), (T)(q[1] * e));
            if (S) S[c * Ntot + i] = inc ? mkc((T)(P.is_in[0] * e), (T)(P.is_in[1] * e)) : mkc((T)0, (T)0);
            if (Tf) Tf[c * Ntot + i] = inc ? mkc((T)(P.it_in[0] * e), (T)(P.it_in[1] * e)) : mkc((T)0, (T)0);
        }
    }
}

// One block after each row pass, of up to FIN_WARPS warps (one warp when the
// row pass ran at most 64 blocks): sums partials[b][v] over the row pass's
// blocks in a fixed order (lane-strided running sums, warp reduce-scatter,
// then across the warps), then thread 0 runs the scalar recurrence.  The FP64
// additions on the critical path are what this kernel costs on small grids.
// (Running it in the last block of the row pass itself, found by an atomic
// arrival count, measured slower: the row kernel lost 30 us at 8192^2 from the
// extra code alone.)
constexpr int FIN_WARPS = 8;

__global__ void __launch_bounds__(FIN_WARPS * 32)
finalize_kernel(const double* __restrict__ partials, int nblocks, int nv, const SchemeParams P,
                Ctrl* __restrict__ ctrl, double* __restrict__ hist, int final_mode) {
    constexpr int NVMAX = 16;   // nv = 4 d + 1 <= 13
    __shared__ double tot[NVMAX];
    __shared__ double red[FIN_WARPS][NVMAX];
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // the partials are read before the control block, so that both round trips
    // to memory overlap (reading them is harmless when the solve is done)
    const int done = final_mode ? 0 : ctrl->done;
    double x[NVMAX];
#pragma unroll
    for (int v = 0; v < NVMAX; ++v) x[v] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double* pb = partials + (int64_t)b * nv;
#pragma unroll
        for (int v = 0; v < NVMAX; ++v)
            if (v < nv) x[v] += pb[v];
    }
    if (done) {
        if (threadIdx.x == 0) ctrl->skipB = 1;
        return;
    }
    int idx;
    const double s = warp_sum_scatter<NVMAX>(x, idx);   // lane pairs share an index
    if (nw == 1) {   // one warp (row passes of at most 64 blocks): its sums are the totals
        if ((lane & 1) == 0) tot[idx] = s;
        __syncwarp();
        if (lane == 0) finalize_update(tot, P, ctrl, hist, final_mode);
        return;
    }
    if ((lane & 1) == 0) red[warp][idx] = s;
    __syncthreads();
    if (warp == 0) {
        double y[NVMAX];
#pragma unroll
        for (int v = 0; v < NVMAX; ++v) y[v] = lane < nw ? red[lane][v] : 0.0;
        const double t = warp_sum_scatter<NVMAX>(y, idx);
        if ((lane & 1) == 0) tot[idx] = t;
        __syncwarp();
        if (lane == 0) finalize_update(tot, P, ctrl, hist, final_mode);
    }
}

static int finalize_threads(int nblocks) {
    // one warp per 64 row-pass blocks, at most FIN_WARPS
    const int w = (nblocks + 63) / 64;
    return 32 * (w < 1 ? 1 : w > FIN_WARPS ? FIN_WARPS : w);
}

template <typename T>
cudaError_t launch_init(cx<T>* X, cx<T>* S, cx<T>* Tf, const uint8_t* mask, const SchemeParams& prm, int64_t Ntot,
                        int d, int packed, const cx<T>* sigma, int sm_count, cudaStream_t s) {
    int64_t blocks = (Ntot + 255) / 256;
    const int64_t cap = (int64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    init_state_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(X, S, Tf, mask, prm, Ntot, d, packed, sigma);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblocks, int nv, const SchemeParams& prm, Ctrl* ctrl,
                            double* hist, int final_mode, int programmatic, cudaStream_t s) {
    return launch_pdl(finalize_kernel, dim3(1), dim3(finalize_threads(nblocks)), 0, s, programmatic, partials,
                      nblocks, nv, prm, ctrl, hist, final_mode);
}

// Small device-to-host transfers (the control block, the history) written by
// one block into mapped pinned host memory: they do not queue on a copy engine
// behind a large field copy running on another stream.
__global__ void copy_words_kernel(unsigned long long* __restrict__ dst, const unsigned long long* __restrict__ src,
                                  int64_t words) {
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_copy_words(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes % 8 != 0) return cudaErrorInvalidValue;
    if (bytes == 0) return cudaSuccess;
    copy_words_kernel<<<1, 256, 0, s>>>((unsigned long long*)dst, (const unsigned long long*)src,
                                        (int64_t)(bytes / 8));
    return cudaGetLastError();
}

template cudaError_t launch_init<float>(cx<float>*, cx<float>*, cx<float>*, const uint8_t*, const SchemeParams&,
                                        int64_t, int, int, const cx<float>*, int, cudaStream_t);
template cudaError_t launch_init<double>(cx<double>*, cx<double>*, cx<double>*, const uint8_t*, const SchemeParams&,
                                         int64_t, int, int, const cx<double>*, int, cudaStream_t);

}  // namespace lsfft

// ---------------------------------------------------------------------------
// Lanczos vector kernels on flat complex arrays of length L (FP64 reductions).
// ---------------------------------------------------------------------------
namespace lsfft {

constexpr int VEC_THREADS = 256;

__device__ __forceinline__ void vec_block_sum(double x, double* __restrict__ out) {
    __shared__ double red[VEC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < VEC_THREADS / 32; ++w) s += red[w];
        out[blockIdx.x] = s;
    }
}

// v = chi e (d components), partial sums of |v|^2
template <typename T>
__global__ void vec_init_masked_e(cx<T>* __restrict__ v, const uint8_t* __restrict__ mask, int64_t N, int d, double e0,
                                  double e1, double e2, double* __restrict__ partials) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)VEC_THREADS + threadIdx.x; i < N; i += (int64_t)gridDim.x * VEC_THREADS) {
        const bool inc = mask[i] != 0;
        const double e[3] = {e0, e1, e2};
        for (int c = 0; c < d; ++c) {
            const double val = inc ? e[c] : 0.0;
            v[c * N + i] = mkc((T)val, (T)0);
            acc += val * val;
        }
    }
    vec_block_sum(acc, partials);
}

// partial sums of Re sum conj(a) b
template <typename T>
__global__ void vec_dot(const cx<T>* __restrict__ a, const cx<T>* __restrict__ b, int64_t L,
                        double* __restrict__ partials) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)VEC_THREADS + threadIdx.x; i < L; i += (int64_t)gridDim.x * VEC_THREADS)
        acc += (double)a[i].x * (double)b[i].x + (double)a[i].y * (double)b[i].y;
    vec_block_sum(acc, partials);
}

// w <- w - alpha v - beta u, partial sums of |w|^2
template <typename T>
__global__ void vec_axpy_norm(cx<T>* __restrict__ w, const cx<T>* __restrict__ v, const cx<T>* __restrict__ u,
                              double alpha, double beta, int64_t L, double* __restrict__ partials) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)VEC_THREADS + threadIdx.x; i < L; i += (int64_t)gridDim.x * VEC_THREADS) {
        const double x = (double)w[i].x - alpha * (double)v[i].x - beta * (double)u[i].x;
        const double y = (double)w[i].y - alpha * (double)v[i].y - beta * (double)u[i].y;
        w[i] = mkc((T)x, (T)y);
        acc += x * x + y * y;
    }
    vec_block_sum(acc, partials);
}

template <typename T>
__global__ void vec_scale(cx<T>* __restrict__ dst, const cx<T>* __restrict__ src, double s, int64_t L) {
    for (int64_t i = blockIdx.x * (int64_t)VEC_THREADS + threadIdx.x; i < L; i += (int64_t)gridDim.x * VEC_THREADS)
        dst[i] = mkc((T)((double)src[i].x * s), (T)((double)src[i].y * s));
}

// One warp: lane l sums partials l, l + 32, ... in order, then a fixed shuffle
// tree (deterministic; the loads of a lane are independent, so they overlap).
__global__ void vec_sum_partials(const double* __restrict__ partials, int n, double* __restrict__ out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += 32) s += partials[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[0] = s;
}

template <typename T>
cudaError_t lanczos_init(cx<T>* v, const uint8_t* mask, int64_t N, int d, const double* e, int blocks,
                         double* partials, double* out, cudaStream_t s) {
    vec_init_masked_e<T><<<blocks, VEC_THREADS, 0, s>>>(v, mask, N, d, e[0], e[1], d > 2 ? e[2] : 0.0, partials);
    vec_sum_partials<<<1, 32, 0, s>>>(partials, blocks, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t lanczos_dot(const cx<T>* a, const cx<T>* b, int64_t L, int blocks, double* partials, double* out,
                        cudaStream_t s) {
    vec_dot<T><<<blocks, VEC_THREADS, 0, s>>>(a, b, L, partials);
    vec_sum_partials<<<1, 32, 0, s>>>(partials, blocks, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t lanczos_axpy_norm(cx<T>* w, const cx<T>* v, const cx<T>* u, double alpha, double beta, int64_t L,
                              int blocks, double* partials, double* out, cudaStream_t s) {
    vec_axpy_norm<T><<<blocks, VEC_THREADS, 0, s>>>(w, v, u, alpha, beta, L, partials);
    vec_sum_partials<<<1, 32, 0, s>>>(partials, blocks, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t lanczos_scale(cx<T>* dst, const cx<T>* src, double sc, int64_t L, int blocks, cudaStream_t s) {
    vec_scale<T><<<blocks, VEC_THREADS, 0, s>>>(dst, src, sc, L);
    return cudaGetLastError();
}

#define LSFFT_INST_VEC(T)                                                                                         \
    template cudaError_t lanczos_init<T>(cx<T>*, const uint8_t*, int64_t, int, const double*, int, double*, double*, \
                                         cudaStream_t);                                                           \
    template cudaError_t lanczos_dot<T>(const cx<T>*, const cx<T>*, int64_t, int, double*, double*, cudaStream_t); \
    template cudaError_t lanczos_axpy_norm<T>(cx<T>*, const cx<T>*, const cx<T>*, double, double, int64_t, int,    \
                                              double*, double*, cudaStream_t);                                    \
    template cudaError_t lanczos_scale<T>(cx<T>*, const cx<T>*, double, int64_t, int, cudaStream_t);
LSFFT_INST_VEC(float)
LSFFT_INST_VEC(double)

}  // namespace lsfft

// ---------------------------------------------------------------------------
// Gradient of sigma_* (first variation of the energy <sigma E.E> = sigma_* |e|^2,
// Eq. J12/J13): d sigma_*/d sigma(x) = E(x).E(x) / (N |e|^2) with the bilinear dot.
// Also the sums sum_x chi(x) g(x) (= d sigma_*/d sigma_1) and <sigma E.E>/|e|^2.
// ---------------------------------------------------------------------------
namespace lsfft {

template <typename T>
__global__ void gradient_kernel(const cx<T>* __restrict__ E, const uint8_t* __restrict__ mask,
                                const cx<T>* __restrict__ sigma, double s1re, double s1im, int d, int64_t N,
                                double inv_ne2, cx<T>* __restrict__ grad, double* __restrict__ partials) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)VEC_THREADS + threadIdx.x; i < N; i += (int64_t)gridDim.x * VEC_THREADS) {
        double gr = 0.0, gi = 0.0;
        for (int c = 0; c < d; ++c) {
            const double er = (double)E[c * N + i].x, ei = (double)E[c * N + i].y;
            gr += er * er - ei * ei;
            gi += 2.0 * er * ei;
        }
        if (grad) grad[i] = mkc((T)(gr * inv_ne2), (T)(gi * inv_ne2));
        double sr, si;
        if (sigma) {
            sr = (double)sigma[i].x;
            si = (double)sigma[i].y;
        } else {
            const bool inc = mask[i] != 0;
            sr = inc ? s1re : 1.0;
            si = inc ? s1im : 0.0;
        }
        if (mask[i]) {
            acc[0] += gr;
            acc[1] += gi;
        }
        acc[2] += sr * gr - si * gi;
        acc[3] += sr * gi + si * gr;
    }
    __shared__ double red[VEC_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < 4; ++v) {
        double x = acc[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < VEC_THREADS / 32; ++w) s += red[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

template <typename T>
__global__ void convert_field_kernel(cx<T>* __restrict__ dst, const double2* __restrict__ src, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = mkc((T)src[i].x, (T)src[i].y);
}

template <typename T>
cudaError_t launch_gradient(const cx<T>* E, const uint8_t* mask, const cx<T>* sigma, double s1re, double s1im, int d,
                            int64_t N, double inv_ne2, cx<T>* grad, int blocks, double* partials, cudaStream_t s) {
    gradient_kernel<T><<<blocks, VEC_THREADS, 0, s>>>(E, mask, sigma, s1re, s1im, d, N, inv_ne2, grad, partials);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert_field(cx<T>* dst, const double2* src, int64_t N, int sm_count, cudaStream_t s) {
    convert_field_kernel<T><<<sm_count * 8, 256, 0, s>>>(dst, src, N);
    return cudaGetLastError();
}

template cudaError_t launch_gradient<float>(const cx<float>*, const uint8_t*, const cx<float>*, double, double, int,
                                            int64_t, double, cx<float>*, int, double*, cudaStream_t);
template cudaError_t launch_gradient<double>(const cx<double>*, const uint8_t*, const cx<double>*, double, double, int,
                                             int64_t, double, cx<double>*, int, double*, cudaStream_t);
template cudaError_t launch_convert_field<float>(cx<float>*, const double2*, int64_t, int, cudaStream_t);
template cudaError_t launch_convert_field<double>(cx<double>*, const double2*, int64_t, int, cudaStream_t);

}  // namespace lsfft

// ---------------------------------------------------------------------------
// FP32 FMA throughput probe (the arithmetic ceiling reported beside the passes'
// HBM fractions).  Eight independent chains per thread keep every FMA pipe busy
// past its latency; the result is stored only if it equals an impossible value,
// so the chains are not removed.
// ---------------------------------------------------------------------------
namespace lsfft {

constexpr int FMA_THREADS = 256, FMA_ITERS = 4096;

template <bool PAIRED>
__global__ void __launch_bounds__(FMA_THREADS) fma_peak_kernel(float* __restrict__ sink, float a, float b) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i);
    if constexpr (PAIRED) {
        unsigned long long y[4], av, bv;
        asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
        asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
        for (int i = 0; i < 4; ++i) asm("mov.b64 %0, {%1, %2};" : "=l"(y[i]) : "f"(x[2 * i]), "f"(x[2 * i + 1]));
        for (int k = 0; k < FMA_ITERS; ++k) {
#pragma unroll
            for (int i = 0; i < 4; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(y[i]) : "l"(av), "l"(bv));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) asm("mov.b64 {%0, %1}, %2;" : "=f"(x[2 * i]), "=f"(x[2 * i + 1]) : "l"(y[i]));
    } else {
        for (int k = 0; k < FMA_ITERS; ++k) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

cudaError_t measure_fma_peak(int paired, int reps, double* tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&sink, sizeof(float) * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, 0);
        if (paired) fma_peak_kernel<true><<<blocks, FMA_THREADS>>>(sink, 0.999f, 1e-3f);
        else fma_peak_kernel<false><<<blocks, FMA_THREADS>>>(sink, 0.999f, 1e-3f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms > 0.f) {   // launch 0 warms up
            const double flops = 2.0 * 8.0 * FMA_ITERS * (double)blocks * FMA_THREADS;
            const double tf = flops / (ms * 1e-3) / 1e12;
            if (tf > best) best = tf;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    *tflops = best;
    return e;
}

}  // namespace lsfft
