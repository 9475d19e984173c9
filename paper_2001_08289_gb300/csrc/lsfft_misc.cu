// Small kernels around the passes: initial state and the FP64 finalize step
// (volume averages, sigma_k of Eq. J13, stop rule).
#include <math.h>

#include "lsfft_misc.h"

namespace lsfft {

// Initial state.  Complex layout: Q = iq e, S = is e, T = it e (S, T on phase 1).
// Packed real layout (d = 2): one plane z = iq (e_x + i e_y), with S = i s and
// T = i tau stored as s = Im(is) (e_x + i e_y), tau = Im(it) (e_x + i e_y).
template <typename T>
__global__ void init_state_kernel(cx<T>* __restrict__ X, cx<T>* __restrict__ S, cx<T>* __restrict__ Tf,
                                  const uint8_t* __restrict__ mask, const SchemeParams P, int64_t Ntot, int d,
                                  int packed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Ntot; i += (int64_t)gridDim.x * blockDim.x) {
        const bool inc = mask[i] != 0;
        if (packed) {
            const double q = inc ? P.iq_in[0] : P.iq_out[0];
            X[i] = mkc((T)(q * P.e[0]), (T)(q * P.e[1]));
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

// One block of FIN_THREADS threads.  Sums partials[b][v] over blocks in a fixed
// order (deterministic), then thread 0 updates the scalar recurrence.
constexpr int FIN_THREADS = 256;

__global__ void __launch_bounds__(FIN_THREADS)
finalize_kernel(const double* __restrict__ partials, int nblocks, int nv, const SchemeParams P,
                Ctrl* __restrict__ ctrl, double* __restrict__ hist, int final_mode) {
    __shared__ double tot[16];
    __shared__ double red[FIN_THREADS / 32];
    if (!final_mode && ctrl->done) {
        if (threadIdx.x == 0) ctrl->skipB = 1;
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = 0; v < nv; ++v) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += FIN_THREADS) x += partials[(int64_t)b * nv + v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < FIN_THREADS / 32; ++w) s += red[w];
            tot[v] = s;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const int d = P.d;
    // sigma_k = (<J>.e) / (<E>.e); the 1/N factors cancel
    double je_re = 0, je_im = 0, ee_re = 0, ee_im = 0;
    for (int c = 0; c < d; ++c) {
        ee_re += tot[4 * c + 0] * P.e[c];
        ee_im += tot[4 * c + 1] * P.e[c];
        je_re += tot[4 * c + 2] * P.e[c];
        je_im += tot[4 * c + 3] * P.e[c];
    }
    const double den = ee_re * ee_re + ee_im * ee_im;
    const double s_re = (je_re * ee_re + je_im * ee_im) / den;
    const double s_im = (je_im * ee_re - je_re * ee_im) / den;
    const double norm = tot[4 * d] * P.inv_ntot;
    const int k = ctrl->iter;
    const double mag = sqrt(s_re * s_re + s_im * s_im);
    double rel = INFINITY;
    if (k >= 1 && mag != 0.0) {
        const double dr = s_re - ctrl->prev[0], di = s_im - ctrl->prev[1];
        rel = sqrt(dr * dr + di * di) / mag;
    }
    hist[(int64_t)k * HIST_STRIDE + 0] = s_re;
    hist[(int64_t)k * HIST_STRIDE + 1] = s_im;
    hist[(int64_t)k * HIST_STRIDE + 2] = rel;
    hist[(int64_t)k * HIST_STRIDE + 3] = norm;
    ctrl->sigma[0] = s_re;
    ctrl->sigma[1] = s_im;
    for (int c = 0; c < d; ++c) {
        ctrl->meanE[c][0] = tot[4 * c + 0] * P.inv_ntot;
        ctrl->meanE[c][1] = tot[4 * c + 1] * P.inv_ntot;
        ctrl->meanJ[c][0] = tot[4 * c + 2] * P.inv_ntot;
        ctrl->meanJ[c][1] = tot[4 * c + 3] * P.inv_ntot;
    }
    ctrl->prev[0] = s_re;
    ctrl->prev[1] = s_im;
    if (final_mode) return;
    if (k == 0) ctrl->norm0 = norm;
    ctrl->run = (rel < P.tol) ? ctrl->run + 1 : 0;
    const bool diverged = !isfinite(s_re) || !isfinite(s_im) || !isfinite(norm) ||
                          norm > DIVERGENCE_FACTOR * ctrl->norm0;
    if (diverged) {
        ctrl->status = ST_DIVERGED;
        ctrl->done = 1;
    } else if (ctrl->run >= P.consecutive) {
        ctrl->status = ST_OK;
        ctrl->done = 1;
    } else if (k + 1 >= P.max_iter) {
        ctrl->status = ST_NOTCONV;
        ctrl->done = 1;
    }
    ctrl->iter = k + 1;
}

template <typename T>
cudaError_t launch_init(cx<T>* X, cx<T>* S, cx<T>* Tf, const uint8_t* mask, const SchemeParams& prm, int64_t Ntot,
                        int d, int packed, int sm_count, cudaStream_t s) {
    int64_t blocks = (Ntot + 255) / 256;
    const int64_t cap = (int64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    init_state_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(X, S, Tf, mask, prm, Ntot, d, packed);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblocks, int nv, const SchemeParams& prm, Ctrl* ctrl,
                            double* hist, int final_mode, cudaStream_t s) {
    finalize_kernel<<<1, FIN_THREADS, 0, s>>>(partials, nblocks, nv, prm, ctrl, hist, final_mode);
    return cudaGetLastError();
}

template cudaError_t launch_init<float>(cx<float>*, cx<float>*, cx<float>*, const uint8_t*, const SchemeParams&,
                                        int64_t, int, int, int, cudaStream_t);
template cudaError_t launch_init<double>(cx<double>*, cx<double>*, cx<double>*, const uint8_t*, const SchemeParams&,
                                         int64_t, int, int, int, cudaStream_t);

}  // namespace lsfft
