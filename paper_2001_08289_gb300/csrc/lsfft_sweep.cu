// Persistent executor for a batch of 2-D solves on grids of uneven sizes: one
// kernel launch runs every iteration of every solve.
//
// Work queue.  Each solve advances through epochs; an epoch is one pass over
// its state: the row pass (inverse x-DFT, scheme update and volume sums, forward
// x-DFT; rows in items of LPB rows), the strided pass (forward y-DFT, Gamma,
// inverse y-DFT; columns in items of COLS columns), or the output pass (the
// field of the last iterate).  The solve's 64-bit word holds
// [63:40] epoch, [39:32] pass kind, [31:0] next item ticket.  A block claims an
// item with one atomicAdd on the word, which returns the epoch, pass and ticket
// consistently; tickets beyond the pass's item count are dropped.  After an
// item, a block barrier and one GPU-scope fence publish the block's writes and
// the block counts the item as done;
// the block that completes the last item of an epoch makes the transition:
//   row pass done     -> finalize (FP64 sums of the row items' partials in a
//                        fixed order, sigma_k of Eq. J13, stop rule) -> strided pass
//   strided pass done -> row pass, or the output pass once the stop rule fired
//   output pass done  -> final averages and sigma_*, solve finished
// (so, as in the single-grid path, the update that follows the iterate on which
// the stop rule fired is applied, and the returned field belongs to it).
//
// A pass item never waits on anything, so blocks only wait when no item is
// claimable; that wait polls with a sleep and is bounded: a block that could
// claim nothing for two seconds while solves remain sets the error flag and
// leaves.  State is read through L2 (cp.async.cg, ld.global.cg), never from a
// possibly stale L1 line, since the blocks that write a pass's output are not
// the ones that read it.
//
// Layout per solve: the complex layout of the single-grid path (component
// planes X[c][y][x], kept as x-spectra between passes; S, T on phase 1).
#include <cuda_runtime.h>

#include "lsfft_finalize.cuh"
#include "lsfft_kernels.cuh"
#include "lsfft_misc.h"
#include "lsfft_sweep.h"

namespace lsfft {

namespace {

constexpr int SW_THREADS = 256;
constexpr int SW_NV = 9;   // 4 d + 1 volume sums, d = 2
constexpr int CLAIM = 4;   // consecutive items claimed at once when a pass has many

enum { PH_FIRST = 0, PH_ROW = 1, PH_COL = 2, PH_OUT = 3 };

template <int N>
struct SwRow {   // row items: LPB whole rows of both planes
    static constexpr int E = 16, TL = N / E, LPB = SW_THREADS / TL;
    using P = Pitch<float, N, TL>;
    static constexpr int S_BYTES = 2 * LPB * P::S * 8;
    static constexpr int X_BYTES = LPB * P::X * 8;
    static constexpr int M_BYTES = roundup16(LPB * N);
    static constexpr int SMEM = S_BYTES + X_BYTES + M_BYTES;
};

template <int N>
struct SwCol {   // column items: COLS adjacent columns of both planes
    static constexpr int E = 16, TL = N / E, COLS = SW_THREADS / (2 * TL);
    static constexpr int XP = roundup16(N + N / 16) + 8;
    static constexpr int DATA = 2 * N * COLS * 8;
    static constexpr int SMEM = DATA > 2 * COLS * XP * 8 ? DATA : 2 * COLS * XP * 8;
};

__host__ __device__ constexpr int sw_smem() {
    return cmax(cmax(cmax(SwRow<128>::SMEM, SwRow<256>::SMEM), cmax(SwRow<512>::SMEM, SwRow<1024>::SMEM)),
                cmax(cmax(SwCol<128>::SMEM, SwCol<256>::SMEM), cmax(SwCol<512>::SMEM, SwCol<1024>::SMEM)));
}

__device__ __forceinline__ float2 ldcg2(const float2* p) { return __ldcg(p); }

// One row item: rows [item LPB, item LPB + LPB) of job J.
template <int N>
__device__ void sweep_row_item(const SweepJob& J, int item, int phase, unsigned char* smem) {
    using Cfg = SwRow<N>;
    using C = float2;
    constexpr int E = Cfg::E, TL = Cfg::TL, LPB = Cfg::LPB, PS = Cfg::P::S, PX = Cfg::P::X;
    const int64_t Ntot = (int64_t)N * J.ny;
    C* Sb = reinterpret_cast<C*>(smem);                                   // [2][LPB][PS]
    const int g = threadIdx.x / TL, t = threadIdx.x % TL;
    C* Xb = reinterpret_cast<C*>(smem + Cfg::S_BYTES) + g * PX;
    uint8_t* Mb = smem + Cfg::S_BYTES + Cfg::X_BYTES;                      // [LPB][N]
    const bool first = phase == PH_FIRST, outm = phase == PH_OUT;
    const int64_t row0 = (int64_t)item * LPB;
    // stage both planes (not on the first pass, which starts from the mask) and the mask rows
    if (!first) {
        constexpr int CH = N * 8 / 16;   // 16-byte chunks per row
        for (int i = threadIdx.x; i < 2 * LPB * CH; i += SW_THREADS) {
            const int ch = i % CH, r = (i / CH) % LPB, c = i / (CH * LPB);
            cp_async16(reinterpret_cast<unsigned char*>(Sb + (c * LPB + r) * PS) + 16 * ch,
                       reinterpret_cast<const unsigned char*>(J.X + c * Ntot + (row0 + r) * N) + 16 * ch);
        }
    }
    for (int i = threadIdx.x; i < LPB * N / 16; i += SW_THREADS) {
        const int ch = i % (N / 16), r = i / (N / 16);
        cp_async16(Mb + r * N + 16 * ch, J.mask + (row0 + r) * N + 16 * ch);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const KConst<float>& K = J.k;
    // 1. real-space values of both planes at the thread's positions
    for (int c = 0; c < 2; ++c) {
        C* Sl = Sb + (c * LPB + g) * PS;
        C v[E];
        if (first) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const bool inc = Mb[g * N + t + TL * m] != 0;
                const C q = inc ? K.iq_in : K.iq_out;
                v[m] = mkc(q.x * K.e[c], q.y * K.e[c]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = Sl[t + TL * m];
            LineFFT<float, N, E, 16, true, true>::run(v, Xb, t, nullptr);
        }
#pragma unroll
        for (int m = 0; m < E; ++m) Sl[t + TL * m] = v[m];
    }
    __syncthreads();
    // 2. scheme update and volume sums (S, T read through L2; initial S, T on the first pass)
    float acc[SW_NV];
#pragma unroll
    for (int i = 0; i < SW_NV; ++i) acc[i] = 0.0f;
    const bool sub = K.scheme == SCHEME_MS_SUB || K.scheme == SCHEME_EM_SUB;
    const C s_in = mkc((float)J.prm.is_in[0], (float)J.prm.is_in[1]);
    const C t_in = mkc((float)J.prm.it_in[0], (float)J.prm.it_in[1]);
#pragma unroll 4
    for (int m = 0; m < E; ++m) {
        const int pos = t + TL * m;
        const int64_t idx = (row0 + g) * N + pos;
        const bool inc = Mb[g * N + pos] != 0;
        C q[2], Ev[2], Jv[2], sl[2] = {mkc(0.f, 0.f), mkc(0.f, 0.f)}, tl[2] = {mkc(0.f, 0.f), mkc(0.f, 0.f)};
#pragma unroll
        for (int c = 0; c < 2; ++c) q[c] = Sb[(c * LPB + g) * PS + pos];
        if (sub && inc) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                sl[c] = first ? mkc(s_in.x * K.e[c], s_in.y * K.e[c]) : ldcg2(J.S + c * Ntot + idx);
                if (J.T) tl[c] = first ? mkc(t_in.x * K.e[c], t_in.y * K.e[c]) : ldcg2(J.T + c * Ntot + idx);
            }
        }
        switch (K.scheme) {
            case SCHEME_MS: pointwise<float, 2, SCHEME_MS>(K, q, inc, sl, tl, 1, Ev, Jv, !outm); break;
            case SCHEME_EM: pointwise<float, 2, SCHEME_EM>(K, q, inc, sl, tl, 1, Ev, Jv, !outm); break;
            case SCHEME_MS_SUB: pointwise<float, 2, SCHEME_MS_SUB>(K, q, inc, sl, tl, 1, Ev, Jv, !outm); break;
            default: pointwise<float, 2, SCHEME_EM_SUB>(K, q, inc, sl, tl, 1, Ev, Jv, !outm); break;
        }
        if (sub && inc && !outm) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                J.S[c * Ntot + idx] = sl[c];
                if (J.T) J.T[c * Ntot + idx] = tl[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            Sb[(c * LPB + g) * PS + pos] = q[c];
            acc[4 * c + 0] += Ev[c].x;
            acc[4 * c + 1] += Ev[c].y;
            acc[4 * c + 2] += Jv[c].x;
            acc[4 * c + 3] += Jv[c].y;
            acc[8] += Ev[c].x * Ev[c].x + Ev[c].y * Ev[c].y;
            if (outm) J.Eout[c * Ntot + idx] = Ev[c];
        }
    }
    double dacc[SW_NV];
#pragma unroll
    for (int i = 0; i < SW_NV; ++i) dacc[i] = (double)acc[i];
    block_reduce_store<SW_NV, SW_THREADS>(dacc, J.partials + (int64_t)item * SW_NV);
    if (outm) return;
    // 3. forward x-DFTs and stores
    __syncthreads();
    for (int c = 0; c < 2; ++c) {
        C* Sl = Sb + (c * LPB + g) * PS;
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = Sl[t + TL * m];
        LineFFT<float, N, E, 16, false, true>::run(v, Xb, t, nullptr);
#pragma unroll
        for (int m = 0; m < E; ++m) J.X[c * Ntot + (row0 + g) * N + t + TL * m] = v[m];
    }
}

// One column item: columns [item COLS, item COLS + COLS) of both planes, length N = n_y.
template <int N>
__device__ void sweep_col_item(const SweepJob& J, int item, unsigned char* smem) {
    using Cfg = SwCol<N>;
    using C = float2;
    constexpr int E = Cfg::E, TL = Cfg::TL, COLS = Cfg::COLS, XP = Cfg::XP;
    const int nx = J.nx;
    const int64_t Ntot = (int64_t)nx * N;
    C* Bi = reinterpret_cast<C*>(smem);                                  // [2][N][COLS], then exchange lines
    const int w = threadIdx.x % COLS;
    const int t = (threadIdx.x / COLS) % TL;
    const int c = threadIdx.x / (COLS * TL);
    const int col0 = item * COLS;
    constexpr int CH = COLS * 8 / 16;                                   // 16-byte chunks per row segment
    for (int i = threadIdx.x; i < 2 * N * CH; i += SW_THREADS) {
        const int ch = i % CH, j = (i / CH) % N, cc = i / (CH * N);
        cp_async16(reinterpret_cast<unsigned char*>(Bi + (cc * N + j) * COLS) + 16 * ch,
                   reinterpret_cast<const unsigned char*>(J.X + cc * Ntot + (int64_t)j * nx + col0) + 16 * ch);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    C* Yc = Bi + c * N * COLS;
    C* Xb = Bi + (c * COLS + w) * XP;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = Yc[(t + TL * m) * COLS + w];
    LineFFT<float, N, E, 16, false, true>::run(v, Xb, t, nullptr);
    __syncthreads();   // the exchange lines share the buffer: all reads done
#pragma unroll
    for (int m = 0; m < E; ++m) Yc[(t + TL * m) * COLS + w] = v[m];
    __syncthreads();
    const int nn[3] = {nx, N, 1};
    for (int p = threadIdx.x; p < N * COLS; p += SW_THREADS) {
        const int kl = p / COLS, wc = p % COLS;
        const int ki[3] = {col0 + wc, kl, 0};
        C q[2] = {Bi[kl * COLS + wc], Bi[(N + kl) * COLS + wc]};
        gamma_apply_k<float, 2>(q, ki, J.k, nn, J.fd);
        Bi[kl * COLS + wc] = q[0];
        Bi[(N + kl) * COLS + wc] = q[1];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = Yc[(t + TL * m) * COLS + w];
    LineFFT<float, N, E, 16, true, true>::run(v, Xb, t, nullptr);
    C* dst = J.X + c * Ntot + col0 + w;
#pragma unroll
    for (int m = 0; m < E; ++m) dst[(int64_t)(t + TL * m) * nx] = v[m];
}

// FP64 sums of the row items' partials (fixed order) and the scalar recurrence,
// on a shared copy of the control block read and written through L2.
__device__ void sweep_finalize(SweepJob& J, int final_mode, unsigned char* smem) {
    double* tot = reinterpret_cast<double*>(smem);          // [16]
    double* red = tot + 16;                                  // [8][16]
    Ctrl* cs = reinterpret_cast<Ctrl*>(red + 8 * 16);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double x[SW_NV];
#pragma unroll
    for (int v = 0; v < SW_NV; ++v) x[v] = 0.0;
    for (int b = threadIdx.x; b < J.row_items; b += SW_THREADS)
#pragma unroll
        for (int v = 0; v < SW_NV; ++v) x[v] += __ldcg(J.partials + (int64_t)b * SW_NV + v);
#pragma unroll
    for (int v = 0; v < SW_NV; ++v) {
        for (int o = 16; o > 0; o >>= 1) x[v] += __shfl_down_sync(0xffffffffu, x[v], o);
        if (lane == 0) red[warp * 16 + v] = x[v];
    }
    // the control block, through L2
    constexpr int CW = (int)(sizeof(Ctrl) / 8);
    for (int i = threadIdx.x; i < CW; i += SW_THREADS)
        reinterpret_cast<unsigned long long*>(cs)[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&J.ctrl) + i);
    __syncthreads();
    if (threadIdx.x < SW_NV) {
        double s = 0.0;
        for (int w = 0; w < SW_THREADS / 32; ++w) s += red[w * 16 + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) finalize_update(tot, J.prm, cs, J.hist, final_mode);
    __syncthreads();
    for (int i = threadIdx.x; i < CW; i += SW_THREADS)
        __stcg(reinterpret_cast<unsigned long long*>(&J.ctrl) + i, reinterpret_cast<unsigned long long*>(cs)[i]);
    __threadfence();
    __syncthreads();
}

__device__ void row_item(const SweepJob& J, int item, int phase, unsigned char* smem) {
    switch (J.lognx) {
        case 7: sweep_row_item<128>(J, item, phase, smem); break;
        case 8: sweep_row_item<256>(J, item, phase, smem); break;
        case 9: sweep_row_item<512>(J, item, phase, smem); break;
        default: sweep_row_item<1024>(J, item, phase, smem); break;
    }
}
__device__ void col_item(const SweepJob& J, int item, unsigned char* smem) {
    switch (J.logny) {
        case 7: sweep_col_item<128>(J, item, smem); break;
        case 8: sweep_col_item<256>(J, item, smem); break;
        case 9: sweep_col_item<512>(J, item, smem); break;
        default: sweep_col_item<1024>(J, item, smem); break;
    }
}

__device__ __forceinline__ int pass_items(const SweepJob& J, int phase) {
    return phase == PH_COL ? J.col_items : J.row_items;
}

__host__ __device__ constexpr unsigned long long word_of(unsigned long long epoch, int phase) {
    return (epoch << 40) | ((unsigned long long)phase << 32);
}

__global__ void __launch_bounds__(SW_THREADS, 2)
sweep_kernel(SweepJob* __restrict__ jobs, int njobs, SweepGlobal* __restrict__ glob, long long idle_limit_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_job, s_item, s_nitems, s_phase, s_last;
    unsigned start = blockIdx.x;
    unsigned long long t_idle = 0;
    for (;;) {
        // the first warp looks for work: its 32 lanes probe 32 solves per round trip,
        // the claimable ones (by ballot) are tried in order with one atomicAdd each
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int found = -1, item = 0, phase = 0, nitems = 1;
            bool stop = false;
            if (*(volatile int*)&glob->jobs_done >= njobs || *(volatile int*)&glob->error) stop = true;
            for (int c0 = 0; c0 < njobs && found < 0 && !stop; c0 += 32) {
                const int j = (int)((start + (unsigned)(c0 + lane)) % (unsigned)njobs);
                bool ok = false;
                if (c0 + lane < njobs) {
                    SweepJob& J = jobs[j];
                    const unsigned long long wd = *(volatile unsigned long long*)&J.word;
                    const int ph = (int)((wd >> 32) & 0xff);
                    ok = !*(volatile int*)&J.finished && (wd & 0xffffffffull) < (unsigned long long)pass_items(J, ph);
                }
                unsigned mask = __ballot_sync(0xffffffffu, ok);
                while (mask && found < 0) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    int got = -1, it2 = 0, ph2 = 0, k2 = 0;
                    if (lane == src) {
                        SweepJob& J = jobs[j];
                        // passes with many items hand out CLAIM consecutive items per atomic
                        const int cnt = pass_items(J, (int)((*(volatile unsigned long long*)&J.word >> 32) & 0xff));
                        const unsigned long long want = cnt >= 16 * CLAIM ? CLAIM : 1;
                        const unsigned long long old = atomicAdd(&J.word, want);
                        ph2 = (int)((old >> 32) & 0xff);
                        const unsigned long long ticket = old & 0xffffffffull;
                        const unsigned long long count = (unsigned long long)pass_items(J, ph2);
                        if (ticket < count) {
                            got = j;
                            it2 = (int)ticket;
                            k2 = (int)((ticket + want <= count ? want : count - ticket));
                        }
                    }
                    got = __shfl_sync(0xffffffffu, got, src);
                    it2 = __shfl_sync(0xffffffffu, it2, src);
                    ph2 = __shfl_sync(0xffffffffu, ph2, src);
                    k2 = __shfl_sync(0xffffffffu, k2, src);
                    if (got >= 0) {
                        found = got;
                        item = it2;
                        phase = ph2;
                        nitems = k2;
                    }
                }
            }
            if (lane == 0) {
                s_job = stop ? -2 : found;
                s_item = item;
                s_nitems = nitems;
                s_phase = phase;
                if (found >= 0) {
                    start = (unsigned)found;   // stay with this solve while it has items
                    t_idle = 0;
                } else if (!stop) {
                    unsigned long long now;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                    if (t_idle == 0) t_idle = now;
                    if ((long long)(now - t_idle) > idle_limit_ns) {   // nothing claimable for too long
                        atomicExch(&glob->error, 1);
                        s_job = -2;
                    }
                }
                __threadfence();   // acquire: the claimed pass's input was published before its epoch
            }
            start = __shfl_sync(0xffffffffu, start, 0);
        }
        __syncthreads();
        const int j = s_job;
        if (j == -2) break;
        if (j == -1) {
            __nanosleep(2000);
            ++start;
            continue;
        }
        SweepJob& J = jobs[j];
        const int phase = s_phase, nit = s_nitems;
        for (int i = 0; i < nit; ++i) {
            if (i > 0) __syncthreads();   // shared memory of the previous item is free
            if (phase == PH_COL) col_item(J, s_item + i, smem);
            else row_item(J, s_item + i, phase, smem);
        }
        __syncthreads();   // the block's writes of the items are done ...
        if (threadIdx.x == 0) {
            __threadfence();   // ... and published (cumulatively, through the barrier) before the count
            const unsigned prev = atomicAdd(&J.completed, (unsigned)nit);
            s_last = prev + (unsigned)nit == (unsigned)pass_items(J, phase);
        }
        __syncthreads();
        if (!s_last) continue;
        // the last item of the epoch: transition
        int next = -1;
        if (phase == PH_FIRST || phase == PH_ROW) {
            sweep_finalize(J, 0, smem);
            next = PH_COL;
        } else if (phase == PH_COL) {
            next = __ldcg(&J.ctrl.done) ? PH_OUT : PH_ROW;
        } else {
            sweep_finalize(J, 1, smem);
        }
        if (threadIdx.x == 0) {
            atomicExch(&J.completed, 0u);
            __threadfence();
            if (next < 0) {
                atomicExch(&J.finished, 1);
                atomicAdd(&glob->jobs_done, 1);
            } else {
                const unsigned long long old = *(volatile unsigned long long*)&J.word;
                atomicExch(&J.word, word_of((old >> 40) + 1, next));
            }
        }
        __syncthreads();
    }
}

}  // namespace

int sweep_smem_bytes() { return sw_smem(); }
int sweep_threads() { return SW_THREADS; }
int sweep_row_lpb(int n) { return SW_THREADS / (n / 16); }
int sweep_col_cols(int n) { return SW_THREADS / (2 * (n / 16)); }

cudaError_t sweep_prepare(int* blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sw_smem());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep_kernel, SW_THREADS, sw_smem());
}

cudaError_t sweep_launch(SweepJob* jobs, int njobs, SweepGlobal* glob, int blocks, long long idle_limit_ns,
                         cudaStream_t s) {
    sweep_kernel<<<blocks, SW_THREADS, sw_smem(), s>>>(jobs, njobs, glob, idle_limit_ns);
    return cudaGetLastError();
}

}  // namespace lsfft
