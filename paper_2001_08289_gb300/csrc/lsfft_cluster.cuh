// Strided (y) pass for long 2-D columns on a thread-block cluster.
//
// One SM cannot stage enough adjacent columns of length N >= 2048 to read
// whole 32-byte sectors, so a cluster of CL = 4 blocks shares the work of an
// item of W adjacent columns (W x 8 B = 32 B per row, W = 4 for FP32, 2 for
// FP64).  With rows r = q + CL j (block rank q, j < M = N/CL) the length-N DFT
// splits as
//     X[k + M m] = sum_q W_CL^(q m) W_N^(q k) Y_q[k],
//     Y_q[k]     = sum_j x[q + CL j] W_M^(j k),            k < M, m < CL.
// Block q loads its rows of all item lines (coalesced across the W columns),
// computes the M-point transforms Y_q in shared memory, and after one cluster
// barrier each block takes a quarter of the k range: it reads Y_q[k] of every
// block through distributed shared memory, forms the CL-point combinations
// (all frequencies k + M m of all lines of the item are then in one thread),
// applies the Gamma step, runs the inverse combination and writes the results
// back to the same remote slots it read.  Every slot is read and rewritten by
// exactly one thread, so a second cluster barrier suffices before the local
// inverse M-point transforms.  Lines of an item: the d = 2 component planes
// (complex layout) or the two half-spectrum planes (packed layout) of W
// adjacent columns.
#pragma once

#include <cooperative_groups.h>

#include "lsfft_kernels.cuh"

namespace lsfft {

template <typename T, int N>
struct CluCfg {
    static constexpr int CL = 4;
    static constexpr int M = N / CL;
    static constexpr int CS = (int)sizeof(cx<T>);
    static constexpr int W = 32 / CS;                  // adjacent columns per item
    static constexpr int LS = 2;                       // slots per column: the two planes
    static constexpr int LINES = LS * W;
    static constexpr int E = sizeof(T) == 4 ? 16 : 8;
    static constexpr int RMAX = sizeof(T) == 4 ? 16 : 8;
    static constexpr int TL = M >= E ? M / E : 1;      // (only N >= 2048 is ever launched)
    static constexpr int THREADS = cmin(512, LINES * TL);
    static constexpr int G = THREADS / TL;             // lines transformed concurrently
    static constexpr int ROUNDS = (LINES + G - 1) / G;
    static constexpr bool SLOT_ROUNDS = G == W && ROUNDS == LS;   // round rd transforms exactly slot rd
    static constexpr int YP = M + 4;                   // staged line pitch (bank offset between lines)
    static constexpr int XP = roundup16(M + M / 16);   // exchange line pitch
    static constexpr int Y_BYTES = LINES * YP * CS;
    static constexpr int SMEM = Y_BYTES + G * XP * CS;
    static constexpr bool SUPPORTED = N >= 2048 && SMEM <= 227 * 1024 && G >= 1 && (LINES % G == 0 || G > LINES);
};

template <typename T, int N>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(CluCfg<T, N>::THREADS, 1)
col_pass_cluster(const PassArgs<T> A) {
    namespace cg = cooperative_groups;
    using Cfg = CluCfg<T, N>;
    using C = cx<T>;
    constexpr int CL = Cfg::CL, M = Cfg::M, W = Cfg::W, LS = Cfg::LS, LINES = Cfg::LINES;
    constexpr int E = Cfg::E, TL = Cfg::TL, G = Cfg::G, YP = Cfg::YP, XP = Cfg::XP;
    constexpr int KQ = M / CL;                         // k range owned by one block in the exchange
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (A.ctrl->skipB) return;                         // uniform over the grid: no barrier is reached

    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int64_t cid = blockIdx.x / CL, ncl = gridDim.x / CL;
    C* Y = reinterpret_cast<C*>(smem_raw);
    const int g = threadIdx.x / TL, t = threadIdx.x % TL;
    C* Xg = reinterpret_cast<C*>(smem_raw + Cfg::Y_BYTES) + g * XP;
    // lines of an item: the two component planes (slots) of W adjacent columns;
    // n_inner need not be a multiple of W (the half-spectrum planes hold
    // n_x/2 + 1 columns within a padded pitch): the last item runs into padding
    const int64_t n_items = (A.n_inner + W - 1) / W;

    C* Yr[CL];                                          // the item buffers of every block of the cluster
#pragma unroll
    for (int p = 0; p < CL; ++p) Yr[p] = cluster.map_shared_rank(Y, p);

    // stage / store slot s (W lines) of an item: lanes run over the W adjacent
    // columns first.  THREADS is a multiple of W, so a thread keeps one column
    // w = threadIdx.x % W for the whole loop and only the row advances.
    static_assert(Cfg::THREADS % W == 0, "thread count must be a multiple of W");
    const int wt = threadIdx.x % W;
    const int j0 = threadIdx.x / W;
    constexpr int JSTEP = Cfg::THREADS / W;
    auto prefetch_slot = [&](int64_t item, int s) {
        C* dst = Y + (s * W + wt) * YP;
        const C* src = A.X + s * A.Ntot + item * W + wt;
        for (int j = j0; j < M; j += JSTEP) {
            const C* sp = src + (int64_t)(q + CL * j) * A.ls;
            if constexpr (sizeof(C) == 16) cp_async16(dst + j, sp);
            else cp_async8(dst + j, sp);
        }
        cp_async_commit();
    };
    auto store_slot = [&](int64_t item, int s) {
        const C* src = Y + (s * W + wt) * YP;
        C* dst = A.X + s * A.Ntot + item * W + wt;
        for (int j = j0; j < M; j += JSTEP) dst[(int64_t)(q + CL * j) * A.ls] = src[j];
    };
    // W_N^(p k) for p = 0..CL-1 (forward sign)
    auto twiddles = [&](int k, C (&w)[CL]) {
        w[0] = mkc((T)1, (T)0);
        if constexpr (sizeof(T) == 4) {
            float s, c;
            sincospif(2.0f * (float)k / (float)N, &s, &c);
            w[1] = mkc(c, -s);
        } else {
            w[1] = A.tw[k];
        }
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
    };

    int64_t item = cid;
    if (item < n_items)
        for (int s = 0; s < LS; ++s) prefetch_slot(item, s);
    for (; item < n_items; item += ncl) {
        const int64_t next = item + ncl;
        // 1. local forward M-point transforms, parked in place.  When one round
        //    covers exactly one slot (G == W), round rd starts as soon as slot rd
        //    has landed, while the later slot is still in flight.
        for (int rd = 0; rd < Cfg::ROUNDS; ++rd) {
            if (Cfg::SLOT_ROUNDS) cp_async_wait_pending(LS - 1 - rd);
            else if (rd == 0) cp_async_wait_all();
            __syncthreads();
            const int l = rd * G + g;
            C v[E];
            C* Yl = Y + (l < LINES ? l : 0) * YP;
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = Yl[t + TL * m];
            LineFFT<T, M, E, Cfg::RMAX, false>::run(v, Xg, t, A.tw, CL);
            if (l < LINES) {
#pragma unroll
                for (int m = 0; m < E; ++m) Yl[t + TL * m] = v[m];
            }
        }
        cluster.sync();
        // 2. exchange: combine, Gamma, inverse combine over the owned k range
        for (int idx = threadIdx.x; idx < W * KQ; idx += Cfg::THREADS) {
            const int k = q * KQ + idx % KQ, w = idx / KQ;
            C tw[CL];
            twiddles(k, tw);
            C x[LS][CL];
#pragma unroll
            for (int s = 0; s < LS; ++s) {
                C y[CL];
#pragma unroll
                for (int p = 0; p < CL; ++p) y[p] = cmul(Yr[p][(s * W + w) * YP + k], tw[p]);
                // 4-point DFT over p: x[m] = sum_p y[p] (-i)^(p m)
                const C a0 = cadd(y[0], y[2]), a1 = csub(y[0], y[2]);
                const C b0 = cadd(y[1], y[3]), b1 = csub(y[1], y[3]);
                const C b1r = mkc(b1.y, -b1.x);   // -i b1
                x[s][0] = cadd(a0, b0);
                x[s][2] = csub(a0, b0);
                x[s][1] = cadd(a1, b1r);
                x[s][3] = csub(a1, b1r);
            }
            const int kx = (int)(item * W + w);
#pragma unroll
            for (int m = 0; m < CL; ++m) {
                C vq[2] = {x[0][m], x[1][m]};
                const int ki[3] = {kx, k + M * m, 0};
                gamma_apply<T, 2>(vq, ki, A);
                x[0][m] = vq[0];
                x[1][m] = vq[1];
            }
#pragma unroll
            for (int s = 0; s < LS; ++s) {
                // inverse 4-point DFT over m: y[p] = sum_m x[m] (+i)^(p m), then * conj W_N^(p k)
                const C a0 = cadd(x[s][0], x[s][2]), a1 = csub(x[s][0], x[s][2]);
                const C b0 = cadd(x[s][1], x[s][3]), b1 = csub(x[s][1], x[s][3]);
                const C b1r = mkc(-b1.y, b1.x);   // +i b1
                C y[CL];
                y[0] = cadd(a0, b0);
                y[2] = csub(a0, b0);
                y[1] = cadd(a1, b1r);
                y[3] = csub(a1, b1r);
#pragma unroll
                for (int p = 0; p < CL; ++p) Yr[p][(s * W + w) * YP + k] = cmulc(y[p], tw[p]);
            }
        }
        cluster.sync();
        // 3. local inverse M-point transforms, parked in place; coalesced stores;
        //    the next item's slots are staged as soon as they are stored (with
        //    G == W, slot rd is stored and restaged while round rd + 1 computes)
        for (int rd = 0; rd < Cfg::ROUNDS; ++rd) {
            const int l = rd * G + g;
            C v[E];
            C* Yl = Y + (l < LINES ? l : 0) * YP;
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = Yl[t + TL * m];
            LineFFT<T, M, E, Cfg::RMAX, true>::run(v, Xg, t, A.tw, CL);
            if (l < LINES) {
#pragma unroll
                for (int m = 0; m < E; ++m) Yl[t + TL * m] = v[m];
            }
            if (Cfg::SLOT_ROUNDS) {
                __syncthreads();
                store_slot(item, rd);
                __syncthreads();
                if (next < n_items) prefetch_slot(next, rd);
            }
        }
        if (!Cfg::SLOT_ROUNDS) {
            __syncthreads();
            for (int s = 0; s < LS; ++s) {
                store_slot(item, s);
                __syncthreads();
                if (next < n_items) prefetch_slot(next, s);
            }
        }
    }
    cp_async_wait_all();
    cluster.sync();   // no block leaves while a peer may still address its shared memory
}

}  // namespace lsfft
