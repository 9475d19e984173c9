// Strided (y) pass for long 2-D columns on a thread-block cluster, with its
// tiles moved by the tensor memory accelerator (TMA).
//
// One SM cannot stage enough adjacent columns of length N >= 4096, so a
// cluster of CL = 2 blocks shares the work of an item of W adjacent columns
// (16-byte row segments: W = 2 in FP32, 1 in FP64).  With rows r = q + CL j
// (block rank q, j < M = N/CL) the length-N DFT splits as
//     X[k + M m] = sum_q W_CL^(q m) W_N^(q k) Y_q[k],
//     Y_q[k]     = sum_j x[q + CL j] W_M^(j k),            k < M, m < CL.
// Block q fetches its rows of each plane of the item with one TMA box (rows
// q + CL j, W columns; shared-memory layout [j][w]), computes the M-point
// transforms Y_q in place, and after one cluster barrier each block takes its
// share of the k range: it reads Y_q[k] of every block through distributed
// shared memory, forms the CL-point combinations (all frequencies k + M m of
// all lines of the item are then in one thread), applies the Gamma step, runs
// the inverse combination and writes the results back to the same remote slots
// it read.  Every slot is read and rewritten by exactly one thread, so a second
// cluster barrier suffices before the local inverse M-point transforms.  The
// transforms run in place in the slot's buffer (the W lines interleaved), so
// three buffers fit: a producer warp stores each slot by TMA as soon as its
// inverse transforms are done and fetches the slot three places ahead into the
// buffer once the store has read it, so loads and stores run under the work of
// the next slots.  Lines of an item: the d = 2 component planes (complex
// layout) or the two half-spectrum planes (packed layout) of W adjacent columns.
//
// Staging the same tiles with one 8-byte copy per thread and row segment was
// limited by the number of requests an SM keeps in flight; a TMA box is one
// request for the whole tile.
#pragma once

#include <cooperative_groups.h>

#include "lsfft_kernels.cuh"

namespace lsfft {

template <typename T, int N>
struct CluCfg {
    // blocks per cluster: pairs move a third less data through distributed
    // shared memory per column than groups of 4 and tile all 152 SMs
    static constexpr int CL = 2;
    static constexpr int M = N / CL;
    static constexpr int CS = (int)sizeof(cx<T>);
    static constexpr int W = 16 / CS;                  // adjacent columns per item: 16-byte row segments
    static constexpr int LS = 2;                       // slots per item: the two planes
    static constexpr int E = sizeof(T) == 4 ? 16 : 8;
    static constexpr int RMAX = sizeof(T) == 4 ? 16 : 8;
    static constexpr int TL = M >= E ? M / E : 1;      // threads per line
    static constexpr int COMPUTE = cmin(512, LS * W * TL);   // threads that transform and exchange
    static constexpr int THREADS = COMPUTE + 32;       // + one producer warp for the TMA traffic
    static constexpr int SPR = COMPUTE / (W * TL);     // slots per round
    static constexpr int ROUNDS = LS / (SPR > 0 ? SPR : 1);
    static constexpr int BJ = 256;                     // rows of the inner TMA box dimension
    static constexpr int EPC = CS / 8;                 // 8-byte tensor elements per complex value
    static constexpr int SLOT_BYTES = M * W * CS;      // one plane of an item, dense [j][w]
    // a slot buffer also holds its W lines' transforms in place: padded
    // positions (one slot per 16), the W lines interleaved position by position
    static constexpr int PP = (M + M / 16 + 7) / 8 * 8;
    static constexpr int BUF = (PP * W * CS + 1023) / 1024 * 1024;
    static constexpr int NB = 3;                       // rotating slot buffers
    static constexpr int SLOT_WARPS = W * TL / 32;     // warps that transform one slot
    static constexpr int SMEM = NB * BUF + 64;         // + six mbarriers
    // 2048-point columns fit the plain strided pass (two 16-byte columns per item),
    // measured 30 % faster there; the cluster pass takes 4096 and 8192
    static constexpr bool SUPPORTED = N >= 4096 && SMEM <= 227 * 1024 && SPR >= 1 && LS % SPR == 0 &&
                                      M % BJ == 0 && COMPUTE == SPR * W * TL && (W * TL) % 32 == 0;
};

template <typename T, int N>
__global__ void __cluster_dims__(CluCfg<T, N>::CL, 1, 1) __launch_bounds__(CluCfg<T, N>::THREADS, 1)
col_pass_cluster(const __grid_constant__ PassArgs<T> A) {
    namespace cg = cooperative_groups;
    using Cfg = CluCfg<T, N>;
    using C = cx<T>;
    constexpr int CL = Cfg::CL, M = Cfg::M, W = Cfg::W, LS = Cfg::LS, NB = Cfg::NB;
    constexpr int E = Cfg::E, TL = Cfg::TL, SPR = Cfg::SPR, EPC = Cfg::EPC, BJ = Cfg::BJ;
    constexpr int COMPUTE = Cfg::COMPUTE, BUFC = Cfg::BUF / Cfg::CS;   // buffer size in values
    constexpr int KQ = M / CL;                         // k range owned by one block in the exchange
    static_assert(M % BJ == 0, "rows of a block must fill whole TMA boxes");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    pdl_wait();
    if (A.pdl_early) pdl_trigger();
    if (A.ctrl->skipB) return;                         // uniform over the grid: no barrier is reached

    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int64_t cid = blockIdx.x / CL, ncl = gridDim.x / CL;
    C* Y = reinterpret_cast<C*>(smem_raw);             // NB buffers of BUFC values
    const bool producer = threadIdx.x >= COMPUTE;
    // transform threads -> (slot within the round, line position t, column w), columns fastest
    const int w = threadIdx.x % W;
    const int t = (threadIdx.x / W) % TL;
    const int sl = (threadIdx.x / (W * TL)) % SPR;
    // mbarriers: full[b] (TMA load landed) at bar0 + 8 b, done[b] (slot transformed) at bar0 + 24 + 8 b
    const uint32_t bar0 = smem_u32(smem_raw + NB * Cfg::BUF);
    const CUtensorMap* map = &A.tmap;
    // n_inner need not be a multiple of W (the half-spectrum planes hold
    // n_x/2 + 1 columns within a padded pitch): the last item runs into padding
    const int64_t n_items = (A.n_inner + W - 1) / W;
    const int64_t my_items = cid < n_items ? (n_items - cid + ncl - 1) / ncl : 0;
    const int64_t QN = 2 * my_items;                   // slots of this cluster, in order q = 2 it + s
    const bool leader = threadIdx.x == COMPUTE;        // lane 0 of the producer warp

    C* Yr[CL];                                          // buffer 0 of every block of the cluster
#pragma unroll
    for (int p = 0; p < CL; ++p) Yr[p] = cluster.map_shared_rank(Y, p);

    // slot q = 2 it + s (item cid + it ncl, plane s) lives in buffer q % NB
    auto load_q = [&](int64_t qq) {                     // producer only
        const int b = (int)(qq % NB);
        const int64_t item = cid + (qq / 2) * ncl;
        mbar_expect_tx(bar0 + 8 * b, Cfg::SLOT_BYTES + A.extra_tx);
        tma_load_5d(smem_u32(Y + b * BUFC), map, (int)(item * W * EPC), q, 0, 0, (int)(qq & 1), bar0 + 8 * b);
    };
    auto store_q = [&](int64_t qq) {                    // producer only
        const int b = (int)(qq % NB);
        const int64_t item = cid + (qq / 2) * ncl;
        tma_store_5d(map, (int)(item * W * EPC), q, 0, 0, (int)(qq & 1), smem_u32(Y + b * BUFC));
        bulk_commit();
    };
    // W_N^(p k) for p = 0..CL-1 (forward sign)
    auto twiddles = [&](int k, C (&tw)[CL]) {
        tw[0] = mkc((T)1, (T)0);
        if constexpr (sizeof(T) == 4) {
            float s, c;
            sincospif(2.0f * (float)k / (float)N, &s, &c);
            tw[1] = mkc(c, -s);
        } else {
            tw[1] = A.tw[k];
        }
#pragma unroll
        for (int p = 2; p < CL; ++p) tw[p] = cmul(tw[p - 1], tw[1]);
    };

    if (threadIdx.x == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(bar0 + 8 * b, 1);
            mbar_init(bar0 + 24 + 8 * b, Cfg::SLOT_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool fault = false;
    int64_t item = cid;
    if (producer) {
        // The producer warp: stores each slot as soon as its transforms are done
        // and fetches slot q + NB into the buffer once the store has read it.
        if (leader)
            for (int64_t qq = 0; qq < NB && qq < QN; ++qq) load_q(qq);
        for (uint32_t it = 0; item < n_items; item += ncl, ++it) {
            cluster.sync();   // the transform threads' first barrier of this item
            cluster.sync();   // ... and their second
            if (leader) {
                for (int s = 0; s < LS; ++s) {
                    const int64_t qq = 2 * (int64_t)it + s;
                    const int b = (int)(qq % NB);
                    if (!mbar_wait(bar0 + 24 + 8 * b, (uint32_t)((qq / NB) & 1), A.wait_limit)) fault = true;
                    store_q(qq);
                    bulk_wait_read(0);
                    if (qq + NB < QN) load_q(qq + NB);
                }
            }
            __syncwarp();
        }
        if (leader) bulk_wait_all();
    } else {
        for (uint32_t it = 0; item < n_items; item += ncl, ++it) {
            // 1. local forward M-point transforms, in place in the slot's buffer;
            //    round rd covers slots rd*SPR .. rd*SPR + SPR - 1
            for (int rd = 0; rd < Cfg::ROUNDS; ++rd) {
                const int s = rd * SPR + sl;
                const int64_t qq = 2 * (int64_t)it + s;
                const int b = (int)(qq % NB);
                if (!mbar_wait(bar0 + 8 * b, (uint32_t)((qq / NB) & 1), A.wait_limit)) fault = true;
                C* Yb = Y + b * BUFC;
                C v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = Yb[(t + TL * m) * W + w];
                LineFFT<T, M, E, Cfg::RMAX, false, false, COMPUTE, W>::run(v, Yb + w, t, A.tw, CL);
                line_sync<COMPUTE>();   // every thread has read its last-stage inputs
#pragma unroll
                for (int m = 0; m < E; ++m) Yb[(t + TL * m) * W + w] = v[m];
            }
            cluster.sync();
            // 2. exchange: combine, Gamma, inverse combine over the owned k range
            const int b0 = (int)((2 * (int64_t)it) % NB), b1 = (int)((2 * (int64_t)it + 1) % NB);
            for (int idx = threadIdx.x; idx < W * KQ; idx += COMPUTE) {
                const int wc = idx % W, k = q * KQ + idx / W;
                C tw[CL];
                twiddles(k, tw);
                C x[LS][CL];
#pragma unroll
                for (int s = 0; s < LS; ++s) {
                    const int off = (s == 0 ? b0 : b1) * BUFC + k * W + wc;
                    C y[CL];
#pragma unroll
                    for (int p = 0; p < CL; ++p) y[p] = cmul(Yr[p][off], tw[p]);
                    dft<CL, false, false>(y);   // x[m] = sum_p y[p] W_CL^(p m)
#pragma unroll
                    for (int m = 0; m < CL; ++m) x[s][m] = y[m];
                }
                const int kx = (int)(item * W + wc);
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
                    const int off = (s == 0 ? b0 : b1) * BUFC + k * W + wc;
                    // inverse CL-point DFT over m, then * conj W_N^(p k)
                    dft<CL, true, false>(x[s]);
#pragma unroll
                    for (int p = 0; p < CL; ++p) Yr[p][off] = cmulc(x[s][p], tw[p]);
                }
            }
            cluster.sync();
            // 3. local inverse M-point transforms in place; each slot is handed to
            //    the producer warp when its warps are done with it
            for (int rd = 0; rd < Cfg::ROUNDS; ++rd) {
                const int s = rd * SPR + sl;
                const int b = (int)((2 * (int64_t)it + s) % NB);
                C* Yb = Y + b * BUFC;
                C v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = Yb[(t + TL * m) * W + w];
                LineFFT<T, M, E, Cfg::RMAX, true, false, COMPUTE, W>::run(v, Yb + w, t, A.tw, CL);
                line_sync<COMPUTE>();
#pragma unroll
                for (int m = 0; m < E; ++m) Yb[(t + TL * m) * W + w] = v[m];
                fence_proxy_async_smem();   // the TMA store reads what the threads wrote
                __syncwarp();
                if ((threadIdx.x & 31) == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar0 + 24 + 8 * b) : "memory");
            }
        }
    }
    if (fault) atomicExch(&A.ctrl->fault, 1);
    cluster.sync();   // no block leaves while a peer may still address its shared memory
}

}  // namespace lsfft
