// Strided (y) pass for long 2-D columns on a thread-block cluster, with its
// tiles moved by the tensor memory accelerator (TMA).
//
// One SM cannot stage enough adjacent columns of length N >= 4096, so a
// cluster of CL blocks shares the work of an item of W adjacent columns
// (16-byte row segments for CL = 2: W = 2 in FP32, 1 in FP64; 32-byte ones
// for CL = 4).  With rows r = q + CL j (block rank q, j < M = N/CL) the length-N DFT
// splits as
//     X[k + M m] = sum_q W_CL^(q m) W_N^(q k) Y_q[k],
//     Y_q[k]     = sum_j x[q + CL j] W_M^(j k),            k < M, m < CL.
// Block q fetches its rows of each plane of the item with one TMA box (rows
// q + CL j, W columns; shared-memory layout [j][w]), computes the M-point
// transforms Y_q in place, and after one cluster barrier each block takes a
// quarter of the k range: it reads Y_q[k] of every block through distributed
// shared memory, forms the CL-point combinations (all frequencies k + M m of
// all lines of the item are then in one thread), applies the Gamma step, runs
// the inverse combination and writes the results back to the same remote slots
// it read.  Every slot is read and rewritten by exactly one thread, so a second
// cluster barrier suffices before the local inverse M-point transforms.  Each
// plane goes back by one TMA store as soon as its inverse transforms are done,
// and the next item's plane is fetched into the same buffer as soon as that
// store has read it, so loads and stores run under the transforms.  Lines of an
// item: the d = 2 component planes (complex layout) or the two half-spectrum
// planes (packed layout) of W adjacent columns.
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
    // blocks per cluster: the code also runs with 4 (32-byte row segments), but
    // pairs move a third less data through distributed shared memory per column
    // and tile all 152 SMs; measured 13 % faster at 8192^2
    static constexpr int CL = 2;
    static constexpr int M = N / CL;
    static constexpr int CS = (int)sizeof(cx<T>);
    static constexpr int ROWB = CL == 4 ? 32 : 16;     // bytes of a row segment of an item
    static constexpr int W = ROWB / CS;                // adjacent columns per item
    static constexpr int LS = 2;                       // slots per column: the two planes
    static constexpr int LINES = LS * W;
    static constexpr int E = sizeof(T) == 4 ? 16 : 8;
    static constexpr int RMAX = sizeof(T) == 4 ? 16 : 8;
    static constexpr int TL = M >= E ? M / E : 1;      // threads per line (only N >= 4096 is launched)
    static constexpr int COMPUTE = cmin(512, LINES * TL);   // threads that transform and exchange
    static constexpr int THREADS = COMPUTE + 32;       // + one producer warp for the TMA traffic
    static constexpr int G = COMPUTE / TL;             // lines transformed concurrently
    static constexpr int SPR = G / W;                  // slots per round
    static constexpr int ROUNDS = LS / (SPR > 0 ? SPR : 1);
    static constexpr int BJ = 256;                     // rows of the inner TMA box dimension
    static constexpr int EPC = CS / 8;                 // 8-byte tensor elements per complex value
    static constexpr int SLOT_BYTES = M * W * CS;      // one plane of an item: [j][w]
    // exchange line pitch: a multiple of 8 but not of 16 elements, so that the
    // lines w and w + 1 of a warp at equal positions fall into disjoint banks
    static constexpr int XP = roundup16(M + M / 16) + 8;
    static constexpr int Y_BYTES = LS * SLOT_BYTES;
    static constexpr int SLOT_WARPS = W * TL / 32;     // warps that transform one slot
    static constexpr int SMEM = Y_BYTES + G * XP * CS + 64;   // + four mbarriers
    // 2048-point columns fit the plain strided pass (two 16-byte columns per item),
    // measured 30 % faster there than on clusters; the cluster pass takes 4096 and 8192
    static constexpr bool SUPPORTED = N >= 4096 && SMEM <= 227 * 1024 && SPR >= 1 && G == SPR * W &&
                                      LS % SPR == 0 && M % BJ == 0 && COMPUTE == G * TL &&
                                      (W * TL) % 32 == 0;
};

template <typename T, int N>
__global__ void __cluster_dims__(CluCfg<T, N>::CL, 1, 1) __launch_bounds__(CluCfg<T, N>::THREADS, 1)
col_pass_cluster(const __grid_constant__ PassArgs<T> A) {
    namespace cg = cooperative_groups;
    using Cfg = CluCfg<T, N>;
    using C = cx<T>;
    constexpr int CL = Cfg::CL, M = Cfg::M, W = Cfg::W, LS = Cfg::LS;
    constexpr int E = Cfg::E, TL = Cfg::TL, XP = Cfg::XP, SPR = Cfg::SPR, EPC = Cfg::EPC, BJ = Cfg::BJ;
    constexpr int KQ = M / CL;                         // k range owned by one block in the exchange
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (A.ctrl->skipB) return;                         // uniform over the grid: no barrier is reached

    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int64_t cid = blockIdx.x / CL, ncl = gridDim.x / CL;
    C* Y = reinterpret_cast<C*>(smem_raw);             // [LS][M][W]
    constexpr int COMPUTE = Cfg::COMPUTE;
    const bool producer = threadIdx.x >= COMPUTE;
    // transform threads -> (slot within the round, line position t, column w), columns fastest
    const int w = threadIdx.x % W;
    const int t = (threadIdx.x / W) % TL;
    const int sl = (threadIdx.x / (W * TL)) % SPR;
    C* Xg = reinterpret_cast<C*>(smem_raw + Cfg::Y_BYTES) + (sl * W + w) * XP;
    // mbarriers: full[s] (TMA load landed) at bar0 + 8 s, done[s] (slot transformed) at bar0 + 16 + 8 s
    const uint32_t bar0 = smem_u32(smem_raw + Cfg::Y_BYTES + Cfg::G * XP * Cfg::CS);
    const CUtensorMap* map = &A.tmap;
    // n_inner need not be a multiple of W (the half-spectrum planes hold
    // n_x/2 + 1 columns within a padded pitch): the last item runs into padding
    const int64_t n_items = (A.n_inner + W - 1) / W;
    const bool leader = threadIdx.x == COMPUTE;         // lane 0 of the producer warp

    C* Yr[CL];                                          // the item buffers of every block of the cluster
#pragma unroll
    for (int p = 0; p < CL; ++p) Yr[p] = cluster.map_shared_rank(Y, p);

    auto load_slot = [&](int64_t item, int s) {         // producer only
        const uint32_t bar = bar0 + 8 * s;
        mbar_expect_tx(bar, Cfg::SLOT_BYTES + A.extra_tx);
        tma_load_5d(smem_u32(Y) + s * Cfg::SLOT_BYTES, map, (int)(item * W * EPC), q, 0, 0, s, bar);
    };
    auto store_slot = [&](int64_t item, int s) {        // producer only
        tma_store_5d(map, (int)(item * W * EPC), q, 0, 0, s, smem_u32(Y) + s * Cfg::SLOT_BYTES);
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
    static_assert(M % BJ == 0, "rows of a block must fill whole TMA boxes");

    if (threadIdx.x == 0) {
        for (int s = 0; s < LS; ++s) {
            mbar_init(bar0 + 8 * s, 1);
            mbar_init(bar0 + 16 + 8 * s, Cfg::SLOT_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool fault = false;
    int64_t item = cid;
    if (producer) {
        // The producer warp: stores each slot as soon as its transforms are done,
        // and fetches the next item's tile into it once the store has read it.
        if (leader && item < n_items)
            for (int s = 0; s < LS; ++s) load_slot(item, s);
        for (uint32_t it = 0; item < n_items; item += ncl, ++it) {
            const int64_t next = item + ncl;
            cluster.sync();   // the transform threads' first barrier of this item
            cluster.sync();   // ... and their second
            if (leader) {
                for (int s = 0; s < LS; ++s) {
                    if (!mbar_wait(bar0 + 16 + 8 * s, it & 1u, A.wait_limit)) fault = true;
                    store_slot(item, s);
                    bulk_wait_read(0);
                    if (next < n_items) load_slot(next, s);
                }
            }
            __syncwarp();
        }
        if (leader) bulk_wait_all();
    } else {
        for (uint32_t it = 0; item < n_items; item += ncl, ++it) {
            // 1. local forward M-point transforms in place; round rd covers slots
            //    rd*SPR .. rd*SPR + SPR - 1 and starts when they have landed
            for (int rd = 0; rd < Cfg::ROUNDS; ++rd) {
                const int s = rd * SPR + sl;
                if (!mbar_wait(bar0 + 8 * s, it & 1u, A.wait_limit)) fault = true;
                C* Ys = Y + s * M * W;
                C v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = Ys[(t + TL * m) * W + w];
                LineFFT<T, M, E, Cfg::RMAX, false, false, COMPUTE>::run(v, Xg, t, A.tw, CL);
#pragma unroll
                for (int m = 0; m < E; ++m) Ys[(t + TL * m) * W + w] = v[m];
            }
            cluster.sync();
            // 2. exchange: combine, Gamma, inverse combine over the owned k range
            for (int idx = threadIdx.x; idx < W * KQ; idx += COMPUTE) {
                const int wc = idx % W, k = q * KQ + idx / W;
                C tw[CL];
                twiddles(k, tw);
                C x[LS][CL];
#pragma unroll
                for (int s = 0; s < LS; ++s) {
                    C y[CL];
#pragma unroll
                    for (int p = 0; p < CL; ++p) y[p] = cmul(Yr[p][(s * M + k) * W + wc], tw[p]);
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
                    // inverse CL-point DFT over m, then * conj W_N^(p k)
                    dft<CL, true, false>(x[s]);
#pragma unroll
                    for (int p = 0; p < CL; ++p) Yr[p][(s * M + k) * W + wc] = cmulc(x[s][p], tw[p]);
                }
            }
            cluster.sync();
            // 3. local inverse M-point transforms in place; each slot is handed to
            //    the producer warp when its warps are done with it
            for (int rd = 0; rd < Cfg::ROUNDS; ++rd) {
                const int s = rd * SPR + sl;
                C* Ys = Y + s * M * W;
                C v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = Ys[(t + TL * m) * W + w];
                LineFFT<T, M, E, Cfg::RMAX, true, false, COMPUTE>::run(v, Xg, t, A.tw, CL);
#pragma unroll
                for (int m = 0; m < E; ++m) Ys[(t + TL * m) * W + w] = v[m];
                fence_proxy_async_smem();   // the TMA store reads what the threads wrote
                __syncwarp();
                if ((threadIdx.x & 31) == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar0 + 16 + 8 * s) : "memory");
            }
        }
    }
    if (fault) atomicExch(&A.ctrl->fault, 1);
    cluster.sync();   // no block leaves while a peer may still address its shared memory
}

}  // namespace lsfft
