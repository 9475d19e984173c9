// Host-side launch helpers: one switch per (precision, d) over the line length.
// Each lsfft_inst_*.cu translation unit expands one LSFFT_DEFINE_*_DISPATCH
// and so compiles one family of kernels; the build runs them in parallel.
#pragma once

#include <cuda_runtime.h>

#include "lsfft_cluster.cuh"
#include "lsfft_kernels.cuh"
#include "lsfft_misc.h"

namespace lsfft {

template <typename T, int N, int D>
cudaError_t row_op(int op, const PassArgs<T>* A, cudaStream_t s, Geom* g) {
    using Cfg = RowCfg<T, N, D>;
    static int bps = 0;   // resident blocks per SM, set by OP_PREPARE
    if constexpr (!Cfg::SUPPORTED) {
        if (op == OP_QUERY) g->supported = false;
        return op == OP_QUERY ? cudaSuccess : cudaErrorInvalidValue;
    } else {
        if (op == OP_QUERY) {
            g->threads = Cfg::THREADS;
            g->per_block = Cfg::LPB;
            g->smem = Cfg::SMEM;
            g->blocks_per_sm = bps;
            g->supported = true;
            return cudaSuccess;
        }
        if (op == OP_PREPARE) {
            cudaError_t e = cudaFuncSetAttribute(row_pass<T, N, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg::SMEM);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, row_pass<T, N, D>, Cfg::THREADS, Cfg::SMEM);
        }
        return launch_pdl(row_pass<T, N, D>, dim3((unsigned)A->grid_blocks), dim3(Cfg::THREADS), Cfg::SMEM, s,
                          A->pdl, *A);
    }
}

template <typename T, int N, int D>
cudaError_t col_op(int op, const PassArgs<T>* A, cudaStream_t s, Geom* g) {
    if constexpr (D == 2 && CluCfg<T, N>::SUPPORTED) {
        // long 2-D columns (4096, 8192): cluster kernel (item = W adjacent columns, both planes)
        using Cfg = CluCfg<T, N>;
        static int max_clusters = 0;
        if (op == OP_QUERY) {
            g->threads = Cfg::THREADS;
            g->per_block = Cfg::W;
            g->smem = Cfg::SMEM;
            g->blocks_per_sm = 1;
            g->cluster = Cfg::CL;
            g->max_clusters = max_clusters;
            g->supported = true;
            return cudaSuccess;
        }
        if (op == OP_PREPARE) {
            cudaError_t e = cudaFuncSetAttribute(col_pass_cluster<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg::SMEM);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(Cfg::CL, 1, 1);
            cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
            cfg.dynamicSmemBytes = Cfg::SMEM;
            return cudaOccupancyMaxActiveClusters(&max_clusters, (const void*)col_pass_cluster<T, N>, &cfg);
        }
        return launch_pdl(col_pass_cluster<T, N>, dim3((unsigned)A->grid_blocks), dim3(Cfg::THREADS), Cfg::SMEM, s,
                          A->pdl, *A);
    } else {
        using Cfg = ColCfg<T, N, D>;
        static int bps = 0;
        if constexpr (!Cfg::SUPPORTED) {
            if (op == OP_QUERY) g->supported = false;
            return op == OP_QUERY ? cudaSuccess : cudaErrorInvalidValue;
        } else {
            if (op == OP_QUERY) {
                g->threads = Cfg::THREADS;
                g->per_block = Cfg::COLS;
                g->smem = Cfg::SMEM;
                g->blocks_per_sm = bps;
                g->cluster = 0;
                g->supported = true;
                return cudaSuccess;
            }
            if (op == OP_PREPARE) {
                cudaError_t e = cudaFuncSetAttribute(col_pass<T, N, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     Cfg::SMEM);
                if (e != cudaSuccess) return e;
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, col_pass<T, N, D>, Cfg::THREADS,
                                                                     Cfg::SMEM);
            }
            return launch_pdl(col_pass<T, N, D>, dim3((unsigned)A->grid_blocks), dim3(Cfg::THREADS), Cfg::SMEM, s,
                          A->pdl, *A);
        }
    }
}

// Switches over log2(N); d = 2 supports N = 16..8192, d = 3 supports N = 16..512.
// The dispatch templates are declared in lsfft_misc.h.

#define LSFFT_SWITCH_2D(FN)                                  \
    switch (logn) {                                          \
        case 4: return FN<T, 16, D>(op, A, s, g);            \
        case 5: return FN<T, 32, D>(op, A, s, g);            \
        case 6: return FN<T, 64, D>(op, A, s, g);            \
        case 7: return FN<T, 128, D>(op, A, s, g);           \
        case 8: return FN<T, 256, D>(op, A, s, g);           \
        case 9: return FN<T, 512, D>(op, A, s, g);           \
        case 10: return FN<T, 1024, D>(op, A, s, g);         \
        case 11: return FN<T, 2048, D>(op, A, s, g);         \
        case 12: return FN<T, 4096, D>(op, A, s, g);         \
        case 13: return FN<T, 8192, D>(op, A, s, g);         \
        default: if (g) g->supported = false; return cudaErrorInvalidValue; \
    }

#define LSFFT_SWITCH_3D(FN)                                  \
    switch (logn) {                                          \
        case 4: return FN<T, 16, D>(op, A, s, g);            \
        case 5: return FN<T, 32, D>(op, A, s, g);            \
        case 6: return FN<T, 64, D>(op, A, s, g);            \
        case 7: return FN<T, 128, D>(op, A, s, g);           \
        case 8: return FN<T, 256, D>(op, A, s, g);           \
        case 9: return FN<T, 512, D>(op, A, s, g);           \
        default: if (g) g->supported = false; return cudaErrorInvalidValue; \
    }

#define LSFFT_DEFINE_ROW_DISPATCH(TT, DD)                                                          \
    template <>                                                                                    \
    cudaError_t row_dispatch<TT, DD>(int logn, int op, const PassArgs<TT>* A, cudaStream_t s,     \
                                     Geom* g) {                                                    \
        using T = TT;                                                                              \
        constexpr int D = DD;                                                                      \
        if constexpr (D == 2) { LSFFT_SWITCH_2D(row_op) } else { LSFFT_SWITCH_3D(row_op) }       \
    }

#define LSFFT_DEFINE_COL_DISPATCH(TT, DD)                                                          \
    template <>                                                                                    \
    cudaError_t col_dispatch<TT, DD>(int logn, int op, const PassArgs<TT>* A, cudaStream_t s,     \
                                     Geom* g) {                                                    \
        using T = TT;                                                                              \
        constexpr int D = DD;                                                                      \
        if constexpr (D == 2) { LSFFT_SWITCH_2D(col_op) } else { LSFFT_SWITCH_3D(col_op) }       \
    }

}  // namespace lsfft
