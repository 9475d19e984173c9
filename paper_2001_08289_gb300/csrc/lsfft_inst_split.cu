// Kernel family: the split layout of long 2-D columns (row pass on row pairs,
// strided pass on half-length columns), FP32 packed fields.
#include "lsfft_misc.h"
#include "lsfft_split.cuh"

namespace lsfft {

namespace {

template <int N, int SCH>
cudaError_t split_row_sch(int op, const PassArgs<float>* A, cudaStream_t s, Geom* g) {
    using Cfg = SplitRowCfg<N>;
    static int bps = 0;
    if constexpr (!Cfg::SUPPORTED) {
        if (op == OP_QUERY) g->supported = false;
        return op == OP_QUERY ? cudaSuccess : cudaErrorInvalidValue;
    } else {
        if (op == OP_QUERY) {
            g->threads = Cfg::THREADS;
            g->per_block = 1;   // one row pair per work item
            g->smem = Cfg::SMEM;
            g->blocks_per_sm = bps;
            g->supported = true;
            return cudaSuccess;
        }
        if (op == OP_PREPARE) {
            cudaError_t e = cudaFuncSetAttribute(row_pass_split<N, SCH>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, row_pass_split<N, SCH>, Cfg::THREADS, Cfg::SMEM);
            // resident blocks share the SM's 512 tensor-memory columns
            if (e == cudaSuccess && bps * Cfg::TMEM_COLS > 512) bps = 512 / Cfg::TMEM_COLS;
            return e;
        }
        return launch_pdl(row_pass_split<N, SCH>, dim3((unsigned)A->grid_blocks), dim3(Cfg::THREADS), Cfg::SMEM, s,
                          A->pdl, *A);
    }
}

// every scheme is prepared (OP_PREPARE) so that a later solve with another
// scheme finds its kernel ready; queries and launches go to the solve's scheme
template <int N>
cudaError_t split_row_op(int op, const PassArgs<float>* A, cudaStream_t s, Geom* g) {
    if (op == OP_PREPARE) {
        cudaError_t e = split_row_sch<N, SCHEME_MS>(op, A, s, g);
        if (e == cudaSuccess) e = split_row_sch<N, SCHEME_EM>(op, A, s, g);
        if (e == cudaSuccess) e = split_row_sch<N, SCHEME_MS_SUB>(op, A, s, g);
        if (e == cudaSuccess) e = split_row_sch<N, SCHEME_EM_SUB>(op, A, s, g);
        return e;
    }
    const int sch = A ? A->k.scheme : SCHEME_MS;
    switch (sch) {
        case SCHEME_EM: return split_row_sch<N, SCHEME_EM>(op, A, s, g);
        case SCHEME_MS_SUB: return split_row_sch<N, SCHEME_MS_SUB>(op, A, s, g);
        case SCHEME_EM_SUB: return split_row_sch<N, SCHEME_EM_SUB>(op, A, s, g);
        default: return split_row_sch<N, SCHEME_MS>(op, A, s, g);
    }
}

template <int M>
cudaError_t split_col_op(int op, const PassArgs<float>* A, cudaStream_t s, Geom* g) {
    using Cfg = SplitColCfg<M>;
    static int bps = 0;
    if constexpr (!Cfg::SUPPORTED) {
        if (op == OP_QUERY) g->supported = false;
        return op == OP_QUERY ? cudaSuccess : cudaErrorInvalidValue;
    } else {
        if (op == OP_QUERY) {
            g->threads = Cfg::THREADS;
            g->per_block = Cfg::W;
            g->smem = Cfg::SMEM;
            g->blocks_per_sm = bps;
            g->supported = true;
            return cudaSuccess;
        }
        if (op == OP_PREPARE) {
            cudaError_t e = cudaFuncSetAttribute(col_pass_split<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg::SMEM);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, col_pass_split<M>, Cfg::THREADS, Cfg::SMEM);
        }
        return launch_pdl(col_pass_split<M>, dim3((unsigned)A->grid_blocks), dim3(Cfg::THREADS), Cfg::SMEM, s,
                          A->pdl, *A);
    }
}

}  // namespace

cudaError_t split_row_dispatch(int logn, int op, const PassArgs<float>* A, cudaStream_t s, Geom* g) {
    switch (logn) {
        case 12: return split_row_op<4096>(op, A, s, g);
        case 13: return split_row_op<8192>(op, A, s, g);
        default: if (g) g->supported = false; return cudaErrorInvalidValue;
    }
}

cudaError_t split_col_dispatch(int logm, int op, const PassArgs<float>* A, cudaStream_t s, Geom* g) {
    switch (logm) {
        case 11: return split_col_op<2048>(op, A, s, g);
        case 12: return split_col_op<4096>(op, A, s, g);
        default: if (g) g->supported = false; return cudaErrorInvalidValue;
    }
}

}  // namespace lsfft
