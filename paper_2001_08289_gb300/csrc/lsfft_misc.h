// Declarations of the launch helpers defined in lsfft_misc.cu and the
// lsfft_inst_*.cu translation units.
#pragma once

#include <cuda_runtime.h>

#include "lsfft_fft.cuh"
#include "lsfft_params.h"

namespace lsfft {

template <typename T> struct PassArgs;

// Launch geometry reported by the dispatch functions.
struct Geom {
    int threads = 0;     // threads per block
    int per_block = 0;   // rows (row pass) or line starts (strided pass) per block
    int smem = 0;        // dynamic shared memory bytes
    int blocks_per_sm = 0;   // resident blocks per SM (after OP_PREPARE)
    int cluster = 0;         // > 0: cluster kernel with this many blocks per cluster
    int max_clusters = 0;    // co-resident clusters (after OP_PREPARE)
    bool supported = false;
};

enum { OP_QUERY = 0, OP_PREPARE = 1, OP_LAUNCH = 2 };

template <typename T>
cudaError_t launch_init(cx<T>* X, cx<T>* S, cx<T>* Tf, const uint8_t* mask, const SchemeParams& prm, int64_t Ntot,
                        int d, int packed, const cx<T>* sigma, int sm_count, cudaStream_t s);

cudaError_t measure_fma_peak(int paired, int reps, double* tflops);
cudaError_t launch_finalize(const double* partials, int nblocks, int nv, const SchemeParams& prm, Ctrl* ctrl,
                            double* hist, int final_mode, int programmatic, cudaStream_t s);

// Copy `bytes` (a multiple of 8) from device memory to the device view of
// mapped pinned host memory with one small kernel on stream s.
cudaError_t launch_copy_words(void* dst, const void* src, size_t bytes, cudaStream_t s);

}  // namespace lsfft

namespace lsfft {
// Defined in the lsfft_inst_*.cu translation units.
template <typename T, int D>
cudaError_t row_dispatch(int logn, int op, const PassArgs<T>* A, cudaStream_t s, Geom* g);
template <typename T, int D>
cudaError_t col_dispatch(int logn, int op, const PassArgs<T>* A, cudaStream_t s, Geom* g);
template <> cudaError_t row_dispatch<float, 2>(int, int, const PassArgs<float>*, cudaStream_t, Geom*);
template <> cudaError_t row_dispatch<float, 3>(int, int, const PassArgs<float>*, cudaStream_t, Geom*);
template <> cudaError_t row_dispatch<double, 2>(int, int, const PassArgs<double>*, cudaStream_t, Geom*);
template <> cudaError_t row_dispatch<double, 3>(int, int, const PassArgs<double>*, cudaStream_t, Geom*);
template <> cudaError_t col_dispatch<float, 2>(int, int, const PassArgs<float>*, cudaStream_t, Geom*);
template <> cudaError_t col_dispatch<float, 3>(int, int, const PassArgs<float>*, cudaStream_t, Geom*);
template <> cudaError_t col_dispatch<double, 2>(int, int, const PassArgs<double>*, cudaStream_t, Geom*);
template <> cudaError_t col_dispatch<double, 3>(int, int, const PassArgs<double>*, cudaStream_t, Geom*);
// Split layout of long 2-D columns, FP32 packed fields (lsfft_inst_split.cu):
// row pass on row pairs of lines 2^logn, strided pass on columns of 2^logm = n_y / 2.
cudaError_t split_row_dispatch(int logn, int op, const PassArgs<float>* A, cudaStream_t s, Geom* g);
cudaError_t split_col_dispatch(int logm, int op, const PassArgs<float>* A, cudaStream_t s, Geom* g);
}  // namespace lsfft

namespace lsfft {
// Lanczos vector kernels (lsfft_misc.cu); `out` receives one FP64 scalar.
template <typename T>
cudaError_t lanczos_init(cx<T>* v, const uint8_t* mask, int64_t N, int d, const double* e, int blocks,
                         double* partials, double* out, cudaStream_t s);
template <typename T>
cudaError_t lanczos_dot(const cx<T>* a, const cx<T>* b, int64_t L, int blocks, double* partials, double* out,
                        cudaStream_t s);
template <typename T>
cudaError_t lanczos_axpy_norm(cx<T>* w, const cx<T>* v, const cx<T>* u, double alpha, double beta, int64_t L,
                              int blocks, double* partials, double* out, cudaStream_t s);
template <typename T>
cudaError_t lanczos_scale(cx<T>* dst, const cx<T>* src, double sc, int64_t L, int blocks, cudaStream_t s);
}  // namespace lsfft

namespace lsfft {
// Gradient of sigma_* and conversion of the per-voxel conductivity (lsfft_misc.cu).
template <typename T>
cudaError_t launch_gradient(const cx<T>* E, const uint8_t* mask, const cx<T>* sigma, double s1re, double s1im, int d,
                            int64_t N, double inv_ne2, cx<T>* grad, int blocks, double* partials, cudaStream_t s);
template <typename T>
cudaError_t launch_convert_field(cx<T>* dst, const double2* src, int64_t N, int sm_count, cudaStream_t s);
}  // namespace lsfft
