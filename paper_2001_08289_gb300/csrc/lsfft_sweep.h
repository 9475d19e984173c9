// Job descriptors of the persistent batch executor (lsfft_sweep.cu), shared
// by the host code that fills them and the kernel that runs them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lsfft_kernels.cuh"
#include "lsfft_params.h"

namespace lsfft {

// One solve: written by the host before the launch; the kernel updates ctrl,
// word, completed and finished, and the buffers it points to.
struct SweepJob {
    float2* X;               // state, complex planes [2][N] (x-spectra between passes)
    float2* S;               // substituted schemes: S on phase-1 voxels [2][N], else null
    float2* T;               // EM in H'': T [2][N], else null
    float2* Eout;            // field of the final iterate [2][N]
    const uint8_t* mask;     // [N]
    const float2* fd[2];     // forward-difference symbol per axis (FP32)
    double* partials;        // [row_items][9] volume sums of the last row pass
    double* hist;            // [(max_iter + 1) * HIST_STRIDE]
    KConst<float> k;         // scheme constants in FP32 (Gamma coefficients carry 1/N)
    SchemeParams prm;        // the same in FP64, for the scalar recurrence
    Ctrl ctrl;               // iteration count, stop rule, sigma_k, averages
    int nx, ny, lognx, logny;
    int row_items, col_items;
    unsigned long long word; // [63:40] epoch, [39:32] pass, [31:0] next item ticket
    unsigned int completed;  // items of the current epoch done
    int finished;            // output pass done: result complete
};

struct SweepGlobal {
    int jobs_done;
    int error;               // a block found nothing to claim for longer than the idle limit
};

int sweep_smem_bytes();
int sweep_threads();
int sweep_row_lpb(int n);    // rows per row item for lines of n points
int sweep_col_cols(int n);   // columns per column item for columns of n points
cudaError_t sweep_prepare(int* blocks_per_sm);
cudaError_t sweep_launch(SweepJob* jobs, int njobs, SweepGlobal* glob, int blocks, long long idle_limit_ns,
                         cudaStream_t s);

}  // namespace lsfft
