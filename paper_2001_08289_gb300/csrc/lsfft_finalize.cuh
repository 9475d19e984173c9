// Scalar recurrence of one iteration (FP64, one thread): sigma_k of Eq. J13
// projected on e from the volume sums, the relative changes of sigma_k and of
// <|E|^2>, the history entry, and the stop rule (K consecutive changes below
// tol, divergence, iteration cap).  tot[4c + 0..3] = sums of Re, Im E_c and
// Re, Im J_c; tot[4d] = sum of |E|^2 (all over the N voxels).  final_mode: the
// output pass of a finished solve (history and averages only).
#pragma once

#include <math.h>

#include "lsfft_params.h"

namespace lsfft {

__device__ __forceinline__ void finalize_update(const double* tot, const SchemeParams& P, Ctrl* ctrl, double* hist,
                                                int final_mode) {
    const int d = P.d;
    // the control block's inputs, loaded together before any store (the stores to
    // hist and ctrl could otherwise alias them and force one round trip each)
    const int k = ctrl->iter;
    const int run0 = ctrl->run;
    const double prev_re = ctrl->prev[0], prev_im = ctrl->prev[1];
    const double prev_norm = ctrl->prev_norm;
    const double norm0_in = ctrl->norm0;
    // sigma_k = (<J>.e) / (<E>.e); the 1/N factors cancel
    double je_re = 0, je_im = 0, ee_re = 0, ee_im = 0;
    for (int c = 0; c < d; ++c) {
        ee_re += tot[4 * c + 0] * P.e[c];
        ee_im += tot[4 * c + 1] * P.e[c];
        je_re += tot[4 * c + 2] * P.e[c];
        je_im += tot[4 * c + 3] * P.e[c];
    }
    // (one reciprocal and one square root: FP64 division and sqrt are long
    // instruction sequences on this GPU's narrow FP64 pipe, and this thread is
    // on every iteration's critical path)
    const double inv_den = 1.0 / (ee_re * ee_re + ee_im * ee_im);
    const double s_re = (je_re * ee_re + je_im * ee_im) * inv_den;
    const double s_im = (je_im * ee_re - je_re * ee_im) * inv_den;
    const double norm = tot[4 * d] * P.inv_ntot;
    const double mag2 = s_re * s_re + s_im * s_im;
    double rel = INFINITY;
    if (k >= 1 && mag2 != 0.0) {
        const double dr = s_re - prev_re, di = s_im - prev_im;
        rel = sqrt((dr * dr + di * di) / mag2);
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
    // relative change of <|E|^2>: the field must settle as well as sigma_*
    const double nrel = (k >= 1 && norm != 0.0) ? fabs(norm - prev_norm) / norm : INFINITY;
    ctrl->prev[0] = s_re;
    ctrl->prev[1] = s_im;
    ctrl->prev_norm = norm;
    if (final_mode) return;
    const double norm0 = k == 0 ? norm : norm0_in;
    if (k == 0) ctrl->norm0 = norm;
    const int run = (rel < P.tol && nrel < P.tol) ? run0 + 1 : 0;
    ctrl->run = run;
    const bool diverged = !isfinite(s_re) || !isfinite(s_im) || !isfinite(norm) ||
                          norm > DIVERGENCE_FACTOR * norm0;
    if (diverged) {
        ctrl->status = ST_DIVERGED;
        ctrl->done = 1;
    } else if (run >= P.consecutive) {
        ctrl->status = ST_OK;
        ctrl->done = 1;
    } else if (k + 1 >= P.max_iter) {
        ctrl->status = ST_NOTCONV;
        ctrl->done = 1;
    }
    ctrl->iter = k + 1;
}

}  // namespace lsfft
