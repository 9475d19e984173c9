// Constants and control block shared by the host code and the kernels.
// All scalars are FP64 (the scheme coefficients and the scalar recurrence are
// computed on the host in double precision); kernels round them to the field
// precision where they multiply field values.
#pragma once

#include <stdint.h>

namespace lsfft {

enum { SCHEME_MS = 0, SCHEME_EM = 1, SCHEME_MS_SUB = 2, SCHEME_EM_SUB = 3, SCHEME_MATVEC = 4 };
enum { GREEN_TRIG = 0, GREEN_FD = 1 };
enum { MODE_ROW_FIRST = 0, MODE_ROW_ITER = 1, MODE_ROW_OUTPUT = 2 };
enum { MODE_COL_FWD = 0, MODE_COL_INV = 1, MODE_COL_GAMMA = 2 };
enum { ST_RUNNING = -1, ST_OK = 0, ST_NOTCONV = 3, ST_DIVERGED = 4 };

constexpr int HIST_STRIDE = 4;              // sigma re, sigma im, rel change, <|E|^2>
constexpr double DIVERGENCE_FACTOR = 1e12;  // <|E|^2> growth that counts as divergence

struct SchemeParams {
    int scheme, green, d, max_iter, consecutive, pad0;
    double tol;
    double inv_ntot;            // 1 / N
    double e[3];                // applied field
    double sigma1[2];
    // pointwise coefficients (complex as re, im)
    double a_in[2], a_out[2];   // MS: sigma/sigma_0 - 1 per phase; EM: W per phase
    double k1[2], k2[2], k3[2]; // MS in H'': tau_Q = k1 c + k2 Q, tau_S = k3 c + k2 S
    double tm1p1[2];            // (t - 1) p_1
    double p1[2], p2[2], p3[2];
    double w[2];                // EM in H'': (1 - sqrt t)/(1 + sqrt t)
    double inv2s0[2];           // 1/(2 sigma_0) (EM) or 1/(2 sqrt t) (EM in H'')
    // Gamma step: out = a v + b Gamma v (k != 0); out = a0 v + ce e (k = 0), times 1/N
    double g_a[2], g_b[2], g_a0[2], g_ce[2];
    // initial state: Q = (phase 1 ? iq_in : iq_out) e, S = is_in e, T = it_in e on phase 1
    double iq_in[2], iq_out[2], is_in[2], it_in[2];
    // per-voxel conductivity mode (MS / EM only): reference medium sigma_0 and 1/sigma_0
    double s0[2], inv_s0[2];
};

struct Ctrl {
    int done;        // stop criterion met: later row passes and finalizes skip
    int skipB;       // set by a row pass (or finalize) that found `done`: later strided passes skip
    int iter;        // number of sigma_k evaluated so far
    int run;         // consecutive relative changes below tol
    int status;      // ST_*
    int fault;       // a bounded device wait gave up (the results are not valid)
    int pad1, pad2;
    double prev[2];  // sigma_{k-1}
    double prev_norm;   // <|E_{k-1}|^2>
    double norm0;    // <|E_0|^2>
    double sigma[2];
    double meanE[3][2], meanJ[3][2];
};

}  // namespace lsfft
