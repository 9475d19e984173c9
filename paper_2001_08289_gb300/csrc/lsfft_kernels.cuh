// Iteration kernels of the FFT Lippmann-Schwinger solver.
//
// State layout: the Q field (E for Moulinec-Suquet, the polarisation
// P = J + sigma_0 E for Eyre-Milton, the Q component of H'' for the substituted
// schemes) is stored component-planar, X[c][z][y][x], in the half-transformed
// domain (DFT along x done, y/z in real space) between iterations.  S and T,
// the extra components of H'' (Eq. J27, J36), live in real space and are
// touched only on phase-1 voxels (they vanish on phase 2).
//
// One iteration (2-D): row pass [inverse x-DFT -> pointwise scheme update and
// volume averages -> forward x-DFT], finalize (FP64 sums, sigma_k, stop rule),
// strided pass over y [forward y-DFT -> Gamma multiply per frequency -> inverse
// y-DFT].  3-D: row pass, finalize, y forward, z [forward, Gamma, inverse],
// y inverse.  Every pass is in place.
#pragma once

#include "lsfft_fft.cuh"
#include "lsfft_params.h"

namespace lsfft {

// ---------------------------------------------------------------------------
// Launch geometry, shared by the kernels and the host dispatch.
// ---------------------------------------------------------------------------
template <typename T, int N>
struct RowCfg {
    static constexpr int E0 = sizeof(T) == 4 ? 16 : 8;
    static constexpr int E = (N < E0) ? N : ((N / 512 > E0) ? N / 512 : E0);
    static constexpr int RMAX = sizeof(T) == 4 ? 16 : 8;
    static constexpr int TL = N / E;
    static constexpr int LPB = (256 / TL) > 0 ? (256 / TL) : 1;      // rows per block
    static constexpr int THREADS = LPB * TL;
    static constexpr int SMEM = LPB * LinePad<N>::size * (int)sizeof(cx<T>);
};

template <typename T, int N, int D>
struct ColCfg {
    static constexpr int CS = (int)sizeof(cx<T>);
    static constexpr int E0 = sizeof(T) == 4 ? 16 : 8;
    static constexpr int EMAX = sizeof(T) == 4 ? 32 : 16;
    static constexpr int COLMAX = sizeof(T) == 4 ? 4 : 2;    // 32-byte sectors
    static constexpr int RMAX = sizeof(T) == 4 ? 16 : 8;
    static constexpr int e_for(int cols) {
        return (N < E0) ? N : ((cols * D * N / 512 > E0) ? cols * D * N / 512 : E0);
    }
    static constexpr bool ok(int cols) {
        return e_for(cols) <= EMAX && cols * D * LinePad<N>::size * CS <= 200 * 1024;
    }
    static constexpr int COLS = ok(COLMAX) ? COLMAX : (ok(COLMAX / 2) ? COLMAX / 2 : 1);
    static constexpr int E = e_for(COLS);
    static constexpr int TL = N / E;
    static constexpr int G = COLS * D;                 // line groups per block
    static constexpr int THREADS = G * TL;
    static constexpr int SMEM = G * LinePad<N>::size * CS;
    static constexpr bool SUPPORTED = ok(COLS) && THREADS <= 1024;
};

// ---------------------------------------------------------------------------
// Reductions: thread-local FP64 -> warp shuffle -> block -> partials[block][NV]
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NV], double* __restrict__ out) {
    __shared__ double red[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double x = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][v] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double x = lane < nw ? red[lane][v] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) out[v] = x;
        }
    }
}

// ---------------------------------------------------------------------------
// Pointwise scheme update on one voxel (all d components).
//   q[c]   : Q component (real space) on entry; on exit the field handed to the
//            forward DFT (tau for MS-type schemes, W P for EM-type schemes).
//   S, T   : read and written in place on phase-1 voxels (substituted schemes).
//   E, J   : the physical fields of the current iterate, for the averages.
// ---------------------------------------------------------------------------
template <typename T, int D>
struct Pointwise {
    using C = cx<T>;
    C a_in, a_out, k1, k2, k3, p1, p2, p3, w, inv2s0, tm1p1, half;
    C s1;
    int scheme;

    __device__ __forceinline__ void load(const SchemeParams& P) {
        scheme = P.scheme;
        a_in = mkc((T)P.a_in[0], (T)P.a_in[1]);
        a_out = mkc((T)P.a_out[0], (T)P.a_out[1]);
        k1 = mkc((T)P.k1[0], (T)P.k1[1]);
        k2 = mkc((T)P.k2[0], (T)P.k2[1]);
        k3 = mkc((T)P.k3[0], (T)P.k3[1]);
        p1 = mkc((T)P.p1[0], (T)P.p1[1]);
        p2 = mkc((T)P.p2[0], (T)P.p2[1]);
        p3 = mkc((T)P.p3[0], (T)P.p3[1]);
        w = mkc((T)P.w[0], (T)P.w[1]);
        inv2s0 = mkc((T)P.inv2s0[0], (T)P.inv2s0[1]);
        tm1p1 = mkc((T)P.tm1p1[0], (T)P.tm1p1[1]);
        s1 = mkc((T)P.sigma1[0], (T)P.sigma1[1]);
    }

    // S/T pointers already offset to this voxel; comp stride cs.
    __device__ __forceinline__ void apply(C (&q)[D], bool inc, C* __restrict__ Sv, C* __restrict__ Tv,
                                          int64_t cs, C (&E)[D], C (&J)[D], bool write_st) const {
        if (scheme == SCHEME_MS) {
            const C a = inc ? a_in : a_out;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                E[c] = q[c];
                J[c] = inc ? cmul(s1, q[c]) : q[c];
                q[c] = cmul(a, q[c]);
            }
        } else if (scheme == SCHEME_EM) {
            const C W = inc ? a_in : a_out;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const C wp = cmul(W, q[c]);
                E[c] = cmul(csub(q[c], wp), inv2s0);
                J[c] = cscale(cadd(q[c], wp), (T)0.5);
                q[c] = wp;
            }
        } else if (scheme == SCHEME_MS_SUB) {
            if (inc) {
                C s[D];
#pragma unroll
                for (int c = 0; c < D; ++c) s[c] = Sv[c * cs];
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const C cc = cadd(cmul(p1, q[c]), cmul(p2, s[c]));
                    E[c] = q[c];
                    J[c] = cadd(q[c], cmul(tm1p1, cc));
                    const C tq = cadd(cmul(k1, cc), cmul(k2, q[c]));
                    const C ts = cadd(cmul(k3, cc), cmul(k2, s[c]));
                    q[c] = tq;
                    s[c] = cneg(ts);
                }
                if (write_st) {
#pragma unroll
                    for (int c = 0; c < D; ++c) Sv[c * cs] = s[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    E[c] = q[c];
                    J[c] = q[c];
                    q[c] = cmul(k2, q[c]);
                }
            }
        } else {   // SCHEME_EM_SUB
            if (inc) {
                C s[D], tt[D];
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    s[c] = Sv[c * cs];
                    tt[c] = Tv[c * cs];
                }
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const C cc = cadd(cadd(cmul(p1, q[c]), cmul(p2, s[c])), cmul(p3, tt[c]));
                    const C cc2 = cadd(cc, cc);
                    const C wq = cmul(w, csub(q[c], cmul(p1, cc2)));
                    const C ws = cmul(w, csub(s[c], cmul(p2, cc2)));
                    const C wt = cmul(w, csub(tt[c], cmul(p3, cc2)));
                    E[c] = cmul(csub(q[c], wq), inv2s0);
                    J[c] = cscale(cadd(q[c], wq), (T)0.5);
                    q[c] = wq;
                    s[c] = cneg(ws);
                    tt[c] = wt;
                }
                if (write_st) {
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        Sv[c * cs] = s[c];
                        Tv[c * cs] = tt[c];
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const C wq = cmul(w, q[c]);
                    E[c] = cmul(csub(q[c], wq), inv2s0);
                    J[c] = cscale(cadd(q[c], wq), (T)0.5);
                    q[c] = wq;
                }
            }
        }
    }
};

template <typename T>
struct PassArgs {
    cx<T>* X;                 // state, [D][Ntot]
    cx<T>* S;                 // H'' S component, [D][Ntot] (or null)
    cx<T>* Tf;                // H'' T component, [D][Ntot] (or null)
    cx<T>* Eout;              // output field, [D][Ntot] (row pass, output mode)
    const uint8_t* mask;      // [Ntot]
    const SchemeParams* prm;
    Ctrl* ctrl;
    double* partials;         // [gridDim.x][NV]
    const cx<T>* tw;          // FP64 twiddle table W_N^k of the pass's line length
    const cx<T>* fd[3];       // forward-difference symbol u_a(k), per axis
    int64_t Ntot;
    int64_t n_lines;          // row pass: number of rows
    int64_t ls;               // strided pass: element stride along the line
    int64_t n_inner;          // strided pass: contiguous line starts per outer slab
    int64_t outer_stride;     // strided pass: stride between outer slabs
    int64_t n_outer;          // strided pass: number of outer slabs
    int n[3];                 // grid extents (x, y, z)
    int line_axis;            // strided pass: 1 (y) or 2 (z)
    int mode;                 // PassMode
};

// ---------------------------------------------------------------------------
// Row pass: lines along x (contiguous).
// ---------------------------------------------------------------------------
template <typename T, int N, int D>
__global__ void __launch_bounds__(RowCfg<T, N>::THREADS)
row_pass(const PassArgs<T> A) {
    using Cfg = RowCfg<T, N>;
    using C = cx<T>;
    constexpr int E = Cfg::E, TL = Cfg::TL, NV = 4 * D + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int mode = A.mode;
    if (mode != MODE_ROW_OUTPUT && A.ctrl->done) return;

    const int g = threadIdx.x / TL, t = threadIdx.x % TL;
    C* sm = reinterpret_cast<C*>(smem_raw) + g * LinePad<N>::size;
    const int64_t row = (int64_t)blockIdx.x * Cfg::LPB + g;
    const bool active = row < A.n_lines;
    const int64_t base = row * N;

    Pointwise<T, D> pw;
    pw.load(*A.prm);

    C v[D][E];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[c][m] = active ? A.X[c * A.Ntot + base + t + TL * m] : mkc((T)0, (T)0);

    if (mode != MODE_ROW_FIRST) {
#pragma unroll
        for (int c = 0; c < D; ++c) LineFFT<T, N, E, Cfg::RMAX, true>::run(v[c], sm, t, A.tw);
    }

    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    if (active) {
        T sE[D][2], sJ[D][2], sE2 = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) sE[c][0] = sE[c][1] = sJ[c][0] = sJ[c][1] = 0;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int64_t idx = base + t + TL * m;
            const bool inc = A.mask[idx] != 0;
            C q[D], Ev[D], Jv[D];
#pragma unroll
            for (int c = 0; c < D; ++c) q[c] = v[c][m];
            pw.apply(q, inc, A.S ? A.S + idx : nullptr, A.Tf ? A.Tf + idx : nullptr, A.Ntot, Ev, Jv,
                     mode != MODE_ROW_OUTPUT);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                v[c][m] = q[c];
                sE[c][0] += Ev[c].x;
                sE[c][1] += Ev[c].y;
                sJ[c][0] += Jv[c].x;
                sJ[c][1] += Jv[c].y;
                sE2 += Ev[c].x * Ev[c].x + Ev[c].y * Ev[c].y;
                if (mode == MODE_ROW_OUTPUT) A.Eout[c * A.Ntot + idx] = Ev[c];
            }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            acc[4 * c + 0] = (double)sE[c][0];
            acc[4 * c + 1] = (double)sE[c][1];
            acc[4 * c + 2] = (double)sJ[c][0];
            acc[4 * c + 3] = (double)sJ[c][1];
        }
        acc[4 * D] = (double)sE2;
    }

    if (mode != MODE_ROW_OUTPUT) {
#pragma unroll
        for (int c = 0; c < D; ++c) LineFFT<T, N, E, Cfg::RMAX, false>::run(v[c], sm, t, A.tw);
        if (active) {
#pragma unroll
            for (int c = 0; c < D; ++c)
#pragma unroll
                for (int m = 0; m < E; ++m) A.X[c * A.Ntot + base + t + TL * m] = v[c][m];
        }
    }
    block_reduce_store<NV>(acc, A.partials + (int64_t)blockIdx.x * NV);
}

// ---------------------------------------------------------------------------
// Gamma multiply on one frequency: out = A v + B Gamma(k) v (k != 0),
// out = A0 v + ce e (k = 0); coefficients carry the 1/N of the inverse DFT.
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void gamma_apply(cx<T> (&v)[D], const int (&ki)[3], const PassArgs<T>& A,
                                            const SchemeParams& P) {
    using C = cx<T>;
    bool zero = true;
#pragma unroll
    for (int a = 0; a < D; ++a) zero = zero && (ki[a] == 0);
    const T s = (T)P.inv_ntot;
    if (zero) {
        const C a0 = mkc((T)(P.g_a0[0] * P.inv_ntot), (T)(P.g_a0[1] * P.inv_ntot));
        const C ce = mkc((T)P.g_ce[0], (T)P.g_ce[1]);
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = cadd(cmul(a0, v[c]), cscale(ce, (T)P.e[c]));
        return;
    }
    const C ga = mkc((T)P.g_a[0] * s, (T)P.g_a[1] * s);
    const C gb = mkc((T)P.g_b[0] * s, (T)P.g_b[1] * s);
    C u[D];
    bool nyq = false;
    if (P.green == GREEN_TRIG) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int n = A.n[a];
            const int k = ki[a] < n / 2 ? ki[a] : ki[a] - n;
            nyq = nyq || (ki[a] == n / 2);
            u[a] = mkc((T)k, (T)0);
        }
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = A.fd[a][ki[a]];
    }
    C out[D];
    if (nyq) {
#pragma unroll
        for (int c = 0; c < D; ++c) out[c] = cmul(ga, v[c]);
    } else {
        T nrm = 0;
        C dot = mkc((T)0, (T)0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            nrm += u[a].x * u[a].x + u[a].y * u[a].y;
            dot = cadd(dot, cmulc(v[a], u[a]));    // conj(u_a) v_a
        }
        const C proj = cscale(cmul(gb, dot), (T)1 / nrm);
#pragma unroll
        for (int c = 0; c < D; ++c) out[c] = cadd(cmul(ga, v[c]), cmul(proj, u[c]));
    }
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = out[c];
}

// ---------------------------------------------------------------------------
// Strided pass: lines along y (or z) with element stride ls; each block takes
// COLS adjacent line starts and every component (one thread group per line).
// ---------------------------------------------------------------------------
template <typename T, int N, int D>
__global__ void __launch_bounds__(ColCfg<T, N, D>::THREADS)
col_pass(const PassArgs<T> A) {
    using Cfg = ColCfg<T, N, D>;
    using C = cx<T>;
    constexpr int E = Cfg::E, TL = Cfg::TL, COLS = Cfg::COLS, G = Cfg::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (A.ctrl->skipB) return;
    const int mode = A.mode;

    const int g = threadIdx.x % G, t = threadIdx.x / G;
    const int col = g % COLS, comp = g / COLS;
    C* sm = reinterpret_cast<C*>(smem_raw) + g * LinePad<N>::size;

    const int64_t cblocks = A.n_inner / COLS;
    const int64_t outer = blockIdx.x / cblocks;
    const int64_t inner0 = (blockIdx.x % cblocks) * COLS;
    const int64_t base = comp * A.Ntot + outer * A.outer_stride + inner0 + col;

    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = A.X[base + (int64_t)(t + TL * m) * A.ls];

    if (mode == MODE_COL_INV) {
        LineFFT<T, N, E, Cfg::RMAX, true>::run(v, sm, t, A.tw);
    } else {
        LineFFT<T, N, E, Cfg::RMAX, false>::run(v, sm, t, A.tw);
        if (mode == MODE_COL_GAMMA) {
            const SchemeParams& P = *A.prm;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) sm[pad16(t + TL * m)] = v[m];
            __syncthreads();
            C* lines = reinterpret_cast<C*>(smem_raw);
            for (int idx = threadIdx.x; idx < COLS * N; idx += blockDim.x) {
                const int cc = idx % COLS, kl = idx / COLS;
                int ki[3] = {0, 0, 0};
                const int64_t inner = inner0 + cc;
                if (A.line_axis == 1) {            // 2-D: inner = kx, line = ky
                    ki[0] = (int)inner;
                    ki[1] = kl;
                } else {                            // 3-D z pass: inner = kx + nx ky, line = kz
                    ki[0] = (int)(inner % A.n[0]);
                    ki[1] = (int)(inner / A.n[0]);
                    ki[2] = kl;
                }
                C q[D];
#pragma unroll
                for (int c = 0; c < D; ++c) q[c] = lines[(cc + COLS * c) * LinePad<N>::size + pad16(kl)];
                gamma_apply<T, D>(q, ki, A, P);
#pragma unroll
                for (int c = 0; c < D; ++c) lines[(cc + COLS * c) * LinePad<N>::size + pad16(kl)] = q[c];
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = sm[pad16(t + TL * m)];
            LineFFT<T, N, E, Cfg::RMAX, true>::run(v, sm, t, A.tw);
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) A.X[base + (int64_t)(t + TL * m) * A.ls] = v[m];
}

}  // namespace lsfft
