// Iteration kernels of the FFT Lippmann-Schwinger solver.
//
// State layout: the Q field (E for Moulinec-Suquet, the polarisation
// P = J + sigma_0 E for Eyre-Milton, the Q component of H'' for the substituted
// schemes) is stored component-planar, X[c][z][y][x], in the half-transformed
// domain (DFT along x done, y/z in real space) between iterations.  S and T,
// the extra components of H'' (Eq. J27, J36), live in real space and are
// touched only on phase-1 voxels (they vanish on phase 2).
//
// Packed real layout (2-D, every scheme coefficient real, i.e. real sigma_1 and
// a real reference medium): the fields are real (S and T purely imaginary), so
// the row pass transforms the two components as one complex line
// Z = F_x + i F_y (S and T as s_x + i s_y with S = i s) and keeps the x-spectra
// of F_x and F_y as two half-spectrum planes (k_x = 0..n_x/2, padded pitch):
// half the bytes and transforms of the complex layout, and the strided pass
// sees ordinary columns.
//
// One iteration (2-D): row pass [inverse x-DFT -> pointwise scheme update and
// volume averages -> forward x-DFT], finalize (FP64 sums, sigma_k, stop rule),
// strided pass over y [forward y-DFT -> Gamma multiply per frequency -> inverse
// y-DFT].  3-D: row pass, finalize, y forward, z [forward, Gamma, inverse],
// y inverse.  Every pass is in place.
//
// Both passes are persistent: a block owns a stream of work items (a few rows,
// or a few line starts of the strided axis).  Row items are staged in shared
// memory by cp.async (contiguous rows), strided items by one TMA box; a thread
// transforms one line at a time in registers (positions t + TL*m), and the next
// item is staged as soon as the current one has been read.
#pragma once

#include <cuda.h>   // CUtensorMap (the encoding itself goes through the runtime's driver entry point)

#include "lsfft_fft.cuh"
#include "lsfft_params.h"
#include "lsfft_pdl.cuh"
#include "lsfft_reduce.cuh"
#include "lsfft_tma.cuh"

namespace lsfft {

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int roundup16(int v) { return (v + 15) / 16 * 16; }

// Line pitches: the stage buffer keeps lines dense (cp.async destinations,
// 16-byte aligned); the exchange buffer is padded one slot per 16 elements.
// When fewer than 16 threads share a line, consecutive line groups are offset
// by TL slots so that the groups of one warp fall into different banks.
template <typename T, int N, int TL>
struct Pitch {
    static constexpr int GPAD = TL < 16 ? cmax(TL, 2) : 0;
    static constexpr int S = N + GPAD;
    static constexpr int X = roundup16(N + N / 16) + GPAD;
};

// ---------------------------------------------------------------------------
// Launch geometry, shared by the kernels and the host dispatch.  MINB is the
// number of blocks per SM the shared-memory footprint allows (at most 4); it is
// passed to __launch_bounds__ so that registers do not become the tighter limit.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int min_blocks(int smem, int threads) {
    return cmax(1, cmin(cmin(8, (227 * 1024) / (smem + 1024)), 2048 / threads));
}

// Row pitch (elements) of the two half-spectrum planes of the packed layout:
// k_x = 0..n_x/2 plus padding to a 32-byte multiple, so that the strided pass can
// move whole 32-byte row segments of any aligned group of adjacent columns.
__host__ __device__ constexpr int64_t half_pitch(int64_t nx) { return nx / 2 + 4; }

// Points per thread (E) and largest radix of a line transform.  FP64 2-D lines
// of at most 64 points take two points per thread, so that one line fills a
// warp: the FP64 pipe of this GPU gave a warp with 8 of 32 lanes active nearly
// the time of a full one (64^2 rows: one row of 8 threads per warp instead of
// four made the pass only 1.25x faster), so fewer instructions per thread win.
template <typename T, int N, int D>
struct LineShape {
    static constexpr bool NARROW64 = sizeof(T) == 8 && D == 2 && N >= 4 && N <= 64;
    static constexpr int E = NARROW64 ? 2 : sizeof(T) == 4 ? (N < 16 ? N : 16) : (N < 8 ? N : 8);
    static constexpr int RMAX = NARROW64 ? 2 : sizeof(T) == 4 ? 16 : 8;
};

template <typename T, int N, int D>
struct RowCfg {
    static constexpr int CS = (int)sizeof(cx<T>);
    static constexpr int E = LineShape<T, N, D>::E;
    static constexpr int RMAX = LineShape<T, N, D>::RMAX;
    static constexpr int TL = N / E;
    // rows per item: small blocks, so that several fit an SM (measured 25 %
    // faster than 256-thread items at 256^3 and 512^3, 14 % at 256^2).  FP64
    // 2-D rows are bound by the FP64 pipe, whose rate is per warp scheduler: one
    // row per item puts each row of a small grid on a scheduler of its own (64^2
    // lattice: 64 rows on 64 schedulers, where 16-row items used 16).
    static constexpr int LPB = sizeof(T) == 8 && D == 2 ? 1 : cmax(1, (D == 3 ? 64 : 128) / TL);
    static constexpr int THREADS = LPB * TL;
    using P = Pitch<T, N, TL>;
    // packed layout: two staged half rows of pitch HPS; for FP32 lines of >= 2048
    // points a second exchange line follows them (DBX), so that the packed path's
    // transforms alternate between two exchange lines (one barrier per stage)
    static constexpr int HPS = (int)(N / 2 + 4);
    static constexpr bool DBX = sizeof(T) == 4 && D == 2 && N >= 2048;
    static constexpr int S_BYTES = cmax(D * LPB * P::S * CS, DBX ? (2 * LPB * HPS + LPB * P::X) * CS : 0);
    static constexpr int X_BYTES = LPB * P::X * CS;
    static constexpr int M_BYTES = roundup16(LPB * N);
    static constexpr int SMEM = S_BYTES + X_BYTES + M_BYTES;
    static constexpr bool SUPPORTED = SMEM <= 227 * 1024 && THREADS <= 1024;
    // FP64 lines are bound by the FP64 pipe, not by latency: give them the
    // registers of one block per SM rather than spill
    static constexpr int MINB = sizeof(T) == 8 ? 1 : min_blocks(SMEM, THREADS);
    static constexpr bool PAIRED = THREADS <= 256;
};

template <typename T, int N, int D>
struct ColCfg {
    static constexpr int CS = (int)sizeof(cx<T>);
    static constexpr int E = LineShape<T, N, D>::E;
    static constexpr int RMAX = LineShape<T, N, D>::RMAX;
    static constexpr int TL = N / E;
    static constexpr int EPC = CS / 8;                            // 8-byte tensor elements per value
    static constexpr int item_bytes(int cols) { return D * N * cols * CS; }
    static constexpr int xp() { return roundup16(N + N / 16) + 8; }
    // a slot holds the item as the TMA box delivers it (dense), and once the
    // threads have read it into registers, the padded exchange lines of its
    // D * cols transforms: no separate exchange buffer
    static constexpr int slot_bytes(int cols) {
        return (cmax(item_bytes(cols), D * cols * xp() * CS) + 1023) / 1024 * 1024;
    }
    static constexpr int bytes(int cols) { return 2 * slot_bytes(cols) + 64; }
    // adjacent line starts per item: a 32-byte row segment, or 16 bytes when
    // two item buffers of 32-byte segments do not fit.  FP64 2-D columns take
    // one line start per item (16 bytes): the FP64 pipe, not DRAM, bounds them,
    // and small grids then spread over twice as many SMs.
    static constexpr int COLS = sizeof(T) == 8 && D == 2 ? 16 / CS
                                : bytes(32 / CS) <= 220 * 1024 ? 32 / CS : 16 / CS;
    static constexpr int THREADS = D * COLS * TL;                 // every line of an item at once
    static constexpr int ITEM_BYTES = item_bytes(COLS);
    static constexpr int SLOT_BYTES = slot_bytes(COLS);
    static constexpr int XP = xp();
    static constexpr int BJ0 = N < 256 ? N : 256;                 // TMA box rows: inner and outer dimension
    static constexpr int BJ1 = N / BJ0;
    static constexpr int SMEM = bytes(COLS);
    static constexpr bool SUPPORTED = SMEM <= 227 * 1024 && THREADS <= 1024 && COLS * CS >= 16;
    static constexpr int MINB = min_blocks(SMEM, THREADS);
    static constexpr bool PAIRED = THREADS <= 256;
};

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, valid on sm_103a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// Wait until at most `n` (0..2) of this thread's most recent groups are pending.
__device__ __forceinline__ void cp_async_wait_pending(int n) {
    if (n <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// Reductions: thread-local FP64 -> warp shuffle -> block -> partials[block][NV]
// ---------------------------------------------------------------------------
template <int NV, int NT>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NV], double* __restrict__ out) {
    __shared__ double red[32][NV];
    if constexpr (NT < 32) {
        // a block narrower than a warp (short FP64 rows): thread 0 adds the
        // threads' sums in order
#pragma unroll
        for (int v = 0; v < NV; ++v) red[threadIdx.x][v] = acc[v];
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double x = 0.0;
                for (int i = 0; i < NT; ++i) x += red[i][v];
                out[v] = x;
            }
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int LOW = 32 / pow2_at_least(NV) - 1;   // lanes with these bits zero hold distinct sums
    int idx;
    const double x = warp_sum_scatter<NV>(acc, idx);
    if ((lane & LOW) == 0 && idx < NV) {
        if constexpr (NT == 32) out[idx] = x;   // one warp: its sum is the block's
        else red[warp][idx] = x;
    }
    if constexpr (NT == 32) return;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double y[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) y[v] = lane < nw ? red[lane][v] : 0.0;
        const double s = warp_sum_scatter<NV>(y, idx);
        if ((lane & LOW) == 0 && idx < NV) out[idx] = s;
    }
}

// Scheme constants rounded to the field precision, passed by value as a
// kernel parameter (they sit in the constant bank and feed the FMAs directly).
template <typename T>
struct KConst {
    cx<T> a_in, a_out;          // MS: sigma/sigma_0 - 1 per phase; EM: W per phase
    cx<T> k1, k2, k3, tm1p1;    // MS in H''
    cx<T> p1, p2, p3, w;        // EM in H''
    cx<T> inv2s0, s1;
    cx<T> s0, inv_s0;           // per-voxel conductivity mode: reference medium and its inverse
    cx<T> g_a, g_b, g_a0;       // Gamma step coefficients, already divided by N
    cx<T> g_ce;                 // zero-mode source coefficient
    cx<T> iq_in, iq_out;        // initial Q = iq e per phase (two-phase media)
    T e[3];
    int scheme, green;
    int real_coef;              // the Gamma-step coefficients g_a, g_b, g_a0, g_ce are real
};

// Compile-time integer (a scheme, a count) for code specialised outside a loop.
template <int V>
struct IntTag {
    static constexpr int value = V;
};

// ---------------------------------------------------------------------------
// Pointwise scheme update on one voxel (all d components).
//   q[c]   : Q component (real space) on entry; on exit the field handed to the
//            forward DFT (tau for MS-type schemes, W P for EM-type schemes).
//   S, T   : read and written in place on phase-1 voxels (substituted schemes).
//   E, J   : the physical fields of the current iterate, for the averages.
// ---------------------------------------------------------------------------
template <typename T, int D, int SCH>
__device__ __forceinline__ void pointwise(const KConst<T>& K, cx<T> (&q)[D], bool inc, cx<T>* __restrict__ Sv,
                                          cx<T>* __restrict__ Tv, int64_t cs, cx<T> (&E)[D], cx<T> (&J)[D],
                                          bool write_st) {
    using C = cx<T>;
    if constexpr (SCH == SCHEME_MS) {            // Eq. J0-0: tau = (sigma/sigma_0 - 1) E
        const C a = inc ? K.a_in : K.a_out;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            E[c] = q[c];
            J[c] = inc ? cmul(K.s1, q[c]) : q[c];
            q[c] = cmul(a, q[c]);
        }
    } else if constexpr (SCH == SCHEME_EM) {     // W P with W = (sigma - sigma_0)/(sigma + sigma_0)
        const C W = inc ? K.a_in : K.a_out;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const C wp = cmul(W, q[c]);
            E[c] = cmul(csub(q[c], wp), K.inv2s0);
            J[c] = cscale(cadd(q[c], wp), (T)0.5);
            q[c] = wp;
        }
    } else if constexpr (SCH == SCHEME_MATVEC) { // chi v (the operator chi Gamma_1 chi of the pole problem)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            E[c] = inc ? q[c] : mkc((T)0, (T)0);
            J[c] = mkc((T)0, (T)0);
            q[c] = E[c];
        }
    } else if constexpr (SCH == SCHEME_MS_SUB) { // Eq. J36, J42a: tau'' = (L''/sigma_0'' - 1) E''
        if (inc) {
            C s[D];
#pragma unroll
            for (int c = 0; c < D; ++c) s[c] = Sv[c * cs];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const C cc = cadd(cmul(K.p1, q[c]), cmul(K.p2, s[c]));
                E[c] = q[c];
                J[c] = cadd(q[c], cmul(K.tm1p1, cc));
                const C tq = cadd(cmul(K.k1, cc), cmul(K.k2, q[c]));
                const C ts = cadd(cmul(K.k3, cc), cmul(K.k2, s[c]));
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
                q[c] = cmul(K.k2, q[c]);
            }
        }
    } else {                                // Eq. J36, J43: W'' = w (I - 2 p p^T) on phase 1
        if (inc) {
            C s[D], tt[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                s[c] = Sv[c * cs];
                tt[c] = Tv[c * cs];
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const C cc = cadd(cadd(cmul(K.p1, q[c]), cmul(K.p2, s[c])), cmul(K.p3, tt[c]));
                const C cc2 = cadd(cc, cc);
                const C wq = cmul(K.w, csub(q[c], cmul(K.p1, cc2)));
                const C ws = cmul(K.w, csub(s[c], cmul(K.p2, cc2)));
                const C wt = cmul(K.w, csub(tt[c], cmul(K.p3, cc2)));
                E[c] = cmul(csub(q[c], wq), K.inv2s0);
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
                const C wq = cmul(K.w, q[c]);
                E[c] = cmul(csub(q[c], wq), K.inv2s0);
                J[c] = cscale(cadd(q[c], wq), (T)0.5);
                q[c] = wq;
            }
        }
    }
}

// The same update in the packed real layout: z = Q_x + i Q_y and, on phase 1,
// s = s_x + i s_y, tau = tau_x + i tau_y with S = i s, T = i tau.  Every
// coefficient is real here; with p_2 = i q_2 and p_3 = i q_3 one has
// p . (Q, S, T) = p_1 Q - q_2 s - q_3 tau componentwise.
template <typename T, int SCH>
__device__ __forceinline__ void pointwise_packed(const KConst<T>& K, cx<T>& z, bool inc, cx<T>& s, cx<T>& tt,
                                                 cx<T>& E, cx<T>& J) {
    // s, tt: S and T of a phase-1 voxel, updated in place (the caller loads and
    // stores them); unused elsewhere.
    using C = cx<T>;
    if constexpr (SCH == SCHEME_MS) {
        E = z;
        J = inc ? cscale(z, K.s1.x) : z;
        z = cscale(z, inc ? K.a_in.x : K.a_out.x);
    } else if constexpr (SCH == SCHEME_EM) {
        const C wp = cscale(z, inc ? K.a_in.x : K.a_out.x);
        E = cscale(csub(z, wp), K.inv2s0.x);
        J = cscale(cadd(z, wp), (T)0.5);
        z = wp;
    } else if constexpr (SCH == SCHEME_MS_SUB) {
        if (inc) {
            const C cc = csub(cscale(z, K.p1.x), cscale(s, K.p2.y));
            E = z;
            J = cadd(z, cscale(cc, K.tm1p1.x));
            s = cneg(cadd(cscale(cc, K.k3.y), cscale(s, K.k2.x)));
            z = cadd(cscale(cc, K.k1.x), cscale(z, K.k2.x));
        } else {
            E = z;
            J = z;
            z = cscale(z, K.k2.x);
        }
    } else {
        if (inc) {
            const C cc = csub(csub(cscale(z, K.p1.x), cscale(s, K.p2.y)), cscale(tt, K.p3.y));
            const C cc2 = cadd(cc, cc);
            const C wq = cscale(csub(z, cscale(cc2, K.p1.x)), K.w.x);
            s = cscale(csub(s, cscale(cc2, K.p2.y)), -K.w.x);
            tt = cscale(csub(tt, cscale(cc2, K.p3.y)), K.w.x);
            E = cscale(csub(z, wq), K.inv2s0.x);
            J = cscale(cadd(z, wq), (T)0.5);
            z = wq;
        } else {
            const C wq = cscale(z, K.w.x);
            E = cscale(csub(z, wq), K.inv2s0.x);
            J = cscale(cadd(z, wq), (T)0.5);
            z = wq;
        }
    }
}

// Per-voxel conductivity sigma(x) (a medium with any number of phases), for the
// Moulinec-Suquet and Eyre-Milton schemes with a caller-chosen reference sigma_0.
template <typename T, int D>
__device__ __forceinline__ void pointwise_field(const KConst<T>& K, cx<T> (&q)[D], cx<T> sg, cx<T> (&E)[D],
                                                cx<T> (&J)[D]) {
    using C = cx<T>;
    if (K.scheme == SCHEME_MS) {            // tau = (sigma/sigma_0 - 1) E, J = sigma E
        const C a = csub(cmul(sg, K.inv_s0), mkc((T)1, (T)0));
#pragma unroll
        for (int c = 0; c < D; ++c) {
            E[c] = q[c];
            J[c] = cmul(sg, q[c]);
            q[c] = cmul(a, q[c]);
        }
    } else {                                // W = (sigma - sigma_0)/(sigma + sigma_0)
        const C num = csub(sg, K.s0), den = cadd(sg, K.s0);
        const T dd = den.x * den.x + den.y * den.y;
        const C W = cscale(cmulc(num, den), (T)1 / dd);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const C wp = cmul(W, q[c]);
            E[c] = cmul(csub(q[c], wp), K.inv2s0);
            J[c] = cscale(cadd(q[c], wp), (T)0.5);
            q[c] = wp;
        }
    }
}

template <typename T>
__device__ __forceinline__ void pointwise_field_packed(const KConst<T>& K, cx<T>& z, T sg, cx<T>& E, cx<T>& J) {
    if (K.scheme == SCHEME_MS) {
        E = z;
        J = cscale(z, sg);
        z = cscale(z, sg * K.inv_s0.x - (T)1);
    } else {
        const T W = (sg - K.s0.x) / (sg + K.s0.x);
        const cx<T> wp = cscale(z, W);
        E = cscale(csub(z, wp), K.inv2s0.x);
        J = cscale(cadd(z, wp), (T)0.5);
        z = wp;
    }
}

template <typename T>
struct PassArgs {
    cx<T>* X;                 // state, [D][Ntot]; packed: [2][Nh], rows of hp, k_x = 0..n_x/2
    cx<T>* S;                 // H'' S component, [D][Ntot] (or null)
    cx<T>* Tf;                // H'' T component, [D][Ntot] (or null)
    cx<T>* Eout;              // output field, [D][Ntot] (row pass, output mode)
    const uint8_t* mask;      // [Ntot]
    const cx<T>* sigma;       // per-voxel conductivity [Ntot] (MS / EM only), or null for two phases
    Ctrl* ctrl;
    double* partials;         // [gridDim.x][NV]
    const cx<T>* tw;          // FP64 twiddle table W_N^k of the pass's line length
    const cx<T>* fd[3];       // forward-difference symbol u_a(k), per axis
    int64_t Ntot;             // voxels; plane stride of the strided passes
    int64_t hp;               // packed layout: row pitch of the two half-spectrum planes
    int64_t Nh;               // packed layout: plane stride of the half-spectrum planes
    int64_t n_lines;          // row pass: number of rows
    int64_t ls;               // strided pass: element stride along the line
    int64_t n_inner;          // strided pass: contiguous line starts per outer slab
    int64_t outer_stride;     // strided pass: stride between outer slabs
    int64_t n_outer;          // strided pass: number of outer slabs
    int n[3];                 // grid extents (x, y, z)
    int line_axis;            // strided pass: 1 (y) or 2 (z)
    int mode;                 // PassMode
    int grid_blocks;          // persistent grid size chosen by the host
    int packed;               // packed real layout (2-D row pass only; the strided pass sees two planes)
    int pdl;                  // host-side: launch programmatically after the previous kernel (lsfft_pdl.cuh)
    int pdl_early;            // signal dependents at the kernel's start (small grids), else at block exit
    KConst<T> k;
    long long wait_limit;     // bound of every mbarrier wait, in clock cycles
    int extra_tx;             // test hook: bytes announced but never delivered (0 in normal runs)
    CUtensorMap tmap;         // strided passes: TMA view of the planes (encoded by the host)
};

// ---------------------------------------------------------------------------
// Row pass: lines along x (contiguous).  Work item = LPB consecutive rows.
// ---------------------------------------------------------------------------
template <typename T, int N, int D>
__global__ void __launch_bounds__(RowCfg<T, N, D>::THREADS, RowCfg<T, N, D>::MINB)
row_pass(const PassArgs<T> A) {
    using Cfg = RowCfg<T, N, D>;
    using C = cx<T>;
    using InvFFT = LineFFT<T, N, Cfg::E, Cfg::RMAX, true, Cfg::PAIRED>;
    using FwdFFT = LineFFT<T, N, Cfg::E, Cfg::RMAX, false, Cfg::PAIRED>;
    constexpr int E = Cfg::E, TL = Cfg::TL, LPB = Cfg::LPB, NV = 4 * D + 1;
    constexpr int PS = Cfg::P::S, PX = Cfg::P::X, HPS = Cfg::HPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    if (A.pdl_early) pdl_trigger();
    const int mode = A.mode;
    if (mode != MODE_ROW_OUTPUT && A.ctrl->done) {   // uniform: before any allocation or barrier
        // the solve stopped before this update: its strided passes skip as well
        // (they run beside the finalize step and read only this flag)
        if (blockIdx.x == 0 && threadIdx.x == 0) A.ctrl->skipB = 1;
        return;
    }

    C* Sb = reinterpret_cast<C*>(smem_raw);                                    // [L][LPB][PS]
    const int g = threadIdx.x / TL, t = threadIdx.x % TL;
    C* Xb = reinterpret_cast<C*>(smem_raw + Cfg::S_BYTES) + g * PX;            // exchange line
    // packed path: the second exchange line, after the two staged half rows
    C* Xb2 = Sb + 2 * LPB * HPS + g * PX;
    uint8_t* Mb = smem_raw + Cfg::S_BYTES + Cfg::X_BYTES;                      // [LPB][N]
    const int64_t n_items = (A.n_lines + LPB - 1) / LPB;
    // staged lines per row: the d component planes, or in the packed layout the
    // two half-spectrum planes (none on the first pass, which starts from the mask)
    const int L = A.packed ? 2 : D;
    const bool stage_x = !(A.packed && mode == MODE_ROW_FIRST);
    constexpr int HP = (int)half_pitch(N);

    // Stage line l of the rows of `item` (and the mask with line 0): one commit group.
    // (chunk counts are compile-time constants in both branches: no runtime division)
    auto stage_rows = [&](int64_t item, int l, const C* src0, auto chunks, int64_t pitch, int dpitch) {
        constexpr int CHL = decltype(chunks)::value;
        for (int i = threadIdx.x; i < LPB * CHL; i += Cfg::THREADS) {
            const int ch = i % CHL, r = i / CHL;
            const int64_t row = item * LPB + r;
            if (row < A.n_lines)
                cp_async16(reinterpret_cast<unsigned char*>(Sb + (l * LPB + r) * dpitch) + 16 * ch,
                           reinterpret_cast<const unsigned char*>(src0 + row * pitch) + 16 * ch);
        }
    };
    auto prefetch_line = [&](int64_t item, int l) {
        if (A.packed) {
            if (stage_x) stage_rows(item, l, A.X + l * A.Nh, IntTag<HP * (int)sizeof(C) / 16>{}, HP, HPS);
        } else {
            stage_rows(item, l, A.X + l * A.Ntot, IntTag<N * (int)sizeof(C) / 16>{}, N, PS);
        }
        if (l == 0) {
            constexpr int MCH = N / 16;
            for (int i = threadIdx.x; i < LPB * MCH; i += Cfg::THREADS) {
                const int ch = i % MCH, r = i / MCH;
                const int64_t row = item * LPB + r;
                if (row < A.n_lines) cp_async16(Mb + r * N + 16 * ch, A.mask + row * N + 16 * ch);
            }
        }
        cp_async_commit();
    };

    // Running per-thread sums over items in the field precision, compensated
    // (Kahan) in FP32: the FP64 pipe of the GPU is far slower than FP32, so in
    // FP32 mode doubles enter only in the block and grid reductions at the end.
    T acc[NV], cmp[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = cmp[i] = (T)0;
    auto kahan_add = [&](int i, T x) {
        if constexpr (sizeof(T) == 8) {   // FP64 needs no compensation (and its pipe is slow)
            acc[i] += x;
            return;
        }
        const T y = x - cmp[i];
        const T tsum = acc[i] + y;
        cmp[i] = (tsum - acc[i]) - y;
        acc[i] = tsum;
    };

    // Packed real layout: the line stays in registers from the join of the half
    // spectra (Z(k) = X(k) + i Y(k) for k <= n/2, conj(X(n-k)) + i conj(Y(n-k))
    // above) through the inverse DFT, the scheme update and the forward DFT to
    // their split (X = (Z(k) + conj Z(n-k))/2, Y = (Z(k) - conj Z(n-k))/(2i)), and
    // the next item is staged as soon as the join has read this one.
    // Substituted schemes in the packed layout: bring the S (and T) rows of item
    // `nxt` into L2 while the current item works, so that the scheme update finds
    // them there (measured 5 % faster at 8192^2; with the three planes of the
    // complex layout the extra requests cost more than they save).
    auto prefetch_st = [&](int64_t nxt) {
        if (!A.S) return;
        constexpr int LINES128 = LPB * N * (int)sizeof(C) / 128;
        const int64_t first = nxt * LPB * N;
        const int64_t rows_left = A.n_lines - nxt * LPB;
        const int lines = rows_left >= LPB ? LINES128 : (int)(rows_left * N * (int64_t)sizeof(C) / 128);
        for (int i = threadIdx.x; i < lines; i += Cfg::THREADS) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(A.S + first) + 128 * i));
            if (A.Tf)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(A.Tf + first) + 128 * i));
        }
    };
    auto packed_item = [&](int64_t row, bool active, int64_t base, int64_t next, bool has_next) {
        cp_async_wait_all();
        __syncthreads();
        C v[E];
        uint32_t incb = 0;   // phase of the thread's points, read before the mask is restaged
#pragma unroll
        for (int m = 0; m < E; ++m) incb |= (Mb[g * N + t + TL * m] != 0 ? 1u : 0u) << m;
        if (mode == MODE_ROW_FIRST) {
            // the first pass starts from Q = iq e (or the per-voxel reference)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                T qv;
                if (A.sigma)
                    qv = A.k.scheme == SCHEME_EM ? A.sigma[base + t + TL * m].x + A.k.s0.x : (T)1;
                else
                    qv = (incb >> m) & 1u ? A.k.iq_in.x : A.k.iq_out.x;
                v[m] = mkc(qv * A.k.e[0], qv * A.k.e[1]);
            }
            __syncthreads();
        } else {
            const C* Hx = Sb + g * HPS;
            const C* Hy = Sb + (LPB + g) * HPS;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int k = t + TL * m;
                if (k <= N / 2) {
                    const C x = Hx[k], y = Hy[k];
                    v[m] = mkc(x.x - y.y, x.y + y.x);
                } else {
                    const C x = Hx[N - k], y = Hy[N - k];
                    v[m] = mkc(x.x + y.y, y.x - x.y);
                }
            }
            // (the previous readers of Xb, the split of the last item, are behind the
            // barrier at the start of this item)
            if constexpr (Cfg::DBX) InvFFT::run2(v, Xb, Xb2, t, A.tw);
            else InvFFT::run(v, Xb, t, A.tw);
            if constexpr (N <= Cfg::RMAX) __syncthreads();   // (a one-stage transform has no barrier)
        }
        // every thread has read the staging buffers: stage the next item
        if (has_next) {
            for (int l = 0; l < 2; ++l) prefetch_line(next, l);
            prefetch_st(next);
        }

        if (active) {
            T sE[2] = {0, 0}, sJ[2] = {0, 0}, sE2 = 0;
            const bool wst = mode != MODE_ROW_OUTPUT;
            const bool outm = mode == MODE_ROW_OUTPUT;
            auto points = [&](auto tag) {
                constexpr int SCH = decltype(tag)::value;
                constexpr bool SUB = SCH == SCHEME_MS_SUB || SCH == SCHEME_EM_SUB;
                // in batches of HB points: S (T) of the phase-1 points first, so
                // that their global loads are in flight together (fully unrolled:
                // v is indexed by compile-time positions only)
                constexpr int HB = (sizeof(T) == 4 ? 4 : 2) < E ? (sizeof(T) == 4 ? 4 : 2) : E;
#pragma unroll
                for (int m0 = 0; m0 < E; m0 += HB) {
                    C sv[HB], tv[HB];
#pragma unroll
                    for (int h = 0; h < HB; ++h) {
                        const int pos = t + TL * (m0 + h);
                        const bool inc = (incb >> (m0 + h)) & 1u;
                        sv[h] = tv[h] = mkc((T)0, (T)0);
                        if constexpr (SUB) {
                            if (inc) sv[h] = A.S[base + pos];
                        }
                        if constexpr (SCH == SCHEME_EM_SUB) {
                            if (inc) tv[h] = A.Tf[base + pos];
                        }
                    }
#pragma unroll
                    for (int h = 0; h < HB; ++h) {
                        const int m = m0 + h;
                        const int64_t idx = base + t + TL * m;
                        const bool inc = (incb >> m) & 1u;
                        C z = v[m], Ez, Jz;
                        if (!SUB && A.sigma)
                            pointwise_field_packed<T>(A.k, z, A.sigma[idx].x, Ez, Jz);
                        else
                            pointwise_packed<T, SCH>(A.k, z, inc, sv[h], tv[h], Ez, Jz);
                        if constexpr (SUB) {
                            if (inc && wst) {
                                A.S[idx] = sv[h];
                                if constexpr (SCH == SCHEME_EM_SUB) A.Tf[idx] = tv[h];
                            }
                        }
                        v[m] = z;
                        sE[0] += Ez.x;
                        sE[1] += Ez.y;
                        sJ[0] += Jz.x;
                        sJ[1] += Jz.y;
                        sE2 += Ez.x * Ez.x + Ez.y * Ez.y;
                        if (outm) {
                            A.Eout[idx] = mkc(Ez.x, (T)0);
                            A.Eout[A.Ntot + idx] = mkc(Ez.y, (T)0);
                        }
                    }
                }
            };
            switch (A.k.scheme) {
                case SCHEME_MS: points(IntTag<SCHEME_MS>{}); break;
                case SCHEME_EM: points(IntTag<SCHEME_EM>{}); break;
                case SCHEME_MS_SUB: points(IntTag<SCHEME_MS_SUB>{}); break;
                default: points(IntTag<SCHEME_EM_SUB>{}); break;
            }
            kahan_add(0, sE[0]);   // (the imaginary parts, slots 1, 3, 5, 7, stay zero)
            kahan_add(2, sJ[0]);
            kahan_add(4, sE[1]);
            kahan_add(6, sJ[1]);
            kahan_add(4 * D, sE2);
        }
        if (mode == MODE_ROW_OUTPUT) return;
        // Split of Z into the half spectra: thread t holds Z(t + TL m); the partner
        // Z(n - k) of k <= n/2 is Z((TL - t) + TL (E - 1 - m)) (t > 0) or Z(TL (E - m))
        // (t = 0), always among the upper halves m >= E/2 (k = 0 is its own partner),
        // so only those go through shared memory.
        C* Xs;
        if constexpr (Cfg::DBX) {
            // two exchange lines: the forward transform starts on the one the inverse
            // transform did not read last, and the split uses the one the forward
            // transform did not read last, so neither needs a barrier before it
            constexpr int NEX = FwdFFT::NEX, INV_LAST = (NEX - 1) % 2, FWD0 = 1 - INV_LAST;
            constexpr int SPLIT = 1 - (FWD0 + NEX - 1) % 2;
            FwdFFT::run2(v, FWD0 == 0 ? Xb : Xb2, FWD0 == 0 ? Xb2 : Xb, t, A.tw);
            Xs = SPLIT == 0 ? Xb : Xb2;
        } else {
            FwdFFT::run(v, Xb, t, A.tw);
            __syncthreads();   // the transform's last reads of the exchange line are done
            Xs = Xb;
        }
#pragma unroll
        for (int m = E / 2; m < E; ++m) Xs[pad16(t + TL * m)] = v[m];
        __syncthreads();
        if (active) {
            C* Ho = A.X + row * HP;
#pragma unroll
            for (int m = 0; m <= E / 2; ++m) {
                const int k = t + TL * m;
                if (k <= N / 2) {
                    const C z = v[m], zp = (m == 0 && t == 0) ? v[0] : Xs[pad16((N - k) & (N - 1))];
                    Ho[k] = mkc((T)0.5 * (z.x + zp.x), (T)0.5 * (z.y - zp.y));
                    Ho[A.Nh + k] = mkc((T)0.5 * (z.y + zp.y), (T)0.5 * (zp.x - z.x));
                }
            }
        }
    };

    int64_t item = blockIdx.x;
    if (item < n_items)
        for (int l = 0; l < L; ++l) prefetch_line(item, l);
    for (; item < n_items; item += A.grid_blocks) {
        const int64_t row = item * LPB + g;
        const bool active = row < A.n_lines;
        const int64_t base = row * N;
        const int64_t next = item + A.grid_blocks;
        const bool has_next = next < n_items;
        if constexpr (D == 2) {
            if (A.packed) {
                packed_item(row, active, base, next, has_next);
                continue;
            }
        }

        // 1. inverse x-DFT of every line, parked at this thread's own positions
        for (int l = 0; l < L; ++l) {
            cp_async_wait_pending(L - 1 - l);
            __syncthreads();
            C* Sl = Sb + (l * LPB + g) * PS;
            C v[E];
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = Sl[t + TL * m];
            if (mode != MODE_ROW_FIRST) LineFFT<T, N, E, Cfg::RMAX, true, Cfg::PAIRED>::run(v, Xb, t, A.tw);
#pragma unroll
            for (int m = 0; m < E; ++m) Sl[t + TL * m] = v[m];
        }

        // 2. pointwise scheme update and volume averages on real-space values,
        //    specialised per scheme outside the loop over the thread's points
        if (active) {
            T sE[D][2], sJ[D][2], sE2 = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) sE[c][0] = sE[c][1] = sJ[c][0] = sJ[c][1] = 0;
            const bool wst = mode != MODE_ROW_OUTPUT;
            const bool outm = mode == MODE_ROW_OUTPUT;
            auto points = [&](auto tag) {
                constexpr int SCH = decltype(tag)::value;
                constexpr bool SUB = SCH == SCHEME_MS_SUB || SCH == SCHEME_EM_SUB;
#pragma unroll 4
                for (int m = 0; m < E; ++m) {
                    const int pos = t + TL * m;
                    const int64_t idx = base + pos;
                    const bool inc = Mb[g * N + pos] != 0;
                    C q[D], Ev[D], Jv[D];
#pragma unroll
                    for (int c = 0; c < D; ++c) q[c] = Sb[(c * LPB + g) * PS + pos];
                    if (!SUB && A.sigma)
                        pointwise_field<T, D>(A.k, q, A.sigma[idx], Ev, Jv);
                    else
                        pointwise<T, D, SCH>(A.k, q, inc, A.S ? A.S + idx : nullptr,
                                             A.Tf ? A.Tf + idx : nullptr, A.Ntot, Ev, Jv, wst);
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        Sb[(c * LPB + g) * PS + pos] = q[c];
                        sE[c][0] += Ev[c].x;
                        sE[c][1] += Ev[c].y;
                        sJ[c][0] += Jv[c].x;
                        sJ[c][1] += Jv[c].y;
                        sE2 += Ev[c].x * Ev[c].x + Ev[c].y * Ev[c].y;
                        if (outm) A.Eout[c * A.Ntot + idx] = Ev[c];
                    }
                }
            };
            switch (A.k.scheme) {
                case SCHEME_MS: points(IntTag<SCHEME_MS>{}); break;
                case SCHEME_EM: points(IntTag<SCHEME_EM>{}); break;
                case SCHEME_MS_SUB: points(IntTag<SCHEME_MS_SUB>{}); break;
                case SCHEME_EM_SUB: points(IntTag<SCHEME_EM_SUB>{}); break;
                default: points(IntTag<SCHEME_MATVEC>{}); break;
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                kahan_add(4 * c + 0, sE[c][0]);
                kahan_add(4 * c + 1, sE[c][1]);
                kahan_add(4 * c + 2, sJ[c][0]);
                kahan_add(4 * c + 3, sJ[c][1]);
            }
            kahan_add(4 * D, sE2);
        }

        // 3. forward x-DFT and store; the next item's line l is staged as soon as
        //    every thread has read line l of this item
        if (mode != MODE_ROW_OUTPUT) {
            for (int l = 0; l < L; ++l) {
                C* Sl = Sb + (l * LPB + g) * PS;
                C v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = Sl[t + TL * m];
                __syncthreads();
                if (has_next) prefetch_line(next, l);
                LineFFT<T, N, E, Cfg::RMAX, false, Cfg::PAIRED>::run(v, Xb, t, A.tw);
                if (active) {
#pragma unroll
                    for (int m = 0; m < E; ++m) A.X[l * A.Ntot + base + t + TL * m] = v[m];
                }
            }
        } else {
            __syncthreads();
            if (has_next)
                for (int l = 0; l < L; ++l) prefetch_line(next, l);
        }
    }
    cp_async_wait_all();
    double dacc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) dacc[i] = (double)acc[i] - (double)cmp[i];
    block_reduce_store<NV, Cfg::THREADS>(dacc, A.partials + (int64_t)blockIdx.x * NV);
}

// ---------------------------------------------------------------------------
// Gamma multiply on one frequency: out = a v + b Gamma(k) v (k != 0),
// out = a0 v + ce e (k = 0); a, b, a0 carry the 1/N of the inverse DFT.
// TRIG: Gamma(k) = k k^T/|k|^2 (Eq. J11), 0 if a component is at the Nyquist
// index; FD: Gamma(k) = u u^H/|u|^2 with u_a = exp(2 pi i k_a/n_a) - 1.
// ---------------------------------------------------------------------------
// Real coefficients a, b, a0, ce (real sigma_1 and reference medium: every
// packed-layout solve): the same step with real arithmetic on the coefficients,
// and for the trigonometric symbol a real u = k, about half the instructions.
template <typename T, int D>
__device__ __forceinline__ void gamma_apply_real(cx<T> (&v)[D], const int (&ki)[3], const KConst<T>& K,
                                                 const int* nn, const cx<T>* const* fd) {
    using C = cx<T>;
    bool zero = true;
#pragma unroll
    for (int a = 0; a < D; ++a) zero = zero && (ki[a] == 0);
    if (zero) {
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = mkc(K.g_a0.x * v[c].x + K.g_ce.x * K.e[c], K.g_a0.x * v[c].y);
        return;
    }
    if (K.green == GREEN_TRIG) {
        T k[D];
        bool nyq = false;
        T nrm = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int n = nn[a];
            k[a] = (T)(ki[a] < n / 2 ? ki[a] : ki[a] - n);
            nyq = nyq || (ki[a] == n / 2);
            nrm += k[a] * k[a];
        }
        if (nyq) {
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = cscale(v[c], K.g_a.x);
            return;
        }
        C dot = mkc((T)0, (T)0);   // k . v
#pragma unroll
        for (int a = 0; a < D; ++a) dot = mkc(dot.x + k[a] * v[a].x, dot.y + k[a] * v[a].y);
        const T sb = K.g_b.x / nrm;
        const C proj = cscale(dot, sb);
#pragma unroll
        for (int c = 0; c < D; ++c)
            v[c] = mkc(K.g_a.x * v[c].x + proj.x * k[c], K.g_a.x * v[c].y + proj.y * k[c]);
        return;
    }
    C u[D];
    T nrm = 0;
    C dot = mkc((T)0, (T)0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = fd[a][ki[a]];
        nrm += u[a].x * u[a].x + u[a].y * u[a].y;
        dot = cadd(dot, cmulc(v[a], u[a]));    // conj(u_a) v_a
    }
    const C proj = cscale(dot, K.g_b.x / nrm);
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = cadd(cscale(v[c], K.g_a.x), cmul(proj, u[c]));
}

template <typename T, int D>
__device__ __forceinline__ void gamma_apply_k(cx<T> (&v)[D], const int (&ki)[3], const KConst<T>& K, const int* nn,
                                              const cx<T>* const* fd) {
    using C = cx<T>;
    if (K.real_coef) {
        gamma_apply_real<T, D>(v, ki, K, nn, fd);
        return;
    }
    bool zero = true;
#pragma unroll
    for (int a = 0; a < D; ++a) zero = zero && (ki[a] == 0);
    if (zero) {
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = cadd(cmul(K.g_a0, v[c]), cscale(K.g_ce, K.e[c]));
        return;
    }
    C u[D];
    bool nyq = false;
    if (K.green == GREEN_TRIG) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int n = nn[a];
            const int k = ki[a] < n / 2 ? ki[a] : ki[a] - n;
            nyq = nyq || (ki[a] == n / 2);
            u[a] = mkc((T)k, (T)0);
        }
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = fd[a][ki[a]];
    }
    if (nyq) {
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = cmul(K.g_a, v[c]);
        return;
    }
    T nrm = 0;
    C dot = mkc((T)0, (T)0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        nrm += u[a].x * u[a].x + u[a].y * u[a].y;
        dot = cadd(dot, cmulc(v[a], u[a]));    // conj(u_a) v_a
    }
    const C proj = cscale(cmul(K.g_b, dot), (T)1 / nrm);
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = cadd(cmul(K.g_a, v[c]), cmul(proj, u[c]));
}

template <typename T, int D>
__device__ __forceinline__ void gamma_apply(cx<T> (&v)[D], const int (&ki)[3], const PassArgs<T>& A) {
    gamma_apply_k<T, D>(v, ki, A.k, A.n, A.fd);
}

// ---------------------------------------------------------------------------
// Strided pass: lines along y (or z) with element stride ls.  Work item =
// COLS adjacent line starts of one outer slab with their d component lines.  In
// 2-D with the packed layout the components are the two half-spectrum planes
// (k_x = 0..n_x/2), so Gamma(k_x, k_y) acts on each column on its own.
//
// One TMA box brings a whole item (all d planes, N rows of COLS adjacent
// values: shared-memory layout [plane][row][column]) into one of two buffers,
// two items ahead; every thread transforms one line position range of one
// (plane, column) line, columns fastest, and stores its results from registers.
// The buffer an item came in is refilled as soon as its last transform has read
// it.  Staging the same tiles with 8-byte copies per thread was limited by the
// number of requests an SM keeps in flight.
// ---------------------------------------------------------------------------
template <typename T, int N, int D>
__global__ void __launch_bounds__(ColCfg<T, N, D>::THREADS, ColCfg<T, N, D>::MINB)
col_pass(const __grid_constant__ PassArgs<T> A) {
    using Cfg = ColCfg<T, N, D>;
    using C = cx<T>;
    constexpr int E = Cfg::E, TL = Cfg::TL, COLS = Cfg::COLS, XP = Cfg::XP, EPC = Cfg::EPC;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    pdl_wait();
    if (A.pdl_early) pdl_trigger();
    if (A.ctrl->skipB) return;
    const int mode = A.mode;

    // two slots, each [D][N][COLS] as loaded, then the exchange lines [D * COLS][XP]
    const int w = threadIdx.x % COLS;
    const int t = (threadIdx.x / COLS) % TL;
    const int c = threadIdx.x / (COLS * TL);                                   // component plane
    const uint32_t bar0 = smem_u32(smem_raw + 2 * Cfg::SLOT_BYTES);
    const int nx = A.n[0];
    // n_inner need not be a multiple of COLS (the half-spectrum planes hold
    // n_x/2 + 1 columns within a padded pitch): the last group runs into padding
    const int64_t cblocks = (A.n_inner + COLS - 1) / COLS;
    const int64_t n_items = cblocks * A.n_outer;
    const bool leader = threadIdx.x == 0;

    auto load_item = [&](int64_t item, int b) {   // leader only
        const uint32_t bar = bar0 + 8 * b;
        mbar_expect_tx(bar, Cfg::ITEM_BYTES + A.extra_tx);
        tma_load_5d(smem_u32(smem_raw) + b * Cfg::SLOT_BYTES, &A.tmap, (int)((item % cblocks) * COLS * EPC), 0, 0,
                    (int)(item / cblocks), 0, bar);
    };

    if (leader) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int64_t item = blockIdx.x;
    if (leader) {
        if (item < n_items) load_item(item, 0);
        if (item + A.grid_blocks < n_items) load_item(item + A.grid_blocks, 1);
    }
    bool fault = false;
    for (uint32_t it = 0; item < n_items; item += A.grid_blocks, ++it) {
        const int b = it & 1;
        const int64_t after = item + 2 * (int64_t)A.grid_blocks;   // the next item for this buffer
        if (!mbar_wait(bar0 + 8 * b, (it >> 1) & 1u, A.wait_limit)) fault = true;
        C* Bi = reinterpret_cast<C*>(smem_raw + b * Cfg::SLOT_BYTES);
        C* Yc = Bi + c * N * COLS;                                             // this thread's plane
        C* Xb = Bi + (c * COLS + w) * XP;                                      // its exchange line
        C v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = Yc[(t + TL * m) * COLS + w];
        if (mode == MODE_COL_GAMMA) {
            // forward transforms, Gamma on every position of the item, inverse transforms
            LineFFT<T, N, E, Cfg::RMAX, false, Cfg::PAIRED>::run(v, Xb, t, A.tw);
            __syncthreads();   // the exchange lines share the slot: all reads done
#pragma unroll
            for (int m = 0; m < E; ++m) Yc[(t + TL * m) * COLS + w] = v[m];
            __syncthreads();
            const int64_t inner0 = (item % cblocks) * COLS;
            const bool two_d = A.line_axis == 1;   // 2-D: inner = kx, line = ky; 3-D z: inner = kx + nx ky
            // the COLS line starts of an item share ky (COLS divides nx): one division per item
            const int kx0 = two_d ? (int)inner0 : (int)(inner0 % nx);
            const int ky0 = two_d ? 0 : (int)(inner0 / nx);
            for (int p = threadIdx.x; p < N * COLS; p += Cfg::THREADS) {
                const int kl = p / COLS, wc = p % COLS;
                const int ki[3] = {kx0 + wc, two_d ? kl : ky0, two_d ? 0 : kl};
                C q[D];
#pragma unroll
                for (int cc = 0; cc < D; ++cc) q[cc] = Bi[(cc * N + kl) * COLS + wc];
                gamma_apply<T, D>(q, ki, A);
#pragma unroll
                for (int cc = 0; cc < D; ++cc) Bi[(cc * N + kl) * COLS + wc] = q[cc];
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = Yc[(t + TL * m) * COLS + w];
            LineFFT<T, N, E, Cfg::RMAX, true, Cfg::PAIRED>::run(v, Xb, t, A.tw);
        } else if (mode == MODE_COL_INV) {
            LineFFT<T, N, E, Cfg::RMAX, true, Cfg::PAIRED>::run(v, Xb, t, A.tw);
        } else {
            LineFFT<T, N, E, Cfg::RMAX, false, Cfg::PAIRED>::run(v, Xb, t, A.tw);
        }
        __syncthreads();   // every thread has read buffer b: refill it
        if (leader && after < n_items) load_item(after, b);
        C* dst = A.X + c * A.Ntot + (item / cblocks) * A.outer_stride + (item % cblocks) * COLS + w;
#pragma unroll
        for (int m = 0; m < E; ++m) dst[(int64_t)(t + TL * m) * A.ls] = v[m];
    }
    if (fault) atomicExch(&A.ctrl->fault, 1);
}

}  // namespace lsfft
