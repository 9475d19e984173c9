// Split layout for long 2-D columns (n_y = 4096 or 8192) in the packed real
// layout: the first radix-2 step of every y-DFT runs in the row pass, so the
// strided pass transforms independent columns of n_y / 2 points on one SM each
// and needs no exchange between SMs.
//
// Decimation in frequency along y (M = n_y / 2, W = exp(-2 pi i / n_y)):
//     a_j = x_j + x_{j+M},   b_j = (x_j - x_{j+M}) W^j,          j < M,
//     Xhat[2k]     = sum_j a_j W_M^(jk),   Xhat[2k + 1] = sum_j b_j W_M^(jk),
// and back: with A', B' the inverse M-point DFTs of the even and odd
// frequencies (the 1/N of the inverse DFT rides on the Gamma coefficients),
//     x'_j = A'_j + W^-j B'_j,   x'_{j+M} = A'_j - W^-j B'_j.
// Every x here is a row of x-spectra (two half-spectrum planes, X and Y, of the
// packed layout), and the butterflies act on them element by element.
//
// State between iterations: four half-spectrum planes [h][p][j][k_x] (h = 0: a,
// even k_y; h = 1: b, odd k_y; p = X, Y; j < M; row pitch n_x / 2 + 4).
//
// Row pass (row_pass_split<N>, N = n_x): one pair of rows (j, j + M) per work
// item and block.  The four staged half-rows (a'_j, b'_j of X and Y) and both
// mask rows arrive by bulk copies on one mbarrier; each thread forms the
// inverse butterfly and the join Z = X + i Y of both rows at its positions,
// parks row j + M in tensor memory, and the stage buffer is released for the
// next pair.  Each row then runs inverse x-DFT, scheme update and averages,
// forward x-DFT; the forward butterfly combines the two rows, and the split
// into half spectra (one shared-memory exchange per combined row) writes
// a_j and b_j.
//
// Strided pass (col_pass_split<M>): one work item is W = 2 adjacent columns of
// one half h, both planes; one TMA box (16-byte rows, M rows) per plane into
// three rotating slot buffers, a producer warp storing each slot as soon as it
// is done and refilling it.  Both planes are transformed forward in place,
// Gamma(k_x, k_y = 2k + h) runs over the item in shared memory, then the inverse
// DFTs run in place.
#pragma once

#include "lsfft_kernels.cuh"
#include "lsfft_tmem.cuh"

namespace lsfft {

template <int N>
struct SplitRowCfg {
    static constexpr int E = 16;
    static constexpr int TL = N / E;
    static constexpr int THREADS = TL;                         // one line of 16 points per thread
    static constexpr int HP = (int)half_pitch(N);
    static constexpr int XP = roundup16(N + N / 16);            // padded exchange line
    static constexpr int STAGE_BYTES = 4 * HP * 8;              // a'X, a'Y, b'X, b'Y
    static constexpr int MASK_BYTES = 2 * N;
    static constexpr int X_BYTES = XP * 8;
    static constexpr int SMEM = STAGE_BYTES + MASK_BYTES + X_BYTES + 16;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int COLS_PER_WARP = 64;                    // two parked lines, 32 columns each
    static constexpr int TMEM_COLS = ((WARPS + 3) / 4) * COLS_PER_WARP;
    static constexpr bool SUPPORTED = (N == 4096 || N == 8192) && SMEM <= 227 * 1024 && TMEM_COLS <= 512;
    static constexpr int MINB = min_blocks(SMEM, THREADS);
    static constexpr int NV = 9;                                // 4 d + 1 averages, d = 2
};

template <int M>
struct SplitColCfg {
    static constexpr int W = 2;                                 // adjacent columns per item: 16-byte rows
    static constexpr int E = 16;
    static constexpr int TL = M / E;
    static constexpr int COMPUTE = W * TL;                      // transform threads: one slot per round
    static constexpr int THREADS = COMPUTE + 32;                // + one producer warp for the TMA traffic
    static constexpr int PP = (M + M / 16 + 7) / 8 * 8;        // padded positions of the in-place transform
    static constexpr int BUF = (PP * W * 8 + 1023) / 1024 * 1024;
    static constexpr int NB = 3;                                // rotating slot buffers
    static constexpr int SLOT_BYTES = M * W * 8;                // one plane of an item, dense [j][w]
    static constexpr int SLOT_WARPS = COMPUTE / 32;
    static constexpr int SMEM = NB * BUF + 64;                  // + six mbarriers
    static constexpr bool SUPPORTED = (M == 2048 || M == 4096) && SMEM <= 227 * 1024 && M % 256 == 0;
};

// Scheme update of the packed real layout on one row, positions t + TL m of the
// thread (z = Q_x + i Q_y in v[m]); phase bits in incb; S, T rows at `base`.
// Adds the row's sums of E, J and |E|^2 to s[0..4]; writes E in output mode.
template <int SCH, int E_>
__device__ __forceinline__ void split_row_update(const PassArgs<float>& A, float2 (&v)[E_], uint32_t incb,
                                                 int64_t base, int t, int TL, bool wst, bool outm,
                                                 float (&s)[5]) {
    constexpr bool SUB = SCH == SCHEME_MS_SUB || SCH == SCHEME_EM_SUB;
    constexpr int HB = 4;
#pragma unroll
    for (int m0 = 0; m0 < E_; m0 += HB) {
        float2 sv[HB], tv[HB];
#pragma unroll
        for (int h = 0; h < HB; ++h) {
            const int pos = t + TL * (m0 + h);
            const bool inc = (incb >> (m0 + h)) & 1u;
            sv[h] = tv[h] = mkc(0.0f, 0.0f);
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
            float2 z = v[m], Ez, Jz;
            if (!SUB && A.sigma)
                pointwise_field_packed<float>(A.k, z, A.sigma[idx].x, Ez, Jz);
            else
                pointwise_packed<float, SCH>(A.k, z, inc, sv[h], tv[h], Ez, Jz);
            if constexpr (SUB) {
                if (inc && wst) {
                    A.S[idx] = sv[h];
                    if constexpr (SCH == SCHEME_EM_SUB) A.Tf[idx] = tv[h];
                }
            }
            v[m] = z;
            s[0] += Ez.x;
            s[1] += Jz.x;
            s[2] += Ez.y;
            s[3] += Jz.y;
            s[4] += Ez.x * Ez.x + Ez.y * Ez.y;
            if (outm) {
                A.Eout[idx] = mkc(Ez.x, 0.0f);
                A.Eout[A.Ntot + idx] = mkc(Ez.y, 0.0f);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Row pass on row pairs (j, j + M), specialised per scheme SCH.  A.X: the four
// planes, plane stride A.Nh = M * HP; A.n_lines = M; A.n[1] = n_y.
// ---------------------------------------------------------------------------
template <int N, int SCH>
__global__ void __launch_bounds__(SplitRowCfg<N>::THREADS, SplitRowCfg<N>::MINB)
row_pass_split(const PassArgs<float> A) {
    using Cfg = SplitRowCfg<N>;
    using C = float2;
    constexpr int E = Cfg::E, TL = Cfg::TL, HP = Cfg::HP;
    using FwdFFT = LineFFT<float, N, E, 16, false>;
    using InvFFT = LineFFT<float, N, E, 16, true>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();   // before any access and before the tensor-memory allocation
    if (A.pdl_early) pdl_trigger();
    const int mode = A.mode;
    if (mode != MODE_ROW_OUTPUT && A.ctrl->done) {   // uniform: before any allocation or barrier
        // the solve stopped before this update: its strided passes skip as well
        // (they run beside the finalize step and read only this flag)
        if (blockIdx.x == 0 && threadIdx.x == 0) A.ctrl->skipB = 1;
        return;
    }

    C* St = reinterpret_cast<C*>(smem_raw);                                         // [4][HP]
    const uint8_t* Mb = smem_raw + Cfg::STAGE_BYTES;                                // [2][N]
    C* Xb = reinterpret_cast<C*>(smem_raw + Cfg::STAGE_BYTES + Cfg::MASK_BYTES);    // exchange line
    const uint32_t bar = smem_u32(smem_raw + Cfg::STAGE_BYTES + Cfg::MASK_BYTES + Cfg::X_BYTES);
    // tensor-memory base address, written by the allocating warp (kept in the dynamic
    // region: a static shared variable would move the dynamic base)
    uint32_t& tmem_base_s = *reinterpret_cast<uint32_t*>(smem_raw + Cfg::STAGE_BYTES + Cfg::MASK_BYTES +
                                                         Cfg::X_BYTES + 8);
    const int t = threadIdx.x, warp = t >> 5;
    const int64_t M = A.n_lines;
    const float ny = (float)A.n[1];
    const bool stage_x = mode != MODE_ROW_FIRST;
    const bool wst = mode != MODE_ROW_OUTPUT, outm = mode == MODE_ROW_OUTPUT;

    if (warp == 0) tmem_alloc_warp(&tmem_base_s, Cfg::TMEM_COLS);
    if (t == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t park_in = tmem_warp_addr(tmem_base_s, warp, Cfg::COLS_PER_WARP), park_out = park_in + 32;

    // bulk copies need 16-byte aligned ends: checked once, a bad base is reported
    // and nothing is copied (the waits then run out and the solve reports a fault)
    const bool aligned = ((smem_u32(smem_raw) & 15u) == 0) && ((reinterpret_cast<uintptr_t>(A.X) & 15u) == 0) &&
                         ((reinterpret_cast<uintptr_t>(A.mask) & 15u) == 0);
    auto prefetch = [&](int64_t pair) {   // thread 0 only
        if (!aligned) {
            atomicExch(&A.ctrl->fault, 1);
            return;
        }
        mbar_expect_tx(bar, (stage_x ? Cfg::STAGE_BYTES : 0) + Cfg::MASK_BYTES + A.extra_tx);
        if (stage_x)
            for (int q = 0; q < 4; ++q)
                bulk_load(smem_u32(St + q * HP), A.X + q * A.Nh + pair * HP, HP * 8, bar);
        bulk_load(smem_u32(smem_raw + Cfg::STAGE_BYTES), A.mask + pair * N, N, bar);
        bulk_load(smem_u32(smem_raw + Cfg::STAGE_BYTES + N), A.mask + (pair + M) * N, N, bar);
    };

    float acc[Cfg::NV], cmp[Cfg::NV];
#pragma unroll
    for (int i = 0; i < Cfg::NV; ++i) acc[i] = cmp[i] = 0.0f;
    auto kahan_add = [&](int i, float x) {
        const float y = x - cmp[i];
        const float tsum = acc[i] + y;
        cmp[i] = (tsum - acc[i]) - y;
        acc[i] = tsum;
    };
    auto update_row = [&](C (&v)[E], uint32_t incb, int64_t row) {
        float s[5] = {0, 0, 0, 0, 0};
        const int64_t base = row * N;
        split_row_update<SCH>(A, v, incb, base, t, TL, wst, outm, s);
        kahan_add(0, s[0]);   // slots 1, 3, 5, 7 (imaginary parts) stay zero
        kahan_add(2, s[1]);
        kahan_add(4, s[2]);
        kahan_add(6, s[3]);
        kahan_add(8, s[4]);
    };
    auto first_field = [&](C (&v)[E], uint32_t incb, int64_t row) {   // Q = iq e (or the per-voxel reference)
#pragma unroll
        for (int m = 0; m < E; ++m) {
            float qv;
            if (A.sigma)
                qv = A.k.scheme == SCHEME_EM ? A.sigma[row * N + t + TL * m].x + A.k.s0.x : 1.0f;
            else
                qv = (incb >> m) & 1u ? A.k.iq_in.x : A.k.iq_out.x;
            v[m] = mkc(qv * A.k.e[0], qv * A.k.e[1]);
        }
    };
    // split of a combined row Z into half spectra, times w, stored to planes q, q + 1 at row j
    auto split_store = [&](const C (&v)[E], C w, int q, int64_t j) {
        __syncthreads();   // previous readers of the exchange line are done
#pragma unroll
        for (int m = 0; m < E; ++m) Xb[pad16(t + TL * m)] = v[m];
        __syncthreads();
        C* Hx = A.X + q * A.Nh + j * HP;
        C* Hy = Hx + A.Nh;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + TL * m;
            if (k <= N / 2) {
                const C z = v[m], zp = Xb[pad16((N - k) & (N - 1))];
                const C hx = mkc(0.5f * (z.x + zp.x), 0.5f * (z.y - zp.y));
                const C hy = mkc(0.5f * (z.y + zp.y), 0.5f * (zp.x - z.x));
                Hx[k] = cmul(hx, w);
                Hy[k] = cmul(hy, w);
            }
        }
    };

    bool fault = false;
    int64_t pair = blockIdx.x;
    if (t == 0 && pair < M) prefetch(pair);
    for (uint32_t it = 0; pair < M; pair += A.grid_blocks, ++it) {
        if (!mbar_wait(bar, it & 1u, A.wait_limit)) fault = true;
        uint32_t inc0 = 0, inc1 = 0;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            inc0 |= (Mb[t + TL * m] != 0 ? 1u : 0u) << m;
            inc1 |= (Mb[N + t + TL * m] != 0 ? 1u : 0u) << m;
        }
        float sw, cw;   // W^-j = exp(+2 pi i j / n_y)
        sincospif(2.0f * (float)pair / ny, &sw, &cw);
        C v0[E];
        // row j + M first (parked), then row j: sgn = -1, +1 in x = a' + sgn W^-j b'
        auto form = [&](C (&v)[E], float sgn, uint32_t incb, int64_t row) {
            if (!stage_x) {
                first_field(v, incb, row);
                return;
            }
            const C wm = mkc(sgn * cw, sgn * sw);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int k = t + TL * m;
                const int kk = k <= N / 2 ? k : N - k;
                const C x = cadd(St[kk], cmul(St[2 * HP + kk], wm));
                const C y = cadd(St[HP + kk], cmul(St[3 * HP + kk], wm));
                // Z = X + i Y at k <= N/2; Z(N - k) = conj X(k) + i conj Y(k) above
                v[m] = k <= N / 2 ? mkc(x.x - y.y, x.y + y.x) : mkc(x.x + y.y, y.x - x.y);
            }
        };
        form(v0, -1.0f, inc1, pair + M);
        tmem_park16(park_in, v0);
        form(v0, 1.0f, inc0, pair);
        __syncthreads();   // every thread has read the stage buffer and the mask rows
        if (t == 0 && pair + A.grid_blocks < M) prefetch(pair + A.grid_blocks);

        if (stage_x) InvFFT::run(v0, Xb, t, nullptr);
        update_row(v0, inc0, pair);
        if (!outm) {
            FwdFFT::run(v0, Xb, t, nullptr);
            tmem_park16(park_out, v0);
        }
        tmem_wait_st();
        tmem_fetch16(park_in, v0);
        if (stage_x) InvFFT::run(v0, Xb, t, nullptr);
        update_row(v0, inc1, pair + M);
        if (outm) {
            __syncthreads();   // the exchange line is reused by the next pair's transforms
            continue;
        }
        FwdFFT::run(v0, Xb, t, nullptr);
        // forward butterfly: a = Z_j + Z_{j+M} now, b = (Z_j - Z_{j+M}) parked until a is stored
        {
            C v1[E];
            tmem_wait_st();
            tmem_fetch16(park_out, v1);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const C a = cadd(v1[m], v0[m]), b = csub(v1[m], v0[m]);
                v0[m] = a;
                v1[m] = b;
            }
            tmem_park16(park_in, v1);
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            if (h == 1) {
                tmem_wait_st();
                tmem_fetch16(park_in, v0);
            }
            split_store(v0, h == 0 ? mkc(1.0f, 0.0f) : mkc(cw, -sw), 2 * h, pair);   // b times W^j
        }
    }
    __syncthreads();
    double dacc[Cfg::NV];
#pragma unroll
    for (int i = 0; i < Cfg::NV; ++i) dacc[i] = (double)acc[i] - (double)cmp[i];
    block_reduce_store<Cfg::NV, Cfg::THREADS>(dacc, A.partials + (int64_t)blockIdx.x * Cfg::NV);
    if (fault) atomicExch(&A.ctrl->fault, 1);

    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc_warp(tmem_base_s, Cfg::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Strided pass of the split layout: columns of M = n_y / 2 points, Gamma at
// k_y = 2k + h.  A.n_inner = n_x / 2 + 1 columns; A.tmap views the four planes
// (x element, row j0 < 256, row block j1, plane p, half h).
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(SplitColCfg<M>::THREADS, 1)
col_pass_split(const __grid_constant__ PassArgs<float> A) {
    using Cfg = SplitColCfg<M>;
    using C = float2;
    constexpr int W = Cfg::W, NB = Cfg::NB, E = Cfg::E, TL = Cfg::TL, COMPUTE = Cfg::COMPUTE;
    constexpr int BUFC = Cfg::BUF / 8;
    using FwdFFT = LineFFT<float, M, E, 16, false, false, COMPUTE, W>;
    using InvFFT = LineFFT<float, M, E, 16, true, false, COMPUTE, W>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    pdl_wait();
    if (A.pdl_early) pdl_trigger();
    if (A.ctrl->skipB) return;   // uniform over the grid
    // TMA tile destinations need a 128-byte aligned base: the kernel declares no
    // static shared variable, so the dynamic region starts at the window's origin.
    // Checked rather than assumed: a misaligned base is reported, not used.
    if (smem_u32(smem_raw) & 1023u) {
        if (threadIdx.x == 0) atomicExch(&A.ctrl->fault, 1);
        return;
    }

    C* Y = reinterpret_cast<C*>(smem_raw);
    const bool producer = threadIdx.x >= COMPUTE;
    const int w = threadIdx.x % W;
    const int t = (threadIdx.x / W) % TL;
    // mbarriers: full[b] at bar0 + 8 b, done[b] at bar0 + 24 + 8 b
    const uint32_t bar0 = smem_u32(smem_raw + NB * Cfg::BUF);
    const int64_t G = (A.n_inner + W - 1) / W;   // column groups per half
    const int64_t n_items = 2 * G;
    const int64_t cid = blockIdx.x, ncl = gridDim.x;
    const int64_t my_items = cid < n_items ? (n_items - cid + ncl - 1) / ncl : 0;
    const int64_t QN = 2 * my_items;             // slots of this block: q = 2 it + p
    const bool leader = threadIdx.x == COMPUTE;

    auto load_q = [&](int64_t qq) {              // producer only
        const int b = (int)(qq % NB);
        const int64_t item = cid + (qq / 2) * ncl;
        mbar_expect_tx(bar0 + 8 * b, Cfg::SLOT_BYTES + A.extra_tx);
        tma_load_5d(smem_u32(Y + b * BUFC), &A.tmap, (int)((item % G) * W), 0, 0, (int)(qq & 1), (int)(item / G),
                    bar0 + 8 * b);
    };
    auto store_q = [&](int64_t qq) {             // producer only
        const int b = (int)(qq % NB);
        const int64_t item = cid + (qq / 2) * ncl;
        tma_store_5d(&A.tmap, (int)((item % G) * W), 0, 0, (int)(qq & 1), (int)(item / G), smem_u32(Y + b * BUFC));
        bulk_commit();
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
    if (producer) {
        if (leader) {
            for (int64_t qq = 0; qq < NB && qq < QN; ++qq) load_q(qq);
            // per item: the Y plane finishes first, then X; each buffer still receives
            // its slots in increasing order (q and q + NB)
            for (int64_t it = 0; it < my_items; ++it) {
                for (int s = 1; s >= 0; --s) {
                    const int64_t qq = 2 * it + s;
                    const int b = (int)(qq % NB);
                    if (!mbar_wait(bar0 + 24 + 8 * b, (uint32_t)((qq / NB) & 1), A.wait_limit)) fault = true;
                    store_q(qq);
                    bulk_wait_read(0);
                    if (qq + NB < QN) load_q(qq + NB);
                }
            }
            bulk_wait_all();
        }
        __syncwarp();
    } else {
        for (int64_t it = 0; it < my_items; ++it) {
            const int64_t item = cid + it * ncl;
            const int h = (int)(item / G);
            C* const Bx = Y + (int)((2 * it) % NB) * BUFC;       // plane X of the item
            C* const By = Y + (int)((2 * it + 1) % NB) * BUFC;   // plane Y
            // forward DFTs of both planes in place, results back in natural order
#pragma unroll 1
            for (int p = 0; p < 2; ++p) {
                const int64_t qq = 2 * it + p;
                const int b = (int)(qq % NB);
                C* Bp = Y + b * BUFC;
                if (!mbar_wait(bar0 + 8 * b, (uint32_t)((qq / NB) & 1), A.wait_limit)) fault = true;
                C v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = Bp[(t + TL * m) * W + w];
                FwdFFT::run(v, Bp + w, t, nullptr);
                line_sync<COMPUTE>();   // every thread has read its last-stage inputs
#pragma unroll
                for (int m = 0; m < E; ++m) Bp[(t + TL * m) * W + w] = v[m];
            }
            line_sync<COMPUTE>();
            // Gamma on both planes at (k_x, k_y = 2 k + h)
            const int kx0 = (int)((item % G) * W);
            for (int pidx = threadIdx.x; pidx < M * W; pidx += COMPUTE) {
                const int kl = pidx / W, wc = pidx % W;
                C q[2] = {Bx[pidx], By[pidx]};
                const int ki[3] = {kx0 + wc, 2 * kl + h, 0};
                gamma_apply<float, 2>(q, ki, A);
                Bx[pidx] = q[0];
                By[pidx] = q[1];
            }
            line_sync<COMPUTE>();
            // inverse DFTs in place, plane Y then X; each slot is handed to the
            // producer warp when its transform is done
#pragma unroll 1
            for (int p = 1; p >= 0; --p) {
                const int64_t qq = 2 * it + p;
                const int b = (int)(qq % NB);
                C* Bp = Y + b * BUFC;
                C v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = Bp[(t + TL * m) * W + w];
                InvFFT::run(v, Bp + w, t, nullptr);
                line_sync<COMPUTE>();
#pragma unroll
                for (int m = 0; m < E; ++m) Bp[(t + TL * m) * W + w] = v[m];
                fence_proxy_async_smem();   // the TMA store reads what the threads wrote
                __syncwarp();
                if ((threadIdx.x & 31) == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar0 + 24 + 8 * b) : "memory");
            }
        }
    }
    if (fault) atomicExch(&A.ctrl->fault, 1);
}

}  // namespace lsfft
