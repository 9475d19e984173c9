// Shared-memory Stockham FFT of one line, held in registers between stages.
//
// A line of N complex points (N a power of two) is owned by T_LINE = N/E
// threads; thread t holds the elements with index t + T_LINE*m, m = 0..E-1,
// in v[m].  fft_line<...>::run() returns, in the same layout, the unnormalised
// DFT  X[k] = sum_j x[j] exp(-+2 pi i j k / N)  (forward sign -, inverse +).
//
// Stage s (radix R <= RMAX, NS = product of earlier radices): butterfly j
// (0 <= j < N/R) takes x[j + r N/R], r = 0..R-1, multiplies leg r by
// W_{NS R}^{(j mod NS) r}, forms a radix-R DFT in registers and writes leg r to
// position (j / NS) NS R + (j mod NS) + r NS.  With thread t handling
// j = t + T_LINE*i, its inputs are always x[t + T_LINE*m], so every stage reads
// shared memory with unit stride across threads, and the last stage (NS R = N)
// writes its outputs straight back into the thread's own registers in natural
// order: no shared-memory pass after it.  Shared memory is padded with one
// slot per 16 elements so that the strided writes of the first stage do not
// collide in banks.
//
// Twiddles: FP32 uses sincospif() for W^{(j mod NS)} once per butterfly and
// forms the other powers as products of W^{jm}, W^{2jm}, W^{4jm}, W^{8jm};
// FP64 reads them from a table W_L^k built on the host in double precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lsfft {

template <typename T> struct CxOf;
template <> struct CxOf<float> { using type = float2; };
template <> struct CxOf<double> { using type = double2; };
template <typename T> using cx = typename CxOf<T>::type;

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cneg(C a) { return mkc(-a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return mkc(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return mkc(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }


// cos and sin of 2 pi k / 16 (mathematical constants), written as a select
// chain so that a compile-time k folds to a literal.
__device__ __forceinline__ double cos16(int k) {
    k &= 15;
    const int m = k <= 8 ? k : 16 - k;             // cos is even
    return m == 0 ? 1.0 : m == 1 ? 0.92387953251128675613 : m == 2 ? 0.70710678118654752440
         : m == 3 ? 0.38268343236508977173 : m == 4 ? 0.0 : m == 5 ? -0.38268343236508977173
         : m == 6 ? -0.70710678118654752440 : m == 7 ? -0.92387953251128675613 : -1.0;
}
__device__ __forceinline__ double sin16(int k) { return cos16(k + 12); }

// a * exp(-+2 pi i q / 16), q a compile-time constant after unrolling.
template <bool INV, typename C>
__device__ __forceinline__ C mul_root16(C a, int q) {
    using T = decltype(a.x);
    q &= 15;
    if (q == 0) return a;
    if (q == 8) return cneg(a);
    if (q == 4) return INV ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
    if (q == 12) return INV ? mkc(a.y, -a.x) : mkc(-a.y, a.x);
    const T c = (T)cos16(q);
    const T s = INV ? (T)sin16(q) : -(T)sin16(q);
    if (q == 2 || q == 6 || q == 10 || q == 14) {
        const T h = (T)0.70710678118654752440;
        // c and s are +-h
        const T cs = c > 0 ? h : -h, ss = s > 0 ? h : -h;
        return mkc(cs * a.x - ss * a.y, cs * a.y + ss * a.x);
    }
    return mkc(c * a.x - s * a.y, c * a.y + s * a.x);
}

// Paired FP32 arithmetic (sm_100 family): one instruction applies the same
// operation to both halves of a 64-bit register pair, so a complex add or
// subtract issues once instead of twice.  Its operands must sit in aligned
// register pairs, which costs moves where registers are scarce: the kernels
// enable it only where they run at most 256 threads per block.
__device__ __forceinline__ unsigned long long pk2(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
    return upk2(d);
}

// Radix-2 butterfly with the odd leg rotated by exp(-+2 pi i q / 16):
// (e + w o, e - w o).
template <bool INV, bool PAIRED, typename C>
__device__ __forceinline__ void butterfly16(const C& e, const C& o, int q, C& lo, C& hi) {
    using T = decltype(e.x);
    q &= 15;
    if constexpr (PAIRED && sizeof(T) == 4) {
        if (q == 0) {
            lo = add2(e, o);
            hi = sub2(e, o);
            return;
        }
        if (q != 4 && q != 8 && q != 12) {
            // w o = (c, c) o + (-s, s) (o.y, o.x) with w = c + i s
            const float c = (float)cos16(q);
            const float s = INV ? (float)sin16(q) : -(float)sin16(q);
            const float2 t = fma2(mkc(-s, s), mkc(o.y, o.x), mul2(mkc(c, c), o));
            lo = add2(e, t);
            hi = sub2(e, t);
            return;
        }
    }
    const C t = mul_root16<INV>(o, q);
    lo = cadd(e, t);
    hi = csub(e, t);
}

// In-register DFT of the R elements a[OFF + STRIDE*i] (R | 16) into out[0..R-1],
// natural order, by recursive even/odd splitting; every index is a template
// constant so the whole transform stays in registers.
template <int R, int STRIDE, int OFF, bool INV, bool PAIRED, typename C, int NA>
__device__ __forceinline__ void dft_rec(const C (&a)[NA], C (&out)[R]) {
    if constexpr (R == 1) {
        out[0] = a[OFF];
    } else {
        C ev[R / 2], od[R / 2];
        dft_rec<R / 2, 2 * STRIDE, OFF, INV, PAIRED>(a, ev);
        dft_rec<R / 2, 2 * STRIDE, OFF + STRIDE, INV, PAIRED>(a, od);
#pragma unroll
        for (int k = 0; k < R / 2; ++k)
            butterfly16<INV, PAIRED>(ev[k], od[k], k * (16 / R), out[k], out[k + R / 2]);
    }
}

template <int R, bool INV, bool PAIRED, typename C>
__device__ __forceinline__ void dft(C (&a)[R]) {
    C out[R];
    dft_rec<R, 1, 0, INV, PAIRED>(a, out);
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = out[i];
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <int N> struct LinePad { static constexpr int size = N + N / 16 + 1; };

// Barrier over the threads that run line transforms: the whole block, or (SYNC
// > 0) the first SYNC threads on hardware barrier 1, when other warps of the
// block do other work.
template <int SYNC>
__device__ __forceinline__ void line_sync() {
    if constexpr (SYNC == 0) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"n"(SYNC) : "memory");
}

// Number of stages of an n-point line transform with radices <= rmax that
// exchange through shared memory (all but the last).
__host__ __device__ constexpr int line_exchanges(int n, int rmax) {
    int ns = 1, k = 0;
    while (ns * (n / ns >= rmax ? rmax : n / ns) < n) {
        ns *= (n / ns >= rmax ? rmax : n / ns);
        ++k;
    }
    return k;
}

// SMS: element stride of the exchange line in shared memory (SMS lines
// interleaved position by position share one buffer).
template <typename T, int N, int E, int RMAX, bool INV, bool PAIRED = false, int SYNC = 0, int SMS = 1>
struct LineFFT {
    using C = cx<T>;
    static constexpr int TL = N / E;   // threads per line
    static_assert(N % E == 0, "E must divide N");

    template <int R>
    __device__ __forceinline__ static void twiddle(C (&a)[R], int jm, int span, const C* __restrict__ tw,
                                                   int tws) {
        // a[r] *= W_span^{jm r}, forward W = exp(-2 pi i / span)
        if constexpr (sizeof(T) == 4) {
            // W^(jm r), r = lo + 4 hi (lo, hi < 4), as W^(jm lo) W^(4 jm hi): the
            // powers 1..3 and 4, 8, 12 of W^(jm) from one sincospif and five
            // products, then one product for each r with lo, hi both nonzero
            // (14 complex products for R = 16).  Each power is formed when needed,
            // so no table of R twiddles stays live in registers.
            float s, c;
            sincospif(2.0f * (float)jm / (float)span, &s, &c);
            C p[4], h[4];
            p[0] = h[0] = mkc(1.0f, 0.0f);
            p[1] = mkc(c, INV ? s : -s);
            if constexpr (R > 2) p[2] = cmul(p[1], p[1]);
            if constexpr (R > 3) p[3] = cmul(p[2], p[1]);
            if constexpr (R > 4) h[1] = cmul(p[2], p[2]);
            if constexpr (R > 8) h[2] = cmul(h[1], h[1]);
            if constexpr (R > 12) h[3] = cmul(h[2], h[1]);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const int lo = r & 3, hi = r >> 2;
                const C w = lo == 0 ? h[hi] : hi == 0 ? p[lo] : cmul(h[hi], p[lo]);
                a[r] = cmul(a[r], w);
            }
        } else {
            const int step = (N / span) * jm * tws;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[step * r];
                if (INV) w = cconj(w);
                a[r] = cmul(a[r], w);
            }
        }
    }

    // FP64 lines of two points per thread (radix 2 throughout): every stage's
    // single twiddle is loaded up front, so that the table reads of the stages
    // are in flight together instead of one cache latency per stage.
    static constexpr bool PRE = sizeof(T) == 8 && E == 2 && RMAX == 2;
    static constexpr int LOGN = ilog2c(N);

    static constexpr int NEX = line_exchanges(N, RMAX);

    // DB: the stages alternate between two exchange buffers (sm, then sm2, ...), so
    // that a stage writes a buffer whose last readers have already passed the
    // previous stage's barrier: one barrier per stage instead of two.
    template <int NS, bool DB = false>
    __device__ __forceinline__ static void stage(C (&v)[E], C* __restrict__ sm, int t, const C* __restrict__ tw,
                                                 int tws, const C* pre, C* __restrict__ sm2 = nullptr) {
        constexpr int REM = N / NS;
        constexpr int R = REM >= RMAX ? RMAX : REM;
        constexpr bool LAST = (NS * R == N);
        constexpr int B = E / R;
        static_assert(E % R == 0, "radix must divide E");
        if constexpr (!LAST && !DB) line_sync<SYNC>();   // previous readers of sm are done
        // A last stage with several butterflies per thread (R < E): butterfly i has
        // j = t + TL i < NS, so its twiddles W_N^((t + TL i) r) = W_N^(t r) W_E^(i r)
        // share the powers of W_N^t and differ by exact 16th roots of unity
        // (FP32; FP64 reads its table).
        constexpr bool SHARED_TW = LAST && B > 1 && NS > 1 && sizeof(T) == 4 && (16 % E == 0);
        C pw[R];
        if constexpr (SHARED_TW) {
            float s, c;
            sincospif(2.0f * (float)t / (float)N, &s, &c);
            pw[0] = mkc((T)1, (T)0);
            pw[1] = mkc(c, INV ? s : -s);
#pragma unroll
            for (int r = 2; r < R; ++r) pw[r] = cmul(pw[r - 1], pw[1]);
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int j = t + TL * i;
            C a[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = v[i + r * B];
            if constexpr (SHARED_TW) {
#pragma unroll
                for (int r = 1; r < R; ++r) a[r] = cmul(a[r], mul_root16<INV>(pw[r], (i * r * (16 / E)) & 15));
            } else if constexpr (NS > 1 && PRE) {
                a[1] = INV ? cmulc(a[1], pre[ilog2c(NS)]) : cmul(a[1], pre[ilog2c(NS)]);
            } else if constexpr (NS > 1) {
                twiddle<R>(a, j % NS, NS * R, tw, tws);
            }
            dft<R, INV, PAIRED>(a);
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[i + r * B] = a[r];
            } else {
                const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
                for (int r = 0; r < R; ++r) sm[pad16(base + r * NS) * SMS] = a[r];
            }
        }
        if constexpr (!LAST) {
            line_sync<SYNC>();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = sm[pad16(t + TL * m) * SMS];
            if constexpr (DB) stage<NS * R, true>(v, sm2, t, tw, tws, pre, sm);
            else stage<NS * R>(v, sm, t, tw, tws, pre);
        }
    }

    // Must be called by every thread of the block (or of the SYNC transform
    // threads: it contains barriers whenever N > RMAX); threads of inactive lines
    // pass dummy data.  FP64:
    // `tw` holds W_L^k of a length L = N * tws (tws = 1 unless the line is a
    // decimated part of a longer one).
    __device__ __forceinline__ static void run(C (&v)[E], C* __restrict__ sm, int t, const C* __restrict__ tw,
                                               int tws = 1) {
        C pre[PRE ? LOGN : 1];
        if constexpr (PRE) {
            // stage NS = 2^s (s >= 1): W_{2 NS}^(t mod NS) = W_L^((N / (2 NS)) (t mod NS) tws)
#pragma unroll
            for (int s = 1; s < LOGN; ++s) pre[s] = tw[(int64_t)(N >> (s + 1)) * (t & ((1 << s) - 1)) * tws];
        }
        stage<1>(v, sm, t, tw, tws, pre);
    }

    // The same transform with the exchanges alternating between sm (first) and
    // sm2.  No barrier precedes the first write into sm: the caller guarantees
    // that no thread of the line group still reads it.
    __device__ __forceinline__ static void run2(C (&v)[E], C* __restrict__ sm, C* __restrict__ sm2, int t,
                                                const C* __restrict__ tw, int tws = 1) {
        static_assert(!PRE, "two-point FP64 lines keep the single-buffer form");
        stage<1, true>(v, sm, t, tw, tws, nullptr, sm2);
    }
};

}  // namespace lsfft
