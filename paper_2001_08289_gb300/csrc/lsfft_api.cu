// Host side of the C ABI declared in include/lsfft.h: argument checks, scheme
// constants in FP64, workspace, the CUDA-graph iteration loop and results.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>
#include <string>
#include <tuple>

#include "lsfft.h"
#include "lsfft_kernels.cuh"
#include "lsfft_misc.h"
#include "lsfft_sweep.h"

using namespace lsfft;
using cplx = std::complex<double>;

static thread_local std::string g_last_error;

#define LSFFT_VERSION_STRING "lsfft-gb300 0.1 (sm_103a)"

namespace {

int fail_cuda(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    g_last_error = buf;
    return LSFFT_ECUDA;
}

#define CK(...)                                                    \
    do {                                                           \
        cudaError_t _e = (__VA_ARGS__);                            \
        if (_e != cudaSuccess) return fail_cuda(_e, #__VA_ARGS__); \
    } while (0)

constexpr double kPi = 3.14159265358979323846;

// Stream-ordered memory pool (one per device) for the large buffers: grid
// workspaces and result fields.  A freed block stays cached in the pool for the
// next grid or solve instead of being unmapped and mapped again (a 1 GB field
// cost about 1.4 ms per cudaFree from the default pool, which returns memory at
// every synchronisation); the pool is trimmed once no such buffer is alive.
struct BigPool {
    std::mutex mu;
    cudaMemPool_t pool[64] = {};
    long live = 0;
};
BigPool& big_pool() {
    static BigPool p;
    return p;
}

cudaError_t big_alloc(void** ptr, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    BigPool& P = big_pool();
    std::lock_guard<std::mutex> lk(P.mu);
    if (!P.pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&P.pool[dev], &props);
        if (e != cudaSuccess) {
            P.pool[dev] = nullptr;
            return e;
        }
        unsigned long long keep = ~0ull;
        e = cudaMemPoolSetAttribute(P.pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    e = cudaMallocFromPoolAsync(ptr, bytes, P.pool[dev], s);
    if (e == cudaSuccess) ++P.live;
    return e;
}

// Release a big_alloc buffer (waits for the device, as cudaFree does); null is a no-op.
void big_free(void* ptr) {
    if (!ptr) return;
    cudaFree(ptr);
    BigPool& P = big_pool();
    std::lock_guard<std::mutex> lk(P.mu);
    if (--P.live == 0)
        for (int d = 0; d < 64; ++d)
            if (P.pool[d]) cudaMemPoolTrimTo(P.pool[d], 0);
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2i(int64_t v) {
    int r = 0;
    while ((int64_t(1) << r) < v) ++r;
    return r;
}
void put(double (&dst)[2], cplx v) {
    dst[0] = v.real();
    dst[1] = v.imag();
}

struct GraphKey {
    int precision, st, check_every;
    bool operator<(const GraphKey& o) const {
        return std::tie(precision, st, check_every) < std::tie(o.precision, o.st, o.check_every);
    }
};

}  // namespace

struct lsfft_grid {
    int d = 0;
    int64_t n[3] = {1, 1, 1};
    int logn[3] = {0, 0, 0};
    int64_t N = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;        // created by the library when the caller passed NULL
    // the finalize step of each update runs on a stream of its own, beside the
    // strided pass (which does not read its result), joined before the next row pass
    cudaStream_t fin_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    int sm_count = 0;
    uint8_t* mask = nullptr;
    // workspace
    int ws_prec = -1;
    int ws_st = -1;                 // 0: Q only, 1: Q and S, 2: Q, S and T
    void* X = nullptr;
    void* S = nullptr;
    void* T = nullptr;
    double* partials = nullptr;
    int64_t partials_cap = 0;
    double* hist = nullptr;
    int hist_cap = 0;
    SchemeParams* prm_host = nullptr;   // constants of the current solve (kernel parameters)
    Ctrl* ctrl_dev = nullptr;
    Ctrl* ctrl_host = nullptr;          // pinned
    Ctrl* ctrl_host_dev = nullptr;      // its device view (written by a small kernel)
    void* tw[3] = {nullptr, nullptr, nullptr};   // FP64 twiddles W_n^k per axis
    void* fd[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};   // FD symbol per axis, FP32/FP64
    bool prepared[2] = {false, false};
    int packed = 0;                 // packed real layout for the current solve
    int split = 0;                  // packed FP32 2-D with n_y >= 4096: split layout (lsfft_split.cuh)
    bool no_split = true;           // lsfft_set_column_split(grid, 1) selects the split layout
    // solve in flight (begin_solve / poll_solve)
    int phase = 0;                  // 0 idle, 1 in flight
    bool phase_finish = false;      // the output pass has been enqueued
    cudaGraphExec_t cur_exec = nullptr;
    int cur_st = 0, cur_nblocks = 0, cur_per_iter = 0, cur_check_every = 0;
    int64_t cur_launches = 0, cur_max_launches = 0, cur_kernels = 0;
    void* cur_E = nullptr;
    lsfft_result* cur_res = nullptr;
    double* hist_host = nullptr;    // pinned copy of the history
    double* hist_host_dev = nullptr;   // its device view
    int hist_host_cap = 0;
    cudaEvent_t ev_check = nullptr;
    // per-voxel conductivity mode (lsfft_set_sigma_field)
    double2* sigma64 = nullptr;     // device copy, FP64 complex [N]
    void* sigma_t = nullptr;        // the same in the precision of the last solve
    int sigma_t_prec = -1;
    double sig_min = 0.0, sig_max = 0.0;   // extremes of Re sigma
    bool sig_real = false;
    double sigma0_user[2] = {0.0, 0.0};
    int bench_prec = -1;            // precision of the state set up by lsfft_prepare (-1: none)
    int inject_tx = 0;              // test hook (lsfft_debug_inject): TMA bytes announced, never sent
    long long wait_limit = MBAR_WAIT_LIMIT;
    int bench_st = 0;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

// Both of the grid's streams (the finalize stream is joined into the main one
// after every update, but not on an error path).
void sync_grid(lsfft_grid* g) {
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->fin_stream) cudaStreamSynchronize(g->fin_stream);
}

void clear_graphs(lsfft_grid* g) {
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
    g->graphs.clear();
}

Geom row_geom(const lsfft_grid* g, int prec) {
    Geom geo;
    if (prec == LSFFT_FP32) {
        if (g->d == 2) row_dispatch<float, 2>(g->logn[0], OP_QUERY, nullptr, nullptr, &geo);
        else row_dispatch<float, 3>(g->logn[0], OP_QUERY, nullptr, nullptr, &geo);
    } else {
        if (g->d == 2) row_dispatch<double, 2>(g->logn[0], OP_QUERY, nullptr, nullptr, &geo);
        else row_dispatch<double, 3>(g->logn[0], OP_QUERY, nullptr, nullptr, &geo);
    }
    return geo;
}

int64_t persistent_blocks(const lsfft_grid* g, int64_t n_items, int blocks_per_sm) {
    const int64_t cap = (int64_t)g->sm_count * (blocks_per_sm > 0 ? blocks_per_sm : 1);
    return n_items < cap ? n_items : cap;
}

// The split layout of long 2-D columns: FP32 packed fields, n_x and n_y in {4096, 8192}.
bool split_shape(const lsfft_grid* g) {
    return g->d == 2 && (g->n[0] == 4096 || g->n[0] == 8192) && (g->n[1] == 4096 || g->n[1] == 8192);
}

// Number of row-pass blocks (= partial-sum rows), valid after the kernels were prepared.
int row_blocks(const lsfft_grid* g, int prec) {
    if (g->split && prec == LSFFT_FP32) {
        Geom geo;
        split_row_dispatch(g->logn[0], OP_QUERY, nullptr, nullptr, &geo);
        return (int)persistent_blocks(g, g->n[1] / 2, geo.blocks_per_sm);
    }
    const Geom geo = row_geom(g, prec);
    const int64_t rows = g->N / g->n[0];
    return (int)persistent_blocks(g, (rows + geo.per_block - 1) / geo.per_block, geo.blocks_per_sm);
}

template <typename T>
bool col_supported(const lsfft_grid* g) {
    Geom rg = row_geom(g, sizeof(T) == 4 ? LSFFT_FP32 : LSFFT_FP64);
    if (!rg.supported) return false;
    for (int a = 1; a < g->d; ++a) {
        Geom geo;
        if (g->d == 2) col_dispatch<T, 2>(g->logn[a], OP_QUERY, nullptr, nullptr, &geo);
        else col_dispatch<T, 3>(g->logn[a], OP_QUERY, nullptr, nullptr, &geo);
        if (!geo.supported) return false;
    }
    return true;
}

template <typename T>
int prepare_kernels(lsfft_grid* g) {
    if (g->d == 2) {
        CK(row_dispatch<T, 2>(g->logn[0], OP_PREPARE, nullptr, nullptr, nullptr));
        CK(col_dispatch<T, 2>(g->logn[1], OP_PREPARE, nullptr, nullptr, nullptr));
        if (sizeof(T) == 4 && split_shape(g)) {
            CK(split_row_dispatch(g->logn[0], OP_PREPARE, nullptr, nullptr, nullptr));
            CK(split_col_dispatch(g->logn[1] - 1, OP_PREPARE, nullptr, nullptr, nullptr));
        }
    } else {
        CK(row_dispatch<T, 3>(g->logn[0], OP_PREPARE, nullptr, nullptr, nullptr));
        CK(col_dispatch<T, 3>(g->logn[1], OP_PREPARE, nullptr, nullptr, nullptr));
        CK(col_dispatch<T, 3>(g->logn[2], OP_PREPARE, nullptr, nullptr, nullptr));
    }
    return LSFFT_OK;
}

int ensure_workspace(lsfft_grid* g, int prec, int st, int max_iter) {
    if (g->ws_prec != prec || g->ws_st < st) {
        clear_graphs(g);
        big_free(g->X);
        big_free(g->S);
        big_free(g->T);
        g->X = g->S = g->T = nullptr;
        g->ws_prec = -1;
        const size_t bytes = (size_t)g->d * g->N * (prec == LSFFT_FP32 ? 8 : 16);
        if (big_alloc(&g->X, bytes, g->stream) != cudaSuccess) return fail_cuda(cudaErrorMemoryAllocation, "workspace X");
        if (st >= 1 && big_alloc(&g->S, bytes, g->stream) != cudaSuccess)
            return fail_cuda(cudaErrorMemoryAllocation, "workspace S");
        if (st >= 2 && big_alloc(&g->T, bytes, g->stream) != cudaSuccess)
            return fail_cuda(cudaErrorMemoryAllocation, "workspace T");
        g->ws_prec = prec;
        g->ws_st = st;
    }
    const int64_t need = (int64_t)g->sm_count * 32 * (4 * g->d + 1);   // >= any persistent row grid
    if (need > g->partials_cap) {
        clear_graphs(g);
        cudaFree(g->partials);
        g->partials = nullptr;
        g->partials_cap = 0;
        CK(cudaMalloc(&g->partials, need * sizeof(double)));
        g->partials_cap = need;
    }
    if (max_iter + 1 > g->hist_cap) {
        clear_graphs(g);
        cudaFree(g->hist);
        g->hist = nullptr;
        g->hist_cap = 0;
        CK(cudaMalloc(&g->hist, (size_t)(max_iter + 1) * HIST_STRIDE * sizeof(double)));
        g->hist_cap = max_iter + 1;
    }
    return LSFFT_OK;
}

// Tables built in FP64 on the host: twiddles W_n^k = exp(-2 pi i k/n) and the
// forward-difference symbol u(k) = exp(2 pi i k/n) - 1 = -2 sin^2(pi k/n) + i sin(2 pi k/n).
int build_tables(lsfft_grid* g) {
    for (int a = 0; a < g->d; ++a) {
        const int64_t n = g->n[a];
        double* tw = (double*)malloc(sizeof(double) * 2 * n);
        double* fd64 = (double*)malloc(sizeof(double) * 2 * n);
        float* fd32 = (float*)malloc(sizeof(float) * 2 * n);
        if (!tw || !fd64 || !fd32) {
            free(tw);
            free(fd64);
            free(fd32);
            return LSFFT_ENOMEM;
        }
        for (int64_t k = 0; k < n; ++k) {
            const double th = 2.0 * kPi * (double)k / (double)n;
            tw[2 * k] = cos(th);
            tw[2 * k + 1] = -sin(th);
            const double h = sin(kPi * (double)k / (double)n);
            fd64[2 * k] = -2.0 * h * h;
            fd64[2 * k + 1] = sin(th);
            fd32[2 * k] = (float)fd64[2 * k];
            fd32[2 * k + 1] = (float)fd64[2 * k + 1];
        }
        int rc = LSFFT_OK;
        if (cudaMalloc(&g->tw[a], sizeof(double) * 2 * n) != cudaSuccess ||
            cudaMalloc(&g->fd[a][1], sizeof(double) * 2 * n) != cudaSuccess ||
            cudaMalloc(&g->fd[a][0], sizeof(float) * 2 * n) != cudaSuccess)
            rc = fail_cuda(cudaErrorMemoryAllocation, "tables");
        if (rc == LSFFT_OK) {
            cudaError_t e = cudaMemcpy(g->tw[a], tw, sizeof(double) * 2 * n, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(g->fd[a][1], fd64, sizeof(double) * 2 * n, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(g->fd[a][0], fd32, sizeof(float) * 2 * n, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) rc = fail_cuda(e, "table upload");
        }
        free(tw);
        free(fd64);
        free(fd32);
        if (rc != LSFFT_OK) return rc;
    }
    return LSFFT_OK;
}

int create_common(int d, const int64_t n[3], const uint8_t* mask, bool on_device, void* stream, lsfft_grid** out) {
    if (!out || !n || !mask) {
        g_last_error = "null argument";
        return LSFFT_EINVAL;
    }
    *out = nullptr;
    if (d != 2 && d != 3) {
        g_last_error = "d must be 2 or 3";
        return LSFFT_EINVAL;
    }
    const int64_t nmax = d == 2 ? 8192 : 512;
    for (int a = 0; a < d; ++a) {
        if (!is_pow2(n[a]) || n[a] < 16 || n[a] > nmax) {
            g_last_error = "every n[a] must be a power of two in [16, 8192] (2-D) or [16, 512] (3-D)";
            return LSFFT_EINVAL;
        }
    }
    lsfft_grid* g = new (std::nothrow) lsfft_grid();
    if (!g) return LSFFT_ENOMEM;
    g->d = d;
    g->N = 1;
    for (int a = 0; a < d; ++a) {
        g->n[a] = n[a];
        g->logn[a] = ilog2i(n[a]);
        g->N *= n[a];
    }
    g->stream = (cudaStream_t)stream;
    int rc = LSFFT_OK;
    cudaError_t e = cudaSuccess;
    if (!g->stream) {
        // CUDA graphs cannot be captured on the legacy default stream.
        e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
        g->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaMalloc(&g->mask, (size_t)g->N);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->mask, mask, (size_t)g->N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            g->stream);
    if (e == cudaSuccess) {
        g->prm_host = new (std::nothrow) SchemeParams();
        if (!g->prm_host) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaMalloc(&g->ctrl_dev, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost(&g->ctrl_host, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&g->ctrl_host_dev, g->ctrl_host, 0);
    if (e == cudaSuccess) e = cudaEventCreate(&g->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&g->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_check, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->fin_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = fail_cuda(e, "create_grid");
    if (rc == LSFFT_OK) rc = build_tables(g);
    if (rc == LSFFT_OK) {
        e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) rc = fail_cuda(e, "create_grid sync");
    }
    if (rc != LSFFT_OK) {
        lsfft_destroy_grid(g);
        return rc;
    }
    *out = g;
    return LSFFT_OK;
}

bool finite_c(cplx v) { return std::isfinite(v.real()) && std::isfinite(v.imag()); }

// Scheme constants (FP64).  Returns an empty string if valid, else the reason.
std::string build_params(const lsfft_grid* g, cplx s1, const double* e, const lsfft_opts* o, SchemeParams* P) {
    memset(P, 0, sizeof(*P));
    P->scheme = o->scheme;
    P->green = o->green;
    P->d = g->d;
    P->max_iter = o->max_iter;
    P->consecutive = o->stop_consecutive;
    P->tol = o->tol;
    P->inv_ntot = 1.0 / (double)g->N;
    for (int c = 0; c < g->d; ++c) P->e[c] = e[c];
    put(P->sigma1, s1);
    const cplx one(1.0, 0.0);
    if (g->sigma64) {
        // per-voxel conductivity: MS or EM with a reference medium sigma_0 (the
        // caller's, else (min + max)/2 for MS and sqrt(min max) for EM over Re sigma)
        if (o->scheme != LSFFT_MS && o->scheme != LSFFT_EM)
            return "a per-voxel conductivity field needs the MS or EM scheme";
        cplx s0(g->sigma0_user[0], g->sigma0_user[1]);
        if (s0 == 0.0)
            s0 = o->scheme == LSFFT_MS ? cplx((g->sig_min + g->sig_max) / 2.0, 0.0)
                                       : cplx(std::sqrt(std::max(g->sig_min * g->sig_max, 0.0)), 0.0);
        if (s0 == 0.0) return "reference medium sigma_0 = 0";
        put(P->s0, s0);
        put(P->inv_s0, one / s0);
        if (o->scheme == LSFFT_MS) {
            put(P->g_b, cplx(-1.0));
            put(P->g_ce, one);
        } else {
            put(P->inv2s0, one / (2.0 * s0));
            put(P->g_a, one);
            put(P->g_b, cplx(-2.0));
            put(P->g_a0, one);
            put(P->g_ce, 2.0 * s0);
        }
        return "";
    }
    switch (o->scheme) {
        case LSFFT_MS: {   // Eq. J0-0 with sigma_0 = (sigma_1 + 1)/2 (Eq. J1)
            const cplx s0 = (s1 + one) / 2.0;
            if (s0 == 0.0) return "Moulinec-Suquet reference medium is 0 (sigma_1 = -1)";
            put(P->a_in, s1 / s0 - one);
            put(P->a_out, one / s0 - one);
            put(P->g_b, cplx(-1.0));
            put(P->g_ce, one);
            put(P->iq_in, one);
            put(P->iq_out, one);
            break;
        }
        case LSFFT_EM: {   // reference sqrt(sigma_1) (Eq. J2)
            const cplx s0 = std::sqrt(s1);
            if (s0 == 0.0) return "Eyre-Milton is undefined at sigma_1 = 0";
            put(P->a_in, (s1 - s0) / (s1 + s0));
            put(P->a_out, (one - s0) / (one + s0));
            put(P->inv2s0, one / (2.0 * s0));
            put(P->g_a, one);
            put(P->g_b, cplx(-2.0));
            put(P->g_a0, one);
            put(P->g_ce, 2.0 * s0);
            put(P->iq_in, s1 + s0);
            put(P->iq_out, one + s0);
            break;
        }
        case LSFFT_MS_SUB:
        case LSFFT_EM_SUB: {
            const double al = o->alpha, be = o->beta;
            if (!(al > 0.0 && be > al && std::isfinite(be))) return "substituted schemes need 0 < alpha < beta";
            // p from Eq. J24 with p1^2 + p2^2 + p3^2 = 1; t from Eq. J3
            const double dd = be - al;
            const double p1sq = (1.0 + al) * (1.0 + be) / dd, p2sq = -(1.0 + al) / dd, p3sq = -al * (1.0 + be) / dd;
            const cplx p1(sqrt(p1sq), 0.0), p2(0.0, sqrt(-p2sq)), p3(0.0, sqrt(-p3sq));
            if (s1 + be == 0.0) return "sigma_1 = -beta maps to t = infinity";
            const cplx t = (s1 + al) * (1.0 + be) / ((s1 + be) * (1.0 + al));
            put(P->p1, p1);
            put(P->p2, p2);
            put(P->p3, p3);
            put(P->tm1p1, (t - one) * p1);
            if (o->scheme == LSFFT_MS_SUB) {   // Eq. J42a, reference (t + 1)/2
                const cplx s0 = (t + one) / 2.0;
                if (s0 == 0.0) return "MS in H'' reference medium is 0 (t = -1)";
                put(P->k1, (t - one) * p1 / s0);
                put(P->k2, (one - s0) / s0);
                put(P->k3, (t - one) * p2 / s0);
                put(P->g_b, cplx(-1.0));
                put(P->g_ce, one);
                put(P->iq_in, one);
                put(P->iq_out, one);
            } else {                           // Eq. J43, reference sqrt(t)
                const cplx rt = std::sqrt(t);
                if (rt == 0.0) return "sigma_1 = -alpha maps to t = 0";
                put(P->w, (one - rt) / (one + rt));
                put(P->inv2s0, one / (2.0 * rt));
                put(P->g_a, one);
                put(P->g_b, cplx(-2.0));
                put(P->g_a0, one);
                put(P->g_ce, 2.0 * rt);
                put(P->iq_in, one + rt + (t - one) * p1 * p1);
                put(P->iq_out, one + rt);
                put(P->is_in, (t - one) * p1 * p2);
                put(P->it_in, (t - one) * p1 * p3);
            }
            break;
        }
        default:
            return "unknown scheme";
    }
    return "";
}

template <typename T>
cx<T> kc(const double (&v)[2], double scale = 1.0) {
    cx<T> r;
    r.x = (T)(v[0] * scale);
    r.y = (T)(v[1] * scale);
    return r;
}

// Scheme constants rounded to the field precision for the kernels.
template <typename T>
KConst<T> make_kconst(const SchemeParams& P) {
    KConst<T> K;
    memset(&K, 0, sizeof(K));
    K.a_in = kc<T>(P.a_in);
    K.a_out = kc<T>(P.a_out);
    K.k1 = kc<T>(P.k1);
    K.k2 = kc<T>(P.k2);
    K.k3 = kc<T>(P.k3);
    K.tm1p1 = kc<T>(P.tm1p1);
    K.p1 = kc<T>(P.p1);
    K.p2 = kc<T>(P.p2);
    K.p3 = kc<T>(P.p3);
    K.w = kc<T>(P.w);
    K.inv2s0 = kc<T>(P.inv2s0);
    K.s1 = kc<T>(P.sigma1);
    K.s0 = kc<T>(P.s0);
    K.inv_s0 = kc<T>(P.inv_s0);
    K.g_a = kc<T>(P.g_a, P.inv_ntot);
    K.g_b = kc<T>(P.g_b, P.inv_ntot);
    K.g_a0 = kc<T>(P.g_a0, P.inv_ntot);
    K.g_ce = kc<T>(P.g_ce);
    K.iq_in = kc<T>(P.iq_in);
    K.iq_out = kc<T>(P.iq_out);
    for (int c = 0; c < 3; ++c) K.e[c] = (T)P.e[c];
    K.scheme = P.scheme;
    K.green = P.green;
    K.real_coef = (P.g_a[1] == 0.0 && P.g_b[1] == 0.0 && P.g_a0[1] == 0.0 && P.g_ce[1] == 0.0) ? 1 : 0;
    return K;
}

// The packed real layout applies in 2-D when every coefficient the scheme
// multiplies real fields by is real (p_2, p_3 and what they scale are purely
// imaginary): then Q, J and E stay real and S, T purely imaginary.
bool packed_layout(const lsfft_grid* g, const SchemeParams& P) {
    if (g->d != 2) return false;
    if (g->sigma64 && !g->sig_real) return false;
    const double* re_only[] = {P.sigma1, P.a_in, P.a_out, P.k1, P.k2, P.tm1p1, P.p1, P.w, P.inv2s0,
                               P.g_a, P.g_b, P.g_a0, P.g_ce, P.iq_in, P.iq_out, P.s0, P.inv_s0};
    for (const double* v : re_only)
        if (v[1] != 0.0) return false;
    const double* im_only[] = {P.p2, P.p3, P.k3, P.is_in, P.it_in};
    for (const double* v : im_only)
        if (v[0] != 0.0) return false;
    return true;
}

template <typename T>
PassArgs<T> base_args(lsfft_grid* g, int st) {
    PassArgs<T> A;
    memset(&A, 0, sizeof(A));
    const int p = sizeof(T) == 4 ? 0 : 1;
    A.X = (cx<T>*)g->X;
    A.S = st >= 1 ? (cx<T>*)g->S : nullptr;
    A.Tf = st >= 2 ? (cx<T>*)g->T : nullptr;
    A.mask = g->mask;
    A.sigma = (g->sigma64 && g->sigma_t_prec == (int)(sizeof(T) == 8)) ? (const cx<T>*)g->sigma_t : nullptr;
    A.packed = g->packed;
    A.pdl = 1;                        // programmatic launches, dependents signalled ...
    A.pdl_early = g->N <= 128 * 128;  // ... at the kernel's start on small grids, else at exit (lsfft_pdl.cuh)
    A.k = make_kconst<T>(*g->prm_host);
    A.ctrl = g->ctrl_dev;
    A.partials = g->partials;
    for (int a = 0; a < 3; ++a) A.fd[a] = a < g->d ? (const cx<T>*)g->fd[a][p] : nullptr;
    A.wait_limit = g->wait_limit;
    A.extra_tx = g->inject_tx;
    A.Ntot = g->N;
    A.hp = half_pitch(g->n[0]);
    A.Nh = (g->N / g->n[0]) * A.hp;
    for (int a = 0; a < 3; ++a) A.n[a] = (int)g->n[a];
    return A;
}

template <typename T>
cudaError_t launch_row(lsfft_grid* g, int st, int mode, cx<T>* Eout) {
    PassArgs<T> A = base_args<T>(g, st);
    A.Eout = Eout;
    A.tw = sizeof(T) == 8 ? (const cx<T>*)g->tw[0] : nullptr;
    A.n_lines = g->N / g->n[0];
    A.mode = mode;
    A.grid_blocks = row_blocks(g, sizeof(T) == 4 ? LSFFT_FP32 : LSFFT_FP64);
    if constexpr (sizeof(T) == 4) {
        if (g->split) {   // row pairs (j, j + n_y/2); four half-spectrum planes of n_y/2 rows
            A.n_lines = g->n[1] / 2;
            A.Nh = A.n_lines * A.hp;
            return split_row_dispatch(g->logn[0], OP_LAUNCH, &A, g->stream, nullptr);
        }
    }
    if (g->d == 2) return row_dispatch<T, 2>(g->logn[0], OP_LAUNCH, &A, g->stream, nullptr);
    return row_dispatch<T, 3>(g->logn[0], OP_LAUNCH, &A, g->stream, nullptr);
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link-time
// dependence on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// TMA view of the two planes of a 2-D strided pass for the cluster kernel:
// 8-byte elements; dimensions (x element within the row pitch, row residue
// q < CL, inner row block j0 < 256, outer row block j1, plane), so that one box
// {W columns, 1, 256, M/256, 1} is the rows q + CL j of W adjacent columns.
template <typename T>
cudaError_t encode_cluster_map(PassArgs<T>* A, int ny, int W, int CL) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t cs = sizeof(cx<T>), epc = sizeof(cx<T>) / 8;
    const int M = ny / CL;
    if (M % 256 != 0) return cudaErrorInvalidValue;
    const cuuint64_t row = (cuuint64_t)A->ls * cs;
    cuuint64_t dims[5] = {(cuuint64_t)A->ls * epc, (cuuint64_t)CL, 256, (cuuint64_t)(M / 256), 2};
    cuuint64_t strides[4] = {row, CL * row, 256 * CL * row, (cuuint64_t)A->Ntot * cs};
    cuuint32_t box[5] = {(cuuint32_t)(W * epc), 1, 256, (cuuint32_t)(M / 256), 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(&A->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, (void*)A->X, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// TMA view of an item of the plain strided pass: 8-byte elements; dimensions
// (x element of the line starts of a slab, inner line position j0 < 256, outer
// line position j1, slab, plane), so that one box {COLS values, BJ0, BJ1, 1, d}
// is every line of one item.
template <typename T>
cudaError_t encode_col_map(PassArgs<T>* A, int N, int cols, int d) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t cs = sizeof(cx<T>), epc = sizeof(cx<T>) / 8;
    const int bj0 = N < 256 ? N : 256, bj1 = N / bj0;
    const int64_t groups = (A->n_inner + cols - 1) / cols;
    const cuuint64_t line = (cuuint64_t)A->ls * cs;
    const cuuint64_t slab = A->n_outer > 1 ? (cuuint64_t)A->outer_stride * cs : (cuuint64_t)bj1 * bj0 * line;
    cuuint64_t dims[5] = {(cuuint64_t)(groups * cols) * epc, (cuuint64_t)bj0, (cuuint64_t)bj1,
                          (cuuint64_t)A->n_outer, (cuuint64_t)d};
    cuuint64_t strides[4] = {line, bj0 * line, slab, (cuuint64_t)A->Ntot * cs};
    cuuint32_t box[5] = {(cuuint32_t)(cols * epc), (cuuint32_t)bj0, (cuuint32_t)bj1, 1, (cuuint32_t)d};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(&A->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, (void*)A->X, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// TMA view of the four half-spectrum planes of the split layout: 8-byte
// elements; dimensions (x element within the row pitch, row j0 < 256, row block
// j1, plane p, half h), so that one box {W columns, 256, M/256, 1, 1} is one
// plane of W adjacent columns of one half.
cudaError_t encode_split_map(PassArgs<float>* A, int M, int W) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return cudaErrorNotSupported;
    if (M % 256 != 0) return cudaErrorInvalidValue;
    const cuuint64_t row = (cuuint64_t)A->hp * 8;
    cuuint64_t dims[5] = {(cuuint64_t)A->hp, 256, (cuuint64_t)(M / 256), 2, 2};
    cuuint64_t strides[4] = {row, 256 * row, (cuuint64_t)M * row, 2 * (cuuint64_t)M * row};
    cuuint32_t box[5] = {(cuuint32_t)W, 256, (cuuint32_t)(M / 256), 1, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(&A->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, (void*)A->X, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_cols_split(lsfft_grid* g, PassArgs<float>* A) {
    const int M = (int)(g->n[1] / 2);
    Geom geo;
    split_col_dispatch(g->logn[1] - 1, OP_QUERY, nullptr, nullptr, &geo);
    A->n_inner = g->n[0] / 2 + 1;
    A->Nh = (int64_t)M * A->hp;
    A->line_axis = 1;
    A->mode = MODE_COL_GAMMA;
    const int64_t items = 2 * ((A->n_inner + geo.per_block - 1) / geo.per_block);
    A->grid_blocks = (int)persistent_blocks(g, items, geo.blocks_per_sm);
    cudaError_t e = encode_split_map(A, M, geo.per_block);
    if (e != cudaSuccess) return e;
    return split_col_dispatch(g->logn[1] - 1, OP_LAUNCH, A, g->stream, nullptr);
}

template <typename T>
cudaError_t col_launch(lsfft_grid* g, int axis, PassArgs<T>* A) {
    Geom geo;
    if (g->d == 2) col_dispatch<T, 2>(g->logn[axis], OP_QUERY, nullptr, nullptr, &geo);
    else col_dispatch<T, 3>(g->logn[axis], OP_QUERY, nullptr, nullptr, &geo);
    const int64_t items = (A->n_inner + geo.per_block - 1) / geo.per_block * A->n_outer;
    if (geo.cluster > 0) {
        cudaError_t e = encode_cluster_map<T>(A, (int)g->n[axis], geo.per_block, geo.cluster);
        if (e != cudaSuccess) return e;
        const int64_t ncl = items < geo.max_clusters ? items : (geo.max_clusters > 0 ? geo.max_clusters : 1);
        A->grid_blocks = (int)(ncl * geo.cluster);
    } else {
        A->grid_blocks = (int)persistent_blocks(g, items, geo.blocks_per_sm);
        cudaError_t e = encode_col_map<T>(A, (int)g->n[axis], geo.per_block, g->d);
        if (e != cudaSuccess) return e;
    }
    if (g->d == 2) return col_dispatch<T, 2>(g->logn[axis], OP_LAUNCH, A, g->stream, nullptr);
    return col_dispatch<T, 3>(g->logn[axis], OP_LAUNCH, A, g->stream, nullptr);
}

template <typename T>
cudaError_t launch_cols(lsfft_grid* g, int st) {
    PassArgs<T> A = base_args<T>(g, st);
    if constexpr (sizeof(T) == 4) {
        if (g->split) return launch_cols_split(g, &A);
    }
    if (g->d == 2) {
        A.tw = sizeof(T) == 8 ? (const cx<T>*)g->tw[1] : nullptr;
        A.ls = g->n[0];
        A.n_inner = g->n[0];
        if (A.packed) {   // the two half-spectrum planes, columns k_x = 0..n_x/2
            A.packed = 0;
            A.Ntot = A.Nh;
            A.ls = A.hp;
            A.n_inner = g->n[0] / 2 + 1;
        }
        A.outer_stride = 0;
        A.n_outer = 1;
        A.line_axis = 1;
        A.mode = MODE_COL_GAMMA;
        return col_launch<T>(g, 1, &A);
    }
    PassArgs<T> Y = A;
    Y.tw = sizeof(T) == 8 ? (const cx<T>*)g->tw[1] : nullptr;
    Y.ls = g->n[0];
    Y.n_inner = g->n[0];
    Y.outer_stride = g->n[0] * g->n[1];
    Y.n_outer = g->n[2];
    Y.line_axis = 1;
    Y.mode = MODE_COL_FWD;
    cudaError_t e = col_launch<T>(g, 1, &Y);
    if (e != cudaSuccess) return e;
    PassArgs<T> Z = A;
    Z.tw = sizeof(T) == 8 ? (const cx<T>*)g->tw[2] : nullptr;
    Z.ls = g->n[0] * g->n[1];
    Z.n_inner = g->n[0] * g->n[1];
    Z.outer_stride = 0;
    Z.n_outer = 1;
    Z.line_axis = 2;
    Z.mode = MODE_COL_GAMMA;
    e = col_launch<T>(g, 2, &Z);
    if (e != cudaSuccess) return e;
    Y.mode = MODE_COL_INV;
    return col_launch<T>(g, 1, &Y);
}

// One update: the row pass, then the finalize step (sums, sigma_k, stop rule)
// and the strided pass(es) side by side, joined before the next update.  The
// strided passes need only `skipB`, which the row pass sets when it finds the
// solve already done (the finalize step of this update may set `done`, after
// which this update still completes, as the stop rule intends); the finalize
// step reads the row pass's partial sums, which the next row pass overwrites,
// hence the join.  On small grids this takes the finalize (a few microseconds
// of dependent loads and FP64 scalar work) off the critical path.
template <typename T>
cudaError_t launch_iteration(lsfft_grid* g, int st, int nblocks, int row_mode) {
    cudaError_t e = launch_row<T>(g, st, row_mode, nullptr);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(g->ev_fork, g->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->fin_stream, g->ev_fork, 0);
    if (e == cudaSuccess)
        e = launch_finalize(g->partials, nblocks, 4 * g->d + 1, *g->prm_host, g->ctrl_dev, g->hist, 0, 1,
                            g->fin_stream);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_join, g->fin_stream);
    if (e != cudaSuccess) return e;
    e = launch_cols<T>(g, st);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(g->stream, g->ev_join, 0);
}

// The iteration graph bakes the scheme constants into its kernel parameters, so
// it is captured anew for every solve and, when a graph of the same shape is
// cached, applied to it with cudaGraphExecUpdate (cheap) instead of a fresh
// instantiation.
template <typename T>
int get_graph(lsfft_grid* g, int st, int nblocks, int check_every, cudaGraphExec_t* out) {
    const GraphKey key{(int)sizeof(T), st, check_every};
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < check_every && le == cudaSuccess; ++i) le = launch_iteration<T>(g, st, nblocks, MODE_ROW_ITER);
    cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
    if (le != cudaSuccess) {
        if (ce == cudaSuccess) cudaGraphDestroy(graph);
        return fail_cuda(le, "graph capture launch");
    }
    if (ce != cudaSuccess) return fail_cuda(ce, "cudaStreamEndCapture");
    auto it = g->graphs.find(key);
    if (it != g->graphs.end()) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(it->second, graph, &info) == cudaSuccess) {
            cudaGraphDestroy(graph);
            *out = it->second;
            return LSFFT_OK;
        }
        cudaGetLastError();
        cudaGraphExecDestroy(it->second);
        g->graphs.erase(it);
    }
    cudaGraphExec_t exec;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail_cuda(ie, "cudaGraphInstantiate");
    g->graphs[key] = exec;
    *out = exec;
    return LSFFT_OK;
}

template <typename T>
int ensure_prepared(lsfft_grid* g) {
    if (!g->prepared[sizeof(T) == 8]) {
        int rc = prepare_kernels<T>(g);
        if (rc != LSFFT_OK) return rc;
        g->prepared[sizeof(T) == 8] = true;
    }
    return LSFFT_OK;
}

// The per-voxel conductivity in the precision of the solve (converted once).
template <typename T>
int prepare_sigma(lsfft_grid* g) {
    if (!g->sigma64 || g->sigma_t_prec == (int)(sizeof(T) == 8)) return LSFFT_OK;
    CK(cudaStreamSynchronize(g->stream));
    cudaFree(g->sigma_t);
    g->sigma_t = nullptr;
    g->sigma_t_prec = -1;
    CK(cudaMalloc(&g->sigma_t, (size_t)g->N * sizeof(cx<T>)));
    CK(launch_convert_field<T>((cx<T>*)g->sigma_t, g->sigma64, g->N, g->sm_count, g->stream));
    g->sigma_t_prec = (int)(sizeof(T) == 8);
    return LSFFT_OK;
}

// Upload the constants, write the initial state and run the first update.
template <typename T>
int start_solve(lsfft_grid* g, int st) {
    int rc0 = ensure_prepared<T>(g);
    if (rc0 != LSFFT_OK) return rc0;
    const int nblocks = row_blocks(g, sizeof(T) == 4 ? LSFFT_FP32 : LSFFT_FP64);
    rc0 = prepare_sigma<T>(g);
    if (rc0 != LSFFT_OK) return rc0;
    CK(cudaMemsetAsync(g->ctrl_dev, 0, sizeof(Ctrl), g->stream));
    CK(cudaEventRecord(g->ev0, g->stream));
    if (g->packed) {   // padding columns of the half-spectrum planes: defined, never read back
        const int64_t hp = half_pitch(g->n[0]), c0 = g->n[0] / 2 + 1;
        CK(cudaMemset2DAsync((cx<T>*)g->X + c0, hp * sizeof(cx<T>), 0, (hp - c0) * sizeof(cx<T>),
                             2 * (g->N / g->n[0]), g->stream));
    }
    CK(launch_init<T>((cx<T>*)g->X, st >= 1 ? (cx<T>*)g->S : nullptr, st >= 2 ? (cx<T>*)g->T : nullptr, g->mask,
                      *g->prm_host, g->N, g->d, g->packed,
                      g->sigma64 ? (const cx<T>*)g->sigma_t : nullptr, g->sm_count, g->stream));
    CK(launch_iteration<T>(g, st, nblocks, MODE_ROW_FIRST));
    return LSFFT_OK;
}

// Drop a solve that failed: wait for its work and release its output buffer.
void abandon_solve(lsfft_grid* g) {
    sync_grid(g);
    cudaGetLastError();
    big_free(g->cur_E);
    g->cur_E = nullptr;
    g->phase = 0;
    g->phase_finish = false;
}

// A solve is a small state machine so that lsfft_solve_batch can keep one
// solve in flight per grid without blocking: begin_solve enqueues the start and
// the first stop check; poll_solve advances on completed events (another graph
// chunk, or the output pass once the device reported `done`) and fills the
// result when the output has landed.
template <typename T>
int begin_solve(lsfft_grid* g, const lsfft_opts* o, int st, lsfft_result* res) {
    int rc = ensure_prepared<T>(g);   // shared-memory limits must be set before capture
    if (rc != LSFFT_OK) return rc;
    rc = prepare_sigma<T>(g);         // the captured kernels point at the converted field
    if (rc != LSFFT_OK) return rc;
    const int nblocks = row_blocks(g, sizeof(T) == 4 ? LSFFT_FP32 : LSFFT_FP64);
    rc = get_graph<T>(g, st, nblocks, o->check_every, &g->cur_exec);
    if (rc != LSFFT_OK) return rc;
    rc = start_solve<T>(g, st);
    if (rc != LSFFT_OK) return rc;
    if (g->hist_host_cap < g->hist_cap) {
        if (g->hist_host) cudaFreeHost(g->hist_host);
        g->hist_host = nullptr;
        g->hist_host_cap = 0;
        CK(cudaMallocHost(&g->hist_host, sizeof(double) * HIST_STRIDE * g->hist_cap));
        g->hist_host_cap = g->hist_cap;
        CK(cudaHostGetDevicePointer((void**)&g->hist_host_dev, g->hist_host, 0));
    }
    // Every finalize either sets `done` or advances the iteration count, so at
    // most max_iter / check_every + 1 graph launches are needed; the bound only
    // guards against kernels that silently did not run.
    g->cur_max_launches = (int64_t)o->max_iter / o->check_every + 2;
    g->cur_launches = 0;
    g->cur_per_iter = g->d == 2 ? 3 : 5;      // row pass, finalize, strided pass(es)
    g->cur_kernels = 2 + g->cur_per_iter;     // init + first update + control block readback
    g->cur_check_every = o->check_every;
    g->cur_st = st;
    g->cur_nblocks = nblocks;
    g->cur_E = nullptr;
    g->cur_res = res;
    CK(launch_copy_words(g->ctrl_host_dev, g->ctrl_dev, sizeof(Ctrl), g->stream));
    CK(cudaEventRecord(g->ev_check, g->stream));
    g->phase = 1;
    return LSFFT_OK;
}

// Returns 0 while the solve is in flight, 1 once the result is filled, or an
// error status (the solve is then abandoned).
template <typename T>
int poll_solve(lsfft_grid* g) {
    const cudaError_t q = cudaEventQuery(g->ev_check);
    if (q == cudaErrorNotReady) return 0;
    g->phase = 0;
    if (q != cudaSuccess) return fail_cuda(q, "solve");
    lsfft_result* res = g->cur_res;
    if (g->phase_finish) {
        g->phase_finish = false;
        const Ctrl& C = *g->ctrl_host;
        if (C.fault) {
            g_last_error = "a bounded wait for a TMA transfer gave up on the device; the solve is invalid";
            return LSFFT_ECUDA;
        }
        res->E_device = g->cur_E;
        g->cur_E = nullptr;
        res->iters = C.iter;
        res->status = C.status;
        res->hist_len = C.iter + 1;
        res->sigma_star.re = C.sigma[0];
        res->sigma_star.im = C.sigma[1];
        for (int c = 0; c < g->d; ++c) {
            res->mean_E[c].re = C.meanE[c][0];
            res->mean_E[c].im = C.meanE[c][1];
            res->mean_J[c].re = C.meanJ[c][0];
            res->mean_J[c].im = C.meanJ[c][1];
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        res->solve_ms = ms;
        res->kernel_launches = g->cur_kernels;
        res->packed = g->packed ? (g->split ? 2 : 1) : 0;
        const int L = res->hist_len;
        res->hist_sigma_re = (double*)malloc(sizeof(double) * L);
        res->hist_sigma_im = (double*)malloc(sizeof(double) * L);
        res->hist_rel_change = (double*)malloc(sizeof(double) * L);
        res->hist_field_norm = (double*)malloc(sizeof(double) * L);
        if (!res->hist_sigma_re || !res->hist_sigma_im || !res->hist_rel_change || !res->hist_field_norm)
            return LSFFT_ENOMEM;
        const double* h = g->hist_host;
        for (int k = 0; k < L; ++k) {
            res->hist_sigma_re[k] = h[HIST_STRIDE * k + 0];
            res->hist_sigma_im[k] = h[HIST_STRIDE * k + 1];
            res->hist_rel_change[k] = h[HIST_STRIDE * k + 2];
            res->hist_field_norm[k] = h[HIST_STRIDE * k + 3];
        }
        return 1;
    }
    if (g->ctrl_host->done) {
        // output pass: E of the last iterate, its sigma_* and averages, history
        g->cur_kernels += 4;   // output row pass, finalize, two readbacks
        const size_t ebytes = (size_t)g->d * g->N * sizeof(cx<T>);
        CK(big_alloc(&g->cur_E, ebytes, g->stream));
        CK(launch_row<T>(g, g->cur_st, MODE_ROW_OUTPUT, (cx<T>*)g->cur_E));
        CK(launch_finalize(g->partials, g->cur_nblocks, 4 * g->d + 1, *g->prm_host, g->ctrl_dev, g->hist, 1, 1,
                           g->stream));
        CK(cudaEventRecord(g->ev1, g->stream));
        CK(launch_copy_words(g->ctrl_host_dev, g->ctrl_dev, sizeof(Ctrl), g->stream));
        const int L = g->ctrl_host->iter + 1;
        CK(launch_copy_words(g->hist_host_dev, g->hist, sizeof(double) * HIST_STRIDE * L, g->stream));
        CK(cudaEventRecord(g->ev_check, g->stream));
        g->phase_finish = true;
        g->phase = 1;
        return 0;
    }
    if (g->cur_launches++ > g->cur_max_launches) {
        g_last_error = "iteration control block never reported completion";
        return LSFFT_ECUDA;
    }
    CK(cudaGraphLaunch(g->cur_exec, g->stream));
    g->cur_kernels += (int64_t)g->cur_per_iter * g->cur_check_every + 1;
    CK(launch_copy_words(g->ctrl_host_dev, g->ctrl_dev, sizeof(Ctrl), g->stream));
    CK(cudaEventRecord(g->ev_check, g->stream));
    g->phase = 1;
    return 0;
}

template <typename T>
int run_solve(lsfft_grid* g, const lsfft_opts* o, int st, lsfft_result* res) {
    int rc = begin_solve<T>(g, o, st, res);
    while (rc == LSFFT_OK) {
        const int p = poll_solve<T>(g);
        if (p == 1) return LSFFT_OK;
        if (p != 0) {
            rc = p;
            break;
        }
        cudaEventSynchronize(g->ev_check);
    }
    abandon_solve(g);
    return rc;
}

}  // namespace

extern "C" {

const char* lsfft_version(void) { return LSFFT_VERSION_STRING; }
const char* lsfft_last_error(void) { return g_last_error.c_str(); }

const char* lsfft_strerror(int status) {
    switch (status) {
        case LSFFT_OK: return "ok";
        case LSFFT_EINVAL: return "invalid argument";
        case LSFFT_ENOMEM: return "out of memory";
        case LSFFT_ENOTCONV: return "not converged within max_iter";
        case LSFFT_EDIVERGED: return "iteration diverged";
        case LSFFT_ECUDA: return "CUDA error";
        default: return "unknown status";
    }
}

int lsfft_create_grid(int d, const int64_t n[3], const uint8_t* phase_mask_host, void* cuda_stream, lsfft_grid** out) {
    return create_common(d, n, phase_mask_host, false, cuda_stream, out);
}

int lsfft_create_grid_device(int d, const int64_t n[3], const uint8_t* phase_mask_device, void* cuda_stream,
                             lsfft_grid** out) {
    return create_common(d, n, phase_mask_device, true, cuda_stream, out);
}

void lsfft_destroy_grid(lsfft_grid* g) {
    if (!g) return;
    sync_grid(g);
    clear_graphs(g);
    cudaFree(g->mask);
    big_free(g->X);
    big_free(g->S);
    big_free(g->T);
    cudaFree(g->partials);
    cudaFree(g->hist);
    cudaFree(g->ctrl_dev);
    delete g->prm_host;
    if (g->ctrl_host) cudaFreeHost(g->ctrl_host);
    for (int a = 0; a < 3; ++a) {
        cudaFree(g->tw[a]);
        cudaFree(g->fd[a][0]);
        cudaFree(g->fd[a][1]);
    }
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->ev_check) cudaEventDestroy(g->ev_check);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->fin_stream) cudaStreamDestroy(g->fin_stream);
    if (g->hist_host) cudaFreeHost(g->hist_host);
    big_free(g->cur_E);
    cudaFree(g->sigma64);
    cudaFree(g->sigma_t);
    if (g->own_stream) cudaStreamDestroy(g->stream);
    delete g;
}

void lsfft_default_opts(lsfft_opts* o) {
    if (!o) return;
    o->scheme = LSFFT_MS;
    o->precision = LSFFT_FP32;
    o->green = LSFFT_GREEN_TRIG;
    o->max_iter = 1000;
    o->stop_consecutive = 3;
    o->check_every = 8;
    o->tol = 1e-6;
    o->alpha = 0.0;
    o->beta = 0.0;
}

}  // extern "C"

namespace {
// Shared argument checks and set-up of lsfft_solve and lsfft_prepare.
int check_and_setup(lsfft_grid* g, lsfft_c128 sigma1, const double* e, const lsfft_opts* o, int* st_out) {
    if (!g || !e || !o) {
        g_last_error = "null argument";
        return LSFFT_EINVAL;
    }
    if (o->scheme < 0 || o->scheme > 3 || (o->precision != 0 && o->precision != 1) || (o->green != 0 && o->green != 1) ||
        o->max_iter < 1 || o->stop_consecutive < 1 || o->check_every < 1 || !(o->tol >= 0.0) || !std::isfinite(o->tol)) {
        g_last_error = "option out of range";
        return LSFFT_EINVAL;
    }
    const cplx s1(sigma1.re, sigma1.im);
    if (!finite_c(s1)) {
        g_last_error = "sigma_1 must be finite";
        return LSFFT_EINVAL;
    }
    double e2 = 0.0;
    for (int c = 0; c < g->d; ++c) {
        if (!std::isfinite(e[c])) {
            g_last_error = "e must be finite";
            return LSFFT_EINVAL;
        }
        e2 += e[c] * e[c];
    }
    if (e2 == 0.0) {
        g_last_error = "e must not vanish";
        return LSFFT_EINVAL;
    }
    const bool fp32 = o->precision == LSFFT_FP32;
    if (!(fp32 ? col_supported<float>(g) : col_supported<double>(g))) {
        g_last_error = "grid size not supported in this precision (FP64: x lines up to 4096 points)";
        return LSFFT_EINVAL;
    }
    std::string why = build_params(g, s1, e, o, g->prm_host);
    if (!why.empty()) {
        g_last_error = why;
        return LSFFT_EINVAL;
    }
    const int st = o->scheme == LSFFT_EM_SUB ? 2 : (o->scheme == LSFFT_MS_SUB ? 1 : 0);
    *st_out = st;
    g->packed = packed_layout(g, *g->prm_host) ? 1 : 0;
    g->split = (g->packed && o->precision == LSFFT_FP32 && split_shape(g) && !g->no_split) ? 1 : 0;
    g->bench_prec = -1;
    return ensure_workspace(g, o->precision, st, o->max_iter);
}
}  // namespace

extern "C" {

int lsfft_solve(lsfft_grid* g, lsfft_c128 sigma1, const double* e, const lsfft_opts* o, lsfft_result** out) {
    if (!out) {
        g_last_error = "null out";
        return LSFFT_EINVAL;
    }
    *out = nullptr;
    int st = 0;
    int rc = check_and_setup(g, sigma1, e, o, &st);
    if (rc != LSFFT_OK) return rc;
    const bool fp32 = o->precision == LSFFT_FP32;
    lsfft_result* res = (lsfft_result*)calloc(1, sizeof(lsfft_result));
    if (!res) return LSFFT_ENOMEM;
    res->precision = o->precision;
    res->sigma1 = sigma1;
    res->d = g->d;
    for (int a = 0; a < 3; ++a) res->n[a] = a < g->d ? g->n[a] : 1;
    rc = fp32 ? run_solve<float>(g, o, st, res) : run_solve<double>(g, o, st, res);
    if (rc != LSFFT_OK) {
        lsfft_free_result(res);
        return rc;
    }
    *out = res;
    return res->status == ST_OK ? LSFFT_OK : res->status;
}

int lsfft_copy_field(const lsfft_result* res, void* dst, int dst_on_device) {
    if (!res || !dst || !res->E_device) {
        g_last_error = "null argument";
        return LSFFT_EINVAL;
    }
    size_t N = 1;
    for (int a = 0; a < res->d; ++a) N *= (size_t)res->n[a];
    const size_t bytes = (size_t)res->d * N * (res->precision == LSFFT_FP32 ? 8 : 16);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(dst, res->E_device, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return LSFFT_OK;
}

int lsfft_copy_field_async(const lsfft_result* res, void* dst, int dst_on_device, void* cuda_stream) {
    if (!res || !dst || !res->E_device) {
        g_last_error = "null argument";
        return LSFFT_EINVAL;
    }
    size_t N = 1;
    for (int a = 0; a < res->d; ++a) N *= (size_t)res->n[a];
    const size_t bytes = (size_t)res->d * N * (res->precision == LSFFT_FP32 ? 8 : 16);
    CK(cudaMemcpyAsync(dst, res->E_device, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       (cudaStream_t)cuda_stream));
    return LSFFT_OK;
}

int lsfft_prepare(lsfft_grid* g, lsfft_c128 sigma1, const double* e, const lsfft_opts* o) {
    int st = 0;
    int rc = check_and_setup(g, sigma1, e, o, &st);
    if (rc != LSFFT_OK) return rc;
    rc = o->precision == LSFFT_FP32 ? start_solve<float>(g, st) : start_solve<double>(g, st);
    if (rc != LSFFT_OK) return rc;
    CK(cudaStreamSynchronize(g->stream));
    g->bench_prec = o->precision;
    g->bench_st = st;
    return LSFFT_OK;
}

int lsfft_launch_passes(lsfft_grid* g, int kind, int count) {
    if (!g || kind < 0 || kind > 2 || count < 0 || g->bench_prec < 0) {
        g_last_error = "lsfft_launch_passes: bad kind/count or no prepared state";
        return LSFFT_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        cudaError_t e = cudaSuccess;
        if (g->bench_prec == LSFFT_FP32) {
            if (kind != 1) e = launch_row<float>(g, g->bench_st, MODE_ROW_ITER, nullptr);
            if (e == cudaSuccess && kind != 0) e = launch_cols<float>(g, g->bench_st);
        } else {
            if (kind != 1) e = launch_row<double>(g, g->bench_st, MODE_ROW_ITER, nullptr);
            if (e == cudaSuccess && kind != 0) e = launch_cols<double>(g, g->bench_st);
        }
        if (e != cudaSuccess) return fail_cuda(e, "lsfft_launch_passes");
    }
    return LSFFT_OK;
}

int lsfft_fma_peak(int paired, int reps, double* tflops) {
    if (!tflops || reps < 1) {
        g_last_error = "lsfft_fma_peak: null output or reps < 1";
        return LSFFT_EINVAL;
    }
    const cudaError_t e = measure_fma_peak(paired ? 1 : 0, reps, tflops);
    if (e != cudaSuccess) return fail_cuda(e, "lsfft_fma_peak");
    return LSFFT_OK;
}

void lsfft_free_result(lsfft_result* res) {
    if (!res) return;
    big_free(res->E_device);
    free(res->hist_sigma_re);
    free(res->hist_sigma_im);
    free(res->hist_rel_change);
    free(res->hist_field_norm);
    free(res);
}

// ---------------------------------------------------------------------------
// Lanczos estimate of the pole interval (section "Estimating the parameters
// alpha and beta").  The poles of sigma_*(sigma_1) are 1 - 1/m_n, m_n the
// eigenvalues of chi Gamma_1 chi weighted by |u_n^H chi e|^2; Lanczos from
// chi e builds the Jacobi matrix of that spectral measure, whose eigenvalues
// (Gauss nodes) and squared first eigenvector components give the weights.
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

// Eigenvalues of the symmetric tridiagonal matrix (a diagonal, b off-diagonal)
// and the first component of each normalised eigenvector, by the implicit QL
// iteration with Wilkinson-type shifts.  Returns false if an eigenvalue needs
// more than 60 sweeps.
bool tridiag_eig(std::vector<double>& a, std::vector<double> b, std::vector<double>& first) {
    const int m = (int)a.size();
    b.resize(m, 0.0);
    first.assign(m, 0.0);
    first[0] = 1.0;   // row 0 of the accumulated rotation
    for (int l = 0; l < m; ++l) {
        int sweeps = 0;
        for (;;) {
            int k = l;
            for (; k < m - 1; ++k) {
                const double scale = std::fabs(a[k]) + std::fabs(a[k + 1]);
                if (std::fabs(b[k]) <= 1e-15 * scale) break;
            }
            if (k == l) break;
            if (++sweeps > 60) return false;
            // shift from the trailing 2x2 block at l
            double g = (a[l + 1] - a[l]) / (2.0 * b[l]);
            double r = std::hypot(g, 1.0);
            g = a[k] - a[l] + b[l] / (g + (g >= 0 ? r : -r));
            double sn = 1.0, cs = 1.0, p = 0.0;
            bool deflated = false;
            for (int i = k - 1; i >= l; --i) {
                const double f = sn * b[i], h = cs * b[i];
                r = std::hypot(f, g);
                b[i + 1] = r;
                if (r == 0.0) {
                    a[i + 1] -= p;
                    b[k] = 0.0;
                    deflated = true;
                    break;
                }
                sn = f / r;
                cs = g / r;
                g = a[i + 1] - p;
                r = (a[i] - g) * sn + 2.0 * cs * h;
                p = sn * r;
                a[i + 1] = g + p;
                g = cs * r - h;
                const double z = first[i + 1];
                first[i + 1] = sn * first[i] + cs * z;
                first[i] = cs * first[i] - sn * z;
            }
            if (deflated) continue;
            a[l] -= p;
            b[l] = g;
            b[k] = 0.0;
        }
    }
    return true;
}

template <typename T>
int run_lanczos(lsfft_grid* g, const double* evec, int steps, std::vector<double>& al, std::vector<double>& be,
                double* norm0_out) {
    int rc = ensure_prepared<T>(g);
    if (rc != LSFFT_OK) return rc;
    const int64_t L = (int64_t)g->d * g->N;
    const size_t bytes = (size_t)L * sizeof(cx<T>);
    const int blocks = g->sm_count * 4;
    cx<T>*V[3] = {nullptr, nullptr, nullptr};
    double* part = nullptr;
    double* scal = nullptr;
    double* host = nullptr;
    auto cleanup = [&]() {
        for (auto& v : V) cudaFree(v);
        cudaFree(part);
        cudaFree(scal);
        if (host) cudaFreeHost(host);
    };
    cudaError_t e0 = cudaSuccess;
    for (auto& v : V)
        if (e0 == cudaSuccess) e0 = cudaMalloc(&v, bytes);
    if (e0 == cudaSuccess) e0 = cudaMalloc(&part, sizeof(double) * blocks);
    if (e0 == cudaSuccess) e0 = cudaMalloc(&scal, sizeof(double) * 2);
    if (e0 == cudaSuccess) e0 = cudaMallocHost(&host, sizeof(double) * 2);
    if (e0 != cudaSuccess) {
        cleanup();
        return fail_cuda(e0, "lanczos buffers");
    }
    cx<T>* vprev = V[0];
    cx<T>* v = V[1];
    cx<T>* w = V[2];
    auto read_scalar = [&](double* out) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(host, scal, sizeof(double), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        *out = host[0];
        return e;
    };
    cudaError_t e = cudaMemsetAsync(g->ctrl_dev, 0, sizeof(Ctrl), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(vprev, 0, bytes, g->stream);
    if (e == cudaSuccess) e = lanczos_init<T>(v, g->mask, g->N, g->d, evec, blocks, part, scal, g->stream);
    double nrm2 = 0.0;
    if (e == cudaSuccess) e = read_scalar(&nrm2);
    if (e == cudaSuccess && nrm2 <= 0.0) {
        cleanup();
        g_last_error = "chi e vanishes (no inclusion voxel or e = 0)";
        return LSFFT_EINVAL;
    }
    const double nrm0 = std::sqrt(nrm2);
    *norm0_out = nrm0;
    if (e == cudaSuccess) e = lanczos_scale<T>(v, v, 1.0 / nrm0, L, blocks, g->stream);
    double beta_prev = 0.0;
    for (int j = 0; j < steps && e == cudaSuccess; ++j) {
        // w = chi Gamma_1 chi v: row pass (chi, forward x-DFT), strided pass(es)
        // (forward, Gamma, inverse), row pass (inverse x-DFT, chi) into w
        e = cudaMemcpyAsync(g->X, v, bytes, cudaMemcpyDeviceToDevice, g->stream);
        if (e == cudaSuccess) e = launch_row<T>(g, 0, MODE_ROW_FIRST, nullptr);
        if (e == cudaSuccess) e = launch_cols<T>(g, 0);
        if (e == cudaSuccess) e = launch_row<T>(g, 0, MODE_ROW_OUTPUT, w);
        double a_j = 0.0, b2 = 0.0;
        if (e == cudaSuccess) e = lanczos_dot<T>(v, w, L, blocks, part, scal, g->stream);
        if (e == cudaSuccess) e = read_scalar(&a_j);
        if (e == cudaSuccess) e = lanczos_axpy_norm<T>(w, v, vprev, a_j, beta_prev, L, blocks, part, scal, g->stream);
        if (e == cudaSuccess) e = read_scalar(&b2);
        if (e != cudaSuccess) break;
        al.push_back(a_j);
        const double b_j = std::sqrt(std::max(b2, 0.0));
        if (j == steps - 1 || b_j <= 1e-10) break;   // last step, or an invariant subspace was reached
        be.push_back(b_j);
        // rotate: vprev <- v, v <- w / b_j
        cx<T>* old_prev = vprev;
        vprev = v;
        e = lanczos_scale<T>(old_prev, w, 1.0 / b_j, L, blocks, g->stream);
        v = old_prev;
        beta_prev = b_j;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cleanup();
    if (e != cudaSuccess) return fail_cuda(e, "lanczos");
    be.resize(al.size() > 0 ? al.size() - 1 : 0);
    return LSFFT_OK;
}

}  // namespace

extern "C" {

int lsfft_tridiag_gauss(int m, const double* a, const double* b, double* nodes, double* first2) {
    if (m < 1 || !a || (m > 1 && !b) || !nodes || !first2) {
        g_last_error = "lsfft_tridiag_gauss: bad arguments";
        return LSFFT_EINVAL;
    }
    std::vector<double> d(a, a + m), off(m > 1 ? b : a, m > 1 ? b + (m - 1) : a), z;
    if (!tridiag_eig(d, off, z)) {
        g_last_error = "lsfft_tridiag_gauss: QL iteration did not converge";
        return LSFFT_ENOTCONV;
    }
    for (int i = 0; i < m; ++i) {
        nodes[i] = d[i];
        first2[i] = z[i] * z[i];
    }
    return LSFFT_OK;
}

int lsfft_lanczos_hull(lsfft_grid* g, const double* e, int green, int precision, int steps, double cutoff,
                       double* alpha, double* beta, double* nodes, double* weights, int* n_nodes) {
    if (!g || !e || !alpha || !beta || (green != 0 && green != 1) || (precision != 0 && precision != 1) ||
        steps < 2 || steps > 4096 || !(cutoff >= 0.0 && cutoff < 1.0)) {
        g_last_error = "lsfft_lanczos_hull: bad arguments";
        return LSFFT_EINVAL;
    }
    double e2 = 0.0;
    for (int c = 0; c < g->d; ++c) e2 += e[c] * e[c];
    if (!(e2 > 0.0) || !std::isfinite(e2)) {
        g_last_error = "e must be finite and non-zero";
        return LSFFT_EINVAL;
    }
    const bool fp32 = precision == LSFFT_FP32;
    if (!(fp32 ? col_supported<float>(g) : col_supported<double>(g))) {
        g_last_error = "grid size not supported in this precision";
        return LSFFT_EINVAL;
    }
    // operator chi Gamma_1 chi: pointwise chi, Gamma step out = Gamma(k) v (k != 0), 0 at k = 0
    SchemeParams* P = g->prm_host;
    memset(P, 0, sizeof(*P));
    P->scheme = SCHEME_MATVEC;
    P->green = green;
    P->d = g->d;
    P->max_iter = 1;
    P->consecutive = 1;
    P->inv_ntot = 1.0 / (double)g->N;
    for (int c = 0; c < g->d; ++c) P->e[c] = e[c];
    P->g_b[0] = 1.0;
    g->packed = 0;
    g->split = 0;
    g->bench_prec = -1;
    int rc = ensure_workspace(g, precision, 0, 1);
    if (rc != LSFFT_OK) return rc;
    std::vector<double> al, be;
    double nrm0 = 0.0;
    rc = fp32 ? run_lanczos<float>(g, e, steps, al, be, &nrm0) : run_lanczos<double>(g, e, steps, al, be, &nrm0);
    if (rc != LSFFT_OK) return rc;
    const int m = (int)al.size();
    std::vector<double> th(m), w2(m);
    rc = lsfft_tridiag_gauss(m, al.data(), be.data(), th.data(), w2.data());
    if (rc != LSFFT_OK) return rc;
    double wsum = 0.0;
    for (int i = 0; i < m; ++i) {
        w2[i] *= nrm0 * nrm0;
        wsum += w2[i];
    }
    double tmin = INFINITY, tmax = -INFINITY;
    for (int i = 0; i < m; ++i) {
        if (w2[i] > cutoff * wsum && th[i] > 1e-14) {
            tmin = std::min(tmin, th[i]);
            tmax = std::max(tmax, th[i]);
        }
    }
    if (!(tmax > 0.0)) {
        g_last_error = "no weighted Lanczos node above the cutoff";
        return LSFFT_ENOTCONV;
    }
    *alpha = 1.0 / tmax - 1.0;
    *beta = 1.0 / tmin - 1.0;
    if (n_nodes) *n_nodes = m;
    for (int i = 0; i < m; ++i) {
        if (nodes) nodes[i] = th[i];
        if (weights) weights[i] = w2[i];
    }
    return LSFFT_OK;
}

int lsfft_set_column_split(lsfft_grid* g, int split) {
    if (!g) {
        g_last_error = "lsfft_set_column_split: null grid";
        return LSFFT_EINVAL;
    }
    sync_grid(g);
    clear_graphs(g);
    g->no_split = split == 0;
    g->bench_prec = -1;
    return LSFFT_OK;
}

int lsfft_autotune(lsfft_grid* g, lsfft_c128 sigma1, const double* e, const lsfft_opts* opts, int iters,
                   lsfft_tuning* out) {
    if (!g || !e || !opts || !out || iters < 1 || iters > 100000) {
        g_last_error = "lsfft_autotune: bad arguments";
        return LSFFT_EINVAL;
    }
    const bool both_layouts = split_shape(g) && opts->precision == LSFFT_FP32;
    const bool saved_no_split = g->no_split;
    const int ces[] = {4, 8, 16, 32, 64};
    double best = INFINITY;
    int best_ce = opts->check_every, best_split = saved_no_split ? 0 : 1, count = 0;
    for (int split = 1; split >= 0; --split) {
        if (!both_layouts && split == 0) break;
        lsfft_set_column_split(g, split);
        for (int ce : ces) {
            lsfft_opts o = *opts;
            o.check_every = ce;
            o.tol = 0.0;
            o.max_iter = iters;
            double ms = INFINITY;
            for (int rep = 0; rep < 2; ++rep) {   // the first run captures the graph
                lsfft_result* r = nullptr;
                const int rc = lsfft_solve(g, sigma1, e, &o, &r);
                if (!r) {
                    lsfft_set_column_split(g, saved_no_split ? 0 : 1);
                    return rc;
                }
                if (rep == 1) ms = r->solve_ms / (double)(r->iters > 0 ? r->iters : 1);
                lsfft_free_result(r);
            }
            ++count;
            if (ms < best) {
                best = ms;
                best_ce = ce;
                best_split = both_layouts ? split : (saved_no_split ? 0 : 1);
            }
        }
    }
    lsfft_set_column_split(g, best_split);
    out->check_every = best_ce;
    out->column_split = best_split;
    out->ms_per_iter = best;
    out->candidates = count;
    return LSFFT_OK;
}

int lsfft_debug_inject(lsfft_grid* g, int kind) {
    if (!g || kind < 0 || kind > 1) {
        g_last_error = "lsfft_debug_inject: null grid or unknown kind";
        return LSFFT_EINVAL;
    }
    sync_grid(g);
    clear_graphs(g);
    g->inject_tx = kind == 1 ? 16 : 0;
    g->wait_limit = kind == 1 ? 20000000LL : MBAR_WAIT_LIMIT;
    return LSFFT_OK;
}

int lsfft_set_sigma_field(lsfft_grid* g, const lsfft_c128* sigma, int on_device, lsfft_c128 sigma0) {
    if (!g) {
        g_last_error = "null grid";
        return LSFFT_EINVAL;
    }
    sync_grid(g);
    clear_graphs(g);
    cudaFree(g->sigma64);
    cudaFree(g->sigma_t);
    g->sigma64 = nullptr;
    g->sigma_t = nullptr;
    g->sigma_t_prec = -1;
    if (!sigma) return LSFFT_OK;   // back to the two-phase medium of the mask
    const size_t bytes = (size_t)g->N * sizeof(lsfft_c128);
    std::vector<lsfft_c128> h((size_t)g->N);
    if (on_device) {
        CK(cudaMemcpy(h.data(), sigma, bytes, cudaMemcpyDeviceToHost));
    } else {
        memcpy(h.data(), sigma, bytes);
    }
    double mn = INFINITY, mx = -INFINITY;
    bool real = true;
    for (const auto& v : h) {
        if (!std::isfinite(v.re) || !std::isfinite(v.im)) {
            g_last_error = "sigma field must be finite";
            return LSFFT_EINVAL;
        }
        mn = std::min(mn, v.re);
        mx = std::max(mx, v.re);
        real = real && v.im == 0.0;
    }
    CK(cudaMalloc(&g->sigma64, bytes));
    CK(cudaMemcpy(g->sigma64, h.data(), bytes, cudaMemcpyHostToDevice));
    g->sig_min = mn;
    g->sig_max = mx;
    g->sig_real = real && sigma0.im == 0.0;
    g->sigma0_user[0] = sigma0.re;
    g->sigma0_user[1] = sigma0.im;
    return LSFFT_OK;
}

}  // extern "C"

template <typename T>
static int gradient_impl(lsfft_grid* g, const lsfft_result* res, const double* e, void* grad_device,
                         lsfft_c128* dsigma1, lsfft_c128* energy) {
    const int blocks = g->sm_count * 4;
    double e2 = 0.0;
    for (int c = 0; c < g->d; ++c) e2 += e[c] * e[c];
    const cx<T>* sig = nullptr;
    if (g->sigma64) {
        if (g->sigma_t_prec != (int)(sizeof(T) == 8)) {
            g_last_error = "the conductivity field was not prepared in the result's precision";
            return LSFFT_EINVAL;
        }
        sig = (const cx<T>*)g->sigma_t;
    }
    CK(launch_gradient<T>((const cx<T>*)res->E_device, g->mask, sig, res->sigma1.re, res->sigma1.im, g->d, g->N,
                          1.0 / ((double)g->N * e2), (cx<T>*)grad_device, blocks, g->partials, g->stream));
    std::vector<double> h((size_t)blocks * 4);
    CK(cudaMemcpyAsync(h.data(), g->partials, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    double acc[4] = {0, 0, 0, 0};
    for (int b = 0; b < blocks; ++b)
        for (int v = 0; v < 4; ++v) acc[v] += h[(size_t)b * 4 + v];
    if (dsigma1) {
        dsigma1->re = acc[0] / ((double)g->N * e2);
        dsigma1->im = acc[1] / ((double)g->N * e2);
    }
    if (energy) {
        energy->re = acc[2] / ((double)g->N * e2);
        energy->im = acc[3] / ((double)g->N * e2);
    }
    return LSFFT_OK;
}

extern "C" {

int lsfft_gradient(lsfft_grid* g, const lsfft_result* res, const double* e, void* grad_device, lsfft_c128* dsigma1,
                   lsfft_c128* energy) {
    if (!g || !res || !e || !res->E_device || res->d != g->d) {
        g_last_error = "lsfft_gradient: bad arguments";
        return LSFFT_EINVAL;
    }
    for (int a = 0; a < g->d; ++a)
        if (res->n[a] != g->n[a]) {
            g_last_error = "lsfft_gradient: result and grid differ in size";
            return LSFFT_EINVAL;
        }
    if (!g->partials) {
        g_last_error = "lsfft_gradient: the grid has not solved yet";
        return LSFFT_EINVAL;
    }
    return res->precision == LSFFT_FP32 ? gradient_impl<float>(g, res, e, grad_device, dsigma1, energy)
                                        : gradient_impl<double>(g, res, e, grad_device, dsigma1, energy);
}

int lsfft_solve_batch(int njobs, const lsfft_job* jobs, lsfft_result** results, int* statuses) {
    if (njobs < 0 || (njobs > 0 && (!jobs || !results || !statuses))) {
        g_last_error = "lsfft_solve_batch: bad arguments";
        return LSFFT_EINVAL;
    }
    for (int j = 0; j < njobs; ++j) {
        results[j] = nullptr;
        statuses[j] = LSFFT_EINVAL;
        if (!jobs[j].grid) {
            g_last_error = "lsfft_solve_batch: job without grid";
            return LSFFT_EINVAL;
        }
    }
    // jobs of one grid run in order on its stream; different grids run concurrently
    std::vector<lsfft_grid*> grids;
    std::map<lsfft_grid*, std::vector<int>> queue;
    for (int j = 0; j < njobs; ++j) {
        if (!queue.count(jobs[j].grid)) grids.push_back(jobs[j].grid);
        queue[jobs[j].grid].push_back(j);
    }
    std::map<lsfft_grid*, size_t> next;
    std::map<lsfft_grid*, int> cur, cur_prec;
    for (auto* g : grids) {
        next[g] = 0;
        cur[g] = -1;
    }
    int remaining = njobs;
    while (remaining > 0) {
        bool progress = false;
        for (auto* g : grids) {
            const int j = cur[g];
            if (j < 0) {
                if (next[g] >= queue[g].size()) continue;
                const int k = queue[g][next[g]++];
                progress = true;
                const lsfft_job& J = jobs[k];
                int st = 0;
                int rc = check_and_setup(g, J.sigma1, J.e, &J.opts, &st);
                lsfft_result* res = nullptr;
                if (rc == LSFFT_OK) {
                    res = (lsfft_result*)calloc(1, sizeof(lsfft_result));
                    if (!res) rc = LSFFT_ENOMEM;
                }
                if (rc == LSFFT_OK) {
                    res->precision = J.opts.precision;
                    res->sigma1 = J.sigma1;
                    res->d = g->d;
                    for (int a = 0; a < 3; ++a) res->n[a] = a < g->d ? g->n[a] : 1;
                    rc = J.opts.precision == LSFFT_FP32 ? begin_solve<float>(g, &J.opts, st, res)
                                                        : begin_solve<double>(g, &J.opts, st, res);
                    if (rc != LSFFT_OK) {
                        abandon_solve(g);
                        lsfft_free_result(res);
                    }
                }
                if (rc != LSFFT_OK) {
                    statuses[k] = rc;
                    --remaining;
                    continue;
                }
                cur[g] = k;
                cur_prec[g] = J.opts.precision;
                continue;
            }
            const int p = cur_prec[g] == LSFFT_FP32 ? poll_solve<float>(g) : poll_solve<double>(g);
            if (p == 0) continue;
            progress = true;
            lsfft_result* res = g->cur_res;
            if (p == 1) {
                results[j] = res;
                statuses[j] = res->status == ST_OK ? LSFFT_OK : res->status;
            } else {
                abandon_solve(g);
                lsfft_free_result(res);
                statuses[j] = p;
            }
            cur[g] = -1;
            --remaining;
        }
        if (!progress) std::this_thread::yield();
    }
    return LSFFT_OK;
}

int lsfft_effective_tensor(lsfft_grid* g, lsfft_c128 sigma1, const lsfft_opts* o, lsfft_c128* out,
                           lsfft_result** results) {
    if (!g || !o || !out) {
        g_last_error = "lsfft_effective_tensor: null argument";
        return LSFFT_EINVAL;
    }
    const int d = g->d;
    lsfft_result* res[3] = {nullptr, nullptr, nullptr};
    auto release = [&]() {
        for (int a = 0; a < d; ++a) lsfft_free_result(res[a]);
    };
    // columns a of [<J>] and [<E>]: the solve with applied field e_a
    cplx Jm[3][3], Em[3][3];
    int worst = LSFFT_OK;
    for (int a = 0; a < d; ++a) {
        double e[3] = {0.0, 0.0, 0.0};
        e[a] = 1.0;
        const int rc = lsfft_solve(g, sigma1, e, o, &res[a]);
        if (!res[a]) {   // an error: nothing to assemble
            release();
            return rc;
        }
        if (rc != LSFFT_OK && worst != LSFFT_EDIVERGED) worst = rc;
        for (int i = 0; i < d; ++i) {
            Jm[i][a] = cplx(res[a]->mean_J[i].re, res[a]->mean_J[i].im);
            Em[i][a] = cplx(res[a]->mean_E[i].re, res[a]->mean_E[i].im);
        }
    }
    // S [E] = [J]  <=>  [E]^T S^T = [J]^T: solve for the rows of S by elimination
    // on [E]^T with partial pivoting, all d right-hand sides at once
    cplx A[3][3], B[3][3];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            A[i][j] = Em[j][i];
            B[i][j] = Jm[j][i];
        }
    double scale = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) scale = std::max(scale, std::abs(A[i][j]));
    for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
            if (std::abs(A[r][c]) > std::abs(A[piv][c])) piv = r;
        if (!(std::abs(A[piv][c]) > 1e-14 * scale)) {
            g_last_error = "lsfft_effective_tensor: the matrix of mean fields <E> is singular";
            if (results) {
                for (int a = 0; a < d; ++a) results[a] = nullptr;
            }
            release();
            return LSFFT_EINVAL;
        }
        for (int j = 0; j < d; ++j) {
            std::swap(A[c][j], A[piv][j]);
            std::swap(B[c][j], B[piv][j]);
        }
        for (int r = c + 1; r < d; ++r) {
            const cplx f = A[r][c] / A[c][c];
            for (int j = 0; j < d; ++j) {
                A[r][j] -= f * A[c][j];
                B[r][j] -= f * B[c][j];
            }
        }
    }
    cplx X[3][3];   // X = S^T
    for (int j = 0; j < d; ++j)
        for (int r = d - 1; r >= 0; --r) {
            cplx acc = B[r][j];
            for (int k = r + 1; k < d; ++k) acc -= A[r][k] * X[k][j];
            X[r][j] = acc / A[r][r];
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            out[i * d + j].re = X[j][i].real();
            out[i * d + j].im = X[j][i].imag();
        }
    if (results) {
        for (int a = 0; a < d; ++a) results[a] = res[a];
    } else {
        release();
    }
    return worst;
}

int lsfft_solve_sweep(int njobs, const lsfft_job* jobs, lsfft_result** results, int* statuses) {
    if (njobs < 0 || (njobs > 0 && (!jobs || !results || !statuses))) {
        g_last_error = "lsfft_solve_sweep: bad arguments";
        return LSFFT_EINVAL;
    }
    if (njobs == 0) return LSFFT_OK;
    auto pow2_in = [](int64_t v) { return v >= 128 && v <= 1024 && (v & (v - 1)) == 0; };
    for (int j = 0; j < njobs; ++j) {
        results[j] = nullptr;
        statuses[j] = LSFFT_EINVAL;
        const lsfft_job& J = jobs[j];
        lsfft_grid* g = J.grid;
        if (!g || g->d != 2 || !pow2_in(g->n[0]) || !pow2_in(g->n[1]) || g->sigma64 ||
            J.opts.precision != LSFFT_FP32 || J.opts.max_iter < 1 || J.opts.stop_consecutive < 1 ||
            !(J.opts.tol >= 0.0) || J.opts.scheme < 0 || J.opts.scheme > 3 || (J.opts.green != 0 && J.opts.green != 1)) {
            g_last_error = "lsfft_solve_sweep: every job needs a 2-D grid with n_x, n_y in {128, ..., 1024}, "
                           "a two-phase medium, FP32 fields and valid options";
            return LSFFT_EINVAL;
        }
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    static std::mutex mu;
    static int bps_dev[64] = {0};
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 0 || dev >= 64) return fail_cuda(cudaErrorInvalidDevice, "lsfft_solve_sweep");
        if (!bps_dev[dev]) CK(sweep_prepare(&bps_dev[dev]));
    }
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // descriptors (FP64 constants per job, as lsfft_solve would form them)
    std::vector<SweepJob> hj((size_t)njobs);
    std::vector<SchemeParams> prm((size_t)njobs);
    std::vector<int> hist_off((size_t)njobs), part_off((size_t)njobs);
    int64_t hist_total = 0, part_total = 0;
    for (int j = 0; j < njobs; ++j) {
        const lsfft_job& J = jobs[j];
        lsfft_grid* g = J.grid;
        std::string why = build_params(g, cplx(J.sigma1.re, J.sigma1.im), J.e, &J.opts, &prm[j]);
        if (!why.empty()) {
            g_last_error = "lsfft_solve_sweep: job " + std::to_string(j) + ": " + why;
            return LSFFT_EINVAL;
        }
        SweepJob& D = hj[j];
        memset(&D, 0, sizeof(D));
        D.k = make_kconst<float>(prm[j]);
        D.prm = prm[j];
        D.nx = (int)g->n[0];
        D.ny = (int)g->n[1];
        D.lognx = g->logn[0];
        D.logny = g->logn[1];
        D.row_items = D.ny / sweep_row_lpb(D.nx);
        D.col_items = D.nx / sweep_col_cols(D.ny);
        D.mask = g->mask;
        D.fd[0] = (const float2*)g->fd[0][0];
        D.fd[1] = (const float2*)g->fd[1][0];
        hist_off[j] = (int)hist_total;
        hist_total += (int64_t)(J.opts.max_iter + 1) * HIST_STRIDE;
        part_off[j] = (int)part_total;
        part_total += (int64_t)D.row_items * 9;
    }
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    std::vector<void*> owned;   // buffers freed at the end (the fields E stay with the results)
    std::vector<void*> fields((size_t)njobs, nullptr);
    SweepJob* djobs = nullptr;
    SweepJob* pinned = nullptr;
    SweepGlobal* dglob = nullptr;
    SweepGlobal* hglob = nullptr;
    double* dhist = nullptr;
    double* dpart = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&](bool keep_fields) {
        if (s) cudaStreamSynchronize(s);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (void* p : owned) big_free(p);
        if (!keep_fields)
            for (void* p : fields) big_free(p);
        cudaFree(djobs);
        cudaFree(dglob);
        cudaFree(dhist);
        cudaFree(dpart);
        if (pinned) cudaFreeHost(pinned);
        if (hglob) cudaFreeHost(hglob);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    };
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < njobs && e == cudaSuccess; ++j) {
        SweepJob& D = hj[j];
        const size_t fb = (size_t)2 * D.nx * D.ny * sizeof(float2);
        const int st = jobs[j].opts.scheme == LSFFT_EM_SUB ? 2 : (jobs[j].opts.scheme == LSFFT_MS_SUB ? 1 : 0);
        void* p = nullptr;
        if ((e = big_alloc(&p, fb, s)) != cudaSuccess) break;
        owned.push_back(p);
        D.X = (float2*)p;
        if (st >= 1) {
            if ((e = big_alloc(&p, fb, s)) != cudaSuccess) break;
            owned.push_back(p);
            D.S = (float2*)p;
        }
        if (st >= 2) {
            if ((e = big_alloc(&p, fb, s)) != cudaSuccess) break;
            owned.push_back(p);
            D.T = (float2*)p;
        }
        if ((e = big_alloc(&p, fb, s)) != cudaSuccess) break;
        fields[j] = p;
        D.Eout = (float2*)p;
    }
    if (e == cudaSuccess) e = cudaMalloc(&djobs, sizeof(SweepJob) * njobs);
    if (e == cudaSuccess) e = cudaMalloc(&dglob, sizeof(SweepGlobal));
    if (e == cudaSuccess) e = cudaMalloc(&dhist, sizeof(double) * hist_total);
    if (e == cudaSuccess) e = cudaMalloc(&dpart, sizeof(double) * part_total);
    if (e == cudaSuccess) e = cudaMallocHost(&pinned, sizeof(SweepJob) * njobs);
    if (e == cudaSuccess) e = cudaMallocHost(&hglob, sizeof(SweepGlobal));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup(false);
        return fail_cuda(e, "lsfft_solve_sweep buffers");
    }
    for (int j = 0; j < njobs; ++j) {
        hj[j].hist = dhist + hist_off[j];
        hj[j].partials = dpart + part_off[j];
    }
    memcpy(pinned, hj.data(), sizeof(SweepJob) * njobs);
    // the batch as one captured graph: descriptors in, counters cleared, the one
    // persistent launch, descriptors and counters back
    const int blocks = sms * std::max(1, bps_dev[dev]);
    const long long idle_limit_ns = 2000000000LL;
    const char* step = "cudaStreamBeginCapture";
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaMemcpyAsync(djobs, pinned, sizeof(SweepJob) * njobs, cudaMemcpyHostToDevice, s);
        const char* lstep = "descriptor upload";
        if (le == cudaSuccess && (le = cudaMemsetAsync(dglob, 0, sizeof(SweepGlobal), s)) != cudaSuccess)
            lstep = "counter reset";
        if (le == cudaSuccess && (le = sweep_launch(djobs, njobs, dglob, blocks, idle_limit_ns, s)) != cudaSuccess)
            lstep = "persistent launch";
        if (le == cudaSuccess &&
            (le = cudaMemcpyAsync(pinned, djobs, sizeof(SweepJob) * njobs, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            lstep = "descriptor readback";
        if (le == cudaSuccess &&
            (le = cudaMemcpyAsync(hglob, dglob, sizeof(SweepGlobal), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            lstep = "counter readback";
        step = "cudaStreamEndCapture";
        e = cudaStreamEndCapture(s, &graph);
        if (e == cudaSuccess && le != cudaSuccess) {
            e = le;
            step = lstep;
        }
    }
    if (e == cudaSuccess) {
        step = "cudaGraphInstantiate";
        e = cudaGraphInstantiate(&exec, graph, 0);
    }
    if (e == cudaSuccess) {
        // timing events outside the captured graph (an event recorded during capture
        // is not recorded when the graph runs)
        step = "cudaGraphLaunch";
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    }
    if (e == cudaSuccess) {
        step = "the persistent launch (cudaStreamSynchronize)";
        e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        cleanup(false);
        return fail_cuda(e, (std::string("lsfft_solve_sweep: ") + step).c_str());
    }
    if (hglob->error || hglob->jobs_done != njobs) {
        cleanup(false);
        g_last_error = "lsfft_solve_sweep: the persistent launch stopped early (a block found no work for two "
                       "seconds while solves remained)";
        return LSFFT_ECUDA;
    }
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
        cleanup(false);
        return fail_cuda(e, "lsfft_solve_sweep: elapsed time");
    }
    std::vector<double> hh((size_t)hist_total);
    e = cudaMemcpy(hh.data(), dhist, sizeof(double) * hist_total, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cleanup(false);
        return fail_cuda(e, "lsfft_solve_sweep history");
    }
    for (int j = 0; j < njobs; ++j) {
        const SweepJob& D = pinned[j];
        const lsfft_job& J = jobs[j];
        lsfft_result* res = (lsfft_result*)calloc(1, sizeof(lsfft_result));
        if (!res) {
            statuses[j] = LSFFT_ENOMEM;
            continue;
        }
        res->precision = LSFFT_FP32;
        res->sigma1 = J.sigma1;
        res->d = 2;
        res->n[0] = D.nx;
        res->n[1] = D.ny;
        res->n[2] = 1;
        res->iters = D.ctrl.iter;
        res->status = D.ctrl.status;
        res->sigma_star.re = D.ctrl.sigma[0];
        res->sigma_star.im = D.ctrl.sigma[1];
        for (int c = 0; c < 2; ++c) {
            res->mean_E[c].re = D.ctrl.meanE[c][0];
            res->mean_E[c].im = D.ctrl.meanE[c][1];
            res->mean_J[c].re = D.ctrl.meanJ[c][0];
            res->mean_J[c].im = D.ctrl.meanJ[c][1];
        }
        res->solve_ms = ms;             // the whole batch's device time
        res->kernel_launches = 1;       // the one persistent launch, shared by every job
        res->packed = 0;
        const int L = D.ctrl.iter + 1;
        res->hist_len = L;
        res->hist_sigma_re = (double*)malloc(sizeof(double) * L);
        res->hist_sigma_im = (double*)malloc(sizeof(double) * L);
        res->hist_rel_change = (double*)malloc(sizeof(double) * L);
        res->hist_field_norm = (double*)malloc(sizeof(double) * L);
        if (!res->hist_sigma_re || !res->hist_sigma_im || !res->hist_rel_change || !res->hist_field_norm) {
            lsfft_free_result(res);
            statuses[j] = LSFFT_ENOMEM;
            continue;
        }
        const double* h = hh.data() + hist_off[j];
        for (int k = 0; k < L; ++k) {
            res->hist_sigma_re[k] = h[HIST_STRIDE * k + 0];
            res->hist_sigma_im[k] = h[HIST_STRIDE * k + 1];
            res->hist_rel_change[k] = h[HIST_STRIDE * k + 2];
            res->hist_field_norm[k] = h[HIST_STRIDE * k + 3];
        }
        res->E_device = fields[j];
        fields[j] = nullptr;
        results[j] = res;
        statuses[j] = res->status == ST_OK ? LSFFT_OK : res->status;
    }
    cleanup(false);   // fields handed to results are no longer in `fields`
    return LSFFT_OK;
}

int lsfft_substitution_rates(lsfft_c128 sigma1, double alpha, double beta, double* rate, double* limit) {
    if (!(alpha > 0.0 && beta > alpha && std::isfinite(beta)) || !rate || !limit) {
        g_last_error = "lsfft_substitution_rates: need 0 < alpha < beta and output pointers";
        return LSFFT_EINVAL;
    }
    auto zabs = [](cplx t) {
        const cplx r = std::sqrt(t);
        return std::abs((r - 1.0) / (r + 1.0));
    };
    const cplx s1(sigma1.re, sigma1.im);
    const cplx t = (s1 + alpha) * (1.0 + beta) / ((s1 + beta) * (1.0 + alpha));   // Eq. J3
    const double t0 = alpha * (1.0 + beta) / (beta * (1.0 + alpha));              // t(0)
    const double tinf = (1.0 + beta) / (1.0 + alpha);                             // t(infinity)
    *rate = zabs(t);
    *limit = std::min(zabs(cplx(t0, 0.0)), zabs(cplx(tinf, 0.0)));
    return LSFFT_OK;
}

}  // extern "C"
