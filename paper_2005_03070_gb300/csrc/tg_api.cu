// Host side of the tg library: handles, workspaces, the solver drivers and the C ABI
// declared in include/tg.h.  Every numerical step runs in the kernels of
// tg_kernels.cuh, tg_small.cu and tg_setup.cu; the host only launches them, reads a few
// scalars per cycle and takes the restart decisions of the algorithms.
#include <algorithm>
#include <atomic>
#include <climits>
#include <memory>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "tg_idr.cuh"
#include "tg_kernels.cuh"
#include "tg_mrhs.cuh"
#include "tg_batch.cuh"
#include "tg_setup.cuh"
#include "tg_small.cuh"

namespace tg {

// ============================================================================= errors
static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

int cuda_status(cudaError_t e, const char *where) {
    set_error("%s: %s", where, cudaGetErrorString(e));
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TG_OOM : TG_CUDA_ERROR;
}

#define TG_ARG(cond, ...)                 \
    do {                                  \
        if (!(cond)) {                    \
            ::tg::set_error(__VA_ARGS__); \
            return TG_BAD_ARG;            \
        }                                 \
    } while (0)

int num_sms() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    return v;
}

int grid_for(int64_t n, int per_sm) {
    int64_t b = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * per_sm;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

static int tiles_grid(int64_t n, int per_sm) {
    int64_t b = (n + 31) / 32;
    int64_t cap = (int64_t)num_sms() * per_sm;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// ============================================================================= instrumentation
// Optional per-kernel-class timing: CUDA events around each launch (only while enabled)
// and a count of every launch.  Algorithmic bytes and float64-equivalent flops of each
// launch are recorded with it, so achieved bandwidth / arithmetic rates come out per class.
enum ProfClass {
    P_APPLY, P_DOT, P_RESIDUAL, P_BI_INIT, P_BI_V, P_BI_S, P_BI_T, P_BI_X, P_GEMV_T, P_SUM_PART, P_GEMV_N,
    P_PROJ, P_TSM, P_GRAM, P_SMALL, P_GDR_RESTART, P_SCALE, P_TRANSFER, P_SETUP, P_CONVERT, P_GRAD, P_GIVENS,
    P_NOOP, P_REORTH, P_IDR_MV, P_IDR_UPD, P_COUNT
};
static const char *kProfName[P_COUNT] = {
    "apply", "dot", "residual", "bicg_init", "bicg_v", "bicg_s", "bicg_t", "bicg_x", "gemv_t", "sum_part",
    "gemv_n", "proj_update", "tsm", "gram", "small_dense", "gmresdr_restart", "scale", "transfer", "setup",
    "convert", "kappa_grad", "givens", "bicg_noop", "reorth_pass", "idr_apply", "idr_update"};

struct ProfRec {
    int cls;
    int ev;
    double bytes, flops;
};
struct Prof {
    long long gdr_phase[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool on = false;
    std::vector<cudaEvent_t> events;
    std::vector<ProfRec> recs;
    size_t next = 0;
    long long launches = 0;
};
static Prof g_prof;

static std::mutex g_prof_mu;

static int prof_begin(cudaStream_t s) {
    if (!g_prof.on) {
        __atomic_add_fetch(&g_prof.launches, 1, __ATOMIC_RELAXED);
        return -1;
    }
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof.launches += 1;
    if (g_prof.next + 2 > g_prof.events.size()) {
        size_t add = g_prof.events.size() < 4096 ? 4096 : g_prof.events.size();
        for (size_t i = 0; i < add; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            g_prof.events.push_back(e);
        }
    }
    int ev = (int)g_prof.next;
    g_prof.next += 2;
    cudaEventRecord(g_prof.events[ev], s);
    return ev;
}
static void prof_end(int ev, int cls, double bytes, double flops, cudaStream_t s) {
    if (ev < 0) return;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    cudaEventRecord(g_prof.events[ev + 1], s);
    g_prof.recs.push_back(ProfRec{cls, ev, bytes, flops});
}
#define TG_PROF(cls, bytes, flops, ...)                                  \
    do {                                                                 \
        int _ev = ::tg::prof_begin(s);                                   \
        __VA_ARGS__;                                                     \
        ::tg::prof_end(_ev, cls, (double)(bytes), (double)(flops), s);   \
    } while (0)

// Algorithmic cost of one operator application per point: extra words read beyond the
// source and destination vectors (coefficients, links), and flops (float64 equivalent).
static void op_cost(const DevOp &A, double *extra_bytes, double *flops) {
    switch (A.kind) {
        case DK_CD2D: *extra_bytes = 0; *flops = 10; break;
        case DK_CD3D: *extra_bytes = 0; *flops = 14; break;
        case DK_VAR2D: *extra_bytes = 5 * 8; *flops = 10; break;
        case DK_U1: *extra_bytes = 4 * 16; *flops = 66; break;
        default: *extra_bytes = 9 * 16; *flops = 72; break;
    }
}

// ============================================================================= buffers
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int ensure(size_t b) {
        if (bytes >= b && p) return TG_OK;
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            return cuda_status(e, "cudaMalloc");
        }
        bytes = b;
        return TG_OK;
    }
    template <class U> U *as() const { return reinterpret_cast<U *>(p); }
};

struct PinBuf {
    void *p = nullptr;
    size_t bytes = 0;
    PinBuf() = default;
    PinBuf(const PinBuf &) = delete;
    PinBuf &operator=(const PinBuf &) = delete;
    ~PinBuf() {
        if (p) cudaFreeHost(p);
    }
    int ensure(size_t b) {
        if (bytes >= b && p) return TG_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cudaError_t e = cudaMallocHost(&p, b);
        if (e != cudaSuccess) return cuda_status(e, "cudaMallocHost");
        bytes = b;
        return TG_OK;
    }
};

enum Slot {
    S_PART, S_TICKET, S_SMALL, S_RH, S_P, S_V, S_S, S_T, S_R32, S_E32, S_R64,
    S_GV, S_GV2, S_GH, S_GH2, S_GC, S_GX, S_GD, S_GRES, S_GZ, S_GP, S_GCN, S_GTHETA, S_GWR, S_GWI,
    S_GORD, S_GERES, S_GWORK, S_GY, S_GG, S_GINFO, S_GTMP, S_GB, S_GH1, S_GHV,
    S_FV, S_FH, S_FCS, S_FSN, S_FG, S_FY, S_FSTATE, S_BC,
    S_CQ_G, S_CQ_R1, S_CQ_R1I, S_CQ_R2, S_CQ_R2I, S_GAL_RY, S_GAL_RYI, S_GAL_W, S_GYC, S_XBAK,
    S_IG, S_IU, S_IP, S_IPR, S_IPRI, S_IT, S_IINFO,
    S_AE_S, S_AE_W, S_AE_H, S_AE_WW, S_AE_HA, S_AE_Y, S_AE_U, S_AE_P, S_AE_Z, S_AE_TH, S_AE_WR, S_AE_WI,
    S_AE_ORD, S_AE_ERES, S_AE_WORK, S_AE_YW, S_AE_GW, S_AE_INFO, S_AE_DUM, S_PADX, S_PADR, S_AE_HR, S_AE_WWR, S_IP32,
    S_COUNT
};

}  // namespace tg

using namespace tg;

struct Level {
    DevOp A, AT;
    DevOp32 A32, AT32;
};

namespace tg {
// One captured coarse GMRES-DR cycle (Arnoldi extension from column j0 to m, the restart
// kernel and the x_c update), valid while the workspace generation is unchanged.
struct GdrGraph {
    const void *V = nullptr, *H = nullptr;
    int j0 = -1, m = 0, k = 0, nev = 0, transpose = 0, esz = 0;   // esz: basis element size
    double rtolev = 0;
    unsigned gen = 0;
    cudaGraphExec_t exec = nullptr;
    long long nkern = 0;
};
}  // namespace tg

struct tg_op {
    int kind = 0;
    int dim = 2;
    int N = 0, Nc = 0;
    int n = 0, nc = 0;
    bool cplx_ = false;
    double beta[3] = {0, 0, 0};
    double mass = 0;
    int interp = TG_INTERP_LINEAR;
    Level fine, coarse;
    DBuf kappa, kappa_c, coef, coef32, coefT, coefT32, ccoef, ccoef32, ccoefT, ccoefT32;
    DBuf links, pw, cst;
    DBuf ws[S_COUNT];
    PinBuf pin;
    unsigned ws_gen = 0;                 // bumped whenever a workspace buffer is (re)allocated
    std::vector<tg::GdrGraph> graphs;    // captured coarse GMRES-DR cycles
    cudaStream_t cap_stream = nullptr;   // private stream for captures (the caller's may be
                                         // the legacy stream, which cannot be captured)
    tg_op() = default;
    tg_op(const tg_op &) = delete;
    tg_op &operator=(const tg_op &) = delete;
    ~tg_op() {
        for (auto &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

struct tg_defl {
    int kk = 0;
    int n = 0;
    int proj = TG_PROJ_MINRES;
    int precision = TG_F64;
    bool cplx_ = false;
    bool transposed = false;
    DBuf Y, AY, Q, AV, R, M, info;
    DBuf W32, B1_32, B2_32;
};

namespace tg {

static int elem_size(const tg_op *op) { return op->cplx_ ? 16 : 8; }

template <class U> static U *wsp(tg_op *op, Slot s) { return op->ws[s].as<U>(); }
static int wsx(tg_op *op, Slot s, size_t bytes) {
    const void *p0 = op->ws[s].p;
    const int rc = op->ws[s].ensure(bytes);
    if (op->ws[s].p != p0) ++op->ws_gen;
    return rc;
}

// Layout of the small result area (bytes): device scalars of the solvers.  Vectors of
// coefficients hold up to kMaxCols complex entries (kMaxCols * 16 <= 8192).
struct SmallArea {
    static constexpr size_t bistate = 0;        // BiState
    static constexpr size_t dot_out = 1024;     // dot_host results
    static constexpr size_t res_out = 2048;     // true-residual norms
    static constexpr size_t idr = 4096;         // IdrState
    static constexpr size_t proj_c = 8192;      // projection coefficients c
    static constexpr size_t proj_d = 16384;     // projection coefficients d
    static constexpr size_t arn_h1 = 24576;     // Arnoldi: V^H w, first pass (and ||w||^2)
    static constexpr size_t arn_h2 = 32768;     // Arnoldi: second pass
    static constexpr size_t arn_nrm = 40960;    // ||w||^2, 1 / ||w|| (+ 32), re-orthogonalisation flag (+ 64)
    static constexpr size_t gmres_inv = 41984;  // 1 / ||r|| of a GMRES cycle
    static constexpr size_t bytes = 1 << 16;
};
static_assert(kMaxCols * 16 <= 8192, "coefficient vectors must fit their slots");

// reduction scratch: partials (sized generously), a ticket, a small result area
// The ticket is zeroed on the stream that will use it (a plain cudaMemset runs on the
// legacy stream, which streams created non-blocking do not wait for).
static int red_ready(tg_op *op, size_t part_bytes, cudaStream_t s) {
    TG_CHECK(wsx(op, S_PART, part_bytes < (4 << 20) ? (4 << 20) : part_bytes));
    if (!op->ws[S_TICKET].p) {
        TG_CHECK(wsx(op, S_TICKET, 64));
        TG_CHECK_CUDA(cudaMemsetAsync(op->ws[S_TICKET].p, 0, 64, s));
    }
    TG_CHECK(wsx(op, S_SMALL, SmallArea::bytes));
    TG_CHECK(op->pin.ensure(1 << 16));
    return TG_OK;
}

static int readback(tg_op *op, const void *dev, size_t bytes, cudaStream_t s) {
    TG_CHECK_CUDA(cudaMemcpyAsync(op->pin.p, dev, bytes, cudaMemcpyDeviceToHost, s));
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

static double dnorm2(double v) { return v; }
static double dnorm2(cplx v) { return v.re; }

// ||a||^2 and (optionally) <a, b>, read back to the host.
template <class T>
static int dot_host(tg_op *op, const T *a, const T *b, int n, double *aa, typename ST<T>::D *ab, cudaStream_t s) {
    using D = typename ST<T>::D;
    TG_CHECK(red_ready(op, 0, s));
    int g = grid_for(n, 4);
    D *out = reinterpret_cast<D *>(wsp<char>(op, S_SMALL) + SmallArea::dot_out);
    TG_PROF(P_DOT, (b ? 2.0 : 1.0) * n * sizeof(T), (b ? 4.0 : 2.0) * n, k_dot<T><<<g, kThreads, 0, s>>>(a, b, n, wsp<D>(op, S_PART), wsp<unsigned>(op, S_TICKET), out));
    TG_LAUNCH_CHECK();
    TG_CHECK(readback(op, out, 2 * sizeof(D), s));
    const D *h = reinterpret_cast<const D *>(op->pin.p);
    *aa = dnorm2(h[0]);
    if (ab) *ab = h[1];
    return TG_OK;
}

static const DevOp &pick(const tg_op *op, int level, int transpose) {
    const Level &L = level == TG_COARSE ? op->coarse : op->fine;
    return transpose ? L.AT : L.A;
}
static const DevOp32 &pick32(const tg_op *op, int level, int transpose) {
    const Level &L = level == TG_COARSE ? op->coarse : op->fine;
    return transpose ? L.AT32 : L.A32;
}

template <class T>
static int launch_apply(const DevOp &A, const DevOp32 &A32, const T *x, T *y, cudaStream_t s) {
    double xb, fl;
    op_cost(A, &xb, &fl);
    TG_PROF(P_APPLY, (2.0 * sizeof(T) + xb * (sizeof(T) == 4 ? 0.5 : 1.0)) * A.n, fl * A.n, k_apply<T><<<grid_for(A.n, 8), kThreads, 0, s>>>(A, A32, x, y));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

// ----------------------------------------------------------------------------- tall-skinny helpers
// Allows a kernel the device's full dynamic shared memory.  Always the same value, so
// concurrent host threads setting it cannot lower it under each other's launches.
static int max_dyn_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) v = 48 * 1024;
    return v;
}

template <class T>
static int set_smem(const void *fn, size_t bytes) {
    if (bytes > 48 * 1024) {
        const int mx = max_dyn_smem();
        if ((int)bytes > mx) {
            set_error("a launch needs %zu bytes of shared memory, more than the %d available", bytes, mx);
            return TG_BAD_ARG;
        }
        TG_CHECK_CUDA(smem_attr_once(fn, mx));
    }
    return TG_OK;
}

// Out (n x q) = In (n x p) S (p x q)
template <class T>
static int tsm(const T *In, size_t ldi, int p, const T *S, int lds, int q, T *Out, size_t ldo, int n, cudaStream_t s) {
    size_t smem = (size_t)32 * p * sizeof(T);
    TG_CHECK(set_smem<T>((const void *)k_tsm<T>, smem));
    TG_PROF(P_TSM, (double)(p + q) * n * sizeof(T), 2.0 * p * q * n * (sizeof(T) == 16 ? 4 : 1), k_tsm<T><<<tiles_grid(n, 4), kThreads, smem, s>>>(In, ldi, p, S, lds, q, Out, ldo, n));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

// Out (n x q) = In (n x p) S (p x q) for a float32 basis and a float64 S; Out float32 or float64
template <class TO>
static int tsm_f(const float *In, size_t ldi, int p, const double *S, int lds, int q, TO *Out, size_t ldo, int n,
                 cudaStream_t s) {
    TG_ARG(q >= 1 && p >= 1, "float32 tall-skinny product: need q, p >= 1 (q=%d, p=%d)", q, p);
    if (q > 128) {                 // column groups of at most 128 output columns
        for (int c0 = 0; c0 < q; c0 += 128)
            TG_CHECK(tsm_f<TO>(In, ldi, p, S + (size_t)c0 * lds, lds, std::min(128, q - c0), Out + (size_t)c0 * ldo,
                               ldo, n, s));
        return TG_OK;
    }
    TG_ARG(!((uintptr_t)In & 15) && ldi % 4 == 0 && ldi >= (size_t)(n + 63) / 64 * 64,
           "float32 tall-skinny product: In needs 16-byte aligned columns and 64-row padding");
    TG_ARG(((uintptr_t)Out & 15) == 0, "float32 tall-skinny product: Out must be 16-byte aligned");
    const size_t smem = ((size_t)p * q + (size_t)2 * 64 * p) * sizeof(float);
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 63) / 64, (int64_t)num_sms() * 4));
    auto go = [&](auto cpt) -> int {
        constexpr int C = decltype(cpt)::value;
        TG_CHECK(set_smem<float>((const void *)k_tsm_f<TO, C>, smem));
        TG_PROF(P_TSM, (double)p * n * 4 + (double)q * n * sizeof(TO), 2.0 * p * q * n,
                k_tsm_f<TO, C><<<gb, kThreads, smem, s>>>(In, ldi, p, S, lds, q, Out, ldo, n));
        return TG_OK;
    };
    if (q <= 16) TG_CHECK(go(std::integral_constant<int, 1>{}));
    else if (q <= 32) TG_CHECK(go(std::integral_constant<int, 2>{}));
    else if (q <= 64) TG_CHECK(go(std::integral_constant<int, 4>{}));
    else TG_CHECK(go(std::integral_constant<int, 8>{}));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

// h = V^H w (ncol entries, device D array)
// Whether the pipelined V^H w kernel applies (float64 or float32): 16-byte aligned columns
// and room for whole chunks below the leading dimension.
template <class T>
static bool pipe_ok(const T *V, size_t ldv, const T *w, int n, int ncol) {
    if (sizeof(T) != 8 && sizeof(T) != 4) return false;
    const int R = sizeof(T) == 8 ? PipeRows<double>::value : PipeRows<float>::value;
    if ((ldv * sizeof(T)) % 16 || ldv < (size_t)((n + R - 1) / R) * R) return false;
    if (((uintptr_t)V | (uintptr_t)w) & 15) return false;
    return ncol >= 1 && n >= R;
}

// partials of V^H w into part (gb blocks); returns gb
template <class T>
static int gemv_t_part_launch(const T *V, size_t ldv, int ncol, const T *w, int n, typename ST<T>::D *part,
                              cudaStream_t s, bool *used_pipe) {
    if constexpr (sizeof(T) == 8 || sizeof(T) == 4) {
        if (pipe_ok<T>(V, ldv, w, n, ncol)) {
            using E = typename std::conditional<sizeof(T) == 8, double, float>::type;
            constexpr int R = PipeRows<E>::value;
            const int ngr = (ncol + kPipeCols - 1) / kPipeCols;            // column groups (grid y)
            const size_t smem = (size_t)kPipeStages * (std::min(ncol, kPipeCols) + 1) * R * sizeof(E);
            if (smem_attr_once((const void *)k_gemv_t_pipe<E>, max_dyn_smem()) != cudaSuccess) {
                (void)cudaGetLastError();
                goto plain;      // the limit could not be raised: the non-pipelined kernel needs none
            }
            const int per_sm = smem <= 100 * 1024 ? 2 : 1;
            const int nchunks = (n + R - 1) / R;
            const int gb = std::max(1, std::min(nchunks, num_sms() * per_sm));
            k_gemv_t_pipe<E><<<dim3(gb, ngr), kThreads, smem, s>>>(reinterpret_cast<const E *>(V), ldv, ncol,
                                                        reinterpret_cast<const E *>(w), n,
                                                        reinterpret_cast<double *>(part));
            *used_pipe = true;
            return gb;
        }
    }
plain:
    const int gb = (int)std::min<int64_t>((n + 127) / 128, (int64_t)num_sms() * 8);
    k_gemv_t_part<T><<<dim3(std::max(gb, 1), (ncol + kGemvTCols - 1) / kGemvTCols), kThreads, 0, s>>>(V, ldv, ncol,
                                                                                                    w, n, part);
    *used_pipe = false;
    return std::max(gb, 1);
}

template <class T>
static int gemv_t(tg_op *op, const T *V, size_t ldv, int ncol, const T *w, int n, typename ST<T>::D *h, cudaStream_t s) {
    using D = typename ST<T>::D;
    TG_CHECK(red_ready(op, (size_t)num_sms() * 8 * (ncol + 1) * sizeof(D), s));
    bool piped = false;
    int gb = 1;
    TG_PROF(P_GEMV_T, (double)(ncol + 1) * n * sizeof(T), 2.0 * ncol * n * (sizeof(T) == 16 ? 4 : 1),
            gb = gemv_t_part_launch<T>(V, ldv, ncol, w, n, wsp<D>(op, S_PART), s, &piped));
    TG_LAUNCH_CHECK();
    TG_PROF(P_SUM_PART, (double)gb * ncol * sizeof(D), (double)gb * ncol, k_sum_part<D><<<(ncol + 7) / 8, 256, 0, s>>>(wsp<D>(op, S_PART), gb, ncol, h, 0));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

// G = A^H B (k x k, device D array, column-major), sym = 1 for A = B (upper triangle
// computed, the lower one mirrored)
template <class T, int EPT>
static int gram_ept(tg_op *op, const T *A, const T *B, size_t ld, int k, int n, int sym, typename ST<T>::D *G,
                    cudaStream_t s, int kb) {
    using D = typename ST<T>::D;
    const int nent = sym ? k * (k + 1) / 2 : k * kb;
    const int gy = (nent + kThreads * EPT - 1) / (kThreads * EPT);
    const int gx = std::max(1, tiles_grid(n, 4) / gy);
    TG_CHECK(red_ready(op, (size_t)gx * nent * sizeof(D) + (size_t)nent * sizeof(D), s));
    D *part = wsp<D>(op, S_PART);
    D *packed = part + (size_t)gx * nent;
    const size_t smem = (size_t)(A == B ? k : k + kb) * 33 * sizeof(T);
    TG_CHECK(set_smem<T>((const void *)k_gram_packed<T, EPT>, smem));
    TG_PROF(P_GRAM, (A == B ? 1.0 * k : 1.0 * (k + kb)) * n * sizeof(T), 2.0 * nent * n * (sizeof(T) == 16 ? 4 : 1),
            k_gram_packed<T, EPT><<<dim3(gx, gy), kThreads, smem, s>>>(A, B, ld, k, n, sym, nent, part, kb));
    TG_LAUNCH_CHECK();
    TG_PROF(P_SUM_PART, (double)gx * nent * sizeof(D), (double)gx * nent,
            k_sum_part<D><<<(nent + 7) / 8, 256, 0, s>>>(part, gx, nent, packed, 0));
    TG_PROF(P_SMALL, 0, 0, k_gram_unpack<D><<<(nent + 255) / 256, 256, 0, s>>>(packed, k, sym, G, kb));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

// G = A^H B: A has k columns, B has kb columns (kb < 0: kb = k); sym requires B = A.
template <class T>
static int gram(tg_op *op, const T *A, const T *B, size_t ld, int k, int n, int sym, typename ST<T>::D *G,
                cudaStream_t s, int kb = -1) {
    if (kb < 0) kb = k;
    const int nent = sym ? k * (k + 1) / 2 : k * kb;
    if (nent <= kThreads) return gram_ept<T, 1>(op, A, B, ld, k, n, sym, G, s, kb);
    if (nent <= 2 * kThreads) return gram_ept<T, 2>(op, A, B, ld, k, n, sym, G, s, kb);
    if (nent <= 4 * kThreads) return gram_ept<T, 4>(op, A, B, ld, k, n, sym, G, s, kb);
    return gram_ept<T, 8>(op, A, B, ld, k, n, sym, G, s, kb);
}

// CholQR2: A (n x k) = Q R.  Writes Q (n x k), R and Rinv (k x k, device D).
template <class T>
static int cholqr2(tg_op *op, const T *A, int k, int n, T *Q, T *R, T *Rinv, int *info_dev, cudaStream_t s) {
    // k x k scratch from the operator's workspace (no allocation after the first call)
    size_t kb = (size_t)k * k * sizeof(T);
    TG_CHECK(wsx(op, S_CQ_G, kb));
    TG_CHECK(wsx(op, S_CQ_R1, kb));
    TG_CHECK(wsx(op, S_CQ_R1I, kb));
    TG_CHECK(wsx(op, S_CQ_R2, kb));
    TG_CHECK(wsx(op, S_CQ_R2I, kb));
    DBuf &G = op->ws[S_CQ_G], &R1 = op->ws[S_CQ_R1], &R1i = op->ws[S_CQ_R1I], &R2 = op->ws[S_CQ_R2],
         &R2i = op->ws[S_CQ_R2I];
    TG_CHECK(gram<T>(op, A, A, n, k, n, 1, G.as<T>(), s));
    TG_PROF(P_SMALL, 0, 1.0 * k * k * k, launch_chol_inv<T>(G.as<T>(), k, R1.as<T>(), R1i.as<T>(), info_dev, s));
    TG_LAUNCH_CHECK();
    TG_CHECK(tsm<T>(A, n, k, R1i.as<T>(), k, k, Q, n, n, s));
    TG_CHECK(gram<T>(op, Q, Q, n, k, n, 1, G.as<T>(), s));
    TG_PROF(P_SMALL, 0, 1.0 * k * k * k, launch_chol_inv<T>(G.as<T>(), k, R2.as<T>(), R2i.as<T>(), info_dev + 1, s));
    TG_LAUNCH_CHECK();
    TG_CHECK(tsm<T>(Q, n, k, R2i.as<T>(), k, k, Q, n, n, s));   // in place: each tile is staged first
    TG_CHECK(tsm<T>(R2.as<T>(), k, k, R1.as<T>(), k, k, R, k, k, s));     // R = R2 R1
    TG_CHECK(tsm<T>(R1i.as<T>(), k, k, R2i.as<T>(), k, k, Rinv, k, k, s));  // R^-1 = R1^-1 R2^-1
    return TG_OK;
}

}  // namespace tg

// ============================================================================= operator set-up
extern "C" const char *tg_status_string(int status) {
    switch (status) {
        case TG_OK: return "ok";
        case TG_NOT_CONVERGED: return "not converged";
        case TG_BREAKDOWN: return "breakdown";
        case TG_NAN: return "NaN or Inf encountered";
        case TG_BAD_ARG: return "bad argument";
        case TG_OOM: return "out of device memory";
        case TG_CUDA_ERROR: return "CUDA error";
        case TG_SYNC_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

extern "C" const char *tg_last_error(void) { return g_err.c_str(); }

static void const_coefs(DevOp &A, DevOp &AT, DevOp32 &A32, DevOp32 &AT32, int kind, int N, const double *beta,
                        double shift) {
    const double h = 1.0 / (N + 1);
    const double d = -1.0 / (h * h);
    const int dim = kind == TG_CD3D ? 3 : 2;
    A.c0 = 2.0 * dim / (h * h) + shift;
    double bx = beta[0], by = dim == 3 ? beta[1] : 0.0, bz = dim == 3 ? beta[2] : 0.0;
    A.cxm = d - bx / (2 * h);
    A.cxp = d + bx / (2 * h);
    A.cym = d - by / (2 * h);
    A.cyp = d + by / (2 * h);
    A.czm = d - bz / (2 * h);
    A.czp = d + bz / (2 * h);
    AT.c0 = A.c0;
    AT.cxm = A.cxp; AT.cxp = A.cxm;
    AT.cym = A.cyp; AT.cyp = A.cym;
    AT.czm = A.czp; AT.czp = A.czm;
    auto f = [](const DevOp &o, DevOp32 &o32) {
        o32.c0 = (float)o.c0; o32.cxm = (float)o.cxm; o32.cxp = (float)o.cxp; o32.cym = (float)o.cym;
        o32.cyp = (float)o.cyp; o32.czm = (float)o.czm; o32.czp = (float)o.czp;
    };
    f(A, A32);
    f(AT, AT32);
}

extern "C" int tg_setup_operator(tg_op **op_out, int kind, const int64_t *dims, int ndim, const double *beta,
                                 const double *mass, const void *coeffs, int coarse_factor, void *stream) {
    TG_ARG(op_out != nullptr, "op_out is NULL");
    *op_out = nullptr;
    TG_ARG(dims != nullptr && ndim >= 1, "dims must give the grid size");
    TG_ARG(coarse_factor == 2, "coarse_factor must be 2 (got %d)", coarse_factor);
    TG_ARG(kind == TG_CD2D || kind == TG_CD3D || kind == TG_U1_4D || kind == TG_VARK2D || kind == TG_EXP2D,
           "unknown operator kind %d", kind);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = dims[0];
    tg_op *op = new tg_op();
    op->kind = kind;
    op->N = (int)N;
    int rc = TG_OK;
    auto fail = [&](int code) {
        delete op;
        return code;
    };
    if (kind == TG_U1_4D) {
        if (!(N >= 4 && N % 2 == 0 && N <= 64)) { set_error("lattice size L must be even, 4..64 (got %lld)", (long long)N); return fail(TG_BAD_ARG); }
        if (!mass || !coeffs) { set_error("the lattice needs mass and links"); return fail(TG_BAD_ARG); }
        op->cplx_ = true;
        op->dim = 4;
        op->Nc = (int)N / 2;
        op->n = (int)(N * N * N * N);
        op->nc = op->Nc * op->Nc * op->Nc * op->Nc;
        op->mass = *mass;
        const int V = op->n, Vc = op->nc, L = (int)N;
        if ((rc = op->links.ensure((size_t)4 * V * 16)) || (rc = op->pw.ensure((size_t)V * 16)) ||
            (rc = op->cst.ensure((size_t)9 * Vc * 16)))
            return fail(rc);
        if (cudaMemcpyAsync(op->links.p, coeffs, (size_t)4 * V * 16, cudaMemcpyDefault, s) != cudaSuccess) {
            set_error("copy of the links failed");
            return fail(TG_CUDA_ERROR);
        }
        launch_lattice_weights(grid_for(V, 8), s, op->links.as<cplx>(), L, op->pw.as<cplx>());
        launch_lattice_coarse(grid_for(Vc, 8), s, op->links.as<cplx>(), op->pw.as<cplx>(), L,
                                                               op->mass + 8.0, op->cst.as<cplx>());
        DevOp A{};
        A.kind = DK_U1; A.N = L; A.n = V; A.links = op->links.as<cplx>(); A.mdiag = op->mass + 8.0;
        op->fine.A = op->fine.AT = A;
        DevOp C{};
        C.kind = DK_U1C; C.N = op->Nc; C.n = Vc; C.cst = op->cst.as<cplx>();
        op->coarse.A = op->coarse.AT = C;
    } else {
        const int dim = kind == TG_CD3D ? 3 : 2;
        if (!(N >= 3 && N % 2 == 1)) { set_error("grid size N must be odd and >= 3 (got %lld)", (long long)N); return fail(TG_BAD_ARG); }
        const double nn = dim == 3 ? (double)N * N * N : (double)N * N;
        if (nn >= 2147483647.0) { set_error("grid too large"); return fail(TG_BAD_ARG); }
        if (!beta) { set_error("beta is NULL"); return fail(TG_BAD_ARG); }
        op->dim = dim;
        op->Nc = (int)(N - 1) / 2;
        op->n = (int)nn;
        op->nc = dim == 3 ? op->Nc * op->Nc * op->Nc : op->Nc * op->Nc;
        for (int a = 0; a < 3; ++a) op->beta[a] = (a < dim || kind == TG_EXP2D) ? beta[a] : 0.0;
        op->mass = mass ? *mass : 0.0;      // reaction coefficient (diagonal shift) of the grid PDEs
        if (kind == TG_VARK2D && op->mass != 0.0) { set_error("TG_VARK2D takes no shift"); return fail(TG_BAD_ARG); }
        if (kind == TG_EXP2D) {
            const int n = op->n, nc = op->nc;
            if ((rc = op->coef.ensure((size_t)5 * n * 8)) || (rc = op->coef32.ensure((size_t)5 * n * 4)) ||
                (rc = op->coefT.ensure((size_t)5 * n * 8)) || (rc = op->coefT32.ensure((size_t)5 * n * 4)) ||
                (rc = op->ccoef.ensure((size_t)5 * nc * 8)) || (rc = op->ccoef32.ensure((size_t)5 * nc * 4)) ||
                (rc = op->ccoefT.ensure((size_t)5 * nc * 8)) || (rc = op->ccoefT32.ensure((size_t)5 * nc * 4)))
                return fail(rc);
            const double bx = beta[0], by = beta[1], gm = beta[2], sh = op->mass;
            launch_exp2d_coefs(grid_for(n, 8), s, (int)N, bx, by, gm, sh, 0, op->coef.as<double>(), op->coef32.as<float>());
            launch_exp2d_coefs(grid_for(n, 8), s, (int)N, bx, by, gm, sh, 1, op->coefT.as<double>(), op->coefT32.as<float>());
            launch_exp2d_coefs(grid_for(nc, 8), s, op->Nc, bx, by, gm, sh, 0, op->ccoef.as<double>(), op->ccoef32.as<float>());
            launch_exp2d_coefs(grid_for(nc, 8), s, op->Nc, bx, by, gm, sh, 1, op->ccoefT.as<double>(), op->ccoefT32.as<float>());
            DevOp A{};
            A.kind = DK_VAR2D; A.N = (int)N; A.n = n;
            DevOp AT = A, C = A, CT = A;
            A.vc = op->coef.as<double>(); A.vc32 = op->coef32.as<float>();
            AT.vc = op->coefT.as<double>(); AT.vc32 = op->coefT32.as<float>();
            C.N = op->Nc; C.n = nc; C.vc = op->ccoef.as<double>(); C.vc32 = op->ccoef32.as<float>();
            CT.N = op->Nc; CT.n = nc; CT.vc = op->ccoefT.as<double>(); CT.vc32 = op->ccoefT32.as<float>();
            op->fine.A = A; op->fine.AT = AT; op->coarse.A = C; op->coarse.AT = CT;
        } else if (kind == TG_VARK2D) {
            if (!coeffs) { set_error("TG_VARK2D needs kappa"); return fail(TG_BAD_ARG); }
            const int NP = (int)N + 2, NPc = op->Nc + 2;
            const int n = op->n, nc = op->nc;
            if ((rc = op->kappa.ensure((size_t)NP * NP * 8)) || (rc = op->kappa_c.ensure((size_t)NPc * NPc * 8)) ||
                (rc = op->coef.ensure((size_t)5 * n * 8)) || (rc = op->coef32.ensure((size_t)5 * n * 4)) ||
                (rc = op->coefT.ensure((size_t)5 * n * 8)) || (rc = op->coefT32.ensure((size_t)5 * n * 4)) ||
                (rc = op->ccoef.ensure((size_t)5 * nc * 8)) || (rc = op->ccoef32.ensure((size_t)5 * nc * 4)) ||
                (rc = op->ccoefT.ensure((size_t)5 * nc * 8)) || (rc = op->ccoefT32.ensure((size_t)5 * nc * 4)))
                return fail(rc);
            if (cudaMemcpyAsync(op->kappa.p, coeffs, (size_t)NP * NP * 8, cudaMemcpyDefault, s) != cudaSuccess) {
                set_error("copy of kappa failed");
                return fail(TG_CUDA_ERROR);
            }
            launch_inject_kappa(grid_for(NPc * NPc, 8), s, op->kappa.as<double>(), (int)N, op->kappa_c.as<double>());
            launch_vark_coefs(grid_for(n, 8), s, op->kappa.as<double>(), (int)N, beta[0], 1, op->coef.as<double>(), op->coef32.as<float>());
            launch_vark_coefs(grid_for(n, 8), s, op->kappa.as<double>(), (int)N, beta[0], -1, op->coefT.as<double>(), op->coefT32.as<float>());
            launch_vark_coefs(grid_for(nc, 8), s, op->kappa_c.as<double>(), op->Nc, beta[0], 1, op->ccoef.as<double>(), op->ccoef32.as<float>());
            launch_vark_coefs(grid_for(nc, 8), s, op->kappa_c.as<double>(), op->Nc, beta[0], -1, op->ccoefT.as<double>(), op->ccoefT32.as<float>());
            DevOp A{};
            A.kind = DK_VAR2D; A.N = (int)N; A.n = n;
            DevOp AT = A, C = A, CT = A;
            A.vc = op->coef.as<double>(); A.vc32 = op->coef32.as<float>();
            AT.vc = op->coefT.as<double>(); AT.vc32 = op->coefT32.as<float>();
            C.N = op->Nc; C.n = nc; C.vc = op->ccoef.as<double>(); C.vc32 = op->ccoef32.as<float>();
            CT.N = op->Nc; CT.n = nc; CT.vc = op->ccoefT.as<double>(); CT.vc32 = op->ccoefT32.as<float>();
            op->fine.A = A; op->fine.AT = AT; op->coarse.A = C; op->coarse.AT = CT;
        } else {
            DevOp A{}, AT{}, C{}, CT{};
            A.kind = AT.kind = C.kind = CT.kind = (kind == TG_CD3D) ? DK_CD3D : DK_CD2D;
            A.N = AT.N = (int)N;
            A.n = AT.n = op->n;
            C.N = CT.N = op->Nc;
            C.n = CT.n = op->nc;
            const_coefs(A, AT, op->fine.A32, op->fine.AT32, kind, (int)N, op->beta, op->mass);
            const_coefs(C, CT, op->coarse.A32, op->coarse.AT32, kind, op->Nc, op->beta, op->mass);
            op->fine.A = A; op->fine.AT = AT; op->coarse.A = C; op->coarse.AT = CT;
        }
    }
    for (DevOp *d : {&op->fine.A, &op->fine.AT, &op->coarse.A, &op->coarse.AT}) {
        d->fN = FastDiv::of((unsigned)std::max(d->N, 1));
        d->fNN = FastDiv::of((unsigned)std::max<int64_t>((int64_t)d->N * d->N, 1));
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_status(e, "tg_setup_operator"));
    *op_out = op;
    return TG_OK;
}

extern "C" int tg_destroy_op(tg_op *op) {
    delete op;
    return TG_OK;
}

extern "C" int64_t tg_op_size(const tg_op *op, int level) {
    if (!op) return -1;
    return level == TG_COARSE ? op->nc : op->n;
}

extern "C" int tg_apply(const tg_op *op, int level, int transpose, int precision, const void *x, void *y, void *stream) {
    TG_ARG(op && x && y, "NULL argument");
    TG_ARG(level == TG_FINE || level == TG_COARSE, "bad level");
    cudaStream_t s = (cudaStream_t)stream;
    const DevOp &A = pick(op, level, transpose);
    const DevOp32 &A32 = pick32(op, level, transpose);
    if (op->cplx_) {
        TG_ARG(precision == TG_F64, "the lattice operator is complex128 only");
        return launch_apply<cplx>(A, A32, (const cplx *)x, (cplx *)y, s);
    }
    if (precision == TG_F32_IR) return launch_apply<float>(A, A32, (const float *)x, (float *)y, s);
    return launch_apply<double>(A, A32, (const double *)x, (double *)y, s);
}

// ============================================================================= transfer
static int prolong_impl(const tg_op *op, const void *coarse, void *fine, int ncols, cudaStream_t s) {
    for (int c = 0; c < ncols; ++c) {
        if (op->cplx_) {
            const cplx *uc = (const cplx *)coarse + (size_t)c * op->nc;
            cplx *uf = (cplx *)fine + (size_t)c * op->n;
            TG_PROF(P_TRANSFER, (double)(op->n + op->nc) * elem_size(op), 0, launch_prolong_lattice(grid_for(op->n, 8), s, uc, op->pw.as<cplx>(), op->N, uf));
        } else {
            const double *uc = (const double *)coarse + (size_t)c * op->nc;
            double *uf = (double *)fine + (size_t)c * op->n;
            const double bytes = (double)(op->n + op->nc) * elem_size(op);
            if (op->interp == TG_INTERP_CUBIC) {
                if (op->dim == 3) TG_PROF(P_TRANSFER, bytes, 0, launch_prolong3d_cubic(grid_for(op->n, 8), s, uc, op->Nc, uf));
                else TG_PROF(P_TRANSFER, bytes, 0, launch_prolong2d_cubic(grid_for(op->n, 8), s, uc, op->Nc, uf));
            } else {
                if (op->dim == 3) TG_PROF(P_TRANSFER, bytes, 0, launch_prolong3d(grid_for(op->n, 8), s, uc, op->Nc, uf));
                else TG_PROF(P_TRANSFER, bytes, 0, launch_prolong2d(grid_for(op->n, 8), s, uc, op->Nc, uf));
            }
        }
        TG_LAUNCH_CHECK();
    }
    return TG_OK;
}

static int restrict_impl(const tg_op *op, const void *fine, void *coarse, int ncols, cudaStream_t s) {
    for (int c = 0; c < ncols; ++c) {
        if (op->cplx_) {
            const cplx *uf = (const cplx *)fine + (size_t)c * op->n;
            cplx *uc = (cplx *)coarse + (size_t)c * op->nc;
            TG_PROF(P_TRANSFER, (double)(op->n + op->nc) * elem_size(op), op->n * 2.0, launch_restrict_lattice(grid_for(op->nc, 8), s, uf, op->pw.as<cplx>(), op->N, uc));
        } else {
            const double *uf = (const double *)fine + (size_t)c * op->n;
            double *uc = (double *)coarse + (size_t)c * op->nc;
            if (op->dim == 3) TG_PROF(P_TRANSFER, (double)(op->n + op->nc) * elem_size(op), op->n * 2.0, launch_restrict3d(grid_for(op->nc, 8), s, uf, op->N, uc));
            else TG_PROF(P_TRANSFER, (double)(op->n + op->nc) * elem_size(op), op->n * 2.0, launch_restrict2d(grid_for(op->nc, 8), s, uf, op->N, uc));
        }
        TG_LAUNCH_CHECK();
    }
    return TG_OK;
}

extern "C" int tg_prolong(const tg_op *op, const void *coarse, void *fine, int ncols, void *stream) {
    TG_ARG(op && coarse && fine && ncols >= 0, "bad argument");
    return prolong_impl(op, coarse, fine, ncols, (cudaStream_t)stream);
}

extern "C" int tg_op_set_interp(tg_op *op, int interp) {
    TG_ARG(op, "NULL operator");
    TG_ARG(interp == TG_INTERP_LINEAR || interp == TG_INTERP_CUBIC, "unknown interpolation %d", interp);
    TG_ARG(!op->cplx_ || interp == TG_INTERP_LINEAR, "the lattice transfer is block transport only");
    op->interp = interp;
    return TG_OK;
}

extern "C" int tg_restrict(const tg_op *op, const void *fine, void *coarse, int ncols, void *stream) {
    TG_ARG(op && coarse && fine && ncols >= 0, "bad argument");
    return restrict_impl(op, fine, coarse, ncols, (cudaStream_t)stream);
}

// ============================================================================= deflation
namespace tg {

template <class T>
static int build_defl(tg_op *op, int transpose, tg_defl *d, cudaStream_t s) {
    const int n = op->n, kk = d->kk;
    const DevOp &A = pick(op, TG_FINE, transpose);
    const DevOp32 &A32 = pick32(op, TG_FINE, transpose);
    size_t nb = (size_t)n * kk * sizeof(T);
    size_t kb = (size_t)kk * kk * sizeof(T);
    TG_CHECK(d->AY.ensure(nb));
    TG_CHECK(d->Q.ensure(nb));
    TG_CHECK(d->R.ensure(kb));
    TG_CHECK(d->M.ensure(kb));
    TG_CHECK(d->info.ensure(64));
    TG_CHECK_CUDA(cudaMemsetAsync(d->info.p, 0, 64, s));
    const T *Y = d->Y.as<T>();
    T *AY = d->AY.as<T>();
    for (int c = 0; c < kk; ++c) TG_CHECK(launch_apply<T>(A, A32, Y + (size_t)c * n, AY + (size_t)c * n, s));
    int *info = d->info.as<int>();
    if (d->proj == TG_PROJ_MINRES) {
        TG_CHECK(cholqr2<T>(op, AY, kk, n, d->Q.as<T>(), d->R.as<T>(), d->M.as<T>(), info, s));
    } else {
        // V = orth(Y) (in Q), A V = A Y Ry^{-1} (in AV), H = V^H A V (in R), M = H^{-1}
        TG_CHECK(wsx(op, S_GAL_RY, kb));
        TG_CHECK(wsx(op, S_GAL_RYI, kb));
        TG_CHECK(wsx(op, S_GAL_W, 2 * kb));
        DBuf &Ry = op->ws[S_GAL_RY], &Ryi = op->ws[S_GAL_RYI], &W = op->ws[S_GAL_W];
        TG_CHECK(d->AV.ensure(nb));
        TG_CHECK(cholqr2<T>(op, Y, kk, n, d->Q.as<T>(), Ry.as<T>(), Ryi.as<T>(), info, s));
        TG_CHECK(tsm<T>(AY, n, kk, Ryi.as<T>(), kk, kk, d->AV.as<T>(), n, n, s));
        TG_CHECK(gram<T>(op, d->Q.as<T>(), d->AV.as<T>(), n, kk, n, 0, d->R.as<T>(), s));
        TG_PROF(P_SMALL, 0, 2.0 * kk * kk * kk, launch_inverse<T>(d->R.as<T>(), kk, d->M.as<T>(), W.as<T>(), info + 2, s));
        TG_LAUNCH_CHECK();
        TG_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    int hinfo[3] = {0, 0, 0};
    TG_CHECK_CUDA(cudaMemcpy(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost));
    if (hinfo[0] || hinfo[1] || hinfo[2]) {
        set_error("deflation basis is numerically rank deficient (Cholesky/pivot failure %d %d %d)", hinfo[0], hinfo[1], hinfo[2]);
        return TG_BREAKDOWN;
    }
    if (d->precision == TG_F32_IR && !d->cplx_) {
        // float copies: W (Q or V), B1 (Y or V), B2 (Q or A V)
        TG_CHECK(d->W32.ensure((size_t)n * kk * 4));
        TG_CHECK(d->B1_32.ensure((size_t)n * kk * 4));
        TG_CHECK(d->B2_32.ensure((size_t)n * kk * 4));
        const double *B1 = d->proj == TG_PROJ_MINRES ? (const double *)d->Y.p : (const double *)d->Q.p;
        const double *B2 = d->proj == TG_PROJ_MINRES ? (const double *)d->Q.p : (const double *)d->AV.p;
        TG_PROF(P_CONVERT, 12.0 * n * kk, 0, launch_d2f(grid_for((int64_t)n * kk, 8), s, (const double *)d->Q.p, d->W32.as<float>(), (size_t)n * kk));
        TG_PROF(P_CONVERT, 12.0 * n * kk, 0, launch_d2f(grid_for((int64_t)n * kk, 8), s, B1, d->B1_32.as<float>(), (size_t)n * kk));
        TG_PROF(P_CONVERT, 12.0 * n * kk, 0, launch_d2f(grid_for((int64_t)n * kk, 8), s, B2, d->B2_32.as<float>(), (size_t)n * kk));
        TG_LAUNCH_CHECK();
    }
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

// One projection: c = W^H r; d = M c; x += B1 d; r -= B2 e (e = c for MinRes, d for Galerkin).
template <class T>
static int project_impl(tg_op *op, const tg_defl *df, const T *W, const T *B1, const T *B2, T *x, T *r, int n,
                        cudaStream_t s) {
    using D = typename ST<T>::D;
    const int kk = df->kk;
    TG_CHECK(red_ready(op, 0, s));
    D *cvec = reinterpret_cast<D *>(wsp<char>(op, S_SMALL) + SmallArea::proj_c);
    D *dvec = reinterpret_cast<D *>(wsp<char>(op, S_SMALL) + SmallArea::proj_d);
    TG_CHECK(gemv_t<T>(op, W, n, kk, r, n, cvec, s));
    TG_PROF(P_SMALL, 0, 2.0 * kk * kk, launch_small_gemv<D>(df->M.as<D>(), kk, cvec, dvec, s));
    TG_LAUNCH_CHECK();
    const D *e = df->proj == TG_PROJ_MINRES ? cvec : dvec;
    if (kk <= kSmallCols)
        TG_PROF(P_PROJ, (2.0 * kk + 4) * n * sizeof(T), 4.0 * kk * n * (sizeof(T) == 16 ? 4 : 1), k_proj_update<T, kSmallCols><<<grid_for(n, 8), kThreads, 0, s>>>(B1, B2, n, kk, dvec, e, x, r, n));
    else
        TG_PROF(P_PROJ, (2.0 * kk + 4) * n * sizeof(T), 4.0 * kk * n * (sizeof(T) == 16 ? 4 : 1), k_proj_update<T><<<grid_for(n, 8), kThreads, 0, s>>>(B1, B2, n, kk, dvec, e, x, r, n));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

template <class T>
static int project64(tg_op *op, const tg_defl *df, T *x, T *r, cudaStream_t s) {
    const T *W = df->Q.as<T>();
    const T *B1 = df->proj == TG_PROJ_MINRES ? df->Y.as<T>() : df->Q.as<T>();
    const T *B2 = df->proj == TG_PROJ_MINRES ? df->Q.as<T>() : df->AV.as<T>();
    return project_impl<T>(op, df, W, B1, B2, x, r, op->n, s);
}

}  // namespace tg

static int defl_create(tg_op *op, int transpose, int kk, int proj, int precision, tg_defl **out) {
    tg_defl *d = new tg_defl();
    d->kk = kk;
    d->n = op->n;
    d->proj = proj;
    d->precision = precision;
    d->cplx_ = op->cplx_;
    d->transposed = transpose != 0;
    int rc = d->Y.ensure((size_t)op->n * kk * elem_size(op));
    if (rc) {
        delete d;
        return rc;
    }
    *out = d;
    return TG_OK;
}

extern "C" int tg_defl_from_basis(tg_op *op, int transpose, const void *Y, int k, int proj, int precision,
                                  tg_defl **defl_out, void *stream) {
    TG_ARG(op && Y && defl_out, "NULL argument");
    TG_ARG(k >= 1 && k <= kMaxM, "k must be in 1..%d (got %d)", kMaxM, k);
    TG_ARG(proj == TG_PROJ_MINRES || proj == TG_PROJ_GALERKIN, "bad projection kind");
    TG_ARG(precision == TG_F64 || precision == TG_F32_IR, "bad precision");
    TG_ARG(!(op->cplx_ && precision == TG_F32_IR), "the lattice path is complex128 only");
    cudaStream_t s = (cudaStream_t)stream;
    *defl_out = nullptr;
    tg_defl *d;
    TG_CHECK(defl_create(op, transpose, k, proj, precision, &d));
    int rc = cudaMemcpyAsync(d->Y.p, Y, (size_t)op->n * k * elem_size(op), cudaMemcpyDefault, s) == cudaSuccess
                 ? TG_OK : TG_CUDA_ERROR;
    if (!rc) rc = op->cplx_ ? build_defl<cplx>(op, transpose, d, s) : build_defl<double>(op, transpose, d, s);
    if (rc) {
        delete d;
        return rc;
    }
    *defl_out = d;
    return TG_OK;
}

extern "C" int tg_destroy_defl(tg_defl *d) {
    delete d;
    return TG_OK;
}

extern "C" int tg_defl_copy(const tg_defl *d, int what, void *dst, int *kk_out, void *stream) {
    TG_ARG(d, "NULL deflation handle");
    if (kk_out) *kk_out = d->kk;
    if (!dst) return TG_OK;
    const size_t es = d->cplx_ ? 16 : 8;
    const void *src = nullptr;
    size_t bytes = 0;
    switch (what) {
        case 0: src = d->Y.p; bytes = (size_t)d->n * d->kk * es; break;
        case 1: src = d->Q.p; bytes = (size_t)d->n * d->kk * es; break;
        case 2: src = d->AY.p; bytes = (size_t)d->n * d->kk * es; break;
        case 3: src = d->R.p; bytes = (size_t)d->kk * d->kk * es; break;
        default: set_error("what must be 0..3"); return TG_BAD_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    TG_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

extern "C" int tg_project(const tg_op *op_c, const tg_defl *d, void *x, void *r, void *stream) {
    TG_ARG(op_c && d && x && r, "NULL argument");
    tg_op *op = const_cast<tg_op *>(op_c);
    cudaStream_t s = (cudaStream_t)stream;
    if (op->cplx_) return project64<cplx>(op, d, (cplx *)x, (cplx *)r, s);
    return project64<double>(op, d, (double *)x, (double *)r, s);
}

// ============================================================================= BiCGStab cycles
namespace tg {

template <class T> struct BiVecs {
    T *rh, *p, *v, *s, *t;
};

template <class T>
static int bicg_vecs(tg_op *op, int n, BiVecs<T> *w) {
    size_t b = (size_t)n * sizeof(T);
    TG_CHECK(wsx(op, S_RH, b));
    TG_CHECK(wsx(op, S_P, b));
    TG_CHECK(wsx(op, S_V, b));
    TG_CHECK(wsx(op, S_S, b));
    TG_CHECK(wsx(op, S_T, b));
    w->rh = wsp<T>(op, S_RH);
    w->p = wsp<T>(op, S_P);
    w->v = wsp<T>(op, S_V);
    w->s = wsp<T>(op, S_S);
    w->t = wsp<T>(op, S_T);
    return TG_OK;
}

struct CycleOut {
    int mvps = 0;
    int iters = 0;
    int status = 0;
    double rr = 0;
};

// One BiCGStab cycle on A e = r, updating x and r in place (device-resident scalars).
// A float32 cycle on a 3D constant-coefficient grid runs in the padded layout of
// k_bi_pad (rows of pitch P, a multiple of 4 above N, zero padding): x and r are copied in
// at the start and back at the end, and every vector of the cycle has length P N^2.
// padded > 0: x and r are already in that layout (the cycle proper).
template <class T>
static int bicg_cycle(tg_op *op, const DevOp &A, const DevOp32 &A32, T *x, T *r, int n, double target2, int cap,
                      CycleOut *out, cudaStream_t s, int padded = 0) {
    using D = typename ST<T>::D;
    if constexpr (std::is_same<T, float>::value) {
        if (A.kind == DK_CD3D && !padded) {
            const size_t np = (size_t)pad_pitch(A.N) * A.N * A.N;
            TG_CHECK(wsx(op, S_PADX, np * 4));
            TG_CHECK(wsx(op, S_PADR, np * 4));
            float *xp = wsp<float>(op, S_PADX), *rp = wsp<float>(op, S_PADR);
            const int gpk = grid_for((int64_t)np, 8), gn = grid_for(n, 8);
            TG_PROF(P_CONVERT, 8.0 * n, 0, k_pad3d<<<gpk, kThreads, 0, s>>>(x, xp, A.N));
            TG_PROF(P_CONVERT, 8.0 * n, 0, k_pad3d<<<gpk, kThreads, 0, s>>>(r, rp, A.N));
            TG_LAUNCH_CHECK();
            TG_CHECK(bicg_cycle<float>(op, A, A32, xp, rp, (int)np, target2, cap, out, s, n));
            TG_PROF(P_CONVERT, 8.0 * n, 0, k_unpad3d<<<gn, kThreads, 0, s>>>(xp, x, A.N));
            TG_PROF(P_CONVERT, 8.0 * n, 0, k_unpad3d<<<gn, kThreads, 0, s>>>(rp, r, A.N));
            TG_LAUNCH_CHECK();
            return TG_OK;
        }
    }
    const int nb = padded ? padded : n;      // grid points (byte and flop accounting)
    BiVecs<T> w;
    TG_CHECK(bicg_vecs<T>(op, n, &w));
    const int g = grid_for(n, 8);
    // the padded float32 3D stencil kernels, each block marching zlen planes; zlen is chosen
    // so that one wave of resident blocks (two blocks of 32 x kPadRows threads per SM) covers the grid
    const bool use_plane = std::is_same<T, float>::value && padded > 0;
    int zlen_v = 0, zlen_t = 0, gp_v = 0, gp_t = 0;
    if (use_plane) {
        const int tiles = pad_tiles(A.N);
        auto pick_z = [&](int per_sm, int *zl, int *blocks) {
            const int nz = std::max(1, std::min(A.N, num_sms() * per_sm / tiles));
            *zl = (A.N + nz - 1) / nz;
            *blocks = tiles * ((A.N + *zl - 1) / *zl);
        };
        pick_z(2, &zlen_v, &gp_v);
        pick_z(2, &zlen_t, &gp_t);
    }
    const int gp = std::max(gp_v, gp_t);
    TG_CHECK(red_ready(op, (size_t)(g > gp ? g : gp) * 4 * sizeof(D), s));
    D *part = wsp<D>(op, S_PART);
    unsigned *tk = wsp<unsigned>(op, S_TICKET);
    BiState<D> *st = reinterpret_cast<BiState<D> *>(wsp<char>(op, S_SMALL) + SmallArea::bistate);
    TG_PROF(P_BI_INIT, 3.0 * nb * sizeof(T), 2.0 * nb, k_bi_init<T><<<g, kThreads, 0, s>>>(r, w.rh, w.p, n, target2, cap, part, tk, st));
    TG_LAUNCH_CHECK();
    // float32 streaming updates with 16-byte aligned vectors: 4 points per thread
    bool use_v4 = false;
    if constexpr (std::is_same<T, float>::value)
        use_v4 = !(((uintptr_t)x | (uintptr_t)r | (uintptr_t)w.p | (uintptr_t)w.v | (uintptr_t)w.s | (uintptr_t)w.t) & 15);
    const int g4 = grid_for((n + 3) / 4, 8);
    int chunk = 2;
    int launched = 0;
    BiState<D> h{};
    double xb, fl;
    op_cost(A, &xb, &fl);
    const double es = sizeof(T), cf = sizeof(T) == 16 ? 4.0 : 1.0, xbs = sizeof(T) == 4 ? 0.5 * xb : xb;
    const size_t rec0 = g_prof.recs.size();
    double rr_prev = -1.0;
    int iters_prev = 0;
    while (true) {
        for (int c = 0; c < chunk; ++c) {
            if (use_plane) {
                if constexpr (std::is_same<T, float>::value)
                    TG_PROF(P_BI_V, (3 * es + xbs) * nb, (fl + 2 * cf) * nb, k_bi_pad<0><<<gp_v, 32 * kPadRows, 0, s>>>(A, A32, w.p, w.rh, w.v, part, tk, st, zlen_v));
            } else {
                TG_PROF(P_BI_V, (3 * es + xbs) * nb, (fl + 2 * cf) * nb, k_bi_v<T><<<g, kThreads, 0, s>>>(A, A32, w.p, w.rh, w.v, part, tk, st));
            }
            if (use_v4) {
                if constexpr (std::is_same<T, float>::value)
                    TG_PROF(P_BI_S, 3 * es * nb, 4 * cf * nb, k_bi_s_f4<<<g4, kThreads, 0, s>>>(r, w.v, w.s, n, part, tk, st));
            } else {
                TG_PROF(P_BI_S, 3 * es * nb, 4 * cf * nb, k_bi_s<T><<<g, kThreads, 0, s>>>(r, w.v, w.s, n, part, tk, st));
            }
            if (use_plane) {
                if constexpr (std::is_same<T, float>::value)
                    TG_PROF(P_BI_T, (3 * es + xbs) * nb, (fl + 8 * cf) * nb, k_bi_pad<1><<<gp_t, 32 * kPadRows, 0, s>>>(A, A32, w.s, w.rh, w.t, part, tk, st, zlen_t));
            } else {
                TG_PROF(P_BI_T, (3 * es + xbs) * nb, (fl + 8 * cf) * nb, k_bi_t<T><<<g, kThreads, 0, s>>>(A, A32, w.s, w.rh, w.t, part, tk, st));
            }
            if (use_v4) {
                if constexpr (std::is_same<T, float>::value)
                    TG_PROF(P_BI_X, 8 * es * nb, 12 * cf * nb, k_bi_x_f4<<<g4, kThreads, 0, s>>>(x, r, w.p, w.s, w.t, w.v, n, part, tk, st));
            } else {
                TG_PROF(P_BI_X, 8 * es * nb, 12 * cf * nb, k_bi_x<T><<<g, kThreads, 0, s>>>(x, r, w.p, w.s, w.t, w.v, n, part, tk, st));
            }
        }
        TG_LAUNCH_CHECK();
        launched += chunk;
        TG_CHECK(readback(op, st, sizeof(BiState<D>), s));
        memcpy(&h, op->pin.p, sizeof(h));
        if (h.status != 0) break;
        if (launched > cap + 8) {   // the cap test ends a cycle after `cap` products; this cannot trigger
            set_error("BiCGStab cycle exceeded its product cap");
            return TG_SYNC_TIMEOUT;
        }
        // next batch: the iterations still allowed by the cap, and the iterations the
        // observed residual reduction rate predicts until the target (at most 32)
        int left = (h.cap - h.mvps + 1) / 2;
        int want = 32;
        if (rr_prev > 0 && h.rr > 0 && h.rr < rr_prev && h.iters > iters_prev) {
            double rate = log(h.rr / rr_prev) / (h.iters - iters_prev);     // per iteration, < 0
            double need = log(h.target2 / h.rr) / rate;
            if (need < want) want = (int)ceil(need) + 1;
        } else if (rr_prev < 0) {
            want = 4;
        }
        rr_prev = h.rr;
        iters_prev = h.iters;
        chunk = std::max(1, std::min(std::min(want, left), 32));
    }
    // launches queued after the cycle ended returned at once: relabel them so the
    // per-class totals hold only the iterations that ran
    if (g_prof.on) {
        const int ran = h.iters;       // full or half iterations executed
        int it = 0;
        for (size_t q = rec0; q < g_prof.recs.size(); ++q) {
            ProfRec &pr = g_prof.recs[q];
            if (pr.cls == P_BI_V) ++it;
            if (it > ran || (pr.cls == P_BI_T && it == ran && h.half)) {   // a half-step exit skips the t-kernel
                pr.cls = P_NOOP;
                pr.bytes = pr.flops = 0;
            }
        }
    }
    out->mvps = h.mvps;
    out->iters = h.iters;
    out->status = h.status;
    out->rr = h.rr;
    return TG_OK;
}

static double cycle_tol(double rtol, double nr0, double nr, int icyc, int ncyc) {
    double a = pow(rtol * nr0 / nr, 1.0 / (ncyc - icyc + 1));
    double b = (nr0 / nr) * pow(rtol, (double)icyc / ncyc);
    return a < b ? a : b;
}

struct SolveCfg {
    double rtol;
    int ncyc;
    int restart_mvps;
    int m3;
    int64_t max_mvps;
};

static void hist_push(tg_stats *st, double relres, double rt, int64_t mvps) {
    if (!st) return;
    if (st->history && st->history_len < st->history_cap) {
        double *h = st->history + 3 * (size_t)st->history_len;
        h[0] = relres;
        h[1] = rt;
        h[2] = (double)mvps;
    }
    st->history_len += 1;
}

// r = b - A x (float64 / complex128); returns ||r||, ||b||.
template <class T>
static int true_residual(tg_op *op, const DevOp &A, const T *b, const T *x, T *r, double *nr, double *nb, cudaStream_t s) {
    using D = typename ST<T>::D;
    const int n = A.n;
    const int g = grid_for(n, 8);
    TG_CHECK(red_ready(op, (size_t)g * 2 * sizeof(D), s));
    D *out = reinterpret_cast<D *>(wsp<char>(op, S_SMALL) + SmallArea::res_out);
    double xb, fl;
    op_cost(A, &xb, &fl);
    TG_PROF(P_RESIDUAL, (3.0 * sizeof(T) + xb) * n, (fl + 6) * n, k_residual<T><<<g, kThreads, 0, s>>>(A, b, x, r, wsp<D>(op, S_PART), wsp<unsigned>(op, S_TICKET), out));
    TG_LAUNCH_CHECK();
    TG_CHECK(readback(op, out, 2 * sizeof(D), s));
    const D *h = reinterpret_cast<const D *>(op->pin.p);
    *nr = sqrt(dnorm2(h[0]));
    *nb = sqrt(dnorm2(h[1]));
    return TG_OK;
}

// BiCGStab(ncyc)-Proj(k) in float64 / complex128 (Section 4.1, step 3).
template <class T>
static int solve_bicg64(tg_op *op, int transpose, const tg_defl *df, const T *b, T *x, const SolveCfg &cfg,
                        tg_stats *st, cudaStream_t s) {
    const DevOp &A = pick(op, TG_FINE, transpose);
    const DevOp32 &A32 = pick32(op, TG_FINE, transpose);
    const int n = op->n;
    TG_CHECK(wsx(op, S_R64, (size_t)n * sizeof(T)));
    T *r = wsp<T>(op, S_R64);
    double nr, nb;
    TG_CHECK(true_residual<T>(op, A, b, x, r, &nr, &nb, s));
    int64_t mvps = 0;
    int cyc = 0;
    int status = TG_NOT_CONVERGED;
    if (!std::isfinite(nr)) status = TG_NAN;
    else if (nb == 0.0 || nr <= cfg.rtol * nb) status = TG_OK;
    while (status == TG_NOT_CONVERGED) {
        ++cyc;
        const bool sched = cfg.ncyc && cyc <= cfg.ncyc;   // beyond ncyc: finish with rtol ||b|| / ||r||
        if (df && df->kk > 0) {                                    // step a
            TG_CHECK(project64<T>(op, df, x, r, s));
            double rr;
            TG_CHECK(dot_host<T>(op, r, nullptr, n, &rr, nullptr, s));
            nr = sqrt(rr);
        }
        double rt = sched ? cycle_tol(cfg.rtol, nb, nr, cyc, cfg.ncyc) : cfg.rtol * nb / nr;   // step b
        hist_push(st, nr / nb, rt, mvps);
        int64_t cap64 = cfg.max_mvps - mvps;
        if (cfg.restart_mvps > 0 && cap64 > cfg.restart_mvps) cap64 = cfg.restart_mvps;
        if (cap64 > INT_MAX / 2) cap64 = INT_MAX / 2;
        CycleOut co;
        TG_CHECK(bicg_cycle<T>(op, A, A32, x, r, n, (rt * nr) * (rt * nr), (int)cap64, &co, s));   // step c
        mvps += co.mvps;
        if (co.status == 4) { status = TG_NAN; break; }
        TG_CHECK(true_residual<T>(op, A, b, x, r, &nr, &nb, s));
        if (!std::isfinite(nr)) { status = TG_NAN; break; }
        if (nr <= cfg.rtol * nb) { status = TG_OK; break; }        // step d
        if (mvps >= cfg.max_mvps) break;
        if (co.mvps == 0) { status = TG_BREAKDOWN; break; }   // no progress possible
    }
    if (st) {
        st->mvps = mvps;
        st->cycles = cyc;
        st->relres = nb > 0 ? nr / nb : 0.0;
        st->status = status;
        st->vops = mvps * 7;
    }
    return status;
}

// float32 inner cycles with float64 refinement (real operators only).
constexpr int64_t kIrCycleCap = 2000;
constexpr double kIrGrowth = 4.0;        // batched form: a correction raising ||r|| more than this is undone
static int solve_bicg_ir(tg_op *op, int transpose, const tg_defl *df, const double *b, double *x, const SolveCfg &cfg,
                         tg_stats *st, cudaStream_t s) {
    const DevOp &A = pick(op, TG_FINE, transpose);
    const DevOp32 &A32 = pick32(op, TG_FINE, transpose);
    const int n = op->n;
    TG_CHECK(wsx(op, S_R64, (size_t)n * 8));
    TG_CHECK(wsx(op, S_R32, (size_t)n * 4));
    TG_CHECK(wsx(op, S_E32, (size_t)n * 4));
    TG_CHECK(wsx(op, S_XBAK, (size_t)n * 8));
    double *xbak = wsp<double>(op, S_XBAK);
    int fp64_cycles = 0;
    double *r = wsp<double>(op, S_R64);
    float *r32 = wsp<float>(op, S_R32), *e32 = wsp<float>(op, S_E32);
    double nr, nb;
    TG_CHECK(true_residual<double>(op, A, b, x, r, &nr, &nb, s));
    int64_t mvps = 0;
    int cyc = 0;
    int status = TG_NOT_CONVERGED;
    if (!std::isfinite(nr)) status = TG_NAN;
    else if (nb == 0.0 || nr <= cfg.rtol * nb) status = TG_OK;
    const int g = grid_for(n, 8);
    while (status == TG_NOT_CONVERGED) {
        ++cyc;
        const bool sched = cfg.ncyc && cyc <= cfg.ncyc;   // beyond ncyc: finish with rtol ||b|| / ||r||
        // correction equation A e = r, scaled so that ||r32|| = 1
        TG_PROF(P_CONVERT, 12.0 * n, n, launch_d2f_scaled(g, s, r, r32, n, 1.0 / nr));
        TG_CHECK_CUDA(cudaMemsetAsync(e32, 0, (size_t)n * 4, s));
        double scale = nr;
        double nrel = 1.0;
        if (df && df->kk > 0) {
            TG_CHECK(project_impl<float>(op, df, df->W32.as<float>(), df->B1_32.as<float>(), df->B2_32.as<float>(), e32,
                                         r32, n, s));
            double rr;
            TG_CHECK(dot_host<float>(op, r32, nullptr, n, &rr, nullptr, s));
            nrel = sqrt(rr);
        }
        const double nrp = nrel * scale;    // residual norm after the projection
        double rt = sched ? cycle_tol(cfg.rtol, nb, nrp, cyc, cfg.ncyc) : cfg.rtol * nb / nrp;
        if (rt < 1e-6) rt = 1e-6;   // a float32 cycle cannot resolve more; refinement continues
        hist_push(st, nrp / nb, rt, mvps);
        int64_t cap64 = cfg.max_mvps - mvps;
        // a float32 cycle that stagnates above its target ends after kIrCycleCap products
        const int64_t cyc_cap = cfg.restart_mvps > 0 ? cfg.restart_mvps : kIrCycleCap;
        if (cap64 > cyc_cap) cap64 = cyc_cap;
        if (cap64 > INT_MAX / 2) cap64 = INT_MAX / 2;
        CycleOut co;
        TG_CHECK(bicg_cycle<float>(op, A, A32, e32, r32, n, (rt * nrel) * (rt * nrel), (int)cap64, &co, s));
        mvps += co.mvps;
        // keep x: a float32 correction that does not lower the float64 residual is undone
        TG_CHECK_CUDA(cudaMemcpyAsync(xbak, x, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        const double nr_before = nr;
        TG_PROF(P_CONVERT, 20.0 * n, 2.0 * n, launch_add_f2d_scaled(g, s, x, e32, n, scale));
        TG_LAUNCH_CHECK();
        TG_CHECK(true_residual<double>(op, A, b, x, r, &nr, &nb, s));
        if (std::isfinite(nr) && nr <= cfg.rtol * nb) { status = TG_OK; break; }
        if (!std::isfinite(nr) || nr >= nr_before || co.status == 4 || co.status == 5) {
            // float32 cannot resolve this system (its rounding times the condition number is
            // too large): restore x and finish with float64 cycles on the GPU
            TG_CHECK_CUDA(cudaMemcpyAsync(x, xbak, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
            SolveCfg c64 = cfg;
            c64.max_mvps = std::max<int64_t>(1, cfg.max_mvps - mvps);
            c64.ncyc = 0;
            if (c64.restart_mvps <= 0) c64.restart_mvps = 1000;
            tg_stats s64{};
            s64.history = nullptr;
            const int rc64 = solve_bicg64<double>(op, transpose, df, b, x, c64, &s64, s);
            mvps += s64.mvps;
            cyc += s64.cycles;
            fp64_cycles = s64.cycles;
            nr = s64.relres * nb;
            status = rc64;
            break;
        }
        if (mvps >= cfg.max_mvps) break;
        if (co.mvps == 0) { status = TG_BREAKDOWN; break; }
    }
    if (st) {
        st->mvps = mvps;
        st->cycles = cyc;
        st->relres = nb > 0 ? nr / nb : 0.0;
        st->status = status;
        st->vops = mvps * 7;
        st->fp64_cycles = fp64_cycles;
    }
    return status;
}

// ----------------------------------------------------------------------------- IDR(s)
struct IdrCfg {
    int s;
    double kappa;
    const void *P_in;      // caller's n x s shadow columns (orthonormalised once per solve)
};

// One IDR(s) cycle on A e = r (updating x and r); device-resident scalars, status read
// once per batch of rounds.
template <class T>
static int idr_cycle(tg_op *op, const DevOp &A, const DevOp32 &A32, T *x, T *r, int n, const T *P, int sd,
                     double kappa, double target2, int cap, CycleOut *out, cudaStream_t s) {
    using D = typename ST<T>::D;
    const size_t ld = (size_t)n;
    TG_CHECK(wsx(op, S_IG, (size_t)n * sd * sizeof(T)));
    TG_CHECK(wsx(op, S_IU, (size_t)n * sd * sizeof(T)));
    TG_CHECK(wsx(op, S_IT, (size_t)n * sizeof(T)));
    T *G = wsp<T>(op, S_IG), *U = wsp<T>(op, S_IU), *t = wsp<T>(op, S_IT);
    const int g = grid_for(n, 8);
    TG_CHECK(red_ready(op, (size_t)g * (kIdrMaxS + 1) * sizeof(D) + sizeof(IdrState<D>), s));
    D *part = wsp<D>(op, S_PART);
    unsigned *tk = wsp<unsigned>(op, S_TICKET);
    IdrState<D> *st = reinterpret_cast<IdrState<D> *>(wsp<char>(op, S_SMALL) + SmallArea::idr);
    const double es = sizeof(T);
    double xb, fl;
    op_cost(A, &xb, &fl);
    const double cf = sizeof(T) == 16 ? 4.0 : 1.0;
    TG_PROF(P_IDR_UPD, (1.0 + sd) * n * es, 2.0 * (sd + 1) * n * cf,
            k_idr_init<T><<<g, kThreads, 0, s>>>(r, P, ld, n, sd, target2, cap, kappa, part, tk, st));
    TG_LAUNCH_CHECK();
    int batch = 1, launched = 0;
    IdrState<D> h{};
    while (true) {
        for (int b = 0; b < batch; ++b) {
            const int first = launched + b == 0;
            for (int k = 0; k < sd; ++k) {
                TG_PROF(P_IDR_UPD, (2.0 + (first ? 0.0 : 2.0 * (sd - k))) * n * es, 4.0 * (sd - k) * n * cf,
                        k_idr_u<T><<<g, kThreads, 0, s>>>(r, G, U, ld, n, k, first, st));
                TG_PROF(P_IDR_MV, (2.0 + sd) * n * es + xb * n, (fl + 2.0 * sd * cf) * n,
                        k_idr_g<T><<<g, kThreads, 0, s>>>(A, A32, U, G, P, ld, k, part, tk, st));
                TG_PROF(P_IDR_UPD, (2.0 * k + 8.0) * n * es, (4.0 * k + 6.0) * n * cf,
                        k_idr_upd<T><<<g, kThreads, 0, s>>>(G, U, ld, r, x, n, k, part, tk, st));
            }
            TG_PROF(P_IDR_MV, 2.0 * n * es + xb * n, (fl + 6.0 * cf) * n,
                    k_idr_t<T><<<g, kThreads, 0, s>>>(A, A32, r, t, part, tk, st));
            TG_PROF(P_IDR_UPD, (5.0 + sd) * n * es, (4.0 + 2.0 * (sd + 1)) * n * cf,
                    k_idr_xr<T><<<g, kThreads, 0, s>>>(x, r, t, P, ld, n, part, tk, st));
        }
        TG_LAUNCH_CHECK();
        launched += batch;
        TG_CHECK(readback(op, st, sizeof(IdrState<D>), s));
        memcpy(&h, op->pin.p, sizeof(h));
        if (h.status != 0) break;
        if ((int64_t)launched * (sd + 1) > (int64_t)cap + 2 * (sd + 1)) {   // the cap test ends the cycle first
            set_error("IDR cycle exceeded its product cap");
            return TG_SYNC_TIMEOUT;
        }
        const int left = (h.cap - h.mvps) / (sd + 1) + 1;
        batch = std::max(1, std::min(std::min(2 * batch, left), 16));
    }
    out->mvps = h.mvps;
    out->iters = h.rounds;
    out->status = h.status;
    out->rr = h.rr;
    return TG_OK;
}

// IDR(ncyc)-Proj(k) in float64 / complex128: the Section 4.1 schedule of solve_bicg64 with
// IDR(s) cycles.  The shadow space is the caller's n x s columns orthonormalised by CholQR2
// (positive-diagonal R), the same for every cycle.
template <class T>
static int solve_idr64(tg_op *op, const tg_defl *df, const T *b, T *x, const SolveCfg &cfg, const IdrCfg &ic,
                       tg_stats *st, cudaStream_t s) {
    const DevOp &A = pick(op, TG_FINE, 0);
    const int n = op->n, sv = ic.s;
    TG_CHECK(wsx(op, S_R64, (size_t)n * sizeof(T)));
    TG_CHECK(wsx(op, S_IP, (size_t)n * sv * sizeof(T)));
    TG_CHECK(wsx(op, S_IPR, (size_t)sv * sv * sizeof(T)));
    TG_CHECK(wsx(op, S_IPRI, (size_t)sv * sv * sizeof(T)));
    TG_CHECK(wsx(op, S_IINFO, 64));
    TG_CHECK_CUDA(cudaMemsetAsync(op->ws[S_IINFO].p, 0, 64, s));
    T *P = wsp<T>(op, S_IP);
    TG_CHECK(cholqr2<T>(op, static_cast<const T *>(ic.P_in), sv, n, P, wsp<T>(op, S_IPR), wsp<T>(op, S_IPRI),
                        wsp<int>(op, S_IINFO), s));
    {
        int info[2] = {0, 0};
        TG_CHECK(readback(op, wsp<int>(op, S_IINFO), 2 * sizeof(int), s));
        memcpy(info, op->pin.p, sizeof(info));
        if (info[0] || info[1]) {
            set_error("the shadow columns are linearly dependent (Cholesky of P^H P failed)");
            return TG_BAD_ARG;
        }
    }
    T *r = wsp<T>(op, S_R64);
    double nr, nb;
    TG_CHECK(true_residual<T>(op, A, b, x, r, &nr, &nb, s));
    int64_t mvps = 0;
    int cyc = 0;
    int status = TG_NOT_CONVERGED;
    if (!std::isfinite(nr)) status = TG_NAN;
    else if (nb == 0.0 || nr <= cfg.rtol * nb) status = TG_OK;
    while (status == TG_NOT_CONVERGED) {
        ++cyc;
        const bool sched = cfg.ncyc && cyc <= cfg.ncyc;
        if (df && df->kk > 0) {
            TG_CHECK(project64<T>(op, df, x, r, s));
            double rr;
            TG_CHECK(dot_host<T>(op, r, nullptr, n, &rr, nullptr, s));
            nr = sqrt(rr);
        }
        const double rt = sched ? cycle_tol(cfg.rtol, nb, nr, cyc, cfg.ncyc) : cfg.rtol * nb / nr;
        hist_push(st, nr / nb, rt, mvps);
        int64_t cap64 = cfg.max_mvps - mvps;
        if (cfg.restart_mvps > 0 && cap64 > cfg.restart_mvps) cap64 = cfg.restart_mvps;
        if (cap64 > INT_MAX / 2) cap64 = INT_MAX / 2;
        CycleOut co;
        TG_CHECK(idr_cycle<T>(op, A, pick32(op, TG_FINE, 0), x, r, n, P, sv, ic.kappa, (rt * nr) * (rt * nr),
                              (int)cap64, &co, s));
        mvps += co.mvps;
        if (co.status == 4) { status = TG_NAN; break; }
        TG_CHECK(true_residual<T>(op, A, b, x, r, &nr, &nb, s));
        if (!std::isfinite(nr)) { status = TG_NAN; break; }
        if (nr <= cfg.rtol * nb) { status = TG_OK; break; }
        if (mvps >= cfg.max_mvps) break;
        if (co.mvps == 0) { status = TG_BREAKDOWN; break; }
    }
    if (st) {
        st->mvps = mvps;
        st->cycles = cyc;
        st->relres = nb > 0 ? nr / nb : 0.0;
        st->status = status;
        st->vops = mvps * (4 * sv + 8) / (sv + 1);
    }
    return status;
}

// IDR(ncyc)-Proj(k) in the float32 + refinement form (real operators): each cycle solves the
// correction equation A e = r / ||r|| by float32 IDR(s) (float32 shadow space: the float64
// orthonormalised one rounded once), after a float32 projection; x += ||r|| e in float64 and
// the true residual is recomputed in float64.  A correction that does not lower the float64
// residual is undone and float64 IDR(s)-Proj cycles finish the solve, as in solve_bicg_ir.
static int solve_idr_ir(tg_op *op, const tg_defl *df, const double *b, double *x, const SolveCfg &cfg,
                        const IdrCfg &ic, tg_stats *st, cudaStream_t s) {
    const DevOp &A = pick(op, TG_FINE, 0);
    const DevOp32 &A32 = pick32(op, TG_FINE, 0);
    const int n = op->n, sv = ic.s;
    TG_CHECK(wsx(op, S_IP, (size_t)n * sv * 8));
    TG_CHECK(wsx(op, S_IPR, (size_t)sv * sv * 8));
    TG_CHECK(wsx(op, S_IPRI, (size_t)sv * sv * 8));
    TG_CHECK(wsx(op, S_IINFO, 64));
    TG_CHECK(wsx(op, S_IP32, (size_t)n * sv * 4));
    TG_CHECK_CUDA(cudaMemsetAsync(op->ws[S_IINFO].p, 0, 64, s));
    double *P = wsp<double>(op, S_IP);
    float *P32 = wsp<float>(op, S_IP32);
    TG_CHECK(cholqr2<double>(op, static_cast<const double *>(ic.P_in), sv, n, P, wsp<double>(op, S_IPR),
                             wsp<double>(op, S_IPRI), wsp<int>(op, S_IINFO), s));
    {
        int info[2] = {0, 0};
        TG_CHECK(readback(op, wsp<int>(op, S_IINFO), 2 * sizeof(int), s));
        memcpy(info, op->pin.p, sizeof(info));
        if (info[0] || info[1]) {
            set_error("the shadow columns are linearly dependent (Cholesky of P^H P failed)");
            return TG_BAD_ARG;
        }
    }
    TG_PROF(P_CONVERT, 12.0 * n * sv, 0, launch_d2f(grid_for((int64_t)n * sv, 8), s, P, P32, (size_t)n * sv));
    TG_LAUNCH_CHECK();
    TG_CHECK(wsx(op, S_R64, (size_t)n * 8));
    TG_CHECK(wsx(op, S_R32, (size_t)n * 4));
    TG_CHECK(wsx(op, S_E32, (size_t)n * 4));
    TG_CHECK(wsx(op, S_XBAK, (size_t)n * 8));
    double *xbak = wsp<double>(op, S_XBAK), *r = wsp<double>(op, S_R64);
    float *r32 = wsp<float>(op, S_R32), *e32 = wsp<float>(op, S_E32);
    const int g = grid_for(n, 8);
    double nr, nb;
    TG_CHECK(true_residual<double>(op, A, b, x, r, &nr, &nb, s));
    int64_t mvps = 0;
    int cyc = 0, fp64_cycles = 0;
    int status = TG_NOT_CONVERGED;
    if (!std::isfinite(nr)) status = TG_NAN;
    else if (nb == 0.0 || nr <= cfg.rtol * nb) status = TG_OK;
    while (status == TG_NOT_CONVERGED) {
        ++cyc;
        const bool sched = cfg.ncyc && cyc <= cfg.ncyc;
        TG_PROF(P_CONVERT, 12.0 * n, n, launch_d2f_scaled(g, s, r, r32, n, 1.0 / nr));
        TG_CHECK_CUDA(cudaMemsetAsync(e32, 0, (size_t)n * 4, s));
        const double scale = nr;
        double nrel = 1.0;
        if (df && df->kk > 0) {
            TG_CHECK(project_impl<float>(op, df, df->W32.as<float>(), df->B1_32.as<float>(), df->B2_32.as<float>(), e32,
                                         r32, n, s));
            double rr;
            TG_CHECK(dot_host<float>(op, r32, nullptr, n, &rr, nullptr, s));
            nrel = sqrt(rr);
        }
        const double nrp = nrel * scale;
        double rt = sched ? cycle_tol(cfg.rtol, nb, nrp, cyc, cfg.ncyc) : cfg.rtol * nb / nrp;
        if (rt < 1e-6) rt = 1e-6;   // a float32 cycle cannot resolve more; refinement continues
        hist_push(st, nrp / nb, rt, mvps);
        int64_t cap64 = cfg.max_mvps - mvps;
        const int64_t cyc_cap = cfg.restart_mvps > 0 ? cfg.restart_mvps : kIrCycleCap;
        if (cap64 > cyc_cap) cap64 = cyc_cap;
        if (cap64 > INT_MAX / 2) cap64 = INT_MAX / 2;
        CycleOut co;
        TG_CHECK(idr_cycle<float>(op, A, A32, e32, r32, n, P32, sv, ic.kappa, (rt * nrel) * (rt * nrel), (int)cap64,
                                  &co, s));
        mvps += co.mvps;
        TG_CHECK_CUDA(cudaMemcpyAsync(xbak, x, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        const double nr_before = nr;
        TG_PROF(P_CONVERT, 20.0 * n, 2.0 * n, launch_add_f2d_scaled(g, s, x, e32, n, scale));
        TG_LAUNCH_CHECK();
        TG_CHECK(true_residual<double>(op, A, b, x, r, &nr, &nb, s));
        if (std::isfinite(nr) && nr <= cfg.rtol * nb) { status = TG_OK; break; }
        if (!std::isfinite(nr) || nr >= nr_before || co.status == 4) {
            TG_CHECK_CUDA(cudaMemcpyAsync(x, xbak, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
            SolveCfg c64 = cfg;
            c64.max_mvps = std::max<int64_t>(1, cfg.max_mvps - mvps);
            c64.ncyc = 0;
            if (c64.restart_mvps <= 0) c64.restart_mvps = 1000;
            tg_stats s64{};
            s64.history = nullptr;
            const int rc64 = solve_idr64<double>(op, df, b, x, c64, ic, &s64, s);
            mvps += s64.mvps;
            cyc += s64.cycles;
            fp64_cycles = s64.cycles;
            nr = s64.relres * nb;
            status = rc64;
            break;
        }
        if (mvps >= cfg.max_mvps) break;
        if (co.mvps == 0) { status = TG_BREAKDOWN; break; }
    }
    if (st) {
        st->mvps = mvps;
        st->cycles = cyc;
        st->relres = nb > 0 ? nr / nb : 0.0;
        st->status = status;
        st->vops = mvps * (4 * sv + 8) / (sv + 1);
        st->fp64_cycles = fp64_cycles;
    }
    return status;
}

// ----------------------------------------------------------------------------- Arnoldi (CGS2)
// Extends V (ld ldv, columns 0..j orthonormal) by column j+1 = A v_j orthogonalised; writes
// Hbar column j (ld ldh).  Two classical Gram-Schmidt passes as tall-skinny products.
// w -= V h and ||w||^2 (k_gemv_n_norm), with the float4 kernel for an aligned float32 basis
// (its rows in groups of 4; no re-orthogonalisation flag, which no caller reads there)
template <class T>
static void gemv_n_norm_launch(int g, const T *V, size_t ldv, int ncol, const typename ST<T>::D *h, T *w, int n,
                               typename ST<T>::D *part, unsigned *tk, double *nrm,
                               const typename ST<T>::D *nrm_before, int *flag, double eta2, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (ldv % 4 == 0 && !(((uintptr_t)V | (uintptr_t)w) & 15)) {
            if (ncol <= kSmallCols) k_gemv_n_norm_f4<kSmallCols><<<g, kThreads, 0, s>>>(V, ldv, ncol, h, w, n, part, tk, nrm);
            else k_gemv_n_norm_f4<><<<g, kThreads, 0, s>>>(V, ldv, ncol, h, w, n, part, tk, nrm);
            return;
        }
    }
    if (ncol <= kSmallCols)
        k_gemv_n_norm<T, kSmallCols><<<g, kThreads, 0, s>>>(V, ldv, ncol, h, w, n, nullptr, part, tk, nrm, nrm_before, flag, eta2);
    else
        k_gemv_n_norm<T><<<g, kThreads, 0, s>>>(V, ldv, ncol, h, w, n, nullptr, part, tk, nrm, nrm_before, flag, eta2);
}

template <class T, class HT = T>
static int arnoldi_step(tg_op *op, const DevOp &A, const DevOp32 &A32, T *V, size_t ldv, int n, int j, HT *H, int ldh,
                        cudaStream_t s) {
    using D = typename ST<T>::D;
    // w = A v_j, then two classical Gram-Schmidt passes, each a tall-skinny V^H w and a
    // fused update + norm
    T *w = V + (size_t)(j + 1) * ldv;
    TG_CHECK(launch_apply<T>(A, A32, V + (size_t)j * ldv, w, s));
    TG_CHECK(red_ready(op, 0, s));
    char *sm = wsp<char>(op, S_SMALL);
    D *h1 = reinterpret_cast<D *>(sm + SmallArea::arn_h1);   // j+2 entries: V_j^H w and ||w||^2
    D *h2 = reinterpret_cast<D *>(sm + SmallArea::arn_h2);
    double *nrm = reinterpret_cast<double *>(sm + SmallArea::arn_nrm);
    double *inv = nrm + 4;
    int *flag = reinterpret_cast<int *>(sm + SmallArea::arn_nrm + 64);
    const int g = grid_for(n, 8);
    const int gb = (int)std::min<int64_t>((n + 127) / 128, (int64_t)num_sms() * 8);
    const int ncol = j + 1;
    D *part = wsp<D>(op, S_PART);
    unsigned *tk = wsp<unsigned>(op, S_TICKET);
    TG_CHECK(red_ready(op, (size_t)gb * (ncol + 1) * sizeof(D), s));
    part = wsp<D>(op, S_PART);
    // pass 1: h1 = [V_j, w]^H w
    bool piped = false;
    int gbt = gb;
    TG_PROF(P_GEMV_T, (double)(ncol + 1) * n * sizeof(T), 2.0 * (ncol + 1) * n * (sizeof(T) == 16 ? 4 : 1),
            gbt = gemv_t_part_launch<T>(V, ldv, ncol + 1, w, n, part, s, &piped));
    TG_PROF(P_SUM_PART, (double)gbt * (ncol + 1) * sizeof(D), (double)gbt * (ncol + 1),
            k_sum_part<D><<<(ncol + 1 + 7) / 8, 256, 0, s>>>(part, gbt, ncol + 1, h1, 0));
    TG_PROF(P_GEMV_N, (ncol + 2.0) * n * sizeof(T), 2.0 * ncol * n * (sizeof(T) == 16 ? 4 : 1),
            gemv_n_norm_launch<T>(g, V, ldv, ncol, h1, w, n, part, tk, nrm, h1 + ncol, flag, 0.5, s));
    // pass 2 (classical Gram-Schmidt twice: on this operator the selective criterion of
    // Daniel, Gragg, Kaufman and Stewart asked for the second pass on nearly every step)
    TG_PROF(P_GEMV_T, (double)(ncol + 1) * n * sizeof(T), 2.0 * ncol * n * (sizeof(T) == 16 ? 4 : 1),
            gbt = gemv_t_part_launch<T>(V, ldv, ncol, w, n, part, s, &piped));
    TG_PROF(P_SUM_PART, (double)gbt * ncol * sizeof(D), (double)gbt * ncol,
            k_sum_part<D><<<(ncol + 7) / 8, 256, 0, s>>>(part, gbt, ncol, h2, 0));
    TG_PROF(P_GEMV_N, (ncol + 2.0) * n * sizeof(T), 2.0 * ncol * n * (sizeof(T) == 16 ? 4 : 1),
            gemv_n_norm_launch<T>(g, V, ldv, ncol, h2, w, n, part, tk, nrm, nullptr, nullptr, 0.0, s));
    TG_PROF(P_SMALL, 0, j, k_arnoldi_finish2<T, HT><<<1, 128, 0, s>>>(h1, h2, nrm, j, H + (size_t)j * ldh, inv));
    TG_PROF(P_SCALE, 2.0 * n * sizeof(T), n, k_scale_by<T><<<g, kThreads, 0, s>>>(w, n, inv));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

// GMRES(m)-Proj(k) (Section 2.2) in float64 / complex128.
template <class T>
static int solve_gmres64(tg_op *op, int transpose, const tg_defl *df, const T *b, T *x, const SolveCfg &cfg,
                         tg_stats *st, cudaStream_t s) {
    using D = typename ST<T>::D;
    const DevOp &A = pick(op, TG_FINE, transpose);
    const DevOp32 &A32 = pick32(op, TG_FINE, transpose);
    const int n = op->n, m = cfg.m3;
    const int ldh = m + 1;
    TG_CHECK(wsx(op, S_R64, (size_t)n * sizeof(T)));
    TG_CHECK(wsx(op, S_FV, (size_t)n * (m + 1) * sizeof(T)));
    TG_CHECK(wsx(op, S_FH, (size_t)(m + 1) * m * sizeof(T)));
    TG_CHECK(wsx(op, S_FCS, (size_t)(m + 1) * sizeof(D)));
    TG_CHECK(wsx(op, S_FSN, (size_t)(m + 1) * sizeof(D)));
    TG_CHECK(wsx(op, S_FG, (size_t)(m + 1) * sizeof(D)));
    TG_CHECK(wsx(op, S_FY, (size_t)(m + 1) * sizeof(D)));
    TG_CHECK(wsx(op, S_FSTATE, sizeof(GivensState)));
    T *r = wsp<T>(op, S_R64);
    T *V = wsp<T>(op, S_FV);
    D *H = wsp<D>(op, S_FH);
    GivensState *gs = wsp<GivensState>(op, S_FSTATE);
    double nr, nb;
    TG_CHECK(true_residual<T>(op, A, b, x, r, &nr, &nb, s));
    int64_t mvps = 0;
    int cyc = 0;
    int status = TG_NOT_CONVERGED;
    if (!std::isfinite(nr)) status = TG_NAN;
    else if (nb == 0.0 || nr <= cfg.rtol * nb) status = TG_OK;
    while (status == TG_NOT_CONVERGED && mvps < cfg.max_mvps) {
        ++cyc;
        if (df && df->kk > 0) {
            TG_CHECK(project64<T>(op, df, x, r, s));
            double rr;
            TG_CHECK(dot_host<T>(op, r, nullptr, n, &rr, nullptr, s));
            nr = sqrt(rr);
        }
        hist_push(st, nr / nb, 0.0, mvps);
        // v_0 = r / ||r||; g = ||r|| e_1
        TG_CHECK_CUDA(cudaMemcpyAsync(V, r, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        GivensState h0{};
        h0.target = cfg.rtol * nb;
        h0.resid = nr;
        double *inv = reinterpret_cast<double *>(wsp<char>(op, S_SMALL) + SmallArea::gmres_inv);
        double hinv = 1.0 / nr;
        TG_CHECK_CUDA(cudaMemcpyAsync(inv, &hinv, sizeof(double), cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemcpyAsync(gs, &h0, sizeof(h0), cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemsetAsync(wsp<D>(op, S_FG), 0, (size_t)(m + 1) * sizeof(D), s));
        D g0{};
        memcpy(&g0, &nr, sizeof(double));
        TG_CHECK_CUDA(cudaMemcpyAsync(wsp<D>(op, S_FG), &g0, sizeof(D), cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemsetAsync(H, 0, (size_t)(m + 1) * m * sizeof(D), s));
        TG_PROF(P_SCALE, 2.0 * n * sizeof(T), n, k_scale_by<T><<<grid_for(n, 8), kThreads, 0, s>>>(V, n, inv));
        TG_LAUNCH_CHECK();
        int steps = 0;
        const int mm = (int)((cfg.max_mvps - mvps) < m ? (cfg.max_mvps - mvps) : m);
        for (int j = 0; j < mm; ++j) {
            TG_CHECK(arnoldi_step<T>(op, A, A32, V, n, n, j, reinterpret_cast<T *>(H), ldh, s));
            TG_PROF(P_GIVENS, 0, 6.0 * j, launch_givens_step<D>(H, ldh, j, wsp<D>(op, S_FCS), wsp<D>(op, S_FSN), wsp<D>(op, S_FG), gs, s));
            TG_LAUNCH_CHECK();
            TG_CHECK(readback(op, gs, sizeof(GivensState), s));
            GivensState hg;
            memcpy(&hg, op->pin.p, sizeof(hg));
            steps = hg.steps;
            if (hg.done) break;
        }
        mvps += steps;
        TG_PROF(P_GIVENS, 0, 1.0 * m * m, launch_givens_solve<D>(H, ldh, wsp<D>(op, S_FG), wsp<D>(op, S_FY), gs, s));
        TG_PROF(P_GEMV_N, (steps + 2.0) * n * sizeof(T), 2.0 * steps * n, k_gemv_n<T><<<grid_for(n, 8), kThreads, 0, s>>>(V, n, steps, wsp<D>(op, S_FY), 1.0, x, n));
        TG_LAUNCH_CHECK();
        TG_CHECK(true_residual<T>(op, A, b, x, r, &nr, &nb, s));
        if (!std::isfinite(nr)) { status = TG_NAN; break; }
        if (nr <= cfg.rtol * nb) { status = TG_OK; break; }
    }
    if (st) {
        st->mvps = mvps;
        st->cycles = cyc;
        st->relres = nb > 0 ? nr / nb : 0.0;
        st->status = status;
    }
    return status;
}

}  // namespace tg

extern "C" int tg_solve_proj(tg_op *op, const tg_defl *defl, int method, int precision, const void *b, void *x,
                             int nrhs, double rtol, int ncyc, int restart_mvps, int m3, int64_t max_mvps,
                             tg_stats *stats, void *stream) {
    TG_ARG(op && b && x, "NULL argument");
    TG_ARG(nrhs >= 1, "nrhs must be >= 1");
    TG_ARG(method == TG_BICGSTAB || method == TG_GMRES, "bad method");
    TG_ARG(precision == TG_F64 || precision == TG_F32_IR, "bad precision");
    TG_ARG(!(op->cplx_ && precision == TG_F32_IR), "the lattice path is complex128 only");
    TG_ARG(!(method == TG_GMRES && precision == TG_F32_IR), "GMRES-Proj runs in float64");
    TG_ARG(rtol > 0 && rtol < 1, "rtol must be in (0, 1)");
    TG_ARG(ncyc >= 0 && restart_mvps >= 0, "ncyc and restart_mvps must be >= 0");
    TG_ARG(ncyc > 0 || restart_mvps > 0 || method == TG_GMRES, "fixed-length restarting needs restart_mvps > 0");
    TG_ARG(method != TG_GMRES || (m3 >= 1 && m3 <= kMaxM), "m3 must be in 1..%d", kMaxM);
    TG_ARG(max_mvps > 0, "max_mvps must be > 0");
    TG_ARG(!defl || (defl->n == op->n && !defl->transposed), "deflation handle does not match this operator");
    TG_ARG(!defl || precision == TG_F64 || defl->precision == TG_F32_IR,
           "the deflation handle was built without float32 copies (precision TG_F64)");
    cudaStream_t s = (cudaStream_t)stream;
    SolveCfg cfg{rtol, ncyc, restart_mvps, m3, max_mvps};
    int worst = TG_OK;
    const size_t es = elem_size(op);
    for (int c = 0; c < nrhs; ++c) {
        tg_stats *st = stats ? stats + c : nullptr;
        if (st) {
            st->history_len = 0;
            st->coarse_mvps = 0;
        }
        const char *bc = (const char *)b + (size_t)c * op->n * es;
        char *xc = (char *)x + (size_t)c * op->n * es;
        int rc;
        if (method == TG_GMRES) {
            rc = op->cplx_ ? solve_gmres64<cplx>(op, 0, defl, (const cplx *)bc, (cplx *)xc, cfg, st, s)
                           : solve_gmres64<double>(op, 0, defl, (const double *)bc, (double *)xc, cfg, st, s);
        } else if (precision == TG_F32_IR) {
            rc = solve_bicg_ir(op, 0, defl, (const double *)bc, (double *)xc, cfg, st, s);
        } else {
            rc = op->cplx_ ? solve_bicg64<cplx>(op, 0, defl, (const cplx *)bc, (cplx *)xc, cfg, st, s)
                           : solve_bicg64<double>(op, 0, defl, (const double *)bc, (double *)xc, cfg, st, s);
        }
        if (rc != TG_OK && worst == TG_OK) worst = rc;
        if (rc == TG_CUDA_ERROR || rc == TG_OOM || rc == TG_BAD_ARG) return rc;
    }
    return worst;
}

extern "C" int tg_solve_idr(tg_op *op, const tg_defl *defl, int precision, const void *b, void *x, int nrhs,
                            double rtol, int ncyc, int restart_mvps, int s, const void *P, double kappa,
                            int64_t max_mvps, tg_stats *stats, void *stream) {
    TG_ARG(op && b && x && P, "NULL argument");
    TG_ARG(nrhs >= 1, "nrhs must be >= 1");
    TG_ARG(precision == TG_F64 || precision == TG_F32_IR, "bad precision");
    TG_ARG(!(op->cplx_ && precision == TG_F32_IR), "the lattice path is complex128 only");
    TG_ARG(!defl || precision == TG_F64 || defl->precision == TG_F32_IR,
           "the deflation handle was built without float32 copies (precision TG_F64)");
    TG_ARG(s >= 1 && s <= kIdrMaxS, "s must be in 1..%d (got %d)", kIdrMaxS, s);
    TG_ARG(s < op->n, "s must be smaller than the problem size");
    TG_ARG(rtol > 0 && rtol < 1, "rtol must be in (0, 1)");
    TG_ARG(ncyc >= 0 && restart_mvps >= 0, "ncyc and restart_mvps must be >= 0");
    TG_ARG(ncyc > 0 || restart_mvps > 0, "fixed-length restarting needs restart_mvps > 0");
    TG_ARG(kappa >= 0 && kappa < 1, "kappa must be in [0, 1)");
    TG_ARG(max_mvps > 0, "max_mvps must be > 0");
    TG_ARG(!defl || (defl->n == op->n && !defl->transposed), "deflation handle does not match this operator");
    cudaStream_t st = (cudaStream_t)stream;
    SolveCfg cfg{rtol, ncyc, restart_mvps, 0, max_mvps};
    IdrCfg ic{s, kappa, P};
    int worst = TG_OK;
    const size_t es = elem_size(op);
    for (int c = 0; c < nrhs; ++c) {
        tg_stats *sp = stats ? stats + c : nullptr;
        if (sp) {
            sp->history_len = 0;
            sp->coarse_mvps = 0;
        }
        const char *bc = (const char *)b + (size_t)c * op->n * es;
        char *xc = (char *)x + (size_t)c * op->n * es;
        const int rc = op->cplx_ ? solve_idr64<cplx>(op, defl, (const cplx *)bc, (cplx *)xc, cfg, ic, sp, st)
                       : precision == TG_F32_IR ? solve_idr_ir(op, defl, (const double *)bc, (double *)xc, cfg, ic, sp, st)
                                                : solve_idr64<double>(op, defl, (const double *)bc, (double *)xc, cfg, ic, sp, st);
        if (rc != TG_OK && worst == TG_OK) worst = rc;
        if (rc == TG_CUDA_ERROR || rc == TG_OOM || rc == TG_BAD_ARG) return rc;
    }
    return worst;
}

// ============================================================================= GMRES-DR
namespace tg {

// One GMRES-DR cycle after the restart recombination: Arnoldi from column j0 to m, the
// restart kernel (least squares, harmonic Ritz pairs, P_{k+1}, Hnew, cnew) and x_c += V_m d.
// With per-launch profiling off, the cycle is captured once as a CUDA graph per (basis
// buffer, Hessenberg buffer, j0) and replayed: about 10 (m - j0) launches become one.
template <class T, class HT = T>
static int gdr_cycle(tg_op *op, const DevOp &A, const DevOp32 &A32, T *V, size_t ldv, int nc, int j0, int m, HT *H,
                     int ldh, HT *H2, const GdrArgs<HT> &a, T *xc, int transpose, cudaStream_t s) {
    using D = typename ST<T>::D;
    const cudaStream_t s_caller = s;
    // the cycle's launches, queued on stream s (the caller's, or the capture stream)
    auto body = [&](cudaStream_t s) -> int {
        for (int j = j0; j < m; ++j) TG_CHECK((arnoldi_step<T, HT>(op, A, A32, V, ldv, nc, j, H, ldh, s)));
        TG_CHECK_CUDA(cudaMemsetAsync(H2, 0, (size_t)ldh * m * sizeof(HT), s));
        cudaError_t le = cudaSuccess;
        TG_PROF(P_GDR_RESTART, 0, 30.0 * m * m * m, le = launch_gmresdr_restart<HT>(a, s));
        if (le != cudaSuccess) return cuda_status(le, "launching k_gmresdr_restart (shared-memory limit or launch)");
        // x_c += V_m d
        TG_PROF(P_GEMV_N, (m + 2.0) * nc * sizeof(T), 2.0 * m * nc,
                k_gemv_n<T><<<grid_for(nc, 8), kThreads, 0, s>>>(V, ldv, m, a.d, 1.0, xc, nc));
        TG_LAUNCH_CHECK();
        return TG_OK;
    };
    if (g_prof.on) return body(s_caller);
    // the reduction scratch the Arnoldi steps use, at its largest, before any capture: a
    // capture may not allocate
    const int gb = (int)std::min<int64_t>((nc + 127) / 128, (int64_t)num_sms() * 8);
    TG_CHECK(red_ready(op, (size_t)std::max(gb, 1) * (m + 2) * sizeof(D), s));
    // entries of older workspace generations refer to freed buffers: drop them
    for (auto &g : op->graphs)
        if (g.gen != op->ws_gen && g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
    op->graphs.erase(std::remove_if(op->graphs.begin(), op->graphs.end(),
                                    [op](const GdrGraph &g) { return g.gen != op->ws_gen; }),
                     op->graphs.end());
    GdrGraph *hit = nullptr;
    for (auto &g : op->graphs)
        if (g.V == V && g.H == H && g.j0 == j0 && g.m == m && g.k == a.k && g.nev == a.nev && g.rtolev == a.rtolev &&
            g.transpose == transpose && g.esz == (int)sizeof(T)) {
            hit = &g;
            break;
        }
    if (!hit) {
        // first use of this cycle shape: run it directly (this also makes every one-time
        // driver call, such as shared memory limits, outside any capture); capture on reuse
        GdrGraph ent;
        ent.V = V; ent.H = H; ent.j0 = j0; ent.m = m; ent.k = a.k; ent.nev = a.nev; ent.rtolev = a.rtolev;
        ent.transpose = transpose; ent.esz = (int)sizeof(T); ent.gen = op->ws_gen;
        // a bounded cache: an operator reused with many (k, nev, rtolev) settings drops its
        // oldest shapes first
        constexpr size_t kMaxGraphs = 16;
        if (op->graphs.size() >= kMaxGraphs) {
            if (op->graphs.front().exec) cudaGraphExecDestroy(op->graphs.front().exec);
            op->graphs.erase(op->graphs.begin());
        }
        op->graphs.push_back(ent);
        return body(s_caller);
    }
    if (!hit->exec) {
        if (!op->cap_stream) TG_CHECK_CUDA(cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking));
        const unsigned gen0 = op->ws_gen;
        cudaGraph_t graph = nullptr;
        TG_CHECK_CUDA(cudaStreamBeginCapture(op->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = body(op->cap_stream);
        const cudaError_t e = cudaStreamEndCapture(op->cap_stream, &graph);
        if (rc != TG_OK || e != cudaSuccess || op->ws_gen != gen0) {
            if (graph) cudaGraphDestroy(graph);
            if (rc != TG_OK) return rc;
            if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
            set_error("a workspace buffer was reallocated during a graph capture");
            return TG_BAD_ARG;
        }
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        long long nkern = 0;
        if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
            for (size_t q = 0; q < nn; ++q) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nkern;
            }
        const cudaError_t ei = cudaGraphInstantiate(&hit->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            hit->exec = nullptr;
            return cuda_status(ei, "cudaGraphInstantiate");
        }
        hit->nkern = nkern;
        // the capture counted launches that did not run; the replays count them
        __atomic_sub_fetch(&g_prof.launches, nkern, __ATOMIC_RELAXED);
    }
    TG_CHECK_CUDA(cudaGraphLaunch(hit->exec, s_caller));
    __atomic_add_fetch(&g_prof.launches, hit->nkern, __ATOMIC_RELAXED);
    return TG_OK;
}

// Coarse GMRES-DR(m, k).  T is the basis type (the Arnoldi vectors, operator products and
// orthogonalisation), HT the type of the Hessenberg matrix and the small dense restart step
// (least squares, harmonic Ritz pairs, recombination matrices) and of the outputs: T = HT
// (float64 or complex128), or T = float, HT = double for the float32 + refinement form.
template <class T, class HT = T>
static int gmresdr_impl(tg_op *op, int transpose, const void *b_fine, int m, int k, int nev, double rtolev,
                        double rtol, int max_cycles, void *xc_out, tg_defl **defl_out, int proj, int precision,
                        tg_stats *stats, cudaStream_t s, tg_defl *reuse = nullptr) {
    constexpr bool kMixed = !std::is_same<T, HT>::value;
    const DevOp &A = pick(op, TG_COARSE, transpose);
    const DevOp32 &A32 = pick32(op, TG_COARSE, transpose);
    const int nc = op->nc;
    const int ldh = m + 1;
    const size_t es = sizeof(T), hs = sizeof(HT);
    // basis leading dimension rounded up to whole pipeline chunks (64 float64 / 128 float32
    // rows, 512 bytes): every column starts 16-byte aligned and whole chunks stay inside the
    // allocation (pipelined V^H w).  Rounding a float64 basis to 128 rows instead made
    // the 255^3 column stride a multiple of 4 KiB and V^H w 15% slower.
    const size_t rows_chunk = sizeof(T) == 4 ? 128 : 64;
    const size_t ldv = ((size_t)nc + rows_chunk - 1) / rows_chunk * rows_chunk;
    TG_CHECK(wsx(op, S_GV, ldv * (m + 1) * es));
    TG_CHECK(wsx(op, S_GV2, ldv * (m + 1) * es));
    TG_CHECK(wsx(op, S_GH, (size_t)ldh * m * hs));
    TG_CHECK(wsx(op, S_GH2, (size_t)ldh * m * hs));
    TG_CHECK(wsx(op, S_GC, (size_t)(m + 1) * hs));
    TG_CHECK(wsx(op, S_GX, (size_t)nc * es));
    TG_CHECK(wsx(op, S_GD, (size_t)(m + 1) * hs));
    TG_CHECK(wsx(op, S_GRES, (size_t)(m + 1) * hs));
    TG_CHECK(wsx(op, S_GZ, (size_t)(m + 1) * hs));
    TG_CHECK(wsx(op, S_GP, (size_t)(m + 1) * (m + 2) * hs));
    TG_CHECK(wsx(op, S_GCN, (size_t)(m + 2) * hs));
    TG_CHECK(wsx(op, S_GTHETA, (size_t)2 * m * 8));
    TG_CHECK(wsx(op, S_GWR, (size_t)m * 8));
    TG_CHECK(wsx(op, S_GWI, (size_t)m * 8));
    TG_CHECK(wsx(op, S_GORD, (size_t)m * 4));
    TG_CHECK(wsx(op, S_GERES, (size_t)m * 8));
    TG_CHECK(wsx(op, S_GWORK, ((size_t)(m + 1) * m + 2 * (size_t)m * m + 3 * (size_t)m + 4) * hs));
    TG_CHECK(wsx(op, S_GY, (size_t)m * m * 16));
    TG_CHECK(wsx(op, S_GG, (size_t)m * m * 16));
    TG_CHECK(wsx(op, S_GINFO, sizeof(GdrInfo)));
    TG_CHECK(wsx(op, S_GB, (size_t)nc * hs));
    TG_CHECK(wsx(op, S_GTMP, (size_t)(m + 2) * hs));
    T *V = wsp<T>(op, S_GV), *V2 = wsp<T>(op, S_GV2);
    HT *H = wsp<HT>(op, S_GH), *H2 = wsp<HT>(op, S_GH2);
    HT *c = wsp<HT>(op, S_GC), *bc = wsp<HT>(op, S_GB);
    T *xc = wsp<T>(op, S_GX);
    // b_c = restrict(b); v_0 = b_c / ||b_c||; x_c = 0
    TG_CHECK(restrict_impl(op, b_fine, bc, 1, s));
    double nbc2;
    TG_CHECK(dot_host<HT>(op, bc, nullptr, nc, &nbc2, nullptr, s));
    const double nbc = sqrt(nbc2);
    TG_ARG(nbc > 0 && std::isfinite(nbc), "restricted right-hand side is zero or not finite");
    if constexpr (kMixed) {
        TG_PROF(P_CONVERT, 12.0 * nc, nc, launch_d2f_scaled(grid_for(nc, 8), s, bc, V, nc, 1.0 / nbc));
        TG_LAUNCH_CHECK();
    } else {
        TG_CHECK_CUDA(cudaMemcpyAsync(V, bc, (size_t)nc * es, cudaMemcpyDeviceToDevice, s));
        double *inv = reinterpret_cast<double *>(wsp<char>(op, S_SMALL) + SmallArea::gmres_inv);
        double hinv = 1.0 / nbc;
        TG_CHECK_CUDA(cudaMemcpyAsync(inv, &hinv, sizeof(double), cudaMemcpyHostToDevice, s));
        TG_PROF(P_SCALE, 2.0 * nc * sizeof(T), nc, k_scale_by<T><<<grid_for(nc, 8), kThreads, 0, s>>>(V, nc, inv));
    }
    TG_CHECK_CUDA(cudaMemsetAsync(xc, 0, (size_t)nc * es, s));
    TG_CHECK_CUDA(cudaMemsetAsync(H, 0, (size_t)ldh * m * hs, s));
    TG_CHECK_CUDA(cudaMemsetAsync(c, 0, (size_t)(m + 1) * hs, s));
    HT c0{};
    memcpy(&c0, &nbc, sizeof(double));
    TG_CHECK_CUDA(cudaMemcpyAsync(c, &c0, sizeof(HT), cudaMemcpyHostToDevice, s));
    int j0 = 0;
    int cycles = 0;
    int64_t cmvps = 0;
    GdrInfo info{};
    int kk = k;
    bool converged = false;
    while (true) {
        ++cycles;
        GdrArgs<HT> a;
        a.H = H; a.ldh = ldh; a.c = c; a.m = m; a.k = k; a.nev = nev; a.rtolev = rtolev;
        a.d = wsp<HT>(op, S_GD); a.res = wsp<HT>(op, S_GRES); a.z = wsp<HT>(op, S_GZ);
        a.theta = wsp<double>(op, S_GTHETA); a.wr = wsp<double>(op, S_GWR); a.wi = wsp<double>(op, S_GWI);
        a.order = wsp<int>(op, S_GORD); a.eres = wsp<double>(op, S_GERES); a.P = wsp<HT>(op, S_GP);
        a.Hnew = H2; a.cnew = wsp<HT>(op, S_GCN); a.work = wsp<HT>(op, S_GWORK);
        a.ywork = wsp<cplx>(op, S_GY); a.gwork = wsp<cplx>(op, S_GG); a.info = wsp<GdrInfo>(op, S_GINFO);
        TG_CHECK((gdr_cycle<T, HT>(op, A, A32, V, ldv, nc, j0, m, H, ldh, H2, a, xc, transpose, s)));
        cmvps += m - j0;
        TG_CHECK(readback(op, a.info, sizeof(GdrInfo), s));
        memcpy(&info, op->pin.p, sizeof(info));
        if (g_prof.on)
            for (int q = 0; q < 8; ++q) g_prof.gdr_phase[q] += info.phase[q];
        kk = info.kk;
        if (info.status != 0) {
            set_error("harmonic Ritz QR iteration did not converge");
            return TG_NOT_CONVERGED;
        }
        if (!std::isfinite(info.rnorm)) return TG_NAN;
        converged = info.rnorm <= rtol * nbc && info.nconv >= (nev < kk ? nev : kk);
        if (converged || cycles >= max_cycles) break;
        // restart: V_{k+1} = V_{m+1} P_{k+1}; Hbar = Hnew; c = cnew
        if constexpr (kMixed) TG_CHECK(tsm_f<float>(V, ldv, m + 1, a.P, m + 1, kk + 1, V2, ldv, nc, s));
        else TG_CHECK(tsm<T>(V, ldv, m + 1, a.P, m + 1, kk + 1, V2, ldv, nc, s));
        std::swap(V, V2);
        std::swap(H, H2);
        TG_CHECK_CUDA(cudaMemsetAsync(c, 0, (size_t)(m + 1) * hs, s));
        TG_CHECK_CUDA(cudaMemcpyAsync(c, a.cnew, (size_t)(kk + 1) * hs, cudaMemcpyDeviceToDevice, s));
        // re-orthogonalise v_{k+1} against V_k and normalise
        {
            using DD = typename ST<T>::D;
            T *w = V + (size_t)kk * ldv;
            DD *h1 = reinterpret_cast<DD *>(wsp<char>(op, S_SMALL) + SmallArea::arn_h1);
            DD *nrm = reinterpret_cast<DD *>(wsp<char>(op, S_SMALL) + SmallArea::arn_nrm);
            TG_CHECK(gemv_t<T>(op, V, ldv, kk, w, nc, h1, s));
            TG_PROF(P_GEMV_N, (kk + 2.0) * nc * sizeof(T), 2.0 * kk * nc, k_gemv_n<T><<<grid_for(nc, 8), kThreads, 0, s>>>(V, ldv, kk, h1, -1.0, w, nc));
            TG_PROF(P_DOT, 1.0 * nc * sizeof(T), 2.0 * nc, k_dot<T><<<grid_for(nc, 4), kThreads, 0, s>>>(w, nullptr, nc, wsp<DD>(op, S_PART), wsp<unsigned>(op, S_TICKET), nrm));
            TG_PROF(P_SMALL, 0, 1, launch_inv_sqrt(s, reinterpret_cast<const double *>(nrm), reinterpret_cast<double *>(nrm) + 4));
            TG_PROF(P_SCALE, 2.0 * nc * sizeof(T), nc, k_scale_by<T><<<grid_for(nc, 8), kThreads, 0, s>>>(w, nc, reinterpret_cast<double *>(nrm) + 4));
            TG_LAUNCH_CHECK();
        }
        j0 = kk;
    }
    // the V_m P_k basis of the final cycle, prolonged; x_c out
    if (stats) {
        stats->coarse_mvps = cmvps;
        stats->cycles = cycles;
        stats->coarse_relres = info.rnorm / nbc;
        stats->kk = kk;
        stats->eig_converged = info.nconv;
        stats->status = converged ? TG_OK : TG_NOT_CONVERGED;
    }
    if (xc_out) {
        if constexpr (kMixed) {
            TG_CHECK_CUDA(cudaMemsetAsync(xc_out, 0, (size_t)nc * hs, s));
            TG_PROF(P_CONVERT, 12.0 * nc, nc, launch_add_f2d_scaled(grid_for(nc, 8), s, (double *)xc_out, xc, nc, 1.0));
            TG_LAUNCH_CHECK();
        } else {
            TG_CHECK_CUDA(cudaMemcpyAsync(xc_out, xc, (size_t)nc * es, cudaMemcpyDeviceToDevice, s));
        }
    }
    if (defl_out) {
        TG_CHECK(wsx(op, S_GYC, (size_t)nc * kk * hs));
        DBuf &Yc = op->ws[S_GYC];
        if constexpr (kMixed) TG_CHECK(tsm_f<double>(V, ldv, m, wsp<HT>(op, S_GP), m + 1, kk, Yc.as<double>(), nc, nc, s));
        else TG_CHECK(tsm<T>(V, ldv, m, wsp<T>(op, S_GP), m + 1, kk, Yc.as<T>(), nc, nc, s));
        tg_defl *d = reuse;
        if (d) {
            // rebuild in the caller's handle: its buffers grow only when needed
            d->kk = kk; d->n = op->n; d->proj = proj; d->precision = precision; d->cplx_ = op->cplx_;
            d->transposed = transpose != 0;
            TG_CHECK(d->Y.ensure((size_t)op->n * kk * hs));
        } else {
            TG_CHECK(defl_create(op, transpose, kk, proj, precision, &d));
        }
        int rc = prolong_impl(op, Yc.p, d->Y.p, kk, s);
        if (!rc) rc = build_defl<HT>(op, transpose, d, s);
        if (rc) {
            if (!reuse) delete d;
            return rc;
        }
        *defl_out = d;
    }
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    return converged ? TG_OK : TG_NOT_CONVERGED;
}

}  // namespace tg

extern "C" int tg_coarse_gmresdr(tg_op *op, int transpose, const void *b_fine, int m, int k, int nev, double rtolev,
                                 double rtol, int max_cycles, void *xc_out, tg_defl **defl_out, int proj,
                                 int precision, tg_stats *stats, void *stream) {
    TG_ARG(op && b_fine, "NULL argument");
    TG_ARG(m >= 2 && m <= kMaxM && k >= 1 && k < m - 1, "need 1 <= k < m - 1 and m <= %d (m=%d, k=%d)", kMaxM, m, k);
    TG_ARG(m < op->nc, "m must be smaller than the coarse problem size");
    TG_ARG(nev >= 0 && nev <= k, "nev must be in 0..k");
    TG_ARG(max_cycles >= 1, "max_cycles must be >= 1");
    TG_ARG(proj == TG_PROJ_MINRES || proj == TG_PROJ_GALERKIN, "bad projection kind");
    TG_ARG(precision == TG_F64 || precision == TG_F32_IR, "bad precision");
    TG_ARG(!(op->cplx_ && precision == TG_F32_IR), "the lattice path is complex128 only");
    if (defl_out) *defl_out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (op->cplx_)
        return gmresdr_impl<cplx>(op, transpose, b_fine, m, k, nev, rtolev, rtol, max_cycles, xc_out, defl_out, proj,
                                  precision, stats, s);
    if (precision == TG_F32_IR)
        return gmresdr_impl<float, double>(op, transpose, b_fine, m, k, nev, rtolev, rtol, max_cycles, xc_out, defl_out,
                                           proj, precision, stats, s);
    return gmresdr_impl<double>(op, transpose, b_fine, m, k, nev, rtolev, rtol, max_cycles, xc_out, defl_out, proj,
                                precision, stats, s);
}

// ============================================================================= adjoint
// ============================================================================= Arnoldi-E
namespace tg {

// Orthogonalises column j of V (leading dimension ldv) against columns 0..j-1 by classical
// Gram-Schmidt applied twice and normalises it; *kept = false (and nothing normalised) when
// less than drop_rel of its norm survives, i.e. the column lies in the span of the others.
template <class T>
static int cgs2_column(tg_op *op, T *V, size_t ldv, int n, int j, double drop_rel, bool *kept, cudaStream_t s) {
    using D = typename ST<T>::D;
    T *w = V + (size_t)j * ldv;
    TG_CHECK(red_ready(op, (size_t)num_sms() * 8 * (j + 2) * sizeof(D), s));
    char *sm = wsp<char>(op, S_SMALL);
    D *h1 = reinterpret_cast<D *>(sm + SmallArea::arn_h1);
    D *h2 = reinterpret_cast<D *>(sm + SmallArea::arn_h2);
    double *nrm = reinterpret_cast<double *>(sm + SmallArea::arn_nrm);
    double *inv = nrm + 4;
    D *part = wsp<D>(op, S_PART);
    unsigned *tk = wsp<unsigned>(op, S_TICKET);
    const int g = grid_for(n, 8);
    double before = 0.0, after = 0.0;
    if (j == 0) {
        TG_CHECK(dot_host<T>(op, w, nullptr, n, &before, nullptr, s));
        after = before;
        TG_CHECK_CUDA(cudaMemcpyAsync(nrm, &after, sizeof(double), cudaMemcpyHostToDevice, s));
    } else {
        bool piped = false;
        int gbt = 1;
        TG_PROF(P_GEMV_T, (double)(j + 1) * n * sizeof(T), 2.0 * (j + 1) * n, gbt = gemv_t_part_launch<T>(V, ldv, j + 1, w, n, part, s, &piped));
        TG_PROF(P_SUM_PART, 0, 0, k_sum_part<D><<<(j + 1 + 7) / 8, 256, 0, s>>>(part, gbt, j + 1, h1, 0));
        TG_PROF(P_GEMV_N, (j + 2.0) * n * sizeof(T), 2.0 * j * n,
                gemv_n_norm_launch<T>(g, V, ldv, j, h1, w, n, part, tk, nrm, nullptr, nullptr, 0.0, s));
        TG_PROF(P_GEMV_T, (double)(j + 1) * n * sizeof(T), 2.0 * j * n, gbt = gemv_t_part_launch<T>(V, ldv, j, w, n, part, s, &piped));
        TG_PROF(P_SUM_PART, 0, 0, k_sum_part<D><<<(j + 7) / 8, 256, 0, s>>>(part, gbt, j, h2, 0));
        TG_PROF(P_GEMV_N, (j + 2.0) * n * sizeof(T), 2.0 * j * n,
                gemv_n_norm_launch<T>(g, V, ldv, j, h2, w, n, part, tk, nrm, nullptr, nullptr, 0.0, s));
        TG_LAUNCH_CHECK();
        TG_CHECK(readback(op, h1 + j, sizeof(D), s));
        D hb;
        memcpy(&hb, op->pin.p, sizeof(D));
        before = dnorm2(hb);
        TG_CHECK(readback(op, nrm, sizeof(double), s));
        memcpy(&after, op->pin.p, sizeof(double));
    }
    *kept = after > drop_rel * drop_rel * before && after > 0.0;
    if (*kept) {
        TG_PROF(P_SMALL, 0, 1, launch_inv_sqrt(s, nrm, inv));
        TG_PROF(P_SCALE, 2.0 * n * sizeof(T), n, k_scale_by<T><<<g, kThreads, 0, s>>>(w, n, inv));
        TG_LAUNCH_CHECK();
    }
    return TG_OK;
}

// Rayleigh-Ritz on span(S) (cols orthonormal columns, leading dimension ld) with W = A S:
// H = S^H W, WW = W^H W, the small dense kernel in Rayleigh-Ritz mode (ordered Ritz pairs,
// k kept, k + 1 if a pair would split); then Y = S P_k and u = S z (Ritz vector start_q).
// Rayleigh-Ritz matrices of an Arnoldi-E cycle whose first p + 1 basis columns K are an
// Arnoldi basis (A K[:, :p] = K Ha, Ha (p+1) x p upper Hessenberg, ld p+1) and whose other
// columns are orthogonal to K: with W_R = A S[:, p:] (q = cols - p columns), HR = S^H W_R
// (cols x q) and WWR = W_R^H W_R (q x q), the cycle's matrices are
//   H  = S^H A S:       columns j < p are [Ha[:, j]; 0], columns p.. are HR;
//   WW = (A S)^H (A S): [[Ha^H Ha, Ha^H HR[:p+1, :]], [HR[:p+1, :]^H Ha, WWR]],
// so A is applied, and the long Gram products run, on the q columns of W_R only.
template <class T>
__global__ void k_ae_assemble(const T *__restrict__ Ha, int p, const T *__restrict__ HR,
                              const T *__restrict__ WWR, int cols, T *__restrict__ H, T *__restrict__ WW) {
    const int q = cols - p, ldh = p + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cols * cols; e += gridDim.x * blockDim.x) {
        const int i = e % cols, j = e / cols;
        T h = ST<T>::zero();
        if (j >= p) h = HR[i + (size_t)(j - p) * cols];
        else if (i <= j + 1) h = Ha[i + (size_t)j * ldh];
        H[e] = h;
        T w = ST<T>::zero();
        if (i < p && j < p) {
            const int lmax = (i < j ? i : j) + 1;          // Ha[l, c] = 0 for l > c + 1
            for (int l = 0; l <= lmax; ++l) w = w + dconj(Ha[l + (size_t)i * ldh]) * Ha[l + (size_t)j * ldh];
        } else if (i < p) {
            for (int l = 0; l <= i + 1; ++l) w = w + dconj(Ha[l + (size_t)i * ldh]) * HR[l + (size_t)(j - p) * cols];
        } else if (j < p) {
            for (int l = 0; l <= j + 1; ++l) w = w + dconj(HR[l + (size_t)(i - p) * cols]) * Ha[l + (size_t)j * ldh];
        } else {
            w = WWR[(i - p) + (size_t)(j - p) * q];
        }
        WW[e] = w;
    }
}

template <class T>
static int rayleigh_ritz(tg_op *op, const T *S, const T *W, size_t ld, int n, int cols, int k, int nev,
                         double rtolev, int start_q, T *Y, T *u, GdrInfo *info_h, cudaStream_t s,
                         const T *Ha = nullptr, int p = 0) {
    using D = typename ST<T>::D;
    const int m = cols;
    TG_CHECK(wsx(op, S_AE_H, (size_t)m * m * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_WW, (size_t)m * m * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_P, (size_t)(m + 1) * (m + 2) * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_Z, (size_t)(m + 1) * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_TH, (size_t)2 * m * 8));
    TG_CHECK(wsx(op, S_AE_WR, (size_t)m * 8));
    TG_CHECK(wsx(op, S_AE_WI, (size_t)m * 8));
    TG_CHECK(wsx(op, S_AE_ORD, (size_t)m * 4));
    TG_CHECK(wsx(op, S_AE_ERES, (size_t)m * 8));
    TG_CHECK(wsx(op, S_AE_WORK, ((size_t)(m + 1) * m + 2 * (size_t)m * m + 3 * (size_t)m + 4) * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_YW, (size_t)m * m * 16));
    TG_CHECK(wsx(op, S_AE_GW, (size_t)m * m * 16));
    TG_CHECK(wsx(op, S_AE_INFO, sizeof(GdrInfo)));
    TG_CHECK(wsx(op, S_AE_DUM, (size_t)(m + 2) * (m + 2) * sizeof(T)));
    T *H = wsp<T>(op, S_AE_H), *WW = wsp<T>(op, S_AE_WW);
    if (p > 0) {
        const int q = m - p;
        TG_CHECK(wsx(op, S_AE_HR, (size_t)m * q * sizeof(T)));
        TG_CHECK(wsx(op, S_AE_WWR, (size_t)q * q * sizeof(T)));
        T *HR = wsp<T>(op, S_AE_HR), *WWR = wsp<T>(op, S_AE_WWR);
        const T *WR = W + (size_t)p * ld;
        TG_CHECK(gram<T>(op, S, WR, ld, m, n, 0, reinterpret_cast<D *>(HR), s, q));
        TG_CHECK(gram<T>(op, WR, WR, ld, q, n, 1, reinterpret_cast<D *>(WWR), s));
        TG_PROF(P_SMALL, 0, 0, k_ae_assemble<T><<<(m * m + 255) / 256, 256, 0, s>>>(Ha, p, HR, WWR, m, H, WW));
        TG_LAUNCH_CHECK();
    } else {
        TG_CHECK(gram<T>(op, S, W, ld, m, n, 0, reinterpret_cast<D *>(H), s));
        TG_CHECK(gram<T>(op, W, W, ld, m, n, 1, reinterpret_cast<D *>(WW), s));
    }
    GdrArgs<T> a;
    T *dum = wsp<T>(op, S_AE_DUM);
    a.H = H; a.ldh = m; a.c = dum; a.m = m; a.k = k; a.nev = nev; a.rtolev = rtolev;
    a.d = dum; a.res = dum; a.z = wsp<T>(op, S_AE_Z);
    a.theta = wsp<double>(op, S_AE_TH); a.wr = wsp<double>(op, S_AE_WR); a.wi = wsp<double>(op, S_AE_WI);
    a.order = wsp<int>(op, S_AE_ORD); a.eres = wsp<double>(op, S_AE_ERES); a.P = wsp<T>(op, S_AE_P);
    a.Hnew = dum; a.cnew = dum; a.work = wsp<T>(op, S_AE_WORK); a.ywork = wsp<cplx>(op, S_AE_YW);
    a.gwork = wsp<cplx>(op, S_AE_GW); a.info = wsp<GdrInfo>(op, S_AE_INFO);
    a.mode = 1;
    a.WW = WW;
    a.start_q = start_q;
    cudaError_t le = cudaSuccess;
    TG_PROF(P_GDR_RESTART, 0, 30.0 * m * m * m, le = launch_gmresdr_restart<T>(a, s));
    if (le != cudaSuccess) return cuda_status(le, "launching the Rayleigh-Ritz step");
    TG_CHECK(readback(op, a.info, sizeof(GdrInfo), s));
    memcpy(info_h, op->pin.p, sizeof(GdrInfo));
    if (info_h->status) {
        set_error("Rayleigh-Ritz: the QR iteration did not converge");
        return TG_NOT_CONVERGED;
    }
    const int kk = info_h->kk;
    TG_CHECK(tsm<T>(S, ld, m, a.P, m + 1, kk, Y, ld, n, s));
    TG_CHECK(tsm<T>(S, ld, m, a.z, m, 1, u, ld, n, s));
    return TG_OK;
}

// Arnoldi-E improvement of a deflation basis on the fine grid (see tg_improve_defl).
template <class T>
static int improve_impl(tg_op *op, tg_defl *d, int m, int cycles, int nstart, int nev, double rtolev,
                        double *theta_out, tg_stats *st, cudaStream_t s) {
    const DevOp &A = pick(op, TG_FINE, d->transposed ? 1 : 0);
    const DevOp32 &A32 = pick32(op, TG_FINE, d->transposed ? 1 : 0);
    const int n = op->n, k = d->kk, p = m - k;
    const size_t ld = ((size_t)n + 63) / 64 * 64;     // whole 64-row chunks: the pipelined V^H w applies
    TG_CHECK(wsx(op, S_AE_S, ld * (m + 2) * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_W, ld * (m + 2) * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_HA, (size_t)(p + 1) * p * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_Y, ld * (k + 2) * sizeof(T)));
    TG_CHECK(wsx(op, S_AE_U, ld * sizeof(T)));
    T *S = wsp<T>(op, S_AE_S), *W = wsp<T>(op, S_AE_W), *Ha = wsp<T>(op, S_AE_HA);
    T *Y = wsp<T>(op, S_AE_Y), *u = wsp<T>(op, S_AE_U);
    TG_CHECK_CUDA(cudaMemsetAsync(S, 0, ld * (m + 2) * sizeof(T), s));
    int64_t mvps = 0;
    GdrInfo info{};
    // Rayleigh-Ritz on span(Y) orders the given vectors as Ritz vectors
    int cols = 0;
    for (int c = 0; c < k; ++c) {
        TG_CHECK_CUDA(cudaMemcpyAsync(S + (size_t)cols * ld, d->Y.as<T>() + (size_t)c * n, (size_t)n * sizeof(T),
                                      cudaMemcpyDeviceToDevice, s));
        bool kept = false;
        TG_CHECK(cgs2_column<T>(op, S, ld, n, cols, 1e-10, &kept, s));
        if (kept) ++cols;
    }
    TG_ARG(cols == k, "the deflation basis is numerically rank deficient");
    for (int c = 0; c < cols; ++c) TG_CHECK(launch_apply<T>(A, A32, S + (size_t)c * ld, W + (size_t)c * ld, s));
    mvps += cols;
    TG_CHECK(rayleigh_ritz<T>(op, S, W, ld, n, cols, k, nev, rtolev, 0 % nstart, Y, u, &info, s));
    int kk = info.kk, done = 0;
    for (int cyc = 0; cyc < cycles; ++cyc) {
        // Krylov part from u: S[:, 0..p] by Arnoldi (classical Gram-Schmidt twice)
        TG_CHECK_CUDA(cudaMemcpyAsync(S, u, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        bool kept = false;
        TG_CHECK(cgs2_column<T>(op, S, ld, n, 0, 0.0, &kept, s));
        for (int j = 0; j < p; ++j) TG_CHECK((arnoldi_step<T, T>(op, A, A32, S, ld, n, j, Ha, p + 1, s)));
        mvps += p;
        cols = p + 1;
        // then the current approximate eigenvectors (u lies in their span: one drops out)
        for (int c = 0; c < kk && cols < m + 1; ++c) {
            TG_CHECK_CUDA(cudaMemcpyAsync(S + (size_t)cols * ld, Y + (size_t)c * ld, (size_t)n * sizeof(T),
                                          cudaMemcpyDeviceToDevice, s));
            TG_CHECK(cgs2_column<T>(op, S, ld, n, cols, 1e-10, &kept, s));
            if (kept) ++cols;
        }
        // A S[:, :p] = S[:, :p+1] Ha is known from the Arnoldi step: only the last Krylov column
        // and the appended vectors are multiplied
        for (int c = p; c < cols; ++c) TG_CHECK(launch_apply<T>(A, A32, S + (size_t)c * ld, W + (size_t)c * ld, s));
        mvps += cols - p;
        TG_CHECK(rayleigh_ritz<T>(op, S, W, ld, n, cols, k, nev, rtolev, (cyc + 1) % nstart, Y, u, &info, s, Ha, p));
        kk = info.kk;
        done = cyc + 1;
        if (rtolev > 0 && nev > 0 && info.nconv >= nev) break;
    }
    if (theta_out) {
        TG_CHECK(readback(op, wsp<double>(op, S_AE_TH), (size_t)2 * kk * 8, s));
        memcpy(theta_out, op->pin.p, (size_t)2 * kk * 8);
    }
    // the improved basis replaces the handle's and its projection data are rebuilt
    if (kk != d->kk) TG_CHECK(d->Y.ensure((size_t)n * kk * sizeof(T)));
    TG_CHECK_CUDA(cudaMemcpy2DAsync(d->Y.p, (size_t)n * sizeof(T), Y, ld * sizeof(T), (size_t)n * sizeof(T), kk,
                                    cudaMemcpyDeviceToDevice, s));
    d->kk = kk;
    TG_CHECK(build_defl<T>(op, d->transposed ? 1 : 0, d, s));
    mvps += kk;
    if (st) {
        st->cycles = done;
        st->mvps = mvps;
        st->kk = kk;
        st->eig_converged = info.nconv;
        st->status = TG_OK;
    }
    return TG_OK;
}

}  // namespace tg

extern "C" int tg_improve_defl(tg_op *op, tg_defl *defl, int m, int cycles, int nstart, int nev, double rtolev,
                               double *theta_out, tg_stats *stats, void *stream) {
    TG_ARG(op && defl, "NULL argument");
    TG_ARG(defl->n == op->n, "deflation handle does not match this operator");
    TG_ARG(m > defl->kk && m <= kMaxM, "need kk < m <= %d (kk = %d, m = %d)", kMaxM, defl->kk, m);
    TG_ARG(m + 2 <= op->n, "m too large for the problem size");
    TG_ARG(cycles >= 0 && nstart >= 1 && nstart <= defl->kk, "need cycles >= 0 and 1 <= nstart <= kk");
    TG_ARG(nev >= 0 && nev <= defl->kk && rtolev >= 0, "bad nev / rtolev");
    cudaStream_t s = (cudaStream_t)stream;
    return op->cplx_ ? improve_impl<cplx>(op, defl, m, cycles, nstart, nev, rtolev, theta_out, stats, s)
                     : improve_impl<double>(op, defl, m, cycles, nstart, nev, rtolev, theta_out, stats, s);
}

extern "C" int tg_kappa_gradient(const tg_op *op, const void *x, const void *lambda, void *dkappa, void *stream) {
    TG_ARG(op && x && lambda && dkappa, "NULL argument");
    TG_ARG(op->kind == TG_VARK2D, "the kappa gradient needs a TG_VARK2D operator");
    cudaStream_t s = (cudaStream_t)stream;
    const int NP = op->N + 2;
    TG_PROF(P_GRAD, 16.0 * op->n, 8.0 * op->n, launch_kappa_grad(grid_for(NP * NP, 8), s, (const double *)x, (const double *)lambda, op->N,
                                                          (double *)dkappa));
    TG_LAUNCH_CHECK();
    return TG_OK;
}

extern "C" int tg_adjoint_solve(tg_op *op, const tg_defl *defl_left, const void *g, void *lambda, const void *x,
                                void *dkappa, double rtol, int ncyc, int restart_mvps, int precision, tg_stats *stats,
                                void *stream) {
    TG_ARG(op && g && lambda, "NULL argument");
    TG_ARG(!op->cplx_, "the adjoint form is for the real operators");
    TG_ARG(!defl_left || (defl_left->transposed && defl_left->n == op->n), "defl_left must be built with transpose = 1");
    TG_ARG(ncyc > 0 || restart_mvps > 0, "fixed-length restarting needs restart_mvps > 0");
    TG_ARG(precision == TG_F64 || precision == TG_F32_IR, "bad precision");
    TG_ARG(!defl_left || precision == TG_F64 || defl_left->precision == TG_F32_IR, "defl_left lacks float32 copies");
    TG_ARG(!dkappa || x, "the gradient needs x");
    cudaStream_t s = (cudaStream_t)stream;
    SolveCfg cfg{rtol, ncyc, restart_mvps, 0, (int64_t)1 << 40};
    int rc = precision == TG_F32_IR
                 ? solve_bicg_ir(op, 1, defl_left, (const double *)g, (double *)lambda, cfg, stats, s)
                 : solve_bicg64<double>(op, 1, defl_left, (const double *)g, (double *)lambda, cfg, stats, s);
    if (rc != TG_OK) return rc;
    if (dkappa && op->kind == TG_VARK2D) TG_CHECK(tg_kappa_gradient(op, x, lambda, dkappa, stream));
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    return TG_OK;
}

// ============================================================================= test hook
extern "C" int tg_harmonic_ritz(const void *Hbar, int m, int k, int complex_, void *theta_out, void *basis_out,
                                void *eres_out, int *kk_out, void *stream) {
    TG_ARG(Hbar && theta_out && basis_out && kk_out, "NULL argument");
    TG_ARG(m >= 2 && m <= kMaxM && k >= 1 && k < m, "need 1 <= k < m <= %d", kMaxM);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = complex_ ? 16 : 8;
    DBuf c, d, res, z, P, Hn, cn, th, wr, wi, ord, er, work, yw, gw, inf;
    int rc;
    if ((rc = c.ensure((m + 1) * es)) || (rc = d.ensure((m + 1) * es)) || (rc = res.ensure((m + 1) * es)) ||
        (rc = z.ensure((m + 1) * es)) || (rc = P.ensure((size_t)(m + 1) * (m + 2) * es)) ||
        (rc = Hn.ensure((size_t)(m + 1) * m * es)) || (rc = cn.ensure((m + 2) * es)) || (rc = th.ensure(2 * m * 8)) ||
        (rc = wr.ensure(m * 8)) || (rc = wi.ensure(m * 8)) || (rc = ord.ensure(m * 4)) || (rc = er.ensure(m * 8)) ||
        (rc = work.ensure(((size_t)(m + 1) * m + 2 * (size_t)m * m + 3 * m + 4) * es)) ||
        (rc = yw.ensure((size_t)m * m * 16)) || (rc = gw.ensure((size_t)m * m * 16)) || (rc = inf.ensure(sizeof(GdrInfo))))
        return rc;
    TG_CHECK_CUDA(cudaMemsetAsync(c.p, 0, (m + 1) * es, s));
    double one = 1.0;
    TG_CHECK_CUDA(cudaMemcpyAsync(c.p, &one, 8, cudaMemcpyHostToDevice, s));
    auto launch = [&](auto tag) -> int {
        using T = decltype(tag);
        GdrArgs<T> a;
        a.H = (const T *)Hbar; a.ldh = m + 1; a.c = c.as<T>(); a.m = m; a.k = k; a.nev = k; a.rtolev = 0.0;
        a.d = d.as<T>(); a.res = res.as<T>(); a.z = z.as<T>(); a.theta = th.as<double>(); a.wr = wr.as<double>();
        a.wi = wi.as<double>(); a.order = ord.as<int>(); a.eres = er.as<double>(); a.P = P.as<T>(); a.Hnew = Hn.as<T>();
        a.cnew = cn.as<T>(); a.work = work.as<T>(); a.ywork = yw.as<cplx>(); a.gwork = gw.as<cplx>();
        a.info = inf.as<GdrInfo>();
        cudaError_t le = cudaSuccess;
        TG_PROF(P_GDR_RESTART, 0, 30.0 * m * m * m, le = launch_gmresdr_restart<T>(a, s));
        if (le != cudaSuccess) return cuda_status(le, "launching k_gmresdr_restart (shared-memory limit or launch)");
        return TG_OK;
    };
    TG_CHECK(complex_ ? launch(cplx{}) : launch(double{}));
    GdrInfo info;
    TG_CHECK_CUDA(cudaMemcpyAsync(&info, inf.p, sizeof(info), cudaMemcpyDeviceToHost, s));
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    *kk_out = info.kk;
    TG_CHECK_CUDA(cudaMemcpyAsync(theta_out, th.p, 2 * m * 8, cudaMemcpyDefault, s));
    TG_CHECK_CUDA(cudaMemcpy2DAsync(basis_out, m * es, P.p, (m + 1) * es, m * es, info.kk, cudaMemcpyDefault, s));
    if (eres_out) TG_CHECK_CUDA(cudaMemcpyAsync(eres_out, er.p, info.kk * 8, cudaMemcpyDefault, s));
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    return info.status ? TG_NOT_CONVERGED : TG_OK;
}

// ============================================================================= instrumentation ABI
extern "C" int tg_profile_enable(int on) {
    if (on) {
        g_prof.recs.clear();
        g_prof.next = 0;
        for (int q = 0; q < 8; ++q) g_prof.gdr_phase[q] = 0;
        g_prof.recs.reserve(1 << 16);
    }
    g_prof.on = on != 0;
    return TG_OK;
}

extern "C" int tg_profile_read(char *json, int cap) {
    TG_ARG(json && cap > 0, "NULL buffer");
    double ms[P_COUNT] = {0}, bytes[P_COUNT] = {0}, flops[P_COUNT] = {0};
    long long cnt[P_COUNT] = {0};
    for (const ProfRec &r : g_prof.recs) {
        TG_CHECK_CUDA(cudaEventSynchronize(g_prof.events[r.ev + 1]));
        float t = 0.f;
        TG_CHECK_CUDA(cudaEventElapsedTime(&t, g_prof.events[r.ev], g_prof.events[r.ev + 1]));
        ms[r.cls] += t;
        bytes[r.cls] += r.bytes;
        flops[r.cls] += r.flops;
        cnt[r.cls] += 1;
    }
    std::string out = "{";
    bool first = true;
    for (int c = 0; c < P_COUNT; ++c) {
        if (!cnt[c]) continue;
        char buf[256];
        snprintf(buf, sizeof(buf), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"bytes\": %.6e, \"flops\": %.6e}",
                 first ? "" : ", ", kProfName[c], cnt[c], ms[c], bytes[c], flops[c]);
        out += buf;
        first = false;
    }
    {
        char buf[256];
        snprintf(buf, sizeof(buf), "%s\"gmresdr_restart_phase_cycles\": [%lld, %lld, %lld, %lld, %lld, %lld, %lld, %lld]",
                 first ? "" : ", ", g_prof.gdr_phase[0], g_prof.gdr_phase[1], g_prof.gdr_phase[2], g_prof.gdr_phase[3],
                 g_prof.gdr_phase[4], g_prof.gdr_phase[5], g_prof.gdr_phase[6], g_prof.gdr_phase[7]);
        out += buf;
    }
    out += "}";
    if ((int)out.size() + 1 > cap) {
        set_error("profile buffer too small (%d bytes needed)", (int)out.size() + 1);
        return TG_BAD_ARG;
    }
    memcpy(json, out.c_str(), out.size() + 1);
    return TG_OK;
}

extern "C" int64_t tg_launch_count(void) { return g_prof.launches; }

// ============================================================================= batched solver
// Many independent instances (each its own operator, coarse grid and deflation basis),
// each with R right-hand sides stored point-major (element (j, q) of instance i at
// offset_i + j * R + q).  Both phases advance all instances together in lock-step cycles,
// one launch per phase for all of them (tg_batch.cuh): the set-up runs the instances'
// coarse GMRES-DR cycles (float32 basis, one batched restart launch per cycle), then
// prolongs and factors each basis; the solve runs the float32-inner / float64-refinement
// BiCGStab(ncyc)-Proj(k) on the R columns of every instance (one read of the basis and of
// the stencil neighbourhood serves all R), the iteration sequence captured once as a CUDA
// graph and replayed, its blocks-per-instance shape chosen by timing (the autotuner).
namespace tg {

constexpr int kBatchR = 8;
constexpr int kGraphIters = 8;

struct BatchInst {
    DBuf tmp;
    // batched coarse phase: basis pair, restart scratch, coarse right-hand side
    DBuf cV, cV2, cbc, cc, cd, cres, cz, ctheta, cwr, cwi, cord, ceres, cP, ccn, cwork, cyw, cgw, cYc;
    PinBuf pin;
    cudaStream_t stream = nullptr;
    ~BatchInst() {
        if (stream) cudaStreamDestroy(stream);
    }
};

}  // namespace tg

// Device state of the batched coarse phase shared by all instances.
namespace tg {
struct BatchCoarse {
    DBuf H, H2, small, part, ticket, seg, args, active, info;
    int m = 0;
};
}  // namespace tg

// Device state of the batched solve: the work vectors of every instance concatenated (the
// instances' offsets are those of the right-hand sides), per-instance column states and
// reduction slices, the instance table, and the captured iteration graph.
namespace tg {
struct BatchAll {
    DBuf rh, p, v, s, t, r32, e32, r64, rsave, part, st, ctl, ticket, small, seg, colb, colx;
    PinBuf pin;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_gx = 0;
    int gx = 0;                    // tuned blocks per instance (0: not tuned yet)
    double tune_us[8] = {0};       // us per iteration of each candidate
    int tune_gx[8] = {0};
    int ntune = 0;
    ~BatchAll() {
        if (graph) cudaGraphExecDestroy(graph);
        if (stream) cudaStreamDestroy(stream);
    }
};
}  // namespace tg

struct tg_batch {
    int count = 0;
    int R = tg::kBatchR;
    std::vector<tg_op *> ops;
    std::vector<tg_defl *> defls;
    std::vector<int64_t> off;
    int64_t total = 0;
    int device = 0;
    std::vector<std::unique_ptr<tg::BatchInst>> inst;
    tg::BatchAll all;
    tg::BatchCoarse coarse;
    ~tg_batch() {
        for (auto *d : defls) delete d;
        for (auto *o : ops) delete o;
    }
};

namespace tg {

// Runs f(i) for i in [0, count) on up to `threads` host threads (each bound to `device`).
template <class F>
static int parallel_for(int count, int threads, int device, F f) {
    std::atomic<int> next{0};
    std::atomic<int> first_err{TG_OK};
    std::mutex err_mu;
    std::string err_text;
    auto worker = [&]() {
        cudaSetDevice(device);
        while (true) {
            const int i = next.fetch_add(1);
            if (i >= count || first_err.load() != TG_OK) break;
            const int rc = f(i);
            if (rc != TG_OK) {
                int expected = TG_OK;
                if (first_err.compare_exchange_strong(expected, rc)) {
                    std::lock_guard<std::mutex> lock(err_mu);
                    err_text = g_err;
                }
            }
        }
    };
    threads = std::max(1, std::min(threads, count));
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
    worker();
    for (auto &th : pool) th.join();
    if (first_err.load() != TG_OK) g_err = err_text;
    return first_err.load();
}


static int batch_inst_ready(tg_batch *b, int i) {
    BatchInst &I = *b->inst[i];
    if (!I.stream) TG_CHECK_CUDA(cudaStreamCreateWithFlags(&I.stream, cudaStreamNonBlocking));
    TG_CHECK(I.pin.ensure(4096));
    return TG_OK;
}

}  // namespace tg

namespace tg {

// Batched float32-inner / float64-refinement BiCGStab(ncyc)-Proj(k) over every instance at
// once: all instances advance their cycles in lock-step, one launch per phase for all of
// them (grid (gx, count)), the 8-iteration sequence of the four BiCGStab phases is one CUDA
// graph replayed until every column of the cycle has finished.  Per column: the schedule,
// safeguards and statistics of the single-instance float32 refinement.  gx (blocks per
// instance) is chosen once
// per handle by timing the iteration graph for each candidate (the autotuner).
constexpr int kMrPartW = 4 * kBatchR > 32 * kBatchR ? 4 * kBatchR : 32 * kBatchR;

static int batch_all_ready(tg_batch *b) {
    constexpr int R = kBatchR;
    BatchAll &A = b->all;
    const size_t tot = (size_t)b->total;
    TG_CHECK(A.rh.ensure(tot * 4));
    TG_CHECK(A.p.ensure(tot * 4));
    TG_CHECK(A.v.ensure(tot * 4));
    TG_CHECK(A.s.ensure(tot * 4));
    TG_CHECK(A.t.ensure(tot * 4));
    TG_CHECK(A.r32.ensure(tot * 4));
    TG_CHECK(A.e32.ensure(tot * 4));
    TG_CHECK(A.rsave.ensure(tot * 4));
    TG_CHECK(A.r64.ensure(tot * 8));
    TG_CHECK(A.part.ensure((size_t)b->count * 128 * kMrPartW * 8));   // up to 128 blocks per instance
    TG_CHECK(A.st.ensure((size_t)b->count * R * sizeof(BiState<double>)));
    TG_CHECK(A.ctl.ensure((size_t)b->count * sizeof(MrCtl)));
    // target2, inv, scale (R each), norms (2 R), cvec, dvec (32 R each), capv (R) per instance
    TG_CHECK(A.small.ensure((size_t)b->count * (2 * R + 2 * R + 2 * R + 2 * 32 * R) * 8));
    TG_CHECK(A.seg.ensure((size_t)b->count * sizeof(MrSeg)));
    TG_CHECK(A.pin.ensure((size_t)b->count * (R * sizeof(BiState<double>) + 4 * R * 8 + sizeof(GdrInfo)) + 4096));
    if (!A.stream) TG_CHECK_CUDA(cudaStreamCreateWithFlags(&A.stream, cudaStreamNonBlocking));
    if (!A.ticket.p) {
        TG_CHECK(A.ticket.ensure((size_t)b->count * sizeof(unsigned)));
        TG_CHECK_CUDA(cudaMemsetAsync(A.ticket.p, 0, (size_t)b->count * sizeof(unsigned), A.stream));
    }
    return TG_OK;
}

static MrBatchPtrs batch_ptrs(tg_batch *b, int cap) {
    constexpr int R = kBatchR;
    BatchAll &A = b->all;
    MrBatchPtrs P;
    double *sm = A.small.as<double>();
    const size_t B = b->count;
    P.seg = A.seg.as<MrSeg>();
    P.st = A.st.as<BiState<double>>();
    P.ctl = A.ctl.as<MrCtl>();
    P.ticket = A.ticket.as<unsigned>();
    P.part = A.part.as<double>();
    P.partw = kMrPartW;
    P.target2 = sm;
    P.inv = sm + B * R;
    P.scale = sm + 2 * B * R;
    P.norms = sm + 3 * B * R;
    P.cvec = sm + 5 * B * R;
    P.dvec = sm + 5 * B * R + B * 32 * R;
    P.cap = cap;
    P.capv = sm + 69 * B * R;
    return P;
}

static void batch_iters_all(tg_batch *b, const MrBatchPtrs &P, int gx, int iters, cudaStream_t s) {
    constexpr int R = kBatchR;
    BatchAll &A = b->all;
    const dim3 grid(gx, b->count);
    float *rh = A.rh.as<float>(), *p = A.p.as<float>(), *v = A.v.as<float>(), *sv = A.s.as<float>(),
          *t = A.t.as<float>(), *r = A.r32.as<float>(), *x = A.e32.as<float>();
    for (int it = 0; it < iters; ++it) {
        k_mrb_bi_v<R><<<grid, kThreads, 0, s>>>(p, rh, v, P);
        k_mrb_bi_s<R><<<grid, kThreads, 0, s>>>(r, v, sv, P);
        k_mrb_bi_t<R><<<grid, kThreads, 0, s>>>(sv, rh, t, P);
        k_mrb_bi_x<R><<<grid, kThreads, 0, s>>>(x, r, p, sv, t, v, P);
    }
}

// the iteration graph for gx blocks per instance (captured once per gx)
static int batch_graph(tg_batch *b, int gx) {
    BatchAll &A = b->all;
    if (A.graph && A.graph_gx == gx) return TG_OK;
    if (A.graph) {
        cudaGraphExecDestroy(A.graph);
        A.graph = nullptr;
    }
    const MrBatchPtrs P = batch_ptrs(b, 0);
    cudaGraph_t graph;
    TG_CHECK_CUDA(cudaStreamBeginCapture(A.stream, cudaStreamCaptureModeThreadLocal));
    batch_iters_all(b, P, gx, kGraphIters, A.stream);
    TG_CHECK_CUDA(cudaStreamEndCapture(A.stream, &graph));
    const cudaError_t e = cudaGraphInstantiate(&A.graph, graph, 0);
    cudaGraphDestroy(graph);
    TG_CHECK_CUDA(e);
    A.graph_gx = gx;
    return TG_OK;
}

static int batch_readback(tg_batch *b, const void *dev, size_t bytes) {
    TG_CHECK_CUDA(cudaMemcpyAsync(b->all.pin.p, dev, bytes, cudaMemcpyDeviceToHost, b->all.stream));
    TG_CHECK_CUDA(cudaStreamSynchronize(b->all.stream));
    return TG_OK;
}

// The autotuner: with r32 of the first cycle in place, each candidate gx runs the iteration
// graph on all columns (no column may finish: targets 0) and the fastest per iteration is
// kept; r32 is restored and e32 cleared afterwards.
static int batch_tune(tg_batch *b) {
    constexpr int R = kBatchR;
    BatchAll &A = b->all;
    const size_t tot = (size_t)b->total;
    cudaStream_t s = A.stream;
    TG_CHECK_CUDA(cudaMemcpyAsync(A.rsave.p, A.r32.p, tot * 4, cudaMemcpyDeviceToDevice, s));
    const int cands[] = {8, 16, 32, 64, 128};
    std::vector<double> zeros((size_t)b->count * R, 0.0);
    MrBatchPtrs P0 = batch_ptrs(b, INT_MAX / 2);
    P0.capv = nullptr;
    cudaEvent_t e0, e1;
    TG_CHECK_CUDA(cudaEventCreate(&e0));
    TG_CHECK_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int best_gx = 16;
    A.ntune = 0;
    for (int gx : cands) {
        TG_CHECK_CUDA(cudaMemcpyAsync(P0.target2, zeros.data(), zeros.size() * 8, cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemcpyAsync(A.r32.p, A.rsave.p, tot * 4, cudaMemcpyDeviceToDevice, s));
        TG_CHECK_CUDA(cudaMemsetAsync(A.e32.p, 0, tot * 4, s));
        k_mrb_bi_init<R><<<dim3(gx, b->count), kThreads, 0, s>>>(A.r32.as<float>(), A.rh.as<float>(), A.p.as<float>(), P0);
        TG_LAUNCH_CHECK();
        TG_CHECK(batch_graph(b, gx));
        TG_CHECK_CUDA(cudaGraphLaunch(A.graph, s));          // warm
        TG_CHECK_CUDA(cudaEventRecord(e0, s));
        TG_CHECK_CUDA(cudaGraphLaunch(A.graph, s));
        TG_CHECK_CUDA(cudaEventRecord(e1, s));
        TG_CHECK_CUDA(cudaStreamSynchronize(s));
        float ms = 0.f;
        TG_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double us = 1e3 * ms / kGraphIters;
        A.tune_gx[A.ntune] = gx;
        A.tune_us[A.ntune] = us;
        ++A.ntune;
        if (us < best) { best = us; best_gx = gx; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TG_CHECK_CUDA(cudaMemcpyAsync(A.r32.p, A.rsave.p, tot * 4, cudaMemcpyDeviceToDevice, s));
    TG_CHECK_CUDA(cudaMemsetAsync(A.e32.p, 0, tot * 4, s));
    A.gx = best_gx;
    __atomic_add_fetch(&g_prof.launches, (int64_t)A.ntune * (2 * 4 * kGraphIters + 1), __ATOMIC_RELAXED);
    return TG_OK;
}

static int batch_solve_all(tg_batch *b, const double *Bv, double *X, const SolveCfg &cfg, tg_stats *stats) {
    constexpr int R = kBatchR;
    const int count = b->count;
    TG_CHECK(batch_all_ready(b));
    BatchAll &A = b->all;
    cudaStream_t s = A.stream;
    // the instance table
    std::vector<MrSeg> seg(count);
    for (int i = 0; i < count; ++i) {
        const tg_op *op = b->ops[i];
        const tg_defl *df = b->defls.empty() ? nullptr : b->defls[i];
        MrSeg &g = seg[i];
        g.op = op->fine.A;
        g.o32 = op->fine.A32;
        g.off = (size_t)b->off[i];
        g.kk = df ? df->kk : 0;
        if (g.kk > 32) {
            set_error("batched projection supports k <= 32 (got %d)", g.kk);
            return TG_BAD_ARG;
        }
        g.proj = df ? df->proj : TG_PROJ_MINRES;
        g.W = df ? df->W32.as<float>() : nullptr;
        g.B1 = df ? df->B1_32.as<float>() : nullptr;
        g.B2 = df ? df->B2_32.as<float>() : nullptr;
        g.M = df ? df->M.as<double>() : nullptr;
    }
    TG_CHECK_CUDA(cudaMemcpyAsync(A.seg.p, seg.data(), seg.size() * sizeof(MrSeg), cudaMemcpyHostToDevice, s));
    bool any_defl = false;
    for (const MrSeg &g : seg) any_defl |= g.kk > 0;
    const int gres = 16;                                          // blocks per instance, refinement kernels
    MrBatchPtrs P = batch_ptrs(b, 0);
    double *hp = reinterpret_cast<double *>(A.pin.p);
    const size_t BR = (size_t)count * R;
    std::vector<double> nr(BR), nb(BR), nrel(BR), hv(BR), nr_before(BR), hcap(BR);
    std::vector<int64_t> mv(BR, 0);
    // per-column cycle cap: halved after a cycle whose correction raised the float64 residual
    // more than kIrGrowth-fold (the correction is then undone), so that the next cycle keeps
    // only the early, still contracting part of a float32 BiCGStab that diverges later;
    // smaller rises are kept (restarted BiCGStab is not monotone, later cycles recover them)
    std::vector<int64_t> capc(BR, cfg.restart_mvps > 0 ? cfg.restart_mvps : kIrCycleCap);
    std::vector<int> status(BR);
    auto residual = [&]() -> int {
        TG_PROF(P_RESIDUAL, (3.0 * 8) * b->total, 12.0 * b->total,
                k_mrb_residual<R><<<dim3(gres, count), kThreads, 0, s>>>(Bv, X, A.r64.as<double>(), P));
        TG_LAUNCH_CHECK();
        TG_CHECK(batch_readback(b, P.norms, (size_t)count * 2 * R * 8));
        for (int i = 0; i < count; ++i)
            for (int q = 0; q < R; ++q) {
                nr[i * R + q] = sqrt(hp[(size_t)i * 2 * R + q]);
                nb[i * R + q] = sqrt(hp[(size_t)i * 2 * R + R + q]);
            }
        return TG_OK;
    };
    TG_CHECK(residual());
    for (size_t c = 0; c < BR; ++c) status[c] = (nb[c] == 0.0 || nr[c] <= cfg.rtol * nb[c]) ? TG_OK : TG_NOT_CONVERGED;
    int cyc = 0;
    std::vector<int> cycles(count, 0);
    while (true) {
        bool any = false;
        for (size_t c = 0; c < BR; ++c) any |= status[c] == TG_NOT_CONVERGED;
        if (!any) break;
        ++cyc;
        const bool sched = cfg.ncyc && cyc <= cfg.ncyc;   // beyond ncyc: finish with rtol ||b|| / ||r||
        for (int i = 0; i < count; ++i) {
            bool on_i = false;
            for (int q = 0; q < R; ++q) on_i |= status[i * R + q] == TG_NOT_CONVERGED;
            if (on_i) cycles[i] = cyc;
        }
        // correction equations A e = r / ||r|| in float32
        for (size_t c = 0; c < BR; ++c) hv[c] = status[c] == TG_NOT_CONVERGED ? 1.0 / nr[c] : 0.0;
        TG_CHECK_CUDA(cudaMemcpyAsync(P.inv, hv.data(), BR * 8, cudaMemcpyHostToDevice, s));
        TG_PROF(P_CONVERT, 16.0 * b->total, b->total,
                k_mrb_scale<R><<<dim3(gres, count), kThreads, 0, s>>>(A.r64.as<double>(), A.r32.as<float>(),
                                                                         A.e32.as<float>(), P));
        TG_LAUNCH_CHECK();
        for (size_t c = 0; c < BR; ++c) nrel[c] = 1.0;
        if (any_defl) {
            const size_t smem = ((size_t)32 * 128 + 128 * R) * sizeof(float);
            TG_CHECK(set_smem<float>((const void *)k_mrb_proj_dots<R>, smem));
            TG_PROF(P_GEMV_T, 0, 0, k_mrb_proj_dots<R><<<dim3(gres, count), kThreads, smem, s>>>(A.r32.as<float>(), P));
            TG_PROF(P_SMALL, 0, 0, k_mrb_small<R><<<count, 256, 0, s>>>(P));
            TG_PROF(P_PROJ, 0, 0, k_mrb_proj_update<R><<<dim3(gres, count), kThreads, 0, s>>>(A.e32.as<float>(),
                                                                                            A.r32.as<float>(), P));
            TG_LAUNCH_CHECK();
            TG_CHECK(batch_readback(b, P.norms, (size_t)count * 2 * R * 8));
            for (int i = 0; i < count; ++i)
                if (seg[i].kk > 0)
                    for (int q = 0; q < R; ++q) nrel[i * R + q] = sqrt(hp[(size_t)i * 2 * R + q]);
        }
        int64_t cap64 = cfg.max_mvps;
        for (size_t c = 0; c < BR; ++c) {
            double t2 = -1.0;
            if (status[c] == TG_NOT_CONVERGED) {
                const double nrp = nrel[c] * nr[c];
                const int i = (int)(c / R);
                (void)i;
                double rt = sched ? cycle_tol(cfg.rtol, nb[c], nrp, cyc, cfg.ncyc) : cfg.rtol * nb[c] / nrp;
                if (rt < 1e-6) rt = 1e-6;
                t2 = (rt * nrel[c]) * (rt * nrel[c]);
                cap64 = std::min<int64_t>(cap64, cfg.max_mvps - mv[c]);
            }
            hv[c] = t2;
        }
        // per-column caps (a column whose cap was halved does not shorten the others' cycles);
        // cap64, the largest, bounds the host loop
        int64_t capmax = 1;
        for (size_t c = 0; c < BR; ++c) {
            const int64_t cc = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(cap64, capc[c]), INT_MAX / 2));
            hcap[c] = (double)cc;
            if (status[c] == TG_NOT_CONVERGED) capmax = std::max(capmax, cc);
        }
        TG_CHECK_CUDA(cudaMemcpyAsync(const_cast<double *>(P.capv), hcap.data(), BR * 8, cudaMemcpyHostToDevice, s));
        cap64 = capmax;
        if (A.gx == 0) TG_CHECK(batch_tune(b));           // once per handle, on the first cycle's r32
        const int gx = A.gx;
        TG_CHECK_CUDA(cudaMemcpyAsync(P.target2, hv.data(), BR * 8, cudaMemcpyHostToDevice, s));
        const MrBatchPtrs Pc = batch_ptrs(b, (int)cap64);
        TG_PROF(P_BI_INIT, 12.0 * b->total, 2.0 * b->total,
                k_mrb_bi_init<R><<<dim3(gx, count), kThreads, 0, s>>>(A.r32.as<float>(), A.rh.as<float>(),
                                                                        A.p.as<float>(), Pc));
        TG_LAUNCH_CHECK();
        TG_CHECK(batch_graph(b, gx));
        int graphs = 0;
        while (true) {
            TG_CHECK_CUDA(cudaGraphLaunch(A.graph, s));
            __atomic_add_fetch(&g_prof.launches, 4 * kGraphIters, __ATOMIC_RELAXED);
            ++graphs;
            TG_CHECK(batch_readback(b, P.ctl, (size_t)count * sizeof(MrCtl)));
            const MrCtl *hc = reinterpret_cast<const MrCtl *>(A.pin.p);
            int active = 0;
            for (int i = 0; i < count; ++i) active += hc[i].active;
            if (active == 0) break;
            if ((int64_t)graphs * kGraphIters > cap64 + 8) {
                set_error("batched BiCGStab cycle exceeded its product cap");
                return TG_SYNC_TIMEOUT;
            }
        }
        TG_CHECK(batch_readback(b, P.st, BR * sizeof(BiState<double>)));
        std::vector<BiState<double>> hs(BR);
        memcpy(hs.data(), A.pin.p, BR * sizeof(BiState<double>));
        std::vector<char> bad(BR, 0);
        for (size_t c = 0; c < BR; ++c) {     // a diverged or NaN float32 correction is not added
            bad[c] = status[c] == TG_NOT_CONVERGED && (hs[c].status == 4 || hs[c].status == 5);
            hv[c] = (status[c] == TG_NOT_CONVERGED && !bad[c]) ? nr[c] : 0.0;
            nr_before[c] = nr[c];
        }
        TG_CHECK_CUDA(cudaMemcpyAsync(P.scale, hv.data(), BR * 8, cudaMemcpyHostToDevice, s));
        TG_PROF(P_CONVERT, 12.0 * b->total, 2.0 * b->total,
                k_mrb_add<R><<<dim3(gres, count), kThreads, 0, s>>>(X, A.e32.as<float>(), P));
        TG_LAUNCH_CHECK();
        TG_CHECK(residual());
        // a correction that raised the float64 residual kIrGrowth-fold is undone (x -= ||r|| e)
        bool undo = false;
        for (size_t c = 0; c < BR; ++c) {
            const bool worse = status[c] == TG_NOT_CONVERGED && !bad[c] && !(nr[c] <= kIrGrowth * nr_before[c]);
            hv[c] = worse ? -nr_before[c] : 0.0;
            if (worse || bad[c]) {
                capc[c] = std::max<int64_t>(1, std::min<int64_t>(capc[c], hs[c].mvps) / 2);
                undo |= worse;
            }
        }
        if (undo) {
            TG_CHECK_CUDA(cudaMemcpyAsync(P.scale, hv.data(), BR * 8, cudaMemcpyHostToDevice, s));
            TG_PROF(P_CONVERT, 12.0 * b->total, 2.0 * b->total,
                    k_mrb_add<R><<<dim3(gres, count), kThreads, 0, s>>>(X, A.e32.as<float>(), P));
            TG_LAUNCH_CHECK();
            TG_CHECK(residual());
        }
        bool stuck = true;
        for (size_t c = 0; c < BR; ++c) {
            if (status[c] != TG_NOT_CONVERGED) continue;
            mv[c] += hs[c].mvps;
            if (hs[c].mvps > 0) stuck = false;
            if (!std::isfinite(nr[c])) status[c] = TG_NAN;
            else if (nr[c] <= cfg.rtol * nb[c]) status[c] = TG_OK;
            else if (mv[c] >= cfg.max_mvps) status[c] = TG_NOT_CONVERGED + 100;   // out of budget
            else if (capc[c] < 4) status[c] = TG_BREAKDOWN;      // no float32 cycle lowers its residual
        }
        if (stuck) break;
    }
    // columns no float32 cycle can advance finish with float64 BiCGStab(-Proj) cycles on the
    // instance's own operator and basis, as the single-system float32 form does: the column is
    // gathered from the point-major block, solved, and scattered back
    std::vector<int> fp64_cyc(count, 0);
    for (size_t c = 0; c < BR; ++c) {
        if (status[c] != TG_BREAKDOWN && status[c] != TG_NAN) continue;
        const int i = (int)(c / R), q = (int)(c % R);
        tg_op *op = b->ops[i];
        const tg_defl *df = b->defls.empty() ? nullptr : b->defls[i];
        const size_t n = (size_t)op->n;
        TG_CHECK(A.colb.ensure(n * 8));
        TG_CHECK(A.colx.ensure(n * 8));
        double *cb = A.colb.as<double>(), *cx = A.colx.as<double>();
        const size_t off = (size_t)b->off[i] + q;
        TG_CHECK_CUDA(cudaMemcpy2DAsync(cb, 8, Bv + off, R * 8, 8, n, cudaMemcpyDeviceToDevice, s));
        TG_CHECK_CUDA(cudaMemcpy2DAsync(cx, 8, X + off, R * 8, 8, n, cudaMemcpyDeviceToDevice, s));
        SolveCfg c64 = cfg;
        c64.ncyc = 0;
        c64.max_mvps = std::max<int64_t>(1, cfg.max_mvps - mv[c]);
        if (c64.restart_mvps <= 0) c64.restart_mvps = 1000;
        tg_stats s64{};
        s64.history = nullptr;
        const int rc64 = solve_bicg64<double>(op, 0, df, cb, cx, c64, &s64, s);
        if (rc64 == TG_BAD_ARG || rc64 == TG_OOM || rc64 == TG_CUDA_ERROR) return rc64;
        TG_CHECK_CUDA(cudaMemcpy2DAsync(X + off, R * 8, cx, 8, 8, n, cudaMemcpyDeviceToDevice, s));
        mv[c] += s64.mvps;
        nr[c] = s64.relres * nb[c];
        status[c] = rc64;
        fp64_cyc[i] += s64.cycles;
    }
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    int worst = TG_OK;
    for (size_t c = 0; c < BR; ++c) {
        if (status[c] == TG_NOT_CONVERGED + 100) status[c] = TG_NOT_CONVERGED;
        if (stats) {
            tg_stats &o = stats[c];
            o.mvps = mv[c];
            o.cycles = cycles[c / R];
            o.relres = nb[c] > 0 ? nr[c] / nb[c] : 0.0;
            o.status = status[c];
            o.vops = mv[c] * 7;
            o.fp64_cycles = fp64_cyc[c / R];
        }
        if (status[c] != TG_OK && worst == TG_OK) worst = status[c];
    }
    return worst;
}

}  // namespace tg

namespace tg {

// The coarse GMRES-DR(m,k) of every instance in lock-step cycles (float32 basis, float64
// Hessenberg and restart step, as gmresdr_impl<float, double>): one launch per Arnoldi
// sub-step for all instances, one batched restart launch (one block per instance), then
// the recombination V <- V P_{k+1} and the re-orthogonalisation of v_{kk} for all.  An
// instance leaves the loop when its least-squares residual is below rtol ||b_c|| and nev
// pairs have converged, or after max_cycles.  Afterwards each instance's basis V_m P_k is
// prolonged and factored (A Y, CholQR2, float32 copies) as in tg_coarse_gmresdr.
constexpr int kGbBlocks = 64;             // blocks per instance of the coarse kernels
constexpr int kGbPartW = 64;              // >= m + 2 columns of partial sums

static int batch_setup_all(tg_batch *b, const double *R0, int m, int k, int nev, double rtolev, double rtol,
                           int max_cycles, int proj, int threads, tg_stats *stats) {
    const int count = b->count;
    TG_CHECK(batch_all_ready(b));
    BatchAll &A = b->all;
    BatchCoarse &C = b->coarse;
    cudaStream_t s = A.stream;
    const int ldh = m + 1;
    TG_ARG(m + 2 <= kGbPartW && m + 1 <= kSmallCols, "the batched coarse phase takes m <= %d", kGbPartW - 2);
    // shared coarse state
    TG_CHECK(C.H.ensure((size_t)count * ldh * m * 8));
    TG_CHECK(C.H2.ensure((size_t)count * ldh * m * 8));
    TG_CHECK(C.small.ensure((size_t)count * 3 * 256 * 8));      // h1, h2, nrm per instance
    TG_CHECK(C.part.ensure((size_t)count * kGbBlocks * kGbPartW * 8));
    TG_CHECK(C.seg.ensure((size_t)count * sizeof(GdrSeg)));
    TG_CHECK(C.args.ensure((size_t)count * sizeof(GdrArgs<double>)));
    TG_CHECK(C.active.ensure((size_t)count * sizeof(int)));
    TG_CHECK(C.info.ensure((size_t)count * sizeof(GdrInfo)));
    if (!C.ticket.p) {
        TG_CHECK(C.ticket.ensure((size_t)count * sizeof(unsigned)));
        TG_CHECK_CUDA(cudaMemsetAsync(C.ticket.p, 0, (size_t)count * sizeof(unsigned), s));
    }
    int parts = 0;
    gmresdr_restart_smem<double>(m, &parts);
    std::vector<GdrSeg> seg(count);
    std::vector<GdrArgs<double>> args(count);
    std::vector<double *> Hc(count), H2c(count);
    std::vector<float *> V2(count);
    std::vector<double> nbc(count);
    std::vector<int> active(count, 1), cycles(count, 0);
    std::vector<int64_t> cmvps(count, 0);
    std::vector<GdrInfo> info(count);
    double *small = C.small.as<double>();
    for (int i = 0; i < count; ++i) {
        tg_op *op = b->ops[i];
        BatchInst &I = *b->inst[i];
        const int nc = op->nc;
        TG_ARG(m < nc && k < m - 1 && nev >= 0 && nev <= k, "bad GMRES-DR sizes for instance %d", i);
        const size_t ldv = ((size_t)nc + 127) / 128 * 128;
        TG_CHECK(I.cV.ensure(ldv * (m + 1) * 4));
        TG_CHECK(I.cV2.ensure(ldv * (m + 1) * 4));
        TG_CHECK(I.cbc.ensure((size_t)nc * 8));
        TG_CHECK(I.tmp.ensure((size_t)op->n * 8));
        TG_CHECK(I.cd.ensure((size_t)(m + 1) * 8));
        TG_CHECK(I.cc.ensure((size_t)(m + 1) * 8));
        TG_CHECK(I.cres.ensure((size_t)(m + 1) * 8));
        TG_CHECK(I.cz.ensure((size_t)(m + 1) * 8));
        TG_CHECK(I.ctheta.ensure((size_t)2 * m * 8));
        TG_CHECK(I.cwr.ensure((size_t)m * 8));
        TG_CHECK(I.cwi.ensure((size_t)m * 8));
        TG_CHECK(I.cord.ensure((size_t)m * 4));
        TG_CHECK(I.ceres.ensure((size_t)m * 8));
        TG_CHECK(I.cP.ensure((size_t)(m + 1) * (m + 2) * 8));
        TG_CHECK(I.ccn.ensure((size_t)(m + 2) * 8));
        TG_CHECK(I.cwork.ensure(((size_t)(m + 1) * m + 2 * (size_t)m * m + 3 * (size_t)m + 4) * 8));
        TG_CHECK(I.cyw.ensure((size_t)m * m * 16));
        TG_CHECK(I.cgw.ensure((size_t)m * m * 16));
        TG_CHECK(I.cYc.ensure((size_t)nc * (k + 2) * 8));
        // b_c = restrict(column 0), ||b_c||, v_0 = b_c / ||b_c|| (float32)
        k_mr_extract<kBatchR><<<grid_for(op->n, 8), kThreads, 0, s>>>(R0 + b->off[i], 0, op->n, I.tmp.as<double>());
        TG_LAUNCH_CHECK();
        TG_CHECK(restrict_impl(op, I.tmp.p, I.cbc.p, 1, s));
        double nb2 = 0.0;
        TG_CHECK(red_ready(op, 0, s));
        TG_CHECK(dot_host<double>(op, I.cbc.as<double>(), nullptr, nc, &nb2, nullptr, s));
        nbc[i] = sqrt(nb2);
        TG_ARG(nbc[i] > 0 && std::isfinite(nbc[i]), "restricted right-hand side of instance %d is zero or not finite", i);
        launch_d2f_scaled(grid_for(nc, 8), s, I.cbc.as<double>(), I.cV.as<float>(), nc, 1.0 / nbc[i]);
        TG_LAUNCH_CHECK();
        Hc[i] = C.H.as<double>() + (size_t)i * ldh * m;
        H2c[i] = C.H2.as<double>() + (size_t)i * ldh * m;
        V2[i] = I.cV2.as<float>();
        GdrSeg &g = seg[i];
        g.op = op->coarse.A;
        g.o32 = op->coarse.A32;
        g.V = I.cV.as<float>();
        g.xc = nullptr;
        g.H = Hc[i];
        g.h1 = small + (size_t)i * 3 * 256;
        g.h2 = g.h1 + 256;
        g.nrm = g.h2 + 256;
        g.d = I.cd.as<double>();
        g.ldv = ldv;
        g.nc = nc;
        g.j0 = 0;
        g.kk = 0;
        g.active = 1;
        // c = ||b_c|| e_1 in the least-squares right-hand side (the restart kernel reads it from a.c)
        GdrArgs<double> &a = args[i];
        a.ldh = ldh; a.m = m; a.k = k; a.nev = nev; a.rtolev = rtolev;
        a.d = I.cd.as<double>(); a.res = I.cres.as<double>(); a.z = I.cz.as<double>();
        a.theta = I.ctheta.as<double>(); a.wr = I.cwr.as<double>(); a.wi = I.cwi.as<double>();
        a.order = I.cord.as<int>(); a.eres = I.ceres.as<double>(); a.P = I.cP.as<double>();
        a.cnew = I.ccn.as<double>(); a.work = I.cwork.as<double>(); a.ywork = I.cyw.as<cplx>();
        a.gwork = I.cgw.as<cplx>(); a.info = C.info.as<GdrInfo>() + i;
        a.smem = parts;
        a.mode = 0;
    }
    TG_CHECK_CUDA(cudaMemsetAsync(C.H.p, 0, (size_t)count * ldh * m * 8, s));
    // least-squares right-hand sides c = ||b_c|| e_1
    std::vector<double> c0(m + 1, 0.0);
    for (int i = 0; i < count; ++i) {
        BatchInst &I = *b->inst[i];
        c0[0] = nbc[i];
        TG_CHECK_CUDA(cudaMemcpyAsync(I.cc.p, c0.data(), (size_t)(m + 1) * 8, cudaMemcpyHostToDevice, s));
        args[i].c = I.cc.as<double>();
    }
    GdrBatchPtrs P{C.seg.as<GdrSeg>(), C.part.as<double>(), kGbPartW, C.ticket.as<unsigned>()};
    const dim3 grid(kGbBlocks, count);
    // V^H w through the pipelined kernel when its shared memory can be granted
    static_assert(kGbPartW <= kGbPipeCols + 1, "the pipelined batched V^H w covers every column count");
    bool gb_pipe = smem_attr_once((const void *)k_gb_gemv_t_pipe, (int)kGbPipeSmem) == cudaSuccess;
    if (!gb_pipe) (void)cudaGetLastError();
    auto gemv_t_all = [&](int j, int ncol_step, int reorth, int which) {
        if (gb_pipe) k_gb_gemv_t_pipe<<<grid, kThreads, kGbPipeSmem, s>>>(P, j, ncol_step, reorth, which);
        else k_gb_gemv_t<<<grid, kThreads, 0, s>>>(P, j, ncol_step, reorth, which);
    };
    int any = count;
    int cyc = 0;
    while (any) {
        ++cyc;
        // table and restart arguments of this cycle
        int jmin = m;
        for (int i = 0; i < count; ++i) {
            seg[i].active = active[i];
            args[i].H = Hc[i];
            args[i].Hnew = H2c[i];
            if (active[i]) jmin = std::min(jmin, seg[i].j0);
        }
        TG_CHECK_CUDA(cudaMemcpyAsync(C.seg.p, seg.data(), seg.size() * sizeof(GdrSeg), cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemcpyAsync(C.args.p, args.data(), args.size() * sizeof(GdrArgs<double>),
                                      cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemcpyAsync(C.active.p, active.data(), active.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        // Arnoldi from each instance's j0 to m
        for (int j = jmin; j < m; ++j) {
            TG_PROF(P_APPLY, 0, 0, k_gb_apply<<<grid, kThreads, 0, s>>>(P, j));
            TG_PROF(P_GEMV_T, 0, 0, gemv_t_all(j, j + 2, 0, 0));
            TG_PROF(P_GEMV_N, 0, 0, k_gb_gemv_n_norm<<<grid, kThreads, 0, s>>>(P, j, j + 1, 0, 0));
            TG_PROF(P_GEMV_T, 0, 0, gemv_t_all(j, j + 1, 0, 1));
            TG_PROF(P_GEMV_N, 0, 0, k_gb_gemv_n_norm<<<grid, kThreads, 0, s>>>(P, j, j + 1, 0, 1));
            TG_PROF(P_SMALL, 0, 0, k_gb_finish<<<(count + 127) / 128, 128, 0, s>>>(P, count, j, ldh, 0));
            TG_PROF(P_SCALE, 0, 0, k_gb_scale<<<grid, kThreads, 0, s>>>(P, j, 0));
        }
        TG_LAUNCH_CHECK();
        // the restart matrices are written into each instance's other Hbar buffer (which of
        // the two pools holds it alternates with the instance's restarts)
        for (int i = 0; i < count; ++i)
            if (active[i]) TG_CHECK_CUDA(cudaMemsetAsync(H2c[i], 0, (size_t)ldh * m * 8, s));
        cudaError_t le = cudaSuccess;
        TG_PROF(P_GDR_RESTART, 0, 30.0 * m * m * m * count,
                le = launch_gmresdr_restart_batch<double>(C.args.as<GdrArgs<double>>(), C.active.as<int>(), count, m, s));
        if (le != cudaSuccess) return cuda_status(le, "launching the batched restart step");
        // the instances' restart results
        TG_CHECK(batch_readback(b, C.info.p, (size_t)count * sizeof(GdrInfo)));
        {
            const GdrInfo *hi = reinterpret_cast<const GdrInfo *>(A.pin.p);
            for (int i = 0; i < count; ++i)
                if (active[i]) info[i] = hi[i];
        }
        std::vector<int> cont(count, 0);
        for (int i = 0; i < count; ++i) {
            if (!active[i]) continue;
            cmvps[i] += m - seg[i].j0;
            cycles[i] = cyc;
            if (info[i].status != 0) {
                set_error("harmonic Ritz QR iteration did not converge (instance %d)", i);
                return TG_NOT_CONVERGED;
            }
            const int kk = info[i].kk;
            const bool conv = info[i].rnorm <= rtol * nbc[i] && info[i].nconv >= (nev < kk ? nev : kk);
            seg[i].kk = kk;
            if (conv || cyc >= max_cycles || !std::isfinite(info[i].rnorm)) {
                active[i] = 0;            // done: its V, Hbar and P stay for the final basis
            } else {
                cont[i] = 1;
            }
        }
        any = 0;
        for (int i = 0; i < count; ++i) any += cont[i];
        if (!any) break;
        // restart of the continuing instances: V2 = V P_{k+1}, Hbar <- Hnew, c <- cnew, then
        // re-orthogonalise v_kk and normalise it
        for (int i = 0; i < count; ++i) seg[i].active = cont[i];
        TG_CHECK_CUDA(cudaMemcpyAsync(C.seg.p, seg.data(), seg.size() * sizeof(GdrSeg), cudaMemcpyHostToDevice, s));
        {
            std::vector<const double *> Pp(count);
            std::vector<float *> Op(count);
            std::vector<size_t> ldo(count);
            for (int i = 0; i < count; ++i) {
                Pp[i] = args[i].P;
                Op[i] = V2[i];
                ldo[i] = seg[i].ldv;
            }
            TG_CHECK(A.rsave.ensure(std::max<size_t>(A.rsave.bytes, (size_t)count * 24)));
            char *tb = A.rsave.as<char>();
            TG_CHECK_CUDA(cudaMemcpyAsync(tb, Pp.data(), (size_t)count * 8, cudaMemcpyHostToDevice, s));
            TG_CHECK_CUDA(cudaMemcpyAsync(tb + (size_t)count * 8, Op.data(), (size_t)count * 8, cudaMemcpyHostToDevice, s));
            TG_CHECK_CUDA(cudaMemcpyAsync(tb + (size_t)count * 16, ldo.data(), (size_t)count * 8, cudaMemcpyHostToDevice, s));
            TG_PROF(P_TSM, 0, 0, k_gb_tsm<float><<<grid, kThreads, 0, s>>>(
                P, reinterpret_cast<const double *const *>(tb), m + 1, m + 1, 1,
                reinterpret_cast<float *const *>(tb + (size_t)count * 8), reinterpret_cast<const size_t *>(tb + (size_t)count * 16)));
            TG_LAUNCH_CHECK();
            TG_CHECK_CUDA(cudaStreamSynchronize(s));     // the tables are reused below
        }
        for (int i = 0; i < count; ++i) {
            if (!cont[i]) continue;
            std::swap(seg[i].V, V2[i]);
            std::swap(Hc[i], H2c[i]);
            seg[i].H = Hc[i];
            BatchInst &I = *b->inst[i];
            // c = cnew (kk + 1 entries), zero beyond
            TG_CHECK_CUDA(cudaMemsetAsync(I.cc.p, 0, (size_t)(m + 1) * 8, s));
            TG_CHECK_CUDA(cudaMemcpyAsync(I.cc.p, I.ccn.p, (size_t)(seg[i].kk + 1) * 8, cudaMemcpyDeviceToDevice, s));
            seg[i].j0 = seg[i].kk;
        }
        TG_CHECK_CUDA(cudaMemcpyAsync(C.seg.p, seg.data(), seg.size() * sizeof(GdrSeg), cudaMemcpyHostToDevice, s));
        TG_PROF(P_REORTH, 0, 0, gemv_t_all(0, 0, 1, 0));
        TG_PROF(P_REORTH, 0, 0, k_gb_gemv_n_norm<<<grid, kThreads, 0, s>>>(P, 0, 0, 1, 0));
        TG_PROF(P_SMALL, 0, 0, k_gb_finish<<<(count + 127) / 128, 128, 0, s>>>(P, count, 0, ldh, 1));
        TG_PROF(P_SCALE, 0, 0, k_gb_scale<<<grid, kThreads, 0, s>>>(P, 0, 1));
        TG_LAUNCH_CHECK();
        for (int i = 0; i < count; ++i) active[i] = cont[i];
    }
    // final bases Yc = V_m P_k (float64), for every instance
    for (int i = 0; i < count; ++i) seg[i].active = 1;
    TG_CHECK_CUDA(cudaMemcpyAsync(C.seg.p, seg.data(), seg.size() * sizeof(GdrSeg), cudaMemcpyHostToDevice, s));
    {
        std::vector<const double *> Pp(count);
        std::vector<double *> Op(count);
        std::vector<size_t> ldo(count);
        for (int i = 0; i < count; ++i) {
            Pp[i] = args[i].P;
            Op[i] = b->inst[i]->cYc.as<double>();
            ldo[i] = (size_t)seg[i].nc;
        }
        char *tb = A.rsave.as<char>();
        TG_CHECK_CUDA(cudaMemcpyAsync(tb, Pp.data(), (size_t)count * 8, cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemcpyAsync(tb + (size_t)count * 8, Op.data(), (size_t)count * 8, cudaMemcpyHostToDevice, s));
        TG_CHECK_CUDA(cudaMemcpyAsync(tb + (size_t)count * 16, ldo.data(), (size_t)count * 8, cudaMemcpyHostToDevice, s));
        TG_PROF(P_TSM, 0, 0, k_gb_tsm<double><<<grid, kThreads, 0, s>>>(
            P, reinterpret_cast<const double *const *>(tb), m + 1, m, 0,
            reinterpret_cast<double *const *>(tb + (size_t)count * 8), reinterpret_cast<const size_t *>(tb + (size_t)count * 16)));
        TG_LAUNCH_CHECK();
    }
    TG_CHECK_CUDA(cudaStreamSynchronize(s));
    // per instance: prolong the basis, A Y and its factorisation (float64 and float32 copies)
    if ((int)b->defls.size() != count) b->defls.assign(count, nullptr);
    return parallel_for(count, threads, b->device, [&](int i) -> int {
        TG_CHECK(batch_inst_ready(b, i));
        BatchInst &I = *b->inst[i];
        tg_op *op = b->ops[i];
        const int kk = seg[i].kk;
        tg_defl *d = b->defls[i];
        if (d) {
            d->kk = kk; d->n = op->n; d->proj = proj; d->precision = TG_F32_IR; d->cplx_ = false; d->transposed = false;
            TG_CHECK(d->Y.ensure((size_t)op->n * kk * 8));
        } else {
            TG_CHECK(defl_create(op, 0, kk, proj, TG_F32_IR, &d));
            b->defls[i] = d;
        }
        TG_CHECK(prolong_impl(op, I.cYc.p, d->Y.p, kk, I.stream));
        TG_CHECK(build_defl<double>(op, 0, d, I.stream));
        if (stats) {
            tg_stats &o = stats[i];
            o = tg_stats{};
            o.coarse_mvps = cmvps[i];
            o.cycles = cycles[i];
            o.coarse_relres = info[i].rnorm / nbc[i];
            o.kk = kk;
            o.eig_converged = info[i].nconv;
            o.status = (info[i].rnorm <= rtol * nbc[i] && info[i].nconv >= (nev < kk ? nev : kk)) ? TG_OK
                                                                                                 : TG_NOT_CONVERGED;
        }
        return TG_OK;
    });
}

}  // namespace tg

extern "C" int tg_batch_tuning(const tg_batch *b, int *blocks_per_instance, double *us_per_iteration, int *ncand,
                               int *cand_blocks, double *cand_us) {
    TG_ARG(b, "NULL batch");
    const BatchAll &A = b->all;
    if (blocks_per_instance) *blocks_per_instance = A.gx;
    double best = 0.0;
    for (int q = 0; q < A.ntune; ++q)
        if (A.tune_gx[q] == A.gx) best = A.tune_us[q];
    if (us_per_iteration) *us_per_iteration = best;
    if (ncand) *ncand = A.ntune;
    for (int q = 0; q < A.ntune; ++q) {
        if (cand_blocks) cand_blocks[q] = A.tune_gx[q];
        if (cand_us) cand_us[q] = A.tune_us[q];
    }
    return TG_OK;
}

extern "C" int tg_batch_create(tg_batch **out, int count, const int64_t *Ns, const double *betas, int nrhs,
                               void *stream) {
    TG_ARG(out && Ns && betas && count >= 1, "bad argument");
    TG_ARG(nrhs == kBatchR, "the batched solver takes %d right-hand sides per instance (got %d)", kBatchR, nrhs);
    *out = nullptr;
    tg_batch *b = new tg_batch();
    b->count = count;
    cudaGetDevice(&b->device);
    for (int i = 0; i < count; ++i) {
        tg_op *op = nullptr;
        const double beta3[3] = {betas[i], 0.0, 0.0};
        int rc = tg_setup_operator(&op, TG_CD2D, Ns + i, 1, beta3, nullptr, nullptr, 2, stream);
        if (rc != TG_OK) {
            delete b;
            return rc;
        }
        b->ops.push_back(op);
        b->off.push_back(b->total);
        b->total += (int64_t)op->n * kBatchR;
        b->inst.emplace_back(new BatchInst());
    }
    *out = b;
    return TG_OK;
}

extern "C" int tg_destroy_batch(tg_batch *b) {
    delete b;
    return TG_OK;
}

extern "C" int tg_batch_layout(const tg_batch *b, int i, int64_t *offset, int64_t *n) {
    TG_ARG(b && i >= 0 && i < b->count, "bad instance index");
    if (offset) *offset = b->off[i];
    if (n) *n = b->ops[i]->n;
    return TG_OK;
}

extern "C" int tg_batch_setup(tg_batch *b, const void *rhs, int m, int k, int nev, double rtolev, double rtol,
                              int max_cycles, int proj, int threads, tg_stats *stats, void *stream) {
    TG_ARG(b && rhs, "NULL argument");
    TG_ARG(k >= 1 && k <= 32, "the batched projection takes 1 <= k <= 32 (got %d)", k);
    TG_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if ((int)b->defls.size() != b->count) b->defls.assign(b->count, nullptr);   // handles are rebuilt in place
    const double *R0 = static_cast<const double *>(rhs);
    if (m + 2 <= kGbPartW)
        return batch_setup_all(b, R0, m, k, nev, rtolev, rtol, max_cycles, proj, threads, stats);
    return parallel_for(b->count, threads, b->device, [&](int i) -> int {
        TG_CHECK(batch_inst_ready(b, i));
        BatchInst &I = *b->inst[i];
        tg_op *op = b->ops[i];
        TG_CHECK(I.tmp.ensure((size_t)op->n * 8));
        k_mr_extract<kBatchR><<<grid_for(op->n, 8), kThreads, 0, I.stream>>>(R0 + b->off[i], 0, op->n, I.tmp.as<double>());
        TG_LAUNCH_CHECK();
        tg_stats st{};
        tg_defl *d = nullptr;
        TG_ARG(m >= 2 && m <= kMaxM && k < m - 1 && m < op->nc && nev >= 0 && nev <= k, "bad GMRES-DR sizes");
        int rc = gmresdr_impl<double>(op, 0, I.tmp.p, m, k, nev, rtolev, rtol, max_cycles, nullptr, &d, proj,
                                      TG_F32_IR, &st, I.stream, b->defls[i]);
        if (stats) stats[i] = st;
        if (rc != TG_OK && rc != TG_NOT_CONVERGED) return rc;
        b->defls[i] = d;
        return TG_OK;
    });
}

extern "C" int tg_batch_solve(tg_batch *b, const void *rhs, void *x, double rtol, int ncyc, int restart_mvps,
                              int64_t max_mvps, int threads, tg_stats *stats, void *stream) {
    TG_ARG(b && rhs && x, "NULL argument");
    TG_ARG(rtol > 0 && rtol < 1, "rtol must be in (0, 1)");
    TG_ARG(ncyc > 0 || restart_mvps > 0, "fixed-length restarting needs restart_mvps > 0");
    TG_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    SolveCfg cfg{rtol, ncyc, restart_mvps, 0, max_mvps};
    const double *B = static_cast<const double *>(rhs);
    double *X = static_cast<double *>(x);
    (void)threads;     // one batched launch per phase for all instances: no host threads
    return batch_solve_all(b, B, X, cfg, stats);
}
