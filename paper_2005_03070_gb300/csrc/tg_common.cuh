// Shared device types and helpers of the tg library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>
#include <string>
#include <utility>
#include <vector>
#include "tg.h"

namespace tg {

// Raise a kernel's dynamic shared memory limit to `bytes` once per (kernel, device).  The
// value for a given kernel is always the same, so concurrent callers cannot lower it under
// each other, and later calls make no driver call (safe inside a stream capture).
inline cudaError_t smem_attr_once(const void *fn, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &d : done)
        if (d.first == fn && d.second == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.emplace_back(fn, dev);
    return e;
}

// ----------------------------------------------------------------------------- status
void set_error(const char *fmt, ...);
int cuda_status(cudaError_t e, const char *where);

#define TG_CHECK_CUDA(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) return ::tg::cuda_status(_e, #expr);                \
    } while (0)
#define TG_CHECK(expr)                                                             \
    do {                                                                           \
        int _s = (expr);                                                           \
        if (_s != TG_OK) return _s;                                                \
    } while (0)
#define TG_LAUNCH_CHECK() TG_CHECK_CUDA(cudaGetLastError())

// ----------------------------------------------------------------------------- complex
struct __align__(16) cplx {
    double re, im;
};
__host__ __device__ __forceinline__ cplx mkc(double a, double b) { return cplx{a, b}; }
__host__ __device__ __forceinline__ cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a) { return {-a.re, -a.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, cplx b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cplx operator*(double s, cplx a) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, double s) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cplx conj(cplx a) { return {a.re, -a.im}; }
__host__ __device__ __forceinline__ double abs2(cplx a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    double r = b.re / b.im, d = b.im + b.re * r;
    return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
__host__ __device__ __forceinline__ double cabs_(cplx a) { return hypot(a.re, a.im); }

// ----------------------------------------------------------------------------- scalar traits
// Vector element type T; D = type of an inner product (double for real T, cplx for
// complex T).  conj_mul(a, b) = conj(a) * b.
template <class T> struct ST;
template <> struct ST<double> {
    using D = double;
    __host__ __device__ static __forceinline__ double zero() { return 0.0; }
    __host__ __device__ static __forceinline__ double conj_mul(double a, double b) { return a * b; }
    __host__ __device__ static __forceinline__ double fma_cm(double a, double b, double acc) { return fma(a, b, acc); }
    __host__ __device__ static __forceinline__ double scale(double s, double a) { return s * a; }
    __host__ __device__ static __forceinline__ double from(double d) { return d; }
};
template <> struct ST<float> {
    using D = double;
    __host__ __device__ static __forceinline__ float zero() { return 0.0f; }
    __host__ __device__ static __forceinline__ float conj_mul(float a, float b) { return a * b; }
    __host__ __device__ static __forceinline__ float fma_cm(float a, float b, float acc) { return fmaf(a, b, acc); }
    __host__ __device__ static __forceinline__ float scale(float s, float a) { return s * a; }
    __host__ __device__ static __forceinline__ float from(double d) { return (float)d; }
};
template <> struct ST<cplx> {
    using D = cplx;
    __host__ __device__ static __forceinline__ cplx zero() { return {0.0, 0.0}; }
    __host__ __device__ static __forceinline__ cplx conj_mul(cplx a, cplx b) {
        return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
    }
    __host__ __device__ static __forceinline__ cplx fma_cm(cplx a, cplx b, cplx acc) {
        return {fma(a.re, b.re, fma(a.im, b.im, acc.re)), fma(a.re, b.im, fma(-a.im, b.re, acc.im))};
    }
    __host__ __device__ static __forceinline__ cplx from(cplx d) { return d; }
};

// Dot accumulators: per-thread partial in P, block/grid totals in D.
template <class T> struct Acc { using P = T; };
__device__ __forceinline__ double to_d(double a) { return a; }
__device__ __forceinline__ double to_d(float a) { return (double)a; }
__device__ __forceinline__ cplx to_d(cplx a) { return a; }

__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ cplx shfl_down(cplx v, int o) {
    return {__shfl_down_sync(0xffffffffu, v.re, o), __shfl_down_sync(0xffffffffu, v.im, o)};
}
__device__ __forceinline__ double dadd(double a, double b) { return a + b; }
__device__ __forceinline__ float dadd(float a, float b) { return a + b; }
__device__ __forceinline__ cplx dadd(cplx a, cplx b) { return a + b; }

template <class P> __device__ __forceinline__ P warp_sum(P v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = dadd(v, shfl_down(v, o));
    return v;
}

// ----------------------------------------------------------------------------- operators
enum DevKind { DK_CD2D = 0, DK_CD3D = 1, DK_U1 = 2, DK_VAR2D = 3, DK_U1C = 4 };

// Device-side description of one operator level (passed by value to kernels).
// floor(n / d) for 0 <= n < 2^32 by one high multiply, add and shifts: unsigned division
// by an invariant integer (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, unsigned case): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n), q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
// A runtime integer division costs tens of instructions; the stencils need two or three per
// point, which bounded the float32 kernels.
struct FastDiv {
    unsigned m;
    int s1, s2;
    __host__ static FastDiv of(unsigned d) {
        int l = 0;
        while ((1ull << l) < d) ++l;
        FastDiv f;
        f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
        f.s1 = l < 1 ? l : 1;
        f.s2 = l > 1 ? l - 1 : 0;
        return f;
    }
    __device__ __forceinline__ unsigned div(unsigned n) const {
        const unsigned t = __umulhi(m, n);
        return (t + ((n - t) >> s1)) >> s2;
    }
};

struct DevOp {
    int kind;
    int N;          // points per axis (grids) or L (lattice)
    int n;          // unknowns (sites); the host rejects n >= 2^31
    FastDiv fN, fNN;   // division by N and by N^2 (set with the operator)
    // constant-coefficient stencil (cd2d / cd3d), already including 1/h^2 and beta/(2h)
    double c0, cxm, cxp, cym, cyp, czm, czp;
    // variable coefficient: coefficient arrays [5][n]: diag, west, east, south, north
    // (stored as the coefficient of u_nb in (A u)_ij, so y = sum coef * u)
    const double *vc;
    const float *vc32;
    // lattice
    const cplx *links;     // [4][V]
    double mdiag;          // m + 8
    // coarse lattice: [9][Vc]: diag, fwd mu=0..3, bwd mu=0..3
    const cplx *cst;
};

// float copies of the constant coefficients
struct DevOp32 {
    float c0, cxm, cxp, cym, cyp, czm, czp;
};

__host__ __device__ __forceinline__ int lat_shift(int x, int L, int mu, int sign) {
    int stride = 1;
    for (int a = 0; a < mu; ++a) stride *= L;
    int c = (x / stride) % L;
    int cn = c + sign;
    if (cn < 0) cn += L;
    if (cn >= L) cn -= L;
    return x + (cn - c) * stride;
}

// (A u)(idx) for real grids, u read through the functor `ld(j)`.
template <class T, class LD>
__device__ __forceinline__ T apply_real(const DevOp &op, const DevOp32 &o32, int idx, LD ld);

template <class LD>
__device__ __forceinline__ double apply_real_d(const DevOp &op, int idx, LD ld) {
    const int N = op.N;
    if (op.kind == DK_CD2D) {
        const int j = (int)op.fN.div((unsigned)idx), i = idx - j * N;
        double y = op.c0 * ld(idx);
        if (i > 0) y = fma(op.cxm, ld(idx - 1), y);
        if (i < N - 1) y = fma(op.cxp, ld(idx + 1), y);
        if (j > 0) y = fma(op.cym, ld(idx - N), y);
        if (j < N - 1) y = fma(op.cyp, ld(idx + N), y);
        return y;
    } else if (op.kind == DK_CD3D) {
        int NN = N * N;
        const int q = (int)op.fN.div((unsigned)idx), k = (int)op.fNN.div((unsigned)idx);
        const int i = idx - q * N, j = q - k * N;
        double y = op.c0 * ld(idx);
        if (i > 0) y = fma(op.cxm, ld(idx - 1), y);
        if (i < N - 1) y = fma(op.cxp, ld(idx + 1), y);
        if (j > 0) y = fma(op.cym, ld(idx - N), y);
        if (j < N - 1) y = fma(op.cyp, ld(idx + N), y);
        if (k > 0) y = fma(op.czm, ld(idx - NN), y);
        if (k < N - 1) y = fma(op.czp, ld(idx + NN), y);
        return y;
    } else {  // DK_VAR2D
        const int j = (int)op.fN.div((unsigned)idx), i = idx - j * N;
        const int n = op.n;
        const double *c = op.vc;
        double y = c[idx] * ld(idx);
        if (i > 0) y = fma(c[n + idx], ld(idx - 1), y);
        if (i < N - 1) y = fma(c[2 * n + idx], ld(idx + 1), y);
        if (j > 0) y = fma(c[3 * n + idx], ld(idx - N), y);
        if (j < N - 1) y = fma(c[4 * n + idx], ld(idx + N), y);
        return y;
    }
}

template <class LD>
__device__ __forceinline__ float apply_real_f(const DevOp &op, const DevOp32 &o, int idx, LD ld) {
    // every operand is loaded first (predicated on the boundary tests), then the terms are
    // summed in the fixed order of the float64 stencil: the loads of a point are in flight
    // together instead of one per dependent step of the sum (the float32 kernels are bound by
    // load latency)
    const int N = op.N;
    if (op.kind == DK_CD2D) {
        const int j = (int)op.fN.div((unsigned)idx), i = idx - j * N;
        const bool bw = i > 0, be = i < N - 1, bs = j > 0, bn = j < N - 1;
        const float xc = ld(idx);
        const float xw = bw ? ld(idx - 1) : 0.0f, xe = be ? ld(idx + 1) : 0.0f;
        const float xs = bs ? ld(idx - N) : 0.0f, xn = bn ? ld(idx + N) : 0.0f;
        float y = o.c0 * xc;
        y = bw ? fmaf(o.cxm, xw, y) : y;
        y = be ? fmaf(o.cxp, xe, y) : y;
        y = bs ? fmaf(o.cym, xs, y) : y;
        y = bn ? fmaf(o.cyp, xn, y) : y;
        return y;
    } else if (op.kind == DK_CD3D) {
        const int NN = N * N;
        const int q = (int)op.fN.div((unsigned)idx), k = (int)op.fNN.div((unsigned)idx);
        const int i = idx - q * N, j = q - k * N;
        const bool bw = i > 0, be = i < N - 1, bs = j > 0, bn = j < N - 1, bd = k > 0, bu = k < N - 1;
        const float xc = ld(idx);
        const float xw = bw ? ld(idx - 1) : 0.0f, xe = be ? ld(idx + 1) : 0.0f;
        const float xs = bs ? ld(idx - N) : 0.0f, xn = bn ? ld(idx + N) : 0.0f;
        const float xd = bd ? ld(idx - NN) : 0.0f, xu = bu ? ld(idx + NN) : 0.0f;
        float y = o.c0 * xc;
        y = bw ? fmaf(o.cxm, xw, y) : y;
        y = be ? fmaf(o.cxp, xe, y) : y;
        y = bs ? fmaf(o.cym, xs, y) : y;
        y = bn ? fmaf(o.cyp, xn, y) : y;
        y = bd ? fmaf(o.czm, xd, y) : y;
        y = bu ? fmaf(o.czp, xu, y) : y;
        return y;
    } else {
        const int j = (int)op.fN.div((unsigned)idx), i = idx - j * N;
        const int n = op.n;
        const float *c = op.vc32;
        const bool bw = i > 0, be = i < N - 1, bs = j > 0, bn = j < N - 1;
        const float xc = ld(idx), cc = c[idx];
        const float xw = bw ? ld(idx - 1) : 0.0f, cw = bw ? c[n + idx] : 0.0f;
        const float xe = be ? ld(idx + 1) : 0.0f, ce = be ? c[2 * n + idx] : 0.0f;
        const float xs = bs ? ld(idx - N) : 0.0f, cs = bs ? c[3 * n + idx] : 0.0f;
        const float xn = bn ? ld(idx + N) : 0.0f, cn = bn ? c[4 * n + idx] : 0.0f;
        float y = cc * xc;
        y = bw ? fmaf(cw, xw, y) : y;
        y = be ? fmaf(ce, xe, y) : y;
        y = bs ? fmaf(cs, xs, y) : y;
        y = bn ? fmaf(cn, xn, y) : y;
        return y;
    }
}

template <class LD>
__device__ __forceinline__ cplx apply_cplx(const DevOp &op, int x, LD ld) {
    const int L = op.N;
    if (op.kind == DK_U1) {
        const int V = op.n;
        cplx y = op.mdiag * ld(x);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            int xp = lat_shift(x, L, mu, +1), xm = lat_shift(x, L, mu, -1);
            cplx uf = op.links[mu * V + x];
            cplx ub = op.links[mu * V + xm];
            y = y - uf * ld(xp);
            y = y - conj(ub) * ld(xm);
        }
        return y;
    } else {  // DK_U1C: general 9-point coarse stencil
        const int V = op.n;
        cplx y = op.cst[x] * ld(x);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            int xp = lat_shift(x, L, mu, +1), xm = lat_shift(x, L, mu, -1);
            y = y + op.cst[(1 + mu) * V + x] * ld(xp);
            y = y + op.cst[(5 + mu) * V + x] * ld(xm);
        }
        return y;
    }
}

// Generic entry used by templated kernels.
template <class T> struct Apply;
template <> struct Apply<double> {
    template <class LD>
    __device__ static __forceinline__ double at(const DevOp &op, const DevOp32 &, int idx, LD ld) {
        return apply_real_d(op, idx, ld);
    }
};
template <> struct Apply<float> {
    template <class LD>
    __device__ static __forceinline__ float at(const DevOp &op, const DevOp32 &o, int idx, LD ld) {
        return apply_real_f(op, o, idx, ld);
    }
};
template <> struct Apply<cplx> {
    template <class LD>
    __device__ static __forceinline__ cplx at(const DevOp &op, const DevOp32 &, int idx, LD ld) {
        return apply_cplx(op, idx, ld);
    }
};

// ----------------------------------------------------------------------------- sizes
constexpr int kMaxM = 256;              // largest GMRES-DR / GMRES subspace dimension m, and
                                        // largest deflation basis k
constexpr int kMaxCols = kMaxM + 2;     // coefficient vectors staged per block (m + 1 columns)
constexpr int kSmallCols = 136;         // the staging size of the kernels' common instance

// ----------------------------------------------------------------------------- launch shape
constexpr int kThreads = 256;
int num_sms();
// Blocks for a grid-stride pass over n elements: a multiple of the SM count, at most
// `per_sm` resident blocks per SM, and no more blocks than there is work for.
int grid_for(int64_t n, int per_sm = 8);

// ----------------------------------------------------------------------------- reductions
// Deterministic two-level reduction: every block writes its partial sums (in a fixed
// order over its grid-stride elements) to `part[block * nd + d]`; the last block to
// finish (atomic ticket) adds the partials in block order and runs the finaliser.
struct RedSlot {
    void *part;          // nblocks * nd * sizeof(D)
    unsigned *ticket;    // one counter, zero between uses
};

template <class P, class D, int ND>
__device__ __forceinline__ void block_reduce_store(P (&v)[ND], D *part, D *red_smem) {
    // red_smem: (blockDim.x/32) * ND entries.  Warp sums in the per-thread type P,
    // block sums in D, both in a fixed order.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        P w = warp_sum(v[d]);
        if (lane == 0) red_smem[warp * ND + d] = to_d(w);
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        const int d = threadIdx.x;
        D s = red_smem[d];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = dadd(s, red_smem[w * ND + d]);
        part[(size_t)blockIdx.x * ND + d] = s;
    }
}

// Returns true in exactly one block (the last); that block's threads then see all partials.
__device__ __forceinline__ bool last_block(unsigned *ticket) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return am_last;
}

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ cplx ldcg(const cplx *p) {
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}

// In the last block: totals[d] = sum over blocks of part[b * ND + d].  A warp reduces each
// entry: lane l adds blocks l, l + 32, ... in order, then the lanes are combined by the
// fixed shuffle tree, so the result does not depend on block scheduling.
template <class D>
__device__ __forceinline__ D dzero() { return D{}; }

template <class D, int ND>
__device__ __forceinline__ void final_sum(const D *part, D *totals_smem, unsigned *ticket) {
    // warp w reduces entries w, w + 8, ... (more entries than warps take several rounds)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int d = warp; d < ND; d += nw) {
        D s = dzero<D>();
        for (int b = lane; b < (int)gridDim.x; b += 32) s = dadd(s, ldcg(part + (size_t)b * ND + d));
        s = warp_sum(s);
        if (lane == 0) totals_smem[d] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

}  // namespace tg
