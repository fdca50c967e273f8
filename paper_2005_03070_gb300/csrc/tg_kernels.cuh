// Templated device kernels of the tg library: stencil products, the BiCGStab iteration,
// residuals, tall-skinny products and reductions.  T is the vector element type:
// double (float64 path), float (inner iteration and coarse Arnoldi basis of the float32 +
// refinement path) or cplx (complex128 lattice).  Reductions of float vectors accumulate
// per thread in float and across threads and blocks in double.
#pragma once

#include <type_traits>

#include "tg_common.cuh"

namespace tg {

// ----------------------------------------------------------------------------- elementwise
__device__ __forceinline__ double axpy(double a, double x, double y) { return fma(a, x, y); }
__device__ __forceinline__ float axpy(float a, float x, float y) { return fmaf(a, x, y); }
__device__ __forceinline__ cplx axpy(cplx a, cplx x, cplx y) {
    return {fma(a.re, x.re, fma(-a.im, x.im, y.re)), fma(a.re, x.im, fma(a.im, x.re, y.im))};
}
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ float sub(float a, float b) { return a - b; }
__device__ __forceinline__ cplx sub(cplx a, cplx b) { return a - b; }
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ cplx neg(cplx a) { return -a; }

// kernel-side scalar of a reduction result
template <class T> struct KS;
template <> struct KS<double> { __device__ static double of(double d) { return d; } };
template <> struct KS<float> { __device__ static float of(double d) { return (float)d; } };
template <> struct KS<cplx> { __device__ static cplx of(cplx d) { return d; } };

__host__ __device__ __forceinline__ double dabs(double a) { return fabs(a); }
__host__ __device__ __forceinline__ double dabs(cplx a) { return hypot(a.re, a.im); }
__host__ __device__ __forceinline__ double dreal(double a) { return a; }
__host__ __device__ __forceinline__ double dreal(cplx a) { return a.re; }
__host__ __device__ __forceinline__ double ddiv(double a, double b) { return a / b; }
__host__ __device__ __forceinline__ cplx ddiv(cplx a, cplx b) { return cdiv(a, b); }
__host__ __device__ __forceinline__ double dmul(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ float dmul(float a, float b) { return a * b; }
__host__ __device__ __forceinline__ cplx dmul(cplx a, cplx b) { return a * b; }
__host__ __device__ __forceinline__ double dsub(double a, double b) { return a - b; }
__host__ __device__ __forceinline__ cplx dsub(cplx a, cplx b) { return a - b; }
__host__ __device__ __forceinline__ bool dfinite(double a) { return isfinite(a); }
__host__ __device__ __forceinline__ bool dfinite(cplx a) { return isfinite(a.re) && isfinite(a.im); }

template <class T> struct Part { using P = T; };          // per-thread partial type
template <> struct Part<float> { using P = float; };

// ----------------------------------------------------------------------------- y = A x
template <class T>
__global__ void __launch_bounds__(kThreads) k_apply(DevOp op, DevOp32 o32, const T *__restrict__ x,
                                                     T *__restrict__ y) {
    const int n = op.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = Apply<T>::at(op, o32, i, [&](int j) { return x[j]; });
}

// ----------------------------------------------------------------------------- norms
// out[0] = ||a||^2 (and out[1] = <a, b> when b != nullptr); deterministic.
template <class T>
__global__ void __launch_bounds__(kThreads) k_dot(const T *__restrict__ a, const T *__restrict__ b, int n,
                                                   typename ST<T>::D *part, unsigned *ticket,
                                                   typename ST<T>::D *out) {
    using D = typename ST<T>::D;
    using P = typename Part<T>::P;
    __shared__ D red[(kThreads / 32) * 2];
    __shared__ D tot[2];
    P acc[2] = {ST<T>::zero(), ST<T>::zero()};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T ai = a[i];
        acc[0] = ST<T>::fma_cm(ai, ai, acc[0]);
        if (b) acc[1] = ST<T>::fma_cm(ai, b[i], acc[1]);
    }
    block_reduce_store<P, D, 2>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 2>(part, tot, ticket);
        if (threadIdx.x == 0) {
            out[0] = tot[0];
            out[1] = tot[1];
        }
    }
}

// ----------------------------------------------------------------------------- true residual
// r = b - A x in the outer precision (double / cplx); out[0] = ||r||^2, out[1] = ||b||^2.
template <class T>
__global__ void __launch_bounds__(kThreads) k_residual(DevOp op, const T *__restrict__ b, const T *__restrict__ x,
                                                        T *__restrict__ r, typename ST<T>::D *part,
                                                        unsigned *ticket, typename ST<T>::D *out) {
    using D = typename ST<T>::D;
    __shared__ D red[(kThreads / 32) * 2];
    __shared__ D tot[2];
    DevOp32 o32{};
    T acc[2] = {ST<T>::zero(), ST<T>::zero()};
    const int n = op.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T ax = Apply<T>::at(op, o32, i, [&](int j) { return x[j]; });
        T bi = b[i];
        T ri = sub(bi, ax);
        r[i] = ri;
        acc[0] = ST<T>::fma_cm(ri, ri, acc[0]);
        acc[1] = ST<T>::fma_cm(bi, bi, acc[1]);
    }
    block_reduce_store<T, D, 2>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 2>(part, tot, ticket);
        if (threadIdx.x == 0) {
            out[0] = tot[0];
            out[1] = tot[1];
        }
    }
}

// ----------------------------------------------------------------------------- BiCGStab
// Device-resident state of one BiCGStab cycle.  Kernels of an iteration read the
// scalars they need from here; the last block of each reduction writes the next ones,
// so the host only launches and, once per batch of iterations, reads `status`.
template <class D>
struct BiState {
    D rho;          // <r_hat, r> for the current r
    D alpha, omega, beta;
    D rho_next;
    double rr;      // ||r||^2 (last full step)
    double ss;      // ||s||^2 (last half step)
    double target2; // (rticyc ||r_cycle_start||)^2
    double div2;    // divergence bound: the cycle stops (status 5) once ||r||^2 exceeds it
    int mvps;       // operator applications in this cycle
    int cap;        // at most this many (INT_MAX: no cap)
    int iters;
    int status;     // 0 running, 1 converged, 2 breakdown, 3 capped, 4 NaN, 5 diverged
    int half;       // a half-step exit is pending: the t-kernel skips, the x-kernel applies omega = 0
    int pending;    // status to take when the pending half step is applied
};

constexpr double kTiny = 1e-300;

// r_hat = r, p = r; rho = <r, r>.
template <class T>
__global__ void __launch_bounds__(kThreads) k_bi_init(const T *__restrict__ r, T *__restrict__ rh,
                                                       T *__restrict__ p, int n, double target2, int cap,
                                                       typename ST<T>::D *part, unsigned *ticket,
                                                       BiState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    using P = typename Part<T>::P;
    __shared__ D red[(kThreads / 32)];
    __shared__ D tot[1];
    P acc[1] = {ST<T>::zero()};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T ri = r[i];
        rh[i] = ri;
        p[i] = ri;
        acc[0] = ST<T>::fma_cm(ri, ri, acc[0]);
    }
    block_reduce_store<P, D, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            D rho = tot[0];
            st->rho = rho;
            st->rr = dreal(rho);
            st->ss = 0.0;
            st->target2 = target2;
            // float32 cycles stop once ||r|| has grown 1e8-fold (divergence on its way to
            // overflow; transient BiCGStab peaks stay far below that); float64 cycles never
            st->div2 = sizeof(T) == 4 ? 1e16 * dreal(rho) : 1.7e308;
            st->mvps = 0;
            st->cap = cap;
            st->iters = 0;
            st->half = 0;
            st->pending = 0;
            st->alpha = st->omega = st->beta = st->rho_next = rho;
            if (!dfinite(rho)) st->status = 4;
            else if (dreal(rho) <= target2) st->status = 1;
            else if (dabs(rho) < kTiny) st->status = 2;
            else st->status = 0;
        }
    }
}

// v = A p; sigma = <r_hat, v>; alpha = rho / sigma.
template <class T>
__global__ void __launch_bounds__(kThreads) k_bi_v(DevOp op, DevOp32 o32, const T *__restrict__ p,
                                                    const T *__restrict__ rh, T *__restrict__ v,
                                                    typename ST<T>::D *part, unsigned *ticket,
                                                    BiState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    using P = typename Part<T>::P;
    if (st->status != 0) return;
    __shared__ D red[(kThreads / 32)];
    __shared__ D tot[1];
    P acc[1] = {ST<T>::zero()};
    const int n = op.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T y = Apply<T>::at(op, o32, i, [&](int j) { return p[j]; });
        v[i] = y;
        acc[0] = ST<T>::fma_cm(rh[i], y, acc[0]);
    }
    block_reduce_store<P, D, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            D sigma = tot[0];
            st->mvps += 1;
            if (!dfinite(sigma)) st->status = 4;
            else if (dabs(sigma) < kTiny) st->status = 2;
            else st->alpha = ddiv(st->rho, sigma);
        }
    }
}

// s = r - alpha v; ||s||^2; half-step convergence / cap test.
template <class T>
__global__ void __launch_bounds__(kThreads) k_bi_s(const T *__restrict__ r, const T *__restrict__ v,
                                                    T *__restrict__ s, int n, typename ST<T>::D *part,
                                                    unsigned *ticket, BiState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    using P = typename Part<T>::P;
    if (st->status != 0) return;
    __shared__ D red[(kThreads / 32)];
    __shared__ D tot[1];
    const T malpha = neg(KS<T>::of(st->alpha));
    P acc[1] = {ST<T>::zero()};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T si = axpy(malpha, v[i], r[i]);
        s[i] = si;
        acc[0] = ST<T>::fma_cm(si, si, acc[0]);
    }
    block_reduce_store<P, D, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            double ss = dreal(tot[0]);
            st->ss = ss;
            if (!isfinite(ss)) st->status = 4;
            else if (ss <= st->target2) { st->half = 1; st->pending = 1; }
            else if (ss > st->div2) st->status = 5;
            else if (st->mvps >= st->cap) { st->half = 1; st->pending = 3; }
        }
    }
}

// t = A s; <t,s>, <t,t>, <r_hat,s>, <r_hat,t>; omega = <t,s>/<t,t>;
// rho_next = <r_hat, s - omega t> = <r_hat,s> - omega <r_hat,t>; beta = (rho_next/rho)(alpha/omega).
template <class T>
__global__ void __launch_bounds__(kThreads) k_bi_t(DevOp op, DevOp32 o32, const T *__restrict__ s,
                                                    const T *__restrict__ rh, T *__restrict__ t,
                                                    typename ST<T>::D *part, unsigned *ticket,
                                                    BiState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    using P = typename Part<T>::P;
    if (st->status != 0 || st->half) return;
    __shared__ D red[(kThreads / 32) * 4];
    __shared__ D tot[4];
    P acc[4] = {ST<T>::zero(), ST<T>::zero(), ST<T>::zero(), ST<T>::zero()};
    const int n = op.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T ti = Apply<T>::at(op, o32, i, [&](int j) { return s[j]; });
        t[i] = ti;
        T si = s[i], ri = rh[i];
        acc[0] = ST<T>::fma_cm(ti, si, acc[0]);
        acc[1] = ST<T>::fma_cm(ti, ti, acc[1]);
        acc[2] = ST<T>::fma_cm(ri, si, acc[2]);
        acc[3] = ST<T>::fma_cm(ri, ti, acc[3]);
    }
    block_reduce_store<P, D, 4>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 4>(part, tot, ticket);
        if (threadIdx.x == 0) {
            st->mvps += 1;
            double tt = dreal(tot[1]);
            if (!isfinite(tt) || !dfinite(tot[0])) {
                st->status = 4;
            } else if (tt < kTiny) {
                st->half = 1;
                st->pending = 2;
            } else {
                D omega = ddiv(tot[0], D(tot[1]));
                st->omega = omega;
                D rn = dsub(tot[2], dmul(omega, tot[3]));
                st->rho_next = rn;
                if (dabs(omega) >= kTiny)
                    st->beta = dmul(ddiv(rn, st->rho), ddiv(st->alpha, omega));
            }
        }
    }
}

// Full step: x += alpha p + omega s; r = s - omega t; p = r + beta (p - omega v); ||r||^2.
// Pending half step: x += alpha p; r = s.
template <class T>
__global__ void __launch_bounds__(kThreads) k_bi_x(T *__restrict__ x, T *__restrict__ r, T *__restrict__ p,
                                                    const T *__restrict__ s, const T *__restrict__ t,
                                                    const T *__restrict__ v, int n, typename ST<T>::D *part,
                                                    unsigned *ticket, BiState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    using P = typename Part<T>::P;
    if (st->status != 0) return;
    __shared__ D red[(kThreads / 32)];
    __shared__ D tot[1];
    const T alpha = KS<T>::of(st->alpha);
    if (st->half) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            x[i] = axpy(alpha, p[i], x[i]);
            r[i] = s[i];
        }
        if (last_block(ticket)) {
            if (threadIdx.x == 0) {
                *ticket = 0u;
                st->rr = st->ss;
                st->status = st->pending;
                st->iters += 1;
            }
        }
        return;
    }
    const T omega = KS<T>::of(st->omega);
    const T momega = neg(omega);
    const T beta = KS<T>::of(st->beta);
    P acc[1] = {ST<T>::zero()};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T si = s[i];
        T pi = p[i];
        x[i] = axpy(omega, si, axpy(alpha, pi, x[i]));
        T ri = axpy(momega, t[i], si);
        r[i] = ri;
        p[i] = axpy(beta, axpy(momega, v[i], pi), ri);
        acc[0] = ST<T>::fma_cm(ri, ri, acc[0]);
    }
    block_reduce_store<P, D, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            double rr = dreal(tot[0]);
            st->rr = rr;
            st->iters += 1;
            st->rho = st->rho_next;
            if (!isfinite(rr)) st->status = 4;
            else if (rr <= st->target2) st->status = 1;
            else if (rr > st->div2) st->status = 5;
            else if (dabs(st->omega) < kTiny) st->status = 2;
            else if (dabs(st->rho_next) < kTiny) st->status = 2;
            else if (st->mvps >= st->cap) st->status = 3;
        }
    }
}

// ----------------------------------------------------------------------------- float32 streaming updates, 4 points per thread
// The float32 BiCGStab updates touch only their own points: thread g takes the 4 consecutive
// points 4g .. 4g + 3 as aligned float4, 16 bytes per request, so each thread keeps four
// times the DRAM bytes of the one-point kernels in flight.  A partial last group runs the
// one-point code.
__device__ __forceinline__ float4 ld4(const float *__restrict__ p, int a) {
    return *reinterpret_cast<const float4 *>(p + a);
}

// k_bi_s for float32 with 16-byte aligned vectors, 4 points per thread: s = r - alpha v, <s,s>.
__global__ void __launch_bounds__(kThreads) k_bi_s_f4(const float *__restrict__ r, const float *__restrict__ v,
                                                       float *__restrict__ s, int n, double *part,
                                                       unsigned *ticket, BiState<double> *st) {
    if (st->status != 0) return;
    __shared__ double red[(kThreads / 32)];
    __shared__ double tot[1];
    const float malpha = -(float)st->alpha;
    float acc[1] = {0.0f};
    const int ng = n >> 2;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const float4 rv = ld4(r, 4 * g), vv = ld4(v, 4 * g);
        const float4 sv = make_float4(fmaf(malpha, vv.x, rv.x), fmaf(malpha, vv.y, rv.y),
                                      fmaf(malpha, vv.z, rv.z), fmaf(malpha, vv.w, rv.w));
        *reinterpret_cast<float4 *>(s + 4 * g) = sv;
        acc[0] = fmaf(sv.x, sv.x, acc[0]);
        acc[0] = fmaf(sv.y, sv.y, acc[0]);
        acc[0] = fmaf(sv.z, sv.z, acc[0]);
        acc[0] = fmaf(sv.w, sv.w, acc[0]);
    }
    for (int i = 4 * ng + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float si = fmaf(malpha, v[i], r[i]);
        s[i] = si;
        acc[0] = fmaf(si, si, acc[0]);
    }
    block_reduce_store<float, double, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<double, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            const double ss = tot[0];
            st->ss = ss;
            if (!isfinite(ss)) st->status = 4;
            else if (ss <= st->target2) { st->half = 1; st->pending = 1; }
            else if (ss > st->div2) st->status = 5;
            else if (st->mvps >= st->cap) { st->half = 1; st->pending = 3; }
        }
    }
}

// k_bi_x for float32 with 16-byte aligned vectors, 4 points per thread: x += alpha p + omega s,
// r = s - omega t, p = r + beta (p - omega v), <r,r> (or the half step x += alpha p, r = s).
__device__ __forceinline__ float4 f4_axpy(float a, const float4 &x, const float4 &y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__global__ void __launch_bounds__(kThreads) k_bi_x_f4(float *__restrict__ x, float *__restrict__ r,
                                                       float *__restrict__ p, const float *__restrict__ s,
                                                       const float *__restrict__ t, const float *__restrict__ v,
                                                       int n, double *part, unsigned *ticket, BiState<double> *st) {
    if (st->status != 0) return;
    __shared__ double red[(kThreads / 32)];
    __shared__ double tot[1];
    const float alpha = (float)st->alpha;
    const int ng = n >> 2;
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    if (st->half) {
        for (int g = g0; g < ng; g += gs) {
            *reinterpret_cast<float4 *>(x + 4 * g) = f4_axpy(alpha, ld4(p, 4 * g), ld4(x, 4 * g));
            *reinterpret_cast<float4 *>(r + 4 * g) = ld4(s, 4 * g);
        }
        for (int i = 4 * ng + g0; i < n; i += gs) {
            x[i] = fmaf(alpha, p[i], x[i]);
            r[i] = s[i];
        }
        if (last_block(ticket)) {
            if (threadIdx.x == 0) {
                *ticket = 0u;
                st->rr = st->ss;
                st->status = st->pending;
                st->iters += 1;
            }
        }
        return;
    }
    const float omega = (float)st->omega, momega = -omega, beta = (float)st->beta;
    float acc[1] = {0.0f};
    for (int g = g0; g < ng; g += gs) {
        const float4 sv = ld4(s, 4 * g), pv = ld4(p, 4 * g);
        *reinterpret_cast<float4 *>(x + 4 * g) = f4_axpy(omega, sv, f4_axpy(alpha, pv, ld4(x, 4 * g)));
        const float4 rv = f4_axpy(momega, ld4(t, 4 * g), sv);
        *reinterpret_cast<float4 *>(r + 4 * g) = rv;
        *reinterpret_cast<float4 *>(p + 4 * g) = f4_axpy(beta, f4_axpy(momega, ld4(v, 4 * g), pv), rv);
        acc[0] = fmaf(rv.x, rv.x, acc[0]);
        acc[0] = fmaf(rv.y, rv.y, acc[0]);
        acc[0] = fmaf(rv.z, rv.z, acc[0]);
        acc[0] = fmaf(rv.w, rv.w, acc[0]);
    }
    for (int i = 4 * ng + g0; i < n; i += gs) {
        const float si = s[i], pi = p[i];
        x[i] = fmaf(omega, si, fmaf(alpha, pi, x[i]));
        const float ri = fmaf(momega, t[i], si);
        r[i] = ri;
        p[i] = fmaf(beta, fmaf(momega, v[i], pi), ri);
        acc[0] = fmaf(ri, ri, acc[0]);
    }
    block_reduce_store<float, double, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<double, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            const double rr = tot[0];
            st->rr = rr;
            st->iters += 1;
            st->rho = st->rho_next;
            if (!isfinite(rr)) st->status = 4;
            else if (rr <= st->target2) st->status = 1;
            else if (rr > st->div2) st->status = 5;
            else if (fabs(st->omega) < kTiny) st->status = 2;
            else if (fabs(st->rho_next) < kTiny) st->status = 2;
            else if (st->mvps >= st->cap) st->status = 3;
        }
    }
}

// ----------------------------------------------------------------------------- tall-skinny
// Partial products of h = V^H w over row tiles: part[block][c] = sum over the block's rows
// of conj(V[row, c]) w[row], c < ncol.  Columns come in groups of kGemvTCols (blockIdx.y);
// within a group warp w owns columns w, w + 8, ...; each pass covers 128 rows (4 rows per
// lane) so that four loads per column are in flight per lane.
constexpr int kGemvTCols = 136;          // 8 warps x 17 columns
template <class T>
__global__ void __launch_bounds__(kThreads) k_gemv_t_part(const T *__restrict__ V, size_t ldv, int ncol,
                                                           const T *__restrict__ w, int n,
                                                           typename ST<T>::D *part, const int *cond = nullptr) {
    using P = typename Part<T>::P;
    if (cond && !*cond) return;     // a skipped re-orthogonalisation pass
    constexpr int kMaxPerWarp = kGemvTCols / 8;
    constexpr int kU = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cbase = blockIdx.y * kGemvTCols;
    P acc[kMaxPerWarp];
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) acc[q] = ST<T>::zero();
    for (int row0 = blockIdx.x * 32 * kU; row0 < n; row0 += gridDim.x * 32 * kU) {
        T wv[kU];
        int rr[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            rr[u] = row0 + 32 * u + lane;
            wv[u] = rr[u] < n ? w[rr[u]] : ST<T>::zero();
        }
#pragma unroll
        for (int q = 0; q < kMaxPerWarp; ++q) {
            const int c = cbase + warp + 8 * q;
            if (c < ncol) {
                const T *vc = V + (size_t)c * ldv;
                T vv[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) vv[u] = rr[u] < n ? vc[rr[u]] : ST<T>::zero();
#pragma unroll
                for (int u = 0; u < kU; ++u) acc[q] = ST<T>::fma_cm(vv[u], wv[u], acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) {
        const int c = cbase + warp + 8 * q;
        if (c < ncol) {       // reduce only the columns this warp owns
            P s = warp_sum(acc[q]);
            if (lane == 0) part[(size_t)blockIdx.x * ncol + c] = to_d(s);
        }
    }
}

// h = V^H w partials for a float64 or float32 V with 16-byte aligned columns (V and w
// 16-byte aligned, ldv a multiple of 16 bytes and >= the rows rounded up to whole chunks):
// the rows are walked in chunks of PipeRows<E> rows (64 float64 / 128 float32 rows, 512
// bytes per column) staged in shared memory by a 3-deep cp.async pipeline, so that loads of
// the next chunks are in flight while the arithmetic pipe works on the current one.  Block
// b takes chunks b, b + G, ...  Columns come in groups of kPipeCols (blockIdx.y); within a
// group warp w owns columns w, w + 8, ...; lane l rows l + 32 u of a chunk.  Accumulation in
// E; partials written as float64 to part[block x][column].  Shared memory:
// 3 x (group columns + 1) x PipeRows<E> elements (w is the extra column).
template <class E> struct PipeRows;
template <> struct PipeRows<double> { static constexpr int value = 64; };
template <> struct PipeRows<float> { static constexpr int value = 128; };
constexpr int kPipeRows = 64;          // float64 chunk (the float32 chunk holds the same bytes)
constexpr int kPipeStages = 3;
constexpr int kPipeCols = 128;         // columns per group: 3 x 129 x 512 B of shared memory

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <class E>
__global__ void __launch_bounds__(kThreads, 2) k_gemv_t_pipe(const E *__restrict__ V, size_t ldv, int ncol,
                                                           const E *__restrict__ w, int n, double *part) {
    constexpr int kMaxPerWarp = kPipeCols / 8;
    constexpr int R = PipeRows<E>::value;
    constexpr int PE = 16 / sizeof(E);           // elements per 16-byte piece
    constexpr int U = R / 32;                    // rows per lane per chunk
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E *buf = reinterpret_cast<E *>(smem_raw);
    const int cbase = blockIdx.y * kPipeCols;    // this block's columns: cbase .. cbase + ng - 1
    const int ncol_all = ncol;
    ncol = min(ncol_all - cbase, kPipeCols);
    V += (size_t)cbase * ldv;
    const int cols = ncol + 1;                      // w staged as column ncol
    const size_t stage_elems = (size_t)cols * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nchunks = (n + R - 1) / R;
    const int G = gridDim.x;
    const int mine = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / G + 1 : 0;
    auto issue = [&](int it) {
        if (it < mine) {
            const size_t row0 = (size_t)(blockIdx.x + (size_t)it * G) * R;
            E *dst = buf + (size_t)(it % kPipeStages) * stage_elems;
            // (cols x R rows) as 16-byte pieces: piece e -> column e / (R / PE), rows PE (e % (R / PE)) ..
            for (int e = threadIdx.x; e < cols * (R / PE); e += blockDim.x) {
                const int c = e / (R / PE), rp = e % (R / PE);
                const E *src = (c < ncol ? V + (size_t)c * ldv : w) + row0 + PE * rp;
                cp_async16(dst + (size_t)c * R + PE * rp, src);
            }
        }
        cp_async_commit();
    };
    E acc[kMaxPerWarp];
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) acc[q] = E(0);
#pragma unroll
    for (int s = 0; s < kPipeStages - 1; ++s) issue(s);
    for (int it = 0; it < mine; ++it) {
        cp_async_wait<kPipeStages - 2>();
        __syncthreads();
        issue(it + kPipeStages - 1);              // the buffer of iteration it - 1, read by everyone already
        const E *st = buf + (size_t)(it % kPipeStages) * stage_elems;
        const int row0 = (blockIdx.x + it * G) * R;
        E wv[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = row0 + lane + 32 * u < n;
            wv[u] = ok[u] ? st[(size_t)ncol * R + lane + 32 * u] : E(0);
        }
#pragma unroll
        for (int q = 0; q < kMaxPerWarp; ++q) {
            const int c = warp + 8 * q;
            if (c < ncol) {
                const E *sc = st + (size_t)c * R;
#pragma unroll
                for (int u = 0; u < U; ++u) acc[q] = fma(ok[u] ? sc[lane + 32 * u] : E(0), wv[u], acc[q]);
            }
        }
    }
    cp_async_wait<0>();
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) {
        const int c = warp + 8 * q;
        if (c < ncol) {
            const E s = warp_sum(acc[q]);
            if (lane == 0) part[(size_t)blockIdx.x * ncol_all + cbase + c] = (double)s;
        }
    }
}

// out[e] (mode 0: =, mode 1: +=) sum_b part[b * nent + e].  One warp per entry: lane l
// adds blocks l, l + 32, ... in order, then the fixed shuffle tree (deterministic).
template <class D>
__global__ void k_sum_part(const D *__restrict__ part, int nblk, int nent, D *out, int mode,
                           const int *cond = nullptr) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (e >= nent) return;
    if (cond && !*cond) {           // skipped pass: its coefficients are zero
        if (lane == 0 && !mode) out[e] = D{};
        return;
    }
    D s = D{};
    for (int b = lane; b < nblk; b += 32) s = dadd(s, part[(size_t)b * nent + e]);
    s = warp_sum(s);
    if (lane == 0) out[e] = mode ? dadd(out[e], s) : s;
}

// w[row] += sign * sum_c V[row, c] h[c]   (h: device, D type, ncol <= MC).  The coefficient
// kernels take their staging size MC as a template argument: a small instance (136) for the
// usual column counts keeps the static shared memory of each block at the size it needs
// (the kMaxCols instance was 15% slower on the Arnoldi update at 60 columns).
template <class T, int MC = kMaxCols>
__global__ void __launch_bounds__(kThreads) k_gemv_n(const T *__restrict__ V, size_t ldv, int ncol,
                                                      const typename ST<T>::D *__restrict__ h, double sign,
                                                      T *__restrict__ w, int n) {
    // coefficients converted to the vector type once per block (a per-element float64 ->
    // float32 conversion would run on the float64 pipe)
    __shared__ T hs[MC];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) hs[c] = KS<T>::of(h[c]);
    __syncthreads();
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        T acc = ST<T>::zero();
        for (int c = 0; c < ncol; ++c) acc = axpy(hs[c], V[(size_t)c * ldv + row], acc);
        w[row] = sign > 0 ? dadd(w[row], acc) : sub(w[row], acc);
    }
}

// Arnoldi orthogonalisation pass: w -= V h (ncol columns), then ||w||^2 (deterministic);
// the last block writes nrm2_out[0] and, when flag_out is given, the selective
// re-orthogonalisation decision (Daniel, Gragg, Kaufman and Stewart): a second pass is
// needed when the pass cancelled more than half of ||w||^2, i.e. ||w_new||^2 < eta2 ||w||^2
// with ||w||^2 = real(nrm2_before[0]).  cond: skip the whole kernel when *cond == 0.
template <class T, int MC = kMaxCols>
__global__ void __launch_bounds__(kThreads) k_gemv_n_norm(const T *__restrict__ V, size_t ldv, int ncol,
                                                           const typename ST<T>::D *__restrict__ h,
                                                           T *__restrict__ w, int n, const int *cond,
                                                           typename ST<T>::D *part, unsigned *ticket,
                                                           double *nrm2_out,
                                                           const typename ST<T>::D *nrm2_before,
                                                           int *flag_out, double eta2) {
    using D = typename ST<T>::D;
    using P = typename Part<T>::P;
    if (cond && !*cond) return;
    __shared__ T hs[MC];         // coefficients in the vector type, converted once per block
    __shared__ D red[(kThreads / 32)];
    __shared__ D tot[1];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) hs[c] = KS<T>::of(h[c]);
    __syncthreads();
    P acc[1] = {ST<T>::zero()};
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        T a = ST<T>::zero();
        for (int c = 0; c < ncol; ++c) a = axpy(hs[c], V[(size_t)c * ldv + row], a);
        const T wv = sub(w[row], a);
        w[row] = wv;
        acc[0] = ST<T>::fma_cm(wv, wv, acc[0]);
    }
    block_reduce_store<P, D, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            const double nn = dreal(tot[0]);
            nrm2_out[0] = nn;
            if (flag_out) flag_out[0] = (nn < eta2 * dreal(nrm2_before[0])) ? 1 : 0;
        }
    }
}

// k_gemv_n_norm for float32 V with 16-byte aligned columns (ldv a multiple of 4, V and w
// 16-byte aligned): each thread takes 4 consecutive rows as float4 loads; the rows beyond
// the last whole group of 4 are taken one by one by the first threads.
template <int MC = kMaxCols>
__global__ void __launch_bounds__(kThreads) k_gemv_n_norm_f4(const float *__restrict__ V, size_t ldv, int ncol,
                                                              const double *__restrict__ h, float *__restrict__ w,
                                                              int n, double *part, unsigned *ticket,
                                                              double *nrm2_out) {
    __shared__ float hs[MC];
    __shared__ double red[(kThreads / 32)];
    __shared__ double tot[1];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) hs[c] = (float)h[c];
    __syncthreads();
    float acc[1] = {0.0f};
    const int n4 = n >> 2;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += gridDim.x * blockDim.x) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < ncol; ++c) {
            const float4 v = reinterpret_cast<const float4 *>(V + (size_t)c * ldv)[g];
            const float hc = hs[c];
            a.x = fmaf(hc, v.x, a.x); a.y = fmaf(hc, v.y, a.y); a.z = fmaf(hc, v.z, a.z); a.w = fmaf(hc, v.w, a.w);
        }
        float4 wv = reinterpret_cast<float4 *>(w)[g];
        wv.x -= a.x; wv.y -= a.y; wv.z -= a.z; wv.w -= a.w;
        reinterpret_cast<float4 *>(w)[g] = wv;
        acc[0] = fmaf(wv.x, wv.x, fmaf(wv.y, wv.y, fmaf(wv.z, wv.z, fmaf(wv.w, wv.w, acc[0]))));
    }
    for (int row = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        float a = 0.0f;
        for (int c = 0; c < ncol; ++c) a = fmaf(hs[c], V[(size_t)c * ldv + row], a);
        const float wv = w[row] - a;
        w[row] = wv;
        acc[0] = fmaf(wv, wv, acc[0]);
    }
    block_reduce_store<float, double, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<double, 1>(part, tot, ticket);
        if (threadIdx.x == 0) nrm2_out[0] = tot[0];
    }
}

// Out (n x q) = In (n x p) * S (p x q), float32 In, float64 S (column-major, leading
// dimension lds, staged once per block as float32), float32 accumulation, Out float32 or
// float64.  In needs 16-byte aligned columns and ldi >= n rounded up to 64 rows: 64-row
// tiles of In are copied to shared memory by cp.async, double buffered (rows past n are read
// from the padding and never stored).  Register tiles: thread (rg, cg), rg, cg < 16,
// computes rows 4 rg .. 4 rg + 3 and columns cg + 16 j (j < CPT, q <= 16 CPT), reading its 4
// rows of each In column as one float4 (float32 Out: written as float4 too).
template <class TO, int CPT>
__global__ void __launch_bounds__(kThreads) k_tsm_f(const float *__restrict__ In, size_t ldi, int p,
                                                     const double *__restrict__ S, int lds, int q,
                                                     TO *__restrict__ Out, size_t ldo, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tiles = reinterpret_cast<float *>(smem_raw);         // 2 x [p][64]
    float *Ss = tiles + (size_t)2 * p * 64;                     // [q][p]
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
        const int i = e % p, c = e / p;
        Ss[e] = (float)S[i + (size_t)c * lds];
    }
    const int ntiles = (n + 63) / 64;
    const int mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto issue = [&](int it) {
        if (it < mine) {
            const size_t row0 = (size_t)(blockIdx.x + (size_t)it * gridDim.x) * 64;
            float *dst = tiles + (size_t)(it & 1) * p * 64;
            for (int e = threadIdx.x; e < p * 16; e += blockDim.x) {     // 16-byte pieces
                const int c = e >> 4, rp = e & 15;
                cp_async16(dst + (size_t)c * 64 + 4 * rp, In + (size_t)c * ldi + row0 + 4 * rp);
            }
        }
        cp_async_commit();
    };
    const int rg = threadIdx.x & 15, cg = threadIdx.x >> 4;
    issue(0);
    for (int it = 0; it < mine; ++it) {
        issue(it + 1);                           // the other buffer, released by the barrier below
        cp_async_wait<1>();
        __syncthreads();
        const float *tile = tiles + (size_t)(it & 1) * p * 64;
        const int row0 = (blockIdx.x + it * gridDim.x) * 64;
        float acc[CPT][4];
#pragma unroll
        for (int j = 0; j < CPT; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[j][u] = 0.0f;
        // columns past q read row 0 of S's staging (valid memory) and are never stored
        int soff[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) soff[j] = (cg + 16 * j < q ? cg + 16 * j : 0) * p;
        for (int i = 0; i < p; ++i) {
            const float4 v = reinterpret_cast<const float4 *>(tile + (size_t)i * 64)[rg];
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const float sv = Ss[soff[j] + i];
                acc[j][0] = fmaf(sv, v.x, acc[j][0]);
                acc[j][1] = fmaf(sv, v.y, acc[j][1]);
                acc[j][2] = fmaf(sv, v.z, acc[j][2]);
                acc[j][3] = fmaf(sv, v.w, acc[j][3]);
            }
        }
        const int rowb = row0 + 4 * rg;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = cg + 16 * j;
            if (c >= q) continue;
            TO *oc = Out + (size_t)c * ldo;
            if (std::is_same<TO, float>::value && rowb + 3 < n && ldo % 4 == 0) {
                *reinterpret_cast<float4 *>(oc + rowb) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (rowb + u < n) oc[rowb + u] = (TO)acc[j][u];
            }
        }
        __syncthreads();                         // everyone is done with this buffer
    }
    cp_async_wait<0>();
}

// Hbar column j: H[i] = h1[i] + h2[i] (i <= j), H[j+1] = sqrt(nrm2[0]), inv[0] = 1/H[j+1].
// HT is the Hessenberg type: the basis type, or float64 for a float32 basis.
template <class T, class HT = T>
__global__ void k_arnoldi_finish2(const typename ST<T>::D *h1, const typename ST<T>::D *h2, const double *nrm2,
                                  int j, HT *Hcol, double *inv) {
    for (int i = threadIdx.x; i <= j; i += blockDim.x) Hcol[i] = dadd(h1[i], h2[i]);
    if (threadIdx.x == 0) {
        const double nn = sqrt(nrm2[0]);
        HT hv = ST<HT>::zero();
        *reinterpret_cast<double *>(&hv) = nn;
        Hcol[j + 1] = hv;
        inv[0] = nn > 0 ? 1.0 / nn : 0.0;
    }
}

// Projection update: x += B1 d; r -= B2 e.  (B1, B2: n x k; d, e: device D vectors.)
template <class T, int MC = kMaxCols>
__global__ void __launch_bounds__(kThreads) k_proj_update(const T *__restrict__ B1, const T *__restrict__ B2,
                                                           size_t ld, int k,
                                                           const typename ST<T>::D *__restrict__ d,
                                                           const typename ST<T>::D *__restrict__ e,
                                                           T *__restrict__ x, T *__restrict__ r, int n) {
    __shared__ T ds[MC], es[MC];   // in the vector type, converted once per block
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        ds[c] = KS<T>::of(d[c]);
        es[c] = KS<T>::of(e[c]);
    }
    __syncthreads();
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        T ax = ST<T>::zero(), ar = ST<T>::zero();
        for (int c = 0; c < k; ++c) {
            ax = axpy(ds[c], B1[(size_t)c * ld + row], ax);
            ar = axpy(es[c], B2[(size_t)c * ld + row], ar);
        }
        x[row] = dadd(x[row], ax);
        r[row] = sub(r[row], ar);
    }
}

// Out (n x q) = In (n x p) * S (p x q), S column-major with leading dimension lds.
// 32-row tiles of In staged in shared memory (column-major [p][32]).
template <class T>
__global__ void __launch_bounds__(kThreads) k_tsm(const T *__restrict__ In, size_t ldi, int p,
                                                   const T *__restrict__ S, int lds, int q,
                                                   T *__restrict__ Out, size_t ldo, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    for (int row0 = blockIdx.x * 32; row0 < n; row0 += gridDim.x * 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * p; e += blockDim.x) {
            const int r = e & 31, c = e >> 5;
            const int row = row0 + r;
            tile[c * 32 + r] = row < n ? In[(size_t)c * ldi + row] : ST<T>::zero();
        }
        __syncthreads();
        for (int o = threadIdx.x; o < 32 * q; o += blockDim.x) {
            const int r = o & 31, c = o >> 5;
            const int row = row0 + r;
            T acc = ST<T>::zero();
            const T *sc = S + (size_t)c * lds;
            for (int i = 0; i < p; ++i) acc = axpy(sc[i], tile[i * 32 + r], acc);
            if (row < n) Out[(size_t)c * ldo + row] = acc;
        }
    }
}

// Partial Gram products G = A^H B over 32-row tiles, on a packed list of output entries:
// sym = 1 takes the upper triangle i <= j column by column (entry e = j (j + 1) / 2 + i; the
// lower triangle is its conjugate), sym = 0 all k x kb entries (e = i + j k; B has kb columns,
// kb = k for a square Gram).  Block (x, y)
// takes row tiles x, x + gridDim.x, ... and entries y * kThreads * EPT + threadIdx.x +
// q * kThreads, q < EPT, and writes part[x * nent + e].  Tiles are staged with a row stride of
// 33 elements, so the lanes of a warp (consecutive i) read distinct shared-memory banks; each
// lane's FMAs are for live entries only (no idle half for the symmetric case).
template <class T, int EPT>
__global__ void __launch_bounds__(kThreads) k_gram_packed(const T *__restrict__ A, const T *__restrict__ B,
                                                           size_t ld, int k, int n, int sym, int nent,
                                                           typename ST<T>::D *part, int kb) {
    using D = typename ST<T>::D;
    constexpr int kS = 33;                   // staged row stride (elements)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ta = reinterpret_cast<T *>(smem_raw);
    const bool same = A == B;
    T *tb = same ? ta : ta + (size_t)kS * k;
    int ii[EPT], jj[EPT];
    D acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        acc[q] = D{};
        const int e = blockIdx.y * (kThreads * EPT) + threadIdx.x + q * kThreads;
        int i = -1, j = 0;
        if (e < nent) {
            if (sym) {
                j = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (j > 0 && j * (j + 1) / 2 > e) --j;
                while ((j + 1) * (j + 2) / 2 <= e) ++j;
                i = e - j * (j + 1) / 2;
            } else {
                j = e / k;
                i = e - j * k;
            }
        }
        ii[q] = i;
        jj[q] = j;
    }
    for (int row0 = blockIdx.x * 32; row0 < n; row0 += gridDim.x * 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * k; e += blockDim.x) {
            const int r = e & 31, c = e >> 5;
            const int row = row0 + r;
            ta[c * kS + r] = row < n ? A[(size_t)c * ld + row] : ST<T>::zero();
        }
        if (!same)
            for (int e = threadIdx.x; e < 32 * kb; e += blockDim.x) {
                const int r = e & 31, c = e >> 5;
                const int row = row0 + r;
                tb[c * kS + r] = row < n ? B[(size_t)c * ld + row] : ST<T>::zero();
            }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            if (ii[q] >= 0) {
                const T *a = ta + ii[q] * kS, *b = tb + jj[q] * kS;
                typename Part<T>::P s = ST<T>::zero();
#pragma unroll 8
                for (int r = 0; r < 32; ++r) s = ST<T>::fma_cm(a[r], b[r], s);
                acc[q] = dadd(acc[q], to_d(s));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const int e = blockIdx.y * (kThreads * EPT) + threadIdx.x + q * kThreads;
        if (e < nent) part[(size_t)blockIdx.x * nent + e] = acc[q];
    }
}

// G (k x kb, column-major) from the packed entries; sym (kb = k): the lower triangle is the conjugate.
__device__ __forceinline__ double dconj(double a) { return a; }
__device__ __forceinline__ cplx dconj(cplx a) { return conj(a); }
template <class D>
__global__ void k_gram_unpack(const D *__restrict__ packed, int k, int sym, D *G, int kb) {
    const int nent = sym ? k * (k + 1) / 2 : k * kb;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
        int i, j;
        if (sym) {
            j = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while (j > 0 && j * (j + 1) / 2 > e) --j;
            while ((j + 1) * (j + 2) / 2 <= e) ++j;
            i = e - j * (j + 1) / 2;
        } else {
            j = e / k;
            i = e - j * k;
        }
        const D v = packed[e];
        G[i + (size_t)j * k] = v;
        if (sym && i != j) G[j + (size_t)i * k] = dconj(v);
    }
}

// ----------------------------------------------------------------------------- misc vector ops
__device__ __forceinline__ double scal(double s, double a) { return s * a; }
__device__ __forceinline__ float scal(double s, float a) { return (float)s * a; }
__device__ __forceinline__ cplx scal(double s, cplx a) { return s * a; }

template <class T>
__global__ void k_scale_by(T *__restrict__ w, int n, const double *__restrict__ inv) {
    // w *= inv[0]
    const double s = inv[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] = scal(s, w[i]);
}

// Hbar column j of an Arnoldi step: H[i] = h1[i] + h2[i] (i <= j), H[j+1] = ||w||,
// inv[0] = 1 / ||w|| (0 if w vanished: an invariant subspace was found).
template <class T>
__global__ void k_arnoldi_finish(const typename ST<T>::D *h1, const typename ST<T>::D *h2,
                                 const typename ST<T>::D *nrm2, int j, T *Hcol, double *inv) {
    for (int i = threadIdx.x; i <= j; i += blockDim.x) Hcol[i] = dadd(h1[i], h2[i]);
    if (threadIdx.x == 0) {
        const double nn = sqrt(dreal(nrm2[0]));
        T hv = ST<T>::zero();
        *reinterpret_cast<double *>(&hv) = nn;
        Hcol[j + 1] = hv;
        inv[0] = nn > 0 ? 1.0 / nn : 0.0;
    }
}




// ----------------------------------------------------------------------------- float32 3D stencil, padded rows
// Inside a float32 BiCGStab cycle on a 3D constant-coefficient grid the cycle's vectors are
// kept in a padded layout: element (x, y, z) at z P N + y P + x with the row pitch P a multiple
// of 4 and greater than N, and x = N .. P-1 a zero column (the Dirichlet neighbour in x).  Rows
// are then 16-byte aligned, so the stencil moves every operand as float4: a thread takes 4
// consecutive points of a row and marches planes.  Its p at planes k-1..k+2 sit in a ring of
// four float4 registers, r_hat and the y neighbours (float4 loads of the rows above and below)
// in rings of two; after the compute of plane k the dead slots are refilled with p(k+3),
// r_hat(k+2) and the y neighbours at k+2.  The loop is unrolled by the ring length, so no
// register is copied and no load is waited on before the plane that needs it (a rotating copy
// would wait for a load issued in the same plane).  The x neighbours come from the
// neighbouring lanes' float4; the block-edge lanes take theirs (one value in the neighbouring
// tile) from another ring of two, also loaded two planes ahead: loaded at the plane that uses
// it, that one value held every warp for a full memory latency.  Outputs at padding points
// are written as zeros, so every vector of the cycle keeps zero padding and the cycle's dots
// need no mask.  Summation order per point is that of the one-point float32 stencil (centre,
// -x, +x, -y, +y, -z, +z).

__host__ __device__ __forceinline__ int pad_pitch(int N) { return (N + 1 + 3) / 4 * 4; }
constexpr int kPadRows = 16;     // rows per xy tile: a block of 32 x kPadRows threads
__host__ __device__ __forceinline__ int pad_tiles(int N) {
    const int G = pad_pitch(N) / 4;
    return ((G + 31) / 32) * ((N + kPadRows - 1) / kPadRows);
}

// in (N^3, x fastest) -> outp (padded, zero padding)
__global__ void k_pad3d(const float *__restrict__ in, float *__restrict__ outp, int N) {
    const unsigned P = (unsigned)pad_pitch(N), n = P * (unsigned)N * (unsigned)N;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned x = i % P, row = i / P;
        outp[i] = x < (unsigned)N ? in[row * (unsigned)N + x] : 0.0f;
    }
}

// inp (padded) -> out (N^3)
__global__ void k_unpad3d(const float *__restrict__ inp, float *__restrict__ out, int N) {
    const unsigned P = (unsigned)pad_pitch(N), n = (unsigned)N * (unsigned)N * (unsigned)N;
    for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const unsigned x = j % (unsigned)N, row = j / (unsigned)N;
        out[j] = inp[row * P + x];
    }
}

__device__ __forceinline__ float4 ld4c(bool ok, const float *__restrict__ p, unsigned i) {
    return ok ? *reinterpret_cast<const float4 *>(p + i) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float st7(const DevOp32 &o, float c, float w, float e, float s, float n, float d, float u) {
    float v = o.c0 * c;
    v = fmaf(o.cxm, w, v);
    v = fmaf(o.cxp, e, v);
    v = fmaf(o.cym, s, v);
    v = fmaf(o.cyp, n, v);
    v = fmaf(o.czm, d, v);
    return fmaf(o.czp, u, v);
}

// MODE 0: out = A p, <r_hat, out> -> alpha;  MODE 1: out = A p (p = s), the four dots -> omega,
// rho_next, beta (or the half-step exit), as k_bi_v / k_bi_t.  Block b takes xy tile b % tiles
// (32 float4 groups x kPadRows rows) and planes (b / tiles) * zlen .. + zlen - 1.
template <int MODE>
__global__ void __launch_bounds__(32 * kPadRows, 2) k_bi_pad(DevOp op, DevOp32 o, const float *__restrict__ p,
                                                             const float *__restrict__ rh, float *__restrict__ out,
                                                             double *part, unsigned *ticket, BiState<double> *st,
                                                             int zlen) {
    if (st->status != 0) return;
    if (MODE == 1 && st->half) return;
    constexpr int ND = MODE == 0 ? 1 : 4;
    constexpr int RP = 4, RR = 2;     // ring lengths: p planes, r_hat / y-neighbour planes
    __shared__ double red[kPadRows * ND];
    __shared__ double tot[ND];
    const int N = op.N;
    const int P = pad_pitch(N), G = P / 4;
    const int ntx = (G + 31) / 32, tiles = pad_tiles(N);
    const int b = blockIdx.x, xy = b % tiles;
    const int g0 = (xy % ntx) * 32, y0 = (xy / ntx) * kPadRows, z0 = (b / tiles) * zlen;
    const int z1 = min(z0 + zlen, N);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = g0 + lane, y = y0 + w, x = 4 * g;
    const bool act = g < G && y < N;
    const bool hs = act && y > 0, hn = act && y < N - 1;
    const bool hw = act && lane == 0 && x > 0, he = act && lane == 31 && g + 1 < G;
    const unsigned PS = (unsigned)P * (unsigned)N;
    const unsigned col = act ? (unsigned)y * P + x : 0u;
    auto at = [&](int z) { return (unsigned)z * PS + col; };
    // slots: p at plane z in (z - z0 + 1) % RP; r_hat, the y neighbours and the x-edge values
    // (lane 0: x - 1, lane 31: x + 4, both in the neighbouring tiles) at plane z in (z - z0) % RR
    float4 q[RP], r[RR], ys[RR], yn[RR];
    float xwr[RR], xer[RR];
#pragma unroll
    for (int i = 0; i < RP; ++i) {
        const int z = z0 - 1 + i;
        q[i] = ld4c(act && z >= 0 && z < N, p, at(z));
    }
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        const int z = z0 + i;
        r[i] = ld4c(act && z < z1, rh, at(z));
        ys[i] = ld4c(hs && z < z1, p, at(z) - P);
        yn[i] = ld4c(hn && z < z1, p, at(z) + P);
        xwr[i] = hw && z < z1 ? p[at(z) - 1] : 0.0f;
        xer[i] = he && z < z1 ? p[at(z) + 4] : 0.0f;
    }
    // which of the 4 points are grid points (x + i < N); the rest are padding
    const bool in1 = x + 1 < N, in2 = x + 2 < N, in3 = x + 3 < N;
    const int zp = min(N, z1 + 1);     // p is needed up to plane z1
    float acc[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) acc[d] = 0.0f;
    for (int kb = z0; kb < z1; kb += RP) {
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const int k = kb + j;
            if (k >= z1) break;
            const float4 pm = q[j], pc = q[(j + 1) % RP], pn = q[(j + 2) % RP];
            const float4 rc = r[j % RR], ysc = ys[j % RR], ync = yn[j % RR];
            float xw = __shfl_up_sync(0xffffffffu, pc.w, 1);
            float xe = __shfl_down_sync(0xffffffffu, pc.x, 1);
            if (lane == 0) xw = xwr[j % RR];
            if (lane == 31) xe = xer[j % RR];
            float4 v;
            v.x = st7(o, pc.x, xw, pc.y, ysc.x, ync.x, pm.x, pn.x);
            v.y = in1 ? st7(o, pc.y, pc.x, pc.z, ysc.y, ync.y, pm.y, pn.y) : 0.0f;
            v.z = in2 ? st7(o, pc.z, pc.y, pc.w, ysc.z, ync.z, pm.z, pn.z) : 0.0f;
            v.w = in3 ? st7(o, pc.w, pc.z, xe, ysc.w, ync.w, pm.w, pn.w) : 0.0f;
            if (x >= N) v.x = 0.0f;
            if (act) {
                *reinterpret_cast<float4 *>(out + at(k)) = v;
                if (MODE == 0) {
                    acc[0] = fmaf(rc.x, v.x, acc[0]);
                    acc[0] = fmaf(rc.y, v.y, acc[0]);
                    acc[0] = fmaf(rc.z, v.z, acc[0]);
                    acc[0] = fmaf(rc.w, v.w, acc[0]);
                } else {
                    const float vv[4] = {v.x, v.y, v.z, v.w}, cc[4] = {pc.x, pc.y, pc.z, pc.w};
                    const float rr[4] = {rc.x, rc.y, rc.z, rc.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        acc[0] = fmaf(vv[e], cc[e], acc[0]);
                        acc[ND > 1 ? 1 : 0] = fmaf(vv[e], vv[e], acc[ND > 1 ? 1 : 0]);
                        acc[ND > 2 ? 2 : 0] = fmaf(rr[e], cc[e], acc[ND > 2 ? 2 : 0]);
                        acc[ND > 3 ? 3 : 0] = fmaf(rr[e], vv[e], acc[ND > 3 ? 3 : 0]);
                    }
                }
            }
            // refill the slots this plane freed
            q[j] = ld4c(act && k + RP - 1 < zp, p, at(k + RP - 1));
            r[j % RR] = ld4c(act && k + RR < z1, rh, at(k + RR));
            ys[j % RR] = ld4c(hs && k + RR < z1, p, at(k + RR) - P);
            yn[j % RR] = ld4c(hn && k + RR < z1, p, at(k + RR) + P);
            xwr[j % RR] = hw && k + RR < z1 ? p[at(k + RR) - 1] : 0.0f;
            xer[j % RR] = he && k + RR < z1 ? p[at(k + RR) + 4] : 0.0f;
        }
    }
    block_reduce_store<float, double, ND>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<double, ND>(part, tot, ticket);
        if (threadIdx.x == 0) {
            st->mvps += 1;
            if (MODE == 0) {
                const double sigma = tot[0];
                if (!isfinite(sigma)) st->status = 4;
                else if (fabs(sigma) < kTiny) st->status = 2;
                else st->alpha = st->rho / sigma;
            } else {
                const double tt = tot[ND > 1 ? 1 : 0];
                if (!isfinite(tt) || !isfinite(tot[0])) {
                    st->status = 4;
                } else if (tt < kTiny) {
                    st->half = 1;
                    st->pending = 2;
                } else {
                    const double omega = tot[0] / tt;
                    st->omega = omega;
                    const double rn2 = tot[ND > 2 ? 2 : 0] - omega * tot[ND > 3 ? 3 : 0];
                    st->rho_next = rn2;
                    if (fabs(omega) >= kTiny) st->beta = (rn2 / st->rho) * (st->alpha / omega);
                }
            }
        }
    }
}

}  // namespace tg
