// Multi-right-hand-side kernels: R systems with the same operator, stored point-major
// (element (point j, right-hand side r) at j * R + r), one thread per point handling all R.
// The inner BiCGStab iteration runs in float32 (the refinement form); every right-hand
// side keeps its own scalars and status in device memory, and a right-hand side whose
// cycle has ended keeps its vectors unchanged.  Used by the batched solver (tg_batch_*).
#pragma once

#include "tg_kernels.cuh"

namespace tg {

// ----------------------------------------------------------------------------- helpers
template <int R> struct VecR { float v[R]; };

template <int R>
__device__ __forceinline__ VecR<R> ldR(const float *__restrict__ p, int j) {
    VecR<R> o;
    const float4 *q = reinterpret_cast<const float4 *>(p + (size_t)j * R);
#pragma unroll
    for (int h = 0; h < R / 4; ++h) {
        float4 a = q[h];
        o.v[4 * h] = a.x; o.v[4 * h + 1] = a.y; o.v[4 * h + 2] = a.z; o.v[4 * h + 3] = a.w;
    }
    return o;
}
template <int R>
__device__ __forceinline__ void stR(float *__restrict__ p, int j, const VecR<R> &o) {
    float4 *q = reinterpret_cast<float4 *>(p + (size_t)j * R);
#pragma unroll
    for (int h = 0; h < R / 4; ++h) q[h] = make_float4(o.v[4 * h], o.v[4 * h + 1], o.v[4 * h + 2], o.v[4 * h + 3]);
}

// y = A u for the R interleaved columns of u at point idx (float32, real grids)
template <int R>
__device__ __forceinline__ VecR<R> applyR(const DevOp &op, const DevOp32 &o, int idx, const float *__restrict__ u) {
    VecR<R> y;
    const int N = op.N;
    if (op.kind == DK_CD2D || op.kind == DK_VAR2D) {
        const int j = (int)op.fN.div((unsigned)idx), i = idx - j * N;
        float c0, cw, ce, cs, cn;
        if (op.kind == DK_CD2D) {
            c0 = o.c0; cw = o.cxm; ce = o.cxp; cs = o.cym; cn = o.cyp;
        } else {
            const int n = op.n;
            c0 = op.vc32[idx]; cw = op.vc32[n + idx]; ce = op.vc32[2 * n + idx];
            cs = op.vc32[3 * n + idx]; cn = op.vc32[4 * n + idx];
        }
        VecR<R> a = ldR<R>(u, idx);
#pragma unroll
        for (int r = 0; r < R; ++r) y.v[r] = c0 * a.v[r];
        if (i > 0) { a = ldR<R>(u, idx - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) y.v[r] = fmaf(cw, a.v[r], y.v[r]); }
        if (i < N - 1) { a = ldR<R>(u, idx + 1);
#pragma unroll
            for (int r = 0; r < R; ++r) y.v[r] = fmaf(ce, a.v[r], y.v[r]); }
        if (j > 0) { a = ldR<R>(u, idx - N);
#pragma unroll
            for (int r = 0; r < R; ++r) y.v[r] = fmaf(cs, a.v[r], y.v[r]); }
        if (j < N - 1) { a = ldR<R>(u, idx + N);
#pragma unroll
            for (int r = 0; r < R; ++r) y.v[r] = fmaf(cn, a.v[r], y.v[r]); }
        return y;
    }
    // 3D
    const int NN = N * N;
    const int q = (int)op.fN.div((unsigned)idx), k = (int)op.fNN.div((unsigned)idx);
    const int i = idx - q * N, j = q - k * N;
    VecR<R> a = ldR<R>(u, idx);
#pragma unroll
    for (int r = 0; r < R; ++r) y.v[r] = o.c0 * a.v[r];
    const int nb[6] = {i > 0 ? idx - 1 : -1, i < N - 1 ? idx + 1 : -1, j > 0 ? idx - N : -1,
                       j < N - 1 ? idx + N : -1, k > 0 ? idx - NN : -1, k < N - 1 ? idx + NN : -1};
    const float cf[6] = {o.cxm, o.cxp, o.cym, o.cyp, o.czm, o.czp};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (nb[q] < 0) continue;
        a = ldR<R>(u, nb[q]);
#pragma unroll
        for (int r = 0; r < R; ++r) y.v[r] = fmaf(cf[q], a.v[r], y.v[r]);
    }
    return y;
}

// Block reduction of ND x R per-thread float partials into part[block][d * R + r] (double),
// fixed order: warp shuffle tree, then warps in order.
template <int ND, int R>
__device__ __forceinline__ void mr_block_store(float (&acc)[ND][R], double *part, double *red /* 8*ND*R */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float s = warp_sum(acc[d][r]);
            if (lane == 0) red[(warp * ND + d) * R + r] = (double)s;
        }
    __syncthreads();
    for (int q = threadIdx.x; q < ND * R; q += blockDim.x) {
        double s = red[q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s += red[w * ND * R + q];
        part[(size_t)blockIdx.x * ND * R + q] = s;
    }
}

// In the last block: tot[q] = sum over blocks of part[b][q], q < NQ; warps take entries in
// turn, lanes stride over blocks, fixed shuffle tree (deterministic).
template <int NQ>
__device__ __forceinline__ void mr_final(const double *part, double *tot, unsigned *ticket) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < NQ; q += nw) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(part + (size_t)b * NQ + q);
        s = warp_sum(s);
        if (lane == 0) tot[q] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

struct MrCtl {
    int active;                 // right-hand sides still iterating in this cycle
};

// ----------------------------------------------------------------------------- BiCGStab (float32, R columns)
// r_hat = r, p = r for the columns in the cycle; rho_r = ||r_r||^2; per-column state from
// target2[r] (negative: the column is not in this cycle) and cap.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_bi_init(const float *__restrict__ r, float *__restrict__ rh,
                                                          float *__restrict__ p, int n, const double *target2,
                                                          int cap, double *part, unsigned *ticket,
                                                          BiState<double> *st, MrCtl *ctl) {
    __shared__ double red[8 * R];
    __shared__ double tot[R];
    float acc[1][R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[0][q] = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        VecR<R> a = ldR<R>(r, j);
        stR<R>(rh, j, a);
        stR<R>(p, j, a);
#pragma unroll
        for (int q = 0; q < R; ++q) acc[0][q] = fmaf(a.v[q], a.v[q], acc[0][q]);
    }
    mr_block_store<1, R>(acc, part, red);
    if (last_block(ticket)) {
        mr_final<R>(part, tot, ticket);
        if (threadIdx.x == 0) {
            int active = 0;
            for (int q = 0; q < R; ++q) {
                BiState<double> &s = st[q];
                const double rho = tot[q];
                s.rho = rho; s.rr = rho; s.ss = 0.0; s.target2 = target2[q]; s.div2 = 1e16 * rho;   // 1e8-fold growth
                s.mvps = 0; s.cap = cap; s.iters = 0; s.half = 0; s.pending = 0;
                s.alpha = s.omega = s.beta = s.rho_next = 1.0;
                if (target2[q] < 0.0) s.status = 1;            // not in this cycle
                else if (!isfinite(rho)) s.status = 4;
                else if (rho <= target2[q]) s.status = 1;
                else if (fabs(rho) < kTiny) s.status = 2;
                else s.status = 0;
                active += s.status == 0;
            }
            ctl->active = active;
        }
    }
}

// v = A p; sigma_r = <r_hat_r, v_r>; alpha_r = rho_r / sigma_r (columns in state 0).
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_bi_v(DevOp op, DevOp32 o32, const float *__restrict__ p,
                                                       const float *__restrict__ rh, float *__restrict__ v,
                                                       double *part, unsigned *ticket, BiState<double> *st,
                                                       const MrCtl *ctl) {
    if (ctl->active == 0) return;
    __shared__ double red[8 * R];
    __shared__ double tot[R];
    bool on[R];
#pragma unroll
    for (int q = 0; q < R; ++q) on[q] = st[q].status == 0;
    float acc[1][R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[0][q] = 0.f;
    const int n = op.n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        VecR<R> y = applyR<R>(op, o32, j, p);
        VecR<R> old = ldR<R>(v, j);
        VecR<R> h = ldR<R>(rh, j);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (!on[q]) y.v[q] = old.v[q];
            else acc[0][q] = fmaf(h.v[q], y.v[q], acc[0][q]);
        }
        stR<R>(v, j, y);
    }
    mr_block_store<1, R>(acc, part, red);
    if (last_block(ticket)) {
        mr_final<R>(part, tot, ticket);
        if (threadIdx.x == 0) {
            for (int q = 0; q < R; ++q) {
                BiState<double> &s = st[q];
                if (s.status != 0) continue;
                const double sigma = tot[q];
                s.mvps += 1;
                if (!isfinite(sigma)) s.status = 4;
                else if (fabs(sigma) < kTiny) s.status = 2;
                else s.alpha = s.rho / sigma;
            }
        }
    }
}

// s = r - alpha v; ||s||^2; half-step test per column.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_bi_s(const float *__restrict__ r, const float *__restrict__ v,
                                                       float *__restrict__ s, int n, double *part, unsigned *ticket,
                                                       BiState<double> *st, const MrCtl *ctl) {
    if (ctl->active == 0) return;
    __shared__ double red[8 * R];
    __shared__ double tot[R];
    bool on[R];
    float ma[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        on[q] = st[q].status == 0;
        ma[q] = -(float)st[q].alpha;
    }
    float acc[1][R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[0][q] = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        VecR<R> a = ldR<R>(r, j), b = ldR<R>(v, j), o = ldR<R>(s, j);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (on[q]) {
                o.v[q] = fmaf(ma[q], b.v[q], a.v[q]);
                acc[0][q] = fmaf(o.v[q], o.v[q], acc[0][q]);
            }
        }
        stR<R>(s, j, o);
    }
    mr_block_store<1, R>(acc, part, red);
    if (last_block(ticket)) {
        mr_final<R>(part, tot, ticket);
        if (threadIdx.x == 0) {
            for (int q = 0; q < R; ++q) {
                BiState<double> &b = st[q];
                if (b.status != 0) continue;
                const double ss = tot[q];
                b.ss = ss;
                if (!isfinite(ss)) b.status = 4;
                else if (ss <= b.target2) { b.half = 1; b.pending = 1; }
                else if (ss > b.div2) b.status = 5;
                else if (b.mvps >= b.cap) { b.half = 1; b.pending = 3; }
            }
        }
    }
}

// t = A s; <t,s>, <t,t>, <r_hat,s>, <r_hat,t> per column; omega, rho_next, beta.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_bi_t(DevOp op, DevOp32 o32, const float *__restrict__ s,
                                                       const float *__restrict__ rh, float *__restrict__ t,
                                                       double *part, unsigned *ticket, BiState<double> *st,
                                                       const MrCtl *ctl) {
    if (ctl->active == 0) return;
    __shared__ double red[8 * 4 * R];
    __shared__ double tot[4 * R];
    bool on[R];
#pragma unroll
    for (int q = 0; q < R; ++q) on[q] = st[q].status == 0 && !st[q].half;
    float acc[4][R];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int q = 0; q < R; ++q) acc[d][q] = 0.f;
    const int n = op.n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        VecR<R> y = applyR<R>(op, o32, j, s);
        VecR<R> old = ldR<R>(t, j), sv = ldR<R>(s, j), h = ldR<R>(rh, j);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (!on[q]) { y.v[q] = old.v[q]; continue; }
            acc[0][q] = fmaf(y.v[q], sv.v[q], acc[0][q]);
            acc[1][q] = fmaf(y.v[q], y.v[q], acc[1][q]);
            acc[2][q] = fmaf(h.v[q], sv.v[q], acc[2][q]);
            acc[3][q] = fmaf(h.v[q], y.v[q], acc[3][q]);
        }
        stR<R>(t, j, y);
    }
    mr_block_store<4, R>(acc, part, red);
    if (last_block(ticket)) {
        mr_final<4 * R>(part, tot, ticket);
        if (threadIdx.x == 0) {
            for (int q = 0; q < R; ++q) {
                BiState<double> &b = st[q];
                if (b.status != 0 || b.half) continue;
                b.mvps += 1;
                const double ts = tot[q], tt = tot[R + q], rs = tot[2 * R + q], rt = tot[3 * R + q];
                if (!isfinite(tt) || !isfinite(ts)) b.status = 4;
                else if (tt < kTiny) { b.half = 1; b.pending = 2; }
                else {
                    const double om = ts / tt;
                    b.omega = om;
                    const double rn = rs - om * rt;
                    b.rho_next = rn;
                    if (fabs(om) >= kTiny) b.beta = (rn / b.rho) * (b.alpha / om);
                }
            }
        }
    }
}

// x += alpha p + omega s; r = s - omega t; p = r + beta (p - omega v); ||r||^2 per column.
// A pending half step: x += alpha p; r = s.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_bi_x(float *__restrict__ x, float *__restrict__ r,
                                                       float *__restrict__ p, const float *__restrict__ s,
                                                       const float *__restrict__ t, const float *__restrict__ v,
                                                       int n, double *part, unsigned *ticket, BiState<double> *st,
                                                       MrCtl *ctl) {
    if (ctl->active == 0) return;
    __shared__ double red[8 * R];
    __shared__ double tot[R];
    int mode[R];      // 0 idle, 1 full step, 2 half step
    float al[R], om[R], be[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const BiState<double> &b = st[q];
        mode[q] = b.status != 0 ? 0 : (b.half ? 2 : 1);
        al[q] = (float)b.alpha;
        om[q] = (float)b.omega;
        be[q] = (float)b.beta;
    }
    float acc[1][R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[0][q] = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        VecR<R> xv = ldR<R>(x, j), rv = ldR<R>(r, j), pv = ldR<R>(p, j), sv = ldR<R>(s, j), tv = ldR<R>(t, j),
                vv = ldR<R>(v, j);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (mode[q] == 1) {
                xv.v[q] = fmaf(om[q], sv.v[q], fmaf(al[q], pv.v[q], xv.v[q]));
                const float rn = fmaf(-om[q], tv.v[q], sv.v[q]);
                rv.v[q] = rn;
                pv.v[q] = fmaf(be[q], fmaf(-om[q], vv.v[q], pv.v[q]), rn);
                acc[0][q] = fmaf(rn, rn, acc[0][q]);
            } else if (mode[q] == 2) {
                xv.v[q] = fmaf(al[q], pv.v[q], xv.v[q]);
                rv.v[q] = sv.v[q];
            }
        }
        stR<R>(x, j, xv);
        stR<R>(r, j, rv);
        stR<R>(p, j, pv);
    }
    mr_block_store<1, R>(acc, part, red);
    if (last_block(ticket)) {
        mr_final<R>(part, tot, ticket);
        if (threadIdx.x == 0) {
            int active = 0;
            for (int q = 0; q < R; ++q) {
                BiState<double> &b = st[q];
                if (b.status == 0 && b.half) {
                    b.rr = b.ss;
                    b.status = b.pending;
                    b.iters += 1;
                } else if (b.status == 0) {
                    const double rr = tot[q];
                    b.rr = rr;
                    b.iters += 1;
                    b.rho = b.rho_next;
                    if (!isfinite(rr)) b.status = 4;
                    else if (rr <= b.target2) b.status = 1;
                    else if (rr > b.div2) b.status = 5;
                    else if (fabs(b.omega) < kTiny) b.status = 2;
                    else if (fabs(b.rho_next) < kTiny) b.status = 2;
                    else if (b.mvps >= b.cap) b.status = 3;
                }
                active += b.status == 0;
            }
            ctl->active = active;
        }
    }
}

// ----------------------------------------------------------------------------- refinement
// r64 = b - A x (float64, R columns); out[q] = ||r_q||^2, out[R + q] = ||b_q||^2.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_residual(DevOp op, const double *__restrict__ b,
                                                           const double *__restrict__ x, double *__restrict__ r,
                                                           double *part, unsigned *ticket, double *out) {
    __shared__ double red[8 * 2 * R];
    __shared__ double tot[2 * R];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[2][R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[0][q] = acc[1][q] = 0.0;
    const int n = op.n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const double ax = apply_real_d(op, j, [&](int jj) { return x[(size_t)jj * R + q]; });
            const double bi = b[(size_t)j * R + q];
            const double ri = bi - ax;
            r[(size_t)j * R + q] = ri;
            acc[0][q] = fma(ri, ri, acc[0][q]);
            acc[1][q] = fma(bi, bi, acc[1][q]);
        }
    }
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            double s2 = warp_sum(acc[d][q]);
            if (lane == 0) red[(warp * 2 + d) * R + q] = s2;
        }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * R; q += blockDim.x) {
        double s2 = red[q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s2 += red[w * 2 * R + q];
        part[(size_t)blockIdx.x * 2 * R + q] = s2;
    }
    if (last_block(ticket)) {
        mr_final<2 * R>(part, tot, ticket);
        for (int q = threadIdx.x; q < 2 * R; q += blockDim.x) out[q] = tot[q];
    }
}

// r32 = r64 * inv[q], e32 = 0 (float).
template <int R>
__global__ void k_mr_scale(const double *__restrict__ r64, float *__restrict__ r32, float *__restrict__ e32, int n,
                           const double *__restrict__ inv) {
    const size_t tot = (size_t)n * R;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        r32[e] = (float)(r64[e] * inv[e % R]);
        e32[e] = 0.f;
    }
}

// x64 += scale[q] * e32 for the columns with scale != 0.
template <int R>
__global__ void k_mr_add(double *__restrict__ x, const float *__restrict__ e32, int n, const double *__restrict__ scale) {
    const size_t tot = (size_t)n * R;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const double sc = scale[e % R];
        if (sc != 0.0) x[e] = fma(sc, (double)e32[e], x[e]);
    }
}

// ----------------------------------------------------------------------------- projection
// part[block][c * R + q] = sum over the block's points of W[c][j] r[j][q]; W float32 n x k
// column-major (one read of the basis serves all R columns).
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_proj_dots(const float *__restrict__ W, int k,
                                                            const float *__restrict__ r, int n, double *part) {
    constexpr int kChunk = 128;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ws = reinterpret_cast<float *>(smem_raw);     // k x kChunk
    float *rs = ws + (size_t)k * kChunk;                   // kChunk x R
    const int nent = k * R;
    float acc = 0.f;                                       // entry threadIdx.x (< nent)
    const int c = threadIdx.x / R, q = threadIdx.x % R;
    for (int j0 = blockIdx.x * kChunk; j0 < n; j0 += gridDim.x * kChunk) {
        __syncthreads();
        for (int e = threadIdx.x; e < k * kChunk; e += blockDim.x) {
            const int cc = e / kChunk, jj = e % kChunk;
            ws[e] = j0 + jj < n ? W[(size_t)cc * n + j0 + jj] : 0.f;
        }
        for (int e = threadIdx.x; e < kChunk * R; e += blockDim.x)
            rs[e] = j0 + e / R < n ? r[(size_t)j0 * R + e] : 0.f;
        __syncthreads();
        if (threadIdx.x < nent) {
            const float *wc = ws + (size_t)c * kChunk;
            for (int jj = 0; jj < kChunk; ++jj) acc = fmaf(wc[jj], rs[jj * R + q], acc);
        }
    }
    if (threadIdx.x < nent) part[(size_t)blockIdx.x * nent + threadIdx.x] = (double)acc;
}

// d[c, q] = sum_c' M[c, c'] cvec[c', q] (k x k float64 M, column-major; one block).
template <int R>
__global__ void k_mr_small(const double *__restrict__ M, int k, const double *__restrict__ cvec, double *__restrict__ d) {
    for (int e = threadIdx.x; e < k * R; e += blockDim.x) {
        const int c = e / R, q = e % R;
        double s = 0.0;
        for (int cc = 0; cc < k; ++cc) s = fma(M[c + (size_t)cc * k], cvec[cc * R + q], s);
        d[e] = s;
    }
}

// e += B1 d; r -= B2 ee (per column q; ee = d for Galerkin, the dots for MinRes); then
// ||r_q||^2 per column into out[q] (last block).
template <int R>
__global__ void __launch_bounds__(kThreads) k_mr_proj_update(const float *__restrict__ B1, const float *__restrict__ B2,
                                                              int k, const double *__restrict__ d,
                                                              const double *__restrict__ ee, float *__restrict__ e,
                                                              float *__restrict__ r, int n, double *part,
                                                              unsigned *ticket, double *out) {
    __shared__ float ds[32 * R], es[32 * R];
    __shared__ double red[8 * R];
    __shared__ double tot[R];
    for (int q = threadIdx.x; q < k * R; q += blockDim.x) {
        ds[q] = (float)d[q];
        es[q] = (float)ee[q];
    }
    __syncthreads();
    float acc[1][R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[0][q] = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        VecR<R> ev = ldR<R>(e, j), rv = ldR<R>(r, j);
        for (int c = 0; c < k; ++c) {
            const float b1 = B1[(size_t)c * n + j], b2 = B2[(size_t)c * n + j];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                ev.v[q] = fmaf(b1, ds[c * R + q], ev.v[q]);
                rv.v[q] = fmaf(-b2, es[c * R + q], rv.v[q]);
            }
        }
        stR<R>(e, j, ev);
        stR<R>(r, j, rv);
#pragma unroll
        for (int q = 0; q < R; ++q) acc[0][q] = fmaf(rv.v[q], rv.v[q], acc[0][q]);
    }
    mr_block_store<1, R>(acc, part, red);
    if (last_block(ticket)) {
        mr_final<R>(part, tot, ticket);
        for (int q = threadIdx.x; q < R; q += blockDim.x) out[q] = tot[q];
    }
}

// column q of an interleaved n x R float64 block, as a plain vector
template <int R>
__global__ void k_mr_extract(const double *__restrict__ src, int q, int n, double *__restrict__ dst) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) dst[j] = src[(size_t)j * R + q];
}

}  // namespace tg
