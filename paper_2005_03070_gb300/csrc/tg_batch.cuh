// Batched multi-instance kernels: many independent instances (each its own operator,
// deflation basis and R = 8 right-hand sides stored point-major) advanced together, one
// launch per phase for all of them.  Launch grid (gx, B): blockIdx.y selects the instance,
// its gx blocks stride over the instance's points, so instances of very different sizes
// share one launch and the hardware block scheduler balances them.  Reductions are per
// instance: block partials in a per-instance slice of `part`, the last of the instance's gx
// blocks (per-instance ticket) adds them in block order (deterministic) and updates that
// instance's R column states.  An instance whose columns have all finished their cycle
// returns at once (MrCtl::active == 0), so the lock-step host loop wastes no bandwidth on
// it.  Per point: float32 BiCGStab with the R columns' scalars in device memory (a column
// whose cycle has ended keeps its vectors), float64 refinement, float32 projection with
// float64 coefficients.
#pragma once

#include "tg_mrhs.cuh"

namespace tg {

// One instance of a batch (device copy, read by every block of the instance).
struct MrSeg {
    DevOp op;                   // fine operator (DK_CD2D)
    DevOp32 o32;
    size_t off;                 // first element of the instance's n x R block
    const float *W, *B1, *B2;   // float32 deflation data (n x kk, ld n): W^H r, x += B1 d, r -= B2 e
    const double *M;            // kk x kk float64 projection matrix
    int kk;
    int proj;                   // TG_PROJ_MINRES / TG_PROJ_GALERKIN
};

// per-instance slices of the batch's device state
struct MrBatchPtrs {
    const MrSeg *seg;
    BiState<double> *st;        // [B][R]
    MrCtl *ctl;                 // [B]
    unsigned *ticket;           // [B]
    double *part;               // [B][gx][partw]
    int partw;                  // doubles per block slot (>= 4 R, >= kk R)
    double *target2;            // [B][R] (negative: the column sits out this cycle)
    double *inv;                // [B][R]
    double *scale;              // [B][R]
    double *norms;              // [B][2 R]
    double *cvec, *dvec;        // [B][32 R]
    int cap;                    // product cap of the cycle (all instances)
    const double *capv = nullptr;   // [B][R] per-column product caps (nullptr: cap for all)
};

template <int R>
__device__ __forceinline__ double *seg_part(const MrBatchPtrs &P) {
    return P.part + (size_t)blockIdx.y * gridDim.x * P.partw;
}

// Block reduction of ND x R per-thread float partials into the instance's slice:
// slice[block * partw + d * R + r] (double), fixed order: warp shuffle tree, then warps in order.
template <int ND, int R>
__device__ __forceinline__ void mrb_block_store(float (&acc)[ND][R], double *slice, int partw, double *red) {
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
        slice[(size_t)blockIdx.x * partw + q] = s;
    }
}

template <int NQ>
__device__ __forceinline__ void mrb_final(const double *slice, int partw, double *tot, unsigned *ticket) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < NQ; q += nw) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(slice + (size_t)b * partw + q);
        s = warp_sum(s);
        if (lane == 0) tot[q] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

// ----------------------------------------------------------------------------- BiCGStab phases
template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_bi_init(const float *__restrict__ r, float *__restrict__ rh,
                                                           float *__restrict__ p, MrBatchPtrs P) {
    const int b = blockIdx.y;
    const MrSeg &S = P.seg[b];
    const int n = S.op.n;
    r += S.off; rh += S.off; p += S.off;
    BiState<double> *st = P.st + (size_t)b * R;
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
    double *slice = seg_part<R>(P);
    mrb_block_store<1, R>(acc, slice, P.partw, red);
    if (last_block(P.ticket + b)) {
        mrb_final<R>(slice, P.partw, tot, P.ticket + b);
        if (threadIdx.x == 0) {
            int active = 0;
            const double *t2 = P.target2 + (size_t)b * R;
            for (int q = 0; q < R; ++q) {
                BiState<double> &s = st[q];
                const double rho = tot[q];
                s.rho = rho; s.rr = rho; s.ss = 0.0; s.target2 = t2[q]; s.div2 = 1e16 * rho;   // 1e8-fold growth
                s.mvps = 0; s.cap = P.capv ? (int)P.capv[(size_t)b * R + q] : P.cap;
                s.iters = 0; s.half = 0; s.pending = 0;
                s.alpha = s.omega = s.beta = s.rho_next = 1.0;
                if (t2[q] < 0.0) s.status = 1;                 // not in this cycle
                else if (!isfinite(rho)) s.status = 4;
                else if (rho <= t2[q]) s.status = 1;
                else if (fabs(rho) < kTiny) s.status = 2;
                else s.status = 0;
                active += s.status == 0;
            }
            P.ctl[b].active = active;
        }
    }
}

template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_bi_v(const float *__restrict__ p, const float *__restrict__ rh,
                                                        float *__restrict__ v, MrBatchPtrs P) {
    const int b = blockIdx.y;
    if (P.ctl[b].active == 0) return;
    const MrSeg &S = P.seg[b];
    const DevOp op = S.op;
    const DevOp32 o32 = S.o32;
    p += S.off; rh += S.off; v += S.off;
    BiState<double> *st = P.st + (size_t)b * R;
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
        // every column's A p is stored: a column that has left the cycle never reads its v, s
        // or t again (its x and r are frozen; the next cycle starts from p = r), so its
        // values need not be preserved, and the old values are not read
        VecR<R> y = applyR<R>(op, o32, j, p);
        VecR<R> h = ldR<R>(rh, j);
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (on[q]) acc[0][q] = fmaf(h.v[q], y.v[q], acc[0][q]);
        stR<R>(v, j, y);
    }
    double *slice = seg_part<R>(P);
    mrb_block_store<1, R>(acc, slice, P.partw, red);
    if (last_block(P.ticket + b)) {
        mrb_final<R>(slice, P.partw, tot, P.ticket + b);
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

template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_bi_s(const float *__restrict__ r, const float *__restrict__ v,
                                                        float *__restrict__ s, MrBatchPtrs P) {
    const int b = blockIdx.y;
    if (P.ctl[b].active == 0) return;
    const MrSeg &S = P.seg[b];
    const int n = S.op.n;
    r += S.off; v += S.off; s += S.off;
    BiState<double> *st = P.st + (size_t)b * R;
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
        VecR<R> a = ldR<R>(r, j), bb = ldR<R>(v, j), o;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            o.v[q] = fmaf(ma[q], bb.v[q], a.v[q]);     // stored for every column, as in k_mrb_bi_v
            if (on[q]) acc[0][q] = fmaf(o.v[q], o.v[q], acc[0][q]);
        }
        stR<R>(s, j, o);
    }
    double *slice = seg_part<R>(P);
    mrb_block_store<1, R>(acc, slice, P.partw, red);
    if (last_block(P.ticket + b)) {
        mrb_final<R>(slice, P.partw, tot, P.ticket + b);
        if (threadIdx.x == 0) {
            for (int q = 0; q < R; ++q) {
                BiState<double> &c = st[q];
                if (c.status != 0) continue;
                const double ss = tot[q];
                c.ss = ss;
                if (!isfinite(ss)) c.status = 4;
                else if (ss <= c.target2) { c.half = 1; c.pending = 1; }
                else if (ss > c.div2) c.status = 5;
                else if (c.mvps >= c.cap) { c.half = 1; c.pending = 3; }
            }
        }
    }
}

template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_bi_t(const float *__restrict__ s, const float *__restrict__ rh,
                                                        float *__restrict__ t, MrBatchPtrs P) {
    const int b = blockIdx.y;
    if (P.ctl[b].active == 0) return;
    const MrSeg &S = P.seg[b];
    const DevOp op = S.op;
    const DevOp32 o32 = S.o32;
    s += S.off; rh += S.off; t += S.off;
    BiState<double> *st = P.st + (size_t)b * R;
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
        VecR<R> sv = ldR<R>(s, j), h = ldR<R>(rh, j);     // t stored for every column, as in k_mrb_bi_v
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (!on[q]) continue;
            acc[0][q] = fmaf(y.v[q], sv.v[q], acc[0][q]);
            acc[1][q] = fmaf(y.v[q], y.v[q], acc[1][q]);
            acc[2][q] = fmaf(h.v[q], sv.v[q], acc[2][q]);
            acc[3][q] = fmaf(h.v[q], y.v[q], acc[3][q]);
        }
        stR<R>(t, j, y);
    }
    double *slice = seg_part<R>(P);
    mrb_block_store<4, R>(acc, slice, P.partw, red);
    if (last_block(P.ticket + b)) {
        mrb_final<4 * R>(slice, P.partw, tot, P.ticket + b);
        if (threadIdx.x == 0) {
            for (int q = 0; q < R; ++q) {
                BiState<double> &c = st[q];
                if (c.status != 0 || c.half) continue;
                c.mvps += 1;
                const double ts = tot[q], tt = tot[R + q], rs = tot[2 * R + q], rt = tot[3 * R + q];
                if (!isfinite(tt) || !isfinite(ts)) c.status = 4;
                else if (tt < kTiny) { c.half = 1; c.pending = 2; }
                else {
                    const double om = ts / tt;
                    c.omega = om;
                    const double rn = rs - om * rt;
                    c.rho_next = rn;
                    if (fabs(om) >= kTiny) c.beta = (rn / c.rho) * (c.alpha / om);
                }
            }
        }
    }
}

template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_bi_x(float *__restrict__ x, float *__restrict__ r,
                                                        float *__restrict__ p, const float *__restrict__ s,
                                                        const float *__restrict__ t, const float *__restrict__ v,
                                                        MrBatchPtrs P) {
    const int b = blockIdx.y;
    if (P.ctl[b].active == 0) return;
    const MrSeg &S = P.seg[b];
    const int n = S.op.n;
    x += S.off; r += S.off; p += S.off; s += S.off; t += S.off; v += S.off;
    BiState<double> *st = P.st + (size_t)b * R;
    __shared__ double red[8 * R];
    __shared__ double tot[R];
    int mode[R];      // 0 idle, 1 full step, 2 half step
    float al[R], om[R], be[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const BiState<double> &c = st[q];
        mode[q] = c.status != 0 ? 0 : (c.half ? 2 : 1);
        al[q] = (float)c.alpha;
        om[q] = (float)c.omega;
        be[q] = (float)c.beta;
    }
    // with every column on a full step the new r is s - omega t throughout, and the old r
    // (read only to keep the other columns' r) is not loaded
    bool full = true;
#pragma unroll
    for (int q = 0; q < R; ++q) full = full && mode[q] == 1;
    float acc[1][R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[0][q] = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        VecR<R> xv = ldR<R>(x, j), pv = ldR<R>(p, j), sv = ldR<R>(s, j), tv = ldR<R>(t, j), vv = ldR<R>(v, j);
        VecR<R> rv;
        if (full) {
#pragma unroll
            for (int q = 0; q < R; ++q) rv.v[q] = 0.0f;
        } else {
            rv = ldR<R>(r, j);
        }
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
    double *slice = seg_part<R>(P);
    mrb_block_store<1, R>(acc, slice, P.partw, red);
    if (last_block(P.ticket + b)) {
        mrb_final<R>(slice, P.partw, tot, P.ticket + b);
        if (threadIdx.x == 0) {
            int active = 0;
            for (int q = 0; q < R; ++q) {
                BiState<double> &c = st[q];
                if (c.status == 0 && c.half) {
                    c.rr = c.ss;
                    c.status = c.pending;
                    c.iters += 1;
                } else if (c.status == 0) {
                    const double rr = tot[q];
                    c.rr = rr;
                    c.iters += 1;
                    c.rho = c.rho_next;
                    if (!isfinite(rr)) c.status = 4;
                    else if (rr <= c.target2) c.status = 1;
                    else if (rr > c.div2) c.status = 5;
                    else if (fabs(c.omega) < kTiny) c.status = 2;
                    else if (fabs(c.rho_next) < kTiny) c.status = 2;
                    else if (c.mvps >= c.cap) c.status = 3;
                }
                active += c.status == 0;
            }
            P.ctl[b].active = active;
        }
    }
}

// ----------------------------------------------------------------------------- refinement
// r64 = b - A x (float64); norms[b][q] = ||r_q||^2, norms[b][R + q] = ||b_q||^2.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_residual(const double *__restrict__ B, const double *__restrict__ X,
                                                            double *__restrict__ r64, MrBatchPtrs P) {
    const int b = blockIdx.y;
    const MrSeg &S = P.seg[b];
    const DevOp op = S.op;
    B += S.off; X += S.off; r64 += S.off;
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
            const double ax = apply_real_d(op, j, [&](int jj) { return X[(size_t)jj * R + q]; });
            const double bi = B[(size_t)j * R + q];
            const double ri = bi - ax;
            r64[(size_t)j * R + q] = ri;
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
    double *slice = seg_part<R>(P);
    for (int q = threadIdx.x; q < 2 * R; q += blockDim.x) {
        double s2 = red[q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s2 += red[w * 2 * R + q];
        slice[(size_t)blockIdx.x * P.partw + q] = s2;
    }
    if (last_block(P.ticket + b)) {
        mrb_final<2 * R>(slice, P.partw, tot, P.ticket + b);
        for (int q = threadIdx.x; q < 2 * R; q += blockDim.x) P.norms[(size_t)b * 2 * R + q] = tot[q];
    }
}

// r32 = r64 * inv[q], e32 = 0.
template <int R>
__global__ void k_mrb_scale(const double *__restrict__ r64, float *__restrict__ r32, float *__restrict__ e32,
                            MrBatchPtrs P) {
    const int b = blockIdx.y;
    const MrSeg &S = P.seg[b];
    const size_t tot = (size_t)S.op.n * R;
    r64 += S.off; r32 += S.off; e32 += S.off;
    const double *inv = P.inv + (size_t)b * R;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        r32[e] = (float)(r64[e] * inv[e % R]);
        e32[e] = 0.f;
    }
}

// x64 += scale[q] e32 (columns with scale != 0).
template <int R>
__global__ void k_mrb_add(double *__restrict__ X, const float *__restrict__ e32, MrBatchPtrs P) {
    const int b = blockIdx.y;
    const MrSeg &S = P.seg[b];
    const size_t tot = (size_t)S.op.n * R;
    X += S.off; e32 += S.off;
    const double *scale = P.scale + (size_t)b * R;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const double sc = scale[e % R];
        if (sc != 0.0) X[e] = fma(sc, (double)e32[e], X[e]);
    }
}

// ----------------------------------------------------------------------------- projection
// cvec[b][c R + q] = sum over the instance's points of W[c][j] r[j][q] (per-instance kk);
// the last of the instance's blocks reduces in block order.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_proj_dots(const float *__restrict__ r, MrBatchPtrs P) {
    constexpr int kChunk = 128;
    const int b = blockIdx.y;
    const MrSeg &S = P.seg[b];
    const int k = S.kk, n = S.op.n;
    if (k == 0) return;
    r += S.off;
    const float *W = S.W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ws = reinterpret_cast<float *>(smem_raw);     // k x kChunk
    float *rs = ws + (size_t)k * kChunk;                   // kChunk x R
    __shared__ double tot1[32 * R];
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
    double *slice = seg_part<R>(P);
    if (threadIdx.x < nent) slice[(size_t)blockIdx.x * P.partw + threadIdx.x] = (double)acc;
    if (last_block(P.ticket + b)) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int e = warp; e < nent; e += nw) {
            double s = 0.0;
            for (int bb = lane; bb < (int)gridDim.x; bb += 32) s += __ldcg(slice + (size_t)bb * P.partw + e);
            s = warp_sum(s);
            if (lane == 0) tot1[e] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) P.ticket[b] = 0u;
        double *cv = P.cvec + (size_t)b * 32 * R;
        for (int e = threadIdx.x; e < nent; e += blockDim.x) cv[e] = tot1[e];
    }
}

// dvec[b] = M cvec[b] (one block per instance).
template <int R>
__global__ void k_mrb_small(MrBatchPtrs P) {
    const int b = blockIdx.x;
    const MrSeg &S = P.seg[b];
    const int k = S.kk;
    const double *cv = P.cvec + (size_t)b * 32 * R;
    double *dv = P.dvec + (size_t)b * 32 * R;
    for (int e = threadIdx.x; e < k * R; e += blockDim.x) {
        const int c = e / R, q = e % R;
        double s = 0.0;
        for (int cc = 0; cc < k; ++cc) s = fma(S.M[c + (size_t)cc * k], cv[cc * R + q], s);
        dv[e] = s;
    }
}

// e += B1 d; r -= B2 ee (ee = the dots for MinRes, d for Galerkin); norms[b][q] = ||r_q||^2.
template <int R>
__global__ void __launch_bounds__(kThreads) k_mrb_proj_update(float *__restrict__ e, float *__restrict__ r,
                                                               MrBatchPtrs P) {
    const int b = blockIdx.y;
    const MrSeg &S = P.seg[b];
    const int k = S.kk, n = S.op.n;
    if (k == 0) return;
    e += S.off; r += S.off;
    const double *d = P.dvec + (size_t)b * 32 * R;
    const double *ee = S.proj == TG_PROJ_MINRES ? P.cvec + (size_t)b * 32 * R : d;
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
            const float b1 = S.B1[(size_t)c * n + j], b2 = S.B2[(size_t)c * n + j];
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
    double *slice = seg_part<R>(P);
    mrb_block_store<1, R>(acc, slice, P.partw, red);
    if (last_block(P.ticket + b)) {
        mrb_final<R>(slice, P.partw, tot, P.ticket + b);
        for (int q = threadIdx.x; q < R; q += blockDim.x) P.norms[(size_t)b * 2 * R + q] = tot[q];
    }
}

// ============================================================================= batched coarse GMRES-DR
// The coarse phase of every instance in lock-step cycles (float32 Arnoldi basis, float64
// Hessenberg and restart step, as in the single-instance float32 + refinement form): step j
// of the Arnoldi extension is one launch per sub-step for all instances; an instance takes
// part when j0 <= j (its cycle starts at its own j0 = kk) and while it is active.
struct GdrSeg {
    DevOp op;                   // coarse operator (float32 constants in o32)
    DevOp32 o32;
    float *V;                   // current basis, nc x (m + 1), leading dimension ldv
    float *xc;                  // coarse solution (float32)
    double *H;                  // Hbar, (m + 1) x m, ld m + 1
    double *h1, *h2;            // the two Gram-Schmidt coefficient vectors (m + 2 each)
    double *nrm;                // [0] ||w||^2, [4] 1 / ||w||
    const double *d;            // least-squares solution of the restart step (m)
    size_t ldv;
    int nc;
    int j0;                     // first Arnoldi column of the current cycle
    int kk;                     // kept vectors after the last restart
    int active;
};

struct GdrBatchPtrs {
    const GdrSeg *seg;
    double *part;               // [B][gx][partw]
    int partw;
    unsigned *ticket;           // [B]
};

__device__ __forceinline__ bool gdr_takes(const GdrSeg &S, int j) { return S.active && j >= S.j0; }

// w = A v_j (float32) for the instances taking part in step j
__global__ void __launch_bounds__(kThreads) k_gb_apply(GdrBatchPtrs P, int j) {
    const GdrSeg &S = P.seg[blockIdx.y];
    if (!gdr_takes(S, j)) return;
    const DevOp op = S.op;
    const DevOp32 o32 = S.o32;
    const float *x = S.V + (size_t)j * S.ldv;
    float *y = S.V + (size_t)(j + 1) * S.ldv;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < op.n; i += gridDim.x * blockDim.x)
        y[i] = apply_real_f(op, o32, i, [&](int jj) { return x[jj]; });
}

// h = V[:, 0..ncol-1]^H w (ncol = ncol_step, or the instance's kk when reorth), w = column
// wcol of V; per-instance partials, the last block of the instance adds them in block order.
// Warp w owns columns w, w + 8, ...; 4 rows per lane per pass (as k_gemv_t_part).
__global__ void __launch_bounds__(kThreads) k_gb_gemv_t(GdrBatchPtrs P, int j, int ncol_step, int reorth,
                                                         int which) {
    constexpr int kMaxPerWarp = 17;
    constexpr int kU = 4;
    const int b = blockIdx.y;
    const GdrSeg &S = P.seg[b];
    const bool on = reorth ? (S.active != 0) : gdr_takes(S, j);
    if (!on) return;
    const int ncol = reorth ? S.kk : ncol_step;
    const int wcol = reorth ? S.kk : j + 1;
    const float *V = S.V;
    const float *w = S.V + (size_t)wcol * S.ldv;
    const int n = S.nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[kMaxPerWarp];
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) acc[q] = 0.f;
    for (int row0 = blockIdx.x * 32 * kU; row0 < n; row0 += gridDim.x * 32 * kU) {
        float wv[kU];
        int rr[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            rr[u] = row0 + 32 * u + lane;
            wv[u] = rr[u] < n ? w[rr[u]] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kMaxPerWarp; ++q) {
            const int c = warp + 8 * q;
            if (c < ncol) {
                const float *vc = V + (size_t)c * S.ldv;
#pragma unroll
                for (int u = 0; u < kU; ++u) acc[q] = fmaf(rr[u] < n ? vc[rr[u]] : 0.f, wv[u], acc[q]);
            }
        }
    }
    double *slice = P.part + (size_t)b * gridDim.x * P.partw;
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) {
        const int c = warp + 8 * q;
        if (c < ncol) {
            const float sum = warp_sum(acc[q]);
            if (lane == 0) slice[(size_t)blockIdx.x * P.partw + c] = (double)sum;
        }
    }
    if (last_block(P.ticket + b)) {
        double *h = which ? S.h2 : S.h1;
        for (int c = warp; c < ncol; c += (int)(blockDim.x >> 5)) {
            double sum = 0.0;
            for (int bb = lane; bb < (int)gridDim.x; bb += 32) sum += __ldcg(slice + (size_t)bb * P.partw + c);
            sum = warp_sum(sum);
            if (lane == 0) h[c] = sum;
        }
        __syncthreads();
        if (threadIdx.x == 0) P.ticket[b] = 0u;
    }
}

// The same product with the rows staged through shared memory by a 3-deep cp.async chunk
// pipeline (as k_gemv_t_pipe): block (x, i) takes instance i's 128-row chunks x, x + gx, ...,
// each copied as (ncol + 1) columns x 512 bytes (w is the extra column) while the block
// works on the previous chunk.  The basis columns start 16-byte aligned and ldv is a multiple
// of 128 rows, so every chunk lies inside the allocation (rows at or beyond nc are masked).
// ncol <= kGbPipeCols; dynamic shared memory 3 x (kGbPipeCols + 1) x 512 bytes.
constexpr int kGbPipeCols = 64;
constexpr size_t kGbPipeSmem = (size_t)3 * (kGbPipeCols + 1) * 128 * sizeof(float);
__global__ void __launch_bounds__(kThreads, 2) k_gb_gemv_t_pipe(GdrBatchPtrs P, int j, int ncol_step, int reorth,
                                                              int which) {
    constexpr int R = 128, PE = 4, U = R / 32, kStages = 3, kMaxPerWarp = kGbPipeCols / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>(smem_raw);
    const int b = blockIdx.y;
    const GdrSeg &S = P.seg[b];
    const bool on = reorth ? (S.active != 0) : gdr_takes(S, j);
    if (!on) return;
    const int ncol = reorth ? S.kk : ncol_step;
    const int wcol = reorth ? S.kk : j + 1;
    const float *V = S.V;
    const float *w = S.V + (size_t)wcol * S.ldv;
    const int n = S.nc;
    const int cols = ncol + 1;
    const size_t stage = (size_t)cols * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nchunks = (n + R - 1) / R, G = gridDim.x;
    const int mine = (int)blockIdx.x < nchunks ? (nchunks - 1 - (int)blockIdx.x) / G + 1 : 0;
    auto issue = [&](int it) {
        if (it < mine) {
            const size_t row0 = ((size_t)blockIdx.x + (size_t)it * G) * R;
            float *dst = buf + (size_t)(it % kStages) * stage;
            for (int e = threadIdx.x; e < cols * (R / PE); e += blockDim.x) {
                const int c = e / (R / PE), rp = e % (R / PE);
                const float *src = (c < ncol ? V + (size_t)c * S.ldv : w) + row0 + PE * rp;
                cp_async16(dst + (size_t)c * R + PE * rp, src);
            }
        }
        cp_async_commit();
    };
    float acc[kMaxPerWarp];
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) acc[q] = 0.f;
#pragma unroll
    for (int st = 0; st < kStages - 1; ++st) issue(st);
    for (int it = 0; it < mine; ++it) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        issue(it + kStages - 1);          // the buffer of chunk it - 1, which every thread has read
        const float *sb = buf + (size_t)(it % kStages) * stage;
        const int row0 = ((int)blockIdx.x + it * G) * R;
        float wv[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = row0 + lane + 32 * u < n;
            wv[u] = ok[u] ? sb[(size_t)ncol * R + lane + 32 * u] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kMaxPerWarp; ++q) {
            const int c = warp + 8 * q;
            if (c < ncol) {
                const float *sc = sb + (size_t)c * R;
#pragma unroll
                for (int u = 0; u < U; ++u) acc[q] = fmaf(ok[u] ? sc[lane + 32 * u] : 0.f, wv[u], acc[q]);
            }
        }
    }
    cp_async_wait<0>();
    double *slice = P.part + (size_t)b * gridDim.x * P.partw;
#pragma unroll
    for (int q = 0; q < kMaxPerWarp; ++q) {
        const int c = warp + 8 * q;
        if (c < ncol) {
            const float sum = warp_sum(acc[q]);
            if (lane == 0) slice[(size_t)blockIdx.x * P.partw + c] = (double)sum;
        }
    }
    if (last_block(P.ticket + b)) {
        double *h = which ? S.h2 : S.h1;
        for (int c = warp; c < ncol; c += (int)(blockDim.x >> 5)) {
            double sum = 0.0;
            for (int bb = lane; bb < (int)gridDim.x; bb += 32) sum += __ldcg(slice + (size_t)bb * P.partw + c);
            sum = warp_sum(sum);
            if (lane == 0) h[c] = sum;
        }
        __syncthreads();
        if (threadIdx.x == 0) P.ticket[b] = 0u;
    }
}

// w -= V[:, 0..ncol-1] h (float32, coefficients rounded once per block), then ||w||^2 into
// nrm[0] (per instance, deterministic).
__global__ void __launch_bounds__(kThreads) k_gb_gemv_n_norm(GdrBatchPtrs P, int j, int ncol_step, int reorth,
                                                              int which) {
    const int b = blockIdx.y;
    const GdrSeg &S = P.seg[b];
    const bool on = reorth ? (S.active != 0) : gdr_takes(S, j);
    if (!on) return;
    const int ncol = reorth ? S.kk : ncol_step;
    const int wcol = reorth ? S.kk : j + 1;
    __shared__ float hs[kSmallCols];
    __shared__ double red[(kThreads / 32)];
    __shared__ double tot[1];
    const double *h = which ? S.h2 : S.h1;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) hs[c] = (float)h[c];
    __syncthreads();
    const float *V = S.V;
    float *w = S.V + (size_t)wcol * S.ldv;
    const int n = S.nc;
    float acc[1] = {0.f};
    // thread g takes rows 4g .. 4g + 3 as float4 (ldv a multiple of 128, V 16-byte aligned);
    // rows at and beyond n (the padding) are computed but neither stored nor summed
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; 4 * g < n; g += gridDim.x * blockDim.x) {
        const int r = 4 * g;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int c = 0; c < ncol; ++c) {
            const float4 v = ld4(V + (size_t)c * S.ldv, r);
            const float hc = hs[c];
            a0 = fmaf(hc, v.x, a0);
            a1 = fmaf(hc, v.y, a1);
            a2 = fmaf(hc, v.z, a2);
            a3 = fmaf(hc, v.w, a3);
        }
        const float4 wo = ld4(w, r);
        const float4 wn = make_float4(wo.x - a0, wo.y - a1, wo.z - a2, wo.w - a3);
        if (r + 4 <= n) {
            *reinterpret_cast<float4 *>(w + r) = wn;
            acc[0] = fmaf(wn.x, wn.x, acc[0]);
            acc[0] = fmaf(wn.y, wn.y, acc[0]);
            acc[0] = fmaf(wn.z, wn.z, acc[0]);
            acc[0] = fmaf(wn.w, wn.w, acc[0]);
        } else {
            const float e[4] = {wn.x, wn.y, wn.z, wn.w};
            for (int i = 0; i < n - r; ++i) {
                w[r + i] = e[i];
                acc[0] = fmaf(e[i], e[i], acc[0]);
            }
        }
    }
    double *slice = P.part + (size_t)b * gridDim.x * P.partw;
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const float ws = warp_sum(acc[0]);
        if (lane == 0) red[warp] = (double)ws;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = red[0];
            for (int q = 1; q < (int)(blockDim.x >> 5); ++q) sum += red[q];
            slice[(size_t)blockIdx.x * P.partw] = sum;
        }
    }
    if (last_block(P.ticket + b)) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (warp == 0) {
            double sum = 0.0;
            for (int bb = lane; bb < (int)gridDim.x; bb += 32) sum += __ldcg(slice + (size_t)bb * P.partw);
            sum = warp_sum(sum);
            if (lane == 0) tot[0] = sum;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.nrm[0] = tot[0];
            P.ticket[b] = 0u;
        }
    }
}

// Hbar column j = h1 + h2 (rows 0..j), H[j+1, j] = ||w||, nrm[4] = 1 / ||w|| (one thread per
// instance); reorth = 1: only nrm[4] (the re-orthogonalised v_kk is normalised).
__global__ void k_gb_finish(GdrBatchPtrs P, int count, int j, int ldh, int reorth) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const GdrSeg &S = P.seg[b];
    const bool on = reorth ? (S.active != 0) : gdr_takes(S, j);
    if (!on) return;
    const double nn = sqrt(S.nrm[0]);
    S.nrm[4] = nn > 0 ? 1.0 / nn : 0.0;
    if (reorth) return;
    double *Hcol = S.H + (size_t)j * ldh;
    for (int i = 0; i <= j; ++i) Hcol[i] = S.h1[i] + S.h2[i];
    Hcol[j + 1] = nn;
}

// v *= 1 / ||w|| for column j + 1 (or kk when reorth)
__global__ void k_gb_scale(GdrBatchPtrs P, int j, int reorth) {
    const GdrSeg &S = P.seg[blockIdx.y];
    const bool on = reorth ? (S.active != 0) : gdr_takes(S, j);
    if (!on) return;
    float *w = S.V + (size_t)(reorth ? S.kk : j + 1) * S.ldv;
    const float sc = (float)S.nrm[4];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.nc; i += gridDim.x * blockDim.x) w[i] *= sc;
}

// x_c += V[:, 0..m-1] d (coefficients of the restart step's least-squares solution)
__global__ void __launch_bounds__(kThreads) k_gb_xc(GdrBatchPtrs P, int m) {
    const GdrSeg &S = P.seg[blockIdx.y];
    if (!S.active) return;
    __shared__ float ds[kSmallCols];
    for (int c = threadIdx.x; c < m; c += blockDim.x) ds[c] = (float)S.d[c];
    __syncthreads();
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < S.nc; row += gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int c = 0; c < m; ++c) a = fmaf(ds[c], S.V[(size_t)c * S.ldv + row], a);
        S.xc[row] += a;
    }
}

// Out[:, 0..q-1] = V[:, 0..p-1] Pm (Pm (p x q) float64, ld ldp), q = the instance's kk + 1
// (restart recombination) or kk (final basis; Out float64 then).  Pm staged once per block
// as float32; one thread per row.
template <class TO>
__global__ void __launch_bounds__(kThreads) k_gb_tsm(GdrBatchPtrs P, const double *const *Pm, int ldp, int p,
                                                      int plus_one, TO *const *Out, const size_t *ldo) {
    const int b = blockIdx.y;
    const GdrSeg &S = P.seg[b];
    if (!S.active) return;
    const int q = S.kk + plus_one;
    __shared__ float ps[(kSmallCols) * 34];
    const double *Pb = Pm[b];
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
        const int i = e % p, c = e / p;
        ps[c * p + i] = (float)Pb[i + (size_t)c * ldp];
    }
    __syncthreads();
    TO *O = Out[b];
    const size_t lo = ldo[b];
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < S.nc; row += gridDim.x * blockDim.x) {
        float acc[34];
#pragma unroll
        for (int c = 0; c < 34; ++c) acc[c] = 0.f;
        for (int i = 0; i < p; ++i) {
            const float v = S.V[(size_t)i * S.ldv + row];
#pragma unroll
            for (int c = 0; c < 34; ++c)
                if (c < q) acc[c] = fmaf(ps[c * p + i], v, acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 34; ++c)
            if (c < q) O[(size_t)c * lo + row] = (TO)acc[c];
    }
}

}  // namespace tg
