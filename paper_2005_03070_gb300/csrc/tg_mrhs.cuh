// Multi-right-hand-side helpers: R systems with the same operator, stored point-major
// (element (point j, right-hand side r) at j * R + r), one thread per point handling all R
// with float4 loads; the batched kernels of tg_batch.cuh are built on them.
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

struct MrCtl {
    int active;                 // right-hand sides still iterating in this cycle
};

// column q of an interleaved n x R float64 block, as a plain vector
template <int R>
__global__ void k_mr_extract(const double *__restrict__ src, int q, int n, double *__restrict__ dst) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) dst[j] = src[(size_t)j * R + q];
}

}  // namespace tg
