// IDR(s) cycle kernels (float64 / complex128, and float32 for the float32 + refinement form,
// whose scalars stay float64): the biorthogonal IDR(s) of van Gijzen and
// Sonneveld, the paper's other fine-grid solver (Section 4.1, IDR(ncyc)-Proj(k)).
//
// One round of s + 1 operator products, with every scalar of the recurrence kept on the
// device (IdrState) and computed by the last block of the producing reduction:
//   step k = 0..s-1:
//     k_idr_u    c = M[k:, k:]^{-1} f[k:] (each block, forward substitution, M lower
//                triangular);  U_k = U[:, k:] c + omega (r - G[:, k:] c)
//     k_idr_g    G_k = A U_k and d = P^H G_k;  last block: the biorthogonalisation
//                coefficients alpha (M[:k, :k] alpha = d[:k]), the new column
//                M[k:, k] = d[k:] - M[k:, :k] alpha, beta = f_k / M_kk, f[k+1:] -= beta M[k+1:, k]
//     k_idr_upd  G_k -= G[:, :k] alpha, U_k -= U[:, :k] alpha, r -= beta G_k, x += beta U_k, ||r||^2
//   dimension reduction:
//     k_idr_t    t = A r and <t, r>, <t, t>, <r, r>;  last block: omega = <t, r> / <t, t>,
//                enlarged to omega kappa / |rho| when |rho| = |<t, r>| / (||t|| ||r||) < kappa
//     k_idr_xr   x += omega r, r -= omega t, f = P^H r, ||r||^2
// The biorthogonalisation is written in its classical form (all P_i^H G_k from one pass,
// then a triangular solve with M) where the published algorithm subtracts one column at a
// time: in exact arithmetic the two agree (P_i^H G_j = M_ij for j <= i), and the classical
// form reads G_k once instead of k times.  A kernel returns at once when the cycle's status
// is set (converged, breakdown, product cap, NaN), so the host can queue several rounds
// between status reads.
#pragma once

#include "tg_kernels.cuh"

namespace tg {

constexpr int kIdrMaxS = 8;

template <class D>
struct IdrState {
    D M[kIdrMaxS * kIdrMaxS];   // M[i + j * kIdrMaxS] = P_i^H G_j, i >= j (lower triangle)
    D f[kIdrMaxS];              // P^H r
    D alpha[kIdrMaxS];
    D beta, omega;
    double rr;                  // ||r||^2 after the last update
    double target2;             // (rticyc ||r_cycle_start||)^2
    double kappa;               // angle safeguard of omega
    int s;
    int mvps, cap, rounds;
    int status;                 // 0 running, 1 converged, 2 breakdown, 3 capped, 4 NaN
};

__device__ __forceinline__ double dmod(double a) { return fabs(a); }
__device__ __forceinline__ double dmod(cplx a) { return hypot(a.re, a.im); }

// f = P^H r, ||r||^2; the state of a new cycle (M = I, omega = 1).
template <class T>
__global__ void __launch_bounds__(kThreads) k_idr_init(const T *__restrict__ r, const T *__restrict__ P, size_t ld,
                                                        int n, int s, double target2, int cap, double kappa,
                                                        typename ST<T>::D *part, unsigned *ticket,
                                                        IdrState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    __shared__ D red[(kThreads / 32) * (kIdrMaxS + 1)];
    __shared__ D tot[kIdrMaxS + 1];
    T acc[kIdrMaxS + 1];
#pragma unroll
    for (int q = 0; q <= kIdrMaxS; ++q) acc[q] = ST<T>::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T ri = r[i];
#pragma unroll
        for (int q = 0; q < kIdrMaxS; ++q)
            if (q < s) acc[q] = ST<T>::fma_cm(P[(size_t)q * ld + i], ri, acc[q]);
        acc[kIdrMaxS] = ST<T>::fma_cm(ri, ri, acc[kIdrMaxS]);
    }
    block_reduce_store<T, D, kIdrMaxS + 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, kIdrMaxS + 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            for (int e = 0; e < kIdrMaxS * kIdrMaxS; ++e) st->M[e] = D{};
            for (int q = 0; q < kIdrMaxS; ++q) {
                st->f[q] = q < s ? tot[q] : D{};
                st->alpha[q] = D{};
            }
            const double rr = dreal(tot[kIdrMaxS]);
            st->rr = rr;
            st->target2 = target2;
            st->kappa = kappa;
            st->s = s;
            st->mvps = 0;
            st->cap = cap;
            st->rounds = 0;
            st->beta = D{};
            D one{};
            *reinterpret_cast<double *>(&one) = 1.0;
            st->omega = one;
            for (int q = 0; q < kIdrMaxS; ++q) st->M[q + q * kIdrMaxS] = one;
            if (!isfinite(rr)) st->status = 4;
            else if (rr <= target2) st->status = 1;
            else st->status = 0;
        }
    }
}

// U_k = U[:, k:] c + omega (r - G[:, k:] c), c = M[k:, k:]^{-1} f[k:].  first: the cycle's
// first round, where the columns k.. of G and U are not yet written (they count as zero).
template <class T>
__global__ void __launch_bounds__(kThreads) k_idr_u(const T *__restrict__ r, const T *__restrict__ G, T *__restrict__ U,
                                                     size_t ld, int n, int k, int first,
                                                     const IdrState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    if (st->status != 0) return;
    __shared__ T cs[kIdrMaxS];
    __shared__ T om_s;
    const int s = st->s;
    if (threadIdx.x == 0) {
        D c[kIdrMaxS];
        for (int a = k; a < s; ++a) {
            D v = st->f[a];
            for (int b = k; b < a; ++b) v = dsub(v, dmul(st->M[a + b * kIdrMaxS], c[b - k]));
            c[a - k] = ddiv(v, st->M[a + a * kIdrMaxS]);
            cs[a - k] = KS<T>::of(c[a - k]);
        }
        om_s = KS<T>::of(st->omega);
    }
    __syncthreads();
    const T om = om_s;
    const int nc = s - k;
    T *Uk = U + (size_t)k * ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T v = r[i];
        T u = ST<T>::zero();
        if (!first) {
            for (int q = 0; q < nc; ++q) {
                v = sub(v, dmul(cs[q], G[(size_t)(k + q) * ld + i]));
                u = axpy(cs[q], U[(size_t)(k + q) * ld + i], u);
            }
        }
        Uk[i] = axpy(om, v, u);
    }
}

// G_k = A U_k; d = P^H G_k; last block: alpha, M[k:, k], beta, f.
template <class T>
__global__ void __launch_bounds__(kThreads) k_idr_g(DevOp op, DevOp32 o32, const T *__restrict__ U, T *__restrict__ G,
                                                     const T *__restrict__ P, size_t ld, int k,
                                                     typename ST<T>::D *part, unsigned *ticket,
                                                     IdrState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    if (st->status != 0) return;
    __shared__ D red[(kThreads / 32) * kIdrMaxS];
    __shared__ D tot[kIdrMaxS];
    const int s = st->s;
    const int n = op.n;
    const T *Uk = U + (size_t)k * ld;
    T *Gk = G + (size_t)k * ld;
    T acc[kIdrMaxS];
#pragma unroll
    for (int q = 0; q < kIdrMaxS; ++q) acc[q] = ST<T>::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T g = Apply<T>::at(op, o32, i, [&](int j) { return Uk[j]; });
        Gk[i] = g;
#pragma unroll
        for (int q = 0; q < kIdrMaxS; ++q)
            if (q < s) acc[q] = ST<T>::fma_cm(P[(size_t)q * ld + i], g, acc[q]);
    }
    block_reduce_store<T, D, kIdrMaxS>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, kIdrMaxS>(part, tot, ticket);
        if (threadIdx.x == 0) {
            st->mvps += 1;
            D al[kIdrMaxS];
            bool finite = true;
            for (int i = 0; i < k; ++i) {            // M[:k, :k] alpha = d[:k]
                D v = tot[i];
                for (int b = 0; b < i; ++b) v = dsub(v, dmul(st->M[i + b * kIdrMaxS], al[b]));
                al[i] = ddiv(v, st->M[i + i * kIdrMaxS]);
                st->alpha[i] = al[i];
            }
            for (int j = k; j < s; ++j) {            // M[j, k] = P_j^H (G_k - G[:, :k] alpha)
                D v = tot[j];
                for (int b = 0; b < k; ++b) v = dsub(v, dmul(al[b], st->M[j + b * kIdrMaxS]));
                st->M[j + k * kIdrMaxS] = v;
                finite = finite && dfinite(v);
            }
            const D mkk = st->M[k + k * kIdrMaxS];
            if (!finite) st->status = 4;
            else if (dmod(mkk) < kTiny) st->status = 2;
            else {
                const D beta = ddiv(st->f[k], mkk);
                st->beta = beta;
                for (int j = k + 1; j < s; ++j) st->f[j] = dsub(st->f[j], dmul(beta, st->M[j + k * kIdrMaxS]));
            }
        }
    }
}

// G_k -= G[:, :k] alpha; U_k -= U[:, :k] alpha; r -= beta G_k; x += beta U_k; ||r||^2.
template <class T>
__global__ void __launch_bounds__(kThreads) k_idr_upd(T *__restrict__ G, T *__restrict__ U, size_t ld, T *__restrict__ r,
                                                       T *__restrict__ x, int n, int k, typename ST<T>::D *part,
                                                       unsigned *ticket, IdrState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    if (st->status != 0) return;
    __shared__ T al_s[kIdrMaxS];
    __shared__ T beta_s;
    __shared__ D red[(kThreads / 32)];
    __shared__ D tot[1];
    if (threadIdx.x < k) al_s[threadIdx.x] = KS<T>::of(st->alpha[threadIdx.x]);
    if (threadIdx.x == 0) beta_s = KS<T>::of(st->beta);
    __syncthreads();
    const T beta = beta_s;
    T *Gk = G + (size_t)k * ld;
    T *Uk = U + (size_t)k * ld;
    T acc[1] = {ST<T>::zero()};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T g = Gk[i], u = Uk[i];
        for (int b = 0; b < k; ++b) {
            g = sub(g, dmul(al_s[b], G[(size_t)b * ld + i]));
            u = sub(u, dmul(al_s[b], U[(size_t)b * ld + i]));
        }
        Gk[i] = g;
        Uk[i] = u;
        const T ri = sub(r[i], dmul(beta, g));
        r[i] = ri;
        x[i] = axpy(beta, u, x[i]);
        acc[0] = ST<T>::fma_cm(ri, ri, acc[0]);
    }
    block_reduce_store<T, D, 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            const double rr = dreal(tot[0]);
            st->rr = rr;
            if (!isfinite(rr)) st->status = 4;
            else if (rr <= st->target2) st->status = 1;
            else if (st->mvps >= st->cap) st->status = 3;
        }
    }
}

// t = A r; <t, r>, <t, t>, <r, r>; last block: omega with the angle safeguard.
template <class T>
__global__ void __launch_bounds__(kThreads) k_idr_t(DevOp op, DevOp32 o32, const T *__restrict__ r, T *__restrict__ t,
                                                     typename ST<T>::D *part, unsigned *ticket,
                                                     IdrState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    if (st->status != 0) return;
    __shared__ D red[(kThreads / 32) * 3];
    __shared__ D tot[3];
    const int n = op.n;
    T acc[3] = {ST<T>::zero(), ST<T>::zero(), ST<T>::zero()};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T ti = Apply<T>::at(op, o32, i, [&](int j) { return r[j]; });
        t[i] = ti;
        const T ri = r[i];
        acc[0] = ST<T>::fma_cm(ti, ri, acc[0]);
        acc[1] = ST<T>::fma_cm(ti, ti, acc[1]);
        acc[2] = ST<T>::fma_cm(ri, ri, acc[2]);
    }
    block_reduce_store<T, D, 3>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, 3>(part, tot, ticket);
        if (threadIdx.x == 0) {
            st->mvps += 1;
            const double tt = dreal(tot[1]), rr = dreal(tot[2]);
            if (!isfinite(tt) || !dfinite(tot[0])) {
                st->status = 4;
            } else if (tt < kTiny) {
                st->status = 2;
            } else {
                D om = ddiv(tot[0], D(tot[1]));
                const double rho = dmod(tot[0]) / sqrt(tt * rr);
                if (rho < st->kappa) om = om * (st->kappa / rho);
                if (dmod(om) < kTiny) st->status = 2;
                else st->omega = om;
            }
        }
    }
}

// x += omega r; r -= omega t; f = P^H r; ||r||^2; the end of a round.
template <class T>
__global__ void __launch_bounds__(kThreads) k_idr_xr(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ t,
                                                      const T *__restrict__ P, size_t ld, int n,
                                                      typename ST<T>::D *part, unsigned *ticket,
                                                      IdrState<typename ST<T>::D> *st) {
    using D = typename ST<T>::D;
    if (st->status != 0) return;
    __shared__ D red[(kThreads / 32) * (kIdrMaxS + 1)];
    __shared__ D tot[kIdrMaxS + 1];
    const int s = st->s;
    const T om = KS<T>::of(st->omega);
    T acc[kIdrMaxS + 1];
#pragma unroll
    for (int q = 0; q <= kIdrMaxS; ++q) acc[q] = ST<T>::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T ri = r[i];
        x[i] = axpy(om, ri, x[i]);
        const T rn = sub(ri, dmul(om, t[i]));
        r[i] = rn;
#pragma unroll
        for (int q = 0; q < kIdrMaxS; ++q)
            if (q < s) acc[q] = ST<T>::fma_cm(P[(size_t)q * ld + i], rn, acc[q]);
        acc[kIdrMaxS] = ST<T>::fma_cm(rn, rn, acc[kIdrMaxS]);
    }
    block_reduce_store<T, D, kIdrMaxS + 1>(acc, part, red);
    if (last_block(ticket)) {
        final_sum<D, kIdrMaxS + 1>(part, tot, ticket);
        if (threadIdx.x == 0) {
            for (int q = 0; q < s; ++q) st->f[q] = tot[q];
            const double rr = dreal(tot[kIdrMaxS]);
            st->rr = rr;
            st->rounds += 1;
            if (!isfinite(rr)) st->status = 4;
            else if (rr <= st->target2) st->status = 1;
            else if (st->mvps >= st->cap) st->status = 3;
        }
    }
}

}  // namespace tg
