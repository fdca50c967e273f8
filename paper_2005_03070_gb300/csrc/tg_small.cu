// Single-CTA float64 kernels for the small dense problems of the method:
//   - the GMRES-DR restart step (Section 2.1): least squares min ||c - Hbar d||, harmonic
//     Ritz pairs of Hbar (eigenpairs of H_m + |h_{m+1,m}|^2 f e_m^T, H_m^H f = e_m),
//     selection of the k smallest, orthonormal basis P_k of their span, the restart
//     matrices P_{k+1}, Hbar_k = P_{k+1}^H Hbar P_k, c_k = P_{k+1}^H (c - Hbar d);
//   - Cholesky and triangular inverse for CholQR2 (the projection set-up);
//   - Gauss-Jordan inverse of the Galerkin matrix H = V^H A V;
//   - incremental Givens least squares for GMRES(m) cycles;
//   - the k x k solve of each projection.
// The eigenvalue algorithms are the textbook ones (Golub & Van Loan, Matrix Computations,
// Sections 7.4-7.6): Householder reduction to Hessenberg form, Francis double-shift QR
// (real matrices, real Schur form with 2 x 2 blocks for complex pairs) or Wilkinson
// single-shift QR (complex matrices), with accumulated Schur vectors, and eigenvectors
// by back substitution on the (quasi-)triangular factor.  The restart kernel is one block
// of kGdrThreads threads whose work matrices sit in shared memory while they fit (global
// scratch otherwise); the other kernels are one block of kSmallThreads threads on global
// scratch.  On this GPU every float64 warp instruction holds its sub-partition's float64
// unit for tens of cycles whatever the active lanes, and sqrt, division and hypot are
// long sequences of them: the serial chains (QR sweeps, reflectors) are written to keep
// few float64 instructions on the critical path (see the Schur form section).
#include <cfloat>
#include <cmath>
#include "tg_small.cuh"

namespace tg {

namespace {

constexpr double kEps = DBL_EPSILON;


// ----------------------------------------------------------------------------- generic helpers
template <class T> struct Cx;
template <> struct Cx<double> {
    __device__ static double cj(double a) { return a; }
    __device__ static double ab2(double a) { return a * a; }
    __device__ static double mul(double a, double b) { return a * b; }
    __device__ static double div(double a, double b) { return a / b; }
    __device__ static double re(double a) { return a; }
    __device__ static double zero() { return 0.0; }
    __device__ static double one() { return 1.0; }
    __device__ static double sc(double s, double a) { return s * a; }
};
template <> struct Cx<cplx> {
    __device__ static cplx cj(cplx a) { return conj(a); }
    __device__ static double ab2(cplx a) { return abs2(a); }
    __device__ static cplx mul(cplx a, cplx b) { return a * b; }
    __device__ static cplx div(cplx a, cplx b) { return cdiv(a, b); }
    __device__ static double re(cplx a) { return a.re; }
    __device__ static cplx zero() { return {0.0, 0.0}; }
    __device__ static cplx one() { return {1.0, 0.0}; }
    __device__ static cplx sc(double s, cplx a) { return s * a; }
};

__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ cplx add(cplx a, cplx b) { return a + b; }
__device__ __forceinline__ double subt(double a, double b) { return a - b; }
__device__ __forceinline__ cplx subt(cplx a, cplx b) { return a - b; }

// Householder vector for x[0..len-1] (strided): v with v[0] = 1 and tau such that
// (I - tau v v^H) x = beta e_1.  Written to v[], returns tau (0 if x is already beta e_1).
template <class T>
__device__ T house(const T *x, int stride, int len, T *v, T *beta_out) {
    double nrm2 = 0.0;
    for (int i = 1; i < len; ++i) nrm2 += Cx<T>::ab2(x[i * stride]);
    T x0 = x[0];
    if (nrm2 == 0.0) {
        v[0] = Cx<T>::one();
        for (int i = 1; i < len; ++i) v[i] = Cx<T>::zero();
        *beta_out = x0;
        return Cx<T>::zero();
    }
    double a0 = sqrt(Cx<T>::ab2(x0));
    double alpha = sqrt(Cx<T>::ab2(x0) + nrm2);
    // beta = -phase(x0) * alpha
    T ph = a0 > 0 ? Cx<T>::sc(1.0 / a0, x0) : Cx<T>::one();
    T beta = Cx<T>::sc(-alpha, ph);
    T v0 = subt(x0, beta);                       // x0 + phase * alpha
    for (int i = 1; i < len; ++i) v[i] = Cx<T>::div(x[i * stride], v0);
    v[0] = Cx<T>::one();
    *beta_out = beta;
    // tau = (beta - x0) / beta
    return Cx<T>::div(subt(beta, x0), beta);
}

// Block-parallel Householder vector: the same reflector as house(), with the norm summed
// by all threads (fixed order: per-thread strided partials, then warp shuffles, then
// warps in order) and one reciprocal instead of a division per element.  x and v may
// not overlap.  Every thread of the block must call it; returns tau, *beta_out.
template <class T>
__device__ T house_par(const T *x, int len, T *v, T *beta_out) {
    __shared__ double red_s[32];
    __shared__ T tau_sh, beta_sh, inv_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double p = 0.0;
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) p += Cx<T>::ab2(x[i]);
    p = warp_sum(p);
    if (lane == 0) red_s[warp] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        double nrm2 = 0.0;
        for (int w = 0; w < nw; ++w) nrm2 += red_s[w];
        T x0 = x[0];
        if (nrm2 == 0.0) {
            tau_sh = Cx<T>::zero();
            beta_sh = x0;
            inv_sh = Cx<T>::zero();
        } else {
            // beta = -phase(x0) alpha, alpha = ||x||; v0 = x0 - beta = phase(x0) (|x0| + alpha);
            // tau = -v0 / beta = (|x0| + alpha) / alpha; 1 / v0 = conj(phase) / (|x0| + alpha).
            // One rsqrt per square root and one reciprocal (long float64 sequences on this GPU).
            const double ax2 = Cx<T>::ab2(x0);
            const double n2 = ax2 + nrm2;
            const double ia = rsqrt(n2);                      // 1 / alpha
            const double alpha = n2 * ia;
            double a0 = 0.0;
            T ph = Cx<T>::one();
            if (ax2 > 0.0) {
                const double ia0 = rsqrt(ax2);
                a0 = ax2 * ia0;
                ph = Cx<T>::sc(ia0, x0);
            }
            const double s = a0 + alpha;
            beta_sh = Cx<T>::sc(-alpha, ph);
            inv_sh = Cx<T>::sc(1.0 / s, Cx<T>::cj(ph));
            tau_sh = Cx<T>::sc(s * ia, Cx<T>::one());
        }
    }
    __syncthreads();
    const T inv = inv_sh;
    const bool zero = Cx<T>::ab2(tau_sh) == 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x)
        v[i] = i == 0 ? Cx<T>::one() : (zero ? Cx<T>::zero() : Cx<T>::mul(x[i], inv));
    *beta_out = beta_sh;
    const T tau = tau_sh;
    __syncthreads();
    return tau;
}

// ----------------------------------------------------------------------------- least squares
// Householder QR of the (rows x m) matrix W (copy of Hbar) and of the right-hand side;
// d = R^{-1} (Q^H c)[0..m-1].  All threads participate.
template <class T>
__device__ void lsq_solve(T *W, int ldw, int rows, int m, T *rhs, T *d, T *v) {
    // last row that can be nonzero in column j once columns 0..j-1 are reduced: the running
    // maximum of each column's last nonzero row (a Hessenberg column j ends at j + 1; the
    // full leading block left by a GMRES-DR restart ends at k); the reflector of column j
    // only needs rows j..end_j, which keeps the factorisation exact.
    __shared__ int end_s[kMaxM + 1];
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        int e = 0;
        for (int i = rows - 1; i > 0; --i) {
            const T w = W[i + (size_t)c * ldw];
            const unsigned long long *b = reinterpret_cast<const unsigned long long *>(&w);
            bool nz = (b[0] << 1) != 0ull;                    // nonzero, sign bit ignored
            if (sizeof(T) == 16) nz = nz || (b[1] << 1) != 0ull;
            if (nz) { e = i; break; }
        }
        end_s[c] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 1; c < m; ++c) end_s[c] = max(end_s[c], end_s[c - 1]);
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        const int len = max(end_s[j], j) - j + 1;
        T beta;
        const T tau = house_par<T>(W + j + (size_t)j * ldw, len, v, &beta);
        // apply H = I - tau v v^H to columns j+1..m-1 and to rhs (column index m)
        for (int c = j + 1 + threadIdx.x; c <= m; c += blockDim.x) {
            T *col = (c < m) ? (W + (size_t)c * ldw) : rhs;
            T s = Cx<T>::zero();
            for (int i = 0; i < len; ++i) s = add(s, Cx<T>::mul(Cx<T>::cj(v[i]), col[j + i]));
            s = Cx<T>::mul(tau, s);
            for (int i = 0; i < len; ++i) col[j + i] = subt(col[j + i], Cx<T>::mul(v[i], s));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += blockDim.x) W[j + i + (size_t)j * ldw] = i == 0 ? beta : Cx<T>::zero();
        __syncthreads();
    }
    // back substitution R d = rhs, column oriented: d_i, then all rows above updated at once
    __shared__ T di_s;
    for (int i = m - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            T rii = W[i + (size_t)i * ldw];
            di_s = Cx<T>::ab2(rii) > 0 ? Cx<T>::div(rhs[i], rii) : Cx<T>::zero();
            d[i] = di_s;
        }
        __syncthreads();
        const T di = di_s;
        for (int r = threadIdx.x; r < i; r += blockDim.x) rhs[r] = subt(rhs[r], Cx<T>::mul(W[r + (size_t)i * ldw], di));
        __syncthreads();
    }
}

// Solve A^H f = e_last for the m x m matrix A (column-major, ld lda) by Gaussian
// elimination with partial pivoting on a copy B = A^H.
template <class T>
__device__ void solve_adjoint_last(const T *A, int lda, int m, T *B, T *f, int *piv) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        B[i + (size_t)j * m] = Cx<T>::cj(A[j + (size_t)i * lda]);
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) f[i] = (i == m - 1) ? Cx<T>::one() : Cx<T>::zero();
    __syncthreads();
    __shared__ int p_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < m; ++j) {
        if (warp == 0) {
            // partial pivoting: the largest |B[i, j]|, ties to the smallest i
            double best = -1.0;
            int p = j;
            for (int i = j + lane; i < m; i += 32) {
                double a = Cx<T>::ab2(B[i + (size_t)j * m]);
                if (a > best) { best = a; p = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                double ob = __shfl_down_sync(0xffffffffu, best, o);
                int op = __shfl_down_sync(0xffffffffu, p, o);
                if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
            }
            if (lane == 0) { p_s = p; piv[j] = p; }
        }
        __syncthreads();
        const int p = p_s;
        if (p != j) {
            for (int c = threadIdx.x; c < m; c += blockDim.x) {
                T t = B[j + (size_t)c * m];
                B[j + (size_t)c * m] = B[p + (size_t)c * m];
                B[p + (size_t)c * m] = t;
            }
            if (threadIdx.x == 0) { T t = f[j]; f[j] = f[p]; f[p] = t; }
        }
        __syncthreads();
        const T pivv = B[j + (size_t)j * m];
        const bool ok = Cx<T>::ab2(pivv) > 0;
        const T ipiv = ok ? Cx<T>::div(Cx<T>::one(), pivv) : Cx<T>::zero();
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
            if (!ok) break;
            T l = Cx<T>::mul(B[i + (size_t)j * m], ipiv);
            for (int c = j + 1; c < m; ++c) B[i + (size_t)c * m] = subt(B[i + (size_t)c * m], Cx<T>::mul(l, B[j + (size_t)c * m]));
            f[i] = subt(f[i], Cx<T>::mul(l, f[j]));
            B[i + (size_t)j * m] = Cx<T>::zero();
        }
        __syncthreads();
    }
    // back substitution U f = f, column oriented
    __shared__ T fi_s;
    for (int i = m - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            T bii = B[i + (size_t)i * m];
            fi_s = Cx<T>::ab2(bii) > 0 ? Cx<T>::div(f[i], bii) : Cx<T>::zero();
            f[i] = fi_s;
        }
        __syncthreads();
        const T fi = fi_s;
        for (int r = threadIdx.x; r < i; r += blockDim.x) f[r] = subt(f[r], Cx<T>::mul(B[r + (size_t)i * m], fi));
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- Hessenberg form
// A (m x m, ld m) <- Q^H A Q upper Hessenberg; Z <- Q (Z must hold I on entry).
template <class T>
__device__ void hessenberg(T *A, int m, T *Z, T *v) {
    for (int j = 0; j + 2 < m; ++j) {
        const int len = m - j - 1;
        T beta;
        const T tau = house_par<T>(A + (j + 1) + (size_t)j * m, len, v, &beta);
        if (Cx<T>::ab2(tau) == 0.0) continue;
        // left: rows j+1..m-1, columns j..m-1: A <- H A = A - tau v (v^H A)
        for (int c = j + threadIdx.x; c < m; c += blockDim.x) {
            T *col = A + (size_t)c * m + j + 1;
            T s = Cx<T>::zero();
            for (int i = 0; i < len; ++i) s = add(s, Cx<T>::mul(Cx<T>::cj(v[i]), col[i]));
            s = Cx<T>::mul(tau, s);
            for (int i = 0; i < len; ++i) col[i] = subt(col[i], Cx<T>::mul(v[i], s));
        }
        __syncthreads();
        // right: all rows, columns j+1..m-1: A <- A H^H = A - conj(tau) (A v) v^H; Z <- Z H^H
        for (int rr = threadIdx.x; rr < 2 * m; rr += blockDim.x) {
            T *M = rr < m ? A : Z;
            const int r = rr < m ? rr : rr - m;
            T s = Cx<T>::zero();
            for (int i = 0; i < len; ++i) s = add(s, Cx<T>::mul(M[r + (size_t)(j + 1 + i) * m], v[i]));
            s = Cx<T>::mul(s, Cx<T>::cj(tau));
            for (int i = 0; i < len; ++i)
                M[r + (size_t)(j + 1 + i) * m] = subt(M[r + (size_t)(j + 1 + i) * m], Cx<T>::mul(s, Cx<T>::cj(v[i])));
        }
        __syncthreads();
    }
    // clean below the subdiagonal
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        if (i > j + 1) A[e] = Cx<T>::zero();
    }
    __syncthreads();
}

// ----------------------------------------------------------------------------- Schur form: shared pieces
// Cost model of the QR sweeps on this GPU: every float64 warp instruction occupies its SM
// sub-partition's float64 unit for tens of cycles whatever the number of active lanes, and
// sqrt / division / hypot are long sequences of them.  So a bulge-chasing step is organised
// as two phases between two barriers: (1) all warps apply the current transform to the rows
// it touches (and to part of the Schur vector rows), (2) warp 0 updates the few entries that
// define the next transform and computes it with one rsqrt (and, real case, one reciprocal),
// lanes in parallel, while warps 1.. apply the column transform to the remaining rows and
// Schur vector rows.  Bulge entries that the next transform annihilates are stored as exact
// zeros, so no clean-up pass is needed.
constexpr unsigned kFull = 0xffffffffu;

// Complex Givens rotation G = [conj(a) conj(b); -b a] with G [x; y] = [r; 0], r = ||(x, y)||:
// a = x / r, b = y / r.  Warp-wide call; lanes 0..3 hold x.re, x.im, y.re, y.im in v and
// write a.re, a.im, b.re, b.im to rs[0..3].  (x, y) = 0 gives the identity.
__device__ __forceinline__ void givens_warp(double v, double *rs) {
    const int lane = threadIdx.x & 31;
    double s2 = v * v;
    s2 += __shfl_xor_sync(kFull, s2, 1);
    s2 += __shfl_xor_sync(kFull, s2, 2);
    s2 = __shfl_sync(kFull, s2, 0);
    double out;
    if (s2 == 0.0) {
        out = lane == 0 ? 1.0 : 0.0;
    } else if (s2 > 1e-280 && s2 < 1e280) {
        out = v * rsqrt(s2);
    } else {
        // scale by the largest component first (no overflow or underflow in the squares)
        double mx = fabs(v);
        mx = fmax(mx, __shfl_xor_sync(kFull, mx, 1));
        mx = fmax(mx, __shfl_xor_sync(kFull, mx, 2));
        mx = __shfl_sync(kFull, mx, 0);
        const double w = v * (1.0 / mx);
        double t2 = w * w;
        t2 += __shfl_xor_sync(kFull, t2, 1);
        t2 += __shfl_xor_sync(kFull, t2, 2);
        t2 = __shfl_sync(kFull, t2, 0);
        out = w * rsqrt(t2);
    }
    if (lane < 4) rs[lane] = out;
}

// Householder reflector (I - tau u u^T), u = (1, u1, u2), mapping (x, y, z) to (beta, 0, 0),
// beta = -sign(x) ||(x, y, z)||: tau = (beta - x) / beta, u_i = (y, z) / (x - beta).
// Warp-wide call; lanes 0..2 hold x, y, z in v (z = 0 for a 2-vector); writes tau, u1, u2
// to hs[0..2].  y = z = 0 gives tau = 0 (the identity).
__device__ __forceinline__ void house3_warp(double v, double *hs) {
    const int lane = threadIdx.x & 31;
    const double x = __shfl_sync(kFull, v, 0), y = __shfl_sync(kFull, v, 1), z = __shfl_sync(kFull, v, 2);
    const double sn = y * y + z * z;
    if (lane == 0) {
        double tau = 0.0, u1 = 0.0, u2 = 0.0;
        if (sn != 0.0) {
            double n2 = x * x + sn;
            double xs = x, ys = y, zs = z;
            if (!(n2 > 1e-280 && n2 < 1e280)) {      // rescale (the reflector is scale invariant)
                const double mx = fmax(fabs(x), fmax(fabs(y), fabs(z)));
                const double r = 1.0 / mx;
                xs = x * r; ys = y * r; zs = z * r;
                n2 = xs * xs + (ys * ys + zs * zs);
            }
            const double inv = rsqrt(n2);                  // 1 / ||(x, y, z)||
            const double beta = -copysign(n2 * inv, xs);
            const double u0 = xs - beta;
            const double ru0 = 1.0 / u0;
            tau = u0 * copysign(inv, xs);                  // -u0 / beta
            u1 = ys * ru0;
            u2 = zs * ru0;
        }
        hs[0] = tau;
        hs[1] = u1;
        hs[2] = u2;
    }
}

// ----------------------------------------------------------------------------- real Schur form
// Francis double-shift QR on the real upper Hessenberg H (m x m, ld m), accumulating Z.
// Returns 0 on success, 1 if an eigenvalue failed to converge in 40 m sweeps.
__device__ int real_schur(double *H, int m, double *Z) {
    __shared__ int hi_s, l_s, status_s, act_s;
    __shared__ double hs_s[3];
    __shared__ double x_s, y_s, z_s;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) { hi_s = m - 1; status_s = 0; }
    __syncthreads();
    int its = 0, total = 0;
    while (true) {
        if (tid < 32) {
            // the active block: the largest l <= hi with a negligible H[l, l-1] (0 if none),
            // found by warp 0 with a ballot over the candidates
            const int hi = hi_s;
            __syncwarp();          // every lane has read hi_s before lane 0 may update it
            int l = 0;
            if (hi > 0) {
                for (int base = hi; base > 0 && l == 0; base -= 32) {
                    const int cand = base - lane;
                    bool neg = false;
                    if (cand > 0) {
                        double s = fabs(H[(cand - 1) + (size_t)(cand - 1) * m]) + fabs(H[cand + (size_t)cand * m]);
                        if (s == 0.0) s = 1.0;
                        neg = fabs(H[cand + (size_t)(cand - 1) * m]) <= kEps * s;
                    }
                    const unsigned bal = __ballot_sync(kFull, neg);
                    if (bal) l = base - (__ffs(bal) - 1);     // lowest lane = largest index
                }
            }
            if (lane == 0) {
                if (l > 0) H[l + (size_t)(l - 1) * m] = 0.0;
                act_s = 0;
                if (hi < 0) act_s = -1;
                else {
                    l_s = l;
                    if (l == hi) { hi_s = hi - 1; act_s = 1; }
                    else if (l == hi - 1) { act_s = 2; }   // 2x2 block: standardise below
                    else act_s = 3;                         // QR sweep on l..hi
                }
            }
        }
        __syncthreads();
        const int act = act_s;
        if (act < 0) break;
        if (act == 1) { its = 0; continue; }
        const int hi = hi_s, l = l_s;
        if (act == 2) {
            // 2x2 block [a b; c d] at (hi-1, hi): real eigenvalues -> rotate to triangular form
            __shared__ double cs_s, sn_s;
            __shared__ int rot_s;
            if (tid == 0) {
                double a = H[(hi - 1) + (size_t)(hi - 1) * m], b = H[(hi - 1) + (size_t)hi * m];
                double c = H[hi + (size_t)(hi - 1) * m], d = H[hi + (size_t)hi * m];
                double p = 0.5 * (a - d);
                double disc = p * p + b * c;
                rot_s = 0;
                if (disc >= 0.0 && c != 0.0) {
                    // real eigenvalues: lam - d = p + sign(p) sqrt(disc) (no cancellation);
                    // (lam - d, c) is an eigenvector of the block, and the rotation whose
                    // first column it is makes the block upper triangular
                    double e0 = p + copysign(sqrt(disc), p), e1 = c;
                    double nr = hypot(e0, e1);
                    if (nr > 0) {
                        cs_s = e0 / nr;
                        sn_s = e1 / nr;
                        rot_s = 1;
                    }
                }
            }
            __syncthreads();
            if (rot_s) {
                const double cs = cs_s, sn = sn_s;
                // rows hi-1, hi: H <- G^T H for columns hi-1..m-1
                for (int c = hi - 1 + tid; c < m; c += nt) {
                    double h1 = H[(hi - 1) + (size_t)c * m], h2 = H[hi + (size_t)c * m];
                    H[(hi - 1) + (size_t)c * m] = cs * h1 + sn * h2;
                    H[hi + (size_t)c * m] = -sn * h1 + cs * h2;
                }
                __syncthreads();
                // columns hi-1, hi: H <- H G for rows 0..hi, Z <- Z G
                for (int rr = tid; rr < 2 * m; rr += nt) {
                    double *M = rr < m ? H : Z;
                    const int r = rr < m ? rr : rr - m;
                    if (M == H && r > hi) continue;
                    double h1 = M[r + (size_t)(hi - 1) * m], h2 = M[r + (size_t)hi * m];
                    M[r + (size_t)(hi - 1) * m] = cs * h1 + sn * h2;
                    M[r + (size_t)hi * m] = -sn * h1 + cs * h2;
                }
                __syncthreads();
                if (tid == 0) H[hi + (size_t)(hi - 1) * m] = 0.0;
            }
            if (tid == 0) hi_s = hi - 2;
            __syncthreads();
            its = 0;
            continue;
        }
        // ---- double-shift sweep on rows/cols l..hi
        ++its;
        ++total;
        if (total > 40 * m) {
            if (tid == 0) status_s = 1;
            __syncthreads();
            break;
        }
        if (tid == 0) {
            double s, t;
            if (its % 10 == 0) {
                // exceptional shift
                double w = fabs(H[hi + (size_t)(hi - 1) * m]) + fabs(H[(hi - 1) + (size_t)(hi - 2 >= 0 ? hi - 2 : 0) * m]);
                s = 1.5 * w + H[hi + (size_t)hi * m];
                t = w * w;
            } else {
                double a = H[(hi - 1) + (size_t)(hi - 1) * m], b = H[(hi - 1) + (size_t)hi * m];
                double c = H[hi + (size_t)(hi - 1) * m], d = H[hi + (size_t)hi * m];
                s = a + d;
                t = a * d - b * c;
            }
            // first column of (H - s1 I)(H - s2 I) = H^2 - s H + t I
            double h00 = H[l + (size_t)l * m], h01 = H[l + (size_t)(l + 1) * m];
            double h10 = H[(l + 1) + (size_t)l * m], h11 = H[(l + 1) + (size_t)(l + 1) * m];
            x_s = h00 * h00 + h01 * h10 - s * h00 + t;
            y_s = h10 * (h00 + h11 - s);
            z_s = (l + 2 <= hi) ? h10 * H[(l + 2) + (size_t)(l + 1) * m] : 0.0;
        }
        __syncthreads();
        if (warp == 0) house3_warp(lane == 0 ? x_s : lane == 1 ? y_s : lane == 2 ? z_s : 0.0, hs_s);
        __syncthreads();
        for (int kk = l; kk <= hi - 1; ++kk) {
            const int nr = (kk <= hi - 2) ? 3 : 2;
            const double tau = hs_s[0], v1 = hs_s[1], v2 = nr == 3 ? hs_s[2] : 0.0;
            // phase 1: rows kk..kk+nr-1 over columns c0..m-1; Schur vector rows [0, zs)
            const int c0 = kk > l ? kk - 1 : l;
            const int ncol = m - c0;
            const int zs = min(m, max(0, nt - ncol));
            for (int t = tid; t < ncol + zs; t += nt) {
                if (t < ncol) {
                    const int c = c0 + t;
                    const double h0 = H[kk + (size_t)c * m], h1 = H[kk + 1 + (size_t)c * m];
                    const double h2 = nr == 3 ? H[kk + 2 + (size_t)c * m] : 0.0;
                    const double s = tau * fma(v2, h2, fma(v1, h1, h0));
                    const bool bulge = kk > l && c == kk - 1;     // entries the reflector annihilates
                    H[kk + (size_t)c * m] = h0 - s;
                    H[kk + 1 + (size_t)c * m] = bulge ? 0.0 : fma(-s, v1, h1);
                    if (nr == 3) H[kk + 2 + (size_t)c * m] = bulge ? 0.0 : fma(-s, v2, h2);
                } else {
                    double *zr = Z + (t - ncol);
                    const double h0 = zr[(size_t)kk * m], h1 = zr[(size_t)(kk + 1) * m];
                    const double h2 = nr == 3 ? zr[(size_t)(kk + 2) * m] : 0.0;
                    const double s = tau * fma(v2, h2, fma(v1, h1, h0));
                    zr[(size_t)kk * m] = h0 - s;
                    zr[(size_t)(kk + 1) * m] = fma(-s, v1, h1);
                    if (nr == 3) zr[(size_t)(kk + 2) * m] = fma(-s, v2, h2);
                }
            }
            __syncthreads();
            // phase 2: columns kk..kk+nr-1 of rows 0..rmax and of Schur vector rows [zs, m)
            const int rmax = (kk + 3 < hi) ? kk + 3 : hi;
            if (warp == 0) {
                // rows kk+1..rmax (at most 3, one per lane), then the next reflector from
                // column kk of those rows
                const int r = kk + 1 + lane;
                double xv = 0.0;
                if (lane < 3 && r <= rmax) {
                    double *hr = H + r;
                    const double h0 = hr[(size_t)kk * m], h1 = hr[(size_t)(kk + 1) * m];
                    const double h2 = nr == 3 ? hr[(size_t)(kk + 2) * m] : 0.0;
                    const double s = tau * fma(v2, h2, fma(v1, h1, h0));
                    xv = h0 - s;
                    hr[(size_t)kk * m] = xv;
                    hr[(size_t)(kk + 1) * m] = fma(-s, v1, h1);
                    if (nr == 3) hr[(size_t)(kk + 2) * m] = fma(-s, v2, h2);
                }
                __syncwarp();
                if (kk < hi - 1) house3_warp(xv, hs_s);      // z = 0 when kk + 3 > hi
            } else {
                const int nh = kk + 1;            // rows 0..kk
                const int nz = m - zs;
                for (int t = tid - 32; t < nh + nz; t += nt - 32) {
                    double *hr = t < nh ? H + t : Z + zs + (t - nh);
                    const double h0 = hr[(size_t)kk * m], h1 = hr[(size_t)(kk + 1) * m];
                    const double h2 = nr == 3 ? hr[(size_t)(kk + 2) * m] : 0.0;
                    const double s = tau * fma(v2, h2, fma(v1, h1, h0));
                    hr[(size_t)kk * m] = h0 - s;
                    hr[(size_t)(kk + 1) * m] = fma(-s, v1, h1);
                    if (nr == 3) hr[(size_t)(kk + 2) * m] = fma(-s, v2, h2);
                }
            }
            __syncthreads();
        }
    }
    return status_s;
}

// ----------------------------------------------------------------------------- complex Schur form
// Wilkinson single-shift QR on the complex upper Hessenberg H, accumulating Z.  The
// negligibility test uses |re| + |im| (no square roots).
__device__ __forceinline__ double cabs1(cplx a) { return fabs(a.re) + fabs(a.im); }

__device__ int complex_schur(cplx *H, int m, cplx *Z) {
    __shared__ int hi_s, l_s, act_s, status_s;
    __shared__ double rs_s[4];      // a.re, a.im, b.re, b.im of the current rotation
    __shared__ cplx x_s, y_s;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) { hi_s = m - 1; status_s = 0; }
    __syncthreads();
    int its = 0, total = 0;
    while (true) {
        if (tid < 32) {
            const int hi = hi_s;
            __syncwarp();          // every lane has read hi_s before lane 0 may update it
            int l = 0;
            if (hi > 0) {
                for (int base = hi; base > 0 && l == 0; base -= 32) {
                    const int cand = base - lane;
                    bool neg = false;
                    if (cand > 0) {
                        double s = cabs1(H[(cand - 1) + (size_t)(cand - 1) * m]) + cabs1(H[cand + (size_t)cand * m]);
                        if (s == 0.0) s = 1.0;
                        neg = cabs1(H[cand + (size_t)(cand - 1) * m]) <= kEps * s;
                    }
                    const unsigned bal = __ballot_sync(kFull, neg);
                    if (bal) l = base - (__ffs(bal) - 1);
                }
            }
            if (lane == 0) {
                if (l > 0) H[l + (size_t)(l - 1) * m] = {0.0, 0.0};
                act_s = 0;
                if (hi <= 0) act_s = -1;
                else {
                    l_s = l;
                    if (l == hi) { hi_s = hi - 1; act_s = 1; }
                    else act_s = 2;
                }
            }
        }
        __syncthreads();
        const int act = act_s;
        if (act < 0) break;
        if (act == 1) { its = 0; continue; }
        ++its;
        ++total;
        if (total > 40 * m) {
            if (tid == 0) status_s = 1;
            __syncthreads();
            break;
        }
        const int hi = hi_s, l = l_s;
        if (tid == 0) {
            cplx a = H[(hi - 1) + (size_t)(hi - 1) * m], b = H[(hi - 1) + (size_t)hi * m];
            cplx c = H[hi + (size_t)(hi - 1) * m], d = H[hi + (size_t)hi * m];
            cplx mu;
            if (its % 10 == 0) {
                mu = d + mkc(1.5 * cabs_(c), 0.0);
            } else {
                // eigenvalue of [a b; c d] closer to d
                cplx p = 0.5 * (a - d);
                cplx disc = p * p + b * c;
                // principal square root
                double r = cabs_(disc);
                double sr = sqrt(0.5 * (r + disc.re));
                double si = sqrt(fmax(0.0, 0.5 * (r - disc.re)));
                if (disc.im < 0) si = -si;
                cplx sq_ = mkc(sr, si);
                cplx e1 = p + sq_, e2 = p - sq_;
                mu = d + ((abs2(e1) < abs2(e2)) ? e1 : e2);
            }
            x_s = H[l + (size_t)l * m] - mu;
            y_s = H[(l + 1) + (size_t)l * m];
        }
        __syncthreads();
        if (warp == 0) givens_warp(lane == 0 ? x_s.re : lane == 1 ? x_s.im : lane == 2 ? y_s.re : y_s.im, rs_s);
        __syncthreads();
        for (int kk = l; kk <= hi - 1; ++kk) {
            const cplx a = mkc(rs_s[0], rs_s[1]), b = mkc(rs_s[2], rs_s[3]);
            // phase 1: rows kk, kk+1 over columns c0..m-1 (H <- G H); Schur vector rows [0, zs)
            const int c0 = kk > l ? kk - 1 : l;
            const int ncol = m - c0;
            const int zs = min(m, max(0, nt - ncol));
            for (int t = tid; t < ncol + zs; t += nt) {
                if (t < ncol) {
                    const int c = c0 + t;
                    const cplx h1 = H[kk + (size_t)c * m], h2 = H[kk + 1 + (size_t)c * m];
                    H[kk + (size_t)c * m] = conj(a) * h1 + conj(b) * h2;
                    // the entry the rotation annihilates (the bulge) is stored as an exact zero
                    H[kk + 1 + (size_t)c * m] = (kk > l && c == kk - 1) ? mkc(0.0, 0.0) : a * h2 - b * h1;
                } else {
                    cplx *zr = Z + (t - ncol);
                    const cplx h1 = zr[(size_t)kk * m], h2 = zr[(size_t)(kk + 1) * m];
                    zr[(size_t)kk * m] = h1 * a + h2 * b;
                    zr[(size_t)(kk + 1) * m] = h2 * conj(a) - h1 * conj(b);
                }
            }
            __syncthreads();
            // phase 2: columns kk, kk+1 (M <- M G^H) of rows 0..rmax and Schur vector rows [zs, m)
            const int rmax = (kk + 2 < hi) ? kk + 2 : hi;
            if (warp == 0) {
                // rows kk+1..rmax: lane q < 8 computes one real part: column kk + (q >> 2),
                // row kk + 1 + ((q >> 1) & 1), real (q even) or imaginary part; then the next
                // rotation from column kk of rows kk+1, kk+2 (lanes 0..3)
                const int q = lane & 7;
                const int r = kk + 1 + ((q >> 1) & 1);
                const int col = kk + (q >> 2);
                const bool live = lane < 8 && r <= rmax;
                double val = 0.0;
                if (live) {
                    const cplx h1 = H[r + (size_t)kk * m], h2 = H[r + (size_t)(kk + 1) * m];
                    const cplx o = (q >> 2) == 0 ? h1 * a + h2 * b : h2 * conj(a) - h1 * conj(b);
                    val = (q & 1) ? o.im : o.re;
                }
                __syncwarp();
                if (live) reinterpret_cast<double *>(H + r + (size_t)col * m)[q & 1] = val;
                __syncwarp();
                if (kk < hi - 1) givens_warp(val, rs_s);
            } else {
                const int nh = kk + 1;            // rows 0..kk
                const int nz = m - zs;
                for (int t = tid - 32; t < nh + nz; t += nt - 32) {
                    cplx *hr = t < nh ? H + t : Z + zs + (t - nh);
                    const cplx h1 = hr[(size_t)kk * m], h2 = hr[(size_t)(kk + 1) * m];
                    hr[(size_t)kk * m] = h1 * a + h2 * b;
                    hr[(size_t)(kk + 1) * m] = h2 * conj(a) - h1 * conj(b);
                }
            }
            __syncthreads();
        }
    }
    return status_s;
}

// ----------------------------------------------------------------------------- eigenvalues
// From the real Schur form T: eigenvalue j as (re, im).  2 x 2 blocks are the complex pairs.
__device__ void real_schur_eigs(const double *T, int m, double *wr, double *wi) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const bool lower = (j + 1 < m) && T[(j + 1) + (size_t)j * m] != 0.0;   // j is top of a block
        const bool upper = (j > 0) && T[j + (size_t)(j - 1) * m] != 0.0;       // j is bottom of a block
        if (lower || upper) {
            const int t = lower ? j : j - 1;
            double a = T[t + (size_t)t * m], b = T[t + (size_t)(t + 1) * m];
            double c = T[(t + 1) + (size_t)t * m], d = T[(t + 1) + (size_t)(t + 1) * m];
            double p = 0.5 * (a - d);
            double disc = p * p + b * c;
            double im = sqrt(fmax(-disc, 0.0));
            wr[j] = 0.5 * (a + d);
            wi[j] = lower ? im : -im;
        } else {
            wr[j] = T[j + (size_t)j * m];
            wi[j] = 0.0;
        }
    }
    __syncthreads();
}

// Back substitution for the eigenvector of eigenvalue (lr, li) at Schur position j of the
// real quasi-triangular T (one thread).  Output y (complex, length m, zero below j).
__device__ void real_schur_vector(const double *T, int m, int j, double lr, double li, cplx *y,
                                  double tnorm) {
    const double small = fmax(kEps * tnorm, 1e-300);
    const cplx lam = mkc(lr, li);
    for (int i = 0; i < m; ++i) y[i] = {0.0, 0.0};
    int top;
    if (li == 0.0) {
        y[j] = {1.0, 0.0};
        top = j - 1;
    } else {
        // 2x2 block at (t, t+1) containing j
        const bool jtop = (j + 1 < m) && T[(j + 1) + (size_t)j * m] != 0.0;
        const int t = jtop ? j : j - 1;
        double a = T[t + (size_t)t * m], b = T[t + (size_t)(t + 1) * m];
        double c = T[(t + 1) + (size_t)t * m], d = T[(t + 1) + (size_t)(t + 1) * m];
        if (fabs(b) >= fabs(c)) {
            y[t] = {1.0, 0.0};
            y[t + 1] = cdiv(lam - mkc(a, 0.0), mkc(b, 0.0));      // (a - lam) y0 + b y1 = 0
        } else {
            y[t + 1] = {1.0, 0.0};
            y[t] = cdiv(lam - mkc(d, 0.0), mkc(c, 0.0));          // c y0 + (d - lam) y1 = 0
        }
        top = t - 1;
        j = t + 1;
    }
    int i = top;
    while (i >= 0) {
        const bool blk = (i > 0) && T[i + (size_t)(i - 1) * m] != 0.0;   // rows (i-1, i) form a block
        if (!blk) {
            cplx s = {0.0, 0.0};
            for (int l = i + 1; l <= j; ++l) s = s + T[i + (size_t)l * m] * y[l];
            cplx den = mkc(T[i + (size_t)i * m], 0.0) - lam;
            if (cabs_(den) < small) den = mkc(small, 0.0);
            y[i] = cdiv(-s, den);
            i -= 1;
        } else {
            const int t = i - 1;
            cplx s0 = {0.0, 0.0}, s1 = {0.0, 0.0};
            for (int l = i + 1; l <= j; ++l) {
                s0 = s0 + T[t + (size_t)l * m] * y[l];
                s1 = s1 + T[i + (size_t)l * m] * y[l];
            }
            // [a-lam b; c d-lam] [y_t; y_i] = -[s0; s1]
            cplx a = mkc(T[t + (size_t)t * m], 0.0) - lam, b = mkc(T[t + (size_t)i * m], 0.0);
            cplx c = mkc(T[i + (size_t)t * m], 0.0), d = mkc(T[i + (size_t)i * m], 0.0) - lam;
            cplx det = a * d - b * c;
            if (cabs_(det) < small * small) det = mkc(small * small, 0.0);
            y[t] = cdiv(-(d * s0) + b * s1, det);
            y[i] = cdiv(c * s0 - a * s1, det);
            i -= 2;
        }
    }
}

__device__ void complex_schur_vector(const cplx *T, int m, int j, cplx *y, double tnorm) {
    const double small = fmax(kEps * tnorm, 1e-300);
    const cplx lam = T[j + (size_t)j * m];
    for (int i = 0; i < m; ++i) y[i] = {0.0, 0.0};
    y[j] = {1.0, 0.0};
    for (int i = j - 1; i >= 0; --i) {
        cplx s = {0.0, 0.0};
        for (int l = i + 1; l <= j; ++l) s = s + T[i + (size_t)l * m] * y[l];
        cplx den = T[i + (size_t)i * m] - lam;
        if (cabs_(den) < small) den = mkc(small, 0.0);
        y[i] = cdiv(-s, den);
    }
}

// order: by |theta|, then Re, then Im >= 0 first (one thread, insertion sort; moduli given)
__device__ bool ritz_less_m(double ma, double ar, double ai, double mb, double br, double bi) {
    if (ma != mb) return ma < mb;
    if (ar != br) return ar < br;
    int ka = ai >= 0 ? 0 : 1, kb = bi >= 0 ? 0 : 1;
    return ka < kb;
}

}  // namespace

// ============================================================================= kernels

// Cholesky G = R^H R (G Hermitian positive definite, upper triangle given, k x k) and
// Rinv = R^{-1}.  info[0] = 0 on success, j+1 if the j-th pivot is not positive.
template <class D>
__global__ void k_chol_inv(const D *G, int k, D *R, D *Rinv, int *info) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        int i = e % k, j = e / k;
        R[e] = i <= j ? G[e] : Cx<D>::zero();
        Rinv[e] = Cx<D>::zero();
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            double djj = Cx<D>::re(R[j + (size_t)j * k]);
            for (int i = 0; i < j; ++i) djj -= Cx<D>::ab2(R[i + (size_t)j * k]);
            if (!(djj > 0.0) && !bad) bad = j + 1;
            R[j + (size_t)j * k] = Cx<D>::sc(sqrt(fmax(djj, 1e-300)), Cx<D>::one());
        }
        __syncthreads();
        const D rjj = R[j + (size_t)j * k];
        for (int c = j + 1 + threadIdx.x; c < k; c += blockDim.x) {
            D s = R[j + (size_t)c * k];
            for (int i = 0; i < j; ++i) s = subt(s, Cx<D>::mul(Cx<D>::cj(R[i + (size_t)j * k]), R[i + (size_t)c * k]));
            R[j + (size_t)c * k] = Cx<D>::div(s, rjj);
        }
        __syncthreads();
    }
    // Rinv: solve R X = I column by column (thread per column)
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        for (int i = c; i >= 0; --i) {
            D s = (i == c) ? Cx<D>::one() : Cx<D>::zero();
            for (int l = i + 1; l <= c; ++l) s = subt(s, Cx<D>::mul(R[i + (size_t)l * k], Rinv[l + (size_t)c * k]));
            Rinv[i + (size_t)c * k] = Cx<D>::div(s, R[i + (size_t)i * k]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) info[0] = bad;
}

// Inverse of a general k x k matrix by Gauss-Jordan with partial pivoting (W: scratch
// 2 k^2).  info[0] = 0, or j+1 for a zero pivot.
template <class D>
__global__ void k_inverse(const D *H, int k, D *Hinv, D *W, int *info) {
    __shared__ int p_s, bad;
    D *A = W;
    D *B = W + (size_t)k * k;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        A[e] = H[e];
        B[e] = (e % k == e / k) ? Cx<D>::one() : Cx<D>::zero();
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            int p = j;
            double best = Cx<D>::ab2(A[j + (size_t)j * k]);
            for (int i = j + 1; i < k; ++i)
                if (Cx<D>::ab2(A[i + (size_t)j * k]) > best) { best = Cx<D>::ab2(A[i + (size_t)j * k]); p = i; }
            if (best == 0.0 && !bad) bad = j + 1;
            p_s = p;
        }
        __syncthreads();
        const int p = p_s;
        if (p != j) {
            for (int c = threadIdx.x; c < k; c += blockDim.x) {
                D t = A[j + (size_t)c * k]; A[j + (size_t)c * k] = A[p + (size_t)c * k]; A[p + (size_t)c * k] = t;
                t = B[j + (size_t)c * k]; B[j + (size_t)c * k] = B[p + (size_t)c * k]; B[p + (size_t)c * k] = t;
            }
        }
        __syncthreads();
        const D piv = A[j + (size_t)j * k];
        if (Cx<D>::ab2(piv) == 0.0) { __syncthreads(); continue; }
        // scale row j
        for (int c = threadIdx.x; c < k; c += blockDim.x) {
            A[j + (size_t)c * k] = Cx<D>::div(A[j + (size_t)c * k], piv);
            B[j + (size_t)c * k] = Cx<D>::div(B[j + (size_t)c * k], piv);
        }
        __syncthreads();
        // eliminate column j from the other rows (thread per row)
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            if (i == j) continue;
            D f = A[i + (size_t)j * k];
            for (int c = 0; c < k; ++c) {
                A[i + (size_t)c * k] = subt(A[i + (size_t)c * k], Cx<D>::mul(f, A[j + (size_t)c * k]));
                B[i + (size_t)c * k] = subt(B[i + (size_t)c * k], Cx<D>::mul(f, B[j + (size_t)c * k]));
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) Hinv[e] = B[e];
    if (threadIdx.x == 0) info[0] = bad;
}

// out = M c (k x k times k), one thread per row.
template <class D>
__global__ void k_small_gemv(const D *M, int k, const D *c, D *out) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        D s = Cx<D>::zero();
        for (int j = 0; j < k; ++j) s = add(s, Cx<D>::mul(M[i + (size_t)j * k], c[j]));
        out[i] = s;
    }
}

// ----------------------------------------------------------------------------- GMRES-DR restart
// See tg_small.cuh for the argument layout.
template <class T>
__device__ __forceinline__ void gmresdr_restart_body(const GdrArgs<T> &a) {
    const int m = a.m;
    const int rows = m + 1;
    const int ldh = a.ldh;
    // W: (m+1) x m (least-squares copy), later the m x m eigen matrix / Schur form;
    // Z: m x m Schur vectors.  Both live in shared memory when the launch provided it
    // (the QR sweeps are a long chain of dependent small steps, so their latency rules).
    extern __shared__ __align__(16) unsigned char gdr_smem[];
    T *sm = reinterpret_cast<T *>(gdr_smem);
    T *W = a.smem >= 1 ? sm : a.work;
    T *Z = a.smem >= 2 ? sm + (size_t)rows * m : a.work + (size_t)rows * m;
    T *B = a.smem >= 3 ? sm + (size_t)rows * m + (size_t)m * m : a.work + (size_t)rows * m + (size_t)m * m;  // m x m (LU)
    T *vtmp = a.work + (size_t)rows * m + 2 * (size_t)m * m;   // 2 (m+1) vectors
    T *f = vtmp + 2 * (m + 1);
    cplx *Ysm = a.smem >= 4 ? reinterpret_cast<cplx *>(sm + (size_t)rows * m + 2 * (size_t)m * m) : a.ywork;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    T *res = a.res;
    __shared__ int piv_s[kMaxM + 1];

    long long t_mark = clock64();
    const bool rr_mode = a.mode == 1;
    if (rr_mode) {
        // Rayleigh-Ritz: the eigen matrix is H itself
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = e % m, j = e / m;
            W[e] = a.H[i + (size_t)j * ldh];
            Z[e] = (i == j) ? Cx<T>::one() : Cx<T>::zero();
        }
        if (threadIdx.x == 0) a.info->rnorm = 0.0;
        __syncthreads();
    } else {
    // ---- 1. least squares: d = argmin ||c - Hbar d||, res = c - Hbar d
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
        int i = e % rows, j = e / rows;
        W[i + (size_t)j * rows] = a.H[i + (size_t)j * ldh];
    }
    for (int i = threadIdx.x; i < rows; i += blockDim.x) vtmp[m + 1 + i] = a.c[i];
    __syncthreads();
    lsq_solve<T>(W, rows, rows, m, vtmp + (m + 1), a.d, vtmp);
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        T s = a.c[i];
        for (int j = 0; j < m; ++j) s = subt(s, Cx<T>::mul(a.H[i + (size_t)j * ldh], a.d[j]));
        res[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < rows; ++i) s += Cx<T>::ab2(res[i]);
        a.info->rnorm = sqrt(s);
    }

    __syncthreads();
    if (threadIdx.x == 0) { long long _t = clock64(); a.info->phase[0] = _t - t_mark; t_mark = _t; }
    // ---- 2. f = H_m^{-H} e_m and the harmonic matrix M = H_m + |h|^2 f e_m^T (in W, ld m)
    solve_adjoint_last<T>(a.H, ldh, m, B, f, piv_s);
    const T hm = a.H[m + (size_t)(m - 1) * ldh];
    const double hm2 = Cx<T>::ab2(hm);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        T v = a.H[i + (size_t)j * ldh];
        if (j == m - 1) v = add(v, Cx<T>::sc(hm2, f[i]));
        W[e] = v;
        Z[e] = (i == j) ? Cx<T>::one() : Cx<T>::zero();
    }
    __syncthreads();
    // z = [-|h|^2 f; h] (restart direction), kept in a.z
    for (int i = threadIdx.x; i < rows; i += blockDim.x) a.z[i] = (i < m) ? Cx<T>::sc(-hm2, f[i]) : hm;

    __syncthreads();
    if (threadIdx.x == 0) { long long _t = clock64(); a.info->phase[1] = _t - t_mark; t_mark = _t; }
    }   // steps 1-2: GMRES-DR restart only
    // ---- 3. eigen-decomposition of M: Hessenberg, Schur, eigenvalues
    hessenberg<T>(W, m, Z, vtmp);
    __syncthreads();
    if (threadIdx.x == 0) { long long _t = clock64(); a.info->phase[2] = _t - t_mark; t_mark = _t; }
    int st;
    double *wr = a.wr, *wi = a.wi;
    if constexpr (sizeof(T) == sizeof(double)) {
        st = real_schur(reinterpret_cast<double *>(W), m, reinterpret_cast<double *>(Z));
        real_schur_eigs(reinterpret_cast<double *>(W), m, wr, wi);
    } else {
        st = complex_schur(reinterpret_cast<cplx *>(W), m, reinterpret_cast<cplx *>(Z));
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            cplx t = reinterpret_cast<cplx *>(W)[j + (size_t)j * m];
            wr[j] = t.re;
            wi[j] = t.im;
        }
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) { long long _t = clock64(); a.info->phase[3] = _t - t_mark; t_mark = _t; }
    double tnorm = 0.0;
    {
        __shared__ double tn_s[32];
        double s2 = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) s2 = fmax(s2, Cx<T>::ab2(W[e]));
        for (int o = 16; o > 0; o >>= 1) s2 = fmax(s2, __shfl_down_sync(0xffffffffu, s2, o));
        if (lane == 0) tn_s[warp] = s2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double mx = 0.0;
            for (int w = 0; w < nwarps; ++w) mx = fmax(mx, tn_s[w]);
            tn_s[0] = sqrt(mx);
        }
        __syncthreads();
        tnorm = tn_s[0];
    }

    // ---- 4. order and select
    __shared__ int kk_s;
    int *ord = a.order;
    __shared__ double mod_s[kMaxM];
    __shared__ double wr_s[kMaxM], wi_s[kMaxM];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        mod_s[i] = hypot(wr[i], wi[i]);
        wr_s[i] = wr[i];
        wi_s[i] = wi[i];
    }
    __syncthreads();
    // stable rank sort, one thread per value: the rank of i is the number of values before it
    // in the order plus the equal values of smaller index (the order a stable sort gives)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int r = 0;
        for (int j = 0; j < m; ++j) {
            if (j == i) continue;
            const bool jl = ritz_less_m(mod_s[j], wr_s[j], wi_s[j], mod_s[i], wr_s[i], wi_s[i]);
            const bool il = ritz_less_m(mod_s[i], wr_s[i], wi_s[i], mod_s[j], wr_s[j], wi_s[j]);
            if (jl || (j < i && !il)) ++r;
        }
        ord[r] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int kk = a.k;
        if (sizeof(T) == sizeof(double) && kk < m) {
            int t = ord[kk - 1];
            if (wi[t] > 0.0) kk += 1;     // keep both members of the conjugate pair
        }
        kk_s = kk;
        a.info->status = st;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a.theta[2 * i] = wr_s[ord[i]];
        a.theta[2 * i + 1] = wi_s[ord[i]];
    }
    __syncthreads();
    const int kk = kk_s;

    __syncthreads();
    if (threadIdx.x == 0) { long long _t = clock64(); a.info->phase[4] = _t - t_mark; t_mark = _t; }
    // ---- 5. eigenvectors of the kept pairs: g = Z y (complex), unit norm; residuals
    // a.gwork holds the kept eigenvectors as complex columns (m x kk)
    cplx *G = a.gwork;
    cplx *Y = Ysm;
    for (int q = threadIdx.x; q < kk; q += blockDim.x) {
        const int j = ord[q];
        cplx *y = Y + (size_t)q * m;
        if constexpr (sizeof(T) == sizeof(double))
            real_schur_vector(reinterpret_cast<const double *>(W), m, j, wr[j], wi[j], y, tnorm);
        else
            complex_schur_vector(reinterpret_cast<const cplx *>(W), m, j, y, tnorm);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * kk; e += blockDim.x) {
        const int i = e % m, q = e / m;
        const cplx *y = Y + (size_t)q * m;
        cplx s = {0.0, 0.0};
        if constexpr (sizeof(T) == sizeof(double)) {
            // real Schur vectors: two real products per term
            const double *Zd = reinterpret_cast<const double *>(Z);
            for (int l = 0; l < m; ++l) {
                const double zl = Zd[i + (size_t)l * m];
                s.re = fma(zl, y[l].re, s.re);
                s.im = fma(zl, y[l].im, s.im);
            }
        } else {
            for (int l = 0; l < m; ++l) s = s + *reinterpret_cast<const cplx *>(&Z[i + (size_t)l * m]) * y[l];
        }
        G[i + (size_t)q * m] = s;
    }
    __syncthreads();
    __shared__ double znorm_s;
    if (warp == 0 && !rr_mode) {
        double z2 = 0.0;
        for (int i = lane; i < rows; i += 32) z2 += Cx<T>::ab2(a.z[i]);
        z2 = warp_sum(z2);
        if (lane == 0) znorm_s = sqrt(z2);
    }
    __syncthreads();
    const double znorm = rr_mode ? 0.0 : znorm_s;
    for (int q = warp; q < kk; q += nwarps) {
        cplx *g = G + (size_t)q * m;
        double nr = 0.0;
        for (int i = lane; i < m; i += 32) nr += abs2(g[i]);
        nr = sqrt(warp_sum(nr));
        nr = __shfl_sync(0xffffffffu, nr, 0);
        for (int i = lane; i < m; i += 32) g[i] = g[i] * (1.0 / nr);
        __syncwarp();
        // residual ||Hbar g - theta [g; 0]|| = |g_m| ||z||: an eigenpair of
        // H_m + |h|^2 f e_m^T satisfies H_m g - theta g = -|h|^2 f g_m, and the last row of
        // Hbar g is h g_m, so the residual vector is g_m z with z = [-|h|^2 f; h]
        if (!rr_mode) {
            if (lane == 0) a.eres[q] = sqrt(abs2(g[m - 1])) * znorm;
        } else {
            // Rayleigh-Ritz: ||W g - theta Q g||^2 = g^H (W^H W) g - |theta|^2 for Q^H W g = theta g
            double acc = 0.0;
            for (int i = lane; i < m; i += 32) {
                cplx wg = {0.0, 0.0};
                for (int l = 0; l < m; ++l) {
                    const T w = a.WW[i + (size_t)l * m];
                    cplx wc;
                    if constexpr (sizeof(T) == sizeof(double)) wc = mkc(*reinterpret_cast<const double *>(&w), 0.0);
                    else wc = *reinterpret_cast<const cplx *>(&w);
                    wg = wg + wc * g[l];
                }
                acc += (conj(g[i]) * wg).re;
            }
            acc = warp_sum(acc);
            if (lane == 0) {
                const int j = ord[q];
                a.eres[q] = sqrt(fmax(acc - (wr[j] * wr[j] + wi[j] * wi[j]), 0.0));
            }
        }
    }
    __syncthreads();
    if (rr_mode && warp == 0 && a.start_q < kk) {
        // coefficients of the start vector: Ritz vector start_q with its largest entry made
        // real and positive (ties: the smallest index); real problems keep the real part
        const cplx *g = G + (size_t)a.start_q * m;
        double best = -1.0;
        int imax = 0;
        for (int i = lane; i < m; i += 32)
            if (abs2(g[i]) > best) { best = abs2(g[i]); imax = i; }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, imax, o);
            if (ob > best || (ob == best && oi < imax)) { best = ob; imax = oi; }
        }
        imax = __shfl_sync(0xffffffffu, imax, 0);
        best = __shfl_sync(0xffffffffu, best, 0);
        const cplx ph = conj(g[imax]) * (1.0 / sqrt(best));
        for (int i = lane; i < m; i += 32) {
            const cplx v = g[i] * ph;
            if constexpr (sizeof(T) == sizeof(double)) reinterpret_cast<double *>(a.z)[i] = v.re;
            else reinterpret_cast<cplx *>(a.z)[i] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nconv = 0;
        for (int q = 0; q < a.nev && q < kk; ++q)
            if (a.eres[q] <= a.rtolev * hypot(a.theta[2 * q], a.theta[2 * q + 1])) ++nconv;
        a.info->nconv = nconv;
        a.info->kk = kk;
    }

    __syncthreads();
    if (threadIdx.x == 0) { long long _t = clock64(); a.info->phase[5] = _t - t_mark; t_mark = _t; }
    // ---- 6. P_k: orthonormal basis of the kept span (real: Re/Im of pairs), m x kk
    //          then P_{k+1} = orth([[P_k; 0], z]), stored (m+1) x (kk+1) with ld m+1.
    T *P = a.P;
    __shared__ int ncol_s;
    __shared__ int colof_s[kMaxM + 1];
    if (threadIdx.x == 0) {
        int col = 0;
        for (int q = 0; q < kk; ++q) {
            const double im = a.theta[2 * q + 1];
            if (sizeof(T) == sizeof(double)) {
                if (im == 0.0) { colof_s[q] = col; col += 1; }
                else if (im > 0.0) { colof_s[q] = col; col += 2; }
                else colof_s[q] = -1;      // the partner (Im > 0) supplies both columns
            } else {
                colof_s[q] = col++;
            }
        }
        ncol_s = col;
    }
    __syncthreads();
    for (int q = warp; q < kk; q += nwarps) {
        const int c0 = colof_s[q];
        if (c0 < 0) continue;
        const cplx *g = G + (size_t)q * m;
        const double im = a.theta[2 * q + 1];
        if constexpr (sizeof(T) == sizeof(double)) {
            double *Pd = reinterpret_cast<double *>(P);
            if (im == 0.0) {
                // a real eigenvector computed in complex arithmetic carries a common phase:
                // rotate it onto the real axis through its largest entry (ties: smallest index)
                double best = -1.0;
                int imax = 0;
                for (int i = lane; i < m; i += 32)
                    if (abs2(g[i]) > best) { best = abs2(g[i]); imax = i; }
                for (int o = 16; o > 0; o >>= 1) {
                    double ob = __shfl_down_sync(0xffffffffu, best, o);
                    int oi = __shfl_down_sync(0xffffffffu, imax, o);
                    if (ob > best || (ob == best && oi < imax)) { best = ob; imax = oi; }
                }
                imax = __shfl_sync(0xffffffffu, imax, 0);
                best = __shfl_sync(0xffffffffu, best, 0);
                const cplx ph = conj(g[imax]) * (1.0 / sqrt(best));
                for (int i = lane; i < m; i += 32) Pd[i + (size_t)c0 * rows] = (g[i] * ph).re;
                if (lane == 0) Pd[m + (size_t)c0 * rows] = 0.0;
            } else {
                for (int i = lane; i < m; i += 32) {
                    Pd[i + (size_t)c0 * rows] = g[i].re;
                    Pd[i + (size_t)(c0 + 1) * rows] = g[i].im;
                }
                if (lane == 0) {
                    Pd[m + (size_t)c0 * rows] = 0.0;
                    Pd[m + (size_t)(c0 + 1) * rows] = 0.0;
                }
            }
        } else {
            cplx *Pc = reinterpret_cast<cplx *>(P);
            for (int i = lane; i < m; i += 32) Pc[i + (size_t)c0 * rows] = g[i];
            if (lane == 0) Pc[m + (size_t)c0 * rows] = {0.0, 0.0};
        }
    }
    __syncthreads();
    const int nc = ncol_s;     // == kk
    // append z as column kk (GMRES-DR restart only)
    if (!rr_mode)
        for (int i = threadIdx.x; i < rows; i += blockDim.x) P[i + (size_t)nc * rows] = a.z[i];
    __syncthreads();
    // classical Gram-Schmidt applied twice over the nc + 1 columns (length m+1): per column,
    // the projections on the previous columns in parallel, then the update in parallel
    __shared__ T proj_s[kMaxM + 2];
    __shared__ double nrm_s;
    const int clast = rr_mode ? nc - 1 : nc;
    for (int c = 0; c <= clast; ++c) {
        T *pc = P + (size_t)c * rows;
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = threadIdx.x; q < c; q += blockDim.x) {
                const T *pq = P + (size_t)q * rows;
                T sacc = Cx<T>::zero();
                for (int i = 0; i < rows; ++i) sacc = add(sacc, Cx<T>::mul(Cx<T>::cj(pq[i]), pc[i]));
                proj_s[q] = sacc;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < rows; i += blockDim.x) {
                T acc = pc[i];
                for (int q = 0; q < c; ++q) acc = subt(acc, Cx<T>::mul(proj_s[q], P[i + (size_t)q * rows]));
                pc[i] = acc;
            }
            __syncthreads();
        }
        if (warp == 0) {
            double sq2 = 0.0;
            for (int i = lane; i < rows; i += 32) sq2 += Cx<T>::ab2(pc[i]);
            sq2 = warp_sum(sq2);
            if (lane == 0) nrm_s = sqrt(sq2);
        }
        __syncthreads();
        const double inv = nrm_s > 0 ? 1.0 / nrm_s : 0.0;
        for (int i = threadIdx.x; i < rows; i += blockDim.x) pc[i] = Cx<T>::sc(inv, pc[i]);
        __syncthreads();
    }

    __syncthreads();
    if (threadIdx.x == 0) { long long _t = clock64(); a.info->phase[6] = _t - t_mark; t_mark = _t; }
    if (rr_mode) return;
    // ---- 7. Hnew = P_{k+1}^H Hbar P_k  ((kk+1) x kk, ld m+1 into a.Hnew), cnew = P_{k+1}^H res
    // T1 = Hbar P_k ((m+1) x kk) into W
    for (int e = threadIdx.x; e < rows * nc; e += blockDim.x) {
        const int i = e % rows, q = e / rows;
        T s = Cx<T>::zero();
        for (int j = 0; j < m; ++j) s = add(s, Cx<T>::mul(a.H[i + (size_t)j * ldh], P[j + (size_t)q * rows]));
        W[i + (size_t)q * rows] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (nc + 1) * nc; e += blockDim.x) {
        const int i = e % (nc + 1), q = e / (nc + 1);
        T s = Cx<T>::zero();
        for (int l = 0; l < rows; ++l) s = add(s, Cx<T>::mul(Cx<T>::cj(P[l + (size_t)i * rows]), W[l + (size_t)q * rows]));
        a.Hnew[i + (size_t)q * ldh] = s;
    }
    for (int i = threadIdx.x; i <= nc; i += blockDim.x) {
        T s = Cx<T>::zero();
        for (int l = 0; l < rows; ++l) s = add(s, Cx<T>::mul(Cx<T>::cj(P[l + (size_t)i * rows]), res[l]));
        a.cnew[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.info->phase[7] = clock64() - t_mark;
}

template <class T>
__global__ void __launch_bounds__(kGdrThreads) k_gmresdr_restart(GdrArgs<T> a) {
    gmresdr_restart_body<T>(a);
}

// many independent restart steps, one block each (the batched coarse phase): block b runs
// args[b] when active[b] is set
template <class T>
__global__ void __launch_bounds__(kGdrThreads) k_gmresdr_restart_batch(const GdrArgs<T> *args, const int *active) {
    if (!active[blockIdx.x]) return;
    const GdrArgs<T> a = args[blockIdx.x];
    gmresdr_restart_body<T>(a);
}

// ----------------------------------------------------------------------------- GMRES(m) Givens step
// Column j of the Arnoldi Hessenberg (h[0..j+1], ld = m+1) is rotated by the previous
// rotations, a new rotation zeroes h[j+1]; g (the least-squares right-hand side) is
// updated; state->resid = |g[j+1]|; state->done = 1 when resid <= target or h[j,j] = 0.
template <class D>
__global__ void k_givens_step(D *H, int ldh, int j, D *cs, D *sn, D *g, GivensState *state) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (state->done) return;
    D *h = H + (size_t)j * ldh;
    for (int i = 0; i < j; ++i) {
        D a = h[i], b = h[i + 1];
        h[i] = add(Cx<D>::mul(Cx<D>::cj(cs[i]), a), Cx<D>::mul(Cx<D>::cj(sn[i]), b));
        h[i + 1] = subt(Cx<D>::mul(cs[i], b), Cx<D>::mul(sn[i], a));
    }
    D a = h[j], b = h[j + 1];
    double den = sqrt(Cx<D>::ab2(a) + Cx<D>::ab2(b));
    if (den == 0.0) {
        cs[j] = Cx<D>::one();
        sn[j] = Cx<D>::zero();
    } else {
        cs[j] = Cx<D>::sc(1.0 / den, a);
        sn[j] = Cx<D>::sc(1.0 / den, b);
    }
    h[j] = Cx<D>::sc(den, Cx<D>::one());
    h[j + 1] = Cx<D>::zero();
    g[j + 1] = Cx<D>::sc(-1.0, Cx<D>::mul(sn[j], g[j]));
    g[j] = Cx<D>::mul(Cx<D>::cj(cs[j]), g[j]);
    double resid = sqrt(Cx<D>::ab2(g[j + 1]));
    state->resid = resid;
    state->steps = j + 1;
    if (!(resid > state->target) || den == 0.0 || !isfinite(resid)) state->done = 1;
}

// y = R^{-1} g[0..kj-1] for the rotated (upper triangular) Hessenberg.
template <class D>
__global__ void k_givens_solve(const D *H, int ldh, const D *g, D *y, const GivensState *state) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int kj = state->steps;
    for (int i = kj - 1; i >= 0; --i) {
        D s = g[i];
        for (int c = i + 1; c < kj; ++c) s = subt(s, Cx<D>::mul(H[i + (size_t)c * ldh], y[c]));
        D hii = H[i + (size_t)i * ldh];
        y[i] = Cx<D>::ab2(hii) > 0 ? Cx<D>::div(s, hii) : Cx<D>::zero();
    }
}

// ----------------------------------------------------------------------------- launchers
template <class D>
void launch_chol_inv(const D *G, int k, D *R, D *Rinv, int *info, cudaStream_t s) {
    k_chol_inv<D><<<1, kSmallThreads, 0, s>>>(G, k, R, Rinv, info);
}
template <class D>
void launch_inverse(const D *H, int k, D *Hinv, D *W, int *info, cudaStream_t s) {
    k_inverse<D><<<1, kSmallThreads, 0, s>>>(H, k, Hinv, W, info);
}
template <class D>
void launch_small_gemv(const D *M, int k, const D *c, D *out, cudaStream_t s) {
    k_small_gemv<D><<<1, kSmallThreads, 0, s>>>(M, k, c, out);
}
template <class T>
cudaError_t launch_gmresdr_restart(const GdrArgs<T> &a_in, cudaStream_t s) {
    GdrArgs<T> a = a_in;
    // W, Z, B (T) and the eigenvector work Y (complex, m x m) go to shared memory in that
    // order while they fit
    const size_t m = a.m;
    const size_t parts[4] = {(m + 1) * m * sizeof(T), m * m * sizeof(T), m * m * sizeof(T), m * m * sizeof(cplx)};
    size_t smem = 0;
    a.smem = 0;
    for (int q = 0; q < 4 && smem + parts[q] <= kGdrSmemMax; ++q) {
        smem += parts[q];
        a.smem = q + 1;
    }
    if (smem > 48 * 1024) {
        // without the raised limit the launch would fail; report the attribute call instead
        const cudaError_t e = smem_attr_once((const void *)k_gmresdr_restart<T>, (int)kGdrSmemMax);
        if (e != cudaSuccess) return e;
    }
    k_gmresdr_restart<T><<<1, kGdrThreads, smem, s>>>(a);
    return cudaGetLastError();
}
template <class T>
size_t gmresdr_restart_smem(int m, int *parts) {
    const size_t mm = m;
    const size_t sizes[4] = {(mm + 1) * mm * sizeof(T), mm * mm * sizeof(T), mm * mm * sizeof(T), mm * mm * sizeof(cplx)};
    size_t smem = 0;
    *parts = 0;
    for (int q = 0; q < 4 && smem + sizes[q] <= kGdrSmemMax; ++q) {
        smem += sizes[q];
        *parts = q + 1;
    }
    return smem;
}
template <class T>
cudaError_t launch_gmresdr_restart_batch(const GdrArgs<T> *args, const int *active, int count, int m, cudaStream_t s) {
    int parts = 0;
    const size_t smem = gmresdr_restart_smem<T>(m, &parts);
    if (smem > 48 * 1024) {
        const cudaError_t e = smem_attr_once((const void *)k_gmresdr_restart_batch<T>, (int)kGdrSmemMax);
        if (e != cudaSuccess) return e;
    }
    k_gmresdr_restart_batch<T><<<count, kGdrThreads, smem, s>>>(args, active);
    return cudaGetLastError();
}
template <class D>
void launch_givens_step(D *H, int ldh, int j, D *cs, D *sn, D *g, GivensState *state, cudaStream_t s) {
    k_givens_step<D><<<1, 1, 0, s>>>(H, ldh, j, cs, sn, g, state);
}
template <class D>
void launch_givens_solve(const D *H, int ldh, const D *g, D *y, const GivensState *state, cudaStream_t s) {
    k_givens_solve<D><<<1, 1, 0, s>>>(H, ldh, g, y, state);
}

#define TG_INST(D)                                                                                   \
    template void launch_chol_inv<D>(const D *, int, D *, D *, int *, cudaStream_t);                 \
    template void launch_inverse<D>(const D *, int, D *, D *, int *, cudaStream_t);                  \
    template void launch_small_gemv<D>(const D *, int, const D *, D *, cudaStream_t);                \
    template cudaError_t launch_gmresdr_restart<D>(const GdrArgs<D> &, cudaStream_t);                \
    template size_t gmresdr_restart_smem<D>(int, int *);                                              \
    template cudaError_t launch_gmresdr_restart_batch<D>(const GdrArgs<D> *, const int *, int, int, cudaStream_t); \
    template void launch_givens_step<D>(D *, int, int, D *, D *, D *, GivensState *, cudaStream_t);  \
    template void launch_givens_solve<D>(const D *, int, const D *, D *, const GivensState *, cudaStream_t);
TG_INST(double)
TG_INST(cplx)
#undef TG_INST

}  // namespace tg
