// Operator set-up and grid-transfer kernels of the tg library.
//
//  - variable-coefficient stencil coefficients from node kappa (arithmetic face means), and
//    those of Example 1's operator -exp(gamma x y) Lap u + beta . grad u;
//  - lattice block-transport weights P[x, X] = (1/4) conj(W(x)) and the Galerkin coarse
//    operator P^H A P as a 9-point stencil (Section 5.4's lattice problem; the paper's
//    Schwinger-model coarse operator is not specified, this build uses 2^4 blocking);
//  - bilinear / trilinear and cubic prolongation with a fixed summation order, full-weighting
//    restriction, lattice prolongation / restriction (Section 3, phase 1: moving the
//    coarse eigenvectors and solution to the fine grid);
//  - the kappa-gradient contraction of the adjoint form and precision conversions.
#include "tg_setup.cuh"

namespace tg {

// ----------------------------------------------------------------------------- coefficients
// coef[5][n] for A (sgn = +1) or A^T (sgn = -1): diag, west, east, south, north.
__global__ void k_vark_coefs(const double *__restrict__ kappa, int N, double beta, int sgn,
                             double *__restrict__ coef, float *__restrict__ coef32) {
    const int n = N * N;
    const double h = 1.0 / (N + 1);
    const double s = 0.5 / (h * h);
    const double cb = sgn * beta / (2.0 * h);
    const int NP = N + 2;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int i = idx % N + 1, j = idx / N + 1;
        const double kc = kappa[j * NP + i];
        const double ww = (kc + kappa[j * NP + i - 1]) * s;
        const double we = (kc + kappa[j * NP + i + 1]) * s;
        const double ws = (kc + kappa[(j - 1) * NP + i]) * s;
        const double wn = (kc + kappa[(j + 1) * NP + i]) * s;
        const double c[5] = {ww + we + ws + wn, -ww - cb, -we + cb, -ws, -wn};
        for (int q = 0; q < 5; ++q) {
            coef[(size_t)q * n + idx] = c[q];
            coef32[(size_t)q * n + idx] = (float)c[q];
        }
    }
}

// coef[5][n] of -exp(gamma x y)(u_xx + u_yy) + bx u_x + by u_y + shift u (Example 1's operator
// with gamma = 5, bx = by = 40), centred differences, x = i h, y = j h: for A (transpose = 0)
// the coefficients of u_nb in (A u)(i, j); for A^T (transpose = 1) those of (A^T u)(i, j),
// i.e. A[nb, (i, j)]: the diffusion weight is taken at the neighbour and the convection sign
// flips (A = D_a L + C with L symmetric and C antisymmetric, so A^T = L D_a - C).
__global__ void k_exp2d_coefs(int N, double bx, double by, double gamma, double shift, int transpose,
                              double *__restrict__ coef, float *__restrict__ coef32) {
    const int n = N * N;
    const double h = 1.0 / (N + 1);
    const double ih2 = 1.0 / (h * h);
    const double cx = bx / (2.0 * h), cy = by / (2.0 * h);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int i = idx % N + 1, j = idx / N + 1;
        const double x = i * h, y = j * h;
        const double a = exp(gamma * x * y);
        double c[5];
        c[0] = 4.0 * a * ih2 + shift;
        if (!transpose) {
            c[1] = -a * ih2 - cx;
            c[2] = -a * ih2 + cx;
            c[3] = -a * ih2 - cy;
            c[4] = -a * ih2 + cy;
        } else {
            c[1] = -exp(gamma * (x - h) * y) * ih2 + cx;     // A[(i-1, j), (i, j)]
            c[2] = -exp(gamma * (x + h) * y) * ih2 - cx;     // A[(i+1, j), (i, j)]
            c[3] = -exp(gamma * x * (y - h)) * ih2 + cy;     // A[(i, j-1), (i, j)]
            c[4] = -exp(gamma * x * (y + h)) * ih2 - cy;     // A[(i, j+1), (i, j)]
        }
        for (int q = 0; q < 5; ++q) {
            coef[(size_t)q * n + idx] = c[q];
            coef32[(size_t)q * n + idx] = (float)c[q];
        }
    }
}

// kappa_c(I, J) = kappa(2I, 2J) on the coarse (Nc+2)^2 node grid.
__global__ void k_inject_kappa(const double *__restrict__ kappa, int N, double *__restrict__ kc) {
    const int Nc = (N - 1) / 2;
    const int NPc = Nc + 2, NP = N + 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NPc * NPc; e += gridDim.x * blockDim.x) {
        const int I = e % NPc, J = e / NPc;
        kc[e] = kappa[(2 * J) * NP + 2 * I];
    }
}

// ----------------------------------------------------------------------------- lattice
__device__ __forceinline__ cplx cmul_nofma(cplx a, cplx b) {
    return {__dsub_rn(__dmul_rn(a.re, b.re), __dmul_rn(a.im, b.im)),
            __dadd_rn(__dmul_rn(a.re, b.im), __dmul_rn(a.im, b.re))};
}

// pw[x] = (1/4) conj(W(x)), W(x) the product of links along the path from the block
// corner 2X to x, one step in each mu = 0, 1, 2, 3 with delta_mu = 1.
__global__ void k_lattice_weights(const cplx *__restrict__ links, int L, cplx *__restrict__ pw) {
    const int V = L * L * L * L;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        int c[4] = {x % L, (x / L) % L, (x / (L * L)) % L, x / (L * L * L)};
        int y[4] = {c[0] & ~1, c[1] & ~1, c[2] & ~1, c[3] & ~1};
        cplx W = {1.0, 0.0};
        for (int mu = 0; mu < 4; ++mu) {
            if (c[mu] & 1) {
                const int site = y[0] + L * (y[1] + L * (y[2] + L * y[3]));
                W = cmul_nofma(W, links[(size_t)mu * V + site]);
                y[mu] += 1;
            }
        }
        pw[x] = {0.25 * W.re, -0.25 * W.im};
    }
}

__device__ __forceinline__ int site_of(const int c[4], int L) { return c[0] + L * (c[1] + L * (c[2] + L * c[3])); }

// Galerkin coarse stencil of A = (m+8) I - hops: cst[0][X] = diag, cst[1+mu][X] = A_c[X, X+mu],
// cst[5+mu][X] = A_c[X, X-mu].  Sums over the 16 block sites in order delta = 0..15.
__global__ void k_lattice_coarse(const cplx *__restrict__ links, const cplx *__restrict__ pw, int L,
                                 double mdiag, cplx *__restrict__ cst) {
    const int Lc = L / 2;
    const int V = L * L * L * L, Vc = Lc * Lc * Lc * Lc;
    for (int X = blockIdx.x * blockDim.x + threadIdx.x; X < Vc; X += gridDim.x * blockDim.x) {
        const int C[4] = {X % Lc, (X / Lc) % Lc, (X / (Lc * Lc)) % Lc, X / (Lc * Lc * Lc)};
        cplx diag = {0.0, 0.0};
        cplx fwd[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}}, bwd[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        for (int d = 0; d < 16; ++d) {
            int c[4];
            for (int a = 0; a < 4; ++a) c[a] = 2 * C[a] + ((d >> a) & 1);
            const int x = site_of(c, L);
            const cplx px = pw[x];
            const cplx cpx = conj(px);
            diag = diag + (mdiag * abs2(px)) * cplx{1.0, 0.0};
            for (int mu = 0; mu < 4; ++mu) {
                const int xp = lat_shift(x, L, mu, +1), xm = lat_shift(x, L, mu, -1);
                const cplx uf = links[(size_t)mu * V + x];
                const cplx ub = conj(links[(size_t)mu * V + xm]);
                // A[x, x+mu] = -U_mu(x): x+mu is in this block when delta_mu = 0
                cplx tf = cpx * (-(uf * pw[xp]));
                cplx tb = cpx * (-(ub * pw[xm]));
                if (((d >> mu) & 1) == 0) diag = diag + tf; else fwd[mu] = fwd[mu] + tf;
                if (((d >> mu) & 1) == 1) diag = diag + tb; else bwd[mu] = bwd[mu] + tb;
            }
        }
        cst[X] = diag;
        for (int mu = 0; mu < 4; ++mu) {
            cst[(size_t)(1 + mu) * Vc + X] = fwd[mu];
            cst[(size_t)(5 + mu) * Vc + X] = bwd[mu];
        }
    }
}

// ----------------------------------------------------------------------------- transfer
__device__ __forceinline__ double cval2(const double *uc, int Nc, int I, int J) {
    return (I >= 1 && I <= Nc && J >= 1 && J <= Nc) ? uc[(J - 1) * Nc + (I - 1)] : 0.0;
}

// Bilinear prolongation of one column (fine 1-based (i, j); coarse I, J).
__global__ void k_prolong2d(const double *__restrict__ uc, int Nc, double *__restrict__ uf) {
    const int N = 2 * Nc + 1;
    const int n = N * N;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int i = idx % N + 1, j = idx / N + 1;
        const int I = i >> 1, J = j >> 1;
        const int px = i & 1, py = j & 1;
        double v;
        if (!px && !py) v = cval2(uc, Nc, I, J);
        else if (px && !py) v = 0.5 * (cval2(uc, Nc, I, J) + cval2(uc, Nc, I + 1, J));
        else if (!px && py) v = 0.5 * (cval2(uc, Nc, I, J) + cval2(uc, Nc, I, J + 1));
        else v = 0.25 * ((cval2(uc, Nc, I, J) + cval2(uc, Nc, I + 1, J)) +
                         (cval2(uc, Nc, I, J + 1) + cval2(uc, Nc, I + 1, J + 1)));
        uf[idx] = v;
    }
}

__device__ __forceinline__ double cval3(const double *uc, int Nc, int I, int J, int K) {
    return (I >= 1 && I <= Nc && J >= 1 && J <= Nc && K >= 1 && K <= Nc)
               ? uc[(I - 1) + (size_t)Nc * ((J - 1) + (size_t)Nc * (K - 1))]
               : 0.0;
}

// Trilinear prolongation: pairs along x, then y, then z; weight 2^-(px+py+pz) last.
__global__ void k_prolong3d(const double *__restrict__ uc, int Nc, double *__restrict__ uf) {
    const int N = 2 * Nc + 1;
    const int n = N * N * N;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int i = idx % N + 1, j = (idx / N) % N + 1, k = idx / (N * N) + 1;
        const int I = i >> 1, J = j >> 1, K = k >> 1;
        const int px = i & 1, py = j & 1, pz = k & 1;
        double ys[2];
        for (int dz = 0; dz <= pz; ++dz) {
            double xs[2];
            for (int dy = 0; dy <= py; ++dy) {
                double a = cval3(uc, Nc, I, J + dy, K + dz);
                xs[dy] = px ? a + cval3(uc, Nc, I + 1, J + dy, K + dz) : a;
            }
            ys[dz] = py ? xs[0] + xs[1] : xs[0];
        }
        double tot = pz ? ys[0] + ys[1] : ys[0];
        const double w = (px + py + pz == 0) ? 1.0 : (px + py + pz == 1) ? 0.5 : (px + py + pz == 2) ? 0.25 : 0.125;
        uf[idx] = w * tot;
    }
}

// ----------------------------------------------------------------------------- cubic prolongation
// Fourth-order interpolation in place of the paper's splines (Section 3, phase 1): a fine
// point halfway between coarse nodes a and a + 1 takes (-1, 9, 9, -1)/16 of nodes a-1..a+2,
// a fine point on a coarse node copies it; beyond the Dirichlet boundary the function is
// continued oddly (nodes 0 and Nc+1 are zero, node -1 is -u(1), node Nc+2 is -u(Nc)).
// Tensor product over x, then y, then z; each sum ((w0 v0 + w1 v1) + w2 v2) + w3 v3 uses
// separately rounded products and sums (no contraction), so the result is reproducible.
struct CubAxis {
    int cnt;         // 1 (on a coarse node) or 4
    int node[4];     // coarse nodes, 1..Nc after folding (0 when the term is a boundary zero)
    double sgn[4];   // +1, or -1 for a reflected node
};

__device__ __forceinline__ CubAxis cub_axis(int i, int Nc) {
    CubAxis c;
    if (!(i & 1)) {
        c.cnt = 1;
        c.node[0] = i >> 1;
        c.sgn[0] = 1.0;
        return c;
    }
    c.cnt = 4;
    const int a = (i - 1) >> 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int nd = a - 1 + q;
        if (nd == -1) { c.node[q] = 1; c.sgn[q] = -1.0; }
        else if (nd == Nc + 2) { c.node[q] = Nc; c.sgn[q] = -1.0; }
        else if (nd < 1 || nd > Nc) { c.node[q] = 0; c.sgn[q] = 0.0; }
        else { c.node[q] = nd; c.sgn[q] = 1.0; }
    }
    return c;
}

__device__ __forceinline__ double cub_sum(const double (&v)[4]) {
    constexpr double w0 = -0.0625, w1 = 0.5625;
    return __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(w0, v[0]), __dmul_rn(w1, v[1])), __dmul_rn(w1, v[2])),
                     __dmul_rn(w0, v[3]));
}

// value of a reflected term: sgn * u (exact), or the boundary zero
__device__ __forceinline__ double cub_term(double sgn, double u) { return sgn == 0.0 ? 0.0 : (sgn < 0.0 ? -u : u); }

__global__ void k_prolong2d_cubic(const double *__restrict__ uc, int Nc, double *__restrict__ uf) {
    const int N = 2 * Nc + 1;
    const int n = N * N;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int i = idx % N + 1, j = idx / N + 1;
        const CubAxis ax = cub_axis(i, Nc), ay = cub_axis(j, Nc);
        double t[4];
        for (int b = 0; b < ay.cnt; ++b) {
            // the x-interpolated row ay.node[b] (a zero row at the boundary)
            double xv;
            if (ay.sgn[b] == 0.0) {
                xv = 0.0;
            } else {
                const double *row = uc + (size_t)(ay.node[b] - 1) * Nc;
                if (ax.cnt == 1) {
                    xv = row[ax.node[0] - 1];
                } else {
                    double v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = ax.sgn[q] == 0.0 ? 0.0 : cub_term(ax.sgn[q], row[ax.node[q] - 1]);
                    xv = cub_sum(v);
                }
            }
            t[b] = cub_term(ay.sgn[b], xv);
        }
        uf[idx] = ay.cnt == 1 ? t[0] : cub_sum(t);
    }
}

__global__ void k_prolong3d_cubic(const double *__restrict__ uc, int Nc, double *__restrict__ uf) {
    const int N = 2 * Nc + 1;
    const int64_t n = (int64_t)N * N * N;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % N) + 1, j = (int)((idx / N) % N) + 1, k = (int)(idx / ((int64_t)N * N)) + 1;
        const CubAxis ax = cub_axis(i, Nc), ay = cub_axis(j, Nc), az = cub_axis(k, Nc);
        double tz[4];
        for (int c = 0; c < az.cnt; ++c) {
            double ty[4];
            for (int b = 0; b < ay.cnt; ++b) {
                double xv;
                if (az.sgn[c] == 0.0 || ay.sgn[b] == 0.0) {
                    xv = 0.0;
                } else {
                    const double *row = uc + (size_t)Nc * ((ay.node[b] - 1) + (size_t)Nc * (az.node[c] - 1));
                    if (ax.cnt == 1) {
                        xv = row[ax.node[0] - 1];
                    } else {
                        double v[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[q] = ax.sgn[q] == 0.0 ? 0.0 : cub_term(ax.sgn[q], row[ax.node[q] - 1]);
                        xv = cub_sum(v);
                    }
                }
                ty[b] = cub_term(ay.sgn[b], xv);
            }
            const double yv = ay.cnt == 1 ? ty[0] : cub_sum(ty);
            tz[c] = cub_term(az.sgn[c], yv);
        }
        uf[idx] = az.cnt == 1 ? tz[0] : cub_sum(tz);
    }
}

// Full weighting: uc(I, J) = (1/4) sum_f P[f, (I,J)] uf(f) (weights 1, 1/2, 1/4).
__global__ void k_restrict2d(const double *__restrict__ uf, int N, double *__restrict__ uc) {
    const int Nc = (N - 1) / 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Nc * Nc; e += gridDim.x * blockDim.x) {
        const int I = e % Nc + 1, J = e / Nc + 1;
        double s = 0.0;
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj;
                const double w = (di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0);
                s += w * uf[(j - 1) * N + (i - 1)];
            }
        uc[e] = 0.25 * s;
    }
}

__global__ void k_restrict3d(const double *__restrict__ uf, int N, double *__restrict__ uc) {
    const int Nc = (N - 1) / 2;
    const int nc = Nc * Nc * Nc;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc; e += gridDim.x * blockDim.x) {
        const int I = e % Nc + 1, J = (e / Nc) % Nc + 1, K = e / (Nc * Nc) + 1;
        double s = 0.0;
        for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
                    const double w = (di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0);
                    s += w * uf[(i - 1) + (size_t)N * ((j - 1) + (size_t)N * (k - 1))];
                }
        uc[e] = 0.125 * s;
    }
}

__global__ void k_prolong_lattice(const cplx *__restrict__ uc, const cplx *__restrict__ pw, int L,
                                  cplx *__restrict__ uf) {
    const int V = L * L * L * L, Lc = L / 2;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) {
        const int c0 = x % L, c1 = (x / L) % L, c2 = (x / (L * L)) % L, c3 = x / (L * L * L);
        const int X = (c0 >> 1) + Lc * ((c1 >> 1) + Lc * ((c2 >> 1) + Lc * (c3 >> 1)));
        uf[x] = cmul_nofma(pw[x], uc[X]);
    }
}

__global__ void k_restrict_lattice(const cplx *__restrict__ uf, const cplx *__restrict__ pw, int L,
                                   cplx *__restrict__ uc) {
    const int Lc = L / 2, Vc = Lc * Lc * Lc * Lc;
    for (int X = blockIdx.x * blockDim.x + threadIdx.x; X < Vc; X += gridDim.x * blockDim.x) {
        const int C[4] = {X % Lc, (X / Lc) % Lc, (X / (Lc * Lc)) % Lc, X / (Lc * Lc * Lc)};
        cplx s = {0.0, 0.0};
        for (int d = 0; d < 16; ++d) {
            int c[4];
            for (int a = 0; a < 4; ++a) c[a] = 2 * C[a] + ((d >> a) & 1);
            const int x = site_of(c, L);
            s = s + cmul_nofma(conj(pw[x]), uf[x]);
        }
        uc[X] = s;
    }
}

// ----------------------------------------------------------------------------- adjoint gradient
// dkappa_p = -1/2 sum_{faces (p, q)} (lam_p - lam_q)(x_p - x_q) / h^2 over the (N+2)^2 nodes
// (lam = x = 0 on boundary nodes; faces with both nodes on the boundary contribute 0).
__global__ void k_kappa_grad(const double *__restrict__ x, const double *__restrict__ lam, int N,
                             double *__restrict__ g) {
    const int NP = N + 2;
    const double h = 1.0 / (N + 1);
    const double s = -0.5 / (h * h);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NP * NP; e += gridDim.x * blockDim.x) {
        const int i = e % NP, j = e / NP;
        auto val = [&](const double *v, int ii, int jj) -> double {
            return (ii >= 1 && ii <= N && jj >= 1 && jj <= N) ? v[(jj - 1) * N + (ii - 1)] : 0.0;
        };
        const double lp = val(lam, i, j), xp = val(x, i, j);
        double acc = 0.0;
        const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
        for (int q = 0; q < 4; ++q) {
            const int ii = i + di[q], jj = j + dj[q];
            if (ii < 0 || ii > N + 1 || jj < 0 || jj > N + 1) continue;
            acc += (lp - val(lam, ii, jj)) * (xp - val(x, ii, jj));
        }
        g[e] = s * acc;
    }
}

__global__ void k_inv_sqrt(const double *in, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = in[0] > 0 ? 1.0 / sqrt(in[0]) : 0.0;
}

// ----------------------------------------------------------------------------- conversions
__global__ void k_d2f_scaled(const double *__restrict__ a, float *__restrict__ b, int n, double s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (float)(a[i] * s);
}
__global__ void k_add_f2d_scaled(double *__restrict__ x, const float *__restrict__ e, int n, double s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = fma(s, (double)e[i], x[i]);
}
__global__ void k_d2f(const double *__restrict__ a, float *__restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ----------------------------------------------------------------------------- launchers
#define TG_L(name, params, args) \
    void launch_##name params { k_##name<<<grid, kThreads, 0, s>>> args; }
TG_L(vark_coefs, (int grid, cudaStream_t s, const double *kappa, int N, double beta, int sgn, double *coef, float *coef32),
     (kappa, N, beta, sgn, coef, coef32))
TG_L(exp2d_coefs, (int grid, cudaStream_t s, int N, double bx, double by, double gamma, double shift, int transpose,
                   double *coef, float *coef32), (N, bx, by, gamma, shift, transpose, coef, coef32))
TG_L(inject_kappa, (int grid, cudaStream_t s, const double *kappa, int N, double *kc), (kappa, N, kc))
TG_L(lattice_weights, (int grid, cudaStream_t s, const cplx *links, int L, cplx *pw), (links, L, pw))
TG_L(lattice_coarse, (int grid, cudaStream_t s, const cplx *links, const cplx *pw, int L, double mdiag, cplx *cst),
     (links, pw, L, mdiag, cst))
TG_L(prolong2d, (int grid, cudaStream_t s, const double *uc, int Nc, double *uf), (uc, Nc, uf))
TG_L(prolong3d, (int grid, cudaStream_t s, const double *uc, int Nc, double *uf), (uc, Nc, uf))
TG_L(prolong2d_cubic, (int grid, cudaStream_t s, const double *uc, int Nc, double *uf), (uc, Nc, uf))
TG_L(prolong3d_cubic, (int grid, cudaStream_t s, const double *uc, int Nc, double *uf), (uc, Nc, uf))
TG_L(restrict2d, (int grid, cudaStream_t s, const double *uf, int N, double *uc), (uf, N, uc))
TG_L(restrict3d, (int grid, cudaStream_t s, const double *uf, int N, double *uc), (uf, N, uc))
TG_L(prolong_lattice, (int grid, cudaStream_t s, const cplx *uc, const cplx *pw, int L, cplx *uf), (uc, pw, L, uf))
TG_L(restrict_lattice, (int grid, cudaStream_t s, const cplx *uf, const cplx *pw, int L, cplx *uc), (uf, pw, L, uc))
TG_L(kappa_grad, (int grid, cudaStream_t s, const double *x, const double *lam, int N, double *g), (x, lam, N, g))
TG_L(d2f_scaled, (int grid, cudaStream_t s, const double *a, float *b, int n, double sc), (a, b, n, sc))
TG_L(add_f2d_scaled, (int grid, cudaStream_t s, double *x, const float *e, int n, double sc), (x, e, n, sc))
TG_L(d2f, (int grid, cudaStream_t s, const double *a, float *b, size_t n), (a, b, n))
#undef TG_L
void launch_inv_sqrt(cudaStream_t s, const double *in, double *out) { k_inv_sqrt<<<1, 1, 0, s>>>(in, out); }

}  // namespace tg
