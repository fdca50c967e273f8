// Host launchers of the set-up and transfer kernels (tg_setup.cu); `grid` blocks of
// kThreads threads on stream s.
#pragma once

#include "tg_common.cuh"

namespace tg {

void launch_vark_coefs(int grid, cudaStream_t s, const double *kappa, int N, double beta, int sgn, double *coef,
                       float *coef32);
void launch_exp2d_coefs(int grid, cudaStream_t s, int N, double bx, double by, double gamma, double shift,
                        int transpose, double *coef, float *coef32);
void launch_inject_kappa(int grid, cudaStream_t s, const double *kappa, int N, double *kc);
void launch_lattice_weights(int grid, cudaStream_t s, const cplx *links, int L, cplx *pw);
void launch_lattice_coarse(int grid, cudaStream_t s, const cplx *links, const cplx *pw, int L, double mdiag, cplx *cst);
void launch_prolong2d(int grid, cudaStream_t s, const double *uc, int Nc, double *uf);
void launch_prolong3d(int grid, cudaStream_t s, const double *uc, int Nc, double *uf);
void launch_prolong2d_cubic(int grid, cudaStream_t s, const double *uc, int Nc, double *uf);
void launch_prolong3d_cubic(int grid, cudaStream_t s, const double *uc, int Nc, double *uf);
void launch_restrict2d(int grid, cudaStream_t s, const double *uf, int N, double *uc);
void launch_restrict3d(int grid, cudaStream_t s, const double *uf, int N, double *uc);
void launch_prolong_lattice(int grid, cudaStream_t s, const cplx *uc, const cplx *pw, int L, cplx *uf);
void launch_restrict_lattice(int grid, cudaStream_t s, const cplx *uf, const cplx *pw, int L, cplx *uc);
void launch_kappa_grad(int grid, cudaStream_t s, const double *x, const double *lam, int N, double *g);
void launch_d2f_scaled(int grid, cudaStream_t s, const double *a, float *b, int n, double sc);
void launch_add_f2d_scaled(int grid, cudaStream_t s, double *x, const float *e, int n, double sc);
void launch_d2f(int grid, cudaStream_t s, const double *a, float *b, size_t n);
void launch_inv_sqrt(cudaStream_t s, const double *in, double *out);

}  // namespace tg
