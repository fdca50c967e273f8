// Declarations of the single-CTA float64 small dense kernels (tg_small.cu).
#pragma once

#include "tg_common.cuh"

namespace tg {

constexpr int kSmallThreads = 256;
constexpr int kGdrThreads = 128;                 // GMRES-DR restart kernel block
constexpr size_t kGdrSmemMax = 210 * 1024;       // shared memory for W and Z when they fit

struct GdrInfo {
    double rnorm;   // ||c - Hbar d||
    int nconv;      // kept pairs (first nev) with residual <= rtolev |theta|
    int kk;         // kept pairs (k or k+1)
    int status;     // 0, or 1 if the QR iteration did not converge
    int pad;
    long long phase[8];   // SM cycles spent in each phase (instrumentation)
};

// Arguments of the GMRES-DR restart kernel (all pointers device memory).
template <class T>
struct GdrArgs {
    const T *H;      // Hbar, (m+1) x m, leading dimension ldh
    int ldh;
    const T *c;      // least-squares right-hand side, m+1
    int m, k, nev;
    double rtolev;
    T *d;            // out: least-squares solution, m
    T *res;          // out: c - Hbar d, m+1
    T *z;            // out: restart direction [-|h|^2 f; h], m+1
    double *theta;   // out: 2m doubles, harmonic Ritz values (re, im) in selection order
    double *wr, *wi; // scratch: m each
    int *order;      // scratch: m
    double *eres;    // out: residual norms of the kept pairs (up to m)
    T *P;            // out: P_{k+1}, (m+1) x (kk+1), ld m+1; its first kk columns (m rows) are P_k
    T *Hnew;         // out: P_{k+1}^H Hbar P_k, (kk+1) x kk, leading dimension ldh
    T *cnew;         // out: P_{k+1}^H res, kk+1
    T *work;         // scratch: (m+1) m + 2 m^2 + 3 m + 2 elements of T
    cplx *ywork;     // scratch: m * m complex
    cplx *gwork;     // scratch: m * m complex
    GdrInfo *info;
    int smem;        // set by the launcher: W and Z in shared memory
    // Rayleigh-Ritz mode (mode = 1, the Arnoldi-E improvement): H is a dense m x m matrix
    // Q^H A Q (ld ldh) of an orthonormal Q; the least-squares solve, the harmonic
    // modification and the restart matrices are skipped; the Ritz pairs of H are ordered and
    // selected as above, P gets the orthonormal m x kk basis of the kept span, eres the
    // residuals ||A Q g - theta Q g|| = sqrt(g^H WW g - |theta|^2) (WW = (A Q)^H A Q, ld m,
    // ||g|| = 1), and z the coefficients of Ritz vector start_q (phase fixed so that its
    // largest entry is real and positive; real problems keep the real part).
    int mode = 0;
    const T *WW = nullptr;
    int start_q = 0;
};

struct GivensState {
    double target;  // stop when |g[j+1]| <= target
    double resid;
    int steps;      // columns processed
    int done;
};

// Host launchers (one block of kSmallThreads threads each, queued on stream s).
template <class D> void launch_chol_inv(const D *G, int k, D *R, D *Rinv, int *info, cudaStream_t s);
template <class D> void launch_inverse(const D *H, int k, D *Hinv, D *W, int *info, cudaStream_t s);
template <class D> void launch_small_gemv(const D *M, int k, const D *c, D *out, cudaStream_t s);
// Returns the error of raising the kernel's shared-memory limit (nothing is launched then)
// or of the launch itself.
template <class T> cudaError_t launch_gmresdr_restart(const GdrArgs<T> &a, cudaStream_t s);
// The dynamic shared memory of the restart kernel for subspace size m, and how many of its
// work matrices it holds (the rest live in the global scratch); a.smem must be set to that
// count in every entry of a batched launch.
template <class T> size_t gmresdr_restart_smem(int m, int *parts);
// count independent restart steps of size m in one launch (one block each; args and active
// in device memory).
template <class T>
cudaError_t launch_gmresdr_restart_batch(const GdrArgs<T> *args, const int *active, int count, int m, cudaStream_t s);
template <class D>
void launch_givens_step(D *H, int ldh, int j, D *cs, D *sn, D *g, GivensState *state, cudaStream_t s);
template <class D>
void launch_givens_solve(const D *H, int ldh, const D *g, D *y, const GivensState *state, cudaStream_t s);

}  // namespace tg
