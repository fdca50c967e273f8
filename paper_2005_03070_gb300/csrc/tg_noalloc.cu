// tg_harmonic_ritz_noalloc: the small dense GMRES-DR restart step (the same kernel as
// tg_harmonic_ritz) with all of its scratch in a fixed device array of this file, so that
// the call allocates no device memory.
//
// Who needs it: callers that own all device memory through their own allocator or a
// fixed pre-reserved pool (a cudaMalloc from inside the library would bypass that pool,
// or fail once the pool holds the memory), and latency-critical loops that cannot take
// the implicit device-wide synchronisation cudaMalloc / cudaFree may cause.
//
// The scratch array (kScratchBytes, enough for m <= 128 in complex arithmetic) is
// reserved on every GPU that loads the library and is held until the process exits.
// In host code the array's name only stands for it; its device address is looked up
// with cudaGetSymbolAddress once per device, on the first call made with that device
// current, and that address is what the kernel receives.
#include <mutex>

#include "tg_small.cuh"

namespace {

constexpr int kNoAllocMaxM = 128;
constexpr size_t kScratchBytes = 2u << 20;     // 2 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_hr_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_dev[kMaxDevices] = {};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves the scratch area into the restart kernel's buffers (base == nullptr: only
// measures).  Returns the bytes used.
template <class T>
size_t carve(char *base, int m, tg::GdrArgs<T> *a, T **c_out) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    const size_t M = (size_t)m;
    *c_out = reinterpret_cast<T *>(take((M + 1) * sizeof(T)));
    a->d = reinterpret_cast<T *>(take((M + 1) * sizeof(T)));
    a->res = reinterpret_cast<T *>(take((M + 1) * sizeof(T)));
    a->z = reinterpret_cast<T *>(take((M + 1) * sizeof(T)));
    a->P = reinterpret_cast<T *>(take((M + 1) * (M + 2) * sizeof(T)));
    a->Hnew = reinterpret_cast<T *>(take((M + 1) * M * sizeof(T)));
    a->cnew = reinterpret_cast<T *>(take((M + 2) * sizeof(T)));
    a->theta = reinterpret_cast<double *>(take(2 * M * sizeof(double)));
    a->wr = reinterpret_cast<double *>(take(M * sizeof(double)));
    a->wi = reinterpret_cast<double *>(take(M * sizeof(double)));
    a->order = reinterpret_cast<int *>(take(M * sizeof(int)));
    a->eres = reinterpret_cast<double *>(take(M * sizeof(double)));
    a->work = reinterpret_cast<T *>(take(((M + 1) * M + 2 * M * M + 3 * M + 4) * sizeof(T)));
    a->ywork = reinterpret_cast<tg::cplx *>(take(M * M * sizeof(tg::cplx)));
    a->gwork = reinterpret_cast<tg::cplx *>(take(M * M * sizeof(tg::cplx)));
    a->info = reinterpret_cast<tg::GdrInfo *>(take(sizeof(tg::GdrInfo)));
    return off;
}

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return tg::cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        tg::set_error("device %d is beyond the %d devices this entry point supports", dev, kMaxDevices);
        return TG_BAD_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_hr_scratch);
        if (e != cudaSuccess) return tg::cuda_status(e, "cudaGetSymbolAddress(g_hr_scratch)");
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return TG_OK;
}

template <class T>
int run(const void *Hbar, int m, int k, void *theta_out, void *basis_out, void *eres_out, int *kk_out,
        cudaStream_t s) {
    tg::GdrArgs<T> a{};
    T *c = nullptr;
    const size_t need = carve<T>(nullptr, m, &a, &c);
    if (need > kScratchBytes) {
        tg::set_error("m = %d needs %zu bytes of scratch, more than the %zu this entry point holds", m, need,
                      kScratchBytes);
        return TG_BAD_ARG;
    }
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != TG_OK) return rc;
    carve<T>(static_cast<char *>(base), m, &a, &c);
    a.H = static_cast<const T *>(Hbar);
    a.ldh = m + 1;
    a.c = c;
    a.m = m;
    a.k = k;
    a.nev = k;
    a.rtolev = 0.0;
    // the array keeps the previous call's contents: the least-squares right-hand side must
    // be e_1 on entry; every other buffer is written by the kernel before it is read
    cudaError_t e = cudaMemsetAsync(c, 0, (size_t)(m + 1) * sizeof(T), s);
    const double one = 1.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c, &one, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return tg::cuda_status(e, "tg_harmonic_ritz_noalloc: clearing the scratch");
    e = tg::launch_gmresdr_restart<T>(a, s);
    if (e != cudaSuccess) return tg::cuda_status(e, "tg_harmonic_ritz_noalloc: launch");
    tg::GdrInfo info;
    e = cudaMemcpyAsync(&info, a.info, sizeof(info), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return tg::cuda_status(e, "tg_harmonic_ritz_noalloc: reading the result");
    *kk_out = info.kk;
    e = cudaMemcpyAsync(theta_out, a.theta, 2 * (size_t)m * sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(basis_out, (size_t)m * sizeof(T), a.P, (size_t)(m + 1) * sizeof(T),
                              (size_t)m * sizeof(T), info.kk, cudaMemcpyDefault, s);
    if (e == cudaSuccess && eres_out)
        e = cudaMemcpyAsync(eres_out, a.eres, (size_t)info.kk * sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return tg::cuda_status(e, "tg_harmonic_ritz_noalloc: copying the outputs");
    return info.status ? TG_NOT_CONVERGED : TG_OK;
}

}  // namespace

extern "C" int tg_harmonic_ritz_noalloc(const void *Hbar, int m, int k, int complex_, void *theta_out,
                                        void *basis_out, void *eres_out, int *kk_out, void *stream) {
    if (!Hbar || !theta_out || !basis_out || !kk_out) {
        tg::set_error("tg_harmonic_ritz_noalloc: NULL argument");
        return TG_BAD_ARG;
    }
    if (m < 2 || m > kNoAllocMaxM || k < 1 || k >= m) {
        tg::set_error("tg_harmonic_ritz_noalloc: need 1 <= k < m <= %d (got m = %d, k = %d)", kNoAllocMaxM, m, k);
        return TG_BAD_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (complex_) return run<tg::cplx>(Hbar, m, k, theta_out, basis_out, eres_out, kk_out, s);
    return run<double>(Hbar, m, k, theta_out, basis_out, eres_out, kk_out, s);
}
