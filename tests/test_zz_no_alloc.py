"""tg_harmonic_ritz_noalloc: the GMRES-DR restart step for callers that cannot allocate
device memory (they own every byte through their own allocator or a fixed pool, or run
latency-critical loops that cannot take cudaMalloc's synchronisation).  Its scratch is a
fixed device array of the library.  Checked through the C ABI against the allocating
entry point tg_harmonic_ritz, on two calls in a row (the second must not see the first
call's leftovers), within the tolerances the harmonic-Ritz tests use.  Kept in a file that
pytest collects last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_03070_gb300 import build, tg
    build.build()
    return tg.load()


def _hessenberg(m, seed, complex_):
    rng = np.random.default_rng([seed, 77])
    H = rng.standard_normal((m + 1, m))
    if complex_:
        H = H + 1j * rng.standard_normal((m + 1, m))
    for c in range(m):
        H[c + 2:, c] = 0.0
    H[:m, :m] += 3.0 * np.eye(m)
    return H


def _call(lib, name, H, m, k, complex_):
    dt = torch.complex128 if complex_ else torch.float64
    Hd = torch.from_numpy(np.ascontiguousarray(H.T)).cuda()          # column-major (m+1) x m
    theta = torch.empty(2 * m, dtype=torch.float64, device="cuda")
    basis = torch.empty(m * m, dtype=dt, device="cuda")
    eres = torch.empty(m, dtype=torch.float64, device="cuda")
    kk = C.c_int()
    st = getattr(lib, name)(C.c_void_p(Hd.data_ptr()), m, k, int(complex_), C.c_void_p(theta.data_ptr()),
                            C.c_void_p(basis.data_ptr()), C.c_void_p(eres.data_ptr()), C.byref(kk),
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.tg_last_error()
    torch.cuda.synchronize()
    n = kk.value
    return theta.cpu().numpy().reshape(m, 2), basis[: n * m].cpu().numpy().reshape(n, m).T, eres[:n].cpu().numpy()


def _span_gap(A, B):
    Qa = np.linalg.qr(A)[0]
    Qb = np.linalg.qr(B)[0]
    return np.linalg.norm(Qb - Qa @ (Qa.conj().T @ Qb), 2)


def test_noalloc_matches_the_allocating_entry_point_on_two_calls(lib):
    # two calls in a row on different problems (a larger one first, then a smaller one)
    for (m, k, seed, cplx) in [(60, 30, 1, False), (24, 9, 2, False), (40, 12, 3, True)]:
        H = _hessenberg(m, seed, cplx)
        th_a, b_a, e_a = _call(lib, "tg_harmonic_ritz", H, m, k, cplx)
        th_b, b_b, e_b = _call(lib, "tg_harmonic_ritz_noalloc", H, m, k, cplx)
        z_a = th_a[:, 0] + 1j * th_a[:, 1]
        z_b = th_b[:, 0] + 1j * th_b[:, 1]
        assert np.max(np.abs(z_a - z_b) / np.abs(z_a)) <= 1e-10
        assert b_a.shape == b_b.shape
        assert _span_gap(b_a, b_b) <= 1e-8
        assert np.allclose(e_a, e_b, rtol=1e-10, atol=1e-14)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    H = torch.zeros((130, 129), dtype=torch.float64, device="cuda")
    theta = torch.empty(2 * 129, dtype=torch.float64, device="cuda")
    basis = torch.empty(129 * 129, dtype=torch.float64, device="cuda")
    kk = C.c_int()
    st = lib.tg_harmonic_ritz_noalloc(C.c_void_p(H.data_ptr()), 129, 10, 0, C.c_void_p(theta.data_ptr()),
                                      C.c_void_p(basis.data_ptr()), None, C.byref(kk), None)
    assert st == 4
    assert b"m <= 128" in lib.tg_last_error()


@pytest.mark.parametrize("cplx", [True, False])
def test_noalloc_at_its_size_limit(lib, cplx):
    """m = 128, the largest size the fixed array is carved for (complex arithmetic needs the
    most of it), against the allocating entry point, twice in a row."""
    m, k = 128, 40
    for seed in (4, 5):
        H = _hessenberg(m, seed, cplx)
        th_a, b_a, e_a = _call(lib, "tg_harmonic_ritz", H, m, k, cplx)
        th_b, b_b, e_b = _call(lib, "tg_harmonic_ritz_noalloc", H, m, k, cplx)
        z_a = th_a[:, 0] + 1j * th_a[:, 1]
        z_b = th_b[:, 0] + 1j * th_b[:, 1]
        assert np.max(np.abs(z_a - z_b) / np.abs(z_a)) <= 1e-10
        assert b_a.shape == b_b.shape
        assert _span_gap(b_a, b_b) <= 1e-8
        assert np.allclose(e_a, e_b, rtol=1e-10, atol=1e-14)
