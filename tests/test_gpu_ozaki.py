"""FP64 complex GEMM emulated on the BF16 tensor cores (tdvp_zgemm_ozaki) against the definition.

The reference is the plain complex128 product A @ B on the host (numpy).  The bound is the one
the header states: |C - A B| <= 2k (s + 3) 2^(-7s) 2^(eR + fc) + 2^-47 * 2k 2^(eR + fc) per
element, with 2^eR, 2^fc the powers of two just above the largest magnitude (real or imaginary
part) of row R of A and column c of B, computed here with numpy's frexp.  Integer inputs within
one 7-bit slice per row scale are exact with one slice (bit-exact comparison).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402


def _ozaki(A, B, slices, reps=1):
    m, k = A.shape
    n = B.shape[1]
    dev = torch.device("cuda")
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    Bd = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    Cd = torch.full((m, n), np.nan + 0j, dtype=torch.complex128, device=dev)
    wsb = pkg.zgemm_ozaki_workspace(m, n, k, slices)
    assert wsb > 0
    ws = torch.empty(wsb // 8 + 128, dtype=torch.float64, device=dev)
    wp = (ws.data_ptr() + 1023) // 1024 * 1024
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(reps):
        pkg.zgemm_ozaki(m, n, k, Ad.data_ptr(), Bd.data_ptr(), Cd.data_ptr(), slices, wp, wsb, stream)
        pkg.zgemm_ozaki_status(wp, stream)
        outs.append(Cd.cpu().numpy().copy())
    return outs


def _bound(A, B, s):
    k = A.shape[1]
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
    cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=0)
    eR = np.where(ra > 0, np.frexp(ra)[1], -1074)
    fc = np.where(cb > 0, np.frexp(cb)[1], -1074)
    scale = np.ldexp(1.0, eR[:, None] + fc[None, :])
    return 2 * k * ((s + 3) * 2.0 ** (-7 * s) + 2.0 ** -47) * scale


def _rand(rng, m, k, n):
    A = rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k))
    B = rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n))
    return A, B


@pytest.mark.parametrize("m,n,k", [(100, 70, 45), (256, 64, 1000), (130, 65, 33), (1, 1, 1), (640, 64, 64)])
@pytest.mark.parametrize("slices", [4, 6, 8])
def test_ozaki_zgemm_within_its_bound(m, n, k, slices):
    rng = np.random.default_rng(m * 7 + n * 3 + k + slices)
    A, B = _rand(rng, m, k, n)
    C = _ozaki(A, B, slices)[0]
    err = np.abs(C - A @ B)
    ratio = float((err / _bound(A, B, slices)).max())
    print(f"{m}x{n}x{k} slices {slices}: max err / bound {ratio:.2e}, "
          f"max rel {err.max() / np.abs(A @ B).max():.1e}")
    assert np.all(np.isfinite(C)) and ratio <= 1.0


def test_ozaki_zgemm_with_graded_rows_and_columns():
    """Rows and columns over 30 decades: each is scaled on its own, so small rows keep their
    relative accuracy."""
    rng = np.random.default_rng(5)
    A, B = _rand(rng, 300, 200, 90)
    A *= np.logspace(-15, 15, 300)[:, None]
    B *= np.logspace(10, -10, 90)[None, :]
    C = _ozaki(A, B, 8)[0]
    assert float((np.abs(C - A @ B) / _bound(A, B, 8)).max()) <= 1.0


def test_ozaki_zgemm_is_exact_on_small_integers_with_one_slice():
    rng = np.random.default_rng(6)
    A = rng.integers(-100, 101, size=(150, 77)) + 1j * rng.integers(-100, 101, size=(150, 77))
    B = rng.integers(-100, 101, size=(77, 66)) + 1j * rng.integers(-100, 101, size=(77, 66))
    C = _ozaki(A, B, 1)[0]
    ref = (A.real.astype(np.int64) @ B.real.astype(np.int64) - A.imag.astype(np.int64) @ B.imag.astype(np.int64)
           + 1j * (A.real.astype(np.int64) @ B.imag.astype(np.int64) + A.imag.astype(np.int64) @ B.real.astype(np.int64)))
    assert np.array_equal(C, ref)


def test_ozaki_zgemm_zero_rows_columns_and_repeat_calls():
    rng = np.random.default_rng(7)
    A, B = _rand(rng, 200, 100, 70)
    A[3] = 0
    B[:, 9] = 0
    outs = _ozaki(A, B, 8, reps=2)
    assert np.array_equal(outs[0], outs[1])
    assert np.all(outs[0][3] == 0) and np.all(outs[0][:, 9] == 0)
    assert float((np.abs(outs[0] - A @ B) / np.maximum(_bound(A, B, 8), 1e-300)).max()) <= 1.0
    Z = _ozaki(np.zeros((40, 30), complex), B[:30, :50], 8)[0]
    assert np.all(Z == 0)
