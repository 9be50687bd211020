"""tdvp_lq_noalloc: the gauge shift for callers that must not allocate device memory.

Such callers (a framework that owns all device memory through its own pool, or a path that
cannot afford cudaMalloc's implicit synchronisation) pass their own input and output buffers;
the library keeps its scratch in a fixed static device array.  This file is collected last so
that a stop-at-first-failure run has already run every other test.  Two calls in a row are
checked against the library's allocating gauge-shift entry point, with the same tolerance as
the other QR parity tests.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1907_12044_b300 as pkg  # noqa: E402
from oracle import lq_rr  # noqa: E402


def _noalloc(X):
    n, m = X.shape
    xd = torch.from_numpy(np.ascontiguousarray(X).view(np.float64).copy()).cuda()
    qd = torch.zeros(n * m * 2, dtype=torch.float64, device="cuda")
    ld = torch.zeros(n * n * 2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pkg.lq_noalloc(n, m, xd.data_ptr(), qd.data_ptr(), ld.data_ptr(), stream)
    Q = qd.cpu().numpy().view(np.complex128).reshape(n, m)
    L = ld.cpu().numpy().view(np.complex128).reshape(n, n)
    return Q, L


def _reference(eng, X):
    # the allocating entry point computes C = Q R on columns; X = L Q is its transpose
    Qc, Rc = eng.debug_qr(X.T)
    return Qc.T, Rc.T


def test_noalloc_lq_matches_allocating_gauge_shift_twice_in_a_row():
    p = wl.fmo_sized()
    eng = pkg.Engine()
    eng.build_mpo(0, p)
    eng.init_mps(0, 64, p.exciton_site)        # work buffers large enough for 64 x 640
    rng = np.random.default_rng(77)
    full = rng.normal(size=(64, 640)) + 1j * rng.normal(size=(64, 640))
    deficient = (rng.normal(size=(20, 4)) + 1j * rng.normal(size=(20, 4))) @ rng.normal(size=(4, 100))
    for X in (full, deficient):
        Q, L = _noalloc(X)
        Qr, Lr = _reference(eng, X)
        assert np.abs(Q - Qr).max() < 1e-12
        assert np.abs(L - Lr).max() < 1e-11 * max(1.0, np.abs(Lr).max())
        assert np.abs(Q @ Q.conj().T - np.eye(X.shape[0])).max() < 1e-12


def _rank_deficient_in_later_block(rng, n=256, m=16384, rank=250, support=260):
    """Rank-250 rows supported on the first 260 columns: the 250 kept rows span almost all of
    those columns (distance of each e_p far below 1/2), so the completions of the 6 dropped rows
    are e_260..e_265, which lie in the second column slab of the kernel's blocks."""
    G = rng.normal(size=(n, rank)) + 1j * rng.normal(size=(n, rank))
    H = np.zeros((rank, m), dtype=complex)
    H[:, :support] = rng.normal(size=(rank, support)) + 1j * rng.normal(size=(rank, support))
    return G @ H


def test_noalloc_lq_at_its_largest_sizes_matches_the_oracle_twice():
    """n = 256 rows over m = 16384 columns (the documented limits; the block count is clamped
    to the kernel's maximum): full rank, and rank deficient with the completion columns in a
    block other than the first, against the oracle's gauge shift, each called twice in a row."""
    rng = np.random.default_rng(256)
    full = rng.normal(size=(256, 16384)) + 1j * rng.normal(size=(256, 16384))
    deficient = _rank_deficient_in_later_block(rng)
    for X in (full, deficient):
        Lo, Qo = lq_rr(X)
        for _ in range(2):
            Q, L = _noalloc(X)
            assert np.abs(Q - Qo).max() < 1e-12
            assert np.abs(L - Lo).max() < 1e-11 * np.abs(Lo).max()
            assert np.abs(Q @ Q.conj().T - np.eye(256)).max() < 1e-12
    kept = np.abs(np.diag(Lo)) > 0
    assert kept.sum() == 250
    comp = [int(np.argmax(np.abs(Qo[j]))) for j in np.nonzero(~kept)[0]]
    assert min(comp) >= 256                       # completions outside block 0's slab


def test_noalloc_rejects_sizes_beyond_its_limits():
    with pytest.raises(pkg.TDVPError) as e:
        pkg.lq_noalloc(257, 300, 1, 1, 1, 0)
    assert e.value.code == -1
    with pytest.raises(pkg.TDVPError) as e:
        pkg.lq_noalloc(8, 16385, 1, 1, 1, 0)
    assert e.value.code == -1
