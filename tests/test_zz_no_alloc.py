"""GPU test of otm_syev_noalloc, the entry point that takes its scratch from a
fixed array inside the library instead of a caller workspace.

Two calls in a row (different sizes, so the second one runs on scratch that
still holds the first one's bytes) are each compared with otm_syev on the same
matrix, within the eigensolver tests' tolerances.  Collected last so that it
also runs after every other test in the same process.
"""
import numpy as np
import pytest

import synth
from tests._util import to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _matrix(seed, n):
    """Symmetric matrix with well-separated eigenvalues (gaps >= 1/n of the
    spread), so eigenvectors are unique up to the sign the library fixes."""
    Qm = synth.haar_orthonormal(seed, n).astype(np.float64)
    lam = np.linspace(3.0, -1.0, n) + 0.1 * np.random.default_rng(seed).random(n) / n
    return (Qm * lam) @ Qm.T


def test_syev_noalloc_matches_syev_two_calls():
    from paper_1309_0787_gb300 import otm
    for seed, n in ((5, 160), (6, 37)):
        A = torch.as_tensor(_matrix(seed, n)).cuda()
        ev_ref, vec_ref = otm.syev(A)
        ev = torch.empty(n, dtype=torch.float64, device="cuda")
        vec = torch.empty(n, n, dtype=torch.float64, device="cuda")
        otm.syev_noalloc(A, ev, vec)
        torch.cuda.synchronize()
        nrm = np.linalg.norm(to_np(A), 2)
        assert np.abs(to_np(ev) - to_np(ev_ref)).max() <= 1e-12 * nrm
        assert np.abs(to_np(vec) - to_np(vec_ref)).max() <= 1e-10
        # and the decomposition itself: A V = V diag(ev), V orthonormal
        V = to_np(vec)
        assert np.abs(to_np(A) @ V - V * to_np(ev)).max() <= 1e-12 * nrm * n
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-11


def test_syev_noalloc_allocates_nothing():
    """The point of the entry point: once a warm-up call has loaded its kernels,
    a further call takes no device memory (neither from the driver nor from
    torch's caching allocator)."""
    from paper_1309_0787_gb300 import otm
    n = 120
    A = torch.as_tensor(_matrix(7, n)).cuda()
    ev = torch.empty(n, dtype=torch.float64, device="cuda")
    vec = torch.empty(n, n, dtype=torch.float64, device="cuda")
    otm.syev_noalloc(A, ev, vec)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch0 = torch.cuda.memory_reserved()
    otm.syev_noalloc(A, ev, vec)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == torch0


def test_syev_noalloc_rejects_too_large():
    from paper_1309_0787_gb300 import otm
    n = 161
    A = torch.eye(n, dtype=torch.float64, device="cuda")
    ev = torch.empty(n, dtype=torch.float64, device="cuda")
    vec = torch.empty(n, n, dtype=torch.float64, device="cuda")
    with pytest.raises(otm.OtmError) as e:
        otm.syev_noalloc(A, ev, vec)
    assert e.value.status == 1 and "160" in str(e.value)
