"""CPU pins of the counter-based instance generator (Philox4x32-10 and the
Marsaglia-Tsang gamma draws) and of the whitened-LDA instance model."""
import numpy as np

import synth
from oracle import stgd


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 published with Random123
    (Salmon et al., SC 2011)."""
    cases = [((0, 0, 0, 0, 0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
             ((0xffffffff,) * 6, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
             ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344, 0xa4093822, 0x299f31d0),
              (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for args, want in cases:
        got = tuple(int(x) for x in synth.philox4x32(*args))
        assert got == want


def test_unit_map_open_interval():
    x = np.array([0, 1, 511, 512, 0xFFFFFFFF], dtype=np.uint32)
    u = synth.bits_to_unit(x)
    assert u.dtype == np.float32 and np.all(u > 0) and np.all(u < 1)
    assert u[0] == u[2] and u[3] > u[0]
    np.testing.assert_allclose(u[-1], 1 - 2.0 ** -24, rtol=0)


def test_dirichlet_moments_and_whitened_identities():
    """h ~ Dir(alpha): mean alpha/alpha0 and variance alpha(alpha0-alpha)/
    (alpha0^2 (alpha0+1)); whitened samples y = m h satisfy (alpha0+1) E[yy^T]
    - alpha0 ybar ybar^T = I and a whitened third moment sum lam_i u_i^(x)3 --
    all up to sampling error at n = 2e5 (k = 4, alpha_i down to 0.03)."""
    inst = synth.whitened_lda_instances(11, 2, 4, alpha0_range=(0.3, 1.5))
    Y = synth.whitened_lda_samples(inst, 200000, 12)
    for i in range(2):
        a0, al = inst["alpha0"][i], inst["alpha"][i]
        y = Y[i].astype(np.float64)
        h = np.linalg.solve(inst["m"][i].astype(np.float64), y.T).T
        np.testing.assert_allclose(h.sum(axis=1), 1.0, atol=1e-5)
        assert h.min() >= -1e-6
        var = al * (a0 - al) / (a0 ** 2 * (a0 + 1))
        assert np.abs(h.mean(axis=0) - al / a0).max() < 5 * np.sqrt(var.max() / 2e5)
        assert np.abs(h.var(axis=0) - var).max() < 0.03 * var.max()
        yb = y.mean(axis=0)
        M2 = (a0 + 1) * y.T @ y / len(y) - a0 * np.outer(yb, yb)
        assert np.abs(M2 - np.eye(4)).max() < 0.02
        T = stgd.whitened_tensor(y, y, y, (yb, yb, yb), a0)
        U, lam = inst["U"][i], inst["lam"][i]
        Tst = np.einsum("i,ai,bi,ci->abc", lam, U, U, U)
        assert np.linalg.norm(T - Tst) / np.linalg.norm(Tst) < 0.02


def test_gamma_draws_match_gamma_law():
    """Marsaglia-Tsang draws (with the alpha < 1 boost): mean alpha and
    variance alpha of Gamma(alpha, 1), for alpha below and above 1."""
    for a in (0.2, 0.9, 3.5):
        L = synth._log_gamma_draws(np.array([a], dtype=np.float32),
                                   np.arange(100000, dtype=np.uint32),
                                   np.array([0], dtype=np.uint32), 3, (np.uint32(5), np.uint32(0)))
        g = np.exp(L[:, 0].astype(np.float64))
        assert abs(g.mean() - a) < 4 * np.sqrt(a / 1e5)
        assert abs(g.var() - a) < 0.05 * a + 4 * np.sqrt(2 * a * a / 1e5)


def test_samples_reproducible_by_instance_index():
    inst = synth.whitened_lda_instances(2, 3, 5)
    a = synth.whitened_lda_samples(inst, 50, 9)
    b = synth.whitened_lda_samples(inst, 50, 9, first=1, count=2)
    np.testing.assert_array_equal(a[1:], b)


def test_signed_column_selection_structure():
    S = synth.signed_column_selection(3, 50, 12)
    assert S.shape == (50, 12) and S.dtype == np.float32
    assert (np.count_nonzero(S, axis=0) == 1).all()
    assert set(np.unique(S[S != 0])) <= {-1.0, 1.0}
    rows = np.nonzero(S.T)[1]
    assert len(set(rows.tolist())) == 12                 # distinct rows
    np.testing.assert_array_equal(S, synth.signed_column_selection(3, 50, 12))
