"""GPU tests of the batched tensor-core STGD (one persistent launch running
many independent decompositions).

Each chain of the batch runs the same Lemma 3 schedule as a single
otm_sgd_run_lp call; with the same cluster size the two are bit-identical, with
another cluster size they differ only in FP32 summation order.  Against the
FP64 oracle the tolerance of the single-chain tests (2e-2 relative) holds for BF16
and FP8.
"""
import numpy as np
import pytest

import synth
from oracle import stgd as ostgd
from tests._util import rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def otm():
    from paper_1309_0787_gb300 import otm as _otm
    return _otm


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _problem(otm, seed, k, n, b, epochs, restarts, beta0, prec, sigma=0.05):
    o = synth.orthogonal_samples(seed, k, n, sigma)
    Y = o["Y"]
    yb = Y.astype(np.float64).mean(axis=0)
    perm = synth.epoch_permutations(seed + 1, n, epochs)
    V0 = np.stack([synth.haar_orthonormal(seed + 2 + r, k) for r in range(restarts)])
    Yq, sc = otm.quantize_samples(_dev(Y), prec)
    return {"Y": Y, "yb": yb, "perm_np": perm, "V0": V0,
            "Yq": Yq, "scales": sc, "ybar3": _dev(np.stack([yb] * 3)), "perm": _dev(perm),
            # V is component-contiguous: restart r's matrix is V0[r]^T
            "V": _dev(np.ascontiguousarray(V0.transpose(0, 2, 1)).astype(np.float32)),
            "epochs": epochs, "b": b, "beta0": beta0, "theta": 1.0, "alpha0": 0.0}


def _items(k, restarts):
    """Work items of one problem: restarts of a problem with k <= 64 run
    floor(128 / k) to an item."""
    per = 128 // k if k <= 64 else 1
    return -(-restarts // per)


def _single(otm, p, r, prec):
    Vd = _dev(p["V0"][r].T.copy().astype(np.float32))
    q = (p["Yq"], p["scales"])
    otm.sgd_run_lp(Vd, q, q, q, p["ybar3"], p["perm"], p["epochs"], p["b"], p["beta0"],
                   p["theta"], p["alpha0"], prec)
    return Vd


def test_batched_equals_single_same_cluster(otm):
    """One problem, three restarts, cluster size forced to the one the single
    call picks for k = 100, b = 1024 (8): results agree to rounding."""
    prec = otm.PREC_BF16
    p = _problem(otm, 11, 100, 4096, 1024, 2, 3, 1e-2, prec)
    batch = otm.SgdBatch([p], prec, cluster=8)
    assert batch.nitems == 3 and batch.cluster == 8
    batch.launch()
    batch.check()
    for r in range(3):
        Vs = _single(otm, p, r, prec)
        torch.cuda.synchronize()
        a, s = to_np(p["V"][r]), to_np(Vs)
        assert np.abs(a - s).max() <= 1e-6 * np.abs(s).max(), (r, np.abs(a - s).max())


@pytest.mark.parametrize("prec_name", ["PREC_BF16", "PREC_FP8"])
def test_batched_mixed_sizes_autotuned(otm, prec_name):
    """Problems of different k, n, b and epochs in one launch (autotuned
    cluster size): every chain matches its own single-chain run."""
    prec = getattr(otm, prec_name)
    specs = [(21, 8, 600, 64, 3, 5), (22, 37, 1500, 256, 2, 3), (23, 100, 3000, 512, 1, 2),
             (24, 128, 2048, 1024, 2, 1)]
    probs = [_problem(otm, s, k, n, b, e, r, 5e-3, prec) for s, k, n, b, e, r in specs]
    batch = otm.SgdBatch(probs, prec)
    assert batch.nitems == sum(_items(s[1], s[-1]) for s in specs)
    assert batch.cluster in (1, 2, 4, 8, 16)
    # the tuned schedule: sample stages and V-image buffering recorded in the plan
    assert 1 <= batch.plan.stages <= 4 and batch.plan.vimg2 in (0, 1)
    assert batch.plan.vimg2 == 0 or batch.cluster > 1
    batch.launch()
    batch.check()
    tol = 1e-2 if prec == otm.PREC_BF16 else 2e-2
    for p in probs:
        for r in range(p["V0"].shape[0]):
            Vs = _single(otm, p, r, prec)
            torch.cuda.synchronize()
            assert rel(to_np(p["V"][r]), to_np(Vs)) < tol


@pytest.mark.parametrize("k,restarts", [(16, 8), (24, 3), (16, 10)])
def test_batched_stacked_restarts_equal_single(otm, k, restarts):
    """Restarts of one problem stacked into one chain of R k components (one
    tile load and one pair of products for all of them, the Gram term masked to
    each restart's block) give each restart's single-chain result up to FP32
    summation order; with k = 24 the restart boundaries fall inside 8-component
    groups."""
    prec = otm.PREC_BF16
    p = _problem(otm, 101 + k, k, 1500, 256, 2, restarts, 5e-3, prec)
    batch = otm.SgdBatch([p], prec, cluster=1)
    assert batch.nitems == _items(k, restarts)  # (16, 10): items of 8 and 2 restarts
    batch.launch()
    batch.check()
    for r in range(restarts):
        Vs = _single(otm, p, r, prec)
        torch.cuda.synchronize()
        a, s = to_np(p["V"][r]), to_np(Vs)
        assert np.abs(a - s).max() <= 1e-5 * np.abs(s).max(), (r, np.abs(a - s).max())


def test_batched_two_groups_beyond_128(otm):
    """Problems with k <= 128 and k > 128 in one batch (two persistent launches):
    every chain matches its own single-chain run."""
    prec = otm.PREC_BF16
    specs = [(71, 48, 800, 128, 2, 2), (72, 200, 1024, 256, 1, 2), (73, 256, 1024, 512, 1, 1)]
    probs = [_problem(otm, s, k, n, b, e, r, 5e-3, prec) for s, k, n, b, e, r in specs]
    batch = otm.SgdBatch(probs, prec)
    assert batch.nitems == 4 and batch.plan.nitems_wide == 3
    batch.launch()
    batch.check()
    for p in probs:
        for r in range(p["V0"].shape[0]):
            Vs = _single(otm, p, r, prec)
            torch.cuda.synchronize()
            assert rel(to_np(p["V"][r]), to_np(Vs)) < 1e-2


def test_batched_two_groups_fp8(otm):
    """FP8 with chains beyond k = 128 (their master rows in the workspace):
    every chain matches its own single-chain FP8 run."""
    prec = otm.PREC_FP8
    specs = [(91, 64, 800, 128, 2, 2), (92, 200, 1024, 256, 1, 2)]
    probs = [_problem(otm, s, k, n, b, e, r, 5e-3, prec) for s, k, n, b, e, r in specs]
    batch = otm.SgdBatch(probs, prec)
    assert batch.plan.nitems_wide == 2 and batch.plan.cluster_wide in (4, 8, 16)
    assert 1 <= batch.plan.stages_wide <= 4 and batch.plan.vimg2_wide in (0, 1)
    batch.launch()
    batch.check()
    for p in probs:
        for r in range(p["V0"].shape[0]):
            Vs = _single(otm, p, r, prec)
            torch.cuda.synchronize()
            assert rel(to_np(p["V"][r]), to_np(Vs)) < 2e-2


def test_batched_two_groups_forced_cluster(otm):
    """Both groups with the narrow cluster size given (1): the kernel's launch
    attributes must admit the larger of the two plans' shared memory."""
    prec = otm.PREC_BF16
    specs = [(81, 128, 1024, 256, 1, 2), (82, 256, 1024, 512, 1, 1), (83, 16, 512, 64, 2, 2)]
    probs = [_problem(otm, s, k, n, b, e, r, 5e-3, prec) for s, k, n, b, e, r in specs]
    batch = otm.SgdBatch(probs, prec, cluster=1)
    assert batch.cluster == 1 and batch.plan.nitems_wide == 1
    batch.launch()
    batch.check()
    for p in probs:
        for r in range(p["V0"].shape[0]):
            Vs = _single(otm, p, r, prec)
            torch.cuda.synchronize()
            assert rel(to_np(p["V"][r]), to_np(Vs)) < 1e-2


@pytest.mark.parametrize("prec_name", ["PREC_BF16", "PREC_FP8"])
def test_batched_tracks_oracle(otm, prec_name):
    """Batched BF16 and FP8 chains against the FP64 oracle run of Lemma 3."""
    prec = getattr(otm, prec_name)
    probs = [_problem(otm, 31, 16, 2000, 256, 4, 2, 5e-3, prec),
             _problem(otm, 41, 24, 1200, 128, 3, 2, 5e-3, prec)]
    batch = otm.SgdBatch(probs, prec)
    batch.launch()
    batch.check()
    torch.cuda.synchronize()
    for p in probs:
        for r in range(2):
            Vo, _ = ostgd.sgd_run(p["V0"][r], p["Y"], p["Y"], p["Y"], (p["yb"],) * 3,
                                  p["perm_np"], p["b"], p["beta0"], 1.0, 0.0)
            assert rel(to_np(p["V"][r]).T, Vo) < 2e-2


def test_batched_graph_replay(otm):
    """The launch captured in a CUDA graph and replayed gives the eager result."""
    prec = otm.PREC_BF16
    p = _problem(otm, 51, 32, 1000, 200, 2, 4, 5e-3, prec)
    V0 = p["V"].clone()
    batch = otm.SgdBatch([p], prec)
    batch.launch()
    batch.check()
    eager = p["V"].clone()
    p["V"].copy_(V0)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.launch()
    p["V"].copy_(V0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    batch.check()
    assert torch.equal(p["V"], eager)


def test_batched_rejects_bad_problem(otm):
    p = _problem(otm, 61, 8, 100, 10, 1, 1, 1e-2, otm.PREC_BF16)
    p["V"] = torch.zeros(1, 8, 8, device="cuda", dtype=torch.float32)
    bad = dict(p)
    bad["b"] = 0
    with pytest.raises(otm.OtmError):
        otm.SgdBatch([bad], otm.PREC_BF16)
    with pytest.raises(otm.OtmError):
        otm.SgdBatch([p], otm.PREC_BF16, cluster=3)
