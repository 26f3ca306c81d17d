"""GPU parity of the whole community-model hot path at full size against the
FP64 oracle: the mixed-membership blockmodel of four parts of 5,000 nodes,
k = 100, p = 0.1, q = 0.005, pi ~ Dir(0.01 1_k) (alpha0 = 1), randomised
whitening (oversampling 20, 2 power iterations) -> projection of the three
views (Section 2.2, Eqs. (7)-(11)) -> means -> 100 STGD steps (b = 1,024,
beta_t = 1e-2/sqrt(t), theta = 1) -> unwhitening (Lemma 4) -> membership of
the X nodes -> p-value validation (recovery ratio R, average error E).

Two comparisons:
  * stage by stage, each oracle stage fed the GPU's output of the stage before
    (tolerances from the arithmetic of each stage: float32 sparse products
    and STGD steps, FP64 unwhitening and validation), checked over the whole
    result and for every column (component) on its own;
  * the oracle's own pipeline from the same seeded inputs.  The float32 range
    finder reproduces the oracle's whitening to about 1e-3 (its power
    iterations amplify the float32 rounding of nearly equal eigenvalues of
    M2), so this comparison uses results that do not depend on the order or
    signs of the whitened coordinates: the eigenvalues of the whitening, the
    recovery ratio and the average error.
"""
import numpy as np
import pytest

import synth
from oracle import community as oc
from oracle import moments as om
from oracle import post as opost
from oracle import stgd as ostgd
from oracle import whiten as ow
from tests._util import rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_PER, K, KT, B, EPOCHS, BETA0, THETA, ALPHA0 = 5000, 100, 120, 1024, 20, 1e-2, 1.0, 1.0


@pytest.fixture(scope="module")
def run():
    from paper_1309_0787_gb300 import otm
    g = synth.mmsb_graph(0, N_PER, K, 0.01, 0.1, 0.005)
    S_pairs = synth.gaussian(1, N_PER, KT)
    S_w = synth.gaussian(2, N_PER, KT)
    perm = synth.epoch_permutations(3, N_PER, EPOCHS)
    V0 = synth.haar_orthonormal(4, K)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    D = {x: otm.DeviceCSR.from_host(g[x]) for x in ("G_XA", "G_XB", "G_XC")}
    wh = otm.whiten_community(D["G_XA"], D["G_XB"], D["G_XC"], dev(S_pairs), dev(S_w), K, 2,
                              ALPHA0)
    Y = [otm.project(D[x], wh[w]) for x, w in (("G_XA", "W"), ("G_XB", "W_B"), ("G_XC", "W_C"))]
    yb = torch.stack([otm.column_mean(y) for y in Y])
    V = dev(V0.T.copy())
    otm.sgd_run(V, *Y, yb, dev(perm), EPOCHS, B, BETA0, THETA, ALPHA0)
    post = otm.unwhiten(V, wh["Q"], wh["Cp"], THETA, False)
    Pi_hat = otm.membership(Y[0], V, THETA)
    truth = dev(g["Pi"]["X"].T.astype(np.float32))
    val = otm.pvalue_match(Pi_hat, truth, 0.01)
    torch.cuda.synchronize()
    gpu = {"W": [to_np(wh[w]).astype(np.float64) for w in ("W", "W_B", "W_C")],
           "eig": to_np(wh["eig"]), "Y": [to_np(y).astype(np.float64) for y in Y],
           "yb": to_np(yb), "V": to_np(V).T.astype(np.float64),
           "Wplus": to_np(wh["Q"]).astype(np.float64) @ to_np(wh["Cp"]),
           "comps": to_np(post["comps"]), "lambda": to_np(post["lambda"]),
           "Pi_hat": to_np(Pi_hat).astype(np.float64), "pvalues": to_np(val["pvalues"]),
           "scores": to_np(val["scores"])}
    return {"g": g, "S_pairs": S_pairs, "S_w": S_w, "perm": perm, "V0": V0,
            # the memberships exactly as the GPU received them (float32)
            "truth": g["Pi"]["X"].T.astype(np.float32).astype(np.float64), "gpu": gpu}


def _colwise(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float((np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300))
                 .max())


def test_projection_and_means_of_gpu_whitening(run):
    """Section 2.2: y_A = G_{X,A} W, y_B = G_{X,B} W_B, y_C = G_{X,C} W_C and
    their means, from the GPU's whitening matrices (float32 sums of a node's
    about 30 edges: relative error far below 1e-6)."""
    g, gpu = run["g"], run["gpu"]
    for v, x in enumerate(("G_XA", "G_XB", "G_XC")):
        ref = om.as_sparse(g[x]) @ gpu["W"][v]
        assert rel(gpu["Y"][v], ref) < 1e-6
        assert _colwise(gpu["Y"][v], ref) < 1e-5
        np.testing.assert_allclose(gpu["yb"][v], gpu["Y"][v].mean(axis=0), rtol=1e-5,
                                   atol=1e-7 * np.abs(gpu["yb"][v]).max())


def test_stgd_run_on_gpu_samples(run):
    """Lemma 3, 100 steps with the line's schedule on the GPU's whitened views:
    the float32 persistent kernel against the FP64 oracle (matrix form), for the
    whole V and for every component."""
    gpu = run["gpu"]
    Vo, _ = ostgd.sgd_run(run["V0"], *gpu["Y"], tuple(gpu["yb"]), run["perm"], B, BETA0, THETA,
                          ALPHA0, gemm=True)
    assert rel(gpu["V"], Vo) < 1e-5
    assert _colwise(gpu["V"], Vo) < 1e-4


def test_unwhitening_of_gpu_components(run):
    """Lemma 4 in FP64 from the GPU's float32 components and factors."""
    gpu = run["gpu"]
    ref = opost.unwhiten(gpu["V"], gpu["Wplus"], THETA, False)
    np.testing.assert_allclose(gpu["lambda"], ref["lambda"], rtol=1e-12)
    assert rel(gpu["comps"], ref["mu"]) < 1e-10
    assert _colwise(gpu["comps"], ref["mu"]) < 1e-10


def test_membership_and_validation_of_gpu_results(run):
    """Lemma 4 (community case) on the GPU's view-A samples and components
    (float32 dot products: each entry within 2 k 2^-24 of the scaled sum of
    absolute products), then the p-value validation in FP64 on the GPU's
    membership: p-values within 1e-9, R identical, E within 1e-9."""
    gpu = run["gpu"]
    YA, V = gpu["Y"][0], gpu["V"]
    want = oc.membership(YA, V, THETA)
    norms = np.linalg.norm(V, axis=0)
    lam = ostgd.kappa(THETA) * norms ** 3
    scale = np.sum(lam ** -2.0) ** (-1.0 / 6.0) / (lam * norms)
    bound = 2.0 * K * 2.0 ** -24 * scale[:, None] * (np.abs(V).T @ np.abs(YA).T)
    assert np.all(np.abs(gpu["Pi_hat"] - want) <= bound + np.abs(want) * 2.0 ** -24 + 1e-30)
    ref = oc.match_scores(gpu["Pi_hat"], run["truth"], 0.01)
    np.testing.assert_allclose(gpu["pvalues"], ref["pvalues"], rtol=1e-9, atol=1e-14)
    assert gpu["scores"][0] == ref["recovery"]
    assert abs(gpu["scores"][1] - ref["error"]) <= 1e-9 * ref["error"]


def test_pipeline_against_oracle_pipeline(run):
    """The oracle's own pipeline on the same seeded inputs (its FP64 whitening,
    projections, STGD, membership and validation): the whitening eigenvalues
    within 1e-3 (float32 range finder), and the validation outcome -- R
    identical, E within 1e-3 relative."""
    g, gpu = run["g"], run["gpu"]
    wh = ow.community_whiten_randomized(g["G_XA"], g["G_XB"], g["G_XC"], K, ALPHA0,
                                        run["S_pairs"].astype(np.float64),
                                        run["S_w"].astype(np.float64), 2)
    np.testing.assert_allclose(gpu["eig"], wh["eig"], rtol=1e-3)
    Y = [om.as_sparse(g[x]) @ wh[w] for x, w in (("G_XA", "W"), ("G_XB", "W_B"),
                                                 ("G_XC", "W_C"))]
    yb = tuple(y.mean(axis=0) for y in Y)
    Vo, _ = ostgd.sgd_run(run["V0"], *Y, yb, run["perm"], B, BETA0, THETA, ALPHA0, gemm=True)
    ref = oc.match_scores(oc.membership(Y[0], Vo, THETA), run["truth"], 0.01)
    assert gpu["scores"][0] == ref["recovery"]
    assert abs(gpu["scores"][1] - ref["error"]) <= 1e-3 * ref["error"]
