"""Host-side logic of bench.py that needs no GPU: the algorithmic flop count
behind the STGD roofline, the per-rank workload, and the oracle stage checks of
the LDA precision workload (fed the oracle's own results, they report zero)."""
import numpy as np

import bench
import synth
from oracle import moments as om
from oracle import stgd as ostgd


def test_sgd_flops_closed_form():
    # per step 6 k^2 b_s (two projections and the data product, three views) + 4 k^3
    cfg = dict(bench.CFG)
    flops, steps = bench.sgd_flops(cfg)
    n, b, k, ep = cfg["n_per"], cfg["b"], cfg["k"], cfg["epochs"]
    per_epoch = -(-n // b)
    assert steps == per_epoch * ep
    assert flops == ep * (6 * k * k * n + per_epoch * 4 * k ** 3)
    assert flops == 6.4e9                           # the MMSB k = 100 line


def test_make_inputs_shapes_and_rank_seeds():
    cfg = dict(bench.CFG)
    cfg.update(n_per=80, k=5, oversample=3, epochs=2)
    a = bench.make_inputs(cfg, 0)
    b = bench.make_inputs(cfg, 1)
    assert a["S_pairs"].shape == (80, 8) and a["perm"].shape == (2, 80)
    assert a["V0"].shape == (5, 5) and a["Pi_X"].shape == (80, 5)
    np.testing.assert_allclose(a["V0"].T @ a["V0"], np.eye(5), atol=1e-5)
    assert not np.array_equal(a["S_w"], b["S_w"])


def test_lda_oracle_checks_zero_on_oracle_inputs():
    c = dict(bench.LDA)
    c.update(k=6, b=40)
    corp = synth.lda_corpus(1, 300, 50, 6, 0.1, 0.1, 30)
    X = corp["X"]
    W = np.random.default_rng(2).standard_normal((50, 6))
    Xs = om.as_sparse(X)
    Y = (Xs @ W) / np.asarray(Xs.sum(axis=1)).ravel()[:, None]
    docs = np.arange(0, 300, 11).astype(np.int32)
    V0 = synth.haar_orthonormal(3, 6).astype(np.float64)
    Yb, yb = Y[:40], Y.mean(axis=0)
    V1 = ostgd.sgd_step(V0, Yb, Yb, Yb, (yb, yb, yb), c["theta"], c["beta0"],
                        6 * c["alpha_i"])
    out = bench.lda_oracle_checks(c, X, W, Y[docs], docs, Yb, yb, V0,
                                  {"fp32": V1, "off": V0 + 1.1 * (V1 - V0)})
    assert out["projection_rows_rel_err"] < 1e-14
    st = out["step"]
    assert st["fp32"]["update_rel_err"] < 1e-12 and st["fp32"]["grad_rel_err"] < 1e-12
    assert st["fp32"]["grad_rel_err_worst_component"] < 1e-12
    assert abs(st["off"]["update_rel_err"] - 0.1) < 1e-9
    # the gradient error is relative to the two terms, never above the update error
    assert 0 < st["off"]["grad_rel_err"] <= st["off"]["update_rel_err"]


def test_lda_inputs_shapes_and_rank_seeds(tmp_path, monkeypatch):
    import tempfile
    monkeypatch.setattr(tempfile, "gettempdir", lambda: str(tmp_path))
    c = dict(bench.LDA)
    c.update(n_docs=200, d=60, k=5, epochs=2, doc_len=20)
    a = bench.lda_inputs(c, 0)
    assert not a["cached"]
    a2 = bench.lda_inputs(c, 0)           # second call loads the cached corpus
    assert a2["cached"]
    for f in ("row_ptr", "col", "val"):
        np.testing.assert_array_equal(getattr(a["X"], f), getattr(a2["X"], f))
    b = bench.lda_inputs(c, 1)
    assert a["S"].shape == (60, 25) and a["perm"].shape == (2, 200) and a["V0"].shape == (5, 5)
    assert not np.array_equal(a["S"], b["S"])


def test_cpu_oracle_sample_extrapolates_whitening(tmp_path, monkeypatch):
    """The oracle timing leg runs on a small corpus and returns positive times;
    the whitening estimate is at least the largest sampled fraction's time."""
    import tempfile
    monkeypatch.setattr(tempfile, "gettempdir", lambda: str(tmp_path))
    c = dict(bench.LDA)
    c.update(n_docs=400, d=80, k=4, epochs=1, doc_len=30, b=64)
    host = bench.lda_inputs(c, 0)
    r = bench.lda_oracle_sample(c, host, (0.25, 0.5), None)
    assert r["stgd_steps_run"] == r["stgd_steps_total"] == 7
    assert r["whiten_s"] >= r["whiten_sample_s"][-1] > 0
    assert r["project_means_s"] > 0 and r["stgd_s"] > 0


def test_sym_sgd_flops_closed_form():
    # 300,000 samples, b = 1,024: 292 full minibatches and one of 992 per epoch
    f = bench.sym_sgd_flops(300000, 1024, 100, 20)
    assert f == 20 * (4 * 100 ** 2 * 300000 + 293 * 4 * 100 ** 3)


def test_sgd_grid_traffic_only_for_the_captured_kernel_and_workload(tmp_path, monkeypatch):
    """The captured DRAM bytes are reported for the grid form on the default corpus
    while the kernel source hashes as captured; otherwise null."""
    c = dict(bench.LDA)
    assert bench.sgd_grid_traffic("auto", c) == bench.SGD_GRID_TRAFFIC["bytes"]
    assert bench.sgd_grid_traffic("split", c) is None
    c2 = dict(c)
    c2["k"] = 50
    assert bench.sgd_grid_traffic("grid", c2) is None
    src = tmp_path / bench.SGD_GRID_TRAFFIC["source"]
    src.parent.mkdir(parents=True)
    src.write_text("// another kernel\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.sgd_grid_traffic("auto", c) is None
