"""GPU tests of the three FP32 kernels of the fused STGD step (Lemma 3): the
cluster form (one thread-block cluster, V in shared memory), the grid form
(one cooperative launch over many SMs, partial products reduced through L2)
and the split form (clusters own blocks of components, their CTAs split the
minibatch, partial columns reduced through distributed shared memory, one
grid barrier per step).  All are checked against the FP64 oracle at the FP32
tolerance (1e-5) and against each other; the form is a process-wide setting,
restored to the default after every test."""
import numpy as np
import pytest

import synth
from oracle import stgd as ostgd
from tests._util import grad_errs, rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def otm():
    from paper_1309_0787_gb300 import otm as _otm
    return _otm


@pytest.fixture
def form(otm, request):
    otm.sgd_set_form(request.param)
    yield request.param
    otm.sgd_set_form(otm.SGD_FORM_AUTO)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _views(g, n, k, sym):
    Ys = [(g.standard_normal((n, k)) * 0.3 + 0.2 * s).astype(np.float32) for s in (1, -1, 0.5)]
    if sym:
        Ys = [Ys[0]] * 3
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    return Ys, yb


def _dev_views(Ys, sym):
    Yd = [_dev(Y) for Y in Ys]
    return [Yd[0]] * 3 if sym else Yd


@pytest.mark.parametrize("form", [1, 2, 3], indirect=True)
@pytest.mark.parametrize("k,b,sym,a0", [(100, 1024, False, 1.0), (128, 2000, True, 2.0),
                                        (17, 300, False, 0.7), (1, 64, True, 1.0),
                                        (64, 4096, False, 0.0), (33, 16, False, 1.0)])
def test_step_gradient_both_forms(otm, form, k, b, sym, a0):
    """One step with beta = 1 returns V - G; G against the oracle's implicit
    gradient (the sum of the Gram and data terms), normwise 1e-5."""
    g = np.random.default_rng(k * 31 + b)
    Ys, yb = _views(g, b, k, sym)
    V0 = (0.5 * g.standard_normal((k, k))).astype(np.float32)
    Vd = _dev(V0.T.copy())
    otm.sgd_step(Vd, *_dev_views(Ys, sym), _dev(yb), 1.0, 1.0, a0)
    torch.cuda.synchronize()
    Gk = V0.astype(np.float64) - to_np(Vd).T
    V64 = V0.astype(np.float64)
    G = ostgd.grad_implicit(V64, *[Y.astype(np.float64) for Y in Ys], tuple(yb), 1.0, a0)
    gram = ostgd.kappa(1.0) * V64 @ (V64.T @ V64) ** 2
    frob, col = grad_errs(Gk, G, gram)
    assert frob < 1e-5 and col < 1e-5, (frob, col)


@pytest.mark.parametrize("form", [1, 2, 3], indirect=True)
@pytest.mark.parametrize("k,n,b,epochs,sym", [(12, 700, 128, 3, True), (100, 3000, 1024, 2, False),
                                              (40, 2500, 512, 2, False)])
def test_run_schedule_both_forms(otm, form, k, n, b, epochs, sym):
    """Epochs with permutations, a partial last minibatch and snapshots."""
    g = np.random.default_rng(k + n)
    o = synth.orthogonal_samples(k + 1, k, n, 0.05)
    Ys = [o["Y"]] * 3 if sym else [o["Y"], (o["Y"] + 0.01 * g.standard_normal(o["Y"].shape))
                                   .astype(np.float32), o["Y"][::-1].copy()]
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    perm = synth.epoch_permutations(k + 2, n, epochs)
    V0 = synth.haar_orthonormal(k + 3, k)
    spe = (n + b - 1) // b
    Vd = _dev(V0.T.copy())
    snaps = otm.sgd_run(Vd, *_dev_views(Ys, sym), _dev(yb), _dev(perm), epochs, b, 2e-3, 1.0, 0.5,
                        snapshot_every=spe)
    torch.cuda.synchronize()
    Vo, so = ostgd.sgd_run(V0, *Ys, tuple(yb), perm, b, 2e-3, 1.0, 0.5, snapshot_every=spe)
    assert rel(to_np(Vd).T, Vo) < 1e-5
    assert snaps.shape[0] == len(so) == epochs
    for s_gpu, s_ref in zip(to_np(snaps), so):
        assert rel(s_gpu.T, s_ref) < 1e-5


def test_forms_agree(otm):
    """The three forms on the same run differ only by FP32 summation order."""
    k, n, b, epochs = 100, 5000, 1024, 3
    g = np.random.default_rng(5)
    Ys, yb = _views(g, n, k, False)
    perm = synth.epoch_permutations(6, n, epochs)
    V0 = synth.haar_orthonormal(7, k).astype(np.float32)
    out = {}
    try:
        for f in (otm.SGD_FORM_CLUSTER, otm.SGD_FORM_GRID, otm.SGD_FORM_SPLIT):
            otm.sgd_set_form(f)
            Vd = _dev(V0.T.copy())
            otm.sgd_run(Vd, *_dev_views(Ys, False), _dev(yb), _dev(perm), epochs, b, 1e-2, 1.0,
                        1.0)
            torch.cuda.synchronize()
            out[f] = to_np(Vd)
    finally:
        otm.sgd_set_form(otm.SGD_FORM_AUTO)
    assert rel(out[otm.SGD_FORM_GRID], out[otm.SGD_FORM_CLUSTER]) < 1e-5
    assert rel(out[otm.SGD_FORM_SPLIT], out[otm.SGD_FORM_CLUSTER]) < 1e-5


def test_grid_form_limits(otm):
    """Forcing the grid form outside its range is an error; auto falls back."""
    k = 8
    g = np.random.default_rng(9)
    Ys, yb = _views(g, 8, k, True)
    Vd = _dev(np.eye(k, dtype=np.float32))
    try:
        otm.sgd_set_form(otm.SGD_FORM_GRID)
        with pytest.raises(otm.OtmError):   # b = 8 < 16
            otm.sgd_step(Vd, *_dev_views(Ys, True), _dev(yb), 1.0, 1e-3, 1.0)
        with pytest.raises(otm.OtmError):
            otm.sgd_set_form(4)
        otm.sgd_set_form(otm.SGD_FORM_AUTO)
        otm.sgd_step(Vd, *_dev_views(Ys, True), _dev(yb), 1.0, 1e-3, 1.0)
        torch.cuda.synchronize()
        assert np.isfinite(to_np(Vd)).all()
    finally:
        otm.sgd_set_form(otm.SGD_FORM_AUTO)


@pytest.mark.parametrize("form", [1, 2, 3], indirect=True)
def test_invalid_permutation_entries_read_as_zero_samples(otm, form):
    """A permutation entry outside [0, n) contributes a zero sample (both forms):
    the result equals the oracle's run on samples with a zero row appended and
    those entries pointed at it."""
    k, n, b, epochs = 24, 600, 256, 2
    g = np.random.default_rng(17)
    Ys, yb = _views(g, n, k, False)
    perm = synth.epoch_permutations(18, n, epochs).copy()
    perm[0, 5] = -3
    perm[1, 100] = n + 7
    V0 = synth.haar_orthonormal(19, k)
    Vd = _dev(V0.T.copy())
    otm.sgd_run(Vd, *_dev_views(Ys, False), _dev(yb), _dev(perm), epochs, b, 1e-2, 1.0, 1.0)
    torch.cuda.synchronize()
    Yz = [np.vstack([Y, np.zeros((1, k), np.float32)]) for Y in Ys]
    pz = perm.copy()
    pz[(pz < 0) | (pz >= n)] = n
    # the oracle visits perm[e, :n] of the (n + 1)-row sample matrix
    Vo, _ = ostgd.sgd_run(V0, *Yz, tuple(yb), np.ascontiguousarray(pz), b, 1e-2, 1.0, 1.0)
    assert rel(to_np(Vd).T, Vo) < 1e-5


@pytest.mark.parametrize("k,n,b,sym,offset", [(100, 45000, 20000, False, 0), (64, 30000, 30000, True, 0),
                                              (37, 9000, 4000, False, 0), (128, 20000, 7000, True, 1)])
def test_split_form_large_minibatches(otm, k, n, b, sym, offset):
    """The split form with minibatches far larger than one chunk per CTA
    (several chunks per step, the last one partial), up to a full-batch step,
    a partial last minibatch, k = 37 and views that are not 16-byte aligned
    (scalar copies), against the oracle's run at the FP32 tolerance."""
    g = np.random.default_rng(k + b)
    Ys = [(g.standard_normal((n, k)) * 0.05 + 0.1 * g.standard_normal(k)).astype(np.float32)
          for _ in range(3)]
    if sym:
        Ys = [Ys[0]] * 3
    yb = np.stack([Y.astype(np.float64).mean(axis=0) for Y in Ys])
    epochs = 1
    perm = synth.epoch_permutations(k + 5, n, epochs)
    V0 = synth.haar_orthonormal(k + 6, k)
    views = []
    for Y in (Ys[:1] if sym else Ys):
        buf = torch.zeros(n * k + offset, device="cuda", dtype=torch.float32)
        buf[offset:] = _dev(Y).reshape(-1)
        views.append(buf[offset:].view(n, k))
    if sym:
        views = views * 3
    Vd = _dev(V0.T.copy())
    try:
        otm.sgd_set_form(otm.SGD_FORM_SPLIT)
        otm.sgd_run(Vd, *views, _dev(yb), _dev(perm), epochs, b, 5e-2, 1.0, 1.0)
        torch.cuda.synchronize()
    finally:
        otm.sgd_set_form(otm.SGD_FORM_AUTO)
    Vo, _ = ostgd.sgd_run(V0, *Ys, tuple(yb), perm, b, 5e-2, 1.0, 1.0, gemm=True)
    assert rel(to_np(Vd).T, Vo) < 1e-5

