"""Pins of the oracle's learned rank predictor (oracle/predictor.py) against things other
than itself: torch's bfloat16 conversion and Adam (independent library routines), central
finite differences, closed forms of special cases, and invariants of the features."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import predictor as pr
from oracle.nd import nested_dissection
from oracle.spalu import Options, factor, solve


def test_bf16_matches_torch_including_ties():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-8, 8, 20000)).astype(np.float32)
    # exact ties: low 16 bits = 0x8000 (even and odd upper halves)
    bits = rng.integers(0, 2 ** 31, 2000, dtype=np.uint64).astype(np.uint32)
    ties = ((bits & np.uint32(0x7F7F0000)) | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties, -ties, np.float32([0.0, -0.0, 1.0, 65504.0])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(pr.bf16(x).view(np.uint32), ref.view(np.uint32))


def _data(n=96, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, pr.NFEAT)) * 2.0 + 1.0
    Y = np.stack([rng.uniform(1, 5, n), rng.uniform(2, 5, n)], axis=1)
    return X, Y


def test_gradient_matches_central_differences():
    X, Y = _data()
    p = pr.init_params(3).astype(np.float64)
    mu, isd = pr.fit_norm(X)
    loss, g = pr.loss_grad(p, mu, isd, X, Y)
    rng = np.random.default_rng(4)
    idx = rng.choice(pr.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (pr.loss_grad(p + e, mu, isd, X, Y)[0] - pr.loss_grad(p - e, mu, isd, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_loss_is_half_mean_squared_error_of_outputs():
    X, Y = _data(32, 5)
    p = pr.init_params(6)
    mu, isd = pr.fit_norm(X)
    _, _, _, o = pr.forward(p, mu, isd, X)
    loss, _ = pr.loss_grad(p, mu, isd, X, Y)
    assert loss == pytest.approx(float(np.mean(np.sum((o - Y) ** 2, axis=1))) / 2.0, rel=1e-12)


def test_adam_first_step_is_lr_times_sign_and_matches_torch():
    torch = pytest.importorskip("torch")
    X, Y = _data(64, 7)
    p0 = pr.init_params(8).astype(np.float64)
    mu, isd = pr.fit_norm(X)
    _, g = pr.loss_grad(p0, mu, isd, X, Y)
    p1, m, v = pr.adam_step(p0, np.zeros_like(p0), np.zeros_like(p0), g, 1, 1e-3)
    big = np.abs(g) > 1e-4
    assert np.allclose((p0 - p1)[big], 1e-3 * np.sign(g[big]), rtol=1e-3, atol=0)
    # five steps against torch.optim.Adam on the same gradients
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    rng = np.random.default_rng(9)
    for step in range(1, 6):
        gs = rng.standard_normal(p0.size)
        opt.zero_grad()
        t.grad = torch.tensor(gs)
        opt.step()
        p, m, v = pr.adam_step(p, m, v, gs, step, 1e-3)
    assert np.allclose(p, t.detach().numpy(), rtol=0, atol=1e-12)


def test_bf16_inference_is_exact_when_every_sum_is_representable():
    """Parameters and standardised inputs that are small dyadic numbers make every float32
    sum exact, so the BF16 inference must equal the FP64 forward pass bit for bit."""
    rng = np.random.default_rng(10)
    W1 = rng.integers(-4, 5, (pr.NHID, pr.NFEAT)) / 8.0
    b1 = rng.integers(-4, 5, pr.NHID) / 8.0
    W2 = rng.integers(-4, 5, (pr.NOUT, pr.NHID)) / 8.0
    b2 = rng.integers(-4, 5, pr.NOUT) / 8.0
    p = pr.pack(W1, b1, W2, b2, np.float32)
    X = rng.integers(-8, 9, (50, pr.NFEAT)) / 4.0
    mu = np.zeros(pr.NFEAT, np.float32)
    isd = np.ones(pr.NFEAT, np.float32)
    o = pr.infer_bf16(p, mu, isd, X)
    _, a, h, o64 = pr.forward(p, mu, isd, X)
    # hidden units are multiples of 1/32 below 2^8: representable in bfloat16 only if they
    # have at most 8 significant bits, which holds here (|a| < 8)
    assert np.all(np.abs(a) < 8)
    assert np.array_equal(o.astype(np.float64), o64)


def test_sketch_size_special_cases():
    p, h0 = 5, 16
    for k in (0, 3, 12, 20):
        o = np.float32([math.log2(1 + k), math.log2(k + p)])
        assert pr.sketch_size(o, 1000, 40, p, h0, 0.0) == k + p
    # clamps: far rows, and the adaptive bound max(h0, 2(e+p))
    assert pr.sketch_size(np.float32([10.0, 10.0]), 37, 40, p, h0, 0.0) == 37
    assert pr.sketch_size(np.float32([10.0, 10.0]), 1000, 10, p, h0, 0.0) == 30
    assert pr.sketch_size(np.float32([np.nan, -1e9]), 1000, 10, p, h0, 0.0) >= 1


def test_id_error_test_accepts_exact_and_rejects_perturbed():
    rng = np.random.default_rng(11)
    Bs = rng.standard_normal((40, 6))
    T = rng.standard_normal((6, 9))
    B = np.hstack([Bs, Bs @ T])
    perm = np.arange(15)
    assert pr.id_error_ok(B, perm, 6, T, 1e-10)
    assert not pr.id_error_ok(B, perm, 6, T + 1e-6, 1e-10)
    # shuffled columns: the permutation is honoured
    q = rng.permutation(15)
    Bq = B[:, np.argsort(q)]
    assert pr.id_error_ok(Bq, q, 6, T, 1e-10)


def _records(kind, n, seed, eps=1e-8):
    P = W.make_problem(kind, n, seed=seed, nrhs=1)
    rec = []
    factor(P.A, nested_dissection(n, n), Options(eps=eps, symmetric=P.symmetric, record=rec))
    return P, rec


def test_feature_invariants():
    # records come from the segments the predictor serves (e + p > 2 h0): 127^2 has a few dozen
    _, lap = _records("laplace", 127, 1)
    _, hel = _records("helmholtz", 127, 2)
    _, cdf = _records("convdiff", 127, 3)
    for recs in (lap, hel, cdf):
        X = np.array([r[0] for r in recs])
        assert np.all(np.isfinite(X))
        dec = X[:, 11:16]
        assert np.all(np.diff(dec, axis=1) <= 1e-9)          # pivoted R: |R_jj| non-increasing
        assert np.all(dec <= 8.0 + 1e-9)                       # ratio <= 1, minus log10(1e-8)
        assert np.all(X[:, 5] <= 1e-12) and np.all(X[:, 6] >= -1e-12)
    Xl = np.array([r[0] for r in lap])
    assert np.allclose(Xl[:, 5:8], 0.0, atol=1e-12)           # constant diagonal
    assert np.allclose(Xl[:, 10], 0.0)                         # symmetric
    assert np.all(Xl[:, 8] >= -1e-12)                          # 4/h^2 over <= 4/h^2
    Xh = np.array([r[0] for r in hel])
    assert np.all(Xh[:, 9] > Xl[:, 9].max())                   # the k^2 shift shows
    Xc = np.array([r[0] for r in cdf])
    assert np.all(Xc[:, 10] > 0.0)                             # convection shows
    for r in lap:                                              # targets are well defined
        k, nF, e, l = r[1:]
        assert 0 <= k <= e and nF > 16 and e + 5 > 2 * 16     # only segments past the rank bound


def test_oracle_predictor_saves_passes_and_keeps_the_solution():
    """Train the oracle network on adaptive records of small problems; on a held-out problem
    the predicted one-pass IDs save ID passes (most predicted segments save the second
    adaptive pass) and the solution stays within the ID tolerance of the adaptive one."""
    rec = []
    for kind, n, seed in [("diffusion", 127, 1), ("diffusion", 255, 2), ("laplace", 127, 3),
                          ("convdiff", 127, 4)]:
        rec += _records(kind, n, seed)[1]
    X = np.array([r[0] for r in rec])
    Y = np.array([pr.targets(r[1], r[2], 5) for r in rec])
    mu, isd = pr.fit_norm(X)
    p, losses = pr.train(pr.init_params(0), mu, isd, X, Y, epochs=150, batch=64, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0]
    P = W.make_problem("diffusion", 127, seed=11, nrhs=1)
    nd = nested_dissection(127, 127)
    Fa = factor(P.A, nd, Options(eps=1e-8, symmetric=True))
    Fp = factor(P.A, nd, Options(eps=1e-8, symmetric=True,
                                 predictor={"params": p.astype(np.float32), "mu": mu, "isd": isd}))
    pa = sum(v["passes"] for v in Fa.stats["levels"].values())
    pp = sum(v["passes"] for v in Fp.stats["levels"].values())
    npred = sum(v["predicted"] for v in Fp.stats["levels"].values())
    nfb = sum(v["fallbacks"] for v in Fp.stats["levels"].values())
    assert npred > 0 and pa - pp >= 0.4 * npred and nfb <= 0.3 * npred, (pa, pp, npred, nfb)
    xa, xp = solve(Fa, P.B), solve(Fp, P.B)
    assert np.linalg.norm(xp - xa) <= 1e-5 * np.linalg.norm(xa)
