"""Batched factorization and solve (independent problems of different sizes on several
streams, through spalu_factor_numeric_batch / spalu_solve_batch) against the same problems
factored and solved one at a time, and one of them against the CPU oracle."""
import numpy as np
import pytest

import workloads as W
from parity import assert_close, rel_errors
from oracle.nd import nested_dissection
from oracle.spalu import Options as OOpts, factor as ofactor, solve as osolve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _problem(n, seed, dev):
    P = W.make_problem("diffusion", n, seed=seed, nrhs=1)
    A = P.A
    csr = (torch.from_numpy(A.indptr).to(dev), torch.from_numpy(A.indices).to(dev), torch.from_numpy(A.data).to(dev))
    return P, csr, torch.from_numpy(np.ascontiguousarray(P.B.T)).to(dev)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_one_at_a_time(precision):
    from paper_2408_14193_gb300 import Factor, NestedDissection, factor_batch, solve_batch
    dev = torch.device("cuda:0")
    sizes = [63, 127, 63, 255, 127, 63, 31]
    nds = {n: NestedDissection(n) for n in set(sizes)}
    probs = [_problem(n, 100 + i, dev) for i, n in enumerate(sizes)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    fs = [Factor(nds[n], eps_id=1e-8, symmetric=1, precision=precision) for n in sizes]
    st = [streams[i % 3] for i in range(len(sizes))]
    torch.cuda.synchronize()
    factor_batch(fs, [p[1] for p in probs], st)
    Xs = [torch.empty_like(p[2]) for p in probs]
    solve_batch(fs, [p[2] for p in probs], Xs, st)
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        g = Factor(nds[n], eps_id=1e-8, symmetric=1, precision=precision)
        g.factor(*probs[i][1])
        Y = g.solve(probs[i][2])
        torch.cuda.synchronize()
        x, y = Xs[i].cpu().numpy().T, Y.cpu().numpy().T       # (N, nrhs): one column per RHS
        # the solve adds separator contributions with atomics, in a run-dependent order: FP64
        # rounding for the plain form; FP32 rounding of an FP32 factor for the mixed one (its
        # direct solve is only accurate to ~1e-4 at this eps, refinement restores 1e-10; single
        # entries near a zero of the solution move by up to ~1e-3 of its largest entry)
        if precision == 0:
            assert_close(x, y, 1e-12, f"problem {i}, n {n}")
        else:
            nrm, ent = rel_errors(x, y)
            assert nrm <= 1e-4 and ent <= 5e-3, f"problem {i}, n {n}: {nrm:.3e}, {ent:.3e}"
    # one problem of the batch against the oracle (FP64 parity bar)
    if precision == 0:
        P = probs[3][0]
        xo = osolve(ofactor(P.A, nested_dissection(255, 255), OOpts(eps=1e-8, symmetric=True)), P.B)
        x = Xs[3].cpu().numpy().T
        assert_close(x, xo, 1e-6, f"oracle, n {n}")


def test_batch_rejects_bad_arguments():
    from paper_2408_14193_gb300 import Factor, NestedDissection, SpaluError, factor_batch
    dev = torch.device("cuda:0")
    nd = NestedDissection(63)
    f = Factor(nd, eps_id=1e-8, symmetric=1)
    _, csr, _ = _problem(63, 5, dev)
    with pytest.raises(ValueError):
        factor_batch([f], [csr, csr], [torch.cuda.current_stream()])
    big = torch.zeros(csr[2].numel() * 10, dtype=torch.float64, device=dev)
    with pytest.raises(SpaluError):
        factor_batch([f], [(csr[0], csr[1], big)], [torch.cuda.current_stream()])


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_graph_matches_one_at_a_time(precision):
    """Independent problems of different sizes as one CUDA graph (factor, solve, one GMRES
    cycle each, spread over 3 branches): every problem refined to 1e-10 (CPU residual), the
    replay follows new values written into the same buffers."""
    from paper_2408_14193_gb300 import BatchGraph, Factor, NestedDissection
    dev = torch.device("cuda:0")
    sizes = [63, 127, 63, 255, 31]
    nds = {n: NestedDissection(n) for n in set(sizes)}
    probs = [_problem(n, 200 + i, dev) for i, n in enumerate(sizes)]
    eps = 1e-8 if precision == 0 else 5e-7
    fs = [Factor(nds[n], eps_id=eps, symmetric=1, precision=precision) for n in sizes]
    Xs = [torch.zeros_like(p[2]) for p in probs]
    bg = BatchGraph(fs, [p[1] for p in probs], [p[2] for p in probs], Xs, nstreams=3)

    def check(Ps):
        for P, X in zip(Ps, Xs):
            x = X.cpu().numpy().T
            res = np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0)
            assert np.all(res <= 1e-10), res

    for _ in range(2):
        for X in Xs:
            X.zero_()
        it, rel = bg.run()
        assert np.all(rel <= 1e-10) and np.all(it >= 1)
        check([p[0] for p in probs])
    # new matrices (other seeds) in the same buffers, same right-hand sides
    new = []
    for i, (n, p) in enumerate(zip(sizes, probs)):
        Q = W.make_problem("diffusion", n, seed=300 + i, nrhs=1)
        Q.B = p[0].B
        p[1][2].copy_(torch.from_numpy(Q.A.data).to(dev))
        new.append(Q)
    it, rel = bg.run()
    check(new)


def test_batch_graph_rejects_bad_arguments():
    from paper_2408_14193_gb300 import BatchGraph, Factor, NestedDissection, SpaluError
    dev = torch.device("cuda:0")
    nd = NestedDissection(31)
    f = Factor(nd, eps_id=1e-8, symmetric=1)
    P, csr, B = _problem(31, 5, dev)
    with pytest.raises(SpaluError):                 # the same handle twice
        BatchGraph([f, f], [csr, csr], [B, B.clone()], [torch.zeros_like(B), torch.zeros_like(B)])
    with pytest.raises(SpaluError):                 # X aliasing B
        BatchGraph([f], [csr], [B], [B])
