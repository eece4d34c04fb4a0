"""The whole step as one CUDA graph (spalu_factor_solve_graph) and the device-side GMRES
least-squares bookkeeping: the graph path gives what the plain calls give (refined to 1e-10,
checked by a CPU residual, and the same iteration count), replays with new matrix values in
the same buffers, falls back outside the graph when the new factor outgrows the captured
capacities, and continues outside it when one GMRES cycle of K steps is not enough."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _dev(P):
    d = torch.device("cuda:0")
    A = P.A
    return (torch.from_numpy(A.indptr).to(d), torch.from_numpy(A.indices).to(d),
            torch.from_numpy(A.data).to(d), torch.from_numpy(np.ascontiguousarray(P.B.T)).to(d))


def _cpu_res(P, X):
    x = X.cpu().numpy().T
    return np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0)


@pytest.mark.parametrize("precision,eps", [(0, 1e-8), (1, 5e-7)])
def test_graph_step_matches_plain_calls(precision, eps):
    from paper_2408_14193_gb300 import Factor, NestedDissection
    from paper_2408_14193_gb300.spalu import kernel_launches
    n = 255
    P = W.make_problem("diffusion", n, seed=71, nrhs=5)
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(n)
    f = Factor(nd, eps_id=eps, symmetric=1, precision=precision)
    f.factor(rp, ci, va)
    Xp = f.solve(B)
    itp, _ = f.refine(B, Xp)
    g = Factor(nd, eps_id=eps, symmetric=1, precision=precision)
    X = torch.empty_like(B)
    for call in range(3):                      # plain + capture, then two replays
        X.zero_()
        l0 = kernel_launches()
        it, rel = g.factor_solve_graph(rp, ci, va, B, X)
        launched = kernel_launches() - l0
        res = _cpu_res(P, X)
        assert np.all(res <= 1e-10), (call, res)
        assert np.allclose(rel, res, rtol=1e-3, atol=1e-13)
        assert abs(it - itp) <= 1, (call, it, itp)
        assert launched > 50
    sg = g.stats()["step_graph"]
    assert sg["captures"] == 1 and sg["replays"] == 2 and sg["refits"] == 0, sg
    # the refined solutions agree to the refinement's accuracy
    d = (X - Xp).cpu().numpy()
    assert np.linalg.norm(d) <= 1e-8 * np.linalg.norm(Xp.cpu().numpy())


def test_graph_replay_follows_new_values_and_falls_back():
    """New values in the same buffers are factored inside the graph; a matrix whose factor
    outgrows the captured capacities (a Laplace capture, then a high-contrast field) still
    gets the right answer through the fallback, and so do later calls."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    n = 127
    Pl = W.make_problem("laplace", n, seed=72, nrhs=2)
    Pd = W.make_problem("diffusion", n, seed=73, nrhs=2)
    Pd.B = Pl.B                                  # same right-hand sides in the same buffer
    rp, ci, va, B = _dev(Pl)
    f = Factor(NestedDissection(n), eps_id=1e-8, symmetric=1)
    X = torch.empty_like(B)
    f.factor_solve_graph(rp, ci, va, B, X)          # plain + capture on the Laplace matrix
    f.factor_solve_graph(rp, ci, va, B, X)          # replay
    assert np.all(_cpu_res(Pl, X) <= 1e-10)
    for P in (Pd, Pl, Pd):
        va.copy_(torch.from_numpy(P.A.data).cuda())
        X.zero_()
        f.factor_solve_graph(rp, ci, va, B, X)
        assert np.all(_cpu_res(P, X) <= 1e-10)


def test_graph_continues_when_one_cycle_is_not_enough():
    """A loose eps_ID needs more Arnoldi steps than the graph holds: the rest runs outside."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    n = 127
    P = W.make_problem("convdiff", n, seed=74, nrhs=3)
    rp, ci, va, B = _dev(P)
    f = Factor(NestedDissection(n), eps_id=1e-2, symmetric=0, precision=1, gmres_m=6)
    X = torch.empty_like(B)
    for _ in range(3):
        X.zero_()
        it, rel = f.factor_solve_graph(rp, ci, va, B, X)
        assert np.all(_cpu_res(P, X) <= 1e-10) and it >= 4


def test_graph_rejects_aliasing():
    from paper_2408_14193_gb300 import Factor, NestedDissection, SpaluError
    P = W.make_problem("laplace", 31, seed=75, nrhs=1)
    rp, ci, va, B = _dev(P)
    f = Factor(NestedDissection(31), eps_id=1e-8, symmetric=1)
    with pytest.raises(SpaluError):
        f.factor_solve_graph(rp, ci, va, B, B)
