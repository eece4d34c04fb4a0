"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

Bars: integer tables (ND order, segment node lists) bit-exact; FP64 solutions within a
relative 1e-6 of the oracle's at eps_ID = 1e-8 (skeleton choices may differ at pivot
ties); eps_ID = 0 (exact block LU) within 1e-11 of a dense solve; refinement to a relative
residual <= 1e-10 checked by a CPU residual.
"""
import numpy as np
import pytest

import workloads as W
from oracle.nd import nested_dissection, _sides
from parity import assert_close, rel_errors
from oracle.spalu import Options as OOpts, factor as ofactor, solve as osolve

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


def _gpu_solve(P, eps, nx=None, ny=None, refine=False, symmetric=None):
    from paper_2408_14193_gb300 import Factor, NestedDissection
    nx = nx or P.nx
    ny = ny or P.ny
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(nx, ny)
    sym = P.symmetric if symmetric is None else symmetric
    f = Factor(nd, eps_id=eps, symmetric=1 if sym else 0)
    f.factor(rp, ci, va)
    X = f.solve(B)
    info = None
    if refine:
        info = f.refine(B, X)
    torch.cuda.synchronize()
    return X.cpu().numpy().T, f, info


# ------------------------------------------------------------------ ND tables, bit-exact
@pytest.mark.parametrize("nx,ny", [(15, 15), (31, 31), (63, 63), (127, 31), (31, 127), (255, 255),
                                   (1023, 1023)])
def test_nd_order_bit_exact(nx, ny):
    from paper_2408_14193_gb300 import NestedDissection
    nd = NestedDissection(nx, ny)
    perm, iperm, L, table = nd.export()
    ond = nested_dissection(nx, ny)
    assert L == ond.L
    assert np.array_equal(perm.astype(np.int64), ond.perm)
    assert np.array_equal(iperm[perm], np.arange(nx * ny))
    for l in range(1, L + 1):
        lev = ond.levels[l]
        bx, by, w, h, vc, nseg, ncor, nsep = table[l - 1]
        assert (w, h) == (lev.boxes[0].w, lev.boxes[0].h)
        assert nseg == len(lev.segments) and ncor == len(lev.corners) and nsep == len(lev.separators)
    if L:
        segs = nd.finest_segments(int(table[L - 1][5]))
        for s in ond.levels[L].segments.values():
            assert np.array_equal(segs[s.sid].astype(np.int64), s.nodes)


# ------------------------------------------------------------------ exact special case
@pytest.mark.parametrize("kind,n", [("laplace", 15), ("diffusion", 31), ("convdiff", 31),
                                    ("helmholtz", 63), ("diffusion", 63)])
def test_eps0_equals_dense_solve(kind, n):
    P = W.make_problem(kind, n, seed=21, nrhs=3)
    X, _, _ = _gpu_solve(P, 0.0)
    Xd = np.linalg.solve(P.A.to_dense(), P.B)
    assert_close(X, Xd, 1e-11, f"{kind} {n} eps 0")


# ------------------------------------------------------------------ FP64 parity with the oracle
@pytest.mark.parametrize("kind,n,nrhs", [("laplace", 127, 1), ("diffusion", 127, 4),
                                         ("convdiff", 127, 2), ("diffusion", 255, 2),
                                         ("helmholtz", 63, 2), ("aniso", 127, 2)])
def test_fp64_matches_oracle(kind, n, nrhs):
    P = W.make_problem(kind, n, seed=22, nrhs=nrhs)
    X, f, _ = _gpu_solve(P, 1e-8)
    F = ofactor(P.A, nested_dissection(n, n), OOpts(eps=1e-8, symmetric=P.symmetric))
    Xo = osolve(F, P.B)
    assert_close(X, Xo, 1e-6, f"{kind} {n}")
    # rank statistics agree level by level (pivot ties may move a rank by one)
    st = f.stats()
    for lv in st["levels"]:
        o = F.stats["levels"][lv["level"]]
        assert lv["e_max"] == o["e_max"] or abs(lv["e_max"] - o["e_max"]) <= 2
        assert abs(lv["k_max"] - o["k_max"]) <= 2


@pytest.mark.parametrize("kind", ["diffusion", "convdiff"])
def test_pure_randomized_sampling_matches_oracle(kind):
    """near_radius = -1: no near field, every neighbour row is sketched (Sec. 4.2.1), against
    the oracle in the same mode."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    n = 127
    P = W.make_problem(kind, n, seed=36, nrhs=2)
    rp, ci, va, B = _dev(P)
    f = Factor(NestedDissection(n), eps_id=1e-8, symmetric=1 if P.symmetric else 0, near_radius=-1)
    f.factor(rp, ci, va)
    X = f.solve(B).cpu().numpy().T
    F = ofactor(P.A, nested_dissection(n, n), OOpts(eps=1e-8, symmetric=P.symmetric, near_radius=-1))
    assert_close(X, osolve(F, P.B), 1e-6, f"pure randomized {kind}")
    for lv in f.stats()["levels"]:
        o = F.stats["levels"][lv["level"]]
        assert abs(lv["k_max"] - o["k_max"]) <= 2


@pytest.mark.parametrize("nx,ny", [(127, 31), (31, 63)])
def test_rectangular_grids(nx, ny):
    P = W.make_problem("diffusion", nx, seed=23, nrhs=2, ny=ny)
    X, _, _ = _gpu_solve(P, 1e-8, nx=nx, ny=ny)
    Xo = osolve(ofactor(P.A, nested_dissection(nx, ny), OOpts(eps=1e-8, symmetric=True)), P.B)
    assert_close(X, Xo, 1e-6, f"{nx}x{ny}")


def test_nonsymmetric_flag_on_symmetric_matrix():
    """Stacked ID on a symmetric matrix gives the same solution as the symmetric ID."""
    P = W.make_problem("diffusion", 63, seed=24, nrhs=1)
    X1, _, _ = _gpu_solve(P, 1e-8, symmetric=True)
    X2, _, _ = _gpu_solve(P, 1e-8, symmetric=False)
    Xd = np.linalg.solve(P.A.to_dense(), P.B)
    for X in (X1, X2):
        assert_close(X, Xd, 1e-5)


# ------------------------------------------------------------------ refinement
@pytest.mark.parametrize("kind,n,eps", [("diffusion", 127, 1e-6), ("convdiff", 127, 1e-6),
                                        ("helmholtz", 127, 1e-8)])
def test_refine_reaches_tolerance(kind, n, eps):
    P = W.make_problem(kind, n, seed=25, nrhs=3)
    X, f, (it, rel) = _gpu_solve(P, eps, refine=True)
    res = np.linalg.norm(P.B - P.A.matvec(X), axis=0) / np.linalg.norm(P.B, axis=0)
    assert np.all(res <= 1e-10), res
    assert np.all(rel <= 1e-10)
    assert it >= 1


# ------------------------------------------------------------------ API edge cases
def test_solve_aliasing_and_host_entry_points():
    from paper_2408_14193_gb300 import Factor, NestedDissection
    P = W.make_problem("laplace", 63, seed=26, nrhs=2)
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(63)
    f = Factor(nd, eps_id=1e-8, symmetric=1)
    f.factor(rp, ci, va)
    X = f.solve(B)
    Y = B.clone()
    f.solve(Y, Y)                                   # X may alias B
    torch.cuda.synchronize()
    # separator updates of shared boundary unknowns are atomic additions, so two solves agree
    # to rounding, not bit for bit
    assert torch.linalg.norm(X - Y) <= 1e-12 * torch.linalg.norm(X)
    g = Factor(nd, eps_id=1e-8, symmetric=1)
    g.factor_host(P.A.indptr, P.A.indices, P.A.data)
    Xh, it, rel = g.solve_host(np.ascontiguousarray(P.B.T), refine=True)
    res = np.linalg.norm(P.B - P.A.matvec(Xh.T), axis=0) / np.linalg.norm(P.B, axis=0)
    assert np.all(res <= 1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_factor_solve_host_matches_separate_calls(precision):
    """spalu_factor_solve_host (B uploaded on a second stream during the factorization, device
    buffers kept by the handle) gives what spalu_factor_numeric_host + spalu_solve_host give:
    the direct solve to rounding (atomic separator updates), the refined one to 1e-10; repeated
    calls with more right-hand sides grow the buffers; no right-hand sides only factors."""
    from paper_2408_14193_gb300 import Factor, NestedDissection, SpaluError
    n = 127
    P = W.make_problem("diffusion", n, seed=45, nrhs=3)
    nd = NestedDissection(n)
    eps = 1e-8 if precision == 0 else 1e-6
    Bh = np.ascontiguousarray(P.B.T)
    g = Factor(nd, eps_id=eps, symmetric=1, precision=precision)
    g.factor_host(P.A.indptr, P.A.indices, P.A.data)
    X0, _, _ = g.solve_host(Bh)
    f = Factor(nd, eps_id=eps, symmetric=1, precision=precision)
    X1, _, _ = f.factor_solve_host(P.A.indptr, P.A.indices, P.A.data, Bh[:1])
    X2, _, _ = f.factor_solve_host(P.A.indptr, P.A.indices, P.A.data, Bh)
    tol = 1e-12 if precision == 0 else 1e-3      # mixed: FP32 atomic order
    assert np.linalg.norm(X2 - X0) <= tol * np.linalg.norm(X0)
    assert np.linalg.norm(X1 - X0[:1]) <= tol * np.linalg.norm(X0[:1])
    X3, it, rel = f.factor_solve_host(P.A.indptr, P.A.indices, P.A.data, Bh, refine=True)
    res = np.linalg.norm(P.B - P.A.matvec(X3.T), axis=0) / np.linalg.norm(P.B, axis=0)
    assert it >= 1 and np.all(res <= 1e-10) and np.allclose(rel, res, rtol=1e-3, atol=1e-13)
    X4, _, _ = f.factor_solve_host(P.A.indptr, P.A.indices, P.A.data, np.zeros((0, n * n)))
    assert X4.shape == (0, n * n)
    with pytest.raises(SpaluError):                 # nnz above the handle's capacity
        f.factor_solve_host(P.A.indptr, np.zeros(6 * n * n, np.int32), np.zeros(6 * n * n), Bh)
    with pytest.raises(ValueError):                 # a short right-hand side is refused before the call
        f.factor_solve_host(P.A.indptr, P.A.indices, P.A.data, Bh[:, :-1])


def test_errors_are_reported_not_raised_on_device():
    from paper_2408_14193_gb300 import Factor, NestedDissection, SpaluError
    nd = NestedDissection(31)
    f = Factor(nd, eps_id=1e-8)
    B = torch.zeros(31 * 31, dtype=torch.float64, device="cuda")
    with pytest.raises(SpaluError):
        f.solve(B)                                 # not factored yet -> state error
    # a zero row makes a leaf interior block singular
    P = W.make_problem("laplace", 31, seed=27)
    A = P.A
    val = A.data.copy()
    r = 5 + 31 * 5
    val[A.indptr[r]:A.indptr[r + 1]] = 0.0
    rp, ci, _, _ = _dev(P)
    with pytest.raises(SpaluError) as e:
        f.factor(rp, ci, torch.from_numpy(val).cuda())
    assert e.value.status == -3


def test_full_size_diffusion_1023_refined():
    """The 1023 x 1023 variable-coefficient problem (16 RHS) at full size: ND order
    bit-exact (above) and the refined residual checked on the CPU."""
    P = W.make_problem("diffusion", 1023, seed=1, nrhs=16)
    X, f, (it, rel) = _gpu_solve(P, 1e-8, refine=True)
    res = np.linalg.norm(P.B - P.A.matvec(X), axis=0) / np.linalg.norm(P.B, axis=0)
    assert np.all(res <= 1e-10), res
    st = f.stats()
    assert st["L"] == 12 and st["q_tilde"] <= 1.0


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("kind,n,eps", [("diffusion", 127, 1e-6), ("diffusion", 255, 1e-6),
                                        ("convdiff", 127, 1e-6), ("laplace", 127, 1e-6),
                                        ("helmholtz", 63, 1e-6), ("aniso", 127, 1e-6)])
def test_mixed_precision_refined(kind, n, eps):
    """Mixed mode (FP32 factors / solve, FP64 leaf LU, FP64 QR pivots and norms) refined by
    GMRES with an FP64 residual to 1e-10; the direct solve's error against the FP64 oracle
    at the same tolerance is stated (printed) and bounded."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    P = W.make_problem(kind, n, seed=28, nrhs=2)
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(n)
    f = Factor(nd, eps_id=eps, symmetric=1 if P.symmetric else 0, precision=1)
    f.factor(rp, ci, va)
    X = f.solve(B)
    torch.cuda.synchronize()
    x0 = X.cpu().numpy().T
    Xo = osolve(ofactor(P.A, nested_dissection(n, n), OOpts(eps=eps, symmetric=P.symmetric)), P.B)
    err_n, err = rel_errors(x0, Xo)
    print(f"mixed {kind} {n}: direct-solve error vs FP64 oracle {err_n:.2e} (norm-wise), "
          f"{err:.2e} (entry-wise)")
    # FP32 factors: forward error ~ cond x 6e-8.  The k^2-shifted Helmholtz operator is
    # indefinite and far worse conditioned than the others: over seeds 28-30 its 63^2 direct
    # solve lands anywhere in 5e-4..2e-2, so it gets a wider bound; the refinement to 1e-10
    # below is the requirement either way.
    assert err <= (1e-1 if kind == "helmholtz" else 1e-2)
    it, rel = f.refine(B, X)
    torch.cuda.synchronize()
    x = X.cpu().numpy().T
    res = np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0)
    assert np.all(res <= 1e-10), res


@pytest.mark.parametrize("kind,n,nrhs", [("diffusion", 255, 16), ("helmholtz", 127, 3), ("convdiff", 127, 16)])
def test_leaf_backward_forms(kind, n, nrhs):
    """The two forms of the mixed backward leaf step x_I -= A_II^{-1} A_Id x_d (Eq. (WV)):
    leaf_bwd = 0 (one product with the stored G = A_II^{-1} A_Id) and leaf_bwd = 1 (a band
    sweep pair on the stored factors with the coupling table; the interchange variant on the
    Helmholtz leaves, idle lanes with 3 right-hand sides) agree to FP32 rounding on the same
    factorization, both refine to 1e-10, and on the definite operators both meet the mixed bar
    against the FP64 oracle."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    P = W.make_problem(kind, n, seed=41, nrhs=nrhs)
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(n)
    sym = 1 if P.symmetric else 0
    xs, fs = [], []
    for form in (0, 1):
        f = Factor(nd, eps_id=1e-6, symmetric=sym, precision=1, leaf_bwd=form)
        f.factor(rp, ci, va)
        xs.append(f.solve(B).cpu().numpy().T)
        fs.append(f)
    nrm, ent = rel_errors(xs[1], xs[0])
    print(f"{kind} {n}: sweeps vs G: {nrm:.2e} (norm-wise), {ent:.2e} (entry-wise)")
    assert nrm <= (1e-3 if kind == "helmholtz" else 1e-4) and ent <= (1e-2 if kind == "helmholtz" else 1e-3)
    if kind != "helmholtz":
        # the FP32 direct solve of the indefinite Helmholtz operator at 127^2 lands anywhere
        # near 0.1 of the FP64 oracle (run to run); its requirement is the refinement below
        Xo = osolve(ofactor(P.A, nested_dissection(n, n), OOpts(eps=1e-6, symmetric=P.symmetric)), P.B)
        for x in xs:
            assert rel_errors(x, Xo)[0] <= 1e-2
    for f in fs:
        X = f.solve(B)
        f.refine(B, X)
        x = X.cpu().numpy().T
        res = np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0)
        assert np.all(res <= 1e-10), res


@pytest.mark.parametrize("kind,n,which", [("diffusion", 255, "schur_tc"), ("convdiff", 127, "schur_tc"),
                                          ("diffusion", 255, "sketch_tc"), ("convdiff", 127, "sketch_tc")])
def test_contractions_on_tensor_cores(kind, n, which):
    """schur_tc / sketch_tc = 1: the separators' Schur updates / the sketch products on the
    tensor cores (3xTF32 mma.sync) give the FP32 CUDA-core result to FP32 rounding (through the
    factorization: the skeleton choices may move), the mixed bar against the FP64 oracle, and
    the refinement to 1e-10."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    P = W.make_problem(kind, n, seed=37, nrhs=2)
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(n)
    sym = 1 if P.symmetric else 0
    out = []
    for tc in (0, 1):
        kw = {"schur_tc": 0, "sketch_tc": 0}
        kw[which] = tc
        f = Factor(nd, eps_id=1e-6, symmetric=sym, precision=1, **kw)
        f.factor(rp, ci, va)
        out.append((f, f.solve(B).cpu().numpy().T))
    nrm, ent = rel_errors(out[1][1], out[0][1])
    print(f"{kind} {n} {which}: tensor cores vs CUDA cores: {nrm:.2e} (norm-wise), {ent:.2e} (entry-wise)")
    assert nrm <= 1e-3
    Xo = osolve(ofactor(P.A, nested_dissection(n, n), OOpts(eps=1e-6, symmetric=P.symmetric)), P.B)
    assert rel_errors(out[1][1], Xo)[0] <= 1e-2
    f = out[1][0]
    X = f.solve(B)
    f.refine(B, X)
    x = X.cpu().numpy().T
    res = np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0)
    assert np.all(res <= 1e-10), res


# ------------------------------------------------------------------ right-hand-side chunks
@pytest.mark.parametrize("nrhs", [17, 20])
def test_many_rhs_ragged_chunks(nrhs):
    """More right-hand sides than one solve chunk (16) and one GMRES vector chunk (8), with a
    ragged last chunk: the FP64 form against the oracle, the mixed form refined to 1e-10."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    n = 63
    P = W.make_problem("diffusion", n, seed=41, nrhs=nrhs)
    X, _, _ = _gpu_solve(P, 1e-8)
    Xo = osolve(ofactor(P.A, nested_dissection(n, n), OOpts(eps=1e-8, symmetric=True)), P.B)
    assert_close(X, Xo, 1e-6, f"{nrhs} RHS")
    rp, ci, va, B = _dev(P)
    f = Factor(NestedDissection(n), eps_id=1e-6, symmetric=1, precision=1)
    f.factor(rp, ci, va)
    Xm = f.solve(B)
    it, rel = f.refine(B, Xm)
    x = Xm.cpu().numpy().T
    res = np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0)
    assert res.shape == (nrhs,) and np.all(res <= 1e-10), res
    # every column solved as if alone: column 17 of the batch against a one-column solve
    c = nrhs - 1
    g = Factor(NestedDissection(n), eps_id=1e-8, symmetric=1)
    g.factor(rp, ci, va)
    Y = g.solve(B[c:c + 1].contiguous())
    torch.cuda.synchronize()
    assert np.linalg.norm(Y.cpu().numpy()[0] - X[:, c]) <= 1e-12 * np.linalg.norm(X[:, c])


def test_zero_rhs_is_a_no_op():
    from paper_2408_14193_gb300 import Factor, NestedDissection
    P = W.make_problem("diffusion", 31, seed=42, nrhs=1)
    rp, ci, va, _ = _dev(P)
    f = Factor(NestedDissection(31), eps_id=1e-8, symmetric=1)
    f.factor(rp, ci, va)
    lib = f.lib
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    import ctypes
    st = lib.spalu_solve(f.handle, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), 0,
                         f.N, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_solve_matches_default(precision):
    """spalu_tune_solve only changes CTA widths and right-hand-side groups of the level solves:
    same solution (up to the order of the atomic separator updates), kept across a
    re-factorization."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    n = 255
    P = W.make_problem("diffusion", n, seed=43, nrhs=4)
    rp, ci, va, B = _dev(P)
    f = Factor(NestedDissection(n), eps_id=1e-8, symmetric=1, precision=precision)
    f.factor(rp, ci, va)
    X0 = f.solve(B)
    f.tune_solve(4)
    X1 = f.solve(B)
    f.factor(rp, ci, va)
    X2 = f.solve(B)
    torch.cuda.synchronize()
    tol = 1e-12 if precision == 0 else 1e-3
    for X in (X1, X2):
        assert torch.linalg.norm(X - X0) <= tol * torch.linalg.norm(X0)


@pytest.mark.parametrize("precision", [0, 1])
def test_sparsify_budgets_and_tuning_match_oracle(precision):
    """The sparsify kernel's shared-memory budget (spars_ctas, and the per-level choice of
    spalu_tune_factor) only moves segments between shared and global scratch: under every
    budget, including ones that push the finest level's sketch into global memory, the FP64
    form stays within the oracle parity bar and the mixed form within its FP32 bound; the
    tuned choice is kept across a re-factorization."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    n = 255
    eps = 1e-8 if precision == 0 else 1e-6
    P = W.make_problem("diffusion", n, seed=44, nrhs=2)
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(n)
    Xo = osolve(ofactor(P.A, nested_dissection(n, n), OOpts(eps=eps, symmetric=True)), P.B)
    bar = 1e-6 if precision == 0 else 1e-2

    def err(f):
        x = f.solve(B).cpu().numpy().T
        return max(rel_errors(x, Xo))

    for ctas in (0, 4, 12, 16):
        f = Factor(nd, eps_id=eps, symmetric=1, precision=precision, spars_ctas=ctas)
        f.factor(rp, ci, va)
        assert err(f) <= bar, ctas
        if ctas == 4:
            f.set_timing(True)
            f.factor(rp, ci, va)
            before = f.stats()["timing_ms"]
            f.tune_factor()
            assert f.stats()["timing_ms"] == before        # the tuner leaves the timings alone
            f.set_timing(False)
            assert err(f) <= bar
            f.factor(rp, ci, va)
            assert err(f) <= bar


def test_ranks_do_not_depend_on_the_sparsify_budget():
    """The sketch is summed in blocks of 16 far unknowns whatever chunk the shared-memory
    budget allows (and the pivoted QR is the same in shared or global memory), so the mixed
    factorization takes the same skeletons under every budget: identical per-level ranks, and
    solutions equal up to the run-dependent order of the solve's separator atomics."""
    from paper_2408_14193_gb300 import Factor, NestedDissection
    n = 255
    P = W.make_problem("diffusion", n, seed=45, nrhs=2)
    rp, ci, va, B = _dev(P)
    nd = NestedDissection(n)
    ranks, xs = [], []
    for ctas in (0, 2, 4, 12):
        f = Factor(nd, eps_id=5e-7, symmetric=1, precision=1, spars_ctas=ctas)
        f.factor(rp, ci, va)
        ranks.append([(lv["k_sum"], lv["k_max"], lv["passes"]) for lv in f.stats()["levels"]])
        xs.append(f.solve(B).cpu().numpy().T)
    for r, x in zip(ranks[1:], xs[1:]):
        assert r == ranks[0]
        assert rel_errors(x, xs[0])[0] <= 1e-5


def test_bad_sparsify_budget_is_rejected():
    from paper_2408_14193_gb300 import Factor, NestedDissection, SpaluError
    for ctas in (-1, 33):
        with pytest.raises(SpaluError):
            Factor(NestedDissection(31), eps_id=1e-8, symmetric=1, spars_ctas=ctas)


def test_tune_requires_a_factor():
    from paper_2408_14193_gb300 import Factor, NestedDissection, SpaluError
    f = Factor(NestedDissection(31), eps_id=1e-8, symmetric=1)
    with pytest.raises(SpaluError):
        f.tune_solve(1)
    with pytest.raises(SpaluError):
        f.tune_factor()
