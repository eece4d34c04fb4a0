"""spalu_residual_noalloc: the residual-norm entry point that allocates no device memory.

It exists for callers that cannot let the library allocate when they check a solution
(hosts that own all device memory through their own pool, processes at the edge of device
memory).  Its result must match the relative residuals spalu_refine reports (computed there
with buffers the library allocates), on two calls in a row.  This file is collected last
so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__ as g
    g.build()
    from paper_2408_14193_gb300 import Factor, NestedDissection
    P = W.make_problem("diffusion", 63, seed=31, nrhs=3)
    d = torch.device("cuda:0")
    rp = torch.from_numpy(P.A.indptr).to(d)
    ci = torch.from_numpy(P.A.indices).to(d)
    va = torch.from_numpy(P.A.data).to(d)
    B = torch.from_numpy(np.ascontiguousarray(P.B.T)).to(d)
    nd = NestedDissection(63)
    # gmres_maxit = 0: spalu_refine only measures the residual of the given X
    f = Factor(nd, eps_id=1e-4, symmetric=1, gmres_maxit=0)
    f.factor(rp, ci, va)
    return P, f, B


def _refine_relres(f, B, X):
    Y = X.clone()
    _, rel = f.refine(B, Y, check=False)
    return rel


def test_noalloc_matches_refine_residual_twice(setup):
    P, f, B = setup
    X = f.solve(B)
    torch.cuda.synchronize()
    ref = _refine_relres(f, B, X)
    r1 = f.residual_noalloc(B, X)                   # first call on this device (set-up)
    free1 = torch.cuda.mem_get_info()[0]
    r2 = f.residual_noalloc(B, X)                   # second call: same answer, no new memory
    free2 = torch.cuda.mem_get_info()[0]
    assert np.allclose(r1, ref, rtol=1e-10, atol=0)
    assert np.array_equal(r1, r2)
    assert free2 == free1
    # a different solution on the next call: the shared scratch carries nothing over
    X2 = X.clone()
    X2[1] *= 1.5
    ref2 = _refine_relres(f, B, X2)
    r3 = f.residual_noalloc(B, X2)
    assert np.allclose(r3, ref2, rtol=1e-10, atol=0)
    assert r3[1] > 1e-3 and abs(r3[0] - r1[0]) <= 1e-10 * r1[0]
    # independent check on the CPU
    x = X.cpu().numpy().T
    cpu = np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0)
    assert np.allclose(r1, cpu, rtol=1e-8)


def test_noalloc_rejects_too_many_columns(setup):
    P, f, _ = setup
    N = P.A.n
    B = torch.zeros((65, N), dtype=torch.float64, device="cuda")
    rel = np.full(65, -1.0)
    st = f.lib.spalu_residual_noalloc(f.handle, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                      65, N, rel.ctypes.data, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1
    assert np.all(rel == -1.0)


def _call(f, Bp, Xp, nrhs, ld):
    rel = np.full(max(nrhs, 1), -1.0)
    st = f.lib.spalu_residual_noalloc(f.handle, ctypes.c_void_p(Bp), ctypes.c_void_p(Xp), nrhs, ld,
                                      rel.ctypes.data, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return rel[:nrhs]


def _cpu_relres(P, Bc, Xc):
    return np.linalg.norm(Bc - P.A.matvec(Xc), axis=0) / np.linalg.norm(Bc, axis=0)


def test_noalloc_padded_leading_dimension(setup):
    """B and X inside a buffer with leading dimension N + 7 (columns start at c (N + 7))."""
    P, f, B = setup
    N = P.A.n
    ld = N + 7
    X = f.solve(B)
    Bpad = torch.full((3, ld), 1e30, dtype=torch.float64, device="cuda")
    Xpad = torch.full((3, ld), 1e30, dtype=torch.float64, device="cuda")
    Bpad[:, :N] = B
    Xpad[:, :N] = X
    Xpad[2, :N] *= 0.5
    torch.cuda.synchronize()
    r = _call(f, Bpad.data_ptr(), Xpad.data_ptr(), 3, ld)
    Xc = Xpad[:, :N].cpu().numpy().T
    assert np.allclose(r, _cpu_relres(P, P.B, Xc), rtol=1e-8)
    assert r[2] > 0.3 and r[0] < 0.1          # half a solution leaves half of B


def test_noalloc_largest_column_count(setup):
    """nrhs = 64, the largest count the fixed array holds, against the CPU residual."""
    P, f, _ = setup
    N = P.A.n
    rng = np.random.default_rng(7)
    Bc = rng.standard_normal((N, 64))
    Xc = rng.standard_normal((N, 64)) * 1e-3
    Bd = torch.from_numpy(np.ascontiguousarray(Bc.T)).cuda()
    Xd = torch.from_numpy(np.ascontiguousarray(Xc.T)).cuda()
    r1 = _call(f, Bd.data_ptr(), Xd.data_ptr(), 64, N)
    r2 = _call(f, Bd.data_ptr(), Xd.data_ptr(), 64, N)
    assert np.allclose(r1, _cpu_relres(P, Bc, Xc), rtol=1e-10)
    assert np.array_equal(r1, r2)
