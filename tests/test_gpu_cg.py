"""GPU parity of the preconditioned conjugate gradient outer iteration
(SAP_KRYLOV_CG: Sec. 3, the outer loop for a symmetric positive definite A)
against the oracle's PCG (Saad, Algorithm 9.1), all through the C ABI.

Iterates: with FP64 factors the GPU iterate after k CG steps equals the
oracle's to 1e-10 (relative; the same recurrences, different summation
orders in the sweeps and reductions).  Solutions: relres <= 1e-10 and the
oracle's solution within 1e-8 for both variants and both factor precisions;
for the symmetric A the adjoint solve is the same system; sap_solve_pair
runs the two CG solves concurrently and returns what the separate calls
return, bit for bit; batches of SPD systems run CG per system."""
import numpy as np
import pytest
import torch

import oracle as O
import sap_inputs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_07919_gb300 as S
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_cg_iterates_match_oracle(sap):
    N, K, P = 4000, 8, 4
    band = G.dense_banded_spd(N, K, 1.0, 2101)
    b = O.spmv(band, N, K, G.x_true(N, 2101))
    o = O.Sap(band, N, K, P, O.SAP_D)
    for k in (1, 2, 5):
        h = sap.sap_factor(dev(band), N, K, P=P, precision=sap.SAP_FP64, krylov=sap.SAP_KRYLOV_CG,
                           max_iters=k, tol=1e-30)
        x, info, st = sap.sap_solve(h, dev(b), raise_on_error=False)
        assert st == sap.SAP_ERR_NOT_CONVERGED and info.iters == k and info.n_matvec == k
        xo, io = o.solve_cg(b, tol=0.0, max_iters=k)
        assert io.iters == k
        assert relerr(host(x), xo) <= 1e-10, (k, relerr(host(x), xo))
        assert abs(info.relres - io.relres) <= 1e-4 * io.relres


@pytest.mark.parametrize("variant,prec", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_cg_solution_adjoint_and_pair_match_oracle(sap, variant, prec):
    N, K, P = 20000, 20, 8
    band = G.dense_banded_spd(N, K, 1.0, 2102)
    xt = G.x_true(N, 2102)
    b = O.spmv(band, N, K, xt)
    xo, io, _ = O.solve_cg(band, N, K, b, P, variant)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=prec, krylov=sap.SAP_KRYLOV_CG)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10 and info.graphed == 1
    assert info.iters == int(info.iters)
    assert relerr(host(x), xo) <= 1e-8 and relerr(host(x), xt) <= 1e-8
    g = G.adjoint_seed(N, 2102)
    lo, _, _ = O.solve_cg(band, N, K, g, P, variant)
    lam, ai, ast = sap.sap_solve_adjoint(h, dev(g))
    assert ast == sap.SAP_OK and ai.relres <= 1e-10 and relerr(host(lam), lo) <= 1e-8
    x2, l2, ix, il, st2 = sap.sap_solve_pair(h, dev(b), dev(g))
    assert st2 == sap.SAP_OK and ix.relres <= 1e-10 and il.relres <= 1e-10
    np.testing.assert_array_equal(host(x2), host(x))
    np.testing.assert_array_equal(host(l2), host(lam))


def test_cg_full_size_spd_n200k_k50_p50(sap):
    """The C2 sizes with the SPD band: FP32 factors, SaP-D."""
    N, K, P = 200000, 50, 50
    band = G.dense_banded_spd(N, K, 1.0, 2103)
    xt = G.x_true(N, 2103)
    b = O.spmv(band, N, K, xt)
    h = sap.sap_factor(dev(band), N, K, P=P, precision=sap.SAP_FP32, krylov=sap.SAP_KRYLOV_CG)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.relres <= 1e-10
    xo, io, _ = O.solve_cg(band, N, K, b, P, O.SAP_D)
    assert relerr(host(x), xo) <= 1e-8 and relerr(host(x), xt) <= 1e-8
    assert abs(info.iters - io.iters) <= 2


def test_cg_options(sap):
    N, K = 2000, 4
    band = G.dense_banded_spd(N, K, 1.0, 2104)
    with pytest.raises(sap.SapError) as e:
        sap.sap_factor(dev(band), N, K, P=2, krylov=2)
    assert e.value.status == sap.SAP_ERR_INVALID_ARG
    assert sap.sap_default_options().krylov == sap.SAP_KRYLOV_BICGSTAB2


def test_cg_restart_and_iteration_cap_on_the_device(sap):
    """A tolerance below rounding: the recursive residual passes, the true one
    cannot, so every passing step restarts from x (counted in n_restarts) until
    the device stops the solve at the iteration cap, in a round that ends
    early; the oracle does the same and its iterate matches.  SaP-D's M^{-1} A
    is the identity plus a term of rank <= 2K(P-1) = 24, so CG reaches rounding
    level within about 25 steps and the caps lie beyond that."""
    N, K, P = 3000, 6, 3
    band = G.dense_banded_spd(N, K, 1.0, 2106)
    b = O.spmv(band, N, K, G.x_true(N, 2106))
    for cap in (37, 38):
        h = sap.sap_factor(dev(band), N, K, P=P, precision=sap.SAP_FP64, krylov=sap.SAP_KRYLOV_CG,
                           max_iters=cap, tol=1e-17)
        x, info, st = sap.sap_solve(h, dev(b), raise_on_error=False)
        xo, io = O.Sap(band, N, K, P, O.SAP_D).solve_cg(b, tol=1e-17, max_iters=cap)
        assert st == sap.SAP_ERR_NOT_CONVERGED == io.status and info.iters == cap == io.iters
        assert info.n_restarts >= 1 and io.n_restarts >= 1
        assert info.relres <= 1e-14 and relerr(host(x), xo) <= 1e-12


def test_cg_batch_of_spd_systems(sap):
    """SPD systems of uneven N and K through the batched calls with CG, every
    system against the oracle's CG with the same partition count."""
    specs = [(3000, 5, 2111), (7000, 12, 2112), (5000, 30, 2113)]
    bands = [G.dense_banded_spd(N, K, 1.0, sd) for N, K, sd in specs]
    bs = [O.spmv(bd, N, K, G.x_true(N, sd)) for bd, (N, K, sd) in zip(bands, specs)]
    bh = sap.sap_factor_batched([dev(b) for b in bands], [s[0] for s in specs], [s[1] for s in specs],
                                precision=sap.SAP_FP32, krylov=sap.SAP_KRYLOV_CG)
    Ps = sap.sap_batch_partitions(bh)
    xs, infos, stats, st = sap.sap_solve_batched(bh, [dev(b) for b in bs])
    assert st == sap.SAP_OK
    for i, (N, K, _) in enumerate(specs):
        assert infos[i].relres <= 1e-10 and infos[i].iters == int(infos[i].iters)
        xo, io, _ = O.solve_cg(bands[i], N, K, bs[i], Ps[i], O.SAP_D)
        assert relerr(host(xs[i]), xo) <= 1e-8
