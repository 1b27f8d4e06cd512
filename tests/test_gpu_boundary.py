"""GPU tests of the boundary options of include/sap.h that change what a call
does: the spin limit of the bounded device waits, P = 0 (autotuned partition
count), the phase timers of sap_info_t, and the host-buffer solve."""
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


def make(N, K, d, seed):
    band = G.dense_banded(N, K, d, seed)
    xt = G.x_true(N, seed)
    return band, xt, O.spmv(band, N, K, xt)


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_spin_limit_takes_effect(sap):
    """spin_limit = 1: a bounded wait that polls once gives up on a copy that
    has not landed yet, stops further copies, drains those in flight, and the
    call reports SAP_ERR_TIMEOUT (the factorisation when the block LU's wait
    gave up, else the solve).  Whether one poll comes too early is a matter
    of timing; on a wide band (K = 300, 45 KB of sweep matrices per 32-row
    chunk, 2 chunks prefetched) the sweeps' first poll precedes the landing,
    so the test asks for a timeout in one of three attempts, and every attempt
    must end with TIMEOUT or a clean status.  A handle with a large limit
    (clamped to 2^31 - 1) on the same context then solves to the usual
    tolerances, and so does the default (0)."""
    import ctypes
    N, K, P = 40000, 300, 4
    band, xt, b = make(N, K, 1.0, 911)
    bd, bdev = dev(band), dev(b)
    seen = []
    for attempt in range(3):
        opts = sap.sap_default_options(P=P, variant=sap.SAP_D, precision=sap.SAP_FP32, spin_limit=1, max_iters=3)
        hp = ctypes.c_void_p()
        st = sap._lib.sap_factor(bd.data_ptr(), N, K, ctypes.byref(opts),
                                 torch.cuda.current_stream().cuda_stream, ctypes.byref(hp))
        if st == sap.SAP_OK:
            h1 = sap.Handle(hp.value, bd, N, K, opts)
            _, _, st = sap.sap_solve(h1, bdev, raise_on_error=False)
            del h1
        torch.cuda.synchronize()
        seen.append(st)
        assert st in (sap.SAP_ERR_TIMEOUT, sap.SAP_OK, sap.SAP_ERR_NOT_CONVERGED), seen
        if st == sap.SAP_ERR_TIMEOUT:
            break
    assert sap.SAP_ERR_TIMEOUT in seen, seen
    xo, _, _ = O.solve(band, N, K, b, P, O.SAP_D)
    for lim in (1 << 40, 0):
        h = sap.sap_factor(bd, N, K, P=P, variant=sap.SAP_D, precision=sap.SAP_FP32, spin_limit=lim)
        x, info, st = sap.sap_solve(h, bdev)
        assert st == sap.SAP_OK and info.relres <= 1e-10
        assert relerr(host(x), xo) <= 1e-8


@pytest.mark.parametrize("var,prec", [(0, 1), (1, 1), (0, 0)])
def test_P0_runs_the_autotuner(sap, var, prec):
    """P = 0 in sap_factor picks P by measurement among the autotuner's
    default candidates; the handle reports it and solves like the oracle with
    that P."""
    N, K = 60000, 16
    band, xt, b = make(N, K, 1.0, 912 + var)
    h = sap.sap_factor(dev(band), N, K, P=0, variant=var, precision=prec)
    P = sap.sap_num_partitions(h)
    pmax = N // (2 * K) if var == sap.SAP_C else N // 64
    cands = {max(1, min(pmax, (N + r // 2) // r)) for r in (16000, 8000, 4000, 2000, 1000)}
    cands |= {p for p in (152, 304) if p <= pmax}
    assert P in cands
    assert len(sap.sap_get_partition(h)) == P + 1
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK and info.P == P and info.relres <= 1e-10
    xo, io, _ = O.solve(band, N, K, b, P, var)
    assert relerr(host(x), xo) <= 1e-8


@pytest.mark.parametrize("K,fused", [(20, True), (150, False)])
def test_phase_timers(sap, K, fused):
    """sap_info_t's paper timers (Sec. 4.3.2 breakdown): T_BC is 0 (B_i, C_{i+1}
    are read in place), T_LUrdcd is measured where the reduced systems have
    kernels of their own (wide bands) and 0 where the tip kernel forms them,
    T_Kry equals the Krylov phase time."""
    N, P = 12 * K * 10, 10
    band, xt, b = make(N, K, 1.0, 913)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_C, precision=sap.SAP_FP32)
    x, info, st = sap.sap_solve(h, dev(b))
    assert st == sap.SAP_OK
    assert info.t_bc_ms == 0.0
    assert info.t_kry_ms == info.t_solve_ms > 0.0
    assert info.t_lu_ms > 0.0 and info.t_spk_ms > 0.0
    if fused:
        assert info.t_rdcd_ms < 0.05 * info.t_spk_ms
    else:
        assert info.t_rdcd_ms > 0.0
    assert info.t_factor_ms >= info.t_spk_ms + info.t_rdcd_ms - 1e-3
    assert info.n_matvec == round(4 * info.iters)


def test_solve_host_buffers(sap):
    """sap_solve_host: b from (pinned) host memory, x back to host memory,
    the copies inside the call; the result is the device-pointer solve's bit
    for bit and the oracle's to 1e-8."""
    N, K, P = 30000, 12, 6
    band, xt, b = make(N, K, 1.0, 914)
    h = sap.sap_factor(dev(band), N, K, P=P, variant=sap.SAP_C, precision=sap.SAP_FP32)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    xh, info, st = sap.sap_solve_host(h, bh, xh)
    assert st == sap.SAP_OK and info.relres <= 1e-10
    xd, _, _ = sap.sap_solve(h, dev(b))
    np.testing.assert_array_equal(xh.numpy(), host(xd))
    xo, _, _ = O.solve(band, N, K, b, P, O.SAP_C)
    assert relerr(xh.numpy(), xo) <= 1e-8
    # pageable host buffers work too
    xp = torch.empty(N, dtype=torch.float64)
    xp, _, st = sap.sap_solve_host(h, torch.from_numpy(b.copy()), xp)
    assert st == sap.SAP_OK
    np.testing.assert_array_equal(xp.numpy(), host(xd))


@pytest.mark.parametrize("variant", [0, 1])
def test_host_buffer_factor_refactor_and_pair(sap, variant):
    """sap_factor_host / sap_refactor_host / sap_solve_pair_host: the band,
    b and g from host memory and x, lambda back to host memory, the copies
    inside the calls; the results equal the device-pointer calls' bit for bit,
    before and after a refactor with new band values.  A handle whose band is
    borrowed refuses sap_refactor_host."""
    N, K, P = 40000, 20, 8
    band, xt, b = make(N, K, 1.0, 915)
    g = G.adjoint_seed(N, 915)
    bh = torch.from_numpy(band).pin_memory()
    h = sap.sap_factor_host(bh, N, K, P=P, variant=variant, precision=sap.SAP_FP32)
    hd = sap.sap_factor(dev(band), N, K, P=P, variant=variant, precision=sap.SAP_FP32)
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    lh = torch.empty(N, dtype=torch.float64).pin_memory()
    bb = torch.from_numpy(b).pin_memory()
    gg = torch.from_numpy(g).pin_memory()
    for rnd in range(2):
        if rnd == 1:
            band2, _, b2 = make(N, K, 1.05, 916)
            bh.copy_(torch.from_numpy(band2))
            bb.copy_(torch.from_numpy(b2))
            sap.sap_refactor_host(h, bh)
            hd.band.copy_(dev(band2))
            sap.sap_refactor(hd)
        _, _, ix, il, st = sap.sap_solve_pair_host(h, bb, gg, xh, lh)
        assert st == sap.SAP_OK and ix.relres <= 1e-10 and il.relres <= 1e-10
        xd, ld, _, _, st2 = sap.sap_solve_pair(hd, dev(bb.numpy()), dev(g))
        assert st2 == sap.SAP_OK
        np.testing.assert_array_equal(xh.numpy(), host(xd))
        np.testing.assert_array_equal(lh.numpy(), host(ld))
    with pytest.raises(sap.SapError) as e:
        sap.sap_refactor_host(hd, bh)
    assert e.value.status == sap.SAP_ERR_INVALID_ARG
