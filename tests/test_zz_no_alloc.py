"""tomo_objective_noalloc: the objective without a plan and without any
device allocation, for callers that cannot allocate device memory where they
need it (memory pools or arenas that own every allocation of the process,
frameworks that forbid allocation and its device synchronisation inside their
hot loop).  Checked through the C ABI against tomo_objective on the same
inputs, on two calls in a row with different problems (the static scratch
keeps the previous call's contents, which must not leak into the next), and
for its size limit.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# both paths evaluate the objective in double (weights differ by ~1e-15)
REL = 1e-12
MAX_ROWS = 262144  # TOMO_NOALLOC_MAX_ROWS of include/tomo.h


@pytest.fixture(scope="module")
def tomo():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_02844_gb300 as t
    from paper_2404_02844_gb300 import build
    build.build()
    t.lib()
    return t


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def noalloc(tomo, M, N, lam_d, band_k, gamma, P_d, Th_d, f_d):
    stream = torch.cuda.current_stream().cuda_stream
    st = tomo.lib().tomo_objective_noalloc(M, N, lam_d.shape[0], lam_d.data_ptr(), band_k, gamma,
                                          P_d.data_ptr(), Th_d.data_ptr(), f_d.data_ptr(),
                                          ctypes.c_void_p(stream))
    assert st == 0, tomo.tomo_last_error()
    torch.cuda.synchronize()
    return float(f_d.item())


def case(M, bins, D, X, gamma, band_k, seed):
    w = workloads.small_case(M=M, bins=bins, D=D, X=X, gamma=gamma, band_k=band_k, seed=seed)
    Th = workloads.random_feasible_theta(w.M, w.N, np.random.default_rng(seed))
    return w, Th


def test_noalloc_objective_matches_plan_objective_twice(tomo):
    f_d = torch.empty(1, dtype=torch.float64, device="cuda")
    # the first problem is larger than the second: the second call must not
    # read the first call's leftovers in the shared scratch
    problems = [case(300, 36, 333, 250.0, 1e-2, 10.0, 5), case(64, 8, 100, 30.0, 1e-3, 0.0, 6)]
    for w, Th in problems:
        with tomo.Plan.from_workload(w) as pl:
            f_ref = pl.objective(dev(w.P), dev(Th))
        got = noalloc(tomo, w.M, w.N, dev(w.lam), w.band_k, w.gamma, dev(w.P), dev(Th), f_d)
        assert got == pytest.approx(f_ref, rel=REL), (w.name, got, f_ref)
    # and the same problem twice in a row gives the same value bit for bit
    w, Th = problems[0]
    a = noalloc(tomo, w.M, w.N, dev(w.lam), w.band_k, w.gamma, dev(w.P), dev(Th), f_d)
    b = noalloc(tomo, w.M, w.N, dev(w.lam), w.band_k, w.gamma, dev(w.P), dev(Th), f_d)
    assert a == b


def test_noalloc_rejects_sizes_beyond_its_scratch(tomo):
    f_d = torch.empty(1, dtype=torch.float64, device="cuda")
    lam = dev(np.linspace(0.0, 10.0, 8))
    P = dev(np.full((8, 3), 1.0 / 3))
    Th = dev(np.full((4, 3), 1.0 / 3))
    L = tomo.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # D + M one past the limit (the pointers are never dereferenced)
    st = L.tomo_objective_noalloc(MAX_ROWS, 3, 1, lam.data_ptr(), 10.0, 0.0, P.data_ptr(),
                                  Th.data_ptr(), f_d.data_ptr(), stream)
    assert st == 1
    assert "TOMO_NOALLOC_MAX_ROWS" in tomo.tomo_last_error()
    st = L.tomo_objective_noalloc(4, 3, 8, lam.data_ptr(), 10.0, 0.0, P.data_ptr(), Th.data_ptr(),
                                  None, stream)
    assert st == 1
    # sizes whose sum overflows int64 are rejected too, before anything is read
    big = 2 ** 62
    st = L.tomo_objective_noalloc(big, 3, big, lam.data_ptr(), 10.0, 0.0, P.data_ptr(),
                                  Th.data_ptr(), f_d.data_ptr(), stream)
    assert st == 1


def test_noalloc_invalid_lambda_gives_nan(tomo):
    # lambda lives in device memory, so an invalid entry cannot be refused on
    # the host: the objective comes back NaN instead of a value computed from
    # an undefined band
    f_d = torch.empty(1, dtype=torch.float64, device="cuda")
    w, Th = case(64, 8, 100, 30.0, 1e-3, 10.0, 7)
    for bad in (-1.0, float("nan"), float("inf")):
        lam = w.lam.copy()
        lam[17] = bad
        got = noalloc(tomo, w.M, w.N, dev(lam), w.band_k, w.gamma, dev(w.P), dev(Th), f_d)
        assert np.isnan(got), (bad, got)
    # and a valid call right after is unaffected
    with tomo.Plan.from_workload(w) as pl:
        f_ref = pl.objective(dev(w.P), dev(Th))
    got = noalloc(tomo, w.M, w.N, dev(w.lam), w.band_k, w.gamma, dev(w.P), dev(Th), f_d)
    assert got == pytest.approx(f_ref, rel=REL)
