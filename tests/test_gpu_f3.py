"""Liu-shaped near-dense geometry (Sec. Application to other detector
geometries) on the GPU: solves against the oracle optimum at N = 10, products
on sampled rows at N = 300 and N = 1000 (eight column blocks)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc"])
def test_small_liu_case_reaches_the_oracle_optimum(tomo, prec):
    w = workloads.config_f3(10, gamma=1e-3)
    pr = oracle.Problem.from_workload(w)
    _, rep_o, _ = pr.fit(w.P, eps_kkt=1e-12, max_newton=3000)
    with tomo.Plan.from_workload(w, precision=prec) as pl:
        Th, rep = pl.fit(dev(w.P), eps_kkt=1e-12, max_newton=3000)
    f = pr.objective(w.P, Th.cpu().numpy())
    assert (f - rep_o["f"]) / rep_o["f"] <= 1e-8, (f, rep_o["f"], rep)


@pytest.mark.parametrize("N", [300, 1000])
def test_liu_products_on_sampled_rows(tomo, N):
    M, D = workloads.liu_sizes(N)
    lam = workloads.probe_intensities(D, 0.75 * M)
    rng = np.random.default_rng(N)
    X = rng.random((M, N))
    X /= X.sum(1, keepdims=True)
    pr = oracle.Problem(M, N, lam, 10.0, 1e-4, store_F=False)
    rows_d = np.unique(np.concatenate([[0, D - 1], rng.integers(0, D, 10)]))
    rows_i = np.unique(np.concatenate([[0, M - 1], rng.integers(0, M, 10)]))
    O64 = pr.apply_F_rows(X, np.arange(D))
    ref_h = 2.0 * pr.apply_Ft_rows(O64, rows_i)
    scale_h = 2.0 * pr.apply_Ft_rows(np.abs(O64), rows_i)
    # 2 gamma L X on the sampled rows
    for k, i in enumerate(rows_i):
        lx = np.zeros(N)
        if i < M - 1:
            lx += X[i] - X[i + 1]
        if i > 0:
            lx += X[i] - X[i - 1]
        ref_h[k] += 2e-4 * lx
        scale_h[k] += 2e-4 * np.abs(lx)
    Xd = dev(X)
    for prec, tol in (("fp32", 2e-5), ("tc", 2e-4)):
        with tomo.Plan(M, N, lam, 10.0, 1e-4, precision=prec) as pl:
            O = pl.apply_F(Xd)
            g = O[torch.from_numpy(rows_d).cuda()].cpu().numpy()
            ref = O64[rows_d]
            sc = pr.apply_F_rows(np.abs(X), rows_d)
            assert np.all(np.abs(g - ref) <= tol * sc + 1e-300), prec
            HV = pl.hvp(Xd)
            gh = HV[torch.from_numpy(rows_i).cuda()].cpu().numpy()
            assert np.all(np.abs(gh - ref_h) <= tol * scale_h + 1e-300), prec
