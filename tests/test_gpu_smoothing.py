"""Long-range smoothing and the stage-2-only refit (Sec. "Regularisation and
smoothing", Eq. smoothing) through the C ABI, against the oracle."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# The oracle sums each window directly in double (relative error <= (k-1) u
# for k non-negative terms, k <= 2M/div + 1); the kernels use double-double
# prefix sums (error ~1e-32 of a column prefix) and one rounded division.
# 2e-13 covers windows of up to ~900 rows.
RTOL = 2e-13
ATOL = 1e-26


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


def povm_like(M, N, seed):
    """A detector-shaped POVM with entries spanning ~1e-300..1 down each
    column (the case that defeats a plain double prefix difference), plus
    random zeros."""
    bins = N - 1
    th = workloads.detector_povm(M, bins, 0.6, p_dark=1e-6)
    rng = np.random.default_rng(seed)
    th = th * (1.0 + 0.2 * rng.random(th.shape))
    th[rng.random(th.shape) < 0.05] = 0.0
    th[:, 0] += 1e-300
    return th / th.sum(1, keepdims=True)


SHAPES = [
    # M, N, exclude, div, what
    (700, 5, 100, 50.0, "paper settings, ragged last block"),
    (4096, 128, 100, 50.0, "c2 shape"),
    (333, 9, 0, 3.0, "wide windows, nothing excluded"),
    (257, 33, 300, 50.0, "everything excluded"),
    (1, 4, 0, 50.0, "one row"),
    (129, 1024, 10, 7.5, "maximum N, fractional divisor"),
]


@pytest.mark.parametrize("M,N,exclude,div,what", SHAPES, ids=[s[4] for s in SHAPES])
def test_smooth_matches_oracle(tomo, M, N, exclude, div, what):
    X = povm_like(M, N, M + N) if N > 1 else np.ones((M, 1))
    pr = oracle.Problem(M, N, np.array([1.0]), 0.0, 0.0)
    ref = pr.smooth(X, exclude, div)
    with tomo.Plan(M, N, np.array([1.0, 2.0]), band_k=0.0, gamma=0.0) as pl:
        got = pl.smooth(dev(X), exclude, div).cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=RTOL, atol=ATOL)
        np.testing.assert_array_equal(got[:exclude], X[:exclude])
        assert got.min() >= 0.0
        # in place (Y == X) gives the same bits
        Xd = dev(X)
        pl.smooth(Xd, exclude, div, out=Xd)
        np.testing.assert_array_equal(Xd.cpu().numpy(), got)


def test_smooth_rejects_bad_arguments(tomo):
    with tomo.Plan(8, 3, np.array([1.0, 2.0]), band_k=0.0, gamma=0.0) as pl:
        X = dev(np.full((8, 3), 1.0 / 3))
        for exclude, div in ((-1, 50.0), (0, 0.0), (0, -2.0), (0, float("nan"))):
            with pytest.raises(tomo.TomoError):
                pl.smooth(X, exclude, div)


def test_fit_smoothed_matches_oracle(tomo):
    """Algorithm 3, smoothing, then stage 2 only: the GPU smoothing of the
    GPU's first fit equals the oracle's smoothing of that same array, and both
    refits end at the unique optimum of the strictly convex problem."""
    # c1 sizes with a short exclusion and divisor so that most rows move
    w = workloads.config_c1()
    EX, DIV = 16, 8.0
    opts = dict(eps_kkt=1e-11, max_newton=800)
    pr = oracle.Problem.from_workload(w)
    Th_o, rep1_o, rep2_o, Ts_o = pr.fit_smoothed(w.P, exclude=EX, div=DIV, **opts)
    f_o = pr.objective(w.P, Th_o)
    with tomo.Plan.from_workload(w, precision="fp64") as pl:
        P = dev(w.P)
        Th1, rep1 = pl.fit(P, **opts)
        Th1_h = Th1.cpu().numpy().copy()
        Ts = pl.smooth(Th1, EX, DIV)
        np.testing.assert_allclose(Ts.cpu().numpy(), pr.smooth(Th1_h, EX, DIV), rtol=RTOL, atol=ATOL)
        Th, r1, r2 = pl.fit_smoothed(P, exclude=EX, div=DIV, **opts)
        assert r1["status"] == "TOMO_OK" and r2["status"] == "TOMO_OK", (r1, r2)
        assert r2["iters_s1"] == 0 and r2["iters_s2"] > 0
        f_g = pl.objective(P, Th)
    Th = Th.cpu().numpy()
    assert Th.min() >= 0.0
    np.testing.assert_allclose(Th.sum(1), 1.0, atol=1e-13 * w.N)
    assert abs(f_g - f_o) <= 1e-8 * f_o, (f_g, f_o)
