"""Learned warm start through the C ABI (tomo_ws_*), against the numpy oracle
of oracle/warmstart.py: loss and gradient, one Adam step, bf16 inference,
parameter files, and the warm-started fit on held-out detectors."""
import numpy as np
import pytest

import workloads
from oracle import warmstart as ows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# float kernels against the float64 oracle on the same float32 parameters
RTOL_LOSS = 2e-5
GRAD_TOL = 2e-5      # relative to the largest gradient entry


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


SHAPES = [
    ows.Shape(D=16, C0=4, M=6, C1=3, C2=2, K=3, S1=2, S2=2, H=3),
    ows.Shape(D=64, C0=40, M=16, C1=5, C2=4, K=5, S1=2, S2=4, H=8),
]


def batch(shape, rng, ncols):
    B = len(ncols)
    P = rng.random((B, shape.D, shape.C0))
    T = rng.random((B, shape.M, shape.C0))
    for b, nc in enumerate(ncols):
        P[b, :, nc:] = 0.0
        T[b, :, nc:] = 0.0
    T /= T.sum(2, keepdims=True)
    return P, T


def make_ws(tomo, shape, B, seed=3):
    return tomo.WarmStart(shape.D, shape.C0, shape.M, C1=shape.C1, C2=shape.C2, K=shape.K, S1=shape.S1,
                          S2=shape.S2, H=shape.H, max_batch=B, seed=seed)


@pytest.mark.parametrize("shape", SHAPES, ids=["tiny", "ragged"])
def test_loss_and_gradient_match_oracle(tomo, shape):
    rng = np.random.default_rng(11)
    ncols = [shape.C0, max(2, shape.C0 - 3), 2]
    P, T = batch(shape, rng, ncols)
    with make_ws(tomo, shape, len(ncols)) as ws:
        assert ws.param_count == shape.count()
        theta = (rng.standard_normal(shape.count()) * 0.3).astype(np.float32)
        ws.set_params(theta)
        loss, g = ws.loss_grad(dev(P), dev(T), ncols)
    L_ref, g_ref = ows.loss_and_grad(shape, theta.astype(np.float64), list(P), list(T), ncols)
    assert loss == pytest.approx(L_ref, rel=RTOL_LOSS)
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= GRAD_TOL * scale, np.abs(g - g_ref).max() / scale


def test_adam_step_matches_oracle(tomo):
    shape = SHAPES[1]
    rng = np.random.default_rng(12)
    ncols = [shape.C0, 7]
    P, T = batch(shape, rng, ncols)
    with make_ws(tomo, shape, 2) as ws:
        theta = ws.params()
        _, g = ws.loss_grad(dev(P), dev(T), ncols)
        m = np.zeros(theta.size)
        v = np.zeros(theta.size)
        th = theta.astype(np.float64)
        for step in (1, 2):
            _, gs = ws.loss_grad(dev(P), dev(T), ncols)
            ws.train_step(dev(P), dev(T), ncols, lr=1e-2)
            th, m, v = ows.adam_step(th, m, v, gs.astype(np.float64), step, 1e-2)
            got = ws.params()
            np.testing.assert_allclose(got, th, rtol=1e-5, atol=1e-6)
            th = got.astype(np.float64)


def test_inference_uses_bf16_weights_and_gives_simplex_rows(tomo):
    shape = SHAPES[1]
    rng = np.random.default_rng(13)
    N = 23
    P = rng.random((shape.D, N))
    with make_ws(tomo, shape, 1) as ws:
        theta = (rng.standard_normal(shape.count()) * 0.3).astype(np.float32)
        ws.set_params(theta)
        Th0 = ws.infer(dev(P)).cpu().numpy()
    Pp = np.zeros((shape.D, shape.C0))
    Pp[:, :N] = P
    ref = ows.forward(shape, ows.round_bf16(theta), Pp, N)["Theta0"][:, :N]
    assert Th0.shape == (shape.M, N)
    np.testing.assert_allclose(Th0, ref, rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(Th0.sum(1), 1.0, atol=1e-5)
    assert Th0.min() >= 0.0


def test_parameter_file_round_trip(tomo, tmp_path):
    shape = SHAPES[0]
    with make_ws(tomo, shape, 1, seed=5) as a, make_ws(tomo, shape, 1, seed=6) as b:
        assert not np.array_equal(a.params(), b.params())
        a.save(tmp_path / "w.bin")
        b.load(tmp_path / "w.bin")
        np.testing.assert_array_equal(a.params(), b.params())
    other = SHAPES[1]
    with make_ws(tomo, other, 1) as c:
        with pytest.raises(tomo.TomoError):
            c.load(tmp_path / "w.bin")


def test_training_lowers_the_loss_and_warm_starts_save_iterations(tomo):
    """A scaled-down detector population (D = 256 probes, M = 128, up to 16
    outcomes): a short training run lowers the held-out loss, and fits started
    from the network's Theta0 reach the same optimum as cold fits in fewer
    Newton iterations on average."""
    D, M, X, C0 = 256, 128, 96.0, 16
    lam = workloads.probe_intensities(D, X)
    F = workloads.dense_poisson(M, lam)
    kw = dict(F=F, M=M, D=D, X=X, bins_range=(4, 15), C0=C0)
    Ptr, Ttr, nctr, _ = workloads.c5_batch(range(0, 192), **kw)
    Pte, Tte, ncte, wte = workloads.c5_batch(range(10000, 10008), **kw)
    shape = ows.Shape(D=D, C0=C0, M=M, C1=16, C2=16, K=5, S1=2, S2=4, H=32)
    Ptr_d, Ttr_d = dev(Ptr), dev(Ttr)
    with make_ws(tomo, shape, 32, seed=7) as ws:
        l0, _ = ws.loss_grad(dev(Pte), dev(Tte), ncte)
        rng = np.random.default_rng(0)
        for it in range(600):
            idx = rng.choice(len(nctr), 32, replace=False)
            ws.train_step(Ptr_d[idx].contiguous(), Ttr_d[idx].contiguous(), nctr[idx], lr=3e-3)
        l1, _ = ws.loss_grad(dev(Pte), dev(Tte), ncte)
        assert l1 < 0.7 * l0, (l0, l1)
        cold, warm = [], []
        for w in wte:
            with tomo.Plan.from_workload(w, precision="fp32") as pl:
                P = dev(w.P)
                Thc, rc = pl.fit(P, eps_kkt=1e-9, max_newton=2000)
                Thw, rw, used = tomo.fit_warm(pl, ws, P, eps_kkt=1e-9, max_newton=2000)
                fc, fw = pl.objective(P, Thc), pl.objective(P, Thw)
            assert abs(fw - fc) <= 1e-6 * fc, (w.name, fc, fw)
            cold.append(rc["iters_s1"] + rc["iters_s2"])
            warm.append(rw["iters_s1"] + rw["iters_s2"])
    assert np.mean(warm) < np.mean(cold), (cold, warm)


def test_fit_warm_fallback_rule_runs_in_the_library(tomo):
    """tomo_fit_warm: the library starts from the network's Theta0 exactly when
    f(Theta0) < f(1/N) and otherwise from 1/N (for an untrained network whose
    parameters are all zero, Theta0 is uniform up to float rounding), reaches
    the cold fit's optimum either way, and refuses a handle whose shape does
    not match the plan."""
    D, M, X, C0 = 256, 128, 96.0, 16
    lam = workloads.probe_intensities(D, X)
    F = workloads.dense_poisson(M, lam)
    kw = dict(F=F, M=M, D=D, X=X, bins_range=(4, 15), C0=C0)
    Ptr, Ttr, nctr, _ = workloads.c5_batch(range(0, 96), **kw)
    _, _, _, wte = workloads.c5_batch(range(20000, 20002), **kw)
    shape = ows.Shape(D=D, C0=C0, M=M, C1=8, C2=8, K=5, S1=2, S2=4, H=16)

    def check(ws, w):
        with tomo.Plan.from_workload(w, precision="fp32") as pl:
            P = dev(w.P)
            Thc, rc = pl.fit(P, eps_kkt=1e-10, max_newton=2000)
            Thw, rw, used = tomo.fit_warm(pl, ws, P, eps_kkt=1e-10, max_newton=2000)
            uni = torch.full((w.M, w.N), 1.0 / w.N, dtype=torch.float64, device="cuda")
            assert used == (pl.objective(P, ws.infer(P)) < pl.objective(P, uni))
            if not used:
                # the cold path is the plain fit, bit for bit
                assert torch.equal(Thw, Thc)
            fc, fw = pl.objective(P, Thc), pl.objective(P, Thw)
            assert abs(fw - fc) <= 1e-7 * fc, (fc, fw)
            # the sparsified start (small entries of Theta0 set to their bound)
            # goes through the same rule and reaches the same optimum
            Ths, rs, _ = tomo.fit_warm(pl, ws, P, zero_below=1e-3, eps_kkt=1e-10, max_newton=2000)
            T = Ths.cpu().numpy()
            assert np.abs(T.sum(1) - 1).max() <= 1e-12 and T.min() >= 0.0
            fs = pl.objective(P, Ths)
            assert abs(fs - fc) <= 1e-7 * fc, (fc, fs)
        return used

    with make_ws(tomo, shape, 32, seed=11) as ws:
        ws.set_params(np.zeros(ws.param_count, dtype=np.float32))
        check(ws, wte[0])
        Ptr_d, Ttr_d = dev(Ptr), dev(Ttr)
        rng = np.random.default_rng(1)
        for _ in range(300):
            idx = rng.choice(len(nctr), 32, replace=False)
            ws.train_step(Ptr_d[idx].contiguous(), Ttr_d[idx].contiguous(), nctr[idx], lr=3e-3)
        for w in wte:
            check(ws, w)
    other = ows.Shape(D=D, C0=C0, M=M // 2, C1=4, C2=4, K=3, S1=2, S2=2, H=4)
    with make_ws(tomo, other, 4) as ws2:
        w = wte[0]
        with tomo.Plan.from_workload(w, precision="fp32") as pl:
            with pytest.raises(tomo.TomoError) as e:
                tomo.fit_warm(pl, ws2, dev(w.P))
            assert e.value.status == 1
    with make_ws(tomo, shape, 4) as ws3:
        w = wte[0]
        with tomo.Plan.from_workload(w, precision="fp32") as pl:
            with pytest.raises(tomo.TomoError) as e:
                tomo.fit_warm(pl, ws3, dev(w.P), zero_below=1.5)
            assert e.value.status == 1
