"""The batched population's generator (workloads.config_c4) is reproducible
instance by instance: config_c4_instance(j) alone, and in spawned host
processes (as the batched evaluation generates large populations), gives
exactly the instances of config_c4 -- same sizes, probes and frequencies."""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import workloads


def test_c4_instances_are_reproducible_alone_and_in_spawned_workers():
    serial = workloads.config_c4(n_instances=4, max_M=600)
    alone = [workloads.config_c4_instance(j, 600) for j in range(4)]
    with ProcessPoolExecutor(2, mp_context=mp.get_context("spawn")) as ex:
        spawned = list(ex.map(workloads.config_c4_instance, range(4), [600] * 4))
    for a, b, c in zip(serial, alone, spawned):
        assert (a.M, a.N, a.D) == (b.M, b.N, b.D) == (c.M, c.N, c.D)
        assert 256 <= a.M <= 600 and 8 <= a.N <= 128 and a.D == 2 * a.M
        np.testing.assert_array_equal(a.lam, b.lam)
        np.testing.assert_array_equal(a.lam, c.lam)
        np.testing.assert_array_equal(a.P, b.P)
        np.testing.assert_array_equal(a.P, c.P)
        np.testing.assert_array_equal(a.theta_true, c.theta_true)
