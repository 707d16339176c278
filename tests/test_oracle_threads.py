"""The oracle's node loops on several host threads give bitwise the single-thread results.

Threads only split the nodes among themselves (moments, gradient, history, collision and streaming, the
history-only driver); every node's arithmetic is the same sequence of operations, so any difference
would mean a race (a node written by two threads, or shared scratch).
"""
import numpy as np
import pytest

import oracle
from paper_1504_06123_gb300 import inputs


@pytest.fixture
def restore_threads():
    n = oracle.threads()
    yield
    oracle.set_threads(n)


@pytest.mark.parametrize("lattice,nx,ny,nz,trace_full", [
    (oracle.D2Q9, 3, 40, 1, True),
    (oracle.D2Q9, 5, 17, 1, False),
    (oracle.D3Q19, 3, 6, 5, True),
])
def test_channel_bitwise_across_thread_counts(restore_threads, lattice, nx, ny, nz, trace_full):
    N = nx * ny * nz
    rho = inputs.initial_density(N, 1e-4, seed=21)
    out = {}
    for th in (1, 3, 0):
        oracle.set_threads(th)
        ch = oracle.Channel(lattice, nx, ny, nz, tau_lb=0.9, G_inf=0.01, tau=30.0, gamma_c=0.1, g=(2e-5, 0, 0),
                            C=8, B=3, rho_init=rho, trace_full=trace_full)
        ch.step(90)
        out[th] = (ch.fields(), ch.populations())
        ch.close()
    for th in (3, 0):
        for k, v in out[1][0].items():
            assert np.array_equal(v, out[th][0][k]), (th, k)
        assert np.array_equal(out[1][1], out[th][1])


def test_history_run_bitwise_across_thread_counts(restore_threads):
    kseq = inputs.kappa_sequence(60, 37, 2, 2e-3, seed=5, shear=1e-3)
    res = []
    for th in (1, 4):
        oracle.set_threads(th)
        res.append(oracle.history_run(kseq, 8, 3, 0.02, 40.0, 0.1))
    assert np.array_equal(res[0], res[1])


def test_thread_count_reported(restore_threads):
    assert oracle.set_threads(1) == 1
    assert oracle.threads() == 1
    n = oracle.set_threads(0)
    assert n >= 1 and oracle.threads() == n
