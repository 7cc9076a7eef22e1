"""CPU pins of the Burgers validation workload (Sec. 4.3): the generator is the
analytic solution of the viscous Burgers equation, and the oracle's streaming
run on it recovers the serial SVD's leading modes."""
import numpy as np
import torch

import oracle
from paper_2108_08845_gb300 import synthetic


def test_burgers_solves_the_pde():
    # central differences of u on a fine grid: u_t + u u_x - nu u_xx vanishes up to
    # the O(dx^2 + dt^2) truncation error (a wrong factor or sign gives O(1))
    M, N, Re = 4097, 2001, 1000.0
    U = synthetic.burgers(M, N, Re).numpy()
    dx, dt, nu = 1.0 / (M - 1), 2.0 / (N - 1), 1.0 / Re
    ut = (U[1:-1, 2:] - U[1:-1, :-2]) / (2 * dt)
    ux = (U[2:, 1:-1] - U[:-2, 1:-1]) / (2 * dx)
    uxx = (U[2:, 1:-1] - 2 * U[1:-1, 1:-1] + U[:-2, 1:-1]) / dx ** 2
    u = U[1:-1, 1:-1]
    r = ut + u * ux - nu * uxx
    scale = max(np.abs(ut).max(), np.abs(u * ux).max(), np.abs(nu * uxx).max())
    assert np.abs(r).max() <= 1e-3 * scale
    # boundary conditions: u(0, t) = 0, u(1, t) ~ 0
    assert np.all(U[0] == 0.0) and np.abs(U[-1]).max() < 1e-8


def test_oracle_stream_recovers_serial_modes_on_burgers():
    # ff = 1 and K well above the resolved rank: the streamed modes 1-2 are the
    # serial SVD's (the paper's serial-vs-parallel comparison, on the oracle)
    A = synthetic.burgers(2048, 240).numpy()
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    bs = [np.asfortranarray(A[:, i:i + 60]) for i in range(0, 240, 60)]
    Uo, Do = oracle.stream_run(bs, 40, 1.0)
    assert np.all(np.abs(Do[:2] - s[:2]) <= 1e-9 * s[:2])
    for j in range(2):
        assert abs(abs(Uo[:, j] @ U[:, j]) - 1.0) <= 1e-9
