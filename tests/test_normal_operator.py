"""The Toeplitz normal operator E^H D E (tffr_normal_setup / tffr_normal_apply)
against the explicit FP64 matrix on small grids, against the route through the
forward twin and the adjoint, and inside conjugate gradients (GPU)."""

import numpy as np
import pytest
import torch

import oracle
from synth import random_points, stolt_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dense_normal(lx, ly, D, Mx, My, f):
    """(E^H D E f) from the definition E[n, (jy, jx)] = exp(-2 pi i (lx x_jx + ly y_jy)), in FP64."""
    x = (np.arange(Mx) - Mx / 2) / Mx
    y = (np.arange(My) - My / 2) / My
    E = np.exp(-2j * np.pi * (lx[:, None, None] * x[None, None, :] + ly[:, None, None] * y[None, :, None]))
    E = E.reshape(lx.shape[0], My * Mx)
    return (E.conj().T @ (D * (E @ f.reshape(-1)))).reshape(My, Mx)


@pytest.mark.parametrize("case", ["random_square", "stolt_rows_non_square"])
def test_normal_operator_against_the_explicit_matrix(case):
    from paper_1910_10908_gb300 import Plan
    g = np.random.default_rng(11)
    if case == "random_square":
        Mx = My = 32
        lx, ly, _ = random_points(2500, 32, seed=12, extent=0.5)
        tau = 1.0
    else:
        Mx, My = 32, 16
        lx, ly, _ = stolt_points(40, 80, 32)
        ly = ly * 0.5
        tau = 0.97
    D = oracle.tffr_weights(lx, Mx, tau=tau)
    f = g.standard_normal((My, Mx)) + 1j * g.standard_normal((My, Mx))
    ref = dense_normal(lx, ly, D, Mx, My, f)
    with Plan(Mx, My, width=8) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(tau=tau, count=False)
        plan.normal_setup()
        ft = dev(f.astype(np.complex64))
        nt = plan.normal(ft).cpu().numpy().astype(np.complex128)
        via = plan.adjoint(plan.forward(ft, apply_weights=False)).cpu().numpy().astype(np.complex128)
        same = plan.normal(ft, out=ft).cpu().numpy().astype(np.complex128)    # in place
    assert rel(nt, ref) <= 1e-5
    assert rel(via, ref) <= 1e-5
    assert rel(same, nt) <= 1e-6


def test_cg_with_the_toeplitz_operator():
    """Same jittered, twice-oversampled problem as the CG test of the differentiable module."""
    from paper_1910_10908_gb300 import Plan
    from paper_1910_10908_gb300.differentiable import cg_normal
    M = 16
    g = np.random.default_rng(3)
    k = np.arange(-M, M) / 2.0
    KX, KY = np.meshgrid(k, k)
    lx = KX.ravel() + g.uniform(-0.2, 0.2, KX.size)
    ly = KY.ravel() + g.uniform(-0.2, 0.2, KY.size)
    N = lx.shape[0]
    f_true = g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))
    x = (np.arange(M) - M / 2) / M
    E = np.exp(-2j * np.pi * (lx[:, None, None] * x[None, None, :] + ly[:, None, None] * x[None, :, None]))
    E = E.reshape(N, M * M)
    y = E @ f_true.reshape(-1) + 0.01 * (g.standard_normal(N) + 1j * g.standard_normal(N))
    D = oracle.tffr_weights(lx, M)
    f_ls = np.linalg.lstsq(np.sqrt(D)[:, None] * E, np.sqrt(D) * y, rcond=None)[0].reshape(M, M)
    with Plan(M, width=8) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(count=False)
        f, hist = cg_normal(plan, dev(y.astype(np.complex64)), iters=25, toeplitz=True)
    f = f.cpu().numpy().astype(np.complex128)
    assert hist[-1] < 1e-5 * hist[0]
    assert rel(f, f_ls) < 1e-4


def test_normal_operator_needs_setup_for_the_current_points():
    from paper_1910_10908_gb300 import Plan, TffrError
    lx, ly, _ = random_points(500, 16, seed=13, extent=0.5)
    with Plan(16) as plan:
        plan.set_points(dev(lx), dev(ly))
        plan.weights(count=False)
        img = torch.zeros((16, 16), dtype=torch.complex64, device="cuda")
        with pytest.raises(TffrError):
            plan.normal(img)
        plan.normal_setup()
        plan.normal(img)
        plan.set_points(dev(lx), dev(ly))        # new points: the operator must be rebuilt
        plan.weights(count=False)
        with pytest.raises(TffrError):
            plan.normal(img)
    with Plan(4096) as big:
        big.set_points(dev(lx), dev(ly))
        big.weights(count=False)
        with pytest.raises(TffrError):
            big.normal_setup()                    # sides above 2048
