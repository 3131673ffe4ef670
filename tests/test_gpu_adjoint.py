"""Gradients through K x-line block-Jacobi sweeps (library adjoint sweeps behind autograd).

L = 0.5 ||u_K - u_t||^2.  Checked against the oracle's reverse-mode gradients, against
central finite differences (exact for the u0 and b directions, which L is quadratic in;
O(h^2) for the coefficients) and for invariance to the checkpoint interval.
"""
import numpy as np
import pytest

from brs_inputs import SEED_TARGET, initial_guess, rhs, uniform_field
from gpu_common import rel_max_err, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def gpu_grads(brs, b, u0, ut, a, K, ckpt, dt):
    import torch

    bt = to_dev(b, dt).requires_grad_(True)
    u0t = to_dev(u0, dt).requires_grad_(True)
    at = torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
    u = brs.block_smooth(bt, u0t, at, K, ckpt=ckpt)
    d = u.double() - to_dev(ut, "f64")
    loss = 0.5 * (d * d).sum()
    loss.backward()
    return float(loss.detach()), to_np(u0t.grad), to_np(bt.grad), at.grad.cpu().numpy()


@pytest.mark.parametrize("ckpt", [1, 2, 4])
def test_adjoint_matches_oracle_small(brs, orc, ckpt):
    shape = (8, 10, 12)
    a = (1.0, 0.7, 0.3)
    rng = np.random.default_rng(5)
    u0, b, ut = (rng.uniform(-1, 1, shape) for _ in range(3))
    K = 4
    L, gu, gb, ga = gpu_grads(brs, b, u0, ut, a, K, ckpt, "f64")
    Lr, gur, gbr, gar = orc.adjoint_gradients(u0, b, a, K, ut, block="line", omega=0.8)
    assert abs(L - Lr) <= 1e-12 * abs(Lr)
    assert rel_max_err(gu, gur) <= 1e-11
    assert rel_max_err(gb, gbr) <= 1e-11
    np.testing.assert_allclose(ga, gar, rtol=1e-10)


def test_adjoint_fp32_vs_oracle(brs, orc):
    n = 32
    shape = (n, n, n)
    a = (1.0, 1.0, 1.0)
    u0 = initial_guess(shape).astype(np.float32).astype(np.float64)
    b = rhs(shape).astype(np.float32).astype(np.float64)
    ut = uniform_field(shape, SEED_TARGET)
    _, gu, gb, ga = gpu_grads(brs, b, u0, ut, a, 8, 4, "f32")
    _, gur, gbr, gar = orc.adjoint_gradients(u0, b, a, 8, ut, block="line", omega=0.8)
    assert rel_max_err(gu, gur) <= 2e-5
    assert rel_max_err(gb, gbr) <= 2e-5
    np.testing.assert_allclose(ga, gar, rtol=1e-4)


def test_adjoint_128_fp64_vs_oracle(brs, orc):
    """The 128^3 differentiation workload: 8 sweeps, u_target ~ U[-1,1] (seed 3)."""
    n = 128
    shape = (n, n, n)
    a = (1.0, 1.0, 1.0)
    u0, b, ut = initial_guess(shape), rhs(shape), uniform_field(shape, SEED_TARGET)
    L, gu, gb, ga = gpu_grads(brs, b, u0, ut, a, 8, 4, "f64")
    Lr, gur, gbr, gar = orc.adjoint_gradients(u0, b, a, 8, ut, block="line", omega=0.8)
    assert abs(L - Lr) <= 1e-12 * abs(Lr)
    assert rel_max_err(gu, gur) <= 1e-11
    assert rel_max_err(gb, gbr) <= 1e-11
    np.testing.assert_allclose(ga, gar, rtol=1e-9)


@pytest.mark.parametrize("n", [128, 384])
def test_adjoint_fp32_bench_sizes_vs_oracle(brs, orc, n):
    """The FP32 differentiation workloads (8 sweeps, checkpoint every 4) in the benchmark's
    kernels (z-march update, one-wave line M^-1), element by element against the oracle's
    FP64 reverse-mode gradients."""
    shape = (n, n, n)
    a = (1.0, 1.0, 1.0)
    u0 = initial_guess(shape).astype(np.float32).astype(np.float64)
    b = rhs(shape).astype(np.float32).astype(np.float64)
    ut = uniform_field(shape, SEED_TARGET)
    L, gu, gb, ga = gpu_grads(brs, b, u0, ut, a, 8, 4, "f32")
    Lr, gur, gbr, gar = orc.adjoint_gradients(u0, b, a, 8, ut, block="line", omega=0.8)
    assert abs(L - Lr) <= 1e-5 * abs(Lr)
    assert rel_max_err(gu, gur) <= 2e-5
    assert rel_max_err(gb, gbr) <= 2e-5
    np.testing.assert_allclose(ga, gar, rtol=1e-4)


def _loss(brs, b, u0, ut, a, K, dt="f64"):
    import torch

    nz, ny, nx = b.shape
    with brs.Context(nx, ny, nz, a, block="line", method="jacobi", dtype=dt) as c:
        u = u0.clone()
        c.sweep(u, b, K)
        d = u.double() - ut
        return float(0.5 * (d * d).sum())


def test_adjoint_384_checkpointing_and_finite_differences(brs):
    """384^3, 8 sweeps, checkpoint every 4: gradients equal the no-recompute ones bitwise and
    match central differences (exact along u0 and b; O(h^2) along the coefficients)."""
    import torch

    n = 384
    shape = (n, n, n)
    a = (1.0, 1.0, 1.0)
    gen = torch.Generator(device="cuda").manual_seed(9)
    mk = lambda s=1.0: (torch.rand(shape, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1) * s
    u0, b, ut, d = mk(), mk(1.0 / (n + 1) ** 2), mk(), mk()
    res = {}
    for ck in (4, 8):
        bt = b.clone().requires_grad_(True)
        u0t = u0.clone().requires_grad_(True)
        at = torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
        u = brs.block_smooth(bt, u0t, at, 8, ckpt=ck)
        diff = u - ut
        (0.5 * (diff * diff).sum()).backward()
        res[ck] = (u0t.grad.clone(), bt.grad.clone(), at.grad.clone())
        del bt, u0t, u, diff
    for x, y in zip(res[4], res[8]):
        assert torch.equal(x, y)
    gu, gb, ga = res[4]
    eps = 0.5  # L is exactly quadratic in u0 and b: a large step has no truncation error
    fd_u = (_loss(brs, b, u0 + eps * d, ut, a, 8) - _loss(brs, b, u0 - eps * d, ut, a, 8)) / (2 * eps)
    assert abs(fd_u - float((gu * d).sum())) <= 1e-8 * abs(fd_u)
    fd_b = (_loss(brs, b + eps * d, u0, ut, a, 8) - _loss(brs, b - eps * d, u0, ut, a, 8)) / (2 * eps)
    assert abs(fd_b - float((gb * d).sum())) <= 1e-8 * max(abs(fd_b), 1e-30) + 1e-9
    for dd in range(3):
        h = 1e-3
        ap, am = list(a), list(a)
        ap[dd] += h
        am[dd] -= h
        fd = (_loss(brs, b, u0, ut, ap, 8) - _loss(brs, b, u0, ut, am, 8)) / (2 * h)
        assert abs(fd - float(ga[dd])) <= 1e-5 * abs(fd), (dd, fd, float(ga[dd]))


def test_adjoint_unsupported_paths(brs):
    import torch

    with brs.Context(8, 8, 8, block="plane", method="jacobi") as c:
        z = torch.zeros(512, dtype=torch.float64, device="cuda")
        ga = torch.zeros(3, dtype=torch.float64, device="cuda")
        p = z.data_ptr()
        assert brs.brsmooth_adjoint_sweep(c.h, p, p, p, p, ga.data_ptr(), 0) == brs.BRS_ERR_UNSUPPORTED
    with brs.Context(8, 8, 8, block="line", method="gs") as c:
        assert brs.brsmooth_adjoint_sweep(c.h, p, p, p, p, ga.data_ptr(), 0) == brs.BRS_ERR_UNSUPPORTED
