"""The adjoint kernel (Hessian-vector product, parameter derivatives) and the reverse-time pass
through velocity-Verlet, against the FP64 oracle and central finite differences.

Target: gradients within relative 1e-3 of finite differences and of the FP64 oracle gradient.
"""
import numpy as np
import pytest

import oracle as O
from paper_1012_2677_gb300 import ljmd, synth

pytestmark = pytest.mark.gpu

RC = 2.5  # r_c / sigma


def _state(M, rho, T, seed, steps=40, dt=0.005, p=O.LJParams()):
    x, L = O.fcc_lattice(M, rho)
    v = O.init_velocities(len(x), T, seed)
    x, v, *_ = O.vv_run(x, v, L, dt, steps, p)
    return synth.dyadic(x), v, L


def _sys(precision, eps=1.0, sigma=1.0, margin=0.5):
    return ljmd.System(eps=eps, sigma=sigma, cutoff=RC * sigma, margin=margin, precision=precision, energy_every=0)


@pytest.mark.parametrize("precision,tol", [(ljmd.LJ_MIXED, 2e-4), (ljmd.LJ_FP64, 1e-10)])
@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (1.3, 0.9)])
def test_hvp_and_parameter_derivatives(precision, tol, eps, sigma):
    p = O.LJParams(eps=eps, sigma=sigma, rc_over_sigma=RC)
    x, v, L = _state(8, 0.6, 1.2, 3, p=p)
    L = L  # sigma = 0.9 keeps the same box; the liquid is just more dilute in units of sigma
    w = synth.gaussian((len(x), 3), 11)
    ref = O.hvp(x, L, w, p)
    dpe, vjp = O.param_derivs(x, L, p, lam=w)
    with _sys(precision, eps, sigma) as s:
        s.set_state(x, None, L)
        hw, dth = s.hvp(w)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    assert np.sqrt(((hw - ref) ** 2).sum(1)).max() / rms <= tol
    for got, want in zip(dth, (vjp[0], vjp[1], dpe[0], dpe[1])):
        assert got == pytest.approx(want, rel=max(tol, 1e-12), abs=tol * 1e-3 * abs(dpe[0]))


@pytest.mark.parametrize("precision,gtol,ltol", [(ljmd.LJ_MIXED, 1e-3, 1e-5), (ljmd.LJ_FP64, 1e-8, 1e-12)])
@pytest.mark.parametrize("nsteps,n_pe,ckpt", [(12, 4, 5), (10, 10, 10), (7, 1, 2)])
def test_trajectory_gradient_matches_oracle(precision, gtol, ltol, nsteps, n_pe, ckpt):
    p = O.LJParams(eps=1.0, sigma=1.0, rc_over_sigma=RC)
    x, v, L = _state(5, 0.6, 1.2, 5, p=p)  # 500 particles, 3 cells per side
    dt = 0.005
    loss_o, gx_o, gv_o, gth_o = O.traj_loss_grad(x, v, L, dt, nsteps, n_pe, p)
    with _sys(precision) as s:
        loss, gx, gv, gth = s.traj_loss_grad(x, v, L, dt, nsteps, n_pe, ckpt)
    assert loss == pytest.approx(loss_o, rel=ltol)
    for got, want in ((gx, gx_o), (gv, gv_o)):
        assert np.abs(got - want).max() <= gtol * np.abs(want).max()
    for got, want in zip(gth, gth_o):
        assert got == pytest.approx(want, rel=gtol)


def test_trajectory_gradient_matches_finite_differences():
    """Central differences (h = 1e-4) of the FP64-form loss along random directions."""
    x, v, L = _state(5, 0.6, 1.2, 7)
    dt, nsteps, n_pe, ckpt = 0.005, 12, 4, 5
    d = synth.gaussian(x.shape, 21)
    e = synth.gaussian(v.shape, 22)
    with _sys(ljmd.LJ_FP64) as s:
        loss, gx, gv, gth = s.traj_loss_grad(x, v, L, dt, nsteps, n_pe, ckpt)

        def f(xx, vv, eps=1.0, sigma=1.0):
            with _sys(ljmd.LJ_FP64, eps, sigma) as t:
                n = xx.size // 3
                val, _ = ljmd.ljmd_traj_loss_grad(t.h, n, L, np.ascontiguousarray(xx), np.ascontiguousarray(vv), dt,
                                                 nsteps, n_pe, ckpt)
                return val
        h = 1e-4
        fd_x = (f(x + h * d, v) - f(x - h * d, v)) / (2 * h)
        fd_v = (f(x, v + h * e) - f(x, v - h * e)) / (2 * h)
        fd_e = (f(x, v, eps=1.0 + h) - f(x, v, eps=1.0 - h)) / (2 * h)
        fd_s = (f(x, v, sigma=1.0 + h) - f(x, v, sigma=1.0 - h)) / (2 * h)
    assert (gx * d).sum() == pytest.approx(fd_x, rel=1e-3)
    assert (gv * e).sum() == pytest.approx(fd_v, rel=1e-3)
    assert gth[0] == pytest.approx(fd_e, rel=1e-3)
    assert gth[1] == pytest.approx(fd_s, rel=1e-3)


def test_trajectory_gradient_32k_mixed_vs_fp64():
    """The differentiable-trajectory workload: 32,000 particles (FCC 20^3 x 4), rho = 0.6, T = 1.2,
    50 steps, loss over the last 10, checkpoints every 10.  The mixed form's gradients agree with
    the FP64 form (pinned to the oracle above) to 1e-3, and the FP64 form's x0-gradient with a
    central difference along a random direction."""
    x, L = O.fcc_lattice(20, 0.6)
    v = O.init_velocities(len(x), 1.2, 5)
    dt, nsteps, n_pe, ckpt = 0.005, 50, 10, 10
    out = {}
    for prec in (ljmd.LJ_MIXED, ljmd.LJ_FP64):
        with _sys(prec) as s:
            out[prec] = s.traj_loss_grad(x, v, L, dt, nsteps, n_pe, ckpt)
    lm, gxm, gvm, gthm = out[ljmd.LJ_MIXED]
    l6, gx6, gv6, gth6 = out[ljmd.LJ_FP64]
    assert lm == pytest.approx(l6, rel=1e-5)
    assert np.linalg.norm(gxm - gx6) <= 1e-3 * np.linalg.norm(gx6)
    assert np.linalg.norm(gvm - gv6) <= 1e-3 * np.linalg.norm(gv6)
    assert gthm[0] == pytest.approx(gth6[0], rel=1e-3)
    assert gthm[1] == pytest.approx(gth6[1], rel=1e-3)
    d = synth.gaussian(x.shape, 31)
    h = 1e-4
    vals = []
    for sgn in (1, -1):
        with _sys(ljmd.LJ_FP64) as s:
            val, _ = ljmd.ljmd_traj_loss_grad(s.h, len(x), L, np.ascontiguousarray(x + sgn * h * d), v, dt, nsteps,
                                             n_pe, ckpt)
            vals.append(val)
    assert (gx6 * d).sum() == pytest.approx((vals[0] - vals[1]) / (2 * h), rel=1e-3)


def test_autograd_function_backward():
    torch = pytest.importorskip("torch")
    from paper_1012_2677_gb300.autograd import LJTrajectory

    x, v, L = _state(5, 0.6, 1.2, 9)
    dt, nsteps, n_pe, ckpt = 0.005, 12, 4, 5
    with _sys(ljmd.LJ_MIXED) as s:
        loss_ref, gx_ref, gv_ref, gth_ref = s.traj_loss_grad(x, v, L, dt, nsteps, n_pe, ckpt)
    dev = torch.device("cuda", 0)
    xt = torch.tensor(x, device=dev, requires_grad=True)
    vt = torch.tensor(v, device=dev, requires_grad=True)
    et = torch.tensor(1.0, dtype=torch.float64, device=dev, requires_grad=True)
    st = torch.tensor(1.0, dtype=torch.float64, device=dev, requires_grad=True)
    loss = LJTrajectory.apply(xt, vt, et, st, L, dt, nsteps, n_pe, ckpt)
    (2.0 * loss).backward()
    assert float(loss.detach()) == pytest.approx(loss_ref, rel=1e-6)
    np.testing.assert_allclose(xt.grad.cpu().numpy(), 2.0 * gx_ref, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(vt.grad.cpu().numpy(), 2.0 * gv_ref, rtol=1e-6, atol=1e-9)
    assert float(et.grad) == pytest.approx(2.0 * gth_ref[0], rel=1e-6)
    assert float(st.grad) == pytest.approx(2.0 * gth_ref[1], rel=1e-6)
