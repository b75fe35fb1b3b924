"""Adjoint gradients dJ/d(E0, omega, sigma) of J = sum_n w_n . Re mu(t_n) through RK4
(rtcc_propagate_vjp) against central finite differences (delta = 1e-5) of the float64 forward
propagation, on the GPU and with the CPU oracle, against the oracle's forward-mode tangent, and
through torch.autograd."""
import numpy as np
import pytest

from oracle import rk
from paper_2205_05175_gb300 import synth

pytestmark = pytest.mark.gpu


def _weights(nsteps, h, center, width, comp=2):
    t = h * np.arange(nsteps + 1)
    w = np.zeros((nsteps + 1, 3))
    w[:, comp] = np.exp(-0.5 * (t - center) ** 2 / width ** 2)
    return w


def _J_gpu(H, y0, theta, h, nsteps, w):
    from paper_2205_05175_gb300 import rtcc
    H.set_state(0, y0, 0.0, 0.0)
    f = rtcc.make_field(E0=theta[0], omega=theta[1], sigma=theta[2], t0=1.0)
    _, m, n = H.propagate([f], rtcc.make_integrator(rtcc.RK4, h=h, nsteps=nsteps), nsteps + 1)
    return float(np.sum(w * m[0, :n[0]].real))


@pytest.mark.parametrize("prec,rtol", [(0, 2e-6), (3, 2e-3)])
def test_vjp_matches_float64_finite_differences(prec, rtol):
    from paper_2205_05175_gb300 import rtcc
    o, v = 3, 8
    f, B, mu = synth.make_system(o, v)
    h, nsteps = 0.05, 30
    w = _weights(nsteps, h, 1.0, 0.4)
    theta = np.array([0.05, 0.5, 0.5])
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as H64:
        H64.ground_state(tol=1e-12)
        y0 = H64.get_state(0)[0]
        fd = []
        for j in range(3):
            d = np.zeros(3)
            d[j] = 1e-5
            fd.append((_J_gpu(H64, y0, theta + d, h, nsteps, w) - _J_gpu(H64, y0, theta - d, h, nsteps, w)) / 2e-5)
        J64 = _J_gpu(H64, y0, theta, h, nsteps, w)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=prec) as H:
        H.set_state(0, y0, 0.0, 0.0)
        J, g = H.propagate_vjp([rtcc.make_field(E0=theta[0], omega=theta[1], sigma=theta[2], t0=1.0)], h, nsteps, w,
                               ckpt_every=7)
        y_after = H.get_state(0)[0]
    assert np.abs(y_after - y0).max() == 0.0          # the handle's state is left unchanged
    assert abs(J[0] - J64) < (1e-12 if prec == 0 else 1e-5) * max(1.0, abs(J64))
    fd = np.array(fd)
    assert np.abs(g[0] - fd).max() < rtol * np.abs(fd).max(), (g[0], fd)


def test_vjp_matches_oracle_finite_differences():
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 5
    f, B, mu = synth.make_system(o, v)
    h, nsteps = 0.05, 20
    w = _weights(nsteps, h, 0.6, 0.3, comp=0)
    theta = np.array([0.08, 0.7, 0.4])
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-12)

    def J_oracle(th):
        fld = rk.Field(E0=th[0], omega=th[1], sigma=th[2], t0=1.0)
        _, m, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="rk4", h=h, nsteps=nsteps))
        return float(np.sum(w * m.real))

    fd = np.array([(J_oracle(theta + d) - J_oracle(theta - d)) / 2e-5 for d in 1e-5 * np.eye(3)])
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as H:
        H.set_state(0, y0, 0.0, 0.0)
        J, g = H.propagate_vjp([rtcc.make_field(E0=theta[0], omega=theta[1], sigma=theta[2], t0=1.0)], h, nsteps, w,
                               ckpt_every=25)
    assert abs(J[0] - J_oracle(theta)) < 1e-11
    assert np.abs(g[0] - fd).max() < 2e-6 * np.abs(fd).max()
    # the oracle's forward tangent differentiates the same discrete RK4 map exactly
    from oracle import tangent
    _, gt = tangent.tangent_gradient(s, y0, rk.Field(E0=theta[0], omega=theta[1], sigma=theta[2], t0=1.0), h, nsteps, w)
    assert np.abs(g[0] - gt).max() < 1e-7 * np.abs(gt).max()


def test_autograd_function_backward():
    import torch

    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 6
    f, B, mu = synth.make_system(o, v)
    h, nsteps = 0.05, 12
    w = _weights(nsteps, h, 0.4, 0.3)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as H:
        H.ground_state(tol=1e-12)
        obj = rtcc.make_objective(H, h, nsteps, w, ckpt_every=5, field_kw={"t0": 1.0})
        theta = torch.tensor([0.05, 0.5, 0.5], dtype=torch.float64, requires_grad=True)
        J = obj(theta)
        (2.0 * J).backward()
        J2, g = H.propagate_vjp([rtcc.make_field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0)], h, nsteps, w, 5)
    assert abs(J.item() - J2[0]) < 1e-14
    assert np.allclose(theta.grad.numpy(), 2.0 * g[0], rtol=1e-14, atol=0)
