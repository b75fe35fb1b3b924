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


@pytest.mark.parametrize("o,v", [(3, 8), (4, 24)])
def test_rhs_vjp_dot_product(o, v):
    """<u, J v> = <J^T u, v> for the right-hand side F of Eqs. derivT/derivL (holomorphic pairing,
    no conjugation), two batched trajectories under different fields.  J^T u comes from the
    library's vector-Jacobian program (rtcc_rhs_vjp); J v from the library's own right-hand side
    by the five-point stencil in a complex scalar, exact because F is at most quartic in y."""
    from paper_2205_05175_gb300 import rtcc
    from tests.gpu_common import state_from
    f, B, mu = synth.make_system(o, v)
    nz = 2
    ys, us, vs = [], [], []
    for z in range(nz):
        ys.append(state_from(*synth.random_amplitudes(o, v, seed=600 + z, s1=0.05, s2=0.02),
                             *synth.random_amplitudes(o, v, seed=610 + z, s1=0.05, s2=0.02)))
        us.append(state_from(*synth.random_amplitudes(o, v, seed=620 + z, s1=1.0, s2=1.0),
                             *synth.random_amplitudes(o, v, seed=630 + z, s1=1.0, s2=1.0)))
        vs.append(state_from(*synth.random_amplitudes(o, v, seed=640 + z, s1=1.0, s2=1.0),
                             *synth.random_amplitudes(o, v, seed=650 + z, s1=1.0, s2=1.0)))
    y, u, vv = np.stack(ys), np.stack(us), np.stack(vs)
    fields = [rtcc.make_field(E0=0.3 * (z + 1), omega=0.5, sigma=0.5, t0=1.0, pol=(0.3, 0.5, 0.8)) for z in range(nz)]
    times = np.array([0.7, 1.3])
    with rtcc.Handle(f, B, mu, o, v, ntraj=nz, prec=rtcc.P64) as H:
        ybar = H.rhs_vjp(y, fields, times, u)
        hs = 0.05
        Fs = [H.rhs(y + s * vv, fields, times) for s in (-2 * hs, -hs, hs, 2 * hs)]
    jv = (Fs[0] - 8 * Fs[1] + 8 * Fs[2] - Fs[3]) / (12 * hs)
    for z in range(nz):
        lhs = np.sum(u[z] * jv[z])
        rhs = np.sum(ybar[z] * vv[z])
        assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(lhs)), (z, lhs, rhs)
        assert abs(lhs) > 1e-2
