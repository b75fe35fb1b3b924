"""Parity at the full benchmark shape (o=30, v=114, naux=576) in the launch configuration the
benchmark times: 12 trajectories batched in one handle, BF16x3 contractions, one right-hand side
(Eqs. derivT/derivL) for every trajectory in one call, states and results resident on the device,
and the dipole (Eq. dipole) of the last trajectory.

The oracle evaluates the last trajectory of the batch in full (about a minute of CPU and 20 GB of
host memory); the first slot is given the same state, field and time, so its output must equal
the last slot's, which checks both ends of the batch layout against the oracle.  The other ten
slots carry distinct inputs and must give finite, distinct outputs.

Tolerance: a BF16x3 product drops only the lo*lo term (relative 2^-16 per product) and
accumulates in float32; over contraction lengths up to v^2 = 12996 the expected relative error of
the residual is a few 1e-5 of its largest element, and 2e-4 leaves room for the cancellation
between terms while any indexing error gives O(1)."""
import numpy as np
import pytest

from oracle import closed, rk
from paper_2205_05175_gb300 import synth
from tests.gpu_common import rel_err, state_from, system

pytestmark = [pytest.mark.gpu, pytest.mark.last]

O, V, NTRAJ = 30, 114, 12
TOL = 2e-4
POLS = ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))


def _available_host_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return float("inf")


def test_rhs_parity_hexamer_shape_twelve_trajectories():
    if _available_host_gb() < 32:
        pytest.skip("the oracle's full-shape right-hand side needs about 21 GB of host memory")
    import torch

    from paper_2205_05175_gb300 import rtcc
    f, B, mu = system(O, V)
    t1, t2 = synth.random_amplitudes(O, V, seed=301, s1=0.01, s2=0.005)
    l1, l2 = synth.random_amplitudes(O, V, seed=302, s1=0.01, s2=0.005)
    base = state_from(t1, t2, l1, l2)
    last = NTRAJ - 1
    slot = [last] + list(range(1, NTRAJ))          # slot 0 repeats the inputs of slot 11
    scale = [1.0 + 0.02 * z for z in slot]
    E0 = [0.01 * (1 + z // 3) for z in slot]
    pol = [POLS[z % 3] for z in slot]
    times = np.array([0.7 + 0.05 * z for z in slot])
    fields = [rtcc.make_field(E0=E0[k], omega=0.5, sigma=0.5, t0=1.0, pol=pol[k]) for k in range(NTRAJ)]
    base_d = torch.from_numpy(base.view(np.float64)).cuda()
    ys = torch.stack([base_d * s for s in scale])
    with rtcc.Handle(f, B, mu, O, V, ntraj=NTRAJ, prec=rtcc.P32_BF16X3) as h:
        out = h.rhs(ys, fields, times)
        h.set_state(last, base * scale[last])
        dip = h.dipole()[last]
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    got = out[last].cpu().numpy().view(np.complex128)
    fld = rk.Field(E0=E0[last], omega=0.5, sigma=0.5, t0=1.0, pol=pol[last])
    ref = rk.RTCC(f, B, mu, O).rhs(float(times[last]), base * scale[last], fld)
    assert rel_err(got, ref) < TOL, rel_err(got, ref)
    peak = float(out[last].abs().max())
    assert float((out[0] - out[last]).abs().max()) < 1e-5 * peak
    for k in range(1, last):
        assert float((out[k] - out[last]).abs().max()) > 1e-3 * peak, k
    # Eq. dipole through the density program; these random amplitudes put |mu| near 5 au, so the
    # bound is relative (same error model as above)
    sc = scale[last]
    ref_mu = closed.dipole(t1 * sc, t2 * sc, l1 * sc, l2 * sc, mu, O)
    assert np.abs(dip - ref_mu).max() < 1e-4 * np.abs(ref_mu).max(), np.abs(dip - ref_mu).max()
