#!/usr/bin/env python
"""Benchmark of the batched RT-CCSD hot path on GB300.

Workload (default): water-hexamer-shaped closed-shell system, o=30 occupied and v=114
virtual orbitals, naux=576, seeded synthetic integrals; 12 trajectories sharing one
integral set (x/y/z polarisation x E0 in {0.001, 0.01, 0.05, 0.1} au, sine pulse
omega=0.5, sigma=0.5, t0=1), each with its own Cash-Karp step size (tol 1e-6, h0=0.01),
starting from the field-free CCSD/Lambda ground state.  One "step" is one accepted
Cash-Karp step of one trajectory (six right-hand-side evaluations of the T and Lambda
equations, the fifth-order combination, the error estimate, the controller and the
dipole); rejected attempts are part of the timed work.

value  = trajectory-steps per second, all GPUs (inputs resident in HBM).
e2e    = the same through the public C-ABI with the initial states copied from pinned
         host memory and the dipole samples copied back inside the timed region.
The reference arm (--impl reference) times the CPU oracle on a bounded sample.

--config c2|c3|c5 runs one of the accuracy / integrator / adjoint measurements instead of the
throughput line (one JSON line each):
  c2  water-dimer shape (o=10, v=38), RK4 h=0.02 for 1000 steps, E0=0.01 z sine pulse: every
      reduced-precision mode against the float64 GPU path, max|dmu(t)| and the shift of the
      absorption-spectrum peaks (zero-padded transform, parabolic peak interpolation)
  c3  water-tetramer shape (o=20, v=76), BF16x3, E0=0.5, sigma=0.3, t0=1.8, 20 au: Cash-Karp
      (tol 1e-6) against mixed-step RK4 (h=0.005 to t=3.6, then 0.05): steps, RHS evaluations,
      time and the largest dipole difference at common times
  c5  water-dimer shape, RK4 h=0.05 for 500 steps, J = sum_t w(t) mu_z(t), w Gaussian at 15 au
      (width 2 au): dJ/d(E0, omega, sigma) by the checkpointed adjoint (every 25 steps) in
      TF32 and float64 against float64 central differences (delta 1e-5)
  f1  water-dimer shape, the paper's narrowest strong pulse (E0=100, sigma=1e-6, t0=5e-6, kick
      2.5e-4 au) by mixed-step RK4 (h1=1e-7 through the pulse, then h2=0.01 to 10 au): every
      reduced mode against float64, max|dmu(t)| and the delta-kick spectrum peaks
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RT-CCSD steps/s at o=30,v=114; tensor-pipe % of peak; max |dmu(t)| vs FP64"
UNIT = "trajectory-steps/s"
WORKLOAD = "water-hexamer-shaped RT-CCSD, o={o} v={v} naux={naux}, {nz} Cash-Karp trajectories (tol 1e-6)"
E0S = (0.001, 0.01, 0.05, 0.1)
POLS = ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25      # dense tensor-core rate ratio (nominal)
PASSES = {0: 1, 1: 1, 2: 3, 3: 3}         # tensor-core passes per algorithmic product, per precision mode
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture of the same build
# (the summary and its command are in profiles/); None until such a capture exists for the shape
TRAFFIC = {}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def precision_peak(prec, bf16_sus, src):
    """Rate of one algorithmic flop in a precision mode, and where it comes from."""
    if prec == 3:
        return bf16_sus / 3.0, f"{src}: sustained bf16 cuBLAS rate / 3 (three BF16 passes per product)"
    if prec in (1, 2):
        tf = measure_tf32_tflops()
        if tf is None:
            tf, how = bf16_sus * NOMINAL_TF32_OVER_BF16, f"{src} sustained bf16 x nominal tf32/bf16 ratio 0.49"
        else:
            how = "tf32 cuBLAS rate measured in this run (8192^3, best of 10)"
        return (tf / 3.0, how + " / 3 (three TF32 passes)") if prec == 2 else (tf, how)
    f64 = measure_f64_tflops()
    return f64, "float64 cuBLAS rate measured in this run (8192^3, best of 5)"


def _matmul_tflops(dtype, n=8192, reps=10, tf32=False):
    import torch
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        torch.matmul(a, b)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        del a, b
        return 2.0 * n ** 3 / best / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old


def measure_tf32_tflops():
    try:
        import torch
        return _matmul_tflops(torch.float32, tf32=True)
    except Exception:
        return None


def measure_f64_tflops():
    import torch
    return _matmul_tflops(torch.float64, reps=5)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].isdigit():
                    rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [int(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# --- CPU oracle timing (reference arm and cpu_baseline) ------------------------------

def _omega_seconds(o, v, repeats, warmup):
    """Median wall time of the oracle's T-residual (one trajectory) at (o, v) after warm-up runs."""
    from oracle import closed, rk
    from paper_2205_05175_gb300 import synth
    f, B, mu = synth.make_system(o, v)
    s = rk.RTCC(f, B, mu, o)
    t1, t2 = synth.random_amplitudes(o, v, seed=1, s1=0.01, s2=0.005)
    for blk in ("vvvv", "ovvv", "oovv", "ovvo", "ovov", "ooov", "oovo", "oooo", "ovoo", "vvvo"):
        s.V(blk)
    for _ in range(warmup):
        closed.omega(t1, t2, s.f, s.V)
    times = []
    for _ in range(repeats):
        a = time.perf_counter()
        closed.omega(t1, t2, s.f, s.V)
        times.append(time.perf_counter() - a)
    return statistics.median(times), times


def _rhs_over_omega(o=10, v=38, repeats=3):
    """Cost of a full right-hand side (T and Lambda residuals) over a T-residual, measured at
    the dimer shape (median of `repeats` after one untimed run of each)."""
    from oracle import closed, rk
    from paper_2205_05175_gb300 import synth
    f, B, mu = synth.make_system(o, v)
    s = rk.RTCC(f, B, mu, o)
    t1, t2 = synth.random_amplitudes(o, v, seed=1, s1=0.01, s2=0.005)
    l1, l2 = synth.random_amplitudes(o, v, seed=2, s1=0.01, s2=0.005)
    closed.omega(t1, t2, s.f, s.V)
    closed.rhs(t1, t2, l1, l2, s.f, s.V)
    tom, trhs = [], []
    for _ in range(repeats):
        a = time.perf_counter()
        closed.omega(t1, t2, s.f, s.V)
        tom.append(time.perf_counter() - a)
        a = time.perf_counter()
        closed.rhs(t1, t2, l1, l2, s.f, s.V)
        trhs.append(time.perf_counter() - a)
    return statistics.median(trhs) / statistics.median(tom)


def _single_thread_omega(o, v, repeats, warmup):
    """The same T-residual timing in a child process whose BLAS runs one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "m, t = bench._omega_seconds(%d, %d, %d, %d); print(json.dumps([m, t]))" % (ROOT, o, v, repeats, warmup))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])[0]


def oracle_sample(o=30, v=114, repeats=3, warmup=1, single_thread=True):
    """Time the oracle on a bounded sample of the workload and scale it to trajectory-steps/s:
    the T-residual of one trajectory at the full shape (median of `repeats` after `warmup`
    untimed runs, BLAS on all cores) x the RHS / T-residual cost ratio measured at the dimer shape
    x 6 right-hand sides per Cash-Karp step.  With single_thread, the same T-residual is timed with
    one BLAS thread at the tetramer shape (o=20, v=76) and scaled to the full shape by the oracle's
    own flop count (tests/golden/rhs_flops.json)."""
    ratio = _rhs_over_omega()
    med, times = _omega_seconds(o, v, repeats, warmup)
    t_step = med * ratio * 6.0
    out = {"value": 1.0 / t_step, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"T-residual of one trajectory at o={o},v={v}: median {med:.2f} s of {repeats} runs "
                      f"({', '.join(f'{x:.2f}' for x in times)}) after {warmup} untimed, x RHS/T-residual cost ratio "
                      f"{ratio:.2f} (median of 3 at o=10,v=38) x 6 right-hand sides per Cash-Karp step; numpy "
                      f"complex128, BLAS threads = all {os.cpu_count()} cores"),
           "sample_seconds": med, "rhs_over_omega": ratio}
    if single_thread:
        ot, vt = 20, 76
        m1 = _single_thread_omega(ot, vt, 3, 1)
        if m1 is not None:
            fl = _flop_table()
            scale = _omega_flops(fl, o, v) / _omega_flops(fl, ot, vt)
            out["single_thread"] = {"value": 1.0 / (m1 * scale * ratio * 6.0), "unit": UNIT, "cores": 1,
                                    "sample": (f"T-residual at o={ot},v={vt} with one BLAS thread: median {m1:.2f} s "
                                               f"of 3 after 1 untimed, x {scale:.1f} (oracle flop ratio of the "
                                               f"T-residual, o={o},v={v} over o={ot},v={vt}) x {ratio:.2f} x 6")}
    return out


def _flop_table():
    return json.load(open(os.path.join(ROOT, "tests", "golden", "rhs_flops.json")))["rows"]


def _omega_flops(rows, o, v):
    return sum(c * float(o) ** p * float(v) ** q for _, ph, c, p, q in rows if ph == "omega")


def rhs_flops(o, v):
    """Algorithmic real flops of one right-hand side (T and Lambda residuals) of one trajectory:
    the oracle's per-term count (tests/golden/rhs_flops.json, written by
    tests/golden/make_rhs_flops.py) evaluated at (o, v)."""
    return sum(c * float(o) ** p * float(v) ** q for _, _, c, p, q in _flop_table())


def run_reference(args, rank, world):
    """The oracle as the reference arm.  One full trajectory step of this workload is minutes of
    CPU time, so each of the K timed steps (and each of the W untimed ones) is one bounded
    sample: the oracle's T-residual of one trajectory at the full shape.  ms_per_step is that
    sample's time; value scales it to trajectory-steps/s by the measured RHS / T-residual ratio
    and the six right-hand sides of a Cash-Karp step."""
    if rank != 0:
        return 0
    o, v = getattr(args, "o", 30), getattr(args, "v", 114)
    nz = getattr(args, "ntraj", 12)
    t0 = time.perf_counter()
    ratio = _rhs_over_omega()
    med, times = _omega_seconds(o, v, args.steps, args.warmup)
    wall = time.perf_counter() - t0
    value = 1.0 / (med * ratio * 6.0)
    sample = (f"each step is one sample: the oracle's T-residual of one trajectory at o={o},v={v} (median "
              f"{med:.2f} s over {args.steps} timed after {args.warmup} untimed), scaled to trajectory-steps/s by the "
              f"RHS/T-residual cost ratio {ratio:.2f} (o=10,v=38) and 6 right-hand sides per Cash-Karp step; numpy "
              f"complex128, BLAS threads = all {os.cpu_count()} cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "step_kind": "sample (one T-residual evaluation of one trajectory)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(o=o, v=v, naux=4 * (o + v), nz=nz), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)
    return 0


# --- GPU arm -------------------------------------------------------------------------

def dipole_error(prec: int, o=10, v=38, nsteps=50, h=0.02):
    """max |mu_prec(t) - mu_f64(t)| over an RK4 segment of the dimer-shaped system (both on the GPU)."""
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    f, B, mu = synth.make_system(o, v)
    out = {}
    for p in (rtcc.P64, prec):
        with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=p) as H:
            H.ground_state(tol=1e-10)
            _, m, n = H.propagate([rtcc.make_field(E0=0.01)], rtcc.make_integrator(rtcc.RK4, h=h, nsteps=nsteps),
                                  nsteps + 1)
            out[p] = m[0, :n[0]]
    return float(np.abs(out[prec] - out[rtcc.P64]).max())


def _peaks(om, I, count=4):
    """Largest local maxima of a sampled spectrum, refined by a parabola through three samples."""
    import numpy as np
    idx = [k for k in range(1, len(I) - 1) if I[k] > I[k - 1] and I[k] >= I[k + 1]]
    idx = sorted(idx, key=lambda k: -I[k])[:count]
    out = []
    for k in sorted(idx):
        y0, y1, y2 = I[k - 1], I[k], I[k + 1]
        den = y0 - 2 * y1 + y2
        off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        out.append(float(om[k] + off * (om[1] - om[0])))
    return out


def config_c2():
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v, h, n = 10, 38, 0.02, 1000
    f, B, mu = synth.make_system(o, v)
    fld = rtcc.make_field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.0, 1.0))
    om = np.linspace(0.05, 3.0, 6000)
    res, ref = {}, None
    for name in ("p64", "tf32", "3xtf32", "bf16x3"):
        with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.PRECISIONS[name]) as H:
            H.ground_state(tol=1e-10)
            t0 = time.perf_counter()
            t, m, k = H.propagate([fld], rtcc.make_integrator(rtcc.RK4, h=h, nsteps=n), n + 1)
            wall = time.perf_counter() - t0
        t, m = t[0, :k[0]], m[0, :k[0]]
        I = rtcc.rtcc_spectrum(t, m.real, fld, om, kappa=0.0, gamma=0.05)
        res[name] = {"t": t, "mu": m, "peaks": _peaks(om, I), "wall_s": wall}
    ref = res["p64"]
    out = {"config": "c2", "workload": "o=10 v=38 RK4 h=0.02 x1000, E0=0.01 z sine pulse", "peaks_p64": ref["peaks"],
           "wall_s_p64": round(ref["wall_s"], 3), "modes": {}}
    for name in ("tf32", "3xtf32", "bf16x3"):
        r = res[name]
        shift = max(abs(a - b) for a, b in zip(r["peaks"], ref["peaks"])) if len(r["peaks"]) == len(ref["peaks"]) else None
        out["modes"][name] = {"max_abs_dmu": float(np.abs(r["mu"] - ref["mu"]).max()), "max_peak_shift_eh": shift,
                              "wall_s": round(r["wall_s"], 3)}
    return out


def config_c3():
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v = 20, 76
    f, B, mu = synth.make_system(o, v)
    fld = rtcc.make_field(E0=0.5, omega=0.5, sigma=0.3, t0=1.8, pol=(0.0, 0.0, 1.0))
    runs = {}
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P32_BF16X3) as H:
        H.ground_state(tol=1e-8, maxiter=300)
        y0 = H.get_state(0)[0]
        for name, integ, nmax in (("cash_karp", rtcc.make_integrator(rtcc.CK, h=0.01, tol=1e-6, t_end=20.0), 20000),
                                  ("mixed_rk4", rtcc.make_integrator(rtcc.MIXED_RK4, h1=0.005, h2=0.05, t_switch=3.6,
                                                                     t_end=20.0), 20000)):
            H.set_state(0, y0, 0.0, 0.0)
            t0 = time.perf_counter()
            t, m, k = H.propagate([fld], integ, nmax)
            wall = time.perf_counter() - t0
            acc, rej, nrhs, _ = H.last_stats()
            runs[name] = {"t": t[0, :k[0]], "mu": m[0, :k[0]], "accepted": acc, "rejected": rej, "rhs": nrhs,
                          "wall_s": round(wall, 3)}
    ck, mx = runs["cash_karp"], runs["mixed_rk4"]
    # compare at the mixed-step sample times by cubic interpolation of the Cash-Karp samples
    from scipy.interpolate import CubicSpline
    sp = CubicSpline(ck["t"], ck["mu"].real, axis=0)
    sel = mx["t"] <= ck["t"][-1]
    dmu = float(np.abs(sp(mx["t"][sel]) - mx["mu"][sel].real).max())
    out = {"config": "c3", "workload": "o=20 v=76 BF16x3, E0=0.5 sigma=0.3 t0=1.8, 20 au", "max_abs_dmu_re": dmu}
    for name, r in runs.items():
        out[name] = {k: r[k] for k in ("accepted", "rejected", "rhs", "wall_s")}
        out[name]["t_end"] = float(r["t"][-1])
    return out


def config_c5():
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v, h, n, ck = 10, 38, 0.05, 500, 25
    f, B, mu = synth.make_system(o, v)
    tt = h * np.arange(n + 1)
    w = np.zeros((n + 1, 3))
    w[:, 2] = np.exp(-((tt - 15.0) ** 2) / (2 * 2.0 ** 2))
    theta = np.array([0.01, 0.5, 0.5])

    def fld(th):
        return rtcc.make_field(E0=th[0], omega=th[1], sigma=th[2], t0=1.0, pol=(0.0, 0.0, 1.0))

    out = {"config": "c5", "workload": "o=10 v=38 RK4 h=0.05 x500, checkpoints every 25, w Gaussian at 15 au"}
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P64) as H:
        H.ground_state(tol=1e-10)
        y0 = H.get_state(0)[0]

        def J(th):
            H.set_state(0, y0, 0.0, 0.0)
            t, m, k = H.propagate([fld(th)], rtcc.make_integrator(rtcc.RK4, h=h, nsteps=n), n + 1)
            return float(np.sum(w * m[0, :k[0]].real))

        t0 = time.perf_counter()
        fd = np.zeros(3)
        for i in range(3):
            e = np.zeros(3)
            e[i] = 1e-5
            fd[i] = (J(theta + e) - J(theta - e)) / 2e-5
        out["fd_wall_s"] = round(time.perf_counter() - t0, 3)
        out["grad_fd_f64"] = fd.tolist()
        for name, prec in (("f64", rtcc.P64), ("tf32", rtcc.P32_TF32)):
            with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=prec) as G:
                G.set_state(0, y0, 0.0, 0.0)
                t0 = time.perf_counter()
                _, g = G.propagate_vjp([fld(theta)], h, n, w, ckpt_every=ck)
                wall = time.perf_counter() - t0
            out[f"grad_adjoint_{name}"] = g[0].tolist()
            out[f"rel_err_adjoint_{name}_vs_fd"] = float(np.abs(g[0] - fd).max() / np.abs(fd).max())
            out[f"adjoint_wall_s_{name}"] = round(wall, 3)
    return out


def config_f1():
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v = 10, 38
    f, B, mu = synth.make_system(o, v)
    E0, sigma, t0 = 100.0, 1e-6, 5e-6          # the paper's narrowest pulse (Sec. 4.2)
    kick = E0 * sigma * np.sqrt(2.0 * np.pi)
    fld = rtcc.make_field(E0=E0, omega=0.0, sigma=sigma, t0=t0, pol=(0.0, 0.0, 1.0), carrier=rtcc.CARRIER_COS)
    integ = rtcc.make_integrator(rtcc.MIXED_RK4, h1=1e-7, h2=0.01, t_switch=2 * t0, t_end=10.0)
    om = np.linspace(0.05, 3.0, 6000)
    res = {}
    for name in ("p64", "tf32", "3xtf32", "bf16x3"):
        with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.PRECISIONS[name]) as H:
            H.ground_state(tol=1e-10)
            t0w = time.perf_counter()
            t, m, k = H.propagate([fld], integ, 4096)
            wall = time.perf_counter() - t0w
            acc = H.last_stats()[0]
        t, m = t[0, :k[0]], m[0, :k[0]]
        I = rtcc.rtcc_spectrum(t, m.real, fld, om, kappa=kick, gamma=0.05, dt=0.01)
        res[name] = {"t": t, "mu": m, "peaks": _peaks(om, I), "wall_s": round(wall, 3), "steps": acc}
    ref = res["p64"]
    out = {"config": "f1", "workload": "o=10 v=38, E0=100 sigma=1e-6 t0=5e-6 kick (Sec. 4.2), mixed RK4 h1=1e-7 to "
                                       "t=1e-5 then h2=0.01 to 10 au",
           "kick_au": kick, "steps": ref["steps"], "peaks_p64": ref["peaks"], "wall_s_p64": ref["wall_s"],
           "max_abs_mu_induced_p64": float(np.abs(ref["mu"].real - ref["mu"][0].real).max()), "modes": {}}
    for name in ("tf32", "3xtf32", "bf16x3"):
        r = res[name]
        shift = max(abs(a - b) for a, b in zip(r["peaks"], ref["peaks"])) if len(r["peaks"]) == len(ref["peaks"]) else None
        out["modes"][name] = {"max_abs_dmu": float(np.abs(r["mu"] - ref["mu"]).max()), "max_peak_shift_eh": shift,
                              "wall_s": r["wall_s"]}
    return out


def config_f3():
    """Implicit Gauss-Legendre against RK4: at RK4's step (stages by sweeps and by Newton-GMRES) and
    at a step beyond RK4's stability limit (Newton-GMRES only; RK4 diverges there): accuracy against
    a float64 RK4 run at a quarter of the short step, right-hand-side evaluations and wall time
    (dimer shape, 6 au)."""
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v, h, hl, T = 10, 38, 0.05, 0.4, 6.0
    f, B, mu = synth.make_system(o, v)
    fld = rtcc.make_field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.0, 1.0))
    n, nl = int(round(T / h)), int(round(T / hl))
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P64) as H:
        H.ground_state(tol=1e-10)
        _, mref, k = H.propagate([fld], rtcc.make_integrator(rtcc.RK4, h=h / 4, nsteps=4 * n), 4 * n + 1)
    mref = mref[0, :k[0]]
    out = {"config": "f3", "workload": f"o={o} v={v}, E0=0.01 z sine pulse, {T} au at h={h} and h={hl}; "
                                       f"reference float64 RK4 h={h / 4}", "runs": {}}
    for prec in ("p64", "bf16x3"):
        with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.PRECISIONS[prec]) as H:
            H.ground_state(tol=1e-10)
            y0 = H.get_state(0)[0]
            for name, hs, integ in (
                    ("rk4", h, rtcc.make_integrator(rtcc.RK4, h=h, nsteps=n)),
                    ("gl2", h, rtcc.make_integrator(rtcc.GL2, h=h, nsteps=n, tol=1e-6, sweeps=20)),
                    ("gl2n", h, rtcc.make_integrator(rtcc.GL2_NEWTON, h=h, nsteps=n, tol=1e-6, sweeps=2, krylov=4)),
                    ("rk4_long", hl, rtcc.make_integrator(rtcc.RK4, h=hl, nsteps=nl)),
                    ("gl2n_long", hl, rtcc.make_integrator(rtcc.GL2_NEWTON, h=hl, nsteps=nl, tol=1e-6))):
                H.set_state(0, y0, 0.0, 0.0)
                stride = int(round(4 * hs / h))
                t0 = time.perf_counter()
                try:
                    _, m, k = H.propagate([fld], integ, int(round(T / hs)) + 1)
                except rtcc.RtccError as e:
                    out["runs"][f"{name}_{prec}"] = {"status": e.status, "wall_s": round(time.perf_counter() - t0, 3)}
                    continue
                wall = time.perf_counter() - t0
                out["runs"][f"{name}_{prec}"] = {"h": hs, "max_abs_dmu": float(np.abs(m[0, :k[0]] - mref[::stride]).max()),
                                                 "rhs": H.last_stats()[2], "wall_s": round(wall, 3)}
    return out


def config_f4():
    """Pade-accelerated against plain spectra of a short record: the peaks of a 100 au record's
    transform are the reference; a 20 au record is transformed both ways (dimer shape, BF16x3,
    weak cos kick, RK4 h=0.05)."""
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v, h, T, Ts = 10, 38, 0.05, 100.0, 20.0
    f, B, mu = synth.make_system(o, v)
    E0, sigma, t0 = 0.05, 0.05, 0.3
    kick = E0 * sigma * np.sqrt(2.0 * np.pi)
    fld = rtcc.make_field(E0=E0, omega=0.0, sigma=sigma, t0=t0, pol=(0.0, 0.0, 1.0), carrier=rtcc.CARRIER_COS)
    n = int(round(T / h))
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P32_BF16X3) as H:
        H.ground_state(tol=1e-10)
        t, m, k = H.propagate([fld], rtcc.make_integrator(rtcc.RK4, h=h, nsteps=n), n + 1)
    t, m = t[0, :k[0]], m[0, :k[0]].real
    sel = t >= 2 * t0                                   # after the kick
    t, m = t[sel], m[sel]
    om = np.linspace(0.05, 3.0, 6000)
    ref = _peaks(om, rtcc.rtcc_spectrum(t, m, fld, om, kappa=kick, gamma=0.005))
    ns = int(round(Ts / h)) + 1
    a = time.perf_counter()
    Ip = rtcc.rtcc_spectrum_pade(t[:ns], m[:ns], fld, om, kappa=kick, gamma=0.005)
    wall_pade = time.perf_counter() - a
    Id = rtcc.rtcc_spectrum(t[:ns], m[:ns], fld, om, kappa=kick, gamma=0.005)

    def shift(p):
        return max(min(abs(x - y) for x in p) for y in ref) if p else None
    pp, pd = _peaks(om, Ip), _peaks(om, Id)
    return {"config": "f4", "workload": f"o={o} v={v} BF16x3, cos kick {kick:.2e} au, RK4 h={h}; reference {T} au "
                                        f"record, short record {Ts} au ({ns} samples)",
            "peaks_reference": ref, "peaks_pade_short": pp, "peaks_dft_short": pd,
            "max_peak_error_pade_eh": shift(pp), "max_peak_error_dft_eh": shift(pd), "wall_s_pade": round(wall_pade, 3)}


def config_x1():
    """The noise study of Sec. 4.1 (Fig. sp-noise) on the library's own path: a float64 monomer-
    shaped trajectory after the paper's noise-study pulse (E0 = 0.01, nu = 0.05, sigma = 0.01, cos
    carrier factor 1, 300 au), uniform noise of amplitude 10^-k added to mu_z(t), and the spectrum
    of each against the clean one (mixed-step RK4: h1 = 1e-3 through the pulse, then h2 = 0.05)."""
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v, T = 5, 19, 300.0
    f, B, mu = synth.make_system(o, v)
    E0, nu, sigma = 0.01, 0.05, 0.01
    kick = E0 * sigma * np.sqrt(2.0 * np.pi)
    fld = rtcc.make_field(E0=E0, omega=0.0, sigma=sigma, t0=nu, pol=(0.0, 0.0, 1.0), carrier=rtcc.CARRIER_COS)
    integ = rtcc.make_integrator(rtcc.MIXED_RK4, h1=1e-3, h2=0.05, t_switch=0.1, t_end=T)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P64) as H:
        H.ground_state(tol=1e-11)
        a = time.perf_counter()
        t, m, k = H.propagate([fld], integ, 8000)
        wall = time.perf_counter() - a
    t, m = t[0, :k[0]], m[0, :k[0]].real
    sel = t >= 0.1 - 1e-12
    t, m = t[sel], m[sel].copy()
    om = np.linspace(0.05, 3.0, 6000)
    I0 = rtcc.rtcc_spectrum(t, m, fld, om, kappa=kick, gamma=0.01)
    p0 = _peaks(om, I0)
    rng = np.random.Generator(np.random.PCG64(2205_05175))
    rows = {}
    for e in range(3, 9):
        eps = 10.0 ** -e
        mn = m.copy()
        mn[1:, 2] += rng.uniform(-eps, eps, len(t) - 1)
        I = rtcc.rtcc_spectrum(t, mn, fld, om, kappa=kick, gamma=0.01)
        pk = _peaks(om, I)
        shift = max(min(abs(x - y) for x in pk) for y in p0) if pk else None
        rows[f"1e-{e}"] = {"max_abs_dI_rel": float(np.abs(I - I0).max() / np.abs(I0).max()), "max_peak_shift_eh": shift}
    return {"config": "x1", "workload": f"o={o} v={v} float64, cos pulse E0={E0} nu={nu} sigma={sigma} (kick {kick:.3e} au), "
                                        f"{T} au, {len(t)} samples after the pulse",
            "wall_s": round(wall, 3), "peaks_clean": p0, "noise": rows}


def config_c4():
    """The batched configuration as specified: water-hexamer shape (o=30, v=114), 12 trajectories
    (x/y/z polarisation x E0 in {0.001, 0.01, 0.05, 0.1} au, sine pulse omega=0.5, sigma=0.5, t0=1)
    sharing one integral set, each with its own Cash-Karp step (tol 1e-6, h0 = 0.01), from the
    ground state to t = 10 au (t_end mode: trajectories that finish early leave the batch).  Reports
    trajectory-steps/s over the whole run and per-trajectory step counts.  Beside it, at the same
    shape and from the same ground state (placed at t = 0.8 au, near the pulse maximum): one
    trajectory (z, E0 = 0.1) by RK4 h = 0.05 for 4 steps in float64 and in the reduced mode, giving the float64 right-hand-side rate (the plain float64
    GPU form) and max|dmu(t)| of the reduced mode against float64."""
    import numpy as np

    from paper_2205_05175_gb300 import rtcc, synth
    o, v, T = 30, 114, 10.0
    prec = rtcc.P32_BF16X3
    f, B, mu = synth.make_system(o, v)
    fields = [rtcc.make_field(E0=e, omega=0.5, sigma=0.5, t0=1.0, pol=p) for p in POLS for e in E0S]
    nz = len(fields)
    out = {"config": "c4", "workload": f"o={o} v={v} naux={4 * (o + v)}, {nz} Cash-Karp trajectories (tol 1e-6, h0 0.01), "
                                       f"t_end {T} au, BF16x3 contractions, float64 state"}
    with rtcc.Handle(f, B, mu, o, v, ntraj=nz, prec=prec) as H:
        a = time.perf_counter()
        H.ground_state(tol=1e-8, maxiter=300)
        out["ground_state_s"] = round(time.perf_counter() - a, 2)
        y0 = H.get_state(0)[0]
        a = time.perf_counter()
        out["tuned_gemm_shapes"] = H.autotune()
        out["autotune_s"] = round(time.perf_counter() - a, 2)
        integ = rtcc.make_integrator(rtcc.CK, h=0.01, tol=1e-6, t_end=T)
        import torch
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record()
            t, m, n = H.propagate(fields, integ, 20000)
            e1.record()
            torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        acc, rej, nrhs, launches = H.last_stats()
        out.update({"seconds": secs, "accepted_steps": acc, "rejected_attempts": rej, "rhs_evaluations": nrhs,
                    "trajectory_steps_per_s": acc / secs, "trajectory_rhs_per_s": nrhs / secs,
                    "steps_per_trajectory": [int(x) - 1 for x in n],
                    "t_end_reached": [float(t[z, n[z] - 1]) for z in range(nz)], "clocks": clk.summary()})
        fl = rhs_flops(o, v)
        out["algorithmic_tflops"] = fl * nrhs / secs / 1e12
    # float64 against the reduced mode, one trajectory, same start, fixed RK4 steps
    fz = [rtcc.make_field(E0=0.1, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.0, 1.0))]
    integ = rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=4)
    res = {}
    for name, p in (("p64", rtcc.P64), ("bf16x3", prec)):
        with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=p) as H:
            H.set_state(0, y0, 0.8, 0.0)        # start near the pulse maximum
            import torch
            torch.cuda.synchronize()
            a = time.perf_counter()
            _, m, n = H.propagate(fz, integ, 8)
            secs = time.perf_counter() - a
            nr = H.last_stats()[2]
        res[name] = {"mu": m[0, :n[0]], "seconds": secs, "rhs": nr}
    out["p64_one_trajectory"] = {"seconds": round(res["p64"]["seconds"], 2), "rhs_evaluations": res["p64"]["rhs"],
                                 "trajectory_rhs_per_s": res["p64"]["rhs"] / res["p64"]["seconds"]}
    out["reduced_one_trajectory"] = {"seconds": round(res["bf16x3"]["seconds"], 2),
                                     "trajectory_rhs_per_s": res["bf16x3"]["rhs"] / res["bf16x3"]["seconds"]}
    out["speedup_batched_reduced_over_plain_f64"] = out["trajectory_rhs_per_s"] / out["p64_one_trajectory"]["trajectory_rhs_per_s"]
    out["max_abs_dmu_bf16x3_vs_f64_au"] = float(np.abs(res["bf16x3"]["mu"] - res["p64"]["mu"]).max())
    out["dmu_segment"] = "RK4 h=0.05, 4 steps from the ground state placed at t = 0.8 au, z pulse E0=0.1 (t = 0.8 .. 1.0 au)"
    return out


def run_gpu(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2205_05175_gb300 import rtcc, synth
    torch.cuda.set_device(local)
    prec = rtcc.PRECISIONS[args.prec]
    o, v = args.o, args.v
    fields = [rtcc.make_field(E0=e, omega=0.5, sigma=0.5, t0=1.0, pol=p) for p in POLS for e in E0S]
    fields = fields[:args.ntraj]     # fewer trajectories: profiling runs only (the workload has 12)
    nz = len(fields)
    f, B, mu = synth.make_system(o, v)
    t_setup = time.perf_counter()
    H = rtcc.Handle(f, B, mu, o, v, ntraj=nz, prec=prec)
    ecorr, mu0 = H.ground_state(tol=args.gs_tol, maxiter=300)
    t_setup = time.perf_counter() - t_setup
    integ = rtcc.make_integrator(rtcc.CK, h=0.01, tol=1e-6, nsteps=args.warmup)
    max_out = args.steps + args.warmup + 2
    tout = torch.zeros((nz, max_out), dtype=torch.float64, device="cuda")
    mout = torch.zeros((nz, max_out, 3, 2), dtype=torch.float64, device="cuda")
    # warm-up: W accepted steps per trajectory (continues from the ground state)
    H.propagate(fields, integ, max_out, tout, mout)
    torch.cuda.synchronize()
    # the states and times where the timed segment starts: the end-to-end run below replays it
    snap = None if args.skip_e2e else [H.get_state(z)[:2] for z in range(nz)]
    # timed region: K accepted Cash-Karp steps of every trajectory, every launch timed by CUDA events
    integ = rtcc.make_integrator(rtcc.CK, h=0.01, tol=1e-6, nsteps=args.steps)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        H.profile_start()
        torch.cuda.nvtx.range_push("rtcc_timed")
        ev0.record()
        H.propagate(fields, integ, max_out, tout, mout)
        ev1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        prof = H.profile_stop()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    acc, rej, nrhs, launches = H.last_stats()
    ms_max = reduce_max(ms, world)
    value = world * acc / (ms_max / 1e3)
    # dominant kernel (largest total device time in the timed region)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    hbm, bf16, bf16_sus, src = measured_peaks()
    alg_rhs = rhs_flops(o, v)
    if dom == "tc_gemm":
        # algorithmic flops: the oracle's per-term count of one right-hand side x the trajectory
        # right-hand sides evaluated in the timed region, over the tensor-core GEMM's device time;
        # the peak is the rate of one algorithmic flop in this precision (a third of the sustained
        # bf16 rate for the three BF16x3 passes; TF32 measured by cuBLAS on this GPU)
        peak, psrc = precision_peak(prec, bf16_sus, src)
        roof = {"bound": "tensor", "achieved": alg_rhs * nrhs / (d["ms"] / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "algorithmic_flops_per_rhs": alg_rhs, "rhs_evaluations": nrhs,
                "executed_tflops": d["flops"] / (d["ms"] / 1e3) / 1e12,
                "executed_frac_of_bf16_sustained": d["flops"] / (d["ms"] / 1e3) / 1e12 / bf16_sus,
                "executed_over_algorithmic": d["flops"] / max(1.0, alg_rhs * nrhs) / PASSES[prec],
                "peak_source": psrc}
    elif dom == "f64_gemm":
        peak, psrc = precision_peak(prec, bf16_sus, src)
        roof = {"bound": "alu", "achieved": alg_rhs * nrhs / (d["ms"] / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "algorithmic_flops_per_rhs": alg_rhs, "rhs_evaluations": nrhs, "peak_source": psrc}
    else:
        roof = {"bound": "hbm", "achieved": d["bytes"] / (d["ms"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": f"{src} copy bandwidth"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC.get((o, v, nz, args.prec))
    roof["kernel"] = dom
    roof["launches"] = d["launches"]
    roof["avg_launch_ms"] = d["ms"] / max(1, d["launches"])
    share = {k: round(prof[k]["ms"] / max(1e-9, sum(p["ms"] for p in prof.values())), 4) for k in prof}
    if args.skip_e2e:
        acc_e2e, ms_e2e, h2d, d2h = acc, ms_max, 0.0, 0.0
    else:
        # end to end: the same segment again (same start states and times, same steps), with the
        # start states copied in from pinned host memory and the dipoles copied back to the host
        # inside the timed region
        yh = torch.from_numpy(np.stack([sn[0] for sn in snap]).view(np.float64)).pin_memory()
        tz = [sn[1] for sn in snap]
        snap = None
        th = np.zeros((nz, max_out))
        mh = np.zeros((nz, max_out, 3), complex)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for z in range(nz):
            H.set_state(z, yh[z].numpy().view(np.complex128), tz[z], 0.0)
        H.propagate(fields, integ, max_out, th, mh)
        e1.record()
        torch.cuda.synchronize()
        ms_e2e = reduce_max(e0.elapsed_time(e1), world)
        acc_e2e = H.last_stats()[0]
        h2d = yh.numel() * 8 / max(1, acc_e2e)
        d2h = (th.nbytes + mh.nbytes) / max(1, acc_e2e)
    H.close()
    line = None
    if rank == 0:
        derr = dipole_error(prec) if not args.skip_dipole_error else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / max(1, acc / nz), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
                "config": {"workload": WORKLOAD.format(o=o, v=v, naux=4 * (o + v), nz=nz), "o": o, "v": v, "naux": 4 * (o + v), "trajectories_per_gpu": nz,
                           "precision": args.prec, "accepted_steps": acc, "rejected_attempts": rej,
                           "rhs_evaluations": nrhs, "l2": "inputs larger than L2 (state 4.5 GB, vvvv 1.35 GB)",
                           "parallelism": f"replicas x{world}", "ground_state_setup_s": round(t_setup, 2),
                           "e_corr": ecorr},
                "roofline": roof, "kernel_share": share,
                "e2e": {"value": world * acc_e2e / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clk.summary(),
                "dipole_error_vs_f64": {"value": derr, "unit": "au",
                                        "config": "o=10,v=38, RK4 h=0.02, 50 steps, E0=0.01 z sine pulse"}}
        if not args.skip_cpu_baseline and world == 1:
            line["cpu_baseline"] = oracle_sample()
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["p64", "tf32", "3xtf32", "bf16x3"])
    ap.add_argument("--o", type=int, default=30)
    ap.add_argument("--v", type=int, default=114)
    ap.add_argument("--ntraj", type=int, default=12, help="trajectories (the workload has 12; fewer for profiling)")
    ap.add_argument("--gs-tol", type=float, default=1e-8)
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-dipole-error", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--config", default=None, choices=["c2", "c3", "c4", "c5", "f1", "f3", "f4", "x1"],
                    help="run an accuracy / integrator / adjoint measurement instead of the throughput line")
    args = ap.parse_args(argv)
    if args.config is not None:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "config": args.config,
                              "unavailable": "configuration runs compare the library's own precision modes"}))
            return 0
        line = {"c2": config_c2, "c3": config_c3, "c4": config_c4, "c5": config_c5, "f1": config_f1, "f3": config_f3,
                "f4": config_f4, "x1": config_x1}[args.config]()
        print(json.dumps(line), flush=True)
        return 0
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_gpu(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
