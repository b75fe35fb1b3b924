"""Helpers shared by the GPU parity tests (seeded inputs, oracle references)."""
import numpy as np

from paper_2205_05175_gb300 import synth


def system(o, v, seed=synth.SEED_BASE):
    return synth.make_system(o, v, seed=seed)


def state_from(t1, t2, l1, l2):
    return np.concatenate([t1.ravel(), t2.ravel(), l1.ravel(), l2.ravel()]).astype(complex)


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
