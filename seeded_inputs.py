"""Seeded synthetic inputs shared by the tests, the oracle-side scripts and bench.py.

This module holds no arithmetic of the method: it only draws numbers.  Every
input is produced by splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so the same seed gives
bit-identical arrays on every machine.

Seed convention: 1000 * workload_index + case_index.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """Return `count` successive splitmix64 outputs (uint64) for `seed`."""
    count = int(count)
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + idx * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """`count` doubles uniform in [-1, 1) from the top 53 bits of splitmix64."""
    z = splitmix64_stream(seed, count)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def random_vector(seed: int, n_total: int) -> np.ndarray:
    """I.i.d. uniform[-1, 1) entries for a whole coefficient vector."""
    return uniform_pm1(seed, n_total)


def manufactured_coefficients(seed: int) -> dict:
    """Coefficients of the seeded manufactured Stokes solution.

    The velocity is the curl of three stream functions
        psi_c = sum_{t<3} alpha[c,t] G_{a}(x) G_{b}(y) G_{c}(z),
        G_a(s) = s^2 (1-s)^2 sin(a pi s),
    and the pressure is  p = sum_{t<3} beta[t] cos(a pi x) cos(b pi y) cos(c pi z),
    with every frequency drawn from {1, 2}.  Only the numbers are drawn here.
    Returns arrays: psi_freq (3,3,3) int32, psi_amp (3,3) float64,
    p_freq (3,3) int32, p_amp (3,) float64.
    """
    z = splitmix64_stream(seed, 64)
    pos = 0

    def nxt():
        nonlocal pos
        v = int(z[pos])
        pos += 1
        return v

    def freq():
        return 1 + (nxt() >> 63)

    def amp():
        return ((nxt() >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0

    psi_freq = np.zeros((3, 3, 3), dtype=np.int32)
    psi_amp = np.zeros((3, 3), dtype=np.float64)
    for c in range(3):
        for t in range(3):
            psi_freq[c, t] = [freq(), freq(), freq()]
            psi_amp[c, t] = amp()
    p_freq = np.zeros((3, 3), dtype=np.int32)
    p_amp = np.zeros(3, dtype=np.float64)
    for t in range(3):
        p_freq[t] = [freq(), freq(), freq()]
        p_amp[t] = amp()
    return {"psi_freq": psi_freq, "psi_amp": psi_amp, "p_freq": p_freq, "p_amp": p_amp}
