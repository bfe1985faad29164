"""Seeded instance list of the batched linear-tearing scan: independent 2D
pair-plasma double Harris sheets (Sec. 2 setup, Sec. 3.1 linear tearing)
whose box length L_x, sheet half-thickness delta and magnetisation sigma are
drawn per instance; L_y = L_x / 2 and 32 particles per cell per species.

The draws come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds and a final xor-shift. Each instance takes
three consecutive outputs, reduced modulo the list lengths: L_x, then delta,
then sigma. Instance i is generated with particle seed i.

Like the rest of this package it holds no arithmetic of the method.
"""
from __future__ import annotations

from .harris import HarrisConfig

__all__ = ["splitmix64", "tearing_scan", "SCAN_LX", "SCAN_DELTA", "SCAN_SIGMA"]

SCAN_LX = (128, 192, 256, 384, 512, 768)
SCAN_DELTA = (0.5, 1.0, 2.0)
SCAN_SIGMA = (1.0, 10.0, 40.0)
_M64 = (1 << 64) - 1


def splitmix64(state: int):
    """One SplitMix64 step: returns (new state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def tearing_scan(count: int = 48, seed: int = 0, ppc: int = 32, pert: float = 1e-3, dt: float = 0.5,
                 theta_T: float = 0.3, lx_choices=SCAN_LX) -> list:
    """HarrisConfig of each instance, in draw order."""
    st = seed & _M64
    out = []
    for i in range(count):
        st, a = splitmix64(st)
        st, b = splitmix64(st)
        st, c = splitmix64(st)
        lx = lx_choices[a % len(lx_choices)]
        out.append(HarrisConfig(nx=lx, ny=lx // 2, ppc=ppc, theta_T=theta_T,
                                delta=SCAN_DELTA[b % len(SCAN_DELTA)],
                                sigma=SCAN_SIGMA[c % len(SCAN_SIGMA)], pert=pert, dt=dt, seed=i))
    return out
