"""Counter-based SplitMix64 and Box-Muller normals for the initial velocity noise.

Test infrastructure (see the package docstring).

The paper initialises with a mean profile only (Sec. II.B); the seeded Gaussian
noise on top of it belongs to the synthetic workload.  Both this oracle and the
CUDA library implement the same published generator independently:

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the n-th output (n = 0, 1, ...) of a generator seeded
  with s is mix64(s + (n + 1) * gamma), gamma = 0x9E3779B97F4A7C15, where mix64 is
  the generator's published output finaliser.
* Box-Muller (Box and Muller 1958): z = sqrt(-2 ln u1) cos(2 pi u2).

Draw layout: the normal for flat cell index c and velocity component k uses the
outputs n1 = 2 (3 c + k) and n2 = n1 + 1, with u1 = ((out1 >> 11) + 1) 2^-53 in
(0, 1] and u2 = (out2 >> 11) 2^-53 in [0, 1).
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MUL1 = np.uint64(0xBF58476D1CE4E5B9)
MUL2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * MUL1
        z = (z ^ (z >> np.uint64(27))) * MUL2
    return z ^ (z >> np.uint64(31))


def splitmix64_at(seed, n):
    """Output number n (0-based) of SplitMix64 seeded with `seed`; n may be an array."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + (n + np.uint64(1)) * GAMMA
    return mix64(state)


def normal_at(seed, cell, comp):
    """Standard normal for (flat cell index, component) under the layout above."""
    cell = np.asarray(cell, dtype=np.uint64)
    n1 = np.uint64(2) * (np.uint64(3) * cell + np.uint64(comp))
    o1 = splitmix64_at(seed, n1)
    o2 = splitmix64_at(seed, n1 + np.uint64(1))
    u1 = ((o1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (o2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
