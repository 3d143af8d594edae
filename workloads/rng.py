"""Counter-based random numbers: SplitMix64 (Steele, Lea and Flood 2014) plus
the Box-Muller transform.

The i-th draw of a stream with seed ``s`` is ``mix(s + (i + 1) * G)`` with
``G = 0x9E3779B97F4A7C15`` and ``mix`` the SplitMix64 finaliser, so any slice
of a stream can be produced independently and the values are the same on every
machine and numpy version.
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed, count, offset=0):
    """Return ``count`` uint64 draws of the SplitMix64 stream ``seed``,
    starting at draw ``offset``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        return _mix(z)


def stream_seed(seed, tag):
    """Derive an independent stream seed from a base seed and a string tag."""
    h = 1469598103934665603
    for ch in tag.encode():
        h = ((h ^ ch) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    with np.errstate(over="ignore"):
        return int(_mix(np.array([(seed ^ h) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0])


def uniform01(seed, count, offset=0):
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed, count):
    """Standard normal doubles by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1], so the log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:count]


def ginibre_states(seed, d, B):
    """``B`` random density matrices of size d x d, returned as a (B, d*d)
    complex128 array of row-major vectors.

    Each is G G^dagger / Tr(G G^dagger) with G a d x d Ginibre matrix whose
    entries are (N(0,1) + i N(0,1)) / sqrt(2)."""
    z = normal(seed, 2 * B * d * d).reshape(B, d, d, 2)
    G = (z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0)
    rho = G @ np.conj(np.transpose(G, (0, 2, 1)))
    tr = np.real(np.trace(rho, axis1=1, axis2=2))
    rho = rho / tr[:, None, None]
    return np.ascontiguousarray(rho.reshape(B, d * d))
