"""SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) in numpy, and the differential-evolution draws built on it as `tfs_de_draw`
states them: the host-side definition the device draws are checked against."""
import numpy as np

_U = np.uint64
GAMMA = 0x9E3779B97F4A7C15


def splitmix64_at(seed: int, k) -> np.ndarray:
    """The generator's output for the state after k steps from `seed` (k >= 1 gives the k-th
    output): the golden-gamma increment added k times mod 2^64, then the 64-bit finaliser."""
    with np.errstate(over="ignore"):
        z = _U(seed) + np.asarray(k, dtype=np.uint64) * _U(GAMMA)
        z = (z ^ (z >> _U(30))) * _U(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U(27))) * _U(0x94D049BB133111EB)
        return z ^ (z >> _U(31))


def de_draws(seed: int, it: int, n_chunks: int, W: int, f_lo: float, f_hi: float):
    """r1, r2 (int64 walker indices) and F (float32) of iteration `it` for n_chunks chunks of W
    walkers: a = 1 + hi32(z1) (W-1) / 2^32, b = 1 + hi32(z2) (W-2) / 2^32 skipping a, partners at
    offsets a and b from the walker within its chunk, F = f_lo + (f_hi - f_lo) u with
    u = (z3 >> 40) 2^-24, each float32 operation rounded on its own."""
    n = n_chunks * W
    with np.errstate(over="ignore"):
        k = _U(3) * (_U(it) * _U(n) + np.arange(n, dtype=np.uint64))
        z1, z2, z3 = (splitmix64_at(seed, k + _U(j)) for j in (1, 2, 3))
        a = 1 + (((z1 >> _U(32)) * _U(W - 1)) >> _U(32)).astype(np.int64)
        b = 1 + (((z2 >> _U(32)) * _U(W - 2)) >> _U(32)).astype(np.int64)
    b = b + (b >= a)
    g = np.arange(n, dtype=np.int64)
    t = g % W
    r1 = g - t + (t + a) % W
    r2 = g - t + (t + b) % W
    u = (z3 >> _U(40)).astype(np.float32) * np.float32(2.0 ** -24)
    F = np.float32(f_lo) + (np.float32(f_hi) - np.float32(f_lo)) * u
    return r1, r2, F.astype(np.float32)
