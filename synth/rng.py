"""Counter-based random numbers: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a hash of
(seed, stream, counter).  Every draw is addressed by its counter, so the values
do not depend on vectorisation order or on the machine."""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of one named random stream under a seed."""
    with np.errstate(over="ignore"):
        s = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * np.uint64(stream + 1))
    return np.uint64(s)


def bits(seed: int, stream: int, counter) -> np.ndarray:
    """64 random bits for each counter (uint64 array)."""
    key = stream_key(seed, stream)
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + (c + np.uint64(1)) * _GOLDEN)


def uniform(seed: int, stream: int, counter) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    b = bits(seed, stream, counter) >> np.uint64(11)
    return (b.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, counter) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform; each counter uses two
    uniforms (counters 2c and 2c+1 of the stream)."""
    c = np.asarray(counter, dtype=np.uint64)
    u1 = uniform(seed, stream, c * np.uint64(2))
    u2 = uniform(seed, stream, c * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
