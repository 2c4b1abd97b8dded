"""splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators", 2014),
the counter-based generator used wherever the method needs deterministic "random" numbers:
aggregation priorities (distance-2 MIS) and the power-iteration start vector.  Written from
the published definition; the CUDA side implements the same definition independently.

Pinned by tests/test_oracle_amg.py against the published first outputs of the generator
seeded with 0 (values reproduced in tests/golden/splitmix64.txt).
"""
import numpy as np

_M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(x):
    """The splitmix64 output function applied to counter values ``x`` (uint64 array or int):
    z = x + golden; z = (z ^ z>>30) * C1; z = (z ^ z>>27) * C2; return z ^ z>>31 (mod 2^64)."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(GOLDEN))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


# salts that separate the streams used by different steps / levels
SALT_MIS = 0x4D495332  # 'MIS2'
SALT_POWER = 0x504F5752  # 'POWR'


def mis_keys(n, level):
    """Unique 64-bit priorities of the n nodes of an aggregation level: the top 31 bits of a
    hash followed by the node index (+1 so that 0 stays free as the 'no candidate' value)."""
    i = np.arange(n, dtype=np.uint64)
    h = splitmix64(i + np.uint64((SALT_MIS << 24) + (level << 40)))
    return ((h >> np.uint64(33)) << np.uint64(32)) + i + np.uint64(1)


def unit_uniform(n, salt):
    """n numbers in [-0.5, 0.5): (splitmix64(i + salt) >> 11) * 2^-53 - 0.5."""
    i = np.arange(n, dtype=np.uint64)
    h = splitmix64(i + np.uint64(salt))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5
