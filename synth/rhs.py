"""Seeded right-hand sides (boundary potentials on the panels)."""
import numpy as np

_MASK = (1 << 64) - 1


def _splitmix64_stream(count: int, seed: int) -> np.ndarray:
    """``count`` outputs of Vigna's SplitMix64 generator started from ``seed``
    (state += 0x9E3779B97F4A7C15; two xor-shift-multiply rounds; final xor-shift)."""
    out = np.empty(count, dtype=np.uint64)
    s = seed & _MASK
    for k in range(count):
        s = (s + 0x9E3779B97F4A7C15) & _MASK
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out[k] = z ^ (z >> 31)
    return out


def splitmix64_uniform(count: int, seed: int) -> np.ndarray:
    """Uniform doubles in [0,1) from the top 53 bits of each SplitMix64 output."""
    z = _splitmix64_stream(count, seed)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def splitmix64_normal(count: int, seed: int) -> np.ndarray:
    """Standard normal doubles by Box-Muller on consecutive uniform pairs
    (u1 mapped to (0,1] so the logarithm is finite)."""
    m = (count + 1) // 2
    u = splitmix64_uniform(2 * m, seed)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def rhs_constant(mesh, value: float = 1.0) -> np.ndarray:
    """phi_i = value on every panel (unit-potential conductor)."""
    return np.full(mesh.n, float(value))


def rhs_one_plus_half_z(mesh) -> np.ndarray:
    """phi_i = 1 + 0.5 * z_i at each collocation point."""
    return 1.0 + 0.5 * mesh.centroid[:, 2]


def rhs_two_spheres(mesh) -> np.ndarray:
    """+1 on the first half of the panels (sphere 1), -1 on the second (sphere 2)."""
    n = mesh.n
    b = np.ones(n)
    b[n // 2:] = -1.0
    return b


def rhs_normal_columns(n: int, nrhs: int, seed: int = 20191101) -> np.ndarray:
    """N(0,1) panel potentials, column-major (n, nrhs): all of column 0 first."""
    z = splitmix64_normal(n * nrhs, seed)
    return np.asfortranarray(z.reshape(nrhs, n).T)
