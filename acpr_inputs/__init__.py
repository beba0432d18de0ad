"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the method itself: it only draws random
numbers and spells out the workload shapes.  Everything is generated on the
host in float64 from a counter-based generator, so the same (seed, stream,
index) triple gives the same value on every machine.

Generator: the SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to a counter.  For a
triple (seed, stream, i):

    key = mix64(seed * G + stream)            (uint64 arithmetic, wraps)
    z   = mix64(key + (i + 1) * G)
    u   = (z >> 11) * 2**-53                  in [0, 1)

with G = 0x9E3779B97F4A7C15 and mix64 the SplitMix64 finaliser.  Normal
variates use Box-Muller on the pair (u[2i], u[2i+1]).

Workloads follow the paper's experiments (random "grain coarsening" initial
data, Sec. 4.2; the merging-bubbles closed form, Sec. 4.2) at the sizes the
benchmarks use.
"""
from __future__ import annotations

import dataclasses
import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids keep unrelated draws apart
STREAM_IC = 1
STREAM_WEIGHTS = 2
STREAM_BIAS = 3
STREAM_PROBLEMS = 4
STREAM_MISC = 5


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` float64 values in [0, 1) for counters offset..offset+count-1."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([seed], dtype=np.uint64) * _G + np.uint64(stream))
        idx = np.arange(offset, offset + count, dtype=np.uint64) + np.uint64(1)
        z = _mix64(key + idx * _G)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int, sigma: float = 1.0) -> np.ndarray:
    """Box-Muller normals N(0, sigma^2), float64."""
    u = uniform01(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def random_field(n: int, seed: int, amp: float = 0.9, zero_mean: bool = False) -> np.ndarray:
    """Initial datum u0 ~ U(-amp, amp) per grid point on an n x n grid (float64).

    zero_mean=True subtracts the float64 mean of the draw (the mass-conserving
    workload starts from a zero-mass field).
    """
    u = -amp + 2.0 * amp * uniform01(seed, STREAM_IC, n * n)
    u = u.reshape(n, n)
    if zero_mean:
        u = u - u.mean()
    return u


def bubbles_field(n: int, length: float = 1.0, eps: float = 0.01) -> np.ndarray:
    """Merging-bubbles datum of Sec. 4.2: the larger of tanh((0.2 - r)/eps) over
    two discs centred at (+-0.14, 0), on grid points x_i = -L/2 + i*h.
    """
    h = length / n
    x = -length / 2 + h * np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    r1 = np.sqrt((X - 0.14) ** 2 + Y ** 2)
    r2 = np.sqrt((X + 0.14) ** 2 + Y ** 2)
    a = np.tanh((0.2 - r1) / eps)
    b = np.tanh((0.2 - r2) / eps)
    return np.maximum(a, b)


def cnn_layer_dims(layers: int, channels: int):
    """(cin, cout) for each 3x3 conv of a 1 -> C -> ... -> C -> 1 stack."""
    dims = []
    for l in range(layers):
        cin = 1 if l == 0 else channels
        cout = 1 if l == layers - 1 else channels
        dims.append((cin, cout))
    return dims


def cnn_weights(layers: int, channels: int, seed: int, sigma: float = 0.01):
    """Untrained conv-stack parameters, N(0, sigma^2) for weights and biases.

    Returns (w, b) float64: w is the concatenation of W_l[cout][cin][3][3] over
    the layers, b the concatenation of b_l[cout].
    """
    dims = cnn_layer_dims(layers, channels)
    nw = sum(ci * co * 9 for ci, co in dims)
    nb = sum(co for _, co in dims)
    return normal(seed, STREAM_WEIGHTS, nw, sigma), normal(seed, STREAM_BIAS, nb, sigma)


def acnn_layer_dims(channels: int, blocks: int):
    """(cin, cout) of each convolution of the ResBlock ACNN, in parameter order:
    input conv, two per block, output conv."""
    return [(1, channels)] + [(channels, channels)] * (2 * blocks) + [(channels, 1)]


def acnn_weights(channels: int, blocks: int, seed: int, gain: float = 1.0):
    """Initial ResBlock ACNN parameters: every weight and bias of a convolution
    with fan-in 9 cin uniform in (-gain/sqrt(9 cin), gain/sqrt(9 cin)) (the usual
    default initialisation of a 3x3 convolution).  Returns (w, b) float64 in the
    concatenated layout of the network's parameters."""
    dims = acnn_layer_dims(channels, blocks)
    w, b = [], []
    ow = ob = 0
    for ci, co in dims:
        bound = gain / np.sqrt(9.0 * ci)
        w.append(bound * (2.0 * uniform01(seed, STREAM_WEIGHTS, ci * co * 9, offset=ow) - 1.0))
        b.append(bound * (2.0 * uniform01(seed, STREAM_BIAS, co, offset=ob) - 1.0))
        ow += ci * co * 9
        ob += co
    return np.concatenate(w), np.concatenate(b)


def acnn3d_weights(channels: int, blocks: int, seed: int, gain: float = 1.0):
    """Initial parameters of the ResBlock ACNN with 3 x 3 x 3 convolutions:
    uniform in (-gain/sqrt(27 cin), gain/sqrt(27 cin)) per convolution, in
    the concatenated layout W_l[cout][cin][3][3][3] / b_l[cout]."""
    dims = acnn_layer_dims(channels, blocks)
    w, b = [], []
    ow = ob = 0
    for ci, co in dims:
        bound = gain / np.sqrt(27.0 * ci)
        w.append(bound * (2.0 * uniform01(seed, STREAM_WEIGHTS, ci * co * 27, offset=ow) - 1.0))
        b.append(bound * (2.0 * uniform01(seed, STREAM_BIAS, co, offset=ob) - 1.0))
        ow += ci * co * 27
        ob += co
    return np.concatenate(w), np.concatenate(b)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One Allen-Cahn Parareal workload (all problems share these settings)."""
    name: str
    n: int
    eps: float
    S: float
    dt: float
    slices: int
    steps: int          # fine steps per slice (c)
    variant: int        # 0 classic, 1 mass-conserving
    precision: int      # 0 float64 everywhere, 1 float32 fields + bf16 conv
    layers: int
    channels: int
    act: int            # 0 tanh, 1 gelu (erf form)
    problems: int
    tol: float
    kmax: int
    zero_mean: bool
    length: float = 1.0
    seed0: int = 0
    weight_seed: int = 0
    mass_fix: int = 0   # mACNN uniform mass shift on the coarse net

    def ics(self) -> np.ndarray:
        return np.stack([random_field(self.n, self.seed0 + p, zero_mean=self.zero_mean)
                         for p in range(self.problems)])

    def weights(self):
        return cnn_weights(self.layers, self.channels, self.weight_seed)


# 64x64 classic AC in float64, 8 slices x 100 steps, tanh conv 1-16-16-16-1
PLAIN_F64_64 = Workload("ac-classic-f64-64sq-8x100", n=64, eps=0.025, S=2.0, dt=1e-4,
                        slices=8, steps=100, variant=0, precision=0, layers=4,
                        channels=16, act=0, problems=1, tol=1e-10, kmax=8,
                        zero_mean=False)

# 256x256 mass-conserving AC, 16 zero-mean ICs, 32 slices x 200 steps, gelu conv C=32 L=6
MASS_F32_256 = Workload("ac-mass-f32-256sq-16ic-32x200", n=256, eps=0.01, S=2.0, dt=5e-5,
                        slices=32, steps=200, variant=1, precision=1, layers=6,
                        channels=32, act=1, problems=16, tol=1e-6, kmax=32,
                        zero_mean=True, mass_fix=1)

# 1024x1024 classic AC, one problem, 128 slices x 500 steps, gelu conv C=64 L=8
LARGE_F32_1024 = Workload("ac-classic-f32-1024sq-128x500", n=1024, eps=0.004, S=2.0, dt=2e-5,
                          slices=128, steps=500, variant=0, precision=1, layers=8,
                          channels=64, act=1, problems=1, tol=1e-6, kmax=128,
                          zero_mean=False)


def uneven_problems(count: int = 64, seed: int = 1000):
    """Batch of independent classic-AC problems of uneven size.

    Problem p draws from seed+p: n uniform in {128, 256, 512}, slices in
    16..64, steps per slice in 50..400; eps = 2.5 h, dt = 5e-5, S = 2.
    """
    out = []
    for p in range(count):
        u = uniform01(seed + p, STREAM_PROBLEMS, 3)
        n = (128, 256, 512)[min(int(u[0] * 3), 2)]
        slices = 16 + min(int(u[1] * 49), 48)
        steps = 50 + min(int(u[2] * 351), 350)
        out.append(dict(n=n, slices=slices, steps=steps, eps=2.5 / n, dt=5e-5, S=2.0,
                        seed=seed + p))
    return out
